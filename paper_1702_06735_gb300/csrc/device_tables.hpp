// Plain-old-data tables shared between the host library and the kernels.
#pragma once
#include <cstdint>

#include "model.hpp"

namespace tdmix {

// Model structure as the kernels read it (device global memory, written once).
struct DevModel {
  int U, NO, NB, NR, NS, NX, n_chains, n_params;
  int chain_comp[kMaxChains];
  int chain_amp[kMaxChains];
  int res_shape[kMaxRes];
  int res_L[kMaxRes];
  double res_ma[kMaxRes], res_mb[kMaxRes];
  double r_res, r_parent, gamma;
  int term_spin[kMaxTerms];
  int term_parts[kMaxTerms][4];
  int splane_mask[kMaxSPlanes];
  int xplane_s[kMaxXPlanes];
  int xplane_L[kMaxXPlanes];
  double xplane_ma[kMaxXPlanes], xplane_mb[kMaxXPlanes];
};

// Per-evaluation constants derived from the parameter vector on the device.
struct EvalConst {
  double m0[kMaxRes], g0[kMaxRes], m2[kMaxRes];
  double kappa[kMaxRes];     // m0 Gamma(s) = kappa * X(s)
  double dk_dm[kMaxRes], dk_dg[kMaxRes];
  float m2_hi[kMaxRes], m2_lo[kMaxRes], kappa_f[kMaxRes];
  double cA[kMaxComp][2], cB[kMaxComp][2];   // coefficient of each component in A_f, Abar_f
  float cAf[kMaxComp][2], cBf[kMaxComp][2];
  double x, y, gamma;
  double alpha, beta, gc, dc;                 // time-integral weights of |A|^2, |Abar|^2, Re, Im
  float alpha_f, beta_f, gc_f, dc_f;
  int status;                                 // tdmix_status of the parameter check
};

// Device view of one event sample (data or phase-space MC).
struct SampleDev {
  int64_t n, pitch;
  void* s;            // invariants: fp64 [NS][pitch]; fp32 [2][NS][pitch] (hi, lo)
  void* x;            // width factors X(s) [NX][pitch]
  void* k;            // spin x barrier factors [U*NO][pitch]
  const double* t;    // decay times (data)
  const void* w;      // event weights (MC) or null
  void* cache;        // per-event components [2][U][pitch] (data)
};

// Layout of one block-partial row.
struct RowLayout {
  // MC rows
  static constexpr int mc_sumw = 0;
  static int mc_gre(int U) { return 1; }                 // U*U, upper triangle used
  static int mc_gim(int U) { return 1 + U * U; }
  static int mc_s1(int U) { return 1 + 2 * U * U; }
  static int mc_s2(int U, int NR) { return 1 + 2 * U * U + NR; }
  static int mc_width(int U, int NR) { return 1 + 2 * U * U + 2 * NR; }
  // data rows
  static constexpr int d_lnb = 0, d_bad = 1, d_gx = 2, d_gy = 3;
  static int d_ga(int U) { return 4; }                    // [re U][im U]
  static int d_gb(int U) { return 4 + 2 * U; }
  static int d_s1(int U) { return 4 + 4 * U; }
  static int d_s2(int U, int NR) { return 4 + 4 * U + NR; }
  static int d_width(int U, int NR) { return 4 + 4 * U + 2 * NR; }
};

// Result vector written by the final kernel: [nll, N, n_bad, sum ln B, grad...]
constexpr int kResHeader = 4;

}  // namespace tdmix
