// Amplitude-model description and its compilation into the tables the
// kernels use.  Host code only.
//
// A model (Sec. 3) is a list of resonances and a list of decay chains; each
// chain belongs to A_f (direct decay) or Abar_f (decay after mixing, Sec. 2)
// and is built from a spin factor with its barrier (form) factors, one or two
// lineshapes and, with two identical final-state particles, the
// Bose-symmetrised sum over both orderings.  Compilation removes recurring
// building blocks, as the paper's time-dependent model does on creation:
//   * components:   chains with the same topology, resonances and particle
//                   assignment share one per-event amplitude a_j;
//   * lineshapes:   one Breit-Wigner per distinct (resonance, invariant);
//   * invariants:   one s plane per distinct set of final-state particles;
//   * width planes: one per distinct (s plane, daughter masses, L).
#pragma once
#include <string>
#include <vector>

namespace tdmix {

enum SpinType { SPIN_VV_S = 0, SPIN_VV_P = 1, SPIN_VV_D = 2, SPIN_AP_S = 3, SPIN_NR = 4 };
enum ShapeType { SHAPE_MDW = 0, SHAPE_CONST = 1, SHAPE_NONE = 2 };

constexpr int kMaxRes = 16;
constexpr int kMaxComp = 16;
constexpr int kMaxOrder = 2;
constexpr int kMaxTerms = kMaxComp * kMaxOrder;
constexpr int kMaxBW = 32;
constexpr int kMaxSPlanes = 16;
constexpr int kMaxXPlanes = 16;
constexpr int kMaxChains = 64;

struct ResonanceDef {
  std::string name;
  double mass = 0, width = 0;
  int shape = SHAPE_MDW;
  int L = 0;
  double ma = 0, mb = 0;  // nominal daughter masses of the width (MDW)
  bool floating = true;
};

struct ChainDef {
  std::string name;
  int amp = 0;  // 0: A_f, 1: Abar_f
  int spin = SPIN_NR;
  std::vector<int> res;
  int parts[4] = {0, 1, 2, 3};
  double cre = 0, cim = 0;
  bool floating = true;
};

struct Term {           // one ordering o of one component j
  int spin;
  int parts[4];         // particle indices (a, b, c, d) after the ordering
  int b[2];             // Breit-Wigner instance per slot, -1 if none
};

struct BWInstance {
  int res;
  int splane;
  int xplane;           // -1 unless the resonance has a mass-dependent width
};

struct XPlane {
  int splane;
  double ma, mb;
  int L;
};

struct CompiledModel {
  std::string name;
  double parent_mass = 0;
  double masses[4] = {0, 0, 0, 0};
  double tau = 0, r_res = 1.5, r_parent = 5.0;
  int bose[2] = {-1, -1};
  double x = 0, y = 0;
  bool float_xy = true;
  // Gaussian decay-time resolution (ps); 0: none.  An extension the paper
  // leaves out (Sec. 4); evaluated by the runtime-table kernels.
  double sigma_t = 0;
  // Background (an extension the paper leaves out, Sec. 4): a fraction of
  // the data events flat in phase space with an exponential decay time of
  // lifetime bkg_tau; evaluated by the runtime-table kernels.
  double bkg_fraction = 0, bkg_tau = 1;
  bool dedup = true;
  std::vector<ResonanceDef> res;
  std::vector<ChainDef> chains;

  int U = 0, NO = 1;
  std::vector<int> chain_comp;        // component of each chain
  std::vector<Term> terms;            // U * NO, index j * NO + o
  std::vector<BWInstance> bws;
  std::vector<int> splane_mask;       // bit mask of final-state particles
  std::vector<XPlane> xplanes;

  int n_params() const { return 2 * int(chains.size()) + 2 * int(res.size()) + 2; }
  int NB() const { return int(bws.size()); }
  int NS() const { return int(splane_mask.size()); }
  int NX() const { return int(xplanes.size()); }
  int NR() const { return int(res.size()); }
  // Structural signature: equal signatures mean identical kernel tables.
  std::string signature() const;
  std::vector<double> default_params() const;
  std::vector<int> floating_mask() const;
};

// Throws std::runtime_error with a readable message on invalid input.
CompiledModel compile_model(const std::string& json_text);

}  // namespace tdmix
