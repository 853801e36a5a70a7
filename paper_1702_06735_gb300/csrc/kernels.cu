// Model-independent kernels: kinematic precompute (once per event load),
// per-evaluation constants, and the final fixed-order reduction that forms
// the normalisation, the NLL and its gradient.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "device_tables.hpp"
#include "kernels.hpp"
#include "kinematics.cuh"

namespace tdmix {

// ---------------------------------------------------------------------------
// Kinematic precompute (one thread per event, fp64): invariants s, width
// factors X(s) = q^(2L+1) F_L(q r)^2 / sqrt(s) and the spin x barrier factor
// K_{j,o} of every component ordering.  None depends on fit parameters.
// ---------------------------------------------------------------------------
template <bool F32>
__global__ void __launch_bounds__(256) k_precompute(Momenta mom, int64_t n, int64_t pitch,
                                                    const DevModel* __restrict__ dm, void* s_out,
                                                    void* x_out, void* k_out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  V4 p[4];
  for (int a = 0; a < 4; ++a)
    p[a] = {__ldg(mom.p[a][0] + i), __ldg(mom.p[a][1] + i), __ldg(mom.p[a][2] + i), __ldg(mom.p[a][3] + i)};
  const int NS = dm->NS, NX = dm->NX, NT = dm->U * dm->NO;
  double sv[kMaxSPlanes];
  for (int sp = 0; sp < NS; ++sp) {
    V4 P = {0, 0, 0, 0};
    const int mask = dm->splane_mask[sp];
    for (int a = 0; a < 4; ++a)
      if (mask & (1 << a)) P = P + p[a];
    const double s = dot(P, P);
    sv[sp] = s;
    if (F32) {
      float hi = float(s);
      float lo = float(s - double(hi));
      static_cast<float*>(s_out)[sp * pitch + i] = hi;
      static_cast<float*>(s_out)[(NS + sp) * pitch + i] = lo;
    } else {
      static_cast<double*>(s_out)[sp * pitch + i] = s;
    }
  }
  for (int xp = 0; xp < NX; ++xp) {
    const double s = sv[dm->xplane_s[xp]];
    const int L = dm->xplane_L[xp];
    const double ma = dm->xplane_ma[xp], mb = dm->xplane_mb[xp];
    const double q2 = breakup2(s, ma * ma, mb * mb);
    const double q = sqrt(q2);
    double qp = q;
    for (int l = 0; l < L; ++l) qp *= q2;
    const double F = barrier(L, q2 * dm->r_res * dm->r_res);
    const double X = qp * F * F / sqrt(s);
    if (F32) static_cast<float*>(x_out)[xp * pitch + i] = float(X);
    else static_cast<double*>(x_out)[xp * pitch + i] = X;
  }
  for (int t = 0; t < NT; ++t) {
    const int* pt = dm->term_parts[t];
    const double K = spin_barrier(dm->term_spin[t], p[pt[0]], p[pt[1]], p[pt[2]], p[pt[3]], dm->r_res,
                                  dm->r_parent);
    if (F32) static_cast<float*>(k_out)[t * pitch + i] = float(K);
    else static_cast<double*>(k_out)[t * pitch + i] = K;
  }
}

void launch_precompute(bool f32, const Momenta& mom, int64_t n, int64_t pitch, const DevModel* dm, void* s_out,
                       void* x_out, void* k_out, cudaStream_t st) {
  if (n <= 0) return;
  const int threads = 256;
  const unsigned blocks = unsigned((n + threads - 1) / threads);
  if (f32) k_precompute<true><<<blocks, threads, 0, st>>>(mom, n, pitch, dm, s_out, x_out, k_out);
  else k_precompute<false><<<blocks, threads, 0, st>>>(mom, n, pitch, dm, s_out, x_out, k_out);
}

// Fixed-order sum of a vector (one block).
__global__ void __launch_bounds__(1024) k_sum(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
  __shared__ double part[1024];
  double a = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += v[i];
  part[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

void launch_sum(const double* v, int64_t n, double* out, cudaStream_t st) {
  k_sum<<<1, 1024, 0, st>>>(v, n, out);
}

__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = float(in[i]);
}

void launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  k_to_f32<<<unsigned((n + 255) / 256), 256, 0, st>>>(in, out, n);
}

// ---------------------------------------------------------------------------
// Per-evaluation constants from the parameter vector (one thread).
// ---------------------------------------------------------------------------
__device__ inline double dlnF_dz(int L, double z) {
  if (L == 0) return 0.0;
  if (L == 1) return -0.5 / (1.0 + z);
  return -0.5 * (3.0 + 2.0 * z) / (9.0 + 3.0 * z + z * z);
}

// Threads work in parallel: thread k checks parameter k, thread c places
// chain c's coefficient, thread r derives resonance r's constants.
__global__ void __launch_bounds__(64) k_prepare(const double* __restrict__ params, const DevModel* __restrict__ dm,
                                                EvalConst* __restrict__ ec) {
  __shared__ int st_nonfinite, st_domain;
  const int tid = threadIdx.x;
  const int nc = dm->n_chains, NR = dm->NR, U = dm->U, np = dm->n_params;
  if (tid == 0) st_nonfinite = st_domain = 0;
  __syncthreads();
  for (int k = tid; k < np; k += blockDim.x)
    if (!isfinite(params[k])) atomicOr(&st_nonfinite, 1);
  for (int j = tid; j < U; j += blockDim.x) ec->cA[j][0] = ec->cA[j][1] = ec->cB[j][0] = ec->cB[j][1] = 0.0;
  __syncthreads();
  for (int c = tid; c < nc; c += blockDim.x) {
    const int j = dm->chain_comp[c];
    double(*dst)[2] = dm->chain_amp[c] == 0 ? ec->cA : ec->cB;
    dst[j][0] = params[2 * c];
    dst[j][1] = params[2 * c + 1];
  }
  const double r2 = dm->r_res * dm->r_res;
  for (int r = tid; r < NR; r += blockDim.x) {
    const double m0 = params[2 * nc + 2 * r], g0 = params[2 * nc + 2 * r + 1];
    const int shape = dm->res_shape[r];
    ec->m0[r] = m0;
    ec->g0[r] = g0;
    ec->m2[r] = m0 * m0;
    double kap = 0, dkm = 0, dkg = 0;
    if (shape != SHAPE_NONE && !(m0 > 0 && g0 > 0)) atomicOr(&st_domain, 1);
    if (shape == SHAPE_CONST) {
      kap = m0 * g0;
      dkm = g0;
      dkg = m0;
    } else if (shape == SHAPE_MDW) {
      const int L = dm->res_L[r];
      const double a = dm->res_ma[r] * dm->res_ma[r], b = dm->res_mb[r] * dm->res_mb[r];
      const double u = m0 * m0;
      const double q02 = breakup2(u, a, b);
      if (!(q02 > 0)) atomicOr(&st_domain, 1);
      const double q0 = sqrt(q02);
      double q0p = q0;
      for (int l = 0; l < L; ++l) q0p *= q02;
      const double z0 = q02 * r2;
      const double F = barrier(L, z0);
      kap = u * g0 / (q0p * F * F);
      // d q0^2 / d m0 = 2 m0 (u^2 - (a - b)^2) / (4 u^2)
      const double dq2 = 2.0 * m0 * (u * u - (a - b) * (a - b)) / (4.0 * u * u);
      const double dlnk = 2.0 / m0 - (2 * L + 1) * dq2 / (2.0 * q02) - 2.0 * dlnF_dz(L, z0) * r2 * dq2;
      dkm = kap * dlnk;
      dkg = kap / g0;
    }
    ec->kappa[r] = kap;
    ec->dk_dm[r] = dkm;
    ec->dk_dg[r] = dkg;
    const float hi = float(m0 * m0);
    ec->m2_hi[r] = hi;
    ec->m2_lo[r] = float(m0 * m0 - double(hi));
    ec->kappa_f[r] = float(kap);
  }
  if (tid == 0) {
    const double x = params[2 * nc + 2 * NR], y = params[2 * nc + 2 * NR + 1];
    if (!(fabs(y) < 1.0)) atomicOr(&st_domain, 1);
    const double gamma = dm->gamma;
    const double a = 1.0 / (1.0 - y * y), c = 1.0 / (1.0 + x * x);
    ec->x = x;
    ec->y = y;
    ec->gamma = gamma;
    ec->alpha = a + c;
    ec->beta = (x * x + y * y) * a * c;
    ec->gc = y * a;
    ec->dc = x * c;
    ec->alpha_f = float(ec->alpha);
    ec->beta_f = float(ec->beta);
    ec->gc_f = float(ec->gc);
    ec->dc_f = float(ec->dc);
  }
  __syncthreads();
  for (int j = tid; j < U; j += blockDim.x) {
    ec->cAf[j][0] = float(ec->cA[j][0]); ec->cAf[j][1] = float(ec->cA[j][1]);
    ec->cBf[j][0] = float(ec->cB[j][0]); ec->cBf[j][1] = float(ec->cB[j][1]);
  }
  if (tid == 0) ec->status = st_nonfinite ? -5 : (st_domain ? -6 : 0);
}

void launch_prepare(const double* params, const DevModel* dm, EvalConst* ec, cudaStream_t st) {
  k_prepare<<<1, 64, 0, st>>>(params, dm, ec);
}

// ---------------------------------------------------------------------------
// Final kernel: sums block rows in fixed order and forms
//   N = <alpha |A|^2 + beta |Abar|^2 - 2 gc Re(A Abar*) - 2 dc Im(A Abar*)> / Gamma
// (Eq. (mix) integrated over t in [0, inf), averaged over the MC sample),
//   NLL = -sum ln B + Gamma sum t + N_d ln N,
// and the gradient.  Result: [nll, N, n_bad, sum ln B, grad...].
// ---------------------------------------------------------------------------
constexpr int kFinalThreads = 256;
constexpr int kFinalColsPerBlock = kFinalThreads / 32;
constexpr int kMaxMcWidth = 1 + kMaxComp * kMaxComp + 2 * kMaxRes;
constexpr int kMaxDataWidth = 4 + 4 * kMaxComp + 2 * kMaxRes;

// Final kernel, many blocks: warp c of the grid sums column c of the block
// partials (MC columns first when an MC pass ran, then data columns); lane l
// takes rows l, l + 32, ... in order and a fixed shuffle tree combines the
// lanes.  The last block to finish (atomic counter) then forms
//   N = <alpha |A|^2 + beta |Abar|^2 - 2 gc Re(A Abar*) - 2 dc Im(A Abar*)> / Gamma
// (Eq. (mix) integrated over t in [0, inf), averaged over the MC sample),
//   NLL = -sum ln B + Gamma sum t + N_d ln N,
// and the gradient.  Result: [nll, N, n_bad or status, sum ln B, grad...].
__global__ void __launch_bounds__(kFinalThreads) k_final(FinalArgs fa, int wmc, int wd) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nmc = fa.mc_part ? wmc : 0;
  const int col = blockIdx.x * kFinalColsPerBlock + warp;
  if (col < nmc + wd) {
    const double* src;
    int n;
    if (col < nmc) {
      src = fa.mc_part + int64_t(col) * fa.mc_ld;
      n = fa.n_mc_rows;
    } else {
      src = fa.data_part + int64_t(col - nmc) * fa.data_ld;
      n = fa.n_data_rows;
    }
    double a = 0;
    for (int r = lane; r < n; r += 32) a += src[r];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) fa.colsum[col] = a;
  }
  __threadfence();
  __syncthreads();
  __shared__ unsigned last;
  if (threadIdx.x == 0) last = atomicAdd(fa.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();

  const DevModel* dm = fa.dm;
  const EvalConst* ec = fa.ec;
  const int U = dm->U, NR = dm->NR, nc = dm->n_chains, np = dm->n_params;
  const int NRE = U * (U + 1) / 2, NIM = U * (U - 1) / 2;
  const int tid = threadIdx.x;
  __shared__ double mcs[kMaxMcWidth];
  __shared__ double ds[kMaxDataWidth];
  __shared__ double Ire[kMaxComp * kMaxComp], Iim[kMaxComp * kMaxComp];
  __shared__ double vA[kMaxComp][2], vB[kMaxComp][2];
  __shared__ double sh[8];  // AA, BB, Xr, Xi, nbar
  for (int v = tid; v < wmc; v += blockDim.x) {
    if (fa.mc_part) {
      mcs[v] = __ldcg(fa.colsum + v);
      fa.gram_store[v] = mcs[v];
    } else {
      mcs[v] = fa.gram_store[v];
    }
  }
  for (int v = tid; v < wd; v += blockDim.x) ds[v] = __ldcg(fa.colsum + nmc + v);
  if (tid == 0) *fa.counter = 0u;
  __syncthreads();
  const double sw = mcs[0];
  for (int e = tid; e < U * U; e += blockDim.x) {
    const int j = e / U, k = e % U;
    const int lo = j < k ? j : k, hi = j < k ? k : j;
    // compact index of (lo, hi) in the row-major upper triangle
    const int ire = lo * U - lo * (lo - 1) / 2 + (hi - lo);
    const int iim = lo * (U - 1) - lo * (lo - 1) / 2 + (hi - lo - 1);
    Ire[e] = mcs[1 + ire] / sw;
    Iim[e] = j == k ? 0.0 : (j < k ? 1.0 : -1.0) * mcs[1 + NRE + iim] / sw;
  }
  __syncthreads();
  double* res = fa.result;
  const int timed_out = *fa.err;
  const int status = timed_out ? -7 : ec->status;
  __syncthreads();
  if (tid == 0 && timed_out) *fa.err = 0;
  if (status != 0) {
    for (int k = tid; k < kResHeader + np; k += blockDim.x) res[k] = k == 2 ? double(status) : nan("");
    return;
  }
  // vA = I cA, vB = I cB (thread j)
  for (int j = tid; j < U; j += blockDim.x) {
    double ar = 0, ai = 0, br = 0, bi = 0;
    for (int k = 0; k < U; ++k) {
      const double ir = Ire[j * U + k], ii = Iim[j * U + k];
      ar += ir * ec->cA[k][0] - ii * ec->cA[k][1];
      ai += ir * ec->cA[k][1] + ii * ec->cA[k][0];
      br += ir * ec->cB[k][0] - ii * ec->cB[k][1];
      bi += ir * ec->cB[k][1] + ii * ec->cB[k][0];
    }
    vA[j][0] = ar; vA[j][1] = ai; vB[j][0] = br; vB[j][1] = bi;
  }
  __syncthreads();
  const double al = ec->alpha, be = ec->beta, gc = ec->gc, dc = ec->dc, x = ec->x, y = ec->y;
  const double gamma = ec->gamma;
  const double Nd = double(fa.n_data);
  if (tid == 0) {
    double AA = 0, BB = 0, Xr = 0, Xi = 0;
    for (int j = 0; j < U; ++j) {
      AA += ec->cA[j][0] * vA[j][0] + ec->cA[j][1] * vA[j][1];   // Re(cA^dagger I cA)
      BB += ec->cB[j][0] * vB[j][0] + ec->cB[j][1] * vB[j][1];
      Xr += ec->cB[j][0] * vA[j][0] + ec->cB[j][1] * vA[j][1];   // cB^dagger I cA = <A Abar*>
      Xi += ec->cB[j][0] * vA[j][1] - ec->cB[j][1] * vA[j][0];
    }
    const double nbar = al * AA + be * BB - 2.0 * gc * Xr - 2.0 * dc * Xi;
    const double N = nbar / gamma;
    const double sum_lnb = ds[0];
    const double nbad = ds[1];
    double nll = -sum_lnb + gamma * fa.sum_t + Nd * log(N);
    if (nbad > 0 || !(N > 0)) nll = nan("");
    res[0] = nll;
    res[1] = N;
    res[2] = nbad;
    res[3] = sum_lnb;
    sh[0] = AA; sh[1] = BB; sh[2] = Xr; sh[3] = Xi; sh[4] = nbar;
  }
  __syncthreads();
  if (!fa.want_grad) return;
  const double AA = sh[0], BB = sh[1], Xr = sh[2], Xi = sh[3], nbar = sh[4];
  const double sc = Nd / nbar;  // d(N_d ln N) = N_d dnbar / nbar
  // data columns: [sum ln B, n_bad, d/dx, d/dy, Re gA, Im gA, Re gB, Im gB, s1, s2]
  for (int c = tid; c < nc; c += blockDim.x) {
    const int j = dm->chain_comp[c];
    double dnr, dni, gr, gi;
    if (dm->chain_amp[c] == 0) {
      dnr = 2 * al * vA[j][0] - 2 * gc * vB[j][0] + 2 * dc * vB[j][1];
      dni = 2 * al * vA[j][1] - 2 * gc * vB[j][1] - 2 * dc * vB[j][0];
      gr = ds[4 + j];
      gi = ds[4 + U + j];
    } else {
      dnr = 2 * be * vB[j][0] - 2 * gc * vA[j][0] - 2 * dc * vA[j][1];
      dni = 2 * be * vB[j][1] - 2 * gc * vA[j][1] + 2 * dc * vA[j][0];
      gr = ds[4 + 2 * U + j];
      gi = ds[4 + 3 * U + j];
    }
    // d sum ln B / d Re c = 2 Re(g), d / d Im c = -2 Im(g)
    res[kResHeader + 2 * c] = fa.floating[2 * c] ? -(2 * gr) + sc * dnr : 0.0;
    res[kResHeader + 2 * c + 1] = fa.floating[2 * c + 1] ? -(-2 * gi) + sc * dni : 0.0;
  }
  for (int r = tid; r < NR; r += blockDim.x) {
    const double m0 = ec->m0[r];
    double dm_n = 0, dg_n = 0, dm_d = 0, dg_d = 0;
    if (fa.have_res_grad) {
      const double s1m = mcs[1 + NRE + NIM + r], s2m = mcs[1 + NRE + NIM + NR + r];
      dm_n = (-4 * m0 * s1m - 2 * ec->dk_dm[r] * s2m) / sw;
      dg_n = (-2 * ec->dk_dg[r] * s2m) / sw;
      const double s1d = ds[4 + 4 * U + r], s2d = ds[4 + 4 * U + NR + r];
      dm_d = -4 * m0 * s1d - 2 * ec->dk_dm[r] * s2d;
      dg_d = -2 * ec->dk_dg[r] * s2d;
    }
    const int k = 2 * nc + 2 * r;
    res[kResHeader + k] = fa.floating[k] ? -dm_d + sc * dm_n : 0.0;
    res[kResHeader + k + 1] = fa.floating[k + 1] ? -dg_d + sc * dg_n : 0.0;
  }
  if (tid == 0) {
    const double a = 1.0 / (1.0 - y * y), c = 1.0 / (1.0 + x * x);
    const double dal_dx = -2 * x * c * c, dal_dy = 2 * y * a * a;
    const double dbe_dx = 2 * x * c * c, dbe_dy = 2 * y * a * a;
    const double dgc_dy = (1 + y * y) * a * a, ddc_dx = (1 - x * x) * c * c;
    const double dn_dx = dal_dx * AA + dbe_dx * BB - 2 * ddc_dx * Xi;
    const double dn_dy = dal_dy * AA + dbe_dy * BB - 2 * dgc_dy * Xr;
    const int k = 2 * nc + 2 * NR;
    res[kResHeader + k] = fa.floating[k] ? -ds[2] + sc * dn_dx : 0.0;
    res[kResHeader + k + 1] = fa.floating[k + 1] ? -ds[3] + sc * dn_dy : 0.0;
  }
}

void launch_final(const FinalArgs& fa, int mc_width, int data_width, cudaStream_t st) {
  const int cols = (fa.mc_part ? mc_width : 0) + data_width;
  const int blocks = (cols + kFinalColsPerBlock - 1) / kFinalColsPerBlock;
  k_final<<<blocks, kFinalThreads, 0, st>>>(fa, mc_width, data_width);
}

}  // namespace tdmix
