// Pseudo-event generation on the GPU (Sec. 3.1: flat phase-space points,
// then time-dependent pseudo-events by accept/reject on the model).
//
// Every candidate has an index c and draws only from Philox4x32-10 at the
// counter (c lo, c hi, stream, d) for draw word d (key: the seed), so a
// candidate is the same whichever thread or batch draws it:
//   * flat four-body phase space by GENBOD (F. James, CERN 68-15): the two
//     intermediate masses of (p0 p1) and (p0 p1 p2) from sorted uniforms,
//     kept with probability (product of the three breakup momenta) / (its
//     maximum); isotropic two-body decays boosted into the parent frame
//     (the try decided in single precision with a band, double precision
//     inside it; momenta built in double precision where they are kept);
//   * a decay time t ~ Exp(lambda), lambda = (1 - |y|) Gamma;
//   * the time-dependent rate R = e^{-Gamma t} B (Eq. (mix), factorised, in
//     double precision) from the event's invariants, width factors and
//     spin x barrier factors (the same double-precision kinematics as the
//     event loader) and the model at the given parameters;
//   * acceptance if u env < R e^{lambda t} (env: the envelope).
// The weight is first formed in single precision (this GPU runs its FP32
// pipe about 64 times faster than its FP64 one) with an error band of
// 1e-3 of the weight plus 1e-4 of its cancellation-free scale (hundreds of
// times the single-precision error); only candidates whose u env falls
// inside the band are decided on the double-precision weight, so the
// decisions are those of the double-precision rate (a flag turns the
// pre-screen off; tests compare the two samples bit for bit).
// Pass 1 evaluates candidates and writes one accept bit each (a warp's 32
// consecutive candidates form one word), the accepted count of every block
// and the largest weight R e^{lambda t}; pass 2 regenerates the accepted
// candidates of each block and writes them, in candidate order, at the
// block's offset, so the output does not depend on scheduling.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "eval.cuh"
#include "fused.cuh"
#include "kinematics.cuh"
#include "philox.cuh"

namespace tdmix {

constexpr int kGenThreads = 256;
constexpr int kGenIters = 16;                           // candidates per thread per batch
constexpr int kGenPerBlock = kGenThreads * kGenIters;   // contiguous candidates of one block
constexpr int kGenMaxTries = 64;                        // GENBOD tries per candidate

struct GenArgs {
  ModelConst km;
  double hp[kMaxParams];     // parameters (host values)
  const DevModel* dm;        // structure tables of the kinematics
  double mD, m[4], tecm, inv_wtmax;
  double lambda;             // decay-time proposal rate (1 - |y|) Gamma
  double env;                // envelope; 0 in the pilot (nothing accepted)
  uint32_t key0, key1, stream;
  int flat;                  // 1: flat phase space only (every GENBOD point accepted)
  int prescreen;             // 1: single-precision weight first (see above)
  int64_t cand0;             // first candidate of this batch
  uint32_t* mask;            // pass 1: [batch / 32] accept bits
  uint32_t* block_count;     // pass 1: [grid] accepted per block
  unsigned long long* wmax;  // pass 1: largest weight (bits of a non-negative double)
  const int64_t* block_pos;  // pass 2: [grid] output position of each block's first accepted event
  double* p_out;             // pass 2: [16][ld] planes (particle a, component c at (4a + c) ld)
  double* t_out;             // pass 2: decay times (may be null)
  int64_t ld, out_end;       // plane stride; positions >= out_end are not written
};

// The random draws of one candidate: draw word d of its counter gives two
// doubles in [0, 1) (d = 0: decay time and acceptance; d = 1: the Gaussian
// of a decay-time resolution; d = 8 + 5 try + j: GENBOD try `try`).
struct CandRng {
  uint32_t c0, c1, stream, k0, k1;
  __device__ double2 pair(uint32_t d) const {
    const Philox4 r = philox4x32_10(Philox4{{c0, c1, stream, d}}, k0, k1);
    return make_double2(u01(r.v[0], r.v[1]), u01(r.v[2], r.v[3]));
  }
};

template <class T>
__device__ __forceinline__ T breakup(T M, T a, T b) {
  const T s = M * M;
  const T l = (s - (a + b) * (a + b)) * (s - (a - b) * (a - b));
  return l > 0 ? sqrt(l) / (T(2) * M) : T(0);
}

template <class T>
__device__ __forceinline__ V4T<T> boost(V4T<T> p, T bx, T by, T bz) {
  const T b2 = bx * bx + by * by + bz * bz;
  const T g = T(1) / sqrt(T(1) - b2);
  const T bp = bx * p.x + by * p.y + bz * p.z;
  const T k = b2 > 0 ? (g - T(1)) / b2 * bp + g * p.e : T(0);
  return V4T<T>{g * (p.e + bp), p.x + k * bx, p.y + k * by, p.z + k * bz};
}

// GENBOD weight of try `tr` of a candidate in precision T: the product of
// the three breakup momenta over its maximum, from the try's two sorted
// mass uniforms; u_acc is the try's acceptance uniform.
template <class T>
__device__ __forceinline__ T genbod_weight(const GenArgs& a, const CandRng& rng, int tr, double& u_acc) {
  const uint32_t d0 = 8u + 5u * uint32_t(tr);
  const double2 u0 = rng.pair(d0), u1 = rng.pair(d0 + 1);
  u_acc = u1.x;
  const T ra = T(fmin(u0.x, u0.y)), rb = T(fmax(u0.x, u0.y));
  const T m0 = T(a.m[0]), m1 = T(a.m[1]), m2 = T(a.m[2]), m3 = T(a.m[3]), te = T(a.tecm);
  const T M1 = m0 + m1 + ra * te, M2 = m0 + m1 + m2 + rb * te;
  return breakup(M1, m0, m1) * breakup(M2, M1, m2) * breakup(T(a.mD), M2, m3) * T(a.inv_wtmax);
}

// Breakup momentum from the factors of the Kallen function, with the
// threshold factor given directly: M - a - b = gap (no cancellation).
__device__ __forceinline__ float breakup_gap(float M, float a, float b, float gap) {
  const float l = gap * (M + a + b) * (M - a + b) * (M + a - b);
  return sqrtf(fmaxf(l, 0.f)) / (2.f * M);
}

// The GENBOD weight of try `tr` in single precision: the three mass gaps
// ra, rb - ra, 1 - rb (in units of the kinetic energy) are taken in double
// precision and rounded once, and each breakup momentum comes from the
// factored Kallen function, so the weight is within a few float roundings
// (about 1e-6 relative) of its double-precision value even next to a
// threshold, where M^2 - (a + b)^2 would cancel.
__device__ __forceinline__ float genbod_weight_f(const GenArgs& a, const CandRng& rng, int tr, double& u_acc) {
  const uint32_t d0 = 8u + 5u * uint32_t(tr);
  const double2 u0 = rng.pair(d0), u1 = rng.pair(d0 + 1);
  u_acc = u1.x;
  const double rad = fmin(u0.x, u0.y), rbd = fmax(u0.x, u0.y);
  const float te = float(a.tecm);
  const float g1 = float(rad) * te, g2 = float(rbd - rad) * te, g3 = float(1.0 - rbd) * te;
  const float m0 = float(a.m[0]), m1 = float(a.m[1]), m2 = float(a.m[2]), m3 = float(a.m[3]);
  const float M1 = m0 + m1 + float(rad) * te, M2 = m0 + m1 + m2 + float(rbd) * te;
  return breakup_gap(M1, m0, m1, g1) * breakup_gap(M2, M1, m2, g2) * breakup_gap(float(a.mD), M2, m3, g3) *
         float(a.inv_wtmax);
}

// The first accepted GENBOD try of a candidate (-1 if all kGenMaxTries
// fail).  Each try's weight is formed in single precision (genbod_weight_f)
// with a band of 1e-5 of it (about ten times its rounding error); a try
// whose uniform falls inside the band is decided on the double-precision
// weight, so the try found is the one double precision finds.
__device__ inline int genbod_try(const GenArgs& a, const CandRng& rng) {
  for (int tr = 0; tr < kGenMaxTries; ++tr) {
    double u;
    const float w = genbod_weight_f(a, rng, tr, u);
    const double lo = double(w) * (1.0 - 1e-5), hi = double(w) * (1.0 + 1e-5);
    if (u < lo) return tr;
    if (u >= hi) continue;
    double u64;
    if (u < genbod_weight<double>(a, rng, tr, u64)) return tr;
  }
  return -1;
}

// Momenta of GENBOD try `tr` (accepted) in precision T: isotropic two-body
// decays of (p0 p1), then p2 against (p0 p1), p3 against (p0 p1 p2), each
// subsystem boosted into the next one's rest frame, ending in the parent's.
template <class T>
__device__ inline void genbod_momenta(const GenArgs& a, const CandRng& rng, int tr, V4T<T> (&p)[4]) {
  const uint32_t d0 = 8u + 5u * uint32_t(tr);
  const double2 u0 = rng.pair(d0), u1 = rng.pair(d0 + 1), u2 = rng.pair(d0 + 2), u3 = rng.pair(d0 + 3),
                u4 = rng.pair(d0 + 4);
  const T ra = T(fmin(u0.x, u0.y)), rb = T(fmax(u0.x, u0.y));
  const T m[4] = {T(a.m[0]), T(a.m[1]), T(a.m[2]), T(a.m[3])};
  const T te = T(a.tecm);
  const T M1 = m[0] + m[1] + ra * te, M2 = m[0] + m[1] + m[2] + rb * te;
  const T q1 = breakup(M1, m[0], m[1]), q2 = breakup(M2, M1, m[2]), q3 = breakup(T(a.mD), M2, m[3]);
  const double ang[6] = {u1.y, u2.x, u2.y, u3.x, u3.y, u4.x};
  T dir[3][3];
  for (int j = 0; j < 3; ++j) {
    const T ct = T(2) * T(ang[2 * j]) - T(1), st = sqrt(fmax(T(0), T(1) - ct * ct));
    T sp, cp;
    sincospi(T(2) * T(ang[2 * j + 1]), &sp, &cp);
    dir[j][0] = st * cp;
    dir[j][1] = st * sp;
    dir[j][2] = ct;
  }
  p[0] = V4T<T>{sqrt(q1 * q1 + m[0] * m[0]), q1 * dir[0][0], q1 * dir[0][1], q1 * dir[0][2]};
  p[1] = V4T<T>{sqrt(q1 * q1 + m[1] * m[1]), -q1 * dir[0][0], -q1 * dir[0][1], -q1 * dir[0][2]};
  const T qs[2] = {q2, q3}, Ms[2] = {M1, M2};
  for (int j = 0; j < 2; ++j) {
    const T q = qs[j];
    const T e = sqrt(q * q + Ms[j] * Ms[j]);
    const T bx = -q / e * dir[j + 1][0], by = -q / e * dir[j + 1][1], bz = -q / e * dir[j + 1][2];
    for (int i = 0; i <= j + 1; ++i) p[i] = boost(p[i], bx, by, bz);
    p[j + 2] = V4T<T>{sqrt(q * q + m[j + 2] * m[j + 2]), q * dir[j + 1][0], q * dir[j + 1][1], q * dir[j + 1][2]};
  }
}

// Register source of an event's precomputed quantities for EventCore.
template <class S>
struct RegSrc {
  const double* sv;
  const double* xv;
  const double* kv;
  __device__ __forceinline__ double s_hi(int sp) const { return sv[sp]; }
  __device__ __forceinline__ double x(int xp) const { return xv[xp]; }
  __device__ __forceinline__ double k(int t) const { return kv[t]; }
};

// e^{-Gamma t} B of one event from its momenta (double precision).
template <class S>
__device__ inline double event_rate(const DevModel* __restrict__ dm, const BlockConst<double>& bc, const V4 (&p)[4],
                                    double t) {
  constexpr int NS = S::NS > 0 ? S::NS : 1, NX = S::NX > 0 ? S::NX : 1, NT = S::U * S::NO;
  double sv[NS], xv[NX], kv[NT];
#pragma unroll
  for (int sp = 0; sp < S::NS; ++sp) {
    V4 P = {0, 0, 0, 0};
    const int mask = dm->splane_mask[sp];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (mask & (1 << q)) P = P + p[q];
    sv[sp] = dot(P, P);
  }
#pragma unroll
  for (int xp = 0; xp < S::NX; ++xp) {
    const double s = sv[dm->xplane_s[xp]];
    const int L = dm->xplane_L[xp];
    const double ma = dm->xplane_ma[xp], mb = dm->xplane_mb[xp];
    const double q2 = breakup2(s, ma * ma, mb * mb);
    const double q = sqrt(q2);
    double qp = q;
    for (int l = 0; l < L; ++l) qp *= q2;
    const double F = barrier(L, q2 * dm->r_res * dm->r_res);
    xv[xp] = qp * F * F / sqrt(s);
  }
#pragma unroll
  for (int tm = 0; tm < NT; ++tm) {
    const int* pt = dm->term_parts[tm];
    kv[tm] = spin_barrier(dm->term_spin[tm], p[pt[0]], p[pt[1]], p[pt[2]], p[pt[3]], dm->r_res, dm->r_parent);
  }
  const RegSrc<S> src{sv, xv, kv};
  EventCore<PrecF64, S> ev;
  ev.lineshapes(src, bc);
  ev.components(src);
  double Ar, Ai, Br, Bi;
  ev.amplitudes(bc, Ar, Ai, Br, Bi);
  const unsigned long long tb = static_cast<unsigned long long>(__double_as_longlong(t));
  const int tier = tb <= bc.tlim[0] ? 0 : (tb <= bc.tlim[1] ? 1 : 2);
  double cha, sha, cb, sb;
  mixing_trig(bc.hy * t, bc.hx * t, tier, cha, sha, cb, sb);
  const double chr = cha * cb, chi = sha * sb, shr = sha * cb, shi = cha * sb;
  const double Zr = chr * Ar - chi * Ai - (shr * Br - shi * Bi);
  const double Zi = chr * Ai + chi * Ar - (shr * Bi + shi * Br);
  return exp(-bc.gamma * t) * 2.0 * (Zr * Zr + Zi * Zi);
}

// Single-precision source of an event's precomputed quantities (no lo parts).
template <class S>
struct RegSrcF {
  const float* sv;
  const float* xv;
  const float* kv;
  __device__ __forceinline__ float s_hi(int sp) const { return sv[sp]; }
  __device__ __forceinline__ float s_lo(int) const { return 0.0f; }
  __device__ __forceinline__ float x(int xp) const { return xv[xp]; }
  __device__ __forceinline__ float k(int t) const { return kv[t]; }
};

// The acceptance weight R e^{lambda t} = 2 |Z|^2 e^{-|y| Gamma t} of one
// candidate in single precision (kinematics, lineshapes, components,
// amplitudes and Z), and a band that contains the double-precision weight:
// 2 e^{-|y| Gamma t} (1e-3 |Z|^2 + 1e-4 S_Z^2), S_Z = cosh|w| S_A + sinh|w| S_B
// the magnitude the rounding errors of Z scale with (see ill_conditioned).
template <class S>
__device__ inline void event_weight_f32(const DevModel* __restrict__ dm, const BlockConst<float>& bc,
                                        const V4T<float> (&q)[4], double t, float& w, float& band) {
  constexpr int NS = S::NS > 0 ? S::NS : 1, NX = S::NX > 0 ? S::NX : 1, NT = S::U * S::NO;
  float sv[NS], xv[NX], kv[NT];
#pragma unroll
  for (int sp = 0; sp < S::NS; ++sp) {
    V4T<float> P = {0.f, 0.f, 0.f, 0.f};
    const int mask = dm->splane_mask[sp];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (mask & (1 << i)) P = P + q[i];
    sv[sp] = dot(P, P);
  }
  const float rr = float(dm->r_res), rD = float(dm->r_parent);
#pragma unroll
  for (int xp = 0; xp < S::NX; ++xp) {
    const float s = sv[dm->xplane_s[xp]];
    const int L = dm->xplane_L[xp];
    const float ma = float(dm->xplane_ma[xp]), mb = float(dm->xplane_mb[xp]);
    const float q2 = breakup2(s, ma * ma, mb * mb);
    float qp = sqrtf(q2);
    for (int l = 0; l < L; ++l) qp *= q2;
    const float F = barrier(L, q2 * rr * rr);
    xv[xp] = qp * F * F / sqrtf(s);
  }
#pragma unroll
  for (int tm = 0; tm < NT; ++tm) {
    const int* pt = dm->term_parts[tm];
    kv[tm] = spin_barrier(dm->term_spin[tm], q[pt[0]], q[pt[1]], q[pt[2]], q[pt[3]], rr, rD);
  }
  const RegSrcF<S> src{sv, xv, kv};
  EventCore<PrecF32, S> ev;
  float sc[S::U];
  ev.lineshapes(src, bc);
  ev.template components<true>(src, sc);
  float Ar, Ai, Br, Bi;
  ev.template amplitudes<true>(bc, Ar, Ai, Br, Bi);
  float SA = 0.f, SB = 0.f;
#pragma unroll
  for (int j = 0; j < S::U; ++j) {
    const Quad<float> C = bc.cab[j];
    SA = fmaf(fabsf(C.x) + fabsf(C.y), sc[j], SA);
    SB = fmaf(fabsf(C.z) + fabsf(C.w), sc[j], SB);
  }
  const float tg = bc.gammaf * float(t);
  const float a = 0.5f * bc.yf * tg, b = 0.5f * bc.xf * tg;
  float cha, sha, cb, sb, chw, shw, c0, s0;
  mixing_trig_f32(a, b, cha, sha, cb, sb);
  mixing_trig_f32(fabsf(a) + fabsf(b), 0.f, chw, shw, c0, s0);
  const float cr = cha * cb, ci = sha * sb, sr = sha * cb, si = cha * sb;
  const float Zr = cr * Ar - ci * Ai - (sr * Br - si * Bi);
  const float Zi = cr * Ai + ci * Ar - (sr * Bi + si * Br);
  const float SZ = chw * SA + shw * SB;
  const float f = 2.0f * expf(-fabsf(bc.yf) * tg);
  const float z2 = Zr * Zr + Zi * Zi;
  w = f * z2;
  band = f * (1e-3f * z2 + 1e-4f * SZ * SZ);
}

template <class S>
__device__ inline void gen_prologue(const GenArgs& a, CtaConst& cc, BlockConst<double>& bc, BlockConst<float>& bf) {
  derive_load<double, S::U>(nullptr, a.hp, a.km, cc, bc);
  __syncthreads();
  derive_compute<double, S::U, S::NR>(a.km, cc, bc);
  __syncthreads();
  derive_load<float, S::U>(nullptr, a.hp, a.km, cc, bf);
  __syncthreads();
  derive_compute<float, S::U, S::NR>(a.km, cc, bf);
  __syncthreads();
}

template <class S>
// Two blocks per SM (128 registers, a little spilled): 6 % more candidates per
// second than one block at 160 registers for the full model; the pass is bound
// by instruction fetch and latency, which the extra warps hide.
__global__ void __launch_bounds__(kGenThreads, 2) k_gen_pass1(const __grid_constant__ GenArgs a) {
  __shared__ CtaConst cc;
  __shared__ BlockConst<double> bc;
  __shared__ BlockConst<float> bf;
  __shared__ uint32_t s_count;
  __shared__ unsigned long long s_wmax;
  const int tid = threadIdx.x, lane = tid & 31;
  if (!a.flat) gen_prologue<S>(a, cc, bc, bf);
  if (tid == 0) {
    s_count = 0;
    s_wmax = 0;
  }
  __syncthreads();
  uint32_t my_count = 0;
  double my_wmax = 0.0;
  for (int it = 0; it < kGenIters; ++it) {
    const int64_t local = int64_t(it) * kGenThreads + tid;  // within the block
    const int64_t c = a.cand0 + int64_t(blockIdx.x) * kGenPerBlock + local;
    const CandRng rng{uint32_t(c), uint32_t(uint64_t(c) >> 32), a.stream, a.key0, a.key1};
    const int tr = genbod_try(a, rng);
    bool acc = tr >= 0;
    if (acc && !a.flat) {
      const double2 u = rng.pair(0);
      const double t = -log1p(-u.x) / a.lambda;
      const double thr = u.y * a.env;
      bool decided = false;
      if (a.prescreen) {
        V4T<float> pf[4];
        genbod_momenta<float>(a, rng, tr, pf);
        float w32, band;
        event_weight_f32<S>(a.dm, bf, pf, t, w32, band);
        const double hi = double(w32) + double(band);
        // decided in single precision unless u env lies in the band, or the
        // weight could exceed the envelope (the violation check uses exact
        // weights; the pilot, which sets the envelope, runs without the
        // pre-screen)
        if (hi <= a.env) {
          if (thr < double(w32) - double(band)) {
            acc = decided = true;
          } else if (thr > hi) {
            acc = false;
            decided = true;
          }
        }
      }
      if (!decided) {
        V4 p[4];
        genbod_momenta<double>(a, rng, tr, p);
        const double w = event_rate<S>(a.dm, bc, p, t) * exp(a.lambda * t);
        my_wmax = fmax(my_wmax, w);
        acc = thr < w;
      }
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, acc);
    if (lane == 0) a.mask[(int64_t(blockIdx.x) * kGenPerBlock + local) / 32] = bits;
    my_count += acc ? 1u : 0u;
  }
  atomicAdd(&s_count, my_count);
  atomicMax(&s_wmax, static_cast<unsigned long long>(__double_as_longlong(my_wmax)));
  __syncthreads();
  if (tid == 0) {
    a.block_count[blockIdx.x] = s_count;
    atomicMax(a.wmax, s_wmax);
  }
}

template <class S>
__global__ void __launch_bounds__(kGenThreads) k_gen_pass2(const __grid_constant__ GenArgs a) {
  __shared__ uint32_t s_warp_base[kGenThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int64_t pos = a.block_pos[blockIdx.x];
  for (int it = 0; it < kGenIters; ++it) {
    const int64_t local = int64_t(it) * kGenThreads + tid;
    const uint32_t bits = a.mask[(int64_t(blockIdx.x) * kGenPerBlock + local) / 32];
    // exclusive prefix of the accepted counts of the block's warps, in order
    if (lane == 0) s_warp_base[warp] = __popc(bits);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kGenThreads / 32; ++w) {
      const uint32_t n = s_warp_base[w];
      before += w < warp ? n : 0u;
      total += n;
    }
    __syncthreads();
    if ((bits >> lane) & 1u) {
      const int64_t o = pos + before + __popc(bits & ((1u << lane) - 1u));
      if (o < a.out_end) {
        const int64_t c = a.cand0 + int64_t(blockIdx.x) * kGenPerBlock + local;
        const CandRng rng{uint32_t(c), uint32_t(uint64_t(c) >> 32), a.stream, a.key0, a.key1};
        V4 p[4];
        genbod_momenta<double>(a, rng, genbod_try(a, rng), p);  // the try pass 1 found
        for (int q = 0; q < 4; ++q) {
          a.p_out[(4 * q + 0) * a.ld + o] = p[q].e;
          a.p_out[(4 * q + 1) * a.ld + o] = p[q].x;
          a.p_out[(4 * q + 2) * a.ld + o] = p[q].y;
          a.p_out[(4 * q + 3) * a.ld + o] = p[q].z;
        }
        if (a.t_out) {
          double t = a.flat ? 0.0 : -log1p(-rng.pair(0).x) / a.lambda;
          if (!a.flat && a.km.sigma_t > 0) {
            // a decay-time resolution: the measured time is the accepted true
            // time plus a Gaussian of width sigma_t (Box-Muller, draw word 1)
            const double2 u = rng.pair(1);
            t += a.km.sigma_t * sqrt(-2.0 * log1p(-u.x)) * cospi(2.0 * u.y);
          }
          a.t_out[o] = t;
        }
      }
    }
    pos += total;
  }
}

}  // namespace tdmix
