// Pseudo-event generation on the GPU (Sec. 3.1: flat phase-space points,
// then time-dependent pseudo-events by accept/reject on the model).
//
// Every candidate has an index c and draws only from Philox4x32-10 at the
// counter (c lo, c hi, stream, d) for draw word d (key: the seed), so a
// candidate is the same whichever thread or batch draws it:
//   * flat four-body phase space by GENBOD (F. James, CERN 68-15): the two
//     intermediate masses of (p0 p1) and (p0 p1 p2) from sorted uniforms,
//     kept with probability (product of the three breakup momenta) / (its
//     maximum); isotropic two-body decays boosted into the parent frame;
//   * a decay time t ~ Exp(lambda), lambda = (1 - |y|) Gamma;
//   * the time-dependent rate R = e^{-Gamma t} B (Eq. (mix), factorised, in
//     double precision) from the event's invariants, width factors and
//     spin x barrier factors (the same double-precision kinematics as the
//     event loader) and the model at the given parameters;
//   * acceptance if u env < R e^{lambda t} (env: the envelope).
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
// doubles in [0, 1) (d = 0: decay time and acceptance; d = 8 + 5 try + j:
// GENBOD try `try`).
struct CandRng {
  uint32_t c0, c1, stream, k0, k1;
  __device__ double2 pair(uint32_t d) const {
    const Philox4 r = philox4x32_10(Philox4{{c0, c1, stream, d}}, k0, k1);
    return make_double2(u01(r.v[0], r.v[1]), u01(r.v[2], r.v[3]));
  }
};

__device__ __forceinline__ double breakup(double M, double a, double b) {
  const double s = M * M;
  const double l = (s - (a + b) * (a + b)) * (s - (a - b) * (a - b));
  return l > 0 ? sqrt(l) / (2.0 * M) : 0.0;
}

__device__ __forceinline__ V4 boost(V4 p, double bx, double by, double bz) {
  const double b2 = bx * bx + by * by + bz * bz;
  const double g = 1.0 / sqrt(1.0 - b2);
  const double bp = bx * p.x + by * p.y + bz * p.z;
  const double k = b2 > 0 ? (g - 1.0) / b2 * bp + g * p.e : 0.0;
  return V4{g * (p.e + bp), p.x + k * bx, p.y + k * by, p.z + k * bz};
}

// Flat four-body phase space of one candidate: false if every try failed
// (probability (1 - acceptance)^64).
__device__ inline bool genbod4(const GenArgs& a, const CandRng& rng, V4 (&p)[4]) {
  for (int tr = 0; tr < kGenMaxTries; ++tr) {
    const uint32_t d0 = 8u + 5u * uint32_t(tr);
    const double2 u0 = rng.pair(d0), u1 = rng.pair(d0 + 1);
    const double ra = fmin(u0.x, u0.y), rb = fmax(u0.x, u0.y);
    const double M1 = a.m[0] + a.m[1] + ra * a.tecm;
    const double M2 = a.m[0] + a.m[1] + a.m[2] + rb * a.tecm;
    const double q1 = breakup(M1, a.m[0], a.m[1]), q2 = breakup(M2, M1, a.m[2]), q3 = breakup(a.mD, M2, a.m[3]);
    if (!(u1.x < q1 * q2 * q3 * a.inv_wtmax)) continue;
    // isotropic directions from the remaining uniforms
    const double2 u2 = rng.pair(d0 + 2), u3 = rng.pair(d0 + 3), u4 = rng.pair(d0 + 4);
    const double ang[6] = {u1.y, u2.x, u2.y, u3.x, u3.y, u4.x};
    double dir[3][3];
    for (int j = 0; j < 3; ++j) {
      const double ct = 2.0 * ang[2 * j] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
      double sp, cp;
      sincospi(2.0 * ang[2 * j + 1], &sp, &cp);
      dir[j][0] = st * cp;
      dir[j][1] = st * sp;
      dir[j][2] = ct;
    }
    // p0, p1 back to back in the rest frame of (p0 p1)
    p[0] = V4{sqrt(q1 * q1 + a.m[0] * a.m[0]), q1 * dir[0][0], q1 * dir[0][1], q1 * dir[0][2]};
    p[1] = V4{sqrt(q1 * q1 + a.m[1] * a.m[1]), -q1 * dir[0][0], -q1 * dir[0][1], -q1 * dir[0][2]};
    // then p2 against (p0 p1), p3 against (p0 p1 p2): boost the subsystem
    const double qs[2] = {q2, q3}, Ms[2] = {M1, M2};
    for (int j = 0; j < 2; ++j) {
      const double q = qs[j];
      const double e = sqrt(q * q + Ms[j] * Ms[j]);
      const double bx = -q / e * dir[j + 1][0], by = -q / e * dir[j + 1][1], bz = -q / e * dir[j + 1][2];
      for (int i = 0; i <= j + 1; ++i) p[i] = boost(p[i], bx, by, bz);
      p[j + 2] = V4{sqrt(q * q + a.m[j + 2] * a.m[j + 2]), q * dir[j + 1][0], q * dir[j + 1][1], q * dir[j + 1][2]};
    }
    return true;
  }
  return false;
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

template <class S>
__device__ inline void gen_prologue(const GenArgs& a, CtaConst& cc, BlockConst<double>& bc) {
  derive_load<double, S::U>(nullptr, a.hp, a.km, cc, bc);
  __syncthreads();
  derive_compute<double, S::U, S::NR>(a.km, cc, bc);
  __syncthreads();
}

template <class S>
__global__ void __launch_bounds__(kGenThreads) k_gen_pass1(const __grid_constant__ GenArgs a) {
  __shared__ CtaConst cc;
  __shared__ BlockConst<double> bc;
  __shared__ uint32_t s_count;
  __shared__ unsigned long long s_wmax;
  const int tid = threadIdx.x, lane = tid & 31;
  if (!a.flat) gen_prologue<S>(a, cc, bc);
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
    V4 p[4];
    bool acc = genbod4(a, rng, p);
    if (acc && !a.flat) {
      const double2 u = rng.pair(0);
      const double t = -log1p(-u.x) / a.lambda;
      const double w = event_rate<S>(a.dm, bc, p, t) * exp(a.lambda * t);
      my_wmax = fmax(my_wmax, w);
      acc = u.y * a.env < w;
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
        genbod4(a, rng, p);  // accepted before: succeeds identically
        for (int q = 0; q < 4; ++q) {
          a.p_out[(4 * q + 0) * a.ld + o] = p[q].e;
          a.p_out[(4 * q + 1) * a.ld + o] = p[q].x;
          a.p_out[(4 * q + 2) * a.ld + o] = p[q].y;
          a.p_out[(4 * q + 3) * a.ld + o] = p[q].z;
        }
        if (a.t_out) a.t_out[o] = a.flat ? 0.0 : -log1p(-rng.pair(0).x) / a.lambda;
      }
    }
    pos += total;
  }
}

}  // namespace tdmix
