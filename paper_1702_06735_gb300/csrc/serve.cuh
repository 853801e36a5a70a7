// Batched evaluation of many likelihood requests (serving).
//
// A request is (sample, parameter vector) with the amplitude model's masses
// and widths fixed, so each resident sample keeps its per-event component
// cache and the MC normalisation sums are shared by all requests.  One
// persistent kernel evaluates a whole batch: the work items are chunks of
// consecutive event tiles of one request; a block takes chunks b, b + grid,
// ...  Each chunk's partial sums go to its own row, and the block that
// finishes the last chunk of a request sums that request's rows in chunk
// order and forms its NLL and gradient.  The chunk partition of a request
// depends only on its size, so a request's result does not depend on which
// other requests share the batch.
#pragma once
#include "fused.cuh"

namespace tdmix {


template <class P, class S>
struct ServeLayout {
  using T = typename P::T;
  static constexpr int U = S::U, NR = S::NR;
  static constexpr int WD = Layout<P, S>::WD;  // same data columns as the evaluation kernel
  // row stride of the chunk-partial array: even, so that every row starts on
  // a 16-byte boundary and a run of rows is a whole number of 16-byte units
  // (the bulk copy of a request's rows needs both)
  static constexpr int WR = (WD + 1) & ~1;
  static constexpr int stage_bytes = 2 * U * kTile * int(sizeof(T)) + kTile * 8;
  static constexpr int smem_bytes() {
    const int st = 2 * stage_bytes, pr = kServeMaxChunks * WR * 8;
    return st > pr ? st : pr;
  }
};

template <class P, class S, bool GRAD>
__global__ void __launch_bounds__(kTile, 1) k_serve(const __grid_constant__ ServeArgs a) {
  using T = typename P::T;
  using LY = ServeLayout<P, S>;
  constexpr int U = S::U, NR = S::NR, WD = LY::WD, WR = LY::WR, TE = kTile, ES = int(sizeof(T));
  constexpr int WMC = Layout<P, S>::WMC;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ CtaConst cc;
  __shared__ BlockConst<T> bc;
  __shared__ T red[(kTile / 32) * (2 + 4 * U)];
  __shared__ double red_lnb[kTile / 32];
  __shared__ int red_bad[kTile / 32];
  __shared__ float2 rowp[WD];
  __shared__ double colsum[WMC + WD];
  __shared__ int chunk_start[kServeMaxRequests + 1];
  __shared__ unsigned is_last;
  __shared__ int s_timed_out;
  __shared__ double2 logtab[kLogTable];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  unsigned char* stage[2] = {smem_raw, smem_raw + LY::stage_bytes};
  for (int r = tid; r < a.n_req; r += blockDim.x) chunk_start[r] = a.reqs[r].chunk_begin;
  for (int j = tid; j < kLogTable; j += blockDim.x) logtab[j] = static_cast<const double2*>(a.logtab)[j];
  if (tid == 0) {
    chunk_start[a.n_req] = a.total_chunks;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const int np = a.km.n_params, nc = a.km.n_chains;
  uint32_t uses = 0;  // completed barrier phases (both stages), for parity tracking
  bool failed = false;

  for (int c = blockIdx.x; c < a.total_chunks && !failed; c += G) {
    int lo = 0, hi = a.n_req;  // request r with chunk_start[r] <= c < chunk_start[r + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (chunk_start[mid] <= c) lo = mid;
      else hi = mid;
    }
    const int r = lo;
    const ServeReq q = a.reqs[r];
    const int lc = c - q.chunk_begin;
    const int t0 = lc * q.chunk_tiles;
    const int t1 = min(t0 + q.chunk_tiles, q.n_tiles);
    const int ntl = t1 - t0;
    auto issue = [&](int j, uint32_t use) {  // tile t0 + j into stage use & 1 (one bulk copy)
      const int st = int(use & 1);
      mbar_arrive_expect_tx(&bars[st], uint32_t(q.tile_bytes));
      bulk_g2s(stage[st], static_cast<const unsigned char*>(q.cache) + int64_t(t0 + j) * q.tile_bytes,
               uint32_t(q.tile_bytes), &bars[st]);
    };
    if (tid == 0) {
      issue(0, uses);
      if (ntl > 1) issue(1, uses + 1);
    }
    derive_load<T, U>(a.params + size_t(r) * np, nullptr, a.km, cc, bc);
    __syncthreads();
    derive_compute<T, U, NR>(a.km, cc, bc);
    __syncthreads();

    double lnb = 0.0;  // sum ln B = lnb + lexp ln 2
    int bad = 0, lexp = 0;
    T gx = 0, gy = 0, gAr[U], gAi[U], gBr[U], gBi[U];
#pragma unroll
    for (int j = 0; j < U; ++j) gAr[j] = gAi[j] = gBr[j] = gBi[j] = 0;
    for (int j = 0; j < ntl; ++j, ++uses) {
      const int st = int(uses & 1);
      const bool ok = mbar_wait_bounded(&bars[st], (uses >> 1) & 1u, kWaitNs);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      const int64_t i = int64_t(t0 + j) * TE + tid;
      if (i < q.n) {
        const T* sbase = reinterpret_cast<const T*>(stage[st]);
        const double t_e = reinterpret_cast<const double*>(stage[st] + 2 * U * TE * ES)[tid];
        EventCore<P, S> ev;
#pragma unroll
        for (int k = 0; k < U; ++k) {
          ev.ar[k] = sbase[k * TE + tid];
          ev.ai[k] = sbase[(U + k) * TE + tid];
        }
        T Ar_, Ai_, Br_, Bi_;
        ev.template amplitudes<true>(bc, Ar_, Ai_, Br_, Bi_);
        T tAr, tAi, tBr, tBi;
        if (mix_event<P, GRAD>(bc, logtab, double(Ar_), double(Ai_), double(Br_), double(Bi_), Ar_, Ai_, Br_, Bi_,
                               t_e, lnb, lexp, nullptr, tAr, tAi, tBr, tBi, gx, gy)) {
          if constexpr (GRAD) {
#pragma unroll
            for (int k = 0; k < U; ++k) {
              cmac(gAr[k], gAi[k], tAr, tAi, ev.ar[k], ev.ai[k]);
              cmac(gBr[k], gBi[k], tBr, tBi, ev.ar[k], ev.ai[k]);
            }
          }
        } else {
          bad += 1;
        }
      }
      __syncthreads();
      if (tid == 0 && j + 2 < ntl) issue(j + 2, uses + 2);
    }
    if (failed) {
      if (tid == 0) {
        atomicOr(a.err, 1);
        for (uint32_t u = uses; u < uses + 2; ++u) mbar_wait_bounded(&bars[u & 1], (u >> 1) & 1u, kWaitNs);
      }
      __syncthreads();
    }
    // chunk partial -> its row (double-float; see block_sum_df)
    {
      const double v0 = warp_sum(fma(double(lexp), kLn2, lnb));
      const int v1 = warp_sum(bad);
      if (lane == 0) {
        red_lnb[warp] = v0;
        red_bad[warp] = v1;
      }
      T vt[2 + 4 * U];
      vt[0] = gx;
      vt[1] = gy;
#pragma unroll
      for (int k = 0; k < U; ++k) {
        vt[2 + k] = gAr[k];
        vt[2 + U + k] = gAi[k];
        vt[2 + 2 * U + k] = gBr[k];
        vt[2 + 3 * U + k] = gBi[k];
      }
      block_sum_df<T, 2 + 4 * U>(vt, red, rowp + 2);  // ends with a barrier
    }
    float2* part = static_cast<float2*>(a.part);
    if (tid == 0) {
      double sl = 0;
      int sb = 0;
      for (int w = 0; w < kTile / 32; ++w) {
        sl += red_lnb[w];
        sb += red_bad[w];
      }
      rowp[0] = to_df(sl);
      rowp[1] = make_float2(float(sb), 0.f);
    }
    __syncthreads();
    for (int v = tid; v < WR; v += blockDim.x)
      part[size_t(c) * WR + v] = v < 4 + 4 * U ? rowp[v] : make_float2(0.f, 0.f);
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(a.counters + r, 1u) == unsigned(q.n_chunks - 1);
    __syncthreads();
    if (!is_last) continue;
    // ---- last chunk of request r: sum its rows in chunk order, then the likelihood
    __threadfence();
    float2* sp = reinterpret_cast<float2*>(smem_raw);
    if (tid == 0) {
      asm volatile("fence.proxy.async.global;" ::: "memory");
      mbar_init(&bars[2], 1);
      mbar_fence_init();
      const uint32_t bytes = uint32_t(q.n_chunks) * uint32_t(WR) * 8u;  // a multiple of 16
      mbar_arrive_expect_tx(&bars[2], bytes);
      bulk_g2s(sp, part + size_t(q.chunk_begin) * WR, bytes, &bars[2]);  // 16-byte aligned
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bars[2], 0, kWaitNs);
    if (__syncthreads_or(!ok) && tid == 0) atomicOr(a.err, 1);
    for (int v = tid; v < WMC; v += blockDim.x) colsum[v] = a.mc_cols[v];
    for (int v = tid; v < WD; v += blockDim.x) {
      float s = 0.f, e = 0.f;
      for (int row = 0; row < q.n_chunks; ++row) {
        const float2 x = sp[size_t(row) * WR + v];
        float t, er;
        two_sum(s, x.x, t, er);
        s = t;
        e += er + x.y;
      }
      colsum[WMC + v] = double(s) + double(e);
    }
    if (tid == 0) {
      // a bounded wait that gave up anywhere in the batch is reported (once)
      s_timed_out = *static_cast<volatile int*>(a.err);
      if (s_timed_out) *a.err = 0;
      a.counters[r] = 0u;
    }
    __syncthreads();
    finish_likelihood<S>(a.results + size_t(r) * (kResHeader + np), nullptr, nullptr, nc, np, cc, colsum,
                         colsum + WMC, double(q.n), q.sum_t, a.inv_sum_w, GRAD, false, s_timed_out, logtab, nullptr);
    __syncthreads();
    // the bulk-copy target overlapped the stages: stages restart clean below
  }
}

}  // namespace tdmix
