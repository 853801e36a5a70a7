// Device-resident serving loop: many likelihood requests from concurrent
// minimisers (the paper's sensitivity study fits pseudo-experiments with a
// fixed model and floating x, y, Sec. 4).
//
// A request is (sample, parameter vector) with the model's masses and
// widths fixed, so each resident sample keeps its per-event component cache
// and the MC normalisation sums are shared by all requests.  The host
// writes a request into a slot of page-locked, device-mapped memory and
// publishes it as the next ring entry (a release store of the ring's tail).
// A persistent kernel (one block per SM, leaving some SMs to admission and
// generation work) takes work items (entry, chunk of consecutive event
// tiles) as they appear:
//   * thread 0 of a block claims a chunk of the entry at its cursor with an
//     atomic counter and moves the cursor to the next entry (round robin
//     over the entries with unclaimed chunks, so a short request published
//     while a long one runs is served at once);
//   * the block evaluates the chunk from the cached components (Eq. (mix),
//     ln B, adjoint) and writes its partial row;
//   * the block that finishes a request's last chunk sums the request's
//     rows in chunk order, forms the NLL and gradient into the slot, makes
//     them visible system-wide and then stores `done` with release
//     semantics.
// The chunk partition of a request depends only on its size and its rows
// are summed in chunk order, so a result does not depend on which other
// requests are in flight.  Every wait is bounded: a wait for new work gives
// up after idle_ns (status 2) and the block exits; the host stops the loop
// (ring.stop) when it has nothing in flight.
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
  // stages of the tile ring: as many as fit 160 KiB, 2 to 6 (a chunk's
  // tiles stream from HBM; the lookahead covers the copy latency)
  static constexpr int stages() {
    const int n = 160 * 1024 / stage_bytes;
    return n < 2 ? 2 : (n > 6 ? 6 : n);
  }
  static constexpr int smem_bytes() {
    const int st = stages() * stage_bytes, pr = kServeMaxChunks * WR * 8;
    return st > pr ? st : pr;
  }
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_relaxed_sys(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <class P, class S, bool GRAD>
__global__ void __launch_bounds__(kTile, 1) k_serve_loop(const __grid_constant__ ServeLoopArgs a) {
  using T = typename P::T;
  using LY = ServeLayout<P, S>;
  constexpr int U = S::U, NR = S::NR, WD = LY::WD, WR = LY::WR, TE = kTile, ES = int(sizeof(T));
  constexpr int WMC = Layout<P, S>::WMC;
  constexpr int NST = LY::stages();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[NST + 1];  // one per stage, then the row copy's
  __shared__ CtaConst cc;
  __shared__ BlockConst<T> bc;
  __shared__ T red[(kTile / 32) * (2 + 4 * U)];
  __shared__ double red_lnb[kTile / 32];
  __shared__ int red_bad[kTile / 32];
  __shared__ float2 rowp[WD];
  __shared__ double colsum[WMC + WD];
  __shared__ double2 logtab[kLogTable];
  __shared__ float4 logtab_f[P::kF32 ? kLogTable : 1];  // the same entries as double-float pairs
  __shared__ long long s_entry;
  __shared__ int s_chunk, s_slot;
  __shared__ unsigned s_last;
  __shared__ ServeSlot s_req;  // the request's fields (one read of mapped memory)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto stage = [&](int st) { return smem_raw + st * LY::stage_bytes; };
  for (int j = tid; j < kLogTable; j += blockDim.x) {
    const double2 v = static_cast<const double2*>(a.logtab)[j];
    logtab[j] = v;
    if constexpr (P::kF32) {
      const DF r = df_from_double(v.x), l = df_from_double(v.y);
      logtab_f[j] = make_float4(r.hi, r.lo, l.hi, l.lo);
    }
  }
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) mbar_init(&bars[q], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const int np = a.km.n_params, nc = a.km.n_chains;
  uint32_t uses = 0;                    // stage uses so far: stage uses % NST, phase parity (uses / NST) & 1
  unsigned long long cursor = a.head;   // thread 0: next entry to try
  float2* part_all = static_cast<float2*>(a.part);

  for (;;) {
    // ---- thread 0 claims the next chunk: (entry, chunk), or stops
    if (tid == 0) {
      long long e = -1;
      int c = 0, slot = 0;
      unsigned long long idle_since = 0;
      for (;;) {
        if (ld_relaxed_sys(&a.ring->stop)) break;
        const unsigned long long tail = ld_acquire_sys(&a.ring->tail);
        const unsigned long long low = *static_cast<volatile unsigned long long*>(a.low);
        if (cursor < low || cursor >= tail) cursor = low;  // round robin over [low, tail)
        if (cursor >= tail) {                                // every published chunk is claimed
          const unsigned long long now = global_ns();
          if (idle_since == 0) {
            idle_since = now;
          } else if (now - idle_since > a.idle_ns) {
            atomicOr(a.status, 2);
            break;
          }
          __nanosleep(200);
          continue;
        }
        idle_since = 0;
        const int idx = int(cursor - a.head);
        const int sl = a.ring->slot[idx];
        const int nch = a.slots[sl].n_chunks;
        const unsigned k = atomicAdd(&a.claimed[idx], 1u);
        if (k < unsigned(nch)) {
          e = (long long)cursor;
          c = int(k);
          slot = sl;
          ++cursor;
          break;
        }
        // this entry has no unclaimed chunk left; only the oldest such entry
        // moves `low` on (a newer one being exhausted says nothing about
        // the older entries the round robin still has to visit)
        atomicCAS(a.low, cursor, cursor + 1);
        ++cursor;
      }
      s_entry = e;
      s_chunk = c;
      s_slot = slot;
      if (e >= 0) {
        const ServeSlot& q = a.slots[slot];
        s_req.cache = q.cache;
        s_req.n = q.n;
        s_req.tile_bytes = q.tile_bytes;
        s_req.n_chunks = q.n_chunks;
        s_req.chunk_tiles = q.chunk_tiles;
        s_req.n_tiles = q.n_tiles;
        s_req.sum_t = q.sum_t;
      }
    }
    __syncthreads();
    const long long e = s_entry;
    if (e < 0) break;
    const int c = s_chunk, slot = s_slot, eidx = int(e - (long long)a.head);
    const int t0 = c * s_req.chunk_tiles;
    const int t1 = min(t0 + s_req.chunk_tiles, s_req.n_tiles);
    const int ntl = t1 - t0;
    const void* cache = s_req.cache;
    const int64_t tile_bytes = s_req.tile_bytes, n_ev = s_req.n;
    auto issue = [&](int j, uint32_t use) {  // tile t0 + j into stage use % NST (one bulk copy)
      const int st = int(use % NST);
      mbar_arrive_expect_tx(&bars[st], uint32_t(tile_bytes));
      bulk_g2s(stage(st), static_cast<const unsigned char*>(cache) + int64_t(t0 + j) * tile_bytes,
               uint32_t(tile_bytes), &bars[st]);
    };
    if (tid == 0)
      for (int q = 0; q < NST && q < ntl; ++q) issue(q, uses + q);
    derive_load<T, U>(a.slots[slot].params, nullptr, a.km, cc, bc);
    __syncthreads();
    derive_compute<T, U, NR>(a.km, cc, bc);
    __syncthreads();

    double lnb = 0.0;     // sum ln B = lnb + lexp ln 2 (fp64 path)
    DF lnbf{0.0f, 0.0f};  // the same as a double-float pair (fp32 path)
    int bad = 0, lexp = 0;
    bool failed = false;
    int failed_at = 0;
    T gx = 0, gy = 0, gAr[U], gAi[U], gBr[U], gBi[U];
#pragma unroll
    for (int j = 0; j < U; ++j) gAr[j] = gAi[j] = gBr[j] = gBi[j] = 0;
    for (int j = 0; j < ntl; ++j, ++uses) {
      const int st = int(uses % NST);
      const bool ok = mbar_wait_bounded(&bars[st], (uses / NST) & 1u, kWaitNs);
      if (__syncthreads_or(!ok)) {
        failed = true;
        failed_at = j;
        break;
      }
      const int64_t i = int64_t(t0 + j) * TE + tid;
      if (i < n_ev) {
        const T* sbase = reinterpret_cast<const T*>(stage(st));
        // decay time: a double (fp64 path) or a double-float pair (fp32 path)
        const unsigned char* tplane = stage(st) + 2 * U * TE * ES;
        const double t_e = P::kF32 ? 0.0 : reinterpret_cast<const double*>(tplane)[tid];
        const float2 t_f = P::kF32 ? reinterpret_cast<const float2*>(tplane)[tid] : float2{0.f, 0.f};
        EventCore<P, S> ev;
#pragma unroll
        for (int k = 0; k < U; ++k) {
          ev.ar[k] = sbase[k * TE + tid];
          ev.ai[k] = sbase[(U + k) * TE + tid];
        }
        T Ar_, Ai_, Br_, Bi_;
        ev.template amplitudes<!(P::kF32 && GRAD)>(bc, Ar_, Ai_, Br_, Bi_);  // see coef_residue_term
        T tAr, tAi, tBr, tBi;
        bool ok_ev;
        if constexpr (P::kF32)
          ok_ev = mix_event_df<GRAD>(bc, logtab, logtab_f, DF{Ar_, 0.0f}, DF{Ai_, 0.0f}, DF{Br_, 0.0f},
                                     DF{Bi_, 0.0f}, t_f.x, t_f.y, lnbf, lexp, nullptr, tAr, tAi, tBr, tBi, gx, gy);
        else
          ok_ev = mix_event<P, GRAD>(bc, logtab, Ar_, Ai_, Br_, Bi_, Ar_, Ai_, Br_, Bi_, t_e, lnb, lexp, nullptr, tAr,
                                     tAi, tBr, tBi, gx, gy);
        if (ok_ev) {
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
      if (tid == 0 && j + NST < ntl) issue(j + NST, uses + NST);
    }
    if (failed) {
      // the copies of tiles failed_at .. failed_at + NST - 1 (those that
      // exist) are in flight: let them land before shared memory is
      // reused, and count their stage phases
      const uint32_t in_flight = uint32_t(ntl - failed_at < NST ? ntl - failed_at : NST);
      if (tid == 0) {
        atomicOr(a.status, 1);
        for (uint32_t u = uses; u < uses + in_flight; ++u)
          mbar_wait_bounded(&bars[u % NST], (u / NST) & 1u, kWaitNs);
      }
      __syncthreads();
      uses += in_flight;
    }
    // chunk partial -> its row (double-float; see block_sum_df)
    {
      const double v0 = warp_sum(fma(double(lexp), kLn2, P::kF32 ? df_to_double(lnbf) : lnb));
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
    float2* part = part_all + size_t(slot) * kServeMaxChunks * WR;
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
    if (tid == 0) s_last = atomicAdd(&a.finished[eidx], 1u) == unsigned(s_req.n_chunks - 1);
    __syncthreads();
    if (!s_last) continue;
    // ---- last chunk of the request: sum its rows in chunk order, then the likelihood
    __threadfence();
    float2* sp = reinterpret_cast<float2*>(smem_raw);
    const int nch = s_req.n_chunks;
    if (tid == 0) {
      asm volatile("fence.proxy.async.global;" ::: "memory");
      mbar_init(&bars[NST], 1);
      mbar_fence_init();
      const uint32_t bytes = uint32_t(nch) * uint32_t(WR) * 8u;  // a multiple of 16
      mbar_arrive_expect_tx(&bars[NST], bytes);
      bulk_g2s(sp, part, bytes, &bars[NST]);  // 16-byte aligned
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bars[NST], 0, kWaitNs);
    if (__syncthreads_or(!ok) && tid == 0) atomicOr(a.status, 1);
    for (int v = tid; v < WMC; v += blockDim.x) colsum[v] = a.mc_cols[v];
    for (int v = tid; v < WD; v += blockDim.x) {
      float s = 0.f, er = 0.f;
      for (int row = 0; row < nch; ++row) {
        const float2 x = sp[size_t(row) * WR + v];
        float t, err;
        two_sum(s, x.x, t, err);
        s = t;
        er += err + x.y;
      }
      colsum[WMC + v] = double(s) + double(er);
    }
    __syncthreads();
    const int timed_out = *static_cast<volatile int*>(a.status) & 1;
    finish_likelihood<S, P::kF32 && GRAD>(a.slots[slot].result, nullptr, nullptr, nc, np, cc, colsum, colsum + WMC, double(n_ev),
                         s_req.sum_t, a.inv_sum_w, GRAD, false, timed_out, logtab, nullptr);
    __threadfence_system();
    __syncthreads();
    if (tid == 0) st_release_sys(&a.slots[slot].done, (unsigned long long)(e + 1));
    // the row copy overlapped the stages; later chunks refill them from scratch
  }
}

}  // namespace tdmix
