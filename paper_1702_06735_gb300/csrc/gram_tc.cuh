// The phase-space normalisation matrix on the tensor cores (fp32 path).
//
// Over one tile of 256 MC events the real Gram matrix G = X^T X of the
// event-by-component matrix X (columns: Re a_j then Im a_j, times sqrt(w)
// for weighted events; I_jk = <a_j^* a_k> follows from G, Sec. 3.1) is
// computed by one chain of tcgen05 MMAs, exactly:
//   * each column c gets the power of two 2^s_c that brings the tile's
//     largest |x_c| just below 128 (the exponent maximum over the tile by
//     warp reductions and a shared-memory atomic max);
//   * every value is split into four integer pieces,
//       x 2^s_c = d0 + d1 / 2^8 + d2 / 2^16 + d3 / 2^24,  |d_p| <= 128,
//     each exact in bf16, with the rounding of the last piece the only
//     approximation (below 2^-31 of the tile's largest |x_c|, unbiased);
//   * one MMA chain forms D = [P0; P1; P2; P3] [P0; P1]^T over the 256
//     events (P_p: the pieces as a component-by-event matrix), M = 4 x
//     8-padded 2U rows (64 or 128), N = 2 x 8-padded 2U, K = 16 per
//     instruction; every entry is a sum of 256 products of integers below
//     2^14, an integer below 2^22, so the tensor core's truncating
//     accumulation is exact;
//   * D is staged from tensor memory to shared memory and folded into a
//     double-float accumulator per entry c <= d of G:
//       G_cd += 2^-(s_c + s_d) [D00 + (D01 + D10) / 2^8 + (D02 + D11 + D20) / 2^16
//                               + (D03 + D12 + D21 + D30) / 2^24]
//     (D_pq the P_p P_q^T block; D02 = D20^T, D03 = D30^T, D12 = D21^T; the
//     products of pieces p + q > 3 are below 2^-32 of the largest and are
//     left out); each numerator is an exact integer sum below 2^24 and the
//     bracket is exact in double-float, so the only rounding is the
//     accumulation itself.
// The pieces are stored MN-major (8 consecutive components of one event in
// 16 contiguous bytes: one 128-bit store per thread and piece), so the
// same shared-memory buffer is both MMA operands.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "tcgen05.cuh"

namespace tdmix {

template <int U>
struct TcGram {
  static constexpr int TE = kTileEvents;
  static constexpr int C = 2 * U;                 // real columns of X
  static constexpr int CP = (C + 7) / 8 * 8;      // rows per piece (padded to whole core matrices)
  static constexpr int NP = 4;                    // pieces per value
  static constexpr int ROWS = NP * CP;            // A rows holding pieces 0 .. 3
  static constexpr int M = ROWS <= 64 ? 64 : 128;
  static constexpr int N = 2 * CP;                // B rows: pieces 0 and 1
  static constexpr int KSTEP = 16;                // events per bf16 MMA
  static constexpr int CORE_K = 128;              // bytes between K-adjacent core matrices
  static constexpr int CORE_MN = (TE / 8) * CORE_K;  // bytes between M-adjacent core matrices (4 KB)
  static constexpr int NE = C * (C + 1) / 2;      // entries c <= d of G
  static constexpr int DS = N + 4;                // staging row stride (floats)
  static constexpr int TMEM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  static_assert(ROWS <= 128 && N <= 256, "tensor-core normalisation matrix supports up to 16 components");
  static_assert(M == 64 ? N % 8 == 0 : N % 16 == 0, "MMA shape");
  // shared-memory regions (bytes, each a multiple of 128)
  static constexpr int piece_bytes = (M / 8) * CORE_MN;
  static constexpr int stage_bytes = (ROWS * DS * 4 + 127) / 128 * 128;
  static constexpr int acc_bytes = (NE * 8 + 127) / 128 * 128;
  static constexpr int pair_bytes = (NE * 2 + 127) / 128 * 128;
  static constexpr int extra_bytes = piece_bytes + stage_bytes + acc_bytes + pair_bytes;
  static constexpr uint32_t idesc() { return idesc_bf16_mn_major(M, N); }
  // TMEM lane of accumulator row r
  __device__ static constexpr int lane_of_row(int r) { return M == 128 ? r : 32 * (r / 16) + r % 16; }
  // packed index of entry (c, d), c <= d
  __host__ __device__ static constexpr int idx(int c, int d) { return c * (2 * C - c + 1) / 2 + (d - c); }
};

// Biased exponent of |v| (0 for zero).
__device__ __forceinline__ unsigned exp_bits(float v) { return (__float_as_uint(v) >> 23) & 0xFFu; }

// Shared-memory state of the tensor-core Gram in one block.
template <int U>
struct TcGramSmem {
  using L = TcGram<U>;
  unsigned char* piece;  // MMA operand buffer (MN-major pieces)
  float* dstage;         // [ROWS][DS] accumulator copy
  float2* acc;           // [NE] double-float G_cd
  uint16_t* pairs;       // [NE] (c | d << 8)

  __device__ static TcGramSmem at(unsigned char* base) {
    TcGramSmem s;
    s.piece = base;
    s.dstage = reinterpret_cast<float*>(base + L::piece_bytes);
    s.acc = reinterpret_cast<float2*>(base + L::piece_bytes + L::stage_bytes);
    s.pairs = reinterpret_cast<uint16_t*>(base + L::piece_bytes + L::stage_bytes + L::acc_bytes);
    return s;
  }

  // Zeroes the operand buffer (rows beyond the pieces stay zero) and the
  // accumulators, and fills the pair table (all threads; caller syncs).
  __device__ void init() const {
    for (int i = threadIdx.x; i < L::piece_bytes / 16; i += blockDim.x)
      reinterpret_cast<uint4*>(piece)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = threadIdx.x; i < L::NE; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
    for (int c = threadIdx.x; c < L::C; c += blockDim.x)
      for (int d = c; d < L::C; ++d) pairs[L::idx(c, d)] = uint16_t(c | (d << 8));
  }

  // This thread's event (slot e of the tile): quantise x[CP] with the
  // tile's column exponents E[c] (max biased exponent, clamped to >= 7) and
  // store the four pieces; then make the stores visible to the tensor core.
  __device__ void store_pieces(const float (&x)[L::CP], const unsigned* E, int e) const {
#pragma unroll
    for (int g = 0; g < L::CP / 8; ++g) {
      uint32_t w[L::NP][4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float d[L::NP][2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int c = 8 * g + 2 * h + q;
          const float sc = __uint_as_float((260u - E[c]) << 23);  // 2^(133 - E): |x sc| < 128
          float r = x[c] * sc;
#pragma unroll
          for (int p = 0; p < L::NP; ++p) {
            d[p][q] = rintf(r);
            r = (r - d[p][q]) * 256.f;  // exact: |r - d| <= 1/2 on r's own grid
          }
        }
#pragma unroll
        for (int p = 0; p < L::NP; ++p) {
          const __nv_bfloat162 b = __floats2bfloat162_rn(d[p][0], d[p][1]);  // .x (low half) = even c
          w[p][h] = *reinterpret_cast<const uint32_t*>(&b);
        }
      }
#pragma unroll
      for (int p = 0; p < L::NP; ++p) {
        const int row_core = (p * L::CP + 8 * g) / 8;
        *reinterpret_cast<uint4*>(piece + row_core * L::CORE_MN + (e / 8) * L::CORE_K + (e % 8) * 16) =
            make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
      }
    }
    fence_async_smem();
  }

  // One thread: the MMA chain of the tile into TMEM at taddr, then a commit
  // on `bar`.  Call after a barrier that follows every thread's store_pieces.
  __device__ void issue(uint32_t taddr, uint64_t* bar) const {
    tc_fence_after_sync();
    const uint32_t base = smem_u32(piece);
#pragma unroll 1
    for (int s = 0; s < L::TE / L::KSTEP; ++s) {
      const uint64_t dsc = smem_matrix_desc(base + uint32_t(s) * 2u * L::CORE_K, L::CORE_K, L::CORE_MN);
      tc_mma_bf16(taddr, dsc, dsc, L::idesc(), s > 0);
    }
    tc_commit(bar);
  }

  // Warps 0..3: copy the accumulator rows of their TMEM lane quarter to the
  // staging buffer (after the MMA commit completed).
  __device__ void stage(uint32_t taddr) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= 4) return;
    const int row = L::M == 128 ? 32 * warp + lane : (lane < 16 ? 16 * warp + lane : L::ROWS);
#pragma unroll
    for (int n0 = 0; n0 < L::N; n0 += 16) {
      uint32_t v[16];
      tmem_ld16(taddr + (uint32_t(32 * warp) << 16) + uint32_t(n0), v);
      tmem_wait_ld();
      if (row < L::ROWS) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<uint4*>(dstage + row * L::DS + n0 + j) = make_uint4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
    }
  }

  // All threads: fold the staged tile into the accumulators (entries
  // tid, tid + blockDim, ...), with the tile's column exponents E.
  __device__ void fold(const unsigned* E) const {
    for (int q = threadIdx.x; q < L::NE; q += blockDim.x) {
      const int pr = pairs[q], c = pr & 0xFF, d = pr >> 8;
      const float* rc0 = dstage + c * L::DS;
      const float* rc1 = dstage + (L::CP + c) * L::DS;
      const float* rc2 = dstage + (2 * L::CP + c) * L::DS;
      const float* rc3 = dstage + (3 * L::CP + c) * L::DS;
      const float* rd2 = dstage + (2 * L::CP + d) * L::DS;
      const float* rd3 = dstage + (3 * L::CP + d) * L::DS;
      const float s1 = rc0[L::CP + d] + rc1[d];                              // D01 + D10 (< 2^23)
      const float s2 = (rc1[L::CP + d] + rc2[d]) + rd2[c];                   // D11 + D20 + D02 (< 2^24)
      const float s3 = (rc3[d] + rc2[L::CP + d]) + (rd2[L::CP + c] + rd3[c]);  // D30 + D21 + D12 + D03 (< 2^24)
      const DF v1 = df_two_sum(rc0[d], s1 * (1.0f / 256.0f));                // all exact
      const DF v2 = df_two_sum(v1.hi, s2 * (1.0f / 65536.0f));
      const DF v3 = df_two_sum(v2.hi, s3 * (1.0f / 16777216.0f));
      DF v = df_fast_two_sum(v3.hi, v3.lo + (v2.lo + v1.lo));
      const float fc = __uint_as_float((E[c] - 6u) << 23), fd = __uint_as_float((E[d] - 6u) << 23);  // 2^(E - 133)
      v.hi = v.hi * fc * fd;
      v.lo = v.lo * fc * fd;
      const float2 a = acc[q];
      const DF s = df_add(DF{a.x, a.y}, v);
      acc[q] = make_float2(s.hi, s.lo);
    }
  }

  // Real and imaginary parts of the complex normalisation sums from G:
  // Re S_jk = G[j][k] + G[U+j][U+k] (j <= k), Im S_jk = G[j][U+k] - G[U+j][k]
  // (j < k; G symmetric), in the column order of the evaluation kernel.
  __device__ void finish(float2* re, float2* im) const {
    for (int q = threadIdx.x; q < U * (U + 1) / 2 + U * (U - 1) / 2; q += blockDim.x) {
      const bool is_re = q < U * (U + 1) / 2;
      int r = is_re ? q : q - U * (U + 1) / 2, j = 0;
      // (j, k) of the q-th pair in row-major order over j <= k (re) or j < k (im)
      for (;;) {
        const int len = is_re ? U - j : U - 1 - j;
        if (r < len) break;
        r -= len;
        ++j;
      }
      const int k = is_re ? j + r : j + 1 + r;
      DF a, b;
      if (is_re) {
        const float2 x = acc[L::idx(j, k)], y = acc[L::idx(U + j, U + k)];
        a = DF{x.x, x.y};
        b = DF{y.x, y.y};
        const DF s = df_add(a, b);
        re[q] = make_float2(s.hi, s.lo);
      } else {
        const float2 x = acc[L::idx(j, U + k)], y = acc[L::idx(k, U + j)];
        a = DF{x.x, x.y};
        b = DF{y.x, y.y};
        const DF s = df_sub(a, b);
        im[q - U * (U + 1) / 2] = make_float2(s.hi, s.lo);
      }
    }
  }
};

}  // namespace tdmix
