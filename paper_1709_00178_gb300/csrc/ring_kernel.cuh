// The generic ring-transform coding kernels (paper Sec. 2.3.2 and Sec. 3): the staged pipeline of
// ring_staged.cuh with a multiply-accumulate step driven by the job's ring masks at run time, and
// a plain-load form for packets that bulk copies cannot move.
#pragma once

#include <cuda_runtime.h>

#include "pyrit_internal.h"
#include "ring_staged.cuh"

namespace pyrit {


// acc += x^S * d in R_{2,N}: packet q of the embedded source lands in accumulator (q + S) mod N.
template <int N, int WORDS, int S>
__device__ __forceinline__ void xor_rotated(uint32_t (&acc)[N][WORDS], const uint32_t (&d)[RingDim<N>::W][WORDS]) {
  if constexpr (S < N) {
#pragma unroll
    for (int q = 0; q < RingDim<N>::W; ++q)
#pragma unroll
      for (int x = 0; x < WORDS; ++x) acc[(q + S) % N][x] ^= d[q][x];
  }
}

// acc += x^s * d for a run-time shift s < N. The rotation is resolved by a warp-uniform jump to
// straight-line code with static register indices (all lanes share the job, so no divergence).
template <int N, int WORDS>
__device__ __forceinline__ void xor_rotated_dyn(uint32_t (&acc)[N][WORDS],
                                                const uint32_t (&d)[RingDim<N>::W][WORDS], int s) {
  switch (s) {
    case 0: xor_rotated<N, WORDS, 0>(acc, d); break;
    case 1: xor_rotated<N, WORDS, 1>(acc, d); break;
    case 2: xor_rotated<N, WORDS, 2>(acc, d); break;
    case 3: xor_rotated<N, WORDS, 3>(acc, d); break;
    case 4: xor_rotated<N, WORDS, 4>(acc, d); break;
    case 5: xor_rotated<N, WORDS, 5>(acc, d); break;
    case 6: xor_rotated<N, WORDS, 6>(acc, d); break;
    case 7: xor_rotated<N, WORDS, 7>(acc, d); break;
    case 8: xor_rotated<N, WORDS, 8>(acc, d); break;
    case 9: xor_rotated<N, WORDS, 9>(acc, d); break;
    case 10: xor_rotated<N, WORDS, 10>(acc, d); break;
    case 11: xor_rotated<N, WORDS, 11>(acc, d); break;
    case 12: xor_rotated<N, WORDS, 12>(acc, d); break;
    default: break;
  }
}

// acc += (x^S1 + x^S2) * d in R_{2,N} in one pass: accumulator t receives d[t - S1] ^ d[t - S2]
// (one three-input XOR), or a single term where the other index is a zero packet (index >= W).
template <int N, int WORDS, int S1, int S2>
__device__ __forceinline__ void xor_pair(uint32_t (&acc)[N][WORDS], const uint32_t (&d)[RingDim<N>::W][WORDS]) {
  constexpr int W = RingDim<N>::W;
#pragma unroll
  for (int t = 0; t < N; ++t) {
    const int q1 = (t - S1 + N) % N, q2 = (t - S2 + N) % N;
#pragma unroll
    for (int x = 0; x < WORDS; ++x) {
      if (q1 < W && q2 < W)
        acc[t][x] ^= d[q1][x] ^ d[q2][x];
      else if (q1 < W)
        acc[t][x] ^= d[q1][x];
      else if (q2 < W)
        acc[t][x] ^= d[q2][x];
    }
  }
}

#include "ring_network.inc"

// acc_i += r_ij * d for every output i of the group, one rotation per set bit of r_ij. The masks
// arrive as warp-uniform 32-bit words (two 16-bit masks each), so every branch below is uniform.
//   DISPATCH 0: one uniform test per shift S (static code per (i, S); no indirect jump).
//   DISPATCH 1: iterate over the set bits and jump to the rotation's code through a switch.
//   DISPATCH 2: the generated pairing automaton: consecutive set bits fused into one pass of
//               three-input XORs, static forward branches only (ring_network.inc).
template <int N, int WORDS, int MG, int DISPATCH>
__device__ __forceinline__ void ring_mac(uint32_t (&acc)[MG][N][WORDS], const uint32_t (&d)[RingDim<N>::W][WORDS],
                                         const uint32_t (&mu)[(MG + 1) / 2]) {
#pragma unroll
  for (int i = 0; i < MG; ++i) {
    const uint32_t m = (mu[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
    if constexpr (DISPATCH == 0) {
#pragma unroll
      for (int s = 0; s < N; ++s) {
        if (m & (1u << s)) {
#pragma unroll
          for (int q = 0; q < RingDim<N>::W; ++q)
#pragma unroll
            for (int x = 0; x < WORDS; ++x) acc[i][(q + s) % N][x] ^= d[q][x];
        }
      }
    } else if constexpr (DISPATCH == 2) {
      ring_mac_pairs<N, WORDS>(acc[i], d, m);
    } else {
      uint32_t r = m;
      while (r) {
        const int s = __ffs(r) - 1;
        r &= r - 1;
        xor_rotated_dyn<N, WORDS>(acc[i], d, s);
      }
    }
  }
}

// Multiply-accumulate driven by the job's masks at run time (the generic kernels). Lane l holds
// the mask words of sources l and l + 32 for its group's outputs (one 16-byte row per source: the
// masks of outputs 0..7); each source's masks are broadcast from its lane by a warp OR-reduction,
// uniform across the warp by construction, which keeps the dispatch on uniform branches.
template <int MG, int DISPATCH>
struct MaskMac : DirectStore {
  static constexpr int MW = (MG + 1) / 2;  // 32-bit mask words per source for MG outputs
  uint32_t rw[2][MW];                      // [0]: source lane, [1]: source lane + 32

  // The group's mask words out of one source row.
  __device__ __forceinline__ static void group_words(const uint4& row, int g, uint32_t (&out)[MW]) {
    if constexpr (MG == 1) {
      // one output per warp: output g's mask is half (g & 1) of word g / 2
      const int wi = g >> 1;
      const uint32_t wv = wi == 0 ? row.x : wi == 1 ? row.y : wi == 2 ? row.z : row.w;
      out[0] = (wv >> (16 * (g & 1))) & 0xFFFFu;
    } else {
#pragma unroll
      for (int x = 0; x < MW; ++x) {
        const int idx = g * MW + x;
        out[x] = idx == 0 ? row.x : idx == 1 ? row.y : idx == 2 ? row.z : idx == 3 ? row.w : 0u;
      }
    }
  }

  __device__ __forceinline__ void tile(const JobDesc* J, int g, int lane) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint4 row = make_uint4(0u, 0u, 0u, 0u);
      if (lane + 32 * h < J->nin) row = *reinterpret_cast<const uint4*>(&J->mask[lane + 32 * h][0]);
      group_words(row, g, rw[h]);
    }
  }

  template <int N, int WORDS, int MG_>
  __device__ __forceinline__ void apply(uint32_t (&acc)[MG_][N][WORDS], const uint32_t (&d)[RingDim<N>::W][WORDS],
                                        int j, int, int lane) {
    const int h = j >> 5, jl = j & 31;  // warp-uniform
    uint32_t mu[MW];
#pragma unroll
    for (int x = 0; x < MW; ++x) mu[x] = __reduce_or_sync(0xFFFFFFFFu, lane == jl ? (h ? rw[1][x] : rw[0][x]) : 0u);
    ring_mac<N, WORDS, MG, DISPATCH>(acc, d, mu);
  }
};

template <int N, int WORDS, int MG, int MINB, int DISPATCH, int NC>
__global__ void __launch_bounds__((NC + 1) * 32, MINB) ring_staged_kernel(const __grid_constant__ CodeArgs a) {
  ring_staged_body<N, WORDS, MG, NC, MaskMac<MG, DISPATCH>>(a);
}

// Plain-load form for any packet size and alignment: one thread per byte column of one job, no
// staging. The same ring arithmetic on byte-wide lanes; all outputs per thread.
template <int N>
__global__ void __launch_bounds__(256) ring_plain_kernel(const __grid_constant__ JobDesc job) {
  constexpr int W = RingDim<N>::W, S = RingDim<N>::S;
  const uint64_t P = job.P;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < P; c += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t acc[kMaxOut][N][1];
#pragma unroll
    for (int i = 0; i < kMaxOut; ++i)
#pragma unroll
      for (int r = 0; r < N; ++r) acc[i][r][0] = 0u;
    for (int j = 0; j < job.nin; ++j) {
      uint32_t d[W][1];
#pragma unroll
      for (int q = 0; q < W; ++q) d[q][0] = job.in[j][(uint64_t)q * P + c];
      const uint4 row = *reinterpret_cast<const uint4*>(&job.mask[j][0]);
      const uint32_t mu[4] = {row.x, row.y, row.z, row.w};
      ring_mac<N, 1, kMaxOut, 1>(acc, d, mu);
    }
#pragma unroll
    for (int i = 0; i < kMaxOut; ++i) {
      if (i < job.nout) {
#pragma unroll
        for (int r = 0; r < W; ++r) job.out[i][(uint64_t)r * P + c] = (uint8_t)(acc[i][r][0] ^ acc[i][W + r % S][0]);
      }
    }
  }
}

}  // namespace pyrit
