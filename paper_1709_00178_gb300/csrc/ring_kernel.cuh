// The fused ring-transform coding kernels (paper Sec. 2.3.2 and Sec. 3).
//
// A coding job computes out[i] = sum_j u_ij in[j] over GF(2^w), w = N - 1, for every symbol lane
// of bit-sliced blocks (packet q of a block holds coefficient q). Each coefficient arrives as its
// ring representative r_ij = phi_S(u_ij) (an N-bit mask, Sec. 2.2). Per 32-bit column word the
// kernel:
//   1. embeds the source block in R_{2,N} (phi_E): its W packets plus an implicit zero packet;
//   2. for every set bit s of r_ij, XORs the source rotated by s packets into the N ring
//      accumulators of output i (x^s times a ring element is a cyclic shift of its coefficients;
//      the zero packet contributes nothing, so each set bit costs W XORs -- Sec. 3);
//   3. reduces each accumulator mod p (phi_E^{-1}): out[t] = acc[t] ^ acc[W] (Sec. 2.3.2), then
//      stores the W field packets.
// The extra ring packet is never written to memory, as in the paper's register scheme (Sec. 3).
//
// GB300 mapping (prior art: the paper's x86 SIMD register schedule). A CTA owns a column tile of
// `tw` bytes of one job. A producer warp streams the job's source blocks, one block (W packets
// x tw bytes, one lane per packet) per pipeline stage, into a shared-memory ring with bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier); NC consumer warps (8 or 16) read their 4*WORDS bytes
// of every packet into registers and release the stage, then run the XOR network out of registers.
// When a job has more outputs than one warp's accumulators hold (MG), the consumer warps split
// into output groups that read the same staged tile, so every source byte leaves HBM once.
#pragma once

#include <cuda_runtime.h>

#include "ptx.cuh"
#include "pyrit_internal.h"

namespace pyrit {


// acc += x^S * d in R_{2,N}: packet q of the embedded source lands in accumulator (q + S) mod N.
template <int N, int WORDS, int S>
__device__ __forceinline__ void xor_rotated(uint32_t (&acc)[N][WORDS], const uint32_t (&d)[N - 1][WORDS]) {
  if constexpr (S < N) {
#pragma unroll
    for (int q = 0; q < N - 1; ++q)
#pragma unroll
      for (int x = 0; x < WORDS; ++x) acc[(q + S) % N][x] ^= d[q][x];
  }
}

// acc += x^s * d for a run-time shift s < N. The rotation is resolved by a warp-uniform jump to
// straight-line code with static register indices (all lanes share the job, so no divergence).
template <int N, int WORDS>
__device__ __forceinline__ void xor_rotated_dyn(uint32_t (&acc)[N][WORDS], const uint32_t (&d)[N - 1][WORDS],
                                                int s) {
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
// (one three-input XOR), or a single term where the other index is the zero packet d[N-1].
template <int N, int WORDS, int S1, int S2>
__device__ __forceinline__ void xor_pair(uint32_t (&acc)[N][WORDS], const uint32_t (&d)[N - 1][WORDS]) {
  constexpr int W = N - 1;
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
__device__ __forceinline__ void ring_mac(uint32_t (&acc)[MG][N][WORDS], const uint32_t (&d)[N - 1][WORDS],
                                         const uint32_t (&mu)[(MG + 1) / 2]) {
#pragma unroll
  for (int i = 0; i < MG; ++i) {
    const uint32_t m = (mu[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
    if constexpr (DISPATCH == 0) {
#pragma unroll
      for (int s = 0; s < N; ++s) {
        if (m & (1u << s)) {
#pragma unroll
          for (int q = 0; q < N - 1; ++q)
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

__device__ __forceinline__ const JobDesc* tile_job(const CodeArgs& a, uint32_t t, uint32_t& col0) {
  uint32_t jid;
  if (a.tiles) {
    const uint2 v = a.tiles[t];
    jid = v.x;
    col0 = v.y;
  } else {
    jid = t / a.tiles_per_job;
    col0 = (t - jid * a.tiles_per_job) * a.tw;
  }
  return a.jobs ? a.jobs + jid : &a.job0;
}

template <int WORDS>
struct Vec;
template <>
struct Vec<1> {
  using T = uint32_t;
};
template <>
struct Vec<2> {
  using T = uint2;
};
template <>
struct Vec<4> {
  using T = uint4;
};

// Word x of a 1-, 2- or 4-word vector, and the vector of WORDS words.
template <int WORDS>
__device__ __forceinline__ uint32_t vword(const typename Vec<WORDS>::T& v, int x) {
  if constexpr (WORDS == 1) {
    return v;
  } else if constexpr (WORDS == 2) {
    return x == 0 ? v.x : v.y;
  } else {
    return x == 0 ? v.x : x == 1 ? v.y : x == 2 ? v.z : v.w;
  }
}
template <int WORDS>
__device__ __forceinline__ typename Vec<WORDS>::T vmake(const uint32_t (&w)[WORDS]) {
  if constexpr (WORDS == 1) {
    return w[0];
  } else if constexpr (WORDS == 2) {
    return make_uint2(w[0], w[1]);
  } else {
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int N, int WORDS, int MG, int MINB, int DISPATCH, int NC>
__global__ void __launch_bounds__((NC + 1) * 32, MINB) ring_staged_kernel(const __grid_constant__ CodeArgs a) {
  constexpr int W = N - 1;
  constexpr int MW = (MG + 1) / 2;  // 32-bit mask words per source for MG outputs
  using V = typename Vec<WORDS>::T;
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t S = a.stages, TW = a.tw;
  uint8_t* buf = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * W * TW);
  uint64_t* empty = full + S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == NC) {
    // ---- producer warp: streams source blocks into the stage ring --------------------------
    // Lane 0 waits for the stage to be free and arms its barrier with the stage's byte count;
    // then lane q issues the bulk copy of packet q, so the W copies of a stage leave together.
    const uint64_t pol = l2_evict_first_policy();
    uint32_t stage = 0, phase = 0;
    uint64_t armed = 0;  // stages armed so far
    bool ok = true;
    for (uint32_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      uint32_t col0;
      const JobDesc* J = tile_job(a, t, col0);
      const uint64_t P = J->P;
      if (col0 >= P) continue;  // a tiling that does not match the tile width codes nothing past P
      const uint32_t width = (uint32_t)(P - col0 < (uint64_t)TW ? P - col0 : (uint64_t)TW);
      const int nin = J->nin;
      for (int j = 0; j < nin; ++j) {
        bool free_ok = true;
        if (lane == 0) {
          free_ok = mbar_wait(&empty[stage], phase ^ 1u, a.err, 1);
          if (free_ok) mbar_arrive_expect_tx(&full[stage], (uint32_t)W * width);
        }
        ok = __all_sync(0xFFFFFFFFu, free_ok);  // also orders the arming before the copies
        if (!ok) break;
        if (lane < W)
          bulk_load(buf + ((size_t)stage * W + lane) * TW, J->in[j] + col0 + (size_t)lane * P, width, &full[stage], pol);
        ++armed;
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    // Drain: wait (bounded) until every copy this warp issued has landed, so that no bulk copy
    // is still writing shared memory when the CTA exits, on the normal and the error path alike.
    if (lane == 0)
      for (uint32_t s = 0; s < S; ++s) {
        if (armed <= s) break;
        const uint64_t times = (armed - 1 - s) / S + 1;
        mbar_wait(&full[s], (uint32_t)((times - 1) & 1u), a.err, 3);
      }
    return;
  }

  // ---- consumers -------------------------------------------------------------------------
  const int wpg = NC / (int)a.groups;  // warps per output group
  const int g = warp / wpg;
  const uint32_t off = (uint32_t)((warp % wpg) * 32 + lane) * (4u * WORDS);
  uint32_t stage = 0, phase = 0;
  for (uint32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    uint32_t col0;
    const JobDesc* J = tile_job(a, t, col0);
    const uint64_t P = J->P;
    if (col0 >= P) continue;  // same rule as the producer: such a tile has no stages
    const uint32_t width = (uint32_t)(P - col0 < (uint64_t)TW ? P - col0 : (uint64_t)TW);
    const bool valid = off < width;
    const int nin = J->nin, nout = J->nout;

    // Lane l holds the mask words of source l for this group's outputs (one 16-byte row per
    // source: the masks of outputs 0..7).
    uint32_t rw[MW];
    {
      uint4 row = make_uint4(0u, 0u, 0u, 0u);
      if (lane < nin) row = *reinterpret_cast<const uint4*>(&J->mask[lane][0]);
      if constexpr (MG == 1) {
        // one output per warp: output g's mask is half (g & 1) of word g / 2
        const int wi = g >> 1;
        const uint32_t wv = wi == 0 ? row.x : wi == 1 ? row.y : wi == 2 ? row.z : row.w;
        rw[0] = (wv >> (16 * (g & 1))) & 0xFFFFu;
      } else {
#pragma unroll
        for (int x = 0; x < MW; ++x) {
          const int idx = g * MW + x;
          rw[x] = idx == 0 ? row.x : idx == 1 ? row.y : idx == 2 ? row.z : idx == 3 ? row.w : 0u;
        }
      }
    }

    uint32_t acc[MG][N][WORDS];
#pragma unroll
    for (int i = 0; i < MG; ++i)
#pragma unroll
      for (int r = 0; r < N; ++r)
#pragma unroll
        for (int x = 0; x < WORDS; ++x) acc[i][r][x] = 0u;

    for (int j = 0; j < nin; ++j) {
      // Every lane observes the phase (so the staged bytes are visible to it); the give-up
      // decision is made warp-uniform before anyone leaves.
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(&full[stage], phase, a.err, 2))) return;
      uint32_t d[W][WORDS];
      const uint8_t* sb = buf + (size_t)stage * W * TW + off;
#pragma unroll
      for (int q = 0; q < W; ++q) {
        V v;
        if (valid) {
          v = *reinterpret_cast<const V*>(sb + (size_t)q * TW);
        } else {
          v = V{};
        }
#pragma unroll
        for (int x = 0; x < WORDS; ++x) d[q][x] = vword<WORDS>(v, x);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (++stage == S) {
        stage = 0;
        phase ^= 1u;
      }
      // Source j's masks, broadcast from lane j by a warp OR-reduction: the result is uniform
      // across the warp by construction, which keeps the dispatch below on uniform branches.
      uint32_t mu[MW];
#pragma unroll
      for (int x = 0; x < MW; ++x) mu[x] = __reduce_or_sync(0xFFFFFFFFu, lane == j ? rw[x] : 0u);
      ring_mac<N, WORDS, MG, DISPATCH>(acc, d, mu);
    }

    // phi_E^{-1}: reduce mod the AOP and store the W field packets of every output.
    if (valid) {
#pragma unroll
      for (int i = 0; i < MG; ++i) {
        const int o = g * MG + i;
        if (o < nout) {
          uint8_t* dst = J->out[o] + col0 + off;
#pragma unroll
          for (int r = 0; r < W; ++r) {
            uint32_t o4[WORDS];
#pragma unroll
            for (int x = 0; x < WORDS; ++x) o4[x] = acc[i][r][x] ^ acc[i][W][x];
            *reinterpret_cast<V*>(dst + (size_t)r * P) = vmake<WORDS>(o4);
          }
        }
      }
    }
  }
}

// Plain-load form for any packet size and alignment: one thread per byte column of one job, no
// staging. The same ring arithmetic on byte-wide lanes; all outputs per thread.
template <int N>
__global__ void __launch_bounds__(256) ring_plain_kernel(const __grid_constant__ JobDesc job) {
  constexpr int W = N - 1;
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
        for (int r = 0; r < W; ++r) job.out[i][(uint64_t)r * P + c] = (uint8_t)(acc[i][r][0] ^ acc[i][W][0]);
      }
    }
  }
}

}  // namespace pyrit
