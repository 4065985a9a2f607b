// The staged ring-transform coding pipeline (paper Sec. 2.3.2 and Sec. 3), shared by the generic
// kernels (compiled by nvcc) and the plan-specialised ones (generated at run time and compiled by
// NVRTC). It is written for both compilers: no standard headers, only ring_abi.h and ptx.cuh.
//
// A coding job computes out[i] = sum_j u_ij in[j] over GF(2^w), w = RingDim<N>::W (N - 1 for an
// all-one polynomial, 6 for N = 9), for every symbol lane of bit-sliced blocks (packet q of a
// block holds coefficient q). Each coefficient arrives as its ring representative
// r_ij = phi_S(u_ij) (an N-bit mask, Sec. 2.2). Per 32-bit column word the pipeline:
//   1. embeds the source block in R_{2,N} (phi_E): its W packets plus S = N - W implicit zero
//      packets;
//   2. for every set bit s of r_ij, XORs the source rotated by s packets into the N ring
//      accumulators of output i (x^s times a ring element is a cyclic shift of its coefficients;
//      the zero packets contribute nothing, so each set bit costs W XORs -- Sec. 3); this step is
//      the policy `Mac`, either driven by the masks at run time or a network fixed at compile time;
//   3. reduces each accumulator mod the field's modulus (phi_E^{-1}): out[t] = acc[t] ^
//      acc[W + t mod S] (Sec. 2.3.2 for S = 1, Sec. 2.4.2 for the ESP), then stores the W field
//      packets.
// The extra ring packets are never written to memory, as in the paper's register scheme (Sec. 3).
//
// GB300 mapping (prior art: the paper's x86 SIMD register schedule). A CTA owns a column tile of
// `tw` bytes of one job. A producer warp streams the job's source blocks, one block (W packets
// x tw bytes, one lane per packet) per pipeline stage, into a shared-memory ring with bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier); NC consumer warps read
// their 4*WORDS bytes of every packet into registers and release the stage, then run the XOR
// network out of registers. When a job has more outputs than one warp's accumulators hold (MG),
// the consumer warps split into output groups that read the same staged tile, so every source
// byte leaves HBM once.
//
// The policy Mac provides, per consumer warp:
//   void tile(const JobDesc* J, int g, int lane);      // once per tile (e.g. load the masks)
//   template <int N, int WORDS, int MG>
//   void apply(uint32_t (&acc)[MG][N][WORDS], const uint32_t (&d)[RingDim<N>::W][WORDS], int j,
//              int g, int lane);                      // acc_i += r_ij * d for the group's outputs
//   template <int N, int WORDS, int MG>
//   void apply2(acc, d, d2, j, g, lane);                // sources j and j + 1 together (only for
//                                                      // a body instantiated with PAIR)
//   template <int N, int WORDS, int MG>
//   void store(uint32_t (&acc)[MG][N][WORDS], const JobDesc* J, int g, uint32_t col0,
//              uint32_t off, bool valid);              // phi_E^{-1} and the stores of the tile;
//                                                      // called by every lane (warp-collective
//                                                      // steps allowed), stores only if valid
//   static constexpr bool kSparse;                     // sources with a null pointer are absent
// DirectStore supplies the usual store (output g*MG + i is acc[i] reduced) and kSparse = false.
#pragma once

#include "ptx.cuh"
#include "ring_abi.h"

namespace pyrit {

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

// A value every lane of a warp reads from the same job descriptor, broadcast from lane 0 (called
// by all 32 lanes): the compiler then knows it warp-uniform and keeps tests and branches on it on
// the uniform datapath. Used where a warp branches on descriptor values many times per tile (the
// syndrome decode's second phase: on GB300 the decode 3.5% faster for GF(2^10) k=10 m=4 and 7%
// for GF(2^12) k=16 m=4; broadcasting every descriptor read instead cost the encodes up to 2%).
__device__ __forceinline__ uint32_t warp_uniform(uint32_t v) { return __shfl_sync(0xFFFFFFFFu, v, 0); }

// a ^ b ^ c in one three-input logic instruction (truth table 0x96). Generated networks spell
// their XORs this way so that each instruction absorbs two source terms.
__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
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

// phi_E^{-1} and the stores of a direct job: output g*MG + i is acc[i] reduced mod the field's
// modulus (out[t] = acc[t] ^ acc[W + t mod S]); its W field packets are stored at col0 + off.
struct DirectStore {
  static constexpr bool kSparse = false;

  template <int N, int WORDS, int MG>
  __device__ __forceinline__ void store(uint32_t (&acc)[MG][N][WORDS], const JobDesc* J, int g, uint32_t col0,
                                        uint32_t off, bool valid) {
    constexpr int W = RingDim<N>::W, S = RingDim<N>::S;
    using V = typename Vec<WORDS>::T;
    if (!valid) return;
    const uint64_t P = J->P;
    const int nout = J->nout;
#pragma unroll
    for (int i = 0; i < MG; ++i) {
      const int o = g * MG + i;
      if (o < nout) {
        uint8_t* dst = J->out[o] + col0 + off;
#pragma unroll
        for (int r = 0; r < W; ++r) {
          uint32_t o4[WORDS];
#pragma unroll
          for (int x = 0; x < WORDS; ++x) o4[x] = acc[i][r][x] ^ acc[i][W + r % S][x];
          *reinterpret_cast<V*>(dst + (size_t)r * P) = vmake<WORDS>(o4);
        }
      }
    }
  }
};

// Syndrome-form decoding (the second phase of a decode network; the first phase is a network for
// the plan's parity-check matrix H = [C | I_m], which depends only on the plan).
//
// A systematic code has parity p_r = sum_j C_rj d_j. When blocks E are lost, decoding reads the
// survivors S = the first k blocks not in E: the surviving data D_s and the first a surviving
// parity rows U (a = number of lost data blocks). The first phase accumulates, for every parity
// row r, acc_r = sum over j in D_s of C_rj d_j, plus p_r when r is in U. For r in U this is the
// syndrome s_r = sum over lost data j of C_rj d_j; for a lost parity row r it is the partial sum
// t_r over the surviving data. Then (Sec. 4.3: the decoding matrix depends on the loss pattern)
//   lost data     d_E = X s_U,            X = (C restricted to rows U, lost data columns)^{-1}
//   lost parity   p_r = t_r + (C_{r, lost data} X) s_U,
// every square submatrix of C being invertible for an MDS code. The small per-pattern matrices
// arrive in the job: for output o, mask[r][o] (r < MG) is phi_S of the coefficient of acc_r and
// mask[kSyndromeBaseRow][o] is 1 + the row whose partial sum is added (0: none). Rows are first
// reduced in place (phi_E^{-1}), products are formed in the ring with the reduced rows embedded
// (phi_E), and each output is reduced once more before its store.
// PSI: the jobs code under the parity transform (Sec. 2.3.1, Sec. 2.4.1). The first phase's rows
// then reduce to field values in the psi domain (psi(d) = phi_P(d) mod the field's modulus:
// coefficient t of d plus the parity of its interleaved word t mod S, i.e. for an AOP
// d + par(d) (1 + ... + x^{W-1}), for the ESP the swap of d's two halves), the second phase is the
// same linear algebra there, and each output finally goes through psi^{-1} = psi (an involution):
// the parity of each interleaved word is XORed into that word's packets.
template <bool PSI>
struct SyndromeStoreT {
  static constexpr bool kSparse = true;  // erased columns and unused parity are absent sources
  uint32_t need;                         // rows the pattern uses (read once per tile)

  __device__ __forceinline__ void load_rows(const JobDesc* J) { need = warp_uniform(J->mask[kSyndromeNeedRow][0]); }

  template <int N, int WORDS, int MG>
  __device__ __forceinline__ void store(uint32_t (&acc)[MG][N][WORDS], const JobDesc* J, int, uint32_t col0,
                                        uint32_t off, bool valid) {
    // lanes past the tile's width take part in nothing here but the stores they skip
    constexpr int W = RingDim<N>::W, S = RingDim<N>::S;
    using V = typename Vec<WORDS>::T;
#pragma unroll
    for (int r = 0; r < MG; ++r) {
      if (!(need & (1u << r))) continue;  // rows the pattern does not use are never read
#pragma unroll
      for (int t = 0; t < W; ++t)
#pragma unroll
        for (int x = 0; x < WORDS; ++x) acc[r][t][x] ^= acc[r][W + t % S][x];
    }
    const uint64_t P = ((uint64_t)warp_uniform((uint32_t)(J->P >> 32)) << 32) | warp_uniform((uint32_t)J->P);
    // (the output count, packet size and output pointers are broadcast too: measured on GB300,
    // the config-2 decode's best shape 2.8% faster, the GF(2^12) k=16 m=4 decode within 1%)
    const int nout = (int)warp_uniform((uint32_t)J->nout);
    for (int o = 0; o < nout; ++o) {
      const uint32_t base = warp_uniform(J->mask[kSyndromeBaseRow][o]);
      uint32_t res[N][WORDS];
#pragma unroll
      for (int t = 0; t < N; ++t)
#pragma unroll
        for (int x = 0; x < WORDS; ++x) res[t][x] = 0u;
#pragma unroll
      for (int r = 0; r < MG; ++r) {
        if (base == (uint32_t)(r + 1)) {
#pragma unroll
          for (int t = 0; t < W; ++t)
#pragma unroll
            for (int x = 0; x < WORDS; ++x) res[t][x] = acc[r][t][x];
        }
      }
#pragma unroll
      for (int r = 0; r < MG; ++r) {
        const uint32_t c = warp_uniform(J->mask[r][o]);
        if (c == 0u) continue;
        // res += c * acc_r: one rotation of the reduced row per set bit of c
#pragma unroll
        for (int sh = 0; sh < N; ++sh) {
          if (c & (1u << sh)) {
#pragma unroll
            for (int q = 0; q < W; ++q)
#pragma unroll
              for (int x = 0; x < WORDS; ++x) res[(q + sh) % N][x] ^= acc[r][q][x];
          }
        }
      }
      const uintptr_t dp = reinterpret_cast<uintptr_t>(J->out[o]);
      uint8_t* dst = reinterpret_cast<uint8_t*>(((uint64_t)warp_uniform((uint32_t)((uint64_t)dp >> 32)) << 32) |
                                                warp_uniform((uint32_t)(uint64_t)dp)) + col0 + off;
      if (valid) {
        uint32_t par[S][WORDS];
#pragma unroll
        for (int j = 0; j < S; ++j)
#pragma unroll
          for (int x = 0; x < WORDS; ++x) par[j][x] = 0u;
        if constexpr (PSI) {
#pragma unroll
          for (int t = 0; t < W; ++t)
#pragma unroll
            for (int x = 0; x < WORDS; ++x) par[t % S][x] ^= res[t][x] ^ res[W + t % S][x];
        }
#pragma unroll
        for (int t = 0; t < W; ++t) {
          uint32_t o4[WORDS];
#pragma unroll
          for (int x = 0; x < WORDS; ++x) o4[x] = res[t][x] ^ res[W + t % S][x] ^ par[t % S][x];
          *reinterpret_cast<V*>(dst + (size_t)t * P) = vmake<WORDS>(o4);
        }
      }
    }
  }
};
using SyndromeStore = SyndromeStoreT<false>;
using SyndromePsiStore = SyndromeStoreT<true>;

// phi_P^{-1} and the stores of a direct job under the parity transform (Sec. 2.3.1, Sec. 2.4.1):
// every source entered the ring padded with its parity packets, so each ring result lies in the
// ideal A_1 and its field packets are its first W coefficients (the top S are dropped, never
// computed).
struct ParityStore {
  static constexpr bool kSparse = false;

  template <int N, int WORDS, int MG>
  __device__ __forceinline__ void store(uint32_t (&acc)[MG][N][WORDS], const JobDesc* J, int g, uint32_t col0,
                                        uint32_t off, bool valid) {
    constexpr int W = RingDim<N>::W;
    using V = typename Vec<WORDS>::T;
    if (!valid) return;
    const uint64_t P = J->P;
    const int nout = J->nout;
#pragma unroll
    for (int i = 0; i < MG; ++i) {
      const int o = g * MG + i;
      if (o < nout) {
        uint8_t* dst = J->out[o] + col0 + off;
#pragma unroll
        for (int r = 0; r < W; ++r) *reinterpret_cast<V*>(dst + (size_t)r * P) = vmake<WORDS>(acc[i][r]);
      }
    }
  }
};

// W: the field's degree, the packets of a block (the native field of R_{2,N} by default; a
// generated network for another factor of x^N + 1 passes its own, with its own reduction).
// PAIR: consumers take two staged sources per step (Mac::apply2), for generated networks whose
// every source is present (direct networks of wide jobs).
// TRACK: the kernel counts each job's finished tiles and stamps its completion when the launch
// passes CodeArgs::done_cnt (the served path). It is a compile-time choice because the code, even
// never executed, costs the other launches: on GB300 the GF(2^12) k=16 m=4 encode ran 3-6% slower
// with it compiled in.
template <int N, int WORDS, int MG, int NC, class Mac, int W = RingDim<N>::W, bool TRACK = false,
          bool PAIR = false>
__device__ __forceinline__ void ring_staged_body(const CodeArgs& a) {
  static_assert(!(PAIR && Mac::kSparse), "source pairs need every source present");
  using V = typename Vec<WORDS>::T;
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t S = a.stages, TW = a.tw;
  uint8_t* buf = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * W * TW);
  uint64_t* empty = full + S;
  uint64_t* tdone = empty + S;  // consumer warps finished with the tile (served launches)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC);
    }
    mbar_init(tdone, NC);
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
        if constexpr (Mac::kSparse) {
          if (J->in[j] == nullptr) continue;
        }
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
  uint32_t stage = 0, phase = 0, tphase = 0;
  for (uint32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    uint32_t col0;
    const JobDesc* J = tile_job(a, t, col0);
    const uint64_t P = J->P;
    if (col0 >= P) continue;  // same rule as the producer: such a tile has no stages
    const uint32_t width = (uint32_t)(P - col0 < (uint64_t)TW ? P - col0 : (uint64_t)TW);
    const bool valid = off < width;
    const int nin = J->nin;

    Mac mac;
    mac.tile(J, g, lane);

    uint32_t acc[MG][N][WORDS];
#pragma unroll
    for (int i = 0; i < MG; ++i)
#pragma unroll
      for (int r = 0; r < N; ++r)
#pragma unroll
        for (int x = 0; x < WORDS; ++x) acc[i][r][x] = 0u;

    // Takes the next stage: every lane observes its phase (so the staged bytes are visible to it;
    // the give-up decision is made warp-uniform before anyone leaves), reads its words of the W
    // packets into registers and releases the stage. False when the wait gave up.
    auto take_stage = [&](uint32_t (&dst)[W][WORDS]) -> bool {
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(&full[stage], phase, a.err, 2))) return false;
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
        for (int x = 0; x < WORDS; ++x) dst[q][x] = vword<WORDS>(v, x);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (++stage == S) {
        stage = 0;
        phase ^= 1u;
      }
      return true;
    };

    for (int j = 0; j < nin; ++j) {
      if constexpr (Mac::kSparse) {
        if (J->in[j] == nullptr) continue;  // the producer staged nothing for it either
      }
      uint32_t d[W][WORDS];
      if (!take_stage(d)) return;
      if constexpr (PAIR) {
        // the next source too (the producer streams every source of the job in order)
        if (j + 1 < nin) {
          uint32_t d2[W][WORDS];
          if (!take_stage(d2)) return;
          mac.template apply2<N, WORDS, MG>(acc, d, d2, j, g, lane);
          ++j;
          continue;
        }
      }
      mac.template apply<N, WORDS, MG>(acc, d, j, g, lane);
    }

    mac.template store<N, WORDS, MG>(acc, J, g, col0, off, valid);

    if (TRACK && a.done_cnt) {
      // Per-job completion: each consumer warp releases its stores to the CTA on the tile barrier;
      // consumer warp 0 acquires them all and counts the tile once at device scope (release); the
      // count that completes the job (its tiles) acquires the other CTAs' stores, leaves the
      // counter at zero for the next launch and stamps the job done in host memory after a
      // system-scope fence.
      __syncwarp();
      if (lane == 0) mbar_arrive(tdone);
      if (warp == 0 && lane == 0 && mbar_wait(tdone, tphase, a.err, 4)) {
        const uint32_t jid = a.tiles ? a.tiles[t].x : t / a.tiles_per_job;
        const uint64_t Pj = J->P;
        const uint32_t target = (uint32_t)((Pj + TW - 1) / TW);
        if (count_release_gpu(&a.done_cnt[jid]) + 1u == target) {
          fence_acq_rel_gpu();
          a.done_cnt[jid] = 0u;
          fence_acq_rel_sys();
          const uint64_t now = global_timer_ns();
          *reinterpret_cast<volatile uint64_t*>(&a.done_ns[jid]) = now ? now : 1ull;
        }
      }
      tphase ^= 1u;
    }
  }
}

}  // namespace pyrit
