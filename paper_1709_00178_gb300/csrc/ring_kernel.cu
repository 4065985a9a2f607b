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
// `tw` bytes of one job. One producer thread streams the job's source blocks, one block (W packets
// x tw bytes) per pipeline stage, into a shared-memory ring with bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier); NC consumer warps read their 4*WORDS bytes
// of every packet into registers and release the stage, then run the XOR network out of registers.
// When a job has more outputs than one warp's accumulators hold (MG), the consumer warps split
// into output groups that read the same staged tile, so every source byte leaves HBM once.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>

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

// acc_i += r_ij * d for every output i of the group: one rotation per set bit of r_ij.
template <int N, int WORDS, int MG>
__device__ __forceinline__ void ring_mac(uint32_t (&acc)[MG][N][WORDS], const uint32_t (&d)[N - 1][WORDS],
                                         const uint16_t (&msk)[MG]) {
#pragma unroll
  for (int i = 0; i < MG; ++i) {
    uint32_t m = msk[i];
    while (m) {
      const int s = __ffs(m) - 1;
      m &= m - 1;
      xor_rotated_dyn<N, WORDS>(acc[i], d, s);
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

template <int N, int WORDS, int MG, int NC>
__global__ void __launch_bounds__((NC + 1) * 32, 1) ring_staged_kernel(const __grid_constant__ CodeArgs a) {
  constexpr int W = N - 1;
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
    // ---- producer: one thread streams source blocks into the stage ring -------------------
    if (lane != 0) return;
    const uint64_t pol = l2_evict_first_policy();
    uint32_t stage = 0, phase = 0;
    uint64_t armed = 0;  // stages armed so far
    bool ok = true;
    for (uint32_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      uint32_t col0;
      const JobDesc* J = tile_job(a, t, col0);
      const uint64_t P = J->P;
      const uint32_t width = (uint32_t)(P - col0 < (uint64_t)TW ? P - col0 : (uint64_t)TW);
      const int nin = J->nin;
      for (int j = 0; j < nin; ++j) {
        if (!mbar_wait(&empty[stage], phase ^ 1u, a.err, 1)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[stage], (uint32_t)W * width);
        const uint8_t* src = J->in[j] + col0;
        uint8_t* dst = buf + (size_t)stage * W * TW;
#pragma unroll 1
        for (int q = 0; q < W; ++q) bulk_load(dst + (size_t)q * TW, src + (size_t)q * P, width, &full[stage], pol);
        ++armed;
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    // Drain: wait (bounded) until every copy this thread issued has landed, so that no bulk copy
    // is still writing shared memory when the CTA exits, on the normal and the error path alike.
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
    const uint32_t width = (uint32_t)(P - col0 < (uint64_t)TW ? P - col0 : (uint64_t)TW);
    const bool valid = off < width;
    const int nin = J->nin, nout = J->nout;

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
        if constexpr (WORDS == 1) {
          d[q][0] = v;
        } else {
          d[q][0] = v.x;
          d[q][1] = v.y;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (++stage == S) {
        stage = 0;
        phase ^= 1u;
      }
      // The ring masks of source j for this group's outputs (zero for outputs >= nout).
      const uint4 mv = *reinterpret_cast<const uint4*>(&J->mask[j][0]);
      const uint16_t all[8] = {(uint16_t)(mv.x & 0xFFFFu), (uint16_t)(mv.x >> 16), (uint16_t)(mv.y & 0xFFFFu),
                               (uint16_t)(mv.y >> 16),     (uint16_t)(mv.z & 0xFFFFu), (uint16_t)(mv.z >> 16),
                               (uint16_t)(mv.w & 0xFFFFu), (uint16_t)(mv.w >> 16)};
      uint16_t msk[MG];
#pragma unroll
      for (int i = 0; i < MG; ++i) {
        const int o = g * MG + i;
        msk[i] = (o < kMaxOut) ? all[o & (kMaxOut - 1)] : (uint16_t)0;
      }
      ring_mac<N, WORDS, MG>(acc, d, msk);
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
            V v;
            if constexpr (WORDS == 1) {
              v = acc[i][r][0] ^ acc[i][W][0];
            } else {
              v = make_uint2(acc[i][r][0] ^ acc[i][W][0], acc[i][r][1] ^ acc[i][W][1]);
            }
            *reinterpret_cast<V*>(dst + (size_t)r * P) = v;
          }
        }
      }
    }
  }
}

// Plain-load form for any packet size and alignment: one thread per byte column of one job, no
// staging. The same ring arithmetic on byte-wide lanes.
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
      uint16_t msk[kMaxOut];
#pragma unroll
      for (int i = 0; i < kMaxOut; ++i) msk[i] = job.mask[j][i];
      ring_mac<N, 1, kMaxOut>(acc, d, msk);
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

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------

namespace {

constexpr int kConsumerWarps = 8;
constexpr int kMaxDevices = 64;

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

// Per-kernel, per-device one-time setup (shared-memory opt-in) and occupancy.
struct KernelInfo {
  std::once_flag once[kMaxDevices];
  int max_smem_set[kMaxDevices];
};

template <int N, int WORDS, int MG>
int launch_staged_t(const TileShape& sh, const CodeArgs& args, int grid, cudaStream_t st) {
  auto kern = ring_staged_kernel<N, WORDS, MG, kConsumerWarps>;
  static KernelInfo info;
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return PYRIT_E_CUDA;
  std::call_once(info.once[dev], [&] {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  const size_t smem = (size_t)sh.stages * (N - 1) * sh.tw + 2 * sh.stages * sizeof(uint64_t);
  kern<<<grid, (kConsumerWarps + 1) * 32, smem, st>>>(args);
  return cudaGetLastError() == cudaSuccess ? PYRIT_OK : PYRIT_E_CUDA;
}

template <int N, int WORDS, int MG>
int occupancy_t(const TileShape& sh) {
  auto kern = ring_staged_kernel<N, WORDS, MG, kConsumerWarps>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  const size_t smem = (size_t)sh.stages * (N - 1) * sh.tw + 2 * sh.stages * sizeof(uint64_t);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, (kConsumerWarps + 1) * 32, smem) != cudaSuccess)
    return 1;
  return std::max(nb, 1);
}

// Outputs held per consumer warp, by ring size (register budget: MG * N * WORDS accumulators).
constexpr int mg_for(int n) { return n <= 5 ? 8 : 4; }

}  // namespace

int sm_count() {
  static int cache[kMaxDevices] = {0};
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return 1;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

int* device_error_word() {
  static int* words[kMaxDevices] = {nullptr};
  static std::mutex mu;
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!words[dev]) {
    int* p = nullptr;
    if (cudaMalloc(&p, 2 * sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, 2 * sizeof(int)) != cudaSuccess) return nullptr;
    words[dev] = p;
  }
  return words[dev];
}

bool job_is_staged(const JobDesc& j) {
  if (j.P % 16 != 0) return false;
  for (int i = 0; i < j.nin; ++i)
    if (reinterpret_cast<uintptr_t>(j.in[i]) % 16 != 0) return false;
  for (int i = 0; i < j.nout; ++i)
    if (reinterpret_cast<uintptr_t>(j.out[i]) % 16 != 0) return false;
  return true;
}

TileShape default_shape(int n, int max_nout, size_t P) {
  (void)P;
  TileShape s;
  s.words = 2;
  s.warps = kConsumerWarps;
  const int mg = mg_for(n);
  s.groups = std::max(1, std::min(kMaxOut / mg, (max_nout + mg - 1) / mg));
  s.tw = (s.warps / s.groups) * 32 * 4 * s.words;
  const int w = n - 1;
  // Stage ring of about 96 KiB so that two CTAs share an SM.
  s.stages = std::max(2, std::min(8, (96 * 1024) / (w * s.tw)));
  s.ctas_per_sm = 0;
  return s;
}

int launch_staged(int n, const TileShape& sh, const JobDesc* job0, const JobDesc* jobs_dev, const uint2* tiles_dev,
                  uint32_t ntiles, uint32_t tiles_per_job, int grid_ctas, cudaStream_t stream) {
  if (ntiles == 0) return PYRIT_OK;
  CodeArgs a;
  a.jobs = jobs_dev;
  a.tiles = tiles_dev;
  a.ntiles = ntiles;
  a.tiles_per_job = tiles_per_job;
  a.tw = (uint32_t)sh.tw;
  a.groups = (uint32_t)sh.groups;
  a.stages = (uint32_t)sh.stages;
  a.err = device_error_word();
  if (job0)
    a.job0 = *job0;
  else
    memset(&a.job0, 0, sizeof(a.job0));
  int occ = sh.ctas_per_sm;
  if (occ <= 0) {
    switch (n) {
      case 3: occ = occupancy_t<3, 2, mg_for(3)>(sh); break;
      case 5: occ = occupancy_t<5, 2, mg_for(5)>(sh); break;
      case 11: occ = occupancy_t<11, 2, mg_for(11)>(sh); break;
      case 13: occ = occupancy_t<13, 2, mg_for(13)>(sh); break;
      default: return PYRIT_E_UNSUPPORTED_FIELD;
    }
  }
  int grid = grid_ctas > 0 ? grid_ctas : sm_count() * occ;
  grid = (int)std::min<uint32_t>((uint32_t)grid, ntiles);
  switch (n) {
    case 3: return launch_staged_t<3, 2, mg_for(3)>(sh, a, grid, stream);
    case 5: return launch_staged_t<5, 2, mg_for(5)>(sh, a, grid, stream);
    case 11: return launch_staged_t<11, 2, mg_for(11)>(sh, a, grid, stream);
    case 13: return launch_staged_t<13, 2, mg_for(13)>(sh, a, grid, stream);
    default: return PYRIT_E_UNSUPPORTED_FIELD;
  }
}

int launch_plain(int n, const JobDesc& job, cudaStream_t stream) {
  if (job.P == 0 || job.nout == 0) return PYRIT_OK;
  const uint64_t blocks64 = (job.P + 255) / 256;
  const int grid = (int)std::min<uint64_t>(blocks64, (uint64_t)sm_count() * 8);
  switch (n) {
    case 3: ring_plain_kernel<3><<<grid, 256, 0, stream>>>(job); break;
    case 5: ring_plain_kernel<5><<<grid, 256, 0, stream>>>(job); break;
    case 11: ring_plain_kernel<11><<<grid, 256, 0, stream>>>(job); break;
    case 13: ring_plain_kernel<13><<<grid, 256, 0, stream>>>(job); break;
    default: return PYRIT_E_UNSUPPORTED_FIELD;
  }
  return cudaGetLastError() == cudaSuccess ? PYRIT_OK : PYRIT_E_CUDA;
}

}  // namespace pyrit
