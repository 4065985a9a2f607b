// Synthetic input generator (no coding arithmetic): counter-mode SplitMix64 (Steele, Lea, Flood,
// OOPSLA 2014). Word i of stream `seed` is mix(seed + (i + 1) * gamma); bytes are little-endian.
#include <cuda_runtime.h>

#include "pyrit_internal.h"

namespace {

__device__ __forceinline__ uint64_t splitmix64_word(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One thread per destination 8-byte chunk; the stream offset need not be aligned to 8.
__global__ void synth_fill_kernel(uint8_t* dst, uint64_t nbytes, uint64_t seed, uint64_t offset) {
  const uint64_t nchunk = (nbytes + 7) / 8;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunk; c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b0 = offset + c * 8;  // stream byte of dst[c * 8]
    const uint64_t wi = b0 >> 3;
    const unsigned sh = (unsigned)(b0 & 7u);
    const uint64_t lo = splitmix64_word(seed, wi);
    const uint64_t v = sh ? ((lo >> (8 * sh)) | (splitmix64_word(seed, wi + 1) << (64 - 8 * sh))) : lo;
    const uint64_t base = c * 8;
    if (base + 8 <= nbytes && (reinterpret_cast<uintptr_t>(dst + base) & 7u) == 0) {
      *reinterpret_cast<uint64_t*>(dst + base) = v;
    } else {
      for (unsigned k = 0; k < 8 && base + k < nbytes; ++k) dst[base + k] = (uint8_t)(v >> (8 * k));
    }
  }
}

}  // namespace

extern "C" int pyrit_synth_fill(void* dst, size_t nbytes, uint64_t seed, uint64_t offset, pyrit_stream_t stream) {
  if (nbytes == 0) return PYRIT_OK;
  if (!dst) return PYRIT_E_INVALID_ARG;
  const uint64_t nchunk = (nbytes + 7) / 8;
  const int grid = (int)(nchunk / 256 + 1 < 65536 ? nchunk / 256 + 1 : 65536);
  synth_fill_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(static_cast<uint8_t*>(dst), nbytes,
                                                                              seed, offset);
  return cudaGetLastError() == cudaSuccess ? PYRIT_OK : PYRIT_E_CUDA;
}
