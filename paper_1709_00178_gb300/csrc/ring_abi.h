// Plain-data types shared by the host library and every device compilation of the ring kernels:
// nvcc for the generic kernels and the run-time compiler (NVRTC) for plan-specialised networks.
// Both compilers see this exact text, so the layouts agree by construction.
#pragma once

#ifdef __CUDACC_RTC__
// The run-time compiler has no C++ standard headers; LP64 (x86_64 and aarch64 Linux) widths.
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long uint64_t;
typedef unsigned long uintptr_t;
#else
#include <cstddef>
#include <cstdint>
#include <vector_types.h>
#endif

namespace pyrit {

// Ring sizes and field degrees. GF(2^w) is carried by R_{2,n}: n = w + 1 for a field defined by
// the all-one polynomial of degree w (Sec. 2.3), n = 9 for GF(2^6) defined by the equally spaced
// polynomial x^6 + x^3 + 1 (Sec. 2.4: n = s (r + 1), w = s r, s = 3, r = 2). The S = n - w top
// ring coefficients are the ones the embedding pads with zeros; reduction mod the field's modulus
// folds coefficient w + j into every coefficient t < w with t = j (mod S).
template <int N>
struct RingDim {
  static constexpr int W = N == 9 ? 6 : N - 1;
  static constexpr int S = N - W;
};

constexpr int kMaxIn = 64;  // sources of one coding job (data blocks or survivors)
constexpr int kMaxOut = 8;  // destinations of one coding job (a stripe's outputs split into jobs of 8)
// Syndrome-form decode jobs keep, for output o, 1 + the row of their partial sum (0: none) in
// mask[kSyndromeBaseRow][o]; rows 0..kMaxOut-1 hold the per-row coefficients.
constexpr int kSyndromeBaseRow = kMaxOut;
// ... and in mask[kSyndromeNeedRow][0] the bit set of parity rows whose accumulators are used.
constexpr int kSyndromeNeedRow = kMaxOut + 1;

// One coding job: out[i] = sum_j u_ij * in[j] over GF(2^w) in every symbol lane, where the
// coefficient u_ij is given by its ring representative mask[j][i] (bit s = coefficient of x^s).
// Encoding a stripe is the job (data -> parity, the generator's parity rows); decoding is the job
// (survivors -> erased blocks, the decoding matrix). Lives in kernel parameters or device memory.
struct alignas(16) JobDesc {
  const uint8_t* in[kMaxIn];
  uint8_t* out[kMaxOut];
  uint16_t mask[kMaxIn][kMaxOut];  // source-major so one 16-byte load gives every output's mask
  uint64_t P;                      // packet bytes
  int32_t nin, nout;
  int32_t table;                   // which table of a multi-table generated network codes this job
  int32_t reserved;
};

// Launch arguments of the staged ring kernel. Tiles are (job, column range [col0, col0 + tw)).
// With tiles == nullptr every job has the same P and tiles_per_job = ceil(P / tw) tiles, tile t
// covering job t / tiles_per_job.
struct CodeArgs {
  const JobDesc* jobs;  // device array; nullptr: the single job `job0`
  const uint2* tiles;   // optional explicit tile list {job, col0}
  uint32_t ntiles;
  uint32_t tiles_per_job;
  uint32_t tw;          // tile width in bytes (multiple of 16)
  uint32_t groups;      // consumer warps are split into this many output groups
  uint32_t stages;      // shared-memory pipeline depth
  int* err;             // device error word (code, site) or nullptr
  // Per-job completion (the served path; nullptr elsewhere). done_cnt[j] counts the consumer warps
  // that have stored job j's tiles (device memory, zero before the launch and left zero after it);
  // the warp completing the count writes the global timer into done_ns[j] (host-mapped memory).
  uint32_t* done_cnt;
  uint64_t* done_ns;
  JobDesc job0;
};

}  // namespace pyrit
