// Stripe coding without any device allocation.
//
// Some callers cannot call cudaMalloc: a storage I/O path whose device memory is entirely reserved
// by another allocator (a framework's caching pool, or a pre-sized arena), where cudaMalloc fails
// or would steal from that pool; or a latency-bound request path that cannot afford cudaMalloc's
// implicit device synchronisation. The batched path allocates its job descriptors and tile list
// with cudaMalloc, and the library's error word is allocated on first use. This entry point keeps
// all of that scratch in one fixed file-scope device array instead, so it allocates nothing. The
// caller still passes every input and output buffer.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ring_kernel.cuh"

using namespace pyrit;

namespace {

constexpr int kNaMaxStripes = PYRIT_NOALLOC_MAX_STRIPES;
constexpr int kNaMaxTiles = PYRIT_NOALLOC_MAX_TILES;
constexpr size_t kNaStatusBytes = 256;
constexpr size_t kNaJobsBytes = sizeof(JobDesc) * kNaMaxStripes;
constexpr size_t kNaTilesBytes = sizeof(uint2) * kNaMaxTiles;
constexpr size_t kNaScratchBytes = kNaStatusBytes + kNaJobsBytes + kNaTilesBytes;
static_assert(kNaJobsBytes % 256 == 0, "tile list must stay 256-byte aligned");

// The scratch: [status words | job descriptors | tile list]. It is part of the module image, so
// every GPU that loads the library holds it until the process exits. Calls share it and it keeps
// the last call's contents.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNaScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;                     // serialises host callers (one host staging image)
uint8_t* g_scratch_dev[kMaxDevices];  // device address of g_noalloc_scratch, per device
JobDesc g_host_jobs[kNaMaxStripes];   // host staging of the descriptors (static: no allocation)
uint2 g_host_tiles[kNaMaxTiles];

// Device address of the scratch on the current device. Host code cannot use the array's name as
// a device address, so it is looked up once per device with that device current.
int scratch_address(uint8_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PYRIT_E_CUDA;
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PYRIT_E_CUDA;
    g_scratch_dev[dev] = static_cast<uint8_t*>(p);
  }
  *out = g_scratch_dev[dev];
  return PYRIT_OK;
}

// Rings the plain-load kernel is instantiated for (launch_plain).
bool plain_ring(int n) { return n == 3 || n == 5 || n == 9 || n == 11 || n == 13; }

// The one job of a stripe. The fixed kernels have no parity transform and only the native fields
// (those run only on generated networks), and a stripe with more than kMaxOut parity (or erased) blocks is several jobs, which
// the fixed scratch does not hold: both are PYRIT_E_UNSUPPORTED here.
int stripe_job(const pyrit_stripe_t& s, JobDesc* job) {
  JobDesc jobs[kMaxJobs];
  int nj = 0;
  uint64_t alg = 0, src = 0;
  const int rc = stripe_jobs(s, jobs, &nj, &alg, &src);
  if (rc != PYRIT_OK) return rc;
  if (network_only(s.plan) || nj > 1) return PYRIT_E_UNSUPPORTED;
  if (nj == 1)
    *job = jobs[0];
  else
    std::memset(job, 0, sizeof(*job));
  return PYRIT_OK;
}

}  // namespace

extern "C" int pyrit_code_stripes_noalloc(const pyrit_stripe_t* stripes, int count, pyrit_stream_t stream) {
  if (count < 0 || (count > 0 && !stripes)) return PYRIT_E_INVALID_ARG;
  if (count > kNaMaxStripes) return PYRIT_E_SCRATCH_LIMIT;
  if (count == 0) return PYRIT_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The descriptors are uploaded from static pageable host arrays that the next call rewrites: a
  // graph captured from this call could not replay it, so capture is refused.
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &capture) != cudaSuccess) {
    cudaGetLastError();
    return PYRIT_E_CUDA;
  }
  if (capture != cudaStreamCaptureStatusNone) return PYRIT_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  uint8_t* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != PYRIT_OK) return rc;

  // Validate every stripe and build its job before touching the device; stripes are grouped by
  // ring size (one staged launch per size) and odd sizes or alignments go to the plain kernel,
  // whose job travels in its launch parameters.
  static int ring_of[kNaMaxStripes];
  static bool staged[kNaMaxStripes];
  for (int i = 0; i < count; ++i) {
    rc = stripe_job(stripes[i], &g_host_jobs[i]);
    if (rc != PYRIT_OK) return rc;
    ring_of[i] = stripes[i].plan->n;
    staged[i] = g_host_jobs[i].nout > 0 && job_is_staged(g_host_jobs[i]);
    if (g_host_jobs[i].nout > 0 && !staged[i] && !plain_ring(ring_of[i])) return PYRIT_E_UNSUPPORTED_FIELD;
  }
  struct Launch {
    TileShape shape;
    uint32_t first_job, njobs, first_tile, ntiles;
  } launches[16];
  int nl = 0;
  uint32_t njobs = 0, ntiles = 0;
  static JobDesc sorted[kNaMaxStripes];
  for (int n = 0; n < 16; ++n) {
    uint32_t first = njobs;
    int max_nout = 0;
    for (int i = 0; i < count; ++i)
      if (staged[i] && ring_of[i] == n) {
        sorted[njobs++] = g_host_jobs[i];
        max_nout = max_nout > g_host_jobs[i].nout ? max_nout : g_host_jobs[i].nout;
      }
    if (njobs == first) continue;
    Launch L;
    if (!choose_shape(n, max_nout, ShapeHint(), &L.shape)) return PYRIT_E_UNSUPPORTED_FIELD;
    L.first_job = first;
    L.njobs = njobs - first;
    L.first_tile = ntiles;
    for (uint32_t j = first; j < njobs; ++j)
      for (uint64_t c = 0; c < sorted[j].P; c += (uint64_t)L.shape.tw) {
        if (ntiles >= (uint32_t)kNaMaxTiles) return PYRIT_E_SCRATCH_LIMIT;
        g_host_tiles[ntiles++] = make_uint2(j - first, (uint32_t)c);
      }
    L.ntiles = ntiles - L.first_tile;
    resolve_grid(&L.shape);
    launches[nl++] = L;
  }

  // Upload (pageable source: the copy is staged before the call returns, so the static host
  // image may be reused by the next call) and clear the status words, which must start at zero.
  uint8_t* jobs_dev = scratch + kNaStatusBytes;
  uint8_t* tiles_dev = jobs_dev + kNaJobsBytes;
  if (cudaMemsetAsync(scratch, 0, kNaStatusBytes, st) != cudaSuccess) return PYRIT_E_CUDA;
  if (njobs && cudaMemcpyAsync(jobs_dev, sorted, njobs * sizeof(JobDesc), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PYRIT_E_CUDA;
  if (ntiles && cudaMemcpyAsync(tiles_dev, g_host_tiles, ntiles * sizeof(uint2), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess)
    return PYRIT_E_CUDA;

  for (int l = 0; l < nl; ++l) {
    const Launch& L = launches[l];
    CodeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.jobs = reinterpret_cast<const JobDesc*>(jobs_dev) + L.first_job;
    a.tiles = reinterpret_cast<const uint2*>(tiles_dev) + L.first_tile;
    a.ntiles = L.ntiles;
    a.tiles_per_job = 0;
    a.tw = (uint32_t)L.shape.tw;
    a.groups = (uint32_t)L.shape.groups;
    a.stages = (uint32_t)L.shape.stages;
    a.err = reinterpret_cast<int*>(scratch);
    const size_t smem = staged_smem_bytes(L.shape.stages, L.shape.v->w, L.shape.tw);
    const int grid = (int)(L.ntiles < (uint32_t)L.shape.grid ? L.ntiles : (uint32_t)L.shape.grid);
    void* args[] = {&a};
    if (cudaLaunchKernel(L.shape.v->fn, dim3(grid), dim3((L.shape.v->nc + 1) * 32), args, smem, st) != cudaSuccess)
      return PYRIT_E_CUDA;
  }
  for (int i = 0; i < count; ++i)
    if (!staged[i] && g_host_jobs[i].nout > 0) {
      rc = launch_plain(ring_of[i], g_host_jobs[i], st);
      if (rc != PYRIT_OK) return rc;
    }
  return PYRIT_OK;
}

namespace {

// Bounded-wait self-test: thread 0 waits on an mbarrier that nothing arrives at, with the given
// limit, exactly as a pipeline wait does; it gives up and records PYRIT_E_TIMEOUT and kSelftestSite
// in `err`. The wait always ends (after limit_ns) and touches no memory but `err`.
constexpr int kSelftestSite = 100;

__global__ void bounded_wait_selftest_kernel(int* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_wait_for(&bar, 0u, err, kSelftestSite, limit_ns);
  }
}

}  // namespace

extern "C" int pyrit_noalloc_status(int* code_out, int* where_out, pyrit_stream_t stream) {
  if (!code_out) return PYRIT_E_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_mu);
  uint8_t* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != PYRIT_OK) return rc;
  int h[2] = {0, 0};
  // Ordered after the calls queued on `stream`; the copy into pageable host memory completes
  // before it returns, and the stream is synchronised once more before the words are cleared.
  if (cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PYRIT_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PYRIT_E_CUDA;
  if (cudaMemsetAsync(scratch, 0, sizeof(h), st) != cudaSuccess) return PYRIT_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PYRIT_E_CUDA;
  *code_out = h[0];
  if (where_out) *where_out = h[1];
  return PYRIT_OK;
}

extern "C" int pyrit_selftest_bounded_wait(int channel, uint64_t limit_ns, pyrit_stream_t stream) {
  if ((channel != 0 && channel != 1) || limit_ns == 0 || limit_ns > 1000000000ull) return PYRIT_E_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* err = nullptr;
  if (channel == 0) {
    err = device_error_word();
    if (!err) return PYRIT_E_CUDA;
  } else {
    std::lock_guard<std::mutex> lk(g_mu);
    uint8_t* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != PYRIT_OK) return rc;
    err = reinterpret_cast<int*>(scratch);
  }
  bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(err, limit_ns);
  return cudaGetLastError() == cudaSuccess ? PYRIT_OK : PYRIT_E_CUDA;
}
