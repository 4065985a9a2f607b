// Host side of the ring kernels: variant registry, tile-shape choice, launches, the device error
// word and the plain-load kernel's instantiations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "ring_kernel.cuh"

namespace pyrit {

const Variant* variants_small(int* count);
const Variant* variants_n9(int* count);
const Variant* variants_n11(int* count);
const Variant* variants_n13(int* count);

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxVariants = 64;

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

struct Registry {
  Variant all[kMaxVariants];
  int count = 0;
  Registry() {
    const Variant* (*srcs[])(int*) = {variants_small, variants_n9, variants_n11, variants_n13};
    for (auto f : srcs) {
      int c = 0;
      const Variant* t = f(&c);
      for (int i = 0; i < c && count < kMaxVariants; ++i) all[count++] = t[i];
    }
  }
};

const Registry& registry() {
  static Registry r;
  return r;
}

// One-time per (kernel, device) opt-in to the large dynamic shared-memory carve-out; kernels are
// the registered variants and the loaded generated networks.
std::mutex g_attr_mu;
std::set<std::pair<const void*, int>> g_attr_done;

void ensure_attr(const Variant* v) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done.insert({v->fn, dev}).second)
    cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

size_t smem_bytes(const TileShape& s) { return staged_smem_bytes(s.stages, s.v->w, s.tw); }

int occupancy(const TileShape& s) {
  ensure_attr(s.v);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, s.v->fn, (s.v->nc + 1) * 32, smem_bytes(s)) !=
      cudaSuccess)
    return 1;
  return std::max(nb, 1);
}

}  // namespace

const Variant* variants(int* count) {
  *count = registry().count;
  return registry().all;
}

const Variant* find_variant(int n, int words, int dispatch, int mg, int minb, int nc) {
  const Registry& r = registry();
  const Variant* best = nullptr;
  for (int i = 0; i < r.count; ++i) {
    const Variant& v = r.all[i];
    if (v.n != n || (words && v.words != words) || (dispatch >= 0 && v.dispatch != dispatch) || (mg && v.mg != mg) ||
        (minb && v.minb != minb) || (nc && v.nc != nc))
      continue;
    if (!best) best = &v;  // the first registered match is the preferred one
  }
  return best;
}

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

bool shape_for_variant(const Variant* v, int max_nout, const ShapeHint& h, TileShape* out) {
  if (!v) return false;
  TileShape s;
  s.v = v;
  const int groups = output_groups(v->mg, max_nout, v->nc);
  s.groups = groups;
  s.tw = (v->nc / groups) * 32 * 4 * v->words;
  const int w = v->w;
  // Shared memory per CTA for the stage ring at the target occupancy. Generated networks leave
  // about 26 KB of the 228 KB to the L1 data cache, which holds the jobs' descriptors and
  // coefficients: on GB300 the config-2 encode runs best at 7 stages (197 KB) rather than 8
  // (225 KB), and the syndrome decode at 4-5 (143-179 KB) rather than 6 (215 KB).
  const int budget = (v->dispatch == PYRIT_DISPATCH_NETWORK ? 200 * 1024 : 226 * 1024) / v->minb - 1024;
  s.stages = h.stages > 0 ? h.stages : std::max(2, std::min(8, budget / (w * s.tw)));
  s.grid = 0;
  if (h.ctas_per_sm > 0) s.grid = h.ctas_per_sm * sm_count();
  *out = s;
  return true;
}

bool choose_shape(int n, int max_nout, const ShapeHint& h, TileShape* out, bool shared_masks) {
  // Default: the first registered variant of the ring size, the one measured fastest on its
  // workload; hints narrow the choice. When every job of the launch has the same masks, all warps
  // walk the same branches and the larger pairing network (dispatch 2) pays off, so a variant of
  // the default's shape with that dispatch is preferred.
  const Variant* v = find_variant(n, h.words, h.dispatch, h.mg, h.minb, h.nc);
  if (!v) v = find_variant(n, 0, -1, 0, 0, 0);
  if (!v) return false;
  if (shared_masks && h.dispatch < 0 && v->dispatch != 2) {
    const Variant* p = find_variant(n, v->words, 2, v->mg, v->minb, v->nc);
    if (p) v = p;
  }
  return shape_for_variant(v, max_nout, h, out);
}

void resolve_grid(TileShape* s) {
  if (!s->v) return;
  ensure_attr(s->v);
  if (s->grid <= 0) s->grid = sm_count() * occupancy(*s);
}

int launch_staged(const TileShape& sh, const JobDesc* job0, const JobDesc* jobs_dev, const uint2* tiles_dev,
                  uint32_t ntiles, uint32_t tiles_per_job, cudaStream_t stream, uint32_t* done_cnt,
                  uint64_t* done_ns) {
  if (ntiles == 0) return PYRIT_OK;
  if (!sh.v) return PYRIT_E_INVALID_ARG;
  CodeArgs a;
  a.jobs = jobs_dev;
  a.tiles = tiles_dev;
  a.ntiles = ntiles;
  a.tiles_per_job = tiles_per_job;
  a.tw = (uint32_t)sh.tw;
  a.groups = (uint32_t)sh.groups;
  a.stages = (uint32_t)sh.stages;
  a.err = device_error_word();
  a.done_cnt = done_ns ? done_cnt : nullptr;
  a.done_ns = done_cnt ? done_ns : nullptr;
  if (job0)
    a.job0 = *job0;
  else
    std::memset(&a.job0, 0, sizeof(a.job0));
  ensure_attr(sh.v);
  int grid = sh.grid > 0 ? sh.grid : sm_count() * occupancy(sh);
  grid = (int)std::min<uint32_t>((uint32_t)grid, ntiles);
  void* args[] = {&a};
  const cudaError_t e = cudaLaunchKernel(sh.v->fn, dim3(grid), dim3((sh.v->nc + 1) * 32), args, smem_bytes(sh),
                                         stream);
  return e == cudaSuccess ? PYRIT_OK : PYRIT_E_CUDA;
}

int launch_plain(int n, const JobDesc& job, cudaStream_t stream) {
  if (job.P == 0 || job.nout == 0) return PYRIT_OK;
  const uint64_t blocks64 = (job.P + 255) / 256;
  const int grid = (int)std::min<uint64_t>(blocks64, (uint64_t)sm_count() * 8);
  switch (n) {
    case 3: ring_plain_kernel<3><<<grid, 256, 0, stream>>>(job); break;
    case 5: ring_plain_kernel<5><<<grid, 256, 0, stream>>>(job); break;
    case 9: ring_plain_kernel<9><<<grid, 256, 0, stream>>>(job); break;
    case 11: ring_plain_kernel<11><<<grid, 256, 0, stream>>>(job); break;
    case 13: ring_plain_kernel<13><<<grid, 256, 0, stream>>>(job); break;
    default: return PYRIT_E_UNSUPPORTED_FIELD;
  }
  return cudaGetLastError() == cudaSuccess ? PYRIT_OK : PYRIT_E_CUDA;
}

}  // namespace pyrit

extern "C" int pyrit_variants(int* params_out, int cap) {
  int n = 0;
  const pyrit::Variant* v = pyrit::variants(&n);
  for (int i = 0; i < n && i < cap && params_out; ++i) {
    int* r = params_out + 6 * i;
    r[0] = v[i].n;
    r[1] = v[i].words;
    r[2] = v[i].mg;
    r[3] = v[i].minb;
    r[4] = v[i].dispatch;
    r[5] = v[i].nc;
  }
  return n;
}
