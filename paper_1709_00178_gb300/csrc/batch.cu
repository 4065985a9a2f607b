// Batched coding: many stripes (possibly of different codes, operations and packet sizes) coded by
// one persistent launch of the staged ring kernel per ring size, optionally replayed from a CUDA
// graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "pyrit_internal.h"

using namespace pyrit;

namespace {

struct Group {
  TileShape shape;
  size_t jobs_off = 0, tiles_off = 0;  // offsets into the batch's device allocation
  uint32_t njobs = 0, ntiles = 0, tiles_per_job = 0;
  bool explicit_tiles = false;
};

}  // namespace

struct pyrit_batch_s {
  std::vector<Group> groups;
  std::vector<std::pair<int, JobDesc>> plain;  // (ring size, job) coded by the plain-load kernel
  uint8_t* dev = nullptr;
  uint64_t alg_bytes = 0, src_bytes = 0, tiles = 0;
  int launches = 0;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

namespace {

int build_job(const pyrit_stripe_t& s, JobDesc* job, uint64_t* alg, uint64_t* src) {
  pyrit_plan_s* p = s.plan;
  if (!p || !s.blocks || s.packet_bytes == 0 || s.packet_bytes > (1ull << 40)) return PYRIT_E_INVALID_ARG;
  if (s.op != PYRIT_OP_ENCODE && s.op != PYRIT_OP_DECODE) return PYRIT_E_INVALID_ARG;
  for (int b = 0; b < p->k + p->m; ++b)
    if (!s.blocks[b]) return PYRIT_E_INVALID_ARG;
  const uint64_t blk = (uint64_t)p->w * s.packet_bytes;
  *src = (uint64_t)p->k * blk;
  if (s.op == PYRIT_OP_ENCODE) {
    make_encode_job(p, s.blocks, s.blocks + p->k, s.packet_bytes, job);
    *alg = (uint64_t)(p->k + p->m) * blk;
    return PYRIT_OK;
  }
  DecodeEntry e;
  const int rc = plan_decode_entry(p, s.erasures, &e);
  if (rc != PYRIT_OK) return rc;
  make_decode_job(p, e, s.blocks, s.packet_bytes, job);
  *alg = (uint64_t)(p->k + e.ne) * blk;
  return PYRIT_OK;
}

int enqueue(pyrit_batch_s* b, cudaStream_t st) {
  for (const Group& g : b->groups) {
    const JobDesc* jobs = reinterpret_cast<const JobDesc*>(b->dev + g.jobs_off);
    const uint2* tiles = g.explicit_tiles ? reinterpret_cast<const uint2*>(b->dev + g.tiles_off) : nullptr;
    const int rc = launch_staged(g.shape, nullptr, jobs, tiles, g.ntiles, g.tiles_per_job, st);
    if (rc != PYRIT_OK) return rc;
  }
  for (const auto& pj : b->plain) {
    const int rc = launch_plain(pj.first, pj.second, st);
    if (rc != PYRIT_OK) return rc;
  }
  return PYRIT_OK;
}

}  // namespace

extern "C" {

int pyrit_batch_create(const pyrit_stripe_t* stripes, int count, const pyrit_tile_t* tile, pyrit_batch_t* out) {
  if (!out || count < 0 || (count > 0 && !stripes)) return PYRIT_E_INVALID_ARG;
  *out = nullptr;
  ShapeHint hint;
  if (tile) {
    hint.words = tile->words;
    hint.mg = tile->mg;
    hint.minb = tile->minb;
    hint.nc = tile->nc;
    hint.dispatch = tile->dispatch;
    hint.stages = tile->stages;
    hint.ctas_per_sm = tile->ctas_per_sm;
  }
  pyrit_batch_s* b = new (std::nothrow) pyrit_batch_s;
  if (!b) return PYRIT_E_OOM;
  cudaGetDevice(&b->device);

  // Jobs per ring size, in stripe order.
  std::vector<std::vector<JobDesc>> by_n(16);
  for (int i = 0; i < count; ++i) {
    JobDesc job;
    uint64_t alg = 0, src = 0;
    const int rc = build_job(stripes[i], &job, &alg, &src);
    if (rc != PYRIT_OK) {
      delete b;
      return rc;
    }
    b->src_bytes += src;
    if (job.nout == 0) continue;
    b->alg_bytes += alg;
    const int n = stripes[i].plan->n;
    if (job_is_staged(job))
      by_n[n].push_back(job);
    else
      b->plain.emplace_back(n, job);
  }

  // Shapes, tile lists and the device image.
  std::vector<uint8_t> image;
  auto place = [&](const void* src, size_t bytes) {
    const size_t off = (image.size() + 255) / 256 * 256;
    image.resize(off + bytes);
    std::memcpy(image.data() + off, src, bytes);
    return off;
  };
  for (int n = 0; n < 16; ++n) {
    std::vector<JobDesc>& jobs = by_n[n];
    if (jobs.empty()) continue;
    Group g;
    int max_nout = 0;
    bool same_p = true;
    for (const JobDesc& j : jobs) {
      max_nout = std::max(max_nout, (int)j.nout);
      same_p = same_p && j.P == jobs[0].P;
    }
    if (!choose_shape(n, max_nout, hint, &g.shape)) {
      delete b;
      return PYRIT_E_UNSUPPORTED_FIELD;
    }
    g.njobs = (uint32_t)jobs.size();
    g.jobs_off = place(jobs.data(), jobs.size() * sizeof(JobDesc));
    if (same_p) {
      g.tiles_per_job = tiles_for(jobs[0].P, g.shape);
      g.ntiles = g.tiles_per_job * g.njobs;
    } else {
      std::vector<uint2> tl;
      for (uint32_t ji = 0; ji < g.njobs; ++ji)
        for (uint64_t c = 0; c < jobs[ji].P; c += (uint64_t)g.shape.tw) tl.push_back(make_uint2(ji, (uint32_t)c));
      g.explicit_tiles = true;
      g.ntiles = (uint32_t)tl.size();
      g.tiles_off = place(tl.data(), tl.size() * sizeof(uint2));
    }
    b->tiles += g.ntiles;
    b->groups.push_back(g);
  }
  b->launches = (int)(b->groups.size() + b->plain.size());

  if (!image.empty()) {
    if (cudaMalloc(&b->dev, image.size()) != cudaSuccess) {
      delete b;
      return PYRIT_E_OOM;
    }
    if (cudaMemcpy(b->dev, image.data(), image.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(b->dev);
      delete b;
      return PYRIT_E_CUDA;
    }
  }
  // Resolve grids and one-time device state now, so that a later graph capture makes no
  // allocation or attribute call.
  if (!device_error_word()) {
    cudaFree(b->dev);
    delete b;
    return PYRIT_E_CUDA;
  }
  for (Group& g : b->groups) resolve_grid(&g.shape);
  *out = b;
  return PYRIT_OK;
}

int pyrit_batch_run(pyrit_batch_t b, pyrit_stream_t stream, int graph) {
  if (!b) return PYRIT_E_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!graph) return enqueue(b, st);
  if (!b->exec) {
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PYRIT_E_CUDA;
    cudaGraph_t g = nullptr;
    int rc = PYRIT_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PYRIT_E_CUDA;
    if (rc == PYRIT_OK) rc = enqueue(b, cs);
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess && rc == PYRIT_OK) rc = PYRIT_E_CUDA;
    if (rc == PYRIT_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) rc = PYRIT_E_CUDA;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc != PYRIT_OK) {
      b->exec = nullptr;
      return rc;
    }
  }
  return cudaGraphLaunch(b->exec, st) == cudaSuccess ? PYRIT_OK : PYRIT_E_CUDA;
}

int pyrit_batch_stats(pyrit_batch_t b, uint64_t* alg_bytes, uint64_t* src_bytes, int* launches, uint64_t* tiles) {
  if (!b) return PYRIT_E_INVALID_ARG;
  if (alg_bytes) *alg_bytes = b->alg_bytes;
  if (src_bytes) *src_bytes = b->src_bytes;
  if (launches) *launches = b->launches;
  if (tiles) *tiles = b->tiles;
  return PYRIT_OK;
}

void pyrit_batch_destroy(pyrit_batch_t b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

}  // extern "C"
