// Batched coding: many stripes (possibly of different codes, operations and packet sizes) coded by
// one persistent launch of the staged ring kernel per ring size (and, for stripes the generic
// kernel codes, per class of output count), optionally replayed from a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "pyrit_internal.h"

using namespace pyrit;

namespace {

struct Group {
  TileShape shape;
  size_t jobs_off = 0;           // offset of the group's jobs in the batch's device allocation
  std::vector<uint64_t> job_P;   // packet size of every job (the tiling depends on the tile width)
  uint2* tiles_dev = nullptr;    // explicit tile list when the jobs' P differ (own allocation)
  uint32_t njobs = 0, ntiles = 0, tiles_per_job = 0;
  int max_nout = 0;
  TuneKey key;
  bool netable = false;         // the jobs share nin and use at most kMaxJobs tables: a network applies
  std::vector<JobDesc> tables;  // one job per distinct (nout, mask table), in the order jobs use them
  const pyrit_plan_s* syn_plan = nullptr;  // all jobs decode this plan: its syndrome network applies
  int syn_allrows = 1;  // that network with its all-rows body (most of the jobs need every parity row)
  size_t syn_off = 0;                      // the syndrome-form jobs in the device allocation
  int transform = PYRIT_TRANSFORM_EMBEDDING;  // the group's stripes all use this transform
  uint32_t net_g = 0;     // the field's modulus for generated networks (0: the ring's native field)
  bool net_only = false;  // only generated networks code the group (parity transform, other field)
};

// The group's device job array for a variant (syndrome networks take syndrome-form jobs).
const JobDesc* group_jobs(const uint8_t* dev, const Group& g, const Variant* v) {
  return reinterpret_cast<const JobDesc*>(dev + (v && syndrome_mode(v->mode) ? g.syn_off : g.jobs_off));
}

// Tiling of a group's jobs under a shape: with one P for all jobs, tile t covers job
// t / tiles_per_job; otherwise an explicit list {job, col0} is built and copied to the device.
int make_tiling(const Group& g, const TileShape& sh, uint2** tiles_dev, uint32_t* ntiles, uint32_t* tpj) {
  *tiles_dev = nullptr;
  bool same = true;
  for (uint64_t P : g.job_P) same = same && P == g.job_P[0];
  if (same) {
    *tpj = tiles_for(g.job_P[0], sh);
    *ntiles = *tpj * g.njobs;
    return PYRIT_OK;
  }
  std::vector<uint2> tl;
  for (uint32_t ji = 0; ji < g.njobs; ++ji)
    for (uint64_t c = 0; c < g.job_P[ji]; c += (uint64_t)sh.tw) tl.push_back(make_uint2(ji, (uint32_t)c));
  *tpj = 0;
  *ntiles = (uint32_t)tl.size();
  if (cudaMalloc(tiles_dev, tl.size() * sizeof(uint2)) != cudaSuccess) return PYRIT_E_OOM;
  if (cudaMemcpy(*tiles_dev, tl.data(), tl.size() * sizeof(uint2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(*tiles_dev);
    *tiles_dev = nullptr;
    return PYRIT_E_CUDA;
  }
  return PYRIT_OK;
}

// Compiles network candidates side by side (host threads), loads them and appends them to the
// tuner's candidates, leaving out shapes whose registers spilled (more than 64 bytes of spill
// stores) unless every one did.
void add_networks(const NetSpec* specs, int ns, std::vector<const Variant*>* cands) {
  std::vector<std::thread> th;
  for (int i = 0; i < ns; ++i) th.emplace_back([specs, i] { net_compile(specs[i]); });
  for (auto& t : th) t.join();
  std::vector<const Variant*> lean, all;
  for (int i = 0; i < ns; ++i) {
    const Variant* v = net_variant(specs[i], true);
    if (!v) continue;
    all.push_back(v);
    if (net_spill_bytes(specs[i]) <= 64) lean.push_back(v);
  }
  const std::vector<const Variant*>& use = lean.empty() ? all : lean;
  cands->insert(cands->end(), use.begin(), use.end());
}

int log2_floor(uint64_t v) {
  int r = -1;
  while (v) {
    v >>= 1;
    ++r;
  }
  return r;
}

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

int enqueue(pyrit_batch_s* b, cudaStream_t st) {
  for (const Group& g : b->groups) {
    const int rc = launch_staged(g.shape, nullptr, group_jobs(b->dev, g, g.shape.v), g.tiles_dev, g.ntiles,
                                 g.tiles_per_job, st);
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

  // Jobs per (ring size, transform, field), in stripe order (with the stripe each came from): one
  // launch group each.
  struct SlotKey {
    int n, transform;
    uint32_t g;
  };
  std::vector<SlotKey> keys;
  std::vector<std::vector<JobDesc>> by_n;
  std::vector<std::vector<int>> src_of;
  auto slot_of = [&](const pyrit_plan_s* p) {
    const SlotKey k{p->n, p->transform == PYRIT_TRANSFORM_PARITY ? PYRIT_TRANSFORM_PARITY : PYRIT_TRANSFORM_EMBEDDING,
                    plan_net_g(p)};
    for (size_t i = 0; i < keys.size(); ++i)
      if (keys[i].n == k.n && keys[i].transform == k.transform && keys[i].g == k.g) return i;
    keys.push_back(k);
    by_n.emplace_back();
    src_of.emplace_back();
    return keys.size() - 1;
  };
  for (int i = 0; i < count; ++i) {
    JobDesc jobs[kMaxJobs];
    int nj = 0;
    uint64_t alg = 0, src = 0;
    const int rc = stripe_jobs(stripes[i], jobs, &nj, &alg, &src);
    if (rc != PYRIT_OK) {
      delete b;
      return rc;
    }
    b->src_bytes += src;
    if (nj == 0) continue;
    b->alg_bytes += alg;
    const int n = stripes[i].plan->n;
    const bool net_only = network_only(stripes[i].plan);
    // a stripe's jobs (one per group of up to kMaxOut outputs) stay adjacent in the group, so
    // that their tiles, which read the same source columns, run close together and share L2
    for (int q = 0; q < nj; ++q) {
      if (job_is_staged(jobs[q])) {
        const size_t slot = slot_of(stripes[i].plan);
        by_n[slot].push_back(jobs[q]);
        src_of[slot].push_back(i);
      } else if (net_only) {  // the plain-load kernel has neither the parity transform nor other fields
        delete b;
        return PYRIT_E_UNSUPPORTED;
      } else {
        b->plain.emplace_back(n, jobs[q]);
      }
    }
  }

  // Groups that only the generic kernel will code -- run-time compilation off, or more distinct
  // mask tables than a network holds (or different source counts) and not the decodes of one plan
  // -- are split by their jobs' output counts (1-2, 3-4, 5-8): a launch is shaped for its largest
  // job, and a job with fewer outputs would leave the other output groups' warps idle on its
  // tiles. A stripe's jobs stay in one class (its wide stripes' jobs stay adjacent).
  if (!(tile && hint.dispatch == PYRIT_DISPATCH_NETWORK)) {
    const bool jit_on = jit_mode() != PYRIT_JIT_OFF;
    std::vector<SlotKey> keys2;
    std::vector<std::vector<JobDesc>> by_n2;
    std::vector<std::vector<int>> src_of2;
    for (size_t slot = 0; slot < keys.size(); ++slot) {
      const std::vector<JobDesc>& jobs = by_n[slot];
      const bool net_only = keys[slot].transform == PYRIT_TRANSFORM_PARITY || keys[slot].g != 0;
      bool generic = !net_only;
      if (generic && jit_on) {
        std::vector<const JobDesc*> tabs;
        bool same_in = true;
        for (const JobDesc& j : jobs) {
          same_in = same_in && j.nin == jobs[0].nin;
          bool seen = false;
          for (const JobDesc* t : tabs)
            seen = seen || (t->nout == j.nout && std::memcmp(t->mask, j.mask, sizeof(j.mask)) == 0);
          if (!seen && tabs.size() <= (size_t)kMaxJobs) tabs.push_back(&j);
        }
        const pyrit_plan_s* plan0 = stripes[src_of[slot][0]].plan;
        bool syn = plan0->k + plan0->m <= kMaxIn && plan0->m <= kMaxOut && plan0->native;
        for (int si : src_of[slot]) syn = syn && stripes[si].op == PYRIT_OP_DECODE && stripes[si].plan == plan0;
        generic = !(same_in && tabs.size() <= (size_t)kMaxJobs) && !syn;
      }
      if (!generic) {
        keys2.push_back(keys[slot]);
        by_n2.push_back(jobs);
        src_of2.push_back(src_of[slot]);
        continue;
      }
      // outputs of each stripe in the group: the class of its jobs
      std::vector<int> outs(count, 0);
      for (size_t q = 0; q < jobs.size(); ++q) outs[src_of[slot][q]] += jobs[q].nout;
      for (int cls = 0; cls < 3; ++cls) {
        SlotKey k = keys[slot];
        std::vector<JobDesc> part;
        std::vector<int> part_src;
        for (size_t q = 0; q < jobs.size(); ++q) {
          const int o = outs[src_of[slot][q]];
          if ((o <= 2 ? 0 : o <= 4 ? 1 : 2) != cls) continue;
          part.push_back(jobs[q]);
          part_src.push_back(src_of[slot][q]);
        }
        if (part.empty()) continue;
        keys2.push_back(k);
        by_n2.push_back(std::move(part));
        src_of2.push_back(std::move(part_src));
      }
    }
    keys.swap(keys2);
    by_n.swap(by_n2);
    src_of.swap(src_of2);
  }

  // Shapes, tile lists and the device image.
  std::vector<uint8_t> image;
  auto place = [&](const void* src, size_t bytes) {
    const size_t off = (image.size() + 255) / 256 * 256;
    image.resize(off + bytes);
    std::memcpy(image.data() + off, src, bytes);
    return off;
  };
  for (size_t slot = 0; slot < keys.size(); ++slot) {
    std::vector<JobDesc>& jobs = by_n[slot];
    if (jobs.empty()) continue;
    const int n = keys[slot].n;
    Group g;
    g.transform = keys[slot].transform;
    g.net_g = keys[slot].g;
    g.net_only = g.transform == PYRIT_TRANSFORM_PARITY || g.net_g != 0;
    const bool parity = g.net_only;  // generated networks only
    int max_nout = 0;
    bool same_p = true, shared = true;
    for (const JobDesc& j : jobs) {
      max_nout = std::max(max_nout, (int)j.nout);
      same_p = same_p && j.P == jobs[0].P;
      shared = shared && std::memcmp(j.mask, jobs[0].mask, sizeof(j.mask)) == 0;
    }
    // Distinct tables (nout and masks): a generated network holds up to kMaxJobs of them (the
    // output groups of wide stripes), and each job carries its table's index.
    bool same_in = true;
    for (JobDesc& j : jobs) {
      same_in = same_in && j.nin == jobs[0].nin;
      int t = 0;
      while (t < (int)g.tables.size() &&
             !(g.tables[t].nout == j.nout && std::memcmp(g.tables[t].mask, j.mask, sizeof(j.mask)) == 0))
        ++t;
      if (t == (int)g.tables.size() && (int)g.tables.size() <= kMaxJobs) g.tables.push_back(j);
      j.table = t < kMaxJobs ? t : 0;
    }
    g.max_nout = max_nout;
    g.key = TuneKey{n, shared ? 1 : 0, max_nout, same_p ? log2_floor(jobs[0].P) : -1};
    g.netable = same_in && (int)g.tables.size() <= kMaxJobs;
    std::vector<const JobDesc*> tptr;
    for (const JobDesc& t : g.tables) tptr.push_back(&t);
    auto table_spec = [&](int words, int mg, int minb, int nc) {
      return net_spec_tables(n, tptr.data(), (int)tptr.size(), words, mg, minb, nc, g.transform, g.net_g);
    };
    // Syndrome decoding: every job decodes a stripe of one plan whose columns fit a job.
    const pyrit_plan_s* plan0 = stripes[src_of[slot][0]].plan;
    // one decode job per stripe; the syndrome store reduces in the native fields only
    bool syn = plan0->k + plan0->m <= kMaxIn && plan0->m <= kMaxOut && plan0->native;
    for (int si : src_of[slot]) syn = syn && stripes[si].op == PYRIT_OP_DECODE && stripes[si].plan == plan0;
    std::vector<JobDesc> syn_jobs;
    if (syn) {
      for (int si : src_of[slot]) {
        DecodeEntry e;
        if (plan_decode_entry(stripes[si].plan, stripes[si].erasures, &e) != PYRIT_OK || !e.syn_ok) {
          syn = false;
          break;
        }
        JobDesc sj;
        make_syndrome_job(plan0, e, stripes[si].blocks, stripes[si].packet_bytes, &sj);
        syn_jobs.push_back(sj);
      }
    }
    if (syn) {
      g.syn_plan = plan0;
      // the all-rows body pays when most stripes lose as many blocks as the code has parity
      // (config-3-like batches: 0.60 -> 0.68 of HBM); a mix of fewer losses runs as well without it
      const uint32_t full = (1u << plan0->m) - 1u;
      size_t nfull = 0;
      for (const JobDesc& sj : syn_jobs) nfull += sj.mask[kSyndromeNeedRow][0] == full;
      g.syn_allrows = 2 * nfull >= syn_jobs.size() ? 1 : 0;
    }
    // Decodes of several patterns of one plan take its syndrome network, compiled once per plan; a
    // multi-table direct network would be compiled again for every new set of patterns.
    if (g.syn_plan && g.tables.size() > 1) g.netable = false;
    const bool jit_on = jit_mode() != PYRIT_JIT_OFF;
    const Variant* v = nullptr;
    ShapeHint sh_hint = hint;
    TuneVal tv;
    if (parity && (!jit_on || (!g.netable && !g.syn_plan) || (tile && hint.dispatch != PYRIT_DISPATCH_NETWORK))) {
      // only a generated network codes under the parity transform
      delete b;
      return PYRIT_E_UNSUPPORTED;
    }
    if (!tile && tune_lookup(g.key, &tv)) {
      sh_hint = ShapeHint();
      sh_hint.stages = tv.stages;
      if (tv.dispatch != PYRIT_DISPATCH_NETWORK) {
        if (!parity) v = find_variant(n, tv.words, tv.dispatch, tv.mg, tv.minb, tv.nc);
      } else if (g.netable && jit_on)
        v = net_variant(table_spec(tv.words, tv.mg, tv.minb, tv.nc), true);
      else if (g.syn_plan && jit_on)
        v = net_variant(net_spec_syndrome(g.syn_plan, tv.words, tv.minb, tv.nc, g.syn_allrows), true);
    }
    if (!v && tile && hint.dispatch == PYRIT_DISPATCH_NETWORK) {
      // an explicit request for a generated network must be honoured or fail: the group's own
      // table when its jobs share one, else the plan's syndrome network
      if (!g.netable && !g.syn_plan) {
        delete b;
        return PYRIT_E_INVALID_ARG;
      }
      if (jit_on)
        v = g.netable ? net_variant(table_spec(hint.words, hint.mg, hint.minb, hint.nc), true)
                      : net_variant(net_spec_syndrome(g.syn_plan, hint.words, hint.minb, hint.nc, g.syn_allrows), true);
      if (!v) {
        delete b;
        return PYRIT_E_JIT;
      }
    }
    if (!v && !tile && jit_on) {
      sh_hint = ShapeHint();
      // a failure leaves the generic kernel (under the parity transform: an error)
      if (g.netable)
        v = net_variant(table_spec(0, 0, 0, 0), true);
      else if (g.syn_plan)
        v = net_variant(net_spec_syndrome(g.syn_plan, 0, 0, 0, g.syn_allrows), true);
    }
    if (parity && !v) {
      delete b;
      return PYRIT_E_JIT;
    }
    if (v) {
      shape_for_variant(v, max_nout, sh_hint, &g.shape);
    } else if (!choose_shape(n, max_nout, hint, &g.shape, shared)) {
      delete b;
      return PYRIT_E_UNSUPPORTED_FIELD;
    }
    g.njobs = (uint32_t)jobs.size();
    g.jobs_off = place(jobs.data(), jobs.size() * sizeof(JobDesc));
    if (g.syn_plan) g.syn_off = place(syn_jobs.data(), syn_jobs.size() * sizeof(JobDesc));
    for (const JobDesc& j : jobs) g.job_P.push_back(j.P);
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
  // Tilings, grids and one-time device state now, so that a later graph capture makes no
  // allocation or attribute call.
  if (!device_error_word()) {
    pyrit_batch_destroy(b);
    return PYRIT_E_CUDA;
  }
  for (Group& g : b->groups) {
    resolve_grid(&g.shape);
    const int rc = make_tiling(g, g.shape, &g.tiles_dev, &g.ntiles, &g.tiles_per_job);
    if (rc != PYRIT_OK) {
      pyrit_batch_destroy(b);
      return rc;
    }
    b->tiles += g.ntiles;
  }
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

int pyrit_batch_tune(pyrit_batch_t b, pyrit_stream_t stream, int iters) {
  if (!b || iters < 1) return PYRIT_E_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PYRIT_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PYRIT_E_CUDA;
  }
  int rc = PYRIT_OK;
  int nv = 0;
  const Variant* all = variants(&nv);
  for (Group& g : b->groups) {
    std::vector<const Variant*> cands;
    const bool parity = g.net_only;  // generated networks only
    for (int i = 0; i < nv && !parity; ++i)
      if (all[i].n == g.key.n) cands.push_back(&all[i]);
    if (g.netable && jit_mode() != PYRIT_JIT_OFF) {
      // the network shapes, compiled side by side (host threads) before they are loaded and timed
      NetSpec specs[8];
      const int ns = net_candidate_shapes(g.key.n, g.max_nout, specs, 8);
      std::vector<const JobDesc*> tptr;
      for (const JobDesc& t : g.tables) tptr.push_back(&t);
      for (int i = 0; i < ns; ++i)
        specs[i] = net_spec_tables(g.key.n, tptr.data(), (int)tptr.size(), specs[i].words, specs[i].mg,
                                   specs[i].minb, specs[i].nc, g.transform, g.net_g);
      add_networks(specs, ns, &cands);
    } else if (g.syn_plan && jit_mode() != PYRIT_JIT_OFF) {
      NetSpec specs[8];
      const int ns = net_syndrome_shapes(g.syn_plan, specs, 8, g.syn_allrows);
      add_networks(specs, ns, &cands);
    }
    // Every candidate at its default pipeline depth; generated networks at every depth from 3
    // stages to as many as shared memory holds: the best depth depends on the code and the
    // network (measured on GB300: the syndrome decodes 4-5 stages, the config-2 encode 7, the
    // GF(2^12) k=16 m=4 encode 6).
    struct Try {
      const Variant* v;
      int stages;  // 0: the default
    };
    std::vector<Try> tries;
    for (const Variant* v : cands) {
      tries.push_back({v, 0});
      if (v->dispatch == PYRIT_DISPATCH_NETWORK) {
        TileShape def;
        if (!shape_for_variant(v, g.max_nout, ShapeHint(), &def)) continue;
        const int fit = (int)std::min<size_t>(8, (226 * 1024 / v->minb - 1024) / ((size_t)v->w * def.tw));
        for (int st = 3; st <= fit; ++st)
          if (st != def.stages) tries.push_back({v, st});
      }
    }
    float best = 1e30f;
    TileShape best_shape = g.shape;
    for (size_t i = 0; i < tries.size() && rc == PYRIT_OK; ++i) {
      TileShape sh;
      ShapeHint th;
      th.stages = tries[i].stages;
      if (!shape_for_variant(tries[i].v, g.max_nout, th, &sh)) continue;
      resolve_grid(&sh);
      uint2* tiles = nullptr;  // the tiling depends on the candidate's tile width
      uint32_t ntiles = 0, tpj = 0;
      rc = make_tiling(g, sh, &tiles, &ntiles, &tpj);
      if (rc != PYRIT_OK) break;
      const JobDesc* jobs = group_jobs(b->dev, g, tries[i].v);
      rc = launch_staged(sh, nullptr, jobs, tiles, ntiles, tpj, st);  // warm-up
      if (rc == PYRIT_OK) {
        cudaEventRecord(e0, st);
        for (int it = 0; it < iters && rc == PYRIT_OK; ++it) rc = launch_staged(sh, nullptr, jobs, tiles, ntiles, tpj, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = PYRIT_E_CUDA;
      }
      if (tiles) cudaFree(tiles);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)iters;
      if (rc == PYRIT_OK && ms < best) {
        best = ms;
        best_shape = sh;
      }
    }
    if (rc != PYRIT_OK) break;
    if (g.tiles_dev) cudaFree(g.tiles_dev);
    g.tiles_dev = nullptr;
    g.shape = best_shape;
    b->tiles -= g.ntiles;
    rc = make_tiling(g, g.shape, &g.tiles_dev, &g.ntiles, &g.tiles_per_job);
    if (rc != PYRIT_OK) break;
    b->tiles += g.ntiles;
    const Variant* v = best_shape.v;
    tune_record(g.key, TuneVal{v->words, v->mg, v->minb, v->nc, v->dispatch, best_shape.stages, best});
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (b->exec) {  // the captured launches used the old shapes
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return rc;
}

int pyrit_batch_stats(pyrit_batch_t b, uint64_t* alg_bytes, uint64_t* src_bytes, int* launches, uint64_t* tiles) {
  if (!b) return PYRIT_E_INVALID_ARG;
  if (alg_bytes) *alg_bytes = b->alg_bytes;
  if (src_bytes) *src_bytes = b->src_bytes;
  if (launches) *launches = b->launches;
  if (tiles) *tiles = b->tiles;
  return PYRIT_OK;
}

int pyrit_batch_shape(pyrit_batch_t b, int group, int* params_out) {
  if (!b || !params_out || group < 0 || group >= (int)b->groups.size()) return PYRIT_E_INVALID_ARG;
  const TileShape& s = b->groups[(size_t)group].shape;
  const Variant* v = s.v;
  const int r[11] = {v->n, v->words, v->mg, v->minb, v->dispatch, v->nc, s.groups, s.tw, s.stages, s.grid, v->mode};
  std::memcpy(params_out, r, sizeof(r));
  return PYRIT_OK;
}

void pyrit_batch_destroy(pyrit_batch_t b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (Group& g : b->groups)
    if (g.tiles_dev) cudaFree(g.tiles_dev);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

}  // extern "C"
