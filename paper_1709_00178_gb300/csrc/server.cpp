// Served coding with continuous batching.
//
// Callers submit stripe requests (encode or decode, any plan, any packet size) as they arrive. A
// scheduler thread admits them while the bytes of the requests in flight stay within an HBM budget
// and, whenever one of its stream slots is free, packs everything admitted into one batch: the jobs
// are copied into that slot's device descriptor table and coded by one persistent launch of the
// staged ring kernel per ring size on the slot's stream -- or, for requests whose plan has a
// compiled generated network (its encode table, or its syndrome-decode network), one launch of
// that network per plan and operation; a missing network is queued for the background compiler and
// the generic kernel serves meanwhile, so the scheduler never waits for a compilation. Batches on
// different slots overlap on the device, so requests that arrive while others are running start as
// soon as a slot and budget free up. Completion is timestamped on the device timeline (CUDA events
// measured against an origin event), so a request's latency is its arrival to the end of the GPU
// work that coded it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <map>
#include <thread>
#include <vector>

#include "pyrit_internal.h"

using namespace pyrit;

namespace {

int64_t host_now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Pending {
  JobDesc job;
  JobDesc syn_job;               // the syndrome form of a decode job (when syn)
  const pyrit_plan_s* plan;
  int op;
  bool syn = false;
  int n;
  uint64_t bytes;    // device bytes of the stripe ((k+m) w P): what the admission budget counts
  uint64_t tiles;    // column tiles of the stripe at the narrowest tile width that could code it
  uint64_t tag;
  int64_t arrival;   // server clock, ns
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  JobDesc* dev_jobs = nullptr;
  uint2* dev_tiles = nullptr;
  JobDesc* host_jobs = nullptr;  // pinned staging
  uint2* host_tiles = nullptr;
  std::vector<Pending> reqs;
  uint64_t bytes = 0;
  uint64_t tiles = 0;  // sum of the admitted requests' tile bounds
  int64_t launch_ns = 0;
  bool busy = false;
};

}  // namespace

struct pyrit_server_s {
  TileShape shapes[16][kMaxOut + 1];  // launch shape per (ring size, largest output count), lazily
  bool shape_set[16][kMaxOut + 1] = {};
  std::map<const Variant*, TileShape> net_shapes;  // launch shapes of the generated networks used
  // Per (plan serial, syndrome form, output count): the compiled network that codes such requests
  // (only ready networks are kept), and the tile width of the network shape that would serve them.
  std::map<uint64_t, const Variant*> nets;
  std::map<uint64_t, uint32_t> net_tw;
  uint32_t generic_tw[16] = {};  // narrowest generic tile width per ring size (0: not computed)
  size_t budget = 0;
  int max_batch = 0;
  uint32_t max_tiles = 0;
  int device = 0;
  int64_t origin_host = 0;  // host time of the origin event
  cudaEvent_t origin = nullptr;
  std::vector<Slot> slots;

  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> arrivals;
  std::vector<pyrit_completion_t> done;
  size_t queue_cap = 0;
  uint64_t inflight = 0, max_inflight = 0;
  uint64_t batches = 0, completed = 0, submitted = 0, launches = 0;
  std::atomic<bool> stop{false};
  int fatal = PYRIT_OK;
  std::thread worker;

  int64_t now() const { return host_now_ns() - origin_host; }
};

namespace {

// Device time of an event that has completed, on the server clock.
int64_t event_ns(pyrit_server_s* s, cudaEvent_t e) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, s->origin, e);
  return (int64_t)((double)ms * 1e6);
}

// Retires every slot whose work has finished. Called with the lock held.
void reap(pyrit_server_s* s) {
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    const int status = q == cudaSuccess ? PYRIT_OK : PYRIT_E_CUDA;
    const int64_t t_start = status == PYRIT_OK ? event_ns(s, sl.start) : sl.launch_ns;
    const int64_t t_done = status == PYRIT_OK ? event_ns(s, sl.done) : s->now();
    for (const Pending& p : sl.reqs) {
      pyrit_completion_t c;
      c.tag = p.tag;
      c.status = status;
      c.arrival_ns = p.arrival;
      c.start_ns = t_start;
      c.done_ns = t_done;
      s->done.push_back(c);
    }
    s->completed += sl.reqs.size();
    s->inflight -= sl.bytes;
    sl.reqs.clear();
    sl.bytes = 0;
    sl.tiles = 0;
    sl.busy = false;
  }
}

// Launch shape for a batch whose ring-size-n jobs have at most max_nout outputs: the tuned shape of
// that key for mixed packet sizes if the autotuner has one, else the default. Cached.
int slot_shape(pyrit_server_s* s, int n, int max_nout, TileShape* out) {
  if (n < 0 || n >= 16 || max_nout < 1 || max_nout > kMaxOut) return PYRIT_E_INVALID_ARG;
  if (!s->shape_set[n][max_nout]) {
    TileShape sh;
    TuneVal tv;
    const Variant* v = nullptr;
    if (tune_lookup(TuneKey{n, 0, max_nout, -1}, &tv)) v = find_variant(n, tv.words, tv.dispatch, tv.mg, tv.minb, tv.nc);
    if (v) {
      ShapeHint h;
      h.stages = tv.stages;
      shape_for_variant(v, max_nout, h, &sh);
    } else if (!choose_shape(n, max_nout, ShapeHint(), &sh)) {
      return PYRIT_E_UNSUPPORTED_FIELD;
    }
    resolve_grid(&sh);
    s->shapes[n][max_nout] = sh;
    s->shape_set[n][max_nout] = true;
  }
  *out = s->shapes[n][max_nout];
  return PYRIT_OK;
}

// Cache key of the requests of one plan, form (syndrome decode or not) and output count.
uint64_t request_key(const Pending& p) { return p.plan->serial << 5 | (p.syn ? 16u : 0u) | (uint64_t)p.job.nout; }

// The generated network that would code request p now (nullptr: the generic kernel), queued for
// the background compiler if it is missing. A ready network is remembered per request key, so
// later requests of the same plan and form skip building its spec. Called with the lock held.
const Variant* request_network(pyrit_server_s* s, const Pending& p) {
  if (p.job.nout == 0 || jit_mode() == PYRIT_JIT_OFF) return nullptr;
  if (p.op != PYRIT_OP_ENCODE && !p.syn) return nullptr;
  const uint64_t key = request_key(p);
  auto it = s->nets.find(key);
  if (it != s->nets.end()) return it->second;
  const Variant* v = p.op == PYRIT_OP_ENCODE
                         ? net_variant(net_spec(p.n, p.job, 0, 0, 0, 0, PYRIT_TRANSFORM_EMBEDDING), false)
                         : net_variant(net_spec_syndrome(p.plan, 0, 0, 0), false);
  if (v) s->nets.emplace(key, v);
  return v;
}

// Launch shape of a generated network (cached).
const TileShape& network_shape(pyrit_server_s* s, const Variant* v) {
  auto it = s->net_shapes.find(v);
  if (it == s->net_shapes.end()) {
    TileShape sh;
    shape_for_variant(v, v->nout, ShapeHint(), &sh);  // the output split it was compiled for
    resolve_grid(&sh);
    it = s->net_shapes.emplace(v, sh).first;
  }
  return it->second;
}

// Column tiles request p needs, an upper bound whichever kernel codes it: its packet size over the
// narrowest tile width among its ring size's generic shapes (for any output count of the batch it
// joins) and the default shape of the network that would code it, so that neither the batch's
// composition nor a network finishing its compilation between admission and launch can overflow
// a slot's tile table. Widths are cached. Called with the lock held.
uint64_t request_tiles(pyrit_server_s* s, const Pending& p) {
  if (p.job.nout == 0) return 0;
  if (p.n < 0 || p.n >= 16) return ~0ull;
  uint32_t& gtw = s->generic_tw[p.n];
  if (gtw == 0) {
    uint32_t tw = ~0u;
    for (int mo = 1; mo <= kMaxOut; ++mo) {
      TileShape sh;
      if (slot_shape(s, p.n, mo, &sh) != PYRIT_OK) return ~0ull;
      tw = std::min<uint32_t>(tw, (uint32_t)sh.tw);
    }
    gtw = tw;
  }
  uint64_t tw = gtw;
  const uint64_t key = request_key(p);
  auto it = s->net_tw.find(key);
  if (it == s->net_tw.end()) {
    uint32_t ntw = ~0u;
    NetSpec cand[1];  // the default network shape is the one served
    const int nc = p.syn ? net_syndrome_shapes(p.plan, cand, 1) : net_candidate_shapes(p.n, p.job.nout, cand, 1);
    if (nc == 1) {
      const int groups = output_groups(cand[0].mg, cand[0].nout, cand[0].nc);
      ntw = (uint32_t)(cand[0].nc / groups) * 32u * 4u * (uint32_t)cand[0].words;
    }
    it = s->net_tw.emplace(key, ntw).first;
  }
  tw = std::min<uint64_t>(tw, it->second);
  return tw ? (p.job.P + tw - 1) / tw : ~0ull;
}

// Packs the slot's admitted requests into launches: requests with a compiled network grouped by
// that network (encode table or plan's syndrome decode), the rest by ring size on the generic
// kernel. A group of one request carries its job in the kernel parameters with implicit tiles
// (nothing to copy first); larger groups get an explicit tile list, staged with their jobs in
// pinned memory and copied on the slot's stream.
int launch_slot(pyrit_server_s* s, Slot& sl) {
  uint32_t nj = 0, nt = 0;
  struct G {
    TileShape shape;
    uint32_t job0, njobs, tile0, ntiles;
    bool single;     // one job, passed by value
    JobDesc job;     // that job
  };
  std::vector<G> groups;
  std::vector<const Variant*> net(sl.reqs.size());
  for (size_t i = 0; i < sl.reqs.size(); ++i) net[i] = request_network(s, sl.reqs[i]);
  auto add_group = [&](const TileShape& shape, auto member, bool syn_form) -> int {
    G g{};
    g.shape = shape;
    g.job0 = nj;
    g.tile0 = nt;
    size_t members = 0, first = 0;
    for (size_t i = 0; i < sl.reqs.size(); ++i)
      if (sl.reqs[i].job.nout != 0 && member(i) && members++ == 0) first = i;
    if (members == 1) {
      const Pending& p = sl.reqs[first];
      g.single = true;
      g.job = syn_form ? p.syn_job : p.job;
      g.njobs = 1;
      g.ntiles = (uint32_t)((p.job.P + (uint64_t)g.shape.tw - 1) / (uint64_t)g.shape.tw);
      groups.push_back(g);
      return PYRIT_OK;
    }
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
      const Pending& p = sl.reqs[i];
      if (p.job.nout == 0 || !member(i)) continue;
      sl.host_jobs[nj] = syn_form ? p.syn_job : p.job;
      for (uint64_t c = 0; c < p.job.P; c += (uint64_t)g.shape.tw) {
        if (nt >= s->max_tiles) return PYRIT_E_INVALID_ARG;  // admission keeps batches within the table
        sl.host_tiles[nt++] = make_uint2(nj - g.job0, (uint32_t)c);
      }
      ++nj;
    }
    g.njobs = nj - g.job0;
    g.ntiles = nt - g.tile0;
    if (g.njobs) groups.push_back(g);
    return PYRIT_OK;
  };
  // generated networks, one launch each
  std::vector<const Variant*> used;
  for (const Variant* v : net)
    if (v && std::find(used.begin(), used.end(), v) == used.end()) used.push_back(v);
  for (const Variant* v : used) {
    const int rc = add_group(network_shape(s, v), [&](size_t i) { return net[i] == v; }, syndrome_mode(v->mode));
    if (rc != PYRIT_OK) return rc;
  }
  // the generic kernel per ring size for the rest
  for (int n = 0; n < 16; ++n) {
    int max_nout = 0;
    for (size_t i = 0; i < sl.reqs.size(); ++i)
      if (!net[i] && sl.reqs[i].n == n) max_nout = std::max(max_nout, (int)sl.reqs[i].job.nout);
    if (max_nout == 0) continue;
    TileShape sh;
    const int rc = slot_shape(s, n, max_nout, &sh);
    if (rc != PYRIT_OK) return rc;
    const int rc2 = add_group(sh, [&](size_t i) { return !net[i] && sl.reqs[i].n == n; }, false);
    if (rc2 != PYRIT_OK) return rc2;
  }
  cudaEventRecord(sl.start, sl.st);
  if (nj && cudaMemcpyAsync(sl.dev_jobs, sl.host_jobs, nj * sizeof(JobDesc), cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
    return PYRIT_E_CUDA;
  if (nt && cudaMemcpyAsync(sl.dev_tiles, sl.host_tiles, nt * sizeof(uint2), cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
    return PYRIT_E_CUDA;
  for (const G& g : groups) {
    const int rc = g.single ? launch_staged(g.shape, &g.job, nullptr, nullptr, g.ntiles, g.ntiles, sl.st)
                            : launch_staged(g.shape, nullptr, sl.dev_jobs + g.job0, sl.dev_tiles + g.tile0, g.ntiles,
                                            0, sl.st);
    if (rc != PYRIT_OK) return rc;
    ++s->launches;
  }
  if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) return PYRIT_E_CUDA;
  return PYRIT_OK;
}

void run(pyrit_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    reap(s);
    if (s->stop && s->arrivals.empty()) {
      bool busy = false;
      for (const Slot& sl : s->slots) busy = busy || sl.busy;
      if (!busy) break;
    }
    Slot* free_slot = nullptr;
    for (Slot& sl : s->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    bool launched = false;
    if (free_slot && !s->arrivals.empty() && s->fatal == PYRIT_OK) {
      // Admit in arrival order while the budget, the batch size and the slot's tile table allow.
      while (!s->arrivals.empty() && (int)free_slot->reqs.size() < s->max_batch) {
        const Pending& p = s->arrivals.front();
        if (s->inflight + free_slot->bytes + p.bytes > s->budget) break;
        if (free_slot->tiles + p.tiles > s->max_tiles) break;
        free_slot->reqs.push_back(p);
        free_slot->bytes += p.bytes;
        free_slot->tiles += p.tiles;
        s->arrivals.pop_front();
      }
      if (!free_slot->reqs.empty()) {
        s->inflight += free_slot->bytes;
        s->max_inflight = std::max(s->max_inflight, s->inflight);
        free_slot->busy = true;
        free_slot->launch_ns = s->now();
        ++s->batches;
        const int rc = launch_slot(s, *free_slot);
        if (rc != PYRIT_OK) s->fatal = rc;
        launched = true;
      }
    }
    if (!launched) {
      // Nothing to start: wait briefly for an arrival or for a slot to finish.
      s->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace

extern "C" {

int pyrit_server_create(size_t hbm_budget, int max_batch, int slots, int queue_cap, pyrit_server_t* out) {
  if (!out || hbm_budget == 0 || max_batch < 1 || max_batch > 4096 || slots < 1 || slots > 16 || queue_cap < 1)
    return PYRIT_E_INVALID_ARG;
  *out = nullptr;
  pyrit_server_s* s = new (std::nothrow) pyrit_server_s;
  if (!s) return PYRIT_E_OOM;
  s->budget = hbm_budget;
  s->max_batch = max_batch;
  s->queue_cap = (size_t)queue_cap;
  s->max_tiles = 1u << 17;
  cudaGetDevice(&s->device);
  s->slots.resize(slots);
  int rc = device_error_word() ? PYRIT_OK : PYRIT_E_CUDA;
  for (Slot& sl : s->slots) {
    if (rc != PYRIT_OK) break;
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.start) != cudaSuccess || cudaEventCreate(&sl.done) != cudaSuccess ||
        cudaMalloc(&sl.dev_jobs, sizeof(JobDesc) * max_batch) != cudaSuccess ||
        cudaMalloc(&sl.dev_tiles, sizeof(uint2) * s->max_tiles) != cudaSuccess ||
        cudaMallocHost(&sl.host_jobs, sizeof(JobDesc) * max_batch) != cudaSuccess ||
        cudaMallocHost(&sl.host_tiles, sizeof(uint2) * s->max_tiles) != cudaSuccess)
      rc = PYRIT_E_OOM;
  }
  if (rc == PYRIT_OK && (cudaEventCreate(&s->origin) != cudaSuccess ||
                         cudaEventRecord(s->origin, s->slots[0].st) != cudaSuccess ||
                         cudaEventSynchronize(s->origin) != cudaSuccess))
    rc = PYRIT_E_CUDA;
  if (rc != PYRIT_OK) {
    pyrit_server_destroy(s);
    return rc;
  }
  s->origin_host = host_now_ns();
  s->worker = std::thread(run, s);
  *out = s;
  return PYRIT_OK;
}

int64_t pyrit_server_now_ns(pyrit_server_t s) { return s ? s->now() : 0; }

int pyrit_server_submit(pyrit_server_t s, const pyrit_request_t* reqs, int count) {
  if (!s || count < 0 || (count > 0 && !reqs)) return PYRIT_E_INVALID_ARG;
  std::vector<Pending> batch;
  batch.reserve(count);
  for (int i = 0; i < count; ++i) {
    Pending p;
    uint64_t alg = 0, src = 0;
    JobDesc jobs[kMaxJobs];
    int nj = 0;
    const int rc = stripe_jobs(reqs[i].stripe, jobs, &nj, &alg, &src);
    if (rc != PYRIT_OK) return rc;
    // requests wait for no compilation, and only a generated network has the parity transform;
    // a request is one job (at most kMaxOut parity or erased blocks)
    if (network_only(reqs[i].stripe.plan) || nj > 1) return PYRIT_E_UNSUPPORTED;
    if (nj == 1)
      p.job = jobs[0];
    else
      std::memset(&p.job, 0, sizeof(p.job));
    p.n = reqs[i].stripe.plan->n;
    p.plan = reqs[i].stripe.plan;
    p.op = reqs[i].stripe.op;
    if (p.op == PYRIT_OP_DECODE && p.job.nout > 0) {
      DecodeEntry e;
      if (plan_decode_entry(reqs[i].stripe.plan, reqs[i].stripe.erasures, &e) == PYRIT_OK && e.syn_ok) {
        make_syndrome_job(p.plan, e, reqs[i].stripe.blocks, reqs[i].stripe.packet_bytes, &p.syn_job);
        p.syn = true;
      }
    }
    p.bytes = (uint64_t)(reqs[i].stripe.plan->k + reqs[i].stripe.plan->m) * reqs[i].stripe.plan->w *
              reqs[i].stripe.packet_bytes;
    if (p.bytes > s->budget) return PYRIT_E_BUDGET;
    if (!job_is_staged(p.job) && p.job.nout > 0) return PYRIT_E_INVALID_ARG;  // served stripes must be 16-byte aligned
    {
      // one request must fit a slot's tile table even at the narrowest tiles of its ring size
      std::lock_guard<std::mutex> lk(s->mu);
      p.tiles = request_tiles(s, p);
      if (p.tiles > s->max_tiles) return PYRIT_E_INVALID_ARG;
    }
    p.tag = reqs[i].tag;
    batch.push_back(p);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != PYRIT_OK) return s->fatal;
  if (s->arrivals.size() + batch.size() > s->queue_cap) return PYRIT_E_BUSY;
  const int64_t now = s->now();
  for (size_t i = 0; i < batch.size(); ++i) {
    batch[i].arrival = reqs[i].arrival_ns > 0 ? reqs[i].arrival_ns : now;
    s->arrivals.push_back(batch[i]);
  }
  s->submitted += batch.size();
  s->cv.notify_one();
  return PYRIT_OK;
}

int pyrit_server_poll(pyrit_server_t s, pyrit_completion_t* out, int cap) {
  if (!s || cap < 0 || (cap > 0 && !out)) return PYRIT_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const int n = (int)std::min<size_t>((size_t)cap, s->done.size());
  for (int i = 0; i < n; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + n);
  return n;
}

int pyrit_server_drain(pyrit_server_t s, int timeout_ms) {
  if (!s) return PYRIT_E_INVALID_ARG;
  const int64_t limit = host_now_ns() + (int64_t)timeout_ms * 1000000;
  while (true) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->fatal != PYRIT_OK) return s->fatal;
      bool busy = !s->arrivals.empty();
      for (const Slot& sl : s->slots) busy = busy || sl.busy;
      if (!busy) return PYRIT_OK;
    }
    if (host_now_ns() > limit) return PYRIT_E_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int pyrit_server_stats(pyrit_server_t s, uint64_t* stats_out) {
  if (!s || !stats_out) return PYRIT_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  stats_out[0] = s->submitted;
  stats_out[1] = s->completed;
  stats_out[2] = s->batches;
  stats_out[3] = s->launches;
  stats_out[4] = s->inflight;
  stats_out[5] = s->max_inflight;
  stats_out[6] = s->budget;
  return PYRIT_OK;
}

void pyrit_server_destroy(pyrit_server_t s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
      s->cv.notify_one();
    }
    s->worker.join();
  }
  for (Slot& sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.dev_jobs) cudaFree(sl.dev_jobs);
    if (sl.dev_tiles) cudaFree(sl.dev_tiles);
    if (sl.host_jobs) cudaFreeHost(sl.host_jobs);
    if (sl.host_tiles) cudaFreeHost(sl.host_tiles);
    if (sl.start) cudaEventDestroy(sl.start);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  if (s->origin) cudaEventDestroy(s->origin);
  delete s;
}

}  // extern "C"
