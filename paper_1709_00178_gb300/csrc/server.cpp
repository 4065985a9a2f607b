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
// soon as a slot and budget free up. Each request completes on its own, inside a shared launch:
// the kernel counts the consumer warps that have stored each job's tiles and the warp completing
// the count writes the job's completion stamp into host-mapped memory. The scheduler, which spins
// while work is in flight, retires a request (and its admission bytes) as soon as it sees the
// stamp, and frees the slot when its launches have ended. A request's latency is its arrival to
// that moment, on the server clock.
//
// Threads. Submitters validate requests (and size their tiles, under the shape-cache lock) and
// append them to an inbox under the queue lock, which the scheduler holds only to take the inbox
// and to publish completions; the slots, the admission queue and the launches belong to the
// scheduler thread alone, and the counters callers read are atomics. So a scheduler that polls
// continuously never holds up a submission.
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

// Pending::idx when a request has no completion stamp: nothing to code, or coded by a kernel that
// does not stamp completions (the generic kernels; they complete when the slot's launches end).
constexpr int kNoWork = -1;
constexpr int kUntracked = -2;
// How long an idle scheduler polls for submissions before it sleeps on the condition variable.
constexpr int64_t kIdleSpinNs = 500000;

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
  int idx = -1;      // completion stamp of the request in its slot's table, or kNoWork / kUntracked
  bool finished = false;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaStream_t aux = nullptr;        // second stream: a batch's launch groups alternate between the two
  cudaEvent_t staged = nullptr;      // on st after the job and tile copies (aux waits for it)
  cudaEvent_t aux_done = nullptr;    // on aux after its launches (st waits for it)
  cudaEvent_t done = nullptr;  // recorded after the slot's launches
  JobDesc* dev_jobs = nullptr;
  uint2* dev_tiles = nullptr;
  JobDesc* host_jobs = nullptr;  // pinned staging
  uint2* host_tiles = nullptr;
  uint32_t* dev_cnt = nullptr;    // per-request count of finished warp-tiles (zero between launches)
  uint64_t* host_done = nullptr;  // per-request completion stamps, host-mapped (0: not done)
  uint64_t* dev_done = nullptr;   // the same memory as the kernels address it
  std::vector<Pending> reqs;
  size_t open = 0;     // requests of the slot not yet retired
  uint64_t bytes = 0;
  uint64_t tiles = 0;  // sum of the admitted requests' tile bounds
  int64_t launch_ns = 0;
  int64_t queried_ns = 0;  // last query of `done` while requests were still open
  bool busy = false;
};

}  // namespace

struct pyrit_server_s {
  // Shape caches (cache_mu): submitters size requests' tiles with them, the scheduler shapes launches.
  std::mutex cache_mu;
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
  size_t queue_cap = 0;
  int64_t origin_host = 0;  // host steady-clock time of the server clock's zero

  // The scheduler thread's own state.
  std::vector<Slot> slots;
  std::deque<Pending> arrivals;  // taken from the inbox, waiting for admission

  // Queue lock: the inbox, the completions and the stop flag.
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> inbox;
  std::vector<pyrit_completion_t> done;
  bool stop = false;

  std::atomic<int> fatal{PYRIT_OK};
  std::atomic<uint64_t> queued{0};  // inbox + arrivals
  std::atomic<uint64_t> inflight{0}, max_inflight{0};
  std::atomic<uint64_t> batches{0}, completed{0}, submitted{0}, launches{0};
  std::thread worker;

  int64_t now() const { return host_now_ns() - origin_host; }
};

namespace {

// Retires request p of a slot at server time t with `status` into `fin`.
void retire(pyrit_server_s* s, Slot& sl, Pending& p, int status, int64_t t, std::vector<pyrit_completion_t>& fin) {
  pyrit_completion_t c;
  c.tag = p.tag;
  c.status = status;
  c.arrival_ns = p.arrival;
  c.start_ns = sl.launch_ns;
  c.done_ns = t;
  fin.push_back(c);
  p.finished = true;
  --sl.open;
  s->inflight -= p.bytes;
}

// Retires every request whose completion stamp has arrived, and frees every slot whose launches
// have ended (a request still unstamped then did not complete: a bounded device wait gave up, or
// the launch failed; requests coded by a kernel that stamps nothing complete then). A slot's
// completion event is queried once all its stamped requests are in, or while it holds requests that
// complete only with it, and otherwise at most every 200 us, to notice a launch that ended without
// completing its requests.
void reap(pyrit_server_s* s, std::vector<pyrit_completion_t>& fin) {
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    const int64_t t = s->now();
    if (sl.open)
      for (Pending& p : sl.reqs)
        if (!p.finished && p.idx >= 0 && reinterpret_cast<volatile uint64_t*>(sl.host_done)[p.idx] != 0)
          retire(s, sl, p, PYRIT_OK, t, fin);
    bool untracked = false;  // such requests complete only with the slot's event: query it now
    for (const Pending& p : sl.reqs) untracked = untracked || (!p.finished && p.idx == kUntracked);
    if (sl.open && !untracked && t - sl.queried_ns < 200000) continue;
    sl.queried_ns = t;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (sl.open) {
      // the launches ended: stamps written before the end are visible now
      bool incomplete = false;
      for (Pending& p : sl.reqs) {
        if (p.finished) continue;
        const bool stamped = p.idx >= 0 && reinterpret_cast<volatile uint64_t*>(sl.host_done)[p.idx] != 0;
        const bool ok = stamped || p.idx == kUntracked;  // an untracked request is done when its launch is
        incomplete = incomplete || !ok || q != cudaSuccess;
        retire(s, sl, p, q != cudaSuccess ? PYRIT_E_CUDA : ok ? PYRIT_OK : PYRIT_E_TIMEOUT, t, fin);
      }
      // an incomplete count would offset the next launch's: clear the table
      if (incomplete) cudaMemsetAsync(sl.dev_cnt, 0, sizeof(uint32_t) * (size_t)s->max_batch, sl.st);
    }
    sl.reqs.clear();
    sl.bytes = 0;
    sl.tiles = 0;
    sl.busy = false;
  }
}

// Launch shape for a batch whose ring-size-n jobs have at most max_nout outputs: the tuned shape of
// that key for mixed packet sizes if the autotuner has one, else the default. Cached; called
// with cache_mu held.
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
// later requests of the same plan and form skip building its spec. Called with cache_mu held.
const Variant* request_network(pyrit_server_s* s, const Pending& p) {
  if (p.job.nout == 0 || jit_mode() == PYRIT_JIT_OFF) return nullptr;
  if (p.op != PYRIT_OP_ENCODE && !p.syn) return nullptr;
  const uint64_t key = request_key(p);
  auto it = s->nets.find(key);
  if (it != s->nets.end()) return it->second;
  // the served form of the network: it stamps each request's completion
  NetSpec spec = p.op == PYRIT_OP_ENCODE ? net_spec(p.n, p.job, 0, 0, 0, 0, PYRIT_TRANSFORM_EMBEDDING)
                                         : net_spec_syndrome(p.plan, 0, 0, 0);
  spec.track = 1;
  const Variant* v = net_variant(spec, false);
  if (v) s->nets.emplace(key, v);
  return v;
}

// Launch shape of a generated network (cached; called with cache_mu held).
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
// a slot's tile table. Widths are cached. Called with cache_mu held.
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
int launch_slot(pyrit_server_s* s, Slot& sl, std::vector<pyrit_completion_t>& fin) {
  std::unique_lock<std::mutex> cache_lk(s->cache_mu);
  uint32_t nj = 0, nt = 0, nd = 0;  // jobs and tiles staged, completion stamps assigned
  struct G {
    TileShape shape;
    uint32_t job0, njobs, tile0, ntiles, done0;
    bool track;      // the group's kernel stamps each job's completion
    bool single;     // one job, passed by value
    JobDesc job;     // that job
  };
  std::vector<G> groups;
  std::vector<const Variant*> net(sl.reqs.size());
  for (size_t i = 0; i < sl.reqs.size(); ++i) net[i] = request_network(s, sl.reqs[i]);
  // A group's jobs take consecutive completion stamps in job order, so that job j of its launch
  // (its position in the launch's job array) owns stamp done0 + j.
  auto add_group = [&](const TileShape& shape, auto member, bool syn_form) -> int {
    G g{};
    g.shape = shape;
    g.job0 = nj;
    g.tile0 = nt;
    g.done0 = nd;
    const bool track = shape.v && shape.v->track;  // else its requests complete when the slot's launches end
    size_t members = 0, first = 0;
    for (size_t i = 0; i < sl.reqs.size(); ++i)
      if (sl.reqs[i].job.nout != 0 && member(i) && members++ == 0) first = i;
    if (members == 1) {
      Pending& p = sl.reqs[first];
      g.single = true;
      g.job = syn_form ? p.syn_job : p.job;
      g.njobs = 1;
      g.ntiles = (uint32_t)((p.job.P + (uint64_t)g.shape.tw - 1) / (uint64_t)g.shape.tw);
      g.track = track;
      p.idx = track ? (int)nd++ : kUntracked;
      groups.push_back(g);
      return PYRIT_OK;
    }
    // members in increasing size: the persistent CTAs walk the tile list in order, so the small
    // requests of a shared launch complete first
    std::vector<size_t> order;
    for (size_t i = 0; i < sl.reqs.size(); ++i)
      if (sl.reqs[i].job.nout != 0 && member(i)) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return sl.reqs[a].bytes < sl.reqs[b].bytes; });
    for (size_t i : order) {
      Pending& p = sl.reqs[i];
      sl.host_jobs[nj] = syn_form ? p.syn_job : p.job;
      for (uint64_t c = 0; c < p.job.P; c += (uint64_t)g.shape.tw) {
        if (nt >= s->max_tiles) return PYRIT_E_INVALID_ARG;  // admission keeps batches within the table
        sl.host_tiles[nt++] = make_uint2(nj - g.job0, (uint32_t)c);
      }
      ++nj;
      p.idx = track ? (int)nd++ : kUntracked;
    }
    g.track = track;
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
  cache_lk.unlock();
  // The slot's previous launches have ended (it was freed at their completion event): no kernel
  // writes these stamps now.
  for (uint32_t d = 0; d < nd; ++d) sl.host_done[d] = 0;
  if (nj && cudaMemcpyAsync(sl.dev_jobs, sl.host_jobs, nj * sizeof(JobDesc), cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
    return PYRIT_E_CUDA;
  if (nt && cudaMemcpyAsync(sl.dev_tiles, sl.host_tiles, nt * sizeof(uint2), cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
    return PYRIT_E_CUDA;
  // Launch groups alternate between the slot's two streams so that, e.g., a batch's decodes do not
  // wait for its encodes to finish: the second stream waits for the copies, and the first for the
  // second's launches before the slot's completion event.
  const bool two = groups.size() > 1;
  if (two && (cudaEventRecord(sl.staged, sl.st) != cudaSuccess || cudaStreamWaitEvent(sl.aux, sl.staged, 0) != cudaSuccess))
    return PYRIT_E_CUDA;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const G& g = groups[gi];
    const cudaStream_t st = two && (gi & 1) ? sl.aux : sl.st;
    uint32_t* cnt = g.track ? sl.dev_cnt + g.done0 : nullptr;
    uint64_t* stamp = g.track ? sl.dev_done + g.done0 : nullptr;
    const int rc = g.single ? launch_staged(g.shape, &g.job, nullptr, nullptr, g.ntiles, g.ntiles, st, cnt, stamp)
                            : launch_staged(g.shape, nullptr, sl.dev_jobs + g.job0, sl.dev_tiles + g.tile0, g.ntiles,
                                            0, st, cnt, stamp);
    if (rc != PYRIT_OK) return rc;
    s->launches += 1;
  }
  if (two && (cudaEventRecord(sl.aux_done, sl.aux) != cudaSuccess || cudaStreamWaitEvent(sl.st, sl.aux_done, 0) != cudaSuccess))
    return PYRIT_E_CUDA;
  if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) return PYRIT_E_CUDA;
  // requests with nothing to code (a decode with no block lost) are done at once
  for (Pending& p : sl.reqs)
    if (p.idx == kNoWork) retire(s, sl, p, PYRIT_OK, s->now(), fin);
  return PYRIT_OK;
}

// Publishes retired requests to pyrit_server_poll before counting them complete (so a drain that
// sees every request complete finds every completion).
void publish(pyrit_server_s* s, std::vector<pyrit_completion_t>& fin) {
  if (fin.empty()) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.insert(s->done.end(), fin.begin(), fin.end());
  }
  s->completed += fin.size();
  fin.clear();
}

void run(pyrit_server_s* s) {
  cudaSetDevice(s->device);
  std::vector<pyrit_completion_t> fin;
  uint64_t taken = 0;  // requests moved out of the inbox
  while (true) {
    bool busy = false;
    for (const Slot& sl : s->slots) busy = busy || sl.busy;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (!busy && s->arrivals.empty() && s->inbox.empty()) {
        // idle: poll for a while without the lock (a request that arrives soon is taken without a
        // thread wake-up), then sleep until a submission or shutdown
        lk.unlock();
        const int64_t until = host_now_ns() + kIdleSpinNs;
        while (s->submitted.load(std::memory_order_acquire) == taken && host_now_ns() < until)
          std::this_thread::yield();
        lk.lock();
        s->cv.wait(lk, [&] { return s->stop || !s->inbox.empty(); });
        if (s->inbox.empty()) break;  // stopped with nothing left to do
      }
      while (!s->inbox.empty()) {
        s->arrivals.push_back(s->inbox.front());
        s->inbox.pop_front();
        ++taken;
      }
    }
    reap(s, fin);
    bool launched = false;
    while (!s->arrivals.empty() && s->fatal == PYRIT_OK) {
      Slot* free_slot = nullptr;
      int nfree = 0;
      for (Slot& sl : s->slots)
        if (!sl.busy) {
          if (!free_slot) free_slot = &sl;
          ++nfree;
        }
      if (!free_slot) break;
      // Batch only under contention: while other slots are free each request gets a slot of its
      // own (a launch of one request carries its job in the kernel parameters, with nothing to copy
      // first); the last free slot takes everything admitted, up to the batch size.
      const int cap = nfree > 1 ? 1 : s->max_batch;
      // Admit in arrival order while the budget, the batch size and the slot's tile table allow.
      while (!s->arrivals.empty() && (int)free_slot->reqs.size() < cap) {
        const Pending& p = s->arrivals.front();
        if (s->inflight + free_slot->bytes + p.bytes > s->budget) break;
        if (free_slot->tiles + p.tiles > s->max_tiles) break;
        free_slot->reqs.push_back(p);
        free_slot->bytes += p.bytes;
        free_slot->tiles += p.tiles;
        s->arrivals.pop_front();
        s->queued -= 1;
      }
      if (!free_slot->reqs.empty()) {
        s->inflight += free_slot->bytes;
        const uint64_t cur = s->inflight;
        if (cur > s->max_inflight) s->max_inflight = cur;
        free_slot->busy = true;
        free_slot->open = free_slot->reqs.size();
        free_slot->launch_ns = s->now();
        free_slot->queried_ns = free_slot->launch_ns;
        s->batches += 1;
        const int rc = launch_slot(s, *free_slot, fin);
        if (rc != PYRIT_OK) s->fatal = rc;
        launched = true;
      } else {
        break;  // the budget or the tile table holds the next request back
      }
    }
    publish(s, fin);
    if (!launched) {
      // Work in flight, or admission waiting for a slot or budget: poll again at once (a timed
      // wait would sleep for the kernel's timer slack, tens of microseconds). This thread holds no
      // lock here.
      std::this_thread::yield();
    }
  }
  publish(s, fin);
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
        cudaStreamCreateWithFlags(&sl.aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.staged, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.aux_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.dev_jobs, sizeof(JobDesc) * max_batch) != cudaSuccess ||
        cudaMalloc(&sl.dev_tiles, sizeof(uint2) * s->max_tiles) != cudaSuccess ||
        cudaMalloc(&sl.dev_cnt, sizeof(uint32_t) * max_batch) != cudaSuccess ||
        cudaMemset(sl.dev_cnt, 0, sizeof(uint32_t) * max_batch) != cudaSuccess ||
        cudaMallocHost(&sl.host_jobs, sizeof(JobDesc) * max_batch) != cudaSuccess ||
        cudaMallocHost(&sl.host_tiles, sizeof(uint2) * s->max_tiles) != cudaSuccess ||
        cudaHostAlloc(&sl.host_done, sizeof(uint64_t) * max_batch, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&sl.dev_done, sl.host_done, 0) != cudaSuccess)
      rc = PYRIT_E_OOM;
  }
  if (rc == PYRIT_OK && cudaDeviceSynchronize() != cudaSuccess) rc = PYRIT_E_CUDA;
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
      std::lock_guard<std::mutex> lk(s->cache_mu);
      p.tiles = request_tiles(s, p);
      if (p.tiles > s->max_tiles) return PYRIT_E_INVALID_ARG;
    }
    p.tag = reqs[i].tag;
    batch.push_back(p);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != PYRIT_OK) return s->fatal;
  if (s->queued + batch.size() > s->queue_cap) return PYRIT_E_BUSY;
  const int64_t now = s->now();
  for (size_t i = 0; i < batch.size(); ++i) {
    batch[i].arrival = reqs[i].arrival_ns > 0 ? reqs[i].arrival_ns : now;
    s->inbox.push_back(batch[i]);
  }
  s->queued += batch.size();
  s->submitted += batch.size();
  s->cv.notify_one();
  return PYRIT_OK;
}

int pyrit_server_replay(pyrit_server_t s, const pyrit_request_t* reqs, int count) {
  if (!s || count < 0 || (count > 0 && !reqs)) return PYRIT_E_INVALID_ARG;
  for (int i = 1; i < count; ++i)
    if (reqs[i].arrival_ns < reqs[i - 1].arrival_ns) return PYRIT_E_INVALID_ARG;
  // Each pass submits every request whose arrival time has come, in one call; the thread spins
  // between arrivals (it is the load generator: it must not sleep past an arrival).
  int i = 0;
  while (i < count) {
    const int64_t now = s->now();
    int j = i;
    while (j < count && reqs[j].arrival_ns <= now) ++j;
    if (j > i) {
      const int rc = pyrit_server_submit(s, reqs + i, j - i);
      if (rc != PYRIT_OK) return rc;
      i = j;
    }
  }
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
    if (s->fatal != PYRIT_OK) return s->fatal;
    if (s->completed >= s->submitted) return PYRIT_OK;
    if (host_now_ns() > limit) return PYRIT_E_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int pyrit_server_stats(pyrit_server_t s, uint64_t* stats_out) {
  if (!s || !stats_out) return PYRIT_E_INVALID_ARG;
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
    if (sl.dev_cnt) cudaFree(sl.dev_cnt);
    if (sl.host_done) cudaFreeHost(sl.host_done);
    if (sl.aux) cudaStreamSynchronize(sl.aux);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.staged) cudaEventDestroy(sl.staged);
    if (sl.aux_done) cudaEventDestroy(sl.aux_done);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.aux) cudaStreamDestroy(sl.aux);
  }
  delete s;
}

}  // extern "C"
