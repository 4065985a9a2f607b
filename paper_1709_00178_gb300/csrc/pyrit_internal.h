// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <cuda_runtime_api.h>

#include "../../include/pyrit.h"
#include "ring_abi.h"

namespace pyrit {

static_assert(kMaxIn == PYRIT_MAX_K && kMaxOut == PYRIT_JOB_OUTPUTS, "job limits follow the C ABI's");
constexpr int kMaxBlocks = PYRIT_MAX_BLOCKS;                      // k + m of a stripe
constexpr int kMaxJobs = (PYRIT_MAX_M + kMaxOut - 1) / kMaxOut;  // jobs of one stripe
static_assert(sizeof(JobDesc) == 1632, "the job descriptor size is documented in pyrit.h (no-alloc scratch)");

// Field degree w carried by the ring R_{2,n}: RingDim<n>::W for a run-time n.
inline int field_degree(int n) { return n == 9 ? 6 : n - 1; }
static_assert(RingDim<9>::W == 6 && RingDim<11>::W == 10, "field_degree follows RingDim");

// Dynamic shared memory of the staged kernel: S stages of W packets x tw bytes, 2 S + 1 mbarriers.
inline size_t staged_smem_bytes(int stages, int w, int tw) {
  return (size_t)stages * w * tw + sizeof(uint64_t) * (2 * stages + 1);
}

// A compiled instance of the staged ring kernel.
struct Variant {
  int n;         // ring size N (w = field_degree(N))
  int words;     // 32-bit words per consumer thread per packet
  int mg;        // outputs accumulated per consumer warp
  int minb;      // CTAs per SM the register budget is sized for
  int dispatch;  // 0: uniform test per shift; 1: switch per set bit; 2: pairing automaton;
                 // 3: a network generated for one mask table (PYRIT_DISPATCH_NETWORK)
  int nc;        // consumer warps per CTA (one more warp is the producer)
  const void* fn;
  int mode;      // generated networks: NetSpec mode (syndrome modes take syndrome-form jobs)
  int nout;      // generated networks: the output count they were compiled for (0: generic)
  int w;         // field degree: packets per block
  int track = 0; // generated networks: built to stamp each job's completion (NetSpec::track)
};

// Generated networks whose jobs are in syndrome form (modes 1 and 3).
inline bool syndrome_mode(int mode) { return mode == 1 || mode == 3; }

// Output groups of a launch: the smallest power of two g with g * mg >= nout (and g < nc); the
// consumer warps split evenly into them. Generated networks are compiled for this same split.
inline int output_groups(int mg, int nout, int nc) {
  int g = 1;
  while (g * mg < nout && g < nc) g *= 2;
  return g;
}

// Tile-shape choice of one launch.
struct TileShape {
  const Variant* v = nullptr;
  int groups = 1;  // output groups (power of two dividing the consumer warps)
  int tw = 0;      // tile width (bytes, multiple of 16)
  int stages = 0;  // pipeline depth
  int grid = 0;    // CTAs (0: SMs x occupancy)
};

// Optional overrides of the automatic shape choice (0 or -1 = automatic).
struct ShapeHint {
  int words = 0;
  int dispatch = -1;
  int mg = 0;
  int minb = 0;
  int nc = 0;
  int stages = 0;
  int ctas_per_sm = 0;
};

// ---- planner (host) -------------------------------------------------------------------------
// Native fields (generic kernels built for them): the AOP rings n = w + 1 in {3, 5, 11, 13} and
// GF(2^6) from x^6 + x^3 + 1 on n = 9.
bool field_native(int w, int n);
// The modulus of GF(2^w) on R_{2,n}: the native AOP / ESP, else the smallest irreducible factor of
// degree w of x^n + 1 (n odd <= 15); 0 if none.
uint32_t field_modulus(int w, int n);
uint32_t gf_mul(uint32_t g, int w, uint32_t a, uint32_t b);
uint32_t gf_inv(uint32_t g, int w, uint32_t a);
uint32_t sparse_rep(uint32_t g, int w, int n, uint32_t u);

struct DecodeEntry {
  int status = PYRIT_OK;
  int ne = 0;
  int surv[kMaxIn];
  int erased[kMaxBlocks];
  uint16_t mask[kMaxBlocks][kMaxIn];  // row r = erased block erased[r], column s = survivor surv[s]
  // Syndrome form (k + m <= kMaxIn, m <= kMaxOut): syn[r][o] = phi_S of the coefficient of row r's
  // accumulator for output o; syn[kSyndromeBaseRow][o] = 1 + the row whose partial sum output o
  // adds (an erased parity block), 0 for an erased data block.
  bool syn_ok = false;
  uint16_t syn[kSyndromeBaseRow + 1][kMaxOut];
};

}  // namespace pyrit

struct pyrit_plan_s {
  int w, n, k, m;
  uint64_t serial = 0;  // unique in the process (keys caches that must not confuse a new plan
                        // allocated at a destroyed plan's address with the old one)
  uint32_t g = 0;       // the field's modulus
  bool native = true;   // the generic kernels serve this field (else generated networks only)
  int transform = PYRIT_TRANSFORM_EMBEDDING;
  std::vector<uint32_t> G;         // (k+m) x k
  std::vector<uint16_t> enc_mask;  // m x k
  std::mutex mu;
  std::unordered_map<uint64_t, pyrit::DecodeEntry> dcache;
};

namespace pyrit {
// Looks up or computes the decoding matrix of `erasures` (thread-safe). Returns a status.
int plan_decode_entry(pyrit_plan_s* p, uint64_t erasures, DecodeEntry* out);
// Fills the jobs that encode one stripe: output group g (parity blocks 8g..8g+7) is jobs[g], each
// reading all k data blocks. Returns the job count, ceil(m / 8) (0 when m = 0).
int make_encode_jobs(const pyrit_plan_s* p, const void* const* data, void* const* parity, size_t P,
                     JobDesc* jobs /* [kMaxJobs] */);
// Validates a stripe request and builds its coding jobs (alg / src: algorithmic and source bytes);
// *njobs = how many (0 when there is nothing to code).
int stripe_jobs(const pyrit_stripe_t& s, JobDesc* jobs /* [kMaxJobs] */, int* njobs, uint64_t* alg, uint64_t* src);
// Fills the jobs that decode one stripe with a decode entry (erased blocks 8g..8g+7 in jobs[g]).
// Returns the job count, ceil(ne / 8).
int make_decode_jobs(const pyrit_plan_s* p, const DecodeEntry& e, void* const* blocks, size_t P,
                     JobDesc* jobs /* [kMaxJobs] */);
// Fills the syndrome-form decode job (requires e.syn_ok): sources are the k + m block columns in
// index order, absent (null) unless they are survivors; outputs are the erased blocks.
void make_syndrome_job(const pyrit_plan_s* p, const DecodeEntry& e, void* const* blocks, size_t P, JobDesc* job);

// ---- kernels (device launchers) --------------------------------------------------------------
// Registered variants (all translation units).
const Variant* variants(int* count);
const Variant* find_variant(int n, int words, int dispatch, int mg, int minb, int nc);
// True when every pointer of the job is 16-byte aligned and P is a multiple of 16.
bool job_is_staged(const JobDesc& j);
// Tile shape for ring size n, the largest output count of the launch's jobs and optional hints;
// shared_masks: every job of the launch has the same masks. Returns false if no variant matches.
bool choose_shape(int n, int max_nout, const ShapeHint& hint, TileShape* out, bool shared_masks = false);
// Tile shape of a given variant.
bool shape_for_variant(const Variant* v, int max_nout, const ShapeHint& hint, TileShape* out);

// ---- autotuner table (process-wide) ---------------------------------------------------------
// A launch group is keyed by ring size, whether its jobs share masks, its largest output count
// and its packet-size class (log2 P, or -1 when P varies).
struct TuneKey {
  int n, shared, nout, plog2;
  bool operator<(const TuneKey& o) const {
    return n != o.n ? n < o.n : shared != o.shared ? shared < o.shared : nout != o.nout ? nout < o.nout : plog2 < o.plog2;
  }
};
struct TuneVal {
  int words, mg, minb, nc, dispatch, stages;
  float ms;
};
bool tune_lookup(const TuneKey& k, TuneVal* v);
void tune_record(const TuneKey& k, const TuneVal& v);
// ---- plan-specialised networks (net_jit.cpp) ------------------------------------------------
// A network is the staged kernel with its multiply-accumulate step generated for one mask table:
// the XOR of rotated source packets that every (source, output) coefficient contributes is written
// out as straight-line code, so no mask bit is tested at run time. Generated, compiled (NVRTC) and
// cached per NetSpec; `mask` holds the table for j < nin, o < nout and zeros elsewhere.
struct NetSpec {
  int32_t n, nin, nout, words, mg, minb, nc;  // nout: the largest output count of its tables
  int32_t mode;  // 0 / 2: direct (the jobs' own tables), 1 / 3: syndrome decode of a plan (table
                 // [C | I]); 0 and 1 under the embedding transform, 2 and 3 under the parity one
  int32_t ntables;           // direct modes: tables; a job's JobDesc::table picks one (syndrome: 1)
  int32_t tnout[kMaxJobs];   // output count of each table
  int32_t w;                 // field degree (packets per block)
  uint32_t g;                // 0: the native field of R_{2,n}; else the modulus, a factor of x^n + 1
                             // whose reduction the network emits (direct mode 0 only)
  int32_t track;             // 1: the kernel counts each job's finished tiles and stamps its
                             // completion (launched by the server with CodeArgs::done_cnt / done_ns)
  int32_t allrows;           // syndrome modes: 1 adds a first-phase body for tiles that need every
                             // parity row (terms shared across rows), 0 keeps only the guarded rows
  int32_t pair;              // direct modes: 1 takes two staged sources per step, so that one
                             // three-input XOR can combine terms of both
  uint16_t mask[kMaxJobs][kMaxIn][kMaxOut];
};
// The network spec of one job under a shape (zero fields: the default shape for (n, nout)) and a
// transform (PYRIT_TRANSFORM_EMBEDDING or _PARITY): one table, which the job must select as 0.
NetSpec net_spec(int n, const JobDesc& job, int words, int mg, int minb, int nc, int transform, uint32_t g = 0);
// The network spec of several tables (each given by one job that uses it, all with the same nin):
// the jobs of a launch then carry their table's index in JobDesc::table.
NetSpec net_spec_tables(int n, const JobDesc* const* tables, int ntables, int words, int mg, int minb, int nc,
                        int transform, uint32_t g = 0);
// The `g` a plan's network specs take: 0 for a native field, else the plan's modulus.
inline uint32_t plan_net_g(const pyrit_plan_s* p) { return p->native ? 0u : p->g; }
// Plans that only generated networks code: the parity transform, or a field that the generic
// kernels are not built for.
inline bool network_only(const pyrit_plan_s* p) { return p->transform == PYRIT_TRANSFORM_PARITY || !p->native; }
// The syndrome-decode network spec of a plan, under its transform (requires k + m <= kMaxIn and
// m <= kMaxOut; zero fields: default).
NetSpec net_spec_syndrome(const pyrit_plan_s* p, int words, int minb, int nc, int allrows = 1);
// Candidate shapes of a plan's syndrome network, the default first.
int net_syndrome_shapes(const pyrit_plan_s* p, NetSpec* out, int cap, int allrows = 1);
// Candidate shapes for (n, nout), the default first; returns how many were written (<= cap).
int net_candidate_shapes(int n, int nout, NetSpec* out, int cap);
// Run-time compilation policy (PYRIT_JIT_*).
int jit_mode();
// The compiled network of `s` loaded on the current device, or nullptr. With block, a missing
// network is compiled now (or a pending one awaited); without, a missing one is queued for the
// background compiler when the policy is PYRIT_JIT_ASYNC and nullptr is returned until it is ready.
const Variant* net_variant(const NetSpec& s, bool block);
// Compiles a spec into the cache (host only, no device call). PYRIT_OK or PYRIT_E_JIT.
int net_compile(const NetSpec& s);
// Spill stores (bytes) the assembler reported for a compiled network; -1 if not compiled or unknown.
int net_spill_bytes(const NetSpec& s);

// Fills shape->grid (SMs x occupancy) if it is 0; makes the one-time per-device attribute calls.
void resolve_grid(TileShape* shape);
// Tiles of one job of packet size P under a shape.
inline uint32_t tiles_for(uint64_t P, const TileShape& s) { return (uint32_t)((P + s.tw - 1) / s.tw); }
// Launches the staged ring kernel. `jobs_dev` may be null for a single job passed by value. With
// done_cnt / done_ns (the served path) job j of the launch counts its finished warp-tiles in
// done_cnt[j] (zero before, left zero) and stamps done_ns[j] (host-mapped) when its last one ends.
int launch_staged(const TileShape& sh, const JobDesc* job0, const JobDesc* jobs_dev, const uint2* tiles_dev,
                  uint32_t ntiles, uint32_t tiles_per_job, cudaStream_t stream, uint32_t* done_cnt = nullptr,
                  uint64_t* done_ns = nullptr);
// Launches the plain-load kernel (any P and alignment) for one job.
int launch_plain(int n, const JobDesc& job, cudaStream_t stream);
// Device error word of the current device (allocated on first use), or nullptr on failure.
int* device_error_word();
// Multiprocessor count of the current device.
int sm_count();

}  // namespace pyrit
