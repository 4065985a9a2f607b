/*
 * pyrit.h -- C ABI of the GB300 PYRIT erasure codec.
 *
 * PYRIT (polynomial ring transform; Detchart & Lacan, arXiv:1709.00178) computes systematic MDS
 * erasure codes over the field GF(2^w) = F2[x]/(p(x)) by doing every multiplication in the ring
 * R_{2,n} = F2[x]/(x^n + 1). p is the all-one polynomial (AOP) of degree w with n = w + 1
 * (Sec. 2.3), or for GF(2^6) the equally spaced polynomial (ESP) x^6 + x^3 + 1 with n = 9
 * (Sec. 2.4); in both cases p divides x^n + 1.
 *   - each generator (or decoding-matrix) coefficient u is replaced by its sparsest ring
 *     representative phi_S(u) (Sec. 2.2, "the sparse transform");
 *   - each source block is embedded in the ring by padding it with n - w zero packets (phi_E,
 *     Sec. 2.3.2, 2.4.2), so multiplying it by x^s is a cyclic rotation of its packets and
 *     multiplying by phi_S(u) is an XOR of one rotation per set bit of phi_S(u) (Sec. 3);
 *   - the ring result is mapped back to the field by the remainder mod p: for an AOP "XOR the top
 *     packet into every other packet", for the ESP "XOR the top three packets into both lower
 *     groups of three" (phi_E^{-1}).
 *
 * Data layout. A block is w packets of P bytes, contiguous, packet q at byte offset q*P. Bit b of
 * byte t of packet q is coefficient q (of x^q) of the field symbol in lane (t, b); every lane is
 * an independent codeword. A stripe is k data blocks and m parity blocks; block index e runs
 * over data (0..k-1) then parity (k..k+m-1).
 *
 * Ownership. The caller owns every data buffer (device memory, e.g. a torch tensor's data_ptr());
 * the library owns plans, batches, servers and the device memory they hold.
 *
 * Asynchrony. Coding calls enqueue work on the caller's stream and return; they never
 * synchronise except where stated. Buffers must stay valid until that work completes.
 *
 * Errors. Every int-returning call returns PYRIT_OK (0) or a negative PYRIT_E_* code and never
 * launches work when it fails validation. No C++ exception crosses this boundary.
 * pyrit_strerror() names a code.
 *
 * Alignment. The staged (TMA) kernel is used when P is a multiple of 16 and every block pointer
 * is 16-byte aligned; any other P or alignment is accepted and coded by a plain-load kernel.
 */
#ifndef PYRIT_H
#define PYRIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exported symbols (the library is built with hidden visibility by default). */
#if defined(__GNUC__)
#define PYRIT_API __attribute__((visibility("default")))
#else
#define PYRIT_API
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* pyrit_stream_t;

/* ---- status codes ------------------------------------------------------------------------ */
#define PYRIT_OK 0
#define PYRIT_E_INVALID_ARG -1        /* null pointer, P = 0, k/m out of range, bad mask bits  */
#define PYRIT_E_UNSUPPORTED_FIELD -2  /* x^n + 1 (n odd, 3 <= n <= 15) has no irreducible
                                         factor of degree w                                     */
#define PYRIT_E_TOO_LONG -3           /* k + m > 2^w: the default Cauchy code needs distinct points */
#define PYRIT_E_NOT_MDS -4            /* generator not systematic, entry >= 2^w, or a singular
                                         k x k submatrix was found                              */
#define PYRIT_E_TOO_MANY_ERASURES -5  /* more than m blocks erased                              */
#define PYRIT_E_CUDA -6               /* a CUDA runtime call failed                             */
#define PYRIT_E_OOM -7                /* host or device allocation failed                       */
#define PYRIT_E_BUDGET -8             /* server: request larger than the admission budget      */
#define PYRIT_E_TIMEOUT -9            /* a bounded device or host wait gave up                  */
#define PYRIT_E_BUSY -10              /* server: request queue full, retry later               */
#define PYRIT_E_SCRATCH_LIMIT -11     /* more stripes or tiles than pyrit_code_stripes_noalloc's
                                         fixed scratch holds                                     */
#define PYRIT_E_JIT -12               /* run-time compilation or loading of a plan-specialised
                                         network failed (pyrit_jit_log has the compiler's log)  */
#define PYRIT_E_UNSUPPORTED -13       /* the request needs a path this build does not provide for
                                         it: the parity transform outside generated networks, or
                                         a stripe of several jobs (more than PYRIT_JOB_OUTPUTS
                                         parity or erased blocks) in the server or the
                                         allocation-free entry point                             */

/* Limits of this build. */
#define PYRIT_MAX_K 64      /* data blocks per stripe                                     */
#define PYRIT_MAX_M 63      /* parity blocks per stripe                                   */
#define PYRIT_MAX_BLOCKS 64 /* k + m (erasure patterns are 64-bit masks)                  */
#define PYRIT_JOB_OUTPUTS 8 /* outputs one coding job writes: a stripe with more parity (or
                               erased) blocks is coded as ceil(count / 8) jobs that read the
                               same sources                                               */

/* Operations. */
#define PYRIT_OP_ENCODE 0
#define PYRIT_OP_DECODE 1
#define PYRIT_OP_DECODE_ANY 2 /* pyrit_plan_specialise only: the plan's syndrome-decode network */

/* Name of a status code (static string). */
PYRIT_API const char* pyrit_strerror(int status);

/* ---- plan (host only; no GPU needed) ------------------------------------------------------ */

typedef struct pyrit_plan_s* pyrit_plan_t;

/* Creates a coding plan for a systematic (k+m, k) code over GF(2^w) carried by R_{2,n}.
 *   w, n : field degree and ring size. Either n = w + 1 with the AOP of degree w irreducible
 *          (w+1 prime with 2 a primitive root mod w+1, Sec. 2.3), or the s-ESP of degree w = s r,
 *          n = s (r + 1), irreducible by the criterion Sec. 2.4 quotes. The generic kernels are
 *          built for (w, n) in {(2, 3), (4, 5), (6, 9), (10, 11), (12, 13)}; (6, 9) is GF(2^6)
 *          from x^6 + x^3 + 1. Any other odd n <= 15 with an irreducible factor of degree w of
 *          x^n + 1 (Props. 1-2; e.g. GF(8) on n = 7, GF(16) from x^4 + x + 1 on n = 15) gives a
 *          field whose modulus is the smallest such factor: the embedding only, coded by generated
 *          networks only (single calls and batches; the server and the allocation-free entry point
 *          return PYRIT_E_UNSUPPORTED).
 *   k, m : 1 <= k <= PYRIT_MAX_K, 0 <= m <= PYRIT_MAX_M, k + m <= PYRIT_MAX_BLOCKS.
 *   G    : NULL for the default generator [I_k ; C], C[i][j] = 1/(x_i + y_j) with x_i = k+i,
 *          y_j = j (a Cauchy matrix, Sec. 3 "generalized Cauchy matrices"; requires
 *          k + m <= 2^w), or a host array of (k+m)*k uint32 entries, row-major, whose top k rows
 *          must be the identity. A user G is checked for the MDS property (every k x k row
 *          subset invertible, Sec. 2.2) when there are at most 20000 subsets; otherwise a
 *          singular subset is reported by pyrit_decode as PYRIT_E_NOT_MDS.
 * Computes phi_S of every parity coefficient (Sec. 2.2). Host memory only: no device call.
 * On success *out owns the plan; release it with pyrit_plan_destroy. */
PYRIT_API int pyrit_plan_create(int w, int n, int k, int m, const uint32_t* G, pyrit_plan_t* out);

/* pyrit_plan_create with 16-bit generator entries (every field this build codes has w <= 15, so
 * an entry fits; G NULL: the default generator). Same checks, codes and ownership. */
PYRIT_API int pyrit_plan(int w, int n, int k, int m, const uint16_t* G, pyrit_plan_t* out);
PYRIT_API void pyrit_plan_destroy(pyrit_plan_t plan);

/* A weight-optimised generalized Cauchy generator to pass to pyrit_plan_create (Sec. 3 codes with
 * "generalized Cauchy matrices"; Sec. 2.2 makes the cost the number of ones of the sparse ring
 * representatives). G_out[(k+m)*k] = [I_k ; C'] with C'[i][j] = a_i b_j / (x_i + y_j),
 * x_i = k+i, y_j = j: row and column scalings of the default Cauchy matrix, which keep every
 * square submatrix nonsingular (the code stays MDS). The scalings are chosen by coordinate descent
 * on the total weight of phi_S over C': starting from a = b = 1, each round sets every b_j
 * (ascending j), then every a_i (ascending i), to the nonzero element minimising the weight summed
 * over its column (row), the smallest element on ties, until a round changes nothing (at most 8
 * rounds). weights_out[2] (may be NULL): total weight of the default and of the returned parity
 * part. Host only; deterministic. Errors: as pyrit_plan_create for (w, n, k, m). */
PYRIT_API int pyrit_generator_weighted(int w, int n, int k, int m, uint32_t* G_out, uint64_t* weights_out);

/* Field-to-ring transform of a plan (Sec. 2.3.1-2.3.2). EMBEDDING (the default): phi_E pads each
 * block with a zero packet and phi_E^{-1} reduces mod p; the code is the field code. PARITY:
 * phi_P pads each source block with its parity packet and phi_P^{-1} drops the top packet; encoder
 * and decoder must both use it, and the code is the field code conjugated symbol by symbol by
 * psi(d) = d + par(d)(1 + x + ... + x^{w-1}). AUTO: the paper's rule, parity when k < m. The
 * parity transform runs only on generated networks (pyrit_jit_mode must not be OFF): batches whose
 * parity-transform stripes cannot use one (mixed tables of several plans, an unaligned stripe),
 * the server and pyrit_code_stripes_noalloc return PYRIT_E_UNSUPPORTED for them. */
#define PYRIT_TRANSFORM_EMBEDDING 0
#define PYRIT_TRANSFORM_PARITY 1
#define PYRIT_TRANSFORM_AUTO 2

/* Sets the plan's transform (before it codes anything: a plan must not change code mid-stream).
 * Returns the transform now in force (AUTO resolved) or PYRIT_E_INVALID_ARG. */
PYRIT_API int pyrit_plan_set_transform(pyrit_plan_t plan, int transform);

/* Plan parameters (any pointer may be NULL). */
PYRIT_API int pyrit_plan_info(pyrit_plan_t plan, int* w, int* n, int* k, int* m);

/* The plan's field: its modulus g (bit i = coefficient of x^i) and whether the generic kernels are
 * built for it (*native_out = 1 for the AOP rings and GF(2^6) on n = 9; 0 for a field from another
 * factor of x^n + 1, which only generated networks code). Any pointer may be NULL. */
PYRIT_API int pyrit_plan_modulus(pyrit_plan_t plan, uint32_t* g_out, int* native_out);

/* Copies the (k+m) x k generator, row-major, into G_out. */
PYRIT_API int pyrit_plan_generator(pyrit_plan_t plan, uint32_t* G_out);

/* Copies the m x k ring masks of the parity rows, row-major: masks_out[i*k + j] = phi_S(G[k+i][j])
 * as an n-bit mask (bit s = coefficient of x^s). */
PYRIT_API int pyrit_plan_encode_masks(pyrit_plan_t plan, uint16_t* masks_out);

/* The decoding matrix for an erasure pattern (bit e of `erasures` = block e lost), as ring masks:
 * the survivors are the first k non-erased blocks in index order; every erased block is rebuilt:
 * an erased data block e from row e of Inv = (G restricted to the survivors' rows)^{-1}, an erased
 * parity block from G[e] * Inv (Sec. 4.3: the decoding matrix depends on the loss pattern).
 * Outputs (host arrays): survivors_out[k]; erased_out[ne] (ascending); masks_out[ne*k] with
 * masks_out[r*k + s] = phi_S(D[r][s]); *ne_out = number of erased blocks (may be 0).
 * Computed once per (plan, pattern) and cached in the plan. */
PYRIT_API int pyrit_plan_decode_masks(pyrit_plan_t plan, uint64_t erasures, int* survivors_out,
                            int* erased_out, uint16_t* masks_out, int* ne_out);

/* The syndrome form of the decoding for an erasure pattern (used by the plan's syndrome-decode
 * network; requires m <= PYRIT_JOB_OUTPUTS). With U the first a surviving parity rows (a = erased
 * data blocks) and, for parity row r, acc_r = (sum of C[r][j] d_j over surviving data j) + p_r
 * when r is in U, every erased block (ascending, as in pyrit_plan_decode_masks) is a sum of the
 * rows' values: output o = acc_{base-1} (when base = syn_out[8*8 + o] > 0: an erased parity block
 * adds its own partial sum) + sum over rows r of phi_S^{-1}(syn_out[r*8 + o]) * acc_r.
 * syn_out: host array of 9 x 8 uint16 (rows r = 0..7, then the base row), zero past the erased
 * count *ne_out. Host only. */
PYRIT_API int pyrit_plan_syndrome_masks(pyrit_plan_t plan, uint64_t erasures, uint16_t* syn_out, int* ne_out);

/* phi_S of one field element u < 2^w: the lightest of its 2^(n-w) ring representatives
 * u + h(x) p(x), deg h < n - w (Sec. 2.2; the smallest integer on ties, which an AOP with odd n
 * never has).
 * Returns the n-bit mask, or 0xFFFFFFFF for a bad argument. */
PYRIT_API uint32_t pyrit_sparse_transform(int w, int n, uint32_t u);

/* Field product in GF(2^w) under the library's modulus for w (the ESP x^6 + x^3 + 1 for w = 6, else
 * the AOP of degree w), computed by the planner (host). */
PYRIT_API uint32_t pyrit_gf_mul(int w, uint32_t a, uint32_t b);

/* ---- single-stripe coding (device; asynchronous on `stream`) ------------------------------ */

/* Encodes one stripe: parity[i] = sum_j G[k+i][j] * data[j] in every symbol lane.
 *   data   : host array of k device pointers, each to a block of w*P bytes (read).
 *   parity : host array of m device pointers, each to a block of w*P bytes (written).
 *   P      : packet bytes, >= 1.
 * The fused ring kernel stages the sources through shared memory with bulk-async copies,
 * embeds them (phi_E), accumulates XORs of packet rotations for every set bit of phi_S(G[k+i][j])
 * and reduces mod p (phi_E^{-1}) before storing. No coding state is allocated on the device (the
 * first use of a generated network loads its module: see "plan-specialised networks"). */
PYRIT_API int pyrit_encode(pyrit_plan_t plan, const void* const* data, void* const* parity, size_t P,
                 pyrit_stream_t stream);

/* Decodes one stripe in place: every block whose bit is set in `erasures` is rebuilt.
 *   blocks    : host array of k+m device pointers (data then parity); erased blocks are written,
 *               the others read.
 *   erasures  : bit e set = block e lost; popcount <= m, else PYRIT_E_TOO_MANY_ERASURES.
 * The decoding matrix comes from the plan's cache (a miss computes it on the host, Sec. 4.3).
 * Erasures == 0 is a no-op. */
PYRIT_API int pyrit_decode(pyrit_plan_t plan, void* const* blocks, uint64_t erasures, size_t P,
                 pyrit_stream_t stream);

/* ---- batched coding: many stripes in one persistent launch -------------------------------- */

typedef struct pyrit_batch_s* pyrit_batch_t;

/* One stripe of a batch. */
typedef struct {
  pyrit_plan_t plan;    /* the stripe's code (plans may differ between stripes)              */
  int op;               /* PYRIT_OP_ENCODE or PYRIT_OP_DECODE                                 */
  uint64_t erasures;    /* decode: bit e set = block e lost (ignored for encode)              */
  size_t packet_bytes;  /* P >= 1                                                             */
  void* const* blocks;  /* host array of k+m device pointers: data 0..k-1, parity k..k+m-1;
                           encode writes parity, decode rewrites the erased blocks            */
} pyrit_stripe_t;

/* Tile-shape overrides for a batch; a zero field (dispatch: -1) means automatic. */
typedef struct {
  int words;        /* 32-bit words per consumer thread per packet (1 or 2)              */
  int mg;           /* outputs accumulated per consumer warp (2, 4 or 8)                 */
  int minb;         /* CTAs per multiprocessor the kernel's registers are sized for      */
  int nc;           /* consumer warps per CTA (8 or 16)                                  */
  int dispatch;     /* 0: uniform test per ring shift; 1: switch per set mask bit;
                       2: pairing automaton; 3 (PYRIT_DISPATCH_NETWORK): a network generated
                       for the group's mask table (every stripe of the group must share it)  */
  int stages;       /* shared-memory pipeline depth (2..8)                               */
  int ctas_per_sm;  /* persistent grid = multiprocessors x ctas_per_sm                   */
} pyrit_tile_t;

/* Prepares a batch: validates every stripe (the same checks and codes as pyrit_encode /
 * pyrit_decode), resolves the decoding matrices through the plans' caches, builds one coding job
 * per stripe (stripes with nothing erased are dropped) and a work list of column tiles, and copies
 * both to library-owned device memory (synchronous). Stripes are grouped by ring size (stripes that
 * the generic kernel codes also by output count: 1-2, 3-4 or 5-8 per job, so that a launch's shape
 * fits its jobs); each group is one persistent launch of the staged kernel in which every CTA walks
 * the tile list. Stripes whose
 * P or pointers do not allow 16-byte bulk copies run on the plain-load kernel, one launch each.
 *   stripes : host array of `count` stripes (copied; the block pointer arrays are read here only).
 *   tile    : NULL for the automatic shape, else overrides.
 * The batch keeps pointers to the caller's buffers: they must stay valid while it is run. */
PYRIT_API int pyrit_batch_create(const pyrit_stripe_t* stripes, int count, const pyrit_tile_t* tile,
                       pyrit_batch_t* out);

/* Enqueues the batch's launches on `stream` (asynchronous). With graph != 0 the launches are
 * captured once into a CUDA graph on first use and replayed from then on. */
PYRIT_API int pyrit_batch_run(pyrit_batch_t batch, pyrit_stream_t stream, int graph);

/* Autotunes the batch: for every launch group, times each compiled kernel variant of its ring size
 * (one warm-up and `iters` timed launches of the real work, on `stream`; coding is idempotent, so
 * the caller's outputs end up as one run leaves them) and keeps the fastest shape. The choice is
 * recorded in the process-wide tuning table, keyed by ring size, shared-or-mixed masks, output
 * count and packet-size class, which later pyrit_batch_create calls without tile overrides use.
 * Synchronises `stream`; drops a captured graph. */
PYRIT_API int pyrit_batch_tune(pyrit_batch_t batch, pyrit_stream_t stream, int iters);

/* Saves / loads the tuning table as JSON (one object per key). Load returns the number of entries
 * read (>= 0) or a negative status. */
PYRIT_API int pyrit_tune_save(const char* path);
PYRIT_API int pyrit_tune_load(const char* path);

/* Forgets every tuned shape (later batches use the automatic choice); returns how many there were. */
PYRIT_API int pyrit_tune_clear(void);

/* The compiled kernel variants, for introspection and tuning: writes up to `cap` rows of six ints
 * (n, words, mg, minb, dispatch, nc) into params_out (host) and returns the total count. */
PYRIT_API int pyrit_variants(int* params_out, int cap);

/* Algorithmic HBM bytes of one run ((k + m) * w * P per encoded stripe, (k + e) * w * P per
 * decoded stripe with e erasures), source bytes (k * w * P per stripe), launches per run and
 * column tiles. Any pointer may be NULL. */
PYRIT_API int pyrit_batch_stats(pyrit_batch_t batch, uint64_t* alg_bytes, uint64_t* src_bytes, int* launches,
                      uint64_t* tiles);

/* The launch shape of group `group` (0-based, groups ordered by ring size) of a batch, as eleven
 * ints: n, words, mg, minb, dispatch, nc, output groups, tile bytes, pipeline stages, grid CTAs,
 * network mode. dispatch 3 marks a plan-specialised network, of the group's own mask table (mode
 * 0) or a plan's syndrome decode (mode 1). PYRIT_E_INVALID_ARG past the last group. */
PYRIT_API int pyrit_batch_shape(pyrit_batch_t batch, int group, int* params_out);

/* Frees the batch's device memory and graph (synchronises the device). */
PYRIT_API void pyrit_batch_destroy(pyrit_batch_t batch);

/* One-shot batched coding under the names of the hot path's boundary: pyrit_batch_create over the
 * `count` stripes (automatic shapes), one pyrit_batch_run on `stream`, a wait for its launches, then
 * pyrit_batch_destroy. Every stripe must carry PYRIT_OP_ENCODE (pyrit_encode_batch) or
 * PYRIT_OP_DECODE (pyrit_decode_batch). Each call allocates and frees the batch's device tables and
 * synchronises `stream`; a batch coded again and again belongs in pyrit_batch_create /
 * pyrit_batch_run. Returns PYRIT_OK (also for count == 0), PYRIT_E_INVALID_ARG for a NULL array,
 * a negative count or a stripe of the other operation (before any device work), the codes of
 * pyrit_batch_create, or PYRIT_E_CUDA when the launches or the wait fail. */
PYRIT_API int pyrit_encode_batch(const pyrit_stripe_t* stripes, int count, pyrit_stream_t stream);
PYRIT_API int pyrit_decode_batch(const pyrit_stripe_t* stripes, int count, pyrit_stream_t stream);

/* ---- plan-specialised networks (run-time compilation) ---------------------------------------
 *
 * The generic kernels test every bit of phi_S(u) at run time to decide which packet rotations to
 * XOR (Sec. 3). When every job of a launch shares one mask table -- the stripes of one code and
 * operation, or decodes of one erasure pattern -- the library can instead generate the kernel's
 * multiply-accumulate step for that table: per source, each ring accumulator receives one XOR
 * expression over the rotated source packets that the coefficient's set bits select, with no bit
 * tested. The generated step is compiled with NVRTC into an sm_103a cubin together with the same
 * staging, phi_E^{-1} and store code as the generic kernels, cached per (shape, mask table) for the
 * life of the process (at most 1024 networks, never unloaded) and loaded as a CUDA library.
 *
 * Where it is used. pyrit_batch_create specialises every launch group whose stripes share one mask
 * table, compiling in the calling thread (about a second per new table), unless the policy is
 * PYRIT_JIT_OFF or tile overrides are given (tile->dispatch = 3 asks for a network with the
 * tile's words, mg, minb and nc); pyrit_batch_tune times the network shapes beside the generic
 * variants. pyrit_encode / pyrit_decode and the server use a network
 * when one for the job's table is already compiled; otherwise, under PYRIT_JIT_ASYNC, they queue
 * it for a background compiler thread (at most 16 waiting) and run the generic kernel meanwhile.
 * pyrit_code_stripes_noalloc never uses networks (loading one allocates device memory).
 * A network that fails to compile or load leaves the generic kernel in use (pyrit_jit_stats counts
 * the failure; pyrit_jit_log has the log), except where tile overrides ask for dispatch 3, which
 * then fails with PYRIT_E_JIT. */
#define PYRIT_DISPATCH_NETWORK 3
#define PYRIT_JIT_OFF 0   /* generic kernels only                                              */
#define PYRIT_JIT_SYNC 1  /* compile a missing network in the calling thread, then use it     */
#define PYRIT_JIT_ASYNC 2 /* default: batches compile in the caller; single calls and the
                             server queue a missing network and use the generic kernel meanwhile */

/* Sets the process-wide policy (PYRIT_JIT_*) and returns the previous one; mode < 0 only queries. */
PYRIT_API int pyrit_jit_mode(int mode);

/* Compiles (host only, no device call) the network of a plan's encode (op PYRIT_OP_ENCODE), of
 * its decode for one erasure pattern (PYRIT_OP_DECODE), or its syndrome-decode network, which
 * serves every erasure pattern (PYRIT_OP_DECODE_ANY; requires m <= PYRIT_JOB_OUTPUTS), into the
 * cache, so that later calls find it: in two forms, compiled side by side, the one batches and
 * single calls launch and the one servers launch (it also stamps each request's completion, a step
 * the other form leaves out because even unused it slows the kernel).
 * tile: NULL for the default shape, else its words, mg, minb and nc (0 = default) select one.
 * PYRIT_OK (also when there is nothing to code), a planning error, or PYRIT_E_JIT. */
PYRIT_API int pyrit_plan_specialise(pyrit_plan_t plan, int op, uint64_t erasures, const pyrit_tile_t* tile);

/* Resource use of the network pyrit_plan_specialise would compile for the same arguments (it is
 * compiled first if missing; host only). info_out[9] (host): registers per thread, stack frame,
 * spill stores and spill loads in bytes (from the assembler's report; -1 if it gave none), compile
 * time in ms, then the network's words, mg, nc and mode (0 direct, 1 syndrome, 2 direct under the
 * parity transform, 3 syndrome under the parity transform). PYRIT_E_INVALID_ARG when there is
 * nothing to code, a planning error, or PYRIT_E_JIT. */
PYRIT_API int pyrit_plan_network_info(pyrit_plan_t plan, int op, uint64_t erasures, const pyrit_tile_t* tile,
                                      int* info_out);

/* The CUDA C++ source of the network pyrit_plan_specialise would compile for the same arguments
 * (the first job's, for a stripe of several jobs), NUL-terminated (truncated to cap - 1) into buf;
 * returns its length, PYRIT_E_INVALID_ARG when there is nothing to code, or a planning error.
 * For inspection and tests; host only. */
PYRIT_API int pyrit_plan_network_source(pyrit_plan_t plan, int op, uint64_t erasures, const pyrit_tile_t* tile,
                                        char* buf, int cap);

/* Waits up to timeout_ms for the background compiler to finish its queue: PYRIT_OK or
 * PYRIT_E_TIMEOUT. */
PYRIT_API int pyrit_jit_wait(int timeout_ms);

/* Drops the background compiler's queued specs (they are compiled again when next needed) and
 * waits up to timeout_ms for a compilation in progress: PYRIT_OK or PYRIT_E_TIMEOUT. For process
 * shutdown (the Python binding calls it at interpreter exit) and for tests. */
PYRIT_API int pyrit_jit_quiesce(int timeout_ms);

/* stats_out[8]: networks cached, compiled, failed, compilations pending, lookups that returned a
 * network, networks loaded, total compile time (us), specs ever queued for the background. */
PYRIT_API int pyrit_jit_stats(uint64_t* stats_out);

/* Copies the log of the last failed compilation or load (NUL-terminated, truncated to cap - 1)
 * into buf; returns its full length. */
PYRIT_API int pyrit_jit_log(char* buf, int cap);

/* The CUDA C++ source generated for a mask table (masks[o*nin + j] = phi_S mask of output o,
 * source j, as in pyrit_plan_encode_masks) over R_{2,n}, under the default shape or tile's
 * overrides, for the embedding or the parity transform (PYRIT_TRANSFORM_*). Copies it NUL-terminated (truncated to cap - 1) into buf and returns its length, or
 * PYRIT_E_INVALID_ARG. For inspection and tests; host only. */
PYRIT_API int pyrit_jit_source(int n, int nin, int nout, const uint16_t* masks, const pyrit_tile_t* tile,
                               int transform, char* buf, int cap);

/* ---- served coding: continuous batching ---------------------------------------------------- */

typedef struct pyrit_server_s* pyrit_server_t;

/* One served request: a stripe (any plan, operation and packet size; P a multiple of 16 and
 * 16-byte aligned blocks), the caller's tag, and its arrival time on the server clock (ns since the
 * server was created; <= 0: the time of submission). */
typedef struct {
  pyrit_stripe_t stripe;
  uint64_t tag;
  int64_t arrival_ns;
} pyrit_request_t;

/* A finished request: times on the server clock. start_ns is when the scheduler launched the batch
 * that coded it; done_ns when the scheduler saw the request's own completion stamp (written by the
 * kernel when the request's last tile was stored, before the rest of a shared launch ends). status
 * is PYRIT_OK, or PYRIT_E_TIMEOUT when the launch ended without completing the request (a bounded
 * device wait gave up), or PYRIT_E_CUDA when the launch failed. */
typedef struct {
  uint64_t tag;
  int status;
  int64_t arrival_ns, start_ns, done_ns;
} pyrit_completion_t;

/* Starts a server on the current device. A scheduler thread admits submitted requests in arrival
 * order while the device bytes of the requests in flight ((k+m) w P each) stay within hbm_budget,
 * and whenever one of `slots` stream slots is free it packs the admitted requests (at most
 * max_batch) into one batch, coded on the slot's stream by one persistent launch per kernel: the
 * plan's compiled network (encode table or syndrome decode) where it has one, else the staged
 * ring kernel per ring size. A launch of one request passes its job in the kernel parameters;
 * larger launches copy their jobs into the slot's device descriptor table first. Batches on
 * different slots overlap on the device; new arrivals join the next free slot (continuous
 * batching). Each request completes on its own: the kernel stamps a request done when its last
 * tile is stored, and the scheduler then retires it and releases its admission bytes, while the
 * slot itself is reused once its launches have ended. The scheduler thread spins (yielding) while
 * any work is in flight, keeps polling for 0.5 ms once idle (a request arriving then starts without
 * a thread wake-up), and then sleeps. Decoding matrices come from the plans' caches;
 * launch shapes from the autotuner's table when it has the key. queue_cap bounds the requests
 * waiting for admission. Allocates its slots' device tables, pinned staging and host-mapped
 * completion stamps. */
PYRIT_API int pyrit_server_create(size_t hbm_budget, int max_batch, int slots, int queue_cap, pyrit_server_t* out);

/* Validates and enqueues requests (all or none). Errors before any device work: the codes of
 * pyrit_batch_create, PYRIT_E_BUDGET for a stripe larger than the budget, PYRIT_E_INVALID_ARG
 * for a misaligned stripe or one too large for a slot, PYRIT_E_BUSY when the queue is full. */
PYRIT_API int pyrit_server_submit(pyrit_server_t server, const pyrit_request_t* reqs, int count);

/* Replays a request trace against the server from the calling thread: submits each request (as
 * pyrit_server_submit) once the server clock reaches its arrival_ns, all requests whose time has
 * come in one call, spinning in between, and returns when the last has been submitted (it does
 * not wait for completions). Requests must be in non-decreasing arrival order. A load generator
 * for measuring served latency without a caller-side submission delay: each request is validated
 * when it arrives, as a client's would be. Returns PYRIT_OK, PYRIT_E_INVALID_ARG (before any
 * submission) for NULL arguments or an arrival out of order, or the first failing submission's
 * code (the requests before it were submitted). */
PYRIT_API int pyrit_server_replay(pyrit_server_t server, const pyrit_request_t* reqs, int count);

/* Moves up to `cap` completions into out (host array); returns how many. */
PYRIT_API int pyrit_server_poll(pyrit_server_t server, pyrit_completion_t* out, int cap);

/* Waits until every submitted request has completed, for at most timeout_ms: PYRIT_OK, or
 * PYRIT_E_TIMEOUT when the limit passes first (the requests keep running). */
PYRIT_API int pyrit_server_drain(pyrit_server_t server, int timeout_ms);

/* The server clock: ns since the server was created (host steady clock). */
PYRIT_API int64_t pyrit_server_now_ns(pyrit_server_t server);

/* stats_out[7]: submitted, completed, batches, launches, bytes in flight, largest bytes in flight
 * observed, budget. */
PYRIT_API int pyrit_server_stats(pyrit_server_t server, uint64_t* stats_out);

/* Waits for every submitted request, stops the scheduler and frees the server. */
PYRIT_API void pyrit_server_destroy(pyrit_server_t server);

/* ---- coding without device allocation --------------------------------------------------- */

#define PYRIT_NOALLOC_MAX_STRIPES 256  /* stripes per call                                       */
#define PYRIT_NOALLOC_MAX_TILES 16384  /* column tiles per call (about P / 1 KiB per stripe)     */

/* Codes up to PYRIT_NOALLOC_MAX_STRIPES stripes (each encode or decode, as in pyrit_batch_create)
 * without allocating any device memory. The paper has no counterpart: this exists for callers that
 * cannot call cudaMalloc -- an I/O path whose device memory is wholly reserved by another allocator
 * (a framework's caching pool or a pre-sized arena, where cudaMalloc fails or eats into that pool),
 * or a latency-bound path that cannot take cudaMalloc's implicit device synchronisation.
 *
 * Scratch. The job descriptors, the tile list and two status words live in one fixed file-scope
 * device array of 536 KiB (256 + PYRIT_NOALLOC_MAX_STRIPES * 1632 + PYRIT_NOALLOC_MAX_TILES * 8
 * bytes) inside the library's module image: every GPU that loads the library holds it until the
 * process exits. The caller passes every input and output buffer; no cudaMalloc, cudaFree or other
 * allocating routine is called (on the host, a decoding matrix for an erasure pattern that a plan has
 * not seen is computed and kept in the plan's cache, as pyrit_decode does).
 * Set-up. The first call on each device, with that device current, looks up the array's device
 * address (cudaGetSymbolAddress).
 * Capture. The call uploads its descriptors from static pageable host arrays that the next call
 * rewrites, so it cannot be captured into a CUDA graph: on a stream that is capturing it returns
 * PYRIT_E_INVALID_ARG before any device work (call it eagerly).
 * Sharing. Every call reuses the same array, which keeps the last call's contents; each call clears
 * the status words and rewrites the descriptors on `stream` before its launches. Calls whose work
 * overlaps on the GPU (for example on two streams at once) race on the array: order them on one
 * stream or wait between them. Host callers are serialised by a lock.
 * Errors. More than PYRIT_NOALLOC_MAX_STRIPES stripes or PYRIT_NOALLOC_MAX_TILES tiles returns
 * PYRIT_E_SCRATCH_LIMIT before any device work; invalid stripes (and a ring size no kernel is built
 * for) return the codes of pyrit_batch_create, also before any device work. A device-side bounded
 * wait that gives up (its outputs are then incomplete) is recorded in the array's status words,
 * not in the word pyrit_device_status reads: read it with pyrit_noalloc_status after the call's work
 * and before the next call, which clears the words. Asynchronous on `stream` otherwise. */
PYRIT_API int pyrit_code_stripes_noalloc(const pyrit_stripe_t* stripes, int count, pyrit_stream_t stream);

/* Reads and clears the status words of pyrit_code_stripes_noalloc's fixed array on the current
 * device, after the work already queued on `stream` (synchronises `stream`). *code_out receives 0 or
 * PYRIT_E_TIMEOUT (a bounded device wait gave up); *where_out (may be NULL) the kernel site id. Like
 * the entry point it serves (the paper has no counterpart), it allocates nothing: one copy into the
 * caller's stack and one memset of the array. */
PYRIT_API int pyrit_noalloc_status(int* code_out, int* where_out, pyrit_stream_t stream);

/* ---- device status ----------------------------------------------------------------------- */

/* Reads and clears the device-side error word of the current device (synchronises the device).
 * Kernels set it when a bounded wait gives up (PYRIT_E_TIMEOUT) instead of spinning forever.
 * *code_out receives 0 or a PYRIT_E_* code; *where_out (may be NULL) a kernel-specific site id. */
PYRIT_API int pyrit_device_status(int* code_out, int* where_out);

/* Self-test of the bounded waits (no counterpart in the paper): enqueues on `stream` one thread that
 * waits, with the same bounded mbarrier wait every pipeline stage uses, on a barrier that nothing
 * completes, for limit_ns (1 ns .. 1 s). The wait gives up, records PYRIT_E_TIMEOUT and site 100,
 * and the kernel returns normally: the context stays usable. channel 0 records into the word
 * pyrit_device_status reads, channel 1 into the status words pyrit_noalloc_status reads. For
 * callers that want to check, on their own device, that a wait that runs out is reported. */
PYRIT_API int pyrit_selftest_bounded_wait(int channel, uint64_t limit_ns, pyrit_stream_t stream);

/* ---- synthetic inputs (device) ------------------------------------------------------------ */

/* Fills dst[0, nbytes) with bytes [offset, offset + nbytes) of the counter-mode SplitMix64 stream
 * `seed` (word i = mix(seed + (i+1) * 0x9E3779B97F4A7C15), little-endian bytes; Steele et al.,
 * OOPSLA 2014). Input generator for tests and benchmarks; no coding arithmetic. */
PYRIT_API int pyrit_synth_fill(void* dst, size_t nbytes, uint64_t seed, uint64_t offset,
                     pyrit_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PYRIT_H */
