// Plan-specialised ring networks: the staged kernel with its multiply-accumulate step generated
// for one mask table, compiled at run time (NVRTC) and loaded as a CUDA library.
//
// The generic kernels apply a coefficient r = phi_S(u) by testing its bits at run time: one XOR of
// the source rotated by s packets per set bit s (paper Sec. 3). When every job of a launch has the
// same mask table (all stripes of one code and operation: an encode batch, or decodes of one
// erasure pattern) those tests are known before the launch. The generated step writes them out:
// for source j and output i, ring accumulator t receives the XOR of the source packets
// q = t - s (mod N) over the set bits s of r_ij, where q = W (the zero packet that phi_E pads,
// Sec. 2.3.2) drops out -- one XOR expression per accumulator, no bit tested, with pairs and
// triples of packets that several accumulators receive formed once (share_terms). Per source the
// kernel takes one warp-uniform branch (a switch on the source index) into that straight-line
// code. Staging, phi_E^{-1} and the stores are the generic kernels' own text (ring_staged.cuh).
//
// Compiled networks are cached per NetSpec (shape + mask table) for the life of the process and
// never unloaded (a captured graph may still launch them). Compilation runs in the caller's thread
// when it blocks, else in one background thread that takes queued specs in order.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <iterator>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "jit_sources.inc"
#include "pyrit_internal.h"

namespace pyrit {
namespace {

constexpr const char* kKernelName = "ring_staged_net";
constexpr const char* kArch = "-arch=sm_103a";
constexpr size_t kMaxEntries = 1024;  // networks kept per process
constexpr size_t kMaxQueued = 16;     // specs waiting for the background compiler

enum State { kPending, kReady, kFailed };

struct Entry {
  NetSpec spec;
  State state = kPending;
  bool queued = false;  // waiting in the background queue (not yet taken)
  std::vector<char> cubin;
  cudaLibrary_t lib = nullptr;
  bool loaded = false;
  Variant v{};
  int res[5] = {-1, -1, -1, -1, 0};  // registers, stack frame, spill stores, spill loads (bytes), compile ms
};

struct Jit {
  std::mutex mu;
  std::condition_variable cv;
  std::map<std::string, std::unique_ptr<Entry>> cache;
  std::deque<Entry*> queue;
  std::thread worker;
  int busy = 0;  // compilations running
  bool stop = false;
  std::atomic<int> mode{PYRIT_JIT_ASYNC};
  uint64_t compiled = 0, failed = 0, hits = 0, queued_total = 0, loaded = 0, compile_us = 0;
  std::string last_log;

  ~Jit() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
      queue.clear();
    }
    cv.notify_all();
    if (worker.joinable()) worker.join();
  }
};

Jit& jit() {
  static Jit j;
  return j;
}

std::string key_of(const NetSpec& s) { return std::string(reinterpret_cast<const char*>(&s), sizeof(s)); }

void put(std::string& o, const char* fmt, long a = 0, long b = 0, long c = 0, long d = 0, long e = 0, long f = 0) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), fmt, a, b, c, d, e, f);
  o += buf;
}

// One accumulator a case body updates: acc[out][t] ^= the XOR of its columns. Columns 0..W-1 are
// the staged source packets d[q], W..N-1 the parity transform's padding packets dp[q - W], and
// N.. the temporaries share_terms introduces.
struct XorRow {
  int out, t;
  std::vector<int> cols;  // sorted
};
struct XorTemp {
  int id;
  std::vector<int> cols;  // 2 or 3 columns (earlier temporaries allowed)
};

// Common subexpressions of one case body. Accumulating c columns into a row costs ceil(c / 2)
// three-input XORs; a temporary (one XOR of two or three columns) that replaces those columns in
// several rows lowers that sum. The same ring coefficient puts the same pair of source packets,
// d[q] and d[q - s + s'] for two set bits s, s', into many accumulators t (every rotation), and
// the coefficients of one source in different outputs share pairs too. Greedy: take the pair or
// triple with the largest saving (the triple: one step in every row holding it; the pair: one
// step in every row of odd length holding it), minus the temporary's own step, ties to the
// smallest column tuple, until nothing saves. The XOR each row receives is unchanged.
void share_terms(std::vector<XorRow>& rows, int first_id, std::vector<XorTemp>* temps) {
  int next = first_id;
  for (;;) {
    std::map<std::vector<int>, int> gain;  // candidate -> rows where it saves a step
    for (const XorRow& r : rows) {
      const std::vector<int>& c = r.cols;
      const size_t len = c.size();
      for (size_t a = 0; a < len; ++a)
        for (size_t b = a + 1; b < len; ++b) {
          if (len & 1u) ++gain[{c[a], c[b]}];
          for (size_t e = b + 1; e < len; ++e) ++gain[{c[a], c[b], c[e]}];
        }
    }
    const std::vector<int>* best = nullptr;
    int best_gain = 1;  // a temporary costs one step: it must save at least two
    for (const auto& kv : gain)
      if (kv.second > best_gain) {
        best_gain = kv.second;
        best = &kv.first;
      }
    if (!best) return;
    const std::vector<int> take = *best;
    const int id = next++;
    temps->push_back({id, take});
    for (XorRow& r : rows) {
      if (!std::includes(r.cols.begin(), r.cols.end(), take.begin(), take.end())) continue;
      std::vector<int> rest;
      std::set_difference(r.cols.begin(), r.cols.end(), take.begin(), take.end(), std::back_inserter(rest));
      rest.push_back(id);  // ids grow, so the row stays sorted
      r.cols.swap(rest);
    }
  }
}

// Writes rows (after share_terms) as statements inside a `for (x ...)` loop: each temporary just
// before the first row that needs it (recursively), then each row's accumulation.
// Under source pairs (pair), columns kPairCol.. are the second source's packets (d2, dp2) and the
// temporaries start at kPairTemp.
constexpr int kPairCol = 64, kPairTemp = 128;
void emit_rows(std::string& o, const std::vector<XorRow>& rows, const std::vector<XorTemp>& temps, int W, int N,
               bool pair = false) {
  auto name = [&](int c) {
    char buf[32];
    if (c < W)
      std::snprintf(buf, sizeof(buf), "d[%d][x]", c);
    else if (c < N)
      std::snprintf(buf, sizeof(buf), "dp[%d][x]", c - W);
    else if (pair && c >= kPairCol && c < kPairCol + W)
      std::snprintf(buf, sizeof(buf), "d2[%d][x]", c - kPairCol);
    else if (pair && c >= kPairCol + W && c < kPairCol + N)
      std::snprintf(buf, sizeof(buf), "dp2[%d][x]", c - kPairCol - W);
    else
      std::snprintf(buf, sizeof(buf), "e%d", c);
    return std::string(buf);
  };
  std::vector<char> done(temps.size(), 0);
  std::map<int, size_t> index;
  for (size_t i = 0; i < temps.size(); ++i) index[temps[i].id] = i;
  std::function<void(int)> need = [&](int c) {
    auto it = index.find(c);
    if (it == index.end() || done[it->second]) return;
    const XorTemp& tp = temps[it->second];
    for (int x : tp.cols) need(x);
    done[it->second] = 1;
    o += "          const uint32_t " + name(c) + " = ";
    if (tp.cols.size() == 3)
      o += "xor3(" + name(tp.cols[0]) + ", " + name(tp.cols[1]) + ", " + name(tp.cols[2]) + ");\n";
    else
      o += name(tp.cols[0]) + " ^ " + name(tp.cols[1]) + ";\n";
  };
  for (const XorRow& r : rows) {
    for (int c : r.cols) need(c);
    char acc[32];
    std::snprintf(acc, sizeof(acc), "acc[%d][%d][x]", r.out, r.t);
    size_t i = 0;
    for (; i + 1 < r.cols.size(); i += 2)
      o += std::string("          ") + acc + " = xor3(" + acc + ", " + name(r.cols[i]) + ", " + name(r.cols[i + 1]) + ");\n";
    if (i < r.cols.size()) o += std::string("          ") + acc + " ^= " + name(r.cols[i]) + ";\n";
  }
}

// CUDA C++ source of a network (compiled together with the embedded ring_staged.cuh).
std::string net_source(const NetSpec& s) {
  const int N = s.n, W = s.w, S = N - W;
  const int groups = output_groups(s.mg, s.nout, s.nc);
  std::string o;
  o += "#include \"ring_staged.cuh\"\n"
       "namespace pyrit {\n"
       "struct NetMac : ";
  // modes: 0 direct / 1 syndrome under the embedding transform, 2 direct / 3 syndrome under the
  // parity transform (each source enters the ring with its parity packets as packets W..N-1)
  static const char* const kStore[4] = {"DirectStore", "SyndromeStore", "ParityStore", "SyndromePsiStore"};
  const bool syndrome = s.mode == 1 || s.mode == 3, parity = s.mode >= 2;
  o += kStore[s.mode];
  o += " {\n";
  const bool multi = s.ntables > 1;
  if (syndrome) {
    // syndrome decode: only the rows a tile's erasure pattern uses are accumulated
    o += "  __device__ __forceinline__ void tile(const JobDesc* J, int, int) { load_rows(J); }\n";
  } else if (multi) {
    // several tables (the output groups of wide stripes): the tile's job names its table
    o += "  int tbl;\n  __device__ __forceinline__ void tile(const JobDesc* J, int, int) { tbl = J->table; }\n";
  } else {
    o += "  __device__ __forceinline__ void tile(const JobDesc*, int, int) {}\n";
  }
  if (s.g) {
    // A field from another factor g of x^n + 1 (Props. 1-2): phi_E^{-1} is the remainder mod g,
    // out_t = acc_t + the accumulators q >= W whose x^q mod g has coefficient t, written out here.
    o += "  template <int N, int WORDS, int MG>\n"
         "  __device__ __forceinline__ void store(uint32_t (&acc)[MG][N][WORDS], const JobDesc* J, int g,\n"
         "                                        uint32_t col0, uint32_t off, bool valid) {\n"
         "    using V = typename Vec<WORDS>::T;\n"
         "    if (!valid) return;\n"
         "    const uint64_t P = J->P;\n"
         "    const int nout = J->nout;\n"
         "#pragma unroll\n"
         "    for (int i = 0; i < MG; ++i) {\n"
         "      const int o = g * MG + i;\n"
         "      if (o >= nout) continue;\n"
         "      uint8_t* dst = J->out[o] + col0 + off;\n";
    for (int t = 0; t < W; ++t) {
      std::vector<int> qs;
      for (int q = W; q < N; ++q) {
        uint32_t r = 1u << q;  // x^q mod g
        for (int d = q; d >= W; --d)
          if ((r >> d) & 1u) r ^= s.g << (d - W);
        if ((r >> t) & 1u) qs.push_back(q);
      }
      put(o, "      {\n        uint32_t r[WORDS];\n#pragma unroll\n        for (int x = 0; x < WORDS; ++x) {\n"
             "          r[x] = acc[i][%ld][x];\n", t);
      size_t i = 0;
      for (; i + 1 < qs.size(); i += 2)
        put(o, "          r[x] = xor3(r[x], acc[i][%ld][x], acc[i][%ld][x]);\n", qs[i], qs[i + 1]);
      if (i < qs.size()) put(o, "          r[x] ^= acc[i][%ld][x];\n", qs[i]);
      put(o, "        }\n        *reinterpret_cast<V*>(dst + (size_t)%ld * P) = vmake<WORDS>(r);\n      }\n", t);
    }
    o += "    }\n  }\n";
  }
  put(o, "  template <int N, int WORDS, int MG>\n"
         "  __device__ __forceinline__ void apply(uint32_t (&acc)[MG][N][WORDS],\n"
         "                                        const uint32_t (&d)[%ld][WORDS], int j, int g, int) {\n", W);
  // phi_P: parity packet j (ring packet W + j) is the XOR of the source's packets j, j + S, ...
  // (one packet, the XOR of all W, for an all-one polynomial; S = 3 interleaved words for the ESP)
  auto emit_dp = [&](const char* dp, const char* d) {
    std::string t = "    uint32_t " + std::string(dp) + "[%ld][WORDS];\n#pragma unroll\n    for (int x = 0; x < WORDS; ++x) {\n";
    put(o, t.c_str(), S);
    for (int j = 0; j < S; ++j) {
      put(o, ("      " + std::string(dp) + "[%ld][x] = " + d + "[%ld][x];\n").c_str(), j, j);
      int q = j + S;
      for (; q + S < W; q += 2 * S)
        put(o, ("      " + std::string(dp) + "[%ld][x] = xor3(" + dp + "[%ld][x], " + d + "[%ld][x], " + d +
                "[%ld][x]);\n").c_str(), j, j, q, q + S);
      if (q < W) put(o, ("      " + std::string(dp) + "[%ld][x] ^= " + d + "[%ld][x];\n").c_str(), j, q);
    }
    o += "    }\n";
  };
  if (parity) emit_dp("dp", "d");
  // Syndrome networks guard each parity row with one warp-uniform test of the tile's needed rows
  // (a switch on the needed-row set with one block per set measured no faster and compiled
  // several times longer).
  const bool guard = syndrome;
  if (multi)
    put(o, "    switch ((tbl * %ld + g) * %ld + j) {\n", groups, s.nin);
  else
    put(o, "    switch (g * %ld + j) {\n", s.nin);
  // The accumulators source j updates in each output slot of group g of table tb, its packet
  // columns offset by `base` (kPairCol for the second source of a pair).
  auto source_rows = [&](int tb, int g, int j, int base) {
    std::vector<std::vector<XorRow>> slot(s.mg);
    for (int ii = 0; ii < s.mg; ++ii) {
      const int out = g * s.mg + ii;
      if (out >= s.tnout[tb]) break;
      const uint32_t r = s.mask[tb][j][out];
      for (int t = 0; t < N; ++t) {
        // under the parity transform a direct network never builds the top accumulators
        // (phi_P^{-1} drops them)
        if (parity && !syndrome && t >= W) continue;
        // accumulator t receives packet t - s for every set bit s; packets W..N-1 are the zero
        // packets of phi_E (dropped) or the parity packets of phi_P
        XorRow row{ii, t, {}};
        for (int sh = 0; sh < N; ++sh) {
          if (!((r >> sh) & 1u)) continue;
          const int q = (t - sh + N) % N;
          if (q < W || parity) row.cols.push_back(base + q);
        }
        if (row.cols.empty()) continue;
        std::sort(row.cols.begin(), row.cols.end());
        slot[ii].push_back(std::move(row));
      }
    }
    return slot;
  };
  for (int cs = 0; cs < s.ntables * groups; ++cs) {
    const int tb = cs / groups, g = cs % groups;
    for (int j = 0; j < s.nin; ++j) {
      // under source pairs this step codes only an odd job's last source
      if (s.pair && !(s.nin % 2 == 1 && j == s.nin - 1)) continue;
      put(o, "      case %ld: {\n", ((long)tb * groups + g) * s.nin + j);
      std::vector<std::vector<XorRow>> slot = source_rows(tb, g, j, 0);
      if (!guard) {
        // one body for every output of the group: terms shared across outputs are formed once
        std::vector<XorRow> rows;
        for (auto& v : slot) rows.insert(rows.end(), v.begin(), v.end());
        std::vector<XorTemp> temps;
        share_terms(rows, N, &temps);
        o += "#pragma unroll\n        for (int x = 0; x < WORDS; ++x) {\n";
        emit_rows(o, rows, temps, W, N);
        o += "        }\n";
      } else {
        // Syndrome networks: when the tile's pattern needs every parity row (always when m blocks
        // are lost) one body updates all rows, with terms shared across rows as in the encode;
        // otherwise each parity row is guarded by one warp-uniform test of the needed rows, and
        // terms are shared within a row only.
        if (s.allrows) {
          std::vector<XorRow> all;
          for (auto& v : slot) all.insert(all.end(), v.begin(), v.end());
          std::vector<XorTemp> all_temps;
          share_terms(all, N, &all_temps);
          put(o, "        if (need == %ldu) {\n#pragma unroll\n        for (int x = 0; x < WORDS; ++x) {\n",
              (1L << s.mg) - 1);
          emit_rows(o, all, all_temps, W, N);
          o += "        }\n        } else {\n";
        } else {
          o += "        {\n";
        }
        int next_id = N;  // temporaries are numbered across the case's blocks
        for (int ii = 0; ii < s.mg; ++ii) {
          if (slot[ii].empty()) continue;
          std::vector<XorTemp> temps;
          share_terms(slot[ii], next_id, &temps);
          next_id += (int)temps.size();
          put(o, "        if (need & %ldu) {\n#pragma unroll\n        for (int x = 0; x < WORDS; ++x) {\n", 1L << ii);
          emit_rows(o, slot[ii], temps, W, N);
          o += "        }\n        }\n";
        }
        o += "        }\n";
      }
      o += "      } break;\n";
    }
  }
  o += "      default: break;\n    }\n  }\n";
  if (s.pair) {
    // Two sources per step (sources j and j + 1, j even): every accumulator row holds the terms of
    // both, so one three-input XOR can take one term of each, and shared terms may mix them.
    put(o, "  template <int N, int WORDS, int MG>\n"
           "  __device__ __forceinline__ void apply2(uint32_t (&acc)[MG][N][WORDS], const uint32_t (&d)[%ld][WORDS],\n"
           "                                         const uint32_t (&d2)[%ld][WORDS], int j, int g, int) {\n", W, W);
    if (parity) {
      emit_dp("dp", "d");
      emit_dp("dp2", "d2");
    }
    const int npairs = s.nin / 2;
    if (multi)
      put(o, "    switch ((tbl * %ld + g) * %ld + j / 2) {\n", groups, npairs);
    else
      put(o, "    switch (g * %ld + j / 2) {\n", npairs);
    for (int cs = 0; cs < s.ntables * groups; ++cs) {
      const int tb = cs / groups, g = cs % groups;
      for (int pi = 0; pi < npairs; ++pi) {
        put(o, "      case %ld: {\n", ((long)tb * groups + g) * npairs + pi);
        std::vector<std::vector<XorRow>> a = source_rows(tb, g, 2 * pi, 0);
        std::vector<std::vector<XorRow>> b = source_rows(tb, g, 2 * pi + 1, kPairCol);
        std::map<std::pair<int, int>, std::vector<int>> merged;  // (slot, accumulator) -> columns
        for (auto* side : {&a, &b})
          for (auto& v : *side)
            for (XorRow& r : v) {
              std::vector<int>& c = merged[{r.out, r.t}];
              c.insert(c.end(), r.cols.begin(), r.cols.end());
            }
        std::vector<XorRow> rows;
        for (auto& kv : merged) {
          XorRow r{kv.first.first, kv.first.second, kv.second};
          std::sort(r.cols.begin(), r.cols.end());
          rows.push_back(std::move(r));
        }
        std::vector<XorTemp> temps;
        share_terms(rows, kPairTemp, &temps);
        o += "#pragma unroll\n        for (int x = 0; x < WORDS; ++x) {\n";
        emit_rows(o, rows, temps, W, N, true);
        o += "        }\n      } break;\n";
      }
    }
    o += "      default: break;\n    }\n  }\n";
  }
  o += "};\n}  // namespace pyrit\n\n";
  put(o, "extern \"C\" __global__ void __launch_bounds__(%ld, %ld)\n", (s.nc + 1) * 32, s.minb);
  o += kKernelName;
  o += "(const __grid_constant__ pyrit::CodeArgs a) {\n";
  put(o, "  pyrit::ring_staged_body<%ld, %ld, %ld, %ld, pyrit::NetMac, %ld, ", N, s.words, s.mg, s.nc, W);
  o += s.track ? "true, " : "false, ";
  o += s.pair ? "true>(a);\n}\n" : "false>(a);\n}\n";
  return o;
}

// The first integer after `key` in the assembler's resource report, or -1.
int report_value(const std::string& log, const char* key, bool before) {
  const size_t at = log.find(key);
  if (at == std::string::npos) return -1;
  if (before) {  // "<value> <key>"
    size_t e = at;
    while (e > 0 && log[e - 1] == ' ') --e;
    size_t b = e;
    while (b > 0 && log[b - 1] >= '0' && log[b - 1] <= '9') --b;
    return b < e ? std::atoi(log.substr(b, e - b).c_str()) : -1;
  }
  size_t b = at + std::strlen(key);
  while (b < log.size() && log[b] == ' ') ++b;
  return b < log.size() && log[b] >= '0' && log[b] <= '9' ? std::atoi(log.c_str() + b) : -1;
}

// Compiles one spec into a cubin. Returns PYRIT_OK or PYRIT_E_JIT (log filled). The assembler's
// resource report (registers, stack frame, spills) is parsed into res[0..3].
int compile_spec(const NetSpec& s, std::vector<char>* cubin, std::string* log, uint64_t* us, int* res) {
  const auto t0 = std::chrono::steady_clock::now();
  const std::string src = net_source(s);
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "ring_staged_net.cu", kJitHeaderCount, kJitHeaders, kJitHeaderNames) !=
      NVRTC_SUCCESS) {
    *log = "nvrtcCreateProgram failed";
    return PYRIT_E_JIT;
  }
  const char* opts[] = {kArch, "-std=c++17", "-lineinfo", "--ptxas-options=-v"};
  const nvrtcResult r = nvrtcCompileProgram(prog, 4, opts);
  size_t ls = 0;
  nvrtcGetProgramLogSize(prog, &ls);
  log->assign(ls, '\0');
  if (ls) nvrtcGetProgramLog(prog, &(*log)[0]);
  res[0] = report_value(*log, "Used", false);
  res[1] = report_value(*log, "bytes stack frame", true);
  res[2] = report_value(*log, "bytes spill stores", true);
  res[3] = report_value(*log, "bytes spill loads", true);
  int rc = PYRIT_E_JIT;
  size_t cs = 0;
  if (r == NVRTC_SUCCESS && nvrtcGetCUBINSize(prog, &cs) == NVRTC_SUCCESS && cs > 0) {
    cubin->resize(cs);
    if (nvrtcGetCUBIN(prog, cubin->data()) == NVRTC_SUCCESS) rc = PYRIT_OK;
  }
  if (r != NVRTC_SUCCESS) *log = std::string(nvrtcGetErrorString(r)) + "\n" + *log;
  nvrtcDestroyProgram(&prog);
  *us = (uint64_t)std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

// Records a finished compilation (lock held).
void finish(Jit& J, Entry* e, int rc, std::vector<char>& cubin, const std::string& log, uint64_t us) {
  J.compile_us += us;
  if (rc == PYRIT_OK) {
    e->cubin.swap(cubin);
    e->state = kReady;
    ++J.compiled;
  } else {
    e->state = kFailed;
    J.last_log = log;
    ++J.failed;
  }
}

// Compiles `e` in this thread (lock held on entry and exit, released meanwhile).
void compile_here(Jit& J, Entry* e, std::unique_lock<std::mutex>& lk) {
  ++J.busy;
  lk.unlock();
  std::vector<char> cubin;
  std::string log;
  uint64_t us = 0;
  int res[4];
  const int rc = compile_spec(e->spec, &cubin, &log, &us, res);
  lk.lock();
  for (int i = 0; i < 4; ++i) e->res[i] = res[i];
  e->res[4] = (int)(us / 1000);
  finish(J, e, rc, cubin, log, us);
  --J.busy;
  J.cv.notify_all();
}

void worker_main(Jit* J) {
  std::unique_lock<std::mutex> lk(J->mu);
  while (true) {
    J->cv.wait(lk, [&] { return J->stop || !J->queue.empty(); });
    if (J->stop) return;
    Entry* e = J->queue.front();
    J->queue.pop_front();
    e->queued = false;
    compile_here(*J, e, lk);
  }
}

// The cache entry of `s` after the policy's step: compiled (or failed) when `block`, else possibly
// still pending. nullptr when the cache is full or the queue has no room.
Entry* obtain(Jit& J, const NetSpec& s, bool block, std::unique_lock<std::mutex>& lk) {
  const std::string key = key_of(s);
  auto it = J.cache.find(key);
  Entry* e = it == J.cache.end() ? nullptr : it->second.get();
  if (!e) {
    if (J.cache.size() >= kMaxEntries || (!block && J.queue.size() >= kMaxQueued)) return nullptr;
    std::unique_ptr<Entry> up(new Entry);
    up->spec = s;
    e = up.get();
    J.cache.emplace(key, std::move(up));
    if (!block) {
      e->queued = true;
      J.queue.push_back(e);
      ++J.queued_total;
      if (!J.worker.joinable()) J.worker = std::thread(worker_main, &J);
      J.cv.notify_all();
      return e;
    }
    compile_here(J, e, lk);
    return e;
  }
  if (e->state == kPending && block) {
    if (e->queued) {  // not started: take it out of the queue and compile it here
      J.queue.erase(std::find(J.queue.begin(), J.queue.end(), e));
      e->queued = false;
      compile_here(J, e, lk);
    } else {
      J.cv.wait(lk, [&] { return e->state != kPending; });
    }
  }
  return e;
}

struct Shape4 {
  int words, half, minb, nc;  // half: mg = ceil(nout / 2) (two output groups) instead of nout
};

// Registers a thread may use at (nc + 1) warps and minb CTAs per SM: the SM's 65536 registers
// are four schedulers' 16384 each, and a scheduler holds ceil(warps / 4) of the block's warps.
int reg_cap(int nc, int minb) {
  const int per_sched = ((nc + 1) * minb + 3) / 4;
  const int r = (16384 / (32 * per_sched)) & ~7;
  return r > 255 ? 255 : r;
}

}  // namespace

int jit_mode() { return jit().mode.load(); }

int shapes_for(int n, int nout, bool syndrome, NetSpec* out, int cap);

int net_candidate_shapes(int n, int nout, NetSpec* out, int cap) {
  return shapes_for(n, nout, false, out, cap);
}

int shapes_for(int n, int nout, bool syndrome, NetSpec* out, int cap) {
  // Per ring size, kind of network and output count, in measured order (GB300 sweeps of every
  // (words, consumer warps) pair on 2-3 GiB batches of GF(2^10) k=10 m=4 and k=4 m=8, GF(2^12)
  // k=16 m=4 and k=2 m=6, GF(16) k=8 m=4, GF(4) k=1 m=2): the first shape whose accumulators fit
  // the register budget is the default, the rest are the tuner's other candidates. Few outputs
  // favour two words per thread; eight outputs fill the registers at one word. For GF(2^12)
  // k=16 m=4 (re-measured with the current networks) the direct network runs best at two words
  // and 11 warps (0.97 of HBM against 0.83 at one word and 16 warps; one 1 MiB stripe in 51 us
  // instead of 57), and the syndrome network defaults to one word and 19 warps (96 registers, 20
  // warps per SM): untuned, the 4-erasure decode runs at 0.65 against 0.61 at 16 warps, and a
  // served 1 MiB decode finishes in 73 us instead of 89 (two words and 11 warps, 0.68, needs a
  // 4-stage ring, which the tuner finds).
  static const Shape4 n11_d[] = {{2, 0, 1, 11}, {2, 0, 1, 10}, {2, 0, 1, 12}, {2, 0, 1, 15},
                                 {1, 0, 1, 15}, {1, 0, 1, 16}, {1, 0, 1, 11}, {1, 1, 1, 16}};
  static const Shape4 n11_dw[] = {{1, 0, 1, 15}, {1, 0, 1, 11}, {1, 0, 1, 12}, {1, 0, 1, 14},
                                  {2, 0, 1, 11}, {1, 0, 1, 8}, {1, 1, 1, 16}, {2, 1, 1, 11}};
  static const Shape4 n11_s[] = {{2, 0, 1, 15}, {2, 0, 1, 14}, {2, 0, 1, 12}, {2, 0, 1, 11},
                                 {2, 0, 1, 10}, {1, 0, 1, 16}, {1, 0, 1, 15}, {1, 0, 1, 8}};
  static const Shape4 n11_sw[] = {{1, 0, 1, 15}, {1, 0, 1, 14}, {1, 0, 1, 12}, {1, 0, 1, 11},
                                  {1, 0, 1, 8}, {1, 0, 1, 16}, {2, 0, 1, 11}, {2, 0, 1, 8}};
  static const Shape4 n13_d[] = {{2, 0, 1, 11}, {2, 0, 1, 10}, {1, 0, 1, 16}, {1, 0, 1, 19},
                                 {1, 0, 1, 15}, {1, 0, 1, 14}, {2, 0, 1, 8}, {1, 1, 1, 16}};
  static const Shape4 n13_dw[] = {{1, 0, 1, 11}, {1, 0, 1, 12}, {1, 0, 1, 14}, {1, 0, 1, 15},
                                  {1, 0, 1, 8}, {1, 1, 1, 16}, {1, 0, 1, 16}, {2, 1, 1, 11}};
  static const Shape4 n13_s[] = {{1, 0, 1, 19}, {2, 0, 1, 11}, {1, 0, 1, 16}, {1, 0, 1, 15},
                                 {1, 0, 1, 14}, {2, 0, 1, 8}, {1, 0, 1, 12}, {1, 0, 1, 11}};
  static const Shape4 n13_sw[] = {{1, 0, 1, 14}, {1, 0, 1, 15}, {1, 0, 1, 12}, {1, 0, 1, 11},
                                  {1, 0, 1, 16}, {1, 0, 1, 8}, {2, 0, 1, 8}, {2, 0, 1, 11}};
  static const Shape4 small_d[] = {{4, 0, 1, 12}, {2, 0, 1, 24}, {4, 0, 1, 8}, {4, 0, 1, 15},
                                   {2, 0, 1, 11}, {2, 0, 1, 16}, {4, 0, 1, 11}, {2, 0, 1, 8}};
  static const Shape4 small_s[] = {{2, 0, 1, 11}, {4, 0, 1, 8}, {4, 0, 1, 12}, {2, 0, 1, 24},
                                   {4, 0, 1, 15}, {2, 0, 1, 8}, {4, 0, 1, 11}, {2, 0, 1, 16}};
  static const Shape4 n9_d[] = {{2, 0, 1, 11}, {2, 0, 1, 12}, {4, 0, 1, 8}, {2, 0, 1, 15},
                                {1, 0, 1, 16}, {4, 0, 1, 11}, {2, 1, 1, 11}, {1, 0, 1, 12}};
  static const Shape4 n9_s[] = {{2, 0, 1, 15}, {2, 0, 1, 12}, {2, 0, 1, 11}, {4, 0, 1, 8},
                                {1, 0, 1, 16}, {2, 0, 1, 8}, {1, 0, 1, 15}, {4, 0, 1, 11}};
  // GF(2^6) with 5-8 outputs per job (the paper's (60, 40) and (60, 20) codes): one word per thread
  // and 15 warps measured best, two words spill at 8 outputs
  static const Shape4 n9_w[] = {{1, 0, 1, 15}, {1, 0, 1, 11}, {1, 0, 1, 12}, {1, 0, 1, 16},
                                {2, 0, 1, 11}, {2, 0, 1, 15}, {1, 0, 1, 8}, {2, 0, 1, 8}};
  const bool wide = nout > 4;
  const Shape4* list = n == 9    ? (wide ? n9_w : (syndrome ? n9_s : n9_d))
                       : n == 11 ? (syndrome ? (wide ? n11_sw : n11_s) : (wide ? n11_dw : n11_d))
                       : n == 13 ? (syndrome ? (wide ? n13_sw : n13_s) : (wide ? n13_dw : n13_d))
                                 : (syndrome ? small_s : small_d);
  int count = 0;
  for (int i = 0; i < 8 && count < cap; ++i) {
    const Shape4& c = list[i];
    const int mg = c.half ? (nout + 1) / 2 : nout;
    if (mg < 1 || (c.half && (nout < 2 || syndrome))) continue;  // syndrome decode needs every row
    const int groups = output_groups(mg, nout, c.nc);
    if (c.nc % groups != 0 || groups * mg < nout) continue;
    // accumulators (+ an output under construction for syndrome decoding), one staged source and
    // addressing and loop state against the register budget; the estimate runs about 20 above
    // what the compiler allocates without spilling (measured), hence the allowance
    // (direct networks of more than four outputs hold a second staged source; the estimate leaves
    // it out, since under the parity transform their top accumulators are never built, and the
    // tuner times every candidate)
    if ((mg + (syndrome ? 1 : 0)) * n * c.words + (n - 1) * c.words + 16 > reg_cap(c.nc, c.minb) + 20) continue;
    NetSpec s;
    std::memset(&s, 0, sizeof(s));
    s.n = n;
    s.nout = nout;
    s.words = c.words;
    s.mg = mg;
    s.minb = c.minb;
    s.nc = c.nc;
    out[count++] = s;
  }
  return count;
}

NetSpec net_spec_tables(int n, const JobDesc* const* tables, int ntables, int words, int mg, int minb, int nc,
                        int transform, uint32_t g) {
  NetSpec s;
  std::memset(&s, 0, sizeof(s));
  int nout = 0;
  for (int t = 0; t < ntables; ++t) nout = std::max(nout, (int)tables[t]->nout);
  NetSpec def[1];
  if (net_candidate_shapes(n, nout, def, 1) == 1) s = def[0];
  s.n = n;
  s.nin = tables[0]->nin;
  s.nout = nout;
  if (words) s.words = words;
  if (mg) s.mg = mg;
  if (minb) s.minb = minb;
  if (nc) s.nc = nc;
  if (!s.words) s.words = 1;
  if (!s.mg) s.mg = nout;
  if (!s.minb) s.minb = 1;
  if (!s.nc) s.nc = 16;
  s.mode = transform == PYRIT_TRANSFORM_PARITY ? 2 : 0;
  s.g = g;
  s.w = g ? 31 - __builtin_clz(g) : field_degree(n);
  s.ntables = ntables < kMaxJobs ? ntables : kMaxJobs;
  for (int t = 0; t < s.ntables; ++t) {
    const JobDesc& job = *tables[t];
    s.tnout[t] = job.nout;
    for (int j = 0; j < job.nin && j < kMaxIn; ++j)
      for (int o = 0; o < job.nout && o < kMaxOut; ++o) s.mask[t][j][o] = job.mask[j][o];
  }
  if (ntables > kMaxJobs) s.ntables = 0;  // rejected by spec_valid
  // Jobs of more than four outputs (the paper's wide GF(2^6) codes) are bound by their XOR work:
  // two sources per step let one three-input XOR take a term of each (measured on GB300: the
  // (60,40) embedding 0.252-0.265 -> 0.265-0.290 of HBM, the (60,20) parity transform 0.293-0.342
  // -> 0.299-0.371, bit-exact). Jobs of up to four outputs keep one source per step: their
  // encodes run at HBM speed already, and the second source's registers cost the GF(2^12) k=16
  // m=4 encode its 8-byte shape (0.98 -> 0.84).
  s.pair = s.nout > 4 ? 1 : 0;
  return s;
}

NetSpec net_spec(int n, const JobDesc& job, int words, int mg, int minb, int nc, int transform, uint32_t g) {
  const JobDesc* t = &job;
  return net_spec_tables(n, &t, 1, words, mg, minb, nc, transform, g);
}

NetSpec net_spec_syndrome(const pyrit_plan_s* p, int words, int minb, int nc, int allrows) {
  NetSpec s;
  std::memset(&s, 0, sizeof(s));
  NetSpec def[1];
  if (shapes_for(p->n, p->m, true, def, 1) == 1) s = def[0];
  s.n = p->n;
  s.mode = p->transform == PYRIT_TRANSFORM_PARITY ? 3 : 1;
  s.allrows = allrows ? 1 : 0;
  s.nin = p->k + p->m;
  s.nout = p->m;
  s.mg = p->m;
  s.ntables = 1;
  s.tnout[0] = p->m;
  s.w = p->w;
  s.g = plan_net_g(p);  // rejected by spec_valid unless native: the syndrome store folds natively
  if (words) s.words = words;
  if (minb) s.minb = minb;
  if (nc) s.nc = nc;
  if (!s.words) s.words = 1;
  if (!s.minb) s.minb = 1;
  if (!s.nc) s.nc = 8;
  if (s.nin > kMaxIn || p->m > kMaxOut) return s;  // rejected by spec_valid
  // H = [C | I_m]: data column j carries the parity rows' coefficients, parity column k + r only
  // its own row with coefficient 1 (mask x^0)
  for (int r = 0; r < p->m; ++r) {
    for (int j = 0; j < p->k; ++j) s.mask[0][j][r] = p->enc_mask[r * p->k + j];
    s.mask[0][p->k + r][r] = 1;
  }
  return s;
}

int net_syndrome_shapes(const pyrit_plan_s* p, NetSpec* out, int cap, int allrows) {
  NetSpec shapes[8];
  const int c = shapes_for(p->n, p->m, true, shapes, cap < 8 ? cap : 8);
  for (int i = 0; i < c; ++i) out[i] = net_spec_syndrome(p, shapes[i].words, shapes[i].minb, shapes[i].nc, allrows);
  return c;
}

static bool spec_valid(const NetSpec& s) {
  const bool words_ok = s.words == 1 || s.words == 2 || s.words == 4;
  const bool nc_ok = s.nc >= 1 && s.nc <= 31;
  if (s.mode < 0 || s.mode > 3 || (s.track != 0 && s.track != 1) || (s.allrows != 0 && s.allrows != 1)) return false;
  if (s.allrows && !(s.mode == 1 || s.mode == 3)) return false;
  if ((s.pair != 0 && s.pair != 1) || (s.pair && !(s.mode == 0 || s.mode == 2))) return false;
  if ((s.mode == 1 || s.mode == 3) && !(s.mg == s.nout && s.nout <= kSyndromeBaseRow && s.ntables == 1)) return false;
  if (s.ntables < 1 || s.ntables > kMaxJobs) return false;
  // a native field of its ring, or (direct embedding networks only) a factor g of x^n + 1 of degree w
  if (s.g == 0) {
    if (!(s.n == 3 || s.n == 5 || s.n == 9 || s.n == 11 || s.n == 13) || s.w != field_degree(s.n)) return false;
  } else {
    if (s.mode != 0 || (s.n & 1) == 0 || s.n < 3 || s.n > 15 || s.w < 2 || s.w >= s.n ||
        s.w != 31 - __builtin_clz(s.g))
      return false;
    uint32_t r = (1u << s.n) | 1u;  // x^n + 1 mod g must vanish
    for (int d = s.n; d >= s.w; --d)
      if ((r >> d) & 1u) r ^= s.g << (d - s.w);
    if (r != 0) return false;
  }
  for (int t = 0; t < s.ntables; ++t)
    if (s.tnout[t] < 1 || s.tnout[t] > s.nout) return false;
  return s.nin >= 1 && s.nin <= kMaxIn && s.nout >= 1 &&
         s.nout <= kMaxOut && words_ok && s.mg >= 1 && s.mg <= kMaxOut && s.minb >= 1 && s.minb <= 4 && nc_ok &&
         output_groups(s.mg, s.nout, s.nc) * s.mg >= s.nout && s.nc % output_groups(s.mg, s.nout, s.nc) == 0;
}

int net_compile(const NetSpec& s) {
  if (!spec_valid(s)) return PYRIT_E_INVALID_ARG;
  Jit& J = jit();
  std::unique_lock<std::mutex> lk(J.mu);
  Entry* e = obtain(J, s, true, lk);
  return e && e->state == kReady ? PYRIT_OK : PYRIT_E_JIT;
}

int net_spill_bytes(const NetSpec& s) {
  Jit& J = jit();
  std::lock_guard<std::mutex> lk(J.mu);
  auto it = J.cache.find(key_of(s));
  return it == J.cache.end() || it->second->state != kReady ? -1 : it->second->res[2];
}

const Variant* net_variant(const NetSpec& s, bool block) {
  Jit& J = jit();
  const int mode = J.mode.load();
  if (mode == PYRIT_JIT_OFF || !spec_valid(s)) return nullptr;
  if (mode == PYRIT_JIT_SYNC) block = true;
  std::unique_lock<std::mutex> lk(J.mu);
  Entry* e = obtain(J, s, block, lk);
  if (!e || e->state != kReady) return nullptr;
  if (!e->loaded) {
    // cudaLibraryLoadData makes the module available on every device of the process.
    cudaKernel_t k = nullptr;
    if (cudaLibraryLoadData(&e->lib, e->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
        cudaLibraryGetKernel(&k, e->lib, kKernelName) != cudaSuccess) {
      cudaGetLastError();  // load failures are not sticky; clear them for the caller
      e->state = kFailed;
      J.last_log = "cudaLibraryLoadData / cudaLibraryGetKernel failed";
      ++J.failed;
      return nullptr;
    }
    e->v = Variant{s.n,    s.words, s.mg,   s.minb, PYRIT_DISPATCH_NETWORK, s.nc, reinterpret_cast<const void*>(k),
                   s.mode, s.nout,  s.w,   s.track};
    e->loaded = true;
    ++J.loaded;
  }
  ++J.hits;
  return &e->v;
}

}  // namespace pyrit

using namespace pyrit;

extern "C" {

int pyrit_jit_mode(int mode) {
  Jit& J = jit();
  if (mode < 0) return J.mode.load();
  if (mode > PYRIT_JIT_ASYNC) return PYRIT_E_INVALID_ARG;
  return J.mode.exchange(mode);
}

int pyrit_jit_wait(int timeout_ms) {
  Jit& J = jit();
  std::unique_lock<std::mutex> lk(J.mu);
  const bool done = J.cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                  [&] { return J.queue.empty() && J.busy == 0; });
  return done ? PYRIT_OK : PYRIT_E_TIMEOUT;
}

int pyrit_jit_quiesce(int timeout_ms) {
  Jit& J = jit();
  std::unique_lock<std::mutex> lk(J.mu);
  for (Entry* e : J.queue) J.cache.erase(key_of(e->spec));  // never started: forget them
  J.queue.clear();
  const bool done = J.cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                  [&] { return J.busy == 0; });
  return done ? PYRIT_OK : PYRIT_E_TIMEOUT;
}

int pyrit_jit_stats(uint64_t* stats_out) {
  if (!stats_out) return PYRIT_E_INVALID_ARG;
  Jit& J = jit();
  std::lock_guard<std::mutex> lk(J.mu);
  stats_out[0] = J.cache.size();
  stats_out[1] = J.compiled;
  stats_out[2] = J.failed;
  stats_out[3] = J.queue.size() + (uint64_t)J.busy;
  stats_out[4] = J.hits;
  stats_out[5] = J.loaded;
  stats_out[6] = J.compile_us;
  stats_out[7] = J.queued_total;
  return PYRIT_OK;
}

int pyrit_jit_log(char* buf, int cap) {
  Jit& J = jit();
  std::lock_guard<std::mutex> lk(J.mu);
  const int len = (int)J.last_log.size();
  if (buf && cap > 0) {
    const int c = std::min(len, cap - 1);
    std::memcpy(buf, J.last_log.data(), (size_t)c);
    buf[c] = '\0';
  }
  return len;
}

}  // extern "C"

namespace {

// The networks a plan's operation uses, one per job (a stripe with more than kMaxOut parity or
// erased blocks is several jobs): fills s[0..count) and returns count, 0 when there is nothing to
// code (no parity rows, no erasure), or an error status.
int plan_network_specs(pyrit_plan_s* plan, int op, uint64_t erasures, const pyrit_tile_t* tile,
                       NetSpec* s /* [kMaxJobs] */) {
  if (!plan) return PYRIT_E_INVALID_ARG;
  std::vector<void*> none((size_t)(plan->k + plan->m), nullptr);  // only the masks are used
  JobDesc jobs[kMaxJobs];
  int nj = 0;
  if (op == PYRIT_OP_ENCODE) {
    nj = make_encode_jobs(plan, none.data(), none.data() + plan->k, 16, jobs);
  } else if (op == PYRIT_OP_DECODE_ANY) {
    if (plan->m == 0) return 0;
    if (plan->k + plan->m > kMaxIn || plan->m > kMaxOut) return PYRIT_E_INVALID_ARG;
    s[0] = tile ? net_spec_syndrome(plan, tile->words, tile->minb, tile->nc) : net_spec_syndrome(plan, 0, 0, 0);
    return 1;
  } else if (op == PYRIT_OP_DECODE) {
    DecodeEntry e;
    const int rc = plan_decode_entry(plan, erasures, &e);
    if (rc != PYRIT_OK) return rc;
    nj = make_decode_jobs(plan, e, none.data(), 16, jobs);
  } else {
    return PYRIT_E_INVALID_ARG;
  }
  for (int i = 0; i < nj; ++i)
    s[i] = tile ? net_spec(plan->n, jobs[i], tile->words, tile->mg, tile->minb, tile->nc, plan->transform,
                           plan_net_g(plan))
                : net_spec(plan->n, jobs[i], 0, 0, 0, 0, plan->transform, plan_net_g(plan));
  return nj;
}

}  // namespace

extern "C" {

int pyrit_plan_specialise(pyrit_plan_t plan, int op, uint64_t erasures, const pyrit_tile_t* tile) {
  NetSpec s[3 * kMaxJobs];
  const int ns = plan_network_specs(plan, op, erasures, tile, s);
  if (ns < 0) return ns;
  // each network in the forms later calls look for, compiled side by side: the one batches and
  // single calls launch, the one the server launches (it stamps each request's completion), and for
  // a syndrome-decode network also the form without the all-rows body (batches whose stripes mostly
  // need fewer rows)
  int total = ns;
  for (int i = 0; i < ns; ++i) {
    s[total] = s[i];
    s[total++].track = 1;
  }
  for (int i = 0; i < ns && total < 3 * kMaxJobs; ++i)
    if (s[i].allrows) {
      s[total] = s[i];
      s[total++].allrows = 0;
    }
  int rcs[3 * kMaxJobs];
  std::vector<std::thread> th;
  for (int i = 0; i < total; ++i) th.emplace_back([&s, &rcs, i] { rcs[i] = net_compile(s[i]); });
  for (auto& t : th) t.join();
  for (int i = 0; i < total; ++i)
    if (rcs[i] != PYRIT_OK) return rcs[i];
  return PYRIT_OK;
}

int pyrit_plan_network_source(pyrit_plan_t plan, int op, uint64_t erasures, const pyrit_tile_t* tile, char* buf,
                              int cap) {
  NetSpec specs[kMaxJobs];
  const int rc = plan_network_specs(plan, op, erasures, tile, specs);
  if (rc == 0) return PYRIT_E_INVALID_ARG;
  if (rc < 0) return rc;
  if (!spec_valid(specs[0])) return PYRIT_E_INVALID_ARG;
  const std::string src = net_source(specs[0]);
  if (buf && cap > 0) {
    const int c = std::min((int)src.size(), cap - 1);
    std::memcpy(buf, src.data(), (size_t)c);
    buf[c] = '\0';
  }
  return (int)src.size();
}

int pyrit_plan_network_info(pyrit_plan_t plan, int op, uint64_t erasures, const pyrit_tile_t* tile, int* info_out) {
  if (!info_out) return PYRIT_E_INVALID_ARG;
  NetSpec specs[kMaxJobs];
  int rc = plan_network_specs(plan, op, erasures, tile, specs);
  if (rc == 0) return PYRIT_E_INVALID_ARG;  // nothing to code: no network
  if (rc < 0) return rc;
  const NetSpec& s = specs[0];  // the first job's network (all jobs of a stripe share its shape)
  rc = net_compile(s);
  if (rc != PYRIT_OK) return rc;
  Jit& J = jit();
  std::lock_guard<std::mutex> lk(J.mu);
  auto it = J.cache.find(key_of(s));
  if (it == J.cache.end()) return PYRIT_E_JIT;
  const Entry& e = *it->second;
  const int shape[4] = {s.words, s.mg, s.nc, s.mode};
  std::memcpy(info_out, e.res, sizeof(e.res));
  std::memcpy(info_out + 5, shape, sizeof(shape));
  return PYRIT_OK;
}

int pyrit_jit_source(int n, int nin, int nout, const uint16_t* masks, const pyrit_tile_t* tile, int transform,
                     char* buf, int cap) {
  if (!masks || nin < 1 || nin > kMaxIn || nout < 1 || nout > kMaxOut) return PYRIT_E_INVALID_ARG;
  if (transform != PYRIT_TRANSFORM_EMBEDDING && transform != PYRIT_TRANSFORM_PARITY) return PYRIT_E_INVALID_ARG;
  JobDesc job;
  std::memset(&job, 0, sizeof(job));
  job.nin = nin;
  job.nout = nout;
  for (int o = 0; o < nout; ++o)
    for (int j = 0; j < nin; ++j) job.mask[j][o] = masks[o * nin + j];
  const NetSpec s = tile ? net_spec(n, job, tile->words, tile->mg, tile->minb, tile->nc, transform)
                         : net_spec(n, job, 0, 0, 0, 0, transform);
  if (!spec_valid(s)) return PYRIT_E_INVALID_ARG;
  const std::string src = net_source(s);
  if (buf && cap > 0) {
    const int c = std::min((int)src.size(), cap - 1);
    std::memcpy(buf, src.data(), (size_t)c);
    buf[c] = '\0';
  }
  return (int)src.size();
}

}  // extern "C"
