// The autotuner's table: the fastest measured tile shape per launch-group key, process-wide,
// with a plain-text JSON save/load so a tuned table can be reused across runs.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "pyrit_internal.h"

namespace pyrit {
namespace {
std::mutex g_mu;
std::map<TuneKey, TuneVal>& table() {
  static std::map<TuneKey, TuneVal> t;
  return t;
}
}  // namespace

bool tune_lookup(const TuneKey& k, TuneVal* v) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = table().find(k);
  if (it == table().end()) return false;
  *v = it->second;
  return true;
}

void tune_record(const TuneKey& k, const TuneVal& v) {
  std::lock_guard<std::mutex> lk(g_mu);
  table()[k] = v;
}

}  // namespace pyrit

using namespace pyrit;

extern "C" {

int pyrit_tune_save(const char* path) {
  if (!path) return PYRIT_E_INVALID_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) return PYRIT_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  std::fprintf(f, "[\n");
  size_t i = 0;
  for (const auto& kv : table()) {
    const TuneKey& k = kv.first;
    const TuneVal& v = kv.second;
    std::fprintf(f,
                 "  {\"n\": %d, \"shared\": %d, \"nout\": %d, \"plog2\": %d, \"words\": %d, \"mg\": %d, \"minb\": %d, "
                 "\"nc\": %d, \"dispatch\": %d, \"stages\": %d, \"ms\": %.6f}%s\n",
                 k.n, k.shared, k.nout, k.plog2, v.words, v.mg, v.minb, v.nc, v.dispatch, v.stages, v.ms,
                 ++i < table().size() ? "," : "");
  }
  std::fprintf(f, "]\n");
  std::fclose(f);
  return PYRIT_OK;
}

int pyrit_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  const int n = (int)table().size();
  table().clear();
  return n;
}

int pyrit_tune_load(const char* path) {
  if (!path) return PYRIT_E_INVALID_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return PYRIT_E_INVALID_ARG;
  char line[512];
  int n = 0;
  while (std::fgets(line, sizeof(line), f)) {
    TuneKey k;
    TuneVal v;
    if (std::sscanf(line,
                    " {\"n\": %d, \"shared\": %d, \"nout\": %d, \"plog2\": %d, \"words\": %d, \"mg\": %d, \"minb\": %d, "
                    "\"nc\": %d, \"dispatch\": %d, \"stages\": %d, \"ms\": %f}",
                    &k.n, &k.shared, &k.nout, &k.plog2, &v.words, &v.mg, &v.minb, &v.nc, &v.dispatch, &v.stages,
                    &v.ms) == 11) {
      tune_record(k, v);
      ++n;
    }
  }
  std::fclose(f);
  return n;
}

}  // extern "C"
