// Host planner: field checks, the sparse transform phi_S, generator validation and the decoding
// matrices (paper Secs. 2.2, 2.3, 3 and 4.3). Host memory only; no CUDA call.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>

#include "pyrit_internal.h"

namespace pyrit {

namespace {

// Sec. 2.3: the AOP of degree r is irreducible iff r+1 is prime and 2 generates the
// multiplicative group of F_{r+1} (read from the text's "w generates F*_{w+1}", which its own
// GF(16) example contradicts literally).
bool aop_irreducible(int r) {
  const int p = r + 1;
  if (r < 2) return false;  // the criteria below need r + 1 an odd prime (x^s + 1 is reducible)
  for (int d = 2; d * d <= p; ++d)
    if (p % d == 0) return false;
  int order = 1;
  for (int v = 2 % p; v != 1; v = (v * 2) % p) ++order;
  return order == r;
}

uint64_t pow_mod(uint64_t b, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  b %= m;
  while (e) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return r;
}

// Sec. 2.4 (citing Itoh and Tsujii): the s-ESP p(x^s) of degree s r, p the AOP of degree r, is
// irreducible iff p is and s = (r+1)^(t-1) for some t >= 2 with 2^(r (r+1)^(t-2)) != 1 mod
// (r+1)^t. s = 1 is the AOP itself.
bool esp_irreducible(int s, int r) {
  if (!aop_irreducible(r)) return false;
  if (s == 1) return true;
  uint64_t pw = (uint64_t)r + 1;  // (r+1)^(t-1), t = 2
  for (int t = 2; pw <= (uint64_t)s; ++t, pw *= (uint64_t)(r + 1))
    if (pw == (uint64_t)s) return pow_mod(2, (uint64_t)r * (pw / (uint64_t)(r + 1)), pw * (uint64_t)(r + 1)) != 1;
  return false;
}

}  // namespace

// The native fields, which the generic kernels are built for: the s-ESP of degree w = s r with
// n = s (r + 1) (s = 1: the AOP, n = w + 1), irreducible by the paper's criteria, on the ring
// sizes 3, 5, 11, 13 (AOPs) and 9 (x^6 + x^3 + 1).
bool field_native(int w, int n) {
  if (w < 2 || w > 15 || n <= w) return false;
  const int s = n - w;
  if (w % s != 0 || !esp_irreducible(s, w / s)) return false;
  return field_degree(n) == w && (n == 3 || n == 5 || n == 9 || n == 11 || n == 13);
}

namespace {

int poly_degree(uint32_t p) { return 31 - __builtin_clz(p); }

// Remainder of a by p over F2.
uint32_t poly_rem(uint32_t a, uint32_t p) {
  const int dp = poly_degree(p);
  for (int d = 31; d >= dp; --d)
    if ((a >> d) & 1u) a ^= p << (d - dp);
  return a;
}

bool poly_irreducible(uint32_t p) {
  const int w = poly_degree(p);
  for (int d = 1; d <= w / 2; ++d)
    for (uint32_t f = 1u << d; f < (2u << d); ++f)
      if (poly_rem(p, f) == 0) return false;
  return true;
}

}  // namespace

// The modulus of GF(2^w) on R_{2,n}: for a native field its AOP or ESP; otherwise (Props. 1-2:
// any irreducible factor p of x^n + 1, n odd, makes mod p a homomorphism R_{2,n} -> F2[x]/(p))
// the smallest irreducible factor of degree w of x^n + 1, for odd n <= 15 (masks are 16-bit).
// 0: no such field.
uint32_t field_modulus(int w, int n) {
  if (field_native(w, n)) return n == 9 ? 0x49u /* 1 + x^3 + x^6 */ : (1u << (w + 1)) - 1;
  if (w < 2 || w >= n || n < 3 || n > 15 || (n & 1) == 0) return 0;
  const uint32_t xn1 = (1u << n) | 1u;
  for (uint32_t p = 1u << w; p < (2u << w); ++p)
    if (poly_rem(xn1, p) == 0 && poly_irreducible(p)) return p;
  return 0;
}

// Product in GF(2^w) = F2[x]/(g): shift-and-add, reducing each time the shifted multiplicand
// reaches degree w (x^w = g minus its leading term).
uint32_t gf_mul(uint32_t g, int w, uint32_t a, uint32_t b) {
  uint32_t r = 0;
  for (int i = 0; i < w; ++i) {
    if ((b >> i) & 1u) r ^= a;
    a <<= 1;
    if ((a >> w) & 1u) a ^= g;
  }
  return r;
}

// a^{-1} = a^{2^w - 2} (Fermat), by square-and-multiply. gf_inv(0) = 0.
uint32_t gf_inv(uint32_t g, int w, uint32_t a) {
  uint32_t e = (1u << w) - 2, r = 1, s = a;
  while (e) {
    if (e & 1u) r = gf_mul(g, w, r, s);
    s = gf_mul(g, w, s, s);
    e >>= 1;
  }
  return a ? r : 0;
}

// phi_S (Sec. 2.2): the ring elements of R_{2,n} reducing to u mod the modulus g are u + h g for
// the 2^(n-w) polynomials h of degree < n - w. The lightest is taken, the smallest on ties. For an
// AOP that is u or its complement in n bits (weights t and n - t, never tied for odd n); for the
// ESP of GF(2^6) one of eight.
uint32_t sparse_rep(uint32_t g, int w, int n, uint32_t u) {
  u &= (1u << w) - 1;
  uint32_t best = u;
  int bw = __builtin_popcount(u);
  for (uint32_t h = 1; h < (1u << (n - w)); ++h) {
    uint32_t hg = 0;  // carry-less h * g
    for (int i = 0; i < n - w; ++i)
      if ((h >> i) & 1u) hg ^= g << i;
    const uint32_t r = u ^ hg;
    const int c = __builtin_popcount(r);
    if (c < bw || (c == bw && r < best)) {
      best = r;
      bw = c;
    }
  }
  return best;
}

// Inverse over GF(2^w) by elimination with row swaps (k <= 64). Returns false if singular.
static bool invert(uint32_t g, int w, int k, const uint32_t* A, uint32_t* out) {
  uint32_t a[kMaxIn][kMaxIn], b[kMaxIn][kMaxIn];
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < k; ++c) {
      a[r][c] = A[r * k + c];
      b[r][c] = (r == c);
    }
  for (int c = 0; c < k; ++c) {
    int piv = c;
    while (piv < k && a[piv][c] == 0) ++piv;
    if (piv == k) return false;
    if (piv != c)
      for (int x = 0; x < k; ++x) {
        std::swap(a[c][x], a[piv][x]);
        std::swap(b[c][x], b[piv][x]);
      }
    const uint32_t s = gf_inv(g, w, a[c][c]);
    for (int x = 0; x < k; ++x) {
      a[c][x] = gf_mul(g, w, a[c][x], s);
      b[c][x] = gf_mul(g, w, b[c][x], s);
    }
    for (int r = 0; r < k; ++r) {
      if (r == c || a[r][c] == 0) continue;
      const uint32_t f = a[r][c];
      for (int x = 0; x < k; ++x) {
        a[r][x] ^= gf_mul(g, w, f, a[c][x]);
        b[r][x] ^= gf_mul(g, w, f, b[c][x]);
      }
    }
  }
  for (int r = 0; r < k; ++r)
    for (int c = 0; c < k; ++c) out[r * k + c] = b[r][c];
  return true;
}

// Every k x k row subset of G invertible (the MDS property, Sec. 2.2), by enumeration.
static bool all_subsets_invertible(uint32_t g, int w, int k, int m, const uint32_t* G) {
  int idx[kMaxBlocks];
  for (int i = 0; i < k; ++i) idx[i] = i;
  uint32_t sub[kMaxIn * kMaxIn], inv[kMaxIn * kMaxIn];
  const int nrow = k + m;
  while (true) {
    for (int r = 0; r < k; ++r)
      for (int c = 0; c < k; ++c) sub[r * k + c] = G[idx[r] * k + c];
    if (!invert(g, w, k, sub, inv)) return false;
    int i = k - 1;
    while (i >= 0 && idx[i] == nrow - k + i) --i;
    if (i < 0) return true;
    ++idx[i];
    for (int j = i + 1; j < k; ++j) idx[j] = idx[j - 1] + 1;
  }
}

static double binom(int a, int b) {
  double r = 1;
  for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
  return r;
}

// The syndrome form of a decode entry (see SyndromeStore in ring_staged.cuh): with D the lost
// data blocks (a of them), U the first a surviving parity rows and X = (C_{U,D})^{-1}, lost data
// block D_i is row i of X applied to the syndromes of U, and lost parity row r is its partial
// sum plus (C_{r,D} X) applied to them. C_{U,D} is a square submatrix of the parity part of an MDS
// systematic generator, hence invertible whenever the survivors' matrix is.
static void syndrome_entry(const pyrit_plan_s* p, DecodeEntry* e) {
  const int k = p->k, m = p->m, w = p->w, n = p->n;
  e->syn_ok = false;
  std::memset(e->syn, 0, sizeof(e->syn));
  if (k + m > kMaxIn || m > kMaxOut) return;
  int D[kMaxOut], U[kMaxOut], a = 0, nu = 0;
  for (int r = 0; r < e->ne; ++r)
    if (e->erased[r] < k) D[a++] = e->erased[r];
  for (int s = 0; s < k; ++s)
    if (e->surv[s] >= k) U[nu++] = e->surv[s] - k;
  if (nu != a) return;
  uint32_t A[kMaxOut * kMaxOut], X[kMaxOut * kMaxOut];
  for (int i = 0; i < a; ++i)
    for (int j = 0; j < a; ++j) A[i * a + j] = p->G[(k + U[i]) * k + D[j]];
  if (a > 0 && !invert(p->g, w, a, A, X)) return;
  for (int o = 0; o < e->ne; ++o) {
    const int b = e->erased[o];
    for (int s = 0; s < a; ++s) {
      uint32_t v = 0;
      if (b < k) {
        int i = 0;
        while (D[i] != b) ++i;
        v = X[i * a + s];
      } else {
        for (int i = 0; i < a; ++i) v ^= gf_mul(p->g, w, p->G[b * k + D[i]], X[i * a + s]);
      }
      e->syn[U[s]][o] = (uint16_t)sparse_rep(p->g, w, n, v);
    }
    e->syn[kSyndromeBaseRow][o] = (uint16_t)(b < k ? 0 : b - k + 1);
  }
  e->syn_ok = true;
}

int plan_decode_entry(pyrit_plan_s* p, uint64_t erasures, DecodeEntry* out) {
  const int k = p->k, m = p->m, w = p->w, n = p->n;
  if (k + m < 64 && (erasures >> (k + m)) != 0) return PYRIT_E_INVALID_ARG;
  if (__builtin_popcountll(erasures) > m) return PYRIT_E_TOO_MANY_ERASURES;
  {
    std::lock_guard<std::mutex> lk(p->mu);
    auto it = p->dcache.find(erasures);
    if (it != p->dcache.end()) {
      *out = it->second;
      return out->status;
    }
  }
  DecodeEntry e;
  int ns = 0;
  for (int b = 0; b < k + m; ++b) {
    if ((erasures >> b) & 1u)
      e.erased[e.ne++] = b;
    else if (ns < k)
      e.surv[ns++] = b;
  }
  std::memset(e.mask, 0, sizeof(e.mask));
  if (e.ne > 0) {
    uint32_t Gs[kMaxIn * kMaxIn], Inv[kMaxIn * kMaxIn];
    for (int s = 0; s < k; ++s)
      for (int c = 0; c < k; ++c) Gs[s * k + c] = p->G[e.surv[s] * k + c];
    if (!invert(p->g, w, k, Gs, Inv)) {
      e.status = PYRIT_E_NOT_MDS;
    } else {
      for (int r = 0; r < e.ne; ++r) {
        const int b = e.erased[r];
        for (int s = 0; s < k; ++s) {
          uint32_t v;
          if (b < k) {
            v = Inv[b * k + s];
          } else {  // an erased parity block: G[b] times Inv
            v = 0;
            for (int j = 0; j < k; ++j) v ^= gf_mul(p->g, w, p->G[b * k + j], Inv[j * k + s]);
          }
          e.mask[r][s] = (uint16_t)sparse_rep(p->g, w, n, v);
        }
      }
      syndrome_entry(p, &e);
    }
  }
  {
    std::lock_guard<std::mutex> lk(p->mu);
    p->dcache.emplace(erasures, e);
  }
  *out = e;
  return e.status;
}

int make_encode_jobs(const pyrit_plan_s* p, const void* const* data, void* const* parity, size_t P,
                     JobDesc* jobs) {
  const int nj = (p->m + kMaxOut - 1) / kMaxOut;
  for (int g = 0; g < nj; ++g) {
    JobDesc* job = &jobs[g];
    std::memset(job, 0, sizeof(*job));
    const int o0 = g * kMaxOut, no = std::min(kMaxOut, p->m - o0);
    job->nin = p->k;
    job->nout = no;
    job->P = P;
    job->table = g;
    for (int j = 0; j < p->k; ++j) job->in[j] = static_cast<const uint8_t*>(data[j]);
    for (int i = 0; i < no; ++i) job->out[i] = static_cast<uint8_t*>(parity[o0 + i]);
    for (int i = 0; i < no; ++i)
      for (int j = 0; j < p->k; ++j) job->mask[j][i] = p->enc_mask[(o0 + i) * p->k + j];
  }
  return nj;
}

int make_decode_jobs(const pyrit_plan_s* p, const DecodeEntry& e, void* const* blocks, size_t P,
                     JobDesc* jobs) {
  const int nj = (e.ne + kMaxOut - 1) / kMaxOut;
  for (int g = 0; g < nj; ++g) {
    JobDesc* job = &jobs[g];
    std::memset(job, 0, sizeof(*job));
    const int o0 = g * kMaxOut, no = std::min(kMaxOut, e.ne - o0);
    job->nin = p->k;
    job->nout = no;
    job->P = P;
    job->table = g;
    for (int s = 0; s < p->k; ++s) job->in[s] = static_cast<const uint8_t*>(blocks[e.surv[s]]);
    for (int r = 0; r < no; ++r) job->out[r] = static_cast<uint8_t*>(blocks[e.erased[o0 + r]]);
    for (int r = 0; r < no; ++r)
      for (int s = 0; s < p->k; ++s) job->mask[s][r] = e.mask[o0 + r][s];
  }
  return nj;
}

void make_syndrome_job(const pyrit_plan_s* p, const DecodeEntry& e, void* const* blocks, size_t P, JobDesc* job) {
  std::memset(job, 0, sizeof(*job));
  const int k = p->k, m = p->m;
  job->nin = k + m;
  job->nout = e.ne;
  job->P = P;
  for (int s = 0; s < k; ++s) job->in[e.surv[s]] = static_cast<const uint8_t*>(blocks[e.surv[s]]);
  for (int o = 0; o < e.ne; ++o) job->out[o] = static_cast<uint8_t*>(blocks[e.erased[o]]);
  uint32_t need = 0;  // parity rows that are syndromes or partial sums of this pattern
  for (int o = 0; o < e.ne; ++o) {
    for (int r = 0; r < m; ++r)
      if (e.syn[r][o]) need |= 1u << r;
    if (e.syn[kSyndromeBaseRow][o]) need |= 1u << (e.syn[kSyndromeBaseRow][o] - 1);
  }
  for (int r = 0; r <= kSyndromeBaseRow; ++r)
    for (int o = 0; o < e.ne; ++o) job->mask[r][o] = e.syn[r][o];
  job->mask[kSyndromeNeedRow][0] = (uint16_t)need;
}

// Validates a stripe request and builds its coding jobs; alg / src receive its algorithmic and
// source bytes.
int stripe_jobs(const pyrit_stripe_t& s, JobDesc* jobs, int* njobs, uint64_t* alg, uint64_t* src) {
  pyrit_plan_s* p = s.plan;
  if (!p || !s.blocks || s.packet_bytes == 0 || s.packet_bytes > (1ull << 40)) return PYRIT_E_INVALID_ARG;
  if (s.op != PYRIT_OP_ENCODE && s.op != PYRIT_OP_DECODE) return PYRIT_E_INVALID_ARG;
  for (int b = 0; b < p->k + p->m; ++b)
    if (!s.blocks[b]) return PYRIT_E_INVALID_ARG;
  const uint64_t blk = (uint64_t)p->w * s.packet_bytes;
  *src = (uint64_t)p->k * blk;
  if (s.op == PYRIT_OP_ENCODE) {
    *njobs = make_encode_jobs(p, s.blocks, s.blocks + p->k, s.packet_bytes, jobs);
    *alg = (uint64_t)(p->k + p->m) * blk;
    return PYRIT_OK;
  }
  DecodeEntry e;
  const int rc = plan_decode_entry(p, s.erasures, &e);
  if (rc != PYRIT_OK) return rc;
  *njobs = make_decode_jobs(p, e, s.blocks, s.packet_bytes, jobs);
  *alg = (uint64_t)(p->k + e.ne) * blk;
  return PYRIT_OK;
}

}  // namespace pyrit

using namespace pyrit;

extern "C" {

const char* pyrit_strerror(int s) {
  switch (s) {
    case PYRIT_OK: return "ok";
    case PYRIT_E_INVALID_ARG: return "invalid argument";
    case PYRIT_E_UNSUPPORTED_FIELD:
      return "unsupported field (n = w+1 with an irreducible AOP, or w = 6, n = 9 for x^6+x^3+1)";
    case PYRIT_E_TOO_LONG: return "code too long for the field (k+m > 2^w)";
    case PYRIT_E_NOT_MDS: return "generator is not systematic MDS";
    case PYRIT_E_TOO_MANY_ERASURES: return "more erasures than parity blocks";
    case PYRIT_E_CUDA: return "CUDA error";
    case PYRIT_E_OOM: return "out of memory";
    case PYRIT_E_BUDGET: return "request exceeds the admission budget";
    case PYRIT_E_TIMEOUT: return "bounded wait timed out";
    case PYRIT_E_BUSY: return "queue full";
    case PYRIT_E_SCRATCH_LIMIT: return "request exceeds the fixed scratch of the no-allocation entry point";
    case PYRIT_E_JIT: return "run-time compilation or loading of a generated network failed";
    case PYRIT_E_UNSUPPORTED: return "the parity transform runs only on generated networks";
    default: return "unknown status";
  }
}

int pyrit_plan_create(int w, int n, int k, int m, const uint32_t* G, pyrit_plan_t* out) {
  if (!out) return PYRIT_E_INVALID_ARG;
  *out = nullptr;
  if (k < 1 || k > PYRIT_MAX_K || m < 0 || m > PYRIT_MAX_M || k + m > kMaxBlocks) return PYRIT_E_INVALID_ARG;
  const uint32_t g = field_modulus(w, n);
  if (!g) return PYRIT_E_UNSUPPORTED_FIELD;
  if (!G && (uint64_t)k + (uint64_t)m > (1ull << w)) return PYRIT_E_TOO_LONG;
  pyrit_plan_s* p = new (std::nothrow) pyrit_plan_s;
  if (!p) return PYRIT_E_OOM;
  static std::atomic<uint64_t> next_serial{1};
  p->serial = next_serial.fetch_add(1);
  p->w = w;
  p->n = n;
  p->g = g;
  p->native = field_native(w, n);
  p->k = k;
  p->m = m;
  p->G.assign((size_t)(k + m) * k, 0);
  if (G) {
    for (int r = 0; r < k + m; ++r)
      for (int c = 0; c < k; ++c) {
        const uint32_t v = G[r * k + c];
        if (v >= (1u << w) || (r < k && v != (uint32_t)(r == c))) {
          delete p;
          return PYRIT_E_NOT_MDS;
        }
        p->G[r * k + c] = v;
      }
    if (binom(k + m, k) <= 20000.0 && !all_subsets_invertible(g, w, k, m, p->G.data())) {
      delete p;
      return PYRIT_E_NOT_MDS;
    }
  } else {
    // Cauchy: C[i][j] = 1 / (x_i + y_j), x_i = k + i, y_j = j (all points distinct).
    for (int r = 0; r < k; ++r) p->G[r * k + r] = 1;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < k; ++j) p->G[(k + i) * k + j] = gf_inv(g, w, (uint32_t)(k + i) ^ (uint32_t)j);
  }
  p->enc_mask.resize((size_t)m * k);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < k; ++j) p->enc_mask[i * k + j] = (uint16_t)sparse_rep(g, w, n, p->G[(k + i) * k + j]);
  *out = p;
  return PYRIT_OK;
}

void pyrit_plan_destroy(pyrit_plan_t p) { delete p; }

int pyrit_plan(int w, int n, int k, int m, const uint16_t* G, pyrit_plan_t* out) {
  if (!G) return pyrit_plan_create(w, n, k, m, nullptr, out);
  if (k < 1 || m < 0 || k > PYRIT_MAX_K || m > PYRIT_MAX_M || k + m > PYRIT_MAX_BLOCKS) return PYRIT_E_INVALID_ARG;
  std::vector<uint32_t> g32(G, G + (size_t)(k + m) * (size_t)k);
  return pyrit_plan_create(w, n, k, m, g32.data(), out);
}

int pyrit_plan_set_transform(pyrit_plan_t p, int transform) {
  if (!p) return PYRIT_E_INVALID_ARG;
  // the parity transform is defined for the all-one and equally spaced polynomials (Sec. 2.3.1,
  // Sec. 2.4.1), whose ideals are characterised by parities; other factors take the embedding
  if (transform == PYRIT_TRANSFORM_AUTO)
    transform = p->k < p->m && p->native ? PYRIT_TRANSFORM_PARITY : PYRIT_TRANSFORM_EMBEDDING;
  if (transform != PYRIT_TRANSFORM_EMBEDDING && transform != PYRIT_TRANSFORM_PARITY) return PYRIT_E_INVALID_ARG;
  if (transform == PYRIT_TRANSFORM_PARITY && !p->native) return PYRIT_E_UNSUPPORTED;
  p->transform = transform;
  return transform;
}

int pyrit_plan_modulus(pyrit_plan_t p, uint32_t* g_out, int* native_out) {
  if (!p) return PYRIT_E_INVALID_ARG;
  if (g_out) *g_out = p->g;
  if (native_out) *native_out = p->native ? 1 : 0;
  return PYRIT_OK;
}

int pyrit_plan_info(pyrit_plan_t p, int* w, int* n, int* k, int* m) {
  if (!p) return PYRIT_E_INVALID_ARG;
  if (w) *w = p->w;
  if (n) *n = p->n;
  if (k) *k = p->k;
  if (m) *m = p->m;
  return PYRIT_OK;
}

int pyrit_plan_generator(pyrit_plan_t p, uint32_t* G_out) {
  if (!p || !G_out) return PYRIT_E_INVALID_ARG;
  std::memcpy(G_out, p->G.data(), p->G.size() * sizeof(uint32_t));
  return PYRIT_OK;
}

int pyrit_plan_encode_masks(pyrit_plan_t p, uint16_t* masks_out) {
  if (!p || !masks_out) return PYRIT_E_INVALID_ARG;
  std::memcpy(masks_out, p->enc_mask.data(), p->enc_mask.size() * sizeof(uint16_t));
  return PYRIT_OK;
}

int pyrit_generator_weighted(int w, int n, int k, int m, uint32_t* G_out, uint64_t* weights_out) {
  if (!G_out || k < 1 || k > PYRIT_MAX_K || m < 0 || m > PYRIT_MAX_M || k + m > kMaxBlocks) return PYRIT_E_INVALID_ARG;
  const uint32_t g = field_modulus(w, n);
  if (!g) return PYRIT_E_UNSUPPORTED_FIELD;
  if ((uint64_t)k + (uint64_t)m > (1ull << w)) return PYRIT_E_TOO_LONG;
  const uint32_t q = 1u << w;
  // weight of phi_S(u), the number of ones of the sparsest representative
  std::vector<int> wt(q);
  for (uint32_t u = 0; u < q; ++u) wt[u] = __builtin_popcount(sparse_rep(g, w, n, u));
  std::vector<uint32_t> c((size_t)m * k);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < k; ++j) c[(size_t)i * k + j] = gf_inv(g, w, (uint32_t)(k + i) ^ (uint32_t)j);
  std::vector<uint32_t> a(m, 1u), b(k, 1u);
  auto entry = [&](int i, int j, uint32_t ai, uint32_t bj) {
    return gf_mul(g, w, gf_mul(g, w, ai, bj), c[(size_t)i * k + j]);
  };
  uint64_t before = 0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < k; ++j) before += (uint64_t)wt[c[(size_t)i * k + j]];
  for (int round = 0; round < 8; ++round) {
    bool changed = false;
    for (int j = 0; j < k; ++j) {  // column scalings, then row scalings; smallest element on ties
      uint32_t best = 0;
      long bw = -1;
      for (uint32_t sc = 1; sc < q; ++sc) {
        long sum = 0;
        for (int i = 0; i < m; ++i) sum += wt[entry(i, j, a[i], sc)];
        if (bw < 0 || sum < bw) {
          bw = sum;
          best = sc;
        }
      }
      changed = changed || best != b[j];
      b[j] = best;
    }
    for (int i = 0; i < m; ++i) {
      uint32_t best = 0;
      long bw = -1;
      for (uint32_t sc = 1; sc < q; ++sc) {
        long sum = 0;
        for (int j = 0; j < k; ++j) sum += wt[entry(i, j, sc, b[j])];
        if (bw < 0 || sum < bw) {
          bw = sum;
          best = sc;
        }
      }
      changed = changed || best != a[i];
      a[i] = best;
    }
    if (!changed) break;
  }
  uint64_t after = 0;
  for (int r = 0; r < k; ++r)
    for (int cc = 0; cc < k; ++cc) G_out[r * k + cc] = r == cc ? 1u : 0u;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < k; ++j) {
      const uint32_t v = entry(i, j, a[i], b[j]);
      G_out[(k + i) * k + j] = v;
      after += (uint64_t)wt[v];
    }
  if (weights_out) {
    weights_out[0] = before;
    weights_out[1] = after;
  }
  return PYRIT_OK;
}

int pyrit_plan_syndrome_masks(pyrit_plan_t p, uint64_t erasures, uint16_t* syn_out, int* ne_out) {
  if (!p || !syn_out) return PYRIT_E_INVALID_ARG;
  DecodeEntry e;
  const int rc = plan_decode_entry(p, erasures, &e);
  if (rc != PYRIT_OK) return rc;
  if (!e.syn_ok && e.ne > 0) return PYRIT_E_INVALID_ARG;
  for (int r = 0; r <= kSyndromeBaseRow; ++r)
    for (int o = 0; o < kMaxOut; ++o) syn_out[r * kMaxOut + o] = o < e.ne ? e.syn[r][o] : 0;
  if (ne_out) *ne_out = e.ne;
  return PYRIT_OK;
}

int pyrit_plan_decode_masks(pyrit_plan_t p, uint64_t erasures, int* survivors_out, int* erased_out,
                            uint16_t* masks_out, int* ne_out) {
  if (!p) return PYRIT_E_INVALID_ARG;
  DecodeEntry e;
  const int rc = plan_decode_entry(p, erasures, &e);
  if (rc != PYRIT_OK) return rc;
  if (ne_out) *ne_out = e.ne;
  if (survivors_out)
    for (int s = 0; s < p->k; ++s) survivors_out[s] = e.surv[s];
  if (erased_out)
    for (int r = 0; r < e.ne; ++r) erased_out[r] = e.erased[r];
  if (masks_out)
    for (int r = 0; r < e.ne; ++r)
      for (int s = 0; s < p->k; ++s) masks_out[r * p->k + s] = e.mask[r][s];
  return PYRIT_OK;
}

uint32_t pyrit_sparse_transform(int w, int n, uint32_t u) {
  const uint32_t g = field_modulus(w, n);
  if (!g || u >= (1u << w)) return 0xFFFFFFFFu;
  return sparse_rep(g, w, n, u);
}

uint32_t pyrit_gf_mul(int w, uint32_t a, uint32_t b) {
  if (w < 2 || w > 15) return 0;
  const uint32_t g = w == 6 ? 0x49u : (1u << (w + 1)) - 1;  // the field of w on its native ring
  return gf_mul(g, w, a & ((1u << w) - 1), b & ((1u << w) - 1));
}

}  // extern "C"
