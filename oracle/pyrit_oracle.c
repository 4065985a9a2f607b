/*
 * PYRIT CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow and deliberately literal CPU implementation of what the coding path computes:
 * systematic MDS erasure encoding and decoding over GF(2^w) = F2[x]/(p(x)), p the all-one
 * polynomial (AOP) of degree w when that is irreducible (Sec. 2.3), else an irreducible equally
 * spaced polynomial (ESP) of degree w (Sec. 2.4: GF(2^6) from x^6 + x^3 + 1), with log/antilog
 * tables and a Cauchy generator matrix.
 * It also holds a small reference for the ring R_{2,n} = F2[x]/(x^n+1) that the tests use to
 * check the paper's algebraic claims.
 *
 * It shares no code, header, table or constant with the CUDA library. Only the tests, the
 * package's smoke check and the benchmark's CPU-baseline leg may load it. The product path
 * never calls it.
 *
 * Paper: J. Detchart, J. Lacan, "Improving the coding speed of erasure codes with polynomial
 * ring transforms", arXiv:1709.00178. Citations below name its sections and equations.
 *
 * Conventions (all readings of the paper are listed in the design notes):
 *  - A field or ring element is an integer whose bit i is the coefficient of x^i (Sec. 2.1).
 *  - A block is w packets of P bytes, packet q at byte offset q*P. Bit b of byte t of packet q
 *    is coefficient q of symbol (t, b): every (t, b) is an independent symbol lane.
 *  - Generator G is (k+m) x k, row-major, systematic (top k x k = identity).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_W 16
#define ORACLE_MAX_K 64

/* ------------------------------------------------------------------------------------------ */
/* Polynomials over F2 (Sec. 2.1)                                                              */
/* ------------------------------------------------------------------------------------------ */

/* Degree of a nonzero polynomial; -1 for the zero polynomial. */
static int poly_deg(uint64_t a) {
  int d = -1;
  while (a) {
    d++;
    a >>= 1;
  }
  return d;
}

/* Remainder of a(x) divided by p(x) over F2, by schoolbook long division. */
uint64_t oracle_poly_mod(uint64_t a, uint64_t p) {
  int dp = poly_deg(p);
  if (dp < 0) return 0;
  for (int d = 63; d >= dp; d--)
    if ((a >> d) & 1) a ^= p << (d - dp);
  return a;
}

/* Carry-less (F2[x]) product of two polynomials of degree < 32. */
uint64_t oracle_poly_mul(uint64_t a, uint64_t b) {
  uint64_t r = 0;
  for (int i = 0; i < 32; i++)
    if ((b >> i) & 1) r ^= a << i;
  return r;
}

/* The all-one polynomial of degree w: 1 + x + ... + x^w (Sec. 2.3). */
uint64_t oracle_aop(int w) { return (((uint64_t)1) << (w + 1)) - 1; }

/* Irreducibility of p (degree 1..30), by trial division by every polynomial of degree
 * 1..deg(p)/2: the definition of irreducible, not the paper's number-theoretic criteria, so that
 * the tests can check those criteria against it. Returns 1 if irreducible. */
int oracle_poly_irreducible(uint64_t p) {
  const int w = poly_deg(p);
  if (w < 1 || w > 30) return 0;
  for (int d = 1; d <= w / 2; d++)
    for (uint64_t f = (uint64_t)1 << d; f < ((uint64_t)1 << (d + 1)); f++)
      if (oracle_poly_mod(p, f) == 0) return 0;
  return 1;
}

/* Irreducibility of the AOP of degree w. Returns 1 if irreducible. */
int oracle_aop_irreducible(int w) { return w >= 1 && w <= 30 && oracle_poly_irreducible(oracle_aop(w)); }

/* The s-equally spaced polynomial of degree s r (Sec. 2.4, its definition): p(x^s) for the AOP p
 * of degree r, i.e. 1 + x^s + x^{2s} + ... + x^{rs}. s = 1 gives the AOP itself. */
uint64_t oracle_esp(int s, int r) {
  uint64_t g = 0;
  for (int i = 0; i <= r; i++) g |= (uint64_t)1 << (s * i);
  return g;
}

/* The modulus of GF(2^w) in this codec: the AOP of degree w when irreducible, else the
 * irreducible ESP p(x^s) of degree w = s r with the smallest s > 1, else 0 (no such field). The
 * ring that carries it is R_{2,n}, n = s (r + 1), since x^{s(r+1)} + 1 = g(x) (x^s + 1). */
static int field_spacing_search(int w) {
  if (w < 2 || w > ORACLE_MAX_W) return 0;
  if (oracle_aop_irreducible(w)) return 1;
  for (int s = 2; s <= w / 2; s++)
    if (w % s == 0 && oracle_poly_irreducible(oracle_esp(s, w / s))) return s;
  return 0;
}

/* The search above, once per w (the field product calls it for every multiplication). */
static pthread_mutex_t spacing_mu = PTHREAD_MUTEX_INITIALIZER;
static int spacing_of[ORACLE_MAX_W + 1];
static int spacing_known[ORACLE_MAX_W + 1];

static int field_spacing(int w) {
  if (w < 2 || w > ORACLE_MAX_W) return 0;
  pthread_mutex_lock(&spacing_mu);
  if (!spacing_known[w]) {
    spacing_of[w] = field_spacing_search(w);
    spacing_known[w] = 1;
  }
  const int s = spacing_of[w];
  pthread_mutex_unlock(&spacing_mu);
  return s;
}

uint64_t oracle_field_poly(int w) {
  const int s = field_spacing(w);
  return s ? oracle_esp(s, w / s) : 0;
}

/* n of the ring R_{2,n} the field GF(2^w) is embedded in (0 if the field is not supported). */
int oracle_ring_size(int w) {
  const int s = field_spacing(w);
  return s ? s * (w / s + 1) : 0;
}

/* ------------------------------------------------------------------------------------------ */
/* The field GF(2^w) = F2[x]/(AOP or ESP) (Sec. 2.1, Sec. 2.3, Sec. 2.4)                       */
/* ------------------------------------------------------------------------------------------ */

/* Field product by the definition: carry-less product, then remainder mod the modulus `poly`
 * (any irreducible polynomial of degree w: the AOP, an ESP, or another factor of x^n + 1). */
uint32_t oracle_gf_mul_mod(int w, uint64_t poly, uint32_t a, uint32_t b) {
  (void)w;
  return (uint32_t)oracle_poly_mod(oracle_poly_mul(a, b), poly);
}

/* The same under the library's default modulus for w. */
uint32_t oracle_gf_mul_slow(int w, uint32_t a, uint32_t b) { return oracle_gf_mul_mod(w, oracle_field_poly(w), a, b); }

/* Multiplicative order of a nonzero element (0 if its powers reach 0 or never return to 1,
 * which only happens when the modulus is reducible). */
static uint32_t gf_order_mod(int w, uint64_t poly, uint32_t g) {
  uint32_t q = (1u << w);
  uint32_t v = g;
  for (uint32_t e = 1; e <= q; e++) {
    if (v == 1) return e;
    if (v == 0) return 0;
    v = oracle_gf_mul_mod(w, poly, v, g);
  }
  return 0;
}

uint32_t oracle_gf_order(int w, uint32_t g) { return gf_order_mod(w, oracle_field_poly(w), g); }

/* The smallest irreducible factor of degree w of x^n + 1 (n odd, Props. 1-2: x^n + 1 is then a
 * product of distinct irreducible polynomials), by trial over the degree-w polynomials in
 * increasing order; 0 if there is none. */
uint64_t oracle_ring_factor(int w, int n) {
  if (w < 1 || w > ORACLE_MAX_W || n < 3 || n > 31 || (n & 1) == 0) return 0;
  const uint64_t xn1 = ((uint64_t)1 << n) | 1;
  for (uint64_t p = (uint64_t)1 << w; p < ((uint64_t)1 << (w + 1)); p++)
    if (oracle_poly_mod(xn1, p) == 0 && oracle_poly_irreducible(p)) return p;
  return 0;
}

typedef struct {
  int w;
  uint32_t q1;    /* 2^w - 1, the order of the multiplicative group */
  uint32_t g;     /* the primitive element used for the tables */
  uint32_t* log;  /* log[a] for a != 0 */
  uint32_t* alog; /* alog[e] = g^e, e in [0, 2^w - 1) */
} gf_t;

/* The primitive element: the smallest integer >= 2 whose order is 2^w - 1. Under an AOP the
 * element x (= 2) has order w+1 (x^{w+1} = 1), under an ESP of degree s r order s (r + 1), so it
 * is not primitive; the paper does not name a generator, hence the search. Returns 0 if none
 * exists. */
static uint32_t gf_primitive_mod(int w, uint64_t poly) {
  if (w < 2 || w > ORACLE_MAX_W || !poly || poly_deg(poly) != w || !oracle_poly_irreducible(poly)) return 0;
  uint32_t q1 = (1u << w) - 1;
  for (uint32_t g = 2; g <= q1; g++)
    if (gf_order_mod(w, poly, g) == q1) return g;
  return 0;
}

uint32_t oracle_gf_primitive(int w) { return gf_primitive_mod(w, oracle_field_poly(w)); }

/* Log/antilog tables of GF(2^w) = F2[x]/(poly) over its smallest primitive element. */
static int gf_init_mod(gf_t* f, int w, uint64_t poly) {
  f->w = w;
  f->q1 = (1u << w) - 1;
  f->g = gf_primitive_mod(w, poly);
  f->log = NULL;
  f->alog = NULL;
  if (!f->g) return -1;
  f->log = (uint32_t*)calloc((size_t)1 << w, sizeof(uint32_t));
  f->alog = (uint32_t*)calloc((size_t)1 << w, sizeof(uint32_t));
  if (!f->log || !f->alog) return -1;
  uint32_t v = 1;
  for (uint32_t e = 0; e < f->q1; e++) {
    f->alog[e] = v;
    f->log[v] = e;
    v = oracle_gf_mul_mod(w, poly, v, f->g);
  }
  return 0;
}

static int gf_init(gf_t* f, int w) { return gf_init_mod(f, w, oracle_field_poly(w)); }

static void gf_free(gf_t* f) {
  free(f->log);
  free(f->alog);
}

static inline uint32_t gf_mul(const gf_t* f, uint32_t a, uint32_t b) {
  if (!a || !b) return 0;
  return f->alog[(f->log[a] + f->log[b]) % f->q1];
}

static inline uint32_t gf_inv(const gf_t* f, uint32_t a) {
  return f->alog[(f->q1 - f->log[a]) % f->q1];
}

/* Exported table access so that the tests can pin the tables against the definition. */
int oracle_gf_tables(int w, uint32_t* log_out, uint32_t* alog_out, uint32_t* g_out) {
  gf_t f;
  if (gf_init(&f, w)) {
    gf_free(&f);
    return -1;
  }
  memcpy(log_out, f.log, sizeof(uint32_t) << w);
  memcpy(alog_out, f.alog, sizeof(uint32_t) << w);
  *g_out = f.g;
  gf_free(&f);
  return 0;
}

/* Table-based product and inverse, exported for the tests (0 has no inverse: returns 0). */
uint32_t oracle_gf_mul(int w, uint32_t a, uint32_t b) {
  gf_t f;
  if (gf_init(&f, w)) {
    gf_free(&f);
    return 0;
  }
  uint32_t r = gf_mul(&f, a, b);
  gf_free(&f);
  return r;
}

/* ------------------------------------------------------------------------------------------ */
/* Generator and matrix inverse (Sec. 3: "generalized Cauchy matrices")                        */
/* ------------------------------------------------------------------------------------------ */

/* Systematic generator G = [I_k ; C], C[i][j] = 1 / (x_i + y_j) with x_i = k + i and y_j = j.
 * The paper names generalized Cauchy matrices without their parameters; this is the plain
 * Cauchy matrix on those points. It needs k + m <= 2^w so that all points are distinct.
 * Returns 0, or -1 for an unsupported field, -2 for k + m > 2^w. */
int oracle_cauchy_mod(int w, uint64_t poly, int k, int m, uint32_t* G) {
  if (k < 1 || m < 0 || k > ORACLE_MAX_K) return -2;
  if ((uint64_t)k + (uint64_t)m > ((uint64_t)1 << w)) return -2;
  gf_t f;
  if (gf_init_mod(&f, w, poly)) {
    gf_free(&f);
    return -1;
  }
  for (int r = 0; r < k; r++)
    for (int c = 0; c < k; c++) G[r * k + c] = (r == c);
  for (int i = 0; i < m; i++)
    for (int j = 0; j < k; j++) G[(k + i) * k + j] = gf_inv(&f, (uint32_t)(k + i) ^ (uint32_t)j);
  gf_free(&f);
  return 0;
}

int oracle_cauchy(int w, int k, int m, uint32_t* G) { return oracle_cauchy_mod(w, oracle_field_poly(w), k, m, G); }

/* Gauss-Jordan inverse of a k x k matrix over GF(2^w). The pivot of column c is the first row
 * at or below row c with a nonzero entry in column c. Returns 0, or -1 if singular. */
static int gf_invert(const gf_t* f, int k, const uint32_t* A, uint32_t* Inv) {
  uint32_t* M = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)k * (size_t)(2 * k));
  if (!M) return -1;
  for (int r = 0; r < k; r++)
    for (int c = 0; c < 2 * k; c++) M[r * 2 * k + c] = (c < k) ? A[r * k + c] : (uint32_t)(c - k == r);
  for (int c = 0; c < k; c++) {
    int piv = -1;
    for (int r = c; r < k; r++)
      if (M[r * 2 * k + c]) {
        piv = r;
        break;
      }
    if (piv < 0) {
      free(M);
      return -1;
    }
    if (piv != c)
      for (int x = 0; x < 2 * k; x++) {
        uint32_t t = M[c * 2 * k + x];
        M[c * 2 * k + x] = M[piv * 2 * k + x];
        M[piv * 2 * k + x] = t;
      }
    uint32_t s = gf_inv(f, M[c * 2 * k + c]);
    for (int x = 0; x < 2 * k; x++) M[c * 2 * k + x] = gf_mul(f, M[c * 2 * k + x], s);
    for (int r = 0; r < k; r++) {
      if (r == c || !M[r * 2 * k + c]) continue;
      uint32_t e = M[r * 2 * k + c];
      for (int x = 0; x < 2 * k; x++) M[r * 2 * k + x] ^= gf_mul(f, e, M[c * 2 * k + x]);
    }
  }
  for (int r = 0; r < k; r++)
    for (int c = 0; c < k; c++) Inv[r * k + c] = M[r * 2 * k + k + c];
  free(M);
  return 0;
}

int oracle_gf_invert_mod(int w, uint64_t poly, int k, const uint32_t* A, uint32_t* Inv) {
  gf_t f;
  if (gf_init_mod(&f, w, poly)) {
    gf_free(&f);
    return -2;
  }
  int rc = gf_invert(&f, k, A, Inv);
  gf_free(&f);
  return rc;
}

int oracle_gf_invert(int w, int k, const uint32_t* A, uint32_t* Inv) {
  return oracle_gf_invert_mod(w, oracle_field_poly(w), k, A, Inv);
}

/* ------------------------------------------------------------------------------------------ */
/* Encode and decode on bit-sliced blocks (Sec. 3, Sec. 4)                                     */
/* ------------------------------------------------------------------------------------------ */

/* Symbol (t, b) of a block: coefficient q is bit b of byte t of packet q. */
static inline uint32_t gather_symbol(const uint8_t* blk, int w, size_t P, size_t t, int b) {
  uint32_t s = 0;
  for (int q = 0; q < w; q++) s |= (uint32_t)((blk[(size_t)q * P + t] >> b) & 1) << q;
  return s;
}

static inline void scatter_symbol(uint8_t* blk, int w, size_t P, size_t t, int b, uint32_t s) {
  for (int q = 0; q < w; q++) {
    uint8_t* byte = &blk[(size_t)q * P + t];
    *byte = (uint8_t)((*byte & ~(1u << b)) | (((s >> q) & 1) << b));
  }
}

typedef struct {
  const gf_t* f;
  int k, m;
  const uint32_t* G;
  const uint8_t* data;
  uint8_t* parity;
  size_t P, t0, t1;
} enc_job_t;

/* parity_i = sum_j G[k+i][j] * d_j for every symbol lane in byte range [t0, t1). */
static void* enc_run(void* arg) {
  enc_job_t* J = (enc_job_t*)arg;
  int w = J->f->w;
  size_t blk = (size_t)w * J->P;
  uint32_t d[ORACLE_MAX_K];
  for (size_t t = J->t0; t < J->t1; t++)
    for (int b = 0; b < 8; b++) {
      for (int j = 0; j < J->k; j++) d[j] = gather_symbol(J->data + (size_t)j * blk, w, J->P, t, b);
      for (int i = 0; i < J->m; i++) {
        uint32_t acc = 0;
        for (int j = 0; j < J->k; j++) acc ^= gf_mul(J->f, J->G[(J->k + i) * J->k + j], d[j]);
        scatter_symbol(J->parity + (size_t)i * blk, w, J->P, t, b, acc);
      }
    }
  return NULL;
}

/* Splits the byte range over threads: every thread codes a different part of every symbol,
 * the decomposition of Sec. 4.2. */
static void run_threads(void* (*fn)(void*), void* jobs, size_t job_size, int nthreads) {
  pthread_t th[256];
  if (nthreads > 256) nthreads = 256;
  for (int i = 1; i < nthreads; i++) pthread_create(&th[i], NULL, fn, (char*)jobs + i * job_size);
  fn(jobs);
  for (int i = 1; i < nthreads; i++) pthread_join(th[i], NULL);
}

/* Encodes one stripe. data: k blocks of w*P bytes, contiguous; parity: m blocks, written.
 * Returns 0, -1 for an unsupported field, -3 for bad sizes. */
int oracle_encode_mod(int w, uint64_t poly, int k, int m, const uint32_t* G, const uint8_t* data,
                      uint8_t* parity, size_t P, int nthreads) {
  if (k < 1 || k > ORACLE_MAX_K || m < 0 || P == 0) return -3;
  if (nthreads < 1) nthreads = 1;
  if ((size_t)nthreads > P) nthreads = (int)P;
  gf_t f;
  if (gf_init_mod(&f, w, poly)) {
    gf_free(&f);
    return -1;
  }
  enc_job_t jobs[256];
  if (nthreads > 256) nthreads = 256;
  for (int i = 0; i < nthreads; i++) {
    jobs[i] = (enc_job_t){&f, k, m, G, data, parity, P, P * (size_t)i / (size_t)nthreads,
                          P * (size_t)(i + 1) / (size_t)nthreads};
  }
  run_threads(enc_run, jobs, sizeof(enc_job_t), nthreads);
  gf_free(&f);
  return 0;
}

int oracle_encode(int w, int k, int m, const uint32_t* G, const uint8_t* data, uint8_t* parity, size_t P,
                  int nthreads) {
  return oracle_encode_mod(w, oracle_field_poly(w), k, m, G, data, parity, P, nthreads);
}

typedef struct {
  const gf_t* f;
  int k, m;
  const uint32_t* G;
  const uint32_t* Inv;  /* k x k inverse of the survivors' rows */
  const int* surv;      /* the k survivor indices */
  uint64_t erased;
  uint8_t* blocks;
  size_t P, t0, t1;
} dec_job_t;

/* Recovers the data symbols d = Inv * (survivor symbols), writes the erased data blocks,
 * then re-encodes every erased parity block from the full data vector. */
static void* dec_run(void* arg) {
  dec_job_t* J = (dec_job_t*)arg;
  int w = J->f->w, k = J->k, m = J->m;
  size_t blk = (size_t)w * J->P;
  uint32_t y[ORACLE_MAX_K], d[ORACLE_MAX_K];
  for (size_t t = J->t0; t < J->t1; t++)
    for (int b = 0; b < 8; b++) {
      for (int s = 0; s < k; s++) y[s] = gather_symbol(J->blocks + (size_t)J->surv[s] * blk, w, J->P, t, b);
      for (int j = 0; j < k; j++) {
        uint32_t acc = 0;
        for (int s = 0; s < k; s++) acc ^= gf_mul(J->f, J->Inv[j * k + s], y[s]);
        d[j] = acc;
      }
      for (int e = 0; e < k + m; e++) {
        if (!((J->erased >> e) & 1)) continue;
        uint32_t val;
        if (e < k) {
          val = d[e];
        } else {
          val = 0;
          for (int j = 0; j < k; j++) val ^= gf_mul(J->f, J->G[e * k + j], d[j]);
        }
        scatter_symbol(J->blocks + (size_t)e * blk, w, J->P, t, b, val);
      }
    }
  return NULL;
}

/* Decodes one stripe in place. blocks: k+m blocks of w*P bytes, contiguous (data then parity);
 * bit e of `erased` marks block e lost; every erased block is rebuilt. The survivors are the
 * first k non-erased blocks in index order (the paper does not say which to use; the result
 * is the same for any choice because the code is MDS).
 * Returns 0, -1 unsupported field, -3 bad sizes, -4 more than m erasures, -5 singular. */
int oracle_decode_mod(int w, uint64_t poly, int k, int m, const uint32_t* G, uint8_t* blocks,
                      uint64_t erased, size_t P, int nthreads) {
  if (k < 1 || k > ORACLE_MAX_K || m < 0 || k + m > 64 || P == 0) return -3;
  int ne = 0;
  for (int e = 0; e < k + m; e++) ne += (int)((erased >> e) & 1);
  if ((erased >> (k + m)) != 0 && k + m < 64) return -3;
  if (ne > m) return -4;
  if (ne == 0) return 0;
  gf_t f;
  if (gf_init_mod(&f, w, poly)) {
    gf_free(&f);
    return -1;
  }
  int surv[ORACLE_MAX_K];
  int ns = 0;
  for (int e = 0; e < k + m && ns < k; e++)
    if (!((erased >> e) & 1)) surv[ns++] = e;
  uint32_t* Gs = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)k * (size_t)k);
  uint32_t* Inv = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)k * (size_t)k);
  for (int s = 0; s < k; s++)
    for (int c = 0; c < k; c++) Gs[s * k + c] = G[surv[s] * k + c];
  int rc = gf_invert(&f, k, Gs, Inv);
  if (rc == 0) {
    if (nthreads < 1) nthreads = 1;
    if ((size_t)nthreads > P) nthreads = (int)P;
    if (nthreads > 256) nthreads = 256;
    dec_job_t jobs[256];
    for (int i = 0; i < nthreads; i++)
      jobs[i] = (dec_job_t){&f, k, m, G, Inv, surv, erased, blocks, P,
                            P * (size_t)i / (size_t)nthreads, P * (size_t)(i + 1) / (size_t)nthreads};
    run_threads(dec_run, jobs, sizeof(dec_job_t), nthreads);
  } else {
    rc = -5;
  }
  free(Gs);
  free(Inv);
  gf_free(&f);
  return rc;
}

int oracle_decode(int w, int k, int m, const uint32_t* G, uint8_t* blocks, uint64_t erased, size_t P,
                  int nthreads) {
  return oracle_decode_mod(w, oracle_field_poly(w), k, m, G, blocks, erased, P, nthreads);
}

/* ------------------------------------------------------------------------------------------ */
/* Ring reference R_{2,n} = F2[x]/(x^n + 1) (Sec. 2.1, Props. 1-2, Sec. 2.3)                    */
/* ------------------------------------------------------------------------------------------ */

/* Product in R_{2,n}: cyclic convolution of the coefficient vectors (x^n = 1). */
uint32_t oracle_ring_mul(int n, uint32_t a, uint32_t b) {
  uint32_t r = 0;
  for (int i = 0; i < n; i++)
    if ((a >> i) & 1)
      for (int j = 0; j < n; j++)
        if ((b >> j) & 1) r ^= 1u << ((i + j) % n);
  return r;
}

/* Every idempotent e (e*e = e) of R_{2,n}, by brute force over all 2^n elements.
 * Returns how many were written to out (capacity cap). */
int oracle_ring_idempotents(int n, uint32_t* out, int cap) {
  int c = 0;
  for (uint32_t e = 0; e < (1u << n); e++)
    if (oracle_ring_mul(n, e, e) == e) {
      if (c < cap) out[c] = e;
      c++;
    }
  return c;
}

/* All ring elements r with r mod p = u (the set from which the sparse transform picks), by
 * brute force over all 2^n elements. Returns the count (written up to cap). */
int oracle_ring_representatives(int w, int n, uint32_t u, uint32_t* out, int cap) {
  uint64_t p = oracle_field_poly(w);
  int c = 0;
  for (uint32_t r = 0; r < (1u << n); r++)
    if (oracle_poly_mod(r, p) == u) {
      if (c < cap) out[c] = r;
      c++;
    }
  return c;
}

static int popcount32(uint32_t v) {
  int c = 0;
  while (v) {
    c += (int)(v & 1);
    v >>= 1;
  }
  return c;
}

/* Sparse transform phi_S (Sec. 2.2): the representative of u with the fewest ones; ties go to
 * the smallest integer. Ties cannot occur for an AOP with n odd (weights t and n - t) and do not for
 * GF(2^6) on n = 9; they do for GF(4) from x^2 + x + 1 in R_{2,9} and R_{2,15}. */
uint32_t oracle_sparse_rep_mod(int w, int n, uint64_t p, uint32_t u) {
  (void)w;
  uint32_t best = 0;
  int bw = 99;
  for (uint32_t r = 0; r < (1u << n); r++)
    if (oracle_poly_mod(r, p) == u) {
      int wt = popcount32(r);
      if (wt < bw) {
        bw = wt;
        best = r;
      }
    }
  return best;
}

uint32_t oracle_sparse_rep(int w, int n, uint32_t u) { return oracle_sparse_rep_mod(w, n, oracle_field_poly(w), u); }

/* ------------------------------------------------------------------------------------------ */
/* Element-wise batch forms of the above, so that exhaustive tests do not pay one foreign call */
/* per pair. Each is the same definition applied to cnt pairs.                                 */
/* ------------------------------------------------------------------------------------------ */

int oracle_gf_mul_vec(int w, const uint32_t* a, const uint32_t* b, uint32_t* out, size_t cnt) {
  gf_t f;
  if (gf_init(&f, w)) {
    gf_free(&f);
    return -1;
  }
  for (size_t i = 0; i < cnt; i++) out[i] = gf_mul(&f, a[i], b[i]);
  gf_free(&f);
  return 0;
}

void oracle_gf_mul_slow_vec(int w, const uint32_t* a, const uint32_t* b, uint32_t* out, size_t cnt) {
  for (size_t i = 0; i < cnt; i++) out[i] = oracle_gf_mul_slow(w, a[i], b[i]);
}

void oracle_ring_mul_vec(int n, const uint32_t* a, const uint32_t* b, uint32_t* out, size_t cnt) {
  for (size_t i = 0; i < cnt; i++) out[i] = oracle_ring_mul(n, a[i], b[i]);
}

void oracle_poly_mod_vec(uint64_t p, const uint32_t* a, uint32_t* out, size_t cnt) {
  for (size_t i = 0; i < cnt; i++) out[i] = (uint32_t)oracle_poly_mod(a[i], p);
}

/* ------------------------------------------------------------------------------------------ */
/* Weight-optimised generalized Cauchy generator (Sec. 3 names "generalized Cauchy matrices"   */
/* and Sec. 2.2 makes the coding cost the number of ones of the sparse representatives)       */
/* ------------------------------------------------------------------------------------------ */

/* wt[u] = number of ones of phi_S(u), for every u < 2^w: the fewest ones over all ring elements
 * r with r mod p = u, in one pass over the 2^n ring elements. */
static void sparse_weights(int w, int n, int* wt) {
  uint64_t p = oracle_field_poly(w);
  for (uint32_t u = 0; u < (1u << w); u++) wt[u] = 99;
  for (uint32_t r = 0; r < (1u << n); r++) {
    uint32_t u = (uint32_t)oracle_poly_mod(r, p);
    int c = popcount32(r);
    if (c < wt[u]) wt[u] = c;
  }
}

/* The generator [I_k ; C'] with C'[i][j] = a_i b_j / (x_i + y_j), x_i = k + i, y_j = j: scaling
 * the rows and columns of a Cauchy matrix by nonzero elements keeps every square submatrix
 * nonsingular, so the code stays MDS. The scalings minimise the total weight of phi_S over C' by
 * coordinate descent: starting from a = b = 1, each round sets every b_j (j ascending), then
 * every a_i (i ascending), to the element of 1..2^w-1 that minimises the weight summed over its
 * column (row) -- the smallest such element on ties -- and the rounds stop when one changes
 * nothing, or after 8. weights[0] / weights[1]: total weight before and after. */
int oracle_cauchy_weighted(int w, int k, int m, uint32_t* G, uint64_t* weights) {
  if (k < 1 || m < 0 || k > ORACLE_MAX_K || w < 2 || w > ORACLE_MAX_W) return -2;
  if ((uint64_t)k + (uint64_t)m > ((uint64_t)1 << w)) return -2;
  gf_t f;
  if (gf_init(&f, w)) {
    gf_free(&f);
    return -1;
  }
  const int n = oracle_ring_size(w);
  const uint32_t q = 1u << w;
  int* wt = (int*)malloc(sizeof(int) * q);
  uint32_t* c = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1) * (size_t)k);
  uint32_t a[64], b[64];
  if (!wt || !c || m > 64) {
    free(wt);
    free(c);
    gf_free(&f);
    return -1;
  }
  sparse_weights(w, n, wt);
  for (int i = 0; i < m; i++)
    for (int j = 0; j < k; j++) c[i * k + j] = gf_inv(&f, (uint32_t)(k + i) ^ (uint32_t)j);
  for (int i = 0; i < m; i++) a[i] = 1;
  for (int j = 0; j < k; j++) b[j] = 1;
  uint64_t w0 = 0;
  for (int i = 0; i < m; i++)
    for (int j = 0; j < k; j++) w0 += (uint64_t)wt[c[i * k + j]];
  for (int round = 0; round < 8; round++) {
    int changed = 0;
    for (int j = 0; j < k; j++) {
      uint32_t best = 0;
      long bw = -1;
      for (uint32_t s = 1; s < q; s++) {
        long sum = 0;
        for (int i = 0; i < m; i++) sum += wt[gf_mul(&f, gf_mul(&f, a[i], s), c[i * k + j])];
        if (bw < 0 || sum < bw) {
          bw = sum;
          best = s;
        }
      }
      if (best != b[j]) changed = 1;
      b[j] = best;
    }
    for (int i = 0; i < m; i++) {
      uint32_t best = 0;
      long bw = -1;
      for (uint32_t s = 1; s < q; s++) {
        long sum = 0;
        for (int j = 0; j < k; j++) sum += wt[gf_mul(&f, gf_mul(&f, s, b[j]), c[i * k + j])];
        if (bw < 0 || sum < bw) {
          bw = sum;
          best = s;
        }
      }
      if (best != a[i]) changed = 1;
      a[i] = best;
    }
    if (!changed) break;
  }
  uint64_t w1 = 0;
  for (int r = 0; r < k; r++)
    for (int cc = 0; cc < k; cc++) G[r * k + cc] = (r == cc);
  for (int i = 0; i < m; i++)
    for (int j = 0; j < k; j++) {
      uint32_t v = gf_mul(&f, gf_mul(&f, a[i], b[j]), c[i * k + j]);
      G[(k + i) * k + j] = v;
      w1 += (uint64_t)wt[v];
    }
  if (weights) {
    weights[0] = w0;
    weights[1] = w1;
  }
  free(wt);
  free(c);
  gf_free(&f);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* The parity transform (Sec. 2.3.1), written literally in the ring                            */
/* ------------------------------------------------------------------------------------------ */

/* phi_P pads a field element b with parity bits so that it lands in the ideal A_1. For an AOP
 * (n = w + 1) one bit, the parity of b, at x^w (Sec. 2.3.1); for the ESP p(x^s) of degree w = s r
 * (n = s (r + 1)) one bit per interleaved word: coefficient w + j is the parity of the
 * coefficients j, j + s, ..., j + (r-1) s of b (Sec. 2.4.1; s = 1 is the AOP case). phi_P^{-1}
 * drops the n - w top coefficients. */
static uint32_t phi_P(int w, int n, uint32_t b) {
  const int s = n - w;
  uint32_t r = b;
  for (int j = 0; j < s; j++) {
    uint32_t par = 0;
    for (int q = j; q < w; q += s) par ^= (b >> q) & 1u;
    r |= par << (w + j);
  }
  return r;
}
static uint32_t phi_P_inv(int w, uint32_t r) { return r & ((1u << w) - 1); }

/* phi_P as an export for the tests. */
uint32_t oracle_phi_P(int w, int n, uint32_t b) { return phi_P(w, n, b); }

typedef struct {
  int w, n, k, nout;
  const uint32_t* R;     /* nout x k ring masks (phi_S of the coefficients) */
  const int* src;        /* block index of source s */
  const int* dst;        /* block index of output o */
  uint8_t* blocks;       /* all blocks, contiguous */
  size_t P, t0, t1;
} pt_job_t;

/* out_o = phi_P^{-1}( sum_s R[o][s] * phi_P(y_s) ) in R_{2,n}, symbol lane by symbol lane. */
static void* pt_run(void* arg) {
  pt_job_t* J = (pt_job_t*)arg;
  const int w = J->w, n = J->n;
  size_t blk = (size_t)w * J->P;
  uint32_t y[ORACLE_MAX_K];
  for (size_t t = J->t0; t < J->t1; t++)
    for (int b = 0; b < 8; b++) {
      for (int s = 0; s < J->k; s++) y[s] = phi_P(w, n, gather_symbol(J->blocks + (size_t)J->src[s] * blk, w, J->P, t, b));
      for (int o = 0; o < J->nout; o++) {
        uint32_t acc = 0;
        for (int s = 0; s < J->k; s++) acc ^= oracle_ring_mul(n, J->R[o * J->k + s], y[s]);
        scatter_symbol(J->blocks + (size_t)J->dst[o] * blk, w, J->P, t, b, phi_P_inv(w, acc));
      }
    }
  return NULL;
}

static void pt_code(int w, int n, int k, int nout, const uint32_t* R, const int* src, const int* dst,
                    uint8_t* blocks, size_t P, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if ((size_t)nthreads > P) nthreads = (int)P;
  if (nthreads > 256) nthreads = 256;
  pt_job_t jobs[256];
  for (int i = 0; i < nthreads; i++)
    jobs[i] = (pt_job_t){w, n, k, nout, R, src, dst, blocks, P, P * (size_t)i / (size_t)nthreads,
                         P * (size_t)(i + 1) / (size_t)nthreads};
  run_threads(pt_run, jobs, sizeof(pt_job_t), nthreads);
}

/* Encoding with the parity transform (both encoder and decoder must use it, Sec. 2.3.1).
 * blocks: k+m blocks of w*P bytes, contiguous; the m parity blocks are written.
 * Returns 0, -1 unsupported field, -3 bad sizes. */
int oracle_encode_pt(int w, int k, int m, const uint32_t* G, uint8_t* blocks, size_t P, int nthreads) {
  if (k < 1 || k > ORACLE_MAX_K || m < 0 || m > 64 || P == 0) return -3;
  const int n = oracle_ring_size(w);
  if (!n) return -1;
  uint32_t* R = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1) * (size_t)k);
  int src[ORACLE_MAX_K], dst[64];
  for (int i = 0; i < m; i++)
    for (int j = 0; j < k; j++) R[i * k + j] = oracle_sparse_rep(w, n, G[(k + i) * k + j]);
  for (int j = 0; j < k; j++) src[j] = j;
  for (int i = 0; i < m; i++) dst[i] = k + i;
  pt_code(w, n, k, m, R, src, dst, blocks, P, nthreads);
  free(R);
  return 0;
}

/* Decoding with the parity transform: the erased blocks (bit e of `erased`) are rebuilt from the
 * first k survivors with the pattern's decoding matrix (erased data e: row e of the survivors'
 * inverse; erased parity e: G[e] times it), each coefficient through phi_S as in encoding.
 * Returns 0, -1 unsupported field, -3 bad sizes, -4 too many erasures, -5 singular. */
int oracle_decode_pt(int w, int k, int m, const uint32_t* G, uint8_t* blocks, uint64_t erased, size_t P,
                     int nthreads) {
  if (k < 1 || k > ORACLE_MAX_K || m < 0 || k + m > 64 || P == 0) return -3;
  if ((erased >> (k + m)) != 0 && k + m < 64) return -3;
  int ne = 0, er[64], surv[ORACLE_MAX_K], ns = 0;
  for (int e = 0; e < k + m; e++) {
    if ((erased >> e) & 1)
      er[ne++] = e;
    else if (ns < k)
      surv[ns++] = e;
  }
  if (ne > m) return -4;
  if (ne == 0) return 0;
  gf_t f;
  if (gf_init(&f, w)) {
    gf_free(&f);
    return -1;
  }
  const int n = oracle_ring_size(w);
  uint32_t* Gs = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)k * (size_t)k);
  uint32_t* Inv = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)k * (size_t)k);
  uint32_t* R = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)ne * (size_t)k);
  for (int s = 0; s < k; s++)
    for (int c = 0; c < k; c++) Gs[s * k + c] = G[surv[s] * k + c];
  int rc = gf_invert(&f, k, Gs, Inv) == 0 ? 0 : -5;
  if (rc == 0) {
    for (int r = 0; r < ne; r++)
      for (int s = 0; s < k; s++) {
        uint32_t v = 0;
        if (er[r] < k) {
          v = Inv[er[r] * k + s];
        } else {
          for (int j = 0; j < k; j++) v ^= gf_mul(&f, G[er[r] * k + j], Inv[j * k + s]);
        }
        R[r * k + s] = oracle_sparse_rep(w, n, v);
      }
    pt_code(w, n, k, ne, R, surv, er, blocks, P, nthreads);
  }
  free(Gs);
  free(Inv);
  free(R);
  gf_free(&f);
  return rc;
}
