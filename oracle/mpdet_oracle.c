/*
 * CPU oracle for fixed-precision multiprecision Gaussian elimination.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the GPU library computes. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Number format (the method fixes a p-bit working precision, Sec. 4.3):
 *   x = (-1)^s * m * 2^(e - p),  m an integer in [2^(p-1), 2^p) held as
 *   n = p/32 little-endian uint32 limbs, e an int64.  Zero is +0:
 *   s = 0, m = 0, e = INT64_MIN.  No infinities, no NaN.
 * Every operation returns the exact result rounded to nearest, ties to even,
 * at p bits: RN(a*b), RN(a+b), RN(a-b), RN(1/a).  The one rounding routine
 * `rnd` below is used by all of them.
 *
 * Elimination (Sec. 3, "Gauss elimination without pivoting"; Alg. 1 read as
 * in the text that surrounds it, the augmented matrix [A I]):
 *   for k = 1..N:
 *     D_k = RN(D_{k-1} * a_kk), D_0 = 1             (Alg. 1 step 2.1)
 *     stop if a_kk == 0 and k < N
 *     r_k = RN(1 / a_kk)
 *     z_ik = RN(a_ik * r_k),  i > k                  (Alg. 1 step 2.2.1)
 *     a_ij = RN(a_ij - RN(z_ik * a_kj)),  i > k, j > k   (step 2.2.2)
 *   In "lastcol" mode the same row operation is applied to the identity
 *   block of [A I], whose non-zero part is stored in A's strict lower
 *   triangle (Sec. 3, storage in N^2 + O(N)):
 *     l_ij = RN(l_ij - RN(z_ik * l_kj)),  i > k, j < k
 *     l_ik = -z_ik   (exact)
 *   The signed minors of the last column (eq. minorsdef) are then
 *     C_jN = RN(D_{N-1} * l_Nj) (j < N),  C_NN = D_{N-1}.
 *
 * Adjoint.  All (N-1) x (N-1) minors are partial derivatives of the
 * determinant (Sec. 3, the Strassen argument), so d log|det| / dA = A^-T.
 * With L A = U from the lastcol elimination, A^-1 = U^-1 L, solved by back
 * substitution in right-looking order (rows from the bottom up):
 *     S = L (unit diagonal, zeros above it)
 *     for k = N..1:  X_kc = RN(S_kc * RN(1/u_kk)),  all c
 *                    S_ic = RN(S_ic - RN(u_ik * X_kc)),  i < k, all c
 * and each X_ji is rounded to binary64 (nearest even, subnormals included).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <math.h>

#define ZEXP INT64_MIN

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EZEROPIVOT = 4, OR_EZERODIV = 7 };

/* ------------------------------------------------------------------------- */
/* Plain big-integer helpers on little-endian uint32 limb arrays.            */
/* ------------------------------------------------------------------------- */

/* Number of significant bits of x (0 for x == 0). */
static int64_t bitlen(const uint32_t *x, int L) {
  for (int i = L - 1; i >= 0; --i)
    if (x[i]) return (int64_t)i * 32 + (32 - __builtin_clz(x[i]));
  return 0;
}

static int getbit(const uint32_t *x, int L, int64_t i) {
  if (i < 0 || i >= (int64_t)L * 32) return 0;
  return (x[i >> 5] >> (i & 31)) & 1u;
}

/* 1 if any bit of x with index < i is set. */
static int anybelow(const uint32_t *x, int L, int64_t i) {
  if (i <= 0) return 0;
  if (i > (int64_t)L * 32) i = (int64_t)L * 32;
  int64_t full = i >> 5;
  for (int64_t w = 0; w < full; ++w)
    if (x[w]) return 1;
  int rem = (int)(i & 31);
  if (rem && (x[full] & ((1u << rem) - 1u))) return 1;
  return 0;
}

/* out[0..Lo) = floor(x / 2^sh) truncated to Lo limbs (sh >= 0). */
static void shr(const uint32_t *x, int L, int64_t sh, uint32_t *out, int Lo) {
  int64_t q = sh >> 5;
  int r = (int)(sh & 31);
  for (int i = 0; i < Lo; ++i) {
    int64_t s = i + q;
    uint64_t lo = (s < L) ? x[s] : 0;
    uint64_t hi = (s + 1 < L) ? x[s + 1] : 0;
    out[i] = (uint32_t)(((hi << 32) | lo) >> r);
  }
}

/* out[0..Lo) = (x * 2^sh) truncated to Lo limbs (sh >= 0). */
static void shl(const uint32_t *x, int L, int64_t sh, uint32_t *out, int Lo) {
  int64_t q = sh >> 5;
  int r = (int)(sh & 31);
  for (int i = 0; i < Lo; ++i) {
    int64_t s = i - q;
    uint64_t cur = (s >= 0 && s < L) ? x[s] : 0;
    uint64_t low = (s - 1 >= 0 && s - 1 < L) ? x[s - 1] : 0;
    uint64_t v = (cur << r) | (r ? (low >> (32 - r)) : 0);
    out[i] = (uint32_t)v;
  }
}

/* -1, 0, +1 comparing two L-limb integers. */
static int cmpn(const uint32_t *a, const uint32_t *b, int L) {
  for (int i = L - 1; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  }
  return 0;
}

/* a += b (L limbs), returns carry. */
static uint32_t addn(uint32_t *a, const uint32_t *b, int L) {
  uint64_t c = 0;
  for (int i = 0; i < L; ++i) {
    c += (uint64_t)a[i] + b[i];
    a[i] = (uint32_t)c;
    c >>= 32;
  }
  return (uint32_t)c;
}

/* a -= b (L limbs), returns borrow. */
static uint32_t subn(uint32_t *a, const uint32_t *b, int L) {
  int64_t br = 0;
  for (int i = 0; i < L; ++i) {
    int64_t d = (int64_t)a[i] - (int64_t)b[i] - br;
    br = d < 0;
    a[i] = (uint32_t)(d + (br ? ((int64_t)1 << 32) : 0));
  }
  return (uint32_t)br;
}

/* r[0..2n) = a * b, schoolbook. */
static void muln(const uint32_t *a, const uint32_t *b, int n, uint32_t *r) {
  memset(r, 0, sizeof(uint32_t) * 2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    uint64_t c = 0;
    for (int j = 0; j < n; ++j) {
      uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + c;
      r[i + j] = (uint32_t)t;
      c = t >> 32;
    }
    r[i + n] = (uint32_t)c;
  }
}

/* ------------------------------------------------------------------------- */
/* The one rounding routine.                                                 */
/* Rounds the non-negative exact value (X + f) * 2^E to p bits, where X is an */
/* L-limb integer and f is a fraction in (0,1) when sticky_in is set, else 0. */
/* sticky_in requires bitlen(X) > p, so that the round bit lies inside X.     */
/* Writes mantissa (n limbs), exponent and sign s.  X == 0 gives +0.          */
/* ------------------------------------------------------------------------- */
static void rnd(const uint32_t *X, int L, int64_t E, int sticky_in, int p, int n, int s, int8_t *os,
                int64_t *oe, uint32_t *om) {
  int64_t t = bitlen(X, L);
  if (t == 0) {
    *os = 0;
    *oe = ZEXP;
    memset(om, 0, sizeof(uint32_t) * n);
    return;
  }
  if (t <= p) { /* exact: X fits in p bits (sticky_in must be 0 here) */
    shl(X, L, p - t, om, n);
    *os = (int8_t)s;
    *oe = t + E;
    return;
  }
  int64_t sh = t - p;
  shr(X, L, sh, om, n);
  int rbit = getbit(X, L, sh - 1);
  int st = anybelow(X, L, sh - 1) || sticky_in;
  if (rbit && (st || (om[0] & 1u))) {
    uint64_t c = 1;
    for (int i = 0; i < n && c; ++i) {
      c += om[i];
      om[i] = (uint32_t)c;
      c >>= 32;
    }
    if (c) { /* mantissa overflowed to 2^p: renormalise to 2^(p-1) */
      memset(om, 0, sizeof(uint32_t) * n);
      om[n - 1] = 0x80000000u;
      t += 1;
    }
  }
  *os = (int8_t)s;
  *oe = t + E;
}

/* ------------------------------------------------------------------------- */
/* Operations on numbers.                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
  int p, n;
  uint32_t *buf; /* scratch, 6n+8 limbs */
} ctx_t;

static int iszero(int64_t e) { return e == ZEXP; }

static void setzero(int8_t *s, int64_t *e, uint32_t *m, int n) {
  *s = 0;
  *e = ZEXP;
  memset(m, 0, sizeof(uint32_t) * n);
}

static void copynum(int8_t s, int64_t e, const uint32_t *m, int n, int8_t *os, int64_t *oe, uint32_t *om) {
  *os = s;
  *oe = e;
  if (om != m) memmove(om, m, sizeof(uint32_t) * n);
}

/* RN(a * b) */
static void op_mul(ctx_t *c, int8_t sa, int64_t ea, const uint32_t *ma, int8_t sb, int64_t eb, const uint32_t *mb,
                   int8_t *os, int64_t *oe, uint32_t *om) {
  int n = c->n, p = c->p;
  if (iszero(ea) || iszero(eb)) {
    setzero(os, oe, om, n);
    return;
  }
  uint32_t *X = c->buf; /* 2n limbs */
  muln(ma, mb, n, X);
  /* a*b = ma*mb * 2^(ea+eb-2p) */
  rnd(X, 2 * n, ea + eb - 2 * (int64_t)p, 0, p, n, (sa ^ sb) & 1, os, oe, om);
}

/* RN(a + (-1)^negb * b) */
static void op_add(ctx_t *c, int8_t sa, int64_t ea, const uint32_t *ma, int8_t sb0, int64_t eb, const uint32_t *mb,
                   int negb, int8_t *os, int64_t *oe, uint32_t *om) {
  int n = c->n, p = c->p;
  int sb = (sb0 ^ negb) & 1;
  if (iszero(eb)) {
    if (iszero(ea)) setzero(os, oe, om, n);
    else copynum(sa, ea, ma, n, os, oe, om);
    return;
  }
  if (iszero(ea)) {
    copynum((int8_t)sb, eb, mb, n, os, oe, om);
    return;
  }
  /* Order by magnitude: |A| >= |B|. */
  int swap = (eb > ea) || (eb == ea && cmpn(mb, ma, n) > 0);
  int8_t sA = swap ? (int8_t)sb : sa, sB = swap ? sa : (int8_t)sb;
  int64_t eA = swap ? eb : ea, eB = swap ? ea : eb;
  const uint32_t *mA = swap ? mb : ma, *mB = swap ? ma : mb;
  int64_t d = eA - eB; /* >= 0 */
  if (d >= (int64_t)p + 2) {
    /* |B| < 2^eB <= 2^(eA-p-2) = ulp(A)/4.  A +- B lies strictly within a
       quarter ulp of A (within half an ulp of the finer binade below A when
       A is a power of two), so RN returns A. */
    copynum(sA, eA, mA, n, os, oe, om);
    return;
  }
  /* Exact: X = mA*2^d +- mB, value = X * 2^(eB-p); X < 2^(p+d+1) <= 2^(2p+2). */
  int L = 2 * n + 2;
  uint32_t *X = c->buf, *Y = c->buf + L;
  shl(mA, n, d, X, L);
  memset(Y, 0, sizeof(uint32_t) * L);
  memcpy(Y, mB, sizeof(uint32_t) * n);
  if (sA == sB) addn(X, Y, L);
  else subn(X, Y, L); /* X >= Y since |A| >= |B| */
  rnd(X, L, eB - p, 0, p, n, sA, os, oe, om);
}

/* RN(1 / a); returns OR_EZERODIV for a == 0. */
static int op_recip(ctx_t *c, int8_t sa, int64_t ea, const uint32_t *ma, int8_t *os, int64_t *oe, uint32_t *om) {
  int n = c->n, p = c->p;
  if (iszero(ea)) return OR_EZERODIV;
  /* 2^(2p) = q*m + r by restoring binary long division, q < 2^(p+2). */
  int L = n + 2;
  uint32_t *q = c->buf, *r = c->buf + L, *m = c->buf + 2 * L;
  memset(q, 0, sizeof(uint32_t) * L);
  memset(r, 0, sizeof(uint32_t) * L);
  memset(m, 0, sizeof(uint32_t) * L);
  memcpy(m, ma, sizeof(uint32_t) * n);
  for (int64_t i = 2 * (int64_t)p; i >= 0; --i) {
    /* r = 2r + (bit i of 2^(2p)) */
    uint32_t carry = (i == 2 * (int64_t)p) ? 1u : 0u;
    for (int w = 0; w < L; ++w) {
      uint32_t nc = r[w] >> 31;
      r[w] = (r[w] << 1) | carry;
      carry = nc;
    }
    if (cmpn(r, m, L) >= 0) {
      subn(r, m, L);
      if (i < (int64_t)L * 32) q[i >> 5] |= 1u << (i & 31);
    }
  }
  int rem_nz = bitlen(r, L) != 0;
  /* 1/a = 2^(p-ea)/ma = (q + r/ma) * 2^(-p-ea); q > 2^p has > p bits. */
  rnd(q, L, -(int64_t)p - ea, rem_nz, p, n, sa & 1, os, oe, om);
  return OR_OK;
}

/* RN(a / b) with one rounding (the correctly rounded division that the
 * elimination's default two-rounding multiplier RN(a * RN(1/b)) stands in
 * for); OR_EZERODIV for b == 0. */
static int op_div(ctx_t *c, int8_t sa, int64_t ea, const uint32_t *ma, int8_t sb, int64_t eb, const uint32_t *mb,
                  int8_t *os, int64_t *oe, uint32_t *om) {
  int n = c->n, p = c->p;
  if (iszero(eb)) return OR_EZERODIV;
  if (iszero(ea)) {
    setzero(os, oe, om, n);
    return OR_OK;
  }
  /* ma * 2^(p+1) = q*mb + r by restoring binary long division, 2^p < q < 2^(p+2). */
  int L = n + 2;
  uint32_t *q = c->buf, *r = c->buf + L, *m = c->buf + 2 * L;
  memset(q, 0, sizeof(uint32_t) * L);
  memset(r, 0, sizeof(uint32_t) * L);
  memset(m, 0, sizeof(uint32_t) * L);
  memcpy(m, mb, sizeof(uint32_t) * n);
  for (int64_t i = 2 * (int64_t)p; i >= 0; --i) {
    /* r = 2r + (bit i of ma * 2^(p+1)), i.e. bit i - p - 1 of ma */
    int64_t src = i - (int64_t)p - 1;
    uint32_t carry = (src >= 0) ? ((ma[src >> 5] >> (src & 31)) & 1u) : 0u;
    for (int w = 0; w < L; ++w) {
      uint32_t nc = r[w] >> 31;
      r[w] = (r[w] << 1) | carry;
      carry = nc;
    }
    if (cmpn(r, m, L) >= 0) {
      subn(r, m, L);
      if (i < (int64_t)L * 32) q[i >> 5] |= 1u << (i & 31);
    }
  }
  int rem_nz = bitlen(r, L) != 0;
  /* a/b = (ma/mb) * 2^(ea-eb) = (q + r/mb) * 2^(ea - eb - p - 1) */
  rnd(q, L, ea - eb - (int64_t)p - 1, rem_nz, p, n, (sa ^ sb) & 1, os, oe, om);
  return OR_OK;
}


/* Exact lift of a double (finite) to p bits, p >= 64. */
static void op_from_f64(ctx_t *c, double v, int8_t *os, int64_t *oe, uint32_t *om) {
  int n = c->n, p = c->p;
  if (v == 0.0) {
    setzero(os, oe, om, n);
    return;
  }
  uint64_t bits;
  memcpy(&bits, &v, 8);
  int s = (int)(bits >> 63);
  int bexp = (int)((bits >> 52) & 0x7ff);
  uint64_t frac = bits & ((1ull << 52) - 1);
  uint64_t M;
  int64_t E;
  if (bexp == 0) { /* subnormal */
    M = frac;
    E = -1074;
  } else {
    M = frac | (1ull << 52);
    E = bexp - 1075;
  }
  uint32_t X[2] = {(uint32_t)M, (uint32_t)(M >> 32)};
  rnd(X, 2, E, 0, p, n, s, os, oe, om);
}

static void op_from_i64(ctx_t *c, int64_t v, int8_t *os, int64_t *oe, uint32_t *om) {
  int n = c->n, p = c->p;
  if (v == 0) {
    setzero(os, oe, om, n);
    return;
  }
  int s = v < 0;
  uint64_t M = s ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
  uint32_t X[2] = {(uint32_t)M, (uint32_t)(M >> 32)};
  rnd(X, 2, 0, 0, p, n, s, os, oe, om);
}

/* ------------------------------------------------------------------------- */
/* Exported element-wise operations on SoA arrays (count elements each).      */
/* ------------------------------------------------------------------------- */
static int ctx_init(ctx_t *c, int p) {
  if (p < 64 || p % 32) return OR_EINVAL;
  c->p = p;
  c->n = p / 32;
  c->buf = (uint32_t *)calloc((size_t)6 * c->n + 16, sizeof(uint32_t));
  return c->buf ? OR_OK : OR_ENOMEM;
}

int or_div_v(int64_t cnt, int p, const int8_t *as, const int64_t *ae, const uint32_t *am, const int8_t *bs,
             const int64_t *be, const uint32_t *bm, int8_t *os, int64_t *oe, uint32_t *om) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  int n = c.n;
  for (int64_t i = 0; i < cnt && st == OR_OK; ++i)
    st = op_div(&c, as[i], ae[i], am + i * n, bs[i], be[i], bm + i * n, os + i, oe + i, om + i * n);
  free(c.buf);
  return st;
}

int or_mul_v(int64_t cnt, int p, const int8_t *sa, const int64_t *ea, const uint32_t *ma, const int8_t *sb,
             const int64_t *eb, const uint32_t *mb, int8_t *so, int64_t *eo, uint32_t *mo) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  int n = c.n;
  for (int64_t i = 0; i < cnt; ++i)
    op_mul(&c, sa[i], ea[i], ma + i * n, sb[i], eb[i], mb + i * n, so + i, eo + i, mo + i * n);
  free(c.buf);
  return OR_OK;
}

int or_add_v(int64_t cnt, int p, int negb, const int8_t *sa, const int64_t *ea, const uint32_t *ma, const int8_t *sb,
             const int64_t *eb, const uint32_t *mb, int8_t *so, int64_t *eo, uint32_t *mo) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  int n = c.n;
  for (int64_t i = 0; i < cnt; ++i)
    op_add(&c, sa[i], ea[i], ma + i * n, sb[i], eb[i], mb + i * n, negb, so + i, eo + i, mo + i * n);
  free(c.buf);
  return OR_OK;
}

int or_recip_v(int64_t cnt, int p, const int8_t *sa, const int64_t *ea, const uint32_t *ma, int8_t *so, int64_t *eo,
               uint32_t *mo) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  int n = c.n;
  for (int64_t i = 0; i < cnt && st == OR_OK; ++i) st = op_recip(&c, sa[i], ea[i], ma + i * n, so + i, eo + i, mo + i * n);
  free(c.buf);
  return st;
}

int or_from_f64_v(int64_t cnt, int p, const double *v, int8_t *so, int64_t *eo, uint32_t *mo) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  for (int64_t i = 0; i < cnt; ++i) op_from_f64(&c, v[i], so + i, eo + i, mo + i * c.n);
  free(c.buf);
  return OR_OK;
}

int or_from_i64_v(int64_t cnt, int p, const int64_t *v, int8_t *so, int64_t *eo, uint32_t *mo) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  for (int64_t i = 0; i < cnt; ++i) op_from_i64(&c, v[i], so + i, eo + i, mo + i * c.n);
  free(c.buf);
  return OR_OK;
}

/* One Cauchy entry: s = RN(x + y) into (ts, te, tm), then RN(1 / s) into
 * (so, eo, mo); x and y are lifted exactly.  xm, ym: n-limb scratch. */
static int cauchy_entry(ctx_t *c, double x, double y, uint32_t *xm, uint32_t *ym, int8_t *ts, int64_t *te,
                        uint32_t *tm, int8_t *so, int64_t *eo, uint32_t *mo) {
  int8_t xs, ys;
  int64_t xe, ye;
  op_from_f64(c, x, &xs, &xe, xm);
  op_from_f64(c, y, &ys, &ye, ym);
  op_add(c, xs, xe, xm, ys, ye, ym, 0, ts, te, tm);
  return op_recip(c, *ts, *te, tm, so, eo, mo);
}

/* Cauchy matrix A_ij = RN(1 / RN(x_i + y_j)), x_i and y_j lifted exactly. */
int or_cauchy(int64_t N, int p, const double *x, const double *y, int8_t *so, int64_t *eo, uint32_t *mo) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  int n = c.n;
  uint32_t *tm = (uint32_t *)calloc((size_t)3 * n, sizeof(uint32_t));
  uint32_t *xm = tm + n, *ym = tm + 2 * n;
  for (int64_t i = 0; i < N && st == OR_OK; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      int8_t ts;
      int64_t te, idx = i * N + j;
      st = cauchy_entry(&c, x[i], y[j], xm, ym, &ts, &te, tm, so + idx, eo + idx, mo + idx * n);
      if (st) break;
    }
  }
  free(tm);
  free(c.buf);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Gaussian elimination without pivoting, in place, with a row-parallel      */
/* thread pool (the rows of one step are independent; splitting them among   */
/* threads does not change any result, as in the paper's pthread scheme).     */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t N;
  int p, n, lastcol;
  int8_t *S;
  int64_t *E;
  uint32_t *M;
  /* current step data */
  int64_t k;
  int8_t *zs;
  int64_t *ze;
  uint32_t *zm;
} ge_t;

typedef struct {
  ge_t *g;
  int64_t i0, i1;
  int err;
} work_t;

static void *update_rows(void *arg) {
  work_t *w = (work_t *)arg;
  ge_t *g = w->g;
  ctx_t c;
  if (ctx_init(&c, g->p)) {
    w->err = OR_ENOMEM;
    return NULL;
  }
  int n = g->n;
  int64_t N = g->N, k = g->k;
  uint32_t *t = (uint32_t *)calloc(n, sizeof(uint32_t));
  for (int64_t i = w->i0; i < w->i1; ++i) {
    int64_t zi = i - (k + 1);
    int8_t zs = g->zs[zi];
    int64_t ze = g->ze[zi];
    const uint32_t *zm = g->zm + zi * n;
    for (int64_t j = g->lastcol ? 0 : k + 1; j < N; ++j) {
      if (j == k) continue;
      int64_t ij = i * N + j, kj = k * N + j;
      int8_t ts;
      int64_t te;
      op_mul(&c, zs, ze, zm, g->S[kj], g->E[kj], g->M + kj * n, &ts, &te, t);
      op_add(&c, g->S[ij], g->E[ij], g->M + ij * n, ts, te, t, 1, g->S + ij, g->E + ij, g->M + ij * n);
    }
    if (g->lastcol) { /* l_ik = -z_ik, exact; +0 stays +0 */
      int64_t ik = i * N + k;
      int8_t s = iszero(ze) ? 0 : (int8_t)(zs ^ 1);
      copynum(s, ze, zm, n, g->S + ik, g->E + ik, g->M + ik * n);
    }
  }
  free(t);
  free(c.buf);
  return NULL;
}

/*
 * In-place elimination of the N x N row-major matrix (S, E, M) at p bits.
 * D (N numbers) receives the leading minors D_1..D_N.  *zero_k receives the
 * 1-based index of the first exactly zero pivot (0 if none).  Returns
 * OR_EZEROPIVOT when that pivot is at k < N (elimination stopped, D_k..D_N
 * are +0), else OR_OK.  k_end limits the steps run (k_end = N for all):
 * steps k0+1..k_end are run, with D holding D_1..D_k0 on entry.
 */
static int ge_range(int64_t N, int p, int lastcol, int nthreads, int64_t k0, int64_t k_end, int8_t *S, int64_t *E,
                    uint32_t *M, int8_t *Ds, int64_t *De, uint32_t *Dm, int64_t *zero_k, int divide) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  if (N < 1 || k0 < 0 || k_end > N || k0 > k_end) {
    free(c.buf);
    return OR_EINVAL;
  }
  if (nthreads < 1) nthreads = 1;
  int n = c.n;
  ge_t g = {N, p, n, lastcol, S, E, M, 0, NULL, NULL, NULL};
  g.zs = (int8_t *)calloc(N, 1);
  g.ze = (int64_t *)calloc(N, sizeof(int64_t));
  g.zm = (uint32_t *)calloc((size_t)N * n, sizeof(uint32_t));
  uint32_t *r = (uint32_t *)calloc(n, sizeof(uint32_t));
  uint32_t *one = (uint32_t *)calloc(n, sizeof(uint32_t));
  one[n - 1] = 0x80000000u; /* 1 = 2^(p-1) * 2^(1-p) */
  pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
  work_t *wk = (work_t *)calloc(nthreads, sizeof(work_t));
  if (zero_k) *zero_k = 0;
  for (int64_t k = k0; k < k_end; ++k) { /* 0-based step k = paper's k+1 */
    int64_t kk = k * N + k;
    /* D_k = RN(D_{k-1} * a_kk), D_0 = 1 */
    if (k == 0) op_mul(&c, 0, 1, one, S[kk], E[kk], M + kk * n, Ds, De, Dm);
    else op_mul(&c, Ds[k - 1], De[k - 1], Dm + (k - 1) * n, S[kk], E[kk], M + kk * n, Ds + k, De + k, Dm + k * n);
    if (iszero(E[kk])) {
      if (zero_k) *zero_k = k + 1;
      for (int64_t q = k; q < N; ++q) setzero(Ds + q, De + q, Dm + q * n, n);
      if (k < N - 1) st = OR_EZEROPIVOT;
      break;
    }
    if (k == N - 1) break;
    int8_t rs;
    int64_t re;
    op_recip(&c, S[kk], E[kk], M + kk * n, &rs, &re, r);
    /* multipliers z_ik = RN(a_ik * r_k) (or, as an option for accuracy
     * comparisons, the correctly rounded RN(a_ik / a_kk)) */
    for (int64_t i = k + 1; i < N; ++i) {
      int64_t ik = i * N + k, zi = i - (k + 1);
      if (divide)
        op_div(&c, S[ik], E[ik], M + ik * n, S[kk], E[kk], M + kk * n, g.zs + zi, g.ze + zi, g.zm + zi * n);
      else
        op_mul(&c, S[ik], E[ik], M + ik * n, rs, re, r, g.zs + zi, g.ze + zi, g.zm + zi * n);
    }
    g.k = k;
    int64_t rows = N - (k + 1);
    int T = nthreads;
    if (T > rows) T = (int)rows;
    for (int t = 0; t < T; ++t) {
      wk[t].g = &g;
      wk[t].i0 = k + 1 + rows * t / T;
      wk[t].i1 = k + 1 + rows * (t + 1) / T;
      wk[t].err = 0;
    }
    if (T == 1) update_rows(&wk[0]);
    else {
      for (int t = 0; t < T; ++t) pthread_create(&th[t], NULL, update_rows, &wk[t]);
      for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
    }
    for (int t = 0; t < T; ++t)
      if (wk[t].err) st = wk[t].err;
    if (st) break;
  }
  free(wk);
  free(th);
  free(one);
  free(r);
  free(g.zm);
  free(g.ze);
  free(g.zs);
  free(c.buf);
  return st;
}

int or_ge_range(int64_t N, int p, int lastcol, int nthreads, int64_t k0, int64_t k_end, int8_t *S, int64_t *E,
                uint32_t *M, int8_t *Ds, int64_t *De, uint32_t *Dm, int64_t *zero_k) {
  return ge_range(N, p, lastcol, nthreads, k0, k_end, S, E, M, Ds, De, Dm, zero_k, 0);
}

/* The same elimination with correctly rounded multipliers z_ik = RN(a_ik /
 * a_kk) (one rounding) instead of RN(a_ik * RN(1/a_kk)): not the method's
 * arithmetic, an option to measure what the two-rounding multiplier costs. */
int or_ge_range_div(int64_t N, int p, int lastcol, int nthreads, int64_t k0, int64_t k_end, int8_t *S, int64_t *E,
                    uint32_t *M, int8_t *Ds, int64_t *De, uint32_t *Dm, int64_t *zero_k) {
  return ge_range(N, p, lastcol, nthreads, k0, k_end, S, E, M, Ds, De, Dm, zero_k, 1);
}

/*
 * Last-column signed minors from an eliminated matrix in lastcol mode:
 *   C_jN = RN(D_{N-1} * l_Nj), j < N;  C_NN = D_{N-1}   (eq. minorsdef)
 * normalised != 0 returns delta_{N,j} = C_jN / C_1N instead (eq. minors),
 * formed as RN(l_Nj * RN(1 / l_N1)) with delta_{N,1} = 1, delta_{N,N} =
 * RN(1 / l_N1).  Dnm1 is D_{N-1} (D_0 = 1 when N == 1).
 */
int or_lastcol(int64_t N, int p, int normalised, const int8_t *S, const int64_t *E, const uint32_t *M, int8_t dsg,
               int64_t dex, const uint32_t *dm, int8_t *os, int64_t *oe, uint32_t *om) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  int n = c.n;
  const int64_t row = (N - 1) * N;
  if (!normalised) {
    for (int64_t j = 0; j + 1 < N; ++j)
      op_mul(&c, dsg, dex, dm, S[row + j], E[row + j], M + (row + j) * n, os + j, oe + j, om + j * n);
    copynum(dsg, dex, dm, n, os + N - 1, oe + N - 1, om + (N - 1) * n);
  } else {
    uint32_t *r = (uint32_t *)calloc(n, sizeof(uint32_t));
    int8_t rs;
    int64_t re;
    if (N == 1) { /* delta_{1,1} = 1 */
      memset(om, 0, sizeof(uint32_t) * n);
      om[n - 1] = 0x80000000u;
      os[0] = 0;
      oe[0] = 1;
    } else {
      st = op_recip(&c, S[row], E[row], M + row * n, &rs, &re, r);
      if (st == OR_OK) {
        memset(om, 0, sizeof(uint32_t) * n);
        om[n - 1] = 0x80000000u;
        os[0] = 0;
        oe[0] = 1;
        for (int64_t j = 1; j + 1 < N; ++j)
          op_mul(&c, S[row + j], E[row + j], M + (row + j) * n, rs, re, r, os + j, oe + j, om + j * n);
        copynum(rs, re, r, n, os + N - 1, oe + N - 1, om + (N - 1) * n);
      }
    }
    free(r);
  }
  free(c.buf);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Adjoint: X = U^-1 L from a lastcol elimination (right-looking back        */
/* substitution in the order stated at the top of this file).                */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t N;
  int p, n;
  const int8_t *US;
  const int64_t *UE;
  const uint32_t *UM; /* eliminated array (U above, L below) */
  int8_t *S;
  int64_t *E;
  uint32_t *M; /* S / X */
  int64_t k;
  int64_t i0, i1;
} us_t;

static void *usolve_rows(void *arg) {
  us_t *u = (us_t *)arg;
  ctx_t c;
  if (ctx_init(&c, u->p)) return NULL;
  int n = u->n;
  int64_t N = u->N, k = u->k;
  uint32_t *t = (uint32_t *)calloc(n, sizeof(uint32_t));
  for (int64_t i = u->i0; i < u->i1; ++i) {
    int64_t ik = i * N + k;
    for (int64_t col = 0; col < N; ++col) {
      int64_t ic = i * N + col, kc = k * N + col;
      int8_t ts;
      int64_t te;
      op_mul(&c, u->US[ik], u->UE[ik], u->UM + ik * n, u->S[kc], u->E[kc], u->M + kc * n, &ts, &te, t);
      op_add(&c, u->S[ic], u->E[ic], u->M + ic * n, ts, te, t, 1, u->S + ic, u->E + ic, u->M + ic * n);
    }
  }
  free(t);
  free(c.buf);
  return NULL;
}

/* X (N*N numbers, row-major) = A^-1 from the lastcol-mode array (S,E,M) of
 * or_ge_range.  Returns OR_EZERODIV if a pivot is zero. */
int or_usolve(int64_t N, int p, int nthreads, const int8_t *S, const int64_t *E, const uint32_t *M, int8_t *XS,
              int64_t *XE, uint32_t *XM) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  int n = c.n;
  if (nthreads < 1) nthreads = 1;
  /* S = L: l_ij below the diagonal, 1 on it, +0 above */
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = 0; j < N; ++j) {
      int64_t ij = i * N + j;
      if (j < i) copynum(S[ij], E[ij], M + ij * n, n, XS + ij, XE + ij, XM + ij * n);
      else if (j == i) {
        setzero(XS + ij, XE + ij, XM + ij * n, n);
        XM[ij * n + n - 1] = 0x80000000u;
        XE[ij] = 1;
      } else setzero(XS + ij, XE + ij, XM + ij * n, n);
    }
  uint32_t *r = (uint32_t *)calloc(n, sizeof(uint32_t));
  pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
  us_t *wk = (us_t *)calloc(nthreads, sizeof(us_t));
  for (int64_t k = N - 1; k >= 0 && st == OR_OK; --k) {
    int64_t kk = k * N + k;
    int8_t rs;
    int64_t re;
    st = op_recip(&c, S[kk], E[kk], M + kk * n, &rs, &re, r);
    if (st) break;
    for (int64_t col = 0; col < N; ++col) { /* X_kc = RN(S_kc * r_k) */
      int64_t kc = k * N + col;
      op_mul(&c, XS[kc], XE[kc], XM + kc * n, rs, re, r, XS + kc, XE + kc, XM + kc * n);
    }
    int T = nthreads;
    if (T > k) T = (int)k;
    for (int t = 0; t < T; ++t) {
      us_t w = {N, p, n, S, E, M, XS, XE, XM, k, k * t / T, k * (t + 1) / T};
      wk[t] = w;
    }
    if (T <= 1) {
      if (k > 0) {
        us_t w = {N, p, n, S, E, M, XS, XE, XM, k, 0, k};
        usolve_rows(&w);
      }
    } else {
      for (int t = 0; t < T; ++t) pthread_create(&th[t], NULL, usolve_rows, &wk[t]);
      for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
    }
  }
  free(wk);
  free(th);
  free(r);
  free(c.buf);
  return st;
}

/* RN to binary64, nearest even, with subnormals and overflow to +-inf.
 * value = m * 2^(e-p) lies in [2^(e-1), 2^e); binary64 keeps multiples of the
 * quantum 2^q, q = max(e - 53, -1074).  K = m * 2^(e-p-q) rounded to an
 * integer (a right shift by p + q - e >= p - 53 bits, the shifted-out bits
 * round); the result is K * 2^q, exact in binary64 (K <= 2^53). */
static double to_f64_one(int p, int n, int8_t s, int64_t e, const uint32_t *m) {
  if (e == ZEXP) return 0.0;
  if (e > 1100) return s ? -HUGE_VAL : HUGE_VAL;
  if (e < -1100) return s ? -0.0 : 0.0;
  int64_t q = (e - 53 < -1074) ? -1074 : e - 53;
  int64_t rs = (int64_t)p + q - e;
  uint32_t buf[2];
  shr(m, n, rs, buf, 2);
  uint64_t K = ((uint64_t)buf[1] << 32) | buf[0];
  int rbit = getbit(m, n, rs - 1);
  int st = anybelow(m, n, rs - 1);
  if (rbit && (st || (K & 1))) K += 1;
  double v = ldexp((double)K, (int)q);
  return s ? -v : v;
}

int or_to_f64_v(int64_t cnt, int p, const int8_t *S, const int64_t *E, const uint32_t *M, double *out) {
  if (p < 64 || p % 32) return OR_EINVAL;
  int n = p / 32;
  for (int64_t i = 0; i < cnt; ++i) out[i] = to_f64_one(p, n, S[i], E[i], M + i * n);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Ball mode: rigorous error bounds beside the method's values.              */
/*                                                                           */
/* The paper leaves rigorous bounds as future work (Sec. 4.4): interval      */
/* arithmetic gives upper and lower bounds at every operation.  Here every   */
/* number x~ of the elimination (computed exactly as above, round to nearest) */
/* carries a radius rho with |x* - x~| <= rho, where x* is the value exact    */
/* arithmetic would give at the same place of the elimination of the exact   */
/* input (midpoint-radius intervals).  Radii are small numbers              */
/*   rho = m * 2^(e - 32),  m in [2^31, 2^32) (or m = 0: rho = 0),           */
/* every radius operation rounds up (down where a lower bound is needed), in  */
/* integer arithmetic only.  e = RAD_INF marks an unbounded radius.          */
/* Rules (u~ = RN(result); hu = half an ulp of u~ at p bits, 2^(e_u - p - 1), */
/* 0 when u~ = 0; |x~|^ and |x~|_ are upper and lower bounds of |x~| from its */
/* top limb):                                                                 */
/*   u~ = RN(x~ y~):  rho_u = ((hu + |x~|^ rho_y) + |y~|^ rho_x) + rho_x rho_y  */
/*   u~ = RN(x~ - t~): rho_u = (hu + rho_x) + rho_t                           */
/*   u~ = RN(1/a~):  rho_u = hu + rho_a / (|a~|_ (|a~|_ - rho_a)),            */
/*                   unbounded unless |a~|_ > rho_a                          */
/*   negation and copies keep the radius.                                    */
/* Exact inputs (lifted doubles and integers) have radius 0.                 */
/* ------------------------------------------------------------------------- */
#define RAD_INF INT64_MAX

typedef struct {
  uint32_t m;
  int64_t e;
} rad_t;

static const rad_t RAD_ZERO = {0, ZEXP};
static const rad_t RAD_UNB = {0xffffffffu, RAD_INF};

static int rad_is_zero(rad_t a) { return a.m == 0; }
static int rad_is_inf(rad_t a) { return a.e == RAD_INF; }

/* the smallest radius >= V * 2^E (up != 0) or the largest <= V * 2^E */
static rad_t rad_from64(uint64_t V, int64_t E, int up) {
  if (!V) return RAD_ZERO;
  int t = 64 - __builtin_clzll(V);
  uint64_t m;
  if (t <= 32) m = V << (32 - t);
  else {
    m = V >> (t - 32);
    if (up && (V & ((1ull << (t - 32)) - 1))) m += 1;
    if (m >> 32) { /* rounded up to 2^32 */
      m >>= 1;
      t += 1;
    }
  }
  rad_t r = {(uint32_t)m, E + t};
  return r;
}

/* b at the scale 2^(ea - 63) (a's), rounded up; d = ea - eb >= 0 */
static uint64_t rad_align_up(rad_t b, int64_t d) {
  if (d <= 31) return (uint64_t)b.m << (31 - d);
  int64_t sh = d - 31;
  if (sh >= 32) return 1; /* 0 < b < one unit of that scale */
  uint64_t v = (uint64_t)b.m >> sh;
  if ((uint64_t)b.m & ((1ull << sh) - 1)) v += 1;
  return v;
}

static rad_t rad_add(rad_t a, rad_t b) {
  if (rad_is_inf(a) || rad_is_inf(b)) return RAD_UNB;
  if (rad_is_zero(a)) return b;
  if (rad_is_zero(b)) return a;
  if (b.e > a.e) {
    rad_t t = a;
    a = b;
    b = t;
  }
  uint64_t A = (uint64_t)a.m << 31;
  return rad_from64(A + rad_align_up(b, a.e - b.e), a.e - 63, 1);
}

static rad_t rad_mul(rad_t a, rad_t b, int up) {
  if (rad_is_zero(a) || rad_is_zero(b)) return RAD_ZERO;
  if (rad_is_inf(a) || rad_is_inf(b)) return RAD_UNB;
  return rad_from64((uint64_t)a.m * b.m, a.e + b.e - 64, up);
}

/* a / b rounded up (b > 0 finite) */
static rad_t rad_div_up(rad_t a, rad_t b) {
  if (rad_is_zero(a)) return RAD_ZERO;
  if (rad_is_inf(a)) return RAD_UNB;
  uint64_t num = (uint64_t)a.m << 32;
  uint64_t q = num / b.m;
  if (q * b.m != num) q += 1;
  return rad_from64(q, a.e - b.e - 32, 1);
}

/* a - b rounded down; *pos = 0 when a - b <= 0 */
static rad_t rad_sub_down(rad_t a, rad_t b, int *pos) {
  *pos = 0;
  if (rad_is_inf(b) || rad_is_zero(a)) return RAD_ZERO;
  if (rad_is_zero(b)) {
    *pos = 1;
    return a;
  }
  if (b.e > a.e) return RAD_ZERO;
  uint64_t A = (uint64_t)a.m << 31, B = rad_align_up(b, a.e - b.e);
  if (B >= A) return RAD_ZERO;
  *pos = 1;
  return rad_from64(A - B, a.e - 63, 0);
}

/* bounds of |x| for a p-bit number from its top limb */
static rad_t rad_mag(int64_t e, const uint32_t *m, int n, int up) {
  if (iszero(e)) return RAD_ZERO;
  uint64_t top = m[n - 1];
  if (up) {
    int rest = 0;
    for (int i = 0; i < n - 1; ++i) rest |= m[i] != 0;
    top += (uint64_t)rest;
  }
  return rad_from64(top, e - 32, up);
}

/* half an ulp of a p-bit result with exponent e (0 for a zero result) */
static rad_t rad_hu(int64_t e, int p) {
  if (iszero(e)) return RAD_ZERO;
  rad_t r = {0x80000000u, e - p};
  return r;
}

static rad_t ball_mul(int p, int n, int64_t eu, int64_t ex, const uint32_t *mx, rad_t rx, int64_t ey,
                      const uint32_t *my, rad_t ry) {
  rad_t r = rad_add(rad_hu(eu, p), rad_mul(rad_mag(ex, mx, n, 1), ry, 1));
  r = rad_add(r, rad_mul(rad_mag(ey, my, n, 1), rx, 1));
  return rad_add(r, rad_mul(rx, ry, 1));
}

static rad_t ball_sub(int p, int64_t eu, rad_t rx, rad_t rt) { return rad_add(rad_add(rad_hu(eu, p), rx), rt); }

static rad_t ball_recip(int p, int n, int64_t eu, int64_t ea, const uint32_t *ma, rad_t ra) {
  rad_t lo = rad_mag(ea, ma, n, 0);
  int pos = 0;
  rad_t gap = rad_sub_down(lo, ra, &pos);
  if (!pos) return RAD_UNB;
  return rad_add(rad_hu(eu, p), rad_div_up(ra, rad_mul(lo, gap, 0)));
}

/* Radius arithmetic on its own (tests of the rounding directions):
 * op 0: a + b up, 1: a * b up, 2: a * b down, 3: a / b up, 4: a - b down
 * (*pos receives 0 when a - b <= 0). */
int or_rad_op(int op, uint32_t am, int64_t ae, uint32_t bm, int64_t be, uint32_t *om, int64_t *oe, int *pos) {
  rad_t a = {am, ae}, b = {bm, be}, r = RAD_ZERO;
  int ps = 1;
  switch (op) {
    case 0: r = rad_add(a, b); break;
    case 1: r = rad_mul(a, b, 1); break;
    case 2: r = rad_mul(a, b, 0); break;
    case 3: r = rad_div_up(a, b); break;
    case 4: r = rad_sub_down(a, b, &ps); break;
    default: return OR_EINVAL;
  }
  *om = r.m;
  *oe = r.e;
  if (pos) *pos = ps;
  return OR_OK;
}

/* Cauchy entries with radii: s = RN(x_i + y_j) (x, y exact), a = RN(1/s). */
int or_cauchy_ball(int64_t N, int p, const double *x, const double *y, int8_t *so, int64_t *eo, uint32_t *mo,
                   uint32_t *rm, int64_t *re) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  int n = c.n;
  uint32_t *tm = (uint32_t *)calloc((size_t)3 * n, sizeof(uint32_t));
  uint32_t *xm = tm + n, *ym = tm + 2 * n;
  for (int64_t i = 0; i < N && st == OR_OK; ++i)
    for (int64_t j = 0; j < N; ++j) {
      int8_t ts;
      int64_t te, idx = i * N + j;
      st = cauchy_entry(&c, x[i], y[j], xm, ym, &ts, &te, tm, so + idx, eo + idx, mo + idx * n);
      if (st) break;
      rad_t rs = ball_sub(p, te, RAD_ZERO, RAD_ZERO);
      rad_t ra = ball_recip(p, n, eo[idx], te, tm, rs);
      rm[idx] = ra.m;
      re[idx] = ra.e;
    }
  free(tm);
  free(c.buf);
  return st;
}

/* The elimination of ge_range (one thread, all N steps) with radii: the
 * values are the same operations in the same order; RX (N*N radii, in/out)
 * holds the input's radii on entry, RD (N) receives those of D_1..D_N. */
int or_ge_ball(int64_t N, int p, int lastcol, int8_t *S, int64_t *E, uint32_t *M, uint32_t *RXm, int64_t *RXe,
               int8_t *Ds, int64_t *De, uint32_t *Dm, uint32_t *RDm, int64_t *RDe, int64_t *zero_k) {
  ctx_t c;
  int st = ctx_init(&c, p);
  if (st) return st;
  if (N < 1) {
    free(c.buf);
    return OR_EINVAL;
  }
  int n = c.n;
  uint32_t *r = (uint32_t *)calloc(n, sizeof(uint32_t));
  uint32_t *one = (uint32_t *)calloc(n, sizeof(uint32_t));
  uint32_t *t = (uint32_t *)calloc(n, sizeof(uint32_t));
  uint32_t *zm = (uint32_t *)calloc((size_t)N * n, sizeof(uint32_t));
  int8_t *zs = (int8_t *)calloc(N, 1);
  int64_t *ze = (int64_t *)calloc(N, sizeof(int64_t));
  rad_t *zr = (rad_t *)calloc(N, sizeof(rad_t));
  one[n - 1] = 0x80000000u;
  if (zero_k) *zero_k = 0;
#define RX(ij) ((rad_t){RXm[ij], RXe[ij]})
  rad_t rprev = RAD_ZERO; /* radius of D_{k-1}; D_0 = 1 exactly */
  for (int64_t k = 0; k < N; ++k) {
    int64_t kk = k * N + k;
    if (k == 0) op_mul(&c, 0, 1, one, S[kk], E[kk], M + kk * n, Ds, De, Dm);
    else op_mul(&c, Ds[k - 1], De[k - 1], Dm + (k - 1) * n, S[kk], E[kk], M + kk * n, Ds + k, De + k, Dm + k * n);
    rad_t rd = (k == 0) ? ball_mul(p, n, De[k], 1, one, RAD_ZERO, E[kk], M + kk * n, RX(kk))
                        : ball_mul(p, n, De[k], De[k - 1], Dm + (k - 1) * n, rprev, E[kk], M + kk * n, RX(kk));
    RDm[k] = rd.m;
    RDe[k] = rd.e;
    rprev = rd;
    if (iszero(E[kk])) { /* D_k = 0 keeps its radius; D_k+1.. are not computed: unbounded */
      if (zero_k) *zero_k = k + 1;
      for (int64_t q = k; q < N; ++q) setzero(Ds + q, De + q, Dm + q * n, n);
      for (int64_t q = k + 1; q < N; ++q) {
        RDm[q] = RAD_UNB.m;
        RDe[q] = RAD_UNB.e;
      }
      if (k < N - 1) st = OR_EZEROPIVOT;
      break;
    }
    if (k == N - 1) break;
    int8_t rs;
    int64_t re;
    op_recip(&c, S[kk], E[kk], M + kk * n, &rs, &re, r);
    rad_t rr = ball_recip(p, n, re, E[kk], M + kk * n, RX(kk));
    for (int64_t i = k + 1; i < N; ++i) {
      int64_t ik = i * N + k;
      op_mul(&c, S[ik], E[ik], M + ik * n, rs, re, r, zs + i, ze + i, zm + i * n);
      zr[i] = ball_mul(p, n, ze[i], E[ik], M + ik * n, RX(ik), re, r, rr);
    }
    for (int64_t i = k + 1; i < N; ++i) {
      for (int64_t j = lastcol ? 0 : k + 1; j < N; ++j) {
        if (j == k) continue;
        const int64_t ij = i * N + j;
        const int64_t kj = k * N + j;
        int8_t ts;
        int64_t te;
        op_mul(&c, zs[i], ze[i], zm + i * n, S[kj], E[kj], M + kj * n, &ts, &te, t);
        rad_t rt = ball_mul(p, n, te, ze[i], zm + i * n, zr[i], E[kj], M + kj * n, RX(kj));
        rad_t rx = RX(ij);
        op_add(&c, S[ij], E[ij], M + ij * n, ts, te, t, 1, S + ij, E + ij, M + ij * n);
        rad_t ru = ball_sub(p, E[ij], rx, rt);
        RXm[ij] = ru.m;
        RXe[ij] = ru.e;
      }
      if (lastcol) {
        int64_t ik = i * N + k;
        copynum(iszero(ze[i]) ? 0 : (int8_t)(zs[i] ^ 1), ze[i], zm + i * n, n, S + ik, E + ik, M + ik * n);
        RXm[ik] = zr[i].m;
        RXe[ik] = zr[i].e;
      }
    }
  }
#undef RX
  free(zr);
  free(ze);
  free(zs);
  free(zm);
  free(t);
  free(one);
  free(r);
  free(c.buf);
  return st;
}

/* Last-column minors (as or_lastcol) with radii: C_jN = RN(D_{N-1} l_Nj),
 * C_NN = D_{N-1}; normalised: delta_j = RN(l_Nj * RN(1/l_N1)), delta_1 = 1
 * (radius 0), delta_N = RN(1/l_N1).  rdm/rde: radius of D_{N-1}; RXm/RXe:
 * the radii of the eliminated array. */
int or_lastcol_ball(int64_t N, int p, int normalised, const int8_t *S, const int64_t *E, const uint32_t *M,
                    const uint32_t *RXm, const int64_t *RXe, int8_t dsg, int64_t dex, const uint32_t *dm, uint32_t rdm,
                    int64_t rde, int8_t *os, int64_t *oe, uint32_t *om, uint32_t *rm, int64_t *re) {
  int st = or_lastcol(N, p, normalised, S, E, M, dsg, dex, dm, os, oe, om);
  if (st) return st;
  int n = p / 32;
  const int64_t row = (N - 1) * N;
  rad_t rD = {rdm, rde};
  if (!normalised) {
    for (int64_t j = 0; j + 1 < N; ++j) {
      rad_t rl = {RXm[row + j], RXe[row + j]};
      rad_t r = ball_mul(p, n, oe[j], dex, dm, rD, E[row + j], M + (row + j) * n, rl);
      rm[j] = r.m;
      re[j] = r.e;
    }
    rm[N - 1] = rdm;
    re[N - 1] = rde;
  } else {
    rm[0] = 0;
    re[0] = ZEXP;
    if (N > 1) {
      rad_t rl1 = {RXm[row], RXe[row]};
      rad_t rr = ball_recip(p, n, oe[N - 1], E[row], M + row * n, rl1);
      for (int64_t j = 1; j + 1 < N; ++j) {
        rad_t rl = {RXm[row + j], RXe[row + j]};
        rad_t r = ball_mul(p, n, oe[j], E[row + j], M + (row + j) * n, rl, oe[N - 1], om + (N - 1) * n, rr);
        rm[j] = r.m;
        re[j] = r.e;
      }
      rm[N - 1] = rr.m;
      re[N - 1] = rr.e;
    }
  }
  return OR_OK;
}
