/* CPU baseline of the compressed H-matrix-vector product, in plain C with OpenMP (oracle;
 * TEST INFRASTRUCTURE ONLY: timed by the benchmark's CPU baseline and reference legs and
 * checked by the tests; the product library never loads it).
 *
 * It restates, independently of the GPU library, what Section 5.4 does on a CPU: every leaf
 * block is stored compressed (Section 3.2: AFL; Section 3.3: one AFL unit per column of W and X
 * at precision eps sigma_0 / sigma_i, dense leaves one unit at eps) and the product
 * y += A~ x decodes each unit when it is used and applies it with plain FP64 loops:
 *   phase A: t_b = Sigma_b X~_b^T x|sigma for every lowrank block (a column is decoded, then
 *            dotted with x);
 *   phase B: y|tau += W~_b t_b (a column decoded, then an axpy) and y|tau += D~_b x|sigma.
 * Blocks are distributed over the threads (phase B round-robin); every thread adds into its own
 * copy of y, and the copies are summed in thread order, so a run with a given thread count is
 * deterministic.
 * The same loops over the FP64 factors themselves (no decoding) give the plain FP64
 * H-matrix-vector product.
 *
 * The codec follows the readings of the oracle (oracle/afl.py): m = ceil(-log2 u) from the
 * binary exponent of u, m_min the smallest nonzero |a|, v = |a| / m_min + 1 rounded half up
 * on its bit pattern to m mantissa bits, field = biased exponent - 1023, e the bit length of
 * the largest field, code = sign << (e + m) | field << m | mantissa, packed LSB-first at bit
 * j w; decoding (v - 1) * m_min in IEEE FP64 without contraction (built with
 * -ffp-contract=off).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t n;        /* values */
  double m_min;
  int32_t e, m, w;
  uint8_t *data;    /* LSB-first codes, 8 bytes readable past the last code */
} unit_t;

typedef struct {
  int64_t row0, nrows, col0, ncols;
  int32_t kind, rank;          /* kind 0 dense, 1 lowrank */
  const double *D, *W, *S, *X; /* the FP64 factors (for the plain product) */
  int64_t u0;                  /* first unit */
} blk_t;

typedef struct {
  int64_t n, nb, nu;
  const int64_t *perm;         /* copied */
  int64_t *perm_own;
  blk_t *b;
  unit_t *u;
  int64_t max_len;             /* longest unit */
  double *t;                   /* t_b for every lowrank column, [rank_sum] */
  int64_t *t0;                 /* first t index per block */
} hmat_t;

/* m = ceil(-log2 u) clamped to [0, 52]: with u = f 2^E, f in [1/2, 1), it is 1 - E */
int hlro_mantissa_bits(double u) {
  int E = 0;
  frexp(u, &E);
  int m = 1 - E;
  return m < 0 ? 0 : m > 52 ? 52 : m;
}

static uint64_t bits_of(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
}
static double double_of(uint64_t b) {
  double x;
  memcpy(&x, &b, 8);
  return x;
}

/* Bytes of the stream of n codes of w bits, padded to 16, plus 8 readable bytes. */
static size_t stream_alloc(int64_t n, int w) { return (((size_t)n * (size_t)w + 7) / 8 + 15) / 16 * 16 + 8; }

/* AFL-encode a[0..n) at precision u into *U (allocates U->data). Returns 0, or -1 for
 * non-finite input or a failed allocation. */
int hlro_encode_unit(const double *a, int64_t n, double u, unit_t *U) {
  const int m = hlro_mantissa_bits(u);
  double m_min = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    if (!isfinite(a[j])) return -1;
    const double x = fabs(a[j]);
    if (x != 0.0 && (m_min == 0.0 || x < m_min)) m_min = x;
  }
  uint64_t *rb = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  if (!rb) return -1;
  int64_t fmax = 0;
  for (int64_t j = 0; j < n; ++j) {
    const double x = fabs(a[j]);
    if (x == 0.0 || m_min == 0.0) {
      rb[j] = bits_of(1.0); /* zero: v = 1, field 0, mantissa 0 */
      continue;
    }
    uint64_t b = bits_of(x / m_min + 1.0);
    if (m < 52) {
      b += (uint64_t)1 << (51 - m);
      b &= ~(((uint64_t)1 << (52 - m)) - 1);
    }
    rb[j] = b;
    const int64_t f = (int64_t)(b >> 52) - 1023;
    if (f > fmax) fmax = f;
  }
  int e = 0;
  while (((int64_t)1 << e) <= fmax) ++e; /* bit length of the largest field */
  const int w = 1 + e + m;
  U->n = n;
  U->m_min = m_min;
  U->e = e;
  U->m = m;
  U->w = w;
  U->data = (uint8_t *)calloc(stream_alloc(n, w), 1);
  if (!U->data) {
    free(rb);
    return -1;
  }
  for (int64_t j = 0; j < n; ++j) {
    const uint64_t b = rb[j];
    const uint64_t field = (b >> 52) - 1023;
    const uint64_t mant = (b & (((uint64_t)1 << 52) - 1)) >> (52 - m);
    const uint64_t sign = a[j] < 0.0 ? 1 : 0;
    const uint64_t code = (sign << (e + m)) | (field << m) | mant;
    /* OR the w bits of the code in from stream bit j w: byte k of (code << sh) goes to byte
     * (bit >> 3) + k, and the bits shifted out of the 64-bit word to the ninth byte */
    const uint64_t bit0 = (uint64_t)j * (uint64_t)w;
    const int sh = (int)(bit0 & 7);
    uint8_t *q = U->data + (bit0 >> 3);
    const uint64_t lo = code << sh;
    for (int k = 0; k < 8; ++k) q[k] |= (uint8_t)(lo >> (8 * k));
    if (sh + w > 64) q[8] |= (uint8_t)(code >> (64 - sh));
  }
  free(rb);
  return 0;
}

/* Value j of a unit: the code at bits [j w, (j + 1) w), then (v - 1) * m_min. */
static double decode_value(const unit_t *U, int64_t j) {
  const uint64_t bit0 = (uint64_t)j * (uint64_t)U->w;
  const int sh = (int)(bit0 & 7);
  const uint8_t *q = U->data + (bit0 >> 3);
  uint64_t word = 0; /* bytes bit0 >> 3 .. + 7, little-endian */
  for (int k = 0; k < 8; ++k) word |= (uint64_t)q[k] << (8 * k);
  uint64_t code = word >> sh;
  if (sh + U->w > 64) code |= (uint64_t)q[8] << (64 - sh);
  if (U->w < 64) code &= ((uint64_t)1 << U->w) - 1;
  const int e = U->e, m = U->m;
  const uint64_t mant = code & (((uint64_t)1 << m) - 1);
  const uint64_t field = (code >> m) & (((uint64_t)1 << e) - 1);
  const uint64_t sign = (code >> (e + m)) & 1;
  const double v = double_of(((field + 1023) << 52) | (mant << (52 - m)));
  const double a = (v - 1.0) * U->m_min;
  return sign ? -a : a;
}

void hlro_decode_unit(const unit_t *U, double *out) {
  for (int64_t j = 0; j < U->n; ++j) out[j] = decode_value(U, j);
}

void hlro_free(hmat_t *H) {
  if (!H) return;
  for (int64_t u = 0; u < H->nu; ++u) free(H->u[u].data);
  free(H->u);
  free(H->b);
  free(H->t);
  free(H->t0);
  free(H->perm_own);
  free(H);
}

/* Build the compressed matrix from the FP64 blocks (arrays of nb entries; kind 0 dense with
 * D[b] (nrows x ncols column-major), kind 1 lowrank with W[b] (nrows x rank), S[b] (rank),
 * X[b] (ncols x rank)); perm[p] = original index of cluster position p. The factor arrays
 * must stay alive for the plain product. Returns NULL on failure. */
hmat_t *hlro_build(int64_t n, const int64_t *perm, int64_t nb, const int64_t *row0, const int64_t *nrows,
                   const int64_t *col0, const int64_t *ncols, const int32_t *kind, const int32_t *rank,
                   const double *const *D, const double *const *W, const double *const *S, const double *const *X,
                   double eps) {
  hmat_t *H = (hmat_t *)calloc(1, sizeof(hmat_t));
  if (!H) return NULL;
  H->n = n;
  H->nb = nb;
  H->perm_own = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  H->b = (blk_t *)calloc((size_t)nb, sizeof(blk_t));
  H->t0 = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
  if (!H->perm_own || !H->b || !H->t0) {
    hlro_free(H);
    return NULL;
  }
  memcpy(H->perm_own, perm, sizeof(int64_t) * (size_t)n);
  H->perm = H->perm_own;
  int64_t nu = 0, ts = 0;
  for (int64_t i = 0; i < nb; ++i) {
    blk_t *B = &H->b[i];
    B->row0 = row0[i];
    B->nrows = nrows[i];
    B->col0 = col0[i];
    B->ncols = ncols[i];
    B->kind = kind[i];
    B->rank = kind[i] == 0 ? 0 : rank[i];
    B->D = D[i];
    B->W = W[i];
    B->S = S[i];
    B->X = X[i];
    B->u0 = nu;
    H->t0[i] = ts;
    nu += B->kind == 0 ? 1 : 2 * (int64_t)B->rank;
    ts += B->rank;
  }
  H->t0[nb] = ts;
  H->nu = nu;
  H->u = (unit_t *)calloc((size_t)(nu > 0 ? nu : 1), sizeof(unit_t));
  H->t = (double *)calloc((size_t)(ts > 0 ? ts : 1), sizeof(double));
  if (!H->u || !H->t) {
    hlro_free(H);
    return NULL;
  }
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t i = 0; i < nb; ++i) {
    const blk_t *B = &H->b[i];
    if (B->kind == 0) {
      bad |= hlro_encode_unit(B->D, B->nrows * B->ncols, eps, &H->u[B->u0]) != 0;
    } else {
      const double delta = eps * B->S[0];
      for (int k = 0; k < B->rank; ++k) {
        const double uk = delta / B->S[k];
        bad |= hlro_encode_unit(B->W + (size_t)k * B->nrows, B->nrows, uk, &H->u[B->u0 + k]) != 0;
        bad |= hlro_encode_unit(B->X + (size_t)k * B->ncols, B->ncols, uk, &H->u[B->u0 + B->rank + k]) != 0;
      }
    }
  }
  int64_t mx = 0;
  for (int64_t u = 0; u < nu; ++u)
    if (H->u[u].n > mx) mx = H->u[u].n;
  H->max_len = mx;
  if (bad) {
    hlro_free(H);
    return NULL;
  }
  return H;
}

int64_t hlro_units(const hmat_t *H) { return H->nu; }
/* Parameters and stream of unit u (for the tests): n, m_min, e, m, and its bytes. */
void hlro_unit_info(const hmat_t *H, int64_t u, int64_t *n, double *m_min, int32_t *e, int32_t *m) {
  *n = H->u[u].n;
  *m_min = H->u[u].m_min;
  *e = H->u[u].e;
  *m = H->u[u].m;
}
void hlro_unit_decode(const hmat_t *H, int64_t u, double *out) { hlro_decode_unit(&H->u[u], out); }

/* Column k of a factor: decoded into buf (compressed) or the FP64 factor itself (plain). */
static const double *column(const hmat_t *H, const blk_t *B, int which, int k, int raw, double *buf) {
  if (raw) {
    if (which == 0) return B->D;
    return which == 1 ? B->W + (size_t)k * B->nrows : B->X + (size_t)k * B->ncols;
  }
  const unit_t *U = which == 0 ? &H->u[B->u0] : which == 1 ? &H->u[B->u0 + k] : &H->u[B->u0 + B->rank + k];
  hlro_decode_unit(U, buf);
  return buf;
}

/* y += A~ x (original index order) on `threads` threads (0 = the OpenMP default); raw = 1
 * multiplies with the FP64 factors themselves (the plain FP64 H-matrix-vector product).
 * Returns 0, or -1 if scratch memory cannot be allocated. */
int hlro_matvec(hmat_t *H, const double *x, double *y, int raw, int threads) {
  const int64_t n = H->n;
  const int nt = threads > 0 ? threads : omp_get_max_threads();
  double *xp = (double *)malloc(sizeof(double) * (size_t)n);
  double *yt = (double *)calloc((size_t)n * (size_t)nt, sizeof(double));
  if (!xp || !yt) {
    free(xp);
    free(yt);
    return -1;
  }
  for (int64_t p = 0; p < n; ++p) xp[p] = x[H->perm[p]];
  int fail = 0;
#pragma omp parallel num_threads(nt) reduction(| : fail)
  {
    const int tid = omp_get_thread_num();
    double *buf = (double *)malloc(sizeof(double) * (size_t)(H->max_len > 0 ? H->max_len : 1));
    double *yl = yt + (size_t)tid * (size_t)n;
    if (!buf) fail = 1;
    /* phase A: t_b = Sigma_b X~_b^T x|sigma */
#pragma omp for schedule(dynamic, 8)
    for (int64_t i = 0; i < H->nb; ++i) {
      const blk_t *B = &H->b[i];
      if (!buf || B->kind == 0) continue;
      const double *xs = xp + B->col0;
      for (int k = 0; k < B->rank; ++k) {
        const double *c = column(H, B, 2, k, raw, buf);
        double s = 0.0;
        for (int64_t j = 0; j < B->ncols; ++j) s += c[j] * xs[j];
        H->t[H->t0[i] + k] = B->S[k] * s;
      }
    }
    /* phase B: y|tau += W~_b t_b, y|tau += D~_b x|sigma (into this thread's copy of y; a fixed
     * round-robin assignment of blocks to threads, so the sums do not depend on timing) */
#pragma omp for schedule(static, 4)
    for (int64_t i = 0; i < H->nb; ++i) {
      const blk_t *B = &H->b[i];
      if (!buf) continue;
      double *yr = yl + B->row0;
      if (B->kind == 0) {
        const double *Dd = column(H, B, 0, 0, raw, buf);
        const double *xs = xp + B->col0;
        for (int64_t j = 0; j < B->ncols; ++j) {
          const double xj = xs[j];
          const double *cj = Dd + (size_t)j * B->nrows;
          for (int64_t r = 0; r < B->nrows; ++r) yr[r] += cj[r] * xj;
        }
      } else {
        for (int k = 0; k < B->rank; ++k) {
          const double *c = column(H, B, 1, k, raw, buf);
          const double tk = H->t[H->t0[i] + k];
          for (int64_t r = 0; r < B->nrows; ++r) yr[r] += c[r] * tk;
        }
      }
    }
    free(buf);
    /* the threads' copies of y, summed in thread order */
#pragma omp for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
      double s = 0.0;
      for (int q = 0; q < nt; ++q) s += yt[(size_t)q * (size_t)n + p];
      y[H->perm[p]] += s;
    }
  }
  free(xp);
  free(yt);
  return fail ? -1 : 0;
}

/* Algorithmic bytes of one product as the benchmark counts them: stream bytes (unpadded) +
 * 16 per unit + 8 per singular value + 32 n (x, y read and write, permutation); raw = 1: the
 * FP64 factors (8 per value) + 8 per singular value + 32 n. */
double hlro_bytes(const hmat_t *H, int raw) {
  double s = 32.0 * (double)H->n;
  for (int64_t i = 0; i < H->nb; ++i) s += 8.0 * H->b[i].rank;
  for (int64_t u = 0; u < H->nu; ++u) {
    const unit_t *U = &H->u[u];
    s += raw ? 8.0 * (double)U->n : (double)(((uint64_t)U->n * (uint64_t)U->w + 7) / 8) + 16.0;
  }
  return s;
}
