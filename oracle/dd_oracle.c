/*
 * CPU oracle for the algebraic domain-decomposition preconditioned GMRES
 * solve.  TEST INFRASTRUCTURE ONLY: it is called by the test-suite, by the
 * smoke check and by the benchmark's CPU-baseline leg, never by the product
 * path.  Plain, slow and sequential in structure, FP64 throughout; OpenMP only
 * runs independent subdomains / aggregates side by side, as the paper's
 * parallel setup does (Section 4, the parfor over mini Schur complements).
 *
 * What it computes, in the paper's notation (Section 3.2, matrix view):
 *   the permuted matrix P^T C P = [D E; F G], D = blkDiag(A_11..A_mm) holds
 *   the subdomain interiors, G the interface (separator) rows/columns;
 *   Algorithm 1 builds S_hat = blkDiag(S_11..S_kk) over aggregates of
 *   consecutive interface indices r_i..r_{i+1}-1 (eq. aggrV);
 *   the preconditioner is B = [D 0; F S_hat][D^-1 0; 0 S_hat^-1][D E; 0 S_hat]
 *   (Definition of B_MSCN, eq. NDfactor);
 *   Algorithm 2 applies B^-1;
 *   right-preconditioned restarted (flexible) GMRES (Section 5) solves C x = b.
 *
 * Readings where the paper is ambiguous (each one is pinned by a test):
 *   - Algorithm 2 writes (E z1) in the forward sweep and (F x2) in the backward
 *     sweep; with B factored as above the lower-left block F must act on z1
 *     and the upper-right block E on x2 (this is the only order that makes
 *     B^-1 agree with the Banachiewicz inverse, Lemma 1).
 *   - MSCNR: "G - F D^-1 E 1" is read as G_ii - diag(F_ii D_ii^-1 E_ii 1),
 *     the row sums lumped onto the diagonal.
 *   - MSCN takes D_ii, E_ii, F_ii with the same local index range as G_ii
 *     (Algorithm 1, principal submatrices).
 *   - MSCE with unbounded radius (r = infinity): D_{r_i} is every interior
 *     adjacent to the aggregate, so S_ii is the diagonal block of the exact
 *     Schur complement S = G - F D^-1 E (the block-Jacobi reading that
 *     closes Section 3.3).
 *   - MSCE with a finite radius r: D_{r_i} holds the interior nodes within
 *     path length r of the aggregate (first step through F or E, then
 *     through the pattern of D), closed by the D-neighbours of every reached
 *     node with a zero diagonal (a pressure-like node cut down to one
 *     velocity coupling would make D_{r_i} singular).  r = 0 gives LUM.
 *   - Overlapped aggregation (the Remark after eq. aggrV, Algorithm 1):
 *     block i spans indices r_i .. r_{i+1} - 1 + w_i, with 0 <= w_i <=
 *     p_{i+1} and w_k = 0 (the paper both bounds w_i by p_i and uses w =
 *     sz in its tables; the extension stays inside the next aggregate).
 *     OMSCN / OMSCNR / OLUM are MSCN / MSCNR / LUM on these blocks.  S_hat
 *     is assembled by placing the blocks in aggregate order, a later block
 *     overwriting the overlap; it is not block diagonal and is solved whole
 *     (band LU with partial pivoting), as the Remark says the solve phase
 *     loses its parallelism.
 *
 * Exact LU of every A_jj (Section 4: "exact triangular factors") with partial
 * pivoting, the pivot being the first row holding the largest magnitude; a
 * block is singular when |pivot| <= pivtol * max|block|.  Band storage is used
 * for the large blocks; it makes the same pivot choices as the dense
 * factorisation (pinned by a test).
 *
 * Status codes (values shared with the library's public header by contract):
 * 0 ok, 1 invalid argument, 2 invalid partition, 3 singular interior block,
 * 4 singular Schur block, 5 not converged, 6 non-finite value, 8 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OK = 0, ORC_INVALID_ARG = 1, ORC_INVALID_PARTITION = 2, ORC_SINGULAR_BLOCK = 3,
       ORC_SINGULAR_SCHUR = 4, ORC_NOT_CONVERGED = 5, ORC_NONFINITE = 6, ORC_OOM = 8 };

enum { ORC_EXACT = 0, ORC_MSCE_INF = 1, ORC_MSCN = 2, ORC_MSCNR = 3, ORC_LUM = 4,
       ORC_OMSCN = 6, ORC_OMSCNR = 7, ORC_OLUM = 8, ORC_MSCE = 9, ORC_IDENTITY = -1 };

/* overlapped kinds (Remark on overlapped aggregation, Algorithm 1) */
static int is_overlapped(int kind) { return kind == ORC_OMSCN || kind == ORC_OMSCNR || kind == ORC_OLUM; }

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ======================================================================== */
/* Dense LU with partial pivoting (row-major, in place)                      */
/* ======================================================================== */

/* Factor a (n x n, row-major) as P a = L U; piv[k] is the row swapped with k
 * at step k.  Returns 0, or k+1 if column k has no acceptable pivot. */
int orc_dense_lu(int32_t n, double *a, int32_t *piv, double pivtol) {
  double amax = 0.0;
  for (int64_t q = 0; q < (int64_t)n * n; ++q) if (fabs(a[q]) > amax) amax = fabs(a[q]);
  for (int32_t k = 0; k < n; ++k) {
    int32_t p = k;
    double best = fabs(a[(int64_t)k * n + k]);
    for (int32_t i = k + 1; i < n; ++i)
      if (fabs(a[(int64_t)i * n + k]) > best) { best = fabs(a[(int64_t)i * n + k]); p = i; }
    piv[k] = p;
    if (!(best > pivtol * amax)) return k + 1;
    if (p != k)
      for (int32_t j = 0; j < n; ++j) {
        double t = a[(int64_t)k * n + j];
        a[(int64_t)k * n + j] = a[(int64_t)p * n + j];
        a[(int64_t)p * n + j] = t;
      }
    double dkk = a[(int64_t)k * n + k];
    for (int32_t i = k + 1; i < n; ++i) {
      double l = a[(int64_t)i * n + k] / dkk;
      a[(int64_t)i * n + k] = l;
      if (l != 0.0)
        for (int32_t j = k + 1; j < n; ++j) a[(int64_t)i * n + j] -= l * a[(int64_t)k * n + j];
    }
  }
  return 0;
}

/* Solve with the factors of orc_dense_lu, b overwritten by the solution. */
void orc_dense_lu_solve(int32_t n, const double *lu, const int32_t *piv, double *b) {
  for (int32_t k = 0; k < n; ++k)
    if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
  for (int32_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int32_t j = 0; j < i; ++j) s -= lu[(int64_t)i * n + j] * b[j];
    b[i] = s;
  }
  for (int32_t i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int32_t j = i + 1; j < n; ++j) s -= lu[(int64_t)i * n + j] * b[j];
    b[i] = s / lu[(int64_t)i * n + i];
  }
}

/* ======================================================================== */
/* Band LU with partial pivoting                                             */
/* ======================================================================== */
/* Row i keeps columns i-kl .. i+ku+kl at offsets 0 .. 2kl+ku (width wd), so
 * rows brought up by a pivot swap still fit.  The multipliers of step k are
 * kept in lm[k*kl ..] in the row order of that step, with the swaps
 * interleaved (the unpermuted form of a banded LU).                         */
typedef struct {
  int32_t n, kl, ku, wd;
  double *r;   /* n x wd */
  double *lm;  /* n x kl */
  int32_t *piv;
} orc_band;

static inline double *band_at(orc_band *b, int32_t i, int32_t j) {
  return &b->r[(int64_t)i * b->wd + (j - i + b->kl)];
}

/* Fill from a dense row-major matrix (used by the pin tests). */
static int band_alloc(orc_band *b, int32_t n, int32_t kl, int32_t ku) {
  b->n = n; b->kl = kl; b->ku = ku; b->wd = 2 * kl + ku + 1;
  b->r = (double *)calloc((size_t)n * b->wd + 1, sizeof(double));
  b->lm = (double *)calloc((size_t)n * (kl > 0 ? kl : 1) + 1, sizeof(double));
  b->piv = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  return (b->r && b->lm && b->piv) ? 0 : -1;
}

static void band_free(orc_band *b) { free(b->r); free(b->lm); free(b->piv); b->r = 0; b->lm = 0; b->piv = 0; }

/* 2-norms of the columns of the band (before it is factored): the reference
 * of the incomplete factorisation's drop test. */
static void band_colnorms(const orc_band *b, double *cn) {
  for (int32_t j = 0; j < b->n; ++j) {
    double s = 0.0;
    int32_t i0 = j - b->ku > 0 ? j - b->ku : 0, i1 = j + b->kl < b->n - 1 ? j + b->kl : b->n - 1;
    for (int32_t i = i0; i <= i1; ++i) {
      double v = b->r[(int64_t)i * b->wd + (j - i + b->kl)];
      s += v * v;
    }
    cn[j] = sqrt(s);
  }
}

/* Factor in place; returns 0 or k+1 for a failed pivot in column k.
 * tau > 0 (with cn the column norms of the unfactored band): the incomplete
 * factorisation with threshold dropping (Section 5's ILU with tolerance
 * tolA), read as: at step k, after the row exchange, an entry u_kj (j > k)
 * of the pivot row is dropped when |u_kj| < tau * |A(:, j)|, and a multiplier
 * l_ik when |l_ik| < tau * |A(:, k)| / |u_kk|, before either is used in the
 * step's update; the diagonal is kept.  tau = 0 is the exact LU. */
static int band_factor(orc_band *b, double pivtol, double tau, const double *cn) {
  int32_t n = b->n, kl = b->kl, ku = b->ku;
  double amax = 0.0;
  for (int64_t q = 0; q < (int64_t)n * b->wd; ++q) if (fabs(b->r[q]) > amax) amax = fabs(b->r[q]);
  for (int32_t k = 0; k < n; ++k) {
    int32_t last = (k + kl < n - 1) ? k + kl : n - 1;
    int32_t p = k;
    double best = fabs(*band_at(b, k, k));
    for (int32_t i = k + 1; i <= last; ++i)
      if (fabs(*band_at(b, i, k)) > best) { best = fabs(*band_at(b, i, k)); p = i; }
    b->piv[k] = p;
    if (!(best > pivtol * amax)) return k + 1;
    int32_t jend = (k + kl + ku < n - 1) ? k + kl + ku : n - 1;
    if (p != k)
      for (int32_t j = k; j <= jend; ++j) {
        double t = *band_at(b, k, j);
        *band_at(b, k, j) = *band_at(b, p, j);
        *band_at(b, p, j) = t;
      }
    double dkk = *band_at(b, k, k);
    if (tau > 0.0)
      for (int32_t j = k + 1; j <= jend; ++j)
        if (fabs(*band_at(b, k, j)) < tau * cn[j]) *band_at(b, k, j) = 0.0;
    for (int32_t i = k + 1; i <= last; ++i) {
      double l = *band_at(b, i, k) / dkk;
      if (tau > 0.0 && fabs(l) < tau * cn[k] / fabs(dkk)) l = 0.0;
      b->lm[(int64_t)k * kl + (i - k - 1)] = l;
      *band_at(b, i, k) = 0.0;
      if (l != 0.0)
        for (int32_t j = k + 1; j <= jend; ++j) *band_at(b, i, j) -= l * *band_at(b, k, j);
    }
  }
  return 0;
}

static void band_solve(const orc_band *b, double *x) {
  int32_t n = b->n, kl = b->kl, ku = b->ku;
  for (int32_t k = 0; k < n; ++k) {
    int32_t p = b->piv[k];
    if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    int32_t last = (k + kl < n - 1) ? k + kl : n - 1;
    for (int32_t i = k + 1; i <= last; ++i) x[i] -= b->lm[(int64_t)k * kl + (i - k - 1)] * x[k];
  }
  for (int32_t i = n - 1; i >= 0; --i) {
    int32_t jend = (i + kl + ku < n - 1) ? i + kl + ku : n - 1;
    double s = x[i];
    for (int32_t j = i + 1; j <= jend; ++j) s -= b->r[(int64_t)i * b->wd + (j - i + kl)] * x[j];
    x[i] = s / b->r[(int64_t)i * b->wd + kl];
  }
}

/* Pin helper: band-factor a dense row-major n x n matrix with the given
 * bandwidths, return the pivot sequence and solve one right-hand side. */
int orc_band_lu_dense(int32_t n, const double *a, int32_t kl, int32_t ku, double pivtol,
                      int32_t *piv, double *x) {
  orc_band b;
  if (band_alloc(&b, n, kl, ku)) { band_free(&b); return -1; }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = i - kl; j <= i + ku; ++j)
      if (j >= 0 && j < n) *band_at(&b, i, j) = a[(int64_t)i * n + j];
  int rc = band_factor(&b, pivtol, 0.0, NULL);
  if (rc == 0) {
    memcpy(piv, b.piv, sizeof(int32_t) * n);
    band_solve(&b, x);
  }
  band_free(&b);
  return rc;
}

/* Pin helper: the incomplete band factorisation (drop tolerance tau) of a
 * dense row-major n x n matrix; returns the pivots and solves one
 * right-hand side with the incomplete factors. */
int orc_band_ilu_dense(int32_t n, const double *a, int32_t kl, int32_t ku, double pivtol, double tau,
                       int32_t *piv, double *x) {
  orc_band b;
  double *cn = (double *)malloc(sizeof(double) * ((size_t)n + 1));
  if (!cn || band_alloc(&b, n, kl, ku)) { free(cn); band_free(&b); return -1; }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = i - kl; j <= i + ku; ++j)
      if (j >= 0 && j < n) *band_at(&b, i, j) = a[(int64_t)i * n + j];
  band_colnorms(&b, cn);
  int rc = band_factor(&b, pivtol, tau, cn);
  if (rc == 0) {
    memcpy(piv, b.piv, sizeof(int32_t) * n);
    band_solve(&b, x);
  }
  free(cn);
  band_free(&b);
  return rc;
}

/* ======================================================================== */
/* Preconditioner setup (Algorithm 1)                                        */
/* ======================================================================== */
typedef struct {
  int32_t rows;       /* number of rows */
  int32_t *ptr, *col; /* CSR */
  double *val;
} orc_sp;

typedef struct orc {
  int32_t n, m, nI, nG, nagg, kind, bad_block;
  int32_t *perm, *pos;      /* new->old, old->new */
  int32_t *off;             /* interior offsets per subdomain, m+1 */
  int32_t *agg;             /* aggregate offsets into the interface, nagg+1 */
  orc_band *A;              /* factored interior blocks A_jj */
  orc_sp E, F, G;           /* E: interior x interface, F: interface x interior,
                               G: interface x interface (local indices) */
  orc_sp Et;                /* E transposed: interface x interior */
  int32_t *ovl;             /* overlapped kinds: overlap width w_i of every aggregate */
  int32_t radius;           /* MSCE: path-length radius r */
  double ilu_tol;           /* interior blocks: drop tolerance of the incomplete LU (0: exact) */
  orc_band Shat;            /* overlapped kinds: the assembled S_hat (band, factored) */
  double *Shat0;            /* its entries before the factorisation (band rows, unpivoted) */
  double **S;               /* S_hat blocks, row-major (kept unfactored for tests) */
  double **Slu;             /* their LU factors */
  int32_t **Spiv;
  /* the matrix C itself, original numbering, for GMRES */
  int32_t *rowptr, *ccol;
  double *cval;
} orc;

static void sp_free(orc_sp *s) { free(s->ptr); free(s->col); free(s->val); }

void orc_free(orc *h) {
  if (!h) return;
  free(h->perm); free(h->pos); free(h->off); free(h->agg);
  if (h->A) for (int32_t j = 0; j < h->m; ++j) band_free(&h->A[j]);
  free(h->A);
  sp_free(&h->E); sp_free(&h->F); sp_free(&h->G); sp_free(&h->Et);
  if (h->S) for (int32_t i = 0; i < h->nagg; ++i) { free(h->S[i]); free(h->Slu[i]); free(h->Spiv[i]); }
  free(h->S); free(h->Slu); free(h->Spiv);
  free(h->ovl); band_free(&h->Shat); free(h->Shat0);
  free(h->rowptr); free(h->ccol); free(h->cval);
  free(h);
}

/* Extract the rows [r0, r1) of P^T C P restricted to new columns [c0, c1),
 * column indices shifted by -c0. */
static int extract_sp(const orc *h, int32_t r0, int32_t r1, int32_t c0, int32_t c1, orc_sp *out) {
  int32_t rows = r1 - r0;
  out->rows = rows;
  out->ptr = (int32_t *)calloc((size_t)rows + 1, sizeof(int32_t));
  int64_t cnt = 0;
  for (int32_t r = r0; r < r1; ++r) {
    int32_t o = h->perm[r];
    for (int32_t k = h->rowptr[o]; k < h->rowptr[o + 1]; ++k) {
      int32_t c = h->pos[h->ccol[k]];
      if (c >= c0 && c < c1) ++cnt;
    }
  }
  out->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt + 1));
  out->val = (double *)malloc(sizeof(double) * (size_t)(cnt + 1));
  if (!out->ptr || !out->col || !out->val) return -1;
  int64_t w = 0;
  for (int32_t r = r0; r < r1; ++r) {
    int32_t o = h->perm[r];
    for (int32_t k = h->rowptr[o]; k < h->rowptr[o + 1]; ++k) {
      int32_t c = h->pos[h->ccol[k]];
      if (c >= c0 && c < c1) { out->col[w] = c - c0; out->val[w] = h->cval[k]; ++w; }
    }
    out->ptr[r - r0 + 1] = (int32_t)w;
  }
  return 0;
}

/* value of the sparse row-major block at (r, c), 0 if absent */
static double sp_get(const orc_sp *s, int32_t r, int32_t c) {
  double v = 0.0;
  for (int32_t k = s->ptr[r]; k < s->ptr[r + 1]; ++k) if (s->col[k] == c) v += s->val[k];
  return v;
}

/* Interior block A_jj: rows/cols [off[j], off[j+1]) of P^T C P, band form. */
static int build_interior(orc *h, int32_t j, double pivtol) {
  int32_t r0 = h->off[j], r1 = h->off[j + 1], nj = r1 - r0;
  int32_t kl = 0, ku = 0;
  for (int32_t r = r0; r < r1; ++r) {
    int32_t o = h->perm[r];
    for (int32_t k = h->rowptr[o]; k < h->rowptr[o + 1]; ++k) {
      int32_t c = h->pos[h->ccol[k]];
      if (c < r0 || c >= r1) continue;
      if (r - c > kl) kl = r - c;
      if (c - r > ku) ku = c - r;
    }
  }
  if (band_alloc(&h->A[j], nj, kl, ku)) return ORC_OOM;
  for (int32_t r = r0; r < r1; ++r) {
    int32_t o = h->perm[r];
    for (int32_t k = h->rowptr[o]; k < h->rowptr[o + 1]; ++k) {
      int32_t c = h->pos[h->ccol[k]];
      if (c < r0 || c >= r1) continue;
      *band_at(&h->A[j], r - r0, c - r0) += h->cval[k];
    }
  }
  if (nj == 0) return ORC_OK;
  double *cn = NULL;
  if (h->ilu_tol > 0.0) {
    cn = (double *)malloc(sizeof(double) * (size_t)nj);
    if (!cn) return ORC_OOM;
    band_colnorms(&h->A[j], cn);
  }
  int f = band_factor(&h->A[j], pivtol, h->ilu_tol, cn);
  free(cn);
  return f ? ORC_SINGULAR_BLOCK : ORC_OK;
}

/* Which subdomain owns interior (new) index i */
static int32_t owner(const orc *h, int32_t i) {
  int32_t lo = 0, hi = h->m;
  while (hi - lo > 1) { int32_t mid = (lo + hi) / 2; if (h->off[mid] <= i) lo = mid; else hi = mid; }
  return lo;
}

/* S(R_i, R_i) for MSCE_INF / EXACT:
 *   G(R_i,R_i) - sum_j F(R_i, I_j) A_jj^-1 E(I_j, R_i).
 * For each column c of the aggregate and each subdomain j that E couples to
 * c, solve A_jj x = E(I_j, c) and subtract F(R_i, I_j) x.                  */
static int schur_msce(orc *h, int32_t i, double *S) {
  int32_t a0 = h->agg[i], a1 = h->agg[i + 1], p = a1 - a0;
  double *x = NULL;
  int32_t xcap = 0;
  int8_t *touch = (int8_t *)calloc((size_t)h->m, 1);
  if (!touch) return ORC_OOM;
  for (int32_t r = 0; r < p; ++r)
    for (int32_t c = 0; c < p; ++c) S[(int64_t)r * p + c] = sp_get(&h->G, a0 + r, a0 + c);
  for (int32_t c = 0; c < p; ++c) {
    int32_t gc = a0 + c;
    /* subdomains that the column E(:, gc) touches */
    memset(touch, 0, (size_t)h->m);
    for (int32_t k = h->Et.ptr[gc]; k < h->Et.ptr[gc + 1]; ++k)
      if (h->Et.val[k] != 0.0) touch[owner(h, h->Et.col[k])] = 1;
    for (int32_t j = 0; j < h->m; ++j) {
      if (!touch[j]) continue;
      int32_t r0 = h->off[j], nj = h->off[j + 1] - r0;
      if (nj > xcap) { free(x); xcap = nj; x = (double *)malloc(sizeof(double) * nj); if (!x) { free(touch); return ORC_OOM; } }
      for (int32_t q = 0; q < nj; ++q) x[q] = 0.0;
      for (int32_t k = h->Et.ptr[gc]; k < h->Et.ptr[gc + 1]; ++k) {
        int32_t ri = h->Et.col[k];
        if (ri >= r0 && ri < r0 + nj) x[ri - r0] += h->Et.val[k];
      }
      band_solve(&h->A[j], x);
      for (int32_t r = 0; r < p; ++r) {
        double s = 0.0;
        int32_t gr = a0 + r;
        for (int32_t k = h->F.ptr[gr]; k < h->F.ptr[gr + 1]; ++k) {
          int32_t ci = h->F.col[k];
          if (ci >= r0 && ci < r0 + nj) s += h->F.val[k] * x[ci - r0];
        }
        S[(int64_t)r * p + c] -= s;
      }
    }
  }
  free(x);
  free(touch);
  return ORC_OK;
}

/* MSCN / MSCNR (Algorithm 1): principal submatrices with the same local
 * index range [a0, a1) in D, E, F and G (the aggregate, or for OMSCN /
 * OMSCNR the aggregate extended by its overlap).
 *   MSCN:  S_ii = G_ii - F_ii D_ii^-1 E_ii
 *   MSCNR: S_ii = G_ii - diag(F_ii D_ii^-1 E_ii 1)                          */
static int schur_mscn(orc *h, int32_t a0, int32_t a1, double *S, int rowsum, double pivtol) {
  int32_t p = a1 - a0;
  if (a1 > h->nI) return ORC_INVALID_ARG;
  double *Dii = (double *)calloc((size_t)p * p, sizeof(double));
  double *Eii = (double *)calloc((size_t)p * p, sizeof(double));
  double *Fii = (double *)calloc((size_t)p * p, sizeof(double));
  int32_t *piv = (int32_t *)calloc((size_t)p, sizeof(int32_t));
  double *x = (double *)calloc((size_t)p, sizeof(double));
  int rc = ORC_OK;
  if (!Dii || !Eii || !Fii || !piv || !x) { rc = ORC_OOM; goto out; }
  int nzE = 0, nzF = 0;
  for (int32_t r = 0; r < p; ++r)
    for (int32_t c = 0; c < p; ++c) {
      S[(int64_t)r * p + c] = sp_get(&h->G, a0 + r, a0 + c);
      Eii[(int64_t)r * p + c] = sp_get(&h->E, a0 + r, a0 + c);
      Fii[(int64_t)r * p + c] = sp_get(&h->F, a0 + r, a0 + c);
      nzE |= Eii[(int64_t)r * p + c] != 0.0;
      nzF |= Fii[(int64_t)r * p + c] != 0.0;
    }
  if (!nzE || !nzF) goto out; /* F_ii D_ii^-1 E_ii = 0 */
  /* D_ii: principal block of D = blkDiag(A_jj) with rows/cols [a0, a1) */
  for (int32_t r = 0; r < p; ++r) {
    int32_t o = h->perm[a0 + r];
    for (int32_t k = h->rowptr[o]; k < h->rowptr[o + 1]; ++k) {
      int32_t c = h->pos[h->ccol[k]];
      if (c >= a0 && c < a1) Dii[(int64_t)r * p + (c - a0)] += h->cval[k];
    }
  }
  if (orc_dense_lu(p, Dii, piv, pivtol)) { rc = ORC_SINGULAR_SCHUR; goto out; }
  if (rowsum) {
    for (int32_t r = 0; r < p; ++r) {
      double s = 0.0;
      for (int32_t c = 0; c < p; ++c) s += Eii[(int64_t)r * p + c];
      x[r] = s;
    }
    orc_dense_lu_solve(p, Dii, piv, x);
    for (int32_t r = 0; r < p; ++r) {
      double s = 0.0;
      for (int32_t c = 0; c < p; ++c) s += Fii[(int64_t)r * p + c] * x[c];
      S[(int64_t)r * p + r] -= s;
    }
  } else {
    for (int32_t c = 0; c < p; ++c) {
      for (int32_t r = 0; r < p; ++r) x[r] = Eii[(int64_t)r * p + c];
      orc_dense_lu_solve(p, Dii, piv, x);
      for (int32_t r = 0; r < p; ++r) {
        double s = 0.0;
        for (int32_t q = 0; q < p; ++q) s += Fii[(int64_t)r * p + q] * x[q];
        S[(int64_t)r * p + c] -= s;
      }
    }
  }
out:
  free(Dii); free(Eii); free(Fii); free(piv); free(x);
  return rc;
}

/* Symmetrised pattern of D (the interior rows and columns of P^T C P):
 * adjacency lists in CSR form over the interior numbering. */
static int build_dadj(const orc *h, int32_t **ptr_out, int32_t **adj_out) {
  int32_t nI = h->nI;
  int32_t *cnt = (int32_t *)calloc((size_t)nI + 1, sizeof(int32_t));
  if (!cnt) return ORC_OOM;
  for (int32_t k = 0; k < nI; ++k) {
    int32_t o = h->perm[k];
    for (int32_t q = h->rowptr[o]; q < h->rowptr[o + 1]; ++q) {
      int32_t j = h->pos[h->ccol[q]];
      if (j < nI && j != k) { cnt[k + 1]++; cnt[j + 1]++; }
    }
  }
  for (int32_t k = 0; k < nI; ++k) cnt[k + 1] += cnt[k];
  int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cnt[nI] + 1));
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nI + 1));
  if (!adj || !fill) { free(cnt); free(adj); free(fill); return ORC_OOM; }
  memcpy(fill, cnt, sizeof(int32_t) * (size_t)nI);
  for (int32_t k = 0; k < nI; ++k) {
    int32_t o = h->perm[k];
    for (int32_t q = h->rowptr[o]; q < h->rowptr[o + 1]; ++q) {
      int32_t j = h->pos[h->ccol[q]];
      if (j < nI && j != k) { adj[fill[k]++] = j; adj[fill[j]++] = k; }
    }
  }
  free(fill);
  *ptr_out = cnt;
  *adj_out = adj;
  return ORC_OK;
}

/* value of P^T C P at (new row r, new column c), 0 if absent */
static double c_at(const orc *h, int32_t r, int32_t c) {
  double v = 0.0;
  int32_t o = h->perm[r];
  for (int32_t q = h->rowptr[o]; q < h->rowptr[o + 1]; ++q) if (h->pos[h->ccol[q]] == c) v += h->cval[q];
  return v;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* MSCE with a finite radius r (Algorithm 1's mini Schur complement on edge
 * connectivity): S_ii = G_pi - F_i D_ri^-1 E_i, where D_ri is the principal
 * submatrix of D on the interior nodes reachable from the aggregate by a
 * path of length <= r: the first step goes from an aggregate node to an
 * interior node it is coupled with (an entry of F or E), the others run
 * through the pattern of D.  Every reached node with a zero diagonal (a
 * pressure-like node) brings all its neighbours in D, so that no row of
 * D_ri is cut down to a single coupling.  r = 0: D_ri is empty and
 * S_ii = G_ii (LUM); r large enough: the whole adjacent interiors, S_ii =
 * S(R_i, R_i) (MSCE_INF). */
static int schur_msce_r(orc *h, int32_t i, double *S, const int32_t *dptr, const int32_t *dadj,
                        double pivtol) {
  int32_t a0 = h->agg[i], a1 = h->agg[i + 1], p = a1 - a0, nI = h->nI;
  for (int32_t r = 0; r < p; ++r)
    for (int32_t c = 0; c < p; ++c) S[(int64_t)r * p + c] = sp_get(&h->G, a0 + r, a0 + c);
  if (h->radius <= 0 || nI == 0) return ORC_OK;
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)nI);
  int32_t *set = (int32_t *)malloc(sizeof(int32_t) * (size_t)nI);
  int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)nI);
  if (!dist || !set || !loc) { free(dist); free(set); free(loc); return ORC_OOM; }
  for (int32_t k = 0; k < nI; ++k) { dist[k] = -1; loc[k] = -1; }
  int32_t d = 0;
  /* level 1: interior nodes coupled with the aggregate through F or E */
  for (int32_t g = a0; g < a1; ++g) {
    for (int32_t q = h->F.ptr[g]; q < h->F.ptr[g + 1]; ++q) {
      int32_t j = h->F.col[q];
      if (h->F.val[q] != 0.0 && dist[j] < 0) { dist[j] = 1; set[d++] = j; }
    }
    for (int32_t q = h->Et.ptr[g]; q < h->Et.ptr[g + 1]; ++q) {
      int32_t j = h->Et.col[q];
      if (h->Et.val[q] != 0.0 && dist[j] < 0) { dist[j] = 1; set[d++] = j; }
    }
  }
  /* levels 2 .. r through the pattern of D (breadth first) */
  for (int32_t head = 0; head < d; ++head) {
    int32_t k = set[head];
    if (dist[k] >= h->radius) continue;
    for (int32_t q = dptr[k]; q < dptr[k + 1]; ++q) {
      int32_t j = dadj[q];
      if (dist[j] < 0) { dist[j] = dist[k] + 1; set[d++] = j; }
    }
  }
  /* closure: a reached pressure-like node brings its neighbours */
  int32_t d0 = d;
  for (int32_t q0 = 0; q0 < d0; ++q0) {
    int32_t k = set[q0];
    if (c_at(h, k, k) != 0.0) continue;
    for (int32_t q = dptr[k]; q < dptr[k + 1]; ++q) {
      int32_t j = dadj[q];
      if (dist[j] < 0) { dist[j] = h->radius + 1; set[d++] = j; }
    }
  }
  qsort(set, (size_t)d, sizeof(int32_t), cmp_i32);
  for (int32_t q = 0; q < d; ++q) loc[set[q]] = q;
  double *Dr = (double *)calloc((size_t)d * d + 1, sizeof(double));
  double *Er = (double *)calloc((size_t)d * p + 1, sizeof(double));
  int32_t *piv = (int32_t *)calloc((size_t)d + 1, sizeof(int32_t));
  double *x = (double *)calloc((size_t)d + 1, sizeof(double));
  int rc = ORC_OK;
  if (!Dr || !Er || !piv || !x) { rc = ORC_OOM; goto out; }
  for (int32_t q = 0; q < d; ++q) {
    int32_t k = set[q], o = h->perm[k];
    for (int32_t e = h->rowptr[o]; e < h->rowptr[o + 1]; ++e) {
      int32_t c = h->pos[h->ccol[e]];
      if (c < nI && loc[c] >= 0) Dr[(int64_t)q * d + loc[c]] += h->cval[e];
    }
    for (int32_t e = h->E.ptr[k]; e < h->E.ptr[k + 1]; ++e) {
      int32_t c = h->E.col[e];
      if (c >= a0 && c < a1) Er[(int64_t)q * p + (c - a0)] += h->E.val[e];
    }
  }
  if (d > 0 && orc_dense_lu(d, Dr, piv, pivtol)) { rc = ORC_SINGULAR_SCHUR; goto out; }
  for (int32_t c = 0; c < p && d > 0; ++c) {
    for (int32_t q = 0; q < d; ++q) x[q] = Er[(int64_t)q * p + c];
    orc_dense_lu_solve(d, Dr, piv, x);
    for (int32_t r = 0; r < p; ++r) {
      double sacc = 0.0;
      for (int32_t q = h->F.ptr[a0 + r]; q < h->F.ptr[a0 + r + 1]; ++q) {
        int32_t j = h->F.col[q];
        if (loc[j] >= 0) sacc += h->F.val[q] * x[loc[j]];
      }
      S[(int64_t)r * p + c] -= sacc;
    }
  }
out:
  free(dist); free(set); free(loc); free(Dr); free(Er); free(piv); free(x);
  return rc;
}

/*
 * Build B for the given approximation kind (Algorithm 1).
 *   C          n x n CSR, original numbering (copied)
 *   part       subdomain 0..m-1 per node, -1 for the interface
 *   perm       new->old order (interiors of subdomain 0, 1, ..., then the
 *              interface); NULL: ascending index inside each group
 *   agg_off    nagg+1 aggregate offsets into the interface numbering, or
 *              NULL for consecutive chunks of sz (eq. aggrV)
 *   kind       0 EXACT, 1 MSCE_INF, 2 MSCN, 3 MSCNR, 4 LUM, -1 identity
 */
int orc_setup3(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, int32_t m,
               const int32_t *part, const int32_t *perm, int32_t nagg, const int32_t *agg_off,
               int32_t sz, int32_t kind, double pivtol, const int32_t *ovl, int32_t ovl_w, int32_t radius,
               double ilu_tol, orc **out) {
  *out = NULL;
  if (!(ilu_tol >= 0.0)) return ORC_INVALID_ARG;
  if (n <= 0 || m <= 0 || !rowptr || !col || !val || !part) return ORC_INVALID_ARG;
  if (kind < -1 || kind > 9 || kind == 5) return ORC_INVALID_ARG;
  if (kind == ORC_MSCE && radius < 0) return ORC_INVALID_ARG;
  if (rowptr[0] != 0) return ORC_INVALID_ARG;
  for (int32_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return ORC_INVALID_ARG;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= n) return ORC_INVALID_ARG;
      if (!isfinite(val[k])) return ORC_NONFINITE;
    }
  }
  for (int32_t i = 0; i < n; ++i) if (part[i] < -1 || part[i] >= m) return ORC_INVALID_PARTITION;
  /* the separator property: no entry couples two different interiors */
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int32_t j = col[k];
      if (part[i] >= 0 && part[j] >= 0 && part[i] != part[j] && val[k] != 0.0)
        return ORC_INVALID_PARTITION;
    }
  orc *h = (orc *)calloc(1, sizeof(orc));
  if (!h) return ORC_OOM;
  h->n = n; h->m = m; h->kind = kind; h->bad_block = -1; h->radius = radius; h->ilu_tol = ilu_tol;
  int rc = ORC_OK;
  h->rowptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  h->ccol = (int32_t *)malloc(sizeof(int32_t) * ((size_t)rowptr[n] + 1));
  h->cval = (double *)malloc(sizeof(double) * ((size_t)rowptr[n] + 1));
  h->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  h->pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  h->off = (int32_t *)calloc((size_t)m + 1, sizeof(int32_t));
  h->A = (orc_band *)calloc((size_t)m, sizeof(orc_band));
  if (!h->rowptr || !h->ccol || !h->cval || !h->perm || !h->pos || !h->off || !h->A) { rc = ORC_OOM; goto fail; }
  memcpy(h->rowptr, rowptr, sizeof(int32_t) * ((size_t)n + 1));
  memcpy(h->ccol, col, sizeof(int32_t) * (size_t)rowptr[n]);
  memcpy(h->cval, val, sizeof(double) * (size_t)rowptr[n]);
  /* ordering */
  for (int32_t i = 0; i < n; ++i) if (part[i] >= 0) h->off[part[i] + 1]++;
  for (int32_t j = 0; j < m; ++j) h->off[j + 1] += h->off[j];
  h->nI = h->off[m];
  h->nG = n - h->nI;
  if (perm) {
    for (int32_t i = 0; i < n; ++i) h->pos[i] = -1;
    for (int32_t k = 0; k < n; ++k) {
      int32_t o = perm[k];
      if (o < 0 || o >= n || h->pos[o] >= 0) { rc = ORC_INVALID_PARTITION; goto fail; }
      h->pos[o] = k;
      h->perm[k] = o;
      int32_t expect;
      if (k < h->nI) { expect = owner(h, k); if (part[o] != expect) { rc = ORC_INVALID_PARTITION; goto fail; } }
      else if (part[o] != -1) { rc = ORC_INVALID_PARTITION; goto fail; }
    }
  } else {
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
    if (!fill) { rc = ORC_OOM; goto fail; }
    memcpy(fill, h->off, sizeof(int32_t) * ((size_t)m + 1));
    int32_t g = h->nI;
    for (int32_t i = 0; i < n; ++i) {
      int32_t k = (part[i] >= 0) ? fill[part[i]]++ : g++;
      h->perm[k] = i;
      h->pos[i] = k;
    }
    free(fill);
  }
  /* aggregates of the interface numbering (eq. aggrV) */
  if (kind == ORC_EXACT) nagg = (h->nG > 0) ? 1 : 0;
  else if (!agg_off) {
    if (sz <= 0) { rc = ORC_INVALID_ARG; goto fail; }
    nagg = (h->nG + sz - 1) / sz;
  }
  h->nagg = nagg;
  h->agg = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nagg + 1));
  if (!h->agg) { rc = ORC_OOM; goto fail; }
  for (int32_t i = 0; i <= nagg; ++i) {
    if (kind == ORC_EXACT) h->agg[i] = i ? h->nG : 0;
    else if (agg_off) h->agg[i] = agg_off[i];
    else h->agg[i] = (i * sz < h->nG) ? i * sz : h->nG;
  }
  if (h->agg[0] != 0 || h->agg[nagg] != h->nG) { rc = ORC_INVALID_ARG; goto fail; }
  for (int32_t i = 0; i < nagg; ++i) if (h->agg[i + 1] <= h->agg[i]) { rc = ORC_INVALID_ARG; goto fail; }
  /* overlap widths (Algorithm 1): aggregate i is extended by w_i indices into
   * aggregate i + 1, 0 <= w_i <= p_{i+1}, and w_k = 0; given per aggregate,
   * or min(ovl_w, p_{i+1}) */
  h->ovl = (int32_t *)calloc((size_t)nagg + 1, sizeof(int32_t));
  if (!h->ovl) { rc = ORC_OOM; goto fail; }
  if (is_overlapped(kind))
    for (int32_t i = 0; i + 1 < nagg; ++i) {
      int32_t pn = h->agg[i + 2] - h->agg[i + 1];
      int32_t w = ovl ? ovl[i] : (ovl_w < pn ? ovl_w : pn);
      if (w < 0 || w > pn) { rc = ORC_INVALID_ARG; goto fail; }
      h->ovl[i] = w;
    }
  if (is_overlapped(kind) && ovl && nagg > 0 && ovl[nagg - 1] != 0) { rc = ORC_INVALID_ARG; goto fail; }
  /* blocks of P^T C P = [D E; F G] */
  if (extract_sp(h, 0, h->nI, h->nI, n, &h->E) || extract_sp(h, h->nI, n, 0, h->nI, &h->F) ||
      extract_sp(h, h->nI, n, h->nI, n, &h->G)) { rc = ORC_OOM; goto fail; }
  {
    int32_t nG = h->nG;
    h->Et.rows = nG;
    h->Et.ptr = (int32_t *)calloc((size_t)nG + 2, sizeof(int32_t));
    int32_t nzE = h->E.ptr[h->nI];
    h->Et.col = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nzE + 1));
    h->Et.val = (double *)malloc(sizeof(double) * ((size_t)nzE + 1));
    if (!h->Et.ptr || !h->Et.col || !h->Et.val) { rc = ORC_OOM; goto fail; }
    for (int32_t k = 0; k < nzE; ++k) h->Et.ptr[h->E.col[k] + 2]++;
    for (int32_t c = 0; c < nG; ++c) h->Et.ptr[c + 2] += h->Et.ptr[c + 1];
    for (int32_t r = 0; r < h->nI; ++r)
      for (int32_t k = h->E.ptr[r]; k < h->E.ptr[r + 1]; ++k) {
        int32_t w = h->Et.ptr[h->E.col[k] + 1]++;
        h->Et.col[w] = r;
        h->Et.val[w] = h->E.val[k];
      }
  }
  if (kind == ORC_IDENTITY) { *out = h; return ORC_OK; }
  /* exact LU of every interior block, subdomains independent */
  {
    int32_t bad = -1, brc = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < m; ++j) {
      int r = build_interior(h, j, pivtol);
      if (r != ORC_OK) {
#pragma omp critical
        { if (bad < 0 || j < bad) { bad = j; brc = r; } }
      }
    }
    if (bad >= 0) { h->bad_block = bad; rc = brc; goto fail_keep; }
  }
  /* mini Schur complements, aggregates independent */
  int32_t *dptr = NULL, *dadj = NULL;
  if (kind == ORC_MSCE && (rc = build_dadj(h, &dptr, &dadj)) != ORC_OK) goto fail;
  h->S = (double **)calloc((size_t)nagg + 1, sizeof(double *));
  h->Slu = (double **)calloc((size_t)nagg + 1, sizeof(double *));
  h->Spiv = (int32_t **)calloc((size_t)nagg + 1, sizeof(int32_t *));
  if (!h->S || !h->Slu || !h->Spiv) { rc = ORC_OOM; goto fail; }
  {
    int32_t bad = -1, brc = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < nagg; ++i) {
      /* the block's index range: the aggregate, extended by its overlap */
      int32_t a0 = h->agg[i], p = h->agg[i + 1] - a0 + h->ovl[i];
      int r = ORC_OK;
      h->S[i] = (double *)calloc((size_t)p * p, sizeof(double));
      h->Slu[i] = (double *)calloc((size_t)p * p, sizeof(double));
      h->Spiv[i] = (int32_t *)calloc((size_t)p, sizeof(int32_t));
      if (!h->S[i] || !h->Slu[i] || !h->Spiv[i]) r = ORC_OOM;
      else if (kind == ORC_EXACT || kind == ORC_MSCE_INF) r = schur_msce(h, i, h->S[i]);
      else if (kind == ORC_MSCN || kind == ORC_OMSCN) r = schur_mscn(h, a0, a0 + p, h->S[i], 0, pivtol);
      else if (kind == ORC_MSCNR || kind == ORC_OMSCNR) r = schur_mscn(h, a0, a0 + p, h->S[i], 1, pivtol);
      else if (kind == ORC_MSCE) r = schur_msce_r(h, i, h->S[i], dptr, dadj, pivtol);
      else
        for (int32_t a = 0; a < p; ++a)
          for (int32_t c = 0; c < p; ++c)
            h->S[i][(int64_t)a * p + c] = sp_get(&h->G, a0 + a, a0 + c);
      /* overlapped kinds: only the assembled S_hat is factored (below) */
      if (r == ORC_OK && !is_overlapped(kind)) {
        memcpy(h->Slu[i], h->S[i], sizeof(double) * (size_t)p * p);
        if (orc_dense_lu(p, h->Slu[i], h->Spiv[i], pivtol)) r = ORC_SINGULAR_SCHUR;
      }
      if (r != ORC_OK) {
#pragma omp critical
        { if (bad < 0 || i < bad) { bad = i; brc = r; } }
      }
    }
    free(dptr);
    free(dadj);
    if (bad >= 0) { h->bad_block = bad; rc = brc; goto fail_keep; }
  }
  if (is_overlapped(kind) && nagg > 0) {
    /* S_hat with overlapping blocks (the Remark on overlapped aggregation):
     * every S_ii is placed at its index range, aggregate after aggregate,
     * a later block overwriting the overlap.  S_hat is then a band matrix,
     * no longer block diagonal, and is factored whole. */
    int32_t bw = 0;
    for (int32_t i = 0; i < nagg; ++i) {
      int32_t q = h->agg[i + 1] - h->agg[i] + h->ovl[i];
      if (q - 1 > bw) bw = q - 1;
    }
    if (band_alloc(&h->Shat, h->nG, bw, bw)) { rc = ORC_OOM; goto fail; }
    for (int32_t i = 0; i < nagg; ++i) {
      int32_t a0 = h->agg[i], q = h->agg[i + 1] - a0 + h->ovl[i];
      for (int32_t r = 0; r < q; ++r)
        for (int32_t c = 0; c < q; ++c) *band_at(&h->Shat, a0 + r, a0 + c) = h->S[i][(int64_t)r * q + c];
    }
    size_t nb = (size_t)h->nG * h->Shat.wd;
    h->Shat0 = (double *)malloc(sizeof(double) * (nb + 1));
    if (!h->Shat0) { rc = ORC_OOM; goto fail; }
    memcpy(h->Shat0, h->Shat.r, sizeof(double) * nb);
    if (band_factor(&h->Shat, pivtol, 0.0, NULL)) { h->bad_block = nagg; rc = ORC_SINGULAR_SCHUR; goto fail_keep; }
  }
  *out = h;
  return ORC_OK;
fail_keep:
  /* keep the handle so a caller can read bad_block; it cannot be applied */
  h->kind = -2;
  *out = h;
  return rc;
fail:
  orc_free(h);
  return rc;
}

int orc_setup2(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, int32_t m,
               const int32_t *part, const int32_t *perm, int32_t nagg, const int32_t *agg_off,
               int32_t sz, int32_t kind, double pivtol, const int32_t *ovl, int32_t ovl_w, int32_t radius,
               orc **out) {
  return orc_setup3(n, rowptr, col, val, m, part, perm, nagg, agg_off, sz, kind, pivtol, ovl, ovl_w, radius, 0.0,
                    out);
}

int orc_setup(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, int32_t m,
              const int32_t *part, const int32_t *perm, int32_t nagg, const int32_t *agg_off,
              int32_t sz, int32_t kind, double pivtol, orc **out) {
  return orc_setup2(n, rowptr, col, val, m, part, perm, nagg, agg_off, sz, kind, pivtol, NULL, 0, 0, out);
}

int32_t orc_bad_block(const orc *h) { return h ? h->bad_block : -1; }

/* rows of S_hat block i (the aggregate plus its overlap) */
int32_t orc_block_size(const orc *h, int32_t i) {
  if (!h || i < 0 || i >= h->nagg) return -1;
  return h->agg[i + 1] - h->agg[i] + (h->ovl ? h->ovl[i] : 0);
}

/* the overlap widths w_i (nagg entries) */
void orc_overlaps(const orc *h, int32_t *o) {
  for (int32_t i = 0; i < h->nagg; ++i) o[i] = h->ovl ? h->ovl[i] : 0;
}

/* S_hat as a dense nG x nG row-major matrix (before any factorisation) */
int orc_schur_dense(const orc *h, double *o) {
  if (!h->S || h->kind == -2) return -1;
  int32_t nG = h->nG;
  memset(o, 0, sizeof(double) * (size_t)nG * nG);
  if (is_overlapped(h->kind)) {
    int32_t kl = h->Shat.kl, ku = h->Shat.ku, wd = h->Shat.wd;
    for (int32_t r = 0; r < nG; ++r)
      for (int32_t c = r - kl; c <= r + ku; ++c)
        if (c >= 0 && c < nG) o[(int64_t)r * nG + c] = h->Shat0[(int64_t)r * wd + (c - r + kl)];
    return 0;
  }
  for (int32_t i = 0; i < h->nagg; ++i) {
    int32_t a0 = h->agg[i], p = h->agg[i + 1] - a0;
    for (int32_t r = 0; r < p; ++r)
      for (int32_t c = 0; c < p; ++c) o[(int64_t)(a0 + r) * nG + a0 + c] = h->S[i][(int64_t)r * p + c];
  }
  return 0;
}

/* n, m, nI, nG, nagg, kind */
void orc_sizes(const orc *h, int64_t *o) {
  o[0] = h->n; o[1] = h->m; o[2] = h->nI; o[3] = h->nG; o[4] = h->nagg; o[5] = h->kind;
}

void orc_agg_offsets(const orc *h, int32_t *o) { memcpy(o, h->agg, sizeof(int32_t) * ((size_t)h->nagg + 1)); }
void orc_perm(const orc *h, int32_t *o) { memcpy(o, h->perm, sizeof(int32_t) * (size_t)h->n); }
void orc_interior_offsets(const orc *h, int32_t *o) { memcpy(o, h->off, sizeof(int32_t) * ((size_t)h->m + 1)); }
/* bandwidths (kl, ku) of every interior block */
void orc_bandwidths(const orc *h, int32_t *o) {
  for (int32_t j = 0; j < h->m; ++j) { o[2 * j] = h->A[j].kl; o[2 * j + 1] = h->A[j].ku; }
}

/* Replace S_hat block i by blk (row-major, p x p) when blk passes the pivot
 * test of its LU; otherwise keep the block it had (the fallback of the
 * learned approximation) and return ORC_SINGULAR_SCHUR. */
int orc_replace_block(orc *h, int32_t i, const double *blk, double pivtol) {
  if (!h->S || i < 0 || i >= h->nagg || !h->S[i] || h->kind == -2) return ORC_INVALID_ARG;
  int32_t p = h->agg[i + 1] - h->agg[i];
  double *lu = (double *)malloc(sizeof(double) * (size_t)p * p);
  int32_t *piv = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
  if (!lu || !piv) { free(lu); free(piv); return ORC_OOM; }
  memcpy(lu, blk, sizeof(double) * (size_t)p * p);
  if (orc_dense_lu(p, lu, piv, pivtol)) { free(lu); free(piv); return ORC_SINGULAR_SCHUR; }
  memcpy(h->S[i], blk, sizeof(double) * (size_t)p * p);
  free(h->Slu[i]);
  free(h->Spiv[i]);
  h->Slu[i] = lu;
  h->Spiv[i] = piv;
  return ORC_OK;
}

/* copy S_hat block i (row-major, unfactored) */
int orc_schur_block(const orc *h, int32_t i, double *o) {
  if (!h->S || i < 0 || i >= h->nagg || !h->S[i]) return -1;
  int32_t p = orc_block_size(h, i);
  memcpy(o, h->S[i], sizeof(double) * (size_t)p * p);
  return 0;
}

/* ======================================================================== */
/* Apply x = B^-1 y (Algorithm 2, with the E/F reading stated above)        */
/* ======================================================================== */
int orc_apply(const orc *h, const double *y, double *x) {
  int32_t n = h->n, nI = h->nI, nG = h->nG;
  if (h->kind == -2) return ORC_INVALID_ARG;
  if (h->kind == ORC_IDENTITY) { memcpy(x, y, sizeof(double) * (size_t)n); return ORC_OK; }
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  double *u = (double *)malloc(sizeof(double) * ((size_t)nI + 1));
  if (!z || !u) { free(z); free(u); return ORC_OOM; }
  for (int32_t k = 0; k < n; ++k) z[k] = y[h->perm[k]];
  /* forward sweep: z1 = D^-1 y1, subdomain by subdomain */
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t j = 0; j < h->m; ++j)
    if (h->A[j].n) band_solve(&h->A[j], z + h->off[j]);
  /* z2_i = S_ii^-1 (y2 - F z1)_i */
  double *t = z + nI;
  for (int32_t r = 0; r < nG; ++r) {
    double s = 0.0;
    for (int32_t k = h->F.ptr[r]; k < h->F.ptr[r + 1]; ++k) s += h->F.val[k] * z[h->F.col[k]];
    t[r] -= s;
  }
  if (is_overlapped(h->kind)) {
    if (nG > 0) band_solve(&h->Shat, t); /* the assembled S_hat: one band solve */
  } else {
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < h->nagg; ++i)
      orc_dense_lu_solve(h->agg[i + 1] - h->agg[i], h->Slu[i], h->Spiv[i], t + h->agg[i]);
  }
  /* backward sweep: x2 = z2, x1 = z1 - D^-1 (E x2) */
  for (int32_t r = 0; r < nI; ++r) {
    double s = 0.0;
    for (int32_t k = h->E.ptr[r]; k < h->E.ptr[r + 1]; ++k) s += h->E.val[k] * t[h->E.col[k]];
    u[r] = s;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t j = 0; j < h->m; ++j)
    if (h->A[j].n) band_solve(&h->A[j], u + h->off[j]);
  for (int32_t r = 0; r < nI; ++r) z[r] -= u[r];
  for (int32_t k = 0; k < n; ++k) x[h->perm[k]] = z[k];
  free(z);
  free(u);
  return ORC_OK;
}

/* ======================================================================== */
/* Right-preconditioned restarted flexible GMRES (Section 5)                */
/* ======================================================================== */
static void csr_mv(const orc *h, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < h->n; ++i) {
    double s = 0.0;
    for (int32_t k = h->rowptr[i]; k < h->rowptr[i + 1]; ++k) s += h->cval[k] * x[h->ccol[k]];
    y[i] = s;
  }
}

static double dot(int32_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/*
 * Solve C x = b with x0 = 0.  Each Arnoldi step: z_j = B^-1 v_j,
 * w = C z_j, classical Gram-Schmidt applied twice (CGS2), Givens rotations
 * (r = hypot(a, b), c = a/r, s = b/r).  The inner loop stops when the Givens
 * residual estimate |g_{j+1}| / ||b|| <= tol, on a breakdown
 * (h_{j+1,j} <= 1e-14 ||w before orthogonalisation||) or at maxit; then
 * x += Z y, and the true residual decides between stopping and restarting.
 * iters counts Arnoldi steps over all restarts; hist[k] is the estimate
 * after step k (up to hist_cap entries).  Returns 0, 5 (not converged, x is
 * the last iterate) or 6 (non-finite residual).
 */
int orc_fgmres(const orc *h, const double *b, double *x, double tol, int32_t restart, int32_t maxit,
               int32_t *iters_out, int32_t *restarts_out, double *relres_out, double *hist,
               int32_t hist_cap) {
  int32_t n = h->n, R = restart;
  *iters_out = 0;
  if (restarts_out) *restarts_out = 0;
  *relres_out = 0.0;
  if (R <= 0 || maxit <= 0) return ORC_INVALID_ARG;
  for (int32_t i = 0; i < n; ++i) if (!isfinite(b[i])) return ORC_NONFINITE;
  double nb = sqrt(dot(n, b, b));
  for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
  if (nb == 0.0) return ORC_OK;
  double *V = (double *)malloc(sizeof(double) * (size_t)n * (R + 1));
  double *Z = (double *)malloc(sizeof(double) * (size_t)n * R);
  double *H = (double *)calloc((size_t)(R + 1) * R, sizeof(double)); /* H[i*R + j] */
  double *cs = (double *)calloc((size_t)R, sizeof(double));
  double *sn = (double *)calloc((size_t)R, sizeof(double));
  double *g = (double *)calloc((size_t)R + 1, sizeof(double));
  double *hc = (double *)calloc((size_t)R + 1, sizeof(double));
  double *yv = (double *)calloc((size_t)R + 1, sizeof(double));
  double *r = (double *)malloc(sizeof(double) * (size_t)n);
  int rc = ORC_NOT_CONVERGED;
  int32_t iters = 0, restarts = 0;
  if (!V || !Z || !H || !cs || !sn || !g || !hc || !yv || !r) { rc = ORC_OOM; goto out; }
  memcpy(r, b, sizeof(double) * (size_t)n);
  for (;;) {
    double beta = sqrt(dot(n, r, r));
    if (!isfinite(beta)) { rc = ORC_NONFINITE; break; }
    for (int32_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int32_t q = 0; q <= R; ++q) g[q] = 0.0;
    g[0] = beta;
    int32_t jlast = -1;
    for (int32_t j = 0; j < R; ++j) {
      double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n, *w = V + (size_t)(j + 1) * n;
      orc_apply(h, vj, zj);
      csr_mv(h, zj, w);
      double w0 = sqrt(dot(n, w, w));
      for (int32_t q = 0; q <= j; ++q) H[(size_t)q * R + j] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int32_t q = 0; q <= j; ++q) hc[q] = dot(n, V + (size_t)q * n, w);
        for (int32_t q = 0; q <= j; ++q) {
          const double *vq = V + (size_t)q * n;
          for (int32_t i = 0; i < n; ++i) w[i] -= hc[q] * vq[i];
          H[(size_t)q * R + j] += hc[q];
        }
      }
      double hn = sqrt(dot(n, w, w));
      H[(size_t)(j + 1) * R + j] = hn;
      int breakdown = !(hn > 1e-14 * w0);
      if (!breakdown) for (int32_t i = 0; i < n; ++i) w[i] /= hn;
      for (int32_t q = 0; q < j; ++q) {
        double a = H[(size_t)q * R + j], c2 = H[(size_t)(q + 1) * R + j];
        H[(size_t)q * R + j] = cs[q] * a + sn[q] * c2;
        H[(size_t)(q + 1) * R + j] = -sn[q] * a + cs[q] * c2;
      }
      double a = H[(size_t)j * R + j], c2 = H[(size_t)(j + 1) * R + j];
      double rr = hypot(a, c2);
      cs[j] = a / rr;
      sn[j] = c2 / rr;
      H[(size_t)j * R + j] = rr;
      H[(size_t)(j + 1) * R + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      double est = fabs(g[j + 1]) / nb;
      if (hist && iters - 1 < hist_cap) hist[iters - 1] = est;
      jlast = j;
      if (!isfinite(est)) { rc = ORC_NONFINITE; goto out; }
      if (est <= tol || breakdown || iters >= maxit) break;
    }
    /* y = H^-1 g (upper triangular), x += Z y */
    for (int32_t q = jlast; q >= 0; --q) {
      double s = g[q];
      for (int32_t c = q + 1; c <= jlast; ++c) s -= H[(size_t)q * R + c] * yv[c];
      yv[q] = s / H[(size_t)q * R + q];
    }
    for (int32_t q = 0; q <= jlast; ++q) {
      const double *zq = Z + (size_t)q * n;
      for (int32_t i = 0; i < n; ++i) x[i] += yv[q] * zq[i];
    }
    csr_mv(h, x, r);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double rel = sqrt(dot(n, r, r)) / nb;
    *relres_out = rel;
    if (!isfinite(rel)) { rc = ORC_NONFINITE; break; }
    if (rel <= tol) { rc = ORC_OK; break; }
    if (iters >= maxit) { rc = ORC_NOT_CONVERGED; break; }
    ++restarts;
  }
out:
  *iters_out = iters;
  if (restarts_out) *restarts_out = restarts;
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(hc); free(yv); free(r);
  return rc;
}

/* Stand-alone sparse matrix-vector product y = C x (pin helper). */
void orc_spmv(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
              const double *x, double *y) {
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}
