/*
 * Seeded synthetic workload generator: MAC finite-volume Oseen systems and
 * their algebraic (graph) partition.
 *
 * This module produces INPUTS only: the saddle-point matrix C = [D E^T; -E 0]
 * of the linearised (Picard/Oseen) Navier-Stokes equations (Section 1 of the
 * paper), a right-hand side, and the vertex-separator partition P^T C P whose
 * interiors become the (1,1) blocks A_ii and whose separator becomes the
 * interface (Section 1, the graph-partitioner paragraph; Section 3.2, matrix
 * view).  It holds none of the preconditioner's arithmetic: no factorisation,
 * no Schur complement, no Krylov step.  Both the CUDA library and the CPU
 * oracle consume what it writes.
 *
 * Discretisation (the paper used Q2-Q1 elements from IFISS; those matrices are
 * not available, a MAC staggered finite-volume system stands in for them):
 *   unknowns   p at cell centres, u at interior vertical faces, v at interior
 *              horizontal faces; numbered cell-interleaved, row-major over
 *              cells (p, then u if the cell has an east interior face, then v
 *              if it has a north interior face).
 *   momentum   integrated over the face control volume: two-point diffusion
 *              nu*A_f/dist, first-order upwind convection with face fluxes
 *              equal to exact stream-function differences (so every control
 *              volume is discretely divergence free), pressure force
 *              (p_E - p_W) * A.
 *   continuity integrated over the cell: sum of outward normal velocities
 *              times face lengths (Div_FV).  C = [D, Grad; Div, 0] with
 *              Grad = -Div^T exactly, i.e. E = -Div and E^T = Grad.
 *   walls      no-slip; tangential velocity by a mirror ghost (half-distance
 *              flux), lid velocity 1 on y = 1.
 *   pin        p(0,0) row and column replaced by the identity.
 *   scaling    each row divided by its largest absolute entry (Section 5).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Random numbers: xoshiro256** seeded through SplitMix64 (Blackman & Vigna) */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t s[4]; } ddg_rng;

static uint64_t splitmix64_next(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(ddg_rng *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static uint64_t rng_next(ddg_rng *r) {
  uint64_t *s = r->s;
  uint64_t result = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return result;
}

/* uniform in [0,1) with 53 random bits */
static double rng_uniform(ddg_rng *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* Fill out[0..n) with uniform values in [lo, hi) from xoshiro256**(seed). */
void ddg_uniform(uint64_t seed, int64_t n, double lo, double hi, double *out) {
  ddg_rng r;
  rng_seed(&r, seed);
  for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * rng_uniform(&r);
}

/* Raw 64-bit stream, exposed so tests can compare against published vectors. */
void ddg_raw(uint64_t seed, int64_t n, uint64_t *out) {
  ddg_rng r;
  rng_seed(&r, seed);
  for (int64_t i = 0; i < n; ++i) out[i] = rng_next(&r);
}

/* ------------------------------------------------------------------------ */
/* Grid and wind                                                             */
/* ------------------------------------------------------------------------ */
#define DDG_MODES 8
#define DDG_PI 3.14159265358979323846

typedef struct {
  int n;
  double *X, *Y;   /* face lines, n+1 each */
  double *Xc, *Yc; /* cell centres, n each */
  double *hx, *hy; /* cell widths */
  int wind;        /* 0: none, 1: (1-x^2)(1-y^2), 2: seeded Fourier modes */
  double amp;      /* stream function scale for wind 2 */
  int mk[DDG_MODES], nk[DDG_MODES];
  double ak[DDG_MODES];
} ddg_grid;

/* Cell widths: symmetric geometric spacing h_k ~ r^k from each wall. */
void ddg_spacing(int n, double r, double *h) {
  int half = n / 2;
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    int d = (k < half) ? k : (n - 1 - k);
    h[k] = pow(r, (double)d);
    s += h[k];
  }
  for (int k = 0; k < n; ++k) h[k] /= s;
}

static double psi_raw(const ddg_grid *g, double x, double y) {
  if (g->wind == 1) return (1.0 - x * x) * (1.0 - y * y);
  if (g->wind == 2) {
    double s = 0.0;
    for (int k = 0; k < DDG_MODES; ++k)
      s += g->ak[k] * sin(DDG_PI * g->mk[k] * x) * sin(DDG_PI * g->nk[k] * y);
    return s;
  }
  return 0.0;
}

static double psi(const ddg_grid *g, double x, double y) { return g->amp * psi_raw(g, x, y); }

/* analytic wind w = (-psi_y, psi_x) of the unscaled stream function */
static void wind_raw(const ddg_grid *g, double x, double y, double *wx, double *wy) {
  if (g->wind == 1) {
    *wx = 2.0 * y * (1.0 - x * x);
    *wy = -2.0 * x * (1.0 - y * y);
    return;
  }
  double px = 0.0, py = 0.0;
  if (g->wind == 2) {
    for (int k = 0; k < DDG_MODES; ++k) {
      double a = g->ak[k], m = DDG_PI * g->mk[k], q = DDG_PI * g->nk[k];
      px += a * m * cos(m * x) * sin(q * y);
      py += a * q * sin(m * x) * cos(q * y);
    }
  }
  *wx = -py;
  *wy = px;
}

static int grid_init(ddg_grid *g, int n, double stretch, int wind, uint64_t wind_seed) {
  memset(g, 0, sizeof(*g));
  g->n = n;
  g->X = (double *)malloc(sizeof(double) * (n + 1));
  g->Y = (double *)malloc(sizeof(double) * (n + 1));
  g->Xc = (double *)malloc(sizeof(double) * n);
  g->Yc = (double *)malloc(sizeof(double) * n);
  g->hx = (double *)malloc(sizeof(double) * n);
  g->hy = (double *)malloc(sizeof(double) * n);
  if (!g->X || !g->Y || !g->Xc || !g->Yc || !g->hx || !g->hy) return -1;
  ddg_spacing(n, stretch, g->hx);
  ddg_spacing(n, stretch, g->hy);
  g->X[0] = 0.0;
  g->Y[0] = 0.0;
  for (int i = 0; i < n; ++i) {
    g->X[i + 1] = g->X[i] + g->hx[i];
    g->Y[i + 1] = g->Y[i] + g->hy[i];
  }
  g->X[n] = 1.0;
  g->Y[n] = 1.0;
  for (int i = 0; i < n; ++i) {
    g->Xc[i] = 0.5 * (g->X[i] + g->X[i + 1]);
    g->Yc[i] = 0.5 * (g->Y[i] + g->Y[i + 1]);
  }
  g->wind = wind;
  g->amp = 1.0;
  if (wind == 2) {
    ddg_rng r;
    rng_seed(&r, wind_seed);
    for (int k = 0; k < DDG_MODES; ++k) {
      g->mk[k] = 1 + (int)(4.0 * rng_uniform(&r));
      g->nk[k] = 1 + (int)(4.0 * rng_uniform(&r));
      double u1 = 1.0 - rng_uniform(&r); /* (0,1] */
      double u2 = rng_uniform(&r);
      g->ak[k] = sqrt(-2.0 * log(u1)) * cos(2.0 * DDG_PI * u2);
    }
    /* scale so that max |w| over all interior face centres is 1 */
    double wmax = 0.0, wx, wy;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i + 1 < n; ++i) {
        wind_raw(g, g->X[i + 1], g->Yc[j], &wx, &wy);
        double a = sqrt(wx * wx + wy * wy);
        if (a > wmax) wmax = a;
      }
    for (int j = 0; j + 1 < n; ++j)
      for (int i = 0; i < n; ++i) {
        wind_raw(g, g->Xc[i], g->Y[j + 1], &wx, &wy);
        double a = sqrt(wx * wx + wy * wy);
        if (a > wmax) wmax = a;
      }
    g->amp = (wmax > 0.0) ? 1.0 / wmax : 1.0;
  }
  return 0;
}

static void grid_free(ddg_grid *g) {
  free(g->X); free(g->Y); free(g->Xc); free(g->Yc); free(g->hx); free(g->hy);
}

/* Exposes the wind scale and modes (for documentation and tests). */
int ddg_wind_info(int n, double stretch, int wind, uint64_t wind_seed, double *amp,
                  int32_t *mk, int32_t *nk, double *ak) {
  ddg_grid g;
  if (grid_init(&g, n, stretch, wind, wind_seed)) { grid_free(&g); return -1; }
  *amp = g.amp;
  for (int k = 0; k < DDG_MODES; ++k) { mk[k] = g.mk[k]; nk[k] = g.nk[k]; ak[k] = g.ak[k]; }
  grid_free(&g);
  return 0;
}

/* Unknown numbering: cell-interleaved, row-major over cells. */
int64_t ddg_mac_size(int n) { return 3LL * n * n - 2LL * n; }

int64_t ddg_mac_nnz_bound(int n) {
  return 7LL * 2 * (int64_t)(n - 1) * n + 4LL * n * n;
}

static void mac_index(int n, int32_t *ip, int32_t *iu, int32_t *iv) {
  int32_t k = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      int c = j * n + i;
      ip[c] = k++;
      iu[c] = (i < n - 1) ? k++ : -1;
      iv[c] = (j < n - 1) ? k++ : -1;
    }
}

/* Exposes the numbering: for every unknown its kind (0 p, 1 u, 2 v) and cell. */
void ddg_mac_layout(int n, int8_t *kind, int32_t *cell) {
  int32_t k = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      int c = j * n + i;
      kind[k] = 0; cell[k++] = c;
      if (i < n - 1) { kind[k] = 1; cell[k++] = c; }
      if (j < n - 1) { kind[k] = 2; cell[k++] = c; }
    }
}

/* ------------------------------------------------------------------------ */
/* Assembly                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t c[16];
  double v[16];
  int k;
} rowbuf;

static void rb_add(rowbuf *r, int32_t c, double v) {
  for (int i = 0; i < r->k; ++i)
    if (r->c[i] == c) { r->v[i] += v; return; }
  r->c[r->k] = c;
  r->v[r->k++] = v;
}

static void rb_sort(rowbuf *r) {
  for (int i = 1; i < r->k; ++i) {
    int32_t c = r->c[i];
    double v = r->v[i];
    int j = i - 1;
    while (j >= 0 && r->c[j] > c) { r->c[j + 1] = r->c[j]; r->v[j + 1] = r->v[j]; --j; }
    r->c[j + 1] = c;
    r->v[j + 1] = v;
  }
}

/* one control-volume face: two-point diffusion plus first-order upwind
 * convection; nb < 0 means a wall with Dirichlet value g */
static void cv_face(rowbuf *r, double *diag, double *rhs, int32_t nb, double g, double nu,
                    double area, double dist, double F) {
  double a = nu * area / dist;
  *diag += a + (F > 0.0 ? F : 0.0);
  double coef = -a + (F < 0.0 ? F : 0.0);
  if (nb >= 0) rb_add(r, nb, coef);
  else *rhs -= coef * g;
}

/*
 * Assemble the MAC Oseen matrix on an n x n grid.
 *   nu       viscosity
 *   stretch  geometric ratio r of neighbouring cell widths (1 = uniform)
 *   wind     0 none, 1 w = (2y(1-x^2), -2x(1-y^2)), 2 seeded Fourier modes
 *   lid      tangential wall velocity on y = 1
 *   pin      replace row/column of p(0,0) by the identity
 *   scale    divide each row (and rhs entry) by its max-abs entry
 * rowptr must hold N+1 entries, col/val ddg_mac_nnz_bound(n), rhs N.
 * Returns nnz, or -1 on allocation failure.
 */
int64_t ddg_mac_assemble(int n, double nu, double stretch, int wind, uint64_t wind_seed,
                         double lid, int pin, int scale, int32_t *rowptr, int32_t *col,
                         double *val, double *rhs) {
  ddg_grid g;
  if (grid_init(&g, n, stretch, wind, wind_seed)) { grid_free(&g); return -1; }
  int32_t *ip = (int32_t *)malloc(sizeof(int32_t) * n * n);
  int32_t *iu = (int32_t *)malloc(sizeof(int32_t) * n * n);
  int32_t *iv = (int32_t *)malloc(sizeof(int32_t) * n * n);
  if (!ip || !iu || !iv) { free(ip); free(iu); free(iv); grid_free(&g); return -1; }
  mac_index(n, ip, iu, iv);
  const double *X = g.X, *Y = g.Y, *Xc = g.Xc, *Yc = g.Yc, *hx = g.hx, *hy = g.hy;
  int64_t nz = 0;
  int32_t row = 0;
  rowptr[0] = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      int c = j * n + i;
      for (int kind = 0; kind < 3; ++kind) {
        rowbuf r;
        r.k = 0;
        double b = 0.0;
        if (kind == 0) { /* continuity: Div_FV of the cell */
          if (i < n - 1) rb_add(&r, iu[c], hy[j]);
          if (i > 0) rb_add(&r, iu[c - 1], -hy[j]);
          if (j < n - 1) rb_add(&r, iv[c], hx[i]);
          if (j > 0) rb_add(&r, iv[c - n], -hx[i]);
        } else if (kind == 1) { /* u-momentum at face (i+1/2, j) */
          if (i >= n - 1) continue;
          double xw = Xc[i], xe = Xc[i + 1], ys = Y[j], yn = Y[j + 1], d = 0.0;
          cv_face(&r, &d, &b, (i + 1 <= n - 2) ? iu[c + 1] : -1, 0.0, nu, hy[j], hx[i + 1],
                  psi(&g, xe, ys) - psi(&g, xe, yn));
          cv_face(&r, &d, &b, (i >= 1) ? iu[c - 1] : -1, 0.0, nu, hy[j], hx[i],
                  psi(&g, xw, yn) - psi(&g, xw, ys));
          if (j <= n - 2)
            cv_face(&r, &d, &b, iu[c + n], 0.0, nu, xe - xw, 0.5 * (hy[j] + hy[j + 1]),
                    psi(&g, xe, yn) - psi(&g, xw, yn));
          else
            cv_face(&r, &d, &b, -1, lid, nu, xe - xw, 0.5 * hy[j], psi(&g, xe, yn) - psi(&g, xw, yn));
          if (j >= 1)
            cv_face(&r, &d, &b, iu[c - n], 0.0, nu, xe - xw, 0.5 * (hy[j - 1] + hy[j]),
                    psi(&g, xw, ys) - psi(&g, xe, ys));
          else
            cv_face(&r, &d, &b, -1, 0.0, nu, xe - xw, 0.5 * hy[j], psi(&g, xw, ys) - psi(&g, xe, ys));
          rb_add(&r, iu[c], d);
          rb_add(&r, ip[c + 1], hy[j]);
          rb_add(&r, ip[c], -hy[j]);
        } else { /* v-momentum at face (i, j+1/2) */
          if (j >= n - 1) continue;
          double xw = X[i], xe = X[i + 1], ys = Yc[j], yn = Yc[j + 1], d = 0.0;
          cv_face(&r, &d, &b, (j + 1 <= n - 2) ? iv[c + n] : -1, 0.0, nu, hx[i], hy[j + 1],
                  psi(&g, xe, yn) - psi(&g, xw, yn));
          cv_face(&r, &d, &b, (j >= 1) ? iv[c - n] : -1, 0.0, nu, hx[i], hy[j],
                  psi(&g, xw, ys) - psi(&g, xe, ys));
          if (i <= n - 2)
            cv_face(&r, &d, &b, iv[c + 1], 0.0, nu, yn - ys, 0.5 * (hx[i] + hx[i + 1]),
                    psi(&g, xe, ys) - psi(&g, xe, yn));
          else
            cv_face(&r, &d, &b, -1, 0.0, nu, yn - ys, 0.5 * hx[i], psi(&g, xe, ys) - psi(&g, xe, yn));
          if (i >= 1)
            cv_face(&r, &d, &b, iv[c - 1], 0.0, nu, yn - ys, 0.5 * (hx[i - 1] + hx[i]),
                    psi(&g, xw, yn) - psi(&g, xw, ys));
          else
            cv_face(&r, &d, &b, -1, 0.0, nu, yn - ys, 0.5 * hx[i], psi(&g, xw, yn) - psi(&g, xw, ys));
          rb_add(&r, iv[c], d);
          rb_add(&r, ip[c + n], hx[i]);
          rb_add(&r, ip[c], -hx[i]);
        }
        if (pin) {
          if (row == ip[0]) { r.k = 0; rb_add(&r, row, 1.0); b = 0.0; }
          else {
            int w = 0;
            for (int q = 0; q < r.k; ++q)
              if (r.c[q] != ip[0]) { r.c[w] = r.c[q]; r.v[w++] = r.v[q]; }
            r.k = w;
          }
        }
        rb_sort(&r);
        double mx = 0.0;
        for (int q = 0; q < r.k; ++q) if (fabs(r.v[q]) > mx) mx = fabs(r.v[q]);
        for (int q = 0; q < r.k; ++q) {
          col[nz] = r.c[q];
          val[nz] = (scale && mx > 0.0) ? r.v[q] / mx : r.v[q];
          ++nz;
        }
        rhs[row] = (scale && mx > 0.0) ? b / mx : b;
        ++row;
        rowptr[row] = (int32_t)nz;
      }
    }
  free(ip); free(iu); free(iv);
  grid_free(&g);
  return nz;
}

/* ------------------------------------------------------------------------ */
/* Algebraic partition: recursive BFS level-set bisection of the graph of    */
/* C + C^T, separator trimming, enclosed-pressure repair, RCM inside each    */
/* subdomain.  Only the sparsity pattern (and, for the pressure test, the    */
/* values) of C are used: nothing is assumed about the grid.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n;
  int32_t *xadj, *adj;
} ddg_graph;

static int graph_build(int32_t n, const int32_t *rowptr, const int32_t *col, ddg_graph *g) {
  g->n = n;
  g->xadj = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t *cnt = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  if (!g->xadj || !cnt) { free(cnt); return -1; }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int32_t j = col[k];
      if (j == i) continue;
      cnt[i + 1]++;
      cnt[j + 1]++;
    }
  for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cnt[n] + 1));
  int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!tmp || !pos) { free(cnt); free(tmp); free(pos); return -1; }
  memcpy(pos, cnt, sizeof(int32_t) * ((size_t)n + 1));
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int32_t j = col[k];
      if (j == i) continue;
      tmp[pos[i]++] = j;
      tmp[pos[j]++] = i;
    }
  /* sort + dedupe each list (lists are short: insertion sort) */
  int32_t w = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t a = cnt[i], b = cnt[i + 1];
    for (int32_t p = a + 1; p < b; ++p) {
      int32_t v = tmp[p], q = p - 1;
      while (q >= a && tmp[q] > v) { tmp[q + 1] = tmp[q]; --q; }
      tmp[q + 1] = v;
    }
    g->xadj[i] = w;
    for (int32_t p = a; p < b; ++p)
      if (p == a || tmp[p] != tmp[p - 1]) tmp[w++] = tmp[p];
  }
  g->xadj[n] = w;
  g->adj = tmp;
  free(cnt);
  free(pos);
  return 0;
}

typedef struct {
  int32_t *queue;  /* BFS order */
  int32_t *lstart; /* level starts into queue, nlev+1 entries */
  int32_t nlev;
  int32_t *stamp;  /* visit stamps */
  int32_t cur;
} ddg_bfs;

static int32_t deg_in(const ddg_graph *g, const int32_t *label, int32_t lab, int32_t v) {
  int32_t d = 0;
  for (int32_t k = g->xadj[v]; k < g->xadj[v + 1]; ++k) d += (label[g->adj[k]] == lab);
  return d;
}

/* level-set BFS from root inside the nodes carrying label lab; returns count */
static int32_t bfs_levels(const ddg_graph *g, const int32_t *label, int32_t lab, int32_t root,
                          ddg_bfs *b) {
  int32_t st = ++b->cur;
  int32_t head = 0, tail = 0;
  b->queue[tail++] = root;
  b->stamp[root] = st;
  b->nlev = 0;
  b->lstart[0] = 0;
  while (head < tail) {
    int32_t lend = tail;
    b->lstart[++b->nlev] = lend;
    for (; head < lend; ++head) {
      int32_t v = b->queue[head];
      for (int32_t k = g->xadj[v]; k < g->xadj[v + 1]; ++k) {
        int32_t u = g->adj[k];
        if (label[u] == lab && b->stamp[u] != st) {
          b->stamp[u] = st;
          b->queue[tail++] = u;
        }
      }
    }
  }
  b->lstart[b->nlev] = tail;
  return tail;
}

/* George-Liu pseudo-peripheral node search starting from s */
static int32_t pseudo_peripheral(const ddg_graph *g, const int32_t *label, int32_t lab, int32_t s,
                                 ddg_bfs *b) {
  int32_t root = s;
  bfs_levels(g, label, lab, root, b);
  int32_t ecc = b->nlev;
  for (int it = 0; it < 64; ++it) {
    int32_t best = -1, bestd = 0;
    for (int32_t q = b->lstart[b->nlev - 1]; q < b->lstart[b->nlev]; ++q) {
      int32_t v = b->queue[q];
      int32_t d = deg_in(g, label, lab, v);
      if (best < 0 || d < bestd || (d == bestd && v < best)) { best = v; bestd = d; }
    }
    bfs_levels(g, label, lab, best, b);
    if (b->nlev > ecc) { root = best; ecc = b->nlev; }
    else break;
  }
  bfs_levels(g, label, lab, root, b);
  return root;
}

/* Bisect the nodes carrying label lab (listed ascending in V[0..nv)) into
 * labels la / lb and separator -1, written to newlab. */
static void bisect(const ddg_graph *g, const int32_t *label, int32_t lab, const int32_t *V,
                   int32_t nv, int32_t la, int32_t lb, int32_t *newlab, ddg_bfs *b,
                   int32_t *order, int32_t *lev_of, int32_t *seen) {
  /* components in order of their lowest index; level sequences concatenated */
  int32_t norder = 0, nlevels = 0;
  int32_t *lsz = lev_of; /* reuse: level sizes accumulate in lsz[level] */
  for (int32_t q = 0; q < nv; ++q) {
    int32_t s = V[q];
    if (seen[s]) continue;
    pseudo_peripheral(g, label, lab, s, b);
    for (int32_t L = 0; L < b->nlev; ++L) {
      lsz[nlevels + L] = b->lstart[L + 1] - b->lstart[L];
      for (int32_t t = b->lstart[L]; t < b->lstart[L + 1]; ++t) {
        int32_t v = b->queue[t];
        seen[v] = 1;
        order[norder++] = v;
      }
    }
    nlevels += b->nlev;
  }
  /* cut: first level at which the cumulative count reaches ceil(nv/2) */
  int32_t half = (nv + 1) / 2, cum = 0, pos = 0;
  int32_t cut = nlevels - 1;
  for (int32_t L = 0; L < nlevels; ++L) {
    if (cum + lsz[L] >= half) { cut = L; break; }
    cum += lsz[L];
  }
  for (int32_t L = 0; L < nlevels; ++L) {
    int32_t lab2 = (L < cut) ? la : (L == cut ? -1 : lb);
    for (int32_t t = 0; t < lsz[L]; ++t) newlab[order[pos++]] = lab2;
  }
  /* separator trimming, ascending index: a separator node without a
   * neighbour on one side joins the other side */
  for (int32_t q = 0; q < nv; ++q) {
    int32_t s = V[q];
    seen[s] = 0;
    if (newlab[s] != -1) continue;
    int hasA = 0, hasB = 0;
    for (int32_t k = g->xadj[s]; k < g->xadj[s + 1]; ++k) {
      int32_t u = g->adj[k];
      if (label[u] != lab) continue;
      hasA |= (newlab[u] == la);
      hasB |= (newlab[u] == lb);
    }
    if (!hasB) newlab[s] = la;
    else if (!hasA) newlab[s] = lb;
  }
}

/* union-find helpers for the enclosed-pressure test */
static int32_t uf_find(int32_t *p, int32_t x) {
  while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
  return x;
}

/*
 * An interior block A_jj that contains a closed pressure region P (every
 * velocity row of the block couples to P with zero row sum) has the null
 * vector (0, 1_P).  Such components are opened by moving their lowest-index
 * node to the interface.  Returns the number of nodes moved.
 */
static int32_t repair_enclosed_pressure(int32_t n, const int32_t *rowptr, const int32_t *col,
                                        const double *val, int32_t *label) {
  int8_t *isp = (int8_t *)calloc((size_t)n, 1);
  int32_t *uf = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int8_t *open = (int8_t *)calloc((size_t)n, 1);
  int32_t moved = 0;
  if (!isp || !uf || !open) { free(isp); free(uf); free(open); return -1; }
  for (int32_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) d = val[k];
    isp[i] = (d == 0.0);
  }
  for (int pass = 0; pass < 8; ++pass) {
    for (int32_t i = 0; i < n; ++i) { uf[i] = i; open[i] = 0; }
    for (int32_t r = 0; r < n; ++r) {
      if (label[r] < 0) continue;
      int32_t first = -1;
      for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
        int32_t c = col[k];
        if (!isp[c] || label[c] != label[r]) continue;
        if (first < 0) first = c;
        else {
          int32_t a = uf_find(uf, first), b = uf_find(uf, c);
          if (a != b) { if (a < b) uf[b] = a; else uf[a] = b; }
        }
      }
    }
    for (int32_t r = 0; r < n; ++r) {
      if (label[r] < 0) continue;
      int32_t comp[16];
      double sum[16], mx = 0.0;
      int nc = 0;
      for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
        if (fabs(val[k]) > mx) mx = fabs(val[k]);
        int32_t c = col[k];
        if (!isp[c] || label[c] != label[r]) continue;
        int32_t rt = uf_find(uf, c);
        int q = 0;
        while (q < nc && comp[q] != rt) ++q;
        if (q == nc) {
          if (nc == 16) { open[rt] = 1; continue; }
          comp[nc] = rt; sum[nc] = 0.0; ++nc;
        }
        sum[q] += val[k];
      }
      for (int q = 0; q < nc; ++q)
        if (fabs(sum[q]) > 1e-12 * mx) open[comp[q]] = 1;
    }
    int32_t moved_now = 0;
    for (int32_t i = 0; i < n; ++i) /* roots are the lowest index of each set */
      if (isp[i] && label[i] >= 0 && uf[i] == i && !open[i]) {
        label[i] = -1;
        ++moved_now;
      }
    moved += moved_now;
    if (!moved_now) break;
  }
  free(isp); free(uf); free(open);
  return moved;
}

/*
 * An interface node with a structural zero diagonal (a pressure-like node)
 * has a zero row in G_ii unless one of its neighbours sits in the same
 * aggregate; aggregates are runs of consecutive indices, so each such node
 * gets a partner: its neighbour nearest in numbering (lowest index on ties)
 * is moved to the interface when it is interior.  Returns the number moved.
 */
static int32_t partner_interface_pressure(int32_t n, const int32_t *rowptr, const int32_t *col,
                                          const double *val, int32_t *label) {
  int32_t moved = 0;
  for (int32_t p = 0; p < n; ++p) {
    if (label[p] >= 0) continue;
    double d = 0.0;
    int32_t best = -1;
    for (int32_t k = rowptr[p]; k < rowptr[p + 1]; ++k) {
      int32_t c = col[k];
      if (c == p) { d = val[k]; continue; }
      if (val[k] == 0.0) continue;
      int32_t dc = c > p ? c - p : p - c, db = best > p ? best - p : p - best;
      if (best < 0 || dc < db || (dc == db && c < best)) best = c;
    }
    if (d != 0.0 || best < 0 || label[best] < 0) continue;
    label[best] = -1;
    ++moved;
  }
  return moved;
}

/* Reverse Cuthill-McKee order of the nodes carrying label lab (ascending in
 * V[0..nv)); neighbours are visited by (degree, index). */
static void rcm_order(const ddg_graph *g, const int32_t *label, int32_t lab, const int32_t *V,
                      int32_t nv, ddg_bfs *b, int32_t *out, int32_t *mark, int32_t *deg,
                      int32_t *tmp) {
  int32_t k = 0;
  for (int32_t q = 0; q < nv; ++q) deg[V[q]] = deg_in(g, label, lab, V[q]);
  for (int32_t q = 0; q < nv; ++q) {
    int32_t s = V[q];
    if (mark[s]) continue;
    int32_t root = pseudo_peripheral(g, label, lab, s, b);
    int32_t head = k;
    out[k++] = root;
    mark[root] = 1;
    while (head < k) {
      int32_t v = out[head++];
      int32_t nt = 0;
      for (int32_t e = g->xadj[v]; e < g->xadj[v + 1]; ++e) {
        int32_t u = g->adj[e];
        if (label[u] == lab && !mark[u]) { mark[u] = 1; tmp[nt++] = u; }
      }
      for (int32_t a = 1; a < nt; ++a) { /* sort by (degree, index) */
        int32_t u = tmp[a], c = a - 1;
        while (c >= 0 && (deg[tmp[c]] > deg[u] || (deg[tmp[c]] == deg[u] && tmp[c] > u))) {
          tmp[c + 1] = tmp[c];
          --c;
        }
        tmp[c + 1] = u;
      }
      for (int32_t a = 0; a < nt; ++a) out[k++] = tmp[a];
    }
  }
  for (int32_t a = 0, z = nv - 1; a < z; ++a, --z) { int32_t t = out[a]; out[a] = out[z]; out[z] = t; }
  for (int32_t q = 0; q < nv; ++q) mark[V[q]] = 0;
}

/*
 * Partition the n x n CSR matrix into m (a power of two) subdomain interiors
 * and an interface.
 *   part[i]  subdomain 0..m-1 of node i, or -1 for the interface
 *   perm[k]  original index of the k-th node of P^T C P: the interiors of
 *            subdomain 0 in RCM order, then subdomain 1, ..., then the
 *            interface, in ascending original index (iface_order 0) or in
 *            RCM order of the interface subgraph (iface_order 1)
 *   stats    [0] nodes moved by the enclosed-pressure repair
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int ddg_partition(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                  int32_t m, int32_t iface_order, int32_t *part, int32_t *perm, int64_t *stats) {
  if (n <= 0 || m <= 0 || (m & (m - 1))) return -1;
  ddg_graph g;
  if (graph_build(n, rowptr, col, &g)) return -1;
  ddg_bfs b;
  b.queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  b.lstart = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 2));
  b.stamp = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  b.cur = 0;
  int32_t *newlab = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *lev = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t *seen = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  int32_t *bucket = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *bstart = (int32_t *)calloc((size_t)m + 2, sizeof(int32_t));
  int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int rc = -1;
  if (!b.queue || !b.lstart || !b.stamp || !newlab || !order || !lev || !seen || !bucket ||
      !bstart || !deg)
    goto done;
  for (int32_t i = 0; i < n; ++i) part[i] = 0;
  for (int32_t nparts = 1; nparts < m; nparts *= 2) {
    /* bucket nodes by label, ascending within each bucket */
    memset(bstart, 0, sizeof(int32_t) * ((size_t)m + 2));
    for (int32_t i = 0; i < n; ++i) if (part[i] >= 0) bstart[part[i] + 1]++;
    for (int32_t p = 0; p < nparts; ++p) bstart[p + 1] += bstart[p];
    for (int32_t p = 0; p <= nparts; ++p) lev[p] = bstart[p];
    for (int32_t i = 0; i < n; ++i) if (part[i] >= 0) bucket[lev[part[i]]++] = i;
    for (int32_t i = 0; i < n; ++i) newlab[i] = part[i];
    for (int32_t p = 0; p < nparts; ++p) {
      int32_t nv = bstart[p + 1] - bstart[p];
      if (nv == 0) continue;
      bisect(&g, part, p, bucket + bstart[p], nv, 2 * p, 2 * p + 1, newlab, &b, order, lev + 0,
             seen);
      /* bisect reused lev as scratch; rebuild the bucket fill pointers */
      for (int32_t q = 0; q <= nparts; ++q) lev[q] = bstart[q];
    }
    memcpy(part, newlab, sizeof(int32_t) * (size_t)n);
  }
  {
    int64_t mv = 0, pm = 0;
    for (int it = 0; it < 16; ++it) {
      int32_t a = repair_enclosed_pressure(n, rowptr, col, val, part);
      if (a < 0) goto done;
      int32_t b2 = partner_interface_pressure(n, rowptr, col, val, part);
      mv += a;
      pm += b2;
      if (!a && !b2) break;
    }
    if (stats) { stats[0] = mv; stats[1] = pm; }
  }
  /* perm: RCM inside each subdomain, then the interface ascending */
  memset(bstart, 0, sizeof(int32_t) * ((size_t)m + 2));
  for (int32_t i = 0; i < n; ++i) if (part[i] >= 0) bstart[part[i] + 1]++;
  for (int32_t p = 0; p < m; ++p) bstart[p + 1] += bstart[p];
  for (int32_t p = 0; p <= m; ++p) lev[p] = bstart[p];
  for (int32_t i = 0; i < n; ++i) if (part[i] >= 0) bucket[lev[part[i]]++] = i;
  for (int32_t i = 0; i < n; ++i) seen[i] = 0;
  for (int32_t p = 0; p < m; ++p) {
    int32_t nv = bstart[p + 1] - bstart[p];
    if (nv == 0) continue;
    rcm_order(&g, part, p, bucket + bstart[p], nv, &b, perm + bstart[p], seen, deg, order);
  }
  {
    int32_t k = bstart[m], k0 = bstart[m];
    for (int32_t i = 0; i < n; ++i) if (part[i] < 0) perm[k++] = i;
    if (iface_order == 1 && k > k0) {
      /* RCM of the interface subgraph: consecutive chunks become connected
       * pieces of the separator */
      for (int32_t q = k0; q < k; ++q) bucket[q - k0] = perm[q];
      rcm_order(&g, part, -1, bucket, k - k0, &b, perm + k0, seen, deg, order);
    }
  }
  rc = 0;
done:
  free(g.xadj); free(g.adj);
  free(b.queue); free(b.lstart); free(b.stamp);
  free(newlab); free(order); free(lev); free(seen); free(bucket); free(bstart); free(deg);
  return rc;
}

/*
 * Aggregates of consecutive interface indices (eq. aggrV) of nominal size sz.
 * A chunk end is pushed forward (up to 2*sz) while the chunk holds a
 * pressure-like node (structural zero diagonal) none of whose interface
 * neighbours lies inside the chunk, since such a chunk has a zero row in
 * G_ii.  off must hold ceil(nG/1)+1 entries; returns the number of aggregates.
 */
int32_t ddg_aggregates(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                       const int32_t *part, const int32_t *perm, int32_t sz, int32_t *off) {
  int32_t nI = 0;
  for (int32_t i = 0; i < n; ++i) nI += (part[i] >= 0);
  int32_t nG = n - nI;
  int32_t *gpos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!gpos || sz <= 0) { free(gpos); return -1; }
  for (int32_t i = 0; i < n; ++i) gpos[i] = -1;
  for (int32_t k = nI; k < n; ++k) gpos[perm[k]] = k - nI;
  int32_t na = 0, a = 0;
  off[0] = 0;
  while (a < nG) {
    int32_t e = (a + sz < nG) ? a + sz : nG;
    int32_t emax = (a + 2 * sz < nG) ? a + 2 * sz : nG;
    for (;;) {
      int closed = 1;
      for (int32_t q = a; q < e && closed; ++q) {
        int32_t o = perm[nI + q];
        double d = 0.0;
        int inside = 0;
        for (int32_t k = rowptr[o]; k < rowptr[o + 1]; ++k) {
          int32_t c = col[k];
          if (c == o) { d = val[k]; continue; }
          int32_t g = gpos[c];
          if (g >= a && g < e && val[k] != 0.0) inside = 1;
        }
        if (d == 0.0 && !inside) closed = 0;
      }
      if (closed || e >= emax) break;
      ++e;
    }
    /* do not leave a tail shorter than sz/4: merge it */
    if (nG - e > 0 && nG - e < sz / 4) e = nG;
    off[++na] = e;
    a = e;
  }
  free(gpos);
  return na;
}
