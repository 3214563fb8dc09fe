// Internal declarations shared by the translation units of libdd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <climits>

#include <string>
#include <vector>

#include "dd.h"

// Tile width of the blocked band sweeps: one warp owns a tile's columns.
#define DD_NB 32
// Columns of a sweep tile: 64 (two LU panels, so a sweep takes half as many
// dependent tile steps) when two ring stages of such tiles fit in shared
// memory beside the resident vectors, else 32 (one panel).  Chosen per
// handle at setup; the sweep kernels run 8 threads per tile row.
#define DD_TB_WIDE 64

// Per-subdomain geometry of the interior factors (device-visible).
struct BandInfo {
  int32_t n;        // rows of A_jj
  int32_t kl, ku;   // lower / upper bandwidth of A_jj in its local order
  int32_t ntiles;   // LU panels: ceil(n / DD_NB)
  int32_t nst;      // sweep tiles: ceil(n / tile width)
  int32_t panel0;   // index of the first panel in the per-panel width tables
  int64_t band_off; // band rows (elements): row i at band_off + i*wd
  int64_t lraw_off; // the LU's per-tile multipliers, (NB+kl) x NB column-major each
  int64_t piv_off;  // pivots (n entries)
  int32_t row0;     // first row in the permuted interior numbering
  int32_t tile0;    // index of the first sweep tile in the packed tile tables
  int32_t jf0, njf; // forward jobs [jf0, jf0 + njf) of the sweep ring
  int32_t jb0, njb; // backward jobs (in the lookahead split: CTA 0's)
  int32_t jl0, njl; // lookahead split: CTA 1's backward jobs
};

__host__ __device__ inline int bi_wd(const BandInfo &b) { return 2 * b.kl + b.ku + 1; }
__host__ __device__ inline int bi_ku2(const BandInfo &b) { return b.kl + b.ku; }
__host__ __device__ inline int64_t bi_lraw_elems(const BandInfo &b) {
  return (int64_t)(DD_NB + b.kl) * DD_NB;
}

// One packed sweep tile (offsets in elements of T / int32 for src):
//   forward  K  wl x NB, row-major with 16-byte chunks swizzled by row
//            (chunk c of row r stored at chunk c ^ (r & 7)); src wl entries
//   backward Kb NB x wu, row-major
struct TileMeta {
  int64_t lofs, uofs, sofs;
  int32_t wl, wu;
  // 2-CTA sweeps: byte offsets of CTA p's forward slice (its K rows, then
  // the tile's src) and backward slice (its Kb rows) in the cluster layout
  int64_t cfo[2], cbo[2];
  // 2-CTA lookahead sweeps: byte offsets of CTA p's columns of the backward
  // tile (la_cols) in the lookahead layout
  int64_t lao[2];
};

// a job of the sweep ring: tiles [lo, hi) of one subdomain, one bulk copy
struct SweepJob {
  int32_t lo, hi;
};

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

// Columns of a backward tile (wu wide, tb rows) that CTA p of a lookahead
// pair takes: p = 0 the first la_split columns, p = 1 the rest.  CTA 0's
// share always holds the columns of b_T and of the next tile's x (those its
// step depends on at once); CTA 1's only x at least two tiles ahead, known
// one step earlier.  Beyond that the split halves the row.  wu and tb are
// multiples of 4, so every slice row is a multiple of 16 bytes.
__host__ __device__ inline int la_split(int wu, int tb) {
  const int half = ((wu >> 1) + 3) & ~3;
  const int s = half > 2 * tb ? half : 2 * tb;
  return s < wu ? s : wu;
}
__host__ __device__ inline int la_cols(int wu, int tb, int p) {
  const int s = la_split(wu, tb);
  return p == 0 ? s : wu - s;
}

// Sweeps split over a cluster of cl CTAs (cl = 1 or 2): CTA p of the cluster
// takes forward-tile rows [fwd_split(wl, p), fwd_split(wl, p + 1)) and
// backward-tile rows [p TB / cl, (p + 1) TB / cl).  Split points are
// multiples of 4 rows, so every slice of a tile starts on a 16-byte boundary.
__host__ __device__ inline int fwd_split(int wl, int p, int cl) {
  if (p <= 0) return 0;
  if (p >= cl) return wl;
  const int r = round4((wl * p + cl - 1) / cl);
  return r < wl ? r : wl;
}

// Launch plan of the sweep kernels: ring stage size, threads per CTA, and,
// when there are more subdomains than resident CTAs, a persistent grid whose
// CTA c takes the tasks sched[sched_off[c] .. sched_off[c+1]) (longest
// first, balanced on the host); sched_off == nullptr means one CTA per
// subdomain.
// Rows and CTAs of the systems a Krylov kernel works on.  nseg == 1: the
// whole vector, every CTA, one set of per-system state (the other pointers
// may be null).  nseg > 1: system s owns rows [seg_row0[s], seg_row0[s+1])
// and CTAs [seg_cta0[s], seg_cta0[s+1]); cta_seg maps a CTA to its system;
// act[s] != 0 while system s takes Arnoldi steps (null: all).  rmax sets the
// strides of the per-system state arrays.
struct SegMap {
  int nseg = 1;
  int rmax = 0;
  int nctas = 0;  // set on the device from the grid
  const int32_t *cta_seg = nullptr;
  const int32_t *seg_cta0 = nullptr;
  const int64_t *seg_row0 = nullptr;
  const int32_t *act = nullptr;
};

struct SweepPlan {
  uint32_t stage_bytes = 0;
  int threads = 256;
  int grid = 0;
  const int32_t *sched = nullptr;
  const int32_t *sched_off = nullptr;
  // batched solves: subdomain j is skipped while act[task_sys[j]] == 0 (its
  // system has stopped stepping); null: every subdomain
  const int32_t *task_sys = nullptr;
  const int32_t *act = nullptr;
  // polls of the first mbarrier wait of every sweep CTA (a test hook of the
  // timeout path); larger than the normal bound means the normal bound
  uint32_t first_wait = 0xffffffffu;
  // CTAs per subdomain: 1, or 2 (a thread-block cluster; threads = 4 TB);
  // grid counts CTAs, so a persistent grid holds grid / cl task lists
  int cl = 1;
  // L2 prefetch distance in jobs beyond the ring (0: none)
  int pf = 0;
  // cl = 2: the tiles in the cluster layout (TileMeta cfo / cbo)
  const unsigned char *cld = nullptr;
  // cl = 2 with la = 1: the lookahead split instead (CTA 0 runs the forward
  // sweep alone and the near columns of every backward step, CTA 1 the far
  // columns one step ahead); backward slices in lad (TileMeta lao), 8 TB
  // threads per CTA
  int la = 0;
  const unsigned char *lad = nullptr;
};

// Device-side error word: first failure wins.
struct DevStatus {
  int32_t code;   // 0 ok, else a dd_status
  int32_t block;  // failing block (DD_ERR_CHECK: the check's site)
};

#ifdef __CUDACC__
// Warp-wide argmax of (v, L): the largest v, then the lowest L, with v >= 0
// for candidates and v < 0 (or NaN mapped to < 0) for none.  Positive
// floating-point values order as their bit patterns, so the maximum is taken
// with integer warp reductions on the bits; zero, negative and NaN values
// count as key 0 (a candidate of value 0 still wins over a non-candidate,
// whose L is INT_MAX; its pivot then fails the threshold test).  Every lane
// gets the winner's v, L and r.
__device__ __forceinline__ uint32_t warp_key_max(uint32_t k) { return __reduce_max_sync(0xffffffffu, k); }
template <typename T>
__device__ __forceinline__ void warp_argmax(T &v, int &L, int &r) {
  bool tie;
  if constexpr (sizeof(T) == 4) {
    const uint32_t k = v > T(0) ? __float_as_uint((float)v) : 0u;
    tie = k == warp_key_max(k);
  } else {
    const uint64_t b = v > T(0) ? (uint64_t)__double_as_longlong((double)v) : 0ull;
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const bool th = hi == warp_key_max(hi);
    const uint32_t lm = __reduce_max_sync(0xffffffffu, th ? lo : 0u);
    tie = th && lo == lm;
  }
  const int Lm = __reduce_min_sync(0xffffffffu, tie ? L : INT_MAX);
  const int src = __ffs(__ballot_sync(0xffffffffu, tie && L == Lm)) - 1;
  v = __shfl_sync(0xffffffffu, v, src);
  L = Lm;
  r = __shfl_sync(0xffffffffu, r, src);
}
#endif

// Checked build (compiled with -DDD_CHECKED): the sweep, SpMV and interface
// kernels test every index, size and alignment they compute before the
// access; a failed test records DD_ERR_CHECK with the site number and the
// access is skipped (no trap).  Without DD_CHECKED the tests compile away.
#ifdef __CUDACC__
__device__ inline bool dd_check(DevStatus *st, bool ok, int site) {
#ifdef DD_CHECKED
  if (!ok && st && atomicCAS(&st->code, 0, (int)DD_ERR_CHECK) == 0) st->block = site;
  return ok;
#else
  (void)st; (void)site;
  return true;
#endif
}
#endif

struct Workspace;  // defined in dd_api.cu

// ---- kernels exposed to dd_api.cu (implemented in k_band.cu / k_dense.cu /
// ---- k_krylov.cu).  All return cudaGetLastError() of their launch.
// Tile ring of the apply sweeps: how many stages of stage_bytes fit next to
// the resident right-hand side (0: the subdomain is too large).
int band_sweep_stages(int max_n, int max_kl, int max_ku2, int tb, int cl, int elem_size,
                      uint32_t stage_bytes);
// largest stage size that leaves room for two stages (0: the vectors alone do not fit)
size_t band_sweep_max_stage(int max_n, int max_kl, int max_ku2, int elem_size, int tb, int cl = 1);
// Blocked banded LU; ltraw receives each tile's multipliers ((NB+kl) x NB,
// column-major, exchanged), wscratch holds the windows when they do not fit
// in shared memory (band_lu_window_bytes per subdomain, else unused).
// sched / sched_off: optional persistent task lists of `grid` CTAs (as in
// SweepPlan).  ilu_tol > 0: the incomplete factorisation (entries of U below
// ilu_tol times their column's 2-norm, multipliers below ilu_tol times the
// pivot column's norm over the pivot, dropped before use); cnorm then holds
// n_I values of scratch for the column norms.
size_t band_lu_window_bytes(int max_kl, int max_ku, int elem_size);
template <typename T>
cudaError_t launch_band_lu(const BandInfo *d_info, int m, int max_kl, int max_ku, T *band, T *ltraw,
                           int32_t *piv, T *wscratch, double pivtol, DevStatus *st, int threads,
                           int grid, const int32_t *sched, const int32_t *sched_off, T *cnorm,
                           double ilu_tol, cudaStream_t s);
// resident CTAs per SM of the band LU (0 on error)
template <typename T>
int band_lu_occupancy(int max_kl, int max_ku, int threads);
// Widths of every tile (forward rows wl and backward columns wu that hold
// nonzeros after the factorisation), written to wl/wu at tile0 + t.
template <typename T>
cudaError_t launch_tile_widths(const BandInfo *d_info, int m, int max_panels, const T *band,
                               const T *lraw, const int32_t *piv, int32_t *wl, int32_t *wu,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_band_tiles(const BandInfo *d_info, int m, int max_tiles, int max_kl, int tb,
                              const TileMeta *tm, const T *band, const T *lraw, const int32_t *piv,
                              T *ltile, T *utile, int32_t *src, cudaStream_t s);
// z = A_jj^-1 y_j per subdomain; y gathered through perm (original
// numbering), z in the interior numbering.
template <typename T>
cudaError_t launch_band_solve_fwd(const BandInfo *d_info, int m, int max_n, int max_kl,
                                  int max_ku2, const SweepPlan &pl, const TileMeta *tm,
                                  const SweepJob *jobs, const T *ltile, const T *utile,
                                  const int32_t *src, const double *y, const int32_t *perm, T *z,
                                  DevStatus *st, cudaStream_t s);
// x1 = z1 - A^-1 (E z2) per subdomain, scattered to x (original numbering).
template <typename T>
cudaError_t launch_band_solve_bwd(const BandInfo *d_info, int m, int max_n, int max_kl,
                                  int max_ku2, const SweepPlan &pl, const TileMeta *tm,
                                  const SweepJob *jobs, const T *ltile, const T *utile,
                                  const int32_t *src, const int32_t *e_ptr, const int32_t *e_col,
                                  const T *e_val, const T *z2, const T *z1, const int32_t *perm,
                                  double *x, DevStatus *st, cudaStream_t s);
// subdomains the sweep kernels hold resident at once (CTAs for cl = 1,
// clusters for cl = 2; la = 1 the lookahead split's 8 TB-thread clusters) at
// this stage size; 0: they do not fit
template <typename T>
int band_sweep_slots(int max_n, int max_kl, int max_ku2, int tb, int cl, uint32_t stage_bytes, int la = 0);
// The 2-CTA sweep layout: bytes of CTA p's forward / backward slice of a tile,
// and the copy of every tile's slices to cld at TileMeta cfo / cbo
void cluster_slice_bytes(const TileMeta &mt, int tb, int elem_size, int p, int64_t &fwd, int64_t &bwd);
template <typename T>
cudaError_t launch_cluster_pack(int ntiles, int tb, const TileMeta *tm, const T *ltile, const T *utile,
                                const int32_t *srcs, unsigned char *cld, cudaStream_t s);
// The lookahead sweep layout: CTA p's columns of every backward tile
// (la_cols) copied to lad at TileMeta lao[p]
template <typename T>
cudaError_t launch_la_pack(int ntiles, int tb, const TileMeta *tm, const T *utile, unsigned char *lad,
                           cudaStream_t s);
// X = A_jj^-1 X in place; X column-major with leading dimension n_j starting
// at x_off[j], ncols[j] columns.
template <typename T>
cudaError_t launch_band_solve_multi(const BandInfo *d_info, int m, const int32_t *ncols,
                                    const int64_t *x_off, int max_cols, int max_kl, int max_ku2, int tb,
                                    const TileMeta *tm, const T *ltile, const T *utile,
                                    const int32_t *src, T *X, cudaStream_t s);

// Dense blocks (k_dense.cu): block b of size p[b] at offset off[b], row-major.
template <typename T>
cudaError_t launch_block_amax(int nblk, const int32_t *d_p, const int64_t *d_off, const T *A,
                              T *amax, cudaStream_t s);
// In-place explicit inverses (Gauss-Jordan, partial pivoting); ipiv holds
// p[b] entries per block at poff[b]; failing blocks are flagged and reported
// through st with status_code.  tc = 1 (FP32 only): the rank-64 updates on
// TF32 tensor cores, each product in three TF32 terms (DD_FP32_TF32).
// scratch (elements of T) of launch_gj_inverse for nblk blocks of total size sum_p
int64_t gj_scratch_elems(int nblk, int64_t sum_p, int elem_size);
// kernel launches of one launch_gj_inverse call for blocks of size <= pmax
int64_t gj_launch_count(int pmax, int elem_size);
template <typename T>
cudaError_t launch_gj_inverse(int nblk, const int32_t *d_p, const int64_t *d_off, int pmax, T *A,
                              int32_t *ipiv, const int64_t *d_poff, const T *amax, int32_t *failed,
                              T *scratch, double pivtol, DevStatus *st, int status_code,
                              cudaStream_t s, int tc = 0);
template <typename T>
cudaError_t launch_scatter_coo(int64_t nnz, const int64_t *idx, const double *val, T *dst,
                               cudaStream_t s);
template <typename T>
// one colour of subdomains: jlist (device) holds its nj subdomains, no two of
// which share an interface row
cudaError_t launch_schur_accumulate(int nj, const int32_t *jlist, const int32_t *fr_ptr, const int32_t *fr_row,
                                    const int32_t *fr_agg, const int32_t *f_ptr,
                                    const int32_t *f_col, const T *f_val, const int32_t *gam_ptr,
                                    const int32_t *gam_idx, const int32_t *gam_agg,
                                    const int64_t *x_off, const BandInfo *d_info, const T *X,
                                    const int32_t *agg_off, const int64_t *s_off, T *S,
                                    int max_fr, int max_gam, cudaStream_t s);
template <typename T>
cudaError_t launch_block_gemm(int nblk, const int32_t *d_p, const int64_t *d_off, int pmax,
                              const T *A, const T *B, T *C, T alpha, T beta, cudaStream_t s);
// overlapped kinds: S_hat (dense n_G x n_G) from the blocks of the k
// aggregates extended by w (block a: q_a x q_a at xoff[a] in Sx), a later
// block overwriting the overlap
template <typename T>
cudaError_t launch_assemble_overlapped(int ng, int k, const int32_t *agg, const int32_t *w, const int64_t *xoff,
                                       const T *Sx, T *S, cudaStream_t s);
// C_b = alpha A_b B_b + beta C_b, rectangular row-major blocks: dims (M, N, K)
// and offs (A, B, C offsets) three per block
template <typename T>
cudaError_t launch_rect_gemm(int nblk, const int32_t *dims, const int64_t *offs, int maxM, int maxN, const T *A,
                             const T *B, T *C, T alpha, T beta, cudaStream_t s);
template <typename T>
cudaError_t launch_mscnr_diag(int nblk, const int32_t *d_p, const int64_t *d_off, int pmax,
                              const T *Dinv, const T *E, const T *F, T *S, cudaStream_t s);
// z2 = S_hat^-1 (y2 - F z1) with explicit inverses; also writes x2 = z2 to x
// (original numbering).
// (two kernels: t = y2 - F z1 into t, then the block GEMV)
template <typename T>
cudaError_t launch_schur_apply(int nagg, const int32_t *agg_off, const int64_t *s_off, int pmax,
                               const T *Sinv, const int32_t *f_ptr, const int32_t *f_col,
                               const T *f_val, const double *y, const int32_t *perm_iface,
                               const T *z1, T *z2, T *t, int ng, double *x, const int32_t *agg_sys,
                               const int32_t *act, cudaStream_t s);

// Krylov (k_krylov.cu), FP64
// C in SELL-32 form: slices of 32 rows; slice s holds w_s = (off[s+1] -
// off[s]) / 32 entries per row, stored entry-major (entry k of lane r at
// off[s] + 32 k + r), each row's entries in CSR order and padded with value 0
// at its last column.  Rows are sorted by decreasing length inside windows
// of DD_SELL_WINDOW rows, so a slice's rows have nearly equal lengths;
// row[32 s + r] is the matrix row of lane r (-1: padding past the last row).
#define DD_SELL_WINDOW 256
struct SellC {
  int64_t nslices = 0;
  int64_t n = 0;              // rows = columns of C
  DevStatus *st = nullptr;    // DD_CHECKED: where a failed index check is recorded
  const int64_t *off = nullptr;
  const int32_t *row = nullptr;
  const int32_t *col = nullptr;
  const double *val = nullptr;
};
cudaError_t launch_spmv(const SellC &c, const double *x, double *y, cudaStream_t s);
// y = C x on the rows i with act[row_sys[i]] != 0 (the other rows untouched)
cudaError_t launch_spmv_masked(const SellC &c, const double *x, double *y, const int32_t *row_sys,
                               const int32_t *act, cudaStream_t s);
// FP64 FMA probe: blocks x 256 threads, 8 chains of `iters` FMAs each
cudaError_t launch_fma_probe(int blocks, int iters, cudaStream_t s);
// r = b - C x
cudaError_t launch_residual(const SellC &c, const double *x, const double *b, double *r, cudaStream_t s);
cudaError_t launch_multidot(int n, int k, const double *V, int64_t ldv, const double *w,
                            double *partial, int nblocks, cudaStream_t s);
cudaError_t launch_reduce_cols(int nblocks, int k, const double *partial, double *out,
                               int accumulate, cudaStream_t s);
cudaError_t launch_gemv_sub(int n, int k, const double *V, int64_t ldv, const double *h,
                            double *w, cudaStream_t s);
cudaError_t launch_copy_scaled(int n, const double *src, const double *nrm_sq, double *dst,
                               cudaStream_t s);
cudaError_t launch_scale_by(int n, const double *scal, double *w, cudaStream_t s);
cudaError_t launch_givens2(int j, int R, double *H, const double *hc1, const double *hc2,
                           const double *nsq, double *cs, double *sn, double *g, double bnorm,
                           double *out, cudaStream_t s);
cudaError_t launch_hess_solve_update(int n, int jlast, int R, const double *H, const double *g,
                                     double *y, const double *Z, int64_t ldz, double *x,
                                     cudaStream_t s);
cudaError_t launch_init_g(double *g, int R, const double *nsq, cudaStream_t s);
cudaError_t launch_zero(double *p, int64_t n, cudaStream_t s);
// One Arnoldi orthogonalisation step (CGS2 + Givens + normalisation) as a
// single cooperative kernel; partial holds nblocks * pk doubles, pk >= R + 2.
int cgs2_blocks(int per_sm, int cap, int threads);
// threads: 256 or 512 per CTA
cudaError_t launch_cgs2(int64_t n, int j, int R, const double *V, int64_t ldv, double *w, double *partial,
                        int pk, double *hc1, double *hc2, double *H, double *cs, double *sn, double *g,
                        const double *bn2, double *scal, const SegMap &sm, int nblocks, int threads,
                        cudaStream_t s);
// Batched FGMRES over a SegMap (nseg >= 2, nblocks = seg_cta0[nseg] CTAs):
// out[s] = ||v_s||^2; v0 = r / ||r_s|| and g_s = ||r_s|| e_0 for active
// systems; y_s = H_s^-1 g_s and x_s += Z y_s for systems with jl[s] >= 0.
cudaError_t launch_seg_norms(int64_t n, const double *v, double *partial, double *out, const SegMap &sm,
                             int nblocks, cudaStream_t s);
cudaError_t launch_seg_start(int64_t n, const double *r, const double *nsq, double *v0, double *g,
                             const SegMap &sm, int nblocks, cudaStream_t s);
cudaError_t launch_seg_hess_update(int64_t n, int R, const int32_t *jl, const double *H, const double *g,
                                   double *y, const double *Z, int64_t ldz, double *x, const SegMap &sm,
                                   int nblocks, cudaStream_t s);

// ---------------------------------------------------------------------------
// DD_LEARNED setup: per-entry features, the network and Delta added to S.
// Index arrays in the permuted numbering (interface rows local to the
// interface); values FP64.
// ---------------------------------------------------------------------------
struct LearnedArgs {
  int64_t n_ent = 0;
  const int32_t *ent = nullptr;         // 3 per entry: aggregate, local row, local column
  const int32_t *agg_off = nullptr;     // nagg + 1
  const int64_t *s_off = nullptr;       // block offsets in S
  const int32_t *perm_iface = nullptr;  // interface index -> original index
  const int32_t *c_rowptr = nullptr, *c_col = nullptr;  // C, original numbering
  const double *c_val = nullptr;
  const int32_t *f_ptr = nullptr, *f_col = nullptr;    // F: interface rows -> interior
  const double *f_val = nullptr;
  const int32_t *e_ptr = nullptr, *e_col = nullptr;    // E: interior rows -> interface
  const double *e_val = nullptr;
  const int32_t *et_ptr = nullptr;                     // E^T values per interface row
  const double *et_val = nullptr;
  const double *dinv = nullptr;                        // 1 / D(k, k), 0 where D(k, k) = 0
  const float *wbf = nullptr;                          // BF16-rounded parameters (DD_MLP_NPARAM)
  const float *mean = nullptr, *stdv = nullptr;        // feature normalisation
  float out_scale = 1.f;
  double *feat = nullptr;                              // optional: raw features out
  float *delta = nullptr;                              // optional: Delta per entry out
};
template <typename T>
cudaError_t launch_learned_delta(const LearnedArgs &a, T *S, cudaStream_t s);
