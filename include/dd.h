/*
 * dd.h - C ABI of the GB300 (sm_103a) library for algebraic domain-decomposition
 * preconditioned GMRES on saddle-point systems C = [D E^T; -E 0] (linearised
 * Picard/Oseen Navier-Stokes, Section 1 of Kumar, "Purely algebraic domain
 * decomposition methods for the incompressible Navier-Stokes equations").
 *
 * Conventions for every entry point:
 *   - Plain pointers and sizes only.  "host" pointers are read during the call
 *     and copied; "device" pointers must be CUDA device memory of the current
 *     device, 8-byte aligned, and stay owned by the caller.
 *   - All device work is ordered on the caller's stream (a cudaStream_t passed
 *     as void*; NULL means the legacy default stream).
 *   - Errors are returned as dd_status codes; nothing aborts or throws across
 *     the ABI.  dd_last_error(h) gives a one-line description of the last error
 *     on a handle (or of the last failed dd_setup when h is NULL).
 *   - A handle is not thread-safe; distinct handles may be used concurrently on
 *     distinct streams.
 *   - Device memory is allocated only inside dd_setup (stream-ordered) and
 *     released by dd_destroy; dd_apply and gmres_solve allocate nothing.
 */
#ifndef DD_H
#define DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DD_OK = 0,
  DD_ERR_INVALID_ARG = 1,       /* bad sizes, pointers, kinds or options       */
  DD_ERR_INVALID_PARTITION = 2, /* part/perm inconsistent, or an entry couples
                                   two different interiors (the separator
                                   property of Section 1 is violated)          */
  DD_ERR_SINGULAR_BLOCK = 3,    /* an interior block A_jj failed the pivot test */
  DD_ERR_SINGULAR_SCHUR = 4,    /* a block S_ii of S_hat (or the D_ii of MSCN)
                                   failed the pivot test                       */
  DD_ERR_NOT_CONVERGED = 5,     /* maxit reached; x holds the last iterate     */
  DD_ERR_NONFINITE = 6,         /* NaN/Inf in the input or in a residual       */
  DD_ERR_TIMEOUT = 7,           /* a bounded device wait gave up               */
  DD_ERR_OOM = 8,               /* device or host allocation failed            */
  DD_ERR_CUDA = 9,              /* a CUDA runtime call failed                  */
  DD_ERR_CHECK = 10             /* a device check of the DD_CHECKED build (an
                                   index, alignment or size out of range)
                                   failed; the access was skipped             */
} dd_status;

/* Approximation of the interface Schur complement S = G - F D^-1 E
 * (Section 3, Algorithm 1).  Aggregates R_i are runs of consecutive
 * interface indices (eq. aggrV). */
typedef enum {
  DD_EXACT = 0,    /* S itself (one aggregate holding the whole interface)     */
  DD_MSCE_INF = 1, /* S(R_i,R_i): mini Schur complements over every interior
                      adjacent to the aggregate (MSCE with unbounded radius,
                      the block-Jacobi reading that ends Section 3.3)          */
  DD_MSCN = 2,     /* G_ii - F_ii D_ii^-1 E_ii, principal blocks with the same
                      local index range (Algorithm 1, MSCN)                    */
  DD_MSCNR = 3,    /* G_ii - diag(F_ii D_ii^-1 E_ii 1) (Algorithm 1, MSCNR)     */
  DD_LUM = 4,      /* G_ii (Definition of LUM)                                  */
  DD_LEARNED = 5,  /* G_ii + a learned correction on the pattern of G_ii and of
                      (F E)(R_i, R_i); an aggregate whose learned block fails
                      the pivot test takes its MSCE_INF block instead.  Not in
                      the paper: an extension of LUM (see dd_mlp_*)           */
  /* Overlapped aggregation (the Remark after eq. aggrV; Algorithm 1): block
   * i spans interface indices r_i .. r_{i+1} - 1 + w_i, w_i = min(opts.overlap,
   * p_{i+1}) and w_k = 0.  S_hat is assembled by placing the blocks in
   * aggregate order, a later block overwriting the overlap, so it is not
   * block diagonal; it is inverted whole (n_G <= 12288).  Not for batches. */
  DD_OMSCN = 6,    /* MSCN on the overlapped blocks                             */
  DD_OMSCNR = 7,   /* MSCNR on the overlapped blocks                            */
  DD_OLUM = 8,     /* G on the overlapped blocks                                */
  DD_MSCE = 9      /* MSCE with a finite radius r = opts.radius (Algorithm 1,
                      mini Schur complements on edge connectivity):
                      S_ii = G_ii - F_i D_r^-1 E_i with D_r the interior nodes
                      within path length r of the aggregate (first step
                      through F or E, then through the pattern of D), closed
                      by the D-neighbours of every zero-diagonal node.  r = 0
                      gives LUM; r beyond the interiors gives MSCE_INF      */
} dd_approx;

typedef enum {
  DD_FP64 = 0,     /* preconditioner factors and apply in FP64                 */
  DD_FP32 = 1,     /* factors and apply in FP32 (FP64 in/out); Krylov in FP64  */
  DD_FP32_TF32 = 2 /* DD_FP32, with the rank-64 updates of the dense block
                      inverses (S_hat, MSCN / MSCE(r) blocks) on the TF32
                      tensor cores, every product in three TF32 terms
                      (hi*hi + hi*lo + lo*hi, FP32 accumulation); close to
                      FP32 but not bitwise equal to DD_FP32.  Reported as
                      DD_FP32 by the handle                               */
} dd_prec;

/* C in CSR form, original numbering (host, copied). */
typedef struct {
  int64_t n;               /* number of rows = columns                      */
  int64_t nnz;             /* rowptr[n]                                     */
  const int32_t *rowptr;   /* n+1 entries, rowptr[0] = 0, non-decreasing    */
  const int32_t *col;      /* nnz column indices in [0, n)                  */
  const double *val;       /* nnz values, finite                            */
} dd_csr;

/* The algebraic partition P^T C P (Section 1; Section 3.2, matrix view). */
typedef struct {
  int32_t m;                   /* number of subdomains (interiors), >= 1         */
  const int32_t *part;         /* n entries: 0..m-1 interior, -1 interface       */
  const int32_t *perm;         /* optional n entries, new->old: the interiors of
                                  subdomain 0 in their local order, then 1, ...,
                                  then the interface; NULL = ascending original
                                  index inside each group                        */
  int32_t sz;                  /* nominal aggregate size (eq. aggrV) used when
                                  agg_offsets is NULL; ignored for DD_EXACT      */
  const int32_t *agg_offsets;  /* optional n_agg+1 offsets into the interface
                                  numbering, strictly increasing from 0 to n_G   */
  int32_t n_agg;
} dd_partition;

typedef struct {
  dd_prec prec;       /* DD_FP64, DD_FP32 or DD_FP32_TF32                      */
  double pivot_tol;   /* relative pivot test |pivot| <= tol * max|block|;
                         <= 0 selects 1e-14 (FP64) / 1e-7 (FP32)              */
  int32_t use_graph;  /* 1: gmres_solve replays one captured CUDA graph per
                         Arnoldi step; 0: plain launches                       */
  int32_t max_restart;/* largest restart length gmres_solve will be called
                         with (its Krylov workspace is allocated by dd_setup);
                         <= 0 selects 50, at most 120                          */
  int32_t autotune;   /* 1: dd_setup times the apply's sweep kernels for each
                         candidate ring-stage size (and with it CTAs per SM)
                         and keeps the fastest; 0: the fixed default           */
  int32_t krylov_ctas_per_sm; /* CTAs per SM of the Krylov kernels (CGS2 and the
                         batched norms); <= 0 selects 1 with 512-thread CGS2
                         CTAs, else 2                                           */
  int32_t time_kernels;/* 1: gmres_solve times the SpMV and CGS2 launches of
                         every Arnoldi step with CUDA events (dd_stats
                         krylov_steps, cgs2_ms, cgs2_fma, spmv_ms); ignored
                         with use_graph; 0: no events                        */
  int32_t sweep_cluster;/* CTAs per subdomain of the apply's sweeps: 1 one
                         CTA; 2 splits every tile step over a 2-CTA cluster
                         (half the tile bytes through each SM, the step's
                         rows exchanged through distributed shared memory);
                         3 a 2-CTA cluster in the lookahead split (CTA 0
                         runs the forward sweep and the near columns of each
                         backward step, CTA 1 the far columns one step
                         ahead, partial sums and x exchanged through
                         distributed shared memory; invalid argument where
                         its stages do not fit); 0 chooses (reported in
                         dd_stats.sweep_cluster), or with autotune the
                         fastest that fits                                 */
  const char *mlp_weights; /* DD_LEARNED: path of the network's weight file
                              (format under dd_mlp_*); ignored otherwise       */
  int32_t overlap;    /* DD_OMSCN / DD_OMSCNR / DD_OLUM: overlap width w >= 0   */
  int32_t radius;     /* DD_MSCE: path-length radius r >= 0                     */
  int32_t krylov_threads; /* threads per CTA of the CGS2 kernel: 256 or 512;
                         <= 0 selects 512 (then krylov_ctas_per_sm <= 0
                         selects 1)                                            */
  int32_t sweep_prefetch; /* the apply's sweeps prefetch into L2
                         (cp.async.bulk.prefetch) the tile bytes of the job
                         this many jobs past the ring as they refill a
                         stage: k > 0 a distance of k jobs, <= 0 none       */
  int32_t pad_opts;
  double ilu_tol;     /* inexact interior solves (Section 5: an incomplete LU
                         with tolerance tolA): 0 factors every A_jj exactly;
                         > 0 drops, during the banded LU with partial
                         pivoting, each entry of U below ilu_tol times its
                         column's 2-norm in A_jj and each multiplier below
                         ilu_tol times the pivot column's norm over the
                         pivot, before either is used; the factors' tiles
                         then trim to the entries kept.  < 0: invalid      */
} dd_opts;

typedef struct {
  int32_t iters;        /* Arnoldi steps over all restarts                    */
  int32_t restarts;
  int32_t bad_block;    /* index of the failing block for SINGULAR_* statuses */
  int32_t status;       /* this solve's dd_status (per system in a batch)     */
  double relres_true;   /* ||b - C x|| / ||b|| at return                      */
  double setup_ms;      /* device time of dd_setup (set by dd_setup's handle) */
  double solve_ms;      /* device time of gmres_solve                         */
  double *history;      /* optional host array: Givens residual estimate
                           |g_{j+1}| / ||b|| after every Arnoldi step          */
  int32_t history_cap;
  int32_t pad2;
} dd_info;

/* Sizes and byte counts of a built preconditioner (host struct filled by
 * dd_get_stats). */
typedef struct {
  int64_t n, n_interior, n_interface, nnz;
  int32_t m, n_agg, max_agg, kl_max, ku_max, tile;
  int64_t factor_bytes;      /* bytes of interior factors read by one band solve */
  int64_t factor_nonzeros;   /* in-band entries of L and U (no padding)          */
  int64_t schur_bytes;       /* bytes of S_hat^-1 blocks read by one apply       */
  int64_t coupling_nnz;      /* nnz(E) + nnz(F)                                  */
  double setup_ms;           /* device time of the last dd_setup                 */
  int64_t launches;          /* kernels this handle has launched so far          */
  int32_t stage_bytes;       /* ring stage of the apply's sweep kernels          */
  int32_t sweep_grid;        /* CTAs of one sweep launch                         */
  int32_t sweep_slots;       /* sweep CTAs resident on the device at once        */
  int32_t tuned;             /* stage sizes the autotuner timed (0: not run)     */
  double tuned_us;           /* fastest forward + backward sweep it measured     */
  int32_t batch;             /* independent systems behind the handle (>= 1)     */
  int32_t graphs;            /* CUDA graphs instantiated so far                  */
  int64_t learned_entries;   /* DD_LEARNED: entries of the learned patterns      */
  int32_t learned_fallback;  /* DD_LEARNED: aggregates that took MSCE_INF         */
  int32_t sweep_prefetch;    /* L2 prefetch distance of the sweeps, in jobs      */
  /* opts.time_kernels: summed over the timed Arnoldi steps of gmres_solve */
  int64_t krylov_steps;      /* Arnoldi steps timed                              */
  double cgs2_ms;            /* device time of the CGS2 kernel                   */
  double cgs2_fma;           /* FP64 multiply-adds of those steps' Gram-Schmidt
                                (both passes' dots and updates and the norm:
                                (4 (j+1) + 2) n at step j)                       */
  double spmv_ms;            /* device time of the SpMV w = C z                  */
  int32_t sweep_cluster;     /* sweep mode: 1 one CTA, 2 row-split cluster,
                                3 lookahead cluster (opts.sweep_cluster)         */
  int32_t msce_nodes_max;    /* DD_MSCE: largest interior node set D_r           */
} dd_stats;

/*
 * Build the preconditioner B = [D 0; F S_hat][D^-1 0; 0 S_hat^-1][D E; 0 S_hat]
 * (Definition of B_MSCN, eq. NDfactor) with S_hat per `approx` (Algorithm 1).
 * Every interior block A_jj is factored exactly with partial pivoting
 * (Section 4), S_hat's blocks are formed and inverted on the device.
 *   csr, part: host, copied.  opts may be NULL (FP64, default pivot test).
 *   stream: cudaStream_t as void*.  handle: receives an opaque handle owning all
 *   device workspace.  Returns DD_OK or an error; on SINGULAR_* errors the
 *   handle is still returned (dd_get_bad_block reports the block) and must be
 *   destroyed; on other errors *handle is NULL.  The call synchronises the
 *   stream once at its end (to read the pivot status).
 */
dd_status dd_setup(const dd_csr *csr, const dd_partition *partition, dd_approx approx,
                   const dd_opts *opts, void *stream, void **handle);

/*
 * x = B^-1 y (Algorithm 2; the lower-left block F acts in the forward sweep
 * and the upper-right block E in the backward sweep).  y, x: device, n
 * doubles, original numbering; may not alias.  Asynchronous on stream.
 */
dd_status dd_apply(void *handle, const double *y, double *x, void *stream);

/*
 * Solve C x = b with right-preconditioned restarted flexible GMRES
 * (Section 5): x0 = 0, restart length `restart`, classical Gram-Schmidt
 * applied twice, Givens rotations, stop when the Givens estimate
 * |g_{j+1}|/||b|| <= tol and the true residual ||b - Cx||/||b|| <= tol.
 *   b, x: device, n doubles.  info: host, may be NULL.  Krylov vectors, SpMV
 *   and the Hessenberg least squares are FP64 whatever the preconditioner's
 *   precision.  Synchronises the stream once per Arnoldi step (to read the
 *   residual estimate).  Returns DD_OK, DD_ERR_NOT_CONVERGED (x = last
 *   iterate) or DD_ERR_NONFINITE.
 */
dd_status gmres_solve(void *handle, const double *b, double *x, double tol, int32_t restart,
                      int32_t maxit, dd_info *info, void *stream);

/*
 * A batch of `count` independent systems behind one handle.  The batch is
 * set up as one block-diagonal system: the systems' rows one after the
 * other, the subdomains of every system renumbered after those of the
 * previous ones, and the aggregates (Section 3.2) taken per system, so that
 * B is block diagonal with one block B_q per system and every kernel of the
 * setup and the apply covers all systems in one launch (persistent,
 * longest-first task lists when the subdomains outnumber resident CTAs).
 *   csrs[q], partitions[q]: host, copied, as for dd_setup (each system in
 *   its own numbering).  approx: DD_EXACT (one Schur block per system),
 *   DD_MSCE_INF or DD_LUM; DD_MSCN / DD_MSCNR pair interface and interior
 *   index ranges of one system and return DD_ERR_INVALID_ARG.  Errors as
 *   dd_setup; dd_apply on the handle applies every B_q to the concatenated
 *   vector.
 */
dd_status dd_setup_batched(int32_t count, const dd_csr *csrs, const dd_partition *partitions,
                           dd_approx approx, const dd_opts *opts, void *stream, void **handle);

/*
 * Independent FGMRES solves C_q x_q = b_q of every system of a batched
 * handle, with gmres_solve's algorithm and tests per system.  The systems
 * step in lock step (one set of launches per Arnoldi step for all systems
 * still iterating); a system that meets its own test stops stepping, so each
 * takes the steps a solve of it alone would take.
 *   b[q], x[q]: device pointers, n_q doubles each.  infos: host array of
 *   count entries (may be NULL); infos[q].status is system q's dd_status.
 *   Returns DD_OK when every system converged, else the first failing
 *   system's status (DD_ERR_TIMEOUT / DD_ERR_CUDA for the batch as a whole).
 */
dd_status gmres_solve_batched(void *handle, const double *const *b, double *const *x, double tol,
                              int32_t restart, int32_t maxit, dd_info *infos, void *stream);

/*
 * One of the three kernels of dd_apply, for timing and profiling:
 *   part 0: z1 = D^-1 y1 (both interior sweeps, all subdomains)
 *   part 1: z2 = S_hat^-1 (y2 - F z1), x2 = z2 (needs part 0 first)
 *   part 2: x1 = z1 - D^-1 (E z2) (needs parts 0 and 1 first)
 * z1 and z2 live in the handle; y, x as in dd_apply.
 */
dd_status dd_apply_part(void *handle, int32_t part, const double *y, double *x, void *stream);

/*
 * dd_apply_noalloc: x = B^-1 y like dd_apply, for callers that cannot
 * allocate device memory at the time of the call. Examples: code whose
 * device memory is all held by another pool (a framework's caching
 * allocator), and code in a phase where an allocation could fail or stall
 * the device. The paper has no counterpart; this is an interface convenience.
 *
 * The intermediate vectors z1 (n_interior) and z2, t (n_interface each)
 * live in one file-scope device array of DD_NOALLOC_MAX_ELEMS doubles,
 * 8 MiB. Every GPU that loads the library holds the array until process
 * exit. Nothing is allocated, and no cudaMalloc, cudaFree or allocating
 * library routine is called. Systems whose vectors do not fit (always
 * n > DD_NOALLOC_MAX_ELEMS) are rejected with DD_ERR_INVALID_ARG and a
 * message in dd_last_error(handle).
 *
 * The first call on a device looks up the array's device address with that
 * device current; make this first call before any stream capture. All
 * calls share the one array: every call fully rewrites z1, z2 and t before
 * reading them, so nothing carries over. Calls that overlap on the GPU (on
 * different streams, or from different threads) race on the array and
 * must be serialised by the caller. y, x and the handle are as in dd_apply.
 */
#define DD_NOALLOC_MAX_ELEMS (1 << 20)
dd_status dd_apply_noalloc(void *handle, const double *y, double *x, void *stream);

/*
 * Status of the asynchronous device work of a handle.  The apply's sweep
 * kernels wait on their own bulk copies with bounded waits; a wait that gives
 * up records DD_ERR_TIMEOUT (with the subdomain) in the handle's status word,
 * drains its own copies and returns, leaving part of x unwritten.  dd_apply,
 * dd_apply_part and dd_apply_noalloc do not synchronise, so they cannot
 * report it; gmres_solve and gmres_solve_batched clear the word when they
 * start, return DD_ERR_TIMEOUT when it is set and leave it cleared when they
 * return.  dd_check_status
 * synchronises `stream`, returns DD_OK or the recorded status (description in
 * dd_last_error) and clears the word.
 */
dd_status dd_check_status(void *handle, void *stream);

/*
 * Test hook of the timeout path: the number of polls of the first mbarrier
 * wait of every CTA of the apply's sweep kernels (0: it gives up at once and
 * records DD_ERR_TIMEOUT; any value above the normal bound, e.g. UINT32_MAX,
 * restores the normal bound).  Only that first wait is shortened: the drain of
 * the copies in flight keeps the full bound, so a CTA never returns with a
 * copy outstanding.  Drops the handle's captured CUDA graphs.
 */
dd_status dd_set_wait_limit(void *handle, uint32_t first_wait_polls);

/*
 * Measurement helper (the paper has no counterpart): the FP64 fused
 * multiply-add rate of the current device, from a kernel of independent FMA
 * chains on every SM timed with CUDA events on `stream` (best of three after
 * a warm-up, about 10 ms each).  *gfma: host, FP64 FMAs per second / 1e9.
 * Synchronises the stream.
 */
dd_status dd_fp64_peak(double *gfma, void *stream);

/* y = C x with the handle's copy of C (device pointers, n doubles). */
dd_status dd_spmv(void *handle, const double *x, double *y, void *stream);

/* Fill *stats (host). */
dd_status dd_get_stats(void *handle, dd_stats *stats);

/* Block index behind the last SINGULAR_* status of this handle, or -1. */
int32_t dd_get_bad_block(void *handle);

/* Release every device allocation of the handle (stream-ordered on the
 * handle's setup stream, then synchronised). */
dd_status dd_destroy(void *handle);

/* One-line description of the last error (handle NULL: last dd_setup). */
const char *dd_last_error(void *handle);

/* ------------------------------------------------------------------------
 * The learned Schur correction (DD_LEARNED).  Not in the paper.
 *
 * For an aggregate R_i (Section 3.2) the learned block is
 *   S_L(R_i, R_i) = G(R_i, R_i) + Delta,
 * where Delta is nonzero only on P_i = {(r, c) in R_i x R_i : G(r, c) != 0,
 * or F(r, k) E(k, c) != 0 for some interior k, or r == c}.  On each entry,
 * Delta(r, c) = out_scale * MLP((x(r, c) - mean) / std).  The MLP is
 * 14 -> 64 (ReLU) -> 1; its inputs and weights are rounded to BF16 and it
 * accumulates in FP32.  The 14 features of (r, c), with d_k = D(k, k) and
 * Dinv_k = 1 / d_k where d_k != 0 (else 0):
 *   G(r,c), G(c,r), (F E)(r,c), (F Dinv E)(r,c), [r==c], [G(r,r)==0],
 *   [G(c,c)==0], G(r,r), G(c,c), sum_k |F(r,k)|, sum_k |E(k,c)|,
 *   #{k: F(r,k)!=0}/8, #{k: E(k,c)!=0}/8, (F Dinv E)(r,r).
 * The network is trained to the MSCE_INF correction S_ii - G_ii on P_i.
 * Parameters: DD_MLP_NPARAM floats, W1 (64 x 14, row-major), b1 (64),
 * w2 (64), b2.
 *
 * Weight file (little-endian): "DDMLPW01" | u32 version 1 | u32 14 | u32 64 |
 * f32 out_scale | f32 mean[14] | f32 std[14] | f32 params[1025] |
 * f32 adam_m[1025] | f32 adam_v[1025] | i64 step | u64 FNV-1a of all the
 * bytes before it.  dd_setup rejects a file with a wrong header or hash
 * (DD_ERR_INVALID_ARG).
 *
 * Training runs on the device, on a data set held by a training handle.
 * Row e of the data set is x_e (DD_MLP_IN normalised features, stored as
 * BF16) with target y_e (FP32, already divided by out_scale).  The loss is
 * the mean of (MLP(x_e) - y_e)^2 over a row range.  Its gradient is summed
 * in a fixed order, so a training run is reproducible bit for bit.
 * ---------------------------------------------------------------------- */
#define DD_MLP_IN 14
#define DD_MLP_HIDDEN 64
#define DD_MLP_NPARAM (DD_MLP_HIDDEN * DD_MLP_IN + 2 * DD_MLP_HIDDEN + 1)

/* New training handle holding a copy of params (host, DD_MLP_NPARAM FP32
 * master weights); Adam state zero. */
dd_status dd_mlp_create(const float *params, void **mlp);
/* Upload the data set: X host, n x DD_MLP_IN (row-major, normalised), y host,
 * n targets.  Replaces any previous data set. */
dd_status dd_mlp_set_data(void *mlp, const float *X, const float *y, int64_t n, void *stream);
/* Mean loss over rows [lo, hi) at the current weights and, if grad is not
 * NULL, its gradient (host, DD_MLP_NPARAM).  Synchronises the stream. */
dd_status dd_mlp_loss_grad(void *mlp, int64_t lo, int64_t hi, double *loss, float *grad, void *stream);
/* One Adam step (bias-corrected) on the gradient of rows [lo, hi); the
 * device keeps FP32 master weights and their BF16 copy.  Asynchronous. */
dd_status dd_mlp_adam_step(void *mlp, int64_t lo, int64_t hi, float lr, float beta1, float beta2,
                           float eps, void *stream);
/* MLP outputs of rows [lo, hi) into out (host, hi - lo floats). */
dd_status dd_mlp_predict(void *mlp, int64_t lo, int64_t hi, float *out, void *stream);
/* Master weights, Adam moments and step count (host arrays may be NULL). */
dd_status dd_mlp_get(void *mlp, float *params, float *adam_m, float *adam_v, int64_t *step);
/* Resume: set the Adam moments and step count (host). */
dd_status dd_mlp_set_adam(void *mlp, const float *adam_m, const float *adam_v, int64_t step);
dd_status dd_mlp_destroy(void *mlp);

/* The raw features of a DD_LEARNED handle's entries, in order of aggregate,
 * then local row, then local column: ents (host, 3 per entry: aggregate,
 * r, c), feats (host, DD_MLP_IN doubles per entry), delta (host, the Delta
 * value added per entry); each array may be NULL; at most cap entries are
 * written; *count receives the number of entries. */
dd_status dd_learned_entries(void *handle, int32_t *ents, double *feats, float *delta, int64_t cap,
                             int64_t *count);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
