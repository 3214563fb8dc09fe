// C ABI of libdd (include/dd.h): host-side validation and block extraction of
// P^T C P = [D E; F G], device setup of B (Algorithm 1), the apply
// x = B^-1 y (Algorithm 2) and right-preconditioned restarted FGMRES
// (Section 5).  Every arithmetic step of the setup, the apply and the solve
// runs in the kernels of k_band.cu, k_dense.cu and k_krylov.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dd_internal.h"

namespace {

thread_local std::string g_setup_error;

template <typename T>
struct PrecBufs {
  T *band = nullptr, *lm = nullptr, *ltile = nullptr, *utile = nullptr;
  T *e_val = nullptr, *f_val = nullptr, *fsub_val = nullptr;
  T *S = nullptr, *amax = nullptr, *X = nullptr;
  T *z1 = nullptr, *z2 = nullptr, *t = nullptr;
  T *Dm = nullptr, *Em = nullptr, *Fm = nullptr, *Tm = nullptr;
  T *gj = nullptr;  // scratch of the blocked Gauss-Jordan inverses
};

struct DDHandle {
  int prec = DD_FP64;
  dd_approx kind = DD_MSCE_INF;
  int64_t n = 0, nnz = 0;
  int m = 0, nI = 0, nG = 0, nagg = 0, pmax = 0;
  int max_n = 0, max_kl = 0, max_ku = 0, max_ku2 = 0, max_tiles = 0;
  int tb = DD_NB;              // columns of a sweep tile (DD_NB or DD_TB_WIDE)
  SweepPlan plan;              // sweep ring stage size, threads and persistent schedule
  uint32_t first_wait = 0xffffffffu;  // test hook: polls of each sweep CTA's first wait
  int sweep_cl_opt = 0;        // opts.sweep_cluster: 0 choose, 1, 2 or 3
  int gj_tc = 0;               // DD_FP32_TF32: Gauss-Jordan updates on TF32 tensor cores
  int sweep_pf_opt = 0;        // opts.sweep_prefetch: k > 0 k jobs, else none
  int overlap = 0, radius = 0; // opts.overlap (overlapped kinds), opts.radius (DD_MSCE)
  double ilu_tol = 0.0;        // opts.ilu_tol: drop tolerance of the incomplete interior LU (0: exact)
  std::vector<BandInfo> h_info;  // host copies of the subdomain and tile tables (re-planning)
  std::vector<TileMeta> h_tm;
  size_t max_tile = 0;           // bytes of the largest packed tile
  int32_t *sweep_sched = nullptr, *sweep_off = nullptr;
  int sweep_sched_cap = 0;
  void *lu_scratch = nullptr;  // windows of the blocked LU (when not in shared memory)
  TileMeta *tm = nullptr;      // packed sweep tiles
  bool tiles_ready = false;    // the packed tiles are written (or queued)
  unsigned char *cld = nullptr;  // the tiles in the 2-CTA sweep layout (built on first use)
  unsigned char *lad = nullptr;  // the backward tiles in the lookahead layout (built on first use)
  SweepJob *jobs = nullptr;    // jobs of the sweep ring
  cudaStream_t stream = nullptr;
  // setup: while astream is set, allocations and uploads go to it (the side
  // stream ustream, so that pageable copies need not wait for the band LU
  // on stream); uev joins it back into stream
  cudaStream_t astream = nullptr, ustream = nullptr;
  cudaEvent_t uev = nullptr;
  std::vector<void *> allocs;
  BandInfo *d_info = nullptr;
  int32_t *piv = nullptr, *src = nullptr;
  int32_t *d_perm = nullptr;
  int32_t *e_ptr = nullptr, *e_col = nullptr, *f_ptr = nullptr, *f_col = nullptr;
  int32_t *agg_off = nullptr, *d_p = nullptr, *ipiv = nullptr, *failed = nullptr;
  int64_t *s_off = nullptr, *poff = nullptr;
  int32_t *c_rowptr = nullptr, *c_col = nullptr;
  double *c_val = nullptr;
  SellC sell;                  // C in SELL-32 form for the SpMV and residuals
  int64_t sell_entries = 0;    // stored entries of sell (nnz plus padding)
  DevStatus *st = nullptr;
  PrecBufs<double> pd;
  PrecBufs<float> pf;
  // FGMRES workspace; per-system arrays hold nseg systems (strides from Rmax)
  int Rmax = 0, nblocks = 304, cgs_blocks = 0;
  int64_t ldv = 0;
  double *V = nullptr, *Z = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr,
         *y = nullptr, *hc1 = nullptr, *hc2 = nullptr, *nsq = nullptr, *out = nullptr,
         *partial = nullptr, *r = nullptr;
  double *h_out = nullptr;  // pinned host scalars (4 per system)
  // batch of independent systems (nseg > 1): rows, CTAs and state per system
  int nseg = 1, seg_ctas = 0;
  std::vector<int64_t> seg_row0_h;
  int32_t *cta_seg = nullptr, *seg_cta0 = nullptr, *d_act = nullptr, *d_jl = nullptr;
  int32_t *cta_seg_act = nullptr, *seg_cta0_act = nullptr, *row_sys = nullptr;
  int64_t *seg_row0 = nullptr;
  int32_t *h_act = nullptr;  // pinned: act then jl, nseg each
  std::vector<int32_t> sub_sys_h, agg_sys_h;  // system of every subdomain / aggregate
  int32_t *sub_sys = nullptr, *agg_sys = nullptr;
  bool masked = false;       // the apply skips systems that have stopped stepping
  // DD_LEARNED: the network and its entries
  std::string mlp_path;
  std::vector<int32_t> l_ents;  // 3 per entry
  double *l_feat = nullptr;
  float *l_delta = nullptr;
  DevStatus *st_probe = nullptr;  // status word of the first (learned) inversion
  double *bcat = nullptr, *xcat = nullptr, *bn2 = nullptr, *rn2 = nullptr;
  // CUDA graphs of the Arnoldi steps (use_graph), one per step index
  int use_graph = 0, graph_key = -1;
  int krylov_per_sm = 2;
  int krylov_threads = 256;    // threads per CTA of the CGS2 kernel (256 or 512)
  int time_kernels = 0;        // events around the SpMV and CGS2 of every Arnoldi step
  cudaEvent_t kev[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t sev[2] = {nullptr, nullptr};  // end of Arnoldi steps j (parity): the host waits on them
  std::vector<cudaGraphExec_t> gexec;
  std::vector<int64_t> glaunch;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  std::string err;
  int bad_block = -1;
  dd_stats stats{};
};

#define CK(call)                                                                     \
  do {                                                                               \
    if (strncmp(#call, "launch_", 7) == 0) h->stats.launches += launch_cost(#call, h);  \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
      return DD_ERR_CUDA;                                                            \
    }                                                                                \
  } while (0)

// kernels behind one launcher call (the Gauss-Jordan inverse is 2 per pivot
// step plus the final column exchange; the Hessenberg update is two)
int64_t launch_cost(const char *call, const DDHandle *h);

template <typename P>
dd_status dalloc(DDHandle *h, P **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void *q = nullptr;
  cudaError_t e = cudaMallocAsync(&q, count * sizeof(P), h->astream ? h->astream : h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DD_ERR_OOM : DD_ERR_CUDA;
  }
  h->allocs.push_back(q);
  *p = static_cast<P *>(q);
  return DD_OK;
}

// count values of the caller's host array (pageable: staged at once)
template <typename P>
dd_status upload_ptr(DDHandle *h, P **p, const P *src, size_t count) {
  dd_status s = dalloc(h, p, count);
  if (s != DD_OK) return s;
  if (count)
    CK(cudaMemcpyAsync(*p, src, count * sizeof(P), cudaMemcpyHostToDevice, h->astream ? h->astream : h->stream));
  return DD_OK;
}

template <typename P>
dd_status upload(DDHandle *h, P **p, const std::vector<P> &v) {
  dd_status s = dalloc(h, p, v.size());
  if (s != DD_OK) return s;
  if (!v.empty())
    CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(P), cudaMemcpyHostToDevice,
                       h->astream ? h->astream : h->stream));
  return DD_OK;
}

#define TRY(x)                    \
  do {                            \
    dd_status s_ = (x);           \
    if (s_ != DD_OK) return s_;   \
  } while (0)

// band rows of A_jj filled from C (one thread per original row)
template <typename T>
__global__ void fill_band_kernel(int n, const int32_t *__restrict__ rowptr,
                                 const int32_t *__restrict__ col, const double *__restrict__ val,
                                 const int32_t *__restrict__ part, const int32_t *__restrict__ pos,
                                 const BandInfo *__restrict__ info, T *band) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = part[i];
  if (j < 0) return;
  const BandInfo b = info[j];
  const int wd = 2 * b.kl + b.ku + 1;
  const int r = pos[i] - b.row0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const int c = col[k];
    if (part[c] != j) continue;
    const int cc = pos[c] - b.row0;
    band[b.band_off + (int64_t)r * wd + (cc - r + b.kl)] += T(val[k]);
  }
}

template <typename T>
__global__ void convert_kernel(int64_t n, const double *__restrict__ a, T *b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = T(a[i]);
}

template <typename T>
dd_status upload_T(DDHandle *h, T **p, const std::vector<double> &v) {
  if (sizeof(T) == sizeof(double)) return upload(h, reinterpret_cast<double **>(p), v);
  double *tmp = nullptr;
  TRY(upload(h, &tmp, v));
  TRY(dalloc(h, p, v.size()));
  if (!v.empty()) {
    h->stats.launches += 1;
    convert_kernel<T><<<(unsigned)((v.size() + 255) / 256), 256, 0, h->astream ? h->astream : h->stream>>>(
        (int64_t)v.size(), tmp, *p);
    CK(cudaGetLastError());
  }
  return DD_OK;
}

template <typename T>
PrecBufs<T> &bufs(DDHandle *h);
template <>
PrecBufs<double> &bufs<double>(DDHandle *h) { return h->pd; }
template <>
PrecBufs<float> &bufs<float>(DDHandle *h) { return h->pf; }

// ---------------------------------------------------------------------------
// Host-side description of P^T C P
// ---------------------------------------------------------------------------
struct HostBlocks {
  std::vector<int32_t> perm, pos, off;      // new->old, old->new, interior offsets
  std::vector<int32_t> agg;                 // aggregate offsets (interface numbering)
  std::vector<int32_t> kl, ku;
  // E: interior rows (new) -> interface cols (local); F: interface rows -> interior cols (new)
  std::vector<int32_t> e_ptr, e_col, f_ptr, f_col;
  std::vector<double> e_val, f_val;
};

// Rows [0, n) in contiguous chunks over the host cores; f(w, r0, r1) runs
// chunk w.  Results that depend on order are merged by chunk index.
int host_workers(int64_t n) {
  const unsigned hc = std::thread::hardware_concurrency();
  const int64_t by_size = std::max<int64_t>(1, n / 16384);
  return (int)std::min<int64_t>(std::min<int64_t>(hc ? hc : 1, 32), by_size);
}
// Host threads kept for the setup's row loops: starting a dozen threads per
// loop cost more than the loop's work.  One job at a time (callers from
// several threads take turns); the caller works on the job too.  The
// threads leave when the process destroys the pool.
class HostPool {
 public:
  static HostPool &get() {
    static HostPool pool;
    return pool;
  }
  // f(w) for w = 0 .. n-1, spread over the pool and the caller
  void run(int n, const std::function<void(int)> &f) {
    std::lock_guard<std::mutex> turn(run_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &f;
      njob_ = n;
      next_ = 0;
      pending_ = n;
      ++gen_;
    }
    cv_.notify_all();
    std::unique_lock<std::mutex> lk(mu_);
    work(lk);
    done_.wait(lk, [&] { return pending_ == 0; });
    job_ = nullptr;
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (std::thread &t : th_) t.join();
  }

 private:
  HostPool() {
    const unsigned hc = std::thread::hardware_concurrency();
    const int nt = (int)std::min<unsigned>(hc ? hc : 1, 32) - 1;
    for (int i = 0; i < nt; ++i) th_.emplace_back([this] { loop(); });
  }
  // take items of the current job until none is left (mu_ held on entry and exit)
  void work(std::unique_lock<std::mutex> &lk) {
    while (job_ && next_ < njob_) {
      const int w = next_++;
      const std::function<void(int)> *f = job_;
      lk.unlock();
      (*f)(w);
      lk.lock();
      if (--pending_ == 0) done_.notify_all();
    }
  }
  void loop() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
      if (stop_) return;
      seen = gen_;
      work(lk);
    }
  }
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_;
  std::vector<std::thread> th_;
  const std::function<void(int)> *job_ = nullptr;
  int njob_ = 0, next_ = 0, pending_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

template <typename F>
void parallel_rows(int64_t n, int workers, F &&f) {
  if (workers <= 1) { f(0, (int64_t)0, n); return; }
  const std::function<void(int)> job = [&](int w) { f(w, n * w / workers, n * (w + 1) / workers); };
  HostPool::get().run(workers, job);
}

dd_status validate_and_order(DDHandle *h, const dd_csr *csr, const dd_partition *pt, HostBlocks &hb) {
  const int64_t n = csr->n;
  if (n <= 0 || n > INT32_MAX - 1 || !csr->rowptr || !csr->col || !csr->val) {
    h->err = "invalid CSR arguments";
    return DD_ERR_INVALID_ARG;
  }
  if (csr->rowptr[0] != 0 || csr->rowptr[n] != csr->nnz) {
    h->err = "rowptr[0] must be 0 and rowptr[n] == nnz";
    return DD_ERR_INVALID_ARG;
  }
  const int nw = host_workers(n);
  {
    // first offending row of each chunk; the lowest one is reported
    std::vector<int64_t> bad(nw, -1);
    std::vector<int> why(nw, 0);
    parallel_rows(n, nw, [&](int w, int64_t r0, int64_t r1) {
      for (int64_t i = r0; i < r1 && bad[w] < 0; ++i) {
        if (csr->rowptr[i + 1] < csr->rowptr[i]) { bad[w] = i; why[w] = 1; break; }
        for (int64_t k = csr->rowptr[i]; k < csr->rowptr[i + 1]; ++k) {
          if (csr->col[k] < 0 || csr->col[k] >= n) { bad[w] = i; why[w] = 2; break; }
          if (!isfinite(csr->val[k])) { bad[w] = i; why[w] = 3; break; }
        }
      }
    });
    for (int w = 0; w < nw; ++w)
      if (bad[w] >= 0) {
        if (why[w] == 1) { h->err = "rowptr decreases"; return DD_ERR_INVALID_ARG; }
        if (why[w] == 2) { h->err = "column index out of range"; return DD_ERR_INVALID_ARG; }
        h->err = "non-finite matrix entry";
        return DD_ERR_NONFINITE;
      }
  }
  const int m = pt->m;
  if (m <= 0 || !pt->part) { h->err = "partition needs m >= 1 and part"; return DD_ERR_INVALID_ARG; }
  for (int64_t i = 0; i < n; ++i)
    if (pt->part[i] < -1 || pt->part[i] >= m) { h->err = "part value out of range"; return DD_ERR_INVALID_PARTITION; }
  {
    std::vector<int64_t> bad(nw, -1), badk(nw, -1);
    parallel_rows(n, nw, [&](int w, int64_t r0, int64_t r1) {
      for (int64_t i = r0; i < r1 && bad[w] < 0; ++i)
        for (int64_t k = csr->rowptr[i]; k < csr->rowptr[i + 1]; ++k) {
          const int a = pt->part[i], b = pt->part[csr->col[k]];
          if (a >= 0 && b >= 0 && a != b && csr->val[k] != 0.0) { bad[w] = i; badk[w] = k; break; }
        }
    });
    for (int w = 0; w < nw; ++w)
      if (bad[w] >= 0) {
        const int64_t i = bad[w], k = badk[w];
        char buf[160];
        snprintf(buf, sizeof buf, "entry (%lld,%d) couples interiors %d and %d", (long long)i, csr->col[k],
                 pt->part[i], pt->part[csr->col[k]]);
        h->err = buf;
        return DD_ERR_INVALID_PARTITION;
      }
  }
  hb.off.assign(m + 1, 0);
  for (int64_t i = 0; i < n; ++i) if (pt->part[i] >= 0) hb.off[pt->part[i] + 1]++;
  for (int j = 0; j < m; ++j) hb.off[j + 1] += hb.off[j];
  const int nI = hb.off[m];
  hb.perm.assign(n, 0);
  hb.pos.assign(n, -1);
  if (pt->perm) {
    int j = 0;
    for (int64_t k = 0; k < n; ++k) {
      int o = pt->perm[k];
      if (o < 0 || o >= n || hb.pos[o] >= 0) { h->err = "perm is not a permutation"; return DD_ERR_INVALID_PARTITION; }
      hb.pos[o] = (int32_t)k;
      hb.perm[k] = o;
      if (k < nI) {
        while (j < m && hb.off[j + 1] <= k) ++j;
        if (pt->part[o] != j) { h->err = "perm does not list the interiors subdomain by subdomain"; return DD_ERR_INVALID_PARTITION; }
      } else if (pt->part[o] != -1) {
        h->err = "perm lists an interior node among the interface";
        return DD_ERR_INVALID_PARTITION;
      }
    }
  } else {
    std::vector<int32_t> fill(hb.off.begin(), hb.off.end());
    int32_t g = nI;
    for (int64_t i = 0; i < n; ++i) {
      int32_t k = (pt->part[i] >= 0) ? fill[pt->part[i]]++ : g++;
      hb.perm[k] = (int32_t)i;
      hb.pos[i] = k;
    }
  }
  return DD_OK;
}

dd_status build_aggregates(DDHandle *h, const dd_partition *pt, dd_approx kind, HostBlocks &hb) {
  const int nG = h->nG;
  hb.agg.clear();
  if (nG == 0) { hb.agg.push_back(0); return DD_OK; }
  if (kind == DD_EXACT && !(h->nseg > 1 && pt->agg_offsets)) {  // a batch: one block per system
    hb.agg = {0, nG};
  } else if (pt->agg_offsets) {
    if (pt->n_agg <= 0) { h->err = "n_agg must be positive"; return DD_ERR_INVALID_ARG; }
    hb.agg.assign(pt->agg_offsets, pt->agg_offsets + pt->n_agg + 1);
  } else {
    if (pt->sz <= 0) { h->err = "aggregate size sz must be positive"; return DD_ERR_INVALID_ARG; }
    for (int a = 0; a < nG; a += pt->sz) hb.agg.push_back(a);
    hb.agg.push_back(nG);
  }
  if (hb.agg.front() != 0 || hb.agg.back() != nG) { h->err = "aggregate offsets must run from 0 to n_G"; return DD_ERR_INVALID_ARG; }
  for (size_t i = 0; i + 1 < hb.agg.size(); ++i)
    if (hb.agg[i + 1] <= hb.agg[i]) { h->err = "aggregate offsets must increase"; return DD_ERR_INVALID_ARG; }
  if ((kind == DD_MSCN || kind == DD_MSCNR || kind == DD_OMSCN || kind == DD_OMSCNR) && hb.agg.back() > h->nI) {
    h->err = "MSCN needs n_interior >= n_interface (same local index ranges)";
    return DD_ERR_INVALID_ARG;
  }
  return DD_OK;
}

void extract_blocks(DDHandle *h, const dd_csr *csr, const dd_partition *pt, HostBlocks &hb) {
  const int m = h->m, nI = h->nI, nG = h->nG;
  const int64_t n = h->n;
  hb.kl.assign(m, 0);
  hb.ku.assign(m, 0);
  hb.e_ptr.assign(nI + 1, 0);
  hb.f_ptr.assign(nG + 1, 0);
  const int nw = host_workers(n);
  // bandwidths (per chunk, merged) and per-row counts, rows in the new numbering
  std::vector<std::vector<int32_t>> kl(nw), ku(nw);
  parallel_rows(n, nw, [&](int w, int64_t r0, int64_t r1) {
    kl[w].assign(m, 0);
    ku[w].assign(m, 0);
    for (int64_t r = r0; r < r1; ++r) {
      const int o = hb.perm[r];
      const int jr = pt->part[o];
      int32_t ne = 0;
      for (int64_t k = csr->rowptr[o]; k < csr->rowptr[o + 1]; ++k) {
        const int c = hb.pos[csr->col[k]];
        const int jc = pt->part[csr->col[k]];
        if (jr >= 0 && jc == jr) {
          kl[w][jr] = std::max(kl[w][jr], (int)(r - c));
          ku[w][jr] = std::max(ku[w][jr], (int)(c - r));
        } else if ((jr >= 0 && jc < 0) || (jr < 0 && jc >= 0)) {
          ++ne;
        }
      }
      if (jr >= 0) hb.e_ptr[r + 1] = ne;
      else hb.f_ptr[r - nI + 1] = ne;
    }
  });
  for (int w = 0; w < nw; ++w)
    for (int j = 0; j < m; ++j) {
      hb.kl[j] = std::max(hb.kl[j], kl[w][j]);
      hb.ku[j] = std::max(hb.ku[j], ku[w][j]);
    }
  for (int i = 0; i < nI; ++i) hb.e_ptr[i + 1] += hb.e_ptr[i];
  for (int i = 0; i < nG; ++i) hb.f_ptr[i + 1] += hb.f_ptr[i];
  hb.e_col.assign(hb.e_ptr[nI], 0);
  hb.e_val.assign(hb.e_ptr[nI], 0.0);
  hb.f_col.assign(hb.f_ptr[nG], 0);
  hb.f_val.assign(hb.f_ptr[nG], 0.0);
  // each row fills its own segment, in the order of its entries in C
  parallel_rows(n, nw, [&](int, int64_t r0, int64_t r1) {
    for (int64_t r = r0; r < r1; ++r) {
      const int o = hb.perm[r];
      const int jr = pt->part[o];
      int32_t q = (jr >= 0) ? hb.e_ptr[r] : hb.f_ptr[r - nI];
      for (int64_t k = csr->rowptr[o]; k < csr->rowptr[o + 1]; ++k) {
        const int c = hb.pos[csr->col[k]];
        const int jc = pt->part[csr->col[k]];
        if (jr >= 0 && jc < 0) {
          hb.e_col[q] = c - nI;
          hb.e_val[q++] = csr->val[k];
        } else if (jr < 0 && jc >= 0) {
          hb.f_col[q] = c;
          hb.f_val[q++] = csr->val[k];
        }
      }
    }
  });
}

int64_t launch_cost(const char *call, const DDHandle *h) {
  if (strstr(call, "launch_gj_inverse")) return gj_launch_count(h->pmax, h->prec == DD_FP32 ? 4 : 8);
  if (strstr(call, "launch_hess_solve_update")) return 2;
  if (strstr(call, "launch_schur_apply")) return 2;
  if (strstr(call, "launch_seg_norms")) return 2;
  if (strstr(call, "launch_seg_hess_update")) return 2;
  return 1;
}

}  // namespace

namespace {

// Jobs of the sweep ring for one stage size: runs of consecutive tiles of
// one subdomain whose packed bytes fit a stage (a larger tile is a job of
// its own); forward jobs ascend, backward jobs descend.
void build_jobs(std::vector<BandInfo> &info, const std::vector<TileMeta> &tm, size_t stage, size_t es,
                int tb, int cl, std::vector<SweepJob> &jobs) {
  jobs.clear();
  for (BandInfo &b : info) {
    b.jf0 = (int32_t)jobs.size();
    for (int lo = 0; lo < b.nst;) {
      size_t bytes = 0;
      int hi = lo;
      while (hi < b.nst) {
        const TileMeta &q = tm[b.tile0 + hi];
        // the largest slice of a cluster's CTAs (rank 0's forward rows)
        const size_t nb = (size_t)fwd_split(q.wl, 1, cl) * tb * es + (size_t)round4(q.wl) * 4;
        if (hi > lo && bytes + nb > stage) break;
        bytes += nb;
        ++hi;
      }
      jobs.push_back(SweepJob{lo, hi});
      lo = hi;
    }
    b.njf = (int32_t)jobs.size() - b.jf0;
    b.jb0 = (int32_t)jobs.size();
    for (int hi = b.nst; hi > 0;) {
      size_t bytes = 0;
      int lo = hi;
      while (lo > 0) {
        const TileMeta &q = tm[b.tile0 + lo - 1];
        const size_t nb = (size_t)(tb / cl) * q.wu * es;
        if (lo < hi && bytes + nb > stage) break;
        bytes += nb;
        --lo;
      }
      jobs.push_back(SweepJob{lo, hi});
      hi = lo;
    }
    b.njb = (int32_t)jobs.size() - b.jb0;
    b.jl0 = (int32_t)jobs.size();
    b.njl = 0;
  }
}

// Jobs of the lookahead sweeps: the forward jobs of the one-CTA plan, then
// per subdomain CTA 0's and CTA 1's backward jobs, each sized by that CTA's
// slices of the tiles (a job of CTA 1 whose tiles have no columns for it
// copies nothing).
void build_jobs_la(std::vector<BandInfo> &info, const std::vector<TileMeta> &tm, size_t stage, size_t es,
                   int tb, std::vector<SweepJob> &jobs) {
  build_jobs(info, tm, stage, es, tb, 1, jobs);
  std::vector<SweepJob> out;
  for (BandInfo &b : info) {
    const int jf = (int)out.size();
    for (int q = 0; q < b.njf; ++q) out.push_back(jobs[b.jf0 + q]);
    b.jf0 = jf;
    for (int p = 0; p < 2; ++p) {
      const int j0 = (int)out.size();
      for (int hi = b.nst; hi > 0;) {
        size_t bytes = 0;
        int lo = hi;
        while (lo > 0) {
          const size_t nb = (size_t)tb * la_cols(tm[b.tile0 + lo - 1].wu, tb, p) * es;
          if (lo < hi && bytes + nb > stage) break;
          bytes += nb;
          --lo;
        }
        out.push_back(SweepJob{lo, hi});
        hi = lo;
      }
      if (p == 0) { b.jb0 = j0; b.njb = (int)out.size() - j0; }
      else { b.jl0 = j0; b.njl = (int)out.size() - j0; }
    }
  }
  jobs.swap(out);
}

// Longest processing time first: tasks in order of decreasing cost (ties by
// index), each to the least loaded of `slots` CTAs (ties by CTA index); CTA
// c's tasks are sched[off[c] .. off[c+1]), longest first.
void lpt_schedule(const std::vector<double> &cost, int slots, std::vector<int32_t> &sched,
                  std::vector<int32_t> &off) {
  const int m = (int)cost.size();
  std::vector<int32_t> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  std::vector<double> load(slots, 0.0);
  std::vector<std::vector<int32_t>> lists(slots);
  for (int32_t t : order) {
    int best = 0;
    for (int c = 1; c < slots; ++c)
      if (load[c] < load[best]) best = c;
    load[best] += cost[t];
    lists[best].push_back(t);
  }
  sched.clear();
  off.assign(slots + 1, 0);
  for (int c = 0; c < slots; ++c) {
    sched.insert(sched.end(), lists[c].begin(), lists[c].end());
    off[c + 1] = (int32_t)sched.size();
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// CTAs per subdomain of the sweeps: the option if given; else, in FP64, a
// 2-CTA cluster when every subdomain's cluster is resident at once on the
// device's SMs, and one CTA otherwise.  Measured on the 256x256 workload (64
// subdomains): FP64 interior solves 369 / 391 us with clusters against 398 /
// 410 us with one CTA (the FP64 multiply-adds of a step are split over two
// SMs); FP32 105 / 108 against 97 / 96 us (a step's message round trip costs
// more than halving each SM's shared-memory traffic saves).  The autotuner
// tries both.
template <typename T>
int choose_cluster(const DDHandle *h, size_t stage) {
  (void)stage;
  if (h->sweep_cl_opt >= 1 && h->sweep_cl_opt <= 3) return h->sweep_cl_opt;
  return (sizeof(T) == 8 && 2 * h->m <= sm_count()) ? 2 : 1;
}

// The tiles in the layout of the 2-CTA sweeps (once per handle, after the
// packed tiles): CTA p's slices of every subdomain, forward slices in
// ascending and backward slices in descending tile order, so that a job of
// either direction is one contiguous copy per CTA.
template <typename T>
dd_status build_cluster_layout(DDHandle *h) {
  if (h->cld) return DD_OK;
  int64_t off = 0;
  for (int p = 0; p < 2; ++p)
    for (const BandInfo &b : h->h_info) {
      for (int t = 0; t < b.nst; ++t) {
        int64_t fb, bb;
        cluster_slice_bytes(h->h_tm[b.tile0 + t], h->tb, (int)sizeof(T), p, fb, bb);
        h->h_tm[b.tile0 + t].cfo[p] = off;
        off += fb;
      }
      for (int t = b.nst - 1; t >= 0; --t) {
        int64_t fb, bb;
        cluster_slice_bytes(h->h_tm[b.tile0 + t], h->tb, (int)sizeof(T), p, fb, bb);
        h->h_tm[b.tile0 + t].cbo[p] = off;
        off += bb;
      }
    }
  const int ntiles = (int)h->h_tm.size();
  if (ntiles)
    CK(cudaMemcpyAsync(h->tm, h->h_tm.data(), sizeof(TileMeta) * ntiles, cudaMemcpyHostToDevice, h->stream));
  TRY(dalloc(h, &h->cld, (size_t)std::max<int64_t>(off, 16)));
  CK(launch_cluster_pack<T>(ntiles, h->tb, h->tm, static_cast<const T *>(bufs<T>(h).ltile),
                            static_cast<const T *>(bufs<T>(h).utile), h->src, h->cld, h->stream));
  return DD_OK;
}

// The backward tiles in the layout of the lookahead sweeps (once per handle,
// after the packed tiles): per subdomain, CTA 0's columns of every tile in
// ascending tile order, then CTA 1's, so that a backward job is one
// contiguous copy per CTA.
template <typename T>
dd_status build_la_layout(DDHandle *h) {
  if (h->lad) return DD_OK;
  int64_t off = 0;
  for (const BandInfo &b : h->h_info)
    for (int p = 0; p < 2; ++p)
      for (int t = 0; t < b.nst; ++t) {
        TileMeta &q = h->h_tm[b.tile0 + t];
        q.lao[p] = off;
        off += (int64_t)h->tb * la_cols(q.wu, h->tb, p) * (int64_t)sizeof(T);
      }
  const int ntiles = (int)h->h_tm.size();
  if (ntiles)
    CK(cudaMemcpyAsync(h->tm, h->h_tm.data(), sizeof(TileMeta) * ntiles, cudaMemcpyHostToDevice, h->stream));
  TRY(dalloc(h, &h->lad, (size_t)std::max<int64_t>(off, 16)));
  CK(launch_la_pack<T>(ntiles, h->tb, h->tm, static_cast<const T *>(bufs<T>(h).utile), h->lad, h->stream));
  return DD_OK;
}

// The largest piece a CTA of the lookahead sweeps copies: a forward tile
// with its src (CTA 0), or one CTA's columns of a backward tile
template <typename T>
size_t la_max_unit(const DDHandle *h) {
  size_t u = 0;
  for (const TileMeta &q : h->h_tm)
    u = std::max({u, (size_t)q.wl * h->tb * sizeof(T) + (size_t)round4(q.wl) * 4,
                  (size_t)h->tb * la_cols(q.wu, h->tb, 0) * sizeof(T),
                  (size_t)h->tb * la_cols(q.wu, h->tb, 1) * sizeof(T)});
  return u;
}

// The layout a plan's sweeps stream from, once the packed tiles exist
template <typename T>
dd_status plan_layout(DDHandle *h) {
  if (!h->tiles_ready) return DD_OK;
  if (h->plan.la) {
    TRY(build_la_layout<T>(h));
  } else if (h->plan.cl > 1) {
    TRY(build_cluster_layout<T>(h));
  }
  h->plan.cld = h->cld;
  h->plan.lad = h->lad;
  return DD_OK;
}

// The sweep plan for one stage size: the job table, and a persistent LPT
// schedule when the subdomains outnumber the CTAs that fit on the device.
// mode: 1 one CTA per subdomain, 2 a 2-CTA cluster splitting every step's
// rows, 3 a 2-CTA cluster in the lookahead split (stage 0: its own choice).
template <typename T>
dd_status set_sweep_plan(DDHandle *h, size_t stage, int mode) {
  const int cl = mode == 1 ? 1 : 2, la = mode == 3 ? 1 : 0;
  if (la) {
    // the largest piece either CTA copies; a stage of it or more, three
    // stages when three fit (two copies in flight while one is read)
    const size_t unit = (la_max_unit<T>(h) + 127) & ~(size_t)127;
    const size_t smax = band_sweep_max_stage(h->max_n, h->max_kl, h->max_ku2, sizeof(T), h->tb, cl);
    const size_t s3 = (smax * 2 / 3) & ~(size_t)127;
    if (stage == 0) stage = unit <= s3 ? s3 : smax;
    if (stage > smax && unit <= smax) stage = smax;
    if (stage < unit) stage = unit;
  } else if (cl > 1) {
    // the exchange buffers take room: shrink the stage to what two stages
    // leave, as long as the largest slice of a tile still fits
    const size_t smax = band_sweep_max_stage(h->max_n, h->max_kl, h->max_ku2, sizeof(T), h->tb, cl);
    size_t slice = 0;
    for (const TileMeta &q : h->h_tm)
      slice = std::max({slice, (size_t)fwd_split(q.wl, 1, cl) * h->tb * sizeof(T) + (size_t)round4(q.wl) * 4,
                        (size_t)(h->tb / cl) * q.wu * sizeof(T)});
    slice = (slice + 127) & ~(size_t)127;
    if (stage > smax && slice <= smax) stage = smax;
  }
  std::vector<SweepJob> jobs;
  if (la) build_jobs_la(h->h_info, h->h_tm, stage, sizeof(T), h->tb, jobs);
  else build_jobs(h->h_info, h->h_tm, stage, sizeof(T), h->tb, cl, jobs);
  const int m = h->m;
  if (!h->jobs) TRY(dalloc(h, &h->jobs, 3 * std::max<size_t>(h->h_tm.size(), 1)));
  if (!jobs.empty())
    CK(cudaMemcpyAsync(h->jobs, jobs.data(), sizeof(SweepJob) * jobs.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_info, h->h_info.data(), sizeof(BandInfo) * m, cudaMemcpyHostToDevice, h->stream));
  h->plan.stage_bytes = (uint32_t)stage;
  h->plan.cl = cl;
  h->plan.la = la;
  TRY(plan_layout<T>(h));
  h->plan.threads = la ? 8 * h->tb : 8 * h->tb / cl;
  const int slots = band_sweep_slots<T>(h->max_n, h->max_kl, h->max_ku2, h->tb, cl, h->plan.stage_bytes, la);
  if (slots <= 0) {
    h->err = "a subdomain is too large for the shared-memory sweep (reduce its size or use FP32)";
    return DD_ERR_INVALID_ARG;
  }
  h->stats.sweep_cluster = mode;
  h->stats.sweep_slots = slots;
  h->stats.stage_bytes = (int32_t)stage;
  if (m > slots) {
    std::vector<double> cost(m);
    for (int j = 0; j < m; ++j) {
      const BandInfo &b = h->h_info[j];
      double bytes = 0;
      for (int t = 0; t < b.nst; ++t) {
        const TileMeta &q = h->h_tm[b.tile0 + t];
        bytes += (double)(q.wl + q.wu) * h->tb * sizeof(T);
      }
      cost[j] = 2.0 * b.nst + bytes / 32768.0;  // dependent tile steps + streamed bytes
    }
    std::vector<int32_t> sched, off;
    lpt_schedule(cost, slots, sched, off);
    if (!h->sweep_sched) TRY(dalloc(h, &h->sweep_sched, std::max(m, 1)));
    if (h->sweep_sched_cap < slots + 1) {
      TRY(dalloc(h, &h->sweep_off, slots + 1));
      h->sweep_sched_cap = slots + 1;
    }
    CK(cudaMemcpyAsync(h->sweep_sched, sched.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->sweep_off, off.data(), sizeof(int32_t) * (slots + 1), cudaMemcpyHostToDevice, h->stream));
    // pageable sources: make the copies complete before the vectors go
    CK(cudaStreamSynchronize(h->stream));
    h->plan.grid = slots * cl;
    h->plan.sched = h->sweep_sched;
    h->plan.sched_off = h->sweep_off;
  } else {
    CK(cudaStreamSynchronize(h->stream));
    h->plan.grid = m * cl;
    h->plan.sched = nullptr;
    h->plan.sched_off = nullptr;
  }
  // L2 prefetch of later jobs: only on request.  A streaming probe with 64
  // CTAs and a ring of two 84 KB stages copied 103 GB/s per SM with a
  // prefetch two jobs ahead against 88 without, but the sweeps of the
  // 256x256 workload (64 CTAs) measured slower with it (forward sweep
  // 103 against 95 us).
  h->plan.pf = std::max(h->sweep_pf_opt, 0);
  h->stats.sweep_prefetch = h->plan.pf;
  h->stats.sweep_grid = h->plan.grid;
  return DD_OK;
}

// The network's weight file (format in dd.h): header, FNV-1a hash, then
// out_scale, the feature normalisation and the FP32 master parameters.
struct MlpFile {
  float out_scale = 1.f;
  float mean[DD_MLP_IN], stdv[DD_MLP_IN];
  std::vector<float> params;
};

bool read_mlp_file(const std::string &path, MlpFile &w, std::string &err) {
  FILE *f = fopen(path.c_str(), "rb");
  if (!f) { err = "cannot open the weight file " + path; return false; }
  std::vector<unsigned char> raw;
  unsigned char buf[65536];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) raw.insert(raw.end(), buf, buf + k);
  fclose(f);
  const size_t want = 8 + 12 + 4 + 8 * DD_MLP_IN + 12 * (size_t)DD_MLP_NPARAM + 8 + 8;
  if (raw.size() != want) { err = "weight file has the wrong size"; return false; }
  uint64_t hsh = 0xCBF29CE484222325ull;
  for (size_t i = 0; i + 8 < raw.size(); ++i) { hsh ^= raw[i]; hsh *= 0x100000001B3ull; }
  uint64_t stored = 0;
  for (int i = 7; i >= 0; --i) stored = (stored << 8) | raw[raw.size() - 8 + i];
  if (stored != hsh) { err = "weight file checksum mismatch"; return false; }
  if (memcmp(raw.data(), "DDMLPW01", 8) != 0) { err = "not a weight file"; return false; }
  auto u32 = [&](size_t o) { uint32_t v; memcpy(&v, raw.data() + o, 4); return v; };
  if (u32(8) != 1 || u32(12) != DD_MLP_IN || u32(16) != DD_MLP_HIDDEN) {
    err = "unsupported weight file version or shape";
    return false;
  }
  size_t o = 20;
  memcpy(&w.out_scale, raw.data() + o, 4); o += 4;
  memcpy(w.mean, raw.data() + o, 4 * DD_MLP_IN); o += 4 * DD_MLP_IN;
  memcpy(w.stdv, raw.data() + o, 4 * DD_MLP_IN); o += 4 * DD_MLP_IN;
  w.params.resize(DD_MLP_NPARAM);
  memcpy(w.params.data(), raw.data() + o, 4 * (size_t)DD_MLP_NPARAM);
  for (int i = 0; i < DD_MLP_IN; ++i)
    if (!(w.stdv[i] > 0.f) || !isfinite(w.mean[i])) { err = "weight file: invalid normalisation"; return false; }
  for (float v : w.params)
    if (!isfinite(v)) { err = "weight file: non-finite parameter"; return false; }
  return true;
}

// BF16 value of v (round to nearest even), as a float
float bf16_round(float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return v;  // inf / nan kept
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// DD_LEARNED blocks: G_ii + Delta on the patterns, inverted; a block whose
// inversion fails the pivot test takes its MSCE_INF block (built and
// inverted only when some block fails).
template <typename T, typename Msce>
dd_status learned_blocks(DDHandle *h, const dd_csr *csr, HostBlocks &hb, const std::vector<int32_t> &agg_of,
                         const std::vector<int32_t> &p, const std::vector<int64_t> &soff,
                         const std::vector<int64_t> &poff, double pivtol, Msce &msce_into,
                         const int64_t *d_gidx, const double *d_gval, int64_t gcount) {
  PrecBufs<T> &B = bufs<T>(h);
  cudaStream_t s = h->stream;
  const int nI = h->nI, nG = h->nG, nagg = h->nagg;
  MlpFile w;
  std::string err;
  if (!read_mlp_file(h->mlp_path, w, err)) { h->err = err; return DD_ERR_INVALID_ARG; }
  // the patterns P_a: G entries, the structure of F E, and the diagonal
  std::vector<int32_t> ents;
  {
    std::vector<int32_t> cols;
    for (int a = 0; a < nagg; ++a) {
      const int g0 = hb.agg[a], g1 = hb.agg[a + 1];
      for (int r = g0; r < g1; ++r) {
        cols.clear();
        cols.push_back(r);
        const int o = hb.perm[nI + r];
        for (int64_t k = csr->rowptr[o]; k < csr->rowptr[o + 1]; ++k) {
          const int c = hb.pos[csr->col[k]] - nI;
          if (c >= g0 && c < g1 && csr->val[k] != 0.0) cols.push_back(c);
        }
        for (int q = hb.f_ptr[r]; q < hb.f_ptr[r + 1]; ++q) {
          if (hb.f_val[q] == 0.0) continue;
          const int kk = hb.f_col[q];
          for (int e = hb.e_ptr[kk]; e < hb.e_ptr[kk + 1]; ++e) {
            const int c = hb.e_col[e];
            if (c >= g0 && c < g1 && hb.e_val[e] != 0.0) cols.push_back(c);
          }
        }
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        for (int c : cols) { ents.push_back(a); ents.push_back(r - g0); ents.push_back(c - g0); }
      }
    }
  }
  const int64_t ne = (int64_t)ents.size() / 3;
  h->l_ents = ents;
  h->stats.learned_entries = ne;
  // E^T (values per interface column), 1 / diag(D)
  std::vector<int32_t> et_ptr(nG + 1, 0);
  for (int k = 0; k < nI; ++k)
    for (int e = hb.e_ptr[k]; e < hb.e_ptr[k + 1]; ++e) et_ptr[hb.e_col[e] + 1]++;
  for (int g = 0; g < nG; ++g) et_ptr[g + 1] += et_ptr[g];
  std::vector<double> et_val(et_ptr[nG]);
  {
    std::vector<int32_t> fill(et_ptr.begin(), et_ptr.end() - 1);
    for (int k = 0; k < nI; ++k)
      for (int e = hb.e_ptr[k]; e < hb.e_ptr[k + 1]; ++e) et_val[fill[hb.e_col[e]]++] = hb.e_val[e];
  }
  std::vector<double> dinv(std::max(nI, 1), 0.0);
  for (int k = 0; k < nI; ++k) {
    const int o = hb.perm[k];
    double d = 0.0;
    for (int64_t q = csr->rowptr[o]; q < csr->rowptr[o + 1]; ++q)
      if (csr->col[q] == o) d = csr->val[q];
    dinv[k] = d != 0.0 ? 1.0 / d : 0.0;
  }
  std::vector<float> wbf(DD_MLP_NPARAM);
  for (int q = 0; q < DD_MLP_NPARAM; ++q) wbf[q] = bf16_round(w.params[q]);
  std::vector<float> mean(w.mean, w.mean + DD_MLP_IN), stdv(w.stdv, w.stdv + DD_MLP_IN);
  LearnedArgs la;
  int32_t *d_ent, *d_et_ptr, *d_fp, *d_fc, *d_ep, *d_ec;
  double *d_etv, *d_dinv, *d_fv, *d_ev;
  float *d_w, *d_mean, *d_std;
  TRY(upload(h, &d_ent, ents));
  TRY(upload(h, &d_et_ptr, et_ptr));
  TRY(upload(h, &d_etv, et_val));
  TRY(upload(h, &d_dinv, dinv));
  TRY(upload(h, &d_fp, hb.f_ptr));
  TRY(upload(h, &d_fc, hb.f_col));
  TRY(upload(h, &d_fv, hb.f_val));
  TRY(upload(h, &d_ep, hb.e_ptr));
  TRY(upload(h, &d_ec, hb.e_col));
  TRY(upload(h, &d_ev, hb.e_val));
  TRY(upload(h, &d_w, wbf));
  TRY(upload(h, &d_mean, mean));
  TRY(upload(h, &d_std, stdv));
  TRY(dalloc(h, &h->l_feat, (size_t)std::max<int64_t>(ne, 1) * DD_MLP_IN));
  TRY(dalloc(h, &h->l_delta, (size_t)std::max<int64_t>(ne, 1)));
  la.n_ent = ne;
  la.ent = d_ent;
  la.agg_off = h->agg_off;
  la.s_off = h->s_off;
  la.perm_iface = h->d_perm + nI;
  la.c_rowptr = h->c_rowptr;
  la.c_col = h->c_col;
  la.c_val = h->c_val;
  la.f_ptr = d_fp; la.f_col = d_fc; la.f_val = d_fv;
  la.e_ptr = d_ep; la.e_col = d_ec; la.e_val = d_ev;
  la.et_ptr = d_et_ptr; la.et_val = d_etv;
  la.dinv = d_dinv;
  la.wbf = d_w;
  la.mean = d_mean;
  la.stdv = d_std;
  la.out_scale = w.out_scale;
  la.feat = h->l_feat;
  la.delta = h->l_delta;
  h->stats.launches += 1;
  CK(launch_learned_delta<T>(la, B.S, s));
  // invert; failures go to a scratch status word and the failed flags
  TRY(dalloc(h, &h->st_probe, 1));
  CK(cudaMemsetAsync(h->st_probe, 0, sizeof(DevStatus), s));
  CK(launch_block_amax<T>(nagg, h->d_p, h->s_off, B.S, B.amax, s));
  CK(launch_gj_inverse<T>(nagg, h->d_p, h->s_off, h->pmax, B.S, h->ipiv, h->poff, B.amax, h->failed, B.gj,
                          pivtol, h->st_probe, DD_ERR_SINGULAR_SCHUR, s, h->gj_tc));
  std::vector<int32_t> failed(nagg, 0);
  if (nagg) CK(cudaMemcpyAsync(failed.data(), h->failed, sizeof(int32_t) * nagg, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int32_t> fb;
  for (int a = 0; a < nagg; ++a)
    if (failed[a]) fb.push_back(a);
  h->stats.learned_fallback = (int32_t)fb.size();
  if (fb.empty()) return DD_OK;
  // fallback: MSCE_INF blocks into a second buffer, the failed ones inverted and copied over
  T *S2 = nullptr;
  TRY(dalloc(h, &S2, soff[nagg]));
  CK(cudaMemsetAsync(S2, 0, sizeof(T) * std::max<int64_t>(soff[nagg], 1), s));
  CK(launch_scatter_coo<T>(gcount, d_gidx, d_gval, S2, s));
  TRY(msce_into(S2));
  std::vector<int32_t> fp;
  std::vector<int64_t> fo, fpo(1, 0);
  int fpmax = 0;
  for (int a : fb) {
    fp.push_back(p[a]);
    fo.push_back(soff[a]);
    fpo.push_back(fpo.back() + p[a]);
    fpmax = std::max(fpmax, p[a]);
  }
  int32_t *d_fpp, *d_ff;
  int64_t *d_fo, *d_fpo;
  T *famax;
  TRY(upload(h, &d_fpp, fp));
  TRY(upload(h, &d_fo, fo));
  TRY(upload(h, &d_fpo, fpo));
  TRY(dalloc(h, &d_ff, fb.size()));
  TRY(dalloc(h, &famax, fb.size()));
  CK(launch_block_amax<T>((int)fb.size(), d_fpp, d_fo, S2, famax, s));
  CK(launch_gj_inverse<T>((int)fb.size(), d_fpp, d_fo, fpmax, S2, h->ipiv, d_fpo, famax, d_ff, B.gj, pivtol,
                          h->st, DD_ERR_SINGULAR_SCHUR, s, h->gj_tc));
  for (size_t q = 0; q < fb.size(); ++q)
    CK(cudaMemcpyAsync(B.S + soff[fb[q]], S2 + soff[fb[q]], sizeof(T) * (size_t)p[fb[q]] * p[fb[q]],
                       cudaMemcpyDeviceToDevice, s));
  (void)poff;
  (void)agg_of;
  return DD_OK;
}

// C in SELL-32 form (SellC): inside every window of DD_SELL_WINDOW rows the
// rows are ordered by decreasing length (a counting sort, ties by row), cut
// into slices of 32, and each slice is stored entry-major at the width of its
// longest row, the shorter rows padded with value 0 at their last column.
dd_status build_sell(DDHandle *h, const dd_csr *csr) {
  const int64_t n = h->n, ns = (n + 31) / 32, W = DD_SELL_WINDOW;
  int32_t lmax = 0;
  for (int64_t i = 0; i < n; ++i) lmax = std::max(lmax, csr->rowptr[i + 1] - csr->rowptr[i]);
  std::vector<int32_t> order(ns * 32, -1);
  {
    std::vector<int32_t> cnt(lmax + 2);
    for (int64_t w0 = 0; w0 < n; w0 += W) {
      const int64_t w1 = std::min(n, w0 + W);
      std::fill(cnt.begin(), cnt.end(), 0);
      for (int64_t i = w0; i < w1; ++i) ++cnt[lmax - (csr->rowptr[i + 1] - csr->rowptr[i]) + 1];
      for (int q = 1; q <= lmax + 1; ++q) cnt[q] += cnt[q - 1];
      for (int64_t i = w0; i < w1; ++i) order[w0 + cnt[lmax - (csr->rowptr[i + 1] - csr->rowptr[i])]++] = (int32_t)i;
    }
  }
  std::vector<int64_t> off(ns + 1, 0);
  for (int64_t sl = 0; sl < ns; ++sl) {
    int32_t w = 0;
    for (int r = 0; r < 32; ++r) {
      const int32_t row = order[sl * 32 + r];
      if (row >= 0) w = std::max(w, csr->rowptr[row + 1] - csr->rowptr[row]);
    }
    off[sl + 1] = off[sl] + 32 * (int64_t)w;
  }
  std::vector<int32_t> col(std::max<int64_t>(off[ns], 1));
  std::vector<double> val(std::max<int64_t>(off[ns], 1));
  parallel_rows(ns, host_workers(n), [&](int, int64_t s0, int64_t s1) {
    for (int64_t sl = s0; sl < s1; ++sl) {
      const int w = (int)((off[sl + 1] - off[sl]) / 32);
      for (int r = 0; r < 32; ++r) {
        const int32_t row = order[sl * 32 + r];
        const int32_t k0 = row >= 0 ? csr->rowptr[row] : 0, len = row >= 0 ? csr->rowptr[row + 1] - k0 : 0;
        for (int k = 0; k < w; ++k) {
          const int64_t e = off[sl] + 32 * (int64_t)k + r;
          col[e] = k < len ? csr->col[k0 + k] : (len > 0 ? csr->col[k0 + len - 1] : std::max(row, 0));
          val[e] = k < len ? csr->val[k0 + k] : 0.0;
        }
      }
    }
  });
  int64_t *d_off;
  int32_t *d_row, *d_col;
  double *d_val;
  TRY(upload(h, &d_off, off));
  TRY(upload(h, &d_row, order));
  TRY(upload(h, &d_col, col));
  TRY(upload(h, &d_val, val));
  h->sell.nslices = ns;
  h->sell.n = n;
  h->sell.st = h->st;
  h->sell.off = d_off;
  h->sell.row = d_row;
  h->sell.col = d_col;
  h->sell.val = d_val;
  h->sell_entries = off[ns];
  return DD_OK;
}

// MSCN / MSCNR blocks on index ranges [g0[a], g1[a]) of the interface
// (Algorithm 1's principal submatrices with the same local range in D, E, F
// and G): S_a -= F_a D_a^-1 E_a (rowsum: only the row sums, on the
// diagonal).  S holds G_a already, block a at d_soff[a]; d_p, d_soff,
// d_poff, ipiv, failed, gj and amax describe / serve these blocks.  A range
// whose E_a or F_a vanishes keeps G_a (D_a is then not needed: identity).
template <typename T>
dd_status principal_blocks(DDHandle *h, const dd_csr *csr, const HostBlocks &hb, const std::vector<int32_t> &g0v,
                           const std::vector<int32_t> &g1v, bool rowsum, T *S, const int32_t *d_p,
                           const int64_t *d_soff, const int64_t *d_poff, int32_t *ipiv, int32_t *failed, T *gj,
                           T *amax, double pivtol) {
  PrecBufs<T> &B = bufs<T>(h);
  cudaStream_t s = h->stream;
  const int nb = (int)g0v.size();
  std::vector<int64_t> soff(nb + 1, 0);
  int pmax = 0;
  for (int a = 0; a < nb; ++a) {
    const int pa = g1v[a] - g0v[a];
    soff[a + 1] = soff[a] + (int64_t)pa * pa;
    pmax = std::max(pmax, pa);
  }
  std::vector<int64_t> di, ei, fi;
  std::vector<double> dv, ev, fv;
  for (int a = 0; a < nb; ++a) {
    const int g0 = g0v[a], g1 = g1v[a], pa = g1 - g0;
    bool nzE = false, nzF = false;
    size_t e0 = ei.size(), f0 = fi.size();
    for (int r = g0; r < g1; ++r)
      for (int k = hb.e_ptr[r]; k < hb.e_ptr[r + 1]; ++k) {
        int c = hb.e_col[k];
        if (c >= g0 && c < g1 && hb.e_val[k] != 0.0) {
          ei.push_back(soff[a] + (int64_t)(r - g0) * pa + (c - g0));
          ev.push_back(hb.e_val[k]);
          nzE = true;
        }
      }
    for (int r = g0; r < g1; ++r)
      for (int k = hb.f_ptr[r]; k < hb.f_ptr[r + 1]; ++k) {
        int c = hb.f_col[k];
        if (c >= g0 && c < g1 && hb.f_val[k] != 0.0) {
          fi.push_back(soff[a] + (int64_t)(r - g0) * pa + (c - g0));
          fv.push_back(hb.f_val[k]);
          nzF = true;
        }
      }
    if (!nzE || !nzF) {
      // F_a D_a^-1 E_a vanishes: D_a is not needed, take the identity
      ei.resize(e0); ev.resize(e0); fi.resize(f0); fv.resize(f0);
      for (int r = 0; r < pa; ++r) { di.push_back(soff[a] + (int64_t)r * pa + r); dv.push_back(1.0); }
      continue;
    }
    for (int r = g0; r < g1; ++r) {
      const int o = hb.perm[r];
      for (int64_t k = csr->rowptr[o]; k < csr->rowptr[o + 1]; ++k) {
        const int c = hb.pos[csr->col[k]];
        if (c >= g0 && c < g1) { di.push_back(soff[a] + (int64_t)(r - g0) * pa + (c - g0)); dv.push_back(csr->val[k]); }
      }
    }
  }
  TRY(dalloc(h, &B.Dm, soff[nb]));
  TRY(dalloc(h, &B.Em, soff[nb]));
  TRY(dalloc(h, &B.Fm, soff[nb]));
  TRY(dalloc(h, &B.Tm, soff[nb]));
  T *blocks4[4] = {B.Dm, B.Em, B.Fm, B.Tm};
  for (int q = 0; q < 4; ++q)
    CK(cudaMemsetAsync(blocks4[q], 0, sizeof(T) * std::max<int64_t>(soff[nb], 1), s));
  int64_t *d_i;
  double *d_v;
  TRY(upload(h, &d_i, di)); TRY(upload(h, &d_v, dv));
  CK(launch_scatter_coo<T>((int64_t)di.size(), d_i, d_v, B.Dm, s));
  TRY(upload(h, &d_i, ei)); TRY(upload(h, &d_v, ev));
  CK(launch_scatter_coo<T>((int64_t)ei.size(), d_i, d_v, B.Em, s));
  TRY(upload(h, &d_i, fi)); TRY(upload(h, &d_v, fv));
  CK(launch_scatter_coo<T>((int64_t)fi.size(), d_i, d_v, B.Fm, s));
  CK(launch_block_amax<T>(nb, d_p, d_soff, B.Dm, amax, s));
  CK(launch_gj_inverse<T>(nb, d_p, d_soff, pmax, B.Dm, ipiv, d_poff, amax, failed, gj, pivtol, h->st,
                          DD_ERR_SINGULAR_SCHUR, s, h->gj_tc));
  if (!rowsum) {
    CK(launch_block_gemm<T>(nb, d_p, d_soff, pmax, B.Dm, B.Em, B.Tm, T(1), T(0), s));
    CK(launch_block_gemm<T>(nb, d_p, d_soff, pmax, B.Fm, B.Tm, S, T(-1), T(1), s));
  } else {
    CK(launch_mscnr_diag<T>(nb, d_p, d_soff, pmax, B.Dm, B.Em, B.Fm, S, s));
  }
  return DD_OK;
}

// S_hat of the overlapped kinds (OMSCN / OMSCNR / OLUM) into S (dense
// n_G x n_G): block a spans agg[a] .. agg[a+1] - 1 + w_a with w_a =
// min(overlap, p_{a+1}), w_k = 0 (Algorithm 1); G on each block, minus the
// MSCN / MSCNR term, then the blocks placed in aggregate order with a later
// block overwriting the overlap.
template <typename T>
dd_status overlapped_schur(DDHandle *h, const dd_csr *csr, const HostBlocks &hb, double pivtol, T *S) {
  cudaStream_t s = h->stream;
  const int k = (int)hb.agg.size() - 1, nG = h->nG, nI = h->nI;
  if (k <= 0) return DD_OK;
  std::vector<int32_t> w(k, 0), g0(k), g1(k), q(k);
  std::vector<int64_t> xoff(k + 1, 0), qoff(k + 1, 0);
  for (int a = 0; a < k; ++a) {
    if (a + 1 < k) w[a] = std::min(h->overlap, hb.agg[a + 2] - hb.agg[a + 1]);
    g0[a] = hb.agg[a];
    g1[a] = hb.agg[a + 1] + w[a];
    q[a] = g1[a] - g0[a];
    xoff[a + 1] = xoff[a] + (int64_t)q[a] * q[a];
    qoff[a + 1] = qoff[a] + q[a];
  }
  // G on every extended block
  std::vector<int64_t> gi;
  std::vector<double> gv;
  for (int a = 0; a < k; ++a)
    for (int g = g0[a]; g < g1[a]; ++g) {
      const int o = hb.perm[nI + g];
      for (int64_t e = csr->rowptr[o]; e < csr->rowptr[o + 1]; ++e) {
        const int c = hb.pos[csr->col[e]] - nI;
        if (c < g0[a] || c >= g1[a]) continue;
        gi.push_back(xoff[a] + (int64_t)(g - g0[a]) * q[a] + (c - g0[a]));
        gv.push_back(csr->val[e]);
      }
    }
  T *Sx;
  TRY(dalloc(h, &Sx, xoff[k]));
  CK(cudaMemsetAsync(Sx, 0, sizeof(T) * std::max<int64_t>(xoff[k], 1), s));
  int64_t *d_gi;
  double *d_gv;
  TRY(upload(h, &d_gi, gi));
  TRY(upload(h, &d_gv, gv));
  CK(launch_scatter_coo<T>((int64_t)gi.size(), d_gi, d_gv, Sx, s));
  int32_t *d_q, *d_agg, *d_w, *ipiv, *failed;
  int64_t *d_xoff, *d_qoff;
  TRY(upload(h, &d_q, q));
  TRY(upload(h, &d_xoff, xoff));
  TRY(upload(h, &d_qoff, qoff));
  TRY(upload(h, &d_agg, hb.agg));
  TRY(upload(h, &d_w, w));
  if (h->kind != DD_OLUM) {
    T *gj, *amax;
    TRY(dalloc(h, &ipiv, qoff[k]));
    TRY(dalloc(h, &failed, k));
    TRY(dalloc(h, &gj, gj_scratch_elems(k, qoff[k], sizeof(T))));
    TRY(dalloc(h, &amax, k));
    TRY(principal_blocks<T>(h, csr, hb, g0, g1, h->kind == DD_OMSCNR, Sx, d_q, d_xoff, d_qoff, ipiv, failed, gj,
                            amax, pivtol));
  }
  CK(launch_assemble_overlapped<T>(nG, k, d_agg, d_w, d_xoff, Sx, S, s));
  return DD_OK;
}

// MSCE with a finite radius r (DD_MSCE): S_a -= F(R_a, D_r) D_r^-1
// E(D_r, R_a), where D_r holds the interior nodes within path length r of
// aggregate a (first step through F or E, then through the pattern of D),
// closed by the D-neighbours of every zero-diagonal node.  The node sets are
// host index work; D_r, E and F go to dense blocks, D_r is inverted by the
// blocked Gauss-Jordan kernels and the two products are batched GEMMs.
template <typename T>
dd_status msce_radius_blocks(DDHandle *h, const dd_csr *csr, const HostBlocks &hb, double pivtol, T *S,
                             const std::vector<int64_t> &soff) {
  cudaStream_t s = h->stream;
  const int k = (int)hb.agg.size() - 1, nI = h->nI;
  const int R = h->radius;
  if (R <= 0 || nI == 0 || k <= 0) return DD_OK;  // r = 0: S_a = G_a (LUM)
  // symmetrised pattern of D and its zero-diagonal nodes
  std::vector<int32_t> aptr(nI + 1, 0), adj;
  std::vector<char> zdiag(nI, 1);
  for (int kk = 0; kk < nI; ++kk) {
    const int o = hb.perm[kk];
    for (int64_t e = csr->rowptr[o]; e < csr->rowptr[o + 1]; ++e) {
      const int j = hb.pos[csr->col[e]];
      if (j == kk && csr->val[e] != 0.0) zdiag[kk] = 0;
      if (j < nI && j != kk) { aptr[kk + 1]++; aptr[j + 1]++; }
    }
  }
  for (int kk = 0; kk < nI; ++kk) aptr[kk + 1] += aptr[kk];
  adj.resize(aptr[nI]);
  {
    std::vector<int32_t> fill(aptr.begin(), aptr.end() - 1);
    for (int kk = 0; kk < nI; ++kk) {
      const int o = hb.perm[kk];
      for (int64_t e = csr->rowptr[o]; e < csr->rowptr[o + 1]; ++e) {
        const int j = hb.pos[csr->col[e]];
        if (j < nI && j != kk) { adj[fill[kk]++] = j; adj[fill[j]++] = kk; }
      }
    }
  }
  // E transposed: interior rows of every interface column
  std::vector<int32_t> etp(h->nG + 1, 0), etr;
  for (int r = 0; r < nI; ++r)
    for (int e = hb.e_ptr[r]; e < hb.e_ptr[r + 1]; ++e)
      if (hb.e_val[e] != 0.0) etp[hb.e_col[e] + 1]++;
  for (int g = 0; g < h->nG; ++g) etp[g + 1] += etp[g];
  etr.resize(etp[h->nG]);
  {
    std::vector<int32_t> fill(etp.begin(), etp.end() - 1);
    for (int r = 0; r < nI; ++r)
      for (int e = hb.e_ptr[r]; e < hb.e_ptr[r + 1]; ++e)
        if (hb.e_val[e] != 0.0) etr[fill[hb.e_col[e]]++] = r;
  }
  // the node set of every aggregate, then the dense blocks
  std::vector<int32_t> bd, ba;  // blocks with a non-empty D_r: their size, aggregate
  std::vector<int64_t> doff(1, 0), eoff(1, 0), poff(1, 0);
  std::vector<int64_t> di, ei, fi;
  std::vector<double> dv, ev, fv;
  std::vector<int32_t> dist(nI, -1), loc(nI, -1), set;
  int dmax = 0, pmax = 0;
  for (int a = 0; a < k; ++a) {
    const int g0 = hb.agg[a], g1 = hb.agg[a + 1], pa = g1 - g0;
    set.clear();
    for (int g = g0; g < g1; ++g) {
      for (int e = hb.f_ptr[g]; e < hb.f_ptr[g + 1]; ++e) {
        const int j = hb.f_col[e];
        if (hb.f_val[e] != 0.0 && dist[j] < 0) { dist[j] = 1; set.push_back(j); }
      }
      for (int e = etp[g]; e < etp[g + 1]; ++e) {
        const int j = etr[e];
        if (dist[j] < 0) { dist[j] = 1; set.push_back(j); }
      }
    }
    for (size_t head = 0; head < set.size(); ++head) {
      const int kk = set[head];
      if (dist[kk] >= R) continue;
      for (int e = aptr[kk]; e < aptr[kk + 1]; ++e)
        if (dist[adj[e]] < 0) { dist[adj[e]] = dist[kk] + 1; set.push_back(adj[e]); }
    }
    const size_t d0 = set.size();
    for (size_t q0 = 0; q0 < d0; ++q0) {
      const int kk = set[q0];
      if (!zdiag[kk]) continue;
      for (int e = aptr[kk]; e < aptr[kk + 1]; ++e)
        if (dist[adj[e]] < 0) { dist[adj[e]] = R + 1; set.push_back(adj[e]); }
    }
    std::sort(set.begin(), set.end());
    const int d = (int)set.size();
    for (int q2 = 0; q2 < d; ++q2) loc[set[q2]] = q2;
    if (d > 0) {
      const int b = (int)bd.size();
      bd.push_back(d);
      ba.push_back(a);
      for (int q2 = 0; q2 < d; ++q2) {
        const int kk = set[q2], o = hb.perm[kk];
        for (int64_t e = csr->rowptr[o]; e < csr->rowptr[o + 1]; ++e) {
          const int c = hb.pos[csr->col[e]];
          if (c < nI && loc[c] >= 0) { di.push_back(doff[b] + (int64_t)q2 * d + loc[c]); dv.push_back(csr->val[e]); }
        }
        for (int e = hb.e_ptr[kk]; e < hb.e_ptr[kk + 1]; ++e) {
          const int c = hb.e_col[e];
          if (c >= g0 && c < g1) { ei.push_back(eoff[b] + (int64_t)q2 * pa + (c - g0)); ev.push_back(hb.e_val[e]); }
        }
      }
      for (int g = g0; g < g1; ++g)
        for (int e = hb.f_ptr[g]; e < hb.f_ptr[g + 1]; ++e) {
          const int j = hb.f_col[e];
          if (loc[j] >= 0) { fi.push_back(eoff[b] + (int64_t)(g - g0) * d + loc[j]); fv.push_back(hb.f_val[e]); }
        }
      doff.push_back(doff[b] + (int64_t)d * d);
      eoff.push_back(eoff[b] + (int64_t)d * pa);
      poff.push_back(poff[b] + d);
      dmax = std::max(dmax, d);
      pmax = std::max(pmax, pa);
    }
    for (int kk : set) { dist[kk] = -1; loc[kk] = -1; }
  }
  const int nb = (int)bd.size();
  if (nb == 0) return DD_OK;
  if (dmax > 12288) { h->err = "MSCE: a reached interior set exceeds 12288 nodes (reduce the radius)"; return DD_ERR_INVALID_ARG; }
  h->stats.msce_nodes_max = dmax;
  // device blocks
  T *Dr, *Er, *Fr, *Tr, *gj, *amax;
  int32_t *ipiv, *failed, *d_bd;
  int64_t *d_doff, *d_poff;
  TRY(dalloc(h, &Dr, doff[nb]));
  TRY(dalloc(h, &Er, eoff[nb]));
  TRY(dalloc(h, &Fr, eoff[nb]));
  TRY(dalloc(h, &Tr, eoff[nb]));
  CK(cudaMemsetAsync(Dr, 0, sizeof(T) * doff[nb], s));
  CK(cudaMemsetAsync(Er, 0, sizeof(T) * std::max<int64_t>(eoff[nb], 1), s));
  CK(cudaMemsetAsync(Fr, 0, sizeof(T) * std::max<int64_t>(eoff[nb], 1), s));
  int64_t *d_i;
  double *d_v;
  TRY(upload(h, &d_i, di)); TRY(upload(h, &d_v, dv));
  CK(launch_scatter_coo<T>((int64_t)di.size(), d_i, d_v, Dr, s));
  TRY(upload(h, &d_i, ei)); TRY(upload(h, &d_v, ev));
  CK(launch_scatter_coo<T>((int64_t)ei.size(), d_i, d_v, Er, s));
  TRY(upload(h, &d_i, fi)); TRY(upload(h, &d_v, fv));
  CK(launch_scatter_coo<T>((int64_t)fi.size(), d_i, d_v, Fr, s));
  TRY(upload(h, &d_bd, bd));
  TRY(upload(h, &d_doff, doff));
  TRY(upload(h, &d_poff, poff));
  TRY(dalloc(h, &ipiv, poff[nb]));
  TRY(dalloc(h, &failed, nb));
  TRY(dalloc(h, &gj, gj_scratch_elems(nb, poff[nb], sizeof(T))));
  TRY(dalloc(h, &amax, nb));
  CK(launch_block_amax<T>(nb, d_bd, d_doff, Dr, amax, s));
  CK(launch_gj_inverse<T>(nb, d_bd, d_doff, dmax, Dr, ipiv, d_poff, amax, failed, gj, pivtol, h->st,
                          DD_ERR_SINGULAR_SCHUR, s, h->gj_tc));
  // T_b = D_r^-1 E_b (d x p), then S_a -= F_b T_b (p x p)
  std::vector<int32_t> dims1, dims2;
  std::vector<int64_t> offs1, offs2;
  for (int b = 0; b < nb; ++b) {
    const int a = ba[b], d = bd[b], pa = hb.agg[a + 1] - hb.agg[a];
    dims1.insert(dims1.end(), {d, pa, d});
    offs1.insert(offs1.end(), {doff[b], eoff[b], eoff[b]});
    dims2.insert(dims2.end(), {pa, pa, d});
    offs2.insert(offs2.end(), {eoff[b], eoff[b], soff[a]});
  }
  int32_t *d_dims1, *d_dims2;
  int64_t *d_offs1, *d_offs2;
  TRY(upload(h, &d_dims1, dims1));
  TRY(upload(h, &d_offs1, offs1));
  TRY(upload(h, &d_dims2, dims2));
  TRY(upload(h, &d_offs2, offs2));
  CK(launch_rect_gemm<T>(nb, d_dims1, d_offs1, dmax, pmax, Dr, Er, Tr, T(1), T(0), s));
  CK(launch_rect_gemm<T>(nb, d_dims2, d_offs2, pmax, pmax, Fr, Tr, S, T(-1), T(1), s));
  return DD_OK;
}

template <typename T>
dd_status setup_device(DDHandle *h, const dd_csr *csr, const dd_partition *pt, HostBlocks &hb,
                       double pivtol) {
  PrecBufs<T> &B = bufs<T>(h);
  const int m = h->m, nI = h->nI, nG = h->nG;
  cudaStream_t s = h->stream;
  // ---- interior factors: geometry
  std::vector<BandInfo> info(m);
  int64_t band = 0, lraw = 0, pivo = 0, fac_nz = 0;
  int32_t tiles = 0, panels = 0;
  int max_panels = 0;
  h->max_n = h->max_kl = h->max_ku = h->max_ku2 = h->max_tiles = 0;
  for (int j = 0; j < m; ++j) {
    BandInfo &b = info[j];
    memset(&b, 0, sizeof b);
    b.n = hb.off[j + 1] - hb.off[j];
    b.kl = hb.kl[j];
    b.ku = hb.ku[j];
    b.ntiles = (b.n + DD_NB - 1) / DD_NB;
    b.row0 = hb.off[j];
    b.band_off = band; band += (int64_t)b.n * bi_wd(b);
    b.lraw_off = lraw; lraw += (int64_t)b.ntiles * bi_lraw_elems(b);
    b.piv_off = pivo; pivo += b.n;
    b.panel0 = panels; panels += b.ntiles;
    h->max_kl = std::max(h->max_kl, b.kl);
    h->max_ku = std::max(h->max_ku, b.ku);
    h->max_ku2 = std::max(h->max_ku2, b.kl + b.ku);
    max_panels = std::max(max_panels, b.ntiles);
    // in-band entries of L (kl per column) and U (kl+ku+1 per row), clipped
    for (int i = 0; i < b.n; ++i) fac_nz += std::min(b.kl, b.n - 1 - i) + std::min(b.kl + b.ku, b.n - 1 - i) + 1;
  }
  h->stats.factor_nonzeros = fac_nz;
  h->stats.kl_max = h->max_kl;
  h->stats.ku_max = h->max_ku;
  TRY(upload(h, &h->d_info, info));
  TRY(dalloc(h, &B.band, band));
  CK(cudaMemsetAsync(B.band, 0, sizeof(T) * std::max<int64_t>(band, 1), s));
  TRY(dalloc(h, &B.lm, lraw));  // the blocked LU's multipliers, one block per tile
  {
    const size_t wb = band_lu_window_bytes(h->max_kl, h->max_ku, sizeof(T));
    T *wscr = nullptr;
    if (wb > 200 * 1024) TRY(dalloc(h, &wscr, (wb / sizeof(T)) * (size_t)m));
    h->lu_scratch = wscr;
  }
  TRY(dalloc(h, &h->piv, pivo));
  // ---- C itself (FP64, original numbering) for the SpMV
  TRY(upload_ptr(h, &h->c_rowptr, csr->rowptr, (size_t)h->n + 1));
  TRY(upload_ptr(h, &h->c_col, csr->col, (size_t)h->nnz));
  TRY(upload_ptr(h, &h->c_val, csr->val, (size_t)h->nnz));
  int32_t *d_part = nullptr, *d_pos = nullptr;
  TRY(upload_ptr(h, &d_part, pt->part, (size_t)h->n));
  TRY(upload(h, &d_pos, hb.pos));
  TRY(upload(h, &h->d_perm, hb.perm));
  h->stats.launches += 1;
  fill_band_kernel<T><<<(unsigned)((h->n + 255) / 256), 256, 0, s>>>(
      (int)h->n, h->c_rowptr, h->c_col, h->c_val, d_part, d_pos, h->d_info, B.band);
  CK(cudaGetLastError());
  {
    // persistent LPT task lists when the subdomains outnumber resident CTAs
    const int lu_threads = sizeof(T) == 4 ? 512 : 256;  // the kernel's launch bound per precision
    const int occ = band_lu_occupancy<T>(h->max_kl, h->max_ku, lu_threads);
    if (occ <= 0) { h->err = "band LU: no resident CTA fits"; return DD_ERR_CUDA; }
    const int slots = occ * sm_count();
    int32_t *d_sched = nullptr, *d_off = nullptr;
    if (m > slots) {
      std::vector<double> cost(m);
      for (int j = 0; j < m; ++j)
        cost[j] = (double)info[j].n * (info[j].kl + 1) * (info[j].kl + info[j].ku + 1);
      std::vector<int32_t> sched, off;
      lpt_schedule(cost, slots, sched, off);
      TRY(upload(h, &d_sched, sched));
      TRY(upload(h, &d_off, off));
    }
    T *cnorm = nullptr;  // column norms of the incomplete factorisation
    if (h->ilu_tol > 0) TRY(dalloc(h, &cnorm, std::max(nI, 1)));
    CK(launch_band_lu<T>(h->d_info, m, h->max_kl, h->max_ku, B.band, B.lm, h->piv,
                         static_cast<T *>(h->lu_scratch), pivtol, h->st, lu_threads, slots, d_sched, d_off,
                         cnorm, h->ilu_tol, s));
  }
  // ---- host work while the band LU runs.  Its allocations and uploads go
  // to the side stream: a pageable copy queued behind the LU on the main
  // stream would hold the host until the LU ends.  The main stream waits
  // for the side stream before the tile packing.
  if (!h->ustream) CK(cudaStreamCreateWithFlags(&h->ustream, cudaStreamNonBlocking));
  if (!h->uev) CK(cudaEventCreateWithFlags(&h->uev, cudaEventDisableTiming));
  h->astream = h->ustream;
  TRY(build_sell(h, csr));
  // ---- couplings E (interior x interface) and F (interface x interior)
  TRY(upload(h, &h->e_ptr, hb.e_ptr));
  TRY(upload(h, &h->e_col, hb.e_col));
  TRY(upload_T(h, &B.e_val, hb.e_val));
  TRY(upload(h, &h->f_ptr, hb.f_ptr));
  TRY(upload(h, &h->f_col, hb.f_col));
  TRY(upload_T(h, &B.f_val, hb.f_val));
  h->stats.coupling_nnz = (int64_t)hb.e_col.size() + (int64_t)hb.f_col.size();
  // ---- interface blocks.  The overlapped kinds build their blocks apart and
  // assemble S_hat into one block of the whole interface, which the apply
  // then inverts whole (the blocks of the apply are aggA).
  const bool ovl_kind = h->kind == DD_OMSCN || h->kind == DD_OMSCNR || h->kind == DD_OLUM;
  const std::vector<int32_t> aggA = ovl_kind ? std::vector<int32_t>{0, nG} : hb.agg;
  const int nagg = (int)aggA.size() - 1;
  h->nagg = nagg;
  std::vector<int32_t> p(nagg), agg_of(nG);
  std::vector<int64_t> soff(nagg + 1, 0), poff(nagg + 1, 0);
  h->pmax = 0;
  for (int a = 0; a < nagg; ++a) {
    p[a] = aggA[a + 1] - aggA[a];
    soff[a + 1] = soff[a] + (int64_t)p[a] * p[a];
    poff[a + 1] = poff[a] + p[a];
    h->pmax = std::max(h->pmax, p[a]);
    for (int g = aggA[a]; g < aggA[a + 1]; ++g) agg_of[g] = a;
  }
  if (h->pmax > 12288) {
    h->err = ovl_kind ? "overlapped kinds invert the whole interface: n_G must be <= 12288"
                      : "an aggregate exceeds 12288 interface nodes";
    return DD_ERR_INVALID_ARG;
  }
  h->stats.n_agg = (int32_t)hb.agg.size() - 1;
  h->stats.max_agg = h->pmax;
  h->stats.schur_bytes = soff[nagg] * (int64_t)sizeof(T);
  TRY(upload(h, &h->agg_off, aggA));
  TRY(upload(h, &h->d_p, p));
  TRY(upload(h, &h->s_off, soff));
  TRY(upload(h, &h->poff, poff));
  TRY(dalloc(h, &B.S, soff[nagg]));
  TRY(dalloc(h, &B.amax, nagg));
  TRY(dalloc(h, &B.gj, gj_scratch_elems(nagg, poff[nagg], sizeof(T))));
  TRY(dalloc(h, &h->ipiv, poff[nagg]));
  TRY(dalloc(h, &h->failed, nagg));
  // G(R_a, R_a): the entries' positions in S (scattered after the join)
  int64_t *d_gidx = nullptr;
  double *d_gval = nullptr;
  size_t gcount = 0;
  if (!ovl_kind) {
    std::vector<int64_t> idx;
    std::vector<double> val;
    for (int g = 0; g < nG; ++g) {
      const int o = hb.perm[nI + g];
      const int a = agg_of[g];
      for (int64_t k = csr->rowptr[o]; k < csr->rowptr[o + 1]; ++k) {
        const int c = hb.pos[csr->col[k]] - nI;
        if (c < 0 || agg_of[c] != a) continue;
        idx.push_back(soff[a] + (int64_t)(g - hb.agg[a]) * p[a] + (c - hb.agg[a]));
        val.push_back(csr->val[k]);
      }
    }
    TRY(upload(h, &d_gidx, idx));
    TRY(upload(h, &d_gval, val));
    gcount = idx.size();
  }
  // S_dst(R_a, R_a) -= sum_j F(R_a, I_j) A_jj^-1 E(I_j, R_a) (MSCE_INF / EXACT,
  // and the learned kind's base): per subdomain the interface columns of E
  // (gam) and interface rows of F (fr), the scatter of E into the columns
  // X_j, and the colours of the accumulation, all built on the host while
  // the band LU runs
  struct MsceLists {
    int32_t *gam_ptr = nullptr, *gam_idx = nullptr, *gam_agg = nullptr, *fr_ptr = nullptr, *fr_row = nullptr,
            *fr_agg = nullptr, *fs_ptr = nullptr, *fs_col = nullptr, *ncols = nullptr, *jlist = nullptr;
    int64_t *xoff = nullptr, *xidx = nullptr;
    double *xval = nullptr;
    int64_t nx = 0, xsize = 0;
    int max_fr = 0, max_gam = 0;
    std::vector<int32_t> cptr;
  } ml;
  auto msce_prep = [&]() -> dd_status {
    std::vector<int32_t> gam_ptr(m + 1, 0), gam_idx, gam_agg, fr_ptr(m + 1, 0), fr_row, fr_agg;
    std::vector<int32_t> fs_ptr(1, 0), fs_col;
    std::vector<double> fs_val;
    std::vector<int32_t> ncols(m, 0);
    std::vector<int64_t> xoff(m + 1, 0);
    std::vector<int32_t> mark(nG, -1);
    std::vector<std::vector<int32_t>> frs(m);
    for (int g = 0; g < nG; ++g) {
      int last = -1;
      for (int k = hb.f_ptr[g]; k < hb.f_ptr[g + 1]; ++k) {
        int c = hb.f_col[k];
        int j = (int)(std::upper_bound(hb.off.begin(), hb.off.end(), c) - hb.off.begin()) - 1;
        if (j != last && (frs[j].empty() || frs[j].back() != g)) frs[j].push_back(g);
        last = j;
      }
    }
    std::vector<int64_t> xidx;
    std::vector<double> xval;
    for (int j = 0; j < m; ++j) {
      const int r0 = hb.off[j], r1 = hb.off[j + 1], nj = r1 - r0;
      std::vector<int32_t> cols;
      for (int r = r0; r < r1; ++r)
        for (int k = hb.e_ptr[r]; k < hb.e_ptr[r + 1]; ++k) cols.push_back(hb.e_col[k]);
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      for (size_t q = 0; q < cols.size(); ++q) mark[cols[q]] = (int32_t)q;
      ncols[j] = (int32_t)cols.size();
      xoff[j + 1] = xoff[j] + (int64_t)nj * cols.size();
      for (int c : cols) { gam_idx.push_back(c); gam_agg.push_back(agg_of[c]); }
      gam_ptr[j + 1] = (int32_t)gam_idx.size();
      for (int r = r0; r < r1; ++r)
        for (int k = hb.e_ptr[r]; k < hb.e_ptr[r + 1]; ++k) {
          xidx.push_back(xoff[j] + (int64_t)mark[hb.e_col[k]] * nj + (r - r0));
          xval.push_back(hb.e_val[k]);
        }
      for (int c : cols) mark[c] = -1;
      for (int g : frs[j]) {
        fr_row.push_back(g);
        fr_agg.push_back(agg_of[g]);
        for (int k = hb.f_ptr[g]; k < hb.f_ptr[g + 1]; ++k) {
          int c = hb.f_col[k];
          if (c >= r0 && c < r1) { fs_col.push_back(c - r0); fs_val.push_back(hb.f_val[k]); }
        }
        fs_ptr.push_back((int32_t)fs_col.size());
      }
      fr_ptr[j + 1] = (int32_t)fr_row.size();
      ml.max_fr = std::max(ml.max_fr, (int)frs[j].size());
      ml.max_gam = std::max(ml.max_gam, (int)cols.size());
    }
    // colours: a subdomain takes the first colour that no earlier subdomain
    // sharing an interface row with it holds, so the sum over j of every
    // entry of S runs in colour order, the same on every run (no atomics)
    std::vector<int32_t> color(m, -1), jlist;
    ml.cptr.assign(1, 0);
    {
      std::vector<std::vector<int32_t>> subs_of(nG);  // subdomains of each interface row
      for (int j = 0; j < m; ++j)
        for (int q = fr_ptr[j]; q < fr_ptr[j + 1]; ++q) subs_of[fr_row[q]].push_back(j);
      int ncolor = 0;
      std::vector<int32_t> seen;  // colour -> last subdomain that saw it taken
      for (int j = 0; j < m; ++j) {
        seen.assign(ncolor + 1, -1);
        for (int q = fr_ptr[j]; q < fr_ptr[j + 1]; ++q)
          for (int j2 : subs_of[fr_row[q]])
            if (j2 < j && color[j2] >= 0) seen[color[j2]] = j;
        int c = 0;
        while (c < ncolor && seen[c] == j) ++c;
        color[j] = c;
        ncolor = std::max(ncolor, c + 1);
      }
      for (int c = 0; c < ncolor; ++c) {
        for (int j = 0; j < m; ++j)
          if (color[j] == c) jlist.push_back(j);
        ml.cptr.push_back((int32_t)jlist.size());
      }
    }
    TRY(upload(h, &ml.gam_ptr, gam_ptr));
    TRY(upload(h, &ml.gam_idx, gam_idx));
    TRY(upload(h, &ml.gam_agg, gam_agg));
    TRY(upload(h, &ml.fr_ptr, fr_ptr));
    TRY(upload(h, &ml.fr_row, fr_row));
    TRY(upload(h, &ml.fr_agg, fr_agg));
    TRY(upload(h, &ml.fs_ptr, fs_ptr));
    TRY(upload(h, &ml.fs_col, fs_col));
    TRY(upload_T(h, &B.fsub_val, fs_val));
    TRY(upload(h, &ml.ncols, ncols));
    TRY(upload(h, &ml.xoff, xoff));
    TRY(upload(h, &ml.xidx, xidx));
    TRY(upload(h, &ml.xval, xval));
    TRY(upload(h, &ml.jlist, jlist));
    TRY(dalloc(h, &B.X, xoff[m]));
    ml.nx = (int64_t)xidx.size();
    ml.xsize = xoff[m];
    return DD_OK;
  };
  auto msce_into = [&](T *Sdst) -> dd_status {
    CK(cudaMemsetAsync(B.X, 0, sizeof(T) * std::max<int64_t>(ml.xsize, 1), s));
    CK(launch_scatter_coo<T>(ml.nx, ml.xidx, ml.xval, B.X, s));
    // X_j = A_jj^-1 E(I_j, gam_j)
    CK(launch_band_solve_multi<T>(h->d_info, m, ml.ncols, ml.xoff, ml.max_gam, h->max_kl, h->max_ku2, h->tb,
                                  h->tm, B.ltile, B.utile, h->src, B.X, s));
    // S(R_a,R_a) -= F(R_a, I_j) X_j, one launch per colour of subdomains
    for (size_t c = 0; c + 1 < ml.cptr.size(); ++c)
      CK(launch_schur_accumulate<T>(ml.cptr[c + 1] - ml.cptr[c], ml.jlist + ml.cptr[c], ml.fr_ptr, ml.fr_row,
                                    ml.fr_agg, ml.fs_ptr, ml.fs_col, B.fsub_val, ml.gam_ptr, ml.gam_idx,
                                    ml.gam_agg, ml.xoff, h->d_info, B.X, h->agg_off, h->s_off, Sdst, ml.max_fr,
                                    ml.max_gam, s));
    return DD_OK;
  };
  if (h->kind == DD_MSCE_INF || h->kind == DD_EXACT || h->kind == DD_LEARNED) TRY(msce_prep());
  CK(cudaEventRecord(h->uev, h->ustream));
  h->astream = nullptr;
  CK(cudaStreamWaitEvent(s, h->uev, 0));
  // ---- packed sweep tiles: widths from the factors, offsets and jobs here
  {
    int32_t *d_wl = nullptr, *d_wu = nullptr;
    TRY(dalloc(h, &d_wl, panels));
    TRY(dalloc(h, &d_wu, panels));
    CK(launch_tile_widths<T>(h->d_info, m, max_panels, B.band, B.lm, h->piv, d_wl, d_wu, s));
    std::vector<int32_t> pwl(panels), pwu(panels);
    if (panels) {
      CK(cudaMemcpyAsync(pwl.data(), d_wl, sizeof(int32_t) * panels, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(pwu.data(), d_wu, sizeof(int32_t) * panels, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    // A sweep tile's widths cover those of its panels (offset by the
    // panel's start within the tile).  The wide tile is taken when two ring
    // stages of its largest tile fit beside the resident vectors.
    std::vector<int32_t> wl, wu;
    std::vector<TileMeta> tm;
    int64_t lofs = 0, uofs = 0, sofs = 0;
    size_t max_tile = 0, smax = 0;
    int tb = 0;
    for (int cand : {DD_TB_WIDE, DD_NB}) {
      tiles = 0;
      int max_n = 0, max_t = 0;
      for (int j = 0; j < m; ++j) {
        BandInfo &b = info[j];
        b.nst = (b.n + cand - 1) / cand;
        b.tile0 = tiles;
        tiles += b.nst;
        max_n = std::max(max_n, b.nst * cand);
        max_t = std::max(max_t, b.nst);
      }
      wl.assign(tiles, 0);
      wu.assign(tiles, 0);
      for (int j = 0; j < m; ++j) {
        const BandInfo &b = info[j];
        for (int t = 0; t < b.nst; ++t) {
          int l = cand, u = cand;
          for (int q = 0; q < cand / DD_NB; ++q) {
            const int pn = t * (cand / DD_NB) + q;
            if (pn >= b.ntiles) break;
            l = std::max(l, q * DD_NB + pwl[b.panel0 + pn]);
            u = std::max(u, q * DD_NB + pwu[b.panel0 + pn]);
          }
          wl[b.tile0 + t] = round4(l);
          wu[b.tile0 + t] = round4(u);
        }
      }
      tm.assign(tiles, TileMeta{});
      lofs = uofs = sofs = 0;
      max_tile = 0;
      for (int t = 0; t < tiles; ++t) {
        tm[t].lofs = lofs; tm[t].uofs = uofs; tm[t].sofs = sofs;
        tm[t].wl = wl[t]; tm[t].wu = wu[t];
        lofs += (int64_t)wl[t] * cand;
        uofs += (int64_t)cand * wu[t];
        sofs += round4(wl[t]);
        max_tile = std::max(max_tile, std::max((size_t)wl[t] * cand * sizeof(T) + (size_t)round4(wl[t]) * 4,
                                               (size_t)cand * wu[t] * sizeof(T)));
      }
      smax = band_sweep_max_stage(max_n, h->max_kl, h->max_ku2, sizeof(T), cand);
      if (((max_tile + 127) & ~(size_t)127) <= smax || cand == DD_NB) {
        tb = cand;
        h->max_n = max_n;
        h->max_tiles = max_t;
        break;
      }
    }
    h->tb = tb;
    h->stats.tile = tb;
    // stage: ~84 KiB, or one whole tile when a tile is larger; smaller when
    // two such stages do not fit beside the resident vectors
    size_t stage = std::max<size_t>(84 * 1024, max_tile);
    stage = (stage + 127) & ~(size_t)127;
    if (stage > smax) stage = std::max((max_tile + 127) & ~(size_t)127, smax);
    h->max_tile = max_tile;
    h->h_info = info;
    h->h_tm = tm;
    TRY(upload(h, &h->tm, tm));
    const int mode = choose_cluster<T>(h, stage);
    TRY(set_sweep_plan<T>(h, mode == 3 ? 0 : stage, mode));  // 0: the lookahead split sizes its own stages
    info = h->h_info;
    TRY(dalloc(h, &B.ltile, lofs));
    TRY(dalloc(h, &B.utile, uofs));
    TRY(dalloc(h, &h->src, sofs));
    h->stats.factor_bytes = (lofs + uofs) * (int64_t)sizeof(T) + sofs * (int64_t)sizeof(int32_t);
    CK(launch_band_tiles<T>(h->d_info, m, h->max_tiles, h->max_kl, h->tb, h->tm, B.band, B.lm, h->piv,
                            B.ltile, B.utile, h->src, s));
    h->tiles_ready = true;
    TRY(plan_layout<T>(h));
  }
  // G(R_a, R_a) into S
  CK(cudaMemsetAsync(B.S, 0, sizeof(T) * std::max<int64_t>(soff[nagg], 1), s));
  if (ovl_kind) {
    TRY(overlapped_schur<T>(h, csr, hb, pivtol, B.S));
  } else {
    CK(launch_scatter_coo<T>((int64_t)gcount, d_gidx, d_gval, B.S, s));
  }
  if (h->kind == DD_MSCE_INF || h->kind == DD_EXACT) {
    TRY(msce_into(B.S));
  } else if (h->kind == DD_LEARNED) {
    TRY(learned_blocks<T>(h, csr, hb, agg_of, p, soff, poff, pivtol, msce_into, d_gidx, d_gval,
                          (int64_t)gcount));
    TRY(dalloc(h, &B.z1, std::max(nI, 1)));
    TRY(dalloc(h, &B.z2, std::max(nG, 1)));
    TRY(dalloc(h, &B.t, std::max(nG, 1)));
    return DD_OK;  // the blocks are inverted (with their fallbacks)
  } else if (h->kind == DD_MSCE) {
    TRY(msce_radius_blocks<T>(h, csr, hb, pivtol, B.S, soff));
  } else if (h->kind == DD_MSCN || h->kind == DD_MSCNR) {
    std::vector<int32_t> g0(nagg), g1(nagg);
    for (int a = 0; a < nagg; ++a) { g0[a] = hb.agg[a]; g1[a] = hb.agg[a + 1]; }
    TRY(principal_blocks<T>(h, csr, hb, g0, g1, h->kind == DD_MSCNR, B.S, h->d_p, h->s_off, h->poff,
                            h->ipiv, h->failed, B.gj, B.amax, pivtol));
  }
  // ---- explicit inverses of the S_hat blocks
  CK(launch_block_amax<T>(nagg, h->d_p, h->s_off, B.S, B.amax, s));
  CK(launch_gj_inverse<T>(nagg, h->d_p, h->s_off, h->pmax, B.S, h->ipiv, h->poff, B.amax,
                          h->failed, B.gj, pivtol, h->st, DD_ERR_SINGULAR_SCHUR, s, h->gj_tc));
  TRY(dalloc(h, &B.z1, std::max(nI, 1)));
  TRY(dalloc(h, &B.z2, std::max(nG, 1)));
  TRY(dalloc(h, &B.t, std::max(nG, 1)));
  return DD_OK;
}

template <typename T>
dd_status apply_T(DDHandle *h, const double *y, double *x, cudaStream_t s, int part = -1) {
  PrecBufs<T> &B = bufs<T>(h);
  SweepPlan pl = h->plan;
  pl.first_wait = h->first_wait;
  const int32_t *agg_sys = nullptr, *act = nullptr;
  if (h->masked) {
    pl.task_sys = h->sub_sys;
    pl.act = h->d_act;
    agg_sys = h->agg_sys;
    act = h->d_act;
  }
  if (part == 0 || part < 0)
  CK(launch_band_solve_fwd<T>(h->d_info, h->m, h->max_n, h->max_kl, h->max_ku2, pl,
                              h->tm, h->jobs, B.ltile, B.utile, h->src, y, h->d_perm, B.z1, h->st, s));
  if (part == 1 || part < 0)
  CK(launch_schur_apply<T>(h->nagg, h->agg_off, h->s_off, h->pmax, B.S, h->f_ptr, h->f_col,
                           B.f_val, y, h->d_perm + h->nI, B.z1, B.z2, B.t, h->nG, x, agg_sys, act, s));
  if (part == 2 || part < 0)
  CK(launch_band_solve_bwd<T>(h->d_info, h->m, h->max_n, h->max_kl, h->max_ku2, pl,
                              h->tm, h->jobs, B.ltile, B.utile, h->src, h->e_ptr, h->e_col, B.e_val,
                              B.z2, B.z1, h->d_perm, x, h->st, s));
  return DD_OK;
}

dd_status apply_any(DDHandle *h, const double *y, double *x, cudaStream_t s, int part = -1) {
  return h->prec == DD_FP32 ? apply_T<float>(h, y, x, s, part) : apply_T<double>(h, y, x, s, part);
}

}  // namespace

namespace {

// CTAs of the batched Krylov kernels over the systems with act[q] != 0
// (all when act is null): proportional to the rows, at least one each, all
// nb CTAs used; c0[q] is system q's first CTA, cseg[c] CTA c's system.
void assign_ctas(const std::vector<int64_t> &row0, const int32_t *act, int nb, std::vector<int32_t> &c0,
                 std::vector<int32_t> &cseg) {
  const int S = (int)row0.size() - 1;
  std::vector<int64_t> rows(S);
  int64_t N = 0;
  int na = 0;
  for (int q = 0; q < S; ++q) {
    rows[q] = (!act || act[q]) ? row0[q + 1] - row0[q] : 0;
    N += rows[q];
    na += (!act || act[q]) ? 1 : 0;
  }
  std::vector<int32_t> cnt(S, 0);
  int tot = 0;
  if (na > 0)
    for (int q = 0; q < S; ++q) {
      if (act && !act[q]) continue;
      cnt[q] = (int32_t)std::max<int64_t>(1, (rows[q] * nb) / std::max<int64_t>(N, 1));
      tot += cnt[q];
    }
  while (na > 0 && tot > nb) {  // trim the system with the most CTAs
    const int q = (int)(std::max_element(cnt.begin(), cnt.end()) - cnt.begin());
    --cnt[q];
    --tot;
  }
  while (na > 0 && tot < nb) {  // add to the system with the most rows per CTA
    int best = -1;
    double worst = -1.0;
    for (int q = 0; q < S; ++q) {
      if (cnt[q] == 0) continue;
      const double per = (double)rows[q] / cnt[q];
      if (per > worst) { worst = per; best = q; }
    }
    ++cnt[best];
    ++tot;
  }
  c0.assign(S + 1, 0);
  cseg.clear();
  for (int q = 0; q < S; ++q) {
    c0[q + 1] = c0[q] + cnt[q];
    for (int c = 0; c < cnt[q]; ++c) cseg.push_back(q);
  }
}

dd_status alloc_krylov(DDHandle *h, int R) {
  const int S = h->nseg;
  h->Rmax = R;
  h->ldv = ((h->n + 31) / 32) * 32;
  TRY(dalloc(h, &h->V, (size_t)h->ldv * (R + 1)));
  TRY(dalloc(h, &h->Z, (size_t)h->ldv * R));
  // the batched apply reads every system's vectors, stepping or not
  CK(cudaMemsetAsync(h->V, 0, sizeof(double) * (size_t)h->ldv * (R + 1), h->stream));
  CK(cudaMemsetAsync(h->Z, 0, sizeof(double) * (size_t)h->ldv * R, h->stream));
  TRY(dalloc(h, &h->H, (size_t)S * (R + 1) * R));
  TRY(dalloc(h, &h->cs, (size_t)S * R));
  TRY(dalloc(h, &h->sn, (size_t)S * R));
  TRY(dalloc(h, &h->g, (size_t)S * (R + 1)));
  TRY(dalloc(h, &h->y, (size_t)S * (R + 1)));
  TRY(dalloc(h, &h->hc1, (size_t)S * (R + 2)));
  TRY(dalloc(h, &h->hc2, (size_t)S * (R + 2)));
  TRY(dalloc(h, &h->nsq, 4));
  TRY(dalloc(h, &h->out, (size_t)S * 4));
  h->cgs_blocks = cgs2_blocks(h->krylov_per_sm, 1024, h->krylov_threads);
  if (h->cgs_blocks <= 0) { h->err = "no resident blocks for the cooperative CGS2 kernel"; return DD_ERR_CUDA; }
  TRY(dalloc(h, &h->partial, 3 * (size_t)std::max(h->nblocks, h->cgs_blocks) * (R + 2)));
  TRY(dalloc(h, &h->r, h->ldv));
  cudaError_t e = cudaMallocHost(&h->h_out, sizeof(double) * std::max(8, 4 * S));
  if (e != cudaSuccess) { h->err = "cudaMallocHost failed"; return DD_ERR_OOM; }
  if (S > 1) {
    // CTAs of the batched Krylov kernels: proportional to the rows, at least one each
    const int nb = h->cgs_blocks;
    if (S > nb) { h->err = "more systems in the batch than resident CTAs of the CGS2 kernel"; return DD_ERR_INVALID_ARG; }
    std::vector<int32_t> c0, cseg;
    assign_ctas(h->seg_row0_h, nullptr, nb, c0, cseg);
    h->seg_ctas = c0[S];
    TRY(upload(h, &h->seg_cta0, c0));
    TRY(upload(h, &h->cta_seg, cseg));
    // the CGS2 kernel's map over the systems still stepping (rewritten when
    // that set changes); starts as the full map
    TRY(upload(h, &h->seg_cta0_act, c0));
    TRY(upload(h, &h->cta_seg_act, cseg));
    {
      std::vector<int32_t> rs(h->n);
      for (int q = 0; q < S; ++q)
        for (int64_t i = h->seg_row0_h[q]; i < h->seg_row0_h[q + 1]; ++i) rs[i] = q;
      TRY(upload(h, &h->row_sys, rs));
    }
    TRY(upload(h, &h->seg_row0, h->seg_row0_h));
    TRY(dalloc(h, &h->d_act, S));
    TRY(dalloc(h, &h->d_jl, S));
    TRY(upload(h, &h->sub_sys, h->sub_sys_h));
    TRY(upload(h, &h->agg_sys, h->agg_sys_h));
    if ((int)h->agg_sys_h.size() != h->nagg || (int)h->sub_sys_h.size() != h->m) {
      h->err = "batch maps do not match the subdomains and aggregates";
      return DD_ERR_INVALID_ARG;
    }
    TRY(dalloc(h, &h->bcat, (size_t)h->n));
    TRY(dalloc(h, &h->xcat, (size_t)h->n));
    TRY(dalloc(h, &h->bn2, S));
    TRY(dalloc(h, &h->rn2, S));
    e = cudaMallocHost(&h->h_act, sizeof(int32_t) * 2 * S);
    if (e != cudaSuccess) { h->err = "cudaMallocHost failed"; return DD_ERR_OOM; }
  }
  return DD_OK;
}

SegMap single_map(const DDHandle *h) {
  SegMap sm;
  sm.nseg = 1;
  sm.rmax = h->Rmax;
  return sm;
}

SegMap batch_map(const DDHandle *h) {
  SegMap sm;
  sm.nseg = h->nseg;
  sm.rmax = h->Rmax;
  sm.cta_seg = h->cta_seg;
  sm.seg_cta0 = h->seg_cta0;
  sm.seg_row0 = h->seg_row0;
  sm.act = h->d_act;
  return sm;
}

// the map of the Arnoldi step: every CTA on a system still stepping
SegMap step_map(const DDHandle *h) {
  SegMap sm = batch_map(h);
  sm.cta_seg = h->cta_seg_act;
  sm.seg_cta0 = h->seg_cta0_act;
  return sm;
}

// new active set: the step map follows it (host copy, then upload)
dd_status remap_active(DDHandle *h, cudaStream_t s) {
  std::vector<int32_t> c0, cseg;
  assign_ctas(h->seg_row0_h, h->h_act, h->cgs_blocks, c0, cseg);
  if ((int)cseg.size() != h->cgs_blocks) return DD_OK;  // nothing stepping
  CK(cudaMemcpyAsync(h->seg_cta0_act, c0.data(), sizeof(int32_t) * c0.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->cta_seg_act, cseg.data(), sizeof(int32_t) * cseg.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return DD_OK;
}

// nsq[slot] = ||v||^2
dd_status norm_sq(DDHandle *h, const double *v, int slot, cudaStream_t s) {
  CK(launch_multidot((int)h->n, 1, v, h->ldv, v, h->partial, h->nblocks, s));
  CK(launch_reduce_cols(h->nblocks, 1, h->partial, h->nsq + slot, 0, s));
  return DD_OK;
}

dd_status read_scalars(DDHandle *h, const double *d, int count, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->h_out, d, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return DD_OK;
}

// The launches of Arnoldi step j: z_j = B^-1 v_j, w = C z_j, CGS2 with the
// Givens update, and the step's scalars (4 per system) to pinned host memory.
dd_status arnoldi_step(DDHandle *h, int j, int R, const SegMap &sm, int ncta, const double *bn2,
                       cudaStream_t s) {
  double *vj = h->V + (int64_t)j * h->ldv, *zj = h->Z + (int64_t)j * h->ldv;
  double *w = h->V + (int64_t)(j + 1) * h->ldv;
  TRY(apply_any(h, vj, zj, s));
  const bool timed = h->time_kernels && sm.nseg == 1;
  if (timed) CK(cudaEventRecord(h->kev[0], s));
  if (sm.nseg > 1)  // a batch: only the rows of systems still stepping
    CK(launch_spmv_masked(h->sell, zj, w, h->row_sys, sm.act, s));
  else
    CK(launch_spmv(h->sell, zj, w, s));
  if (timed) CK(cudaEventRecord(h->kev[1], s));
  CK(launch_cgs2(h->n, j, R, h->V, h->ldv, w, h->partial, h->Rmax + 2, h->hc1, h->hc2, h->H, h->cs,
                 h->sn, h->g, bn2, h->out, sm, ncta, h->krylov_threads, s));
  if (timed) CK(cudaEventRecord(h->kev[2], s));
  // one system: the scalars of steps j and j + 1 go to different halves of
  // the pinned buffer, so a step launched ahead cannot overwrite the ones the
  // host is about to read
  double *dst = sm.nseg > 1 ? h->h_out : h->h_out + 4 * (j & 1);
  CK(cudaMemcpyAsync(dst, h->out, sizeof(double) * 4 * sm.nseg, cudaMemcpyDeviceToHost, s));
  return DD_OK;
}

void drop_graphs(DDHandle *h) {
  for (cudaGraphExec_t &e : h->gexec)
    if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  h->graph_key = -1;
}

// Step j as one CUDA graph, captured on first use (per restart length and
// mode) and replayed afterwards; without use_graph, plain launches.
dd_status run_step(DDHandle *h, int j, int R, const SegMap &sm, int ncta, const double *bn2,
                   cudaStream_t s) {
  if (!h->use_graph) return arnoldi_step(h, j, R, sm, ncta, bn2, s);
  const int key = 2 * R + (sm.nseg > 1 ? 1 : 0);
  if (h->graph_key != key) {
    drop_graphs(h);
    h->graph_key = key;
    h->gexec.assign(h->Rmax, nullptr);
    h->glaunch.assign(h->Rmax, 0);
  }
  if (!h->gexec[j]) {
    const int64_t l0 = h->stats.launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const dd_status rc = arnoldi_step(h, j, R, sm, ncta, bn2, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (rc != DD_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ec != cudaSuccess) { h->err = std::string("graph capture: ") + cudaGetErrorString(ec); return DD_ERR_CUDA; }
    const cudaError_t ei = cudaGraphInstantiate(&h->gexec[j], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->gexec[j] = nullptr;
      h->err = std::string("graph instantiate: ") + cudaGetErrorString(ei);
      return DD_ERR_CUDA;
    }
    h->glaunch[j] = h->stats.launches - l0;  // counted while capturing, charged per replay
    h->stats.launches = l0;
    h->stats.graphs += 1;
  }
  h->stats.launches += h->glaunch[j];
  CK(cudaGraphLaunch(h->gexec[j], s));
  return DD_OK;
}

// The status word the apply's kernels record into (a bounded wait that gave
// up); reading it synchronises the stream.  clear: reset it to DD_OK.
dd_status device_status(DDHandle *h, cudaStream_t s, bool clear = false) {
  DevStatus dst{};
  CK(cudaMemcpyAsync(&dst, h->st, sizeof dst, cudaMemcpyDeviceToHost, s));
  if (clear) CK(cudaMemsetAsync(h->st, 0, sizeof dst, s));
  CK(cudaStreamSynchronize(s));
  if (dst.code != 0) {
    char buf[96];
    snprintf(buf, sizeof buf, "a bounded device wait gave up in an apply sweep (subdomain %d)", dst.block);
    h->err = buf;
    return (dd_status)dst.code;
  }
  return DD_OK;
}

dd_status fgmres(DDHandle *h, const double *b, double *x, double tol, int R, int maxit,
                 dd_info *info, cudaStream_t s) {
  const int n = (int)h->n;
  int iters = 0, restarts = 0;
  double relres = 0.0;
  dd_status rc = DD_ERR_NOT_CONVERGED;
  const SegMap sm = single_map(h);
  CK(cudaMemsetAsync(h->st, 0, sizeof(DevStatus), s));  // this solve's own status
  CK(launch_zero(x, n, s));
  TRY(norm_sq(h, b, 2, s));
  TRY(read_scalars(h, h->nsq + 2, 1, s));
  const double bnorm = sqrt(h->h_out[0]);
  if (!isfinite(bnorm)) return DD_ERR_NONFINITE;
  if (bnorm == 0.0) {
    if (info) { info->iters = 0; info->restarts = 0; info->relres_true = 0.0; }
    return DD_OK;
  }
  CK(cudaMemcpyAsync(h->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  for (;;) {
    TRY(norm_sq(h, h->r, 0, s));
    CK(launch_init_g(h->g, R, h->nsq, s));
    CK(launch_copy_scaled(n, h->r, h->nsq, h->V, s));
    int jlast = -1, launched = -1;
    for (int j = 0; j < R; ++j) {
      // Step j + 1 is launched before the host reads step j's residual
      // estimate, so the GPU never waits for the host between steps.  When
      // step j ends the cycle, the extra step has only written column j + 1
      // of H, g[j + 1] and V_{j+2}, none of which the update of x or the next
      // cycle reads: the iterates are those of stepping one at a time.
      if (launched < j) {
        TRY(run_step(h, j, R, sm, h->cgs_blocks, h->nsq + 2, s));
        CK(cudaEventRecord(h->sev[j & 1], s));
        launched = j;
      }
      if (!h->time_kernels && j + 1 < R && iters + 1 < maxit) {
        TRY(run_step(h, j + 1, R, sm, h->cgs_blocks, h->nsq + 2, s));
        CK(cudaEventRecord(h->sev[(j + 1) & 1], s));
        launched = j + 1;
      }
      CK(cudaEventSynchronize(h->sev[j & 1]));
      if (h->time_kernels) {
        float t0 = 0.f, t1 = 0.f;
        CK(cudaEventElapsedTime(&t0, h->kev[0], h->kev[1]));
        CK(cudaEventElapsedTime(&t1, h->kev[1], h->kev[2]));
        h->stats.krylov_steps += 1;
        h->stats.spmv_ms += t0;
        h->stats.cgs2_ms += t1;
        h->stats.cgs2_fma += (4.0 * (j + 1) + 2.0) * (double)n;
      }
      ++iters;
      const double est = h->h_out[4 * (j & 1) + 2];
      const bool breakdown = h->h_out[4 * (j & 1) + 1] != 0.0;
      if (info && info->history && iters - 1 < info->history_cap) info->history[iters - 1] = est;
      jlast = j;
      if (!isfinite(est)) {
        // a sweep that gave up leaves z unwritten: report that first
        const dd_status ds = device_status(h, s, true);
        rc = ds != DD_OK ? ds : DD_ERR_NONFINITE;
        goto done;
      }
      if (est <= tol || breakdown || iters >= maxit) break;
    }
    CK(launch_hess_solve_update(n, jlast, R, h->H, h->g, h->y, h->Z, h->ldv, x, s));
    CK(launch_residual(h->sell, x, b, h->r, s));
    TRY(norm_sq(h, h->r, 3, s));
    TRY(read_scalars(h, h->nsq + 3, 1, s));
    {
      const dd_status ds = device_status(h, s, true);
      if (ds != DD_OK) { rc = ds; break; }
    }
    relres = sqrt(h->h_out[0]) / bnorm;
    if (!isfinite(relres)) { rc = DD_ERR_NONFINITE; break; }
    if (relres <= tol) { rc = DD_OK; break; }
    if (iters >= maxit) { rc = DD_ERR_NOT_CONVERGED; break; }
    ++restarts;
  }
done:
  if (info) { info->iters = iters; info->restarts = restarts; info->relres_true = relres; }
  return rc;
}

// Independent FGMRES solves of every system of a batched handle, in lock
// step: each Arnoldi step is one set of launches over all systems still
// stepping.  A system leaves the cycle when its own test says so and the
// others go on; cycles end together, then every system that stepped forms
// its x and is tested on its true residual.  Each system so takes exactly
// the steps a solve of it alone would take.
dd_status fgmres_batched(DDHandle *h, const double *const *b, double *const *x, double tol, int R,
                         int maxit, dd_info *infos, cudaStream_t s) {
  const int S = h->nseg, nc = h->seg_ctas;
  const int64_t n = h->n;
  const SegMap sm = batch_map(h);
  const SegMap stm = step_map(h);  // the CGS2 kernel's CTAs on the systems still stepping
  // the apply skips the subdomains and aggregates of systems not stepping
  struct Mask {
    DDHandle *h;
    explicit Mask(DDHandle *hh) : h(hh) { h->masked = true; }
    ~Mask() { h->masked = false; }
  } mask(h);
  SegMap all = sm;
  all.act = nullptr;
  CK(cudaMemsetAsync(h->st, 0, sizeof(DevStatus), s));  // this solve's own status
  for (int q = 0; q < S; ++q) {
    const int64_t r0 = h->seg_row0_h[q], ns = h->seg_row0_h[q + 1] - r0;
    if (ns > 0)
      CK(cudaMemcpyAsync(h->bcat + r0, b[q], sizeof(double) * ns, cudaMemcpyDeviceToDevice, s));
  }
  CK(launch_zero(h->xcat, n, s));
  CK(launch_seg_norms(n, h->bcat, h->partial, h->bn2, all, nc, s));
  CK(cudaMemcpyAsync(h->h_out, h->bn2, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> bnorm(S), relres(S, 0.0);
  std::vector<int> iters(S, 0), restarts(S, 0), done(S, 0);
  std::vector<dd_status> st(S, DD_ERR_NOT_CONVERGED);
  int32_t *act = h->h_act, *jl = h->h_act + S;
  for (int q = 0; q < S; ++q) {
    bnorm[q] = sqrt(h->h_out[q]);
    if (!isfinite(bnorm[q])) { st[q] = DD_ERR_NONFINITE; done[q] = 1; }
    else if (bnorm[q] == 0.0) { st[q] = DD_OK; done[q] = 1; }
  }
  CK(cudaMemcpyAsync(h->r, h->bcat, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  dd_status rc_dev = DD_OK;
  for (;;) {
    int nact = 0;
    for (int q = 0; q < S; ++q) {
      act[q] = done[q] ? 0 : 1;
      jl[q] = -1;
      nact += act[q];
    }
    if (nact == 0) break;
    CK(cudaMemcpyAsync(h->d_act, act, sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
    TRY(remap_active(h, s));
    CK(launch_seg_norms(n, h->r, h->partial, h->rn2, all, nc, s));
    CK(launch_seg_start(n, h->r, h->rn2, h->V, h->g, sm, nc, s));
    for (int j = 0; j < R && nact > 0; ++j) {
      TRY(run_step(h, j, R, stm, nc, h->bn2, s));
      CK(cudaStreamSynchronize(s));
      bool changed = false;
      for (int q = 0; q < S; ++q) {
        if (!act[q]) continue;
        ++iters[q];
        const double est = h->h_out[4 * q + 2];
        const bool breakdown = h->h_out[4 * q + 1] != 0.0;
        dd_info *inf = infos ? &infos[q] : nullptr;
        if (inf && inf->history && iters[q] - 1 < inf->history_cap) inf->history[iters[q] - 1] = est;
        jl[q] = j;
        if (!isfinite(est)) {
          st[q] = DD_ERR_NONFINITE;
          done[q] = 1;
          jl[q] = -1;  // no update of x from a non-finite cycle
        }
        if (done[q] || est <= tol || breakdown || iters[q] >= maxit) {
          act[q] = 0;
          changed = true;
          --nact;
        }
      }
      // copies from pinned memory read it when they run: wait before the next change
      if (changed && nact > 0) {
        CK(cudaMemcpyAsync(h->d_act, act, sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
        TRY(remap_active(h, s));
      }
    }
    CK(cudaMemcpyAsync(h->d_jl, jl, sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
    CK(launch_seg_hess_update(n, R, h->d_jl, h->H, h->g, h->y, h->Z, h->ldv, h->xcat, all, nc, s));
    CK(launch_residual(h->sell, h->xcat, h->bcat, h->r, s));
    CK(launch_seg_norms(n, h->r, h->partial, h->rn2, all, nc, s));
    CK(cudaMemcpyAsync(h->h_out, h->rn2, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
    rc_dev = device_status(h, s, true);
    if (rc_dev != DD_OK) break;
    for (int q = 0; q < S; ++q) {
      if (done[q] || jl[q] < 0) continue;
      relres[q] = sqrt(h->h_out[q]) / bnorm[q];
      if (!isfinite(relres[q])) { st[q] = DD_ERR_NONFINITE; done[q] = 1; }
      else if (relres[q] <= tol) { st[q] = DD_OK; done[q] = 1; }
      else if (iters[q] >= maxit) { st[q] = DD_ERR_NOT_CONVERGED; done[q] = 1; }
      else ++restarts[q];
    }
  }
  for (int q = 0; q < S; ++q) {
    const int64_t r0 = h->seg_row0_h[q], ns = h->seg_row0_h[q + 1] - r0;
    if (ns > 0) CK(cudaMemcpyAsync(x[q], h->xcat + r0, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s));
    if (infos) {
      infos[q].iters = iters[q];
      infos[q].restarts = restarts[q];
      infos[q].relres_true = relres[q];
      infos[q].status = rc_dev != DD_OK ? rc_dev : st[q];
    }
  }
  if (rc_dev != DD_OK) return rc_dev;
  dd_status rc = DD_OK;
  for (int q = 0; q < S; ++q)
    if (st[q] != DD_OK && rc == DD_OK) rc = st[q];
  return rc;
}

void release(DDHandle *h) {
  drop_graphs(h);
  if (h->ustream) { cudaStreamSynchronize(h->ustream); cudaStreamDestroy(h->ustream); h->ustream = nullptr; }
  if (h->uev) { cudaEventDestroy(h->uev); h->uev = nullptr; }
  h->astream = nullptr;
  if (h->gstream) { cudaStreamSynchronize(h->gstream); cudaStreamDestroy(h->gstream); h->gstream = nullptr; }
  for (cudaEvent_t &e : h->gev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
  for (cudaEvent_t &e : h->kev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
  for (cudaEvent_t &e : h->sev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
  for (void *p : h->allocs) cudaFreeAsync(p, h->stream);
  h->allocs.clear();
  cudaStreamSynchronize(h->stream);
  if (h->h_out) cudaFreeHost(h->h_out);
  h->h_out = nullptr;
  if (h->h_act) cudaFreeHost(h->h_act);
  h->h_act = nullptr;
}

// ---------------------------------------------------------------------------
// Scratch of dd_apply_noalloc: one file-scope device array (8 MiB), shared
// by every call.  Host code only ever sees its symbol; the device address is
// looked up once per device with that device current.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_scratch[DD_NOALLOC_MAX_ELEMS];

#define DD_NOALLOC_DEVICES 64
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[DD_NOALLOC_DEVICES] = {nullptr};

// device address of the scratch array on the current device, or nullptr
cudaError_t noalloc_scratch(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= DD_NOALLOC_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// the three kernels of the apply with z1, z2 in the given scratch
template <typename T>
dd_status apply_scratch_T(DDHandle *h, const double *y, double *x, double *scratch, cudaStream_t s) {
  PrecBufs<T> &B = bufs<T>(h);
  T *z1 = reinterpret_cast<T *>(scratch);
  // z2 after z1, on a 256-byte boundary
  const size_t z1_elems = (((size_t)std::max(h->nI, 1) * sizeof(T) + 255) / 256) * 256 / sizeof(T);
  const size_t z2_elems = (((size_t)std::max(h->nG, 1) * sizeof(T) + 255) / 256) * 256 / sizeof(T);
  T *z2 = z1 + z1_elems;
  SweepPlan pl = h->plan;
  pl.first_wait = h->first_wait;
  CK(launch_band_solve_fwd<T>(h->d_info, h->m, h->max_n, h->max_kl, h->max_ku2, pl,
                              h->tm, h->jobs, B.ltile, B.utile, h->src, y, h->d_perm, z1, h->st, s));
  CK(launch_schur_apply<T>(h->nagg, h->agg_off, h->s_off, h->pmax, B.S, h->f_ptr, h->f_col,
                           B.f_val, y, h->d_perm + h->nI, z1, z2, z2 + z2_elems, h->nG, x, nullptr,
                           nullptr, s));
  CK(launch_band_solve_bwd<T>(h->d_info, h->m, h->max_n, h->max_kl, h->max_ku2, pl,
                              h->tm, h->jobs, B.ltile, B.utile, h->src, h->e_ptr, h->e_col, B.e_val,
                              z2, z1, h->d_perm, x, h->st, s));
  return DD_OK;
}

// Autotuner of the apply's sweep kernels: each candidate ring-stage size
// (which fixes the stages, the CTAs per SM and so the persistent schedule)
// is timed on the handle's own factors, forward plus backward sweep, best
// of three after a warm-up; the fastest stays.  y and x are scratch vectors.
template <typename T>
dd_status autotune_sweeps(DDHandle *h, double *y, double *x) {
  PrecBufs<T> &B = bufs<T>(h);
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(y, 0, sizeof(double) * h->n, s));
  CK(cudaMemsetAsync(B.z2, 0, sizeof(T) * std::max(h->nG, 1), s));
  std::vector<size_t> cand;
  const size_t base = (h->max_tile + 127) & ~(size_t)127;
  for (size_t kb : {24, 32, 48, 64, 84, 112, 144}) cand.push_back(std::max(base, kb * 1024));
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  size_t best = 0;
  int best_cl = 1;
  float best_ms = 1e30f;
  int tried = 0;
  for (int mode = 1; mode <= 3; ++mode)
  for (size_t st : cand) {
    if (h->sweep_cl_opt && mode != h->sweep_cl_opt) continue;
    const int cl = mode == 1 ? 1 : 2, la = mode == 3 ? 1 : 0;
    if (la && st < la_max_unit<T>(h)) continue;
    if (band_sweep_stages(h->max_n, h->max_kl, h->max_ku2, h->tb, cl, sizeof(T), (uint32_t)st) < 2) continue;
    if (band_sweep_slots<T>(h->max_n, h->max_kl, h->max_ku2, h->tb, cl, (uint32_t)st, la) <= 0) continue;
    dd_status rc = set_sweep_plan<T>(h, st, mode);
    if (rc != DD_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    float tmin = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, s);
      TRY(apply_T<T>(h, y, x, s, 0));
      TRY(apply_T<T>(h, y, x, s, 2));
      cudaEventRecord(e1, s);
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = std::min(tmin, ms);
    }
    ++tried;
    if (tmin < best_ms) { best_ms = tmin; best = st; best_cl = mode; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tried == 0) { h->err = "autotune: no stage size fits"; return DD_ERR_INVALID_ARG; }
  TRY(set_sweep_plan<T>(h, best, best_cl));
  h->stats.tuned = tried;
  h->stats.tuned_us = 1000.0 * best_ms;
  return DD_OK;
}

// Validation, extraction and device setup of a new handle (stream, nseg and
// seg_row0_h already set); times itself with events on the handle's stream.
dd_status setup_handle(DDHandle *h, const dd_csr *csr, const dd_partition *partition, dd_approx approx,
                       const dd_opts *opts) {
  if ((int)approx < DD_EXACT || (int)approx > DD_MSCE) { h->err = "unknown approximation"; return DD_ERR_INVALID_ARG; }
  dd_opts o{};
  o.prec = DD_FP64;
  if (opts) o = *opts;
  if (approx == DD_LEARNED) {
    if (!o.mlp_weights) { h->err = "DD_LEARNED needs opts.mlp_weights"; return DD_ERR_INVALID_ARG; }
    h->mlp_path = o.mlp_weights;
  }
  if (o.prec != DD_FP64 && o.prec != DD_FP32 && o.prec != DD_FP32_TF32) {
    h->err = "unknown precision";
    return DD_ERR_INVALID_ARG;
  }
  // DD_FP32_TF32 is the FP32 preconditioner with its dense block inverses'
  // rank-64 updates on the TF32 tensor cores
  h->gj_tc = o.prec == DD_FP32_TF32 ? 1 : 0;
  h->prec = o.prec == DD_FP32_TF32 ? DD_FP32 : o.prec;
  h->kind = approx;
  h->use_graph = o.use_graph != 0;
  if (o.krylov_threads != 0 && o.krylov_threads != 256 && o.krylov_threads != 512) {
    h->err = "krylov_threads must be 0, 256 or 512";
    return DD_ERR_INVALID_ARG;
  }
  // default: one 512-thread CTA per SM (fewer CTAs per grid barrier; measured
  // 80.5 us per CGS2 step on the 256x256 workload against 83.9 with two
  // 256-thread CTAs per SM)
  h->krylov_threads = o.krylov_threads > 0 ? o.krylov_threads : 512;
  h->krylov_per_sm = o.krylov_ctas_per_sm > 0 ? o.krylov_ctas_per_sm : (h->krylov_threads == 512 ? 1 : 2);
  h->time_kernels = o.time_kernels != 0 && !h->use_graph;
  if (o.sweep_cluster < 0 || o.sweep_cluster > 3) { h->err = "sweep_cluster must be 0, 1, 2 or 3"; return DD_ERR_INVALID_ARG; }
  h->sweep_cl_opt = o.sweep_cluster;
  h->sweep_pf_opt = o.sweep_prefetch;
  if (!(o.ilu_tol >= 0.0) || !std::isfinite(o.ilu_tol)) { h->err = "ilu_tol must be finite and >= 0"; return DD_ERR_INVALID_ARG; }
  h->ilu_tol = o.ilu_tol;
  if (o.overlap < 0 || o.radius < 0) { h->err = "overlap and radius must be >= 0"; return DD_ERR_INVALID_ARG; }
  h->overlap = o.overlap;
  h->radius = o.radius;
  const double pivtol = o.pivot_tol > 0 ? o.pivot_tol : (h->prec == DD_FP32 ? 1e-7 : 1e-14);
  const int R = o.max_restart > 0 ? o.max_restart : 50;
  if (R > 120) { h->err = "max_restart must be <= 120"; return DD_ERR_INVALID_ARG; }
  HostBlocks hb;
  dd_status rc = validate_and_order(h, csr, partition, hb);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == DD_OK) {
    h->n = csr->n;
    h->nnz = csr->nnz;
    h->m = partition->m;
    h->nI = hb.off[h->m];
    h->nG = (int)(h->n - h->nI);
    rc = build_aggregates(h, partition, approx, hb);
  }
  if (rc == DD_OK) {
    extract_blocks(h, csr, partition, hb);
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      h->err = "cudaEventCreate failed";
      rc = DD_ERR_CUDA;
    }
  }
  if (rc == DD_OK) {
    cudaEventRecord(e0, h->stream);
    rc = dalloc(h, &h->st, 1);
    if (rc == DD_OK && cudaMemsetAsync(h->st, 0, sizeof(DevStatus), h->stream) != cudaSuccess) rc = DD_ERR_CUDA;
    if (rc == DD_OK) rc = (h->prec == DD_FP32) ? setup_device<float>(h, csr, partition, hb, pivtol)
                                               : setup_device<double>(h, csr, partition, hb, pivtol);
    if (rc == DD_OK) rc = alloc_krylov(h, R);
    if (rc == DD_OK && o.autotune)
      rc = (h->prec == DD_FP32) ? autotune_sweeps<float>(h, h->V, h->V + h->ldv)
                                : autotune_sweeps<double>(h, h->V, h->V + h->ldv);
    if (rc == DD_OK && h->use_graph) {
      if (cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->gev[0], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->gev[1], cudaEventDisableTiming) != cudaSuccess) {
        h->err = "graph stream or event creation failed";
        rc = DD_ERR_CUDA;
      }
    }
    for (cudaEvent_t &e : h->sev)
      if (rc == DD_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        h->err = "event creation failed";
        rc = DD_ERR_CUDA;
      }
    if (rc == DD_OK && h->time_kernels)
      for (cudaEvent_t &e : h->kev)
        if (cudaEventCreate(&e) != cudaSuccess) { h->err = "event creation failed"; rc = DD_ERR_CUDA; break; }
    cudaEventRecord(e1, h->stream);
    cudaError_t se = cudaStreamSynchronize(h->stream);
    if (rc == DD_OK && se != cudaSuccess) { h->err = cudaGetErrorString(se); rc = DD_ERR_CUDA; }
    if (rc == DD_OK) {
      DevStatus st{};
      if (cudaMemcpy(&st, h->st, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) { rc = DD_ERR_CUDA; }
      else if (st.code != 0) {
        rc = (dd_status)st.code;
        h->bad_block = st.block;
        char buf[128];
        snprintf(buf, sizeof buf, "%s in block %d",
                 st.code == DD_ERR_SINGULAR_BLOCK ? "singular interior block" : "singular Schur block", st.block);
        h->err = buf;
      }
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->stats.setup_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->stats.n = h->n;
  h->stats.n_interior = h->nI;
  h->stats.n_interface = h->nG;
  h->stats.nnz = h->nnz;
  h->stats.m = h->m;
  h->stats.batch = h->nseg;
  return rc;
}

// hands the handle out (also on SINGULAR_*, for dd_get_bad_block) or frees it
dd_status finish_setup(DDHandle *h, dd_status rc, void **handle) {
  g_setup_error = h->err;
  if (rc == DD_OK || rc == DD_ERR_SINGULAR_BLOCK || rc == DD_ERR_SINGULAR_SCHUR) {
    *handle = h;
    return rc;
  }
  release(h);
  delete h;
  return rc;
}

// The batch as one block-diagonal system: rows of system q follow those of
// q-1; interiors renumbered after the previous systems' subdomains, the
// interface of every system after all interiors, aggregates per system.
struct BatchInput {
  std::vector<int32_t> rowptr, col, partv, perm, agg, sub_sys, agg_sys;
  std::vector<double> val;
  std::vector<int64_t> row0;
  dd_csr csr{};
  dd_partition pt{};
};

dd_status concat_batch(int count, const dd_csr *csrs, const dd_partition *pts, dd_approx approx, BatchInput &bi) {
  int64_t N = 0, NNZ = 0;
  bi.row0.assign(count + 1, 0);
  for (int q = 0; q < count; ++q) {
    const dd_csr &c = csrs[q];
    if (c.n <= 0 || !c.rowptr || !c.col || !c.val || !pts[q].part || pts[q].m <= 0) {
      g_setup_error = "batch member " + std::to_string(q) + ": invalid CSR or partition";
      return DD_ERR_INVALID_ARG;
    }
    N += c.n;
    NNZ += c.nnz;
    bi.row0[q + 1] = N;
  }
  if (N > INT32_MAX - 1 || NNZ > INT32_MAX) { g_setup_error = "batch too large for 32-bit indices"; return DD_ERR_INVALID_ARG; }
  bi.rowptr.assign(N + 1, 0);
  bi.col.resize(NNZ);
  bi.val.resize(NNZ);
  bi.partv.resize(N);
  std::vector<int32_t> inter, iface;  // concatenated interior order, then interface order
  std::vector<int32_t> gsz;           // interface size per system
  int64_t k = 0;
  int32_t moff = 0;
  for (int q = 0; q < count; ++q) {
    const dd_csr &c = csrs[q];
    const dd_partition &p = pts[q];
    const int64_t r0 = bi.row0[q];
    if (c.rowptr[0] != 0 || c.rowptr[c.n] != c.nnz) {
      g_setup_error = "batch member " + std::to_string(q) + ": rowptr[0] must be 0 and rowptr[n] == nnz";
      return DD_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < c.n; ++i) {
      for (int64_t e = c.rowptr[i]; e < c.rowptr[i + 1]; ++e) {
        const int32_t cc = c.col[e];
        bi.col[k] = (cc >= 0 && cc < c.n) ? (int32_t)(cc + r0) : -1;  // -1 fails validation
        bi.val[k++] = c.val[e];
      }
      bi.rowptr[r0 + i + 1] = (int32_t)k;
      const int32_t pv = p.part[i];
      bi.partv[r0 + i] = (pv >= 0 && pv < p.m) ? pv + moff : (pv == -1 ? -1 : INT32_MIN);
    }
    // this system's order: its perm, or interiors by subdomain then interface, ascending
    std::vector<int32_t> order;
    int64_t nI = 0;
    for (int64_t i = 0; i < c.n; ++i) nI += (p.part[i] >= 0);
    if (p.perm) {
      order.assign(p.perm, p.perm + c.n);
    } else {
      std::vector<int32_t> cnt(p.m + 1, 0);
      for (int64_t i = 0; i < c.n; ++i) if (p.part[i] >= 0 && p.part[i] < p.m) cnt[p.part[i] + 1]++;
      for (int j = 0; j < p.m; ++j) cnt[j + 1] += cnt[j];
      order.assign(c.n, 0);
      int64_t g = nI;
      for (int64_t i = 0; i < c.n; ++i) {
        if (p.part[i] >= 0 && p.part[i] < p.m) order[cnt[p.part[i]]++] = (int32_t)i;
        else if (g < c.n) order[g++] = (int32_t)i;
      }
    }
    for (int64_t i = 0; i < c.n; ++i) {
      const int32_t o = order[i];
      if (o < 0 || o >= c.n) { g_setup_error = "batch member " + std::to_string(q) + ": perm out of range"; return DD_ERR_INVALID_PARTITION; }
      (i < nI ? inter : iface).push_back((int32_t)(o + r0));
    }
    // aggregates of this system in its own interface numbering
    const int32_t nG = (int32_t)(c.n - nI);
    gsz.push_back(nG);
    const int32_t g0 = bi.agg.empty() ? 0 : bi.agg.back();
    if (bi.agg.empty()) bi.agg.push_back(0);
    if (nG > 0) {
      if (approx == DD_EXACT) {
        bi.agg.push_back(g0 + nG);
      } else if (p.agg_offsets) {
        if (p.n_agg <= 0 || p.agg_offsets[0] != 0 || p.agg_offsets[p.n_agg] != nG) {
          g_setup_error = "batch member " + std::to_string(q) + ": aggregate offsets must run from 0 to n_G";
          return DD_ERR_INVALID_ARG;
        }
        for (int a = 1; a <= p.n_agg; ++a) bi.agg.push_back(g0 + p.agg_offsets[a]);
      } else {
        if (p.sz <= 0) { g_setup_error = "aggregate size sz must be positive"; return DD_ERR_INVALID_ARG; }
        for (int32_t a = p.sz; a < nG; a += p.sz) bi.agg.push_back(g0 + a);
        bi.agg.push_back(g0 + nG);
      }
    }
    moff += p.m;
    for (int j = 0; j < p.m; ++j) bi.sub_sys.push_back(q);
    while ((int)bi.agg_sys.size() < (int)bi.agg.size() - 1) bi.agg_sys.push_back(q);
  }
  bi.perm = inter;
  bi.perm.insert(bi.perm.end(), iface.begin(), iface.end());
  bi.csr.n = N;
  bi.csr.nnz = NNZ;
  bi.csr.rowptr = bi.rowptr.data();
  bi.csr.col = bi.col.data();
  bi.csr.val = bi.val.data();
  bi.pt.m = moff;
  bi.pt.part = bi.partv.data();
  bi.pt.perm = bi.perm.data();
  bi.pt.sz = 0;
  bi.pt.agg_offsets = bi.agg.data();
  bi.pt.n_agg = (int32_t)bi.agg.size() - 1;
  return DD_OK;
}

// Runs a solve on the caller's stream, or, with graphs, on the handle's
// capture stream ordered after and before the caller's work.
template <typename F>
dd_status timed_solve(DDHandle *h, cudaStream_t s, F &&solve, float &ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  dd_status rc;
  if (h->use_graph) {
    cudaEventRecord(h->gev[0], s);
    cudaStreamWaitEvent(h->gstream, h->gev[0], 0);
    rc = solve(h->gstream);
    cudaEventRecord(h->gev[1], h->gstream);
    cudaStreamWaitEvent(s, h->gev[1], 0);
  } else {
    rc = solve(s);
  }
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" {

dd_status dd_apply_noalloc(void *handle, const double *y, double *x, void *stream) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !y || !x) return DD_ERR_INVALID_ARG;
  if (h->bad_block >= 0) { h->err = "preconditioner failed in setup"; return DD_ERR_INVALID_ARG; }
  // z1 and z2, each rounded up to 256 bytes, must fit the scratch array
  const size_t es = h->prec == DD_FP32 ? sizeof(float) : sizeof(double);
  const size_t need = ((size_t)std::max(h->nI, 1) * es + 255) / 256 * 256 +
                      2 * (((size_t)std::max(h->nG, 1) * es + 255) / 256 * 256);
  if (h->n > DD_NOALLOC_MAX_ELEMS || need > sizeof(double) * (size_t)DD_NOALLOC_MAX_ELEMS) {
    char buf[160];
    snprintf(buf, sizeof buf, "dd_apply_noalloc: n = %lld exceeds the scratch limit of %d elements",
             (long long)h->n, DD_NOALLOC_MAX_ELEMS);
    h->err = buf;
    return DD_ERR_INVALID_ARG;
  }
  double *scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) {
    h->err = std::string("dd_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return DD_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return h->prec == DD_FP32 ? apply_scratch_T<float>(h, y, x, scratch, s)
                            : apply_scratch_T<double>(h, y, x, scratch, s);
}


dd_status dd_setup(const dd_csr *csr, const dd_partition *partition, dd_approx approx,
                   const dd_opts *opts, void *stream, void **handle) {
  if (!handle) return DD_ERR_INVALID_ARG;
  *handle = nullptr;
  g_setup_error.clear();
  if (!csr || !partition) { g_setup_error = "csr and partition are required"; return DD_ERR_INVALID_ARG; }
  DDHandle *h = new (std::nothrow) DDHandle();
  if (!h) return DD_ERR_OOM;
  h->stream = static_cast<cudaStream_t>(stream);
  h->nseg = 1;
  h->seg_row0_h = {0, csr->n};
  const dd_status rc = setup_handle(h, csr, partition, approx, opts);
  return finish_setup(h, rc, handle);
}

dd_status dd_setup_batched(int32_t count, const dd_csr *csrs, const dd_partition *partitions,
                           dd_approx approx, const dd_opts *opts, void *stream, void **handle) {
  if (!handle) return DD_ERR_INVALID_ARG;
  *handle = nullptr;
  g_setup_error.clear();
  if (count <= 0 || !csrs || !partitions) { g_setup_error = "count >= 1, csrs and partitions are required"; return DD_ERR_INVALID_ARG; }
  if (approx == DD_MSCN || approx == DD_MSCNR || approx == DD_OMSCN || approx == DD_OMSCNR) {
    g_setup_error = "MSCN and MSCNR pair interface and interior index ranges of one system; not available in a batch";
    return DD_ERR_INVALID_ARG;
  }
  if (approx == DD_OLUM) {
    g_setup_error = "overlapped blocks would join the systems of a batch; not available in a batch";
    return DD_ERR_INVALID_ARG;
  }
  BatchInput bi;
  const dd_status rc0 = concat_batch(count, csrs, partitions, approx, bi);
  if (rc0 != DD_OK) return rc0;
  DDHandle *h = new (std::nothrow) DDHandle();
  if (!h) return DD_ERR_OOM;
  h->stream = static_cast<cudaStream_t>(stream);
  h->nseg = count;
  h->seg_row0_h = bi.row0;
  h->sub_sys_h = bi.sub_sys;
  h->agg_sys_h = bi.agg_sys;
  const dd_status rc = setup_handle(h, &bi.csr, &bi.pt, approx, opts);
  return finish_setup(h, rc, handle);
}

dd_status dd_apply(void *handle, const double *y, double *x, void *stream) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !y || !x) return DD_ERR_INVALID_ARG;
  if (h->bad_block >= 0) { h->err = "preconditioner failed in setup"; return DD_ERR_INVALID_ARG; }
  return apply_any(h, y, x, static_cast<cudaStream_t>(stream));
}

dd_status dd_apply_part(void *handle, int32_t part, const double *y, double *x, void *stream) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !y || !x || part < 0 || part > 2) return DD_ERR_INVALID_ARG;
  if (h->bad_block >= 0) { h->err = "preconditioner failed in setup"; return DD_ERR_INVALID_ARG; }
  return apply_any(h, y, x, static_cast<cudaStream_t>(stream), part);
}

dd_status gmres_solve(void *handle, const double *b, double *x, double tol, int32_t restart,
                      int32_t maxit, dd_info *info, void *stream) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !b || !x || restart <= 0 || restart > h->Rmax || maxit <= 0 || !(tol > 0)) {
    if (h) h->err = "invalid gmres_solve arguments (restart must be <= max_restart of dd_setup)";
    return DD_ERR_INVALID_ARG;
  }
  if (h->bad_block >= 0) { h->err = "preconditioner failed in setup"; return DD_ERR_INVALID_ARG; }
  float ms = 0.f;
  const dd_status rc = timed_solve(
      h, static_cast<cudaStream_t>(stream),
      [&](cudaStream_t s2) { return fgmres(h, b, x, tol, restart, maxit, info, s2); }, ms);
  if (info) {
    info->solve_ms = ms;
    info->setup_ms = h->stats.setup_ms;
    info->bad_block = h->bad_block;
    info->status = rc;
  }
  return rc;
}

dd_status gmres_solve_batched(void *handle, const double *const *b, double *const *x, double tol,
                              int32_t restart, int32_t maxit, dd_info *infos, void *stream) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !b || !x || restart <= 0 || restart > h->Rmax || maxit <= 0 || !(tol > 0)) {
    if (h) h->err = "invalid gmres_solve_batched arguments (restart must be <= max_restart of dd_setup)";
    return DD_ERR_INVALID_ARG;
  }
  if (h->nseg < 2) { h->err = "gmres_solve_batched needs a handle from dd_setup_batched with >= 2 systems"; return DD_ERR_INVALID_ARG; }
  for (int q = 0; q < h->nseg; ++q)
    if (!b[q] || !x[q]) { h->err = "null right-hand side or solution pointer"; return DD_ERR_INVALID_ARG; }
  if (h->bad_block >= 0) { h->err = "preconditioner failed in setup"; return DD_ERR_INVALID_ARG; }
  float ms = 0.f;
  const dd_status rc = timed_solve(
      h, static_cast<cudaStream_t>(stream),
      [&](cudaStream_t s2) { return fgmres_batched(h, b, x, tol, restart, maxit, infos, s2); }, ms);
  if (infos)
    for (int q = 0; q < h->nseg; ++q) {
      infos[q].solve_ms = ms;
      infos[q].setup_ms = h->stats.setup_ms;
      infos[q].bad_block = h->bad_block;
    }
  return rc;
}

dd_status dd_fp64_peak(double *gfma, void *stream) {
  if (!gfma) return DD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DD_ERR_CUDA;
  const int blocks = 8 * sms, iters = 2048;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DD_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return DD_ERR_CUDA; }
  float best = 1e30f;
  dd_status rc = DD_OK;
  for (int rep = 0; rep < 4 && rc == DD_OK; ++rep) {
    cudaEventRecord(e0, s);
    if (launch_fma_probe(blocks, iters, s) != cudaSuccess) rc = DD_ERR_CUDA;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = DD_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms > 0.f) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DD_OK) return rc;
  *gfma = (double)blocks * 256.0 * 8.0 * iters / (best * 1e-3) / 1e9;
  return DD_OK;
}

dd_status dd_check_status(void *handle, void *stream) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h) return DD_ERR_INVALID_ARG;
  return device_status(h, static_cast<cudaStream_t>(stream), true);
}

dd_status dd_set_wait_limit(void *handle, uint32_t first_wait_polls) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h) return DD_ERR_INVALID_ARG;
  h->first_wait = first_wait_polls;
  drop_graphs(h);  // captured steps hold the old kernel arguments
  return DD_OK;
}

dd_status dd_spmv(void *handle, const double *x, double *y, void *stream) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !x || !y) return DD_ERR_INVALID_ARG;
  cudaError_t e = launch_spmv(h->sell, x, y, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) { h->err = cudaGetErrorString(e); return DD_ERR_CUDA; }
  return DD_OK;
}

dd_status dd_learned_entries(void *handle, int32_t *ents, double *feats, float *delta, int64_t cap,
                             int64_t *count) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !count || cap < 0) return DD_ERR_INVALID_ARG;
  if (h->kind != DD_LEARNED) { h->err = "not a DD_LEARNED handle"; return DD_ERR_INVALID_ARG; }
  const int64_t ne = (int64_t)h->l_ents.size() / 3;
  *count = ne;
  const int64_t k = std::min(ne, cap);
  if (k <= 0) return DD_OK;
  if (ents) memcpy(ents, h->l_ents.data(), sizeof(int32_t) * 3 * (size_t)k);
  if (feats && cudaMemcpy(feats, h->l_feat, sizeof(double) * DD_MLP_IN * (size_t)k, cudaMemcpyDeviceToHost) != cudaSuccess)
    return DD_ERR_CUDA;
  if (delta && cudaMemcpy(delta, h->l_delta, sizeof(float) * (size_t)k, cudaMemcpyDeviceToHost) != cudaSuccess)
    return DD_ERR_CUDA;
  return DD_OK;
}

dd_status dd_get_stats(void *handle, dd_stats *stats) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !stats) return DD_ERR_INVALID_ARG;
  *stats = h->stats;
  return DD_OK;
}

int32_t dd_get_bad_block(void *handle) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  return h ? h->bad_block : -1;
}

dd_status dd_destroy(void *handle) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h) return DD_ERR_INVALID_ARG;
  release(h);
  delete h;
  return DD_OK;
}

const char *dd_last_error(void *handle) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  return h ? h->err.c_str() : g_setup_error.c_str();
}

}  // extern "C"
