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
#include <mutex>
#include <string>
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
  int max_n = 0, max_kl = 0, max_ku = 0, max_ku2 = 0, max_tiles = 0, sweep_threads = 256;
  uint32_t stage_bytes = 0;
  void *lu_scratch = nullptr;  // windows of the blocked LU (when not in shared memory)
  TileMeta *tm = nullptr;      // packed sweep tiles
  SweepJob *jobs = nullptr;    // jobs of the sweep ring
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  BandInfo *d_info = nullptr;
  int32_t *piv = nullptr, *src = nullptr;
  int32_t *d_perm = nullptr;
  int32_t *e_ptr = nullptr, *e_col = nullptr, *f_ptr = nullptr, *f_col = nullptr;
  int32_t *agg_off = nullptr, *d_p = nullptr, *ipiv = nullptr, *failed = nullptr;
  int64_t *s_off = nullptr, *poff = nullptr;
  int32_t *c_rowptr = nullptr, *c_col = nullptr;
  double *c_val = nullptr;
  DevStatus *st = nullptr;
  PrecBufs<double> pd;
  PrecBufs<float> pf;
  // FGMRES workspace
  int Rmax = 0, nblocks = 304, cgs_blocks = 0;
  int64_t ldv = 0;
  double *V = nullptr, *Z = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr,
         *y = nullptr, *hc1 = nullptr, *hc2 = nullptr, *nsq = nullptr, *out = nullptr,
         *partial = nullptr, *r = nullptr;
  double *h_out = nullptr;  // pinned host scalars
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
  cudaError_t e = cudaMallocAsync(&q, count * sizeof(P), h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DD_ERR_OOM : DD_ERR_CUDA;
  }
  h->allocs.push_back(q);
  *p = static_cast<P *>(q);
  return DD_OK;
}

template <typename P>
dd_status upload(DDHandle *h, P **p, const std::vector<P> &v) {
  dd_status s = dalloc(h, p, v.size());
  if (s != DD_OK) return s;
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(P), cudaMemcpyHostToDevice, h->stream));
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
    convert_kernel<T><<<(unsigned)((v.size() + 255) / 256), 256, 0, h->stream>>>((int64_t)v.size(), tmp, *p);
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
  for (int64_t i = 0; i < n; ++i) {
    if (csr->rowptr[i + 1] < csr->rowptr[i]) { h->err = "rowptr decreases"; return DD_ERR_INVALID_ARG; }
    for (int64_t k = csr->rowptr[i]; k < csr->rowptr[i + 1]; ++k) {
      if (csr->col[k] < 0 || csr->col[k] >= n) { h->err = "column index out of range"; return DD_ERR_INVALID_ARG; }
      if (!isfinite(csr->val[k])) { h->err = "non-finite matrix entry"; return DD_ERR_NONFINITE; }
    }
  }
  const int m = pt->m;
  if (m <= 0 || !pt->part) { h->err = "partition needs m >= 1 and part"; return DD_ERR_INVALID_ARG; }
  for (int64_t i = 0; i < n; ++i)
    if (pt->part[i] < -1 || pt->part[i] >= m) { h->err = "part value out of range"; return DD_ERR_INVALID_PARTITION; }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = csr->rowptr[i]; k < csr->rowptr[i + 1]; ++k) {
      int a = pt->part[i], b = pt->part[csr->col[k]];
      if (a >= 0 && b >= 0 && a != b && csr->val[k] != 0.0) {
        char buf[160];
        snprintf(buf, sizeof buf, "entry (%lld,%d) couples interiors %d and %d", (long long)i, csr->col[k], a, b);
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
  if (kind == DD_EXACT) {
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
  if ((kind == DD_MSCN || kind == DD_MSCNR) && hb.agg.back() > h->nI) {
    h->err = "MSCN needs n_interior >= n_interface (same local index ranges)";
    return DD_ERR_INVALID_ARG;
  }
  return DD_OK;
}

void extract_blocks(DDHandle *h, const dd_csr *csr, const dd_partition *pt, HostBlocks &hb) {
  const int m = h->m, nI = h->nI, nG = h->nG;
  hb.kl.assign(m, 0);
  hb.ku.assign(m, 0);
  hb.e_ptr.assign(nI + 1, 0);
  hb.f_ptr.assign(nG + 1, 0);
  // bandwidths and counts
  for (int64_t r = 0; r < h->n; ++r) {
    const int o = hb.perm[r];
    const int jr = pt->part[o];
    for (int64_t k = csr->rowptr[o]; k < csr->rowptr[o + 1]; ++k) {
      const int c = hb.pos[csr->col[k]];
      const int jc = pt->part[csr->col[k]];
      if (jr >= 0 && jc == jr) {
        hb.kl[jr] = std::max(hb.kl[jr], (int)(r - c));
        hb.ku[jr] = std::max(hb.ku[jr], (int)(c - r));
      } else if (jr >= 0 && jc < 0) {
        hb.e_ptr[r + 1]++;
      } else if (jr < 0 && jc >= 0) {
        hb.f_ptr[r - nI + 1]++;
      }
    }
  }
  for (int i = 0; i < nI; ++i) hb.e_ptr[i + 1] += hb.e_ptr[i];
  for (int i = 0; i < nG; ++i) hb.f_ptr[i + 1] += hb.f_ptr[i];
  hb.e_col.assign(hb.e_ptr[nI], 0);
  hb.e_val.assign(hb.e_ptr[nI], 0.0);
  hb.f_col.assign(hb.f_ptr[nG], 0);
  hb.f_val.assign(hb.f_ptr[nG], 0.0);
  std::vector<int32_t> ef(hb.e_ptr.begin(), hb.e_ptr.end() - 1), ff(hb.f_ptr.begin(), hb.f_ptr.end() - 1);
  for (int64_t r = 0; r < h->n; ++r) {
    const int o = hb.perm[r];
    const int jr = pt->part[o];
    for (int64_t k = csr->rowptr[o]; k < csr->rowptr[o + 1]; ++k) {
      const int c = hb.pos[csr->col[k]];
      const int jc = pt->part[csr->col[k]];
      if (jr >= 0 && jc < 0) {
        hb.e_col[ef[r]] = c - nI;
        hb.e_val[ef[r]++] = csr->val[k];
      } else if (jr < 0 && jc >= 0) {
        hb.f_col[ff[r - nI]] = c;
        hb.f_val[ff[r - nI]++] = csr->val[k];
      }
    }
  }
  (void)m;
}

int64_t launch_cost(const char *call, const DDHandle *h) {
  if (strstr(call, "launch_gj_inverse")) return 3LL * ((h->pmax + (h->prec == DD_FP32 ? 15 : 7)) / (h->prec == DD_FP32 ? 16 : 8)) + 1;
  if (strstr(call, "launch_hess_solve_update")) return 2;
  if (strstr(call, "launch_schur_apply")) return 2;
  return 1;
}

}  // namespace

namespace {

template <typename T>
dd_status setup_device(DDHandle *h, const dd_csr *csr, const dd_partition *pt, HostBlocks &hb,
                       double pivtol) {
  PrecBufs<T> &B = bufs<T>(h);
  const int m = h->m, nI = h->nI, nG = h->nG;
  cudaStream_t s = h->stream;
  // ---- interior factors: geometry
  std::vector<BandInfo> info(m);
  int64_t band = 0, lraw = 0, pivo = 0, fac_nz = 0;
  int32_t tiles = 0;
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
    b.tile0 = tiles; tiles += b.ntiles;
    h->max_n = std::max(h->max_n, b.ntiles * DD_NB);
    h->max_kl = std::max(h->max_kl, b.kl);
    h->max_ku = std::max(h->max_ku, b.ku);
    h->max_ku2 = std::max(h->max_ku2, b.kl + b.ku);
    h->max_tiles = std::max(h->max_tiles, b.ntiles);
    // in-band entries of L (kl per column) and U (kl+ku+1 per row), clipped
    for (int i = 0; i < b.n; ++i) fac_nz += std::min(b.kl, b.n - 1 - i) + std::min(b.kl + b.ku, b.n - 1 - i) + 1;
  }
  h->stats.factor_nonzeros = fac_nz;
  h->stats.kl_max = h->max_kl;
  h->stats.ku_max = h->max_ku;
  h->stats.tile = DD_NB;
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
  {
    std::vector<int32_t> rp(csr->rowptr, csr->rowptr + h->n + 1), cc(csr->col, csr->col + h->nnz);
    std::vector<double> vv(csr->val, csr->val + h->nnz);
    TRY(upload(h, &h->c_rowptr, rp));
    TRY(upload(h, &h->c_col, cc));
    TRY(upload(h, &h->c_val, vv));
  }
  int32_t *d_part = nullptr, *d_pos = nullptr;
  TRY(upload(h, &d_part, std::vector<int32_t>(pt->part, pt->part + h->n)));
  TRY(upload(h, &d_pos, hb.pos));
  TRY(upload(h, &h->d_perm, hb.perm));
  h->stats.launches += 1;
  fill_band_kernel<T><<<(unsigned)((h->n + 255) / 256), 256, 0, s>>>(
      (int)h->n, h->c_rowptr, h->c_col, h->c_val, d_part, d_pos, h->d_info, B.band);
  CK(cudaGetLastError());
  CK(launch_band_lu<T>(h->d_info, m, h->max_kl, h->max_ku, B.band, B.lm, h->piv,
                       static_cast<T *>(h->lu_scratch), pivtol, h->st, 256, s));
  // ---- packed sweep tiles: widths from the factors, offsets and jobs here
  {
    int32_t *d_wl = nullptr, *d_wu = nullptr;
    TRY(dalloc(h, &d_wl, tiles));
    TRY(dalloc(h, &d_wu, tiles));
    CK(launch_tile_widths<T>(h->d_info, m, h->max_tiles, B.band, B.lm, h->piv, d_wl, d_wu, s));
    std::vector<int32_t> wl(tiles), wu(tiles);
    if (tiles) {
      CK(cudaMemcpyAsync(wl.data(), d_wl, sizeof(int32_t) * tiles, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(wu.data(), d_wu, sizeof(int32_t) * tiles, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    std::vector<TileMeta> tm(tiles);
    int64_t lofs = 0, uofs = 0, sofs = 0;
    size_t max_tile = 0;
    for (int t = 0; t < tiles; ++t) {
      tm[t].lofs = lofs; tm[t].uofs = uofs; tm[t].sofs = sofs;
      tm[t].wl = wl[t]; tm[t].wu = wu[t];
      lofs += (int64_t)wl[t] * DD_NB;
      uofs += (int64_t)DD_NB * wu[t];
      sofs += round4(wl[t]);
      max_tile = std::max(max_tile, std::max((size_t)wl[t] * DD_NB * sizeof(T) + (size_t)round4(wl[t]) * 4,
                                             (size_t)DD_NB * wu[t] * sizeof(T)));
    }
    // stage: ~84 KiB, or one whole tile when a tile is larger
    size_t stage = std::max<size_t>(84 * 1024, max_tile);
    stage = (stage + 127) & ~(size_t)127;
    h->stage_bytes = (uint32_t)stage;
    std::vector<SweepJob> jobs;
    for (int j = 0; j < m; ++j) {
      BandInfo &b = info[j];
      b.jf0 = (int32_t)jobs.size();
      for (int lo = 0; lo < b.ntiles;) {
        size_t bytes = 0;
        int hi = lo;
        while (hi < b.ntiles) {
          const TileMeta &q = tm[b.tile0 + hi];
          const size_t tb = (size_t)q.wl * DD_NB * sizeof(T) + (size_t)round4(q.wl) * 4;
          if (hi > lo && bytes + tb > stage) break;
          bytes += tb;
          ++hi;
        }
        jobs.push_back(SweepJob{lo, hi});
        lo = hi;
      }
      b.njf = (int32_t)jobs.size() - b.jf0;
      b.jb0 = (int32_t)jobs.size();
      for (int hi = b.ntiles; hi > 0;) {
        size_t bytes = 0;
        int lo = hi;
        while (lo > 0) {
          const TileMeta &q = tm[b.tile0 + lo - 1];
          const size_t tb = (size_t)DD_NB * q.wu * sizeof(T);
          if (lo < hi && bytes + tb > stage) break;
          bytes += tb;
          --lo;
        }
        jobs.push_back(SweepJob{lo, hi});
        hi = lo;
      }
      b.njb = (int32_t)jobs.size() - b.jb0;
    }
    CK(cudaMemcpyAsync(h->d_info, info.data(), sizeof(BandInfo) * m, cudaMemcpyHostToDevice, s));
    TRY(upload(h, &h->tm, tm));
    TRY(upload(h, &h->jobs, jobs));
    TRY(dalloc(h, &B.ltile, lofs));
    TRY(dalloc(h, &B.utile, uofs));
    TRY(dalloc(h, &h->src, sofs));
    h->stats.factor_bytes = (lofs + uofs) * (int64_t)sizeof(T) + sofs * (int64_t)sizeof(int32_t);
    if (band_sweep_stages(h->max_n, h->max_kl, h->max_ku2, h->sweep_threads, sizeof(T), h->stage_bytes) < 2) {
      h->err = "a subdomain is too large for the shared-memory sweep (reduce its size or use FP32)";
      return DD_ERR_INVALID_ARG;
    }
    CK(launch_band_tiles<T>(h->d_info, m, h->max_tiles, h->max_kl, h->tm, B.band, B.lm, h->piv,
                            B.ltile, B.utile, h->src, s));
  }
  // ---- couplings E (interior x interface) and F (interface x interior)
  TRY(upload(h, &h->e_ptr, hb.e_ptr));
  TRY(upload(h, &h->e_col, hb.e_col));
  TRY(upload_T(h, &B.e_val, hb.e_val));
  TRY(upload(h, &h->f_ptr, hb.f_ptr));
  TRY(upload(h, &h->f_col, hb.f_col));
  TRY(upload_T(h, &B.f_val, hb.f_val));
  h->stats.coupling_nnz = (int64_t)hb.e_col.size() + (int64_t)hb.f_col.size();
  // ---- interface blocks
  const int nagg = (int)hb.agg.size() - 1;
  h->nagg = nagg;
  std::vector<int32_t> p(nagg), agg_of(nG);
  std::vector<int64_t> soff(nagg + 1, 0), poff(nagg + 1, 0);
  h->pmax = 0;
  for (int a = 0; a < nagg; ++a) {
    p[a] = hb.agg[a + 1] - hb.agg[a];
    soff[a + 1] = soff[a] + (int64_t)p[a] * p[a];
    poff[a + 1] = poff[a] + p[a];
    h->pmax = std::max(h->pmax, p[a]);
    for (int g = hb.agg[a]; g < hb.agg[a + 1]; ++g) agg_of[g] = a;
  }
  if (h->pmax > 12288) { h->err = "an aggregate exceeds 12288 interface nodes"; return DD_ERR_INVALID_ARG; }
  h->stats.n_agg = nagg;
  h->stats.max_agg = h->pmax;
  h->stats.schur_bytes = soff[nagg] * (int64_t)sizeof(T);
  TRY(upload(h, &h->agg_off, hb.agg));
  TRY(upload(h, &h->d_p, p));
  TRY(upload(h, &h->s_off, soff));
  TRY(upload(h, &h->poff, poff));
  TRY(dalloc(h, &B.S, soff[nagg]));
  CK(cudaMemsetAsync(B.S, 0, sizeof(T) * std::max<int64_t>(soff[nagg], 1), s));
  TRY(dalloc(h, &B.amax, nagg));
  TRY(dalloc(h, &B.gj, gj_scratch_elems(nagg, poff[nagg], sizeof(T))));
  TRY(dalloc(h, &h->ipiv, poff[nagg]));
  TRY(dalloc(h, &h->failed, nagg));
  // G(R_a, R_a) into S
  {
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
    int64_t *d_idx = nullptr;
    double *d_val = nullptr;
    TRY(upload(h, &d_idx, idx));
    TRY(upload(h, &d_val, val));
    CK(launch_scatter_coo<T>((int64_t)idx.size(), d_idx, d_val, B.S, s));
  }
  if (h->kind == DD_MSCE_INF || h->kind == DD_EXACT) {
    // per subdomain: interface columns of E (gam) and interface rows of F (fr)
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
    int max_fr = 0, max_gam = 0;
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
      max_fr = std::max(max_fr, (int)frs[j].size());
      max_gam = std::max(max_gam, (int)cols.size());
    }
    int32_t *d_gam_ptr, *d_gam_idx, *d_gam_agg, *d_fr_ptr, *d_fr_row, *d_fr_agg, *d_fs_ptr, *d_fs_col, *d_ncols;
    int64_t *d_xoff, *d_xidx;
    double *d_xval;
    TRY(upload(h, &d_gam_ptr, gam_ptr));
    TRY(upload(h, &d_gam_idx, gam_idx));
    TRY(upload(h, &d_gam_agg, gam_agg));
    TRY(upload(h, &d_fr_ptr, fr_ptr));
    TRY(upload(h, &d_fr_row, fr_row));
    TRY(upload(h, &d_fr_agg, fr_agg));
    TRY(upload(h, &d_fs_ptr, fs_ptr));
    TRY(upload(h, &d_fs_col, fs_col));
    TRY(upload_T(h, &B.fsub_val, fs_val));
    TRY(upload(h, &d_ncols, ncols));
    TRY(upload(h, &d_xoff, xoff));
    TRY(upload(h, &d_xidx, xidx));
    TRY(upload(h, &d_xval, xval));
    TRY(dalloc(h, &B.X, xoff[m]));
    CK(cudaMemsetAsync(B.X, 0, sizeof(T) * std::max<int64_t>(xoff[m], 1), s));
    CK(launch_scatter_coo<T>((int64_t)xidx.size(), d_xidx, d_xval, B.X, s));
    // X_j = A_jj^-1 E(I_j, gam_j)
    CK(launch_band_solve_multi<T>(h->d_info, m, d_ncols, d_xoff, max_gam, h->max_kl, h->max_ku2,
                                  h->tm, B.ltile, B.utile, h->src, B.X, s));
    // S(R_a,R_a) -= F(R_a, I_j) X_j
    CK(launch_schur_accumulate<T>(m, d_fr_ptr, d_fr_row, d_fr_agg, d_fs_ptr, d_fs_col, B.fsub_val,
                                  d_gam_ptr, d_gam_idx, d_gam_agg, d_xoff, h->d_info, B.X,
                                  h->agg_off, h->s_off, B.S, max_fr, max_gam, s));
  } else if (h->kind == DD_MSCN || h->kind == DD_MSCNR) {
    // principal blocks with the same local index range (Algorithm 1)
    std::vector<int64_t> di, ei, fi;
    std::vector<double> dv, ev, fv;
    for (int a = 0; a < nagg; ++a) {
      const int g0 = hb.agg[a], g1 = hb.agg[a + 1], pa = p[a];
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
        // F_ii D_ii^-1 E_ii vanishes: D_ii is not needed, take the identity
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
    TRY(dalloc(h, &B.Dm, soff[nagg]));
    TRY(dalloc(h, &B.Em, soff[nagg]));
    TRY(dalloc(h, &B.Fm, soff[nagg]));
    TRY(dalloc(h, &B.Tm, soff[nagg]));
    T *blocks4[4] = {B.Dm, B.Em, B.Fm, B.Tm};
    for (int q = 0; q < 4; ++q)
      CK(cudaMemsetAsync(blocks4[q], 0, sizeof(T) * std::max<int64_t>(soff[nagg], 1), s));
    int64_t *d_i;
    double *d_v;
    TRY(upload(h, &d_i, di)); TRY(upload(h, &d_v, dv));
    CK(launch_scatter_coo<T>((int64_t)di.size(), d_i, d_v, B.Dm, s));
    TRY(upload(h, &d_i, ei)); TRY(upload(h, &d_v, ev));
    CK(launch_scatter_coo<T>((int64_t)ei.size(), d_i, d_v, B.Em, s));
    TRY(upload(h, &d_i, fi)); TRY(upload(h, &d_v, fv));
    CK(launch_scatter_coo<T>((int64_t)fi.size(), d_i, d_v, B.Fm, s));
    CK(launch_block_amax<T>(nagg, h->d_p, h->s_off, B.Dm, B.amax, s));
    CK(launch_gj_inverse<T>(nagg, h->d_p, h->s_off, h->pmax, B.Dm, h->ipiv, h->poff, B.amax,
                            h->failed, B.gj, pivtol, h->st, DD_ERR_SINGULAR_SCHUR, s));
    if (h->kind == DD_MSCN) {
      CK(launch_block_gemm<T>(nagg, h->d_p, h->s_off, h->pmax, B.Dm, B.Em, B.Tm, T(1), T(0), s));
      CK(launch_block_gemm<T>(nagg, h->d_p, h->s_off, h->pmax, B.Fm, B.Tm, B.S, T(-1), T(1), s));
    } else {
      CK(launch_mscnr_diag<T>(nagg, h->d_p, h->s_off, h->pmax, B.Dm, B.Em, B.Fm, B.S, s));
    }
  }
  // ---- explicit inverses of the S_hat blocks
  CK(launch_block_amax<T>(nagg, h->d_p, h->s_off, B.S, B.amax, s));
  CK(launch_gj_inverse<T>(nagg, h->d_p, h->s_off, h->pmax, B.S, h->ipiv, h->poff, B.amax,
                          h->failed, B.gj, pivtol, h->st, DD_ERR_SINGULAR_SCHUR, s));
  TRY(dalloc(h, &B.z1, std::max(nI, 1)));
  TRY(dalloc(h, &B.z2, std::max(nG, 1)));
  TRY(dalloc(h, &B.t, std::max(nG, 1)));
  return DD_OK;
}

template <typename T>
dd_status apply_T(DDHandle *h, const double *y, double *x, cudaStream_t s, int part = -1) {
  PrecBufs<T> &B = bufs<T>(h);
  if (part == 0 || part < 0)
  CK(launch_band_solve_fwd<T>(h->d_info, h->m, h->max_n, h->max_kl, h->max_ku2, h->stage_bytes,
                              h->tm, h->jobs, B.ltile, B.utile, h->src, y, h->d_perm, B.z1, h->st,
                              h->sweep_threads, s));
  if (part == 1 || part < 0)
  CK(launch_schur_apply<T>(h->nagg, h->agg_off, h->s_off, h->pmax, B.S, h->f_ptr, h->f_col,
                           B.f_val, y, h->d_perm + h->nI, B.z1, B.z2, B.t, h->nG, x, s));
  if (part == 2 || part < 0)
  CK(launch_band_solve_bwd<T>(h->d_info, h->m, h->max_n, h->max_kl, h->max_ku2, h->stage_bytes,
                              h->tm, h->jobs, B.ltile, B.utile, h->src, h->e_ptr, h->e_col, B.e_val,
                              B.z2, B.z1, h->d_perm, x, h->st, h->sweep_threads, s));
  return DD_OK;
}

dd_status apply_any(DDHandle *h, const double *y, double *x, cudaStream_t s, int part = -1) {
  return h->prec == DD_FP32 ? apply_T<float>(h, y, x, s, part) : apply_T<double>(h, y, x, s, part);
}

}  // namespace

namespace {

dd_status alloc_krylov(DDHandle *h, int R) {
  h->Rmax = R;
  h->ldv = ((h->n + 31) / 32) * 32;
  TRY(dalloc(h, &h->V, (size_t)h->ldv * (R + 1)));
  TRY(dalloc(h, &h->Z, (size_t)h->ldv * R));
  TRY(dalloc(h, &h->H, (size_t)(R + 1) * R));
  TRY(dalloc(h, &h->cs, R));
  TRY(dalloc(h, &h->sn, R));
  TRY(dalloc(h, &h->g, R + 1));
  TRY(dalloc(h, &h->y, R + 1));
  TRY(dalloc(h, &h->hc1, R + 2));
  TRY(dalloc(h, &h->hc2, R + 2));
  TRY(dalloc(h, &h->nsq, 4));
  TRY(dalloc(h, &h->out, 4));
  h->cgs_blocks = cgs2_blocks(304);
  if (h->cgs_blocks <= 0) { h->err = "no resident blocks for the cooperative CGS2 kernel"; return DD_ERR_CUDA; }
  TRY(dalloc(h, &h->partial, 3 * (size_t)std::max(h->nblocks, h->cgs_blocks) * (R + 2)));
  TRY(dalloc(h, &h->r, h->ldv));
  cudaError_t e = cudaMallocHost(&h->h_out, 8 * sizeof(double));
  if (e != cudaSuccess) { h->err = "cudaMallocHost failed"; return DD_ERR_OOM; }
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

dd_status fgmres(DDHandle *h, const double *b, double *x, double tol, int R, int maxit,
                 dd_info *info, cudaStream_t s) {
  const int n = (int)h->n;
  int iters = 0, restarts = 0;
  double relres = 0.0;
  dd_status rc = DD_ERR_NOT_CONVERGED;
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
    int jlast = -1;
    for (int j = 0; j < R; ++j) {
      double *vj = h->V + (int64_t)j * h->ldv, *zj = h->Z + (int64_t)j * h->ldv;
      double *w = h->V + (int64_t)(j + 1) * h->ldv;
      TRY(apply_any(h, vj, zj, s));
      CK(launch_spmv(n, h->c_rowptr, h->c_col, h->c_val, zj, w, s));
      CK(launch_cgs2(n, j, R, h->V, h->ldv, w, h->partial, h->Rmax + 2, h->hc1, h->hc2, h->H, h->cs,
                     h->sn, h->g, bnorm, h->out, h->cgs_blocks, s));
      TRY(read_scalars(h, h->out, 3, s));
      ++iters;
      const double est = h->h_out[2];
      const bool breakdown = h->h_out[1] != 0.0;
      if (info && info->history && iters - 1 < info->history_cap) info->history[iters - 1] = est;
      jlast = j;
      if (!isfinite(est)) { rc = DD_ERR_NONFINITE; goto done; }
      if (est <= tol || breakdown || iters >= maxit) break;
    }
    CK(launch_hess_solve_update(n, jlast, R, h->H, h->g, h->y, h->Z, h->ldv, x, s));
    CK(launch_residual(n, h->c_rowptr, h->c_col, h->c_val, x, b, h->r, s));
    TRY(norm_sq(h, h->r, 3, s));
    TRY(read_scalars(h, h->nsq + 3, 1, s));
    {
      DevStatus dst{};
      CK(cudaMemcpy(&dst, h->st, sizeof dst, cudaMemcpyDeviceToHost));
      if (dst.code != 0) {
        h->err = "device wait expired in an apply sweep";
        rc = (dd_status)dst.code;
        break;
      }
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

void release(DDHandle *h) {
  for (void *p : h->allocs) cudaFreeAsync(p, h->stream);
  h->allocs.clear();
  cudaStreamSynchronize(h->stream);
  if (h->h_out) cudaFreeHost(h->h_out);
  h->h_out = nullptr;
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
  CK(launch_band_solve_fwd<T>(h->d_info, h->m, h->max_n, h->max_kl, h->max_ku2, h->stage_bytes,
                              h->tm, h->jobs, B.ltile, B.utile, h->src, y, h->d_perm, z1, h->st,
                              h->sweep_threads, s));
  CK(launch_schur_apply<T>(h->nagg, h->agg_off, h->s_off, h->pmax, B.S, h->f_ptr, h->f_col,
                           B.f_val, y, h->d_perm + h->nI, z1, z2, z2 + z2_elems, h->nG, x, s));
  CK(launch_band_solve_bwd<T>(h->d_info, h->m, h->max_n, h->max_kl, h->max_ku2, h->stage_bytes,
                              h->tm, h->jobs, B.ltile, B.utile, h->src, h->e_ptr, h->e_col, B.e_val,
                              z2, z1, h->d_perm, x, h->st, h->sweep_threads, s));
  return DD_OK;
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
  if ((int)approx < DD_EXACT || (int)approx > DD_LUM) { g_setup_error = "unknown approximation"; return DD_ERR_INVALID_ARG; }
  dd_opts o{};
  o.prec = DD_FP64;
  if (opts) o = *opts;
  if (o.prec != DD_FP64 && o.prec != DD_FP32) { g_setup_error = "unknown precision"; return DD_ERR_INVALID_ARG; }
  DDHandle *h = new (std::nothrow) DDHandle();
  if (!h) return DD_ERR_OOM;
  h->stream = static_cast<cudaStream_t>(stream);
  h->prec = o.prec;
  h->kind = approx;
  const double pivtol = o.pivot_tol > 0 ? o.pivot_tol : (o.prec == DD_FP32 ? 1e-7 : 1e-14);
  const int R = o.max_restart > 0 ? o.max_restart : 50;
  if (R > 120) { g_setup_error = "max_restart must be <= 120"; delete h; return DD_ERR_INVALID_ARG; }
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
  if (rc == DD_OK || rc == DD_ERR_SINGULAR_BLOCK || rc == DD_ERR_SINGULAR_SCHUR) {
    *handle = h;
    g_setup_error = h->err;
    return rc;
  }
  g_setup_error = h->err;
  release(h);
  delete h;
  return rc;
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  dd_status rc = fgmres(h, b, x, tol, restart, maxit, info, s);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) { info->solve_ms = ms; info->setup_ms = h->stats.setup_ms; info->bad_block = h->bad_block; }
  return rc;
}

dd_status dd_spmv(void *handle, const double *x, double *y, void *stream) {
  DDHandle *h = static_cast<DDHandle *>(handle);
  if (!h || !x || !y) return DD_ERR_INVALID_ARG;
  cudaError_t e = launch_spmv((int)h->n, h->c_rowptr, h->c_col, h->c_val, x, y, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) { h->err = cudaGetErrorString(e); return DD_ERR_CUDA; }
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
