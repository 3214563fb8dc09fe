// Interior blocks A_jj: banded LU with partial pivoting, conversion of the
// factors into sweep tiles, and the blocked forward/backward sweeps
// (Section 4: exact triangular factors of every D_ii, all subdomains in one
// launch; Algorithm 2: z1 = A^-1 y1 and x1 = z1 - A^-1 (E x2)).
//
// Storage (per subdomain j, rows in the local RCM order):
//   band   row i holds columns i-kl .. i+kl+ku at offsets 0 .. 2kl+ku
//   lm     multipliers of step k (rows k+1..k+kl in the row order of step k)
//   piv    row exchanged with k at step k
// Sweep tiles (DD_NB = 32 columns each):
//   forward tile t, window rows c0 .. c0+NB+kl-1 (c0 = t*NB):
//     src[q]   window position whose value moves to q once the tile's row
//              exchanges are applied in order
//     Linv     inverse of the tile's unit lower triangle (multipliers with the
//              later exchanges of the same tile applied), column-major NB x NB
//     L21      the kl rows below the tile, column-major (element (i,c) at c*kl+i)
//   backward tile t, rows r0 .. r0+NB-1:
//     Uinv     inverse of the NB x NB upper triangle, column-major
//     U12      U(r0+i, r0+NB+q), stored [q*NB + i], q < kl+ku
#include <cuda_runtime.h>
#include <stdint.h>

#include "dd_internal.h"

namespace {

template <typename T>
__device__ __forceinline__ T tabs(T v) { return v < T(0) ? -v : v; }

__device__ void set_status(DevStatus *st, int code, int block) {
  if (atomicCAS(&st->code, 0, code) == 0) st->block = block;
}

// ---------------------------------------------------------------------------
// Banded LU, one CTA per subdomain.  The active window (kl+1 rows by kl+ku+1
// columns) stays in L2; the multipliers and the pivot row are staged in
// shared memory for the rank-1 update.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void band_lu_kernel(const BandInfo *__restrict__ info, T *band, T *lm, int32_t *piv,
                               double pivtol, DevStatus *st) {
  const BandInfo b = info[blockIdx.x];
  const int n = b.n, kl = b.kl, ku = b.ku, wd = 2 * kl + ku + 1;
  if (n == 0) return;
  T *A = band + b.band_off;
  T *L = lm + b.lm_off;
  int32_t *P = piv + b.piv_off;
  extern __shared__ unsigned char smraw[];
  T *lsh = reinterpret_cast<T *>(smraw);  // kl multipliers
  T *ush = lsh + (kl + 1);                // kl+ku pivot-row entries
  __shared__ T red[32];
  __shared__ int32_t s_p;
  __shared__ int32_t s_fail;
  __shared__ T s_amax;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
            nw = nt >> 5;

  // largest magnitude of the block (the reference of the pivot test)
  T mx = T(0);
  for (int64_t q = tid; q < (int64_t)n * wd; q += nt) mx = fmax(mx, tabs(A[q]));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  if (tid == 0) {
    T m2 = T(0);
    for (int w = 0; w < nw; ++w) m2 = fmax(m2, red[w]);
    s_amax = m2;
  }
  __syncthreads();
  const T thresh = T(pivtol) * s_amax;

  for (int k = 0; k < n; ++k) {
    const int last = min(n - 1, k + kl), jend = min(n - 1, k + kl + ku);
    if (warp == 0) {
      // first row holding the largest magnitude in column k
      T best = T(-1);
      int bi = n;
      for (int i = k + lane; i <= last; i += 32) {
        T v = tabs(A[(int64_t)i * wd + (k - i + kl)]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        s_p = bi;
        P[k] = bi;
        if (!(best > thresh)) { s_fail = 1; set_status(st, DD_ERR_SINGULAR_BLOCK, blockIdx.x); }
      }
    }
    __syncthreads();
    if (s_fail) return;
    const int p = s_p;
    if (p != k)
      for (int c = k + tid; c <= jend; c += nt) {
        T *a = &A[(int64_t)k * wd + (c - k + kl)];
        T *bq = &A[(int64_t)p * wd + (c - p + kl)];
        T t = *a; *a = *bq; *bq = t;
      }
    __syncthreads();
    const T dkk = A[(int64_t)k * wd + kl];
    for (int i = k + 1 + tid; i <= last; i += nt) {
      T *a = &A[(int64_t)i * wd + (k - i + kl)];
      T l = *a / dkk;
      L[(int64_t)k * kl + (i - k - 1)] = l;
      lsh[i - k - 1] = l;
      *a = T(0);
    }
    for (int c = k + 1 + tid; c <= jend; c += nt) ush[c - k - 1] = A[(int64_t)k * wd + (c - k + kl)];
    __syncthreads();
    const int nr = last - k, nc = jend - k;
    for (int r = warp; r < nr; r += nw) {
      const T l = lsh[r];
      const int i = k + 1 + r;
      T *row = &A[(int64_t)i * wd + (k + 1 - i + kl)];
      for (int c = lane; c < nc; c += 32) row[c] -= l * ush[c];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Sweep tiles: one warp per (subdomain, tile); lane = tile column / row.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void band_tiles_kernel(const BandInfo *__restrict__ info, const T *__restrict__ band,
                                  const T *__restrict__ lm, const int32_t *__restrict__ piv,
                                  T *ltile, T *utile, int32_t *srcs) {
  const BandInfo b = info[blockIdx.x];
  const int t = blockIdx.y;
  if (t >= b.ntiles) return;
  const int n = b.n, kl = b.kl, ku2 = b.kl + b.ku, wd = 2 * b.kl + b.ku + 1;
  const int W = DD_NB + kl;
  const int c0 = t * DD_NB;
  const int lane = threadIdx.x;
  const T *A = band + b.band_off;
  const T *L = lm + b.lm_off;
  const int32_t *P = piv + b.piv_off;
  T *lt = ltile + b.ltile_off + (int64_t)t * bi_ltile_elems(b);
  T *ut = utile + b.utile_off + (int64_t)t * bi_utile_elems(b);
  int32_t *src = srcs + b.src_off + (int64_t)t * W;
  extern __shared__ unsigned char smraw[];
  T *L11 = reinterpret_cast<T *>(smraw);         // NB x NB, [row][col]
  T *vbuf = L11 + DD_NB * DD_NB;                 // 32 columns x W
  int32_t *idx = reinterpret_cast<int32_t *>(vbuf + (size_t)DD_NB * W);

  // (1) composite window permutation of the tile's row exchanges
  if (lane == 0) {
    for (int q = 0; q < W; ++q) idx[q] = q;
    for (int c = c0; c < c0 + DD_NB && c < n; ++c) {
      int a = c - c0, bq = P[c] - c0;
      int tmp = idx[a]; idx[a] = idx[bq]; idx[bq] = tmp;
    }
  }
  __syncwarp();
  for (int q = lane; q < W; q += 32) src[q] = idx[q];

  // (2) multipliers of column c0+lane with the later exchanges applied
  {
    T *v = vbuf + (size_t)lane * W;
    for (int q = 0; q < W; ++q) v[q] = T(0);
    const int c = c0 + lane;
    if (c < n) {
      for (int r = 0; r < kl; ++r) {
        int row = c + 1 + r;
        if (row < n) v[row - c0] = L[(int64_t)c * kl + r];
      }
      for (int c2 = c + 1; c2 < c0 + DD_NB && c2 < n; ++c2) {
        int a = c2 - c0, bq = P[c2] - c0;
        T tmp = v[a]; v[a] = v[bq]; v[bq] = tmp;
      }
    }
    for (int q = 0; q < DD_NB; ++q) L11[q * DD_NB + lane] = (q == lane) ? T(1) : (q > lane ? v[q] : T(0));
    T *L21 = lt + DD_NB * DD_NB;
    for (int r = 0; r < kl; ++r) L21[(int64_t)lane * kl + r] = v[DD_NB + r];
  }
  __syncwarp();
  // (3) Linv: column `lane` of the inverse of the unit lower triangle
  {
    T x[DD_NB];
#pragma unroll
    for (int q = 0; q < DD_NB; ++q) x[q] = T(0);
    x[lane] = T(1);
    for (int q = lane + 1; q < DD_NB; ++q) {
      T s = T(0);
      for (int r = lane; r < q; ++r) s += L11[q * DD_NB + r] * x[r];
      x[q] = -s;
    }
    for (int q = 0; q < DD_NB; ++q) lt[lane * DD_NB + q] = x[q];
  }
  __syncwarp();
  // (4) U11 (row-major in L11's buffer), Uinv, U12
  {
    const int r = c0 + lane;  // row of this lane
    for (int c = 0; c < DD_NB; ++c) {
      T v = T(0);
      if (r < n) {
        int col = c0 + c;
        int off = col - r + kl;
        if (c >= lane && col < n && off < wd) v = A[(int64_t)r * wd + off];
      } else if (c == lane) {
        v = T(1);
      }
      L11[lane * DD_NB + c] = v;
    }
    T *U12 = ut + DD_NB * DD_NB;
    for (int q = 0; q < ku2; ++q) {
      T v = T(0);
      int col = c0 + DD_NB + q;
      if (r < n && col < n) {
        int off = col - r + kl;
        if (off < wd) v = A[(int64_t)r * wd + off];
      }
      U12[(int64_t)q * DD_NB + lane] = v;
    }
  }
  __syncwarp();
  {
    // column `lane` of U11^-1: x[lane] = 1/U(lane,lane), back substitution up
    T x[DD_NB];
#pragma unroll
    for (int q = 0; q < DD_NB; ++q) x[q] = T(0);
    x[lane] = T(1) / L11[lane * DD_NB + lane];
    for (int q = lane - 1; q >= 0; --q) {
      T s = T(0);
      for (int r = q + 1; r <= lane; ++r) s += L11[q * DD_NB + r] * x[r];
      x[q] = -s / L11[q * DD_NB + q];
    }
    for (int q = 0; q < DD_NB; ++q) ut[lane * DD_NB + q] = x[q];
  }
}

// ---------------------------------------------------------------------------
// Single right-hand side sweeps over a vector resident in shared memory.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void sweep_forward(const BandInfo &b, const T *__restrict__ ltile,
                              const int32_t *__restrict__ srcs, T *vec, T *win, T *ysh) {
  const int kl = b.kl, W = DD_NB + kl;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int t = 0; t < b.ntiles; ++t) {
    const int c0 = t * DD_NB;
    const int32_t *src = srcs + b.src_off + (int64_t)t * W;
    const T *lt = ltile + b.ltile_off + (int64_t)t * bi_ltile_elems(b);
    for (int q = tid; q < W; q += nt) win[q] = vec[c0 + src[q]];
    __syncthreads();
    if (warp == 0) {
      T y = T(0);
#pragma unroll 8
      for (int c = 0; c < DD_NB; ++c) y += lt[c * DD_NB + lane] * win[c];
      ysh[lane] = y;
      vec[c0 + lane] = y;
    }
    __syncthreads();
    const T *L21 = lt + DD_NB * DD_NB;
    for (int i = tid; i < kl; i += nt) {
      T s = win[DD_NB + i];
#pragma unroll 8
      for (int c = 0; c < DD_NB; ++c) s -= L21[(int64_t)c * kl + i] * ysh[c];
      vec[c0 + DD_NB + i] = s;
    }
    __syncthreads();
  }
}

template <typename T>
__device__ void sweep_backward(const BandInfo &b, const T *__restrict__ utile, T *vec, T *part,
                               T *ssh) {
  const int ku2 = b.kl + b.ku;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int t = b.ntiles - 1; t >= 0; --t) {
    const int r0 = t * DD_NB;
    const T *ut = utile + b.utile_off + (int64_t)t * bi_utile_elems(b);
    const T *U12 = ut + DD_NB * DD_NB;
    T s = T(0);
    for (int q = warp; q < ku2; q += nw) s += U12[(int64_t)q * DD_NB + lane] * vec[r0 + DD_NB + q];
    part[warp * DD_NB + lane] = s;
    __syncthreads();
    if (warp == 0) {
      T acc = vec[r0 + lane];
      for (int w = 0; w < nw; ++w) acc -= part[w * DD_NB + lane];
      ssh[lane] = acc;
      __syncwarp();
      T x = T(0);
#pragma unroll 8
      for (int c = 0; c < DD_NB; ++c) x += ut[c * DD_NB + lane] * ssh[c];
      vec[r0 + lane] = x;
    }
    __syncthreads();
  }
}

// z = A_jj^-1 y_j with y gathered from the original numbering.
template <typename T>
__global__ void band_solve_fwd_kernel(const BandInfo *__restrict__ info, int max_n, int max_kl,
                                      int max_ku2, const T *__restrict__ ltile,
                                      const T *__restrict__ utile, const int32_t *__restrict__ srcs,
                                      const double *__restrict__ y, const int32_t *__restrict__ perm,
                                      T *z) {
  const BandInfo b = info[blockIdx.x];
  if (b.n == 0) return;
  extern __shared__ unsigned char smraw[];
  T *vec = reinterpret_cast<T *>(smraw);
  int pad = (max_kl > max_ku2 ? max_kl : max_ku2) + 2 * DD_NB;
  T *win = vec + max_n + pad;
  T *ysh = win + DD_NB + max_kl;
  T *part = ysh + DD_NB;
  T *ssh = part + (blockDim.x >> 5) * DD_NB;
  const int ntot = b.ntiles * DD_NB + pad;
  for (int i = threadIdx.x; i < ntot; i += blockDim.x)
    vec[i] = (i < b.n) ? T(y[perm[b.row0 + i]]) : T(0);
  __syncthreads();
  sweep_forward(b, ltile, srcs, vec, win, ysh);
  sweep_backward(b, utile, vec, part, ssh);
  for (int i = threadIdx.x; i < b.n; i += blockDim.x) z[b.row0 + i] = vec[i];
}

// x1 = z1 - A_jj^-1 (E z2)_j, scattered to x in the original numbering.
template <typename T>
__global__ void band_solve_bwd_kernel(const BandInfo *__restrict__ info, int max_n, int max_kl,
                                      int max_ku2, const T *__restrict__ ltile,
                                      const T *__restrict__ utile, const int32_t *__restrict__ srcs,
                                      const int32_t *__restrict__ e_ptr,
                                      const int32_t *__restrict__ e_col,
                                      const T *__restrict__ e_val, const T *__restrict__ z2,
                                      const T *__restrict__ z1, const int32_t *__restrict__ perm,
                                      double *x) {
  const BandInfo b = info[blockIdx.x];
  if (b.n == 0) return;
  extern __shared__ unsigned char smraw[];
  T *vec = reinterpret_cast<T *>(smraw);
  int pad = (max_kl > max_ku2 ? max_kl : max_ku2) + 2 * DD_NB;
  T *win = vec + max_n + pad;
  T *ysh = win + DD_NB + max_kl;
  T *part = ysh + DD_NB;
  T *ssh = part + (blockDim.x >> 5) * DD_NB;
  const int ntot = b.ntiles * DD_NB + pad;
  for (int i = threadIdx.x; i < ntot; i += blockDim.x) {
    T v = T(0);
    if (i < b.n) {
      const int r = b.row0 + i;
      for (int k = e_ptr[r]; k < e_ptr[r + 1]; ++k) v += e_val[k] * z2[e_col[k]];
    }
    vec[i] = v;
  }
  __syncthreads();
  sweep_forward(b, ltile, srcs, vec, win, ysh);
  sweep_backward(b, utile, vec, part, ssh);
  for (int i = threadIdx.x; i < b.n; i += blockDim.x) {
    const int r = b.row0 + i;
    x[perm[r]] = double(z1[r] - vec[i]);
  }
}

// ---------------------------------------------------------------------------
// Multiple right-hand sides (setup of the Schur blocks): X = A_jj^-1 X for a
// chunk of NR columns per CTA; X column-major (leading dimension n_j) in
// global memory, the tile windows staged in shared memory.
// ---------------------------------------------------------------------------
template <typename T, int NR>
__global__ void band_solve_multi_kernel(const BandInfo *__restrict__ info,
                                        const int32_t *__restrict__ ncols,
                                        const int64_t *__restrict__ x_off,
                                        const T *__restrict__ ltile, const T *__restrict__ utile,
                                        const int32_t *__restrict__ srcs, T *Xall) {
  const BandInfo b = info[blockIdx.x];
  const int nc = ncols[blockIdx.x];
  const int k0 = blockIdx.y * NR;
  if (b.n == 0 || k0 >= nc) return;
  const int nr = min(NR, nc - k0);
  const int n = b.n, kl = b.kl, ku2 = b.kl + b.ku, W = DD_NB + kl;
  T *X = Xall + x_off[blockIdx.x] + (int64_t)k0 * n;
  extern __shared__ unsigned char smraw[];
  T *win = reinterpret_cast<T *>(smraw);  // (NB + max(kl,ku2)) x NR, [row][r]
  T *ysh = win + (size_t)(DD_NB + (kl > ku2 ? kl : ku2)) * NR;  // NB x NR
  const int tid = threadIdx.x, nt = blockDim.x;
  // forward
  for (int t = 0; t < b.ntiles; ++t) {
    const int c0 = t * DD_NB;
    const int32_t *src = srcs + b.src_off + (int64_t)t * W;
    const T *lt = ltile + b.ltile_off + (int64_t)t * bi_ltile_elems(b);
    for (int e = tid; e < W * NR; e += nt) {
      int q = e / NR, r = e % NR;
      int row = c0 + src[q];
      win[e] = (row < n && r < nr) ? X[(int64_t)r * n + row] : T(0);
    }
    __syncthreads();
    for (int e = tid; e < DD_NB * NR; e += nt) {
      int i = e / NR, r = e % NR;
      T y = T(0);
      for (int c = 0; c < DD_NB; ++c) y += lt[c * DD_NB + i] * win[c * NR + r];
      ysh[e] = y;
      if (c0 + i < n && r < nr) X[(int64_t)r * n + c0 + i] = y;
    }
    __syncthreads();
    const T *L21 = lt + DD_NB * DD_NB;
    for (int e = tid; e < kl * NR; e += nt) {
      int i = e / NR, r = e % NR;
      T s = win[(DD_NB + i) * NR + r];
      for (int c = 0; c < DD_NB; ++c) s -= L21[(int64_t)c * kl + i] * ysh[c * NR + r];
      if (c0 + DD_NB + i < n && r < nr) X[(int64_t)r * n + c0 + DD_NB + i] = s;
    }
    __syncthreads();
  }
  // backward
  for (int t = b.ntiles - 1; t >= 0; --t) {
    const int r0 = t * DD_NB;
    const T *ut = utile + b.utile_off + (int64_t)t * bi_utile_elems(b);
    const T *U12 = ut + DD_NB * DD_NB;
    for (int e = tid; e < (DD_NB + ku2) * NR; e += nt) {
      int q = e / NR, r = e % NR;
      int row = r0 + q;
      win[e] = (row < n && r < nr) ? X[(int64_t)r * n + row] : T(0);
    }
    __syncthreads();
    for (int e = tid; e < DD_NB * NR; e += nt) {
      int i = e / NR, r = e % NR;
      T s = win[i * NR + r];
      for (int q = 0; q < ku2; ++q) s -= U12[(int64_t)q * DD_NB + i] * win[(DD_NB + q) * NR + r];
      ysh[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < DD_NB * NR; e += nt) {
      int i = e / NR, r = e % NR;
      T x = T(0);
      for (int c = 0; c < DD_NB; ++c) x += ut[c * DD_NB + i] * ysh[c * NR + r];
      if (r0 + i < n && r < nr) X[(int64_t)r * n + r0 + i] = x;
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static size_t lu_smem(int max_kl, int max_ku, size_t es) { return es * (size_t)(2 * max_kl + max_ku + 2); }
static size_t tiles_smem(int max_kl, size_t es) {
  int W = DD_NB + max_kl;
  return es * (size_t)(DD_NB * DD_NB + DD_NB * W) + sizeof(int32_t) * (size_t)W;
}
static size_t sweep_smem(int max_n, int max_kl, int max_ku2, int threads, size_t es) {
  int pad = (max_kl > max_ku2 ? max_kl : max_ku2) + 2 * DD_NB;
  size_t e = (size_t)max_n + pad + (DD_NB + max_kl) + DD_NB + (size_t)(threads / 32) * DD_NB + DD_NB;
  return e * es;
}
#define DD_MULTI_NR 16
static size_t multi_smem(int max_kl, int max_ku2, size_t es) {
  int w = DD_NB + (max_kl > max_ku2 ? max_kl : max_ku2);
  return es * (size_t)(w + DD_NB) * DD_MULTI_NR;
}

template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t band_sweep_smem_bytes(int max_n, int max_kl, int max_ku2, int threads, int elem_size) {
  return sweep_smem(max_n, max_kl, max_ku2, threads, (size_t)elem_size);
}

template <typename T>
cudaError_t launch_band_lu(const BandInfo *d_info, int m, int max_kl, int max_ku, T *band, T *lm,
                           int32_t *piv, double pivtol, DevStatus *st, int threads, cudaStream_t s) {
  size_t smem = lu_smem(max_kl, max_ku, sizeof(T));
  cudaError_t e = ensure_smem(band_lu_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  band_lu_kernel<T><<<m, threads, smem, s>>>(d_info, band, lm, piv, pivtol, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_tiles(const BandInfo *d_info, int m, int max_tiles, int max_kl,
                              const T *band, const T *lm, const int32_t *piv, T *ltile, T *utile,
                              int32_t *src, cudaStream_t s) {
  size_t smem = tiles_smem(max_kl, sizeof(T));
  cudaError_t e = ensure_smem(band_tiles_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(m, max_tiles);
  band_tiles_kernel<T><<<grid, 32, smem, s>>>(d_info, band, lm, piv, ltile, utile, src);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_solve_fwd(const BandInfo *d_info, int m, int max_n, int max_kl,
                                  int max_ku2, const T *ltile, const T *utile, const int32_t *src,
                                  const double *y, const int32_t *perm, T *z, int threads,
                                  cudaStream_t s) {
  size_t smem = sweep_smem(max_n, max_kl, max_ku2, threads, sizeof(T));
  cudaError_t e = ensure_smem(band_solve_fwd_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  band_solve_fwd_kernel<T><<<m, threads, smem, s>>>(d_info, max_n, max_kl, max_ku2, ltile, utile,
                                                     src, y, perm, z);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_solve_bwd(const BandInfo *d_info, int m, int max_n, int max_kl,
                                  int max_ku2, const T *ltile, const T *utile, const int32_t *src,
                                  const int32_t *e_ptr, const int32_t *e_col, const T *e_val,
                                  const T *z2, const T *z1, const int32_t *perm, double *x,
                                  int threads, cudaStream_t s) {
  size_t smem = sweep_smem(max_n, max_kl, max_ku2, threads, sizeof(T));
  cudaError_t e = ensure_smem(band_solve_bwd_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  band_solve_bwd_kernel<T><<<m, threads, smem, s>>>(d_info, max_n, max_kl, max_ku2, ltile, utile,
                                                     src, e_ptr, e_col, e_val, z2, z1, perm, x);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_solve_multi(const BandInfo *d_info, int m, const int32_t *ncols,
                                    const int64_t *x_off, int max_cols, int max_kl, int max_ku2,
                                    const T *ltile, const T *utile, const int32_t *src, T *X,
                                    cudaStream_t s) {
  if (max_cols <= 0) return cudaSuccess;
  size_t smem = multi_smem(max_kl, max_ku2, sizeof(T));
  cudaError_t e = ensure_smem(band_solve_multi_kernel<T, DD_MULTI_NR>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(m, (max_cols + DD_MULTI_NR - 1) / DD_MULTI_NR);
  band_solve_multi_kernel<T, DD_MULTI_NR><<<grid, 256, smem, s>>>(d_info, ncols, x_off, ltile,
                                                                  utile, src, X);
  return cudaGetLastError();
}

#define DD_INST_BAND(T)                                                                          \
  template cudaError_t launch_band_lu<T>(const BandInfo *, int, int, int, T *, T *, int32_t *,   \
                                         double, DevStatus *, int, cudaStream_t);                 \
  template cudaError_t launch_band_tiles<T>(const BandInfo *, int, int, int, const T *,          \
                                            const T *, const int32_t *, T *, T *, int32_t *,     \
                                            cudaStream_t);                                        \
  template cudaError_t launch_band_solve_fwd<T>(const BandInfo *, int, int, int, int, const T *, \
                                                const T *, const int32_t *, const double *,      \
                                                const int32_t *, T *, int, cudaStream_t);         \
  template cudaError_t launch_band_solve_bwd<T>(                                                 \
      const BandInfo *, int, int, int, int, const T *, const T *, const int32_t *,               \
      const int32_t *, const int32_t *, const T *, const T *, const T *, const int32_t *,        \
      double *, int, cudaStream_t);                                                              \
  template cudaError_t launch_band_solve_multi<T>(const BandInfo *, int, const int32_t *,        \
                                                  const int64_t *, int, int, int, const T *,     \
                                                  const T *, const int32_t *, T *, cudaStream_t);

DD_INST_BAND(double)
DD_INST_BAND(float)
