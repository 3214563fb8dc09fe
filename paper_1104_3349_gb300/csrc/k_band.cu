// Interior blocks A_jj: blocked banded LU with partial pivoting, packing of
// the factors into sweep tiles, and the blocked forward/backward sweeps
// (Section 4: exact triangular factors of every D_ii, all subdomains in one
// launch; Algorithm 2: z1 = A^-1 y1 and x1 = z1 - A^-1 (E x2)).
//
// Storage (per subdomain j, rows in the local RCM order):
//   band   row i holds columns i-kl .. i+kl+ku at offsets 0 .. 2kl+ku
//   lraw   per tile of DD_NB = 32 columns, the multipliers in the row order
//          after the tile's exchanges, (NB+kl) x NB column-major
//   piv    row exchanged with k at step k
// Packed sweep tiles (TileMeta) of TB = 64 columns (two LU panels) in FP32
// and 32 in FP64, trimmed to the rows / columns that hold nonzeros after the
// factorisation:
//   forward tile t, window rows c0 .. c0+wl-1 (c0 = t*TB):
//     src[q]   window position whose value moves to q once the tile's row
//              exchanges (both panels', in order) are applied
//     K        wl x TB: rows 0..TB-1 hold Linv, the inverse of the tile's
//              unit lower triangle L11; rows TB.. hold -L21 Linv.  L is in
//              the row order after all of the tile's exchanges (the second
//              panel's exchanges also move the first panel's multipliers).
//              The tile step is w <- [0; w_B] + K w_T on the exchanged
//              window w.
//   backward tile t, rows r0 .. r0+TB-1:
//     Kb       TB x wu: [Uinv | -Uinv U12], Uinv the inverse of the tile's
//              upper triangle, so x_T = Kb [b_T; x_next].
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <climits>

#include <algorithm>
#include <utility>

#include "dd_internal.h"

namespace {

__host__ __device__ inline int src_stride_w(int w) { return round4(w); }
// row stride of a cluster sweep's exchange buffers (room for any tile slice)
__host__ __device__ inline int sweep_xbs(int tb, int max_kl) { return round4(tb + max_kl + 8); }
// elements of one step's message between the two CTAs of a cluster sweep:
// sweep_xbs row values, then the sender's flag and padding
__host__ __device__ inline int sweep_msg(int tb, int max_kl) { return sweep_xbs(tb, max_kl) + 4; }
// zero padding beyond the tiles of the resident vectors: room for the
// widest window or row of a tile, a multiple of 32 elements
__host__ __device__ inline int sweep_pad_hd(int max_kl, int max_ku2) {
  return ((max_kl > max_ku2 ? max_kl : max_ku2) + 2 * DD_TB_WIDE + 31) & ~31;
}

// The band LU's window: R = NB + kl rows by Cw = NB + kl + ku columns, with
// three spare rows and a row stride of at least Cw + 3, odd (so that walks
// down a column are free of bank conflicts).  The rank-NB update then runs in
// whole 4 x 4 micro-tiles without bounds checks: its rows reach R + 2 and its
// columns Cw + 2, and entries computed outside R x Cw land in the spare rows
// and columns, which nothing else reads.
__host__ __device__ inline int lu_ldw(int kl, int ku) { return (DD_NB + kl + ku + 3) | 1; }
__host__ __device__ inline int64_t lu_window_elems(int kl, int ku) {
  return (int64_t)(DD_NB + kl + 3) * lu_ldw(kl, ku);
}

// four consecutive T at a 16-byte aligned address (shared or global)
__device__ __forceinline__ void ld4(const float *p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <typename T>
__device__ __forceinline__ T tabs(T v) { return v < T(0) ? -v : v; }

__device__ void set_status(DevStatus *st, int code, int block) {
  if (atomicCAS(&st->code, 0, code) == 0) st->block = block;
}

// element (r, c) of a forward tile K (row-major, 16-byte chunks swizzled by row)
template <typename T, int TB>
__host__ __device__ __forceinline__ int kidx(int r, int c) {
  constexpr int CH = 16 / sizeof(T);
  return r * TB + (((c / CH) ^ (r & 7)) * CH) + (c % CH);
}

// ---------------------------------------------------------------------------
// Blocked banded LU with partial pivoting, one CTA per subdomain, panel =
// sweep tile (DD_NB columns).  For panel t (columns c0 .. c0+NB-1) the window
// rows c0 .. c0+NB+kl-1 by columns c0 .. c0+NB+kl+ku-1 is loaded (shared
// memory, or global scratch when it does not fit), then
//   - the panel columns are factored column by column (first largest
//     magnitude as pivot, exchanges of whole window rows),
//   - U12 = L11^-1 A12 and A22 -= L21 U12 (rank-NB update),
//   - the window goes back to the band rows and the panel's multipliers, in
//     the row order after the panel's exchanges, to lraw.
// The pivots are those of the column-by-column algorithm; the exchanges of
// later columns reach the multipliers of earlier columns of the same tile
// only, which is the order the forward sweep applies them in.
// ---------------------------------------------------------------------------
// CTA-wide argmax, ordered by value (larger first) then logical row (lower
// first): every thread offers (v, L, r); the warps' winners go to buffer buf.
// Every thread of the CTA must call it.
template <typename T>
__device__ __forceinline__ void offer_max(T v, int L, int r, T (*bv)[32], int (*bL)[32], int (*br)[32], int buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_argmax(v, L, r);
  if (lane == 0) { bv[buf][warp] = v; bL[buf][warp] = L; br[buf][warp] = r; }
}

// Panel factorisation with the row exchanges deferred: window rows stay in
// place while the panel's pivots are chosen (thread r owns row r, R <=
// blockDim.x).  Each thread keeps its row's logical position L, the position
// the exchanges so far would have moved it to, so ties go to the first
// logical row, as in the column-by-column algorithm.  The next column's
// candidates are offered as soon as a row is updated, so each column costs
// one barrier.  The exchanges are then applied, in order, to every column.
// Returns false (status set) if a pivot fails the test.
template <typename T>
__device__ bool lu_panel_lazy(T *W, int ldw, int R, int Cw, int c0, int n, int kl, int nbe, T thresh,
                              int32_t *P, DevStatus *st, int task, const T *cn, T tau) {
  __shared__ T bv[2][32];
  __shared__ int bL[2][32], br[2][32];
  __shared__ int sj[DD_NB];
  const int tid = threadIdx.x, nw = blockDim.x >> 5;
  const int r = tid;
  const bool own = r < R;
  int L = r;
  bool chosen = false;
  {
    const int last = min(min(R - 1, kl), n - 1 - c0);
    T v = T(-1);
    if (own && r <= last) {
      v = tabs(W[r * ldw]);
      if (!(v == v)) v = T(-1);
    }
    offer_max(v, own ? L : INT_MAX, r, bv, bL, br, 0);
  }
  for (int c = 0; c < nbe; ++c) {
    __syncthreads();  // column c's offers and every update of column c-1 are done
    const int buf = c & 1;
    // the warps' winners, one per lane, reduced in every warp
    const int lane = tid & 31;
    T best = lane < nw ? bv[buf][lane] : T(-1);
    int bestL = lane < nw ? bL[buf][lane] : INT_MAX, pr = lane < nw ? br[buf][lane] : 0;
    warp_argmax(best, bestL, pr);
    if (!(best > thresh)) {
      if (tid == 0) set_status(st, DD_ERR_SINGULAR_BLOCK, task);
      return false;
    }
    const int j = bestL;
    if (tid == 0) { P[c0 + c] = c0 + j; sj[c] = j; }
    const int last = min(min(R - 1, c + kl), n - 1 - c0);
    if (own && !chosen && r != pr && r <= last) {
      const T pv = W[pr * ldw + c];
      T l = W[r * ldw + c] / pv;
      if (tau > T(0)) {
        // the incomplete factorisation: a small multiplier, and small entries
        // of the pivot row, are dropped before they are used
        if (tabs(l) < tau * cn[c0 + c] / tabs(pv)) l = T(0);
        W[r * ldw + c] = l;
        for (int q = c + 1; q < DD_NB; ++q) {
          T u = W[pr * ldw + q];
          if (c0 + q < n && tabs(u) < tau * cn[c0 + q]) u = T(0);
          W[r * ldw + q] -= l * u;
        }
      } else {
        W[r * ldw + c] = l;
        for (int q = c + 1; q < DD_NB; ++q) W[r * ldw + q] -= l * W[pr * ldw + q];
      }
    }
    if (r == pr) { chosen = true; L = c; }
    else if (L == c) { L = j; }
    if (c + 1 < nbe) {
      const int lastn = min(min(R - 1, c + 1 + kl), n - 1 - c0);
      T v = T(-1);
      if (own && !chosen && r <= lastn) {
        v = tabs(W[r * ldw + c + 1]);
        if (!(v == v)) v = T(-1);
      }
      offer_max(v, (own && !chosen) ? L : INT_MAX, r, bv, bL, br, (c + 1) & 1);
    }
  }
  __syncthreads();  // every update and the exchange list are done
  for (int q = tid; q < Cw; q += blockDim.x)
    for (int c = 0; c < nbe; ++c) {
      const int j = sj[c];
      if (j != c) {
        const T t = W[c * ldw + q];
        W[c * ldw + q] = W[j * ldw + q];
        W[j * ldw + q] = t;
      }
    }
  __syncthreads();
  return true;
}

template <typename T>
__device__ void band_lu_task(const BandInfo &b, int task, T *band, T *ltraw, int32_t *piv, T *W,
                             double pivtol, DevStatus *st, T *cnorm, T tau) {
  const int n = b.n, kl = b.kl, ku = b.ku, wd = 2 * kl + ku + 1;
  const int R = DD_NB + kl, Cw = DD_NB + kl + ku, ldw = lu_ldw(kl, ku);
  T *A = band + b.band_off;
  int32_t *P = piv + b.piv_off;
  __shared__ T red[32];
  __shared__ int32_t s_p;
  __shared__ int32_t s_fail;
  __shared__ T s_amax;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

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
  // the incomplete factorisation's reference: the 2-norm of every column of
  // the unfactored block (rows ascending; band row i holds column j at
  // offset j - i + kl)
  const T *cn = tau > T(0) ? cnorm + b.row0 : nullptr;
  if (tau > T(0)) {
    for (int j = tid; j < n; j += nt) {
      T sq = T(0);
      for (int i = max(0, j - ku); i <= min(n - 1, j + kl); ++i) {
        const T v = A[(int64_t)i * wd + (j - i + kl)];
        sq += v * v;
      }
      cnorm[b.row0 + j] = sqrt(sq);
    }
    __syncthreads();
  }

  // In shared memory the window slides: the part of panel t's window that
  // panel t + 1 still needs (rows and columns NB on) moves up and left by NB,
  // and only the NB new rows and columns come from the band.  The values a
  // reload would bring are the same: every update stays inside the band.
  const bool slide = __isShared(W);
  for (int t = 0; t < b.ntiles; ++t) {
    const int c0 = t * DD_NB;
    const int nbe = min(DD_NB, n - c0);
    // load the window.  In shared memory: every element by an asynchronous
    // copy (positions outside the band or the matrix are filled with zeros by
    // a zero source size), all in flight before one wait: the warp-per-row
    // loads below waited ~30 times per panel for a dependent round of loads.
    if (slide) {
      auto load_rect = [&](int ra, int rz, int ca, int cz) {
        for (int r = ra + warp; r < rz; r += nw) {
          const int gr = c0 + r;
          const T *arow = A + (int64_t)min(gr, n - 1) * wd;
          T *wrow = W + r * ldw;
          for (int c = ca + lane; c < cz; c += 32) {
            const int gc = c0 + c, off = c - r + kl;
            const bool ok = gr < n && gc < n && off >= 0 && off < wd;
            const unsigned sa = (unsigned)__cvta_generic_to_shared(wrow + c);
            const T *src = ok ? arow + off : arow;
            if (sizeof(T) == 4)
              asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(src), "r"(ok ? 4 : 0)
                           : "memory");
            else
              asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa), "l"(src), "r"(ok ? 8 : 0)
                           : "memory");
          }
        }
      };
      if (t == 0) {
        load_rect(0, R, 0, Cw);
      } else {
        // rows [0, R - NB) x columns [0, Cw - NB) <- rows [NB, R) x columns
        // [NB, Cw), NB rows at a time: a block's source rows are the next
        // block's destination, which is written after a barrier
        const int sw = Cw - DD_NB;
        for (int rb = 0; rb < R - DD_NB; rb += DD_NB) {
          const int nr = min(DD_NB, R - DD_NB - rb);
          for (int e = tid; e < nr * sw; e += nt) {
            const int r = rb + e / sw, c = e % sw;
            W[r * ldw + c] = W[(r + DD_NB) * ldw + c + DD_NB];
          }
          __syncthreads();
        }
        load_rect(R - DD_NB, R, 0, Cw);          // the new rows
        load_rect(0, R - DD_NB, Cw - DD_NB, Cw);  // the new columns of the others
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
    } else
    // in global scratch: a warp per row, lanes along the row's band entries,
    // four loads in flight per lane
    for (int r = warp; r < R; r += nw) {
      const int gr = c0 + r;
      const T *arow = A + (int64_t)gr * wd;
      T *wrow = W + r * ldw;
      for (int cb = 0; cb < Cw; cb += 128) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = cb + lane + 32 * u, gc = c0 + c, off = c - r + kl;
          v[u] = (c < Cw && gr < n && gc < n && off >= 0 && off < wd) ? arow[off] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = cb + lane + 32 * u;
          if (c < Cw) wrow[c] = v[u];
        }
      }
    }
    __syncthreads();
    // panel: column by column (deferred exchanges when a thread owns each
    // window row, else exchanges as they come)
    if (R <= nt) {
      if (!lu_panel_lazy<T>(W, ldw, R, Cw, c0, n, kl, nbe, thresh, P, st, task, cn, tau)) return;
    } else
    for (int c = 0; c < nbe; ++c) {
      const int last = min(min(R - 1, c + kl), n - 1 - c0);
      if (warp == 0) {
        T best = T(-1);
        int bi = R;
        for (int r = c + lane; r <= last; r += 32) {
          T v = tabs(W[r * ldw + c]);
          if (v > best) { best = v; bi = r; }
        }
        for (int o = 16; o; o >>= 1) {
          T ov = __shfl_xor_sync(0xffffffffu, best, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) {
          s_p = bi;
          P[c0 + c] = c0 + bi;
          if (!(best > thresh)) { s_fail = 1; set_status(st, DD_ERR_SINGULAR_BLOCK, task); }
        }
      }
      __syncthreads();
      if (s_fail) return;
      const int pr = s_p;
      if (pr != c)
        for (int q = tid; q < Cw; q += nt) {
          T tq = W[c * ldw + q]; W[c * ldw + q] = W[pr * ldw + q]; W[pr * ldw + q] = tq;
        }
      __syncthreads();
      const T dkk = W[c * ldw + c];
      for (int r = c + 1 + tid; r <= last; r += nt) {
        T l = W[r * ldw + c] / dkk;
        if (tau > T(0) && tabs(l) < tau * cn[c0 + c] / tabs(dkk)) l = T(0);
        W[r * ldw + c] = l;
        for (int q = c + 1; q < DD_NB; ++q) {
          T u = W[c * ldw + q];
          if (tau > T(0) && c0 + q < n && tabs(u) < tau * cn[c0 + q]) u = T(0);
          W[r * ldw + q] -= l * u;
        }
      }
      __syncthreads();
    }
    // the incomplete factorisation: the panel's rows of U as its column
    // steps used them (entries below tau times their column's norm dropped)
    if (tau > T(0)) {
      for (int e = tid; e < nbe * DD_NB; e += nt) {
        const int c = e / DD_NB, q = e % DD_NB;
        if (q > c && q < nbe && tabs(W[c * ldw + q]) < tau * cn[c0 + q]) W[c * ldw + q] = T(0);
      }
      __syncthreads();
    }
    // U12 = L11^-1 A12 (rows 0..NB-1, columns NB..Cw-1): one thread per
    // column, forward substitution with the unit lower L11, the column in
    // registers (the L11 entries are the same for every thread).
    if constexpr (sizeof(T) == 4) {
      // in two 16-row blocks, at most 17 live values: x = rows 0..15 solved
      // with L11's leading block; rows 16..31 less their products with x,
      // each a dot product stored at once; then those rows solved with the
      // trailing block
      static_assert(DD_NB == 32, "two 16-row blocks");
      for (int q = DD_NB + tid; q < Cw; q += nt) {
        // the incomplete factorisation: each entry of U12 dropped (below tau
        // times its column's norm) as soon as it is final, before it is used
        const T th = (tau > T(0) && c0 + q < n) ? tau * cn[c0 + q] : T(0);
        T x[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = W[r * ldw + q];
#pragma unroll
        for (int c = 0; c < 15; ++c) {
          if (tabs(x[c]) < th) x[c] = T(0);
#pragma unroll
          for (int r = c + 1; r < 16; ++r)
            if (c < nbe - 1) x[r] -= W[r * ldw + c] * x[c];
        }
        if (tabs(x[15]) < th) x[15] = T(0);
#pragma unroll
        for (int r = 0; r < 16; ++r) W[r * ldw + q] = x[r];
#pragma unroll 1
        for (int r = 16; r < DD_NB; ++r) {
          T acc = W[r * ldw + q];
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c < nbe - 1) acc -= W[r * ldw + c] * x[c];
          W[r * ldw + q] = acc;
        }
        T y[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) y[r] = W[(16 + r) * ldw + q];
#pragma unroll
        for (int c = 0; c < 15; ++c) {
          if (tabs(y[c]) < th) y[c] = T(0);
#pragma unroll
          for (int r = c + 1; r < 16; ++r)
            if (16 + c < nbe - 1) y[r] -= W[(16 + r) * ldw + 16 + c] * y[c];
        }
        if (tabs(y[15]) < th) y[15] = T(0);
#pragma unroll
        for (int r = 0; r < 16; ++r) W[(16 + r) * ldw + q] = y[r];
      }
    } else {
      for (int q = DD_NB + tid; q < Cw; q += nt) {
        const T th = (tau > T(0) && c0 + q < n) ? tau * cn[c0 + q] : T(0);
        T x[DD_NB];
#pragma unroll
        for (int r = 0; r < DD_NB; ++r) x[r] = W[r * ldw + q];
#pragma unroll
        for (int c = 0; c < DD_NB - 1; ++c) {
          if (tabs(x[c]) < th) x[c] = T(0);
#pragma unroll
          for (int r = c + 1; r < DD_NB; ++r)
            if (c < nbe - 1) x[r] -= W[r * ldw + c] * x[c];
        }
        if (tabs(x[DD_NB - 1]) < th) x[DD_NB - 1] = T(0);
#pragma unroll
        for (int r = 0; r < DD_NB; ++r) W[r * ldw + q] = x[r];
      }
    }
    __syncthreads();
    // A22 -= L21 U12 (rows NB..R-1, columns NB..Cw-1): each thread 4 rows by
    // 4 columns a quarter of the width apart, so neighbouring threads read
    // neighbouring columns
    {
      const int nr = kl, ncol = Cw - DD_NB;
      const int tr = (nr + 3) / 4, qw = (ncol + 3) / 4;
      for (int m = tid; m < tr * qw; m += nt) {
        const int i0 = DD_NB + 4 * (m / qw), jc = DD_NB + (m % qw);
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c2 = 0; c2 < 4; ++c2) acc[a][c2] = T(0);
        for (int k = 0; k < nbe; ++k) {
          T lv[4], uv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) lv[a] = W[(i0 + a) * ldw + k];
#pragma unroll
          for (int c2 = 0; c2 < 4; ++c2) uv[c2] = W[k * ldw + jc + c2 * qw];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) acc[a][c2] += lv[a] * uv[c2];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c2 = 0; c2 < 4; ++c2) W[(i0 + a) * ldw + jc + c2 * qw] -= acc[a][c2];
      }
    }
    __syncthreads();
    // multipliers of the panel (strictly below the diagonal), then the window
    // back to the band rows (multiplier positions zero)
    T *lt = ltraw + b.lraw_off + (int64_t)t * bi_lraw_elems(b);
    for (int c = warp; c < DD_NB; c += nw)  // column c of the multipliers
      for (int r = lane; r < R; r += 32) lt[(int64_t)c * R + r] = (r > c && c < nbe) ? W[r * ldw + c] : T(0);
    // (sliding window: the panel's NB rows are final; the whole band row,
    // with zeros where the multipliers of earlier panels were)
    for (int r = warp; r < (slide ? DD_NB : R); r += nw) {
      const int gr = c0 + r;
      if (gr >= n) continue;
      T *arow = A + (int64_t)gr * wd;
      const T *wrow = W + r * ldw;
      if (slide) {
        for (int off = lane; off < wd; off += 32) {
          const int gc = gr - kl + off, c = gc - c0;
          if (gc >= 0 && gc < n) arow[off] = (c < 0 || (c < DD_NB && r > c)) ? T(0) : wrow[c];
        }
        continue;
      }
      for (int c = lane; c < Cw; c += 32) {
        const int gc = c0 + c, off = c - r + kl;
        if (gc < n && off >= 0 && off < wd) arow[off] = (c < DD_NB && r > c) ? T(0) : wrow[c];
      }
    }
    __syncthreads();
  }
}

// Every subdomain of the CTA's task list (or subdomain blockIdx.x); the
// window sits in shared memory when it fits the launch's smem_bytes, else in
// wscratch (wscratch_stride elements per subdomain).
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256, 1) band_lu_kernel(const BandInfo *__restrict__ info, T *band, T *ltraw, int32_t *piv,
                               T *wscratch, int64_t wscratch_stride, int smem_bytes, double pivtol,
                               const int32_t *__restrict__ sched, const int32_t *__restrict__ sched_off,
                               DevStatus *st, T *cnorm, T tau) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const int t0 = sched_off ? sched_off[blockIdx.x] : (int)blockIdx.x;
  const int t1 = sched_off ? sched_off[blockIdx.x + 1] : (int)blockIdx.x + 1;
  for (int it = t0; it < t1; ++it) {
    const int task = sched ? sched[it] : it;
    const BandInfo b = info[task];
    if (b.n == 0) continue;
    const int64_t wb = lu_window_elems(b.kl, b.ku) * (int64_t)sizeof(T);
    T *W = (wb <= smem_bytes) ? reinterpret_cast<T *>(smraw) : wscratch + (int64_t)task * wscratch_stride;
    __syncthreads();  // the previous task is done with the window and the shared scalars
    band_lu_task<T>(b, task, band, ltraw, piv, W, pivtol, st, cnorm, tau);
  }
}

// ---------------------------------------------------------------------------
// Tile widths, one warp per (subdomain, tile):
//   wl = rows of the forward window that the panel touches: the last
//        nonzero multiplier row of any of its columns, and every pivot row,
//        at least NB, rounded up to 4;
//   wu = NB + the columns right of the panel that its U rows reach, rounded
//        up to 4.
// The host combines the two panels of a sweep tile.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void tile_widths_kernel(const BandInfo *__restrict__ info, const T *__restrict__ band,
                                   const T *__restrict__ lraw, const int32_t *__restrict__ piv,
                                   int32_t *wl, int32_t *wu) {
  const BandInfo b = info[blockIdx.x];
  const int t = blockIdx.y;  // LU panel
  if (t >= b.ntiles) return;
  const int n = b.n, kl = b.kl, wd = 2 * b.kl + b.ku + 1, W = DD_NB + kl;
  const int c0 = t * DD_NB, lane = threadIdx.x;
  int el = DD_NB - 1, eu = -1;
  const int c = c0 + lane;
  if (c < n) {
    const T *col = lraw + b.lraw_off + (int64_t)t * bi_lraw_elems(b) + (int64_t)lane * W;
    for (int q = W - 1; q > lane; --q)
      if (col[q] != T(0)) { el = max(el, q); break; }
    el = max(el, piv[b.piv_off + c] - c0);
    const T *row = band + b.band_off + (int64_t)c * wd;
    for (int off = wd - 1; off >= kl; --off)
      if (row[off] != T(0)) { eu = (c + off - kl) - (c0 + DD_NB); break; }
  }
  for (int o = 16; o; o >>= 1) {
    el = max(el, __shfl_xor_sync(0xffffffffu, el, o));
    eu = max(eu, __shfl_xor_sync(0xffffffffu, eu, o));
  }
  if (lane == 0) {
    wl[b.panel0 + t] = round4(el + 1);
    wu[b.panel0 + t] = round4(DD_NB + max(eu + 1, 0));
  }
}

// ---------------------------------------------------------------------------
// Packed sweep tiles: TB threads per (subdomain, tile); thread c is tile
// column c (forward) and tile row c (backward).
// ---------------------------------------------------------------------------
template <typename T, int TB>
__global__ void __launch_bounds__(4 * TB) band_tiles_kernel(const BandInfo *__restrict__ info,
                                                           const TileMeta *__restrict__ tm,
                                                           const T *__restrict__ band,
                                                           const T *__restrict__ lraw,
                                                           const int32_t *__restrict__ piv, T *ltile,
                                                           T *utile, int32_t *srcs) {
  const BandInfo b = info[blockIdx.x];
  const int t = blockIdx.y;
  if (t >= b.nst) return;
  const TileMeta mt = tm[b.tile0 + t];
  const int n = b.n, kl = b.kl, ku2 = b.kl + b.ku, wd = 2 * b.kl + b.ku + 1;
  const int W = DD_NB + kl;   // window of one LU panel
  const int W2 = TB + kl;  // window of the tile
  const int WL = mt.wl, WU = mt.wu;
  const int c0 = t * TB;
  // thread (tid, part): column / row tid of the tile, one of four parts of
  // the long loops; the triangles are part 0's
  const int tid = threadIdx.x % TB, part = threadIdx.x / TB;
  const int cend = min(c0 + TB, n);
  const int32_t *P = piv + b.piv_off;
  const T *A = band + b.band_off;
  T *K = ltile + mt.lofs;
  T *Kb = utile + mt.uofs;
  int32_t *src = srcs + mt.sofs;
  extern __shared__ __align__(128) unsigned char smraw[];
  T *L11 = reinterpret_cast<T *>(smraw);    // TB x TB
  T *vbuf = L11 + TB * TB;            // TB columns x W2
  T *Lsm = vbuf + (size_t)TB * W2;       // TB x TB
  int32_t *idx = reinterpret_cast<int32_t *>(Lsm + TB * TB);

  // (1) composite window permutation of all the tile's row exchanges
  if (threadIdx.x == 0) {
    for (int q = 0; q < W2; ++q) idx[q] = q;
    for (int c = c0; c < cend; ++c) {
      const int a = c - c0, bq = P[c] - c0;
      const int tmp = idx[a]; idx[a] = idx[bq]; idx[bq] = tmp;
    }
  }
  // (2) multipliers of column tid in the tile's final row order: the panel's
  // own (already exchanged), then the exchanges of the tile's later panels
  if (part == 0) {
    T *v = vbuf + (size_t)tid * W2;
    for (int q = 0; q < W2; ++q) v[q] = T(0);
    const int pr = tid / DD_NB, cc = tid % DD_NB, po = pr * DD_NB;
    const int pnl = t * (TB / DD_NB) + pr;
    if (pnl < b.ntiles) {
      const T *lr = lraw + b.lraw_off + (int64_t)pnl * bi_lraw_elems(b) + (int64_t)cc * W;
      for (int q = 0; q < W; ++q) v[po + q] = lr[q];
    }
    for (int c2 = c0 + po + DD_NB; c2 < cend; ++c2) {
      const int a = c2 - c0, bq = P[c2] - c0;
      const T tmp = v[a]; v[a] = v[bq]; v[bq] = tmp;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < src_stride_w(WL); q += 4 * TB) src[q] = (q < W2) ? idx[q] : q;
  for (int q = part; q < TB; q += 4)
    L11[q * TB + tid] = (q == tid) ? T(1) : (q > tid ? vbuf[(size_t)tid * W2 + q] : T(0));
  __syncthreads();
  // (3) Linv (column tid), then K = [Linv; -L21 Linv] for rows < WL
  if (part == 0) {
    T x[TB];
    for (int q = 0; q < TB; ++q) x[q] = T(0);
    x[tid] = T(1);
    for (int q = tid + 1; q < TB; ++q) {
      T sacc = T(0);
      for (int r = tid; r < q; ++r) sacc += L11[q * TB + r] * x[r];
      x[q] = -sacc;
    }
    for (int q = 0; q < TB; ++q) {
      K[kidx<T, TB>(q, tid)] = x[q];
      Lsm[q * TB + tid] = x[q];
    }
  }
  __syncthreads();
  for (int r = TB + part; r < WL; r += 4) {
    T sacc = T(0);
    if (r < W2)
      for (int k = 0; k < TB; ++k) sacc += vbuf[(size_t)k * W2 + r] * Lsm[k * TB + tid];
    K[kidx<T, TB>(r, tid)] = -sacc;
  }
  __syncthreads();
  // (4) U11 (row-major in L11's buffer) and its inverse; Kb = [Uinv | -Uinv U12]
  {
    const int r = c0 + tid;  // row of this thread
    for (int c = part; c < TB; c += 4) {
      T v = T(0);
      if (r < n) {
        const int col = c0 + c, off = col - r + kl;
        if (c >= tid && col < n && off < wd) v = A[(int64_t)r * wd + off];
      } else if (c == tid) {
        v = T(1);
      }
      L11[tid * TB + c] = v;
    }
  }
  __syncthreads();
  if (part == 0) {
    T x[TB];
    for (int q = 0; q < TB; ++q) x[q] = T(0);
    x[tid] = T(1) / L11[tid * TB + tid];
    for (int q = tid - 1; q >= 0; --q) {
      T sacc = T(0);
      for (int r = q + 1; r <= tid; ++r) sacc += L11[q * TB + r] * x[r];
      x[q] = -sacc / L11[q * TB + q];
    }
    for (int q = 0; q < TB; ++q) Lsm[q * TB + tid] = x[q];  // Uinv(q, tid)
  }
  __syncthreads();
  {
    T *kr = Kb + (int64_t)tid * WU;
    for (int c = part; c < TB; c += 4) kr[c] = Lsm[tid * TB + c];
  }
  // -Uinv U12 as a product in chunks of TB columns of U12: Uinv transposed
  // into L11's buffer (UT[k][r] = Uinv(r, k)), the chunk of U12 (TB rows,
  // zero outside the band and the matrix) staged in vbuf (TB x TB fits its
  // TB x W2); each thread accumulates 4 rows x CW = TB / 16 columns in
  // registers over k in ascending order (Uinv's zeros below the diagonal add
  // exact zeros first, so every output is the same chain as a sum from k =
  // its row)
  constexpr int CW = TB / 16;
  T *UT = L11;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) UT[e] = Lsm[(e % TB) * TB + e / TB];
  const int ri = threadIdx.x / 16, qi = threadIdx.x % 16;  // rows 4 ri.., columns CW qi.. of a chunk
  for (int q0 = 0; q0 < WU - TB; q0 += TB) {
    __syncthreads();  // UT is written; the previous chunk is consumed
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
      const int k = e / TB, q = q0 + e % TB, col = c0 + TB + q, rk = c0 + k;
      const int off = col - rk + kl;
      vbuf[e] = (rk < n && col < n && q < ku2 && off < wd) ? A[(int64_t)rk * wd + off] : T(0);
    }
    __syncthreads();
    T acc[4][CW];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < CW; ++y) acc[x][y] = T(0);
#pragma unroll 4
    for (int k = 0; k < TB; ++k) {
      T u[4], v[CW];
      ld4(UT + k * TB + 4 * ri, u);
#pragma unroll
      for (int y = 0; y < CW; ++y) v[y] = vbuf[k * TB + CW * qi + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < CW; ++y) acc[x][y] += u[x] * v[y];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < CW; ++y) {
        const int q = q0 + CW * qi + y;
        if (q < WU - TB) Kb[(int64_t)(4 * ri + x) * WU + TB + q] = -acc[x][y];
      }
  }
}

// ---------------------------------------------------------------------------
// Single right-hand side sweeps (the apply).  One CTA per subdomain keeps the
// right-hand side in shared memory; the tiles stream through a ring of
// shared-memory stages filled by TMA bulk copies (cp.async.bulk, completion
// on an mbarrier).  A job is a run of consecutive tiles of one sweep packed
// into one copy (a copy's fixed cost is amortised only by copies of tens of
// kilobytes); forward jobs, then backward jobs, form one sequence, so the
// copy of job q+S overlaps the arithmetic of job q.  Every wait on an
// mbarrier is bounded; on expiry the CTA records DD_ERR_TIMEOUT, drains its
// own copies (bounded again) and returns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
#define DD_WAIT_LIMIT (1u << 22)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint32_t limit = DD_WAIT_LIMIT) {
  limit = min(limit, DD_WAIT_LIMIT);
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// job q of subdomain b (forward jobs first), tiles [lo, hi)
__device__ __forceinline__ SweepJob get_job(const BandInfo &b, const SweepJob *jobs, int q, bool &fwd) {
  fwd = q < b.njf;
  return jobs[fwd ? b.jf0 + q : b.jb0 + (q - b.njf)];
}

// Bytes of CTA `rank`'s slice of tile mt in a cluster of CL CTAs: forward,
// its K rows then the tile's whole src; backward, its Kb rows.
template <typename T, int TB, int CL>
__device__ __forceinline__ uint32_t slice_bytes(const TileMeta &mt, bool fwd, int rank) {
  if (fwd)
    return (uint32_t)((fwd_split(mt.wl, rank + 1, CL) - fwd_split(mt.wl, rank, CL)) * TB * sizeof(T) +
                      src_stride_w(mt.wl) * sizeof(int32_t));
  return (uint32_t)((TB / CL) * mt.wu * sizeof(T));
}

// One job into its stage.  CL = 1: the job's tiles are contiguous in the
// packed arrays, one copy for K (or Kb) and one for src.  CL = 2: the CTA's
// slices only, tile by tile (forward in ascending, backward in descending
// tile order, the order they are used), all on the stage's mbarrier.
// DD_CHECKED: a copy whose global address or size is not a multiple of 16
// bytes, or that would run past its stage, is not issued (its wait then
// gives up and the sweep stops).
__device__ __forceinline__ void bulk_g2s_checked(unsigned char *stage, uint32_t off, const void *src,
                                                 uint32_t bytes, uint32_t stage_bytes, uint64_t *bar,
                                                 DevStatus *st) {
  const bool ok = dd_check(st, ((uintptr_t)src & 15) == 0, 11) && dd_check(st, (bytes & 15) == 0, 12) &&
                  dd_check(st, (uint64_t)off + bytes <= stage_bytes, 13);
  if (ok) bulk_g2s(stage + off, src, bytes, bar);
}

template <typename T, int TB, int CL = 1>
__device__ __forceinline__ void issue_job(const BandInfo &b, const TileMeta *tm, const SweepJob *jobs,
                                          int q, const T *ltile, const T *utile, const int32_t *srcs,
                                          unsigned char *stage, uint64_t *bar, int rank, uint32_t stage_bytes,
                                          DevStatus *st, const unsigned char *cld = nullptr) {
  bool fwd;
  const SweepJob jb = get_job(b, jobs, q, fwd);
  const TileMeta &a = tm[b.tile0 + jb.lo];
  if (CL > 1) {
    // the job's slices of this CTA are contiguous in the cluster layout
    // (forward ascending, backward descending): one copy
    uint32_t tot = 0;
    for (int t = jb.lo; t < jb.hi; ++t) tot += slice_bytes<T, TB, CL>(tm[b.tile0 + t], fwd, rank);
    const int64_t o = fwd ? tm[b.tile0 + jb.lo].cfo[rank] : tm[b.tile0 + jb.hi - 1].cbo[rank];
    mbar_expect_tx(bar, tot);
    bulk_g2s_checked(stage, 0, cld + o, tot, stage_bytes, bar, st);
    return;
  }
  if (fwd) {
    const TileMeta &z = tm[b.tile0 + jb.hi - 1];
    const uint32_t lb = (uint32_t)((z.lofs + (int64_t)z.wl * TB - a.lofs) * sizeof(T));
    const uint32_t sb = (uint32_t)((z.sofs + src_stride_w(z.wl) - a.sofs) * sizeof(int32_t));
    mbar_expect_tx(bar, lb + sb);
    bulk_g2s_checked(stage, 0, ltile + a.lofs, lb, stage_bytes, bar, st);
    bulk_g2s_checked(stage, lb, srcs + a.sofs, sb, stage_bytes, bar, st);
  } else {
    const TileMeta &z = tm[b.tile0 + jb.hi - 1];
    const uint32_t ub = (uint32_t)((z.uofs + (int64_t)TB * z.wu - a.uofs) * sizeof(T));
    mbar_expect_tx(bar, ub);
    bulk_g2s_checked(stage, 0, utile + a.uofs, ub, stage_bytes, bar, st);
  }
}

// The bytes of job q (CL = 1 layout) into L2, without a destination in
// shared memory; a hint that changes no result.  The addresses and sizes are
// those its copy will use, so they are in bounds and 16-byte aligned.
template <typename T, int TB>
__device__ __forceinline__ void prefetch_job(const BandInfo &b, const TileMeta *tm, const SweepJob *jobs, int q,
                                             const T *ltile, const T *utile, const int32_t *srcs) {
  bool fwd;
  const SweepJob jb = get_job(b, jobs, q, fwd);
  const TileMeta &a = tm[b.tile0 + jb.lo], &z = tm[b.tile0 + jb.hi - 1];
  const void *p0, *p1 = nullptr;
  uint32_t n0, n1 = 0;
  if (fwd) {
    p0 = ltile + a.lofs;
    n0 = (uint32_t)((z.lofs + (int64_t)z.wl * TB - a.lofs) * sizeof(T));
    p1 = srcs + a.sofs;
    n1 = (uint32_t)((z.sofs + src_stride_w(z.wl) - a.sofs) * sizeof(int32_t));
  } else {
    p0 = utile + a.uofs;
    n0 = (uint32_t)((z.uofs + (int64_t)TB * z.wu - a.uofs) * sizeof(T));
  }
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p0), "r"(n0) : "memory");
  if (n1) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p1), "r"(n1) : "memory");
}

// 16-byte chunk of T values
template <typename T>
struct Chunk;
template <>
struct Chunk<float> {
  using V = float4;
  static constexpr int N = 4;
  // acc + a . b as a chain of fused multiply-adds
  __device__ static float fmadd(const float4 &a, const float4 &b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
  }
};
template <>
struct Chunk<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static double fmadd(const double2 &a, const double2 &b, double acc) {
    acc = fma(a.x, b.x, acc);
    return fma(a.y, b.y, acc);
  }
};

// The first nstages jobs of a task into their stages (thread 0); the stages
// were last read by generic loads of the previous task.
template <typename T, int TB, int CL = 1>
__device__ __forceinline__ void issue_first_jobs(const BandInfo &b, const TileMeta *tm, const SweepJob *jobs,
                                                 const T *ltile, const T *utile, const int32_t *srcs,
                                                 unsigned char *ring, uint32_t stage_bytes, int nstages,
                                                 uint64_t *bars, uint32_t jbase, int rank, DevStatus *st,
                                                 int pf = 0, const unsigned char *cld = nullptr) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int nj = b.njf + b.njb;
  for (int q = 0; q < nstages && q < nj; ++q) {
    const int sq = (int)((jbase + q) % nstages);
    issue_job<T, TB, CL>(b, tm, jobs, q, ltile, utile, srcs, ring + (size_t)sq * stage_bytes, &bars[sq], rank,
                         stage_bytes, st, cld);
  }
  if (CL == 1)
    for (int q = nstages; q < nstages + pf && q < nj; ++q) prefetch_job<T, TB>(b, tm, jobs, q, ltile, utile, srcs);
}

// Forward sweep in place over vec, backward sweep from vec into xout (both in
// shared memory, length >= ntiles*NB + pad, xout zero beyond the tiles).
// Returns false if a wait expired.
template <typename T, int TB>
__device__ bool sweep_pipelined(const BandInfo &b, const TileMeta *__restrict__ tm,
                                const SweepJob *__restrict__ jobs, const T *__restrict__ ltile,
                                const T *__restrict__ utile, const int32_t *__restrict__ srcs,
                                T *vec, T *xout, T *win, unsigned char *ring,
                                uint32_t stage_bytes, int nstages, uint64_t *bars,
                                uint32_t &jbase, int task, bool issued, DevStatus *st,
                                uint32_t first_wait, int wext, int vext, int pf) {
  using CV = typename Chunk<T>::V;
  constexpr int CN = Chunk<T>::N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nj = b.njf + b.njb;
  // job q of this task is job jbase + q of the CTA: its stage and phase
  if (tid == 0 && !issued) issue_first_jobs<T, TB>(b, tm, jobs, ltile, utile, srcs, ring, stage_bytes, nstages, bars, jbase, 0, st, pf);
  bool ok = true;
  int q = 0;
  for (; q < nj; ++q) {
    const uint32_t gq = jbase + q;
    const int sidx = (int)(gq % nstages);
    unsigned char *stage = ring + (size_t)sidx * stage_bytes;
    // every thread waits (bounded); the outcome is made uniform at the
    // first barrier of the job, so no thread can leave the loop alone
    // (the CTA's first wait may be shortened by the timeout test hook; the
    // drain below always takes the full bound)
    const bool got = mbar_wait_bounded(&bars[sidx], (gq / nstages) & 1u, gq == 0 ? first_wait : DD_WAIT_LIMIT);
    bool fwd;
    const SweepJob jb = get_job(b, jobs, q, fwd);
    const TileMeta &a = tm[b.tile0 + jb.lo];
    if (fwd) {
      const TileMeta &z = tm[b.tile0 + jb.hi - 1];
      const size_t kbytes = (size_t)(z.lofs + (int64_t)z.wl * TB - a.lofs) * sizeof(T);
      for (int t = jb.lo; t < jb.hi; ++t) {
        // forward tile t: w <- [0; w_B] + K w_T on the exchanged window
        const TileMeta &mt = tm[b.tile0 + t];
        const int c0 = t * TB, WL = mt.wl;
        const T *K = reinterpret_cast<const T *>(stage + (mt.lofs - a.lofs) * sizeof(T));
        const int32_t *src = reinterpret_cast<const int32_t *>(stage + kbytes) + (mt.sofs - a.sofs);
        // (DD_CHECKED: the window fits win and vec, every source row is inside it)
        const bool wok = dd_check(st, WL <= wext && c0 + WL <= vext, 21);
        if (got && wok)
          for (int e = tid; e < WL; e += nt)
            if (dd_check(st, (unsigned)src[e] < (unsigned)WL, 22)) win[e] = vec[c0 + src[e]];
        if (!__syncthreads_and(got && wok)) { ok = false; break; }
        for (int r = tid; r < WL; r += nt) {
          const CV *kr = reinterpret_cast<const CV *>(K + r * TB);
          const CV *wv = reinterpret_cast<const CV *>(win);
          T a0 = (r < TB) ? T(0) : win[r], a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
          for (int ch = 0; ch < TB / CN; ch += 4) {
            a0 = Chunk<T>::fmadd(kr[ch ^ (r & 7)], wv[ch], a0);
            a1 = Chunk<T>::fmadd(kr[(ch + 1) ^ (r & 7)], wv[ch + 1], a1);
            a2 = Chunk<T>::fmadd(kr[(ch + 2) ^ (r & 7)], wv[ch + 2], a2);
            a3 = Chunk<T>::fmadd(kr[(ch + 3) ^ (r & 7)], wv[ch + 3], a3);
          }
          vec[c0 + r] = (a0 + a1) + (a2 + a3);
        }
        __syncthreads();
      }
      if (!ok) break;
    } else {
      for (int t = jb.hi - 1; t >= jb.lo; --t) {
        // backward tile t: x_T = Kb [b_T; x_next]; 8 threads per output row;
        // the outputs xout[r0..r0+TB) never overlap this tile's inputs
        const TileMeta &mt = tm[b.tile0 + t];
        const int r0 = t * TB, WU = mt.wu, nch = WU / CN;
        const T *Kb = reinterpret_cast<const T *>(stage + (mt.uofs - a.uofs) * sizeof(T));
        const int i = tid >> 3, h = tid & 7;
        T acc = T(0);
        const bool bok = dd_check(st, r0 + WU <= vext, 23);
        if (got && bok) {
          const CV *kr = reinterpret_cast<const CV *>(Kb + (int64_t)i * WU);
          const CV *bv = reinterpret_cast<const CV *>(vec + r0);
          const CV *xv = reinterpret_cast<const CV *>(xout + r0);
          T a0 = T(0), a1 = T(0);
          int ch = h;
          for (; ch < TB / CN; ch += 8) a0 = Chunk<T>::fmadd(kr[ch], bv[ch], a0);
          for (; ch + 8 < nch; ch += 16) {
            a0 = Chunk<T>::fmadd(kr[ch], xv[ch], a0);
            a1 = Chunk<T>::fmadd(kr[ch + 8], xv[ch + 8], a1);
          }
          if (ch < nch) a0 = Chunk<T>::fmadd(kr[ch], xv[ch], a0);
          acc = a0 + a1;
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (h == 0) xout[r0 + i] = acc;
        if (!__syncthreads_and(got && bok)) { ok = false; break; }
      }
      if (!ok) break;
    }
    // the stage is free; vec / xout are current
    if (tid == 0 && q + nstages < nj) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_job<T, TB>(b, tm, jobs, q + nstages, ltile, utile, srcs, stage, &bars[sidx], 0, stage_bytes, st);
      if (pf > 0 && q + nstages + pf < nj) prefetch_job<T, TB>(b, tm, jobs, q + nstages + pf, ltile, utile, srcs);
    }
  }
  if (!ok) {
    if (tid == 0) {
      if (atomicCAS(&st->code, 0, (int)DD_ERR_TIMEOUT) == 0) st->block = task;
    }
    // drain the copies still in flight (jobs q .. q+nstages-1, one per
    // stage), bounded
    const int last_issued = min(nj - 1, q + nstages - 1);
    for (int j = q; j <= last_issued; ++j) {
      const uint32_t gj = jbase + j;
      mbar_wait_bounded(&bars[gj % nstages], (gj / nstages) & 1u);
    }
  }
  jbase += nj;
  return ok;
}

// Barrier of every thread of every CTA of the cluster; the release / acquire
// pair makes the distributed shared-memory stores before it visible after it.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ uint32_t map_peer(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
// one element into the peer CTA's shared memory, counted (bytes) on the
// peer's mbarrier
__device__ __forceinline__ void st_async_peer(uint32_t raddr, float v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(raddr),
               "r"(__float_as_uint(v)), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void st_async_peer(uint32_t raddr, double v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr),
               "l"(__double_as_longlong(v)), "r"(rbar)
               : "memory");
}
// bounded wait on a local mbarrier whose bytes come from the peer CTA
// (acquire at cluster scope, so the peer's stores are visible after it)
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < DD_WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Cluster context of a sweep CTA: its rank and task list index; CL = 2 also
// the message buffers.  Each step s, each CTA sends the peer one message by
// st.async into the peer's buffer xb[s & 1], counted on the peer's mbarrier
// xbar[s & 1]: its flag (1: it had the step's tile bytes and computed its
// rows), then its rows of the step.  Both CTAs know every step's row counts,
// so at step s each arms its own xbar[s & 1] for the peer's message of step
// s (the bytes may arrive before or after the arming).  The phase of step
// s - 2 on that barrier was taken at step s - 1, and the peer sends step s
// only after taking step s - 1, which this CTA sends after taking step s - 2:
// no buffer or barrier phase is overtaken.
template <typename T, int CL>
struct SweepCtx {
  int rank = 0, cid = 0, msg = 0;
  T *xb = nullptr;
  uint64_t *xbar = nullptr;
  uint32_t pxb = 0, pxbar = 0;  // the peer's xb and xbar (shared::cluster addresses)
  uint32_t sstep = 0;
  // lookahead sweeps: messages of earlier tasks in each direction (x from
  // CTA 0, partial sums from CTA 1), tasks finished, and the two task-end
  // flag words (own, and the peer's shared::cluster address)
  uint32_t ubase = 0, vbase = 0, ntask = 0;
  int32_t *okw = nullptr;
  uint32_t pokw = 0;
  __device__ void init(T *xb_, uint64_t *xbar_, int max_kl, int tb) {
    cid = (int)blockIdx.x / CL;
    if (CL > 1) {
      namespace cgx = cooperative_groups;
      rank = (int)cgx::this_cluster().block_rank();
      xb = xb_;
      xbar = xbar_;
      msg = sweep_msg(tb, max_kl);
      if (threadIdx.x == 0) {
        mbar_init(&xbar[0], 1);
        mbar_init(&xbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      pxb = map_peer(smem_u32(xb_), (uint32_t)(rank ^ 1));
      pxbar = map_peer(smem_u32(xbar_), (uint32_t)(rank ^ 1));
      okw = reinterpret_cast<int32_t *>(xbar_ + 2);  // 8 spare bytes after the two message barriers
      pokw = map_peer(smem_u32(okw), (uint32_t)(rank ^ 1));
      cluster_barrier();  // the peer's barriers are set up before any message
    }
  }
  // thread 0: expect the peer's message of step s (its flag and n rows)
  __device__ __forceinline__ void arm(uint32_t s, int n) const {
    if (threadIdx.x == 0) mbar_expect_tx(&xbar[s & 1u], (uint32_t)((n + 1) * sizeof(T)));
  }
  // element e of step s's message (0: the flag, 1 + i: row i) into the
  // peer's buffer
  __device__ __forceinline__ void put(uint32_t s, int e, T v) const {
    const uint32_t q = s & 1u;
    st_async_peer(pxb + (uint32_t)(((int)q * msg + e) * (int)sizeof(T)), v, pxbar + 8u * q);
  }
  // The peer's message of step s (every thread calls it): wait (bounded),
  // its rows into dst[base + lo .. base + hi).  True when it came and
  // carries the peer's flag.
  __device__ bool take(uint32_t s, T *dst, int base, int lo, int hi) {
    const int q = (int)(s & 1u);
    const bool got = __syncthreads_and(mbar_wait_cluster(&xbar[q], (s >> 1) & 1u)) != 0;
    bool pok = false;
    if (got) {
      const T *m = xb + q * msg;
      for (int r = lo + (int)threadIdx.x; r < hi; r += (int)blockDim.x) dst[base + r] = m[1 + r - lo];
      pok = m[0] != T(0);
    }
    __syncthreads();  // every thread has read the message
    return got && pok;
  }
};

// The sweeps of one subdomain split over a 2-CTA cluster.  Each CTA keeps a
// whole copy of vec and xout and streams only its slices of the tiles (half
// the bytes through its shared memory), one contiguous copy per job from
// the cluster layout.  A tile step: take the peer's message of the previous
// step (its rows merged into vec / xout), gather the window, compute the
// CTA's rows, store them locally and send them to the peer.  No cluster
// barrier per step: the only wait is for the peer's previous message.  A
// CTA whose copy wait gives up sends its message with flag 0; the peer stops
// at its next step, and both take the last message sent to them before
// stopping, so none is in flight when the kernel's final cluster barrier
// is reached.  Rows are computed exactly as in the one-CTA sweep, so the
// results are the same bits.
template <typename T, int TB>
__device__ bool sweep_cluster(const BandInfo &b, const TileMeta *__restrict__ tm,
                              const SweepJob *__restrict__ jobs, const unsigned char *__restrict__ cld, T *vec,
                              T *xout, T *win, unsigned char *ring, uint32_t stage_bytes, int nstages,
                              uint64_t *bars, uint32_t &jbase, int task, DevStatus *st, uint32_t first_wait,
                              SweepCtx<T, 2> &cx, int wext, int vext) {
  using CV = typename Chunk<T>::V;
  constexpr int CN = Chunk<T>::N;
  constexpr int CL = 2, BR = TB / CL;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nj = b.njf + b.njb;
  const int rank = cx.rank, XF = cx.msg - 1;  // rows a message holds
  bool ok = true;
  // the peer's message of the last step, still to be taken: into mdst,
  // positions mbase + [mlo, mhi)
  bool pending = false;
  T *mdst = nullptr;
  int mbase = 0, mlo = 0, mhi = 0;
  int q = 0;
  for (; q < nj; ++q) {
    const uint32_t gq = jbase + q;
    const int sidx = (int)(gq % nstages);
    unsigned char *stage = ring + (size_t)sidx * stage_bytes;
    const bool got = mbar_wait_bounded(&bars[sidx], (gq / nstages) & 1u, gq == 0 ? first_wait : DD_WAIT_LIMIT);
    bool fwd;
    const SweepJob jb = get_job(b, jobs, q, fwd);
    uint32_t off = 0;
    for (int u = 0; u < jb.hi - jb.lo; ++u) {
      const int t = fwd ? jb.lo + u : jb.hi - 1 - u;
      const TileMeta &mt = tm[b.tile0 + t];
      const uint32_t s = cx.sstep;
      if (pending) {
        pending = false;
        if (!cx.take(s - 1, mdst, mbase, mlo, mhi)) { ok = false; break; }
      }
      bool cta_ok;
      if (fwd) {
        const int c0 = t * TB, WL = mt.wl;
        const int r0 = fwd_split(WL, rank, CL), r1 = fwd_split(WL, rank + 1, CL);
        const T *K = reinterpret_cast<const T *>(stage + off);
        off += (uint32_t)((r1 - r0) * TB * sizeof(T));
        const int32_t *src = reinterpret_cast<const int32_t *>(stage + off);
        off += (uint32_t)(src_stride_w(WL) * sizeof(int32_t));
        const bool wok = dd_check(st, WL <= wext && c0 + WL <= vext && r1 - r0 <= XF, 31);
        if (got && wok) {
          for (int e = tid; e < TB; e += nt)
            if (dd_check(st, (unsigned)src[e] < (unsigned)WL, 32)) win[e] = vec[c0 + src[e]];
          for (int e = max(r0, TB) + tid; e < r1; e += nt)
            if (dd_check(st, (unsigned)src[e] < (unsigned)WL, 32)) win[e] = vec[c0 + src[e]];
        }
        cx.arm(s, fwd_split(WL, 2 - rank, CL) - fwd_split(WL, 1 - rank, CL));
        cta_ok = __syncthreads_and(got && wok) != 0;
        const int cnt = r1 - r0;
        // element 1 + e of the message is row r0 + e, computed by the
        // thread that sends it; element 0 the flag
        for (int e = tid; e <= cnt; e += nt) {
          T v = T(0);
          if (e < cnt) {
            if (cta_ok) {
              const int r = r0 + e;
              const CV *kr = reinterpret_cast<const CV *>(K + e * TB);
              const CV *wv = reinterpret_cast<const CV *>(win);
              T a0 = (r < TB) ? T(0) : win[r], a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
              for (int ch = 0; ch < TB / CN; ch += 4) {
                a0 = Chunk<T>::fmadd(kr[ch ^ (r & 7)], wv[ch], a0);
                a1 = Chunk<T>::fmadd(kr[(ch + 1) ^ (r & 7)], wv[ch + 1], a1);
                a2 = Chunk<T>::fmadd(kr[(ch + 2) ^ (r & 7)], wv[ch + 2], a2);
                a3 = Chunk<T>::fmadd(kr[(ch + 3) ^ (r & 7)], wv[ch + 3], a3);
              }
              v = (a0 + a1) + (a2 + a3);
              vec[c0 + r] = v;
            }
            cx.put(s, 1 + e, v);
          } else {
            cx.put(s, 0, cta_ok ? T(1) : T(0));
          }
        }
        mdst = vec;
        mbase = c0;
        mlo = fwd_split(WL, 1 - rank, CL);
        mhi = fwd_split(WL, 2 - rank, CL);
      } else {
        // backward tile t: x_T = Kb [b_T; x_next], the CTA's BR rows, 8
        // threads per row; the outputs never overlap this tile's inputs
        const int r0 = t * TB, WU = mt.wu, nch = WU / CN;
        const T *Kb = reinterpret_cast<const T *>(stage + off);
        off += (uint32_t)(BR * WU * sizeof(T));
        const int i = tid >> 3, h = tid & 7;
        const bool bok = dd_check(st, r0 + WU <= vext && BR <= XF, 33);
        cx.arm(s, BR);
        cta_ok = __syncthreads_and(got && bok) != 0;
        T acc = T(0);
        if (cta_ok) {
          const CV *kr = reinterpret_cast<const CV *>(Kb + (int64_t)i * WU);
          const CV *bv = reinterpret_cast<const CV *>(vec + r0);
          const CV *xv = reinterpret_cast<const CV *>(xout + r0);
          T a0 = T(0), a1 = T(0);
          int ch = h;
          for (; ch < TB / CN; ch += 8) a0 = Chunk<T>::fmadd(kr[ch], bv[ch], a0);
          for (; ch + 8 < nch; ch += 16) {
            a0 = Chunk<T>::fmadd(kr[ch], xv[ch], a0);
            a1 = Chunk<T>::fmadd(kr[ch + 8], xv[ch + 8], a1);
          }
          if (ch < nch) a0 = Chunk<T>::fmadd(kr[ch], xv[ch], a0);
          acc = a0 + a1;
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (h == 0) {
          if (cta_ok) xout[r0 + rank * BR + i] = acc;
          cx.put(s, 1 + i, cta_ok ? acc : T(0));
        }
        if (tid == 1) cx.put(s, 0, cta_ok ? T(1) : T(0));
        mdst = xout;
        mbase = r0;
        mlo = (1 - rank) * BR;
        mhi = mlo + BR;
      }
      ++cx.sstep;
      if (!cta_ok) {
        // the peer stops at its next step: take its message of this step
        // (none is then in flight), and stop
        cx.take(s, mdst, mbase, mlo, mhi);
        ok = false;
        break;
      }
      pending = true;
    }
    if (!ok) break;
    // the stage is free once every thread has finished the job's steps
    __syncthreads();
    if (tid == 0 && q + nstages < nj) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_job<T, TB, CL>(b, tm, jobs, q + nstages, nullptr, nullptr, nullptr, stage, &bars[sidx], rank,
                           stage_bytes, st, cld);
    }
  }
  if (ok && pending) {
    pending = false;
    if (!cx.take(cx.sstep - 1, mdst, mbase, mlo, mhi)) ok = false;
  }
  if (!ok) {
    if (tid == 0) {
      if (atomicCAS(&st->code, 0, (int)DD_ERR_TIMEOUT) == 0) st->block = task;
    }
    const int last_issued = min(nj - 1, q + nstages - 1);
    for (int j = q; j <= last_issued; ++j) {
      const uint32_t gj = jbase + j;
      mbar_wait_bounded(&bars[gj % nstages], (gj / nstages) & 1u);
    }
  }
  jbase += nj;
  return ok;
}
// ---------------------------------------------------------------------------
// The lookahead split of one subdomain's sweeps over a 2-CTA cluster.
// CTA 0 runs the forward sweep alone, on the one-CTA tiles: a forward step
// can take pivot rows from anywhere in its window, so splitting its rows
// costs a wait for the peer every step.  The backward step t,
//   x_t = Kb [b_t; x_{t+1}; x_{t+2}; ...],
// is split by columns instead (la_split): CTA 0 takes the columns of b_t and
// x_{t+1} (and more, to balance the bytes), CTA 1 only columns of x_{t+2}
// and beyond, which are final one step before x_{t+1}.  So CTA 1 forms its
// partial sums s_t one step ahead and sends them to CTA 0 (message
// nst - 1 - t, every t); CTA 0 adds them to its own and sends x_t to CTA 1
// (message nst - 1 - t, t >= 2), which needs it for s_{t-2}.  Each side
// waits only for a message the other sent a step earlier.  Every message of
// a task is sent and taken whatever happens (a copy that stayed out, or a
// peer flag of 0, only clears the flag), and the pair decides together at
// the end of each task whether to go on, so no message is in flight when
// either CTA stops.  A CTA takes message k of a direction from slot k & 1
// after taking message k - 2 from it; the peer sends message k only after
// receiving something the CTA sent after that take, so no slot is
// overwritten before it is read.  Each CTA streams its own job list, sized
// by its own slices.  Sums are formed in another order than in the one-CTA
// sweep, so the results agree to rounding, not bit for bit.
// ---------------------------------------------------------------------------
template <typename T, int TB>
__device__ __forceinline__ uint32_t la_bytes(const TileMeta &mt, int rank) {
  return (uint32_t)(TB * la_cols(mt.wu, TB, rank) * sizeof(T));
}

// job q of CTA rank's list into its stage: rank 0 the forward jobs (the
// one-CTA tiles), then its backward slices; rank 1 its backward slices only.
// A job whose slices are all empty copies nothing; its arrival alone
// completes the stage's phase.
template <typename T, int TB>
__device__ __forceinline__ void issue_job_la(const BandInfo &b, const TileMeta *tm, const SweepJob *jobs, int q,
                                             const T *ltile, const int32_t *srcs, const unsigned char *lad,
                                             unsigned char *stage, uint64_t *bar, int rank, uint32_t stage_bytes,
                                             DevStatus *st) {
  if (rank == 0 && q < b.njf) {
    issue_job<T, TB, 1>(b, tm, jobs, q, ltile, nullptr, srcs, stage, bar, 0, stage_bytes, st);
    return;
  }
  const SweepJob jb = jobs[b.jb0 + (rank == 0 ? q - b.njf : q)];
  const TileMeta &a = tm[b.tile0 + jb.lo], &z = tm[b.tile0 + jb.hi - 1];
  const uint32_t tot = (uint32_t)(z.lao[rank] - a.lao[rank]) + la_bytes<T, TB>(z, rank);
  mbar_expect_tx(bar, tot);
  if (tot) bulk_g2s_checked(stage, 0, lad + a.lao[rank], tot, stage_bytes, bar, st);
}

template <typename T, int TB>
__device__ __forceinline__ void issue_first_jobs_la(const BandInfo &b, const TileMeta *tm, const SweepJob *jobs,
                                                    const T *ltile, const int32_t *srcs, const unsigned char *lad,
                                                    unsigned char *ring, uint32_t stage_bytes, int nstages,
                                                    uint64_t *bars, uint32_t jbase, int rank, DevStatus *st) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int nj = rank == 0 ? b.njf + b.njb : b.njb;
  for (int q = 0; q < nstages && q < nj; ++q) {
    const int sq = (int)((jbase + q) % nstages);
    issue_job_la<T, TB>(b, tm, jobs, q, ltile, srcs, lad, ring + (size_t)sq * stage_bytes, &bars[sq], rank,
                        stage_bytes, st);
  }
}

__device__ __forceinline__ int32_t ld_peer_i32(uint32_t raddr) {
  int32_t v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(raddr) : "memory");
  return v;
}

// 16 lanes' partial sums of one output row into every one of them
template <typename T>
__device__ __forceinline__ T sum16(T acc) {
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  acc += __shfl_xor_sync(0xffffffffu, acc, 4);
  acc += __shfl_xor_sync(0xffffffffu, acc, 8);
  return acc;
}

// Forward sweep (CTA 0) and backward sweep (both CTAs) of one subdomain in
// the lookahead split.  vec / xout / win as in the one-CTA sweep; CTA 1's
// xout holds the x it has received.  Returns the pair's combined outcome
// (false: a wait of either CTA expired).
template <typename T, int TB>
__device__ bool sweep_lookahead(const BandInfo &b, const TileMeta *__restrict__ tm,
                                const SweepJob *__restrict__ jobs, const T *__restrict__ ltile,
                                const int32_t *__restrict__ srcs, const unsigned char *__restrict__ lad, T *vec,
                                T *xout, T *win, unsigned char *ring, uint32_t stage_bytes, int nstages,
                                uint64_t *bars, uint32_t &jbase, int task, DevStatus *st, uint32_t first_wait,
                                SweepCtx<T, 2> &cx, int wext, int vext) {
  using CV = typename Chunk<T>::V;
  constexpr int CN = Chunk<T>::N;
  const int tid = threadIdx.x, nt = blockDim.x, rank = cx.rank, nst = b.nst;
  const int nj = rank == 0 ? b.njf + b.njb : b.njb;
  const int i0 = 2 * (tid >> 4), h = tid & 15;  // backward: rows i0, i0 + 1, lane h of their 16
  bool ok = true;    // every copy in time (the same in every thread)
  bool okm = true;   // every message this thread waited for came, flagged by the peer
  bool live = true;  // the ring still copies (false once a copy stayed out twice the bound)
  int qdead = nj;    // the job at which the ring stopped
  for (int q = 0; q < nj; ++q) {
    const uint32_t gq = jbase + q;
    const int sidx = (int)(gq % nstages);
    unsigned char *stage = ring + (size_t)sidx * stage_bytes;
    const uint32_t par = (gq / nstages) & 1u;
    // the first wait may be shortened by the timeout test hook; a second,
    // full one then tells a late copy (the stage may be reused) from a lost
    // one (the ring stops)
    bool w1 = false, w2 = false;
    if (live) {
      w1 = mbar_wait_bounded(&bars[sidx], par, gq == 0 ? first_wait : DD_WAIT_LIMIT);
      w2 = w1 || mbar_wait_bounded(&bars[sidx], par);
    }
    if (!__syncthreads_and(w1)) ok = false;
    const bool have = __syncthreads_and(w2) != 0;
    if (!have && live) {
      live = false;
      qdead = q;
    }
    const bool fwd = rank == 0 && q < b.njf;
    const SweepJob jb = fwd ? jobs[b.jf0 + q] : jobs[b.jb0 + (rank == 0 ? q - b.njf : q)];
    const TileMeta &a = tm[b.tile0 + jb.lo];
    if (fwd) {
      const TileMeta &z = tm[b.tile0 + jb.hi - 1];
      const size_t kbytes = (size_t)(z.lofs + (int64_t)z.wl * TB - a.lofs) * sizeof(T);
      for (int t = jb.lo; t < jb.hi; ++t) {
        // forward tile t: w <- [0; w_B] + K w_T on the exchanged window
        const TileMeta &mt = tm[b.tile0 + t];
        const int c0 = t * TB, WL = mt.wl;
        const T *K = reinterpret_cast<const T *>(stage + (mt.lofs - a.lofs) * sizeof(T));
        const int32_t *src = reinterpret_cast<const int32_t *>(stage + kbytes) + (mt.sofs - a.sofs);
        const bool wok = dd_check(st, WL <= wext && c0 + WL <= vext, 21);
        if (!wok) ok = false;
        const bool run = have && wok;
        if (run)
          for (int e = tid; e < WL; e += nt)
            if (dd_check(st, (unsigned)src[e] < (unsigned)WL, 22)) win[e] = vec[c0 + src[e]];
        __syncthreads();
        if (run)
          for (int r = tid; r < WL; r += nt) {
            const CV *kr = reinterpret_cast<const CV *>(K + r * TB);
            const CV *wv = reinterpret_cast<const CV *>(win);
            T a0 = (r < TB) ? T(0) : win[r], a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
            for (int ch = 0; ch < TB / CN; ch += 4) {
              a0 = Chunk<T>::fmadd(kr[ch ^ (r & 7)], wv[ch], a0);
              a1 = Chunk<T>::fmadd(kr[(ch + 1) ^ (r & 7)], wv[ch + 1], a1);
              a2 = Chunk<T>::fmadd(kr[(ch + 2) ^ (r & 7)], wv[ch + 2], a2);
              a3 = Chunk<T>::fmadd(kr[(ch + 3) ^ (r & 7)], wv[ch + 3], a3);
            }
            vec[c0 + r] = (a0 + a1) + (a2 + a3);
          }
        __syncthreads();
      }
    } else if (rank == 0) {
      for (int t = jb.hi - 1; t >= jb.lo; --t) {
        // backward tile t: CTA 0's columns (b_t, x_{t+1}, ...), each pair
        // of rows by 16 lanes, plus CTA 1's partial sums s_t
        const TileMeta &mt = tm[b.tile0 + t];
        const int r0 = t * TB, WA = la_cols(mt.wu, TB, 0), nch = WA / CN;
        const T *Kb = reinterpret_cast<const T *>(stage + (mt.lao[0] - a.lao[0]));
        const bool bok = dd_check(st, r0 + mt.wu <= vext, 23);
        if (!bok) ok = false;
        T acc0 = T(0), acc1 = T(0);
        if (have && bok) {
          // column c of Kb multiplies b_t (c < TB) or x = xout[r0 + c]
          const CV *k0 = reinterpret_cast<const CV *>(Kb + (int64_t)i0 * WA);
          const CV *k1 = reinterpret_cast<const CV *>(Kb + (int64_t)(i0 + 1) * WA);
          const CV *bv = reinterpret_cast<const CV *>(vec + r0);
          const CV *xv = reinterpret_cast<const CV *>(xout + r0);
          for (int ch = h; ch < nch; ch += 16) {
            const CV w = ch < TB / CN ? bv[ch] : xv[ch];
            acc0 = Chunk<T>::fmadd(k0[ch], w, acc0);
            acc1 = Chunk<T>::fmadd(k1[ch], w, acc1);
          }
        }
        acc0 = sum16(acc0);
        acc1 = sum16(acc1);
        const uint32_t v = cx.vbase + (uint32_t)(nst - 1 - t), u = cx.ubase + (uint32_t)(nst - 1 - t);
        if (tid == 0) cx.arm(v, TB);
        if (h < 2) {
          // s_t straight from the message buffer; x_t out, and to CTA 1
          const int row = i0 + h;
          const bool got = mbar_wait_cluster(&cx.xbar[v & 1u], (v >> 1) & 1u);
          const T *msg = cx.xb + (int)(v & 1u) * cx.msg;
          if (!got || msg[0] == T(0)) okm = false;
          const T x = (h == 0 ? acc0 : acc1) + msg[1 + row];
          xout[r0 + row] = x;
          if (t >= 2) {
            cx.put(u, 1 + row, x);
            if (tid == 0) cx.put(u, 0, (ok && okm) ? T(1) : T(0));
          }
        }
        __syncthreads();  // x_t in xout before the next step reads it
      }
    } else {
      for (int t = jb.hi - 1; t >= jb.lo; --t) {
        // backward tile t, CTA 1's columns (x_{t+2} and beyond): s_t
        const TileMeta &mt = tm[b.tile0 + t];
        const int r0 = t * TB, WS = la_split(mt.wu, TB), WB = mt.wu - WS, nch = WB / CN;
        const T *Kb = reinterpret_cast<const T *>(stage + (mt.lao[1] - a.lao[1]));
        if (t + 2 <= nst - 1) {
          // x_{t+2} into xout, by the threads that copy it
          const uint32_t u = cx.ubase + (uint32_t)(nst - 3 - t);
          if (tid == 0) cx.arm(u, TB);
          if (tid < TB) {
            const bool got = mbar_wait_cluster(&cx.xbar[u & 1u], (u >> 1) & 1u);
            const T *msg = cx.xb + (int)(u & 1u) * cx.msg;
            if (!got || msg[0] == T(0)) okm = false;
            xout[r0 + 2 * TB + tid] = msg[1 + tid];
          }
          __syncthreads();
        }
        const bool bok = dd_check(st, r0 + mt.wu <= vext, 23);
        if (!bok) ok = false;
        T acc0 = T(0), acc1 = T(0);
        if (have && bok) {
          const CV *k0 = reinterpret_cast<const CV *>(Kb + (int64_t)i0 * WB);
          const CV *k1 = reinterpret_cast<const CV *>(Kb + (int64_t)(i0 + 1) * WB);
          const CV *xv = reinterpret_cast<const CV *>(xout + r0 + WS);
          for (int ch = h; ch < nch; ch += 16) {
            const CV w = xv[ch];
            acc0 = Chunk<T>::fmadd(k0[ch], w, acc0);
            acc1 = Chunk<T>::fmadd(k1[ch], w, acc1);
          }
        }
        acc0 = sum16(acc0);
        acc1 = sum16(acc1);
        const uint32_t v = cx.vbase + (uint32_t)(nst - 1 - t);
        if (h < 2) cx.put(v, 1 + i0 + h, h == 0 ? acc0 : acc1);
        if (tid == 0) cx.put(v, 0, (ok && okm) ? T(1) : T(0));
      }
    }
    // the stage is free once every thread has finished the job's steps
    __syncthreads();
    if (tid == 0 && live && q + nstages < nj) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_job_la<T, TB>(b, tm, jobs, q + nstages, ltile, srcs, lad, stage, &bars[sidx], rank, stage_bytes, st);
    }
  }
  if (!live) {
    // the copies still in flight (jobs qdead .. qdead + nstages - 1), bounded
    const int last_issued = min(nj - 1, qdead + nstages - 1);
    for (int j = qdead; j <= last_issued; ++j) {
      const uint32_t gj = jbase + j;
      mbar_wait_bounded(&bars[gj % nstages], (gj / nstages) & 1u);
    }
  }
  ok = __syncthreads_and(ok && okm) != 0;
  if (!ok && tid == 0 && atomicCAS(&st->code, 0, (int)DD_ERR_TIMEOUT) == 0) st->block = task;
  jbase += nj;
  cx.vbase += (uint32_t)nst;
  cx.ubase += (uint32_t)max(nst - 2, 0);
  // the pair's outcome: each CTA's flag into slot ntask & 1, a cluster
  // barrier, the peer's flag read back (a slot is rewritten two tasks later,
  // after a barrier the peer reaches only once it has read it)
  __shared__ int32_t pair_ok;
  const uint32_t slot = cx.ntask & 1u;
  if (tid == 0) cx.okw[slot] = ok ? 1 : 0;
  cluster_barrier();
  if (tid == 0) pair_ok = (ok && ld_peer_i32(cx.pokw + 4u * slot) != 0) ? 1 : 0;
  __syncthreads();
  ++cx.ntask;
  return pair_ok != 0;
}

// shared-memory layout: [bars | vec | xout | win | tile table | job table | ring]
template <typename T, int TB>
__device__ __forceinline__ void carve(unsigned char *smraw, int max_n, int pad, int max_kl,
                                      int max_tiles, int max_jobs, uint64_t *&bars, T *&vec,
                                      T *&xout, T *&win, TileMeta *&tms, SweepJob *&jbs,
                                      unsigned char *&ring, int cl = 1, T **xb = nullptr,
                                      uint64_t **xbar = nullptr) {
  bars = reinterpret_cast<uint64_t *>(smraw);
  if (xbar) *xbar = reinterpret_cast<uint64_t *>(smraw + 32);  // 2 message barriers after <= 4 ring barriers
  vec = reinterpret_cast<T *>(smraw + 64);
  xout = vec + max_n + pad;
  win = xout + max_n + pad;
  if (xb) *xb = win + TB + max_kl + 8;
  size_t used = 64 + sizeof(T) * (2 * ((size_t)max_n + pad) + TB + max_kl + 8 +
                                  (cl > 1 ? 2 * (size_t)sweep_msg(TB, max_kl) : 0));
  used = (used + 15) & ~(size_t)15;
  tms = reinterpret_cast<TileMeta *>(smraw + used);
  used += sizeof(TileMeta) * (size_t)max_tiles;
  jbs = reinterpret_cast<SweepJob *>(smraw + used);
  used += sizeof(SweepJob) * (size_t)max_jobs;
  used = (used + 127) & ~(size_t)127;
  ring = smraw + used;
}

// this subdomain's tile and job tables into shared memory; returns the
// BandInfo with tile0 / jf0 / jb0 rebased onto the local tables
__device__ __forceinline__ BandInfo stage_tables(BandInfo b, const TileMeta *__restrict__ tm,
                                                 const SweepJob *__restrict__ jobs, TileMeta *tms,
                                                 SweepJob *jbs) {
  for (int t = threadIdx.x; t < b.nst; t += blockDim.x) tms[t] = tm[b.tile0 + t];
  for (int q = threadIdx.x; q < b.njf; q += blockDim.x) jbs[q] = jobs[b.jf0 + q];
  for (int q = threadIdx.x; q < b.njb; q += blockDim.x) jbs[b.njf + q] = jobs[b.jb0 + q];
  b.tile0 = 0;
  b.jf0 = 0;
  b.jb0 = b.njf;
  return b;
}

// CTA 1 of a lookahead pair: the tile table and its own backward jobs,
// rebased as its only jobs
__device__ __forceinline__ BandInfo stage_tables_la1(BandInfo b, const TileMeta *__restrict__ tm,
                                                     const SweepJob *__restrict__ jobs, TileMeta *tms,
                                                     SweepJob *jbs) {
  for (int t = threadIdx.x; t < b.nst; t += blockDim.x) tms[t] = tm[b.tile0 + t];
  for (int q = threadIdx.x; q < b.njl; q += blockDim.x) jbs[q] = jobs[b.jl0 + q];
  b.tile0 = 0;
  b.jf0 = 0;
  b.njf = 0;
  b.jb0 = 0;
  b.njb = b.njl;
  b.jl0 = 0;
  return b;
}

__device__ __forceinline__ void init_bars(uint64_t *bars, int nstages) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// Tasks of CTA c: sched[sched_off[c] .. sched_off[c+1]) when a schedule is
// given (more subdomains than resident CTAs), else the one task c.
__device__ __forceinline__ void task_range(const int32_t *sched_off, int &t0, int &t1, int cid) {
  t0 = sched_off ? sched_off[cid] : cid;
  t1 = sched_off ? sched_off[cid + 1] : cid + 1;
}

template <typename T, int TB, int CL, int LA>
__device__ __forceinline__ bool run_sweep(const BandInfo &b, const TileMeta *tm, const SweepJob *jobs,
                                          const T *ltile, const T *utile, const int32_t *srcs,
                                          const unsigned char *cld, T *vec, T *xout, T *win,
                                          unsigned char *ring, uint32_t stage_bytes, int nstages, uint64_t *bars,
                                          uint32_t &jbase, int task, DevStatus *st, uint32_t first_wait,
                                          SweepCtx<T, CL> &cx, int wext, int vext, int pf) {
  if constexpr (CL == 1)
    return sweep_pipelined<T, TB>(b, tm, jobs, ltile, utile, srcs, vec, xout, win, ring, stage_bytes,
                                  nstages, bars, jbase, task, true, st, first_wait, wext, vext, pf);
  else if constexpr (LA)
    return sweep_lookahead<T, TB>(b, tm, jobs, ltile, srcs, cld, vec, xout, win, ring, stage_bytes, nstages, bars,
                                  jbase, task, st, first_wait, cx, wext, vext);
  else
    return sweep_cluster<T, TB>(b, tm, jobs, cld, vec, xout, win, ring, stage_bytes, nstages, bars, jbase, task,
                                st, first_wait, cx, wext, vext);
}

// the first jobs of a task into the ring (thread 0)
template <typename T, int TB, int CL, int LA>
__device__ __forceinline__ void start_task(const BandInfo &b, const TileMeta *tm, const SweepJob *jobs,
                                           const T *ltile, const T *utile, const int32_t *srcs,
                                           const unsigned char *cld, unsigned char *ring, uint32_t stage_bytes,
                                           int nstages, uint64_t *bars, uint32_t jbase, int rank, DevStatus *st,
                                           int pf) {
  if constexpr (LA)
    issue_first_jobs_la<T, TB>(b, tm, jobs, ltile, srcs, cld, ring, stage_bytes, nstages, bars, jbase, rank, st);
  else
    issue_first_jobs<T, TB, CL>(b, tm, jobs, ltile, utile, srcs, ring, stage_bytes, nstages, bars, jbase, rank, st,
                                pf, cld);
}

// z = A_jj^-1 y_j with y gathered from the original numbering.
template <typename T, int TB, int CL, int LA>
__global__ void band_solve_fwd_kernel(const BandInfo *__restrict__ info, int max_n, int max_kl,
                                      int max_ku2, int max_tiles, int max_jobs, int nstages,
                                      uint32_t stage_bytes,
                                      const TileMeta *__restrict__ tm, const SweepJob *__restrict__ jobs,
                                      const T *__restrict__ ltile, const T *__restrict__ utile,
                                      const int32_t *__restrict__ srcs,
                                      const unsigned char *__restrict__ cld, const double *__restrict__ y,
                                      const int32_t *__restrict__ perm, T *z,
                                      const int32_t *__restrict__ sched,
                                      const int32_t *__restrict__ sched_off,
                                      const int32_t *__restrict__ task_sys,
                                      const int32_t *__restrict__ act, DevStatus *st,
                                      uint32_t first_wait, int pf) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const int pad = sweep_pad_hd(max_kl, max_ku2);
  uint64_t *bars; T *vec, *xout, *win; unsigned char *ring;
  TileMeta *tms; SweepJob *jbs;
  T *xb = nullptr;
  uint64_t *xbar = nullptr;
  carve<T, TB>(smraw, max_n, pad, max_kl, max_tiles, max_jobs, bars, vec, xout, win, tms, jbs, ring, CL, &xb,
               &xbar);
  init_bars(bars, nstages);
  SweepCtx<T, CL> cx;
  cx.init(xb, xbar, max_kl, TB);
  int t0, t1;
  task_range(sched_off, t0, t1, cx.cid);
  uint32_t jbase = 0;
  for (int it = t0; it < t1; ++it) {
    const int task = sched ? sched[it] : it;
    const BandInfo bg = info[task];
    if (bg.n == 0 || (act && !act[task_sys[task]])) continue;  // empty, or its system is done
    __syncthreads();  // the previous task's reads of the tables and vectors are done
    const BandInfo b = (LA && cx.rank == 1) ? stage_tables_la1(bg, tm, jobs, tms, jbs)
                                            : stage_tables(bg, tm, jobs, tms, jbs);
    __syncthreads();  // the tables are staged: start the first copies, then gather y
    if (threadIdx.x == 0)
      start_task<T, TB, CL, LA>(b, tms, jbs, ltile, utile, srcs, cld, ring, stage_bytes, nstages, bars, jbase,
                                cx.rank, st, pf);
    const int ntot = b.nst * TB + pad;
    // y gathered through perm: eight indices, then eight values, in flight
    // per thread (a chain of dependent loads per element took ~8 us)
    for (int i0 = threadIdx.x; i0 < ntot; i0 += 8 * blockDim.x) {
      int idx[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * blockDim.x;
        idx[u] = (i < b.n) ? __ldg(&perm[b.row0 + i]) : -1;
      }
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = idx[u] >= 0 ? __ldg(&y[idx[u]]) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < ntot) {
          vec[i] = T(v[u]);
          xout[i] = T(0);
        }
      }
    }
    __syncthreads();
    // a failed sweep stops both CTAs of a cluster at the same step
    if (!run_sweep<T, TB, CL, LA>(b, tms, jbs, ltile, utile, srcs, cld, vec, xout, win, ring, stage_bytes,
                                  nstages, bars, jbase, task, st, first_wait, cx, TB + max_kl + 8, ntot, pf))
      break;
    // both CTAs of a row-split cluster hold the whole result: each writes its
    // share; in the lookahead split CTA 0 holds it
    const int wr = LA ? 0 : cx.rank, wn = LA ? 1 : CL;
    if (wr == cx.rank)
      for (int i = threadIdx.x + wr * blockDim.x; i < b.n; i += wn * blockDim.x) z[b.row0 + i] = xout[i];
  }
  // no CTA of a cluster leaves while its peer may still address its shared
  // memory (every message sent has been taken by then)
  if (CL > 1) cluster_barrier();
}

// x1 = z1 - A_jj^-1 (E z2)_j, scattered to x in the original numbering.
template <typename T, int TB, int CL, int LA>
__global__ void band_solve_bwd_kernel(const BandInfo *__restrict__ info, int max_n, int max_kl,
                                      int max_ku2, int max_tiles, int max_jobs, int nstages,
                                      uint32_t stage_bytes,
                                      const TileMeta *__restrict__ tm, const SweepJob *__restrict__ jobs,
                                      const T *__restrict__ ltile, const T *__restrict__ utile,
                                      const int32_t *__restrict__ srcs,
                                      const unsigned char *__restrict__ cld,
                                      const int32_t *__restrict__ e_ptr,
                                      const int32_t *__restrict__ e_col,
                                      const T *__restrict__ e_val, const T *__restrict__ z2,
                                      const T *__restrict__ z1, const int32_t *__restrict__ perm,
                                      double *x, const int32_t *__restrict__ sched,
                                      const int32_t *__restrict__ sched_off,
                                      const int32_t *__restrict__ task_sys,
                                      const int32_t *__restrict__ act, DevStatus *st,
                                      uint32_t first_wait, int pf) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const int pad = sweep_pad_hd(max_kl, max_ku2);
  uint64_t *bars; T *vec, *xout, *win; unsigned char *ring;
  TileMeta *tms; SweepJob *jbs;
  T *xb = nullptr;
  uint64_t *xbar = nullptr;
  carve<T, TB>(smraw, max_n, pad, max_kl, max_tiles, max_jobs, bars, vec, xout, win, tms, jbs, ring, CL, &xb,
               &xbar);
  init_bars(bars, nstages);
  SweepCtx<T, CL> cx;
  cx.init(xb, xbar, max_kl, TB);
  int t0, t1;
  task_range(sched_off, t0, t1, cx.cid);
  uint32_t jbase = 0;
  for (int it = t0; it < t1; ++it) {
    const int task = sched ? sched[it] : it;
    const BandInfo bg = info[task];
    if (bg.n == 0 || (act && !act[task_sys[task]])) continue;
    __syncthreads();
    const BandInfo b = (LA && cx.rank == 1) ? stage_tables_la1(bg, tm, jobs, tms, jbs)
                                            : stage_tables(bg, tm, jobs, tms, jbs);
    __syncthreads();
    if (threadIdx.x == 0)
      start_task<T, TB, CL, LA>(b, tms, jbs, ltile, utile, srcs, cld, ring, stage_bytes, nstages, bars, jbase,
                                cx.rank, st, pf);
    const int ntot = b.nst * TB + pad;
    // (E z2) of the subdomain's rows: the row bounds of eight rows, then their
    // entries, loaded before use (rows of E hold 0-2 entries)
    for (int i0 = threadIdx.x; i0 < ntot; i0 += 8 * blockDim.x) {
      int k0[8], k1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * blockDim.x;
        k0[u] = (i < b.n) ? __ldg(&e_ptr[b.row0 + i]) : 0;
        k1[u] = (i < b.n) ? __ldg(&e_ptr[b.row0 + i + 1]) : 0;
      }
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        T acc = T(0);
        for (int k = k0[u]; k < k1[u]; ++k) acc += e_val[k] * z2[e_col[k]];
        v[u] = acc;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < ntot) {
          vec[i] = v[u];
          xout[i] = T(0);
        }
      }
    }
    __syncthreads();
    if (!run_sweep<T, TB, CL, LA>(b, tms, jbs, ltile, utile, srcs, cld, vec, xout, win, ring, stage_bytes,
                                  nstages, bars, jbase, task, st, first_wait, cx, TB + max_kl + 8, ntot, pf))
      break;
    const int wr = LA ? 0 : cx.rank, wn = LA ? 1 : CL;
    if (wr == cx.rank)
      for (int i = threadIdx.x + wr * blockDim.x; i < b.n; i += wn * blockDim.x) {
        const int r = b.row0 + i;
        x[perm[r]] = double(z1[r] - xout[i]);
      }
  }
  if (CL > 1) cluster_barrier();
}

// ---------------------------------------------------------------------------
// Multiple right-hand sides (setup of the Schur blocks): X = A_jj^-1 X for a
// chunk of NR columns per CTA; X column-major (leading dimension n_j) in
// global memory, the tile windows staged in shared memory.
// ---------------------------------------------------------------------------
// columns 4ch .. 4ch+3 of row r of a forward tile K (16-byte chunks swizzled
// by row: four floats, or two pairs of doubles)
template <typename T, int TB>
__device__ __forceinline__ void k_row4(const T *__restrict__ K, int r, int ch, T (&o)[4]) {
  if (sizeof(T) == 4) {
    ld4(K + r * TB + ((ch ^ (r & 7)) << 2), o);
  } else {
    const T *row = K + r * TB;
    const double2 a = __ldg(reinterpret_cast<const double2 *>(row + (((2 * ch) ^ (r & 7)) << 1)));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(row + (((2 * ch + 1) ^ (r & 7)) << 1)));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
}

// X = A_jj^-1 X for a chunk of NR = 16 columns per CTA (256 threads).  A
// thread owns 4 right-hand sides (4 rq .. 4 rq + 3) of 4 window rows
// (forward) or of one tile row (backward) and accumulates them in
// registers: each tile value loaded serves 4 right-hand sides and each
// window value 4 rows.  Every output is summed over the tile's columns in
// ascending order, as a single chain of fused multiply-adds.
template <typename T, int NR, int TB>
__global__ void __launch_bounds__(256) band_solve_multi_kernel(const BandInfo *__restrict__ info,
                                                               const int32_t *__restrict__ ncols,
                                                               const int64_t *__restrict__ x_off,
                                                               const TileMeta *__restrict__ tm,
                                                               const T *__restrict__ ltile,
                                                               const T *__restrict__ utile,
                                                               const int32_t *__restrict__ srcs, T *Xall) {
  static_assert(NR == 16, "4 groups of 4 right-hand sides");
  const BandInfo b = info[blockIdx.x];
  const int nc = ncols[blockIdx.x];
  const int k0 = blockIdx.y * NR;
  if (b.n == 0 || k0 >= nc) return;
  const int nr = min(NR, nc - k0);
  const int n = b.n;
  T *X = Xall + x_off[blockIdx.x] + (int64_t)k0 * n;
  extern __shared__ __align__(128) unsigned char smraw[];
  T *win = reinterpret_cast<T *>(smraw);  // max(wl, wu) x NR, [row][r]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int rq = tid & 3, rg = tid >> 2;  // right-hand sides 4 rq.., row group
  // forward: X(window) <- [0; X_B] + K X_T on the exchanged window
  for (int t = 0; t < b.nst; ++t) {
    const TileMeta mt = tm[b.tile0 + t];
    const int c0 = t * TB, WL = mt.wl;
    const int32_t *src = srcs + mt.sofs;
    const T *K = ltile + mt.lofs;
    // along each right-hand side column, so neighbouring threads read
    // neighbouring rows of X
    for (int e = tid; e < WL * NR; e += nt) {
      const int r = e / WL, q = e % WL;
      const int row = c0 + src[q];
      win[q * NR + r] = (row < n && r < nr) ? X[(int64_t)r * n + row] : T(0);
    }
    __syncthreads();
    for (int ib = 0; ib < WL; ib += 256) {
      T acc[4][4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = min(ib + rg + 64 * k, WL - 1);
        T w0[4];
        ld4(win + i * NR + 4 * rq, w0);
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[k][v] = (i >= TB) ? w0[v] : T(0);
      }
#pragma unroll 2
      for (int ch = 0; ch < TB / 4; ++ch) {
        T w[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ld4(win + (4 * ch + u) * NR + 4 * rq, w[u]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          T kv[4];
          k_row4<T, TB>(K, min(ib + rg + 64 * k, WL - 1), ch, kv);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[k][v] = fma(kv[u], w[u][v], acc[k][v]);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = ib + rg + 64 * k;
        if (i < WL && c0 + i < n)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (4 * rq + v < nr) X[(int64_t)(4 * rq + v) * n + c0 + i] = acc[k][v];
      }
    }
    __syncthreads();
  }
  // backward: X_T <- Kb [X_T; X_next]; thread (row rg & 63, right-hand sides
  // 4 rq..), TB <= 64 rows
  for (int t = b.nst - 1; t >= 0; --t) {
    const TileMeta mt = tm[b.tile0 + t];
    const int r0 = t * TB, WU = mt.wu;
    const T *Kb = utile + mt.uofs;
    for (int e = tid; e < WU * NR; e += nt) {
      const int r = e / WU, q = e % WU;
      const int row = r0 + q;
      win[q * NR + r] = (row < n && r < nr) ? X[(int64_t)r * n + row] : T(0);
    }
    __syncthreads();
    const int i = rg;
    if (i < TB) {
      T acc[4] = {T(0), T(0), T(0), T(0)};
      const T *kr = Kb + (int64_t)i * WU;
#pragma unroll 2
      for (int k = 0; k < WU; k += 4) {
        T kv[4], w[4][4];
        ld4(kr + k, kv);
#pragma unroll
        for (int u = 0; u < 4; ++u) ld4(win + (k + u) * NR + 4 * rq, w[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[v] = fma(kv[u], w[u][v], acc[v]);
      }
      if (r0 + i < n)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (4 * rq + v < nr) X[(int64_t)(4 * rq + v) * n + r0 + i] = acc[v];
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static size_t sweep_base_bytes(int max_n, int max_kl, int max_ku2, size_t es, int tb, int cl, int max_tiles,
                               int max_jobs) {
  const int pad = sweep_pad_hd(max_kl, max_ku2);
  size_t used = 64 + es * (2 * ((size_t)max_n + pad) + tb + max_kl + 8 +
                           (cl > 1 ? 2 * (size_t)sweep_msg(tb, max_kl) : 0));
  used = (used + 15) & ~(size_t)15;
  used += sizeof(TileMeta) * (size_t)max_tiles + sizeof(SweepJob) * (size_t)max_jobs;
  return (used + 127) & ~(size_t)127;
}
// dynamic shared memory of a sweep CTA: the 227 KB a block may hold, less
// 256 bytes for the kernels' static shared variables
#define DD_SMEM_LIMIT (227 * 1024 - 256)
#define DD_MAX_STAGES 4
// stages of the ring at this stage size (0: two do not fit) for tiles of tb
// columns swept by clusters of cl CTAs
int band_sweep_stages(int max_n, int max_kl, int max_ku2, int tb, int cl, int elem_size, uint32_t stage_bytes) {
  if ((tb != 32 && tb != 64) || (cl != 1 && cl != 2)) return 0;
  // tables: at most max_n / tb tiles and twice as many jobs
  size_t base = sweep_base_bytes(max_n, max_kl, max_ku2, (size_t)elem_size, tb, cl, max_n / tb,
                                 2 * (max_n / tb));
  if (stage_bytes == 0 || base + 2 * (size_t)stage_bytes > DD_SMEM_LIMIT) return 0;
  int s = (int)((DD_SMEM_LIMIT - base) / stage_bytes);
  return s > DD_MAX_STAGES ? DD_MAX_STAGES : s;
}

#define DD_LU_SMEM (200 * 1024)
// largest ring stage (multiple of 128 bytes) that still leaves room for two
// stages next to the resident vectors and tables; 0 if none does
size_t band_sweep_max_stage(int max_n, int max_kl, int max_ku2, int elem_size, int tb, int cl) {
  const size_t base = sweep_base_bytes(max_n, max_kl, max_ku2, (size_t)elem_size, tb, cl, max_n / tb,
                                       2 * (max_n / tb));
  if (base >= DD_SMEM_LIMIT) return 0;
  return ((DD_SMEM_LIMIT - base) / 2) & ~(size_t)127;
}

size_t band_lu_window_bytes(int max_kl, int max_ku, int elem_size) {
  return (size_t)lu_window_elems(max_kl, max_ku) * elem_size;
}

template <typename T>
cudaError_t launch_band_lu(const BandInfo *d_info, int m, int max_kl, int max_ku, T *band, T *ltraw,
                           int32_t *piv, T *wscratch, double pivtol, DevStatus *st, int threads,
                           int grid, const int32_t *sched, const int32_t *sched_off, T *cnorm, double ilu_tol,
                           cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  if (ilu_tol > 0 && !cnorm) return cudaErrorInvalidValue;
  const size_t wb = band_lu_window_bytes(max_kl, max_ku, sizeof(T));
  const size_t smem = std::min(wb, (size_t)DD_LU_SMEM);
  cudaError_t e = ensure_smem(band_lu_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  band_lu_kernel<T><<<sched_off ? grid : m, threads, smem, s>>>(d_info, band, ltraw, piv, wscratch,
                                                                (int64_t)(wb / sizeof(T)), (int)smem,
                                                                pivtol, sched, sched_off, st, cnorm, T(ilu_tol));
  return cudaGetLastError();
}

// resident CTAs per SM of the band LU
template <typename T>
int band_lu_occupancy(int max_kl, int max_ku, int threads) {
  const size_t smem = std::min(band_lu_window_bytes(max_kl, max_ku, sizeof(T)), (size_t)DD_LU_SMEM);
  if (ensure_smem(band_lu_kernel<T>, smem) != cudaSuccess) return 0;
  int a = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, band_lu_kernel<T>, threads, smem) != cudaSuccess) return 0;
  return a;
}

template <typename T>
cudaError_t launch_tile_widths(const BandInfo *d_info, int m, int max_panels, const T *band,
                               const T *lraw, const int32_t *piv, int32_t *wl, int32_t *wu,
                               cudaStream_t s) {
  if (m <= 0 || max_panels <= 0) return cudaSuccess;
  tile_widths_kernel<T><<<dim3(m, max_panels), 32, 0, s>>>(d_info, band, lraw, piv, wl, wu);
  return cudaGetLastError();
}

template <typename T, int TB>
static cudaError_t tiles_tb(const BandInfo *d_info, int m, int max_tiles, int max_kl, const TileMeta *tm,
                            const T *band, const T *lraw, const int32_t *piv, T *ltile, T *utile,
                            int32_t *src, cudaStream_t s) {
  const int W = TB + max_kl;
  const size_t smem = sizeof(T) * (size_t)(2 * TB * TB + TB * W) + sizeof(int32_t) * (size_t)W;
  cudaError_t e = ensure_smem(band_tiles_kernel<T, TB>, smem);
  if (e != cudaSuccess) return e;
  band_tiles_kernel<T, TB><<<dim3(m, max_tiles), 4 * TB, smem, s>>>(d_info, tm, band, lraw, piv, ltile, utile,
                                                                     src);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_tiles(const BandInfo *d_info, int m, int max_tiles, int max_kl, int tb,
                              const TileMeta *tm, const T *band, const T *lraw, const int32_t *piv,
                              T *ltile, T *utile, int32_t *src, cudaStream_t s) {
  if (m <= 0 || max_tiles <= 0) return cudaSuccess;
  if (tb == 64) return tiles_tb<T, 64>(d_info, m, max_tiles, max_kl, tm, band, lraw, piv, ltile, utile, src, s);
  if (tb == 32) return tiles_tb<T, 32>(d_info, m, max_tiles, max_kl, tm, band, lraw, piv, ltile, utile, src, s);
  return cudaErrorInvalidValue;
}

// The tiles in the layout of the 2-CTA sweeps: CTA p's forward slice of
// tile t (its K rows [fwd_split(wl, p), fwd_split(wl, p + 1)), then the
// tile's src) at byte cfo[p], and its backward slice (Kb rows
// [p TB / 2, (p + 1) TB / 2)) at cbo[p].  Every piece is a multiple of 16
// bytes at a 16-byte aligned offset; one CTA per (tile, p, direction).
template <typename T, int TB>
__global__ void cluster_pack_kernel(int ntiles, const TileMeta *__restrict__ tm, const T *__restrict__ ltile,
                                    const T *__restrict__ utile, const int32_t *__restrict__ srcs,
                                    unsigned char *cld) {
  const int t = blockIdx.x, p = blockIdx.y;
  if (t >= ntiles) return;
  const TileMeta mt = tm[t];
  const uint4 *src[2];
  uint4 *dst[2];
  int64_t n16[2] = {0, 0};
  if (blockIdx.z == 0) {
    const int r0 = fwd_split(mt.wl, p, 2), r1 = fwd_split(mt.wl, p + 1, 2);
    const int64_t kb = (int64_t)(r1 - r0) * TB * sizeof(T);
    src[0] = reinterpret_cast<const uint4 *>(ltile + mt.lofs + (int64_t)r0 * TB);
    dst[0] = reinterpret_cast<uint4 *>(cld + mt.cfo[p]);
    n16[0] = kb / 16;
    src[1] = reinterpret_cast<const uint4 *>(srcs + mt.sofs);
    dst[1] = reinterpret_cast<uint4 *>(cld + mt.cfo[p] + kb);
    n16[1] = (int64_t)src_stride_w(mt.wl) * sizeof(int32_t) / 16;
  } else {
    src[0] = reinterpret_cast<const uint4 *>(utile + mt.uofs + (int64_t)p * (TB / 2) * mt.wu);
    dst[0] = reinterpret_cast<uint4 *>(cld + mt.cbo[p]);
    n16[0] = (int64_t)(TB / 2) * mt.wu * sizeof(T) / 16;
    src[1] = nullptr;
    dst[1] = nullptr;
  }
  for (int k = 0; k < 2; ++k)
    for (int64_t i = threadIdx.x; i < n16[k]; i += blockDim.x) dst[k][i] = src[k][i];
}

// Bytes of CTA p's forward and backward slices of one tile in the cluster
// layout (host side of cluster_pack_kernel's offsets).
void cluster_slice_bytes(const TileMeta &mt, int tb, int elem_size, int p, int64_t &fwd, int64_t &bwd) {
  const int r0 = fwd_split(mt.wl, p, 2), r1 = fwd_split(mt.wl, p + 1, 2);
  fwd = (int64_t)(r1 - r0) * tb * elem_size + (int64_t)src_stride_w(mt.wl) * 4;
  bwd = (int64_t)(tb / 2) * mt.wu * elem_size;
}

template <typename T>
cudaError_t launch_cluster_pack(int ntiles, int tb, const TileMeta *tm, const T *ltile, const T *utile,
                                const int32_t *srcs, unsigned char *cld, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  const dim3 grid(ntiles, 2, 2);
  if (tb == 64) cluster_pack_kernel<T, 64><<<grid, 128, 0, s>>>(ntiles, tm, ltile, utile, srcs, cld);
  else if (tb == 32) cluster_pack_kernel<T, 32><<<grid, 128, 0, s>>>(ntiles, tm, ltile, utile, srcs, cld);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// The backward tiles in the layout of the lookahead sweeps: CTA p's columns
// of tile t (la_cols), row by row, at byte lao[p].  Rows, column offsets and
// widths are multiples of 16 bytes; one CTA per (tile, p).
template <typename T, int TB>
__global__ void la_pack_kernel(int ntiles, const TileMeta *__restrict__ tm, const T *__restrict__ utile,
                               unsigned char *lad) {
  const int t = blockIdx.x, p = blockIdx.y;
  if (t >= ntiles) return;
  const TileMeta mt = tm[t];
  const int c0 = p == 0 ? 0 : la_split(mt.wu, TB), w = la_cols(mt.wu, TB, p);
  const int v16 = w * (int)sizeof(T) / 16;
  uint4 *dst = reinterpret_cast<uint4 *>(lad + mt.lao[p]);
  for (int e = threadIdx.x; e < TB * v16; e += blockDim.x) {
    const int r = e / v16, k = e % v16;
    dst[e] = reinterpret_cast<const uint4 *>(utile + mt.uofs + (int64_t)r * mt.wu + c0)[k];
  }
}

template <typename T>
cudaError_t launch_la_pack(int ntiles, int tb, const TileMeta *tm, const T *utile, unsigned char *lad,
                           cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  const dim3 grid(ntiles, 2);
  if (tb == 64) la_pack_kernel<T, 64><<<grid, 128, 0, s>>>(ntiles, tm, utile, lad);
  else if (tb == 32) la_pack_kernel<T, 32><<<grid, 128, 0, s>>>(ntiles, tm, utile, lad);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// one sweep launch: a plain grid, or clusters of cl CTAs
template <typename... KArgs, typename... Args>
static cudaError_t launch_sweep(void (*kernel)(KArgs...), int grid, int threads, size_t smem, int cl,
                                cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = cl > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T, int TB, int CL>
static size_t sweep_smem(int max_n, int max_kl, int max_ku2, int ns, uint32_t stage_bytes) {
  const int mt = max_n / TB, mj = 2 * mt;
  return sweep_base_bytes(max_n, max_kl, max_ku2, sizeof(T), TB, CL, mt, mj) + (size_t)ns * stage_bytes;
}

template <typename T, int TB, int CL, int LA = 0>
static cudaError_t fwd_tb(const BandInfo *d_info, int m, int max_n, int max_kl, int max_ku2, const SweepPlan &pl,
                          int ns, const TileMeta *tm, const SweepJob *jobs, const T *ltile, const T *utile,
                          const int32_t *src, const double *y, const int32_t *perm, T *z, DevStatus *st,
                          cudaStream_t s) {
  const int mt = max_n / TB, mj = 2 * mt;
  const int grid = pl.sched_off ? pl.grid : m * CL;
  const size_t smem = sweep_smem<T, TB, CL>(max_n, max_kl, max_ku2, ns, pl.stage_bytes);
  cudaError_t e = ensure_smem(band_solve_fwd_kernel<T, TB, CL, LA>, smem);
  if (e != cudaSuccess) return e;
  if (grid <= 0) return cudaSuccess;
  return launch_sweep(band_solve_fwd_kernel<T, TB, CL, LA>, grid, LA ? 8 * TB : 8 * TB / CL, smem, CL, s, d_info,
                      max_n, max_kl, max_ku2, mt, mj, ns, pl.stage_bytes, tm, jobs, ltile, utile, src,
                      LA ? pl.lad : pl.cld, y, perm, z, pl.sched, pl.sched_off, pl.task_sys, pl.act, st,
                      pl.first_wait, pl.pf);
}

// tile width of a plan: 8 TB / cl threads per CTA (8 TB in the lookahead split)
static inline int plan_tb(const SweepPlan &pl) { return pl.la ? pl.threads / 8 : pl.threads * pl.cl / 8; }

template <typename T>
cudaError_t launch_band_solve_fwd(const BandInfo *d_info, int m, int max_n, int max_kl,
                                  int max_ku2, const SweepPlan &pl, const TileMeta *tm,
                                  const SweepJob *jobs, const T *ltile, const T *utile,
                                  const int32_t *src, const double *y, const int32_t *perm, T *z,
                                  DevStatus *st, cudaStream_t s) {
  const int tb = plan_tb(pl);
  const int ns = band_sweep_stages(max_n, max_kl, max_ku2, tb, pl.cl, sizeof(T), pl.stage_bytes);
  if (ns < 2) return cudaErrorInvalidValue;
  // the backward tile step maps exactly 8 threads to each of the CTA's rows
  if (pl.la && pl.cl == 2 && tb == 64)
    return fwd_tb<T, 64, 2, 1>(d_info, m, max_n, max_kl, max_ku2, pl, ns, tm, jobs, ltile, utile, src, y, perm, z, st,
                               s);
  if (pl.la && pl.cl == 2 && tb == 32)
    return fwd_tb<T, 32, 2, 1>(d_info, m, max_n, max_kl, max_ku2, pl, ns, tm, jobs, ltile, utile, src, y, perm, z, st,
                               s);
  if (pl.la) return cudaErrorInvalidValue;
  if (tb == 64 && pl.cl == 1)
    return fwd_tb<T, 64, 1>(d_info, m, max_n, max_kl, max_ku2, pl, ns, tm, jobs, ltile, utile, src, y, perm, z, st, s);
  if (tb == 64 && pl.cl == 2)
    return fwd_tb<T, 64, 2>(d_info, m, max_n, max_kl, max_ku2, pl, ns, tm, jobs, ltile, utile, src, y, perm, z, st, s);
  if (tb == 32 && pl.cl == 1)
    return fwd_tb<T, 32, 1>(d_info, m, max_n, max_kl, max_ku2, pl, ns, tm, jobs, ltile, utile, src, y, perm, z, st, s);
  if (tb == 32 && pl.cl == 2)
    return fwd_tb<T, 32, 2>(d_info, m, max_n, max_kl, max_ku2, pl, ns, tm, jobs, ltile, utile, src, y, perm, z, st, s);
  return cudaErrorInvalidValue;
}

template <typename T, int TB, int CL, int LA = 0>
static cudaError_t bwd_tb(const BandInfo *d_info, int m, int max_n, int max_kl, int max_ku2, const SweepPlan &pl,
                          int ns, const TileMeta *tm, const SweepJob *jobs, const T *ltile, const T *utile,
                          const int32_t *src, const int32_t *e_ptr, const int32_t *e_col, const T *e_val,
                          const T *z2, const T *z1, const int32_t *perm, double *x, DevStatus *st,
                          cudaStream_t s) {
  const int mt = max_n / TB, mj = 2 * mt;
  const int grid = pl.sched_off ? pl.grid : m * CL;
  const size_t smem = sweep_smem<T, TB, CL>(max_n, max_kl, max_ku2, ns, pl.stage_bytes);
  cudaError_t e = ensure_smem(band_solve_bwd_kernel<T, TB, CL, LA>, smem);
  if (e != cudaSuccess) return e;
  if (grid <= 0) return cudaSuccess;
  return launch_sweep(band_solve_bwd_kernel<T, TB, CL, LA>, grid, LA ? 8 * TB : 8 * TB / CL, smem, CL, s, d_info,
                      max_n, max_kl, max_ku2, mt, mj, ns, pl.stage_bytes, tm, jobs, ltile, utile, src,
                      LA ? pl.lad : pl.cld, e_ptr, e_col, e_val, z2, z1, perm, x, pl.sched, pl.sched_off, pl.task_sys,
                      pl.act, st, pl.first_wait, pl.pf);
}

template <typename T>
cudaError_t launch_band_solve_bwd(const BandInfo *d_info, int m, int max_n, int max_kl,
                                  int max_ku2, const SweepPlan &pl, const TileMeta *tm,
                                  const SweepJob *jobs, const T *ltile, const T *utile,
                                  const int32_t *src, const int32_t *e_ptr, const int32_t *e_col,
                                  const T *e_val, const T *z2, const T *z1, const int32_t *perm,
                                  double *x, DevStatus *st, cudaStream_t s) {
  const int tb = plan_tb(pl);
  const int ns = band_sweep_stages(max_n, max_kl, max_ku2, tb, pl.cl, sizeof(T), pl.stage_bytes);
  if (ns < 2) return cudaErrorInvalidValue;
#define DD_BWD_CASE(TBV, CLV, LAV)                                                                  \
  if (tb == TBV && pl.cl == CLV && pl.la == LAV)                                                        \
    return bwd_tb<T, TBV, CLV, LAV>(d_info, m, max_n, max_kl, max_ku2, pl, ns, tm, jobs, ltile, utile, src, \
                                    e_ptr, e_col, e_val, z2, z1, perm, x, st, s);
  DD_BWD_CASE(64, 1, 0)
  DD_BWD_CASE(64, 2, 0)
  DD_BWD_CASE(32, 1, 0)
  DD_BWD_CASE(32, 2, 0)
  DD_BWD_CASE(64, 2, 1)
  DD_BWD_CASE(32, 2, 1)
#undef DD_BWD_CASE
  return cudaErrorInvalidValue;
}

// Subdomains the sweep kernels hold resident at once at this stage size
// (both kernels; the smaller): CTAs per SM times SMs for cl = 1, the device's
// active clusters for cl = 2.  0 when they do not fit.
template <typename T, int TB, int CL, int LA = 0>
static int slots_tb(int max_n, int max_kl, int max_ku2, int ns, uint32_t stage_bytes) {
  const size_t smem = sweep_smem<T, TB, CL>(max_n, max_kl, max_ku2, ns, stage_bytes);
  if (ensure_smem(band_solve_fwd_kernel<T, TB, CL, LA>, smem) != cudaSuccess) return 0;
  if (ensure_smem(band_solve_bwd_kernel<T, TB, CL, LA>, smem) != cudaSuccess) return 0;
  int a = 0, b = 0;
  if (CL == 1) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, band_solve_fwd_kernel<T, TB, CL, LA>, 8 * TB, smem) !=
        cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, band_solve_bwd_kernel<T, TB, CL, LA>, 8 * TB, smem) !=
        cudaSuccess)
      return 0;
    return (a < b ? a : b) * sms;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL * 64);
  cfg.blockDim = dim3(LA ? 8 * TB : 8 * TB / CL);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaOccupancyMaxActiveClusters(&a, band_solve_fwd_kernel<T, TB, CL, LA>, &cfg) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveClusters(&b, band_solve_bwd_kernel<T, TB, CL, LA>, &cfg) != cudaSuccess) return 0;
  return a < b ? a : b;
}

template <typename T>
int band_sweep_slots(int max_n, int max_kl, int max_ku2, int tb, int cl, uint32_t stage_bytes, int la) {
  const int ns = band_sweep_stages(max_n, max_kl, max_ku2, tb, cl, sizeof(T), stage_bytes);
  if (ns < 2) return 0;
  if (la) {
    if (cl != 2) return 0;
    if (tb == 64) return slots_tb<T, 64, 2, 1>(max_n, max_kl, max_ku2, ns, stage_bytes);
    if (tb == 32) return slots_tb<T, 32, 2, 1>(max_n, max_kl, max_ku2, ns, stage_bytes);
    return 0;
  }
  if (tb == 64 && cl == 1) return slots_tb<T, 64, 1>(max_n, max_kl, max_ku2, ns, stage_bytes);
  if (tb == 64 && cl == 2) return slots_tb<T, 64, 2>(max_n, max_kl, max_ku2, ns, stage_bytes);
  if (tb == 32 && cl == 1) return slots_tb<T, 32, 1>(max_n, max_kl, max_ku2, ns, stage_bytes);
  if (tb == 32 && cl == 2) return slots_tb<T, 32, 2>(max_n, max_kl, max_ku2, ns, stage_bytes);
  return 0;
}

#define DD_MULTI_NR 16
template <typename T, int TB>
static cudaError_t multi_tb(const BandInfo *d_info, int m, const int32_t *ncols, const int64_t *x_off,
                            int max_cols, int max_kl, int max_ku2, const TileMeta *tm, const T *ltile,
                            const T *utile, const int32_t *src, T *X, cudaStream_t s) {
  const int w = round4(TB + (max_kl > max_ku2 ? max_kl : max_ku2));
  size_t smem = sizeof(T) * (size_t)w * DD_MULTI_NR;
  cudaError_t e = ensure_smem(band_solve_multi_kernel<T, DD_MULTI_NR, TB>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(m, (max_cols + DD_MULTI_NR - 1) / DD_MULTI_NR);
  band_solve_multi_kernel<T, DD_MULTI_NR, TB><<<grid, 256, smem, s>>>(d_info, ncols, x_off, tm, ltile, utile,
                                                                      src, X);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_solve_multi(const BandInfo *d_info, int m, const int32_t *ncols,
                                    const int64_t *x_off, int max_cols, int max_kl, int max_ku2, int tb,
                                    const TileMeta *tm, const T *ltile, const T *utile,
                                    const int32_t *src, T *X, cudaStream_t s) {
  if (max_cols <= 0) return cudaSuccess;
  if (tb == 64) return multi_tb<T, 64>(d_info, m, ncols, x_off, max_cols, max_kl, max_ku2, tm, ltile, utile, src, X, s);
  if (tb == 32) return multi_tb<T, 32>(d_info, m, ncols, x_off, max_cols, max_kl, max_ku2, tm, ltile, utile, src, X, s);
  return cudaErrorInvalidValue;
}

#define DD_INST_BAND(T)                                                                            \
  template cudaError_t launch_band_lu<T>(const BandInfo *, int, int, int, T *, T *, int32_t *,     \
                                         T *, double, DevStatus *, int, int, const int32_t *,       \
                                         const int32_t *, T *, double, cudaStream_t);               \
  template int band_lu_occupancy<T>(int, int, int);                                                \
  template cudaError_t launch_tile_widths<T>(const BandInfo *, int, int, const T *, const T *,     \
                                             const int32_t *, int32_t *, int32_t *, cudaStream_t); \
  template cudaError_t launch_band_tiles<T>(const BandInfo *, int, int, int, int, const TileMeta *,\
                                            const T *, const T *, const int32_t *, T *, T *,       \
                                            int32_t *, cudaStream_t);                               \
  template cudaError_t launch_band_solve_fwd<T>(const BandInfo *, int, int, int, int,             \
                                                const SweepPlan &, const TileMeta *,                \
                                                const SweepJob *, const T *, const T *,             \
                                                const int32_t *, const double *, const int32_t *,   \
                                                T *, DevStatus *, cudaStream_t);                    \
  template cudaError_t launch_band_solve_bwd<T>(                                                   \
      const BandInfo *, int, int, int, int, const SweepPlan &, const TileMeta *,                   \
      const SweepJob *, const T *, const T *, const int32_t *, const int32_t *, const int32_t *,    \
      const T *, const T *, const T *, const int32_t *, double *, DevStatus *, cudaStream_t);      \
  template int band_sweep_slots<T>(int, int, int, int, int, uint32_t, int);                         \
  template cudaError_t launch_la_pack<T>(int, int, const TileMeta *, const T *, unsigned char *,     \
                                         cudaStream_t);                                             \
  template cudaError_t launch_cluster_pack<T>(int, int, const TileMeta *, const T *, const T *,    \
                                              const int32_t *, unsigned char *, cudaStream_t);      \
  template cudaError_t launch_band_solve_multi<T>(const BandInfo *, int, const int32_t *,          \
                                                  const int64_t *, int, int, int, int,             \
                                                  const TileMeta *, const T *, const T *,          \
                                                  const int32_t *, T *, cudaStream_t);

DD_INST_BAND(double)
DD_INST_BAND(float)
