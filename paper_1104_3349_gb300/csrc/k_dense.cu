// Interface blocks: assembly of the mini Schur complements S_ii (Algorithm 1),
// their explicit inverses (Gauss-Jordan with partial pivoting, the same pivot
// sequence as LU with partial pivoting), and the interface step of the apply
// z2_i = S_ii^-1 (y2 - F z1)_i (Algorithm 2).
//
// Dense blocks are stored row-major, block b at offset off[b], size p[b].
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dd_internal.h"

namespace {

template <typename T>
__device__ __forceinline__ T tabs(T v) { return v < T(0) ? -v : v; }

__device__ void set_status2(DevStatus *st, int code, int block) {
  if (atomicCAS(&st->code, 0, code) == 0) st->block = block;
}

// largest |A| of every block: CTA (x, b) scans slice x of block b, and the
// slices meet in an atomic max on the bit pattern (order-independent for
// non-negative values, so the result is deterministic)
__device__ __forceinline__ void atomic_max_nonneg(float *a, float v) {
  atomicMax(reinterpret_cast<unsigned int *>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double *a, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(a), (unsigned long long)__double_as_longlong(v));
}
template <typename T>
__global__ void block_amax_kernel(const int32_t *__restrict__ P, const int64_t *__restrict__ off,
                                  const T *__restrict__ A, T *amax) {
  const int b = blockIdx.y;
  const int p = P[b];
  const T *a = A + off[b];
  const int64_t total = (int64_t)p * p;
  const int64_t chunk = (total + gridDim.x - 1) / gridDim.x;
  const int64_t q0 = (int64_t)blockIdx.x * chunk, q1 = min(total, q0 + chunk);
  T mx = T(0);
  for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) mx = fmax(mx, tabs(a[q]));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ T red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    T m2 = T(0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, red[w]);
    if (m2 > T(0)) atomic_max_nonneg(&amax[b], m2);
  }
}

// The column exchanges that undo the row exchanges (in reverse order) are
// one permutation of the columns, the same for every row: cidx[c] = the
// column whose entry ends in column c.  One CTA per block composes it.
__global__ void gj_colperm_kernel(const int32_t *__restrict__ P, const int32_t *__restrict__ ipiv,
                                  const int64_t *__restrict__ poff, const int32_t *__restrict__ failed,
                                  int32_t *cidx) {
  const int b = blockIdx.x;
  const int p = P[b];
  if (failed[b]) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  int32_t *ix = reinterpret_cast<int32_t *>(smraw);
  for (int c = threadIdx.x; c < p; c += blockDim.x) ix[c] = c;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = p - 1; k >= 0; --k) {
      const int q = ipiv[poff[b] + k];
      if (q != k) { const int t = ix[k]; ix[k] = ix[q]; ix[q] = t; }
    }
  __syncthreads();
  for (int c = threadIdx.x; c < p; c += blockDim.x) cidx[poff[b] + c] = ix[c];
}

// row r of block b (CTA (r, b)) gathered through shared memory
template <typename T>
__global__ void gj_unscramble_kernel(const int32_t *__restrict__ P, const int64_t *__restrict__ off,
                                     T *A, const int32_t *__restrict__ cidx,
                                     const int64_t *__restrict__ poff,
                                     const int32_t *__restrict__ failed) {
  const int b = blockIdx.y, r = blockIdx.x;
  const int p = P[b];
  if (r >= p || failed[b]) return;
  T *row = A + off[b] + (int64_t)r * p;
  extern __shared__ __align__(128) unsigned char smraw[];
  T *ts = reinterpret_cast<T *>(smraw);
  for (int c = threadIdx.x; c < p; c += blockDim.x) ts[c] = row[c];
  __syncthreads();
  const int32_t *ix = cidx + poff[b];
  for (int c = threadIdx.x; c < p; c += blockDim.x) row[c] = ts[ix[c]];
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan inverse with two levels of blocking.  For each outer
// block of NO columns k0..k0+NO-1 (NO = 64 in FP32, 32 in FP64):
//  (1) copy: W = A(k0:p, panel), a tall p-k0 x NO panel in scratch;
//  (2) LU with partial pivoting of W, NB columns at a time (NB = 16 / 8):
//      panel kernel (one CTA per block: pivots, multipliers, the exchanges
//      on the other columns of W, U12 = L11^-1 A12) then a trailing update
//      of W's remaining columns (many CTAs per block);
//  (3) the NO row exchanges on whole rows of A, through a staged copy of
//      the touched rows;
//  (4) A11^-1 from W's L11 and U11 (forward and back substitution on the
//      identity, one warp per column); row block Rnew = A11^-1 A(R, :) as a
//      small product; and a copy Pcol = A(:, panel);
//  (5) update kernel (tiled):
//        A(R, panel) = A11^-1,  A(R, j) = Rnew(:, j),
//        A(i, panel) = -Pcol(i, :) A11^-1,  A(i, j) -= Pcol(i, :) Rnew(:, j).
// The pivots are those of LU with partial pivoting (largest magnitude, then
// lowest row), so in exact arithmetic the result is the inverse Gauss-Jordan
// computes column by column, with the rank-1 passes grouped into rank-NO
// updates of the whole matrix.  The row exchanges are undone as column
// exchanges at the end.
// Scratch per block b at gj_base(b) = 6*NO*poff[b] + (NO*NO + 4*NO)*b:
//   [W p x NO | panel copy p x (NB+1) (when it does not fit in shared memory)
//    within NO*p | Pcol p x NO | Rnew NO x p | staged rows 2NO x p |
//    A11^-1 NO x NO | exchange list 4*NO int32]
// ---------------------------------------------------------------------------
template <typename T>
struct BgjNB { static const int value = 16; };
template <>
struct BgjNB<double> { static const int value = 8; };
template <typename T>
struct BgjNO { static const int value = 64; };
template <>
struct BgjNO<double> { static const int value = 32; };

// 16-byte vector of T
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static void unpack(const float4 &a, float *v) { v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; }
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static void unpack(const double2 &a, double *v) { v[0] = a.x; v[1] = a.y; }
};

template <typename T, int NO>
__device__ __forceinline__ T *gj_base(T *scratch, const int64_t *poff, int b) {
  return scratch + 6 * (int64_t)NO * poff[b] + (int64_t)(NO * NO + 4 * NO) * b;
}

// (1) W(r, c) = A(k0 + r, k0 + c), zero beyond the matrix
template <typename T, int NO>
__global__ void bgj_copy_kernel(int k0, const int32_t *__restrict__ P, const int64_t *__restrict__ off,
                                const T *__restrict__ A, T *scratch, const int64_t *__restrict__ poff,
                                const int32_t *__restrict__ failed) {
  const int b = blockIdx.y;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int rows = p - k0, nbo = min(NO, rows);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * NO) return;
  const int r = (int)(e / NO), c = (int)(e % NO);
  T *W = gj_base<T, NO>(scratch, poff, b);
  W[e] = (c < nbo) ? A[off[b] + (int64_t)(k0 + r) * p + k0 + c] : T(0);
}

// The end of a pivot panel (both panel kernels): the panel's row exchanges
// applied to W's other columns, then U12 = L11^-1 W(c0:c0+nbe, right) with
// L11 (unit lower, row stride ldl) in shared memory.  The panel's own
// columns are already back in Wg.  Every thread of the CTA calls it.
template <typename T, int NB, int NO>
__device__ void bgj_panel_tail(T *Wg, const T *L11, int ldl, const int *s_q, int c0, int nbe, int nbo) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __syncthreads();  // the panel is written and s_q complete
  // The same exchanges on W's other columns.  Exchanges c0+c <-> q_c (c in
  // order, q_c >= c0+c) touch at most 2 nbe rows; destination d ends up
  // holding the old row tau_0(tau_1(...tau_{nbe-1}(d))), found by walking the
  // transpositions backwards.  One thread per column loads all touched rows
  // before storing any.
  static_assert(2 * NB <= 32, "one warp lists the exchanged rows");
  __shared__ int s_dst[2 * NB], s_src[2 * NB];
  __shared__ int s_cnt;
  if (warp == 0) {
    int d = -1, x = -1;
    if (lane < 2 * nbe) {
      d = lane < nbe ? c0 + lane : s_q[lane - nbe];
      if (lane >= nbe && d < c0 + nbe) d = -1;  // a panel row, already listed
      x = d;
      if (d >= 0)
        for (int c = nbe - 1; c >= 0; --c) {
          const int q = s_q[c];
          if (x == c0 + c) x = q;
          else if (x == q) x = c0 + c;
        }
    }
    const bool moved = d >= 0 && x != d;
    const unsigned m = __ballot_sync(0xffffffffu, moved);
    if (moved) {
      const int pos = __popc(m & ((1u << lane) - 1u));
      s_src[pos] = x;
      s_dst[pos] = d;
    }
    if (lane == 0) s_cnt = __popc(m);
  }
  __syncthreads();
  {
    const int cnt = s_cnt;
    const int j = tid < c0 ? tid : tid + nbe;  // the columns outside this step
    if (tid < nbo - nbe) {
      T v[2 * NB];
#pragma unroll
      for (int t = 0; t < 2 * NB; ++t)
        if (t < cnt) v[t] = Wg[(int64_t)s_src[t] * NO + j];
#pragma unroll
      for (int t = 0; t < 2 * NB; ++t)
        if (t < cnt) Wg[(int64_t)s_dst[t] * NO + j] = v[t];
    }
  }
  __syncthreads();
  // U12 = L11^-1 W(c0:c0+nbe, j) for the columns right of this step
  {
    const int j = c0 + nbe + tid;
    if (j < nbo) {
      T x[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) x[c] = (c < nbe) ? Wg[(int64_t)(c0 + c) * NO + j] : T(0);
#pragma unroll
      for (int c = 1; c < NB; ++c) {
        if (c < nbe) {
          T t = x[c];
#pragma unroll
          for (int q = 0; q < c; ++q) t -= L11[c * ldl + q] * x[q];
          x[c] = t;
        }
      }
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < nbe) Wg[(int64_t)(c0 + c) * NO + j] = x[c];
    }
  }
}

// (2a) Columns c0..c0+nbe-1 of W (c0 = NB*s), rows c0..: LU with partial
// pivoting on a copy in shared memory (or scratch), written back; the row
// exchanges applied to W's other columns; U12 = L11^-1 W(c0:c0+nbe, right).
// 512 threads: at 1024 the 64-register cap made the kernel spill
#define DD_GJ_PANEL_THREADS 512
template <typename T, int NB, int NO>
__global__ void __launch_bounds__(DD_GJ_PANEL_THREADS, 1) bgj_panel_kernel(int k0, int s, const int32_t *__restrict__ P,
                                                            T *scratch, const int64_t *__restrict__ poff,
                                                            int32_t *ipiv, const T *__restrict__ amax,
                                                            double pivtol, int32_t *failed, DevStatus *st,
                                                            int code, int smem_rows) {
  const int b = blockIdx.x;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int rows_all = p - k0, nbo = min(NO, rows_all), c0 = NB * s;
  if (c0 >= nbo) return;
  const int nbe = min(NB, nbo - c0), rows = rows_all - c0;
  T *Wg = gj_base<T, NO>(scratch, poff, b);
  extern __shared__ __align__(128) unsigned char smraw[];
  // rows x NB with row stride NB+1 (conflict-free for row- and column-wise access)
  constexpr int LD = NB + 1;
  T *W = (rows <= smem_rows) ? reinterpret_cast<T *>(smraw) : Wg + (int64_t)NO * p;
  __shared__ T bv[32];
  __shared__ int bi[32];
  __shared__ int s_piv;
  __shared__ int s_fail;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  if (tid == 0) s_fail = 0;
  // eight loads in flight per thread before their stores
  for (int e0 = tid; e0 < rows * NB; e0 += 8 * nt) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nt, r = e / NB, c = e % NB;
      v[u] = (e < rows * NB && c < nbe) ? Wg[(int64_t)(c0 + r) * NO + c0 + c] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nt;
      if (e < rows * NB) W[(e / NB) * LD + e % NB] = v[u];
    }
  }
  __syncthreads();
  const T thresh = T(pivtol) * amax[b];
  // Column c: warp 0 picks the pivot row pr among the candidates (largest
  // |W(r, c)|, then lowest r) and copies rows pr and c; then, in one pass,
  // row c takes the pivot row, row pr takes the old row c, every row below c
  // is eliminated, and its entry of column c+1 is offered as the next
  // candidate.  Two barriers per column; the arithmetic is that of exchanging
  // rows c and pr and then eliminating.
  __shared__ T prow[NB], crow[NB];
  {
    T best = T(-1);
    int besti = rows;
    for (int r = tid; r < rows; r += nt) {
      const T v = tabs(W[r * LD]);
      if (v > best) { best = v; besti = r; }
    }
    int unused = 0;
    warp_argmax(best, besti, unused);
    if (lane == 0) { bv[warp] = best; bi[warp] = besti; }
  }
  __syncthreads();
  __shared__ int s_q[NB];  // W row of the pivot of column c0 + c
  for (int c = 0; c < nbe; ++c) {
    if (warp == 0) {
      T bb = lane < nw ? bv[lane] : T(-1);
      int ii = lane < nw ? bi[lane] : rows, unused = 0;
      warp_argmax(bb, ii, unused);
      if (lane == 0) {
        if (!(bb > thresh)) {
          s_fail = 1;
          failed[b] = 1;
          set_status2(st, code, b);
        }
        s_piv = ii;
        s_q[c] = c0 + ii;
        ipiv[poff[b] + k0 + c0 + c] = k0 + c0 + ii;
      }
      if (lane < NB && ii < rows) {
        prow[lane] = W[ii * LD + lane];
        crow[lane] = W[c * LD + lane];
      }
    }
    __syncthreads();
    if (s_fail) return;
    const int pr = s_piv;
    const T piv = prow[c];
    if (tid < NB) W[c * LD + tid] = prow[tid];
    T best = T(-1);
    int besti = rows;
    // the pivot row in registers; each row's entries loaded before any of
    // its stores (the column loops are unrolled with predicates)
    T pv[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) pv[q] = prow[q];
    for (int r = c + 1 + tid; r < rows; r += nt) {
      const bool sw = (r == pr);
      T *wr = W + r * LD;
      const T *src = sw ? crow : wr;
      const T l = src[c] / piv;
      T a[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q > c && q < nbe) a[q] = src[q];
      wr[c] = l;
      if (sw)
        for (int q = 0; q < c; ++q) wr[q] = crow[q];
      T next = T(-1);
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q > c && q < nbe) {
          const T t = a[q] - l * pv[q];
          wr[q] = t;
          if (q == c + 1) next = tabs(t);
        }
      if (next > best) { best = next; besti = r; }
    }
    int unused = 0;
    warp_argmax(best, besti, unused);
    if (lane == 0) { bv[warp] = best; bi[warp] = besti; }
    __syncthreads();
  }
  // the factored columns back into W
  for (int e = tid; e < rows * nbe; e += nt) {
    const int r = e / nbe, c = e % nbe;
    Wg[(int64_t)(c0 + r) * NO + c0 + c] = W[r * LD + c];
  }
  bgj_panel_tail<T, NB, NO>(Wg, W, LD, s_q, c0, nbe, nbo);
}


// (2a') The same panel with every thread's rows in registers: rows
// r = tid + k * blockDim.x (k < RPT) of the panel's rows_all - c0.  Per
// column: the warps' winners reduced in every warp, the owners of the
// pivot row and of row c publish them, one barrier, then each thread
// exchanges and eliminates its rows without touching shared memory and
// offers its candidates for the next column.  Same pivots and arithmetic
// as bgj_panel_kernel; used when the panel's rows fit RPT per thread.
template <typename T, int NB, int NO, int RPT>
__global__ void __launch_bounds__(DD_GJ_PANEL_THREADS, 1) bgj_panel_reg_kernel(int k0, int s,
                                                                const int32_t *__restrict__ P, T *scratch,
                                                                const int64_t *__restrict__ poff, int32_t *ipiv,
                                                                const T *__restrict__ amax, double pivtol,
                                                                int32_t *failed, DevStatus *st, int code) {
  const int b = blockIdx.x;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int rows_all = p - k0, nbo = min(NO, rows_all), c0 = NB * s;
  if (c0 >= nbo) return;
  const int nbe = min(NB, nbo - c0), rows = rows_all - c0;
  T *Wg = gj_base<T, NO>(scratch, poff, b);
  constexpr int LD = NB + 1;
  __shared__ T bv[32];
  __shared__ int bi[32];
  __shared__ T prow[NB], crow[NB];
  __shared__ T L11[NB * LD];
  __shared__ int s_q[NB];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  T a[RPT][NB];
  // each row's NB entries in 16-byte loads (rows of Wg start on 16-byte
  // boundaries: NO and c0 are multiples of 16 / sizeof(T))
  using Vt = typename Vec16<T>::V;
  constexpr int VN = Vec16<T>::N;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int r = tid + k * nt;
    const Vt *src = reinterpret_cast<const Vt *>(Wg + (int64_t)(c0 + r) * NO + c0);
#pragma unroll
    for (int v = 0; v < NB / VN; ++v) {
      T u[VN];
      if (r < rows) Vec16<T>::unpack(src[v], u);
#pragma unroll
      for (int e = 0; e < VN; ++e) a[k][v * VN + e] = (r < rows && v * VN + e < nbe) ? u[e] : T(0);
    }
  }
  const T thresh = T(pivtol) * amax[b];
  {
    T best = T(-1);
    int besti = rows, unused = 0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int r = tid + k * nt;
      const T v = tabs(a[k][0]);
      if (r < rows && v > best) { best = v; besti = r; }
    }
    warp_argmax(best, besti, unused);
    if (lane == 0) { bv[warp] = best; bi[warp] = besti; }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c >= nbe) break;
    // the pivot: every warp reduces the warps' winners
    T bb = lane < nw ? bv[lane] : T(-1);
    int pr = lane < nw ? bi[lane] : rows, unused = 0;
    warp_argmax(bb, pr, unused);
    if (!(bb > thresh)) {
      if (tid == 0) {
        failed[b] = 1;
        set_status2(st, code, b);
      }
      return;  // every thread of the CTA takes the same decision
    }
    if (tid == 0) {
      s_q[c] = c0 + pr;
      ipiv[poff[b] + k0 + c0 + c] = k0 + c0 + pr;
    }
    // slot k and thread of the pivot row and of row c (uniform over the CTA,
    // so only one slot's code runs, and only in the owning warp)
    const int kp = pr / nt, tp = pr % nt, kc = c / nt, tc = c % nt;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (k == kp && tid == tp)
#pragma unroll
        for (int q = 0; q < NB; ++q) prow[q] = a[k][q];
      if (k == kc && tid == tc)
#pragma unroll
        for (int q = 0; q < NB; ++q) crow[q] = a[k][q];
    }
    __syncthreads();  // prow / crow published; every warp has read bv / bi
    // one reciprocal per column: a multiply per row instead of a division
    // (a rounding of the multipliers, within the parity bounds)
    const T rpiv = T(1) / prow[c];
    T best = T(-1);
    int besti = rows;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int r = tid + k * nt;
      if (k == kc && tid == tc) {
#pragma unroll
        for (int q = 0; q < NB; ++q) a[k][q] = prow[q];
      } else if (k == kp && tid == tp) {
#pragma unroll
        for (int q = 0; q < NB; ++q) a[k][q] = crow[q];
      }
      if (r > c && r < rows) {
        const T l = a[k][c] * rpiv;
        a[k][c] = l;
#pragma unroll
        for (int q = c + 1; q < NB; ++q)
          if (q < nbe) a[k][q] -= l * prow[q];
        if (c + 1 < nbe) {
          const T v = tabs(a[k][c + 1]);
          if (v > best) { best = v; besti = r; }
        }
      }
    }
    warp_argmax(best, besti, unused);
    if (lane == 0) { bv[warp] = best; bi[warp] = besti; }
    __syncthreads();  // the offers are in; prow / crow are free again
  }
  // the factored columns back to Wg; rows 0..nbe-1 (L11 / U11) also to shared memory
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int r = tid + k * nt;
    if (r < rows)
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < nbe) {
          Wg[(int64_t)(c0 + r) * NO + c0 + q] = a[k][q];
          if (r < NB) L11[r * LD + q] = a[k][q];
        }
  }
  bgj_panel_tail<T, NB, NO>(Wg, L11, LD, s_q, c0, nbe, nbo);
}

// (2') The whole NO-column slab of an outer step at once (FP32, rows of W
// below k0 up to DD_GJ_CL * DD_GJ_SLAB_THREADS): LU with partial pivoting,
// column by column, over a cluster of DD_GJ_CL CTAs.  Thread t of CTA r
// holds the slab row that starts at position r * DD_GJ_SLAB_THREADS + t,
// all NO entries in registers.  Rows never move while the slab is factored:
// each thread tracks where the interchanges so far have put its row, and
// stores the row there at the end.  Per pivot column c:
//   - every warp's best candidate among the rows at positions >= c (largest
//     |entry|, then lowest position) publishes its whole row in a slot of
//     shared memory; warp 0 reduces the CTA's warps to one candidate;
//   - one cluster barrier; warp 0 of every CTA reads the CTAs' candidates
//     through distributed shared memory, reduces them to the same pivot and
//     copies the pivot row;
//   - the interchange of positions c and p_c goes to ipiv; every other row
//     at a position >= c takes its multiplier (one reciprocal per column)
//     and its rank-one update.
// Slots, candidates and the pivot row copy alternate between two buffers
// by column parity: a buffer is rewritten two columns later, after a
// cluster barrier that every reader of it has passed.  The outcome of the
// pivot test is the same in every CTA, so all of them take the same cluster
// barriers; a last one keeps every CTA resident until the others have read
// its slots.  The result is that of the four panel steps and three trailing
// updates, with the rank-one updates in another order.
#define DD_GJ_CL 8
#define DD_GJ_SLAB_THREADS 512
__device__ __forceinline__ int32_t ld_cluster_i32(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ uint32_t cluster_addr(const void *local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
  return r;
}
__device__ __forceinline__ void gj_cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

template <int NO>
__global__ void __launch_bounds__(DD_GJ_SLAB_THREADS, 1) bgj_slab_kernel(int k0, const int32_t *__restrict__ P,
                                                                      float *scratch,
                                                                      const int64_t *__restrict__ poff,
                                                                      int32_t *ipiv, const float *__restrict__ amax,
                                                                      double pivtol, int32_t *failed, DevStatus *st,
                                                                      int code) {
  constexpr int NT = DD_GJ_SLAB_THREADS, NW = NT / 32;
  static_assert(NO % 4 == 0 && NO / 4 <= 32 && DD_GJ_CL <= 32, "one warp copies a row and reduces the CTAs");
  const int rank = (int)(blockIdx.x % DD_GJ_CL), b = (int)(blockIdx.x / DD_GJ_CL);
  const int p = P[b];
  if (k0 >= p || failed[b]) return;  // the same in every CTA of the cluster, before any barrier
  const int rows_all = p - k0, nbo = min(NO, rows_all);
  float *Wg = gj_base<float, NO>(scratch, poff, b);
  __shared__ __align__(16) float slot[2][NW][NO];
  __shared__ __align__(16) float prow[2][NO];
  __shared__ float wv[NW];
  __shared__ int wpos[NW];
  __shared__ int32_t cand[2][4];  // the CTA's candidate: |value| bits, position, warp
  __shared__ int s_pc[2], s_ok[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int mypos = rank * NT + tid;
  const bool has = mypos < rows_all;
  float a[NO];
  {
    const float4 *src = reinterpret_cast<const float4 *>(Wg + (int64_t)(has ? mypos : 0) * NO);
#pragma unroll
    for (int v = 0; v < NO / 4; ++v) {
      const float4 q = has ? src[v] : make_float4(0.f, 0.f, 0.f, 0.f);
      a[4 * v] = q.x;
      a[4 * v + 1] = q.y;
      a[4 * v + 2] = q.z;
      a[4 * v + 3] = q.w;
    }
  }
  const float thresh = (float)pivtol * amax[b];
  bool ok = true;
#pragma unroll
  for (int c = 0; c < NO; ++c) {
    if (!ok || c >= nbo) continue;  // the same in every thread of the cluster
    const int buf = c & 1;
    const bool act = has && mypos >= c;
    float v = act ? fabsf(a[c]) : -1.f;
    int L = act ? mypos : INT_MAX, unused = 0;
    warp_argmax(v, L, unused);
    if (act && mypos == L) {
      float4 *dst = reinterpret_cast<float4 *>(slot[buf][warp]);
#pragma unroll
      for (int q = 0; q < NO / 4; ++q) dst[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
    }
    if (lane == 0) {
      wv[warp] = v;
      wpos[warp] = L;
    }
    __syncthreads();
    if (warp == 0) {
      float bv = lane < NW ? wv[lane] : -1.f;
      int bl = lane < NW ? wpos[lane] : INT_MAX, bw = lane;
      warp_argmax(bv, bl, bw);
      if (lane == 0) {
        cand[buf][0] = __float_as_int(bv);
        cand[buf][1] = bl;
        cand[buf][2] = bw;
      }
    }
    gj_cluster_barrier();
    if (warp == 0) {
      float cv = -1.f;
      int cl = INT_MAX, pay = 0;
      if (lane < DD_GJ_CL) {
        const uint32_t ra = cluster_addr(&cand[buf][0], (uint32_t)lane);
        cv = __int_as_float(ld_cluster_i32(ra));
        cl = ld_cluster_i32(ra + 4);
        pay = lane * NW + ld_cluster_i32(ra + 8);
      }
      warp_argmax(cv, cl, pay);
      if (lane < NO / 4) {
        const uint32_t ra = cluster_addr(&slot[buf][pay % NW][4 * lane], (uint32_t)(pay / NW));
        reinterpret_cast<float4 *>(prow[buf])[lane] = ld_cluster_f4(ra);
      }
      if (lane == 0) {
        s_pc[buf] = cl;
        s_ok[buf] = cv > thresh ? 1 : 0;
      }
    }
    __syncthreads();
    const int pc = s_pc[buf];
    if (!s_ok[buf]) {
      ok = false;
      continue;
    }
    if (rank == 0 && tid == 0) ipiv[poff[b] + k0 + c] = k0 + pc;
    if (act) {
      if (mypos == pc) {
        mypos = c;  // the pivot row: row c of U
      } else {
        if (mypos == c) mypos = pc;  // the row exchanged with the pivot row
        const float l = a[c] * (1.f / prow[buf][c]);
        a[c] = l;
#pragma unroll
        for (int q = c + 1; q < NO; ++q) a[q] -= l * prow[buf][q];
      }
    }
  }
  gj_cluster_barrier();  // every CTA has read the others' slots
  if (!ok) {
    if (rank == 0 && tid == 0) {
      failed[b] = 1;
      set_status2(st, code, b);
    }
    return;
  }
  if (has) {
    float4 *dst = reinterpret_cast<float4 *>(Wg + (int64_t)mypos * NO);
#pragma unroll
    for (int q = 0; q < NO / 4; ++q) dst[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
  }
}

// (2b) W(i, j) -= L21(i, :) U12(:, j) for the rows below and the columns
// right of step s; CTA x takes 64 rows
template <typename T, int NB, int NO>
__global__ void __launch_bounds__(256) bgj_trail_kernel(int k0, int s, const int32_t *__restrict__ P,
                                                        T *scratch, const int64_t *__restrict__ poff,
                                                        const int32_t *__restrict__ failed) {
  const int b = blockIdx.y;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int rows_all = p - k0, nbo = min(NO, rows_all), c0 = NB * s;
  if (c0 >= nbo) return;
  const int nbe = min(NB, nbo - c0), j0 = c0 + nbe, ncol = nbo - j0;
  const int i0 = j0 + 64 * blockIdx.x;
  if (ncol <= 0 || i0 >= rows_all) return;
  const int nr = min(64, rows_all - i0);
  T *Wg = gj_base<T, NO>(scratch, poff, b);
  __shared__ T Us[NB][NO];
  __shared__ T Ls[64][NB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NO; e += blockDim.x) {
    const int c = e / NO, q = e % NO;
    Us[c][q] = (c < nbe && q < ncol) ? Wg[(int64_t)(c0 + c) * NO + j0 + q] : T(0);
  }
  for (int e = tid; e < 64 * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    Ls[r][c] = (r < nr && c < nbe) ? Wg[(int64_t)(i0 + r) * NO + c0 + c] : T(0);
  }
  __syncthreads();
  for (int e = tid; e < nr * ncol; e += blockDim.x) {
    const int r = e / ncol, q = e % ncol;
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < NB; ++c) acc += Ls[r][c] * Us[c][q];
    T *o = &Wg[(int64_t)(i0 + r) * NO + j0 + q];
    *o = *o - acc;
  }
}

// (3) The outer block's exchanges k0+c <-> ipiv(k0+c), c < nbo, in order, on
// whole rows of A: every CTA lists the touched rows (destination d holds the
// old row found by walking the exchanges backwards; at most 2 nbo rows),
// CTA 0 stores the list, and each thread stages its column of the touched
// rows.  The write kernel then stores them in their new places.
template <int NO>
__device__ __forceinline__ void gj_exchange_list(int k0, int nbo, const int32_t *ip, int *s_q, int *s_dst,
                                                 int *s_src) {
  const int tid = threadIdx.x;
  if (tid < nbo) s_q[tid] = ip[k0 + tid];
  __syncthreads();
  if (tid < 2 * NO) {
    int d = -1, x = -1;
    if (tid < 2 * nbo) {
      d = tid < nbo ? k0 + tid : s_q[tid - nbo];
      if (tid >= nbo && d < k0 + nbo) d = -1;  // a row of the block, already listed
      x = d;
      if (d >= 0)
        for (int c = nbo - 1; c >= 0; --c) {
          const int q = s_q[c];
          if (x == k0 + c) x = q;
          else if (x == q) x = k0 + c;
        }
    }
    s_dst[tid] = (d >= 0 && x != d) ? d : -1;
    s_src[tid] = x;
  }
  __syncthreads();
}

template <typename T, int NO>
__global__ void __launch_bounds__(256) bgj_stage_kernel(int k0, const int32_t *__restrict__ P,
                                                        const int64_t *__restrict__ off, const T *__restrict__ A,
                                                        T *scratch, const int64_t *__restrict__ poff,
                                                        const int32_t *__restrict__ ipiv,
                                                        const int32_t *__restrict__ failed) {
  static_assert(2 * NO <= 256, "one thread per listed row");
  const int b = blockIdx.y;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int nbo = min(NO, p - k0);
  T *base = gj_base<T, NO>(scratch, poff, b);
  T *Tst = base + 4 * (int64_t)NO * p;
  int32_t *lst = reinterpret_cast<int32_t *>(base + 6 * (int64_t)NO * p + NO * NO);
  __shared__ int s_q[NO], s_dst[2 * NO], s_src[2 * NO];
  gj_exchange_list<NO>(k0, nbo, ipiv + poff[b], s_q, s_dst, s_src);
  if (blockIdx.x == 0 && threadIdx.x < 2 * NO) {
    lst[threadIdx.x] = s_dst[threadIdx.x];
    lst[2 * NO + threadIdx.x] = s_src[threadIdx.x];
  }
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  const T *a = A + off[b];
  for (int t = 0; t < 2 * nbo; ++t)
    if (s_dst[t] >= 0) Tst[(int64_t)t * p + j] = a[(int64_t)s_src[t] * p + j];
}

template <typename T, int NO>
__global__ void __launch_bounds__(256) bgj_write_kernel(int k0, const int32_t *__restrict__ P,
                                                        const int64_t *__restrict__ off, T *A,
                                                        T *scratch, const int64_t *__restrict__ poff,
                                                        const int32_t *__restrict__ failed) {
  const int b = blockIdx.y;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int nbo = min(NO, p - k0);
  T *base = gj_base<T, NO>(scratch, poff, b);
  const T *Tst = base + 4 * (int64_t)NO * p;
  const int32_t *lst = reinterpret_cast<const int32_t *>(base + 6 * (int64_t)NO * p + NO * NO);
  __shared__ int s_dst[2 * NO];
  if (threadIdx.x < 2 * NO) s_dst[threadIdx.x] = lst[threadIdx.x];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  T *a = A + off[b];
  for (int t = 0; t < 2 * nbo; ++t)
    if (s_dst[t] >= 0) a[(int64_t)s_dst[t] * p + j] = Tst[(int64_t)t * p + j];
}

// (4a) A11^-1 = U11^-1 L11^-1 from W's leading nbo x nbo block: one warp per
// column of the identity.  Lane l holds rows l + 32 u; each step broadcasts
// the finished entry and the rows below (or above) take their multiple of it.
template <typename T, int NO>
__global__ void __launch_bounds__(1024) bgj_a11inv_kernel(int k0, const int32_t *__restrict__ P, T *scratch,
                                                          const int64_t *__restrict__ poff,
                                                          const int32_t *__restrict__ failed) {
  constexpr int RU = NO / 32;
  static_assert(NO % 32 == 0, "whole rows per lane");
  const int b = blockIdx.y;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int nbo = min(NO, p - k0);
  T *base = gj_base<T, NO>(scratch, poff, b);
  T *a11inv = base + 6 * (int64_t)NO * p;
  __shared__ T LU[NO][NO + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < NO * NO; e += blockDim.x) {
    const int r = e / NO, c = e % NO;
    LU[r][c] = (r < nbo && c < nbo) ? base[(int64_t)r * NO + c] : T(0);
  }
  __syncthreads();
  const int col = blockIdx.x * (blockDim.x >> 5) + warp;
  if (col >= NO) return;  // whole warps leave
  T x[RU];
#pragma unroll
  for (int u = 0; u < RU; ++u) x[u] = (lane + 32 * u == col && col < nbo) ? T(1) : T(0);
  for (int c = col; c < nbo; ++c) {  // L11 y = e_col (unit lower), by columns
    T own = x[0];
#pragma unroll
    for (int u = 1; u < RU; ++u)
      if (u == c / 32) own = x[u];
    const T xc = __shfl_sync(0xffffffffu, own, c & 31);
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int r = lane + 32 * u;
      if (r > c && r < nbo) x[u] -= LU[r][c] * xc;
    }
  }
  for (int c = nbo - 1; c >= 0; --c) {  // U11 z = y, by columns
    const int uo = c / 32;
#pragma unroll
    for (int u = 0; u < RU; ++u)
      if (u == uo && lane == (c & 31)) x[u] = x[u] / LU[c][c];
    T own = x[0];
#pragma unroll
    for (int u = 1; u < RU; ++u)
      if (u == uo) own = x[u];
    const T xc = __shfl_sync(0xffffffffu, own, c & 31);
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int r = lane + 32 * u;
      if (r < c) x[u] -= LU[r][c] * xc;
    }
  }
#pragma unroll
  for (int u = 0; u < RU; ++u) a11inv[(lane + 32 * u) * NO + col] = x[u];
}

// (4b) Rnew(:, j) = A11^-1 A(k0:k0+nbo, j) for the columns outside the block:
// 64 columns per CTA; thread (g, q) forms rows 16 g .. 16 g + 15 of column
// j0 + q.
template <typename T, int NO>
__global__ void __launch_bounds__(256) bgj_rowblock_kernel(int k0, const int32_t *__restrict__ P,
                                                           const int64_t *__restrict__ off, const T *__restrict__ A,
                                                           T *scratch, const int64_t *__restrict__ poff,
                                                           const int32_t *__restrict__ failed) {
  constexpr int NC = 64, RG = NO / 4;  // 4 row groups of RG rows
  const int b = blockIdx.y;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int nbo = min(NO, p - k0);
  const int j0 = blockIdx.x * NC;
  if (j0 >= p) return;
  T *base = gj_base<T, NO>(scratch, poff, b);
  T *Rnew = base + 3 * (int64_t)NO * p;
  const T *a11inv = base + 6 * (int64_t)NO * p;
  __shared__ T Ai[NO][NO];
  __shared__ T Xs[NO][NC + 1];
  const int tid = threadIdx.x;
  const T *a = A + off[b];
  for (int e = tid; e < NO * NO; e += blockDim.x) Ai[e / NO][e % NO] = a11inv[e];
  for (int e = tid; e < NO * NC; e += blockDim.x) {
    const int c = e / NC, q = e % NC, j = j0 + q;
    Xs[c][q] = (c < nbo && j < p) ? a[(int64_t)(k0 + c) * p + j] : T(0);
  }
  __syncthreads();
  const int q = tid % NC, g = tid / NC;
  const int j = j0 + q;
  T acc[RG];
#pragma unroll
  for (int r = 0; r < RG; ++r) acc[r] = T(0);
#pragma unroll 8
  for (int c = 0; c < NO; ++c) {
    const T xv = Xs[c][q];
#pragma unroll
    for (int r = 0; r < RG; ++r) acc[r] += Ai[g * RG + r][c] * xv;
  }
  if (j >= p || (j >= k0 && j < k0 + nbo)) return;
#pragma unroll
  for (int r = 0; r < RG; ++r) Rnew[(int64_t)(g * RG + r) * p + j] = acc[r];
}

// Pcol(i, :) = A(i, k0:k0+nbo) for every row i, zero beyond nbo; consecutive
// threads copy consecutive columns of a row
template <typename T, int NO>
__global__ void __launch_bounds__(256) bgj_pcol_kernel(int k0, const int32_t *__restrict__ P,
                                                       const int64_t *__restrict__ off, const T *__restrict__ A,
                                                       T *scratch, const int64_t *__restrict__ poff,
                                                       const int32_t *__restrict__ failed) {
  const int b = blockIdx.y;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int nbo = min(NO, p - k0);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * NO) return;
  const int i = (int)(e / NO), c = (int)(e % NO);
  T *Pcol = gj_base<T, NO>(scratch, poff, b) + 2 * (int64_t)NO * p;
  Pcol[e] = (c < nbo) ? A[off[b] + (int64_t)i * p + k0 + c] : T(0);
}

#define DD_BGJ_TILE 64
#define DD_BGJ_RT 4
#define DD_BGJ_UPD_THREADS ((DD_BGJ_TILE / DD_BGJ_RT) * (DD_BGJ_TILE / DD_BGJ_RT))

// TF32 tensor-core products with near-FP32 accuracy (the DD_FP32_TF32
// precision): x = hi + lo with hi the TF32 rounding of x and lo that of the
// remainder; a b ~ a_lo b_hi + a_hi b_lo + a_hi b_hi (the a_lo b_lo term and
// the rounding of the lo parts are below FP32's unit roundoff relative to
// a b), accumulated in FP32 by the tensor cores.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
// c += a b for one m16n8k8 fragment (a 16 x 8 row-major, b 8 x 8 column-
// major, c 16 x 8, in the register layouts of the warp-level mma)
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Rank-NB update of one 64 x 64 tile from a transposed P column chunk and an
// R row chunk staged in shared memory.  Each of the 256 threads owns 4
// consecutive rows by 4 consecutive columns and accumulates the outer
// products in registers; with TC (FP32 only, DD_FP32_TF32) each of the 8
// warps takes a 16 x 32 block as four m16n8 fragments on the tensor cores,
// every product in three TF32 terms (split_tf32).
template <typename T, int NB, int TC = 0>
__global__ void __launch_bounds__(DD_BGJ_UPD_THREADS, 3) bgj_update_kernel(int k0, const int32_t *__restrict__ P,
                                                         const int64_t *__restrict__ off, T *A,
                                                         const T *__restrict__ scratch,
                                                         const int64_t *__restrict__ poff,
                                                         const int32_t *__restrict__ failed) {
  const int b = blockIdx.z;
  const int p = P[b];
  if (k0 >= p || failed[b]) return;
  const int i0 = blockIdx.y * DD_BGJ_TILE, j0 = blockIdx.x * DD_BGJ_TILE;
  if (i0 >= p || j0 >= p) return;
  const int nbe = min(NB, p - k0);
  T *a = A + off[b];
  const T *scr = gj_base<const T, NB>(scratch, poff, b);
  const T *Pcol = scr + 2 * (int64_t)NB * p;
  const T *Rnew = scr + 3 * (int64_t)NB * p;
  const T *a11inv = scr + 6 * (int64_t)NB * p;
  constexpr int LD = DD_BGJ_TILE + 4;  // keeps every row 16-byte aligned
  __shared__ __align__(16) T Pt[NB][LD];  // Pt[c][r] = Pcol(i0 + r, c)
  __shared__ __align__(16) T Rs[NB][LD];  // Rs[c][q] = new row c at column j0 + q
  const int tid = threadIdx.x;
  constexpr int NT = DD_BGJ_UPD_THREADS;
  {
    // Pcol rows i0.. are contiguous: 16-byte loads, all issued before the
    // transposed stores
    using V = typename Vec16<T>::V;
    constexpr int VN = Vec16<T>::N;
    constexpr int NL = DD_BGJ_TILE * NB / VN / NT;
    static_assert(NB % VN == 0 && (DD_BGJ_TILE * NB / VN) % NT == 0, "whole 16-byte chunks per thread");
    const V *src = reinterpret_cast<const V *>(Pcol + (int64_t)i0 * NB);
    V v[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int e = tid + k * NT, r = (e * VN) / NB;
      if (i0 + r < p) v[k] = src[e];
    }
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int e = tid + k * NT, r = (e * VN) / NB, c = (e * VN) % NB;
      T u[VN];
      if (i0 + r < p) Vec16<T>::unpack(v[k], u);
      else
        for (int w = 0; w < VN; ++w) u[w] = T(0);
#pragma unroll
      for (int w = 0; w < VN; ++w) Pt[c + w][r] = u[w];
    }
  }
  {
    constexpr int NL = NB * DD_BGJ_TILE / NT;
    static_assert((NB * DD_BGJ_TILE) % NT == 0, "whole row chunks per thread");
    T v[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int e = tid + k * NT, c = e / DD_BGJ_TILE, j = j0 + e % DD_BGJ_TILE;
      v[k] = T(0);
      if (j < p) v[k] = (j >= k0 && j < k0 + nbe) ? a11inv[c * NB + (j - k0)] : Rnew[(int64_t)c * p + j];
    }
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int e = tid + k * NT;
      Rs[e / DD_BGJ_TILE][e % DD_BGJ_TILE] = v[k];
    }
  }
  __syncthreads();
  constexpr int RT = DD_BGJ_RT, TH = DD_BGJ_TILE / DD_BGJ_RT;
  constexpr bool TCU = TC && sizeof(T) == 4 && NB % 8 == 0 && DD_BGJ_UPD_THREADS == 256 && DD_BGJ_TILE == 64;
  const int tr = tid / TH, tc = tid % TH;
  const int rb = RT * tr, qb = RT * tc;
  // TCU: warp w holds rows mb + g, mb + g + 8 and columns nb + 8 j + 2 t4,
  // + 1 of fragment j (g = lane / 4, t4 = lane % 4)
  const int g = (tid & 31) >> 2, t4 = tid & 3;
  const int mb = 16 * ((tid >> 5) & 3), nb = 32 * (tid >> 7);
  float cf[4][4];
  T acc[RT][RT];
  if constexpr (TCU) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) cf[j][e] = 0.f;
#pragma unroll 2
    for (int k0 = 0; k0 < NB; k0 += 8) {
      uint32_t ah[4], al[4];
      split_tf32((float)Pt[k0 + t4][mb + g], ah[0], al[0]);
      split_tf32((float)Pt[k0 + t4][mb + g + 8], ah[1], al[1]);
      split_tf32((float)Pt[k0 + t4 + 4][mb + g], ah[2], al[2]);
      split_tf32((float)Pt[k0 + t4 + 4][mb + g + 8], ah[3], al[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t bh[2], bl[2];
        split_tf32((float)Rs[k0 + t4][nb + 8 * j + g], bh[0], bl[0]);
        split_tf32((float)Rs[k0 + t4 + 4][nb + 8 * j + g], bh[1], bl[1]);
        mma_tf32(cf[j], al, bh);
        mma_tf32(cf[j], ah, bl);
        mma_tf32(cf[j], ah, bh);
      }
    }
  } else {
#pragma unroll
    for (int x = 0; x < RT; ++x)
#pragma unroll
      for (int y = 0; y < RT; ++y) acc[x][y] = T(0);
#pragma unroll 8
    for (int c = 0; c < NB; ++c) {
      T pv[RT], rv[RT];
#pragma unroll
      for (int x = 0; x < RT; ++x) { pv[x] = Pt[c][rb + x]; rv[x] = Rs[c][qb + x]; }
#pragma unroll
      for (int x = 0; x < RT; ++x)
#pragma unroll
        for (int y = 0; y < RT; ++y) acc[x][y] += pv[x] * rv[y];
    }
  }
  // Epilogue through shared memory (over Pt, no longer read), CH rows at a
  // time, so that consecutive threads update consecutive columns of A.
  constexpr int SL = DD_BGJ_TILE + 1;
  constexpr int CH = ((NB * LD) / SL) / RT * RT < DD_BGJ_TILE ? ((NB * LD) / SL) / RT * RT : DD_BGJ_TILE;
  static_assert(CH >= RT && DD_BGJ_TILE % CH == 0, "whole thread rows per epilogue chunk");
  T *S = &Pt[0][0];
  for (int h = 0; h < DD_BGJ_TILE; h += CH) {
    __syncthreads();
    if constexpr (TCU) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = mb + g + 8 * (e >> 1), q = nb + 8 * j + 2 * t4 + (e & 1);
          if (r >= h && r < h + CH) S[(r - h) * SL + q] = (T)cf[j][e];
        }
    } else if (rb >= h && rb < h + CH) {
#pragma unroll
      for (int x = 0; x < RT; ++x)
#pragma unroll
        for (int y = 0; y < RT; ++y) S[(rb - h + x) * SL + qb + y] = acc[x][y];
    }
    __syncthreads();
    // every load of the chunk before any store
    constexpr int NE = CH * DD_BGJ_TILE / NT;
    static_assert((CH * DD_BGJ_TILE) % NT == 0, "whole chunk per thread");
    T cur[NE];
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      const int e = tid + k * NT, i = i0 + h + e / DD_BGJ_TILE, j = j0 + e % DD_BGJ_TILE;
      cur[k] = (i < p && j < p) ? a[(int64_t)i * p + j] : T(0);
    }
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      const int e = tid + k * NT, r = e / DD_BGJ_TILE, q = e % DD_BGJ_TILE;
      const int i = i0 + h + r, j = j0 + q;
      if (i >= p || j >= p) continue;
      T v;
      if (i >= k0 && i < k0 + nbe) v = Rs[i - k0][q];            // pivot row
      else if (j >= k0 && j < k0 + nbe) v = -S[r * SL + q];      // panel column
      else v = cur[k] - S[r * SL + q];
      a[(int64_t)i * p + j] = v;
    }
  }
}

template <typename T>
__global__ void scatter_coo_kernel(int64_t nnz, const int64_t *__restrict__ idx,
                                   const double *__restrict__ val, T *dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nnz) dst[idx[i]] += T(val[i]);
}

// S(R_a, R_a) -= F(r, I_j) X_j(:, c) for every interface pair (r, c) that
// the subdomain j couples (r: rows of F into I_j, c: columns of E from I_j)
// and that fall into the same aggregate a, for the subdomains j = jlist[x]
// of one colour.  No two subdomains of a colour share an interface row, and
// within one subdomain every (r, c) is a different entry, so the updates are
// plain read-modify-writes; the colours run one after the other in a fixed
// order, so the sum over j of every entry is taken in the same order on
// every run.
template <typename T>
__global__ void schur_accumulate_kernel(const int32_t *__restrict__ jlist,
                                        const int32_t *__restrict__ fr_ptr,
                                        const int32_t *__restrict__ fr_row,
                                        const int32_t *__restrict__ fr_agg,
                                        const int32_t *__restrict__ f_ptr,
                                        const int32_t *__restrict__ f_col,
                                        const T *__restrict__ f_val,
                                        const int32_t *__restrict__ gam_ptr,
                                        const int32_t *__restrict__ gam_idx,
                                        const int32_t *__restrict__ gam_agg,
                                        const int64_t *__restrict__ x_off,
                                        const BandInfo *__restrict__ info, const T *__restrict__ X,
                                        const int32_t *__restrict__ agg_off,
                                        const int64_t *__restrict__ s_off, T *S) {
  const int j = jlist[blockIdx.x];
  const int r_lo = fr_ptr[j], r_hi = fr_ptr[j + 1];
  const int rr = r_lo + blockIdx.y;
  if (rr >= r_hi) return;
  const int g_lo = gam_ptr[j], g_hi = gam_ptr[j + 1];
  const int nj = info[j].n;
  const T *Xj = X + x_off[j];
  const int a = fr_agg[rr];
  const int row = fr_row[rr];
  const int p = agg_off[a + 1] - agg_off[a];
  T *Sa = S + s_off[a];
  for (int g = g_lo + threadIdx.x; g < g_hi; g += blockDim.x) {
    if (gam_agg[g] != a) continue;
    const int col = gam_idx[g];
    const T *xc = Xj + (int64_t)(g - g_lo) * nj;
    T s = T(0);
    for (int k = f_ptr[rr]; k < f_ptr[rr + 1]; ++k) s += f_val[k] * xc[f_col[k]];
    Sa[(int64_t)(row - agg_off[a]) * p + (col - agg_off[a])] -= s;
  }
}

// C = alpha * A B + beta * C for square blocks (row-major), 16x16 tiles.
template <typename T>
__global__ void block_gemm_kernel(const int32_t *__restrict__ P, const int64_t *__restrict__ off,
                                  const T *__restrict__ A, const T *__restrict__ B, T *C, T alpha,
                                  T beta) {
  const int b = blockIdx.z;
  const int p = P[b];
  const int r0 = blockIdx.y * 16, c0 = blockIdx.x * 16;
  if (r0 >= p || c0 >= p) return;
  const T *a = A + off[b];
  const T *bb = B + off[b];
  T *c = C + off[b];
  __shared__ T As[16][17], Bs[16][17];
  const int tr = threadIdx.y, tc = threadIdx.x;
  T acc = T(0);
  for (int k0 = 0; k0 < p; k0 += 16) {
    As[tr][tc] = (r0 + tr < p && k0 + tc < p) ? a[(int64_t)(r0 + tr) * p + k0 + tc] : T(0);
    Bs[tr][tc] = (k0 + tr < p && c0 + tc < p) ? bb[(int64_t)(k0 + tr) * p + c0 + tc] : T(0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc += As[tr][q] * Bs[q][tc];
    __syncthreads();
  }
  if (r0 + tr < p && c0 + tc < p) {
    T *o = &c[(int64_t)(r0 + tr) * p + c0 + tc];
    *o = alpha * acc + beta * *o;
  }
}

// S_hat of the overlapped kinds, dense n_G x n_G: entry (r, c) belongs to
// the block of the aggregate a holding min(r, c) when max(r, c) < agg[a+1] +
// w[a] (the blocks placed in aggregate order, a later block overwriting the
// overlap, leave exactly this), else it is 0.  Block a is q_a x q_a,
// q_a = agg[a+1] - agg[a] + w[a], row-major at xoff[a] in Sx.
template <typename T>
__global__ void assemble_overlapped_kernel(int ng, int k, const int32_t *__restrict__ agg,
                                           const int32_t *__restrict__ w, const int64_t *__restrict__ xoff,
                                           const T *__restrict__ Sx, T *S) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ng * ng) return;
  const int r = (int)(e / ng), c = (int)(e % ng);
  const int lo = min(r, c), hi = max(r, c);
  int a0 = 0, a1 = k;  // aggregate of lo: agg[a] <= lo < agg[a+1]
  while (a1 - a0 > 1) {
    const int mid = (a0 + a1) >> 1;
    if (agg[mid] <= lo) a0 = mid; else a1 = mid;
  }
  const int q = agg[a0 + 1] - agg[a0] + w[a0];
  T v = T(0);
  if (hi < agg[a0] + q) v = Sx[xoff[a0] + (int64_t)(r - agg[a0]) * q + (c - agg[a0])];
  S[e] = v;
}

// C_b = alpha A_b B_b + beta C_b for rectangular row-major blocks: dims
// holds (M, N, K) and offs the offsets of A (M x K), B (K x N), C (M x N)
// of block b; 16 x 16 output tiles, K in steps of 16.
template <typename T>
__global__ void rect_gemm_kernel(const int32_t *__restrict__ dims, const int64_t *__restrict__ offs,
                                 const T *__restrict__ A, const T *__restrict__ Bm, T *C, T alpha, T beta) {
  const int b = blockIdx.z;
  const int M = dims[3 * b], N = dims[3 * b + 1], K = dims[3 * b + 2];
  const int r0 = blockIdx.y * 16, c0 = blockIdx.x * 16;
  if (r0 >= M || c0 >= N) return;
  const T *a = A + offs[3 * b];
  const T *bb = Bm + offs[3 * b + 1];
  T *cc = C + offs[3 * b + 2];
  __shared__ T As[16][17], Bs[16][17];
  const int tr = threadIdx.y, tc = threadIdx.x;
  T acc = T(0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    As[tr][tc] = (r0 + tr < M && k0 + tc < K) ? a[(int64_t)(r0 + tr) * K + k0 + tc] : T(0);
    Bs[tr][tc] = (k0 + tr < K && c0 + tc < N) ? bb[(int64_t)(k0 + tr) * N + c0 + tc] : T(0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc += As[tr][q] * Bs[q][tc];
    __syncthreads();
  }
  if (r0 + tr < M && c0 + tc < N) {
    T *o = &cc[(int64_t)(r0 + tr) * N + c0 + tc];
    *o = alpha * acc + beta * *o;
  }
}

// MSCNR: S -= diag(F Dinv E 1), one CTA per block.
template <typename T>
__global__ void mscnr_diag_kernel(const int32_t *__restrict__ P, const int64_t *__restrict__ off,
                                  const T *__restrict__ Dinv, const T *__restrict__ E,
                                  const T *__restrict__ F, T *S) {
  const int b = blockIdx.x;
  const int p = P[b];
  extern __shared__ __align__(128) unsigned char smraw[];
  T *v = reinterpret_cast<T *>(smraw);
  T *w = v + p;
  const T *e = E + off[b], *d = Dinv + off[b], *f = F + off[b];
  T *s = S + off[b];
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    T acc = T(0);
    for (int c = 0; c < p; ++c) acc += e[(int64_t)r * p + c];
    v[r] = acc;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    T acc = T(0);
    for (int c = 0; c < p; ++c) acc += d[(int64_t)r * p + c] * v[c];
    w[r] = acc;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    T acc = T(0);
    for (int c = 0; c < p; ++c) acc += f[(int64_t)r * p + c] * w[c];
    s[(int64_t)r * p + r] -= acc;
  }
}

// t = y2 - F z1 (one thread per interface row)
template <typename T>
__global__ void schur_rhs_kernel(int ng, const int32_t *__restrict__ f_ptr, const int32_t *__restrict__ f_col,
                                 const T *__restrict__ f_val, const double *__restrict__ y,
                                 const int32_t *__restrict__ perm_iface, const T *__restrict__ z1, T *t) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  T s = T(y[perm_iface[g]]);
  for (int k = f_ptr[g]; k < f_ptr[g + 1]; ++k) s -= f_val[k] * z1[f_col[k]];
  t[g] = s;
}

// z2 = S_hat^-1 t per aggregate, one warp per row of S_hat^-1 with 16-byte
// loads; x2 = z2 written to x.  A row of p entries starts on a 16-byte
// boundary only when p (and the block's offset) allow it, so each row takes
// h = (its misalignment) leading entries one by one, then 16-byte chunks,
// then the remainder.  The chunks need t shifted by h: shared memory holds
// V = 16 / sizeof(T) copies, copy h holding t[h..], so every chunk of t is a
// 16-byte load too.  Eight chunks per lane in flight, 16 rows per CTA (two
// per warp): enough bytes in flight per SM for HBM.
#define DD_SROWS 16
template <typename T>
__global__ void schur_gemv_kernel(const int32_t *__restrict__ agg_off, const int64_t *__restrict__ s_off,
                                  const T *__restrict__ Sinv, const T *__restrict__ t,
                                  const int32_t *__restrict__ perm_iface, T *z2, double *x,
                                  const int32_t *__restrict__ agg_sys, const int32_t *__restrict__ act,
                                  int ldt) {
  const int a = blockIdx.y;
  if (act && !act[agg_sys[a]]) return;  // a batched system that has stopped stepping
  const int g0 = agg_off[a], p = agg_off[a + 1] - g0;
  const int rbase = blockIdx.x * DD_SROWS;
  if (rbase >= p) return;
  constexpr int V = 16 / sizeof(T);
  using Vt = typename Vec16<T>::V;
  extern __shared__ __align__(128) unsigned char smraw[];
  T *ts = reinterpret_cast<T *>(smraw);  // V copies of ldt entries (ldt a multiple of V)
  for (int r = threadIdx.x; r < p + V; r += blockDim.x) {
    const T v = r < p ? t[g0 + r] : T(0);
#pragma unroll
    for (int h = 0; h < V; ++h)
      if (r >= h && r - h < ldt) ts[h * ldt + r - h] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T *Sa = Sinv + s_off[a];
  for (int rr = warp; rr < DD_SROWS; rr += nw) {
    const int r = rbase + rr;
    if (r >= p) break;
    const T *row = Sa + (int64_t)r * p;
    const int h = min(p, (int)((V - (int)((reinterpret_cast<uintptr_t>(row) / sizeof(T)) % V)) % V));
    const int m = (p - h) / V;  // whole 16-byte chunks
    const Vt *rv = reinterpret_cast<const Vt *>(row + h);
    const Vt *tv = reinterpret_cast<const Vt *>(ts + h * ldt);
    T acc0 = T(0), acc1 = T(0), acc2 = T(0), acc3 = T(0);
    if (lane < h) acc0 = row[lane] * ts[lane];
    int k = lane;
    for (; k + 224 < m; k += 256) {
      Vt v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = rv[k + 32 * u];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        T a0[V], b0[V];
        Vec16<T>::unpack(v[u], a0);
        Vec16<T>::unpack(tv[k + 32 * u], b0);
        T &acc = (u & 3) == 0 ? acc0 : (u & 3) == 1 ? acc1 : (u & 3) == 2 ? acc2 : acc3;
#pragma unroll
        for (int e = 0; e < V; ++e) acc += a0[e] * b0[e];
      }
    }
    for (; k + 96 < m; k += 128) {
      const Vt v0 = rv[k], v1 = rv[k + 32], v2 = rv[k + 64], v3 = rv[k + 96];
      const Vt t0 = tv[k], t1 = tv[k + 32], t2 = tv[k + 64], t3 = tv[k + 96];
      T a0[V], a1[V], a2[V], a3[V], b0[V], b1[V], b2[V], b3[V];
      Vec16<T>::unpack(v0, a0); Vec16<T>::unpack(v1, a1); Vec16<T>::unpack(v2, a2); Vec16<T>::unpack(v3, a3);
      Vec16<T>::unpack(t0, b0); Vec16<T>::unpack(t1, b1); Vec16<T>::unpack(t2, b2); Vec16<T>::unpack(t3, b3);
#pragma unroll
      for (int u = 0; u < V; ++u) {
        acc0 += a0[u] * b0[u];
        acc1 += a1[u] * b1[u];
        acc2 += a2[u] * b2[u];
        acc3 += a3[u] * b3[u];
      }
    }
    for (; k < m; k += 32) {
      T a0[V], b0[V];
      Vec16<T>::unpack(rv[k], a0);
      Vec16<T>::unpack(tv[k], b0);
#pragma unroll
      for (int u = 0; u < V; ++u) acc0 += a0[u] * b0[u];
    }
    const int c = h + m * V + lane;  // the remainder, fewer than V entries
    if (c < p) acc1 += row[c] * ts[c];
    T acc = (acc0 + acc1) + (acc2 + acc3);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      z2[g0 + r] = acc;
      x[perm_iface[g0 + r]] = double(acc);
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_block_amax(int nblk, const int32_t *d_p, const int64_t *d_off, const T *A,
                              T *amax, cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(T) * nblk, s);
  if (e != cudaSuccess) return e;
  block_amax_kernel<T><<<dim3(64, nblk), 256, 0, s>>>(d_p, d_off, A, amax);
  return cudaGetLastError();
}

int64_t gj_scratch_elems(int nblk, int64_t sum_p, int elem_size) {
  const int no = elem_size == 8 ? BgjNO<double>::value : BgjNO<float>::value;
  return 6 * (int64_t)no * sum_p + (int64_t)(no * no + 4 * no) * nblk;
}

int64_t gj_launch_count(int pmax, int elem_size) {
  const int nb = elem_size == 8 ? BgjNB<double>::value : BgjNB<float>::value;
  const int no = elem_size == 8 ? BgjNO<double>::value : BgjNO<float>::value;
  int64_t n = 2;
  for (int k0 = 0; k0 < pmax; k0 += no)  // FP32 slabs that fit a cluster: copy, slab and six launches
    n += (elem_size == 4 && pmax - k0 <= DD_GJ_CL * DD_GJ_SLAB_THREADS) ? 8 : 2 * (no / nb) + 6;
  return n;
}

// One launch of the slab kernel: a cluster of DD_GJ_CL CTAs per block
template <int NO>
static cudaError_t launch_gj_slab(int nblk, int k0, const int32_t *d_p, float *scratch, const int64_t *d_poff,
                                  int32_t *ipiv, const float *amax, double pivtol, int32_t *failed, DevStatus *st,
                                  int code, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nblk * DD_GJ_CL));
  cfg.blockDim = dim3(DD_GJ_SLAB_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = DD_GJ_CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bgj_slab_kernel<NO>, k0, d_p, scratch, d_poff, ipiv, amax, pivtol, failed, st,
                            code);
}
// Explicit inverse of every block (in place), blocked Gauss-Jordan; blocks
// that fail the pivot test are flagged and reported through st.
template <typename T>
cudaError_t launch_gj_inverse(int nblk, const int32_t *d_p, const int64_t *d_off, int pmax, T *A,
                              int32_t *ipiv, const int64_t *d_poff, const T *amax, int32_t *failed,
                              T *scratch, double pivtol, DevStatus *st, int status_code,
                              cudaStream_t s, int tc) {
  if (nblk <= 0) return cudaSuccess;
  constexpr int NB = BgjNB<T>::value, NO = BgjNO<T>::value;
  static_assert(NO % NB == 0 && NO <= DD_BGJ_TILE, "outer block of whole inner panels");
  cudaError_t e = cudaMemsetAsync(failed, 0, sizeof(int32_t) * nblk, s);
  if (e != cudaSuccess) return e;
  const size_t smem_cap = 200 * 1024;
  const int smem_rows = (int)(smem_cap / ((NB + 1) * sizeof(T)));
  const size_t smem = (size_t)std::min(pmax, smem_rows) * (NB + 1) * sizeof(T);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(bgj_panel_kernel<T, NB, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const dim3 cg((unsigned)(((int64_t)pmax * NO + 255) / 256), nblk);
  const dim3 tg((pmax + 63) / 64, nblk);
  const dim3 sg((pmax + 255) / 256, nblk);
  const dim3 rg((pmax + 63) / 64, nblk);
  const dim3 ag(NO / 32, nblk);
  const dim3 ug((pmax + DD_BGJ_TILE - 1) / DD_BGJ_TILE, (pmax + DD_BGJ_TILE - 1) / DD_BGJ_TILE, nblk);
  for (int k0 = 0; k0 < pmax; k0 += NO) {
    bgj_copy_kernel<T, NO><<<cg, 256, 0, s>>>(k0, d_p, d_off, A, scratch, d_poff, failed);
    bool slab = false;
    if constexpr (sizeof(T) == 4) {
      // the whole slab in one launch when its rows fit a cluster's threads
      if (pmax - k0 <= DD_GJ_CL * DD_GJ_SLAB_THREADS) {
        e = launch_gj_slab<NO>(nblk, k0, d_p, reinterpret_cast<float *>(scratch), d_poff, ipiv,
                               reinterpret_cast<const float *>(amax), pivtol, failed, st, status_code, s);
        if (e != cudaSuccess) return e;
        slab = true;
      }
    }
    for (int sp = 0; sp < NO / NB && !slab; ++sp) {
      // the panel's rows in registers when they fit DD_GJ_REG_RPT per thread
      const int rpt = (pmax - k0 - NB * sp + DD_GJ_PANEL_THREADS - 1) / DD_GJ_PANEL_THREADS;
#define DD_GJ_REG(R)                                                                                     \
  case R:                                                                                                \
    bgj_panel_reg_kernel<T, NB, NO, R><<<nblk, DD_GJ_PANEL_THREADS, 0, s>>>(k0, sp, d_p, scratch, d_poff, \
                                                                          ipiv, amax, pivtol, failed, st, \
                                                                          status_code);                   \
    break;
      switch (rpt) {
        DD_GJ_REG(1)
        DD_GJ_REG(2)
        DD_GJ_REG(3)
        DD_GJ_REG(4)
        DD_GJ_REG(5)
        default:
          bgj_panel_kernel<T, NB, NO><<<nblk, DD_GJ_PANEL_THREADS, smem, s>>>(k0, sp, d_p, scratch, d_poff, ipiv,
                                                                             amax, pivtol, failed, st,
                                                                             status_code, smem_rows);
      }
#undef DD_GJ_REG
      if (sp + 1 < NO / NB) bgj_trail_kernel<T, NB, NO><<<tg, 256, 0, s>>>(k0, sp, d_p, scratch, d_poff, failed);
    }
    bgj_stage_kernel<T, NO><<<sg, 256, 0, s>>>(k0, d_p, d_off, A, scratch, d_poff, ipiv, failed);
    bgj_write_kernel<T, NO><<<sg, 256, 0, s>>>(k0, d_p, d_off, A, scratch, d_poff, failed);
    bgj_a11inv_kernel<T, NO><<<ag, 1024, 0, s>>>(k0, d_p, scratch, d_poff, failed);
    bgj_rowblock_kernel<T, NO><<<rg, 256, 0, s>>>(k0, d_p, d_off, A, scratch, d_poff, failed);
    bgj_pcol_kernel<T, NO><<<cg, 256, 0, s>>>(k0, d_p, d_off, A, scratch, d_poff, failed);
    if (tc && sizeof(T) == 4)
      bgj_update_kernel<T, NO, 1><<<ug, DD_BGJ_UPD_THREADS, 0, s>>>(k0, d_p, d_off, A, scratch, d_poff, failed);
    else
      bgj_update_kernel<T, NO><<<ug, DD_BGJ_UPD_THREADS, 0, s>>>(k0, d_p, d_off, A, scratch, d_poff, failed);
  }
  // the composite column permutation in the (now free) scratch, then the rows
  int32_t *cidx = reinterpret_cast<int32_t *>(scratch);
  const size_t psm = sizeof(int32_t) * (size_t)pmax, rsm = sizeof(T) * (size_t)pmax;
  if (psm > 48 * 1024) {
    e = cudaFuncSetAttribute(gj_colperm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    if (e != cudaSuccess) return e;
  }
  if (rsm > 48 * 1024) {
    e = cudaFuncSetAttribute(gj_unscramble_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
    if (e != cudaSuccess) return e;
  }
  gj_colperm_kernel<<<nblk, 256, psm, s>>>(d_p, ipiv, d_poff, failed, cidx);
  gj_unscramble_kernel<T><<<dim3(pmax, nblk), 256, rsm, s>>>(d_p, d_off, A, cidx, d_poff, failed);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_coo(int64_t nnz, const int64_t *idx, const double *val, T *dst,
                               cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  scatter_coo_kernel<T><<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(nnz, idx, val, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_schur_accumulate(int nj, const int32_t *jlist, const int32_t *fr_ptr, const int32_t *fr_row,
                                    const int32_t *fr_agg, const int32_t *f_ptr,
                                    const int32_t *f_col, const T *f_val, const int32_t *gam_ptr,
                                    const int32_t *gam_idx, const int32_t *gam_agg,
                                    const int64_t *x_off, const BandInfo *d_info, const T *X,
                                    const int32_t *agg_off, const int64_t *s_off, T *S,
                                    int max_fr, int max_gam, cudaStream_t s) {
  if (nj <= 0 || max_fr <= 0 || max_gam <= 0) return cudaSuccess;
  dim3 grid(nj, max_fr);
  schur_accumulate_kernel<T><<<grid, 128, 0, s>>>(jlist, fr_ptr, fr_row, fr_agg, f_ptr, f_col, f_val,
                                                  gam_ptr, gam_idx, gam_agg, x_off, d_info, X,
                                                  agg_off, s_off, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_assemble_overlapped(int ng, int k, const int32_t *agg, const int32_t *w, const int64_t *xoff,
                                       const T *Sx, T *S, cudaStream_t s) {
  const int64_t tot = (int64_t)ng * ng;
  if (tot <= 0 || k <= 0) return cudaSuccess;
  assemble_overlapped_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ng, k, agg, w, xoff, Sx, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rect_gemm(int nblk, const int32_t *dims, const int64_t *offs, int maxM, int maxN, const T *A,
                             const T *B, T *C, T alpha, T beta, cudaStream_t s) {
  if (nblk <= 0 || maxM <= 0 || maxN <= 0) return cudaSuccess;
  dim3 grid((maxN + 15) / 16, (maxM + 15) / 16, nblk);
  rect_gemm_kernel<T><<<grid, dim3(16, 16), 0, s>>>(dims, offs, A, B, C, alpha, beta);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_block_gemm(int nblk, const int32_t *d_p, const int64_t *d_off, int pmax,
                              const T *A, const T *B, T *C, T alpha, T beta, cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  dim3 grid((pmax + 15) / 16, (pmax + 15) / 16, nblk);
  block_gemm_kernel<T><<<grid, dim3(16, 16), 0, s>>>(d_p, d_off, A, B, C, alpha, beta);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mscnr_diag(int nblk, const int32_t *d_p, const int64_t *d_off, int pmax,
                              const T *Dinv, const T *E, const T *F, T *S, cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  size_t smem = sizeof(T) * 2 * (size_t)pmax;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(mscnr_diag_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  mscnr_diag_kernel<T><<<nblk, 256, smem, s>>>(d_p, d_off, Dinv, E, F, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_schur_apply(int nagg, const int32_t *agg_off, const int64_t *s_off, int pmax,
                               const T *Sinv, const int32_t *f_ptr, const int32_t *f_col,
                               const T *f_val, const double *y, const int32_t *perm_iface,
                               const T *z1, T *z2, T *t, int ng, double *x, const int32_t *agg_sys,
                               const int32_t *act, cudaStream_t s) {
  if (nagg <= 0) return cudaSuccess;
  schur_rhs_kernel<T><<<(ng + 255) / 256, 256, 0, s>>>(ng, f_ptr, f_col, f_val, y, perm_iface, z1, t);
  // V = 16 / sizeof(T) shifted copies of t, each padded to a multiple of V
  constexpr int V = 16 / sizeof(T);
  const int ldt = (pmax + V - 1) / V * V;
  size_t smem = sizeof(T) * (size_t)ldt * V;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(schur_gemv_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((pmax + DD_SROWS - 1) / DD_SROWS, nagg);
  schur_gemv_kernel<T><<<grid, 256, smem, s>>>(agg_off, s_off, Sinv, t, perm_iface, z2, x, agg_sys, act, ldt);
  return cudaGetLastError();
}

#define DD_INST_DENSE(T)                                                                          \
  template cudaError_t launch_block_amax<T>(int, const int32_t *, const int64_t *, const T *, T *, \
                                            cudaStream_t);                                         \
  template cudaError_t launch_gj_inverse<T>(int, const int32_t *, const int64_t *, int, T *,      \
                                            int32_t *, const int64_t *, const T *, int32_t *, T *, \
                                            double, DevStatus *, int, cudaStream_t, int);         \
  template cudaError_t launch_scatter_coo<T>(int64_t, const int64_t *, const double *, T *,       \
                                             cudaStream_t);                                        \
  template cudaError_t launch_assemble_overlapped<T>(int, int, const int32_t *, const int32_t *,          \
                                                     const int64_t *, const T *, T *, cudaStream_t);    \
  template cudaError_t launch_rect_gemm<T>(int, const int32_t *, const int64_t *, int, int, const T *,     \
                                           const T *, T *, T, T, cudaStream_t);                          \
  template cudaError_t launch_schur_accumulate<T>(                                                \
      int, const int32_t *, const int32_t *, const int32_t *, const int32_t *, const int32_t *,   \
      const int32_t *,                                                                            \
      const T *, const int32_t *, const int32_t *, const int32_t *, const int64_t *,              \
      const BandInfo *, const T *, const int32_t *, const int64_t *, T *, int, int, cudaStream_t); \
  template cudaError_t launch_block_gemm<T>(int, const int32_t *, const int64_t *, int, const T *, \
                                            const T *, T *, T, T, cudaStream_t);                   \
  template cudaError_t launch_mscnr_diag<T>(int, const int32_t *, const int64_t *, int, const T *, \
                                            const T *, const T *, T *, cudaStream_t);              \
  template cudaError_t launch_schur_apply<T>(int, const int32_t *, const int64_t *, int, const T *, \
                                             const int32_t *, const int32_t *, const T *,          \
                                             const double *, const int32_t *, const T *, T *, T *, \
                                             int, double *, const int32_t *, const int32_t *,      \
                                             cudaStream_t);

DD_INST_DENSE(double)
DD_INST_DENSE(float)
