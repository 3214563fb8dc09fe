// FP64 Krylov kernels of right-preconditioned restarted FGMRES (Section 5):
// CSR SpMV, classical Gram-Schmidt twice (multi-dot + update), norms, Givens
// rotations of the Hessenberg column and the final least-squares update.
// Reductions are deterministic: per-CTA partial sums are combined in a fixed
// order by a single CTA.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cooperative_groups.h>

#include "dd_internal.h"

namespace cg = cooperative_groups;

namespace {

// ---------------------------------------------------------------------------
// SpMV on C in SELL-32 form (see SellC in dd_internal.h): one thread per row,
// the 32 rows of a slice in the 32 lanes of a warp, so every load of a column
// index or a value is one coalesced 128- or 256-byte access of the warp.  The
// column indices and values of four entries are loaded before their four
// gathers of x, so each thread has several independent loads in flight.  A
// row's entries are summed in their CSR order with fused multiply-adds, as
// the oracle's plain CSR product does; the padding entries (value 0, the
// row's last column) add nothing.
//   MODE 0: y = C x;  MODE 1: y = b - C x;  MODE 2: y = C x on the rows whose
//   system is still stepping (act[row_sys[row]] != 0), others untouched.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256, 6) sell_spmv_kernel(SellC c, const double *__restrict__ x,
                                                        const double *__restrict__ b, double *__restrict__ y,
                                                        const int32_t *__restrict__ row_sys,
                                                        const int32_t *__restrict__ act) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t sl = gt >> 5;
  if (sl >= c.nslices) return;
  const int row = __ldg(&c.row[gt]);
  if (row < 0) return;  // padding row of the last slice
  if (!dd_check(c.st, row < c.n, 101)) return;
  if (MODE == 2 && !__ldg(&act[__ldg(&row_sys[row])])) return;
  const int64_t o = __ldg(&c.off[sl]);
  const int w = (int)((__ldg(&c.off[sl + 1]) - o) >> 5);
  const int32_t *cp = c.col + o + (gt & 31);
  const double *vp = c.val + o + (gt & 31);
  double acc = 0.0;
  for (int k0 = 0; k0 < w; k0 += 4) {
    int ci[4];
    double vv[4], xx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k0 + u < w) {
        ci[u] = __ldg(cp + 32 * (k0 + u));
        vv[u] = __ldg(vp + 32 * (k0 + u));
      }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k0 + u < w) xx[u] = dd_check(c.st, (unsigned)ci[u] < (unsigned)c.n, 102) ? __ldg(x + ci[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k0 + u < w) acc = fma(vv[u], xx[u], acc);
  }
  y[row] = MODE == 1 ? b[row] - acc : acc;
}

// partial[b*k + q] = sum over this CTA's rows of V_q[i] * w[i]
__global__ void multidot_kernel(int n, int k, const double *__restrict__ V, int64_t ldv,
                                const double *__restrict__ w, double *__restrict__ partial) {
  const int nb = gridDim.x;
  const int chunk = (n + nb - 1) / nb;
  const int i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  extern __shared__ double sm[];
  const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *red = sm;  // nw * k
  for (int q = 0; q < k; ++q) {
    const double *v = V + (int64_t)q * ldv;
    double s = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += v[i] * w[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp * k + q] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    double s = 0.0;
    for (int ww = 0; ww < nw; ++ww) s += red[ww * k + q];
    partial[(int64_t)blockIdx.x * k + q] = s;
  }
}

__global__ void reduce_cols_kernel(int nblocks, int k, const double *__restrict__ partial,
                                   double *out, int accumulate) {
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * k + q];
    out[q] = accumulate ? out[q] + s : s;
  }
}

// w -= V h
__global__ void gemv_sub_kernel(int n, int k, const double *__restrict__ V, int64_t ldv,
                                const double *__restrict__ h, double *__restrict__ w) {
  extern __shared__ double hs[];
  for (int q = threadIdx.x; q < k; q += blockDim.x) hs[q] = h[q];
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = w[i];
  for (int q = 0; q < k; ++q) s -= hs[q] * V[(int64_t)q * ldv + i];
  w[i] = s;
}

// dst = src / sqrt(nrm_sq[0])
__global__ void copy_scaled_kernel(int n, const double *__restrict__ src,
                                   const double *__restrict__ nrm_sq, double *__restrict__ dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = src[i] / sqrt(nrm_sq[0]);
}

// w /= norm unless the step broke down (scal[1] != 0)
__global__ void scale_kernel(int n, const double *__restrict__ scal, double *__restrict__ w) {
  if (scal[1] != 0.0) return;
  const double h = scal[0];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] /= h;
}

// Column j of H from the two CGS passes, breakdown test, previous rotations,
// the new rotation and the residual estimate.
//   hc1, hc2: the two passes' coefficients (j+1 entries)
//   nsq: [0] ||w||^2 after orthogonalisation, [1] ||w||^2 before
//   out: [0] h_{j+1,j}, [1] breakdown flag, [2] |g_{j+1}| / ||b||
__global__ void givens_kernel(int j, int R, double *H, const double *__restrict__ hc1,
                              const double *__restrict__ hc2, const double *__restrict__ nsq,
                              double *cs, double *sn, double *g, double bnorm, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q <= j; ++q) H[(int64_t)q * R + j] = hc1[q] + hc2[q];
  const double hn = sqrt(nsq[0]);
  const double w0 = sqrt(nsq[1]);
  const int breakdown = !(hn > 1e-14 * w0);
  H[(int64_t)(j + 1) * R + j] = hn;
  for (int q = 0; q < j; ++q) {
    double a = H[(int64_t)q * R + j], b = H[(int64_t)(q + 1) * R + j];
    H[(int64_t)q * R + j] = cs[q] * a + sn[q] * b;
    H[(int64_t)(q + 1) * R + j] = -sn[q] * a + cs[q] * b;
  }
  double a = H[(int64_t)j * R + j], b = H[(int64_t)(j + 1) * R + j];
  double r = hypot(a, b);
  cs[j] = a / r;
  sn[j] = b / r;
  H[(int64_t)j * R + j] = r;
  H[(int64_t)(j + 1) * R + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  out[0] = hn;
  out[1] = breakdown ? 1.0 : 0.0;
  out[2] = fabs(g[j + 1]) / bnorm;
}

// y = H(0:j,0:j)^-1 g(0:j) (upper triangular), one thread
__global__ void hess_solve_kernel(int jlast, int R, const double *__restrict__ H,
                                  const double *__restrict__ g, double *y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = jlast; q >= 0; --q) {
    double s = g[q];
    for (int c = q + 1; c <= jlast; ++c) s -= H[(int64_t)q * R + c] * y[c];
    y[q] = s / H[(int64_t)q * R + q];
  }
}

// x += Z y
__global__ void update_x_kernel(int n, int k, const double *__restrict__ y,
                                const double *__restrict__ Z, int64_t ldz, double *__restrict__ x) {
  extern __shared__ double ys[];
  for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = y[q];
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = x[i];
  for (int q = 0; q < k; ++q) s += ys[q] * Z[(int64_t)q * ldz + i];
  x[i] = s;
}

__global__ void init_g_kernel(double *g, int R, const double *__restrict__ nsq) {
  for (int q = threadIdx.x; q <= R; q += blockDim.x) g[q] = (q == 0) ? sqrt(nsq[0]) : 0.0;
}

__global__ void zero_kernel(double *p, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}

// ---------------------------------------------------------------------------
// One Arnoldi orthogonalisation step as a single cooperative kernel: classical
// Gram-Schmidt applied twice to w = V_{j+1} against V_0..V_j, the norms, the
// Givens rotation of the new Hessenberg column and the normalisation of w.
// Every CTA owns a contiguous chunk of rows.  Three grid-wide barriers:
//   A  partial dots V^T w, w^T w                          -> bufA
//   B  every CTA sums bufA (h1), w -= V h1, dots V^T w    -> bufB
//   C  every CTA sums bufB (h2), w -= V h2, partial w^T w -> bufC
//   D  every CTA sums bufC (||w||), w /= ||w|| unless breakdown;
//      CTA 0 also forms the Hessenberg column and applies the rotations.
// Each sum runs over the CTAs in the same fixed order in every CTA, so all
// CTAs hold bit-identical coefficients and results do not depend on
// scheduling.  scal: [0] h_{j+1,j}, [1] breakdown flag, [2] |g_{j+1}|/||b||
// ---------------------------------------------------------------------------
#define DD_CGS_MAXK 128  // restart lengths up to DD_CGS_MAXK - 2

// Sum over a warp of G per-lane values (G = 4, 8 or 16), transposed: each
// butterfly step hands half of the remaining values to the partner lane and
// keeps the other half, then the last value is summed over the lanes that
// share it.  On return lane l holds the warp sum of value
// v(l) = sum over the halving steps st of [bit (16 >> st) of l] * (G >> (st+1)),
// and the lanes with l % (32 / G) == 0 hold distinct values.  G - 1 + 5 -
// log2(G) FP64 additions per lane: FP64 is the scarce pipe on GB300.
template <int G>
__device__ __forceinline__ double warp_sum_t(double (&a)[G]) {
  constexpr int LOG = G == 16 ? 4 : (G == 8 ? 3 : 2);
  static_assert((1 << LOG) == G, "G must be 4, 8 or 16");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int st = 0; st < LOG; ++st) {
    const int off = 16 >> st, half = G >> (st + 1);
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int s2 = 0; s2 < half; ++s2) {
      const double give = hi ? a[s2] : a[s2 + half], keep = hi ? a[s2 + half] : a[s2];
      a[s2] = keep + __shfl_xor_sync(0xffffffffu, give, off);
    }
  }
  double e = a[0];
#pragma unroll
  for (int off = 16 >> LOG; off >= 1; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
  return e;
}

// Partial dots of the ktot = k (+1 with self: w's own square) columns over
// this CTA's rows.  Columns go in groups of 4; one pass takes up to 8 groups
// and gives each R threads (R a multiple of 32, so a warp stays inside one
// group and its loads of a column are coalesced).  A thread accumulates its
// 4 columns over rows i0 + r, i0 + r + R, ..., two rows per iteration; each
// warp then sums its 4 values by the transposed butterfly and the warps of a
// group are summed through shared memory in a fixed order.  Splitting the
// columns over threads cuts the partial sums to reduce (and the FP64 additions
// that reduce them) to R per column instead of one per CTA thread.
__device__ void block_dots(int i0, int i1, int k, const double *__restrict__ V, int64_t ldv,
                           const double *__restrict__ w, bool self, double *out, double *red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  const int ktot = k + (self ? 1 : 0);
  const int ngroups = (ktot + 3) / 4;
  for (int g0 = 0; g0 < ngroups; g0 += 8) {
    const int gn = min(8, ngroups - g0);
    const int R = (nt / gn) & ~31;
    const int cg = tid / R, rl = tid % R;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    if (cg < gn) {
      const int q0 = (g0 + cg) * 4;
      if (q0 + 4 <= k) {  // four basis columns: no tests in the loop
        const double *v0 = V + (int64_t)q0 * ldv;
        int i = i0 + rl;
        for (; i + R < i1; i += 2 * R) {
          const double wa = w[i], wb = w[i + R];
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) {
            a[s2] += v0[(int64_t)s2 * ldv + i] * wa;
            a[s2] += v0[(int64_t)s2 * ldv + i + R] * wb;
          }
        }
        if (i < i1) {
          const double wa = w[i];
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) a[s2] += v0[(int64_t)s2 * ldv + i] * wa;
        }
      } else {
        for (int i = i0 + rl; i < i1; i += R) {
          const double wi = w[i];
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) {
            const int q = q0 + s2;
            if (q < k) a[s2] += V[(int64_t)q * ldv + i] * wi;
            else if (q == k && self) a[s2] += wi * wi;
          }
        }
      }
    }
    const double ws = warp_sum_t<4>(a);
    if ((lane & 7) == 0) red[warp * 4 + ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1)] = ws;
    __syncthreads();
    if (tid < gn * 4) {
      const int gg = tid >> 2, s2 = tid & 3, q = (g0 + gg) * 4 + s2;
      if (q < ktot) {
        double t = 0.0;
        for (int ww = gg * (R >> 5); ww < (gg + 1) * (R >> 5); ++ww) t += red[ww * 4 + s2];
        out[q] = t;
      }
    }
    __syncthreads();
  }
}

// w_i - sum_q h_q V_q[i] as one chain of fused multiply-adds: on GB300 the
// FP64 pipe's issue rate, not its latency, bounds this loop, so extra
// accumulators would only add the FP64 additions that combine them; the
// loads are independent of the chain and stay in flight
__device__ __forceinline__ double row_update(int i, int k, const double *__restrict__ V, int64_t ldv,
                                             const double *hs, double wi) {
  double s = wi;
#pragma unroll 8
  for (int q = 0; q < k; ++q) s = fma(-hs[q], V[(int64_t)q * ldv + i], s);
  return s;
}

// The rows, CTAs and per-system state a CTA works on.  With one system the
// CTA owns chunk b of [0, n) and the state arrays hold one system; with
// several, CTA b belongs to system cta_seg[b] and owns a chunk of its rows.
struct SegCta {
  int s, c0, nc;   // system, its first CTA, its CTA count
  int64_t i0, i1;  // this CTA's rows
  bool act;        // the system takes this step
};
__device__ __forceinline__ SegCta seg_cta(const SegMap &sm, int b, int nb, int64_t n) {
  SegCta c;
  int64_t r0 = 0, r1 = n;
  if (sm.nseg == 1) {
    c.s = 0; c.c0 = 0; c.nc = nb;
  } else {
    c.s = sm.cta_seg[b];
    c.c0 = sm.seg_cta0[c.s];
    c.nc = sm.seg_cta0[c.s + 1] - c.c0;
    r0 = sm.seg_row0[c.s];
    r1 = sm.seg_row0[c.s + 1];
  }
  const int64_t ns = r1 - r0, chunk = (ns + c.nc - 1) / c.nc;
  c.i0 = r0 + min(ns, (int64_t)(b - c.c0) * chunk);
  c.i1 = min(r1, c.i0 + chunk);
  c.act = sm.act ? sm.act[c.s] != 0 : true;
  if (!c.act) c.i1 = c.i0;
  return c;
}

// Every CTA of a system sums the system's partials of `ncols` columns over
// its CTAs itself, in one fixed order, so every CTA holds the same bits and
// no grid barrier is needed to share the sums: warp w takes columns w,
// w + nw, ..., lane l the CTAs c0 + l, c0 + l + 32, ..., then a butterfly.
// out[q] in shared memory; the system's first CTA also stores them to dst.
__device__ void cta_column_sums(const SegCta &me, int b, int ncols, int pk, const double *__restrict__ partial,
                                double *out, double *dst) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = warp; q < ncols; q += nw) {
    double t = 0.0;
    for (int c = me.c0 + lane; c < me.c0 + me.nc; c += 32) t += partial[(int64_t)c * pk + q];
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      out[q] = t;
      if (b == me.c0) dst[q] = t;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One Arnoldi orthogonalisation step as a single cooperative kernel: classical
// Gram-Schmidt applied twice to w = V_{j+1} against V_0..V_j, the norms, the
// Givens rotation of the new Hessenberg column and the normalisation of w,
// for one system or for every active system of a batch at once (each system
// its own rows, CTAs, sums and Hessenberg matrix).  Three grid-wide
// barriers follow
//   1 partial dots V^T w, w^T w            every CTA then sums the system's
//                                            partials itself -> h1
//   2 w -= V h1, partial dots V^T w        every CTA: -> h2
//   3 w -= V h2, partial w^T w             every CTA: the system's norm from
//                                            the partials, w *= 1/h_{j+1,j}
//                                            unless breakdown; the system's
//                                            first CTA: Hessenberg column and
//                                            rotations
// Every CTA sums the partials in the same fixed order, so all hold the same
// h1, h2 and norm without a barrier to share them.
// The FP64 pipe bounds this kernel on GB300; the redundant sums cost each
// CTA (2k+1) times the system's CTA count additions, against the
// ~4(k+1)n / CTAs multiply-adds of its rows.
// Per-system state (strides from sm.rmax): hc1/hc2 rmax+2, H (rmax+1)*rmax
// with row stride R, cs/sn rmax, g rmax+1, bn2 (||b||^2) 1, scal 4:
// [0] h_{j+1,j}, [1] breakdown flag, [2] |g_{j+1}| / ||b||.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT) cgs2_kernel(
    int64_t n, int j, int R, const double *__restrict__ V, int64_t ldv, double *w, double *partial,
    int pk, double *hc1, double *hc2, double *H, double *cs, double *sn, double *g,
    const double *__restrict__ bn2, double *scal, SegMap sm) {
  cg::grid_group grid = cg::this_grid();
  const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  sm.nctas = nb;
  const SegCta me = seg_cta(sm, b, nb, n);
  const int i0 = (int)me.i0, i1 = (int)me.i1;
  const int k = j + 1, hst = sm.rmax + 2;
  __shared__ double red[(NT / 32) * 16];
  __shared__ double hs[DD_CGS_MAXK + 8];
  __shared__ double hs1[DD_CGS_MAXK + 8], hs2[DD_CGS_MAXK + 8];
  // pass 1 and the final norm use the partials in buffer A, pass 2 buffer B
  // (a CTA may still read pass 1's partials while another writes pass 2's)
  double *partB = partial + (int64_t)nb * pk;
  // 1
  block_dots(i0, i1, k, V, ldv, w, true, partial + (int64_t)b * pk, red);
  grid.sync();
  // 2: every CTA: h1[0..k-1] and h1[k] = ||w||^2 before orthogonalisation
  if (me.act) cta_column_sums(me, b, k + 1, pk, partial, hs1, hc1 + (int64_t)me.s * hst);
  // 3
  for (int i = i0 + tid; i < i1; i += blockDim.x) w[i] = row_update(i, k, V, ldv, hs1, w[i]);
  __syncthreads();
  block_dots(i0, i1, k, V, ldv, w, false, partB + (int64_t)b * pk, red);
  grid.sync();
  // 4: every CTA: h2
  if (me.act) cta_column_sums(me, b, k, pk, partB, hs2, hc2 + (int64_t)me.s * hst);
  // 5
  {
    double nn = 0.0;
    for (int i = i0 + tid; i < i1; i += blockDim.x) {
      const double s2 = row_update(i, k, V, ldv, hs2, w[i]);
      w[i] = s2;
      nn += s2 * s2;
    }
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane == 0) red[warp] = nn;
    __syncthreads();
    if (tid == 0) {
      double u = 0.0;
      for (int ww = 0; ww < nw; ++ww) u += red[ww];
      partial[(int64_t)b * pk] = u;
    }
  }
  grid.sync();
  // 6: every CTA of a system sums the system's ||w||^2 partials in the same
  // fixed order (so all hold the same bits), scales its own rows by 1/h_{j+1,j}
  // unless the step broke down, and the system's first CTA also forms the
  // Hessenberg column and applies the rotations; no further grid barrier
  if (me.act) {
    const int sys = me.s;
    const double *h1 = hs1, *h2 = hs2;
    {
      const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
      double t = 0.0;
      for (int c = me.c0 + tid; c < me.c0 + me.nc; c += blockDim.x) t += partial[(int64_t)c * pk];
      for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) red[warp] = t;
      __syncthreads();
      if (tid == 0) {
        double u = 0.0;
        for (int ww = 0; ww < nw; ++ww) u += red[ww];
        hs[DD_CGS_MAXK] = u;
      }
      __syncthreads();
    }
    const double hn = sqrt(hs[DD_CGS_MAXK]);
    const bool breakdown = !(hn > 1e-14 * sqrt(h1[k]));
    if (!breakdown) {
      const double inv = 1.0 / hn;
      for (int i = i0 + tid; i < i1; i += blockDim.x) w[i] *= inv;
    }
    if (b == me.c0) {
      double *Hs = H + (int64_t)sys * (sm.rmax + 1) * sm.rmax;
      double *css = cs + (int64_t)sys * sm.rmax, *sns = sn + (int64_t)sys * sm.rmax;
      double *gs = g + (int64_t)sys * (sm.rmax + 1), *scs = scal + (int64_t)sys * 4;
      // column j of H (passes 1 + 2) and the rotations, in shared memory
      __syncthreads();
      for (int q = tid; q <= j; q += blockDim.x) hs[q] = h1[q] + h2[q];
      __syncthreads();
      if (tid == 0) {
        hs[j + 1] = hn;
        for (int q = 0; q < j; ++q) {
          const double a = hs[q], c2 = hs[q + 1], c = css[q], sv = sns[q];
          hs[q] = c * a + sv * c2;
          hs[q + 1] = -sv * a + c * c2;
        }
        const double a = hs[j], c2 = hs[j + 1];
        const double r = hypot(a, c2);
        css[j] = a / r;
        sns[j] = c2 / r;
        hs[j] = r;
        hs[j + 1] = 0.0;
        const double gj = gs[j];
        gs[j + 1] = -sns[j] * gj;
        gs[j] = css[j] * gj;
        scs[0] = hn;
        scs[1] = breakdown ? 1.0 : 0.0;
        scs[2] = fabs(gs[j + 1]) / sqrt(bn2[sys]);
      }
      __syncthreads();
      for (int q = tid; q <= j + 1; q += blockDim.x) Hs[(int64_t)q * R + j] = hs[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Batched helpers: the same per-system quantities as the single-system
// kernels above, over a SegMap.
// ---------------------------------------------------------------------------
// partial[b] = sum of v[i]^2 over CTA b's rows (every system, active or not)
__global__ void seg_sumsq_kernel(int64_t n, const double *__restrict__ v, double *partial, SegMap sm) {
  sm.act = nullptr;
  sm.nctas = gridDim.x;
  const SegCta me = seg_cta(sm, blockIdx.x, gridDim.x, n);
  __shared__ double red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double t = 0.0;
  for (int64_t i = me.i0 + tid; i < me.i1; i += blockDim.x) t += v[i] * v[i];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) red[warp] = t;
  __syncthreads();
  if (tid == 0) {
    double u = 0.0;
    for (int ww = 0; ww < nw; ++ww) u += red[ww];
    partial[blockIdx.x] = u;
  }
}

// out[s] = sum of partial over system s's CTAs, in order (one CTA per system)
__global__ void seg_reduce_kernel(const double *__restrict__ partial, double *out, SegMap sm) {
  const int sys = blockIdx.x;
  const int b0 = sm.seg_cta0[sys], b1 = sm.seg_cta0[sys + 1];
  __shared__ double red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double t = 0.0;
  for (int b = b0 + tid; b < b1; b += blockDim.x) t += partial[b];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) red[warp] = t;
  __syncthreads();
  if (tid == 0) {
    double u = 0.0;
    for (int ww = 0; ww < nw; ++ww) u += red[ww];
    out[sys] = u;
  }
}

// start of a cycle for the active systems: v0 = r / ||r||, g = ||r|| e_0
__global__ void seg_start_kernel(int64_t n, const double *__restrict__ r, const double *__restrict__ nsq,
                                 double *v0, double *g, SegMap sm) {
  sm.nctas = gridDim.x;
  const SegCta me = seg_cta(sm, blockIdx.x, gridDim.x, n);
  if (me.act) {
    const double nr = sqrt(nsq[me.s]);
    for (int64_t i = me.i0 + threadIdx.x; i < me.i1; i += blockDim.x) v0[i] = r[i] / nr;
  }
  if (blockIdx.x == me.c0 && me.act)
    for (int q = threadIdx.x; q <= sm.rmax; q += blockDim.x)
      g[(int64_t)me.s * (sm.rmax + 1) + q] = (q == 0) ? sqrt(nsq[me.s]) : 0.0;
}

// y_s = H_s(0:jl,0:jl)^-1 g_s(0:jl) for every system with jl[s] >= 0
__global__ void seg_hess_solve_kernel(int R, const int32_t *__restrict__ jl, const double *__restrict__ H,
                                      const double *__restrict__ g, double *y, SegMap sm) {
  const int sys = blockIdx.x;
  const int jlast = jl[sys];
  if (threadIdx.x != 0 || jlast < 0) return;
  const double *Hs = H + (int64_t)sys * (sm.rmax + 1) * sm.rmax;
  const double *gs = g + (int64_t)sys * (sm.rmax + 1);
  double *ys = y + (int64_t)sys * (sm.rmax + 1);
  for (int q = jlast; q >= 0; --q) {
    double t = gs[q];
    for (int c = q + 1; c <= jlast; ++c) t -= Hs[(int64_t)q * R + c] * ys[c];
    ys[q] = t / Hs[(int64_t)q * R + q];
  }
}

// x += Z y_s over the rows of every system with jl[s] >= 0
__global__ void seg_update_x_kernel(int64_t n, const int32_t *__restrict__ jl, const double *__restrict__ y,
                                    const double *__restrict__ Z, int64_t ldz, double *x, SegMap sm) {
  sm.act = nullptr;
  sm.nctas = gridDim.x;
  const SegCta me = seg_cta(sm, blockIdx.x, gridDim.x, n);
  const int k = jl[me.s] + 1;
  if (k <= 0) return;
  __shared__ double ys[DD_CGS_MAXK];
  for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = y[(int64_t)me.s * (sm.rmax + 1) + q];
  __syncthreads();
  for (int64_t i = me.i0 + threadIdx.x; i < me.i1; i += blockDim.x) {
    double t = x[i];
    for (int q = 0; q < k; ++q) t += ys[q] * Z[(int64_t)q * ldz + i];
    x[i] = t;
  }
}

}  // namespace

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// FP64 multiply-add rate: every thread runs 8 independent chains of dependent
// FMAs (a <- a * b + c); the result goes to a file-scope sink so the chains
// are not removed.  FMAs per launch: blocks * 256 * 8 * iters.
// ---------------------------------------------------------------------------
__device__ double g_fma_sink;

__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = 1e-3 * (threadIdx.x + u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(a[u], b, c);
  }
  double t = 0.0;
#pragma unroll
  for (int u = 0; u < 8; ++u) t += a[u];
  if (t == 12345.678) g_fma_sink = t;  // never true for the probe's inputs
}

cudaError_t launch_fma_probe(int blocks, int iters, cudaStream_t s) {
  fma_probe_kernel<<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-7);
  return cudaGetLastError();
}

static inline unsigned sell_blocks(const SellC &c) { return (unsigned)((c.nslices * 32 + 255) / 256); }

cudaError_t launch_spmv(const SellC &c, const double *x, double *y, cudaStream_t s) {
  if (c.nslices <= 0) return cudaSuccess;
  sell_spmv_kernel<0><<<sell_blocks(c), 256, 0, s>>>(c, x, nullptr, y, nullptr, nullptr);
  return cudaGetLastError();
}
cudaError_t launch_spmv_masked(const SellC &c, const double *x, double *y, const int32_t *row_sys,
                               const int32_t *act, cudaStream_t s) {
  if (c.nslices <= 0) return cudaSuccess;
  sell_spmv_kernel<2><<<sell_blocks(c), 256, 0, s>>>(c, x, nullptr, y, row_sys, act);
  return cudaGetLastError();
}
cudaError_t launch_residual(const SellC &c, const double *x, const double *b, double *r, cudaStream_t s) {
  if (c.nslices <= 0) return cudaSuccess;
  sell_spmv_kernel<1><<<sell_blocks(c), 256, 0, s>>>(c, x, b, r, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_multidot(int n, int k, const double *V, int64_t ldv, const double *w,
                            double *partial, int nblocks, cudaStream_t s) {
  size_t smem = sizeof(double) * 8 * (size_t)k;
  multidot_kernel<<<nblocks, 256, smem, s>>>(n, k, V, ldv, w, partial);
  return cudaGetLastError();
}

cudaError_t launch_reduce_cols(int nblocks, int k, const double *partial, double *out,
                               int accumulate, cudaStream_t s) {
  reduce_cols_kernel<<<1, 64, 0, s>>>(nblocks, k, partial, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_gemv_sub(int n, int k, const double *V, int64_t ldv, const double *h,
                            double *w, cudaStream_t s) {
  gemv_sub_kernel<<<nblk(n, 256), 256, sizeof(double) * (size_t)k, s>>>(n, k, V, ldv, h, w);
  return cudaGetLastError();
}

cudaError_t launch_copy_scaled(int n, const double *src, const double *nrm_sq, double *dst,
                               cudaStream_t s) {
  copy_scaled_kernel<<<nblk(n, 256), 256, 0, s>>>(n, src, nrm_sq, dst);
  return cudaGetLastError();
}

cudaError_t launch_scale_by(int n, const double *scal, double *w, cudaStream_t s) {
  scale_kernel<<<nblk(n, 256), 256, 0, s>>>(n, scal, w);
  return cudaGetLastError();
}

cudaError_t launch_givens2(int j, int R, double *H, const double *hc1, const double *hc2,
                           const double *nsq, double *cs, double *sn, double *g, double bnorm,
                           double *out, cudaStream_t s) {
  givens_kernel<<<1, 32, 0, s>>>(j, R, H, hc1, hc2, nsq, cs, sn, g, bnorm, out);
  return cudaGetLastError();
}

cudaError_t launch_hess_solve_update(int n, int jlast, int R, const double *H, const double *g,
                                     double *y, const double *Z, int64_t ldz, double *x,
                                     cudaStream_t s) {
  hess_solve_kernel<<<1, 32, 0, s>>>(jlast, R, H, g, y);
  update_x_kernel<<<nblk(n, 256), 256, sizeof(double) * (size_t)(jlast + 1), s>>>(n, jlast + 1, y,
                                                                                   Z, ldz, x);
  return cudaGetLastError();
}

cudaError_t launch_init_g(double *g, int R, const double *nsq, cudaStream_t s) {
  init_g_kernel<<<1, 64, 0, s>>>(g, R, nsq);
  return cudaGetLastError();
}

// blocks of the cooperative CGS2 kernel that can be resident at once (capped)
template <int NT>
static int cgs2_blocks_t(int per_sm, int cap) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cgs2_kernel<NT>, NT, 0) != cudaSuccess) return 0;
  const int want = per_sm > 0 ? per_sm : 2;
  int nb = sms * (per < want ? per : want);
  return nb < cap ? nb : cap;
}
int cgs2_blocks(int per_sm, int cap, int threads) {
  return threads == 512 ? cgs2_blocks_t<512>(per_sm, cap) : cgs2_blocks_t<256>(per_sm, cap);
}
cudaError_t launch_cgs2(int64_t n, int j, int R, const double *V, int64_t ldv, double *w, double *partial,
                        int pk, double *hc1, double *hc2, double *H, double *cs, double *sn, double *g,
                        const double *bn2, double *scal, const SegMap &sm, int nblocks, int threads,
                        cudaStream_t s) {
  SegMap m2 = sm;
  void *args[] = {&n, &j, &R, (void *)&V, &ldv, &w, &partial, &pk, &hc1, &hc2, &H, &cs, &sn, &g,
                  (void *)&bn2, &scal, &m2};
  if (threads == 512)
    return cudaLaunchCooperativeKernel((const void *)cgs2_kernel<512>, dim3(nblocks), dim3(512), args, 0, s);
  return cudaLaunchCooperativeKernel((const void *)cgs2_kernel<256>, dim3(nblocks), dim3(256), args, 0, s);
}

cudaError_t launch_seg_norms(int64_t n, const double *v, double *partial, double *out, const SegMap &sm,
                             int nblocks, cudaStream_t s) {
  seg_sumsq_kernel<<<nblocks, 256, 0, s>>>(n, v, partial, sm);
  seg_reduce_kernel<<<sm.nseg, 256, 0, s>>>(partial, out, sm);
  return cudaGetLastError();
}

cudaError_t launch_seg_start(int64_t n, const double *r, const double *nsq, double *v0, double *g,
                             const SegMap &sm, int nblocks, cudaStream_t s) {
  seg_start_kernel<<<nblocks, 256, 0, s>>>(n, r, nsq, v0, g, sm);
  return cudaGetLastError();
}

cudaError_t launch_seg_hess_update(int64_t n, int R, const int32_t *jl, const double *H, const double *g,
                                   double *y, const double *Z, int64_t ldz, double *x, const SegMap &sm,
                                   int nblocks, cudaStream_t s) {
  seg_hess_solve_kernel<<<sm.nseg, 32, 0, s>>>(R, jl, H, g, y, sm);
  seg_update_x_kernel<<<nblocks, 256, 0, s>>>(n, jl, y, Z, ldz, x, sm);
  return cudaGetLastError();
}

cudaError_t launch_zero(double *p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  zero_kernel<<<nblk(n, 256), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}
