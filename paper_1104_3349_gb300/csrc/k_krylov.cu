// FP64 Krylov kernels of right-preconditioned restarted FGMRES (Section 5):
// CSR SpMV, classical Gram-Schmidt twice (multi-dot + update), norms, Givens
// rotations of the Hessenberg column and the final least-squares update.
// Reductions are deterministic: per-CTA partial sums are combined in a fixed
// order by a single CTA.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dd_internal.h"

namespace {

// one thread per row; rows of C hold at most a handful of entries
__global__ void spmv_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ x,
                            double *__restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * __ldg(&x[col[k]]);
  y[i] = s;
}

__global__ void residual_kernel(int n, const int32_t *__restrict__ rowptr,
                                const int32_t *__restrict__ col, const double *__restrict__ val,
                                const double *__restrict__ x, const double *__restrict__ b,
                                double *__restrict__ r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * __ldg(&x[col[k]]);
  r[i] = b[i] - s;
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

}  // namespace

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_spmv(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                        const double *x, double *y, cudaStream_t s) {
  spmv_kernel<<<nblk(n, 256), 256, 0, s>>>(n, rowptr, col, val, x, y);
  return cudaGetLastError();
}

cudaError_t launch_residual(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                            const double *x, const double *b, double *r, cudaStream_t s) {
  residual_kernel<<<nblk(n, 256), 256, 0, s>>>(n, rowptr, col, val, x, b, r);
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

cudaError_t launch_zero(double *p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  zero_kernel<<<nblk(n, 256), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}
