// The learned Schur correction (not in the paper; an extension of the lumped
// approximation LUM, Definition of B_LUM): per-entry features of an
// aggregate block, the 14 -> 64 -> 1 ReLU network that maps them to the
// correction Delta, and the network's training (forward, backward, Adam).
//
// Precision: inputs and weights are rounded to BF16 (round to nearest even)
// and every product is accumulated in FP32.  The features themselves are
// FP64 (they read C).  The contraction has K = 14 and one output per entry,
// so tensor-core tiles would be idle; FP32 FMAs on the CUDA cores do it.
// Gradients are summed per CTA over a fixed row range, then over CTAs in
// index order, so training is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "dd_internal.h"

#define NIN DD_MLP_IN
#define NHID DD_MLP_HIDDEN
#define NPAR DD_MLP_NPARAM
#define OFF_B1 (NHID * NIN)
#define OFF_W2 (NHID * NIN + NHID)
#define OFF_B2 (NHID * NIN + 2 * NHID)
#define XPAD 16  // BF16 features per stored row (32 bytes)

namespace {

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// out = w2 . relu(W1 x + b1) + b2 with weights W (BF16 values held as float,
// in shared memory); z receives W1 x + b1
__device__ __forceinline__ float mlp_fwd(const float *__restrict__ W, const float (&x)[NIN], float (&z)[NHID]) {
  float out = W[OFF_B2];
#pragma unroll
  for (int j = 0; j < NHID; ++j) {
    float a = W[OFF_B1 + j];
#pragma unroll
    for (int k = 0; k < NIN; ++k) a = fmaf(W[j * NIN + k], x[k], a);
    z[j] = a;
    out = fmaf(W[OFF_W2 + j], fmaxf(a, 0.f), out);
  }
  return out;
}

// ---------------------------------------------------------------------------
// Setup of DD_LEARNED: one thread per pattern entry.  Features in FP64 from
// C (G entries), F, E, E^T and diag(D); then normalise, BF16, the network,
// and Delta added to the entry of the dense block S (which holds G already).
// ---------------------------------------------------------------------------
// value of C(i, j) (original numbering), 0 if not stored
__device__ __forceinline__ double c_at(const LearnedArgs &a, int i, int j) {
  for (int k = a.c_rowptr[i]; k < a.c_rowptr[i + 1]; ++k)
    if (a.c_col[k] == j) return a.c_val[k];
  return 0.0;
}
// E(k, c): interior row k, interface column c
__device__ __forceinline__ double e_at(const LearnedArgs &a, int k, int c) {
  for (int q = a.e_ptr[k]; q < a.e_ptr[k + 1]; ++q)
    if (a.e_col[q] == c) return a.e_val[q];
  return 0.0;
}

template <typename T>
__global__ void learned_delta_kernel(LearnedArgs a, T *S) {
  __shared__ float W[NPAR];
  for (int q = threadIdx.x; q < NPAR; q += blockDim.x) W[q] = a.wbf[q];
  __syncthreads();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n_ent) return;
  const int ag = a.ent[3 * e], r = a.ent[3 * e + 1], c = a.ent[3 * e + 2];
  const int g0 = a.agg_off[ag], p = a.agg_off[ag + 1] - g0;
  const int R = g0 + r, Cc = g0 + c;
  const int oR = a.perm_iface[R], oC = a.perm_iface[Cc];
  double f[NIN];
  f[0] = c_at(a, oR, oC);
  f[1] = c_at(a, oC, oR);
  const double grr = c_at(a, oR, oR), gcc = c_at(a, oC, oC);
  double fe = 0.0, fde = 0.0, fde_rr = 0.0, fabs_r = 0.0, cnt_r = 0.0;
  for (int q = a.f_ptr[R]; q < a.f_ptr[R + 1]; ++q) {
    const double fv = a.f_val[q];
    if (fv == 0.0) continue;
    const int k = a.f_col[q];
    const double dk = a.dinv[k];
    const double ec = e_at(a, k, Cc), er = e_at(a, k, R);
    fe += fv * ec;
    fde += fv * dk * ec;
    fde_rr += fv * dk * er;
    fabs_r += fabs(fv);
    cnt_r += 1.0;
  }
  double eabs_c = 0.0, cnt_c = 0.0;
  for (int q = a.et_ptr[Cc]; q < a.et_ptr[Cc + 1]; ++q) {
    const double ev = a.et_val[q];
    if (ev == 0.0) continue;
    eabs_c += fabs(ev);
    cnt_c += 1.0;
  }
  f[2] = fe;
  f[3] = fde;
  f[4] = (r == c) ? 1.0 : 0.0;
  f[5] = (grr == 0.0) ? 1.0 : 0.0;
  f[6] = (gcc == 0.0) ? 1.0 : 0.0;
  f[7] = grr;
  f[8] = gcc;
  f[9] = fabs_r;
  f[10] = eabs_c;
  f[11] = cnt_r / 8.0;
  f[12] = cnt_c / 8.0;
  f[13] = fde_rr;
  float x[NIN], z[NHID];
#pragma unroll
  for (int k = 0; k < NIN; ++k) {
    if (a.feat) a.feat[e * NIN + k] = f[k];
    x[k] = bf16r(__double2float_rn((f[k] - a.mean[k]) / a.stdv[k]));
  }
  const float d = a.out_scale * mlp_fwd(W, x, z);
  if (a.delta) a.delta[e] = d;
  T *blk = S + a.s_off[ag];
  blk[(int64_t)r * p + c] += T(d);
}

// ---------------------------------------------------------------------------
// Training.  One CTA takes tiles of 256 rows (CTA b: tiles b, b + G, ...);
// each thread one row of the tile: forward with the BF16 weights, the
// residual, and the row's dz = dout * w2 * [z > 0] and h into shared memory;
// then each thread sums its gradient entries over the tile's rows.  The
// per-CTA sums over tiles and the sum over CTAs run in fixed order.
// ---------------------------------------------------------------------------
#define TR 256
#define DZ_LD (NHID + 1)
#define X_LD (NIN + 1)
constexpr size_t kGradSmem = sizeof(float) * ((size_t)NPAR + (size_t)TR * X_LD + 2 * (size_t)TR * DZ_LD + TR);

__global__ void __launch_bounds__(TR) mlp_grad_kernel(const __nv_bfloat16 *__restrict__ X,
                                                      const float *__restrict__ y, int64_t lo, int64_t hi,
                                                      const float *__restrict__ wbf, float *partial,
                                                      double *lossp) {
  extern __shared__ __align__(16) float sm[];
  float *W = sm, *xs = W + NPAR, *dz = xs + TR * X_LD, *hs = dz + TR * DZ_LD, *dout = hs + TR * DZ_LD;
  const int tid = threadIdx.x;
  for (int q = tid; q < NPAR; q += TR) W[q] = wbf[q];
  const int64_t n = hi - lo;
  const float inv_n2 = 2.0f / (float)n;
  float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  double lsum = 0.0;
  const int64_t ntiles = (n + TR - 1) / TR;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();  // W staged / previous tile consumed
    const int64_t e = lo + t * TR + tid;
    float x[NIN], z[NHID];
    const bool live = e < hi;
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = live ? __bfloat162float(X[e * XPAD + k]) : 0.f;
    float out = mlp_fwd(W, x, z);
    const float r = live ? out - y[e] : 0.f;
    lsum += (double)r * (double)r;
    const float g = r * inv_n2;
#pragma unroll
    for (int k = 0; k < NIN; ++k) xs[tid * X_LD + k] = x[k];
#pragma unroll
    for (int j = 0; j < NHID; ++j) {
      dz[tid * DZ_LD + j] = (z[j] > 0.f) ? g * W[OFF_W2 + j] : 0.f;
      hs[tid * DZ_LD + j] = live ? fmaxf(z[j], 0.f) : 0.f;
    }
    dout[tid] = g;
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const int q = tid + s * TR;
      if (q >= NPAR) break;
      float v = 0.f;
      if (q < OFF_B1) {
        const int j = q / NIN, k = q % NIN;
        for (int i = 0; i < TR; ++i) v = fmaf(dz[i * DZ_LD + j], xs[i * X_LD + k], v);
      } else if (q < OFF_W2) {
        const int j = q - OFF_B1;
        for (int i = 0; i < TR; ++i) v += dz[i * DZ_LD + j];
      } else if (q < OFF_B2) {
        const int j = q - OFF_W2;
        for (int i = 0; i < TR; ++i) v = fmaf(hs[i * DZ_LD + j], dout[i], v);
      } else {
        for (int i = 0; i < TR; ++i) v += dout[i];
      }
      acc[s] += v;
    }
  }
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int q = tid + s * TR;
    if (q < NPAR) partial[(int64_t)blockIdx.x * NPAR + q] = acc[s];
  }
  // loss: the CTA's threads in order
  __shared__ double ls[TR];
  ls[tid] = lsum;
  __syncthreads();
  if (tid == 0) {
    double u = 0.0;
    for (int i = 0; i < TR; ++i) u += ls[i];
    lossp[blockIdx.x] = u;
  }
}

// grad[q] = sum over CTAs in order; loss = sum / n
__global__ void mlp_reduce_kernel(const float *__restrict__ partial, const double *__restrict__ lossp,
                                  int nblocks, int64_t n, float *grad, double *loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < NPAR) {
    float v = 0.f;
    for (int b = 0; b < nblocks; ++b) v += partial[(int64_t)b * NPAR + q];
    grad[q] = v;
  }
  if (q == 0) {
    double u = 0.0;
    for (int b = 0; b < nblocks; ++b) u += lossp[b];
    *loss = u / (double)n;
  }
}

// bias-corrected Adam on the FP32 master weights, then their BF16 copy
__global__ void mlp_adam_kernel(float *p, float *m, float *v, float *wbf, const float *__restrict__ grad,
                                float lr, float b1, float b2, float eps, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NPAR) return;
  const float g = grad[q];
  const float mq = b1 * m[q] + (1.f - b1) * g;
  const float vq = b2 * v[q] + (1.f - b2) * g * g;
  m[q] = mq;
  v[q] = vq;
  const float pq = p[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  p[q] = pq;
  wbf[q] = bf16r(pq);
}

__global__ void mlp_round_kernel(const float *__restrict__ p, float *wbf) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < NPAR) wbf[q] = bf16r(p[q]);
}

__global__ void mlp_pack_kernel(const float *__restrict__ Xf, int64_t n, __nv_bfloat16 *X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * XPAD) return;
  const int64_t e = i / XPAD;
  const int k = (int)(i % XPAD);
  X[i] = __float2bfloat16_rn(k < NIN ? Xf[e * NIN + k] : 0.f);
}

__global__ void mlp_predict_kernel(const __nv_bfloat16 *__restrict__ X, int64_t lo, int64_t hi,
                                   const float *__restrict__ wbf, float *out) {
  __shared__ float W[NPAR];
  for (int q = threadIdx.x; q < NPAR; q += blockDim.x) W[q] = wbf[q];
  __syncthreads();
  const int64_t e = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= hi) return;
  float x[NIN], z[NHID];
#pragma unroll
  for (int k = 0; k < NIN; ++k) x[k] = __bfloat162float(X[e * XPAD + k]);
  out[e - lo] = mlp_fwd(W, x, z);
}

}  // namespace

template <typename T>
cudaError_t launch_learned_delta(const LearnedArgs &a, T *S, cudaStream_t s) {
  if (a.n_ent <= 0) return cudaSuccess;
  learned_delta_kernel<T><<<(unsigned)((a.n_ent + 127) / 128), 128, 0, s>>>(a, S);
  return cudaGetLastError();
}
template cudaError_t launch_learned_delta<float>(const LearnedArgs &, float *, cudaStream_t);
template cudaError_t launch_learned_delta<double>(const LearnedArgs &, double *, cudaStream_t);

// ---------------------------------------------------------------------------
// Training handle and its C entry points
// ---------------------------------------------------------------------------
namespace {

struct MlpHandle {
  float *p = nullptr, *m = nullptr, *v = nullptr, *wbf = nullptr, *grad = nullptr, *partial = nullptr;
  double *lossp = nullptr, *loss = nullptr;
  __nv_bfloat16 *X = nullptr;
  float *y = nullptr;
  int64_t n = 0, step = 0;
  int nblocks = 0;
};

dd_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? DD_OK : (e == cudaErrorMemoryAllocation ? DD_ERR_OOM : DD_ERR_CUDA); }

#define MCK(x)                                   \
  do {                                           \
    dd_status r_ = cuda_ok(x);                   \
    if (r_ != DD_OK) return r_;                  \
  } while (0)

dd_status grad_on(MlpHandle *h, int64_t lo, int64_t hi, cudaStream_t s) {
  if (lo < 0 || hi > h->n || hi <= lo) return DD_ERR_INVALID_ARG;
  MCK(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem));
  const int64_t tiles = (hi - lo + TR - 1) / TR;
  const int nb = (int)std::min<int64_t>(h->nblocks, tiles);
  mlp_grad_kernel<<<nb, TR, kGradSmem, s>>>(h->X, h->y, lo, hi, h->wbf, h->partial, h->lossp);
  MCK(cudaGetLastError());
  mlp_reduce_kernel<<<(NPAR + 255) / 256, 256, 0, s>>>(h->partial, h->lossp, nb, hi - lo, h->grad, h->loss);
  MCK(cudaGetLastError());
  return DD_OK;
}

}  // namespace

extern "C" {

dd_status dd_mlp_create(const float *params, void **mlp) {
  if (!params || !mlp) return DD_ERR_INVALID_ARG;
  *mlp = nullptr;
  MlpHandle *h = new (std::nothrow) MlpHandle();
  if (!h) return DD_ERR_OOM;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  h->nblocks = std::max(1, sms);  // one CTA per SM (~150 KB of shared memory each)
  float **bufs[] = {&h->p, &h->m, &h->v, &h->wbf, &h->grad};
  for (float **b : bufs)
    if (cudaMalloc(b, sizeof(float) * NPAR) != cudaSuccess) { dd_mlp_destroy(h); return DD_ERR_OOM; }
  if (cudaMalloc(&h->partial, sizeof(float) * NPAR * (size_t)h->nblocks) != cudaSuccess ||
      cudaMalloc(&h->lossp, sizeof(double) * (size_t)h->nblocks) != cudaSuccess ||
      cudaMalloc(&h->loss, sizeof(double)) != cudaSuccess) {
    dd_mlp_destroy(h);
    return DD_ERR_OOM;
  }
  if (cudaMemcpy(h->p, params, sizeof(float) * NPAR, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->m, 0, sizeof(float) * NPAR) != cudaSuccess ||
      cudaMemset(h->v, 0, sizeof(float) * NPAR) != cudaSuccess) {
    dd_mlp_destroy(h);
    return DD_ERR_CUDA;
  }
  mlp_round_kernel<<<(NPAR + 255) / 256, 256>>>(h->p, h->wbf);
  if (cudaDeviceSynchronize() != cudaSuccess) { dd_mlp_destroy(h); return DD_ERR_CUDA; }
  *mlp = h;
  return DD_OK;
}

dd_status dd_mlp_set_data(void *mlp, const float *X, const float *y, int64_t n, void *stream) {
  MlpHandle *h = static_cast<MlpHandle *>(mlp);
  if (!h || !X || !y || n <= 0) return DD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MCK(cudaStreamSynchronize(s));
  cudaFree(h->X);
  cudaFree(h->y);
  h->X = nullptr;
  h->y = nullptr;
  h->n = 0;
  float *Xf = nullptr;
  MCK(cudaMalloc(&h->X, sizeof(__nv_bfloat16) * XPAD * (size_t)n));
  MCK(cudaMalloc(&h->y, sizeof(float) * (size_t)n));
  MCK(cudaMalloc(&Xf, sizeof(float) * NIN * (size_t)n));
  dd_status rc = cuda_ok(cudaMemcpyAsync(Xf, X, sizeof(float) * NIN * (size_t)n, cudaMemcpyHostToDevice, s));
  if (rc == DD_OK) rc = cuda_ok(cudaMemcpyAsync(h->y, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, s));
  if (rc == DD_OK) {
    mlp_pack_kernel<<<(unsigned)((n * XPAD + 255) / 256), 256, 0, s>>>(Xf, n, h->X);
    rc = cuda_ok(cudaGetLastError());
  }
  if (rc == DD_OK) rc = cuda_ok(cudaStreamSynchronize(s));
  cudaFree(Xf);
  if (rc == DD_OK) h->n = n;
  return rc;
}

dd_status dd_mlp_loss_grad(void *mlp, int64_t lo, int64_t hi, double *loss, float *grad, void *stream) {
  MlpHandle *h = static_cast<MlpHandle *>(mlp);
  if (!h || !loss) return DD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dd_status rc = grad_on(h, lo, hi, s);
  if (rc != DD_OK) return rc;
  MCK(cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (grad) MCK(cudaMemcpyAsync(grad, h->grad, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  return DD_OK;
}

dd_status dd_mlp_adam_step(void *mlp, int64_t lo, int64_t hi, float lr, float beta1, float beta2, float eps,
                           void *stream) {
  MlpHandle *h = static_cast<MlpHandle *>(mlp);
  if (!h || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return DD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dd_status rc = grad_on(h, lo, hi, s);
  if (rc != DD_OK) return rc;
  h->step += 1;
  const float c1 = 1.f - powf(beta1, (float)h->step), c2 = 1.f - powf(beta2, (float)h->step);
  mlp_adam_kernel<<<(NPAR + 255) / 256, 256, 0, s>>>(h->p, h->m, h->v, h->wbf, h->grad, lr, beta1, beta2, eps, c1,
                                                     c2);
  return cuda_ok(cudaGetLastError());
}

dd_status dd_mlp_predict(void *mlp, int64_t lo, int64_t hi, float *out, void *stream) {
  MlpHandle *h = static_cast<MlpHandle *>(mlp);
  if (!h || !out || lo < 0 || hi > h->n || hi <= lo) return DD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float *d = nullptr;
  MCK(cudaMalloc(&d, sizeof(float) * (size_t)(hi - lo)));
  mlp_predict_kernel<<<(unsigned)((hi - lo + 255) / 256), 256, 0, s>>>(h->X, lo, hi, h->wbf, d);
  dd_status rc = cuda_ok(cudaGetLastError());
  if (rc == DD_OK) rc = cuda_ok(cudaMemcpyAsync(out, d, sizeof(float) * (size_t)(hi - lo), cudaMemcpyDeviceToHost, s));
  if (rc == DD_OK) rc = cuda_ok(cudaStreamSynchronize(s));
  cudaFree(d);
  return rc;
}

dd_status dd_mlp_get(void *mlp, float *params, float *adam_m, float *adam_v, int64_t *step) {
  MlpHandle *h = static_cast<MlpHandle *>(mlp);
  if (!h) return DD_ERR_INVALID_ARG;
  MCK(cudaDeviceSynchronize());
  if (params) MCK(cudaMemcpy(params, h->p, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
  if (adam_m) MCK(cudaMemcpy(adam_m, h->m, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
  if (adam_v) MCK(cudaMemcpy(adam_v, h->v, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
  if (step) *step = h->step;
  return DD_OK;
}

dd_status dd_mlp_set_adam(void *mlp, const float *adam_m, const float *adam_v, int64_t step) {
  MlpHandle *h = static_cast<MlpHandle *>(mlp);
  if (!h || !adam_m || !adam_v || step < 0) return DD_ERR_INVALID_ARG;
  MCK(cudaDeviceSynchronize());
  MCK(cudaMemcpy(h->m, adam_m, sizeof(float) * NPAR, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(h->v, adam_v, sizeof(float) * NPAR, cudaMemcpyHostToDevice));
  h->step = step;
  return DD_OK;
}

dd_status dd_mlp_destroy(void *mlp) {
  MlpHandle *h = static_cast<MlpHandle *>(mlp);
  if (!h) return DD_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  void *bufs[] = {h->p, h->m, h->v, h->wbf, h->grad, h->partial, h->lossp, h->loss, h->X, h->y};
  for (void *b : bufs) cudaFree(b);
  delete h;
  return DD_OK;
}

}  // extern "C"
