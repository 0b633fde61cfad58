// Filter-parameter predictor: a 64-128-128-3 perceptron (FP32, GELU) with its
// own forward, backward and Adam kernels, and the feature extraction that
// feeds it (kernel-polynomial density-of-states moments, Sec. 4.1, plus the
// scaled target window).  Its three outputs set the degree constant c_n and
// the window margins m_l, m_r of the interval heuristic that fd_solve uses in
// place of the paper's Lehmann intervals (Sec. 2); the plain heuristic is the
// fallback whenever an output is not finite.
//
// Parameter vector (FP32, 25219 numbers): W1 (64 x 128 row-major), b1, W2
// (128 x 128), b2, W3 (128 x 3), b3.  GELU is the erf form
// x/2 (1 + erf(x / sqrt 2)), evaluated with CUDA's erff and expf.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fd_internal.cuh"

namespace fdi {
namespace {

constexpr int NI = 64, NH = 128, NO = 3;
constexpr int FD_FEATURE_MOMENTS = 48;
constexpr int OFF_W1 = 0, OFF_B1 = NI * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NO, N_PARAMS = OFF_B3 + NO;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// one CTA (128 threads) per sample: z1, z2 stored for the backward pass
__global__ void __launch_bounds__(NH) k_mlp_forward(const float* __restrict__ P,
                                                    const float* __restrict__ X, int B, float* Y,
                                                    float* Z1, float* Z2) {
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= B) return;
  __shared__ float x[NI], h1[NH], h2[NH];
  if (j < NI) x[j] = X[(int64_t)b * NI + j];
  __syncthreads();
  float z = P[OFF_B1 + j];
  for (int i = 0; i < NI; ++i) z = fmaf(x[i], P[OFF_W1 + i * NH + j], z);
  if (Z1) Z1[(int64_t)b * NH + j] = z;
  h1[j] = gelu(z);
  __syncthreads();
  z = P[OFF_B2 + j];
  for (int i = 0; i < NH; ++i) z = fmaf(h1[i], P[OFF_W2 + i * NH + j], z);
  if (Z2) Z2[(int64_t)b * NH + j] = z;
  h2[j] = gelu(z);
  __syncthreads();
  if (j < NO) {
    float y = P[OFF_B3 + j];
    for (int i = 0; i < NH; ++i) y = fmaf(h2[i], P[OFF_W3 + i * NO + j], y);
    Y[(int64_t)b * NO + j] = y;
  }
}

// per sample: dy = 2 (y - t) / (3 B), dz2, dz1, and the squared error
__global__ void __launch_bounds__(NH) k_mlp_backward_sample(const float* __restrict__ P,
                                                            const float* Y, const float* T, int B,
                                                            const float* Z1, const float* Z2,
                                                            float* DY, float* DZ1, float* DZ2,
                                                            float* sq) {
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= B) return;
  __shared__ float dy[NO], dz2[NH];
  if (j < NO) {
    const float r = Y[(int64_t)b * NO + j] - T[(int64_t)b * NO + j];
    dy[j] = 2.0f * r / (3.0f * B);
    DY[(int64_t)b * NO + j] = dy[j];
    sq[(int64_t)b * NO + j] = r * r;
  }
  __syncthreads();
  float d = 0.0f;
  for (int o = 0; o < NO; ++o) d = fmaf(dy[o], P[OFF_W3 + j * NO + o], d);
  d *= gelu_d(Z2[(int64_t)b * NH + j]);
  dz2[j] = d;
  DZ2[(int64_t)b * NH + j] = d;
  __syncthreads();
  float e = 0.0f;
  for (int o = 0; o < NH; ++o) e = fmaf(dz2[o], P[OFF_W2 + j * NH + o], e);
  DZ1[(int64_t)b * NH + j] = e * gelu_d(Z1[(int64_t)b * NH + j]);
}

// weight gradients: each thread owns one parameter and sums over the batch in order
__global__ void k_mlp_weight_grad(const float* __restrict__ X, const float* Z1, const float* Z2,
                                  const float* DY, const float* DZ1, const float* DZ2, int B,
                                  float* G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N_PARAMS) return;
  float s = 0.0f;
  if (p < OFF_B1) {
    const int i = p / NH, j = p % NH;
    for (int b = 0; b < B; ++b) s = fmaf(X[(int64_t)b * NI + i], DZ1[(int64_t)b * NH + j], s);
  } else if (p < OFF_W2) {
    const int j = p - OFF_B1;
    for (int b = 0; b < B; ++b) s += DZ1[(int64_t)b * NH + j];
  } else if (p < OFF_B2) {
    const int i = (p - OFF_W2) / NH, j = (p - OFF_W2) % NH;
    for (int b = 0; b < B; ++b) s = fmaf(gelu(Z1[(int64_t)b * NH + i]), DZ2[(int64_t)b * NH + j], s);
  } else if (p < OFF_W3) {
    const int j = p - OFF_B2;
    for (int b = 0; b < B; ++b) s += DZ2[(int64_t)b * NH + j];
  } else if (p < OFF_B3) {
    const int i = (p - OFF_W3) / NO, o = (p - OFF_W3) % NO;
    for (int b = 0; b < B; ++b) s = fmaf(gelu(Z2[(int64_t)b * NH + i]), DY[(int64_t)b * NO + o], s);
  } else {
    const int o = p - OFF_B3;
    for (int b = 0; b < B; ++b) s += DY[(int64_t)b * NO + o];
  }
  G[p] = s;
}

__global__ void k_sum(const float* a, int n, float* out) {
  __shared__ float sh[256];
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] / n;
}

__global__ void k_adam(float* P, const float* G, float* M, float* V, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float g = G[p];
  const float m = b1 * M[p] + (1.0f - b1) * g;
  const float v = b2 * V[p] + (1.0f - b2) * g * g;
  M[p] = m;
  V[p] = v;
  P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

struct MlpWork {
  float *Y, *Z1, *Z2, *DY, *DZ1, *DZ2, *sq, *G, *loss;
};

fd_status mlp_work(fd_ctx* ctx, int B, MlpWork* w) {
  void* p;
  const size_t n = (size_t)B * (2 * NO + 4 * NH + NO) + N_PARAMS + 8;
  FD_TRY(workspace(ctx, "mlp", sizeof(float) * n, &p));
  float* f = (float*)p;
  w->Y = f; f += (size_t)B * NO;
  w->DY = f; f += (size_t)B * NO;
  w->sq = f; f += (size_t)B * NO;
  w->Z1 = f; f += (size_t)B * NH;
  w->Z2 = f; f += (size_t)B * NH;
  w->DZ1 = f; f += (size_t)B * NH;
  w->DZ2 = f; f += (size_t)B * NH;
  w->G = f; f += N_PARAMS;
  w->loss = f;
  return FD_OK;
}

fd_status mlp_grad(fd_ctx* ctx, const float* P, const float* X, const float* T, int B, MlpWork& w) {
  cudaStream_t st = ctx->stream;
  k_mlp_forward<<<B, NH, 0, st>>>(P, X, B, w.Y, w.Z1, w.Z2);
  FD_LAUNCHED(ctx);
  k_mlp_backward_sample<<<B, NH, 0, st>>>(P, w.Y, T, B, w.Z1, w.Z2, w.DY, w.DZ1, w.DZ2, w.sq);
  FD_LAUNCHED(ctx);
  k_mlp_weight_grad<<<(unsigned)cdiv(N_PARAMS, 256), 256, 0, st>>>(X, w.Z1, w.Z2, w.DY, w.DZ1, w.DZ2, B, w.G);
  FD_LAUNCHED(ctx);
  k_sum<<<1, 256, 0, st>>>(w.sq, B * NO, w.loss);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

}  // namespace
}  // namespace fdi

using namespace fdi;

extern "C" {

int fd_mlp_num_params(void) { return N_PARAMS; }

fd_status fd_mlp_forward(fd_ctx* ctx, const float* params, const float* X, int B, float* Y) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!params || !X || !Y || B < 1 || B > 1 << 20) return set_err(ctx, FD_ERR_ARG, "need params, X, Y and 1 <= B <= 2^20");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  k_mlp_forward<<<B, NH, 0, ctx->stream>>>(params, X, B, Y, nullptr, nullptr);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status fd_mlp_gradient(fd_ctx* ctx, const float* params, const float* X, const float* T, int B,
                          float* grad, float* loss) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!params || !X || !T || !grad || !loss || B < 1 || B > 1 << 20)
    return set_err(ctx, FD_ERR_ARG, "need params, X, T, grad, loss and 1 <= B <= 2^20");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  MlpWork w;
  FD_TRY(mlp_work(ctx, B, &w));
  FD_TRY(mlp_grad(ctx, params, X, T, B, w));
  FD_CUDA(ctx, cudaMemcpyAsync(grad, w.G, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToDevice, ctx->stream));
  FD_CUDA(ctx, cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return FD_OK;
}

fd_status fd_mlp_train_step(fd_ctx* ctx, float* params, float* m, float* v, const float* X,
                            const float* T, int B, int step, float lr, float* loss) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!params || !m || !v || !X || !T || B < 1 || B > 1 << 20 || step < 1 || !(lr > 0))
    return set_err(ctx, FD_ERR_ARG, "need buffers, 1 <= B <= 2^20, step >= 1, lr > 0");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  MlpWork w;
  FD_TRY(mlp_work(ctx, B, &w));
  FD_TRY(mlp_grad(ctx, params, X, T, B, w));
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<(unsigned)cdiv(N_PARAMS, 256), 256, 0, ctx->stream>>>(params, w.G, m, v, N_PARAMS, lr, b1,
                                                                b2, 1e-8f, c1, c2);
  FD_LAUNCHED(ctx);
  if (loss) {
    FD_CUDA(ctx, cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return FD_OK;
}

fd_status fd_filter_features(fd_ctx* ctx, const fd_matrix* A, double a, double b, int n_target,
                             int nb, int ns, uint64_t seed, float* feat) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !feat || !(a <= b) || n_target < 1 || nb < 1 || ns < 1)
    return set_err(ctx, FD_ERR_ARG, "need a matrix, a <= b, n_target, nb, ns >= 1 and an output");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  double lo, hi;
  FD_TRY(spectral_bounds(ctx, A, 20, seed, &lo, &hi));
  const double alpha = 2.0 / (hi - lo), beta = -(hi + lo) / (hi - lo);
  const int M = FD_FEATURE_MOMENTS;
  std::vector<double> mu(M);
  FD_TRY(kpm(ctx, A, M, 16, seed, alpha, beta, mu.data()));
  const double xa = std::max(-1.0, std::min(1.0, alpha * a + beta));
  const double xb = std::max(-1.0, std::min(1.0, alpha * b + beta));
  // eigenvalue count in [a, b] from the Jackson-damped DOS (Sec. 4.1): D sum g_m mu_m c_m
  const int n = M - 1;
  const int N = n + 1;
  const double ang = M_PI / (N + 1);
  const double ta = std::acos(xa), tb = std::acos(xb);
  double cnt = 0.0;
  for (int k = 0; k <= n; ++k) {
    const double g = ((N - k + 1) * std::cos(ang * k) + std::sin(ang * k) / std::tan(ang)) / (N + 1);
    const double c = k == 0 ? (ta - tb) / M_PI : 2.0 * (std::sin(k * ta) - std::sin(k * tb)) / (k * M_PI);
    cnt += g * mu[k] * c;
  }
  cnt = std::max(0.0, cnt * (double)A->D);
  const double sc = std::max(std::fabs(lo), std::fabs(hi));
  std::fill(feat, feat + 64, 0.0f);
  for (int k = 0; k < M; ++k) feat[k] = (float)mu[k];
  float* f = feat + M;
  f[0] = (float)xa;
  f[1] = (float)xb;
  f[2] = (float)(xb - xa);
  f[3] = (float)(n_target / 100.0);
  f[4] = (float)(std::log10((double)A->D) / 8.0);
  f[5] = (float)((double)A->nnz / (double)A->D / 32.0);
  f[6] = (float)(lo / sc);
  f[7] = (float)(hi / sc);
  f[8] = (float)(std::log10(1.0 + cnt) / 6.0);
  f[9] = (float)std::min(4.0, cnt / ns);
  f[10] = (float)(nb / 128.0);
  f[11] = (float)(ns / 1024.0);
  return FD_OK;
}

fd_status fd_predict_filter_params(fd_ctx* ctx, const float* params, const float* feat, double* c_n,
                                   double* m_l, double* m_r, int* fallback) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!params || !feat || !c_n || !m_l || !m_r) return set_err(ctx, FD_ERR_ARG, "null argument");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  void* p;
  FD_TRY(workspace(ctx, "mlp_predict", sizeof(float) * 68, &p));
  float* x = (float*)p;
  float* y = x + 64;
  FD_CUDA(ctx, cudaMemcpyAsync(x, feat, sizeof(float) * 64, cudaMemcpyHostToDevice, ctx->stream));
  k_mlp_forward<<<1, NH, 0, ctx->stream>>>(params, x, 1, y, nullptr, nullptr);
  FD_LAUNCHED(ctx);
  float h[3];
  FD_CUDA(ctx, cudaMemcpyAsync(h, y, sizeof(float) * 3, cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const bool ok = std::isfinite(h[0]) && std::isfinite(h[1]) && std::isfinite(h[2]);
  if (!ok) {  // the plain heuristic is the fallback
    *c_n = 4.0; *m_l = 0.5; *m_r = 0.5;
  } else {
    *c_n = std::exp(std::max(0.0, std::min(std::log(16.0), (double)h[0])));
    *m_l = std::max(0.05, std::min(0.95, (double)h[1]));
    *m_r = std::max(0.05, std::min(0.95, (double)h[2]));
  }
  if (fallback) *fallback = ok ? 0 : 1;
  return FD_OK;
}

}  // extern "C"
