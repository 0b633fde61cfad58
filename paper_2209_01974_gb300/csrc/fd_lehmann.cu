// Lehmann bounds of the eigenvalues nearest a shift (Lehmann 1963), the
// paper's source of the FD target and search intervals (Sec. 2: the extra
// SpMV after orthogonalisation provides the Ritz values and the Lehmann
// intervals).
//
// For a basis V of the search space and a shift rho, W = (A - rho) V gives the
// pencil  A1 x = mu A2 x  with  A1 = V^T W  and  A2 = W^T W  (the Rayleigh-Ritz
// matrices of (A - rho)^-1 on span(W)).  Its negative mu bound the eigenvalues
// below rho from below and its positive mu those above rho from above:
//   k-th eigenvalue below rho >= rho + 1 / mu_neg[k]  (mu_neg ascending),
//   k-th eigenvalue above rho <= rho + 1 / mu_pos[k]  (mu_pos descending).
// The pencil is solved on the device: symmetric diagonal scaling by
// 1/sqrt(A2_ii) (the entries of A2 span many orders of magnitude once pairs
// converge), Cholesky A2' = R^T R, C = R^-T A1' R^-1, Jacobi eigenvalues of C.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fd_internal.cuh"

namespace fdi {
namespace {

// W = AV - rho V (D x n, leading dimensions ldw, ldv)
__global__ void k_shift_cols(const double* AV, int64_t lda, const double* V, int64_t ldv, double rho,
                             int64_t D, int n, double* W, int64_t ldw) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * n) return;
  const int64_t i = t / n;
  const int j = (int)(t % n);
  W[i * ldw + j] = AV[i * lda + j] - rho * V[i * ldv + j];
}

// A1 = diag(theta - rho)
__global__ void k_diag_shift(const double* theta, double rho, int n, double* A1) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  A1[e] = i == j ? theta[i] - rho : 0.0;
}

// A1' = S A1 S, A2' = S A2 S with S = diag(1 / sqrt(A2_ii)) (1 where A2_ii <= 0,
// which the Cholesky then reports)
__global__ void k_scale_pencil(double* A1, double* A2, int n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const double di = A2[(int64_t)i * n + i], dj = A2[(int64_t)j * n + j];
  const double si = di > 0.0 ? rsqrt(di) : 1.0, sj = dj > 0.0 ? rsqrt(dj) : 1.0;
  A1[e] *= si * sj;
  // the diagonal of A2 is read by every thread: write it last, in a second kernel
  if (i != j) A2[e] *= si * sj;
}
__global__ void k_unit_diag(const double* A2, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = A2[(int64_t)i * n + i] > 0.0 ? 1.0 : A2[(int64_t)i * n + i];
}
__global__ void k_set_diag(double* A2, int n, const double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A2[(int64_t)i * n + i] = d[i];
}

// C = A^T B (n x n, row-major)
__global__ void k_atb(const double* A, const double* B, double* C, int n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  double s = 0.0;
  for (int k = 0; k < n; ++k) s = fma(A[(int64_t)k * n + i], B[(int64_t)k * n + j], s);
  C[e] = s;
}

// C <- (C + C^T) / 2
__global__ void k_symmetrize(double* C, int n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (i < j) {
    const double v = 0.5 * (C[e] + C[(int64_t)j * n + i]);
    C[e] = v;
    C[(int64_t)j * n + i] = v;
  }
}

}  // namespace

// Eigenvalues mu (device, ascending) of the n x n pencil A1 x = mu A2 x; A1
// and A2 (device, row-major, symmetric, A2 positive definite) are destroyed.
// *ok = false (no error) if A2 is not numerically positive definite.
fd_status lehmann_pencil(fd_ctx* ctx, double* A1, double* A2, int n, double* mu, bool* ok) {
  cudaStream_t st = ctx->stream;
  const size_t nn = (size_t)n * n;
  void* p;
  FD_TRY(workspace(ctx, "lehmann_small", sizeof(double) * (3 * nn + n) + 64, &p));
  double* R = (double*)p;
  double* Ri = R + nn;
  double* T = Ri + nn;
  double* dg = T + nn;
  int* okd = (int*)(dg + n);
  const unsigned g2 = (unsigned)cdiv((int64_t)nn, 256), g1 = (unsigned)cdiv(n, 256);
  k_unit_diag<<<g1, 256, 0, st>>>(A2, n, dg);
  FD_LAUNCHED(ctx);
  k_scale_pencil<<<g2, 256, 0, st>>>(A1, A2, n);
  FD_LAUNCHED(ctx);
  k_set_diag<<<g1, 256, 0, st>>>(A2, n, dg);
  FD_LAUNCHED(ctx);
  FD_CUDA(ctx, cudaMemsetAsync(okd, 0, sizeof(int), st));
  FD_TRY(cholesky(ctx, A2, n, 0.0, R, okd));
  int hok = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&hok, okd, sizeof(int), cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  *ok = hok != 0;
  if (!*ok) return FD_OK;
  FD_TRY(tri_inverse(ctx, R, n, Ri));
  FD_TRY(small_gemm_dev(ctx, A1, Ri, T, n));  // T = A1' R^-1
  k_atb<<<g2, 256, 0, st>>>(Ri, T, A1, n);    // C = R^-T A1' R^-1 (into A1)
  FD_LAUNCHED(ctx);
  k_symmetrize<<<g2, 256, 0, st>>>(A1, n);
  FD_LAUNCHED(ctx);
  FD_TRY(sym_eig(ctx, A1, n, mu, T, 40));
  return FD_OK;
}

// host: bounds from the pencil's eigenvalues (ascending): below (nearest
// first) from the negative ones, above (nearest first) from the positive ones
void lehmann_from_mu(const std::vector<double>& mu, double rho, std::vector<double>* below,
                     std::vector<double>* above) {
  below->clear();
  above->clear();
  for (double m : mu)
    if (m < 0.0) below->push_back(rho + 1.0 / m);  // ascending mu: most negative first
  for (auto it = mu.rbegin(); it != mu.rend(); ++it)
    if (*it > 0.0) above->push_back(rho + 1.0 / *it);  // largest first
}

// The FD loop's Lehmann bounds at shift rho from the Ritz basis: V holds the
// Ritz vectors (orthonormal), AV = A V and theta their Ritz values, so
// A1 = V^T (A - rho) V = diag(theta - rho); W = AV - rho V overwrites AV.
fd_status lehmann_ritz(fd_ctx* ctx, const double* V, double* AV, int64_t ld, int64_t D, int ns,
                       const double* theta_dev, double rho, std::vector<double>* below,
                       std::vector<double>* above, bool* ok) {
  cudaStream_t st = ctx->stream;
  const size_t nn = (size_t)ns * ns;
  void* p;
  FD_TRY(workspace(ctx, "lehmann_pencil", sizeof(double) * (2 * nn + ns), &p));
  double* A1 = (double*)p;
  double* A2 = A1 + nn;
  double* mu = A2 + nn;
  k_shift_cols<<<(unsigned)cdiv(D * ns, 256), 256, 0, st>>>(AV, ld, V, ld, rho, D, ns, AV, ld);
  FD_LAUNCHED(ctx);
  FD_TRY(gram(ctx, AV, ld, AV, ld, D, ns, ns, A2, ns, true));
  k_diag_shift<<<(unsigned)cdiv((int64_t)nn, 256), 256, 0, st>>>(theta_dev, rho, ns, A1);
  FD_LAUNCHED(ctx);
  FD_TRY(lehmann_pencil(ctx, A1, A2, ns, mu, ok));
  if (!*ok) return FD_OK;
  std::vector<double> h(ns);
  FD_CUDA(ctx, cudaMemcpyAsync(h.data(), mu, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  lehmann_from_mu(h, rho, below, above);
  return FD_OK;
}

}  // namespace fdi

using namespace fdi;

extern "C" fd_status fd_lehmann_bounds(fd_ctx* ctx, const fd_matrix* A, const double* V, int64_t D,
                                       int ns, int64_t ldv, double rho, double* below, int* n_below,
                                       double* above, int* n_above) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !V || !below || !above || !n_below || !n_above) return set_err(ctx, FD_ERR_ARG, "null argument");
  if (D != A->D || ns < 1 || ns > 1024 || ns > D || ldv < ns || !std::isfinite(rho))
    return set_err(ctx, FD_ERR_ARG, "need D = matrix dimension, 1 <= ns <= min(1024, D), ldv >= ns "
                                    "and a finite shift");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int w = ns % 2 ? ns + 1 : ns;  // SpMMV widths are even
  void* p;
  FD_TRY(workspace(ctx, "lehmann_W", sizeof(double) * D * w * 2, &p));
  double* Vp = (double*)p;      // V copied to an even width (aligned SpMMV rows)
  double* W = Vp + D * w;
  FD_CUDA(ctx, cudaMemsetAsync(Vp, 0, sizeof(double) * D * w, st));
  FD_CUDA(ctx, cudaMemcpy2DAsync(Vp, w * 8, V, ldv * 8, ns * 8, D, cudaMemcpyDeviceToDevice, st));
  for (int j = 0; j < w;) {
    const int b = w - j >= 128 ? 128 : w - j >= 64 ? 64 : w - j >= 32 ? 32 : w - j >= 16 ? 16
                : w - j >= 8 ? 8 : w - j >= 4 ? 4 : 2;
    FD_TRY(spmmv(ctx, A, FD_F64, Vp + j, w, W + j, w, b, true));
    j += b;
  }
  k_shift_cols<<<(unsigned)cdiv(D * w, 256), 256, 0, st>>>(W, w, Vp, w, rho, D, w, W, w);
  FD_LAUNCHED(ctx);
  const size_t nn = (size_t)ns * ns;
  FD_TRY(workspace(ctx, "lehmann_pencil", sizeof(double) * (2 * nn + ns), &p));
  double* A1 = (double*)p;
  double* A2 = A1 + nn;
  double* mu = A2 + nn;
  FD_TRY(gram(ctx, Vp, w, W, w, D, ns, ns, A1, ns, false));
  FD_TRY(gram(ctx, W, w, W, w, D, ns, ns, A2, ns, true));
  bool ok = false;
  FD_TRY(lehmann_pencil(ctx, A1, A2, ns, mu, &ok));
  if (!ok) return set_err(ctx, FD_ERR_BREAKDOWN, "(A - rho) V is numerically rank deficient");
  std::vector<double> h(ns), lo, hi;
  FD_CUDA(ctx, cudaMemcpyAsync(h.data(), mu, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  lehmann_from_mu(h, rho, &lo, &hi);
  std::copy(lo.begin(), lo.end(), below);
  std::copy(hi.begin(), hi.end(), above);
  *n_below = (int)lo.size();
  *n_above = (int)hi.size();
  return FD_OK;
}
