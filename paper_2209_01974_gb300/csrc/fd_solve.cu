// The FD outer loop (Sec. 2, Alg. 1) and its spectral-interval preparation.
//
// Alg. 1 is printed as an image; its steps are taken from the prose of Sec. 2:
// an inclusion interval [lam_l, lam_r] from a few Lanczos steps, N_s random
// search vectors, then repeat { orthonormalise; one SpMMV + Rayleigh-Ritz
// giving Ritz values and residuals; stop when the N_t Ritz pairs nearest the
// target have rho <= tol; choose target/search intervals and the degree;
// apply the Chebyshev filter }.  The paper chooses the intervals from Lehmann
// intervals; this driver offers those (fd_lehmann.cu) and a Ritz-value
// heuristic (documented on fd_options).  All vector work runs in the library's kernels; the host keeps
// only the scalar control logic (intervals, degree, the O(n) coefficients).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <vector>

#include "fd_internal.cuh"

namespace fdi {
namespace {

// dot products out[j] = sum_i Q[j * D + i] * w[i], j < k (partials + fixed-order reduce)
__global__ void k_dots_partial(const double* Q, int k, const double* w, int64_t D, double* P) {
  __shared__ double sh[256];
  for (int j = 0; j < k; ++j) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D;
         i += (int64_t)gridDim.x * blockDim.x)
      s = fma(Q[(int64_t)j * D + i], w[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) P[(int64_t)j * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}
__global__ void k_dots_reduce(const double* P, int k, int nb, double* out) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += P[(int64_t)j * nb + b];
    out[j] = s;
  }
}
// w -= sum_j Q_j c_j
__global__ void k_sub_proj(const double* Q, int k, const double* c, int64_t D, double* w) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D) return;
  double s = w[i];
  for (int j = 0; j < k; ++j) s -= Q[(int64_t)j * D + i] * c[j];
  w[i] = s;
}
__global__ void k_scale_copy(const double* w, double f, int64_t D, double* q) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < D) q[i] = w[i] * f;
}
__global__ void k_lanczos_start(const int64_t* perm, int64_t D, uint64_t key, double* r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < D) r[i] = fdrng::irwin_hall(key, (uint64_t)perm[i]);
}
__global__ void k_tridiag(const double* a, const double* b, int k, double* T) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  int i = e / k, j = e % k;
  T[e] = i == j ? a[i] : (j == i + 1 ? b[i] : (i == j + 1 ? b[j] : 0.0));
}
// start block, original row order: V[i][j] = g(seed, stream 2, i * ns + j)
__global__ void k_start_block(double* V, int64_t ld, int64_t D, int ns, uint64_t key) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * ns) return;
  int64_t i = t / ns;
  int j = (int)(t % ns);
  V[i * ld + j] = fdrng::irwin_hall(key, (uint64_t)t);
}
// X[:, c] = sign * V[:, sel[c]], sign making the largest-magnitude entry (first on ties) positive
__global__ void k_extract(const double* V, int64_t ldv, int64_t D, const int* sel, double* X,
                          int64_t ldx) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  const int c = blockIdx.x;
  const int col = sel[c];
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < D; i += blockDim.x) {
    double a = fabs(V[i * ldv + col]);
    if (a > best) { best = a; bi = i; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double a = sv[threadIdx.x + o];
      int64_t ai = si[threadIdx.x + o];
      if (a > sv[threadIdx.x] || (a == sv[threadIdx.x] && ai < si[threadIdx.x])) {
        sv[threadIdx.x] = a;
        si[threadIdx.x] = ai;
      }
    }
    __syncthreads();
  }
  const double sgn = V[si[0] * ldv + col] < 0.0 ? -1.0 : 1.0;
  for (int64_t i = threadIdx.x; i < D; i += blockDim.x) X[i * ldx + c] = sgn * V[i * ldv + col];
}

// ---- host-side filter coefficients (Sec. 2: Chebyshev expansion of a window,
// Jackson-damped as in the kernel polynomial method the paper cites) --------
double cheb_eval(const std::vector<double>& mu, double x) {
  x = std::min(1.0, std::max(-1.0, x));
  const double th = std::acos(x);
  double s = 0.0;
  for (size_t k = 0; k < mu.size(); ++k) s += mu[k] * std::cos((double)k * th);
  return s;
}

}  // namespace

std::vector<double> filter_coeffs(double x_l, double x_r, int n) {
  x_l = std::max(-1.0, x_l);
  x_r = std::min(1.0, x_r);
  const double th_l = std::acos(x_l), th_r = std::acos(x_r);
  const int N = n + 1;
  const double a = M_PI / (N + 1);
  std::vector<double> mu(n + 1);
  for (int k = 0; k <= n; ++k) {
    const double g = ((N - k + 1) * std::cos(a * k) + std::sin(a * k) / std::tan(a)) / (N + 1);
    const double c = k == 0 ? (th_l - th_r) / M_PI
                            : 2.0 * (std::sin(k * th_l) - std::sin(k * th_r)) / (k * M_PI);
    mu[k] = g * c;
  }
  const double p = cheb_eval(mu, 0.5 * (x_l + x_r));
  for (auto& m : mu) m /= p;
  return mu;
}

namespace {

struct Timer {
  cudaEvent_t e0, e1;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) { cudaEventCreate(&e0); cudaEventCreate(&e1); }
  ~Timer() { cudaEventDestroy(e0); cudaEventDestroy(e1); }
  void start() { cudaEventRecord(e0, st); }
  double stop_s() {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms * 1e-3;
  }
};

}  // namespace

fd_status spectral_bounds(fd_ctx* ctx, const fd_matrix* A, int steps, uint64_t seed,
                          double* lam_l, double* lam_r) {
  cudaStream_t st = ctx->stream;
  const int64_t D = A->D;
  const int m = (int)std::min<int64_t>(steps, D);
  const int T = 256;
  const int nbk = (int)std::min<int64_t>(ctx->num_sms * 2, cdiv(D, T));
  void* p;
  FD_TRY(workspace(ctx, "lanczos", sizeof(double) * ((size_t)(m + 2) * D + (size_t)m * nbk + 4 * m + 64 + 4 * (size_t)m * m), &p));
  double* Q = (double*)p;              // m x D, Lanczos vectors
  double* w = Q + (size_t)m * D;       // D
  double* r = w + D;                   // D
  double* P = r + D;                   // m x nbk partials
  double* dots = P + (size_t)m * nbk;  // m
  double* ab = dots + m;               // alpha, beta (2m)
  double* T2 = ab + 2 * m + 64;        // m x m
  double* wk = T2 + (size_t)m * m;     // eigenvalues
  double* Qk = wk + m;                 // m x m eigenvectors
  k_lanczos_start<<<(unsigned)cdiv(D, T), T, 0, st>>>(A->perm, D, fdrng::key(seed, fdrng::STREAM_LANCZOS), r);
  FD_LAUNCHED(ctx);
  auto dot_into = [&](const double* Qm, int k, const double* v) -> fd_status {
    k_dots_partial<<<nbk, T, 0, st>>>(Qm, k, v, D, P);
    FD_LAUNCHED(ctx);
    k_dots_reduce<<<1, 64, 0, st>>>(P, k, nbk, dots);
    FD_LAUNCHED(ctx);
    return FD_OK;
  };
  FD_TRY(dot_into(r, 1, r));
  double nrm2 = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&nrm2, dots, sizeof(double), cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  k_scale_copy<<<(unsigned)cdiv(D, T), T, 0, st>>>(r, 1.0 / std::sqrt(nrm2), D, Q);
  FD_LAUNCHED(ctx);
  std::vector<double> alpha, beta;
  double beta_last = 0.0;
  for (int j = 0; j < m; ++j) {
    FD_TRY(spmv1(ctx, A, Q + (size_t)j * D, w));
    FD_TRY(dot_into(Q + (size_t)j * D, 1, w));
    double a = 0;
    FD_CUDA(ctx, cudaMemcpyAsync(&a, dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    for (int pass = 0; pass < 2; ++pass) {  // full reorthogonalisation, twice
      FD_TRY(dot_into(Q, j + 1, w));
      k_sub_proj<<<(unsigned)cdiv(D, T), T, 0, st>>>(Q, j + 1, dots, D, w);
      FD_LAUNCHED(ctx);
    }
    FD_TRY(dot_into(w, 1, w));
    double b2 = 0;
    FD_CUDA(ctx, cudaMemcpyAsync(&b2, dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaStreamSynchronize(st));
    alpha.push_back(a);
    beta_last = std::sqrt(b2);
    if (j == m - 1 || beta_last <= 1e-14 * std::max(1.0, std::fabs(a))) break;
    beta.push_back(beta_last);
    k_scale_copy<<<(unsigned)cdiv(D, T), T, 0, st>>>(w, 1.0 / beta_last, D, Q + (size_t)(j + 1) * D);
    FD_LAUNCHED(ctx);
  }
  const int k = (int)alpha.size();
  std::vector<double> hab(2 * k, 0.0);
  std::copy(alpha.begin(), alpha.end(), hab.begin());
  std::copy(beta.begin(), beta.end(), hab.begin() + k);
  FD_CUDA(ctx, cudaMemcpyAsync(ab, hab.data(), sizeof(double) * 2 * k, cudaMemcpyHostToDevice, st));
  k_tridiag<<<(unsigned)cdiv(k * k, T), T, 0, st>>>(ab, ab + k, k, T2);
  FD_LAUNCHED(ctx);
  double tmin, tmax, smin, smax;
  if (k == 1) {
    tmin = tmax = alpha[0];
    smin = smax = 1.0;
  } else {
    FD_TRY(sym_eig(ctx, T2, k, wk, Qk, 40));
    std::vector<double> hw(k), hq((size_t)k * k);
    FD_CUDA(ctx, cudaMemcpyAsync(hw.data(), wk, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaMemcpyAsync(hq.data(), Qk, sizeof(double) * k * k, cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaStreamSynchronize(st));
    tmin = hw[0];
    tmax = hw[k - 1];
    smin = hq[(size_t)(k - 1) * k + 0];
    smax = hq[(size_t)(k - 1) * k + (k - 1)];
  }
  const double wdt = std::max(tmax - tmin, 1e-10 * std::max({1.0, std::fabs(tmin), std::fabs(tmax)}));
  double lo = tmin - std::fabs(beta_last * smin) - 0.01 * wdt;
  double hi = tmax + std::fabs(beta_last * smax) + 0.01 * wdt;
  *lam_l = std::max(A->gersh_lo, lo);
  *lam_r = std::min(A->gersh_hi, hi);
  return FD_OK;
}

}  // namespace fdi

using namespace fdi;

namespace {

std::vector<int> nearest_order(const std::vector<double>& th, double tau) {
  std::vector<int> o(th.size());
  std::iota(o.begin(), o.end(), 0);
  std::stable_sort(o.begin(), o.end(), [&](int a, int b) {
    double da = std::fabs(th[a] - tau), db = std::fabs(th[b] - tau);
    if (da != db) return da < db;
    return th[a] < th[b];
  });
  return o;
}

}  // namespace

extern "C" {

fd_status fd_filter_coeffs(double x_l, double x_r, int n, double* mu) {
  if (!mu || n < 2 || !(x_l < x_r) || !std::isfinite(x_l) || !std::isfinite(x_r)) return FD_ERR_ARG;
  std::vector<double> m = filter_coeffs(x_l, x_r, n);
  std::copy(m.begin(), m.end(), mu);
  return FD_OK;
}

fd_status fd_spectral_bounds(fd_ctx* ctx, const fd_matrix* A, int steps, uint64_t seed,
                             double* lam_l, double* lam_r) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !lam_l || !lam_r || steps < 0 || steps > 1000)
    return set_err(ctx, FD_ERR_ARG, "need a matrix, outputs and 0 <= steps <= 1000");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  return spectral_bounds(ctx, A, steps ? steps : 20, seed, lam_l, lam_r);
}

}  // extern "C"

namespace fdi {

// The FD loop.  ck == nullptr: a plain solve.  Otherwise the solve starts
// from the checkpoint (ck->iteration > 0: the filtered block in Vck and the
// loop's scalars), runs at most `max_iter` outer iterations and, if it has not
// converged by then, stops right after a filter application and writes the
// filtered block back to Vck and the scalars to ck.
static fd_status solve_impl(fd_ctx* ctx, const fd_matrix* A, double a, double b, int n_target, int nb,
                            int degree, double tol, const fd_options* opt_in, fd_result* res,
                            double* theta_out, double* resid_out, double* X, int64_t ldx,
                            fd_checkpoint* ck, double* Vck, int max_iter) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  fd_options opt{};
  if (opt_in) opt = *opt_in;
  if (!A || !res || !theta_out || !resid_out) return set_err(ctx, FD_ERR_ARG, "null argument");
  if (!(a <= b) || !std::isfinite(a) || !std::isfinite(b) || !(tol > 0))
    return set_err(ctx, FD_ERR_ARG, "need finite a <= b and tol > 0");
  if (nb != 2 && nb != 4 && nb != 8 && nb != 16 && nb != 32 && nb != 64 && nb != 128)
    return set_err(ctx, FD_ERR_ARG, "nb must be 2, 4, ..., 128");
  if (opt.precision != FD_F64 && opt.precision != FD_F32 && opt.precision != FD_FF)
    return set_err(ctx, FD_ERR_ARG, "bad precision");
  if (opt.finish != FD_FINISH_F64 && opt.finish != FD_FINISH_FF)
    return set_err(ctx, FD_ERR_ARG, "finish must be FD_FINISH_F64 or FD_FINISH_FF");
  if (opt.precision == FD_F32 && nb < 4) return set_err(ctx, FD_ERR_ARG, "FP32 sweeps need nb >= 4");
  // float-float sweeps: the FD_FF form, or the FD_F32 form's finish
  const bool ff_sweeps = opt.precision == FD_FF || (opt.precision == FD_F32 && opt.finish == FD_FINISH_FF);
  if (degree < 2) return set_err(ctx, FD_ERR_ARG, "degree must be >= 2 (Alg. 2)");
  if (opt.intervals != FD_INTERVALS_RITZ && opt.intervals != FD_INTERVALS_LEHMANN)
    return set_err(ctx, FD_ERR_ARG, "intervals must be FD_INTERVALS_RITZ or FD_INTERVALS_LEHMANN");
  const int64_t D = A->D;
  int ns = opt.ns > 0 ? opt.ns : nb * (int)cdiv(4LL * n_target, nb);
  if (n_target < 1 || ns % nb || ns < n_target || ns > D || ns > 1024)
    return set_err(ctx, FD_ERR_ARG, "need 1 <= n_target <= ns <= min(D, 1024), ns a multiple of nb");
  if (X && ldx < n_target) return set_err(ctx, FD_ERR_ARG, "ldx < n_target");
  const int max_outer = opt.max_outer > 0 ? opt.max_outer : 60;
  const int n_max = opt.n_max > 0 ? opt.n_max : 100000;
  const int lsteps = opt.lanczos_steps > 0 ? opt.lanczos_steps : 20;
  const double c_n = opt.c_n > 0 ? opt.c_n : 4.0;
  const double m_l = opt.m_l > 0 ? opt.m_l : 0.5, m_r = opt.m_r > 0 ? opt.m_r : 0.5;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_TRY(debug_check_matrix(ctx, A));
  cudaStream_t st = ctx->stream;
  *res = fd_result{};
  res->ns = ns;
  Timer tm(st), ttot(st);
  ttot.start();

  // workspaces: V, AV (D x ns FP64), W1, W2 (D x nb FP64); FP32 bundle buffers
  void* p;
  FD_TRY(workspace(ctx, "solve_V", sizeof(double) * D * ns, &p)); double* V = (double*)p;
  FD_TRY(workspace(ctx, "solve_AV", sizeof(double) * D * ns, &p)); double* AV = (double*)p;
  FD_TRY(workspace(ctx, "solve_W", sizeof(double) * 2 * D * nb, &p));
  double* W1 = (double*)p;
  double* W2 = W1 + D * nb;
  float *V32 = nullptr, *W132 = nullptr, *W232 = nullptr;
  if (opt.precision == FD_F32) {
    FD_TRY(workspace(ctx, "solve_W32", sizeof(float) * 3 * D * nb, &p));
    V32 = (float*)p; W132 = V32 + D * nb; W232 = W132 + D * nb;
  }
  // float-float bundle (2 floats per element); its recurrence vectors reuse W1, W2
  float* Vff = nullptr;
  if (ff_sweeps) {
    FD_TRY(workspace(ctx, "solve_Wff", sizeof(float) * 2 * D * nb, &p));
    Vff = (float*)p;
  }
  FD_TRY(workspace(ctx, "solve_small", sizeof(double) * 2 * ns + sizeof(int) * ns + 64, &p));
  double* th_dev = (double*)p;
  double* rho_dev = th_dev + ns;
  int* sel_dev = (int*)(rho_dev + ns);

  const bool resume = ck && ck->iteration > 0;
  if (ck && (ck->iteration < 0 || (resume && (ck->D != D || ck->ns != ns || ck->seed != opt.seed))))
    return set_err(ctx, FD_ERR_ARG, "checkpoint of another problem (D, ns or seed differ)");
  double lam_l, lam_r, widen, normH;
  double wl = a, wr = b;
  int n = degree;
  bool use_f32 = opt.precision == FD_F32;
  double prev_max = INFINITY;
  int stall = 0;
  int it = 0;
  if ((opt.lam_l != 0.0 || opt.lam_r != 0.0) &&
      !(std::isfinite(opt.lam_l) && std::isfinite(opt.lam_r) && opt.lam_l < opt.lam_r))
    return set_err(ctx, FD_ERR_ARG, "inclusion interval override needs finite lam_l < lam_r");
  if (!resume) {
    // steps 1-2: inclusion interval (or the caller's)
    tm.start();
    if (opt.lam_l != 0.0 || opt.lam_r != 0.0) {
      lam_l = opt.lam_l;
      lam_r = opt.lam_r;
    } else {
      FD_TRY(spectral_bounds(ctx, A, lsteps, opt.seed, &lam_l, &lam_r));
    }
    res->t_bounds = tm.stop_s();
    widen = 0.01 * (lam_r - lam_l);
    normH = std::max(std::fabs(lam_l), std::fabs(lam_r));
    k_start_block<<<(unsigned)cdiv(D * ns, 256), 256, 0, st>>>(V, ns, D, ns, fdrng::key(opt.seed, fdrng::STREAM_START));
    FD_LAUNCHED(ctx);
  } else {
    lam_l = ck->lam_l; lam_r = ck->lam_r; widen = ck->widen; normH = ck->norm_h;
    wl = ck->window_l; wr = ck->window_r; n = ck->degree;
    use_f32 = ck->use_f32 != 0; prev_max = ck->prev_max; stall = ck->stall; it = ck->iteration;
    res->n_spmmv = ck->n_spmmv; res->n_spmmv_f32 = ck->n_spmmv_f32; res->filter_bytes = ck->filter_bytes;
    res->n_spmmv_ff = ck->n_spmmv_ff;
    FD_CUDA(ctx, cudaMemcpyAsync(V, Vck, sizeof(double) * D * ns, cudaMemcpyDeviceToDevice, st));
  }
  const double tau = 0.5 * (a + b);
  const int it_stop = ck ? std::min(max_outer, it + max_iter) : max_outer;

  std::vector<double> th(ns), rho(ns);
  bool done = false, paused = false;
  for (; it < max_outer; ++it) {
    tm.start();
    FD_TRY(orthonormalize(ctx, V, D, ns, ns, nullptr, nullptr));
    res->t_ortho += tm.stop_s();
    tm.start();
    FD_TRY(rayleigh_ritz_dev(ctx, A, V, AV, D, ns, ns, th_dev, rho_dev));
    FD_CUDA(ctx, cudaMemcpyAsync(th.data(), th_dev, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaMemcpyAsync(rho.data(), rho_dev, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    res->t_rr += tm.stop_s();
    res->n_spmmv += 1;
    std::vector<int> order = nearest_order(th, tau);
    double maxr = 0;
    int nconv = 0;
    for (int i = 0; i < n_target; ++i) {
      maxr = std::max(maxr, rho[order[i]]);
      nconv += rho[order[i]] <= tol;
    }
    if (opt.verbose)
      fprintf(stderr, "fd it %d degree %d window [%.6g, %.6g] conv %d/%d max_resid %.3e %s\n", it, n,
              wl, wr, nconv, n_target, maxr, use_f32 ? "f32" : ff_sweeps ? "ff" : "f64");
    if (nconv == n_target) { done = true; ++it; break; }
    if (it == max_outer - 1) { ++it; break; }  // keep V = Ritz vectors of the last step
    // precision switch: FP32 sweeps until their floor or a stall (two
    // iterations in a row without halving the largest wanted residual)
    stall = maxr > 0.5 * prev_max ? stall + 1 : 0;
    if (use_f32 && (maxr <= 100.0 * 0x1.0p-24 * normH || stall >= 2)) use_f32 = false;
    prev_max = maxr;
    // a Ritz value outside the inclusion interval moves that side out beyond
    // it (outside [-1, 1] the filter grows like cosh(n acosh|x|))
    if (th[0] < lam_l) lam_l = std::min(lam_l - 2 * widen, th[0] - widen);
    if (th[ns - 1] > lam_r) lam_r = std::max(lam_r + 2 * widen, th[ns - 1] + widen);
    const double alpha = 2.0 / (lam_r - lam_l), beta = -(lam_r + lam_l) / (lam_r - lam_l);
    if (it > 0) {
      double t_l = INFINITY, t_r = -INFINITY, s_l = INFINITY, s_r = -INFINITY;
      const int nsrch = (int)std::ceil(0.75 * ns);
      for (int i = 0; i < n_target; ++i) { t_l = std::min(t_l, th[order[i]]); t_r = std::max(t_r, th[order[i]]); }
      for (int i = 0; i < nsrch; ++i) { s_l = std::min(s_l, th[order[i]]); s_r = std::max(s_r, th[order[i]]); }
      s_l = std::min(s_l, t_l);
      s_r = std::max(s_r, t_r);
      if (opt.intervals == FD_INTERVALS_LEHMANN) {
        // each target edge moves out to the Lehmann bound at tau for the count
        // of wanted Ritz values on its side, when that bound lies inside the
        // search interval (while the subspace is poor it lies far outside)
        tm.start();
        std::vector<double> below, above;
        bool ok = false;
        FD_TRY(lehmann_ritz(ctx, V, AV, ns, D, ns, th_dev, tau, &below, &above, &ok));
        res->t_rr += tm.stop_s();
        if (ok) {
          int kb = 0, ka = 0;
          for (int i = 0; i < n_target; ++i) { kb += th[order[i]] < tau; ka += th[order[i]] > tau; }
          if (kb > 0 && kb <= (int)below.size() && s_l < below[kb - 1] && below[kb - 1] <= t_l) t_l = below[kb - 1];
          if (ka > 0 && ka <= (int)above.size() && t_r <= above[ka - 1] && above[ka - 1] < s_r) t_r = above[ka - 1];
        }
      }
      auto ang = [&](double lam) { return std::acos(std::min(1.0, std::max(-1.0, alpha * lam + beta))); };
      const double dth = std::min(ang(s_l) - ang(t_l), ang(t_r) - ang(s_r));
      long long nn = dth <= 0.0 ? n_max : (long long)std::ceil(c_n * M_PI / dth);
      n = (int)std::max<long long>(degree, std::min<long long>(n_max, nn));
      wl = t_l - m_l * (t_l - s_l);
      wr = t_r + m_r * (s_r - t_r);
    }
    std::vector<double> mu = filter_coeffs(alpha * wl + beta, alpha * wr + beta, n);
    tm.start();
    double bytes = 0;
    for (int j = 0; j < ns; j += nb) {
      if (use_f32) {
        FD_TRY(copy_cols_f64_to_f32(ctx, V + j, ns, V32, nb, D, nb));
        FD_TRY(filter(ctx, A, FD_F32, V32, nb, nb, n, mu.data(), alpha, beta, W132, W232, nb, &bytes));
        FD_TRY(copy_cols_f32_to_f64(ctx, V32, nb, V + j, ns, D, nb));
      } else if (ff_sweeps) {
        FD_TRY(copy_cols_f64_to_ff(ctx, V + j, ns, Vff, nb, D, nb));
        FD_TRY(filter(ctx, A, FD_FF, Vff, nb, nb, n, mu.data(), alpha, beta, W1, W2, nb, &bytes));
        FD_TRY(copy_cols_ff_to_f64(ctx, Vff, nb, V + j, ns, D, nb));
      } else {
        FD_TRY(filter(ctx, A, FD_F64, V + j, ns, nb, n, mu.data(), alpha, beta, W1, W2, nb, &bytes));
      }
    }
    res->t_filter += tm.stop_s();
    res->filter_bytes += bytes;
    res->n_spmmv += n;
    if (use_f32) res->n_spmmv_f32 += n;
    else if (ff_sweeps) res->n_spmmv_ff += n;
    if (ck && it + 1 == it_stop && it + 1 < max_outer) {  // pause after this filter application
      ++it;
      paused = true;
      break;
    }
  }
  if (paused) {
    FD_CUDA(ctx, cudaMemcpyAsync(Vck, V, sizeof(double) * D * ns, cudaMemcpyDeviceToDevice, st));
    FD_CUDA(ctx, cudaStreamSynchronize(st));
    ck->iteration = it; ck->degree = n; ck->use_f32 = use_f32 ? 1 : 0; ck->stall = stall;
    ck->lam_l = lam_l; ck->lam_r = lam_r; ck->widen = widen; ck->norm_h = normH;
    ck->window_l = wl; ck->window_r = wr; ck->prev_max = prev_max;
    ck->n_spmmv = res->n_spmmv; ck->n_spmmv_f32 = res->n_spmmv_f32; ck->filter_bytes = res->filter_bytes;
    ck->n_spmmv_ff = res->n_spmmv_ff;
    ck->D = D; ck->ns = ns; ck->seed = opt.seed; ck->converged = 0;
  }
  // outputs: the N_t pairs nearest tau, ascending
  std::vector<int> order = nearest_order(th, tau);
  std::vector<int> sel(order.begin(), order.begin() + n_target);
  std::sort(sel.begin(), sel.end(), [&](int x, int y) { return th[x] < th[y] || (th[x] == th[y] && x < y); });
  for (int i = 0; i < n_target; ++i) {
    theta_out[i] = th[sel[i]];
    resid_out[i] = rho[sel[i]];
  }
  if (X) {
    FD_CUDA(ctx, cudaMemcpyAsync(sel_dev, sel.data(), sizeof(int) * n_target, cudaMemcpyHostToDevice, st));
    k_extract<<<n_target, 256, 0, st>>>(V, ns, D, sel_dev, X, ldx);
    FD_LAUNCHED(ctx);
  }
  res->t_total = ttot.stop_s();
  res->converged = done ? 1 : 0;
  res->iterations = it;
  res->final_degree = n;
  res->lam_l = lam_l;
  res->lam_r = lam_r;
  res->window_l = wl;
  res->window_r = wr;
  if (ck && !paused) {
    ck->iteration = it; ck->converged = done ? 1 : 0;
    ck->D = D; ck->ns = ns; ck->seed = opt.seed;
  }
  if (paused) return set_err(ctx, FD_ERR_NOCONV, "paused after %d outer iterations (checkpoint written)", it);
  if (!done) return set_err(ctx, FD_ERR_NOCONV, "no convergence after %d outer iterations", max_outer);
  return FD_OK;
}

}  // namespace fdi

extern "C" {

fd_status fd_solve(fd_ctx* ctx, const fd_matrix* A, double a, double b, int n_target, int nb,
                   int degree, double tol, const fd_options* opt, fd_result* res,
                   double* theta, double* resid, double* X, int64_t ldx) {
  return solve_impl(ctx, A, a, b, n_target, nb, degree, tol, opt, res, theta, resid, X, ldx, nullptr,
                    nullptr, 0);
}

fd_status fd_solve_checkpointed(fd_ctx* ctx, const fd_matrix* A, double a, double b, int n_target,
                                int nb, int degree, double tol, const fd_options* opt, int max_iter,
                                fd_checkpoint* ck, double* Vck, fd_result* res, double* theta,
                                double* resid, double* X, int64_t ldx) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!ck || !Vck || max_iter < 1 || ((uintptr_t)Vck & 15))
    return set_err(ctx, FD_ERR_ARG, "need a checkpoint, an aligned device block and max_iter >= 1");
  return solve_impl(ctx, A, a, b, n_target, nb, degree, tol, opt, res, theta, resid, X, ldx, ck, Vck,
                    max_iter);
}

}  // extern "C"
