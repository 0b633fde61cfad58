// Batched filter diagonalization: many independent, unevenly sized problems
// solved together.  Every outer iteration (Sec. 2, Alg. 1) of all unconverged
// instances is one CUDA graph: the Chebyshev filters of every search-vector
// bundle of every instance run in ONE persistent cooperative kernel (all
// degree steps, a grid-wide barrier between steps), followed by batched
// Cholesky-QR and Rayleigh-Ritz kernels that each cover all instances in one
// launch, and one copy of all Ritz values and residuals to the host.  The host
// then applies the same interval/degree heuristic as fd_solve per instance.
//
// An autotuner (fd_tune_batched) times the persistent filter over candidate
// block widths nb, SELL chunk heights C and CTA shapes on the actual
// instances and returns the fastest.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fd_internal.cuh"
#include "fd_step.cuh"
#include "fd_ff.cuh"

namespace cg = cooperative_groups;

namespace fdi {
namespace {

using namespace step;
using ffa::ff;

constexpr int BMAX_NS = 96;  // single-CTA shared-memory Jacobi / Cholesky limit

struct BInst {
  SellArgs<double> A;
  SellArgs<float> A32;  // the same SELL arrays with the FP32 values
  SellArgs<ff> Aff;     // ... and with the float-float values
  double* V;      // D x ns, ld = ns
  float* V32;     // FP32 copy of V for FP32 sweeps (nullptr unless the FP32 form is on)
  float* W32;     // (ns / nb) bundles x 2 x D x nb
  double* AV;     // D x ns
  double* W;      // (ns / nb) bundles x 2 x D x nb
  double* G;      // ns x ns (Gram / Rayleigh quotient)
  double* R;      // ns x ns (Cholesky factor)
  double* Ri;     // ns x ns (inverse / eigenvectors)
  double* P;      // gram partials: slices x ns x ns
  double* theta;  // ns
  double* resid;  // ns
  double* rpart;  // residual partials: RBLK x ns
  int ns;
  int pad;
};

struct BParams {  // rewritten by the host before every outer iteration
  int active;     // 0: converged (skipped)
  int degree;     // 0: no filter this iteration
  int mu_off;     // offset of mu_0 in the coefficient table
  int flags;      // device-written: 1 = a Cholesky pass was shifted, 2 = breakdown
  double alpha, beta;
  int f32;        // 1: this iteration's filter runs in FP32 (V32, W32, FP32 values)
  int ff;         // 1: it runs in float-float (V and W hold (hi, lo) pairs in place)
};

struct BTask {
  int inst, bundle;
};

// The tasks (bundles) of the instances still active, rewritten by the host
// before every outer iteration: ordered by their instance's filter degree,
// largest first, so that the tasks still filtering at degree step k are a
// prefix of the list and a step touches only their rows.
struct BatchArgs {
  const BInst* inst;
  BParams* par;
  const BTask* task;
  const int64_t* task_off;  // n_tasks + 1 row offsets (each task padded to RPW rows)
  const int* task_deg;      // n_tasks filter degrees, non-increasing
  const int* n_tasks;       // tasks in the list this iteration
  const double* mu;
  const int* kmax;          // largest degree this iteration
  int nb;
  int spmmv_only;           // 1: AV = A V for all listed bundles, one pass, no barrier
};

constexpr int GSLICES = 8;   // Gram row slices per instance
constexpr int RBLK = 16;     // residual partial blocks per instance

// ---------------------------------------------------------------------------
// persistent batched filter
// ---------------------------------------------------------------------------
template <int NB>
__device__ __forceinline__ void batched_row_group(const BatchArgs& b, int t, int64_t lrow0, int k) {
  const BTask tk = b.task[t];
  const BInst& I = b.inst[tk.inst];
  const BParams& P = b.par[tk.inst];
  const int64_t D = I.A.D;
  double* V = I.V + (int64_t)tk.bundle * NB;
  double* W1 = I.W + (int64_t)tk.bundle * 2 * D * NB;
  double* W2 = W1 + D * NB;
  StepArgs<double> s{};
  if (b.spmmv_only) {
    s.X = V; s.ldx = I.ns; s.Y = I.AV + (int64_t)tk.bundle * NB; s.ldy = I.ns;
    s.c_ax = 1.0; s.c_x = 0.0;
    cheb_rows<double, NB, MODE_SPMMV>(I.A, s, lrow0);
    return;
  }
  const int n = P.degree;
  if (!P.active || k > n) return;
  const double* mu = b.mu + P.mu_off;
  if (k == 1) {
    s.X = V; s.ldx = I.ns; s.Y = W1; s.ldy = NB;
    s.c_ax = P.alpha; s.c_x = P.beta;
    cheb_rows<double, NB, MODE_SPMMV>(I.A, s, lrow0);
  } else if (k == 2) {
    s.X = W1; s.ldx = NB; s.Z = V; s.ldz = I.ns;
    s.Y = n > 2 ? W2 : nullptr; s.ldy = NB;
    s.Vout = V; s.ldvo = I.ns;
    s.c_ax = 2 * P.alpha; s.c_x = 2 * P.beta;
    s.mu0 = mu[0]; s.mu1 = mu[1]; s.mu2 = mu[2];
    cheb_rows<double, NB, MODE_SECOND>(I.A, s, lrow0);
  } else {
    double* X = (k & 1) ? W2 : W1;
    double* Z = (k & 1) ? W1 : W2;
    s.X = X; s.ldx = NB; s.Z = Z; s.ldz = NB;
    s.Y = k < n ? Z : nullptr; s.ldy = NB;
    s.Vin = V; s.ldvi = I.ns; s.Vout = V; s.ldvo = I.ns;
    s.c_ax = 2 * P.alpha; s.c_x = 2 * P.beta; s.mu2 = mu[k];
    cheb_rows<double, NB, MODE_GENERIC>(I.A, s, lrow0);
  }
}

// FP32 sweeps of an instance in the FP32 form: the same steps on V32, W32 and
// the FP32 matrix values (FP32 accumulation), as fd_solve's FP32 sweeps
template <int NB>
__device__ __forceinline__ void batched_row_group_f32(const BatchArgs& b, int t, int64_t lrow0, int k) {
  const BTask tk = b.task[t];
  const BInst& I = b.inst[tk.inst];
  const BParams& P = b.par[tk.inst];
  const int64_t D = I.A.D;
  const int n = P.degree;
  if (!P.active || k > n) return;
  float* V = I.V32 + (int64_t)tk.bundle * NB;
  float* W1 = I.W32 + (int64_t)tk.bundle * 2 * D * NB;
  float* W2 = W1 + D * NB;
  const double* mu = b.mu + P.mu_off;
  StepArgs<float> s{};
  if (k == 1) {
    s.X = V; s.ldx = I.ns; s.Y = W1; s.ldy = NB;
    s.c_ax = (float)P.alpha; s.c_x = (float)P.beta;
    cheb_rows<float, NB, MODE_SPMMV>(I.A32, s, lrow0);
  } else if (k == 2) {
    s.X = W1; s.ldx = NB; s.Z = V; s.ldz = I.ns;
    s.Y = n > 2 ? W2 : nullptr; s.ldy = NB;
    s.Vout = V; s.ldvo = I.ns;
    s.c_ax = (float)(2 * P.alpha); s.c_x = (float)(2 * P.beta);
    s.mu0 = (float)mu[0]; s.mu1 = (float)mu[1]; s.mu2 = (float)mu[2];
    cheb_rows<float, NB, MODE_SECOND>(I.A32, s, lrow0);
  } else {
    float* X = (k & 1) ? W2 : W1;
    float* Z = (k & 1) ? W1 : W2;
    s.X = X; s.ldx = NB; s.Z = Z; s.ldz = NB;
    s.Y = k < n ? Z : nullptr; s.ldy = NB;
    s.Vin = V; s.ldvi = I.ns; s.Vout = V; s.ldvo = I.ns;
    s.c_ax = (float)(2 * P.alpha); s.c_x = (float)(2 * P.beta); s.mu2 = (float)mu[k];
    cheb_rows<float, NB, MODE_GENERIC>(I.A32, s, lrow0);
  }
}

// float-float sweeps of an instance (its FP32 form's finish, or the FF form):
// the same steps on V and W reinterpreted as (hi, lo) pairs, which k_bconvert
// writes in place of the doubles before the filter and turns back after it
template <int NB>
__device__ __forceinline__ void batched_row_group_ff(const BatchArgs& b, int t, int64_t lrow0, int k) {
  const BTask tk = b.task[t];
  const BInst& I = b.inst[tk.inst];
  const BParams& P = b.par[tk.inst];
  const int64_t D = I.A.D;
  const int n = P.degree;
  if (!P.active || k > n) return;
  ff* V = reinterpret_cast<ff*>(I.V + (int64_t)tk.bundle * NB);
  ff* W1 = reinterpret_cast<ff*>(I.W + (int64_t)tk.bundle * 2 * D * NB);
  ff* W2 = W1 + D * NB;
  const double* mu = b.mu + P.mu_off;
  StepArgs<ff> s{};
  if (k == 1) {
    s.X = V; s.ldx = I.ns; s.Y = W1; s.ldy = NB;
    s.c_ax = ff(P.alpha); s.c_x = ff(P.beta);
    cheb_rows<ff, NB, MODE_SPMMV>(I.Aff, s, lrow0);
  } else if (k == 2) {
    s.X = W1; s.ldx = NB; s.Z = V; s.ldz = I.ns;
    s.Y = n > 2 ? W2 : nullptr; s.ldy = NB;
    s.Vout = V; s.ldvo = I.ns;
    s.c_ax = ff(2 * P.alpha); s.c_x = ff(2 * P.beta);
    s.mu0 = ff(mu[0]); s.mu1 = ff(mu[1]); s.mu2 = ff(mu[2]);
    cheb_rows<ff, NB, MODE_SECOND>(I.Aff, s, lrow0);
  } else {
    ff* X = (k & 1) ? W2 : W1;
    ff* Z = (k & 1) ? W1 : W2;
    s.X = X; s.ldx = NB; s.Z = Z; s.ldz = NB;
    s.Y = k < n ? Z : nullptr; s.ldy = NB;
    s.Vin = V; s.ldvi = I.ns; s.Vout = V; s.ldvo = I.ns;
    s.c_ax = ff(2 * P.alpha); s.c_x = ff(2 * P.beta); s.mu2 = ff(mu[k]);
    cheb_rows<ff, NB, MODE_GENERIC>(I.Aff, s, lrow0);
  }
}

// FF: the instantiation with FP32 and float-float rows only, the filter of
// solves that use float-float sweeps.  It runs the shape of the
// single-problem FP32 and float-float steps, 4-warp CTAs and 12 per SM
// (48 warps, <= 40 registers): both are bound by memory latency.
constexpr int BF_FF_WARPS = 4, BF_FF_BLOCKS = 12;
template <int NB, bool FF>
__global__ void __launch_bounds__(FF ? BF_FF_WARPS * 32 : WARPS * 32, FF ? BF_FF_BLOCKS : 3)
    k_batched_filter(BatchArgs b) {
  using L = Layout<double, NB>;
  extern __shared__ int64_t s_off[];  // n_tasks + 1 offsets, then n_tasks degrees
  const int nt = *b.n_tasks;
  int* s_deg = reinterpret_cast<int*>(s_off + nt + 1);
  for (int i = threadIdx.x; i <= nt; i += blockDim.x) s_off[i] = b.task_off[i];
  for (int i = threadIdx.x; i < nt; i += blockDim.x) s_deg[i] = b.task_deg[i];
  __syncthreads();
  const int warps = blockDim.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * warps;
  const int kmax = b.spmmv_only ? 1 : *b.kmax;
  cg::grid_group grid = cg::this_grid();
  int cut = nt;  // tasks still filtering: the prefix with degree >= k
  for (int k = 1; k <= kmax; ++k) {
    if (!b.spmmv_only)
      while (cut > 0 && s_deg[cut - 1] < k) --cut;
    const int64_t ngroups = s_off[cut] / L::RPW;
    for (int64_t g = gw; g < ngroups; g += nw) {
      const int64_t r0 = g * L::RPW;
      int lo = 0, hi = cut - 1;  // last task with s_off[t] <= r0
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= r0) lo = mid; else hi = mid - 1;
      }
      const int64_t lrow0 = r0 - s_off[lo];
      const int inst = b.task[lo].inst;
      if (lrow0 >= b.inst[inst].A.D) continue;
      if constexpr (NB >= 4) {
        // an FP32 warp covers twice the rows of an FP64 one (16-byte vectors hold
        // four floats): FP32 tasks take the even FP64 row groups (task rows are
        // padded to the FP32 granule when the FP32 form is on)
        if (!b.spmmv_only && b.par[inst].f32) {
          if (((lrow0 / L::RPW) & 1) == 0) batched_row_group_f32<NB>(b, lo, lrow0, k);
          continue;
        }
      }
      if constexpr (FF) {
        // a solve with float-float rows has no FP64 rows in its filter (every
        // instance is FP32 or float-float; its Rayleigh-Ritz SpMMV runs in the
        // other instantiation), so this one carries no FP64 path
        batched_row_group_ff<NB>(b, lo, lrow0, k);
      } else {
        batched_row_group<NB>(b, lo, lrow0, k);
      }
    }
    if (!b.spmmv_only) grid.sync();
  }
}

// V32 <- (float) V before an FP32 filter, V <- (double) V32 after it, for the
// instances whose filter runs in FP32 this iteration (blockIdx.y = instance)
// For float-float filters the same kernel splits each double of V in place
// into its (hi, lo) pair and adds the pair back afterwards.
__global__ void k_bconvert(const BInst* insts, const BParams* par, int to32) {
  const BInst& I = insts[blockIdx.y];
  const BParams& P = par[blockIdx.y];
  if (!P.active || P.degree == 0) return;
  const int64_t n = I.A.D * I.ns;
  const int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, de = (int64_t)gridDim.x * blockDim.x;
  if (P.ff) {
    float2* F = reinterpret_cast<float2*>(I.V);
    for (int64_t e = e0; e < n; e += de) {
      if (to32) {
        const double v = I.V[e];
        const float hi = __double2float_rn(v);
        F[e] = make_float2(hi, __double2float_rn(v - (double)hi));
      } else {
        const float2 f = F[e];
        I.V[e] = (double)f.x + (double)f.y;
      }
    }
    return;
  }
  if (!P.f32 || !I.V32) return;
  for (int64_t e = e0; e < n; e += de) {
    if (to32) I.V32[e] = (float)I.V[e];
    else I.V[e] = (double)I.V32[e];
  }
}

// ---------------------------------------------------------------------------
// batched dense kernels (one instance per blockIdx.z or blockIdx.x)
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

// P[slice] = X^T Y over the slice's rows (sym: upper tiles), X = V, Y = V or AV
__global__ void __launch_bounds__(256) k_bgram_partial(const BInst* insts, const BParams* par,
                                                       int use_av, int only_shifted) {
  const BInst& I = insts[blockIdx.z];
  const BParams& Pm = par[blockIdx.z];
  if (!Pm.active || (only_shifted && !(Pm.flags & 1))) return;
  const int ns = I.ns;
  const int nt = (ns + GT - 1) / GT;
  int t = blockIdx.x, ti = 0, rowlen = nt;
  if (t >= nt * (nt + 1) / 2) return;
  while (t >= rowlen) { t -= rowlen; ++ti; --rowlen; }
  const int tj = ti + t;
  const double* X = I.V;
  const double* Y = use_av ? I.AV : I.V;
  const int64_t D = I.A.D;
  const int64_t rps = ((D + GSLICES - 1) / GSLICES + GK - 1) / GK * GK;
  const int64_t k0 = (int64_t)blockIdx.y * rps, k1 = min(D, k0 + rps);
  __shared__ double Xs[GK][GT], Ys[GK][GT];
  const int i0 = ti * GT, j0 = tj * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int64_t kb = k0; kb < k1; kb += GK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = threadIdx.x + q * 256;
      int kk = e / GT, c = e % GT;
      int64_t k = kb + kk;
      Xs[kk][c] = (k < k1 && i0 + c < ns) ? X[k * ns + i0 + c] : 0.0;
      Ys[kk][c] = (k < k1 && j0 + c < ns) ? Y[k * ns + j0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = Xs[kk][ty + 16 * u]; bb[u] = Ys[kk][tx + 16 * u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bb[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* Ps = I.P + (int64_t)blockIdx.y * ns * ns;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < ns && j < ns) Ps[(int64_t)i * ns + j] = acc[u][v];
    }
}

__global__ void k_bgram_reduce(const BInst* insts, const BParams* par, int only_shifted) {
  const BInst& I = insts[blockIdx.y];
  const BParams& Pm = par[blockIdx.y];
  if (!Pm.active || (only_shifted && !(Pm.flags & 1))) return;
  const int ns = I.ns;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ns * ns) return;
  const int i = e / ns, j = e % ns;
  if (i / GT > j / GT) return;
  double s = 0.0;
  for (int q = 0; q < GSLICES; ++q) s += I.P[(int64_t)q * ns * ns + e];
  I.G[e] = s;
  if (i / GT < j / GT) I.G[(int64_t)j * ns + i] = s;
}

// Cholesky of G (shared memory), shifted retry on breakdown, then R^-1 into Ri
__global__ void __launch_bounds__(256) k_bchol_inv(const BInst* insts, BParams* par,
                                                   int only_shifted) {
  const BInst& I = insts[blockIdx.x];
  BParams& Pm = par[blockIdx.x];
  if (!Pm.active || (only_shifted && !(Pm.flags & 1))) return;
  const int n = I.ns;
  extern __shared__ double sm[];
  double* R = sm;            // n x n
  double* x = sm + n * n;    // 8 warps x n
  __shared__ int fail;
  __shared__ double rinv, tr;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += I.G[i * n + i];
    tr = s;
  }
  __syncthreads();
  const double coeff = 11.0 * ((double)I.A.D * n + (double)n * (n + 1)) * 0x1.0p-53;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double shift = attempt ? coeff * tr : 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e / n, j = e % n;
      R[e] = j >= i ? I.G[e] + (i == j ? shift : 0.0) : 0.0;
    }
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      if (threadIdx.x == 0) {
        double d = R[k * n + k];
        if (!(d > 0.0) || !isfinite(d)) fail = 1;
        else { double r = sqrt(d); R[k * n + k] = r; rinv = 1.0 / r; }
      }
      __syncthreads();
      if (fail) break;
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) R[k * n + j] *= rinv;
      __syncthreads();
      const int m = n - k - 1;
      for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = k + 1 + e / m, j = k + 1 + e % m;
        if (j >= i) R[i * n + j] -= R[k * n + i] * R[k * n + j];
      }
      __syncthreads();
    }
    if (!fail) {
      if (attempt && threadIdx.x == 0) Pm.flags |= 1;
      break;
    }
    if (attempt) {
      if (threadIdx.x == 0) Pm.flags |= 2;
      return;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) I.R[e] = R[e];
  // inverse, one warp per column
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* xw = x + w * n;
  for (int j = w; j < n; j += 8) {
    for (int i = j; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1 + lane; k <= j; k += 32) s = fma(R[i * n + k], xw[k], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) xw[i] = ((i == j ? 1.0 : 0.0) - s) / R[i * n + i];
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) I.Ri[i * n + j] = i <= j ? xw[i] : 0.0;
    __syncwarp();
  }
}

// V (or AV) <- V * M, 16 rows per CTA, M = Ri (upper) or the eigenvectors
__global__ void __launch_bounds__(256) k_brotate(const BInst* insts, const BParams* par,
                                                 int which, int upper, int only_shifted) {
  const BInst& I = insts[blockIdx.y];
  const BParams& Pm = par[blockIdx.y];
  if (!Pm.active || (only_shifted && !(Pm.flags & 1)) || (Pm.flags & 2)) return;
  const int n = I.ns;
  const int64_t D = I.A.D;
  const int64_t r0 = (int64_t)blockIdx.x * 16;
  if (r0 >= D) return;
  double* V = which ? I.AV : I.V;
  const double* M = I.Ri;
  extern __shared__ double Vt[];
  const int nr = D - r0 < 16 ? (int)(D - r0) : 16;
  for (int e = threadIdx.x; e < 16 * n; e += 256) {
    int r = e / n, c = e % n;
    Vt[e] = r < nr ? V[(r0 + r) * n + c] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x >> 4, c0 = threadIdx.x & 15;
  for (int cb = 0; cb < n; cb += 64) {
    double acc[4] = {0, 0, 0, 0};
    const int kend = upper ? min(n, cb + 64) : n;
    for (int k = 0; k < kend; ++k) {
      const double a = Vt[r * n + k];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (cb + c0 + 16 * v < n) acc[v] = fma(a, M[k * n + cb + c0 + 16 * v], acc[v]);
    }
    if (r < nr)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int c = cb + c0 + 16 * v;
        if (c < n) V[(r0 + r) * n + c] = acc[v];
      }
  }
}

// cyclic Jacobi on G (n x n, n <= BMAX_NS) in shared memory; eigenvalues
// ascending into theta, eigenvectors (columns) into Ri
__global__ void __launch_bounds__(256) k_bjacobi(const BInst* insts, const BParams* par) {
  const BInst& I = insts[blockIdx.x];
  const BParams& Pm = par[blockIdx.x];
  if (!Pm.active || (Pm.flags & 2)) return;
  const int n = I.ns, np = n + (n & 1), half = np / 2;
  extern __shared__ double sm[];
  double* A = sm;              // np x np
  double* Q = A + np * np;     // np x np
  double* cs = Q + np * np;    // 2 * half
  __shared__ double red[256];
  for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
    int i = e / np, j = e % np;
    A[e] = (i < n && j < n) ? I.G[i * n + j] : 0.0;
    Q[e] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  double fro = 0.0;
  for (int e = threadIdx.x; e < np * np; e += blockDim.x) fro += A[e] * A[e];
  red[threadIdx.x] = fro;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double fro2 = red[0];
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0;
    for (int e = threadIdx.x; e < np * np; e += blockDim.x)
      if (e / np != e % np) off += A[e] * A[e];
    red[threadIdx.x] = off;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    const bool done = red[0] <= 1e-28 * fro2;
    __syncthreads();
    if (done) break;
    for (int round = 0; round < np - 1; ++round) {
      const int m = np - 1;
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int a = k == 0 ? round % m : (round + k) % m;
        int b = k == 0 ? m : (round - k + m) % m;
        int p = min(a, b), q = max(a, b);
        double apq = A[p * np + q], c = 1.0, s = 0.0;
        if (apq != 0.0) {
          double tau = (A[q * np + q] - A[p * np + p]) / (2.0 * apq);
          double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = threadIdx.x; e < half * np; e += blockDim.x) {
        int k = e / np, j = e % np;
        int a = k == 0 ? round % m : (round + k) % m;
        int b = k == 0 ? m : (round - k + m) % m;
        int p = min(a, b), q = max(a, b);
        double c = cs[2 * k], s = cs[2 * k + 1];
        double ap = A[p * np + j], aq = A[q * np + j];
        A[p * np + j] = c * ap - s * aq;
        A[q * np + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, Q <- Q J
      for (int e = threadIdx.x; e < half * np; e += blockDim.x) {
        int k = e / np, i = e % np;
        int a = k == 0 ? round % m : (round + k) % m;
        int b = k == 0 ? m : (round - k + m) % m;
        int p = min(a, b), q = max(a, b);
        double c = cs[2 * k], s = cs[2 * k + 1];
        double ap = A[i * np + p], aq = A[i * np + q];
        A[i * np + p] = c * ap - s * aq;
        A[i * np + q] = s * ap + c * aq;
        double qp = Q[i * np + p], qq = Q[i * np + q];
        Q[i * np + p] = c * qp - s * qq;
        Q[i * np + q] = s * qp + c * qq;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int a = k == 0 ? round % m : (round + k) % m;
        int b = k == 0 ? m : (round - k + m) % m;
        A[a * np + b] = 0.0;
        A[b * np + a] = 0.0;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ai = A[i * np + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double aj = A[j * np + j];
      rank += (aj < ai) || (aj == ai && j < i);
    }
    I.theta[rank] = ai;
    for (int r = 0; r < n; ++r) I.Ri[r * n + rank] = Q[r * np + i];
  }
}

__global__ void k_bresid(const BInst* insts, const BParams* par) {
  const BInst& I = insts[blockIdx.y];
  const BParams& Pm = par[blockIdx.y];
  if (!Pm.active || (Pm.flags & 2)) return;
  const int n = I.ns;
  const int64_t D = I.A.D;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double th = I.theta[c];
    double s = 0.0;
    for (int64_t r = blockIdx.x; r < D; r += gridDim.x) {
      const double d = I.AV[r * n + c] - th * I.V[r * n + c];
      s = fma(d, d, s);
    }
    I.rpart[blockIdx.x * n + c] = s;
  }
}

__global__ void k_bresid_reduce(const BInst* insts, const BParams* par) {
  const BInst& I = insts[blockIdx.x];
  const BParams& Pm = par[blockIdx.x];
  if (!Pm.active || (Pm.flags & 2)) return;
  for (int c = threadIdx.x; c < I.ns; c += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < RBLK; ++b) s += I.rpart[b * I.ns + c];
    I.resid[c] = sqrt(s);
  }
}

__global__ void k_bstart(double* V, int64_t n, uint64_t key) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) V[t] = fdrng::irwin_hall(key, (uint64_t)t);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Batch {
  int n = 0, nb = 0, warps = WARPS, ns_max = 0;
  bool f32 = false;  // FP32 sweeps available (the FP32 form)
  bool ff = false;   // float-float sweeps possible (FF form or float-float finish)
  int rpw = 1;       // row granule of a task
  size_t n_tasks_all = 0;
  int* d_tdeg = nullptr;
  int* d_ntask = nullptr;
  BTask* h_task_p = nullptr;   // pinned mirrors of the per-iteration task list
  int64_t* h_off_p = nullptr;
  int* h_tdeg_p = nullptr;
  std::vector<BInst> h_inst;
  std::vector<BTask> h_task;
  std::vector<int64_t> h_off;
  BInst* d_inst = nullptr;
  BParams* d_par = nullptr;
  BTask* d_task = nullptr;
  int64_t* d_off = nullptr;
  double* d_mu = nullptr;
  int* d_kmax = nullptr;
  size_t mu_cap = 0;
  void* arena = nullptr;
  // pinned host mirrors
  BParams* h_par = nullptr;
  double* h_mu = nullptr;
  int* h_kmax = nullptr;
  double* h_out = nullptr;  // theta and resid of all instances
  int grid = 0;
  int grid_rr = 0, warps_rr = WARPS;  // the Rayleigh-Ritz SpMMV launch (FP64 rows)
  size_t smem_filter = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t max_D = 0;

  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(arena);
    cudaFreeHost(h_par);
    cudaFreeHost(h_mu);
    cudaFreeHost(h_kmax);
    cudaFreeHost(h_out);
    cudaFreeHost(h_task_p);
    cudaFreeHost(h_off_p);
    cudaFreeHost(h_tdeg_p);
    cudaFreeHost(h_ntask);
  }
  // the tasks of the active instances, largest degree first (h_par's degrees)
  void list_tasks() {
    std::vector<int> order;
    for (int i = 0; i < n; ++i)
      if (h_par[i].active) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return h_par[x].degree > h_par[y].degree; });
    size_t t = 0;
    h_off_p[0] = 0;
    for (int i : order)
      for (int bnd = 0; bnd < h_inst[i].ns / nb; ++bnd, ++t) {
        h_task_p[t] = BTask{i, bnd};
        h_tdeg_p[t] = h_par[i].degree;
        h_off_p[t + 1] = h_off_p[t] + cdiv(h_inst[i].A.D, rpw) * rpw;
      }
    *h_ntask = (int)t;
  }
  int* h_ntask = nullptr;
};

template <int NB>
const void* filter_kernel(bool with_ff) {
  return with_ff ? (const void*)k_batched_filter<NB, true> : (const void*)k_batched_filter<NB, false>;
}

const void* filter_kernel_for(int nb, bool with_ff) {
  switch (nb) {
    case 2: return filter_kernel<2>(with_ff);
    case 4: return filter_kernel<4>(with_ff);
    case 8: return filter_kernel<8>(with_ff);
    case 16: return filter_kernel<16>(with_ff);
    case 32: return filter_kernel<32>(with_ff);
    case 64: return filter_kernel<64>(with_ff);
    default: return nullptr;
  }
}

fd_status batch_setup(fd_ctx* ctx, Batch& B, int n, const fd_matrix* const* A, const int* ns,
                      int nb, int warps, size_t mu_cap, bool f32 = false, bool with_ff = false) {
  B.n = n;
  B.nb = nb;
  B.warps = with_ff ? BF_FF_WARPS : warps;  // the float-float instantiation's fixed shape
  B.f32 = f32;
  B.ff = with_ff;
  // rows per warp of the FP64 step; the FP32 step covers twice as many
  const int rpw = (32 / std::min(32, nb * 8 / 16)) * (f32 ? 2 : 1);
  // arena layout per instance
  size_t bytes = 0;
  std::vector<size_t> off(n);
  for (int i = 0; i < n; ++i) {
    const int64_t D = A[i]->D;
    const size_t nn = (size_t)ns[i] * ns[i];
    off[i] = bytes;
    bytes += sizeof(double) * (2 * D * ns[i] + 2 * D * ns[i] + 3 * nn + GSLICES * nn + 2 * ns[i] +
                               RBLK * ns[i]);
    bytes = (bytes + 255) & ~(size_t)255;
    if (f32) bytes += sizeof(float) * 3 * D * ns[i] + 256;  // V32 and the bundles' W32
    bytes = (bytes + 255) & ~(size_t)255;
    B.ns_max = std::max(B.ns_max, ns[i]);
    B.max_D = std::max<int64_t>(B.max_D, D);
  }
  FD_CUDA(ctx, cudaMalloc(&B.arena, bytes));
  B.h_inst.resize(n);
  for (int i = 0; i < n; ++i) {
    const fd_matrix* M = A[i];
    BInst& I = B.h_inst[i];
    I.A.chunk_ptr = M->chunk_ptr; I.A.row_len = M->row_len; I.A.col = M->col; I.A.val = M->val;
    I.A.D = M->D; I.A.C = M->C;
    I.A32.chunk_ptr = M->chunk_ptr; I.A32.row_len = M->row_len; I.A32.col = M->col; I.A32.val = M->val32;
    I.A32.D = M->D; I.A32.C = M->C;
    I.Aff.chunk_ptr = M->chunk_ptr; I.Aff.row_len = M->row_len; I.Aff.col = M->col;
    I.Aff.val = reinterpret_cast<const ff*>(M->valff); I.Aff.D = M->D; I.Aff.C = M->C;
    I.ns = ns[i];
    const int64_t D = M->D;
    const size_t nn = (size_t)ns[i] * ns[i];
    double* p = (double*)((char*)B.arena + off[i]);
    I.V = p; p += D * ns[i];
    I.AV = p; p += D * ns[i];
    I.W = p; p += 2 * D * ns[i];
    I.G = p; p += nn;
    I.R = p; p += nn;
    I.Ri = p; p += nn;
    I.P = p; p += GSLICES * nn;
    I.theta = p; p += ns[i];
    I.resid = p; p += ns[i];
    I.V32 = nullptr;
    I.W32 = nullptr;
    if (f32) {  // after the FP64 part, 256-byte aligned
      char* q = (char*)B.arena + off[i] +
                (((sizeof(double) * (4 * D * ns[i] + 3 * nn + GSLICES * nn + 2 * ns[i] + RBLK * ns[i])) + 255) &
                 ~(size_t)255);
      I.V32 = (float*)q;
      I.W32 = I.V32 + D * ns[i];
    }
    I.rpart = p;
    for (int b = 0; b < ns[i] / nb; ++b) B.h_task.push_back({i, b});
  }
  B.h_off.assign(B.h_task.size() + 1, 0);
  for (size_t t = 0; t < B.h_task.size(); ++t)
    B.h_off[t + 1] = B.h_off[t] + cdiv(B.h_inst[B.h_task[t].inst].A.D, rpw) * rpw;
  B.rpw = rpw;
  B.n_tasks_all = B.h_task.size();
  const size_t nta = B.n_tasks_all;
  void* p;
  FD_TRY(workspace(ctx, "batch_desc", sizeof(BInst) * n + sizeof(BParams) * n + sizeof(BTask) * nta +
                                          sizeof(int64_t) * (nta + 1) + sizeof(int) * (nta + 1) + 64, &p));
  char* c = (char*)p;
  B.d_inst = (BInst*)c; c += sizeof(BInst) * n;
  B.d_par = (BParams*)c; c += sizeof(BParams) * n;
  B.d_task = (BTask*)c; c += sizeof(BTask) * nta;
  c = (char*)(((uintptr_t)c + 15) & ~(uintptr_t)15);
  B.d_off = (int64_t*)c; c += sizeof(int64_t) * (nta + 1);
  B.d_tdeg = (int*)c; c += sizeof(int) * nta;
  B.d_ntask = (int*)c;
  B.mu_cap = mu_cap;
  FD_TRY(workspace(ctx, "batch_mu", sizeof(double) * mu_cap + 64, &p));
  B.d_mu = (double*)p;
  B.d_kmax = (int*)(B.d_mu + mu_cap);
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_inst, B.h_inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice, ctx->stream));
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_task, B.h_task.data(), sizeof(BTask) * B.h_task.size(), cudaMemcpyHostToDevice, ctx->stream));
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_off, B.h_off.data(), sizeof(int64_t) * B.h_off.size(), cudaMemcpyHostToDevice, ctx->stream));
  FD_CUDA(ctx, cudaMallocHost(&B.h_par, sizeof(BParams) * n));
  FD_CUDA(ctx, cudaMallocHost(&B.h_mu, sizeof(double) * mu_cap));
  FD_CUDA(ctx, cudaMallocHost(&B.h_kmax, sizeof(int)));
  FD_CUDA(ctx, cudaMallocHost(&B.h_out, sizeof(double) * 2 * n * B.ns_max + sizeof(BParams) * n));
  FD_CUDA(ctx, cudaMallocHost(&B.h_task_p, sizeof(BTask) * nta));
  FD_CUDA(ctx, cudaMallocHost(&B.h_off_p, sizeof(int64_t) * (nta + 1)));
  FD_CUDA(ctx, cudaMallocHost(&B.h_tdeg_p, sizeof(int) * std::max<size_t>(nta, 1)));
  FD_CUDA(ctx, cudaMallocHost(&B.h_ntask, sizeof(int)));
  // until the caller sets degrees: every task, all degrees 0
  std::copy(B.h_task.begin(), B.h_task.end(), B.h_task_p);
  std::copy(B.h_off.begin(), B.h_off.end(), B.h_off_p);
  std::fill(B.h_tdeg_p, B.h_tdeg_p + nta, 0);
  *B.h_ntask = (int)nta;
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_tdeg, B.h_tdeg_p, sizeof(int) * nta, cudaMemcpyHostToDevice, ctx->stream));
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_ntask, B.h_ntask, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  // persistent filter grid: every CTA resident
  const void* kf = filter_kernel_for(nb, B.ff);
  if (!kf) return set_err(ctx, FD_ERR_ARG, "batched filter supports nb = 2 .. 64");
  B.smem_filter = sizeof(int64_t) * (nta + 1) + sizeof(int) * nta;
  if (B.smem_filter > 48 * 1024)
    FD_CUDA(ctx, cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.smem_filter));
  int per_sm = 0;
  FD_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, B.warps * 32, B.smem_filter));
  if (per_sm < 1) return set_err(ctx, FD_ERR_ARG, "batched filter does not fit on an SM");
  B.grid = per_sm * ctx->num_sms;
  // the SpMMV of the Rayleigh-Ritz step always takes FP64 rows: the FP64
  // instantiation in the tuner's CTA shape
  const void* kr = filter_kernel_for(nb, false);
  B.warps_rr = warps;
  if (B.smem_filter > 48 * 1024)
    FD_CUDA(ctx, cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.smem_filter));
  per_sm = 0;
  FD_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kr, B.warps_rr * 32, B.smem_filter));
  if (per_sm < 1) return set_err(ctx, FD_ERR_ARG, "batched SpMMV does not fit on an SM");
  B.grid_rr = per_sm * ctx->num_sms;
  return FD_OK;
}

// the host's task list (Batch::list_tasks) to the device, on the context's stream
fd_status copy_tasks(fd_ctx* ctx, Batch& B) {
  cudaStream_t st = ctx->stream;
  const size_t nta = B.n_tasks_all;
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_task, B.h_task_p, sizeof(BTask) * nta, cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_off, B.h_off_p, sizeof(int64_t) * (nta + 1), cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_tdeg, B.h_tdeg_p, sizeof(int) * nta, cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_ntask, B.h_ntask, sizeof(int), cudaMemcpyHostToDevice, st));
  return FD_OK;
}

fd_status launch_filter(fd_ctx* ctx, Batch& B, int spmmv_only) {
  BatchArgs a;
  a.inst = B.d_inst; a.par = B.d_par; a.task = B.d_task; a.task_off = B.d_off; a.mu = B.d_mu;
  a.task_deg = B.d_tdeg; a.n_tasks = B.d_ntask;
  a.kmax = B.d_kmax; a.nb = B.nb; a.spmmv_only = spmmv_only;
  void* args[] = {&a};
  const void* kf = filter_kernel_for(B.nb, B.ff);
  if (spmmv_only) {
    FD_CUDA(ctx, cudaLaunchKernel(filter_kernel_for(B.nb, false), B.grid_rr, B.warps_rr * 32, args,
                                  B.smem_filter, ctx->stream));
  } else {
    FD_CUDA(ctx, cudaLaunchCooperativeKernel(kf, B.grid, B.warps * 32, args, B.smem_filter, ctx->stream));
  }
  FD_LAUNCHED(ctx);
  return FD_OK;
}

// one outer iteration after the filter: CholQR (2 passes + conditional third),
// Rayleigh-Ritz, residuals
fd_status launch_ortho_rr(fd_ctx* ctx, Batch& B) {
  cudaStream_t st = ctx->stream;
  const int n = B.n, nsm = B.ns_max;
  const int nt = (nsm + GT - 1) / GT;
  const dim3 ggrid(nt * (nt + 1) / 2, GSLICES, n);
  const dim3 rgrid((unsigned)cdiv(B.max_D, 16), n);
  const size_t chol_smem = sizeof(double) * (nsm * nsm + 8 * nsm);
  const size_t rot_smem = sizeof(double) * 16 * nsm;
  const int np = nsm + (nsm & 1);
  const size_t jac_smem = sizeof(double) * (2 * np * np + np);
  for (int pass = 0; pass < 3; ++pass) {
    const int only_shifted = pass == 2;
    k_bgram_partial<<<ggrid, 256, 0, st>>>(B.d_inst, B.d_par, 0, only_shifted);
    FD_LAUNCHED(ctx);
    k_bgram_reduce<<<dim3((unsigned)cdiv(nsm * nsm, 256), n), 256, 0, st>>>(B.d_inst, B.d_par, only_shifted);
    FD_LAUNCHED(ctx);
    k_bchol_inv<<<n, 256, chol_smem, st>>>(B.d_inst, B.d_par, only_shifted);
    FD_LAUNCHED(ctx);
    k_brotate<<<rgrid, 256, rot_smem, st>>>(B.d_inst, B.d_par, 0, 1, only_shifted);
    FD_LAUNCHED(ctx);
  }
  FD_TRY(launch_filter(ctx, B, 1));  // AV = A V
  k_bgram_partial<<<ggrid, 256, 0, st>>>(B.d_inst, B.d_par, 1, 0);
  FD_LAUNCHED(ctx);
  k_bgram_reduce<<<dim3((unsigned)cdiv(nsm * nsm, 256), n), 256, 0, st>>>(B.d_inst, B.d_par, 0);
  FD_LAUNCHED(ctx);
  k_bjacobi<<<n, 256, jac_smem, st>>>(B.d_inst, B.d_par);
  FD_LAUNCHED(ctx);
  k_brotate<<<rgrid, 256, rot_smem, st>>>(B.d_inst, B.d_par, 0, 0, 0);
  FD_LAUNCHED(ctx);
  FD_TRY(launch_filter(ctx, B, 1));  // A (V Q) directly, cheaper than rotating AV
  k_bresid<<<dim3(RBLK, n), 128, 0, st>>>(B.d_inst, B.d_par);
  FD_LAUNCHED(ctx);
  k_bresid_reduce<<<n, 128, 0, st>>>(B.d_inst, B.d_par);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status set_kernel_smem(fd_ctx* ctx, int nsm) {
  const size_t chol_smem = sizeof(double) * (nsm * nsm + 8 * nsm);
  const size_t rot_smem = sizeof(double) * 16 * nsm;
  const int np = nsm + (nsm & 1);
  const size_t jac_smem = sizeof(double) * (2 * np * np + np);
  FD_CUDA(ctx, cudaFuncSetAttribute(k_bchol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_smem));
  FD_CUDA(ctx, cudaFuncSetAttribute(k_brotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rot_smem));
  FD_CUDA(ctx, cudaFuncSetAttribute(k_bjacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jac_smem));
  return FD_OK;
}

// the whole outer iteration as one stream sequence (captured into a graph)
fd_status enqueue_iteration(fd_ctx* ctx, Batch& B) {
  cudaStream_t st = ctx->stream;
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_par, B.h_par, sizeof(BParams) * B.n, cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_mu, B.h_mu, sizeof(double) * B.mu_cap, cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(B.d_kmax, B.h_kmax, sizeof(int), cudaMemcpyHostToDevice, st));
  FD_TRY(copy_tasks(ctx, B));
  const dim3 cgrid((unsigned)std::max(1, ctx->num_sms * 2), B.n);
  if (B.f32 || B.ff) {
    k_bconvert<<<cgrid, 256, 0, st>>>(B.d_inst, B.d_par, 1);
    FD_LAUNCHED(ctx);
  }
  FD_TRY(launch_filter(ctx, B, 0));
  if (B.f32 || B.ff) {
    k_bconvert<<<cgrid, 256, 0, st>>>(B.d_inst, B.d_par, 0);
    FD_LAUNCHED(ctx);
  }
  FD_TRY(launch_ortho_rr(ctx, B));
  for (int i = 0; i < B.n; ++i) {
    const BInst& I = B.h_inst[i];
    FD_CUDA(ctx, cudaMemcpyAsync(B.h_out + (size_t)2 * i * B.ns_max, I.theta, sizeof(double) * I.ns,
                                 cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaMemcpyAsync(B.h_out + (size_t)2 * i * B.ns_max + B.ns_max, I.resid,
                                 sizeof(double) * I.ns, cudaMemcpyDeviceToHost, st));
  }
  FD_CUDA(ctx, cudaMemcpyAsync(B.h_out + (size_t)2 * B.n * B.ns_max, B.d_par, sizeof(BParams) * B.n,
                               cudaMemcpyDeviceToHost, st));
  return FD_OK;
}

// A CUDA graph cannot be captured on the legacy default stream.  On a context
// without a stream of its own the batched solve runs on a private stream that
// first waits for the work already queued on the legacy stream; the caller's
// stream is restored (and the private stream drained) on every exit.
struct PrivateStream {
  fd_ctx* ctx;
  cudaStream_t saved;
  cudaStream_t own = nullptr;
  explicit PrivateStream(fd_ctx* c) : ctx(c), saved(c->stream) {}
  fd_status open() {
    if (saved != nullptr) return FD_OK;
    FD_CUDA(ctx, cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    cudaEvent_t ev;
    FD_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    FD_CUDA(ctx, cudaEventRecord(ev, nullptr));
    FD_CUDA(ctx, cudaStreamWaitEvent(own, ev, 0));
    FD_CUDA(ctx, cudaEventDestroy(ev));
    ctx->stream = own;
    return FD_OK;
  }
  ~PrivateStream() {
    if (!own) return;
    cudaStreamSynchronize(own);
    ctx->stream = saved;
    cudaStreamDestroy(own);
  }
};

std::vector<int> nearest(const double* th, int ns, double tau) {
  std::vector<int> o(ns);
  std::iota(o.begin(), o.end(), 0);
  std::stable_sort(o.begin(), o.end(), [&](int a, int b) {
    double da = std::fabs(th[a] - tau), db = std::fabs(th[b] - tau);
    if (da != db) return da < db;
    return th[a] < th[b];
  });
  return o;
}

}  // namespace
}  // namespace fdi

using namespace fdi;

extern "C" {

fd_status fd_solve_batched(fd_ctx* ctx, int n_inst, const fd_matrix* const* A,
                           const fd_problem* prob, int nb, int degree, double tol,
                           const fd_options* opt_in, fd_result* res, double* theta,
                           double* resid) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (n_inst < 1 || !A || !prob || !res || !theta || !resid)
    return set_err(ctx, FD_ERR_ARG, "null argument or n_inst < 1");
  fd_options opt{};
  if (opt_in) opt = *opt_in;
  if (nb != 2 && nb != 4 && nb != 8 && nb != 16 && nb != 32 && nb != 64)
    return set_err(ctx, FD_ERR_ARG, "batched nb must be 2 .. 64");
  if (degree < 2 || !(tol > 0)) return set_err(ctx, FD_ERR_ARG, "need degree >= 2 and tol > 0");
  if (opt.precision != FD_F64 && opt.precision != FD_F32 && opt.precision != FD_FF)
    return set_err(ctx, FD_ERR_ARG, "bad precision");
  if (opt.finish != FD_FINISH_F64 && opt.finish != FD_FINISH_FF)
    return set_err(ctx, FD_ERR_ARG, "finish must be FD_FINISH_F64 or FD_FINISH_FF");
  const bool f32 = opt.precision == FD_F32;
  // float-float sweeps: the FF form, or the FP32 form's finish
  const bool ffs = opt.precision == FD_FF || (f32 && opt.finish == FD_FINISH_FF);
  if (f32 && nb < 4) return set_err(ctx, FD_ERR_ARG, "FP32 sweeps need nb >= 4");
  std::vector<int> ns(n_inst);
  for (int i = 0; i < n_inst; ++i) {
    if (!A[i] || !A[i]->identity)
      return set_err(ctx, FD_ERR_ARG, "instance %d: batched solves need matrices with sigma = 1", i);
    ns[i] = opt.ns > 0 ? opt.ns : nb * (int)cdiv(4LL * prob[i].n_target, nb);
    if (prob[i].n_target < 1 || ns[i] > BMAX_NS || ns[i] > A[i]->D || ns[i] % nb ||
        !(prob[i].a <= prob[i].b))
      return set_err(ctx, FD_ERR_ARG, "instance %d: need 1 <= n_target, ns <= min(%d, D), a <= b", i,
                     BMAX_NS);
  }
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  PrivateStream pstream(ctx);
  FD_TRY(pstream.open());
  const int max_outer = opt.max_outer > 0 ? opt.max_outer : 60;
  const int n_max = opt.n_max > 0 ? opt.n_max : 100000;
  const int lsteps = opt.lanczos_steps > 0 ? opt.lanczos_steps : 20;
  const double c_n = opt.c_n > 0 ? opt.c_n : 4.0;
  const double m_l = opt.m_l > 0 ? opt.m_l : 0.5, m_r = opt.m_r > 0 ? opt.m_r : 0.5;
  const int warps = opt.cta_warps == 4 ? 4 : WARPS;  // CTA shape (the tuner's choice)
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);

  Batch B;
  const size_t mu_cap = (size_t)n_inst * (n_max + 1);
  fd_status s = batch_setup(ctx, B, n_inst, A, ns.data(), nb, warps, mu_cap, f32, ffs);
  if (s != FD_OK) { B.release(); return s; }
  s = set_kernel_smem(ctx, B.ns_max);
  if (s != FD_OK) { B.release(); return s; }
  // inclusion intervals and start blocks
  std::vector<double> lam_l(n_inst), lam_r(n_inst), widen(n_inst);
  std::vector<double> wl(n_inst), wr(n_inst);
  std::vector<int> deg(n_inst, degree), conv(n_inst, 0), iters(n_inst, 0);
  std::vector<int64_t> nsp(n_inst, 0), nsp32(n_inst, 0), nspff(n_inst, 0);
  // the FP32 form's switch per instance (fd_solve's rule): FP32 sweeps until the
  // largest wanted residual reaches 100 u32 |H| or fails to halve twice in a row
  std::vector<int> use32(n_inst, f32 ? 1 : 0), stall(n_inst, 0);
  std::vector<double> prev_max(n_inst, INFINITY), norm_h(n_inst, 0.0);
  for (int i = 0; i < n_inst; ++i) {
    s = spectral_bounds(ctx, A[i], lsteps, prob[i].seed, &lam_l[i], &lam_r[i]);
    if (s != FD_OK) { B.release(); return s; }
    widen[i] = 0.01 * (lam_r[i] - lam_l[i]);
    norm_h[i] = std::max(std::fabs(lam_l[i]), std::fabs(lam_r[i]));
    k_bstart<<<(unsigned)cdiv(A[i]->D * ns[i], 256), 256, 0, st>>>(
        B.h_inst[i].V, A[i]->D * ns[i], fdrng::key(prob[i].seed, fdrng::STREAM_START));
    ctx->launches++;
    wl[i] = prob[i].a;
    wr[i] = prob[i].b;
  }
  // first iteration: no filter, orthonormalise + Rayleigh-Ritz
  for (int i = 0; i < n_inst; ++i) B.h_par[i] = BParams{1, 0, 0, 0, 0.0, 0.0, 0, 0};
  *B.h_kmax = 0;
  B.list_tasks();
  // capture one iteration as a graph; replay it every outer iteration
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    s = enqueue_iteration(ctx, B);
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (s != FD_OK || ce != cudaSuccess ||
        cudaGraphInstantiate(&B.exec, graph, 0) != cudaSuccess) {
      use_graph = false;
      cudaGetLastError();
      if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
    }
    if (graph) cudaGraphDestroy(graph);
  } else {
    use_graph = false;
    cudaGetLastError();
  }
  ctx->err.clear();
  int it = 0;
  int n_left = n_inst;
  for (; it < max_outer && n_left > 0; ++it) {
    if (use_graph) {
      FD_CUDA(ctx, cudaGraphLaunch(B.exec, st));
    } else {
      s = enqueue_iteration(ctx, B);
      if (s != FD_OK) { B.release(); return s; }
    }
    FD_CUDA(ctx, cudaStreamSynchronize(st));
    if (opt.verbose) {
      int n32 = 0;
      for (int i = 0; i < n_inst; ++i) n32 += B.h_par[i].active && B.h_par[i].f32 && B.h_par[i].degree > 0;
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float msv = 0;
      cudaEventElapsedTime(&msv, e0, e1);
      fprintf(stderr, "batched it %d: active %d (FP32 sweeps %d), top degree %d, elapsed %.2f s\n", it,
              n_left, n32, *B.h_kmax, msv * 1e-3);
    }
    const BParams* dev_par = (const BParams*)(B.h_out + (size_t)2 * n_inst * B.ns_max);
    int kmax = 0;
    size_t mu_off = 0;
    for (int i = 0; i < n_inst; ++i) {
      BParams& P = B.h_par[i];
      if (!P.active) continue;
      if (P.degree > 0) nsp[i] += P.degree;
      if (P.degree > 0 && P.f32) nsp32[i] += P.degree;
      if (P.degree > 0 && P.ff) nspff[i] += P.degree;
      nsp[i] += 1;
      if (dev_par[i].flags & 2) {
        B.release();
        return set_err(ctx, FD_ERR_BREAKDOWN, "instance %d: shifted Cholesky-QR broke down", i);
      }
      iters[i]++;
      const double* th = B.h_out + (size_t)2 * i * B.ns_max;
      const double* rh = th + B.ns_max;
      const int nsi = ns[i];
      const int nt = prob[i].n_target;
      const double tau = 0.5 * (prob[i].a + prob[i].b);
      std::vector<int> order = nearest(th, nsi, tau);
      int nconv = 0;
      double maxr = 0.0;
      for (int q = 0; q < nt; ++q) {
        nconv += rh[order[q]] <= tol;
        maxr = std::max(maxr, rh[order[q]]);
      }
      if (nconv == nt) {
        conv[i] = 1;
        P.active = 0;
        P.degree = 0;
        --n_left;
        std::vector<int> sel(order.begin(), order.begin() + nt);
        std::sort(sel.begin(), sel.end(), [&](int x, int y) { return th[x] < th[y]; });
        int64_t o = 0;
        for (int q = 0; q < i; ++q) o += prob[q].n_target;
        for (int q = 0; q < nt; ++q) { theta[o + q] = th[sel[q]]; resid[o + q] = rh[sel[q]]; }
        continue;
      }
      if (th[0] < lam_l[i]) lam_l[i] = std::min(lam_l[i] - 2 * widen[i], th[0] - widen[i]);
      if (th[nsi - 1] > lam_r[i]) lam_r[i] = std::max(lam_r[i] + 2 * widen[i], th[nsi - 1] + widen[i]);
      const double alpha = 2.0 / (lam_r[i] - lam_l[i]), beta = -(lam_r[i] + lam_l[i]) / (lam_r[i] - lam_l[i]);
      int n = deg[i];
      if (iters[i] > 1) {
        double t_l = INFINITY, t_r = -INFINITY, s_l = INFINITY, s_r = -INFINITY;
        for (int q = 0; q < nt; ++q) { t_l = std::min(t_l, th[order[q]]); t_r = std::max(t_r, th[order[q]]); }
        const int nsrch = (int)std::ceil(0.75 * nsi);
        for (int q = 0; q < nsrch; ++q) { s_l = std::min(s_l, th[order[q]]); s_r = std::max(s_r, th[order[q]]); }
        s_l = std::min(s_l, t_l);
        s_r = std::max(s_r, t_r);
        auto ang = [&](double lam) { return std::acos(std::min(1.0, std::max(-1.0, alpha * lam + beta))); };
        const double dth = std::min(ang(s_l) - ang(t_l), ang(t_r) - ang(s_r));
        const double cn_i = prob[i].c_n > 0 ? prob[i].c_n : c_n;
        const double ml_i = prob[i].m_l > 0 ? prob[i].m_l : m_l;
        const double mr_i = prob[i].m_r > 0 ? prob[i].m_r : m_r;
        long long nn = dth <= 0.0 ? n_max : (long long)std::ceil(cn_i * M_PI / dth);
        n = (int)std::max<long long>(degree, std::min<long long>(n_max, nn));
        wl[i] = t_l - ml_i * (t_l - s_l);
        wr[i] = t_r + mr_i * (s_r - t_r);
      }
      deg[i] = n;
      std::vector<double> mu = filter_coeffs(alpha * wl[i] + beta, alpha * wr[i] + beta, n);
      std::copy(mu.begin(), mu.end(), B.h_mu + mu_off);
      P.degree = n;
      P.mu_off = (int)mu_off;
      P.alpha = alpha;
      P.beta = beta;
      P.flags = 0;
      stall[i] = maxr > 0.5 * prev_max[i] ? stall[i] + 1 : 0;
      if (use32[i] && (maxr <= 100.0 * 0x1.0p-24 * norm_h[i] || stall[i] >= 2)) use32[i] = 0;
      prev_max[i] = maxr;
      P.f32 = use32[i];
      P.ff = !use32[i] && ffs;
      mu_off += n + 1;
      kmax = std::max(kmax, n);
    }
    *B.h_kmax = kmax;
    B.list_tasks();
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int64_t o = 0;
  for (int i = 0; i < n_inst; ++i) {
    fd_result& r = res[i];
    r = fd_result{};
    r.converged = conv[i];
    r.iterations = iters[i];
    r.n_spmmv = nsp[i];
    r.n_spmmv_f32 = nsp32[i];
    r.n_spmmv_ff = nspff[i];
    r.final_degree = deg[i];
    r.ns = ns[i];
    r.lam_l = lam_l[i];
    r.lam_r = lam_r[i];
    r.window_l = wl[i];
    r.window_r = wr[i];
    r.t_total = ms * 1e-3;
    r.used_graph = use_graph ? 1 : 0;
    if (!conv[i])
      for (int q = 0; q < prob[i].n_target; ++q) { theta[o + q] = NAN; resid[o + q] = INFINITY; }
    o += prob[i].n_target;
  }
  B.release();
  if (n_left > 0) return set_err(ctx, FD_ERR_NOCONV, "%d of %d instances did not converge", n_left, n_inst);
  return FD_OK;
}

fd_status fd_tune_batched(fd_ctx* ctx, int n_inst, const char* const* specs, int n_target,
                          int probe_degree, int* nb_out, int* C_out, int* warps_out,
                          double* gbs_out) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (n_inst < 1 || !specs || !nb_out || !C_out || !warps_out || !gbs_out || n_target < 1 ||
      probe_degree < 3)
    return set_err(ctx, FD_ERR_ARG, "need specs, outputs, n_target >= 1, probe_degree >= 3");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  double best = -1.0;
  const int Cs[] = {32, 64, 128};
  const int nbs[] = {8, 16, 32, 64};
  const int ws[] = {4, 8};
  for (int C : Cs) {
    std::vector<fd_matrix*> M(n_inst, nullptr);
    fd_status s = FD_OK;
    for (int i = 0; i < n_inst && s == FD_OK; ++i) s = fd_build_matrix_sell(ctx, specs[i], C, 1, &M[i]);
    for (int nb : nbs) {
      const int ns = nb * (int)cdiv(4LL * n_target, nb);
      if (s != FD_OK || ns > BMAX_NS) continue;
      bool fits = true;
      for (int i = 0; i < n_inst; ++i) fits &= ns <= M[i]->D;
      if (!fits) continue;
      for (int w : ws) {
        Batch B;
        std::vector<int> nsv(n_inst, ns);
        s = batch_setup(ctx, B, n_inst, M.data(), nsv.data(), nb, w, (size_t)probe_degree + 1);
        if (s != FD_OK) { B.release(); break; }
        double bytes = 0.0;
        for (int i = 0; i < n_inst; ++i) {
          k_bstart<<<(unsigned)cdiv(M[i]->D * ns, 256), 256, 0, st>>>(B.h_inst[i].V, M[i]->D * ns,
                                                                     fdrng::key(i, fdrng::STREAM_START));
          ctx->launches++;
          const double a = 2.0 / (M[i]->gersh_hi - M[i]->gersh_lo + 1e-3);
          const double b = -(M[i]->gersh_hi + M[i]->gersh_lo) / (M[i]->gersh_hi - M[i]->gersh_lo + 1e-3);
          B.h_par[i] = BParams{1, probe_degree, 0, 0, a, b, 0, 0};
          const double vec = (double)nb * M[i]->D * 8.0, mat = (double)M[i]->nnz * 12.0;
          const int n = probe_degree;
          bytes += (ns / nb) * ((mat + 2 * vec) + (mat + 4 * vec) + (n - 3) * (mat + 5 * vec) + (mat + 4 * vec));
        }
        std::vector<double> mu(probe_degree + 1);
        for (int k = 0; k <= probe_degree; ++k) mu[k] = 1.0 / (k + 1);
        std::copy(mu.begin(), mu.end(), B.h_mu);
        *B.h_kmax = probe_degree;
        B.list_tasks();
        s = copy_tasks(ctx, B);
        if (s != FD_OK) { B.release(); break; }
        FD_CUDA(ctx, cudaMemcpyAsync(B.d_par, B.h_par, sizeof(BParams) * n_inst, cudaMemcpyHostToDevice, st));
        FD_CUDA(ctx, cudaMemcpyAsync(B.d_mu, B.h_mu, sizeof(double) * (probe_degree + 1), cudaMemcpyHostToDevice, st));
        FD_CUDA(ctx, cudaMemcpyAsync(B.d_kmax, B.h_kmax, sizeof(int), cudaMemcpyHostToDevice, st));
        s = launch_filter(ctx, B, 0);  // warm-up
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 2 && s == FD_OK; ++r) s = launch_filter(ctx, B, 0);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        B.release();
        if (s != FD_OK) break;
        const double gbs = 2.0 * bytes / (ms * 1e-3) / 1e9;
        if (gbs > best) {
          best = gbs;
          *nb_out = nb;
          *C_out = C;
          *warps_out = w;
          *gbs_out = gbs;
        }
      }
    }
    for (auto* m : M)
      if (m) fd_matrix_free(m);
    if (s != FD_OK) return s;
  }
  if (best < 0) return set_err(ctx, FD_ERR_ARG, "no candidate configuration fits (N_s <= %d)", BMAX_NS);
  return FD_OK;
}

}  // extern "C"
