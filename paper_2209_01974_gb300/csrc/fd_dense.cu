// Dense FP64 kernels of the FD loop: tall-skinny Gram products, in-place block
// rotations, Cholesky and triangular inverse (Cholesky-QR, Sec. 2), the
// parallel cyclic Jacobi eigensolver of the Rayleigh-Ritz step (Sec. 2) and
// the residual norms rho_i = ||A v_i - theta_i v_i||_2 (Sec. 2, Alg. 1).
//
// FP64 arithmetic on GB300 runs at about 1.2 TFLOP/s, so these kernels are
// FP64-ALU bound; they use register tiles fed from shared memory and split the
// long dimension D across CTAs with a deterministic second-pass reduction.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fd_internal.cuh"

namespace cg = cooperative_groups;

namespace fdi {
namespace {

// ---------------------------------------------------------------------------
// Gram: P[slice] = X[rows of slice]^T Y[rows of slice], 64 x 64 output tiles
// ---------------------------------------------------------------------------
constexpr int GT = 64;   // tile edge
constexpr int GK = 16;   // rows per shared-memory stage

__global__ void __launch_bounds__(256)
    k_gram_partial(const double* __restrict__ X, int64_t ldx, const double* __restrict__ Y,
                   int64_t ldy, int64_t D, int m, int n, int ntj, bool sym, int64_t rows_per_slice,
                   double* __restrict__ P) {
  __shared__ double Xs[GK][GT], Ys[GK][GT];
  // tile coordinates
  int t = blockIdx.x, ti, tj;
  if (sym) {  // enumerate ti <= tj
    ti = 0;
    int rowlen = ntj;
    while (t >= rowlen) { t -= rowlen; ++ti; --rowlen; }
    tj = ti + t;
  } else {
    ti = t / ntj;
    tj = t % ntj;
  }
  const int i0 = ti * GT, j0 = tj * GT;
  const int64_t k0 = (int64_t)blockIdx.y * rows_per_slice;
  const int64_t k1 = min(D, k0 + rows_per_slice);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int64_t kb = k0; kb < k1; kb += GK) {
#pragma unroll
    for (int q = 0; q < (GK * GT) / 256; ++q) {
      int e = threadIdx.x + q * 256;
      int kk = e / GT, c = e % GT;
      int64_t k = kb + kk;
      Xs[kk][c] = (k < k1 && i0 + c < m) ? X[k * ldx + i0 + c] : 0.0;
      Ys[kk][c] = (k < k1 && j0 + c < n) ? Y[k * ldy + j0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = Xs[kk][ty + 16 * u]; b[u] = Ys[kk][tx + 16 * u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* Ps = P + (int64_t)blockIdx.y * m * n;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < m && j < n) Ps[(int64_t)i * n + j] = acc[u][v];
    }
}

__global__ void k_gram_reduce(const double* P, int slices, int m, int n, bool sym, double* C,
                              int ldc) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  if (sym && i / GT > j / GT) return;  // computed by the mirrored tile
  double s = 0.0;
  for (int q = 0; q < slices; ++q) s += P[(int64_t)q * m * n + e];
  C[(int64_t)i * ldc + j] = s;
  if (sym && i / GT < j / GT) C[(int64_t)j * ldc + i] = s;
}

// ---------------------------------------------------------------------------
// rotate: V[rows] <- V[rows] * M, in place, TR rows per CTA
// ---------------------------------------------------------------------------
constexpr int RT = 16;  // rows per CTA

__global__ void __launch_bounds__(256)
    k_rotate(double* V, int64_t ldv, int64_t D, int n, const double* __restrict__ M, bool upper) {
  extern __shared__ double Vt[];  // RT x n
  const int64_t r0 = (int64_t)blockIdx.x * RT;
  const int nr = D - r0 < RT ? (int)(D - r0) : RT;
  for (int e = threadIdx.x; e < RT * n; e += 256) {
    int r = e / n, c = e % n;
    Vt[e] = r < nr ? V[(r0 + r) * ldv + c] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x >> 4;   // 0..15
  const int c0 = threadIdx.x & 15;  // columns c0 + 16 v
  for (int cb = 0; cb < n; cb += 64) {
    double acc[4] = {0, 0, 0, 0};
    const int kend = upper ? min(n, cb + 64) : n;
    const double* vr = Vt + r * n;
    for (int k = 0; k < kend; ++k) {
      const double a = vr[k];
      const double* mk = M + (int64_t)k * n + cb + c0;
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (cb + c0 + 16 * v < n) acc[v] = fma(a, __ldg(mk + 16 * v), acc[v]);
    }
    if (r < nr) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int c = cb + c0 + 16 * v;
        if (c < n) V[(r0 + r) * ldv + c] = acc[v];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Cholesky (one CTA): R upper with R^T R = G + shift I, shift = coeff * tr(G)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_cholesky(const double* G, int n, double coeff,
                                                   double* R, int* ok) {
  __shared__ double sh_tr[1024];
  __shared__ int fail;
  __shared__ double rinv;
  double tr = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tr += G[(int64_t)i * n + i];
  sh_tr[threadIdx.x] = tr;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh_tr[threadIdx.x] += sh_tr[threadIdx.x + o];
    __syncthreads();
  }
  const double shift = coeff * sh_tr[0];
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    R[e] = j >= i ? G[e] + (i == j ? shift : 0.0) : 0.0;
  }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double d = R[(int64_t)k * n + k];
      if (!(d > 0.0) || !isfinite(d)) {
        fail = 1;
      } else {
        double r = sqrt(d);
        R[(int64_t)k * n + k] = r;
        rinv = 1.0 / r;
      }
    }
    __syncthreads();
    if (fail) break;
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) R[(int64_t)k * n + j] *= rinv;
    __syncthreads();
    const int m = n - k - 1;
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
      int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
      if (j >= i) R[(int64_t)i * n + j] -= R[(int64_t)k * n + i] * R[(int64_t)k * n + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *ok = fail ? 0 : 1;
}

// Cooperative version (one CTA per SM): the same right-looking elimination,
// each step's trailing update spread over the CTAs by rows, one grid barrier
// per column.  Row k is read unscaled during step k (the update uses
// R_kj R_ki / d) and scaled by its owner after the barrier, when no CTA reads it
// any more.  Reads of R bypass L1 (other CTAs wrote them).
__global__ void __launch_bounds__(256) k_cholesky_coop(const double* G, int n, double coeff, double* R,
                                                       int* ok) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[256];
  double tr = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tr += G[(int64_t)i * n + i];
  red[threadIdx.x] = tr;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double shift = coeff * red[0];
  for (int i = blockIdx.x; i < n; i += gridDim.x)
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      R[(int64_t)i * n + j] = j >= i ? G[(int64_t)i * n + j] + (i == j ? shift : 0.0) : 0.0;
  grid.sync();
  bool fail = false;
  for (int k = 0; k < n; ++k) {
    const double d = __ldcg(R + (int64_t)k * n + k);
    if (!(d > 0.0) || !isfinite(d)) {  // the same value in every CTA: all stop here
      fail = true;
      break;
    }
    const double inv = 1.0 / d;
    const double* rk = R + (int64_t)k * n;
    for (int i = k + 1 + blockIdx.x; i < n; i += gridDim.x) {
      const double a = __ldcg(rk + i) * inv;
      double* ri = R + (int64_t)i * n;
      for (int j = i + threadIdx.x; j < n; j += blockDim.x) ri[j] -= a * __ldcg(rk + j);
    }
    grid.sync();
    if (k % gridDim.x == blockIdx.x) {
      const double r = sqrt(d), rinv = 1.0 / r;
      double* rw = R + (int64_t)k * n;
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) rw[j] *= rinv;
      if (threadIdx.x == 0) rw[k] = r;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *ok = fail ? 0 : 1;
}

// ---------------------------------------------------------------------------
// triangular inverse: X = R^-1 (upper), one warp per column
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tri_inverse(const double* R, int n, double* X) {
  extern __shared__ double xs[];  // 8 warps x n
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + w;
  if (j >= n) return;
  double* x = xs + (int64_t)w * n;
  for (int i = j; i >= 0; --i) {
    double s = 0.0;
    for (int k = i + 1 + lane; k <= j; k += 32) s = fma(R[(int64_t)i * n + k], x[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[i] = ((i == j ? 1.0 : 0.0) - s) / R[(int64_t)i * n + i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) X[(int64_t)i * n + j] = i <= j ? x[i] : 0.0;
}

// C = A * B, n x n (small)
__global__ void k_small_gemm(const double* A, const double* B, double* C, int n) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  double s = 0.0;
  for (int k = 0; k < n; ++k) s = fma(A[(int64_t)i * n + k], B[(int64_t)k * n + j], s);
  C[e] = s;
}

__global__ void k_identity(double* A, int n) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)n * n) A[e] = (e / n == e % n) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// parallel cyclic Jacobi (round-robin pairing), cooperative grid
// ---------------------------------------------------------------------------
struct JacobiArgs {
  double* A0;   // np x np, current
  double* A1;   // np x np, next
  double* Q;    // np x np, accumulated rotations
  double* part; // gridDim.x partial sums
  int n, np;
  int max_sweeps;
  double rel_tol;
  int* sweeps_out;
};

__device__ __forceinline__ void pair_of(int round, int k, int np, int* p, int* q) {
  int a, b;
  const int m = np - 1;
  if (k == 0) { a = round % m; b = m; }
  else { a = (round + k) % m; b = (round - k + m) % m; }
  *p = min(a, b);
  *q = max(a, b);
}

__device__ __forceinline__ void rot_params(const double* A, int np, int p, int q, double* c,
                                           double* s) {
  const double apq = A[(int64_t)p * np + q];
  if (apq == 0.0) { *c = 1.0; *s = 0.0; return; }
  const double app = A[(int64_t)p * np + p], aqq = A[(int64_t)q * np + q];
  const double tau = (aqq - app) / (2.0 * apq);
  const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  *c = 1.0 / sqrt(1.0 + t * t);
  *s = t * (*c);
}

__device__ double grid_sum(cg::grid_group& grid, double v, double* part, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
  grid.sync();
  double s = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) s += part[b];  // same order in every CTA
  grid.sync();  // every CTA has read `part` before it is reused
  return s;
}

__global__ void __launch_bounds__(256) k_jacobi(JacobiArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[256];
  extern __shared__ double cs[];  // np/2 (c, s) pairs for the current round
  const int np = a.np, half = np / 2;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  double* Acur = a.A0;
  double* Anext = a.A1;
  // Frobenius norm of A
  double f = 0.0;
  for (int64_t e = gtid; e < (int64_t)np * np; e += gthreads) f += Acur[e] * Acur[e];
  const double fro2 = grid_sum(grid, f, a.part, sh);
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    double off = 0.0;
    for (int64_t e = gtid; e < (int64_t)np * np; e += gthreads)
      if (e / np != e % np) off += Acur[e] * Acur[e];
    const double off2 = grid_sum(grid, off, a.part, sh);
    if (off2 <= a.rel_tol * a.rel_tol * fro2) break;
    for (int round = 0; round < np - 1; ++round) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int p, q;
        pair_of(round, k, np, &p, &q);
        rot_params(Acur, np, p, q, &cs[2 * k], &cs[2 * k + 1]);
      }
      __syncthreads();
      // 2 x 2 blocks (pair k rows) x (pair l cols): B = J_k^T A J_l
      for (int64_t e = gtid; e < (int64_t)half * half; e += gthreads) {
        const int k = (int)(e / half), l = (int)(e % half);
        int p, q, r, s;
        pair_of(round, k, np, &p, &q);
        pair_of(round, l, np, &r, &s);
        const double ck = cs[2 * k], sk = cs[2 * k + 1], cl = cs[2 * l], sl = cs[2 * l + 1];
        const double apr = Acur[(int64_t)p * np + r], aps = Acur[(int64_t)p * np + s];
        const double aqr = Acur[(int64_t)q * np + r], aqs = Acur[(int64_t)q * np + s];
        const double m0r = ck * apr - sk * aqr, m0s = ck * aps - sk * aqs;
        const double m1r = sk * apr + ck * aqr, m1s = sk * aps + ck * aqs;
        double bpr = m0r * cl - m0s * sl, bps = m0r * sl + m0s * cl;
        double bqr = m1r * cl - m1s * sl, bqs = m1r * sl + m1s * cl;
        if (k == l) { bps = 0.0; bqr = 0.0; }
        Anext[(int64_t)p * np + r] = bpr; Anext[(int64_t)p * np + s] = bps;
        Anext[(int64_t)q * np + r] = bqr; Anext[(int64_t)q * np + s] = bqs;
      }
      // Q <- Q J (rows independent)
      for (int64_t e = gtid; e < (int64_t)np * half; e += gthreads) {
        const int i = (int)(e / half), l = (int)(e % half);
        int r, s;
        pair_of(round, l, np, &r, &s);
        const double cl = cs[2 * l], sl = cs[2 * l + 1];
        const double qr = a.Q[(int64_t)i * np + r], qs = a.Q[(int64_t)i * np + s];
        a.Q[(int64_t)i * np + r] = cl * qr - sl * qs;
        a.Q[(int64_t)i * np + s] = sl * qr + cl * qs;
      }
      grid.sync();
      double* t = Acur; Acur = Anext; Anext = t;
    }
  }
  if (gtid == 0) *a.sweeps_out = sweep;
  // make the final matrix available in A0
  if (Acur != a.A0)
    for (int64_t e = gtid; e < (int64_t)np * np; e += gthreads) a.A0[e] = Acur[e];
}

// sort eigenpairs ascending (ties by index) and copy the n x n leading block
__global__ void k_eig_sort(const double* A, const double* Q, int n, int np, double* w,
                           double* Qout) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ai = A[(int64_t)i * np + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double aj = A[(int64_t)j * np + j];
      rank += (aj < ai) || (aj == ai && j < i);
    }
    w[rank] = ai;
    for (int r = 0; r < n; ++r) Qout[(int64_t)r * n + rank] = Q[(int64_t)r * np + i];
  }
}

__global__ void k_pad_square(const double* H, int n, int np, double* A, double* Q) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)np * np) return;
  int i = (int)(e / np), j = (int)(e % np);
  A[e] = (i < n && j < n) ? H[(int64_t)i * n + j] : 0.0;
  Q[e] = i == j ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// residual norms
// ---------------------------------------------------------------------------
__global__ void k_resid_partial(const double* V, const double* AV, int64_t ld, int64_t D, int n,
                                const double* theta, double* P) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double th = theta[c];
    double s = 0.0;
    for (int64_t r = blockIdx.x; r < D; r += gridDim.x) {
      const double d = AV[r * ld + c] - th * V[r * ld + c];
      s = fma(d, d, s);
    }
    P[(int64_t)blockIdx.x * n + c] = s;
  }
}

__global__ void k_resid_reduce(const double* P, int nb, int n, double* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += P[(int64_t)b * n + c];
  out[c] = sqrt(s);
}

__global__ void k_f64_to_f32(const double* s, int64_t lds, float* d, int64_t ldd, int64_t D, int n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * n) return;
  int64_t i = t / n;
  int j = (int)(t % n);
  d[i * ldd + j] = (float)s[i * lds + j];
}
__global__ void k_f32_to_f64(const float* s, int64_t lds, double* d, int64_t ldd, int64_t D, int n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * n) return;
  int64_t i = t / n;
  int j = (int)(t % n);
  d[i * ldd + j] = (double)s[i * lds + j];
}
// FP64 <-> float-float (element = 2 floats): hi the nearest float, lo the
// nearest float to the exact FP64 remainder; back, hi + lo is exact in FP64
__global__ void k_f64_to_ff(const double* s, int64_t lds, float* d, int64_t ldd, int64_t D, int n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * n) return;
  int64_t i = t / n;
  int j = (int)(t % n);
  const double v = s[i * lds + j];
  const float hi = __double2float_rn(v);
  *reinterpret_cast<float2*>(d + 2 * (i * ldd + j)) = make_float2(hi, __double2float_rn(v - (double)hi));
}
__global__ void k_ff_to_f64(const float* s, int64_t lds, double* d, int64_t ldd, int64_t D, int n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * n) return;
  int64_t i = t / n;
  int j = (int)(t % n);
  const float2 v = *reinterpret_cast<const float2*>(s + 2 * (i * lds + j));
  d[i * ldd + j] = (double)v.x + (double)v.y;
}

}  // namespace

// tall-skinny products large enough for the tensor-core splitting to pay off
static bool use_ozaki(const fd_ctx* ctx, int64_t D, int m, int n) {
  if (ctx->gemm_mode == FD_GEMM_FP64) return false;
  if (ctx->gemm_mode == FD_GEMM_OZAKI) return true;
  return D >= 65536 && m >= 64 && n >= 64;
}

fd_status gram(fd_ctx* ctx, const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t D,
               int m, int n, double* C, int ldc, bool sym) {
  if (use_ozaki(ctx, D, m, n)) {
    bool used = false;
    FD_TRY(oz_gram(ctx, X, ldx, Y, ldy, D, m, n, C, ldc, sym, &used));
    if (used) return FD_OK;
  }
  const int nti = (int)cdiv(m, GT), ntj = (int)cdiv(n, GT);
  const int tiles = sym ? nti * (nti + 1) / 2 : nti * ntj;
  int64_t slices = std::max<int64_t>(1, cdiv(4LL * ctx->num_sms, tiles));
  slices = std::min<int64_t>(slices, std::max<int64_t>(1, cdiv(D, 4 * GK)));
  const int64_t rps = cdiv(cdiv(D, slices), GK) * GK;
  slices = std::max<int64_t>(1, cdiv(D, rps));
  void* p;
  FD_TRY(workspace(ctx, "gram_partial", sizeof(double) * slices * m * n, &p));
  double* P = (double*)p;
  dim3 grid(tiles, (unsigned)slices);
  k_gram_partial<<<grid, 256, 0, ctx->stream>>>(X, ldx, Y, ldy, D, m, n, ntj, sym, rps, P);
  FD_LAUNCHED(ctx);
  k_gram_reduce<<<(unsigned)cdiv((int64_t)m * n, 256), 256, 0, ctx->stream>>>(P, (int)slices, m, n,
                                                                             sym, C, ldc);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status gram_partials(fd_ctx* ctx, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                        int64_t D, int m, int n, double* C, int ldc, bool sym, double* P,
                        int64_t max_slices) {
  const int nti = (int)cdiv(m, GT), ntj = (int)cdiv(n, GT);
  const int tiles = sym ? nti * (nti + 1) / 2 : nti * ntj;
  int64_t slices = std::max<int64_t>(1, cdiv(4LL * ctx->num_sms, tiles));
  slices = std::min<int64_t>(slices, std::max<int64_t>(1, cdiv(D, 4 * GK)));
  slices = std::max<int64_t>(1, std::min<int64_t>(slices, max_slices));
  const int64_t rps = cdiv(cdiv(D, slices), GK) * GK;
  slices = std::max<int64_t>(1, cdiv(D, rps));
  dim3 grid(tiles, (unsigned)slices);
  k_gram_partial<<<grid, 256, 0, ctx->stream>>>(X, ldx, Y, ldy, D, m, n, ntj, sym, rps, P);
  FD_LAUNCHED(ctx);
  k_gram_reduce<<<(unsigned)cdiv((int64_t)m * n, 256), 256, 0, ctx->stream>>>(P, (int)slices, m, n,
                                                                             sym, C, ldc);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status identity_dev(fd_ctx* ctx, double* A, int n) {
  k_identity<<<(unsigned)cdiv((int64_t)n * n, 256), 256, 0, ctx->stream>>>(A, n);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status small_gemm_dev(fd_ctx* ctx, const double* A, const double* B, double* C, int n) {
  k_small_gemm<<<(unsigned)cdiv((int64_t)n * n, 256), 256, 0, ctx->stream>>>(A, B, C, n);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status rotate(fd_ctx* ctx, double* V, int64_t ldv, int64_t D, int n, const double* M, bool upper) {
  if (use_ozaki(ctx, D, n, n)) {
    bool used = false;
    FD_TRY(oz_rotate(ctx, V, ldv, D, n, M, upper, &used));
    if (used) return FD_OK;
  }
  return rotate_fp64(ctx, V, ldv, D, n, M, upper);
}

fd_status rotate_fp64(fd_ctx* ctx, double* V, int64_t ldv, int64_t D, int n, const double* M,
                      bool upper) {
  const size_t smem = sizeof(double) * RT * n;
  if (smem > ctx->smem_optin) return set_err(ctx, FD_ERR_ARG, "block too wide for rotation (%d)", n);
  if (smem > 48 * 1024)
    FD_CUDA(ctx, cudaFuncSetAttribute(k_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_rotate<<<(unsigned)cdiv(D, RT), 256, smem, ctx->stream>>>(V, ldv, D, n, M, upper);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status cholesky(fd_ctx* ctx, const double* G, int n, double coeff, double* R, int* ok_dev) {
  if (n >= 64) {  // one CTA per SM, co-resident (cooperative launch)
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cholesky_coop, 256, 0);
    if (per_sm >= 1) {
      const int grid = std::min(ctx->num_sms, n);
      void* args[] = {(void*)&G, (void*)&n, (void*)&coeff, (void*)&R, (void*)&ok_dev};
      if (cudaLaunchCooperativeKernel((const void*)k_cholesky_coop, grid, 256, args, 0, ctx->stream) ==
          cudaSuccess) {
        ctx->launches++;
        return FD_OK;
      }
      cudaGetLastError();  // cooperative launch unavailable: the one-CTA kernel below
    }
  }
  k_cholesky<<<1, 1024, 0, ctx->stream>>>(G, n, coeff, R, ok_dev);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status tri_inverse(fd_ctx* ctx, const double* R, int n, double* Rinv) {
  const size_t smem = sizeof(double) * 8 * n;
  if (smem > 48 * 1024)
    FD_CUDA(ctx, cudaFuncSetAttribute(k_tri_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_tri_inverse<<<(unsigned)cdiv(n, 8), 256, smem, ctx->stream>>>(R, n, Rinv);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status sym_eig(fd_ctx* ctx, double* H, int n, double* w, double* Q, int max_sweeps) {
  const int np = n + (n & 1);
  void* p;
  FD_TRY(workspace(ctx, "jacobi", sizeof(double) * (3 * (size_t)np * np + 4096) + 64, &p));
  double* A0 = (double*)p;
  double* A1 = A0 + (size_t)np * np;
  double* Qw = A1 + (size_t)np * np;
  double* part = Qw + (size_t)np * np;
  int* sweeps = (int*)(part + 4096);
  const int T = 256;
  k_pad_square<<<(unsigned)cdiv((int64_t)np * np, T), T, 0, ctx->stream>>>(H, n, np, A0, Qw);
  FD_LAUNCHED(ctx);
  const size_t smem = sizeof(double) * np;  // np/2 (c, s) pairs
  int per_sm = 0;
  FD_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, T, smem));
  const int64_t work = std::max<int64_t>((int64_t)np * np / 4, (int64_t)np * np / 2);
  int grid = (int)std::min<int64_t>(cdiv(work, T), (int64_t)per_sm * ctx->num_sms);
  grid = std::max(1, std::min(grid, 4096));
  JacobiArgs a;
  a.A0 = A0; a.A1 = A1; a.Q = Qw; a.part = part; a.n = n; a.np = np;
  a.max_sweeps = max_sweeps; a.rel_tol = 1e-14; a.sweeps_out = sweeps;
  void* args[] = {&a};
  FD_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_jacobi, grid, T, args, smem, ctx->stream));
  FD_LAUNCHED(ctx);
  k_eig_sort<<<1, 512, 0, ctx->stream>>>(A0, Qw, n, np, w, Q);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status resid_norms(fd_ctx* ctx, const double* V, const double* AV, int64_t ld, int64_t D, int n,
                      const double* theta, double* out) {
  const int nb = std::min<int64_t>(ctx->num_sms * 4, std::max<int64_t>(1, D));
  void* p;
  FD_TRY(workspace(ctx, "resid_partial", sizeof(double) * nb * n, &p));
  k_resid_partial<<<nb, 256, 0, ctx->stream>>>(V, AV, ld, D, n, theta, (double*)p);
  FD_LAUNCHED(ctx);
  k_resid_reduce<<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>((double*)p, nb, n, out);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

// The last Cholesky-QR pass factors the Gram matrix of a block the earlier
// passes have orthonormalised: its R is close to the identity.  A diagonal
// entry off by more than a factor 4 means they failed (a numerically rank
// deficient block beyond what the shifted passes recover): FD_ERR_BREAKDOWN
// instead of a block that is not orthonormal.  Synchronises.
fd_status check_last_factor(fd_ctx* ctx, const double* Rk, int ns) {
  std::vector<double> d(ns);
  FD_CUDA(ctx, cudaMemcpy2DAsync(d.data(), sizeof(double), Rk, sizeof(double) * (ns + 1), sizeof(double),
                                 ns, cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < ns; ++i)
    if (!(std::fabs(d[i]) > 0.25 && std::fabs(d[i]) < 4.0))
      return set_err(ctx, FD_ERR_BREAKDOWN,
                     "Cholesky-QR: the block is numerically rank deficient (last-pass R[%d][%d] = %g)", i, i, d[i]);
  return FD_OK;
}

fd_status orthonormalize(fd_ctx* ctx, double* V, int64_t D, int ns, int64_t ldv, double* R,
                         int* passes_out) {
  void* p;
  const size_t nn = (size_t)ns * ns;
  FD_TRY(workspace(ctx, "ortho", sizeof(double) * 4 * nn + 64, &p));
  double* G = (double*)p;
  double* Rk = G + nn;
  double* Ri = Rk + nn;
  double* Rt = Ri + nn;
  int* ok = (int*)(Rt + nn);
  const double coeff = 11.0 * ((double)D * ns + (double)ns * (ns + 1)) * 0x1.0p-53;
  if (R) {
    k_identity<<<(unsigned)cdiv(nn, 256), 256, 0, ctx->stream>>>(R, ns);
    FD_LAUNCHED(ctx);
  }
  bool any_shift = false;
  int passes = 0;
  while (passes < 2 || (any_shift && passes < 3)) {
    FD_TRY(gram(ctx, V, ldv, V, ldv, D, ns, ns, G, ns, true));
    FD_TRY(cholesky(ctx, G, ns, 0.0, Rk, ok));
    int hok = 0;
    FD_CUDA(ctx, cudaMemcpyAsync(&hok, ok, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!hok) {
      FD_TRY(cholesky(ctx, G, ns, coeff, Rk, ok));
      FD_CUDA(ctx, cudaMemcpyAsync(&hok, ok, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (!hok) return set_err(ctx, FD_ERR_BREAKDOWN, "shifted Cholesky-QR broke down (pass %d)", passes + 1);
      any_shift = true;
    }
    FD_TRY(tri_inverse(ctx, Rk, ns, Ri));
    FD_TRY(rotate(ctx, V, ldv, D, ns, Ri, true));
    if (R) {
      k_small_gemm<<<(unsigned)cdiv(nn, 256), 256, 0, ctx->stream>>>(Rk, R, Rt, ns);
      FD_LAUNCHED(ctx);
      FD_CUDA(ctx, cudaMemcpyAsync(R, Rt, sizeof(double) * nn, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    ++passes;
  }
  FD_TRY(check_last_factor(ctx, Rk, ns));
  if (passes_out) *passes_out = passes;
  return FD_OK;
}

static int bundle_width(int remaining) {
  const int w[] = {128, 64, 32, 16, 8, 4, 2};
  for (int x : w)
    if (x <= remaining) return x;
  return 0;
}

fd_status rayleigh_ritz_dev(fd_ctx* ctx, const fd_matrix* A, double* V, double* AV, int64_t D,
                            int ns, int64_t ld, double* theta_dev, double* resid_dev) {
  for (int j = 0; j < ns;) {
    int w = bundle_width(ns - j);
    FD_TRY(spmmv(ctx, A, FD_F64, V + j, ld, AV + j, ld, w, true));
    j += w;
  }
  void* p;
  const size_t nn = (size_t)ns * ns;
  FD_TRY(workspace(ctx, "rr", sizeof(double) * 2 * nn, &p));
  double* H = (double*)p;
  double* Q = H + nn;
  FD_TRY(gram(ctx, V, ld, AV, ld, D, ns, ns, H, ns, true));
  FD_TRY(sym_eig(ctx, H, ns, theta_dev, Q, 40));
  FD_TRY(rotate(ctx, V, ld, D, ns, Q, false));
  // A (V Q) by a second SpMMV instead of rotating AV: on GB300 the rotation is
  // FP64-ALU bound (D ns^2 FMAs) while the SpMMV costs nnz ns FMAs
  for (int j = 0; j < ns;) {
    int w = bundle_width(ns - j);
    FD_TRY(spmmv(ctx, A, FD_F64, V + j, ld, AV + j, ld, w, true));
    j += w;
  }
  FD_TRY(resid_norms(ctx, V, AV, ld, D, ns, theta_dev, resid_dev));
  return FD_OK;
}

fd_status copy_cols_f64_to_f32(fd_ctx* ctx, const double* src, int64_t lds, float* dst, int64_t ldd,
                               int64_t D, int n) {
  k_f64_to_f32<<<(unsigned)cdiv(D * n, 256), 256, 0, ctx->stream>>>(src, lds, dst, ldd, D, n);
  FD_LAUNCHED(ctx);
  return FD_OK;
}
fd_status copy_cols_f32_to_f64(fd_ctx* ctx, const float* src, int64_t lds, double* dst, int64_t ldd,
                               int64_t D, int n) {
  k_f32_to_f64<<<(unsigned)cdiv(D * n, 256), 256, 0, ctx->stream>>>(src, lds, dst, ldd, D, n);
  FD_LAUNCHED(ctx);
  return FD_OK;
}
fd_status copy_cols_f64_to_ff(fd_ctx* ctx, const double* src, int64_t lds, float* dst, int64_t ldd,
                              int64_t D, int n) {
  k_f64_to_ff<<<(unsigned)cdiv(D * n, 256), 256, 0, ctx->stream>>>(src, lds, dst, ldd, D, n);
  FD_LAUNCHED(ctx);
  return FD_OK;
}
fd_status copy_cols_ff_to_f64(fd_ctx* ctx, const float* src, int64_t lds, double* dst, int64_t ldd,
                              int64_t D, int n) {
  k_ff_to_f64<<<(unsigned)cdiv(D * n, 256), 256, 0, ctx->stream>>>(src, lds, dst, ldd, D, n);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

}  // namespace fdi

using namespace fdi;

extern "C" {

fd_status fd_orthonormalize(fd_ctx* ctx, double* V, int64_t D, int ns, int64_t ldv, double* R,
                            int* passes) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!V || D < 1 || ns < 1 || ns > 1024 || ldv < ns || ns > D)
    return set_err(ctx, FD_ERR_ARG, "need V, 1 <= ns <= min(1024, D), ldv >= ns");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  return orthonormalize(ctx, V, D, ns, ldv, R, passes);
}

fd_status fd_gram(fd_ctx* ctx, const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t D,
                   int m, int n, double* C, int ldc) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!X || !Y || !C || D < 1 || m < 1 || n < 1 || m > 4096 || n > 4096 || ldx < m || ldy < n || ldc < n)
    return set_err(ctx, FD_ERR_ARG, "need blocks, D >= 1, 1 <= m, n <= 4096, ld >= width");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  return gram(ctx, X, ldx, Y, ldy, D, m, n, C, ldc, X == Y && ldx == ldy && m == n);
}

fd_status fd_rotate(fd_ctx* ctx, double* V, int64_t ldv, int64_t D, int n, const double* M, int upper) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!V || !M || D < 1 || n < 1 || n > 1024 || ldv < n)
    return set_err(ctx, FD_ERR_ARG, "need blocks, D >= 1, 1 <= n <= 1024, ldv >= n");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  return rotate(ctx, V, ldv, D, n, M, upper != 0);
}

fd_status fd_set_gemm_mode(fd_ctx* ctx, fd_gemm_mode mode) {
  if (!ctx) return FD_ERR_ARG;
  if (mode != FD_GEMM_AUTO && mode != FD_GEMM_FP64 && mode != FD_GEMM_OZAKI)
    return set_err(ctx, FD_ERR_ARG, "unknown gemm mode %d", (int)mode);
  ctx->gemm_mode = (int)mode;
  return FD_OK;
}

fd_status fd_copy_block(fd_ctx* ctx, const void* src, fd_prec sp, int64_t lds, void* dst, fd_prec dp,
                        int64_t ldd, int64_t D, int n) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  auto known = [](fd_prec p) { return p == FD_F64 || p == FD_F32 || p == FD_FF; };
  if (!src || !dst || D < 0 || n < 0 || lds < n || ldd < n || !known(sp) || !known(dp) ||
      (sp == FD_F32 && dp == FD_FF) || (sp == FD_FF && dp == FD_F32))
    return set_err(ctx, FD_ERR_ARG, "need buffers, D, n >= 0, lds, ldd >= n and a supported type pair");
  if (D == 0 || n == 0) return FD_OK;
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  if (sp == FD_F64 && dp == FD_F32)
    return copy_cols_f64_to_f32(ctx, (const double*)src, lds, (float*)dst, ldd, D, n);
  if (sp == FD_F32 && dp == FD_F64)
    return copy_cols_f32_to_f64(ctx, (const float*)src, lds, (double*)dst, ldd, D, n);
  if (sp == FD_F64 && dp == FD_FF)
    return copy_cols_f64_to_ff(ctx, (const double*)src, lds, (float*)dst, ldd, D, n);
  if (sp == FD_FF && dp == FD_F64)
    return copy_cols_ff_to_f64(ctx, (const float*)src, lds, (double*)dst, ldd, D, n);
  const size_t es = sp == FD_F32 ? 4 : 8;
  FD_CUDA(ctx, cudaMemcpy2DAsync(dst, ldd * es, src, lds * es, n * es, D, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
  return FD_OK;
}

fd_status fd_rayleigh_ritz(fd_ctx* ctx, const fd_matrix* A, double* V, double* AV, int64_t D, int ns,
                           int64_t ld, double* theta, double* resid) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !V || !AV || !theta || !resid) return set_err(ctx, FD_ERR_ARG, "null argument");
  if (D != A->D || ns < 2 || ns % 2 || ns > 1024 || ns > D || ld < ns || ld % 2 ||
      ((uintptr_t)V & 15) || ((uintptr_t)AV & 15))
    return set_err(ctx, FD_ERR_ARG, "need D = matrix dimension, even 2 <= ns <= 1024, even ld >= ns, aligned blocks");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  void* p;
  FD_TRY(workspace(ctx, "rr_out", sizeof(double) * 2 * ns, &p));
  double* th = (double*)p;
  FD_TRY(rayleigh_ritz_dev(ctx, A, V, AV, D, ns, ld, th, th + ns));
  FD_CUDA(ctx, cudaMemcpyAsync(theta, th, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaMemcpyAsync(resid, th + ns, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return FD_OK;
}

}  // extern "C"
