// Fused Chebyshev step: SELL-C-sigma SpMMV on a row-major nb-wide block,
// fused with the three-term recurrence and the accumulation of the filter
// coefficients (Alg. 2 fuses the SpMV with the vector update; Sec. 3.2,
// Eq. EstimateT: with the fused kernel W1 is read once and W2, V are read and
// written, kappa = 5).
//
// Work mapping: a group of G lanes owns one SELL row; each lane holds CPL
// 16-byte vectors of the row (G * CPL * 16 bytes = nb * sizeof(T)), so every
// gathered row of W1 is one fully coalesced access.  A warp holds 32/G
// consecutive rows of one SELL chunk, so the warp's matrix loads at entry j
// touch adjacent words of the chunk's column-major slab.  Entry 0 of every
// SELL row is its diagonal, so the row's own W1 vector (needed for the beta
// term) is the first gathered vector.  W2 and V are touched once per step and
// use evict-first (.cs) loads and stores, keeping L2 for the W1 gathers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "fd_internal.cuh"
#include "fd_step.cuh"
#include "fd_ff.cuh"

namespace fdi {
namespace {

using namespace step;
using ffa::ff;

template <typename T, int NB, int MODE>
__global__ void __launch_bounds__(step_warps<T>() * 32, step_min_blocks<T>())
    k_cheb_step(SellArgs<T> A, StepArgs<T> s, unsigned pf) {
  using L = Layout<T, NB>;
  constexpr int WARPS = step_warps<T>();
  // L2 prefetch for the CTA that starts one resident wave (pf CTAs) later:
  // its first loads (row-wise operands, then the SELL slab they index) are a
  // chain of dependent DRAM round trips that no register budget can overlap.
  if (pf > 0 && blockIdx.x + pf < gridDim.x) {
    const int64_t r0 = (int64_t)(blockIdx.x + pf) * (WARPS * L::RPW);
    prefetch_rows<T, NB, MODE>(A, s, r0, r0 + WARPS * L::RPW < A.D ? r0 + WARPS * L::RPW : A.D);
  }
  const int64_t warp = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int64_t row0 = warp * L::RPW;
  if (row0 >= A.D) return;
  cheb_rows<T, NB, MODE>(A, s, row0);
}

template <typename T, int NB, int MODE>
__global__ void __launch_bounds__(WARPS * 32, MIN_BLOCKS_F64)  // 64 registers: no spills
    k_kron_step(KronArgs<T> K, StepArgs<T> s) {
  using L = Layout<T, NB>;
  const int64_t warp = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int64_t row0 = warp * L::RPW;
  if (row0 >= K.D) return;
  kron_rows<T, NB, MODE>(K, s, row0);
}

// debug checks: flag any index outside [0, bound) (a grid-stride scan)
__global__ void k_scan_indices(const int32_t* idx, int64_t n, int64_t bound, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (idx[i] < 0 || idx[i] >= bound) atomicExch(bad, 1);
}
__global__ void k_scan_packed(const uint32_t* ent, int64_t n, uint32_t mask, int64_t bound, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if ((int64_t)(ent[i] & mask) >= bound) atomicExch(bad, 1);
}

// dst[i] = src[perm[i]] (to SELL order) or dst[perm[i]] = src[i] (back)
template <typename T>
__global__ void k_permute_rows(const T* src, int64_t lds, T* dst, int64_t ldd,
                               const int64_t* perm, int64_t D, int nb, int to_sell) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t i = t / nb;
  int j = (int)(t % nb);
  if (i >= D) return;
  int64_t p = perm[i];
  if (to_sell) dst[i * ldd + j] = src[p * lds + j];
  else dst[p * ldd + j] = src[i * lds + j];
}

// ---- dispatch -------------------------------------------------------------
template <typename T, int NB>
fd_status launch_kron_step(fd_ctx* ctx, const fd_matrix* M, int mode, const StepArgs<T>& s) {
  using L = Layout<T, NB>;
  KronArgs<T> K;
  K.D = M->D;
  K.dim_dn = M->kdim[1];
  K.bits_up = M->kbits[0];
  K.bits_dn = M->kbits[1];
  K.ptr_up = M->kptr[0];
  K.col_up = M->kcol[0];
  K.ptr_dn = M->kptr[1];
  K.col_dn = M->kcol[1];
  if constexpr (std::is_same_v<T, double>) {
    K.val_up = M->kval[0];
    K.val_dn = M->kval[1];
    K.diag = M->kdiag;
  } else if constexpr (std::is_same_v<T, float>) {
    K.val_up = M->kval32[0];
    K.val_dn = M->kval32[1];
    K.diag = M->kdiag32;
  } else {
    K.val_up = reinterpret_cast<const ff*>(M->kvalff[0]);
    K.val_dn = reinterpret_cast<const ff*>(M->kvalff[1]);
    K.diag = reinterpret_cast<const ff*>(M->kdiagff);
  }
  const unsigned grid = (unsigned)cdiv(M->D, (int64_t)WARPS * L::RPW);
  if (mode == MODE_SPMMV) k_kron_step<T, NB, MODE_SPMMV><<<grid, WARPS * 32, 0, ctx->stream>>>(K, s);
  else if (mode == MODE_SECOND) k_kron_step<T, NB, MODE_SECOND><<<grid, WARPS * 32, 0, ctx->stream>>>(K, s);
  else k_kron_step<T, NB, MODE_GENERIC><<<grid, WARPS * 32, 0, ctx->stream>>>(K, s);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

template <typename T, int NB>
fd_status launch_step(fd_ctx* ctx, const fd_matrix* M, int mode, const StepArgs<T>& s) {
  if (M->kron) return launch_kron_step<T, NB>(ctx, M, mode, s);
  using L = Layout<T, NB>;
  SellArgs<T> A;
  A.chunk_ptr = M->chunk_ptr; A.row_len = M->row_len; A.col = M->col; A.D = M->D; A.C = M->C;
  if constexpr (std::is_same_v<T, double>) A.val = M->val;
  else if constexpr (std::is_same_v<T, float>) A.val = M->val32;
  else A.val = reinterpret_cast<const ff*>(M->valff);
  constexpr int SW = step_warps<T>();
  const int64_t rows_per_block = (int64_t)SW * L::RPW;
  const unsigned grid = (unsigned)cdiv(M->D, rows_per_block);
  // prefetch distance: one wave of resident CTAs (the launch-bounds occupancy)
  const unsigned pf = (unsigned)ctx->num_sms * step_min_blocks<T>();
  if (mode == MODE_SPMMV) k_cheb_step<T, NB, MODE_SPMMV><<<grid, SW * 32, 0, ctx->stream>>>(A, s, pf);
  else if (mode == MODE_SECOND) k_cheb_step<T, NB, MODE_SECOND><<<grid, SW * 32, 0, ctx->stream>>>(A, s, pf);
  else k_cheb_step<T, NB, MODE_GENERIC><<<grid, SW * 32, 0, ctx->stream>>>(A, s, pf);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

template <typename T>
fd_status step_dispatch(fd_ctx* ctx, const fd_matrix* M, int nb, int mode, const StepArgs<T>& s) {
  switch (nb) {
    case 2: if constexpr (sizeof(T) == 8) return launch_step<T, 2>(ctx, M, mode, s); break;
    case 4: return launch_step<T, 4>(ctx, M, mode, s);
    case 8: return launch_step<T, 8>(ctx, M, mode, s);
    case 16: return launch_step<T, 16>(ctx, M, mode, s);
    case 32: return launch_step<T, 32>(ctx, M, mode, s);
    case 64: return launch_step<T, 64>(ctx, M, mode, s);
    case 128: return launch_step<T, 128>(ctx, M, mode, s);
    default: break;
  }
  return set_err(ctx, FD_ERR_ARG, "unsupported nb %d", nb);
}

bool nb_ok(fd_prec prec, int nb) {
  if (prec == FD_F64 || prec == FD_FF) return nb == 2 || nb == 4 || nb == 8 || nb == 16 || nb == 32 || nb == 64 || nb == 128;
  return nb == 4 || nb == 8 || nb == 16 || nb == 32 || nb == 64 || nb == 128;
}

template <typename T>
fd_status permute(fd_ctx* ctx, const fd_matrix* M, const T* src, int64_t lds, T* dst,
                  int64_t ldd, int nb, bool to_sell) {
  int64_t n = M->D * nb;
  k_permute_rows<T><<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>(src, lds, dst, ldd, M->perm,
                                                                     M->D, nb, to_sell ? 1 : 0);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

template <typename T>
fd_status filter_t(fd_ctx* ctx, const fd_matrix* M, T* V, int64_t ldv, int nb, int n,
                   const double* mu, double alpha, double beta, T* W1, T* W2, int64_t ldw,
                   double* bytes_out) {
  const double Sx = sizeof(T), Sv = sizeof(T);
  const double mat_bytes = (double)M->nnz * (Sv + 4.0);
  const double vec = (double)nb * M->D * Sx;
  double bytes = 0;
  const bool ident = M->identity != 0;
  StepArgs<T> s{};
  // x0 location
  T* x0 = V;
  int64_t ld0 = ldv;
  if (!ident) {
    FD_TRY(permute<T>(ctx, M, V, ldv, W1, ldw, nb, true));
    x0 = W1;
    ld0 = ldw;
  }
  // step 1: x1 = A~ x0
  T* x1 = ident ? W1 : W2;
  s.X = x0; s.ldx = ld0; s.Y = x1; s.ldy = ldw;
  s.c_ax = (T)alpha; s.c_x = (T)beta;
  FD_TRY(step_dispatch<T>(ctx, M, nb, MODE_SPMMV, s));
  bytes += mat_bytes + 2 * vec;
  // step 2: x2 = 2 A~ x1 - x0; acc = mu0 x0 + mu1 x1 + mu2 x2
  T* acc = V;          // accumulator storage (SELL order when not identity)
  int64_t lda = ldv;
  T* x2 = ident ? W2 : W1;  // when not identity x2 overwrites x0 in W1 (same row)
  s = StepArgs<T>{};
  s.X = x1; s.ldx = ldw; s.Z = x0; s.ldz = ld0;
  s.c_ax = (T)(2 * alpha); s.c_x = (T)(2 * beta);
  s.mu0 = (T)mu[0]; s.mu1 = (T)mu[1]; s.mu2 = (T)mu[2];
  if (n > 2) {
    s.Y = x2; s.ldy = ldw;
    s.Vout = acc; s.ldvo = lda;
  } else {
    s.Y = nullptr;
    if (ident) { s.Vout = V; s.ldvo = ldv; }
    else { s.Vout = W1; s.ldvo = ldw; }   // final result in SELL order, unpermuted below
  }
  FD_TRY(step_dispatch<T>(ctx, M, nb, MODE_SECOND, s));
  bytes += mat_bytes + (n > 2 ? 4 : 3) * vec;
  // generic steps: xk = 2 A~ x_{k-1} - x_{k-2}; acc += mu_k xk
  T* xp = x1;  // x_{k-1}
  T* xpp = x2; // x_{k-2} buffer after step 2 is the other one
  // after step 2: x_{k-1} = x2, x_{k-2} = x1
  xp = x2; xpp = x1;
  T* final_buf = nullptr;
  for (int k = 3; k <= n; ++k) {
    s = StepArgs<T>{};
    s.X = xp; s.ldx = ldw; s.Z = xpp; s.ldz = ldw;
    s.c_ax = (T)(2 * alpha); s.c_x = (T)(2 * beta);
    s.mu2 = (T)mu[k];
    s.Vin = acc; s.ldvi = lda;
    const bool last = k == n;
    if (!last) {
      s.Y = xpp; s.ldy = ldw;
      s.Vout = acc; s.ldvo = lda;
      bytes += mat_bytes + 5 * vec;
    } else {
      s.Y = nullptr;
      if (ident) { s.Vout = acc; s.ldvo = lda; }
      else { s.Vout = xpp; s.ldvo = ldw; final_buf = xpp; }
      bytes += mat_bytes + 4 * vec;
    }
    FD_TRY(step_dispatch<T>(ctx, M, nb, MODE_GENERIC, s));
    T* t = xp; xp = xpp; xpp = t;
  }
  if (!ident) {
    if (n == 2) final_buf = W1;
    FD_TRY(permute<T>(ctx, M, final_buf, ldw, V, ldv, nb, false));
  }
  if (bytes_out) *bytes_out += bytes;
  return FD_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// ---- nb = 1 SpMV (Lanczos), lane per row over the SELL chunk ---------------
__global__ void k_spmv1(const int64_t* chunk_ptr, const int32_t* row_len, const int32_t* col,
                        const double* val, int64_t D, int C, const double* x, double* y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D) return;
  int64_t base = chunk_ptr[i / C] + i % C;
  int len = row_len[i];
  double s = 0.0;
  for (int j = 0; j < len; ++j) s = fma(val[base + (int64_t)j * C], x[col[base + (int64_t)j * C]], s);
  y[i] = s;
}

// ---- KPM: Chebyshev iteration on R random vectors with moment partial sums
constexpr int KPM_BLOCKS_PER_SM = 8;

__global__ void k_kpm_init(double* r, int64_t D, int R, const int64_t* perm, uint64_t key) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * R) return;
  int64_t i = t / R;
  int j = (int)(t % R);
  r[t] = fdrng::irwin_hall(key, (uint64_t)(perm[i] * R + j));
}

// one step: x_new = c_ax * A x + c_x * x [- z]; partial[blk] = (sum x_new . x, sum x_new . x_new,
// sum x . x); grid-stride over rows so the number of partials is fixed
template <int NB, bool FIRST>
__global__ void __launch_bounds__(WARPS * 32, 4)
    k_kpm_step(SellArgs<double> A, const double* X, const double* Z, double* Y, double c_ax,
               double c_x, double* partial) {
  using L = Layout<double, NB>;
  constexpr int E = L::E;
  const int lane = threadIdx.x & 31;
  const int g = lane / L::G, gl = lane % L::G;
  double sxy = 0, syy = 0, sxx = 0;
  const int64_t nwarps_total = (int64_t)gridDim.x * WARPS;
  for (int64_t warp = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5); warp * L::RPW < A.D;
       warp += nwarps_total) {
    const int64_t row = warp * L::RPW + g;
    const bool active = row < A.D;
    const int len = active ? A.row_len[row] : 0;
    const int wlen = __reduce_max_sync(0xffffffffu, len);
    V16<double> acc[L::CPL], xi[L::CPL];
    row_product<double, NB>(A, X, NB, row, active, len, wlen, gl, acc, xi);
    if (active) {
#pragma unroll
      for (int v = 0; v < L::CPL; ++v) {
        const int64_t off = row * NB + gl * E + v * L::G * E;
        V16<double> y;
        if (FIRST) {
#pragma unroll
          for (int e = 0; e < E; ++e) y.v[e] = c_ax * acc[v].v[e] + c_x * xi[v].v[e];
        } else {
          V16<double> z;
          z.ldcs(Z + off);
#pragma unroll
          for (int e = 0; e < E; ++e) y.v[e] = c_ax * acc[v].v[e] + c_x * xi[v].v[e] - z.v[e];
        }
        y.st(Y + off);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          sxy = fma(y.v[e], xi[v].v[e], sxy);
          syy = fma(y.v[e], y.v[e], syy);
          sxx = fma(xi[v].v[e], xi[v].v[e], sxx);
        }
      }
    }
  }
  // block reduction (fixed order)
  __shared__ double sh[3][WARPS * 32];
  sh[0][threadIdx.x] = sxy; sh[1][threadIdx.x] = syy; sh[2][threadIdx.x] = sxx;
  __syncthreads();
  for (int o = WARPS * 16; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) partial[(int64_t)blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

// sum the per-block partials of every step in a fixed order
__global__ void k_kpm_reduce(const double* partial, int nblocks, int nsteps, double* out) {
  int s = blockIdx.x;
  if (s >= nsteps) return;
  __shared__ double sh[3][256];
  double a = 0, b = 0, c = 0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
    const double* p = partial + ((int64_t)s * nblocks + k) * 3;
    a += p[0]; b += p[1]; c += p[2];
  }
  sh[0][threadIdx.x] = a; sh[1][threadIdx.x] = b; sh[2][threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[s * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

template <int NB>
fd_status kpm_t(fd_ctx* ctx, const fd_matrix* M, int n_moments, uint64_t seed, double alpha,
                double beta, double* mu_host) {
  cudaStream_t st = ctx->stream;
  const int64_t D = M->D;
  const int nsteps = n_moments <= 1 ? 1 : n_moments / 2;  // steps s = 1..nsteps give a_s, b_s
  const int nblocks = ctx->num_sms * KPM_BLOCKS_PER_SM;
  void* p;
  FD_TRY(workspace(ctx, "kpm_vec", sizeof(double) * 3 * D * NB, &p));
  double* buf[3] = {(double*)p, (double*)p + D * NB, (double*)p + 2 * D * NB};
  FD_TRY(workspace(ctx, "kpm_partial", sizeof(double) * 3 * (size_t)nblocks * nsteps, &p));
  double* partial = (double*)p;
  FD_TRY(workspace(ctx, "kpm_sums", sizeof(double) * 3 * nsteps, &p));
  double* sums = (double*)p;
  SellArgs<double> A;
  A.chunk_ptr = M->chunk_ptr; A.row_len = M->row_len; A.col = M->col; A.val = M->val;
  A.D = D; A.C = M->C;
  k_kpm_init<<<(unsigned)cdiv(D * NB, 256), 256, 0, st>>>(buf[0], D, NB, M->perm,
                                                           fdrng::key(seed, fdrng::STREAM_KPM));
  FD_LAUNCHED(ctx);
  // step 1: x1 = A~ x0
  k_kpm_step<NB, true><<<nblocks, WARPS * 32, 0, st>>>(A, buf[0], nullptr, buf[1], alpha, beta, partial);
  FD_LAUNCHED(ctx);
  int ip = 0, ic = 1, in = 2;  // x_{k-1}, x_k, x_{k+1}
  for (int s = 2; s <= nsteps; ++s) {
    k_kpm_step<NB, false><<<nblocks, WARPS * 32, 0, st>>>(A, buf[ic], buf[ip], buf[in], 2 * alpha,
                                                          2 * beta, partial + (int64_t)(s - 1) * nblocks * 3);
    FD_LAUNCHED(ctx);
    int t = ip; ip = ic; ic = in; in = t;
  }
  k_kpm_reduce<<<nsteps, 256, 0, st>>>(partial, nblocks, nsteps, sums);
  FD_LAUNCHED(ctx);
  std::vector<double> h(3 * nsteps);
  FD_CUDA(ctx, cudaMemcpyAsync(h.data(), sums, sizeof(double) * 3 * nsteps, cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  // a_s = <x_s, x_{s-1}>, b_s = <x_s, x_s>; mu_0 = <x0, x0>, mu_1 = a_1,
  // mu_2k = 2 b_k - mu_0, mu_2k+1 = 2 a_{k+1} - mu_1 (T_m T_n = (T_{m+n} + T_{|m-n|})/2)
  const double norm = 1.0 / ((double)NB * (double)D);
  double mu0 = h[2], mu1 = h[0];
  for (int m = 0; m < n_moments; ++m) {
    double v;
    if (m == 0) v = mu0;
    else if (m == 1) v = mu1;
    else if (m % 2 == 0) v = 2 * h[3 * (m / 2 - 1) + 1] - mu0;
    else v = 2 * h[3 * ((m + 1) / 2 - 1) + 0] - mu1;
    mu_host[m] = v * norm;
  }
  return FD_OK;
}

}  // namespace

fd_status debug_check_matrix(fd_ctx* ctx, const fd_matrix* M) {
  if (!ctx->debug_checks) return FD_OK;
  void* p;
  FD_TRY(workspace(ctx, "debug_flag", sizeof(int), &p));
  int* bad = (int*)p;
  FD_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
  const unsigned grid = (unsigned)std::max(1, ctx->num_sms * 4);
  k_scan_indices<<<grid, 256, 0, ctx->stream>>>(M->col, M->nnz_sell, M->D, bad);
  FD_LAUNCHED(ctx);
  if (M->kron) {
    for (int sp = 0; sp < 2; ++sp) {
      int64_t nh = 0;
      FD_CUDA(ctx, cudaMemcpyAsync(&nh, M->kptr[sp] + M->kdim[sp], sizeof(int64_t), cudaMemcpyDeviceToHost,
                                   ctx->stream));
      FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      k_scan_indices<<<grid, 256, 0, ctx->stream>>>(M->kcol[sp], nh, M->kdim[sp], bad);
      FD_LAUNCHED(ctx);
      if (sp == 1 && M->kdn_ent) {
        k_scan_packed<<<grid, 256, 0, ctx->stream>>>(M->kdn_ent, nh, 0x7fffffffu, M->kdim[1], bad);
        FD_LAUNCHED(ctx);
      }
    }
  }
  int h = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h) return set_err(ctx, FD_ERR_BOUNDS, "debug check: the matrix holds an index outside [0, %lld)",
                        (long long)M->D);
  return FD_OK;
}

fd_status filter(fd_ctx* ctx, const fd_matrix* M, fd_prec prec, void* V, int64_t ldv, int nb,
                 int degree, const double* mu, double alpha, double beta, void* W1, void* W2,
                 int64_t ldw, double* bytes_out) {
  // matrix-free Hubbard operator in FP32: column panels, slabs in RCM order
  // (the FP64 step is bound by GB300's FP64 rate; it keeps the row-major kernel)
  if (M->kron && prec == FD_F32)
    return kron_filter(ctx, M, prec, V, ldv, nb, degree, mu, alpha, beta, W1, W2, ldw, bytes_out);
  if (prec == FD_F64)
    return filter_t<double>(ctx, M, (double*)V, ldv, nb, degree, mu, alpha, beta, (double*)W1,
                            (double*)W2, ldw, bytes_out);
  if (prec == FD_FF)
    return filter_t<ff>(ctx, M, (ff*)V, ldv, nb, degree, mu, alpha, beta, (ff*)W1, (ff*)W2, ldw,
                        bytes_out);
  return filter_t<float>(ctx, M, (float*)V, ldv, nb, degree, mu, alpha, beta, (float*)W1,
                         (float*)W2, ldw, bytes_out);
}

fd_status spmmv(fd_ctx* ctx, const fd_matrix* M, fd_prec prec, const void* X, int64_t ldx,
                void* Y, int64_t ldy, int nb, bool original_order) {
  const size_t es = prec == FD_F32 ? 4 : 8;
  const bool wide = prec != FD_F32;  // double or float-float: 8-byte elements, permuted as such
  const bool ident = M->identity != 0 || !original_order;
  const void* xs = X;
  int64_t ldxs = ldx;
  void* ys = Y;
  int64_t ldys = ldy;
  if (!ident) {
    void* p;
    FD_TRY(workspace(ctx, "spmmv_perm", es * 2 * M->D * nb, &p));
    xs = p;
    ldxs = nb;
    ys = (char*)p + es * M->D * nb;
    ldys = nb;
    if (wide) FD_TRY(permute<double>(ctx, M, (const double*)X, ldx, (double*)xs, nb, nb, true));
    else FD_TRY(permute<float>(ctx, M, (const float*)X, ldx, (float*)xs, nb, nb, true));
  }
  if (prec == FD_F64) {
    StepArgs<double> s{};
    s.X = (const double*)xs; s.ldx = ldxs; s.Y = (double*)ys; s.ldy = ldys; s.c_ax = 1.0; s.c_x = 0.0;
    FD_TRY(step_dispatch<double>(ctx, M, nb, MODE_SPMMV, s));
  } else if (prec == FD_FF) {
    StepArgs<ff> s{};
    s.X = (const ff*)xs; s.ldx = ldxs; s.Y = (ff*)ys; s.ldy = ldys; s.c_ax = ff(1); s.c_x = ff(0);
    FD_TRY(step_dispatch<ff>(ctx, M, nb, MODE_SPMMV, s));
  } else {
    StepArgs<float> s{};
    s.X = (const float*)xs; s.ldx = ldxs; s.Y = (float*)ys; s.ldy = ldys; s.c_ax = 1.0f; s.c_x = 0.0f;
    FD_TRY(step_dispatch<float>(ctx, M, nb, MODE_SPMMV, s));
  }
  if (!ident) {
    if (wide) FD_TRY(permute<double>(ctx, M, (const double*)ys, nb, (double*)Y, ldy, nb, false));
    else FD_TRY(permute<float>(ctx, M, (const float*)ys, nb, (float*)Y, ldy, nb, false));
  }
  return FD_OK;
}

fd_status spmv1(fd_ctx* ctx, const fd_matrix* M, const double* x, double* y) {
  k_spmv1<<<(unsigned)cdiv(M->D, 256), 256, 0, ctx->stream>>>(M->chunk_ptr, M->row_len, M->col,
                                                              M->val, M->D, M->C, x, y);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

fd_status kpm(fd_ctx* ctx, const fd_matrix* M, int n_moments, int R, uint64_t seed, double alpha,
              double beta, double* mu_host) {
  switch (R) {
    case 2: return kpm_t<2>(ctx, M, n_moments, seed, alpha, beta, mu_host);
    case 4: return kpm_t<4>(ctx, M, n_moments, seed, alpha, beta, mu_host);
    case 8: return kpm_t<8>(ctx, M, n_moments, seed, alpha, beta, mu_host);
    case 16: return kpm_t<16>(ctx, M, n_moments, seed, alpha, beta, mu_host);
    case 32: return kpm_t<32>(ctx, M, n_moments, seed, alpha, beta, mu_host);
    case 64: return kpm_t<64>(ctx, M, n_moments, seed, alpha, beta, mu_host);
    default: break;
  }
  return set_err(ctx, FD_ERR_ARG, "n_random must be 2, 4, 8, 16, 32 or 64");
}

}  // namespace fdi

using namespace fdi;

extern "C" {

fd_status fd_filter(fd_ctx* ctx, const fd_matrix* A, fd_prec prec, void* V, int64_t ldv, int nb,
                    int degree, const double* mu, double alpha, double beta, void* W1, void* W2,
                    int64_t ldw) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !V || !mu || !W1 || !W2) return set_err(ctx, FD_ERR_ARG, "null argument");
  if (prec != FD_F64 && prec != FD_F32 && prec != FD_FF) return set_err(ctx, FD_ERR_ARG, "bad precision");
  if (!nb_ok(prec, nb)) return set_err(ctx, FD_ERR_ARG, "unsupported nb %d", nb);
  if (degree < 2) return set_err(ctx, FD_ERR_ARG, "degree must be >= 2 (Alg. 2)");
  const size_t es = prec == FD_F32 ? 4 : 8;
  if (ldv < nb || ldw < nb || (ldv * es) % 16 || (ldw * es) % 16 || !aligned16(V) ||
      !aligned16(W1) || !aligned16(W2))
    return set_err(ctx, FD_ERR_ARG, "ld must be >= nb with 16-byte aligned rows and pointers");
  if (V == W1 || V == W2 || W1 == W2) return set_err(ctx, FD_ERR_ARG, "V, W1, W2 must be distinct");
  for (int k = 0; k <= degree; ++k)
    if (!std::isfinite(mu[k])) return set_err(ctx, FD_ERR_ARG, "mu[%d] is not finite", k);
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_TRY(debug_check_matrix(ctx, A));
  return filter(ctx, A, prec, V, ldv, nb, degree, mu, alpha, beta, W1, W2, ldw, nullptr);
}

fd_status fd_spmmv(fd_ctx* ctx, const fd_matrix* A, fd_prec prec, const void* X, int64_t ldx,
                   void* Y, int64_t ldy, int nb) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !X || !Y) return set_err(ctx, FD_ERR_ARG, "null argument");
  if (prec != FD_F64 && prec != FD_F32 && prec != FD_FF) return set_err(ctx, FD_ERR_ARG, "bad precision");
  if (!nb_ok(prec, nb)) return set_err(ctx, FD_ERR_ARG, "unsupported nb %d", nb);
  const size_t es = prec == FD_F32 ? 4 : 8;
  if (ldx < nb || ldy < nb || (ldx * es) % 16 || (ldy * es) % 16 || !aligned16(X) || !aligned16(Y))
    return set_err(ctx, FD_ERR_ARG, "ld must be >= nb with 16-byte aligned rows and pointers");
  if (X == Y) return set_err(ctx, FD_ERR_ARG, "X and Y must not alias");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_TRY(debug_check_matrix(ctx, A));
  return spmmv(ctx, A, prec, X, ldx, Y, ldy, nb, true);
}

fd_status fd_set_debug_checks(fd_ctx* ctx, int on) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  ctx->debug_checks = on ? 1 : 0;
  return FD_OK;
}

fd_status fd_debug_set_sell_column(fd_ctx* ctx, fd_matrix* A, int64_t entry, int32_t col) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || entry < 0 || entry >= A->nnz_sell) return set_err(ctx, FD_ERR_ARG, "need a matrix and 0 <= entry < nnz_sell");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  FD_CUDA(ctx, cudaMemcpyAsync(A->col + entry, &col, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return FD_OK;
}

fd_status fd_kpm_moments(fd_ctx* ctx, const fd_matrix* A, int n_moments, int n_random,
                         uint64_t seed, double alpha, double beta, double* mu) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !mu || n_moments < 1 || n_moments > 100000)
    return set_err(ctx, FD_ERR_ARG, "need a matrix, 1 <= n_moments <= 100000 and an output");
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return set_err(ctx, FD_ERR_ARG, "alpha/beta not finite");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  return kpm(ctx, A, n_moments, n_random, seed, alpha, beta, mu);
}

}  // extern "C"
