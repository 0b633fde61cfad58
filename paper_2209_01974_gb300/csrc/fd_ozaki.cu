// FP64-accurate Gram and rotation products on bf16 tensor cores (Ozaki scheme).
//
// GB300 executes FP64 at about 1.2 TFLOP/s but bf16 mma.sync at about 600
// TFLOP/s.  The tall-skinny products of Cholesky-QR and Rayleigh-Ritz (Sec. 2)
// are therefore split into exact integer pieces (Ozaki, Ogita, Oishi, Rump,
// "Error-free transformations of matrix multiplication", Numer. Algorithms
// 2012; Mukunoki et al. 2020 on tensor cores):
//
//   a_ik = 2^{e_i} sum_{s<7} d^a_{s,ik} 2^{-8(s+1)},  |d| <= 255 (8-bit digits)
//   b_kj = 2^{f_j} sum_{t<7} d^b_{t,kj} 2^{-8(t+1)}
//   (AB)_ij = 2^{e_i + f_j} sum_{l<7} 2^{-8(l+2)} sum_{s+t=l} sum_k d^a_s d^b_t
//
// with e_i (f_j) the exponent of the largest |a_ik| over k (|b_kj| over k), so
// each operand is cut to 56 bits relative to its row (column) maximum, and the
// pairs s + t >= 7 (weight <= 2^-72) are dropped.  Every digit is an integer of
// magnitude below 2^8 and therefore exact in bf16; a level l sums at most 7
// pairs over a K chunk of 32, all partial sums stay below 7 * 32 * 255^2 <
// 2^24 and the FP32 accumulation of mma.sync.m16n8k16 is exact.  Each level's
// chunk sum is converted to an integer and added, scaled by 2^(8 (6 - l)), into
// two 64-bit integer accumulators (levels 0-2 and 3-6), which is exact for up
// to 2^14 chunks per CTA; one conversion to FP64 at the end.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fd_internal.cuh"

namespace fdi {
namespace {

constexpr int OZ_S = 7;            // digits per operand
constexpr int OZ_B = 8;            // bits per digit
constexpr int OZ_F = OZ_S * OZ_B;  // 56 fraction bits
constexpr int TB = 64;             // CTA tile (rows and columns)
constexpr int KC = 32;             // K chunk
constexpr int SK = KC + 8;         // padded K stride of a digit row (bf16 elements; 80 bytes)
constexpr int OZ_THREADS = 256;
constexpr size_t OZ_SMEM = sizeof(__nv_bfloat16) * 2 * OZ_S * TB * SK;  // 71,680 bytes
constexpr int64_t OZ_MAX_CHUNKS = 1 << 14;  // per CTA, keeps the 64-bit accumulators exact

// fixed-point magnitude y = |x| 2^(56 - e) (< 2^56 for |x| < 2^e) and sign of x
__device__ __forceinline__ unsigned long long fixed56(double x, int e, bool* neg) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (ex) m |= 1ull << 52;
  const int sh = (ex ? ex : 1) - 1075 - e + OZ_F;  // |x| 2^(F - e) = m 2^sh < 2^56
  *neg = (bits >> 63) != 0;
  if (m == 0 || sh <= -64) return 0;
  return sh >= 0 ? m << sh : m >> (-sh);
}

__device__ __forceinline__ uint32_t pack_bf16x2(int lo, int hi) {
  __nv_bfloat162 p = __floats2bfloat162_rn((float)lo, (float)hi);
  return *reinterpret_cast<uint32_t*>(&p);
}

__device__ __forceinline__ int digit(unsigned long long y, bool neg, int s) {
  const int v = (int)((y >> (OZ_F - OZ_B * (s + 1))) & 0xFF);
  return neg ? -v : v;
}

// store the 7 digit slices of 8 consecutive K values of one row (of A or B)
__device__ __forceinline__ void store_digits8(__nv_bfloat16* base_slice0, int row,
                                              const double (&x)[8], int e) {
  unsigned long long y[8];
  bool ng[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) y[q] = fixed56(x[q], e, &ng[q]);
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    uint4 v;
    v.x = pack_bf16x2(digit(y[0], ng[0], s), digit(y[1], ng[1], s));
    v.y = pack_bf16x2(digit(y[2], ng[2], s), digit(y[3], ng[3], s));
    v.z = pack_bf16x2(digit(y[4], ng[4], s), digit(y[5], ng[5], s));
    v.w = pack_bf16x2(digit(y[6], ng[6], s), digit(y[7], ng[7], s));
    *reinterpret_cast<uint4*>(base_slice0 + (size_t)s * TB * SK + (size_t)row * SK) = v;
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Exact accumulator of one output.  Level l carries the weight 2^(8 (6 - l))
// in units of 2^-64 (relative to 2^(e_i + f_j)); value = hi 2^32 + lo.
struct Acc {
  long long hi, lo;  // levels 0-2 (weights 2^16, 2^8, 1) and 3-6 (2^24 .. 1)
};

// Tensor-core part of one K chunk: digits of A (rows) in As[s][m][k], of B
// (columns) in Bs[t][n][k]; every level's exact sum goes into acc.
// Warp w covers rows (w & 3) * 16 .. +16 and columns (w >> 2) * 32 .. +32.
__device__ __forceinline__ void chunk_mma(const __nv_bfloat16* As, const __nv_bfloat16* Bs,
                                          Acc (&acc)[4][4]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = (w & 3) * 16, n0 = (w >> 2) * 32;
  // ldmatrix row addresses: A x4 -> (rows m0 + lane%16, k + 8*(lane/16)); B x2 -> (n + lane%8, k + 8*((lane/8)&1))
  const int ar = m0 + (lane & 15), ak = (lane >> 4) * 8;
  const int br = lane & 7, bk = ((lane >> 3) & 1) * 8;
#pragma unroll 1
  for (int l = 0; l < OZ_S; ++l) {
    float c[4][4] = {};
#pragma unroll 1
    for (int s = 0; s <= l; ++s) {
      const int t = l - s;
      const __nv_bfloat16* Asl = As + (size_t)s * TB * SK;
      const __nv_bfloat16* Bsl = Bs + (size_t)t * TB * SK;
#pragma unroll
      for (int kk = 0; kk < KC; kk += 16) {
        uint32_t a[4];
        ldsm_x4(a, Asl + (size_t)ar * SK + kk + ak);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          uint32_t b[2];
          ldsm_x2(b, Bsl + (size_t)(n0 + nt * 8 + br) * SK + kk + bk);
          mma_bf16(c[nt], a, b);
        }
      }
    }
    // level weight 2^(8 (6 - l)): levels 0-2 go to hi (scaled by 2^-32), 3-6 to lo
    const bool to_hi = l < 3;
    const int sh = to_hi ? 8 * (2 - l) : 8 * (6 - l);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long v = (long long)__float2int_rn(c[nt][q]) * (1ll << sh);
        if (to_hi) acc[nt][q].hi += v;
        else acc[nt][q].lo += v;
      }
  }
}

__device__ __forceinline__ double acc_value(const Acc& a) {
  // per chunk |hi| < 2^38 and |lo| < 2^48, so over 2^14 chunks hi stays exact
  // in FP64 and lo in int64; the sum is rounded once
  return fma((double)a.hi, 0x1.0p32, (double)a.lo);
}

// value of accumulator entry (nt, q) at its tile position, in units of 2^-64
template <typename F>
__device__ __forceinline__ void for_each_out(const Acc (&acc)[4][4], F&& f) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = (w & 3) * 16, n0 = (w >> 2) * 32;
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = m0 + g + (q >= 2 ? 8 : 0);
      const int j = n0 + nt * 8 + t4 * 2 + (q & 1);
      f(i, j, acc_value(acc[nt][q]));
    }
}

// ---------------------------------------------------------------------------
// scales: exponent e with max |x| < 2^e (frexp); flag non-finite input
// ---------------------------------------------------------------------------
__global__ void k_col_maxabs(const double* X, int64_t ld, int64_t D, int n, double* part, int* bad) {
  // grid (n_blocks_rows); each thread owns columns c = tid, tid + 256, ...
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double m = 0.0;
    for (int64_t r = blockIdx.x; r < D; r += gridDim.x) {
      const double v = fabs(X[r * ld + c]);
      if (!(v <= 1.0e300)) *bad = 1;  // NaN or inf
      m = fmax(m, v);
    }
    part[(int64_t)blockIdx.x * n + c] = m;
  }
}
__global__ void k_col_exp(const double* part, int nb, int n, int* ex) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double m = 0.0;
  for (int b = 0; b < nb; ++b) m = fmax(m, part[(int64_t)b * n + c]);
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  ex[c] = e;
}
__global__ void k_row_exp(const double* V, int64_t ld, int64_t D, int n, int* ex, int* bad) {
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= D) return;
  double m = 0.0;
  for (int c = lane; c < n; c += 32) {
    const double v = fabs(V[r * ld + c]);
    if (!(v <= 1.0e300)) *bad = 1;
    m = fmax(m, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    ex[r] = e;
  }
}

// ---------------------------------------------------------------------------
// Gram: P[slice][i][j] = sum over the slice's rows k of X[k][i] Y[k][j]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OZ_THREADS, 2)
    k_oz_gram(const double* __restrict__ X, int64_t ldx, const double* __restrict__ Y, int64_t ldy,
              int64_t D, int m, int n, int ntj, int sym, int64_t rows_per_slice, const int* ex,
              const int* ey, double* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* Bs = As + (size_t)OZ_S * TB * SK;
  int t = blockIdx.x, ti, tj;
  if (sym) {
    ti = 0;
    int rowlen = ntj;
    while (t >= rowlen) { t -= rowlen; ++ti; --rowlen; }
    tj = ti + t;
  } else {
    ti = t / ntj;
    tj = t % ntj;
  }
  const int i0 = ti * TB, j0 = tj * TB;
  const int64_t k0 = (int64_t)blockIdx.y * rows_per_slice;
  const int64_t k1 = min(D, k0 + rows_per_slice);
  Acc acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = Acc{0, 0};
  for (int64_t kb = k0; kb < k1; kb += KC) {
    // digits: work item = (operand, column c, 8 consecutive k); 2 x 64 x 4 items
    for (int item = threadIdx.x; item < 2 * TB * (KC / 8); item += OZ_THREADS) {
      const int op = item / (TB * (KC / 8)), rem = item % (TB * (KC / 8));
      const int c = rem % TB, kg = rem / TB;
      const int col = (op == 0 ? i0 : j0) + c;
      const int lim = op == 0 ? m : n;
      const double* src = op == 0 ? X : Y;
      const int64_t lds = op == 0 ? ldx : ldy;
      double x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t k = kb + kg * 8 + q;
        x[q] = (col < lim && k < k1) ? src[k * lds + col] : 0.0;
      }
      const int e = col < lim ? (op == 0 ? ex[col] : ey[col]) : 0;
      store_digits8((op == 0 ? As : Bs) + kg * 8, c, x, e);
    }
    __syncthreads();
    chunk_mma(As, Bs, acc);
    __syncthreads();
  }
  double* Ps = P + (int64_t)blockIdx.y * m * n;
  for_each_out(acc, [&](int i, int j, double v) {
    const int gi = i0 + i, gj = j0 + j;
    if (gi < m && gj < n) Ps[(int64_t)gi * n + gj] = ldexp(v, ex[gi] + ey[gj] - 64);
  });
}

__global__ void k_oz_gram_reduce(const double* P, int slices, int m, int n, int sym, double* C,
                                 int ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (sym && i / TB > j / TB) return;
  double s = 0.0;
  for (int q = 0; q < slices; ++q) s += P[(int64_t)q * m * n + e];
  C[(int64_t)i * ldc + j] = s;
  if (sym && i / TB < j / TB) C[(int64_t)j * ldc + i] = s;
}

// ---------------------------------------------------------------------------
// rotation: Out[r][j] = sum_k V[r][k] M[k][j]; the digits of M are computed
// once (k_m_digits) as Md[t][j][k] with column exponents em[j]
// ---------------------------------------------------------------------------
__global__ void k_m_digits(const double* M, int n, int npad, const int* em, __nv_bfloat16* Md) {
  // one thread per (j, 8 consecutive k)
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int groups = npad / 8;
  if (item >= (int64_t)npad * groups) return;
  const int j = (int)(item / groups), kg = (int)(item % groups);
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = kg * 8 + q;
    x[q] = (j < n && k < n) ? M[(int64_t)k * n + j] : 0.0;
  }
  const int e = j < n ? em[j] : 0;
  unsigned long long y[8];
  bool ng[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) y[q] = fixed56(x[q], e, &ng[q]);
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    uint4 v;
    v.x = pack_bf16x2(digit(y[0], ng[0], s), digit(y[1], ng[1], s));
    v.y = pack_bf16x2(digit(y[2], ng[2], s), digit(y[3], ng[3], s));
    v.z = pack_bf16x2(digit(y[4], ng[4], s), digit(y[5], ng[5], s));
    v.w = pack_bf16x2(digit(y[6], ng[6], s), digit(y[7], ng[7], s));
    *reinterpret_cast<uint4*>(Md + ((size_t)s * npad + j) * npad + kg * 8) = v;
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 2)
    k_oz_rotate(const double* __restrict__ V, int64_t ldv, int64_t D, int n, int npad, int upper,
                const int* er, const __nv_bfloat16* __restrict__ Md, const int* em,
                double* __restrict__ Out, int64_t ldo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* Bs = As + (size_t)OZ_S * TB * SK;
  const int64_t r0 = (int64_t)blockIdx.x * TB;
  const int j0 = blockIdx.y * TB;
  const int kend = upper ? min(npad, j0 + TB) : npad;  // M upper triangular: rows k <= j
  Acc acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = Acc{0, 0};
  for (int kb = 0; kb < kend; kb += KC) {
    for (int item = threadIdx.x; item < TB * (KC / 8); item += OZ_THREADS) {
      const int r = item % TB, kg = item / TB;
      const int64_t gr = r0 + r;
      double x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = kb + kg * 8 + q;
        x[q] = (gr < D && k < n) ? V[gr * ldv + k] : 0.0;
      }
      store_digits8(As + kg * 8, r, x, gr < D ? er[gr] : 0);
    }
    for (int item = threadIdx.x; item < OZ_S * TB * (KC / 8); item += OZ_THREADS) {
      const int s = item / (TB * (KC / 8)), rem = item % (TB * (KC / 8));
      const int c = rem / (KC / 8), kg = rem % (KC / 8);
      *reinterpret_cast<uint4*>(Bs + ((size_t)s * TB + c) * SK + kg * 8) =
          *reinterpret_cast<const uint4*>(Md + ((size_t)s * npad + j0 + c) * npad + kb + kg * 8);
    }
    __syncthreads();
    chunk_mma(As, Bs, acc);
    __syncthreads();
  }
  for_each_out(acc, [&](int i, int j, double v) {
    const int64_t gr = r0 + i;
    const int gj = j0 + j;
    if (gr < D && gj < n) Out[gr * ldo + gj] = ldexp(v, er[gr] + em[gj] - 64);
  });
}

bool attrs_set = false;

fd_status set_attrs(fd_ctx* ctx) {
  if (attrs_set) return FD_OK;
  FD_CUDA(ctx, cudaFuncSetAttribute(k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
  FD_CUDA(ctx, cudaFuncSetAttribute(k_oz_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
  attrs_set = true;
  return FD_OK;
}

}  // namespace

// Column exponents of X (n columns over D rows); returns false (no error) if X
// holds a non-finite value, in which case the caller uses the FP64 path.
static fd_status col_exponents(fd_ctx* ctx, const double* X, int64_t ld, int64_t D, int n, int* ex,
                               int* bad, bool* finite) {
  const int nb = (int)std::min<int64_t>(ctx->num_sms * 4, std::max<int64_t>(1, D));
  void* p;
  FD_TRY(workspace(ctx, "oz_colmax", sizeof(double) * (size_t)nb * n, &p));
  k_col_maxabs<<<nb, 256, 0, ctx->stream>>>(X, ld, D, n, (double*)p, bad);
  FD_LAUNCHED(ctx);
  k_col_exp<<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>((double*)p, nb, n, ex);
  FD_LAUNCHED(ctx);
  (void)finite;
  return FD_OK;
}

fd_status oz_gram(fd_ctx* ctx, const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t D,
                  int m, int n, double* C, int ldc, bool sym, bool* used) {
  *used = false;
  FD_TRY(set_attrs(ctx));
  void* p;
  FD_TRY(workspace(ctx, "oz_exp", sizeof(int) * ((size_t)m + n + 8), &p));
  int* ex = (int*)p;
  int* ey = ex + m;
  int* bad = ey + n;
  FD_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
  bool fin = true;
  FD_TRY(col_exponents(ctx, X, ldx, D, m, ex, bad, &fin));
  if (Y != X || ldy != ldx) FD_TRY(col_exponents(ctx, Y, ldy, D, n, ey, bad, &fin));
  else FD_CUDA(ctx, cudaMemcpyAsync(ey, ex, sizeof(int) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  int hbad = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hbad) return FD_OK;  // non-finite input: the FP64 path propagates it
  const int nti = (int)cdiv(m, TB), ntj = (int)cdiv(n, TB);
  const int tiles = sym ? nti * (nti + 1) / 2 : nti * ntj;
  int64_t slices = std::max<int64_t>(1, cdiv(4LL * ctx->num_sms, tiles));
  slices = std::min<int64_t>(slices, std::max<int64_t>(1, cdiv(D, 4 * KC)));
  slices = std::max<int64_t>(slices, cdiv(D, OZ_MAX_CHUNKS * KC));  // exact 64-bit accumulation
  const int64_t rps = cdiv(cdiv(D, slices), KC) * KC;
  slices = std::max<int64_t>(1, cdiv(D, rps));
  FD_TRY(workspace(ctx, "oz_gram_partial", sizeof(double) * slices * m * n, &p));
  double* P = (double*)p;
  k_oz_gram<<<dim3(tiles, (unsigned)slices), OZ_THREADS, OZ_SMEM, ctx->stream>>>(
      X, ldx, Y, ldy, D, m, n, ntj, sym ? 1 : 0, rps, ex, ey, P);
  FD_LAUNCHED(ctx);
  k_oz_gram_reduce<<<(unsigned)cdiv((int64_t)m * n, 256), 256, 0, ctx->stream>>>(P, (int)slices, m, n,
                                                                                sym ? 1 : 0, C, ldc);
  FD_LAUNCHED(ctx);
  *used = true;
  return FD_OK;
}

fd_status oz_rotate(fd_ctx* ctx, double* V, int64_t ldv, int64_t D, int n, const double* M, bool upper,
                    bool* used) {
  *used = false;
  FD_TRY(set_attrs(ctx));
  const int npad = (int)cdiv(n, TB) * TB;
  void* p;
  FD_TRY(workspace(ctx, "oz_rot_small", sizeof(int) * ((size_t)n + D + 8) +
                                            sizeof(__nv_bfloat16) * (size_t)OZ_S * npad * npad + 256, &p));
  __nv_bfloat16* Md = (__nv_bfloat16*)p;
  int* em = (int*)(Md + (size_t)OZ_S * npad * npad);
  int* er = em + n;
  int* bad = er + D;
  FD_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
  bool fin = true;
  FD_TRY(col_exponents(ctx, M, n, n, n, em, bad, &fin));
  k_row_exp<<<(unsigned)cdiv(D, 8), 256, 0, ctx->stream>>>(V, ldv, D, n, er, bad);
  FD_LAUNCHED(ctx);
  int hbad = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hbad) return FD_OK;
  const int groups = npad / 8;
  k_m_digits<<<(unsigned)cdiv((int64_t)npad * groups, 256), 256, 0, ctx->stream>>>(M, n, npad, em, Md);
  FD_LAUNCHED(ctx);
  FD_TRY(workspace(ctx, "oz_rot_out", sizeof(double) * (size_t)D * n, &p));
  double* Out = (double*)p;
  k_oz_rotate<<<dim3((unsigned)cdiv(D, TB), (unsigned)(npad / TB)), OZ_THREADS, OZ_SMEM, ctx->stream>>>(
      V, ldv, D, n, npad, upper ? 1 : 0, er, Md, em, Out, n);
  FD_LAUNCHED(ctx);
  FD_CUDA(ctx, cudaMemcpy2DAsync(V, ldv * sizeof(double), Out, n * sizeof(double), n * sizeof(double), D,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
  *used = true;
  return FD_OK;
}

}  // namespace fdi
