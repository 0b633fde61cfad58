// FP64-accurate Gram and rotation products on the tcgen05 tensor cores
// (Ozaki scheme).
//
// GB300 executes FP64 at about 1.2 TFLOP/s but dense bf16 tcgen05.mma at about
// 2 PFLOP/s.  The tall-skinny products of Cholesky-QR and Rayleigh-Ritz
// (Sec. 2) are therefore split into exact integer pieces (Ozaki, Ogita, Oishi,
// Rump, "Error-free transformations of matrix multiplication", Numer.
// Algorithms 2012; Mukunoki et al. 2020 on tensor cores):
//
//   a_ik = 2^{e_i} sum_{s<8} d^a_{s,ik} 2^{-7(s+1)},  |d| <= 127 (7-bit digits)
//   b_kj = 2^{f_j} sum_{t<8} d^b_{t,kj} 2^{-7(t+1)}
//   (AB)_ij = 2^{e_i + f_j} sum_{l<8} 2^{-7(l+2)} sum_{s+t=l} sum_k d^a_s d^b_t
//
// with e_i (f_j) the exponent of the largest |a_ik| over k (|b_kj| over k), so
// each operand is cut to 56 bits relative to its row (column) maximum, and the
// pairs s + t >= 8 (weight <= 2^-63 relative) are dropped.  Every digit is an
// integer of magnitude below 2^7, exact in bf16.  A level l sums at most 8
// digit pairs; over a K chunk of 128 every partial sum stays below
// 8 * 128 * 127^2 < 2^24, so the FP32 accumulation of the tensor core is exact.
//
// Kernel shape (one CTA per SM, 512 threads): a 128 x 64 output tile; the 8
// level accumulators live in TMEM (8 x 64 FP32 columns = all 512 columns).
// The K range runs in sub-chunks of 32: all threads cut the FP64 inputs of a
// sub-chunk into digit slices in shared memory (two buffers, the canonical
// no-swizzle K-major layout of 8-row x 16-byte core matrices), one thread
// issues the 36 pairs x 2 tcgen05.mma (M 128, N 64, K 16) of the sub-chunk and
// commits them to the buffer's mbarrier, and the next sub-chunk's digits are
// cut while the tensor core works.  Every fourth sub-chunk (K = 128) the
// levels are read back with tcgen05.ld, converted to integers and added,
// scaled by 2^(7 (7 - l)), into two 64-bit integer accumulators per output
// (levels 0-3 and 4-7; value = hi 2^28 + lo), exact for up to 2^16 chunks per
// CTA; one conversion to FP64 at the end.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fd_internal.cuh"

namespace fdi {
namespace {

constexpr int OZ_S = 8;             // digits per operand
constexpr int OZ_B = 7;             // bits per digit
constexpr int OZ_F = OZ_S * OZ_B;   // 56 fraction bits
constexpr int TM = 128;             // output tile rows (tcgen05 M)
constexpr int TN = 64;              // output tile columns (tcgen05 N)
constexpr int KS = 32;              // K sub-chunk (digits cut per step)
constexpr int SUBS = 4;             // sub-chunks per exact FP32 chunk (K = 128)
constexpr int OZ_THREADS = 512;
constexpr int A_SLICE = TM * KS * 2;                  // 8192 bytes per digit slice
constexpr int B_SLICE = TN * KS * 2;                  // 4096 bytes
constexpr int BUF = OZ_S * (A_SLICE + B_SLICE);       // 98,304 bytes per buffer
constexpr int CM_K = 128;                             // K-adjacent core matrices (LBO)
constexpr int CM_MN = (KS / 8) * 128;                 // MN-adjacent 8-row groups (SBO) = 512
constexpr size_t OZ_SMEM = 2 * (size_t)BUF + 64;      // + 2 mbarriers and the TMEM address
constexpr int64_t OZ_MAX_CHUNKS = 1 << 16;            // per CTA, keeps the accumulators exact
constexpr unsigned TMEM_COLS = 512;                   // 8 levels x 64 columns

// instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B bf16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4
// at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((CM_K >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((CM_MN >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)));
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// bounded wait for the completion of the barrier phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 4000000000ll) return false;  // about 2 s at 2 GHz
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// fixed-point magnitude y = |x| 2^(56 - e) (< 2^56 for |x| < 2^e) and sign of x
__device__ __forceinline__ unsigned long long fixed56(double x, int e, uint32_t* sign) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (ex) m |= 1ull << 52;
  const int sh = (ex ? ex : 1) - 1075 - e + OZ_F;  // |x| 2^(F - e) = m 2^sh < 2^56
  *sign = (uint32_t)(bits >> 63);
  if (m == 0 || sh <= -64) return 0;
  return sh >= 0 ? m << sh : m >> (-sh);
}

// bf16 bit pattern of the digit v in [0, 127]: the float v is built exactly by
// the 2^23 bias trick and its upper half is the bf16 value (8 significant bits)
__device__ __forceinline__ uint32_t bf16_of_digit(uint32_t v) {
  return __float_as_uint(__uint_as_float(0x4B000000u | v) - 8388608.0f) >> 16;
}

// the 8 digit slices of 8 consecutive K values (k group kg) of one operand
// row, stored as one 16-byte core-matrix row per slice
__device__ __forceinline__ void store_digits8(unsigned char* slice0, int slice_bytes, int row, int kg,
                                              const double (&x)[8], int e) {
  unsigned long long y[8];
  uint32_t sg[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) y[q] = fixed56(x[q], e, &sg[q]);
  uint32_t smask[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) smask[p] = (sg[2 * p] << 15) | (sg[2 * p + 1] << 31);
  const int off = (row >> 3) * CM_MN + kg * CM_K + (row & 7) * 16;
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    const int sh = OZ_F - OZ_B * (s + 1);
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t lo = bf16_of_digit((uint32_t)(y[2 * p] >> sh) & 0x7Fu);
      const uint32_t hi = bf16_of_digit((uint32_t)(y[2 * p + 1] >> sh) & 0x7Fu);
      w[p] = (lo | (hi << 16)) | smask[p];
    }
    *reinterpret_cast<uint4*>(slice0 + (size_t)s * slice_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Exact accumulator of one output: value = hi 2^28 + lo in units of
// 2^-63 2^(e_i + f_j); level l carries the weight 2^(7 (7 - l)).
struct Acc {
  long long hi, lo;
};

// One sub-chunk's tensor-core work (issued by one thread): level l collects
// the pairs (s, l - s) in its TMEM columns l * 64 ..; the first MMA of a level
// in a K chunk overwrites, the rest accumulate.
__device__ __forceinline__ void issue_subchunk(uint32_t tmem, uint32_t a0, uint32_t b0, bool first) {
#pragma unroll 1
  for (int l = 0; l < OZ_S; ++l) {
#pragma unroll 1
    for (int s = 0; s <= l; ++s) {
      const uint32_t a = a0 + (uint32_t)(s * A_SLICE), b = b0 + (uint32_t)((l - s) * B_SLICE);
#pragma unroll
      for (int ks = 0; ks < KS / 16; ++ks)
        umma(tmem + (uint32_t)(l * TN), sdesc(a + ks * 2 * CM_K), sdesc(b + ks * 2 * CM_K),
             (first && s == 0 && ks == 0) ? 0u : 1u);
    }
  }
}

// Read the 8 levels of this thread's 16 outputs (TMEM lane = tile row
// 32 (warp & 3) + lane, columns 16 (warp >> 2) ..) into the accumulators.
__device__ __forceinline__ void flush(uint32_t tmem, Acc (&acc)[16]) {
  const int w = threadIdx.x >> 5;
  const uint32_t base = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(16 * (w >> 2));
#pragma unroll 1
  for (int l = 0; l < OZ_S; ++l) {
    uint32_t r[16];
    tmem_ld16(base + (uint32_t)(l * TN), r);
    const long long wgt = 1ll << (l < 4 ? 7 * (3 - l) : 7 * (7 - l));
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const long long v = __float2ll_rz(__uint_as_float(r[c])) * wgt;
      if (l < 4) acc[c].hi += v;
      else acc[c].lo += v;
    }
  }
}

// The pipeline shared by the Gram and rotation kernels.  `cut(sc, buf)` writes
// the digits of sub-chunk sc into buffer buf (all threads).  Returns false if
// a bounded wait gave up (the same answer in every thread).
template <typename Cut>
__device__ __forceinline__ bool run_tile(unsigned char* smem, uint64_t* bar, uint32_t tmem, int nsub,
                                         Acc (&acc)[16], Cut&& cut) {
  bool ok = true;
  for (int sc = 0; sc < nsub; ++sc) {
    const int b = sc & 1;
    // buffer b is free once the MMAs of sub-chunk sc - 2 have completed
    if (sc >= 2) ok = mbar_wait(&bar[b], (uint32_t)((sc - 2) >> 1) & 1u);
    if (__syncthreads_or(!ok)) return false;
    cut(sc, smem + (size_t)b * BUF);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(smem + (size_t)b * BUF);
      issue_subchunk(tmem, a0, a0 + OZ_S * A_SLICE, (sc % SUBS) == 0);
      umma_commit(&bar[b]);
    }
    if ((sc % SUBS) == SUBS - 1 || sc == nsub - 1) {
      ok = mbar_wait(&bar[b], (uint32_t)(sc >> 1) & 1u);
      if (__syncthreads_or(!ok)) return false;
      tc_fence_after();
      flush(tmem, acc);
      tc_fence_before();
      __syncthreads();
    }
  }
  return true;
}

__device__ __forceinline__ double acc_value(const Acc& a) {
  return fma((double)a.hi, 0x1.0p28, (double)a.lo);
}

// CTA prologue: TMEM (warp 0) and the two mbarriers
__device__ __forceinline__ uint32_t tile_setup(unsigned char* smem, uint64_t** bar) {
  *bar = reinterpret_cast<uint64_t*>(smem + 2 * (size_t)BUF);
  uint32_t* holder = reinterpret_cast<uint32_t*>(smem + 2 * (size_t)BUF + 16);
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(holder)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 32) {
    mbar_init(&(*bar)[0]);
    mbar_init(&(*bar)[1]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *holder;
}

__device__ __forceinline__ void tile_teardown(uint32_t tmem) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// Stage the tile's 16 outputs per thread through shared memory (the digit
// buffers are free once the last flush is done) and hand every output to
// `put(i, j, v)` with consecutive threads on consecutive columns.
template <typename Put>
__device__ __forceinline__ void write_tile(unsigned char* smem, const Acc (&acc)[16], Put&& put) {
  double* st = reinterpret_cast<double*>(smem);  // [TM][TN + 1]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (w & 3) + lane, col0 = 16 * (w >> 2);
#pragma unroll
  for (int c = 0; c < 16; ++c) st[row * (TN + 1) + col0 + c] = acc_value(acc[c]);
  __syncthreads();
  for (int e = threadIdx.x; e < TM * TN; e += OZ_THREADS) {
    const int i = e / TN, j = e % TN;
    put(i, j, st[i * (TN + 1) + j]);
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
// Gram: P[slice][i][j] = sum over the slice's rows k of X[k][i] Y[k][j];
// tile (ti, tj) covers i in [128 ti, +128), j in [64 tj, +64); for a symmetric
// product only the tiles that reach the upper triangle (tj >= 2 ti) run
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gram(const double* __restrict__ X, int64_t ldx, const double* __restrict__ Y, int64_t ldy,
              int64_t D, int m, int n, int ntj, int sym, int64_t rows_per_slice, const int* ex,
              const int* ey, double* __restrict__ P, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  int t = blockIdx.x, ti = 0, tj;
  if (sym) {
    for (;;) {
      const int cnt = ntj - 2 * ti;
      if (t < cnt) break;
      t -= cnt;
      ++ti;
    }
    tj = 2 * ti + t;
  } else {
    ti = t / ntj;
    tj = t % ntj;
  }
  const int i0 = ti * TM, j0 = tj * TN;
  const int64_t k0 = (int64_t)blockIdx.y * rows_per_slice;
  const int64_t k1 = min(D, k0 + rows_per_slice);
  uint64_t* bar;
  const uint32_t tmem = tile_setup(smem, &bar);
  Acc acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = Acc{0, 0};
  const int nsub = (int)((k1 - k0 + KS - 1) / KS);
  // digit work items: A (X columns i0 ..) 128 x 4, then B (Y columns j0 ..) 64 x 4
  auto cut = [&](int sc, unsigned char* buf) {
    const int64_t kb = k0 + (int64_t)sc * KS;
    for (int item = threadIdx.x; item < (TM + TN) * (KS / 8); item += OZ_THREADS) {
      const bool isA = item < TM * (KS / 8);
      const int it = isA ? item : item - TM * (KS / 8);
      const int rows = isA ? TM : TN;
      const int c = it % rows, kg = it / rows;
      const int col = (isA ? i0 : j0) + c;
      const int lim = isA ? m : n;
      const double* src = isA ? X : Y;
      const int64_t lds = isA ? ldx : ldy;
      double x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t k = kb + kg * 8 + q;
        x[q] = (col < lim && k < k1) ? src[k * lds + col] : 0.0;
      }
      const int e = col < lim ? (isA ? ex[col] : ey[col]) : 0;
      store_digits8(buf + (isA ? 0 : OZ_S * A_SLICE), isA ? A_SLICE : B_SLICE, c, kg, x, e);
    }
  };
  const bool ok = run_tile(smem, bar, tmem, nsub, acc, cut);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    double* Ps = P + (int64_t)blockIdx.y * m * n;
    write_tile(smem, acc, [&](int i, int j, double v) {
      const int gi = i0 + i, gj = j0 + j;
      if (gi < m && gj < n) Ps[(int64_t)gi * n + gj] = ldexp(v, ex[gi] + ey[gj] - 63);
    });
  }
  tile_teardown(tmem);
}

__global__ void k_oz_gram_reduce(const double* P, int slices, int m, int n, int sym, double* C,
                                 int ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (sym && i > j) return;
  double s = 0.0;
  for (int q = 0; q < slices; ++q) s += P[(int64_t)q * m * n + e];
  C[(int64_t)i * ldc + j] = s;
  if (sym && i < j) C[(int64_t)j * ldc + i] = s;
}

// ---------------------------------------------------------------------------
// rotation: Out[r][j] = sum_k V[r][k] M[k][j]; the digits of M are computed
// once (k_m_digits) as Md[t][j][k] (npad x npad per slice) with column
// exponents em[j]
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
  uint32_t sg[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) y[q] = fixed56(x[q], e, &sg[q]);
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    const int sh = OZ_F - OZ_B * (s + 1);
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t lo = bf16_of_digit((uint32_t)(y[2 * p] >> sh) & 0x7Fu) | (sg[2 * p] << 15);
      const uint32_t hi = bf16_of_digit((uint32_t)(y[2 * p + 1] >> sh) & 0x7Fu) | (sg[2 * p + 1] << 15);
      w[p] = lo | (hi << 16);
    }
    *reinterpret_cast<uint4*>(Md + ((size_t)s * npad + j) * npad + kg * 8) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_rotate(const double* __restrict__ V, int64_t ldv, int64_t D, int n, int npad, int upper,
                const int* er, const __nv_bfloat16* __restrict__ Md, const int* em,
                double* __restrict__ Out, int64_t ldo, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int64_t r0 = (int64_t)blockIdx.x * TM;
  const int j0 = blockIdx.y * TN;
  const int kend = upper ? min(npad, j0 + TN) : npad;  // M upper triangular: rows k <= j
  uint64_t* bar;
  const uint32_t tmem = tile_setup(smem, &bar);
  Acc acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = Acc{0, 0};
  const int nsub = (kend + KS - 1) / KS;
  auto cut = [&](int sc, unsigned char* buf) {
    const int kb = sc * KS;
    {  // A: rows of V, one (row, 8 consecutive k) item per thread
      const int r = threadIdx.x % TM, kg = threadIdx.x / TM;
      const int64_t gr = r0 + r;
      double x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = kb + kg * 8 + q;
        x[q] = (gr < D && k < n) ? V[gr * ldv + k] : 0.0;
      }
      store_digits8(buf, A_SLICE, r, kg, x, gr < D ? er[gr] : 0);
    }
    // B: the precomputed digits of M, 16 bytes per (slice, column, k group)
    unsigned char* bb = buf + OZ_S * A_SLICE;
    for (int item = threadIdx.x; item < OZ_S * TN * (KS / 8); item += OZ_THREADS) {
      const int s = item / (TN * (KS / 8)), rem = item % (TN * (KS / 8));
      const int c = rem / (KS / 8), kg = rem % (KS / 8);
      *reinterpret_cast<uint4*>(bb + (size_t)s * B_SLICE + (c >> 3) * CM_MN + kg * CM_K + (c & 7) * 16) =
          *reinterpret_cast<const uint4*>(Md + ((size_t)s * npad + j0 + c) * npad + kb + kg * 8);
    }
  };
  const bool ok = run_tile(smem, bar, tmem, nsub, acc, cut);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    write_tile(smem, acc, [&](int i, int j, double v) {
      const int64_t gr = r0 + i;
      const int gj = j0 + j;
      if (gr < D && gj < n) Out[gr * ldo + gj] = ldexp(v, er[gr] + em[gj] - 63);
    });
  }
  tile_teardown(tmem);
}

bool attrs_set = false;

fd_status set_attrs(fd_ctx* ctx) {
  if (attrs_set) return FD_OK;
  FD_CUDA(ctx, cudaFuncSetAttribute(k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
  FD_CUDA(ctx, cudaFuncSetAttribute(k_oz_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
  attrs_set = true;
  return FD_OK;
}

// device error word of the bounded waits: cleared before a launch, read after
fd_status check_wait_flag(fd_ctx* ctx, const int* flag) {
  int h = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h) return set_err(ctx, FD_ERR_TIMEOUT, "tensor-core product: a bounded mbarrier wait gave up");
  return FD_OK;
}

}  // namespace

// Column exponents of X (n columns over D rows); non-finite values raise *bad.
static fd_status col_exponents(fd_ctx* ctx, const double* X, int64_t ld, int64_t D, int n, int* ex,
                               int* bad) {
  const int nb = (int)std::min<int64_t>(ctx->num_sms * 4, std::max<int64_t>(1, D));
  void* p;
  FD_TRY(workspace(ctx, "oz_colmax", sizeof(double) * (size_t)nb * n, &p));
  k_col_maxabs<<<nb, 256, 0, ctx->stream>>>(X, ld, D, n, (double*)p, bad);
  FD_LAUNCHED(ctx);
  k_col_exp<<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>((double*)p, nb, n, ex);
  FD_LAUNCHED(ctx);
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
  int* err = bad + 1;
  FD_CUDA(ctx, cudaMemsetAsync(bad, 0, 2 * sizeof(int), ctx->stream));
  FD_TRY(col_exponents(ctx, X, ldx, D, m, ex, bad));
  if (Y != X || ldy != ldx) FD_TRY(col_exponents(ctx, Y, ldy, D, n, ey, bad));
  else FD_CUDA(ctx, cudaMemcpyAsync(ey, ex, sizeof(int) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  int hbad = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hbad) return FD_OK;  // non-finite input: the FP64 path propagates it
  const int nti = (int)cdiv(m, TM), ntj = (int)cdiv(n, TN);
  int tiles = 0;
  if (sym) {
    for (int ti = 0; ti < nti; ++ti) tiles += std::max(0, ntj - 2 * ti);
  } else {
    tiles = nti * ntj;
  }
  // about four waves of one CTA per SM, K slices in whole 128-row chunks
  int64_t slices = std::max<int64_t>(1, (4LL * ctx->num_sms) / tiles);
  slices = std::min<int64_t>(slices, std::max<int64_t>(1, cdiv(D, 4 * SUBS * KS)));
  slices = std::max<int64_t>(slices, cdiv(D, OZ_MAX_CHUNKS * SUBS * KS));
  const int64_t rps = cdiv(cdiv(D, slices), SUBS * KS) * (SUBS * KS);
  slices = std::max<int64_t>(1, cdiv(D, rps));
  FD_TRY(workspace(ctx, "oz_gram_partial", sizeof(double) * slices * m * n, &p));
  double* P = (double*)p;
  k_oz_gram<<<dim3(tiles, (unsigned)slices), OZ_THREADS, OZ_SMEM, ctx->stream>>>(
      X, ldx, Y, ldy, D, m, n, ntj, sym ? 1 : 0, rps, ex, ey, P, err);
  FD_LAUNCHED(ctx);
  FD_TRY(check_wait_flag(ctx, err));
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
  const int npad = (int)cdiv(n, TN) * TN;
  void* p;
  FD_TRY(workspace(ctx, "oz_rot_small", sizeof(int) * ((size_t)n + D + 8) +
                                            sizeof(__nv_bfloat16) * (size_t)OZ_S * npad * npad + 256, &p));
  __nv_bfloat16* Md = (__nv_bfloat16*)p;
  int* em = (int*)(Md + (size_t)OZ_S * npad * npad);
  int* er = em + n;
  int* bad = er + D;
  int* err = bad + 1;
  FD_CUDA(ctx, cudaMemsetAsync(bad, 0, 2 * sizeof(int), ctx->stream));
  FD_TRY(col_exponents(ctx, M, n, n, n, em, bad));
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
  k_oz_rotate<<<dim3((unsigned)cdiv(D, TM), (unsigned)(npad / TN)), OZ_THREADS, OZ_SMEM, ctx->stream>>>(
      V, ldv, D, n, npad, upper ? 1 : 0, er, Md, em, Out, n, err);
  FD_LAUNCHED(ctx);
  FD_TRY(check_wait_flag(ctx, err));
  FD_CUDA(ctx, cudaMemcpy2DAsync(V, ldv * sizeof(double), Out, n * sizeof(double), n * sizeof(double), D,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
  *used = true;
  return FD_OK;
}

}  // namespace fdi
