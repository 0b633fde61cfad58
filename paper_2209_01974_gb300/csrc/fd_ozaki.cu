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
// Two kernels per product.  A streaming kernel cuts each FP64 operand once
// into its 8 bf16 digit slices and writes them to HBM already in the tensor
// core's shared-memory layout (canonical no-swizzle K-major core matrices,
// one contiguous 2 or 4 KB block per 16-deep K step, slice and 64- or
// 128-wide operand block).  The product kernel (one CTA per SM, 512 threads,
// a 128 x 64 output tile, the 8 level accumulators in TMEM: 8 x 64 FP32
// columns = all 512) is a pure Blackwell pipeline: one thread streams the
// digit blocks of each K step into a four-stage shared-memory ring with
// cp.async.bulk (mbarrier complete_tx), one thread issues the step's 36
// tcgen05.mma (one per digit pair; M 128, N 64, K 16) and commits them to the
// stage's "empty" mbarrier, and every eighth step (K = 128) all threads read
// the levels back with tcgen05.ld, convert them to 32-bit integers, combine
// adjacent levels exactly in 32 bits and add them, scaled by 2^(7 (7 - l)),
// into two 64-bit integer accumulators per output (levels 0-3 and 4-7; value
// = hi 2^28 + lo), exact for up to 2^16 chunks per CTA; one conversion to FP64
// at the end.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "fd_internal.cuh"

namespace fdi {
namespace {

constexpr int OZ_S = 8;             // digits per operand
constexpr int OZ_B = 7;             // bits per digit
constexpr int OZ_F = OZ_S * OZ_B;   // 56 fraction bits
constexpr int TM = 128;             // output tile rows (tcgen05 M)
constexpr int TN = 64;              // output tile columns (tcgen05 N)
constexpr int KS = 16;              // K step (one tcgen05.mma)
constexpr int SUBS = 8;             // K steps per exact FP32 chunk (K = 128)
constexpr int NST = 4;              // shared-memory ring stages
constexpr int OZ_THREADS = 512;
constexpr int A_SLICE = TM * KS * 2;                  // 4096 bytes per digit block
constexpr int B_SLICE = TN * KS * 2;                  // 2048 bytes
constexpr int A_ELEMS = A_SLICE / 2, B_ELEMS = B_SLICE / 2;
constexpr int STAGE = OZ_S * (A_SLICE + B_SLICE);     // 49,152 bytes
constexpr int CM_K = 128;                             // K-adjacent core matrices (LBO)
constexpr int CM_MN = (KS / 8) * 128;                 // MN-adjacent 8-row groups (SBO) = 256
constexpr size_t OZ_SMEM = (size_t)NST * STAGE + 2 * NST * 8 + 16;  // + barriers, TMEM address
constexpr int64_t OZ_MAX_CHUNKS = 1 << 16;            // per CTA, keeps the accumulators exact
constexpr unsigned TMEM_COLS = 512;                   // 8 levels x 64 columns
constexpr int P_THREAD = 0;                           // bulk-copy producer (warp 0, lanes 0-15)
constexpr int M_THREAD = 32;                          // MMA issuer (warp 1)

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
}

// bounded wait for the completion of the barrier phase with the given parity;
// gives up after `limit` SM clock cycles (default about 2 s at 2 GHz)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = 4000000000ll) {
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
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// bulk (TMA engine) copy of `bytes` contiguous bytes, completing on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
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

// the 8 digit slices of 8 consecutive K values of one operand row (or
// column): slice s of the 8 values is one 16-byte core-matrix row, handed to
// put(s, v)
template <typename Put>
__device__ __forceinline__ void cut8(const double (&x)[8], int e, Put&& put) {
  unsigned long long y[8];
  uint32_t sg[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) y[q] = fixed56(x[q], e, &sg[q]);
  uint32_t smask[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) smask[p] = (sg[2 * p] << 15) | (sg[2 * p + 1] << 31);
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
    put(s, make_uint4(w[0], w[1], w[2], w[3]));
  }
}

// byte offset of (row, k) inside one digit block: 8-row x 16-byte core
// matrices, K-adjacent ones 128 bytes apart, row groups 256 bytes apart
__device__ __forceinline__ int core_offset(int row, int k) {
  return (row >> 3) * CM_MN + (k >> 3) * CM_K + (row & 7) * 16 + (k & 7) * 2;
}

// Exact accumulator of one output: value = hi 2^28 + lo in units of
// 2^-63 2^(e_i + f_j); level l carries the weight 2^(7 (7 - l)).
struct Acc {
  long long hi, lo;
};

// One K step's tensor-core work (issued by one thread): level l collects the
// pairs (s, l - s) in its TMEM columns l * 64 ..; the first MMA of a level in
// a K chunk overwrites, the rest accumulate.  Fully unrolled: the descriptor
// of slice s is the base descriptor plus s * slice bytes / 16 in its address
// field, an immediate.
template <bool FIRST>
__device__ __forceinline__ void issue_step(uint32_t tmem, uint64_t adesc, uint64_t bdesc) {
#pragma unroll
  for (int l = 0; l < OZ_S; ++l)
#pragma unroll
    for (int s = 0; s <= l; ++s)
      umma(tmem + (uint32_t)(l * TN), adesc + (uint64_t)((s * A_SLICE) >> 4),
           bdesc + (uint64_t)(((l - s) * B_SLICE) >> 4), (FIRST && s == 0) ? 0u : 1u);
}

// Read the 8 levels of this thread's 16 outputs (TMEM lane = tile row
// 32 (warp & 3) + lane, columns 16 (warp >> 2) ..) into the accumulators.
// Level sums are integers below 2^24 (l + 1 pairs x 128 x 127^2), so two
// adjacent levels combine exactly in 32 bits (c_l 2^7 + c_{l+1} < 2^31) and
// only 32-bit conversions are needed (64-bit ones run on GB300's slow FP64
// units).
__device__ __forceinline__ void flush(uint32_t tmem, Acc (&acc)[16]) {
  const int w = threadIdx.x >> 5;
  const uint32_t base = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(16 * (w >> 2));
#pragma unroll 1
  for (int pr = 0; pr < OZ_S / 2; ++pr) {  // level pairs (0,1) (2,3) (4,5) (6,7)
    uint32_t r0[16], r1[16];
    tmem_ld16(base + (uint32_t)(2 * pr * TN), r0);
    tmem_ld16(base + (uint32_t)((2 * pr + 1) * TN), r1);
    const int sh = (pr & 1) ? 0 : 14;  // pairs (0,1), (4,5) carry 2^14 within hi / lo
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int v = __float2int_rz(__uint_as_float(r0[c])) * 128 + __float2int_rz(__uint_as_float(r1[c]));
      const long long t = (long long)v * (1LL << sh);
      if (pr < 2) acc[c].hi += t;
      else acc[c].lo += t;
    }
  }
}

// The product pipeline of one CTA.  K step sc reads digit block (sc, s) of A
// at A + sc a_kc + s a_s and of B likewise (bf16 elements).  Returns false if
// a bounded wait gave up (the same answer in every thread).
__device__ __forceinline__ bool run_tile(unsigned char* smem, uint64_t* full, uint64_t* empty, uint32_t tmem,
                                         const __nv_bfloat16* A, int64_t a_kc, int64_t a_s,
                                         const __nv_bfloat16* B, int64_t b_kc, int64_t b_s, int nsub,
                                         Acc (&acc)[16]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // producer warp: lane 0 posts the stage's byte count, lanes 0-15 issue one
  // bulk copy each (slice lane / 2 of A or B)
  auto load = [&](int sc) {
    const int st = sc % NST;
    unsigned char* dst = smem + (size_t)st * STAGE;
    if (lane == 0) mbar_expect_tx(&full[st], STAGE);
    __syncwarp();
    if (lane < 2 * OZ_S) {
      const int s = lane >> 1;
      if (lane & 1)
        bulk_g2s(dst + OZ_S * A_SLICE + s * B_SLICE, B + sc * b_kc + s * b_s, B_SLICE, &full[st]);
      else
        bulk_g2s(dst + s * A_SLICE, A + sc * a_kc + s * a_s, A_SLICE, &full[st]);
    }
  };
  bool ok = true;
  if (warp == P_THREAD / 32)
    for (int sc = 0; sc < nsub && sc < NST; ++sc) load(sc);
  for (int sc = 0; sc < nsub; ++sc) {
    const int st = sc % NST;
    const uint32_t par = (uint32_t)(sc / NST) & 1u;
    if (threadIdx.x == M_THREAD && ok) {
      ok = mbar_wait(&full[st], par);
      if (ok) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(smem + (size_t)st * STAGE);
        const uint64_t ad = sdesc(a0), bd = sdesc(a0 + OZ_S * A_SLICE);
        if ((sc % SUBS) == 0) issue_step<true>(tmem, ad, bd);
        else issue_step<false>(tmem, ad, bd);
        umma_commit(&empty[st]);
      }
    }
    if (warp == P_THREAD / 32 && ok && sc + NST < nsub) {
      // the stage is free again once the MMAs of K step sc have completed
      ok = mbar_wait(&empty[st], par);
      if (ok) load(sc + NST);
    }
    if ((sc % SUBS) == SUBS - 1 || sc == nsub - 1) {
      // the issuer observes the completion; the others sleep in the barrier
      if (threadIdx.x == M_THREAD && ok) ok = mbar_wait(&empty[st], par);
      if (__syncthreads_or(!ok)) return false;
      tc_fence_after();
      flush(tmem, acc);
      tc_fence_before();
      __syncthreads();
    }
  }
  return true;
}

// hi 2^28 + lo scaled by 2^sc, rounded once to nearest (ties to even) by
// integer arithmetic: int64 -> FP64 conversions and FP64 arithmetic run on
// GB300's slow FP64 units
__device__ __forceinline__ double acc_value(const Acc& a, int sc) {
  // 128-bit two's complement N = hi 2^28 + lo as (H, L)
  unsigned long long L = (unsigned long long)a.hi << 28;
  long long H = a.hi >> 36;
  const unsigned long long lo = (unsigned long long)a.lo;
  const unsigned long long L2 = L + lo;
  H += (a.lo >> 63) + (L2 < L ? 1 : 0);  // sign extension of lo, carry
  L = L2;
  const bool neg = H < 0;
  unsigned long long mh = (unsigned long long)H, ml = L;
  if (neg) {  // magnitude
    ml = ~ml + 1;
    mh = ~mh + (ml == 0 ? 1 : 0);
  }
  if (mh == 0 && ml == 0) return 0.0;
  const int p = mh ? 127 - __clzll((long long)mh) : 63 - __clzll((long long)ml);  // leading bit
  unsigned long long m;  // 53-bit significand
  if (p <= 52) {
    m = ml << (52 - p);
  } else {
    const int sh = p - 52;  // 1 .. 75
    unsigned long long q, rem_hi, rem_lo;  // q = N >> sh; remainder bits below
    if (sh < 64) {
      q = (ml >> sh) | (mh << (64 - sh));
      rem_hi = (ml >> (sh - 1)) & 1u;
      rem_lo = sh > 1 ? (ml & ((1ull << (sh - 1)) - 1)) : 0;
    } else {
      q = mh >> (sh - 64);
      rem_hi = sh == 64 ? (ml >> 63) : ((mh >> (sh - 65)) & 1u);
      rem_lo = sh == 64 ? (ml & ~(1ull << 63)) : ((mh & ((1ull << (sh - 65)) - 1)) | ml);
    }
    m = q;
    if (rem_hi && (rem_lo || (m & 1u))) ++m;
  }
  int e = p + sc;  // value = m 2^(e - 52)
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  if (e < -1022 || e > 1023) return ldexp(neg ? -(double)m : (double)m, e - 52);
  const unsigned long long bits = ((unsigned long long)(neg ? 1 : 0) << 63) |
                                  ((unsigned long long)(e + 1023) << 52) | (m & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// CTA prologue: TMEM (warp 0) and the full / empty mbarriers of the ring
__device__ __forceinline__ uint32_t tile_setup(unsigned char* smem, uint64_t** full, uint64_t** empty) {
  unsigned char* tail = smem + (size_t)NST * STAGE;
  *full = reinterpret_cast<uint64_t*>(tail);
  *empty = *full + NST;
  uint32_t* holder = reinterpret_cast<uint32_t*>(tail + 2 * NST * 8);
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(holder)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&(*full)[i]);
      mbar_init(&(*empty)[i]);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
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

// Hand every output of the tile to put(i, j, v): the thread owning it
// converts (scale(i, j) gives the power of two), then the values are staged
// through shared memory (free once the last flush is done) so that the
// stores run with consecutive threads on consecutive columns.
template <typename Scale, typename Put>
__device__ __forceinline__ void write_tile(unsigned char* smem, const Acc (&acc)[16], Scale&& scale,
                                           Put&& put) {
  double* st = reinterpret_cast<double*>(smem);  // [TM][TN + 1]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (w & 3) + lane, col0 = 16 * (w >> 2);
#pragma unroll
  for (int c = 0; c < 16; ++c) st[row * (TN + 1) + col0 + c] = acc_value(acc[c], scale(row, col0 + c));
  __syncthreads();
  for (int e = threadIdx.x; e < TM * TN; e += OZ_THREADS) {
    const int i = e / TN, j = e % TN;
    put(i, j, st[i * (TN + 1) + j]);
  }
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// ---------------------------------------------------------------------------
// scales: exponent e with max |x| < 2^e (frexp); flag non-finite input
// ---------------------------------------------------------------------------
__global__ void k_col_maxabs(const double* X, int64_t ld, int64_t D, int n, double* part, int* bad) {
  // grid (n_blocks_rows); each thread owns columns c = tid, tid + 256, ...
  // maxima of |x| as 64-bit integers (the bit patterns of non-negative doubles
  // order like their values, NaN above inf): integer instructions instead of
  // GB300's slow FP64 ones
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    unsigned long long m[4] = {0, 0, 0, 0};  // four independent loads in flight
    const int64_t g = gridDim.x;
    int64_t r = blockIdx.x;
    for (; r + 3 * g < D; r += 4 * g) {
#pragma unroll
      for (int u = 0; u < 4; ++u) m[u] = max(m[u], abs_bits(X[(r + u * g) * ld + c]));
    }
    for (; r < D; r += g) m[0] = max(m[0], abs_bits(X[r * ld + c]));
    const unsigned long long mm = max(max(m[0], m[1]), max(m[2], m[3]));
    if (mm >= 0x7FF0000000000000ull) *bad = 1;  // NaN or inf
    part[(int64_t)blockIdx.x * n + c] = __longlong_as_double((long long)mm);
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

// ---------------------------------------------------------------------------
// digit blocks in HBM
//   column-scaled operand (Gram X or Y, rotation M), w columns over K rows:
//     block (kc, s, cb) of 64 columns x 16 k at ((kc * 8 + s) * ncb + cb) * 1024,
//     so a 128-column A tile is two adjacent blocks (4 KB)
//   row-scaled operand (rotation V), D rows over K = n columns:
//     block (rb, kc, s) of 128 rows x 16 k at ((rb * nkc + kc) * 8 + s) * 2048
// ---------------------------------------------------------------------------
__global__ void k_digits_cols(const double* __restrict__ X, int64_t ld, int64_t D, int w, int wpad,
                              const int* ex, int64_t nkc, __nv_bfloat16* __restrict__ Xd) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= nkc * 2 * wpad) return;
  const int c = (int)(item % wpad);
  const int64_t g = item / wpad;  // group of 8 consecutive k
  const int64_t k0 = 8 * g, kc = g >> 1;
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = (c < w && k0 + q < D) ? X[(k0 + q) * ld + c] : 0.0;
  const int ncb = wpad / 64;
  unsigned char* blk = reinterpret_cast<unsigned char*>(Xd + (kc * 8 * ncb + (c >> 6)) * B_ELEMS);
  const int off = core_offset(c & 63, (int)(k0 & 15));
  cut8(x, c < w ? ex[c] : 0, [&](int s, uint4 v) {
    *reinterpret_cast<uint4*>(blk + (size_t)s * ncb * B_SLICE + off) = v;
  });
}

// one warp per row: the row's exponent (max |v| over the row, written to
// er[r]; a non-finite value raises *bad), then its digit blocks
__global__ void k_digits_rows(const double* __restrict__ V, int64_t ldv, int64_t D, int n, int64_t Dpad,
                              int npad, int vec, int* er, int* bad, __nv_bfloat16* __restrict__ Vd) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= Dpad) return;
  const bool live = r < D;
  const double* row = V + r * ldv;
  unsigned long long mb = 0;  // max |v| as integer bits (see k_col_maxabs)
  if (live)
    for (int c = lane; c < n; c += 32) mb = max(mb, abs_bits(row[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if (mb >= 0x7FF0000000000000ull) {  // NaN or inf
    if (lane == 0) *bad = 1;
    mb = 0;
  }
  int e = 0;
  const double m = __longlong_as_double((long long)mb);
  if (m > 0.0) frexp(m, &e);
  if (live && lane == 0) er[r] = e;
  const int64_t nkc = npad / KS;
  for (int g = lane; g < npad / 8; g += 32) {  // groups of 8 consecutive k (L1-resident row)
    const int k0 = 8 * g;
    double x[8];
    if (vec && live && k0 + 8 <= n) {  // 16-byte aligned rows: four 16-byte loads
      const double2* p = reinterpret_cast<const double2*>(row + k0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 t = __ldg(p + q);
        x[2 * q] = t.x;
        x[2 * q + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = (live && k0 + q < n) ? row[k0 + q] : 0.0;
    }
    unsigned char* blk = reinterpret_cast<unsigned char*>(Vd + ((r >> 7) * nkc + (k0 >> 4)) * 8 * A_ELEMS);
    const int off = core_offset((int)(r & 127), k0 & 15);
    cut8(x, e, [&](int s, uint4 v) { *reinterpret_cast<uint4*>(blk + (size_t)s * A_SLICE + off) = v; });
  }
}

// ---------------------------------------------------------------------------
// Gram: P[slice][i][j] = sum over the slice's K steps of X[k][i] Y[k][j];
// tile (ti, tj) covers i in [128 ti, +128), j in [64 tj, +64); for a symmetric
// product only the tiles that reach the upper triangle (tj >= 2 ti) run
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gram(const __nv_bfloat16* __restrict__ Xd, int ncbx, const __nv_bfloat16* __restrict__ Yd, int ncby,
              int64_t nkc, int m, int n, int ntj, int sym, int64_t kc_per_slice, const int* ex,
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
  const int64_t kc0 = (int64_t)blockIdx.y * kc_per_slice;
  const int nsub = (int)min(kc_per_slice, nkc - kc0);
  uint64_t *full, *empty;
  const uint32_t tmem = tile_setup(smem, &full, &empty);
  Acc acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = Acc{0, 0};
  const int64_t a_kc = 8LL * ncbx * B_ELEMS, a_s = (int64_t)ncbx * B_ELEMS;
  const int64_t b_kc = 8LL * ncby * B_ELEMS, b_s = (int64_t)ncby * B_ELEMS;
  const bool ok = run_tile(smem, full, empty, tmem, Xd + kc0 * a_kc + (int64_t)(2 * ti) * B_ELEMS, a_kc, a_s,
                           Yd + kc0 * b_kc + (int64_t)tj * B_ELEMS, b_kc, b_s, nsub, acc);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    double* Ps = P + (int64_t)blockIdx.y * m * n;
    write_tile(
        smem, acc,
        [&](int i, int j) {
          const int gi = i0 + i, gj = j0 + j;
          return (gi < m && gj < n) ? ex[gi] + ey[gj] - 63 : 0;
        },
        [&](int i, int j, double v) {
          const int gi = i0 + i, gj = j0 + j;
          if (gi < m && gj < n) Ps[(int64_t)gi * n + gj] = v;
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
// rotation: Out[r][j] = sum_k V[r][k] M[k][j] from the row-scaled digits of V
// and the column-scaled digits of M; tile (rb, jt) covers rows [128 rb, +128)
// and columns [64 jt, +64)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_rotate(const __nv_bfloat16* __restrict__ Vd, const __nv_bfloat16* __restrict__ Md, int ncbm,
                int64_t D, int n, int npad, int upper, const int* er, const int* em,
                double* __restrict__ Out, int64_t ldo, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  // the column tiles of one row block are consecutive CTAs, so the row
  // block's digits are read from HBM once and then from L2
  const int njt = npad / TN;
  const int64_t rb = blockIdx.x / njt;
  const int jt = (int)(blockIdx.x % njt), j0 = jt * TN;
  const int kend = upper ? min(npad, j0 + TN) : npad;  // M upper triangular: rows k <= j
  const int64_t nkc = npad / KS;
  uint64_t *full, *empty;
  const uint32_t tmem = tile_setup(smem, &full, &empty);
  Acc acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = Acc{0, 0};
  const int64_t b_kc = 8LL * ncbm * B_ELEMS, b_s = (int64_t)ncbm * B_ELEMS;
  const bool ok = run_tile(smem, full, empty, tmem, Vd + rb * nkc * 8 * A_ELEMS, 8LL * A_ELEMS, A_ELEMS,
                           Md + (int64_t)jt * B_ELEMS, b_kc, b_s, kend / KS, acc);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    const int64_t r0 = rb * TM;
    write_tile(
        smem, acc,
        [&](int i, int j) {
          const int64_t gr = r0 + i;
          const int gj = j0 + j;
          return (gr < D && gj < n) ? er[gr] + em[gj] - 63 : 0;
        },
        [&](int i, int j, double v) {
          const int64_t gr = r0 + i;
          const int gj = j0 + j;
          if (gr < D && gj < n) Out[gr * ldo + gj] = v;
        });
  }
  tile_teardown(tmem);
}

// the failure path in isolation: a barrier nobody arrives on
__global__ void k_wait_unsatisfied(long long limit, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, limit);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(err, 1);
}

// bit d: the shared-memory attribute is set on device d (a function attribute
// is per device; setting it twice is harmless, so racing threads only repeat it)
std::atomic<unsigned long long> attrs_set{0};

fd_status set_attrs(fd_ctx* ctx) {
  const unsigned long long bit = ctx->device < 64 ? 1ull << ctx->device : 0ull;
  if (bit && (attrs_set.load() & bit)) return FD_OK;
  FD_CUDA(ctx, cudaFuncSetAttribute(k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
  FD_CUDA(ctx, cudaFuncSetAttribute(k_oz_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
  attrs_set.fetch_or(bit);
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

// digit workspace; false (no error) if it cannot be allocated: the caller
// then takes the FP64 path
bool digit_workspace(fd_ctx* ctx, const char* name, size_t bytes, __nv_bfloat16** out) {
  void* p = nullptr;
  if (workspace(ctx, name, bytes, &p) != FD_OK) {
    ctx->err.clear();
    return false;
  }
  *out = (__nv_bfloat16*)p;
  return true;
}

// column-scaled digits of a D x w operand (K = D rows, padded to 16)
fd_status cut_cols(fd_ctx* ctx, const double* X, int64_t ld, int64_t D, int w, const int* ex,
                   __nv_bfloat16* Xd, int64_t nkc) {
  const int wpad = (int)cdiv(w, TM) * TM;
  const int64_t items = nkc * 2 * wpad;
  k_digits_cols<<<(unsigned)cdiv(items, 256), 256, 0, ctx->stream>>>(X, ld, D, w, wpad, ex, nkc, Xd);
  FD_LAUNCHED(ctx);
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
  const bool same = Y == X && ldy == ldx;
  const int64_t nkc = cdiv(D, KS);
  const int ncbx = (int)cdiv(m, TM) * 2, ncby = (int)cdiv(n, TM) * 2;
  __nv_bfloat16 *Xd, *Yd;
  if (!digit_workspace(ctx, "oz_digits_a", sizeof(__nv_bfloat16) * (size_t)nkc * KS * ncbx * 64 * OZ_S, &Xd))
    return FD_OK;
  Yd = Xd;
  if (!same &&
      !digit_workspace(ctx, "oz_digits_b", sizeof(__nv_bfloat16) * (size_t)nkc * KS * ncby * 64 * OZ_S, &Yd))
    return FD_OK;
  void* p;
  FD_TRY(workspace(ctx, "oz_exp", sizeof(int) * ((size_t)m + n + 8), &p));
  int* ex = (int*)p;
  int* ey = ex + m;
  int* bad = ey + n;
  int* err = bad + 1;
  FD_CUDA(ctx, cudaMemsetAsync(bad, 0, 2 * sizeof(int), ctx->stream));
  FD_TRY(col_exponents(ctx, X, ldx, D, m, ex, bad));
  if (!same) FD_TRY(col_exponents(ctx, Y, ldy, D, n, ey, bad));
  else FD_CUDA(ctx, cudaMemcpyAsync(ey, ex, sizeof(int) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  int hbad = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hbad) return FD_OK;  // non-finite input: the FP64 path propagates it
  FD_TRY(cut_cols(ctx, X, ldx, D, m, ex, Xd, nkc));
  if (!same) FD_TRY(cut_cols(ctx, Y, ldy, D, n, ey, Yd, nkc));
  const int nti = (int)cdiv(m, TM), ntj = (int)cdiv(n, TN);
  int tiles = 0;
  if (sym) {
    for (int ti = 0; ti < nti; ++ti) tiles += std::max(0, ntj - 2 * ti);
  } else {
    tiles = nti * ntj;
  }
  // about four waves of one CTA per SM; at most 2^16 exact chunks per CTA
  int64_t slices = std::max<int64_t>(1, (4LL * ctx->num_sms) / tiles);
  slices = std::min<int64_t>(slices, std::max<int64_t>(1, cdiv(nkc, 4 * SUBS)));
  slices = std::max<int64_t>(slices, cdiv(nkc, OZ_MAX_CHUNKS * SUBS));
  const int64_t kps = cdiv(nkc, slices);
  slices = cdiv(nkc, kps);
  FD_TRY(workspace(ctx, "oz_gram_partial", sizeof(double) * slices * m * n, &p));
  double* P = (double*)p;
  k_oz_gram<<<dim3(tiles, (unsigned)slices), OZ_THREADS, OZ_SMEM, ctx->stream>>>(
      Xd, ncbx, Yd, ncby, nkc, m, n, ntj, sym ? 1 : 0, kps, ex, ey, P, err);
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
  const int npad = (int)cdiv(n, TN) * TN;  // K of the product, in whole 64-column blocks of M
  const int64_t Dpad = cdiv(D, TM) * TM;
  const int ncbm = (int)cdiv(n, TM) * 2;
  __nv_bfloat16 *Vd, *Md;
  if (!digit_workspace(ctx, "oz_digits_a", sizeof(__nv_bfloat16) * (size_t)Dpad * npad * OZ_S, &Vd))
    return FD_OK;
  if (!digit_workspace(ctx, "oz_digits_m", sizeof(__nv_bfloat16) * (size_t)npad * ncbm * 64 * OZ_S, &Md))
    return FD_OK;
  void* p;
  FD_TRY(workspace(ctx, "oz_rot_small", sizeof(int) * ((size_t)n + D + 8), &p));
  int* em = (int*)p;
  int* er = em + n;
  int* bad = er + D;
  int* err = bad + 1;
  FD_CUDA(ctx, cudaMemsetAsync(bad, 0, 2 * sizeof(int), ctx->stream));
  FD_TRY(col_exponents(ctx, M, n, n, n, em, bad));
  FD_TRY(cut_cols(ctx, M, n, n, n, em, Md, npad / KS));
  const int vec = (((uintptr_t)V & 15) == 0 && (ldv & 1) == 0) ? 1 : 0;
  k_digits_rows<<<(unsigned)cdiv(Dpad, 8), 256, 0, ctx->stream>>>(V, ldv, D, n, Dpad, npad, vec, er, bad, Vd);
  FD_LAUNCHED(ctx);
  int hbad = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hbad) return FD_OK;  // non-finite input: the FP64 path propagates it
  FD_TRY(workspace(ctx, "oz_rot_out", sizeof(double) * (size_t)D * n, &p));
  double* Out = (double*)p;
  k_oz_rotate<<<(unsigned)((Dpad / TM) * (npad / TN)), OZ_THREADS, OZ_SMEM, ctx->stream>>>(
      Vd, Md, ncbm, D, n, npad, upper ? 1 : 0, er, em, Out, n, err);
  FD_LAUNCHED(ctx);
  FD_TRY(check_wait_flag(ctx, err));
  FD_CUDA(ctx, cudaMemcpy2DAsync(V, ldv * sizeof(double), Out, n * sizeof(double), n * sizeof(double), D,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
  *used = true;
  return FD_OK;
}

}  // namespace fdi

using namespace fdi;

extern "C" fd_status fd_check_bounded_wait(fd_ctx* ctx, int limit_us) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (limit_us < 1 || limit_us > 10000000) return set_err(ctx, FD_ERR_ARG, "limit_us must be 1 .. 10^7");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  int khz = 0;
  FD_CUDA(ctx, cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device));
  void* p;
  FD_TRY(workspace(ctx, "wait_check", sizeof(int), &p));
  int* err = (int*)p;
  FD_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  const long long limit = (long long)limit_us * (khz > 0 ? khz : 2000000) / 1000;
  k_wait_unsatisfied<<<1, 32, 0, ctx->stream>>>(limit, err);
  FD_LAUNCHED(ctx);
  return check_wait_flag(ctx, err);
}
