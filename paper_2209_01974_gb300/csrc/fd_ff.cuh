// Float-float ("double-word") arithmetic for the FP64-accurate filter sweeps.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate, so an FP64 Chebyshev
// sweep is bound by FP64 arithmetic, not by HBM.  A float-float number is an
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2: a 48-bit
// significand in the FP32 exponent range, held in the same 8 bytes as a
// double.  The operations are built from error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2 4.2.2):  s + e = a + b exactly, 6 additions;
//   Fast2Sum (Dekker 1971), |a| >= |b|:   s + e = a + b exactly, 3 additions;
//   TwoProd with an FMA:                  p + e = a * b exactly, p = a*b,
//                                         e = fma(a, b, -p).
// The sum below is the "sloppy" double-word addition: TwoSum of the high
// parts, the low parts added in plain FP32, one Fast2Sum to renormalise.  Its
// error is within a few u^2 (u = 2^-24) of |a| + |b| (absolute, like the
// rounding error of an FP64 sum, which is within u64 = 2^-53 of |a| + |b|).
// The product is the double-word times double-word product with FMA (TwoProd
// of the high parts plus the two cross products), relative error a few u^2.
// Every step uses the _rn intrinsics, so the compiler neither contracts nor
// reorders them.  Values must stay inside the FP32 range (the Chebyshev
// recurrence keeps |T_k| <= 1 on the scaled spectrum).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_step.cuh"

namespace fdi {
namespace ffa {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // exact split of an int literal (0, 1) and nearest split of a double
  __host__ __device__ explicit ff(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ explicit ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float aa = __fsub_rn(s, bb);
  e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  ff r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
// c + a * b for running sums (the row sums of the SpMMV): the exact product
// of the high parts (TwoProd) and the exact sum of it with c.hi (TwoSum) give
// the new high part; every remaining term (both rounding errors, the cross
// products, c.lo) is added in plain FP32 to the low part, which is left
// unnormalised.  The low part then carries an error of a few u^2 of the terms
// summed so far, as in the normalised sum; the pair is renormalised by the next
// product or sum (12 FP32 operations instead of 18).
__device__ __forceinline__ ff fma(ff a, ff b, ff c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  float s, t;
  two_sum(c.hi, p, s, t);
  return ff(s, __fadd_rn(__fadd_rn(t, e), c.lo));
}

// read-only loads of one value (matrix entries)
__device__ __forceinline__ ff ldg_val(const ff* p) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  return ff(t.x, t.y);
}

}  // namespace ffa

namespace step {

// two float-float values per 16-byte vector, each stored as (hi, lo)
template <>
struct V16<ffa::ff> {
  using ff = ffa::ff;
  static constexpr int E = 2;
  ff v[2];
  __device__ __forceinline__ void set(const float4& t) { v[0] = ff(t.x, t.y); v[1] = ff(t.z, t.w); }
  __device__ __forceinline__ float4 get() const { return make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo); }
  __device__ __forceinline__ void ldg(const ff* p) { set(__ldg(reinterpret_cast<const float4*>(p))); }
  __device__ __forceinline__ void ldcs(const ff* p) { set(__ldcs(reinterpret_cast<const float4*>(p))); }
  __device__ __forceinline__ void stcs(ff* p) const { __stcs(reinterpret_cast<float4*>(p), get()); }
  __device__ __forceinline__ void st(ff* p) const { *reinterpret_cast<float4*>(p) = get(); }
  __device__ __forceinline__ void ldg_pol(const ff* p, uint64_t pol) {
    float4 t;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;\n"
        : "=f"(t.x), "=f"(t.y), "=f"(t.z), "=f"(t.w) : "l"(p), "l"(pol));
    set(t);
  }
  __device__ __forceinline__ void ld_pol(const ff* p, uint64_t pol) {
    float4 t;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;\n"
                 : "=f"(t.x), "=f"(t.y), "=f"(t.z), "=f"(t.w) : "l"(p), "l"(pol));
    set(t);
  }
  __device__ __forceinline__ void st_pol(ff* p, uint64_t pol) const {
    const float4 t = get();
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;\n"
                 :: "l"(p), "f"(t.x), "f"(t.y), "f"(t.z), "f"(t.w), "l"(pol));
  }
};

// Float-float steps run the FP32 shape: 4-warp CTAs, 12 per SM (<= 40
// registers, no spills up to nb = 64).  Memory latency, not the FP32 pipes,
// bounds the float-float step, and on the GB300 this shape (48 warps per SM)
// took 1.41 ms per L = 128 stencil step at nb = 64 against 1.86 ms with the
// FP64 shape (8-warp CTAs, 4 per SM).
template <>
struct StepShape<ffa::ff> {
  static constexpr int warps = 4;
  static constexpr int min_blocks = MIN_BLOCKS;
};

}  // namespace step
}  // namespace fdi
