// Device building blocks of the fused Chebyshev step (Sec. 2, Alg. 2), shared
// by the single-block filter and the batched persistent filter.
//
// Work mapping: a group of G lanes owns one SELL row; each lane holds CPL
// 16-byte vectors of the row (G * CPL * 16 bytes = nb * sizeof(T)), so every
// gathered row of W1 is one fully coalesced access.  A warp holds 32/G
// consecutive rows of one SELL chunk, so the warp's matrix loads at entry j
// touch adjacent words of the chunk's column-major slab.  Entry 0 of every
// SELL row is its diagonal, so the row's own W1 vector (needed for the beta
// term) is the first gathered vector.  W2 and V are touched once per step and
// use evict-first (.cs) loads and stores, keeping L2 for the W1 gathers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdi {
namespace step {

template <typename T>
struct V16;
template <>
struct V16<double> {
  static constexpr int E = 2;
  double v[2];
  __device__ __forceinline__ void ldg(const double* p) {
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
  }
  __device__ __forceinline__ void ldcs(const double* p) {
    double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
  }
  __device__ __forceinline__ void stcs(double* p) const {
    __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
  }
  __device__ __forceinline__ void st(double* p) const {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
  // loads and stores with an L2 eviction policy (createpolicy); the loads do
  // not allocate in L1.  ldg_pol: read-only data (non-coherent path)
  __device__ __forceinline__ void ldg_pol(const double* p, uint64_t pol) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;\n"
        : "=d"(v[0]), "=d"(v[1]) : "l"(p), "l"(pol));
  }
  __device__ __forceinline__ void ld_pol(const double* p, uint64_t pol) {
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;\n"
                 : "=d"(v[0]), "=d"(v[1]) : "l"(p), "l"(pol));
  }
  __device__ __forceinline__ void st_pol(double* p, uint64_t pol) const {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;\n"
                 :: "l"(p), "d"(v[0]), "d"(v[1]), "l"(pol));
  }
};
template <>
struct V16<float> {
  static constexpr int E = 4;
  float v[4];
  __device__ __forceinline__ void ldg(const float* p) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ __forceinline__ void ldcs(const float* p) {
    float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ __forceinline__ void stcs(float* p) const {
    __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  }
  __device__ __forceinline__ void st(float* p) const {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
  __device__ __forceinline__ void ldg_pol(const float* p, uint64_t pol) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;\n"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p), "l"(pol));
  }
  __device__ __forceinline__ void ld_pol(const float* p, uint64_t pol) {
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;\n"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p), "l"(pol));
  }
  __device__ __forceinline__ void st_pol(float* p, uint64_t pol) const {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;\n"
                 :: "l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "l"(pol));
  }
};

// L2 eviction policies for cache_hint accesses: the whole access range evicts
// last (data re-read within a short window) or first (streamed once)
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}

// read-only load of one matrix value (float-float values have their own)
template <typename T>
__device__ __forceinline__ T ldg_val(const T* p) { return __ldg(p); }

template <typename T>
struct SellArgs {
  const int64_t* chunk_ptr;
  const int32_t* row_len;
  const int32_t* col;
  const T* val;
  int64_t D;
  int C;
};

enum { MODE_SPMMV = 0, MODE_SECOND = 1, MODE_GENERIC = 2 };

template <typename T>
struct StepArgs {
  const T* X; int64_t ldx;   // gathered operand x_{k-1}
  const T* Z; int64_t ldz;   // x_{k-2}, row-wise (may alias Y or Vout at the same row)
  T* Y; int64_t ldy;         // x_k output, or nullptr
  const T* Vin; int64_t ldvi;
  T* Vout; int64_t ldvo;
  T c_ax, c_x;               // x_k = c_ax * (A x_{k-1}) + c_x * x_{k-1} [- x_{k-2}]
  T mu0, mu1, mu2;           // SECOND: Vout = mu0 z + mu1 x + mu2 y; GENERIC: Vout = Vin + mu2 y
};

constexpr int WARPS = 8;
constexpr int BATCH = 4;   // entries per batch; SELL chunk lengths are multiples of 8
constexpr int MIN_BLOCKS = 12;     // FP32 steps: 4-warp CTAs, 48 resident warps per SM (<= 40 registers)
constexpr int MIN_BLOCKS_F64 = 4;  // FP64 steps: 8-warp CTAs with 64 registers (FP64-ALU bound anyway)
// CTA shape of the fused step (k_cheb_step): warps per CTA and resident CTAs
// per SM (the launch bounds).  Smaller CTAs for FP32 (more of them in flight, a
// finer L2 prefetch granule), 8 warps for FP64; other arithmetic types may
// specialise it.
template <typename T>
struct StepShape {
  static constexpr int warps = sizeof(T) == 4 ? 4 : WARPS;
  static constexpr int min_blocks = sizeof(T) == 4 ? MIN_BLOCKS : MIN_BLOCKS_F64;
};
template <typename T>
__host__ __device__ constexpr int step_warps() { return StepShape<T>::warps; }
template <typename T>
__host__ __device__ constexpr int step_min_blocks() { return StepShape<T>::min_blocks; }

template <typename T, int NB>
struct Layout {
  static constexpr int E = V16<T>::E;
  static constexpr int Q = NB / E;                 // 16-byte vectors per row
  static constexpr int G = Q >= 32 ? 32 : Q;        // lanes per row
  static constexpr int CPL = Q / G;                 // vectors per lane
  static constexpr int RPW = 32 / G;                // rows per warp
  static_assert(NB % E == 0 && Q % G == 0, "nb must fill whole 16-byte vectors");
};

// Gather-accumulate s = sum_j a_ij x_j over the SELL row, returning the row's
// own vector xi (entry 0 is the diagonal).  Entries are taken BATCH at a time:
// the matrix loads of a batch, then all its gathers, so a row of up to BATCH
// entries costs one round trip of dependent loads.  Chunk lengths are padded to
// a multiple of BATCH with (0, own row) entries, so the matrix loads need no
// bounds; the gathers and FMAs of entries past the row's own length are
// skipped (FP64 arithmetic, not memory, bounds the FP64 step on GB300).
template <typename T, int NB>
__device__ __forceinline__ void row_product(const SellArgs<T>& A, const T* __restrict__ X,
                                            int64_t ldx, int64_t row, bool active, int len,
                                            int wlen, int gl, V16<T> (&acc)[Layout<T, NB>::CPL],
                                            V16<T> (&xi)[Layout<T, NB>::CPL]) {
  using L = Layout<T, NB>;
  constexpr int E = L::E;
  // Rows at or beyond D inside the last chunk are SELL padding rows: their
  // entries exist (value 0, column 0), but they have no vector row.
  const int64_t base = A.chunk_ptr[row / A.C] + (row % A.C);
  const int32_t* cp = A.col + base;
  const T* vp = A.val + base;
  const uint32_t C = (uint32_t)A.C;
  const uint32_t ld = (uint32_t)ldx;
  const T* xl = X + gl * E;
  {
    int32_t c[BATCH];
    T a[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      c[u] = __ldg(cp + u * C);
      a[u] = ldg_val(vp + u * C);
    }
    if (!active) { c[0] = 0; a[0] = T(0); }
#pragma unroll
    for (int v = 0; v < L::CPL; ++v) {
      xi[v].ldg(xl + (uint64_t)(uint32_t)c[0] * ld + v * L::G * E);
#pragma unroll
      for (int e = 0; e < E; ++e) acc[v].v[e] = a[0] * xi[v].v[e];
    }
#pragma unroll
    for (int u = 1; u < BATCH; ++u) {
      if (u < len) {  // entries past the row's length are padding: skip their FMAs
#pragma unroll
        for (int v = 0; v < L::CPL; ++v) {
          V16<T> x;
          x.ldg(xl + (uint64_t)(uint32_t)c[u] * ld + v * L::G * E);
#pragma unroll
          for (int e = 0; e < E; ++e) acc[v].v[e] = fma(a[u], x.v[e], acc[v].v[e]);
        }
      }
    }
  }
  for (int j0 = BATCH; j0 < wlen; j0 += BATCH) {
    int32_t c[BATCH];
    T a[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      c[u] = __ldg(cp + (j0 + u) * C);
      a[u] = ldg_val(vp + (j0 + u) * C);
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      if (j0 + u < len) {
#pragma unroll
        for (int v = 0; v < L::CPL; ++v) {
          V16<T> x;
          x.ldg(xl + (uint64_t)(uint32_t)c[u] * ld + v * L::G * E);
#pragma unroll
          for (int e = 0; e < E; ++e) acc[v].v[e] = fma(a[u], x.v[e], acc[v].v[e]);
        }
      }
    }
  }
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}
// bulk L2 prefetch of `bytes` contiguous bytes (16-byte aligned address and
// size), issued by one thread to the copy engine; nothing waits for it
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch for the rows [r0, r1) of a later CTA: the 128-byte lines of
// their row-wise operands (the own row of X, Z, Vin) and the SELL slabs of the
// chunks that start inside the range.  A prefetch holds no register and no
// scoreboard entry, so the later CTA finds its first, dependent loads in L2.
template <typename T, int NB, int MODE>
__device__ __forceinline__ void prefetch_rows(const SellArgs<T>& A, const StepArgs<T>& s,
                                              int64_t r0, int64_t r1) {
  constexpr int LPR = (NB * (int)sizeof(T) + 127) / 128;  // lines per vector row
  constexpr int NS = MODE == MODE_GENERIC ? 3 : MODE == MODE_SECOND ? 2 : 1;
  const int n = (int)(r1 - r0) * LPR;
  for (int q = threadIdx.x; q < NS * n; q += blockDim.x) {
    const int st = q / n, rq = q % n;
    const int64_t row = r0 + rq / LPR;
    const int64_t off = (int64_t)(rq % LPR) * (128 / (int)sizeof(T));
    const T* p = st == 0 ? s.X + row * s.ldx : st == 1 ? s.Z + row * s.ldz : s.Vin + row * s.ldvi;
    prefetch_l2(p + off);
  }
  if (threadIdx.x >= blockDim.x - 32) {
    const int64_t c0 = (r0 + A.C - 1) / A.C, c1 = (r1 + A.C - 1) / A.C;
    if (c0 >= c1) return;
    const int64_t e0 = A.chunk_ptr[c0], e1 = A.chunk_ptr[c1];
    const int64_t l0c = (e0 * 4) >> 7, l1c = (e1 * 4 + 127) >> 7;
    const int64_t l0v = (e0 * (int64_t)sizeof(T)) >> 7, l1v = (e1 * (int64_t)sizeof(T) + 127) >> 7;
    const int64_t nc = l1c - l0c, nv = l1v - l0v;
    const char* cb = reinterpret_cast<const char*>(A.col);
    const char* vb = reinterpret_cast<const char*>(A.val);
    for (int64_t q = threadIdx.x & 31; q < nc + nv; q += 32)
      prefetch_l2(q < nc ? cb + ((l0c + q) << 7) : vb + ((l0v + q - nc) << 7));
  }
}

// One fused Chebyshev step (or a plain SpMMV) for the warp's rows row0 ..
// row0 + RPW - 1 (row0 < D, a multiple of RPW); all 32 lanes must call it.
template <typename T, int NB, int MODE>
__device__ __forceinline__ void cheb_rows(const SellArgs<T>& A, const StepArgs<T>& s,
                                          int64_t row0) {
  using L = Layout<T, NB>;
  constexpr int E = L::E;
  const int lane = threadIdx.x & 31;
  const int g = lane / L::G, gl = lane % L::G;
  const int64_t row = row0 + g;
  const bool active = row < A.D;
  const int len = active ? A.row_len[row] : 0;
  const int wlen = __reduce_max_sync(0xffffffffu, len);

  // the row-wise operands do not depend on the gathers: issue them first
  V16<T> z[L::CPL], vin[L::CPL];
  if (MODE != MODE_SPMMV && active) {
#pragma unroll
    for (int v = 0; v < L::CPL; ++v) {
      const int64_t off = gl * E + v * L::G * E;
      z[v].ldcs(s.Z + row * s.ldz + off);
      if (MODE == MODE_GENERIC) vin[v].ldcs(s.Vin + row * s.ldvi + off);
    }
  }
  V16<T> acc[L::CPL], xi[L::CPL];
  row_product<T, NB>(A, s.X, s.ldx, row, active, len, wlen, gl, acc, xi);
  if (!active) return;

#pragma unroll
  for (int v = 0; v < L::CPL; ++v) {
    const int64_t off = gl * E + v * L::G * E;
    V16<T> y;
    if (MODE == MODE_SPMMV) {
#pragma unroll
      for (int e = 0; e < E; ++e) y.v[e] = s.c_ax * acc[v].v[e] + s.c_x * xi[v].v[e];
      y.st(s.Y + row * s.ldy + off);
    } else {
      V16<T> o;
#pragma unroll
      for (int e = 0; e < E; ++e) y.v[e] = s.c_ax * acc[v].v[e] + s.c_x * xi[v].v[e] - z[v].v[e];
      if (MODE == MODE_SECOND) {
#pragma unroll
        for (int e = 0; e < E; ++e)
          o.v[e] = s.mu0 * z[v].v[e] + s.mu1 * xi[v].v[e] + s.mu2 * y.v[e];
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) o.v[e] = vin[v].v[e] + s.mu2 * y.v[e];
      }
      if (s.Y) y.st(s.Y + row * s.ldy + off);
      o.stcs(s.Vout + row * s.ldvo + off);
    }
  }
}

// ---------------------------------------------------------------------------
// Matrix-free Hubbard operator (Sec. 4 runs FD on Hubbard matrices; the
// paper's production runs apply them without storing them):
//   (H x)_(u,d) = U n(u,d) x_(u,d) + sum_u' h_up(u,u') x_(u',d)
//                                  + sum_d' h_dn(d,d') x_(u,d')
// with row (u, d) = u * dim_dn + d.  The up-spin hops of consecutive rows
// (u, d), (u, d + 1) read consecutive rows (u', d), (u', d + 1): whole
// coalesced row blocks; the down-spin hops stay inside the u slab.
// ---------------------------------------------------------------------------
template <typename T>
struct KronArgs {
  int64_t D, dim_dn;
  const uint32_t* bits_up;
  const uint32_t* bits_dn;
  const int64_t* ptr_up;
  const int32_t* col_up;
  const T* val_up;
  const int64_t* ptr_dn;
  const int32_t* col_dn;
  const T* val_dn;
  const T* diag;  // 25 entries: U * n for n doubly occupied sites
};

// s = sum_j h_ij x_j for row (u, d), the entries in the order of the stored
// row (diagonal first, then ascending columns: the up hops to u' < u, the
// down hops, the up hops to u' > u), so the sums round as in the SELL kernel
template <typename T, int NB>
__device__ __forceinline__ void kron_row_product(const KronArgs<T>& K, const T* __restrict__ X, int64_t ldx,
                                                 int64_t row, int gl, V16<T> (&acc)[Layout<T, NB>::CPL],
                                                 V16<T> (&xi)[Layout<T, NB>::CPL]) {
  using L = Layout<T, NB>;
  constexpr int E = L::E;
  const T* xl = X + gl * E;
  const int64_t u = row / K.dim_dn, d = row - u * K.dim_dn;
  const T dg = K.diag[__popc(K.bits_up[u] & K.bits_dn[d])];
#pragma unroll
  for (int v = 0; v < L::CPL; ++v) {
    xi[v].ldg(xl + row * ldx + v * L::G * E);
#pragma unroll
    for (int e = 0; e < E; ++e) acc[v].v[e] = dg * xi[v].v[e];
  }
  auto add = [&](T a, int64_t r) {
#pragma unroll
    for (int v = 0; v < L::CPL; ++v) {
      V16<T> x;
      x.ldg(xl + r * ldx + v * L::G * E);
#pragma unroll
      for (int e = 0; e < E; ++e) acc[v].v[e] = fma(a, x.v[e], acc[v].v[e]);
    }
  };
  int64_t k = K.ptr_up[u];
  const int64_t ke = K.ptr_up[u + 1];
  for (; k < ke && K.col_up[k] < u; ++k) add(K.val_up[k], (int64_t)K.col_up[k] * K.dim_dn + d);
  const int64_t kd1 = K.ptr_dn[d + 1];
  for (int64_t kd = K.ptr_dn[d]; kd < kd1; ++kd) add(K.val_dn[kd], u * K.dim_dn + K.col_dn[kd]);
  for (; k < ke; ++k) add(K.val_up[k], (int64_t)K.col_up[k] * K.dim_dn + d);
}

// One fused Chebyshev step with the matrix-free Hubbard operator; the same
// operand loads and epilogue as cheb_rows
template <typename T, int NB, int MODE>
__device__ __forceinline__ void kron_rows(const KronArgs<T>& K, const StepArgs<T>& s, int64_t row0) {
  using L = Layout<T, NB>;
  constexpr int E = L::E;
  const int lane = threadIdx.x & 31;
  const int g = lane / L::G, gl = lane % L::G;
  const int64_t row = row0 + g;
  if (row >= K.D) return;  // no warp-wide operations follow
  V16<T> z[L::CPL], vin[L::CPL];
  if (MODE != MODE_SPMMV) {
#pragma unroll
    for (int v = 0; v < L::CPL; ++v) {
      const int64_t off = gl * E + v * L::G * E;
      z[v].ldcs(s.Z + row * s.ldz + off);
      if (MODE == MODE_GENERIC) vin[v].ldcs(s.Vin + row * s.ldvi + off);
    }
  }
  V16<T> acc[L::CPL], xi[L::CPL];
  kron_row_product<T, NB>(K, s.X, s.ldx, row, gl, acc, xi);
#pragma unroll
  for (int v = 0; v < L::CPL; ++v) {
    const int64_t off = gl * E + v * L::G * E;
    V16<T> y;
    if (MODE == MODE_SPMMV) {
#pragma unroll
      for (int e = 0; e < E; ++e) y.v[e] = s.c_ax * acc[v].v[e] + s.c_x * xi[v].v[e];
      y.st(s.Y + row * s.ldy + off);
    } else {
      V16<T> o;
#pragma unroll
      for (int e = 0; e < E; ++e) y.v[e] = s.c_ax * acc[v].v[e] + s.c_x * xi[v].v[e] - z[v].v[e];
      if (MODE == MODE_SECOND) {
#pragma unroll
        for (int e = 0; e < E; ++e)
          o.v[e] = s.mu0 * z[v].v[e] + s.mu1 * xi[v].v[e] + s.mu2 * y.v[e];
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) o.v[e] = vin[v].v[e] + s.mu2 * y.v[e];
      }
      if (s.Y) y.st(s.Y + row * s.ldy + off);
      o.stcs(s.Vout + row * s.ldvo + off);
    }
  }
}

}  // namespace step
}  // namespace fdi
