// Matrix-free Hubbard operator in the fused Chebyshev step, laid out for L2
// reuse (the paper applies its Hubbard matrices without storing them, Sec. 4.2;
// the step is Alg. 2's fused SpMMV + recurrence + accumulation, Sec. 3.2):
//   (H x)_(u,d) = U n(u,d) x_(u,d) + sum_u' h_up(u,u') x_(u',d)
//                                  + sum_d' h_dn(d,d') x_(u,d')
// with row (u, d) = u * dim_dn + d.  The rows of one up-spin state u form a
// slab of dim_dn consecutive rows.  The down-spin hops of a row stay inside its
// slab; the up-spin hops read the rows with the same d in the slabs u' of the
// up-spin hopping graph's neighbours of u, which in rank order lie all over the
// vector.
//
// Layout and traversal (FP32 sweeps).  The D x nb block is split into column
// panels of one 16-byte vector per row (4 columns); panel p is a contiguous
// D x 16-byte array, so a slab of a panel is dim_dn * 16 bytes (55 KB for the
// 14-site ring) and a whole panel of x_{k-1} is D * 16 bytes.  The Chebyshev
// recurrence is independent per column, so a step runs the panels one after
// the other (CTA index = panel-major), and within a panel the slabs in reverse
// Cuthill-McKee order of the up-spin hopping graph: the slabs a slab reads are
// then visited close to it in time.  The gathered x_{k-1} is read with the L2
// policy evict_last and the once-streamed rows (x_{k-2}, the accumulator, the
// x_k written) with evict_first, so the x_{k-1} slabs still to be read stay in
// L2 while four times their bytes stream past (without the policies nearly
// every gather missed; the full-width row-major step re-read x_{k-1} about
// three times from HBM).  One CTA processes one slab of one panel: it first
// stages the slab's own rows of x_{k-1} in shared memory (they serve the row's
// own term and every down-spin hop), takes the slab's up-spin hop list (uniform
// over the CTA) into shared memory, and then gives each thread rows d, d + 512,
// ...: the up-spin gathers of a warp read 32 consecutive rows of slab u', one
// fully used 512-byte run, issued KP_BATCH at a time.  The down-spin hop table
// (16-bit byte offsets into the staged slab, with the fermion sign in bit 0) is
// the same for every slab and stays in L1: the shared-memory carve-out is set
// to what the two resident CTAs need.
//
// Each row is summed as diagonal, up-spin hops (ascending u'), down-spin hops
// (ascending d'): the stored SELL row's entries in another order, so results
// agree with the stored-matrix kernel to rounding (both within the oracle's
// bound) rather than bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fd_internal.cuh"
#include "fd_step.cuh"

namespace fdi {
namespace {

using step::MODE_GENERIC;
using step::MODE_SECOND;
using step::MODE_SPMMV;
using step::V16;

constexpr int KP_THREADS = 512;
constexpr int KP_MIN_BLOCKS = 2;
constexpr int KP_BATCH = 6;                      // up-spin gathers issued together
constexpr int KP_MAX_HOPS = 48;                  // 2 L hops at most for L <= 24 sites
constexpr int64_t KP_STAGE_MAX = 64 * 1024;      // own slab staged in shared memory up to this
constexpr int KP_ROWS_UNSTAGED = KP_THREADS * 8; // rows of a slab per CTA when not staged

template <typename T>
struct KronPanel {
  int64_t D;
  int dim_up, dim_dn, chunks;      // chunks: CTAs per slab (1 when staged)
  const int32_t* order;            // slabs in visiting order
  const uint32_t* bits_up;
  const uint32_t* bits_dn;
  const int64_t* ptr_up;
  const int32_t* col_up;
  const T* val_up;
  const uint32_t* dn_ptr;
  const uint32_t* dn_ent;          // target | sign bit << 31 (slabs not staged)
  const uint16_t* dn_ent16;        // 16 target | sign bit (staged slabs, dim_dn <= 4096):
                                   // the 14-site ring's table then stays in L1
  T dn_v0, dn_v1;                  // hop value for sign bit 0 / 1
  const T* diag;                   // U * n for n doubly occupied sites
};

// one step on panel-layout blocks: row r of panel p is the 16-byte vector at
// element (p * D + r) * E
template <typename T>
struct PanelStep {
  const T* X;          // x_{k-1}, gathered
  const T* Z;          // x_{k-2}, row-wise
  T* Y;                // x_k output, or nullptr
  const T* Vin;
  T* Vout;
  T c_ax, c_x;         // x_k = c_ax (H x_{k-1}) + c_x x_{k-1} [- x_{k-2}]
  T mu0, mu1, mu2;     // SECOND: Vout = mu0 z + mu1 x + mu2 y; GENERIC: Vout = Vin + mu2 y
};

template <typename T>
__device__ __forceinline__ void axpy(V16<T>& acc, T a, const V16<T>& x) {
#pragma unroll
  for (int e = 0; e < V16<T>::E; ++e) acc.v[e] = fma(a, x.v[e], acc.v[e]);
}

// N up-spin gathers of row d (slab bases hp[0..N), values hv[0..N)) issued
// together, then their FMAs in order
template <int N, typename T>
__device__ __forceinline__ void hop_batch(V16<T>& acc, const T* const* hp, const T* hv, int d,
                                          uint64_t keep) {
  V16<T> x[N];
#pragma unroll
  for (int q = 0; q < N; ++q) x[q].ldg_pol(hp[q] + (int64_t)d * V16<T>::E, keep);
#pragma unroll
  for (int q = 0; q < N; ++q) axpy(acc, hv[q], x[q]);
}

template <typename T>
__device__ __forceinline__ void up_hops(V16<T>& acc, const T* const* hp, const T* hv, int nh, int d,
                                        uint64_t keep) {
  int k = 0;
  for (; k + KP_BATCH <= nh; k += KP_BATCH) hop_batch<KP_BATCH>(acc, hp + k, hv + k, d, keep);
  switch (nh - k) {  // the hop count is the same for the whole CTA: no divergence
    case 1: hop_batch<1>(acc, hp + k, hv + k, d, keep); break;
    case 2: hop_batch<2>(acc, hp + k, hv + k, d, keep); break;
    case 3: hop_batch<3>(acc, hp + k, hv + k, d, keep); break;
    case 4: if constexpr (KP_BATCH > 4) hop_batch<4>(acc, hp + k, hv + k, d, keep); break;
    case 5: if constexpr (KP_BATCH > 5) hop_batch<5>(acc, hp + k, hv + k, d, keep); break;
    case 6: if constexpr (KP_BATCH > 6) hop_batch<6>(acc, hp + k, hv + k, d, keep); break;
    case 7: if constexpr (KP_BATCH > 7) hop_batch<7>(acc, hp + k, hv + k, d, keep); break;
    default: break;
  }
}

template <typename T, int MODE, bool STAGE>
__global__ void __launch_bounds__(KP_THREADS, KP_MIN_BLOCKS)
    k_kron_panel(KronPanel<T> K, PanelStep<T> s) {
  using V = V16<T>;
  constexpr int E = V::E;
  extern __shared__ __align__(16) unsigned char kp_smem[];
  __shared__ const T* hop_ptr[KP_MAX_HOPS];  // first row of slab u' in this panel
  __shared__ T hop_val[KP_MAX_HOPS];

  const int per_panel = K.dim_up * K.chunks;
  const int p = blockIdx.x / per_panel;
  const int rem = blockIdx.x - p * per_panel;
  const int su = rem / K.chunks;
  const int chunk = rem - su * K.chunks;
  const int u = K.order[su];
  const int64_t pbase = (int64_t)p * K.D;
  const int64_t r0 = (int64_t)u * K.dim_dn;
  const T* X = s.X + pbase * E;
  const int64_t k0 = K.ptr_up[u];
  const int nh = (int)(K.ptr_up[u + 1] - k0);
  for (int k = threadIdx.x; k < nh; k += blockDim.x) {
    hop_ptr[k] = X + (int64_t)K.col_up[k0 + k] * K.dim_dn * E;
    hop_val[k] = K.val_up[k0 + k];
  }
  // x_{k-1} is re-read by the neighbouring slabs' CTAs shortly: keep it in L2
  // ahead of the once-streamed x_{k-2}, accumulator and x_k rows
  const uint64_t keep = step::policy_evict_last();
  const uint64_t stream = step::policy_evict_first();
  V* slab = reinterpret_cast<V*>(kp_smem);
  if (STAGE)
    for (int d = threadIdx.x; d < K.dim_dn; d += blockDim.x) slab[d].ldg_pol(X + (r0 + d) * E, keep);
  __syncthreads();
  const uint32_t bu = K.bits_up[u];
  const int d_beg = STAGE ? 0 : chunk * KP_ROWS_UNSTAGED;
  const int d_end = STAGE ? K.dim_dn : min(K.dim_dn, (chunk + 1) * KP_ROWS_UNSTAGED);
  const T* Zs = s.Z + (pbase + r0) * E;    // row d of the slab at [d * E]
  const T* Vs = s.Vin + (pbase + r0) * E;
  T* Ys = s.Y ? s.Y + (pbase + r0) * E : nullptr;
  T* Os = s.Vout + (pbase + r0) * E;

  // the down-hop range and bit string of the thread's next row are loaded one
  // iteration ahead (the entries they index are then a single L1 round trip)
  uint32_t j0n = 0, j1n = 0, bn = 0;
  if (d_beg + (int)threadIdx.x < d_end) {
    const int d1 = d_beg + threadIdx.x;
    j0n = __ldg(K.dn_ptr + d1);
    j1n = __ldg(K.dn_ptr + d1 + 1);
    bn = __ldg(K.bits_dn + d1);
  }
#pragma unroll 1
  for (int d = d_beg + threadIdx.x; d < d_end; d += blockDim.x) {
    const int64_t o = (int64_t)d * E;
    V z, vin, xi, acc;
    if (MODE != MODE_SPMMV) {
      z.ld_pol(Zs + o, stream);
      if (MODE == MODE_GENERIC) vin.ld_pol(Vs + o, stream);
    }
    const uint32_t j0 = j0n, j1 = j1n, bd = bn;
    {
      const int dn = d + blockDim.x;
      if (dn < d_end) {
        j0n = __ldg(K.dn_ptr + dn);
        j1n = __ldg(K.dn_ptr + dn + 1);
        bn = __ldg(K.bits_dn + dn);
      }
    }
    if (STAGE) xi = slab[d];
    else xi.ldg_pol(X + (r0 + d) * E, keep);
    const T dg = K.diag[__popc(bu & bd)];
#pragma unroll
    for (int e = 0; e < E; ++e) acc.v[e] = dg * xi.v[e];
    // up-spin hops (ascending u'), then the down-spin hops (ascending d')
    up_hops(acc, hop_ptr, hop_val, nh, d, keep);
    uint32_t j = j0;
    if constexpr (STAGE) {
      // entry = byte offset of the target row in the staged slab | sign bit
      const char* sb = reinterpret_cast<const char*>(slab);
      for (; j + 4 <= j1; j += 4) {
        uint32_t e4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) e4[q] = __ldg(K.dn_ent16 + j + q);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          axpy(acc, (e4[q] & 1u) ? K.dn_v1 : K.dn_v0, *reinterpret_cast<const V*>(sb + (e4[q] & 0xfff0u)));
      }
      for (; j < j1; ++j) {
        const uint32_t e1 = __ldg(K.dn_ent16 + j);
        axpy(acc, (e1 & 1u) ? K.dn_v1 : K.dn_v0, *reinterpret_cast<const V*>(sb + (e1 & 0xfff0u)));
      }
    } else {
      for (; j < j1; ++j) {
        const uint32_t e1 = __ldg(K.dn_ent + j);
        V w;
        w.ldg_pol(X + (r0 + (e1 & 0x7fffffffu)) * E, keep);
        axpy(acc, (e1 >> 31) ? K.dn_v1 : K.dn_v0, w);
      }
    }

    V y;
    if (MODE == MODE_SPMMV) {
#pragma unroll
      for (int e = 0; e < E; ++e) y.v[e] = s.c_ax * acc.v[e] + s.c_x * xi.v[e];
      y.st_pol(Ys + o, stream);
    } else {
      V out;
#pragma unroll
      for (int e = 0; e < E; ++e) y.v[e] = s.c_ax * acc.v[e] + s.c_x * xi.v[e] - z.v[e];
      if (MODE == MODE_SECOND) {
#pragma unroll
        for (int e = 0; e < E; ++e) out.v[e] = s.mu0 * z.v[e] + s.mu1 * xi.v[e] + s.mu2 * y.v[e];
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) out.v[e] = vin.v[e] + s.mu2 * y.v[e];
      }
      if (Ys) y.st_pol(Ys + o, stream);
      out.st_pol(Os + o, stream);
    }
  }
}

// Row-major D x nb block (ld) <-> np panels of D x 16 bytes, through a shared
// tile of 32 rows (reads and writes both coalesced; the tile row stride is
// np + 1 vectors so the transposed accesses spread over the banks)
template <typename T, bool TO_PANELS>
__global__ void k_panels(T* V, int64_t ldv, T* P, int64_t D, int np) {
  using Vv = V16<T>;
  constexpr int E = Vv::E;
  extern __shared__ __align__(16) unsigned char pt_smem[];
  Vv* tile = reinterpret_cast<Vv*>(pt_smem);
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int n = 32 * np;
  if (TO_PANELS) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int r = q / np, c = q - r * np;
      if (r0 + r < D) tile[r * (np + 1) + c].ldg(V + (r0 + r) * ldv + c * E);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int c = q / 32, r = q - c * 32;
      if (r0 + r < D) tile[r * (np + 1) + c].st(P + ((int64_t)c * D + r0 + r) * E);
    }
  } else {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int c = q / 32, r = q - c * 32;
      if (r0 + r < D) tile[r * (np + 1) + c].ldg(P + ((int64_t)c * D + r0 + r) * E);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int r = q / np, c = q - r * np;
      if (r0 + r < D) tile[r * (np + 1) + c].st(V + (r0 + r) * ldv + c * E);
    }
  }
}

template <typename T>
fd_status panels(fd_ctx* ctx, T* V, int64_t ldv, T* P, int64_t D, int np, bool to_panels) {
  const size_t smem = sizeof(V16<T>) * 32 * (size_t)(np + 1);
  const unsigned grid = (unsigned)cdiv(D, 32);
  if (to_panels) k_panels<T, true><<<grid, 256, smem, ctx->stream>>>(V, ldv, P, D, np);
  else k_panels<T, false><<<grid, 256, smem, ctx->stream>>>(V, ldv, P, D, np);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

template <typename T>
KronPanel<T> panel_args(const fd_ctx* ctx, const fd_matrix* M) {
  KronPanel<T> K;
  K.D = M->D;
  K.dim_up = (int)M->kdim[0];
  K.dim_dn = (int)M->kdim[1];
  const bool stage = (int64_t)K.dim_dn * 16 <= KP_STAGE_MAX && M->kdn_ent16;
  K.chunks = stage ? 1 : (int)cdiv(K.dim_dn, KP_ROWS_UNSTAGED);
  K.order = M->korder;
  K.bits_up = M->kbits[0];
  K.bits_dn = M->kbits[1];
  K.ptr_up = M->kptr[0];
  K.col_up = M->kcol[0];
  K.dn_ptr = M->kdn_ptr;
  K.dn_ent = M->kdn_ent;
  K.dn_ent16 = M->kdn_ent16;
  if constexpr (sizeof(T) == 8) {
    K.val_up = (const T*)M->kval[0];
    K.diag = (const T*)M->kdiag;
    K.dn_v0 = (T)M->kdn_val[0];
    K.dn_v1 = (T)M->kdn_val[1];
  } else {
    K.val_up = (const T*)M->kval32[0];
    K.diag = (const T*)M->kdiag32;
    K.dn_v0 = M->kdn_val32[0];
    K.dn_v1 = M->kdn_val32[1];
  }
  return K;
}

// shared-memory opt-in of the staged kernels, once per device and instantiation
constexpr int KP_MAX_DEVICES = 64;
bool g_kp_attr[KP_MAX_DEVICES][3] = {};

template <typename T, int MODE, bool STAGE>
fd_status launch_panel(fd_ctx* ctx, const KronPanel<T>& K, int np, const PanelStep<T>& s) {
  const size_t smem = STAGE ? (size_t)K.dim_dn * 16 : 0;
  if (STAGE && smem > 48 * 1024) {
    const int slot = MODE;
    if (ctx->device < 0 || ctx->device >= KP_MAX_DEVICES)
      return set_err(ctx, FD_ERR_ARG, "device ordinal %d out of range", ctx->device);
    if (!g_kp_attr[ctx->device][slot]) {
      FD_CUDA(ctx, cudaFuncSetAttribute(k_kron_panel<T, MODE, STAGE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KP_STAGE_MAX));
      // just the shared memory the resident CTAs need: the rest stays L1,
      // where the down-spin tables every CTA reads are kept
      const int carve = (int)cdiv(100LL * KP_MIN_BLOCKS * (KP_STAGE_MAX + 2048), 228LL * 1024);
      FD_CUDA(ctx, cudaFuncSetAttribute(k_kron_panel<T, MODE, STAGE>,
                                        cudaFuncAttributePreferredSharedMemoryCarveout, std::min(carve, 100)));
      g_kp_attr[ctx->device][slot] = true;
    }
  }
  const int64_t grid = (int64_t)np * K.dim_up * K.chunks;
  if (grid >= (1ll << 31)) return set_err(ctx, FD_ERR_ARG, "panel grid too large");
  k_kron_panel<T, MODE, STAGE><<<(unsigned)grid, KP_THREADS, smem, ctx->stream>>>(K, s);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

template <typename T>
fd_status panel_step(fd_ctx* ctx, const KronPanel<T>& K, int np, int mode, const PanelStep<T>& s) {
  if (K.chunks == 1) {
    if (mode == MODE_SPMMV) return launch_panel<T, MODE_SPMMV, true>(ctx, K, np, s);
    if (mode == MODE_SECOND) return launch_panel<T, MODE_SECOND, true>(ctx, K, np, s);
    return launch_panel<T, MODE_GENERIC, true>(ctx, K, np, s);
  }
  if (mode == MODE_SPMMV) return launch_panel<T, MODE_SPMMV, false>(ctx, K, np, s);
  if (mode == MODE_SECOND) return launch_panel<T, MODE_SECOND, false>(ctx, K, np, s);
  return launch_panel<T, MODE_GENERIC, false>(ctx, K, np, s);
}

// Alg. 2 on the panels: P0 holds x_0 and then the accumulated filter, P1 and
// P2 the two recurrence vectors; x_k overwrites x_{k-2} row by row, and the
// accumulator overwrites x_0 in the second step (same row, read first).
template <typename T>
fd_status kron_filter_t(fd_ctx* ctx, const fd_matrix* M, T* V, int64_t ldv, int nb, int n,
                        const double* mu, double alpha, double beta, T* W1, T* W2, int64_t ldw,
                        double* bytes_out) {
  constexpr int E = V16<T>::E;
  const int np = nb / E;
  const int64_t D = M->D;
  const size_t blk = sizeof(T) * (size_t)D * nb;
  T *P0, *P1, *P2;
  void* p;
  if (ldw == nb) {  // the caller's workspaces are contiguous: use them as panels
    FD_TRY(workspace(ctx, "kron_panels", blk, &p));
    P0 = (T*)p; P1 = W1; P2 = W2;
  } else {
    FD_TRY(workspace(ctx, "kron_panels", 3 * blk, &p));
    P0 = (T*)p; P1 = P0 + (size_t)D * nb; P2 = P1 + (size_t)D * nb;
  }
  const KronPanel<T> K = panel_args<T>(ctx, M);
  FD_TRY(panels<T>(ctx, V, ldv, P0, D, np, true));
  const double vec = (double)nb * D * sizeof(T);
  double bytes = 0;
  PanelStep<T> s{};
  s.X = P0; s.Y = P1; s.c_ax = (T)alpha; s.c_x = (T)beta;
  FD_TRY(panel_step<T>(ctx, K, np, MODE_SPMMV, s));
  bytes += 2 * vec;
  s = PanelStep<T>{};
  s.X = P1; s.Z = P0; s.Y = n > 2 ? P2 : nullptr; s.Vout = P0;
  s.c_ax = (T)(2 * alpha); s.c_x = (T)(2 * beta);
  s.mu0 = (T)mu[0]; s.mu1 = (T)mu[1]; s.mu2 = (T)mu[2];
  FD_TRY(panel_step<T>(ctx, K, np, MODE_SECOND, s));
  bytes += (n > 2 ? 4 : 3) * vec;
  T* xp = P2;   // x_{k-1}
  T* xpp = P1;  // x_{k-2}
  for (int k = 3; k <= n; ++k) {
    s = PanelStep<T>{};
    s.X = xp; s.Z = xpp; s.Vin = P0; s.Vout = P0;
    s.c_ax = (T)(2 * alpha); s.c_x = (T)(2 * beta); s.mu2 = (T)mu[k];
    s.Y = k < n ? xpp : nullptr;
    FD_TRY(panel_step<T>(ctx, K, np, MODE_GENERIC, s));
    bytes += (k < n ? 5 : 4) * vec;
    std::swap(xp, xpp);
  }
  FD_TRY(panels<T>(ctx, V, ldv, P0, D, np, false));
  if (bytes_out) *bytes_out += bytes;
  return FD_OK;
}

// ---- host: reverse Cuthill-McKee order of a symmetric graph (CSR) ----------
// Cuthill-McKee (1969) numbers the nodes breadth first from a start node,
// neighbours by increasing degree; reversing the order (George 1971) keeps the
// profile small.  The start node of each connected component is a
// pseudo-peripheral node found by repeated breadth-first searches (George and
// Liu 1979): from a node of smallest degree, move to a node of smallest degree
// in the last level while the number of levels grows.
std::vector<int32_t> rcm_order(int64_t n, const std::vector<int64_t>& ptr,
                               const std::vector<int32_t>& col) {
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<char> placed(n, 0);
  std::vector<int64_t> level(n, -1), seen_stamp(n, -1), queue;
  queue.reserve(n);
  auto deg = [&](int64_t v) { return ptr[v + 1] - ptr[v]; };
  int64_t stamp = 0;
  // breadth-first levels from r over unplaced nodes; returns the last level
  auto bfs = [&](int64_t r, std::vector<int64_t>* last) {
    ++stamp;
    queue.clear();
    queue.push_back(r);
    seen_stamp[r] = stamp;
    level[r] = 0;
    int64_t maxl = 0;
    for (size_t h = 0; h < queue.size(); ++h) {
      const int64_t v = queue[h];
      for (int64_t k = ptr[v]; k < ptr[v + 1]; ++k) {
        const int64_t w = col[k];
        if (placed[w] || seen_stamp[w] == stamp) continue;
        seen_stamp[w] = stamp;
        level[w] = level[v] + 1;
        maxl = std::max(maxl, level[w]);
        queue.push_back(w);
      }
    }
    last->clear();
    for (int64_t v : queue)
      if (level[v] == maxl) last->push_back(v);
    return maxl;
  };
  std::vector<int64_t> last, comp;
  for (int64_t s0 = 0; s0 < n; ++s0) {
    if (placed[s0]) continue;
    bfs(s0, &comp);
    comp.assign(queue.begin(), queue.end());
    int64_t r = *std::min_element(comp.begin(), comp.end(), [&](int64_t a, int64_t b) {
      return deg(a) != deg(b) ? deg(a) < deg(b) : a < b;
    });
    int64_t ecc = bfs(r, &last);
    for (int it = 0; it < 16; ++it) {
      const int64_t x = *std::min_element(last.begin(), last.end(), [&](int64_t a, int64_t b) {
        return deg(a) != deg(b) ? deg(a) < deg(b) : a < b;
      });
      std::vector<int64_t> last2;
      const int64_t e2 = bfs(x, &last2);
      if (e2 <= ecc) break;
      ecc = e2;
      r = x;
      last.swap(last2);
    }
    // Cuthill-McKee from r
    const size_t first = order.size();
    order.push_back((int32_t)r);
    placed[r] = 1;
    std::vector<int64_t> nbr;
    for (size_t h = first; h < order.size(); ++h) {
      const int64_t v = order[h];
      nbr.clear();
      for (int64_t k = ptr[v]; k < ptr[v + 1]; ++k)
        if (!placed[col[k]]) {
          placed[col[k]] = 1;
          nbr.push_back(col[k]);
        }
      std::sort(nbr.begin(), nbr.end(), [&](int64_t a, int64_t b) {
        return deg(a) != deg(b) ? deg(a) < deg(b) : a < b;
      });
      for (int64_t w : nbr) order.push_back((int32_t)w);
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

}  // namespace

fd_status kron_panel_tables(fd_ctx* ctx, fd_matrix* A, double t) {
  cudaStream_t st = ctx->stream;
  const int64_t du = A->kdim[0], dd = A->kdim[1];
  std::vector<int64_t> pu(du + 1), pd(dd + 1);
  FD_CUDA(ctx, cudaMemcpyAsync(pu.data(), A->kptr[0], sizeof(int64_t) * (du + 1), cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaMemcpyAsync(pd.data(), A->kptr[1], sizeof(int64_t) * (dd + 1), cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  std::vector<int32_t> cu(std::max<int64_t>(pu[du], 1)), cd(std::max<int64_t>(pd[dd], 1));
  std::vector<double> vd(std::max<int64_t>(pd[dd], 1));
  if (pu[du]) FD_CUDA(ctx, cudaMemcpyAsync(cu.data(), A->kcol[0], sizeof(int32_t) * pu[du], cudaMemcpyDeviceToHost, st));
  if (pd[dd]) {
    FD_CUDA(ctx, cudaMemcpyAsync(cd.data(), A->kcol[1], sizeof(int32_t) * pd[dd], cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaMemcpyAsync(vd.data(), A->kval[1], sizeof(double) * pd[dd], cudaMemcpyDeviceToHost, st));
  }
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  if (pd[dd] >= (1ll << 32) || dd >= (1ll << 31))
    return set_err(ctx, FD_ERR_ARG, "down-spin hop table too large for the panel kernel");
  int kmax = 0;
  for (int64_t u = 0; u < du; ++u) kmax = std::max<int>(kmax, (int)(pu[u + 1] - pu[u]));
  if (kmax > KP_MAX_HOPS) return set_err(ctx, FD_ERR_ARG, "%d up-spin hops exceed %d", kmax, KP_MAX_HOPS);
  A->kmax_up = kmax;
  // hop values: -t for fermion sign +1, +t for -1 (compared as bit patterns)
  const double v0 = -t * 1.0, v1 = -t * -1.0;
  std::vector<uint32_t> ptr32(dd + 1), ent(std::max<int64_t>(pd[dd], 1));
  for (int64_t d = 0; d <= dd; ++d) ptr32[d] = (uint32_t)pd[d];
  for (int64_t k = 0; k < pd[dd]; ++k) {
    uint32_t bit;
    if (std::memcmp(&vd[k], &v0, sizeof(double)) == 0) bit = 0;
    else if (std::memcmp(&vd[k], &v1, sizeof(double)) == 0) bit = 1;
    else return set_err(ctx, FD_ERR_ARG, "down-spin hop value %g is neither -t nor t", vd[k]);
    ent[k] = (uint32_t)cd[k] | (bit << 31);
  }
  A->kdn_val[0] = v0;
  A->kdn_val[1] = v1;
  A->kdn_val32[0] = (float)v0;
  A->kdn_val32[1] = (float)v1;
  const std::vector<int32_t> order = rcm_order(du, pu, cu);
  FD_CUDA(ctx, cudaMalloc(&A->korder, sizeof(int32_t) * std::max<int64_t>(du, 1)));
  FD_CUDA(ctx, cudaMalloc(&A->kdn_ptr, sizeof(uint32_t) * (dd + 1)));
  FD_CUDA(ctx, cudaMalloc(&A->kdn_ent, sizeof(uint32_t) * ent.size()));
  FD_CUDA(ctx, cudaMemcpyAsync(A->korder, order.data(), sizeof(int32_t) * du, cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(A->kdn_ptr, ptr32.data(), sizeof(uint32_t) * (dd + 1), cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(A->kdn_ent, ent.data(), sizeof(uint32_t) * ent.size(), cudaMemcpyHostToDevice, st));
  std::vector<uint16_t> ent16;
  if (dd * 16 <= KP_STAGE_MAX) {  // staged slabs: byte offset (target * 16) | sign bit
    ent16.resize(ent.size());
    for (size_t k = 0; k < ent.size(); ++k)
      ent16[k] = (uint16_t)(((ent[k] & 0x7fffffffu) << 4) | (ent[k] >> 31));
    FD_CUDA(ctx, cudaMalloc(&A->kdn_ent16, sizeof(uint16_t) * ent16.size()));
    FD_CUDA(ctx, cudaMemcpyAsync(A->kdn_ent16, ent16.data(), sizeof(uint16_t) * ent16.size(),
                                 cudaMemcpyHostToDevice, st));
  }
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  return FD_OK;
}

fd_status kron_filter(fd_ctx* ctx, const fd_matrix* M, fd_prec prec, void* V, int64_t ldv, int nb,
                      int degree, const double* mu, double alpha, double beta, void* W1, void* W2,
                      int64_t ldw, double* bytes_out) {
  // FP32 only: the FP64 step is bound by GB300's FP64 rate and keeps the
  // row-major matrix-free kernel
  if (prec != FD_F32) return set_err(ctx, FD_ERR_ARG, "the panel kernel runs FP32 sweeps only");
  return kron_filter_t<float>(ctx, M, (float*)V, ldv, nb, degree, mu, alpha, beta, (float*)W1,
                              (float*)W2, ldw, bytes_out);
}

}  // namespace fdi
