// Context, error plumbing, matrix generators (Hubbard, 3D Anderson, chain),
// CSR import, SELL-C-sigma construction and bit-exact CSR export.
//
// Paper: Alvermann, Hager, Fehske, arXiv 2209.01974.  The Hubbard and
// stencil-like matrices are the test matrices of Sec. 3.2 (Table 2) and
// Sec. 4.1 (D = C(n_sites, n_fermions)^2); SELL-C-sigma is the sparse format
// of the GHOST library the paper's kernels use (Kreutzer et al. 2014).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "fd_internal.cuh"

namespace fdi {

fd_status set_err(fd_ctx* ctx, fd_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return st;
}

fd_status workspace(fd_ctx* ctx, const char* name, size_t bytes, void** out) {
  auto& e = ctx->ws[name];
  if (e.second < bytes) {
    size_t b = std::max<size_t>(bytes, 256);
    // a context-level cap (fd_set_workspace_limit) refuses the growth before
    // anything is freed or allocated, exactly like a failed cudaMalloc
    if (ctx->ws_limit && ctx->ws_bytes - e.second + b > ctx->ws_limit)
      return set_err(ctx, FD_ERR_OOM, "workspace '%s' of %zu bytes exceeds the context's limit of %zu bytes",
                     name, b, ctx->ws_limit);
    if (e.first) {
      // the old buffer may still be used by queued work on the stream
      FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      FD_CUDA(ctx, cudaFree(e.first));
      ctx->ws_bytes -= e.second;
      e.first = nullptr;
      e.second = 0;
    }
    void* p = nullptr;
    cudaError_t err = cudaMalloc(&p, b);
    ctx->ws_allocs++;
    if (err != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, FD_ERR_OOM, "cudaMalloc of %zu bytes for workspace '%s' failed: %s",
                     b, name, cudaGetErrorString(err));
    }
    e.first = p;
    e.second = b;
    ctx->ws_bytes += b;
  }
  *out = e.first;
  return FD_OK;
}

fd_status host_stage(fd_ctx* ctx, size_t bytes, void** out) {
  if (ctx->host_stage_bytes < bytes) {
    if (ctx->host_stage) {
      FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      cudaFreeHost(ctx->host_stage);
    }
    ctx->host_stage = nullptr;
    ctx->host_stage_bytes = 0;
    FD_CUDA(ctx, cudaMallocHost(&ctx->host_stage, bytes));
    ctx->host_stage_bytes = bytes;
  }
  *out = ctx->host_stage;
  return FD_OK;
}

// ---------------------------------------------------------------------------
// int64 exclusive scan (three phases; deterministic)
// ---------------------------------------------------------------------------
namespace {
constexpr int SCAN_B = 1024;

__device__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total) {
  // warp-level inclusive scan, then scan of warp sums
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;  // inclusive scan of warp sums
  }
  __syncthreads();
  int64_t pre = (w > 0) ? sh[w - 1] : 0;
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  return pre + x - v;
}

__global__ void k_scan_blocks(const int64_t* in, int64_t n, int64_t* out, int64_t* bsum) {
  __shared__ int64_t sh[32];
  int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  int64_t tot;
  int64_t ex = block_exclusive_scan(v, sh, &tot);
  if (i < n) out[i] = ex;
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* bsum, int64_t nb, int64_t* grand) {
  __shared__ int64_t sh[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += SCAN_B) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    int64_t ex = block_exclusive_scan(v, sh, &tot);
    if (i < nb) bsum[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* bsum) {
  int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
}
}  // namespace

// out[i] = sum_{j<i} in[i] for i < n, out[n] = total (out has n+1 slots)
static fd_status exclusive_scan(fd_ctx* ctx, const int64_t* in, int64_t n, int64_t* out) {
  int64_t nb = std::max<int64_t>(1, cdiv(n, SCAN_B));
  void* ws;
  FD_TRY(workspace(ctx, "scan", sizeof(int64_t) * (nb + 1), &ws));
  int64_t* bsum = (int64_t*)ws;
  k_scan_blocks<<<(unsigned)nb, SCAN_B, 0, ctx->stream>>>(in, n, out, bsum);
  FD_LAUNCHED(ctx);
  k_scan_sums<<<1, SCAN_B, 0, ctx->stream>>>(bsum, nb, out + n);
  FD_LAUNCHED(ctx);
  k_scan_add<<<(unsigned)nb, SCAN_B, 0, ctx->stream>>>(out, n, bsum);
  FD_LAUNCHED(ctx);
  return FD_OK;
}

// ---------------------------------------------------------------------------
// generators
// ---------------------------------------------------------------------------
namespace {

struct HubbardP {
  int L, Nu, Nd, periodic;
  int64_t dim_up, dim_dn, D;
  double t, U;
};

__host__ __device__ inline int64_t binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  int64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// combinatorial number system: the rank of a bitstring among all bitstrings
// with the same popcount, in increasing integer order
__device__ inline int64_t comb_rank(uint32_t s) {
  int64_t r = 0;
  int i = 1;
  while (s) {
    int c = __ffs(s) - 1;
    r += binom(c, i);
    ++i;
    s &= s - 1;
  }
  return r;
}

__device__ inline uint32_t comb_unrank(int64_t r, int N, int L) {
  uint32_t s = 0;
  int c = L - 1;
  for (int i = N; i >= 1; --i) {
    while (binom(c, i) > r) --c;
    r -= binom(c, i);
    s |= 1u << c;
    --c;
  }
  return s;
}

constexpr int HUB_MAX_ENTRIES = 1 + 2 * 2 * 24;

// entries of row `row`; returns count, writes (col, val) unsorted
__device__ int hubbard_row(const HubbardP& p, int64_t row, int64_t* cols, double* vals) {
  int64_t ru = row / p.dim_dn, rd = row % p.dim_dn;
  uint32_t su = comb_unrank(ru, p.Nu, p.L), sd = comb_unrank(rd, p.Nd, p.L);
  int n = 0;
  cols[n] = row;
  vals[n] = __dmul_rn(p.U, (double)__popc(su & sd));
  ++n;
  int nb = p.L - 1 + (p.periodic ? 1 : 0);
  for (int b = 0; b < nb; ++b) {
    int i = b < p.L - 1 ? b : 0;
    int j = b < p.L - 1 ? b + 1 : p.L - 1;
    uint32_t between = ((1u << j) - 1u) ^ ((1u << (i + 1)) - 1u);
    uint32_t flip = (1u << i) | (1u << j);
    for (int spin = 0; spin < 2; ++spin) {
      uint32_t s = spin == 0 ? su : sd;
      if ((((s >> i) ^ (s >> j)) & 1u) == 0) continue;
      uint32_t s2 = s ^ flip;
      double sign = (__popc(s & between) & 1) ? -1.0 : 1.0;
      int64_t col = spin == 0 ? comb_rank(s2) * p.dim_dn + rd : ru * p.dim_dn + comb_rank(s2);
      cols[n] = col;
      vals[n] = -p.t * sign;
      ++n;
    }
  }
  return n;
}

__device__ inline void sort_entries(int64_t* c, double* v, int n) {
  for (int a = 1; a < n; ++a) {
    int64_t kc = c[a];
    double kv = v[a];
    int b = a - 1;
    while (b >= 0 && c[b] > kc) {
      c[b + 1] = c[b];
      v[b + 1] = v[b];
      --b;
    }
    c[b + 1] = kc;
    v[b + 1] = kv;
  }
}

__global__ void k_hubbard_count(HubbardP p, int64_t* cnt) {
  int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= p.D) return;
  int64_t cols[HUB_MAX_ENTRIES];
  double vals[HUB_MAX_ENTRIES];
  cnt[row] = hubbard_row(p, row, cols, vals);
}

// single-species tables of the matrix-free Hubbard operator: the hopping of
// N particles of one spin on L sites, bonds and signs as in hubbard_row
__device__ int kron_hops(int L, int N, int periodic, double t, int64_t r, int64_t* cols, double* vals,
                         uint32_t* bits) {
  const uint32_t s = comb_unrank(r, N, L);
  *bits = s;
  int n = 0;
  const int nbond = L - 1 + (periodic ? 1 : 0);
  for (int b = 0; b < nbond; ++b) {
    const int i = b < L - 1 ? b : 0;
    const int j = b < L - 1 ? b + 1 : L - 1;
    if ((((s >> i) ^ (s >> j)) & 1u) == 0) continue;
    const uint32_t between = ((1u << j) - 1u) ^ ((1u << (i + 1)) - 1u);
    const uint32_t s2 = s ^ ((1u << i) | (1u << j));
    cols[n] = comb_rank(s2);
    vals[n] = -t * ((__popc(s & between) & 1) ? -1.0 : 1.0);
    ++n;
  }
  return n;
}

__global__ void k_kron_count(int L, int N, int periodic, double t, int64_t dim, int64_t* cnt, uint32_t* bits) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= dim) return;
  int64_t c[24];
  double v[24];
  cnt[r] = kron_hops(L, N, periodic, t, r, c, v, bits + r);
}

__global__ void k_kron_fill(int L, int N, int periodic, double t, int64_t dim, const int64_t* ptr,
                            int32_t* col, double* val, float* val32) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= dim) return;
  int64_t c[24];
  double v[24];
  uint32_t bits;
  const int n = kron_hops(L, N, periodic, t, r, c, v, &bits);
  sort_entries(c, v, n);
  const int64_t o = ptr[r];
  for (int k = 0; k < n; ++k) {
    col[o + k] = (int32_t)c[k];
    val[o + k] = v[k];
    val32[o + k] = (float)v[k];
  }
}

// float-float copy of the values: hi the nearest float, lo the nearest float
// to the remainder (exact in FP64), so hi + lo is within 2^-48 of the value
__global__ void k_split_ff(const double* val, int64_t n, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = val[i];
  const float hi = __double2float_rn(v);
  out[2 * i] = hi;
  out[2 * i + 1] = __double2float_rn(v - (double)hi);
}

__global__ void k_hubbard_fill(HubbardP p, const int64_t* rowptr, int32_t* col, double* val) {
  int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= p.D) return;
  int64_t cols[HUB_MAX_ENTRIES];
  double vals[HUB_MAX_ENTRIES];
  int n = hubbard_row(p, row, cols, vals);
  sort_entries(cols, vals, n);
  int64_t o = rowptr[row];
  for (int k = 0; k < n; ++k) {
    col[o + k] = (int32_t)cols[k];
    val[o + k] = vals[k];
  }
}

struct AndersonP {
  int64_t L, D;
  double W, t;
  uint64_t key;
};

__global__ void k_anderson_fill(AndersonP p, int64_t* rowptr, int32_t* col, double* val) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= p.D) return;
  int64_t L = p.L;
  int64_t x = r % L, y = (r / L) % L, z = r / (L * L);
  auto idx = [L](int64_t a, int64_t b, int64_t c) { return a + L * (b + L * c); };
  int64_t cols[7] = {r,
                     idx((x + 1) % L, y, z), idx((x + L - 1) % L, y, z),
                     idx(x, (y + 1) % L, z), idx(x, (y + L - 1) % L, z),
                     idx(x, y, (z + 1) % L), idx(x, y, (z + L - 1) % L)};
  double vals[7];
  double u = fdrng::uniform(p.key, (uint64_t)r);
  vals[0] = __dmul_rn(p.W, __dsub_rn(u, 0.5));
  for (int k = 1; k < 7; ++k) vals[k] = -p.t;
  sort_entries(cols, vals, 7);
  int64_t o = 7 * r;
  for (int k = 0; k < 7; ++k) {
    col[o + k] = (int32_t)cols[k];
    val[o + k] = vals[k];
  }
  rowptr[r] = o;
  if (r == p.D - 1) rowptr[p.D] = 7 * p.D;
}

// road-like planar graph (see fd_build_matrix): edges of node i to its left
// and lower neighbours; the right and upper edges belong to those neighbours
struct RoadP {
  int64_t side, N;
  double q;
  uint64_t ktree, kextra;
};

__device__ inline void road_own_edges(const RoadP& p, int64_t i, bool* left, bool* down) {
  const int64_t x = i % p.side, y = i / p.side;
  const double u = fdrng::uniform(p.ktree, (uint64_t)i);
  const bool pl = (y == 0 && x > 0) || (y > 0 && x > 0 && u < 0.5);
  const bool pd = y > 0 && (x == 0 || u >= 0.5);
  *left = pl || (x > 0 && !pl && fdrng::uniform(p.kextra, (uint64_t)(2 * i)) < p.q);
  *down = pd || (y > 0 && !pd && fdrng::uniform(p.kextra, (uint64_t)(2 * i + 1)) < p.q);
}

// neighbours of node i in ascending order: down, left, (self), right, up
__device__ inline int road_neighbours(const RoadP& p, int64_t i, int64_t* nb) {
  bool l, d, rl = false, ud = false, dummy;
  road_own_edges(p, i, &l, &d);
  const int64_t x = i % p.side, y = i / p.side;
  if (x + 1 < p.side) road_own_edges(p, i + 1, &rl, &dummy);
  if (y + 1 < p.side) road_own_edges(p, i + p.side, &dummy, &ud);
  int n = 0;
  if (d) nb[n++] = i - p.side;
  if (l) nb[n++] = i - 1;
  if (rl) nb[n++] = i + 1;
  if (ud) nb[n++] = i + p.side;
  return n;
}

__global__ void k_road_count(RoadP p, int64_t* cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  int64_t nb[4];
  cnt[i] = 1 + road_neighbours(p, i, nb);
}

__global__ void k_road_fill(RoadP p, const int64_t* rowptr, int32_t* col, double* val) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  int64_t nb[4];
  const int n = road_neighbours(p, i, nb);
  int64_t o = rowptr[i];
  int k = 0;
  for (; k < n && nb[k] < i; ++k) { col[o] = (int32_t)nb[k]; val[o] = -1.0; ++o; }
  col[o] = (int32_t)i; val[o] = (double)n; ++o;
  for (; k < n; ++k) { col[o] = (int32_t)nb[k]; val[o] = -1.0; ++o; }
}

__global__ void k_chain_fill(int64_t n, double t, int64_t* rowptr, int32_t* col, double* val) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  // row r: [r-1] -t, [r] 0, [r+1] -t ; offsets: row 0 has 2 entries, others 3 (last 2)
  int64_t o = r == 0 ? 0 : 3 * r - 1;
  int k = 0;
  if (r > 0) { col[o + k] = (int32_t)(r - 1); val[o + k] = -t; ++k; }
  col[o + k] = (int32_t)r; val[o + k] = 0.0; ++k;
  if (r + 1 < n) { col[o + k] = (int32_t)(r + 1); val[o + k] = -t; ++k; }
  rowptr[r] = o;
  if (r == n - 1) rowptr[n] = o + k;
}

// ---------------------------------------------------------------------------
// SELL-C-sigma construction
// ---------------------------------------------------------------------------

// per original row: SELL length (diagonal always present), diag-added flag,
// and the Gershgorin disc ends
__global__ void k_row_info(const int64_t* rowptr, const int32_t* col, const double* val,
                           int64_t D, int32_t* len, uint8_t* added, double* glo,
                           double* ghi, int* bad) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D) return;
  int64_t s = rowptr[r], e = rowptr[r + 1];
  bool has = false;
  double d = 0.0, rad = 0.0;
  int32_t prev = -1;
  for (int64_t k = s; k < e; ++k) {
    int32_t c = col[k];
    if (c < 0 || c >= D || c <= prev) *bad = 1;  // bounds/ordering check, no fault
    prev = c;
    if (c == r) { has = true; d = val[k]; }
    else rad += fabs(val[k]);
  }
  len[r] = (int32_t)(e - s) + (has ? 0 : 1);
  added[r] = has ? 0 : 1;
  glo[r] = d - rad;
  ghi[r] = d + rad;
}

// stable descending sort of row lengths within windows of sigma rows
__global__ void k_sigma_rank(const int32_t* len, int64_t D, int sigma, int64_t* perm,
                             int64_t* iperm) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D) return;
  int64_t w0 = (r / sigma) * sigma, w1 = min(D, w0 + sigma);
  int32_t lr = len[r];
  int64_t rank = 0;
  for (int64_t q = w0; q < w1; ++q) {
    int32_t lq = len[q];
    rank += (lq > lr) || (lq == lr && q < r);
  }
  perm[w0 + rank] = r;
  iperm[r] = w0 + rank;
}

__global__ void k_identity_perm(int64_t D, int64_t* perm, int64_t* iperm) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < D) { perm[r] = r; iperm[r] = r; }
}

// chunk lengths (in entries = C * max row length) and SELL-order row lengths
__global__ void k_chunk_len(const int32_t* len, const int64_t* perm, const uint8_t* added,
                            int64_t D, int C, int64_t n_chunks, int64_t* chunk_sz,
                            int32_t* row_len, uint8_t* added_sell) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  int32_t m = 0;
  for (int r = 0; r < C; ++r) {
    int64_t i = c * C + r;
    int32_t l = 0;
    if (i < D) {
      l = len[perm[i]];
      added_sell[i] = added[perm[i]];
    }
    row_len[i] = l;
    m = max(m, l);
  }
  // chunk length rounded up to a multiple of 8 entries: the SpMMV kernels take
  // entries in batches of 8 without per-entry predicates
  m = (m + 7) & ~7;
  chunk_sz[c] = (int64_t)m * C;
}

__global__ void k_sell_fill(const int64_t* rowptr, const int32_t* col, const double* val,
                            const int64_t* perm, const int64_t* iperm, const int64_t* chunk_ptr,
                            const int32_t* row_len, int64_t D, int C, int64_t n_chunks,
                            int32_t* scol, double* sval, float* sval32) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_chunks * C) return;
  int64_t c = i / C, rr = i % C;
  int64_t base = chunk_ptr[c] + rr;
  int32_t clen = (int32_t)((chunk_ptr[c + 1] - chunk_ptr[c]) / C);
  int j = 0;
  if (i < D) {
    int64_t r = perm[i];
    int64_t s = rowptr[r], e = rowptr[r + 1];
    double d = 0.0;
    for (int64_t k = s; k < e; ++k)
      if (col[k] == r) d = val[k];
    scol[base] = (int32_t)i;
    sval[base] = d;
    sval32[base] = (float)d;
    j = 1;
    for (int64_t k = s; k < e; ++k) {
      if (col[k] == r) continue;
      int64_t o = base + (int64_t)j * C;
      scol[o] = (int32_t)iperm[col[k]];
      sval[o] = val[k];
      sval32[o] = (float)val[k];
      ++j;
    }
  }
  // padding: zero value, own row (row ids beyond D point at row 0)
  int32_t own = i < D ? (int32_t)i : 0;
  for (; j < clen; ++j) {
    int64_t o = base + (int64_t)j * C;
    scol[o] = own;
    sval[o] = 0.0;
    sval32[o] = 0.0f;
  }
  (void)row_len;
}

__global__ void k_minmax_partial(const double* lo, const double* hi, const int32_t* len,
                                 int64_t D, double* out_lo, double* out_hi, int* out_len) {
  __shared__ double slo[256], shi[256];
  __shared__ int sl[256];
  double a = INFINITY, b = -INFINITY;
  int m = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < D;
       r += (int64_t)gridDim.x * blockDim.x) {
    a = fmin(a, lo[r]);
    b = fmax(b, hi[r]);
    m = max(m, len[r]);
  }
  slo[threadIdx.x] = a; shi[threadIdx.x] = b; sl[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + o]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + o]);
      sl[threadIdx.x] = max(sl[threadIdx.x], sl[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out_lo[blockIdx.x] = slo[0];
    out_hi[blockIdx.x] = shi[0];
    out_len[blockIdx.x] = sl[0];
  }
}

// ---- export ---------------------------------------------------------------
__global__ void k_export_len(const int64_t* perm, const int32_t* row_len, const uint8_t* added,
                             int64_t D, int64_t* cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D) return;
  cnt[perm[i]] = row_len[i] - added[i];
}

__global__ void k_export_fill(const int64_t* perm, const int32_t* row_len, const uint8_t* added,
                              const int64_t* chunk_ptr, const int32_t* scol, const double* sval,
                              int64_t D, int C, const int64_t* rowptr, int32_t* col,
                              double* val) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D) return;
  int64_t r = perm[i];
  int64_t base = chunk_ptr[i / C] + i % C;
  int32_t len = row_len[i];
  int64_t o = rowptr[r];
  double dval = sval[base];
  bool diag_done = added[i] != 0;
  for (int j = 1; j < len; ++j) {
    int64_t c = perm[scol[base + (int64_t)j * C]];
    if (!diag_done && c > r) {
      col[o] = (int32_t)r; val[o] = dval; ++o;
      diag_done = true;
    }
    col[o] = (int32_t)c;
    val[o] = sval[base + (int64_t)j * C];
    ++o;
  }
  if (!diag_done) { col[o] = (int32_t)r; val[o] = dval; }
}

}  // namespace

fd_status sell_from_device_csr(fd_ctx* ctx, fd_matrix* A, const int64_t* d_rowptr,
                               const int32_t* d_col, const double* d_val, int64_t nnz) {
  cudaStream_t st = ctx->stream;
  const int64_t D = A->D;
  const int C = A->C;
  const int T = 256;
  A->nnz = nnz;
  A->n_chunks = cdiv(D, C);
  const int64_t nrows_pad = A->n_chunks * C;

  int32_t* len;
  uint8_t* added;
  double *glo, *ghi;
  int* bad;
  int64_t* chunk_sz;
  void* p;
  FD_TRY(workspace(ctx, "build_len", sizeof(int32_t) * D, &p)); len = (int32_t*)p;
  FD_TRY(workspace(ctx, "build_added", D, &p)); added = (uint8_t*)p;
  FD_TRY(workspace(ctx, "build_glo", sizeof(double) * D, &p)); glo = (double*)p;
  FD_TRY(workspace(ctx, "build_ghi", sizeof(double) * D, &p)); ghi = (double*)p;
  FD_TRY(workspace(ctx, "build_bad", sizeof(int) * 4, &p)); bad = (int*)p;
  FD_TRY(workspace(ctx, "build_chunksz", sizeof(int64_t) * (A->n_chunks + 1), &p));
  chunk_sz = (int64_t*)p;

  FD_CUDA(ctx, cudaMalloc(&A->perm, sizeof(int64_t) * D));
  FD_CUDA(ctx, cudaMalloc(&A->iperm, sizeof(int64_t) * D));
  FD_CUDA(ctx, cudaMalloc(&A->row_len, sizeof(int32_t) * nrows_pad));
  FD_CUDA(ctx, cudaMalloc(&A->diag_added, nrows_pad));
  FD_CUDA(ctx, cudaMalloc(&A->chunk_ptr, sizeof(int64_t) * (A->n_chunks + 1)));

  FD_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_row_info<<<(unsigned)cdiv(D, T), T, 0, st>>>(d_rowptr, d_col, d_val, D, len, added, glo,
                                                 ghi, bad);
  FD_LAUNCHED(ctx);
  if (A->sigma <= 1) {
    k_identity_perm<<<(unsigned)cdiv(D, T), T, 0, st>>>(D, A->perm, A->iperm);
    A->identity = 1;
  } else {
    k_sigma_rank<<<(unsigned)cdiv(D, T), T, 0, st>>>(len, D, A->sigma, A->perm, A->iperm);
    A->identity = 0;
  }
  FD_LAUNCHED(ctx);
  FD_CUDA(ctx, cudaMemsetAsync(A->diag_added, 0, nrows_pad, st));
  k_chunk_len<<<(unsigned)cdiv(A->n_chunks, T), T, 0, st>>>(len, A->perm, added, D, C,
                                                            A->n_chunks, chunk_sz, A->row_len,
                                                            A->diag_added);
  FD_LAUNCHED(ctx);
  FD_TRY(exclusive_scan(ctx, chunk_sz, A->n_chunks, A->chunk_ptr));
  int64_t nnz_sell = 0;
  int hbad = 0;
  FD_CUDA(ctx, cudaMemcpyAsync(&nnz_sell, A->chunk_ptr + A->n_chunks, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  if (hbad) return set_err(ctx, FD_ERR_BOUNDS, "CSR column index out of range or not ascending");
  A->nnz_sell = nnz_sell;
  FD_CUDA(ctx, cudaMalloc(&A->col, sizeof(int32_t) * std::max<int64_t>(1, nnz_sell)));
  FD_CUDA(ctx, cudaMalloc(&A->val, sizeof(double) * std::max<int64_t>(1, nnz_sell)));
  FD_CUDA(ctx, cudaMalloc(&A->val32, sizeof(float) * std::max<int64_t>(1, nnz_sell)));
  k_sell_fill<<<(unsigned)cdiv(nrows_pad, T), T, 0, st>>>(
      d_rowptr, d_col, d_val, A->perm, A->iperm, A->chunk_ptr, A->row_len, D, C, A->n_chunks,
      A->col, A->val, A->val32);
  FD_LAUNCHED(ctx);
  FD_CUDA(ctx, cudaMalloc(&A->valff, 2 * sizeof(float) * std::max<int64_t>(1, nnz_sell)));
  if (nnz_sell > 0) {
    k_split_ff<<<(unsigned)cdiv(nnz_sell, T), T, 0, st>>>(A->val, nnz_sell, A->valff);
    FD_LAUNCHED(ctx);
  }

  // Gershgorin interval and longest row
  const int PB = 256;
  double *plo, *phi;
  int* plen;
  FD_TRY(workspace(ctx, "build_red", (sizeof(double) * 2 + sizeof(int)) * PB, &p));
  plo = (double*)p; phi = plo + PB; plen = (int*)(phi + PB);
  k_minmax_partial<<<PB, 256, 0, st>>>(glo, ghi, len, D, plo, phi, plen);
  FD_LAUNCHED(ctx);
  std::vector<double> hlo(PB), hhi(PB);
  std::vector<int> hl(PB);
  FD_CUDA(ctx, cudaMemcpyAsync(hlo.data(), plo, sizeof(double) * PB, cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaMemcpyAsync(hhi.data(), phi, sizeof(double) * PB, cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaMemcpyAsync(hl.data(), plen, sizeof(int) * PB, cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  A->gersh_lo = INFINITY; A->gersh_hi = -INFINITY; A->max_row = 0;
  for (int b = 0; b < PB; ++b) {
    A->gersh_lo = std::min(A->gersh_lo, hlo[b]);
    A->gersh_hi = std::max(A->gersh_hi, hhi[b]);
    A->max_row = std::max(A->max_row, hl[b]);
  }
  return FD_OK;
}

}  // namespace fdi

using namespace fdi;

// ---------------------------------------------------------------------------
// spec parsing
// ---------------------------------------------------------------------------
namespace {
struct Spec {
  std::string kind;
  std::vector<std::pair<std::string, std::string>> kv;
  const char* get(const char* k) const {
    for (auto& p : kv)
      if (p.first == k) return p.second.c_str();
    return nullptr;
  }
};

bool parse_spec(const char* s, Spec* out) {
  std::string str(s);
  size_t colon = str.find(':');
  out->kind = str.substr(0, colon);
  if (colon == std::string::npos) return !out->kind.empty();
  std::string rest = str.substr(colon + 1);
  size_t pos = 0;
  while (pos < rest.size()) {
    size_t comma = rest.find(',', pos);
    std::string item = rest.substr(pos, comma == std::string::npos ? std::string::npos : comma - pos);
    size_t eq = item.find('=');
    if (eq == std::string::npos) return false;
    out->kv.emplace_back(item.substr(0, eq), item.substr(eq + 1));
    if (comma == std::string::npos) break;
    pos = comma + 1;
  }
  return true;
}

bool get_int(const Spec& s, const char* k, long long* v, bool required, long long def) {
  const char* p = s.get(k);
  if (!p) { *v = def; return !required; }
  char* end;
  *v = strtoll(p, &end, 10);
  return *end == '\0';
}
bool get_dbl(const Spec& s, const char* k, double* v, double def) {
  const char* p = s.get(k);
  if (!p) { *v = def; return true; }
  char* end;
  *v = strtod(p, &end);
  return *end == '\0';
}

fd_status finish_build(fd_ctx* ctx, fd_matrix* A, int64_t* rowptr, int32_t* col, double* val,
                       int64_t nnz, fd_matrix** out) {
  fd_status st = sell_from_device_csr(ctx, A, rowptr, col, val, nnz);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(rowptr);
  cudaFree(col);
  cudaFree(val);
  if (st != FD_OK) {
    fd_matrix_free(A);
    return st;
  }
  *out = A;
  return FD_OK;
}
}  // namespace

extern "C" {

fd_status fd_create(fd_ctx** out, int device, void* stream) {
  if (!out) return FD_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return FD_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return FD_ERR_CUDA;
  fd_ctx* c = new fd_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = optin;
  *out = c;
  return FD_OK;
}

fd_status fd_destroy(fd_ctx* ctx) {
  if (!ctx) return FD_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& e : ctx->ws)
    if (e.second.first) cudaFree(e.second.first);
  if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
  delete ctx;
  return FD_OK;
}

fd_status fd_set_stream(fd_ctx* ctx, void* stream) {
  if (!ctx) return FD_ERR_ARG;
  ctx->stream = (cudaStream_t)stream;
  return FD_OK;
}

const char* fd_last_error(const fd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t fd_kernel_launches(const fd_ctx* ctx) { return ctx ? ctx->launches : -1; }

fd_status fd_workspace_info(const fd_ctx* ctx, size_t* bytes_held, int64_t* allocations) {
  if (!ctx) return FD_ERR_ARG;
  if (bytes_held) *bytes_held = ctx->ws_bytes;
  if (allocations) *allocations = ctx->ws_allocs;
  return FD_OK;
}

fd_status fd_set_workspace_limit(fd_ctx* ctx, size_t limit_bytes) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  ctx->ws_limit = limit_bytes;
  return FD_OK;
}

// the per-species tables of the matrix-free Hubbard operator on A
static fd_status build_kron(fd_ctx* ctx, fd_matrix* A, const HubbardP& p) {
  cudaStream_t st = ctx->stream;
  const int T = 256;
  for (int sp = 0; sp < 2; ++sp) {
    const int N = sp == 0 ? p.Nu : p.Nd;
    const int64_t dim = sp == 0 ? p.dim_up : p.dim_dn;
    A->kdim[sp] = dim;
    int64_t* cnt;
    FD_CUDA(ctx, cudaMalloc(&A->kbits[sp], sizeof(uint32_t) * dim));
    FD_CUDA(ctx, cudaMalloc(&A->kptr[sp], sizeof(int64_t) * (dim + 1)));
    FD_CUDA(ctx, cudaMalloc(&cnt, sizeof(int64_t) * dim));
    k_kron_count<<<(unsigned)cdiv(dim, T), T, 0, st>>>(p.L, N, p.periodic, p.t, dim, cnt, A->kbits[sp]);
    FD_LAUNCHED(ctx);
    FD_TRY(exclusive_scan(ctx, cnt, dim, A->kptr[sp]));
    int64_t nh = 0;
    FD_CUDA(ctx, cudaMemcpyAsync(&nh, A->kptr[sp] + dim, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaStreamSynchronize(st));
    cudaFree(cnt);
    const size_t m = (size_t)std::max<int64_t>(nh, 1);
    FD_CUDA(ctx, cudaMalloc(&A->kcol[sp], sizeof(int32_t) * m));
    FD_CUDA(ctx, cudaMalloc(&A->kval[sp], sizeof(double) * m));
    FD_CUDA(ctx, cudaMalloc(&A->kval32[sp], sizeof(float) * m));
    k_kron_fill<<<(unsigned)cdiv(dim, T), T, 0, st>>>(p.L, N, p.periodic, p.t, dim, A->kptr[sp], A->kcol[sp],
                                                      A->kval[sp], A->kval32[sp]);
    FD_LAUNCHED(ctx);
    FD_CUDA(ctx, cudaMalloc(&A->kvalff[sp], 2 * sizeof(float) * m));
    if (nh > 0) {
      k_split_ff<<<(unsigned)cdiv(nh, T), T, 0, st>>>(A->kval[sp], nh, A->kvalff[sp]);
      FD_LAUNCHED(ctx);
    }
  }
  double dg[25];
  float dg32[25], dgff[50];
  for (int n = 0; n <= 24; ++n) {
    dg[n] = p.U * (double)n;  // the generator's U * popcount
    dg32[n] = (float)dg[n];   // as the FP32 copy of the stored values
    dgff[2 * n] = dg32[n];    // and the float-float split of the FP64 value
    dgff[2 * n + 1] = (float)(dg[n] - (double)dg32[n]);
  }
  FD_CUDA(ctx, cudaMalloc(&A->kdiag, sizeof(dg)));
  FD_CUDA(ctx, cudaMalloc(&A->kdiag32, sizeof(dg32)));
  FD_CUDA(ctx, cudaMalloc(&A->kdiagff, sizeof(dgff)));
  FD_CUDA(ctx, cudaMemcpyAsync(A->kdiag, dg, sizeof(dg), cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(A->kdiag32, dg32, sizeof(dg32), cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaMemcpyAsync(A->kdiagff, dgff, sizeof(dgff), cudaMemcpyHostToDevice, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  FD_TRY(kron_panel_tables(ctx, A, p.t));
  A->kron = 1;
  return FD_OK;
}

fd_status fd_build_matrix(fd_ctx* ctx, const char* spec, fd_matrix** out) {
  return fd_build_matrix_sell(ctx, spec, 32, 1, out);
}

fd_status fd_build_matrix_sell(fd_ctx* ctx, const char* spec, int C, int sigma,
                               fd_matrix** out) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!spec || !out) return set_err(ctx, FD_ERR_ARG, "null spec or output");
  *out = nullptr;
  if (C < 32 || C % 32 != 0 || C > 1024 || sigma < 1 || sigma > 65536)
    return set_err(ctx, FD_ERR_ARG, "C must be a multiple of 32 in [32, 1024], sigma in [1, 65536]");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  Spec s;
  if (!parse_spec(spec, &s)) return set_err(ctx, FD_ERR_ARG, "cannot parse spec '%s'", spec);
  const int T = 256;
  cudaStream_t st = ctx->stream;
  fd_matrix* A = new fd_matrix();
  A->ctx = ctx;
  A->device = ctx->device;
  A->C = C;
  A->sigma = sigma;
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  int64_t nnz = 0;
  bool kron_flag = false;
  HubbardP hub{};

  if (s.kind == "hubbard") {
    long long L, nu, nd;
    double t, U;
    if (!get_int(s, "n_sites", &L, true, 0) || !get_int(s, "n_up", &nu, true, 0) ||
        !get_int(s, "n_dn", &nd, true, 0) || !get_dbl(s, "t", &t, 1.0) || !get_dbl(s, "U", &U, 4.0)) {
      delete A;
      return set_err(ctx, FD_ERR_ARG, "hubbard needs integer n_sites, n_up, n_dn; numeric t, U");
    }
    const char* bc = s.get("bc");
    std::string bcs = bc ? bc : "open";
    if (L < 2 || L > 24 || nu < 0 || nu > L || nd < 0 || nd > L ||
        (bcs != "open" && bcs != "periodic") || (bcs == "periodic" && L < 3)) {
      delete A;
      return set_err(ctx, FD_ERR_ARG, "hubbard: need 2 <= n_sites <= 24 (>= 3 periodic), 0 <= n <= n_sites, bc open|periodic");
    }
    long long kron;
    if (!get_int(s, "kron", &kron, false, 0) || kron < 0 || kron > 1 || (kron && sigma != 1)) {
      delete A;
      return set_err(ctx, FD_ERR_ARG, "hubbard: kron must be 0 or 1, and kron=1 needs sigma = 1");
    }
    kron_flag = kron == 1;
    HubbardP p;
    p.L = (int)L; p.Nu = (int)nu; p.Nd = (int)nd; p.periodic = bcs == "periodic";
    p.dim_up = binom(p.L, p.Nu); p.dim_dn = binom(p.L, p.Nd);
    p.D = p.dim_up * p.dim_dn; p.t = t; p.U = U;
    if (p.D >= (1ll << 31)) { delete A; return set_err(ctx, FD_ERR_ARG, "dimension %lld >= 2^31", (long long)p.D); }
    A->D = p.D;
    int64_t* cnt;
    FD_CUDA(ctx, cudaMalloc(&rowptr, sizeof(int64_t) * (p.D + 1)));
    FD_CUDA(ctx, cudaMalloc(&cnt, sizeof(int64_t) * p.D));
    k_hubbard_count<<<(unsigned)cdiv(p.D, T), T, 0, st>>>(p, cnt);
    FD_LAUNCHED(ctx);
    FD_TRY(exclusive_scan(ctx, cnt, p.D, rowptr));
    FD_CUDA(ctx, cudaMemcpyAsync(&nnz, rowptr + p.D, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaStreamSynchronize(st));
    cudaFree(cnt);
    FD_CUDA(ctx, cudaMalloc(&col, sizeof(int32_t) * nnz));
    FD_CUDA(ctx, cudaMalloc(&val, sizeof(double) * nnz));
    k_hubbard_fill<<<(unsigned)cdiv(p.D, T), T, 0, st>>>(p, rowptr, col, val);
    FD_LAUNCHED(ctx);
    hub = p;
  } else if (s.kind == "anderson3d") {
    long long L, seed;
    double W, t;
    if (!get_int(s, "L", &L, true, 0) || !get_int(s, "seed", &seed, false, 0) ||
        !get_dbl(s, "W", &W, 0.0) || !get_dbl(s, "t", &t, 1.0) || L < 3 || L > 1290) {
      delete A;
      return set_err(ctx, FD_ERR_ARG, "anderson3d needs integer 3 <= L <= 1290, numeric W, t, integer seed");
    }
    AndersonP p;
    p.L = L; p.D = L * L * L; p.W = W; p.t = t;
    p.key = fdrng::key((uint64_t)seed, fdrng::STREAM_DISORDER);
    A->D = p.D;
    nnz = 7 * p.D;
    FD_CUDA(ctx, cudaMalloc(&rowptr, sizeof(int64_t) * (p.D + 1)));
    FD_CUDA(ctx, cudaMalloc(&col, sizeof(int32_t) * nnz));
    FD_CUDA(ctx, cudaMalloc(&val, sizeof(double) * nnz));
    k_anderson_fill<<<(unsigned)cdiv(p.D, T), T, 0, st>>>(p, rowptr, col, val);
    FD_LAUNCHED(ctx);
  } else if (s.kind == "roadgraph") {
    long long side, seed;
    double q;
    if (!get_int(s, "side", &side, true, 0) || !get_int(s, "seed", &seed, false, 0) ||
        !get_dbl(s, "q", &q, 0.3) || side < 2 || side > 46340 || !(q >= 0.0 && q <= 1.0)) {
      delete A;
      return set_err(ctx, FD_ERR_ARG, "roadgraph needs integer 2 <= side <= 46340, 0 <= q <= 1, integer seed");
    }
    RoadP p;
    p.side = side; p.N = side * side; p.q = q;
    p.ktree = fdrng::key((uint64_t)seed, fdrng::STREAM_ROAD_TREE);
    p.kextra = fdrng::key((uint64_t)seed, fdrng::STREAM_ROAD_EXTRA);
    A->D = p.N;
    int64_t* cnt;
    FD_CUDA(ctx, cudaMalloc(&rowptr, sizeof(int64_t) * (p.N + 1)));
    FD_CUDA(ctx, cudaMalloc(&cnt, sizeof(int64_t) * p.N));
    k_road_count<<<(unsigned)cdiv(p.N, T), T, 0, st>>>(p, cnt);
    FD_LAUNCHED(ctx);
    FD_TRY(exclusive_scan(ctx, cnt, p.N, rowptr));
    FD_CUDA(ctx, cudaMemcpyAsync(&nnz, rowptr + p.N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FD_CUDA(ctx, cudaStreamSynchronize(st));
    cudaFree(cnt);
    FD_CUDA(ctx, cudaMalloc(&col, sizeof(int32_t) * nnz));
    FD_CUDA(ctx, cudaMalloc(&val, sizeof(double) * nnz));
    k_road_fill<<<(unsigned)cdiv(p.N, T), T, 0, st>>>(p, rowptr, col, val);
    FD_LAUNCHED(ctx);
  } else if (s.kind == "chain") {
    long long n;
    double t;
    if (!get_int(s, "n", &n, true, 0) || !get_dbl(s, "t", &t, 1.0) || n < 2 || n >= (1ll << 31)) {
      delete A;
      return set_err(ctx, FD_ERR_ARG, "chain needs integer 2 <= n < 2^31 and numeric t");
    }
    A->D = n;
    nnz = 3 * n - 2;
    FD_CUDA(ctx, cudaMalloc(&rowptr, sizeof(int64_t) * (n + 1)));
    FD_CUDA(ctx, cudaMalloc(&col, sizeof(int32_t) * nnz));
    FD_CUDA(ctx, cudaMalloc(&val, sizeof(double) * nnz));
    k_chain_fill<<<(unsigned)cdiv(n, T), T, 0, st>>>(n, t, rowptr, col, val);
    FD_LAUNCHED(ctx);
  } else {
    delete A;
    return set_err(ctx, FD_ERR_ARG, "unknown matrix kind '%s'", s.kind.c_str());
  }
  FD_TRY(finish_build(ctx, A, rowptr, col, val, nnz, out));
  if (kron_flag) {
    const fd_status st = build_kron(ctx, *out, hub);
    if (st != FD_OK) {
      fd_matrix_free(*out);
      *out = nullptr;
      return st;
    }
  }
  return FD_OK;
}

fd_status fd_matrix_from_csr(fd_ctx* ctx, int64_t D, const int64_t* rowptr, const int32_t* col,
                             const double* val, int C, int sigma, fd_matrix** out) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!out || !rowptr || (!col && D > 0) || (!val && D > 0))
    return set_err(ctx, FD_ERR_ARG, "null argument");
  *out = nullptr;
  if (D < 1 || D >= (1ll << 31)) return set_err(ctx, FD_ERR_ARG, "D must be in [1, 2^31)");
  if (C < 32 || C % 32 != 0 || C > 1024 || sigma < 1 || sigma > 65536)
    return set_err(ctx, FD_ERR_ARG, "C must be a multiple of 32 in [32, 1024], sigma in [1, 65536]");
  if (rowptr[0] != 0) return set_err(ctx, FD_ERR_ARG, "rowptr[0] must be 0");
  for (int64_t r = 0; r < D; ++r) {
    if (rowptr[r + 1] < rowptr[r]) return set_err(ctx, FD_ERR_ARG, "rowptr decreases at row %lld", (long long)r);
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      if (col[k] < 0 || col[k] >= D)
        return set_err(ctx, FD_ERR_ARG, "column %d out of range in row %lld", col[k], (long long)r);
      if (k > rowptr[r] && col[k] <= col[k - 1])
        return set_err(ctx, FD_ERR_ARG, "columns not strictly ascending in row %lld", (long long)r);
    }
  }
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  int64_t nnz = rowptr[D];
  fd_matrix* A = new fd_matrix();
  A->ctx = ctx; A->device = ctx->device; A->D = D; A->C = C; A->sigma = sigma;
  int64_t* d_rowptr;
  int32_t* d_col;
  double* d_val;
  FD_CUDA(ctx, cudaMalloc(&d_rowptr, sizeof(int64_t) * (D + 1)));
  FD_CUDA(ctx, cudaMalloc(&d_col, sizeof(int32_t) * std::max<int64_t>(1, nnz)));
  FD_CUDA(ctx, cudaMalloc(&d_val, sizeof(double) * std::max<int64_t>(1, nnz)));
  FD_CUDA(ctx, cudaMemcpyAsync(d_rowptr, rowptr, sizeof(int64_t) * (D + 1), cudaMemcpyHostToDevice, ctx->stream));
  if (nnz > 0) {
    FD_CUDA(ctx, cudaMemcpyAsync(d_col, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, ctx->stream));
    FD_CUDA(ctx, cudaMemcpyAsync(d_val, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, ctx->stream));
  }
  return finish_build(ctx, A, d_rowptr, d_col, d_val, nnz, out);
}

fd_status fd_matrix_free(fd_matrix* A) {
  if (!A) return FD_ERR_ARG;
  // the context may already be gone: use the device recorded at creation
  cudaSetDevice(A->device);
  cudaDeviceSynchronize();
  cudaFree(A->chunk_ptr); cudaFree(A->row_len); cudaFree(A->col); cudaFree(A->val);
  cudaFree(A->val32); cudaFree(A->valff); cudaFree(A->perm); cudaFree(A->iperm); cudaFree(A->diag_added);
  for (int sp = 0; sp < 2; ++sp) {
    cudaFree(A->kbits[sp]); cudaFree(A->kptr[sp]); cudaFree(A->kcol[sp]);
    cudaFree(A->kval[sp]); cudaFree(A->kval32[sp]); cudaFree(A->kvalff[sp]);
  }
  cudaFree(A->kdiag); cudaFree(A->kdiag32); cudaFree(A->kdiagff);
  cudaFree(A->korder); cudaFree(A->kdn_ptr); cudaFree(A->kdn_ent); cudaFree(A->kdn_ent16);
  delete A;
  return FD_OK;
}

fd_status fd_matrix_get_info(const fd_matrix* A, fd_matrix_info* info) {
  if (!A || !info) return FD_ERR_ARG;
  info->D = A->D; info->nnz = A->nnz; info->nnz_sell = A->nnz_sell; info->n_chunks = A->n_chunks;
  info->C = A->C; info->sigma = A->sigma; info->max_row = A->max_row;
  info->identity_perm = A->identity; info->gersh_lo = A->gersh_lo; info->gersh_hi = A->gersh_hi;
  return FD_OK;
}

fd_status fd_matrix_to_csr(fd_ctx* ctx, const fd_matrix* A, int64_t* rowptr, int32_t* col,
                           double* val) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !rowptr || !col || !val) return set_err(ctx, FD_ERR_ARG, "null argument");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  const int T = 256;
  cudaStream_t st = ctx->stream;
  const int64_t D = A->D;
  void* p;
  FD_TRY(workspace(ctx, "export_cnt", sizeof(int64_t) * D, &p));
  int64_t* cnt = (int64_t*)p;
  int64_t *d_rowptr, nnz_out = 0;
  int32_t* d_col;
  double* d_val;
  FD_CUDA(ctx, cudaMalloc(&d_rowptr, sizeof(int64_t) * (D + 1)));
  k_export_len<<<(unsigned)cdiv(D, T), T, 0, st>>>(A->perm, A->row_len, A->diag_added, D, cnt);
  FD_LAUNCHED(ctx);
  FD_TRY(exclusive_scan(ctx, cnt, D, d_rowptr));
  FD_CUDA(ctx, cudaMemcpyAsync(&nnz_out, d_rowptr + D, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  FD_CUDA(ctx, cudaMalloc(&d_col, sizeof(int32_t) * std::max<int64_t>(1, nnz_out)));
  FD_CUDA(ctx, cudaMalloc(&d_val, sizeof(double) * std::max<int64_t>(1, nnz_out)));
  k_export_fill<<<(unsigned)cdiv(D, T), T, 0, st>>>(A->perm, A->row_len, A->diag_added,
                                                    A->chunk_ptr, A->col, A->val, D, A->C,
                                                    d_rowptr, d_col, d_val);
  FD_LAUNCHED(ctx);
  FD_CUDA(ctx, cudaMemcpyAsync(rowptr, d_rowptr, sizeof(int64_t) * (D + 1), cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaMemcpyAsync(col, d_col, sizeof(int32_t) * nnz_out, cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaMemcpyAsync(val, d_val, sizeof(double) * nnz_out, cudaMemcpyDeviceToHost, st));
  FD_CUDA(ctx, cudaStreamSynchronize(st));
  cudaFree(d_rowptr); cudaFree(d_col); cudaFree(d_val);
  return FD_OK;
}

fd_status fd_matrix_perm(fd_ctx* ctx, const fd_matrix* A, int64_t* perm) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !perm) return set_err(ctx, FD_ERR_ARG, "null argument");
  FD_CUDA(ctx, cudaMemcpyAsync(perm, A->perm, sizeof(int64_t) * A->D, cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return FD_OK;
}

}  // extern "C"
