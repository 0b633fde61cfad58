// Communication metrics of distributed SpMV (Sec. 3.1), from the sparsity
// pattern on the device.
//
// For the uniform distribution of the rows over N_p processes (process p owns
// rows [floor(p D / N_p), floor((p + 1) D / N_p))), each process's rows are
// scanned once: every stored entry with a nonzero value sets the bit of its
// column in a D-bit map (atomicOr), and a popcount over the map splits the
// distinct columns into the process's own range (n_vm) and the rest (n_vc).
// One map is reused for the processes in turn; the counters of all processes
// are read back once.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "fd_internal.cuh"

namespace fdi {
namespace {

// rows [a, b) of a SELL matrix in original order; thread per row (consecutive
// threads read adjacent words of the chunk's column-major slab)
__global__ void k_comm_mark(const int64_t* __restrict__ chunk_ptr, const int32_t* __restrict__ row_len,
                            const int32_t* __restrict__ col, const double* __restrict__ val, int C,
                            int64_t a, int64_t b, uint32_t* __restrict__ bm) {
  for (int64_t r = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < b;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int len = row_len[r];
    const int64_t base = chunk_ptr[r / C] + r % C;
    for (int j = 0; j < len; ++j) {
      const int64_t e = base + (int64_t)j * C;
      if (val[e] != 0.0) {
        const uint32_t c = (uint32_t)col[e];
        atomicOr(bm + (c >> 5), 1u << (c & 31));
      }
    }
  }
}

// cnt[0] += set bits with index in [a, b), cnt[1] += all set bits
__global__ void k_comm_count(const uint32_t* __restrict__ bm, int64_t nwords, int64_t a, int64_t b,
                             unsigned long long* cnt) {
  unsigned long long loc = 0, tot = 0;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
       w += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = bm[w];
    if (!x) continue;
    tot += __popc(x);
    const int64_t lo = 32 * w, hi = lo + 32;  // bit indices [lo, hi)
    if (hi <= a || lo >= b) continue;
    uint32_t m = 0xffffffffu;
    if (lo < a) m &= ~((1u << (uint32_t)(a - lo)) - 1u);  // a - lo in 1 .. 31
    if (hi > b) m &= (1u << (uint32_t)(b - lo)) - 1u;     // b - lo in 1 .. 31
    loc += __popc(x & m);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    loc += __shfl_xor_sync(0xffffffffu, loc, o);
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
  }
  if ((threadIdx.x & 31) == 0 && tot) {
    atomicAdd(cnt, loc);
    atomicAdd(cnt + 1, tot);
  }
}

}  // namespace
}  // namespace fdi

using namespace fdi;

extern "C" fd_status fd_comm_metrics(fd_ctx* ctx, const fd_matrix* A, int n_p, int64_t* n_vc,
                                     int64_t* n_vm, double* chi) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!A || !chi) return set_err(ctx, FD_ERR_ARG, "null matrix or chi");
  if (n_p < 1 || n_p > A->D) return set_err(ctx, FD_ERR_ARG, "need 1 <= n_p <= D");
  if (!A->identity) return set_err(ctx, FD_ERR_ARG, "communication metrics need sigma = 1 (original row order)");
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t D = A->D, nwords = cdiv(D, 32);
  void* p;
  FD_TRY(workspace(ctx, "comm_bitmap", sizeof(uint32_t) * (size_t)nwords + 16 * (size_t)n_p + 16, &p));
  uint32_t* bm = (uint32_t*)p;
  unsigned long long* cnt = (unsigned long long*)(((uintptr_t)(bm + nwords) + 15) & ~(uintptr_t)15);
  FD_CUDA(ctx, cudaMemsetAsync(cnt, 0, 16 * (size_t)n_p, ctx->stream));
  const int T = 256;
  for (int q = 0; q < n_p; ++q) {
    const int64_t a = q * D / n_p, b = (q + 1) * D / n_p;
    FD_CUDA(ctx, cudaMemsetAsync(bm, 0, sizeof(uint32_t) * (size_t)nwords, ctx->stream));
    if (b > a) {
      const unsigned gm = (unsigned)std::min<int64_t>(cdiv(b - a, T), 16LL * ctx->num_sms);
      k_comm_mark<<<gm, T, 0, ctx->stream>>>(A->chunk_ptr, A->row_len, A->col, A->val, A->C, a, b, bm);
      FD_LAUNCHED(ctx);
    }
    const unsigned gc = (unsigned)std::min<int64_t>(cdiv(nwords, T), 8LL * ctx->num_sms);
    k_comm_count<<<gc, T, 0, ctx->stream>>>(bm, nwords, a, b, cnt + 2 * q);
    FD_LAUNCHED(ctx);
  }
  std::vector<unsigned long long> h(2 * (size_t)n_p);
  FD_CUDA(ctx, cudaMemcpyAsync(h.data(), cnt, 16 * (size_t)n_p, cudaMemcpyDeviceToHost, ctx->stream));
  FD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double chi1 = 0.0, sum_vc = 0.0, max_vc = 0.0;
  for (int q = 0; q < n_p; ++q) {
    const int64_t vm = (int64_t)h[2 * q], vc = (int64_t)(h[2 * q + 1] - h[2 * q]);
    if (n_vc) n_vc[q] = vc;
    if (n_vm) n_vm[q] = vm;
    const double r = vm > 0 ? (double)vc / (double)vm : (vc > 0 ? INFINITY : 0.0);
    chi1 = std::max(chi1, r);
    sum_vc += (double)vc;
    max_vc = std::max(max_vc, (double)vc);
  }
  if (n_p == 1) chi1 = sum_vc = max_vc = 0.0;
  chi[0] = chi1;
  chi[1] = sum_vc / (double)D;
  chi[2] = (double)n_p * max_vc / (double)D;
  return FD_OK;
}
