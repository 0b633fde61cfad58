// Cholesky-QR of a search block with no device allocation.
//
// Some callers cannot let a library call cudaMalloc: applications whose GPU
// memory is already owned by another allocator (a framework's caching
// allocator that has reserved the device, or a serving process that sizes
// its memory pool once at start-up and treats any later allocation as a
// failure).  For them this file offers fd_orthonormalize_noalloc, which does
// the same work as fd_orthonormalize but keeps its scratch (the Gram matrix,
// its partial sums, the Cholesky factor, its inverse) in one file-scope
// device array of fixed size instead of the context's allocated workspaces.
#include <cuda_runtime.h>

#include <mutex>

#include "fd_internal.cuh"

// 32 MiB of scratch per GPU that loads the library, held until the process exits.
static constexpr size_t FD_NOALLOC_DOUBLES = (size_t)4 << 20;
// largest block width accepted (4 ns^2 + one ns^2 partial slice must fit)
static constexpr int FD_NOALLOC_MAX_NS = 256;
static __device__ __align__(256) double fd_noalloc_scratch[FD_NOALLOC_DOUBLES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch[MAX_DEVICES] = {};

// Device address of the scratch array on `device`, looked up once per device
// with that device current.  The array's name is only a host-side handle;
// kernels must be given this address.
fd_status scratch_address(fd_ctx* ctx, double** out) {
  if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
    return fdi::set_err(ctx, FD_ERR_ARG, "device ordinal %d out of range", ctx->device);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[ctx->device]) {
    FD_CUDA(ctx, cudaSetDevice(ctx->device));
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, fd_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fdi::set_err(ctx, FD_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                          cudaGetErrorString(e));
    g_scratch[ctx->device] = p;
  }
  *out = g_scratch[ctx->device];
  return FD_OK;
}
}  // namespace

using namespace fdi;

extern "C" fd_status fd_orthonormalize_noalloc(fd_ctx* ctx, double* V, int64_t D, int ns,
                                               int64_t ldv, double* R, int* passes_out) {
  if (!ctx) return FD_ERR_ARG;
  ctx->err.clear();
  if (!V || D < 1 || ns < 1 || ldv < ns || ns > D)
    return set_err(ctx, FD_ERR_ARG, "need V, 1 <= ns <= D, ldv >= ns");
  if (ns > FD_NOALLOC_MAX_NS)
    return set_err(ctx, FD_ERR_ARG, "ns = %d exceeds the no-allocation maximum of %d columns", ns,
                   FD_NOALLOC_MAX_NS);
  FD_CUDA(ctx, cudaSetDevice(ctx->device));
  double* base = nullptr;
  FD_TRY(scratch_address(ctx, &base));
  // scratch layout: G, Rk, Ri, Rt (ns x ns each), one 8-byte flag slot, then
  // the Gram partial sums (as many ns x ns slices as fit)
  const size_t nn = (size_t)ns * ns;
  double* G = base;
  double* Rk = G + nn;
  double* Ri = Rk + nn;
  double* Rt = Ri + nn;
  int* ok = (int*)(Rt + nn);
  double* P = Rt + nn + 1;
  const int64_t max_slices = (int64_t)((FD_NOALLOC_DOUBLES - 4 * nn - 1) / nn);
  const double coeff = 11.0 * ((double)D * ns + (double)ns * (ns + 1)) * 0x1.0p-53;
  if (R) FD_TRY(identity_dev(ctx, R, ns));
  bool any_shift = false;
  int passes = 0;
  while (passes < 2 || (any_shift && passes < 3)) {
    FD_CUDA(ctx, cudaMemsetAsync(ok, 0, sizeof(int), ctx->stream));
    FD_TRY(gram_partials(ctx, V, ldv, V, ldv, D, ns, ns, G, ns, true, P, max_slices));
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
    // FP64 rotation in place: the tensor-core rotation needs digit workspaces
    FD_TRY(rotate_fp64(ctx, V, ldv, D, ns, Ri, true));
    if (R) {
      FD_TRY(small_gemm_dev(ctx, Rk, R, Rt, ns));
      FD_CUDA(ctx, cudaMemcpyAsync(R, Rt, sizeof(double) * nn, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    ++passes;
  }
  FD_TRY(check_last_factor(ctx, Rk, ns));
  if (passes_out) *passes_out = passes;
  return FD_OK;
}
