// Internal declarations shared by the translation units of libfd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/fd.h"

struct fd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  size_t smem_optin = 0;
  std::string err;
  int64_t launches = 0;
  int gemm_mode = 0;  // fd_gemm_mode: 0 auto, 1 FP64 arithmetic, 2 bf16 tensor-core splitting
  // grow-only device workspaces keyed by purpose
  std::unordered_map<std::string, std::pair<void*, size_t>> ws;
  size_t ws_bytes = 0;      // bytes the workspaces hold now
  int64_t ws_allocs = 0;    // cudaMalloc calls made for workspaces
  size_t ws_limit = 0;      // cap on ws_bytes (0 = none): growth beyond it fails with FD_ERR_OOM
  int debug_checks = 0;     // scan matrix index arrays before step kernels (FD_ERR_BOUNDS)
  // pinned host staging
  void* host_stage = nullptr;
  size_t host_stage_bytes = 0;
};

struct fd_matrix {
  fd_ctx* ctx = nullptr;  // creating context (not dereferenced by fd_matrix_free)
  int device = 0;
  int64_t D = 0, nnz = 0, nnz_sell = 0, n_chunks = 0;
  int C = 32, sigma = 1, max_row = 0, identity = 1;
  double gersh_lo = 0, gersh_hi = 0;
  // SELL-C-sigma arrays (device), rows in SELL order; entry j of SELL row i
  // (chunk c = i / C, r = i % C) sits at chunk_ptr[c] + j * C + r; entry 0 of
  // every row is its diagonal; padding entries hold (0, own row).
  int64_t* chunk_ptr = nullptr;  // n_chunks + 1
  int32_t* row_len = nullptr;    // n_chunks * C (0 beyond D)
  int32_t* col = nullptr;        // nnz_sell, SELL column indices
  double* val = nullptr;         // nnz_sell
  float* val32 = nullptr;        // nnz_sell
  float* valff = nullptr;        // 2 nnz_sell: float-float (hi, lo) pairs of val
  int64_t* perm = nullptr;       // D: SELL row -> original row
  int64_t* iperm = nullptr;      // D: original row -> SELL row
  uint8_t* diag_added = nullptr; // D (SELL order): 1 if the diagonal was not in the input
  // Matrix-free Hubbard operator (spec flag kron=1; rows in original order):
  // H = H_up x 1 + 1 x H_dn + U n_double with row = rank_up * dim_dn + rank_dn.
  // Per spin species s (0 up, 1 down): the states' bit strings and their
  // hopping lists, targets ascending, value -t * fermion sign.
  int kron = 0;
  double* kdiag = nullptr;          // 25: U * n for n doubly occupied sites
  float* kdiag32 = nullptr;         // 25: (float) (U * n)
  float* kdiagff = nullptr;         // 25 float-float pairs of U * n
  int64_t kdim[2] = {0, 0};
  uint32_t* kbits[2] = {nullptr, nullptr};
  int64_t* kptr[2] = {nullptr, nullptr};   // kdim + 1
  int32_t* kcol[2] = {nullptr, nullptr};
  double* kval[2] = {nullptr, nullptr};
  float* kval32[2] = {nullptr, nullptr};
  float* kvalff[2] = {nullptr, nullptr};  // float-float pairs of kval
  // Tables of the panel kernel of the matrix-free operator (fd_kron.cu):
  // korder: the up-spin states (slabs u) in reverse Cuthill-McKee order of the
  // up-spin hopping graph, the order in which a step visits the slabs;
  // kdn_ptr / kdn_ent: the down-spin hops packed as (target | sign bit << 31),
  // the hop value being kdn_val[sign bit] (-t for +1, +t for -1)
  int32_t* korder = nullptr;      // kdim[0]
  uint32_t* kdn_ptr = nullptr;    // kdim[1] + 1
  uint32_t* kdn_ent = nullptr;    // down hops
  uint16_t* kdn_ent16 = nullptr;  // the same as (16 target | sign bit) when dim_dn <= 4096
  double kdn_val[2] = {0, 0};
  float kdn_val32[2] = {0, 0};
  int kmax_up = 0;                // most up hops of one state
};

namespace fdi {

// ---- error plumbing -------------------------------------------------------
fd_status set_err(fd_ctx* ctx, fd_status st, const char* fmt, ...);

#define FD_CUDA(ctx, call)                                                       \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return fdi::set_err((ctx), e_ == cudaErrorMemoryAllocation ? FD_ERR_OOM   \
                                                                  : FD_ERR_CUDA, \
                          "%s failed: %s (%s:%d)", #call,                        \
                          cudaGetErrorString(e_), __FILE__, __LINE__);           \
  } while (0)

#define FD_LAUNCHED(ctx)                                                         \
  do {                                                                           \
    (ctx)->launches++;                                                           \
    cudaError_t e_ = cudaGetLastError();                                         \
    if (e_ != cudaSuccess)                                                       \
      return fdi::set_err((ctx), FD_ERR_CUDA, "kernel launch failed: %s (%s:%d)", \
                          cudaGetErrorString(e_), __FILE__, __LINE__);           \
  } while (0)

#define FD_TRY(expr)                 \
  do {                               \
    fd_status s_ = (expr);           \
    if (s_ != FD_OK) return s_;      \
  } while (0)

// grow-only workspace of at least `bytes` bytes under `name`
fd_status workspace(fd_ctx* ctx, const char* name, size_t bytes, void** out);
fd_status host_stage(fd_ctx* ctx, size_t bytes, void** out);

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- SELL construction (fd_matrix.cu) -------------------------------------
// Build the SELL-C-sigma arrays of `A` from a device CSR (rowptr D+1, col, val),
// columns ascending per row.  Frees nothing it was given.
fd_status sell_from_device_csr(fd_ctx* ctx, fd_matrix* A, const int64_t* d_rowptr,
                               const int32_t* d_col, const double* d_val, int64_t nnz);

// FD_ERR_BOUNDS if A's device index arrays hold an index outside [0, D)
// (only when ctx->debug_checks; fd_filter.cu)
fd_status debug_check_matrix(fd_ctx* ctx, const fd_matrix* A);

// ---- SpMMV / Chebyshev step (fd_filter.cu) --------------------------------
fd_status spmmv(fd_ctx* ctx, const fd_matrix* A, fd_prec prec, const void* X,
                int64_t ldx, void* Y, int64_t ldy, int nb, bool original_order);
fd_status filter(fd_ctx* ctx, const fd_matrix* A, fd_prec prec, void* V, int64_t ldv,
                 int nb, int degree, const double* mu, double alpha, double beta,
                 void* W1, void* W2, int64_t ldw, double* bytes_out);
// the same filter for a matrix-free Hubbard operator: the block in 16-byte
// column panels, slabs in korder (fd_kron.cu)
fd_status kron_filter(fd_ctx* ctx, const fd_matrix* A, fd_prec prec, void* V, int64_t ldv,
                      int nb, int degree, const double* mu, double alpha, double beta,
                      void* W1, void* W2, int64_t ldw, double* bytes_out);
// the panel kernel's tables of A (after the per-species tables exist)
fd_status kron_panel_tables(fd_ctx* ctx, fd_matrix* A, double t);
// nb = 1 SpMV in SELL order, FP64: y = A x (x, y dense vectors in SELL order)
fd_status spmv1(fd_ctx* ctx, const fd_matrix* A, const double* x, double* y);
// KPM Chebyshev iteration with moment epilogue (fd_filter.cu)
fd_status kpm(fd_ctx* ctx, const fd_matrix* A, int n_moments, int R, uint64_t seed,
              double alpha, double beta, double* mu_host);

// ---- dense FP64 (fd_dense.cu) ---------------------------------------------
// C (m x n, row-major, ldc) = X^T Y with X: D x m (ldx), Y: D x n (ldy).
// sym: X == Y, compute upper tiles and mirror.
fd_status gram(fd_ctx* ctx, const double* X, int64_t ldx, const double* Y, int64_t ldy,
               int64_t D, int m, int n, double* C, int ldc, bool sym);
// the same product with the caller's partial-sum buffer P (>= slices * m * n
// doubles, at most max_slices slices); allocates nothing
fd_status gram_partials(fd_ctx* ctx, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                        int64_t D, int m, int n, double* C, int ldc, bool sym, double* P,
                        int64_t max_slices);
fd_status identity_dev(fd_ctx* ctx, double* A, int n);
fd_status small_gemm_dev(fd_ctx* ctx, const double* A, const double* B, double* C, int n);
// V (D x n, ldv) <- V * M, M n x n row-major; upper = M upper triangular
fd_status rotate(fd_ctx* ctx, double* V, int64_t ldv, int64_t D, int n, const double* M,
                 bool upper);
// the same rotation with FP64 arithmetic only (in place, shared-memory rows;
// allocates nothing, whatever the gemm mode)
fd_status rotate_fp64(fd_ctx* ctx, double* V, int64_t ldv, int64_t D, int n, const double* M,
                      bool upper);
// Cholesky of the n x n SPD matrix G (device), upper factor into R; status into
// *ok_dev (1 ok / 0 failed); shift added to the diagonal before factorising.
fd_status cholesky(fd_ctx* ctx, const double* G, int n, double shift_rel_trace_coeff,
                   double* R, int* ok_dev);
fd_status tri_inverse(fd_ctx* ctx, const double* R, int n, double* Rinv);
// symmetric eigensolve of the n x n matrix H (device, destroyed): eigenvalues
// ascending into w (device n), eigenvectors as columns of Q (device n x n)
fd_status sym_eig(fd_ctx* ctx, double* H, int n, double* w, double* Q, int max_sweeps);
// column 2-norms of AV - V diag(theta) (D x n, ld) into out (device n)
fd_status resid_norms(fd_ctx* ctx, const double* V, const double* AV, int64_t ld,
                      int64_t D, int n, const double* theta, double* out);
fd_status orthonormalize(fd_ctx* ctx, double* V, int64_t D, int ns, int64_t ldv,
                         double* R, int* passes);
// FD_ERR_BREAKDOWN if the last Cholesky-QR factor's diagonal (device Rk, ns x ns)
// is not within a factor 4 of 1 (synchronises)
fd_status check_last_factor(fd_ctx* ctx, const double* Rk, int ns);
fd_status rayleigh_ritz_dev(fd_ctx* ctx, const fd_matrix* A, double* V, double* AV,
                            int64_t D, int ns, int64_t ld, double* theta_dev,
                            double* resid_dev);
// Ozaki-scheme products on bf16 tensor cores (fd_ozaki.cu); *used = false
// (and no error) when the input holds non-finite values
fd_status oz_gram(fd_ctx* ctx, const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t D,
                  int m, int n, double* C, int ldc, bool sym, bool* used);
fd_status oz_rotate(fd_ctx* ctx, double* V, int64_t ldv, int64_t D, int n, const double* M, bool upper,
                    bool* used);
// small helpers
fd_status copy_cols_f64_to_f32(fd_ctx* ctx, const double* src, int64_t lds, float* dst,
                               int64_t ldd, int64_t D, int n);
fd_status copy_cols_f32_to_f64(fd_ctx* ctx, const float* src, int64_t lds, double* dst,
                               int64_t ldd, int64_t D, int n);
// FP64 <-> float-float blocks (ld in elements; a float-float element is 2 floats)
fd_status copy_cols_f64_to_ff(fd_ctx* ctx, const double* src, int64_t lds, float* dst, int64_t ldd,
                              int64_t D, int n);
fd_status copy_cols_ff_to_f64(fd_ctx* ctx, const float* src, int64_t lds, double* dst, int64_t ldd,
                              int64_t D, int n);

// ---- Lehmann bounds (fd_lehmann.cu) -----------------------------------------
// eigenvalues (device, ascending) of the pencil A1 x = mu A2 x (A1, A2 destroyed);
// *ok = false if A2 is not numerically positive definite
fd_status lehmann_pencil(fd_ctx* ctx, double* A1, double* A2, int n, double* mu, bool* ok);
// bounds rho + 1/mu: below (nearest rho first) from mu < 0, above from mu > 0
void lehmann_from_mu(const std::vector<double>& mu, double rho, std::vector<double>* below,
                     std::vector<double>* above);
// Lehmann bounds at rho from Ritz vectors V, AV = A V and Ritz values theta_dev
// (device); AV is overwritten by (A - rho) V
fd_status lehmann_ritz(fd_ctx* ctx, const double* V, double* AV, int64_t ld, int64_t D, int ns,
                       const double* theta_dev, double rho, std::vector<double>* below,
                       std::vector<double>* above, bool* ok);

// ---- solver pieces (fd_solve.cu) ------------------------------------------
fd_status spectral_bounds(fd_ctx* ctx, const fd_matrix* A, int steps, uint64_t seed,
                          double* lam_l, double* lam_r);
// Jackson-damped window coefficients, p(window centre) = 1 (host arithmetic)
std::vector<double> filter_coeffs(double x_l, double x_r, int n);

}  // namespace fdi

// ---- SplitMix64 (device + host), Steele, Lea, Flood 2014 -------------------
namespace fdrng {
constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
constexpr int STREAM_DISORDER = 1, STREAM_START = 2, STREAM_LANCZOS = 3, STREAM_KPM = 4;
constexpr int STREAM_ROAD_TREE = 7, STREAM_ROAD_EXTRA = 8;
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t key(uint64_t seed, uint64_t stream) {
  return mix64(seed ^ mix64(stream));
}
__host__ __device__ inline uint64_t raw(uint64_t k, uint64_t i) { return mix64(k + (i + 1) * GAMMA); }
// uniform in [0, 1): (x >> 11) * 2^-53, exact
__device__ inline double uniform(uint64_t k, uint64_t i) {
  return __dmul_rn(__ull2double_rn(raw(k, i) >> 11), 0x1.0p-53);
}
// Irwin-Hall normal-like draw: integer sum of 12 53-bit draws, one conversion
__device__ inline double irwin_hall(uint64_t k, uint64_t e) {
  uint64_t s = 0;
#pragma unroll
  for (int t = 0; t < 12; ++t) s += raw(k, 12 * e + t) >> 11;
  return __dsub_rn(__dmul_rn(__ull2double_rn(s), 0x1.0p-53), 6.0);
}
}  // namespace fdrng
