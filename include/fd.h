/*
 * fd.h -- C ABI of the GB300 filter-diagonalization (FD) library.
 *
 * Filter diagonalization (Alvermann, Hager, Fehske, arXiv 2209.01974) finds
 * the N_t eigenpairs of a large sparse symmetric matrix H nearest a target
 * window by repeatedly applying a Chebyshev polynomial filter to a block of
 * N_s search vectors (Sec. 2, Alg. 1 and Alg. 2), orthonormalising the block,
 * and extracting Ritz pairs with one more sparse matrix-multiple-vector
 * product (SpMMV).  This header exposes the steps of that hot path:
 *
 *   fd_build_matrix / fd_matrix_from_csr   -> on-device SELL-C-sigma matrix
 *   fd_spectral_bounds                     -> inclusion interval (Sec. 2)
 *   fd_filter                              -> V <- p(alpha H + beta) V (Alg. 2)
 *   fd_orthonormalize                      -> Cholesky-QR of the block (Sec. 2)
 *   fd_rayleigh_ritz                       -> Ritz pairs + residuals (Sec. 2)
 *   fd_solve                               -> the whole FD loop (Alg. 1)
 *   fd_kpm_moments                         -> KPM density-of-states moments (Sec. 4.1)
 *
 * Conventions shared by every entry point
 *   - Every call returns fd_status; no C++ exception crosses the ABI.  On an
 *     error, fd_last_error(ctx) returns a message for the last failing call
 *     made with that context.
 *   - Blocks of vectors are caller-owned DEVICE buffers (e.g. the data
 *     pointer of a torch tensor), row-major: element (i, j) of a D x m block
 *     with leading dimension ld sits at p[i * ld + j], rows in the matrix's
 *     ORIGINAL row order.  Base pointers and ld * element size must be
 *     multiples of 16 bytes for the SpMMV kernels.
 *   - All device work is ordered on the context's CUDA stream.  Calls that
 *     write HOST outputs synchronise that stream before returning; the others
 *     return after enqueueing work.
 *   - Matrices are library-owned and freed with fd_matrix_free.
 *   - The library allocates its internal workspaces with cudaMalloc and keeps
 *     them in the context until fd_destroy.
 */
#ifndef FD_H
#define FD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fd_ctx fd_ctx;
typedef struct fd_matrix fd_matrix;

typedef enum {
  FD_OK = 0,
  FD_ERR_ARG = 1,       /* invalid argument (checked before any device work) */
  FD_ERR_CUDA = 2,      /* a CUDA runtime call or kernel launch failed */
  FD_ERR_OOM = 3,       /* device allocation failed */
  FD_ERR_NOCONV = 4,    /* fd_solve reached max_outer without convergence */
  FD_ERR_BREAKDOWN = 5, /* Cholesky-QR failed even with the shift */
  FD_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
  FD_ERR_BOUNDS = 7     /* a device-side bounds check fired (bad CSR / index) */
} fd_status;

/* Arithmetic of the filter sweeps.  FD_FF ("float-float"): every value is an
 * unevaluated sum hi + lo of two floats, stored as the pair (hi, lo) in 8
 * bytes, with sums and products from error-free transformations in FP32
 * arithmetic (about 2^-48 relative, FP32 exponent range).  Not in the paper:
 * GB300 runs FP64 at about 1/64 of its FP32 rate, so FP64-accurate sweeps are
 * cheaper in FP32 pairs than in FP64. */
typedef enum { FD_F64 = 0, FD_F32 = 1, FD_FF = 2 } fd_prec;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`; `stream` is a cudaStream_t (NULL =
 * the legacy default stream).  The context does not own the stream. */
fd_status fd_create(fd_ctx** ctx, int device, void* stream);
/* Destroy the context and free its workspaces.  Matrices must be freed first. */
fd_status fd_destroy(fd_ctx* ctx);
/* Replace the stream all later calls enqueue on. */
fd_status fd_set_stream(fd_ctx* ctx, void* stream);
/* Message of the last failing call on this context ("" if none).  The string
 * is owned by the context and valid until its next call. */
const char* fd_last_error(const fd_ctx* ctx);
/* Number of kernels this context has launched since creation (for audits). */
int64_t fd_kernel_launches(const fd_ctx* ctx);
/* Device memory held by the context's grow-only workspaces (HOST outputs,
 * either may be NULL): the bytes held now and the number of cudaMalloc calls
 * made for them since creation.  The paper has no counterpart; callers use it
 * to audit the library's allocations. */
fd_status fd_workspace_info(const fd_ctx* ctx, size_t* bytes_held, int64_t* allocations);
/* Cap the bytes the context's workspaces may hold together (0 = no cap, the
 * default).  A workspace that would grow beyond the cap is refused before
 * anything is freed or allocated and the call needing it returns FD_ERR_OOM,
 * exactly as when cudaMalloc fails; the tensor-core products instead fall
 * back to FP64 arithmetic when their digit workspace is refused.  Lets a
 * caller bound the library's memory (and tests inject an allocation failure
 * from the host). */
fd_status fd_set_workspace_limit(fd_ctx* ctx, size_t limit_bytes);

/* ------------------------------------------------------------------ matrices */

/* Build a test matrix on the device from a parameter string (the paper names
 * its matrices by ScaMaC parameter strings, Sec. 3.2; Table 2):
 *   "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open"     (bc = open|periodic;
 *                                       kron=1 also builds the per-spin hopping
 *                                       tables: fd_filter and fd_spmmv then apply
 *                                       H = H_up x 1 + 1 x H_dn + U n_double without
 *                                       the stored matrix: FP64 and float-float
 *                                       rows summed in the stored order, FP32 in
 *                                       column panels (equal to rounding); needs
 *                                       sigma = 1)
 *   "anderson3d:L=128,W=2,seed=1,t=1"   periodic cubic lattice, eps_i = W (u_i - 1/2)
 *   "chain:n=1000,t=1"                  open tight-binding chain
 *   "roadgraph:side=2000,q=0.3,seed=0"  Laplacian of a road-like planar graph on a
 *                                       side x side grid: a random spanning tree
 *                                       (each node links to its left or lower
 *                                       neighbour) plus every other grid edge with
 *                                       probability q (mean degree ~ 2(1+q))
 * Generation is integer-exact and bit-identical to the CPU definition (Hubbard
 * basis: occupation bitstrings ranked in increasing order, row = rank_up *
 * dim_dn + rank_dn, hop sign (-1)^(fermions passed)).  The result is stored in
 * SELL-C-sigma (Kreutzer et al. 2014, the format of the GHOST library the
 * paper uses) with chunk height C (a multiple of 32) and sorting window
 * sigma >= 1 (sigma = 1: no reordering).  FP64 values and an FP32 copy are
 * kept.  Errors: FD_ERR_ARG for an unknown kind, a missing or out-of-range
 * parameter, or D >= 2^31. */
fd_status fd_build_matrix(fd_ctx* ctx, const char* spec, fd_matrix** out);
fd_status fd_build_matrix_sell(fd_ctx* ctx, const char* spec, int C, int sigma,
                               fd_matrix** out);

/* Copy a symmetric CSR matrix from HOST arrays (rowptr: D+1 int64, col: nnz
 * int32 strictly ascending per row, val: nnz double).  The arrays are copied;
 * the caller keeps ownership.  A missing diagonal entry is stored as an
 * explicit zero internally but not exported.  Symmetry is the caller's
 * responsibility.  Errors: FD_ERR_ARG for a malformed rowptr, a column out of
 * [0, D) or not ascending. */
fd_status fd_matrix_from_csr(fd_ctx* ctx, int64_t D, const int64_t* rowptr,
                             const int32_t* col, const double* val, int C,
                             int sigma, fd_matrix** out);
fd_status fd_matrix_free(fd_matrix* A);

typedef struct {
  int64_t D;          /* dimension */
  int64_t nnz;        /* stored entries of the CSR form (diagonal included) */
  int64_t nnz_sell;   /* SELL entries including chunk padding */
  int64_t n_chunks;   /* number of SELL chunks */
  int32_t C, sigma;   /* SELL chunk height and sorting window */
  int32_t max_row;    /* longest row (SELL form, diagonal included) */
  int32_t identity_perm; /* 1 if SELL row order equals the original order */
  double gersh_lo, gersh_hi; /* Gershgorin inclusion interval */
} fd_matrix_info;

fd_status fd_matrix_get_info(const fd_matrix* A, fd_matrix_info* info);

/* Export the matrix, reconstructed from its device SELL-C-sigma arrays, as
 * CSR in the original row order into HOST arrays (rowptr: D+1, col and val:
 * info.nnz).  Bit-exact with what was built or imported.  Synchronises. */
fd_status fd_matrix_to_csr(fd_ctx* ctx, const fd_matrix* A, int64_t* rowptr,
                           int32_t* col, double* val);

/* HOST array perm[D]: SELL row i holds original row perm[i].  Synchronises. */
fd_status fd_matrix_perm(fd_ctx* ctx, const fd_matrix* A, int64_t* perm);

/* ------------------------------------------------------------------ hot path */

/* Spectral inclusion interval [lam_l, lam_r] (Sec. 2, Alg. 1 steps 1-2):
 * `steps` Lanczos steps (0 -> 20) with full reorthogonalisation from the start
 * vector of SplitMix64 stream 3 with `seed`; each extreme Ritz value is moved
 * outwards by its Lanczos residual bound |beta_m s_m| plus 1% of the Ritz
 * span, then clipped to the Gershgorin interval.  Host outputs; synchronises. */
fd_status fd_spectral_bounds(fd_ctx* ctx, const fd_matrix* A, int steps,
                             uint64_t seed, double* lam_l, double* lam_r);

/* Chebyshev filter V <- p(A~) V, p(x) = sum_{k=0..degree} mu[k] T_k(x),
 * A~ = alpha H + beta I (Sec. 2, Alg. 2), applied to the nb columns of the
 * D x nb block V (device, leading dimension ldv).  One fused kernel per
 * degree step computes the SpMMV W2 <- 2 A~ W1 - W2 together with
 * V <- V + mu_k W2 (Alg. 2 fuses the SpMV with the vector update so that W2 is
 * not read twice).
 *   prec    FD_F64: V, W1, W2 are double and H's FP64 values are used;
 *           FD_F32: V, W1, W2 are float, H's FP32 copy, FP32 accumulation;
 *           FD_FF: V, W1, W2 hold float-float pairs (2 floats per element,
 *           ld counted in elements), H's float-float copy of its FP64 values
 *           (stored, or the matrix-free tables of kron = 1).
 *   nb      2, 4, 8, 16, 32, 64 or 128 (FP64, FF); 4 .. 128 (FP32)
 *   degree  n >= 2 (Alg. 2 takes degree n >= 2); mu: HOST array of n+1 doubles
 *   W1, W2  device workspaces, D x nb each with leading dimension ldw
 *           (contents are overwritten)
 * Errors: FD_ERR_ARG (bad nb / degree / alignment / NULL), FD_ERR_CUDA. */
fd_status fd_filter(fd_ctx* ctx, const fd_matrix* A, fd_prec prec, void* V,
                    int64_t ldv, int nb, int degree, const double* mu,
                    double alpha, double beta, void* W1, void* W2, int64_t ldw);

/* Filter coefficients mu[0..n] (HOST array of n+1 doubles) of the Chebyshev
 * expansion of the indicator of the window [x_l, x_r] (scaled coordinates,
 * clipped to [-1, 1]) damped by the Jackson kernel, normalised so that p at
 * the window centre is 1 (Sec. 2 expands a window function in Chebyshev
 * polynomials; the Jackson kernel is the KPM kernel the paper cites):
 *   c_0 = (t_l - t_r)/pi, c_k = 2 (sin k t_l - sin k t_r)/(k pi), t = arccos x
 *   g_k = [(N-k+1) cos(pi k/(N+1)) + sin(pi k/(N+1)) cot(pi/(N+1))]/(N+1), N = n+1
 * Pure host arithmetic.  Errors: FD_ERR_ARG for n < 2 or x_l >= x_r. */
fd_status fd_filter_coeffs(double x_l, double x_r, int n, double* mu);

/* Sparse matrix times block: Y <- H X for D x nb blocks (the extra SpMMV of
 * Sec. 2 that precedes the Rayleigh-Ritz step).  Same layout rules as
 * fd_filter. */
fd_status fd_spmmv(fd_ctx* ctx, const fd_matrix* A, fd_prec prec,
                   const void* X, int64_t ldx, void* Y, int64_t ldy, int nb);

/* How the FP64 Gram and rotation products of fd_orthonormalize,
 * fd_rayleigh_ritz and fd_solve are computed.
 *   FD_GEMM_FP64   FP64 FMA arithmetic (GB300 runs FP64 at about 1/64 of FP32)
 *   FD_GEMM_OZAKI  exact splitting into 7-bit integer digits on the tcgen05
 *                  tensor cores (Ozaki scheme, 8 bf16 digits per operand
 *                  relative to each row / column maximum, FP32 level sums in
 *                  TMEM exact over K chunks of 128, 2 x 64-bit integer
 *                  accumulation): FP64 accuracy at tensor-core speed.  Uses a
 *                  grow-only device workspace of 16 bytes per operand element
 *                  for the digit tiles
 *   FD_GEMM_AUTO   Ozaki for D >= 65536 and at least 64 columns, else FP64
 * Inputs holding NaN or infinity always take the FP64 path, and so does a
 * product whose digit workspace cannot be allocated.  A bounded device-side
 * wait that gives up in a tensor-core product returns FD_ERR_TIMEOUT. */
typedef enum { FD_GEMM_AUTO = 0, FD_GEMM_FP64 = 1, FD_GEMM_OZAKI = 2 } fd_gemm_mode;
fd_status fd_set_gemm_mode(fd_ctx* ctx, fd_gemm_mode mode);

/* Debug checks (the paper has no counterpart): with on != 0, fd_filter and
 * fd_spmmv first scan the matrix's device arrays (SELL column indices, or
 * the matrix-free operator's hop tables) for indices outside [0, D) and
 * return FD_ERR_BOUNDS without launching a step kernel if one is found, so a
 * corrupted matrix is reported instead of read out of bounds.  Costs one pass
 * over the index arrays per call.  Off by default. */
fd_status fd_set_debug_checks(fd_ctx* ctx, int on);
/* Test hook of the debug checks: overwrite SELL column entry `entry` (in
 * [0, nnz_sell)) of A on the device with `col` (any value).  A matrix so
 * changed must only be used with debug checks on.  Synchronises. */
fd_status fd_debug_set_sell_column(fd_ctx* ctx, fd_matrix* A, int64_t entry, int32_t col);

/* Diagnostic of the failure path of the tensor-core products (the paper has
 * no counterpart): launches one CTA that initialises an mbarrier nobody
 * arrives on and waits for it with the same bounded wait the products use,
 * given up after `limit_us` microseconds of SM clock (1 .. 10,000,000; other
 * values return FD_ERR_ARG).  Returns FD_ERR_TIMEOUT, with no CUDA error
 * left behind and the context still usable; the GPU does not fault or hang.
 * Synchronises. */
fd_status fd_check_bounded_wait(fd_ctx* ctx, int limit_us);

/* Gram product C = X^T Y (device; X: D x m with ldx, Y: D x n with ldy, C: m x n
 * row-major with ldc), the tall-skinny contraction of Cholesky-QR and
 * Rayleigh-Ritz (Sec. 2).  X == Y (same pointer and ld, m == n) computes the
 * upper tiles and mirrors them.  Arithmetic per fd_set_gemm_mode. */
fd_status fd_gram(fd_ctx* ctx, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                  int64_t D, int m, int n, double* C, int ldc);
/* In-place rotation V <- V M (device; V: D x n with ldv, M: n x n row-major;
 * upper != 0: M is upper triangular and its lower part is not read). */
fd_status fd_rotate(fd_ctx* ctx, double* V, int64_t ldv, int64_t D, int n, const double* M,
                    int upper);

/* Copy the D x n device block src (leading dimension lds, type sp) into dst
 * (ldd, type dp), rounding FP64 to FP32 or widening FP32 to FP64 as needed
 * (the FP32 filter form moves bundles between the FP64 search block and FP32
 * sweep buffers with this call).  FP64 -> FD_FF splits each value into its
 * nearest float and the nearest float to the remainder; FD_FF -> FP64 adds
 * the pair (exact).  FD_F32 <-> FD_FF is FD_ERR_ARG. */
fd_status fd_copy_block(fd_ctx* ctx, const void* src, fd_prec sp, int64_t lds, void* dst,
                        fd_prec dp, int64_t ldd, int64_t D, int n);

/* Orthonormalise the D x ns FP64 block V in place (Sec. 2: orthogonalisation
 * after the random start and after every filter application) by Cholesky-QR
 * twice (G = V^T V, G = R^T R, V <- V R^-1).  A Cholesky pivot that is not
 * > 0 makes that pass use G + s I with s = 11 (D ns + ns (ns+1)) 2^-53 tr(G)
 * (shifted Cholesky-QR, Fukaya et al. 2020) and adds a third pass.
 *   R       optional DEVICE ns x ns row-major output of the upper factor with
 *           V_in = V_out R (NULL = not returned)
 *   passes  optional HOST output: number of passes run (2 or 3)
 * Synchronises (one pivot check per pass).  Errors: FD_ERR_ARG,
 * FD_ERR_BREAKDOWN (the shifted factorisation failed too, e.g. NaN input). */
fd_status fd_orthonormalize(fd_ctx* ctx, double* V, int64_t D, int ns,
                            int64_t ldv, double* R, int* passes);

/* fd_orthonormalize without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * call cudaMalloc, such as applications whose GPU memory is owned by another
 * allocator (a framework's caching allocator that has reserved the device) or
 * serving processes that size their memory once at start-up.  It computes
 * the same Cholesky-QR as fd_orthonormalize (same arguments, same results
 * within rounding) but keeps all scratch in a 32 MiB file-scope device array
 * that every GPU loading the library holds until the process exits.
 *   ns      at most 256 (larger blocks return FD_ERR_ARG)
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  Every call shares the one array: calls
 * that overlap on the GPU (other host threads, other streams) race and must
 * be serialised by the caller.  Every product runs in FP64 arithmetic (the tensor-core products
 * need digit workspaces), whatever fd_set_gemm_mode selected, and the call
 * synchronises the context's stream once per pass (the pivot check).  It
 * never calls cudaMalloc or cudaFree and leaves the context's workspaces
 * untouched (fd_workspace_info reports the same before and after). */
fd_status fd_orthonormalize_noalloc(fd_ctx* ctx, double* V, int64_t D, int ns,
                                    int64_t ldv, double* R, int* passes);

/* Rayleigh-Ritz step (Sec. 2): for an orthonormal D x ns FP64 block V,
 * AV <- H V, Hs = V^T AV, Hs = Q diag(theta) Q^T (theta ascending, FP64
 * Jacobi on the device), V <- V Q, AV <- H V (a second SpMMV, cheaper than
 * rotating AV) and resid_i = ||AV_i - theta_i V_i||_2.  V and AV share the leading dimension ld.  theta and resid
 * are HOST arrays of ns doubles.  Synchronises. */
fd_status fd_rayleigh_ritz(fd_ctx* ctx, const fd_matrix* A, double* V,
                           double* AV, int64_t D, int ns, int64_t ld,
                           double* theta, double* resid);

/* Parameters of the FD loop; zero fields take the defaults in brackets. */
typedef struct {
  int ns;            /* search vectors N_s [nb * ceil(4 N_t / nb)] (Sec. 2: N_s/N_t ~ 4) */
  int max_outer;     /* outer iterations before FD_ERR_NOCONV [60] */
  int n_max;         /* largest filter degree [100000] */
  int lanczos_steps; /* [20] */
  uint64_t seed;     /* start block: SplitMix64 stream 2 (Lanczos: stream 3) [0] */
  int precision;     /* FD_F64: all-FP64 sweeps; FD_F32: FP32 sweeps until the
                        largest wanted residual reaches 100 u32 |H| or fails to
                        halve in two iterations in a row, then the finishing
                        sweeps of `finish`; FD_FF: all sweeps in float-float
                        [FD_F64] */
  double c_n;        /* degree = c_n pi / dtheta [4] */
  double m_l, m_r;   /* window edge = target edge + m (search edge - target edge) [0.5] */
  int verbose;       /* 1: print one line per outer iteration to stderr */
  int cta_warps;     /* batched filter: warps per CTA (4 or 8) [8] */
  int intervals;     /* target and search intervals (Sec. 2):
                        FD_INTERVALS_RITZ: hulls of the N_t and ceil(0.75 N_s)
                        Ritz values nearest the window centre tau;
                        FD_INTERVALS_LEHMANN: the same search interval; each
                        target edge moves out to the Lehmann bound at tau
                        (fd_lehmann_bounds) for the count of wanted Ritz values
                        on its side when that bound lies inside the search
                        interval, so the target interval then provably holds
                        the N_t wanted eigenvalues [FD_INTERVALS_RITZ] */
  double lam_l, lam_r; /* inclusion interval to start from instead of the
                        Lanczos estimate (both 0: Lanczos).  An interval that
                        misses part of the spectrum is widened by 2 % of its
                        width on a side whenever a Ritz value falls outside it
                        on that side [0, 0] */
  int finish;        /* finishing sweeps of the FD_F32 form: FD_FINISH_F64
                        (FP64, the paper's FP64 sweeps) or FD_FINISH_FF
                        (float-float, FP64-like accuracy at FP32 arithmetic
                        rates) [FD_FINISH_F64] */
} fd_options;

enum { FD_FINISH_F64 = 0, FD_FINISH_FF = 1 };

enum { FD_INTERVALS_RITZ = 0, FD_INTERVALS_LEHMANN = 1 };

typedef struct {
  int converged;       /* 1 if all N_t residuals <= tol */
  int iterations;      /* outer iterations (Rayleigh-Ritz steps) */
  int64_t n_spmmv;     /* SpMMVs applied to the full N_s-column block */
  int64_t n_spmmv_f32; /* of which FP32 */
  int final_degree;
  int ns;
  double lam_l, lam_r; /* inclusion interval used last */
  double window_l, window_r;
  double t_total, t_bounds, t_filter, t_ortho, t_rr; /* seconds (CUDA events) */
  double filter_bytes; /* algorithmic bytes of all filter steps (kappa = 5) */
  int used_graph;      /* fd_solve_batched: 1 if the iterations ran as a CUDA graph */
  int64_t n_spmmv_ff;  /* SpMMVs in float-float sweeps */
} fd_result;

/* Lehmann bounds (Lehmann 1963; Sec. 2 takes the FD target and search
 * intervals from Lehmann intervals) of the eigenvalues of H nearest the shift
 * rho, from the search space spanned by the D x ns FP64 block V (device,
 * leading dimension ldv, full column rank; need not be orthonormal).  With
 * W = (H - rho) V the pencil V^T W x = mu W^T W x is solved on the device
 * (diagonal scaling, Cholesky, Jacobi); its negative mu give
 *   below[k] = rho + 1/mu  <=  the (k+1)-th eigenvalue below rho,
 * its positive mu
 *   above[k] = rho + 1/mu  >=  the (k+1)-th eigenvalue above rho,
 * both nearest rho first.  below / above: HOST arrays of ns doubles;
 * n_below + n_above <= ns.  V needs no alignment (it is copied into a
 * workspace of 2 D ns doubles).  Synchronises.  Errors: FD_ERR_ARG,
 * FD_ERR_BREAKDOWN (W numerically rank deficient, e.g. V spans an exact
 * eigenvector with eigenvalue rho). */
fd_status fd_lehmann_bounds(fd_ctx* ctx, const fd_matrix* A, const double* V, int64_t D, int ns,
                            int64_t ldv, double rho, double* below, int* n_below, double* above,
                            int* n_above);

/* Filter diagonalization (Sec. 2, Alg. 1): the n_target eigenpairs of H
 * nearest the centre of the window [a, b] to residual ||H x - theta x||_2 <=
 * tol.  `degree` is the first and smallest filter degree; later degrees and
 * the target/search intervals follow fd_options (intervals: the Ritz-value
 * heuristic, or the paper's Lehmann intervals).
 *   theta, resid  HOST arrays of n_target doubles (ascending theta)
 *   X             optional DEVICE D x n_target FP64 row-major eigenvectors
 *                 (largest-magnitude entry positive), or NULL
 * Returns FD_ERR_NOCONV (with the outputs filled) if max_outer is reached. */
fd_status fd_solve(fd_ctx* ctx, const fd_matrix* A, double a, double b,
                   int n_target, int nb, int degree, double tol,
                   const fd_options* opt, fd_result* res, double* theta,
                   double* resid, double* X, int64_t ldx);

/* State of an interrupted FD solve (the paper's runs last up to 26 hours,
 * Table 6): everything the loop carries from one outer iteration to the next
 * besides the search block itself.  Zero-initialise it to start a solve. */
typedef struct {
  int iteration;        /* outer iterations done (0: start from scratch) */
  int converged;        /* 1 once the solve has converged */
  int degree;           /* degree of the next filter */
  int use_f32;          /* FP32 sweeps still on (FD_F32 precision form) */
  int stall;            /* iterations in a row without halving the residual */
  double lam_l, lam_r;  /* inclusion interval */
  double widen;         /* its widening step */
  double norm_h;        /* |H| estimate of the FP32 switch */
  double window_l, window_r; /* window of the last filter */
  double prev_max;      /* largest wanted residual of the last iteration */
  int64_t n_spmmv, n_spmmv_f32;
  double filter_bytes;
  int64_t D;            /* consistency checks on resume */
  int ns;
  uint64_t seed;
  int64_t n_spmmv_ff;
} fd_checkpoint;

/* fd_solve in slices: starting from *ck (iteration 0: a fresh solve; else the
 * state a previous call wrote, with the filtered search block in Vck), run at
 * most max_iter outer iterations.  If the solve has not converged by then, it
 * stops right after a filter application, writes the filtered D x N_s block
 * to Vck (DEVICE, row-major, leading dimension N_s, caller-owned) and the
 * loop's scalars to *ck, and returns FD_ERR_NOCONV with ck->converged = 0;
 * the caller may save both (e.g. to a file) and resume later, in another
 * process or context, with the same matrix, window, n_target, nb, degree,
 * tol and options.  The resumed solve repeats the uninterrupted one's
 * arithmetic exactly: the same iterations, degrees and eigenvalues.  On
 * convergence the outputs are those of fd_solve, ck->converged = 1 and the
 * call returns FD_OK.  Reaching opt->max_outer iterations in total returns
 * FD_ERR_NOCONV with ck->converged = 0 and no pause.  res counts SpMMVs from
 * the start of the solve and times for this call only.  Errors: FD_ERR_ARG
 * also for a checkpoint whose D, N_s or seed differ from this solve's. */
fd_status fd_solve_checkpointed(fd_ctx* ctx, const fd_matrix* A, double a, double b,
                                int n_target, int nb, int degree, double tol,
                                const fd_options* opt, int max_iter, fd_checkpoint* ck,
                                double* Vck, fd_result* res, double* theta, double* resid,
                                double* X, int64_t ldx);

/* One problem of a batch: the window [a, b], the number of wanted pairs, the
 * seed of its start block and Lanczos vector, and optional per-instance
 * interval constants. */
typedef struct {
  double a, b;
  int n_target;
  uint64_t seed;
  double c_n, m_l, m_r; /* this instance's degree constant and window margins
                           (0: fd_options' values), e.g. the learned ones */
} fd_problem;

/* Filter diagonalization of n_inst independent problems at once (Alg. 1 per
 * instance, instances of different sizes).  Each outer iteration of all
 * unconverged instances runs as one CUDA graph: one persistent cooperative
 * kernel applies the Chebyshev filters of every bundle of every instance (all
 * degree steps, a grid-wide barrier between steps), batched Cholesky-QR and
 * Rayleigh-Ritz kernels cover all instances per launch, and all Ritz values
 * and residuals are copied to the host once.  Instances drop out when they
 * converge.  The per-instance intervals and degrees follow fd_solve's
 * heuristic.  Matrices must be built with sigma = 1; N_s per instance (opt->ns
 * or nb ceil(4 n_target / nb)) must be at most 96; nb in {2, ..., 64}.
 * A graph cannot be captured on the legacy default stream: on a context
 * without a stream the solve runs on a private stream of its own, created for
 * the call and ordered after the work already queued on the legacy stream.
 *   res         n_inst results
 *   theta/resid HOST arrays holding sum(n_target) doubles, instance after
 *               instance, ascending theta within an instance (NaN/inf for an
 *               instance that did not converge)
 * Returns FD_ERR_NOCONV if any instance failed to converge in max_outer. */
fd_status fd_solve_batched(fd_ctx* ctx, int n_inst, const fd_matrix* const* A,
                           const fd_problem* prob, int nb, int degree, double tol,
                           const fd_options* opt, fd_result* res, double* theta,
                           double* resid);

/* Autotuner of the batched filter: for the matrices given by n_inst spec
 * strings, times the persistent batched filter (degree `probe_degree`, FP64)
 * for every combination of block width nb in {8, 16, 32, 64} (with N_s =
 * nb ceil(4 n_target / nb) <= 96), SELL chunk height C in {32, 64, 128} and
 * CTA shape (4 or 8 warps), and returns the fastest with its throughput in
 * algorithmic GB/s (Eq. EstimateT bytes).  Builds and frees its own matrices. */
fd_status fd_tune_batched(fd_ctx* ctx, int n_inst, const char* const* specs, int n_target,
                          int probe_degree, int* nb, int* C, int* cta_warps, double* gbs);

/* Communication metrics of distributed SpMV (Sec. 3.1, Eqs. chi) for the
 * uniform distribution of the rows over n_p processes: process p owns rows
 * [floor(p D / n_p), floor((p + 1) D / n_p)).  Per process, the number of
 * distinct vector entries its rows read (stored entries with a nonzero value)
 * inside its own range (n_vm) and outside it (n_vc); and
 *   chi[0] = chi_1 = max_p n_vc / n_vm,  chi[1] = chi_2 = sum_p n_vc / D,
 *   chi[2] = chi_3 = n_p max_p n_vc / D   (all 0 for n_p = 1).
 * The matrix must be in its original row order (built with sigma = 1, else
 * FD_ERR_ARG); 1 <= n_p <= D.  n_vc, n_vm: HOST arrays of n_p int64 or NULL;
 * chi: HOST array of 3 doubles.  Uses a D-bit device workspace.  Synchronises. */
fd_status fd_comm_metrics(fd_ctx* ctx, const fd_matrix* A, int n_p, int64_t* n_vc,
                          int64_t* n_vm, double* chi);

/* Kernel-polynomial moments mu_m = (1/(R D)) sum_r r^T T_m(A~) r, m <
 * n_moments, with R = n_random normal-like random vectors (SplitMix64 stream
 * 4, `seed`) and A~ = alpha H + beta I (Sec. 4.1 computes the DOS with KPM).
 * n_random in {2, 4, 8, 16, 32, 64}; mu is a HOST array of n_moments doubles.
 * Synchronises. */
fd_status fd_kpm_moments(fd_ctx* ctx, const fd_matrix* A, int n_moments,
                         int n_random, uint64_t seed, double alpha, double beta,
                         double* mu);

/* ------------------------------------------------------- filter-parameter predictor
 * A 64-128-128-3 perceptron (FP32 weights, GELU activations) that predicts
 * the degree constant c_n and the window margins m_l, m_r of fd_solve's
 * interval heuristic from kernel-polynomial density-of-states moments and the
 * target window.  The paper has no learned component; the network is trained
 * on logs of FD runs by the project's own kernels.  Parameters are one FP32
 * device vector of fd_mlp_num_params() numbers: W1 (64x128 row-major), b1,
 * W2 (128x128), b2, W3 (128x3), b3. */
int fd_mlp_num_params(void);
/* Y (device B x 3) = network(X (device B x 64)). */
fd_status fd_mlp_forward(fd_ctx* ctx, const float* params, const float* X, int B, float* Y);
/* Gradient (device, fd_mlp_num_params() floats) of the mean-squared error
 * between the outputs and T (device B x 3); loss is a HOST float. */
fd_status fd_mlp_gradient(fd_ctx* ctx, const float* params, const float* X, const float* T,
                          int B, float* grad, float* loss);
/* One Adam step (Kingma & Ba; b1 = 0.9, b2 = 0.999, eps = 1e-8, step >= 1 is
 * the 1-based update count) on the batch; m, v: device moment vectors (start
 * at zero); loss: optional HOST float (the loss before the update). */
fd_status fd_mlp_train_step(fd_ctx* ctx, float* params, float* m, float* v, const float* X,
                            const float* T, int B, int step, float lr, float* loss);
/* The 64 input features of one problem (HOST floats): the 48 KPM moments of
 * the matrix scaled by its inclusion interval (16 random vectors of `seed`),
 * the scaled window ends and width, n_target/100, log10(D)/8, nnz/(32 D), the
 * interval ends relative to the larger of their magnitudes, log10(1 + KPM
 * eigenvalue count in [a, b])/6, min(4, count/ns), nb/128, ns/1024, zeros. */
fd_status fd_filter_features(fd_ctx* ctx, const fd_matrix* A, double a, double b, int n_target,
                             int nb, int ns, uint64_t seed, float* feat);
/* c_n = exp(y0) in [1, 16], m_l = y1 and m_r = y2 clipped to [0.05, 0.95];
 * a non-finite output selects the plain heuristic (4, 0.5, 0.5) and sets
 * *fallback = 1.  feat: HOST 64 floats. */
fd_status fd_predict_filter_params(fd_ctx* ctx, const float* params, const float* feat,
                                   double* c_n, double* m_l, double* m_r, int* fallback);

#ifdef __cplusplus
}
#endif

#endif /* FD_H */
