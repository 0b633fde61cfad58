"""Python binding of libfd, the GB300 filter-diagonalization library.

Argument marshalling only: every step of the FD hot path runs in the CUDA
kernels of ``libfd.so`` (built by ``paper_2209_01974_gb300.build``).  Device
blocks are torch CUDA tensors (row-major, unit column stride, leading
dimension = ``stride(0)``); host outputs are NumPy arrays.  The functions keep
the names of the C ABI in ``include/fd.h``.  There is no fallback: if the
library is missing, importing the binding raises ``ImportError``.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run paper_2209_01974_gb300.build.build() "
                      "(or __graft_entry__.build()) first")

_lib = ctypes.CDLL(LIB_PATH)

FD_OK, FD_ERR_ARG, FD_ERR_CUDA, FD_ERR_OOM, FD_ERR_NOCONV, FD_ERR_BREAKDOWN, FD_ERR_TIMEOUT, \
    FD_ERR_BOUNDS = range(8)
FD_F64, FD_F32, FD_FF = 0, 1, 2
STATUS_NAMES = {0: "FD_OK", 1: "FD_ERR_ARG", 2: "FD_ERR_CUDA", 3: "FD_ERR_OOM", 4: "FD_ERR_NOCONV",
                5: "FD_ERR_BREAKDOWN", 6: "FD_ERR_TIMEOUT", 7: "FD_ERR_BOUNDS"}

_vp, _i64, _i32, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pi32 = ctypes.POINTER(ctypes.c_int32)


class fd_matrix_info(ctypes.Structure):
    _fields_ = [("D", _i64), ("nnz", _i64), ("nnz_sell", _i64), ("n_chunks", _i64),
                ("C", ctypes.c_int32), ("sigma", ctypes.c_int32), ("max_row", ctypes.c_int32),
                ("identity_perm", ctypes.c_int32), ("gersh_lo", _dbl), ("gersh_hi", _dbl)]


class fd_options(ctypes.Structure):
    _fields_ = [("ns", _i32), ("max_outer", _i32), ("n_max", _i32), ("lanczos_steps", _i32),
                ("seed", ctypes.c_uint64), ("precision", _i32), ("c_n", _dbl), ("m_l", _dbl),
                ("m_r", _dbl), ("verbose", _i32), ("cta_warps", _i32), ("intervals", _i32),
                ("lam_l", _dbl), ("lam_r", _dbl), ("finish", _i32)]

FD_INTERVALS_RITZ, FD_INTERVALS_LEHMANN = 0, 1
FD_FINISH_F64, FD_FINISH_FF = 0, 1


class fd_checkpoint(ctypes.Structure):
    _fields_ = [("iteration", _i32), ("converged", _i32), ("degree", _i32), ("use_f32", _i32),
                ("stall", _i32), ("lam_l", _dbl), ("lam_r", _dbl), ("widen", _dbl), ("norm_h", _dbl),
                ("window_l", _dbl), ("window_r", _dbl), ("prev_max", _dbl), ("n_spmmv", _i64),
                ("n_spmmv_f32", _i64), ("filter_bytes", _dbl), ("D", _i64), ("ns", _i32),
                ("seed", ctypes.c_uint64), ("n_spmmv_ff", _i64)]


class fd_problem(ctypes.Structure):
    _fields_ = [("a", _dbl), ("b", _dbl), ("n_target", _i32), ("seed", ctypes.c_uint64),
                ("c_n", _dbl), ("m_l", _dbl), ("m_r", _dbl)]


class fd_result(ctypes.Structure):
    _fields_ = [("converged", _i32), ("iterations", _i32), ("n_spmmv", _i64),
                ("n_spmmv_f32", _i64), ("final_degree", _i32), ("ns", _i32), ("lam_l", _dbl),
                ("lam_r", _dbl), ("window_l", _dbl), ("window_r", _dbl), ("t_total", _dbl),
                ("t_bounds", _dbl), ("t_filter", _dbl), ("t_ortho", _dbl), ("t_rr", _dbl),
                ("filter_bytes", _dbl), ("used_graph", _i32), ("n_spmmv_ff", _i64)]


_SIGS = {
    "fd_create": (_i32, [ctypes.POINTER(_vp), _i32, _vp]),
    "fd_destroy": (_i32, [_vp]),
    "fd_set_stream": (_i32, [_vp, _vp]),
    "fd_last_error": (ctypes.c_char_p, [_vp]),
    "fd_kernel_launches": (_i64, [_vp]),
    "fd_workspace_info": (_i32, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_i64)]),
    "fd_set_workspace_limit": (_i32, [_vp, ctypes.c_size_t]),
    "fd_set_debug_checks": (_i32, [_vp, _i32]),
    "fd_debug_set_sell_column": (_i32, [_vp, _vp, _i64, ctypes.c_int32]),
    "fd_build_matrix": (_i32, [_vp, ctypes.c_char_p, ctypes.POINTER(_vp)]),
    "fd_build_matrix_sell": (_i32, [_vp, ctypes.c_char_p, _i32, _i32, ctypes.POINTER(_vp)]),
    "fd_matrix_from_csr": (_i32, [_vp, _i64, _pi64, _pi32, _pd, _i32, _i32, ctypes.POINTER(_vp)]),
    "fd_matrix_free": (_i32, [_vp]),
    "fd_matrix_get_info": (_i32, [_vp, ctypes.POINTER(fd_matrix_info)]),
    "fd_matrix_to_csr": (_i32, [_vp, _vp, _pi64, _pi32, _pd]),
    "fd_matrix_perm": (_i32, [_vp, _vp, _pi64]),
    "fd_spectral_bounds": (_i32, [_vp, _vp, _i32, ctypes.c_uint64, _pd, _pd]),
    "fd_filter": (_i32, [_vp, _vp, _i32, _vp, _i64, _i32, _i32, _pd, _dbl, _dbl, _vp, _vp, _i64]),
    "fd_filter_coeffs": (_i32, [_dbl, _dbl, _i32, _pd]),
    "fd_spmmv": (_i32, [_vp, _vp, _i32, _vp, _i64, _vp, _i64, _i32]),
    "fd_set_gemm_mode": (_i32, [_vp, _i32]),
    "fd_check_bounded_wait": (_i32, [_vp, _i32]),
    "fd_comm_metrics": (_i32, [_vp, _vp, _i32, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64), _pd]),
    "fd_gram": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i32, _i32, _vp, _i32]),
    "fd_rotate": (_i32, [_vp, _vp, _i64, _i64, _i32, _vp, _i32]),
    "fd_copy_block": (_i32, [_vp, _vp, _i32, _i64, _vp, _i32, _i64, _i64, _i32]),
    "fd_orthonormalize": (_i32, [_vp, _vp, _i64, _i32, _i64, _vp, ctypes.POINTER(_i32)]),
    "fd_orthonormalize_noalloc": (_i32, [_vp, _vp, _i64, _i32, _i64, _vp, ctypes.POINTER(_i32)]),
    "fd_rayleigh_ritz": (_i32, [_vp, _vp, _vp, _vp, _i64, _i32, _i64, _pd, _pd]),
    "fd_solve": (_i32, [_vp, _vp, _dbl, _dbl, _i32, _i32, _i32, _dbl, ctypes.POINTER(fd_options),
                        ctypes.POINTER(fd_result), _pd, _pd, _vp, _i64]),
    "fd_solve_checkpointed": (_i32, [_vp, _vp, _dbl, _dbl, _i32, _i32, _i32, _dbl, ctypes.POINTER(fd_options),
                                     _i32, ctypes.POINTER(fd_checkpoint), _vp, ctypes.POINTER(fd_result),
                                     _pd, _pd, _vp, _i64]),
    "fd_solve_batched": (_i32, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(fd_problem), _i32,
                                _i32, _dbl, ctypes.POINTER(fd_options), ctypes.POINTER(fd_result),
                                _pd, _pd]),
    "fd_tune_batched": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_char_p), _i32, _i32,
                               ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                               ctypes.POINTER(_dbl)]),
    "fd_mlp_num_params": (_i32, []),
    "fd_mlp_forward": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "fd_mlp_gradient": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, ctypes.POINTER(ctypes.c_float)]),
    "fd_mlp_train_step": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_float,
                                 ctypes.POINTER(ctypes.c_float)]),
    "fd_filter_features": (_i32, [_vp, _vp, _dbl, _dbl, _i32, _i32, _i32, ctypes.c_uint64,
                                  ctypes.POINTER(ctypes.c_float)]),
    "fd_predict_filter_params": (_i32, [_vp, _vp, ctypes.POINTER(ctypes.c_float), _pd, _pd, _pd,
                                        ctypes.POINTER(_i32)]),
    "fd_kpm_moments": (_i32, [_vp, _vp, _i32, _i32, ctypes.c_uint64, _dbl, _dbl, _pd]),
    "fd_lehmann_bounds": (_i32, [_vp, _vp, _vp, _i64, _i32, _i64, _dbl, _pd, ctypes.POINTER(_i32), _pd,
                                 ctypes.POINTER(_i32)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = sorted(_SIGS)


class FDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(ctx, status):
    if status != FD_OK:
        msg = _lib.fd_last_error(ctx.handle if ctx is not None else None)
        raise FDError(status, msg.decode() if msg else "")


def _dptr(a, dtype):
    return a.ctypes.data_as(ctypes.POINTER(dtype))


def _block(t, name):
    """(pointer, ld, D, ncols, prec) of a row-major CUDA tensor block: a 2-D
    float64 or float32 tensor, or a D x n x 2 float32 tensor holding
    float-float values (hi, lo) (FD_FF; ld counted in elements)."""
    import torch
    if (isinstance(t, torch.Tensor) and t.is_cuda and t.dim() == 3 and t.shape[2] == 2
            and t.dtype == torch.float32):
        if t.stride(2) != 1 or t.stride(1) != 2 or t.stride(0) % 2:
            raise ValueError(f"{name}: float-float blocks need (hi, lo) pairs in row-major rows")
        return t.data_ptr(), t.stride(0) // 2, t.shape[0], t.shape[1], FD_FF
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D CUDA tensor")
    if t.stride(1) != 1:
        raise ValueError(f"{name} must have unit column stride")
    if t.dtype == torch.float64:
        prec = FD_F64
    elif t.dtype == torch.float32:
        prec = FD_F32
    else:
        raise ValueError(f"{name} must be float64 or float32")
    return t.data_ptr(), t.stride(0), t.shape[0], t.shape[1], prec


class Ctx:
    def __init__(self, device=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        h = _vp()
        st = _lib.fd_create(ctypes.byref(h), device, _vp(stream))
        if st != FD_OK:
            raise FDError(st, f"fd_create(device={device}) failed")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            _lib.fd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def kernel_launches(self):
        return _lib.fd_kernel_launches(self.handle)

    @property
    def workspace(self):
        """(bytes held by the grow-only workspaces, cudaMalloc calls made for them)."""
        b, n = ctypes.c_size_t(0), _i64(0)
        _check(self, _lib.fd_workspace_info(self.handle, ctypes.byref(b), ctypes.byref(n)))
        return b.value, n.value


class Matrix:
    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.handle = handle

    def free(self):
        if self.handle:
            _lib.fd_matrix_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def info(self):
        inf = fd_matrix_info()
        _check(self.ctx, _lib.fd_matrix_get_info(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in fd_matrix_info._fields_}

    @property
    def D(self):
        return self.info["D"]


def fd_create(device=0, stream=None):
    return Ctx(device, stream)


def fd_set_stream(ctx, stream):
    _check(ctx, _lib.fd_set_stream(ctx.handle, _vp(stream)))


def fd_build_matrix(ctx, spec, C=32, sigma=1):
    h = _vp()
    _check(ctx, _lib.fd_build_matrix_sell(ctx.handle, spec.encode(), C, sigma, ctypes.byref(h)))
    return Matrix(ctx, h)


def fd_matrix_from_csr(ctx, rowptr, col, val, C=32, sigma=1):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    h = _vp()
    _check(ctx, _lib.fd_matrix_from_csr(ctx.handle, len(rowptr) - 1, _dptr(rowptr, ctypes.c_int64),
                                        _dptr(col, ctypes.c_int32), _dptr(val, ctypes.c_double),
                                        C, sigma, ctypes.byref(h)))
    return Matrix(ctx, h)


def fd_matrix_to_csr(ctx, A):
    inf = A.info
    rowptr = np.empty(inf["D"] + 1, dtype=np.int64)
    col = np.empty(max(1, inf["nnz"]), dtype=np.int32)
    val = np.empty(max(1, inf["nnz"]), dtype=np.float64)
    _check(ctx, _lib.fd_matrix_to_csr(ctx.handle, A.handle, _dptr(rowptr, ctypes.c_int64),
                                      _dptr(col, ctypes.c_int32), _dptr(val, ctypes.c_double)))
    return rowptr, col[:inf["nnz"]], val[:inf["nnz"]]


def fd_matrix_perm(ctx, A):
    perm = np.empty(A.D, dtype=np.int64)
    _check(ctx, _lib.fd_matrix_perm(ctx.handle, A.handle, _dptr(perm, ctypes.c_int64)))
    return perm


def fd_spectral_bounds(ctx, A, steps=20, seed=0):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(ctx, _lib.fd_spectral_bounds(ctx.handle, A.handle, steps, seed, ctypes.byref(lo),
                                        ctypes.byref(hi)))
    return lo.value, hi.value


def fd_filter(ctx, A, V, mu, alpha, beta, W1, W2):
    """V <- p(alpha A + beta) V in place; W1, W2: workspaces of V's shape and dtype."""
    pv, ldv, D, nb, prec = _block(V, "V")
    p1, ldw, _, _, prec1 = _block(W1, "W1")
    p2, ldw2, _, _, prec2 = _block(W2, "W2")
    if ldw != ldw2 or prec1 != prec or prec2 != prec:
        raise ValueError("W1 and W2 need the same leading dimension and V's dtype")
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    _check(ctx, _lib.fd_filter(ctx.handle, A.handle, prec, _vp(pv), ldv, nb, len(mu) - 1,
                               _dptr(mu, ctypes.c_double), alpha, beta, _vp(p1), _vp(p2), ldw))


def fd_filter_coeffs(x_l, x_r, n):
    mu = np.empty(n + 1)
    st = _lib.fd_filter_coeffs(x_l, x_r, n, _dptr(mu, ctypes.c_double))
    if st != FD_OK:
        raise FDError(st, "fd_filter_coeffs: need n >= 2 and x_l < x_r")
    return mu


def fd_spmmv(ctx, A, X, Y):
    px, ldx, D, nb, prec = _block(X, "X")
    py, ldy, _, _, precy = _block(Y, "Y")
    if precy != prec:
        raise ValueError("X and Y must have the same dtype")
    _check(ctx, _lib.fd_spmmv(ctx.handle, A.handle, prec, _vp(px), ldx, _vp(py), ldy, nb))


FD_GEMM_AUTO, FD_GEMM_FP64, FD_GEMM_OZAKI = 0, 1, 2


def fd_set_workspace_limit(ctx, limit_bytes):
    """Cap the context's workspace bytes (0 = no cap); growth beyond it is FD_ERR_OOM."""
    _check(ctx, _lib.fd_set_workspace_limit(ctx.handle, int(limit_bytes)))


def fd_set_debug_checks(ctx, on=True):
    _check(ctx, _lib.fd_set_debug_checks(ctx.handle, 1 if on else 0))


def fd_debug_set_sell_column(ctx, A, entry, col):
    _check(ctx, _lib.fd_debug_set_sell_column(ctx.handle, A.handle, int(entry), int(col)))


def fd_set_gemm_mode(ctx, mode):
    """mode: FD_GEMM_AUTO, FD_GEMM_FP64 or FD_GEMM_OZAKI (or 'auto'/'fp64'/'ozaki')."""
    if isinstance(mode, str):
        mode = {"auto": 0, "fp64": 1, "ozaki": 2}[mode]
    _check(ctx, _lib.fd_set_gemm_mode(ctx.handle, mode))


def fd_check_bounded_wait(ctx, limit_us=100000):
    """The bounded-wait diagnostic; returns its fd_status (FD_ERR_TIMEOUT when the
    wait gave up as designed) instead of raising."""
    return _lib.fd_check_bounded_wait(ctx.handle, int(limit_us))


def fd_comm_metrics(ctx, A, n_p):
    """Communication metrics of distributed SpMV over n_p processes (Sec. 3.1):
    (chi_1, chi_2, chi_3, n_vc, n_vm) with int64 arrays n_vc, n_vm per process."""
    n_vc = np.zeros(n_p, dtype=np.int64)
    n_vm = np.zeros(n_p, dtype=np.int64)
    chi = np.zeros(3)
    _check(ctx, _lib.fd_comm_metrics(ctx.handle, A.handle, int(n_p),
                                     n_vc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     n_vm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     _dptr(chi, ctypes.c_double)))
    return float(chi[0]), float(chi[1]), float(chi[2]), n_vc, n_vm


def fd_gram(ctx, X, Y):
    """C = X^T Y for float64 CUDA blocks X (D x m) and Y (D x n); returns C (m x n)."""
    import torch
    px, ldx, D, m, _ = _block(X, "X")
    py, ldy, D2, n, _ = _block(Y, "Y")
    if D != D2:
        raise ValueError("X and Y need the same number of rows")
    C = torch.empty((m, n), dtype=torch.float64, device=X.device)
    _check(ctx, _lib.fd_gram(ctx.handle, _vp(px), ldx, _vp(py), ldy, D, m, n, _vp(C.data_ptr()), n))
    return C


def fd_rotate(ctx, V, M, upper=False):
    """V <- V M in place (V: D x n float64 CUDA block, M: n x n contiguous)."""
    pv, ldv, D, n, _ = _block(V, "V")
    if not M.is_contiguous() or tuple(M.shape) != (n, n):
        raise ValueError("M must be a contiguous n x n tensor")
    _check(ctx, _lib.fd_rotate(ctx.handle, _vp(pv), ldv, D, n, _vp(M.data_ptr()), 1 if upper else 0))


def fd_copy_block(ctx, src, dst):
    """dst <- src (same shape), converting between float64 and float32 or
    float-float (D x n x 2 float32) blocks."""
    ps, lds, D, n, sp = _block(src, "src")
    pd, ldd, D2, n2, dp = _block(dst, "dst")
    if (D, n) != (D2, n2):
        raise ValueError("src and dst shapes differ")
    _check(ctx, _lib.fd_copy_block(ctx.handle, _vp(ps), sp, lds, _vp(pd), dp, ldd, D, n))


def fd_orthonormalize(ctx, V, R=None):
    """In-place Cholesky-QR of the FP64 block V; returns the number of passes."""
    pv, ldv, D, ns, prec = _block(V, "V")
    if prec != FD_F64:
        raise ValueError("fd_orthonormalize works on float64 blocks")
    passes = ctypes.c_int()
    _check(ctx, _lib.fd_orthonormalize(ctx.handle, _vp(pv), D, ns, ldv,
                                       _vp(R.data_ptr() if R is not None else None),
                                       ctypes.byref(passes)))
    return passes.value


def fd_orthonormalize_noalloc(ctx, V, R=None):
    """fd_orthonormalize for callers that cannot let the library allocate device
    memory: scratch lives in the library's fixed 32 MiB device array (ns <= 256)."""
    pv, ldv, D, ns, prec = _block(V, "V")
    if prec != FD_F64:
        raise ValueError("fd_orthonormalize_noalloc works on float64 blocks")
    passes = ctypes.c_int()
    _check(ctx, _lib.fd_orthonormalize_noalloc(ctx.handle, _vp(pv), D, ns, ldv,
                                               _vp(R.data_ptr() if R is not None else None),
                                               ctypes.byref(passes)))
    return passes.value


def fd_rayleigh_ritz(ctx, A, V, AV):
    pv, ld, D, ns, prec = _block(V, "V")
    pa, lda, _, _, _ = _block(AV, "AV")
    if lda != ld or prec != FD_F64:
        raise ValueError("V and AV must be float64 with the same leading dimension")
    theta = np.empty(ns)
    resid = np.empty(ns)
    _check(ctx, _lib.fd_rayleigh_ritz(ctx.handle, A.handle, _vp(pv), _vp(pa), D, ns, ld,
                                      _dptr(theta, ctypes.c_double), _dptr(resid, ctypes.c_double)))
    return theta, resid


def _options(opts):
    """fd_options from keyword arguments ('f32'/'f64' precision and
    'ritz'/'lehmann' intervals accepted as strings)."""
    o = fd_options()
    for k, v in opts.items():
        if k == "precision" and isinstance(v, str):
            v = {"f64": FD_F64, "fp64": FD_F64, "float64": FD_F64, "f32": FD_F32, "fp32": FD_F32,
                 "float32": FD_F32, "ff": FD_FF}[v]
        if k == "finish" and isinstance(v, str):
            v = {"f64": FD_FINISH_F64, "ff": FD_FINISH_FF}[v]
        if k == "intervals" and isinstance(v, str):
            v = {"ritz": FD_INTERVALS_RITZ, "lehmann": FD_INTERVALS_LEHMANN}[v]
        setattr(o, k, v)
    return o


def fd_lehmann_bounds(ctx, A, V, rho):
    """Lehmann bounds at the shift rho from the search space of the float64
    CUDA block V: (below, above), nearest rho first."""
    pv, ldv, D, ns, prec = _block(V, "V")
    if prec != FD_F64:
        raise ValueError("V must be float64")
    below, above = np.empty(ns), np.empty(ns)
    nb_, na_ = _i32(0), _i32(0)
    _check(ctx, _lib.fd_lehmann_bounds(ctx.handle, A.handle, _vp(pv), D, ns, ldv, float(rho),
                                       _dptr(below, ctypes.c_double), ctypes.byref(nb_),
                                       _dptr(above, ctypes.c_double), ctypes.byref(na_)))
    return below[:nb_.value].copy(), above[:na_.value].copy()


def fd_solve(ctx, A, a, b, n_target, nb, degree, tol, X=None, raise_noconv=True, **opts):
    """Filter diagonalization; returns (theta, resid, result dict).  X: optional
    CUDA float64 tensor (D x n_target) that receives the eigenvectors."""
    o = _options(opts)
    res = fd_result()
    theta = np.empty(n_target)
    resid = np.empty(n_target)
    px, ldx = (None, 0)
    if X is not None:
        px, ldx, _, _, _ = _block(X, "X")
    st = _lib.fd_solve(ctx.handle, A.handle, a, b, n_target, nb, degree, tol, ctypes.byref(o),
                       ctypes.byref(res), _dptr(theta, ctypes.c_double), _dptr(resid, ctypes.c_double),
                       _vp(px), ldx)
    if st != FD_OK and not (st == FD_ERR_NOCONV and not raise_noconv):
        _check(ctx, st)
    return theta, resid, {k: getattr(res, k) for k, _ in fd_result._fields_}


class Checkpoint:
    """An interrupted solve: the fd_checkpoint scalars and the filtered search
    block (CUDA float64 tensor, D x N_s).  save/load write and read one .npz
    file (host copies of both)."""

    def __init__(self, state=None, V=None):
        self.state = state if state is not None else fd_checkpoint()
        self.V = V

    def save(self, path):
        fields = {k: getattr(self.state, k) for k, _ in fd_checkpoint._fields_}
        np.savez(path, V=self.V.cpu().numpy(), **{f"s_{k}": v for k, v in fields.items()})

    @classmethod
    def load(cls, path):
        import torch
        z = np.load(path)
        st = fd_checkpoint()
        for k, _ in fd_checkpoint._fields_:
            setattr(st, k, type(getattr(st, k))(z[f"s_{k}"].item()))
        return cls(st, torch.from_numpy(z["V"]).cuda())


def fd_solve_checkpointed(ctx, A, a, b, n_target, nb, degree, tol, max_iter, ckpt=None, X=None, **opts):
    """fd_solve for at most max_iter outer iterations from the checkpoint ckpt
    (None: a fresh solve).  Returns (theta, resid, result dict, ckpt); the
    solve has converged when ckpt.state.converged == 1."""
    import torch
    o = _options(opts)
    ns = o.ns if o.ns > 0 else nb * -(-4 * n_target // nb)
    if ckpt is None:
        ckpt = Checkpoint(V=torch.empty((A.D, ns), dtype=torch.float64, device="cuda"))
    pv, ldv, _, _, _ = _block(ckpt.V, "V")
    if ldv != ns or ckpt.V.shape[1] != ns:
        raise ValueError("the checkpoint block must be contiguous D x N_s")
    res = fd_result()
    theta = np.empty(n_target)
    resid = np.empty(n_target)
    px, ldx = (None, 0)
    if X is not None:
        px, ldx, _, _, _ = _block(X, "X")
    st = _lib.fd_solve_checkpointed(ctx.handle, A.handle, a, b, n_target, nb, degree, tol, ctypes.byref(o),
                                    int(max_iter), ctypes.byref(ckpt.state), _vp(pv), ctypes.byref(res),
                                    _dptr(theta, ctypes.c_double), _dptr(resid, ctypes.c_double), _vp(px), ldx)
    if st != FD_OK and st != FD_ERR_NOCONV:
        _check(ctx, st)
    return theta, resid, {k: getattr(res, k) for k, _ in fd_result._fields_}, ckpt


def fd_solve_batched(ctx, mats, problems, nb, degree, tol, raise_noconv=True, **opts):
    """problems: list of (a, b, n_target, seed) or (a, b, n_target, seed, c_n, m_l,
    m_r).  Returns (list of (theta, resid), list of result dicts)."""
    n = len(mats)
    arr = (_vp * n)(*[m.handle for m in mats])
    pr = (fd_problem * n)(*[fd_problem(*p) for p in problems])
    o = _options(opts)
    res = (fd_result * n)()
    tot = sum(p[2] for p in problems)
    theta = np.empty(tot)
    resid = np.empty(tot)
    st = _lib.fd_solve_batched(ctx.handle, n, arr, pr, nb, degree, tol, ctypes.byref(o), res,
                               _dptr(theta, ctypes.c_double), _dptr(resid, ctypes.c_double))
    if st != FD_OK and not (st == FD_ERR_NOCONV and not raise_noconv):
        _check(ctx, st)
    out, o_ = [], 0
    for p in problems:
        out.append((theta[o_:o_ + p[2]].copy(), resid[o_:o_ + p[2]].copy()))
        o_ += p[2]
    return out, [{k: getattr(r, k) for k, _ in fd_result._fields_} for r in res]


def fd_tune_batched(ctx, specs, n_target, probe_degree=20):
    n = len(specs)
    arr = (ctypes.c_char_p * n)(*[s.encode() for s in specs])
    nb, C, w, g = _i32(), _i32(), _i32(), _dbl()
    _check(ctx, _lib.fd_tune_batched(ctx.handle, n, arr, n_target, probe_degree, ctypes.byref(nb),
                                     ctypes.byref(C), ctypes.byref(w), ctypes.byref(g)))
    return {"nb": nb.value, "C": C.value, "cta_warps": w.value, "gbs": g.value}


def fd_kpm_moments(ctx, A, n_moments, n_random, seed, alpha, beta):
    mu = np.empty(n_moments)
    _check(ctx, _lib.fd_kpm_moments(ctx.handle, A.handle, n_moments, n_random, seed, alpha, beta,
                                    _dptr(mu, ctypes.c_double)))
    return mu


# ---------------------------------------------------------------- predictor
def fd_mlp_num_params():
    return _lib.fd_mlp_num_params()


def _f32(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor")
    return _vp(t.data_ptr())


def fd_mlp_forward(ctx, params, X):
    import torch
    Y = torch.empty((X.shape[0], 3), dtype=torch.float32, device=X.device)
    _check(ctx, _lib.fd_mlp_forward(ctx.handle, _f32(params, "params"), _f32(X, "X"), X.shape[0],
                                    _f32(Y, "Y")))
    return Y


def fd_mlp_gradient(ctx, params, X, T):
    import torch
    g = torch.empty_like(params)
    loss = ctypes.c_float()
    _check(ctx, _lib.fd_mlp_gradient(ctx.handle, _f32(params, "params"), _f32(X, "X"), _f32(T, "T"),
                                     X.shape[0], _f32(g, "grad"), ctypes.byref(loss)))
    return g, loss.value


def fd_mlp_train_step(ctx, params, m, v, X, T, step, lr):
    loss = ctypes.c_float()
    _check(ctx, _lib.fd_mlp_train_step(ctx.handle, _f32(params, "params"), _f32(m, "m"), _f32(v, "v"),
                                       _f32(X, "X"), _f32(T, "T"), X.shape[0], step, lr,
                                       ctypes.byref(loss)))
    return loss.value


def fd_filter_features(ctx, A, a, b, n_target, nb, ns, seed=0):
    f = np.zeros(64, dtype=np.float32)
    _check(ctx, _lib.fd_filter_features(ctx.handle, A.handle, a, b, n_target, nb, ns, seed,
                                        f.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return f


def fd_predict_filter_params(ctx, params, feat):
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    c, ml, mr, fb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), _i32()
    _check(ctx, _lib.fd_predict_filter_params(ctx.handle, _f32(params, "params"),
                                              feat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              ctypes.byref(c), ctypes.byref(ml), ctypes.byref(mr),
                                              ctypes.byref(fb)))
    return {"c_n": c.value, "m_l": ml.value, "m_r": mr.value, "fallback": fb.value}
