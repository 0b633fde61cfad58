"""Batched FD (many uneven instances, one persistent filter launch per outer
iteration, CUDA graph) against dense eigensolvers and against one-by-one solves."""
import numpy as np
import pytest

from oracle import matrices as mat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


@pytest.fixture(scope="module")
def ctx(fd):
    return fd.fd_create(0)


def _nearest(ev, tau, k):
    return np.sort(ev[np.lexsort((ev, np.abs(ev - tau)))[:k]])


SMALL = ["anderson3d:L=6,W=4,seed=1", "anderson3d:L=7,W=8,seed=2", "anderson3d:L=9,W=12,seed=3",
         "chain:n=500", "hubbard:n_sites=6,n_up=3,n_dn=3,t=1,U=4,bc=open",
         "anderson3d:L=8,W=16,seed=4"]


@pytest.mark.parametrize("nb", [8, 16])
def test_small_batch_matches_dense(fd, ctx, nb):
    mats = [fd.fd_build_matrix(ctx, s) for s in SMALL]
    probs = [(-0.3, 0.3, 8, 0)] * 5 + [(7.5, 8.5, 8, 0)]
    probs[4], probs[5] = (7.5, 8.5, 8, 0), (-0.3, 0.3, 8, 0)
    out, res = fd.fd_solve_batched(ctx, mats, probs, nb, 40, 1e-9)
    for spec, (a, b, nt, _), (th, rho), r in zip(SMALL, probs, out, res):
        ev = np.linalg.eigvalsh(mat.to_scipy(mat.build(spec)).toarray())
        assert r["converged"] == 1, spec
        assert rho.max() <= 1e-9, spec
        assert np.abs(th - _nearest(ev, 0.5 * (a + b), nt)).max() <= 1e-10 * np.abs(ev).max(), spec


def test_uneven_anderson_batch_matches_sequential(fd, ctx):
    seeds = [0, 14, 22, 26, 53, 12, 45, 50]        # L = 16 .. 21, W = 9.4 .. 15.6
    specs = []
    for s in seeds:
        L, W = mat.anderson_instance(s)
        specs.append(f"anderson3d:L={L},W={float(W)!r},seed={s}")
    mats = [fd.fd_build_matrix(ctx, s) for s in specs]
    probs = [(-0.01, 0.01, 16, s) for s in seeds]
    out, res = fd.fd_solve_batched(ctx, mats, probs, 16, 200, 1e-9)
    for m, (a, b, nt, sd), (th, rho), r in zip(mats, probs, out, res):
        assert r["converged"] == 1 and rho.max() <= 1e-9
        th1, rho1, r1 = fd.fd_solve(ctx, m, a, b, nt, 16, 200, 1e-9, seed=sd)
        # same start block, bounds and heuristic: the same eigenvalues
        assert np.abs(th - th1).max() <= 1e-10 * max(abs(r1["lam_l"]), abs(r1["lam_r"]))
    # the context has no stream of its own, so the solve ran on a private stream
    # and every outer iteration was replayed from the captured CUDA graph
    assert all(r["used_graph"] == 1 for r in res)


def test_instance_disorder_parses_exactly(fd, ctx):
    L, W = mat.anderson_instance(7)
    spec = f"anderson3d:L={L},W={float(W)!r},seed=7"
    A = fd.fd_build_matrix(ctx, spec)
    rp, c, v = fd.fd_matrix_to_csr(ctx, A)
    o = mat.anderson3d(L, W, 7)
    assert np.array_equal(v.view(np.uint64), o[2].view(np.uint64))


def test_tuner_returns_a_candidate(fd, ctx):
    specs = ["anderson3d:L=16,W=10,seed=0", "anderson3d:L=20,W=12,seed=1", "anderson3d:L=24,W=8,seed=2"]
    t = fd.fd_tune_batched(ctx, specs, 16, 20)
    assert t["nb"] in (8, 16, 32, 64) and t["C"] in (32, 64, 128) and t["cta_warps"] in (4, 8)
    assert t["gbs"] > 0


def test_batched_rejects_sigma_sorted_matrices(fd, ctx):
    A = fd.fd_build_matrix(ctx, "chain:n=100", sigma=32)
    with pytest.raises(fd.FDError) as e:
        fd.fd_solve_batched(ctx, [A], [(-0.1, 0.1, 4, 0)], 8, 20, 1e-9)
    assert e.value.status == fd.FD_ERR_ARG


@pytest.mark.parametrize("nb", [8, 16])
def test_small_batch_fp32_form_matches_dense(fd, ctx, nb):
    # FP32 sweeps with the FP64 finish in the persistent batched filter
    mats = [fd.fd_build_matrix(ctx, s) for s in SMALL]
    probs = [(-0.3, 0.3, 8, 0)] * 5 + [(7.5, 8.5, 8, 0)]
    probs[4], probs[5] = (7.5, 8.5, 8, 0), (-0.3, 0.3, 8, 0)
    out, res = fd.fd_solve_batched(ctx, mats, probs, nb, 40, 1e-9, precision="f32")
    for spec, (a, b, nt, _), (th, rho), r in zip(SMALL, probs, out, res):
        ev = np.linalg.eigvalsh(mat.to_scipy(mat.build(spec)).toarray())
        assert r["converged"] == 1, spec
        assert rho.max() <= 1e-9, spec
        assert np.abs(th - _nearest(ev, 0.5 * (a + b), nt)).max() <= 1e-10 * np.abs(ev).max(), spec
    assert any(r["n_spmmv_f32"] > 0 for r in res)


def test_uneven_anderson_batch_fp32_form_matches_sequential(fd, ctx):
    # the FP32 form batched and one by one: the same switch rule and the same
    # fused FP32 step, so the same eigenvalues
    seeds = [0, 14, 22, 26, 53, 12]
    specs = []
    for s_ in seeds:
        L, W = mat.anderson_instance(s_)
        specs.append(f"anderson3d:L={L},W={float(W)!r},seed={s_}")
    mats = [fd.fd_build_matrix(ctx, s_) for s_ in specs]
    probs = [(-0.01, 0.01, 16, s_) for s_ in seeds]
    out, res = fd.fd_solve_batched(ctx, mats, probs, 16, 200, 1e-9, precision="f32")
    for m, (a, b, nt, sd), (th, rho), r in zip(mats, probs, out, res):
        assert r["converged"] == 1 and rho.max() <= 1e-9
        assert 0 < r["n_spmmv_f32"] < r["n_spmmv"]
        th1, rho1, r1 = fd.fd_solve(ctx, m, a, b, nt, 16, 200, 1e-9, seed=sd, precision="f32")
        assert np.abs(th - th1).max() <= 1e-10 * max(abs(r1["lam_l"]), abs(r1["lam_r"]))


def test_batched_fp32_form_needs_nb_4(fd, ctx):
    A = fd.fd_build_matrix(ctx, "chain:n=100")
    with pytest.raises(fd.FDError) as e:
        fd.fd_solve_batched(ctx, [A], [(-0.1, 0.1, 1, 0)], 2, 20, 1e-9, precision="f32")
    assert e.value.status == fd.FD_ERR_ARG


@pytest.mark.parametrize("form", [{"precision": "ff"}, {"precision": "f32", "finish": "ff"}])
def test_small_batch_ff_forms_match_dense(fd, ctx, form):
    # float-float rows in the persistent batched filter (all sweeps, or the
    # FP32 form's finish), the Rayleigh-Ritz SpMMV in the FP64 instantiation
    mats = [fd.fd_build_matrix(ctx, s) for s in SMALL]
    probs = [(-0.3, 0.3, 8, 0)] * 5 + [(7.5, 8.5, 8, 0)]
    probs[4], probs[5] = (7.5, 8.5, 8, 0), (-0.3, 0.3, 8, 0)
    out, res = fd.fd_solve_batched(ctx, mats, probs, 8, 40, 1e-9, **form)
    for spec, (a, b, nt, _), (th, rho), r in zip(SMALL, probs, out, res):
        ev = np.linalg.eigvalsh(mat.to_scipy(mat.build(spec)).toarray())
        assert r["converged"] == 1, spec
        assert rho.max() <= 1e-9, spec
        assert np.abs(th - _nearest(ev, 0.5 * (a + b), nt)).max() <= 1e-10 * np.abs(ev).max(), spec
    assert any(r["n_spmmv_ff"] > 0 for r in res)
    if form["precision"] == "ff":
        assert all(r["n_spmmv_f32"] == 0 for r in res)


def test_uneven_anderson_batch_ff_finish_matches_sequential(fd, ctx):
    # FP32 sweeps with the float-float finish, batched and one by one: the same
    # switch rule and the same arithmetic per row, so the same eigenvalues
    seeds = [0, 14, 22, 53]
    specs = []
    for s_ in seeds:
        L, W = mat.anderson_instance(s_)
        specs.append(f"anderson3d:L={L},W={float(W)!r},seed={s_}")
    mats = [fd.fd_build_matrix(ctx, s_) for s_ in specs]
    probs = [(-0.01, 0.01, 16, s_) for s_ in seeds]
    out, res = fd.fd_solve_batched(ctx, mats, probs, 16, 200, 1e-9, precision="f32", finish="ff")
    for m, (a, b, nt, sd), (th, rho), r in zip(mats, probs, out, res):
        assert r["converged"] == 1 and rho.max() <= 1e-9
        assert r["n_spmmv_ff"] > 0
        th1, rho1, r1 = fd.fd_solve(ctx, m, a, b, nt, 16, 200, 1e-9, seed=sd, precision="f32", finish="ff")
        assert np.abs(th - th1).max() <= 1e-10 * max(abs(r1["lam_l"]), abs(r1["lam_r"]))
