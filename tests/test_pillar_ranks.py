"""The pillar layout (Sec. 3.4, 3.5) on CPU with two and three gloo ranks: each
rank filters only its own bundles, one all-gather per outer iteration, then
every rank repeats orthonormalisation and Rayleigh-Ritz on identical data.
Three outer iterations give exactly the single-process result (the filter is
column-wise, so no rounding differs), with the oracle standing in for the
filter and the dense steps."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SPEC = "hubbard:n_sites=6,n_up=3,n_dn=3,t=1,U=4,bc=open"
NB, NS, DEG, ITERS = 4, 24, 30, 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    sys.path.insert(0, ROOT)
    from oracle import chebyshev as ch
    from oracle import lanczos
    from oracle import matrices as mat
    csr = mat.build(SPEC)
    A = mat.to_scipy(csr)
    lo, hi = lanczos.gershgorin(csr)
    alpha, beta = ch.scale_params(lo - 0.01, hi + 0.01)
    mu = ch.filter_coeffs(alpha * 7.0 + beta, alpha * 9.0 + beta, DEG)
    V0 = np.random.default_rng(3).standard_normal((A.shape[0], NS))
    return A, V0, mu, alpha, beta


def _iterate(V, A, mu, alpha, beta, step):
    """ITERS outer iterations; step(V, filter_fn) is the filter stage."""
    import torch
    from oracle import chebyshev as ch
    from oracle import ortho, rayleigh_ritz

    def filt(cols):
        cols.copy_(torch.from_numpy(ch.cheb_filter(A, cols.numpy(), mu, alpha, beta)))

    thetas = []
    for _ in range(ITERS):
        step(V, filt)
        Q, _, _ = ortho.cholqr2(V.numpy())
        theta, Qr, _, _ = rayleigh_ritz.rayleigh_ritz(A, Q)
        V.copy_(torch.from_numpy(Qr))
        thetas.append(theta)
    return np.array(thetas)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2209_01974_gb300 import pillar
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A, V0, mu, alpha, beta = _problem()
    V = torch.from_numpy(V0.copy())
    ranges = []

    def step(V, filt):
        ranges.append(pillar.pillar_step(V, NB, filt, rank, world))

    th = _iterate(V, A, mu, alpha, beta, step)
    out[rank] = (th, V.numpy().copy(), ranges[0])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_pillar_ranks_equal_one_process(world):
    import torch
    sys.path.insert(0, ROOT)
    from paper_2209_01974_gb300 import pillar
    A, V0, mu, alpha, beta = _problem()
    ref_V = torch.from_numpy(V0.copy())
    ref = _iterate(ref_V, A, mu, alpha, beta, lambda V, f: pillar.filter_own(V, (0, NS), NB, f))
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        th, V, rng = out[r]
        assert np.array_equal(th, ref)
        assert np.array_equal(V, ref_V.numpy())
        assert [tuple(x) for x in rng] == pillar.bundle_ranges(NS, NB, world)


def test_bundle_ranges():
    sys.path.insert(0, ROOT)
    from paper_2209_01974_gb300 import pillar
    assert pillar.bundle_ranges(384, 64, 4) == [(0, 128), (128, 256), (256, 320), (320, 384)]
    assert pillar.bundle_ranges(64, 16, 8)[4:] == [(64, 64)] * 4
    r = pillar.bundle_ranges(448, 64, 3)
    assert r[0][0] == 0 and r[-1][1] == 448 and all(a[1] == b[0] for a, b in zip(r, r[1:]))
    with pytest.raises(ValueError):
        pillar.bundle_ranges(100, 64, 2)
