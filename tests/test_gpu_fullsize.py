"""Full-size workloads, in the launch configuration bench.py times (autotuned
plan, CUDA-graph loop): 2D n = 1023 (a = exp(ln10 xy), lambda = 100i) and 3D
n = 127 (a = 1 + 0.9 sin2pix sin2piy sin2piz, lambda = -5+50i).  The oracle
cannot solve these in test time, so the checks are what holds at any size:
the true relative residual of the returned z, evaluated by the oracle's own
FP64 operator, and the iteration count against the one the oracle reached on
the same input (tests/golden/oracle_iterations.txt, written by
make_oracle_iterations.py from oracle/ alone).  Sampled entries of (K + lam I) z
are recomputed one by one from the stencil definition (Eq. 1)."""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csl():
    import __graft_entry__ as g
    g.build()
    import paper_2408_00488_gb300 as csl
    return csl


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy()


def golden(name):
    p = os.path.join(os.path.dirname(__file__), "golden", "oracle_iterations.txt")
    for line in open(p):
        if line.startswith(name + " "):
            return int(line.split()[1])
    raise KeyError(name)


def point_apply(faces, lam, z, idx):
    """(K + lam I) z at one grid point idx (C order, x last), from the face
    coefficients directly: sum over faces of a_e (z_p - z_q) / h^2."""
    dim = z.ndim
    n = z.shape[0]
    h2 = 1.0 / (n + 1) ** 2
    acc = lam * z[idx]
    mag = abs(acc)  # sum of term magnitudes: the scale of the rounding error
    for ax in range(dim):
        fa = faces[ax]            # axis ax (0 = x = last array axis) faces
        arr_ax = dim - 1 - ax     # array axis of grid axis ax
        for side in (0, 1):
            fidx = list(idx)
            fidx[arr_ax] = idx[arr_ax] + side
            a = fa[tuple(fidx)]
            q = list(idx)
            q[arr_ax] = idx[arr_ax] + (1 if side else -1)
            zq = z[tuple(q)] if 0 <= q[arr_ax] < n else 0.0
            acc += a * (z[idx] - zq) / h2
            mag += a * (abs(z[idx]) + abs(zq)) / h2
    return acc, mag


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["config1", "config2"])
def test_full_size_solve(csl, name, precision):
    s = getattr(W, name)()
    with csl.Plan([dev(x) for x in s.faces], s.lam, precision=precision) as plan:
        z, info = plan.solve(dev(s.f), tol=1e-8, maxit=2000)
    zg = host(z)
    res = O.complex_residual(s.faces, s.lam, zg, s.f)
    it = golden(name)
    print(f"{name} {precision}: iters {info.iters} (oracle {it}) relres {res:.3e} (device {info.relres:.3e})")
    assert info.converged and res <= 1e-8
    assert abs(res - info.relres) <= 1e-3 * res
    band = 2 if precision == "fp64" else 2 + int(0.06 * it)
    assert abs(info.iters - it) <= band, (info.iters, it)
    # sampled outputs of the operator, one by one, against the device's apply
    rng = np.random.default_rng(34)
    with csl.Plan([dev(x) for x in s.faces], s.lam) as plan:
        Az = host(plan.apply(dev(zg)))
    for _ in range(64):
        idx = tuple(int(rng.integers(0, s.n)) for _ in range(zg.ndim))
        ref, mag = point_apply(s.faces, s.lam, zg, idx)
        assert abs(Az[idx] - ref) <= 1e-14 * mag, (idx, Az[idx], ref, mag)
