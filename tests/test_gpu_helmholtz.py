"""Shifted-Laplace preconditioned Helmholtz solve (csl_helmholtz_*: flexible
GMRES around the library's MINRES solve of the complex-shifted system) against
dense LU, the oracle's own flexible GMRES, and, at a larger grid, the true
residual by the oracle's operator."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,k2,coef", [(15, 64.0, W.coef_c0), (31, 256.0, W.coef_c1), (31, 400.0, W.coef_c0)])
def test_helmholtz_matches_dense_lu_and_oracle(csl, n, k2, coef, precision):
    faces = W.sample_faces(2, n, coef)
    f = W.rhs_uniform((n, n), 70)
    K = O.assemble_K_dense(faces)
    ref = np.linalg.solve(K - k2 * np.eye(n * n), f.ravel()).reshape(n, n)
    shift = -k2 * (1 - 0.5j)
    _, oinfo = O.helmholtz_fgmres(faces, -k2, shift, f, tol=1e-10, maxit=300, restart=60, inner_tol=1e-8)
    with csl.Helmholtz([dev(x) for x in faces], -k2, shift, restart=60, precision=precision) as hz:
        u, info = hz.solve(dev(f), tol=1e-10, maxit=300, inner_tol=1e-8)
    ug = host(u)
    assert info.status == 0 and info.relres <= 1e-10, (info.status, info.relres, info.iters)
    assert np.linalg.norm(ug - ref) / np.linalg.norm(ref) < 1e-7
    assert abs(info.iters - oinfo["iters"]) <= 2 + oinfo["iters"] // 10, (info.iters, oinfo["iters"])


def test_helmholtz_larger_grid_true_residual(csl):
    """n = 127, k^2 = 1024 (k h = 0.25), a as config 0, restarted every 150
    steps (outer GMRES steps grow about linearly with k for this
    preconditioner, so short restart windows stagnate at high k)."""
    n, k2 = 127, 1024.0
    faces = W.sample_faces(2, n, W.coef_c0)
    f = W.rhs_uniform((n, n), 71)
    with csl.Helmholtz([dev(x) for x in faces], -k2, -k2 * (1 - 0.5j), restart=150, precision="fp32") as hz:
        u, info = hz.solve(dev(f), tol=1e-8, maxit=600, inner_tol=1e-4)
    ug = host(u)
    print(f"Helmholtz n=127 k^2=1024: {info.iters} outer steps, {info.restarts} restarts, "
          f"{info.inner_iters_total} inner MINRES iterations, relres {info.relres:.2e}")
    assert info.status == 0
    r = f - (O.apply_K(faces, ug) - k2 * ug)
    assert np.linalg.norm(r) / np.linalg.norm(f) <= 1.01e-8
