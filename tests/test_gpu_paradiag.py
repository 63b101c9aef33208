"""All-at-once backward-Euler solve (csl_paradiag_*): the alpha-circulant
preconditioned Richardson built on the batched shifted solves, against the
oracle's step-by-step time integration (dense LU on small grids, the oracle's
MINRES on larger ones) and its own Richardson sweep count."""
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


def dense_time_stepping(faces, tau, u0, g):
    K = O.assemble_K_dense(faces)
    m = K.shape[0]
    Mstep = K + np.eye(m) / tau
    out = np.empty((g.shape[0], m), dtype=np.complex128)
    prev = u0.ravel()
    for t in range(g.shape[0]):
        out[t] = np.linalg.solve(Mstep, g[t].ravel() + prev / tau)
        prev = out[t]
    return out.reshape(g.shape)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,L,a", [(2, 15, 8, 1e-3), (2, 31, 16, 1e-4), (3, 7, 4, 1e-2)])
def test_paradiag_matches_backward_euler(csl, dim, n, L, a, precision):
    tau = 1.0 / L
    faces = W.sample_faces(dim, n, W.coef_c0 if dim == 2 else W.coef_c2)
    shape = W.grid_array_shape(dim, n)
    u0 = W.rhs_uniform(shape, 60)
    g = W.rhs_normal((L,) + shape, 61)
    ref = dense_time_stepping(faces, tau, u0, g)
    _, hist = O.paradiag_solve(faces, tau, a, u0, g, tol=1e-10, maxit=20)
    with csl.ParaDiag([dev(f) for f in faces], L, tau, a, precision=precision) as pd:
        u, info = pd.solve(dev(u0), dev(g), tol=1e-10, maxit=20, inner_tol=1e-10)
    ug = host(u)
    assert info.status == 0 and info.relres <= 1e-10, (info.status, info.relres)
    assert np.linalg.norm(ug - ref) / np.linalg.norm(ref) < 1e-9
    # Richardson residual computed independently by the oracle's operator
    R = O.paradiag_rhs(tau, u0, g) - O.paradiag_apply(faces, tau, ug)
    assert np.linalg.norm(R) / np.linalg.norm(O.paradiag_rhs(tau, u0, g)) <= 1.01e-10
    assert abs(info.sweeps - (len(hist) - 1)) <= 1, (info.sweeps, len(hist) - 1)


def test_paradiag_config3_grid(csl):
    """The config-3 setting: n = 127, L = 64 steps on [0, 1], a = 1e-4 (the
    shifted systems are config 3's n = 127 group); against the oracle's
    step-by-step integration with MINRES at tol 1e-13."""
    n, L, a = 127, 64, 1e-4
    tau = 1.0 / L
    faces = W.sample_faces(2, n, W.coef_c0)
    u0 = W.rhs_uniform((n, n), 62)
    g = W.rhs_normal((L, n, n), 63) * 0.1
    ref = O.paradiag_time_stepping(faces, tau, u0, g, tol=1e-13)
    with csl.ParaDiag([dev(f) for f in faces], L, tau, a, precision="fp32") as pd:
        u, info = pd.solve(dev(u0), dev(g), tol=1e-10, maxit=10, inner_tol=1e-10)
    ug = host(u)
    print(f"ParaDiag n=127 L=64: sweeps {info.sweeps} relres {info.relres:.2e} inner max {info.inner_iters_max}")
    assert info.status == 0 and info.sweeps <= 4
    assert np.linalg.norm(ug - ref) / np.linalg.norm(ref) < 1e-9


def test_paradiag_rejects_bad_arguments(csl):
    faces = [dev(f) for f in W.sample_faces(2, 15, W.coef_c0)]
    for L, tau, a in [(6, 0.1, 1e-3), (8, -1.0, 1e-3), (8, 0.1, 1.5), (8, 0.1, 0.0)]:
        with pytest.raises(csl.CSLError):
            csl.ParaDiag(faces, L, tau, a)
