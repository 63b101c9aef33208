"""Rectangular grids (n_x != n_y [!= n_z], spacing 1/(n_a + 1) per axis; the
sine transform is per axis, so only the per-axis tables differ): operator,
P^{-1} and solves against the FP64 oracle in every precision, with the
tensor-core transform on the axes whose lines have 32, 64 or 128 points."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL_P = {"fp64": 1e-12, "fp32": 2e-5, "bf16x3": 3e-5, "bf16x6": 1e-5}
RECTS = [((63, 31), W.coef_c1), ((31, 127), W.coef_c0), ((255, 15), W.coef_c1),
         ((31, 15, 63), W.coef_c2), ((15, 63, 31), W.coef_c2), ((63, 7, 31), W.coef_c2)]


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


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("ns,coef", RECTS)
def test_rect_apply(csl, ns, coef):
    dim = len(ns)
    faces = W.sample_faces(dim, ns, coef)
    z = W.rhs_normal(W.grid_array_shape(dim, ns), 36)
    lam = -5 + 50j
    ref = O.apply_K(faces, z) + lam * z
    with csl.Plan([dev(f) for f in faces], lam) as plan:
        assert plan.shape == W.grid_array_shape(dim, ns)
        out = host(plan.apply(dev(z)))
    assert rel(out, ref) < 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("ns,coef", RECTS)
def test_rect_precondition(csl, ns, coef, precision):
    dim = len(ns)
    faces = W.sample_faces(dim, ns, coef)
    lam = 1 + 10j
    v = W.rhs_uniform(W.grid_array_shape(dim, ns), 37)
    gamma = O.gamma_from_faces(faces)
    r1, r2 = O.precond_apply(v.real, v.imag, gamma, lam.real, lam.imag)
    with csl.Plan([dev(f) for f in faces], lam, precision=precision) as plan:
        out = host(plan.precondition(dev(v)))
        tc_axes = [a for a in range(1, dim) if ns[a] + 1 in (32, 64, 128)]
        if precision.startswith("bf16") and tc_axes:
            assert "tcgen05" in plan.config, plan.config
    assert rel(out, r1 + 1j * r2) < TOL_P[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x6"])
@pytest.mark.parametrize("ns,coef,lam", [((63, 31), W.coef_c1, 100j), ((15, 63, 31), W.coef_c2, -5 + 50j),
                                         ((31, 7), W.coef_c0, 1 + 10j)])
def test_rect_solve(csl, ns, coef, lam, precision):
    dim = len(ns)
    faces = W.sample_faces(dim, ns, coef)
    f = W.rhs_uniform(W.grid_array_shape(dim, ns), 38)
    zr, oinfo = O.solve(faces, lam, f, 1e-8, 800)
    with csl.Plan([dev(x) for x in faces], lam, precision=precision) as plan:
        z, info = plan.solve(dev(f), tol=1e-8, maxit=800)
    zg = host(z)
    res = O.complex_residual(faces, lam, zg, f)
    err = np.linalg.norm(zg - zr) / np.linalg.norm(zr)
    assert info.converged and res <= 1e-8 and err <= 1e-7, (info, res, err)
    band = 2 if precision == "fp64" else 2 + int(0.06 * oinfo.iters)
    assert abs(info.iters - oinfo.iters) <= band, (info.iters, oinfo.iters)


def test_rect_coef_grad(csl):
    ns = (31, 15)
    faces = W.sample_faces(2, ns, W.coef_c0)
    lam = 1 + 20j
    shape = W.grid_array_shape(2, ns)
    f = W.rhs_uniform(shape, 39)
    d = np.random.default_rng(40).standard_normal(shape)
    zr, _ = O.solve(faces, lam, f, 1e-12, 800)
    Yr, _ = O.adjoint_solve(faces, lam, O.loss_c4_grad(zr, d), 1e-12, 800)
    gr = O.coef_grad(faces, zr, Yr)
    with csl.Plan([dev(x) for x in faces], lam) as plan:
        z, _ = plan.solve(dev(f), tol=1e-12, maxit=800)
        y, _ = plan.adjoint(dev(O.loss_c4_grad(host(z), d)), tol=1e-12, maxit=800)
        g = [host(t) for t in plan.coef_grad(z, y)]
    for a, b in zip(g, gr):
        assert a.shape == b.shape
        assert np.abs(a - b).max() / np.abs(b).max() < 1e-8
