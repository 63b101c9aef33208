"""Float-pair stencil of the FP32-preconditioner forms: (K + alpha I) z of
Eq. 1 in difference form, alpha z_p + sum_e c_e (z_p - z_q), evaluated with
pairs of floats, with the beta block term of Eq. 2 and delta = <A z, z> in
pairs too.  Checked against the FP64 oracle (true residual of the returned
iterate by the oracle's operator, iteration count, error) and against the
plan's FP64-arithmetic stencil on the same input; the range gate that keeps
pairs normal falls back to the FP64 stencil."""
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


def smooth_rhs(shape, seed):
    """The lowest sine mode plus 1e-3 noise: the case where the direct form
    (K + alpha) z = d z_p - sum c z_q cancels most."""
    axes = [np.arange(1, m + 1) / (m + 1) for m in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    f = np.ones(shape)
    for g in grids:
        f = f * np.sin(np.pi * g)
    return f * (1 + 0.5j) + 1e-3 * W.rhs_uniform(shape, seed)


CASES = [(2, 31, W.coef_c0, 1 + 10j, "uniform"), (2, 255, W.coef_c1, 100j, "uniform"),
         (2, 127, W.coef_c1, -5 + 50j, "smooth"), (3, 31, W.coef_c2, -5 + 50j, "uniform"),
         (3, 63, W.coef_c2, 1 + 10j, "smooth"), (2, (63, 31), W.coef_c1, 100j, "smooth"),
         (3, (31, 15, 63), W.coef_c2, 1 + 10j, "uniform")]


@pytest.mark.parametrize("precision", ["fp32", "bf16x6"])
@pytest.mark.parametrize("dim,n,coef,lam,kind", CASES)
def test_float_pair_solve(csl, dim, n, coef, lam, kind, precision):
    faces = W.sample_faces(dim, n, coef)
    shape = W.grid_array_shape(dim, n)
    f = W.rhs_uniform(shape, 41) if kind == "uniform" else smooth_rhs(shape, 42)
    zr, oinfo = O.solve(faces, lam, f, 1e-8, 1000)
    dfaces = [dev(x) for x in faces]
    out = {}
    for ff in (True, False):
        with csl.Plan(dfaces, lam, precision=precision, float_pair_stencil=ff) as plan:
            assert ("stencil[float-pair" if ff else "stencil[fp64") in plan.config, plan.config
            z, info = plan.solve(dev(f), tol=1e-8, maxit=1000)
        zg = host(z)
        res = O.complex_residual(faces, lam, zg, f)
        err = np.linalg.norm(zg - zr) / np.linalg.norm(zr)
        print(f"{precision} ff={ff} dim {dim} n {n} {kind}: iters {info.iters} (oracle {oinfo.iters}) "
              f"relres {res:.2e} (device {info.relres:.2e}) err {err:.2e}")
        assert info.converged, info
        assert res <= 1e-8 and abs(res - info.relres) <= 1e-3 * res + 1e-15
        assert err <= 1e-7, err
        band = 2 + int(0.06 * oinfo.iters)
        assert abs(info.iters - oinfo.iters) <= band, (info.iters, oinfo.iters)
        out[ff] = (zg, info.iters)
    # the two stencils apply the same operator up to rounding
    assert abs(out[True][1] - out[False][1]) <= 2, (out[True][1], out[False][1])
    d = np.linalg.norm(out[True][0] - out[False][0]) / np.linalg.norm(zr)
    assert d <= 1e-7, d


def test_float_pair_repeatable(csl):
    """Deterministic reductions: two solves are bitwise equal."""
    faces = W.sample_faces(2, 127, W.coef_c1)
    f = W.rhs_uniform((127, 127), 43)
    with csl.Plan([dev(x) for x in faces], 100j, precision="fp32") as plan:
        z1, i1 = plan.solve(dev(f), tol=1e-8, maxit=500)
        z1 = host(z1)
        z2, i2 = plan.solve(dev(f), tol=1e-8, maxit=500)
    assert i1.iters == i2.iters and np.array_equal(z1, host(z2))


def test_float_pair_range_gate(csl):
    """Faces a/h^2 above 2^60 take the FP64 stencil; the solve still meets
    the tolerance (system and solution scaled by 2^64)."""
    scale = 2.0 ** 64
    faces = [x * scale for x in W.sample_faces(2, 31, W.coef_c0)]
    lam = (1 + 10j) * scale
    f = W.rhs_uniform((31, 31), 44)
    with csl.Plan([dev(x) for x in faces], lam, precision="fp32") as plan:
        assert "stencil[fp64" in plan.config, plan.config
        z, info = plan.solve(dev(f), tol=1e-8, maxit=500)
    assert info.converged
    assert O.complex_residual(faces, lam, host(z), f) <= 1e-8


def test_float_pair_batch_mixed_range(csl):
    """A batch group with one system outside the pair range runs the FP64
    stencil for the whole group; every system converges."""
    base = W.sample_faces(2, 63, W.coef_c0)
    scaled = [x * 2.0 ** 64 for x in base]
    rng = np.random.default_rng(45)
    systems = [(base, 1 + 10j), (scaled, (1 + 10j) * 2.0 ** 64), (base, 100j)]
    fs = [rng.uniform(-1, 1, (63, 63)) + 1j * rng.uniform(-1, 1, (63, 63)) for _ in systems]
    with csl.Batch([([dev(x) for x in fc], lam) for fc, lam in systems], precision="fp32") as B:
        zs, infos = B.solve([dev(f) for f in fs], tol=1e-8, maxit=500)
    for (fc, lam), f, z, info in zip(systems, fs, zs, infos):
        assert info.converged, info
        assert O.complex_residual(fc, lam, host(z), f) <= 1e-8


def test_fp32_scale_range(csl):
    """Per-mode scales of P^-1 below the FP32 range: the FP32 form refuses
    the plan (CSL_INVALID_ARG) instead of solving with zero scales, and the
    FP64 form solves the same system."""
    scale = 2.0 ** 200
    faces = [x * scale for x in W.sample_faces(2, 31, W.coef_c0)]
    lam = (1 + 10j) * scale
    f = W.rhs_uniform((31, 31), 46)
    dfaces = [dev(x) for x in faces]
    with pytest.raises(csl.CSLError) as e:
        csl.Plan(dfaces, lam, precision="fp32")
    assert e.value.status == csl.INVALID_ARG
    with csl.Plan(dfaces, lam, precision="fp64") as plan:
        z, info = plan.solve(dev(f), tol=1e-8, maxit=500)
    assert info.converged
    assert O.complex_residual(faces, lam, host(z), f) <= 1e-8
