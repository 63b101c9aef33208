"""Auxiliaries of the solver through the C ABI: the warm start (an initial
guess x_0; MINRES on the correction, stopping test still relative to
||f||), the per-iteration residual history, the scheduling options of the
iteration graph (where the w/x update runs, iterations per WHILE body),
and the autotuner's cache file.  Checked against the oracle's solve and the
plain (cold, default) solve of the same plan."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_precond"])
def test_warm_start(csl, precision):
    s = W.config0()
    zr, oinfo = O.solve(s.faces, s.lam, s.f, 1e-12, 500)
    faces = [dev(x) for x in s.faces]
    fd = dev(s.f)
    with csl.Plan(faces, s.lam, precision=precision) as cold, \
            csl.Plan(faces, s.lam, precision=precision, warm_start=True) as warm:
        z0, i0 = cold.solve(fd, tol=1e-8, maxit=300)
        # x0 = 0 is the cold solve, bit for bit
        z1, i1 = warm.solve(fd, tol=1e-8, maxit=300)
        assert i1.iters == i0.iters and np.array_equal(host(z0), host(z1))
        # a good guess (the exact solution, perturbed at 1e-4) needs fewer iterations
        rng = np.random.default_rng(7)
        x0 = zr * (1 + 1e-4 * rng.standard_normal(zr.shape))
        z2, i2 = warm.solve(fd, tol=1e-8, maxit=300, x0=dev(x0))
        assert i2.converged and i2.iters < i0.iters, (i2.iters, i0.iters)
        zg = host(z2)
        assert O.complex_residual(s.faces, s.lam, zg, s.f) <= 1e-8
        assert np.linalg.norm(zg - zr) / np.linalg.norm(zr) <= 1e-7
        # a guess that already meets the tolerance is returned as it is
        z3, i3 = warm.solve(fd, tol=1e-8, maxit=300, x0=dev(zr))
        assert i3.converged and i3.iters == 0 and np.array_equal(host(z3), zr)
        # host buffers: z_host holds x0 on entry
        import torch
        fh = torch.from_numpy(s.f.copy()).pin_memory()
        zh = torch.from_numpy(x0.copy()).pin_memory()
        i4 = warm.solve_host(fh, zh, tol=1e-8, maxit=300)
        assert i4.iters == i2.iters and np.array_equal(zh.numpy(), zg)


def test_warm_start_adjoint(csl):
    n = 15
    faces = W.sample_faces(2, n, W.coef_c0)
    lam = 1 + 20j
    g = W.rhs_uniform((n, n), 27)
    Yr, _ = O.adjoint_solve(faces, lam, g, 1e-12, 500)
    with csl.Plan([dev(x) for x in faces], lam, warm_start=True) as plan:
        y0 = dev(Yr * (1 + 1e-3))
        y, info = plan.adjoint(dev(g), tol=1e-10, maxit=500, out=y0)
        assert info.converged
        assert np.linalg.norm(host(y) - Yr) / np.linalg.norm(Yr) < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_residual_history(csl, precision):
    s = W.config0()
    with csl.Plan([dev(x) for x in s.faces], s.lam, precision=precision, history=1000) as plan:
        z, info = plan.solve(dev(s.f), tol=1e-8, maxit=300)
        h = plan.history()
    assert len(h) == info.iters > 0
    assert all(b <= a * (1 + 1e-12) for a, b in zip(h, h[1:])), "MINRES residual estimate must not increase"
    assert 0 < h[-1] < h[0] <= 1.0
    with csl.Plan([dev(x) for x in s.faces], s.lam) as plan:
        with pytest.raises(csl.CSLError):
            plan.history()


def test_schedule_options_give_identical_solves(csl):
    s = W.config0()
    faces = [dev(x) for x in s.faces]
    fd = dev(s.f)
    out = {}
    for prec in ("fp64", "fp32"):
        for kw in ({}, {"update_mode": 2}, {"update_mode": 3}, {"body_iters": 4}, {"body_iters": 8},
                   {"use_graph": False}):
            with csl.Plan(faces, s.lam, precision=prec, **kw) as plan:
                z, info = plan.solve(fd, tol=1e-8, maxit=300)
                out[(prec, tuple(kw.items()))] = (host(z), info.iters)
        ref = out[(prec, ())]
        for k, (z, it) in out.items():
            if k[0] == prec:
                assert it == ref[1] and np.array_equal(z, ref[0]), k


def test_bad_options_rejected(csl):
    s = W.config0()
    faces = [dev(x) for x in s.faces]
    for kw in ({"update_mode": 5}, {"body_iters": 3}, {"history": -1}):
        with pytest.raises(csl.CSLError) as e:
            csl.Plan(faces, s.lam, **kw)
        assert e.value.status == csl.INVALID_ARG


def test_tune_cache_round_trip(csl, tmp_path):
    n = 255
    faces = [dev(x) for x in W.sample_faces(2, n, W.coef_c0)]
    with csl.Plan(faces, 1 + 10j, precision="fp32") as p1:
        cfg = p1.config
    path = str(tmp_path / "tune.txt")
    csl.tune_cache_save(path)
    text = open(path).read().splitlines()
    assert text[0] == "csl-tune-cache 1" and len(text) >= 2
    csl.tune_cache_load(path)
    with csl.Plan(faces, 1 + 10j, precision="fp32") as p2:
        assert p2.config == cfg
    bad = str(tmp_path / "bad.txt")
    with open(bad, "w") as fh:
        fh.write("csl-tune-cache 1\n4 2 1000 255 1 0 4\n")  # N = 1000 is not a power of two
    with pytest.raises(csl.CSLError):
        csl.tune_cache_load(bad)
    with pytest.raises(csl.CSLError):
        csl.tune_cache_load(str(tmp_path / "missing.txt"))
