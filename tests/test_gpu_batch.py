"""Batched solves (csl_batch_*): many shifts lambda_k from an alpha-circulant
time discretisation and grids of different sizes in one graph launch.  Each
system must match the single-system solve (same kernels and launch shapes)
and the FP64 CPU oracle."""
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


def _systems(ns, nshift, seed):
    lams = W.alpha_circulant_shifts(64, 1e-4)
    pick = [0, 32] + list(range(1, 64, max(1, 64 // max(1, nshift - 2))))[: max(0, nshift - 2)]
    rng = np.random.default_rng(seed)
    out = []
    for n in ns:
        faces = W.sample_faces(2, n, W.coef_c0)
        for k in pick[:nshift]:
            f = rng.uniform(-1, 1, (n, n)) + 1j * rng.uniform(-1, 1, (n, n))
            out.append((faces, complex(lams[k]), f))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_solves_and_oracle(csl, precision):
    systems = _systems([15, 31, 63], 5, 41)
    dfaces = {}
    for faces, lam, f in systems:
        dfaces.setdefault(id(faces), [dev(x) for x in faces])
    with csl.Batch([(dfaces[id(fc)], lam) for fc, lam, _ in systems], precision=precision) as B:
        zs, infos = B.solve([dev(f) for _, _, f in systems], tol=1e-8, maxit=400)
    for (faces, lam, f), z, info in zip(systems, zs, infos):
        assert info.converged and info.relres <= 1e-8, info
        with csl.Plan(dfaces[id(faces)], lam, precision=precision) as p:
            zz, i1 = p.solve(dev(f), tol=1e-8, maxit=400)
        assert i1.iters == info.iters
        a, b = host(z), host(zz)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12
        zr, oi = O.solve(faces, lam, f, 1e-8, 400)
        assert np.linalg.norm(a - zr) / np.linalg.norm(zr) < 1e-7
        assert O.complex_residual(faces, lam, a, f) <= 1e-8


def test_batch_config3_subset_converges(csl):
    # the config-3 mix (n = 127, 255, 511; alpha-circulant shifts incl. the real
    # ones k = 0 and 32) on a subset of shifts, FP32 preconditioner
    systems = _systems([127, 255, 511], 4, 43)
    dfaces = {}
    for faces, lam, f in systems:
        dfaces.setdefault(id(faces), [dev(x) for x in faces])
    with csl.Batch([(dfaces[id(fc)], lam) for fc, lam, _ in systems], precision="fp32") as B:
        zs, infos = B.solve([dev(f) for _, _, f in systems], tol=1e-8, maxit=400)
        # a second solve reuses the graph
        zs2, infos2 = B.solve([dev(f) for _, _, f in systems], tol=1e-8, maxit=400)
    for (faces, lam, f), z, z2, info, info2 in zip(systems, zs, zs2, infos, infos2):
        assert info.converged and info2.iters == info.iters
        zg = host(z)
        assert np.array_equal(zg, host(z2))
        assert O.complex_residual(faces, lam, zg, f) <= 1e-8
