"""The synchronisation-cost measurement hook (csl_probe_sync_cost): a kernel
boundary in a CUDA graph against a grid barrier in one cooperative kernel,
and its bounded wait.  With every barrier target out of reach, each CTA's
wait runs out after its budget (about 1 ms), the CTA returns (it has nothing
in flight), the call reports CSL_TIMEOUT, and the context stays usable: a
solve right after it matches the oracle."""
import math

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


def test_sync_cost_measured(csl):
    r = csl.probe_sync_cost(kernels=100, barriers=200)
    for k in ("graph_pdl_us", "graph_us", "grid_barrier_us"):
        assert math.isfinite(r[k]) and 0.0 < r[k] < 1000.0, r


def test_sync_wait_runs_out_and_context_survives(csl):
    import torch
    with pytest.raises(csl.CSLError) as e:
        csl.probe_sync_cost(kernels=1, barriers=10, unreachable=True)
    assert e.value.status == csl.TIMEOUT
    assert "ran out" in csl.lib.csl_last_error().decode()
    s = W.config0()
    faces = [torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0") for x in s.faces]
    with csl.Plan(faces, s.lam, precision="fp64") as plan:
        z, info = plan.solve(torch.from_numpy(s.f).to("cuda:0"), tol=1e-8, maxit=200)
        zg = z.cpu().numpy()
    zr, oinfo = O.solve(s.faces, s.lam, s.f, 1e-8, 200)
    assert info.converged and abs(info.iters - oinfo.iters) <= 2
    assert np.linalg.norm(zg - zr) / np.linalg.norm(zr) <= 1e-7


def test_sync_probe_rejects_bad_args(csl):
    out = (__import__("ctypes").c_double * 3)()
    assert csl.lib.csl_probe_sync_cost(0, 10, 0, out) == csl.INVALID_ARG
    assert csl.lib.csl_probe_sync_cost(10, 0, 0, out) == csl.INVALID_ARG
    assert csl.lib.csl_probe_sync_cost(10, 10, 0, None) == csl.INVALID_ARG
