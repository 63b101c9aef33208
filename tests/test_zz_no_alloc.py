"""csl_precondition_static: the allocation-free P^{-1} v for callers that
cannot allocate device memory (a memory-pool-managed runtime that owns all
device memory, a fixed-budget embedded service, code running under stream
capture).  It keeps its scratch in static device arrays of the library; here
its output is checked, through the C ABI, against the plan-based
csl_precondition on two calls in a row (the second call reuses the static
scratch the first one left behind), with the tolerances of the other
preconditioner parity tests."""
import numpy as np
import pytest

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


def rel(a, b):
    a = a.detach().cpu().numpy()
    b = b.detach().cpu().numpy()
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("dim,n,coef,lam", [(2, 511, W.coef_c0, 1 + 10j), (3, 63, W.coef_c2, -5 + 50j),
                                            (2, 31, W.coef_c1, 100j)])
def test_static_precondition_matches_plan(csl, dim, n, coef, lam, precision, tol):
    import torch
    faces = W.sample_faces(dim, n, coef)
    with csl.Plan([dev(f) for f in faces], lam, precision=precision) as plan:
        for seed in (31, 32):  # two calls in a row
            v = dev(W.rhs_uniform((n,) * dim, seed))
            ref = plan.precondition(v)
            out = csl._binding.precondition_static(v, plan.gamma, lam, precision)
            torch.cuda.synchronize()
            assert rel(out, ref) < tol


def test_static_precondition_rejects_oversize_grid(csl):
    import torch
    n = 1023  # 1,046,529 points > the 262,144-point static capacity
    v = torch.zeros((n, n), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(csl.CSLError) as e:
        csl._binding.precondition_static(v, 1.0, 1 + 1j)
    assert e.value.status == csl.UNSUPPORTED_SIZE
    assert "static scratch capacity" in csl.lib.csl_last_error().decode()
