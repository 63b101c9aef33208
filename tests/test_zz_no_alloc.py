"""csl_precondition_static: the allocation-free P^{-1} v, for callers that
cannot allocate device memory (a runtime whose memory pool owns all device
memory, a fixed-budget embedded service).  It keeps its scratch in static
device arrays of the library.  Its output is checked, through the C ABI,
against the plan-based csl_precondition on two calls in a row (the second
call reuses the static scratch the first one left behind) and against the
oracle's P^{-1} (Eq. 4 via Section 2.3), with the tolerances of the other
preconditioner parity tests; its argument checks mirror the plan's."""
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


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else a
    b = b.detach().cpu().numpy() if hasattr(b, "detach") else b
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = [(2, 511, W.coef_c0, 1 + 10j), (3, 63, W.coef_c2, -5 + 50j), (2, 31, W.coef_c1, 100j)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("dim,n,coef,lam", CASES)
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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("dim,n,coef,lam", CASES)
def test_static_precondition_matches_oracle(csl, dim, n, coef, lam, precision, tol):
    import torch
    faces = W.sample_faces(dim, n, coef)
    gamma = O.gamma_from_faces(faces)
    v = W.rhs_normal((n,) * dim, 33)
    r1, r2 = O.precond_apply(v.real, v.imag, gamma, lam.real, lam.imag)
    out = csl._binding.precondition_static(dev(v), gamma, lam, precision)
    torch.cuda.synchronize()
    assert rel(out, r1 + 1j * r2) < tol


def test_static_precondition_block_pair_form(csl):
    # float64 block pairs (grid + (2,)) give the same numbers as complex128
    import torch
    n = 31
    v = W.rhs_uniform((n, n), 34)
    pairs = np.stack([v.real, v.imag], axis=-1)
    a = csl._binding.precondition_static(dev(v), 1.3, 2 + 5j)
    b = csl._binding.precondition_static(dev(pairs), 1.3, 2 + 5j)
    torch.cuda.synchronize()
    assert np.array_equal(torch.view_as_real(a).cpu().numpy(), b.cpu().numpy())


def test_static_precondition_rejects_bad_tensors(csl):
    import torch
    n = 31
    flat = torch.zeros((n, n), dtype=torch.float64, device="cuda:0")  # no trailing pair dimension
    with pytest.raises(ValueError):
        csl._binding.precondition_static(flat, 1.0, 1 + 1j)
    v = torch.zeros((n, n), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(ValueError):
        csl._binding.precondition_static(v, 1.0, 1 + 1j, out=torch.empty((n, n - 1), dtype=torch.complex128,
                                                                           device="cuda:0"))
    with pytest.raises(ValueError):
        csl._binding.precondition_static(v, 1.0, 1 + 1j, out=torch.empty((n, n, 2), dtype=torch.float64,
                                                                           device="cuda:0"))


def test_static_precondition_singular_rejected(csl):
    # beta = 0, alpha = -gamma (mu_1 + mu_1): the mode (1, 1) of P is zero
    import torch
    n = 7
    mu = O.laplacian_eigs_1d(n, 1.0 / (n + 1))
    v = torch.ones((n, n), dtype=torch.complex128, device="cuda:0")
    for precision in ("fp64", "fp32"):
        with pytest.raises(csl.CSLError) as e:
            csl._binding.precondition_static(v, 1.0, complex(-(mu[0] + mu[0]), 0.0), precision)
        assert e.value.status == csl.SINGULAR_PRECOND


def test_static_precondition_fp32_range(csl):
    # |beta| = 1e37: the scales (about 1.6e-39) are below the FP32 range: refused
    # like csl_plan_create; |beta| = 1e20 needs the power-of-two prescale of the
    # FP32 scale arguments and then matches the FP64 result
    import torch
    n = 15
    v = dev(W.rhs_uniform((n, n), 35))
    with pytest.raises(csl.CSLError) as e:
        csl._binding.precondition_static(v, 1.0, 1 + 1e37j, "fp32")
    assert e.value.status == csl.INVALID_ARG
    a = csl._binding.precondition_static(v, 1.0, 1 + 1e20j, "fp32")
    b = csl._binding.precondition_static(v, 1.0, 1 + 1e20j, "fp64")
    torch.cuda.synchronize()
    assert float(b.abs().max()) > 0 and rel(a, b) < 2e-5


def test_static_precondition_rejects_oversize_grid(csl):
    import torch
    n = 1023  # 1,046,529 points > the 262,144-point static capacity
    v = torch.zeros((n, n), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(csl.CSLError) as e:
        csl._binding.precondition_static(v, 1.0, 1 + 1j)
    assert e.value.status == csl.UNSUPPORTED_SIZE
    assert "static scratch capacity" in csl.lib.csl_last_error().decode()
