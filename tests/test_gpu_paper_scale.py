"""Long transform lines (N = 2048 .. 16384, 2D): the grid sizes of the paper's
largest tables (Tables 1(a) and 2(a) print n = 2^12 - 1 and 2^14 - 1; lines
of 16384 FP64 points run on two-CTA clusters).

  - n = 2047: operator and P^{-1} element by element against the oracle;
  - n = 4095, 8191 and 16383 (FP64): P^{-1} of sums of sine eigenmodes, which
    Section 2.3 maps to the same modes scaled by
    1/sqrt((gamma (mu_i + mu_j) + alpha)^2 + beta^2), a closed form that holds
    at any size;
  - the tables' solves at n = 4095 (FP64 and FP32), 8191 and 16383 (FP64)
    against the iteration counts the paper prints (2 for a = 1, Table 1(a);
    14 for a = (20+x^2)(20+y^2), Table 2(a)), with the residual checked by the
    oracle's operator (n = 4095) or point by point from the stencil
    definition (larger grids)."""
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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# FP32: the rounding of a length-N FFT grows like log N; 2.6e-5 measured at N = 2048
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-5)])
def test_n2047_against_oracle(csl, precision, tol):
    n = 2047
    faces = W.sample_faces(2, n, W.coef_c1)
    lam = 1 + 10j
    v = W.rhs_uniform((n, n), 80)
    gamma = O.gamma_from_faces(faces)
    r1, r2 = O.precond_apply(v.real, v.imag, gamma, lam.real, lam.imag)
    with csl.Plan([dev(f) for f in faces], lam, precision=precision) as plan:
        assert "long-line" in plan.config, plan.config
        out = host(plan.precondition(dev(v)))
        az = host(plan.apply(dev(v)))
    assert rel(out, r1 + 1j * r2) < tol
    assert rel(az, O.apply_K(faces, v) + lam * v) < 1e-13


def _modes(n, modes, coefs):
    import torch
    x = (torch.arange(1, n + 1, dtype=torch.float64, device="cuda:0")) / (n + 1)
    v = torch.zeros((n, n), dtype=torch.complex128, device="cuda:0")
    for (kx, ky), c in zip(modes, coefs):
        v += c * torch.outer(torch.sin(math.pi * ky * x), torch.sin(math.pi * kx * x)).to(torch.complex128)
    return v


# FP32: a single high-frequency mode carries the transform's rounding scaled by
# the spread of the per-mode factor, about eps_32 kappa(P) (kappa ~ n^2): 2e-4
# measured at n = 1023, and the bound below at n = 4095
@pytest.mark.parametrize("n,precision,tol", [(4095, "fp64", 1e-11), (8191, "fp64", 1e-11), (16383, "fp64", 1e-11),
                                             (4095, "fp32", 5e-3)])
def test_sine_modes_closed_form(csl, n, precision, tol):
    import torch
    faces = W.sample_faces(2, n, W.coef_const(1.0))
    lam = -100 + 100j
    modes = [(1, 1), (7, 3000 % n), (n - 2, 5)]
    coefs = [1.0, 0.5 - 0.25j, 2.0j]
    v = _modes(n, modes, coefs)
    h2 = 1.0 / (n + 1) ** 2
    mu = lambda k: 4.0 / h2 * math.sin(k * math.pi / (2 * (n + 1))) ** 2
    with csl.Plan([dev(f) for f in faces], lam, precision=precision) as plan:
        gamma = plan.gamma
        out = plan.precondition(v)
    expect = torch.zeros_like(v)
    for (kx, ky), c in zip(modes, coefs):
        s = 1.0 / math.sqrt((gamma * (mu(kx) + mu(ky)) + lam.real) ** 2 + lam.imag ** 2)
        expect += _modes(n, [(kx, ky)], [c * s])
    err = float((out - expect).abs().max() / expect.abs().max())
    print(f"sine modes n={n} {precision}: max rel error {err:.2e}")
    assert err < tol


def point_apply(faces, lam, z, idx):
    n = z.shape[0]
    h2 = 1.0 / (n + 1) ** 2
    acc = lam * z[idx]
    mag = abs(acc)
    for ax in range(2):
        arr_ax = 1 - ax
        for side in (0, 1):
            fidx = list(idx)
            fidx[arr_ax] = idx[arr_ax] + side
            a = faces[ax][tuple(fidx)]
            q = list(idx)
            q[arr_ax] = idx[arr_ax] + (1 if side else -1)
            zq = z[tuple(q)] if 0 <= q[arr_ax] < n else 0.0
            acc += a * (z[idx] - zq) / h2
            mag += a * (abs(z[idx]) + abs(zq)) / h2
    return acc, mag


@pytest.mark.parametrize("n,precision", [(4095, "fp64"), (4095, "fp32"), (8191, "fp64"), (16383, "fp64")])
@pytest.mark.parametrize("table", ["1a", "2a"])
def test_paper_tables_at_scale(csl, n, precision, table):
    coef = W.coef_const(1.0) if table == "1a" else W.coef_table2
    shifts = W.TABLE1_SHIFTS if table == "1a" else W.TABLE2_SHIFTS
    printed = 2 if table == "1a" else 14
    faces = W.sample_faces(2, n, coef)
    f = W.rhs_normal((n, n), 81)
    dfaces = [dev(x) for x in faces]
    fd = dev(f)
    rng = np.random.default_rng(82)
    for alpha, beta in shifts:
        lam = alpha + 1j * beta
        with csl.Plan(dfaces, lam, precision=precision) as plan:
            z, info = plan.solve(fd, tol=1e-8, maxit=200)
            zg = host(z)
        print(f"Table {table} n={n} {precision} ({alpha},{beta}): Iter {info.iters} (paper {printed}) "
              f"relres {info.relres:.2e}")
        assert info.converged and info.relres <= 1e-8
        if precision == "fp64" and table == "2a":
            assert abs(info.iters - printed) <= 2, (alpha, beta, info.iters)
        elif precision == "fp64":
            # Table 1(a): exactly 2 (Theorem 2.2), except that the stopping test is on
            # the true residual (reading C6) and FP64 rounding in P^{-1} grows like
            # eps_64 kappa(P): at n = 16383 the nearly resonant shift (-100, 1) (kappa(P)
            # about 2e9) leaves relres just above 1e-8 after the two ideal steps (n = 8191:
            # 6.2e-9), so one more pair of steps is allowed there
            assert info.iters == printed or (n >= 16383 and info.iters <= printed + 2), (alpha, beta, info.iters)
        elif table == "1a":
            # the FP32 P^{-1} is |A|^{-1} only to about eps_32 kappa(P): at n = 4095
            # 8 iterations, 21 for the nearly real shift (-100, 1)
            assert 2 <= info.iters <= 25, (alpha, beta, info.iters)
        else:
            assert abs(info.iters - printed) <= 2 + int(0.06 * printed), (alpha, beta, info.iters)
        if n <= 4095:
            assert O.complex_residual(faces, lam, zg, f) <= 1e-8
        else:
            # (K + lam I) z by the library's stencil, its entries checked at
            # sampled points against the definition, then the true residual
            Az = host(plan_apply(csl, dfaces, lam, z))
            for _ in range(32):
                idx = (int(rng.integers(0, n)), int(rng.integers(0, n)))
                ref, mag = point_apply(faces, lam, zg, idx)
                assert abs(Az[idx] - ref) <= 1e-14 * mag
            assert np.linalg.norm(f - Az) / np.linalg.norm(f) <= 1e-8


def plan_apply(csl, dfaces, lam, z):
    with csl.Plan(dfaces, lam, autotune=False) as p:
        return p.apply(z)
