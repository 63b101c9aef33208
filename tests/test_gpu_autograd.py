"""Gradients through the solve (torch.autograd.Function over csl_solve,
csl_adjoint and csl_coef_grad) for L = 0.5 ||Re z - d||^2:
  - against the oracle's gradient (adjoint MINRES + per-face formula) on a small grid;
  - torch.autograd.gradcheck on a tiny grid (backward runs twice on one graph);
  - config 4 (n = 511, smoothed random coefficient, lambda = 1+20i): central
    finite differences with step 1e-6 along 32 random directions in the joint
    (f, coefficient) space.  Directions have i.i.d. standard normal entries, so
    the step moves every entry by about 1e-6.  The loss difference is formed as
    0.5 <Re(z+ - z-), Re(z+ + z-) - 2d>: neither L(+) - L(-) (a loss of about
    1e5) nor r+ - r- with r = Re z - d (each entry rounded at the size of d)
    resolves a change of 1e-6 in z.  The FD solves run to relres 1e-13."""
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


def dev(a, grad=False):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
    return t.requires_grad_(grad)


def loss_of(z, d):
    return 0.5 * ((z.real - d) ** 2).sum()


def test_autograd_matches_oracle_gradient(csl):
    n = 31
    faces = W.sample_faces(2, n, W.coef_c0)
    lam = 1 + 20j
    f = W.rhs_uniform((n, n), 51)
    d = np.random.default_rng(52).standard_normal((n, n))
    ft = dev(f, True)
    ftaces = [dev(x, True) for x in faces]
    z = csl.solve(ft, ftaces, lam, tol=1e-12, maxit=600)
    loss_of(z, dev(d)).backward()
    zr, _ = O.solve(faces, lam, f, 1e-12, 600)
    Yr, _ = O.adjoint_solve(faces, lam, O.loss_c4_grad(zr, d), 1e-12, 600)
    gfr = O.coef_grad(faces, zr, Yr)
    g = ft.grad.detach().cpu().numpy()
    assert np.linalg.norm(g - Yr) / np.linalg.norm(Yr) < 1e-9
    for a, b in zip(ftaces, gfr):
        ga = a.grad.detach().cpu().numpy()
        assert np.abs(ga - b).max() / np.abs(b).max() < 1e-9


def test_gradcheck_tiny(csl):
    import torch
    n = 7
    faces = [dev(x, True) for x in W.sample_faces(2, n, W.coef_c1)]
    f = dev(W.rhs_uniform((n, n), 53), True)
    d = dev(np.random.default_rng(54).standard_normal((n, n)))

    def fn(f, ax, ay):
        z = csl.solve(f, [ax, ay], -5 + 50j, tol=1e-14, maxit=400)
        return loss_of(z, d)

    assert torch.autograd.gradcheck(fn, (f, faces[0], faces[1]), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_config4_finite_difference_32_directions(csl):
    import torch
    s, d = W.config4()
    n = s.n
    faces = [np.array(x) for x in s.faces]
    dd = dev(d)
    ft = dev(s.f, True)
    ftaces = [dev(x, True) for x in faces]
    z = csl.solve(ft, ftaces, s.lam, tol=1e-13, maxit=3000)
    loss_of(z, dd).backward()
    gf = ft.grad.detach().cpu().numpy()
    ga = [a.grad.detach().cpu().numpy() for a in ftaces]
    sizes = [2 * n * n] + [x.size for x in faces]
    dirs = W.fd_directions(32, sizes, seed=6)
    eps = 1e-6

    def solved(fv, fc):
        assert all(float(x.min()) > 0 for x in fc)
        with csl.Plan([dev(x) for x in fc], s.lam) as p:
            zz, info = p.solve(dev(fv), tol=1e-13, maxit=3000)
        assert info.converged, info
        return zz.real

    worst = 0.0
    for v in dirs:
        o = 0
        dfr = v[o:o + n * n].reshape(n, n)
        o += n * n
        dfi = v[o:o + n * n].reshape(n, n)
        o += n * n
        dfaces = []
        for x in faces:
            dfaces.append(v[o:o + x.size].reshape(x.shape))
            o += x.size
        df = dfr + 1j * dfi
        rp = solved(s.f + eps * df, [x + eps * e for x, e in zip(faces, dfaces)])
        rm = solved(s.f - eps * df, [x - eps * e for x, e in zip(faces, dfaces)])
        fd = float(0.5 * torch.sum((rp - rm) * (rp + rm - 2 * dd))) / (2 * eps)
        an = float(np.sum(gf.real * dfr + gf.imag * dfi)) + sum(float(np.sum(g * e)) for g, e in zip(ga, dfaces))
        err = abs(fd - an) / max(abs(an), 1e-300)
        worst = max(worst, err)
        assert err <= 1e-5, (fd, an, err)
    print(f"config 4 FD check: worst relative error over 32 directions {worst:.2e}")
