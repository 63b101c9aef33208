"""Pins for the CPU oracle: each test checks the oracle against something
other than itself (a library routine, a closed form, a theorem of the paper,
a value the paper prints, or brute force), chosen so that a dropped term, a
wrong sign or index, or a transposed operand fails at least one of them."""
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.linalg
import scipy.sparse as sp

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                a, b, it = line.split()
                rows.append((float(a), float(b), int(it)))
    return rows


# --- sine transform (Section 2.3) --------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 7, 63])
def test_dst_symmetric_orthogonal(n):
    Wm = O.dst1_matrix(n)
    assert np.allclose(Wm, Wm.T, atol=0, rtol=0)
    assert np.abs(Wm @ Wm - np.eye(n)).max() < 1e-13


@pytest.mark.parametrize("n", [1, 5, 31, 64])
def test_dst_matches_scipy(n):
    rng = np.random.default_rng(n)
    v = rng.standard_normal((3, n))
    ours = O.dst(v, 0)
    ref = scipy.fft.dst(v, type=1, norm="ortho", axis=-1)
    assert np.abs(ours - ref).max() < 1e-13
    v3 = rng.standard_normal((4, 5, 6))
    for a in range(3):
        ref = scipy.fft.dst(v3, type=1, norm="ortho", axis=2 - a)
        assert np.abs(O.dst(v3, a) - ref).max() < 1e-13


@pytest.mark.parametrize("n", [1, 2, 7, 63])
def test_laplacian_eigs_closed_form(n):
    h = 1.0 / (n + 1)
    mu = O.laplacian_eigs_1d(n, h)
    k = np.arange(1, n + 1)
    closed = 2.0 * (1.0 - np.cos(k * np.pi / (n + 1))) / h ** 2
    assert np.allclose(mu, closed, rtol=1e-13, atol=0)
    T = (np.diag(2 * np.ones(n)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)) / h ** 2
    assert np.allclose(np.sort(mu), scipy.linalg.eigvalsh(T), rtol=1e-10)
    Wm = O.dst1_matrix(n)
    assert np.abs(Wm @ T @ Wm - np.diag(mu)).max() < 1e-9 * mu.max()


# --- operator K (Eq. 1) -------------------------------------------------------
def _scipy_laplacian(shape):
    """-Delta_h with Dirichlet data built from 1D tridiagonals by Kronecker sums."""
    dim = len(shape)
    mats = []
    for ax in range(dim):
        n = shape[ax]
        h = 1.0 / (n + 1)
        mats.append(sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h ** 2)
    L = None
    for ax in range(dim):
        term = None
        for bx in range(dim):
            m = mats[ax] if bx == ax else sp.identity(shape[bx])
            term = m if term is None else sp.kron(term, m)
        L = term if L is None else L + term
    return L.tocsr()


@pytest.mark.parametrize("shape", [(7, 7), (8, 5), (4, 5, 6)])
def test_K_constant_equals_scipy_laplacian(shape):
    dim = len(shape)
    n = shape[0]
    faces = []
    for a in range(dim):
        fs = list(shape)
        fs[dim - 1 - a] += 1
        faces.append(np.ones(fs))
    rng = np.random.default_rng(1)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = (_scipy_laplacian(shape) @ z.ravel()).reshape(shape)
    assert np.abs(O.apply_K(faces, z) - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 3)])
def test_K_dense_assembly_matches_slicing_and_is_symmetric(dim, n):
    faces = W.sample_faces(dim, n, W.coef_c0 if dim == 2 else W.coef_c2)
    K = O.assemble_K_dense(faces)
    assert np.allclose(K, K.T, rtol=0, atol=0)
    rng = np.random.default_rng(2)
    z = rng.standard_normal((n,) * dim)
    assert np.allclose(O.apply_K(faces, z).ravel(), K @ z.ravel(), rtol=1e-13, atol=1e-9)
    # K is an M-matrix with positive diagonal and row sums >= 0
    assert (np.diag(K) > 0).all()
    assert (K.sum(axis=1) >= -1e-9).all()


def test_K_exact_on_quadratic_variable_coefficient():
    # a = 1 + x, u = x(1-x) y(1-y): the conservative scheme with face-midpoint
    # samples is exact, -div(a grad u) = y(1-y)(1+4x) + 2(1+x) x(1-x).
    n = 9
    h = 1.0 / (n + 1)
    faces = W.sample_faces(2, n, lambda x, y: 1.0 + x + 0 * y)
    c = (np.arange(n) + 1.0) * h
    X, Y = np.meshgrid(c, c)  # Y rows, X columns (x fastest)
    u = X * (1 - X) * Y * (1 - Y)
    exact = Y * (1 - Y) * (1 + 4 * X) + 2 * (1 + X) * X * (1 - X)
    assert np.abs(O.apply_K(faces, u) - exact).max() < 1e-11


def test_K_exact_on_quadratic_3d():
    n = 6
    h = 1.0 / (n + 1)
    faces = W.sample_faces(3, n, W.coef_const(1.0))
    c = (np.arange(n) + 1.0) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    q = lambda t: t * (1 - t)
    u = q(X) * q(Y) * q(Z)
    exact = 2 * (q(Y) * q(Z) + q(X) * q(Z) + q(X) * q(Y))
    assert np.abs(O.apply_K(faces, u) - exact).max() < 1e-11


@pytest.mark.parametrize("dim,lo_axis,hi_axis", [(2, 1, 0), (2, 0, 1), (3, 2, 1), (3, 1, 2), (3, 0, 2)])
def test_gamma_from_faces_over_every_axis(dim, lo_axis, hi_axis):
    # Eq. 4: gamma = sqrt(a_min a_max) with a_min, a_max over ALL face samples
    # (reading C4).  The global minimum (0.25) sits only in the faces of
    # lo_axis and the global maximum (9.0) only in those of hi_axis; every
    # other sample is 2.0, so gamma = sqrt(0.25 * 9) = 1.5 exactly.  A min or
    # max taken over one axis's faces gives 0.25*2, 2*9 or 2*2 under the root.
    n = 3
    shape = (n,) * dim
    faces = []
    for a in range(dim):
        s = list(shape)
        s[dim - 1 - a] += 1
        faces.append(np.full(s, 2.0))
    faces[lo_axis][(1,) * dim] = 0.25
    faces[hi_axis][(0,) * dim] = 9.0
    assert O.gamma_from_faces(faces) == 1.5
    # Lemma 2.3 with these a_min, a_max: the generalised eigenvalues of (K, L)
    # lie in [0.25, 9] and the bounds are not met by the 2.0 samples alone
    if dim == 2:
        ev = scipy.linalg.eigh(O.assemble_K_dense(faces), O.assemble_L_dense(shape), eigvals_only=True)
        assert ev.min() >= 0.25 - 1e-12 and ev.max() <= 9.0 + 1e-12
        assert ev.min() < 2.0 - 1e-3 and ev.max() > 2.0 + 1e-3


def test_lemma23_rayleigh_bounds():
    # Lemma 2.3: a_min L <= K <= a_max L and L >= c0 I
    n = 15
    faces = W.sample_faces(2, n, W.coef_c1)
    amin = min(f.min() for f in faces)
    amax = max(f.max() for f in faces)
    L = O.assemble_L_dense((n, n))
    K = O.assemble_K_dense(faces)
    rng = np.random.default_rng(3)
    for _ in range(20):
        v = rng.standard_normal(n * n)
        q = (v @ K @ v) / (v @ L @ v)
        assert amin - 1e-12 <= q <= amax + 1e-12
    ev = scipy.linalg.eigh(K, L, eigvals_only=True)
    assert ev.min() >= amin - 1e-9 and ev.max() <= amax + 1e-9
    assert abs(scipy.linalg.eigvalsh(L).min() - O.c0_exact((n, n))) < 1e-8


# --- preconditioner (Eq. 3, Eq. 4) -------------------------------------------
@pytest.mark.parametrize("dim,n,alpha,beta", [(2, 5, 1.0, 10.0), (2, 6, -100.0, 1.0), (3, 3, -5.0, 50.0),
                                              (2, 4, 30.0, 0.0)])
def test_precond_equals_dense_matrix_function(dim, n, alpha, beta):
    faces = W.sample_faces(dim, n, W.coef_c0 if dim == 2 else W.coef_c2)
    gamma = O.gamma_from_faces(faces)
    L = O.assemble_L_dense((n,) * dim)
    B = gamma * L + alpha * np.eye(L.shape[0])
    P1 = np.real(scipy.linalg.sqrtm(B @ B + beta * beta * np.eye(L.shape[0])))
    rng = np.random.default_rng(4)
    v1 = rng.standard_normal((n,) * dim)
    v2 = rng.standard_normal((n,) * dim)
    z1, z2 = O.precond_apply(v1, v2, gamma, alpha, beta)
    assert np.allclose(P1 @ z1.ravel(), v1.ravel(), atol=1e-9 * np.abs(v1).max())
    assert np.allclose(P1 @ z2.ravel(), v2.ravel(), atol=1e-9 * np.abs(v2).max())


@pytest.mark.parametrize("alpha,beta", [(100.0, 100.0), (-100.0, 1.0), (1.0, -100.0)])
def test_eq3_is_matrix_abs_of_A(alpha, beta):
    # a = 1: P equals |A| computed from A's eigendecomposition (Section 1 definition)
    n = 4
    faces = W.sample_faces(2, n, W.coef_const(1.0))
    A = O.assemble_A_dense(faces, alpha, beta)
    absA = O.matrix_abs(A)
    M = n * n
    e = np.eye(2 * M)
    cols = [np.concatenate([c.ravel() for c in O.precond_apply(e[:M, j].reshape(n, n),
                                                                e[M:, j].reshape(n, n), 1.0, alpha, beta)])
            for j in range(2 * M)]
    Pinv = np.array(cols).T
    assert np.abs(absA @ Pinv - np.eye(2 * M)).max() < 1e-9


def _dense_preconditioned(faces, alpha, beta):
    n = faces[0].shape[0]
    dim = len(faces)
    shape = (n,) * dim
    M = n ** dim
    A = O.assemble_A_dense(faces, alpha, beta)
    gamma = O.gamma_from_faces(faces)
    e = np.eye(2 * M)
    cols = [np.concatenate([c.ravel() for c in O.precond_apply(e[:M, j].reshape(shape),
                                                                e[M:, j].reshape(shape), gamma, alpha, beta)])
            for j in range(2 * M)]
    return np.array(cols).T @ A


@pytest.mark.parametrize("alpha,beta", [(100.0, 100.0), (-100.0, -100.0), (-100.0, 1.0), (1.0, -100.0),
                                        (20.0, 0.0)])
def test_theorem21_eigenvalues_pm1(alpha, beta):
    faces = W.sample_faces(2, 5, W.coef_const(2.5))
    ev = np.linalg.eigvals(_dense_preconditioned(faces, alpha, beta))
    assert np.abs(np.abs(ev) - 1.0).max() < 1e-9
    assert np.abs(ev.imag).max() < 1e-9


@pytest.mark.parametrize("alpha,beta", [(0.0, 100.0), (1.0, 10.0), (50.0, 5.0), (-5.0, 50.0), (-20.0, 40.0),
                                        (-15.0, 10.0), (-12.0, 2.0)])
def test_theorem23_spectral_bounds(alpha, beta):
    n = 6
    faces = W.sample_faces(2, n, W.coef_c1)
    amin = min(f.min() for f in faces)
    amax = max(f.max() for f in faces)
    c0 = O.c0_exact((n, n))
    iv = O.theorem23_interval(amin, amax, c0, alpha, beta)
    assert iv is not None
    ev = np.linalg.eigvals(_dense_preconditioned(faces, alpha, beta))
    assert np.abs(ev.imag).max() < 1e-8
    mags = np.abs(ev.real)
    assert mags.min() >= iv[0] * (1 - 1e-12)
    assert mags.max() <= iv[1] * (1 + 1e-12)
    if alpha < 0 and O.theorem23_printed_form_applies(amin, amax, alpha, beta):
        lo, hi = O.theorem23_interval(amin, amax, c0, alpha, beta, as_printed=True)
        assert mags.min() >= lo * (1 - 1e-12) and mags.max() <= hi * (1 + 1e-12)


def test_theorem23_printed_case_ii_lower_bound_gap():
    # alpha = -5, beta = 50 on this grid: the printed mu1~ exceeds the true
    # smallest |eigenvalue|, while min(1/mu0, mu1~) holds (see theorem23_interval).
    n = 6
    faces = W.sample_faces(2, n, W.coef_c1)
    amin = min(f.min() for f in faces)
    amax = max(f.max() for f in faces)
    c0 = O.c0_exact((n, n))
    assert not O.theorem23_printed_form_applies(amin, amax, -5.0, 50.0)
    lo_printed, _ = O.theorem23_interval(amin, amax, c0, -5.0, 50.0, as_printed=True)
    mags = np.abs(np.linalg.eigvals(_dense_preconditioned(faces, -5.0, 50.0)).real)
    assert mags.min() < lo_printed


# --- MINRES (Lemma 2.1 solver) and the whole solve ----------------------------
@pytest.mark.parametrize("dim,n,coef,lam", [(2, 7, W.coef_c0, 1 + 10j), (2, 9, W.coef_c1, 100j),
                                            (3, 5, W.coef_c2, -5 + 50j), (2, 8, W.coef_c0, -100 + 1j)])
def test_solve_matches_dense_complex_lu(dim, n, coef, lam):
    faces = W.sample_faces(dim, n, coef)
    f = W.rhs_uniform((n,) * dim, 7)
    z, info = O.solve(faces, lam, f, tol=1e-13, maxit=400)
    K = O.assemble_K_dense(faces)
    ref = np.linalg.solve(K + lam * np.eye(K.shape[0]), f.ravel()).reshape(f.shape)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 1e-10
    assert O.complex_residual(faces, lam, z, f) < 1e-12


def test_rhs_order_matters():
    # the other reading of Eq. 2's right-hand side ([Re f; Im f]) gives a wrong z
    n = 6
    faces = W.sample_faces(2, n, W.coef_c0)
    f = W.rhs_uniform((n, n), 8)
    plan = O.make_plan(faces, 1 + 10j)
    x, _ = O.minres(plan.A, plan.Pinv, (f.real.copy(), f.imag.copy()), 1e-12, 200)
    z_wrong = x[0] + 1j * x[1]
    assert O.complex_residual(faces, 1 + 10j, z_wrong, f) > 1e-2


@pytest.mark.parametrize("n", [15, 63])
def test_table1a_two_iterations(n):
    faces = W.sample_faces(2, n, W.coef_const(1.0))
    f = W.rhs_normal((n, n), 11)
    for alpha, beta, iters in _golden("table1a_iterations.txt"):
        z, info = O.solve(faces, alpha + 1j * beta, f, 1e-8, 50)
        assert info.converged and info.iters == iters, (alpha, beta, info.iters)


@pytest.mark.parametrize("n", [63])
def test_table2a_fourteen_iterations(n):
    faces = W.sample_faces(2, n, W.coef_table2)
    f = W.rhs_normal((n, n), 12)
    for alpha, beta, iters in _golden("table2a_iterations.txt"):
        z, info = O.solve(faces, alpha + 1j * beta, f, 1e-8, 100)
        assert info.converged and abs(info.iters - iters) <= 1, (alpha, beta, info.iters)


def test_minres_preconditioned_residual_monotone_and_lemma21_bound():
    n = 31
    faces = W.sample_faces(2, n, W.coef_c1)
    f = W.rhs_uniform((n, n), 13)
    alpha, beta = 0.0, 100.0
    z, info = O.solve(faces, alpha + 1j * beta, f, 1e-10, 600)
    p = np.array(info.pnorm)
    assert (np.diff(p) <= 1e-12 * p[0]).all()
    amin = min(x.min() for x in faces)
    amax = max(x.max() for x in faces)
    theta = O.theorem24_factor(amin, amax, O.c0_exact((n, n)), alpha, beta)
    # Lemma 2.1 / Theorem 2.4 (i): ||r_k||_{P^-1} <= 2 theta^floor(k/2) ||r_0||_{P^-1}
    plan = O.make_plan(faces, alpha + 1j * beta)
    b = O.block_rhs(f)
    pb = plan.Pinv(b)
    r0 = math.sqrt(float(np.sum(pb[0] * b[0]) + np.sum(pb[1] * b[1])))
    for k, pk in enumerate(p, start=1):
        assert pk <= 2 * theta ** (k // 2) * r0 * (1 + 1e-9)


def test_zero_rhs_and_beta_zero():
    n = 7
    faces = W.sample_faces(2, n, W.coef_c0)
    z, info = O.solve(faces, 3.0 + 0j, np.zeros((n, n), complex))
    assert info.converged and np.all(z == 0)
    f = W.rhs_uniform((n, n), 9)
    z, info = O.solve(faces, 3.0 + 0j, f, 1e-12)
    K = O.assemble_K_dense(faces)
    ref = np.linalg.solve(K + 3.0 * np.eye(n * n), f.ravel()).reshape(n, n)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 1e-9


# --- gradients through the solve ---------------------------------------------
def _dense_solve(faces, lam, f):
    K = O.assemble_K_dense(faces)
    return np.linalg.solve(K + lam * np.eye(K.shape[0]), f.ravel()).reshape(f.shape)


def test_adjoint_and_coef_grad_against_dense_and_fd():
    n = 6
    faces = tuple(np.array(x) for x in W.sample_faces(2, n, W.coef_c0))
    lam = 1 + 20j
    f = W.rhs_uniform((n, n), 14)
    d = np.random.default_rng(15).standard_normal((n, n))
    z, _ = O.solve(faces, lam, f, 1e-13, 400)
    G = O.loss_c4_grad(z, d)
    Y, _ = O.adjoint_solve(faces, lam, G, 1e-13, 400)
    K = O.assemble_K_dense(faces)
    Yref = np.linalg.solve((K + np.conj(lam) * np.eye(n * n)), G.ravel()).reshape(n, n)
    assert np.linalg.norm(Y - Yref) / np.linalg.norm(Yref) < 1e-10
    gfaces = O.coef_grad(faces, z, Y)

    def loss_of(fc, ff):
        return O.loss_c4(_dense_solve(fc, lam, ff), d)

    eps = 1e-6
    rng = np.random.default_rng(16)
    for _ in range(4):
        dirs = [rng.standard_normal(x.shape) for x in faces]
        df = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        plus = loss_of(tuple(x + eps * e for x, e in zip(faces, dirs)), f + eps * df)
        minus = loss_of(tuple(x - eps * e for x, e in zip(faces, dirs)), f - eps * df)
        fd = (plus - minus) / (2 * eps)
        an = sum(float(np.sum(g * e)) for g, e in zip(gfaces, dirs))
        an += float(np.sum(Y.real * df.real + Y.imag * df.imag))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd))


# --- workloads -----------------------------------------------------------------
def test_workload_face_layout():
    n = 5
    ax, ay = W.sample_faces(2, n, lambda x, y: 10 * x + y)
    h = 1.0 / (n + 1)
    assert ax.shape == (n, n + 1) and ay.shape == (n + 1, n)
    assert abs(ax[2, 0] - (10 * 0.5 * h + 3 * h)) < 1e-14
    assert abs(ay[0, 2] - (10 * 3 * h + 0.5 * h)) < 1e-14
    fx, fy, fz = W.sample_faces(3, 3, lambda x, y, z: x + 10 * y + 100 * z)
    assert fx.shape == (3, 3, 4) and fy.shape == (3, 4, 3) and fz.shape == (4, 3, 3)


def test_workload_shifts_and_determinism():
    lam = W.alpha_circulant_shifts(64, 1e-4)
    assert abs(lam[0].imag) < 1e-12 and abs(lam[32].imag) < 1e-12
    assert 8.5 < lam.real.min() < 8.7 and 119.3 < lam.real.max() < 119.5
    assert np.abs(lam.imag).max() < 55.5
    a = W.rhs_uniform((4, 4), 3)
    b = W.rhs_uniform((4, 4), 3)
    assert np.array_equal(a, b) and np.abs(a.real).max() <= 1


# --- rectangular grids (n_x != n_y [!= n_z], h_a = 1/(n_a + 1) per axis) ---
def _tridiag_laplacian(n, h):
    return (2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)) / (h * h)


@pytest.mark.parametrize("ns", [(5, 3), (3, 7), (4, 3, 2), (2, 5, 3)])
def test_rectangular_K_is_kronecker_sum(ns):
    """a = 1 on an n_x x n_y (x n_z) grid: K is the Kronecker sum of the 1D
    Dirichlet Laplacians, each with its own spacing (x fastest in C order)."""
    dim = len(ns)
    faces = W.sample_faces(dim, ns, W.coef_const(1.0))
    K = O.assemble_K_dense(faces)
    T = [_tridiag_laplacian(n, 1.0 / (n + 1)) for n in ns]
    I = [np.eye(n) for n in ns]
    if dim == 2:
        ref = np.kron(I[1], T[0]) + np.kron(T[1], I[0])
    else:
        ref = (np.kron(np.kron(I[2], I[1]), T[0]) + np.kron(np.kron(I[2], T[1]), I[0]) +
               np.kron(np.kron(T[2], I[1]), I[0]))
    assert np.allclose(K, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("ns", [(7, 3), (3, 15), (7, 3, 5)])
def test_rectangular_laplacian_eigs_closed_form(ns):
    """The sine transform's eigenvalues sum_a 4/h_a^2 sin^2(k_a pi / (2(n_a+1)))
    are the spectrum of the dense rectangular Laplacian."""
    dim = len(ns)
    faces = W.sample_faces(dim, ns, W.coef_const(1.0))
    K = O.assemble_K_dense(faces)
    shape = W.grid_array_shape(dim, ns)
    mu = np.sort(O.laplacian_eigs(shape).ravel())
    ev = np.sort(np.linalg.eigvalsh(K))
    assert np.allclose(mu, ev, rtol=1e-12, atol=0)


@pytest.mark.parametrize("ns,coef,lam", [((7, 3), W.coef_c1, 100j), ((3, 7), W.coef_c0, -5 + 50j),
                                         ((3, 7, 5), W.coef_c2, 1 + 10j)])
def test_rectangular_solve_matches_dense_lu(ns, coef, lam):
    dim = len(ns)
    faces = W.sample_faces(dim, ns, coef)
    shape = W.grid_array_shape(dim, ns)
    f = W.rhs_uniform(shape, 35)
    z, info = O.solve(faces, lam, f, 1e-12, 500)
    K = O.assemble_K_dense(faces)
    zr = np.linalg.solve(K + lam * np.eye(K.shape[0]), f.ravel()).reshape(shape)
    assert info.converged
    assert np.linalg.norm(z - zr) / np.linalg.norm(zr) < 1e-9
