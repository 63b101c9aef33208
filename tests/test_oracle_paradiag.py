"""Pins of the oracle's all-at-once time solve (the alpha-circulant setting of
Section 1 that produces the shifted systems) against independent
constructions: the dense alpha-circulant matrix, the config-3 shift set, the
dense all-at-once matrix, and sequential backward Euler by dense LU."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def same_set(a, b, tol):
    """Every element of a has one of b within tol and vice versa (order-free)."""
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return len(a) == len(b) and all(np.abs(b - x).min() <= tol for x in a) and \
        all(np.abs(a - y).min() <= tol for y in b)


@pytest.mark.parametrize("L,a", [(8, 1e-4), (8, 0.3), (5, 0.05)])
def test_alpha_circulant_is_diagonalised_by_scaled_dft(L, a):
    tau = 1.0 / L
    C = O.paradiag_circulant(L, tau, a)
    # the corner entry and the subdiagonal are the definition of C_a
    assert C[0, L - 1] == pytest.approx(-a / tau) and np.allclose(np.diag(C, -1), -1.0 / tau)
    j = np.arange(L)
    Gam = np.diag(a ** (-j / L))
    Fd = np.exp(-2j * np.pi * np.outer(j, j) / L)
    rebuilt = Gam @ np.linalg.inv(Fd) @ np.diag(O.paradiag_shifts(L, tau, a)) @ Fd @ np.linalg.inv(Gam)
    assert np.allclose(rebuilt, C, atol=1e-10 * np.abs(C).max())
    # and its eigenvalues are the shifts
    ev = np.linalg.eigvals(C)
    d = O.paradiag_shifts(L, tau, a)
    assert same_set(ev, d, 1e-8 * np.abs(d).max())


def test_shifts_are_the_config3_workload():
    """config 3's lambda_k = (1 - eps^{1/L} e^{2 pi i k/L}) L is the shift set
    of backward Euler on [0, 1] with L = 64 steps and a = eps = 1e-4."""
    d = O.paradiag_shifts(64, 1.0 / 64, 1e-4)
    lam = W.alpha_circulant_shifts(64, 1e-4)
    assert same_set(d, lam, 1e-12 * 64)


def _dense_K(faces):
    return O.assemble_K_dense(faces)


def test_all_at_once_apply_matches_dense_kronecker():
    n, L, tau = 3, 4, 0.2
    faces = W.sample_faces(2, n, W.coef_c0)
    K = _dense_K(faces)
    B = O.paradiag_time_matrix(L, tau)
    A = np.kron(B, np.eye(n * n)) + np.kron(np.eye(L), K)
    U = W.rhs_normal((L, n, n), 50)
    assert np.allclose(O.paradiag_apply(faces, tau, U).ravel(), A @ U.ravel(), atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("a", [1e-4, 0.1])
def test_preconditioner_inverts_P_alpha(a):
    n, L, tau = 7, 8, 1.0 / 8
    faces = W.sample_faces(2, n, W.coef_c1)
    K = _dense_K(faces)
    P = np.kron(O.paradiag_circulant(L, tau, a), np.eye(n * n)) + np.kron(np.eye(L), K)
    U = W.rhs_normal((L, n, n), 51)
    R = (P @ U.ravel()).reshape(U.shape)
    Z = O.paradiag_precond(faces, tau, a, R, tol=1e-13)
    assert np.linalg.norm(Z - U) / np.linalg.norm(U) < 1e-9


def test_richardson_converges_to_backward_euler():
    n, L, tau, a = 7, 8, 1.0 / 8, 1e-3
    faces = W.sample_faces(2, n, W.coef_c0)
    u0 = W.rhs_uniform((n, n), 52)
    g = W.rhs_normal((L, n, n), 53)
    # reference: step by step with dense LU, independent of MINRES
    K = _dense_K(faces)
    Mstep = K + np.eye(n * n) / tau
    ref = np.empty((L, n * n), dtype=np.complex128)
    prev = u0.ravel()
    for t in range(L):
        ref[t] = np.linalg.solve(Mstep, g[t].ravel() + prev / tau)
        prev = ref[t]
    U, hist = O.paradiag_solve(faces, tau, a, u0, g, tol=1e-11, maxit=10)
    assert hist[-1] <= 1e-11
    assert np.linalg.norm(U.reshape(L, -1) - ref) / np.linalg.norm(ref) < 1e-10
    # contraction per sweep of the order of a / (1 - a)
    for h0, h1 in zip(hist[:-1], hist[1:]):
        assert h1 <= 0.05 * h0
    # the step-by-step oracle solve agrees with dense LU as well
    ts = O.paradiag_time_stepping(faces, tau, u0, g)
    assert np.linalg.norm(ts.reshape(L, -1) - ref) / np.linalg.norm(ref) < 1e-10
