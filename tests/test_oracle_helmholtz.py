"""Pins of the oracle's shifted-Laplace preconditioned Helmholtz solve
(Section 1's first setting): dense LU of (K + lam_A I), and the closed form
of the exactly preconditioned spectrum: with lam_A = -k^2 and
lam_M = -k^2 (1 - i b), every eigenvalue mu = (l - k^2)/(l - k^2 + i b k^2) of
(K + lam_A I)(K + lam_M I)^{-1} (l an eigenvalue of K) lies on |mu - 1/2| = 1/2."""
import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.mark.parametrize("k2,b", [(200.0, 0.5), (900.0, 0.5), (900.0, 1.0)])
def test_exactly_preconditioned_spectrum_on_the_circle(k2, b):
    n = 7
    faces = W.sample_faces(2, n, W.coef_c1)
    K = O.assemble_K_dense(faces)
    I = np.eye(n * n)
    A = K - k2 * I
    Mm = K - k2 * (1 - 1j * b) * I
    mu = np.linalg.eigvals(A @ np.linalg.inv(Mm))
    assert np.allclose(np.abs(mu - 0.5), 0.5, atol=1e-10)
    # and through the eigenvalues of K directly
    lk = np.linalg.eigvalsh(K)
    mu2 = (lk - k2) / (lk - k2 + 1j * b * k2)
    assert np.allclose(np.sort_complex(np.round(mu, 9)), np.sort_complex(np.round(mu2, 9)), atol=1e-8)


# resolved wave numbers: k h between about 0.5 and 0.8
@pytest.mark.parametrize("n,k2,coef", [(15, 64.0, W.coef_c0), (31, 256.0, W.coef_c1), (31, 400.0, W.coef_c0)])
def test_fgmres_matches_dense_lu(n, k2, coef):
    faces = W.sample_faces(2, n, coef)
    f = W.rhs_uniform((n, n), 70)
    K = O.assemble_K_dense(faces)
    ref = np.linalg.solve(K - k2 * np.eye(n * n), f.ravel()).reshape(n, n)
    u, info = O.helmholtz_fgmres(faces, -k2, -k2 * (1 - 0.5j), f, tol=1e-10, maxit=300, restart=60,
                                 inner_tol=1e-8)
    assert info["relres"] <= 1e-10 * 1.01
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-7
    # the Arnoldi estimate is the true residual of the minimiser (exact arithmetic, flexible GMRES)
    assert info["hist"][-1] == pytest.approx(info["relres"], rel=1e-3, abs=1e-13)
