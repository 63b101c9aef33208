"""Plain FP64 CPU oracle for the absolute-value-preconditioned MINRES solve of
complex-shifted Laplacian systems (arXiv 2408.00488).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
the benchmark do.  It shares no code with the CUDA path; the two meet only at
the seeded input generators in `workloads`.

Everything is float64 / complex128 NumPy, written for readability: dense
matrices and O(n^2) sine transforms, explicit slicing for the stencil, the
textbook preconditioned MINRES recurrence.  Function by function:

  apply_K            Eq. 1 operator K = FD discretisation of -div(a grad)
                     (Section 1; 5/7-point conservative stencil, face samples)
  assemble_K_dense   the same matrix built entry by entry (tiny grids)
  block_apply        Eq. 2, the 2x2 block real matrix A
  dst1_matrix / dst  Section 2.3, the real symmetric orthogonal sine transform W
  laplacian_eigs_1d  Section 2.3, the diagonal of L = W Lambda W in 1D
  precond_apply      Eq. 3 / Eq. 4, P^{-1} v = W diag(1/sqrt((gamma Lambda+alpha)^2+beta^2)) W v
  gamma_from_faces   Eq. 4, gamma = sqrt(a_min a_max)
  minres             Lemma 2.1's solver (preconditioned MINRES, zero guess)
  solve              Section 3: the whole solve for (K + lambda I) z = f
  adjoint_solve / coef_grad
                     gradients of a loss through the solve (not in the paper;
                     derived from Eq. 2 by differentiating A x = r)
  matrix_abs / theorem helpers
                     the definitions of |H| and sqrt(H) (Section 1) and the
                     bounds of Theorem 2.3 / 2.4, for invariant tests.
  helmholtz_fgmres   the other setting of Section 1: the shifted system as
                     the (shifted-Laplace) preconditioner of an outer
                     Krylov solve of (K + lambda_A I) u = f, lambda_A = -k^2
                     (flexible GMRES, right preconditioning).
  paradiag_*         the all-at-once time solve that motivates the shifted
                     systems (Section 1): backward Euler for u' + K u = g as
                     one block system, the alpha-circulant approximation of
                     its time matrix, its diagonalisation by the DFT in time
                     into complex-shifted Laplacian systems, and the
                     preconditioned Richardson iteration built on them.

Readings where the paper is silent or garbled (each is also listed in the
design notes): unit square/cube with homogeneous Dirichlet data and
h = 1/(n+1); coefficient sampled at face midpoints; the right-hand side of
Eq. 2 taken as [Im f; Re f] so that z = z1 + i z2 solves Eq. 1; gamma from the
min/max of the supplied face samples; orthonormal DST-I; stopping on the true
relative residual ||f - (K + lambda I) z|| / ||f||; "Iter" = number of
A-products in the MINRES loop.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np


# ---------------------------------------------------------------------------
# Operator K (Eq. 1): (K z)_p = sum over the faces e of p of a_e (z_p - z_q)/h_e^2,
# z_q = 0 across the Dirichlet boundary.
# ---------------------------------------------------------------------------
def _np_axis(dim: int, spatial_axis: int) -> int:
    """numpy axis of spatial axis 0=x, 1=y, 2=z (x is the last numpy axis)."""
    return dim - 1 - spatial_axis


def grid_shape(faces) -> Tuple[int, ...]:
    dim = len(faces)
    shape = list(faces[0].shape)
    shape[_np_axis(dim, 0)] -= 1
    return tuple(shape)


def spacings(shape) -> List[float]:
    """h per spatial axis on the unit square/cube, h = 1/(n+1)."""
    dim = len(shape)
    return [1.0 / (shape[_np_axis(dim, a)] + 1) for a in range(dim)]


def apply_K(faces, z: np.ndarray) -> np.ndarray:
    """(K z) for the conservative FD discretisation of -div(a grad z),
    Section 1 (Eq. 1).  Works for real or complex z of the grid's shape."""
    dim = len(faces)
    h = spacings(z.shape)
    out = np.zeros_like(z)
    for a in range(dim):
        ax = _np_axis(dim, a)
        pad = [(0, 0)] * dim
        pad[ax] = (1, 1)
        zp = np.pad(z, pad)  # zero Dirichlet neighbours
        n_a = z.shape[ax]
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[ax] = slice(0, n_a + 1)
        hi[ax] = slice(1, n_a + 2)
        # flux through face i (between grid indices i-1 and i): a_i (z_i - z_{i-1})
        flux = faces[a] * (zp[tuple(hi)] - zp[tuple(lo)])
        left = [slice(None)] * dim
        right = [slice(None)] * dim
        left[ax] = slice(0, n_a)
        right[ax] = slice(1, n_a + 1)
        out = out + (flux[tuple(left)] - flux[tuple(right)]) / (h[a] * h[a])
    return out


def assemble_K_dense(faces) -> np.ndarray:
    """Dense M x M matrix of K, entry by entry (tiny grids only).  Point
    numbering is the C order of the grid (x fastest)."""
    dim = len(faces)
    shape = grid_shape(faces)
    h = spacings(shape)
    M = int(np.prod(shape))
    K = np.zeros((M, M))
    for p in range(M):
        idx = np.unravel_index(p, shape)
        for a in range(dim):
            ax = _np_axis(dim, a)
            for side in (-1, +1):
                # face between idx and idx+side along ax; face index = idx[ax] (+1 if side>0)
                fidx = list(idx)
                fidx[ax] = idx[ax] + (1 if side > 0 else 0)
                ae = faces[a][tuple(fidx)] / (h[a] * h[a])
                K[p, p] += ae
                q = list(idx)
                q[ax] = idx[ax] + side
                if 0 <= q[ax] < shape[ax]:
                    K[p, np.ravel_multi_index(tuple(q), shape)] -= ae
    return K


def assemble_L_dense(shape) -> np.ndarray:
    """Dense matrix of the constant-coefficient Laplacian L (a = 1)."""
    dim = len(shape)
    faces = []
    for a in range(dim):
        fs = list(shape)
        fs[_np_axis(dim, a)] += 1
        faces.append(np.ones(fs))
    return assemble_K_dense(faces)


# ---------------------------------------------------------------------------
# Eq. 2: the 2x2 block real system  A = [[beta I, K + alpha I], [K + alpha I, -beta I]].
# Right-hand side [Im f; Re f] (reading of the garbled right-hand side: with
# z = z1 + i z2, row 1 is Im((K+lambda)z) and row 2 is Re((K+lambda)z)).
# ---------------------------------------------------------------------------
def block_apply(faces, alpha: float, beta: float, x1: np.ndarray, x2: np.ndarray):
    Kx1 = apply_K(faces, x1)
    Kx2 = apply_K(faces, x2)
    y1 = beta * x1 + Kx2 + alpha * x2
    y2 = Kx1 + alpha * x1 - beta * x2
    return y1, y2


def block_rhs(f: np.ndarray):
    return np.ascontiguousarray(f.imag), np.ascontiguousarray(f.real)


def assemble_A_dense(faces, alpha: float, beta: float) -> np.ndarray:
    K = assemble_K_dense(faces)
    M = K.shape[0]
    I = np.eye(M)
    return np.block([[beta * I, K + alpha * I], [K + alpha * I, -beta * I]])


# ---------------------------------------------------------------------------
# Section 2.3: W = real symmetric orthogonal DST-I, L = W Lambda W.
# ---------------------------------------------------------------------------
def dst1_matrix(n: int) -> np.ndarray:
    """W_{jk} = sqrt(2/(n+1)) sin(j k pi/(n+1)), j, k = 1..n."""
    j = np.arange(1, n + 1, dtype=np.float64)
    return math.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(j, j) / (n + 1))


def dst(v: np.ndarray, spatial_axis: int) -> np.ndarray:
    """Orthonormal DST-I along one spatial axis as a dense O(n^2) product."""
    dim = v.ndim
    ax = _np_axis(dim, spatial_axis)
    W = dst1_matrix(v.shape[ax])
    return np.moveaxis(np.tensordot(W, v, axes=([1], [ax])), 0, ax)


def dst_all(v: np.ndarray) -> np.ndarray:
    """W (x) W (x) W applied to a grid function (all axes)."""
    for a in range(v.ndim):
        v = dst(v, a)
    return v


def laplacian_eigs_1d(n: int, h: float) -> np.ndarray:
    """Eigenvalues of the 1D Dirichlet Laplacian tridiag(-1, 2, -1)/h^2 in the
    sine basis: mu_k = (4/h^2) sin^2(k pi / (2(n+1))), k = 1..n."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return 4.0 / (h * h) * np.sin(k * np.pi / (2.0 * (n + 1))) ** 2


def laplacian_eigs(shape) -> np.ndarray:
    """Eigenvalues of L on the grid, arranged like the grid (sum over axes)."""
    dim = len(shape)
    h = spacings(shape)
    lam = np.zeros(shape)
    for a in range(dim):
        ax = _np_axis(dim, a)
        mu = laplacian_eigs_1d(shape[ax], h[a])
        s = [1] * dim
        s[ax] = mu.size
        lam = lam + mu.reshape(s)
    return lam


# ---------------------------------------------------------------------------
# Eq. 4 (and Eq. 3 when a is constant):
#   P = blkdiag(sqrt((gamma L + alpha I)^2 + beta^2 I), same),  gamma = sqrt(a_min a_max).
#   P^{-1} v = W diag(1/sqrt((gamma Lambda + alpha)^2 + beta^2)) W v, per block.
# ---------------------------------------------------------------------------
def gamma_from_faces(faces) -> float:
    amin = min(float(np.min(f)) for f in faces)
    amax = max(float(np.max(f)) for f in faces)
    return math.sqrt(amin * amax)


def precond_eigs(shape, gamma: float, alpha: float, beta: float) -> np.ndarray:
    """sqrt((gamma Lambda + alpha)^2 + beta^2): the eigenvalues of each block of P."""
    lam = laplacian_eigs(shape)
    return np.sqrt((gamma * lam + alpha) ** 2 + beta * beta)


def precond_apply(v1: np.ndarray, v2: np.ndarray, gamma: float, alpha: float, beta: float):
    d = precond_eigs(v1.shape, gamma, alpha, beta)
    z1 = dst_all(dst_all(v1) / d)
    z2 = dst_all(dst_all(v2) / d)
    return z1, z2


# ---------------------------------------------------------------------------
# Section 1: |H| and sqrt(H) for real symmetric H, by the eigendecomposition.
# ---------------------------------------------------------------------------
def matrix_abs(H: np.ndarray) -> np.ndarray:
    w, Q = np.linalg.eigh(H)
    return (Q * np.abs(w)) @ Q.T


def matrix_sqrt(H: np.ndarray) -> np.ndarray:
    w, Q = np.linalg.eigh(H)
    if np.min(w) < -1e-12 * max(1.0, np.max(np.abs(w))):
        raise ValueError("sqrt of a matrix with negative eigenvalues")
    return (Q * np.sqrt(np.maximum(w, 0.0))) @ Q.T


# ---------------------------------------------------------------------------
# Lemma 2.1's solver: preconditioned MINRES (Paige-Saunders recurrence in the
# form of Elman, Silvester & Wathen), zero initial guess.
# Vectors are pairs (block 1, block 2); <u, v> is the real inner product on R^{2M}.
# ---------------------------------------------------------------------------
def _dot(u, v) -> float:
    return float(np.vdot(u[0], v[0]).real + np.vdot(u[1], v[1]).real)


def _axpy(a, x, y):  # a*x + y
    return (a * x[0] + y[0], a * x[1] + y[1])


def _scale(a, x):
    return (a * x[0], a * x[1])


@dataclass
class MinresInfo:
    iters: int = 0
    relres: float = float("nan")
    converged: bool = False
    history: List[float] = field(default_factory=list)   # true relres per iteration
    pnorm: List[float] = field(default_factory=list)     # |eta|: P^{-1}-norm residual estimate
    breakdown: bool = False


def minres(apply_A: Callable, apply_Pinv: Callable, b, tol: float = 1e-8,
           maxit: int = 500, x0=None) -> Tuple[tuple, MinresInfo]:
    """Preconditioned MINRES for the symmetric A x = b with SPD preconditioner P.

    Lanczos in the P^{-1} inner product: v_{j+1} = A z_j - (delta_j/gamma_j) v_j
    - (gamma_j/gamma_{j-1}) v_{j-1}, z_j = P^{-1} v_j / gamma_j,
    gamma_j = sqrt(<P^{-1} v_j, v_j>), delta_j = <A z_j, z_j>; the tridiagonal
    least-squares problem is solved by Givens rotations (c, s), the iterate by
    the three-term direction recurrence w.  Stops when the TRUE relative
    residual ||b - A x|| / ||b|| <= tol (computed explicitly every iteration)
    or on a lucky breakdown gamma_{j+1} = 0 (x exact).
    """
    info = MinresInfo()
    if x0 is None:
        x = (np.zeros_like(b[0]), np.zeros_like(b[1]))
        r = b
    else:
        x = x0
        Ax = apply_A(x)
        r = (b[0] - Ax[0], b[1] - Ax[1])
    bnorm = math.sqrt(_dot(b, b))
    if bnorm == 0.0:
        info.converged, info.relres = True, 0.0
        return x, info
    zero = (np.zeros_like(b[0]), np.zeros_like(b[1]))
    v_old, v = zero, r
    z = apply_Pinv(v)
    g2 = _dot(z, v)
    if not (g2 > 0.0) or not math.isfinite(g2):
        info.breakdown = True
        return x, info
    gam_old, gam = 1.0, math.sqrt(g2)
    eta = gam
    c_old, c = 1.0, 1.0
    s_old, s = 0.0, 0.0
    w_old, w = zero, zero
    gam1 = gam
    for j in range(1, maxit + 1):
        z = _scale(1.0 / gam, z)
        Az = apply_A(z)
        delta = _dot(Az, z)
        v_new = (Az[0] - (delta / gam) * v[0] - (gam / gam_old) * v_old[0],
                 Az[1] - (delta / gam) * v[1] - (gam / gam_old) * v_old[1])
        z_new = apply_Pinv(v_new)
        g2 = _dot(z_new, v_new)
        if g2 < 0.0 or not math.isfinite(g2):
            info.breakdown = True
            info.iters = j
            break
        gam_new = math.sqrt(g2)
        a0 = c * delta - c_old * s * gam
        a1 = math.sqrt(a0 * a0 + gam_new * gam_new)
        a2 = s * delta + c_old * c * gam
        a3 = s_old * gam
        c_new, s_new = a0 / a1, gam_new / a1
        w_new = ((z[0] - a3 * w_old[0] - a2 * w[0]) / a1,
                 (z[1] - a3 * w_old[1] - a2 * w[1]) / a1)
        x = _axpy(c_new * eta, w_new, x)
        eta = -s_new * eta
        Ax = apply_A(x)
        res = (b[0] - Ax[0], b[1] - Ax[1])
        relres = math.sqrt(_dot(res, res)) / bnorm
        info.history.append(relres)
        info.pnorm.append(abs(eta))
        info.iters, info.relres = j, relres
        v_old, v = v, v_new
        z = z_new
        gam_old, gam = gam, gam_new
        w_old, w = w, w_new
        c_old, c = c, c_new
        s_old, s = s, s_new
        if relres <= tol:
            info.converged = True
            break
        if gam_new <= 1e-14 * gam1:  # lucky breakdown: Krylov space invariant
            info.converged = relres <= tol
            break
    return x, info


# ---------------------------------------------------------------------------
# Section 3: the whole solve of (K + lambda I) z = f through Eq. 2 and Eq. 4.
# ---------------------------------------------------------------------------
@dataclass
class Plan:
    faces: tuple
    alpha: float
    beta: float
    gamma: float

    @property
    def shape(self):
        return grid_shape(self.faces)

    def A(self, x):
        return block_apply(self.faces, self.alpha, self.beta, x[0], x[1])

    def Pinv(self, v):
        return precond_apply(v[0], v[1], self.gamma, self.alpha, self.beta)


def make_plan(faces, lam: complex, gamma: Optional[float] = None) -> Plan:
    faces = tuple(np.asarray(f, dtype=np.float64) for f in faces)
    g = gamma_from_faces(faces) if gamma is None else float(gamma)
    return Plan(faces, float(np.real(lam)), float(np.imag(lam)), g)


def solve(faces, lam: complex, f: np.ndarray, tol: float = 1e-8, maxit: int = 500,
          gamma: Optional[float] = None):
    """z with (K + lambda I) z = f by preconditioned MINRES on Eq. 2; returns
    (z complex128, MinresInfo)."""
    plan = make_plan(faces, lam, gamma)
    b = block_rhs(np.asarray(f, dtype=np.complex128))
    x, info = minres(plan.A, plan.Pinv, b, tol, maxit)
    return x[0] + 1j * x[1], info


def complex_residual(faces, lam: complex, z: np.ndarray, f: np.ndarray) -> float:
    """||f - (K + lambda I) z|| / ||f|| evaluated directly in complex form."""
    r = f - (apply_K(faces, z) + lam * z)
    return float(np.linalg.norm(r) / np.linalg.norm(f))


# ---------------------------------------------------------------------------
# Gradients through the solve (not in the paper; derived from Eq. 2).
# With x = A^{-1} [Im f; Re f] and g = [dL/dRe z; dL/dIm z], y = A^{-1} g
# (A is symmetric).  In complex form Y = y2 + i y1 solves (K + conj(lambda) I) Y = G,
# G = dL/dRe z + i dL/dIm z, and
#   dL/df   = Y                                  (dL/dRe f + i dL/dIm f),
#   dL/da_e = -h_e^{-2} Re(conj(D_e Y) D_e z),    D_e u = u_p - u_q (zero outside).
# ---------------------------------------------------------------------------
def adjoint_solve(faces, lam: complex, G: np.ndarray, tol: float = 1e-8,
                  maxit: int = 500, gamma: Optional[float] = None):
    return solve(faces, np.conj(lam), G, tol, maxit, gamma)


def coef_grad(faces, z: np.ndarray, Y: np.ndarray):
    """dL/da_e for every face sample, given the solution z and the adjoint Y."""
    dim = len(faces)
    h = spacings(z.shape)
    grads = []
    for a in range(dim):
        ax = _np_axis(dim, a)
        pad = [(0, 0)] * dim
        pad[ax] = (1, 1)
        zp = np.pad(z, pad)
        yp = np.pad(Y, pad)
        n_a = z.shape[ax]
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[ax] = slice(0, n_a + 1)
        hi[ax] = slice(1, n_a + 2)
        dz = zp[tuple(hi)] - zp[tuple(lo)]
        dy = yp[tuple(hi)] - yp[tuple(lo)]
        grads.append(-np.real(np.conj(dy) * dz) / (h[a] * h[a]))
    return tuple(grads)


def loss_c4(z: np.ndarray, d: np.ndarray) -> float:
    """0.5 ||Re z - d||^2 and its complex gradient G = dL/dRe z + i dL/dIm z."""
    return 0.5 * float(np.sum((z.real - d) ** 2))


def loss_c4_grad(z: np.ndarray, d: np.ndarray) -> np.ndarray:
    return (z.real - d) + 0j


# ---------------------------------------------------------------------------
# Theorem 2.3 / 2.4 bounds, for invariant tests.
# ---------------------------------------------------------------------------
def c0_exact(shape) -> float:
    """lambda_min(L) on the grid (the sharpest c0 of Lemma 2.3 (ii))."""
    return float(np.min(laplacian_eigs(shape)))


def theorem23_interval(amin: float, amax: float, c0: float, alpha: float, beta: float,
                       as_printed: bool = False):
    """(lower, upper) bounds of |eig(P^{-1} A)| from Theorem 2.3, or None when
    its assumption for alpha < 0 does not hold.

    Case (i), alpha >= 0: [1/mu0, mu0], mu0 = sqrt(2 a_max/a_min).
    Case (ii), alpha < 0 and a_min c0 + |beta| + alpha > 0: the printed
    [mu1~, mu0~].  The proof's last step bounds a quotient
    (c l + d)/(l + e) over l >= c0 by its value at l = c0, which is the
    supremum only when the numerator coefficient is positive; otherwise the
    supremum is the l -> infinity limit, which is the case-(i) value.  So,
    unless `as_printed`, case (ii) returns [min(1/mu0, mu1~), max(mu0, mu0~)],
    which equals the printed interval whenever both coefficients are positive.
    """
    gamma = math.sqrt(amin * amax)
    mu0 = math.sqrt(2.0 * amax / amin)
    if alpha >= 0:
        # case (i): its proof uses only K + alpha I >= 0, so no further assumption
        return 1.0 / mu0, mu0
    if amin * c0 + abs(beta) + alpha <= 0:  # case (ii) assumption (= amin c0 + |beta| - |alpha| > 0)
        return None
    mt0 = math.sqrt(2.0) * (c0 * amax + abs(beta) - alpha) / (c0 * gamma + abs(beta) + alpha)
    mt1 = math.sqrt(2.0) * (c0 * amin + abs(beta) + alpha) / (2.0 * (c0 * gamma + abs(beta) - alpha))
    if as_printed:
        return mt1, mt0
    return min(1.0 / mu0, mt1), max(mu0, mt0)


def theorem23_printed_form_applies(amin: float, amax: float, alpha: float, beta: float) -> bool:
    """True when both numerator coefficients in the case-(ii) proof are
    positive, so that the printed mu0~ and mu1~ are the bounds."""
    gamma = math.sqrt(amin * amax)
    up = (1.0 / amax - 1.0 / gamma) * abs(beta) + (1.0 / amax + 1.0 / gamma) * abs(alpha)
    lo = (1.0 / gamma + 1.0 / amin) * abs(alpha) + (1.0 / gamma - 1.0 / amin) * abs(beta)
    return up > 0 and lo > 0


def theorem24_factor(amin: float, amax: float, c0: float, alpha: float, beta: float):
    iv = theorem23_interval(amin, amax, c0, alpha, beta)
    if iv is None:
        return None
    lo, hi = iv
    if alpha >= 0:
        mu0sq = hi * hi
        return (mu0sq - 1.0) / (mu0sq + 1.0)
    return (hi - lo) / (hi + lo)


# ---------------------------------------------------------------------------
# All-at-once time solve (Section 1: triangular time-discretisation matrices
# approximated by alpha-circulant ones, block-diagonalised into
# complex-shifted Laplacian systems).  Backward Euler for u' + K u = g on
# L steps of size tau:
#     (B kron I + I kron K) U = F,  B = (I - S)/tau  (S: ones on the subdiagonal),
#     F_0 = g_0 + u_0 / tau,  F_n = g_n  (n >= 1).
# alpha-circulant approximation: C_a = (I - S_a)/tau, S_a = S plus a at (0, L-1).
# With Gam = diag(a^{-j/L}) and the DFT matrix Fd[k, j] = exp(-2 pi i j k / L),
#     C_a = Gam Fd^{-1} diag(d_k) Fd Gam^{-1},  d_k = (1 - a^{1/L} exp(-2 pi i k/L)) / tau,
# so P_a = C_a kron I + I kron K is inverted by a scaled DFT in time, L
# shifted solves (d_k I + K) Z_k = R_k, and the inverse.
# ---------------------------------------------------------------------------
def paradiag_time_matrix(L: int, tau: float) -> np.ndarray:
    """B = (I - S)/tau, the backward-Euler time matrix (dense, L x L)."""
    return (np.eye(L) - np.eye(L, k=-1)) / tau


def paradiag_circulant(L: int, tau: float, a: float) -> np.ndarray:
    """C_a = (I - S_a)/tau: B with a in the top-right corner of the shift."""
    S = np.eye(L, k=-1)
    S[0, L - 1] = a
    return (np.eye(L) - S) / tau


def paradiag_shifts(L: int, tau: float, a: float) -> np.ndarray:
    """d_k = (1 - a^{1/L} exp(-2 pi i k/L)) / tau, the eigenvalues of C_a."""
    k = np.arange(L)
    return (1.0 - a ** (1.0 / L) * np.exp(-2j * np.pi * k / L)) / tau


def paradiag_apply(faces, tau: float, U: np.ndarray) -> np.ndarray:
    """(B kron I + I kron K) U for U of shape (L, *grid): time slices first."""
    out = np.empty_like(U, dtype=np.complex128)
    for n in range(U.shape[0]):
        out[n] = apply_K(faces, U[n]) + U[n] / tau
        if n > 0:
            out[n] -= U[n - 1] / tau
    return out


def paradiag_rhs(tau: float, u0: np.ndarray, g: np.ndarray) -> np.ndarray:
    F = np.array(g, dtype=np.complex128)
    F[0] = F[0] + u0 / tau
    return F


def paradiag_time_stepping(faces, tau: float, u0: np.ndarray, g: np.ndarray, tol: float = 1e-13,
                           maxit: int = 2000) -> np.ndarray:
    """The exact all-at-once solution by sequential backward Euler:
    (K + I/tau) u_n = g_n + u_{n-1}/tau, each step solved with `solve`."""
    U = np.empty(np.shape(g), dtype=np.complex128)
    prev = np.asarray(u0, dtype=np.complex128)
    for n in range(U.shape[0]):
        U[n], _ = solve(faces, 1.0 / tau, g[n] + prev / tau, tol, maxit)
        prev = U[n]
    return U


def paradiag_precond(faces, tau: float, a: float, R: np.ndarray, tol: float = 1e-12, maxit: int = 2000):
    """P_a^{-1} R: R_hat = Fd Gam^{-1} R (time slice j scaled by a^{j/L}, then
    the DFT over the slices), Z_k = (d_k I + K)^{-1} R_hat_k, Z = Gam Fd^{-1} Z_hat."""
    L = R.shape[0]
    j = np.arange(L).reshape((L,) + (1,) * (R.ndim - 1))
    Fd = np.exp(-2j * np.pi * np.outer(np.arange(L), np.arange(L)) / L)
    Rh = np.tensordot(Fd, (a ** (j / L)) * R, axes=(1, 0))
    d = paradiag_shifts(L, tau, a)
    Zh = np.empty_like(Rh)
    for k in range(L):
        Zh[k], _ = solve(faces, d[k], Rh[k], tol, maxit)
    Z = np.tensordot(np.conj(Fd) / L, Zh, axes=(1, 0))
    return (a ** (-j / L)) * Z


def paradiag_solve(faces, tau: float, a: float, u0: np.ndarray, g: np.ndarray, tol: float = 1e-10,
                   maxit: int = 20, inner_tol: float = 1e-12):
    """Preconditioned Richardson on the all-at-once system, U_0 = 0,
    U <- U + P_a^{-1}(F - A U), stopping when ||F - A U|| <= tol ||F||.
    Returns (U, list of relative residual norms before each update)."""
    F = paradiag_rhs(tau, u0, g)
    U = np.zeros_like(F)
    fn = np.linalg.norm(F)
    hist = []
    for _ in range(maxit + 1):
        R = F - paradiag_apply(faces, tau, U)
        hist.append(float(np.linalg.norm(R) / fn))
        if hist[-1] <= tol or len(hist) > maxit:
            break
        U = U + paradiag_precond(faces, tau, a, R, inner_tol)
    return U, hist


# ---------------------------------------------------------------------------
# Shifted-Laplace preconditioning of an outer Krylov solve (Section 1: the
# complex-shifted Laplacian "was initially introduced as a preconditioner"
# for Helmholtz problems).  Restarted flexible GMRES (right preconditioning)
# for (K + lam_A I) u = f, with z_j = M^{-1} v_j given by `solve` on
# (K + lam_M I) to a relative residual inner_tol.  Arnoldi with two passes of
# classical Gram-Schmidt; complex inner product <v, w> = sum conj(v) w.
# ---------------------------------------------------------------------------
def helmholtz_fgmres(faces, lam_A: complex, lam_M: complex, f: np.ndarray, tol: float = 1e-8,
                     maxit: int = 200, restart: int = 30, inner_tol: float = 1e-6, inner_maxit: int = 2000):
    """Returns (u, info dict: iters, relres history of the Arnoldi estimate,
    final true relres)."""
    f = np.asarray(f, dtype=np.complex128)
    fn = np.linalg.norm(f)
    x = np.zeros_like(f)
    A = lambda u: apply_K(faces, u) + lam_A * u
    iters = 0
    hist = []
    while True:
        r = f - A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * fn or iters >= maxit:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        jdone = 0
        for j in range(restart):
            z, _ = solve(faces, lam_M, V[j], inner_tol, inner_maxit)
            Z.append(z)
            w = A(z)
            for _pass in range(2):
                for i in range(j + 1):
                    hij = np.vdot(V[i], w)
                    H[i, j] += hij
                    w = w - hij * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
            # Givens rotations on the new column: with c = a/rho, s = b/rho,
            # (top, bottom) -> (conj(c) top + conj(s) bottom, -s top + c bottom)
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a_, b_ = H[j, j], H[j + 1, j]
            den = math.sqrt(abs(a_) ** 2 + abs(b_) ** 2)
            cs[j] = a_ / den if den != 0 else 1.0
            sn[j] = b_ / den if den != 0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            iters += 1
            jdone = j + 1
            hist.append(float(abs(g[j + 1]) / fn))
            if hist[-1] <= tol or iters >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:jdone, :jdone]), g[:jdone])
        for i in range(jdone):
            x = x + y[i] * Z[i]
    rel = float(np.linalg.norm(f - A(x)) / fn)
    return x, {"iters": iters, "hist": hist, "relres": rel}

