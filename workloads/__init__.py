"""Seeded synthetic inputs for the complex-shifted Laplacian solve.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It holds no arithmetic of the method (no stencil, no sine
transform, no Krylov step): it only samples the coefficient functions of the
paper's problem class (Eq. 1: a(x) on the unit square/cube) at face midpoints,
draws right-hand sides, and produces the shifts that an alpha-circulant time
discretisation hands to the spatial solver (Section 1).

Conventions (used by both sides):
  * grid: unit square/cube, homogeneous Dirichlet boundary, n interior points
    per axis, h = 1/(n+1); vectors are C-order arrays of shape (n,)*dim with x
    the fastest (last) axis, point (i_x, i_y[, i_z]) at ((i_x+1)h, (i_y+1)h, ...).
  * coefficient samples: one array per spatial axis, ordered (x, y[, z]).
    The x-face array has n+1 entries along the x axis and n along the others;
    entry i along its own axis is the face between grid indices i-1 and i, at
    coordinate (i + 1/2) h.  Same for y and z.
  * random draws: numpy.random.default_rng(seed) (PCG64); complex arrays draw
    the real part (all M values, C-order) first, then the imaginary part.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence, Tuple

import numpy as np

AXES = ("x", "y", "z")


def grid_h(n: int) -> float:
    return 1.0 / (n + 1)


def axis_sizes(dim: int, n) -> Tuple[int, ...]:
    """Points per spatial axis (x, y[, z]): n is one int (square / cube grid)
    or a sequence (nx, ny[, nz]) for a rectangular grid."""
    if isinstance(n, (int, np.integer)):
        return (int(n),) * dim
    t = tuple(int(v) for v in n)
    assert len(t) == dim
    return t


def face_coordinates(dim: int, n, axis: int):
    """Coordinates of the face midpoints normal to spatial axis `axis`
    (0 = x, 1 = y, 2 = z) as a list of broadcastable arrays ordered (x, y, z),
    each shaped like the face array (C-order, x fastest).  Axis a has
    n_a points and spacing h_a = 1/(n_a + 1)."""
    ns = axis_sizes(dim, n)
    coords = []
    for a in range(dim):
        h = grid_h(ns[a])
        if a == axis:
            c = (np.arange(ns[a] + 1, dtype=np.float64) + 0.5) * h
        else:
            c = (np.arange(ns[a], dtype=np.float64) + 1.0) * h
        shape = [1] * dim
        shape[dim - 1 - a] = c.size  # spatial axis a is numpy axis dim-1-a
        coords.append(c.reshape(shape))
    return coords


def grid_array_shape(dim: int, n) -> Tuple[int, ...]:
    """numpy shape of a grid vector: (ny, nx) or (nz, ny, nx)."""
    return tuple(reversed(axis_sizes(dim, n)))


def sample_faces(dim: int, n, coef: Callable[..., np.ndarray]):
    """Sample a(x[, y[, z]]) at every face midpoint; returns a tuple of
    float64 C-contiguous arrays ordered (x-faces, y-faces[, z-faces]).  n is
    one int or the per-axis sizes (nx, ny[, nz])."""
    ns = axis_sizes(dim, n)
    out = []
    for axis in range(dim):
        c = face_coordinates(dim, ns, axis)
        shape = list(reversed(ns))
        shape[dim - 1 - axis] += 1
        vals = np.broadcast_to(np.asarray(coef(*c), dtype=np.float64), shape)
        out.append(np.ascontiguousarray(vals))
    return tuple(out)


# --- coefficient functions of the workloads -------------------------------
def coef_const(value: float = 1.0):
    return lambda *c: np.full(np.broadcast_shapes(*[x.shape for x in c]), value)


def coef_c0(x, y):  # 1 + 0.5 sin(pi x) sin(pi y)
    return 1.0 + 0.5 * np.sin(np.pi * x) * np.sin(np.pi * y)


def coef_c1(x, y):  # exp(ln(10) x y): contrast 10
    return np.exp(math.log(10.0) * x * y)


def coef_c2(x, y, z):  # 1 + 0.9 sin(2 pi x) sin(2 pi y) sin(2 pi z)
    return 1.0 + 0.9 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)


def coef_table2(x, y):  # (20 + x^2)(20 + y^2), Example 2 of the paper
    return (20.0 + x * x) * (20.0 + y * y)


def smoothed_field_faces(n: int, seed: int = 4, passes: int = 8):
    """Face samples of a = 1 + 0.5*s, s a smoothed i.i.d. uniform field on the
    (n+2)^2 node grid (3x3 box filter, edge replication, `passes` times,
    min-max rescaled to [0, 1]); a face takes the mean of its two nodes."""
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.0, 1.0, size=(n + 2, n + 2))
    for _ in range(passes):
        p = np.pad(s, 1, mode="edge")
        acc = np.zeros_like(s)
        for dy in range(3):
            for dx in range(3):
                acc += p[dy:dy + n + 2, dx:dx + n + 2]
        s = acc / 9.0
    s = (s - s.min()) / (s.max() - s.min())
    node = 1.0 + 0.5 * s  # node (iy, ix) at (ix h, iy h), ix, iy = 0..n+1
    ax = 0.5 * (node[1:n + 1, 0:n + 1] + node[1:n + 1, 1:n + 2])  # (n, n+1)
    ay = 0.5 * (node[0:n + 1, 1:n + 1] + node[1:n + 2, 1:n + 1])  # (n+1, n)
    return (np.ascontiguousarray(ax), np.ascontiguousarray(ay))


# --- right-hand sides ------------------------------------------------------
def rhs_uniform(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    m = int(np.prod(shape))
    re = rng.uniform(-1.0, 1.0, size=m)
    im = rng.uniform(-1.0, 1.0, size=m)
    return (re + 1j * im).reshape(shape)


def rhs_normal(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    m = int(np.prod(shape))
    re = rng.standard_normal(m)
    im = rng.standard_normal(m)
    return (re + 1j * im).reshape(shape)


def alpha_circulant_shifts(L: int = 64, eps: float = 1e-4) -> np.ndarray:
    """lambda_k = (1 - eps^(1/L) exp(2 pi i k / L)) * L, k = 0..L-1: the
    eigenvalues an alpha-circulant (alpha = eps) backward-Euler time block
    with step 1/L hands to the spatial solves."""
    k = np.arange(L)
    return (1.0 - eps ** (1.0 / L) * np.exp(2j * np.pi * k / L)) * L


# --- the workload configurations -----------------------------------------
@dataclass
class System:
    dim: int
    n: int
    faces: tuple
    lam: complex
    f: np.ndarray

    @property
    def h(self) -> float:
        return grid_h(self.n)

    @property
    def M(self) -> int:
        return self.n ** self.dim


def config0() -> System:
    """2D n=63, a = 1 + 0.5 sin(pi x) sin(pi y), lambda = 1+10i, f ~ U[-1,1]^2, seed 0."""
    n = 63
    return System(2, n, sample_faces(2, n, coef_c0), 1 + 10j, rhs_uniform((n, n), 0))


def config1(n: int = 1023) -> System:
    """2D n=1023, a = exp(ln10 x y), lambda = 100i, f ~ U[-1,1]^2, seed 1."""
    return System(2, n, sample_faces(2, n, coef_c1), 100j, rhs_uniform((n, n), 1))


def config2(n: int = 127) -> System:
    """3D n=127, a = 1 + 0.9 sin(2 pi x) sin(2 pi y) sin(2 pi z), lambda = -5+50i,
    f standard normal complex, seed 2."""
    return System(3, n, sample_faces(3, n, coef_c2), -5 + 50j, rhs_normal((n, n, n), 2))


def config3(ns: Sequence[int] = (127, 255, 511), L: int = 64, eps: float = 1e-4):
    """Batched shifts: for each n (ascending) and k = 0..L-1 (ascending), the
    system with a as in config0, lambda_k from `alpha_circulant_shifts`, and
    f ~ U[-1,1]^2 drawn from ONE generator seeded 3 in that order."""
    rng = np.random.default_rng(3)
    lams = alpha_circulant_shifts(L, eps)
    out = []
    for n in sorted(ns):
        faces = sample_faces(2, n, coef_c0)
        for k in range(L):
            m = n * n
            re = rng.uniform(-1.0, 1.0, size=m)
            im = rng.uniform(-1.0, 1.0, size=m)
            out.append(System(2, n, faces, complex(lams[k]), (re + 1j * im).reshape(n, n)))
    return out


def config4(n: int = 511):
    """Adjoint workload: 2D n=511, smoothed random coefficient (seed 4),
    lambda = 1+20i, f ~ U[-1,1]^2 (seed 4 stream is the coefficient; f uses
    seed 40), data d ~ N(0,1) (seed 5) for the loss 0.5*||Re z - d||^2."""
    faces = smoothed_field_faces(n, seed=4)
    f = rhs_uniform((n, n), 40)
    d = np.random.default_rng(5).standard_normal((n, n))
    return System(2, n, faces, 1 + 20j, f), d


def fd_directions(count: int, sizes: Sequence[int], seed: int = 6, normalise: bool = False):
    """`count` random directions over the concatenation of arrays of the given
    sizes: i.i.d. standard normal entries, so that a step h moves every entry
    by about h.  With normalise=True each direction has unit 2-norm instead."""
    rng = np.random.default_rng(seed)
    tot = int(sum(sizes))
    out = []
    for _ in range(count):
        d = rng.standard_normal(tot)
        out.append(d / np.linalg.norm(d) if normalise else d)
    return out


TABLE1_SHIFTS = [(100, 100), (-100, -100), (100, -100), (-100, 100), (-100, 1), (1, -100)]
TABLE2_SHIFTS = [(-600, 150), (-100, -25), (100, -100), (-100, 100), (-100, 1), (1, -100)]
