"""Seeded synthetic inputs for the Wilson-clover multigrid solver.

This module only draws numbers: gauge links, right-hand sides, random test
vectors and gauge transformations.  It holds none of the solver's arithmetic
(no Dirac operator, no smoother, no transfer operator), so both the CPU
oracle and the CUDA library can be fed from it without sharing method code.

Layouts (all complex128, C-contiguous, so ``.view(np.float64)`` is the C-ABI
layout with interleaved re/im):

* gauge field ``U[t, z, y, x, mu, a, b]`` with ``mu`` = 0..3 = (t, z, y, x);
* fine spinor fields ``psi[n, t, z, y, x, 12]`` with index ``spin*3 + colour``;
* coarse fields ``phi[n, t, z, y, x, dof]``.

The gauge generator follows the recipe of the benchmark configurations: a
complex 3x3 matrix with independent N(0,1) real and imaginary parts, its
Hermitian traceless part H, U = exp(i*eps*H) (through a Hermitian
eigendecomposition), then re-unitarisation (Gram-Schmidt on rows 1 and 2,
row 3 = conj(row1 x row2)) so that det U = 1 to rounding.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "su3_field", "unit_gauge", "su3_matrices", "random_spinors", "random_fields",
    "point_sources", "random_test_vectors", "lattice_volume",
]


def lattice_volume(dims) -> int:
    T, Z, Y, X = dims
    return int(T) * int(Z) * int(Y) * int(X)


def su3_matrices(shape, eps: float, rng: np.random.Generator) -> np.ndarray:
    """Random SU(3) matrices exp(i*eps*H), re-unitarised; ``shape`` excludes (3, 3)."""
    full = tuple(shape) + (3, 3)
    a = rng.standard_normal(full) + 1j * rng.standard_normal(full)
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    w, v = np.linalg.eigh(h)
    u = np.einsum("...ik,...k,...jk->...ij", v, np.exp(1j * eps * w), np.conj(v))
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.ascontiguousarray(np.stack([r0, r1, r2], axis=-2))


def su3_field(dims, eps: float, seed: int) -> np.ndarray:
    """Gauge links U[t,z,y,x,mu,3,3] for a T x Z x Y x X lattice."""
    rng = np.random.default_rng(seed)
    return su3_matrices(tuple(dims) + (4,), eps, rng)


def unit_gauge(dims) -> np.ndarray:
    g = np.zeros(tuple(dims) + (4, 3, 3), dtype=np.complex128)
    g[..., 0, 0] = g[..., 1, 1] = g[..., 2, 2] = 1.0
    return g


def random_fields(n: int, dims, ndof: int, seed: int) -> np.ndarray:
    """n complex N(0,1) fields (independent real and imaginary parts) of ndof per site."""
    rng = np.random.default_rng(seed)
    shape = (n,) + tuple(dims) + (ndof,)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_spinors(n: int, dims, seed: int) -> np.ndarray:
    return random_fields(n, dims, 12, seed)


def point_sources(dims, seed: int) -> np.ndarray:
    """12 point sources delta_{x,x0} delta_{spin,s} delta_{colour,c} at a seeded site x0."""
    rng = np.random.default_rng(seed)
    x0 = tuple(int(rng.integers(0, d)) for d in dims)
    out = np.zeros((12,) + tuple(dims) + (12,), dtype=np.complex128)
    for k in range(12):
        out[(k,) + x0 + (k,)] = 1.0
    return out


def random_test_vectors(dims_per_level, n_tv, seed: int):
    """Random start vectors for the setup, one array per level.

    Level 0 gets ``n_tv[0]`` fine spinor fields.  A coarser level l >= 1 gets
    ``max(0, n_tv[l] - n_tv[l-1])`` fields of ``2*n_tv[l-1]`` degrees of freedom
    per site: those fill up the test vectors that restriction from the level
    above does not provide.  ``dims_per_level[l]`` are the lattice dimensions
    of level l.
    """
    out = []
    for lvl, dims in enumerate(dims_per_level[:len(n_tv)]):
        if lvl == 0:
            out.append(random_fields(n_tv[0], dims, 12, seed))
        else:
            extra = max(0, n_tv[lvl] - n_tv[lvl - 1])
            out.append(random_fields(extra, dims, 2 * n_tv[lvl - 1], seed + 7919 * lvl)
                       if extra else None)
    return out
