"""Dirac matrices in a chiral basis.

The paper fixes Gamma_5 as the identity on spins 1, 2 and minus the identity
on spins 3, 4 (Sec. 1).  A basis with that property is the chiral one:

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   (k = x, y, z)
    gamma_t = [[0, 1], [1, 0]]

These are Hermitian, satisfy {gamma_mu, gamma_nu} = 2 delta_{mu nu}, and
gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1).  The tests check all
three facts numerically.  Direction order is mu = 0..3 = (t, z, y, x).
"""
from __future__ import annotations

import numpy as np

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _gamma_space(k: int) -> np.ndarray:
    s = SIGMA[k]
    return np.block([[_Z2, -1j * s], [1j * s, _Z2]])


GAMMA_X = _gamma_space(0)
GAMMA_Y = _gamma_space(1)
GAMMA_Z = _gamma_space(2)
GAMMA_T = np.block([[_Z2, _I2], [_I2, _Z2]])

# indexed by mu = (t, z, y, x)
GAMMA = np.stack([GAMMA_T, GAMMA_Z, GAMMA_Y, GAMMA_X])
GAMMA5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128)
I4 = np.eye(4, dtype=np.complex128)
I3 = np.eye(3, dtype=np.complex128)


def spin_colour(S: np.ndarray, M: np.ndarray) -> np.ndarray:
    """S (x) M on the 12 spin-colour components, index spin*3 + colour."""
    return np.kron(S, M)


def gamma5_signs(ndof: int) -> np.ndarray:
    """Diagonal of Gamma_5 on a level with ndof degrees of freedom per site.

    On the fine level (12 dof) spins 0, 1 are +1 and spins 2, 3 are -1; on a
    coarse level with 2N dof the first N (chirality +) are +1 and the rest -1.
    In both cases this is: the first half +1, the second half -1.
    """
    s = np.ones(ndof)
    s[ndof // 2:] = -1.0
    return s
