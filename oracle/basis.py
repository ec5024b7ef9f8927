"""Orthonormal basis of symmetric traceless 3x3 tensors (oracle, test infrastructure).

The paper (Sec. 2.2.1, text after Fig. ptpsopt) states that the stresslet has 5
independent components but gives no basis.  Reading: the
orthonormal basis
    Y1 = (xx - yy)/sqrt2, Y2 = (xx + yy - 2zz)/sqrt6,
    Y3 = (xy + yx)/sqrt2, Y4 = (xz + zx)/sqrt2, Y5 = (yz + zy)/sqrt2,
so that S:E = sum_k s_k e_k and every block of the grand mobility is symmetric.
Parity: pinned (tests check orthonormality, symmetry and tracelessness).
"""
import numpy as np

_r2 = np.sqrt(2.0)
_r6 = np.sqrt(6.0)

Y = np.zeros((5, 3, 3))
Y[0, 0, 0], Y[0, 1, 1] = 1 / _r2, -1 / _r2
Y[1, 0, 0], Y[1, 1, 1], Y[1, 2, 2] = 1 / _r6, 1 / _r6, -2 / _r6
Y[2, 0, 1] = Y[2, 1, 0] = 1 / _r2
Y[3, 0, 2] = Y[3, 2, 0] = 1 / _r2
Y[4, 1, 2] = Y[4, 2, 1] = 1 / _r2


def to_tensor(s):
    """(..., 5) components -> (..., 3, 3) symmetric traceless tensor."""
    return np.einsum('...k,kij->...ij', s, Y)


def to_comp(T):
    """(..., 3, 3) tensor -> (..., 5) components T:Y_k."""
    return np.einsum('...ij,kij->...k', T, Y)
