"""Orthonormal basis of symmetric traceless 3x3 tensors (oracle, test infrastructure).

The paper (Sec. 2.2.1, text after Fig. ptpsopt) states that the stresslet has 5
independent components but gives no basis.  Reading: the
orthonormal basis
    Y1 = (xx - yy)/sqrt2, Y2 = (xx + yy - 2zz)/sqrt6,
    Y3 = (xy + yx)/sqrt2, Y4 = (xz + zx)/sqrt2, Y5 = (yz + zy)/sqrt2,
so that S:E = sum_k s_k e_k and every block of the grand mobility is symmetric.
Torques and angular velocities (Sec. 2.2.1, rigid-particle relation) enter
through the antisymmetric part of the couplet and of the velocity gradient.
Reading (physical conventions): with D_ij = d_j u_i (the Faxen volume average
of Eq. fax2a) and the couplet C_mn as indexed in the mobility tensors M_UC,imn
and M_DC,ijmn (m the force component, n the moment arm), the angular velocity
is Omega = curl(u)/2, Omega_k = A_k : D, and a torque L adds sum_k L_k A_k to the
couplet, with the same basis A_k = -eps_k../2 on both sides, so that the
11-component grand mobility is symmetric.  A_k : A_l = delta_kl / 2.
Parity: pinned (tests check orthonormality, symmetry and tracelessness; the
torque basis through the free-space rotation mobilities).
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


_EPS = np.zeros((3, 3, 3))
_EPS[0, 1, 2] = _EPS[1, 2, 0] = _EPS[2, 0, 1] = 1.0
_EPS[0, 2, 1] = _EPS[2, 1, 0] = _EPS[1, 0, 2] = -1.0

A = -0.5 * _EPS                      # A[k, i, j] = -eps_kij / 2

# couplet / velocity-gradient basis of the 11-moment form: torque (3), stresslet (5)
G = np.concatenate([A, Y], axis=0)   # (8, 3, 3)
