"""Real-space split mobility M^(r) (oracle, test infrastructure only).

Definition followed: Sec. 2.2 states that the real-space functions are the
inverse Fourier transform of M - M^(w), i.e. of (1 - H(k, xi)) times the
Fourier-space pair mobilities (Eqs. MUF-MDC).  Written out in real space:

* Eq. hasimoto with (1 - H) gives the split Green's function
      J^(r)_im = (1/eta) [ delta_im phi0(r) + d_i d_m psi0(r) ],
  phi0 = FT^-1[(1-H)/k^2],  psi0 = FT^-1[(1-H)/k^4]  (so lap psi0 = -phi0).
* The shape factors of Eqs. MUF-MDC are Fourier transforms of normalised
  densities: sin(ka)/ka is the sphere shell (surface of radius a) and
  3 (sin ka - ka cos ka)/(ka)^3 is the ball of radius a.  Hence
      M_UF        = shell*shell * J^(r)
      M_UC_imn    = -d_n  [shell*ball * J^(r)]_im
      M_DF_ijm    = +d_j  [shell*ball * J^(r)]_im
      M_DC_ijmn   = -d_j d_n [ball*ball * J^(r)]_im
  (the i k_n factor of the couplet shape factor is a derivative, 3 s1 = FT(ball)).
* A 3D convolution of radial functions reduces to a 1D convolution of the
  profiles u(t) = t f(t):  r (kappa*f)(r) = int w_kappa(s) u(r - s) ds, with
  w_kappa an even piecewise polynomial on [-2a, 2a] (derived from the kernels,
  normalised to unit integral).

phi0 and psi0 are split into a free-space part (Oseen tensor) and an entire
remainder, so each 1D convolution is a piecewise-polynomial x smooth integral,
evaluated by Gauss-Legendre quadrature with breakpoints at every kink.
Derivatives of the radial functions are assembled into Cartesian tensors with
the chain rule in rho = r^2/2 and projected onto the stresslet basis Y.

Parity: pinned (tests/test_oracle_realspace.py) against the paper's printed
F1, F2 (App. A, both cases), K3, the self terms (Case 3 of App. A), the
textbook Faxen forms of the free-space mobility for r > 2a, the RPY overlap form,
brute-force radial Fourier quadrature of the definition for r < 2a and r > 2a,
and, through tests/test_oracle_ewald.py, xi-independence and positivity.
Pairs closer than about 0.2a lose digits to 1/r^7 cancellation (documented).
"""
import numpy as np
from scipy.special import erf

from .basis import G, Y

_C = 1.0 / (8.0 * np.pi)
_SQPI = np.sqrt(np.pi)
_NODES, _WEIGHTS = np.polynomial.legendre.leggauss(64)

KINDS = ('aa', 'ab', 'bb')   # shell*shell, shell*ball, ball*ball


# ---- 1D convolution kernels w_kappa(x) (even, support |x| <= 2a) --------------
def w_kernel(kind, x, a):
    ax = np.abs(x)
    if kind == 'aa':
        w = (2 * a - ax) / (4 * a * a)
    elif kind == 'ab':
        w = (4 * a ** 3 - 3 * a * ax * ax + ax ** 3) / (8 * a ** 4)
    else:
        w = 3.0 * (32 * a ** 5 - 40 * a ** 3 * ax ** 2 + 20 * a * a * ax ** 3 - ax ** 5) / (160 * a ** 6)
    return np.where(ax <= 2 * a, w, 0.0)


def w_kernel_d(kind, x, a, order):
    """order-th derivative of w_kappa at x > 0 (one-sided at the breakpoints)."""
    x = np.asarray(x, dtype=float)
    inside = x < 2 * a
    if kind == 'aa':
        d = {1: -np.ones_like(x) / (4 * a * a), 2: np.zeros_like(x)}[order]
    elif kind == 'ab':
        d = {1: (-6 * a * x + 3 * x * x) / (8 * a ** 4), 2: (-6 * a + 6 * x) / (8 * a ** 4)}[order]
    else:
        d = {1: 3.0 * (-80 * a ** 3 * x + 60 * a * a * x * x - 5 * x ** 4) / (160 * a ** 6),
             2: 3.0 * (-80 * a ** 3 + 120 * a * a * x - 20 * x ** 3) / (160 * a ** 6)}[order]
    return np.where(inside, d, 0.0)


# ---- profiles u(t) = t psi0(t) -------------------------------------------------
def u_psi_smooth(t, xi, n):
    """n-th derivative of the entire part of t*psi0(t)."""
    E = erf(xi * t)
    g = np.exp(-(xi * t) ** 2)
    if n == 0:
        return _C * (t * t * E + t * g / (xi * _SQPI))
    if n == 1:
        return _C * (2 * t * E + g / (xi * _SQPI))
    if n == 2:
        return _C * (2 * E + (2 * xi / _SQPI) * t * g)
    if n == 3:
        return _C * (2 * xi / _SQPI) * g * (3 - 2 * (xi * t) ** 2)
    if n == 4:
        return _C * (4 * xi ** 3 / _SQPI) * t * g * (2 * (xi * t) ** 2 - 5)
    if n == 5:
        return _C * (4 * xi ** 3 / _SQPI) * g * (-4 * (xi * t) ** 4 + 16 * (xi * t) ** 2 - 5)
    raise ValueError(n)


def u_psi_free(t, n):
    """Regular part of the n-th derivative of the free-space profile -t|t|/(8 pi)."""
    if n == 0:
        return -_C * t * np.abs(t)
    if n == 1:
        return -2 * _C * np.abs(t)
    if n == 2:
        return -2 * _C * np.sign(t)
    return np.zeros_like(t)   # n >= 3: point masses, handled in conv_U


def conv_U(kind, r, xi, a, n, free_only=False):
    """U^(n)(r) = int w_kappa(s) u^(n)(r - s) ds for r >= 0 (vectorised over r).

    u = u_free + u_smooth; the free part has point masses for n >= 3:
    u''' = -4C delta, u'''' = -4C delta', u''''' = -4C delta''.
    """
    r = np.atleast_1d(np.asarray(r, dtype=float))
    rb = np.minimum(r, 2 * a)
    pieces = [(np.full_like(r, -2 * a), np.zeros_like(r)), (np.zeros_like(r), rb),
              (rb, np.full_like(r, 2 * a))]
    total = np.zeros_like(r)
    for lo, hi in pieces:
        half = 0.5 * (hi - lo)
        mid = 0.5 * (hi + lo)
        s = mid[:, None] + half[:, None] * _NODES[None, :]
        t = r[:, None] - s
        f = u_psi_free(t, n) if n <= 2 else 0.0
        if not free_only:
            f = f + u_psi_smooth(t, xi, n)
        total += half * np.sum(_WEIGHTS[None, :] * w_kernel(kind, s, a) * f, axis=1)
    if n == 3:
        total += -4 * _C * w_kernel(kind, r, a)
    elif n == 4:
        total += -4 * _C * w_kernel_d(kind, r, a, 1)
    elif n == 5:
        total += -4 * _C * w_kernel_d(kind, r, a, 2)
    return total


def radial_derivs(kind, r, xi, a, free_only=False):
    """Phi, Phi', Phi'' and Psi', ..., Psi'''' for kernel kind at r > 0."""
    U = [conv_U(kind, r, xi, a, n, free_only) for n in range(5)]
    r = np.atleast_1d(np.asarray(r, dtype=float))
    # Psi = U/r
    p1 = U[1] / r - U[0] / r ** 2
    p2 = U[2] / r - 2 * U[1] / r ** 2 + 2 * U[0] / r ** 3
    p3 = U[3] / r - 3 * U[2] / r ** 2 + 6 * U[1] / r ** 3 - 6 * U[0] / r ** 4
    p4 = U[4] / r - 4 * U[3] / r ** 2 + 12 * U[2] / r ** 3 - 24 * U[1] / r ** 4 + 24 * U[0] / r ** 5
    # Phi = V/r with V = r Phi = -U''  (lap psi0 = -phi0)
    V0, V1, V2 = -U[2], -U[3], -U[4]
    f0 = V0 / r
    f1 = V1 / r - V0 / r ** 2
    f2 = V2 / r - 2 * V1 / r ** 2 + 2 * V0 / r ** 3
    return (f0, f1, f2), (p1, p2, p3, p4)


def _rho_derivs(f1, f2, f3, f4, r):
    """D_n = ((1/r) d/dr)^n f from ordinary r-derivatives (D3, D4 may be None)."""
    D1 = f1 / r
    D2 = f2 / r ** 2 - f1 / r ** 3
    D3 = None if f3 is None else f3 / r ** 3 - 3 * f2 / r ** 4 + 3 * f1 / r ** 5
    D4 = None if f4 is None else (f4 / r ** 4 - 6 * f3 / r ** 5 + 15 * f2 / r ** 6 - 15 * f1 / r ** 7)
    return D1, D2, D3, D4


_I = np.eye(3)


def _grad2(D1, D2, x):
    return D2[:, None, None] * np.einsum('pi,pj->pij', x, x) + D1[:, None, None] * _I


def _grad3(D2, D3, x):
    xxx = np.einsum('pi,pj,pk->pijk', x, x, x)
    dx = (np.einsum('ij,pk->pijk', _I, x) + np.einsum('ik,pj->pijk', _I, x)
          + np.einsum('jk,pi->pijk', _I, x))
    return D3[:, None, None, None] * xxx + D2[:, None, None, None] * dx


def _grad4(D2, D3, D4, x):
    x4 = np.einsum('pi,pj,pk,pl->pijkl', x, x, x, x)
    dxx = (np.einsum('ij,pk,pl->pijkl', _I, x, x) + np.einsum('ik,pj,pl->pijkl', _I, x, x)
           + np.einsum('il,pj,pk->pijkl', _I, x, x) + np.einsum('jk,pi,pl->pijkl', _I, x, x)
           + np.einsum('jl,pi,pk->pijkl', _I, x, x) + np.einsum('kl,pi,pj->pijkl', _I, x, x))
    dd = (np.einsum('ij,kl->ijkl', _I, _I) + np.einsum('ik,jl->ijkl', _I, _I)
          + np.einsum('il,jk->ijkl', _I, _I))
    return (D4[:, None, None, None, None] * x4 + D3[:, None, None, None, None] * dxx
            + D2[:, None, None, None, None] * dd[None])


def cartesian_blocks(x, xi, a, eta, free_only=False):
    """Full Cartesian real-space pair tensors for separation vectors x (p, 3), |x| > 0.

    x = x_alpha - x_beta; the blocks give the response of alpha to moments of beta.
    Returns M_UF (p,3,3), M_UC (p,3,3,3)[i,m,n], M_DF (p,3,3,3)[i,j,m], M_DC (p,3,3,3,3)[i,j,m,n].
    """
    x = np.atleast_2d(np.asarray(x, dtype=float))
    r = np.linalg.norm(x, axis=1)
    out = {}
    for kind in KINDS:
        (f0, f1, f2), (p1, p2, p3, p4) = radial_derivs(kind, r, xi, a, free_only)
        out[kind] = (f0, f1, f2, p1, p2, p3, p4)
    # T_im = (1/eta)[delta_im Phi + d_i d_m Psi]
    f0, f1, f2, p1, p2, p3, p4 = out['aa']
    P1, P2, _, _ = _rho_derivs(p1, p2, None, None, r)
    M_UF = (f0[:, None, None] * _I + _grad2(P1, P2, x)) / eta
    # d_j T_im = (1/eta)[delta_im d_j Phi + d_i d_j d_m Psi]
    f0, f1, f2, p1, p2, p3, p4 = out['ab']
    F1, _, _, _ = _rho_derivs(f1, f2, None, None, r)
    P1, P2, P3, _ = _rho_derivs(p1, p2, p3, None, r)
    gradPhi = F1[:, None] * x                                     # (p, j)
    dT = (np.einsum('im,pj->pijm', _I, gradPhi) + _grad3(P2, P3, x)) / eta   # [i, j, m]
    M_DF = dT                                                     # [i, j, m]
    M_UC = -np.einsum('pinm->pimn', dT)                           # -d_n T_im -> [i, m, n]
    # d_j d_n T_im = (1/eta)[delta_im d_j d_n Phi + d_i d_j d_m d_n Psi]
    f0, f1, f2, p1, p2, p3, p4 = out['bb']
    F1, F2, _, _ = _rho_derivs(f1, f2, None, None, r)
    P1, P2, P3, P4 = _rho_derivs(p1, p2, p3, p4, r)
    hPhi = _grad2(F1, F2, x)                                      # (p, j, n)
    ddT = (np.einsum('im,pjn->pijmn', _I, hPhi) + _grad4(P2, P3, P4, x)) / eta  # [i,j,m,n]
    M_DC = -ddT
    return M_UF, M_UC, M_DF, M_DC


def pair_blocks(x, xi, a, eta, free_only=False):
    """8x8 real-space blocks [[UF, US], [EF, ES]] in the Y basis for separations x (p,3)."""
    M_UF, M_UC, M_DF, M_DC = cartesian_blocks(x, xi, a, eta, free_only)
    p = M_UF.shape[0]
    B = np.zeros((p, 8, 8))
    B[:, :3, :3] = M_UF
    B[:, :3, 3:] = np.einsum('pimn,lmn->pil', M_UC, Y)
    B[:, 3:, :3] = np.einsum('kij,pijm->pkm', Y, M_DF)
    B[:, 3:, 3:] = np.einsum('kij,pijmn,lmn->pkl', Y, M_DC, Y)
    return B


def self_block(xi, a, eta, free_only=False):
    """Real-space self mobility (r -> 0 limit; App. A Case 3) as an 8x8 block.

    UF: (2/3) Phi_aa(0)/eta I with Phi(0) = V'(0) = -U'''(0).
    ES: U_bb^(5)(0)/(5 eta) I_5  (from d_j d_n of a smooth radial tensor at 0).
    UC/DF vanish by parity.
    """
    z = np.zeros(1)
    phi_aa0 = -conv_U('aa', z, xi, a, 3, free_only)[0]
    u5_bb = conv_U('bb', z, xi, a, 5, free_only)[0]
    B = np.zeros((8, 8))
    B[:3, :3] = (2.0 / 3.0) * phi_aa0 / eta * np.eye(3)
    B[3:, 3:] = u5_bb / (5.0 * eta) * np.eye(5)
    return B


def pair_blocks11(x, xi, a, eta, free_only=False):
    """11x11 real-space blocks [[UF, UL, US], [OF, OL, OS], [EF, EL, ES]] for separations x (p, 3):
    the couplet / gradient basis G = [A (torque, rotation), Y (stresslet, strain)] (Sec. 2.2.1)."""
    M_UF, M_UC, M_DF, M_DC = cartesian_blocks(x, xi, a, eta, free_only)
    p = M_UF.shape[0]
    B = np.zeros((p, 11, 11))
    B[:, :3, :3] = M_UF
    B[:, :3, 3:] = np.einsum('pimn,lmn->pil', M_UC, G)
    B[:, 3:, :3] = np.einsum('kij,pijm->pkm', G, M_DF)
    B[:, 3:, 3:] = np.einsum('kij,pijmn,lmn->pkl', G, M_DC, G)
    return B


def self_block11(xi, a, eta, free_only=False):
    """11x11 real-space self mobility: UF as self_block, rotation-torque U_bb^(5)(0)/(6 eta) I_3
    (from the isotropic r -> 0 limit of M_DC on antisymmetric couplets: D = -Phi''(0)/eta C,
    Phi''(0) = -U_bb^(5)(0)/3, Omega = A : D), strain-stresslet U_bb^(5)(0)/(5 eta) I_5."""
    z = np.zeros(1)
    phi_aa0 = -conv_U('aa', z, xi, a, 3, free_only)[0]
    u5_bb = conv_U('bb', z, xi, a, 5, free_only)[0]
    B = np.zeros((11, 11))
    B[:3, :3] = (2.0 / 3.0) * phi_aa0 / eta * np.eye(3)
    B[3:6, 3:6] = u5_bb / (6.0 * eta) * np.eye(3)
    B[6:, 6:] = u5_bb / (5.0 * eta) * np.eye(5)
    return B
