"""Parameter selection for PSE (oracle, test infrastructure only).

Follows
* Sec. 2.3.1: real-space error eps_r ~ exp(-xi^2 r_cut^2)  ->  r_cut = sqrt(ln(1/eps))/xi.
* Eq. (bound) with lambda_max = 1 and the rule m = sqrt(pi P) stated after Table
  (tab:lmax): eps_q <= exp(-pi P / 2) + erfc(sqrt(pi P / 2)); P is the smallest
  integer meeting the tolerance (C = 1 reading).
* eta = (h P xi / m)^2 (text before Eq. bound), Gaussian kernel
  K(r) = (2 xi^2/(pi eta))^{3/2} exp(-2 xi^2 r^2 / eta).
* Readings where the paper is silent: k_cut from
  H(k_cut, xi) <= eps with H the Hasimoto splitting function; N_g the smallest
  even 2,3,5,7-smooth integer >= k_cut L / pi; the grid is refined until eta < 1.
* Error budget.  With the bounds taken literally (C = 1, rule='paper') the
  measured relative error against the dense Ewald sum is 2-9 x eps, because
  the bounds carry unknown O(1) constants and the real-space functions decay
  like exp(-xi^2 (r - 2a)^2) near the cutoff (App. A erfc((r-2a)xi) terms).
  The default rule='strict' therefore takes r_cut = a + sqrt(ln(10/eps))/xi and
  P from the bound at eps/10, which keeps the measured error below eps for
  xi a in [0.45, 0.8] at phi = 0.1 and 0.3.

* Deformed lattices (Sec. 2.3.3): the periodic cell is spanned by the columns of
  L A; grid nodes sit at h A n and the support is the P^3 nodes nearest the
  particle in lattice coordinates z = A^{-1} x.  The support rule takes
  Eq. (bound) with lambda_max, the largest eigenvalue of A^T A (lambda_aware,
  default), or with lambda_max = 1 (the orthorhombic rule the paper compares
  against in Fig. fig:shear).  Readings where the paper is silent: the grid
  must hold every wave vector with |k| <= k_cut, k = (2 pi/L) A^{-T} m with
  |m_i| < Ng/2, so Ng >= k_cut L max_i |A e_i| / pi; the real-space sum needs
  r_cut <= L sqrt(lambda_min)/2 (the smallest half-width of the cell), so that a
  pair closer than r_cut has one image only; V = L^3 det A and sigma = h^3 det A.

Parity: pinned (tests/test_oracle_params.py: Table tab:lmax P=5 at 1e-3, P=6 at
1e-4; eta < 1; the lambda_max closed forms; tests/test_oracle_lattice.py: the
lattice metrics against the closed forms of Eqs. lmax1 and lmax2).
"""
import math
from dataclasses import dataclass

import numpy as np

from scipy.special import erfc
from scipy.optimize import brentq


def rcut_rule(xi, tol):
    """Real-space cutoff from exp(-xi^2 r_cut^2) = tol (Sec. 2.3.1)."""
    return math.sqrt(math.log(1.0 / tol)) / xi


def hasimoto_H(k, xi):
    """Hasimoto splitting function H(k, xi) = (1 + k^2/4xi^2) exp(-k^2/4xi^2)."""
    u = k * k / (4.0 * xi * xi)
    return (1.0 + u) * math.exp(-u)


def kcut_rule(xi, tol):
    """Smallest k with H(k, xi) <= tol (reading: wave-space truncation)."""
    # H is decreasing in u = k^2/(4 xi^2); solve (1+u) e^-u = tol.
    f = lambda u: (1.0 + u) * math.exp(-u) - tol
    u = brentq(f, 1e-12, 800.0, xtol=1e-14)
    return 2.0 * xi * math.sqrt(u)


def quadrature_bound(P, lam=1.0):
    """Right-hand side of Eq. (bound) with C = 1 and m = sqrt(pi P)."""
    m = math.sqrt(math.pi * P)
    return math.exp(-math.pi ** 2 * P * P / (2.0 * m * m * lam)) + erfc(m / math.sqrt(2.0 * lam))


def support_rule(tol, lam=1.0):
    """Smallest support size P with quadrature_bound(P, lam) <= tol."""
    P = 1
    while quadrature_bound(P, lam) > tol:
        P += 1
    return P


def lambda_max_shear(gamma):
    """Maximum eigenvalue of A^T A for simple shear (Eq. lmax1)."""
    return 1.0 + gamma * gamma / 2.0 + gamma * math.sqrt(1.0 + gamma * gamma / 4.0)


def lambda_max_ext(eps):
    """Maximum eigenvalue of A^T A for planar extension (Eq. lmax2)."""
    return eps * eps if eps >= 1.0 else 1.0 / (eps * eps)


def shear_tensor(gamma):
    """Deformation tensor of simple shear with strain gamma (Sec. 2.3.3)."""
    return np.array([[1.0, gamma, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def extension_tensor(eps):
    """Deformation tensor of planar extension with stretch eps (Sec. 2.3.3)."""
    return np.diag([eps, 1.0 / eps, 1.0])


def lattice_metrics(A):
    """(lambda_min, lambda_max) of A^T A, det A and the largest column norm of A."""
    A = np.asarray(A, dtype=float)
    ev = np.linalg.eigvalsh(A.T @ A)
    return float(ev[0]), float(ev[-1]), float(np.linalg.det(A)), float(np.max(np.linalg.norm(A, axis=0)))


def _smooth(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def next_grid(n):
    """Smallest even 2,3,5,7-smooth integer >= n."""
    n = max(int(math.ceil(n)), 2)
    while n % 2 or not _smooth(n):
        n += 1
    return n


@dataclass
class Params:
    N: int
    L: float
    a: float
    eta: float      # fluid viscosity
    kT: float
    xi: float
    tol: float
    rcut: float
    kcut: float
    P: int
    m: float
    Ng: int
    h: float
    eta_g: float    # Gaussian width parameter of the spreading kernel
    A: object = None    # lattice deformation (3 x 3), None for the cubic box
    detA: float = 1.0

    @property
    def V(self):
        return self.L ** 3 * self.detA

    @property
    def sigma(self):
        return self.h ** 3 * self.detA


def choose(N, L, a, eta, kT, xi, tol, Ng=None, P=None, rcut=None, rule='strict', A=None,
           lambda_aware=True):
    """All PSE parameters for a periodic box of side L, cubic (A None) or the
    lattice spanned by the columns of L A."""
    lam_min, lam, detA, cmax = 1.0, 1.0, 1.0, 1.0
    if A is not None:
        A = np.array(A, dtype=float).reshape(3, 3)
        lam_min, lam, detA, cmax = lattice_metrics(A)
        if not detA > 0:
            raise ValueError('the lattice deformation needs det A > 0')
    lam_P = lam if lambda_aware else 1.0
    if rule == 'paper':
        rc_auto, P_auto = rcut_rule(xi, tol), support_rule(tol, lam_P)
    elif rule == 'strict':
        rc_auto, P_auto = a + rcut_rule(xi, tol / 10.0), support_rule(tol / 10.0, lam_P)
    else:
        raise ValueError(rule)
    rc = rc_auto if rcut is None else rcut
    kc = kcut_rule(xi, tol)
    PP = P_auto if P is None else int(P)
    m = math.sqrt(math.pi * PP)
    if Ng is None:
        Ng = next_grid(kc * L * cmax / math.pi)
        while True:
            h = L / Ng
            eg = (h * PP * xi / m) ** 2
            if eg < 1.0:
                break
            Ng = next_grid(Ng + 1)
    h = L / Ng
    eg = (h * PP * xi / m) ** 2
    half = 0.5 * L * math.sqrt(lam_min)
    if rc > half * (1 + 1e-12):
        raise ValueError('r_cut = %.4g exceeds the half-width %.4g of the cell: the minimum-image pair sum '
                         'needs a larger box or a larger xi' % (rc, half))
    return Params(N=N, L=L, a=a, eta=eta, kT=kT, xi=xi, tol=tol, rcut=rc, kcut=kc,
                  P=PP, m=m, Ng=int(Ng), h=h, eta_g=eg, A=A, detA=detA)
