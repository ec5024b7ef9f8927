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

Parity: pinned (tests/test_oracle_params.py: Table tab:lmax P=5 at 1e-3, P=6 at
1e-4; eta < 1; the lambda_max closed forms).
"""
import math
from dataclasses import dataclass

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

    @property
    def V(self):
        return self.L ** 3

    @property
    def sigma(self):
        return self.h ** 3


def choose(N, L, a, eta, kT, xi, tol, Ng=None, P=None, rcut=None, rule='strict'):
    """All PSE parameters for a cubic periodic box of side L."""
    if rule == 'paper':
        rc_auto, P_auto = rcut_rule(xi, tol), support_rule(tol)
    elif rule == 'strict':
        rc_auto, P_auto = a + rcut_rule(xi, tol / 10.0), support_rule(tol / 10.0)
    else:
        raise ValueError(rule)
    rc = rc_auto if rcut is None else rcut
    kc = kcut_rule(xi, tol)
    PP = P_auto if P is None else int(P)
    m = math.sqrt(math.pi * PP)
    if Ng is None:
        Ng = next_grid(kc * L / math.pi)
        while True:
            h = L / Ng
            eg = (h * PP * xi / m) ** 2
            if eg < 1.0:
                break
            Ng = next_grid(Ng + 1)
    h = L / Ng
    eg = (h * PP * xi / m) ** 2
    if rc > 0.5 * L:
        raise ValueError('r_cut = %.4g exceeds L/2 = %.4g: the minimum-image pair sum '
                         'needs a larger box or a larger xi' % (rc, 0.5 * L))
    return Params(N=N, L=L, a=a, eta=eta, kT=kT, xi=xi, tol=tol, rcut=rc, kcut=kc,
                  P=PP, m=m, Ng=int(Ng), h=h, eta_g=eg)
