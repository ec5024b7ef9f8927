"""Pins for oracle.realspace (real-space split mobility, Eqs. MUFr-MDCr, App. A).

* F1, F2 (both cases), K3 (both cases) and the two self terms are typed from the
  paper's Appendix A and compared with the oracle's convolution evaluation.
* The xi -> 0 (free-space) part is compared with the textbook Faxen forms
  (1 + a^2/3 lap) J, -d_n (1 + 4a^2/15 lap) J, -d_j d_n (1 + a^2/5 lap) J of the
  Oseen tensor J for r > 2a, and with the Rotne-Prager overlap form for r < 2a.
* The radial profiles are compared with brute-force quadrature of the
  definition (inverse Fourier transform of (1 - H) times the shape factors).
"""
import math

import numpy as np
import pytest
from scipy.special import erfc

from oracle import realspace as R
from oracle.basis import Y

SP = math.sqrt(math.pi)
I3 = np.eye(3)


def F_printed(r, xi, a, case2):
    """App. A: 6 pi eta a M_UF = F1 (I - rr) + F2 rr (both cases typed from the paper)."""
    e = lambda d: math.exp(-d * d * xi * xi)
    x = xi
    f1 = [0, (18 * r ** 2 * x ** 2 + 3) / (64 * SP * a * r ** 2 * x ** 3),
          (2 * x ** 2 * (2 * a - r) * (4 * a * a + 4 * a * r + 9 * r * r) - 2 * a - 3 * r) / (128 * SP * a * r ** 3 * x ** 3),
          (-2 * x ** 2 * (2 * a + r) * (4 * a * a - 4 * a * r + 9 * r * r) + 2 * a - 3 * r) / (128 * SP * a * r ** 3 * x ** 3),
          (3 - 36 * r ** 4 * x ** 4) / (128 * a * r ** 3 * x ** 4),
          (4 * x ** 4 * (r - 2 * a) ** 2 * (4 * a * a + 4 * a * r + 9 * r * r) - 3) / (256 * a * r ** 3 * x ** 4),
          (4 * x ** 4 * (2 * a + r) ** 2 * (4 * a * a - 4 * a * r + 9 * r * r) - 3) / (256 * a * r ** 3 * x ** 4)]
    f2 = [0, (6 * r * r * x * x - 3) / (32 * SP * a * r * r * x ** 3),
          (-2 * x ** 2 * (r - 2 * a) ** 2 * (2 * a + 3 * r) + 2 * a + 3 * r) / (64 * SP * a * r ** 3 * x ** 3),
          (2 * x ** 2 * (2 * a + r) ** 2 * (2 * a - 3 * r) - 2 * a + 3 * r) / (64 * SP * a * r ** 3 * x ** 3),
          -3 * (4 * r ** 4 * x ** 4 + 1) / (64 * a * r ** 3 * x ** 4),
          (3 - 4 * x ** 4 * (2 * a - r) ** 3 * (2 * a + 3 * r)) / (128 * a * r ** 3 * x ** 4),
          (3 - 4 * x ** 4 * (2 * a - 3 * r) * (2 * a + r) ** 3) / (128 * a * r ** 3 * x ** 4)]
    if case2:
        f1[0] = -(r - 2 * a) ** 2 * (4 * a * a + 4 * a * r + 9 * r * r) / (32 * a * r ** 3)
        f2[0] = (2 * a - r) ** 3 * (2 * a + 3 * r) / (16 * a * r ** 3)
    b = [1, e(r), e(r - 2 * a), e(r + 2 * a), erfc(r * x), erfc((r - 2 * a) * x), erfc((r + 2 * a) * x)]
    return sum(c * v for c, v in zip(f1, b)), sum(c * v for c, v in zip(f2, b))


def K3_printed(r, xi, a, case2):
    """App. A, third scalar function of 6 pi eta a M_DC (both cases typed from the paper)."""
    x = xi
    e = lambda d: math.exp(-d * d * x * x)
    k56 = 9 * (16 * x ** 8 * (r * r - 4 * a * a) ** 3 * (4 * a * a + r * r) + 24 * r * r * x ** 4 * (12 * a * a + r * r)
               - 48 * x * x * (10 * a * a + r * r) + 45) / (16384 * a ** 6 * r ** 5 * x ** 8)
    k = [0,
         9 * (32 * a * a * x * x * (-2 * r ** 4 * x ** 4 + r * r * x * x + 15) + 8 * r ** 6 * x ** 6 - 4 * r ** 4 * x ** 4
              + 18 * r * r * x * x - 45) / (4096 * SP * a ** 6 * r ** 4 * x ** 7),
         9 * (-8 * x ** 6 * (r - 2 * a) ** 2 * (2 * a + r) ** 3 * (4 * a * a + r * r) + 4 * x ** 4 * (2 * a + r) ** 3
              * (4 * a * a + r * r) - 6 * x * x * (2 * a + r) ** 2 * (2 * a + 3 * r) + 45 * (r - 2 * a))
         / (8192 * SP * a ** 6 * r ** 5 * x ** 7),
         9 * (-8 * x ** 6 * (r - 2 * a) ** 3 * (2 * a + r) ** 2 * (4 * a * a + r * r) + 4 * x ** 4 * (r - 2 * a) ** 3
              * (4 * a * a + r * r) + 6 * x * x * (r - 2 * a) ** 2 * (2 * a - 3 * r) + 45 * (2 * a + r))
         / (8192 * SP * a ** 6 * r ** 5 * x ** 7),
         9 * (8 * x * x * (4 * a * a * (4 * r ** 6 * x ** 6 - 9 * r * r * x * x + 15) - 2 * r ** 8 * x ** 6
                           - 3 * r ** 4 * x * x + 6 * r * r) - 45) / (8192 * a ** 6 * r ** 5 * x ** 8),
         k56, k56]
    if case2:
        k[0] = 9 * (4 * a * a - r * r) ** 3 * (4 * a * a + r * r) / (512 * a ** 6 * r ** 5)
    b = [1, e(r), e(r - 2 * a), e(r + 2 * a), erfc(r * x), erfc((r - 2 * a) * x), erfc((r + 2 * a) * x)]
    return sum(c * v for c, v in zip(k, b))


@pytest.mark.parametrize('xi', [0.5, 0.8])
@pytest.mark.parametrize('r', [0.6, 1.0, 1.7, 2.0, 2.3, 3.0, 4.5, 6.0])
def test_F1_F2_match_appendix(r, xi):
    a, eta = 1.0, 1.0
    B = R.pair_blocks(np.array([[0.0, 0.0, r]]), xi, a, eta)[0]
    F1, F2 = F_printed(r, xi, a, r <= 2 * a)
    scale = 6 * math.pi * eta * a
    assert B[0, 0] * scale == pytest.approx(F1, abs=1e-12)
    assert B[1, 1] * scale == pytest.approx(F1, abs=1e-12)
    assert B[2, 2] * scale == pytest.approx(F2, abs=1e-12)
    assert abs(B[0, 2]) < 1e-15 and abs(B[0, 1]) < 1e-15


def _printed_DC_basis(rh):
    d = I3
    B1 = np.einsum('ij,mn->ijmn', d, d) + np.einsum('im,jn->ijmn', d, d) - 4 * np.einsum('in,jm->ijmn', d, d)
    B2 = np.einsum('jm,i,n->ijmn', d, rh, rh) - np.einsum('i,j,m,n->ijmn', rh, rh, rh, rh)
    B3 = (np.einsum('ij,m,n->ijmn', d, rh, rh) + np.einsum('im,j,n->ijmn', d, rh, rh)
          + np.einsum('jn,i,m->ijmn', d, rh, rh) + np.einsum('mn,i,j->ijmn', d, rh, rh)
          + np.einsum('in,j,m->ijmn', d, rh, rh) - 6 * np.einsum('i,j,m,n->ijmn', rh, rh, rh, rh)
          - np.einsum('in,jm->ijmn', d, d))
    return B1, B2, B3


@pytest.mark.parametrize('xi', [0.5, 0.7])
@pytest.mark.parametrize('r', [0.8, 1.5, 2.0, 2.5, 3.5, 5.0])
def test_K3_matches_appendix(r, xi):
    """Project 6 pi eta a M_DC onto the printed three-term basis (in the S -> E block)."""
    a, eta = 1.0, 1.0
    proj = lambda T: np.einsum('kij,ijmn,lmn->kl', Y, T, Y).ravel()
    A = np.stack([proj(B) for B in _printed_DC_basis(np.array([0.0, 0.0, 1.0]))], 1)
    _, _, _, DC = R.cartesian_blocks(np.array([[0.0, 0.0, r]]), xi, a, eta)
    sol, res, rank, _ = np.linalg.lstsq(A, 6 * math.pi * eta * a * proj(DC[0]), rcond=None)
    assert rank == 3 and res[0] < 1e-24
    assert sol[2] == pytest.approx(K3_printed(r, xi, a, r <= 2 * a), abs=1e-12)


@pytest.mark.parametrize('xi', [0.3, 0.5, 1.0])
def test_self_terms_match_appendix(xi):
    a, eta = 1.0, 1.0
    B = R.self_block(xi, a, eta)
    uf = (1 - math.exp(-4 * a * a * xi * xi) + 4 * SP * a * xi * erfc(2 * a * xi)) / (4 * SP * xi * a)
    assert B[0, 0] * 6 * math.pi * eta * a == pytest.approx(uf, rel=1e-12)
    k = (-3 * (6 * a * a * xi * xi + 1) / (80 * SP * a ** 6 * xi ** 3)
         + 3 * (10 * a * a * xi * xi + 1) / (80 * SP * a ** 6 * xi ** 3) * math.exp(-4 * a * a * xi * xi)
         - 3 / (10 * a ** 3) * erfc(2 * a * xi))
    # (d_ij d_mn + d_im d_jn - 4 d_in d_jm) : S = -3 S for symmetric traceless S
    assert B[3, 3] * 6 * math.pi * eta * a == pytest.approx(-3 * k, rel=1e-12)
    assert np.allclose(B[3:, 3:], B[3, 3] * np.eye(5), atol=1e-16)
    assert np.allclose(B[:3, 3:], 0) and np.allclose(B[3:, :3], 0)


def test_free_space_self_terms():
    for a in (1.0, 1.7):
        B = R.self_block(0.5, a, 2.0, free_only=True)
        assert B[0, 0] == pytest.approx(1 / (6 * math.pi * 2.0 * a), rel=1e-13)
        assert B[3, 3] == pytest.approx(3 / (20 * math.pi * 2.0 * a ** 3), rel=1e-13)


def test_rotne_prager_free_space():
    a, eta = 1.3, 0.7
    for r in (0.4, 1.1, 2.0, 2.6, 3.5, 7.0):
        B = R.pair_blocks(np.array([[0.0, 0.0, r]]), 0.5, a, eta, free_only=True)[0]
        if r >= 2 * a:
            perp = (1 + 2 * a * a / (3 * r * r)) / (8 * math.pi * eta * r)
            par = perp + (1 - 2 * a * a / (r * r)) / (8 * math.pi * eta * r)
        else:
            perp = (1 - 9 * r / (32 * a)) / (6 * math.pi * eta * a)
            par = perp + (3 * r / (32 * a)) / (6 * math.pi * eta * a)
        assert B[0, 0] == pytest.approx(perp, rel=1e-12)
        assert B[2, 2] == pytest.approx(par, rel=1e-12)


def test_faxen_forms_free_space():
    """Free-space UC, DF, DC for r > 2a against the Faxen operators on the Oseen tensor."""
    sp = pytest.importorskip('sympy')
    a, eta = 1.0, 1.0
    X = sp.symbols('x0 x1 x2', real=True)
    r = sp.sqrt(sum(v * v for v in X))
    J = [[(sp.KroneckerDelta(i, m) / r + X[i] * X[m] / r ** 3) / (8 * sp.pi * eta) for m in range(3)]
         for i in range(3)]
    lap = lambda f: sum(sp.diff(f, v, 2) for v in X)
    A = [[J[i][m] + sp.Rational(4, 15) * a * a * lap(J[i][m]) for m in range(3)] for i in range(3)]
    Bm = [[J[i][m] + sp.Rational(1, 5) * a * a * lap(J[i][m]) for m in range(3)] for i in range(3)]
    pt = {X[0]: 0.7, X[1]: -1.9, X[2]: 2.4}
    x = np.array([[0.7, -1.9, 2.4]])
    UF, UC, DF, DC = R.cartesian_blocks(x, 0.5, a, eta, free_only=True)
    for i in range(3):
        for m in range(3):
            for n in range(3):
                v = float(-sp.diff(A[i][m], X[n]).subs(pt))
                assert UC[0, i, m, n] == pytest.approx(v, abs=1e-12)
                assert DF[0, i, n, m] == pytest.approx(-v, abs=1e-12)
                for j in range(3):
                    w = float(-sp.diff(Bm[i][m], X[j], X[n]).subs(pt))
                    assert DC[0, i, j, m, n] == pytest.approx(w, abs=1e-12)


def _brute_U(kind, r, xi, a, n):
    """(1/2pi^2) int kappa_hat (1-H) k^{n-3} d^n/dr^n sin(kr) dk by composite Gauss-Legendre."""
    x, w = np.polynomial.legendre.leggauss(12)
    edges = np.arange(0.0, 4000.0 + 1e-9, 0.25)
    k = (0.5 * (edges[1:] + edges[:-1])[:, None] + 0.125 * x[None, :]).ravel()
    wk = np.tile(0.125 * w, edges.size - 1)
    ka = k * a
    s0 = np.sin(ka) / ka
    s1 = (np.sin(ka) - ka * np.cos(ka)) / ka ** 3
    small = ka < 1e-2
    s1[small] = 1 / 3 - ka[small] ** 2 / 30
    kap = {'aa': s0 * s0, 'ab': 3 * s0 * s1, 'bb': 9 * s1 * s1}[kind]
    u = k * k / (4 * xi * xi)
    omh = -np.expm1(-u) - u * np.exp(-u)
    trig = np.sin(k * r + n * math.pi / 2)
    return np.sum(wk * kap * omh * k ** (n - 3) * trig) / (2 * math.pi ** 2)


@pytest.mark.parametrize('r', [1.3, 2.7])
def test_profiles_against_fourier_definition(r):
    a, xi = 1.0, 0.6
    for kind, orders in (('aa', (2,)), ('ab', (2, 3)), ('bb', (2, 3, 4))):
        for n in orders:
            got = R.conv_U(kind, np.array([r]), xi, a, n)[0]
            ref = _brute_U(kind, r, xi, a, n)
            assert got == pytest.approx(ref, abs=2e-8), (kind, n)


def test_continuity_at_contact():
    a = 1.0
    lo = R.pair_blocks(np.array([[0.3, 0.4, 0.0]]) * (2 * a - 1e-7) / 0.5, 0.5, a, 1.0)[0]
    hi = R.pair_blocks(np.array([[0.3, 0.4, 0.0]]) * (2 * a + 1e-7) / 0.5, 0.5, a, 1.0)[0]
    assert np.max(np.abs(lo - hi)) < 1e-6


def test_block_symmetry():
    x = np.array([[0.3, -1.2, 2.5], [1.1, 0.2, -0.4], [3.0, 2.0, 1.0]])
    Bp = R.pair_blocks(x, 0.6, 1.0, 1.0)
    Bm = R.pair_blocks(-x, 0.6, 1.0, 1.0)
    assert np.max(np.abs(Bp - np.transpose(Bm, (0, 2, 1)))) < 1e-16
