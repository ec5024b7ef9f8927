"""Pins for oracle.params: Table tab:lmax, Eqs. lmax1/lmax2 and the parameter rules."""
import math
import os

import pytest

from oracle import params

GOLD = os.path.join(os.path.dirname(__file__), 'golden', 'table_lmax.txt')


def _table():
    rows = []
    for line in open(GOLD):
        if line.strip() and not line.startswith('#'):
            rows.append([float(v) for v in line.split()])
    return rows


def test_lambda_max_matches_table():
    for g, ls, _, e, le, _ in _table():
        assert round(params.lambda_max_shear(g), 2) == pytest.approx(ls, abs=1e-9)
        assert round(params.lambda_max_ext(e), 2) == pytest.approx(le, abs=1e-9)


def test_support_size_rows_that_follow_the_bound():
    # The lambda = 1 row and the mild-deformation rows follow Eq. bound with C = 1
    # evaluated at the printed (two-decimal) lambda values.
    rows = _table()
    for g, ls, Ps, e, le, Pe in rows[:2]:
        assert params.support_rule(1e-3, ls) == int(Ps)
        assert params.support_rule(1e-3, le) == int(Pe)
    # The remaining rows of the printed table are not reproduced by the bound
    # (a reading of the table); the bound is monotone in lambda.
    prev = 0
    for g in (0.0, 0.1, 0.5, 1.0):
        P = params.support_rule(1e-3, params.lambda_max_shear(g))
        assert P >= prev
        prev = P


def test_support_size_tolerances():
    assert params.support_rule(1e-3) == 5
    assert params.support_rule(1e-4) == 6
    assert params.quadrature_bound(5) < 1e-3 < params.quadrature_bound(4)


def test_rcut_and_kcut_rules():
    xi, tol = 0.5, 1e-3
    rc = params.rcut_rule(xi, tol)
    assert math.exp(-(xi * rc) ** 2) == pytest.approx(tol, rel=1e-12)
    kc = params.kcut_rule(xi, tol)
    assert params.hasimoto_H(kc, xi) == pytest.approx(tol, rel=1e-9)


@pytest.mark.parametrize('N,phi,xi,tol', [(100, 0.1, 0.5, 1e-3), (10000, 0.3, 0.5, 1e-3),
                                          (1048576, 0.3, 0.5, 1e-3), (1048576, 0.3, 0.4, 1e-4)])
def test_choose_grid_and_width(N, phi, xi, tol):
    L = (4 * math.pi * N / (3 * phi)) ** (1 / 3)
    p = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol)
    assert p.eta_g < 1.0
    assert p.Ng % 2 == 0 and p.Ng >= p.kcut * L / math.pi
    assert p.m == pytest.approx(math.sqrt(math.pi * p.P))
    assert p.eta_g == pytest.approx((p.h * p.P * xi / p.m) ** 2)
    assert params.quadrature_bound(p.P) <= tol / 10
    assert p.rcut == pytest.approx(1.0 + math.sqrt(math.log(10 / tol)) / xi)
    pp = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, rule='paper')
    assert pp.P == params.support_rule(tol)
