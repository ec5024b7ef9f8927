"""Pins for oracle.equilibrium (the equilibrium distributions of Sec. 4)."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import equilibrium as eq


@pytest.mark.parametrize('k,r0', [(5.0, 3.0), (10.0, 2.5), (2.0, 4.0)])
def test_pair_pdf_is_the_normalised_boltzmann_density(k, r0):
    """f(r) equals r^2 exp(-U(r)/kT) normalised by quadrature over r > 0, up to
    the dropped O(exp(-k r0 / kT)) mass on r < 0."""
    kT = 1.3
    w = lambda r: r ** 2 * np.exp(-k * abs(r - r0) / kT)
    Z = quad(w, 0, r0)[0] + quad(w, r0, np.inf)[0]
    tail = np.exp(-k * r0 / kT) * 10
    for r in np.linspace(0.1, r0 + 6 * kT / k, 17):
        assert abs(eq.pair_pdf(r, k, r0, kT) - w(r) / Z) <= 1e-12 + tail * w(r) / Z
    assert abs(quad(lambda r: eq.pair_pdf(r, k, r0, kT), 0, r0)[0]
               + quad(lambda r: eq.pair_pdf(r, k, r0, kT), r0, np.inf)[0] - 1.0) < tail


@pytest.mark.parametrize('k,r0', [(5.0, 3.0), (8.0, 2.2)])
def test_pair_cdf_integrates_the_pdf(k, r0):
    for r in (0.5, r0 - 0.3, r0, r0 + 0.2, r0 + 2.0):
        ref = quad(lambda s: eq.pair_pdf(s, k, r0), 0, r, points=[r0] if r > r0 else None)[0]
        assert abs(eq.pair_cdf(r, k, r0) - ref) < 1e-10
    assert abs(eq.pair_cdf(1e3, k, r0) - 1.0) < 10 * np.exp(-k * r0)


def test_structure_factor_of_uniform_positions_is_one():
    """Uniform independent positions: S(q) has mean 1 (and the exponential law, variance 1)."""
    L, N = 20.0, 4000
    qv, shell, qs = eq.q_shells(L, 4)
    rng = np.random.default_rng(3)
    S = np.array([eq.structure_factor(rng.uniform(0, L, (N, 3)), L, qv) for _ in range(20)])
    m = S.mean()
    assert abs(m - 1.0) < 4.0 / np.sqrt(S.size)
    assert abs(S.var() - 1.0) < 0.2
    # the q = 0 term is N: the shells exclude it, and the definition gives N there
    assert abs(eq.structure_factor(rng.uniform(0, L, (N, 3)), L, np.zeros((1, 3)))[0] - N) < 1e-6 * N
    assert qs[0] == pytest.approx(2 * np.pi / L) and shell.max() + 1 == len(qs)
