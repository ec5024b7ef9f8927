"""Equilibrium validation runs of Sec. 4 on the GPU path (mixed precision).

* Two spheres joined by U = k |r - r0| sample the Boltzmann density of the
  centre distance, f(r) = kt^3 r^2 exp(-kt |r - r0|) / (2 (2 + kt^2 r0^2)), under the
  constrained mid-point step and under the RFD Euler-Maruyama step.  Checked: the
  mean distance against the density's mean within 4 standard errors of batch
  means (batches of 10 time units, many times the 0.4 relaxation time
  (1/kt)^2 / (2 x 0.053)), and the Kolmogorov distance to the CDF below 0.1
  (about 2/sqrt of the number of independent samples, plus the scheme's O(dt)
  bias at dt = 0.01, 2.5 % of the relaxation time).
* Non-interacting spheres keep S(q) = 1 over 30 time units of dynamics: the
  average over the box's wave vectors up to |n| = 12 and over snapshots is 1
  within 4 standard errors, and every shell within 5.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import pse_inputs
from oracle import equilibrium as eq

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

K, R0, L, XI = 5.0, 3.0, 10.0, 1.0


@pytest.fixture(scope='module')
def pkg():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import paper_1709_06946_gb300 as p
    p.build()
    p.load()
    return p


def _check_pair_samples(r, batches=20):
    mean_ref = quad(lambda s: s * eq.pair_pdf(s, K, R0), 0, R0)[0] + quad(lambda s: s * eq.pair_pdf(s, K, R0),
                                                                          R0, np.inf)[0]
    bm = np.array([b.mean() for b in np.array_split(r, batches)])
    se = bm.std(ddof=1) / np.sqrt(batches)
    assert abs(r.mean() - mean_ref) < 4 * se + 1e-3, (r.mean(), mean_ref, se)
    rs = np.sort(r)
    emp = np.arange(1, rs.size + 1) / rs.size
    ks = np.max(np.abs(emp - eq.pair_cdf(rs, K, R0)))
    assert ks < 0.1, ks
    return ks


@pytest.mark.parametrize('scheme,steps,every', [('midpoint', 20000, 10), ('rfd', 6000, 5)])
def test_spring_pair_samples_boltzmann(pkg, scheme, steps, every):
    from paper_1709_06946_gb300.equilibrium import pair_distance_run
    h = pkg.PSE(2, L, xi=XI, tol=1e-3, precision='mixed', use_graph=1)
    x = torch.tensor([[3.0, 5.0, 5.0], [3.0 + R0, 5.0, 5.0]], device='cuda', dtype=torch.float64)
    r = pair_distance_run(h, x, L, K, R0, 0.01, steps, every=every, seed=11, scheme=scheme, delta=0.01, burn=500)
    _check_pair_samples(r)
    h.close()


def test_ideal_particles_keep_unit_structure_factor(pkg):
    from paper_1709_06946_gb300.equilibrium import ideal_structure_factor_run
    N, phi = 8000, 0.2
    Lb = pse_inputs.box_length(N, phi)
    h = pkg.PSE(N, Lb, xi=0.6, tol=1e-3, precision='mixed', use_graph=1)
    x = torch.tensor(pse_inputs.random_positions(N, Lb, seed=5), device='cuda', dtype=torch.float64)
    qs, S, cnt = ideal_structure_factor_run(h, x, Lb, 0.05, 600, 20, 12, seed=3)
    # each S(q) is exponentially distributed with mean 1; counting the snapshots as
    # one (long-wavelength modes decorrelate slowly) the grand mean has error
    # 1/sqrt(number of wave vectors)
    grand = np.average(S, axis=1, weights=cnt).mean()
    assert abs(grand - 1.0) < 4.0 / np.sqrt(cnt.sum()), (grand, S.mean(0))
    assert np.all(np.abs(S.mean(0) - 1.0) < 5.0 / np.sqrt(cnt)), S.mean(0)
    h.close()
