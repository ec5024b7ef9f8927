"""GPU parity of the Euler-Maruyama step with a random-finite-difference drift
(pse_rfd_step, the alternative to the mid-point scheme discussed in Sec. 3.4)
against the oracle's rfd_step on the same noise.

Tolerances: the step (displacement, stresslets of the solve at x_k) 1e-9 in
FP64 and 2e-5 mixed, as for the mid-point step.  The drift alone, the
difference of two steps that differ only in the direction W (W and 0), is a
difference of two constrained products divided by delta; with GMRES stopped at
1e-6 in the mixed form, its error is about 1e-6 |R W| / (delta |div R| |W|),
1e-3 relative at delta = 0.05, so the mixed drift is held to 1e-2 and the FP64
drift (solves to 1e-13) to 1e-8.
"""
import numpy as np
import pytest

import pse_inputs
from oracle import params, philox, pse as opse

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

N, PHI, XI, TOL, DT, DELTA = 150, 0.2, 0.7, 1e-3, 1e-3, 0.05


@pytest.fixture(scope='module')
def pkg():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import paper_1709_06946_gb300 as p
    p.build()
    p.load()
    return p


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _disp(x1, x0, L):
    d = x1 - x0
    return d - L * np.rint(d / L)


def _handle(pkg, prec, L):
    ktol = 1e-13 if prec == 'fp64' else 1e-6
    return pkg.PSE(N, L, xi=XI, tol=TOL, precision=prec, lanczos_tol=0.0, lanczos_maxiter=10, krylov_tol=ktol,
                   krylov_maxiter=100)


def _oracle_params(h, L):
    inf = h.info
    return params.choose(N, L, 1.0, 1.0, 1.0, XI, TOL, Ng=inf['Ng'], P=inf['P'], rcut=inf['rcut'])


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
@pytest.mark.parametrize('with_force', [False, True])
def test_rfd_step_matches_oracle(pkg, prec, with_force):
    pos, L = pse_inputs.rsa_positions(N, PHI, seed=13)
    h = _handle(pkg, prec, L)
    p = _oracle_params(h, L)
    dt_ = torch.float64 if prec == 'fp64' else torch.float32
    w1 = pse_inputs.lanczos_noise(N, seed=14)
    w2 = pse_inputs.wave_noise(p.Ng, seed=15)
    wt = np.random.default_rng(16).standard_normal((N, 3))
    FP = pse_inputs.moments(N, seed=17)[0] * 5.0 if with_force else None

    def gpu(wt_):
        x = torch.tensor(pos, device='cuda')
        S, st = h.rfd_step(x, DT, FP=None if FP is None else torch.tensor(FP, device='cuda', dtype=dt_), delta=DELTA,
                           w1=torch.tensor(w1, device='cuda', dtype=dt_), w2=torch.tensor(w2, device='cuda', dtype=dt_),
                           wt=torch.tensor(wt_, device='cuda', dtype=dt_), want_S=True)
        return x.cpu().numpy(), S.double().cpu().numpy(), st

    x1, S, st = gpu(wt)
    xo, So, drift_o, sto = opse.rfd_step(pos, FP, DT, w1, w2, wt, DELTA, p, lanczos_tol=0.0, lanczos_maxiter=10,
                                         krylov_tol=1e-13, krylov_maxiter=100)
    tol = 1e-9 if prec == 'fp64' else 2e-5
    assert _rel(_disp(x1, pos, L), _disp(xo, pos, L)) < tol
    assert _rel(S, So) < tol
    assert st['krylov_iters'] >= 3 and st['lanczos_iters'] == 10
    # the drift alone: the same step with W = 0 has no drift term
    x0w, _, _ = gpu(np.zeros_like(wt))
    drift = _disp(x1, x0w, L) / DT
    assert _rel(drift, drift_o) < (1e-8 if prec == 'fp64' else 1e-2)
    h.close()


def test_rfd_in_kernel_noise_matches_published_generator(pkg):
    """pse_rfd_step's in-kernel noise (streams 1, 2, 3 of Philox4x32-10) equals the
    same streams generated by the oracle and passed in."""
    pos, L = pse_inputs.rsa_positions(N, PHI, seed=12)
    h = _handle(pkg, 'fp64', L)
    Ng = h.info['Ng']
    seed, step = 0x0123456789ABCDEF, 5
    xa = torch.tensor(pos, device='cuda')
    h.rfd_step(xa, DT, delta=DELTA, seed=seed, step=step)
    xb = torch.tensor(pos, device='cuda')
    h.rfd_step(xb, DT, delta=DELTA, w1=torch.tensor(philox.lanczos_noise(seed, step, N), device='cuda'),
               w2=torch.tensor(philox.wave_noise(seed, step, Ng), device='cuda'),
               wt=torch.tensor(philox.rfd_noise(seed, step, N), device='cuda'))
    d = _disp(xa.cpu().numpy(), pos, L)
    assert _rel(d, _disp(xb.cpu().numpy(), pos, L)) < 1e-12
    h.close()
