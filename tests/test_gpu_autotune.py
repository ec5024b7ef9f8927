"""GPU tests of the autotuner: it times the candidates, keeps the fastest, and
the tuned handle computes the same products as before (parity with the oracle
is independent of lanes and tiles)."""
import numpy as np
import pytest

import pse_inputs
from oracle import params, pse as opse

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_autotune_keeps_results(pkg, prec):
    N, phi, xi, tol = 20000, 0.3, 0.5, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=91)
    F, S = pse_inputs.moments(N, seed=92)
    dt = torch.float64 if prec == 'fp64' else torch.float32
    x = torch.tensor(pos, device='cuda', dtype=torch.float64)
    Ft = torch.tensor(F, device='cuda', dtype=dt)
    St = torch.tensor(S, device='cuda', dtype=dt)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec)
    U0, E0 = h.mobility(x, Ft, St)
    t = h.autotune(x, reps=2)
    assert t['real_lanes'] in (1, 4, 8, 16, 32) and len(t['real_ms']) == 5 and len(t['wave_ms']) >= 2
    tried = list(t['real_ms'].values()) + ([t['real_smem_ms']] if t['real_smem_ms'] > 0 else [])
    assert t['best_real_ms'] == min(tried)
    assert t['real_smem_table'] == (t['real_smem_ms'] > 0 and t['real_smem_ms'] < min(t['real_ms'].values()))
    assert t['best_wave_ms'] == min(t['wave_ms'].values())
    assert tuple(h.info['tile']) == t['tile'] and t['tile'] in t['wave_ms']
    U1, E1 = h.mobility(x, Ft, St)
    got = np.concatenate([U1.double().cpu().numpy(), E1.double().cpu().numpy()], 1)
    ref = np.concatenate([U0.double().cpu().numpy(), E0.double().cpu().numpy()], 1)
    assert _rel(got, ref) < (1e-12 if prec == 'fp64' else 1e-6)
    # and the tuned handle still matches the oracle's NUFFT (tiles must not change the wave part)
    inf = h.info
    p = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, Ng=inf['Ng'], P=inf['P'], rcut=inf['rcut'])
    Uw, Ew = h.mobility(x, Ft, St, parts='wave')
    w = opse.wave_apply(pos, F, S, p)
    wave = np.concatenate([Uw.double().cpu().numpy(), Ew.double().cpu().numpy()], 1)
    assert _rel(wave, np.concatenate([w['U'], w['E']], 1)) < (1e-10 if prec == 'fp64' else 2e-5)
    h.close()


def test_autotune_batch(pkg):
    Ns, Ls, pos = [], [], []
    for k, (n, phi) in enumerate([(3000, 0.1), (8000, 0.3), (1500, 0.4)]):
        x, L = pse_inputs.hard_sphere_positions(n, phi, seed=95 + k)
        Ns.append(n)
        Ls.append(L)
        pos.append(x)
    X = torch.tensor(np.concatenate(pos), device='cuda', dtype=torch.float64)
    F, S = pse_inputs.moments(sum(Ns), seed=99)
    Ft = torch.tensor(F, device='cuda', dtype=torch.float32)
    St = torch.tensor(S, device='cuda', dtype=torch.float32)
    h = pkg.PSE(Ns, Ls, xi=0.5, tol=1e-3, precision='mixed')
    U0, E0 = h.mobility(X, Ft, St)
    h.autotune(X, reps=2)
    U1, E1 = h.mobility(X, Ft, St)
    assert _rel(U1.cpu().numpy(), U0.cpu().numpy()) < 1e-6 and _rel(E1.cpu().numpy(), E0.cpu().numpy()) < 1e-6
    xa = X.clone()
    _, st = h.step(xa, 1e-3, seed=3, step=1)
    assert st['krylov_iters'] >= 1
    h.close()
