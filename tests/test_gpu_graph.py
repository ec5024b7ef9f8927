"""GPU tests of the graph-captured constrained step (use_graph=1): the whole
mid-point step, with the Lanczos and GMRES loops as conditional while nodes and
their scalar steps on the device, gives the same result as the host-launched
step, reuses the graph across steps (new noise each step) and recaptures when
dt or the force changes."""
import numpy as np
import pytest

import pse_inputs

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


def _disp(x, x0, L):
    d = x - x0
    return d - L * np.rint(d / L)


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_graph_step_equals_host_step(pkg, prec):
    N, phi, xi, tol = 3000, 0.25, 0.5, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=121)
    FP = pse_inputs.moments(N, seed=122)[0] * 2.0
    dt = torch.float64 if prec == 'fp64' else torch.float32
    F = torch.tensor(FP, device='cuda', dtype=dt)
    he = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec)
    hg = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, use_graph=1)
    xe = torch.tensor(pos, device='cuda', dtype=torch.float64)
    xg = xe.clone()
    tolr = 1e-10 if prec == 'fp64' else 1e-5
    for k in range(3):                          # the captured graph is reused with new noise each step
        Se, ste = he.step(xe, 1e-3, FP=F, seed=5, step=k, want_S=True)
        Sg, stg = hg.step(xg, 1e-3, FP=F, seed=5, step=k, want_S=True)
        assert hg.graph_ready() == (True, '')
        assert stg['lanczos_iters'] == ste['lanczos_iters'] and stg['krylov_iters'] == ste['krylov_iters']
        assert _rel(_disp(xg.cpu().numpy(), pos, L), _disp(xe.cpu().numpy(), pos, L)) < tolr
        assert _rel(Sg.double().cpu().numpy(), Se.double().cpu().numpy()) < tolr
    # no force and a new dt: recaptured, still equal
    Se, ste = he.step(xe, 2e-3, seed=6, step=9, want_S=True)
    Sg, stg = hg.step(xg, 2e-3, seed=6, step=9, want_S=True)
    assert _rel(_disp(xg.cpu().numpy(), pos, L), _disp(xe.cpu().numpy(), pos, L)) < 10 * tolr
    he.close()
    hg.close()


def test_graph_step_batch(pkg):
    Ns, Ls, pos = [], [], []
    for k, (n, phi) in enumerate([(700, 0.05), (2500, 0.3), (1200, 0.42)]):
        x, L = pse_inputs.hard_sphere_positions(n, phi, seed=130 + k)
        Ns.append(n)
        Ls.append(L)
        pos.append(x)
    X = np.concatenate(pos)
    he = pkg.PSE(Ns, Ls, xi=0.5, tol=1e-3, precision='fp64')
    hg = pkg.PSE(Ns, Ls, xi=0.5, tol=1e-3, precision='fp64', use_graph=1)
    xe = torch.tensor(X, device='cuda', dtype=torch.float64)
    xg = xe.clone()
    for k in range(2):
        he.step(xe, 1e-3, seed=8, step=k)
        hg.step(xg, 1e-3, seed=8, step=k)
    assert hg.graph_ready()[0]
    for s in range(3):
        a, b = hg.system_stats(s), he.system_stats(s)
        assert a['krylov_iters'] == b['krylov_iters'] and a['lanczos_iters'] == b['lanczos_iters']
    assert _rel(xg.cpu().numpy() - X, xe.cpu().numpy() - X) < 1e-9
    he.close()
    hg.close()


def test_graph_step_host_arrays(pkg):
    """Graph steps through host (numpy) arrays: positions copied in and out every step."""
    N, phi = 2000, 0.2
    pos, L = pse_inputs.rsa_positions(N, phi, seed=141)
    h = pkg.PSE(N, L, xi=0.5, tol=1e-3, precision='mixed', use_graph=1)
    x = pos.copy()
    for k in range(2):
        h.step(x, 1e-3, seed=1, step=k)
    d = _disp(x, pos, L)
    assert np.isfinite(d).all() and 0 < np.abs(d).max() < 0.5
    h.close()


def test_graph_step_equals_oracle(pkg):
    """The graph-captured step with in-kernel noise against the oracle's mid-point step driven by the
    same Philox4x32-10 streams (counter = step), FP64, fixed Lanczos length, tight GMRES."""
    from oracle import params, philox, pse as opse
    N, phi, xi, tol, dt = 150, 0.2, 0.7, 1e-3, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=13)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64', use_graph=1, lanczos_tol=0.0, lanczos_maxiter=10,
                krylov_tol=1e-10, krylov_maxiter=100)
    inf = h.info
    p = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, Ng=inf['Ng'], P=inf['P'], rcut=inf['rcut'])
    seed = 0x5EED
    x = torch.tensor(pos, device='cuda', dtype=torch.float64)
    xo = pos.copy()
    for k in range(2):                      # capture, then a replay with the next step's noise
        S, st = h.step(x, dt, seed=seed, step=k, want_S=True)
        w1 = philox.lanczos_noise(seed, k, N)
        w2 = philox.wave_noise(seed, k, p.Ng)
        xo, So, _ = opse.constrained_step(xo, None, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=10,
                                          krylov_tol=1e-13, krylov_maxiter=200)
        assert h.graph_ready() == (True, '')
        assert _rel(_disp(x.cpu().numpy(), pos, L), _disp(xo, pos, L)) < 1e-9
        assert _rel(S.cpu().numpy(), So) < 1e-9
    h.close()
