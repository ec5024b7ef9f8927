"""GPU parity of batched handles (several independent suspensions in one handle).

A batch must give, for every suspension, what the FP64 oracle gives for that
suspension alone (same tolerances as the single-suspension tests), and what a
separate single-suspension handle gives up to rounding.  The batch's arrays are
the concatenation of the suspensions' arrays; in-kernel noise uses global
Philox indices (suspension s's indices follow those of suspensions 0..s-1).
"""
import numpy as np
import pytest

import pse_inputs
from oracle import params, philox, pse as opse

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL = {'fp64': 1e-10, 'mixed': 2e-5}
XI, EPS = 0.5, 1e-3
# (N, phi, position seed): boxes from 16.1 to 19.6, densities 0.05 .. 0.3, ragged sizes
SYSTEMS = [(100, 0.1, 21), (57, 0.05, 22), (300, 0.3, 23), (211, 0.15, 24)]


@pytest.fixture(scope='module')
def pkg():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import paper_1709_06946_gb300 as p
    p.build()
    p.load()
    return p


def _dt(prec):
    return torch.float64 if prec == 'fp64' else torch.float32


def _cuda(x, dtype):
    return torch.tensor(np.ascontiguousarray(x), device='cuda', dtype=dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _inputs():
    pos, Ls, F, S = [], [], [], []
    for k, (N, phi, seed) in enumerate(SYSTEMS):
        x, L = pse_inputs.rsa_positions(N, phi, seed=seed)
        f, s = pse_inputs.moments(N, seed=100 + k)
        pos.append(x)
        Ls.append(L)
        F.append(f)
        S.append(s)
    return pos, Ls, F, S


def _oracle_params(h, s, N, L):
    inf = h.system_info(s)
    assert inf['N'] == N and abs(inf['L'] - L) < 1e-12
    return params.choose(N, L, 1.0, 1.0, 1.0, XI, EPS, Ng=inf['Ng'], P=inf['P'], rcut=inf['rcut'])


def _split(h, arr):
    return [arr[h.offsets[s]:h.offsets[s + 1]] for s in range(h.nsys)]


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_batch_mobility_matches_oracle(pkg, prec):
    pos, Ls, F, S = _inputs()
    Ns = [n for n, _, _ in SYSTEMS]
    h = pkg.PSE(Ns, Ls, xi=XI, tol=EPS, precision=prec)
    assert h.nsys == len(SYSTEMS) and h.N == sum(Ns)
    U, E = h.mobility(_cuda(np.concatenate(pos), torch.float64), _cuda(np.concatenate(F), _dt(prec)),
                      _cuda(np.concatenate(S), _dt(prec)))
    got = np.concatenate([U.double().cpu().numpy(), E.double().cpu().numpy()], 1)
    for s, part in enumerate(_split(h, got)):
        p = _oracle_params(h, s, Ns[s], Ls[s])
        Uo, Eo = opse.mobility_apply(pos[s], F[s], S[s], p)
        assert _rel(part, np.concatenate([Uo, Eo], 1)) < TOL[prec], s
    h.close()


def test_batch_equals_separate_handles(pkg):
    """Mobility, Brownian sample and constrained step (external noise) of a batch
    equal those of one handle per suspension (FP64, up to rounding)."""
    pos, Ls, F, S = _inputs()
    Ns = [n for n, _, _ in SYSTEMS]
    opts = dict(xi=XI, tol=EPS, precision='fp64', lanczos_tol=1e-8, krylov_tol=1e-9)
    hb = pkg.PSE(Ns, Ls, **opts)
    singles = [pkg.PSE(Ns[s], Ls[s], **opts) for s in range(len(Ns))]
    w1 = [pse_inputs.lanczos_noise(Ns[s], seed=200 + s) for s in range(len(Ns))]
    w2 = [pse_inputs.wave_noise(singles[s].info['Ng'], seed=300 + s) for s in range(len(Ns))]
    f64 = torch.float64
    # mobility
    Ub, Eb = hb.mobility(_cuda(np.concatenate(pos), f64), _cuda(np.concatenate(F), f64), _cuda(np.concatenate(S), f64))
    for s, hs in enumerate(singles):
        U1, E1 = hs.mobility(_cuda(pos[s], f64), _cuda(F[s], f64), _cuda(S[s], f64))
        sl = slice(hb.offsets[s], hb.offsets[s + 1])
        assert _rel(Ub[sl].cpu().numpy(), U1.cpu().numpy()) < 1e-12
        assert _rel(Eb[sl].cpu().numpy(), E1.cpu().numpy()) < 1e-12
    # Brownian sample with external noise; per-suspension Lanczos iteration counts
    W1 = np.concatenate(w1)
    W2 = np.concatenate([w.ravel() for w in w2])
    Ub, Eb, stb = hb.brownian(_cuda(np.concatenate(pos), f64), 1e-3, w1=_cuda(W1, f64), w2=_cuda(W2, f64))
    iters = []
    for s, hs in enumerate(singles):
        U1, E1, st1 = hs.brownian(_cuda(pos[s], f64), 1e-3, w1=_cuda(w1[s], f64), w2=_cuda(w2[s], f64))
        sl = slice(hb.offsets[s], hb.offsets[s + 1])
        assert _rel(Ub[sl].cpu().numpy(), U1.cpu().numpy()) < 1e-10
        assert _rel(Eb[sl].cpu().numpy(), E1.cpu().numpy()) < 1e-10
        assert hb.system_stats(s)['lanczos_iters'] == st1['lanczos_iters']
        iters.append(st1['lanczos_iters'])
    assert stb['lanczos_iters'] == max(iters)
    # constrained step with external noise and a force
    FP = [pse_inputs.moments(Ns[s], seed=400 + s)[0] for s in range(len(Ns))]
    xb = _cuda(np.concatenate(pos), f64)
    Sb, stb = hb.step(xb, 1e-3, FP=_cuda(np.concatenate(FP), f64), w1=_cuda(W1, f64), w2=_cuda(W2, f64), want_S=True)
    for s, hs in enumerate(singles):
        x1 = _cuda(pos[s], f64)
        S1, st1 = hs.step(x1, 1e-3, FP=_cuda(FP[s], f64), w1=_cuda(w1[s], f64), w2=_cuda(w2[s], f64), want_S=True)
        sl = slice(hb.offsets[s], hb.offsets[s + 1])
        d_b = xb[sl].cpu().numpy() - pos[s]
        d_1 = x1.cpu().numpy() - pos[s]
        d_b -= Ls[s] * np.rint(d_b / Ls[s])
        d_1 -= Ls[s] * np.rint(d_1 / Ls[s])
        assert _rel(d_b, d_1) < 1e-9
        assert _rel(Sb[sl].cpu().numpy(), S1.cpu().numpy()) < 1e-9
        assert hb.system_stats(s)['krylov_iters'] == st1['krylov_iters']
    for hh in [hb] + singles:
        hh.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_batch_step_matches_oracle(pkg, prec):
    """Constrained step of every suspension of a batch against the oracle (fixed
    Lanczos length, tight GMRES tolerance), external noise."""
    pos, Ls, F, S = _inputs()
    Ns = [n for n, _, _ in SYSTEMS]
    ktol = 1e-10 if prec == 'fp64' else 1e-6
    h = pkg.PSE(Ns, Ls, xi=XI, tol=EPS, precision=prec, lanczos_tol=0.0, lanczos_maxiter=10, krylov_tol=ktol,
                krylov_maxiter=100)
    ps = [_oracle_params(h, s, Ns[s], Ls[s]) for s in range(len(Ns))]
    w1 = [pse_inputs.lanczos_noise(Ns[s], seed=500 + s) for s in range(len(Ns))]
    w2 = [pse_inputs.wave_noise(ps[s].Ng, seed=600 + s) for s in range(len(Ns))]
    FP = [pse_inputs.moments(Ns[s], seed=700 + s)[0] * 3.0 for s in range(len(Ns))]
    x = _cuda(np.concatenate(pos), torch.float64)
    Sg, st = h.step(x, 1e-3, FP=_cuda(np.concatenate(FP), _dt(prec)), w1=_cuda(np.concatenate(w1), _dt(prec)),
                    w2=_cuda(np.concatenate([w.ravel() for w in w2]), _dt(prec)), want_S=True)
    xg = x.cpu().numpy()
    Sg = Sg.double().cpu().numpy()
    for s in range(len(Ns)):
        x1, So, _ = opse.constrained_step(pos[s], FP[s], 1e-3, w1[s], w2[s], ps[s], lanczos_tol=0.0,
                                          lanczos_maxiter=10, krylov_tol=1e-12, krylov_maxiter=200)
        sl = slice(h.offsets[s], h.offsets[s + 1])
        d_o = x1 - pos[s]
        d_g = xg[sl] - pos[s]
        d_o -= Ls[s] * np.rint(d_o / Ls[s])
        d_g -= Ls[s] * np.rint(d_g / Ls[s])
        assert _rel(d_g, d_o) < (1e-9 if prec == 'fp64' else 2e-5), s
        assert _rel(Sg[sl], So) < (1e-9 if prec == 'fp64' else 2e-5), s
        assert h.system_stats(s)['lanczos_iters'] == 10
    h.close()


def test_batch_mixes_tile_kinds(pkg):
    """Mixed precision batch where one suspension has 16^3 spreading tiles (the
    specialised kernels, parity with the oracle in test_gpu_parity) and the
    others smaller grids (the general kernels): the small ones against the
    oracle, the 16^3 one against a handle of its own."""
    systems = [(5000, 0.3, 41), (300, 0.3, 42), (211, 0.15, 43)]
    pos, Ls, F, S = [], [], [], []
    for k, (N, phi, seed) in enumerate(systems):
        x, L = pse_inputs.rsa_positions(N, phi, seed=seed)
        f, s_ = pse_inputs.moments(N, seed=140 + k)
        pos.append(x)
        Ls.append(L)
        F.append(f)
        S.append(s_)
    Ns = [n for n, _, _ in systems]
    h = pkg.PSE(Ns, Ls, xi=XI, tol=EPS, precision='mixed')
    infos = [h.system_info(s) for s in range(len(Ns))]
    assert tuple(infos[0]['tile']) == (16, 16, 16) and infos[0]['Ng'] >= 32
    assert any(tuple(i['tile']) != (16, 16, 16) or i['Ng'] < 32 for i in infos[1:])
    f32 = torch.float32
    U, E = h.mobility(_cuda(np.concatenate(pos), torch.float64), _cuda(np.concatenate(F), f32),
                      _cuda(np.concatenate(S), f32))
    got = np.concatenate([U.double().cpu().numpy(), E.double().cpu().numpy()], 1)
    for s, part in enumerate(_split(h, got)):
        if s == 0:
            continue
        p = _oracle_params(h, s, Ns[s], Ls[s])
        Uo, Eo = opse.mobility_apply(pos[s], F[s], S[s], p)
        assert _rel(part, np.concatenate([Uo, Eo], 1)) < TOL['mixed'], s
    h1 = pkg.PSE(Ns[0], Ls[0], xi=XI, tol=EPS, precision='mixed')
    U1, E1 = h1.mobility(_cuda(pos[0], torch.float64), _cuda(F[0], f32), _cuda(S[0], f32))
    one = np.concatenate([U1.double().cpu().numpy(), E1.double().cpu().numpy()], 1)
    assert _rel(_split(h, got)[0], one) < 1e-6
    h.close()
    h1.close()


def test_batch_in_kernel_noise_uses_global_indices(pkg):
    """In-kernel noise of a batch equals external noise drawn by the oracle's
    Philox with suspension s's indices following those of suspensions 0..s-1."""
    pos, Ls, _, _ = _inputs()
    Ns = [n for n, _, _ in SYSTEMS]
    h = pkg.PSE(Ns, Ls, xi=XI, tol=EPS, precision='fp64', lanczos_tol=1e-12)
    seed, counter = 0xC0FFEE12345, 9
    f64 = torch.float64
    X = _cuda(np.concatenate(pos), f64)
    U, E, _ = h.brownian(X, 1e-2, seed=seed, counter=counter)
    w1 = philox.lanczos_noise(seed, counter, h.N)
    w2, k0 = [], 0
    for s in range(h.nsys):
        Ng = h.system_info(s)['Ng']
        w2.append(philox.wave_noise(seed, counter, Ng, index0=3 * k0).ravel())
        k0 += Ng * Ng * (Ng // 2 + 1)
    U2, E2, _ = h.brownian(X, 1e-2, w1=_cuda(w1, f64), w2=_cuda(np.concatenate(w2), f64))
    a = np.concatenate([U.cpu().numpy(), E.cpu().numpy()], 1)
    b = np.concatenate([U2.cpu().numpy(), E2.cpu().numpy()], 1)
    assert _rel(a, b) < 1e-12
    h.close()


def test_batch_reports_the_suspension_that_fails(pkg):
    """A suspension whose r_cut exceeds L/2 is named in the error."""
    with pytest.raises(pkg.PSEError) as e:
        pkg.PSE([100, 10], [16.2, 9.0], xi=XI, tol=EPS)
    assert e.value.code == 1 and 'suspension 1' in str(e.value)
