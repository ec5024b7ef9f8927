"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative L2 over all outputs): 1e-10 for the FP64 form and 2e-5
for the mixed form against the oracle PSE with identical parameters and
identical noise; both forms within the PSE tolerance eps of the dense Ewald
sum.  Sizes span several spreading tiles and cells; edge cases cover a single
particle, overlapping pairs, positions outside the box, one-sided inputs,
boxes with fewer than five cells per side and even/odd support sizes.
"""
import math

import numpy as np
import pytest

import pse_inputs
from oracle import ewald, params, philox, pse as opse

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL = {'fp64': 1e-10, 'mixed': 2e-5}


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


def _cuda(x, dtype=None):
    return torch.tensor(np.ascontiguousarray(x), device='cuda', dtype=dtype)


def _oracle_params(h, N, L, xi, tol, **kw):
    inf = h.info
    return params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, Ng=inf['Ng'], P=inf['P'], rcut=inf['rcut'], **kw)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _mob(pkg, h, pos, F, S, prec, parts='all'):
    dt = _dt(prec)
    U, E = h.mobility(_cuda(pos, torch.float64), None if F is None else _cuda(F, dt),
                      None if S is None else _cuda(S, dt), parts=parts)
    return np.concatenate([U.double().cpu().numpy(), E.double().cpu().numpy()], 1)


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_mobility_config1(pkg, prec):
    """N=100, phi=0.1, eps=1e-3 (RSA); parity per part and in total, and within eps of Ewald."""
    N, phi, xi, tol = 100, 0.1, 0.5, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec)
    p = _oracle_params(h, N, L, xi, tol)
    op = opse.RealOp(pos, p)
    for parts in ('real', 'wave', 'all'):
        got = _mob(pkg, h, pos, F, S, prec, parts)
        oparts = {'real': ('real',), 'wave': ('wave',), 'all': ('real', 'wave')}[parts]
        Uo, Eo = opse.mobility_apply(pos, F, S, p, parts=oparts, real_op=op)
        assert _rel(got, np.concatenate([Uo, Eo], 1)) < TOL[prec], parts
    M = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15)
    ref = (M @ np.concatenate([F, S], 1).ravel()).reshape(N, 8)
    assert _rel(got, ref) < tol
    h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_mobility_dense_many_tiles(pkg, prec):
    """N=3000 at phi=0.3: several spreading tiles per side and many cells."""
    N, phi, xi, tol = 3000, 0.3, 0.7, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=5)
    F, S = pse_inputs.moments(N, seed=6)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, tile=(8, 8, 8))
    p = _oracle_params(h, N, L, xi, tol)
    assert h.info['Ng'] // 8 >= 3 and h.info['cells_per_side'] >= 3
    got = _mob(pkg, h, pos, F, S, prec)
    Uo, Eo = opse.mobility_apply(pos, F, S, p)
    assert _rel(got, np.concatenate([Uo, Eo], 1)) < TOL[prec]
    h.close()


@pytest.mark.parametrize('tol,Ng,N,xi', [(1e-2, 48, 3000, 0.7), (1e-3, 48, 3000, 0.7), (1e-4, 64, 3000, 0.7),
                                         (1e-3, 32, 1500, 0.5)])
def test_mobility_cubic_tiles(pkg, tol, Ng, N, xi):
    """Mixed precision with 16^3 spreading tiles (the kernels specialised for
    them: column spreading with staged-region interpolation by default, shared-tile
    spreading with column interpolation (wave_kernel=3) and the tile-owned
    interpolation (wave_kernel=16)) against the oracle and against the general kernels (16 x 8 x
    16 tiles); supports of several sizes, and two tiles per side (N_g = 32: the
    tile below and the tile above are the same).  Full product and the reduced
    products (S -> E, S -> U, [F; S] -> U) whose spreading takes 5 or 8
    components."""
    phi = 0.3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=11)
    F, S = pse_inputs.moments(N, seed=12)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', Ng=Ng)
    assert tuple(h.info['tile']) == (16, 16, 16) and h.info['Ng'] == Ng
    hs = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', Ng=Ng, wave_kernel=3)
    ht = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', Ng=Ng, wave_kernel=16)
    hg = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', Ng=Ng, tile=(16, 8, 16))
    assert hg.info['Ng'] == h.info['Ng'] and hg.info['P'] == h.info['P']
    p = _oracle_params(h, N, L, xi, tol)
    got = _mob(pkg, h, pos, F, S, 'mixed')
    shared = _mob(pkg, hs, pos, F, S, 'mixed')
    towned = _mob(pkg, ht, pos, F, S, 'mixed')
    gen = _mob(pkg, hg, pos, F, S, 'mixed')
    Uo, Eo = opse.mobility_apply(pos, F, S, p)
    assert _rel(got, np.concatenate([Uo, Eo], 1)) < TOL['mixed']
    assert _rel(got, gen) < 5e-6 and _rel(shared, gen) < 5e-6 and _rel(towned, gen) < 5e-6
    x, tF, tS = _cuda(pos, torch.float64), _cuda(F, torch.float32), _cuda(S, torch.float32)
    for want, FF in ((('E',), None), (('U',), None), (('U',), tF)):
        Fo = F if FF is not None else 0 * F
        Uo, Eo = opse.mobility_apply(pos, Fo, S, p, parts=('wave',))
        for hh in (h, hs, ht):
            U, E = hh.mobility(x, FF, tS, parts='wave', want=want)
            out, ref = (E, Eo) if want == ('E',) else (U, Uo)
            assert _rel(out.double().cpu().numpy(), ref) < TOL['mixed'], (want, FF is None)
    h.close()
    hs.close()
    ht.close()
    hg.close()


@pytest.mark.parametrize('Ng,N,xi', [(48, 3000, 0.7), (32, 1500, 0.5)])
@pytest.mark.parametrize('with_force', [False, True])
def test_cubic_tiles_sample_and_step(pkg, Ng, N, xi, with_force):
    """The 16^3-tile kernel instances of the benchmark step (mixed precision,
    P = 6 at eps = 1e-3): the 8-component noise interpolation of the Brownian
    sample, the 5-component spread and interpolation of every GMRES product, and
    the final S -> U product ([F; S] -> U and the 8-component EF product with a
    force); sample, displacement and stresslets against the oracle with the same
    external noise.  N_g = 48 has three tiles per side, N_g = 32 two (the tile
    below and the tile above are the same)."""
    phi, tol, dt = 0.3, 1e-3, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=11)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', Ng=Ng, lanczos_tol=0.0, lanczos_maxiter=10,
                krylov_tol=1e-6, krylov_maxiter=100)
    assert tuple(h.info['tile']) == (16, 16, 16) and h.info['Ng'] == Ng and h.info['P'] == 6
    p = _oracle_params(h, N, L, xi, tol)
    w1 = pse_inputs.lanczos_noise(N, seed=14)
    w2 = pse_inputs.wave_noise(p.Ng, seed=15)
    x = _cuda(pos, torch.float64)
    U, E, _ = h.brownian(x, dt, w1=_cuda(w1, torch.float32), w2=_cuda(w2, torch.float32))
    B, _ = opse.brownian_sample(pos, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=10)
    got = np.concatenate([U.double().cpu().numpy(), E.double().cpu().numpy()], 1)
    assert _rel(got, B) < TOL['mixed']
    FP = pse_inputs.moments(N, seed=16)[0] * 5.0 if with_force else None
    S, st = h.step(x, dt, FP=None if FP is None else _cuda(FP, torch.float32), w1=_cuda(w1, torch.float32),
                   w2=_cuda(w2, torch.float32), want_S=True)
    x1, So, _ = opse.constrained_step(pos, FP, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=10,
                                      krylov_tol=1e-12, krylov_maxiter=200)
    disp_o = x1 - pos
    disp_o -= L * np.rint(disp_o / L)
    disp_g = x.cpu().numpy() - pos
    disp_g -= L * np.rint(disp_g / L)
    assert _rel(disp_g, disp_o) < TOL['mixed']
    assert _rel(S.double().cpu().numpy(), So) < TOL['mixed']
    assert 1 <= st['krylov_iters'] <= 100
    h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_edge_cases(pkg, prec):
    # single particle: only self terms and its periodic images (wave space)
    L = 12.0
    pos = np.array([[1.0, 11.5, 6.0]])
    F, S = pse_inputs.moments(1, seed=3)
    h = pkg.PSE(1, L, xi=0.9, tol=1e-3, precision=prec)
    p = _oracle_params(h, 1, L, 0.9, 1e-3)
    Uo, Eo = opse.mobility_apply(pos, F, S, p)
    assert _rel(_mob(pkg, h, pos, F, S, prec), np.concatenate([Uo, Eo], 1)) < TOL[prec]
    h.close()
    # overlapping pairs, positions outside [0, L), tiny box (< 3 cells), even support, one-sided inputs
    N, L = 40, 8.0
    rng = np.random.default_rng(7)
    pos = rng.uniform(-L, 2 * L, (N, 3))
    pos[1] = pos[0] + np.array([0.9, 0.3, -0.2])          # deep overlap r ~ 0.97a
    pos[2] = pos[0] + np.array([2.0, 0.0, 0.0])           # exact contact
    F, S = pse_inputs.moments(N, seed=8)
    for tol, rule in ((1e-3, 'paper'), (1e-4, 'paper')):
        h = pkg.PSE(N, L, xi=0.8, tol=tol, precision=prec, rule=rule)
        assert h.info["cells_per_side"] < 5
        p = _oracle_params(h, N, L, 0.8, tol, rule=rule)
        Uo, Eo = opse.mobility_apply(pos, F, S, p)
        assert _rel(_mob(pkg, h, pos, F, S, prec), np.concatenate([Uo, Eo], 1)) < TOL[prec]
        Uo, Eo = opse.mobility_apply(pos, F, 0 * S, p)
        assert _rel(_mob(pkg, h, pos, F, None, prec), np.concatenate([Uo, Eo], 1)) < TOL[prec]
        Uo, Eo = opse.mobility_apply(pos, 0 * F, S, p)
        assert _rel(_mob(pkg, h, pos, None, S, prec), np.concatenate([Uo, Eo], 1)) < TOL[prec]
        h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_mobility_partial_outputs(pkg, prec):
    """Requests for a part of the outputs take the reduced products: U from S
    alone, U from [F; S], E from S alone; each against the oracle."""
    N, phi, xi, tol = 300, 0.2, 0.6, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=17)
    F, S = pse_inputs.moments(N, seed=18)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec)
    p = _oracle_params(h, N, L, xi, tol)
    dt = _dt(prec)
    x = _cuda(pos, torch.float64)
    Uo, _ = opse.mobility_apply(pos, 0 * F, S, p)
    U, E = h.mobility(x, None, _cuda(S, dt), want=('U',))
    assert E is None and _rel(U.double().cpu().numpy(), Uo) < TOL[prec]
    Uo, _ = opse.mobility_apply(pos, F, S, p)
    U, _ = h.mobility(x, _cuda(F, dt), _cuda(S, dt), want=('U',))
    assert _rel(U.double().cpu().numpy(), Uo) < TOL[prec]
    _, Eo = opse.mobility_apply(pos, 0 * F, S, p)
    _, E = h.mobility(x, None, _cuda(S, dt), want=('E',))
    assert _rel(E.double().cpu().numpy(), Eo) < TOL[prec]
    h.close()


def test_host_arrays_through_the_abi(pkg):
    """numpy (host) arrays are staged by the library and give the same result."""
    N, phi, xi, tol = 100, 0.1, 0.5, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64')
    U, E = h.mobility(pos, F, S)
    got = _mob(pkg, h, pos, F, S, 'fp64')
    assert np.abs(np.concatenate([U, E], 1) - got).max() < 1e-14 * np.abs(got).max()
    h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_brownian_sample_external_noise(pkg, prec):
    N, phi, xi, tol, dt = 200, 0.2, 0.6, 1e-3, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=9)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, lanczos_tol=0.0, lanczos_maxiter=12)
    p = _oracle_params(h, N, L, xi, tol)
    w1 = pse_inputs.lanczos_noise(N, seed=10)
    w2 = pse_inputs.wave_noise(p.Ng, seed=11)
    U, E, st = h.brownian(_cuda(pos, torch.float64), dt, w1=_cuda(w1, _dt(prec)), w2=_cuda(w2, _dt(prec)))
    B, sto = opse.brownian_sample(pos, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=12)
    assert st['lanczos_iters'] == 12 and sto['lanczos_iters'] == 12
    got = np.concatenate([U.double().cpu().numpy(), E.double().cpu().numpy()], 1)
    assert _rel(got, B) < TOL[prec]


def test_long_lanczos_recurrence(pkg):
    """60 Lanczos steps (FP64): the tridiagonal square root is taken by one warp
    with the eigenvectors in shared memory up to 48 rows and by one thread
    beyond; both against the oracle's Lanczos with the same fixed length."""
    N, phi, xi, tol, dt = 200, 0.2, 0.6, 1e-3, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=29)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64', lanczos_tol=0.0, lanczos_maxiter=60)
    p = _oracle_params(h, N, L, xi, tol)
    w1 = pse_inputs.lanczos_noise(N, seed=30)
    w2 = pse_inputs.wave_noise(p.Ng, seed=31)
    U, E, st = h.brownian(_cuda(pos, torch.float64), dt, w1=_cuda(w1, torch.float64), w2=_cuda(w2, torch.float64))
    B, sto = opse.brownian_sample(pos, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=60)
    assert st['lanczos_iters'] == 60 and sto['lanczos_iters'] == 60
    got = np.concatenate([U.cpu().numpy(), E.cpu().numpy()], 1)
    assert _rel(got, B) < TOL['fp64']
    h.close()


def test_in_kernel_noise_matches_published_generator(pkg):
    """In-kernel Philox4x32-10 noise equals the same stream generated by the oracle."""
    N, phi, xi, tol, dt = 150, 0.15, 0.6, 1e-3, 1e-2
    pos, L = pse_inputs.rsa_positions(N, phi, seed=12)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64', lanczos_tol=1e-12)
    Ng = h.info['Ng']
    seed, counter = 0x1234567890ABCDEF, 77
    U, E, _ = h.brownian(_cuda(pos, torch.float64), dt, seed=seed, counter=counter)
    w1 = philox.lanczos_noise(seed, counter, N)
    w2 = philox.wave_noise(seed, counter, Ng)
    U2, E2, _ = h.brownian(_cuda(pos, torch.float64), dt, w1=_cuda(w1, torch.float64), w2=_cuda(w2, torch.float64))
    a = np.concatenate([U.cpu().numpy(), E.cpu().numpy()], 1)
    b = np.concatenate([U2.cpu().numpy(), E2.cpu().numpy()], 1)
    assert _rel(a, b) < 1e-12


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
@pytest.mark.parametrize('with_force', [False, True])
def test_constrained_step(pkg, prec, with_force):
    N, phi, xi, tol, dt = 150, 0.2, 0.7, 1e-3, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=13)
    ktol = 1e-10 if prec == 'fp64' else 1e-6
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, lanczos_tol=0.0, lanczos_maxiter=10, krylov_tol=ktol,
                krylov_maxiter=100)
    p = _oracle_params(h, N, L, xi, tol)
    w1 = pse_inputs.lanczos_noise(N, seed=14)
    w2 = pse_inputs.wave_noise(p.Ng, seed=15)
    FP = pse_inputs.moments(N, seed=16)[0] * 5.0 if with_force else None
    x = _cuda(pos, torch.float64)
    S, st = h.step(x, dt, FP=None if FP is None else _cuda(FP, _dt(prec)), w1=_cuda(w1, _dt(prec)),
                   w2=_cuda(w2, _dt(prec)), want_S=True)
    x1, So, sto = opse.constrained_step(pos, FP, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=10,
                                        krylov_tol=1e-12, krylov_maxiter=200)
    disp_o = x1 - pos
    disp_o -= L * np.rint(disp_o / L)
    disp_g = x.cpu().numpy() - pos
    disp_g -= L * np.rint(disp_g / L)
    assert _rel(disp_g, disp_o) < (1e-9 if prec == 'fp64' else 2e-5)
    assert _rel(S.double().cpu().numpy(), So) < (1e-9 if prec == 'fp64' else 2e-5)
    assert 1 <= st['krylov_iters'] <= 100


def test_step_internal_noise_is_reproducible(pkg):
    N, phi, xi, tol = 300, 0.25, 0.7, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=17)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed')
    xa = _cuda(pos, torch.float64)
    xb = _cuda(pos, torch.float64)
    _, sa = h.step(xa, 1e-3, seed=5, step=3)
    _, sb = h.step(xb, 1e-3, seed=5, step=3)
    assert torch.max(torch.abs(xa - xb)).item() < 1e-6
    assert 1 <= sa['lanczos_iters'] <= 100 and 1 <= sa['krylov_iters'] <= 50
    d = (xa.cpu().numpy() - pos)
    d -= L * np.rint(d / L)
    assert 0 < np.abs(d).max() < 0.5


def test_nonfinite_input_rejected(pkg):
    N, L = 20, 12.0
    pos = pse_inputs.random_positions(N, L, seed=2)
    pos[3, 1] = np.nan
    h = pkg.PSE(N, L, xi=1.0, tol=1e-3, precision='mixed')
    with pytest.raises(pkg.PSEError) as e:
        h.mobility(_cuda(pos, torch.float64), _cuda(np.ones((N, 3)), torch.float32))
    assert e.value.code == 5
    h.close()


@pytest.mark.parametrize('prec', ['mixed'])
def test_full_size_sampled(pkg, prec):
    """N = 1,048,576 at phi = 0.3, eps = 1e-3 (the benchmark workload, launch as in bench.py):
    wave part against the oracle's NUFFT at full size, real part on sampled
    particles, symmetry u.Mv = v.Mu of the full product."""
    from scipy.spatial import cKDTree
    from oracle import realspace as R
    N, phi, xi, tol = 1048576, 0.3, 0.5, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec)
    p = _oracle_params(h, N, L, xi, tol)
    wave = _mob(pkg, h, pos, F, S, prec, 'wave')
    w = opse.wave_apply(pos, F, S, p)
    assert _rel(wave, np.concatenate([w['U'], w['E']], 1)) < TOL[prec]
    real = _mob(pkg, h, pos, F, S, prec, 'real')
    idx = np.random.default_rng(3).choice(N, 64, replace=False)
    tree = cKDTree(np.mod(pos, L), boxsize=L)
    v = np.concatenate([F, S], 1)
    ref = np.zeros((idx.size, 8))
    selfb = R.self_block(xi, 1.0, 1.0)
    for n, i in enumerate(idx):
        nb = np.array([j for j in tree.query_ball_point(pos[i], p.rcut) if j != i])
        d = pos[i] - pos[nb]
        d -= L * np.rint(d / L)
        B = R.pair_blocks(d, xi, 1.0, 1.0)
        ref[n] = selfb @ v[i] + np.einsum('pab,pb->a', B, v[nb])
    assert _rel(real[idx], ref) < TOL[prec]
    # symmetry of the whole operator at full size
    rng = np.random.default_rng(4)
    u = rng.standard_normal((N, 8))
    Mu = _mob(pkg, h, pos, u[:, :3], u[:, 3:], prec)
    Mv = _mob(pkg, h, pos, F, S, prec)
    assert abs(np.sum(u * Mv) - np.sum(v * Mu)) < 1e-5 * abs(np.sum(v * Mv))
    h.close()


def _sampled_real(pos, L, p, v, idx):
    """Oracle real-space rows idx of M_r v (pair sum over the particles within r_cut, plus self)."""
    from scipy.spatial import cKDTree
    from oracle import realspace as R
    tree = cKDTree(np.mod(pos, L), boxsize=L)
    ref = np.zeros((idx.size, 8))
    selfb = R.self_block(p.xi, 1.0, 1.0)
    x = np.mod(pos, L)
    for n, i in enumerate(idx):
        nb = np.array([j for j in tree.query_ball_point(x[i], p.rcut) if j != i])
        d = x[i] - x[nb]
        d -= L * np.rint(d / L)
        ref[n] = selfb @ v[i] + np.einsum('pab,pb->a', R.pair_blocks(d, p.xi, 1.0, 1.0), v[nb])
    return ref


def test_full_size_sample_and_step(pkg):
    """N = 1,048,576 at phi = 0.3, eps = 1e-3 with the benchmark's parameters (N_g = 256,
    P = 6, 16^3 tiles), mixed precision, external noise:
    * Brownian sample: the wave-space noise (the sample minus its part with w2 = 0)
      against the oracle in full; the Lanczos real-space noise (w2 = 0) through
      ||y||^2 = w1 . M_r w1, with M_r w1 from
      the real-space product, itself checked against the oracle on sampled rows;
    * constrained step: the slip equals the sample drawn with the same noise; at the
      mid-point x_{k+1/2} = x_k + dt/2 U^B the returned stresslets satisfy the
      constraint, M_ES S = -E^B within the GMRES residual, and the displacement is
      dt (U^B + M_US S), with M(x_{k+1/2}) [0; S] computed by the full product, whose
      wave part is checked against the oracle in full and whose real part on sampled rows."""
    N, phi, xi, tol, dt = 1048576, 0.3, 0.5, 1e-3, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', lanczos_tol=1e-6, krylov_tol=1e-5, krylov_maxiter=50)
    assert tuple(h.info['tile']) == (16, 16, 16) and h.info['Ng'] == 256 and h.info['P'] == 6
    p = _oracle_params(h, N, L, xi, tol)
    w1 = pse_inputs.lanczos_noise(N, seed=3)
    w2 = pse_inputs.wave_noise(p.Ng, seed=4)
    x = _cuda(pos, torch.float64)
    scale = math.sqrt(2.0 / dt)
    tw1, tw2 = _cuda(w1, torch.float32), _cuda(w2, torch.float32)
    UB, EB, _ = h.brownian(x, dt, w1=tw1, w2=tw2)
    UB, EB = UB.double().cpu().numpy(), EB.double().cpu().numpy()
    Ur, Er, st = h.brownian(x, dt, w1=tw1, w2=torch.zeros_like(tw2))
    y = np.concatenate([Ur.double().cpu().numpy(), Er.double().cpu().numpy()], 1) / scale
    # wave-space noise: the sample minus its real-space part
    wave = np.concatenate([UB, EB], 1) - scale * y
    assert _rel(wave, scale * opse.wave_noise(pos, w2, p)) < TOL['mixed']
    # real-space noise: ||M_r^{1/2} w1||^2 = w1 . M_r w1
    Mw = _mob(pkg, h, pos, w1[:, :3], w1[:, 3:], 'mixed', 'real')
    idx = np.random.default_rng(5).choice(N, 64, replace=False)
    assert _rel(Mw[idx], _sampled_real(pos, L, p, w1, idx)) < TOL['mixed']
    quad = float(np.sum(w1 * Mw))
    assert abs(float(np.sum(y * y)) - quad) < 1e-4 * quad, st
    # the step with the same noise
    S, st = h.step(x, dt, w1=tw1, w2=tw2, want_S=True)
    S = S.double().cpu().numpy()
    xh = np.mod(pos + 0.5 * dt * UB, L)
    US, ES = (a.double().cpu().numpy() for a in h.mobility(_cuda(xh, torch.float64), torch.zeros((N, 3), device='cuda'),
                                                           _cuda(S, torch.float32)))
    assert np.linalg.norm(ES + EB) < 10 * max(st['krylov_relres'], 1e-5) * np.linalg.norm(EB), st
    disp = x.cpu().numpy() - pos
    disp -= L * np.rint(disp / L)
    assert _rel(disp, dt * (UB + US)) < TOL['mixed']
    zero3 = np.zeros((N, 3))
    wave = _mob(pkg, h, xh, zero3, S, 'mixed', 'wave')
    wo = opse.wave_apply(xh, zero3, S, p)
    assert _rel(wave, np.concatenate([wo['U'], wo['E']], 1)) < TOL['mixed']
    real = _mob(pkg, h, xh, zero3, S, 'mixed', 'real')
    v = np.concatenate([zero3, S], 1)
    assert _rel(real[idx], _sampled_real(xh, L, p, v, idx)) < TOL['mixed']
    h.close()
