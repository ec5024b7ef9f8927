"""GPU parity on deformed lattices (Sec. 2.3.3) against the FP64 oracle.

Handles created with a lattice deformation A (simple shear, planar extension,
a general A with det A != 1) run the general spreading / interpolation kernels
with non-separable Gaussian weights, the deformed wave vectors and the
Cartesian mapping in the neighbour search.  Compared with the oracle on the same
parameters and noise: the mobility product per part and in total, the
11-moment product, the Brownian sample and the constrained mid-point step
(FP64 1e-10 / 1e-9 for the step, mixed 2e-5); changing the strain of a handle
(pse_set_deformation) against a fresh oracle evaluation, and its refusals; the
step graph against the host-launched step; the product within eps of the dense
Ewald sum on the deformed lattice.
"""
import numpy as np
import pytest

import pse_inputs
from oracle import ewald, params, pse as opse

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

TOL = {'fp64': 1e-10, 'mixed': 2e-5}
GENERAL = np.array([[1.0, 0.2, 0.1], [0.0, 1.1, 0.15], [0.05, 0.0, 0.9]])
LATTICES = {'shear': params.shear_tensor(0.5), 'extension': params.extension_tensor(1.5), 'general': GENERAL}


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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_params(h, N, L, xi, tol, A):
    inf = h.info
    return params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, Ng=inf['Ng'], P=inf['P'], rcut=inf['rcut'], A=A)


def _mob(h, pos, F, S, prec, parts='all'):
    dt = _dt(prec)
    U, E = h.mobility(_cuda(pos, torch.float64), _cuda(F, dt), _cuda(S, dt), parts=parts)
    return np.concatenate([U.double().cpu().numpy(), E.double().cpu().numpy()], 1)


def _lattice_disp(x1, x0, A, L):
    """x1 - x0 reduced by lattice vectors L A n to the nearest image."""
    d = x1 - x0
    z = d @ np.linalg.inv(A).T
    z -= L * np.rint(z / L)
    return z @ A.T


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
@pytest.mark.parametrize('name', ['shear', 'extension', 'general'])
def test_mobility_deformed(pkg, prec, name):
    """N = 100 (phi = 0.1) and N = 1500 (phi = 0.3, several tiles and cells per side)."""
    A = LATTICES[name]
    for N, phi, seed in ((100, 0.1, 1), (1500, 0.3, 3)):
        xi, tol = 0.8, 1e-3
        pos, L = pse_inputs.rsa_positions(N, phi, seed=seed)
        F, S = pse_inputs.moments(N, seed=seed + 1)
        h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, deform=A)
        inf = h.info
        assert inf['deformed'] == 1 and np.allclose(inf['deform'], A)
        p = _oracle_params(h, N, L, xi, tol, A)
        op = opse.RealOp(pos, p)
        for parts in ('real', 'wave', 'all'):
            got = _mob(h, pos, F, S, prec, parts)
            oparts = {'real': ('real',), 'wave': ('wave',), 'all': ('real', 'wave')}[parts]
            Uo, Eo = opse.mobility_apply(pos, F, S, p, parts=oparts, real_op=op)
            assert _rel(got, np.concatenate([Uo, Eo], 1)) < TOL[prec], (N, parts)
        h.close()


def test_support_follows_lambda_max(pkg):
    """P from Eq. bound with lambda_max (option lambda_support) vs the orthorhombic rule."""
    N, phi = 1500, 0.3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=3)
    A = LATTICES['extension']
    for aware in (1, 0):
        h = pkg.PSE(N, L, xi=0.8, tol=1e-3, precision='mixed', deform=A, lambda_support=aware)
        p = params.choose(N, L, 1.0, 1.0, 1.0, 0.8, 1e-3, A=A, lambda_aware=bool(aware))
        assert h.info['P'] == p.P and h.info['Ng'] >= p.Ng and abs(h.info['rcut'] - p.rcut) < 1e-12
        h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_within_eps_of_dense_ewald_sheared(pkg, prec):
    N, phi, xi, tol = 100, 0.1, 0.7, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    F, S = pse_inputs.moments(N, seed=2)
    A = LATTICES['shear']
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, deform=A)
    got = _mob(h, pos, F, S, prec)
    M = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15, A=A)
    ref = (M @ np.concatenate([F, S], 1).ravel()).reshape(N, 8)
    assert _rel(got, ref) < tol
    h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_mobility11_deformed(pkg, prec):
    N, phi, xi, tol = 400, 0.2, 0.8, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=21)
    F, S = pse_inputs.moments(N, seed=22)
    Lt = pse_inputs.moments(N, seed=23)[0]
    A = LATTICES['shear']
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, deform=A, torque=1)
    p = _oracle_params(h, N, L, xi, tol, A)
    dt = _dt(prec)
    U, Om, E = h.mobility11(_cuda(pos, torch.float64), _cuda(F, dt), _cuda(Lt, dt), _cuda(S, dt))
    got = np.concatenate([U.double().cpu().numpy(), Om.double().cpu().numpy(), E.double().cpu().numpy()], 1)
    Uo, Oo, Eo = opse.mobility_apply11(pos, F, Lt, S, p)
    assert _rel(got, np.concatenate([Uo, Oo, Eo], 1)) < TOL[prec]
    h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_brownian_sample_deformed(pkg, prec):
    N, phi, xi, tol, dt = 300, 0.25, 0.8, 1e-3, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=31)
    A = LATTICES['shear']
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, deform=A, lanczos_tol=0.0, lanczos_maxiter=12)
    p = _oracle_params(h, N, L, xi, tol, A)
    w1 = pse_inputs.lanczos_noise(N, seed=32)
    w2 = pse_inputs.wave_noise(p.Ng, seed=33)
    U, E, st = h.brownian(_cuda(pos, torch.float64), dt, w1=_cuda(w1, _dt(prec)), w2=_cuda(w2, _dt(prec)))
    got = np.concatenate([U.double().cpu().numpy(), E.double().cpu().numpy()], 1)
    ref, _ = opse.brownian_sample(pos, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=12)
    assert _rel(got, ref) < TOL[prec]
    h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
@pytest.mark.parametrize('name', ['shear', 'general'])
def test_constrained_step_deformed(pkg, prec, name):
    N, phi, xi, tol, dt = 300, 0.2, 0.8, 1e-3, 1e-3
    A = LATTICES[name]
    pos, L = pse_inputs.rsa_positions(N, phi, seed=41)
    pos = pos @ A.T      # spread the particles over the deformed cell
    ktol = 1e-10 if prec == 'fp64' else 1e-6
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, deform=A, lanczos_tol=0.0, lanczos_maxiter=10,
                krylov_tol=ktol, krylov_maxiter=100)
    p = _oracle_params(h, N, L, xi, tol, A)
    w1 = pse_inputs.lanczos_noise(N, seed=42)
    w2 = pse_inputs.wave_noise(p.Ng, seed=43)
    FP = pse_inputs.moments(N, seed=44)[0] * 5.0
    x = _cuda(pos, torch.float64)
    S, st = h.step(x, dt, FP=_cuda(FP, _dt(prec)), w1=_cuda(w1, _dt(prec)), w2=_cuda(w2, _dt(prec)), want_S=True)
    x1, So, sto = opse.constrained_step(pos, FP, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=10,
                                        krylov_tol=1e-12, krylov_maxiter=200)
    xg = x.cpu().numpy()
    # the GPU wraps into the deformed cell as the oracle does
    zg = xg @ np.linalg.inv(A).T
    assert np.all(zg > -1e-9) and np.all(zg < L + 1e-9)
    disp_o = _lattice_disp(x1, pos, A, L)
    disp_g = _lattice_disp(xg, pos, A, L)
    assert _rel(disp_g, disp_o) < (1e-9 if prec == 'fp64' else 2e-5)
    assert _rel(S.double().cpu().numpy(), So) < (1e-9 if prec == 'fp64' else 2e-5)
    assert 1 <= st['krylov_iters'] <= 100
    h.close()


def test_set_deformation(pkg):
    """A handle created at strain 1/2 evaluated at strain 0.2 and -0.3 equals the oracle with the
    handle's parameters at those strains; a strain beyond the handle's support or cells is refused."""
    N, phi, xi, tol = 1500, 0.3, 0.8, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=3)
    F, S = pse_inputs.moments(N, seed=4)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64', deform=params.shear_tensor(0.5))
    for g in (0.2, -0.3, 0.0):
        A = params.shear_tensor(g)
        h.set_deformation(A)
        assert np.allclose(h.info['deform'], A)
        p = _oracle_params(h, N, L, xi, tol, A)
        got = _mob(h, pos, F, S, 'fp64')
        Uo, Eo = opse.mobility_apply(pos, F, S, p)
        assert _rel(got, np.concatenate([Uo, Eo], 1)) < TOL['fp64'], g
    for bad in (params.shear_tensor(0.8), params.extension_tensor(1.2)):
        with pytest.raises(pkg.binding.PSEError):
            h.set_deformation(bad)
    h.close()
    hc = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64')
    with pytest.raises(pkg.binding.PSEError):
        hc.set_deformation(params.shear_tensor(0.1))
    hc.close()


def test_graph_step_equals_host_step_deformed(pkg):
    N, phi, xi, tol, dt = 2000, 0.3, 0.8, 1e-3, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=51)
    A = LATTICES['shear']
    he = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', deform=A)
    hg = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', deform=A, use_graph=1)
    xe = _cuda(pos, torch.float64)
    xg = xe.clone()
    for k in range(3):
        he.step(xe, dt, seed=7, step=k)
        hg.step(xg, dt, seed=7, step=k)
        assert hg.graph_ready() == (True, '')
        de = _lattice_disp(xe.cpu().numpy(), pos, A, L)
        dg = _lattice_disp(xg.cpu().numpy(), pos, A, L)
        assert _rel(dg, de) < 1e-5
    he.close()
    hg.close()


@pytest.mark.parametrize('name', ['shear', 'extension'])
def test_sedimentation_error_follows_support_rule(pkg, name):
    """The comparison of Fig. fig:shear on the GPU: the sedimentation velocity (equal forces on all
    particles) against the dense Ewald sum on the deformed lattice is within the tolerance with the
    lambda_max-aware support, and worse with the orthorhombic rule (for lambda_max = 2.25 by more
    than an order of magnitude past the tolerance)."""
    N, phi, xi, tol = 100, 0.1, 0.7, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    A = LATTICES[name]
    F = np.tile([0.0, 0.0, 1.0], (N, 1))
    M = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15, A=A)
    ref = (M @ np.concatenate([F, np.zeros((N, 5))], 1).ravel()).reshape(N, 8)[:, :3]
    errs = {}
    for aware in (1, 0):
        h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64', deform=A, lambda_support=aware)
        U, _ = h.mobility(_cuda(pos, torch.float64), _cuda(F, torch.float64), None)
        errs[aware] = _rel(U.cpu().numpy(), ref)
        h.close()
    assert errs[1] < tol
    assert errs[0] > 3 * errs[1]
    if name == 'extension':
        assert errs[0] > 10 * tol


@pytest.mark.parametrize('Ng,cell', [(48, 'shear'), (64, 'shear'), (48, 'cube')])
def test_tile_kernels_with_ten_point_support(pkg, Ng, cell):
    """Mixed precision with 16^3 tiles and P = 10 (the support Eq. bound gives on a cell sheared by
    1/2; for the cube set explicitly): the register-column spreading and the staged-region
    interpolation, with the x-y coupled weights on the sheared cell and weights formed per lane
    beyond 8 support points; the full product's interpolation (whose 8-component staging does not
    fit) runs as two passes of 5 and 3 components.  Products per part, E and U from S alone, and the step
    against the oracle at 2e-5."""
    N, phi, xi, tol, dt = 3000, 0.3, 0.6, 1e-3, 1e-3
    A = LATTICES['shear'] if cell == 'shear' else np.eye(3)
    pos, L = pse_inputs.rsa_positions(N, phi, seed=61)
    pos = pos @ A.T
    F, S = pse_inputs.moments(N, seed=62)
    kw = dict(deform=A) if cell == 'shear' else dict(P=10)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed', Ng=Ng, lanczos_tol=0.0, lanczos_maxiter=8,
                krylov_tol=1e-6, krylov_maxiter=100, **kw)
    assert h.info['P'] == 10 and h.info['tile_kernels'] == 1
    if cell == 'cube':
        A = None
    p = _oracle_params(h, N, L, xi, tol, A)
    op = opse.RealOp(pos, p)
    for parts in ('wave', 'all'):
        got = _mob(h, pos, F, S, 'mixed', parts)
        Uo, Eo = opse.mobility_apply(pos, F, S, p, parts=('wave',) if parts == 'wave' else ('real', 'wave'),
                                     real_op=op)
        assert _rel(got, np.concatenate([Uo, Eo], 1)) < TOL['mixed'], parts
    # E from S alone and U from S alone take the 5- and 3-component kernels
    U, E = h.mobility(_cuda(pos, torch.float64), None, _cuda(S, torch.float32))
    Uo, Eo = opse.mobility_apply(pos, np.zeros((N, 3)), S, p, real_op=op)
    assert _rel(E.double().cpu().numpy(), Eo) < TOL['mixed']
    assert _rel(U.double().cpu().numpy(), Uo) < TOL['mixed']
    w1 = pse_inputs.lanczos_noise(N, seed=63)
    w2 = pse_inputs.wave_noise(p.Ng, seed=64)
    x = _cuda(pos, torch.float64)
    Sg, st = h.step(x, dt, w1=_cuda(w1, torch.float32), w2=_cuda(w2, torch.float32), want_S=True)
    x1, So, _ = opse.constrained_step(pos, None, dt, w1, w2, p, lanczos_tol=0.0, lanczos_maxiter=8,
                                      krylov_tol=1e-12, krylov_maxiter=200)
    Ad = np.eye(3) if A is None else A
    assert _rel(_lattice_disp(x.cpu().numpy(), pos, Ad, L), _lattice_disp(x1, pos, Ad, L)) < 2e-5
    assert _rel(Sg.double().cpu().numpy(), So) < 2e-5
    h.close()
