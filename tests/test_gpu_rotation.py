"""GPU parity of the 11-moment product [U; Omega; E] = M [F; L; S] (Sec. 2.2.1,
forces, torques and stresslets) through pse_mobility_apply11, against the FP64
oracle with identical parameters.

Tolerances as for the 8-moment product: relative L2 1e-10 (FP64 form) and 2e-5
(mixed form) per part and in total; the total within eps of the dense 11-moment
Ewald sum.  Also: restricted to [U; E] x [F; S] it equals pse_mobility_apply;
one-sided inputs (torques only); the full product is symmetric
(a . M b = b . M a); a handle without the torque option refuses the call.
"""
import numpy as np
import pytest

import pse_inputs
from oracle import ewald, params, pse as opse

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


def _cuda(x, dtype):
    return None if x is None else torch.tensor(np.ascontiguousarray(x), device='cuda', dtype=dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_params(h, N, L, xi, tol):
    inf = h.info
    return params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, Ng=inf['Ng'], P=inf['P'], rcut=inf['rcut'])


def _mob11(h, pos, F, Lt, S, prec, parts='all'):
    dt = _dt(prec)
    out = h.mobility11(_cuda(pos, torch.float64), _cuda(F, dt), _cuda(Lt, dt), _cuda(S, dt), parts=parts)
    return np.concatenate([o.double().cpu().numpy() for o in out], 1)


def _moments11(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, 3)), rng.standard_normal((N, 3)), rng.standard_normal((N, 5))


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
@pytest.mark.parametrize('N,phi,xi', [(100, 0.1, 0.5), (1500, 0.2, 0.6)])
def test_mobility11_parity(pkg, prec, N, phi, xi):
    """Per part and in total against the oracle; N = 1500 has a 40^3 grid (two full
    16^3 tiles and a ragged one per side) and many cells."""
    tol = 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=1)
    F, Lt, S = _moments11(N, 2)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, torque=1)
    p = _oracle_params(h, N, L, xi, tol)
    op = opse.RealOp(pos, p, torque=True)
    for parts in ('real', 'wave', 'all'):
        got = _mob11(h, pos, F, Lt, S, prec, parts)
        oparts = {'real': ('real',), 'wave': ('wave',), 'all': ('real', 'wave')}[parts]
        ref = np.concatenate(opse.mobility_apply11(pos, F, Lt, S, p, parts=oparts, real_op=op), 1)
        assert _rel(got, ref) < TOL[prec], (parts, _rel(got, ref))
    if N <= 100:
        M = ewald.dense_mobility(pos, L, xi=0.6, tol=1e-15, torque=True)
        ref = (M @ np.concatenate([F, Lt, S], 1).ravel()).reshape(N, 11)
        assert _rel(got, ref) < tol
    h.close()


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_mobility11_restricts_to_eight_and_one_sided(pkg, prec):
    N, phi, xi, tol = 500, 0.2, 0.6, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=3)
    F, Lt, S = _moments11(N, 4)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision=prec, torque=1)
    dt = _dt(prec)
    got = _mob11(h, pos, F, None, S, prec)
    U, E = h.mobility(_cuda(pos, torch.float64), _cuda(F, dt), _cuda(S, dt))
    ref8 = np.concatenate([U.double().cpu().numpy(), E.double().cpu().numpy()], 1)
    assert _rel(got[:, [0, 1, 2, 6, 7, 8, 9, 10]], ref8) < TOL[prec]
    # torques only
    p = _oracle_params(h, N, L, xi, tol)
    got = _mob11(h, pos, None, Lt, None, prec)
    ref = np.concatenate(opse.mobility_apply11(pos, 0 * F, Lt, 0 * S, p), 1)
    assert _rel(got, ref) < TOL[prec]
    h.close()


def test_mobility11_symmetric(pkg):
    N, phi, xi, tol = 3000, 0.3, 0.5, 1e-3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=5)
    a, b = np.concatenate(_moments11(N, 6), 1), np.concatenate(_moments11(N, 7), 1)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64', torque=1)
    Ma = _mob11(h, pos, a[:, :3], a[:, 3:6], a[:, 6:], 'fp64')
    Mb = _mob11(h, pos, b[:, :3], b[:, 3:6], b[:, 6:], 'fp64')
    lhs, rhs = float((b * Ma).sum()), float((a * Mb).sum())
    assert abs(lhs - rhs) < 1e-11 * np.linalg.norm(Ma) * np.linalg.norm(b)
    h.close()


def test_mobility11_needs_torque_option(pkg):
    N, L = 50, 12.0
    pos = pse_inputs.random_positions(N, L, seed=2)
    h = pkg.PSE(N, L, xi=1.0, tol=1e-3, precision='fp64')
    with pytest.raises(pkg.PSEError) as e:
        h.mobility11(_cuda(pos, torch.float64), _cuda(np.ones((N, 3)), torch.float64))
    assert e.value.code == 1
    h.close()
