"""Config 2 of the workload list: FP64 constrained steps with pairwise
hard-sphere repulsion, read as a harmonic overlap force F = k (2a - r) rh with
k = 1000 kT/a^2 (the paper leaves the repulsion unspecified).

The force is checked against its definition by brute force; one step with the
force against the oracle (N = 1000, where the oracle takes seconds); and a
100-step trajectory at N = 10,000, phi = 0.3 through its invariants (finite,
overlaps held in check, iteration counts, mean-square displacement in the
range of hindered self-diffusion)."""
import math

import numpy as np
import pytest

import pse_inputs
from oracle import params, pse as opse

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu
KSPRING = 1000.0


@pytest.fixture(scope='module')
def pkg():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import paper_1709_06946_gb300 as p
    p.build()
    p.load()
    return p


def brute_force(pos, L, k, a=1.0):
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    with np.errstate(invalid="ignore", divide="ignore"):
        c = np.where(r < 2 * a, k * (2 * a - r) / r, 0.0)
    return (c[:, :, None] * d).sum(1)


@pytest.mark.parametrize('prec', ['fp64', 'mixed'])
def test_overlap_force_matches_definition(pkg, prec):
    N, L = 600, 16.0
    pos = pse_inputs.random_positions(N, L, seed=150)      # many overlapping pairs
    h = pkg.PSE(N, L, xi=0.5, tol=1e-3, precision=prec)
    F = h.overlap_force(torch.tensor(pos, device='cuda', dtype=torch.float64), KSPRING)
    ref = brute_force(pos, L, KSPRING)
    err = np.linalg.norm(F.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < (1e-12 if prec == 'fp64' else 1e-5)
    h.close()


def test_first_step_with_repulsion_matches_oracle(pkg):
    N, phi, xi, tol, dt = 1000, 0.3, 0.5, 1e-3, 1e-3
    L = pse_inputs.box_length(N, phi)
    pos = pse_inputs.random_positions(N, L, seed=151)       # overlaps, so the force matters
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64', lanczos_tol=0.0, lanczos_maxiter=10, krylov_tol=1e-10,
                krylov_maxiter=100)
    inf = h.info
    p = params.choose(N, L, 1.0, 1.0, 1.0, xi, tol, Ng=inf['Ng'], P=inf['P'], rcut=inf['rcut'])
    w1 = pse_inputs.lanczos_noise(N, seed=152)
    w2 = pse_inputs.wave_noise(p.Ng, seed=153)
    x = torch.tensor(pos, device='cuda', dtype=torch.float64)
    F = h.overlap_force(x, KSPRING)
    h.step(x, dt, FP=F, w1=torch.tensor(w1, device='cuda'), w2=torch.tensor(w2, device='cuda'))
    x1, _, _ = opse.constrained_step(pos, brute_force(pos, L, KSPRING), dt, w1, w2, p, lanczos_tol=0.0,
                                     lanczos_maxiter=10, krylov_tol=1e-12, krylov_maxiter=200)
    d_o = x1 - pos
    d_g = x.cpu().numpy() - pos
    d_o -= L * np.rint(d_o / L)
    d_g -= L * np.rint(d_g / L)
    assert np.linalg.norm(d_g - d_o) / np.linalg.norm(d_o) < 1e-9
    h.close()


def test_config2_trajectory(pkg):
    N, phi, xi, tol, dt, steps = 10000, 0.3, 0.5, 1e-3, 1e-3, 100
    pos, L = pse_inputs.rsa_positions(N, phi, seed=154)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='fp64', use_graph=1)
    x = torch.tensor(pos, device='cuda', dtype=torch.float64)
    unwrapped = pos.copy()
    prev = pos.copy()
    kry = []
    for k in range(steps):
        F = h.overlap_force(x, KSPRING)
        _, st = h.step(x, dt, FP=F, seed=2024, step=k)
        kry.append(st['krylov_iters'])
        cur = x.cpu().numpy()
        d = cur - prev
        d -= L * np.rint(d / L)
        unwrapped += d
        prev = cur
    assert np.isfinite(unwrapped).all()
    assert 1 <= min(kry) and max(kry) <= 50
    msd = float(np.mean(np.sum((unwrapped - pos) ** 2, 1)))
    free = 6.0 / (6.0 * math.pi) * dt * steps               # 6 D0 t with D0 = kT / (6 pi eta a)
    assert 0.3 * free < msd < 1.0 * free                    # hindered self-diffusion at phi = 0.3
    from scipy.spatial import cKDTree
    dmin = cKDTree(np.mod(prev, L), boxsize=L).query(np.mod(prev, L), k=2)[0][:, 1].min()
    assert dmin > 1.8                                       # the repulsion keeps overlaps shallow
    h.close()


def test_krylov_caps_report_not_converged(pkg):
    """A GMRES cap of one iteration and a Lanczos cap of two (with a tolerance
    that cannot be met) complete the step and report NOT_CONVERGED (4)."""
    N, phi = 800, 0.3
    pos, L = pse_inputs.rsa_positions(N, phi, seed=155)
    h = pkg.PSE(N, L, xi=0.5, tol=1e-3, precision='mixed', krylov_maxiter=1, krylov_tol=1e-12)
    x = torch.tensor(pos, device='cuda', dtype=torch.float64)
    _, st = h.step(x, 1e-3, seed=1, step=0)
    assert st['status'] == 4 and st['krylov_iters'] == 1
    with pytest.raises(pkg.PSEError) as e:
        h.step(x, 1e-3, seed=1, step=1, allow_cap=False)
    assert e.value.code == 4
    h.close()
    h = pkg.PSE(N, L, xi=0.5, tol=1e-3, precision='mixed', lanczos_maxiter=2, lanczos_tol=1e-14)
    _, st = h.step(x, 1e-3, seed=1, step=0)
    assert st['status'] == 4 and st['lanczos_iters'] == 2
    h.close()
