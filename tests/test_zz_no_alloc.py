"""GPU test of pse_mobility_real_noalloc, the entry point for callers that cannot
allocate device memory (codes that must not let cudaMalloc/cudaFree synchronise
the device inside their loop, or whose device memory belongs to their own pool
allocator).  It must reproduce the real-space product of the regular entry point,
pse_mobility_apply_parts(PSE_PART_REAL), within the mixed-precision tolerance,
on calls in a row that share its static scratch array: a dense box, a box of
fewer than three cells per side, a dilute box whose cells are clamped to 32 per
side (cells larger than r_cut), and the first case again after the others (its
table is uploaded anew).  Kept in its own file so that pytest collects it last."""
import numpy as np
import pytest

import pse_inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(pkg, mobility_real_noalloc, pos, L, xi, tol, seed):
    N = pos.shape[0]
    F, S = pse_inputs.moments(N, seed=seed + 1)
    tp = torch.tensor(pos, device='cuda')
    tF = torch.tensor(F, device='cuda', dtype=torch.float32)
    tS = torch.tensor(S, device='cuda', dtype=torch.float32)
    U, E = mobility_real_noalloc(tp, tF, tS, L, xi=xi, tol=tol)
    h = pkg.PSE(N, L, xi=xi, tol=tol, precision='mixed')
    Ur, Er = h.mobility(tp, tF, tS, parts='real')
    h.close()
    got = np.concatenate([U.cpu().numpy(), E.cpu().numpy()], 1).astype(np.float64)
    ref = np.concatenate([Ur.cpu().numpy(), Er.cpu().numpy()], 1).astype(np.float64)
    assert _rel(got, ref) < 2e-5, (N, L, _rel(got, ref))


def test_noalloc_matches_regular_real_space_product():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import paper_1709_06946_gb300 as pkg
    from paper_1709_06946_gb300.binding import mobility_real_noalloc
    pkg.build()
    dense = pse_inputs.rsa_positions(3000, 0.3, seed=5)
    # r_cut = 1 + sqrt(ln 1e4)/0.8 = 4.79 at L = 12: two cells per side
    small = (pse_inputs.random_positions(60, 12.0, seed=21), 12.0)
    # r_cut = 1 + sqrt(ln 1e4)/1.0 = 4.03 at L = 140: 34 cells of r_cut, clamped to 32
    dilute = (pse_inputs.random_positions(20000, 140.0, seed=22), 140.0)
    cases = [(dense, 0.7, 1e-3, 5), (pse_inputs.rsa_positions(1200, 0.2, seed=6), 0.8, 1e-4, 6),
             (small, 0.8, 1e-3, 7), (dilute, 1.0, 1e-3, 8), (dense, 0.7, 1e-3, 5)]
    for (pos, L), xi, tol, seed in cases:
        _case(pkg, mobility_real_noalloc, pos, L, xi, tol, seed)
    with pytest.raises(pkg.PSEError):
        big = torch.zeros((70000, 3), dtype=torch.float64, device='cuda')
        mobility_real_noalloc(big, None, None, 100.0)
    with pytest.raises(ValueError):
        mobility_real_noalloc(torch.zeros((10, 3), dtype=torch.float32, device='cuda'), None, None, 100.0)
