"""GPU test of pse_mobility_real_noalloc, the entry point for callers that cannot
allocate device memory (codes that must not let cudaMalloc/cudaFree synchronise
the device inside their loop, or whose device memory belongs to their own pool
allocator).  It must reproduce the real-space product of the regular entry point,
pse_mobility_apply_parts(PSE_PART_REAL), within the mixed-precision tolerance,
on two calls in a row that share its static scratch array.  Kept in its own file
so that pytest collects it last."""
import numpy as np
import pytest

import pse_inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_regular_real_space_product():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import paper_1709_06946_gb300 as pkg
    from paper_1709_06946_gb300.binding import mobility_real_noalloc
    pkg.build()
    cases = [(3000, 0.3, 0.7, 1e-3, 5), (1200, 0.2, 0.8, 1e-4, 6)]
    for N, phi, xi, tol, seed in cases:             # two calls in a row, different tables and cells
        pos, L = pse_inputs.rsa_positions(N, phi, seed=seed)
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
        assert _rel(got, ref) < 2e-5, (N, _rel(got, ref))
    with pytest.raises(pkg.PSEError):
        big = torch.zeros((70000, 3), dtype=torch.float64, device='cuda')
        mobility_real_noalloc(big, None, None, 100.0)
