"""GPU tests of the serving loop (pse_server_*): results are the same alone and
in a mix of concurrent requests, requests overlap on the device, admission
respects the device-memory budget, and oversized requests are rejected."""
import numpy as np
import pytest

import pse_inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

XI, EPS = 0.5, 1e-3


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


def _system(N, phi, seed):
    pos, L = pse_inputs.rsa_positions(N, phi, seed=seed)
    F, S = pse_inputs.moments(N, seed=seed + 1)
    return pos, L, F.astype(np.float32), S.astype(np.float32)


def _run_pair(srv, A, B):
    """A constrained step on A and a mobility product on B; returns their results."""
    posA, LA, FA, _ = A
    posB, LB, FB, SB = B
    xa = posA.copy()
    ta, oa = srv.submit('step', xa, LA, xi=XI, tol=EPS, F=FA, dt=1e-3, seed=7, counter=3)
    tb, ob = srv.submit('mobility', posB, LB, xi=XI, tol=EPS, F=FB, S=SB)
    return ta, tb, xa, oa, ob


def test_same_result_alone_and_in_mix(pkg):
    A = _system(3000, 0.25, 31)
    B = _system(1500, 0.1, 33)
    others = [_system(n, phi, 40 + k) for k, (n, phi) in enumerate([(6000, 0.3), (2000, 0.05), (4000, 0.2)])]
    # alone: one slot, nothing else queued
    srv = pkg.Server(slots=1, budget_bytes=16 << 30)
    ta, tb, xa1, oa1, ob1 = _run_pair(srv, A, B)
    assert srv.wait(ta)[0] in (0, 4) and srv.wait(tb)[0] == 0
    srv.close()
    # in a mix: four slots, the same two requests among others submitted around them
    srv = pkg.Server(slots=4, budget_bytes=16 << 30)
    tickets = []
    for k, (pos, L, F, S) in enumerate(others):
        tickets.append(srv.submit('sample', pos, L, xi=XI, tol=EPS, dt=1e-3, seed=k)[0])
        tickets.append(srv.submit('mobility', pos, L, xi=XI, tol=EPS, F=F, S=S)[0])
    ta, tb, xa2, oa2, ob2 = _run_pair(srv, A, B)
    for k, (pos, L, F, S) in enumerate(others):
        x = pos.copy()
        tickets.append(srv.submit('step', x, L, xi=XI, tol=EPS, dt=1e-3, seed=k, counter=1)[0])
    for t in tickets:
        assert srv.wait(t)[0] in (0, 4)
    assert srv.wait(ta)[0] in (0, 4) and srv.wait(tb)[0] == 0
    st = srv.stats()
    srv.close()
    assert st['completed'] == len(tickets) + 2
    assert st['peak_running'] >= 2                      # requests overlapped on the device
    L = A[1]
    d1 = xa1 - A[0]
    d2 = xa2 - A[0]
    d1 -= L * np.rint(d1 / L)
    d2 -= L * np.rint(d2 / L)
    assert _rel(d2, d1) < 2e-5
    assert _rel(oa2['S'], oa1['S']) < 2e-5
    assert _rel(np.concatenate([ob2['U'], ob2['E']], 1), np.concatenate([ob1['U'], ob1['E']], 1)) < 2e-5


def test_server_result_equals_direct_call(pkg):
    pos, L, F, S = _system(2500, 0.2, 51)
    h = pkg.PSE(len(pos), L, xi=XI, tol=EPS, precision='fp64')
    U, E = h.mobility(pos, F.astype(np.float64), S.astype(np.float64))
    h.close()
    srv = pkg.Server(slots=2, budget_bytes=8 << 30)
    t, o = srv.submit('mobility', pos, L, xi=XI, tol=EPS, precision='fp64', F=F.astype(np.float64),
                      S=S.astype(np.float64))
    assert srv.wait(t)[0] == 0
    srv.close()
    assert _rel(o['U'], U) < 1e-12 and _rel(o['E'], E) < 1e-12


def test_admission_respects_budget_and_evicts(pkg):
    A = _system(20000, 0.3, 61)
    B = _system(12000, 0.2, 63)
    ea = pkg.binding.estimate_bytes(len(A[0]), A[1], xi=XI, tol=EPS)
    eb = pkg.binding.estimate_bytes(len(B[0]), B[1], xi=XI, tol=EPS)
    budget = max(ea, eb) + min(ea, eb) // 2              # never both resident at once
    srv = pkg.Server(slots=3, budget_bytes=budget)
    tickets = []
    for k in range(3):
        for pos, L, F, S in (A, B):
            tickets.append(srv.submit('mobility', pos, L, xi=XI, tol=EPS, F=F, S=S)[0])
    for t in tickets:
        assert srv.wait(t)[0] == 0
    st = srv.stats()
    srv.close()
    assert st['completed'] == 6
    assert st['peak_resident_bytes'] <= budget
    assert st['handles_evicted'] >= 1


def test_oversized_request_rejected(pkg):
    pos, L, F, S = _system(5000, 0.2, 71)
    srv = pkg.Server(slots=1, budget_bytes=1 << 20)
    with pytest.raises(pkg.PSEError) as e:
        srv.submit('mobility', pos, L, xi=XI, tol=EPS, F=F, S=S)
    assert e.value.code == 2
    assert srv.stats()['rejected'] == 1
    srv.close()


def test_wait_is_bounded(pkg):
    """Waiting on a request that cannot finish in the limit returns TIMEOUT (no hang)."""
    pos, L, F, S = _system(200000, 0.3, 81)
    srv = pkg.Server(slots=1, budget_bytes=32 << 30)
    t, _ = srv.submit('step', pos.copy(), L, xi=XI, tol=EPS, dt=1e-3, seed=1)
    with pytest.raises(TimeoutError):
        srv.wait(t, timeout_ms=0.01)
    assert srv.wait(t)[0] in (0, 4)
    srv.close()
