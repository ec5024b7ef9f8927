"""bench.py's per-kernel roofline arithmetic on the CPU: the kernel names follow the
kernels the library launches for each option, and every rate is the algorithmic
bytes (or formula flops) per launch over the mean launch time, so a reader can
reproduce the bench line's `frac` from its own fields."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
VARIANTS = ('full', 'se', 'fsu', 'su')


def _bench():
    spec = importlib.util.spec_from_file_location('bench_under_test', os.path.join(ROOT, 'bench.py'))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _profile(ms, calls):
    """Stage times (ms) and launch counts split by product variant, as pse_profile reports them."""
    stages = ('spread', 'interp', 'scale', 'noise', 'real')
    vm = {st: {v: 0.0 for v in VARIANTS} for st in stages}
    vc = {st: {v: 0 for v in VARIANTS} for st in stages}
    for (st, v), t in ms.items():
        vm[st][v] = t
        vc[st][v] = calls[(st, v)]
    return {'variant_ms': vm, 'variant_calls': vc}


@pytest.mark.parametrize('wave_kernel,spread,interp', [(0, 'k_spread_colq', 'k_interp_halo'),
                                                        (4, 'k_spread_col', 'k_interp_halo'),
                                                        (1, 'k_spread16', 'k_interp_halo'),
                                                        (2, 'k_spread_colq', 'k_interp_col'),
                                                        (16, 'k_spread_colq', 'k_interp16')])
def test_kernel_names_follow_the_options(wave_kernel, spread, interp):
    b = _bench()
    prof = _profile({('spread', 'se'): 8.0, ('interp', 'se'): 7.0}, {('spread', 'se'): 10, ('interp', 'se'): 10})
    ks = {k['stage']: k['kernel'] for k in b.kernel_instances(prof, 1000, 32, 6, 1e5, True, wave_kernel)}
    assert ks['spread'] == '%s<C=5,P=6>' % spread and ks['interp'] == '%s<C=5,P=6>' % interp
    general = {k['stage']: k['kernel'] for k in b.kernel_instances(prof, 1000, 30, 6, 1e5, False, wave_kernel)}
    assert general['spread'] == 'k_spread<C=5,P=6>' and general['interp'] == 'k_interp<C=5,P=6>'


def test_rates_are_algorithmic_units_over_launch_time():
    b = _bench()
    N, Ng, P, npairs = 1048576, 256, 6, 1.1e8
    nkh = Ng * Ng * (Ng // 2 + 1)
    ms = {('spread', 'se'): 6.64, ('scale', 'se'): 1.07, ('noise', 'full'): 0.209, ('real', 'full'): 9.12,
          ('real', 'se'): 6.73, ('interp', 'fsu'): 0.46}
    calls = {('spread', 'se'): 10, ('scale', 'se'): 10, ('noise', 'full'): 1, ('real', 'full'): 10,
             ('real', 'se'): 10, ('interp', 'fsu'): 1}
    ks = {k['kernel']: k for k in b.kernel_instances(_profile(ms, calls), N, Ng, P, npairs, True)}
    sp = ks['k_spread_colq<C=5,P=6>']
    # spreading, 5 components: N (16 + 4 C) bytes of particle data in, 4 C N_g^3 bytes of grid out
    assert sp['algorithmic_bytes_per_launch'] == N * 36 + 20 * Ng ** 3
    assert sp['launches'] == 10 and sp['us_per_launch'] == pytest.approx(664.0)
    assert sp['achieved'] == pytest.approx(sp['algorithmic_bytes_per_launch'] / 664e-6 / 1e9)
    # kernel scaling S -> E: five half-spectrum components read and five written, 8 B each
    sc = ks['k_scale<M_SE>']
    assert sc['algorithmic_bytes_per_launch'] == 10 * nkh * 8 and sc['us_per_launch'] == pytest.approx(107.0)
    assert ks['k_noise']['algorithmic_bytes_per_launch'] == 8 * nkh * 8
    it = ks['k_interp_halo<C=3,P=6>']
    assert it['algorithmic_bytes_per_launch'] == 12 * Ng ** 3 + N * 28
    # pair sum: formula flops per ordered pair x pairs over the launch time
    fl = b.real_flops_per_pair()
    full = ks['k_real<float,M_FULL>']
    assert full['bound'] == 'alu' and full['flops_per_pair'] == fl['full'] == 178
    assert full['algorithmic_flops_per_launch'] == pytest.approx(npairs * 178)
    assert full['achieved'] == pytest.approx(npairs * 178 / 912e-6 / 1e12)
    assert ks['k_real<float,M_SE>']['flops_per_pair'] == fl['se']
    # instances that did not run are left out
    assert 'k_scale<M_FULL>' not in ks and 'k_real<float,M_SU>' not in ks


def test_formula_flops_per_pair_are_ordered():
    fl = _bench().real_flops_per_pair()
    # the full block holds every term of the reduced products
    assert fl['full'] > fl['se'] > fl['fsu'] > fl['su'] > 0
