"""bench.py's reference arm on the CPU: the JSON line it prints follows the
benchmark contract (one line; metric, unit and direction of the main arm; the
oracle's rate as value, cpu_baseline and e2e with no transfers), and the
workloads it does not cover print an `unavailable` line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, 'bench.py'), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith('{')]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run('--impl', 'reference', '--steps', '1', '--warmup', '0', '--ref-N', '400')
    assert d['impl'] == 'reference' and d['unit'] == 'steps/s' and d['higher_is_better'] is True
    assert d['metric'].startswith('Brownian steps/s') and d['n_gpus'] == 1 and d['steps'] == 1
    assert d['value'] > 0 and abs(d['ms_per_step'] - 1000.0 / d['value']) < 1e-6 * d['ms_per_step']
    # the line names the size it ran; the extrapolation to the benchmark size is labelled as such
    assert d['config']['N'] == 400 and d['config']['phi'] == 0.3 and 'N=400' in d['config']['workload']
    assert abs(d['ptps'] - 400 * d['value']) < 1e-9 * d['ptps']
    assert d['extrapolated']['N'] == 1048576 and 'not measured' in d['extrapolated']['basis']
    cb = d['cpu_baseline']
    assert cb['kind'] == 'oracle' and cb['cores'] > 0 and cb['value'] == d['value'] and 'N=400' in cb['sample']
    assert cb['host_cores'] == os.cpu_count() and cb['cpu_model']
    assert d['e2e'] == {'value': d['value'], 'unit': 'steps/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}


def test_reference_arm_other_workloads_unavailable():
    for w in ('batch256', 'serve'):
        d = _run('--impl', 'reference', '--workload', w)
        assert d['impl'] == 'reference' and 'unavailable' in d
