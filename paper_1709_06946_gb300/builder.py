"""Builds the in-tree shared library ``libpse.so`` (CUDA for sm_103a + host C++).

Each translation unit is compiled in parallel; nvcc targets
``-gencode arch=compute_103a,code=sm_103a`` only.  The library links cuFFT and
the shared CUDA runtime from the toolkit at CUDA_HOME (default /usr/local/cuda).
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
BUILD = os.path.join(HERE, '_build')
LIB = os.path.join(HERE, 'libpse.so')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(('.cu', '.cpp')))


def _cmd(src, obj):
    path = os.path.join(CSRC, src)
    if src.endswith('.cu'):
        return [os.path.join(CUDA, 'bin', 'nvcc'), '-O3', '-std=c++17', *ARCH, '-lineinfo',
                '-Xcompiler', '-fPIC', '-Xptxas', '-O3', '-c', path, '-o', obj]
    return ['g++', '-O2', '-std=c++17', '-fPIC', '-I' + os.path.join(CUDA, 'include'), '-c', path, '-o', obj]


def _stale(src, obj):
    if not os.path.exists(obj):
        return True
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(('.cuh', '.h'))]
    deps.append(os.path.join(os.path.dirname(HERE), 'include', 'pse.h'))
    deps.append(os.path.join(CSRC, src))
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, force=False):
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for src in _sources():
        obj = os.path.join(BUILD, src.rsplit('.', 1)[0] + '.o')
        if force or _stale(src, obj):
            jobs.append((src, obj))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        futs = {ex.submit(subprocess.run, _cmd(s, o), capture_output=True, text=True): s for s, o in jobs}
        for f in cf.as_completed(futs):
            r = f.result()
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError('compilation of %s failed' % futs[f])
    objs = [os.path.join(BUILD, s.rsplit('.', 1)[0] + '.o') for s in _sources()]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + '.%d.tmp' % os.getpid()
        link = [os.path.join(CUDA, 'bin', 'nvcc'), '-shared', '--cudart', 'shared', *ARCH, '-o', tmp, *objs,
                '-L' + os.path.join(CUDA, 'lib64'), '-lcufft', '-Xlinker', '-rpath,' + os.path.join(CUDA, 'lib64')]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError('link of libpse.so failed')
        os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(verbose='-v' in sys.argv, force='-f' in sys.argv))
