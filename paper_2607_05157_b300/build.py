"""Build libwd.so (the CUDA path behind include/wd.h) in-tree for sm_103a.

Usage: python paper_2607_05157_b300/build.py [--force] [--ptxas]
Each source in csrc/ is compiled with nvcc (-gencode arch=compute_103a,code=sm_103a)
into _build/, in parallel, then linked into paper_2607_05157_b300/libwd.so.
"""
import concurrent.futures
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
OBJ = os.path.join(ROOT, '_build', 'obj')
LIB = os.path.join(HERE, 'libwd.so')
NVCC = os.environ.get('NVCC', '/usr/local/cuda/bin/nvcc')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '-Xcompiler', '-O3',
         '--expt-relaxed-constexpr', '-I' + os.path.join(ROOT, 'include')]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, '*.cu')) + glob.glob(os.path.join(CSRC, '*.cpp')))


def _headers():
    return glob.glob(os.path.join(CSRC, '*.h')) + glob.glob(os.path.join(CSRC, '*.cuh')) + \
        [os.path.join(ROOT, 'include', 'wd.h')]


def _compile(src, hdr_time, force, extra):
    obj = os.path.join(OBJ, os.path.basename(src) + '.o')
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time):
        return obj, None
    cmd = [NVCC] + ARCH + FLAGS + extra + ['-c', src, '-o', obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        return obj, ' '.join(cmd) + '\n' + p.stdout + p.stderr
    return obj, p.stderr if '-Xptxas' in ' '.join(extra) else None


def build(force=False, verbose=False, ptxas_v=False):
    os.makedirs(OBJ, exist_ok=True)
    hdr_time = max(os.path.getmtime(h) for h in _headers())
    extra = ['-Xptxas', '-v'] if ptxas_v else []
    srcs = _sources()
    objs, errs = [], []
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        for obj, msg in ex.map(lambda s: _compile(s, hdr_time, force or ptxas_v, extra), srcs):
            objs.append(obj)
            if msg and (verbose or ptxas_v or 'error' in msg):
                errs.append(msg)
    failed = [m for m in errs if 'error' in m]
    if failed:
        raise RuntimeError('nvcc failed:\n' + '\n'.join(failed))
    if verbose or ptxas_v:
        for m in errs:
            print(m)
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [NVCC] + ARCH + ['-shared', '-o', LIB] + objs + ['-lcudart']
        subprocess.check_call(cmd)
    return LIB


if __name__ == '__main__':
    build(force='--force' in sys.argv, verbose='-v' in sys.argv, ptxas_v='--ptxas' in sys.argv)
    print(LIB)
