"""Host-side checks of the C ABI (no GPU needed).

- librtg builds for sm_103a and exports every function include/rtg.h declares;
- the binding declares exactly those symbols;
- the Philox round function the kernels use, compiled as host code, gives
  numpy's Philox4x64-10 stream and the oracle's bits.
"""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtg.h")
CSRC = os.path.join(ROOT, "paper_2603_00839_gb300", "csrc")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rtg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_00839_gb300 import _lib
    return _lib.LIB_PATH


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_the_header(lib_path):
    from paper_2603_00839_gb300 import _lib
    assert sorted(_lib.SYMBOLS) == declared_functions()
    lib = _lib.load()
    assert lib.rtg_version() >= 100
    assert lib.rtg_status_string(6).decode() == "RTG_ERR_NONFINITE"


def test_errors_without_gpu_are_reported_not_raised(lib_path):
    from paper_2603_00839_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    st = lib.rtg_create(ctypes.byref(h), 0)
    if st == 0:
        lib.rtg_destroy(h)
        pytest.skip("a GPU is present")
    assert st in (_lib.ERR_CUDA, _lib.ERR_INVALID_ARG)
    assert len(lib.rtg_last_error()) > 0
    assert lib.rtg_create(None, 0) == _lib.ERR_INVALID_ARG


def test_host_compiled_philox_matches_numpy_and_oracle():
    import oracle
    src = r'''
#include <cstdio>
#include <cstdint>
#define __host__
#define __device__
#include "philox.cuh"
int main() {
  const uint64_t keys[3][2] = {{0, 0}, {12345, 7}, {0xFFFFFFFFFFFFFFFFull, 3}};
  for (int k = 0; k < 3; ++k)
    for (uint64_t b = 0; b < 5; ++b) {
      uint64_t r[4];
      rtg::philox4x64_10(b + 1, 0, 0, 0, keys[k][0], keys[k][1], r);
      for (int l = 0; l < 4; ++l) printf("%llu\n", (unsigned long long)r[l]);
    }
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.cpp")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, c, "-o", exe], check=True)
        out = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                              check=True).stdout.split()]
    keys = [(0, 0), (12345, 7), (2**64 - 1, 3)]
    for k, (seed, pid) in enumerate(keys):
        got = out[20 * k:20 * (k + 1)]
        ref = [int(v) for v in np.random.Philox(key=seed + (pid << 64)).random_raw(20)]
        assert got == ref
        assert got == oracle.philox_words(seed, pid, 20)


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Sizes and field offsets of the binding's ctypes mirrors equal those a
    C compiler gives the structs of include/rtg.h."""
    from paper_2603_00839_gb300 import _lib as L
    structs = {"rtg_shape": L.Shape, "rtg_factor": L.Factor, "rtg_opts": L.Opts,
               "rtg_info": L.Info, "rtg_krylov_view": L.KrylovView, "rtg_problem": L.Problem}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rtg.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append(f'  printf("phases %d\\n", (int)RTG_PHASE_COUNT);')
    lines.append('  return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    want = []
    for cname, py in structs.items():
        want.append(f"{cname} size {ctypes.sizeof(py)}")
        for fname, _ in py._fields_:
            want.append(f"{cname} {fname} {getattr(py, fname).offset}")
    want.append(f"phases {L.PHASE_COUNT}")
    assert got[:-1] == want
