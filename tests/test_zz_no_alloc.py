"""rtg_sketch_noalloc, the sketch entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc (a framework next to them already
reserved the device memory for its pool, or their loop cannot afford
cudaMalloc's implicit synchronisation).  rtg_sketch_noalloc serves them
from a fixed static device array.  This test calls it through the C ABI,
twice in a row with different shapes, dtypes and seeds (so the second call
runs on scratch the first one left behind), and checks both results
against rtg_sketch, the entry point that allocates its scratch, within the
tolerance the kernel parity tests use.  It also checks that a size whose
scratch exceeds the static array is rejected with a clear message.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_00839_gb300 import _lib
    return _lib


def _noalloc(L, X, sketch_dims, seed, pid):
    from paper_2603_00839_gb300 import api
    dims = tuple(X.shape)
    sd = tuple(int(min(s, d)) for s, d in zip(sketch_dims, dims))
    SX = api.empty(sd, X.dtype, X.device)
    shape = L.Shape()
    shape.order = len(dims)
    for k, d in enumerate(dims):
        shape.dims[k] = d
    sk = (ctypes.c_int64 * len(dims))(*sketch_dims)
    dt = L.F64 if X.dtype == torch.float64 else L.F32
    st = L.load().rtg_sketch_noalloc(shape, dt, sk, ctypes.c_uint64(seed), ctypes.c_uint64(pid),
                                     X.data_ptr(), SX.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    return st, SX


def test_noalloc_sketch_matches_allocating_sketch_twice(lib):
    from paper_2603_00839_gb300 import api
    h = api.Handle(0)
    cases = [((512, 512, 3), (128, 128, 3), torch.float32, 7, 0),
             ((150, 37, 3, 2), (40, 16, 3, 1), torch.float64, 3, 5)]
    for dims, sk, dt, seed, pid in cases:
        X = api.to_device(np.random.default_rng(seed).standard_normal(dims), dt)
        st, got = _noalloc(lib, X, sk, seed, pid)
        assert st == lib.OK, lib.load().rtg_last_error()
        ref = h.sketch(X, sk, seed, problem_id=pid)
        torch.cuda.synchronize()
        g, r = got.cpu().double().numpy(), ref.cpu().double().numpy()
        assert np.max(np.abs(g - r)) <= TOL[dt] * np.max(np.abs(r))


def test_noalloc_rejects_scratch_beyond_the_static_array(lib):
    from paper_2603_00839_gb300 import api
    X = api.empty((2048, 1024, 3), torch.float32)
    st, _ = _noalloc(lib, X, (1024, 64, 3), 1, 0)
    assert st == lib.ERR_INVALID_ARG
    assert b"static scratch holds" in lib.load().rtg_last_error()


def test_noalloc_rejects_overlap_and_oversized_shapes(lib):
    """The same argument checks as rtg_sketch: no partial overlap of SX with
    X, no tensor above 2^40 elements (nothing is launched for either)."""
    from paper_2603_00839_gb300 import api
    buf = api.empty((64 * 48 * 3 + 256,), torch.float32)
    L = lib.load()
    shape = lib.Shape()
    shape.order = 3
    for k, d in enumerate((64, 48, 3)):
        shape.dims[k] = d
    sk = (ctypes.c_int64 * 3)(16, 16, 3)
    stream = torch.cuda.current_stream().cuda_stream
    # SX starts 64 floats into X: a partial overlap
    st = L.rtg_sketch_noalloc(shape, lib.F32, sk, ctypes.c_uint64(1), ctypes.c_uint64(0),
                              buf.data_ptr(), buf.data_ptr() + 256, stream)
    assert st == lib.ERR_INVALID_ARG and b"overlap" in L.rtg_last_error()
    big = lib.Shape()
    big.order = 3
    for k, d in enumerate((1 << 21, 1 << 21, 2)):
        big.dims[k] = d
    st = L.rtg_sketch_noalloc(big, lib.F32, sk, ctypes.c_uint64(1), ctypes.c_uint64(0),
                              buf.data_ptr(), buf.data_ptr() + 4 * 64 * 48 * 3, stream)
    assert st == lib.ERR_INVALID_ARG and b"too large" in L.rtg_last_error()
    torch.cuda.synchronize()
