"""GPU parity of the individual kernels against the CPU oracle (through the C ABI).

Bars: integer / bit work bit-exact; FP64 data to ~1e-13 relative; FP32 data
to 2e-6 relative to the largest output entry (a few FP32 roundings of sums of
at most a few hundred terms).
"""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_00839_gb300 import api
    return api.Handle(0)


def _api():
    from paper_2603_00839_gb300 import api
    return api


TOL = {torch.float64: 1e-12, torch.float32: 2e-6}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------------------ Philox


@pytest.mark.parametrize("seed,pid,n", [(0, 0, 1), (0, 0, 4099), (12345, 7, 1000),
                                        (2**64 - 1, 2**63 + 1, 257)])
def test_philox_stream_bit_exact(h, seed, pid, n):
    got = h.philox_words(seed, pid, n).cpu().numpy().view(np.uint64)
    ref = np.array(oracle.philox_words(seed, pid, n), dtype=np.uint64)
    assert np.array_equal(got, ref)


def test_philox_empty(h):
    assert h.philox_words(1, 1, 0).numel() == 0


# ------------------------------------------------------------------------ operator

def _factors(dims, spec, rng):
    """spec: list of (mode, kind, radius or size, side) -> (api factors, oracle factor lists)."""
    api = _api()
    A, B, oA, oB = [], [], [], []
    for mode, kind, r, side in spec:
        n = dims[mode - 1]
        if kind == "banded":
            taps = rng.uniform(-1, 1, 2 * r + 1)
            f = api.banded(mode, n, taps)
            of = (mode, "banded", taps)
        elif kind == "dense":
            M = rng.standard_normal((n, n))
            f = api.dense(mode, M)
            of = (mode, "dense", M)
        else:
            f = api.identity(mode, n)
            of = (mode, "identity", None)
        (B if side else A).append(f)
        (oB if side else oA).append(of)
    return A, B, oA, oB


APPLY_CASES = [
    ((64, 64, 3), [(1, "banded", 4, 0), (2, "banded", 4, 0)]),                       # image64
    ((150, 37, 3), [(1, "banded", 7, 0), (2, "banded", 7, 0), (3, "dense", 3, 1)]),  # ragged, fused mix
    ((67, 45, 2), [(1, "banded", 2, 0), (2, "banded", 5, 0), (3, "banded", 1, 1)]),  # banded right factor
    ((5, 3, 3), [(1, "banded", 6, 0), (2, "banded", 6, 0), (3, "dense", 3, 1)]),     # band wider than the mode
    ((40, 33, 3, 6), [(1, "banded", 3, 0), (2, "banded", 3, 0), (3, "dense", 3, 1),
                      (4, "banded", 2, 0)]),                                          # video: unfused path
    ((70, 9, 7), [(1, "dense", 0, 0), (3, "dense", 0, 0)]),                          # dense on mode 1
    ((33, 65, 5), [(3, "dense", 0, 1)]),                                              # mix size 5: unfused
    ((97,), [(1, "banded", 32, 0)]),                                                  # order 1, max radius
    ((31, 29), [(2, "banded", 3, 0)]),                                                # order 2, mode-1 identity
    ((12, 10, 3), []),                                                                # identity operator
    ((64, 48, 3), [(1, "banded", 2, 0), (1, "banded", 1, 0)]),                       # two factors on one mode
]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", range(len(APPLY_CASES)))
def test_operator_apply_parity(h, dt, case):
    dims, spec = APPLY_CASES[case]
    rng = np.random.default_rng(case)
    A, B, oA, oB = _factors(dims, spec, rng)
    X = rng.standard_normal(dims)
    mats = oracle.factor_matrices(dims, oA, oB)
    ref = oracle.apply_operator(X, mats)
    api = _api()
    Y = h.operator_apply(api.to_device(X, dt), A, B)
    torch.cuda.synchronize()
    assert _rel(Y.cpu().double().numpy(), ref) < TOL[dt] * (10 if dt == torch.float32 else 1)


def test_operator_apply_full_size_image512(h):
    """The 512x512x3 operator at full size, checked on sampled outputs computed one by one."""
    p = w.image_config(2)
    api = _api()
    A = [api.banded(m, p.dims[m - 1], t) for m, _, t in p.factors]
    B = [api.dense(3, w.channel_mix())]
    X = p.x_true
    Y = h.operator_apply(api.to_device(X, torch.float32), A, B).cpu().double().numpy()
    a = w.gaussian_taps(2.5, 7)
    Bm = w.channel_mix()
    rng = np.random.default_rng(0)
    for _ in range(200):
        i, j, c = rng.integers(0, 512), rng.integers(0, 512), rng.integers(0, 3)
        acc = 0.0
        for cc in range(3):
            for s in range(-7, 8):
                for t in range(-7, 8):
                    if 0 <= i + s < 512 and 0 <= j + t < 512:
                        acc += Bm[cc, c] * a[7 + s] * a[7 + t] * X[i + s, j + t, cc]
        assert abs(Y[i, j, c] - acc) <= 2e-6 * max(1.0, abs(acc))


def test_operator_apply_rejects_bad_args(h):
    api = _api()
    from paper_2603_00839_gb300._lib import RtgError
    X = api.empty((8, 8, 3), torch.float32)
    with pytest.raises(RtgError):
        h.operator_apply(X, [api.banded(1, 7, [1.0])])            # n mismatch
    with pytest.raises(RtgError):
        h.operator_apply(X, [api.banded(4, 8, [1.0])])            # mode outside order
    with pytest.raises(RtgError):
        h.operator_apply(X, [api.banded(1, 8, np.ones(67))])      # radius 33 > 32
    with pytest.raises(RtgError):
        h.operator_apply(X, [], [], Y=X)                          # aliasing
    with pytest.raises(TypeError):
        h.operator_apply(api.empty((8, 8), torch.float16))


# ------------------------------------------------------------------------ sketch

SKETCH_CASES = [
    ((64, 64, 3), (32, 32, 3), 0),
    ((150, 37, 3), (40, 16, 3), 5),       # ragged: I not a multiple of 32, rows not word aligned
    ((67, 45, 2), (67, 11, 2), 1),        # mode 1 not sketched (s = I)
    ((40, 33, 3, 6), (16, 8, 3, 4), 9),   # order 4
    ((97,), (13,), 3),                    # order 1
    ((12, 10, 3), (12, 10, 3), 0),        # nothing sketched: S = I
    ((33, 20, 5), (1, 1, 2), 4),          # sketch size 1
    ((64, 512, 20), (32, 64, 20), 2),     # >= 608 column tiles: the multi-tile first stage
    ((36, 300, 35), (20, 50, 35), 6),     # multi-tile, ragged rows and a 4-column last tile
    ((320, 64, 160), (80, 16, 16), 7),    # multi-tile, 20 K tiles, two row blocks
    ((300, 21, 3), (200, 10, 3), 8),      # s_1 > 128 (two row tiles), ragged K block and column tile
    ((300, 41, 200), (200, 10, 3), 10),   # the same on the tcgen05 first stage (>= 8192 columns)
    ((150, 64, 130), (40, 16, 13), 11),   # tcgen05 first stage, K not a multiple of 4 (plain loads)
]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", range(len(SKETCH_CASES)))
def test_sketch_parity(h, dt, case):
    dims, sk, seed = SKETCH_CASES[case]
    X = np.random.default_rng(case).standard_normal(dims)
    th = oracle.sketch_matrices(dims, sk, seed, problem_id=0)
    ref = oracle.sketch(X, th)
    api = _api()
    SX = h.sketch(api.to_device(X, dt), sk, seed)
    torch.cuda.synchronize()
    assert SX.shape == ref.shape
    assert _rel(SX.cpu().double().numpy(), ref) < TOL[dt] * (10 if dt == torch.float32 else 1)


def test_sketch_full_size_image512_sampled(h):
    """512x512x3 with sketch (128,128,3): sampled sketch entries against the definition."""
    api = _api()
    X = w.piecewise_image(512, 512, 3, seed=3)
    SX = h.sketch(api.to_device(X, torch.float32), (128, 128, 3), seed=11).cpu().double().numpy()
    th = oracle.sketch_matrices((512, 512, 3), (128, 128, 3), 11)
    rng = np.random.default_rng(1)
    for _ in range(64):
        a, b, c = rng.integers(0, 128), rng.integers(0, 128), rng.integers(0, 3)
        ref = th[0][a] @ X[:, :, c] @ th[1][b]
        assert abs(SX[a, b, c] - ref) <= 2e-6 * max(1.0, np.abs(X[:, :, c]).sum() / 128)


def test_sketch_full_size_video_sampled(h):
    """256x256x3x64 with sketch (96,96,3,32): sampled entries against the definition."""
    api = _api()
    X = np.random.default_rng(4).standard_normal((256, 256, 3, 64))
    SX = h.sketch(api.to_device(X, torch.float32), (96, 96, 3, 32), seed=5).cpu().double().numpy()
    th = oracle.sketch_matrices((256, 256, 3, 64), (96, 96, 3, 32), 5)
    rng = np.random.default_rng(2)
    for _ in range(48):
        a, b, c, d = rng.integers(0, 96), rng.integers(0, 96), rng.integers(0, 3), rng.integers(0, 32)
        ref = np.einsum("i,ijf,j,f->", th[0][a], X[:, :, c, :], th[1][b], th[3][d])
        mag = np.einsum("i,ijf,j,f->", np.abs(th[0][a]), np.abs(X[:, :, c, :]), np.abs(th[1][b]),
                        np.abs(th[3][d]))
        assert abs(SX[a, b, c, d] - ref) <= 1e-6 * mag


def test_sketch_problem_id_changes_signs(h):
    api = _api()
    X = api.to_device(np.random.default_rng(0).standard_normal((64, 64, 3)), torch.float64)
    a = h.sketch(X, (16, 16, 3), 1, problem_id=0).cpu().numpy()
    b = h.sketch(X, (16, 16, 3), 1, problem_id=1).cpu().numpy()
    th = oracle.sketch_matrices((64, 64, 3), (16, 16, 3), 1, problem_id=1)
    assert not np.allclose(a, b)
    assert _rel(b, oracle.sketch(X.cpu().numpy(), th)) < 1e-12


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_sketch_seed_sequence_on_one_handle(h, dt):
    """S(X) with seeds 0, 5, 0 on one handle and shape (Section 3, the global
    sketching operator): every call uses the signs of its own seed."""
    api = _api()
    dims, sk = (96, 80, 3), (32, 24, 3)
    Xh = np.random.default_rng(3).standard_normal(dims)
    X = api.to_device(Xh, dt)
    tol = TOL[dt] * (10 if dt == torch.float32 else 1)
    outs = []
    for seed in (0, 5, 0, 5, 5):
        SX = h.sketch(X, sk, seed).cpu().double().numpy()
        ref = oracle.sketch(Xh, oracle.sketch_matrices(dims, sk, seed))
        assert _rel(SX, ref) < tol, seed
        outs.append(SX)
    assert not np.allclose(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])


def test_sketch_and_apply_on_two_streams_of_one_handle(h):
    """Calls of one handle on two streams: each stream has its own scratch."""
    api = _api()
    dims, sk = (64, 48, 3), (16, 16, 3)
    Xh = [np.random.default_rng(10 + i).standard_normal(dims) for i in range(2)]
    X = [api.to_device(x, torch.float32) for x in Xh]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    SX = [None, None]
    for rep in range(4):
        for i in range(2):
            with torch.cuda.stream(streams[i]):
                SX[i] = h.sketch(X[i], sk, seed=7 * i + rep, stream=streams[i])
        torch.cuda.synchronize()
        for i in range(2):
            ref = oracle.sketch(Xh[i], oracle.sketch_matrices(dims, sk, 7 * i + rep))
            assert _rel(SX[i].cpu().double().numpy(), ref) < 2e-5
