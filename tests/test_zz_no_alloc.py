"""GPU test of fmm_morton_sort_noalloc, the entry point for callers that cannot allocate
device memory (hosts that own all device memory in their own pool, and code that must not
call cudaMalloc/cudaFree because those can synchronise the whole device).

It is called through the C ABI with caller-owned device buffers, twice in a row and
with a smaller input afterwards (its scratch array keeps the previous call's contents),
and must reproduce, bit for bit, the sorted keys, permutation and bounding cube that
fmm_build + fmm_get_keys give for the same positions.  Kept in the last-collected file
so that a run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_2107_07166_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_07166_gb300 import fmm
    return torch, fmm, fmm.load()


def reference_keys(fmm, torch, x):
    f = fmm.FMM(0, stream=torch.cuda.current_stream())
    f.build(x, np.full(x.shape[0], 1.0 / x.shape[0]), 32)
    keys, perm, lo, side = f.get_keys()
    f.close()
    return keys, perm, lo, side


def noalloc_keys(torch, lib, x, stream=None):
    n = x.shape[0]
    xd = torch.from_numpy(x).cuda()
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int64, device="cuda")
    lo = torch.empty(3, dtype=torch.float64, device="cuda")
    side = torch.empty(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    P = ctypes.c_void_p
    rc = lib.fmm_morton_sort_noalloc(P(xd.data_ptr()), n, P(keys.data_ptr()), P(perm.data_ptr()),
                                     P(lo.data_ptr()), P(side.data_ptr()),
                                     None if stream is None else P(stream.cuda_stream))
    assert rc == 0, lib.fmm_last_error().decode()
    return (keys.cpu().numpy().view(np.uint64), perm.cpu().numpy(), lo.cpu().numpy(), float(side.item()))


def test_noalloc_matches_build_path(env):
    torch, fmm, lib = env
    inputs = [synth.plummer(fmm.NOALLOC_MAX_N, 2)[0], synth.hernquist(100003, 5)[0], synth.plummer(777, 9)[0]]
    for x in inputs:
        want = reference_keys(fmm, torch, x)
        for _ in range(2):                    # two calls in a row share the scratch array
            got = noalloc_keys(torch, lib, x)
            assert np.array_equal(got[0], want[0])
            assert np.array_equal(got[1], want[1])
            assert np.array_equal(got[2], want[2])
            assert got[3] == want[3]


def test_noalloc_tiny_inputs_and_own_stream(env):
    """One to a few particles (one sort tile; the keys still make every pass), and the
    same call queued on a caller's stream instead of the default stream."""
    torch, fmm, lib = env
    s = torch.cuda.Stream()
    for n in (1, 2, 5):
        x = synth.plummer(n, 11)[0] if n > 1 else np.array([[0.25, -1.5, 3.0]])
        want = reference_keys(fmm, torch, x)
        for stream in (None, s):
            got = noalloc_keys(torch, lib, x, stream)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
            assert np.array_equal(got[2], want[2]) and got[3] == want[3]
    x = synth.hernquist(50001, 12)[0]
    want = reference_keys(fmm, torch, x)
    got = noalloc_keys(torch, lib, x, s)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_noalloc_rejects_nonfinite_coordinate(env):
    """A NaN coordinate is an input error (-1, FMM_ERR_INVALID), found by the cube kernel's
    finiteness check; the scratch array stays usable for the next call."""
    torch, fmm, lib = env
    P = ctypes.c_void_p
    x = synth.plummer(1000, 13)[0]
    x[417, 1] = np.nan
    xd = torch.from_numpy(x).cuda()
    keys = torch.empty(1000, dtype=torch.int64, device="cuda")
    perm = torch.empty(1000, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    rc = lib.fmm_morton_sort_noalloc(P(xd.data_ptr()), 1000, P(keys.data_ptr()), P(perm.data_ptr()),
                                     None, None, None)
    assert rc == -1
    assert "non-finite" in lib.fmm_last_error().decode()
    x[417, 1] = 0.5
    want = reference_keys(fmm, torch, x)
    got = noalloc_keys(torch, lib, x)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_noalloc_rejects_oversize_and_host_arrays(env):
    torch, fmm, lib = env
    P = ctypes.c_void_p
    n = fmm.NOALLOC_MAX_N + 1
    xd = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    rc = lib.fmm_morton_sort_noalloc(P(xd.data_ptr()), n, P(out.data_ptr()), P(out.data_ptr()), None, None, None)
    assert rc == -5                                            # FMM_ERR_CAPACITY
    assert "FMM_NOALLOC_MAX_N" in lib.fmm_last_error().decode()
    xh = np.zeros((16, 3))
    rc = lib.fmm_morton_sort_noalloc(xh.ctypes.data_as(P), 16, P(out.data_ptr()), P(out.data_ptr()),
                                     None, None, None)
    assert rc == -1                                            # host memory is refused
