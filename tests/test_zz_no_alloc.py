"""The allocation-free candidate mask (disco_candidates_noalloc) against disco_candidates.

Some callers cannot allocate while they run: their device memory belongs to another
allocator's fixed pool, or an allocation's hidden synchronisation would stall a
latency-critical loop. For them the library offers a variant whose temporaries live in a
fixed, library-owned device array. This file is collected last on purpose; it calls both
entry points through the C ABI, twice in a row on different shape pairs (so stale scratch
from the first call would show), and requires identical masks. It also checks that repeated
calls leave the device's free memory unchanged (nothing is allocated), that rows and
columns with fewer than k finite costs give the same masks on both entry points and in the
oracle, and that sizes beyond the fixed array are refused before any GPU work."""
import ctypes

import numpy as np
import pytest

from oracle import problem as P
from synth import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08230_gb300 import _lib
    from paper_2310_08230_gb300.build import build

    build()
    return torch, _lib


def _masks(torch, L, inst, k):
    d = torch.from_numpy(inst.FX).cuda()
    FY = torch.from_numpy(inst.FY).cuda()
    nvx, nvy = inst.X.nv, inst.Y.nv
    dist = torch.empty((nvx, nvy), dtype=torch.float32, device="cuda")
    lib = L.lib()
    stream = torch.cuda.current_stream().cuda_stream
    L.check(lib.disco_pair_costs(d.data_ptr(), FY.data_ptr(), nvx, nvy, inst.FX.shape[1], dist.data_ptr(), stream),
            "pair_costs")
    TX = np.ascontiguousarray(inst.X.T, np.int32)
    TY = np.ascontiguousarray(inst.Y.T, np.int32)
    mx = L.disco_mesh(nvx, TX.shape[0], None, TX.ctypes.data)
    my = L.disco_mesh(nvy, TY.shape[0], None, TY.ctypes.data)
    ref = torch.empty((nvx, nvy), dtype=torch.uint8, device="cuda")
    got = torch.full((nvx, nvy), 7, dtype=torch.uint8, device="cuda")
    L.check(lib.disco_candidates(dist.data_ptr(), nvx, nvy, k, ctypes.byref(mx), ctypes.byref(my), ref.data_ptr(),
                                 stream), "candidates")
    rc = lib.disco_candidates_noalloc(dist.data_ptr(), nvx, nvy, k, ctypes.byref(mx), ctypes.byref(my),
                                      got.data_ptr(), stream)
    assert rc == L.DISCO_OK
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice(env):
    torch, L = env
    for inst, k in ((I.config2(), 10), (I.config1(), 4), (I.config2(), 10)):
        ref, got = _masks(torch, L, inst, k)
        assert np.array_equal(ref, got)
        assert got[np.arange(inst.X.nv), inst.perm].all()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, L = env
    inst = I.config1()
    TX = np.ascontiguousarray(inst.X.T, np.int32)
    mx = L.disco_mesh(inst.X.nv, TX.shape[0], None, TX.ctypes.data)
    d = torch.zeros((inst.X.nv, inst.Y.nv), dtype=torch.float32, device="cuda")
    out = torch.zeros((inst.X.nv, inst.Y.nv), dtype=torch.uint8, device="cuda")
    rc = L.lib().disco_candidates_noalloc(d.data_ptr(), inst.X.nv, inst.Y.nv, 33, ctypes.byref(mx), ctypes.byref(mx),
                                          out.data_ptr(), None)
    assert rc == L.DISCO_ERR_INVALID_ARG
    big = L.disco_mesh(20000, TX.shape[0], None, TX.ctypes.data)
    rc = L.lib().disco_candidates_noalloc(d.data_ptr(), 20000, 20000, 4, ctypes.byref(big), ctypes.byref(big),
                                          out.data_ptr(), None)
    assert rc == L.DISCO_ERR_INVALID_ARG


def test_noalloc_allocates_nothing(env):
    """After the first call (which resolves the array's address and loads the kernels), more
    calls leave cudaMemGetInfo's free bytes exactly where they were."""
    torch, L = env
    inst = I.config2()
    nvx, nvy = inst.X.nv, inst.Y.nv
    d = torch.from_numpy(P.pair_distance(inst.FX, inst.FY).astype(np.float32)).cuda()
    out = torch.empty((nvx, nvy), dtype=torch.uint8, device="cuda")
    TX = np.ascontiguousarray(inst.X.T, np.int32)
    TY = np.ascontiguousarray(inst.Y.T, np.int32)
    mx = L.disco_mesh(nvx, TX.shape[0], None, TX.ctypes.data)
    my = L.disco_mesh(nvy, TY.shape[0], None, TY.ctypes.data)
    lib = L.lib()

    def call():
        return lib.disco_candidates_noalloc(d.data_ptr(), nvx, nvy, 10, ctypes.byref(mx), ctypes.byref(my),
                                            out.data_ptr(), None)

    assert call() == L.DISCO_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert call() == L.DISCO_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_with_non_finite_costs(env):
    """Costs of +inf or NaN are never ranked: rows and columns with fewer than k finite
    entries contribute only those, on both entry points and in the oracle (same FP32 costs)."""
    torch, L = env
    inst = I.config1()
    nvx, nvy = inst.X.nv, inst.Y.nv
    d = P.pair_distance(inst.FX, inst.FY).astype(np.float32)
    d[0, :] = np.inf          # a row with no finite entry
    d[1, 3:] = np.nan         # a row with 3 finite entries (k = 4)
    d[5:, 2] = np.inf         # a column with 5 finite entries
    k = 4
    dd = torch.from_numpy(d).cuda()
    TX = np.ascontiguousarray(inst.X.T, np.int32)
    TY = np.ascontiguousarray(inst.Y.T, np.int32)
    mx = L.disco_mesh(nvx, TX.shape[0], None, TX.ctypes.data)
    my = L.disco_mesh(nvy, TY.shape[0], None, TY.ctypes.data)
    lib = L.lib()
    ref = torch.empty((nvx, nvy), dtype=torch.uint8, device="cuda")
    got = torch.full((nvx, nvy), 7, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    L.check(lib.disco_candidates(dd.data_ptr(), nvx, nvy, k, ctypes.byref(mx), ctypes.byref(my), ref.data_ptr(),
                                 stream), "candidates")
    assert lib.disco_candidates_noalloc(dd.data_ptr(), nvx, nvy, k, ctypes.byref(mx), ctypes.byref(my),
                                        got.data_ptr(), stream) == L.DISCO_OK
    torch.cuda.synchronize()
    want = P.candidate_pairs(d.astype(np.float64), k, inst.X.T, inst.Y.T)
    assert np.array_equal(ref.cpu().numpy().astype(bool), want)
    assert np.array_equal(got.cpu().numpy().astype(bool), want)
