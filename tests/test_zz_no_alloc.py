"""The allocation-free candidate mask (disco_candidates_noalloc) against disco_candidates.

Some callers cannot allocate while they run: their device memory belongs to another
allocator's fixed pool, or an allocation's hidden synchronisation would stall a
latency-critical loop. For them the library offers a variant whose temporaries live in a
fixed, library-owned device array. This file is collected last on purpose; it calls both
entry points through the C ABI, twice in a row on different shape pairs (so stale scratch
from the first call would show), and requires identical masks. It also checks that sizes
beyond the fixed array are refused before any GPU work."""
import ctypes

import numpy as np
import pytest

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
