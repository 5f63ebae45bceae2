"""nrmf_d_noalloc: the binary64 xNRMF entry point that allocates nothing.

Some callers cannot call cudaMalloc (it and cudaFree can synchronise the
whole device, and some applications forbid allocations outside their own
allocator or budget); this entry point keeps its scratch in a static device
array inside the library instead.  These tests call it through the C ABI and
check it against nrmf_d, bit for bit, on two calls in a row (the second
call reuses the scratch the first left behind), at sizes up to its
documented maximum of 2^29 elements, plus its size limit and the empty
vector.  The file is collected last so that a failure here stops a
-x run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_06220_gb300 as nrm
    L = nrm.load()
    f = L.nrmf_d_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return nrm, L


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_nrmf_d_two_calls_in_a_row(lib):
    nrm, L = lib
    dev = "cuda:0"
    # two different tree shapes: 2^10 work items and then fewer, larger ones
    x1 = nrm.nrm_gen((1 << 26) + 12345, 21, 0, torch.float64, device=dev)
    x2 = nrm.nrm_gen(3000017, 22, 0, torch.float64, device=dev)[1:]  # odd element offset
    want = torch.empty(2, dtype=torch.float64, device=dev)
    nrm.nrmf(x1, out=want[0])
    nrm.nrmf(x2, out=want[1])
    got = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    s = _stream()
    assert L.nrmf_d_noalloc(ctypes.c_void_p(x1.data_ptr()), x1.numel(), ctypes.c_void_p(got[0].data_ptr()), s) == 0
    assert L.nrmf_d_noalloc(ctypes.c_void_p(x2.data_ptr()), x2.numel(), ctypes.c_void_p(got[1].data_ptr()), s) == 0
    torch.cuda.synchronize()
    g, w = got.cpu().numpy(), want.cpu().numpy()
    assert g.tobytes() == w.tobytes(), (g, w)
    # and once more on the first input, after the second call's leftovers
    again = torch.empty((), dtype=torch.float64, device=dev)
    assert L.nrmf_d_noalloc(ctypes.c_void_p(x1.data_ptr()), x1.numel(), ctypes.c_void_p(again.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert np.float64(again.item()).tobytes() == w[0].tobytes()


@pytest.mark.parametrize("n", [(1 << 28) + 1, (1 << 29) - 777, 1 << 29])
def test_noalloc_up_to_its_documented_maximum(lib, n):
    """Every n up to NRM_NOALLOC_MAX_N = 2^29 is accepted and bitwise equal
    to nrmf_d: the deepest trees (2^23 rows) use all 2^11 work items and the
    full counter stack."""
    nrm, L = lib
    dev = "cuda:0"
    x = nrm.nrm_gen(n, 23, 0, torch.float64, device=dev)
    want = torch.empty((), dtype=torch.float64, device=dev)
    nrm.nrmf(x, out=want)
    got = torch.full((), float("nan"), dtype=torch.float64, device=dev)
    assert L.nrmf_d_noalloc(ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(got.data_ptr()), _stream()) == 0
    torch.cuda.synchronize()
    assert np.float64(got.item()).tobytes() == np.float64(want.item()).tobytes(), (got.item(), want.item())
    del x
    torch.cuda.empty_cache()


def test_noalloc_limits(lib):
    nrm, L = lib
    x = torch.ones(4, dtype=torch.float64, device="cuda:0")
    out = torch.full((), 7.0, dtype=torch.float64, device="cuda:0")
    s = _stream()
    too_big = (1 << 29) + 1  # NRM_NOALLOC_MAX_N + 1
    assert L.nrmf_d_noalloc(ctypes.c_void_p(x.data_ptr()), too_big, ctypes.c_void_p(out.data_ptr()), s) == \
        nrm.NRM_EINVAL
    assert L.nrmf_d_noalloc(ctypes.c_void_p(x.data_ptr()), -1, ctypes.c_void_p(out.data_ptr()), s) == nrm.NRM_EINVAL
    assert L.nrmf_d_noalloc(ctypes.c_void_p(x.data_ptr()), 4, None, s) == nrm.NRM_EINVAL
    assert L.nrmf_d_noalloc(None, 0, ctypes.c_void_p(out.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert out.item() == 0.0
