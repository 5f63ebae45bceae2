"""CPU-side checks of the C ABI boundary: the library builds for sm_103a,
loads, exports every function include/nrm.h declares, and rejects bad
arguments synchronously (no compute call is made without a GPU)."""
import ctypes

import pytest

import paper_2509_06220_gb300 as nrm
from paper_2509_06220_gb300 import build as nb


@pytest.fixture(scope="module")
def L():
    nb.build()
    return nrm.load()


def test_header_declares_entry_points():
    names = nrm.header_functions()
    for want in ("nrmf_s", "nrmf_d", "nrmp_s", "nrmp_d", "nrm_batch", "nrm_batch_graph", "nrm_host",
                 "nrm_create", "nrm_destroy", "nrm_gen", "nrm_gen_ragged"):
        assert want in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in nrm.header_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(L):
    assert L.nrm_status_string(0) == b"NRM_OK"
    assert L.nrm_status_string(-1) == b"NRM_EINVAL"
    assert L.nrm_status_string(-5) == b"NRM_EBUDGET"


def test_null_context_is_einval(L):
    vp = ctypes.c_void_p
    assert L.nrmf_d(None, vp(0), 10, vp(0), None) == nrm.NRM_EINVAL
    assert L.nrmf_s(None, vp(0), 10, vp(0), None) == nrm.NRM_EINVAL
    assert L.nrmp_d(None, vp(0), 10, 3.0, vp(0), None) == nrm.NRM_EINVAL
    assert L.nrm_batch(None, 1, vp(0), 0, vp(0), 1, 2.0, None, vp(0), vp(0), None) == nrm.NRM_EINVAL
    assert L.nrm_host(None, 1, vp(0), 1, 2.0, vp(0)) == nrm.NRM_EINVAL
    assert L.nrm_destroy(None) == nrm.NRM_OK


def test_generator_rejects_bad_ranges(L):
    vp = ctypes.c_void_p
    assert L.nrm_gen(1, vp(0), -1, 0, 0, 0, -20, 20, None) == nrm.NRM_EINVAL
    assert L.nrm_gen(0, vp(0), 10, 0, 0, 0, -127, 20, None) == nrm.NRM_EINVAL
    assert L.nrm_gen(1, vp(0), 10, 0, 0, 0, 5, 4, None) == nrm.NRM_EINVAL
    assert L.nrm_gen(7, vp(0), 10, 0, 0, 0, -20, 20, None) == nrm.NRM_EINVAL
    assert L.nrm_gen(1, vp(0), 0, 0, 0, 0, -20, 20, None) == nrm.NRM_OK  # empty: nothing enqueued


def test_create_without_device(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert L.nrm_create(ctypes.byref(h), 0) == nrm.NRM_EDEVICE
    assert not h.value


def test_tuning_struct_layout():
    assert ctypes.sizeof(nrm.Tuning) == 16
