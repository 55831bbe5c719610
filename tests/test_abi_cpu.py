"""The C-ABI library loads on a machine without a GPU, exports every entry
point that include/apcg.h declares, and validates arguments on the host."""

import ctypes as C
import subprocess

import pytest

from paper_2306_17801_gb300 import apcg


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return apcg.load()


def test_every_header_function_is_exported(lib):
    declared = apcg.header_functions()
    assert len(declared) >= 60
    out = subprocess.run(["nm", "-D", "--defined-only", apcg.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    for f in declared:
        assert hasattr(lib, f)
    # the binding declares a prototype for each of them, and for nothing else
    assert sorted(declared) == sorted(apcg.PROTOS)


def test_version_and_error_string(lib):
    assert lib.apcg_version() == 10000
    st = lib.apcg_vec_wrap(None, -5, apcg.F64, C.byref(C.c_void_p()))
    assert st == -1
    assert "negative" in apcg.last_error()


def test_host_validation_rejects_bad_arguments(lib):
    h = C.c_void_p()
    # misaligned pointer
    assert lib.apcg_vec_wrap(C.c_void_p(0x1008), 4, apcg.F64, C.byref(h)) == -1
    # nnz beyond the int32 range
    assert lib.apcg_mat_csr_wrap(C.c_void_p(0x1000), C.c_void_p(0x2000), C.c_void_p(0x3000), 4, 4, 2**31, apcg.F64, C.byref(h)) == -1
    # bad options are rejected before any device work
    o = apcg.CgOpts()
    assert lib.apcg_cg_opts_default(C.byref(o)) == 0
    assert o.rtol == 1e-8 and o.check_every == 1 and o.mode == apcg.MODE_AUTO
    assert lib.apcg_cg_plan_create(None, None, C.byref(o), C.byref(h)) == -1


def test_vec_wrap_registers_memory_ids(lib):
    v1 = C.c_void_p()
    v2 = C.c_void_p()
    assert lib.apcg_vec_wrap(C.c_void_p(0x10000), 8, apcg.F64, C.byref(v1)) == 0
    assert lib.apcg_vec_wrap(C.c_void_p(0x10000), 8, apcg.F64, C.byref(v2)) == 0
    i1, i2 = apcg.vec_id(v1.value), apcg.vec_id(v2.value)
    assert i1 == i2 != 0  # same memory, same object ID
    rid = C.c_uint64()
    sz = C.c_size_t()
    assert lib.apcg_get_pointer_attributes(C.c_void_p(0x10000), C.byref(rid), C.byref(sz)) == 0
    assert rid.value == i1 and sz.value == 64
    assert lib.apcg_vec_destroy(v1) == 0 and lib.apcg_vec_destroy(v2) == 0
    assert lib.apcg_unregister_memory(C.c_void_p(0x10000)) == 0


def test_context_creation_fails_loudly_without_a_gpu(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(apcg.ApcgError) as e:
        apcg.ctx_create()
    assert e.value.status == -2
