"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol
(no compute calls: this file runs without a GPU)."""

import ctypes

import pytest

import paper_2405_10923_gb300 as rh
from paper_2405_10923_gb300 import build


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = rh.header_functions()
    assert "rhqr_factor" in declared and "rhqr_sketch_create" in declared
    missing = [f for f in declared if not hasattr(lib, f)]
    assert not missing, missing
    # every declared function is bound by the Python layer under the same name
    assert set(declared) <= set(rh._SIGNATURES), set(declared) - set(rh._SIGNATURES)


def test_host_only_entry_points():
    lib = rh.load()
    assert lib.rhqr_built_arch() == 103
    assert rh.rhqr_status_string(0) == "ok"
    assert "breakdown" in rh.rhqr_status_string(4)
    o = rh.rhqr_default_opts()
    assert (o.alg, o.passes, o.want_Q, o.scaling) == (rh.ALG_REC, 1, 1, 0)


def test_argument_errors_are_synchronous():
    rh.load()
    out = ctypes.c_void_p()
    # invalid shapes / kinds are rejected before any device work
    assert rh.load().rhqr_sketch_create(1, 4, rh.SRHT, 0, 0, None, ctypes.byref(out)) == 1
    assert rh.load().rhqr_sketch_create(100, 4, 7, 0, 0, None, ctypes.byref(out)) == 1
    assert rh.load().rhqr_sketch_create(100, 0, rh.SRHT, 0, 0, None, ctypes.byref(out)) == 1
    assert rh.load().rhqr_factor(None, None, 0, 10, 2, 10, None, None, 0, None, 0, None, None, None, 0, None, 0,
                                 None, None) == 1
    # batch plans: empty batches and null handles are rejected on the host
    assert rh.load().rhqr_batch_create(0, None, None, 0, None, None, None, None, None, None, None, None, None, None,
                                       ctypes.byref(out)) == 1
    assert rh.load().rhqr_factor_batched(None, None, 0, None, None) == 1
    assert rh.load().rhqr_batch_destroy(None) == 0
    with pytest.raises(rh.RHQRError):
        rh.rhqr_batch_set_tuning(None, (512, 64, 0))
    # pipelines: null handles and buffers are rejected on the host
    assert rh.load().rhqr_pipeline_create(None, rh.F32, 100, 4, None, 2, ctypes.byref(out)) == 1
    assert rh.load().rhqr_pipeline_create(None, rh.F32, 100, 4, None, 2, None) == 1
    assert rh.load().rhqr_pipeline_submit(None, None, 0, None, 0, None, None, 0, None, None) == 1
    assert rh.load().rhqr_pipeline_wait(None) == 1
    assert rh.load().rhqr_pipeline_destroy(None) == 0
    # GMRES solution: null handles and buffers are rejected on the host
    assert rh.load().rhqr_arnoldi_solution(None, None, 0, 1, None, None, None, None, None, None) == 1


def test_last_cuda_error_query_without_a_gpu():
    """rhqr_last_cuda_error is 0 until a call returns RHQR_ECUDA, and
    rhqr_cuda_error_name gives the CUDA runtime's name for a code (host only)."""
    import paper_2405_10923_gb300 as rh

    lib = rh.load()
    code, name = rh.rhqr_last_cuda_error()
    assert code == 0 and name == "cudaSuccess"
    assert lib.rhqr_cuda_error_name(912).decode() == "cudaErrorInvalidClusterSize"
