"""The C-ABI library builds, loads and exports every entry point that
include/fciqmc.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fciqmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fciqmc_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ["fciqmc_create", "fciqmc_step", "fciqmc_energy", "fciqmc_destroy"]:
        assert core in names


def test_library_exports_every_declared_symbol():
    import paper_2006_14956_gb300 as fq
    lib = ctypes.CDLL(fq.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(fq.EXPORTED)


def test_struct_sizes_match_header_layout():
    import paper_2006_14956_gb300 as fq
    # 8-byte aligned records; a mismatch would corrupt every call
    assert ctypes.sizeof(fq.fciqmc_iter_stats) == 128
    assert ctypes.sizeof(fq.fciqmc_stats) == 208
    assert ctypes.sizeof(fq.fciqmc_system) == 96
    assert ctypes.sizeof(fq.fciqmc_params) == 184


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        import pytest
        pytest.skip("a GPU is present")
    import paper_2006_14956_gb300 as fq
    import workloads
    try:
        fq.fciqmc_create(workloads.hubbard_1d(4), dict(tau=0.01))
    except fq.FciqmcError as e:
        assert e.code in (fq.FCIQMC_ERR_CUDA, fq.FCIQMC_ERR_OUT_OF_MEMORY)
    else:
        raise AssertionError("create succeeded without a GPU")


def test_invalid_arguments_rejected_before_any_device_work():
    import paper_2006_14956_gb300 as fq
    import workloads
    for bad in [dict(tau=float('nan')), dict(c_min=0.0), dict(p_single=1.5), dict(shift_interval=0)]:
        try:
            fq.fciqmc_create(workloads.hubbard_1d(4), bad, use_torch=False)
        except fq.FciqmcError as e:
            assert e.code == fq.FCIQMC_ERR_INVALID_ARG, (bad, e)
        else:
            raise AssertionError(bad)
    try:
        fq.fciqmc_create(dict(workloads.hubbard_1d(4), lx=2), dict(tau=0.01), use_torch=False)
    except fq.FciqmcError as e:
        assert e.code == fq.FCIQMC_ERR_INVALID_ARG
