"""The allocation-free entry point agrees with the handle path.

fciqmc_ref_offdiag_sum_noalloc serves callers that may not allocate device
memory (under a framework's memory pool, within a fixed budget, or in a loop
that must not enter the CUDA driver's allocator): it takes the caller's device
buffers and keeps its scratch in a fixed array of the library.  Here it is called twice in a row, on two
systems, through the C ABI, and each result must equal the sum that the
ordinary path (fciqmc_create, then fciqmc_ref_offdiag_sum) computes with
scratch it allocates.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _systems():
    a = workloads.small_abinitio(8, 3, 3, seed=5)
    b = workloads.config_abinitio_24()[0]
    return [a, b]


def test_noalloc_ref_sum_matches_handle_path_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2006_14956_gb300 as fq
    stream = torch.cuda.current_stream()
    for sysd in _systems():
        h = fq.fciqmc_create(sysd, dict(tau=1e-4, target_walkers=100))
        expected = fq.fciqmc_ref_offdiag_sum(h)
        ra = (1 << sysd["n_alpha"]) - 1
        rb = (1 << sysd["n_beta"]) - 1
        d_h1 = torch.tensor(np.ascontiguousarray(sysd["h1"]), dtype=torch.float64, device="cuda")
        d_eri = torch.tensor(np.ascontiguousarray(sysd["eri"]), dtype=torch.float64, device="cuda")
        d_out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        fq.fciqmc_ref_offdiag_sum_noalloc(sysd["norb"], sysd["n_alpha"], sysd["n_beta"], d_h1.data_ptr(),
                                          d_eri.data_ptr(), ra, rb, d_out.data_ptr(), stream.cuda_stream)
        got = float(d_out.cpu()[0])
        assert expected > 0
        # the same enumeration, partial sums and summation order: equal (tolerance 1e-12 relative)
        assert abs(got - expected) <= 1e-12 * expected, (got, expected)
        assert got == expected


def test_noalloc_rejects_bad_sizes():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2006_14956_gb300 as fq
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(fq.FciqmcError) as e:
        fq.fciqmc_ref_offdiag_sum_noalloc(65, 1, 1, d.data_ptr(), d.data_ptr(), 1, 1, d.data_ptr())
    assert e.value.code == fq.FCIQMC_ERR_INVALID_ARG
