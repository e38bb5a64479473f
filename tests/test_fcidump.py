"""FCIDUMP reading (the paper's interface format, Sec. X) through the C ABI;
needs no GPU."""
import numpy as np

import workloads


def test_fcidump_roundtrip(tmp_path):
    import paper_2006_14956_gb300 as fq
    h, eri = workloads.synthetic_abinitio(7, 20, 3)
    p = tmp_path / "FCIDUMP"
    workloads.write_fcidump(p, h, eri, 3, 2, ecore=1.25)
    sysd = fq.fciqmc_read_fcidump(p)
    assert (sysd["norb"], sysd["n_alpha"], sysd["n_beta"]) == (7, 3, 2)
    assert sysd["ecore"] == 1.25
    np.testing.assert_array_equal(sysd["h1"], h)
    np.testing.assert_array_equal(sysd["eri"], eri)


def test_fcidump_rejects_bad_files(tmp_path):
    import paper_2006_14956_gb300 as fq
    p = tmp_path / "bad"
    p.write_text(" &FCI NORB=3, &END\n1.0 1 1 1 1\n")
    try:
        fq.fciqmc_read_fcidump(p)
    except fq.FciqmcError as e:
        assert e.code == fq.FCIQMC_ERR_INVALID_ARG
    else:
        raise AssertionError("accepted a namelist without NELEC")
    p.write_text(" &FCI NORB=3,NELEC=2,MS2=0, &END\n1.0 9 1 1 1\n")
    try:
        fq.fciqmc_read_fcidump(p)
    except fq.FciqmcError as e:
        assert e.code == fq.FCIQMC_ERR_INVALID_ARG
    else:
        raise AssertionError("accepted an index beyond NORB")
