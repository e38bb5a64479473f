"""FCIDUMP reading (the paper's interface format, Sec. X) through the C ABI
(no GPU), the integral-grid reading on the oracle, and one GPU run from a
file with tiny entries."""
import numpy as np
import pytest

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


def tiny_entry_integrals(seed=31):
    """An 8-orbital synthetic system whose FCIDUMP carries, beside O(10) Eh
    values, entries of 1e-12 .. 1e-20 Eh (as printed integral files do), so
    that no 128-bit fixed-point grid holds every integral exactly."""
    h, eri = workloads.synthetic_abinitio(8, 24, seed)
    rng = np.random.default_rng(seed)
    idx = rng.choice(eri.size, 40, replace=False)
    eri = eri.copy()
    eri[idx] = rng.choice([-1.0, 1.0], 40) * 10.0 ** rng.uniform(-20.0, -12.0, 40)
    h = h.copy()
    h[0, 7] = h[7, 0] = 3.3e-19
    h[2, 5] = h[5, 2] = -7.1e-17
    return h, eri


def test_fcidump_with_tiny_integrals_reads_exactly(tmp_path):
    import paper_2006_14956_gb300 as fq
    h, eri = tiny_entry_integrals()
    p = tmp_path / "FCIDUMP"
    workloads.write_fcidump(p, h, eri, 3, 3)
    sysd = fq.fciqmc_read_fcidump(p)
    np.testing.assert_array_equal(sysd["h1"], h)
    np.testing.assert_array_equal(sysd["eri"], eri)


def test_oracle_integral_grid_rounds_at_the_stated_scale():
    """Reading: where the integrals' finest bit lies beyond what the 128-bit
    exact sums allow, every integral is rounded to the nearest multiple of
    2^-G, G = 125 - m - 2 - max(ceil(log2(n^2 + 2n + 4)), ceil(log2(N^2)) + 2)
    (m = floor(log2 max |integral|)).  Pinned on a system where that rounding
    is the whole of H_ii - E_ref: 4 orbitals, one alpha and one beta electron,
    h = identity, and only tiny (pp|qq) = 1e-30 .. 1e-36 Eh, so
    H_ii - E_ref = (pp|qq) - (00|00) exactly before rounding.  The oracle must
    stay within two half-grid steps of that, must move a value planted at
    0.75 of a grid step, and a grid 30 bits coarser breaks the bound."""
    from fractions import Fraction
    import oracle
    N = 4
    h = np.eye(N)
    npair = N * (N + 1) // 2
    eri = np.zeros(npair * (npair + 1) // 2)

    def pidx(p, q):
        return p * (p + 1) // 2 + q if p >= q else q * (q + 1) // 2 + p

    G = 125 - 0 - 2 - max(4, 4 + 2)   # n = 2: 12 -> 4 bits; N^2 = 16 -> 4 bits
    rng = np.random.default_rng(8)
    vals = {}
    for p in range(N):
        for q in range(p, N):
            k = pidx(pidx(p, p), pidx(q, q))
            v = float(rng.uniform(1.0, 9.0) * 10.0 ** rng.integers(-36, -29))
            eri[k] = v
            vals[(p, q)] = vals[(q, p)] = Fraction(v)
    eri[pidx(pidx(1, 1), pidx(2, 2))] = 0.75 * 2.0 ** -G
    vals[(1, 2)] = vals[(2, 1)] = Fraction(3, 4) / 2 ** G
    s = oracle.System.abinitio(h, eri, 1, 1)
    half = Fraction(1, 2 ** (G + 1))
    ref = vals[(0, 0)]
    worst = Fraction(0)
    for p in range(N):
        for q in range(N):
            got = Fraction(s.hdiag_rel(1 << p, 1 << q))
            exact = vals[(p, q)] - ref
            assert abs(got - exact) <= 2 * half, (p, q, float(got), float(exact))
            worst = max(worst, abs(got - exact))
    # the rounding is in force (unrounded sums would agree to ~1e-46) ...
    assert worst > half / 4
    # ... and on this grid, not a coarser one: a grid 30 bits coarser rounds
    # every entry here to zero, off by max |exact| >> the bound
    assert max(abs(vals[(p, q)] - ref) for p in range(N) for q in range(N)) > 1000 * 2 * half


def test_oracle_tiny_integrals_do_not_move_ordinary_diagonals():
    """The 8-orbital system with 1e-12 .. 1e-20 Eh entries: H_ii - E_ref of
    the oracle stays within (terms) 2^-(G+1) plus one rounding of the exact
    rational value from the original integrals."""
    import itertools
    from fractions import Fraction
    import oracle
    h, eri = tiny_entry_integrals()
    s = oracle.System.abinitio(h, eri, 3, 3)
    norb, n = 8, 6
    msb = max(int(np.floor(np.log2(np.max(np.abs(h))))), int(np.floor(np.log2(np.max(np.abs(eri))))))
    tb = int(np.ceil(np.log2(n * n + 2 * n + 4)))
    G = 125 - msb - 2 - max(tb, int(np.ceil(np.log2(norb * norb))) + 2)

    def pidx(p, q):
        return p * (p + 1) // 2 + q if p >= q else q * (q + 1) // 2 + p

    def eri4(p, q, r, t):
        return Fraction(float(eri[pidx(pidx(p, q), pidx(r, t))]))

    def hdiag_exact(a, b):
        occ = [(p, 0) for p in range(norb) if (a >> p) & 1] + [(p, 1) for p in range(norb) if (b >> p) & 1]
        x = sum(Fraction(float(h[p, p])) for p, _ in occ)
        for (p, sp), (q, sq) in itertools.combinations(occ, 2):
            x += eri4(p, p, q, q) - (eri4(p, q, q, p) if sp == sq else 0)
        return x

    xref = hdiag_exact(*s.ref)
    bound = Fraction(2 * (n + n * (n - 1) // 2), 2 ** (G + 1))
    dets = s.determinants()
    rng = np.random.default_rng(3)
    for k in rng.choice(len(dets), 300, replace=False):
        a, b = dets[k]
        exact = hdiag_exact(a, b) - xref
        got = Fraction(s.hdiag_rel(a, b))
        assert abs(got - exact) <= bound + abs(exact) * Fraction(1, 2 ** 52), (a, b)


@pytest.mark.gpu
def test_gpu_run_from_fcidump_with_tiny_integrals_matches_oracle(tmp_path):
    """fciqmc_read_fcidump -> fciqmc_create accepts the file with 1e-12 ..
    1e-20 Eh entries (integrals rounded to the 128-bit grid, the reading
    above) and the run agrees bit for bit with the oracle given the original
    arrays, with the uniform and the heat-bath generator."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    import paper_2006_14956_gb300 as fq
    from tests.test_gpu_parity import DAMP, assert_states_equal, assert_stats_equal
    h, eri = tiny_entry_integrals()
    p = tmp_path / "FCIDUMP"
    workloads.write_fcidump(p, h, eri, 3, 3)
    sysd = fq.fciqmc_read_fcidump(p)
    for gen in (0, 1):
        params = dict(DAMP, tau=0.004, target_walkers=2500, initiator_threshold=3.0, seed=21, generator=gen)
        g = fq.fciqmc_create(sysd, params)
        o = oracle.Run(oracle.System.abinitio(h, eri, 3, 3), **params)
        fq.fciqmc_step(g, 150)
        o.step(150)
        assert_states_equal(fq.fciqmc_export_state(g), o.export())
        assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())
