"""GPU path against the oracle on systems shaped like the 50-orbital workload.

Tens of orbitals with 10 + 10 electrons put occupied and empty spin orbitals
in bits 32-63 of both occupation words, which the smaller parity cases never
reach: the excitation generators' bit selection, the fermionic signs across
the word's upper half, the packed integral indices of 40-50 orbitals, the
Slater-Condon sums over 20 electrons and the semi-stochastic space of
thousands of determinants (Sec. III) all run here.  Keys, amplitudes,
H_ii - E_ref, flags, walker numbers, shifts and counters must agree with the
oracle bit for bit, as in test_gpu_parity.py.

The largest case follows the benchmark's own workload and launch
configuration (50 orbitals, D = 1e4, the benchmark's parameters): the GPU
state after growth is handed to the oracle, which selects D from it and runs
the next iteration; the whole list must agree.  At the benchmark's full size
(1e8 walkers) the list is checked through properties the oracle computes
from the exported list itself.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import DAMP, _fq, assert_states_equal, assert_stats_equal, bits

pytestmark = pytest.mark.gpu

# time step of the 50-orbital system: 0.5 / sum_j |H_ref,j| (39309 Eh) rounded down
TAU50 = 1.25e-5


def ref_coupling_sum(sysd):
    """sum_j |<D_j|H|D_ref>| over all single and double excitations of the
    reference, by the oracle's Slater-Condon rules."""
    s = oracle.system_from_workload(sysd)
    ra, rb = s.ref
    N = s.norb
    occ = [[p for p in range(N) if (w >> p) & 1] for w in (ra, rb)]
    emp = [[p for p in range(N) if not (w >> p) & 1] for w in (ra, rb)]
    total = 0.0
    ref = (ra, rb)

    def flip(w, rem, add):
        for p in rem:
            w ^= 1 << p
        for p in add:
            w ^= 1 << p
        return w

    for sp in (0, 1):
        for i in occ[sp]:
            for a in emp[sp]:
                t = [ra, rb]
                t[sp] = flip(t[sp], [i], [a])
                total += abs(s.hoff(ref, tuple(t)))
        for ij in itertools.combinations(occ[sp], 2):
            for ab in itertools.combinations(emp[sp], 2):
                t = [ra, rb]
                t[sp] = flip(t[sp], ij, ab)
                total += abs(s.hoff(ref, tuple(t)))
    for i in occ[0]:
        for j in occ[1]:
            for a in emp[0]:
                for b in emp[1]:
                    total += abs(s.hoff(ref, (flip(ra, [i], [a]), flip(rb, [j], [b]))))
    return total


def high_bits_used(state):
    """Number of determinants with an occupied orbital >= 32 in the alpha and in the beta word."""
    return int(np.count_nonzero(state["alpha"] >> np.uint64(32))), int(np.count_nonzero(state["beta"] >> np.uint64(32)))


def run_pair(sysd, params, n_iter, chunks=2):
    fq = _fq()
    params = dict(DAMP, **params)
    g = fq.fciqmc_create(sysd, params)
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    for _ in range(chunks):
        fq.fciqmc_step(g, n_iter // chunks)
        o.step(n_iter // chunks)
    return fq, g, o


def abinitio_40(na=10, nb=10, seed=40):
    h, eri = workloads.synthetic_abinitio(40, 80, seed)
    return dict(kind="abinitio", norb=40, n_alpha=na, n_beta=nb, h1=h, eri=eri, ecore=0.0)


def tau_of(sysd):
    """0.5 / sum_j |H_ref,j|, rounded down to two significant digits."""
    x = 0.5 / ref_coupling_sum(sysd)
    e = int(np.floor(np.log10(x))) - 1
    return float(np.floor(x / 10.0 ** e) * 10.0 ** e)


def check_pair(fq, g, o):
    gs, os_ = fq.fciqmc_export_state(g), o.export()
    assert_states_equal(gs, os_)
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())
    sh, osh = fq.fciqmc_export_shift(g), o.shift_state()
    assert sh["S"] == osh["S"] and sh["vary"] == osh["vary"] and sh["nw_last"] == osh["nw_last"]
    return gs


def test_abinitio_50_uniform_bit_exact():
    """The 50-orbital, 10 + 10-electron system (200 Cholesky vectors, seed 4),
    uniform generator, initiator threshold 3, at a 2e4-walker target."""
    sysd, params = workloads.config_abinitio_50()
    params = dict(params, tau=TAU50, target_walkers=2e4, initial_walkers=2e3, semistoch_size=0)
    fq, g, o = run_pair(sysd, params, 120)
    gs = check_pair(fq, g, o)
    na, nb = high_bits_used(gs)
    assert na > 100 and nb > 100, (na, nb)
    assert gs["c"].size > 5000


def test_abinitio_40_pchb_bit_exact():
    """40 orbitals, 10 + 10 electrons, pre-computed heat-bath doubles: the
    alias tables of 40 orbitals (hole pairs up to 39) and runs drawn from them."""
    sysd = abinitio_40()
    tau = tau_of(sysd)
    params = dict(tau=tau, target_walkers=2e4, initial_walkers=2e3, initiator_threshold=3.0, seed=41, generator=1)
    fq, g, o = run_pair(sysd, params, 120)
    gs = check_pair(fq, g, o)
    na, nb = high_bits_used(gs)
    assert na > 100 and nb > 100, (na, nb)
    for same, i, j in [(0, 9, 9), (1, 8, 9), (0, 0, 9), (1, 0, 1)]:
        gt = fq.fciqmc_pchb_table(g, same, i, j)
        ot = o.pchb_table(same, i, j)
        assert bits([gt["S"]])[0] == bits([ot["S"]])[0]
        assert bits([gt["lam"]])[0] == bits([ot["lam"]])[0]


def test_abinitio_40_unequal_spins_cmin_half_bit_exact():
    """40 orbitals with 9 alpha and 7 beta electrons, initiator threshold 2,
    c_min = 0.5 (spawn rounding at a power of two other than 1)."""
    sysd = abinitio_40(9, 7, seed=42)
    tau = tau_of(sysd)
    params = dict(tau=tau, target_walkers=1.5e4, initial_walkers=1e3, initiator_threshold=2.0, c_min=0.5, seed=43)
    fq, g, o = run_pair(sysd, params, 100)
    gs = check_pair(fq, g, o)
    na, nb = high_bits_used(gs)
    assert na > 50 and nb > 50, (na, nb)


def test_semistochastic_50_orbitals_ND_2000_bit_exact():
    """Semi-stochastic projection with 2000 determinants in D on the
    50-orbital system: top-N_D selection (ties by key), H^D in CSR from
    Slater-Condon over 20 electrons, the exact update and the removal of
    D -> D spawns."""
    sysd, params = workloads.config_abinitio_50()
    params = dict(params, tau=TAU50, target_walkers=2e4, initial_walkers=2e3, semistoch_size=2000,
                  semistoch_start=8)
    fq, g, o = run_pair(sysd, params, 120)
    gs = check_pair(fq, g, o)
    nd = int(np.sum((gs["flags"] & 2) > 0))
    assert nd == o.semistoch_info()[0] == 2000
    na, nb = high_bits_used(gs)
    assert na > 100 and nb > 100


def grow_until_varying(fq, g, extra, cap):
    """Step until the shift has been varying for `extra` iterations (at most `cap` in all)."""
    done = 0
    while done < cap:
        fq.fciqmc_step(g, 10)
        done += 10
        sh = fq.fciqmc_export_shift(g)
        if sh["vary"] and sh["iteration"] >= sh["shift_start"] + extra:
            return
    raise AssertionError("the walker number did not reach its target in %d iterations" % cap)


def bench_params():
    import bench
    return bench.workload_params(workload="abinitio50")


def test_bench_workload_handoff_one_iteration_with_D_1e4():
    """The benchmark's 50-orbital workload and launch configuration, grown on
    the GPU to a few million walkers; the state is handed to the oracle with
    the semi-stochastic space due at the next iteration, so both select
    D (1e4 determinants) from the same list, build H^D and run one iteration.
    The whole new list and the iteration's statistics must agree."""
    fq = _fq()
    sysd, params = bench_params()
    grow = dict(params, target_walkers=4e6, initial_walkers=4e5, semistoch_size=0)
    g = fq.fciqmc_create(sysd, grow)
    grow_until_varying(fq, g, 10, 400)
    st, sh = fq.fciqmc_export_state(g), fq.fciqmc_export_shift(g)
    assert sh["vary"] == 1 and st["c"].size > 1e6
    args = (sh["iteration"], sh["S"], sh["vary"], sh["shift_start"], sh["cnt"], sh["nw_last"])
    run = dict(params, target_walkers=4e6, initial_walkers=4e5,
               semistoch_start=sh["iteration"] - sh["shift_start"])
    g2 = fq.fciqmc_create(sysd, run)
    fq.fciqmc_import_state(g2, st["alpha"], st["beta"], st["c"], *args)
    o = oracle.Run(oracle.system_from_workload(sysd), **run)
    o.import_state(st["alpha"], st["beta"], st["c"], *args)
    fq.fciqmc_step(g2, 1)
    o.step(1)
    gs, os_ = fq.fciqmc_export_state(g2), o.export()
    assert int(np.sum((gs["flags"] & 2) > 0)) == o.semistoch_info()[0] == 10000
    assert_states_equal(gs, os_)
    gst, ost = fq.fciqmc_iter_stats_get(g2), o.stats()
    for k in ["nw", "shift", "ndet", "attempts", "spawns", "rejected", "annihilated", "e_num", "e_den"]:
        ok = {"shift": "S"}.get(k, k)
        a, b = np.asarray(gst[k][-1:]), np.asarray(ost[ok][-1:])
        if a.dtype.kind == "f":
            assert bits(a)[0] == bits(b)[0], k
        else:
            assert a[0] == b[0], k
    na, nb = high_bits_used(gs)
    assert na > 1000 and nb > 1000


def exact_nw(c):
    """sum floor(|C| 2^32) as an exact integer (|C| < 2^31, so every term and,
    for up to 2^32 walkers, the total fit 64 bits)."""
    f = np.floor(np.abs(c) * 2.0 ** 32).astype(np.uint64)
    return int(np.sum(f, dtype=np.uint64))


def test_bench_workload_full_size_properties():
    """At the benchmark's full size (the 50-orbital workload grown to 1e8
    walkers, D = 1e4, its launch configuration) the exported list is checked
    against what the oracle computes from the list itself: N_w and the
    determinant count of the last iteration, H_ii - E_ref of sampled
    determinants (bit for bit), E_num and E_den of Eq. (9) over the whole
    list, distinct valid keys, the reference and D flags."""
    fq = _fq()
    sysd, params = bench_params()
    g = fq.fciqmc_create(sysd, params)
    grow_until_varying(fq, g, params["semistoch_start"] + 5, 1500)
    lay = fq.fciqmc_layout(g)
    st = fq.fciqmc_export_state(g)
    gst = fq.fciqmc_iter_stats_get(g)
    n = st["c"].size
    assert gst["nw"][-1] > 0.5 * params["target_walkers"], gst["nw"][-1]
    assert gst["ndet"][-1] == n
    # N_w exactly (R10), rounded once
    assert float(exact_nw(st["c"])) * 2.0 ** -32 == gst["nw"][-1]
    # distinct keys with 10 + 10 electrons
    order = np.lexsort((st["beta"], st["alpha"]))
    a, b = st["alpha"][order], st["beta"][order]
    assert not np.any((a[1:] == a[:-1]) & (b[1:] == b[:-1]))
    del order, a, b
    pa = np.unpackbits(st["alpha"].view(np.uint8).reshape(-1, 8), axis=1).sum(axis=1)
    pb = np.unpackbits(st["beta"].view(np.uint8).reshape(-1, 8), axis=1).sum(axis=1)
    assert np.all(pa == 10) and np.all(pb == 10)
    assert not np.any(st["c"] == 0.0) or np.all((st["flags"][st["c"] == 0.0] & 3) > 0)
    # D and the reference
    assert int(np.sum((st["flags"] & 2) > 0)) == 10000
    s = oracle.system_from_workload(sysd)
    ra, rb = s.ref
    iref = np.nonzero((st["alpha"] == np.uint64(ra)) & (st["beta"] == np.uint64(rb)))[0]
    assert iref.size == 1 and (st["flags"][iref[0]] & 1)
    assert bits([st["c"][iref[0]]])[0] == bits([gst["e_den"][-1]])[0]
    # H_ii - E_ref of 3000 sampled determinants by the oracle
    rng = np.random.default_rng(5)
    for i in rng.choice(n, 3000, replace=False):
        assert bits([s.hdiag_rel(int(st["alpha"][i]), int(st["beta"][i]))])[0] == bits([st["hdiag"][i]])[0]
    # E_num = sum_{j != ref} H_ref,j C_j over the list (Eq. (9)), every binary64
    # term truncated to the grid 2^-Fe and summed exactly (R12): bit for bit
    lev = (np.unpackbits((st["alpha"] ^ np.uint64(ra)).view(np.uint8).reshape(-1, 8), axis=1).sum(axis=1) +
           np.unpackbits((st["beta"] ^ np.uint64(rb)).view(np.uint8).reshape(-1, 8), axis=1).sum(axis=1))
    conn = np.nonzero((lev > 0) & (lev <= 4))[0]
    terms = np.array([s.hoff((int(st["alpha"][j]), int(st["beta"][j])), (ra, rb)) * st["c"][j] for j in conn])
    fe = s.enum_grid
    enum = oracle.fsum(np.ldexp(np.trunc(np.ldexp(terms, fe)), -fe))
    assert bits([gst["e_num"][-1]])[0] == bits([enum])[0]
    assert lay["buckets"] >= 1 << 16
