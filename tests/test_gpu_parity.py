"""GPU path against the CPU oracle (needs a GB300).

Both sides run the same seeded system and parameters.  Determinant keys,
amplitudes, H_ii - E_ref, flags, walker numbers, shifts and every counter must
agree bit for bit: every random decision is keyed by (determinant, iteration,
attempt), every multi-term sum that feeds the dynamics is an exact sum rounded
once, and both sides evaluate the remaining binary64 expressions in the same
order without fused multiply-adds.  E_num (Eq. (9)) is the exact sum of its
terms truncated to a fixed grid, so it too agrees bit for bit.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

EXACT_STATS = ["iteration", "nw", "shift", "ndet", "attempts", "spawns", "rejected", "annihilated", "e_num", "e_den",
               "vary"]


def _fq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2006_14956_gb300 as fq
    return fq


def bits(x):
    return np.ascontiguousarray(x, np.float64).view(np.uint64)


def assert_states_equal(g, o):
    assert g["alpha"].size == o["alpha"].size, (g["alpha"].size, o["alpha"].size)
    np.testing.assert_array_equal(g["alpha"], o["alpha"])
    np.testing.assert_array_equal(g["beta"], o["beta"])
    np.testing.assert_array_equal(bits(g["c"]), bits(o["c"]))
    np.testing.assert_array_equal(bits(g["hdiag"]), bits(o["hdiag"]))
    np.testing.assert_array_equal(g["flags"], o["flags"])


def assert_stats_equal(gs, os_, first=0):
    n = len(os_["iter"]) - first
    assert len(gs["iteration"]) >= n
    for k in EXACT_STATS:
        ok = {"iteration": "iter", "shift": "S"}.get(k, k)
        a = np.asarray(gs[k][-n:])
        b = np.asarray(os_[ok][first:])
        if a.dtype.kind == "f":
            np.testing.assert_array_equal(bits(a), bits(b), err_msg=k)
        else:
            np.testing.assert_array_equal(a, b, err_msg=k)


# A critically damped shift (zeta/(A tau) * A tau = zeta = 0.5 over A = 5)
# keeps the population near its target, so the oracle finishes in seconds.
DAMP = dict(shift_damping=0.5, shift_interval=5)


def run_pair(sysd, params, n_iter, chunks=1):
    fq = _fq()
    params = dict(DAMP, **params)
    g = fq.fciqmc_create(sysd, params)
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    per = n_iter // chunks
    for _ in range(chunks):
        fq.fciqmc_step(g, per)
        o.step(per)
    return fq, g, o


CASES = {
    "hubbard_ring_8": (workloads.hubbard_1d(8, 1.0, 4.0),
                       dict(tau=0.01, target_walkers=2000, initial_walkers=10.0, seed=1), 500),
    "hubbard_4x4_initiator": (workloads.hubbard_2d(4, 4, 4.0),
                              dict(tau=0.005, target_walkers=5000, initiator_threshold=3.0, seed=7), 300),
    "hubbard_3x4_open": (dict(workloads.hubbard_2d(3, 4, 8.0), periodic_x=False),
                         dict(tau=0.004, target_walkers=3000, initiator_threshold=3.0, seed=3), 250),
    "abinitio_8_3_3": (workloads.small_abinitio(8, 3, 3, seed=5),
                       dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11), 300),
    "abinitio_8_4_2_plain": (workloads.small_abinitio(8, 4, 2, seed=6),
                             dict(tau=0.004, target_walkers=2000, initiator_threshold=0.0, seed=12), 250),
    "abinitio_cmin_half": (workloads.small_abinitio(7, 3, 2, seed=8),
                           dict(tau=0.004, target_walkers=1500, c_min=0.5, initiator_threshold=2.0, seed=5), 200),
    "abinitio_cmin_two": (workloads.small_abinitio(7, 2, 3, seed=9),
                          dict(tau=0.004, target_walkers=1500, c_min=2.0, initiator_threshold=3.0, seed=6), 200),
    "single_electron": (workloads.small_abinitio(6, 1, 0, seed=10),
                        dict(tau=0.01, target_walkers=500, seed=2), 150),
    "doubles_only": (workloads.small_abinitio(7, 2, 2, seed=13),
                     dict(tau=0.004, target_walkers=1500, p_single=0.0, initiator_threshold=3.0, seed=8), 150),
    "singles_only": (workloads.small_abinitio(7, 2, 2, seed=14),
                     dict(tau=0.004, target_walkers=1500, p_single=1.0, seed=9), 150),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_gpu_matches_oracle_bit_exact(name):
    sysd, params, n = CASES[name]
    fq, g, o = run_pair(sysd, params, n, chunks=2)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())
    sh = fq.fciqmc_export_shift(g)
    osh = o.shift_state()
    assert sh["S"] == osh["S"] and sh["vary"] == osh["vary"] and sh["nw_last"] == osh["nw_last"]


# The 24-orbital system's prescribed tau = 1e-3 exceeds 1/sum_j |H_ref,j| (no
# shift can hold the walker number there); these tests use the benchmark's 2e-4.
TAU24 = 2e-4


def test_abinitio_24_orbitals_bit_exact():
    """The 24-orbital, 6+6-electron synthetic system (96 Cholesky vectors,
    initiator threshold 3) at a reduced walker target."""
    sysd, params = workloads.config_abinitio_24()
    params = dict(params, tau=TAU24, target_walkers=2e4)
    fq, g, o = run_pair(sysd, params, 160, chunks=2)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


def test_heavy_determinants_bit_exact():
    """A reference with 3e5 walkers takes the sliced heavy-determinant path."""
    sysd = workloads.small_abinitio(8, 3, 3, seed=21)
    params = dict(tau=0.002, target_walkers=1e9, initial_walkers=3e5, initiator_threshold=3.0, seed=4)
    fq, g, o = run_pair(sysd, params, 6)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())
    assert o.stats()["attempts"][0] >= 3e5


def test_capacity_growth_is_bit_identical():
    """Starting from one bucket, the list outgrows its buffers several times;
    each overflowing iteration is repeated after growth with identical results."""
    fq = _fq()
    sysd = workloads.hubbard_2d(4, 4, 2.0)
    params = dict(DAMP, tau=0.005, target_walkers=3e4, initiator_threshold=3.0, seed=17, max_dets=16)
    g = fq.fciqmc_create(sysd, params)
    assert fq.fciqmc_layout(g)["buckets"] == 1
    o = oracle.Run(oracle.system_from_workload(sysd), **{k: v for k, v in params.items() if k != "max_dets"})
    fq.fciqmc_step(g, 300)
    o.step(300)
    assert fq.fciqmc_layout(g)["buckets"] > 1
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


@pytest.mark.parametrize("name,sysd,params", [
    ("hubbard_1d_8", workloads.hubbard_1d(8, 1.0, 4.0),
     dict(tau=0.01, target_walkers=2000, seed=11, max_dets=40000, initiator_threshold=3.0)),
    ("abinitio_24_orbitals", workloads.config_abinitio_24()[0],
     dict(workloads.config_abinitio_24()[1], tau=2e-4, target_walkers=2e4, max_dets=5000000)),
])
def test_export_import_device_and_host_fallback_agree(name, sysd, params):
    """The export sorts on the device (compaction, radix sort over the
    orbital bits, gather) and the import places on the device; a run whose
    memory cap leaves no room for their scratch does both on the host.  Both
    must give the oracle's list, before and after further iterations."""
    fq = _fq()
    params = dict(DAMP, **params)
    g = fq.fciqmc_create(sysd, params)
    b0 = fq.fciqmc_layout(g)
    fq.fciqmc_step(g, 150)
    b1 = fq.fciqmc_layout(g)
    assert (b0["buckets"], b0["cap_spawn"]) == (b1["buckets"], b1["cap_spawn"])  # no growth: the capped twin fits
    tight = fq.fciqmc_create(sysd, dict(params, max_device_bytes=b1["device_bytes"] + 4096))
    fq.fciqmc_step(tight, 150)
    o = oracle.Run(oracle.system_from_workload(sysd), **{k: v for k, v in params.items() if k != "max_dets"})
    o.step(150)
    dev, host = fq.fciqmc_export_state(g), fq.fciqmc_export_state(tight)
    assert dev["alpha"].size > 100
    assert_states_equal(dev, o.export())
    assert_states_equal(host, o.export())
    # import the same way round: placed by kernels (g) or laid out on the host
    # (tight: no room for the scratch); H_ii by the slot-list kernel or per
    # bucket; both lists, and the runs continued from them, must agree
    sh = fq.fciqmc_export_shift(g)
    args = (sh["iteration"], sh["S"], sh["vary"], sh["shift_start"], sh["cnt"], sh["nw_last"])
    for h in (g, tight):
        fq.fciqmc_import_state(h, dev["alpha"], dev["beta"], dev["c"], *args)
    assert_states_equal(fq.fciqmc_export_state(g), dev)
    assert_states_equal(fq.fciqmc_export_state(tight), dev)
    fq.fciqmc_step(g, 20)
    fq.fciqmc_step(tight, 20)
    o.step(20)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_states_equal(fq.fciqmc_export_state(tight), o.export())


def test_export_into_caller_arrays():
    """fciqmc_export_state(h, out=...) fills caller-owned arrays (here larger
    than the list) with the same list as the allocating form; arrays of the
    wrong type or too small are not used."""
    fq = _fq()
    sysd, params = workloads.small_abinitio(8, 3, 3, seed=5), dict(DAMP, tau=0.005, target_walkers=3000,
                                                                    initiator_threshold=3.0, seed=11)
    g = fq.fciqmc_create(sysd, params)
    fq.fciqmc_step(g, 120)
    ref = fq.fciqmc_export_state(g)
    n = ref["c"].size
    types = dict(alpha=np.uint64, beta=np.uint64, c=np.float64, hdiag=np.float64, flags=np.int32)
    out = {k: np.full(n + 77, 7, t) for k, t in types.items()}
    got = fq.fciqmc_export_state(g, out=out)
    assert_states_equal(got, ref)
    for k in types:
        assert np.shares_memory(got[k], out[k])
    small = {k: np.zeros(max(n - 1, 1), t) for k, t in types.items()}
    assert_states_equal(fq.fciqmc_export_state(g, out=small), ref)
    wrong = dict(out, c=np.zeros(n + 77, np.float32))
    got2 = fq.fciqmc_export_state(g, out=wrong)
    assert_states_equal(got2, ref)
    assert not np.shares_memory(got2["alpha"], out["alpha"])


def test_checkpoint_restart_continues_identically():
    fq = _fq()
    sysd, params = workloads.small_abinitio(8, 3, 3, seed=5), dict(DAMP, tau=0.005, target_walkers=3000,
                                                                    initiator_threshold=3.0, seed=11)
    g1 = fq.fciqmc_create(sysd, params)
    fq.fciqmc_step(g1, 200)
    st = fq.fciqmc_export_state(g1)
    sh = fq.fciqmc_export_shift(g1)
    g2 = fq.fciqmc_create(sysd, params)
    fq.fciqmc_import_state(g2, st["alpha"], st["beta"], st["c"], sh["iteration"], sh["S"], sh["vary"],
                           sh["shift_start"], sh["cnt"], sh["nw_last"])
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    o.import_state(st["alpha"], st["beta"], st["c"], sh["iteration"], sh["S"], sh["vary"], sh["shift_start"],
                   sh["cnt"], sh["nw_last"])
    assert_states_equal(fq.fciqmc_export_state(g2), o.export())
    fq.fciqmc_step(g1, 50)
    fq.fciqmc_step(g2, 50)
    o.step(50)
    s1, s2 = fq.fciqmc_export_state(g1), fq.fciqmc_export_state(g2)
    assert_states_equal(s1, s2)
    assert_states_equal(s2, o.export())


def test_import_rejects_bad_input_and_keeps_the_run_usable():
    """A wrong electron count or hundreds of copies of one key (more than a
    bucket holds at any bucket count) are refused with INVALID_ARG before
    anything changes; a valid import afterwards continues as a fresh handle."""
    fq = _fq()
    sysd, params = workloads.small_abinitio(8, 3, 3, seed=5), dict(DAMP, tau=0.005, target_walkers=3000,
                                                                    initiator_threshold=3.0, seed=11)
    g1 = fq.fciqmc_create(sysd, params)
    fq.fciqmc_step(g1, 100)
    st, sh = fq.fciqmc_export_state(g1), fq.fciqmc_export_shift(g1)
    args = (sh["iteration"], sh["S"], sh["vary"], sh["shift_start"], sh["cnt"], sh["nw_last"])
    a0 = int(st["alpha"][3])
    free = next(p for p in range(8) if not (a0 >> p) & 1)
    bad_a = st["alpha"].copy()
    bad_a[3] = np.uint64(a0 | (1 << free))  # one alpha electron too many
    for a, b, c in [(bad_a, st["beta"], st["c"]),
                    (np.repeat(st["alpha"][:1], 600), np.repeat(st["beta"][:1], 600), np.ones(600))]:
        with pytest.raises(fq.FciqmcError) as e:
            fq.fciqmc_import_state(g1, a, b, c, *args)
        assert e.value.code == fq.FCIQMC_ERR_INVALID_ARG
    fq.fciqmc_import_state(g1, st["alpha"], st["beta"], st["c"], *args)
    g2 = fq.fciqmc_create(sysd, params)
    fq.fciqmc_import_state(g2, st["alpha"], st["beta"], st["c"], *args)
    fq.fciqmc_step(g1, 30)
    fq.fciqmc_step(g2, 30)
    assert_states_equal(fq.fciqmc_export_state(g1), fq.fciqmc_export_state(g2))


def test_energy_within_3sigma_of_exact_diagonalisation():
    """8-site Hubbard ring, U=4, plain FCIQMC (n_a = 0), 2000 iterations at
    1e4 walkers: E_proj within 3 sigma of the exact ground state."""
    fq = _fq()
    sysd, params = workloads.config_hubbard_ring()
    s = oracle.system_from_workload(sysd)
    e0, _, _ = s.exact_ground_state()
    g = fq.fciqmc_create(sysd, dict(params, initial_shift=e0 + 0.3, initial_walkers=500.0))
    fq.fciqmc_step(g, 2500)
    en = fq.fciqmc_energy(g)
    assert en["n_samples"] > 1000
    assert abs(en["e_proj_mean"] - (e0 + s.eref)) < 3.0 * en["e_proj_sigma"] + 1e-9, en
    assert en["e_proj_sigma"] < 0.05


def test_energy_statistics_match_the_oracle_estimator():
    """fciqmc_energy's E_proj, shift and their blocking errors (host code of
    the library) against the oracle's estimator applied to the same rows of
    the run's statistics: the same blocking level must be chosen, so the
    means agree to rounding and the errors to the rounding of the variance
    sums."""
    fq = _fq()
    sysd, params = workloads.config_hubbard_ring()
    s = oracle.system_from_workload(sysd)
    e0, _, _ = s.exact_ground_state()
    g = fq.fciqmc_create(sysd, dict(params, initial_shift=e0 + 0.3, initial_walkers=500.0, seed=5))
    fq.fciqmc_step(g, 3000)
    en = fq.fciqmc_energy(g)
    st = fq.fciqmc_iter_stats_get(g)
    sel = st["iteration"] >= en["equil_start"]
    assert en["n_samples"] == int(np.sum(sel)) > 1000
    r, sg = oracle.ratio_estimate(st["e_num"][sel], st["e_den"][sel])
    eref = s.eref
    np.testing.assert_allclose(en["e_proj_mean"] - eref, r, rtol=1e-12)
    np.testing.assert_allclose(en["e_proj_sigma"], sg, rtol=1e-9)
    ms, ss, _ = oracle.blocking(st["shift"][sel])
    np.testing.assert_allclose(en["shift_mean"] - eref, ms, rtol=1e-12)
    np.testing.assert_allclose(en["shift_sigma"], ss, rtol=1e-9)
    assert 0.0 < en["e_proj_sigma"] < 0.05


def test_full_size_sampled_parity_abinitio_24():
    """At the full 1e6-walker size of the 24-orbital system, in the launch
    configuration the benchmark times: the GPU state after equilibration is
    handed to the oracle, and one further iteration must agree bit for bit
    over the whole list."""
    fq = _fq()
    sysd, params = workloads.config_abinitio_24()
    params = dict(params, tau=TAU24, initial_walkers=6.25e5, target_walkers=6.25e5, shift_damping=1.0,
                  shift_interval=2)
    g = fq.fciqmc_create(sysd, params)
    fq.fciqmc_step(g, 300)
    st = fq.fciqmc_export_state(g)
    sh = fq.fciqmc_export_shift(g)
    assert st["c"].size > 1e5
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    o.import_state(st["alpha"], st["beta"], st["c"], sh["iteration"], sh["S"], sh["vary"], sh["shift_start"],
                   sh["cnt"], sh["nw_last"])
    fq.fciqmc_step(g, 1)
    o.step(1)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    gs = fq.fciqmc_iter_stats_get(g)
    os_ = o.stats()
    for k in ["nw", "shift", "ndet", "attempts", "spawns", "rejected", "annihilated"]:
        ok = {"shift": "S"}.get(k, k)
        if gs[k].dtype.kind == "f":
            assert bits(gs[k][-1:])[0] == bits(os_[ok][-1:])[0], k
        else:
            assert gs[k][-1] == os_[ok][-1], k


@pytest.mark.parametrize("name,sysd,params,n", [
    ("abinitio_8_D60", workloads.small_abinitio(8, 3, 3, seed=5),
     dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11, semistoch_size=60, semistoch_start=5), 200),
    ("hubbard_4x4_D200", workloads.hubbard_2d(4, 4, 4.0),
     dict(tau=0.005, target_walkers=5000, initiator_threshold=3.0, seed=7, semistoch_size=200, semistoch_start=3), 200),
    ("abinitio_7_D_ties", workloads.small_abinitio(7, 2, 2, seed=13),
     dict(tau=0.004, target_walkers=800, initial_walkers=800.0, initiator_threshold=0.0, seed=8, semistoch_size=150,
          semistoch_start=1), 150),
])
def test_semistochastic_bit_exact(name, sysd, params, n):
    """Deterministic projection inside D (Sec. III): selection of the N_D most
    populated determinants (ties by key), H^D in CSR, exact update, D -> D
    spawns removed.  Keys, amplitudes, D flags and counters match the oracle."""
    fq, g, o = run_pair(sysd, params, n, chunks=2)
    gs, os_ = fq.fciqmc_export_state(g), o.export()
    assert_states_equal(gs, os_)
    assert int(np.sum((gs["flags"] & 2) > 0)) == o.semistoch_info()[0] > 0
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


def test_semistochastic_whole_space_converges_to_exact_energy():
    """D = the whole space: the GPU iteration is the power method with
    1 - dt (H - S) and E_proj reaches the exact E_0 (Sec. III)."""
    fq = _fq()
    sysd = workloads.hubbard_1d(6, 1.0, 4.0)
    s = oracle.system_from_workload(sysd)
    e0, _, dets = s.exact_ground_state()
    g = fq.fciqmc_create(sysd, dict(tau=0.02, target_walkers=4e4, initial_walkers=4e4, seed=3,
                                    semistoch_size=len(dets), semistoch_start=200, shift_damping=0.5,
                                    shift_interval=5, initial_shift=e0))
    fq.fciqmc_step(g, 2500)
    st = fq.fciqmc_iter_stats_get(g)
    st_state = fq.fciqmc_export_state(g)
    assert st_state["c"].size == len(dets) and np.all((st_state["flags"] & 2) > 0)
    e = st["e_num"][-1] / st["e_den"][-1]
    assert abs(e - e0) < 1e-8, (e, e0)
