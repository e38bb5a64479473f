"""Pre-computed heat-bath doubles (App. A) on the GPU against the oracle.

The device builds the alias tables itself, one block per pair of occupied spin
orbitals; the oracle builds them in plain C.  Both follow the same fixed
construction, so the tables must agree bit for bit (sum, |H|/p_gen, coin
thresholds, both hole pairs of every entry), and so must whole runs drawn from
them.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import DAMP, _fq, assert_states_equal, assert_stats_equal, bits

pytestmark = pytest.mark.gpu

PCHB = dict(generator=1)


def oracle_threshold(prob):
    """ceil(prob 2^53) clamped to [0, 2^53]: the integer form of the coin u < prob, u = m 2^-53."""
    p = np.asarray(prob, np.float64)
    t = np.ceil(np.clip(p, 0.0, 1.0) * 2.0 ** 53)
    return t.astype(np.uint64)


def compare_table(g, o, same_spin, i, j):
    gt = _fq().fciqmc_pchb_table(g, same_spin, i, j)
    ot = o.pchb_table(same_spin, i, j)
    assert len(gt["threshold"]) == ot["K"]
    assert bits([gt["S"]])[0] == bits([ot["S"]])[0], (same_spin, i, j)
    assert bits([gt["lam"]])[0] == bits([ot["lam"]])[0], (same_spin, i, j)
    own = (gt["holes"] & 0xffff).astype(np.int64)
    np.testing.assert_array_equal(own & 0xff, ot["a"])
    np.testing.assert_array_equal(own >> 8, ot["b"])
    if ot["S"] > 0.0:  # an empty table is never sampled
        np.testing.assert_array_equal(gt["threshold"], oracle_threshold(ot["prob"]))
        alt = (gt["holes"] >> 16).astype(np.int64)
        np.testing.assert_array_equal(alt & 0xff, ot["a"][ot["alias"]])
        np.testing.assert_array_equal(alt >> 8, ot["b"][ot["alias"]])
    return ot["S"] > 0.0


def test_tables_match_oracle_every_pair_small_system():
    fq = _fq()
    sysd = workloads.small_abinitio(8, 3, 3, seed=5)
    params = dict(tau=0.005, target_walkers=1000, seed=1, **PCHB)
    g = fq.fciqmc_create(sysd, params)
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    N = 8
    nonempty = 0
    for i in range(N):
        for j in range(N):
            nonempty += compare_table(g, o, 0, i, j)
            if i < j:
                nonempty += compare_table(g, o, 1, i, j)
    assert nonempty == N * N + N * (N - 1) // 2


def test_tables_match_oracle_24_orbitals_sampled():
    fq = _fq()
    sysd, params = workloads.config_abinitio_24()
    params = dict(params, tau=2e-4, target_walkers=1e4, **PCHB)
    g = fq.fciqmc_create(sysd, params)
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    rng = np.random.default_rng(3)
    for _ in range(24):
        i, j = (int(x) for x in rng.integers(0, 24, 2))
        compare_table(g, o, 0, i, j)
        if i != j:
            compare_table(g, o, 1, min(i, j), max(i, j))
    compare_table(g, o, 0, 23, 23)
    compare_table(g, o, 1, 22, 23)
    compare_table(g, o, 1, 0, 1)


def run_pair(sysd, params, n_iter, chunks=2):
    fq = _fq()
    params = dict(DAMP, **params, **PCHB)
    g = fq.fciqmc_create(sysd, params)
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    for _ in range(chunks):
        fq.fciqmc_step(g, n_iter // chunks)
        o.step(n_iter // chunks)
    return fq, g, o


CASES = {
    "abinitio_8_3_3": (workloads.small_abinitio(8, 3, 3, seed=5),
                       dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11), 300),
    "abinitio_8_4_2_plain": (workloads.small_abinitio(8, 4, 2, seed=6),
                             dict(tau=0.004, target_walkers=2000, initiator_threshold=0.0, seed=12), 250),
    "doubles_only": (workloads.small_abinitio(7, 2, 2, seed=13),
                     dict(tau=0.004, target_walkers=1500, initial_walkers=300.0, p_single=0.0, initiator_threshold=3.0,
                          seed=8), 150),
    "same_spin_only": (workloads.small_abinitio(8, 4, 0, seed=15),
                       dict(tau=0.004, target_walkers=1000, initiator_threshold=2.0, seed=10), 150),
    "cmin_half": (workloads.small_abinitio(7, 3, 2, seed=8),
                  dict(tau=0.004, target_walkers=1500, c_min=0.5, initiator_threshold=2.0, seed=5), 200),
    "two_electrons": (workloads.small_abinitio(6, 1, 1, seed=16),
                      dict(tau=0.01, target_walkers=500, initial_walkers=200.0, seed=2), 150),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_pchb_runs_bit_exact(name):
    sysd, params, n = CASES[name]
    fq, g, o = run_pair(sysd, params, n)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


def test_pchb_heavy_determinants_bit_exact():
    """3e5 walkers on the reference: the sliced heavy path draws from the tables too."""
    sysd = workloads.small_abinitio(8, 3, 3, seed=21)
    params = dict(tau=0.002, target_walkers=1e9, initial_walkers=3e5, initiator_threshold=3.0, seed=4)
    fq, g, o = run_pair(sysd, params, 6, chunks=1)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


def test_pchb_24_orbitals_bit_exact():
    sysd, params = workloads.config_abinitio_24()
    params = dict(params, tau=2e-4, target_walkers=2e4)
    fq, g, o = run_pair(sysd, params, 160)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


def test_pchb_semistochastic_bit_exact():
    sysd = workloads.small_abinitio(8, 3, 3, seed=5)
    params = dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11, semistoch_size=60,
                  semistoch_start=5)
    fq, g, o = run_pair(sysd, params, 200)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


def test_pchb_energy_within_3sigma_of_exact_diagonalisation():
    """8 orbitals, 3+3 electrons (3136 determinants), two Cholesky vectors (a
    reference-dominated ground state), plain FCIQMC (n_a = 0) with heat-bath
    doubles: E_proj within 3 sigma of the exact ground state."""
    fq = _fq()
    sysd = workloads.small_abinitio(8, 3, 3, n_chol=2, seed=5)
    s = oracle.system_from_workload(sysd)
    e0, _, _ = s.exact_ground_state()
    params = dict(tau=0.01, target_walkers=2e4, initial_walkers=200.0, initiator_threshold=0.0, seed=17,
                  shift_damping=0.1, shift_interval=10, initial_shift=e0 + 0.5, **PCHB)
    g = fq.fciqmc_create(sysd, params)
    fq.fciqmc_step(g, 4000)
    en = fq.fciqmc_energy(g)
    assert en["n_samples"] > 1000
    assert abs(en["e_proj_mean"] - (e0 + s.eref)) < 3.0 * en["e_proj_sigma"] + 1e-9, en
    assert en["e_proj_sigma"] < 0.03
