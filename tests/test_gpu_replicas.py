"""Replica pairs (Sec. V) and the PT2 correction (Sec. VI) on the GPU against
the oracle.

Each replica's walker list and statistics must agree bit for bit with the
oracle's replica of the same index (replica 1 draws with Philox key word 1);
the cross estimators (overlap, variational numerator, PT2 numerator) are sums
of products accumulated in different orders on the two sides and are
compared within 1e-9 of their scale.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import DAMP, _fq, assert_states_equal, assert_stats_equal

pytestmark = pytest.mark.gpu

CROSS = ("x_overlap", "x_var_num", "x_pt2")


def run_pair(sysd, params, n, chunks=2):
    fq = _fq()
    params = dict(DAMP, **params)
    g = fq.fciqmc_create(sysd, dict(params, replicas=2))
    pair = oracle.Pair(oracle.system_from_workload(sysd),
                       **{k: v for k, v in params.items() if k != "max_dets"})
    for _ in range(chunks):
        fq.fciqmc_step(g, n // chunks)
        pair.step(n // chunks)
    return fq, g, pair


def check_pair(fq, g, pair):
    for r in (0, 1):
        gr = fq.fciqmc_replica(g, r)
        assert_states_equal(fq.fciqmc_export_state(gr), pair.r[r].export())
        assert_stats_equal(fq.fciqmc_iter_stats_get(gr), pair.r[r].stats())
    gs, os_ = fq.fciqmc_iter_stats_get(g), pair.r[0].stats()
    n = len(os_["iter"])
    for k in CROSS:
        a, b = np.asarray(gs[k][-n:]), np.asarray(os_[k])
        assert np.all(np.isfinite(b)) and np.all(np.isfinite(a)), k
        scale = max(1.0, float(np.abs(b).max()))
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-9 * scale, err_msg=k)
    assert np.count_nonzero(os_["x_overlap"]) > 10
    g1 = fq.fciqmc_iter_stats_get(fq.fciqmc_replica(g, 1))
    for k in CROSS:
        assert np.all(np.asarray(g1[k]) == 0.0)


CASES = {
    "abinitio_8_3_3": (workloads.small_abinitio(8, 3, 3, seed=5),
                       dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11), 200),
    "hubbard_4x4": (workloads.hubbard_2d(4, 4, 4.0),
                    dict(tau=0.005, target_walkers=5000, initiator_threshold=3.0, seed=7), 200),
    "abinitio_pchb_cmin_half": (workloads.small_abinitio(7, 3, 2, seed=8),
                                dict(tau=0.004, target_walkers=1500, c_min=0.5, initiator_threshold=2.0, seed=5,
                                     generator=1), 200),
    # both replicas with a trial space: the first replica's finalize sums the
    # trial and the cross estimators together
    "abinitio_trial": (workloads.small_abinitio(8, 3, 3, seed=5),
                       dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11, trial_size=25,
                            trial_start=5), 200),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_replica_pair_matches_oracle(name):
    sysd, params, n = CASES[name]
    fq, g, pair = run_pair(sysd, params, n)
    check_pair(fq, g, pair)
    assert np.count_nonzero(pair.r[0].stats()["x_pt2"]) > 0


def test_replica_pair_growth_keeps_lockstep():
    """From one bucket, both replicas outgrow their buffers; an iteration that
    overflows in one replica is repeated by both, and the bucket layouts stay
    equal, with results identical to the oracle."""
    sysd = workloads.hubbard_2d(4, 4, 2.0)
    params = dict(tau=0.005, target_walkers=3e4, initiator_threshold=3.0, seed=17, max_dets=16)
    fq, g, pair = run_pair(sysd, params, 300, chunks=1)
    l0 = fq.fciqmc_layout(fq.fciqmc_replica(g, 0))
    l1 = fq.fciqmc_layout(fq.fciqmc_replica(g, 1))
    assert l0["buckets"] == l1["buckets"] > 1
    check_pair(fq, g, pair)


def test_variational_energy_and_pt2_on_small_system():
    """8 orbitals, 3+3 electrons, two Cholesky vectors, initiator threshold 3 at
    a small walker number: E_var is variational within its noise and E_var +
    PT2 is within 3 sigma of the exact ground state."""
    fq = _fq()
    sysd = workloads.small_abinitio(8, 3, 3, n_chol=2, seed=5)
    s = oracle.system_from_workload(sysd)
    e0, _, _ = s.exact_ground_state()
    params = dict(tau=0.01, target_walkers=3000, initial_walkers=300.0, initiator_threshold=3.0, seed=21,
                  shift_damping=0.1, shift_interval=10, initial_shift=e0 + 0.5, replicas=2)
    g = fq.fciqmc_create(sysd, params)
    fq.fciqmc_step(g, 4000)
    en = fq.fciqmc_energy(g)
    assert en["pair_samples"] > 1000
    exact = e0 + s.eref
    tot = en["e_var_mean"] + en["pt2_mean"]
    sig = float(np.hypot(en["e_var_sigma"], en["pt2_sigma"]))
    assert en["e_var_mean"] >= exact - 3.0 * en["e_var_sigma"]  # variational up to noise
    assert abs(tot - exact) < 3.0 * sig + 1e-6, en
