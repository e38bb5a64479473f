"""Adaptive shift (Sec. V) on the GPU against the oracle.

The local shift f_i S of a non-initiator depends on which of its spawns the
initiator rule accepts and on |H_ji| / |H_jj - E_ref - S| of each; the sums
are exact (weights truncated to 2^-64), so walker lists and statistics must
agree bit for bit, as for the plain method.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import DAMP, _fq, assert_states_equal, assert_stats_equal

pytestmark = pytest.mark.gpu

ADAPT = dict(adaptive_shift=1)

CASES = {
    "abinitio_8_3_3": (workloads.small_abinitio(8, 3, 3, seed=5),
                       dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11), 250),
    "hubbard_4x4": (workloads.hubbard_2d(4, 4, 4.0),
                    dict(tau=0.005, target_walkers=5000, initiator_threshold=3.0, seed=7), 250),
    "abinitio_cmin_half_pchb": (workloads.small_abinitio(7, 3, 2, seed=8),
                                dict(tau=0.004, target_walkers=1500, c_min=0.5, initiator_threshold=2.0, seed=5,
                                     generator=1), 200),
    "abinitio_semistoch": (workloads.small_abinitio(8, 3, 3, seed=5),
                           dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11,
                                semistoch_size=60, semistoch_start=5), 200),
    # 3e5 walkers on the reference: its attempts go through the sliced heavy
    # path, whose slices carry the parent's slot for the weight sums (a
    # non-zero shift, held fixed below the target, so that f_i S differs from S)
    "abinitio_heavy": (workloads.small_abinitio(8, 3, 3, seed=21),
                       dict(tau=0.002, target_walkers=1e9, initial_walkers=3e5, initiator_threshold=3.0, seed=4,
                            initial_shift=-2.0), 6),
    "abinitio_trial": (workloads.small_abinitio(8, 3, 3, seed=5),
                       dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11, trial_size=25,
                            trial_start=5), 200),
}


def run_pair(sysd, params, n, chunks=2):
    fq = _fq()
    params = dict(DAMP, **params, **ADAPT)
    g = fq.fciqmc_create(sysd, params)
    o = oracle.Run(oracle.system_from_workload(sysd), **{k: v for k, v in params.items() if k != "max_dets"})
    for _ in range(chunks):
        fq.fciqmc_step(g, n // chunks)
        o.step(n // chunks)
    return fq, g, o


@pytest.mark.parametrize("name", sorted(CASES))
def test_adaptive_shift_bit_exact(name):
    sysd, params, n = CASES[name]
    fq, g, o = run_pair(sysd, params, n)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())
    # the adaptive shift changed the dynamics
    plain = oracle.Run(oracle.system_from_workload(sysd), **dict(DAMP, **params))
    plain.step(n)
    ep, eo = plain.export(), o.export()
    assert ep["c"].size != eo["c"].size or not np.array_equal(ep["c"], eo["c"])


def test_adaptive_shift_growth_bit_exact():
    """From one bucket: failed iterations discard their weight sums and the
    list index is rebuilt on every new layout."""
    sysd = workloads.hubbard_2d(4, 4, 2.0)
    params = dict(tau=0.005, target_walkers=3e4, initiator_threshold=3.0, seed=17, max_dets=16)
    fq, g, o = run_pair(sysd, params, 300, chunks=1)
    assert fq.fciqmc_layout(g)["buckets"] > 1
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


def test_adaptive_shift_replica_pair_with_set_up_pauses():
    """A replica pair with the adaptive shift and a semi-stochastic space: the
    replicas reach their set-up iterations at different times and must still
    move in lockstep, each identical to the oracle's replica."""
    sysd = workloads.small_abinitio(8, 3, 3, seed=5)
    params = dict(DAMP, tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11, semistoch_size=40,
                  semistoch_start=3, **ADAPT)
    fq = _fq()
    g = fq.fciqmc_create(sysd, dict(params, replicas=2))
    pair = oracle.Pair(oracle.system_from_workload(sysd), **params)
    fq.fciqmc_step(g, 150)
    pair.step(150)
    for r in (0, 1):
        gr = fq.fciqmc_replica(g, r)
        assert_states_equal(fq.fciqmc_export_state(gr), pair.r[r].export())
        assert_stats_equal(fq.fciqmc_iter_stats_get(gr), pair.r[r].stats())
    gs, os_ = fq.fciqmc_iter_stats_get(g), pair.r[0].stats()
    n = len(os_["iter"])
    for k in ("x_overlap", "x_var_num", "x_pt2"):
        a, b = np.asarray(gs[k][-n:]), np.asarray(os_[k])
        scale = max(1.0, float(np.abs(b).max()))
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-9 * scale, err_msg=k)
