"""Trial-wave-function energy estimator (Sec. IV) on the GPU against the oracle.

The trial space T (the N_T largest |C|) must be the same set on both sides;
Psi^T comes from different eigensolvers (parallel Jacobi rotations on the
device, cyclic Jacobi in the oracle), and <Psi^T|H - E_ref|Psi> is summed in
different orders, so E^T, Psi^T and the per-iteration numerator and
denominator are compared within 1e-9 relative (both eigensolvers converge to
1e-15 of the matrix norm; the sums have at most a few 1e5 terms).  The sign
of Psi^T is arbitrary on both sides.  The walker dynamics do not depend on
the estimator and stay bit-exact.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import DAMP, _fq, assert_states_equal, assert_stats_equal

pytestmark = pytest.mark.gpu


def compare_trial(g, o, fq, first_iter):
    gi, oi = fq.fciqmc_trial_info(g), o.trial_info()
    assert gi["nt"] == oi["nt"] > 0
    np.testing.assert_array_equal(gi["alpha"], oi["a"])
    np.testing.assert_array_equal(gi["beta"], oi["b"])
    assert gi["n_w"] == oi["n_w"]
    assert abs(gi["ET"] - oi["ET"]) <= 1e-10 * max(1.0, abs(oi["ET"]))
    sgn = 1.0 if float(gi["cT"] @ oi["cT"]) > 0 else -1.0
    np.testing.assert_allclose(sgn * gi["cT"], oi["cT"], rtol=0, atol=1e-9)
    gs, os_ = fq.fciqmc_iter_stats_get(g), o.stats()
    n = len(os_["iter"])
    gn, gd = sgn * np.asarray(gs["trial_num"][-n:]), sgn * np.asarray(gs["trial_den"][-n:])
    on, od = os_["t_num"], os_["t_den"]
    sel = np.asarray(os_["iter"]) >= first_iter
    assert sel.sum() > 10 and np.all(od[sel] != 0.0)
    scale_n = np.abs(on[sel]).max()
    scale_d = np.abs(od[sel]).max()
    np.testing.assert_allclose(gn[sel], on[sel], rtol=0, atol=1e-9 * scale_n)
    np.testing.assert_allclose(gd[sel], od[sel], rtol=0, atol=1e-9 * scale_d)
    assert np.all(gd[~sel] == 0.0) and np.all(od[~sel] == 0.0)


CASES = {
    "abinitio_8_3_3": (workloads.small_abinitio(8, 3, 3, seed=5),
                       dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11, trial_size=40,
                            trial_start=10), 200),
    "hubbard_4x4": (workloads.hubbard_2d(4, 4, 4.0),
                    dict(tau=0.005, target_walkers=5000, initiator_threshold=3.0, seed=7, trial_size=64,
                         trial_start=20), 200),
    "abinitio_semistoch_and_trial": (workloads.small_abinitio(8, 3, 3, seed=5),
                                     dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11,
                                          semistoch_size=60, semistoch_start=5, trial_size=25, trial_start=5), 150),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_trial_estimator_matches_oracle(name):
    fq = _fq()
    sysd, params, n = CASES[name]
    params = dict(DAMP, **params)
    g = fq.fciqmc_create(sysd, params)
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    fq.fciqmc_step(g, n)
    o.step(n)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())
    sh = o.shift_state()
    compare_trial(g, o, fq, sh["shift_start"] + params["trial_start"])


def test_trial_whole_space_gives_exact_energy():
    """T = the whole FCI space (every determinant imported as occupied when T
    is chosen): E_Trial equals E_0 at every iteration, whatever the walkers."""
    fq = _fq()
    sysd = workloads.small_abinitio(6, 2, 2, n_chol=2, seed=5)
    s = oracle.system_from_workload(sysd)
    e0, _, dets = s.exact_ground_state()
    params = dict(tau=0.01, target_walkers=1000, initial_walkers=1000.0, shift_damping=0.3, shift_interval=5,
                  initiator_threshold=0.0, seed=3, trial_size=1024, trial_start=20)
    g = fq.fciqmc_create(sysd, params)
    fq.fciqmc_import_state(g, [d[0] for d in dets], [d[1] for d in dets], np.full(len(dets), 3.0), 100, 0.0,
                           vary=1, shift_start=80, cnt=0, nw_last=int(3 * len(dets)) << 32)
    fq.fciqmc_step(g, 60)
    ti = fq.fciqmc_trial_info(g)
    assert ti["nt"] == len(dets)
    assert abs(ti["ET"] - e0) < 1e-10
    st = fq.fciqmc_iter_stats_get(g)
    sel = np.asarray(st["trial_den"]) != 0.0
    assert sel.sum() > 30
    np.testing.assert_allclose(np.asarray(st["trial_num"])[sel] / np.asarray(st["trial_den"])[sel], e0,
                               rtol=0, atol=1e-9)
    en = fq.fciqmc_energy(g)
    assert abs(en["e_trial_T"] - (e0 + s.eref)) < 1e-9


def test_trial_estimator_on_24_orbitals():
    """The 24-orbital system with a 200-determinant trial space: the table holds
    T and its connected space, and E_Trial has a smaller error than the
    reference estimator over the same iterations."""
    fq = _fq()
    sysd, params = workloads.config_abinitio_24()
    params = dict(params, tau=2e-4, target_walkers=1e5, initial_walkers=1e5, shift_damping=1.0, shift_interval=2,
                  trial_size=200, trial_start=50)
    g = fq.fciqmc_create(sysd, params)
    fq.fciqmc_step(g, 1500)
    ti = fq.fciqmc_trial_info(g)
    assert ti["nt"] == 200 and ti["n_w"] > 200 * 1000
    en = fq.fciqmc_energy(g)
    assert en["trial_samples"] > 500
    assert np.isfinite(en["e_trial_mean"]) and en["e_trial_sigma"] > 0
    assert en["e_trial_sigma"] < en["e_proj_sigma"], en
