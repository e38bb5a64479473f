"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test ties one part of the oracle to an independent source: a library
routine (numpy Philox, math.fsum, numpy.log), brute-force operator algebra,
closed-form energies, exact enumeration of generation probabilities, and the
exact expectation value of one projector step (Eq. (2) of the paper).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from tests import bruteforce

MASK = (1 << 64) - 1


# ----------------------------------------------------------------- Philox
@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((5, 7), (1, 2, 3, 4)),
                                     ((MASK, 12345), (MASK - 3, 99, 2 ** 63, 17)),
                                     ((0x243F6A8885A308D3, 0x13198A2E03707344), (2 ** 40, 1, 0, 0x1234 << 8 | 1))])
def test_philox_matches_numpy(key, ctr):
    # numpy's Philox is Philox4x64-10; it increments the counter before the first block
    bg = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64))
    raw = bg.random_raw(8)
    c1 = [(ctr[0] + 1) & MASK, ctr[1] + (1 if ctr[0] == MASK else 0), ctr[2], ctr[3]]
    c2 = [(ctr[0] + 2) & MASK, ctr[1] + (1 if ctr[0] >= MASK - 1 else 0), ctr[2], ctr[3]]
    np.testing.assert_array_equal(oracle.philox4x64_10(c1, key), raw[:4])
    np.testing.assert_array_equal(oracle.philox4x64_10(c2, key), raw[4:])


# ----------------------------------------------------------------- exact sums
def test_fsum_matches_math_fsum():
    rng = np.random.default_rng(11)
    cases = [[1e16, 1.0, -1e16], [0.1] * 10, [1e308, 1e308, -1e308], [5e-324, 5e-324, -1e-323],
             [2.0 ** -1074, 1.0, -1.0], [1.0, 2.0 ** -53, 2.0 ** -53], [1.0, 2.0 ** -53],
             [1.0 + 2.0 ** -52, 2.0 ** -53], [-0.0], [], [3.0, -3.0]]
    for _ in range(300):
        n = int(rng.integers(1, 60))
        mag = rng.uniform(-300, 300, size=n)
        x = rng.standard_normal(n) * 10.0 ** mag
        if rng.random() < 0.3:  # heavy cancellation
            x = np.concatenate([x, -x[: n // 2] * (1 + 2.0 ** -50)])
        cases.append(list(x))
    for c in cases:
        exact = float(sum((Fraction(v) for v in c), Fraction(0)))  # correctly rounded exact sum
        assert oracle.fsum(c) == exact, c
        try:
            assert oracle.fsum(c) == math.fsum(c), c
        except OverflowError:  # math.fsum refuses an intermediate overflow
            pass


# ----------------------------------------------------------------- logarithm
def test_ln_within_error_bound():
    rng = np.random.default_rng(3)
    xs = np.concatenate([10.0 ** rng.uniform(-300, 300, 2000), 1.0 + rng.uniform(-0.3, 0.3, 2000),
                         [1.0, 2.0, 0.5, math.sqrt(2.0), np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0),
                          5e-324, 1.7e308]])
    for x in xs:
        got, ref = oracle.ln(float(x)), float(np.log(x))
        tol = 2.0 * np.spacing(abs(ref)) if ref != 0.0 else 0.0
        assert abs(got - ref) <= tol, (x, got, ref)
    assert oracle.ln(1.0) == 0.0


# ----------------------------------------------------------------- Slater-Condon
def _hubbard_integrals(lx, ly, px, py, t, U):
    n = lx * ly
    h = np.zeros((n, n))
    for y in range(ly):
        for x in range(lx):
            p = x + lx * y
            nbrs = []
            if lx > 1:
                nbrs += [((x - 1) % lx, y) if (x > 0 or px) else None, ((x + 1) % lx, y) if (x < lx - 1 or px) else None]
            if ly > 1:
                nbrs += [(x, (y - 1) % ly) if (y > 0 or py) else None, (x, (y + 1) % ly) if (y < ly - 1 or py) else None]
            for nb in nbrs:
                if nb is not None:
                    h[p, nb[0] + lx * nb[1]] = -t
    g = np.zeros((n,) * 4)
    for p in range(n):
        g[p, p, p, p] = U
    return h, g


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (5, 3, 2), (4, 1, 3), (5, 2, 0)])
def test_slater_condon_abinitio_vs_bruteforce(norb, na, nb):
    h, eri = workloads.synthetic_abinitio(norb, 3 * norb, 100 + norb + na)
    ecore = 0.75
    s = oracle.System.abinitio(h, eri, na, nb, ecore)
    dets = s.determinants()
    _, Hrel = s.hamiltonian(dets)
    Hb = bruteforce.hamiltonian(norb, h, bruteforce.eri_full(norb, eri), ecore, dets)
    Ho = Hrel + np.eye(len(dets)) * s.eref
    scale = np.max(np.abs(Hb))
    np.testing.assert_allclose(Ho, Hb, rtol=0, atol=1e-12 * scale)
    # sign and magnitude of every off-diagonal element, symmetric matrix
    np.testing.assert_allclose(Ho, Ho.T, rtol=0, atol=0)


@pytest.mark.parametrize("lx,ly,px,py,na,nb", [(4, 1, 1, 0, 2, 2), (5, 1, 1, 0, 2, 3), (3, 2, 1, 0, 2, 2),
                                               (2, 2, 0, 0, 2, 1)])
def test_slater_condon_hubbard_vs_bruteforce(lx, ly, px, py, na, nb):
    t, U = 1.0, 3.5
    neel = na == nb and 2 * na == lx * ly
    s = oracle.System.hubbard(lx, ly, px, py, t, U, na, nb, ref=None if neel else [(1 << na) - 1, (1 << nb) - 1])
    dets = s.determinants()
    _, Hrel = s.hamiltonian(dets)
    h, g = _hubbard_integrals(lx, ly, px, py, t, U)
    Hb = bruteforce.hamiltonian(lx * ly, h, g, 0.0, dets)
    np.testing.assert_allclose(Hrel + np.eye(len(dets)) * s.eref, Hb, rtol=0, atol=1e-13)


# ----------------------------------------------------------------- exact energies
@pytest.mark.parametrize("lx,ly,na,nb", [(6, 1, 3, 3), (8, 1, 4, 4), (3, 4, 2, 2), (4, 3, 3, 1)])
def test_u0_hubbard_closed_form(lx, ly, na, nb):
    s = oracle.System.hubbard(lx, ly, 1, 1 if ly > 1 else 0, 1.0, 0.0, na, nb,
                              ref=None if (na == nb and 2 * na == lx * ly) else [(1 << na) - 1, (1 << nb) - 1])
    e0, _, _ = s.exact_ground_state()
    exact = oracle.hubbard_u0_energy(lx, ly, 1.0, na, nb)
    assert abs((e0 + s.eref) - exact) < 1e-10
    if (lx, ly) == (8, 1):
        assert abs(exact - 2.0 * (-2.0 - 2.0 * math.sqrt(2.0))) < 1e-12


@pytest.mark.parametrize("U", [0.5, 4.0, 10.0])
def test_two_site_hubbard_closed_form(U):
    s = oracle.System.hubbard(2, 1, 0, 0, 1.0, U, 1, 1, ref=[1, 2])
    e0, _, _ = s.exact_ground_state()
    assert abs((e0 + s.eref) - 0.5 * (U - math.sqrt(U * U + 16.0))) < 1e-12


# ----------------------------------------------------------------- excitation generation
def _word_for(k, m):
    """smallest 64-bit word w with floor(w m / 2^64) == k"""
    return -((-k << 64) // m)


def _enumerate_generator(s, p_single, det, z=2):
    """All discrete outcomes of one generation from ``det`` with their exact
    probabilities; returns {target: probability}, P(fail)."""
    n = s.na + s.nb
    N = s.norb
    ps = Fraction(p_single)
    out = {}
    pfail = Fraction(0)
    def rec(words, prob):
        nonlocal pfail
        cls, tgt = s.generate(p_single, det, words)
        if cls < 0:
            pfail += prob
        else:
            out.setdefault(tgt, []).append((prob, cls))
    if s.kind == "hubbard":
        for e in range(n):
            for k in range(z):
                rec([0, _word_for(e, n), _word_for(k, z), 0], Fraction(1, n * z))
        return out, pfail
    ma, mb = N - s.na, N - s.nb
    single_w0, double_w0 = 0, MASK
    for e in range(n):
        m = ma if e < s.na else mb
        if m == 0:
            rec([single_w0, _word_for(e, n), 0, 0], ps / n)
            continue
        for hh in range(m):
            rec([single_w0, _word_for(e, n), _word_for(hh, m), 0], ps / (n * m))
    if n >= 2:
        for x in range(n * (n - 1)):
            e1, r = divmod(x, n - 1)
            e2 = r + (r >= e1)
            s1, s2 = e1 >= s.na, e2 >= s.na
            base = (1 - ps) / (n * (n - 1))
            if s1 != s2:
                M = ma * mb
            else:
                m = mb if s1 else ma
                M = m * (m - 1)
            if M == 0:
                rec([double_w0, _word_for(x, n * (n - 1)), 0, 0], base)
                continue
            for y in range(M):
                rec([double_w0, _word_for(x, n * (n - 1)), _word_for(y, M), 0], base / M)
    return out, pfail


@pytest.mark.parametrize("which", ["abinitio", "abinitio_asym", "hubbard2d", "hubbard1d"])
def test_pgen_exact_enumeration(which):
    p_single = 0.1
    if which == "abinitio":
        sysd = workloads.small_abinitio(6, 3, 3)
    elif which == "abinitio_asym":
        sysd = workloads.small_abinitio(6, 3, 1)
    elif which == "hubbard2d":
        sysd = workloads.hubbard_2d(3, 4, 4.0)
    else:
        sysd = workloads.hubbard_1d(6, 1.0, 4.0)
    s = oracle.system_from_workload(sysd)
    z = 4 if sysd.get("ly", 1) > 1 else 2
    rng = np.random.default_rng(5)
    dets = s.determinants()
    for det in [s.ref] + [dets[i] for i in rng.choice(len(dets), 5, replace=False)]:
        out, pfail = _enumerate_generator(s, p_single, det, z)
        total = pfail
        for tgt, lst in out.items():
            ptot = sum(p for p, _ in lst)
            cls = lst[0][1]
            assert all(c == cls for _, c in lst)
            # the probability the oracle reports for this class equals the exact one
            assert abs(s.pgen(p_single, cls) - float(ptot)) <= 1e-15 * float(ptot), (tgt, cls)
            total += ptot
            assert tgt != det
            assert bin(tgt[0]).count("1") == s.na and bin(tgt[1]).count("1") == s.nb  # S_z conserved
        assert total == 1
        # every determinant connected to det by a non-zero matrix element is reachable
        for d in dets:
            if d != det and s.hoff(det, d) != 0.0:
                assert d in out, d


def test_generator_frequencies_chi2():
    s = oracle.system_from_workload(workloads.small_abinitio(5, 2, 2))
    det = s.ref
    rng = np.random.default_rng(17)
    n = 40000
    counts = {}
    words = rng.integers(0, 2 ** 63, size=(n, 4), dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=(n, 4), dtype=np.uint64)
    fails = 0
    for w in words:
        cls, tgt = s.generate(0.1, det, w)
        if cls < 0:
            fails += 1
            continue
        counts.setdefault((tgt, cls), 0)
        counts[(tgt, cls)] += 1
    chi2 = 0.0
    for (tgt, cls), k in counts.items():
        e = n * s.pgen(0.1, cls)
        chi2 += (k - e) ** 2 / e
    dof = len(counts)
    assert fails == 0
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


# ----------------------------------------------------------------- projected energy
@pytest.mark.parametrize("which", ["hubbard", "abinitio"])
def test_projected_energy_exact_for_eigenstate(which):
    sysd = workloads.hubbard_1d(6, 1.0, 4.0) if which == "hubbard" else workloads.small_abinitio(6, 3, 2)
    s = oracle.system_from_workload(sysd)
    e0, v, dets = s.exact_ground_state()
    r = oracle.Run(s)
    k = dets.index(s.ref)
    v = v * (1e4 / v[k])
    r.import_state([d[0] for d in dets], [d[1] for d in dets], v, 0, 0.0)
    num, den = r.proj_energy()
    assert abs(num / den - e0) < 1e-10 * max(1.0, abs(e0))


def test_projected_energy_numerator_is_exact_sum_of_truncated_terms():
    """Reading R12: E_num = sum_{j != ref} H_ref,j C_j with every binary64
    product truncated toward zero to a multiple of 2^-Fe, summed exactly and
    rounded once to nearest-even, Fe = min(64, 60 - m - ceil(log2(2n + 1)))
    (m = floor(log2 max |integral|)).  Checked against exact rational
    arithmetic on a list whose amplitudes span 1e-18 .. 1e6, so that some
    products fall below the grid and the in-order binary64 sum differs."""
    sysd = workloads.small_abinitio(8, 3, 3, seed=5)
    s = oracle.system_from_workload(sysd)
    h, eri = np.asarray(sysd["h1"]), np.asarray(sysd["eri"])
    ints = np.concatenate([h.ravel(), eri, [float(sysd.get("ecore", 0.0))]])
    m = max(math.frexp(float(x))[1] - 1 for x in ints if x != 0.0)
    L = math.ceil(math.log2(2 * 6 + 1))
    fe = min(64, 60 - m - L)
    assert s.enum_grid == fe
    dets = s.determinants()
    rng = np.random.default_rng(2)
    c = rng.choice([-1.0, 1.0], len(dets)) * 10.0 ** rng.uniform(-18, 6, len(dets))
    r = oracle.Run(s)
    r.import_state([d[0] for d in dets], [d[1] for d in dets], c, 0, 0.0)
    num, den = r.proj_energy()
    ra, rb = s.ref
    grid = 2 ** fe
    exact = Fraction(0)
    seq = 0.0
    below = 0
    for (a, b), x in zip(dets, c):
        if (a, b) == (ra, rb):
            assert den == x
            continue
        if bin(a ^ ra).count("1") + bin(b ^ rb).count("1") > 4:
            continue
        p = s.hoff((a, b), (ra, rb)) * float(x)  # the binary64 product
        if p == 0.0:
            continue
        f = Fraction(p)
        t = Fraction(math.floor(abs(f) * grid), grid)
        below += t == 0
        exact += t if f > 0 else -t
        seq = seq + p
    assert below > 0
    assert np.float64(num).view(np.uint64) == np.float64(float(exact)).view(np.uint64)
    assert seq != num


# ----------------------------------------------------------------- one projector step
def _expected_step(s, dets, c, tau, S, n_a, Hrel):
    """E[C(t+dt)] for one iteration from amplitudes c (Eq. (4) with the
    initiator rule: a spawn from a non-initiator onto an unoccupied
    determinant is removed)."""
    ref = dets.index(s.ref)
    init = (np.abs(c) > n_a) | (np.arange(len(c)) == ref)
    occ = c != 0.0
    out = c - tau * (np.diag(Hrel) - S) * c
    off = Hrel - np.diag(np.diag(Hrel))
    for j in range(len(c)):
        allowed = init | occ[j]
        out[j] += -tau * np.sum(off[j, :] * c * allowed)
    return out


@pytest.mark.parametrize("case", ["hubbard_plain", "abinitio_plain", "abinitio_initiator", "hubbard_semistoch",
                                  "abinitio_pchb"])
def test_one_step_expectation(case):
    """Averaged over independent seeds, one oracle iteration must reproduce
    (1 - dtau (H - S)) C (plain FCIQMC, Eq. (2)), or its initiator-truncated
    form.  A wrong sign, p_gen, weight, death factor, rounding, initiator
    filter or summation shows up as a biased component."""
    rng = np.random.default_rng(1)
    if case.startswith("hubbard"):
        sysd = workloads.hubbard_1d(6, 1.0, 2.0)
        tau, nseeds = 0.03, 1200
    else:
        sysd = workloads.small_abinitio(5, 2, 2, seed=31)
        tau, nseeds = 0.02, 3000
    s = oracle.system_from_workload(sysd)
    e0, v, dets = s.exact_ground_state()
    _, Hrel = s.hamiltonian(dets)
    n_a = 3.0 if "initiator" in case else 0.0
    if "initiator" in case:
        # half unoccupied, most occupied ones non-initiators: the rule removes a large flux
        c = rng.choice([0.0, 0.0, 2.5, -2.5, 10.0], size=len(dets))
    else:
        c = rng.choice([-1.0, 1.0], size=len(dets)) * rng.uniform(2.0, 12.0, size=len(dets))
    k = dets.index(s.ref)
    c[k] = 20.0
    S = -0.3
    semi = "semistoch" in case
    acc = np.zeros(len(dets))
    acc2 = np.zeros(len(dets))
    index = {d: i for i, d in enumerate(dets)}
    for seed in range(1, nseeds + 1):
        r = oracle.Run(s, tau=tau, seed=seed, initiator_threshold=n_a, initial_shift=S,
                       target_walkers=1e12, semistoch_size=40 if semi else 0, semistoch_start=1,
                       generator=1 if "pchb" in case else 0)
        if semi:
            r.import_state([d[0] for d in dets], [d[1] for d in dets], c, 5, S, vary=1, shift_start=4,
                           cnt=0, nw_last=1 << 70)
        else:
            r.import_state([d[0] for d in dets], [d[1] for d in dets], c, 5, S)
        r.step(1)
        if semi:
            assert r.semistoch_info()[0] == 40
        ex = r.export()
        cn = np.zeros(len(dets))
        for a, b, cc in zip(ex["alpha"], ex["beta"], ex["c"]):
            cn[index[(int(a), int(b))]] = cc
        acc += cn
        acc2 += cn * cn
    mean = acc / nseeds
    var = np.maximum(acc2 / nseeds - mean ** 2, 0.0)
    se = np.sqrt(var / (nseeds - 1))
    exp = _expected_step(s, dets, c, tau, S, n_a, Hrel)
    det_comp = se == 0
    # components with no randomness must be exact
    np.testing.assert_allclose(mean[det_comp], exp[det_comp], rtol=1e-12, atol=1e-12)
    zz = (mean - exp)[~det_comp] / se[~det_comp]
    assert np.max(np.abs(zz)) < 5.0, (np.argmax(np.abs(zz)), np.max(np.abs(zz)))
    chi2 = float(np.sum(zz ** 2))
    assert chi2 < zz.size + 4 * math.sqrt(2 * zz.size), (chi2, zz.size)


# ----------------------------------------------------------------- semi-stochastic limit
def test_semistochastic_whole_space_is_power_method():
    """With D = the whole Hilbert space nothing is sampled: the iteration is the
    deterministic power method with 1 - dtau (H - S), whose projected energy
    converges to the exact E_0 (Sec. III)."""
    s = oracle.system_from_workload(workloads.hubbard_1d(4, 1.0, 4.0))
    e0, v, dets = s.exact_ground_state()
    r = oracle.Run(s, tau=0.05, seed=3, target_walkers=1e12, semistoch_size=len(dets), semistoch_start=1)
    c = np.full(len(dets), 7.0)
    r.import_state([d[0] for d in dets], [d[1] for d in dets], c, 1, e0, vary=1, shift_start=0, cnt=0,
                   nw_last=int(7.0 * len(dets)) << 32)
    r.step(1500)
    assert r.semistoch_info()[0] == len(dets)
    num, den = r.proj_energy()
    assert abs(num / den - e0) < 1e-9


def test_semistochastic_row_sum_is_exact_sum_of_truncated_products():
    """Reading R13: y_k = sum_c H^D_kc C_c with every binary64 product
    truncated toward zero to a multiple of 2^-64, summed exactly and rounded
    once to nearest-even, against exact rational arithmetic (fractions).  The
    amplitudes span 1e-25 .. 1e8 so that products fall on both sides of
    2^-64 and the in-order binary64 sum, or the untruncated exact sum, differ
    from it in some rows."""
    sysd = workloads.small_abinitio(8, 3, 3, seed=5)
    s = oracle.system_from_workload(sysd)
    dets = s.determinants()
    r = oracle.Run(s, tau=0.001, seed=3, target_walkers=1e12, semistoch_size=300, semistoch_start=1)
    c0 = np.linspace(1.0, 50.0, len(dets))
    r.import_state([d[0] for d in dets], [d[1] for d in dets], c0, 1, 0.0, vary=1, shift_start=0, cnt=0,
                   nw_last=0)
    r.step(1)
    csr = r.semistoch_csr()
    nd = csr["rowptr"].size - 1
    assert nd == 300 and csr["val"].size > 3000
    rng = np.random.default_rng(11)
    two64 = 2 ** 64

    def check(cD):
        y = r.semistoch_rows(cD)
        differs_seq = differs_full = 0
        for k in range(nd):
            q0, q1 = csr["rowptr"][k], csr["rowptr"][k + 1]
            p = csr["val"][q0:q1] * cD[csr["col"][q0:q1]]   # binary64 products
            exact = Fraction(0)
            full = Fraction(0)
            for v in p:
                f = Fraction(float(v))
                t = Fraction(math.floor(abs(f) * two64), two64)
                exact += t if f >= 0 else -t
                full += f
            assert np.float64(y[k]).view(np.uint64) == np.float64(float(exact)).view(np.uint64), k
            seq = 0.0
            for v in p:
                seq = seq + float(v)
            differs_seq += seq != float(exact)
            differs_full += float(full) != float(exact)
        return differs_seq, differs_full

    # amplitudes over 33 decades: in-order binary64 sums differ from the exact ones
    assert check(rng.normal(size=nd) * 10.0 ** rng.uniform(-25.0, 8.0, size=nd))[0] > 0
    # amplitudes near 2^-64 / |H|: the truncation decides the rounded sums
    assert check(rng.normal(size=nd) * 1e-19)[1] > 0


# ----------------------------------------------------------------- full runs
@pytest.mark.parametrize("which", ["hubbard", "abinitio"])
def test_fciqmc_energy_within_3sigma_of_exact(which):
    if which == "hubbard":
        sysd, tau = workloads.hubbard_1d(6, 1.0, 4.0), 0.02
    else:
        sysd, tau = workloads.small_abinitio(6, 3, 3, seed=9), 0.005
    s = oracle.system_from_workload(sysd)
    e0, _, dets = s.exact_ground_state()
    # start the shift a little above E_0 so that the growth phase is short
    r = oracle.Run(s, tau=tau, seed=12, target_walkers=2000, initiator_threshold=0.0, initial_walkers=200.0,
                   initial_shift=e0 + 0.3)
    r.step(3000)
    st = r.stats()
    start = int(np.argmax(st["vary"] > 0)) + 300
    num, den = st["e_num"][start:], st["e_den"][start:]
    e, sig = oracle.ratio_estimate(num, den)
    assert sig > 0
    assert abs(e - e0) < 3.0 * sig + 1e-9, (e, e0, sig)
    ms, ss, _ = oracle.blocking(st["S"][start:])
    assert abs(ms - e0) < 5.0 * ss + 0.05 * abs(e0) + 0.05
    ex = r.export()
    for a, b in zip(ex["alpha"], ex["beta"]):
        assert bin(int(a)).count("1") == s.na and bin(int(b)).count("1") == s.nb


def test_run_is_deterministic_and_keyed():
    sysd, prm = workloads.config_hubbard_ring()
    s = oracle.system_from_workload(sysd)
    r1 = oracle.Run(s, **dict(prm, target_walkers=500))
    r2 = oracle.Run(s, **dict(prm, target_walkers=500))
    r1.step(150)
    r2.step(150)
    e1, e2 = r1.export(), r2.export()
    for k in e1:
        np.testing.assert_array_equal(e1[k], e2[k])
    r3 = oracle.Run(s, **dict(prm, target_walkers=500, seed=2))
    r3.step(150)
    assert not np.array_equal(r3.export()["c"], e1["c"]) or len(r3.export()["c"]) != len(e1["c"])


# ----------------------------------------------------------------- heat-bath doubles (App. A, PCHB)
def test_pchb_alias_tables_reproduce_heat_bath_weights():
    """Walker alias tables: the probability of drawing entry k, summed over
    its own bin and the bins aliased to it, equals |H_ij^ab| / sum |H_ij^ab|."""
    s = oracle.system_from_workload(workloads.small_abinitio(7, 3, 2, seed=41))
    r = oracle.Run(s, tau=0.003, generator=1)
    for same, i, j in [(0, 0, 1), (0, 2, 2), (0, 5, 3), (1, 0, 1), (1, 2, 5)]:
        t = r.pchb_table(same, i, j)
        K = t["K"]
        P = np.zeros(K)
        for k in range(K):
            P[k] += t["prob"][k] / K
            P[t["alias"][k]] += (1.0 - t["prob"][k]) / K
        target = np.abs(t["val"]) / t["S"]
        np.testing.assert_allclose(P, target, rtol=1e-12, atol=1e-15)
        assert t["S"] == math.fsum(np.abs(t["val"]))
        assert np.all(P[t["val"] == 0.0] < 1e-15)
        # only double excitations carry weight: no hole on an electron's spin orbital
        a, b = t["a"], t["b"]
        bad = ((a == i) | (a == j) | (b == i) | (b == j)) if same else ((a == i) | (b == j))
        assert np.all(t["val"][bad] == 0.0)
        assert np.any(t["val"][~bad] != 0.0)


def _word_bin_coin(k, K, frac_lo):
    """a 64-bit word whose bin floor(w K / 2^64) is k and whose coin
    (w K mod 2^64) is at least frac_lo (the smallest such word)"""
    return -((-(k << 64) - frac_lo) // K)


def test_pchb_spawn_weight_times_probability_is_tau_H():
    """Unbiasedness (Sec. II, Eq. (5)): summed over every electron pair, bin
    and coin outcome of the heat-bath generator, the probability of reaching a
    target times the spawned weight per walker (|H| / p_gen * dt = lam) equals
    dt |H_ji|; and the generator, fed words that select a given bin and coin
    side, returns exactly the entry that the tables say."""
    tau, ps = 0.003, 0.1
    s = oracle.system_from_workload(workloads.small_abinitio(6, 2, 2, seed=43))
    r = oracle.Run(s, tau=tau, generator=1, p_single=ps)
    det = s.ref
    N, n = s.norb, s.na + s.nb
    occ = [(p, 0) for p in range(N) if det[0] >> p & 1] + [(p, 1) for p in range(N) if det[1] >> p & 1]
    Ptot, lam_of = {}, {}
    checked = 0
    for x in range(n * (n - 1)):
        e1, rr = divmod(x, n - 1)
        e2 = rr + (rr >= e1)
        (o1, s1), (o2, s2) = occ[e1], occ[e2]
        if s1 != s2:
            i, j = (o1, o2) if s1 == 0 else (o2, o1)
            t = r.pchb_table(0, i, j)
        else:
            i, j = min(o1, o2), max(o1, o2)
            t = r.pchb_table(1, i, j)
        K = t["K"]
        if t["S"] == 0.0:
            continue
        pxx = Fraction(1) - Fraction(ps)
        for k in range(K):
            for side, pk, entry in ((0, t["prob"][k], k), (1, 1.0 - t["prob"][k], t["alias"][k])):
                a, b = int(t["a"][entry]), int(t["b"][entry])
                ta, tb = det
                if s1 != s2:
                    if ta >> a & 1 or tb >> b & 1:
                        continue
                    ta ^= (1 << i) | (1 << a)
                    tb ^= (1 << j) | (1 << b)
                else:
                    wd = tb if s1 else ta
                    if wd >> a & 1 or wd >> b & 1:
                        continue
                    wd ^= (1 << o1) | (1 << o2) | (1 << a) | (1 << b)
                    ta, tb = (ta, wd) if s1 else (wd, tb)
                prob = float(pxx) / (n * (n - 1)) * pk / K
                Ptot[(ta, tb)] = Ptot.get((ta, tb), 0.0) + prob
                lam_of[(ta, tb)] = t["lam"]
                if pk > 0 and checked < 400 and (k * 7 + x) % 5 == 0:
                    w1 = -((-(x << 64)) // (n * (n - 1)))
                    w2 = _word_bin_coin(k, K, 0 if side == 0 else (1 << 64) - K)
                    if w2 < 1 << 64 and ((w2 * K) >> 64) == k and (side == 0 or (w2 * K) % (1 << 64) >= 2 ** 64 - K):
                        cls, tgt, lam = r.generate_pchb(det, [MASK, w1, w2, 0])
                        if side == 0 and t["prob"][k] > 2.0 ** -53 or side == 1 and t["prob"][k] < 1.0:
                            assert tgt == (ta, tb) and lam == t["lam"], (x, k, side)
                            checked += 1
    assert checked > 20
    for tgt, P in Ptot.items():
        H = s.hoff(det, tgt)
        assert abs(P * lam_of[tgt] - tau * abs(H)) <= 1e-12 * tau * abs(H), (tgt, P * lam_of[tgt], tau * abs(H))
    # every double excitation with H != 0 is reached
    for d in s.determinants():
        lev = bin(d[0] ^ det[0]).count("1") + bin(d[1] ^ det[1]).count("1")
        if lev == 4 and s.hoff(det, d) != 0.0:
            assert d in Ptot, d


# ---------------------------------------------------------------- trial wave function (Sec. IV)
def test_jacobi_lowest_matches_eigh():
    """The oracle's cyclic Jacobi against LAPACK (numpy.linalg.eigh) on random
    symmetric matrices, one with a degenerate lowest pair."""
    rng = np.random.default_rng(11)
    for n in (1, 2, 5, 17, 40):
        A = rng.normal(size=(n, n))
        A = A + A.T
        E, v = oracle.jacobi_lowest(A)
        w, V = np.linalg.eigh(A)
        assert abs(E - w[0]) <= 1e-12 * np.abs(w).max()
        assert abs(abs(v @ V[:, 0]) - 1.0) < 1e-10
        np.testing.assert_allclose(A @ v, E * v, atol=1e-11 * np.abs(w).max())
    D = np.diag([-3.0, -3.0, 1.0, 2.0])
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    E, v = oracle.jacobi_lowest(Q @ D @ Q.T)
    assert abs(E + 3.0) < 1e-12 and abs(np.linalg.norm(v) - 1.0) < 1e-12


def _trial_run(sysd, **kw):
    s = oracle.system_from_workload(sysd)
    p = dict(tau=0.01, target_walkers=1000, initial_walkers=1000.0, shift_damping=0.3, shift_interval=5,
             initiator_threshold=0.0, seed=3, trial_start=20)
    p.update(kw)
    return s, oracle.Run(s, **p)


def test_trial_numerator_is_psiT_H_psi_by_brute_force():
    """After the trial space is built, every iteration's numerator equals
    sum_j (H - E_ref)_jT cT C_j and the denominator sum_T cT C, computed with
    the dense FCI matrix, so no connected determinant is missed; cT is the
    lowest eigenvector of H^T."""
    sysd = workloads.small_abinitio(6, 2, 2, n_chol=2, seed=5)
    s, r = _trial_run(sysd, trial_size=12)
    r.step(120)
    ti = r.trial_info()
    assert ti["nt"] == 12 and ti["n_w"] > 12
    dets, H = s.hamiltonian()
    idx = {d: k for k, d in enumerate(dets)}
    T = [idx[(int(a), int(b))] for a, b in zip(ti["a"], ti["b"])]
    HT = H[np.ix_(T, T)]
    w, V = np.linalg.eigh(HT)
    assert abs(ti["ET"] - w[0]) < 1e-12 * max(1.0, abs(w[0]))
    np.testing.assert_allclose(HT @ ti["cT"], ti["ET"] * ti["cT"], atol=1e-11)
    for extra in range(3):
        st = r.export()
        c = np.zeros(len(dets))
        for a, b, x in zip(st["alpha"], st["beta"], st["c"]):
            c[idx[(int(a), int(b))]] = x
        num = float(ti["cT"] @ (H[T, :] @ c))
        den = float(ti["cT"] @ c[T])
        last = {k: v[-1] for k, v in r.stats().items()}
        assert abs(last["t_num"] - num) <= 1e-11 * max(1.0, np.abs(H[T, :]).sum() * np.abs(c).max())
        assert abs(last["t_den"] - den) <= 1e-12 * max(1.0, np.abs(c).sum())
        r.step(1)


def test_trial_space_equal_to_fci_space_gives_exact_energy():
    """With T = the whole FCI space, Psi^T is the exact ground state, so
    <Psi^T|H|Psi> / <Psi^T|Psi> = E_0 for whatever Psi the walkers hold."""
    sysd = workloads.small_abinitio(6, 2, 2, n_chol=2, seed=5)
    s, r = _trial_run(sysd, trial_size=10 ** 6)
    e0, _, dets = s.exact_ground_state()
    # every determinant occupied when T is chosen: a state with all of them is
    # imported at the iteration that builds T
    a = [d[0] for d in dets]
    b = [d[1] for d in dets]
    r.import_state(a, b, np.full(len(dets), 3.0), 100, 0.0, vary=1, shift_start=80, cnt=0,
                   nw_last=int(3 * len(dets)) << 32)
    r.step(60)
    ti = r.trial_info()
    assert ti["nt"] == len(dets)
    assert abs(ti["ET"] - e0) < 1e-11
    st = r.stats()
    sel = st["t_den"] != 0.0
    assert sel.sum() > 30
    np.testing.assert_allclose(st["t_num"][sel] / st["t_den"][sel], e0, rtol=0, atol=1e-9)


# ---------------------------------------------------------------- replicas and PT2 (Sec. V, VI)
def test_replica_zero_is_the_single_run_and_replica_one_differs():
    sysd = workloads.small_abinitio(7, 3, 2, seed=8)
    p = dict(tau=0.004, target_walkers=1500, initial_walkers=200.0, initiator_threshold=2.0, seed=5)
    s = oracle.system_from_workload(sysd)
    a, b, c = oracle.Run(s, **p), oracle.Run(s, replica=0, **p), oracle.Run(s, replica=1, **p)
    for r in (a, b, c):
        r.step(40)
    ea, eb, ec = a.export(), b.export(), c.export()
    assert np.array_equal(ea["c"].view(np.uint64), eb["c"].view(np.uint64))
    assert ea["c"].size != ec["c"].size or not np.array_equal(ea["c"], ec["c"])


def _pair_start(seed):
    """Both replicas start from the same list: the 20 largest components of
    the exact ground state, scaled so that some are initiators (|C| > 40) and
    most are not; C_min = 0.05 keeps most spawns unrounded."""
    sysd = workloads.small_abinitio(6, 2, 2, n_chol=2, seed=5)
    s = oracle.system_from_workload(sysd)
    e0, v, dets = s.exact_ground_state()
    top = np.argsort(-np.abs(v))[:20]
    c = np.round(60.0 * v[top] / np.abs(v[top[0]]) * np.sign(v[top[0]]))
    c[c == 0] = 1.0
    keys = [dets[k] for k in top]
    params = dict(tau=0.01, target_walkers=1e9, initial_walkers=10.0, initiator_threshold=40.0, c_min=0.05,
                  seed=seed)
    pair = oracle.Pair(s, **params)
    for r in pair.r:
        r.import_state([k[0] for k in keys], [k[1] for k in keys], c, 10, -0.2, vary=0)
    return s, pair, keys, c


def test_pair_overlap_is_the_start_overlap():
    s, pair, keys, c = _pair_start(1)
    pair.step(1)
    row = {k: v[-1] for k, v in pair.r[0].stats().items()}
    assert row["x_overlap"] == math.fsum(c * c) or abs(row["x_overlap"] - float(c @ c)) < 1e-12 * float(c @ c)
    assert {k: v[-1] for k, v in pair.r[1].stats().items()}["x_overlap"] == 0.0


def test_pair_variational_and_pt2_numerators_are_unbiased():
    """Averaged over independent seeds, x_var_num estimates C (H - E_ref) C of
    the common start vector, and x_pt2 estimates
    sum_j (sum_{i non-initiator} H_ji C_i)^2 / (E_0 - (H_jj - E_ref)) over the
    unoccupied j (the replicas' rejected spawns are independent, each with
    expectation -tau sum_i H_ji C_i)."""
    s, _, keys, c = _pair_start(0)
    dets, H = s.hamiltonian()
    idx = {d: k for k, d in enumerate(dets)}
    cv = np.zeros(len(dets))
    for k, x in zip(keys, c):
        cv[idx[k]] = x
    exact_var = float(cv @ H @ cv)
    non_init = np.where((np.abs(cv) <= 40.0) & (cv != 0.0), cv, 0.0)
    ref = idx[s.ref]
    non_init[ref] = 0.0  # the reference is always an initiator
    Hoff = H - np.diag(np.diag(H))
    g = Hoff @ non_init
    unocc = cv == 0.0
    exact_pt2 = float(np.sum((g[unocc] ** 2) / (-0.2 - np.diag(H)[unocc])))
    var, pt2 = [], []
    for seed in range(1, 401):
        _, pair, _, _ = _pair_start(seed)
        pair.step(1)
        row = {k: v[-1] for k, v in pair.r[0].stats().items()}
        var.append(row["x_var_num"])
        pt2.append(row["x_pt2"])
    var, pt2 = np.array(var), np.array(pt2)
    assert abs(var.mean() - exact_var) < 4.0 * var.std() / math.sqrt(var.size) + 1e-9
    assert abs(pt2.mean() - exact_pt2) < 4.0 * pt2.std() / math.sqrt(pt2.size) + 1e-9
    assert np.count_nonzero(pt2) > 50  # the estimator is exercised


# ---------------------------------------------------------------- adaptive shift (Sec. V)
def test_adaptive_shift_factor_by_definition():
    """f_i of every non-initiator, recomputed from the last iteration's spawns:
    w_ij = |H_ji| / |H_jj - E_ref - S| truncated to 2^-64, summed over the
    spawns onto determinants occupied at the start (A) and over all (T),
    f_i = A / T (1 without spawns); initiators keep 1."""
    sysd = workloads.small_abinitio(7, 3, 2, seed=8)
    s = oracle.system_from_workload(sysd)
    n_a = 2.0
    r = oracle.Run(s, tau=0.004, target_walkers=1500, initial_walkers=200.0, initiator_threshold=n_a, seed=5,
                   shift_damping=0.5, shift_interval=5, initial_shift=-0.3, adaptive_shift=1)
    r.step(40)
    r.keep_last(True)
    r.step(1)
    S_start = r.stats()["S"][-2]
    L, Sp = r.last_iteration()
    occ = {(int(a), int(b)): (c, hd) for a, b, c, hd in zip(L["a"], L["b"], L["c"], L["hd"])}
    checked = 0
    for i in range(len(L["a"])):
        det = (int(L["a"][i]), int(L["b"][i]))
        c = L["c"][i]
        init = abs(c) > n_a or det == s.ref
        if c == 0.0 or init:
            assert L["f"][i] == 1.0
            continue
        A = T = 0
        for k in np.nonzero(Sp["parent"] == i)[0]:
            tgt = (int(Sp["a"][k]), int(Sp["b"][k]))
            cj, hd = occ.get(tgt, (0.0, None))
            if hd is None:
                hd = s.hdiag_rel(*tgt)
            den = abs(hd - S_start)
            if den == 0.0:
                continue
            q = int(abs(s.hoff(det, tgt)) / den * 2.0 ** 64)
            T += q
            if cj != 0.0:
                A += q
        f = float(A) / float(T) if T else 1.0
        assert L["f"][i] == f, (i, L["f"][i], f)
        checked += T > 0
    assert checked > 20


def test_adaptive_shift_is_inert_without_non_initiators():
    """With n_a = 0 every occupied determinant is an initiator: the adaptive
    shift changes nothing, bit for bit."""
    sysd = workloads.small_abinitio(7, 3, 2, seed=8)
    s = oracle.system_from_workload(sysd)
    p = dict(tau=0.004, target_walkers=1500, initial_walkers=100.0, initiator_threshold=0.0, seed=5)
    a, b = oracle.Run(s, **p), oracle.Run(s, adaptive_shift=1, **p)
    a.step(60)
    b.step(60)
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea["c"].view(np.uint64), eb["c"].view(np.uint64))
    c = oracle.Run(s, adaptive_shift=1, **dict(p, initiator_threshold=2.0))
    d = oracle.Run(s, **dict(p, initiator_threshold=2.0))
    c.step(60)
    d.step(60)
    assert not np.array_equal(c.export()["c"], d.export()["c"])
