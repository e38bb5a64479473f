"""CPU oracle for the initiator-FCIQMC projector iteration.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The GPU
library never imports it, and the two share no code.

``fciqmc_oracle.c`` holds the method (Philox4x64-10 draws, uniform and lattice
excitation generation, Slater-Condon rules, spawn / death / annihilation with
the initiator rule, semi-stochastic projection, shift update and the reference
projected energy of Eq. (9) of the paper).  This module wraps it with ctypes and
adds what needs no new arithmetic: exact diagonalisation through
``numpy.linalg.eigh`` on the oracle's own Hamiltonian matrix, the U=0 Hubbard
band energy in closed form, and Flyvbjerg-Petersen blocking statistics.
"""
from __future__ import annotations

import ctypes as C
import itertools
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fciqmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Stat(C.Structure):
    _fields_ = [("iter", C.c_int64), ("nw", C.c_double), ("S", C.c_double), ("e_num", C.c_double),
                ("e_den", C.c_double), ("ndet", C.c_int64), ("attempts", C.c_int64),
                ("spawns", C.c_int64), ("rejected", C.c_int64), ("annihilated", C.c_double),
                ("vary", C.c_int), ("t_num", C.c_double), ("t_den", C.c_double),
                ("x_overlap", C.c_double), ("x_var_num", C.c_double), ("x_pt2", C.c_double)]


class Params(C.Structure):
    _fields_ = [("tau", C.c_double), ("shift_damping", C.c_double), ("target_walkers", C.c_double),
                ("initial_walkers", C.c_double), ("initial_shift", C.c_double),
                ("initiator_threshold", C.c_double), ("c_min", C.c_double), ("p_single", C.c_double),
                ("shift_interval", C.c_int64), ("seed", C.c_uint64),
                ("semistoch_size", C.c_int64), ("semistoch_start", C.c_int64), ("generator", C.c_int64),
                ("trial_size", C.c_int64), ("trial_start", C.c_int64), ("replica", C.c_int64),
                ("adaptive_shift", C.c_int64)]


DEFAULT_PARAMS = dict(tau=0.01, shift_damping=0.1, target_walkers=1e4, initial_walkers=10.0,
                      initial_shift=0.0, initiator_threshold=0.0, c_min=1.0, p_single=0.1,
                      shift_interval=10, seed=1, semistoch_size=0, semistoch_start=100,
                      generator=0, trial_size=0, trial_start=100, replica=0, adaptive_shift=0)

CLASSES = ("single_a", "single_b", "double_ab", "double_aa", "double_bb", "hop")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P, D, I64, U64, I32 = C.c_void_p, C.c_double, C.c_int64, C.c_uint64, C.c_int
            dp = C.POINTER(C.c_double)
            up = C.POINTER(C.c_uint64)
            sig = {
                "orc_philox4x64_10": (None, [up, up, up]),
                "orc_fsum": (D, [dp, I64]),
                "orc_ln": (D, [D]),
                "orc_sys_abinitio": (P, [I32, I32, I32, D, dp, dp, up]),
                "orc_sys_hubbard": (P, [I32, I32, I32, I32, D, D, I32, I32, up]),
                "orc_sys_free": (None, [P]),
                "orc_sys_ref": (None, [P, up]),
                "orc_hdiag_rel": (D, [P, U64, U64]),
                "orc_eref": (D, [P]),
                "orc_hoff": (D, [P, U64, U64, U64, U64]),
                "orc_build_hamiltonian": (None, [P, I64, up, up, dp]),
                "orc_pgen": (D, [P, D, I32]),
                "orc_generate": (I32, [P, D, U64, U64, up, up, up]),
                "orc_create": (P, [P, C.POINTER(Params)]),
                "orc_destroy": (None, [P]),
                "orc_step": (I32, [P, I64]),
                "orc_ndet": (I64, [P]),
                "orc_iter": (I64, [P]),
                "orc_shift": (D, [P]),
                "orc_export": (None, [P, up, up, dp, dp, C.POINTER(C.c_int32)]),
                "orc_export_shift": (None, [P, dp, C.POINTER(C.c_int64), up]),
                "orc_import": (None, [P, I64, up, up, dp, I64, D, I32, I64, I64, U64, U64]),
                "orc_nstats": (I64, [P]),
                "orc_stats": (None, [P, I64, I64, C.POINTER(Stat)]),
                "orc_stat_size": (I32, []),
                "orc_params_size": (I32, []),
                "orc_semistoch_info": (I64, [P, C.POINTER(C.c_int64)]),
                "orc_semistoch_csr": (None, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), dp, up, up]),
                "orc_semistoch_rows": (None, [P, dp, dp]),
                "orc_proj_energy": (None, [P, dp, dp]),
                "orc_enum_grid": (I32, [P]),
                "orc_generate_pchb": (I32, [P, U64, U64, up, up, up, dp]),
                "orc_pchb_table": (I32, [P, I32, I32, I32, dp, dp, dp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int32), dp]),
                "orc_trial_info": (I64, [P, C.POINTER(C.c_int64), dp, up, up, dp]),
                "orc_pair_step": (I32, [P, P, I64]),
                "orc_set_keep_last": (None, [P, I32]),
                "orc_last_iteration": (I64, [P, C.POINTER(C.c_int64), up, up, dp, dp, dp, up, up, dp,
                                             C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
                "orc_jacobi_lowest": (I32, [I32, dp, dp, dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            assert L.orc_stat_size() == C.sizeof(Stat)
            assert L.orc_params_size() == C.sizeof(Params)
            _lib = L
    return _lib


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(C.POINTER(C.c_uint64))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- primitives
def philox4x64_10(counter, key):
    """One Philox4x64-10 block (Salmon et al., SC'11)."""
    c, cp = _u64(counter)
    k, kp = _u64(key)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(cp, kp, out.ctypes.data_as(C.POINTER(C.c_uint64)))
    return out


def fsum(values) -> float:
    """Exact sum of binary64 values, rounded once to nearest-even."""
    v, vp = _f64(values)
    return lib().orc_fsum(vp, v.size)


def ln(x: float) -> float:
    return lib().orc_ln(float(x))


# ---------------------------------------------------------------- systems
class System:
    """Ab initio (FCIDUMP-style integrals) or Hubbard Hamiltonian."""

    def __init__(self, handle, norb, na, nb, kind):
        self.h = handle
        self.norb, self.na, self.nb, self.kind = norb, na, nb, kind

    @classmethod
    def abinitio(cls, h1, eri_packed, na, nb, ecore=0.0, ref=None):
        h1 = np.ascontiguousarray(h1, np.float64)
        norb = h1.shape[0]
        _, hp = _f64(h1)
        e, ep = _f64(eri_packed)
        r = None
        if ref is not None:
            ra, r = _u64(ref)
        hd = lib().orc_sys_abinitio(norb, na, nb, float(ecore), hp, ep, r)
        if not hd:
            raise ValueError("invalid ab initio system")
        s = cls(hd, norb, na, nb, "abinitio")
        s._keep = (h1, e)
        return s

    @classmethod
    def hubbard(cls, lx, ly, periodic_x, periodic_y, t, U, na, nb, ref=None):
        r = None
        if ref is not None:
            ra, r = _u64(ref)
        hd = lib().orc_sys_hubbard(lx, ly, int(periodic_x), int(periodic_y), float(t), float(U), na, nb, r)
        if not hd:
            raise ValueError("invalid Hubbard lattice")
        return cls(hd, lx * ly, na, nb, "hubbard")

    def __del__(self):
        try:
            if self.h:
                lib().orc_sys_free(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def ref(self):
        out = np.zeros(2, np.uint64)
        lib().orc_sys_ref(self.h, out.ctypes.data_as(C.POINTER(C.c_uint64)))
        return int(out[0]), int(out[1])

    @property
    def eref(self) -> float:
        return lib().orc_eref(self.h)

    def hdiag_rel(self, a, b) -> float:
        return lib().orc_hdiag_rel(self.h, a, b)

    @property
    def enum_grid(self) -> int:
        """Fe: E_num's terms are truncated to multiples of 2^-Fe (reading R12)."""
        return lib().orc_enum_grid(self.h)

    def hoff(self, i, j) -> float:
        """<D_j|H|D_i> for determinants i=(a,b), j=(a,b), i != j."""
        return lib().orc_hoff(self.h, i[0], i[1], j[0], j[1])

    def pgen(self, p_single, cls_index) -> float:
        return lib().orc_pgen(self.h, float(p_single), int(cls_index))

    def generate(self, p_single, det, words):
        w, wp = _u64(words)
        ta = C.c_uint64()
        tb = C.c_uint64()
        c = lib().orc_generate(self.h, float(p_single), det[0], det[1], wp, C.byref(ta), C.byref(tb))
        return c, (ta.value, tb.value)

    def determinants(self):
        """All determinants of the FCI space with (na, nb) electrons, ascending key."""
        def words(k):
            return sorted(sum(1 << p for p in c) for c in itertools.combinations(range(self.norb), k))
        wa, wb = words(self.na), words(self.nb)
        return [(a, b) for a in wa for b in wb]

    def hamiltonian(self, dets=None):
        """Dense H - E_ref over ``dets`` (default: the FCI space)."""
        if dets is None:
            dets = self.determinants()
        n = len(dets)
        da, dap = _u64([d[0] for d in dets])
        db, dbp = _u64([d[1] for d in dets])
        H = np.zeros((n, n), np.float64)
        lib().orc_build_hamiltonian(self.h, n, dap, dbp, H.ctypes.data_as(C.POINTER(C.c_double)))
        return dets, H

    def exact_ground_state(self):
        """(E_0 - E_ref, eigenvector, dets) by dense diagonalisation."""
        dets, H = self.hamiltonian()
        w, v = np.linalg.eigh(H)
        return w[0], v[:, 0], dets


def hubbard_u0_energy(lx, ly, t, na, nb):
    """Closed-form U=0 ground state of a periodic lattice: fill the lowest
    single-particle levels eps(k) = -2t sum_d cos(k_d), k_d = 2 pi m / L_d."""
    eps = []
    for mx in range(lx):
        for my in range(ly):
            e = -2.0 * t * math.cos(2.0 * math.pi * mx / lx)
            if ly > 1:
                e += -2.0 * t * math.cos(2.0 * math.pi * my / ly)
            eps.append(e)
    eps.sort()
    return sum(eps[:na]) + sum(eps[:nb])


# ---------------------------------------------------------------- FCIQMC run
class Run:
    def __init__(self, system: System, **params):
        p = dict(DEFAULT_PARAMS)
        p.update(params)
        self.params = p
        self.system = system
        self._p = Params(**{k: p[k] for k, _ in Params._fields_})
        self.h = lib().orc_create(system.h, C.byref(self._p))

    def __del__(self):
        try:
            if self.h:
                lib().orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def step(self, n=1):
        rc = lib().orc_step(self.h, int(n))
        if rc:
            raise RuntimeError("oracle iteration failed with code %d" % rc)

    @property
    def iteration(self):
        return lib().orc_iter(self.h)

    @property
    def shift(self):
        return lib().orc_shift(self.h)

    def export(self):
        n = lib().orc_ndet(self.h)
        a = np.zeros(n, np.uint64)
        b = np.zeros(n, np.uint64)
        c = np.zeros(n, np.float64)
        hd = np.zeros(n, np.float64)
        fl = np.zeros(n, np.int32)
        lib().orc_export(self.h, a.ctypes.data_as(C.POINTER(C.c_uint64)), b.ctypes.data_as(C.POINTER(C.c_uint64)),
                         c.ctypes.data_as(C.POINTER(C.c_double)), hd.ctypes.data_as(C.POINTER(C.c_double)),
                         fl.ctypes.data_as(C.POINTER(C.c_int32)))
        return dict(alpha=a, beta=b, c=c, hdiag=hd, flags=fl)

    def shift_state(self):
        S = C.c_double()
        st = (C.c_int64 * 3)()
        nwl = (C.c_uint64 * 2)()
        lib().orc_export_shift(self.h, C.byref(S), st, nwl)
        return dict(S=S.value, vary=st[0], shift_start=st[1], cnt=st[2], nw_last=(nwl[0] << 64) | nwl[1])

    def import_state(self, alpha, beta, c, iteration, S, vary=0, shift_start=0, cnt=0, nw_last=0):
        a, ap = _u64(alpha)
        b, bp = _u64(beta)
        cc, cp = _f64(c)
        lib().orc_import(self.h, a.size, ap, bp, cp, int(iteration), float(S), int(vary), int(shift_start),
                         int(cnt), (int(nw_last) >> 64) & 0xFFFFFFFFFFFFFFFF, int(nw_last) & 0xFFFFFFFFFFFFFFFF)

    def generate_pchb(self, det, words):
        """One generation with the heat-bath doubles of this run: (class, target, |H|/p_gen)."""
        w, wp = _u64(words)
        ta = C.c_uint64()
        tb = C.c_uint64()
        lam = C.c_double()
        c = lib().orc_generate_pchb(self.h, det[0], det[1], wp, C.byref(ta), C.byref(tb), C.byref(lam))
        return c, (ta.value, tb.value), lam.value

    def pchb_table(self, same_spin, i, j):
        N = self.system.norb
        K = N * N
        prob = np.zeros(K)
        alias = np.zeros(K, np.int32)
        ea = np.zeros(K, np.int32)
        eb = np.zeros(K, np.int32)
        val = np.zeros(K)
        S = C.c_double()
        lam = C.c_double()
        K = lib().orc_pchb_table(self.h, int(same_spin), int(i), int(j), C.byref(S), C.byref(lam),
                                 prob.ctypes.data_as(C.POINTER(C.c_double)),
                                 alias.ctypes.data_as(C.POINTER(C.c_int32)), ea.ctypes.data_as(C.POINTER(C.c_int32)),
                                 eb.ctypes.data_as(C.POINTER(C.c_int32)), val.ctypes.data_as(C.POINTER(C.c_double)))
        return dict(K=K, S=S.value, lam=lam.value, prob=prob[:K], alias=alias[:K], a=ea[:K], b=eb[:K], val=val[:K])

    def last_iteration(self):
        """Start list (keys, C, H_ii - E_ref, adaptive-shift f_i) and spawns (keys,
        weight, initiator flag, parent index) of the last iteration; needs
        keep_last(True) before it."""
        ns = C.c_int64()
        n = lib().orc_last_iteration(self.h, C.byref(ns), None, None, None, None, None, None, None, None, None, None)
        m = ns.value
        L = {k: np.zeros(max(n, 1), t) for k, t in (("a", np.uint64), ("b", np.uint64), ("c", np.float64),
                                                     ("hd", np.float64), ("f", np.float64))}
        S = {k: np.zeros(max(m, 1), t) for k, t in (("a", np.uint64), ("b", np.uint64), ("w", np.float64),
                                                     ("init", np.int32), ("parent", np.int64))}
        u = lambda x: x.ctypes.data_as(C.POINTER(C.c_uint64))
        d = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
        lib().orc_last_iteration(self.h, None, u(L["a"]), u(L["b"]), d(L["c"]), d(L["hd"]), d(L["f"]), u(S["a"]),
                                 u(S["b"]), d(S["w"]), S["init"].ctypes.data_as(C.POINTER(C.c_int32)),
                                 S["parent"].ctypes.data_as(C.POINTER(C.c_int64)))
        return {k: v[:n] for k, v in L.items()}, {k: v[:m] for k, v in S.items()}

    def keep_last(self, on=True):
        lib().orc_set_keep_last(self.h, int(bool(on)))

    def trial_info(self):
        """Trial space of the E_Trial estimator: dict(nt, n_w (|T u C|), ET (E^T - E_ref), a, b, cT)."""
        nw = C.c_int64()
        ET = C.c_double()
        nt = lib().orc_trial_info(self.h, C.byref(nw), C.byref(ET), None, None, None)
        a = np.zeros(max(nt, 1), np.uint64)
        b = np.zeros(max(nt, 1), np.uint64)
        cT = np.zeros(max(nt, 1))
        lib().orc_trial_info(self.h, None, None, a.ctypes.data_as(C.POINTER(C.c_uint64)),
                             b.ctypes.data_as(C.POINTER(C.c_uint64)), cT.ctypes.data_as(C.POINTER(C.c_double)))
        return dict(nt=int(nt), n_w=int(nw.value), ET=ET.value, a=a[:nt], b=b[:nt], cT=cT[:nt])

    def proj_energy(self):
        """(E_num, E_den) of the current list, Eq. (9)."""
        num = C.c_double()
        den = C.c_double()
        lib().orc_proj_energy(self.h, C.byref(num), C.byref(den))
        return num.value, den.value

    def semistoch_info(self):
        nnz = C.c_int64()
        nd = lib().orc_semistoch_info(self.h, C.byref(nnz))
        return nd, nnz.value

    def semistoch_csr(self):
        """D (keys in ascending order) and H^D - E_ref in CSR."""
        nd, nnz = self.semistoch_info()
        rp = np.zeros(nd + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int64)
        val = np.zeros(max(nnz, 1))
        da = np.zeros(max(nd, 1), np.uint64)
        db = np.zeros(max(nd, 1), np.uint64)
        i64 = lambda x: x.ctypes.data_as(C.POINTER(C.c_int64))
        lib().orc_semistoch_csr(self.h, i64(rp), i64(col), val.ctypes.data_as(C.POINTER(C.c_double)),
                                da.ctypes.data_as(C.POINTER(C.c_uint64)), db.ctypes.data_as(C.POINTER(C.c_uint64)))
        return dict(rowptr=rp, col=col[:nnz], val=val[:nnz], alpha=da[:nd], beta=db[:nd])

    def semistoch_rows(self, cD):
        """Row sums y_k = sum_c H^D_kc cD_c of the semi-stochastic update."""
        nd, _ = self.semistoch_info()
        x, xp = _f64(cD)
        assert x.size == nd
        y = np.zeros(nd)
        lib().orc_semistoch_rows(self.h, xp, y.ctypes.data_as(C.POINTER(C.c_double)))
        return y

    def stats(self):
        n = lib().orc_nstats(self.h)
        arr = (Stat * max(n, 1))()
        if n:
            lib().orc_stats(self.h, 0, n, arr)
        cols = {f: np.array([getattr(arr[i], f) for i in range(n)]) for f, _ in Stat._fields_}
        return cols


class Pair:
    """Two replicas (Philox key word 1 = 0 and 1) of one system stepped
    together; the first replica's statistics rows carry the cross estimators
    x_overlap, x_var_num and x_pt2."""

    def __init__(self, system, **params):
        params = dict(params)
        params.pop("replica", None)
        self.r = [Run(system, replica=0, **params), Run(system, replica=1, **params)]

    def step(self, n):
        e = lib().orc_pair_step(self.r[0].h, self.r[1].h, int(n))
        if e:
            raise RuntimeError("oracle pair step failed with code %d" % e)


def jacobi_lowest(A):
    """Lowest eigenpair of a symmetric matrix by the oracle's cyclic Jacobi method."""
    A = np.ascontiguousarray(A, np.float64).copy()
    n = A.shape[0]
    E = C.c_double()
    v = np.zeros(n)
    lib().orc_jacobi_lowest(n, A.ctypes.data_as(C.POINTER(C.c_double)), C.byref(E),
                            v.ctypes.data_as(C.POINTER(C.c_double)))
    return E.value, v


# ---------------------------------------------------------------- statistics
# The paper gives no error analysis for its energy estimators.  Reading: the
# blocking transformation of Flyvbjerg and Petersen (J. Chem. Phys. 91, 461
# (1989)) with the block length chosen by the criterion of Lee, Conduit,
# Nemec, Lopez Rios and Drummond (Phys. Rev. E 83, 066706 (2011)): the
# smallest level k whose block length B = 2^k satisfies
# B^3 > 2 n (SE_k / SE_0)^4, n the number of samples.
def blocking_levels(x):
    """Levels of the blocking transformation: level 0 is the series, level
    k + 1 the means of neighbouring pairs of level k (an odd last element is
    dropped), down to two elements."""
    y = np.asarray(x, np.float64)
    out = []
    while y.size >= 2:
        out.append(y)
        m = y.size // 2
        y = 0.5 * (y[0:2 * m:2] + y[1:2 * m:2])
    return out


def _se(y):
    """Standard error of the mean of a level, treating its elements as independent."""
    return math.sqrt(float(np.mean((y - np.mean(y)) ** 2)) / (y.size - 1))


def optimal_level(x):
    """Index of the blocking level chosen by the B^3 > 2 n (SE_k/SE_0)^4 rule
    (the last level if none satisfies it; 0 for a constant series)."""
    lev = blocking_levels(x)
    if not lev:
        return -1
    n = lev[0].size
    se0 = _se(lev[0])
    if se0 == 0.0:
        return 0
    for k, y in enumerate(lev):
        if (2.0 ** k) ** 3 > 2.0 * n * (_se(y) / se0) ** 4:
            return k
    return len(lev) - 1


def blocking(x):
    """(mean, sigma of the mean, standard error of every level)."""
    x = np.asarray(x, np.float64)
    lev = blocking_levels(x)
    if not lev:
        return float(np.mean(x)) if x.size else float("nan"), float("nan"), []
    errs = [_se(y) for y in lev]
    return float(np.mean(x)), errs[optimal_level(x)], errs


def ratio_estimate(num, den):
    """mean(num) / mean(den) with the delta-method error
    sigma^2 = (s_n^2 - 2 r c + r^2 s_d^2) / mean(den)^2, where s_n, s_d and the
    covariance c of the two means are taken at one blocking level, the larger
    of the two series' optimal levels."""
    num = np.asarray(num, np.float64)
    den = np.asarray(den, np.float64)
    mn, md = float(np.mean(num)), float(np.mean(den))
    r = mn / md
    ln, ld = blocking_levels(num), blocking_levels(den)
    if not ln:
        return r, float("nan")
    k = max(optimal_level(num), optimal_level(den))
    yn, yd = ln[k], ld[k]
    m = yn.size
    vn = float(np.mean((yn - np.mean(yn)) ** 2)) / (m - 1)
    vd = float(np.mean((yd - np.mean(yd)) ** 2)) / (m - 1)
    c = float(np.mean((yn - np.mean(yn)) * (yd - np.mean(yd)))) / (m - 1)
    return r, math.sqrt(max(vn - 2.0 * r * c + r * r * vd, 0.0)) / abs(md)


def system_from_workload(sysd) -> System:
    """Build an oracle System from a ``workloads`` description."""
    if sysd["kind"] == "hubbard":
        return System.hubbard(sysd["lx"], sysd["ly"], sysd["periodic_x"], sysd["periodic_y"],
                              sysd["t"], sysd["U"], sysd["n_alpha"], sysd["n_beta"], ref=sysd.get("ref"))
    if "h1" not in sysd:
        import workloads
        h, eri = workloads.synthetic_abinitio(sysd["norb"], sysd["n_chol"], sysd["integral_seed"])
        sysd = dict(sysd, h1=h, eri=eri)
    return System.abinitio(sysd["h1"], sysd["eri"], sysd["n_alpha"], sysd["n_beta"],
                           sysd.get("ecore", 0.0), ref=sysd.get("ref"))
