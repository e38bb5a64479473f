"""Python binding of the GB300 initiator-FCIQMC library (argument marshalling only).

Every function here has the name of the C entry point it calls in
``include/fciqmc.h``; all arithmetic of the projector iteration runs in the
CUDA kernels of ``libfciqmc_gb300.so``.  PyTorch, when present, provides the
CUDA stream and the device allocator (its caching allocator).  There is no CPU
fallback: if the compiled library is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

if not os.path.exists(_build.LIB) or not _build.up_to_date():
    if os.environ.get("FCIQMC_GB300_AUTOBUILD", "1") == "1":
        _build.build()
    else:
        raise ImportError("libfciqmc_gb300.so is not built; run paper_2006_14956_gb300/build.py")
_lib = C.CDLL(_build.LIB)

FCIQMC_OK = 0
FCIQMC_ERR_INVALID_ARG = 1
FCIQMC_ERR_OUT_OF_MEMORY = 2
FCIQMC_ERR_CAPACITY = 3
FCIQMC_ERR_NUMERIC = 4
FCIQMC_ERR_TIMEOUT = 5
FCIQMC_ERR_CUDA = 6
FCIQMC_ERR_UNSUPPORTED = 7
FCIQMC_ABINITIO = 0
FCIQMC_HUBBARD = 1

ERROR_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CAPACITY", 4: "NUMERIC", 5: "TIMEOUT", 6: "CUDA",
               7: "UNSUPPORTED"}


class FciqmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, msg))
        self.code = code


class fciqmc_system(C.Structure):
    _fields_ = [("kind", C.c_int32), ("norb", C.c_int32), ("n_alpha", C.c_int32), ("n_beta", C.c_int32),
                ("ecore", C.c_double), ("h1", C.POINTER(C.c_double)), ("eri", C.POINTER(C.c_double)),
                ("lx", C.c_int32), ("ly", C.c_int32), ("periodic_x", C.c_int32), ("periodic_y", C.c_int32),
                ("t", C.c_double), ("U", C.c_double), ("has_ref", C.c_int32), ("pad0", C.c_int32),
                ("ref_alpha", C.c_uint64), ("ref_beta", C.c_uint64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class fciqmc_params(C.Structure):
    _fields_ = [("tau", C.c_double), ("shift_damping", C.c_double), ("target_walkers", C.c_double),
                ("initial_walkers", C.c_double), ("initial_shift", C.c_double),
                ("initiator_threshold", C.c_double), ("c_min", C.c_double), ("p_single", C.c_double),
                ("shift_interval", C.c_int64), ("seed", C.c_uint64), ("semistoch_size", C.c_int64),
                ("semistoch_start", C.c_int64), ("max_dets", C.c_int64), ("max_spawns", C.c_int64),
                ("max_device_bytes", C.c_int64), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("generator", C.c_int32), ("replicas", C.c_int32), ("trial_size", C.c_int64), ("trial_start", C.c_int64),
                ("adaptive_shift", C.c_int32), ("pad1", C.c_int32)]


class fciqmc_iter_stats(C.Structure):
    _fields_ = [("iteration", C.c_int64), ("nw", C.c_double), ("shift", C.c_double), ("e_num", C.c_double),
                ("e_den", C.c_double), ("ndet", C.c_int64), ("attempts", C.c_int64), ("spawns", C.c_int64),
                ("rejected", C.c_int64), ("annihilated", C.c_double), ("vary", C.c_int32), ("pad0", C.c_int32),
                ("trial_num", C.c_double), ("trial_den", C.c_double), ("x_overlap", C.c_double),
                ("x_var_num", C.c_double), ("x_pt2", C.c_double)]


class fciqmc_stats(C.Structure):
    _fields_ = [("iteration", C.c_int64), ("ndet", C.c_int64), ("nw", C.c_double), ("eref", C.c_double),
                ("shift", C.c_double), ("e_proj_inst", C.c_double), ("e_proj_mean", C.c_double),
                ("e_proj_sigma", C.c_double), ("shift_mean", C.c_double), ("shift_sigma", C.c_double),
                ("equil_start", C.c_int64), ("n_samples", C.c_int64), ("attempts_total", C.c_int64),
                ("spawns_total", C.c_int64), ("rejected_total", C.c_int64), ("annihilated_total", C.c_double),
                ("vary", C.c_int32), ("pad0", C.c_int32), ("e_trial_mean", C.c_double),
                ("e_trial_sigma", C.c_double), ("e_trial_T", C.c_double), ("trial_samples", C.c_int64),
                ("e_var_mean", C.c_double), ("e_var_sigma", C.c_double), ("pt2_mean", C.c_double),
                ("pt2_sigma", C.c_double), ("pair_samples", C.c_int64)]


class fciqmc_request_status(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("iterations", C.c_int64), ("energy", C.c_double),
                ("sigma", C.c_double), ("shift", C.c_double), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("attempts", C.c_int64), ("device_bytes", C.c_int64), ("tau", C.c_double),
                ("estimator", C.c_int32), ("pad0", C.c_int32), ("t_arrival", C.c_double)]


REQUEST_STATES = {0: "queued", 1: "running", 2: "converged", 3: "max_iters", 4: "failed"}

_H = C.c_void_p
_u64p = C.POINTER(C.c_uint64)
_dp = C.POINTER(C.c_double)
_SIGS = {
    "fciqmc_create": (C.c_int, [C.POINTER(fciqmc_system), C.POINTER(fciqmc_params), C.POINTER(_H)]),
    "fciqmc_step": (C.c_int, [_H, C.c_int64]),
    "fciqmc_step_async": (C.c_int, [_H, C.c_int64]),
    "fciqmc_sync": (C.c_int, [_H]),
    "fciqmc_stream": (C.c_void_p, [_H]),
    "fciqmc_energy": (C.c_int, [_H, C.POINTER(fciqmc_stats)]),
    "fciqmc_destroy": (None, [_H]),
    "fciqmc_last_error": (C.c_char_p, [_H]),
    "fciqmc_num_dets": (C.c_int64, [_H]),
    "fciqmc_export_state": (C.c_int, [_H, C.c_int64, _u64p, _u64p, _dp, _dp, C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int64)]),
    "fciqmc_export_shift": (C.c_int, [_H, C.POINTER(C.c_int64), _dp, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64), _u64p, _u64p]),
    "fciqmc_import_state": (C.c_int, [_H, C.c_int64, _u64p, _u64p, _dp, C.c_int64, C.c_double, C.c_int32,
                                      C.c_int64, C.c_int64, C.c_uint64, C.c_uint64]),
    "fciqmc_iter_stats_get": (C.c_int, [_H, C.c_int64, C.c_int64, C.POINTER(fciqmc_iter_stats)]),
    "fciqmc_iter_stats_count": (C.c_int64, [_H]),
    "fciqmc_step_batch": (C.c_int, [C.POINTER(_H), C.c_int32, C.c_int64]),
    "fciqmc_set_profiling": (C.c_int, [_H, C.c_int32]),
    "fciqmc_kernel_times": (C.c_int, [_H, _dp]),
    "fciqmc_layout": (C.c_int, [_H, C.POINTER(C.c_int64)]),
    "fciqmc_ref_offdiag_sum": (C.c_int, [_H, _dp]),
    "fciqmc_tau": (C.c_double, [_H]),
    "fciqmc_replica": (C.c_void_p, [_H, C.c_int32]),
    "fciqmc_trial_info": (C.c_int64, [_H, C.POINTER(C.c_int64), _dp, _u64p, _u64p, _dp, C.c_int64]),
    "fciqmc_pchb_table": (C.c_int64, [_H, C.c_int32, C.c_int32, C.c_int32, _dp, _dp, _u64p,
                                      C.POINTER(C.c_uint32), C.c_int64]),
    "fciqmc_autotune": (C.c_int, [C.POINTER(_H), C.c_int32, C.c_int64, C.POINTER(C.c_int32)]),
    "fciqmc_read_fcidump": (C.c_int, [C.c_char_p, C.POINTER(fciqmc_system)]),
    "fciqmc_free_system": (None, [C.POINTER(fciqmc_system)]),
    "fciqmc_ref_offdiag_sum_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                                 C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]),
    "fciqmc_graph_kernels": (C.c_int32, [_H]),
    "fciqmc_device_memory": (C.c_int, [C.c_int32, C.POINTER(C.c_int64)]),
    "fciqmc_set_launch_config": (C.c_int, [C.c_int32, C.c_int32, C.c_int32]),
    "fciqmc_get_launch_config": (C.c_int, [C.POINTER(C.c_int32)]),
    "fciqmc_semistoch_info": (C.c_int64, [_H, C.POINTER(C.c_int64)]),
    "fciqmc_server_create": (C.c_int, [C.c_int64, C.c_int32, C.c_void_p, C.POINTER(_H)]),
    "fciqmc_server_submit": (C.c_int, [_H, C.POINTER(fciqmc_system), C.POINTER(fciqmc_params), C.c_double,
                                       C.c_double, C.c_int64, C.POINTER(C.c_int64)]),
    "fciqmc_server_tick": (C.c_int, [_H, C.c_int64, C.POINTER(C.c_int32)]),
    "fciqmc_server_poll": (C.c_int, [_H, C.c_int64, C.POINTER(fciqmc_request_status)]),
    "fciqmc_server_clock": (C.c_double, [_H]),
    "fciqmc_server_destroy": (None, [_H]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def library_path():
    return _build.LIB


def _check(code, handle=None):
    if code != FCIQMC_OK:
        msg = _lib.fciqmc_last_error(handle)
        raise FciqmcError(code, msg.decode() if msg else "")


def _as_u64(x):
    a = np.ascontiguousarray(x, dtype=np.uint64)
    return a, a.ctypes.data_as(_u64p)


def _as_f64(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator."""

    def __init__(self, torch, stream):
        self.torch = torch
        self.stream = stream
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=self.stream)
        except Exception:
            return None

    def _free(self, ptr, ctx):
        try:
            self.torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass


def _system_struct(system):
    s = fciqmc_system()
    keep = []
    if system["kind"] == "hubbard":
        s.kind = FCIQMC_HUBBARD
        s.lx, s.ly = int(system["lx"]), int(system["ly"])
        s.norb = s.lx * s.ly
        s.periodic_x, s.periodic_y = int(bool(system["periodic_x"])), int(bool(system["periodic_y"]))
        s.t, s.U = float(system["t"]), float(system["U"])
    else:
        s.kind = FCIQMC_ABINITIO
        h1, hp = _as_f64(system["h1"])
        eri, ep = _as_f64(system["eri"])
        keep += [h1, eri]
        s.norb = int(h1.shape[0])
        s.h1, s.eri = hp, ep
        s.ecore = float(system.get("ecore", 0.0))
    s.n_alpha, s.n_beta = int(system["n_alpha"]), int(system["n_beta"])
    if system.get("ref") is not None:
        s.has_ref = 1
        s.ref_alpha, s.ref_beta = int(system["ref"][0]), int(system["ref"][1])
    return s, keep


DEFAULTS = dict(tau=0.01, shift_damping=0.1, target_walkers=1e4, initial_walkers=10.0, initial_shift=0.0,
                initiator_threshold=0.0, c_min=1.0, p_single=0.1, shift_interval=10, seed=1, semistoch_size=0,
                semistoch_start=100, max_dets=0, max_spawns=0, max_device_bytes=0, generator=0, replicas=1, trial_size=0, trial_start=100,
                adaptive_shift=0)


def _params_struct(params):
    p = dict(DEFAULTS)
    p.update(params or {})
    prm = fciqmc_params()
    ftypes = dict(fciqmc_params._fields_)
    for k in DEFAULTS:
        setattr(prm, k, float(p[k]) if ftypes[k] is C.c_double else int(p[k]))
    return prm


def fciqmc_create(system, params=None, stream=None, use_torch=True):
    """Create a run; returns an opaque handle (keep the returned object alive)."""
    s, keep = _system_struct(system)
    prm = _params_struct(params)
    allocator = None
    if stream is None and use_torch:
        try:
            import torch
            if torch.cuda.is_available():
                st = torch.cuda.current_stream()
                stream = st.cuda_stream
                allocator = _TorchAllocator(torch, st)
        except ImportError:
            pass
    prm.stream = stream
    if allocator is not None:
        prm.alloc = allocator.alloc_cb
        prm.free = allocator.free_cb
    h = _H()
    _check(_lib.fciqmc_create(C.byref(s), C.byref(prm), C.byref(h)), None)
    return Handle(h, keep, allocator, prm)


class Handle:
    def __init__(self, h, keep, allocator, prm):
        self.h, self._keep, self._allocator, self._prm = h, keep, allocator, prm

    def __del__(self):
        if getattr(self, "h", None):
            _lib.fciqmc_destroy(self.h)
            self.h = None


class _Replica:
    """A replica owned by its pair's first handle (kept alive through it; the
    library releases it together with the first)."""

    def __init__(self, h, parent):
        self.h, self._parent = h, parent


def fciqmc_destroy(handle):
    if handle.h:
        _lib.fciqmc_destroy(handle.h)
        handle.h = None


def fciqmc_step(handle, n_iter):
    _check(_lib.fciqmc_step(handle.h, int(n_iter)), handle.h)


def fciqmc_step_async(handle, n_iter):
    _check(_lib.fciqmc_step_async(handle.h, int(n_iter)), handle.h)


def fciqmc_sync(handle):
    _check(_lib.fciqmc_sync(handle.h), handle.h)


def fciqmc_stream(handle):
    return _lib.fciqmc_stream(handle.h)


def fciqmc_step_batch(handles, n_iter):
    arr = (_H * len(handles))(*[x.h for x in handles])
    _check(_lib.fciqmc_step_batch(arr, len(handles), int(n_iter)), handles[0].h if handles else None)


def fciqmc_energy(handle):
    st = fciqmc_stats()
    _check(_lib.fciqmc_energy(handle.h, C.byref(st)), handle.h)
    return {f: getattr(st, f) for f, _ in fciqmc_stats._fields_ if f != "pad0"}


def fciqmc_num_dets(handle):
    return _lib.fciqmc_num_dets(handle.h)


def fciqmc_export_state(handle, out=None):
    """The walker list (sorted by key) as arrays alpha, beta, c, hdiag, flags.
    `out`: optional dict of caller-owned arrays with those keys (uint64,
    uint64, float64, float64, int32; C-contiguous, e.g. views of pinned host
    memory kept across checkpoints); used when all hold the whole list, and
    the result is then views of them."""
    n = C.c_int64()
    _lib.fciqmc_export_state(handle.h, 0, None, None, None, None, None, C.byref(n))
    m = max(n.value, 1)
    want = (("alpha", np.uint64), ("beta", np.uint64), ("c", np.float64), ("hdiag", np.float64), ("flags", np.int32))
    if out is not None and all(k in out and out[k].dtype == t and out[k].ndim == 1 and out[k].size >= m and
                               out[k].flags["C_CONTIGUOUS"] and out[k].flags["WRITEABLE"] for k, t in want):
        a, b, c, hd, fl = (out[k] for k, _ in want)
        m = min(x.size for x in (a, b, c, hd, fl))
    else:
        # output pages are touched here: a first touch inside the CUDA driver's
        # pageable device-to-host copy costs ten times the copy itself
        a, b = np.empty(m, np.uint64), np.empty(m, np.uint64)
        c, hd = np.empty(m, np.float64), np.empty(m, np.float64)
        fl = np.empty(m, np.int32)
        for x in (a, b, c, hd, fl):
            x.fill(0)
    _check(_lib.fciqmc_export_state(handle.h, m, a.ctypes.data_as(_u64p), b.ctypes.data_as(_u64p),
                                    c.ctypes.data_as(_dp), hd.ctypes.data_as(_dp),
                                    fl.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)), handle.h)
    k = n.value
    return dict(alpha=a[:k], beta=b[:k], c=c[:k], hdiag=hd[:k], flags=fl[:k])


def fciqmc_export_shift(handle):
    it, S, vary, ss, cnt = C.c_int64(), C.c_double(), C.c_int32(), C.c_int64(), C.c_int64()
    hi, lo = C.c_uint64(), C.c_uint64()
    _check(_lib.fciqmc_export_shift(handle.h, C.byref(it), C.byref(S), C.byref(vary), C.byref(ss), C.byref(cnt),
                                    C.byref(hi), C.byref(lo)), handle.h)
    return dict(iteration=it.value, S=S.value, vary=vary.value, shift_start=ss.value, cnt=cnt.value,
                nw_last=(hi.value << 64) | lo.value)


def fciqmc_import_state(handle, alpha, beta, c, iteration, S, vary=0, shift_start=0, cnt=0, nw_last=0):
    a, ap = _as_u64(alpha)
    b, bp = _as_u64(beta)
    cc, cp = _as_f64(c)
    _check(_lib.fciqmc_import_state(handle.h, a.size, ap, bp, cp, int(iteration), float(S), int(vary),
                                    int(shift_start), int(cnt), (int(nw_last) >> 64) & 0xFFFFFFFFFFFFFFFF,
                                    int(nw_last) & 0xFFFFFFFFFFFFFFFF), handle.h)


def fciqmc_iter_stats_get(handle, first=0, count=None):
    n = _lib.fciqmc_iter_stats_count(handle.h)
    if count is None:
        count = n - first
    arr = (fciqmc_iter_stats * max(count, 1))()
    if count:
        _check(_lib.fciqmc_iter_stats_get(handle.h, first, count, arr), handle.h)
    names = [f for f, _ in fciqmc_iter_stats._fields_ if f != "pad0"]
    return {f: np.array([getattr(arr[i], f) for i in range(count)]) for f in names}


def fciqmc_iter_stats_count(handle):
    return _lib.fciqmc_iter_stats_count(handle.h)


def fciqmc_set_profiling(handle, on=True):
    _check(_lib.fciqmc_set_profiling(handle.h, int(bool(on))), handle.h)


def fciqmc_kernel_times(handle):
    out = (C.c_double * 6)()
    _check(_lib.fciqmc_kernel_times(handle.h, out), handle.h)
    return dict(spawn=out[0], spawn_heavy=out[1], annihilate=out[2], finalize=out[3], semistoch=out[4],
                new_diag=out[5])


def fciqmc_layout(handle):
    out = (C.c_int64 * 4)()
    _check(_lib.fciqmc_layout(handle.h, out), handle.h)
    return dict(buckets=out[0], cap_main=out[1], cap_spawn=out[2], device_bytes=out[3])


def fciqmc_graph_kernels(handle):
    """Kernel launches per iteration in the handle's captured graph."""
    return int(_lib.fciqmc_graph_kernels(handle.h))


def fciqmc_device_memory(device=0):
    """(peak memory clock in kHz, bus width in bits) of a CUDA device."""
    out = (C.c_int64 * 2)()
    _check(_lib.fciqmc_device_memory(int(device), out))
    return int(out[0]), int(out[1])


def fciqmc_semistoch_info(handle):
    """dict(nd, nnz): size of the deterministic space and stored entries of H^D."""
    nnz = C.c_int64()
    nd = _lib.fciqmc_semistoch_info(handle.h, C.byref(nnz))
    if nd < 0:
        _check(int(nd), handle.h)
    return dict(nd=int(nd), nnz=int(nnz.value))


def fciqmc_ref_offdiag_sum(handle):
    out = C.c_double()
    _check(_lib.fciqmc_ref_offdiag_sum(handle.h, C.byref(out)), handle.h)
    return out.value


def fciqmc_ref_offdiag_sum_noalloc(norb, n_alpha, n_beta, d_h1, d_eri, ref_alpha, ref_beta, d_out, stream=None):
    """Device pointers (ints) in, device pointer out; see include/fciqmc.h."""
    _check(_lib.fciqmc_ref_offdiag_sum_noalloc(int(norb), int(n_alpha), int(n_beta), d_h1, d_eri, int(ref_alpha),
                                               int(ref_beta), d_out, stream))


def fciqmc_tau(handle):
    return _lib.fciqmc_tau(handle.h)


def fciqmc_replica(handle, r):
    """Replica r of a pair (a handle that the pair owns: do not destroy it), or None."""
    p = _lib.fciqmc_replica(handle.h, int(r))
    if not p:
        return None
    if int(r) == 0:
        return handle
    return _Replica(p, handle)


def fciqmc_trial_info(handle):
    """Trial space of the E_Trial estimator: dict(nt, n_w, ET (E^T - E_ref), alpha, beta, cT)."""
    nw = C.c_int64()
    ET = C.c_double()
    nt = _lib.fciqmc_trial_info(handle.h, C.byref(nw), C.byref(ET), None, None, None, 0)
    if nt < 0:
        _check(int(nt), handle.h)
    a = np.zeros(max(nt, 1), np.uint64)
    b = np.zeros(max(nt, 1), np.uint64)
    cT = np.zeros(max(nt, 1))
    r = _lib.fciqmc_trial_info(handle.h, None, None, a.ctypes.data_as(_u64p), b.ctypes.data_as(_u64p),
                               cT.ctypes.data_as(_dp), nt)
    if r < 0:
        _check(int(r), handle.h)
    return dict(nt=int(nt), n_w=int(nw.value), ET=ET.value, alpha=a[:nt], beta=b[:nt], cT=cT[:nt])


def fciqmc_pchb_table(handle, same_spin, i, j):
    """One heat-bath table: dict(S, lam, threshold (uint64[K]), holes (uint32[K]))."""
    K = _lib.fciqmc_pchb_table(handle.h, int(same_spin), int(i), int(j), None, None, None, None, 0)
    if K < 0:
        _check(int(K), handle.h)
    S, lam = C.c_double(), C.c_double()
    thr = np.zeros(max(K, 1), np.uint64)
    holes = np.zeros(max(K, 1), np.uint32)
    r = _lib.fciqmc_pchb_table(handle.h, int(same_spin), int(i), int(j), C.byref(S), C.byref(lam),
                               thr.ctypes.data_as(_u64p), holes.ctypes.data_as(C.POINTER(C.c_uint32)), K)
    if r < 0:
        _check(int(r), handle.h)
    return dict(S=S.value, lam=lam.value, threshold=thr[:K], holes=holes[:K])


class Server:
    """Owner of a fciqmc_server (device memory is allocated with cudaMalloc)."""

    def __init__(self, h):
        self.h = h
        self._keep = []

    def __del__(self):
        if getattr(self, "h", None):
            _lib.fciqmc_server_destroy(self.h)
            self.h = None


def fciqmc_server_create(mem_budget_bytes, max_active=64, stream=None):
    h = _H()
    _check(_lib.fciqmc_server_create(int(mem_budget_bytes), int(max_active), stream, C.byref(h)))
    return Server(h)


def fciqmc_server_submit(server, system, params, target_sigma, max_iters, t_arrival=-1.0):
    s, keep = _system_struct(system)
    prm = _params_struct(params)
    rid = C.c_int64()
    _check(_lib.fciqmc_server_submit(server.h, C.byref(s), C.byref(prm), float(target_sigma), float(t_arrival),
                                     int(max_iters), C.byref(rid)))
    return rid.value


def fciqmc_server_tick(server, n_iter):
    n = C.c_int32()
    _check(_lib.fciqmc_server_tick(server.h, int(n_iter), C.byref(n)))
    return n.value


def fciqmc_server_poll(server, rid):
    st = fciqmc_request_status()
    _check(_lib.fciqmc_server_poll(server.h, int(rid), C.byref(st)))
    d = {f: getattr(st, f) for f, _ in fciqmc_request_status._fields_}
    d["state_name"] = REQUEST_STATES.get(d["state"], "?")
    return d


def fciqmc_server_clock(server):
    return _lib.fciqmc_server_clock(server.h)


def fciqmc_server_destroy(server):
    if server.h:
        _lib.fciqmc_server_destroy(server.h)
        server.h = None


def fciqmc_read_fcidump(path):
    """Parse an FCIDUMP file with the library's reader; returns a system dict
    (numpy copies of h1 and the packed ERI)."""
    s = fciqmc_system()
    _check(_lib.fciqmc_read_fcidump(str(path).encode(), C.byref(s)))
    try:
        N = s.norb
        npair = N * (N + 1) // 2
        h1 = np.ctypeslib.as_array(s.h1, shape=(N * N,)).reshape(N, N).copy()
        eri = np.ctypeslib.as_array(s.eri, shape=(npair * (npair + 1) // 2,)).copy()
        return dict(kind="abinitio", norb=N, n_alpha=s.n_alpha, n_beta=s.n_beta, h1=h1, eri=eri, ecore=s.ecore)
    finally:
        _lib.fciqmc_free_system(C.byref(s))


def fciqmc_set_launch_config(spawn, heavy, annihilate):
    """Launch configuration of every later launch (see include/fciqmc.h)."""
    _check(_lib.fciqmc_set_launch_config(int(spawn), int(heavy), int(annihilate)))


def fciqmc_get_launch_config():
    out = (C.c_int32 * 3)()
    _check(_lib.fciqmc_get_launch_config(out))
    return dict(spawn=out[0], heavy=out[1], annihilate=out[2])


def fciqmc_autotune(handles, n_iter):
    arr = (_H * len(handles))(*[x.h for x in handles])
    out = (C.c_int32 * 3)()
    _check(_lib.fciqmc_autotune(arr, len(handles), int(n_iter), out), handles[0].h)
    return dict(spawn_blocks_per_sm=out[0], heavy_blocks_per_sm=out[1], annihilate_blocks_per_sm=out[2])
