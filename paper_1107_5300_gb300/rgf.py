"""Python binding of the C ABI in ``include/rgf.h`` (argument marshalling only).

Every numeric step runs in ``librgf.so``; this module only converts arrays,
owns ribbon handles and raises on error codes.  It raises ``ImportError`` at
import time if the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

_LIB_PATH = Path(os.environ.get("RGF_LIB", Path(__file__).resolve().parent / "librgf.so"))
if not _LIB_PATH.exists():
    raise ImportError(f"{_LIB_PATH} not found: build it with `python -m paper_1107_5300_gb300.build`")
lib = C.CDLL(str(_LIB_PATH))

(RGF_OK, RGF_EINVAL, RGF_ENOMEM, RGF_ECUDA, RGF_ENOCONV, RGF_ESINGULAR, RGF_ENONFINITE,
 RGF_ETIMEOUT, RGF_EBOUNDS) = range(9)
RGF_FP64, RGF_MIXED, RGF_MIXED_TC, RGF_FP64_TC = 0, 1, 2, 3
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOCONV", "ESINGULAR", "ENONFINITE", "ETIMEOUT",
                "EBOUNDS"]

# Symbols declared in include/rgf.h (checked by the CPU tests).
EXPORTS = ["rgf_generate_onsite", "rgf_build_ribbon", "rgf_build_ribbon_dev", "rgf_free_ribbon",
           "rgf_lead_selfenergy", "rgf_conductance", "rgf_conductance_dev",
           "rgf_conductance_grad", "rgf_conductance_grad_dev", "rgf_ldos", "rgf_conductance_noalloc", "rgf_zgemm_tc",
           "rgf_zgemm_tc_selftest_timeout", "rgf_profile_enable", "rgf_profile_read",
           "rgf_profile_read_phases", "rgf_set_lead_controls", "rgf_status_str", "rgf_last_error",
           "rgf_version", "rgf_set_schedule", "rgf_get_schedule", "rgf_batch_create",
           "rgf_batch_launch", "rgf_batch_free", "rgf_set_tuning", "rgf_get_tuning",
           "rgf_tune_lookup", "rgf_autotune", "rgf_set_domains", "rgf_get_domains",
           "rgf_auto_domains"]
RGF_SCHED_PERSISTENT, RGF_SCHED_PHASED = 0, 1
RGF_ENGINE_PIPES, RGF_ENGINE_TENSOR = 0, 1
RGF_TUNE_MAX_ENTRIES, RGF_TUNE_MAX_CANDIDATES = 64, 12


class TuneEntry(C.Structure):
    """rgf_tune_entry: the schedule of the chains with ceil(N/2) <= K_max."""
    _fields_ = [("K_max", C.c_int), ("engine", C.c_int), ("panel", C.c_int), ("pairs", C.c_int)]

    def as_dict(self):
        return {"K_max": self.K_max, "engine": self.engine, "panel": self.panel, "pairs": self.pairs}


class _Desc(C.Structure):
    _fields_ = [("N", C.c_int), ("L", C.c_int), ("t", C.c_double),
                ("onsite", C.POINTER(C.c_double)), ("anderson_W", C.c_double),
                ("seed", C.c_uint64), ("edge_p", C.c_double), ("edge_seed", C.c_uint64),
                ("removed", C.POINTER(C.c_uint8))]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_i32p = C.POINTER(C.c_int32)
_u8p = C.POINTER(C.c_uint8)
_vp = C.c_void_p

lib.rgf_generate_onsite.argtypes = [C.POINTER(_Desc), _dp, _u8p]
lib.rgf_build_ribbon.argtypes = [C.POINTER(_Desc), C.POINTER(_vp)]
lib.rgf_build_ribbon_dev.argtypes = [C.c_int, C.c_int, C.c_double, _vp, _vp, _vp, C.POINTER(_vp)]
lib.rgf_free_ribbon.argtypes = [_vp]
lib.rgf_free_ribbon.restype = None
lib.rgf_lead_selfenergy.argtypes = [C.c_int, C.c_double, _dp, C.c_int, C.c_double, C.c_int, _dp, _ip]
lib.rgf_conductance.argtypes = [C.POINTER(_vp), _dp, C.c_int, C.c_double, C.c_double, C.c_int,
                                _dp, _i32p]
lib.rgf_conductance_dev.argtypes = [C.POINTER(_vp), _vp, C.c_int, C.c_double, C.c_double,
                                    C.c_int, _vp, _vp, _vp]
lib.rgf_conductance_grad.argtypes = [C.POINTER(_vp), _dp, C.c_int, C.c_double, C.c_double,
                                     C.c_int, C.c_int, _dp, _dp, _i32p]
lib.rgf_conductance_grad_dev.argtypes = [C.POINTER(_vp), _vp, C.c_int, C.c_double, C.c_double,
                                         C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp]
lib.rgf_ldos.argtypes = [C.POINTER(_vp), _dp, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                         _dp, _dp, _i32p]
lib.rgf_conductance_noalloc.argtypes = [C.c_int, C.c_int, C.c_double, _vp, _vp, _vp, C.c_int,
                                        C.c_double, C.c_double, C.c_int, _vp, _vp, _vp]
lib.rgf_conductance_noalloc.restype = C.c_int
lib.rgf_zgemm_tc.argtypes = [C.c_int, C.c_int, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp, C.c_int,
                             _vp]
lib.rgf_zgemm_tc.restype = C.c_int
lib.rgf_zgemm_tc_selftest_timeout.argtypes = []
lib.rgf_zgemm_tc_selftest_timeout.restype = C.c_int
lib.rgf_profile_enable.argtypes = [C.c_int]
lib.rgf_profile_enable.restype = C.c_int
lib.rgf_profile_read.argtypes = [_dp, _dp]
lib.rgf_profile_read.restype = C.c_int
lib.rgf_profile_read_phases.argtypes = [_dp]
lib.rgf_profile_read_phases.restype = C.c_int
lib.rgf_set_lead_controls.argtypes = [C.c_int, C.c_double]
lib.rgf_set_lead_controls.restype = C.c_int
lib.rgf_set_schedule.argtypes = [C.c_int]
lib.rgf_set_schedule.restype = C.c_int
lib.rgf_get_schedule.argtypes = []
lib.rgf_get_schedule.restype = C.c_int
lib.rgf_batch_create.argtypes = [C.POINTER(_vp), _vp, C.c_int, C.c_double, C.c_double, C.c_int,
                                 _vp, _vp, C.POINTER(_vp)]
lib.rgf_batch_create.restype = C.c_int
lib.rgf_batch_launch.argtypes = [_vp, _vp]
lib.rgf_batch_launch.restype = C.c_int
lib.rgf_batch_free.argtypes = [_vp]
lib.rgf_batch_free.restype = None
lib.rgf_set_tuning.argtypes = [C.c_int, C.POINTER(TuneEntry), C.c_int]
lib.rgf_set_tuning.restype = C.c_int
lib.rgf_get_tuning.argtypes = [C.c_int, C.POINTER(TuneEntry), C.c_int, _ip]
lib.rgf_get_tuning.restype = C.c_int
lib.rgf_tune_lookup.argtypes = [C.c_int, C.c_int, C.POINTER(TuneEntry)]
lib.rgf_tune_lookup.restype = C.c_int
lib.rgf_autotune.argtypes = [C.c_int, _ip, C.c_int, C.c_int, C.c_int, C.POINTER(TuneEntry), _dp, _ip]
lib.rgf_autotune.restype = C.c_int
lib.rgf_set_domains.argtypes = [C.c_int]
lib.rgf_set_domains.restype = C.c_int
lib.rgf_get_domains.argtypes = []
lib.rgf_get_domains.restype = C.c_int
lib.rgf_auto_domains.argtypes = [C.c_int, C.c_int, C.c_int]
lib.rgf_auto_domains.restype = C.c_int
lib.rgf_status_str.restype = C.c_char_p
lib.rgf_status_str.argtypes = [C.c_int]
lib.rgf_last_error.restype = C.c_char_p
lib.rgf_version.restype = C.c_char_p
for _f in ("rgf_generate_onsite", "rgf_build_ribbon", "rgf_build_ribbon_dev", "rgf_lead_selfenergy",
           "rgf_conductance", "rgf_conductance_dev", "rgf_conductance_grad",
           "rgf_conductance_grad_dev", "rgf_ldos"):
    getattr(lib, _f).restype = C.c_int


class RGFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


# Per-chain failures (the call ran and every chain has its status); the other
# codes (RGF_EINVAL, RGF_ENOMEM, RGF_ECUDA from a host-buffer call) mean the
# outputs were not written, and always raise.
_CHAIN_ERRORS = (RGF_ENOCONV, RGF_ESINGULAR, RGF_ENONFINITE, RGF_ETIMEOUT, RGF_EBOUNDS)


def _check(st: int, allow=()):
    if st != RGF_OK and st not in allow:
        raise RGFError(st, lib.rgf_last_error().decode())
    return st


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _desc(N, L, t, onsite, W, seed, edge_p, edge_seed, removed):
    d = _Desc()
    d.N, d.L, d.t = int(N), int(L), float(t)
    d.onsite = _ptr(onsite, C.c_double)
    d.anderson_W, d.seed = float(W), int(seed) & 0xFFFFFFFFFFFFFFFF
    d.edge_p, d.edge_seed = float(edge_p), int(edge_seed) & 0xFFFFFFFFFFFFFFFF
    d.removed = _ptr(removed, C.c_uint8)
    return d


def generate_onsite(N, L, t=-2.7, W=0.0, seed=0, edge_p=0.0, edge_seed=0):
    """Host-only: the (eps, removed) arrays [L, 2N] a seeded ribbon description yields."""
    eps = np.empty((L, 2 * N), dtype=np.float64)
    rem = np.empty((L, 2 * N), dtype=np.uint8)
    d = _desc(N, L, t, None, W, seed, edge_p, edge_seed, None)
    _check(lib.rgf_generate_onsite(C.byref(d), _ptr(eps, C.c_double), _ptr(rem, C.c_uint8)))
    return eps, rem


class Ribbon:
    """A ribbon instance resident on the current CUDA device (rgf_build_ribbon)."""

    def __init__(self, N, L, t=-2.7, onsite=None, W=0.0, seed=0, edge_p=0.0, edge_seed=0,
                 removed=None):
        self.N, self.L, self.t = int(N), int(L), float(t)
        on = None if onsite is None else np.ascontiguousarray(onsite, dtype=np.float64).reshape(-1)
        rm = None if removed is None else np.ascontiguousarray(removed, dtype=np.uint8).reshape(-1)
        if on is not None and on.size != self.L * 2 * self.N:
            raise ValueError("onsite must have L*2N entries")
        if rm is not None and rm.size != self.L * 2 * self.N:
            raise ValueError("removed must have L*2N entries")
        d = _desc(N, L, t, on, W, seed, edge_p, edge_seed, rm)
        h = _vp()
        _check(lib.rgf_build_ribbon(C.byref(d), C.byref(h)))
        self._h = h

    @classmethod
    def from_device(cls, N, L, t, onsite_ptr, removed_ptr=None, stream=0):
        """Build from device buffers (e.g. torch CUDA tensors' data_ptr())."""
        self = cls.__new__(cls)
        self.N, self.L, self.t = int(N), int(L), float(t)
        h = _vp()
        _check(lib.rgf_build_ribbon_dev(self.N, self.L, self.t, _vp(onsite_ptr),
                                        _vp(removed_ptr) if removed_ptr else None,
                                        _vp(stream), C.byref(h)))
        self._h = h
        return self

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib.rgf_free_ribbon(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _handles(ribbons):
    arr = (_vp * len(ribbons))()
    for i, r in enumerate(ribbons):
        arr[i] = r.handle
    return arr


def lead_selfenergy(N, E, eta=1e-8, side=0, t=-2.7, check=True):
    """Full-cell (2N x 2N) lead self-energies, one per energy: returns (sigma[nE,2N,2N], iters)."""
    E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
    M = 2 * N
    out = np.empty((E.size, M, M, 2), dtype=np.float64)
    it = np.empty(E.size, dtype=np.int32)
    st = lib.rgf_lead_selfenergy(int(N), float(t), _ptr(E, C.c_double), E.size, float(eta),
                                 int(side), _ptr(out, C.c_double), it.ctypes.data_as(_ip))
    if check:
        _check(st)
    sig = out[..., 0] + 1j * out[..., 1]
    return sig, it


def conductance(ribbons, E, eta_device=1e-8, eta_lead=1e-8, precision=RGF_FP64, check=True):
    """T for chains (ribbons[c], E[c]); host buffers.  Returns (T, status)."""
    E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
    if len(ribbons) != E.size:
        raise ValueError("one ribbon per energy")
    T = np.empty(E.size)
    st = np.empty(E.size, dtype=np.int32)
    r = lib.rgf_conductance(_handles(ribbons), _ptr(E, C.c_double), E.size, float(eta_device),
                            float(eta_lead), int(precision), _ptr(T, C.c_double),
                            st.ctypes.data_as(_i32p))
    _check(r, allow=() if check else _CHAIN_ERRORS)
    return T, st


def conductance_dev(ribbons, E_ptr, n, T_ptr, status_ptr=0, eta_device=1e-8, eta_lead=1e-8,
                    precision=RGF_FP64, stream=0):
    """Device-buffer variant: pointers to n float64 energies / outputs on the device."""
    _check(lib.rgf_conductance_dev(_handles(ribbons), _vp(E_ptr), int(n), float(eta_device),
                                   float(eta_lead), int(precision), _vp(stream), _vp(T_ptr),
                                   _vp(status_ptr) if status_ptr else None))


def conductance_grad(ribbons, E, eta_device=1e-8, eta_lead=1e-8, precision=RGF_FP64,
                     ckpt_stride=0, check=True):
    """T and dT/d eps [nchains, L, 2N] (host buffers).  Returns (T, grad, status)."""
    E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
    if len(ribbons) != E.size:
        raise ValueError("one ribbon per energy")
    sizes = [r.L * 2 * r.N for r in ribbons]
    if len(set(sizes)) > 1:
        raise ValueError("conductance_grad binding expects ribbons of one size")
    T = np.empty(E.size)
    g = np.empty((E.size, ribbons[0].L, 2 * ribbons[0].N)) if ribbons else np.empty(0)
    st = np.empty(E.size, dtype=np.int32)
    r = lib.rgf_conductance_grad(_handles(ribbons), _ptr(E, C.c_double), E.size,
                                 float(eta_device), float(eta_lead), int(precision),
                                 int(ckpt_stride), _ptr(T, C.c_double), _ptr(g, C.c_double),
                                 st.ctypes.data_as(_i32p))
    _check(r, allow=() if check else _CHAIN_ERRORS)
    return T, g, st


def conductance_grad_dev(ribbons, E_ptr, n, T_ptr, dT_ptr, weights_ptr=0, status_ptr=0,
                         eta_device=1e-8, eta_lead=1e-8, precision=RGF_FP64, ckpt_stride=0,
                         stream=0):
    """Device-buffer gradient: per-chain dT/d eps into dT_ptr, or with weights_ptr
    (n float64 on the device) their weighted sum [L*2N]."""
    _check(lib.rgf_conductance_grad_dev(_handles(ribbons), _vp(E_ptr), int(n), float(eta_device),
                                        float(eta_lead), int(precision), int(ckpt_stride),
                                        _vp(weights_ptr) if weights_ptr else None, _vp(stream),
                                        _vp(T_ptr), _vp(dT_ptr),
                                        _vp(status_ptr) if status_ptr else None))


def ldos(ribbons, E, eta_device=1e-8, eta_lead=1e-8, precision=RGF_FP64, ckpt_stride=0,
         check=True):
    """T and the local density of states -Im G_ii / pi [nchains, L, 2N] (host buffers).
    Returns (T, rho, status)."""
    E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
    if len(ribbons) != E.size:
        raise ValueError("one ribbon per energy")
    sizes = [r.L * 2 * r.N for r in ribbons]
    if len(set(sizes)) > 1:
        raise ValueError("ldos binding expects ribbons of one size")
    T = np.empty(E.size)
    rho = np.empty((E.size, ribbons[0].L, 2 * ribbons[0].N)) if ribbons else np.empty(0)
    st = np.empty(E.size, dtype=np.int32)
    r = lib.rgf_ldos(_handles(ribbons), _ptr(E, C.c_double), E.size, float(eta_device),
                     float(eta_lead), int(precision), int(ckpt_stride), _ptr(T, C.c_double),
                     _ptr(rho, C.c_double), st.ctypes.data_as(_i32p))
    _check(r, allow=() if check else _CHAIN_ERRORS)
    return T, rho, st


def profile_enable(on=True):
    """Record CUDA events around the kernel phases of each conductance call."""
    _check(lib.rgf_profile_enable(1 if on else 0))


def profile_read():
    """(ms_lead, ms_sweep) of the last profiled call (waits for it)."""
    a, b = C.c_double(), C.c_double()
    _check(lib.rgf_profile_read(C.byref(a), C.byref(b)))
    return a.value, b.value


def profile_read_phases():
    """Milliseconds of the last profiled call: (lead, end-column preparation,
    half sweeps or gradient sweep, join and trace)."""
    ms = np.zeros(4)
    _check(lib.rgf_profile_read_phases(_ptr(ms, C.c_double)))
    return tuple(float(x) for x in ms)


def set_lead_controls(max_iter=200, residual_tol=1e-10):
    """Iteration cap and residual tolerance of the lead decimation (process-wide)."""
    _check(lib.rgf_set_lead_controls(int(max_iter), float(residual_tol)))


def conductance_noalloc(N, L, t, onsite_ptr, removed_ptr, E_ptr, n, T_ptr, status_ptr=0,
                        eta_device=1e-8, eta_lead=1e-8, precision=RGF_FP64, stream=0, check=True):
    """Allocation-free call (device pointers in and out; scratch in the library's fixed array)."""
    st = lib.rgf_conductance_noalloc(int(N), int(L), float(t), _vp(onsite_ptr),
                                     _vp(removed_ptr) if removed_ptr else None, _vp(E_ptr), int(n),
                                     float(eta_device), float(eta_lead), int(precision),
                                     _vp(stream), _vp(T_ptr), _vp(status_ptr) if status_ptr else None)
    if check:
        _check(st)
    return st


def zgemm_tc_selftest_timeout():
    """Runs the tensor-core product with its completion wait forced to run out;
    returns the status (RGF_ETIMEOUT when the timeout path works)."""
    return lib.rgf_zgemm_tc_selftest_timeout()


def zgemm_tc(A_ptr, B_ptr, C_ptr, m, n, k, lda=None, ldb=None, ldc=None, stream=0, check=True):
    """C = A B on the tensor cores (device pointers to complex128 row-major data)."""
    st = lib.rgf_zgemm_tc(int(m), int(n), int(k), _vp(A_ptr), int(lda or max(k, 1)), _vp(B_ptr),
                          int(ldb or max(n, 1)), _vp(C_ptr), int(ldc or max(n, 1)), _vp(stream))
    if check:
        _check(st)
    return st


def set_schedule(schedule):
    """RGF_SCHED_PHASED (default) or RGF_SCHED_PERSISTENT for the forward sweep (process-wide)."""
    _check(lib.rgf_set_schedule(int(schedule)))


def get_schedule():
    return int(lib.rgf_get_schedule())


def _table(entries):
    arr = (TuneEntry * max(len(entries), 1))()
    for i, e in enumerate(entries):
        d = e.as_dict() if isinstance(e, TuneEntry) else e
        arr[i] = TuneEntry(int(d["K_max"]), int(d["engine"]), int(d["panel"]), int(d["pairs"]))
    return arr


def set_tuning(precision, entries):
    """Installs a tuning table (list of dicts with K_max, engine, panel, pairs; [] removes it)."""
    arr = _table(entries)
    _check(lib.rgf_set_tuning(int(precision), arr, len(entries)))


def get_tuning(precision):
    arr = (TuneEntry * RGF_TUNE_MAX_ENTRIES)()
    n = C.c_int(0)
    _check(lib.rgf_get_tuning(int(precision), arr, RGF_TUNE_MAX_ENTRIES, C.byref(n)))
    return [arr[i].as_dict() for i in range(n.value)]


def tune_lookup(precision, N):
    """The schedule a ribbon of width N gets from the installed table."""
    e = TuneEntry()
    _check(lib.rgf_tune_lookup(int(precision), int(N), C.byref(e)))
    return e.as_dict()


def autotune(precision, widths, cells=4, reps=2):
    """Times every candidate schedule on one chain per width, installs the
    fastest per column size and returns (table, ms [len(widths), ncand])."""
    Ns = np.ascontiguousarray(widths, dtype=np.int32)
    best = (TuneEntry * len(Ns))()
    ms = np.full((len(Ns), RGF_TUNE_MAX_CANDIDATES), np.nan)
    nc = C.c_int(0)
    _check(lib.rgf_autotune(int(precision), Ns.ctypes.data_as(_ip), len(Ns), int(cells), int(reps),
                            best, _ptr(ms, C.c_double), C.byref(nc)))
    ms = ms.reshape(-1)[: len(Ns) * nc.value].reshape(len(Ns), nc.value)
    return [best[i].as_dict() for i in range(len(Ns))], ms


def save_tuning(path, precisions=(RGF_FP64, RGF_MIXED, RGF_MIXED_TC, RGF_FP64_TC)):
    """Writes the installed tables to a JSON file."""
    import json
    Path(path).write_text(json.dumps({str(p): get_tuning(p) for p in precisions}, indent=1))


def load_tuning(path):
    """Installs the tables of a JSON file written by save_tuning."""
    import json
    for p, entries in json.loads(Path(path).read_text()).items():
        set_tuning(int(p), entries)


class Batch:
    """A prepared batch (rgf_batch_create): the forward path of a fixed list of
    chains as one CUDA graph.  E_ptr, T_ptr, status_ptr: device pointers the
    graph keeps; launch() re-reads the energies and the ribbons each time."""

    def __init__(self, ribbons, E_ptr, n, T_ptr, status_ptr=0, eta_device=1e-8, eta_lead=1e-8,
                 precision=RGF_FP64):
        self._ribbons = list(ribbons)          # kept alive with the graph
        hs = _handles(self._ribbons)
        h = _vp()
        _check(lib.rgf_batch_create(hs, _vp(E_ptr), int(n), float(eta_device), float(eta_lead),
                                    int(precision), _vp(T_ptr),
                                    _vp(status_ptr) if status_ptr else None, C.byref(h)))
        self._h = h

    def launch(self, stream=0):
        _check(lib.rgf_batch_launch(self._h, _vp(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib.rgf_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_domains(ndom):
    """Domains per chain of the forward sweep (default 2; 0 = automatic; process-wide)."""
    _check(lib.rgf_set_domains(int(ndom)))


def get_domains():
    return int(lib.rgf_get_domains())


def auto_domains(nchains, ncol_min, nsm):
    """The automatic domain count for nchains chains, the shortest of ncol_min columns, nsm SMs."""
    return int(lib.rgf_auto_domains(int(nchains), int(ncol_min), int(nsm)))
