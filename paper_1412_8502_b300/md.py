"""Thin ctypes binding of the C ABI in ``include/md.h``.

Argument marshalling only: every step of the MD path runs in the CUDA
kernels of ``libmd_b300.so``.  If the library is missing or cannot be
loaded, importing this module raises; there is no fallback.

Low-level functions keep the C names (``md_create``, ``md_step``, ...);
``System`` and ``Batch`` wrap a handle with numpy in/out.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "libmd_b300.so"

MD_OK = 0
MD_EINVAL = -1
MD_ENOMEM = -2
MD_ECUDA = -3
MD_ETIMEOUT = -4
MD_ENUMERIC = -5
MD_ENODEV = -6
MD_EAGAIN = -7
MD_PREC_SPLIT = 0
MD_PREC_FP64 = 1

_D = ctypes.c_double
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


class md_params(ctypes.Structure):
    _fields_ = [("dt", _D), ("r_nuc", _D), ("r_C", _D), ("lambda_s", _D), ("skin", _D),
                ("rebuild_every", _I64), ("thermostat_every", _I64), ("T", _D),
                ("precision", _I32), ("coulomb", _I32), ("r_pp", _D), ("r_np", _D),
                ("relax_iters", _I64), ("relax_gamma", _D), ("relax_dmax", _D),
                ("energy_every", _I64), ("sort_bits", _I32), ("affine", _I32), ("list_kind", _I32),
                ("verlet_pool", _D), ("cond_graph", _I32), ("force_unroll", _I32),
                ("uf_iter_limit", _I64), ("wait_limit_ns", _I64), ("persistent", _I32)]


class md_energy_t(ctypes.Structure):
    _fields_ = [("KE", _D), ("PE_nuc", _D), ("PE_coul", _D), ("virial", _D), ("L", _D),
                ("t", _D), ("step", _I64), ("pairs_nuc", _I64), ("pairs_coul", _I64),
                ("candidates", _I64)]


class md_state_view(ctypes.Structure):
    _fields_ = [("N", _I64), ("Np", _I64), ("x", ctypes.POINTER(_D)), ("v", ctypes.POINTER(_D)),
                ("type", ctypes.POINTER(ctypes.c_int8)), ("L", _D), ("L_base", _D), ("t", _D),
                ("t_base", _D), ("xi_dot", _D), ("L_F", _D), ("step", _I64), ("f", ctypes.POINTER(_D))]


class md_cluster_stats(ctypes.Structure):
    _fields_ = [("n_clusters", _I64), ("n_free", _I64), ("n_big", _I64), ("m_free_n", _D),
                ("A_mean", _D), ("Z_mean", _D)]


class md_info_t(ctypes.Structure):
    _fields_ = [("N", _I64), ("Np", _I64), ("tiles", _I64), ("rebuilds", _I64),
                ("list_entries", _I64), ("launches", _I64), ("device_bytes", _I64),
                ("need_wrap", _I32), ("sort_bits", _I32), ("tile_halfext_mean", _D), ("tile_halfext_max", _D),
                ("verlet_entries", _I64), ("verlet_slots", _I64), ("verlet_capacity", _I64),
                ("force_code", _I32), ("pad0", _I32), ("force_trials", _I64)]


class md_job(ctypes.Structure):
    _fields_ = [("N", _I64), ("Yp", _D), ("rho", _D), ("T", _D), ("seed", ctypes.c_uint64),
                ("xi_dot", _D), ("steps", _I64)]


class md_result(ctypes.Structure):
    _fields_ = [("id", _I64), ("status", _I32), ("reserved0", _I32), ("N", _I64), ("steps", _I64),
                ("energy", md_energy_t), ("wait_ms", _D), ("run_ms", _D), ("step_p50_ms", _D),
                ("step_p99_ms", _D)]


_P = ctypes.c_void_p
_SIGS = {
    "md_params_default": (None, [ctypes.POINTER(md_params)]),
    "md_create": (ctypes.c_int, [_I64, _D, _D, _D, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "md_create_ex": (ctypes.c_int, [_I64, _D, _D, _D, ctypes.c_uint64, ctypes.POINTER(md_params),
                                    ctypes.POINTER(_P)]),
    "md_destroy": (ctypes.c_int, [_P]),
    "md_get_params": (ctypes.c_int, [_P, ctypes.POINTER(md_params)]),
    "md_set_params": (ctypes.c_int, [_P, ctypes.POINTER(md_params)]),
    "md_set_stream": (ctypes.c_int, [_P, _P]),
    "md_step": (ctypes.c_int, [_P, _I64, _D]),
    "md_step_async": (ctypes.c_int, [_P, _I64, _D]),
    "md_sync": (ctypes.c_int, [_P]),
    "md_forces": (ctypes.c_int, [_P, ctypes.POINTER(_D)]),
    "md_energy": (ctypes.c_int, [_P, ctypes.POINTER(md_energy_t)]),
    "md_step_energy": (ctypes.c_int, [_P, ctypes.POINTER(md_energy_t)]),
    "md_clusters": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                   ctypes.POINTER(md_cluster_stats)]),
    "md_clusters_mste": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                        ctypes.POINTER(md_cluster_stats)]),
    "md_get_state": (ctypes.c_int, [_P, ctypes.POINTER(md_state_view)]),
    "md_set_state": (ctypes.c_int, [_P, ctypes.POINTER(md_state_view)]),
    "md_get_info": (ctypes.c_int, [_P, ctypes.POINTER(md_info_t)]),
    "md_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "md_kernel_times": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.POINTER(_I64), ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_int)]),
    "md_last_error": (ctypes.c_char_p, []),
    "md_debug_fail_alloc": (ctypes.c_int, [_I64]),
    "md_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(md_job), ctypes.POINTER(md_params),
                                       ctypes.POINTER(_P)]),
    "md_batch_step": (ctypes.c_int, [_P, _I64]),
    "md_batch_system": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "md_batch_destroy": (ctypes.c_int, [_P]),
    "md_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(md_params), ctypes.POINTER(_P)]),
    "md_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(md_job), ctypes.POINTER(_I64)]),
    "md_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(md_result)]),
    "md_server_drain": (ctypes.c_int, [_P, _D]),
    "md_server_destroy": (ctypes.c_int, [_P]),
    "md_autotune": (ctypes.c_int, [_P, _I64, ctypes.POINTER(md_params)]),
    "md_batch_autotune": (ctypes.c_int, [_P, _I64, ctypes.POINTER(md_params)]),
    "md_lambda_thomas_fermi": (ctypes.c_double, [_D]),
    "md_clusters_noalloc": (ctypes.c_int, [_P, _I64, _I64, _D, _D, _D, _P, _P, _P, _P, _P]),
}


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"{_LIB_PATH} is missing: run paper_1412_8502_b300.build.build() "
                          "(the CUDA library is required; there is no CPU path)")
    lib = ctypes.CDLL(str(_LIB_PATH))
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


class MDError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = LIB.md_last_error()
        super().__init__(f"{where} failed with {code}: {msg.decode() if msg else ''}")
        self.code = code


def _ck(rc: int, where: str) -> None:
    if rc != MD_OK:
        raise MDError(rc, where)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(_D))


# ---------------------------------------------------------------- C names
def md_params_default() -> md_params:
    p = md_params()
    LIB.md_params_default(ctypes.byref(p))
    return p


def md_create(N, Yp, rho, T, seed, params: md_params | None = None):
    h = _P()
    if params is None:
        _ck(LIB.md_create(int(N), float(Yp), float(rho), float(T), int(seed), ctypes.byref(h)), "md_create")
    else:
        _ck(LIB.md_create_ex(int(N), float(Yp), float(rho), float(T), int(seed), ctypes.byref(params),
                             ctypes.byref(h)), "md_create_ex")
    return h


def md_destroy(h) -> None:
    _ck(LIB.md_destroy(h), "md_destroy")


def md_step(h, n: int, xi_dot: float = 0.0) -> None:
    _ck(LIB.md_step(h, int(n), float(xi_dot)), "md_step")


def md_step_async(h, n: int, xi_dot: float = 0.0) -> None:
    _ck(LIB.md_step_async(h, int(n), float(xi_dot)), "md_step_async")


def md_sync(h) -> None:
    _ck(LIB.md_sync(h), "md_sync")


def md_forces(h, N: int) -> np.ndarray:
    f = np.empty((N, 3), dtype=np.float64)
    _ck(LIB.md_forces(h, _dp(f)), "md_forces")
    return f


def md_energy(h) -> dict:
    e = md_energy_t()
    _ck(LIB.md_energy(h, ctypes.byref(e)), "md_energy")
    return {k: getattr(e, k) for k, _ in md_energy_t._fields_}


def md_step_energy(h) -> dict:
    e = md_energy_t()
    _ck(LIB.md_step_energy(h, ctypes.byref(e)), "md_step_energy")
    return {k: getattr(e, k) for k, _ in md_energy_t._fields_}


def md_get_info(h) -> dict:
    i = md_info_t()
    _ck(LIB.md_get_info(h, ctypes.byref(i)), "md_get_info")
    return {k: getattr(i, k) for k, _ in md_info_t._fields_}


def _state_array(a, N, what):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.shape == (N, 3) and a.flags.c_contiguous):
        raise ValueError(f"{what} must be a C-contiguous float64 array of shape ({N}, 3)")
    return a


def md_get_state(h, N: int, x=True, v=True, type=True, out=None, f=False) -> dict:
    """State in original particle order.  f: also the cached forces (the
    ones the next half-kick uses, evaluated with box side L_F).  `out` may
    supply preallocated (x, v) or (x, v, f) arrays (e.g. pinned host memory)
    of shape (N, 3)."""
    fs = None
    if out is not None:
        xs, vs = _state_array(out[0], N, "x"), _state_array(out[1], N, "v")
        if len(out) > 2 and out[2] is not None:
            fs = _state_array(out[2], N, "f")
    else:
        xs = np.empty((N, 3)) if x else None
        vs = np.empty((N, 3)) if v else None
        fs = np.empty((N, 3)) if f else None
    ts = np.empty(N, dtype=np.int8) if type else None
    view = md_state_view()
    view.x = _dp(xs) if xs is not None else None
    view.v = _dp(vs) if vs is not None else None
    view.f = _dp(fs) if fs is not None else None
    view.type = ts.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)) if ts is not None else None
    _ck(LIB.md_get_state(h, ctypes.byref(view)), "md_get_state")
    return dict(x=xs, v=vs, f=fs, type=ts, N=view.N, Np=view.Np, L=view.L, L_base=view.L_base, t=view.t,
                t_base=view.t_base, xi_dot=view.xi_dot, L_F=view.L_F, step=view.step)


def md_set_state(h, x, v, L, L_base=None, t=0.0, t_base=0.0, xi_dot=0.0, step=0, Np=None, f=None,
                 L_F=None) -> None:
    """Load x, v (and the clock).  With f (forces as md_get_state returns
    them, evaluated with box side L_F) the forces are restored instead of
    re-evaluated."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    N = x.shape[0]
    if f is not None:
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (N, 3):
            raise ValueError(f"f must have shape ({N}, 3)")
    if Np is None:
        Np = md_get_info(h)["Np"]
    view = md_state_view(N=N, Np=Np, x=_dp(x), v=_dp(v), type=None, L=float(L),
                         L_base=float(L if L_base is None else L_base), t=float(t), t_base=float(t_base),
                         xi_dot=float(xi_dot), L_F=float(L if L_F is None else L_F), step=int(step),
                         f=_dp(f) if f is not None else None)
    _ck(LIB.md_set_state(h, ctypes.byref(view)), "md_set_state")


def _out_array(a, n, dt, what):
    if not (isinstance(a, np.ndarray) and a.dtype == dt and a.shape == (n,) and a.flags.c_contiguous
            and a.flags.writeable):
        raise ValueError(f"{what} must be a writeable C-contiguous {np.dtype(dt).name}[{n}] array")
    return a


def md_clusters(h, N: int, Np: int, labels=True, fn="md_clusters", out=None):
    """Labels (int32[N], or None when labels is False), hist_A (int64[N+1]),
    hist_Z (int64[Np+1]) and the statistics.  out: optional (labels or None,
    hist_A, hist_Z) arrays to fill instead of new ones (e.g. page-locked
    buffers reused across calls); they are returned."""
    if out is not None:
        lab, hA, hZ = out
        lab = _out_array(lab, N, np.int32, "labels") if labels else None
        hA = _out_array(hA, N + 1, np.int64, "hist_A")
        hZ = _out_array(hZ, Np + 1, np.int64, "hist_Z")
    else:
        lab = np.empty(N, dtype=np.int32) if labels else None
        hA = np.zeros(N + 1, dtype=np.int64)
        hZ = np.zeros(Np + 1, dtype=np.int64)
    st = md_cluster_stats()
    _ck(getattr(LIB, fn)(h, lab.ctypes.data_as(ctypes.POINTER(_I32)) if lab is not None else None,
                         hA.ctypes.data_as(ctypes.POINTER(_I64)), hZ.ctypes.data_as(ctypes.POINTER(_I64)),
                         ctypes.byref(st)), fn)
    return lab, hA, hZ, {k: getattr(st, k) for k, _ in md_cluster_stats._fields_}


def md_clusters_mste(h, N: int, Np: int, labels=True, out=None):
    return md_clusters(h, N, Np, labels, fn="md_clusters_mste", out=out)


def md_clusters_noalloc(d_x, N, Np, L, r_pp, r_np, d_labels, d_hist_A, d_hist_Z, d_counts, stream=None) -> None:
    """Cluster analysis on caller-owned device buffers (raw device pointers
    as ints); allocates nothing.  See md_clusters_noalloc in md.h."""
    ptr = getattr(stream, "cuda_stream", stream)
    _ck(LIB.md_clusters_noalloc(_P(d_x), int(N), int(Np), float(L), float(r_pp), float(r_np), _P(d_labels),
                                _P(d_hist_A), _P(d_hist_Z), _P(d_counts), _P(ptr or 0)), "md_clusters_noalloc")


def md_get_params(h) -> md_params:
    p = md_params()
    _ck(LIB.md_get_params(h, ctypes.byref(p)), "md_get_params")
    return p


def md_set_params(h, p: md_params) -> None:
    _ck(LIB.md_set_params(h, ctypes.byref(p)), "md_set_params")


def md_set_stream(h, stream) -> None:
    """stream: an int cudaStream_t handle, a torch.cuda.Stream, or None."""
    ptr = getattr(stream, "cuda_stream", stream)
    _ck(LIB.md_set_stream(h, ctypes.c_void_p(ptr or 0)), "md_set_stream")


def md_set_timing(h, on) -> None:
    """on: False/0 off, True/1 every kernel, 2 key kernels only."""
    _ck(LIB.md_set_timing(h, int(on)), "md_set_timing")


def md_kernel_times(h) -> dict:
    n = ctypes.c_int()
    _ck(LIB.md_kernel_times(h, 0, None, None, None, ctypes.byref(n)), "md_kernel_times")
    k = n.value
    names = (ctypes.c_char_p * max(k, 1))()
    cnt = (_I64 * max(k, 1))()
    ms = (_D * max(k, 1))()
    _ck(LIB.md_kernel_times(h, k, names, cnt, ms, ctypes.byref(n)), "md_kernel_times")
    return {names[i].decode(): (cnt[i], ms[i]) for i in range(k)}


def md_lambda_thomas_fermi(n_e: float) -> float:
    return LIB.md_lambda_thomas_fermi(float(n_e))


def md_autotune(h, steps: int = 10) -> md_params:
    p = md_params()
    _ck(LIB.md_autotune(h, int(steps), ctypes.byref(p)), "md_autotune")
    return p


def md_batch_autotune(b, steps: int = 10) -> md_params:
    p = md_params()
    _ck(LIB.md_batch_autotune(b, int(steps), ctypes.byref(p)), "md_batch_autotune")
    return p


def _jobs(jobs):
    arr = (md_job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = md_job(int(j["N"]), float(j["Yp"]), float(j["rho"]), float(j["T"]), int(j["seed"]),
                        float(j.get("xi_dot", 0.0)), int(j.get("steps", 0)))
    return arr


def md_batch_create(jobs, params: md_params | None = None):
    h = _P()
    _ck(LIB.md_batch_create(len(jobs), _jobs(jobs), ctypes.byref(params) if params is not None else None,
                            ctypes.byref(h)), "md_batch_create")
    return h


def md_batch_step(b, n: int) -> None:
    _ck(LIB.md_batch_step(b, int(n)), "md_batch_step")


def md_batch_system(b, i: int):
    h = _P()
    _ck(LIB.md_batch_system(b, int(i), ctypes.byref(h)), "md_batch_system")
    return h


def md_batch_destroy(b) -> None:
    _ck(LIB.md_batch_destroy(b), "md_batch_destroy")


def md_server_create(hbm_budget_bytes: int, params: md_params | None = None):
    h = _P()
    _ck(LIB.md_server_create(int(hbm_budget_bytes), ctypes.byref(params) if params is not None else None,
                             ctypes.byref(h)), "md_server_create")
    return h


def md_server_submit(sv, job: dict) -> int:
    jid = _I64()
    _ck(LIB.md_server_submit(sv, _jobs([job]), ctypes.byref(jid)), "md_server_submit")
    return jid.value


def md_server_poll(sv):
    r = md_result()
    rc = LIB.md_server_poll(sv, ctypes.byref(r))
    if rc == MD_EAGAIN:
        return None
    _ck(rc, "md_server_poll")
    d = {k: getattr(r, k) for k, _ in md_result._fields_ if k not in ("energy", "reserved0")}
    d["energy"] = {k: getattr(r.energy, k) for k, _ in md_energy_t._fields_}
    return d


def md_server_drain(sv, timeout_s: float = 600.0) -> None:
    _ck(LIB.md_server_drain(sv, float(timeout_s)), "md_server_drain")


def md_server_destroy(sv) -> None:
    _ck(LIB.md_server_destroy(sv), "md_server_destroy")


# ---------------------------------------------------------------- wrappers
class System:
    """One MD system (md_create / md_create_ex) with numpy in/out."""

    def __init__(self, N, Yp, rho, T, seed, params: md_params | None = None, handle=None, owner=True):
        self.h = handle if handle is not None else md_create(N, Yp, rho, T, seed, params)
        self.owner = owner
        info = md_get_info(self.h)
        self.N, self.Np = info["N"], info["Np"]

    def close(self):
        if self.h is not None and self.owner:
            md_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n, xi_dot=0.0):
        md_step(self.h, n, xi_dot)

    def step_async(self, n, xi_dot=0.0):
        md_step_async(self.h, n, xi_dot)

    def sync(self):
        md_sync(self.h)

    def forces(self):
        return md_forces(self.h, self.N)

    def energy(self):
        return md_energy(self.h)

    def step_energy(self):
        return md_step_energy(self.h)

    def state(self, out=None, f=False):
        return md_get_state(self.h, self.N, out=out, f=f)

    def set_state(self, x, v, L, **kw):
        md_set_state(self.h, x, v, L, Np=self.Np, **kw)

    def clusters(self, labels=True, out=None):
        return md_clusters(self.h, self.N, self.Np, labels, out=out)

    def clusters_mste(self, labels=True, out=None):
        return md_clusters_mste(self.h, self.N, self.Np, labels, out=out)

    def info(self):
        return md_get_info(self.h)

    @property
    def params(self):
        return md_get_params(self.h)

    @params.setter
    def params(self, p):
        md_set_params(self.h, p)

    def set_stream(self, s):
        md_set_stream(self.h, s)

    def set_timing(self, on=True):
        md_set_timing(self.h, on)

    def kernel_times(self):
        return md_kernel_times(self.h)

    def autotune(self, steps=10):
        return md_autotune(self.h, steps)


class Batch:
    """Independent systems advanced by one graph launch per step."""

    def __init__(self, jobs, params: md_params | None = None):
        self.b = md_batch_create(jobs, params)
        self.systems = [System(0, 0, 0, 0, 0, handle=md_batch_system(self.b, i), owner=False)
                        for i in range(len(jobs))]

    def step(self, n):
        md_batch_step(self.b, n)

    def autotune(self, steps=10):
        return md_batch_autotune(self.b, steps)

    def close(self):
        if self.b is not None:
            for s in self.systems:
                s.h = None
            md_batch_destroy(self.b)
        self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
