"""FP64 CPU oracle for the nucleon MD hot path (arXiv:1412.8502).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The product library (``paper_1412_8502_b300``) never imports, links or falls
back to it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64, brute force over all
pairs, OpenMP over targets); this module only compiles it with gcc and
marshals numpy arrays through ctypes.  Each wrapper names the passage of the
paper its C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_HDR = _HERE / "oracle.h"
_LIB = _HERE / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile ``liboracle.so`` (gcc -O2 -fopenmp -ffp-contract=off)."""
    newest = max(_SRC.stat().st_mtime, _HDR.stat().st_mtime)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < newest:
        tmp = _LIB.with_suffix(".so.tmp%d" % os.getpid())
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-std=c11", str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` (Table I and Sec. II.A constants)."""
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
                ("Lambda", ctypes.c_double), ("lambda_s", ctypes.c_double),
                ("alpha", ctypes.c_double), ("M", ctypes.c_double),
                ("r_nuc", ctypes.c_double), ("r_C", ctypes.c_double),
                ("coulomb", ctypes.c_int)]


class RunParams(ctypes.Structure):
    """Mirror of ``orc_run_params`` (integrator, Eq. 3 expansion, thermostat)."""
    _fields_ = [("dt", ctypes.c_double), ("xi_dot", ctypes.c_double),
                ("L_base", ctypes.c_double), ("t_base", ctypes.c_double),
                ("T", ctypes.c_double), ("thermostat_every", ctypes.c_int64), ("affine", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_I8 = ctypes.POINTER(ctypes.c_int8)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_P = ctypes.POINTER(Params)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        L = _lib
        L.orc_default_params.argtypes = [_P]
        L.orc_pair.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _D, _D, _D]
        L.orc_forces.argtypes = [ctypes.c_int64, _D, _I8, ctypes.c_double, _P,
                                 ctypes.c_int64, ctypes.c_int64, _D, _D]
        L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_init.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_uint64, _P, _D, _D, _I8]
        L.orc_init.restype = ctypes.c_double
        L.orc_relax.argtypes = [ctypes.c_int64, _D, _I8, ctypes.c_double, _P,
                                ctypes.c_int64, ctypes.c_double, ctypes.c_double]
        L.orc_wrap.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_wrap.restype = ctypes.c_double
        L.orc_run.argtypes = [ctypes.c_int64, _D, _D, _D, _I8, _P,
                              ctypes.POINTER(RunParams), ctypes.c_int64, _D, _I64, _D]
        L.orc_lambda_tf.argtypes = [ctypes.c_double]
        L.orc_lambda_tf.restype = ctypes.c_double
        L.orc_kinetic.argtypes = [ctypes.c_int64, _D, ctypes.c_double]
        L.orc_kinetic.restype = ctypes.c_double
        L.orc_clusters.argtypes = [ctypes.c_int64, _D, _I8, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, _I32, _I64, _I64, _D]
        L.orc_mste.argtypes = [ctypes.c_int64, _D, _D, _I8, ctypes.c_double, _P, _I32, _I64, _I64, _D]
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _as(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def params(r_C: float, coulomb: bool = True, **over) -> Params:
    """Table I / Sec. II.A defaults with the Coulomb cutoff r_C set."""
    p = Params()
    lib().orc_default_params(ctypes.byref(p))
    p.r_C = float(r_C)
    p.coulomb = 1 if coulomb else 0
    for k, v in over.items():
        setattr(p, k, v)
    return p


def pair(ti: int, tj: int, r2: float, p: Params):
    """Eq. (1): returns (V_nuc, V_coul, g) with F_i = g (x_i - x_j)."""
    vn, vc, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_pair(ti, tj, r2, ctypes.byref(p), ctypes.byref(vn), ctypes.byref(vc), ctypes.byref(g))
    return vn.value, vc.value, g.value


def forces(x, typ, L: float, p: Params, i0: int = 0, i1: int | None = None):
    """Brute-force forces over nearest images (Sec. II.A, Eq. 1).

    Returns (F [N,3], (PE_nuc, PE_coul, W)) summed over targets [i0, i1).
    Rows of F outside [i0, i1) are zero."""
    x = _as(x, np.float64).reshape(-1, 3)
    typ = _as(typ, np.int8)
    N = x.shape[0]
    i1 = N if i1 is None else i1
    F = np.zeros((N, 3), dtype=np.float64)
    e = np.zeros(3, dtype=np.float64)
    lib().orc_forces(N, _dp(x), typ.ctypes.data_as(_I8), float(L), ctypes.byref(p),
                     int(i0), int(i1), _dp(F), _dp(e))
    return F, tuple(e)


def splitmix64(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64(seed, k))


def init(N: int, Yp: float, rho: float, T: float, seed: int, p: Params):
    """Seeded random start (reading of Sec. III.B): returns (x, v, type, L)."""
    x = np.zeros((N, 3)); v = np.zeros((N, 3)); t = np.zeros(N, dtype=np.int8)
    L = lib().orc_init(N, Yp, rho, T, seed, ctypes.byref(p), _dp(x), _dp(v), t.ctypes.data_as(_I8))
    return x, v, t, L


def relax(x, typ, L, p: Params, iters: int, gamma: float = 0.002, dmax: float = 0.1):
    """Steepest descent x += gamma F (|dx| <= dmax), wrapped; returns new x."""
    x = _as(x, np.float64).reshape(-1, 3).copy()
    typ = _as(typ, np.int8)
    lib().orc_relax(x.shape[0], _dp(x), typ.ctypes.data_as(_I8), float(L), ctypes.byref(p),
                    int(iters), float(gamma), float(dmax))
    return x


def wrap(x: float, L: float) -> float:
    return lib().orc_wrap(x, L)


def lambda_tf(n_e: float) -> float:
    """Eq. (2): Thomas-Fermi screening length (fm) at electron density n_e."""
    return lib().orc_lambda_tf(float(n_e))


def kinetic(v, M: float = 939.0) -> float:
    v = _as(v, np.float64).reshape(-1, 3)
    return lib().orc_kinetic(v.shape[0], _dp(v), M)


def run(x, v, typ, L, p: Params, nsteps: int, dt: float = 2.0, xi_dot: float = 0.0,
        T: float = 0.0, thermostat_every: int = 0, t: float = 0.0, step: int = 0,
        L_base: float | None = None, t_base: float = 0.0, F=None, affine: bool = False):
    """Velocity Verlet + Eq. (3) box growth + rescale (Sec. II.A).

    Returns dict(x, v, F, t, step, L).  When F is None it is computed at the
    entry state first."""
    x = _as(x, np.float64).reshape(-1, 3).copy()
    v = _as(v, np.float64).reshape(-1, 3).copy()
    typ = _as(typ, np.int8)
    N = x.shape[0]
    if F is None:
        F, _ = forces(x, typ, L, p)
    F = _as(F, np.float64).reshape(-1, 3).copy()
    rp = RunParams(dt, xi_dot, L if L_base is None else L_base, t_base, T, thermostat_every, 1 if affine else 0)
    tt = ctypes.c_double(t); ss = ctypes.c_int64(step); LL = ctypes.c_double(L)
    lib().orc_run(N, _dp(x), _dp(v), _dp(F), typ.ctypes.data_as(_I8), ctypes.byref(p),
                  ctypes.byref(rp), int(nsteps), ctypes.byref(tt), ctypes.byref(ss), ctypes.byref(LL))
    return dict(x=x, v=v, F=F, t=tt.value, step=ss.value, L=LL.value)


def clusters(x, typ, L: float, r_pp: float = 4.5, r_np: float = 3.0):
    """Distance-linkage clusters of Sec. II.C.

    Returns (labels [N] int32, hist_A [N+1], hist_Z [Np+1], stats[5])."""
    x = _as(x, np.float64).reshape(-1, 3)
    typ = _as(typ, np.int8)
    N = x.shape[0]
    Np = int((typ == 1).sum())
    lab = np.zeros(N, dtype=np.int32)
    hA = np.zeros(N + 1, dtype=np.int64)
    hZ = np.zeros(Np + 1, dtype=np.int64)
    st = np.zeros(5)
    lib().orc_clusters(N, _dp(x), typ.ctypes.data_as(_I8), float(L), float(r_pp), float(r_np),
                       lab.ctypes.data_as(_I32), hA.ctypes.data_as(_I64),
                       hZ.ctypes.data_as(_I64), _dp(st))
    return lab, hA, hZ, st


def mste(x, v, typ, L: float, p: Params):
    """MSTE clusters (energy criterion; reading of Sec. II.C, which names the
    method): returns (labels [N] int32, hist_A [N+1], hist_Z [Np+1], stats[5])."""
    x = _as(x, np.float64).reshape(-1, 3)
    v = _as(v, np.float64).reshape(-1, 3)
    typ = _as(typ, np.int8)
    N = x.shape[0]
    Np = int((typ == 1).sum())
    lab = np.zeros(N, dtype=np.int32)
    hA = np.zeros(N + 1, dtype=np.int64)
    hZ = np.zeros(Np + 1, dtype=np.int64)
    st = np.zeros(5)
    lib().orc_mste(N, _dp(x), _dp(v), typ.ctypes.data_as(_I8), float(L), ctypes.byref(p),
                   lab.ctypes.data_as(_I32), hA.ctypes.data_as(_I64), hZ.ctypes.data_as(_I64), _dp(st))
    return lab, hA, hZ, st
