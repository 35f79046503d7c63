"""FP64 CPU oracle of the particle <-> dual-grid coupling step (arXiv 1807.11834).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.
The CUDA library never calls it, and it shares no code with the library.

The arithmetic lives in ``cg_oracle.c`` (plain loops, double precision,
compiled with ``-ffp-contract=off``); this module compiles it on first use
and marshals numpy arrays.  Inputs in float32 are widened to float64 exactly
before the call.

Parity pins (all in ``tests/test_oracle_*.py``) tie each function to closed
forms, invariants or brute force; see the docstrings there.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_HDR = os.path.join(_HERE, "cg_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcg_oracle.so")
_LIB_OMP = os.path.join(_BUILD, "libcg_oracle_omp.so")
_lock = threading.Lock()
_libs = {}

NSUMS = 16


def build(force: bool = False, threads: bool = False) -> str:
    """Compile the oracle shared library (gcc, no FMA contraction).  With
    threads the same source is built with -fopenmp: its loops over
    independent particles and cells run on every host core, with results
    bit-identical to the single-thread build."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB_OMP if threads else _LIB
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
               "-ffp-contract=off", "-fno-fast-math"] + (["-fopenmp"] if threads else []) + ["-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


class Grid(C.Structure):
    _fields_ = [("x0", C.c_double * 3), ("L", C.c_double * 3), ("nf", C.c_int32 * 3),
                ("r", C.c_int32), ("law", C.c_int32), ("interp", C.c_int32),
                ("rho_f", C.c_double), ("mu_f", C.c_double), ("rho_p", C.c_double),
                ("eps_switch", C.c_double), ("eps_min", C.c_double), ("g", C.c_double * 3)]


def grid(desc: dict) -> Grid:
    g = Grid()
    g.x0[:] = desc["origin"]
    g.L[:] = desc["extent"]
    g.nf[:] = desc["fine_n"]
    g.r = desc["ratio"]
    g.law = desc["law"]
    g.interp = desc.get("interp", 0)
    g.rho_f, g.mu_f, g.rho_p = desc["rho_f"], desc["mu_f"], desc["rho_p"]
    g.eps_switch, g.eps_min = desc["eps_switch"], desc["eps_min"]
    g.g[:] = desc.get("gravity", (0.0, 0.0, 0.0))
    return g


class BoxGrid(C.Structure):
    _fields_ = [("x0", C.c_double * 3), ("L", C.c_double * 3), ("n", C.c_int32 * 3)]


def box_grid(origin, extent, n) -> BoxGrid:
    g = BoxGrid()
    g.x0[:] = origin
    g.L[:] = extent
    g.n[:] = n
    return g


def _load(threads: bool = False):
    with _lock:
        if threads not in _libs:
            lib = C.CDLL(build(threads=threads))
            P = C.POINTER
            d, i32, i64 = C.c_double, C.c_int32, C.c_int64
            pd, pi = P(d), P(i32)
            pg = P(Grid)
            sig = {
                "or_bin_cell": (i32, [pg, pd, P(C.c_int)]),
                "or_bin": (i64, [pg, i64, pd, pi, pi, pi]),
                "or_deposit_volume": (None, [pg, i64, pd, pi, pi, pd, pd]),
                "or_average": (None, [pg, pd, pd, pd]),
                "or_weights": (None, [pg, pd, pi, pd, P(C.c_int)]),
                "or_gather": (None, [pg, pd, C.c_int, pd, pd]),
                "or_gather_grad": (None, [pg, pd, pd, pd]),
                "or_drag_beta": (d, [pg, d, d, pd, P(C.c_int)]),
                "or_drag": (i64, [pg, i64, pd, pd, pd, pd, pd]),
                "or_deposit_momentum": (None, [pg, i64, pd, pi, pi, pd]),
                "or_implicit": (None, [pg, i64, pd, pd, pd, pd, pi, pi, pd]),
                "or_map_average": (None, [P(BoxGrid), P(BoxGrid), C.c_int, pd, pd]),
                "or_map_project": (None, [P(BoxGrid), P(BoxGrid), C.c_int, pd, pd]),
                "or_particle_state": (None, [pg, i64, pd, pd, pd, pd, pd, pd]),
                "or_mlp_features": (None, [pg, i64, pd, pd, pd, pd, pd, pd, pd, pd, pd]),
                "or_project": (None, [pg, C.c_int, pd, pd]),
                "or_euler": (None, [pg, i64, pd, pd, pd, d]),
                "or_step": (i64, [pg, i64, pd, pd, pd, d, pi, pi, pi, pd, pd, pd, pd, pd, pd, pd, pd]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _libs[threads] = lib
    return _libs[threads]


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _pd(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _pi(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int32))


def dims(desc):
    nf = tuple(desc["fine_n"])
    r = desc["ratio"]
    nb = tuple(v // r for v in nf)
    return nf, nb


def bin_cell(desc, x):
    lib = _load()
    g = grid(desc)
    o = C.c_int(0)
    xx = _f64(x)
    c = lib.or_bin_cell(C.byref(g), _pd(xx), C.byref(o))
    return int(c), bool(o.value)


def bin(desc, pos_d):
    """Returns (cell[n], perm[n], cell_start[nb+1], n_outside)."""
    lib = _load()
    g = grid(desc)
    pos = _f64(pos_d).reshape(-1, 4)
    n = pos.shape[0]
    nf, nb = dims(desc)
    nbulk = nb[0] * nb[1] * nb[2]
    cell = np.zeros(n, np.int32)
    perm = np.zeros(n, np.int32)
    cs = np.zeros(nbulk + 1, np.int32)
    out = lib.or_bin(C.byref(g), n, _pd(pos), _pi(cell), _pi(perm), _pi(cs))
    return cell, perm, cs, int(out)


def deposit_volume(desc, pos_d, cell_start, perm):
    """Returns (eps[nb], phi[nb]) as flat arrays."""
    lib = _load()
    g = grid(desc)
    pos = _f64(pos_d).reshape(-1, 4)
    nf, nb = dims(desc)
    nbulk = nb[0] * nb[1] * nb[2]
    eps = np.zeros(nbulk)
    phi = np.zeros(nbulk)
    cs = np.ascontiguousarray(cell_start, np.int32)
    pm = np.ascontiguousarray(perm, np.int32)
    lib.or_deposit_volume(C.byref(g), pos.shape[0], _pd(pos), _pi(cs), _pi(pm), _pd(eps), _pd(phi))
    return eps, phi


def average(desc, u_fine, want_var=True):
    """Returns (u_bulk[3, nbulk], var[nbulk] or None)."""
    lib = _load()
    g = grid(desc)
    nf, nb = dims(desc)
    nbulk = nb[0] * nb[1] * nb[2]
    u = _f64(u_fine).reshape(3, -1)
    ub = np.zeros((3, nbulk))
    var = np.zeros(nbulk) if want_var else None
    lib.or_average(C.byref(g), _pd(u), _pd(ub), _pd(var))
    return ub, var


def weights(desc, x):
    lib = _load()
    g = grid(desc)
    i0 = np.zeros(3, np.int32)
    t = np.zeros(3)
    cl = (C.c_int * 3)()
    xx = _f64(x)
    lib.or_weights(C.byref(g), _pd(xx), _pi(i0), _pd(t), cl)
    return i0, t, np.array(list(cl), dtype=bool)


def gather(desc, bulk, x):
    lib = _load()
    g = grid(desc)
    b = _f64(bulk)
    ncomp = 1 if b.ndim == 1 else b.shape[0]
    out = np.zeros(ncomp)
    xx = _f64(x)
    lib.or_gather(C.byref(g), _pd(b), ncomp, _pd(xx), _pd(out))
    return out


def gather_grad(desc, bulk, x):
    lib = _load()
    g = grid(desc)
    b = _f64(bulk)
    out = np.zeros(3)
    xx = _f64(x)
    lib.or_gather_grad(C.byref(g), _pd(b), _pd(xx), _pd(out))
    return out


def drag_beta(desc, eps, d, s):
    lib = _load()
    g = grid(desc)
    ss = _f64(s)
    cl = C.c_int(0)
    b = lib.or_drag_beta(C.byref(g), float(eps), float(d), _pd(ss), C.byref(cl))
    return float(b), bool(cl.value)


def drag(desc, pos_d, vel, eps_bulk, u_bulk):
    """Returns (force[3, n], n_clamped)."""
    lib = _load()
    g = grid(desc)
    pos = _f64(pos_d).reshape(-1, 4)
    v = _f64(vel).reshape(-1, 4)
    n = pos.shape[0]
    F = np.zeros((3, n))
    e = _f64(eps_bulk)
    u = _f64(u_bulk)
    ncl = lib.or_drag(C.byref(g), n, _pd(pos), _pd(v), _pd(e), _pd(u), _pd(F))
    return F, int(ncl)


def implicit(desc, pos_d, vel, eps_bulk, u_bulk, cell_start, perm):
    """Semi-implicit exchange coefficients (A[nb], b[3, nb]) with
    A = sum beta_p / V_B and b = sum beta_p u_p / V_B per cell (Eq. UFP's
    F_fpi treated semi-implicitly: F_fpi = -A u_f + b)."""
    lib = _load()
    g = grid(desc)
    pos = _f64(pos_d).reshape(-1, 4)
    v = _f64(vel).reshape(-1, 4)
    n = pos.shape[0]
    nf, nb = dims(desc)
    nbulk = nb[0] * nb[1] * nb[2]
    coef = np.zeros((4, nbulk))
    lib.or_implicit(C.byref(g), n, _pd(pos), _pd(v), _pd(_f64(eps_bulk)), _pd(_f64(u_bulk)),
                    _pi(np.ascontiguousarray(cell_start, np.int32)), _pi(np.ascontiguousarray(perm, np.int32)),
                    _pd(coef))
    return coef[0], coef[1:]


def map_average(bulk, fine, u_fine):
    """Volume-weighted fine -> bulk map between non-nested box grids.
    bulk, fine: (origin, extent, n) triples; u_fine [ncomp][n_f] or [n_f]."""
    lib = _load()
    gb, gf = box_grid(*bulk), box_grid(*fine)
    u = _f64(u_fine)
    one = u.ndim == 1
    u = u.reshape(1 if one else u.shape[0], -1)
    nb = int(np.prod(bulk[2]))
    out = np.zeros((u.shape[0], nb))
    lib.or_map_average(C.byref(gb), C.byref(gf), u.shape[0], _pd(u), _pd(out))
    return out[0] if one else out


def map_project(bulk, fine, s_bulk):
    """Conservative bulk -> fine map between non-nested box grids."""
    lib = _load()
    gb, gf = box_grid(*bulk), box_grid(*fine)
    sb = _f64(s_bulk)
    one = sb.ndim == 1
    sb = sb.reshape(1 if one else sb.shape[0], -1)
    nf = int(np.prod(fine[2]))
    out = np.zeros((sb.shape[0], nf))
    lib.or_map_project(C.byref(gb), C.byref(gf), sb.shape[0], _pd(sb), _pd(out))
    return out[0] if one else out


def particle_state(desc, pos_d, vel, eps_bulk, u_bulk):
    """(eps_p[n], |slip|[n]) as seen by each particle's drag law."""
    lib = _load()
    g = grid(desc)
    pos = _f64(pos_d).reshape(-1, 4)
    v = _f64(vel).reshape(-1, 4)
    n = pos.shape[0]
    e, s = np.zeros(n), np.zeros(n)
    lib.or_particle_state(C.byref(g), n, _pd(pos), _pd(v), _pd(_f64(eps_bulk)), _pd(_f64(u_bulk)), _pd(e), _pd(s))
    return e, s


def mlp_features(desc, pos_d, vel, eps_bulk, u_stale, var_stale, u_fresh):
    """(features[n, 7], target[n], F_stale[3, n]) of the learned closure."""
    lib = _load()
    g = grid(desc)
    pos = _f64(pos_d).reshape(-1, 4)
    v = _f64(vel).reshape(-1, 4)
    n = pos.shape[0]
    feat = np.zeros((n, 7))
    target = np.zeros(n)
    Fs = np.zeros((3, n))
    lib.or_mlp_features(C.byref(g), n, _pd(pos), _pd(v), _pd(_f64(eps_bulk)), _pd(_f64(u_stale)),
                        _pd(_f64(var_stale)), _pd(_f64(u_fresh)), _pd(feat), _pd(target), _pd(Fs))
    return feat, target, Fs


def deposit_momentum(desc, force, cell_start, perm):
    lib = _load()
    g = grid(desc)
    F = _f64(force).reshape(3, -1)
    nf, nb = dims(desc)
    nbulk = nb[0] * nb[1] * nb[2]
    S = np.zeros((3, nbulk))
    cs = np.ascontiguousarray(cell_start, np.int32)
    pm = np.ascontiguousarray(perm, np.int32)
    lib.or_deposit_momentum(C.byref(g), F.shape[1], _pd(F), _pi(cs), _pi(pm), _pd(S))
    return S


def project(desc, bulk):
    lib = _load()
    g = grid(desc)
    b = _f64(bulk)
    ncomp = 1 if b.ndim == 1 else b.shape[0]
    nf, nb = dims(desc)
    nfine = nf[0] * nf[1] * nf[2]
    out = np.zeros((ncomp, nfine))
    lib.or_project(C.byref(g), ncomp, _pd(b), _pd(out))
    return out[0] if b.ndim == 1 else out


def euler(desc, pos_d, vel, force, dt):
    lib = _load()
    g = grid(desc)
    pos = _f64(pos_d).reshape(-1, 4).copy()
    v = _f64(vel).reshape(-1, 4).copy()
    F = _f64(force).reshape(3, -1)
    lib.or_euler(C.byref(g), pos.shape[0], _pd(pos), _pd(v), _pd(F), float(dt))
    return pos, v


def step(desc, pos_d, vel, u_fine, dt=0.0, want_var=True, want_eps_fine=False, threads=False):
    """One whole coupling step; returns a dict of float64 / int32 arrays.
    Particle arrays are copied; with dt > 0 the returned pos_d / vel are
    the advanced state.  threads: run the OpenMP build on every host core
    (bit-identical results)."""
    lib = _load(threads)
    g = grid(desc)
    pos = _f64(pos_d).reshape(-1, 4).copy()
    v = _f64(vel).reshape(-1, 4).copy()
    u = _f64(u_fine).reshape(3, -1)
    n = pos.shape[0]
    nf, nb = dims(desc)
    nbulk = nb[0] * nb[1] * nb[2]
    nfine = nf[0] * nf[1] * nf[2]
    out = dict(
        cell=np.zeros(n, np.int32), perm=np.zeros(n, np.int32),
        cell_start=np.zeros(nbulk + 1, np.int32),
        eps_bulk=np.zeros(nbulk), u_bulk=np.zeros((3, nbulk)),
        var_bulk=np.zeros(nbulk) if want_var else None,
        force=np.zeros((3, n)), S_bulk=np.zeros((3, nbulk)),
        S_fine=np.zeros((3, nfine)),
        eps_fine=np.zeros(nfine) if want_eps_fine else None,
        sums=np.zeros(NSUMS))
    outside = lib.or_step(C.byref(g), n, _pd(pos), _pd(v), _pd(u), float(dt),
                          _pi(out["cell"]), _pi(out["perm"]), _pi(out["cell_start"]),
                          _pd(out["eps_bulk"]), _pd(out["u_bulk"]), _pd(out["var_bulk"]),
                          _pd(out["force"]), _pd(out["S_bulk"]), _pd(out["S_fine"]),
                          _pd(out["eps_fine"]), _pd(out["sums"]))
    out["outside"] = int(outside)
    out["pos_d"] = pos
    out["vel"] = v
    return out
