"""FP64 CPU oracle for the regular-force step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import this package.  The product library never calls it,
and it shares no code with the CUDA path.  The arithmetic lives in
``nb_oracle.c`` (plain C, FP64, ascending-j loops); this module only compiles
it with gcc and marshals numpy arrays through ctypes.

Every function cites the passage of the paper it follows in the C source.
Parity of every function is pinned by tests/test_oracle_pins.py against closed
forms and invariants (two-body Kepler orbit, Newton's third law, jerk as the
time derivative of the acceleration, the Plummer potential energy, energy
conservation, brute-force neighbour sets, finite differences for the adjoint,
partition and Newton's-law invariants of the irregular force, reduction of the
Ahmad-Cohen integrator to the plain Hermite run).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile nb_oracle.c into liboracle.so with gcc (portable flags, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.orc_predict.argtypes = [i64, dbl, P, P, P, P, P, P, P]
        lib.orc_predict.restype = None
        lib.orc_regular_force.argtypes = [i64, P, P, P, i64, P, P, ctypes.c_int, P, P, P, P, P, i32]
        lib.orc_regular_force.restype = ctypes.c_int
        lib.orc_regular_force_vjp.argtypes = [i64, P, P, P, i64, P, P, P, P, P, P, P]
        lib.orc_regular_force_vjp.restype = ctypes.c_int
        lib.orc_energy.argtypes = [i64, P, P, P, P, P]
        lib.orc_energy.restype = None
        lib.orc_hermite_run.argtypes = [i64, P, P, P, dbl, dbl, dbl, dbl, dbl, i64, P]
        lib.orc_hermite_run.restype = ctypes.c_int
        lib.orc_hermite_record.argtypes = [i64, P, P, P, dbl, dbl, dbl, dbl, i64, P, P, P, i64, i64, P]
        lib.orc_hermite_record.restype = ctypes.c_int
        lib.orc_hermite_replay.argtypes = [i64, P, P, P, i64, P, P, P]
        lib.orc_hermite_replay.restype = ctypes.c_int
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def predict(t, x, v, a, jerk, t_last):
    """Hermite predictor of all particles to time t -> (x_p, v_p), each (n,3)."""
    lib = _load()
    x, v, a, jerk = (_c(q, np.float64) for q in (x, v, a, jerk))
    t_last = _c(t_last, np.float64)
    n = x.shape[0]
    xp, vp = np.empty_like(x), np.empty_like(v)
    lib.orc_predict(n, float(t), _p(x), _p(v), _p(a), _p(jerk), _p(t_last), _p(xp), _p(vp))
    return xp, vp


def regular_force(xp, vp, m, idx, rs2, cap: int = 512, lists: bool = True):
    """acc, jerk (n_i,3), pot (n_i), nb_count (n_i), nb_lists (list of int32 arrays, first `cap`)."""
    lib = _load()
    xp, vp, m = _c(xp, np.float64), _c(vp, np.float64), _c(m, np.float64)
    idx = _c(idx, np.int32)
    n, n_i = xp.shape[0], idx.shape[0]
    rs2 = np.atleast_1d(_c(rs2, np.float64))
    scalar = 1 if rs2.shape[0] == 1 and n_i != 1 else 0
    if not scalar and rs2.shape[0] != n_i:
        raise ValueError("rs2 must be a scalar or have one entry per active particle")
    acc = np.empty((n_i, 3)); jerk = np.empty((n_i, 3)); pot = np.empty(n_i)
    cnt = np.empty(n_i, np.int32)
    lst = np.empty((n_i, max(cap, 1)), np.int32) if lists else None
    rc = lib.orc_regular_force(n, _p(xp), _p(vp), _p(m), n_i, _p(idx), _p(rs2), scalar,
                               _p(acc), _p(jerk), _p(pot), _p(cnt), _p(lst), int(cap))
    if rc != 0:
        raise IndexError("active index outside [0, n)")
    out_lists = None
    if lists:
        out_lists = [lst[k, :min(int(cnt[k]), cap)].copy() for k in range(n_i)]
    return acc, jerk, pot, cnt, out_lists


def regular_force_vjp(xp, vp, m, idx, g_acc, g_jerk, g_pot):
    """(g_x, g_v, g_m) of L = Σ g_acc·acc + g_jerk·jerk + g_pot·pot over the active set."""
    lib = _load()
    xp, vp, m = _c(xp, np.float64), _c(vp, np.float64), _c(m, np.float64)
    idx = _c(idx, np.int32)
    g_acc, g_jerk, g_pot = _c(g_acc, np.float64), _c(g_jerk, np.float64), _c(g_pot, np.float64)
    n, n_i = xp.shape[0], idx.shape[0]
    gx = np.empty((n, 3)); gv = np.empty((n, 3)); gm = np.empty(n)
    rc = lib.orc_regular_force_vjp(n, _p(xp), _p(vp), _p(m), n_i, _p(idx), _p(g_acc), _p(g_jerk),
                                   _p(g_pot), _p(gx), _p(gv), _p(gm))
    if rc != 0:
        raise IndexError("active index outside [0, n)")
    return gx, gv, gm


def energy(m, x, v):
    """(K, W) with K = ½Σ m v², W = -Σ_{i<j} m_i m_j / r_ij."""
    lib = _load()
    m, x, v = _c(m, np.float64), _c(x, np.float64), _c(v, np.float64)
    K, W = ctypes.c_double(), ctypes.c_double()
    lib.orc_energy(m.shape[0], _p(m), _p(x), _p(v), ctypes.byref(K), ctypes.byref(W))
    return K.value, W.value


def hermite_run(m, x, v, t_end, eta=0.02, eta_s=0.01, dt_max=0.125, dt_fixed=0.0, max_blocks=0):
    """Block-step Hermite integration to t_end -> (x, v, stats[blocks, particle steps, pairs])."""
    lib = _load()
    m = _c(m, np.float64)
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    stats = np.zeros(4)
    rc = lib.orc_hermite_run(m.shape[0], _p(m), _p(x), _p(v), float(t_end), float(eta), float(eta_s),
                             float(dt_max), float(dt_fixed), int(max_blocks), _p(stats))
    if rc != 0:
        raise RuntimeError("hermite_run stopped at max_blocks")
    return x, v, stats[:3]


def hermite_record(m, x, v, t_end, eta=0.02, eta_s=0.01, dt_max=0.125, max_blocks=0, cap_blocks=1 << 16):
    """Block-step run that records its schedule -> (x, v, [(t_next, active int32 array), ...])."""
    lib = _load()
    m = _c(m, np.float64)
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    n = m.shape[0]
    t_next = np.empty(cap_blocks)
    off = np.empty(cap_blocks + 1, np.int64)
    cap_act = cap_blocks * n if cap_blocks * n < (1 << 26) else (1 << 26)
    act = np.empty(cap_act, np.int32)
    nb = ctypes.c_int64()
    rc = lib.orc_hermite_record(n, _p(m), _p(x), _p(v), float(t_end), float(eta), float(eta_s), float(dt_max),
                                int(max_blocks), _p(t_next), _p(off), _p(act), cap_blocks, cap_act, ctypes.byref(nb))
    if rc not in (0, -2):
        raise RuntimeError(f"hermite_record failed ({rc})")
    sched = [(float(t_next[b]), act[off[b]:off[b + 1]].copy()) for b in range(nb.value)]
    return x, v, sched


def hermite_replay(m, x, v, schedule):
    """Replay a frozen schedule [(t_next, active), ...] from (x, v) at t = 0 -> (x, v)."""
    lib = _load()
    m = _c(m, np.float64)
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    t_next = np.array([s[0] for s in schedule], dtype=np.float64)
    off = np.zeros(len(schedule) + 1, np.int64)
    off[1:] = np.cumsum([len(s[1]) for s in schedule])
    act = np.ascontiguousarray(np.concatenate([np.asarray(s[1], np.int32) for s in schedule]) if schedule
                               else np.zeros(0, np.int32))
    rc = lib.orc_hermite_replay(m.shape[0], _p(m), _p(x), _p(v), len(schedule), _p(t_next), _p(off), _p(act))
    if rc != 0:
        raise RuntimeError(f"hermite_replay failed ({rc})")
    return x, v


def pair_sums(xp, vp, m, idx, jdx):
    """(acc, jerk, pot) of the rows idx summed over the sources jdx only (j != i)."""
    lib = _load()
    if not hasattr(lib, "_ps"):
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.orc_pair_sums.argtypes = [i64, P, P, P, i64, P, i64, P, P, P, P]
        lib.orc_pair_sums.restype = ctypes.c_int
        lib._ps = True
    xp, vp, m = _c(xp, np.float64), _c(vp, np.float64), _c(m, np.float64)
    idx, jdx = _c(idx, np.int32), _c(jdx, np.int32)
    n_i = idx.shape[0]
    acc = np.empty((n_i, 3)); jerk = np.empty((n_i, 3)); pot = np.empty(n_i)
    rc = lib.orc_pair_sums(xp.shape[0], _p(xp), _p(vp), _p(m), n_i, _p(idx), jdx.shape[0], _p(jdx),
                           _p(acc), _p(jerk), _p(pot))
    if rc != 0:
        raise IndexError("index outside [0, n)")
    return acc, jerk, pot


def irregular_force(t, x, v, a, jerk, t_last, m, idx, nb_off, nb_idx):
    """Irregular force: (acc, jerk (n_i,3), pot (n_i)) of the rows idx summed over their
    CSR neighbour lists nb_idx[nb_off[k]:nb_off[k+1]], with i and each listed neighbour
    predicted from its Hermite state to time t."""
    lib = _load()
    if not hasattr(lib, "_irr"):
        P, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        lib.orc_irregular_force.argtypes = [i64, P, P, P, P, P, P, dbl, i64, P, P, P, P, P, P]
        lib.orc_irregular_force.restype = ctypes.c_int
        lib._irr = True
    x, v, a, jerk = (_c(q, np.float64) for q in (x, v, a, jerk))
    t_last, m = _c(t_last, np.float64), _c(m, np.float64)
    idx, nb_off, nb_idx = _c(idx, np.int32), _c(nb_off, np.int64), _c(nb_idx, np.int32)
    n_i = idx.shape[0]
    if nb_off.shape[0] != n_i + 1:
        raise ValueError("nb_off needs n_i + 1 entries")
    acc = np.empty((n_i, 3)); jk = np.empty((n_i, 3)); pot = np.empty(n_i)
    rc = lib.orc_irregular_force(x.shape[0], _p(x), _p(v), _p(a), _p(jerk), _p(t_last), _p(m), float(t), n_i,
                                 _p(idx), _p(nb_off), _p(nb_idx if nb_idx.size else np.zeros(1, np.int32)),
                                 _p(acc), _p(jk), _p(pot))
    if rc != 0:
        raise IndexError("index outside [0, n) or decreasing offsets")
    return acc, jk, pot


def ac_run(m, x, v, rs2, t_end, eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125, nb_opt=0,
           cap=256, max_blocks=0):
    """Ahmad-Cohen Hermite block-step run (see orc_ac_run).  Returns (x, v, rs2, info) with
    info = dict(t, dt, DT, T, nb_count, nb_lists, blocks, irregular_steps, regular_steps,
    neighbour_pairs, all_pairs, rc, acc, jerk, xp, vp): acc and jerk are the total force and its
    derivative each particle holds after its last step, xp and vp the predicted state of the
    last block step (the state those were evaluated on when the end time synchronises all)."""
    lib = _load()
    if not hasattr(lib, "_ac"):
        P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.orc_ac_run.argtypes = [i64, P, P, P, P, dbl, dbl, dbl, dbl, dbl, i32, i32, i64, P, P, P, P, P, P, P,
                                   P, P, P, P]
        lib.orc_ac_run.restype = ctypes.c_int
        lib._ac = True
    m = _c(m, np.float64)
    x, v = _c(x, np.float64).copy(), _c(v, np.float64).copy()
    n = x.shape[0]
    rs2 = np.ascontiguousarray(np.broadcast_to(np.asarray(rs2, np.float64), (n,))).copy()
    stats = np.zeros(6)
    t, dt, DT, T = (np.zeros(n) for _ in range(4))
    nbc = np.zeros(n, np.int32)
    nbl = np.zeros((n, cap), np.int32)
    acc, jerk, xp, vp = (np.zeros((n, 3)) for _ in range(4))
    rc = lib.orc_ac_run(n, _p(m), _p(x), _p(v), _p(rs2), float(t_end), float(eta_irr), float(eta_reg), float(eta_s),
                        float(dt_max), int(nb_opt), int(cap), int(max_blocks), _p(stats), _p(t), _p(dt), _p(DT),
                        _p(T), _p(nbc), _p(nbl), _p(acc), _p(jerk), _p(xp), _p(vp))
    info = dict(t=t, dt=dt, DT=DT, T=T, nb_count=nbc, nb_lists=[nbl[i, :nbc[i]].copy() for i in range(n)],
                blocks=int(stats[0]), irregular_steps=int(stats[1]), regular_steps=int(stats[2]),
                neighbour_pairs=stats[3], all_pairs=stats[4], rc=rc, acc=acc, jerk=jerk, xp=xp, vp=vp)
    return x, v, rs2, info


def loss_fd(xp, vp, m, idx, g_acc, g_jerk, g_pot, which: str, p: int, c: int = 0, h: float = 1e-6):
    """Central difference (Richardson, O(h^4)) of L = Σ g·(acc, jerk, pot) w.r.t. one
    coordinate of particle p (which = 'x', 'v' or 'm'), in O(N) by re-evaluating only
    the sums that involve p: row p over all sources and column p of every other row."""
    idx = np.asarray(idx, np.int32)
    rows = np.nonzero(idx == p)[0]
    others = np.nonzero(idx != p)[0]
    n = xp.shape[0]
    all_j = np.arange(n, dtype=np.int32)

    def L_p(X, V, M):
        tot = 0.0
        if rows.size:
            a, j, pt = pair_sums(X, V, M, idx[rows], all_j)
            tot += (g_acc[rows] * a).sum() + (g_jerk[rows] * j).sum() + (g_pot[rows] * pt).sum()
        a, j, pt = pair_sums(X, V, M, idx[others], np.array([p], np.int32))
        tot += (g_acc[others] * a).sum() + (g_jerk[others] * j).sum() + (g_pot[others] * pt).sum()
        return tot

    def shifted(d):
        X, V, M = xp.copy(), vp.copy(), m.copy()
        if which == "x":
            X[p, c] += d
        elif which == "v":
            V[p, c] += d
        else:
            M[p] += d
        return L_p(X, V, M)
    d1 = (shifted(h) - shifted(-h)) / (2 * h)
    d2 = (shifted(h / 2) - shifted(-h / 2)) / h
    return (4 * d2 - d1) / 3
