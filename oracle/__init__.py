"""FP64 CPU oracle for the SDPD hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``sdpd_oracle.c`` (plain C,
brute-force O(N^2) pairs, sequential colour-ordered sweep) through ctypes and
shares no code with the CUDA library.

Parity unpinned: nothing.  Every function is pinned by a ``-m "not gpu"``
test in ``tests/test_oracle_pins.py`` or ``tests/test_oracle_adjoint.py``
(the gradients) against a closed form, an invariant, a library routine
(numpy's Philox), central differences or brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdpd_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liborc.so")

KERNEL_CUBIC, KERNEL_LUCY = 0, 1
SCHEME_SSA, SCHEME_AMS, SCHEME_EMS, SCHEME_NONE = 0, 1, 2, 3
ACCEPT, REJECT_BOUND, REJECT_METROPOLIS = 0, 1, 2
OK, ERR_NEGATIVE_ENERGY, ERR_NOT_ADJACENT = 0, 4, 9


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_lib/liborc.so (gcc, FP contraction off)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("N", C.c_int64),
        ("L", C.c_double * 3),
        ("m", C.c_double),
        ("h", C.c_double),
        ("kB", C.c_double),
        ("eta", C.c_double),
        ("zeta", C.c_double),
        ("C_K", C.c_double),
        ("c_rho", C.c_double),
        ("kernel", C.c_int),
        ("scheme", C.c_int),
        ("n_c", C.c_int * 3),
        ("cs", C.c_double * 3),
    ]


class FDStats(C.Structure):
    _fields_ = [
        ("n_pairs", C.c_int64),
        ("n_accept", C.c_int64),
        ("n_reject_bound", C.c_int64),
        ("n_reject_metropolis", C.c_int64),
        ("n_negative", C.c_int64),
    ]


PAIR_REC_DTYPE = np.dtype([
    ("id_i", np.int64), ("id_j", np.int64), ("colour", np.int32), ("owner", np.int32),
    ("decision", np.int32), ("pad", np.int32), ("margin", np.float64),
])

_lib = None
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_u64p = C.POINTER(C.c_uint64)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER(Params)
        sig = {
            "orc_W": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "orc_F": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "orc_S": (C.c_double, [P, C.c_double, C.c_double]),
            "orc_T": (C.c_double, [P, C.c_double]),
            "orc_P": (C.c_double, [P, C.c_double, C.c_double]),
            "orc_C": (C.c_double, [P, C.c_double]),
            "orc_E_of_S": (C.c_double, [P, C.c_double, C.c_double]),
            "orc_min_image": (C.c_double, [C.c_double, C.c_double]),
            "orc_wrap": (C.c_double, [C.c_double, C.c_double]),
            "orc_cell_1d": (C.c_int, [P, C.c_int, C.c_double]),
            "orc_cells": (None, [P, _dp, _i32p]),
            "orc_morton3": (C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint32]),
            "orc_sorted_order": (C.c_int, [P, _dp, _i64p]),
            "orc_density": (None, [P, _dp, _dp]),
            "orc_neighbour_counts": (None, [P, _dp, _i32p]),
            "orc_forces": (None, [P, _dp, _dp, _dp, _dp]),
            "orc_density_at": (None, [P, _dp, _i64p, C.c_int64, _dp]),
            "orc_neighbour_count_at": (None, [P, _dp, _i64p, C.c_int64, _i32p]),
            "orc_forces_at": (None, [P, _dp, _dp, _i64p, C.c_int64, _dp]),
            "orc_hamiltonian": (C.c_double, [P, _dp, _dp, _dp]),
            "orc_verlet": (None, [P, _dp, _dp, _dp, C.c_double]),
            "orc_philox4x64_10": (None, [_u64p, _u64p, _u64p]),
            "orc_pair_randoms": (None, [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, _dp, _dp]),
            "orc_fd_pair": (C.c_int, [P, _dp, C.c_double, C.c_double, _dp, _dp, _dp, _dp,
                                      C.c_double, _dp, C.c_double, _dp, C.POINTER(C.c_int)]),
            "orc_pair_owner": (C.c_int, [P, _i32p, _i32p, C.c_int64, _i32p]),
            "orc_owner_bits": (C.c_uint, [C.c_int64]),
            "orc_fd_sweep": (C.c_int, [P, _dp, _dp, _dp, C.c_double, C.c_uint64, C.c_uint64,
                                       C.POINTER(FDStats), C.c_void_p, C.c_int64]),
            "orc_run": (C.c_int, [P, _dp, _dp, _dp, C.c_double, C.c_int64, C.c_int, C.c_int,
                                  C.c_uint64, _u64p, C.POINTER(FDStats)]),
            "orc_observables": (None, [P, _dp, _dp, _dp]),
            "orc_dF_dr": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "orc_dW_dh": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "orc_dF_dh": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "orc_virial_pressure": (C.c_double, [P, _dp, _dp, _dp]),
            "orc_density_vjp": (None, [P, _dp, _dp, _dp, _dp]),
            "orc_virial_vjp": (C.c_double, [P, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
            "orc_vv_vjp": (None, [P, _dp, _dp, _dp, C.c_double, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
            "orc_frozen_run": (None, [P, _dp, _dp, _dp, C.c_double, C.c_int, _dp, _dp]),
            "orc_frozen_vjp": (None, [P, _dp, _dp, _dp, C.c_double, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                      _dp, _dp]),
            "orc_sizeof_params": (C.c_int, []),
            "orc_sizeof_pair_rec": (C.c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        assert L.orc_sizeof_params() == C.sizeof(Params)
        assert L.orc_sizeof_pair_rec() == PAIR_REC_DTYPE.itemsize
        _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Config:
    """Physical and numerical parameters of one run (reduced units, kB = 1)."""

    N: int
    L: tuple
    m: float = 1.0
    h: float = 2.5
    K: float = 100.0
    kB: float = 1.0
    eta: float = 1.0
    zeta: float = 0.0
    c_rho: float | None = None
    kernel: int = KERNEL_LUCY
    scheme: int = SCHEME_EMS
    n_c: tuple | None = None  # cells per axis; None: the largest even n with L/n >= h

    def params(self) -> Params:
        P = Params()
        P.N = self.N
        Ls = self.L if isinstance(self.L, (tuple, list)) else (self.L,) * 3
        for k in range(3):
            P.L[k] = float(Ls[k])
            if self.n_c is not None:
                n = int(self.n_c[k])
                if n < 4 or n % 2 or Ls[k] / n < self.h:
                    raise ValueError("cell grid: need an even n_c >= 4 with L/n_c >= h")
            else:
                n = int(np.floor(Ls[k] / self.h))
                n -= n % 2
            if n < 4:
                raise ValueError("box too small: need an even n_c >= 4 with L/n_c >= h")
            P.n_c[k] = n
            P.cs[k] = float(Ls[k]) / n
        P.m, P.h, P.kB = self.m, self.h, self.kB
        P.eta, P.zeta = self.eta, self.zeta
        P.C_K = heat_capacity(self.K, self.kB)
        P.c_rho = 0.5 * (self.K - 1.0) if self.c_rho is None else self.c_rho
        P.kernel, P.scheme = self.kernel, self.scheme
        return P


def heat_capacity(K: float, kB: float = 1.0) -> float:
    """C_K = 3/2 (K - 1) kB of the ideal gas (Section 4)."""
    return 1.5 * (K - 1.0) * kB


# --- thin wrappers ---------------------------------------------------------

def W(kernel, r, h):
    return lib().orc_W(kernel, r, h)


def F(kernel, r, h):
    return lib().orc_F(kernel, r, h)


def density(P: Params, q) -> np.ndarray:
    q = _f64(q)
    rho = np.empty(P.N)
    lib().orc_density(C.byref(P), _d(q), _d(rho))
    return rho


def neighbour_counts(P: Params, q) -> np.ndarray:
    q = _f64(q)
    out = np.empty(P.N, dtype=np.int32)
    lib().orc_neighbour_counts(C.byref(P), _d(q), out.ctypes.data_as(_i32p))
    return out


def forces(P: Params, q, rho, eps) -> np.ndarray:
    q, rho, eps = _f64(q), _f64(rho), _f64(eps)
    f = np.empty((P.N, 3))
    lib().orc_forces(C.byref(P), _d(q), _d(rho), _d(eps), _d(f))
    return f


def density_at(P: Params, q, idx) -> np.ndarray:
    q = _f64(q)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(len(idx))
    lib().orc_density_at(C.byref(P), _d(q), idx.ctypes.data_as(_i64p), len(idx), _d(out))
    return out


def neighbour_count_at(P: Params, q, idx) -> np.ndarray:
    q = _f64(q)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(len(idx), dtype=np.int32)
    lib().orc_neighbour_count_at(C.byref(P), _d(q), idx.ctypes.data_as(_i64p), len(idx),
                                 out.ctypes.data_as(_i32p))
    return out


def forces_at(P: Params, q, eps, idx) -> np.ndarray:
    q, eps = _f64(q), _f64(eps)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty((len(idx), 3))
    lib().orc_forces_at(C.byref(P), _d(q), _d(eps), idx.ctypes.data_as(_i64p), len(idx), _d(out))
    return out


def cells(P: Params, q) -> np.ndarray:
    q = _f64(q)
    out = np.empty((P.N, 3), dtype=np.int32)
    lib().orc_cells(C.byref(P), _d(q), out.ctypes.data_as(_i32p))
    return out


def sorted_order(P: Params, q) -> np.ndarray:
    q = _f64(q)
    out = np.empty(P.N, dtype=np.int64)
    lib().orc_sorted_order(C.byref(P), _d(q), out.ctypes.data_as(_i64p))
    return out


def morton3(x, y, z) -> int:
    return int(lib().orc_morton3(x, y, z))


def hamiltonian(P: Params, q, p, S) -> float:
    q, p, S = _f64(q), _f64(p), _f64(S)
    return lib().orc_hamiltonian(C.byref(P), _d(q), _d(p), _d(S))


def entropy(P: Params, eps, rho) -> np.ndarray:
    return np.array([lib().orc_S(C.byref(P), e, r) for e, r in zip(np.ravel(eps), np.ravel(rho))])


def verlet(P: Params, q, p, eps, dt):
    q, p, eps = _f64(q).copy(), _f64(p).copy(), _f64(eps).copy()
    lib().orc_verlet(C.byref(P), _d(q), _d(p), _d(eps), dt)
    return q, p, eps


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    lib().orc_philox4x64_10(c.ctypes.data_as(_u64p), k.ctypes.data_as(_u64p),
                            out.ctypes.data_as(_u64p))
    return out


def pair_randoms(seed, fd_step, i, j):
    G = np.empty(3)
    U = C.c_double()
    lib().orc_pair_randoms(seed, fd_step, i, j, _d(G), C.byref(U))
    return G, U.value


def fd_pair(P: Params, r, rho_i, rho_j, p_i, p_j, eps_i, eps_j, dt, G, U):
    """One pair update; returns (decision, margin, negative, p_i, p_j, eps_i, eps_j)."""
    r, G = _f64(r), _f64(G)
    pi, pj = _f64(p_i).copy(), _f64(p_j).copy()
    ei, ej = C.c_double(eps_i), C.c_double(eps_j)
    margin = C.c_double()
    neg = C.c_int(0)
    d = lib().orc_fd_pair(C.byref(P), _d(r), rho_i, rho_j, _d(pi), _d(pj), C.byref(ei),
                          C.byref(ej), dt, _d(G), U, C.byref(margin), C.byref(neg))
    return d, margin.value, neg.value, pi, pj, ei.value, ej.value


def owner_bits(pid) -> int:
    """The three bits of a particle id that choose the owner block along axes
    where a pair's two cells coincide (bit k for axis k)."""
    return int(lib().orc_owner_bits(int(pid)))


def pair_owner(P: Params, ca, cb, id_lo=0):
    """Owner cell of a pair whose lower-id particle (id_lo) sits in cell ca
    and whose other particle sits in cell cb."""
    a = np.ascontiguousarray(ca, dtype=np.int32)
    b = np.ascontiguousarray(cb, dtype=np.int32)
    o = np.empty(3, dtype=np.int32)
    s = lib().orc_pair_owner(C.byref(P), a.ctypes.data_as(_i32p), b.ctypes.data_as(_i32p), int(id_lo),
                             o.ctypes.data_as(_i32p))
    return s, o


def fd_sweep(P: Params, q, p, eps, dt, seed, fd_step, records: bool = False):
    """One FD sweep.  Returns (status, p, eps, stats, records-or-None)."""
    q = _f64(q)
    p, eps = _f64(p).copy(), _f64(eps).copy()
    st = FDStats()
    recs = None
    ptr, cap = None, 0
    if records:
        cap = int(P.N) * 200
        recs = np.zeros(cap, dtype=PAIR_REC_DTYPE)
        ptr = recs.ctypes.data
    s = lib().orc_fd_sweep(C.byref(P), _d(q), _d(p), _d(eps), dt, seed, fd_step, C.byref(st),
                           ptr, cap)
    if records:
        recs = recs[: min(st.n_pairs, cap)].copy()
    return s, p, eps, st, recs


def run(P: Params, q, p, eps, dt, nsteps, seed, theta=1, fd_only=False, fd_step=0):
    """nsteps steps.  Returns (status, q, p, eps, stats, next_fd_step)."""
    q, p, eps = _f64(q).copy(), _f64(p).copy(), _f64(eps).copy()
    st = FDStats()
    ctr = C.c_uint64(fd_step)
    s = lib().orc_run(C.byref(P), _d(q), _d(p), _d(eps), dt, nsteps, theta, int(fd_only), seed,
                      C.byref(ctr), C.byref(st))
    return s, q, p, eps, st, ctr.value


def observables(P: Params, p, eps) -> dict:
    p, eps = _f64(p), _f64(eps)
    out = np.empty(8)
    lib().orc_observables(C.byref(P), _d(p), _d(eps), _d(out))
    return {"E": out[0], "E_int": out[1], "E_kin": out[2], "P": out[3:6].copy(),
            "T_kin": out[6], "T_int": out[7]}


def dF_dr(kernel, r, h):
    return lib().orc_dF_dr(kernel, r, h)


def dW_dh(kernel, r, h):
    return lib().orc_dW_dh(kernel, r, h)


def dF_dh(kernel, r, h):
    return lib().orc_dF_dh(kernel, r, h)


def virial_pressure(P: Params, q, p, eps) -> float:
    """Virial pressure (1/3V)[sum |p|^2/m + sum_{i<j} r_ij . F_ij] of a state."""
    q, p, eps = _f64(q), _f64(p), _f64(eps)
    return lib().orc_virial_pressure(C.byref(P), _d(q), _d(p), _d(eps))


def virial_vjp(P: Params, q, p, eps):
    """(P_virial, dP/dq, dP/dp, dP/deps, dP/d(h, c_rho, C_K)) at fixed energies."""
    q, p, eps = _f64(q), _f64(p), _f64(eps)
    gq = np.zeros((P.N, 3))
    gp = np.zeros((P.N, 3))
    ge = np.zeros(P.N)
    gt = np.zeros(3)
    val = lib().orc_virial_vjp(C.byref(P), _d(q), _d(p), _d(eps), _d(gq), _d(gp), _d(ge), _d(gt))
    return val, gq, gp, ge, gt


def vv_trajectory(P: Params, q0, p0, eps0, dt, nsteps):
    """Final (q, p, eps) after nsteps Velocity Verlet steps (no sweep)."""
    s = P.scheme
    P.scheme = SCHEME_NONE
    try:
        _, q, p, e, _, _ = run(P, q0, p0, eps0, dt, nsteps, seed=0)
    finally:
        P.scheme = s
    return q, p, e


def vv_vjp(P: Params, q0, p0, eps0, dt, nsteps, gqn, gpn, gepsn):
    """Cotangents of (q0, p0, eps0, (h, c_rho, C_K)) of nsteps Velocity
    Verlet steps at fixed entropies, given those of the final state."""
    q0, p0, eps0 = _f64(q0), _f64(p0), _f64(eps0)
    gqn, gpn, gepsn = _f64(gqn), _f64(gpn), _f64(gepsn)
    gq = np.empty((P.N, 3))
    gp = np.empty((P.N, 3))
    ge = np.empty(P.N)
    gt = np.empty(3)
    lib().orc_vv_vjp(C.byref(P), _d(q0), _d(p0), _d(eps0), dt, nsteps, _d(gqn), _d(gpn), _d(gepsn), _d(gq),
                     _d(gp), _d(ge), _d(gt))
    return gq, gp, ge, gt


def vv_virial_grad(P: Params, q0, p0, eps0, dt, nsteps):
    """Virial pressure after nsteps Velocity Verlet steps and its gradient
    (dL/dq0, dL/dp0, dL/deps0, dL/d(h, c_rho, C_K))."""
    qn, pn, en = vv_trajectory(P, q0, p0, eps0, dt, nsteps)
    val, gq, gp, ge, gt = virial_vjp(P, qn, pn, en)
    gq0, gp0, ge0, gt0 = vv_vjp(P, q0, p0, eps0, dt, nsteps, gq, gp, ge)
    return val, gq0, gp0, ge0, gt0 + gt


def _incr(a, shape):
    return None if a is None else np.ascontiguousarray(np.broadcast_to(_f64(a), shape))


def frozen_run(P: Params, q0, p0, eps0, dt, nsteps, dp=None, deps=None):
    """Final (q, p, eps) of nsteps steps x <- VV(x) + increment_k, the
    increments dp [nsteps][N][3] and deps [nsteps][N] held fixed (None: 0)."""
    q, p, e = _f64(q0).copy(), _f64(p0).copy(), _f64(eps0).copy()
    dp = _incr(dp, (nsteps, P.N, 3))
    deps = _incr(deps, (nsteps, P.N))
    lib().orc_frozen_run(C.byref(P), _d(q), _d(p), _d(e), dt, nsteps, _d(dp) if dp is not None else None,
                         _d(deps) if deps is not None else None)
    return q, p, e


def frozen_vjp(P: Params, q0, p0, eps0, dt, nsteps, dp, deps, gqn, gpn, gepsn):
    """Cotangents of (q0, p0, eps0, (h, c_rho, C_K)) of frozen_run, given
    those of its final state."""
    q0, p0, eps0 = _f64(q0), _f64(p0), _f64(eps0)
    gqn, gpn, gepsn = _f64(gqn), _f64(gpn), _f64(gepsn)
    dp = _incr(dp, (nsteps, P.N, 3))
    deps = _incr(deps, (nsteps, P.N))
    gq = np.empty((P.N, 3))
    gp = np.empty((P.N, 3))
    ge = np.empty(P.N)
    gt = np.empty(3)
    lib().orc_frozen_vjp(C.byref(P), _d(q0), _d(p0), _d(eps0), dt, nsteps,
                         _d(dp) if dp is not None else None, _d(deps) if deps is not None else None,
                         _d(gqn), _d(gpn), _d(gepsn), _d(gq), _d(gp), _d(ge), _d(gt))
    return gq, gp, ge, gt


def sweep_increments(P: Params, q0, p0, eps0, dt, nsteps, seed):
    """Increments (dp, deps) of the sweeps of an nsteps full run (Velocity
    Verlet then one sweep per step, sweep counter from 0), and the final
    state of the frozen run that reproduces it."""
    q, p, e = _f64(q0).copy(), _f64(p0).copy(), _f64(eps0).copy()
    dps, des = [], []
    for k in range(nsteps):
        q, p, e = frozen_run(P, q, p, e, dt, 1)
        st, p2, e2, _, _ = fd_sweep(P, q, p, e, dt, seed, k)
        dps.append(p2 - p)
        des.append(e2 - e)
        p, e = p + dps[-1], e + des[-1]
    return np.array(dps), np.array(des), (q, p, e)
