"""ctypes binding of the SDPD C ABI (include/sdpd.h).

Argument marshalling only: every step of the path runs in the CUDA library.
PyTorch provides the device workspace and the stream.  There is no CPU
fallback: if the CUDA library cannot be loaded, importing this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERR_INVALID_ARG, ERR_BOX_TOO_SMALL, ERR_NONPOSITIVE_ENERGY, ERR_NEGATIVE_ENERGY = 1, 2, 3, 4
ERR_NAN, ERR_CUDA, ERR_TIMEOUT, ERR_NO_WORKSPACE, ERR_CAPACITY, ERR_NO_STATE = 5, 6, 7, 8, 9, 10
ERR_HOST_MEMORY = 11
KERNEL_CUBIC, KERNEL_LUCY = 0, 1
SCHEME_SSA, SCHEME_AMS, SCHEME_EMS, SCHEME_NONE = 0, 1, 2, 3
FP64, MIXED = 0, 1
DEBUG_ORDER, DEBUG_CELLS, DEBUG_RHO, DEBUG_FORCE, DEBUG_NCOUNT, DEBUG_PAIRS, DEBUG_BIG = range(7)


class sdpd_params(C.Structure):
    _fields_ = [
        ("kB", C.c_double), ("eta", C.c_double), ("zeta", C.c_double), ("c_rho", C.c_double),
        ("kernel", C.c_int), ("scheme", C.c_int), ("precision", C.c_int), ("fd_only", C.c_int),
        ("theta", C.c_int), ("debug", C.c_int), ("nc", C.c_int * 3), ("sweep_f32", C.c_int),
    ]


class sdpd_tuning(C.Structure):
    _fields_ = [("fd_variant", C.c_int), ("pair_threads", C.c_int)]


FD_VARIANTS = 5


class sdpd_obs(C.Structure):
    _fields_ = [
        ("E", C.c_double), ("E_int", C.c_double), ("E_kin", C.c_double), ("P", C.c_double * 3),
        ("T_kin", C.c_double), ("T_int", C.c_double), ("eps_min", C.c_double),
        ("n_pairs", C.c_int64), ("n_accept", C.c_int64), ("n_reject_bound", C.c_int64),
        ("n_reject_metropolis", C.c_int64), ("fd_step", C.c_int64), ("vv_step", C.c_int64),
        ("status", C.c_int),
    ]


PAIR_REC_DTYPE = np.dtype([
    ("id_i", np.int64), ("id_j", np.int64), ("colour", np.int32), ("owner", np.int32),
    ("decision", np.int32), ("level", np.int32), ("margin", np.float64),
    ("margin_lo", np.float64), ("margin_tol", np.float64),
])

# Every symbol include/sdpd.h declares: (name, restype, argtypes).
_H = C.c_void_p
_dp = C.POINTER(C.c_double)
SIGNATURES = [
    ("sdpd_create", C.c_int, [C.c_int64, _dp, C.c_double, C.c_double, C.POINTER(sdpd_params),
                              C.c_double, C.c_void_p, C.POINTER(_H)]),
    ("sdpd_workspace_bytes", C.c_size_t, [_H]),
    ("sdpd_bind_workspace", C.c_int, [_H, C.c_void_p, C.c_size_t]),
    ("sdpd_set_state", C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    ("sdpd_get_state", C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    ("sdpd_step", C.c_int, [_H, C.c_double, C.c_int64, C.c_uint64]),
    ("sdpd_observables", C.c_int, [_H, C.POINTER(sdpd_obs)]),
    ("sdpd_sync", C.c_int, [_H]),
    ("sdpd_set_fd_step", C.c_int, [_H, C.c_int64]),
    ("sdpd_get_fd_step", C.c_int64, [_H]),
    ("sdpd_reset_counters", C.c_int, [_H]),
    ("sdpd_kernel_launches", C.c_int64, [_H]),
    ("sdpd_enable_stage_timing", C.c_int, [_H, C.c_int]),
    ("sdpd_stage_times", C.c_int, [_H, _dp, C.POINTER(C.c_int64), C.c_int]),
    ("sdpd_debug_get", C.c_int, [_H, C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    ("sdpd_destroy", None, [_H]),
    ("sdpd_ensemble_create", C.c_int, [C.POINTER(_H), C.c_int, C.c_void_p, C.POINTER(_H)]),
    ("sdpd_ensemble_step", C.c_int, [_H, C.c_double, C.c_int64, C.POINTER(C.c_uint64)]),
    ("sdpd_ensemble_kernel_nodes", C.c_int64, [_H]),
    ("sdpd_ensemble_stream", C.c_void_p, [_H]),
    ("sdpd_ensemble_destroy", None, [_H]),
    ("sdpd_density_static", C.c_int, [C.c_int64, _dp, C.c_double, C.c_double, C.c_int, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    ("sdpd_get_tuning", C.c_int, [_H, C.POINTER(sdpd_tuning)]),
    ("sdpd_set_tuning", C.c_int, [_H, C.POINTER(sdpd_tuning)]),
    ("sdpd_autotune", C.c_int, [_H, C.c_double, C.c_int64, C.c_uint64, C.POINTER(sdpd_tuning), _dp]),
    ("sdpd_ensemble_autotune", C.c_int, [_H, C.c_double, C.c_int64, C.POINTER(C.c_uint64), _dp]),
    ("sdpd_tape_bytes", C.c_size_t, [_H, C.c_int64, C.c_int64]),
    ("sdpd_vv_record", C.c_int, [_H, C.c_double, C.c_int64, C.c_int64, C.c_uint64, C.c_void_p, C.c_size_t]),
    ("sdpd_vv_replay", C.c_int, [_H, C.c_void_p, C.c_size_t]),
    ("sdpd_tape_increments", C.c_int, [_H, C.c_void_p, C.c_size_t, C.c_int64, C.c_void_p, C.c_void_p]),
    ("sdpd_vv_adjoint", C.c_int, [_H, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, _dp]),
    ("sdpd_virial", C.c_int, [_H, _dp, C.c_void_p, C.c_void_p, C.c_void_p, _dp]),
    ("sdpd_fma_peak", C.c_int, [C.c_int, C.c_void_p, _dp]),
    ("sdpd_energy_histogram", C.c_int, [_H, C.c_double, C.c_double, C.c_int, C.c_double, C.c_void_p]),
    ("sdpd_strerror", C.c_char_p, [C.c_int]),
]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.LIB
        if not os.path.exists(path):
            _build.build()
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class SDPDError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().sdpd_strerror(status).decode()
        super().__init__("%s: %s (status %d)" % (where, msg, status))
        self.status = status


def _check(status: int, where: str):
    if status != OK:
        raise SDPDError(status, where)


# --- thin wrappers with the C names ------------------------------------------------

def sdpd_create(N, box, m, h, params: sdpd_params, K, stream: int = 0):
    b = (C.c_double * 3)(*[float(x) for x in box])
    out = _H()
    st = load().sdpd_create(int(N), b, float(m), float(h), C.byref(params), float(K),
                            C.c_void_p(stream), C.byref(out))
    return st, out


def sdpd_workspace_bytes(h) -> int:
    return load().sdpd_workspace_bytes(h)


def sdpd_bind_workspace(h, ptr: int, nbytes: int) -> int:
    return load().sdpd_bind_workspace(h, C.c_void_p(ptr), nbytes)


def sdpd_set_state(h, q, p, eps, on_device: int) -> int:
    return load().sdpd_set_state(h, q, p, eps, on_device)


def sdpd_get_state(h, q, p, eps, on_device: int) -> int:
    return load().sdpd_get_state(h, q, p, eps, on_device)


def sdpd_step(h, dt, nsteps, seed) -> int:
    return load().sdpd_step(h, float(dt), int(nsteps), int(seed))


def sdpd_observables(h, out: sdpd_obs) -> int:
    return load().sdpd_observables(h, C.byref(out))


def sdpd_sync(h) -> int:
    return load().sdpd_sync(h)


def sdpd_set_fd_step(h, v) -> int:
    return load().sdpd_set_fd_step(h, int(v))


def sdpd_get_fd_step(h) -> int:
    return load().sdpd_get_fd_step(h)


def sdpd_reset_counters(h) -> int:
    return load().sdpd_reset_counters(h)


def sdpd_kernel_launches(h) -> int:
    return load().sdpd_kernel_launches(h)


NSTAGES = 10
STAGE_NAMES = ["kick1_drift_bin", "sort", "density_eos", "kick2", "fd_schedule", "fd_colours",
               "adj_load", "adj_pass_A", "adj_pass_B", "adj_elementwise"]


def sdpd_enable_stage_timing(h, on) -> int:
    return load().sdpd_enable_stage_timing(h, int(bool(on)))


def sdpd_stage_times(h):
    ms = (C.c_double * NSTAGES)()
    nl = (C.c_int64 * NSTAGES)()
    st = load().sdpd_stage_times(h, ms, nl, NSTAGES)
    return st, list(ms), list(nl)


def sdpd_debug_get(h, what, dst_ptr, cap):
    cnt = C.c_int64(0)
    st = load().sdpd_debug_get(h, int(what), C.c_void_p(dst_ptr), int(cap), C.byref(cnt))
    return st, cnt.value


def sdpd_density_static(N, box, m, h, kernel, q_ptr: int, rho_ptr: int, stream: int = 0) -> int:
    b = (C.c_double * 3)(*[float(x) for x in box])
    return load().sdpd_density_static(int(N), b, float(m), float(h), int(kernel), C.c_void_p(q_ptr),
                                      C.c_void_p(rho_ptr), C.c_void_p(stream))


def sdpd_ensemble_create(handles, stream: int):
    arr = (_H * len(handles))(*handles)
    out = _H()
    st = load().sdpd_ensemble_create(arr, len(handles), C.c_void_p(stream), C.byref(out))
    return st, out


def sdpd_ensemble_step(e, dt, nsteps, seeds) -> int:
    sv = (C.c_uint64 * len(seeds))(*[int(x) for x in seeds])
    return load().sdpd_ensemble_step(e, float(dt), int(nsteps), sv)


def sdpd_ensemble_kernel_nodes(e) -> int:
    return load().sdpd_ensemble_kernel_nodes(e)


def sdpd_ensemble_stream(e) -> int:
    return load().sdpd_ensemble_stream(e) or 0


def sdpd_ensemble_destroy(e):
    load().sdpd_ensemble_destroy(e)


def sdpd_tape_bytes(h, nsteps, every) -> int:
    return load().sdpd_tape_bytes(h, int(nsteps), int(every))


def sdpd_vv_record(h, dt, nsteps, every, seed, tape_ptr: int, nbytes: int) -> int:
    return load().sdpd_vv_record(h, float(dt), int(nsteps), int(every), int(seed) & (2**64 - 1), tape_ptr, nbytes)


def sdpd_vv_replay(h, tape_ptr: int, nbytes: int) -> int:
    return load().sdpd_vv_replay(h, tape_ptr, nbytes)


def sdpd_tape_increments(h, tape_ptr: int, nbytes: int, step: int, dp: int, deps: int) -> int:
    return load().sdpd_tape_increments(h, tape_ptr, nbytes, int(step), dp, deps)


def sdpd_vv_adjoint(h, tape_ptr, nbytes, gq, gp, geps, gq0, gp0, geps0, gtheta) -> int:
    return load().sdpd_vv_adjoint(h, tape_ptr, nbytes, gq, gp, geps, gq0, gp0, geps0,
                                  gtheta.ctypes.data_as(_dp))


def sdpd_virial(h, value, gq, gp, geps, gtheta) -> int:
    th = gtheta.ctypes.data_as(_dp) if gtheta is not None else None
    return load().sdpd_virial(h, C.byref(value), gq, gp, geps, th)


def sdpd_fma_peak(precision, stream: int = 0) -> float:
    """Measured FMA throughput of the current device in FLOP/s."""
    out = C.c_double(0.0)
    _check(load().sdpd_fma_peak(precision, stream, C.byref(out)), "sdpd_fma_peak")
    return out.value


def sdpd_destroy(h):
    load().sdpd_destroy(h)


def sdpd_strerror(st) -> str:
    return load().sdpd_strerror(int(st)).decode()


# --- convenience object ------------------------------------------------------------

def _ptr(a) -> int:
    """Data pointer of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _state_shapes(N):
    return ((N, 3), (N, 3), (N,))


def _as_state(N, q, p, eps):
    """(q, p, eps, on_device) for N particles.  CUDA tensors become contiguous
    float64 CUDA tensors (on_device = 1); anything else (numpy arrays, CPU
    tensors, sequences) becomes contiguous float64 numpy arrays.  The library
    reads exactly N x 3, N x 3 and N doubles, so any other shape, or a mix of
    host and device inputs, raises ValueError."""
    arrs = (q, p, eps)
    cuda = [bool(getattr(a, "is_cuda", False)) for a in arrs]
    if any(cuda) and not all(cuda):
        raise ValueError("q, p and eps must be all CUDA tensors or all host arrays")
    out = []
    for name, a, shape in zip(("q", "p", "eps"), arrs, _state_shapes(N)):
        if cuda[0]:
            a = a.detach().contiguous().double()
        else:
            if hasattr(a, "detach"):
                a = a.detach().cpu().numpy()
            a = np.ascontiguousarray(a, dtype=np.float64)
        if tuple(a.shape) != shape:
            raise ValueError("%s has shape %s, expected %s" % (name, tuple(a.shape), shape))
        out.append(a)
    return out[0], out[1], out[2], int(cuda[0])


def _check_device_out(N, device, q, p, eps):
    """Destination tensors of a device-side state copy: float64, contiguous,
    on the handle's device, shapes N x 3, N x 3, N."""
    for name, a, shape in zip(("q", "p", "eps"), (q, p, eps), _state_shapes(N)):
        if (not getattr(a, "is_cuda", False) or a.device != device or str(a.dtype) != "torch.float64"
                or not a.is_contiguous() or tuple(a.shape) != shape):
            raise ValueError("%s must be a contiguous float64 tensor of shape %s on %s" % (name, shape, device))


class SDPD:
    """One SDPD system on the current CUDA device.

    The workspace is a torch uint8 tensor owned by this object; all work runs
    on ``stream`` (default: torch's current stream)."""

    def __init__(self, N, box, m=1.0, h=2.5, K=100.0, *, kB=1.0, eta=1.0, zeta=0.0, c_rho=-1.0,
                 kernel=KERNEL_LUCY, scheme=SCHEME_EMS, precision=FP64, fd_only=False, theta=1,
                 debug=False, nc=None, sweep_f32=False, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("SDPD needs a CUDA device")
        self.torch = torch
        self.N = int(N)
        self.m, self.h_smooth, self.K = float(m), float(h), float(K)
        prm = sdpd_params(kB=kB, eta=eta, zeta=zeta, c_rho=c_rho, kernel=kernel, scheme=scheme,
                          precision=precision, fd_only=int(bool(fd_only)), theta=int(theta),
                          debug=int(bool(debug)), sweep_f32=int(bool(sweep_f32)))
        if nc is not None:  # cells per axis (0 = the default grid on that axis)
            for d, n in enumerate(nc if np.ndim(nc) else (nc,) * 3):
                prm.nc[d] = int(n)
        self.params = prm
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        st, self.h = sdpd_create(N, box if np.ndim(box) else (box,) * 3, m, h, prm, K,
                                 self.stream.cuda_stream)
        _check(st, "sdpd_create")
        nbytes = sdpd_workspace_bytes(self.h)
        self.workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
        _check(sdpd_bind_workspace(self.h, self.workspace.data_ptr(), nbytes), "sdpd_bind_workspace")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            try:
                sdpd_sync(h)
            finally:
                sdpd_destroy(h)
            self.h = None

    def set_state(self, q, p, eps):
        """Load positions [N,3], momenta [N,3] and internal energies [N] in id
        order, from host arrays or from CUDA tensors on the handle's device."""
        q, p, eps, on_device = _as_state(self.N, q, p, eps)
        if on_device:
            if q.device != self.workspace.device:
                raise ValueError("state tensors are on %s, the handle on %s" % (q.device, self.workspace.device))
            self._keep = (q, p, eps)
        _check(sdpd_set_state(self.h, _ptr(q), _ptr(p), _ptr(eps), on_device), "sdpd_set_state")

    def get_state(self):
        q = np.empty((self.N, 3))
        p = np.empty((self.N, 3))
        e = np.empty(self.N)
        _check(sdpd_get_state(self.h, _ptr(q), _ptr(p), _ptr(e), 0), "sdpd_get_state")
        return q, p, e

    def get_state_device(self, q, p, eps):
        """Copy the state into float64 CUDA tensors (id order); synchronises."""
        _check_device_out(self.N, self.workspace.device, q, p, eps)
        _check(sdpd_get_state(self.h, _ptr(q), _ptr(p), _ptr(eps), 1), "sdpd_get_state")

    def step(self, dt, nsteps=1, seed=0):
        _check(sdpd_step(self.h, dt, nsteps, seed), "sdpd_step")

    def sync(self):
        return sdpd_sync(self.h)

    def energy_histogram(self, lo, hi, nbins, scale=1.0, counts=None):
        """Add the histogram of eps * scale over nbins bins of [lo, hi) (then
        the counts below lo and at or above hi) into ``counts``, a CUDA int64
        tensor of nbins + 2 entries (allocated zeroed when None); returns it."""
        if counts is None:
            counts = self.torch.zeros(nbins + 2, dtype=self.torch.int64, device=self.workspace.device)
        elif (counts.device != self.workspace.device or counts.dtype != self.torch.int64
              or not counts.is_contiguous() or counts.numel() < int(nbins) + 2):
            raise ValueError("counts must be a contiguous int64 tensor of nbins + 2 entries on %s"
                             % self.workspace.device)
        _check(load().sdpd_energy_histogram(self.h, float(lo), float(hi), int(nbins), float(scale),
                                            counts.data_ptr()), "sdpd_energy_histogram")
        return counts

    # -- launch shapes and the autotuner ------------------------------------

    @property
    def tuning(self) -> dict:
        t = sdpd_tuning()
        _check(load().sdpd_get_tuning(self.h, C.byref(t)), "sdpd_get_tuning")
        return {"fd_variant": t.fd_variant, "pair_threads": t.pair_threads}

    def set_tuning(self, fd_variant=-1, pair_threads=0):
        t = sdpd_tuning(fd_variant=int(fd_variant), pair_threads=int(pair_threads))
        _check(load().sdpd_set_tuning(self.h, C.byref(t)), "sdpd_set_tuning")

    def autotune(self, dt, steps=3, seed=0):
        """Times every launch shape on the loaded state, keeps the fastest
        and restores the state; returns (tuning, ms per step)."""
        t = sdpd_tuning()
        ms = C.c_double(0.0)
        _check(load().sdpd_autotune(self.h, float(dt), int(steps), int(seed) & (2**64 - 1), C.byref(t),
                                    C.byref(ms)), "sdpd_autotune")
        return {"fd_variant": t.fd_variant, "pair_threads": t.pair_threads}, ms.value

    # -- gradients of the conservative dynamics (float64 handles) ----------

    def tape_bytes(self, nsteps, every=10) -> int:
        return sdpd_tape_bytes(self.h, nsteps, every)

    def vv_record(self, dt, nsteps, every=10, seed=0):
        """Full steps from the loaded state (Velocity Verlet, then the
        handle's sweep with random numbers keyed by ``seed``), recorded for
        vv_adjoint with a checkpoint every ``every`` steps and each sweep's
        increments frozen.  Returns the tape (a CUDA uint8 tensor that must
        stay alive until the last adjoint)."""
        n = self.tape_bytes(nsteps, every)
        if n == 0:
            raise ValueError("bad nsteps/every")
        tape = self.torch.empty(n, dtype=self.torch.uint8, device=self.workspace.device)
        _check(sdpd_vv_record(self.h, dt, nsteps, every, seed, tape.data_ptr(), n), "sdpd_vv_record")
        self._tape = tape
        return tape

    def vv_replay(self, tape):
        """Applies the recorded frozen map (Verlet steps plus the recorded
        sweep increments) to the currently loaded state."""
        _check(sdpd_vv_replay(self.h, tape.data_ptr(), tape.numel()), "sdpd_vv_replay")

    def tape_increments(self, tape, step):
        """The recorded sweep increments (dp [N,3], deps [N]) of one step."""
        torch = self.torch
        dev = self.workspace.device
        dp = torch.empty((self.N, 3), dtype=torch.float64, device=dev)
        de = torch.empty(self.N, dtype=torch.float64, device=dev)
        _check(sdpd_tape_increments(self.h, tape.data_ptr(), tape.numel(), step, dp.data_ptr(), de.data_ptr()),
               "sdpd_tape_increments")
        return dp, de

    def vv_adjoint(self, tape, gq=None, gp=None, geps=None):
        """Cotangents (gq0, gp0, geps0, gtheta) of the recorded trajectory's
        initial state and of theta = (h, c_rho, C_K), given those of its
        final state (float64 CUDA tensors in id order, None = zero)."""
        torch = self.torch
        dev = self.workspace.device
        keep = [None if g is None else g.detach().contiguous().double() for g in (gq, gp, geps)]
        for name, g, shape in zip(("gq", "gp", "geps"), keep, _state_shapes(self.N)):
            if g is not None and (g.device != dev or tuple(g.shape) != shape):
                raise ValueError("%s must have shape %s on %s" % (name, shape, dev))
        ptr = [0 if g is None else g.data_ptr() for g in keep]
        gq0 = torch.empty((self.N, 3), dtype=torch.float64, device=dev)
        gp0 = torch.empty((self.N, 3), dtype=torch.float64, device=dev)
        ge0 = torch.empty(self.N, dtype=torch.float64, device=dev)
        gth = np.zeros(3)
        _check(sdpd_vv_adjoint(self.h, tape.data_ptr(), tape.numel(), ptr[0] or None, ptr[1] or None,
                               ptr[2] or None, gq0.data_ptr(), gp0.data_ptr(), ge0.data_ptr(), gth),
               "sdpd_vv_adjoint")
        return gq0, gp0, ge0, gth

    def virial(self, grad=False):
        """Virial pressure of the current state; with grad, also
        (dP/dq, dP/dp, dP/deps) as CUDA tensors and dP/dtheta."""
        value = C.c_double(0.0)
        if not grad:
            _check(sdpd_virial(self.h, value, None, None, None, None), "sdpd_virial")
            return value.value
        torch = self.torch
        dev = self.workspace.device
        gq = torch.empty((self.N, 3), dtype=torch.float64, device=dev)
        gp = torch.empty((self.N, 3), dtype=torch.float64, device=dev)
        ge = torch.empty(self.N, dtype=torch.float64, device=dev)
        gth = np.zeros(3)
        _check(sdpd_virial(self.h, value, gq.data_ptr(), gp.data_ptr(), ge.data_ptr(), gth), "sdpd_virial")
        return value.value, gq, gp, ge, gth

    def observables(self, check=True) -> dict:
        o = sdpd_obs()
        st = sdpd_observables(self.h, o)
        if check:
            _check(st, "sdpd_observables")
        return {"E": o.E, "E_int": o.E_int, "E_kin": o.E_kin, "P": np.array(o.P[:]),
                "T_kin": o.T_kin, "T_int": o.T_int, "eps_min": o.eps_min, "n_pairs": o.n_pairs,
                "n_accept": o.n_accept, "n_reject_bound": o.n_reject_bound,
                "n_reject_metropolis": o.n_reject_metropolis, "fd_step": o.fd_step,
                "vv_step": o.vv_step, "status": o.status}

    @property
    def fd_step(self) -> int:
        return sdpd_get_fd_step(self.h)

    @fd_step.setter
    def fd_step(self, v):
        _check(sdpd_set_fd_step(self.h, v), "sdpd_set_fd_step")

    def reset_counters(self):
        _check(sdpd_reset_counters(self.h), "sdpd_reset_counters")

    @property
    def kernel_launches(self) -> int:
        return sdpd_kernel_launches(self.h)

    def enable_stage_timing(self, on=True):
        _check(sdpd_enable_stage_timing(self.h, on), "sdpd_enable_stage_timing")

    def stage_times(self) -> dict:
        st, ms, nl = sdpd_stage_times(self.h)
        _check(st, "sdpd_stage_times")
        return {name: (m, n) for name, m, n in zip(STAGE_NAMES, ms, nl)}

    def _debug(self, what, arr, cap):
        st, n = sdpd_debug_get(self.h, what, _ptr(arr), cap)
        _check(st, "sdpd_debug_get")
        return n

    def order(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int64)
        self._debug(DEBUG_ORDER, out, self.N)
        return out

    def cells(self) -> np.ndarray:
        out = np.empty((self.N, 3), dtype=np.int32)
        self._debug(DEBUG_CELLS, out, self.N)
        return out

    def density(self) -> np.ndarray:
        out = np.empty(self.N)
        self._debug(DEBUG_RHO, out, self.N)
        return out

    def forces(self) -> np.ndarray:
        out = np.empty((self.N, 3))
        self._debug(DEBUG_FORCE, out, 3 * self.N)
        return out

    def neighbour_counts(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int32)
        self._debug(DEBUG_NCOUNT, out, self.N)
        return out

    def big_blocks(self) -> np.ndarray:
        """Per colour, the blocks of the latest sweep schedule swept pair by
        pair (beyond the schedule's capacities)."""
        out = np.empty(8, dtype=np.uint32)
        self._debug(DEBUG_BIG, out, 8)
        return out

    def pair_records(self) -> np.ndarray:
        cap = max(1, self.N) * 64
        out = np.empty(cap, dtype=PAIR_REC_DTYPE)
        n = self._debug(DEBUG_PAIRS, out, cap)
        return out[:n].copy()


class SDPDEnsemble:
    """Independent systems stepped together by one CUDA graph.

    ``members`` are SDPD objects with loaded states, created on streams
    other than the ensemble's; the ensemble launches on ``stream`` (default:
    a stream the library creates for it, exposed as a torch ExternalStream)
    and keeps the members alive."""

    def __init__(self, members, stream=None):
        import torch

        self.members = list(members)
        st, self.e = sdpd_ensemble_create([m.h for m in self.members],
                                          stream.cuda_stream if stream is not None else 0)
        _check(st, "sdpd_ensemble_create")
        self.stream = stream if stream is not None else torch.cuda.ExternalStream(
            sdpd_ensemble_stream(self.e))

    def __del__(self):
        e = getattr(self, "e", None)
        if e:
            sdpd_ensemble_destroy(e)
            self.e = None

    def step(self, dt, nsteps, seeds):
        _check(sdpd_ensemble_step(self.e, dt, nsteps, seeds), "sdpd_ensemble_step")

    def autotune(self, dt, steps=4, seeds=None):
        """Chooses the members' launch shapes for the ensemble as a whole
        (states restored); returns the ensemble's time per step with them."""
        n = len(self.members)
        arr = None
        if seeds is not None:
            arr = (C.c_uint64 * n)(*[int(x) & (2**64 - 1) for x in seeds])
        ms = C.c_double(0.0)
        _check(load().sdpd_ensemble_autotune(self.e, float(dt), int(steps), arr, C.byref(ms)),
               "sdpd_ensemble_autotune")
        return ms.value

    @property
    def kernel_nodes(self) -> int:
        return sdpd_ensemble_kernel_nodes(self.e)
