"""The C-ABI library loads without a GPU and exports every symbol that
include/sdpd.h declares; host-side argument checks need no device."""
import ctypes as C
import os
import re

import pytest

from paper_1707_04232_gb300 import build as B
from paper_1707_04232_gb300 import sdpd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sdpd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdpd_[a-z_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = C.CDLL(path)
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    bound = {name for name, _, _ in sdpd.SIGNATURES}
    assert set(names) == bound


def _params(**kw):
    p = sdpd.sdpd_params(kB=1.0, eta=1.0, zeta=0.0, c_rho=-1.0, kernel=1, scheme=2, precision=0,
                         fd_only=0, theta=1, debug=0)
    for k, v in kw.items():
        if k == "nc":
            for d in range(3):
                p.nc[d] = v[d]
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw,box,K,expect", [
    ({}, (10.0, 10.0, 10.0), 100.0, sdpd.OK),
    ({}, (9.0, 10.0, 10.0), 100.0, sdpd.ERR_BOX_TOO_SMALL),
    ({}, (10.0, 10.0, 10.0), 1.2, sdpd.ERR_INVALID_ARG),   # K <= 4/3
    ({"eta": 0.0}, (10.0, 10.0, 10.0), 100.0, sdpd.ERR_INVALID_ARG),
    ({"zeta": 2.0}, (10.0, 10.0, 10.0), 100.0, sdpd.ERR_INVALID_ARG),  # zeta >= 5 eta / 3
    ({"kernel": 7}, (10.0, 10.0, 10.0), 100.0, sdpd.ERR_INVALID_ARG),
    ({"theta": 0}, (10.0, 10.0, 10.0), 100.0, sdpd.ERR_INVALID_ARG),
    ({"nc": (4, 4, 4)}, (10.0, 10.0, 10.0), 100.0, sdpd.OK),           # the default grid, chosen
    ({"nc": (4, 0, 6)}, (10.0, 10.0, 16.0), 100.0, sdpd.OK),           # 0 = default on that axis
    ({"nc": (6, 4, 4)}, (10.0, 10.0, 10.0), 100.0, sdpd.ERR_BOX_TOO_SMALL),  # cells below h
    ({"nc": (5, 4, 4)}, (20.0, 10.0, 10.0), 100.0, sdpd.ERR_INVALID_ARG),    # odd
    ({"nc": (2, 4, 4)}, (20.0, 10.0, 10.0), 100.0, sdpd.ERR_INVALID_ARG),    # fewer than 4
])
def test_create_validates_on_host(kw, box, K, expect):
    st, h = sdpd.sdpd_create(1000, box, 1.0, 2.5, _params(**kw), K, 0)
    assert st == expect
    if st == sdpd.OK:
        assert sdpd.sdpd_workspace_bytes(h) > 0
        # no workspace bound: every device call is refused without touching a GPU
        assert sdpd.sdpd_step(h, 0.005, 1, 0) == sdpd.ERR_NO_WORKSPACE
        assert sdpd.sdpd_bind_workspace(h, 0, 0) == sdpd.ERR_NO_WORKSPACE
        assert sdpd.sdpd_step(h, -1.0, 1, 0) == sdpd.ERR_INVALID_ARG
        sdpd.sdpd_destroy(h)
    else:
        assert not h


def test_workspace_scales_with_precision():
    st, h64 = sdpd.sdpd_create(32768, (32.0,) * 3, 1.0, 2.5, _params(precision=0), 100.0, 0)
    st2, hm = sdpd.sdpd_create(32768, (32.0,) * 3, 1.0, 2.5, _params(precision=1), 100.0, 0)
    assert st == st2 == sdpd.OK
    assert sdpd.sdpd_workspace_bytes(hm) < sdpd.sdpd_workspace_bytes(h64)
    sdpd.sdpd_destroy(h64)
    sdpd.sdpd_destroy(hm)


def test_strerror_covers_codes():
    for code in range(12):
        assert sdpd.sdpd_strerror(code) != "unknown status"
    assert sdpd.sdpd_strerror(12) == "unknown status"


def test_status_codes_match_the_header():
    text = open(os.path.join(ROOT, "include", "sdpd.h")).read()
    codes = dict(re.findall(r"#define SDPD_(OK|ERR_[A-Z_]+) (\d+)", text))
    assert len(codes) == 12
    for name, value in codes.items():
        assert getattr(sdpd, name) == int(value), name


def test_debug_read_out_refused_without_workspace():
    lib = sdpd.load()
    st, h = sdpd.sdpd_create(1000, (10.0,) * 3, 1.0, 2.5, _params(), 100.0, 0)
    assert st == sdpd.OK
    buf = (C.c_int64 * 1000)()
    n = C.c_int64(-1)
    assert lib.sdpd_debug_get(h, 0, buf, 1000, C.byref(n)) == sdpd.ERR_NO_WORKSPACE
    assert lib.sdpd_debug_get(h, 0, None, 1000, C.byref(n)) == sdpd.ERR_INVALID_ARG
    sdpd.sdpd_destroy(h)


def test_float32_sweep_flag_on_host():
    # accepted on both precisions; a float64 handle with it takes the float32
    # block schedules (all five fit in shared memory)
    lib = sdpd.load()
    st, h = sdpd.sdpd_create(8000, (20.0,) * 3, 1.0, 2.5, _params(precision=0, sweep_f32=1), 100.0, 0)
    assert st == sdpd.OK
    t = sdpd.sdpd_tuning()
    assert lib.sdpd_get_tuning(h, C.byref(t)) == sdpd.OK and t.fd_variant == 0
    for v in range(5):
        assert lib.sdpd_set_tuning(h, C.byref(sdpd.sdpd_tuning(fd_variant=v, pair_threads=128))) == sdpd.OK
    sdpd.sdpd_destroy(h)


def test_coarser_cell_grid_needs_less_workspace():
    st, h1 = sdpd.sdpd_create(32768, (32.0,) * 3, 1.0, 2.5, _params(precision=1), 100.0, 0)
    st2, h2 = sdpd.sdpd_create(32768, (32.0,) * 3, 1.0, 2.5, _params(precision=1, nc=(10, 10, 10)), 100.0, 0)
    assert st == st2 == sdpd.OK
    assert sdpd.sdpd_workspace_bytes(h2) < sdpd.sdpd_workspace_bytes(h1)
    sdpd.sdpd_destroy(h1)
    sdpd.sdpd_destroy(h2)


@pytest.mark.parametrize("precision,default,fits", [
    (0, 1, {0, 1, 2, 3, 4}),    # float64: four block groups of 10.9 KB fit in 48 KB
    (1, 0, {0, 1, 2, 3, 4}),
])
def test_launch_shapes_on_host(precision, default, fits):
    lib = sdpd.load()
    st, h = sdpd.sdpd_create(8000, (20.0,) * 3, 1.0, 2.5, _params(precision=precision), 100.0, 0)
    assert st == sdpd.OK
    t = sdpd.sdpd_tuning()
    assert lib.sdpd_get_tuning(h, C.byref(t)) == sdpd.OK
    assert (t.fd_variant, t.pair_threads) == (default, 128)
    for v in range(-1, sdpd.FD_VARIANTS + 1):
        for pt in (0, 32, 48, 64, 128, 256):
            want = (v == -1 or v in fits) and pt in (0, 32, 64, 128)
            r = lib.sdpd_set_tuning(h, C.byref(sdpd.sdpd_tuning(fd_variant=v, pair_threads=pt)))
            assert r == (sdpd.OK if want else sdpd.ERR_INVALID_ARG), (v, pt)
            if want:
                assert lib.sdpd_get_tuning(h, C.byref(t)) == sdpd.OK
                assert t.fd_variant == (default if v == -1 else v)
                assert t.pair_threads == (128 if pt == 0 else pt)
    # the autotuner needs a workspace and a state; refused without touching a device
    assert lib.sdpd_autotune(h, 0.005, 2, 0, None, None) == sdpd.ERR_NO_WORKSPACE
    assert lib.sdpd_autotune(h, -1.0, 2, 0, None, None) == sdpd.ERR_INVALID_ARG
    assert lib.sdpd_autotune(h, 0.005, 0, 0, None, None) == sdpd.ERR_INVALID_ARG
    sdpd.sdpd_destroy(h)


def test_state_arrays_are_checked_before_the_library_reads_them():
    """The binding hands the library bare pointers to N x 3, N x 3 and N
    doubles, so it converts and checks shapes first (no device needed)."""
    import numpy as np
    torch = pytest.importorskip("torch")
    N = 5
    q, p, e = np.zeros((N, 3), np.float32), torch.ones(N, 3), [1.0] * N
    qq, pp, ee, on_device = sdpd._as_state(N, q, p, e)
    assert on_device == 0
    for a, shape in zip((qq, pp, ee), ((N, 3), (N, 3), (N,))):
        assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.shape == shape
        assert a.flags["C_CONTIGUOUS"]
    assert (pp == 1.0).all() and (ee == 1.0).all()
    for bad in ((np.zeros((N - 1, 3)), p, e), (q, np.zeros(3 * N), e), (q, p, np.zeros((N, 1)))):
        with pytest.raises(ValueError):
            sdpd._as_state(N, *bad)

    class OnDevice:  # stands in for a CUDA tensor
        is_cuda = True

    with pytest.raises(ValueError):
        sdpd._as_state(N, OnDevice(), p, e)
    with pytest.raises(ValueError):  # device-side outputs must be CUDA tensors
        sdpd._check_device_out(N, torch.device("cuda", 0), torch.zeros(N, 3, dtype=torch.float64),
                               torch.zeros(N, 3, dtype=torch.float64), torch.zeros(N, dtype=torch.float64))


def test_product_path_fails_loudly_without_its_library(monkeypatch, tmp_path):
    """No fallback: a missing CUDA library raises, and so does a handle
    without a CUDA device; the package never imports the oracle."""
    monkeypatch.setattr(sdpd, "_lib", None)
    with pytest.raises(OSError):
        sdpd.load(str(tmp_path / "libsdpd.so"))
    monkeypatch.undo()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            sdpd.SDPD(1000, 10.0)
    pkg = os.path.join(ROOT, "paper_1707_04232_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "sdpd_oracle" not in text, f


@pytest.mark.parametrize("N", [1000, 32768])
def test_tape_size_follows_the_header_formula(N):
    """sdpd_tape_bytes is host arithmetic: the states at the checkpoints, the
    final state and one segment (56 B per particle each), every step's
    increments (32 B), the reverse pass's buffers (160 B), plus alignment and
    the reduction partials (a few KiB)."""
    st, h = sdpd.sdpd_create(N, (32.0,) * 3, 1.0, 2.5, _params(), 100.0, 0)
    assert st == sdpd.OK
    for nsteps in (0, 1, 7, 100):
        for every in (1, 3, 10, 200):
            slots = -(-nsteps // every) + max(1, min(every, nsteps))
            expect = (slots * 56 + max(1, nsteps) * 32 + 160) * N
            got = sdpd.sdpd_tape_bytes(h, nsteps, every)
            assert expect <= got <= expect + 64 * 1024, (nsteps, every, got, expect)
    assert sdpd.sdpd_tape_bytes(h, -1, 1) == 0 and sdpd.sdpd_tape_bytes(h, 5, 0) == 0
    sdpd.sdpd_destroy(h)
