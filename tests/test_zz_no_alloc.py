"""The allocation-free density entry point against the library's regular path.

sdpd_density_static serves callers that cannot allocate device memory: it
keeps its working memory in a fixed static array instead of a bound
workspace.  Its densities must equal those of the regular path (workspace,
sdpd_set_state, the density read-out) within the float64 tolerance of the
parity tests, on two calls in a row (the second call reuses the array the
first one left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1707_04232_gb300.inputs import Workload, lattice_state, random_box_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1707_04232_gb300 import sdpd  # noqa: E402


def systems():
    w = Workload(n=10, K=100.0, jitter=0.05, seed=0)
    q, p, e = lattice_state(w)
    yield "lattice1000", q, p, e, (w.L,) * 3
    L = (12.5, 15.0, 17.3)
    N = 3244
    q, p, e = random_box_state(N, 1.0, 1.0, 1.0, 28.5, seed=9)
    q = np.where(q * np.array(L) >= np.array(L), 0.0, q * np.array(L))
    yield "random_rect", q, p, e, L
    # 16^3 = 4096 cells (more than the 1024 threads of the cell scan, which
    # then takes several cells per thread); a few coordinates just below 0
    # and exactly at the box side, which both paths wrap periodically
    L = (40.0,) * 3
    N = 5000
    q, p, e = random_box_state(N, 1.0, 1.0, 1.0, 28.5, seed=12)
    q = q * 40.0
    q[:8, 0] = -1e-12
    q[8:16, 1] = 40.0
    q[16:24, 2] = -1e-12
    yield "random_40_edges", q, p, e, L


@pytest.mark.parametrize("kernel", [sdpd.KERNEL_LUCY, sdpd.KERNEL_CUBIC])
def test_static_density_matches_regular_path_twice(kernel):
    for name, q, p, e, L in systems():
        N = len(e)
        reg = sdpd.SDPD(N, L, m=1.0, h=2.5, K=100.0, precision=sdpd.FP64, kernel=kernel)
        reg.set_state(q, p, e)
        expect = reg.density()
        qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
        stream = torch.cuda.current_stream()
        for call in range(2):
            rho = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
            st = sdpd.sdpd_density_static(N, L, 1.0, 2.5, kernel, qd.data_ptr(), rho.data_ptr(),
                                          stream.cuda_stream)
            assert st == sdpd.OK, (name, call, sdpd.sdpd_strerror(st))
            torch.cuda.synchronize()
            got = rho.cpu().numpy()
            assert np.abs(got - expect).max() <= 1e-12 * expect.max(), (name, call)


def test_static_density_rejects_oversize_inputs():
    """Beyond the fixed working memory: rejected on the host with
    SDPD_ERR_CAPACITY before any device work, with valid buffers too."""
    N = 1000
    qd = torch.rand((N, 3), dtype=torch.float64, device="cuda") * 10.0
    rho = torch.full((N,), -7.0, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    # too many particles
    st = sdpd.sdpd_density_static(65537, (100.0,) * 3, 1.0, 2.5, sdpd.KERNEL_LUCY, 0, 0, s)
    assert st == sdpd.ERR_CAPACITY
    # too many cells: 200^3 cells for a 500^3 box at h = 2.5
    st = sdpd.sdpd_density_static(N, (500.0,) * 3, 1.0, 2.5, sdpd.KERNEL_LUCY, qd.data_ptr(), rho.data_ptr(), s)
    assert st == sdpd.ERR_CAPACITY
    torch.cuda.synchronize()
    assert (rho.cpu().numpy() == -7.0).all()
