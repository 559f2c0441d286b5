"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: a closed
form, an invariant of the dynamics, a library routine, brute force on a tiny
input or an exact sampling property.  No test here needs a GPU.
"""
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as O
from paper_1707_04232_gb300.inputs import Workload, lattice_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_cfg(n=10, K=100.0, kernel=O.KERNEL_LUCY, scheme=O.SCHEME_EMS, **kw):
    return O.Config(N=n ** 3, L=float(n), K=K, kernel=kernel, scheme=scheme, **kw)


# --------------------------------------------------------------------------
# Smoothing kernels (Section 2.1.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [O.KERNEL_CUBIC, O.KERNEL_LUCY])
@pytest.mark.parametrize("h", [1.0, 2.5])
def test_kernel_normalised(kernel, h):
    """The kernel integrates to 1 over R^3 (normalisation of Section 2.1.1)."""
    val, _ = integrate.quad(lambda r: O.W(kernel, r, h) * 4 * np.pi * r * r, 0, h,
                            points=[0.5 * h], epsabs=1e-14, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-11


@pytest.mark.parametrize("kernel", [O.KERNEL_CUBIC, O.KERNEL_LUCY])
def test_kernel_support_and_gradient(kernel):
    """W and F vanish at r >= h; F = -W'(r)/r (grad W = -F r); both are
    continuous at r = h/2."""
    h = 2.5
    for r in (h, h * 1.0001, 3 * h):
        assert O.W(kernel, r, h) == 0.0 and O.F(kernel, r, h) == 0.0
    for r in np.linspace(0.05, h - 0.05, 41):
        if abs(r - 0.5 * h) < 1e-3:
            continue
        d = 1e-6
        dW = (O.W(kernel, r + d, h) - O.W(kernel, r - d, h)) / (2 * d)
        assert abs(-dW / r - O.F(kernel, r, h)) < 1e-7 * max(1.0, abs(dW / r))
    e = 1e-12
    for f in (O.W, O.F):
        assert abs(f(kernel, 0.5 * h - e, h) - f(kernel, 0.5 * h + e, h)) < 1e-9
    assert O.F(kernel, 0.999 * h, h) > 0.0


# --------------------------------------------------------------------------
# Geometry, cells, storage order
# --------------------------------------------------------------------------

def test_perfect_lattice_density_and_neighbours():
    """On a perfect simple-cubic lattice every particle sees the same
    neighbourhood: all densities are equal, every particle has the 80
    neighbours of the shell table, and by symmetry the forces vanish."""
    shells = np.loadtxt(os.path.join(GOLDEN, "lattice_shells.txt"), dtype=int)
    expected = int(shells[shells[:, 0] < 6.25, 1].sum())
    assert expected == 80
    for kernel in (O.KERNEL_CUBIC, O.KERNEL_LUCY):
        w = Workload(n=10, jitter=0.0)
        q, p, eps = lattice_state(w)
        P = small_cfg(kernel=kernel).params()
        rho = O.density(P, q)
        assert np.ptp(rho) < 1e-13
        # a lattice sum of a normalised kernel is close to the mean density m/a^3
        assert abs(rho[0] - 1.0) < 5e-3
        # and equals the self term plus the shell table's sum (Eq. sdpd-rho-v)
        inside = shells[shells[:, 0] < 6.25]
        w_shells = sum(int(c) * float(O.W(kernel, np.sqrt(n2) * w.a, P.h)) for n2, c in inside)
        exact = P.m * (float(O.W(kernel, 0.0, P.h)) + w_shells)
        assert abs(rho[0] - exact) <= 1e-13 * exact
        assert (O.neighbour_counts(P, q) == expected).all()
        f = O.forces(P, q, rho, eps)
        assert np.abs(f).max() < 1e-12


def test_sampled_density_and_force_equal_full_sums():
    """The per-particle entry points used for sampled checks at full size
    compute the same sums as the all-particle ones."""
    w = Workload(n=10, jitter=0.3, seed=13)
    q, p, eps = lattice_state(w)
    eps = eps * (1 + 0.2 * np.random.default_rng(2).random(w.N))
    P = small_cfg().params()
    rho = O.density(P, q)
    f = O.forces(P, q, rho, eps)
    idx = np.array([0, 7, 123, 999])
    assert np.abs(O.density_at(P, q, idx) - rho[idx]).max() <= 1e-14 * rho.max()
    assert (O.neighbour_count_at(P, q, idx) == O.neighbour_counts(P, q)[idx]).all()
    assert np.abs(O.forces_at(P, q, eps, idx) - f[idx]).max() <= 1e-12 * np.abs(f).max()


def test_min_image_and_wrap():
    L = 10.0
    assert O.lib().orc_min_image(6.0, L) == -4.0
    assert O.lib().orc_min_image(-6.0, L) == 4.0
    assert O.lib().orc_min_image(4.9, L) == 4.9
    assert O.lib().orc_wrap(10.25, L) == 0.25
    assert O.lib().orc_wrap(-0.25, L) == 9.75
    assert O.lib().orc_wrap(-1e-17, L) == 0.0  # rounds to L -> wraps to 0


def test_morton_interleave():
    """morton3 interleaves bits x0 y0 z0 x1 y1 z1 ... (brute force decode)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        x, y, z = (int(v) for v in rng.integers(0, 1 << 10, 3))
        c = O.morton3(x, y, z)
        dx = sum(((c >> (3 * b)) & 1) << b for b in range(10))
        dy = sum(((c >> (3 * b + 1)) & 1) << b for b in range(10))
        dz = sum(((c >> (3 * b + 2)) & 1) << b for b in range(10))
        assert (dx, dy, dz) == (x, y, z)
    assert O.morton3(1, 0, 0) == 1 and O.morton3(0, 1, 0) == 2 and O.morton3(0, 0, 1) == 4


def test_cells_and_sorted_order():
    w = Workload(n=10, jitter=0.3, seed=3)
    q, _, _ = lattice_state(w)
    P = small_cfg().params()
    c = O.cells(P, q)
    cs = np.array(P.cs[:])
    # every particle lies inside its cell
    lo, hi = c * cs, (c + 1) * cs
    assert ((q >= lo - 1e-12) & (q < hi + 1e-12)).all()
    order = O.sorted_order(P, q)
    assert sorted(order.tolist()) == list(range(P.N))
    keys = np.array([O.morton3(*c[i]) for i in order])
    ids = order
    assert (np.diff(keys) >= 0).all()
    same = np.diff(keys) == 0
    assert (np.diff(ids)[same] > 0).all()


# --------------------------------------------------------------------------
# Equation of state (Section 2.1.2, Eq. pg-eos)
# --------------------------------------------------------------------------

def test_eos_closed_forms():
    P = small_cfg(K=7.0).params()
    C_K = 1.5 * 6.0
    for eps, rho in [(0.3, 0.9), (9.0, 1.0), (40.0, 1.3)]:
        S = O.lib().orc_S(P, eps, rho)
        # round trip E(S(eps, rho), rho) = eps
        assert abs(O.lib().orc_E_of_S(P, S, rho) - eps) < 1e-13 * eps
        # temperature and heat capacity of the ideal gas
        assert abs(O.lib().orc_T(P, eps) - eps / C_K) < 1e-15 * eps
        assert abs(O.lib().orc_C(P, eps) - C_K) < 1e-13
        # pressure from numerical derivatives of S
        d = 1e-6
        dSe = (O.lib().orc_S(P, eps * (1 + d), rho) - O.lib().orc_S(P, eps * (1 - d), rho)) / (2 * d * eps)
        dSr = (O.lib().orc_S(P, eps, rho * (1 + d)) - O.lib().orc_S(P, eps, rho * (1 - d))) / (2 * d * rho)
        Pfd = -(rho * rho / P.m) * dSr / dSe
        assert abs(O.lib().orc_P(P, eps, rho) - Pfd) < 1e-7 * abs(Pfd)
        # temperature from the numerical derivative of S
        assert abs(O.lib().orc_T(P, eps) - 1.0 / dSe) < 1e-7 * eps


# --------------------------------------------------------------------------
# Conservative forces (Eq. cons-forces) = -grad H (Section 3.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [O.KERNEL_CUBIC, O.KERNEL_LUCY])
def test_force_is_minus_grad_hamiltonian(kernel):
    w = Workload(n=6, jitter=0.25, K=5.0, seed=11)
    q, p, eps = lattice_state(w)
    eps = eps * (1.0 + 0.3 * np.random.default_rng(5).random(w.N))
    cfg = O.Config(N=w.N, L=w.L, K=w.K, kernel=kernel, h=1.45)
    P = cfg.params()
    rho = O.density(P, q)
    S = O.entropy(P, eps, rho)
    f = O.forces(P, q, rho, eps)
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * np.abs(f).max() * w.N
    d = 2e-5
    fmax = np.abs(f).max()
    for i in (0, 17, 101, 200):
        for k in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, k] += d
            qm[i, k] -= d
            g = (O.hamiltonian(P, qp, p, S) - O.hamiltonian(P, qm, p, S)) / (2 * d)
            assert abs(-g - f[i, k]) < 2e-7 * fmax, (i, k, -g, f[i, k])


# --------------------------------------------------------------------------
# Velocity Verlet (Eq. sdpd-verlet)
# --------------------------------------------------------------------------

def test_verlet_time_reversible():
    w = Workload(n=10, jitter=0.1, K=20.0, seed=2)
    q0, p0, e0 = lattice_state(w)
    P = O.Config(N=w.N, L=w.L, K=w.K, scheme=O.SCHEME_NONE).params()
    s, q, p, e, _, _ = O.run(P, q0, p0, e0, 0.01, 15, seed=0)
    s, q, p, e, _, _ = O.run(P, q, -p, e, 0.01, 15, seed=0)
    dq = np.abs(((q - q0) + 0.5 * w.L) % w.L - 0.5 * w.L).max()
    assert dq < 1e-10
    assert np.abs(-p - p0).max() < 1e-9
    assert np.abs(e - e0).max() < 1e-9 * e0.max()


def test_verlet_energy_error_second_order():
    w = Workload(n=10, jitter=0.1, K=20.0, seed=4)
    q0, p0, e0 = lattice_state(w)
    P = O.Config(N=w.N, L=w.L, K=w.K, scheme=O.SCHEME_NONE).params()
    E0 = O.observables(P, p0, e0)["E"]
    errs = []
    for dt, n in ((0.02, 10), (0.01, 20)):
        _, q, p, e, _, _ = O.run(P, q0, p0, e0, dt, n, seed=0)
        errs.append(abs(O.observables(P, p, e)["E"] - E0))
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.3, ratio


# --------------------------------------------------------------------------
# Random numbers (Philox4x64-10, Box-Muller)
# --------------------------------------------------------------------------

def test_philox_matches_numpy():
    """numpy's Philox bit generator is Philox4x64-10; it increments the
    counter before each block, so its first block is our block at ctr+1."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        key = [int(x) for x in rng.integers(0, 2 ** 63, 2, dtype=np.int64)]
        ctr = [int(x) for x in rng.integers(0, 2 ** 62, 4, dtype=np.int64)]
        bg = np.random.Philox(key=key, counter=ctr)
        ref = bg.random_raw(4)
        c1 = list(ctr)
        c1[0] += 1
        out = O.philox4x64_10(c1, key)
        assert (out == ref).all()


def test_pair_random_moments():
    n = 40000
    G = np.empty((n, 3))
    U = np.empty(n)
    for k in range(n):
        G[k], U[k] = O.pair_randoms(12345, k // 200, k % 200, 1000 + k)
    assert np.abs(G.mean(axis=0)).max() < 0.03
    assert np.abs(G.var(axis=0) - 1.0).max() < 0.03
    corr = np.corrcoef(np.column_stack([G, U]).T)
    assert np.abs(corr - np.eye(4)).max() < 0.03
    assert stats.kstest(U, "uniform").pvalue > 1e-3
    for k in range(3):
        assert stats.kstest(G[:, k], "norm").pvalue > 1e-3
    assert ((U > 0) & (U < 1)).all()


# --------------------------------------------------------------------------
# One fluctuation/dissipation pair update (Sections 3.2-3.3)
# --------------------------------------------------------------------------

def _random_pair(rng, P, small_eps=False):
    r = rng.normal(size=3)
    r *= rng.uniform(0.3, 0.95) * P.h / np.linalg.norm(r)
    p_i, p_j = rng.normal(size=3), rng.normal(size=3)
    if small_eps:
        e_i, e_j = rng.uniform(1e-3, 0.2, 2)
    else:
        e_i, e_j = rng.uniform(0.5, 20.0, 2)
    return r, p_i, p_j, e_i, e_j


@pytest.mark.parametrize("scheme", [O.SCHEME_SSA, O.SCHEME_AMS, O.SCHEME_EMS])
def test_fd_pair_conserves_momentum_and_energy(scheme):
    rng = np.random.default_rng(scheme + 10)
    P = small_cfg(K=3.0, scheme=scheme).params()
    n_acc = 0
    for k in range(400):
        r, p_i, p_j, e_i, e_j = _random_pair(rng, P, small_eps=(k % 2 == 0))
        G = rng.normal(size=3)
        U = rng.uniform()
        d, margin, neg, pi, pj, ei, ej = O.fd_pair(P, r, 1.0, 1.1, p_i, p_j, e_i, e_j, 0.3, G, U)
        E0 = e_i + e_j + (p_i @ p_i + p_j @ p_j) / (2 * P.m)
        E1 = ei + ej + (pi @ pi + pj @ pj) / (2 * P.m)
        assert abs(E1 - E0) <= 8 * np.spacing(E0)
        assert np.abs((pi + pj) - (p_i + p_j)).max() <= 4 * np.spacing(np.abs(p_i + p_j).max() + 1)
        # the energy change is shared equally (one rounding of each sum)
        assert abs((ei - e_i) - (ej - e_j)) <= 2 * np.spacing(max(e_i, e_j, ei, ej))
        if d == O.ACCEPT:
            n_acc += 1
        else:
            assert (pi == p_i).all() and ei == e_i and ej == e_j
        if scheme != O.SCHEME_SSA:
            assert ei > 0 and ej > 0
    assert n_acc > 100


def test_ams_is_ssa_with_the_energy_bound_and_ems_shares_its_proposal():
    """Section 3.3.3: AMS takes the SSA move unless an internal energy would
    become non-positive, and then keeps the old state; EMS uses the same
    proposal, so every move it accepts equals AMS's, and it rejects every
    move AMS rejects (the energy bound comes first)."""
    rng = np.random.default_rng(21)
    kw = dict(K=1.5)
    Pssa, Pams, Pems = (small_cfg(scheme=sc, **kw).params() for sc in (O.SCHEME_SSA, O.SCHEME_AMS, O.SCHEME_EMS))
    seen = {"ams_reject": 0, "ems_metropolis": 0, "accept": 0}
    for k in range(600):
        r, p_i, p_j, e_i, e_j = _random_pair(rng, Pssa, small_eps=(k % 3 != 0))
        p_i, p_j = (0.05 * p_i, 0.05 * p_j) if k % 2 else (p_i, p_j)
        G, U, dt = rng.normal(size=3), rng.uniform(), rng.choice([0.05, 0.5, 3.0])
        args = (r, 1.0, 0.95, p_i, p_j, e_i, e_j, dt, G, U)
        ds, _, neg, *xs = O.fd_pair(Pssa, *args)
        da, _, _, *xa = O.fd_pair(Pams, *args)
        de, _, _, *xe = O.fd_pair(Pems, *args)
        assert ds == O.ACCEPT
        ssa_ok = xs[2] > 0 and xs[3] > 0
        if ssa_ok:
            assert da == O.ACCEPT
            for a, b in zip(xa, xs):
                assert np.array_equal(a, b)
        else:
            assert da == O.REJECT_BOUND and neg == 1
            assert (xa[0] == p_i).all() and (xa[1] == p_j).all() and xa[2] == e_i and xa[3] == e_j
            seen["ams_reject"] += 1
        if de == O.ACCEPT:
            for a, b in zip(xe, xa):
                assert np.array_equal(a, b)
            seen["accept"] += 1
        elif de == O.REJECT_BOUND:
            assert da == O.REJECT_BOUND
        else:
            assert de == O.REJECT_METROPOLIS and da == O.ACCEPT
            seen["ems_metropolis"] += 1
    assert min(seen.values()) > 10, seen


def test_ssa_flags_negative_energy_and_bound_rejects():
    rng = np.random.default_rng(3)
    seen_neg = seen_bound = 0
    for scheme in (O.SCHEME_SSA, O.SCHEME_AMS):
        P = small_cfg(K=1.5, scheme=scheme).params()
        for k in range(300):
            r, p_i, p_j, _, _ = _random_pair(rng, P)
            # nearly at rest with tiny internal energies: the noise can take
            # more kinetic energy than the pair's internal energies hold
            p_i, p_j = 1e-3 * p_i, 1e-3 * p_j
            d, margin, neg, pi, pj, ei, ej = O.fd_pair(P, r, 1.0, 1.0, p_i, p_j, 1e-3, 2e-3, 5.0,
                                                       rng.normal(size=3), 0.5)
            if scheme == O.SCHEME_SSA:
                seen_neg += neg
                assert d == O.ACCEPT
            else:
                seen_bound += d == O.REJECT_BOUND
                assert neg == 0
    assert seen_neg > 0 and seen_bound > 0


def test_ems_reverse_ratio_antisymmetric():
    """Detailed balance of the Metropolis ratio: for the move v -> v' with
    noise G, the reverse move v' -> v uses the noise G' that maps v' back to
    v, and its ratio is exactly -a (Eq. metropolis-ratio)."""
    rng = np.random.default_rng(9)
    kw = dict(N=1000, L=10.0, K=2.0, eta=1.3, zeta=0.4)
    P = O.Config(scheme=O.SCHEME_EMS, **kw).params()
    Pssa = O.Config(scheme=O.SCHEME_SSA, **kw).params()
    m = P.m
    rho_i, rho_j, dt = 0.9, 1.05, 0.2

    def proposal(r, pa, pb, ea, eb, g):
        """The move of Eq. (proposal) without accept/reject (SSA)."""
        out = O.fd_pair(Pssa, r, rho_i, rho_j, pa, pb, ea, eb, dt, g, 0.5)
        return out[3], out[4], out[5], out[6]

    checked = 0
    for _ in range(200):
        r, p_i, p_j, e_i, e_j = _random_pair(rng, P)
        G = rng.normal(size=3)
        d, a_minus_lnU, _, _, _, _, _ = O.fd_pair(P, r, rho_i, rho_j, p_i, p_j, e_i, e_j, dt, G, 0.5)
        if d == O.REJECT_BOUND:
            continue
        a = a_minus_lnU + np.log(0.5)
        pi, pj, ei, ej = proposal(r, p_i, p_j, e_i, e_j, G)
        # the reverse noise G' solves v = A(v') v' + B(v') G'; A(v') v' and
        # the columns of B(v') are read off the proposal map at v'
        v = (p_i - p_j) / m
        e = r / np.linalg.norm(r)
        rel = lambda out: (out[0] - out[1]) / m
        Av = rel(proposal(r, pi, pj, ei, ej, np.zeros(3)))
        Bpar = np.dot(rel(proposal(r, pi, pj, ei, ej, e)) - Av, e)
        t = np.cross(e, [1.0, 0.0, 0.0])
        t /= np.linalg.norm(t)
        Bperp = np.dot(rel(proposal(r, pi, pj, ei, ej, t)) - Av, t)
        w = v - Av
        wpar = np.dot(w, e) * e
        Gr = wpar / Bpar + (w - wpar) / Bperp
        d2, arev_minus, _, _, _, _, _ = O.fd_pair(P, r, rho_i, rho_j, pi, pj, ei, ej, dt, Gr, 0.5)
        assert d2 != O.REJECT_BOUND
        arev = arev_minus + np.log(0.5)
        assert abs(a + arev) < 1e-7 * (1 + abs(a)), (a, arev)
        checked += 1
    assert checked > 50


# --------------------------------------------------------------------------
# Pair colouring of the sweep
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,n_c", [(12, None), (16, (4, 6, 4))])  # the default grid; a coarser one
def test_colouring_is_conflict_free(n, n_c):
    w = Workload(n=n, jitter=0.2, seed=8)
    q, p, eps = lattice_state(w)
    P = O.Config(N=w.N, L=w.L, K=w.K, n_c=n_c).params()
    if n_c is not None:
        assert tuple(P.n_c[:]) == n_c
    s, _, _, st, recs = O.fd_sweep(P, q, p, eps, 0.005, 1, 0, records=True)
    assert s == O.OK
    # the pair set is exactly the brute-force neighbour set
    nb = O.neighbour_counts(P, q)
    assert st.n_pairs == nb.sum() // 2 == len(recs)
    cells = O.cells(P, q)
    n_c = np.array(P.n_c[:])
    for rec in recs[:: max(1, len(recs) // 3000)]:
        o = np.array([rec["owner"] % n_c[0], (rec["owner"] // n_c[0]) % n_c[1], rec["owner"] // (n_c[0] * n_c[1])])
        for pid in (rec["id_i"], rec["id_j"]):
            off = (cells[pid] - o) % n_c
            assert ((off == 0) | (off == 1)).all()
        assert rec["colour"] == (o[0] & 1) | ((o[1] & 1) << 1) | ((o[2] & 1) << 2)
    # sweep order: colour, owner, then inside the owner's block by
    # (rank difference, lower rank), ranks of ids among the block's particles
    rank_i = np.empty(len(recs), dtype=np.int64)
    rank_j = np.empty(len(recs), dtype=np.int64)
    for own in np.unique(recs["owner"]):
        sel = np.nonzero(recs["owner"] == own)[0]
        o = np.array([own % n_c[0], (own // n_c[0]) % n_c[1], own // (n_c[0] * n_c[1])])
        members = np.nonzero((((cells - o) % n_c) <= 1).all(axis=1))[0]
        rank_i[sel] = np.searchsorted(members, recs["id_i"][sel])
        rank_j[sel] = np.searchsorted(members, recs["id_j"][sel])
    assert (rank_i < rank_j).all()
    key = np.stack([recs["colour"], recs["owner"], rank_j - rank_i, rank_i])
    assert (np.lexsort(key[::-1]) == np.arange(len(recs))).all()
    # within one colour, different owners touch disjoint particles
    for c in range(8):
        sel = recs[recs["colour"] == c]
        owner_of = {}
        for rec in sel:
            for pid in (int(rec["id_i"]), int(rec["id_j"])):
                assert owner_of.setdefault(pid, rec["owner"]) == rec["owner"]


def test_owner_rule():
    P = small_cfg(n=12).params()  # n_c = 4
    # adjacent on every axis: the lower cell per axis (periodically), whatever the ids
    for pid in (0, 1, 12345):
        s, o = O.pair_owner(P, [0, 3, 1], [3, 0, 2], pid)
        assert s == O.OK and list(o) == [3, 3, 1]
    s, o = O.pair_owner(P, [0, 0, 0], [2, 0, 0])
    assert s == O.ERR_NOT_ADJACENT
    # coinciding on an axis: the block starting at the coordinate or one cell
    # below, as the lower id's bit for that axis says
    for pid in range(64):
        bits = O.owner_bits(pid)
        s, o = O.pair_owner(P, [2, 1, 0], [2, 2, 3], pid)  # x equal, y +1, z -1 periodically
        assert s == O.OK and list(o) == [(2 - (bits & 1)) % 4, 1, 3]
        s, o = O.pair_owner(P, [0, 3, 1], [0, 3, 1], pid)  # the same cell: any of its 8 blocks
        assert list(o) == [(0 - (bits & 1)) % 4, (3 - ((bits >> 1) & 1)) % 4, (1 - ((bits >> 2) & 1)) % 4]
    # exhaustively: every adjacent pair of cells, for several ids, is owned by
    # a block that contains both cells
    rng = np.random.default_rng(0)
    ids = rng.integers(0, 2**31 - 1, size=6)
    offs = [(x, y, z) for x in (-1, 0, 1) for y in (-1, 0, 1) for z in (-1, 0, 1)]
    for a in np.ndindex(4, 4, 4):
        for off in offs:
            b = [(a[k] + off[k]) % 4 for k in range(3)]
            for pid in ids:
                s, o = O.pair_owner(P, list(a), b, int(pid))
                assert s == O.OK
                for c in (a, b):
                    assert all((c[k] - o[k]) % 4 in (0, 1) for k in range(3))


def test_owner_bits_spread_over_the_eight_blocks():
    """The owner bits of consecutive ids (lattice neighbours get nearby ids)
    hit all eight patterns evenly, so a particle's same-cell pairs spread over
    the eight colours."""
    n = 1 << 15
    bits = np.array([O.owner_bits(k) for k in range(n)])
    assert bits.min() == 0 and bits.max() == 7
    counts = np.bincount(bits, minlength=8)
    assert np.abs(counts - n / 8).max() < 5 * np.sqrt(n / 8)
    # no strong correlation between an id and the next one
    same = np.mean(bits[1:] == bits[:-1])
    assert abs(same - 1 / 8) < 0.02


# --------------------------------------------------------------------------
# Statistical pins of the Metropolis scheme
# --------------------------------------------------------------------------

def _two_particle_chain(K, scheme, dt, nsteps, eta=1.0, e0=(0.4, 0.9), seed=5, counts=None):
    """FD-only chain of one pair; |v|^2 after every sweep.  ``counts``, a
    dict, receives the pair updates and acceptances."""
    cfg = O.Config(N=2, L=10.0, K=K, scheme=scheme, eta=eta)
    P = cfg.params()
    q = np.array([[5.0, 5.0, 5.0], [5.9, 5.3, 5.0]])
    p = np.array([[0.5, -0.2, 0.1], [-0.5, 0.2, -0.1]])
    eps = np.array(e0)
    v2 = np.empty(nsteps)
    step = n_pairs = n_accept = 0
    for n in range(nsteps):
        s, p, eps, st, _ = O.fd_sweep(P, q, p, eps, dt, seed, step)
        step += 1
        n_pairs += st.n_pairs
        n_accept += st.n_accept
        v = (p[0] - p[1]) / P.m
        v2[n] = v @ v
    if counts is not None:
        counts.update(n_pairs=n_pairs, n_accept=n_accept)
    return P, p, eps, v2


def test_ems_samples_pair_invariant_measure():
    """Two particles, fluctuation/dissipation only: the relative velocity must
    be distributed as nu(v) ~ exp((S_i+S_j)/kB)/(T_i T_j) (Eq. minv-vij) with
    eps_k(v) from Eq. (energies-vij).  For the ideal gas this is
    (eps_i(v) eps_j(v))^(C_K/kB - 1) on {eps_i, eps_j > 0}."""
    K = 2.0
    P, p, eps, v2 = _two_particle_chain(K, O.SCHEME_EMS, dt=3.0, nsteps=60000)
    C_K = 1.5 * (K - 1.0)
    m = P.m
    # the pair energy budget is conserved: c_k = eps_k + m |v|^2 / 8
    ck = eps + m * v2[-1] / 8.0
    smax = 8.0 * ck.min() / m
    dens = lambda s: np.sqrt(s) * np.prod([(c - m * s / 8.0) ** (C_K - 1) for c in ck], axis=0)
    Z = integrate.quad(dens, 0, smax)[0]
    samples = v2[5000::5]
    edges = np.linspace(0, smax, 21)
    expect = np.array([integrate.quad(dens, a, b)[0] / Z for a, b in zip(edges[:-1], edges[1:])])
    counts, _ = np.histogram(samples, edges)
    chi2 = (((counts - len(samples) * expect) ** 2) / (len(samples) * expect + 1e-12))[expect > 1e-4].sum()
    # ~19 degrees of freedom; residual autocorrelation inflates chi2 a little
    assert chi2 < 80, chi2


def test_ams_small_dt_samples_pair_invariant_measure():
    """At small time steps the proposal alone (AMS, which equals SSA when no
    energy goes negative) is a consistent discretisation of Eq.
    (fd-effective), whose invariant measure is Eq. (minv-vij) only if gamma
    and sigma obey the fluctuation/dissipation relation of Eq.
    (sdpd-gamma-sigma).  A Metropolis step would hide a wrong gamma; the
    unadjusted scheme does not."""
    K = 6.0
    P, p, eps, v2 = _two_particle_chain(K, O.SCHEME_AMS, dt=0.01, nsteps=150000, e0=(2.0, 4.0))
    C_K = 1.5 * (K - 1.0)
    m = P.m
    ck = eps + m * v2[-1] / 8.0
    smax = 8.0 * ck.min() / m
    dens = lambda s: np.sqrt(s) * np.prod([(c - m * s / 8.0) ** (C_K - 1) for c in ck], axis=0)
    Z = integrate.quad(dens, 0, smax)[0]
    mean_exact = integrate.quad(lambda s: s * dens(s), 0, smax)[0] / Z
    samples = v2[10000:]
    # correlation time is ~10 steps: compare the mean with a batch-means error
    batches = samples[: len(samples) // 50 * 50].reshape(50, -1).mean(axis=1)
    se = batches.std(ddof=1) / np.sqrt(len(batches))
    assert abs(samples.mean() - mean_exact) < 4 * se + 0.01 * mean_exact, (samples.mean(), mean_exact, se)


def test_large_heat_capacity_limit():
    """C_K -> infinity (d -> 0): energies barely move, the proposal is the
    exact OU step of Eq. (fd-effective), EMS accepts essentially every move
    and the relative velocity has variance 2 kB T / m per component."""
    K = 1e7
    e0 = (1.5e7, 1.5e7)  # T = 1
    n = {}
    P, p, eps, v2 = _two_particle_chain(K, O.SCHEME_EMS, dt=5.0, nsteps=20000, e0=e0, counts=n)
    assert abs(v2[1000:].mean() / 3.0 - 2.0) < 0.1
    assert n["n_pairs"] == 20000 and n["n_accept"] >= 0.999 * n["n_pairs"], n
    # at an ordinary heat capacity and the same step the ratio does reject
    m = {}
    _two_particle_chain(2.0, O.SCHEME_EMS, dt=5.0, nsteps=2000, counts=m)
    assert m["n_accept"] < 0.99 * m["n_pairs"], m


@pytest.mark.slow
def test_fd_only_energy_distribution_is_gamma():
    """N=1000, fluctuation/dissipation only, EMS: the internal energies follow
    the Gamma law of Eq. (dist-analytic) with beta = 1/T_eq, and the total
    energy is conserved to rounding."""
    w = Workload(n=10, K=5.0, kT=1.0, jitter=0.2, seed=21)
    q, p, eps = lattice_state(w)
    P = O.Config(N=w.N, L=w.L, K=w.K, scheme=O.SCHEME_EMS).params()
    E0 = O.observables(P, p, eps)["E"]
    C_K = 1.5 * (w.K - 1)
    s, q1, p, eps, st, step = O.run(P, q, p, eps, 0.5, 40, seed=3, fd_only=True)
    samples = []
    for _ in range(60):
        s, q1, p, eps, st, step = O.run(P, q, p, eps, 0.5, 2, seed=3, fd_only=True, fd_step=step)
        samples.append(eps.copy())
    assert s == O.OK
    E1 = O.observables(P, p, eps)["E"]
    assert abs(E1 - E0) < 1e-10 * E0
    T_eq = E0 / (1.5 * (w.N - 1) + w.N * C_K)
    x = np.concatenate(samples)
    assert abs(x.mean() / (C_K * T_eq) - 1.0) < 0.02
    # quadratic error of Eq. (error-dist) on the paper's 150 bins over [0.1, 20] kT
    edges = np.linspace(0.1 * T_eq, 20 * T_eq, 151)
    hist, _ = np.histogram(x, edges, density=False)
    width = edges[1] - edges[0]
    nu = hist / (len(x) * width)
    mid = 0.5 * (edges[:-1] + edges[1:])
    mu = stats.gamma.pdf(mid, a=C_K, scale=T_eq)
    err = np.sqrt(((nu - mu) ** 2).sum() / (mu ** 2).sum())
    assert err < 0.12, err
