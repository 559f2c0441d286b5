"""GPU path versus the FP64 oracle, element by element, on seeded inputs.

Tolerances (from the accuracy targets of the library):
  * cell indices, storage order, neighbour sets, pair colours and owners:
    bit-exact (float64 path; the predicate r^2 < h^2 is a fixed sequence of
    correctly rounded operations on both sides);
  * float64 path: rho within 1e-12 relative, F within 1e-12 of max|F|;
    accept/reject decisions equal (no flip);
  * mixed path (float32 pair arithmetic, float64 energies, float64-decided
    Metropolis tests): rho within 1e-5 of max rho, F within 1e-5 of max|F|;
    sweep energy conserved to float64 rounding;
  * trajectories: positions within 1e-6 a after 10 steps (both paths).
"""
import numpy as np
import pytest

import oracle as O
from paper_1707_04232_gb300.inputs import Workload, lattice_state, random_box_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1707_04232_gb300 import sdpd  # noqa: E402

DT = 0.005


def system(kind: str):
    """(q, p, eps, L, K) of a named test system."""
    if kind == "lattice1000":
        w = Workload(n=10, K=100.0)
        q, p, e = lattice_state(w)
        return q, p, e, (w.L,) * 3, w.K
    if kind == "lattice_cold_K5":
        w = Workload(n=10, K=5.0, kT=0.1, jitter=0.05, seed=4)
        q, p, e = lattice_state(w)
        return q, p, e, (w.L,) * 3, w.K
    if kind == "random_rect":  # ragged N, rectangular box, disordered fluid
        L = (12.5, 15.0, 17.3)
        N = int(round(L[0] * L[1] * L[2]))
        C_K = 1.5 * (20.0 - 1.0)
        q, p, e = random_box_state(N, 1.0, 1.0, 1.0, C_K, seed=9)
        q = q * np.array(L)
        q = np.where(q >= np.array(L), 0.0, q)
        e = e * (0.5 + np.random.default_rng(3).random(N))
        return q, p, e, L, 20.0
    if kind == "lattice32k":
        w = Workload(n=32, K=100.0, seed=1)
        q, p, e = lattice_state(w)
        return q, p, e, (w.L,) * 3, w.K
    raise KeyError(kind)


def oparams(N, L, K, kernel=O.KERNEL_LUCY, scheme=O.SCHEME_EMS):
    return O.Config(N=N, L=tuple(L), K=K, kernel=kernel, scheme=scheme).params()


def gpu(N, L, K, precision=sdpd.FP64, kernel=sdpd.KERNEL_LUCY, scheme=sdpd.SCHEME_EMS, **kw):
    return sdpd.SDPD(N, L, m=1.0, h=2.5, K=K, precision=precision, kernel=kernel, scheme=scheme, **kw)


def min_image_err(a, b, L):
    L = np.asarray(L)
    d = (a - b + 0.5 * L) % L - 0.5 * L
    return np.abs(d).max()


# --------------------------------------------------------------------------
# Binning, order, neighbour sets
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["lattice1000", "random_rect", "lattice32k"])
def test_cells_order_and_neighbours_bit_exact(kind):
    q, p, e, L, K = system(kind)
    N = len(e)
    s = gpu(N, L, K)
    s.set_state(q, p, e)
    P = oparams(N, L, K)
    assert (s.cells() == O.cells(P, q)).all()
    assert (s.order() == O.sorted_order(P, q)).all()
    assert (s.neighbour_counts() == O.neighbour_counts(P, q)).all()


# --------------------------------------------------------------------------
# Density (Eq. sdpd-rho-v) and conservative force (Eq. cons-forces)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [sdpd.KERNEL_LUCY, sdpd.KERNEL_CUBIC])
@pytest.mark.parametrize("kind", ["lattice1000", "random_rect", "lattice32k"])
def test_density_and_force_fp64(kind, kernel):
    q, p, e, L, K = system(kind)
    N = len(e)
    s = gpu(N, L, K, kernel=kernel)
    s.set_state(q, p, e)
    P = oparams(N, L, K, kernel=kernel)
    rho = O.density(P, q)
    assert np.abs(s.density() - rho).max() <= 1e-12 * rho.max()
    f = O.forces(P, q, rho, e)
    assert np.abs(s.forces() - f).max() <= 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("kernel", [sdpd.KERNEL_LUCY, sdpd.KERNEL_CUBIC])
@pytest.mark.parametrize("kind", ["lattice1000", "random_rect", "lattice32k"])
def test_density_and_force_mixed(kind, kernel):
    q, p, e, L, K = system(kind)
    N = len(e)
    s = gpu(N, L, K, precision=sdpd.MIXED, kernel=kernel)
    s.set_state(q, p, e)
    P = oparams(N, L, K, kernel=kernel)
    rho = O.density(P, q)
    assert np.abs(s.density() - rho).max() <= 1e-5 * rho.max()
    f = O.forces(P, q, rho, e)
    assert np.abs(s.forces() - f).max() <= 1e-5 * np.abs(f).max()


# --------------------------------------------------------------------------
# One fluctuation/dissipation sweep (Sections 3.2-3.3)
# --------------------------------------------------------------------------

def check_sweep_against_oracle(recs_g, recs_o, tol_flip=0.0):
    """Pair set, colours, owners and per-particle order equal to the
    oracle's; returns the decision flips as (pair, oracle margin, GPU
    margin), each of which must have |oracle margin| < tol_flip (none at the
    default 0: every decision equal)."""
    key = lambda r: (int(r["id_i"]), int(r["id_j"]))
    go = {key(r): r for r in recs_g}
    oo = {key(r): (k, r) for k, r in enumerate(recs_o)}
    assert set(go) == set(oo), "pair sets differ"
    flips = []
    for k, (pos, ro) in oo.items():
        rg = go[k]
        assert rg["colour"] == ro["colour"] and rg["owner"] == ro["owner"]
        if rg["decision"] != ro["decision"]:
            flips.append((k, ro["margin"], rg["margin"]))
    for k, mo, mg in flips:
        assert abs(mo) < tol_flip, "decision flip with margin %g at %s" % (mo, k)
    # the GPU schedule keeps every particle's pairs in the oracle's order
    pos_of = {k: pos for k, (pos, _) in oo.items()}
    per_particle = {}
    for r in recs_g:
        for pid in (int(r["id_i"]), int(r["id_j"])):
            per_particle.setdefault(pid, []).append((int(r["colour"]), int(r["level"]), pos_of[key(r)]))
    for pid, lst in per_particle.items():
        lst.sort()
        seq = [t[2] for t in lst]
        assert seq == sorted(seq), "particle %d: schedule breaks the sweep order" % pid
    return flips


_oracle_sweeps = {}


def oracle_sweep(q, p, e, L, K, scheme, kernel, dt, seed):
    """The oracle's sweep of a state, kept for the other launch shapes of
    the same case."""
    key = (q.tobytes(), p.tobytes(), e.tobytes(), tuple(L), K, scheme, kernel, dt, seed)
    if key not in _oracle_sweeps:
        P = oparams(len(e), L, K, kernel=kernel, scheme=scheme)
        _oracle_sweeps.clear()
        _oracle_sweeps[key] = O.fd_sweep(P, q, p, e, dt, seed, 0, records=True)
    return _oracle_sweeps[key]


def sweep_fp64_vs_oracle(q, p, e, L, K, scheme, kernel=sdpd.KERNEL_LUCY, dt=DT, seed=77, shapes=None):
    """One float64 sweep on the GPU and in the oracle from the same state:
    every decision equal, momenta and energies within 1e-10 (relative to
    the largest).  Returns the GPU pair records."""
    N = len(e)
    s = gpu(N, L, K, scheme=scheme, kernel=kernel, fd_only=True, debug=True)
    if shapes is not None:
        s.set_tuning(*shapes)
    s.set_state(q, p, e)
    s.step(dt, 1, seed=seed)
    qg, pg, eg = s.get_state()
    recs = s.pair_records()
    st, po, eo, stats, recs_o = oracle_sweep(q, p, e, L, K, scheme, kernel, dt, seed)
    flips = check_sweep_against_oracle(recs, recs_o)
    assert flips == []
    obs = s.observables(check=False)
    assert obs["n_pairs"] == stats.n_pairs
    assert obs["n_accept"] == stats.n_accept
    assert np.abs(pg - po).max() <= 1e-10 * max(1.0, np.abs(po).max())
    assert np.abs(eg - eo).max() <= 1e-10 * eo.max()
    assert (qg == q).all()  # the sweep never moves particles
    return recs


@pytest.mark.parametrize("scheme", [sdpd.SCHEME_EMS, sdpd.SCHEME_AMS, sdpd.SCHEME_SSA])
@pytest.mark.parametrize("kind,kernel", [("lattice1000", sdpd.KERNEL_LUCY), ("random_rect", sdpd.KERNEL_LUCY),
                                         ("lattice_cold_K5", sdpd.KERNEL_LUCY),
                                         ("random_rect", sdpd.KERNEL_CUBIC)])
def test_fd_sweep_fp64_matches_oracle(kind, kernel, scheme):
    q, p, e, L, K = system(kind)
    dt = 0.05 if kind == "lattice_cold_K5" else DT
    sweep_fp64_vs_oracle(q, p, e, L, K, scheme, kernel=kernel, dt=dt)


@pytest.mark.parametrize("shapes", [(1, 128), (3, 32), (0, 128)])
@pytest.mark.parametrize("scheme", [sdpd.SCHEME_EMS, sdpd.SCHEME_AMS, sdpd.SCHEME_SSA])
def test_fd_sweep_fp64_matches_oracle_many_blocks(scheme, shapes):
    """32^3 lattice: 12 cells per axis, 216 blocks per colour, several
    blocks per warp or warp per block, taken from the atomic queue deepest
    first -- the launch shapes of the large systems, against the oracle's
    sequential sweep."""
    q, p, e, L, K = system("lattice32k")
    sweep_fp64_vs_oracle(q, p, e, L, K, scheme, shapes=shapes)


def test_fd_sweep_fp64_matches_oracle_deep_blocks():
    """A disordered fluid of 40^3 particles (uniform random positions, so
    local density fluctuates): its deepest blocks run more than 100
    dependency levels (101 in the oracle's order), against the oracle's
    sequential sweep."""
    L = (40.0,) * 3
    N = 40 ** 3
    q, p, e = random_box_state(N, 1.0, 1.0, 1.0, 1.5 * 99.0, seed=21)
    q = q * 40.0
    q = np.where(q >= 40.0, 0.0, q)
    recs = sweep_fp64_vs_oracle(q, p, e, L, 100.0, sdpd.SCHEME_EMS, shapes=(1, 128))
    assert recs["level"].max() >= 100


def test_fd_sweep_mixed_statistics():
    """Mixed precision: same pair set and colouring, same decisions except
    near ties, energy conserved by every sweep to float64 rounding (the
    energy changes are float64 sums of exact products of the float32
    momenta)."""
    q, p, e, L, K = system("lattice_cold_K5")
    N = len(e)
    s = gpu(N, L, K, precision=sdpd.MIXED, fd_only=True, debug=True)
    s.set_state(q, p, e)
    E0 = s.observables()["E"]
    s.step(0.05, 1, seed=5)
    recs = s.pair_records()
    P = oparams(N, L, K)
    st, po, eo, stats, recs_o = O.fd_sweep(P, q, p, e, 0.05, 5, 0, records=True)
    flips = check_sweep_against_oracle(recs, recs_o, tol_flip=1e-4)
    assert len(flips) <= 2
    E1 = s.observables()["E"]
    assert abs(E1 - E0) < 1e-12 * abs(E0)


def test_mixed_records_do_not_change_the_sweep():
    """Kept pair records make every Metropolis test evaluate its float64
    ratio; without records only the near ties do.  Both runs must end in
    the same state bit for bit (the float32 error bound is never wrong)."""
    w = Workload(n=20, K=100.0, kT=1.0, seed=2)
    q, p, e = lattice_state(w)
    out = []
    for debug in (False, True):
        s = gpu(w.N, (w.L,) * 3, w.K, precision=sdpd.MIXED, fd_only=True, debug=debug)
        s.set_state(q, p, e)
        s.step(0.005, 3, seed=8)
        out.append(s.get_state())
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [20, 32])
@pytest.mark.parametrize("dt", [0.001, 0.005, 0.02])
def test_fd_sweep_mixed_metropolis_ratio_accuracy(dt, n):
    """Mixed EMS against the float64 path on the same state (n^3 lattice,
    K = 100, kT = 1).  The mixed path decides each Metropolis test in
    float64: its float32 estimate of a - ln U stays within the error bound
    that selects the float64 re-evaluation, and every decision follows the
    float64 margin.  The two paths differ only through the float32 proposal
    (coefficients and momenta), so decisions can differ only at near ties."""
    w = Workload(n=n, K=100.0, kT=1.0, seed=2)
    q, p, e = lattice_state(w)
    out = {}
    for prec in (sdpd.FP64, sdpd.MIXED):
        s = gpu(w.N, (w.L,) * 3, w.K, precision=prec, fd_only=True, debug=True)
        s.set_state(q, p, e)
        s.step(dt, 1, seed=3)
        r = s.pair_records()
        out[prec] = r[np.lexsort((r["id_j"], r["id_i"]))]
    a, b = out[sdpd.FP64], out[sdpd.MIXED]
    assert np.array_equal(a["id_i"], b["id_i"]) and np.array_equal(a["id_j"], b["id_j"])
    met = b["decision"] != 1
    # the float32 estimate is within its bound, and the decision is the float64 one
    assert (np.abs(b["margin_lo"] - b["margin"])[met] <= b["margin_tol"][met]).all()
    assert np.array_equal(b["decision"][met] == 2, b["margin"][met] < 0.0)
    assert b["margin_tol"][met].max() < 1e-3
    flip = a["decision"] != b["decision"]
    assert flip.mean() <= 1e-5
    assert (np.abs(a["margin"][flip]) < 1e-4).all(), a["margin"][flip]
    near = (np.abs(a["margin"]) < 0.05) & (a["decision"] != 1)
    assert near.sum() > 1000
    assert np.abs(a["margin"][near] - b["margin"][near]).max() < 1e-4


# --------------------------------------------------------------------------
# Full steps
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,scheme,theta,kernel", [("lattice1000", sdpd.SCHEME_EMS, 1, sdpd.KERNEL_LUCY),
                                                      ("lattice1000", sdpd.SCHEME_AMS, 1, sdpd.KERNEL_LUCY),
                                                      ("random_rect", sdpd.SCHEME_EMS, 1, sdpd.KERNEL_LUCY),
                                                      ("lattice1000", sdpd.SCHEME_EMS, 5, sdpd.KERNEL_LUCY),
                                                      ("lattice1000", sdpd.SCHEME_NONE, 1, sdpd.KERNEL_LUCY),
                                                      ("random_rect", sdpd.SCHEME_EMS, 1, sdpd.KERNEL_CUBIC)])
def test_trajectory_fp64_10_steps(kind, scheme, theta, kernel):
    q, p, e, L, K = system(kind)
    N = len(e)
    s = gpu(N, L, K, scheme=scheme, theta=theta, kernel=kernel)
    s.set_state(q, p, e)
    s.step(DT, 10, seed=3)
    qg, pg, eg = s.get_state()
    P = oparams(N, L, K, kernel=kernel, scheme=scheme)
    st, qo, po, eo, stats, nfd = O.run(P, q, p, e, DT, 10, seed=3, theta=theta)
    assert st == O.OK
    assert min_image_err(qg, qo, L) < 1e-6
    assert np.abs(pg - po).max() < 1e-6 * max(1.0, np.abs(po).max())
    assert np.abs(eg - eo).max() < 1e-6 * eo.max()
    obs = s.observables()
    assert obs["fd_step"] == nfd


def test_trajectory_fp64_32k_lattice_3_steps():
    """Full float64 steps (Verlet, schedule from the density pass's lists,
    EMS sweep) on the 32^3 lattice: 216 blocks per colour, blocks of up to
    216 particles whose owner groups take the enumeration several chunks,
    against the oracle's 3 steps."""
    q, p, e, L, K = system("lattice32k")
    N = len(e)
    s = gpu(N, L, K)
    s.set_state(q, p, e)
    s.step(DT, 3, seed=5)
    qg, pg, eg = s.get_state()
    obs = s.observables()
    assert s.big_blocks().sum() == 0
    P = oparams(N, L, K)
    st, qo, po, eo, stats, nfd = O.run(P, q, p, e, DT, 3, seed=5)
    assert st == O.OK
    assert obs["n_pairs"] == stats.n_pairs and obs["n_accept"] == stats.n_accept
    assert min_image_err(qg, qo, L) < 1e-9
    assert np.abs(pg - po).max() < 1e-9 * max(1.0, np.abs(po).max())
    assert np.abs(eg - eo).max() < 1e-9 * eo.max()


def test_mixed_sweep_never_rejects_where_the_bound_is_far():
    """AMS rejects a move only at the energy bound, which no pair comes near
    at K = 100, kT = 1 (eps ~ 150, changes ~ 1): the float64 path rejects
    nothing there, and neither may the mixed path.  A uniform within 2^-25
    of 1 rounds to 1 in float32; Box-Muller must still give a finite normal
    (it once gave NaN, rejected as a bound violation, ~4e-8 of the pairs).
    40 sweeps of the 64^3 lattice draw ~4e8 pairs."""
    w = Workload(n=64, K=100.0, kT=1.0, jitter=0.05, seed=0)
    q, p, e = lattice_state(w)
    s = gpu(w.N, (w.L,) * 3, w.K, precision=sdpd.MIXED, scheme=sdpd.SCHEME_AMS)
    s.set_state(q, p, e)
    s.step(DT, 40, seed=7)
    o = s.observables()
    assert o["status"] == sdpd.OK
    assert o["n_pairs"] > 3e8
    assert o["n_reject_bound"] == 0 and o["n_reject_metropolis"] == 0


def test_mts_sweeps_follow_the_step_count_not_the_call():
    """With theta = 5 a sweep follows every 5th Verlet step since
    set_state, however the steps are split over calls; the result equals the
    oracle's 10-step run."""
    q, p, e, L, K = system("lattice1000")
    N = len(e)
    a = gpu(N, L, K, theta=5)
    a.set_state(q, p, e)
    for part in (1, 3, 2, 4):
        a.step(DT, part, seed=3)
    b = gpu(N, L, K, theta=5)
    b.set_state(q, p, e)
    b.step(DT, 10, seed=3)
    x, y = a.get_state(), b.get_state()
    assert all((u == v).all() for u, v in zip(x, y))
    assert a.observables()["fd_step"] == 2


@pytest.mark.parametrize("precision", [sdpd.FP64, sdpd.MIXED])
def test_fd_only_sweeps_reuse_the_schedule(precision):
    """FD-only: positions never move, so the sweep schedule built for the
    first sweep serves the later ones; 4 sweeps match the oracle's (float64:
    within 1e-9; mixed: per observable)."""
    q, p, e, L, K = system("lattice_cold_K5")
    N = len(e)
    s = gpu(N, L, K, precision=precision, fd_only=True)
    s.set_state(q, p, e)
    s.reset_counters()
    l0 = s.kernel_launches
    s.step(0.2, 4, seed=5)
    assert s.kernel_launches - l0 == 5 + 4 * 9  # one schedule, four sweeps
    qg, pg, eg = s.get_state()
    P = oparams(N, L, K)
    st, qo, po, eo, stats, _ = O.run(P, q, p, e, 0.2, 4, seed=5, fd_only=True)
    if precision == sdpd.FP64:
        assert np.array_equal(qg, q)
    else:  # positions held in 32-bit fixed point: within one unit L / 2^32
        assert min_image_err(qg, q, L) <= max(L) * 2.0 ** -32
    if precision == sdpd.FP64:
        assert np.abs(pg - po).max() < 1e-9 * np.abs(po).max()
        assert np.abs(eg - eo).max() < 1e-9 * eo.max()
    else:
        o_g, o_o = s.observables(), O.observables(P, po, eo)
        assert abs(o_g["E"] - o_o["E"]) < 1e-6 * abs(o_o["E"])
        assert abs(o_g["T_int"] - o_o["T_int"]) < 1e-3 * o_o["T_int"]


@pytest.mark.parametrize("precision", [sdpd.FP64, sdpd.MIXED])
def test_energy_histogram_is_exact(precision):
    q, p, e, L, K = system("random_rect")
    N = len(e)
    s = gpu(N, L, K, precision=precision, fd_only=True)
    s.set_state(q, p, e)
    s.step(0.1, 3, seed=1)
    _, _, eg = s.get_state()
    lo, hi, nb, scale = 0.1, 20.0, 150, 1.0 / 3.0
    got = s.energy_histogram(lo, hi, nb, scale).cpu().numpy()
    x = eg * scale
    w = (hi - lo) / nb
    ref = np.zeros(nb + 2, dtype=np.int64)
    under, over = x < lo, ~(x < hi)
    ref[nb], ref[nb + 1] = under.sum(), over.sum()
    inside = ~(under | over)
    b = np.minimum(np.floor((x[inside] - lo) / w).astype(np.int64), nb - 1)
    np.add.at(ref, b, 1)
    assert np.array_equal(got, ref)
    got2 = s.energy_histogram(lo, hi, nb, scale, counts=torch.as_tensor(got, device="cuda"))
    assert np.array_equal(got2.cpu().numpy(), 2 * ref)
    with pytest.raises(sdpd.SDPDError):
        s.energy_histogram(1.0, 1.0, 10)


@pytest.mark.parametrize("kind", ["lattice1000", "random_rect"])
def test_trajectory_mixed_verlet_10_steps(kind):
    """Deterministic part (Velocity Verlet only): float32 pair arithmetic and
    fixed-point positions stay within 1e-6 a of the float64 oracle after 10
    steps (measured: 3e-8 a on the lattice, 5e-8 a in the random fluid)."""
    q, p, e, L, K = system(kind)
    N = len(e)
    s = gpu(N, L, K, precision=sdpd.MIXED, scheme=sdpd.SCHEME_NONE)
    s.set_state(q, p, e)
    s.step(DT, 10, seed=3)
    qg, pg, eg = s.get_state()
    P = oparams(N, L, K, scheme=O.SCHEME_NONE)
    st, qo, po, eo, stats, _ = O.run(P, q, p, e, DT, 10, seed=3)
    assert min_image_err(qg, qo, L) < 1e-6
    assert np.abs(pg - po).max() < 1e-5 * np.abs(po).max()
    assert np.abs(eg - eo).max() < 1e-6 * eo.max()


@pytest.mark.parametrize("kind", ["lattice1000", "random_rect"])
def test_trajectory_mixed_ems_10_steps(kind):
    """Full steps with the Metropolis sweep against the float64 oracle.  The
    mixed path decides every Metropolis test in float64, for its float32
    proposal; a decision can differ from the oracle's only where the two
    proposals move the margin a - ln U across zero (margins within ~1e-4,
    about 2e-7 of the decisions: ~0.1 expected over these 10 sweeps).  With
    every decision equal, every particle stays within 1e-6 a."""
    q, p, e, L, K = system(kind)
    N = len(e)
    s = gpu(N, L, K, precision=sdpd.MIXED)
    s.set_state(q, p, e)
    s.step(DT, 10, seed=3)
    qg, pg, eg = s.get_state()
    P = oparams(N, L, K)
    st, qo, po, eo, stats, _ = O.run(P, q, p, e, DT, 10, seed=3)
    o_g = s.observables()
    assert o_g["n_pairs"] == stats.n_pairs
    assert o_g["n_accept"] == stats.n_accept, "decisions differ from the oracle's"
    assert min_image_err(qg, qo, L) < 1e-6
    assert np.abs(pg - po).max() < 1e-5 * np.abs(po).max()
    assert np.abs(eg - eo).max() < 1e-6 * eo.max()
    o_o = O.observables(P, po, eo)
    assert abs(o_g["E"] - o_o["E"]) < 1e-7 * abs(o_o["E"])
    assert abs(o_g["T_kin"] - o_o["T_kin"]) < 1e-5 * o_o["T_kin"]
    assert abs(o_g["T_int"] - o_o["T_int"]) < 1e-7 * o_o["T_int"]
    # total momentum: every accepted pair update rounds two float32 sums per
    # component (p_i + dp, p_j - dp), an unbiased error of std <= 2^-24 |p| / sqrt(3)
    # each; the float64 oracle conserves it to rounding.  Five standard
    # deviations of that random walk:
    p_rms = np.sqrt(np.mean(po ** 2))
    tol = 5.0 * np.sqrt(2.0 * o_g["n_accept"]) * 2.0 ** -24 * p_rms / np.sqrt(3.0)
    assert np.abs(o_g["P"] - o_o["P"]).max() < tol, (np.abs(o_g["P"] - o_o["P"]).max(), tol)


# --------------------------------------------------------------------------
# Invariants, restart, edge cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [sdpd.FP64, sdpd.MIXED])
def test_fd_only_conserves_energy_and_momentum(precision):
    q, p, e, L, K = system("lattice_cold_K5")
    N = len(e)
    s = gpu(N, L, K, precision=precision, fd_only=True)
    s.set_state(q, p, e)
    o0 = s.observables()
    s.step(0.1, 20, seed=1)
    o1 = s.observables()
    # float64 energies and float64 energy changes on both paths
    tol = 1e-12 if precision == sdpd.FP64 else 1e-10
    assert abs(o1["E"] - o0["E"]) < tol * abs(o0["E"])
    assert np.abs(o1["P"] - o0["P"]).max() < (1e-11 if precision == sdpd.FP64 else 1e-3)
    assert o1["eps_min"] > 0.0
    assert o1["n_pairs"] > 0 and o1["n_accept"] <= o1["n_pairs"]


@pytest.mark.parametrize("precision", [sdpd.FP64, sdpd.MIXED])
def test_checkpoint_resume_is_bitwise(precision):
    q, p, e, L, K = system("random_rect")
    N = len(e)
    a = gpu(N, L, K, precision=precision)
    a.set_state(q, p, e)
    a.step(DT, 8, seed=11)
    qa, pa, ea = a.get_state()
    b = gpu(N, L, K, precision=precision)
    b.set_state(q, p, e)
    b.step(DT, 4, seed=11)
    qb, pb, eb = b.get_state()
    b.set_state(qb, pb, eb)
    b.fd_step = 4
    b.step(DT, 4, seed=11)
    qb, pb, eb = b.get_state()
    assert (qa == qb).all() and (pa == pb).all() and (ea == eb).all()


def test_ssa_negative_energy_is_reported_not_fatal():
    w = Workload(n=10, K=1.5, kT=1.0)
    q, p, e = lattice_state(w)
    s = gpu(w.N, (w.L,) * 3, w.K, scheme=sdpd.SCHEME_SSA, fd_only=True)
    s.set_state(q, p, e)
    s.step(2.0, 5, seed=2)
    obs = s.observables(check=False)
    assert obs["status"] in (sdpd.ERR_NEGATIVE_ENERGY, sdpd.ERR_NAN)
    # AMS and EMS on the same stress case keep every energy positive
    for scheme in (sdpd.SCHEME_AMS, sdpd.SCHEME_EMS):
        s = gpu(w.N, (w.L,) * 3, w.K, scheme=scheme, fd_only=True)
        s.set_state(q, p, e)
        s.step(2.0, 5, seed=2)
        obs = s.observables()
        assert obs["status"] == 0 and obs["eps_min"] > 0 and obs["n_reject_bound"] > 0


def dense_cluster():
    """300 particles in a unit cube inside a 12^3 box of 800 others: every
    particle of the cluster has ~300 neighbours (list rows hold 160) and
    the 2x2x2 cell blocks around it hold more than 256 particles, 2048
    owned pairs and 255 dependency levels."""
    L = 12.0
    rng = np.random.default_rng(5)
    q = np.concatenate([rng.random((800, 3)) * L, 5.0 + rng.random((300, 3))])
    p = rng.standard_normal(q.shape)
    e = np.full(len(q), 30.0)
    return q, p, e, (L,) * 3, 20.0


def test_capacity_overflow_sweep_matches_oracle():
    """Blocks beyond the shared-memory schedule's capacities are swept pair
    by pair in canonical order: the float64 sweep of the dense cluster
    equals the oracle's pair for pair (set, colours, owners, order,
    decisions), with status OK."""
    q, p, e, L, K = dense_cluster()
    recs = sweep_fp64_vs_oracle(q, p, e, L, K, sdpd.SCHEME_EMS, shapes=(1, 128))
    assert recs["level"].max() > 255  # a block past the level capacity


@pytest.mark.parametrize("precision", [sdpd.FP64, sdpd.MIXED])
def test_uneven_lattice_blocks_stay_in_the_schedule(precision):
    """On the 32^3 lattice (cell side 8/3: cells of 8 to 27 particles,
    blocks of up to 216 with more owner-group entries than one chunk of the
    enumeration's table) every block is scheduled in shared memory; the
    dense cluster's blocks are the ones left to the pair-by-pair sweep."""
    w = Workload(n=32, K=100.0, jitter=0.05, seed=3)
    q, p, e = lattice_state(w)
    s = gpu(w.N, (w.L,) * 3, w.K, precision=precision)
    s.set_state(q, p, e)
    s.step(DT, 1, seed=4)
    assert s.observables()["status"] == sdpd.OK
    assert s.big_blocks().sum() == 0
    q, p, e, L, K = dense_cluster()
    c = gpu(len(e), L, K, precision=precision)
    c.set_state(q, p, e)
    c.step(DT, 1, seed=4)
    assert c.big_blocks().sum() > 0


@pytest.mark.parametrize("precision", [sdpd.FP64, sdpd.MIXED])
def test_capacity_overflow_steps_match_oracle(precision):
    """Full steps of the dense cluster: neighbour rows past 160 entries make
    the force pass walk the cells, and the cluster's blocks are swept pair
    by pair; the steps complete with status OK and match the oracle's."""
    q, p, e, L, K = dense_cluster()
    N = len(e)
    s = gpu(N, L, K, precision=precision)
    s.set_state(q, p, e)
    P = oparams(N, L, K)
    assert s.neighbour_counts().max() > 160
    if precision == sdpd.FP64:
        rho = O.density(P, q)
        f = O.forces(P, q, rho, e)
        assert np.abs(s.forces() - f).max() <= 1e-12 * np.abs(f).max()
    s.step(DT, 2, seed=1)
    obs = s.observables()
    assert obs["status"] == sdpd.OK
    qg, pg, eg = s.get_state()
    st, qo, po, eo, stats, _ = O.run(P, q, p, e, DT, 2, seed=1)
    assert st == O.OK
    assert obs["n_pairs"] == stats.n_pairs and obs["n_accept"] == stats.n_accept
    tol = 1e-9 if precision == sdpd.FP64 else 1e-5
    assert min_image_err(qg, qo, L) < tol
    assert np.abs(pg - po).max() < tol * np.abs(po).max()
    assert np.abs(eg - eo).max() < tol * eo.max()
    # the context and the library stay usable
    ok = gpu(1000, (10.0,) * 3, 100.0, precision=precision)
    qq, pp, ee, _, _ = system("lattice1000")
    ok.set_state(qq, pp, ee)
    ok.step(DT, 1, seed=1)
    assert ok.observables()["status"] == 0


def test_bad_state_and_empty_system():
    q, p, e, L, K = system("lattice1000")
    s = gpu(len(e), L, K)
    bad = e.copy()
    bad[17] = -1.0
    with pytest.raises(sdpd.SDPDError) as ex:
        s.set_state(q, p, bad)
    assert ex.value.status == sdpd.ERR_NONPOSITIVE_ENERGY
    with pytest.raises(sdpd.SDPDError):
        s.step(DT, 1)  # no state loaded
    z = gpu(0, L, K)
    z.set_state(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    z.step(DT, 3, seed=1)
    o = z.observables()
    assert o["E"] == 0.0 and o["status"] == 0


def test_device_state_io_matches_host_io():
    q, p, e, L, K = system("random_rect")
    N = len(e)
    a = gpu(N, L, K)
    a.set_state(q, p, e)
    b = gpu(N, L, K)
    b.set_state(torch.from_numpy(q).cuda(), torch.from_numpy(p).cuda(), torch.from_numpy(e).cuda())
    a.step(DT, 3, seed=4)
    b.step(DT, 3, seed=4)
    qd = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    pd = torch.empty_like(qd)
    ed = torch.empty(N, dtype=torch.float64, device="cuda")
    b.get_state_device(qd, pd, ed)
    qa, pa, ea = a.get_state()
    assert (qd.cpu().numpy() == qa).all() and (pd.cpu().numpy() == pa).all() and (ed.cpu().numpy() == ea).all()


def test_debug_read_outs_refuse_a_short_buffer_untouched():
    """Every debug read-out checks the caller's capacity before it copies
    anything: one element short, the call fails with SDPD_ERR_INVALID_ARG,
    writes nothing and leaves the handle usable."""
    q, p, e, L, K = system("random_rect")
    N = len(e)
    s = gpu(N, L, K, precision=sdpd.MIXED)
    s.set_state(q, p, e)
    s.step(DT, 2, seed=6)
    cases = [(sdpd.DEBUG_ORDER, np.int64, N, s.order),
             (sdpd.DEBUG_CELLS, np.int32, 3 * N, s.cells),
             (sdpd.DEBUG_RHO, np.float64, N, s.density),
             (sdpd.DEBUG_FORCE, np.float64, 3 * N, s.forces),
             (sdpd.DEBUG_NCOUNT, np.int32, N, s.neighbour_counts)]
    for what, dtype, size, full in cases:
        cap = N - 1 if what != sdpd.DEBUG_FORCE else 3 * N - 1
        buf = np.full(size, 7, dtype=dtype)
        st, n = sdpd.sdpd_debug_get(s.h, what, buf.ctypes.data, cap)
        assert st == sdpd.ERR_INVALID_ARG and n == 0, what
        assert (buf == 7).all(), what
        assert full().size == size, what
    assert s.observables()["status"] == sdpd.OK
    assert sdpd.sdpd_debug_get(s.h, 99, np.zeros(N).ctypes.data, N)[0] == sdpd.ERR_INVALID_ARG


def test_binding_rejects_mis_shaped_buffers():
    """Wrong shapes, dtypes or devices are refused before the library is
    called, and the handle keeps its state."""
    q, p, e, L, K = system("lattice1000")
    N = len(e)
    s = gpu(N, L, K)
    s.set_state(q, p, e)
    with pytest.raises(ValueError):
        s.set_state(q[:-1], p[:-1], e[:-1])
    with pytest.raises(ValueError):
        s.set_state(torch.from_numpy(q).cuda(), p, e)
    qd = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        s.get_state_device(qd, torch.empty((N, 3), dtype=torch.float32, device="cuda"), torch.empty(N, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        s.energy_histogram(0.0, 1.0, 10, counts=torch.zeros(11, dtype=torch.int64, device="cuda"))
    # a CPU tensor is a host array, not a device pointer
    s.set_state(torch.from_numpy(q), torch.from_numpy(p), torch.from_numpy(e))
    q2, p2, e2 = s.get_state()
    assert (q2 == q).all() and (p2 == p).all() and (e2 == e).all()
