"""The paper's numerical experiments, run on the GPU (Section 4).

``fd_statistics``: the fluctuation/dissipation dynamics alone (Section 4.1).
For a scheme and a time step given in the reduced time unit of Eq.
(reduced-units), t_K = l_K sqrt(m_K / (K kB T)) with l_K = (m/rho)^(1/3) and
m_K = m, one FD-only run equilibrates and then histograms the internal
energies of ``n_configs`` configurations taken at regular intervals, over
150 bins between 0.1 kB T and 20 kB T.  Returned: the error of Eq.
(error-dist) against the Gamma marginal of Eq. (dist-analytic) (shape
C_K/kB, rate beta = 1/(kB T_eq)), its statistical floor for independent
samples, and the rejection rates split into energy-bound and Metropolis
rejections.  The temperature T_eq = E / (3(N-1)/2 + N C_K/kB) follows from
the conserved energy E (the Gamma marginal and equipartition of the kinetic
energy with the total momentum fixed at 0).

``run_statistics``: one full run (Velocity Verlet and sweep) from the
lattice: rejection rates, energy drift and mean temperatures; the ``stats``
command runs it over K, kT, dt, scheme and precision, so that the mixed
path's statistics at scale can be set against those of the float64 path
(which matches the float64 oracle step by step).

``mts_drift``: the full dynamics with single (STS) and multiple (MTS) time
steps (Section 4.2).  Independent replicas (seeds) run as one ensemble; the
total energy is read at regular intervals and its drift is the slope of a
least-squares line through E(t).  The ratio of the MTS and STS slopes at the
same Verlet step is the paper's measure of the benefit of MTS.

Both are plain drivers over the library's public API; every step runs in the
CUDA library.  ``python -m paper_1707_04232_gb300.experiments fd|mts|stats`` prints
one JSON document.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from .inputs import Workload, lattice_state
from . import sdpd

SCHEMES = {"ssa": sdpd.SCHEME_SSA, "ams": sdpd.SCHEME_AMS, "ems": sdpd.SCHEME_EMS}
PRECISIONS = {"fp64": sdpd.FP64, "mixed": sdpd.MIXED}


def reduced_time_unit(K: float, m: float = 1.0, rho: float = 1.0, kT: float = 1.0) -> float:
    """t_K of Eq. (reduced-units) for particles of mass m at mass density
    rho: l_K sqrt(m_K / eps_K), l_K = (m/rho)^(1/3), m_K = m, eps_K = K kB T."""
    return (m / rho) ** (1.0 / 3.0) * math.sqrt(m / (K * kT))


def gamma_bin_probabilities(C: float, beta_scale: float, lo: float, hi: float, nbins: int) -> np.ndarray:
    """Probability of each bin of [lo, hi) (in units of kB T_eq) under the
    Gamma marginal of Eq. (dist-analytic): shape C = C_K/kB, with x = beta
    eps; beta_scale = T / T_eq converts the bin edges."""
    from scipy import special

    edges = np.linspace(lo, hi, nbins + 1) * beta_scale
    cdf = special.gammainc(C, edges)
    return np.diff(cdf)


def distribution_error(counts: np.ndarray, C: float, beta_scale: float, lo: float, hi: float) -> dict:
    """Eq. (error-dist) on the histogram grid: the L2 distance between the
    empirical density and the Gamma density (each bin's mean density),
    relative to the L2 norm of the Gamma density; and the value expected from
    the multinomial noise of independent samples alone."""
    nbins = len(counts) - 2
    n = counts.sum()
    w = (hi - lo) / nbins
    p = gamma_bin_probabilities(C, beta_scale, lo, hi, nbins)
    nu = counts[:nbins] / (n * w)
    mu = p / w
    err = math.sqrt(((nu - mu) ** 2).sum() / (mu ** 2).sum())
    floor = math.sqrt((p * (1 - p) / (n * w * w)).sum() / (mu ** 2).sum())
    return {"error": err, "floor_independent": floor, "samples": int(n),
            "outside": int(counts[nbins] + counts[nbins + 1])}


def fd_statistics(scheme="ems", dt_reduced=1.0, n=32, K=5.0, kT=1.0, precision="mixed", n_configs=50,
                  t_equil=50.0, t_gap=10.0, seed=1, lo=0.1, hi=20.0, nbins=150) -> dict:
    """One FD-only run: equilibrate for t_equil, then n_configs histograms
    t_gap apart (times in units of t_K).  Returns the statistics as a dict."""
    import torch

    w = Workload(n=n, K=K, kT=kT, seed=seed)
    q, p, e = lattice_state(w)
    tK = reduced_time_unit(K, w.m, w.m / w.a ** 3, kT)
    dt = dt_reduced * tK
    s = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=K, scheme=SCHEMES[scheme], precision=PRECISIONS[precision],
                  fd_only=True)
    s.set_state(q, p, e)
    n_eq = max(1, int(round(t_equil / dt_reduced)))
    n_gap = max(1, int(round(t_gap / dt_reduced)))
    t0 = time.perf_counter()
    s.step(dt, n_eq, seed=seed)
    o = s.observables(check=False)
    if o["status"] != 0:
        return {"scheme": scheme, "dt_reduced": dt_reduced, "dt": dt, "status": sdpd.sdpd_strerror(o["status"]),
                "unstable": True}
    s.reset_counters()
    C = 1.5 * (K - 1.0)
    T_eq = o["E"] / (1.5 * (w.N - 1) + w.N * C)
    counts = torch.zeros(nbins + 2, dtype=torch.int64, device="cuda")
    for _ in range(n_configs):
        s.step(dt, n_gap, seed=seed)
        s.energy_histogram(lo, hi, nbins, 1.0 / T_eq, counts)
    o = s.observables(check=False)
    wall = time.perf_counter() - t0
    out = {"scheme": scheme, "precision": precision, "N": w.N, "K": K, "dt_reduced": dt_reduced, "dt": dt,
           "t_K": tK, "sweeps": n_eq + n_configs * n_gap, "T_eq": T_eq,
           "status": sdpd.sdpd_strerror(o["status"]), "unstable": o["status"] != 0}
    pairs = max(1, o["n_pairs"])
    out["rejection"] = {"total": (o["n_reject_bound"] + o["n_reject_metropolis"]) / pairs,
                        "energy_bound": o["n_reject_bound"] / pairs,
                        "metropolis": o["n_reject_metropolis"] / pairs, "pairs": int(o["n_pairs"])}
    out["distribution"] = distribution_error(counts.cpu().numpy(), C, 1.0, lo, hi)
    out["wall_s"] = wall
    return out


def energy_drift_slope(t: np.ndarray, E: np.ndarray) -> float:
    """Slope of the least-squares line through E(t)."""
    A = np.stack([t, np.ones_like(t)], axis=1)
    return float(np.linalg.lstsq(A, E, rcond=None)[0][0])


def mts_drift(dt_reduced=0.392, thetas=(1, 5, 10), scheme="ems", n=10, K=5.0, kT=1.0, replicas=10,
              t_sim=1000.0, n_samples=100, precision="fp64", seed=11) -> dict:
    """Energy-drift slopes (per unit of t_K, averaged over replicas) of the
    full dynamics with Verlet step dt_reduced t_K and one sweep of step
    theta dt every theta Verlet steps, for each theta; and their ratios to
    theta = 1."""
    import torch

    w0 = Workload(n=n, K=K, kT=kT)
    tK = reduced_time_unit(K, w0.m, w0.m / w0.a ** 3, kT)
    dt = dt_reduced * tK
    nsteps = int(round(t_sim / dt_reduced))
    out = {"scheme": scheme, "precision": precision, "K": K, "N": n ** 3, "replicas": replicas,
           "dt_reduced": dt_reduced, "dt": dt, "t_K": tK, "steps": nsteps, "slopes": {}, "status": {}}
    for theta in thetas:
        nst = nsteps - nsteps % (theta * 2) if theta > 1 else nsteps
        members, seeds = [], []
        for r in range(replicas):
            w = Workload(n=n, K=K, kT=kT, seed=seed + r)
            q, p, e = lattice_state(w)
            m = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=K, scheme=SCHEMES[scheme], precision=PRECISIONS[precision],
                          theta=theta, stream=torch.cuda.Stream())
            m.set_state(q, p, e)
            members.append(m)
            seeds.append(1000 + r)
        ens = sdpd.SDPDEnsemble(members)
        every = max(1, nst // n_samples)
        every -= every % (2 * theta) if every > 2 * theta else 0
        every = max(every, 2 * theta)
        ts, Es = [], [[] for _ in members]
        k = 0
        while k <= nst:
            if k > 0:
                ens.step(dt, every, seeds)
            for i, m in enumerate(members):
                Es[i].append(m.observables(check=False)["E"])
            ts.append(k * dt_reduced)
            k += every
        slopes = [energy_drift_slope(np.array(ts), np.array(E)) for E in Es]
        statuses = {m.observables(check=False)["status"] for m in members}
        out["slopes"][str(theta)] = {"mean": float(np.mean(slopes)), "std": float(np.std(slopes)),
                                     "per_replica": slopes, "E0": float(Es[0][0])}
        out["status"][str(theta)] = sorted(sdpd.sdpd_strerror(x) for x in statuses)
    base = out["slopes"]["1"]["mean"] if "1" in out["slopes"] else None
    if base:
        out["ratio_to_sts"] = {th: v["mean"] / base for th, v in out["slopes"].items()}
    return out


def run_statistics(precision="mixed", scheme="ems", K=100.0, kT=1.0, dt=0.005, n=64, steps=200, every=10,
                   seed=2) -> dict:
    """Full SDPD run of ``steps`` steps from the jittered lattice: rejection
    rates (energy bound, Metropolis), the energy-drift slope (least squares
    through E(t), per unit time and per particle), and the time averages of
    the kinetic and internal temperatures against T_eq = E / (3(N-1)/2 +
    N C_K/kB)."""
    w = Workload(n=n, K=K, kT=kT, seed=seed)
    q, p, e = lattice_state(w)
    s = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=K, scheme=SCHEMES[scheme], precision=PRECISIONS[precision])
    s.set_state(q, p, e)
    t0 = time.perf_counter()
    ts, Es, Tk, Ti = [], [], [], []
    k = 0
    while True:
        o = s.observables(check=False)
        ts.append(k * dt)
        Es.append(o["E"])
        Tk.append(o["T_kin"])
        Ti.append(o["T_int"])
        if k >= steps or o["status"] != 0:
            break
        s.step(dt, every, seed=seed)
        k += every
    wall = time.perf_counter() - t0
    pairs = max(1, o["n_pairs"])
    C = 1.5 * (K - 1.0)
    T_eq = Es[0] / (1.5 * (w.N - 1) + w.N * C)
    return {"precision": precision, "scheme": scheme, "K": K, "kT": kT, "dt": dt, "N": w.N, "steps": k,
            "status": sdpd.sdpd_strerror(o["status"]),
            "rejection": {"total": (o["n_reject_bound"] + o["n_reject_metropolis"]) / pairs,
                          "energy_bound": o["n_reject_bound"] / pairs,
                          "metropolis": o["n_reject_metropolis"] / pairs, "pairs": int(o["n_pairs"])},
            "drift_per_particle": energy_drift_slope(np.array(ts), np.array(Es)) / w.N,
            "T_eq": T_eq, "T_kin_mean": float(np.mean(Tk[1:])) if len(Tk) > 1 else Tk[0],
            "T_int_mean": float(np.mean(Ti[1:])) if len(Ti) > 1 else Ti[0], "wall_s": wall}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="what", required=True)
    a = sub.add_parser("fd", help="FD-only distribution error and rejection rates (Section 4.1)")
    a.add_argument("--n", type=int, default=64)
    a.add_argument("--K", type=float, default=5.0)
    a.add_argument("--schemes", default="ems,ams,ssa")
    a.add_argument("--dts", default="0.02,0.1,0.5,1,2,5")
    a.add_argument("--precision", default="mixed", choices=list(PRECISIONS))
    a.add_argument("--configs", type=int, default=50)
    b = sub.add_parser("mts", help="energy drift with single and multiple time steps (Section 4.2)")
    b.add_argument("--dts", default="0.1,0.2,0.392")
    b.add_argument("--scheme", default="ems", choices=["ems", "ams"])
    b.add_argument("--replicas", type=int, default=10)
    b.add_argument("--t-sim", type=float, default=1000.0)
    b.add_argument("--precision", default="fp64", choices=list(PRECISIONS))
    c = sub.add_parser("stats", help="rejection rates, energy drift and temperatures of full runs (M2 grid)")
    c.add_argument("--n", type=int, default=64)
    c.add_argument("--steps", type=int, default=200)
    args = ap.parse_args()
    if args.what == "stats":
        rows = [run_statistics(pr, sc, K, kT, dt, n=args.n, steps=args.steps)
                for K, kT in ((100.0, 1.0), (5.0, 0.1)) for dt in (0.001, 0.005, 0.02)
                for sc in ("ems", "ams") for pr in ("fp64", "mixed")]
        print(json.dumps({"experiment": "statistics", "rows": rows}))
    elif args.what == "fd":
        rows = [fd_statistics(sc, float(d), n=args.n, K=args.K, precision=args.precision, n_configs=args.configs)
                for sc in args.schemes.split(",") for d in args.dts.split(",")]
        print(json.dumps({"experiment": "fd_statistics", "rows": rows}))
    else:
        rows = [mts_drift(float(d), scheme=args.scheme, replicas=args.replicas, t_sim=args.t_sim,
                          precision=args.precision) for d in args.dts.split(",")]
        print(json.dumps({"experiment": "mts_drift", "rows": rows}))


if __name__ == "__main__":
    main()
