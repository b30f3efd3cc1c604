"""Oracle: CFL time steps and rate-2 clustering (test infrastructure).

Sec. V-A: each element has a CFL time step dt_k; dt_min = min_k dt_k; clusters
C_l = [2^(l-1) lam dt_min, 2^l lam dt_min), l = 1..N_c, the last one open-ended;
every element of C_l advances with 2^(l-1) lam dt_min. Normalisation moves
elements to finer clusters until face neighbours differ by at most one cluster.
lambda is searched in steps of 0.01 to maximise the theoretical speedup over GTS.

Readings (the paper prints no CFL formula and no search range): dt_k = cfl * d_k /
((2 O - 1) vp_k) with d_k the insphere diameter; lambda in {0.51, ..., 1.00};
normalisation applied inside the search; ties go to the larger lambda.
Clusters are numbered 0..N_c-1 here (paper: 1..N_c).
"""
import numpy as np


def cfl_time_steps(dins, vp, order, cfl):
    """dt_k = cfl * d_k / ((2 O - 1) vp_k)."""
    return cfl * np.asarray(dins) / ((2.0 * order - 1.0) * np.asarray(vp))


def assign_clusters(dt, lam, n_clusters):
    """Cluster index c(k) in 0..N_c-1: largest l with 2^l * (lam dt_min) <= dt_k."""
    dt = np.asarray(dt, dtype=float)
    base = lam * dt.min()
    out = np.zeros(len(dt), dtype=np.int64)
    for l in range(1, n_clusters):
        out[dt >= base * 2.0 ** l] = l
    return out


def normalise(clusters, nbr):
    """Fixed point of c(k) <- min(c(k), min over face neighbours c(nbr) + 1)."""
    c = np.array(clusters, dtype=np.int64)
    nbr = np.asarray(nbr)
    has = nbr >= 0
    safe = np.where(has, nbr, 0)
    while True:
        nb = np.where(has, c[safe] + 1, np.iinfo(np.int64).max)
        new = np.minimum(c, nb.min(axis=1))
        if np.array_equal(new, c):
            return c
        c = new


def theoretical_speedup(clusters, lam):
    """GTS cost / LTS cost = K lam / sum_l |C_l| 2^-l (clusters 0-based)."""
    c = np.asarray(clusters)
    return len(c) * lam / np.sum(2.0 ** (-c.astype(float)))


def search_lambda(dt, nbr, n_clusters):
    """Best lambda in {0.51..1.00}; returns (lam, clusters, speedup)."""
    best = None
    for i in range(51, 101):
        lam = i / 100.0
        c = normalise(assign_clusters(dt, lam, n_clusters), nbr)
        s = theoretical_speedup(c, lam)
        if best is None or s >= best[2]:
            best = (lam, c, s)
    return best
