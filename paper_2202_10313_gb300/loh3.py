"""Synthetic layer-over-half-space case after the paper's LOH.3 study (Sec. VII-B).

Runs the same seismic source once with global time stepping (one cluster) and once with
clustered LTS on a jittered layer-over-half-space mesh with the LOH.3 material and
attenuation parameters, and reports the seismogram misfit between the two runs
(E = sum_j (s_j - s^r_j)^2 / sum_j (s^r_j)^2 with the GTS trace as reference, Sec. VII-B),
the wall time of each run on the GPU, the achieved LTS speedup and the theoretical one from
the clustering. The reference seismograms, the Gmsh meshes and the exact source of the
benchmark are not available; mesh, Ricker source and receivers are synthetic stand-ins.

    python -m paper_2202_10313_gb300.loh3 [--nx 64] [--t-end 4.0] [--order 5]
"""
import argparse
import json
import time

import numpy as np

from . import binding, synth

STATION9 = np.array([8647.0, 5764.0])     # LOH.3 receiver 9, relative to the epicentre


def build_case(nx=64, h=250.0, hz_layer=125.0, nz_below=16, grade=4.0):
    mesh = synth.layer_over_halfspace(nx, nx, h, hz_layer=hz_layer, nz_below=nz_below, grade=grade)
    mat = synth.loh3_materials(mesh)
    epi = np.array([0.25 * nx * h, 0.25 * nx * h])
    src = dict(x=np.array([epi[0] + 3.0, epi[1] - 4.0, -2000.0]), m6=np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0]),
               f0=2.0, t0=0.6, m0=1e18)
    recs = [np.array([epi[0] + STATION9[0] * f, epi[1] + STATION9[1] * f, -1.0]) for f in (1.0, 0.5, 0.25)]
    recs = [r for r in recs if r[0] < nx * h and r[1] < nx * h]
    return mesh, mat, src, recs


def run_once(order, n_mech, mesh, mat, src, recs, n_clusters, t_end, dt_rec, device=0):
    import torch
    s = binding.Solver(order, n_mech, device=device)
    s.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    s.set_material(mat["rho"], mat["vp"], mat["vs"], mat.get("qp"), mat.get("qs"), 0.1, 5.0)
    s.add_point_source(src["x"], src["m6"], src["f0"], src["t0"], src["m0"])
    rids = [s.add_receiver(r, dt_rec) for r in recs]
    s.use_torch_memory(n_clusters)
    cl, lam, speedup = s.setup_clusters(n_clusters, 0.5)
    info = s.info()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.advance(t_end)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    traces = [s.seismogram(r) for r in rids]
    out = dict(wall_s=wall, lam=lam, theoretical_speedup=speedup, cluster_elems=info["cluster_elems"].tolist(),
               time=s.info()["time"], updates=int(info["updates_per_macro"].sum()) *
               int(round(s.info()["time"] / (info["finest_dt"] * 2 ** (info["n_clusters"] - 1)))))
    s.close()
    return out, traces


def misfit(sig, ref):
    den = float(np.sum(ref ** 2))
    return float(np.sum((sig - ref) ** 2) / den) if den > 0 else float("nan")


def compare(order=5, n_mech=3, nx=64, t_end=4.0, n_clusters=4, dt_rec=0.01, device=0):
    mesh, mat, src, recs = build_case(nx)
    gts, tr_g = run_once(order, n_mech, mesh, mat, src, recs, 1, t_end, dt_rec, device)
    lts, tr_l = run_once(order, n_mech, mesh, mat, src, recs, n_clusters, t_end, dt_rec, device)
    res = dict(elements=int(mesh["tet"].shape[0]), order=order, n_mech=n_mech, t_end=t_end, gts=gts, lts=lts,
               achieved_speedup=gts["wall_s"] / lts["wall_s"])
    res["efficiency"] = res["achieved_speedup"] / lts["theoretical_speedup"]
    mis = []
    for (tg, vg), (tl, vl) in zip(tr_g, tr_l):
        n = min(len(tg), len(tl))
        assert np.allclose(tg[:n], tl[:n])
        mis.append([misfit(vl[:n, q], vg[:n, q]) for q in (6, 7, 8)])
    res["misfit_uvw"] = mis
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--t-end", type=float, default=4.0)
    ap.add_argument("--order", type=int, default=5)
    ap.add_argument("--mech", type=int, default=3)
    ap.add_argument("--clusters", type=int, default=4)
    a = ap.parse_args()
    print(json.dumps(compare(a.order, a.mech, a.nx, a.t_end, a.clusters)))


if __name__ == "__main__":
    main()
