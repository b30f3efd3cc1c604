"""Weighted partitioning and the face-local compressed exchange (Sec. V-C), on the CPU.

The library's partitioner and exchange plan (host code, host-only handle) are checked
against the paper's weighting and the oracle's mesh tables; then two gloo ranks run one
part each of the oracle's LTS with face-local messages (H = X F-_{j,h}, 9 x F values per
cut face and receiver step) exchanged through torch.distributed, and every rank's elements
must match the unpartitioned oracle run."""
import os
import socket

import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.partitioned import PartRun
from oracle.scheme import Solver as Oracle
from paper_2202_10313_gb300 import binding, synth


def _case(nx=5, ny=4, nz=3, seed=12):
    m = synth.permute_vertex_order(synth.graded_box(nx, ny, nz, 250.0, 125.0, seed=seed), seed=3)
    mat = synth.random_layers(m, n_layers=3, seed=5)
    return m, mat


def _host(m, mat, order=4, n_mech=3, nc=3):
    h = binding.Solver(order, n_mech, device=-1)
    h.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    h.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
    cl, lam, _ = h.setup_clusters(nc, 0.5)
    return h, cl


@pytest.mark.parametrize("n_parts", [2, 3, 4, 8])
def test_weighted_partition_balance_and_stats(n_parts):
    m, mat = _case(8, 8, 4)
    h, cl = _host(m, mat)
    part, st = h.partition(n_parts)
    K = m["tet"].shape[0]
    w = 2 ** (2 - cl)
    assert part.min() == 0 and part.max() == n_parts - 1
    load = np.bincount(part, weights=w, minlength=n_parts)
    mean = w.sum() / n_parts
    assert np.isclose(st["max_load"], load.max() / mean) and np.isclose(st["min_load"], load.min() / mean)
    assert st["max_load"] <= 1.03 + 1e-12 and st["min_load"] >= 0.9
    assert st["total_weight"] == w.sum()
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])
    cut = (om.nbr >= 0) & (part[np.maximum(om.nbr, 0)] != part[:, None])
    assert st["cut_faces"] == cut.sum()
    # one face-local message per cut face and update of the receiving element
    assert st["msgs_per_macro"] == np.sum(cut * w[:, None])
    # compressed volume (9 x F per message) below the whole-buffer scheme (9 x B)
    F, B = 10, 20
    assert st["msgs_per_macro"] * F < st["buffer_msgs_per_macro"] * B
    # deterministic
    part2, _ = h.partition(n_parts)
    assert np.array_equal(part, part2)


def test_partition_follows_the_paper_weighting():
    """Parts of equal weight: a part made of coarse (rarely updated) elements holds more
    elements than one of fine elements (the imbalance in element counts of Sec. V-C)."""
    m, mat = _case(10, 4, 3, seed=2)
    h, cl = _host(m, mat)
    part, st = h.partition(4)
    w = 2 ** (2 - cl)
    counts = np.bincount(part, minlength=4)
    mean_w = np.array([w[part == p].mean() for p in range(4)])
    assert np.corrcoef(counts, mean_w)[0, 1] < 0          # heavier elements -> fewer of them
    assert st["max_load"] <= 1.03 + 1e-12


def test_exchange_plan_matches_mesh_tables():
    m, mat = _case()
    h, cl = _host(m, mat)
    part, _ = h.partition(3)
    plan = h.cut_faces(part)
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])
    want = {(k, i) for k in range(om.K) for i in range(4) if om.nbr[k, i] >= 0 and part[om.nbr[k, i]] != part[k]}
    assert {(int(r[0]), int(r[1])) for r in plan} == want and len(plan) == len(want)
    for r in plan:
        k, i, ks, js, hs, rp, sp, rc = (int(x) for x in r)
        assert om.nbr[k, i] == ks and om.nbr_face[k, i] == js and om.nbr_orient[k, i] == hs
        assert rp == part[k] and sp == part[ks] and rc == cl[k]
        # the sending side's face points back
        assert om.nbr[ks, js] == k
    keys = [(int(r[5]), int(r[6]), int(r[7]), int(r[0]), int(r[1])) for r in plan]
    assert keys == sorted(keys)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, mat = _case()
        h, cl = _host(m, mat)
        part, _ = h.partition(world)
        plan = h.cut_faces(part)
        om = Mesh(m["xyz"], m["tet"], m["face_bc"])
        K = om.K
        init = np.random.default_rng(9).normal(size=(K, 27, 20))
        init[:, :6] *= 1e6
        xs, m6 = np.array([610.0, 540.0, -260.0]), np.array([0.2, -0.4, 0.2, 1.0, 0.1, -0.3])

        def make():
            o = Oracle(4, 3, om, mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
            o.add_point_source(xs, m6, 8.0, 0.06, 1e12)
            o.setup_clusters(3, 0.5)
            assert np.array_equal(o.clusters, cl)
            o.Q = init.copy()
            return o

        nf = 10

        def exchange(out, sources):
            reqs = [dist.isend(torch.from_numpy(np.ascontiguousarray(a).ravel()), dst) for dst, a in out.items()]
            got = {}
            for src in sources:
                n = int(np.sum((plan[:, 5] == rank) & (plan[:, 6] == src) & (plan[:, 7] == cur[0])))
                buf = torch.empty(n * 9 * nf, dtype=torch.float64)
                dist.recv(buf, src)
                got[src] = buf.numpy().reshape(n, 9, nf)
            for r in reqs:
                r.wait()
            return got

        cur = [0]
        mine = make()
        run = PartRun(mine, part, rank, plan, exchange)
        orig = mine._neighbour

        def neighbour(l, n):
            cur[0] = l
            orig(l, n)

        mine._neighbour = neighbour
        mine.run_lts(8)
        full = make()
        full.run_lts(8)
        own = part == rank
        err = np.abs(mine.Q[own] - full.Q[own]).max() / np.abs(full.Q[own]).max()
        np.save(os.path.join(out_dir, "err%d.npy" % rank), np.array([err, own.sum(), len(run.recv_rows)]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_face_local_messages_match_unpartitioned_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        err, n_own, n_recv = np.load(tmp_path / ("err%d.npy" % r))
        assert n_own > 0 and n_recv > 0
        assert err <= 1e-12, (r, err)
