"""Full-size parity on the benchmark configuration (2,101,248 tets, order 5, 3 mechanisms,
5 clusters with the lambda search, CFL 0.5, moment-tensor source, 64 receivers), run
through the same set-up and launches as bench.py for one macro step (16 finest steps).

Sampled outputs: after 16 finest steps an element's state depends only on data within 16
face hops (information crosses at most one face per finest step). Sample centres: the
source element, two receiver elements, an element on the free surface, one on an absorbing
side, and one element of every non-empty cluster. Every element within one face hop of a
centre is a sample (at least 32 in all); the oracle runs the same steps on the ball of
17 + 1 hops around the centre (cut faces absorbing, one hop of margin), with its own
clustering of the full mesh, and each sample's DOFs are compared with the GPU's, per
element and over all samples."""
import numpy as np
import pytest

import bench
from oracle import lts as olts
from oracle.mesh import Mesh
from oracle.scheme import Solver as Oracle
from paper_2202_10313_gb300 import binding, build, synth
from gpu_common import check_parity, rel_l2_groups, report_parity

pytestmark = pytest.mark.gpu
HOPS = 17


def _centres(mesh, om, cl, n_clusters, rng, src_elems, rec_pts):
    """Sample centres: source elements, two receiver elements, a free-surface element, an
    element with an absorbing face (and none on the surface), one element per cluster."""
    out = [int(e) for e in src_elems]
    out += [int(om.locate(np.asarray(r))) for r in rec_pts[:2]]
    bc = mesh["face_bc"]
    free = np.nonzero((bc == 2).any(axis=1))[0]
    absorb = np.nonzero((bc == 1).any(axis=1) & ~(bc == 2).any(axis=1))[0]
    out += [int(rng.choice(free)), int(rng.choice(absorb))]
    out += [int(rng.choice(np.nonzero(cl == l)[0])) for l in range(n_clusters) if np.any(cl == l)]
    return list(dict.fromkeys(out))


def _sub_oracle(mesh, om, ball, mat, order, n_mech, n_clusters, lam, cl, delta):
    """The oracle on the ball's sub-mesh: cut faces absorbing, clusters and time step those
    of the full mesh."""
    tet = mesh["tet"][ball]
    uv, inv = np.unique(tet, return_inverse=True)
    bc = mesh["face_bc"][ball].copy()
    inside = np.isin(om.nbr[ball], ball)
    bc[(om.nbr[ball] >= 0) & ~inside] = 1            # cut faces: absorbing, never reach a sample
    sm = Mesh(mesh["xyz"][uv], inv.reshape(tet.shape), bc)
    if n_mech:
        o = Oracle(order, n_mech, sm, mat["rho"][ball], mat["vp"][ball], mat["vs"][ball],
                   mat["qp"][ball], mat["qs"][ball], 0.1, 5.0)
    else:
        o = Oracle(order, 0, sm, mat["rho"][ball], mat["vp"][ball], mat["vs"][ball])
    o.setup_clusters(n_clusters, bench.CFL, lam=lam, clusters=cl[ball])
    o.delta = delta
    return o


def _ball(nbr, k, hops):
    seen = {int(k)}
    front = [int(k)]
    for _ in range(hops):
        nxt = []
        for e in front:
            for nb in nbr[e]:
                if nb >= 0 and int(nb) not in seen:
                    seen.add(int(nb))
                    nxt.append(int(nb))
        front = nxt
    return np.array(sorted(seen))


@pytest.mark.parametrize("contraction", ["fp32", "sparse", "tf32x3"])
def test_bench_configuration_sampled_parity(contraction):
    """Every engine the autotuner may pick for the bench run."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    mesh, mat, src, recs = bench.make_workload(**bench.FULL)
    K = mesh["tet"].shape[0]
    assert K == 2101248
    # ---- library, set up exactly as bench.py does
    g = binding.Solver(bench.ORDER, bench.NMECH, device=0)
    g.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    g.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
    g.add_point_source(src["x"], src["m6"], src["f0"], src["t0"], src["m0"])
    for r in recs:
        g.add_receiver(r, 0.01)
    g.use_torch_memory(bench.NCLUSTERS)
    g.set_contraction(contraction)
    cl_g, lam_g, sp_g = g.setup_clusters(bench.NCLUSTERS, bench.CFL)
    # ---- oracle clustering of the full mesh
    om = Mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    dt = olts.cfl_time_steps(om.dins, mat["vp"], bench.ORDER, bench.CFL)
    lam, cl, sp = olts.search_lambda(dt, om.nbr, bench.NCLUSTERS)
    assert lam == lam_g and np.array_equal(cl, cl_g)
    delta = lam * dt.min()
    # ---- sample centres, their one-hop neighbourhoods (the samples) and balls
    rng = np.random.default_rng(17)
    src_elem = om.locate(src["x"])
    centres = _centres(mesh, om, cl, bench.NCLUSTERS, rng, [src_elem], recs)
    inner = [_ball(om.nbr, c, 1) for c in centres]
    balls = [_ball(om.nbr, c, HOPS + 1) for c in centres]
    samples = np.concatenate(inner)
    assert len(samples) >= 32
    union = np.unique(np.concatenate(balls))
    init = synth.random_dofs(len(union), 27, 35, seed=23)
    g.set_dofs_subset(union, init)
    row_of = {int(e): i for i, e in enumerate(union)}
    # ---- one macro step on the GPU
    g.advance_steps(2 ** (bench.NCLUSTERS - 1))
    got = g.get_dofs_subset(samples)
    want = np.zeros_like(got)
    worst = {}
    pos = 0
    for c, ins, ball in zip(centres, inner, balls):
        o = _sub_oracle(mesh, om, ball, mat, bench.ORDER, bench.NMECH, bench.NCLUSTERS, lam, cl, delta)
        o.Q = init[[row_of[int(e)] for e in ball]].copy()
        if src_elem in set(ball.tolist()):
            o.add_point_source(src["x"], src["m6"], src["f0"], src["t0"], src["m0"])
        o.run_lts(2 ** (bench.NCLUSTERS - 1))
        for k in ins:
            want[pos] = o.Q[np.searchsorted(ball, k)]
            err = rel_l2_groups(got[pos][None], want[pos][None], 27)
            worst = {n: max(worst.get(n, 0.0), v) for n, v in err.items()}
            for name, v in err.items():
                assert v <= 1e-4, (int(k), int(cl[k]), err)
            pos += 1
    worst.update({"samples_" + k: v for k, v in check_parity(got, want, 27, 1e-4).items()})
    report_parity("anelastic O5, 2,101,248 tets, 5 clusters, one macro step, %s (%d sampled elements)"
                  % (contraction, len(samples)), worst)


def test_fused_configuration_sampled_parity():
    """The fused workload of bench.py --fused 16 (983,040 tets, 16 simulations, one random
    moment-tensor source each): one macro step, then the DOFs of the sample elements (one-hop
    neighbourhoods of the centres, the two simulations' source elements among them) in two
    simulations of different CTA groups against the oracle on balls of 18 hops."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    F = 16
    cfg = bench.FUSED_FULL
    mesh, mat, src, recs = bench.make_workload(**cfg)
    K = mesh["tet"].shape[0]
    assert K == 983040
    g = binding.Solver(bench.ORDER, bench.NMECH, device=0, n_fused=F)
    g.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    g.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
    lx, ly, depth = cfg["nx"] * cfg["h"], cfg["ny"] * cfg["h"], mesh["depth"]
    pos, m6s, f0s = synth.random_sources(F, [0.1 * lx, 0.1 * ly, -0.6 * depth], [0.9 * lx, 0.9 * ly, -0.05 * depth],
                                         f0_range=(1.0, 4.0), seed=7)
    for f in range(F):
        g.add_point_source(pos[f], m6s[f], f0s[f], 1.2 / f0s[f], src["m0"], fused_idx=f)
    g.use_torch_memory(bench.NCLUSTERS)
    cl_g, lam_g, _ = g.setup_clusters(bench.NCLUSTERS, bench.CFL)
    om = Mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    dt = olts.cfl_time_steps(om.dins, mat["vp"], bench.ORDER, bench.CFL)
    lam, cl, _ = olts.search_lambda(dt, om.nbr, bench.NCLUSTERS)
    assert lam == lam_g and np.array_equal(cl, cl_g)
    delta = lam * dt.min()
    rng = np.random.default_rng(19)
    sims = (2, 13)
    src_elems = [om.locate(pos[f]) for f in sims]
    centres = _centres(mesh, om, cl, bench.NCLUSTERS, rng, src_elems, recs)
    inner = [_ball(om.nbr, c, 1) for c in centres]
    balls = [_ball(om.nbr, c, HOPS + 1) for c in centres]
    samples = np.concatenate(inner)
    assert len(samples) >= 32
    union = np.unique(np.concatenate(balls))
    init = np.stack([synth.random_dofs(len(union), 27, 35, seed=60 + f) for f in range(F)])
    g.set_dofs_subset(union, init)
    row_of = {int(e): i for i, e in enumerate(union)}
    g.advance_steps(2 ** (bench.NCLUSTERS - 1))
    got = g.get_dofs_subset(samples)                 # (F, n, 27, 35)
    worst = {}
    for f, src_elem in zip(sims, src_elems):
        want = np.zeros_like(got[f])
        p = 0
        for c, ins, ball in zip(centres, inner, balls):
            o = _sub_oracle(mesh, om, ball, mat, bench.ORDER, bench.NMECH, bench.NCLUSTERS, lam, cl, delta)
            o.Q = init[f][[row_of[int(e)] for e in ball]].copy()
            if src_elem in set(ball.tolist()):
                o.add_point_source(pos[f], m6s[f], f0s[f], 1.2 / f0s[f], src["m0"])
            o.run_lts(2 ** (bench.NCLUSTERS - 1))
            for k in ins:
                want[p] = o.Q[np.searchsorted(ball, k)]
                err = rel_l2_groups(got[f, p][None], want[p][None], 27)
                worst = {n: max(worst.get(n, 0.0), v) for n, v in err.items()}
                for name, v in err.items():
                    assert v <= 1e-4, (f, int(k), err)
                p += 1
        for k, v in check_parity(got[f], want, 27, 1e-4).items():
            worst["samples_" + k] = max(worst.get("samples_" + k, 0.0), v)
    report_parity("anelastic O5, 983,040 tets, 16 fused sources, one macro step (%d sampled elements x 2 simulations)"
                  % len(samples), worst)


def test_elastic_configuration_sampled_parity():
    """The elastic order-5 workload of bench.py --elastic (786,432 tets, three layers, 4
    clusters with the lambda search, 2 Hz Ricker source): one macro step (8 finest steps),
    the one-hop neighbourhoods of the sample centres against the oracle on balls of 10 hops."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    hops = 9
    mesh, mat, src, recs = bench.make_elastic_workload(**bench.ELASTIC_FULL)
    K = mesh["tet"].shape[0]
    assert K == 786432
    nc, order = bench.ELASTIC_CLUSTERS, bench.ELASTIC_ORDER
    g = binding.Solver(order, 0, device=0)
    g.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    g.set_material(mat["rho"], mat["vp"], mat["vs"])
    g.add_point_source(src["x"], src["m6"], src["f0"], src["t0"], src["m0"])
    for r in recs:
        g.add_receiver(r, 0.01)
    g.use_torch_memory(nc)
    cl_g, lam_g, _ = g.setup_clusters(nc, bench.CFL)
    om = Mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    dt = olts.cfl_time_steps(om.dins, mat["vp"], order, bench.CFL)
    lam, cl, _ = olts.search_lambda(dt, om.nbr, nc)
    assert lam == lam_g and np.array_equal(cl, cl_g)
    delta = lam * dt.min()
    rng = np.random.default_rng(29)
    src_elem = om.locate(src["x"])
    centres = _centres(mesh, om, cl, nc, rng, [src_elem], recs)
    inner = [_ball(om.nbr, c, 1) for c in centres]
    balls = [_ball(om.nbr, c, hops + 1) for c in centres]
    samples = np.concatenate(inner)
    assert len(samples) >= 32
    union = np.unique(np.concatenate(balls))
    init = synth.random_dofs(len(union), 9, 35, seed=31)
    g.set_dofs_subset(union, init)
    row_of = {int(e): i for i, e in enumerate(union)}
    g.advance_steps(2 ** (nc - 1))
    got = g.get_dofs_subset(samples)
    want = np.zeros_like(got)
    worst = {}
    p = 0
    for c, ins, ball in zip(centres, inner, balls):
        o = _sub_oracle(mesh, om, ball, mat, order, 0, nc, lam, cl, delta)
        o.Q = init[[row_of[int(e)] for e in ball]].copy()
        if src_elem in set(ball.tolist()):
            o.add_point_source(src["x"], src["m6"], src["f0"], src["t0"], src["m0"])
        o.run_lts(2 ** (nc - 1))
        for k in ins:
            want[p] = o.Q[np.searchsorted(ball, k)]
            err = rel_l2_groups(got[p][None], want[p][None], 9)
            worst = {n: max(worst.get(n, 0.0), v) for n, v in err.items()}
            for name, v in err.items():
                assert v <= 1e-4, (int(k), int(cl[k]), err)
            p += 1
    worst.update({"samples_" + k: v for k, v in check_parity(got, want, 9, 1e-4).items()})
    report_parity("elastic O5, 786,432 tets, 4 clusters, one macro step (%d sampled elements)" % len(samples), worst)


def test_adjoint_configuration_gradient_against_central_differences():
    """The adjoint workload (201,600 tets, elastic order 4, 3 LTS clusters, 2,000 finest
    steps, 32 receivers, checkpoints every 100 finest steps): the gradient w.r.t. rho, lambda
    and mu of 20 elements drawn at random (seeded) against central differences of the GPU
    misfit, each element and parameter on its own. A difference quotient resolves a gradient
    only where a relative step of at most 0.1 moves J well above its FP32 scatter (about
    5e-5 J after 2,000 steps of a 1 % model perturbation): the elements are drawn from those
    whose mu-sensitivity |dJ/dmu_k| mu_k is at least 5e-2 J. The step is h = min(0.1, 5e-3 J /
    |g p|) of the parameter (J moves by about 1 %; near the source J is strongly non-linear in
    an element's parameters), and |fd - g| <= 2e-2 |g| + 1e-4 J / h. Rows that fail are printed."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2202_10313_gb300 import adjoint
    mesh, (rho, lam, mu), blob, rec, src = adjoint._config5(40, 40, 21, 4, 3, 32)
    assert mesh["tet"].shape[0] == 201600
    steps, every = 2000, 25

    def solver(r, l, m, fixed=None):
        s = binding.Solver(4, 0, device=0)
        s.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
        s.set_material(r, np.sqrt((l + 2 * m) / r), np.sqrt(m / r))
        s.add_point_source(*src)
        for x in rec:
            s.add_receiver(x, 0.01)
        if fixed is None:
            cl, lc, _ = s.setup_clusters(3, 0.5)
            return s, (cl, lc, s.info()["finest_dt"])
        s.force_clusters(fixed[0], 3, 0.5, fixed[1])
        s.set_finest_dt(fixed[2])
        return s, fixed

    base, fixed = solver(rho, lam, mu)
    pert, _ = solver(rho * (1 + blob), lam * (1 + blob), mu * (1 + blob), fixed)
    _, data = pert.misfit(steps, np.zeros((steps // 4 + 1, len(rec), 3)), every=every)
    pert.close()
    J, grad, _ = base.misfit_gradient(steps, data, every=every)
    base.close()
    assert J > 0
    params = [rho, lam, mu]
    pool = np.nonzero(np.abs(grad[:, 2]) * mu >= 5e-2 * J)[0]
    assert len(pool) >= 20, len(pool)
    elems = np.random.default_rng(2202).choice(pool, 20, replace=False)
    rows, bad, worst = [], [], 0.0
    for k in elems:
        for p in range(3):
            g = float(grad[k, p])
            h = min(0.1, 5e-3 * J / max(abs(g * params[p][k]), 1e-300)) * params[p][k]
            vals = []
            for sgn in (1, -1):
                pp = [x.copy() for x in params]
                pp[p][k] += sgn * h
                s, _ = solver(*pp, fixed)
                vals.append(s.misfit(steps, data, every=every)[0])
                s.close()
            fd = (vals[0] - vals[1]) / (2 * h)
            floor = 1e-4 * J / h
            err = abs(fd - g)
            rows.append((int(k), "rho lambda mu".split()[p], fd, g, err / max(abs(fd), 1e-300)))
            if err > 2e-2 * abs(g) + floor:
                bad.append(rows[-1])
            if abs(g) > 10 * floor:
                worst = max(worst, err / abs(g))
    for r in bad:
        print("FD MISMATCH element %d d/d%s: central difference %.6e adjoint %.6e relative %.2e" % r)
    assert not bad, bad
    report_parity("adjoint, 201,600 tets, O4, 3 clusters, 2,000 steps: dJ/d(rho, lambda, mu) vs central differences "
                  "on 20 random elements", {"relative": worst})
