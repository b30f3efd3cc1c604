"""Seismogram-misfit gradients as a torch.autograd.Function.

`SeismogramMisfit.apply(rho, lam, mu, problem)` runs the problem's forward simulation on
the GPU with per-element density and Lame parameters taken from the three tensors and
returns the misfit J (a 0-d tensor); `backward` hands out dJ/d(rho, lambda, mu) from the
library's discrete adjoint of the time loop (checkpointed recomputation, exact derivatives
of the star matrices and flux solvers): global time stepping, or the clustered LTS loop
when the problem carries a cluster assignment. The time step (the finest one under LTS) and
the clusters are the problem's and stay fixed when the material changes.
"""
import numpy as np
import torch

from . import binding


class MisfitProblem:
    """Everything but the material: mesh, order, initial DOFs, sources, receivers,
    observed data, step count, fixed time step and checkpoint spacing.

    Global time stepping (clusters=None): data (N+1, n_rec, 3), one row per step, n_steps
    steps of dt. Clustered LTS (clusters = per-element cluster index 0..n_clusters-1, a
    normalised assignment, with its lambda): dt is the finest time step, n_steps counts finest
    steps (a multiple of the macro step 2^(n_clusters-1)), data holds one row per macro-step
    boundary (n_steps / 2^(n_clusters-1) + 1 rows) and `every` counts macro steps.
    n_fused = F > 1: F simulations in one run, source f in simulation f, initial DOFs
    (F, K, 9, B), data (rows, F, n_rec, 3); the misfit is summed over the simulations."""

    def __init__(self, order, mesh, q0, receivers, data, n_steps, dt, sources=(), every=100, device=0, n_fused=1,
                 clusters=None, n_clusters=None, lam=1.0):
        self.order, self.mesh, self.q0 = order, mesh, np.asarray(q0, dtype=np.float64)
        self.receivers, self.data = list(receivers), np.asarray(data, dtype=np.float64)
        self.n_steps, self.dt, self.sources, self.every, self.device = n_steps, dt, list(sources), every, device
        self.n_fused = n_fused
        if n_fused > 1 and len(self.sources) != n_fused:
            raise ValueError("a fused problem takes one source per simulation")
        self.clusters = None if clusters is None else np.ascontiguousarray(clusters, dtype=np.int32)
        self.n_clusters = 1 if clusters is None else int(n_clusters if n_clusters is not None else self.clusters.max() + 1)
        self.lam = float(lam)
        if n_steps % (2 ** (self.n_clusters - 1)):
            raise ValueError("n_steps must be a whole number of macro steps")

    def solver(self, rho, lam, mu):
        s = binding.Solver(self.order, 0, device=self.device, n_fused=self.n_fused)
        m = self.mesh
        s.set_mesh(m["xyz"], m["tet"], m["face_bc"], m.get("period"))
        vp = np.sqrt((lam + 2.0 * mu) / rho)
        vs = np.sqrt(mu / rho)
        s.set_material(rho, vp, vs)
        for f, src in enumerate(self.sources):
            s.add_point_source(*src, fused_idx=f if self.n_fused > 1 else 0)
        for x in self.receivers:
            s.add_receiver(x, self.dt)
        if self.clusters is None:
            s.setup_clusters(1, 0.5)
        else:
            s.force_clusters(self.clusters, self.n_clusters, 0.5, self.lam)
        s.set_finest_dt(self.dt)
        s.set_dofs(self.q0)
        return s


class SeismogramMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, lam, mu, problem):
        r, l, m = (t.detach().to("cpu", torch.float64).numpy() for t in (rho, lam, mu))
        s = problem.solver(r, l, m)
        J, grad, _ = s.misfit_gradient(problem.n_steps, problem.data, every=problem.every)
        s.close()
        g = torch.from_numpy(grad)
        ctx.save_for_backward(g[:, 0].to(rho), g[:, 1].to(lam), g[:, 2].to(mu))
        return torch.tensor(J, dtype=rho.dtype, device=rho.device)

    @staticmethod
    def backward(ctx, gJ):
        gr, gl, gm = ctx.saved_tensors
        return gJ * gr, gJ * gl, gJ * gm, None


def _config5(nx, ny, nz, order, n_clusters, n_rec, seed=11):
    """Elastic layered box with a +1 % (rho, lambda, mu) blob for the observed data."""
    from . import synth
    mesh = synth.graded_box(nx, ny, nz, 250.0, 125.0)
    mat = synth.random_layers(mesh)
    rho = mat["rho"].astype(float)
    mu = rho * mat["vs"] ** 2
    lam = rho * mat["vp"] ** 2 - 2 * mu
    cen = mesh["xyz"][mesh["tet"]].mean(axis=1)
    c0 = np.array([0.45 * nx * 250.0, 0.5 * ny * 250.0, -600.0])
    blob = 0.01 * np.exp(-np.sum((cen - c0) ** 2, axis=1) / (2 * 1000.0 ** 2))
    rng = np.random.default_rng(seed)
    rec = [np.array([x, y, -1.0]) for x, y in rng.uniform([0.1 * nx * 250.0, 0.1 * ny * 250.0],
                                                           [0.9 * nx * 250.0, 0.9 * ny * 250.0], size=(n_rec, 2))]
    src = (np.array([0.4 * nx * 250.0 + 7.0, 0.5 * ny * 250.0 - 3.0, -1000.0]),
           np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0]), 5.0, 0.24, 1e15)
    return mesh, (rho, lam, mu), blob, rec, src


def main():
    """Gradient of the seismogram misfit on the adjoint workload: 40 x 40 x 21 hexes x 6 =
    201,600 jittered graded tets, elastic order 4, 3 LTS clusters, 2,000 finest steps, 32
    surface receivers, observed data from a run with rho, lambda, mu 1 % higher in a
    Gaussian blob, checkpoints every 100 finest steps. With --fused F, F sources (the first
    one and F - 1 at seeded positions) run fused: the gradient of the summed misfit, timed
    beside one single-source gradient. Prints one JSON line."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=40)
    ap.add_argument("--ny", type=int, default=40)
    ap.add_argument("--nz", type=int, default=21)
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--clusters", type=int, default=3)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--checkpoint", type=int, default=100, help="finest steps between checkpoints")
    ap.add_argument("--receivers", type=int, default=32)
    ap.add_argument("--fd", type=int, default=3, help="elements checked by central differences")
    ap.add_argument("--tile", type=int, default=None,
                    help="tile variant of the sparse engine's neighbour kernel (0: 8 elements per CTA, 1: 4)")
    ap.add_argument("--fused", type=int, default=1,
                    help="F > 1: F sources in one fused run (gradient of the summed misfit), timed "
                         "against one single-source gradient")
    a = ap.parse_args()
    mesh, (rho, lam, mu), blob, rec, src = _config5(a.nx, a.ny, a.nz, a.order, a.clusters, a.receivers)
    F = a.fused
    srcs = [src]
    if F > 1:   # further sources at seeded positions and orientations, 1 km deep
        rng = np.random.default_rng(7)
        for _ in range(F - 1):
            x = np.array([rng.uniform(0.2, 0.8) * a.nx * 250.0, rng.uniform(0.2, 0.8) * a.ny * 250.0, -1000.0])
            srcs.append((x, rng.normal(size=6), src[2], src[3], src[4]))
    K = mesh["tet"].shape[0]
    period = 2 ** (a.clusters - 1)
    n_macro = a.steps // period

    def solver(r, l, m, cl=None, lam_c=None, dt=None, nf=F):
        s = binding.Solver(a.order, 0, device=0, n_fused=nf)
        if a.tile is not None:
            s.set_tile(a.tile)
        s.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
        s.set_material(r, np.sqrt((l + 2 * m) / r), np.sqrt(m / r))
        for f in range(nf):
            s.add_point_source(*srcs[f], fused_idx=f)
        for x in rec:
            s.add_receiver(x, 0.01)
        if cl is None:
            cl, lam_c, _ = s.setup_clusters(a.clusters, 0.5)
            dt = s.info()["finest_dt"]
        else:
            s.force_clusters(cl, a.clusters, 0.5, lam_c)
            s.set_finest_dt(dt)
        return s, cl, lam_c, dt

    base, cl, lam_c, dt = solver(rho, lam, mu)
    data0 = np.zeros((n_macro + 1, len(rec), 3) if F == 1 else (n_macro + 1, F, len(rec), 3))
    pert, _, _, _ = solver(rho * (1 + blob), lam * (1 + blob), mu * (1 + blob), cl, lam_c, dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, data = pert.misfit(a.steps, data0, every=a.checkpoint // period)
    t_fwd = time.perf_counter() - t0
    pert.close()
    t0 = time.perf_counter()
    J, grad, _ = base.misfit_gradient(a.steps, data, every=a.checkpoint // period)
    t_grad = time.perf_counter() - t0
    g_m6 = base.source_gradient()
    base.close()
    single = None
    if F > 1:   # one source alone, same material and data of that source
        one, _, _, _ = solver(rho, lam, mu, cl, lam_c, dt, nf=1)
        t0 = time.perf_counter()
        one.misfit_gradient(a.steps, np.ascontiguousarray(data[:, 0]), every=a.checkpoint // period)
        single = time.perf_counter() - t0
        one.close()
    fd = []
    params = [rho, lam, mu]
    for k in np.argsort(-np.abs(grad[:, 2]))[:a.fd]:
        vals = []
        for sgn in (1, -1):
            pp = [x.copy() for x in params]
            pp[2][k] *= 1 + sgn * 1e-3
            s, _, _, _ = solver(*pp, cl, lam_c, dt)
            vals.append(s.misfit(a.steps, data, every=a.checkpoint // period)[0])
            s.close()
        fd.append(dict(element=int(k), adjoint=float(grad[k, 2]),
                       central_difference=float((vals[0] - vals[1]) / (2e-3 * mu[k]))))
    out = dict(elements=int(K), order=a.order, clusters=a.clusters, cluster_elems=np.bincount(cl).tolist(),
               finest_steps=a.steps, macro_steps=n_macro, checkpoint_finest_steps=a.checkpoint, receivers=len(rec),
               fused_sources=F, single_source_gradient_s=single,
               misfit=J, forward_s=t_fwd, misfit_and_gradient_s=t_grad, gradient_over_forward=t_grad / t_fwd,
               grad_norm=[float(np.linalg.norm(grad[:, p])) for p in range(3)],
               moment_tensor_gradient=g_m6.tolist(), fd_check_mu=fd)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
