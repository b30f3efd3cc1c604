"""Seismogram-misfit gradients as a torch.autograd.Function.

`SeismogramMisfit.apply(rho, lam, mu, problem)` runs the problem's forward simulation on
the GPU with per-element density and Lame parameters taken from the three tensors and
returns the misfit J (a 0-d tensor); `backward` hands out dJ/d(rho, lambda, mu) from the
library's discrete adjoint of the global-time-stepping loop (checkpointed recomputation,
exact derivatives of the star matrices and flux solvers). The time step is the problem's
and stays fixed when the material changes.
"""
import numpy as np
import torch

from . import binding


class MisfitProblem:
    """Everything but the material: mesh, order, initial DOFs, sources, receivers,
    observed data (N+1, n_rec, 3), step count, fixed time step and checkpoint spacing."""

    def __init__(self, order, mesh, q0, receivers, data, n_steps, dt, sources=(), every=100, device=0):
        self.order, self.mesh, self.q0 = order, mesh, np.asarray(q0, dtype=np.float64)
        self.receivers, self.data = list(receivers), np.asarray(data, dtype=np.float64)
        self.n_steps, self.dt, self.sources, self.every, self.device = n_steps, dt, list(sources), every, device

    def solver(self, rho, lam, mu):
        s = binding.Solver(self.order, 0, device=self.device)
        m = self.mesh
        s.set_mesh(m["xyz"], m["tet"], m["face_bc"], m.get("period"))
        vp = np.sqrt((lam + 2.0 * mu) / rho)
        vs = np.sqrt(mu / rho)
        s.set_material(rho, vp, vs)
        for src in self.sources:
            s.add_point_source(*src)
        for x in self.receivers:
            s.add_receiver(x, self.dt)
        s.setup_clusters(1, 0.5)
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
