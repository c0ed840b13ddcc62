"""torch.autograd wrapper of the time stepping (forward: hfd_steps; backward: hfd_adjoint).

Rollout.apply(U0, mesh, dt, nsteps, every) advances the internal-order device state U0 by
nsteps SSP-RK3 steps of fixed size dt.  Its backward pass is the discrete adjoint: checkpoints
of the state are kept every `every` steps in the forward pass; the backward pass recomputes the
states of one segment at a time from its checkpoint and applies hfd_adjoint step by step in
reverse, so memory holds nsteps/every + every states.
"""
import torch


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, mesh, dt, nsteps, every):
        X = U0.detach().clone().contiguous()
        ckpts = [X.clone()]
        for i in range(nsteps):
            mesh.step(X, dt)
            if (i + 1) % every == 0 and i + 1 < nsteps:
                ckpts.append(X.clone())
        ctx.mesh, ctx.dt, ctx.nsteps, ctx.every = mesh, float(dt), int(nsteps), int(every)
        ctx.ckpts = ckpts
        return X

    @staticmethod
    def backward(ctx, grad):
        mesh, dt, n, every = ctx.mesh, ctx.dt, ctx.nsteps, ctx.every
        lam = grad.contiguous().clone()
        out = torch.empty_like(lam)
        for seg in range(len(ctx.ckpts) - 1, -1, -1):
            start = seg * every
            stop = min(n, start + every)
            states = [ctx.ckpts[seg].clone()]
            for _ in range(start, stop - 1):
                X = states[-1].clone()
                mesh.step(X, dt)
                states.append(X)
            for U in reversed(states):
                mesh.adjoint(U, lam, out, dt)
                lam, out = out, lam
        ctx.ckpts = None
        return lam, None, None, None, None


def rollout(U0, mesh, dt, nsteps, every=20):
    return Rollout.apply(U0, mesh, dt, nsteps, every)
