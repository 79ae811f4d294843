"""Discrete adjoint of the RK(5,4) integration behind torch.autograd.Function.

Forward: nsteps RK(5,4) steps with libdgcns, keeping the state every
`every` steps (checkpoints in device memory) and the stage inputs of the
last segment.  Backward: segments in reverse; each segment's stage inputs are
recomputed from its checkpoint (the last segment's are kept from the forward
sweep), then dg_cns_rk_stage_adjoint runs the stages in reverse:
    W = lam_dU + B_i lam_U;  lam_U += dt (dL/dU)^T W;  lam_dU = A_i W.
The seed is the gradient of the scalar objective with respect to U(T);
KineticEnergy gives e_k(U) with its gradient from the library.
"""
import torch

__all__ = ["RKIntegrate", "KineticEnergy", "integrate", "kinetic_energy"]


def _stage_inputs(g, U0, nsteps, dt, t0, dU):
    """Run nsteps from U0 (not modified); return the list of the 5*nsteps stage input states and the final state."""
    states = []
    a = U0.clone()
    b = g.empty_state()
    for n in range(nsteps):
        for s in range(5):
            states.append(a.clone())
            g.rk_stage(s, dt, t0 + n * dt, a, dU, b)
            a, b = b, a
    return states, a


class RKIntegrate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, U0, g, nsteps, dt, every):
        U0 = U0.detach().contiguous()
        every = max(1, int(every))
        dU = g.empty_residual()
        ckpts = []
        a = U0.clone()
        b = g.empty_state()
        last_start = ((nsteps - 1) // every) * every if nsteps > 0 else 0
        last_states = []
        for n in range(nsteps):
            if n % every == 0:
                ckpts.append(a.clone())
            for s in range(5):
                if n >= last_start:
                    last_states.append(a.clone())
                g.rk_stage(s, dt, n * dt, a, dU, b)
                a, b = b, a
        fctx.g, fctx.nsteps, fctx.dt, fctx.every = g, nsteps, dt, every
        fctx.ckpts, fctx.last_states, fctx.last_start = ckpts, last_states, last_start
        return a.clone()

    @staticmethod
    def backward(fctx, grad_UT):
        g, nsteps, dt, every = fctx.g, fctx.nsteps, fctx.dt, fctx.every
        lam_U = grad_UT.detach().to(torch.float64).contiguous().clone()
        lam_dU = torch.zeros(g.shape, dtype=g.rdtype, device=lam_U.device)
        dU = g.empty_residual()
        nseg = len(fctx.ckpts)
        for k in reversed(range(nseg)):
            s0 = k * every
            s1 = min(nsteps, s0 + every)
            if s0 == fctx.last_start:
                states = fctx.last_states
            else:
                states, _ = _stage_inputs(g, fctx.ckpts[k], s1 - s0, dt, s0 * dt, dU)
            for j in reversed(range(len(states))):
                g.rk_stage_adjoint(j % 5, dt, states[j], lam_U, lam_dU)
            del states
        fctx.ckpts = fctx.last_states = None
        return lam_U, None, None, None, None


class KineticEnergy(torch.autograd.Function):
    """e_k = 1/V int |u|^2/2 (Sec. 4.2.3) of a state, with its gradient from libdgcns."""

    @staticmethod
    def forward(fctx, U, g):
        U = U.detach().contiguous()
        fctx.g = g
        fctx.save_for_backward(U)
        return torch.tensor(float(g.diagnostics(U)[0]), dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, gout):
        (U,) = fctx.saved_tensors
        G = fctx.g.kinetic_energy_gradient(U)
        return gout.to(G.dtype) * G, None


def integrate(g, U0, nsteps, dt, every=20):
    return RKIntegrate.apply(U0, g, int(nsteps), float(dt), int(every))


def kinetic_energy(g, U):
    return KineticEnergy.apply(U, g)
