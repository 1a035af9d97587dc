"""torch.autograd binding of the adjoint: the mean reaction objective as a differentiable function of
per-facet E0, alpha and sigma_t.  Marshalling only; the forward run and the reverse pass are the CUDA
library's (ldpm_set_facet_params, ldpm_adjoint)."""
from __future__ import annotations

import numpy as np
import torch

from . import ldpm


class ReactionObjective(torch.autograd.Function):
    """J(E0, alpha, sigma_t) = (1/nsteps) sum_n sum_i seed_i R_i(t_n), the time mean of the seeded
    reactions over `nsteps` steps from the model's state at the call; [F] float64 tensors in, a
    scalar out.  With keep_state the model is returned to that state afterwards (a host round trip of
    its checkpoint), so repeated calls evaluate the same function.  The gradient is computed by the
    library's reverse pass in the same call (checkpointed every ckpt_every steps) and handed to
    backward."""

    @staticmethod
    def forward(ctx, E0, alpha, sigma_t, model, nsteps, seed, ckpt_every=250, keep_state=True):
        saved = ldpm.ldpm_save_checkpoint(model.h) if keep_state else None
        model.set_facet_params(*[t.detach().to("cpu", torch.float64).numpy() for t in (E0, alpha, sigma_t)])
        need = any(ctx.needs_input_grad[:3])
        J, gE, ga, gs = model.adjoint(int(nsteps), np.asarray(seed, np.float64), int(ckpt_every), grads=need)
        if saved is not None:
            ldpm.ldpm_load_checkpoint(model.h, saved)
        if need:
            ctx.save_for_backward(*[torch.from_numpy(g).to(E0.device) for g in (gE, ga, gs)])
        return torch.tensor(J, dtype=torch.float64, device=E0.device)

    @staticmethod
    def backward(ctx, grad_out):
        gE, ga, gs = ctx.saved_tensors
        return grad_out * gE, grad_out * ga, grad_out * gs, None, None, None, None, None


def reaction_objective(E0, alpha, sigma_t, model, nsteps, seed, ckpt_every=250, keep_state=True):
    return ReactionObjective.apply(E0, alpha, sigma_t, model, nsteps, seed, ckpt_every, keep_state)
