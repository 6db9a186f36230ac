"""torch.autograd binding of the adjoint sweep.

``evolved_objective(q, state, spec)`` evolves the lattice state ``state``
(tensor [nf, 2, N, N, N]: field f, 0 = field / 1 = momentum, [z][y][x]) with
coupling ``q`` through the CUDA library and returns the final objective J as
a 0-dim tensor.  Its backward pass returns dJ/dq and dJ/d(state) computed by
the library's reversed-pass adjoint kernels (cl_adjoint): the forward and the
adjoint sweep run together in the forward call, and backward only scales the
stored gradients by the incoming gradient.  PyTorch supplies the tensors and
the autograd graph; every step of the evolution and of the adjoint runs in
the library's kernels.
"""
import dataclasses

import numpy as np
import torch

from . import Lattice, OBJ_CHI_FRACTION, make_params


@dataclasses.dataclass(frozen=True)
class RunSpec:
    """What is evolved and measured: model, lattice, run parameters
    (keywords of make_params, without q), steps, checkpoint interval, objective."""
    model: int
    N: int
    kIR: float
    alpha: float
    seed: int
    params: tuple            # sorted (name, value) pairs of make_params keywords
    nsteps: int
    ckpt_every: int = 500
    objective: int = OBJ_CHI_FRACTION
    field: int = 1
    what: int = 0
    dk_bin: float = 1.0
    bin: int = 1

    @staticmethod
    def make(model, N, kIR, alpha, seed, nsteps, ckpt_every=500, objective=OBJ_CHI_FRACTION, field=1,
             what=0, dk_bin=1.0, bin=1, **params):
        def freeze(v):
            return tuple(v) if isinstance(v, (list, np.ndarray)) else v
        items = tuple(sorted((k, freeze(v)) for k, v in params.items() if k != "q"))
        return RunSpec(model, N, kIR, alpha, seed, items, nsteps, ckpt_every, objective, field, what,
                       dk_bin, bin)


class EvolvedObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, state, spec):
        kw = dict(spec.params)
        kw["q"] = float(q.detach().cpu())
        lat = Lattice(spec.model, spec.N, spec.kIR, spec.alpha, spec.seed, make_params(**kw))
        host = state.detach().to("cpu", torch.float64).numpy()
        for f in range(host.shape[0]):
            for w in (0, 1):
                lat.set(f, w, host[f, w])
        J, dq, lam = lat.adjoint(spec.nsteps, spec.ckpt_every, spec.objective, spec.field, spec.what,
                                 spec.dk_bin, spec.bin)
        lat.close()
        ctx.save_for_backward(torch.tensor(dq, dtype=torch.float64),
                              torch.from_numpy(np.ascontiguousarray(lam)))
        ctx.state_meta = (state.dtype, state.device)
        return torch.tensor(J, dtype=torch.float64, device=state.device)

    @staticmethod
    def backward(ctx, g):
        dq, lam = ctx.saved_tensors
        dtype, device = ctx.state_meta
        gq = (g.detach().cpu() * dq).to(device)
        gs = (g.detach().cpu() * lam).to(device=device, dtype=dtype)
        return gq, gs, None


def evolved_objective(q, state, spec):
    """J of the evolution of `state` with coupling `q` (differentiable in both)."""
    return EvolvedObjective.apply(q, state, spec)
