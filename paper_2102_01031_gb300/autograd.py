"""torch.autograd binding of the adjoint sweep.

``evolved_objective(q, state, spec, scale=None)`` evolves the lattice state
``state`` (tensor [nf, 2, N, N, N]: field f, 0 = field / 1 = momentum,
[z][y][x]) with coupling ``q`` through the CUDA library and returns the final
objective J as a 0-dim tensor.  With self-consistent expansion the scale
factor and its derivative at the start may be given as ``scale`` = (a, b)
(else the lattice's own initial values are used, held fixed).  Its backward
pass returns dJ/dq, dJ/d(state) and dJ/d(scale), computed at a fixed initial
(state, a, b) by the library's reversed-pass adjoint kernels (cl_adjoint): the forward and the
adjoint sweep run together in the forward call, and backward only scales the
stored gradients by the incoming gradient.  The state goes to the library and
dJ/d(state) comes back in device memory (a state on the GPU never passes
through the host); the library works on the current torch stream.  PyTorch
supplies the tensors and the autograd graph; every step of the evolution and
of the adjoint runs in the library's kernels.
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
    def forward(ctx, q, state, scale, spec):
        kw = dict(spec.params)
        kw["q"] = float(q.detach())
        dev = state.device if state.is_cuda else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(dev):
            kw["stream"] = torch.cuda.current_stream(dev).cuda_stream
            lat = Lattice(spec.model, spec.N, spec.kIR, spec.alpha, spec.seed, make_params(**kw))
            # the state reaches the library in device memory (a CUDA input is not copied through the host)
            st = state.detach().to(device=dev, dtype=torch.float64).contiguous()
            nf = st.shape[0]
            for f in range(nf):
                for w in (0, 1):
                    lat.set_device(f, w, st[f, w].data_ptr())
            if scale is not None:
                eta0 = lat.scalars()[0]
                a0, b0 = (float(x) for x in scale.detach())
                lat.set_scalars(eta0, a0, b0)
            lam = torch.empty((nf, 2, spec.N, spec.N, spec.N), dtype=torch.float64, device=dev)
            J, dq, _, ab = lat.adjoint(spec.nsteps, spec.ckpt_every, spec.objective, spec.field, spec.what,
                                       spec.dk_bin, spec.bin, scale=True, lam_ptr=lam.data_ptr())
            lat.close()
        ctx.save_for_backward(torch.tensor(dq, dtype=torch.float64, device=dev), lam,
                              torch.tensor(ab, dtype=torch.float64, device=dev))
        ctx.state_meta = (state.dtype, state.device)
        ctx.scale_meta = None if scale is None else (scale.dtype, scale.device)
        return torch.tensor(J, dtype=torch.float64, device=state.device)

    @staticmethod
    def backward(ctx, g):
        dq, lam, ab = ctx.saved_tensors
        dtype, device = ctx.state_meta
        gd = g.detach().to(lam.device, torch.float64)
        gq = (gd * dq).to(device)
        gs = (gd * lam).to(device=device, dtype=dtype)
        gab = None
        if ctx.scale_meta is not None:
            gab = (gd * ab).to(device=ctx.scale_meta[1], dtype=ctx.scale_meta[0])
        return gq, gs, gab, None


def evolved_objective(q, state, spec, scale=None):
    """J of the evolution of `state` with coupling `q` (differentiable in both,
    and in `scale` = (a, b) at the start when given)."""
    return EvolvedObjective.apply(q, state, scale, spec)
