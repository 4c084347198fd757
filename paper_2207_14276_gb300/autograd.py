"""torch.autograd.Function wrappers whose backward is the library's hand-written
force vector-Jacobian product (the double backward of the energy).

    E, F = NNPFunction.apply(coords, weights, potential, species, box, mask)
    loss = ((F - F_target) ** 2).sum()
    loss.backward()        # coords.grad and weights.grad from nnp_force_vjp

`weights` is the flat parameter vector the potential was created with (the
library holds its own device copy; the tensor carries the gradient).
"""
from __future__ import annotations

import torch


class NNPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, weights, potential, species, box=None, mask=None):
        E, F = potential.energy_forces(coords.detach().contiguous(), species, box, mask)
        ctx.potential, ctx.species, ctx.box, ctx.mask = potential, species, box, mask
        ctx.save_for_backward(coords)
        return E, F

    @staticmethod
    def backward(ctx, gE, gF):
        (coords,) = ctx.saved_tensors
        pot = ctx.potential
        gE = torch.zeros(1, dtype=torch.float64, device=coords.device) if gE is None else gE
        gF = torch.zeros_like(coords) if gF is None else gF
        sys = {"coords": coords.detach().contiguous(), "species": ctx.species, "box": ctx.box,
               "mask": ctx.mask}
        _, _, G, W = pot.force_vjp_batch([sys], [float(gE.reshape(-1)[0])], [gF])
        return G[0], W, None, None, None, None


class NNPBatchFunction(torch.autograd.Function):
    """Batch of independent systems concatenated along the atom axis.
    sizes: atoms per system.  Returns energies [n_sys] and forces [sum(sizes), 3]."""

    @staticmethod
    def forward(ctx, coords, weights, potential, species, sizes, boxes=None):
        xs = torch.split(coords.detach().contiguous(), sizes)
        ss = torch.split(species, sizes)
        systems = [{"coords": x.contiguous(), "species": s.contiguous(),
                    "box": None if boxes is None else boxes[k]}
                   for k, (x, s) in enumerate(zip(xs, ss))]
        outs = potential.energy_forces_batch(systems)
        E = torch.cat([o["energy"] for o in outs])
        F = torch.cat([o["forces"] for o in outs])
        ctx.potential, ctx.systems, ctx.sizes = potential, systems, sizes
        return E, F

    @staticmethod
    def backward(ctx, gE, gF):
        n = len(ctx.systems)
        dev = ctx.systems[0]["coords"].device
        gE = torch.zeros(n, dtype=torch.float64, device=dev) if gE is None else gE
        gF = torch.zeros((sum(ctx.sizes), 3), device=dev) if gF is None else gF
        gEs = gE.detach().double().cpu().tolist()
        gFs = [g.contiguous() for g in torch.split(gF.detach().float(), ctx.sizes)]
        _, _, G, W = ctx.potential.force_vjp_batch(ctx.systems, gEs, gFs)
        return torch.cat(G), W, None, None, None, None
