"""One model's refinement step split over ranks by reflections.

Every term of the method is a sum over reflections: the pattern (Eq.
direct_sum, summed over hkl at every pixel), the gradient of the structure
factors' atoms (Eq. structure_factor differentiated: a sum over hkl per atom)
and the gradients of the global parameters (crystallite sizes, g, sigma,
gamma: sums over hkl of per-reflection chain-rule terms).  So a rank that
owns a contiguous slice of the reflection list can compute its slice's part
of all of them on its own GPU, and the step needs exactly two exchanges:

  forward:   all-reduce (sum) of the partial images  -> the full image on every rank
  (loss and dL/dI from the full image, identical on every rank)
  backward:  all-reduce (sum) of the partial gradients -> dfrac [n_atoms, 3],
             dB [n_atoms], the 8 globals (dL_a, dL_b, dL_c, dg_a, dg_b, dg_c,
             dsigma, dgamma)

The compute of a slice is delegated to a backend object with three methods,
`partial_image(begin, end)`, `loss_grad(image)` and
`partial_grads(begin, end, dL_dI)`; `FdxBackend` below runs them through the
library's C-ABI on the local GPU.  The exchange goes through a `reduce`
callable (default: torch.distributed.all_reduce with SUM), so the same code
runs over NCCL between GPUs, over gloo between CPU processes, or with a
caller-supplied reduction.
"""
from __future__ import annotations

from typing import Callable, Tuple

from .replicas import shard_range


def reflection_slice(n_refl: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous slice [begin, end) of the reflection list owned by `rank`."""
    return shard_range(n_refl, rank, world)


def _all_reduce_sum(t):
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


class ShardedRefineStep:
    """Forward + loss + backward of one model with its reflections split over
    `world` ranks.  `reduce(tensor)` must sum the tensor over all ranks in
    place (and return it)."""

    def __init__(self, backend, n_refl: int, rank: int, world: int,
                 reduce: Callable | None = None):
        self.backend = backend
        self.rank, self.world = rank, world
        self.begin, self.end = reflection_slice(n_refl, rank, world)
        self.reduce = reduce if reduce is not None else (_all_reduce_sum if world > 1 else (lambda t: t))

    def forward(self):
        """The full image on every rank: this rank's slice, summed over ranks."""
        img = self.backend.partial_image(self.begin, self.end)
        return self.reduce(img)

    def __call__(self):
        """Returns (image, loss, dfrac, dB, dglobal), identical on every rank."""
        img = self.forward()
        loss, gI = self.backend.loss_grad(img)
        dfrac, dB, dglob = self.backend.partial_grads(self.begin, self.end, gI)
        # one exchange for all gradients: pack, reduce, unpack
        packed = self.backend.pack(dfrac, dB, dglob)
        self.reduce(packed)
        dfrac, dB, dglob = self.backend.unpack(packed, dfrac, dB, dglob)
        return img, loss, dfrac, dB, dglob


class FdxBackend:
    """The slice computations on the local GPU through the C-ABI: structure
    factors of the slice's reflections, the pattern of that slice (zero
    reflections give a zero image), the loss against a target, and the
    adjoint of the slice."""

    def __init__(self, problem, target_image, mask=None, device="cuda"):
        import torch
        from . import fdx
        self.fdx = fdx
        self.problem = problem
        self.device = device
        self.hkl_host = fdx.fdx_reflections(problem.cell, problem.d_min, problem.d_max)
        self.hkl = torch.as_tensor(self.hkl_host, device=device).contiguous()
        self.atoms = fdx.DeviceAtoms(problem.atoms, device)
        n, na = self.hkl.shape[0], problem.atoms.n
        self.F = torch.empty((max(n, 1), 2), dtype=torch.float32, device=device)
        self.M = torch.empty((max(n, 1),), dtype=torch.float32, device=device)
        self.target = target_image
        self.mask = mask
        ny, nx = problem.geom.n_y, problem.geom.n_x
        self.image = torch.empty((ny, nx), dtype=torch.float32, device=device)
        self.gI = torch.empty((ny, nx), dtype=torch.float32, device=device)
        self.loss = torch.empty((), dtype=torch.float64, device=device)
        self.lws = torch.empty(fdx.fdx_loss_workspace_size(nx * ny), dtype=torch.uint8, device=device)
        self.dfrac = torch.empty((na, 3), dtype=torch.float64, device=device)
        self.dB = torch.empty((na,), dtype=torch.float64, device=device)
        self.dglob = torch.empty(8, dtype=torch.float64, device=device)
        self._probs = {}

    def _slice(self, b, e):
        """Problem struct, structure-factor workspace and pattern/backward
        workspaces of the slice [b, e) (built once per slice)."""
        import torch
        key = (b, e)
        if key not in self._probs:
            fdx = self.fdx
            hkl = self.hkl[b:e]
            prob = fdx.make_problem(self.problem.cell, self.problem.br, self.problem.geom, hkl, self.M[b:max(e, b + 1)])
            sf_ws = torch.empty(max(fdx.fdx_sf_workspace_size(self.problem.atoms.n, e - b), 256), dtype=torch.uint8,
                                device=self.device)
            ws = torch.empty(max(fdx.fdx_workspace_size([prob]), 256), dtype=torch.uint8, device=self.device)
            bws = torch.empty(max(fdx.fdx_backward_workspace_size(prob, self.problem.atoms.n,
                                                                  self.problem.atoms.ff.shape[0]), 256),
                              dtype=torch.uint8, device=self.device)
            self._probs[key] = (prob, sf_ws, ws, bws)
        return self._probs[key]

    def partial_image(self, b, e):
        prob, sf_ws, ws, _ = self._slice(b, e)
        if e > b:
            self.fdx.fdx_structure_factors(self.problem.cell, self.atoms, self.hkl[b:e], self.problem.br,
                                           self.F[b:e], self.M[b:e], sf_ws)
        self.fdx.fdx_pattern([prob], [self.image], ws)
        return self.image

    def loss_grad(self, image):
        self.fdx.fdx_loss(image, self.target, self.mask, self.loss, self.gI, self.lws)
        return self.loss, self.gI

    def partial_grads(self, b, e, gI):
        prob, _, _, bws = self._slice(b, e)
        self.fdx.fdx_pattern_backward(prob, self.atoms, self.F[b:max(e, b + 1)], gI, self.dfrac, self.dB, self.dglob,
                                      None, bws)
        return self.dfrac, self.dB, self.dglob

    @staticmethod
    def pack(dfrac, dB, dglob):
        import torch
        return torch.cat([dfrac.reshape(-1), dB.reshape(-1), dglob.reshape(-1)])

    @staticmethod
    def unpack(packed, dfrac, dB, dglob):
        n3, n1 = dfrac.numel(), dB.numel()
        return (packed[:n3].reshape(dfrac.shape), packed[n3:n3 + n1].reshape(dB.shape),
                packed[n3 + n1:].reshape(dglob.shape))
