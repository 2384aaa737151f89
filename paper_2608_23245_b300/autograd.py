"""torch.autograd wrapper of the fiber-diffraction path.

`FiberPattern.apply(frac, B, L, g, sigma, gamma, model)` returns the detector
image; its backward calls the hand-written adjoint (fdx_pattern_backward),
which recomputes the per-reflection profiles instead of storing them (only F
and M from the forward are kept).  Differentiable inputs:

    frac   [n_atoms, 3] float64 CUDA   fractional coordinates
    B      [n_atoms]    float32 CUDA   isotropic B (A^2)
    L, g   [3]          float64 CPU    crystallite sizes (A), Hosemann g
    sigma, gamma  []    float64 CPU    orientation widths (rad)

Everything else (cell, elements, form factors, occupancies, reflection list,
geometry, quadrature settings, patch extent T) is held fixed by `RefineModel`.
All arithmetic runs in libfdx; this module only marshals arguments.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import fdx


class RefineModel:
    """Fixed parts of one refinement problem, resident on the device."""

    def __init__(self, problem, device="cuda"):
        import torch
        self.problem = problem
        self.device = device
        self.hkl_host = fdx.fdx_reflections(problem.cell, problem.d_min, problem.d_max)
        self.hkl = torch.as_tensor(self.hkl_host, device=device).contiguous()
        a = problem.atoms
        self.occ = torch.as_tensor(np.ascontiguousarray(a.occ, np.float32), device=device)
        self.elem = torch.as_tensor(np.ascontiguousarray(a.elem, np.uint8), device=device)
        self.ff = torch.as_tensor(np.ascontiguousarray(a.ff, np.float32).reshape(-1, 9), device=device)
        n = int(self.hkl.shape[0])
        self.F = torch.empty((n, 2), dtype=torch.float32, device=device)
        self.M = torch.empty((n,), dtype=torch.float32, device=device)
        self.image = torch.empty((problem.geom.n_y, problem.geom.n_x), dtype=torch.float32, device=device)
        self.sf_ws = torch.empty(max(fdx.fdx_sf_workspace_size(a.n, n), 256), dtype=torch.uint8, device=device)
        prob = self.struct(problem.br)
        self.ws = torch.empty(max(fdx.fdx_workspace_size([prob]), 256), dtype=torch.uint8, device=device)
        self.bws = torch.empty(max(fdx.fdx_backward_workspace_size(prob, a.n, self.ff.shape[0]), 256),
                               dtype=torch.uint8, device=device)

    def initial(self):
        """The problem's own parameters as tensors (frac, B, L, g, sigma, gamma)."""
        import torch
        a, br = self.problem.atoms, self.problem.br
        return (torch.as_tensor(np.ascontiguousarray(a.frac, np.float64), device=self.device),
                torch.as_tensor(np.ascontiguousarray(a.B, np.float32), device=self.device),
                torch.tensor(br.L, dtype=torch.float64), torch.tensor(br.g, dtype=torch.float64),
                torch.tensor(br.sigma, dtype=torch.float64), torch.tensor(br.gamma, dtype=torch.float64))

    def broadening(self, L, g, sigma, gamma):
        br = self.problem.br
        return replace(br, L=tuple(float(x) for x in L), g=tuple(float(x) for x in g), sigma=float(sigma),
                       gamma=float(gamma))

    def struct(self, br):
        return fdx.make_problem(self.problem.cell, br, self.problem.geom, self.hkl, self.M)

    def atoms_struct(self, frac, B):
        a = fdx.Atoms()
        a.n_atoms, a.n_elem = int(frac.shape[0]), int(self.ff.shape[0])
        a.frac, a.B, a.occ = frac.data_ptr(), B.data_ptr(), self.occ.data_ptr()
        a.elem, a.ff = self.elem.data_ptr(), self.ff.data_ptr()
        return a


class _AtomsView:
    """Adapter giving fdx_* functions the DeviceAtoms interface for given tensors."""

    def __init__(self, model, frac, B):
        self._s = model.atoms_struct(frac, B)
        self.frac = frac

    def struct(self):
        return self._s


def _check_inputs(frac, B):
    import torch
    if frac.dtype != torch.float64 or not frac.is_cuda or frac.dim() != 2 or frac.shape[1] != 3:
        raise TypeError("frac must be a CUDA float64 tensor [n_atoms, 3]")
    if B.dtype != torch.float32 or not B.is_cuda or B.shape[0] != frac.shape[0]:
        raise TypeError("B must be a CUDA float32 tensor [n_atoms]")


def _function():
    import torch

    class FiberPattern(torch.autograd.Function):
        @staticmethod
        def forward(ctx, frac, B, L, g, sigma, gamma, model):
            _check_inputs(frac, B)
            frac, B = frac.contiguous(), B.contiguous()
            br = model.broadening(L.tolist(), g.tolist(), sigma.item(), gamma.item())
            view = _AtomsView(model, frac, B)
            F = torch.empty_like(model.F)
            M = torch.empty_like(model.M)
            fdx.fdx_structure_factors(model.problem.cell, view, model.hkl, br, F, M, model.sf_ws)
            prob = fdx.make_problem(model.problem.cell, br, model.problem.geom, model.hkl, M)
            image = torch.empty_like(model.image)
            fdx.fdx_pattern([prob], [image], model.ws)
            ctx.save_for_backward(frac, B, F, M)
            ctx.model, ctx.br = model, br
            return image

        @staticmethod
        def backward(ctx, gI):
            frac, B, F, M = ctx.saved_tensors
            model, br = ctx.model, ctx.br
            gI = gI.contiguous().to(torch.float32)
            prob = fdx.make_problem(model.problem.cell, br, model.problem.geom, model.hkl, M)
            view = _AtomsView(model, frac, B)
            dfrac = torch.empty_like(frac) if ctx.needs_input_grad[0] else None
            dB64 = torch.empty(B.shape, dtype=torch.float64, device=B.device) if ctx.needs_input_grad[1] else None
            dglob = torch.empty(8, dtype=torch.float64, device=frac.device)
            fdx.fdx_pattern_backward(prob, view, F, gI, dfrac, dB64, dglob, None, model.bws)
            dglob = dglob.cpu()
            dB = dB64.to(B.dtype) if dB64 is not None else None
            return (dfrac, dB, dglob[0:3].clone(), dglob[3:6].clone(), dglob[6].clone(), dglob[7].clone(), None)

    return FiberPattern


_FN = None


def fiber_pattern(frac, B, L, g, sigma, gamma, model):
    """Differentiable detector image (see module docstring)."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(frac, B, L, g, sigma, gamma, model)


def refinement_loss(image, target, mask=None):
    """Differentiable L = sum m (I - I_t)^2 / (I_t + 1) through fdx_loss."""
    import torch

    class _Loss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, I):
            gI = torch.empty_like(I)
            loss, _ = fdx.fdx_loss(I.contiguous(), target.contiguous(), mask, dL_dI=gI)
            ctx.save_for_backward(gI)
            return loss

        @staticmethod
        def backward(ctx, gl):
            (gI,) = ctx.saved_tensors
            return gI * gl.to(gI.dtype)

    return _Loss.apply(image)
