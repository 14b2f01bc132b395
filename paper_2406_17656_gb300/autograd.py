"""torch.autograd wrappers of the SAM build and of its residual.

`SamMap(handle, A_k, A_0, S)` is a differentiable function of the stored
values of A_k and A_0 that returns the map values M_k (CSR order):
forward = `sam_build`, backward = the hand-written adjoint kernel
(`sam_build_backward`), which recomputes each column's QR instead of storing
it.  `SamMap.residual_sq(ak, a0, m)` is ||A_k M - A_0||_F^2 (Eq. (res)) as a
differentiable function of all three; its backward returns the direct
partials, and autograd chains its dependence on M through `SamMap`.

Only argument marshalling happens here; every step runs in libsam.
"""
from __future__ import annotations

import torch

from . import sam as _sam


class _BuildFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ak_val, a0_val, owner):
        h, S = owner.handle, owner.pattern
        ak = _sam.Csr(owner.ak_rp, owner.ak_ci, ak_val.detach().contiguous(), n=owner.n)
        a0 = _sam.Csr(owner.a0_rp, owner.a0_ci, a0_val.detach().contiguous(), n=owner.n)
        tape = None
        if owner.keep_factors:
            # the build's R factors, kept for the backward (sam_set_factor_tape)
            tape = torch.empty((owner.tape_bytes() + 15) // 16 * 2, dtype=torch.float64, device=ak_val.device)
            h.sam_set_factor_tape(_sam.SAM_TAPE_RECORD, tape)
        try:
            ip, ix, mv = h.sam_build(ak, a0, S, owner.precision, owner.refine_steps)
        finally:
            if tape is not None:
                h.sam_set_factor_tape(_sam.SAM_TAPE_OFF)
        owner.indptr, owner.indices = ip, ix
        ctx.owner = owner
        ctx.tape = tape
        ctx.save_for_backward(ak_val.detach(), a0_val.detach(), mv)
        return mv

    @staticmethod
    def backward(ctx, dm):
        owner = ctx.owner
        ak_val, a0_val, mv = ctx.saved_tensors
        ak = _sam.Csr(owner.ak_rp, owner.ak_ci, ak_val.contiguous(), n=owner.n)
        a0 = _sam.Csr(owner.a0_rp, owner.a0_ci, a0_val.contiguous(), n=owner.n)
        h = owner.handle
        if ctx.tape is not None:
            h.sam_set_factor_tape(_sam.SAM_TAPE_REPLAY, ctx.tape)
        try:
            dak, da0 = h.sam_build_backward(ak, a0, owner.pattern, mv, dm.contiguous(), owner.precision,
                                            owner.refine_steps, 0.0)
        finally:
            if ctx.tape is not None:
                h.sam_set_factor_tape(_sam.SAM_TAPE_OFF)
        ctx.tape = None
        return dak, da0, None


class _ResidualSqFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ak_val, a0_val, m_val, owner):
        if owner.indptr is None:
            raise RuntimeError("build the map (call the SamMap) before its residual")
        h = owner.handle
        ak = _sam.Csr(owner.ak_rp, owner.ak_ci, ak_val.detach().contiguous(), n=owner.n)
        a0 = _sam.Csr(owner.a0_rp, owner.a0_ci, a0_val.detach().contiguous(), n=owner.n)
        m = _sam.Csr(owner.indptr, owner.indices, m_val.detach().contiguous(), n=owner.n)
        fro, _ = h.sam_residual(ak, m, a0)
        ctx.owner = owner
        ctx.save_for_backward(ak_val.detach(), a0_val.detach(), m_val.detach())
        return torch.tensor(fro * fro, dtype=torch.float64, device=ak_val.device)

    @staticmethod
    def backward(ctx, dl):
        owner = ctx.owner
        ak_val, a0_val, m_val = ctx.saved_tensors
        ak = _sam.Csr(owner.ak_rp, owner.ak_ci, ak_val.contiguous(), n=owner.n)
        a0 = _sam.Csr(owner.a0_rp, owner.a0_ci, a0_val.contiguous(), n=owner.n)
        dmres = torch.empty_like(m_val)
        dak, da0 = owner.handle.sam_build_backward(ak, a0, owner.pattern, m_val.contiguous(), None, owner.precision,
                                                   owner.refine_steps, float(dl), dM_resid=dmres)
        return dak, da0, dmres, None


class _ApplyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m_val, v, owner):
        if owner.indptr is None:
            raise RuntimeError("build the map (call the SamMap) before applying it")
        m = _sam.Csr(owner.indptr, owner.indices, m_val.detach().contiguous(), n=owner.n)
        vv = v.detach().contiguous()
        y = owner.handle.sam_apply(m, vv)
        ctx.owner = owner
        ctx.save_for_backward(vv)
        return y

    @staticmethod
    def backward(ctx, dy):
        owner = ctx.owner
        (vv,) = ctx.saved_tensors
        m = _sam.Csr(owner.indptr, owner.indices, None, n=owner.n)
        return owner.handle.sam_apply_grad(m, vv, dy.contiguous()), None, None


class SamMap:
    """Differentiable SAM on a fixed pattern.

    handle: sam.Handle; ak_struct / a0_struct: (indptr, indices) int32 device
    tensors of A_k and A_0; pattern: sam.Pattern (e.g. from
    handle.sam_pattern_build); precision "fp32r" (FP32 QR + FP64 refinement)
    or "fp64".  keep_factors: the forward keeps the column problems' R
    factors in device memory for the backward (a factor tape), which then
    skips the QR; the gradients are the same."""

    def __init__(self, handle, ak_struct, a0_struct, pattern, precision="fp32r", refine_steps=1,
                 keep_factors=False):
        self.handle, self.pattern = handle, pattern
        self.ak_rp, self.ak_ci = ak_struct
        self.a0_rp, self.a0_ci = a0_struct
        self.n = int(self.ak_rp.shape[0] - 1)
        self.precision, self.refine_steps = precision, refine_steps
        self.keep_factors = keep_factors
        self._tape_bytes = None
        self.indptr = self.indices = None

    def tape_bytes(self):
        if self._tape_bytes is None:
            self._tape_bytes = self.handle.sam_factor_tape_bytes([self.pattern], self.precision)
        return self._tape_bytes

    def __call__(self, ak_val, a0_val):
        return _BuildFn.apply(ak_val, a0_val, self)

    def residual_sq(self, ak_val, a0_val, m_val):
        return _ResidualSqFn.apply(ak_val, a0_val, m_val, self)

    def matvec(self, m_val, v):
        """M v as a differentiable function of the map values (sam_apply
        forward, sam_apply_grad backward; v is a constant)."""
        return _ApplyFn.apply(m_val, v, self)
