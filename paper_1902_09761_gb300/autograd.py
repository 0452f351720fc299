"""torch.autograd bridge for checkpointed APFC rollouts.

``Rollout(...)(eta0, dB)`` returns (eta^n, F(eta^n)) after n steps of size dt
of the library's step (Alg. 1 with one nonlinear iterate, nonlinear term
explicit), as a differentiable function of the initial amplitudes eta0
(complex128 or complex64, host or CUDA tensor; complex64 is converted by the
library on the device) and of dB (a real tensor).  The
backward pass is the library's checkpointed adjoint (``apfc_rollout_backward``:
one adjoint solve per step with the Hermitian Schur complement, the adjoint of
the nonlinear term with both Wirtinger derivatives, and the dB derivative
through S); the free-energy term uses ``apfc_energy_gradient``.  Everything
numerical runs in libapfc; this module only moves buffers and chains the two
outputs' gradients.  Gradients follow PyTorch's complex convention
(dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch

from . import apfc as A


class Rollout:
    """Differentiable n-step rollout on one grid (owns a library context)."""

    def __init__(self, k, kind, params, shape, h, dt: float, n: int, every: int = 20, opts=None, device=None):
        self.params = params if isinstance(params, A.Params) else A.make_params(*params)
        self.dt, self.n, self.every = float(dt), int(n), int(every)
        self.device = torch.device(device) if device is not None else None
        stream = None
        if self.device is not None and self.device.type == "cuda":
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = A.Context(k, kind, self.params, shape, h, opts, stream=stream)
        self.shape = self.ctx.amp_shape

    def close(self):
        self.ctx.close()

    def __call__(self, eta0: torch.Tensor, dB: torch.Tensor):
        return _RolloutFn.apply(eta0, dB, self)

    # host/device marshalling
    def _view(self, t: torch.Tensor):
        return t if t.is_cuda else t.numpy()

    def _empty(self, like: torch.Tensor, dtype=torch.complex128):
        return torch.empty(self.shape, dtype=dtype, device=like.device)


class _RolloutFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, eta0, dB, ro: Rollout):
        # complex64 and complex128 inputs go to the library as they are (it converts on the
        # device); the output comes back in the input's type, and the final state in
        # complex128 is kept for the energy gradient of the backward pass
        e0 = eta0.detach().contiguous()
        if e0.dtype not in (torch.complex64, torch.complex128):
            raise TypeError("eta0 must be complex64 or complex128")
        if tuple(e0.shape) != tuple(ro.shape):
            raise ValueError(f"eta0 has shape {tuple(e0.shape)}, expected {tuple(ro.shape)}")
        p = ro.params
        ro.ctx.set_params((float(dB), p.Bx, p.t, p.v))
        ro.ctx.set_amplitudes(ro._view(e0))
        ro.ctx.rollout_forward(ro.dt, ro.n, ro.every)
        etaN = ro._empty(e0)
        ro.ctx.get_amplitudes(ro._view(etaN))
        out = etaN
        if e0.dtype == torch.complex64:
            out = ro._empty(e0, torch.complex64)
            ro.ctx.get_amplitudes(ro._view(out))
        F = ro.ctx.energy()
        fctx.ro = ro
        fctx.in_dtype = eta0.dtype
        fctx.dB_meta = (dB.shape, dB.dtype, dB.device) if isinstance(dB, torch.Tensor) else None
        fctx.save_for_backward(etaN)
        return out, torch.tensor(F, dtype=torch.float64, device=e0.device)

    @staticmethod
    def backward(fctx, g_eta, g_F):
        ro = fctx.ro
        (etaN,) = fctx.saved_tensors
        lam = torch.zeros_like(etaN) if g_eta is None else g_eta.detach().to(torch.complex128).contiguous()
        d_dB = 0.0
        gF = 0.0 if g_F is None else float(g_F)
        if gF != 0.0:
            gradF = ro._empty(etaN)
            _, dF = ro.ctx.energy_gradient(ro._view(etaN), ro._view(gradF))
            lam = lam + gF * gradF
            d_dB += gF * dF
        lam0 = ro._empty(etaN)
        _, d = ro.ctx.rollout_backward(ro._view(lam.contiguous()), ro._view(lam0))
        d_dB += d
        g_dB = None
        if fctx.dB_meta is not None:
            shape, dtype, device = fctx.dB_meta
            g_dB = torch.full(shape, d_dB, dtype=dtype, device=device)
        return lam0.to(fctx.in_dtype), g_dB, None
