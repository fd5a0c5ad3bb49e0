"""torch.autograd.Function around the CUDA solver and its adjoint.

Forward: V = (H H^H + xi I)^-1 S and X = H^H V by VR-OAHK (kz_precode).
Backward: kz_precode_adjoint runs the same Kaczmarz operator on the adjoint
system and contracts the gradients with respect to the packed H (VR entries
only), xi and S on the GPU.  Gradients follow PyTorch's convention for
complex tensors (the first-order change of a real loss is Re sum conj(G) dZ).

Tensors: H_packed complex64 (sum vr_len,), S complex64 (nrhs, K) (column j
of the K x nrhs right-hand-side matrix is row j), outputs X (nrhs, Nt) and
V (nrhs, K); everything on one CUDA device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import kzprecode as kp


class KzPrecodeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H_packed, xi, S, vr_offset, vr_len, Nt, tol, max_iter):
        K = len(vr_len)
        plan = kp.kz_plan_create(K, Nt, vr_offset, vr_len, H_packed.detach().contiguous())
        xi_f = float(xi)
        out = kp.precode(plan, S.detach().contiguous(), xi_f, algo="vr_oahk", tol=tol, max_iter=max_iter)
        if not out["converged"]:
            raise kp.KzError(kp.KZ_NOT_CONVERGED, "forward solve did not converge")
        ctx.plan = plan
        ctx.xi = xi_f
        ctx.tol, ctx.max_iter = tol, max_iter
        ctx.xi_is_tensor = isinstance(xi, torch.Tensor)
        ctx.save_for_backward(out["x"], out["v"])
        return out["x"], out["v"]

    @staticmethod
    def backward(ctx, gX, gV):
        X, V = ctx.saved_tensors
        plan = ctx.plan
        nrhs = V.shape[0]
        dev = V.device
        lam = torch.empty_like(V)
        y = torch.empty_like(X)
        gH = torch.empty(plan.sum_len, dtype=torch.complex64, device=dev)
        gxi = torch.empty(1, dtype=torch.float32, device=dev)
        iters = torch.empty(nrhs, dtype=torch.int32, device=dev)
        resid = torch.empty(nrhs, dtype=torch.float64, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        gX = gX.contiguous() if gX is not None else None
        gV = gV.contiguous() if gV is not None else None
        if gX is None and gV is None:
            return None, None, None, None, None, None, None, None
        kp.kz_precode_adjoint(plan, nrhs, ctx.xi, V, X, gV, gX, ctx.tol, ctx.max_iter, lam, y, gH, gxi, iters,
                              resid, status)
        grad_xi = gxi.reshape(()) if ctx.xi_is_tensor else None
        return gH, grad_xi, lam, None, None, None, None, None


def precode(H_packed, xi, S, vr_offset, vr_len, Nt, tol=1e-7, max_iter=2000):
    """Differentiable (X, V) = (H^H V, (H H^H + xi I)^-1 S)."""
    return KzPrecodeFn.apply(H_packed, xi, S, np.asarray(vr_offset, np.int32), np.asarray(vr_len, np.int32),
                             int(Nt), float(tol), int(max_iter))


def sum_rate_loss(H_dense, X, snr_lin):
    """-sum_k log2(1 + SINR_k) of eq. (rate) for F = X / ||X||_F (X: nrhs x Nt, one
    column of the precoder per user, i.e. nrhs = K with identity symbols)."""
    F = X.transpose(0, 1) / torch.linalg.norm(X)
    G = H_dense @ F
    sig = torch.abs(torch.diagonal(G)) ** 2
    tot = torch.sum(torch.abs(G) ** 2, dim=1)
    sinr = sig / (tot - sig + 1.0 / snr_lin)
    return -torch.sum(torch.log2(1.0 + sinr))


def dense_from_packed(H_packed, vr_offset, vr_len, Nt):
    """K x Nt matrix from the packed rows (differentiable gather; tensor ops only)."""
    K = len(vr_len)
    idx_rows, idx_cols = [], []
    for k in range(K):
        idx_rows += [k] * int(vr_len[k])
        idx_cols += list(range(int(vr_offset[k]), int(vr_offset[k]) + int(vr_len[k])))
    H = torch.zeros((K, Nt), dtype=H_packed.dtype, device=H_packed.device)
    r = torch.tensor(idx_rows, device=H_packed.device)
    c = torch.tensor(idx_cols, device=H_packed.device)
    return H.index_put((r, c), H_packed)
