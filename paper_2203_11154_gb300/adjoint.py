"""Differentiable ParaDIAG step: a torch.autograd.Function around paradiag_solve.

Forward: u solves (B kron I_h + kappa I_t kron A) u = f + u0_coef kron u0 (eq. (1) with A
scaled by a diffusion coefficient kappa), B the alpha-circulant backward-Euler matrix.
Backward (the adjoint): with g = dJ/du,
    w = (B^T kron I_h + kappa I_t kron A)^{-1} g,
solved by the same multigrid through the adjoint context (pd_adjoint_setup: shifted
systems kappa A + conj(lam_j) I, transforms V^H and V^{-H}); then
    dJ/df = w,   dJ/du0 = sum_k u0_coef[k] w_k,   dJ/dkappa = -sum_k <w_k, A u_k>.
The backward needs only u from the forward solve (the solve is linear, its adjoint is
another solve), so no multigrid state is stored or recomputed.  Every arithmetic step
runs in the library's kernels; this module only marshals tensors.
"""
import torch

from . import api


class HeatStep:
    """Contexts (forward and adjoint, one pair per kappa) of one problem size."""

    def __init__(self, N, n, tau, alpha, precision=0, **cfg):
        self.N, self.n, self.tau, self.alpha = int(N), int(n), float(tau), float(alpha)
        self.B, self.shifts, self.V, self.Vinv, self.u0_coef = api.pd_alpha_circulant(n, tau, alpha)
        self.precision = precision
        self.cfg = cfg
        self._ctx = {}

    def contexts(self, kappa):
        key = float(kappa)
        if key not in self._ctx:
            cfg = api.config(precision=self.precision, kappa=key, **self.cfg)
            fwd = api.Context(self.N, self.n, self.shifts, self.V, self.Vinv, self.B, self.u0_coef,
                              cfg=cfg)
            self._ctx[key] = (fwd, fwd.adjoint())
        return self._ctx[key]

    def __call__(self, f, u0, kappa):
        """u for f [n][N][N], u0 [N][N] (float64 CUDA tensors) and a scalar tensor kappa."""
        return _HeatSolve.apply(f, u0, kappa, self)


class _HeatSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, u0, kappa, step):
        fwd, _ = step.contexts(float(kappa))
        u = torch.empty_like(f)
        fwd.paradiag_solve(u, f.contiguous(), u0.contiguous())
        ctx.save_for_backward(u)
        ctx.step = step
        ctx.kappa = float(kappa)
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        fwd, adj = ctx.step.contexts(ctx.kappa)
        w = torch.empty_like(u)
        adj.paradiag_solve(w, gu.contiguous(), None)
        gf = w if ctx.needs_input_grad[0] else None
        gu0 = None
        if ctx.needs_input_grad[1]:
            gu0 = torch.empty(u.shape[1:], dtype=u.dtype, device=u.device)
            fwd.pd_initial_value_gradient(w, gu0)
        gk = None
        if ctx.needs_input_grad[2]:
            gk = torch.tensor(-fwd.pd_laplacian_dot(w, u), dtype=u.dtype, device=u.device)
        return gf, gu0, gk, None
