"""Differentiable compliance through the PA solve.

For A(kappa) u = b with b independent of the per-element coefficient
kappa, the compliance J = b^T u has the adjoint state lambda = u (A is
symmetric positive definite), so dJ/dkappa_e = -u^T (dA/dkappa_e) u =
-u_e^T Khat_e u_e. The forward pass runs the library's setup kernel for the
new coefficient, its Jacobi-PCG solve and its deterministic dot product; the
backward pass runs the library's adjoint kernel (fem_compliance_grad).
Autograd only chains the result with the caller's coefficient model
(e.g. kappa = 0.01 + rho^3).
"""

import torch


class _Compliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, form, b, rtol, maxit, precision):
        form.set_coef(kappa.detach().to(torch.float64).contiguous())
        u = torch.zeros_like(b)
        form.solve(b, u, rtol=rtol, maxit=maxit, precision=precision)
        J = form.compliance(b, u)
        ctx.form = form
        ctx.save_for_backward(u)
        ctx.mark_non_differentiable(u)
        return J.reshape(()), u

    @staticmethod
    def backward(ctx, gJ, gu):
        (u,) = ctx.saved_tensors
        g = torch.empty(ctx.form.space.ne, dtype=torch.float64, device=u.device)
        ctx.form.compliance_grad(u, g)
        return gJ * g, None, None, None, None, None


def compliance(kappa, form, b, rtol=1e-12, maxit=20000, precision="f64"):
    """J(kappa) = b^T u(kappa) with A_c(kappa) u = b (b: constrained right-hand
    side with homogeneous essential values; call form.set_essential first).
    Returns (J, u); J is differentiable with respect to kappa."""
    return _Compliance.apply(kappa, form, b, rtol, maxit, precision)
