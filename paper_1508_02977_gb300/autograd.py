"""torch.autograd.Function over of_solve / of_adjoint.

    U = ofsolve_fn(f1, f2, alpha, solver)

U solves the P1 system of Section 2.2 for one frame pair; backward solves
the adjoint system (the operator is symmetric, so it is the same solve with
dL/dU as right-hand side) and forms dL/dalpha per element and dL/df1,
dL/df2 per pixel in the CUDA library.  Only marshalling happens here.
"""
from __future__ import annotations

import torch

from . import ofsolve as S


class Solver:
    """A handle set up for frames of one size (W, H), kept between calls."""

    def __init__(self, W: int, H: int, device: int = 0, precision: int = S.OF_PREC_MIXED, tile=(48, 48),
                 overlap: int = 0, sweeps: int = 4, lam: float = 1.0, rtol: float = 1e-6, omega: float = 1.6,
                 sigma: float = 0.0, rho: float = 0.0, model: int = S.OF_MODEL_ILLUMINATION, coarse: int = 0):
        """sigma, rho: K_sigma pre-smoothing and K_rho integration scales of
        Section 1 (gradients are w.r.t. the frames given to forward);
        model: OF_MODEL_ILLUMINATION or OF_MODEL_CONSTANT; coarse: two-level
        preconditioner spacing (0: one level)."""
        self.W, self.H, self.rtol = int(W), int(H), float(rtol)
        self.precision = precision
        self.h = S.of_create(device)
        S.of_setup_grid(self.h, [(self.W, self.H)], tile=tile, overlap=overlap, sweeps=sweeps,
                        precision=precision, lam=lam, omega=omega, sigma=sigma, rho=rho, model=model,
                        coarse=coarse)

    def close(self):
        if self.h is not None:
            S.of_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class OFSolve(torch.autograd.Function):
    """U = A(f1, f2, alpha)^{-1} b(f1, f2): forward of_solve, backward
    of_adjoint (implicit differentiation)."""

    @staticmethod
    def forward(ctx, f1, f2, alpha, solver: Solver):
        dt = torch.float64 if solver.precision == S.OF_PREC_FP64 else torch.float32
        f1c = f1.detach().to(dt).contiguous()
        f2c = f2.detach().to(dt).contiguous()
        S.of_set_frames(solver.h, 0, f1c, f2c)
        S.of_set_alpha(solver.h, 0, alpha.detach().to(dt).contiguous())
        U = torch.zeros(3, solver.H, solver.W, dtype=torch.float64, device=f1.device)
        S.of_solve(solver.h, [U], rtol=solver.rtol)
        ctx.solver = solver
        ctx.in_dtypes = (f1.dtype, f2.dtype, alpha.dtype)
        # the handle keeps only its last solve: backward re-solves if another
        # forward used the same solver in between
        solver._token = object()
        ctx.token = solver._token
        ctx.save_for_backward(f1c, f2c, alpha.detach().to(dt).contiguous())
        return U.to(f1.dtype)

    @staticmethod
    def backward(ctx, gU):
        solver = ctx.solver
        dev = gU.device
        if getattr(solver, "_token", None) is not ctx.token:
            f1c, f2c, ac = ctx.saved_tensors
            S.of_set_frames(solver.h, 0, f1c, f2c)
            S.of_set_alpha(solver.h, 0, ac)
            U = torch.zeros(3, solver.H, solver.W, dtype=torch.float64, device=dev)
            S.of_solve(solver.h, [U], rtol=solver.rtol)
            solver._token = ctx.token
        gU = gU.detach().to(torch.float64).contiguous()
        da = torch.zeros(solver.H - 1, solver.W - 1, 2, dtype=torch.float64, device=dev)
        d2 = torch.zeros(solver.H, solver.W, dtype=torch.float64, device=dev)
        d1 = torch.zeros_like(d2)
        need = ctx.needs_input_grad
        S.of_adjoint(solver.h, [gU], [da] if need[2] else None, [d2] if need[1] else None,
                     [d1] if need[0] else None)
        t1, t2, ta = ctx.in_dtypes
        return (d1.to(t1) if need[0] else None, d2.to(t2) if need[1] else None,
                da.to(ta) if need[2] else None, None)


def ofsolve_fn(f1, f2, alpha, solver: Solver):
    return OFSolve.apply(f1, f2, alpha, solver)


class OFAdaptSolve(torch.autograd.Function):
    """U_K after `npasses` adaptation passes (Section 2.3 on the fixed mesh:
    solve, error indicator, alpha update) and a final solve, differentiated
    through every pass.  Forward keeps a checkpoint (alpha_k, U_k) per pass;
    backward walks them in reverse: re-establish pass k (alpha_k and a warm
    solve from U_k, which converges at once), of_adjoint for the solve, then
    of_adapt_alpha_vjp for the indicator and update that produced
    alpha_{k+1}; its dL/dU_k is the next adjoint's input."""

    @staticmethod
    def forward(ctx, f1, f2, alpha0, solver: Solver, npasses: int, kappa: float, eta_thr: float,
                alpha_th: float):
        dt = torch.float64 if solver.precision == S.OF_PREC_FP64 else torch.float32
        dev = f1.device
        f1c = f1.detach().to(dt).contiguous()
        f2c = f2.detach().to(dt).contiguous()
        S.of_set_frames(solver.h, 0, f1c, f2c)
        a = alpha0.detach().to(torch.float64).contiguous()
        ckpt = []
        for _ in range(int(npasses)):
            S.of_set_alpha(solver.h, 0, a.to(dt).contiguous())
            Uk = torch.zeros(3, solver.H, solver.W, dtype=torch.float64, device=dev)
            S.of_solve(solver.h, [Uk], rtol=solver.rtol)
            S.of_adapt_alpha(solver.h, kappa, eta_thr, alpha_th)
            a_next = torch.zeros_like(a)
            S.of_get_alpha(solver.h, 0, a_next)
            ckpt.append((a, Uk))
            a = a_next
        S.of_set_alpha(solver.h, 0, a.to(dt).contiguous())
        U = torch.zeros(3, solver.H, solver.W, dtype=torch.float64, device=dev)
        S.of_solve(solver.h, [U], rtol=solver.rtol)
        ctx.solver, ctx.ckpt, ctx.final = solver, ckpt, (a, U.clone())
        ctx.frames = (f1c, f2c)
        ctx.params = (float(kappa), float(eta_thr), float(alpha_th))
        ctx.in_dtypes = (f1.dtype, f2.dtype, alpha0.dtype)
        return U.to(f1.dtype)

    @staticmethod
    def backward(ctx, gU):
        solver = ctx.solver
        dt = torch.float64 if solver.precision == S.OF_PREC_FP64 else torch.float32
        dev = gU.device
        kappa, thr, ath = ctx.params
        S.of_set_frames(solver.h, 0, *ctx.frames)

        def at_pass(a, Uk):  # alpha_k and the solution that belongs to it
            S.of_set_alpha(solver.h, 0, a.to(dt).contiguous())
            Uw = Uk.clone()
            S.of_solve(solver.h, [Uw], rtol=solver.rtol, warm_start=True)

        H, W = solver.H, solver.W
        z_a = lambda: torch.zeros(H - 1, W - 1, 2, dtype=torch.float64, device=dev)
        z_f = lambda: torch.zeros(H, W, dtype=torch.float64, device=dev)
        a, U = ctx.final
        at_pass(a, U)
        v, d2, d1 = z_a(), z_f(), z_f()
        S.of_adjoint(solver.h, [gU.detach().to(torch.float64).contiguous()], [v], [d2], [d1])
        for a, Uk in reversed(ctx.ckpt):
            at_pass(a, Uk)
            da, e2, e1 = z_a(), z_f(), z_f()
            dU = torch.zeros(3, H, W, dtype=torch.float64, device=dev)
            S.of_adapt_alpha_vjp(solver.h, kappa, thr, ath, [v], [da], [dU], [e2], [e1])
            ga, g2, g1 = z_a(), z_f(), z_f()
            S.of_adjoint(solver.h, [dU], [ga], [g2], [g1])
            v = da + ga
            d2 = d2 + e2 + g2
            d1 = d1 + e1 + g1
        t1, t2, ta = ctx.in_dtypes
        return d1.to(t1), d2.to(t2), v.to(ta), None, None, None, None, None


def adapt_solve_fn(f1, f2, alpha0, solver: Solver, npasses: int, kappa: float, eta_thr: float, alpha_th: float):
    return OFAdaptSolve.apply(f1, f2, alpha0, solver, npasses, kappa, eta_thr, alpha_th)
