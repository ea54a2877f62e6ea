"""torch.autograd bindings of the adjoint: one RK4 step and the initial data (prim->cons with B~ = curl A) as
differentiable functions of device state tensors.  The backward passes call the library's adjoint entry points
(asterx_rk4_step_adjoint from a checkpoint of the step's input, asterx_prim2con_adjoint); nothing is computed
here.  Gradients cover the independent entries of the state (zero elsewhere)."""
import torch


class RK4Step(torch.autograd.Function):
    """U_{n+1} = one classical RK4 step of U_n (9 state fields) with `solver` (an asterx.Solver).  P is the
    primitive buffer the recovery uses as its guess and overwrites (not differentiated)."""

    @staticmethod
    def forward(ctx, U, solver, P, dt):
        ckpt = U.detach().clone()
        out = U.detach().clone()
        solver.rk4_step(out, P, dt)
        ctx.solver, ctx.P, ctx.dt = solver, P, float(dt)
        ctx.save_for_backward(ckpt)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (ckpt,) = ctx.saved_tensors
        lam = grad_out.detach().clone().contiguous()
        guess = ctx.P.detach().clone()
        ctx.solver.rk4_step_adjoint(ckpt, guess, lam, ctx.dt)
        return lam, None, None, None


class InitialData(torch.autograd.Function):
    """U_0 = (prim2con(P, B~ = curl A), A, Psi): the conserved variables of primitives P (5 fields) with the
    potentials A, Psi taken from the state-shaped tensor `pot` (its hydro fields are ignored)."""

    @staticmethod
    def forward(ctx, P, pot, solver):
        U = pot.detach().clone()
        U[:5].zero_()
        solver.fill_ghosts(U)
        Pc = P.detach().contiguous()
        solver.prim2con(U, Pc)
        ctx.solver = solver
        ctx.save_for_backward(Pc, U)
        return U

    @staticmethod
    def backward(ctx, grad_out):
        Pc, U = ctx.saved_tensors
        lam = grad_out.detach().clone().contiguous()
        lamP = torch.zeros_like(Pc)
        ctx.solver.prim2con_adjoint(U, Pc, lam, lamP)
        return lamP, lam, None
