"""torch.autograd bridge to the discrete adjoint of libg1g2 (g1g2_adjoint).

`final_time_objective(drive_params, wscale, h, problem, ..., w=None)` returns a
0-d tensor J that autograd can differentiate with respect to the drive
parameters, the interaction scale s (w -> s w), the one-body matrix h and,
when w is given as a tensor, the entries of the interaction w.  The forward pass
propagates nsteps RK4 steps of the FP64 form in the CUDA library and the
backward pass hands back the gradients the library's reverse sweep computed
(one forward + one checkpointed reverse sweep per call; nothing is taped).
Argument marshalling only: no part of the G1-G2 equations runs here.

Conventions:
  * h must be Hermitian; its gradient follows torch's convention for a real
    loss of a complex leaf (dJ/dRe h + i dJ/dIm h) restricted to Hermitian
    perturbations, i.e. the Hermitian matrix G with dJ = Re sum conj(G) dh.
  * The library differentiates w -> s' w at s' = 1; for the problem's w scaled
    by s that is s dJ/ds, so s must be non-zero.
  * w (complex128 or float64, nb^4, with w_ijkl = w_jilk = conj(w_klij)) gets the
    library's gradient on that symmetric subspace (for a complex leaf in torch's
    convention dJ/dRe w + i dJ/dIm w, for a real leaf its real part): exact for
    every perturbation that keeps the symmetries, e.g. through a parameterisation
    such as w = sum_P L^P (x) L^P.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs
from .g1g2 import Propagator

OBJECTIVES = {"double_occupancy": 0, "imbalance": 1, "energy_absorbed": 2}


def _drive(problem, params):
    kind = problem.get("drive_kind", 2)
    p = params.detach().cpu().numpy().astype(np.float64)
    if kind == 2:
        return inputs.PiecewiseLinear(p, problem["ta"], problem["tb"])
    if kind == 1:
        if p.shape != (4,):
            raise ValueError("gauss-sine drive takes (A, omega, t0, sigma)")
        return inputs.GaussSine(*p)
    raise ValueError(f"unknown drive kind {kind}")


class FinalTimeObjective(torch.autograd.Function):
    """J(theta, s, h) of a final-time observable after nsteps RK4 steps (FP64 form, any fermion selfenergy
    in a general basis)."""

    @staticmethod
    def forward(ctx, drive_params, wscale, h, w, problem, dt, nsteps, objective, ckpt_every):
        s = float(wscale)
        if s == 0.0:
            raise ValueError("the w scale must be non-zero")
        hh = h.detach().cpu().numpy().astype(np.complex128)
        ww = problem["w"] if w is None else w.detach().cpu().numpy().astype(np.complex128)
        p = Propagator(hh, s * ww, problem["n0"], problem.get("G2_0"), problem.get("selfenergy", "SOA"), "fp64",
                       restricted=problem.get("restricted", False))
        try:
            p.set_drive(problem["D"], _drive(problem, drive_params))
            res = p.adjoint(dt, nsteps, objective=OBJECTIVES.get(objective, objective), ckpt_every=ckpt_every,
                            n_drive_params=drive_params.numel(), grad_w=w is not None)
        finally:
            p.close()
        J, gd, gws, gh = res[:4]
        # dJ/dw for the library's interaction s w is s times its gradient at s w
        gw = torch.as_tensor(s * res[4]) if w is not None else torch.zeros(())
        if w is not None and not w.is_complex():
            gw = gw.real
        ctx.w_given = w is not None
        ctx.save_for_backward(torch.as_tensor(gd, dtype=drive_params.dtype).reshape(drive_params.shape),
                              torch.tensor(gws / s, dtype=torch.float64),
                              torch.as_tensor(gh, dtype=torch.complex128), gw)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        gd, gws, gh, gw = ctx.saved_tensors
        gw_out = gJ * gw if ctx.w_given else None
        return gJ * gd, gJ * gws, (gJ * gh).to(torch.complex128), gw_out, None, None, None, None, None


def final_time_objective(drive_params, wscale, h, problem, dt, nsteps, objective="double_occupancy", ckpt_every=0,
                         w=None):
    """Differentiable J; `problem` holds w, n0, D, drive_kind (1 or 2), ta/tb, selfenergy, restricted, G2_0.
    A tensor w replaces problem["w"] and receives a gradient."""
    if not torch.is_tensor(wscale):
        wscale = torch.tensor(float(wscale), dtype=torch.float64)
    return FinalTimeObjective.apply(drive_params, wscale, h, w, problem, dt, nsteps, objective, ckpt_every)
