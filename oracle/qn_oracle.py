"""FP64 CPU oracle for the quasi-Newton acceleration of the MM map.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this module.  The CUDA
library never calls it, and it never calls the CUDA library.

Source: the paper's Section 4 names the quasi-Newton acceleration of Zhou,
Alexander & Lange (its reference ZhouAlexanderLange09QN) as the remedy for
the MM algorithms' slow convergence, reports it on the CPU for PET and MDS,
and says its GPU attempts were mixed, suspecting single precision.  The
scheme accelerates any smooth algorithm map F towards a fixed point
x = F(x): from secant pairs u_i = F(x_i) - x_i, v_i = F(F(x_i)) - F(x_i)
(the last q, as columns of U and V) the Jacobian of F at the fixed point is
approximated by M = V (U^T U)^-1 U^T, and a Newton step for x - F(x) = 0
with I - M inverted by the Woodbury identity gives

    x_{n+1} = F(x_n) + V (U^T U - U^T V)^-1 U^T u_n,   u_n = F(x_n) - x_n.

Readings taken here (each listed in the design notes):
  * F is one MM iteration of the model (both factors, as nmf_step does), and
    x stacks W and H;
  * every iteration evaluates F(x_n) and F(F(x_n)) and adds the pair to the
    memory (dropping the oldest beyond q);
  * safeguard: the quasi-Newton point is taken only when all its entries are
    nonnegative and its objective is no worse than that of F(F(x_n)),
    otherwise the iteration ends at F(F(x_n)) (so the objective never gets
    worse than the plain MM iterate's), and a singular q x q system falls
    back the same way;
  * "objective" is the model's minimised quantity (the Frobenius objective;
    minus the loglikelihood for the Poisson model).
"""
from __future__ import annotations

import numpy as np

__all__ = ["qn_step_point", "qn_run"]


def qn_step_point(FX, U, Vm, u_new):
    """F(x_n) + V (U^T U - U^T V)^-1 U^T u_n for column memories U, Vm
    (N x m).  Returns None if the m x m system is singular."""
    A = U.T @ U - U.T @ Vm
    rhs = U.T @ u_new
    try:
        c = np.linalg.solve(A, rhs)
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.isfinite(c)):
        return None
    return FX + Vm @ c


def qn_run(F, g, x0, q, iters, tol=0.0):
    """Quasi-Newton acceleration of the map F (x -> F(x), flat float64
    vectors) with memory q, minimising the objective g, for ``iters``
    iterations or until |g_n - g_{n-1}| / (|g_{n-1}| + 1) < tol.

    Returns (x, gs, accepted): the final point, the objective after each
    iteration (gs[0] at x0), and how many quasi-Newton points were taken."""
    x = np.asarray(x0, dtype=np.float64).copy()
    us, vs = [], []
    gs = [g(x)]
    accepted = 0
    for _ in range(iters):
        x1 = F(x)
        x2 = F(x1)
        us.append(x1 - x)
        vs.append(x2 - x1)
        if len(us) > q:
            us.pop(0)
            vs.pop(0)
        U = np.stack(us, axis=1)
        Vm = np.stack(vs, axis=1)
        g2 = g(x2)
        xq = qn_step_point(x1, U, Vm, us[-1])
        if xq is not None and np.all(xq >= 0.0):
            gq = g(xq)
            if gq <= g2:
                x, gnew = xq, gq
                accepted += 1
            else:
                x, gnew = x2, g2
        else:
            x, gnew = x2, g2
        gs.append(gnew)
        if tol > 0 and abs(gnew - gs[-2]) / (abs(gs[-2]) + 1.0) < tol:
            break
    return x, gs, accepted
