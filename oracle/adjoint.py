"""Oracle: gradients of the fixed-step ROK4E integration w.r.t. ln A (FP64).

TEST INFRASTRUCTURE ONLY.

The differentiated quantity is the final state of ``nsteps`` fixed ROK4E steps
of size h (Algorithm 1 with the step size held fixed, no error control) for
one cell, as a function of the log pre-exponential factors ln A_j.  The oracle
gradient is the complex-step derivative of that whole computation:
d u_final / d ln A_j = Im(u_final(ln A + i eps e_j)) / eps, exact to rounding
because every operation on the path (the kinetics, the Arnoldi process with
analytic norms, the small dense solves, the stage combination) is an analytic
function of ln A.  Central finite differences give an independent,
approximate check.
"""

from __future__ import annotations

import numpy as np

from . import rok4e

CS_EPS = 1e-30


def final_state(kin, u0, p, h, nsteps, M, lnA=None):
    k = kin if lnA is None else kin.with_lnA(lnA)
    f, jv_at = rok4e.reactor(k, p)
    u, info = rok4e.integrate(f, jv_at, np.asarray(u0, dtype=np.result_type(u0, lnA if lnA is not None else 0.0,
                                                                            float)),
                              h * nsteps, 1.0, 1.0, M, fixed_h=h)
    return u


def grad_complex_step(kin, u0, p, h, nsteps, M, js, weights=None):
    """d (w . u_final) / d ln A_j for j in js (w defaults to e_T)."""
    N = len(u0)
    w = np.zeros(N)
    w[-1] = 1.0
    if weights is not None:
        w = np.asarray(weights, dtype=float)
    out = []
    for j in js:
        lnA = kin.lnA_input.astype(complex)
        lnA[j] += 1j * CS_EPS
        uf = final_state(kin, np.asarray(u0, dtype=complex), p, h, nsteps, M, lnA)
        out.append(float(np.imag(w @ uf)) / CS_EPS)
    return np.array(out)


def grad_central_fd(kin, u0, p, h, nsteps, M, js, weights=None, d=1e-6):
    N = len(u0)
    w = np.zeros(N)
    w[-1] = 1.0
    if weights is not None:
        w = np.asarray(weights, dtype=float)
    out = []
    for j in js:
        lp = kin.lnA_input.copy()
        lm = kin.lnA_input.copy()
        lp[j] += d
        lm[j] -= d
        out.append((w @ final_state(kin, u0, p, h, nsteps, M, lp) - w @ final_state(kin, u0, p, h, nsteps, M, lm))
                   / (2 * d))
    return np.array(out)
