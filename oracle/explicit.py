"""Oracle: the explicit Dormand-Prince 5(4) integrator, FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module.

Sec. 4.4 measures ROK4E's efficiency against an explicit Runge-Kutta method
of order 5, Dormand-Prince (RKDP), over splitting intervals h_CFL between
1e-9 and 1e-5 s.  This is that reference method, written from its published
definition (J. R. Dormand and P. J. Prince, "A family of embedded
Runge-Kutta formulae", J. Comput. Appl. Math. 6 (1980) 19-26): seven stages,
the 5th-order solution propagated, the embedded 4th-order solution for the
error, first-same-as-last (the seventh stage is evaluated at the new
solution and is the next step's first stage).

Readings (the paper gives no controller for RKDP):
* the error norm is the one ROK4E uses, RMS over all N components of
  (u5 - u4) / (atol + rtol |u5|);
* the step controller is the elementary one for an order-5 pair,
  h* = h min(5, max(0.2, 0.9 err^(-1/5))), err floored at 1e-10, a
  non-finite error rejecting with factor 0.2;
* h starts at h0 (default t_end), is clipped to t_end - t, the integration
  ends when t_end - t <= 1e-12 t_end, as for ROK4E.
"""

from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np

STATUS_OK, STATUS_MAX_ATTEMPTS, STATUS_NONFINITE, STATUS_STEP_UNDERFLOW = 0, 1, 2, 3

# Butcher tableau, exact rationals (Dormand & Prince 1980, Table 2)
C_EXACT = [Fr(0), Fr(1, 5), Fr(3, 10), Fr(4, 5), Fr(8, 9), Fr(1), Fr(1)]
A_EXACT = [
    [],
    [Fr(1, 5)],
    [Fr(3, 40), Fr(9, 40)],
    [Fr(44, 45), Fr(-56, 15), Fr(32, 9)],
    [Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)],
    [Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)],
    [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)],
]
B_EXACT = [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84), Fr(0)]
BHAT_EXACT = [Fr(5179, 57600), Fr(0), Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200), Fr(187, 2100),
              Fr(1, 40)]

C = np.array([float(c) for c in C_EXACT])
A = [np.array([float(a) for a in row]) for row in A_EXACT]
B = np.array([float(b) for b in B_EXACT])
BHAT = np.array([float(b) for b in BHAT_EXACT])

FAC_MIN, FAC_MAX, SAFETY, ERR_FLOOR = 0.2, 5.0, 0.9, 1e-10
T_END_TOL = 1e-12


def error_norm(u5, u4, rtol, atol):
    sc = atol + rtol * np.abs(u5)
    return float(np.sqrt(np.mean(((u4 - u5) / sc) ** 2)))


def step_factor(err):
    if not np.isfinite(err):
        return FAC_MIN
    return min(FAC_MAX, max(FAC_MIN, SAFETY * max(err, ERR_FLOOR) ** -0.2))


def attempt(f, u, k1, h):
    """One RKDP step from u with k1 = f(u): returns (u5, u4, k7, n_f)."""
    k = [k1]
    for i in range(1, 7):
        arg = u + h * sum(A[i][j] * k[j] for j in range(i))
        k.append(f(arg))
    u5 = u + h * sum(B[j] * k[j] for j in range(7))
    u4 = u + h * sum(BHAT[j] * k[j] for j in range(7))
    return u5, u4, k[6], 6


def integrate(f, u0, t_end, rtol, atol, *, h0=None, max_attempts=1000000, replay=None, fixed_h=None,
              record=False):
    """RKDP over [0, t_end] from u0; same conventions and info keys as the ROK4E
    oracle (replay: a sequence of (h, accepted) attempts to follow)."""
    u = np.array(u0, dtype=float)
    t = 0.0
    h = t_end if h0 is None or h0 <= 0 else float(h0)
    if fixed_h is not None:
        h = float(fixed_h)
    info = dict(n_accept=0, n_reject=0, n_f=0, status=STATUS_OK, errs=[], trace=[])
    k1 = f(u)
    info["n_f"] += 1
    n_att = 0
    h_last = h
    n_fixed = None if fixed_h is None else int(round(t_end / fixed_h))
    while True:
        if n_fixed is not None:
            if info["n_accept"] >= n_fixed:
                break
        elif t_end - t <= T_END_TOL * t_end:
            break
        if n_att >= max_attempts:
            info["status"] = STATUS_MAX_ATTEMPTS
            break
        if replay is not None:
            if n_att >= len(replay):
                break
            h, acc_forced = replay[n_att]
        elif n_fixed is None:
            h = min(h, t_end - t)
        u5, u4, k7, nf = attempt(f, u, k1, h)
        info["n_f"] += nf
        n_att += 1
        err = error_norm(u5, u4, rtol, atol) if n_fixed is None else 0.0
        info["errs"].append(err)
        if n_fixed is not None:
            accept, h_new = True, h
        else:
            h_new = h * step_factor(err)
            accept = bool(np.isfinite(err) and err <= 1.0)
            if replay is not None:
                accept = bool(acc_forced)
        if record or replay is not None:
            info["trace"].append((h, accept))
        if accept:
            if not np.all(np.isfinite(u5)):
                info["status"] = STATUS_NONFINITE
                break
            u = u5
            k1 = k7  # first same as last
            t += h
            info["n_accept"] += 1
            h_last = h_new
            h = h_new
        else:
            info["n_reject"] += 1
            h = h_new
            if replay is None and h < 1e-12 * t_end:
                info["status"] = STATUS_STEP_UNDERFLOW
                break
    info["h_last"] = h_last
    info["t"] = t
    return u, info


def integrate_cells(kin, U, p, dt, rtol, atol, *, src=None, h0=None, replay=None, fixed_h=None,
                    record=False, max_attempts=1000000):
    """Integrate each row of U independently with RKDP (constant-pressure cells)."""
    U = np.asarray(U, dtype=float)
    out = np.empty_like(U)
    infos = []
    for c in range(U.shape[0]):
        s = None if src is None else src[c]
        hc = None if h0 is None else (h0[c] if np.ndim(h0) else h0)
        rp = None if replay is None else replay[c]
        out[c], inf = integrate(lambda u, s=s: kin.rhs(u, p, s), U[c], dt, rtol, atol, h0=hc, replay=rp,
                                fixed_h=fixed_h, record=record, max_attempts=max_attempts)
        infos.append(inf)
    return out, infos
