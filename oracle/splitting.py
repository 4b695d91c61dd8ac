"""Oracle: operator splitting (Sec. 3) and the 1-D reaction-diffusion step, FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module.

Generic split steps take the sub-flows as callables so that the linear
analysis of Sec. 3.3-3.4 can be checked with exact sub-solutions:

* Strang (Sec. 3.1): T over h/2, R over h, T over h/2.
* Balanced splitting (Eq. balanced): T + c_n over h/2, R - c_n over h,
  T + c_n over h/2, with c_n held constant over the step.
* Simple balanced: c_n = (R(U_n) - T(U_n)) / 2.
* Simpler balanced (Eq. simpler_balanced): c_n = -T(U_n); the first transport
  half step is at equilibrium and omitted, leaving
    R(U) - c_n  over [t_n, t_n + h]        from U_n,
    T(U) + c_n  over [t_n + h/2, t_n + h]  from the result.

The 1-D reaction-diffusion case uses transport T(U) = D d^2U/dx^2 on every
state component (constant diffusivity, unit Lewis number) with a second-order
central difference and zero-gradient ends, the reaction sub-step by ROK4E with
the constant source T(U_n), and one SSP-RK3 step (Shu-Osher form) of size h/2
for the transport correction.

The scalar growth factors R(h) and the source factors Q(h) of the recurrence
u_{n+1} = R u_n - Q (a + b) (Eq. balance_recur) are restated for the scalar
linear problem du/dt = A u + a + B u + b with alpha = e^{Ah/2},
beta = e^{Bh}, A* = (alpha - 1)/A, B* = (beta - 1)/B.
"""

from __future__ import annotations

import numpy as np

from . import rok4e


# ------------------------------------------------------------- generic steps
def strang_step(u, h, flow_T, flow_R):
    u1 = flow_T(u, h / 2, 0.0)
    u2 = flow_R(u1, h, 0.0)
    return flow_T(u2, h / 2, 0.0)


def balanced_step(u, h, c, flow_T, flow_R):
    """Eq. balanced with a given constant c_n; flow_X(u, dt, src)."""
    u1 = flow_T(u, h / 2, c)
    u2 = flow_R(u1, h, -c)
    return flow_T(u2, h / 2, c)


def simple_balanced_step(u, h, T_op, R_op, flow_T, flow_R, reaction_first=True):
    """c_n = (R(U_n) - T(U_n))/2.  The paper computes the reaction part first for
    this method (R - c over h/2, T + c over h, R - c over h/2)."""
    c = 0.5 * (R_op(u) - T_op(u))
    if not reaction_first:
        return balanced_step(u, h, c, flow_T, flow_R)
    u1 = flow_R(u, h / 2, -c)
    u2 = flow_T(u1, h, c)
    return flow_R(u2, h / 2, -c)


def simpler_step(u, h, T_op, flow_T, flow_R):
    """Eq. simpler_balanced: c_n = -T(U_n); R - c_n over h, then T + c_n over h/2."""
    c = -T_op(u)
    u1 = flow_R(u, h, -c)
    return flow_T(u1, h / 2, c)


# ------------------------------------------------------ scalar linear analysis
def _stars(A, B, h):
    alpha = np.exp(A * h / 2)
    beta = np.exp(B * h)
    return alpha, beta, (alpha - 1) / A, (beta - 1) / B


def simple_R_Q(A, B, h):
    """Growth and source factors of simple balanced splitting (scalar case), for
    the transport-first ordering of Eq. balanced.  R is the printed expression;
    Q is the printed bracket with the sign that makes u_{n+1} = R u_n - Q (a + b)
    hold (the printed Q belongs to u_{n+1} = R u_n + Q (a + b)).  The
    reaction-first ordering is the same map with A and B exchanged."""
    alpha, beta, As, Bs = _stars(A, B, h)
    R = alpha * beta * alpha + 0.5 * (alpha * Bs - (alpha * beta + 1) * As) * (A - B)
    Q = -0.5 * (alpha * Bs + (alpha * beta + 1) * As)
    return R, Q


def simpler_R_Q(A, B, h):
    """Growth and source factors of Simpler balanced splitting (scalar case).

    R is the printed expression.  With u_{n+1} = R u_n - Q (a + b) the source
    factor that the two-substep scheme produces is Q = -alpha B*; the printed
    Q = alpha B* belongs to u_{n+1} = R u_n + Q (a + b)."""
    alpha, beta, As, Bs = _stars(A, B, h)
    R = alpha * beta * alpha + (alpha * Bs - (alpha * beta + 1) * As) * A
    Q = -alpha * Bs
    return R, Q


def exact_linear_flow(k, const):
    """Exact flow of du/dt = k u + const + src over dt (scalar, k != 0)."""
    def flow(u, dt, src):
        e = np.exp(k * dt)
        return e * u + (e - 1) / k * (const + src)
    return flow


# --------------------------------------------------------- scalar PSR model
def psr_rhs_parts(T, Da, T_in=0.15, T_ad=1.15, T_a=1.8):
    """Eq. scalar_psr split into reaction and mixing parts."""
    react = (T_ad - T) * np.exp(-T_a / T)
    mix = (T_in - T) / Da
    return react, mix


def psr_steady_Da(T, T_in=0.15, T_ad=1.15, T_a=1.8):
    """Damkohler number at which T is a steady state of Eq. scalar_psr (S-curve)."""
    return (T - T_in) / ((T_ad - T) * np.exp(-T_a / T))


# ------------------------------------------------- 1-D reaction-diffusion case
def laplacian_neumann(U, dx):
    """Second-order central d^2/dx^2 along axis 0 with zero-gradient ends."""
    Up = np.concatenate([U[:1], U, U[-1:]], axis=0)
    return (Up[:-2] - 2.0 * Up[1:-1] + Up[2:]) / dx**2


def diffusion_op(U, D, dx):
    return D * laplacian_neumann(U, dx)


def ssprk3(U, dt, g):
    """One SSP-RK3 (Shu-Osher) step of du/dt = g(u)."""
    u1 = U + dt * g(U)
    u2 = 0.75 * U + 0.25 * (u1 + dt * g(u1))
    return U / 3.0 + 2.0 / 3.0 * (u2 + dt * g(u2))


SCHEMES = ("simpler", "strang", "simple_balanced", "simple_balanced_transport_first")


def split_step_1d(kin, U, p, dt, D, dx, rtol, atol, M, scheme="simpler", *, h_cell=None, jv_mode="analytic",
                  max_attempts=100000):
    """One split step of the 1-D reaction-diffusion system with any of the
    splittings of Sec. 3.  Transport sub-steps are one SSP-RK3 step of their
    length; reaction sub-steps are ROK4E per cell with the step's constant
    source.  ``h_cell`` (per-cell first step, updated in place) carries over
    between reaction sub-steps.  Returns the new field.

    simpler                          Eq. simpler_balanced (c_n = -T(U_n))
    strang                           T over h/2, R over h, T over h/2
    simple_balanced                  c_n = (R - T)/2, reaction first:
                                     R - c over h/2, T + c over h, R - c over h/2
    simple_balanced_transport_first  Eq. balanced with c_n = (R - T)/2
    """
    U = np.asarray(U, dtype=float)
    n = U.shape[0]
    hc = np.zeros(n) if h_cell is None else h_cell

    def flow_T(V, t, c):  # dU/dt = T(U) + c over t
        return ssprk3(V, t, lambda X: diffusion_op(X, D, dx) + c)

    def flow_R(V, t, src):  # dU/dt = R(U) + src over t, cell by cell
        out = V.copy()
        for i in range(n):
            s = None if np.isscalar(src) and src == 0.0 else src[i]
            f, jv_at = rok4e.reactor(kin, p, s, jv_mode)
            out[i], inf = rok4e.integrate(f, jv_at, V[i], t, rtol, atol, M, h0=hc[i], max_attempts=max_attempts)
            hc[i] = inf["h_last"]
        return out

    if scheme == "simpler":
        Tn = diffusion_op(U, D, dx)
        return flow_T(flow_R(U, dt, Tn), dt / 2, -Tn)
    if scheme == "strang":
        return strang_step(U, dt, flow_T, flow_R)
    Rn = np.array([kin.rhs(u, p) for u in U])
    c = 0.5 * (Rn - diffusion_op(U, D, dx))
    if scheme == "simple_balanced":
        u1 = flow_R(U, dt / 2, -c)
        u2 = flow_T(u1, dt, c)
        return flow_R(u2, dt / 2, -c)
    if scheme == "simple_balanced_transport_first":
        return balanced_step(U, dt, c, flow_T, flow_R)
    raise ValueError(scheme)


def simpler_split_step_1d(kin, U, p, dt, D, dx, rtol, atol, M, *, h_cell=None,
                          jv_mode="analytic", max_attempts=100000, replay=None, record=False,
                          cells=None):
    """One Simpler split step of the 1-D reaction-diffusion system.

    Returns (U_next, h_next, infos, U_react) where U_react is the state after
    the reaction sub-step.  ``cells`` restricts the reaction sub-step to a
    subset of rows; the other rows keep U_n through the reaction sub-step, so
    only the reaction results of the listed rows are meaningful."""
    U = np.asarray(U, dtype=float)
    Tn = diffusion_op(U, D, dx)  # T(U_n) = -c_n
    rows = range(U.shape[0]) if cells is None else cells
    U1 = U.copy()
    h_next = np.full(U.shape[0], np.nan) if h_cell is None else np.array(h_cell, dtype=float)
    infos = {}
    for c in rows:
        f, jv_at = rok4e.reactor(kin, p, Tn[c], jv_mode)
        hc = None if h_cell is None else h_cell[c]
        rp = None if replay is None else replay[c]
        U1[c], inf = rok4e.integrate(f, jv_at, U[c], dt, rtol, atol, M, h0=hc,
                                     max_attempts=max_attempts, replay=rp, record=record)
        h_next[c] = inf["h_last"]
        infos[c] = inf
    U2 = ssprk3(U1, dt / 2, lambda V: diffusion_op(V, D, dx) - Tn)
    return U2, h_next, infos, U1
