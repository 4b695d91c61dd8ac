"""Oracle: the ROK4E Rosenbrock-Krylov integrator (Sec. 4, Algorithm 1), FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module.

What it computes (Sec. 4.1-4.3):

1. Arnoldi on K_M(J_n, f_n) gives Q_n (N x m) and H_n (m x m), m <= M
   (Sec. 4.1, Eq. jac_proj).  Modified Gram-Schmidt with one full
   reorthogonalisation pass; breakdown when the orthogonalised vector has lost
   all but 1e-12 of the norm of J q_j, which leaves an invariant subspace of
   dimension m.
2. The four stages of the Rosenbrock form (Eq. s_stage_row) with A_n = Q H Q^T,
   solved on the Krylov coordinates and the orthogonal complement separately
   (``attempt``); the same stages as Eq. s_stage_row_transformed with the
   inverse of Eq. solve_kry_jac.  f is evaluated 3 times per attempt.
3. The solution and its embedded order-3 companion (coefficient table of
   Sec. 4.2), the normalised error and the PI controller of Sec. 4.3, and
   accept/reject, repeated until t_end.

Readings of the text (where it is silent or garbled):
* Table coeff_rok4e prints two rows labelled b_2 and bhat_2; the values are
  b = (b1, b2, b3, b4) with b3 = 0 (the text states b3 = 0) and
  bhat = (bhat1, bhat2, bhat3, bhat4) with bhat4 = 0.  Only this reading
  satisfies the order conditions (tests pin it).
* Eq. s_stage_row lacks the factor h in front of A_n sum gamma_ij k_j; the
  transformed form and Algorithm 1 imply it.
* err = sqrt(mean(((u^ - u*) / (atol + rtol |u*|))^2)) (RMS norm).
* PI control h* = h min(5, max(0.2, 0.8 err_n^beta / err*^alpha)),
  alpha = 0.7/4, beta = 0.4/4, err_n = error of the last accepted step
  (1 before the first), both errors floored at 1e-10; a non-finite error
  rejects with factor 0.2.
* h starts at h0 (default t_end), is clipped to t_end - t, and the
  integration ends when t_end - t <= 1e-12 t_end.  A rejected step reuses
  Q_n, H_n and f_n, which depend on u_n only.
"""

from __future__ import annotations

import numpy as np

GAMMA = 0.572816062482135
# gamma_ij (i > j), zero-based stage indices
GAMMA_IJ = np.array([
    [0.0, 0.0, 0.0, 0.0],
    [-0.602765307997356, 0.0, 0.0, 0.0],
    [-1.389195789724843, 1.072950969011413, 0.0, 0.0],
    [0.992356412977094, -1.390032613873701, -0.440875890223325, 0.0],
])
ALPHA_IJ = np.array([
    [0.0, 0.0, 0.0, 0.0],
    [0.432364435748567, 0.0, 0.0, 0.0],
    [-0.514211316876170, 1.382271144617360, 0.0, 0.0],
    [-0.514211316876170, 1.382271144617360, 0.0, 0.0],
])
B = np.array([0.194335256262729, 0.483167813989227, 0.0, 0.322496929748044])
BHAT = np.array([-0.217819895945721, 1.03130847478467, 0.186511421161047, 0.0])
ORDER = 4
PI_ALPHA = 0.7 / ORDER
PI_BETA = 0.4 / ORDER
FAC_MIN, FAC_MAX, SAFETY = 0.2, 5.0, 0.8
ERR_FLOOR = 1e-10
BREAKDOWN_TOL = 1e-12
T_END_TOL = 1e-12

STATUS_OK, STATUS_MAX_ATTEMPTS, STATUS_NONFINITE, STATUS_STEP_UNDERFLOW = 0, 1, 2, 3


def _norm(v):
    """2-norm; for complex input the analytic continuation sqrt(sum v_i^2), so
    that complex-step differentiation passes through the Arnoldi process."""
    if np.iscomplexobj(v):
        return np.sqrt(np.sum(v * v))
    return np.linalg.norm(v)


def arnoldi(jv, f, M):
    """Orthonormal Q (N x m) and Hessenberg H (m x m) with H = Q^T J Q on K_M(J, f)."""
    N = f.shape[0]
    M = min(M, N)
    beta = _norm(f)
    if M == 0 or np.real(beta) == 0.0 or not np.isfinite(beta):
        return np.zeros((N, 0), dtype=f.dtype), np.zeros((0, 0), dtype=f.dtype)
    Q = np.zeros((N, M), dtype=f.dtype)
    H = np.zeros((M, M), dtype=f.dtype)
    Q[:, 0] = f / beta
    m = M
    for j in range(M):
        w = jv(Q[:, j])
        w0 = _norm(w)
        for _pass in range(2):
            for i in range(j + 1):
                hij = Q[:, i] @ w
                H[i, j] += hij
                w = w - hij * Q[:, i]
        hn = _norm(w)
        if j + 1 == M:
            break
        if np.real(hn) <= BREAKDOWN_TOL * np.real(w0) or hn == 0.0:
            m = j + 1
            break
        H[j + 1, j] = hn
        Q[:, j + 1] = w / hn
    return Q[:, :m], H[:m, :m]


def attempt(f, u, fn, Q, H, h):
    """One ROK4E attempt of size h from u with f(u) = fn.  Returns (u*, u^, n_f).

    The stages are those of the Rosenbrock form, Eq. s_stage_row (with the
    factor h on its A_n term), for the projected Jacobian A_n = Q H Q^T of
    Eq. jac_proj.  A_n vanishes on the orthogonal complement of the Krylov
    space and acts as H on the Krylov coordinates, so every stage splits
    exactly into an m x m Rosenbrock stage on the coordinates and an explicit
    part on the complement:

        (I - h gamma H) kappa_i = Q^T f_i + h H sum_{j<i} gamma_ij kappa_j
        k_i = Q kappa_i + (f_i - Q Q^T f_i),   f_i = f(u + h sum_{j<i} alpha_ij k_j).

    This is the stage vector of the transformed form (Eq. s_stage_row_transformed)
    solved with the low-rank inverse of Eq. solve_kry_jac, reached without the
    Woodbury identity.  A stage whose row of alpha_ij equals the previous
    stage's has the same argument (ROK4E: alpha_4j = alpha_3j), so f is
    evaluated at most 3 times per attempt, the first being fn itself.  Then
    u* = u + h sum b_j k_j and u^ = u + h sum bhat_j k_j (Sec. 4.2, embedded
    order-3 formula).
    """
    m = Q.shape[1]
    N = u.shape[0]
    dtype = np.result_type(u, fn, Q, H, float)
    stage_matrix = np.eye(m) - h * GAMMA * H
    K = np.zeros((4, N), dtype=dtype)  # stage vectors k_i
    kappa = np.zeros((4, m), dtype=dtype)  # their Krylov coordinates Q^T k_i
    n_f = 0
    fi = fn
    for i in range(4):
        if i > 0 and not np.array_equal(ALPHA_IJ[i], ALPHA_IJ[i - 1]):
            fi = f(u + h * (ALPHA_IJ[i, :i] @ K[:i]))
            n_f += 1
        if m > 0:
            coupling = h * (H @ (GAMMA_IJ[i, :i] @ kappa[:i]))
            proj = Q.T @ fi
            kappa[i] = np.linalg.solve(stage_matrix, proj + coupling)
            K[i] = Q @ kappa[i] + (fi - Q @ proj)
        else:
            K[i] = fi
    u_star = u + h * (B @ K)
    u_hat = u + h * (BHAT @ K)
    return u_star, u_hat, n_f


def error_norm(u_star, u_hat, rtol, atol):
    sc = atol + rtol * np.abs(u_star)
    return float(np.sqrt(np.mean(((u_hat - u_star) / sc) ** 2)))


def pi_factor(err, err_prev):
    if not np.isfinite(err):
        return FAC_MIN
    e = max(err, ERR_FLOOR)
    return min(FAC_MAX, max(FAC_MIN, SAFETY * err_prev**PI_BETA / e**PI_ALPHA))


def integrate(f, jv_at, u0, t_end, rtol, atol, M, *, h0=None, max_attempts=100000,
              replay=None, fixed_h=None, record=False):
    """Algorithm 1 over [0, t_end] from u0.

    f(u)          right-hand side (constant splitting source already included)
    jv_at(u)      returns a function v -> J(u) v (analytic or finite difference)
    replay        optional sequence of (h, accepted) attempts to follow instead of
                  the controller's own decisions (the error is still computed)
    fixed_h       fixed step size, no error control (all steps accepted)
    Returns (u, info) with info: h_last, n_accept, n_reject, n_f, n_jv, status,
    errs (per attempt) and trace [(h, accepted)] when record or replay.
    """
    u = np.array(u0, dtype=np.result_type(u0, float))
    t = 0.0
    h = t_end if h0 is None or h0 <= 0 else float(h0)
    if fixed_h is not None:
        h = float(fixed_h)
    err_prev = 1.0
    info = dict(n_accept=0, n_reject=0, n_f=0, n_jv=0, status=STATUS_OK, errs=[], trace=[])
    fn = f(u)
    info["n_f"] += 1
    jv = jv_at(u)
    Q, H = arnoldi(jv, fn, M)
    info["n_jv"] += Q.shape[1]
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
        u_star, u_hat, nf = attempt(f, u, fn, Q, H, h)
        info["n_f"] += nf
        n_att += 1
        err = error_norm(u_star, u_hat, rtol, atol) if n_fixed is None else 0.0
        info["errs"].append(err)
        if n_fixed is not None:
            accept = True
            h_new = h
        else:
            h_new = h * pi_factor(err, err_prev)
            accept = bool(np.isfinite(err) and err <= 1.0)
            if replay is not None:
                accept = bool(acc_forced)
        if record or replay is not None:
            info["trace"].append((h, accept))
        if accept:
            if not np.all(np.isfinite(u_star)):  # (complex: both parts)
                info["status"] = STATUS_NONFINITE
                break
            u = u_star
            t += h
            if n_fixed is None:
                err_prev = max(err, ERR_FLOOR)
            info["n_accept"] += 1
            h_last = h_new
            h = h_new
            done = (info["n_accept"] >= n_fixed) if n_fixed is not None else (t_end - t <= T_END_TOL * t_end)
            if not done:
                fn = f(u)
                info["n_f"] += 1
                jv = jv_at(u)
                Q, H = arnoldi(jv, fn, M)
                info["n_jv"] += Q.shape[1]
        else:
            info["n_reject"] += 1
            h = h_new
            if replay is None and h < 1e-12 * t_end:
                info["status"] = STATUS_STEP_UNDERFLOW
                break
    info["h_last"] = h_last
    info["t"] = t
    return u, info


def reactor(kin, p, src=None, jv_mode="analytic"):
    """(f, jv_at) pair for one constant-pressure cell with an optional constant source."""
    def f(u):
        return kin.rhs(u, p, src)

    if jv_mode == "analytic":
        def jv_at(u):
            J = kin.jacobian(u, p)
            return lambda v: J @ v
    elif jv_mode == "fd":
        def jv_at(u):
            f0 = kin.rhs(u, p, src)
            scale = np.sqrt(np.finfo(float).eps) * (1.0 + np.linalg.norm(u))

            def jv(v):
                nv = np.linalg.norm(v)
                if nv == 0.0:
                    return np.zeros_like(v)
                d = scale / nv
                return (kin.rhs(u + d * v, p, src) - f0) / d
            return jv
    else:
        raise ValueError(jv_mode)
    return f, jv_at


def integrate_cells(kin, U, p, dt, rtol, atol, M, *, src=None, h0=None, jv_mode="analytic",
                    max_attempts=100000, replay=None, fixed_h=None, record=False):
    """Integrate each row of U independently (pure-Python loop over cells)."""
    U = np.asarray(U, dtype=float)
    out = np.empty_like(U)
    infos = []
    for c in range(U.shape[0]):
        s = None if src is None else src[c]
        f, jv_at = reactor(kin, p, s, jv_mode)
        hc = None if h0 is None else (h0[c] if np.ndim(h0) else h0)
        rp = None if replay is None else replay[c]
        out[c], inf = integrate(f, jv_at, U[c], dt, rtol, atol, M, h0=hc, max_attempts=max_attempts,
                                replay=rp, fixed_h=fixed_h, record=record)
        infos.append(inf)
    return out, infos
