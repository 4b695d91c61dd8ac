"""Plant plausible mistakes in the oracle, one at a time, and check that the
oracle's pins catch each one (CPU only; about ten minutes in all).

    python -m pytest tests/test_oracle_planted_mistakes.py --runslow -q

Each case copies the oracle, the input generators and the pin files into a
fresh temporary directory, replaces one line of an oracle module there, and
runs the pin files that cover it with pytest in a subprocess; the repository's
own sources are never modified.  A mistake is caught when some pin fails (or a
pin exceeds its 60 s limit).  The entries marked ``equivalent`` change no
result and are expected to survive.  A pattern that no longer matches the
oracle's source exactly once fails its case.

Marked ``slow``: skipped unless pytest runs with --runslow.
"""

import os
import pathlib
import shutil
import subprocess
import sys

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]

KIN = ["tests/test_oracle_kinetics.py", "tests/test_oracle_rok4e.py", "tests/test_oracle_conservative.py",
       "tests/test_oracle_splitting.py"]
ROK = ["tests/test_oracle_rok4e.py", "tests/test_oracle_coefficients.py", "tests/test_oracle_splitting.py"]
SPL = ["tests/test_oracle_splitting.py"]
EXP = ["tests/test_oracle_explicit.py"]
CON = ["tests/test_oracle_conservative.py"]
ADJ = ["tests/test_oracle_adjoint.py"]

# (module, text in the module, replacement, pin files, expected: "caught" or "equivalent")
MISTAKES = [
    # kinetics: equilibrium constant, third body, Arrhenius, density, heat capacity, Troe, rates
    ("oracle/kinetics.py", "Kc = np.exp(-dG_RT) * (P_REF / (R_GAS * T)) ** self.dnu",
     "Kc = np.exp(-dG_RT) * (P_REF / (R_GAS * T)) ** (-self.dnu)", KIN, "caught"),
    ("oracle/kinetics.py", "M = self.eff @ C", "M = np.sum(C) + 0 * (self.eff @ C)", KIN, "caught"),
    ("oracle/kinetics.py", "kf = np.exp(self.lnA + self.b * lnT - self.Ea_R / T)",
     "kf = np.exp(self.lnA + self.b * lnT - self.Ea_R / (2 * T))", KIN, "caught"),
    ("oracle/kinetics.py", 'rho = p / (R_GAS * T * S) if self.reactor == "cp" else p',
     'rho = p / (R_GAS * T) if self.reactor == "cp" else p', KIN, "caught"),
    ("oracle/kinetics.py", 'cbar = np.sum(st["Y"] * (st["cp_R"] - e) / self.W)',
     'cbar = np.sum(st["Y"] * (st["cp_R"]) / self.W)', KIN, "caught"),
    ("oracle/kinetics.py", "        n = 0.75 - 1.27 * lFc", "        n = 0.75 - 1.72 * lFc", KIN, "caught"),
    ("oracle/kinetics.py", "        c = -0.4 - 0.67 * lFc", "        c = -0.4 - 0.76 * lFc", KIN, "caught"),
    ("oracle/kinetics.py", "        D = n - 0.14 * x", "        D = n + 0.14 * x", KIN, "caught"),
    ("oracle/kinetics.py", "            g = 1 / (1 + Pr) + dlF_dL", "            g = 1 / (1 + Pr) - dlF_dL", KIN, "caught"),
    ("oracle/kinetics.py", "        q = m * (k * Pf - kr * Pb)", "        q = m * (k * Pf - kr * Pb * 1.0000001)", KIN, "caught"),
    ("oracle/kinetics.py", "        kr = np.where(self.rev, k / Kc, 0.0)", "        kr = k / Kc", KIN, "caught"),
    ("oracle/kinetics.py", "        m = np.where(self.kind == 1, M, 1.0)", "        m = np.where(self.kind >= 1, M, 1.0)",
     KIN, "caught"),
    ("oracle/kinetics.py", "            Pr = k0 * M / kf", "            Pr = k0 / kf", KIN, "caught"),
    ("oracle/kinetics.py", "            k_t = kf * Pr / (1 + Pr) * F", "            k_t = kf * Pr / (1 + Pr)", KIN, "caught"),
    # thermodynamics and temperature derivatives
    ("oracle/kinetics.py", "        return np.where((np.real(T) < self.nasa[:, 1])[:, None], low, high)",
     "        return np.where((np.real(T) < self.nasa[:, 0])[:, None], low, high)", KIN, "caught"),
    ("oracle/kinetics.py", "        h_RT = a1 + a2 * T / 2 + a3 * T**2 / 3 + a4 * T**3 / 4 + a5 * T**4 / 5 + a6 / T",
     "        h_RT = a1 + a2 * T / 2 + a3 * T**2 / 3 + a4 * T**3 / 4 + a5 * T**4 / 4 + a6 / T", KIN, "caught"),
    ("oracle/kinetics.py", "        s_R = a1 * np.log(T) + a2 * T + a3 * T**2 / 2 + a4 * T**3 / 3 + a5 * T**4 / 4 + a7",
     "        s_R = a1 * np.log(T) + a2 * T + a3 * T**2 / 2 + a4 * T**3 / 3 + a5 * T**4 / 4 - a7", KIN, "caught"),
    ("oracle/kinetics.py", "        dcp_R = a2 + 2 * a3 * T + 3 * a4 * T**2 + 4 * a5 * T**3",
     "        dcp_R = a2 + 2 * a3 * T + 3 * a4 * T**2 + 4 * a5 * T**2", KIN, "caught"),
    ("oracle/kinetics.py", "        dlnKc = (self.nu @ h_RT - self.dnu) / T", "        dlnKc = (self.nu @ h_RT + self.dnu) / T",
     KIN, "caught"),
    ("oracle/kinetics.py", "        dlnkf = (self.b + self.Ea_R / T) / T", "        dlnkf = (self.b - self.Ea_R / T) / T",
     KIN, "caught"),
    # ROK4E: stages (Krylov coordinates and complement), Arnoldi
    ("oracle/rok4e.py", "    stage_matrix = np.eye(m) - h * GAMMA * H", "    stage_matrix = np.eye(m) + h * GAMMA * H",
     ROK, "caught"),
    ("oracle/rok4e.py", "            K[i] = Q @ kappa[i] + (fi - Q @ proj)", "            K[i] = Q @ kappa[i]", ROK,
     "caught"),  # the orthogonal complement dropped
    ("oracle/rok4e.py", "            coupling = h * (H @ (GAMMA_IJ[i, :i] @ kappa[:i]))",
     "            coupling = (H @ (GAMMA_IJ[i, :i] @ kappa[:i]))", ROK, "caught"),  # no h on the A_n term
    ("oracle/rok4e.py", "            coupling = h * (H @ (GAMMA_IJ[i, :i] @ kappa[:i]))",
     "            coupling = h * (H @ (GAMMA_IJ[:i, i] @ kappa[:i]))", ROK, "caught"),  # transposed table
    ("oracle/rok4e.py", "            coupling = h * (H @ (GAMMA_IJ[i, :i] @ kappa[:i]))",
     "            coupling = h * (H.T @ (GAMMA_IJ[i, :i] @ kappa[:i]))", ROK, "caught"),
    ("oracle/rok4e.py", "            kappa[i] = np.linalg.solve(stage_matrix, proj + coupling)",
     "            kappa[i] = np.linalg.solve(stage_matrix.T, proj + coupling)", ROK, "caught"),
    ("oracle/rok4e.py", "            fi = f(u + h * (ALPHA_IJ[i, :i] @ K[:i]))",
     "            fi = f(u + h * (GAMMA_IJ[i, :i] @ K[:i]))", ROK, "caught"),
    ("oracle/rok4e.py", "        if i > 0 and not np.array_equal(ALPHA_IJ[i], ALPHA_IJ[i - 1]):",
     "        if i == 1:", ROK, "caught"),  # stage 3 reuses stage 2's f
    ("oracle/rok4e.py", "        if i > 0 and not np.array_equal(ALPHA_IJ[i], ALPHA_IJ[i - 1]):",
     "        if i > 0:", ROK, "caught"),  # a 4th f per attempt: the count pin (3 per attempt) fails
    ("oracle/rok4e.py", "    u_star = u + h * (B @ K)", "    u_star = u + h * (B[:3] @ K[:3])", ROK, "caught"),
    ("oracle/rok4e.py", "    u_hat = u + h * (BHAT @ K)", "    u_hat = u + h * (BHAT[:3] @ K[:3])", ROK,
     "equivalent"),  # bhat_4 = 0
    ("oracle/rok4e.py", "                H[i, j] += hij", "                H[j, i] += hij", ROK, "caught"),
    ("oracle/rok4e.py", "        for _pass in range(2):", "        for _pass in range(1):", ROK, "caught"),
    ("oracle/rok4e.py", "        Q[:, j + 1] = w / hn", "        Q[:, j + 1] = w / w0", ROK, "caught"),
    ("oracle/rok4e.py", "        H[j + 1, j] = hn", "        H[j + 1, j] = 0.0", ROK, "caught"),
    # ROK4E: error norm, controller, integration loop, finite-difference J v
    ("oracle/rok4e.py", "    return float(np.sqrt(np.mean(((u_hat - u_star) / sc) ** 2)))",
     "    return float(np.max(np.abs((u_hat - u_star) / sc)))", ROK, "caught"),
    ("oracle/rok4e.py", "    sc = atol + rtol * np.abs(u_star)", "    sc = atol + rtol * np.abs(u_hat)", ROK, "caught"),
    ("oracle/rok4e.py", "    return min(FAC_MAX, max(FAC_MIN, SAFETY * err_prev**PI_BETA / e**PI_ALPHA))",
     "    return min(FAC_MAX, max(FAC_MIN, SAFETY * err_prev**PI_ALPHA / e**PI_BETA))", ROK, "caught"),
    ("oracle/rok4e.py", "FAC_MIN, FAC_MAX, SAFETY = 0.2, 5.0, 0.8", "FAC_MIN, FAC_MAX, SAFETY = 0.2, 5.0, 0.9", ROK, "caught"),
    ("oracle/rok4e.py", "            h = min(h, t_end - t)", "            h = h", ROK, "caught"),
    ("oracle/rok4e.py", "                err_prev = max(err, ERR_FLOOR)", "                err_prev = 1.0", ROK, "caught"),
    ("oracle/rok4e.py", "    err_prev = 1.0\n", "    err_prev = 0.5\n", ROK, "caught"),
    ("oracle/rok4e.py", "            h_last = h_new\n            h = h_new", "            h_last = h\n            h = h_new",
     ROK, "caught"),
    ("oracle/rok4e.py", "            u = u_star\n", "            u = u_hat\n", ROK, "caught"),
    ("oracle/rok4e.py", "            scale = np.sqrt(np.finfo(float).eps) * (1.0 + np.linalg.norm(u))",
     "            scale = np.sqrt(np.finfo(float).eps) * (np.linalg.norm(u))", ROK, "caught"),
    # explicit Dormand-Prince
    ("oracle/explicit.py", "    return min(FAC_MAX, max(FAC_MIN, SAFETY * max(err, ERR_FLOOR) ** -0.2))",
     "    return min(FAC_MAX, max(FAC_MIN, SAFETY * max(err, ERR_FLOOR) ** -0.25))", EXP, "caught"),
    ("oracle/explicit.py", "    sc = atol + rtol * np.abs(u5)", "    sc = atol + rtol * np.abs(u4)", EXP, "caught"),
    ("oracle/explicit.py", "    return float(np.sqrt(np.mean(((u4 - u5) / sc) ** 2)))",
     "    return float(np.max(np.abs((u4 - u5) / sc)))", EXP, "caught"),
    ("oracle/explicit.py", "            u = u5\n", "            u = u4\n", EXP, "caught"),
    ("oracle/explicit.py", "            k1 = k7  # first same as last", "            k1 = f(u5)", EXP,
     "equivalent"),  # stage 7 is evaluated at u5
    # splitting and transport
    ("oracle/splitting.py", "    U2 = ssprk3(U1, dt / 2, lambda V: diffusion_op(V, D, dx) - Tn)",
     "    U2 = ssprk3(U1, dt, lambda V: diffusion_op(V, D, dx) - Tn)", SPL, "caught"),
    ("oracle/splitting.py", "    U2 = ssprk3(U1, dt / 2, lambda V: diffusion_op(V, D, dx) - Tn)",
     "    U2 = ssprk3(U1, dt / 2, lambda V: diffusion_op(V, D, dx) + 0 * Tn)", SPL, "caught"),
    ("oracle/splitting.py", "    u2 = 0.75 * U + 0.25 * (u1 + dt * g(u1))", "    u2 = 0.5 * U + 0.5 * (u1 + dt * g(u1))",
     SPL, "caught"),
    ("oracle/splitting.py", "    Up = np.concatenate([U[:1], U, U[-1:]], axis=0)",
     "    Up = np.concatenate([U[-1:], U, U[:1]], axis=0)", SPL, "caught"),
    ("oracle/splitting.py", "    return flow_T(u1, h / 2, c)", "    return flow_T(u1, h, c)", SPL, "caught"),
    ("oracle/splitting.py", "        return flow_T(flow_R(U, dt, Tn), dt / 2, -Tn)",
     "        return flow_T(flow_R(U, dt, Tn), dt, -Tn)", SPL, "caught"),
    ("oracle/splitting.py", "    u2 = flow_R(u1, h, 0.0)", "    u2 = flow_R(u1, h / 2, 0.0)", SPL, "caught"),
    ("oracle/splitting.py", "    c = 0.5 * (R_op(u) - T_op(u))", "    c = 0.5 * (R_op(u) + T_op(u))", SPL, "caught"),
    ("oracle/splitting.py", "    c = 0.5 * (Rn - diffusion_op(U, D, dx))", "    c = 0.5 * (Rn + diffusion_op(U, D, dx))",
     SPL, "caught"),
    ("oracle/splitting.py", "    R = alpha * beta * alpha + (alpha * Bs - (alpha * beta + 1) * As) * A",
     "    R = alpha * beta * alpha + (alpha * Bs - (alpha * beta + 1) * As) * B", SPL, "caught"),
    ("oracle/splitting.py", "    alpha = np.exp(A * h / 2)", "    alpha = np.exp(A * h)", SPL, "caught"),
    ("oracle/splitting.py", "    R = alpha * beta * alpha + 0.5 * (alpha * Bs - (alpha * beta + 1) * As) * (A - B)",
     "    R = alpha * beta * alpha + 0.5 * (alpha * Bs - (alpha * beta + 1) * As) * (A + B)", SPL, "caught"),
    ("oracle/splitting.py", "    Q = -0.5 * (alpha * Bs + (alpha * beta + 1) * As)",
     "    Q = 0.5 * (alpha * Bs + (alpha * beta + 1) * As)", SPL, "caught"),
    ("oracle/splitting.py", "    Q = -alpha * Bs", "    Q = -beta * Bs", SPL, "caught"),
    ("oracle/splitting.py", "        return e * u + (e - 1) / k * (const + src)", "        return e * u + (e - 1) / k * (const - src)",
     SPL, "caught"),
    # scalar PSR model (Eq. scalar_psr)
    ("oracle/splitting.py", "    react = (T_ad - T) * np.exp(-T_a / T)", "    react = (T_ad - T) * np.exp(-T_a * T)", SPL, "caught"),
    ("oracle/splitting.py", "    mix = (T_in - T) / Da", "    mix = (T_in - T) * Da", SPL, "caught"),
    ("oracle/splitting.py", "    return (T - T_in) / ((T_ad - T) * np.exp(-T_a / T))",
     "    return (T - T_in) / ((T_ad - T) * np.exp(-T_a / (2 * T)))", SPL, "caught"),
    # auxiliary-temperature system
    ("oracle/conservative.py", '        e = (st["h_RT"] - 1.0) * R_GAS * T / self.W',
     '        e = (st["h_RT"]) * R_GAS * T / self.W', CON, "caught"),
    ("oracle/conservative.py",
     "        num = -np.sum(e * f[:ns]) + 0.5 * np.dot(vel, vel) * f[ns + 1] - np.dot(vel, f[ns + 2:ns + 5]) + f[ns + 5]",
     "        num = -np.sum(e * f[:ns]) + 0.5 * np.dot(vel, vel) * f[ns + 1] + np.dot(vel, f[ns + 2:ns + 5]) + f[ns + 5]",
     CON, "caught"),
    ("oracle/conservative.py", '        rho_cv = np.sum(rY * (st["cp_R"] - 1.0) * R_GAS / self.W)',
     '        rho_cv = np.sum(rY * (st["cp_R"]) * R_GAS / self.W)', CON, "caught"),
    ("oracle/conservative.py", "        target = rE - 0.5 * np.dot(mom, mom) / rho", "        target = rE - np.dot(mom, mom) / rho",
     CON, "caught"),
    ("oracle/conservative.py", "        u[ns + 5] = self.internal_energy(u) + 0.5 * rho * np.dot(vel, vel)",
     "        u[ns + 5] = self.internal_energy(u) + rho * np.dot(vel, vel)", CON, "caught"),
    ("oracle/conservative.py", "            dg = np.sum(rY * (cp_R - 1.0) * R_GAS / self.W)",
     "            dg = np.sum(rY * (cp_R) * R_GAS / self.W)", CON, "equivalent"),  # same Newton root
    # adjoint's complex-step derivative
    ("oracle/adjoint.py", "        out.append(float(np.imag(w @ uf)) / CS_EPS)",
     "        out.append(float(np.imag(w @ uf)) / CS_EPS * 1.000001)", ADJ, "caught"),
]


COPY = ("oracle", "synth", "tests")


def _run_in_copy(tmp, module, old, new, tests):
    for d in COPY:
        shutil.copytree(ROOT / d, tmp / d, ignore=shutil.ignore_patterns("__pycache__", "*.pyc"))
    path = tmp / module
    src = path.read_text()
    assert src.count(old) == 1, f"pattern not found exactly once in {module}: {old.strip()[:70]}"
    path.write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-B", "-m", "pytest", "-x", "-q", "-m", "not gpu and not slow", "-p", "no:cacheprovider",
           "--timeout=60", *tests]
    try:
        r = subprocess.run(cmd, cwd=tmp, capture_output=True, text=True, timeout=900, env=env)
    except subprocess.TimeoutExpired:
        return "caught", "suite timeout"
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    return ("caught" if r.returncode else "survived"), (lines[-1] if lines else "")


@pytest.mark.slow
@pytest.mark.parametrize("module,old,new,tests,expected", MISTAKES,
                         ids=[f"{i:02d}-{m[0].split('/')[-1][:-3]}" for i, m in enumerate(MISTAKES)])
def test_planted_mistake(tmp_path, module, old, new, tests, expected):
    outcome, last = _run_in_copy(tmp_path, module, old, new, tests)
    assert outcome == ("caught" if expected == "caught" else "survived"), (new.strip(), last)
