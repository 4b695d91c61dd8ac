"""Oracle: constant-pressure 0-D reactor right-hand side and its Jacobian (FP64).

TEST INFRASTRUCTURE ONLY.  This is the plain, slow reference the CUDA path is
checked against; nothing in the library imports it.

The paper's 0-D reactor (Eq. cv_reactor, Sec. 4.4) integrates mass fractions
and temperature with the chemical source term; its kinetics are delegated to
Cantera.  The readings used here:

* Constant pressure: dY_k/dt = W_k w_k / rho,
  dT/dt = -(sum_k h_k w_k) / (rho c_p) with molar enthalpies h_k and the
  mass-specific c_p = sum_k Y_k cp_k / W_k.  (The paper's constant-volume
  form pairs h_k with c_v; the workloads here are constant-pressure cells.)
* Textbook gas kinetics: ideal gas rho = p / (R T sum_k Y_k/W_k),
  C_k = rho Y_k / W_k; NASA-7 polynomials selected by T < T_mid;
  kf = A T^b exp(-Ea/(R T)); Kc = exp(-Delta G/(R T)) (p_ref/(R T))^Delta nu
  with p_ref = 101325 Pa; kr = kf / Kc; third-body concentration
  [M] = sum_k eps_k C_k; Troe falloff k = k_inf Pr/(1+Pr) F with
  Pr = k0 [M] / k_inf and the Troe broadening factor F.
* A is given in cm-mol-s units and converted to SI (m^3/mol) here.
* All Ns mass fractions and T are integrated; negative Y are not clipped.

Every function works for real or complex input (complex-step tests rely on it):
branches use the real part of T and nothing else.
"""

from __future__ import annotations

import numpy as np

R_GAS = 8.314462618  # J/(mol K)
P_REF = 101325.0  # Pa, standard-state pressure of the Gibbs functions
PR_FLOOR = 1e-300
LN10 = np.log(10.0)


class Kinetics:
    """Dense-matrix restatement of a synth.Mechanism for the oracle.

    reactor "cp": constant pressure -- the second argument of rhs/jacobian is p.
    reactor "cv": constant volume (Eq. cv_reactor) -- the second argument is the
    cell's density rho, held fixed; the temperature equation uses the species
    internal energies u_k = h_k - R T and c_v = sum_k Y_k (cp_k - R) / W_k (the
    printed equation pairs h_k with c_v; internal energies are what a closed,
    rigid, adiabatic cell conserves)."""

    def __init__(self, mech, reactor="cp"):
        if reactor not in ("cp", "cv"):
            raise ValueError(reactor)
        self.reactor = reactor
        ns, nr = mech.n_species, mech.n_reactions
        self.ns, self.nr = ns, nr
        self.W = np.asarray(mech.W, dtype=float)
        self.nasa = np.asarray(mech.nasa, dtype=float)
        nu_f = np.zeros((nr, ns))
        nu_r = np.zeros((nr, ns))
        for j in range(nr):
            for s, n in zip(mech.rxn_sp[j], mech.rxn_nu[j]):
                if s < 0:
                    continue
                if n < 0:
                    nu_f[j, s] += -n
                else:
                    nu_r[j, s] += n
        self.nu_f = nu_f  # reactant coefficients
        self.nu_r = nu_r  # product coefficients
        self.nu = nu_r - nu_f  # net, products positive
        self.dnu = self.nu.sum(axis=1)
        self.kind = np.asarray(mech.kind)
        self.rev = np.asarray(mech.reversible).astype(bool)
        self.eff = np.asarray(mech.eff, dtype=float)
        A, b, Ea = (np.asarray(mech.arrh, dtype=float)[:, i] for i in range(3))
        order_f = nu_f.sum(axis=1)
        # concentration order of the rate expression: +1 for a (+M) third body
        conc_order = order_f + (self.kind == 1)
        self.lnA_input = np.log(A)  # ln A as given (cm-mol-s)
        self.lnA = np.log(A) + (conc_order - 1) * np.log(1e-6)
        self.b = b
        self.Ea_R = Ea / R_GAS
        fo = np.asarray(mech.falloff, dtype=float)
        self.troe = self.kind == 2
        with np.errstate(divide="ignore"):
            self.lnA0 = np.where(self.troe, np.log(np.where(self.troe, fo[:, 0], 1.0)) + order_f * np.log(1e-6), 0.0)
        self.b0 = fo[:, 1]
        self.Ea0_R = fo[:, 2] / R_GAS
        self.troe_a, self.T3, self.T1, self.T2 = fo[:, 3], fo[:, 4], fo[:, 5], fo[:, 6]

    def with_lnA(self, lnA):
        """A copy whose ln A (SI) is replaced, e.g. by a complex-perturbed one.
        ``lnA`` is in the input reaction order; the SI conversion offset is kept."""
        import copy
        other = copy.copy(self)
        other.lnA = self.lnA + (np.asarray(lnA) - self.lnA_input)
        return other

    # ------------------------------------------------------------------ thermo
    def coeffs(self, T):
        low = self.nasa[:, 3:10]
        high = self.nasa[:, 10:17]
        return np.where((np.real(T) < self.nasa[:, 1])[:, None], low, high)

    def thermo(self, T):
        """cp/R, h/RT, s/R and d(cp/R)/dT per species (NASA-7)."""
        a = self.coeffs(T)
        a1, a2, a3, a4, a5, a6, a7 = (a[:, i] for i in range(7))
        cp_R = a1 + a2 * T + a3 * T**2 + a4 * T**3 + a5 * T**4
        h_RT = a1 + a2 * T / 2 + a3 * T**2 / 3 + a4 * T**3 / 4 + a5 * T**4 / 5 + a6 / T
        s_R = a1 * np.log(T) + a2 * T + a3 * T**2 / 2 + a4 * T**3 / 3 + a5 * T**4 / 4 + a7
        dcp_R = a2 + 2 * a3 * T + 3 * a4 * T**2 + 4 * a5 * T**3
        return cp_R, h_RT, s_R, dcp_R

    # --------------------------------------------------------------- reactions
    def _troe_F(self, T, Pr):
        a, T3, T1, T2 = self.troe_a, self.T3, self.T1, self.T2
        with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
            e3 = np.exp(-T / np.where(self.troe, T3, 1.0))
            e1 = np.exp(-T / np.where(self.troe, T1, 1.0))
            e2 = np.where(T2 > 0, np.exp(-np.where(T2 > 0, T2, 0.0) / T), 0.0)
        Fc = (1 - a) * e3 + a * e1 + e2
        Fc = np.where(self.troe, Fc, 1.0)
        lFc = np.log10(Fc)
        c = -0.4 - 0.67 * lFc
        n = 0.75 - 1.27 * lFc
        L = np.log10(Pr)
        x = L + c
        D = n - 0.14 * x
        f1 = x / D
        lF = lFc / (1 + f1**2)
        F = 10.0**lF
        # partial derivatives used by the Jacobian
        dlF_dL = -lFc * 2 * f1 / (1 + f1**2) ** 2 * n / D**2
        df1_dlFc = (-0.67 * D + 1.1762 * x) / D**2
        dlF_dlFc = 1 / (1 + f1**2) - lFc * 2 * f1 / (1 + f1**2) ** 2 * df1_dlFc
        with np.errstate(divide="ignore", invalid="ignore"):
            dFc_dT = (-(1 - a) / np.where(self.troe, T3, 1.0) * e3 - a / np.where(self.troe, T1, 1.0) * e1
                      + np.where(T2 > 0, T2 / T**2 * e2, 0.0))
        return F, Fc, dlF_dL, dlF_dlFc, dFc_dT

    def state(self, u, p):
        """Everything the RHS and the Jacobian need at state u = (Y, T)."""
        with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
            return self._state(u, p)

    def _state(self, u, p):
        ns = self.ns
        Y, T = u[:ns], u[ns]
        cp_R, h_RT, s_R, dcp_R = self.thermo(T)
        S = np.sum(Y / self.W)
        rho = p / (R_GAS * T * S) if self.reactor == "cp" else p
        C = rho * Y / self.W
        lnT = np.log(T)
        kf = np.exp(self.lnA + self.b * lnT - self.Ea_R / T)
        dlnkf = (self.b + self.Ea_R / T) / T
        g_RT = h_RT - s_R
        dG_RT = self.nu @ g_RT
        Kc = np.exp(-dG_RT) * (P_REF / (R_GAS * T)) ** self.dnu
        dlnKc = (self.nu @ h_RT - self.dnu) / T
        Pf = np.prod(C[None, :] ** self.nu_f, axis=1)
        Pb = np.prod(C[None, :] ** self.nu_r, axis=1)
        M = self.eff @ C
        st = dict(Y=Y, T=T, cp_R=cp_R, h_RT=h_RT, dcp_R=dcp_R, S=S, rho=rho, C=C,
                  kf=kf, dlnkf=dlnkf, Kc=Kc, dlnKc=dlnKc, Pf=Pf, Pb=Pb, M=M)
        # effective forward coefficient k (so that q = m (k Pf - k/Kc Pb))
        k = kf
        m = np.where(self.kind == 1, M, 1.0)
        if np.any(self.troe):
            k0 = np.exp(self.lnA0 + self.b0 * lnT - self.Ea0_R / T)
            dlnk0 = (self.b0 + self.Ea0_R / T) / T
            Pr = k0 * M / kf
            Pr = np.where(np.real(Pr) > PR_FLOOR, Pr, PR_FLOOR)
            F, Fc, dlF_dL, dlF_dlFc, dFc_dT = self._troe_F(T, Pr)
            k_t = kf * Pr / (1 + Pr) * F
            k = np.where(self.troe, k_t, kf)
            g = 1 / (1 + Pr) + dlF_dL
            dlnk_t = dlnkf + g * (dlnk0 - dlnkf) + dlF_dlFc * dFc_dT / Fc
            st.update(dlnk=np.where(self.troe, dlnk_t, dlnkf),
                      dk_dM=np.where(self.troe, k0 * F / (1 + Pr) * g, 0.0))
        else:
            st.update(dlnk=dlnkf, dk_dM=np.zeros(self.nr))
        kr = np.where(self.rev, k / Kc, 0.0)
        q = m * (k * Pf - kr * Pb)
        omega = self.nu.T @ q
        st.update(k=k, kr=kr, m=m, q=q, omega=omega)
        return st

    def rop(self, u, p):
        return self.state(u, p)["q"]

    def rhs(self, u, p, src=None):
        """f(u) = (dY/dt, dT/dt) (+ src, a constant splitting source)."""
        st = self.state(u, p)
        ns = self.ns
        f = np.empty_like(u)
        f[:ns] = self.W * st["omega"] / st["rho"]
        e = 0.0 if self.reactor == "cp" else 1.0  # u/RT = h/RT - 1, cv/R = cp/R - 1
        cbar = np.sum(st["Y"] * (st["cp_R"] - e) / self.W)
        f[ns] = -st["T"] * np.sum((st["h_RT"] - e) * st["omega"]) / (st["rho"] * cbar)
        if src is not None:
            f = f + src
        return f

    def jacobian(self, u, p):
        """Dense analytic Jacobian df/du (the constant source drops out)."""
        st = self.state(u, p)
        ns, N = self.ns, self.ns + 1
        Y, T, C, rho, S = st["Y"], st["T"], st["C"], st["rho"], st["S"]
        W = self.W
        Wbar = 1.0 / S
        # dC/du and drho/du
        dC = np.zeros((ns, N), dtype=u.dtype)
        drho = np.zeros(N, dtype=u.dtype)
        if self.reactor == "cp":
            dC[:, :ns] = np.diag(rho / W) - np.outer(C, Wbar / W)
            dC[:, ns] = -C / T
            drho[:ns] = -rho * Wbar / W
            drho[ns] = -rho / T
        else:  # density fixed
            dC[:, :ns] = np.diag(rho / W)
        # d(prod C^nu)/dC
        def dprod(nu):
            out = np.zeros((self.nr, ns), dtype=u.dtype)
            for kk in range(ns):
                e = nu[:, kk]
                nz = e > 0
                if not np.any(nz):
                    continue
                nu_m = nu.copy()
                nu_m[:, kk] = np.where(nz, e - 1, 0)
                rest = np.prod(C[None, :] ** nu_m, axis=1)
                out[:, kk] = np.where(nz, e * rest, 0.0)
            return out
        dPf = dprod(self.nu_f)
        dPb = dprod(self.nu_r)
        k, kr, m, Kc = st["k"], st["kr"], st["m"], st["Kc"]
        Pf, Pb = st["Pf"], st["Pb"]
        net = k * Pf - kr * Pb  # q / m
        dq_dC = m[:, None] * (k[:, None] * dPf - kr[:, None] * dPb)
        dq_dC += np.where(self.kind == 1, net, 0.0)[:, None] * self.eff
        # Troe: k depends on [M]; kr = k / Kc follows it
        dk_dM = st["dk_dM"]
        revf = np.where(self.rev, 1.0, 0.0)
        dq_dC += (dk_dM * (Pf - revf * Pb / Kc))[:, None] * self.eff
        dlnk = st["dlnk"]
        dq_dT = m * (k * dlnk * Pf - kr * (dlnk - st["dlnKc"]) * Pb)
        dq = dq_dC @ dC
        dq[:, ns] += dq_dT
        domega = self.nu.T @ dq  # [ns, N]
        omega = st["omega"]
        J = np.zeros((N, N), dtype=u.dtype)
        J[:ns] = (W / rho)[:, None] * domega - (W * omega / rho**2)[:, None] * drho[None, :]
        e = 0.0 if self.reactor == "cp" else 1.0
        h_RT, cp_R, dcp_R = st["h_RT"] - e, st["cp_R"] - e, st["dcp_R"]
        cbar = np.sum(Y * cp_R / W)
        Sh = np.sum(h_RT * omega)
        dSh = h_RT @ domega
        dSh[ns] += np.sum((cp_R - h_RT) / T * omega)
        dcbar = np.zeros(N, dtype=u.dtype)
        dcbar[:ns] = cp_R / W
        dcbar[ns] = np.sum(Y * dcp_R / W)
        eT = np.zeros(N, dtype=u.dtype)
        eT[ns] = 1.0
        J[ns] = -(eT * Sh + T * dSh) / (rho * cbar) + T * Sh * (cbar * drho + rho * dcbar) / (rho * cbar) ** 2
        return J

    def jvp(self, u, p, v):
        return self.jacobian(u, p) @ v

    def jvp_fd(self, u, p, v, src=None):
        """Forward-difference J v with delta = sqrt(eps) (1 + ||u||_2) / ||v||_2."""
        nv = np.linalg.norm(v)
        if nv == 0:
            return np.zeros_like(v)
        delta = np.sqrt(np.finfo(float).eps) * (1.0 + np.linalg.norm(u)) / nv
        return (self.rhs(u + delta * v, p, src) - self.rhs(u, p, src)) / delta


def element_totals(mech, Y):
    """Moles of each element per unit mass: sum_k a_ek Y_k / W_k (rows of Y)."""
    return (np.atleast_2d(Y) / mech.W[None, :]) @ mech.elem.astype(float)
