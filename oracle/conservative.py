"""Oracle: the reaction system with an auxiliary temperature equation, FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module.

For coupling to a compressible solver (Sec. 5, Eq. chemical_source_balanced)
the reaction sub-step integrates the conservative variables together with an
auxiliary temperature that is used only to evaluate thermochemistry:

    d/dt [U; T] = [R(U, T); 0] + [T_n; 0] + [0; w_T]

with U = (rho Y_1 .. rho Y_Ns, rho, rho u, rho E), R the chemical source
(W_k w_k in the species components, zero in mass, momentum and total
energy), T_n the constant balancing term of Simpler splitting and
(Eq. aux_t_equation)

    w_T = ( - sum_k e_k d(rho Y_k)/dt + |u|^2/2 d(rho)/dt
            - u . d(rho u)/dt + d(rho E)/dt ) / (rho c_v).

State layout here (and in the library): [rho Y (Ns), T, rho, rho u_x, rho u_y,
rho u_z, rho E], N = Ns + 6, SI units.

Readings:
* The printed equation weights d(rho Y_k)/dt with h_k; the identity
  rho E = sum_k rho Y_k e_k(T) + rho |u|^2/2, differentiated in time, gives
  the same equation with the specific internal energies e_k = h_k - R T / W_k
  (and c_v = sum_k Y_k c_v,k), which is what makes the auxiliary temperature
  track the one recovered from the conservative variables.  e_k is used.
* Concentrations are C_k = (rho Y_k) / W_k from the species components; the
  mass component rho enters only through u = (rho u) / rho and rho c_v.
* The Jacobian is taken by complex-step differentiation of the right-hand
  side (exact to rounding), not by a hand derivation.
"""

from __future__ import annotations

import numpy as np

from oracle.kinetics import R_GAS, Kinetics

N_EXTRA = 5  # rho, rho u (3), rho E after T


class AuxTReactor:
    def __init__(self, mech):
        self.kin = Kinetics(mech, reactor="cv")
        self.ns = mech.n_species
        self.N = self.ns + 1 + N_EXTRA
        self.W = self.kin.W

    def split(self, u):
        ns = self.ns
        return u[:ns], u[ns], u[ns + 1], u[ns + 2:ns + 5], u[ns + 5]

    def rhs(self, u, src=None):
        ns = self.ns
        rY, T, rho, mom, _ = self.split(u)
        # rates from C_k = rho Y_k / W_k: the constant-volume kinetics with
        # "mass fractions" rho Y_k and unit density
        with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
            st = self.kin._state(np.concatenate([rY, [T]]), 1.0)
        f = np.zeros(self.N, dtype=np.result_type(u, float))
        f[:ns] = self.W * st["omega"]
        if src is not None:
            f = f + src
        # specific internal energies and rho c_v at the auxiliary temperature
        e = (st["h_RT"] - 1.0) * R_GAS * T / self.W
        rho_cv = np.sum(rY * (st["cp_R"] - 1.0) * R_GAS / self.W)
        vel = mom / rho
        num = -np.sum(e * f[:ns]) + 0.5 * np.dot(vel, vel) * f[ns + 1] - np.dot(vel, f[ns + 2:ns + 5]) + f[ns + 5]
        f[ns] = num / rho_cv + (0.0 if src is None else src[ns])
        return f

    def jacobian(self, u, eps=1e-30):
        J = np.empty((self.N, self.N))
        for j in range(self.N):
            du = np.zeros(self.N, dtype=complex)
            du[j] = 1j * eps
            J[:, j] = np.imag(self.rhs(u.astype(complex) + du)) / eps
        return J

    def jacobian_with_src(self, u, src, eps=1e-30):
        """d f / d u with a constant source present (w_T depends on it)."""
        J = np.empty((self.N, self.N))
        for j in range(self.N):
            du = np.zeros(self.N, dtype=complex)
            du[j] = 1j * eps
            J[:, j] = np.imag(self.rhs(u.astype(complex) + du, src)) / eps
        return J

    def internal_energy(self, u, T=None):
        """rho e(T) = sum_k rho Y_k e_k(T), at T (default: the state's own)."""
        ns = self.ns
        rY = u[:ns]
        T = u[ns] if T is None else T
        _, h_RT, _, _ = self.kin.thermo(T)
        return np.sum(rY * (h_RT - 1.0) * R_GAS * T / self.W)

    def T_conservative(self, u, T0=None, iters=50):
        """Temperature recovered from the conservative variables: the root of
        rho e(T) = rho E - |rho u|^2 / (2 rho) (Newton)."""
        ns = self.ns
        rY, T, rho, mom, rE = self.split(u)
        target = rE - 0.5 * np.dot(mom, mom) / rho
        T = float(T if T0 is None else T0)
        for _ in range(iters):
            cp_R, _, _, _ = self.kin.thermo(T)
            g = self.internal_energy(u, T) - target
            dg = np.sum(rY * (cp_R - 1.0) * R_GAS / self.W)
            step = g / dg
            T -= step
            if abs(step) < 1e-13 * T:
                break
        return T

    def state_from(self, Y, T, rho, vel, src_free=True):
        """Conservative state from primitive variables (E from e(T) + |u|^2/2)."""
        ns = self.ns
        u = np.zeros(self.N)
        u[:ns] = rho * np.asarray(Y, dtype=float)
        u[ns] = T
        u[ns + 1] = rho
        u[ns + 2:ns + 5] = rho * np.asarray(vel, dtype=float)
        u[ns + 5] = self.internal_energy(u) + 0.5 * rho * np.dot(vel, vel)
        return u


def reactor(aux, src=None, jv_mode="analytic"):
    """(f, jv_at) pair for the ROK4E oracle (analytic = complex-step Jacobian)."""
    def f(u):
        return aux.rhs(u, src)

    if jv_mode == "analytic":
        def jv_at(u):
            J = aux.jacobian_with_src(u, src) if src is not None else aux.jacobian(u)
            return lambda v: J @ v
    elif jv_mode == "fd":
        def jv_at(u):
            f0 = aux.rhs(u, src)
            nu = np.linalg.norm(u)

            def jv(v):
                nv = np.linalg.norm(v)
                if nv == 0:
                    return np.zeros_like(v)
                d = np.sqrt(np.finfo(float).eps) * (1.0 + nu) / nv
                return (aux.rhs(u + d * v, src) - f0) / d
            return jv
    else:
        raise ValueError(jv_mode)
    return f, jv_at
