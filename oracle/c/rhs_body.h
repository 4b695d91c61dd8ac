/* Body of the constant-pressure reactor right-hand side, included twice by
 * rok4e_oracle.c: once with SCALAR = double (the right-hand side) and once
 * with SCALAR = double complex (complex-step Jacobian-vector products).
 * TEST INFRASTRUCTURE ONLY (part of the C oracle).
 *
 * f(u) for u = (Y_1..Y_Ns, T), Sec. 4.4 / Eq. cv_reactor read for constant
 * pressure: dY_k/dt = W_k w_k / rho, dT/dt = -T sum_k (h_k/RT) w_k / (rho cbar)
 * with cbar = sum_k Y_k (cp_k/R) / W_k, rho = p / (R T sum_k Y_k/W_k),
 * C_k = rho Y_k / W_k; w = nu^T q, q_j = m_j (k_j prod C^nu' - k_j/Kc_j prod C^nu'');
 * textbook kinetics (Arrhenius, Kc from the NASA-7 Gibbs functions at
 * p_ref = 101325 Pa, third body [M] = sum eff C, Troe falloff).  Only the real
 * part of T chooses branches, so the complex instance is analytic in u. */

static void FN(rhs)(const orc_mech* m, const SCALAR* u, const double* src, double p, SCALAR* f) {
  const int ns = m->ns, nr = m->nr;
  SCALAR cpR[ORC_MAX_SP], hRT[ORC_MAX_SP], gRT[ORC_MAX_SP], C[ORC_MAX_SP], om[ORC_MAX_SP];
  SCALAR q[ORC_MAX_RX];
  const SCALAR T = u[ns];
  const SCALAR lnT = log(T);
  SCALAR S = 0.0;
  for (int k = 0; k < ns; ++k) {
    const double* a = m->nasa + 17 * k + (creal(T) < m->nasa[17 * k + 1] ? 3 : 10);
    cpR[k] = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    hRT[k] = a[0] + T * (a[1] / 2 + T * (a[2] / 3 + T * (a[3] / 4 + T * a[4] / 5))) + a[5] / T;
    const SCALAR sR = a[0] * lnT + T * (a[1] + T * (a[2] / 2 + T * (a[3] / 3 + T * a[4] / 4))) + a[6];
    gRT[k] = hRT[k] - sR;
    S += u[k] / m->W[k];
  }
  const SCALAR rho = p / (ORC_R * T * S);
  for (int k = 0; k < ns; ++k) {
    C[k] = rho * u[k] / m->W[k];
    om[k] = 0.0;
  }
  const SCALAR ln_pref_RT = log(ORC_PREF / (ORC_R * T));
  for (int j = 0; j < nr; ++j) {
    const orc_rxn* r = m->rx + j;
    SCALAR kf = exp(r->lnA + r->b * lnT - r->EaR / T);
    SCALAR Pf = 1.0, Pb = 1.0, dG = 0.0;
    for (int e = 0; e < r->n; ++e) {
      const int s = r->sp[e], nu = r->nu[e];
      if (nu < 0)
        for (int t = 0; t < -nu; ++t) Pf *= C[s];
      else
        for (int t = 0; t < nu; ++t) Pb *= C[s];
      dG += nu * gRT[s];
    }
    SCALAR Mc = 0.0;
    if (r->kind != 0)
      for (int k = 0; k < ns; ++k) Mc += m->eff[(size_t)j * ns + k] * C[k];
    SCALAR mult = 1.0;
    if (r->kind == 1) mult = Mc;
    if (r->kind == 2) {
      const SCALAR k0 = exp(r->lnA0 + r->b0 * lnT - r->Ea0R / T);
      SCALAR Pr = k0 * Mc / kf;
      if (!(creal(Pr) > 1e-300)) Pr = 1e-300;
      SCALAR Fc = (1.0 - r->ta) * exp(-T / r->T3) + r->ta * exp(-T / r->T1);
      if (r->T2 > 0.0) Fc += exp(-r->T2 / T);
      const SCALAR lFc = log(Fc) / ORC_LN10;
      const SCALAR c = -0.4 - 0.67 * lFc, nn = 0.75 - 1.27 * lFc;
      const SCALAR x = log(Pr) / ORC_LN10 + c;
      const SCALAR f1 = x / (nn - 0.14 * x);
      const SCALAR F = exp(ORC_LN10 * lFc / (1.0 + f1 * f1));
      kf = kf * Pr / (1.0 + Pr) * F;
    }
    SCALAR rate = kf * Pf;
    if (r->rev) {
      /* k_r = k_f / Kc, Kc = exp(-Delta G/RT) (p_ref/RT)^Delta nu */
      rate -= kf * exp(dG - r->dnu * ln_pref_RT) * Pb;
    }
    q[j] = mult * rate;
  }
  for (int j = 0; j < nr; ++j) {
    const orc_rxn* r = m->rx + j;
    for (int e = 0; e < r->n; ++e) om[r->sp[e]] += r->nu[e] * q[j];
  }
  SCALAR cbar = 0.0, Sh = 0.0;
  for (int k = 0; k < ns; ++k) {
    f[k] = m->W[k] * om[k] / rho;
    cbar += u[k] * cpR[k] / m->W[k];
    Sh += hRT[k] * om[k];
  }
  f[ns] = -T * Sh / (rho * cbar);
  if (src)
    for (int e = 0; e <= ns; ++e) f[e] += src[e];
}
