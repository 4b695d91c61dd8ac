// Discrete adjoint of fixed-step ROK4E (Algorithm 1 with h held fixed) with
// respect to the initial state and the log pre-exponential factors ln A_j.
//
// A group of G lanes of one warp (G = 4, 8, 16 or 32) integrates one cell
// backwards through the recorded steps.  For
// each step n (last first) it reloads u_n from the checkpoints, recomputes the
// step's internals -- f_n, the Arnoldi basis Q and Hessenberg H (CGS2), the
// inverse of L = I - h gamma H, the stage vectors -- and then propagates the
// adjoint u_bar back through, in reverse order:
//   u_{n+1} = u_n + h sum_j b_j k_j
//   k_i = F_i - Q (z_i - y_i) - G_i,  y_i = L^-1 z_i,  z_i = Q^T F_i,
//   F_i = f(u_n + h sum_j alpha_ij k_j) + G_i,  G_i = sum_j (gamma_ij/gamma) k_j,
//   L = I - h gamma H,
//   Arnoldi: w = J q_j, two Gram-Schmidt passes, h_{j+1,j} = |w2|, q_{j+1} = w2 / h_{j+1,j},
//   q_1 = f_n / |f_n|.
// The Jacobian-vector products of the Arnoldi process depend on u_n and on
// ln A through J, so their adjoint needs second derivatives of f: the
// right-hand side is written once for dual numbers (value, tangent), whose
// forward pass with tangent v gives J v and whose reverse pass with cotangent
// w_bar gives J^T w_bar in the values and grad_u (w_bar^T J v) (equal to the
// directional derivative of J^T w_bar along v) in the tangents.
//
// The lanes of a group split every loop over the state, the species and the
// reactions (element e belongs to lane e mod G in every per-element array, so
// those arrays need no synchronisation between loops); sums are butterfly
// reductions, which leave bit-identical values in all lanes, so every lane
// holds the same scalars and small matrices, and lane 0 alone writes the
// small matrices the group keeps in memory.  The reverse pass scatters the
// cotangents of C and g/RT to species through a species-major list of the
// reaction slots each species fills, so every sum has a fixed order and the
// result does not depend on scheduling.
//
// Per-cell arrays live in a workspace record per cell (element e of array a
// at offset a + e of the cell's record), so that a group's lanes access
// consecutive addresses.
#pragma once

namespace rk {

// ------------------------------------------------------------- dual numbers
struct Dual {
  double v, t;
};
__device__ __forceinline__ Dual dd(double v, double t = 0.0) { return Dual{v, t}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.t + b.t}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.t - b.t}; }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual{-a.v, -a.t}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, fma(a.v, b.t, a.t * b.v)}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return Dual{a * b.v, a * b.t}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return Dual{a.v * b, a.t * b}; }
__device__ __forceinline__ Dual operator+(Dual a, double b) { return Dual{a.v + b, a.t}; }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return Dual{a + b.v, b.t}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return Dual{a.v - b, a.t}; }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return Dual{a - b.v, -b.t}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double iv = 1.0 / b.v;
  const double q = a.v * iv;
  return Dual{q, (a.t - q * b.t) * iv};
}
__device__ __forceinline__ Dual operator/(double a, Dual b) { return dd(a) / b; }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return Dual{a.v / b, a.t / b}; }
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) {
  a = a - b;
  return a;
}
__device__ __forceinline__ Dual dexp(Dual a, const double* tab) {
  const double e = exp_fast(a.v, tab);
  return Dual{e, e * a.t};
}
__device__ __forceinline__ Dual dlog(Dual a) { return Dual{log(a.v), a.t / a.v}; }
__device__ __forceinline__ Dual dlog10(Dual a) { return Dual{log10(a.v), a.t / (a.v * 2.302585092994046)}; }

// element e of the current cell in a structure-of-arrays workspace
template <typename T>
struct Col {
  T* p;
  __device__ __forceinline__ T& operator[](int64_t e) const { return p[e]; }
};

// Rows of the adjoint workspace (computed on the host).
struct AdjLayout {
  int N, ns, nr, ntb, M;
  // double rows
  int u, fn, Q, K, F, arg1, arg2, ubar, Kbar, Qbar, fb2, fbn, wbar, w, w1, w2, tmp, H, p1, p2, hn, Linv, zs, ys,
      Lbar, Hbar, scal, theta;
  int rows_d;
  // dual rows: one right-hand-side pass's tape (rows [0, tape_len): ud .. sc,
  // what a forward pass writes and its reverse reads; that of f(u_n)), the
  // arrays a pass uses only within itself (g, q) and the reverse pass's work
  // arrays, then M + 2 more tapes from row tape0: the Arnoldi columns' J q_j
  // passes, f(arg1), f(arg2); all kept for the step's reverse sweep
  int ud, fd, C, cp, h, g, dcp, om, k, rfac, q, Ms, dlnk, dkdM, omg, sc, Cbar, gbar, ombar, Mbar, ubd, fbd, Pbb, drf;
  int tape_len, tape0;
  int rows_D;
};

struct AdjFrame {
  // doubles
  Col<double> u, fn, Q, K, F, arg1, arg2, ubar, Kbar, Qbar, fb2, fbn, wbar, w, w1, w2, tmp, H, p1, p2, hn, Linv,
      zs, ys, Lbar, Hbar, scal, theta;
  // duals
  // (in the reverse pass q holds d/d(prod C^nu') per reaction, Pbb d/d(prod C^nu''), drf the
  // cotangent of ln(k_r/k_f) times k_r/k_f)
  Col<Dual> ud, fd, C, cp, h, g, dcp, om, k, rfac, q, Ms, dlnk, dkdM, omg, sc, Cbar, gbar, ombar, Mbar, ubd, fbd,
      Pbb, drf;
};

__device__ inline AdjFrame adj_frame(double* wsd, Dual* wsD, const AdjLayout& L, int64_t c) {
  AdjFrame f;
  double* bd = wsd + c * L.rows_d;
  Dual* bD = wsD + c * L.rows_D;
  auto D = [&](int row) { return Col<double>{bd + row}; };
  auto X = [&](int row) { return Col<Dual>{bD + row}; };
  f.u = D(L.u); f.fn = D(L.fn); f.Q = D(L.Q); f.K = D(L.K); f.F = D(L.F); f.arg1 = D(L.arg1); f.arg2 = D(L.arg2);
  f.ubar = D(L.ubar); f.Kbar = D(L.Kbar); f.Qbar = D(L.Qbar); f.fb2 = D(L.fb2); f.fbn = D(L.fbn);
  f.wbar = D(L.wbar); f.w = D(L.w); f.w1 = D(L.w1); f.w2 = D(L.w2); f.tmp = D(L.tmp); f.H = D(L.H);
  f.p1 = D(L.p1); f.p2 = D(L.p2); f.hn = D(L.hn); f.Linv = D(L.Linv); f.zs = D(L.zs); f.ys = D(L.ys);
  f.Lbar = D(L.Lbar); f.Hbar = D(L.Hbar); f.scal = D(L.scal); f.theta = D(L.theta);
  f.ud = X(L.ud); f.fd = X(L.fd); f.C = X(L.C); f.cp = X(L.cp); f.h = X(L.h); f.g = X(L.g); f.dcp = X(L.dcp);
  f.om = X(L.om); f.k = X(L.k); f.rfac = X(L.rfac); f.q = X(L.q); f.Ms = X(L.Ms); f.dlnk = X(L.dlnk);
  f.dkdM = X(L.dkdM); f.omg = X(L.omg); f.sc = X(L.sc); f.Cbar = X(L.Cbar); f.gbar = X(L.gbar);
  f.ombar = X(L.ombar); f.Mbar = X(L.Mbar); f.ubd = X(L.ubd); f.fbd = X(L.fbd); f.Pbb = X(L.Pbb); f.drf = X(L.drf);
  return f;
}

// The frame with its tape rows moved by `delta` duals (the stored tape of an
// Arnoldi column); the work arrays stay shared.
__device__ inline AdjFrame adj_tape(const AdjFrame& F, int64_t delta) {
  AdjFrame t = F;
  Col<Dual>* cols[] = {&t.ud, &t.fd, &t.C, &t.cp, &t.h, &t.dcp, &t.om, &t.k, &t.rfac, &t.Ms,
                       &t.dlnk, &t.dkdM, &t.omg, &t.sc};
  for (Col<Dual>* c : cols) c->p += delta;
  return t;
}

// sum over the group (all lanes receive the same bits)
template <int G>
__device__ __forceinline__ Dual gsum(const Grp<G>& g, Dual a) {
  return Dual{g.sum(a.v), g.sum(a.t)};
}
template <int G>
__device__ __forceinline__ double gsum(const Grp<G>& g, double a) {
  return g.sum(a);
}

// The right-hand side passes come in two scalar types: Dual where the
// tangents are needed (the Jacobian-vector products of the Arnoldi process and
// their reverse), double where only values are (f at u_n and at the stage
// arguments, and their reverse), which halves the arithmetic of those passes.
// The tape keeps Duals either way.
template <class Sc>
__device__ __forceinline__ Sc sv(double v);
template <>
__device__ __forceinline__ double sv<double>(double v) {
  return v;
}
template <>
__device__ __forceinline__ Dual sv<Dual>(double v) {
  return Dual{v, 0.0};
}
template <class Sc>
__device__ __forceinline__ Sc rd(const Dual& x);
template <>
__device__ __forceinline__ double rd<double>(const Dual& x) {
  return x.v;
}
template <>
__device__ __forceinline__ Dual rd<Dual>(const Dual& x) {
  return x;
}
// A value pass writes the tape's values only (its reverse reads nothing else,
// and every dual pass writes both parts before it reads them)
__device__ __forceinline__ void put(Dual& d, double a) { d.v = a; }
__device__ __forceinline__ void put(Dual& d, Dual a) { d = a; }
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
__device__ __forceinline__ double dexp(double a, const double* tab) { return exp_fast(a, tab); }
__device__ __forceinline__ double dlog(double a) { return log(a); }
__device__ __forceinline__ double dlog10(double a) { return log10(a); }
// the ln A gradient contribution: the value, or (tangent passes) the tangent
__device__ __forceinline__ double theta_part(double th, bool) { return th; }
__device__ __forceinline__ double theta_part(Dual th, bool tangent) { return tangent ? th.t : th.v; }

enum { SC_T = 0, SC_INVT, SC_S, SC_RHO, SC_CB, SC_SH, SC_LNRTP, SC_N };

// Forward pass of f on the state ud -> fd, keeping the tape.
template <int G, class Sc>
__device__ void adj_rhs_fwd(const MechView& m, const AdjFrame& F, double p) {
  const Grp<G> g;
  const int ns = m.ns, L = g.lane;
  g.sync();  // ud complete
  const Sc T = rd<Sc>(F.ud[ns]);
  const Sc invT = 1.0 / T;
  const Sc lnT = dlog(T);
  Sc S = sv<Sc>(0.0);
  for (int k = L; k < ns; k += G) {
    const double* c = (val(T) < m.Tmid[k]) ? m.lo : m.hi;
    const double a1 = c[k], a2 = c[ns + k], a3 = c[2 * ns + k], a4 = c[3 * ns + k], a5 = c[4 * ns + k];
    const Sc cp = (((a5 * T + a4) * T + a3) * T + a2) * T + a1;
    const Sc hp = ((c[8 * ns + k] * T + c[7 * ns + k]) * T + c[6 * ns + k]) * T + c[5 * ns + k];
    const Sc hrt = hp * T + a1 + c[9 * ns + k] * invT;
    const Sc sp = ((c[12 * ns + k] * T + c[11 * ns + k]) * T + c[10 * ns + k]) * T + a2;
    const Sc sr = a1 * lnT + sp * T + c[13 * ns + k];
    put(F.cp[k], cp);
    put(F.h[k], hrt);
    put(F.g[k], hrt - sr);
    put(F.dcp[k], ((c[16 * ns + k] * T + c[15 * ns + k]) * T + c[14 * ns + k]) * T + a2);
    S += rd<Sc>(F.ud[k]) * m.invW[k];
  }
  S = gsum(g, S);
  const Sc rho = p / (R_GAS * T * S);
  const Sc irho = 1.0 / rho;
  for (int k = L; k < ns; k += G) put(F.C[k], rho * rd<Sc>(F.ud[k]) * m.invW[k]);
  if (L == ns % G) {  // the empty reaction slot: C = 1, h = g = 0
    F.h[ns] = Dual{0.0, 0.0};
    F.g[ns] = Dual{0.0, 0.0};
    F.C[ns] = Dual{1.0, 0.0};
  }
  g.sync();
  for (int t = L; t < m.ntb; t += G) {
    Sc Mc = sv<Sc>(0.0);
    for (int k = 0; k < ns; ++k) Mc += m.eff[(size_t)t * ns + k] * rd<Sc>(F.C[k]);
    put(F.Ms[t], Mc);
  }
  g.sync();
  const Sc lnRTp = dlog(R_GAS * T / P_REF);
  for (int j = L; j < m.nr; j += G) {
    const uint32_t sl = m.slots[j];
    const int ra = sl & 255, rb = (sl >> 8) & 255, pa = (sl >> 16) & 255, pb = sl >> 24;
    const int meta = m.meta[j];
    const int kind = meta & 3;
    const bool rev = (meta >> 2) & 1;
    const int dnu = ((meta >> 4) & 15) - 4;
    const int slot = meta >> 8;
    Sc k = dexp(m.lnA[j] + m.bexp[j] * lnT - m.EaR[j] * invT, m.etab);
    const Sc rfac = rev ? dexp(rd<Sc>(F.g[pa]) + rd<Sc>(F.g[pb]) - rd<Sc>(F.g[ra]) - rd<Sc>(F.g[rb]) +
                                   (double)dnu * lnRTp,
                               m.etab)
                        : sv<Sc>(0.0);
    Sc mfac = sv<Sc>(1.0);
    if (kind == 1) mfac = rd<Sc>(F.Ms[slot]);
    if (kind == 2) {
      const double* fo = m.fo + (size_t)slot * FO_STRIDE;
      const Sc Mc = rd<Sc>(F.Ms[slot]);
      const Sc dlnkinf = (m.bexp[j] + m.EaR[j] * invT) * invT;
      const Sc k0 = dexp(fo[0] + fo[1] * lnT - fo[2] * invT, m.etab);
      const Sc dlnk0 = (fo[1] + fo[2] * invT) * invT;
      Sc Pr = k0 * Mc / k;
      if (!(val(Pr) > 1e-300)) Pr = sv<Sc>(1e-300);
      const double a = fo[3];
      const Sc e3 = dexp(-1.0 * T * fo[4], m.etab), e1 = dexp(-1.0 * T * fo[5], m.etab);
      const Sc e2 = fo[6] > 0.0 ? dexp(-fo[6] * invT, m.etab) : sv<Sc>(0.0);
      const Sc Fc = (1.0 - a) * e3 + a * e1 + e2;
      const Sc lFc = dlog10(Fc);
      const Sc cc = -0.4 - 0.67 * lFc;
      const Sc nn = 0.75 - 1.27 * lFc;
      const Sc x = dlog10(Pr) + cc;
      const Sc D = nn - 0.14 * x;
      const Sc f1 = x / D;
      const Sc den = 1.0 + f1 * f1;
      const Sc lF = lFc / den;
      const Sc Fb = dexp(lF * 2.302585092994046, m.etab);
      const Sc onePr = 1.0 + Pr;
      const Sc dlF_dL = -1.0 * lFc * 2.0 * f1 / (den * den) * nn / (D * D);
      const Sc df1 = (-0.67 * D + 1.1762 * x) / (D * D);
      const Sc dlF_dlFc = 1.0 / den - lFc * 2.0 * f1 / (den * den) * df1;
      const Sc dFc =
          -(1.0 - a) * fo[4] * e3 - a * fo[5] * e1 + (fo[6] > 0.0 ? fo[6] * invT * invT * e2 : sv<Sc>(0.0));
      const Sc gg = 1.0 / onePr + dlF_dL;
      put(F.dlnk[slot], dlnkinf + gg * (dlnk0 - dlnkinf) + dlF_dlFc * dFc / Fc);
      put(F.dkdM[slot], k0 * Fb / onePr * gg);
      put(F.omg[slot], 1.0 - gg);
      k = k * Pr / onePr * Fb;
    }
    const Sc Pf = rd<Sc>(F.C[ra]) * rd<Sc>(F.C[rb]);
    const Sc Pb = rd<Sc>(F.C[pa]) * rd<Sc>(F.C[pb]);
    put(F.k[j], k);
    put(F.rfac[j], rfac);
    put(F.q[j], mfac * (k * Pf - k * rfac * Pb));
  }
  g.sync();
  Sc Sh = sv<Sc>(0.0), cb = sv<Sc>(0.0);
  for (int k = L; k < ns; k += G) {
    Sc om = sv<Sc>(0.0);
    for (int e = m.csr_ptr[k]; e < m.csr_ptr[k + 1]; ++e) om += m.csr_nu[e] * rd<Sc>(F.q[m.csr_j[e]]);
    put(F.om[k], om);
    put(F.fd[k], m.W[k] * om * irho);
    Sh += rd<Sc>(F.h[k]) * om;
    cb += rd<Sc>(F.ud[k]) * rd<Sc>(F.cp[k]) * m.invW[k];
  }
  Sh = gsum(g, Sh);
  cb = gsum(g, cb);
  if (L == ns % G) put(F.fd[ns], -1.0 * T * Sh / (rho * cb));
  if (L == 0) {
    put(F.sc[SC_T], T);
    put(F.sc[SC_INVT], invT);
    put(F.sc[SC_S], S);
    put(F.sc[SC_RHO], rho);
    put(F.sc[SC_CB], cb);
    put(F.sc[SC_SH], Sh);
    put(F.sc[SC_LNRTP], lnRTp);
  }
  g.sync();
}

// Reverse pass: ubd = J^T fbd on the tape of the last adj_rhs_fwd; the ln A
// gradient is added to F.theta from the values (tangent = false) or from the
// tangents (tangent = true, Dual passes only) of the adjoint.  Each lane takes
// its reactions' cotangents (stored per reaction), then its species gather
// them through the species-major slot list.
template <int G, class Sc>
__device__ void adj_rhs_rev(const MechView& m, const AdjFrame& F, bool tangent) {
  const Grp<G> g;
  const int ns = m.ns, L = g.lane;
  g.sync();  // fbd and the tape complete
  const Sc T = rd<Sc>(F.sc[SC_T]), invT = rd<Sc>(F.sc[SC_INVT]), S = rd<Sc>(F.sc[SC_S]);
  const Sc rho = rd<Sc>(F.sc[SC_RHO]), cb = rd<Sc>(F.sc[SC_CB]), Sh = rd<Sc>(F.sc[SC_SH]);
  const Sc irho = 1.0 / rho;
  const Sc fTb = rd<Sc>(F.fbd[ns]);
  const Sc rcb = rho * cb;
  const Sc Tbar0 = -1.0 * Sh / rcb * fTb;
  const Sc Shbar = -1.0 * T / rcb * fTb;
  const Sc rhobar0 = T * Sh / (rho * rcb) * fTb;
  const Sc cbbar = T * Sh / (rcb * cb) * fTb;
  Sc rhobar_l = sv<Sc>(0.0);  // this lane's share of rho_bar
  for (int k = L; k < ns; k += G) {
    const Sc fb = rd<Sc>(F.fbd[k]);
    const Sc wfb = m.W[k] * irho * fb;
    put(F.ombar[k], wfb + rd<Sc>(F.h[k]) * Shbar);
    rhobar_l -= wfb * rd<Sc>(F.om[k]) * irho;
  }
  if (L == ns % G) F.ombar[ns] = Dual{0.0, 0.0};
  for (int t = L; t < m.ntb; t += G) F.Mbar[t] = Dual{0.0, 0.0};
  g.sync();
  Sc Tbar_l = sv<Sc>(0.0);  // this lane's share of T_bar
  for (int j = L; j < m.nr; j += G) {
    const uint32_t sl = m.slots[j];
    const int ra = sl & 255, rb = (sl >> 8) & 255, pa = (sl >> 16) & 255, pb = sl >> 24;
    const int meta = m.meta[j];
    const int kind = meta & 3;
    const bool rev = (meta >> 2) & 1;
    const int dnu = ((meta >> 4) & 15) - 4;
    const int slot = meta >> 8;
    const Sc qbar = rd<Sc>(F.ombar[pa]) + rd<Sc>(F.ombar[pb]) - rd<Sc>(F.ombar[ra]) - rd<Sc>(F.ombar[rb]);
    const Sc k = rd<Sc>(F.k[j]), rfac = rd<Sc>(F.rfac[j]);
    const Sc Pf = rd<Sc>(F.C[ra]) * rd<Sc>(F.C[rb]);
    const Sc Pb = rd<Sc>(F.C[pa]) * rd<Sc>(F.C[pb]);
    const Sc mfac = kind == 1 ? rd<Sc>(F.Ms[slot]) : sv<Sc>(1.0);
    const Sc kr = k * rfac;
    const Sc qm = qbar * mfac;
    const Sc kbar = qm * (Pf - rfac * Pb);
    if (kind == 1) put(F.Mbar[slot], qbar * (k * Pf - kr * Pb));  // slots are one per reaction
    put(F.q[j], qm * k);           // d/d(prod C^nu')
    put(F.Pbb[j], -1.0 * qm * kr);  // d/d(prod C^nu'')
    Sc drf = sv<Sc>(0.0);
    if (rev) {
      drf = rfac * (-1.0 * qm * k * Pb);  // rfac * rfac_bar
      Tbar_l += (double)dnu * drf * invT;
    }
    put(F.drf[j], drf);
    const Sc kk = k * kbar;
    Sc th;
    if (kind == 2) {
      Tbar_l += kk * rd<Sc>(F.dlnk[slot]);
      put(F.Mbar[slot], kbar * rd<Sc>(F.dkdM[slot]));
      th = kk * rd<Sc>(F.omg[slot]);
    } else {
      Tbar_l += kk * ((m.bexp[j] + m.EaR[j] * invT) * invT);
      th = kk;
    }
    F.theta[j] += theta_part(th, tangent);
  }
  g.sync();
  for (int k = L; k < ns; k += G) {
    Sc cbar = sv<Sc>(0.0), gbar = sv<Sc>(0.0);
    for (int i = m.role_ptr[k]; i < m.role_ptr[k + 1]; ++i) {
      const int e = m.role[i], j = e >> 2, role = e & 3;
      // the other factor of the same product: ra <-> rb, pa <-> pb
      const int other = (m.slots[j] >> (8 * (role ^ 1))) & 255;
      cbar += rd<Sc>(role < 2 ? F.q[j] : F.Pbb[j]) * rd<Sc>(F.C[other]);
      gbar = role < 2 ? gbar - rd<Sc>(F.drf[j]) : gbar + rd<Sc>(F.drf[j]);
    }
    for (int t = 0; t < m.ntb; ++t) cbar += m.eff[(size_t)t * ns + k] * rd<Sc>(F.Mbar[t]);
    put(F.Cbar[k], cbar);
    put(F.gbar[k], gbar);
    rhobar_l += rd<Sc>(F.ud[k]) * m.invW[k] * cbar;
  }
  const Sc rhobar = rhobar0 + gsum(g, rhobar_l);
  Sc Tbar = Tbar0 + gsum(g, Tbar_l) - rho * invT * rhobar;
  const Sc Sbar = -1.0 * rho / S * rhobar;
  Sc T2_l = sv<Sc>(0.0);
  for (int k = L; k < ns; k += G) {
    const Sc cpk = rd<Sc>(F.cp[k]), hk = rd<Sc>(F.h[k]);
    const Sc Yb = cpk * m.invW[k] * cbbar + rho * m.invW[k] * rd<Sc>(F.Cbar[k]) + Sbar * m.invW[k];
    put(F.ubd[k], Yb);
    const Sc cpbar = rd<Sc>(F.ud[k]) * m.invW[k] * cbbar;
    const Sc hbar = rd<Sc>(F.om[k]) * Shbar;
    T2_l += cpbar * rd<Sc>(F.dcp[k]) + hbar * (cpk - hk) * invT - rd<Sc>(F.gbar[k]) * hk * invT;
  }
  Tbar += gsum(g, T2_l);
  if (L == ns % G) put(F.ubd[ns], Tbar);
  g.sync();
}

}  // namespace rk

namespace rk {

// Explicit inverse of I - h gamma H (m x m) by Gauss-Jordan with partial
// pivoting; every lane of the group computes it (same bits), lane 0 stores it.
template <int G>
__device__ inline void adj_small_inverse(const AdjFrame& F, int md, double h) {
  const Grp<G> g;
  double A[MAXM][MAXM], B[MAXM][MAXM];
  for (int r = 0; r < md; ++r)
    for (int c = 0; c < md; ++c) {
      A[r][c] = (r == c ? 1.0 : 0.0) - h * GAM * F.H[r * MAXM + c];
      B[r][c] = (r == c ? 1.0 : 0.0);
    }
  for (int c = 0; c < md; ++c) {
    int pr = c;
    for (int r = c + 1; r < md; ++r)
      if (fabs(A[r][c]) > fabs(A[pr][c])) pr = r;
    if (pr != c)
      for (int j = 0; j < md; ++j) {
        double t = A[c][j]; A[c][j] = A[pr][j]; A[pr][j] = t;
        t = B[c][j]; B[c][j] = B[pr][j]; B[pr][j] = t;
      }
    const double inv = 1.0 / A[c][c];
    for (int j = 0; j < md; ++j) {
      A[c][j] *= inv;
      B[c][j] *= inv;
    }
    for (int r = 0; r < md; ++r) {
      if (r == c) continue;
      const double f = A[r][c];
      for (int j = 0; j < md; ++j) {
        A[r][j] = fma(-f, A[c][j], A[r][j]);
        B[r][j] = fma(-f, B[c][j], B[r][j]);
      }
    }
  }
  if (g.lane == 0)
    for (int r = 0; r < md; ++r)
      for (int c = 0; c < md; ++c) F.Linv[r * MAXM + c] = B[r][c];
  g.sync();
}

template <int G>
__device__ inline void adj_load_ud(const AdjFrame& F, int N, const Col<double>& x, const double* tan) {
  const Grp<G> g;
  for (int e = g.lane; e < N; e += G) F.ud[e] = Dual{x[e], tan ? tan[e] : 0.0};
}

// Forward recomputation and reverse sweep of one fixed ROK4E step of size h
// from F.u; on entry F.ubar holds the adjoint of the step's result, on exit
// that of F.u; the ln A gradient accumulates in F.theta.
template <int G>
__device__ void adj_step(const MechView& m, const AdjFrame& F, double p, double h, int M, int64_t tape0,
                         int64_t tape_len) {
  const Grp<G> g;
  const int ns = m.ns, N = ns + 1, L = g.lane;
  constexpr double g21 = G21 / GAM, g31 = G31 / GAM, g32 = G32 / GAM;
  constexpr double g41 = G41 / GAM, g42 = G42 / GAM, g43 = G43 / GAM;
  const double gij[4][3] = {{0, 0, 0}, {g21, 0, 0}, {g31, g32, 0}, {g41, g42, g43}};
  const double bj[4] = {B1, B2, B3, B4};
  if (M > N) M = N;
  double* Q = &F.Q[0];
  // ---------------------------------------------------------------- forward
  // the tapes of f(u_n) (in the frame's own tape rows), f(arg1) and f(arg2)
  // (after the M Arnoldi columns') are kept as well, so the reverse sweep
  // recomputes no forward pass
  const AdjFrame& Fu = F;
  adj_load_ud<G>(Fu, N, F.u, nullptr);
  adj_rhs_fwd<G, double>(m, Fu, p);
  double beta2 = 0.0;
  for (int e = L; e < N; e += G) {
    F.fn[e] = Fu.fd[e].v;
    beta2 = fma(F.fn[e], F.fn[e], beta2);
  }
  const double beta = sqrt(g.sum(beta2));
  if (L == 0)
    for (int i = 0; i < MAXM * MAXM; ++i) F.H[i] = 0.0;
  int md = 0;
  if (M > 0 && beta > 0.0 && isfinite(beta)) {
    md = M;
    for (int e = L; e < N; e += G) Q[e] = F.fn[e] / beta;
    for (int j = 0; j < M; ++j) {
      const AdjFrame Fj = adj_tape(F, tape0 + j * tape_len);  // this column's tape, kept for the reverse sweep
      adj_load_ud<G>(Fj, N, F.u, Q + (int64_t)j * N);
      adj_rhs_fwd<G, Dual>(m, Fj, p);
      double w0 = 0.0;
      for (int e = L; e < N; e += G) {
        F.w[e] = Fj.fd[e].t;
        w0 = fma(F.w[e], F.w[e], w0);
      }
      w0 = sqrt(g.sum(w0));
      for (int pass = 0; pass < 2; ++pass) {
        double pc[MAXM];
        for (int i = 0; i <= j; ++i) {
          double d = 0.0;
          for (int e = L; e < N; e += G) d = fma(Q[(int64_t)i * N + e], F.w[e], d);
          pc[i] = g.sum(d);
        }
        for (int e = L; e < N; e += G) {
          double we = F.w[e];
          for (int i = 0; i <= j; ++i) we = fma(-pc[i], Q[(int64_t)i * N + e], we);
          F.w[e] = we;
        }
        if (L == 0)
          for (int i = 0; i <= j; ++i) {
            F.H[i * MAXM + j] += pc[i];
            (pass == 0 ? F.p1 : F.p2)[j * MAXM + i] = pc[i];
          }
      }
      double hn = 0.0;
      for (int e = L; e < N; e += G) hn = fma(F.w[e], F.w[e], hn);
      hn = sqrt(g.sum(hn));
      if (j + 1 == M) break;
      if (hn <= BREAKDOWN_TOL * w0 || hn == 0.0) {
        md = j + 1;
        break;
      }
      if (L == 0) {
        F.H[(j + 1) * MAXM + j] = hn;
        F.hn[j] = hn;
      }
      for (int e = L; e < N; e += G) Q[(int64_t)(j + 1) * N + e] = F.w[e] / hn;
    }
  }
  g.sync();  // H, p1, p2, hn from lane 0
  if (md > 0) adj_small_inverse<G>(F, md, h);
  // stages
  for (int i = 0; i < 4; ++i) {
    double* Ki = &F.K[(int64_t)i * N];
    double* Fi = &F.F[(int64_t)i * N];
    if (i == 1 || i == 2) {
      const Col<double>& arg = (i == 1) ? F.arg1 : F.arg2;
      for (int e = L; e < N; e += G) {
        const double acc = (i == 1) ? A21 * F.K[e] : fma(A32, F.K[(int64_t)N + e], A31 * F.K[e]);
        arg[e] = F.u[e] + h * acc;
      }
      const AdjFrame Fa = adj_tape(F, tape0 + (int64_t)(M + i - 1) * tape_len);
      adj_load_ud<G>(Fa, N, arg, nullptr);
      adj_rhs_fwd<G, double>(m, Fa, p);
      for (int e = L; e < N; e += G) F.tmp[e] = Fa.fd[e].v;  // f_i (kept for stage 4)
    }
    double z[MAXM];
    for (int l = 0; l < MAXM; ++l) z[l] = 0.0;
    for (int e = L; e < N; e += G) {
      double Ge = 0.0;
      for (int j = 0; j < i; ++j) Ge = fma(gij[i][j], F.K[(int64_t)j * N + e], Ge);
      const double fe = (i == 0) ? F.fn[e] : F.tmp[e];
      Fi[e] = fe + Ge;
      F.w2[e] = Ge;
      for (int l = 0; l < md; ++l) z[l] = fma(Q[(int64_t)l * N + e], Fi[e], z[l]);
    }
    for (int l = 0; l < md; ++l) z[l] = g.sum(z[l]);
    double y[MAXM];
    for (int r = 0; r < md; ++r) {
      double acc = 0.0;
      for (int c = 0; c < md; ++c) acc = fma(F.Linv[r * MAXM + c], z[c], acc);
      y[r] = acc;
    }
    if (L == 0)
      for (int l = 0; l < md; ++l) {
        F.zs[i * MAXM + l] = z[l];
        F.ys[i * MAXM + l] = y[l];
      }
    for (int e = L; e < N; e += G) {
      double acc = 0.0;
      for (int l = 0; l < md; ++l) acc = fma(Q[(int64_t)l * N + e], z[l] - y[l], acc);
      Ki[e] = (Fi[e] - acc) - F.w2[e];
    }
  }
  // ---------------------------------------------------------------- reverse
  g.sync();  // zs, ys from lane 0
  for (int i = 0; i < 4; ++i)
    for (int e = L; e < N; e += G) F.Kbar[(int64_t)i * N + e] = h * bj[i] * F.ubar[e];
  for (int l = 0; l < md; ++l)
    for (int e = L; e < N; e += G) F.Qbar[(int64_t)l * N + e] = 0.0;
  if (L == 0)
    for (int i = 0; i < MAXM * MAXM; ++i) F.Lbar[i] = 0.0;
  for (int e = L; e < N; e += G) {
    F.fb2[e] = 0.0;
    F.fbn[e] = 0.0;
  }
  for (int i = 3; i >= 0; --i) {
    const double* Kb = &F.Kbar[(int64_t)i * N];
    const double* Fi = &F.F[(int64_t)i * N];
    double dbar[MAXM], zbar[MAXM];
    for (int l = 0; l < md; ++l) {
      double d = 0.0;
      for (int e = L; e < N; e += G) d = fma(Q[(int64_t)l * N + e], Kb[e], d);
      dbar[l] = -g.sum(d);
    }
    for (int r = 0; r < md; ++r) {
      double a = 0.0;  // a = L^-T ybar with ybar = -dbar
      for (int c = 0; c < md; ++c) a = fma(F.Linv[c * MAXM + r], -dbar[c], a);
      zbar[r] = dbar[r] + a;
      if (L == 0)
        for (int c = 0; c < md; ++c) F.Lbar[r * MAXM + c] -= a * F.ys[i * MAXM + c];
    }
    for (int l = 0; l < md; ++l) {
      const double dl = F.zs[i * MAXM + l] - F.ys[i * MAXM + l];
      for (int e = L; e < N; e += G) {
        double qb = F.Qbar[(int64_t)l * N + e];
        qb = fma(-dl, Kb[e], qb);
        qb = fma(zbar[l], Fi[e], qb);
        F.Qbar[(int64_t)l * N + e] = qb;
      }
    }
    for (int e = L; e < N; e += G) {
      double Fb = Kb[e];
      for (int l = 0; l < md; ++l) Fb = fma(Q[(int64_t)l * N + e], zbar[l], Fb);
      const double Gb = Fb - Kb[e];
      for (int j = 0; j < i; ++j) F.Kbar[(int64_t)j * N + e] += gij[i][j] * Gb;
      F.w[e] = Fb;  // f_bar of this stage
    }
    if (i == 3) {
      for (int e = L; e < N; e += G) F.fb2[e] += F.w[e];
    } else if (i == 2 || i == 1) {
      const Col<double>& arg = (i == 1) ? F.arg1 : F.arg2;
      if (i == 2)
        for (int e = L; e < N; e += G) F.fb2[e] += F.w[e];
      for (int e = L; e < N; e += G) F.fbd[e] = Dual{i == 2 ? F.fb2[e] : F.w[e], 0.0};
      adj_rhs_rev<G, double>(m, adj_tape(F, tape0 + (int64_t)(M + i - 1) * tape_len), false);
      for (int e = L; e < N; e += G) {
        const double ab = F.ubd[e].v;
        F.ubar[e] += ab;
        if (i == 2) {
          F.Kbar[e] += h * A31 * ab;
          F.Kbar[(int64_t)N + e] += h * A32 * ab;
        } else {
          F.Kbar[e] += h * A21 * ab;
        }
      }
    } else {
      for (int e = L; e < N; e += G) F.fbn[e] += F.w[e];
    }
  }
  if (L == 0)
    for (int i = 0; i < MAXM * MAXM; ++i) F.Hbar[i] = -h * GAM * F.Lbar[i];
  g.sync();  // Hbar from lane 0
  // Arnoldi, last column first
  for (int j = md - 1; j >= 0; --j) {
    const AdjFrame Fj = adj_tape(F, tape0 + j * tape_len);  // the tape of J(u) q_j from the forward sweep
    for (int e = L; e < N; e += G) F.w[e] = Fj.fd[e].t;
    for (int e = L; e < N; e += G) {
      double a = F.w[e];
      for (int i = 0; i <= j; ++i) a = fma(-F.p1[j * MAXM + i], Q[(int64_t)i * N + e], a);
      F.w1[e] = a;
      double b = a;
      for (int i = 0; i <= j; ++i) b = fma(-F.p2[j * MAXM + i], Q[(int64_t)i * N + e], b);
      F.w2[e] = b;
    }
    // w2 -> (h_{j+1,j}, q_{j+1})
    if (j + 1 < md) {
      const double eta = F.hn[j];
      double qw = 0.0;
      for (int e = L; e < N; e += G) qw = fma(F.Qbar[(int64_t)(j + 1) * N + e], F.w2[e], qw);
      qw = g.sum(qw);
      const double c = F.Hbar[(j + 1) * MAXM + j] - qw / (eta * eta);
      for (int e = L; e < N; e += G) F.wbar[e] = (F.Qbar[(int64_t)(j + 1) * N + e] + c * F.w2[e]) / eta;
    } else {
      for (int e = L; e < N; e += G) F.wbar[e] = 0.0;
    }
    double pb2[MAXM], pb1[MAXM];
    for (int i = 0; i <= j; ++i) {  // second pass
      double d = 0.0;
      for (int e = L; e < N; e += G) d = fma(Q[(int64_t)i * N + e], F.wbar[e], d);
      pb2[i] = F.Hbar[i * MAXM + j] - g.sum(d);
    }
    for (int e = L; e < N; e += G) {
      double wb = F.wbar[e];
      for (int i = 0; i <= j; ++i) {
        F.Qbar[(int64_t)i * N + e] += -F.p2[j * MAXM + i] * F.wbar[e] + pb2[i] * F.w1[e];
        wb = fma(pb2[i], Q[(int64_t)i * N + e], wb);
      }
      F.tmp[e] = wb;  // w1_bar
    }
    for (int i = 0; i <= j; ++i) {  // first pass
      double d = 0.0;
      for (int e = L; e < N; e += G) d = fma(Q[(int64_t)i * N + e], F.tmp[e], d);
      pb1[i] = F.Hbar[i * MAXM + j] - g.sum(d);
    }
    for (int e = L; e < N; e += G) {
      double wb = F.tmp[e];
      for (int i = 0; i <= j; ++i) {
        F.Qbar[(int64_t)i * N + e] += -F.p1[j * MAXM + i] * F.tmp[e] + pb1[i] * F.w[e];
        wb = fma(pb1[i], Q[(int64_t)i * N + e], wb);
      }
      F.wbar[e] = wb;
    }
    // w = J(u) q_j: J^T w_bar into q_bar_j, second-order terms into u_bar and theta
    for (int e = L; e < N; e += G) F.fbd[e] = Dual{F.wbar[e], 0.0};
    adj_rhs_rev<G, Dual>(m, Fj, true);
    for (int e = L; e < N; e += G) {
      F.Qbar[(int64_t)j * N + e] += F.ubd[e].v;
      F.ubar[e] += F.ubd[e].t;
    }
  }
  // q_1 = f_n / |f_n|
  if (md > 0) {
    double qf = 0.0;
    for (int e = L; e < N; e += G) qf = fma(F.Qbar[e], F.fn[e], qf);
    qf = g.sum(qf);
    for (int e = L; e < N; e += G) F.fbn[e] += F.Qbar[e] / beta - qf * F.fn[e] / (beta * beta * beta);
  }
  // f_n = f(u)
  for (int e = L; e < N; e += G) F.fbd[e] = Dual{F.fbn[e], 0.0};
  adj_rhs_rev<G, double>(m, Fu, false);
  for (int e = L; e < N; e += G) F.ubar[e] += F.ubd[e].v;
  g.sync();
}

}  // namespace rk
