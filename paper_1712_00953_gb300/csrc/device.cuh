// GB300 (sm_103a) device code of the ROK4E reaction step and the Simpler split
// step: the per-cell kernels as templates, their device functions, and the host
// helpers that size and launch them.  Each heavy kernel instantiation is compiled
// in its own translation unit (k_*.cu, through launchers.cuh) so the build runs
// in parallel; rok4e_kernels.cu holds the small kernels and the C ABI.
//
// Mapping.  A "group" of G consecutive lanes of a warp (G = 32 by default:
// one warp per cell) integrates one cell at a time.  Vector loops over the
// N = Ns + 1 state entries, the Ns species and the Nr reactions are strided by
// G; dot products and norms are butterfly (xor) shuffle reductions, which give
// bit-identical results on every lane so that all lanes of a group take the
// same control-flow decisions.  All per-cell vectors (state, f_n, the Krylov
// basis, the four stage vectors, species and reaction work arrays) live in
// shared memory next to a per-block copy of the mechanism.
//
// Batching.  The integration kernel is persistent: one wave of blocks sized
// to the device.  With carried step sizes the cells are sorted by expected
// cost and dealt to static per-block bins (the most expensive alone on an
// SM), each drained from a shared-memory counter; otherwise each group takes
// the next cell index from a global atomic counter (work stealing).  Either
// way cells needing 1 or 200 substeps share one launch without a tail of
// idle blocks.
//
// Arithmetic.  FP64 throughout.  Three restatements differ from a literal
// transcription of the kinetics while computing the same quantities:
//  * 1/Kc_j = exp(Delta G_j/RT) (RT/p_ref)^dnu_j is formed as a product of the
//    per-species factors E_k = exp(g_k/RT) (RT/p_ref) over the products and
//    1/E_k over the reactants (2 exponentials per species instead of one per
//    reaction, the pressure factor folded in), falling back to one
//    exponential per reaction when some |g/RT + ln(RT/p_ref)| > 170 (where a
//    product of four factors could overflow);
//  * q_j = m_j k_j (prod C^nu' - prod C^nu''/Kc_j), the second product formed
//    from the per-species C_k E_k and the reactants' 1/E_k;
//  * w = nu^T q is a gather over a species-major list (deterministic order).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "exp2_table.h"
#include "internal.h"
#include "rok4e.h"

namespace rk {

// ---------------------------------------------------------------- constants
constexpr double R_GAS = 8.314462618;
constexpr double P_REF = 101325.0;
constexpr double PREF_OVER_R = P_REF / R_GAS, INV_R = 1.0 / R_GAS;
constexpr double LN_R_OVER_PREF = -9.408091968961747;  // ln(R / P_ref)
constexpr double GAM = 0.572816062482135;
// Table coeff_rok4e (Sec. 4.2); b3 = 0, bhat4 = 0.
constexpr double G21 = -0.602765307997356;
constexpr double G31 = -1.389195789724843, G32 = 1.072950969011413;
constexpr double G41 = 0.992356412977094, G42 = -1.390032613873701, G43 = -0.440875890223325;
constexpr double A21 = 0.432364435748567;
constexpr double A31 = -0.514211316876170, A32 = 1.382271144617360;
constexpr double B1 = 0.194335256262729, B2 = 0.483167813989227, B3 = 0.0, B4 = 0.322496929748044;
constexpr double BH1 = -0.217819895945721, BH2 = 1.03130847478467, BH3 = 0.186511421161047, BH4 = 0.0;
// PI controller (Sec. 4.3), p = 4
constexpr double PI_ALPHA = 0.7 / 4.0, PI_BETA = 0.4 / 4.0;
constexpr double FAC_MIN = 0.2, FAC_MAX = 5.0, SAFETY = 0.8, ERR_FLOOR = 1e-10;
constexpr double BREAKDOWN_TOL = 1e-12, T_END_TOL = 1e-12, H_MIN_FRAC = 1e-12;
constexpr int G_OVERFLOW_HI = 0x40654000;  // high word of 170.0
constexpr int MAXM = RK_MAX_KRYLOV;
// Threads per block of the per-cell kernels: 8 warps, so each thread may hold
// up to 255 registers (one such block fills an SM's register file, which the
// cells' shared-memory slots limit the SM to anyway).
constexpr int MAX_BLOCK_THREADS = 256;
constexpr int EXP_TAB_BYTES = RK_EXP2_TABLE_N * 8;  // leads the dynamic shared memory

static __constant__ double c_exp2_table[RK_EXP2_TABLE_N] = {RK_EXP2_TABLE_VALUES};
static __constant__ double c_log_inv_c[RK_LOG_TABLE_N] = {RK_LOG_INV_C_VALUES};
static __constant__ double c_log_ln_c[RK_LOG_TABLE_N] = {RK_LOG_LN_C_VALUES};

// ------------------------------------------------- table-driven exponential
// exp(x) by Tang's table-driven method (ACM TOMS 15(2), 1989) with a 256-entry
// table of 2^(j/256): x = (256 m + j) ln2/256 + r with |r| <= ln2/512,
// exp(x) = 2^m 2^(j/256) (1 + p(r)), p the degree-4 Taylor polynomial of
// e^r - 1 (truncation < 4e-17 relative).  k = 256 m + j comes from adding a
// 1.5 2^52 shifter, r from a two-part ln2/256, and the final scaling by 2^m is
// an integer add to the exponent field, so the fast path costs 9 FP64
// operations.  |x| >= 708, infinities and NaN take the library exp().
constexpr double EXP_SHIFTER = 6755399441055744.0;  // 1.5 * 2^52
constexpr int EXP_LOG2N = 8;                        // log2 of the table size

__device__ __forceinline__ double exp_scale(double y, int e) {
  return __hiloint2double(__double2hiint(y) + (e << 20), __double2loint(y));
}

__device__ __forceinline__ double exp_fast(double x, const double* __restrict__ tab) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40862000) return exp(x);
  const double kt = fma(x, RK_N_OVER_LN2, EXP_SHIFTER);
  const int k = __double2loint(kt);
  const double kd = kt - EXP_SHIFTER;
  double r = fma(-kd, RK_LN2_OVER_N_HI, x);
  r = fma(-kd, RK_LN2_OVER_N_LO, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(r * r, q, r);
  const double t = tab[k & (RK_EXP2_TABLE_N - 1)];
  return exp_scale(fma(t, p, t), k >> EXP_LOG2N);
}

// Mixed-precision exp: the same argument reduction and reconstruction in FP64,
// e^r - 1 = r + r^2 q(r) with the small term r^2 q(r) (|r| <= ln2/512, so at
// most 9.2e-7) in FP32.  Relative error ~1e-13 for 6 FP64 operations instead
// of 9.
__device__ __forceinline__ double exp_mixed(double x, const double* __restrict__ tab) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40862000) return exp(x);
  const double kt = fma(x, RK_N_OVER_LN2, EXP_SHIFTER);
  const int k = __double2loint(kt);
  const double kd = kt - EXP_SHIFTER;
  double r = fma(-kd, RK_LN2_OVER_N_HI, x);
  r = fma(-kd, RK_LN2_OVER_N_LO, r);
  const float rf = __double2float_rn(r);
  const float q = fmaf(fmaf(rf, 1.0f / 24.0f, 1.0f / 6.0f), rf, 0.5f);
  const double p = r + (double)(rf * rf * q);
  const double t = tab[k & (RK_EXP2_TABLE_N - 1)];
  return exp_scale(fma(t, p, t), k >> EXP_LOG2N);
}

// (exp(x), exp(-x)) as exp_mixed, sharing the argument reduction.
__device__ __forceinline__ void exp_pm_mixed(double x, const double* __restrict__ tab, double* ep, double* em) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40862000) {
    *ep = exp(x);
    *em = exp(-x);
    return;
  }
  const double kt = fma(x, RK_N_OVER_LN2, EXP_SHIFTER);
  const int k = __double2loint(kt);
  const double kd = kt - EXP_SHIFTER;
  double r = fma(-kd, RK_LN2_OVER_N_HI, x);
  r = fma(-kd, RK_LN2_OVER_N_LO, r);
  const float rf = __double2float_rn(r);
  const float r2 = rf * rf;
  const float qp = fmaf(fmaf(rf, 1.0f / 24.0f, 1.0f / 6.0f), rf, 0.5f);
  const float qm = fmaf(fmaf(-rf, 1.0f / 24.0f, 1.0f / 6.0f), -rf, 0.5f);
  const double pp = r + (double)(r2 * qp);
  const double pm = (double)(r2 * qm) - r;
  const double tp = tab[k & (RK_EXP2_TABLE_N - 1)];
  const int km = -k;
  const double tm = tab[km & (RK_EXP2_TABLE_N - 1)];
  *ep = exp_scale(fma(tp, pp, tp), k >> EXP_LOG2N);
  *em = exp_scale(fma(tm, pm, tm), km >> EXP_LOG2N);
}

// 1/x by Newton's iteration for the reciprocal, r <- r + r (1 - x r), from
// an FP32 estimate: two steps square the estimate's relative error twice
// ((1e-7)^4), leaving the last rounding.  Four FP64 operations instead of a
// full-precision division; for positive normal x inside the FP32 range (the
// temperature and the mixture sums of a cell).
__device__ __forceinline__ double rcp_newton(double x) {
  double r = (double)__frcp_rn(__double2float_rn(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 1/x: rcp_newton where x and its reciprocal are FP32-normal (|x| in
// [2^-125, 2^125)), a full division elsewhere (zero, subnormal, huge,
// infinite, NaN).  Within ~1 ulp of the division.
__device__ __forceinline__ double rcp_any(double x) {
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  return ex - 898u < 250u ? rcp_newton(x) : 1.0 / x;
}

// ------------------------------------------------- table-driven logarithm
// ln x by Tang's table-driven method (ACM TOMS 16(4), 1990): x = 2^e m with
// m in [1, 2); the significand's top 7 bits pick the interval
// [1 + j/128, 1 + (j+1)/128) and its tabulated centre reciprocal inv_c_j
// (rounded) with ln_c_j = -ln(inv_c_j), so ln x = e ln2 + ln_c_j + ln(1 + r),
// r = m inv_c_j - 1 by one fma (|r| <= 2^-8), ln(1 + r) by its Taylor
// polynomial through r^7 (truncation below 1e-20).  11 FP64 operations;
// absolute error ~1.5e-16 max(1, |ln x|) (a few ulp only where ln x is near
// 0, which the intervals below 1 reach through cancellation against e ln2).
// Zero, negative, subnormal, infinite and NaN arguments take the library log().
__device__ __forceinline__ double log_fast(double x) {
  const int hi = __double2hiint(x);
  if ((unsigned)(hi - 0x00100000) >= 0x7fe00000u) return log(x);
  const int j = (hi >> 13) & (RK_LOG_TABLE_N - 1);
  const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(x));
  // e as a double: 2^52 + biased exponent, less 2^52 + 1023 (exact)
  const double e = __hiloint2double(0x43300000, hi >> 20) - 4503599627371519.0;
  const double r = fma(m, c_log_inv_c[j], -1.0);
  double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(q, r, 0.2);
  q = fma(q, r, -0.25);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double p = fma(__dmul_rn(r, r), q, r);
  return fma(e, RK_LN2_HI, c_log_ln_c[j]) + fma(e, RK_LN2_LO, p);
}

// ---- double-float ("df") arithmetic: a value h + l held as two FP32 numbers
// with |l| <= ulp(h)/2, ~44-bit significand, on the FP32 pipe.  Products by
// the error-free FMA split (Dekker's two-product), sums by Knuth's two-sum,
// each renormalised.  FP32 exponent range: callers keep magnitudes inside it.
struct df2 {
  float h, l;
};
__device__ __forceinline__ df2 df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(df2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ df2 df_norm(float s, float e) {
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_norm(p, e);
}
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float e = ((a.h - (s - bb)) + (b.h - bb)) + (a.l + b.l);
  return df_norm(s, e);
}
__device__ __forceinline__ df2 df_neg(df2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df2 df_scale(float c, df2 a) {  // c * a with the exact product of c and a.h
  const float p = c * a.h;
  const float e = fmaf(c, a.h, -p);
  return df_norm(p, fmaf(c, a.l, e));
}

// (exp(x), exp(-x)) sharing one argument reduction.
__device__ __forceinline__ void exp_pm(double x, const double* __restrict__ tab, double* ep, double* em) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40862000) {
    *ep = exp(x);
    *em = exp(-x);
    return;
  }
  const double kt = fma(x, RK_N_OVER_LN2, EXP_SHIFTER);
  const int k = __double2loint(kt);
  const double kd = kt - EXP_SHIFTER;
  double r = fma(-kd, RK_LN2_OVER_N_HI, x);
  r = fma(-kd, RK_LN2_OVER_N_LO, r);
  const double r2 = r * r;
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double pp = fma(r2, q, r);
  double qm = fma(-r, 1.0 / 24.0, 1.0 / 6.0);
  qm = fma(qm, -r, 0.5);
  const double pm = fma(r2, qm, -r);
  const double tp = tab[k & (RK_EXP2_TABLE_N - 1)];
  const int km = -k;
  const double tm = tab[km & (RK_EXP2_TABLE_N - 1)];
  *ep = exp_scale(fma(tp, pp, tp), k >> EXP_LOG2N);
  *em = exp_scale(fma(tm, pm, tm), km >> EXP_LOG2N);
}

__device__ inline void load_exp_table(double* dst) {
  for (int i = threadIdx.x; i < RK_EXP2_TABLE_N; i += blockDim.x) dst[i] = c_exp2_table[i];
}

// --------------------------------------------------------------- error state
// The library's last error (thread-local; defined in rok4e_kernels.cu).
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* where);

// ------------------------------------------------------------------- views
struct MechView {
  int ns, nr, ntb, ntroe;
  int nx;  // state components after T: 0, or 5 (rho, rho u, rho E) for the auxiliary-temperature system
  const double* etab;  // 2^(j/256) table in shared memory
  const double *W, *invW, *Tmid, *lo, *hi, *lnA, *bexp, *EaR, *eff, *fo, *csr_nu;
  const uint32_t* slots;
  const int32_t *meta, *csr_ptr, *csr_j;
  const int32_t *piece_ptr, *spec_piece;  // gather pieces of the species-major list
  int npiece;
  const float *Wf, *invWf, *bf, *EaRf, *efff, *csr_nuf;  // FP32 copies
  const int32_t* perm;  // input index of each packed reaction
  int nst, nrt;         // nu^T tiles (species, reactions) of the tensor-core gather
  const uint4* nuT;     // their A operands, per tile and lane
  const int32_t *role_ptr, *role;  // species-major reaction slots (r << 2 | role)
};

__host__ __device__ inline MechView make_view(const unsigned char* base, const MechLayout& L) {
  MechView m;
  m.ns = L.ns;
  m.nr = L.nr;
  m.ntb = L.ntb;
  m.ntroe = L.ntroe;
  m.nx = 0;
  m.etab = nullptr;
  m.W = reinterpret_cast<const double*>(base + L.off_W);
  m.invW = reinterpret_cast<const double*>(base + L.off_invW);
  m.Tmid = reinterpret_cast<const double*>(base + L.off_Tmid);
  m.lo = reinterpret_cast<const double*>(base + L.off_lo);
  m.hi = reinterpret_cast<const double*>(base + L.off_hi);
  m.lnA = reinterpret_cast<const double*>(base + L.off_lnA);
  m.bexp = reinterpret_cast<const double*>(base + L.off_b);
  m.EaR = reinterpret_cast<const double*>(base + L.off_EaR);
  m.eff = reinterpret_cast<const double*>(base + L.off_eff);
  m.fo = reinterpret_cast<const double*>(base + L.off_fo);
  m.csr_nu = reinterpret_cast<const double*>(base + L.off_csr_nu);
  m.slots = reinterpret_cast<const uint32_t*>(base + L.off_slots);
  m.meta = reinterpret_cast<const int32_t*>(base + L.off_meta);
  m.csr_ptr = reinterpret_cast<const int32_t*>(base + L.off_csr_ptr);
  m.csr_j = reinterpret_cast<const int32_t*>(base + L.off_csr_j);
  m.piece_ptr = reinterpret_cast<const int32_t*>(base + L.off_piece_ptr);
  m.spec_piece = reinterpret_cast<const int32_t*>(base + L.off_spec_piece);
  m.npiece = L.npiece;
  m.Wf = reinterpret_cast<const float*>(base + L.off_Wf);
  m.invWf = reinterpret_cast<const float*>(base + L.off_invWf);
  m.bf = reinterpret_cast<const float*>(base + L.off_bf);
  m.EaRf = reinterpret_cast<const float*>(base + L.off_EaRf);
  m.efff = reinterpret_cast<const float*>(base + L.off_efff);
  m.csr_nuf = reinterpret_cast<const float*>(base + L.off_csr_nuf);
  m.perm = reinterpret_cast<const int32_t*>(base + L.off_perm);
  m.nst = L.nst;
  m.nrt = L.nrt;
  m.nuT = reinterpret_cast<const uint4*>(base + L.off_nuT);
  m.role_ptr = reinterpret_cast<const int32_t*>(base + L.off_role_ptr);
  m.role = reinterpret_cast<const int32_t*>(base + L.off_role);
  return m;
}

// Per-cell shared-memory slot (offsets in doubles from the slot base).
struct SlotLayout {
  int N, ns, nr, ntb, M;
  int u, src, fn, arg, fr, F, w, Q, K;        // N-vectors (Q: M of them, K: 4)
  int C, dC, cp, hRT, dcp, gRT, E, Einv, CE, om;  // species (+1 sentinel entry)
  int q, kc, krc, qT;                         // reactions (qT: d q_j / dT at u_n, for J v)
  int tb;                                     // [ntb][4]: [M], dk/d[M], dlnk/dT, 1/Kc
  int tro;                                    // [11][ntroe]: Troe falloff scratch
  int part;                                   // [npiece]: gather partial sums
  int C2, dC2;                                // species: double-float C and dC (precision 3, else -1)
  int dig;                                    // BF16 digits of q, [8][16 nrt] (precision 4, else -1)
  int fj;   // precision 6: FP32 species factors of the J v, when they do not fit beside the
            // FP32 reaction caches in the kc/krc/qT storage (else -1)
  int H, LU, piv, red, Bm;                    // small (Bm: I - (I - h gamma H)^-1)
  int fbase;  // FP32 region (mixed precision only), offset in doubles
  int fC, fdC, fh, fcp, fdcp, fom, fq, fkc, fkr, ftb, fQ, fw, fpart;  // offsets in floats from fbase
  int stride;
};

// mixed: the FP32 arrays of precision levels 1 and 2; df: the double-float
// species arrays of precision level 3 (left out otherwise, which lets a 53-species
// mechanism keep 7 cells per block instead of 6).
inline SlotLayout make_slot(const MechLayout& L, int M, bool mixed = false, int nx = 0, bool df = false,
                            bool tc = false, bool f32jv = false) {
  SlotLayout s;
  s.N = L.ns + 1 + nx;
  s.ns = L.ns;
  s.nr = L.nr;
  s.ntb = L.ntb;
  s.M = M;
  int o = 0;
  auto take = [&](int n) {
    const int r = o;
    o += (n + 1) & ~1;  // keep 16-byte alignment
    return r;
  };
  const int N = s.N, ns1 = L.ns + 1;
  s.u = take(N);
  s.src = take(N);
  s.fn = take(N);
  s.arg = take(N);
  s.fr = take(N);
  s.F = take(N);
  s.w = take(N);
  const int Nq = (N + 1) & ~1;  // stride between Krylov / stage vectors
  s.Q = take(Nq * M);
  s.C = take(ns1);
  s.dC = take(ns1);
  s.cp = take(ns1);
  s.hRT = take(ns1);
  s.dcp = take(ns1);
  s.gRT = take(ns1);
  s.E = take(ns1);
  s.Einv = take(ns1);
  s.CE = take(ns1);
  s.om = take(ns1);
  s.q = take(L.nr > 0 ? L.nr : 1);
  s.kc = take(L.nr > 0 ? L.nr : 1);
  s.krc = take(L.nr > 0 ? L.nr : 1);
  s.qT = take(L.nr > 0 ? L.nr : 1);
  // The stage vectors K live only inside an attempt; the J v caches kc, krc,
  // qT (contiguous) only from the caching right-hand side to the end of the
  // Arnoldi process that precedes the attempts.  K shares their storage when
  // it fits there.
  const int nr_even = ((L.nr > 0 ? L.nr : 1) + 1) & ~1;
  s.K = (4 * Nq <= 3 * nr_even) ? s.kc : take(4 * Nq);
  s.tb = take(4 * (L.ntb > 0 ? L.ntb : 1));
  s.tro = take(11 * (L.ntroe > 0 ? L.ntroe : 1));
  s.part = take(L.npiece > 0 ? L.npiece : 1);
  s.C2 = df ? take(ns1) : -1;
  s.dC2 = df ? take(ns1) : -1;
  s.dig = tc ? take(2 * 16 * L.nrt) : -1;  // 8 x 16 nrt BF16 = 2 x 16 nrt doubles
  // precision 6 keeps its FP32 reaction caches in the first half of the kc/krc/qT
  // storage and its 8 FP32 species arrays in the second half when they fit there
  s.fj = (f32jv && 8 * ns1 > 3 * nr_even) ? take((8 * ns1 + 1) / 2) : -1;
  // M x M matrices stored with row stride MAXM: M rows
  s.H = take(M * MAXM);
  s.LU = take(M * MAXM);
  s.piv = take(MAXM);
  s.red = take(4);
  s.Bm = take(M * MAXM);
  s.fbase = o;
  int fo = 0;
  auto ftake = [&](int n) {
    const int r = fo;
    fo += (n + 3) & ~3;  // 16-byte alignment
    return r;
  };
  if (mixed) {
    s.fC = ftake(ns1);
    s.fdC = ftake(ns1);
    s.fh = ftake(ns1);
    s.fcp = ftake(ns1);
    s.fdcp = ftake(ns1);
    s.fom = ftake(ns1);
    s.fq = ftake(L.nr > 0 ? L.nr : 1);
    s.fkc = ftake(L.nr > 0 ? L.nr : 1);
    s.fkr = ftake(L.nr > 0 ? L.nr : 1);
    s.ftb = ftake(4 * (L.ntb > 0 ? L.ntb : 1));
    s.fQ = ftake(Nq * M);
    s.fw = ftake(Nq);
    s.fpart = ftake(L.npiece > 0 ? L.npiece : 1);
  } else {
    s.fC = s.fdC = s.fh = s.fcp = s.fdcp = s.fom = s.fq = s.fkc = s.fkr = s.ftb = s.fQ = s.fw = s.fpart = 0;
  }
  o += (fo + 1) / 2;
  s.stride = (o + 3) & ~3;
  return s;
}

// A group of G lanes inside one warp.
template <int G>
struct Grp {
  unsigned mask;
  int lane;
  __device__ Grp() {
    const int l = threadIdx.x & 31;
    lane = l % G;
    mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (l - lane));
  }
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
  template <typename T>
  __device__ __forceinline__ T sum(T v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
  }
  __device__ __forceinline__ double max(double v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o, G));
    return v;
  }
  __device__ __forceinline__ int imax(int v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = ::max(v, __shfl_xor_sync(mask, v, o, G));
    return v;
  }
  __device__ __forceinline__ int any(int v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(mask, v, o, G);
    return v;
  }
};

// Sum K values (K a power of two, K <= G) across the G lanes of a group; on
// return every lane holds all K sums.  Reduce-scatter: at each of the first
// log2 K butterfly levels a lane keeps half of its values and adds its
// partner's copy of that half, so the adds per lane are K - 1 + log2(G/K)
// instead of K log2 G; the sums are then broadcast from the lanes that hold
// them.  All lanes end with bit-identical values.
template <int G, int K, typename T>
__device__ __forceinline__ void sum_many(const Grp<G>& g, T (&v)[K]) {
  static_assert((K & (K - 1)) == 0 && K <= G, "K must be a power of two <= G");
  constexpr int LG = (G == 32 ? 5 : G == 16 ? 4 : G == 8 ? 3 : G == 4 ? 2 : G == 2 ? 1 : 0);
  constexpr int LK = (K == 8 ? 3 : K == 4 ? 2 : K == 2 ? 1 : 0);
#pragma unroll
  for (int l = 0; l < LK; ++l) {
    const int o = G >> (l + 1);
    const int half = K >> (l + 1);
    const bool hi = (g.lane & o) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const T send = hi ? v[j] : v[j + half];
      const T keep = hi ? v[j + half] : v[j];
      v[j] = keep + __shfl_xor_sync(g.mask, send, o, G);
    }
  }
#pragma unroll
  for (int o = G >> (LK + 1); o > 0; o >>= 1) v[0] += __shfl_xor_sync(g.mask, v[0], o, G);
  const T mine = v[0];
#pragma unroll
  for (int t = 0; t < K; ++t) v[t] = __shfl_sync(g.mask, mine, t << (LG - LK), G);
}

// Sum the first n (<= MAXM) entries of v across the group (entries past n
// must be zero); dispatches on n to the smallest power-of-two reduction.
template <int G, typename T>
__device__ __forceinline__ void sum_first(const Grp<G>& g, T (&v)[MAXM], int n) {
  static_assert(G >= MAXM, "a group needs at least MAXM lanes");
  if (n <= 1) {
    v[0] = g.sum(v[0]);
  } else if (n <= 2) {
    T t[2] = {v[0], v[1]};
    sum_many<G, 2>(g, t);
    v[0] = t[0];
    v[1] = t[1];
  } else if (n <= 4) {
    T t[4] = {v[0], v[1], v[2], v[3]};
    sum_many<G, 4>(g, t);
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = t[i];
  } else {
    sum_many<G, MAXM>(g, v);
  }
}

// Scalars of the last right-hand-side evaluation that the analytic
// Jacobian-vector product needs (uniform across the group).
struct CellScalars {
  double T, invT, lnT, S, invS, rho, invrho, cb, invcb, Sh;
  double pinv;  // 1 / p (constant pressure) or 1 / rho (constant volume): set by the caller
  int prec;     // precision level (3: mixed exp in the RHS, double-float J v core): set by the caller
  // auxiliary-temperature system: sum_k (cp_k/R - 1) F_k / W_k, the T row
  // without its own source, 1 / rho and the velocity
  double B, fT, irho_c, vel[3];
  bool cv;
};

struct SlotPtrs {
  double *u, *src, *fn, *arg, *fr, *F, *w, *Q, *K;
  double *C, *dC, *cp, *hRT, *dcp, *gRT, *E, *Einv, *CE, *om, *q, *kc, *krc, *qT, *tb, *tro, *part;
  df2 *C2, *dC2;
  uint16_t* dig;
  // precision 6: FP32 J v caches in the kc/krc/qT storage -- per reaction k, k/Kc, dq/dT;
  // per species C, rho/W, W/rho, w, h/RT - esh, (cp - h)/T w / RT, Y dcp/dT / W, cp / W
  float *xk, *xkr, *xqT, *xC, *xE, *xEinv, *xom, *xg, *xh, *xdcp, *xcp;
  double *H, *LU, *piv, *red, *Bm;
  float *fC, *fdC, *fh, *fcp, *fdcp, *fom, *fq, *fkc, *fkr, *ftb, *fQ, *fw, *fpart;  // mixed precision
  int Nq;  // stride between Krylov / stage vectors
};

__device__ inline SlotPtrs slot_ptrs(double* b, const SlotLayout& s) {
  SlotPtrs p;
  p.u = b + s.u;
  p.src = b + s.src;
  p.fn = b + s.fn;
  p.arg = b + s.arg;
  p.fr = b + s.fr;
  p.F = b + s.F;
  p.w = b + s.w;
  p.Q = b + s.Q;
  p.K = b + s.K;
  p.C = b + s.C;
  p.dC = b + s.dC;
  p.cp = b + s.cp;
  p.hRT = b + s.hRT;
  p.dcp = b + s.dcp;
  p.gRT = b + s.gRT;
  p.E = b + s.E;
  p.Einv = b + s.Einv;
  p.CE = b + s.CE;
  p.om = b + s.om;
  p.q = b + s.q;
  p.kc = b + s.kc;
  p.krc = b + s.krc;
  p.qT = b + s.qT;
  p.tro = b + s.tro;
  p.part = b + s.part;
  p.C2 = s.C2 >= 0 ? reinterpret_cast<df2*>(b + s.C2) : nullptr;
  p.dC2 = s.dC2 >= 0 ? reinterpret_cast<df2*>(b + s.dC2) : nullptr;
  p.dig = s.dig >= 0 ? reinterpret_cast<uint16_t*>(b + s.dig) : nullptr;
  {
    const int nr_even = ((s.nr > 0 ? s.nr : 1) + 1) & ~1, ns1 = s.ns + 1;
    float* R = reinterpret_cast<float*>(b + s.kc);  // 3 nr_even doubles = 6 nr_even floats
    p.xk = R;
    p.xkr = R + nr_even;
    p.xqT = R + 2 * nr_even;
    float* X = s.fj >= 0 ? reinterpret_cast<float*>(b + s.fj) : R + 3 * nr_even;
    p.xC = X;
    p.xE = X + ns1;
    p.xEinv = X + 2 * ns1;
    p.xom = X + 3 * ns1;
    p.xg = X + 4 * ns1;
    p.xh = X + 5 * ns1;
    p.xdcp = X + 6 * ns1;
    p.xcp = X + 7 * ns1;
  }
  p.tb = b + s.tb;
  p.H = b + s.H;
  p.LU = b + s.LU;
  p.piv = b + s.piv;
  p.Bm = b + s.Bm;
  p.red = b + s.red;
  float* f = reinterpret_cast<float*>(b + s.fbase);
  p.fC = f + s.fC;
  p.fdC = f + s.fdC;
  p.fh = f + s.fh;
  p.fcp = f + s.fcp;
  p.fdcp = f + s.fdcp;
  p.fom = f + s.fom;
  p.fq = f + s.fq;
  p.fkc = f + s.fkc;
  p.fkr = f + s.fkr;
  p.ftb = f + s.ftb;
  p.fQ = f + s.fQ;
  p.fw = f + s.fw;
  p.fpart = f + s.fpart;
  p.Nq = (s.N + 1) & ~1;
  return p;
}

// w = nu^T q, pass 1: the species-major list is cut into pieces of near-equal
// length (chosen when the mechanism is packed); each lane sums whole pieces
// into part[], so the warp's loop runs over the longest piece rather than the
// longest species row.  Pass 2 (piece_sum) adds a species' pieces in order:
// the result does not depend on the launch shape.
template <int G, typename T>
__device__ __forceinline__ void gather_pieces(const MechView& m, int lane, const T* __restrict__ nu,
                                              const T* __restrict__ q, T* part) {
  for (int p = lane; p < m.npiece; p += G) {
    T acc = T(0);
    const int e1 = m.piece_ptr[p + 1];
    for (int e = m.piece_ptr[p]; e < e1; ++e) acc = fma(nu[e], q[m.csr_j[e]], acc);
    part[p] = acc;
  }
}
template <typename T>
__device__ __forceinline__ T piece_sum(const MechView& m, const T* part, int k) {
  const int p1 = m.spec_piece[k + 1];
  int p = m.spec_piece[k];
  T acc = part[p];
  for (++p; p < p1; ++p) acc += part[p];
  return acc;
}

// The same gather in double-float (FP32 pairs, ~44-bit significands, on the
// FP32 pipe): the net coefficients are small integers, exact in FP32, so each
// product nu_e q_j is formed with the pair's precision and summed by two-sums.
template <int G>
__device__ __forceinline__ void gather_pieces_df(const MechView& m, int lane, const df2* __restrict__ q,
                                                 df2* part) {
  for (int p = lane; p < m.npiece; p += G) {
    df2 acc = {0.0f, 0.0f};
    const int e1 = m.piece_ptr[p + 1];
    for (int e = m.piece_ptr[p]; e < e1; ++e) acc = df_add(acc, df_scale(m.csr_nuf[e], q[m.csr_j[e]]));
    part[p] = acc;
  }
}
__device__ __forceinline__ double piece_sum_df(const MechView& m, const df2* part, int k) {
  const int p1 = m.spec_piece[k + 1];
  int p = m.spec_piece[k];
  df2 acc = part[p];
  for (++p; p < p1; ++p) acc = df_add(acc, part[p]);
  return df_to(acc);
}

// ---- w = nu^T q on the tensor cores (precision level 4), exact to FP64 level.
// Each q_j is cut, relative to 2^Es with Es above the cell's largest |q_j|,
// into seven signed 8-bit digits (56 bits below 2^Es; what lies below
// 2^(Es - 56) is dropped, at most 2^-55 of the largest rate); the digits and
// the small-integer net coefficients are exact in BF16, each product is exact
// in FP32 and so is every sum the mma accumulates (|sum| <= 2 x 255 x Nr <
// 2^24), so the FP32 accumulators hold the digit columns of nu^T q exactly.
// mma.m16n8k16: A = a 16 x 16 tile of nu^T (species x reactions, prepacked
// per lane), B = the 16 x 8 tile of digits (reactions x digit 0..6, column 7
// zero), D = 16 species x 8 digit sums; FP64 then adds the seven scaled digit
// sums of each species (rounding once per addition, like a sum of terms).
__device__ __forceinline__ void mma_bf16_m16n8k16(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// A signed integer |v| <= 256 as BF16 (exact: its float's upper half).
__device__ __forceinline__ uint16_t bf16_of_small_int(int v) {
  return (uint16_t)(__float_as_uint((float)v) >> 16);
}

// x * 2^e for a double x holding an integer of magnitude below 2^53 and an
// exponent that keeps the result normal: an integer add to the exponent field.
__device__ __forceinline__ double scale_pow2(double x, int e) {
  return x == 0.0 ? 0.0 : exp_scale(x, e);
}

// out[k] = sum_j nu_jk q_j for the cell (q: Nr doubles in shared memory).
// Returns false, writing nothing, when every |q_j| < 2^-920 (the digit
// weights would leave the normal range): the caller then gathers in FP64.
template <int G>
__device__ bool gather_tc(const MechView& m, const SlotPtrs& s, const double* __restrict__ q,
                          double* __restrict__ out) {
  static_assert(G == 32, "the tensor-core gather runs one cell per warp");
  const Grp<G> g;
  const int lane = g.lane;
  const int nrp = 16 * m.nrt;
  // the scale: 2^(Eb - 1023) above every |q_j| (Eb one above the largest biased exponent)
  int emax = 0;
  for (int j = lane; j < m.nr; j += G) emax = max(emax, (__double2hiint(q[j]) >> 20) & 0x7ff);
  const int Eb = g.imax(emax) + 1;
  if (Eb < 104) return false;
  // digits of |q_j| 2^(56 - Es), most significant first, with q_j's sign
  for (int j = lane; j < m.nr; j += G) {
    const long long bits = __double_as_longlong(q[j]);
    const int e = (int)((bits >> 52) & 0x7ff);
    unsigned long long V = 0ull;
    if (e != 0) {  // zero and subnormal rates (below 2^-1022) drop out
      const unsigned long long mant = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const int sh = e + 4 - Eb;  // V = mant 2^sh < 2^56
      V = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
    }
    const bool neg = bits < 0;
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      const int dn = (int)((V >> (48 - 8 * n)) & 255ull);
      s.dig[n * nrp + j] = bf16_of_small_int(neg ? -dn : dn);
    }
  }
  g.sync();
  const int grp = lane >> 2, tq = lane & 3;
  const uint32_t* drow = reinterpret_cast<const uint32_t*>(s.dig + grp * nrp);
  // digit n weighs 2^(Es - 8 (n + 1)), Es = Eb - 1023
  const int w0 = Eb - 1023 - 8 * (2 * tq + 1), w1 = w0 - 8;
  for (int st = 0; st < m.nst; ++st) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    for (int rt = 0; rt < m.nrt; ++rt) {
      const uint4 a = m.nuT[(st * m.nrt + rt) * 32 + lane];
      mma_bf16_m16n8k16(d, a, drow[8 * rt + tq], drow[8 * rt + tq + 4]);
    }
    // this lane: digits 2tq and 2tq+1 of species rows grp (d0, d1) and grp + 8 (d2, d3)
    double r0 = scale_pow2((double)d[1], w1) + scale_pow2((double)d[0], w0);
    double r1 = scale_pow2((double)d[3], w1) + scale_pow2((double)d[2], w0);
    // add the four lanes of the group, least significant digits first
    r0 = __shfl_xor_sync(g.mask, r0, 1) + r0;
    r1 = __shfl_xor_sync(g.mask, r1, 1) + r1;
    r0 = __shfl_xor_sync(g.mask, r0, 2) + r0;
    r1 = __shfl_xor_sync(g.mask, r1, 2) + r1;
    if (tq == 0) {
      const int k0 = 16 * st + grp, k1 = k0 + 8;
      if (k0 < m.ns) out[k0] = r0;
      if (k1 < m.ns) out[k1] = r1;
    }
  }
  g.sync();
  return true;
}

// ------------------------------------------------------------ chemistry RHS
// out = f(uu) + src (src may be null).  p > 0: constant-pressure reactor at
// pressure p; p < 0: constant-volume reactor of density -p (Eq. cv_reactor with
// internal energies u_k/RT = h_k/RT - 1 and c_v/R = c_p/R - 1 per species).  uu, out: N-vectors in shared memory
// (out must not alias uu).  When `cache` is set, the values the analytic
// Jacobian-vector product reuses are kept (rate coefficients, w, d(cp/R)/dT
// and the cell scalars).  Inlined into the 32-lane FP64 integrator and called
// through rhs_eval_call elsewhere; each product that meets a sum is written as
// an explicit fma or __dmul_rn, so no copy can contract it differently,
// chem_rhs and the integrator compute the same bits and R(u) - R(u) is
// exactly zero in a steady-state cell.
template <int G, bool MIXED = false, bool TC = false>
__device__ __forceinline__ void rhs_eval(const MechView& m, const SlotPtrs& s, const double* uu,
                                      const double* src, double p, double* out, bool cache,
                                      CellScalars* cs) {
  const Grp<G> g;
  const int ns = m.ns;
  const double T = uu[ns];
  const double invT = rcp_newton(T);
  const double lnT = log_fast(T);
  const double lnRTp = LN_R_OVER_PREF + lnT;  // ln(R T / p_ref)
  // species pass 1: thermo, Gibbs factors, sum Y/W
  double S = 0.0;
  int ghi = 0;  // max over species of the high word of |g/RT + ln(RT/p_ref)| (integer compare)
  for (int k = g.lane; k < ns; k += G) {
    const double* c = (T < m.Tmid[k]) ? m.lo : m.hi;
    const double a1 = c[k], a2 = c[ns + k], a3 = c[2 * ns + k], a4 = c[3 * ns + k], a5 = c[4 * ns + k];
    const double cp = fma(fma(fma(fma(a5, T, a4), T, a3), T, a2), T, a1);
    const double hp = fma(fma(fma(c[8 * ns + k], T, c[7 * ns + k]), T, c[6 * ns + k]), T, c[5 * ns + k]);
    const double hrt = fma(c[9 * ns + k], invT, fma(hp, T, a1));
    const double sp = fma(fma(fma(c[12 * ns + k], T, c[11 * ns + k]), T, c[10 * ns + k]), T, a2);
    const double sr = fma(a1, lnT, fma(sp, T, c[13 * ns + k]));
    const double grt = hrt - sr;
    s.cp[k] = cp;
    s.hRT[k] = hrt;
    s.gRT[k] = grt;
    ghi = max(ghi, __double2hiint(grt + lnRTp) & 0x7fffffff);
    if (cache) {
      const double dcp = fma(fma(fma(c[16 * ns + k], T, c[15 * ns + k]), T, c[14 * ns + k]), T, a2);
      s.dcp[k] = dcp;
      // (h/RT - 1)/T, whose sum over a reaction's products less its reactants is
      // d ln Kc/dT; kept in dC, which the J v overwrites later (sentinel entry 0)
      s.dC[k] = __dmul_rn(hrt - 1.0, invT);
      if (MIXED) {
        s.fh[k] = __double2float_rn(hrt);
        s.fcp[k] = __double2float_rn(cp);
        s.fdcp[k] = __double2float_rn(dcp);
      }
    }
    S = fma(uu[k], m.invW[k], S);
  }
  S = g.sum(S);
  ghi = g.imax(ghi);
  const bool direct_kc = ghi >= G_OVERFLOW_HI;  // some |g/RT + ln(RT/p_ref)| >= 170, also NaN
  // auxiliary-temperature system (Eq. chemical_source_balanced): the species
  // components are rho Y_k, so C_k = u_k / W_k and d(rho Y_k)/dt = W_k w_k:
  // the constant-volume arithmetic with unit density
  const bool aux = m.nx > 0;
  const bool cv = p < 0.0 || aux;
  const double esh = cv ? 1.0 : 0.0;  // h/RT -> u/RT and cp/R -> cv/R shift
  const double invS = rcp_newton(S);
  // rho = p / (R T S), 1/rho = R T S / p, with 1/p (or 1/rho) from the caller
  const double rho = aux ? 1.0 : (cv ? -p : p * invT * invS * INV_R);
  const double invrho = aux ? 1.0 : (cv ? cs->pinv : R_GAS * T * S * cs->pinv);
  // concentrations, Gibbs factors, and (for up to MAXM pressure-dependent
  // reactions) the third-body concentrations [M]_t = sum_k eff_tk C_k
  const bool coop_tb = m.ntb > 0 && m.ntb <= MAXM;
  double mp[MAXM];
#pragma unroll
  for (int t = 0; t < MAXM; ++t) mp[t] = 0.0;
  for (int k = g.lane; k < ns; k += G) {
    const double Ck = rho * uu[k] * m.invW[k];
    s.C[k] = Ck;
    if (MIXED && cache) s.fC[k] = __double2float_rn(Ck);
    if (cache && cs->prec == 3) s.C2[k] = df_from(Ck);
    if (!direct_kc) {
      // E = e^{g/RT} (RT/p_ref), Einv = 1/E: 1/Kc of a reaction is the product of
      // E over its products and Einv over its reactants (the pressure factor
      // (RT/p_ref)^dnu included); CE = C E, so k/Kc prod C^nu'' is three products
      // (in FP64 at every precision level: the equilibrium constants come from these)
      const double a = s.gRT[k] + lnRTp;
      exp_pm(a, m.etab, &s.E[k], &s.Einv[k]);
      s.CE[k] = __dmul_rn(Ck, s.E[k]);
    }
    if (coop_tb) {
#pragma unroll
      for (int t = 0; t < MAXM; ++t)
        if (t < m.ntb) mp[t] = fma(m.eff[t * ns + k], Ck, mp[t]);
    }
  }
  if (coop_tb) {
    sum_first<G>(g, mp, m.ntb);
    if (g.lane == 0) {
#pragma unroll
      for (int t = 0; t < MAXM; ++t)
        if (t < m.ntb) s.tb[4 * t] = mp[t];
    }
  }
  g.sync();
  // Troe falloff factors (Sec. 4.4 kinetics; F_cent, Pr, F), spread over the
  // lanes in three passes instead of one lane per reaction running the whole
  // chain: (A) the four exponentials of each reaction, k0/k_inf, e^{-T/T***},
  // e^{-T/T*}, e^{-T**/T}; (B) log10 F_cent and log10 Pr; (C) F, the falloff
  // multiplier Pr/(1+Pr) F and, when caching, d ln k/dT and dk/d[M] / k_inf.
  // Scratch tro (nt = ntroe): [0,4nt) exponentials, [4nt,6nt) logs,
  // [6nt,7nt) multiplier, [7nt,8nt) d ln k/dT, [8nt,9nt) dk/d[M] / k_inf,
  // [9nt,11nt) F_cent and Pr.
  const int nt = m.ntroe;
  if (nt > 0) {
    double* tro = s.tro;
    for (int l = g.lane; l < 4 * nt; l += G) {
      const int i = l >> 2, c = l & 3;
      const double* fo = m.fo + (size_t)i * FO_STRIDE;
      double x;
      if (c == 0) {
        const double lnk_inf = fma(-m.EaR[i], invT, fma(m.bexp[i], lnT, m.lnA[i]));
        x = fma(-fo[2], invT, fma(fo[1], lnT, fo[0])) - lnk_inf;  // ln(k0 / k_inf)
      } else if (c == 1) {
        x = -T * fo[4];
      } else if (c == 2) {
        x = -T * fo[5];
      } else {
        x = fo[6] > 0.0 ? -fo[6] * invT : 0.0;
      }
      const double ex = exp_fast(x, m.etab);
      tro[l] = (c == 3 && !(fo[6] > 0.0)) ? 0.0 : ex;
    }
    g.sync();
    for (int l = g.lane; l < 2 * nt; l += G) {
      const int i = l >> 1;
      const double* fo = m.fo + (size_t)i * FO_STRIDE;
      double y;
      if (l & 1) {
        double Mc;
        if (coop_tb) {
          Mc = s.tb[4 * i];
        } else {
          const double* e = m.eff + (size_t)i * ns;
          Mc = 0.0;
          for (int q = 0; q < ns; ++q) Mc = fma(e[q], s.C[q], Mc);
        }
        y = tro[4 * i] * Mc;  // Pr = [M] k0 / k_inf
        if (!(y > 1e-300)) y = 1e-300;
      } else {
        const double a = fo[3];
        y = fma(1.0 - a, tro[4 * i + 1], fma(a, tro[4 * i + 2], tro[4 * i + 3]));  // F_cent
      }
      tro[9 * nt + l] = y;
      tro[4 * nt + l] = __dmul_rn(log_fast(y), RK_INV_LN10);
    }
    g.sync();
    for (int i = g.lane; i < nt; i += G) {
      const double lFc = tro[4 * nt + 2 * i], lPr = tro[4 * nt + 2 * i + 1];
      const double Fc = tro[9 * nt + 2 * i], Pr = tro[9 * nt + 2 * i + 1];
      const double cc = fma(-0.67, lFc, -0.4);
      const double nn = fma(-1.27, lFc, 0.75);
      const double x = lPr + cc;
      const double D = fma(-0.14, x, nn);
      // one division for 1/(1 + Pr) and 1/(D^2 + x^2):
      //   1/(1 + f1^2) = D^2/(D^2 + x^2) with f1 = x / D
      const double s2 = fma(D, D, x * x);
      const double onePr = 1.0 + Pr;
      const double qd = rcp_any(__dmul_rn(onePr, s2));
      const double iOnePr = s2 * qd;
      const double rr = onePr * qd;  // 1 / (D^2 + x^2)
      const double iden = D * D * rr;
      const double F = exp_fast(lFc * iden * 2.302585092994046, m.etab);  // 10^(lFc / (1 + f1^2))
      tro[6 * nt + i] = Pr * iOnePr * F;
      if (cache) {  // d ln k / dT and d k / d[M] for the analytic J v
        const double* fo = m.fo + (size_t)i * FO_STRIDE;
        const double a = fo[3];
        const double er = tro[4 * i], e3 = tro[4 * i + 1], e1 = tro[4 * i + 2], e2 = tro[4 * i + 3];
        const double dlnk_inf = __dmul_rn(fma(m.EaR[i], invT, m.bexp[i]), invT);
        const double dlnk0 = __dmul_rn(fma(fo[2], invT, fo[1]), invT);
        // d ln F / d log10 Pr = -2 lFc f1 n / (D^2 (1 + f1^2)^2) and
        // d log10 F / d lFc = 1/(1 + f1^2) - 2 lFc f1 (df1/dlFc) / (1 + f1^2)^2,
        // df1/dlFc = (-0.67 D + 1.1762 x) / D^2, written with rr = 1/(D^2 + x^2)
        // (every product that meets a sum is an explicit fma or __dmul_rn, so
        // the compiler cannot contract it differently where this is inlined)
        const double w = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, lFc), x), D), rr), rr);
        const double gg = fma(-w, nn, iOnePr);
        const double dlF_dlFc = fma(-w, fma(-0.67, D, __dmul_rn(1.1762, x)), iden);
        const double e2t = fo[6] > 0.0 ? __dmul_rn(__dmul_rn(__dmul_rn(fo[6], invT), invT), e2) : 0.0;
        const double dFc = fma(-(1.0 - a), __dmul_rn(fo[4], e3), fma(-a, __dmul_rn(fo[5], e1), e2t));
        tro[7 * nt + i] = fma(__dmul_rn(dlF_dlFc, dFc), rcp_any(Fc), fma(gg, dlnk0 - dlnk_inf, dlnk_inf));
        tro[8 * nt + i] = er * F * iOnePr * gg;  // (dk/d[M]) / k_inf
      }
    }
    g.sync();
  }
  // reactions: rate coefficients and rates of progress
  const double m_lnRTp = -lnRTp;
  for (int j = g.lane; j < m.nr; j += G) {
    const uint32_t sl = m.slots[j];
    const int ra = sl & 255, rb = (sl >> 8) & 255, pa = (sl >> 16) & 255, pb = sl >> 24;
    const int meta = m.meta[j];
    const int kind = meta & 3;
    const bool rev = (meta >> 2) & 1;
    const int dnu = ((meta >> 4) & 15) - 4;
    const double lnk = fma(-m.EaR[j], invT, fma(m.bexp[j], lnT, m.lnA[j]));
    double k = (MIXED || cs->prec == 3 || cs->prec >= 5) ? exp_mixed(lnk, m.etab) : exp_fast(lnk, m.etab);
    const double Pf = __dmul_rn(s.C[ra], s.C[rb]);
    // Rb = prod C^nu'' / Kc (the caching evaluation keeps it), rfac = 1/Kc
    // (caching only), PfRb = Pf - Rb: from the per-species factors as
    // (C_pa E_pa C_pb E_pb) (1/E_ra 1/E_rb) subtracted from Pf in one fma
    double Rb = 0.0, rfac = 0.0, PfRb = Pf;
    if (rev) {
      if (!direct_kc) {
        const double X = __dmul_rn(s.CE[pa], s.CE[pb]);
        const double Y = __dmul_rn(s.Einv[ra], s.Einv[rb]);
        PfRb = fma(-X, Y, Pf);
        if (cache) {
          Rb = __dmul_rn(X, Y);
          rfac = __dmul_rn(__dmul_rn(s.E[pa], s.E[pb]), Y);
        }
      } else {
        const double dl = dnu > 0 ? lnRTp : (dnu < 0 ? m_lnRTp : 0.0);
        rfac = exp_fast(s.gRT[pa] + s.gRT[pb] - s.gRT[ra] - s.gRT[rb] + dl, m.etab);
        Rb = __dmul_rn(rfac, __dmul_rn(s.C[pa], s.C[pb]));
        PfRb = __dsub_rn(Pf, Rb);
      }
    }
    double mfac = 1.0;
    double dlnk = 0.0;  // d ln k / dT (cache only)
    if (cache) dlnk = __dmul_rn(fma(m.EaR[j], invT, m.bexp[j]), invT);
    if (kind != 0) {
      const int slot = meta >> 8;
      double Mc;
      if (coop_tb) {
        Mc = s.tb[4 * slot];
      } else {
        const double* e = m.eff + (size_t)slot * ns;
        Mc = 0.0;
        for (int q = 0; q < ns; ++q) Mc = fma(e[q], s.C[q], Mc);
      }
      double dkdM = 0.0;
      if (kind == 1) {
        mfac = Mc;
      } else {
        // Troe: the multiplier and derivatives from the falloff passes above
        // (Troe reactions hold slots 0..ntroe-1)
        if (cache) {
          dlnk = s.tro[7 * nt + slot];
          dkdM = k * s.tro[8 * nt + slot];
        }
        k = k * s.tro[6 * nt + slot];
      }
      if (cache) {
        double* t = s.tb + 4 * (meta >> 8);
        t[0] = Mc;
        t[1] = dkdM;
        t[2] = dlnk;
        t[3] = rfac;
        if (MIXED) {
          float* tf = s.ftb + 4 * (meta >> 8);
          tf[0] = __double2float_rn(Mc);
          tf[1] = __double2float_rn(dkdM);
          tf[2] = __double2float_rn(dlnk);
          tf[3] = __double2float_rn(rfac);
        }
      }
    }
    // q = m k (prod C^nu' - prod C^nu'' / Kc); the third-body factor only where there is one
    const double q0 = __dmul_rn(k, PfRb);
    double qj = q0;
    if (kind == 1) qj = __dmul_rn(mfac, qj);
    if (MIXED) reinterpret_cast<df2*>(s.q)[j] = df_from(qj);  // double-float copy for the gather
    else s.q[j] = qj;
    if (cache) {
      const double kr = __dmul_rn(k, rfac);
      // d q_j / dT at fixed concentrations (without the third-body factor):
      // d ln k/dT q0 + d ln Kc/dT k prod C^nu''/Kc, q0 = k (prod C^nu' - prod C^nu''/Kc),
      // with d ln Kc/dT = (sum_products h/RT - sum_reactants h/RT - dnu) / T
      // summed from the per-species (h/RT - 1)/T
      const double dlnKc = __dsub_rn(__dadd_rn(s.dC[pa], s.dC[pb]), __dadd_rn(s.dC[ra], s.dC[rb]));
      const double qT = fma(dlnk, q0, __dmul_rn(dlnKc, __dmul_rn(k, Rb)));
      if (cs->prec == 3) {  // double-float copies for the J v core, in the same storage
        reinterpret_cast<df2*>(s.qT)[j] = df_from(qT);
        reinterpret_cast<df2*>(s.kc)[j] = df_from(k);
        reinterpret_cast<df2*>(s.krc)[j] = df_from(kr);
      } else if (cs->prec == 6) {  // FP32 copies for the FP32 J v, in the same storage
        s.xk[j] = __double2float_rn(k);
        s.xkr[j] = __double2float_rn(kr);
        s.xqT[j] = __double2float_rn(qT);
      } else {
        s.qT[j] = qT;
        s.kc[j] = k;
        s.krc[j] = kr;
      }
      if (MIXED) {
        s.fkc[j] = __double2float_rn(k);
        s.fkr[j] = __double2float_rn(kr);
      }
    }
  }
  g.sync();
  // species pass 2: w = nu^T q, dY/dt and the sums of the temperature equation
  double Sh = 0.0, cb = 0.0;
  double Ax = 0.0, Bx = 0.0;  // auxiliary T: sum (u_k/RT) F_k / W_k and sum (cv_k/R) F_k / W_k
  bool tc_om = false;  // w already in part[0..ns) from the tensor cores
  if constexpr (TC) tc_om = gather_tc<G>(m, s, s.q, s.part);
  if (MIXED) gather_pieces_df<G>(m, g.lane, reinterpret_cast<const df2*>(s.q), reinterpret_cast<df2*>(s.part));
  else if (!tc_om) gather_pieces<G, double>(m, g.lane, m.csr_nu, s.q, s.part);
  g.sync();
  for (int k = g.lane; k < ns; k += G) {
    double om;
    if (MIXED) {
      om = piece_sum_df(m, reinterpret_cast<const df2*>(s.part), k);
      if (cache) s.fom[k] = __double2float_rn(om);
    } else {
      om = tc_om ? s.part[k] : piece_sum(m, s.part, k);
    }
    if (cache) s.om[k] = om;
    const double r = __dmul_rn(__dmul_rn(m.W[k], om), invrho);
    const double Fk = src ? __dadd_rn(r, src[k]) : r;
    out[k] = Fk;
    Sh = fma(s.hRT[k] - esh, om, Sh);
    cb = fma(uu[k] * (s.cp[k] - esh), m.invW[k], cb);
    if (aux) {
      Ax = fma((s.hRT[k] - 1.0) * Fk, m.invW[k], Ax);
      Bx = fma((s.cp[k] - 1.0) * Fk, m.invW[k], Bx);
    }
    if (cache) {
      // per-species factors of the analytic J v, written over arrays the
      // remaining RHS no longer reads (lane-private entries k):
      //   E: rho/W_k   Einv: W_k/rho   gRT: h_k/RT - esh
      //   hRT: (cp_k/R - h_k/RT) w_k / T   dcp: Y_k (dcp_k/dT) / W_k   cp: (cp_k/R - esh) / W_k
      s.E[k] = rho * m.invW[k];
      s.Einv[k] = m.W[k] * invrho;
      s.gRT[k] = s.hRT[k] - esh;
      s.hRT[k] = (s.cp[k] - s.hRT[k]) * invT * om;
      s.dcp[k] = uu[k] * s.dcp[k] * m.invW[k];
      s.cp[k] = (s.cp[k] - esh) * m.invW[k];
      if (cs->prec == 6) {  // FP32 copies for the FP32 J v
        s.xC[k] = __double2float_rn(s.C[k]);
        s.xE[k] = __double2float_rn(s.E[k]);
        s.xEinv[k] = __double2float_rn(s.Einv[k]);
        s.xom[k] = __double2float_rn(om);
        s.xg[k] = __double2float_rn(s.gRT[k]);
        s.xh[k] = __double2float_rn(s.hRT[k]);
        s.xdcp[k] = __double2float_rn(s.dcp[k]);
        s.xcp[k] = __double2float_rn(s.cp[k]);
      }
    }
  }
  if (aux) {
    double t4[4] = {Sh, cb, Ax, Bx};
    sum_many<G, 4>(g, t4);
    Sh = t4[0];
    cb = t4[1];
    Ax = t4[2];
    Bx = t4[3];
  } else {
    double t2[2] = {Sh, cb};
    sum_many<G, 2>(g, t2);
    Sh = t2[0];
    cb = t2[1];
  }
  const double invcb = rcp_newton(cb);
  double fT = 0.0;
  if (aux) {
    // Eq. aux_t_equation with specific internal energies e_k = (u_k/RT) R T / W_k
    // and rho c_v = R cb:  w_T = (-R T Ax + |v|^2/2 d(rho)/dt - v . d(rho v)/dt
    //                              + d(rho E)/dt) / (R cb)
    const double irc = 1.0 / uu[ns + 1];
    const double v0 = uu[ns + 2] * irc, v1 = uu[ns + 3] * irc, v2 = uu[ns + 4] * irc;
    double X = 0.0;
    if (src) {
      const double kin = 0.5 * fma(v0, v0, fma(v1, v1, v2 * v2));
      X = fma(kin, src[ns + 1], src[ns + 5]) - fma(v0, src[ns + 2], fma(v1, src[ns + 3], v2 * src[ns + 4]));
    }
    fT = fma(-T, Ax, X * INV_R) * invcb;
    if (cache) {
      cs->B = Bx;
      cs->fT = fT;
      cs->irho_c = irc;
      cs->vel[0] = v0;
      cs->vel[1] = v1;
      cs->vel[2] = v2;
    }
    // d(rho)/dt, d(rho v)/dt, d(rho E)/dt: the balancing constants alone
    for (int e = ns + 1 + g.lane; e < ns + 1 + m.nx; e += G) out[e] = src ? src[e] : 0.0;
  }
  if (g.lane == 0) {
    const double r = aux ? fT : -T * Sh * invrho * invcb;
    out[ns] = src ? __dadd_rn(r, src[ns]) : r;
    if (cache && cs->prec == 6) s.xC[ns] = 1.f;  // the empty reaction slot
  }
  if (cache) {
    cs->T = T;
    cs->invT = invT;
    cs->lnT = lnT;
    cs->S = S;
    cs->invS = invS;
    cs->rho = rho;
    cs->invrho = invrho;
    cs->cb = cb;
    cs->invcb = invcb;
    cs->Sh = Sh;
    cs->cv = cv;
  }
  g.sync();
}

// rhs_eval behind a call, where its size matters more than the call: the
// point kernels, the finite-difference J v, the explicit integrator's first
// evaluation and the 8/16-lane and mixed variants of the integrator (one
// inlined copy per call site would multiply the compile time).  Same bits as
// the inlined copies.
template <int G, bool MIXED = false, bool TC = false>
__device__ __noinline__ void rhs_eval_call(const MechView& m, const SlotPtrs& s, const double* uu,
                                           const double* src, double p, double* out, bool cache,
                                           CellScalars* cs) {
  rhs_eval<G, MIXED, TC>(m, s, uu, src, p, out, cache, cs);
}
template <int G, bool MIXED, bool INL, bool TC = false>
__device__ __forceinline__ void rhs_dispatch(const MechView& m, const SlotPtrs& s, const double* uu,
                                             const double* src, double p, double* out, bool cache,
                                             CellScalars* cs) {
  if constexpr (INL) rhs_eval<G, MIXED, TC>(m, s, uu, src, p, out, cache, cs);
  else rhs_eval_call<G, MIXED, TC>(m, s, uu, src, p, out, cache, cs);
}

// Analytic Jacobian-vector product out = J(u_n) v, using the values cached by
// the last rhs_eval(..., cache = true) at u_n.  v, out: N-vectors.  Inlined
// (unlike rhs_eval, nothing requires two call sites to produce the same bits),
// which saves the call's register save and restore four times per attempt.
template <int G, bool DFG = false, bool TC = false>
__device__ __forceinline__ void jvp_eval(const MechView& m, const SlotPtrs& s, const double* uu,
                                      const CellScalars& cs, const double* v, double* out) {
  const Grp<G> g;
  const int ns = m.ns;
  const double vT = v[ns];
  const double T = cs.T, invT = cs.invT;
  double a = 0.0;
  for (int k = g.lane; k < ns; k += G) a = fma(v[k], m.invW[k], a);
  a = g.sum(a);
  const double drr = cs.cv ? 0.0 : -fma(a, cs.invS, vT * invT);  // d rho / rho (0 at fixed volume)
  const bool coop_tb = m.ntb > 0 && m.ntb <= MAXM;
  double mp[MAXM];
#pragma unroll
  for (int t = 0; t < MAXM; ++t) mp[t] = 0.0;
  for (int k = g.lane; k < ns; k += G) {
    const double dCk = fma(s.C[k], drr, s.E[k] * v[k]);  // E: rho / W_k
    s.dC[k] = dCk;
    if (coop_tb) {
#pragma unroll
      for (int t = 0; t < MAXM; ++t)
        if (t < m.ntb) mp[t] = fma(m.eff[t * ns + k], dCk, mp[t]);
    }
  }
  if (coop_tb) sum_first<G>(g, mp, m.ntb);  // d[M]_t, identical on every lane
  g.sync();
  for (int j = g.lane; j < m.nr; j += G) {
    const uint32_t sl = m.slots[j];
    const int ra = sl & 255, rb = (sl >> 8) & 255, pa = (sl >> 16) & 255, pb = sl >> 24;
    const int meta = m.meta[j];
    const int kind = meta & 3;
    const double dPf = fma(s.dC[ra], s.C[rb], s.C[ra] * s.dC[rb]);
    const double dPb = fma(s.dC[pa], s.C[pb], s.C[pa] * s.dC[pb]);
    const double k = s.kc[j], kr = s.krc[j];
    double dq = fma(s.qT[j], vT, fma(k, dPf, -kr * dPb));
    if (kind != 0) {
      const int slot = meta >> 8;
      const double* t = s.tb + 4 * slot;
      const double Pf = s.C[ra] * s.C[rb];
      const double Pb = s.C[pa] * s.C[pb];
      double dM = 0.0;
      if (coop_tb) {
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q == slot) dM = mp[q];
      } else {
        const double* e = m.eff + (size_t)slot * ns;
        for (int q = 0; q < ns; ++q) dM = fma(e[q], s.dC[q], dM);
      }
      if (kind == 1) dq = t[0] * dq + dM * (k * Pf - kr * Pb);
      else dq = dq + t[1] * dM * (Pf - t[3] * Pb);
    }
    if (DFG) reinterpret_cast<df2*>(s.q)[j] = df_from(dq);
    else s.q[j] = dq;
  }
  g.sync();
  bool tc_om = false;  // d w already in part[0..ns) from the tensor cores
  if constexpr (TC) tc_om = gather_tc<G>(m, s, s.q, s.part);
  if (DFG) gather_pieces_df<G>(m, g.lane, reinterpret_cast<const df2*>(s.q), reinterpret_cast<df2*>(s.part));
  else if (!tc_om) gather_pieces<G, double>(m, g.lane, m.csr_nu, s.q, s.part);
  g.sync();
  double dSh = 0.0, dcb = 0.0;
  for (int k = g.lane; k < ns; k += G) {
    const double dom = DFG ? piece_sum_df(m, reinterpret_cast<const df2*>(s.part), k)
                           : (tc_om ? s.part[k] : piece_sum(m, s.part, k));
    out[k] = s.Einv[k] * fma(-s.om[k], drr, dom);  // Einv: W_k / rho
    dSh = fma(s.gRT[k], dom, fma(s.hRT[k], vT, dSh));
    dcb = fma(s.dcp[k], vT, fma(s.cp[k], v[k], dcb));
  }
  if (m.nx > 0) {
    // auxiliary temperature: d w_T = (-vT B - T sum_k (u_k/RT) dF_k/W_k + dX/R - w_T dcb) / cb,
    // dF_k = W_k dw_k, X = |v|^2/2 S_rho - v . S_m + S_E, dv = (d(rho v) - v d rho) / rho
    double D1 = 0.0;
    for (int k = g.lane; k < ns; k += G) D1 = fma(s.gRT[k], out[k] * m.invW[k], D1);  // gRT: h/RT - 1
    double t2[2] = {D1, dcb};
    sum_many<G, 2>(g, t2);
    D1 = t2[0];
    dcb = t2[1];
    if (g.lane == 0) {
      const double irc = cs.irho_c;
      const double dv0 = (v[ns + 2] - cs.vel[0] * v[ns + 1]) * irc;
      const double dv1 = (v[ns + 3] - cs.vel[1] * v[ns + 1]) * irc;
      const double dv2 = (v[ns + 4] - cs.vel[2] * v[ns + 1]) * irc;
      const double* S = s.src;  // the cell's balancing constants
      const double dX = fma(dv0, fma(cs.vel[0], S[ns + 1], -S[ns + 2]),
                            fma(dv1, fma(cs.vel[1], S[ns + 1], -S[ns + 3]), dv2 * fma(cs.vel[2], S[ns + 1], -S[ns + 4])));
      out[ns] = (fma(-vT, cs.B, fma(-T, D1, dX * INV_R)) - cs.fT * dcb) * cs.invcb;
    }
    for (int e = ns + 1 + g.lane; e < ns + 1 + m.nx; e += G) out[e] = 0.0;
    g.sync();
    return;
  }
  {
    double t2[2] = {dSh, dcb};
    sum_many<G, 2>(g, t2);
    dSh = t2[0];
    dcb = t2[1];
  }
  if (g.lane == 0) {
    out[ns] = (-(vT * cs.Sh + T * dSh) + T * cs.Sh * (drr + dcb * cs.invcb)) * (cs.invrho * cs.invcb);
  }
  g.sync();
}

// Analytic J v with its reaction-level core in double-float (precision 3):
// dP = d(C_a C_b), dq_j = qT_j vT + k_j dPf - kr_j dPb and the gather
// dw = nu^T dq run on the FP32 pipe with ~44-bit significands from the
// double-float copies rhs_eval wrote at u_n; the species and temperature rows
// (and the third-body / falloff corrections) stay FP64.  Same derivative as
// jvp_eval to ~1e-13 relative, so the Krylov basis is that of the FP64 path.
template <int G>
__device__ __forceinline__ void jvp_eval_df(const MechView& m, const SlotPtrs& s, const double* uu,
                                         const CellScalars& cs, const double* v, double* out) {
  const Grp<G> g;
  const int ns = m.ns;
  const double vT = v[ns];
  const double T = cs.T, invT = cs.invT;
  double a = 0.0;
  for (int k = g.lane; k < ns; k += G) a = fma(v[k], m.invW[k], a);
  a = g.sum(a);
  const double drr = cs.cv ? 0.0 : -fma(a, cs.invS, vT * invT);
  const bool coop_tb = m.ntb > 0 && m.ntb <= MAXM;
  double mp[MAXM];
#pragma unroll
  for (int t = 0; t < MAXM; ++t) mp[t] = 0.0;
  for (int k = g.lane; k < ns; k += G) {
    const double dCk = fma(s.C[k], drr, s.E[k] * v[k]);  // E: rho / W_k
    s.dC[k] = dCk;
    s.dC2[k] = df_from(dCk);
    if (coop_tb) {
#pragma unroll
      for (int t = 0; t < MAXM; ++t)
        if (t < m.ntb) mp[t] = fma(m.eff[t * ns + k], dCk, mp[t]);
    }
  }
  if (coop_tb) sum_first<G>(g, mp, m.ntb);
  g.sync();
  const df2 vT2 = df_from(vT);
  const df2* k2 = reinterpret_cast<const df2*>(s.kc);
  const df2* kr2 = reinterpret_cast<const df2*>(s.krc);
  const df2* qT2 = reinterpret_cast<const df2*>(s.qT);
  df2* dq2 = reinterpret_cast<df2*>(s.q);
  for (int j = g.lane; j < m.nr; j += G) {
    const uint32_t sl = m.slots[j];
    const int ra = sl & 255, rb = (sl >> 8) & 255, pa = (sl >> 16) & 255, pb = sl >> 24;
    const int meta = m.meta[j];
    const int kind = meta & 3;
    const df2 dPf = df_add(df_mul(s.dC2[ra], s.C2[rb]), df_mul(s.C2[ra], s.dC2[rb]));
    const df2 dPb = df_add(df_mul(s.dC2[pa], s.C2[pb]), df_mul(s.C2[pa], s.dC2[pb]));
    df2 dq = df_add(df_mul(qT2[j], vT2), df_add(df_mul(k2[j], dPf), df_neg(df_mul(kr2[j], dPb))));
    if (kind != 0) {  // third body / falloff: the [M] terms in FP64
      const int slot = meta >> 8;
      const double* t = s.tb + 4 * slot;
      const double Pf = s.C[ra] * s.C[rb];
      const double Pb = s.C[pa] * s.C[pb];
      double dM = 0.0;
      if (coop_tb) {
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q == slot) dM = mp[q];
      } else {
        const double* e = m.eff + (size_t)slot * ns;
        for (int q = 0; q < ns; ++q) dM = fma(e[q], s.dC[q], dM);
      }
      const double dqd = df_to(dq);
      double r;
      if (kind == 1) r = t[0] * dqd + dM * (df_to(k2[j]) * Pf - df_to(kr2[j]) * Pb);
      else r = dqd + t[1] * dM * (Pf - t[3] * Pb);
      dq = df_from(r);
    }
    dq2[j] = dq;
  }
  g.sync();
  gather_pieces_df<G>(m, g.lane, dq2, reinterpret_cast<df2*>(s.part));
  g.sync();
  double dSh = 0.0, dcb = 0.0;
  for (int k = g.lane; k < ns; k += G) {
    const double dom = piece_sum_df(m, reinterpret_cast<const df2*>(s.part), k);
    out[k] = s.Einv[k] * fma(-s.om[k], drr, dom);  // Einv: W_k / rho
    dSh = fma(s.gRT[k], dom, fma(s.hRT[k], vT, dSh));
    dcb = fma(s.dcp[k], vT, fma(s.cp[k], v[k], dcb));
  }
  {
    double t2[2] = {dSh, dcb};
    sum_many<G, 2>(g, t2);
    dSh = t2[0];
    dcb = t2[1];
  }
  if (g.lane == 0) {
    out[ns] = (-(vT * cs.Sh + T * dSh) + T * cs.Sh * (drr + dcb * cs.invcb)) * (cs.invrho * cs.invcb);
  }
  g.sync();
}

// Reduced-precision analytic J v (mixed mode): the same derivative as
// jvp_eval evaluated in FP32 from the FP32 copies cached by
// rhs_eval<G, true>(..., cache = true).  v and out stay FP64 vectors.
template <int G>
__device__ __noinline__ void jvp_eval_f32(const MechView& m, const SlotPtrs& s, const double* uu,
                                          const CellScalars& cs, const double* v, double* out) {
  const Grp<G> g;
  const int ns = m.ns;
  const float vT = __double2float_rn(v[ns]);
  const float T = __double2float_rn(cs.T), invT = __double2float_rn(cs.invT);
  const float invS = __double2float_rn(cs.invS), rho = __double2float_rn(cs.rho);
  const float invrho = __double2float_rn(cs.invrho), Sh = __double2float_rn(cs.Sh);
  const float invcb = __double2float_rn(cs.invcb);
  float a = 0.f;
  for (int k = g.lane; k < ns; k += G) a = fmaf(__double2float_rn(v[k]), m.invWf[k], a);
  a = g.sum(a);
  const float drr = cs.cv ? 0.f : -fmaf(a, invS, vT * invT);
  const float esh = cs.cv ? 1.f : 0.f;
  const bool coop_tb = m.ntb > 0 && m.ntb <= MAXM;
  float mp[MAXM];
#pragma unroll
  for (int t = 0; t < MAXM; ++t) mp[t] = 0.f;
  for (int k = g.lane; k < ns; k += G) {
    const float dCk = fmaf(s.fC[k], drr, rho * __double2float_rn(v[k]) * m.invWf[k]);
    s.fdC[k] = dCk;
    if (coop_tb) {
#pragma unroll
      for (int t = 0; t < MAXM; ++t)
        if (t < m.ntb) mp[t] = fmaf(m.efff[t * ns + k], dCk, mp[t]);
    }
  }
  if (coop_tb) sum_first<G>(g, mp, m.ntb);
  g.sync();
  for (int j = g.lane; j < m.nr; j += G) {
    const uint32_t sl = m.slots[j];
    const int ra = sl & 255, rb = (sl >> 8) & 255, pa = (sl >> 16) & 255, pb = sl >> 24;
    const int meta = m.meta[j];
    const int kind = meta & 3;
    const int dnu = ((meta >> 4) & 15) - 4;
    const float Pf = s.fC[ra] * s.fC[rb];
    const float Pb = s.fC[pa] * s.fC[pb];
    const float dPf = fmaf(s.fdC[ra], s.fC[rb], s.fC[ra] * s.fdC[rb]);
    const float dPb = fmaf(s.fdC[pa], s.fC[pb], s.fC[pa] * s.fdC[pb]);
    const float k = s.fkc[j], kr = s.fkr[j];
    float dlnk = (m.bf[j] + m.EaRf[j] * invT) * invT;
    const float dnud = dnu > 0 ? 1.f : (dnu < 0 ? -1.f : 0.f);
    const float dlnKc = (s.fh[pa] + s.fh[pb] - s.fh[ra] - s.fh[rb] - dnud) * invT;
    if (kind == 2) dlnk = s.ftb[4 * (meta >> 8) + 2];
    float dq = k * fmaf(dlnk * vT, Pf, dPf) - kr * fmaf((dlnk - dlnKc) * vT, Pb, dPb);
    if (kind != 0) {
      const int slot = meta >> 8;
      const float* t = s.ftb + 4 * slot;
      float dM = 0.f;
      if (coop_tb) {
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q == slot) dM = mp[q];
      } else {
        const float* e = m.efff + (size_t)slot * ns;
        for (int q = 0; q < ns; ++q) dM = fmaf(e[q], s.fdC[q], dM);
      }
      if (kind == 1) dq = t[0] * dq + dM * (k * Pf - kr * Pb);
      else dq = dq + t[1] * dM * (Pf - t[3] * Pb);
    }
    s.fq[j] = dq;
  }
  g.sync();
  gather_pieces<G, float>(m, g.lane, m.csr_nuf, s.fq, s.fpart);
  g.sync();
  float dSh = 0.f, dcb = 0.f;
  for (int k = g.lane; k < ns; k += G) {
    const float dom = piece_sum(m, s.fpart, k);
    const float om = s.fom[k];
    const float vk = __double2float_rn(v[k]);
    out[k] = (double)(m.Wf[k] * (dom - om * drr) * invrho);
    dSh = fmaf(s.fh[k] - esh, dom, fmaf((s.fcp[k] - s.fh[k]) * invT * vT, om, dSh));
    dcb = fmaf(fmaf(__double2float_rn(uu[k]) * s.fdcp[k], vT, vk * (s.fcp[k] - esh)), m.invWf[k], dcb);
  }
  {
    float t2[2] = {dSh, dcb};
    sum_many<G, 2>(g, t2);
    dSh = t2[0];
    dcb = t2[1];
  }
  if (g.lane == 0) out[ns] = (double)((-(vT * Sh + T * dSh) + T * Sh * (drr + dcb * invcb)) * (invrho * invcb));
  g.sync();
}

// A small nonzero integer held as a double, as a float, with integer
// operations only (sign, exponent rebased from 1023 to 127, the top 20
// significand bits of the high word): exact for |n| < 2^21.
__device__ __forceinline__ float small_int_to_float(double x) {
  const int hi = __double2hiint(x);
  return __int_as_float((hi & (int)0x80000000) | ((((hi >> 20) & 0x7ff) - 896) << 23) | ((hi & 0xfffff) << 3));
}

// The analytic J v of jvp_eval in FP32 arithmetic (precision level 6): the
// caching right-hand side at u_n left FP32 copies of the per-reaction k, k/Kc,
// dq/dT and of the per-species factors in the spare storage of the FP64 J v
// caches, and the intermediates -- dC, dq and the gather's partial sums -- are
// kept as FP32 in the first half of the FP64 arrays' own storage, so the slot
// layout, the mechanism copy and the occupancy are the FP64 kernel's and the
// product issues almost no FP64 instruction.  FP32's ~1e-7 rounding (amplified
// where k Pf and k/Kc Pb nearly cancel) is what the Krylov basis sees; the
// stages, the error estimate and the state update stay FP64.
template <int G>
__device__ __forceinline__ void jvp_eval_f32x(const MechView& m, const SlotPtrs& s, const double* uu,
                                              const CellScalars& cs, const double* v, double* out) {
  const Grp<G> g;
  const int ns = m.ns;
  float* fdC = reinterpret_cast<float*>(s.dC);
  float* fq = reinterpret_cast<float*>(s.q);
  float* fpart = reinterpret_cast<float*>(s.part);
  auto f = [](double x) { return __double2float_rn(x); };
  const float vT = f(v[ns]);
  const float T = f(cs.T), invT = f(cs.invT);
  float a = 0.f;
  for (int k = g.lane; k < ns; k += G) a = fmaf(f(v[k]), f(m.invW[k]), a);
  a = g.sum(a);
  const float drr = cs.cv ? 0.f : -fmaf(a, f(cs.invS), vT * invT);
  const bool coop_tb = m.ntb > 0 && m.ntb <= MAXM;
  float mp[MAXM];
#pragma unroll
  for (int t = 0; t < MAXM; ++t) mp[t] = 0.f;
  for (int k = g.lane; k < ns; k += G) {
    const float dCk = fmaf(s.xC[k], drr, s.xE[k] * f(v[k]));  // xE: rho / W_k
    fdC[k] = dCk;
    if (coop_tb) {
#pragma unroll
      for (int t = 0; t < MAXM; ++t)
        if (t < m.ntb) mp[t] = fmaf(f(m.eff[t * ns + k]), dCk, mp[t]);
    }
  }
  if (g.lane == 0) fdC[ns] = 0.f;  // the empty reaction slot (its C = 1 is in xC)
  if (coop_tb) sum_first<G>(g, mp, m.ntb);
  g.sync();
  for (int j = g.lane; j < m.nr; j += G) {
    const uint32_t sl = m.slots[j];
    const int ra = sl & 255, rb = (sl >> 8) & 255, pa = (sl >> 16) & 255, pb = sl >> 24;
    const int meta = m.meta[j];
    const int kind = meta & 3;
    const float Cra = s.xC[ra], Crb = s.xC[rb], Cpa = s.xC[pa], Cpb = s.xC[pb];
    const float dPf = fmaf(fdC[ra], Crb, Cra * fdC[rb]);
    const float dPb = fmaf(fdC[pa], Cpb, Cpa * fdC[pb]);
    const float k = s.xk[j], kr = s.xkr[j];
    float dq = fmaf(s.xqT[j], vT, fmaf(k, dPf, -kr * dPb));
    if (kind != 0) {
      const int slot = meta >> 8;
      const double* t = s.tb + 4 * slot;
      const float Pf = Cra * Crb, Pb = Cpa * Cpb;
      float dM = 0.f;
      if (coop_tb) {
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q == slot) dM = mp[q];
      } else {
        const double* e = m.eff + (size_t)slot * ns;
        for (int q = 0; q < ns; ++q) dM = fmaf(f(e[q]), fdC[q], dM);
      }
      if (kind == 1) dq = f(t[0]) * dq + dM * (k * Pf - kr * Pb);
      else dq = dq + f(t[1]) * dM * (Pf - f(t[3]) * Pb);
    }
    fq[j] = dq;
  }
  g.sync();
  for (int p = g.lane; p < m.npiece; p += G) {  // d w = nu^T dq
    float acc = 0.f;
    const int e1 = m.piece_ptr[p + 1];
    for (int e = m.piece_ptr[p]; e < e1; ++e) acc = fmaf(small_int_to_float(m.csr_nu[e]), fq[m.csr_j[e]], acc);
    fpart[p] = acc;
  }
  g.sync();
  float dSh = 0.f, dcb = 0.f;
  for (int k = g.lane; k < ns; k += G) {
    const float dom = piece_sum(m, static_cast<const float*>(fpart), k);
    out[k] = (double)(s.xEinv[k] * fmaf(-s.xom[k], drr, dom));  // xEinv: W_k / rho
    dSh = fmaf(s.xg[k], dom, fmaf(s.xh[k], vT, dSh));
    dcb = fmaf(s.xdcp[k], vT, fmaf(s.xcp[k], f(v[k]), dcb));
  }
  {
    float t2[2] = {dSh, dcb};
    sum_many<G, 2>(g, t2);
    dSh = t2[0];
    dcb = t2[1];
  }
  if (g.lane == 0) {
    const float Sh = f(cs.Sh);
    out[ns] = (double)((-(vT * Sh + T * dSh) + T * Sh * (drr + dcb * f(cs.invcb))) * (f(cs.invrho) * f(cs.invcb)));
  }
  g.sync();
}

// ----------------------------------------------------------------- helpers
template <int G>
__device__ inline double group_dot(const Grp<G>& g, const double* a, const double* b, int N) {
  double acc = 0.0;
  for (int e = g.lane; e < N; e += G) acc = fma(a[e], b[e], acc);
  return g.sum(acc);
}

// J v into out: analytic, or forward difference with the oracle's increment.
template <int G, bool MIXED = false, bool TC = false>
__device__ inline void apply_jv(const MechView& m, const SlotPtrs& s, const CellScalars& cs, int jv_mode,
                                double p, double unorm, const double* v, double* out, int* n_rhs,
                                bool fp32_jv = false) {
  const Grp<G> g;
  const int N = m.ns + 1 + m.nx;
  if (jv_mode == 0) {
    if (MIXED && fp32_jv) jvp_eval_f32<G>(m, s, s.u, cs, v, out);
    else if (!MIXED && cs.prec == 3) jvp_eval_df<G>(m, s, s.u, cs, v, out);
    else if (!MIXED && cs.prec == 6) jvp_eval_f32x<G>(m, s, s.u, cs, v, out);
    else jvp_eval<G, MIXED, TC>(m, s, s.u, cs, v, out);
    return;
  }
  const double nv = sqrt(group_dot<G>(g, v, v, N));
  if (nv == 0.0) {
    for (int e = g.lane; e < N; e += G) out[e] = 0.0;
    g.sync();
    return;
  }
  const double d = sqrt(2.220446049250313e-16) * (1.0 + unorm) / nv;
  for (int e = g.lane; e < N; e += G) s.arg[e] = s.u[e] + d * v[e];
  g.sync();
  CellScalars dummy;
  dummy.pinv = cs.pinv;
  dummy.prec = cs.prec;
  rhs_eval_call<G, MIXED, TC>(m, s, s.arg, s.src, p, out, false, &dummy);
  *n_rhs += 1;
  for (int e = g.lane; e < N; e += G) out[e] = (out[e] - s.fn[e]) / d;
  g.sync();
}

template <int G>
__device__ inline float group_dot_f(const Grp<G>& g, const double* a, const double* b, int N) {
  float acc = 0.f;
  for (int e = g.lane; e < N; e += G) acc = fmaf(__double2float_rn(a[e]), __double2float_rn(b[e]), acc);
  return g.sum(acc);
}

// Arnoldi with classical Gram-Schmidt and one reorthogonalisation pass on
// K_M(J_n, f_n) (Sec. 4.1).  Returns the dimension m <= M; Q and H in the slot.
// MIXED: the first Gram-Schmidt pass takes its inner products in FP32 (from
// the FP32 copy of Q); the reorthogonalisation pass, which removes what the
// first pass left behind -- its FP32 rounding included -- and the norms stay
// FP64, so the basis and H keep FP64 quality (mixed-precision "twice is
// enough").
//
// One FP64 Gram-Schmidt pass of w against the basis vectors q_0..q_{n-1}:
// h = Q^T w (one batched reduction), w <- w - Q h, and hcol += h.  J > 0: n = J
// is known at compile time, so no term carries a predicate (a predicated-off
// FP64 instruction still takes its issue and pipe slot); J = 0: n = jn at run
// time guards each of the MAXM terms.  Either way the same operations in the
// same order for the terms that exist.
template <int G, int J>
__device__ __forceinline__ void cgs_pass(const SlotPtrs& s, int N, int jn, double (&hcol)[MAXM]) {
  const Grp<G> g;
  const int Nq = s.Nq;
  constexpr int LJ = J > 0 ? J : MAXM;
  double hp[MAXM];
#pragma unroll
  for (int i = 0; i < MAXM; ++i) hp[i] = 0.0;
#pragma unroll 1
  for (int e = g.lane; e < N; e += G) {
    const double we = s.w[e];
#pragma unroll
    for (int i = 0; i < LJ; ++i)
      if (J > 0 || i < jn) hp[i] = fma(s.Q[i * Nq + e], we, hp[i]);
  }
  sum_first<G>(g, hp, J > 0 ? J : jn);
#pragma unroll 1
  for (int e = g.lane; e < N; e += G) {
    double we = s.w[e];
#pragma unroll
    for (int i = 0; i < LJ; ++i)
      if (J > 0 || i < jn) we = fma(-hp[i], s.Q[i * Nq + e], we);
    s.w[e] = we;
  }
#pragma unroll
  for (int i = 0; i < LJ; ++i)
    if (J > 0 || i < jn) hcol[i] += hp[i];
}

template <int G, bool MIXED = false, bool TC = false>
__device__ int arnoldi(const MechView& m, const SlotPtrs& s, const CellScalars& cs, int M, int jv_mode,
                       double p, int* n_rhs, bool fp32_jv = false) {
  const Grp<G> g;
  const int N = m.ns + 1 + m.nx;
  const int Nq = s.Nq;
  if (M > N) M = N;
  for (int i = g.lane; i < M * MAXM; i += G) s.H[i] = 0.0;
  // squared norms; 1/||.|| from one reciprocal square root
  const double beta2 = group_dot<G>(g, s.fn, s.fn, N);
  if (M <= 0 || !(beta2 > 0.0) || !isfinite(beta2)) {
    g.sync();
    return 0;
  }
  double unorm = 0.0;
  if (jv_mode != 0) unorm = sqrt(group_dot<G>(g, s.u, s.u, N));
  const double ibeta = rsqrt(beta2);
  for (int e = g.lane; e < N; e += G) {
    const double qe = s.fn[e] * ibeta;
    s.Q[e] = qe;
    if (MIXED) s.fQ[e] = __double2float_rn(qe);
  }
  g.sync();
  constexpr double brk2 = BREAKDOWN_TOL * BREAKDOWN_TOL;  // breakdown ||w_after|| <= tol ||w_before||, on squares
  int mdim = M;
  for (int j = 0; j < M; ++j) {
    apply_jv<G, MIXED, TC>(m, s, cs, jv_mode, p, unorm, s.Q + j * Nq, s.w, n_rhs, fp32_jv);
    // (only the breakdown threshold reads ||J q_j||^2: FP32 is enough there)
    const double w02 = MIXED ? (double)group_dot_f<G>(g, s.w, s.w, N) : group_dot<G>(g, s.w, s.w, N);
    double hcol[MAXM];
#pragma unroll
    for (int i = 0; i < MAXM; ++i) hcol[i] = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      if (MIXED && pass == 0) {
        double hp[MAXM];
        float part[MAXM];
#pragma unroll
        for (int i = 0; i < MAXM; ++i) part[i] = 0.f;
        for (int e = g.lane; e < N; e += G) {
          const float we = __double2float_rn(s.w[e]);
#pragma unroll
          for (int i = 0; i < MAXM; ++i)
            if (i <= j) part[i] = fmaf(s.fQ[i * Nq + e], we, part[i]);
        }
        sum_first<G>(g, part, j + 1);
#pragma unroll
        for (int i = 0; i < MAXM; ++i) hp[i] = (double)part[i];
        for (int e = g.lane; e < N; e += G) {
          double we = s.w[e];
#pragma unroll
          for (int i = 0; i < MAXM; ++i)
            if (i <= j) we = fma(-hp[i], s.Q[i * Nq + e], we);
          s.w[e] = we;
        }
#pragma unroll
        for (int i = 0; i < MAXM; ++i) hcol[i] += hp[i];
      } else if (M <= 4) {  // the common Krylov dimensions: column j + 1 known at compile time
        switch (j) {
          case 0: cgs_pass<G, 1>(s, N, 1, hcol); break;
          case 1: cgs_pass<G, 2>(s, N, 2, hcol); break;
          case 2: cgs_pass<G, 3>(s, N, 3, hcol); break;
          default: cgs_pass<G, 4>(s, N, 4, hcol); break;
        }
      } else {
        cgs_pass<G, 0>(s, N, j + 1, hcol);
      }
    }
    const double hn2 = group_dot<G>(g, s.w, s.w, N);
    if (g.lane == 0) {
#pragma unroll
      for (int i = 0; i < MAXM; ++i)
        if (i <= j) s.H[i * MAXM + j] = hcol[i];
    }
    if (j + 1 == M) break;
    if (hn2 <= brk2 * w02 || hn2 == 0.0) {
      mdim = j + 1;
      break;
    }
    const double ihn = rsqrt(hn2);
    const double hn = hn2 * ihn;
    if (g.lane == 0) s.H[(j + 1) * MAXM + j] = hn;
    for (int e = g.lane; e < N; e += G) {
      const double qe = s.w[e] * ihn;
      s.Q[(j + 1) * Nq + e] = qe;
      if (MIXED) s.fQ[(j + 1) * Nq + e] = __double2float_rn(qe);
    }
    g.sync();
  }
  g.sync();
  return mdim;
}

// Solve (I - h gamma H) y = z in place (every lane, redundantly; the factor
// stores reciprocal pivots, so the solve has no divisions).
__device__ inline void solve_small(const SlotPtrs& s, int mdim, double* z) {
  for (int c = 0; c < mdim; ++c) {
    const int pr = (int)s.piv[c];
    if (pr != c) {
      const double t = z[c];
      z[c] = z[pr];
      z[pr] = t;
    }
  }
  for (int r = 1; r < mdim; ++r)
    for (int c = 0; c < r; ++c) z[r] = fma(-s.LU[r * MAXM + c], z[c], z[r]);
  for (int r = mdim - 1; r >= 0; --r) {
    for (int c = r + 1; c < mdim; ++c) z[r] = fma(-s.LU[r * MAXM + c], z[c], z[r]);
    z[r] = z[r] * s.LU[r * MAXM + r];
  }
}

// LU factorisation with partial pivoting of I - h gamma H (m x m), by lane 0.
template <int G>
__device__ inline void factor_small(const SlotPtrs& s, int mdim, double h) {
  const Grp<G> g;
  if (g.lane == 0) {
    double* A = s.LU;
    const double hg = h * GAM;
    for (int i = 0; i < mdim; ++i)
      for (int j = 0; j < mdim; ++j) A[i * MAXM + j] = fma(-hg, s.H[i * MAXM + j], i == j ? 1.0 : 0.0);
    for (int c = 0; c < mdim; ++c) {
      // partial pivoting; |a| compared through its bit pattern (the order of
      // non-negative doubles is the order of their bits), an integer compare
      int pr = c;
      long long best = __double_as_longlong(fabs(A[c * MAXM + c]));
      for (int r = c + 1; r < mdim; ++r) {
        const long long cand = __double_as_longlong(fabs(A[r * MAXM + c]));
        if (cand > best) {
          best = cand;
          pr = r;
        }
      }
      s.piv[c] = (double)pr;
      if (pr != c)
        for (int j = 0; j < mdim; ++j) {
          const double t = A[c * MAXM + j];
          A[c * MAXM + j] = A[pr * MAXM + j];
          A[pr * MAXM + j] = t;
        }
      const double inv = rcp_any(A[c * MAXM + c]);
      for (int r = c + 1; r < mdim; ++r) {
        const double l = A[r * MAXM + c] * inv;
        A[r * MAXM + c] = l;
        for (int j = c + 1; j < mdim; ++j) A[r * MAXM + j] = fma(-l, A[c * MAXM + j], A[r * MAXM + j]);
      }
      A[c * MAXM + c] = inv;  // the diagonal is kept as its reciprocal
    }
  }
  g.sync();
  // B = I - (I - h gamma H)^-1, one column per lane (a solve with e_l), so each
  // stage applies the low-rank correction as one matrix-vector product
  if (g.lane < mdim) {
    double x[MAXM];
#pragma unroll
    for (int i = 0; i < MAXM; ++i) x[i] = i == g.lane ? 1.0 : 0.0;
    solve_small(s, mdim, x);
    for (int i = 0; i < mdim; ++i) s.Bm[i * MAXM + g.lane] = (i == g.lane ? 1.0 : 0.0) - x[i];
  }
  g.sync();
}

// One stage of the transformed form (Eq. s_stage_row_transformed) with the
// low-rank inverse (Eq. solve_kry_jac), in two parts.  stage_rhs: F_i = f_i +
// G_i with G_i = sum_{j<i} (gamma_ij / gamma) k_j (F_i and G_i left in s.F and
// s.w) and the partial sums of Q^T F_i.  stage_solve: c = (I - (I - h gamma
// H)^-1) Q^T F_i (B = I - (I - h gamma H)^-1 from factor_small) and
// k_i = F_i - Q c - G_i.  I >= 0: the stage known at compile time; MD > 0: the
// basis dimension known at compile time, so no term carries a predicate (a
// predicated-off FP64 instruction still takes its issue and pipe slot);
// I = -1 / MD = 0: from i / mdim at run time, each of the MAXM terms guarded.
// The same operations in the same order either way.
template <int G, int MD, int I>
__device__ __forceinline__ void stage_rhs(const SlotPtrs& s, int N, int i_rt, int mdim_rt, const double* fi,
                                          double (&part)[MAXM]) {
  const Grp<G> g;
  const int Nq = s.Nq;
  const int i = I >= 0 ? I : i_rt;
  const int mdim = MD > 0 ? MD : mdim_rt;
  constexpr int LM = MD > 0 ? MD : MAXM;
  constexpr double g21 = G21 / GAM, g31 = G31 / GAM, g32 = G32 / GAM;
  constexpr double g41 = G41 / GAM, g42 = G42 / GAM, g43 = G43 / GAM;
  const double* K0 = s.K;
  const double* K1 = s.K + Nq;
  const double* K2 = s.K + 2 * Nq;
#pragma unroll
  for (int l = 0; l < MAXM; ++l) part[l] = 0.0;
#pragma unroll 1
  for (int e = g.lane; e < N; e += G) {
    double Ge = 0.0;
    if (i == 1) Ge = g21 * K0[e];
    else if (i == 2) Ge = fma(g32, K1[e], g31 * K0[e]);
    else if (i == 3) Ge = fma(g43, K2[e], fma(g42, K1[e], g41 * K0[e]));
    const double Fe = fi[e] + Ge;
    s.F[e] = Fe;
    s.w[e] = Ge;
#pragma unroll
    for (int l = 0; l < LM; ++l)
      if (MD > 0 || l < mdim) part[l] = fma(s.Q[l * Nq + e], Fe, part[l]);
  }
}

template <int G, int MD>
__device__ __forceinline__ void stage_solve(const SlotPtrs& s, int N, int i, int mdim_rt, double (&part)[MAXM]) {
  const Grp<G> g;
  const int Nq = s.Nq;
  const int mdim = MD > 0 ? MD : mdim_rt;
  constexpr int LM = MD > 0 ? MD : MAXM;
  double* Ki = s.K + i * Nq;
  if (mdim > 0) sum_first<G>(g, part, mdim);
  // lane l < m forms c_l, every lane then reads all
  double cl = 0.0;
  if (g.lane < mdim) {
#pragma unroll
    for (int c = 0; c < LM; ++c)
      if (MD > 0 || c < mdim) cl = fma(s.Bm[g.lane * MAXM + c], part[c], cl);
  }
  double cz[MAXM];
#pragma unroll
  for (int l = 0; l < LM; ++l) cz[l] = __shfl_sync(g.mask, cl, l, G);
#pragma unroll 1
  for (int e = g.lane; e < N; e += G) {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < LM; ++l)
      if (MD > 0 || l < mdim) acc = fma(s.Q[l * Nq + e], cz[l], acc);
    Ki[e] = (s.F[e] - acc) - s.w[e];
  }
  g.sync();
}


// ------------------------------------------------ cost-ordered work queue
// Cells are handed out longest-expected-first: the expected substep count of
// a cell is dt / h with h its carried step (h_cell), binned on a quarter-octave
// log scale; a counting sort (per-block histograms reserved in one atomic per
// bin, then scattered) writes the queue order.  Cells with no carried step or
// h >= dt land in the cheapest bin.
constexpr int ORDER_BINS = 64;
constexpr int ORDER_THREADS = 256;

__device__ __forceinline__ int cost_bin(double h, double dt) {
  if (!(h > 0.0) || !(h < dt)) return 0;
  const float r = __double2float_rn(dt) / __double2float_rn(h);
  const int b = (int)(4.0f * __log2f(r));
  return b < 0 ? 0 : (b >= ORDER_BINS ? ORDER_BINS - 1 : b);
}

// ------------------------------------------------------- integration kernel
struct IntegrateParams {
  const unsigned char* mech;  // packed mechanism (global)
  MechLayout L;
  SlotLayout S;
  double* Y;
  const double* src;
  double* h_cell;
  int64_t ncell;
  double p, dt, rtol, atol, h0, fixed_h;
  int M, jv_mode, max_attempts, trace_cap, precision;
  double* trace;
  int32_t* stats;
  unsigned long long* counter;
  unsigned long long qstride;  // queue position q takes cell (q * qstride) mod ncell
  const int32_t* order;        // or, when set, cell order[q] (longest expected first)
  int subq;                    // > 0: static bins, subq sub-queues per block (queue order 3)
  const unsigned* nhot;        // with static bins: number of hot cells leading the order, or null
  const double* rho_cell;      // constant-volume densities, or null (constant pressure)
  int nx;                      // state components after T (5: auxiliary-temperature system)
  int64_t mech_copy;           // bytes of the mechanism each block copies (a prefix, by precision)
  int64_t tc_bytes;            // precision 4: bytes of nu^T tiles copied after that prefix (else 0)
};

template <int G, bool MIXED, bool TC = false>
__device__ void integrate_cell(const MechView& m, const SlotPtrs& s, const IntegrateParams& P, int64_t cell) {
  const Grp<G> g;
  const int ns = m.ns, N = ns + 1 + m.nx, Nq = s.Nq;
  for (int e = g.lane; e < N; e += G) {
    s.u[e] = P.Y[cell * N + e];
    s.src[e] = P.src ? P.src[cell * N + e] : 0.0;
  }
  g.sync();
  const double* srcp = P.src ? s.src : nullptr;
  const bool fixed = P.fixed_h > 0.0;
  const double pr = P.rho_cell ? -P.rho_cell[cell] : P.p;  // negative: constant-volume density
  const bool fp32_jv = P.precision == 2;
  const double dt = P.dt;
  double h = P.h0 > 0.0 ? P.h0 : dt;
  if (P.h_cell) {
    const double hc = P.h_cell[cell];
    if (hc > 0.0) h = hc;
  }
  if (fixed) h = P.fixed_h;
  const long long n_fixed = fixed ? llround(dt / P.fixed_h) : 0;
  double t = 0.0, h_last = h;
  float lg_err_prev = 0.f;  // log2 err_n; err_n = 1 before the first step
  int n_acc = 0, n_rej = 0, n_rhs = 0, status = RK_CELL_OK, n_att = 0;
  CellScalars cs;
  cs.pinv = 1.0 / fabs(pr);
  cs.prec = (P.precision == 3 || P.precision >= 5) ? P.precision : (TC ? 4 : 0);
  constexpr bool INL = G == 32 && !MIXED;  // the RHS inlined on the main path
  int mdim = 0;
  bool fresh = true;  // f_n and the Krylov basis are due at u (start, or after an accepted step)
  double* K0 = s.K;
  double* K1 = s.K + Nq;
  double* K2 = s.K + 2 * Nq;
  double* K3 = s.K + 3 * Nq;
  while (true) {
    if (fresh) {
      rhs_dispatch<G, MIXED, INL, TC>(m, s, s.u, srcp, pr, s.fn, true, &cs);
      n_rhs += 1;
      mdim = arnoldi<G, MIXED, TC>(m, s, cs, P.M, P.jv_mode, pr, &n_rhs, fp32_jv);
      fresh = false;
    }
    if (fixed) {
      if (n_acc >= n_fixed) break;
    } else if (dt - t <= T_END_TOL * dt) {
      break;
    }
    if (n_att >= P.max_attempts) {
      status = RK_CELL_MAX_ATTEMPTS;
      break;
    }
    if (!fixed) h = fmin(h, dt - t);
    factor_small<G>(s, mdim, h);
    // ---- four stages (Algorithm 1); f is evaluated at stages 2 and 3 only
    for (int i = 0; i < 4; ++i) {
      const double* fi;
      if (i == 0) {
        fi = s.fn;
      } else if (i == 1 || i == 2) {
        for (int e = g.lane; e < N; e += G) {
          const double acc = (i == 1) ? A21 * K0[e] : fma(A32, K1[e], A31 * K0[e]);
          s.arg[e] = s.u[e] + h * acc;
        }
        g.sync();
        rhs_dispatch<G, MIXED, INL, TC>(m, s, s.arg, srcp, pr, s.fr, false, &cs);
        n_rhs += 1;
        fi = s.fr;
      } else {
        fi = s.fr;  // alpha_4j = alpha_3j: same argument as stage 3
      }
      double part[MAXM];
      if (mdim == 4) {  // the common Krylov dimension: stage and dimension known at compile time
        switch (i) {
          case 0: stage_rhs<G, 4, 0>(s, N, 0, 4, fi, part); break;
          case 1: stage_rhs<G, 4, 1>(s, N, 1, 4, fi, part); break;
          case 2: stage_rhs<G, 4, 2>(s, N, 2, 4, fi, part); break;
          default: stage_rhs<G, 4, 3>(s, N, 3, 4, fi, part); break;
        }
        stage_solve<G, 4>(s, N, i, 4, part);
      } else {
        stage_rhs<G, 0, -1>(s, N, i, mdim, fi, part);
        stage_solve<G, 0>(s, N, i, mdim, part);
      }
    }
    // ---- solutions, error estimate
    double part = 0.0;
    int bad = 0;
    for (int e = g.lane; e < N; e += G) {
      const double k0 = K0[e], k1 = K1[e], k2 = K2[e], k3 = K3[e];
      const double ue = s.u[e];
      const double us = ue + h * fma(B4, k3, fma(B3, k2, fma(B2, k1, B1 * k0)));
      const double uh = ue + h * fma(BH4, k3, fma(BH3, k2, fma(BH2, k1, BH1 * k0)));
      const double d = (uh - us) * rcp_any(fma(P.rtol, fabs(us), P.atol));
      part = fma(d, d, part);
      bad |= (__double2hiint(us) & 0x7ff00000) == 0x7ff00000;
      s.arg[e] = us;
    }
    const double err = sqrt(g.sum(part) * (1.0 / N));
    bad = g.any(bad);
    const int att = n_att;
    n_att += 1;
    bool accept;
    double hnew;
    float lg_err = 0.f;
    if (fixed) {
      accept = true;
      hnew = h;
    } else {
      // h* = h min(5, max(0.2, 0.8 err_n^beta / err*^alpha)), the factor in
      // FP32 as 2^(beta log2 err_n - alpha log2 err*) (log2 err_n kept from
      // acceptance); the accept test err <= 1 stays FP64
      const bool fin = (__double2hiint(err) & 0x7ff00000) != 0x7ff00000;
      float fac = (float)FAC_MIN;
      if (fin) {
        lg_err = __log2f(fmaxf(__double2float_rn(err), (float)ERR_FLOOR));
        fac = fminf((float)FAC_MAX,
                    fmaxf((float)FAC_MIN, (float)SAFETY * exp2f((float)PI_BETA * lg_err_prev - (float)PI_ALPHA * lg_err)));
      }
      hnew = h * (double)fac;
      accept = fin && err <= 1.0;
    }
    if (P.trace && att < P.trace_cap && g.lane == 0) P.trace[cell * P.trace_cap + att] = accept ? h : -h;
    if (accept) {
      if (bad) {
        status = RK_CELL_NONFINITE;
        break;
      }
      for (int e = g.lane; e < N; e += G) s.u[e] = s.arg[e];
      g.sync();
      t += h;
      if (!fixed) lg_err_prev = lg_err;
      n_acc += 1;
      h_last = hnew;
      h = hnew;
      const bool done = fixed ? (n_acc >= n_fixed) : (dt - t <= T_END_TOL * dt);
      fresh = !done;
    } else {
      n_rej += 1;
      h = hnew;
      if (h < H_MIN_FRAC * dt) {
        status = RK_CELL_STEP_UNDERFLOW;
        break;
      }
    }
  }
  for (int e = g.lane; e < N; e += G) P.Y[cell * N + e] = s.u[e];
  if (g.lane == 0) {
    if (P.h_cell) P.h_cell[cell] = h_last;
    if (P.stats) {
      P.stats[4 * cell + 0] = n_acc;
      P.stats[4 * cell + 1] = n_rej;
      P.stats[4 * cell + 2] = n_rhs;
      P.stats[4 * cell + 3] = status;
    }
  }
  g.sync();
}

// Copy the packed mechanism into shared memory (16-byte vector copies).
__device__ inline void load_mech(unsigned char* dst, const unsigned char* src, int64_t bytes) {
  const int64_t n16 = bytes / 16;
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) d4[i] = s4[i];
}

template <bool MIXED = false>
__device__ inline void init_sentinels(const SlotPtrs& s, int ns, int lane) {
  if (lane == 0) {
    s.C[ns] = 1.0;
    s.dC[ns] = 0.0;
    if (s.C2) {
      s.C2[ns] = {1.0f, 0.0f};
      s.dC2[ns] = {0.0f, 0.0f};
    }
    s.hRT[ns] = 0.0;
    s.gRT[ns] = 0.0;
    s.E[ns] = 1.0;
    s.Einv[ns] = 1.0;
    s.CE[ns] = 1.0;
    if (MIXED) {
      s.fC[ns] = 1.f;
      s.fdC[ns] = 0.f;
      s.fh[ns] = 0.f;
    }
  }
}

// Hand cells to the warp groups of a persistent launch until the queue is
// empty, calling body(cell) for each.
template <int G, class Body>
__device__ __forceinline__ void drain_queue(const IntegrateParams& P, const Grp<G>& g, int gid, Body&& body) {
  if (P.subq > 0) {
    // Static bins: the queue (longest expected first) is dealt out in snake
    // order over nb = gridDim.x * subq bins, bin k = sub * gridDim.x + block,
    // so every block -- and within a block every group of warps sharing a
    // sub-queue -- receives a near-equal share of the expensive cells.  Round
    // r of bin k holds queue position r * nb + (r even ? k : nb - 1 - k).
    __shared__ unsigned sub_ctr[4];
    if (threadIdx.x < 4) sub_ctr[threadIdx.x] = 0u;
    __syncthreads();
    // The H hot cells that lead the order (when they are few: at most half the
    // blocks and an eighth of the cells) each get a block -- an SM -- of their
    // own: hot cell b runs on sub-queue 0 of block b and that block takes
    // nothing else, so no other cell shares its SM's FP64 units, shared-memory
    // pipe or instruction cache.  The rest are dealt in snake order over the
    // bins of the other blocks.
    const int sub = gid % P.subq;
    const unsigned long long nblk = gridDim.x;
    unsigned long long H = P.nhot ? (unsigned long long)P.nhot[0] : 0ull;
    if (H * 2ull > nblk || H * 8ull > (unsigned long long)P.ncell) H = 0ull;
    if (H > 0ull) {
      // only while the other cells, spread over the other blocks' four
      // sub-partitions, still finish within the hottest cell's expected time
      const float top_cost = __uint_as_float(P.nhot[1]), rest_cost = __uint_as_float(P.nhot[2]);
      if (rest_cost > top_cost * 4.0f * (float)(nblk - H)) H = 0ull;
    }
    const unsigned long long nb = (nblk - H) * (unsigned long long)P.subq;
    const bool hot_block = blockIdx.x < H;
    const unsigned long long k = hot_block ? 0ull : (unsigned long long)sub * (nblk - H) + (blockIdx.x - H);
    while (true) {
      unsigned r = 0u;
      if (g.lane == 0) r = atomicAdd(&sub_ctr[sub], 1u);
      r = __shfl_sync(g.mask, r, 0, G);
      unsigned long long q;
      if (hot_block) {
        q = (sub == 0 && r == 0u) ? (unsigned long long)blockIdx.x : (unsigned long long)P.ncell;
      } else {
        q = H + (unsigned long long)r * nb + ((r & 1u) ? nb - 1ull - k : k);
      }
      if (q >= (unsigned long long)P.ncell) break;
      const unsigned long long cell =
          P.order ? (unsigned long long)P.order[q] : (q * P.qstride) % (unsigned long long)P.ncell;
      body((int64_t)cell);
    }
    return;
  }
  while (true) {
    unsigned long long q = 0;
    if (g.lane == 0) q = atomicAdd(P.counter, 1ull);
    q = __shfl_sync(g.mask, q, 0, G);
    if (q >= (unsigned long long)P.ncell) break;
    // Interleave the queue over the cell index: neighbouring cells (e.g. the
    // hot side of a flame) spread over all SMs instead of filling a few.
    const unsigned long long cell =
        P.order ? (unsigned long long)P.order[q] : (q * P.qstride) % (unsigned long long)P.ncell;
    body((int64_t)cell);
  }
}

template <int G, bool MIXED, bool TC = false>
__global__ void __launch_bounds__(MAX_BLOCK_THREADS, 1) rok4e_integrate_kernel(IntegrateParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_exp_table(reinterpret_cast<double*>(smem));
  load_mech(smem + EXP_TAB_BYTES, P.mech, P.mech_copy);
  if (TC) load_mech(smem + EXP_TAB_BYTES + P.mech_copy, P.mech + P.L.off_nuT, P.tc_bytes);
  __syncthreads();
  MechView m = make_view(smem + EXP_TAB_BYTES, P.L);
  m.etab = reinterpret_cast<const double*>(smem);
  m.nx = P.nx;
  if (TC) m.nuT = reinterpret_cast<const uint4*>(smem + EXP_TAB_BYTES + P.mech_copy);
  const Grp<G> g;
  const int gid = threadIdx.x / G;
  double* base = reinterpret_cast<double*>(smem + EXP_TAB_BYTES + P.mech_copy + (TC ? P.tc_bytes : 0)) +
                 (size_t)gid * P.S.stride;
  const SlotPtrs s = slot_ptrs(base, P.S);
  init_sentinels<MIXED>(s, m.ns, g.lane);
  if (TC)  // digit rows: row 7 and the reaction padding stay zero
    for (int i = g.lane; i < 8 * 16 * m.nrt; i += G) s.dig[i] = 0;
  g.sync();
  drain_queue<G>(P, g, gid, [&](int64_t cell) { integrate_cell<G, MIXED, TC>(m, s, P, cell); });
}

// ------------------------------------------- explicit Dormand-Prince 5(4)
// The explicit reference integrator of the efficiency study (Sec. 4.4):
// seven stages, the 5th-order solution propagated, the embedded 4th-order
// one for the error (J. R. Dormand and P. J. Prince, J. Comput. Appl. Math.
// 6 (1980) 19-26), first-same-as-last; the same RMS error norm as ROK4E and
// the elementary controller h* = h min(5, max(0.2, 0.9 err^-1/5)).
namespace dp {
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 44.0 / 45.0, A42 = -56.0 / 15.0, A43 = 32.0 / 9.0;
constexpr double A51 = 19372.0 / 6561.0, A52 = -25360.0 / 2187.0, A53 = 64448.0 / 6561.0, A54 = -212.0 / 729.0;
constexpr double A61 = 9017.0 / 3168.0, A62 = -355.0 / 33.0, A63 = 46732.0 / 5247.0, A64 = 49.0 / 176.0,
                 A65 = -5103.0 / 18656.0;
constexpr double B1 = 35.0 / 384.0, B3 = 500.0 / 1113.0, B4 = 125.0 / 192.0, B5 = -2187.0 / 6784.0,
                 B6 = 11.0 / 84.0;
// b - bhat (b2 = bhat2 = 0, b7 = 0)
constexpr double E1 = 35.0 / 384.0 - 5179.0 / 57600.0, E3 = 500.0 / 1113.0 - 7571.0 / 16695.0,
                 E4 = 125.0 / 192.0 - 393.0 / 640.0, E5 = -2187.0 / 6784.0 + 92097.0 / 339200.0,
                 E6 = 11.0 / 84.0 - 187.0 / 2100.0, E7 = -1.0 / 40.0;
constexpr double SAFETY = 0.9;
}  // namespace dp

template <int G>
__device__ void integrate_cell_rkdp(const MechView& m, const SlotPtrs& s, const IntegrateParams& P, int64_t cell) {
  const Grp<G> g;
  const int ns = m.ns, N = ns + 1 + m.nx, Nq = s.Nq;
  for (int e = g.lane; e < N; e += G) {
    s.u[e] = P.Y[cell * N + e];
    s.src[e] = P.src ? P.src[cell * N + e] : 0.0;
  }
  g.sync();
  const double* srcp = P.src ? s.src : nullptr;
  const bool fixed = P.fixed_h > 0.0;
  const double pr = P.rho_cell ? -P.rho_cell[cell] : P.p;
  const double dt = P.dt;
  double h = P.h0 > 0.0 ? P.h0 : dt;
  if (P.h_cell) {
    const double hc = P.h_cell[cell];
    if (hc > 0.0) h = hc;
  }
  if (fixed) h = P.fixed_h;
  const long long n_fixed = fixed ? llround(dt / P.fixed_h) : 0;
  double t = 0.0, h_last = h;
  int n_acc = 0, n_rej = 0, n_rhs = 0, status = RK_CELL_OK, n_att = 0;
  CellScalars cs;
  cs.pinv = 1.0 / fabs(pr);
  cs.prec = 0;
  // stage vectors k1..k7; k1 and k7 swap roles after an accepted step
  double* k1 = s.fn;
  double* k2 = s.K;
  double* k3 = s.K + Nq;
  double* k4 = s.K + 2 * Nq;
  double* k5 = s.K + 3 * Nq;
  double* k6 = s.F;
  double* k7 = s.w;
  rhs_eval_call<G>(m, s, s.u, srcp, pr, k1, false, &cs);
  n_rhs += 1;
  while (true) {
    if (fixed) {
      if (n_acc >= n_fixed) break;
    } else if (dt - t <= T_END_TOL * dt) {
      break;
    }
    if (n_att >= P.max_attempts) {
      status = RK_CELL_MAX_ATTEMPTS;
      break;
    }
    if (!fixed) h = fmin(h, dt - t);
    for (int i = 1; i < 7; ++i) {
      for (int e = g.lane; e < N; e += G) {
        double acc;
        if (i == 1) acc = dp::A21 * k1[e];
        else if (i == 2) acc = fma(dp::A32, k2[e], dp::A31 * k1[e]);
        else if (i == 3) acc = fma(dp::A43, k3[e], fma(dp::A42, k2[e], dp::A41 * k1[e]));
        else if (i == 4) acc = fma(dp::A54, k4[e], fma(dp::A53, k3[e], fma(dp::A52, k2[e], dp::A51 * k1[e])));
        else if (i == 5)
          acc = fma(dp::A65, k5[e], fma(dp::A64, k4[e], fma(dp::A63, k3[e], fma(dp::A62, k2[e], dp::A61 * k1[e]))));
        else  // a_7j = b_j: the last argument is the 5th-order solution
          acc = fma(dp::B6, k6[e], fma(dp::B5, k5[e], fma(dp::B4, k4[e], fma(dp::B3, k3[e], dp::B1 * k1[e]))));
        s.arg[e] = fma(h, acc, s.u[e]);
      }
      g.sync();
      double* out = i == 1 ? k2 : i == 2 ? k3 : i == 3 ? k4 : i == 4 ? k5 : i == 5 ? k6 : k7;
      rhs_dispatch<G, false, G == 32>(m, s, s.arg, srcp, pr, out, false, &cs);
      n_rhs += 1;
    }
    double part = 0.0;
    int bad = 0;
    for (int e = g.lane; e < N; e += G) {
      const double us = s.arg[e];
      const double d = h * fma(dp::E7, k7[e], fma(dp::E6, k6[e], fma(dp::E5, k5[e], fma(dp::E4, k4[e],
                                                                                   fma(dp::E3, k3[e], dp::E1 * k1[e])))));
      const double r = d / fma(P.rtol, fabs(us), P.atol);
      part = fma(r, r, part);
      bad |= (__double2hiint(us) & 0x7ff00000) == 0x7ff00000;
    }
    const double err = sqrt(g.sum(part) * (1.0 / N));
    bad = g.any(bad);
    const int att = n_att;
    n_att += 1;
    bool accept;
    double hnew;
    if (fixed) {
      accept = true;
      hnew = h;
    } else {
      const bool fin = (__double2hiint(err) & 0x7ff00000) != 0x7ff00000;
      float fac = (float)FAC_MIN;  // FP32 factor, as in the ROK4E controller
      if (fin)
        fac = fminf((float)FAC_MAX, fmaxf((float)FAC_MIN, (float)dp::SAFETY *
                                                              exp2f(-0.2f * __log2f(fmaxf(__double2float_rn(err),
                                                                                          (float)ERR_FLOOR)))));
      hnew = h * (double)fac;
      accept = fin && err <= 1.0;
    }
    if (P.trace && att < P.trace_cap && g.lane == 0) P.trace[cell * P.trace_cap + att] = accept ? h : -h;
    if (accept) {
      if (bad) {
        status = RK_CELL_NONFINITE;
        break;
      }
      for (int e = g.lane; e < N; e += G) s.u[e] = s.arg[e];
      g.sync();
      double* tk = k1;  // first same as last: f(u_{n+1}) is k7
      k1 = k7;
      k7 = tk;
      t += h;
      n_acc += 1;
      h_last = hnew;
      h = hnew;
    } else {
      n_rej += 1;
      h = hnew;
      if (h < H_MIN_FRAC * dt) {
        status = RK_CELL_STEP_UNDERFLOW;
        break;
      }
    }
  }
  for (int e = g.lane; e < N; e += G) P.Y[cell * N + e] = s.u[e];
  if (g.lane == 0) {
    if (P.h_cell) P.h_cell[cell] = h_last;
    if (P.stats) {
      P.stats[4 * cell + 0] = n_acc;
      P.stats[4 * cell + 1] = n_rej;
      P.stats[4 * cell + 2] = n_rhs;
      P.stats[4 * cell + 3] = status;
    }
  }
  g.sync();
}

template <int G>
__global__ void __launch_bounds__(MAX_BLOCK_THREADS) rkdp_integrate_kernel(IntegrateParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_exp_table(reinterpret_cast<double*>(smem));
  load_mech(smem + EXP_TAB_BYTES, P.mech, P.mech_copy);
  __syncthreads();
  MechView m = make_view(smem + EXP_TAB_BYTES, P.L);
  m.etab = reinterpret_cast<const double*>(smem);
  m.nx = P.nx;
  const Grp<G> g;
  const int gid = threadIdx.x / G;
  double* base = reinterpret_cast<double*>(smem + EXP_TAB_BYTES + P.mech_copy) + (size_t)gid * P.S.stride;
  const SlotPtrs s = slot_ptrs(base, P.S);
  init_sentinels<false>(s, m.ns, g.lane);
  g.sync();
  drain_queue<G>(P, g, gid, [&](int64_t cell) { integrate_cell_rkdp<G>(m, s, P, cell); });
}

}  // namespace rk

#include "adjoint.cuh"

namespace rk {

// ------------------------------------------------------------ adjoint kernels
struct AdjointParams {
  const unsigned char* mech;
  MechLayout L;
  AdjLayout A;
  const double* ckpt;        // [(nsteps + 1) x ncell x N] states at the start of every step
  const double* ubar_final;  // [ncell x N] dL/du(t_end)
  double* grad_u0;           // [ncell x N] dL/du(0), or null
  double* wsd;
  Dual* wsD;
  int64_t ncell;
  double p, h;
  int nsteps, M;
};

// One group of G lanes per cell (see adjoint.cuh); 128-thread blocks, at most
// as many as are resident at once, the cells dealt to them in turn (cell c to
// block c mod gridDim.x) when there are more cells than slots.
template <int G>
__global__ void __launch_bounds__(128) rok4e_adjoint_kernel(AdjointParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_exp_table(reinterpret_cast<double*>(smem));
  load_mech(smem + EXP_TAB_BYTES, P.mech, P.L.off_nuT);
  __syncthreads();
  MechView m = make_view(smem + EXP_TAB_BYTES, P.L);
  m.etab = reinterpret_cast<const double*>(smem);
  const Grp<G> g;
  const int gpb = blockDim.x / G;
  const int64_t stride = (int64_t)gridDim.x * gpb;
  const int N = m.ns + 1;
  // whole groups take each cell, so a group's lanes agree on every branch
  for (int64_t c = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x / G); c < P.ncell; c += stride) {
    const AdjFrame F = adj_frame(P.wsd, P.wsD, P.A, c);
    for (int e = g.lane; e < N; e += G) F.ubar[e] = P.ubar_final[c * N + e];
    for (int j = g.lane; j < m.nr; j += G) F.theta[j] = 0.0;
    for (int n = P.nsteps - 1; n >= 0; --n) {
      const double* un = P.ckpt + ((int64_t)n * P.ncell + c) * N;
      for (int e = g.lane; e < N; e += G) F.u[e] = un[e];
      adj_step<G>(m, F, P.p, P.h, P.M, P.A.tape0, P.A.tape_len);
    }
    if (P.grad_u0)
      for (int e = g.lane; e < N; e += G) P.grad_u0[c * N + e] = F.ubar[e];
    g.sync();
  }
}

// One group per cell: f(u) + src, or J(u) v.
struct PointParams {
  const unsigned char* mech;
  MechLayout L;
  SlotLayout S;
  const double* Y;
  const double* src;
  const double* V;
  double* out;
  int64_t ncell;
  double p;
  int mode;  // 0 rhs, 1 analytic jvp, 2 finite-difference jvp, 3 mixed rhs, 4 FP32 analytic jvp,
             // 5 analytic jvp with the double-float core, 6 rhs with the tensor-core gather,
             // 7 analytic jvp with the tensor-core gather, 8 FP32 analytic jvp on the FP64 caches
  const double* rho_cell;  // constant-volume densities, or null
  int nx;                  // state components after T (5: auxiliary-temperature system)
  int64_t mech_copy;       // bytes of the mechanism copied to shared memory (a prefix)
  int64_t tc_bytes;        // modes 6 and 7: bytes of nu^T tiles copied after that prefix (else 0)
};

template <int G>
__global__ void __launch_bounds__(MAX_BLOCK_THREADS) chem_point_kernel(PointParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_exp_table(reinterpret_cast<double*>(smem));
  load_mech(smem + EXP_TAB_BYTES, P.mech, P.mech_copy);
  if (P.tc_bytes) load_mech(smem + EXP_TAB_BYTES + P.mech_copy, P.mech + P.L.off_nuT, P.tc_bytes);
  __syncthreads();
  MechView m = make_view(smem + EXP_TAB_BYTES, P.L);
  m.etab = reinterpret_cast<const double*>(smem);
  m.nx = P.nx;
  if (P.tc_bytes) m.nuT = reinterpret_cast<const uint4*>(smem + EXP_TAB_BYTES + P.mech_copy);
  const Grp<G> g;
  const int gid = threadIdx.x / G;
  const int gpb = blockDim.x / G;
  const int64_t cell = (int64_t)blockIdx.x * gpb + gid;
  if (cell >= P.ncell) return;
  double* base = reinterpret_cast<double*>(smem + EXP_TAB_BYTES + P.mech_copy + P.tc_bytes) + (size_t)gid * P.S.stride;
  const SlotPtrs s = slot_ptrs(base, P.S);
  if (P.mode >= 3 && P.mode <= 5) init_sentinels<true>(s, m.ns, g.lane);
  else init_sentinels<false>(s, m.ns, g.lane);
  if (P.mode == 6 || P.mode == 7)
    for (int i = g.lane; i < 8 * 16 * m.nrt; i += G) s.dig[i] = 0;
  const int N = m.ns + 1 + m.nx;
  for (int e = g.lane; e < N; e += G) {
    s.u[e] = P.Y[cell * N + e];
    s.src[e] = P.src ? P.src[cell * N + e] : 0.0;
    if (P.V) s.F[e] = P.V[cell * N + e];
  }
  g.sync();
  const double pr = P.rho_cell ? -P.rho_cell[cell] : P.p;
  CellScalars cs;
  cs.pinv = 1.0 / fabs(pr);
  cs.prec = 0;
  if (P.mode == 8) {
    cs.prec = 6;
    rhs_eval_call<G>(m, s, s.u, nullptr, pr, s.fn, true, &cs);
    jvp_eval_f32x<G>(m, s, s.u, cs, s.F, s.w);
    for (int e = g.lane; e < N; e += G) P.out[cell * N + e] = s.w[e];
    return;
  }
  if (P.mode == 7) {
    cs.prec = 4;
    rhs_eval_call<G, false, true>(m, s, s.u, nullptr, pr, s.fn, true, &cs);
    jvp_eval<G, false, true>(m, s, s.u, cs, s.F, s.w);
    for (int e = g.lane; e < N; e += G) P.out[cell * N + e] = s.w[e];
    return;
  }
  if (P.mode == 0 || P.mode == 3 || P.mode == 6) {
    if (P.mode == 3) rhs_eval_call<G, true>(m, s, s.u, P.src ? s.src : nullptr, pr, s.fr, false, &cs);
    else if (P.mode == 6) rhs_eval_call<G, false, true>(m, s, s.u, P.src ? s.src : nullptr, pr, s.fr, false, &cs);
    else rhs_eval_call<G>(m, s, s.u, P.src ? s.src : nullptr, pr, s.fr, false, &cs);
    for (int e = g.lane; e < N; e += G) P.out[cell * N + e] = s.fr[e];
    return;
  }
  if (P.mode == 4) {
    rhs_eval_call<G, true>(m, s, s.u, nullptr, pr, s.fn, true, &cs);
    jvp_eval_f32<G>(m, s, s.u, cs, s.F, s.w);
    for (int e = g.lane; e < N; e += G) P.out[cell * N + e] = s.w[e];
    return;
  }
  if (P.mode == 5) {
    cs.prec = 3;
    rhs_eval_call<G>(m, s, s.u, nullptr, pr, s.fn, true, &cs);
    jvp_eval_df<G>(m, s, s.u, cs, s.F, s.w);
    for (int e = g.lane; e < N; e += G) P.out[cell * N + e] = s.w[e];
    return;
  }
  // the auxiliary-temperature T row depends on the source; elsewhere s.src is
  // zero here, so the finite difference sees the bare source term
  rhs_eval_call<G>(m, s, s.u, m.nx > 0 ? s.src : nullptr, pr, s.fn, true, &cs);
  int n_rhs = 0;
  double unorm = 0.0;
  if (P.mode == 2) unorm = sqrt(group_dot<G>(g, s.u, s.u, N));
  apply_jv<G>(m, s, cs, P.mode == 1 ? 0 : 1, pr, unorm, s.F, s.w, &n_rhs);
  for (int e = g.lane; e < N; e += G) P.out[cell * N + e] = s.w[e];
}

}  // namespace rk

struct rk_mech {
  rk::HostMech host;
  unsigned char* dev = nullptr;
  int device = 0;
};

namespace rk {

struct LaunchPlan {
  int G = 32;
  int cells_per_block = 1;
  size_t smem = 0;
  int blocks = 1;
};

inline int device_props(int* n_sm, size_t* smem_optin) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  int v = 0;
  e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
  *n_sm = v;
  e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
  *smem_optin = (size_t)v;
  return RK_OK;
}

template <int G, typename K>
int plan_for(K kernel, const rk_mech* mech, const SlotLayout& S, int want_cells, int64_t ncell, bool persistent,
             LaunchPlan* plan, int want_blocks_per_sm = 0, bool fill_device = false, int64_t copy_bytes = -1) {
  int n_sm = 0;
  size_t smem_max = 0;
  int rc = device_props(&n_sm, &smem_max);
  if (rc) return rc;
  const size_t mech_bytes = (size_t)(copy_bytes >= 0 ? copy_bytes : mech->host.L.bytes) + EXP_TAB_BYTES;
  const size_t slot_bytes = (size_t)S.stride * sizeof(double);
  smem_max -= 64;  // the kernels' static shared memory (queue counters)
  if (mech_bytes + slot_bytes > smem_max)
    return set_error(RK_E_UNSUPPORTED, "mechanism plus one cell's work arrays exceed shared memory");
  int cells = (int)((smem_max - mech_bytes) / slot_bytes);
  cells = cells > MAX_BLOCK_THREADS / G ? MAX_BLOCK_THREADS / G : cells;
  if (want_cells > 0 && want_cells < cells) cells = want_cells;
  if (!persistent && (int64_t)cells > ncell) cells = (int)(ncell > 0 ? ncell : 1);
  size_t smem = mech_bytes + (size_t)cells * slot_bytes;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, cells * G, smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  while (per_sm == 0 && cells > 1) {  // registers limit: shrink the block
    cells /= 2;
    smem = mech_bytes + (size_t)cells * slot_bytes;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, cells * G, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  }
  if (per_sm == 0) return set_error(RK_E_UNSUPPORTED, "integration kernel cannot be resident on an SM");
  if (want_blocks_per_sm > 0 && want_blocks_per_sm < per_sm) per_sm = want_blocks_per_sm;
  plan->G = G;
  plan->cells_per_block = cells;
  plan->smem = smem;
  const int64_t need = (ncell + cells - 1) / cells;
  int64_t blocks = persistent ? (int64_t)per_sm * n_sm : need;
  if (persistent && blocks > need && !fill_device) blocks = need;
  plan->blocks = (int)(blocks > 0 ? blocks : 1);
  return RK_OK;
}

// Launches of the per-cell kernels.  Each instantiation is defined (and its
// kernel compiled) in one translation unit of its own, through launchers.cuh;
// the C ABI calls them through these declarations.
struct IntegrateLaunch {
  IntegrateParams* P;
  const rk_mech* mech;
  int cells_per_block, blocks_per_sm;
  bool static_bins;  // queue order 3: the block's static bins are dealt in sub-queues
  int64_t ncell;
  cudaStream_t stream;
};
template <int G, bool MIXED, bool TC>
int launch_rok4e(const IntegrateLaunch& a);
template <int G>
int launch_rkdp(const IntegrateLaunch& a);
template <int G>
int launch_adjoint(const AdjointParams& P, size_t smem, cudaStream_t st);

}  // namespace rk
