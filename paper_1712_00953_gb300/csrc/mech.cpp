// Host-side mechanism validation and packing (no CUDA).
//
// The checks enforce what the kernels rely on: species indices fit in 8 bits
// (with one value left for the "empty slot" sentinel), at most two molecules
// on each side of a reaction, integer element balance, positive molar masses
// and pre-exponential factors, valid Troe parameters and NASA-7 polynomials
// that are continuous at T_mid.  Packing converts A from cm-mol-s to SI units
// (m^3/mol per concentration order), divides out the polynomial coefficients
// the kernels use (see internal.h) and builds the species-major list of
// stoichiometric coefficients used for the deterministic gather w = nu^T q.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"
#include "rok4e.h"

namespace rk {
namespace {

constexpr double R_GAS = 8.314462618;

int64_t align16(int64_t x) { return (x + 15) & ~int64_t(15); }

bool fail(std::string* err, const char* fmt, int a = 0, int b = 0) {
  char buf[256];
  snprintf(buf, sizeof(buf), fmt, a, b);
  if (err) *err = buf;
  return false;
}

// cp/R, h/RT, s/R of one NASA-7 coefficient set at T (validation only)
void nasa_eval(const double* a, double T, double* cp, double* h, double* s) {
  *cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
  *h = a[0] + T * (a[1] / 2 + T * (a[2] / 3 + T * (a[3] / 4 + T * a[4] / 5))) + a[5] / T;
  *s = a[0] * log(T) + T * (a[1] + T * (a[2] / 2 + T * (a[3] / 3 + T * a[4] / 4))) + a[6];
}

bool close_rel(double x, double y, double tol) {
  return fabs(x - y) <= tol * std::max(1.0, std::max(fabs(x), fabs(y)));
}

}  // namespace

bool pack_mechanism(const void* vdesc, HostMech* out, std::string* err) {
  const rk_mech_desc* d = static_cast<const rk_mech_desc*>(vdesc);
  if (!d) return fail(err, "null mechanism description");
  const int ns = d->n_species, nr = d->n_reactions;
  if (ns < 1 || ns > RK_MAX_SPECIES) return fail(err, "n_species %d outside 1..%d", ns, RK_MAX_SPECIES);
  if (nr < 0 || nr > (1 << 20)) return fail(err, "n_reactions %d invalid", nr);
  if (!d->elem || !d->W || !d->nasa) return fail(err, "null species array");
  if (nr > 0 && (!d->rxn_sp || !d->rxn_nu || !d->arrh || !d->reversible || !d->kind))
    return fail(err, "null reaction array");

  // ---- species checks
  for (int k = 0; k < ns; ++k) {
    if (!(d->W[k] > 0.0) || !isfinite(d->W[k])) return fail(err, "species %d: molar mass must be > 0", k);
    for (int e = 0; e < 4; ++e)
      if (d->elem[4 * k + e] < 0) return fail(err, "species %d: negative atom count", k);
    const double* nk = d->nasa + 17 * (size_t)k;
    for (int i = 0; i < 17; ++i)
      if (!isfinite(nk[i])) return fail(err, "species %d: non-finite NASA-7 entry %d", k, i);
    if (!(nk[0] > 0.0 && nk[0] < nk[1] && nk[1] < nk[2]))
      return fail(err, "species %d: NASA-7 ranges need 0 < T_lo < T_mid < T_hi", k);
    double c1, h1, s1, c2, h2, s2;
    nasa_eval(nk + 3, nk[1], &c1, &h1, &s1);
    nasa_eval(nk + 10, nk[1], &c2, &h2, &s2);
    if (!close_rel(c1, c2, 1e-3) || !close_rel(h1, h2, 1e-3) || !close_rel(s1, s2, 1e-3))
      return fail(err, "species %d: NASA-7 polynomials discontinuous at T_mid", k);
  }

  // ---- reaction checks
  int n_troe = 0, n_tb = 0;
  for (int j = 0; j < nr; ++j) {
    const int* sp = d->rxn_sp + 4 * (size_t)j;
    const int* nu = d->rxn_nu + 4 * (size_t)j;
    int mol_r = 0, mol_p = 0;
    long long bal[4] = {0, 0, 0, 0};
    for (int s = 0; s < 4; ++s) {
      if (sp[s] < 0) {
        if (nu[s] != 0) return fail(err, "reaction %d: coefficient on an empty slot %d", j, s);
        continue;
      }
      if (sp[s] >= ns) return fail(err, "reaction %d: species index out of range in slot %d", j, s);
      if (s < 2 && nu[s] >= 0) return fail(err, "reaction %d: reactant slot %d needs nu < 0", j, s);
      if (s >= 2 && nu[s] <= 0) return fail(err, "reaction %d: product slot %d needs nu > 0", j, s);
      if (s < 2) mol_r += -nu[s];
      else mol_p += nu[s];
      for (int e = 0; e < 4; ++e) bal[e] += (long long)nu[s] * d->elem[4 * (size_t)sp[s] + e];
    }
    if (sp[0] >= 0 && sp[1] >= 0 && sp[0] == sp[1]) return fail(err, "reaction %d: repeated reactant slot", j);
    if (sp[2] >= 0 && sp[3] >= 0 && sp[2] == sp[3]) return fail(err, "reaction %d: repeated product slot", j);
    if (mol_r < 1 || mol_p < 1) return fail(err, "reaction %d: needs at least one reactant and one product", j);
    if (mol_r > 2 || mol_p > 2) return fail(err, "reaction %d: at most two molecules per side are supported", j);
    for (int e = 0; e < 4; ++e)
      if (bal[e] != 0) return fail(err, "reaction %d: element %d not balanced", j, e);
    const double* ar = d->arrh + 3 * (size_t)j;
    if (!(ar[0] > 0.0) || !isfinite(ar[0]) || !isfinite(ar[1]) || !isfinite(ar[2]))
      return fail(err, "reaction %d: Arrhenius parameters must be finite with A > 0", j);
    const int kind = d->kind[j];
    if (kind < 0 || kind > 2) return fail(err, "reaction %d: kind %d not in {0,1,2}", j, kind);
    if (kind > 0) {
      if (!d->eff) return fail(err, "reaction %d: third-body efficiencies missing", j);
      for (int k = 0; k < ns; ++k) {
        const double e = d->eff[(size_t)j * ns + k];
        if (!(e >= 0.0) || !isfinite(e)) return fail(err, "reaction %d: bad efficiency for species %d", j, k);
      }
    }
    if (kind == 2) {
      if (!d->falloff) return fail(err, "reaction %d: falloff parameters missing", j);
      const double* fo = d->falloff + 7 * (size_t)j;
      if (!(fo[0] > 0.0) || !isfinite(fo[0]) || !isfinite(fo[1]) || !isfinite(fo[2]))
        return fail(err, "reaction %d: low-pressure Arrhenius parameters must be finite with A0 > 0", j);
      if (!isfinite(fo[3]) || !(fo[4] > 0.0) || !(fo[5] > 0.0) || !isfinite(fo[6]) || !isfinite(fo[4]) ||
          !isfinite(fo[5]))
        return fail(err, "reaction %d: Troe parameters need finite a, T***>0, T*>0, T**", j);
      ++n_troe;
    }
    if (kind == 1) ++n_tb;
  }

  // ---- reaction order: Troe, third body, elementary (stable)
  std::vector<int32_t> perm;
  perm.reserve(nr);
  for (int want : {2, 1, 0})
    for (int j = 0; j < nr; ++j)
      if (d->kind[j] == want) perm.push_back(j);

  // ---- species-major stoichiometry list (net coefficients, packed order)
  std::vector<std::vector<std::pair<int, double>>> rows(ns);
  for (int r = 0; r < nr; ++r) {
    const int j = perm[r];
    double net[RK_MAX_SPECIES + 1];
    int touched[4];
    int nt = 0;
    for (int s = 0; s < 4; ++s) {
      const int k = d->rxn_sp[4 * (size_t)j + s];
      if (k < 0) continue;
      bool seen = false;
      for (int t = 0; t < nt; ++t) seen |= (touched[t] == k);
      if (!seen) {
        touched[nt++] = k;
        net[k] = 0.0;
      }
      net[k] += d->rxn_nu[4 * (size_t)j + s];
    }
    for (int t = 0; t < nt; ++t)
      if (net[touched[t]] != 0.0) rows[touched[t]].push_back({r, net[touched[t]]});
  }
  int nnz = 0;
  for (auto& row : rows) nnz += (int)row.size();

  // ---- pieces of the list for the gather w = nu^T q: every species row is cut
  // into near-equal pieces of at most Lp entries; one lane sums one piece, so
  // a warp's loop runs ceil(npiece/32) x Lp times instead of the longest row.
  // Lp minimises that count plus the adds that join a species' pieces.
  int maxdeg = 1;
  for (auto& row : rows) maxdeg = std::max(maxdeg, (int)row.size());
  int Lp = maxdeg;
  {
    long best = -1;
    for (int cand = 1; cand <= maxdeg; ++cand) {
      int P = 0, maxp = 1;
      for (auto& row : rows) {
        const int pk = std::max(1, ((int)row.size() + cand - 1) / cand);
        P += pk;
        maxp = std::max(maxp, pk);
      }
      const long cost = (long)((P + 31) / 32) * cand + (maxp - 1);
      if (best < 0 || cost < best) {
        best = cost;
        Lp = cand;
      }
    }
  }
  std::vector<int32_t> piece_ptr, spec_piece;
  {
    int pos = 0;
    for (int k = 0; k < ns; ++k) {
      spec_piece.push_back((int32_t)piece_ptr.size());
      const int deg = (int)rows[k].size();
      const int pk = std::max(1, (deg + Lp - 1) / Lp);
      for (int i = 0; i < pk; ++i) piece_ptr.push_back(pos + (int)((long)deg * i / pk));
      pos += deg;
    }
    spec_piece.push_back((int32_t)piece_ptr.size());
    piece_ptr.push_back(pos);
  }
  const int npiece = (int)piece_ptr.size() - 1;

  // ---- layout
  MechLayout L;
  L.ns = ns;
  L.nr = nr;
  L.ntb = n_troe + n_tb;
  L.ntroe = n_troe;
  L.nnz = nnz;
  L.npiece = npiece;
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    const int64_t o = off;
    off = align16(off + bytes);
    return o;
  };
  L.off_W = take(8 * ns);
  L.off_invW = take(8 * ns);
  L.off_Tmid = take(8 * ns);
  L.off_lo = take(8 * (int64_t)NCOEF * ns);
  L.off_hi = take(8 * (int64_t)NCOEF * ns);
  L.off_lnA = take(8 * (int64_t)nr);
  L.off_b = take(8 * (int64_t)nr);
  L.off_EaR = take(8 * (int64_t)nr);
  L.off_eff = take(8 * (int64_t)L.ntb * ns);
  L.off_fo = take(8 * (int64_t)L.ntb * FO_STRIDE);
  L.off_csr_nu = take(8 * (int64_t)nnz);
  L.off_slots = take(4 * (int64_t)nr);
  L.off_meta = take(4 * (int64_t)nr);
  L.off_csr_ptr = take(4 * (int64_t)(ns + 1));
  L.off_csr_j = take(4 * (int64_t)nnz);
  L.off_piece_ptr = take(4 * (int64_t)(npiece + 1));
  L.off_spec_piece = take(4 * (int64_t)(ns + 1));
  // what only some kernels read comes last, so a kernel copies a prefix:
  // FP64 paths stop here, the double-float gathers also read csr_nuf, the FP32
  // Jacobian-vector product the other FP32 copies; perm is read from global memory
  L.bytes_fp64 = off;
  L.off_csr_nuf = take(4 * (int64_t)nnz);
  L.bytes_df = off;
  L.off_Wf = take(4 * (int64_t)ns);
  L.off_invWf = take(4 * (int64_t)ns);
  L.off_bf = take(4 * (int64_t)nr);
  L.off_EaRf = take(4 * (int64_t)nr);
  L.off_efff = take(4 * (int64_t)L.ntb * ns);
  L.bytes_f32 = off;
  L.off_perm = take(4 * (int64_t)nr);
  // reaction slots per species (filled below from the packed slots)
  std::vector<std::vector<int32_t>> roles(ns);
  for (int r = 0; r < nr; ++r) {
    const int j = perm[r];
    // the same expansion as the packed slots below: entries 0, 1 reactants, 2, 3 products
    int sl[4] = {ns, ns, ns, ns}, a = 0, b = 2;
    for (int s = 0; s < 4; ++s) {
      const int k = d->rxn_sp[4 * (size_t)j + s], nu = d->rxn_nu[4 * (size_t)j + s];
      if (k < 0) continue;
      for (int t = 0; t < (nu < 0 ? -nu : nu); ++t) {
        if (s < 2 && a < 2) sl[a++] = k;
        else if (s >= 2 && b < 4) sl[b++] = k;
      }
    }
    for (int role = 0; role < 4; ++role)
      if (sl[role] < ns) roles[sl[role]].push_back(r << 2 | role);
  }
  for (auto& v : roles) L.nrole += (int32_t)v.size();
  L.off_role_ptr = take(4 * (int64_t)(ns + 1));
  L.off_role = take(4 * (int64_t)(L.nrole > 0 ? L.nrole : 1));
  L.nst = (ns + 15) / 16;
  L.nrt = (nr + 15) / 16;
  L.off_nuT = take(16 * 32 * (int64_t)L.nst * L.nrt);
  L.bytes = align16(off);

  std::vector<unsigned char> buf((size_t)L.bytes, 0);
  auto D = [&](int64_t o) { return reinterpret_cast<double*>(buf.data() + o); };
  auto I = [&](int64_t o) { return reinterpret_cast<int32_t*>(buf.data() + o); };
  auto U = [&](int64_t o) { return reinterpret_cast<uint32_t*>(buf.data() + o); };

  for (int k = 0; k < ns; ++k) {
    D(L.off_W)[k] = d->W[k];
    D(L.off_invW)[k] = 1.0 / d->W[k];
    const double* nk = d->nasa + 17 * (size_t)k;
    D(L.off_Tmid)[k] = nk[1];
    for (int range = 0; range < 2; ++range) {
      const double* a = nk + 3 + 7 * range;
      double* c = D(range == 0 ? L.off_lo : L.off_hi);
      const double v[NCOEF] = {a[0],       a[1],       a[2],       a[3],       a[4],      a[1] / 2.0,
                               a[2] / 3.0, a[3] / 4.0, a[4] / 5.0, a[5],       a[2] / 2.0, a[3] / 3.0,
                               a[4] / 4.0, a[6],       2.0 * a[2], 3.0 * a[3], 4.0 * a[4]};
      for (int i = 0; i < NCOEF; ++i) c[(size_t)i * ns + k] = v[i];
    }
  }
  int slot_tb = 0;
  for (int r = 0; r < nr; ++r) {
    const int j = perm[r];
    const int* sp = d->rxn_sp + 4 * (size_t)j;
    const int* nu = d->rxn_nu + 4 * (size_t)j;
    // expand to at most two molecules per side; ns is the empty sentinel
    int mr[2] = {ns, ns}, mp[2] = {ns, ns};
    int ir = 0, ip = 0;
    int mol_r = 0, mol_p = 0;
    for (int s = 0; s < 4; ++s) {
      if (sp[s] < 0) continue;
      const int n = nu[s] < 0 ? -nu[s] : nu[s];
      for (int t = 0; t < n; ++t) {
        if (s < 2) mr[ir++] = sp[s];
        else mp[ip++] = sp[s];
      }
      if (s < 2) mol_r += n;
      else mol_p += n;
    }
    U(L.off_slots)[r] = (uint32_t)mr[0] | ((uint32_t)mr[1] << 8) | ((uint32_t)mp[0] << 16) | ((uint32_t)mp[1] << 24);
    const int kind = d->kind[j];
    const int order = mol_r + (kind == 1 ? 1 : 0);  // concentration order of the forward rate
    const double* ar = d->arrh + 3 * (size_t)j;
    D(L.off_lnA)[r] = log(ar[0]) + (order - 1) * log(1e-6);
    D(L.off_b)[r] = ar[1];
    D(L.off_EaR)[r] = ar[2] / R_GAS;
    int slot = 0;
    if (kind > 0) {
      slot = slot_tb++;
      for (int k = 0; k < ns; ++k) D(L.off_eff)[(size_t)slot * ns + k] = d->eff[(size_t)j * ns + k];
      if (kind == 2) {
        const double* fo = d->falloff + 7 * (size_t)j;
        double* o = D(L.off_fo) + (size_t)slot * FO_STRIDE;
        o[0] = log(fo[0]) + mol_r * log(1e-6);  // k0 has one more concentration order
        o[1] = fo[1];
        o[2] = fo[2] / R_GAS;
        o[3] = fo[3];
        o[4] = 1.0 / fo[4];
        o[5] = 1.0 / fo[5];
        o[6] = fo[6];
        o[7] = 0.0;
      }
    }
    const int rev = d->reversible[j] ? 1 : 0;
    const int dnu = mol_p - mol_r;  // -1, 0 or 1
    I(L.off_meta)[r] = kind | (rev << 2) | ((dnu + 4) << 4) | (slot << 8);
  }
  int pos = 0;
  for (int k = 0; k < ns; ++k) {
    I(L.off_csr_ptr)[k] = pos;
    for (auto& e : rows[k]) {
      I(L.off_csr_j)[pos] = e.first;
      D(L.off_csr_nu)[pos] = e.second;
      ++pos;
    }
  }
  I(L.off_csr_ptr)[ns] = pos;
  for (int p = 0; p <= npiece; ++p) I(L.off_piece_ptr)[p] = piece_ptr[p];
  for (int k = 0; k <= ns; ++k) I(L.off_spec_piece)[k] = spec_piece[k];
  auto F = [&](int64_t o) { return reinterpret_cast<float*>(buf.data() + o); };
  for (int k = 0; k < ns; ++k) {
    F(L.off_Wf)[k] = (float)D(L.off_W)[k];
    F(L.off_invWf)[k] = (float)D(L.off_invW)[k];
  }
  for (int r = 0; r < nr; ++r) {
    F(L.off_bf)[r] = (float)D(L.off_b)[r];
    F(L.off_EaRf)[r] = (float)D(L.off_EaR)[r];
  }
  for (int i = 0; i < L.ntb * ns; ++i) F(L.off_efff)[i] = (float)D(L.off_eff)[i];
  for (int i = 0; i < nnz; ++i) F(L.off_csr_nuf)[i] = (float)D(L.off_csr_nu)[i];
  for (int r = 0; r < nr; ++r) I(L.off_perm)[r] = perm[r];
  {
    int pos = 0;
    for (int k = 0; k < ns; ++k) {
      I(L.off_role_ptr)[k] = pos;
      for (int32_t e : roles[k]) I(L.off_role)[pos++] = e;
    }
    I(L.off_role_ptr)[ns] = pos;
  }
  // nu^T tiles for the tensor-core gather: net coefficients (small integers,
  // exact in BF16) placed in each lane's A-operand registers of mma.m16n8k16
  // (register 0: row g, columns 2t, 2t+1; 1: row g+8; 2: row g, columns
  // 2t+8, 2t+9; 3: row g+8; g = lane / 4, t = lane % 4; the lower column in
  // the lower 16 bits)
  {
    std::vector<double> A((size_t)ns * nr, 0.0);
    for (int k = 0; k < ns; ++k)
      for (auto& e : rows[k]) A[(size_t)k * nr + e.first] = e.second;
    auto a = [&](int k, int r) { return (k < ns && r < nr) ? A[(size_t)k * nr + r] : 0.0; };
    auto bf16 = [](double x) {
      const float f = (float)x;  // a small integer: its BF16 is the float's upper half, exactly
      uint32_t u;
      memcpy(&u, &f, 4);
      return u >> 16;
    };
    auto pack = [&](int k, int r) { return bf16(a(k, r)) | (bf16(a(k, r + 1)) << 16); };
    uint32_t* T = U(L.off_nuT);
    for (int st = 0; st < L.nst; ++st)
      for (int rt = 0; rt < L.nrt; ++rt)
        for (int l = 0; l < 32; ++l) {
          const int g = l >> 2, t = l & 3, k0 = 16 * st + g, r0 = 16 * rt + 2 * t;
          uint32_t* R = T + 4 * ((size_t)(st * L.nrt + rt) * 32 + l);
          R[0] = pack(k0, r0);
          R[1] = pack(k0 + 8, r0);
          R[2] = pack(k0, r0 + 8);
          R[3] = pack(k0 + 8, r0 + 8);
        }
  }

  out->L = L;
  out->packed.swap(buf);
  out->perm.swap(perm);
  return true;
}

}  // namespace rk
