// Internal layout shared by the host packing code (mech.cpp) and the kernels.
//
// A loaded mechanism is one contiguous device buffer.  Every block of the
// integration kernels copies a prefix of it verbatim into shared memory (as
// much as its precision level reads), so the offsets below are valid relative
// to either copy.  Reactions are reordered so that
// Troe falloff reactions come first, then third-body reactions, then the
// elementary ones: the lanes that take the longer pressure-dependent code path
// then all sit in the first iteration of the per-lane reaction loop.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace rk {

// Thermo coefficients stored per species and per range, coefficient-major
// ([NCOEF][ns]):
//   0..4   a1..a5                 cp/R = a1 + T(a2 + T(a3 + T(a4 + T a5)))
//   5..8   a2/2, a3/3, a4/4, a5/5 h/RT = a1 + T(c5 + T(c6 + T(c7 + T c8))) + a6/T
//   9      a6
//   10..12 a3/2, a4/3, a5/4       s/R  = a1 ln T + T(a2 + T(c10 + T(c11 + T c12))) + a7
//   13     a7
//   14..16 2a3, 3a4, 4a5          d(cp/R)/dT = a2 + T(c14 + T(c15 + T c16))
constexpr int NCOEF = 17;
constexpr int FO_STRIDE = 8;  // lnA0(SI), b0, Ea0/R, a, 1/T***, 1/T*, T**, unused

struct MechLayout {
  int32_t ns = 0, nr = 0;
  int32_t ntb = 0;  // reactions with kind > 0 (they come first)
  int32_t ntroe = 0;  // Troe falloff reactions: the first ntroe, third-body slots 0..ntroe-1
  int32_t nnz = 0;  // entries of the species-major stoichiometry list
  int32_t npiece = 0;  // pieces the list is split into for the gather (>= ns)
  // byte offsets into the packed buffer (all multiples of 16)
  int64_t off_W = 0, off_invW = 0, off_Tmid = 0, off_lo = 0, off_hi = 0;
  int64_t off_lnA = 0, off_b = 0, off_EaR = 0;
  int64_t off_eff = 0;  // [ntb][ns]
  int64_t off_fo = 0;   // [ntb][FO_STRIDE]
  int64_t off_csr_nu = 0;
  int64_t off_slots = 0;  // uint32 per reaction: ra | rb<<8 | pa<<16 | pb<<24 (ns = empty)
  int64_t off_meta = 0;   // int32 per reaction: kind | rev<<2 | (dnu+4)<<4 | slot<<8
  int64_t off_csr_ptr = 0, off_csr_j = 0;
  int64_t off_piece_ptr = 0;   // int32 [npiece + 1]: list offset of each piece
  int64_t off_spec_piece = 0;  // int32 [ns + 1]: first piece of each species
  // FP32 copies read by the reduced-precision Jacobian-vector product
  int64_t off_Wf = 0, off_invWf = 0, off_bf = 0, off_EaRf = 0, off_efff = 0, off_csr_nuf = 0;
  int64_t off_perm = 0;  // int32 per packed reaction: its index in the input description
  // species-major list of the reaction slots each species fills (the adjoint's
  // deterministic gathers of d/dC and d/dg): entry r << 2 | role, role 0..3 =
  // the slot ra, rb, pa, pb of packed reaction r; species k's entries are
  // role[role_ptr[k] .. role_ptr[k + 1])
  int32_t nrole = 0;
  int64_t off_role_ptr = 0, off_role = 0;
  // nu^T (species x packed reactions) as the A operands of 16 x 16 BF16 mma tiles:
  // tile (st, rt) holds, for each lane, its four 32-bit registers (8 BF16) together
  int32_t nst = 0, nrt = 0;  // species tiles, reaction tiles
  int64_t off_nuT = 0;       // [nst][nrt][32 lanes] x 16 bytes
  int64_t bytes = 0;
  // prefixes of the buffer that kernels copy to shared memory: through the FP64
  // arrays; also csr_nuf (double-float gathers); also the other FP32 copies
  int64_t bytes_fp64 = 0, bytes_df = 0, bytes_f32 = 0;
};

struct HostMech {
  MechLayout L;
  std::vector<unsigned char> packed;  // host copy of the device buffer
  std::vector<int32_t> perm;          // packed reaction r came from input reaction perm[r]
};

// Validate and pack; returns false and fills err on an invalid description.
bool pack_mechanism(const void* desc, HostMech* out, std::string* err);

}  // namespace rk
