// Definitions of the per-cell kernel launches declared in device.cuh.  Only
// the k_*.cu translation units include this header, each explicitly
// instantiating its share, so every heavy kernel is compiled exactly once.
#pragma once
#include "device.cuh"

namespace rk {

// Persistent ROK4E launch: as many cells per block as shared memory allows
// (or a.cells_per_block), one wave of blocks sized to the device.
template <int G, bool MIXED, bool TC>
int launch_rok4e(const IntegrateLaunch& a) {
  IntegrateParams& P = *a.P;
  LaunchPlan plan;
  const int rc = plan_for<G>(rok4e_integrate_kernel<G, MIXED, TC>, a.mech, P.S, a.cells_per_block, a.ncell, true,
                             &plan, a.blocks_per_sm, a.static_bins, P.mech_copy + P.tc_bytes);
  if (rc) return rc;
  if (a.static_bins) P.subq = plan.cells_per_block % 4 == 0 ? 4 : (plan.cells_per_block % 2 == 0 ? 2 : 1);
  rok4e_integrate_kernel<G, MIXED, TC><<<plan.blocks, plan.cells_per_block * G, plan.smem, a.stream>>>(P);
  return RK_OK;
}

// Persistent explicit Dormand-Prince launch, planned like ROK4E's.
template <int G>
int launch_rkdp(const IntegrateLaunch& a) {
  IntegrateParams& P = *a.P;
  LaunchPlan plan;
  const int rc = plan_for<G>(rkdp_integrate_kernel<G>, a.mech, P.S, a.cells_per_block, a.ncell, true, &plan,
                             a.blocks_per_sm, a.static_bins, P.mech_copy);
  if (rc) return rc;
  if (a.static_bins) P.subq = plan.cells_per_block % 4 == 0 ? 4 : (plan.cells_per_block % 2 == 0 ? 2 : 1);
  rkdp_integrate_kernel<G><<<plan.blocks, plan.cells_per_block * G, plan.smem, a.stream>>>(P);
  return RK_OK;
}

// The adjoint: 128-thread blocks of 128 / G cell slots, the mechanism in
// shared memory; enough blocks for one slot per cell, at most as many as the
// device holds at once (the cells are then dealt over them in turn).  Filling
// every resident slot instead, with some warps holding one or two cells,
// measured 28 % slower on 4096 cells at 8 lanes.
template <int G>
int launch_adjoint(const AdjointParams& P, size_t smem, cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(rok4e_adjoint_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
  int n_sm = 0;
  size_t smem_max = 0;
  const int rc = device_props(&n_sm, &smem_max);
  if (rc) return rc;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rok4e_adjoint_kernel<G>, 128, smem);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) return set_error(RK_E_UNSUPPORTED, "adjoint kernel cannot be resident on an SM");
  const int64_t resident = (int64_t)per_sm * n_sm;
  const int64_t need = (P.ncell * G + 127) / 128;
  const int64_t blocks = need < resident ? need : resident;
  rok4e_adjoint_kernel<G><<<(unsigned)blocks, 128, smem, st>>>(P);
  return RK_OK;
}

}  // namespace rk
