// GB300 (sm_103a) C ABI of the ROK4E reaction step and the Simpler split step
// (include/rok4e.h): argument checks, launch planning, the small kernels
// (work-queue ordering, adjoint reduction, 1-D transport, probes) and the
// library's error state.  The per-cell kernels live in device.cuh and are
// compiled in the k_*.cu translation units.
#include "device.cuh"

namespace rk {

// --------------------------------------------------------------- error state
static thread_local std::string g_last_error;
int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int cuda_error(cudaError_t e, const char* where) {
  return set_error(RK_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

__global__ void __launch_bounds__(ORDER_THREADS) order_count_kernel(const double* __restrict__ h, int64_t n,
                                                                    int64_t chunk, double dt, unsigned* hist) {
  __shared__ unsigned sh[ORDER_BINS];
  for (int i = threadIdx.x; i < ORDER_BINS; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&sh[cost_bin(h[i], dt)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < ORDER_BINS; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Also counts the "hot" cells, those within a factor 4 of the most expensive
// expected cost (the eight quarter-octave bins from the highest occupied one
// down), when that cost is at least 2 substeps; the static-bin queue gives
// each of them a group of warps of its own.
__global__ void order_scan_kernel(const unsigned* hist, unsigned* cursor, unsigned* nhot) {
  if (threadIdx.x == 0) {
    unsigned acc = 0u;
    int top = -1;
    for (int b = ORDER_BINS - 1; b >= 0; --b) {  // most expensive bin first
      cursor[b] = acc;
      acc += hist[b];
      if (top < 0 && hist[b] > 0u) top = b;
    }
    unsigned hot = 0u;
    if (top >= 4)
      for (int b = top; b > top - 8 && b >= 0; --b) hot += hist[b];
    // expected substeps (2^(bin/4)) of the hottest cell and of all the others
    float rest = 0.f;
    for (int b = 0; b < ORDER_BINS; ++b)
      if (!(top >= 4 && b > top - 8 && b <= top)) rest += (float)hist[b] * exp2f(0.25f * (float)b);
    nhot[0] = hot;
    nhot[1] = __float_as_uint(top >= 0 ? exp2f(0.25f * (float)top) : 0.f);
    nhot[2] = __float_as_uint(rest);
  }
}

__global__ void __launch_bounds__(ORDER_THREADS) order_scatter_kernel(const double* __restrict__ h, int64_t n,
                                                                      int64_t chunk, double dt, unsigned* cursor,
                                                                      int32_t* perm) {
  __shared__ unsigned cnt[ORDER_BINS], base[ORDER_BINS];
  for (int i = threadIdx.x; i < ORDER_BINS; i += blockDim.x) cnt[i] = 0u;
  __syncthreads();
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&cnt[cost_bin(h[i], dt)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < ORDER_BINS; i += blockDim.x) {
    base[i] = cnt[i] ? atomicAdd(&cursor[i], cnt[i]) : 0u;
    cnt[i] = 0u;
  }
  __syncthreads();
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int b = cost_bin(h[i], dt);
    perm[base[b] + atomicAdd(&cnt[b], 1u)] = (int32_t)i;
  }
}

// grad[perm[r]] = sum over cells of theta[cell][r] (cell records stride doubles
// apart); one block per reaction
// with a fixed-order tree, so the sum does not depend on scheduling.
__global__ void __launch_bounds__(256) adjoint_reduce_kernel(const double* __restrict__ theta, int64_t ncell,
                                                             int64_t stride, const int32_t* __restrict__ perm,
                                                             double* grad) {
  __shared__ double sh[256];
  const int r = blockIdx.x;
  double acc = 0.0;
  for (int64_t c = threadIdx.x; c < ncell; c += blockDim.x) acc += theta[c * stride + r];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad[perm[r]] = sh[0];
}

// ---------------------------------------------------------- 1-D transport
// TU = D (U[i-1] - 2 U[i] + U[i+1]) / dx^2 with zero-gradient ends, and the
// three SSP-RK3 stages of dU/dt = T(U) - Tn over dt/2 (Shu-Osher form).  The
// per-entry arithmetic sits in the inline functions below with every rounding
// explicit (fma, __dmul_rn, __dadd_rn), so the whole-domain kernels and the
// kernels on a slice held with ghost rows give the same bits for the same
// neighbours -- a domain split over ranks reproduces the unsplit step exactly.
__device__ __forceinline__ double diffusion_value(double xm, double x0, double xp, double D, double inv_dx2) {
  const double lap = __dadd_rn(fma(-2.0, x0, xm), xp);
  return __dmul_rn(D, __dmul_rn(lap, inv_dx2));
}

// stage 0: X + k g(X); stage 1: 3/4 U1 + 1/4 (X + k g(X)); stage 2:
// 1/3 U1 + 2/3 (X + k g(X)), with g(X) = T(X) + sigma s and tx = T(X)
__device__ __forceinline__ double ssprk3_combine(int stage, double u1, double x0, double tx, bool has_s, double s,
                                                 double sigma, double k) {
  const double gX = has_s ? fma(sigma, s, tx) : tx;
  const double xk = fma(k, gX, x0);
  if (stage == 0) return xk;
  if (stage == 1) return fma(0.75, u1, __dmul_rn(0.25, xk));
  return fma(2.0 / 3.0, xk, __ddiv_rn(u1, 3.0));
}

// the same with T(X) = D lap X from the neighbours
__device__ __forceinline__ double ssprk3_value(int stage, double u1, double xm, double x0, double xp, bool has_s,
                                               double s, double sigma, double D, double inv_dx2, double k) {
  return ssprk3_combine(stage, u1, x0, diffusion_value(xm, x0, xp, D, inv_dx2), has_s, s, sigma, k);
}

// A stage with T(X) given (the caller's transport operator): Out = the stage of
// U1, X and TX elementwise over n entries.
__global__ void ssprk3_combine_kernel(int stage, const double* __restrict__ U1, const double* __restrict__ X,
                                      const double* __restrict__ TX, const double* __restrict__ S, double sigma,
                                      double* Out, int64_t n, double k) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  Out[idx] = ssprk3_combine(stage, U1[idx], X[idx], TX[idx], S != nullptr, S ? S[idx] : 0.0, sigma, k);
}

// c = (a R + b T) elementwise (the balancing constants of the splittings)
__global__ void axpby_kernel(const double* __restrict__ R, const double* __restrict__ T, double a, double b,
                             double* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * R[i] + b * T[i];
}

__global__ void diffusion_kernel(const double* __restrict__ U, double* __restrict__ TU, int64_t n, int nv,
                                 double D, double inv_dx2) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nv) return;
  const int64_t i = idx / nv;
  const int v = (int)(idx - i * nv);
  const int64_t im = i > 0 ? i - 1 : 0, ip = i + 1 < n ? i + 1 : n - 1;
  TU[idx] = diffusion_value(U[im * nv + v], U[idx], U[ip * nv + v], D, inv_dx2);
}

__global__ void ssprk3_stage_kernel(int stage, const double* __restrict__ U1, const double* __restrict__ X,
                                    const double* __restrict__ S, double sigma, double* Out, int64_t n, int nv,
                                    double D, double inv_dx2, double k) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nv) return;
  const int64_t i = idx / nv;
  const int v = (int)(idx - i * nv);
  const int64_t im = i > 0 ? i - 1 : 0, ip = i + 1 < n ? i + 1 : n - 1;
  Out[idx] = ssprk3_value(stage, U1[idx], X[im * nv + v], X[idx], X[ip * nv + v], S != nullptr,
                          S ? S[idx] : 0.0, sigma, D, inv_dx2, k);
}

// The same two operations on a slice of n points held with one ghost row on
// each side: Xext has n + 2 rows, row r + 1 is the slice's point r.
__global__ void diffusion_ghost_kernel(const double* __restrict__ Xext, double* __restrict__ TU, int64_t n, int nv,
                                       double D, double inv_dx2) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nv) return;
  const double* c = Xext + nv + idx;
  TU[idx] = diffusion_value(c[-nv], c[0], c[nv], D, inv_dx2);
}

__global__ void ssprk3_stage_ghost_kernel(int stage, const double* __restrict__ U1, const double* __restrict__ Xext,
                                          const double* __restrict__ S, double sigma, double* Out, int64_t n,
                                          int nv, double D, double inv_dx2, double k) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nv) return;
  const double* c = Xext + nv + idx;
  Out[idx] = ssprk3_value(stage, U1[idx], c[-nv], c[0], c[nv], S != nullptr, S ? S[idx] : 0.0, sigma, D,
                          inv_dx2, k);
}

// ------------------------------------------------------------------ probes
__global__ void exp_eval_kernel(const double* __restrict__ x, double* __restrict__ y, int64_t n, int which) {
  __shared__ double tab[RK_EXP2_TABLE_N];
  load_exp_table(tab);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (which == 0) {
    y[i] = exp_fast(x[i], tab);
  } else if (which == 6) {
    y[i] = log_fast(x[i]);
  } else if (which == 7) {
    y[i] = rcp_any(x[i]);
  } else if (which == 3) {
    y[i] = exp_mixed(x[i], tab);
  } else if (which == 4 || which == 5) {
    double ep, em;
    exp_pm_mixed(x[i], tab, &ep, &em);
    y[i] = which == 4 ? ep : em;
  } else {
    double ep, em;
    exp_pm(x[i], tab, &ep, &em);
    y[i] = which == 1 ? ep : em;
  }
}

__global__ void probe_fp64_kernel(double* out, int iters, double a, int active_lanes = 32) {
  if ((int)(threadIdx.x & 31) >= active_lanes) return;
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
  double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, a); x1 = fma(x1, a, a); x2 = fma(x2, a, a); x3 = fma(x3, a, a);
    x4 = fma(x4, a, a); x5 = fma(x5, a, a); x6 = fma(x6, a, a); x7 = fma(x7, a, a);
  }
  const double r = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (r == 12345.678) out[0] = r;
}
__global__ void probe_fp32_kernel(float* out, int iters, float a) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-9f + j * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, a);
  }
  float r = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) r += x[j];
  if (r == 12345.678f) out[0] = r;
}
// Double-float (FP32 pair) multiply-add, a*b + c with a 48-bit significand:
// exact product by fmaf, error-free sum (Knuth's two-sum) of the leading parts.
struct f2 {
  float h, l;
};
__device__ __forceinline__ f2 df_fma(f2 a, f2 b, f2 c) {
  const float ph = a.h * b.h;
  float pl = fmaf(a.h, b.h, -ph);
  pl = fmaf(a.h, b.l, pl);
  pl = fmaf(a.l, b.h, pl);
  const float sh = ph + c.h;
  const float bb = sh - ph;
  const float sl = (ph - (sh - bb)) + (c.h - bb);
  const float t = sl + pl + c.l;
  const float h = sh + t;
  return {h, t - (h - sh)};
}
__global__ void probe_df_kernel(float* out, int iters, float ah, float al) {
  const f2 a{ah, al};
  f2 x[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) x[j] = {threadIdx.x * 1e-9f + j * 1e-3f, 0.f};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = df_fma(x[j], a, a);
  }
  float r = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) r += x[j].h + x[j].l;
  if (r == 12345.678f) out[0] = r;
}
__global__ void probe_cvt_kernel(double* out, int iters) {
  double x0 = 1.0 + threadIdx.x * 1e-9, x1 = x0 + 0.25, x2 = x0 + 0.5, x3 = x0 + 0.75;
  for (int i = 0; i < iters; ++i) {  // two conversions and one FP32 multiply per step
    x0 = (double)((float)x0 * 0.9999999f); x1 = (double)((float)x1 * 0.9999999f);
    x2 = (double)((float)x2 * 0.9999999f); x3 = (double)((float)x3 * 0.9999999f);
  }
  const double r = x0 + x1 + x2 + x3;
  if (r == 12345.678) out[0] = r;
}
// int -> double conversions (I2F.F64): eight chains of a conversion, a bit
// move and an integer xor, with no FP64 arithmetic
__global__ void probe_i2f_kernel(double* out, int iters) {
  int k[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) k[j] = (int)threadIdx.x + 1000 * j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) k[j] = __double2hiint((double)k[j]) ^ (k[j] + i);
  }
  int r = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) r ^= k[j];
  if (r == 123456789) out[0] = (double)r;
}
__global__ void probe_exp_kernel(double* out, int iters) {
  double x0 = -threadIdx.x * 1e-6, x1 = x0 - 0.25, x2 = x0 - 0.5, x3 = x0 - 0.75;
  for (int i = 0; i < iters; ++i) {
    x0 = exp(x0) - 1.5; x1 = exp(x1) - 1.5; x2 = exp(x2) - 1.5; x3 = exp(x3) - 1.5;
  }
  const double r = x0 + x1 + x2 + x3;
  if (r == 12345.678) out[0] = r;
}

}  // namespace rk

// =============================================================================
// Host side
// =============================================================================
using namespace rk;

namespace {

// A stride coprime with n near n * 0.618 (golden-ratio interleave of the queue).
unsigned long long queue_stride(int64_t n) {
  if (n <= 2) return 1;
  unsigned long long st = (unsigned long long)((double)n * 0.6180339887498949);
  if (st < 1) st = 1;
  auto gcd = [](unsigned long long a, unsigned long long b) {
    while (b) {
      const unsigned long long t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  while (gcd(st, (unsigned long long)n) != 1) ++st;
  return st % (unsigned long long)n;
}

int check_mech(const rk_mech* mech) {
  if (!mech || !mech->dev) return set_error(RK_E_INVALID_ARGUMENT, "null mechanism handle");
  return RK_OK;
}

// method 0: ROK4E; 1: explicit Dormand-Prince 5(4) (M unused)
int integrate_impl(const rk_mech* mech, double* Y, const double* src, double* h_cell, int64_t ncell, double p,
                   double dt, double rtol, double atol, int32_t M, const rk_opts* opts, int32_t* stats,
                   void* workspace, size_t workspace_bytes, cudaStream_t stream, int method = 0) {
  int rc = check_mech(mech);
  if (rc) return rc;
  if (ncell < 0) return set_error(RK_E_INVALID_ARGUMENT, "ncell < 0");
  if (ncell == 0) return RK_OK;
  if (!Y) return set_error(RK_E_INVALID_ARGUMENT, "null state array");
  if (!(dt > 0.0) || !isfinite(dt)) return set_error(RK_E_INVALID_ARGUMENT, "dt must be finite and > 0");
  if (!(rtol >= 0.0) || !(atol >= 0.0) || !(rtol + atol > 0.0))
    return set_error(RK_E_INVALID_ARGUMENT, "tolerances must be >= 0 with rtol + atol > 0");
  if (!(p > 0.0) || !isfinite(p)) return set_error(RK_E_INVALID_ARGUMENT, "pressure must be finite and > 0");
  if (M < 1 || M > RK_MAX_KRYLOV) return set_error(RK_E_INVALID_ARGUMENT, "krylov_dim outside 1..8");
  rk_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.jv_mode != 0 && o.jv_mode != 1) return set_error(RK_E_INVALID_ARGUMENT, "jv_mode must be 0 or 1");
  if (o.trace_cap < 0 || (o.trace_cap > 0 && !o.trace))
    return set_error(RK_E_INVALID_ARGUMENT, "trace_cap > 0 needs a trace array");
  if (o.fixed_h < 0.0 || !isfinite(o.fixed_h)) return set_error(RK_E_INVALID_ARGUMENT, "fixed_h must be >= 0");
  if (o.precision < 0 || o.precision > 6) return set_error(RK_E_INVALID_ARGUMENT, "precision must be 0..6");
  if (method == 1 && o.precision != 0) return set_error(RK_E_INVALID_ARGUMENT, "the explicit integrator is FP64 only");
  const bool mixed = o.precision == 1 || o.precision == 2;  // level 3 runs the FP64 kernel with cs.prec = 3
  const int G = o.lanes_per_cell == 0 ? 32 : o.lanes_per_cell;
  if (G != 8 && G != 16 && G != 32) return set_error(RK_E_INVALID_ARGUMENT, "lanes_per_cell must be 0, 8, 16 or 32");
  const bool tc = o.precision == 4;
  if (tc && G != 32) return set_error(RK_E_INVALID_ARGUMENT, "precision 4 (tensor-core gather) needs 32 lanes per cell");
  if (!workspace || workspace_bytes < rk_rok4e_workspace_size(mech, ncell, M, opts))
    return set_error(RK_E_WORKSPACE, "workspace missing or smaller than rk_rok4e_workspace_size");
  if (o.reactor < 0 || o.reactor > 2) return set_error(RK_E_INVALID_ARGUMENT, "reactor must be 0, 1 or 2");
  if (o.reactor == 2 && o.precision != 0)
    return set_error(RK_E_INVALID_ARGUMENT, "the auxiliary-temperature system is FP64 only");
  const int nx = o.reactor == 2 ? RK_AUX_EXTRA : 0;
  const int N = mech->host.L.ns + 1 + nx;
  const int Meff = method == 1 ? 1 : (M > N ? N : M);
  IntegrateParams P;
  P.mech = mech->dev;
  P.L = mech->host.L;
  P.nx = nx;
  P.S = make_slot(mech->host.L, Meff, mixed, nx, o.precision == 3, tc, o.precision == 6);
  P.precision = o.precision;
  P.Y = Y;
  P.src = src;
  P.h_cell = h_cell;
  P.ncell = ncell;
  P.p = p;
  P.dt = dt;
  P.rtol = rtol;
  P.atol = atol;
  P.h0 = o.h0;
  P.fixed_h = o.fixed_h;
  P.M = Meff;
  P.jv_mode = o.jv_mode;
  P.max_attempts = o.max_attempts > 0 ? o.max_attempts : 100000;
  P.trace_cap = o.trace_cap;
  P.trace = o.trace;
  P.stats = stats;
  unsigned char* wsb = static_cast<unsigned char*>(workspace);
  P.counter = reinterpret_cast<unsigned long long*>(wsb);
  if (o.reactor == 1 && !o.rho_cell) return set_error(RK_E_INVALID_ARGUMENT, "constant volume needs rho_cell");
  P.rho_cell = o.reactor == 1 ? o.rho_cell : nullptr;
  {
    const MechLayout& L = mech->host.L;
    P.mech_copy = (method == 1 || o.precision == 0 || tc || o.precision >= 5) ? L.bytes_fp64
                                                          : (o.precision == 2 ? L.bytes_f32 : L.bytes_df);
    P.tc_bytes = tc ? (int64_t)16 * 32 * L.nst * L.nrt : 0;
  }
  P.qstride = queue_stride(ncell);
  P.order = nullptr;
  cudaError_t e = cudaMemsetAsync(wsb, 0, 768, stream);  // counter, histogram, cursors
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
  if (o.queue_order < 0 || o.queue_order > 3) return set_error(RK_E_INVALID_ARGUMENT, "queue_order must be 0..3");
  const int order = o.queue_order == 0 ? (h_cell ? 3 : 1) : o.queue_order;
  if (order == 2 && !h_cell) return set_error(RK_E_INVALID_ARGUMENT, "queue_order 2 needs h_cell");
  P.subq = 0;
  P.nhot = nullptr;
  if ((order == 2 || order == 3) && h_cell && ncell > 1 && !(o.fixed_h > 0.0) && ncell < (int64_t)INT32_MAX) {
    unsigned* hist = reinterpret_cast<unsigned*>(wsb + 256);
    unsigned* nhot = reinterpret_cast<unsigned*>(wsb + 64);
    unsigned* cursor = reinterpret_cast<unsigned*>(wsb + 512);
    int32_t* perm = reinterpret_cast<int32_t*>(wsb + 768);
    int64_t nblk = (ncell + 4095) / 4096;
    if (nblk > 1024) nblk = 1024;
    const int64_t chunk = (ncell + nblk - 1) / nblk;
    order_count_kernel<<<(unsigned)nblk, ORDER_THREADS, 0, stream>>>(h_cell, ncell, chunk, dt, hist);
    order_scan_kernel<<<1, 32, 0, stream>>>(hist, cursor, nhot);
    order_scatter_kernel<<<(unsigned)nblk, ORDER_THREADS, 0, stream>>>(h_cell, ncell, chunk, dt, cursor, perm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "work-queue ordering launch");
    P.order = perm;
    P.nhot = nhot;
  }
  // timing events: inside a stream capture they become event-record nodes of
  // the graph (external records), so every replay times the kernel
  unsigned ev_flags = 0u;
  if (o.ev_begin || o.ev_end) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamIsCapturing");
    if (cap == cudaStreamCaptureStatusActive) ev_flags = cudaEventRecordExternal;
  }
  if (o.ev_begin) {
    e = cudaEventRecordWithFlags((cudaEvent_t)o.ev_begin, stream, ev_flags);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  }
  IntegrateLaunch la{&P, mech, o.cells_per_block, o.blocks_per_sm, order == 3, ncell, stream};
  if (method == 1) {
    rc = G == 32 ? launch_rkdp<32>(la) : (G == 16 ? launch_rkdp<16>(la) : launch_rkdp<8>(la));
  } else if (G == 32) {
    rc = tc ? launch_rok4e<32, false, true>(la)
            : (mixed ? launch_rok4e<32, true, false>(la) : launch_rok4e<32, false, false>(la));
  } else if (G == 16) {
    rc = mixed ? launch_rok4e<16, true, false>(la) : launch_rok4e<16, false, false>(la);
  } else {
    rc = mixed ? launch_rok4e<8, true, false>(la) : launch_rok4e<8, false, false>(la);
  }
  if (rc) return rc;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "rok4e_integrate_kernel launch");
  if (o.ev_end) {
    e = cudaEventRecordWithFlags((cudaEvent_t)o.ev_end, stream, ev_flags);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  }
  return RK_OK;
}

}  // namespace

extern "C" {

int rk_mech_validate(const rk_mech_desc* desc, char* msg, size_t msg_len) {
  HostMech hm;
  std::string err;
  const bool ok = pack_mechanism(desc, &hm, &err);
  if (msg && msg_len > 0) {
    snprintf(msg, msg_len, "%s", ok ? "" : err.c_str());
  }
  return ok ? RK_OK : set_error(RK_E_MECH_INVALID, err);
}

int rk_mech_load(const rk_mech_desc* desc, rk_mech** out) {
  if (!out) return set_error(RK_E_INVALID_ARGUMENT, "null output handle");
  *out = nullptr;
  rk_mech* m = new rk_mech();
  std::string err;
  if (!pack_mechanism(desc, &m->host, &err)) {
    delete m;
    return set_error(RK_E_MECH_INVALID, err);
  }
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess) e = cudaMalloc(&m->dev, (size_t)m->host.L.bytes);
  if (e == cudaSuccess) e = cudaMemcpy(m->dev, m->host.packed.data(), (size_t)m->host.L.bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (m->dev) cudaFree(m->dev);
    delete m;
    return cuda_error(e, "rk_mech_load");
  }
  *out = m;
  return RK_OK;
}

int rk_mech_free(rk_mech* mech) {
  if (!mech) return RK_OK;
  cudaError_t e = cudaSuccess;
  if (mech->dev) {
    e = cudaDeviceSynchronize();
    cudaFree(mech->dev);
  }
  delete mech;
  return e == cudaSuccess ? RK_OK : cuda_error(e, "rk_mech_free");
}

int rk_mech_info(const rk_mech* mech, int32_t* n_species, int32_t* n_reactions, size_t* device_bytes) {
  if (!mech) return set_error(RK_E_INVALID_ARGUMENT, "null mechanism handle");
  if (n_species) *n_species = mech->host.L.ns;
  if (n_reactions) *n_reactions = mech->host.L.nr;
  if (device_bytes) *device_bytes = (size_t)mech->host.L.bytes;
  return RK_OK;
}

static int point_call(const rk_mech* mech, const double* Y, const double* src, const double* V, double p,
                      double* out, int64_t ncell, int mode, void* stream, const double* rho_cell = nullptr,
                      int nx = 0) {
  int rc = check_mech(mech);
  if (rc) return rc;
  if (ncell < 0) return set_error(RK_E_INVALID_ARGUMENT, "ncell < 0");
  if (ncell == 0) return RK_OK;
  const bool needs_v = mode == 1 || mode == 2 || mode == 4 || mode == 5 || mode == 7 || mode == 8;
  const bool tc = mode == 6 || mode == 7;
  if (!Y || !out || (needs_v && !V)) return set_error(RK_E_INVALID_ARGUMENT, "null array");
  if (out == Y) return set_error(RK_E_INVALID_ARGUMENT, "output must not alias the state");
  if (!rho_cell && !(p > 0.0)) return set_error(RK_E_INVALID_ARGUMENT, "pressure must be > 0");
  PointParams P;
  P.rho_cell = rho_cell;
  P.nx = nx;
  P.mech = mech->dev;
  P.L = mech->host.L;
  P.S = make_slot(mech->host.L, 1, mode >= 3 && mode <= 5, nx, mode == 5, tc, mode == 8);
  P.Y = Y;
  P.src = src;
  P.V = V;
  P.out = out;
  P.ncell = ncell;
  P.p = p;
  P.mode = mode;
  {
    const MechLayout& L = mech->host.L;  // everything but the nu^T tiles; the tiles only with the FP64 arrays
    P.mech_copy = tc ? L.bytes_fp64 : L.off_nuT;
    P.tc_bytes = tc ? (int64_t)16 * 32 * L.nst * L.nrt : 0;
  }
  LaunchPlan plan;
  rc = plan_for<32>(chem_point_kernel<32>, mech, P.S, 8, ncell, false, &plan, 0, false, P.mech_copy + P.tc_bytes);
  if (rc) return rc;
  chem_point_kernel<32><<<plan.blocks, plan.cells_per_block * 32, plan.smem, (cudaStream_t)stream>>>(P);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RK_OK : cuda_error(e, "chem_point_kernel launch");
}

int rk_chem_rhs(const rk_mech* mech, const double* Y, const double* src, double p, double* dYdt, int64_t ncell,
                void* stream) {
  return point_call(mech, Y, src, nullptr, p, dYdt, ncell, 0, stream);
}

int rk_chem_jvp(const rk_mech* mech, const double* Y, const double* V, double p, double* JV, int64_t ncell,
                int32_t mode, void* stream) {
  if (mode < 0 || mode > 5) return set_error(RK_E_INVALID_ARGUMENT, "mode must be 0..5");
  static const int point_mode[6] = {1, 2, 4, 5, 7, 8};
  return point_call(mech, Y, nullptr, V, p, JV, ncell, point_mode[mode], stream);
}

int rk_chem_rhs_tc(const rk_mech* mech, const double* Y, const double* src, double p, double* dYdt,
                   int64_t ncell, void* stream) {
  return point_call(mech, Y, src, nullptr, p, dYdt, ncell, 6, stream);
}

int rk_chem_rhs_mixed(const rk_mech* mech, const double* Y, const double* src, double p, double* dYdt,
                      int64_t ncell, void* stream) {
  return point_call(mech, Y, src, nullptr, p, dYdt, ncell, 3, stream);
}

int rk_chem_rhs_cv(const rk_mech* mech, const double* Y, const double* src, const double* rho_cell, double* dYdt,
                   int64_t ncell, void* stream) {
  if (!rho_cell && ncell > 0) return set_error(RK_E_INVALID_ARGUMENT, "null density array");
  return point_call(mech, Y, src, nullptr, 1.0, dYdt, ncell, 0, stream, rho_cell);
}

int rk_chem_jvp_cv(const rk_mech* mech, const double* Y, const double* V, const double* rho_cell, double* JV,
                   int64_t ncell, int32_t mode, void* stream) {
  if (mode != 0 && mode != 1) return set_error(RK_E_INVALID_ARGUMENT, "mode must be 0 or 1");
  if (!rho_cell && ncell > 0) return set_error(RK_E_INVALID_ARGUMENT, "null density array");
  return point_call(mech, Y, nullptr, V, 1.0, JV, ncell, mode == 0 ? 1 : 2, stream, rho_cell);
}

int rk_chem_rhs_aux(const rk_mech* mech, const double* U, const double* src, double* dUdt, int64_t ncell,
                    void* stream) {
  return point_call(mech, U, src, nullptr, 1.0, dUdt, ncell, 0, stream, nullptr, RK_AUX_EXTRA);
}

int rk_chem_jvp_aux(const rk_mech* mech, const double* U, const double* src, const double* V, double* JV,
                    int64_t ncell, int32_t mode, void* stream) {
  if (mode != 0 && mode != 1) return set_error(RK_E_INVALID_ARGUMENT, "mode must be 0 or 1");
  return point_call(mech, U, src, V, 1.0, JV, ncell, mode == 0 ? 1 : 2, stream, nullptr, RK_AUX_EXTRA);
}

size_t rk_rok4e_workspace_size(const rk_mech* mech, int64_t ncell, int32_t krylov_dim, const rk_opts* opts) {
  (void)mech;
  (void)krylov_dim;
  (void)opts;
  // work-queue counter, order histogram and cursors, and the queue order
  const size_t order = ncell > 0 ? (size_t)ncell * sizeof(int32_t) : 0;
  return 768 + ((order + 255) & ~(size_t)255);
}

int rk_rok4e_integrate(const rk_mech* mech, double* Y, const double* src, double* h_cell, int64_t ncell, double p,
                       double dt, double rtol, double atol, int32_t krylov_dim, const rk_opts* opts,
                       int32_t* stats, void* workspace, size_t workspace_bytes, void* stream) {
  return integrate_impl(mech, Y, src, h_cell, ncell, p, dt, rtol, atol, krylov_dim, opts, stats, workspace,
                        workspace_bytes, (cudaStream_t)stream);
}

int rk_rkdp_integrate(const rk_mech* mech, double* Y, const double* src, double* h_cell, int64_t ncell, double p,
                      double dt, double rtol, double atol, const rk_opts* opts, int32_t* stats, void* workspace,
                      size_t workspace_bytes, void* stream) {
  return integrate_impl(mech, Y, src, h_cell, ncell, p, dt, rtol, atol, 1, opts, stats, workspace, workspace_bytes,
                        (cudaStream_t)stream, 1);
}

size_t rk_simpler_split_step_workspace_size(const rk_mech* mech, int64_t npts, int32_t krylov_dim,
                                            const rk_opts* opts) {
  if (!mech || npts < 0) return 0;
  const size_t n = (size_t)npts * (size_t)(mech->host.L.ns + 1);
  return 256 + 3 * ((n * sizeof(double) + 255) & ~(size_t)255) +
         rk_rok4e_workspace_size(mech, npts, krylov_dim, opts);
}

int rk_diffusion_1d(const double* U, double* TU, int64_t npts, int32_t nvar, double D, double dx, void* stream) {
  if (npts < 0 || nvar < 1) return set_error(RK_E_INVALID_ARGUMENT, "bad sizes");
  if (npts == 0) return RK_OK;
  if (!U || !TU || U == TU) return set_error(RK_E_INVALID_ARGUMENT, "null or aliased array");
  if (!(dx > 0.0)) return set_error(RK_E_INVALID_ARGUMENT, "dx must be > 0");
  const int64_t n = npts * nvar;
  diffusion_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(U, TU, npts, nvar, D,
                                                                                  1.0 / (dx * dx));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RK_OK : cuda_error(e, "diffusion_kernel launch");
}

int rk_diffusion_1d_ghost(const double* Uext, double* TU, int64_t npts, int32_t nvar, double D, double dx,
                          void* stream) {
  if (npts < 0 || nvar < 1) return set_error(RK_E_INVALID_ARGUMENT, "bad sizes");
  if (npts == 0) return RK_OK;
  if (!Uext || !TU) return set_error(RK_E_INVALID_ARGUMENT, "null array");
  if (TU + npts * nvar > Uext && Uext + (npts + 2) * nvar > TU)
    return set_error(RK_E_INVALID_ARGUMENT, "TU must not overlap Uext");
  if (!(dx > 0.0)) return set_error(RK_E_INVALID_ARGUMENT, "dx must be > 0");
  const int64_t n = npts * nvar;
  diffusion_ghost_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(Uext, TU, npts, nvar, D,
                                                                                        1.0 / (dx * dx));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RK_OK : cuda_error(e, "diffusion_ghost_kernel launch");
}

int rk_ssprk3_stage_ghost(int32_t stage, const double* U1, const double* Xext, const double* S, double sigma,
                          double* Out, int64_t npts, int32_t nvar, double D, double dx, double k, void* stream) {
  if (stage < 0 || stage > 2) return set_error(RK_E_INVALID_ARGUMENT, "stage must be 0, 1 or 2");
  if (npts < 0 || nvar < 1) return set_error(RK_E_INVALID_ARGUMENT, "bad sizes");
  if (npts == 0) return RK_OK;
  if (!U1 || !Xext || !Out) return set_error(RK_E_INVALID_ARGUMENT, "null array");
  if (Out + npts * nvar > Xext && Xext + (npts + 2) * nvar > Out)
    return set_error(RK_E_INVALID_ARGUMENT, "Out must not overlap Xext");
  if (!(dx > 0.0)) return set_error(RK_E_INVALID_ARGUMENT, "dx must be > 0");
  const int64_t n = npts * nvar;
  ssprk3_stage_ghost_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      stage, U1, Xext, S, sigma, Out, npts, nvar, D, 1.0 / (dx * dx), k);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RK_OK : cuda_error(e, "ssprk3_stage_ghost_kernel launch");
}

int rk_simpler_split_step(const rk_mech* mech, double* U, double* h_cell, int64_t npts, double p, double dt,
                          double D, double dx, double rtol, double atol, int32_t krylov_dim, const rk_opts* opts,
                          int32_t* stats, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_mech(mech);
  if (rc) return rc;
  if (opts && opts->reactor == 2)
    return set_error(RK_E_INVALID_ARGUMENT, "the auxiliary-temperature system is for rk_rok4e_integrate and rk_rkdp_integrate");
  if (npts < 0) return set_error(RK_E_INVALID_ARGUMENT, "npts < 0");
  if (npts == 0) return RK_OK;
  if (!U) return set_error(RK_E_INVALID_ARGUMENT, "null state array");
  if (!(dx > 0.0) || !(D >= 0.0)) return set_error(RK_E_INVALID_ARGUMENT, "need dx > 0 and D >= 0");
  const size_t need = rk_simpler_split_step_workspace_size(mech, npts, krylov_dim, opts);
  if (!workspace || workspace_bytes < need) return set_error(RK_E_WORKSPACE, "workspace too small");
  const int nv = mech->host.L.ns + 1;
  const int64_t n = npts * nv;
  const size_t vec = ((size_t)n * sizeof(double) + 255) & ~(size_t)255;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* Tn = reinterpret_cast<double*>(ws + 256);
  double* V1 = reinterpret_cast<double*>(ws + 256 + vec);
  double* V2 = reinterpret_cast<double*>(ws + 256 + 2 * vec);
  void* ws_int = ws + 256 + 3 * vec;
  const size_t ws_int_bytes = workspace_bytes - (256 + 3 * vec);
  cudaStream_t st = (cudaStream_t)stream;
  const double inv_dx2 = 1.0 / (dx * dx);
  const unsigned nb = (unsigned)((n + 255) / 256);
  // c_n = -T(U_n)
  diffusion_kernel<<<nb, 256, 0, st>>>(U, Tn, npts, nv, D, inv_dx2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "diffusion_kernel launch");
  // reaction sub-step over dt with the constant source T(U_n)
  rc = integrate_impl(mech, U, Tn, h_cell, npts, p, dt, rtol, atol, krylov_dim, opts, stats, ws_int, ws_int_bytes,
                      st);
  if (rc) return rc;
  // transport correction over dt/2: one SSP-RK3 step of dU/dt = T(U) - T(U_n)
  const double k = 0.5 * dt;
  ssprk3_stage_kernel<<<nb, 256, 0, st>>>(0, U, U, Tn, -1.0, V1, npts, nv, D, inv_dx2, k);
  ssprk3_stage_kernel<<<nb, 256, 0, st>>>(1, U, V1, Tn, -1.0, V2, npts, nv, D, inv_dx2, k);
  ssprk3_stage_kernel<<<nb, 256, 0, st>>>(2, U, V2, Tn, -1.0, U, npts, nv, D, inv_dx2, k);
  e = cudaGetLastError();
  return e == cudaSuccess ? RK_OK : cuda_error(e, "ssprk3_stage_kernel launch");
}

int rk_simpler_split_step_ext(const rk_mech* mech, double* U, double* h_cell, int64_t npts, double p, double dt,
                              double rtol, double atol, int32_t krylov_dim, rk_transport_fn transport, void* user,
                              const rk_opts* opts, int32_t* stats, void* workspace, size_t workspace_bytes,
                              void* stream) {
  int rc = check_mech(mech);
  if (rc) return rc;
  if (opts && opts->reactor == 2)
    return set_error(RK_E_INVALID_ARGUMENT, "the auxiliary-temperature system is for rk_rok4e_integrate and rk_rkdp_integrate");
  if (npts < 0) return set_error(RK_E_INVALID_ARGUMENT, "npts < 0");
  if (npts == 0) return RK_OK;
  if (!U) return set_error(RK_E_INVALID_ARGUMENT, "null state array");
  const size_t need = rk_split_step_workspace_size(mech, npts, krylov_dim, 0, opts);
  if (!workspace || workspace_bytes < need) return set_error(RK_E_WORKSPACE, "workspace too small");
  const int nv = mech->host.L.ns + 1;
  const int64_t n = npts * nv;
  const size_t vec = ((size_t)n * sizeof(double) + 255) & ~(size_t)255;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* Tn = reinterpret_cast<double*>(ws + 256);
  double* V1 = reinterpret_cast<double*>(ws + 256 + vec);
  double* V2 = reinterpret_cast<double*>(ws + 256 + 2 * vec);
  double* TX = reinterpret_cast<double*>(ws + 256 + 3 * vec);
  void* ws_int = ws + 256 + 4 * vec;
  const size_t ws_int_bytes = workspace_bytes - (256 + 4 * vec);
  cudaStream_t st = (cudaStream_t)stream;
  if (!transport)  // no transport: the reaction step alone (the 0-D case)
    return integrate_impl(mech, U, nullptr, h_cell, npts, p, dt, rtol, atol, krylov_dim, opts, stats, ws_int,
                          ws_int_bytes, st);
  auto call = [&](const double* X, double* out) {
    const int r = transport(X, out, npts, nv, user, stream);
    return r == 0 ? RK_OK : set_error(RK_E_CALLBACK, "the transport callback returned " + std::to_string(r));
  };
  // T(U_n), the constant source of the reaction sub-step
  if ((rc = call(U, Tn))) return rc;
  rc = integrate_impl(mech, U, Tn, h_cell, npts, p, dt, rtol, atol, krylov_dim, opts, stats, ws_int, ws_int_bytes,
                      st);
  if (rc) return rc;
  // transport correction over dt/2: one SSP-RK3 step of dU/dt = T(U) - T(U_n)
  const double k = 0.5 * dt;
  const unsigned nb = (unsigned)((n + 255) / 256);
  const double* X[3] = {U, V1, V2};
  double* Out[3] = {V1, V2, U};
  for (int stage = 0; stage < 3; ++stage) {
    if ((rc = call(X[stage], TX))) return rc;
    ssprk3_combine_kernel<<<nb, 256, 0, st>>>(stage, U, X[stage], TX, Tn, -1.0, Out[stage], n, k);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "ssprk3_combine_kernel launch");
  }
  return RK_OK;
}

// One SSP-RK3 step of dU/dt = D d^2U/dx^2 + sigma S over t, in place (V1, V2 scratch).
static int transport_step(double* U, const double* S, double sigma, double t, double D, double dx, int64_t npts,
                          int nv, double* V1, double* V2, cudaStream_t st) {
  const int64_t n = npts * nv;
  const unsigned nb = (unsigned)((n + 255) / 256);
  const double inv_dx2 = 1.0 / (dx * dx);
  ssprk3_stage_kernel<<<nb, 256, 0, st>>>(0, U, U, S, sigma, V1, npts, nv, D, inv_dx2, t);
  ssprk3_stage_kernel<<<nb, 256, 0, st>>>(1, U, V1, S, sigma, V2, npts, nv, D, inv_dx2, t);
  ssprk3_stage_kernel<<<nb, 256, 0, st>>>(2, U, V2, S, sigma, U, npts, nv, D, inv_dx2, t);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RK_OK : cuda_error(e, "ssprk3_stage_kernel launch");
}

size_t rk_split_step_workspace_size(const rk_mech* mech, int64_t npts, int32_t krylov_dim, int32_t scheme,
                                    const rk_opts* opts) {
  if (!mech || npts < 0) return 0;
  (void)scheme;
  const size_t n = (size_t)npts * (size_t)(mech->host.L.ns + 1);
  return 256 + 4 * ((n * sizeof(double) + 255) & ~(size_t)255) +
         rk_rok4e_workspace_size(mech, npts, krylov_dim, opts);
}

int rk_split_step(const rk_mech* mech, double* U, double* h_cell, int64_t npts, double p, double dt, double D,
                  double dx, double rtol, double atol, int32_t krylov_dim, int32_t scheme, const rk_opts* opts,
                  int32_t* stats, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_mech(mech);
  if (rc) return rc;
  if (opts && opts->reactor == 2)
    return set_error(RK_E_INVALID_ARGUMENT, "the auxiliary-temperature system is for rk_rok4e_integrate and rk_rkdp_integrate");
  if (scheme < 0 || scheme > 3) return set_error(RK_E_INVALID_ARGUMENT, "scheme must be 0..3");
  if (npts < 0) return set_error(RK_E_INVALID_ARGUMENT, "npts < 0");
  if (npts == 0) return RK_OK;
  if (!U) return set_error(RK_E_INVALID_ARGUMENT, "null state array");
  if (!(dx > 0.0) || !(D >= 0.0) || !(dt > 0.0)) return set_error(RK_E_INVALID_ARGUMENT, "need dx, dt > 0, D >= 0");
  const size_t need = rk_split_step_workspace_size(mech, npts, krylov_dim, scheme, opts);
  if (!workspace || workspace_bytes < need) return set_error(RK_E_WORKSPACE, "workspace too small");
  const int nv = mech->host.L.ns + 1;
  const int64_t n = npts * nv;
  const size_t vec = ((size_t)n * sizeof(double) + 255) & ~(size_t)255;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* Tn = reinterpret_cast<double*>(ws + 256);
  double* V1 = reinterpret_cast<double*>(ws + 256 + vec);
  double* V2 = reinterpret_cast<double*>(ws + 256 + 2 * vec);
  double* Cn = reinterpret_cast<double*>(ws + 256 + 3 * vec);
  void* ws_int = ws + 256 + 4 * vec;
  const size_t ws_int_bytes = workspace_bytes - (256 + 4 * vec);
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned nb = (unsigned)((n + 255) / 256);
  auto react = [&](const double* src, double t) {
    return integrate_impl(mech, U, src, h_cell, npts, p, t, rtol, atol, krylov_dim, opts, stats, ws_int,
                          ws_int_bytes, st);
  };
  cudaError_t e;
  if (scheme == 0) {  // Simpler: c_n = -T(U_n); R - c_n over dt; T + c_n over dt/2
    diffusion_kernel<<<nb, 256, 0, st>>>(U, Tn, npts, nv, D, 1.0 / (dx * dx));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "diffusion_kernel launch");
    if ((rc = react(Tn, dt))) return rc;
    return transport_step(U, Tn, -1.0, 0.5 * dt, D, dx, npts, nv, V1, V2, st);
  }
  if (scheme == 1) {  // Strang: T over dt/2, R over dt, T over dt/2
    if ((rc = transport_step(U, nullptr, 0.0, 0.5 * dt, D, dx, npts, nv, V1, V2, st))) return rc;
    if ((rc = react(nullptr, dt))) return rc;
    return transport_step(U, nullptr, 0.0, 0.5 * dt, D, dx, npts, nv, V1, V2, st);
  }
  // simple balanced: c_n = (R(U_n) - T(U_n)) / 2; Cn holds -c_n = (T - R) / 2
  if ((rc = point_call(mech, U, nullptr, nullptr, p, Cn, npts, 0, stream))) return rc;
  diffusion_kernel<<<nb, 256, 0, st>>>(U, Tn, npts, nv, D, 1.0 / (dx * dx));
  axpby_kernel<<<nb, 256, 0, st>>>(Cn, Tn, -0.5, 0.5, Cn, n);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "balancing constant launch");
  if (scheme == 2) {  // reaction first: R - c over dt/2, T + c over dt, R - c over dt/2
    if ((rc = react(Cn, 0.5 * dt))) return rc;
    if ((rc = transport_step(U, Cn, -1.0, dt, D, dx, npts, nv, V1, V2, st))) return rc;
    return react(Cn, 0.5 * dt);
  }
  // transport first (Eq. balanced): T + c over dt/2, R - c over dt, T + c over dt/2
  if ((rc = transport_step(U, Cn, -1.0, 0.5 * dt, D, dx, npts, nv, V1, V2, st))) return rc;
  if ((rc = react(Cn, dt))) return rc;
  return transport_step(U, Cn, -1.0, 0.5 * dt, D, dx, npts, nv, V1, V2, st);
}

// ---- allocation-free split step ---------------------------------------------
// Scratch for rk_simpler_split_step_noalloc: a fixed array in device memory that
// every GPU loading this library reserves until the process exits.  Host code
// may not pass the symbol itself to a kernel (on the host it names a host-side
// placeholder), so its device address is looked up with cudaGetSymbolAddress,
// with the device current, and cached per device together with the ID of the
// CUDA context it belongs to.  A later call in another context of that device
// (after cudaDeviceReset, or once the primary context was released and made
// again, when the module -- and the array -- can sit at another address) looks
// the address up again; inside a stream capture it refuses instead, since the
// lookup may have to load the module.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RK_NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mu;
struct NoallocEntry {
  unsigned long long ctx_id;
  void* ptr;
};
static NoallocEntry g_noalloc[256] = {};

typedef CUresult (*PFN_ctx_get_current)(CUcontext*);
typedef CUresult (*PFN_ctx_get_id)(CUcontext, unsigned long long*);

// ID of the calling thread's current CUDA context, through the driver entry
// points the runtime hands out (no link against the driver library).
static int current_ctx_id(unsigned long long* id) {
  static PFN_ctx_get_current get_current = nullptr;
  static PFN_ctx_get_id get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDriverEntryPointByVersion");
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return set_error(RK_E_CUDA, "the driver does not provide cuCtxGetCurrent / cuCtxGetId");
    get_current = reinterpret_cast<PFN_ctx_get_current>(f1);
    get_id = reinterpret_cast<PFN_ctx_get_id>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return set_error(RK_E_CUDA, "no current CUDA context");
  if (get_id(ctx, id) != CUDA_SUCCESS) return set_error(RK_E_CUDA, "cuCtxGetId failed");
  return RK_OK;
}

static int noalloc_scratch(cudaStream_t stream, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return set_error(RK_E_UNSUPPORTED, "device ordinal out of range");
  // also makes the device's context current on this thread (runtime initialisation)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamIsCapturing");
  unsigned long long id = 0;
  int rc = current_ctx_id(&id);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocEntry& ent = g_noalloc[dev];
  if (!ent.ptr || ent.ctx_id != id) {
    if (cap != cudaStreamCaptureStatusNone)
      return set_error(RK_E_UNSUPPORTED,
                       "rk_simpler_split_step_noalloc: the first call in a CUDA context must come before any "
                       "stream capture (it looks up the static scratch's device address)");
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress");
    ent.ptr = ptr;
    ent.ctx_id = id;
  }
  *out = ent.ptr;
  return RK_OK;
}

// Largest npts whose split-step scratch fits the static array (the workspace
// size grows with npts, so bisection finds it exactly).
static int64_t noalloc_max_points(const rk_mech* mech, int32_t krylov_dim, const rk_opts* opts) {
  int64_t lo = 0, hi = (int64_t)RK_NOALLOC_SCRATCH_BYTES;  // need(hi) > the array: > 8 bytes per point
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (rk_simpler_split_step_workspace_size(mech, mid, krylov_dim, opts) <= (size_t)RK_NOALLOC_SCRATCH_BYTES)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

int rk_simpler_split_step_noalloc(const rk_mech* mech, double* U, double* h_cell, int64_t npts, double p, double dt,
                                  double D, double dx, double rtol, double atol, int32_t krylov_dim,
                                  const rk_opts* opts, int32_t* stats, void* stream) {
  int rc = check_mech(mech);
  if (rc) return rc;
  if (opts && opts->reactor == 2)
    return set_error(RK_E_INVALID_ARGUMENT, "the auxiliary-temperature system is for rk_rok4e_integrate and rk_rkdp_integrate");
  if (npts < 0) return set_error(RK_E_INVALID_ARGUMENT, "npts < 0");
  const size_t need = rk_simpler_split_step_workspace_size(mech, npts, krylov_dim, opts);
  if (need > (size_t)RK_NOALLOC_SCRATCH_BYTES) {
    char msg[320];
    snprintf(msg, sizeof(msg),
             "npts = %lld (x %d values) needs %zu bytes of scratch; the static scratch holds %zu bytes, "
             "at most %lld points of this mechanism: use rk_simpler_split_step with a workspace",
             (long long)npts, mech->host.L.ns + 1, need, (size_t)RK_NOALLOC_SCRATCH_BYTES,
             (long long)noalloc_max_points(mech, krylov_dim, opts));
    return set_error(RK_E_UNSUPPORTED, msg);
  }
  void* scratch = nullptr;
  rc = noalloc_scratch((cudaStream_t)stream, &scratch);
  if (rc) return rc;
  return rk_simpler_split_step(mech, U, h_cell, npts, p, dt, D, dx, rtol, atol, krylov_dim, opts, stats, scratch,
                               (size_t)RK_NOALLOC_SCRATCH_BYTES, stream);
}

// ---- fixed-step forward with checkpoints and its discrete adjoint ----------
static AdjLayout make_adj_layout(const MechLayout& L, int M) {
  AdjLayout A;
  A.N = L.ns + 1;
  A.ns = L.ns;
  A.nr = L.nr;
  A.ntb = L.ntb;
  A.M = M;
  const int N = A.N, ns1 = L.ns + 1, nr = L.nr > 0 ? L.nr : 1, ntb = L.ntb > 0 ? L.ntb : 1;
  int r = 0;
  auto take = [&](int n) {
    const int o = r;
    r += n;
    return o;
  };
  A.u = take(N); A.fn = take(N); A.Q = take(M * N); A.K = take(4 * N); A.F = take(4 * N);
  A.arg1 = take(N); A.arg2 = take(N); A.ubar = take(N); A.Kbar = take(4 * N); A.Qbar = take(M * N);
  A.fb2 = take(N); A.fbn = take(N); A.wbar = take(N); A.w = take(N); A.w1 = take(N); A.w2 = take(N);
  A.tmp = take(N); A.H = take(MAXM * MAXM); A.p1 = take(MAXM * MAXM); A.p2 = take(MAXM * MAXM);
  A.hn = take(MAXM); A.Linv = take(MAXM * MAXM); A.zs = take(4 * MAXM); A.ys = take(4 * MAXM);
  A.Lbar = take(MAXM * MAXM); A.Hbar = take(MAXM * MAXM); A.scal = take(8); A.theta = take(nr);
  A.rows_d = r;
  r = 0;
  // the tape (what a forward pass writes and its reverse reads), then the
  // arrays a pass only uses within itself
  A.ud = take(N); A.fd = take(N); A.C = take(ns1); A.cp = take(ns1); A.h = take(ns1); A.dcp = take(ns1);
  A.om = take(ns1); A.k = take(nr); A.rfac = take(nr); A.Ms = take(ntb); A.dlnk = take(ntb); A.dkdM = take(ntb);
  A.omg = take(ntb); A.sc = take(SC_N);
  A.tape_len = r;
  A.g = take(ns1); A.q = take(nr); A.Cbar = take(ns1);
  A.gbar = take(ns1); A.ombar = take(ns1); A.Mbar = take(ntb); A.ubd = take(N); A.fbd = take(N);
  A.Pbb = take(nr); A.drf = take(nr);
  A.tape0 = take((M + 2) * A.tape_len);
  A.rows_D = r;
  return A;
}

size_t rk_rok4e_adjoint_workspace_size(const rk_mech* mech, int64_t ncell, int32_t krylov_dim) {
  if (!mech || ncell < 0 || krylov_dim < 1 || krylov_dim > RK_MAX_KRYLOV) return 0;
  const int N = mech->host.L.ns + 1;
  const AdjLayout A = make_adj_layout(mech->host.L, krylov_dim > N ? N : krylov_dim);
  const size_t nd = (size_t)A.rows_d * (size_t)ncell * sizeof(double);
  return ((nd + 255) & ~(size_t)255) + (size_t)A.rows_D * (size_t)ncell * sizeof(Dual) + 256;
}

int rk_rok4e_fixed_steps(const rk_mech* mech, double* Y, int64_t ncell, double p, double h, int32_t nsteps,
                         int32_t krylov_dim, double* checkpoints, void* workspace, size_t workspace_bytes,
                         void* stream) {
  int rc = check_mech(mech);
  if (rc) return rc;
  if (ncell < 0 || nsteps < 0) return set_error(RK_E_INVALID_ARGUMENT, "ncell and nsteps must be >= 0");
  if (ncell == 0 || nsteps == 0) return RK_OK;
  if (!Y) return set_error(RK_E_INVALID_ARGUMENT, "null state array");
  if (!(h > 0.0)) return set_error(RK_E_INVALID_ARGUMENT, "h must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)ncell * (size_t)(mech->host.L.ns + 1) * sizeof(double);
  rk_opts o;
  memset(&o, 0, sizeof(o));
  o.fixed_h = h;
  for (int n = 0; n < nsteps; ++n) {
    if (checkpoints) {
      cudaError_t e = cudaMemcpyAsync((char*)checkpoints + (size_t)n * bytes, Y, bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync");
    }
    rc = integrate_impl(mech, Y, nullptr, nullptr, ncell, p, h, 1.0, 1.0, krylov_dim, &o, nullptr, workspace,
                        workspace_bytes, st);
    if (rc) return rc;
  }
  if (checkpoints) {
    cudaError_t e = cudaMemcpyAsync((char*)checkpoints + (size_t)nsteps * bytes, Y, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync");
  }
  return RK_OK;
}

int rk_rok4e_adjoint(const rk_mech* mech, const double* checkpoints, const double* ubar, int64_t ncell, double p,
                     double h, int32_t nsteps, int32_t krylov_dim, double* grad_lnA, double* grad_u0,
                     void* workspace, size_t workspace_bytes, void* stream) {
  return rk_rok4e_adjoint_ex(mech, checkpoints, ubar, ncell, p, h, nsteps, krylov_dim, 0, grad_lnA, grad_u0,
                             workspace, workspace_bytes, stream);
}

int rk_rok4e_adjoint_ex(const rk_mech* mech, const double* checkpoints, const double* ubar, int64_t ncell, double p,
                        double h, int32_t nsteps, int32_t krylov_dim, int32_t lanes_per_cell, double* grad_lnA,
                        double* grad_u0, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_mech(mech);
  if (rc) return rc;
  if (ncell < 0 || nsteps < 0) return set_error(RK_E_INVALID_ARGUMENT, "ncell and nsteps must be >= 0");
  if (krylov_dim < 1 || krylov_dim > RK_MAX_KRYLOV) return set_error(RK_E_INVALID_ARGUMENT, "krylov_dim outside 1..8");
  if (!checkpoints || !ubar || !grad_lnA) return set_error(RK_E_INVALID_ARGUMENT, "null array");
  if (!(h > 0.0) || !(p > 0.0)) return set_error(RK_E_INVALID_ARGUMENT, "need h > 0 and p > 0");
  const size_t need = rk_rok4e_adjoint_workspace_size(mech, ncell, krylov_dim);
  if (!workspace || workspace_bytes < need) return set_error(RK_E_WORKSPACE, "adjoint workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = mech->host.L.ns + 1;
  AdjointParams P;
  P.mech = mech->dev;
  P.L = mech->host.L;
  P.A = make_adj_layout(mech->host.L, krylov_dim > N ? N : krylov_dim);
  P.ckpt = checkpoints;
  P.ubar_final = ubar;
  P.grad_u0 = grad_u0;
  P.wsd = static_cast<double*>(workspace);
  const size_t nd = ((size_t)P.A.rows_d * (size_t)ncell * sizeof(double) + 255) & ~(size_t)255;
  P.wsD = reinterpret_cast<Dual*>(static_cast<unsigned char*>(workspace) + nd);
  P.ncell = ncell;
  P.p = p;
  P.h = h;
  P.nsteps = nsteps;
  P.M = krylov_dim > N ? N : krylov_dim;
  const int nr = mech->host.L.nr;
  if (ncell == 0 || nsteps == 0 || nr == 0) {
    cudaError_t e = cudaMemsetAsync(grad_lnA, 0, (size_t)(nr > 0 ? nr : 0) * sizeof(double), st);
    if (e == cudaSuccess && grad_u0 && ncell > 0)
      e = cudaMemcpyAsync(grad_u0, ubar, (size_t)ncell * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? RK_OK : cuda_error(e, "adjoint trivial case");
  }
  int G = lanes_per_cell;
  if (G == 0) {
    // auto: the fewest lanes (the group's scalar work is repeated on each of
    // them) that still give every SM sub-partition a warp; 8 at most
    int n_sm = 0;
    size_t smem_max = 0;
    rc = device_props(&n_sm, &smem_max);
    if (rc) return rc;
    const int64_t want_threads = (int64_t)n_sm * 4 * 32;
    G = 8;
    while (G < 32 && ncell * G < want_threads) G *= 2;
  }
  if (G != 4 && G != 8 && G != 16 && G != 32)
    return set_error(RK_E_INVALID_ARGUMENT, "lanes_per_cell must be 0, 4, 8, 16 or 32");
  const size_t smem = (size_t)mech->host.L.off_nuT + EXP_TAB_BYTES;
  cudaError_t e = cudaSuccess;
  rc = G == 4 ? launch_adjoint<4>(P, smem, st)
              : (G == 8 ? launch_adjoint<8>(P, smem, st)
                        : (G == 16 ? launch_adjoint<16>(P, smem, st) : launch_adjoint<32>(P, smem, st)));
  if (rc) return rc;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "rok4e_adjoint_kernel launch");
  adjoint_reduce_kernel<<<nr, 256, 0, st>>>(P.wsd + P.A.theta, ncell, P.A.rows_d,
                                           reinterpret_cast<const int32_t*>(mech->dev + mech->host.L.off_perm),
                                           grad_lnA);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "adjoint_reduce_kernel launch");
  return RK_OK;
}

int rk_probe_throughput(int32_t kind, double* ops_per_s) {
  if (!ops_per_s || kind < 0 || kind > 8) return set_error(RK_E_INVALID_ARGUMENT, "bad probe arguments");
  int n_sm = 0;
  size_t smem = 0;
  int rc = device_props(&n_sm, &smem);
  if (rc) return rc;
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 64);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc");
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int threads = 512, blocks = n_sm * 4;
  const int iters = kind == 2 ? 2000 : (kind == 0 ? 20000 : (kind == 3 || kind == 8 ? 20000 : 200000));
  double ops = 0.0;
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {  // first launch warms up
    cudaEventRecord(a);
    if (kind == 0) {
      probe_fp64_kernel<<<blocks, threads>>>((double*)buf, iters, 0.999999);
      ops = (double)blocks * threads * iters * 8.0;
    } else if (kind == 1) {
      probe_fp32_kernel<<<blocks, threads>>>((float*)buf, iters, 0.999999f);
      ops = (double)blocks * threads * iters * 8.0;
    } else if (kind == 2) {
      probe_exp_kernel<<<blocks, threads>>>((double*)buf, iters);
      ops = (double)blocks * threads * iters * 4.0;
    } else if (kind == 4 || kind == 5 || kind == 6) {
      // one block per SM: 1 warp (kind 4), 4 warps (5), 4 warps with one lane
      // active each (6; counted per warp instruction)
      const int t = kind == 4 ? 32 : 128;
      probe_fp64_kernel<<<n_sm, t>>>((double*)buf, iters, 0.999999, kind == 6 ? 1 : 32);
      ops = (double)n_sm * t * iters * 8.0 / (kind == 6 ? 32.0 : 1.0);
    } else if (kind == 7) {
      probe_df_kernel<<<2 * n_sm, 512>>>((float*)buf, iters, 0.9999f, 1e-9f);
      ops = (double)2 * n_sm * 512 * iters * 4.0;
    } else if (kind == 8) {
      probe_i2f_kernel<<<blocks, threads>>>((double*)buf, iters);
      ops = (double)blocks * threads * iters * 8.0;
    } else {
      probe_cvt_kernel<<<blocks, threads>>>((double*)buf, iters);
      ops = (double)blocks * threads * iters * 8.0;  // conversions
    }
    cudaEventRecord(b);
    cudaEventSynchronize(b);
  }
  e = cudaGetLastError();
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_error(e, "probe launch");
  *ops_per_s = ops / (ms * 1e-3);
  return RK_OK;
}

int rk_eval_exp(const double* x, double* y, int64_t n, int32_t which, void* stream) {
  if (n < 0 || which < 0 || which > 7) return set_error(RK_E_INVALID_ARGUMENT, "bad exp arguments");
  if (n == 0) return RK_OK;
  if (!x || !y) return set_error(RK_E_INVALID_ARGUMENT, "null array");
  exp_eval_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n, which);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RK_OK : cuda_error(e, "exp_eval_kernel launch");
}

const char* rk_status_string(int32_t code) {
  switch (code) {
    case RK_OK: return "ok";
    case RK_E_INVALID_ARGUMENT: return "invalid argument";
    case RK_E_MECH_INVALID: return "mechanism invalid";
    case RK_E_CUDA: return "CUDA error";
    case RK_E_UNSUPPORTED: return "unsupported size";
    case RK_E_WORKSPACE: return "workspace missing or too small";
    case RK_E_CALLBACK: return "a caller's callback failed";
    default: return "unknown status";
  }
}

int rk_last_error(char* buf, size_t len) {
  if (buf && len > 0) snprintf(buf, len, "%s", g_last_error.c_str());
  return RK_OK;
}

}  // extern "C"
