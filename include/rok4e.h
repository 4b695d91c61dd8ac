/*
 * rok4e.h -- C ABI of the GB300 ROK4E / Simpler-splitting library.
 *
 * The library integrates the reaction operator of a reacting-flow solver cell
 * by cell with ROK4E, the four-stage, fourth-order Rosenbrock-Krylov scheme of
 * Wu, Ma & Ihme, "Efficient time stepping for reactive turbulent simulations
 * with stiff chemistry" (arXiv:1712.00953), Sec. 4 and Algorithm 1, inside the
 * Simpler balanced splitting step of Sec. 3.4 (Eq. simpler_balanced).
 *
 * Conventions shared by every call:
 *  - State rows.  A cell state is u = (Y_1 .. Y_Ns, T): Ns mass fractions and
 *    the temperature in K, N = Ns + 1 doubles, rows contiguous (row-major
 *    [ncell x N]).  Pressure p is in Pa and constant during a call (the cells
 *    are constant-pressure adiabatic reactors; the paper's Eq. cv_reactor uses
 *    the constant-volume form of the same source term).
 *  - Memory.  Arrays passed to compute calls are DEVICE pointers owned by the
 *    caller unless stated otherwise; only the mechanism handle is owned by the
 *    library.  Compute calls never allocate: scratch comes from the caller's
 *    workspace argument (size from the matching *_workspace_size call).
 *  - Streams.  `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *    default stream.  Compute calls are asynchronous and stream-ordered; a
 *    return value of 0 means the launch was issued.
 *  - Errors.  Calls return RK_OK (0) or a negative RK_E_* code and never throw.
 *    rk_status_string() names a code; rk_last_error() returns a message for
 *    the most recent failure on the calling thread.  Per-cell integration
 *    failures (attempt cap, step-size underflow) do not fail the call: they
 *    are reported in the per-cell statistics.
 */
#ifndef ROK4E_H
#define ROK4E_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes --------------------------------------------------------- */
#define RK_OK 0
#define RK_E_INVALID_ARGUMENT (-1)  /* null pointer, bad size or option          */
#define RK_E_MECH_INVALID (-2)      /* mechanism failed validation              */
#define RK_E_CUDA (-3)              /* a CUDA runtime call failed               */
#define RK_E_UNSUPPORTED (-4)       /* size beyond what the kernels support     */
#define RK_E_WORKSPACE (-5)         /* workspace missing or too small           */
#define RK_E_CALLBACK (-6)          /* a caller-supplied callback returned nonzero */

/* ---- per-cell status codes (stats[4*cell + 3]) ---------------------------- */
#define RK_CELL_OK 0
#define RK_CELL_MAX_ATTEMPTS 1      /* attempt cap reached before t_end          */
#define RK_CELL_NONFINITE 2         /* an accepted state was not finite          */
#define RK_CELL_STEP_UNDERFLOW 3    /* h fell below 1e-12 dt after rejections    */

/* Limits of this build. */
#define RK_MAX_SPECIES 254          /* species indices are packed in 8 bits     */
#define RK_MAX_KRYLOV 8             /* largest Krylov dimension M               */

/* ---- mechanism -------------------------------------------------------------
 * Description of a gas-phase mechanism (host pointers, read during the call).
 * Thermodynamics: NASA-7 polynomials.  Kinetics: kf = A T^b exp(-Ea/(R T));
 * reversible reactions use kr = kf / Kc with Kc from the species Gibbs
 * functions (standard pressure 101325 Pa); third-body reactions multiply the
 * rate by [M] = sum_k eff_k C_k; Troe falloff reactions use
 * k = k_inf Pr/(1+Pr) F with Pr = k0 [M] / k_inf and the Troe form of F.
 * The paper delegates these kinetics to Cantera (Sec. 4.4); the library
 * implements the textbook forms.
 *
 *  elem        int32[Ns*4]   atom counts of C, H, O, N per species
 *  W           f64[Ns]       molar masses, kg/mol (> 0)
 *  nasa        f64[Ns*17]    T_lo, T_mid, T_hi, low-range a1..a7, high-range a1..a7
 *  rxn_sp      int32[Nr*4]   slots 0,1: reactant species, slots 2,3: product
 *                            species, -1 = empty slot
 *  rxn_nu      int32[Nr*4]   signed stoichiometric coefficients of the slots
 *                            (reactants < 0, products > 0); at most two
 *                            molecules per side
 *  arrh        f64[Nr*3]     A (cm, mol, s units), b, Ea (J/mol); for a Troe
 *                            reaction the high-pressure limit
 *  reversible  uint8[Nr]     1 = reversible
 *  kind        int32[Nr]     0 elementary, 1 third body (+M), 2 Troe falloff (+M)
 *  eff         f64[Nr*Ns]    third-body efficiencies (read for kind 1 and 2)
 *  falloff     f64[Nr*7]     A0 (cm, mol, s), b0, Ea0 (J/mol), a, T***, T*, T**
 *                            (T** <= 0 omits that term); read for kind 2
 */
typedef struct rk_mech_desc {
  int32_t n_species;
  int32_t n_reactions;
  const int32_t* elem;
  const double* W;
  const double* nasa;
  const int32_t* rxn_sp;
  const int32_t* rxn_nu;
  const double* arrh;
  const uint8_t* reversible;
  const int32_t* kind;
  const double* eff;
  const double* falloff;
} rk_mech_desc;

typedef struct rk_mech rk_mech; /* opaque, library-owned, immutable after load */

/* Validate a description on the host only (no GPU needed): index ranges,
 * signs, at most two molecules per side, integer element balance
 * sum_k nu_kj a_ek = 0 for every reaction and element, positive W and A,
 * Troe parameters, NASA-7 ranges and continuity of cp, h and s at T_mid
 * (relative 1e-3).  Returns RK_OK or RK_E_MECH_INVALID and writes a message
 * into msg (may be NULL). */
int rk_mech_validate(const rk_mech_desc* desc, char* msg, size_t msg_len);

/* Validate, pack and upload a mechanism to the current CUDA device.  *out
 * receives a handle owned by the library; free it with rk_mech_free.  The
 * handle may be used from any stream of that device. */
int rk_mech_load(const rk_mech_desc* desc, rk_mech** out);

/* Release a handle (NULL is accepted).  Synchronises the device. */
int rk_mech_free(rk_mech* mech);

/* Sizes of a loaded mechanism (any output pointer may be NULL). */
int rk_mech_info(const rk_mech* mech, int32_t* n_species, int32_t* n_reactions,
                 size_t* device_bytes);

/* ---- chemistry source term ---------------------------------------------------
 * dYdt[c] = f(Y[c]) + src[c] for every cell c, with f the constant-pressure
 * reactor source: dY_k/dt = W_k w_k / rho, dT/dt = -sum_k h_k w_k / (rho c_p),
 * w = nu^T q the net molar production rates (Eq. cv_reactor read at constant
 * pressure).  Y, src, dYdt: device [ncell x N]; src may be NULL (zero source).
 * dYdt must not alias Y. */
int rk_chem_rhs(const rk_mech* mech, const double* Y, const double* src, double p,
                double* dYdt, int64_t ncell, void* stream);

/* Jacobian-vector products JV[c] = J(Y[c]) V[c].  mode 0: analytic (exact
 * derivative of rk_chem_rhs); mode 1: forward difference
 * (f(u + d v) - f(u)) / d with d = sqrt(eps) (1 + ||u||_2) / ||v||_2, as in
 * the matrix-free products of Sec. 4.3; mode 2: the analytic product
 * evaluated in FP32 (precision level 2's J v); mode 3: the analytic product
 * with its reaction-level core in double-float (precision level 3); mode 4:
 * the analytic product with nu^T dq formed on the tensor cores as in
 * rk_chem_rhs_tc (precision level 4); mode 5: the analytic product in FP32
 * arithmetic on the FP32 copies of its caches that the caching right-hand
 * side writes at precision level 6 (that level's J v).  Each mode computes
 * exactly what the integrator's J v at that level computes.  All arrays
 * device [ncell x N]; RK_E_INVALID_ARGUMENT for a mode outside 0..5. */
int rk_chem_jvp(const rk_mech* mech, const double* Y, const double* V, double p, double* JV,
                int64_t ncell, int32_t mode, void* stream);

/* Constant-volume source term and Jacobian-vector products (Eq. cv_reactor):
 * cell c has the fixed density rho_cell[c] (device [ncell], kg/m^3);
 * dY_k/dt = W_k w_k / rho, dT/dt = -sum_k u_k w_k / (rho c_v) with the molar
 * internal energies u_k = h_k - R T and c_v = sum_k Y_k (c_p,k - R) / W_k.
 * (The printed equation pairs h_k with c_v; a closed rigid adiabatic cell
 * conserves internal energy, which is what the u_k form expresses.)  mode as
 * in rk_chem_jvp (0 analytic, 1 finite difference). */
int rk_chem_rhs_cv(const rk_mech* mech, const double* Y, const double* src, const double* rho_cell,
                   double* dYdt, int64_t ncell, void* stream);
int rk_chem_jvp_cv(const rk_mech* mech, const double* Y, const double* V, const double* rho_cell,
                   double* JV, int64_t ncell, int32_t mode, void* stream);

/* Mixed-precision source term (the right-hand side of precision levels 1 and
 * 2): as rk_chem_rhs, with w = nu^T q gathered on the FP32 pipe in
 * double-float (FP32 pairs, ~44-bit significands; the small-integer net
 * coefficients are exact in FP32) and the rate-coefficient exponentials'
 * polynomial tails in FP32 (~1e-13 relative), while the Gibbs factors, 1/Kc, the
 * rates of progress q = m (k prod C - k/Kc prod C) and the assembly of f stay
 * FP64.  Needs |q_j| below the FP32 range (3.4e38 mol/m^3/s); rates below
 * 1.2e-38 drop out of w. */
int rk_chem_rhs_mixed(const rk_mech* mech, const double* Y, const double* src, double p,
                      double* dYdt, int64_t ncell, void* stream);

/* Tensor-core source term (the right-hand side of precision level 4): as
 * rk_chem_rhs, with w = nu^T q formed by BF16 mma.  Each cell's rates q_j are
 * cut, relative to a power of two 2^Es above the cell's largest |q_j|, into
 * seven signed 8-bit digits (all of q_j above 2^(Es - 56)); the net
 * coefficients (small integers) and the digits are exact in BF16, every
 * product and every FP32 accumulation of the mma is exact, and FP64 adds the
 * seven scaled digit sums of each species.  So w_k carries no error beyond
 * the dropped tails, at most 2^-55 of the cell's largest rate per reaction,
 * and the six FP64 additions.  A cell whose rates are all below 2^-920
 * gathers in FP64 instead.  Every other step as in rk_chem_rhs. */
int rk_chem_rhs_tc(const rk_mech* mech, const double* Y, const double* src, double p,
                   double* dYdt, int64_t ncell, void* stream);

/* ---- ROK4E integration (Sec. 4, Algorithm 1) ---------------------------------
 * Options; pass NULL for defaults (all zero fields mean "default"). */
typedef struct rk_opts {
  int32_t jv_mode;        /* 0 analytic Jacobian-vector products (default), 1 finite difference */
  int32_t max_attempts;   /* per-cell cap on attempted steps; <= 0: 100000 */
  int32_t lanes_per_cell; /* 0 auto; 8, 16 or 32 lanes of a warp share one cell */
  int32_t cells_per_block;/* 0 auto: as many as shared memory allows, at most
                             256 threads per block (8 cells of 32 lanes) */
  double h0;              /* first step when h_cell is NULL or holds <= 0; <= 0: dt */
  double fixed_h;         /* > 0: fixed steps of this size, no error control */
  int32_t trace_cap;      /* attempts recorded per cell into trace (0: none) */
  int32_t precision;      /* 0: FP64 throughout (default).  Every level keeps in
                             FP64 the equilibrium-constant exponentials, 1/Kc,
                             the rates of progress (forward minus reverse), the
                             stage solves, the error norm and the state update,
                             and meets the library's bar against the FP64
                             oracle (1e-8 + 1e-6 |Y|, 1e-6 K).
                             1: w = nu^T q (in the right-hand side and the
                             Jacobian-vector product) gathered in double-float
                             on the FP32 pipe, the first Gram-Schmidt pass of
                             Arnoldi with FP32 inner products (the
                             reorthogonalisation pass and the norms FP64), the
                             rate-coefficient exponentials' polynomial tails in
                             FP32 (~1e-13 relative).
                             2: as 1 with the Jacobian-vector products in FP32
                             (~1e-5 relative; the Krylov basis tolerates it).
                             3: FP64 Arnoldi; the rate-coefficient exponentials'
                             polynomial tails in FP32; the Jacobian-vector
                             product's reaction-level core (d(C_a C_b), dq,
                             nu^T dq) in double-float on the FP32 pipe.
                             4: FP64 throughout except w = nu^T q (in the
                             right-hand side and the Jacobian-vector product),
                             which is formed on the tensor cores as in
                             rk_chem_rhs_tc; needs lanes_per_cell 0 or 32.
                             5: FP64 throughout except the rate-coefficient
                             exponentials' polynomial tails (FP32): the FP64
                             kernel's layout and occupancy, three FP64
                             instructions fewer per reaction and evaluation.
                             6: as 5 with the Jacobian-vector products in FP32
                             arithmetic on FP32 copies of their caches, which
                             the caching right-hand side writes into the FP64
                             caches' own storage (the FP64 kernel's occupancy;
                             ~1e-6 relative J v) */
  double* trace;          /* device [ncell x trace_cap]: +h accepted, -h rejected, 0 unused */
  void* ev_begin;         /* optional cudaEvent_t recorded on the stream right before the */
  void* ev_end;           /* integration kernel and right after it (timing hook), or NULL;
                             inside a stream capture they are recorded as external
                             event-record nodes, so each replay of the graph records them */
  int32_t queue_order;    /* 0 auto (1 without h_cell, 3 with it), 1 interleaved cell
                             index, 2 longest expected first (dt / h_cell), 3 static
                             balanced bins: the longest-first queue dealt in snake
                             order over (block, warp group) bins, one block per
                             resident slot on every SM, the few cells within a
                             factor 4 of the most expensive each alone on a block
                             (interleaved order without h_cell) */
  int32_t blocks_per_sm;  /* resident blocks per SM for the persistent launch; 0: all
                             that fit */
  int32_t reactor;        /* 0 constant pressure (p, default); 1 constant volume: each
                             cell keeps the density rho_cell[c] (kg/m^3) and the
                             temperature equation uses internal energies and c_v
                             (Eq. cv_reactor); p is then unused.  2 conservative
                             variables with an auxiliary temperature (Eq.
                             chemical_source_balanced, see rk_chem_rhs_aux): rows of
                             N = n_species + 1 + RK_AUX_EXTRA values; FP64 only, and
                             only for rk_rok4e_integrate / rk_rkdp_integrate */
  int32_t reserved1;
  const double* rho_cell; /* device [ncell], read when reactor == 1 */
} rk_opts;

/* ---- Auxiliary-temperature reaction system (compressible coupling) ----------
 * Eq. chemical_source_balanced: the reaction sub-step of a compressible solver
 * integrates the conservative variables with a constant balancing term T_n and
 * an auxiliary temperature used only for thermochemistry,
 *   d/dt [U; T] = [R(U, T) + T_n; w_T],
 *   w_T = (-sum_k e_k d(rho Y_k)/dt + |v|^2/2 d(rho)/dt - v . d(rho v)/dt
 *          + d(rho E)/dt) / (rho c_v)                     (Eq. aux_t_equation)
 * with the specific internal energies e_k = h_k - R T / W_k (the printed
 * equation writes h_k; the energy identity rho E = sum_k rho Y_k e_k +
 * rho |v|^2 / 2 that the equation differentiates needs e_k).  The chemical
 * source R is W_k w_k in the species components and zero in mass, momentum
 * and total energy.  Row layout (SI): [rho Y_1 .. rho Y_Ns, T, rho,
 * rho v_x, rho v_y, rho v_z, rho E], N = Ns + 1 + RK_AUX_EXTRA; concentrations
 * are (rho Y_k) / W_k. */
#define RK_AUX_EXTRA 5

/* dU/dt of the auxiliary-temperature system for ncell rows (device arrays
 * [ncell x N], src = the balancing constants T_n or NULL; out must not alias
 * U).  rk_chem_jvp_aux: J V at U with the same src (mode 0 analytic, 1 forward
 * difference as in rk_chem_jvp). */
int rk_chem_rhs_aux(const rk_mech* mech, const double* U, const double* src, double* dUdt, int64_t ncell,
                    void* stream);
int rk_chem_jvp_aux(const rk_mech* mech, const double* U, const double* src, const double* V, double* JV,
                    int64_t ncell, int32_t mode, void* stream);

/* Bytes of workspace rk_rok4e_integrate needs: a work-queue counter, a
 * histogram and the queue order (768 bytes + 4 bytes per cell, rounded). */
size_t rk_rok4e_workspace_size(const rk_mech* mech, int64_t ncell, int32_t krylov_dim,
                               const rk_opts* opts);

/* Integrate every cell over [0, dt] with ROK4E and adaptive PI step control
 * (Algorithm 1):
 *   Arnoldi on K_M(J_n, f_n) gives Q_n, H_n (Sec. 4.1); each stage solves the
 *   transformed form (Eq. s_stage_row_transformed) with the low-rank inverse
 *   (Eq. solve_kry_jac); the embedded order-3 solution gives the error
 *   err = sqrt(mean(((u^ - u*)/(atol + rtol |u*|))^2)); the PI controller
 *   h* = h min(5, max(0.2, 0.8 err_n^0.1 / err*^0.175)) (Sec. 4.3) sets the
 *   next step; steps are clipped to the end of the interval.
 *  Y         device [ncell x N], in: u(0), out: u(dt)
 *  src       device [ncell x N] constant source added to f (the balancing
 *            constant -c_n = T(U_n) of Simpler splitting), or NULL
 *  h_cell    device [ncell] in/out: first step (<= 0: opts->h0 / dt) and, on
 *            return, the proposed next step; or NULL
 *  krylov_dim  M in 1..8 (clamped to N); M >= 4 keeps order 4
 *  stats     device int32 [ncell x 4]: accepted steps, rejected steps, RHS
 *            evaluations, status (RK_CELL_*); or NULL
 *  workspace device memory of rk_rok4e_workspace_size bytes
 * Cells are independent; one persistent launch processes them from a shared
 * work queue (opts->queue_order).  By default, when h_cell is given and steps
 * are adaptive, cells are sorted longest-expected-first (expected substeps
 * dt/h_cell, binned on a quarter-octave log scale) and dealt to fixed
 * per-block bins; otherwise the queue interleaves the cell index so that
 * neighbouring cells spread over the SMs.  The order changes only the
 * schedule: each cell's result is the same bits either way.
 * Returns RK_E_INVALID_ARGUMENT for null arrays, ncell < 0, dt <= 0, bad
 * tolerances or options; RK_E_WORKSPACE for a missing or short workspace;
 * RK_E_UNSUPPORTED when the mechanism and one cell's work arrays do not fit in
 * an SM's shared memory; RK_E_CUDA when a launch fails.  ncell = 0 is a no-op. */
int rk_rok4e_integrate(const rk_mech* mech, double* Y, const double* src, double* h_cell,
                       int64_t ncell, double p, double dt, double rtol, double atol,
                       int32_t krylov_dim, const rk_opts* opts, int32_t* stats, void* workspace,
                       size_t workspace_bytes, void* stream);

/* Integrate every cell over [0, dt] with the explicit Dormand-Prince 5(4) pair,
 * the explicit reference method of the efficiency comparison (Sec. 4.4; the
 * paper's RKDP of order 5): seven stages, the 5th-order solution propagated,
 * the embedded 4th-order one for the error, first-same-as-last (6 RHS per
 * attempt).  Error norm as in rk_rok4e_integrate; step control
 * h* = h min(5, max(0.2, 0.9 err^(-1/5))).  Arguments, opts, stats, the work
 * queue and the workspace (rk_rok4e_workspace_size with krylov_dim 1) are
 * those of rk_rok4e_integrate; opts->precision must be 0 and jv_mode is
 * ignored.  Returns RK_E_INVALID_ARGUMENT on bad arguments. */
int rk_rkdp_integrate(const rk_mech* mech, double* Y, const double* src, double* h_cell, int64_t ncell,
                      double p, double dt, double rtol, double atol, const rk_opts* opts,
                      int32_t* stats, void* workspace, size_t workspace_bytes, void* stream);

/* ---- Simpler balanced splitting of a 1-D reaction-diffusion system -----------
 * One step of Eq. simpler_balanced on a uniform 1-D grid of npts cells with
 * transport T(U) = D d^2U/dx^2 applied to every state component (constant
 * diffusivity, unit Lewis number; second-order central differences with
 * zero-gradient ends):
 *   c_n = -T(U_n);
 *   reaction:  dU/dt = R(U) - c_n over dt from U_n   (ROK4E, per cell);
 *   transport: dU/dt = T(U) + c_n over dt/2           (one SSP-RK3 step).
 *  U       device [npts x N] in/out;  h_cell as in rk_rok4e_integrate.
 *  stats   as in rk_rok4e_integrate (reaction sub-step), or NULL.
 *  D, dx   diffusivity (m^2/s, >= 0) and grid spacing (m, > 0).
 * Workspace from rk_simpler_split_step_workspace_size; error codes as for
 * rk_rok4e_integrate. */
size_t rk_simpler_split_step_workspace_size(const rk_mech* mech, int64_t npts,
                                            int32_t krylov_dim, const rk_opts* opts);
int rk_simpler_split_step(const rk_mech* mech, double* U, double* h_cell, int64_t npts, double p,
                          double dt, double D, double dx, double rtol, double atol,
                          int32_t krylov_dim, const rk_opts* opts, int32_t* stats,
                          void* workspace, size_t workspace_bytes, void* stream);

/* A caller-supplied transport operator for rk_simpler_split_step_ext: writes
 * TU = T(U) for one field (both device [npts x nvar], row-major; TU never
 * aliases U), enqueuing its work on `stream` (the cudaStream_t the split step
 * was given) and returning 0, or nonzero to stop the step.  It is called on
 * the calling host thread, in stream order with the library's own launches;
 * `user` is passed through unchanged. */
typedef int (*rk_transport_fn)(const double* U, double* TU, int64_t npts, int32_t nvar, void* user,
                               void* stream);

/* Simpler balanced split step (Eq. simpler_balanced) with the caller's own
 * transport operator T, for a grid or a transport model the built-in 1-D
 * diffusion does not cover:
 *   Tn = T(U_n) (one call);
 *   reaction:  dU/dt = R(U) + Tn over dt from U_n   (ROK4E per cell, as
 *              rk_rok4e_integrate with src = Tn);
 *   transport: dU/dt = T(U) - Tn over dt/2          (one SSP-RK3 step: three
 *              calls, on the post-reaction state and the two stage values).
 * transport NULL: the reaction step alone over dt (the 0-D case, src = 0).
 * The npts cells of U are the grid's points in whatever order the operator
 * uses.  U, h_cell, stats, opts as in rk_simpler_split_step; workspace from
 * rk_split_step_workspace_size (any scheme).  With an operator that computes
 * the built-in diffusion the result is bitwise that of rk_simpler_split_step.
 * Returns RK_E_CALLBACK (the step stops where the callback failed, U then
 * partly updated) when the operator returns nonzero, else as
 * rk_simpler_split_step. */
int rk_simpler_split_step_ext(const rk_mech* mech, double* U, double* h_cell, int64_t npts, double p,
                              double dt, double rtol, double atol, int32_t krylov_dim,
                              rk_transport_fn transport, void* user, const rk_opts* opts, int32_t* stats,
                              void* workspace, size_t workspace_bytes, void* stream);

/* Allocation-free variant of rk_simpler_split_step (the paper has no
 * counterpart: this is a library convenience).  Some callers cannot allocate
 * device memory when they take a step -- a solver whose memory pools are
 * fixed before the time loop starts, a host code with no CUDA allocator of its
 * own, or a loop that must not allocate for timing reasons -- so this entry
 * point takes no workspace and calls no cudaMalloc, cudaFree or allocating
 * library routine.  Its scratch (the transport term T(U_n), two SSP-RK3 stage
 * buffers and the work-queue counter) lives in one static device array of
 * RK_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until the
 * process exits.  The call needs rk_simpler_split_step_workspace_size(mech,
 * npts, ...) <= RK_NOALLOC_SCRATCH_BYTES, about 24 (n_species + 1) + 4 bytes
 * per point: at most 5,605 points of a 30-species mechanism (2048 use 1.53 MB)
 * or 3,225 of a 53-species one.  Beyond that it launches nothing and returns
 * RK_E_UNSUPPORTED, with the largest npts that fits this mechanism in
 * rk_last_error.
 *  - The array's device address is looked up with the device current and
 *    cached per device with the ID of its CUDA context.  The first call in a
 *    context -- on each device, and again after cudaDeviceReset or after the
 *    primary context was released and created anew -- does this lookup; make
 *    it before any stream capture (inside a capture such a call returns
 *    RK_E_UNSUPPORTED instead).
 *  - Every call on a device shares the one array and finds the previous call's
 *    contents there (the parts that must start from zero are cleared by the
 *    call).  Calls that overlap on the GPU -- on different streams, or from
 *    several host threads -- race on it: order them on one stream.
 * Arguments and results are those of rk_simpler_split_step. */
#define RK_NOALLOC_SCRATCH_BYTES (4u << 20)
int rk_simpler_split_step_noalloc(const rk_mech* mech, double* U, double* h_cell, int64_t npts, double p,
                                  double dt, double D, double dx, double rtol, double atol,
                                  int32_t krylov_dim, const rk_opts* opts, int32_t* stats, void* stream);

/* Any of the splittings of Sec. 3 on the same 1-D system (one step, in place):
 *  scheme 0  Simpler balanced (Eq. simpler_balanced) -- as rk_simpler_split_step
 *  scheme 1  Strang (Sec. 3.1): T over dt/2, R over dt, T over dt/2
 *  scheme 2  simple balanced, c_n = (R(U_n) - T(U_n))/2 (Sec. 3.3), reaction
 *            first as in the paper's PSR tests: R - c over dt/2, T + c over dt,
 *            R - c over dt/2
 *  scheme 3  simple balanced, transport first (Eq. balanced): T + c over dt/2,
 *            R - c over dt, T + c over dt/2
 * Transport sub-steps are one SSP-RK3 step of their length; reaction sub-steps
 * are rk_rok4e_integrate with the step's constant source, h_cell carrying over
 * between them.  Workspace: rk_split_step_workspace_size. */
size_t rk_split_step_workspace_size(const rk_mech* mech, int64_t npts, int32_t krylov_dim, int32_t scheme,
                                    const rk_opts* opts);
int rk_split_step(const rk_mech* mech, double* U, double* h_cell, int64_t npts, double p, double dt,
                  double D, double dx, double rtol, double atol, int32_t krylov_dim, int32_t scheme,
                  const rk_opts* opts, int32_t* stats, void* workspace, size_t workspace_bytes,
                  void* stream);

/* Transport operator alone: TU = D d^2U/dx^2 (same discretisation). */
int rk_diffusion_1d(const double* U, double* TU, int64_t npts, int32_t nvar, double D, double dx,
                    void* stream);

/* The transport of one slice of the 1-D domain, for a domain split over ranks
 * (the paper's 3-D runs decompose the domain over processes, Sec. 5; the
 * transport's three-point stencil needs one neighbour point per side).  The
 * slice's npts points are held with one ghost row on each side: Uext / Xext
 * are device [(npts + 2) x nvar], row r + 1 holding the slice's point r, row 0
 * and row npts + 1 the neighbouring slices' end points -- or, at an end of
 * the whole domain, a copy of the slice's own end point, which is the
 * zero-gradient boundary.  With the ghost rows filled so, both calls give the
 * same bits at every point as rk_diffusion_1d and the SSP-RK3 stages inside
 * rk_simpler_split_step on the whole domain.
 *  rk_diffusion_1d_ghost: TU [npts x nvar] = D d^2U/dx^2; TU must not overlap
 *    Uext.
 *  rk_ssprk3_stage_ghost: one stage of the SSP-RK3 step (Shu-Osher form) of
 *    dU/dt = D d^2U/dx^2 + sigma S over k: stage 0 Out = X + k g(X); stage 1
 *    Out = 3/4 U1 + 1/4 (X + k g(X)); stage 2 Out = 1/3 U1 + 2/3 (X + k g(X)),
 *    g(X) = D d^2X/dx^2 + sigma S, X from Xext; U1, S (nullable) and Out are
 *    [npts x nvar]; Out may be U1, not Xext.  The Simpler correction of
 *    Eq. simpler_balanced is sigma = -1, S = T(U_n), k = dt / 2.
 * Returns RK_E_INVALID_ARGUMENT for bad sizes, a null array, an overlap or
 * dx <= 0 (nothing launched), RK_E_CUDA if the launch fails. */
int rk_diffusion_1d_ghost(const double* Uext, double* TU, int64_t npts, int32_t nvar, double D, double dx,
                          void* stream);
int rk_ssprk3_stage_ghost(int32_t stage, const double* U1, const double* Xext, const double* S, double sigma,
                          double* Out, int64_t npts, int32_t nvar, double D, double dx, double k, void* stream);

/* ---- fixed-step integration with checkpoints and its adjoint ----------------
 * nsteps fixed ROK4E steps of size h (Algorithm 1 with h held fixed: no error
 * control), state in place; checkpoints (device [(nsteps + 1) x ncell x N],
 * or NULL) receives the state at the start of every step and the final state.
 * Analytic Jacobian-vector products, FP64.  Workspace: rk_rok4e_workspace_size. */
int rk_rok4e_fixed_steps(const rk_mech* mech, double* Y, int64_t ncell, double p, double h,
                         int32_t nsteps, int32_t krylov_dim, double* checkpoints, void* workspace,
                         size_t workspace_bytes, void* stream);

/* Discrete adjoint of rk_rok4e_fixed_steps: given the checkpoints of a forward
 * run and ubar = dL/du(t_end) (device [ncell x N]), returns
 *   grad_lnA[j] = sum_cells dL/d ln A_j   (device [Nr], input reaction order;
 *                 for a Troe reaction A is the high-pressure factor)
 *   grad_u0     = dL/du(0) per cell       (device [ncell x N], or NULL).
 * Each step is recomputed from its checkpoint and differentiated exactly,
 * including the dependence of the Arnoldi basis on the state and on ln A
 * (second derivatives of the source term).  The paper has no adjoint; this is
 * the library's sensitivity extension of its integrator.  Workspace:
 * rk_rok4e_adjoint_workspace_size (about (78 + 16 M) N + (19 + 4 M) Nr
 * doubles per cell for Krylov dimension M, one contiguous record per cell: the
 * tapes of every right-hand-side pass of a step are kept for its reverse
 * sweep).  The sums over cells and within a cell have a fixed order: repeated
 * calls give the same bits. */
size_t rk_rok4e_adjoint_workspace_size(const rk_mech* mech, int64_t ncell, int32_t krylov_dim);
int rk_rok4e_adjoint(const rk_mech* mech, const double* checkpoints, const double* ubar, int64_t ncell,
                     double p, double h, int32_t nsteps, int32_t krylov_dim, double* grad_lnA,
                     double* grad_u0, void* workspace, size_t workspace_bytes, void* stream);
/* As rk_rok4e_adjoint, with lanes_per_cell lanes of a warp (4, 8, 16 or 32)
 * sharing each cell's species, reaction and state loops; 0 chooses from ncell
 * (8, or more when there are too few cells to give every SM sub-partition a
 * warp).  The result does not depend on the lane count beyond rounding. */
int rk_rok4e_adjoint_ex(const rk_mech* mech, const double* checkpoints, const double* ubar, int64_t ncell,
                        double p, double h, int32_t nsteps, int32_t krylov_dim, int32_t lanes_per_cell,
                        double* grad_lnA, double* grad_u0, void* workspace, size_t workspace_bytes,
                        void* stream);

/* ---- diagnostics ---------------------------------------------------------------
 * Throughput probes of the arithmetic units used by the roofline:
 *  kind 0: FP64 FMA, 1: FP32 FMA, 2: FP64 exp(), 3: double<->float
 *  conversions; how the FP64 pipe is shared: 4: FP64 FMA with one warp per
 *  SM, 5: four warps per SM, 6: four warps per SM with one active lane each
 *  (rate of warp instructions); 7: double-float (FP32 pair) multiply-adds;
 *  8: int -> double conversions (with an integer op and a bit move each).
 *  Launches a dependent-operation
 *  grid sized to the device and returns the operation rate (ops/s) measured
 *  with CUDA events in *ops_per_s.  Synchronous. */
int rk_probe_throughput(int32_t kind, double* ops_per_s);

/* The kernels' own elementary functions on a device array (for testing them
 * against the CUDA math library): which 0: y = exp(x); 1: exp(x) and 2:
 * exp(-x) from the shared-reduction pair; 3, 4, 5: the same three in the
 * mixed-precision form (polynomial's small term in FP32, relative error
 * ~1e-13; 3 is the rate-coefficient exponential of precision levels 1, 2, 3,
 * 5 and 6, while the pair 4, 5 is no longer used by any level, whose
 * equilibrium-constant exponentials stay FP64); 6: y = ln x; 7: y = 1/x.
 * Methods: Tang, ACM TOMS 15(2), 1989 (exp: a 256-entry table of 2^(j/256)
 * and a degree-4 polynomial) and 16(4), 1990 (ln: a 128-entry table and a
 * degree-7 polynomial); 1/x by two Newton steps from an FP32 estimate where
 * x and 1/x are FP32-normal, a division elsewhere.  The paper itself delegates
 * kinetics to Cantera and prints none of these.  x, y: n doubles in device
 * memory, distinct arrays; asynchronous on `stream`; RK_E_INVALID_ARGUMENT
 * for n < 0 or which outside 0..7. */
int rk_eval_exp(const double* x, double* y, int64_t n, int32_t which, void* stream);

/* Name of an RK_* return code (a static string; "unknown status" otherwise). */
const char* rk_status_string(int32_t code);

/* Copies the message of the most recent failed call on the calling thread
 * (empty if none) into buf, truncated to len - 1 characters and terminated;
 * buf may be NULL.  Always returns RK_OK. */
int rk_last_error(char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* ROK4E_H */
