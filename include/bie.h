/*
 * bie.h -- C ABI of the GB300 boundary-integral water-wave solver.
 *
 * The library builds and solves the discrete second-kind Fredholm system of
 * Ambrose, Camassa, Marzuola, McLaughlin, Robinson & Wilkening, "Numerical
 * algorithms for water waves with background flow over obstacles and
 * topography" (arXiv 2108.01786), velocity-potential formulation:
 *
 *   A omega = b                                              (Sec. 3.2, eq. Awb)
 *   A = [ -1/2 I + K_00 | G_0j ; -G_k0 | 1/2 I + K_kj - E_k ]  (Sec. 3.3, eq. lin:sys)
 *   K_kj,ml = Im{ zeta_j'(b)/2 cot((zeta_j(b) - zeta_k(a))/2) } / M_j,
 *   G_kj,ml = Re{ ... } / M_j                                (Table 1)
 *   K_jj(a,a) = Im{ zeta_j''(a) / (2 zeta_j'(a)) }           (Sec. 3.2, diagonal limit)
 *   E_k = e e^T / M_k on obstacle blocks k >= 2              (Sec. 3.3, eq. AB:cor)
 *   b_0 = phi~,  b_k = -psi_mv(zeta_k)                       (eq. Awb, eq. Phi:mv)
 *
 * and returns the normal velocity U of the free surface (Sec. 3.4, eqs.
 * d:phi:mv, d:phi:j, d:phi:0) and the obstacle stream-function constants
 * psi|_k = <1_k, omega> (eq. psi:k).
 *
 * Boundaries are numbered in block order: 0 = free surface, 1 = bottom,
 * 2..nb-1 = obstacles (Sec. 2).  Boundary k carries M_k nodes at
 * alpha_kl = 2 pi l / M_k; all per-node arrays are concatenated in block order
 * and have length N = sum_k M_k.  Complex arrays are interleaved (re, im)
 * doubles ("double2"), i.e. 2N doubles.  The surface and the bottom satisfy
 * zeta(alpha + 2pi) = zeta(alpha) + 2pi; obstacles are closed curves traversed
 * clockwise (Sec. 2, eqs. per0, per1, per2N).
 *
 * Memory.  Pointers named *_dev are CUDA device pointers on the context's
 * device; pointers named *_host are host pointers (pageable or pinned).  The
 * caller owns every buffer it passes in; the library never frees or keeps a
 * caller pointer beyond the call (inputs are copied into library-owned device
 * workspace).  The library owns its workspace (matrix storage, Krylov basis,
 * scratch), allocated with cudaMalloc on first use and released by
 * bie_destroy.
 *
 * Streams.  Every call enqueues its work on the stream given to bie_create and
 * returns once it is enqueued, except where a call says it synchronises
 * (bie_solve reads convergence flags and therefore synchronises the stream).
 *
 * Errors.  Every call returns a bie_status.  On error the outputs are
 * unspecified, a message is available from bie_last_error(ctx), and the
 * context stays usable.  No call aborts, traps or exits.
 */
#ifndef BIE_H
#define BIE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bie_ctx bie_ctx;

typedef enum {
  BIE_OK = 0,
  BIE_ERR_ARG = 1,      /* invalid argument (null pointer, bad size, bad enum) */
  BIE_ERR_GEOM = 2,     /* geometry rejected (non-finite node, zero zeta',
                           counter-clockwise obstacle, coincident nodes) */
  BIE_ERR_OOM = 3,      /* device allocation failed */
  BIE_ERR_CUDA = 4,     /* a CUDA runtime call failed */
  BIE_ERR_NOCONV = 5,   /* GMRES / refinement did not reach rtol */
  BIE_ERR_NAN = 6,      /* a non-finite value appeared in the iteration */
  BIE_ERR_TIMEOUT = 7,  /* a bounded device-side wait gave up */
  BIE_ERR_STATE = 8     /* call out of order (e.g. solve before set_geometry) */
} bie_status;

/* Storage precision of the matrix and the solver scheme.
 *   BIE_FP64    : FP64 entries, FP64 GMRES ("plain FP64").
 *   BIE_FP32_IR : FP32 entries for the inner GMRES, with iterative refinement
 *                 on a ~48-bit (FP32 hi + FP32 lo) copy of the same entries.
 *   BIE_BF16_IR : BF16 inner entries, same refinement.
 *   BIE_FP16_IR : FP16 inner entries, same refinement.                         */
typedef enum {
  BIE_FP64 = 0,
  BIE_FP32_IR = 1,
  BIE_BF16_IR = 2,
  BIE_FP16_IR = 3
} bie_precision;

typedef struct {
  double rtol;       /* stop when ||b - A omega||_2 <= rtol ||b||_2, the residual
                        taken with the full-accuracy operator (default 1e-14;
                        U needs a tight residual: its derivative terms amplify
                        high-frequency errors of omega by up to M_0/2).  With
                        rtol >= 1e-14 the refined schemes form their last
                        residuals by updating the previous full-accuracy one
                        with the product of the last increment and a cheaper
                        copy (FP32 part, FP16 / BF16 storage, fewer exact
                        slices), when that copy's rounding times the residual
                        stays below 6e-15 ||b||; such a residual does not see
                        the rounding of omega itself (within 1e-15 ||b|| of the
                        direct one, measured) */
  int restart;       /* Krylov dimension m of one GMRES cycle (default 50) */
  int max_cycles;    /* maximum number of GMRES cycles in total (default 40) */
  double inner_tol;  /* relative residual reduction asked of one inner cycle in
                        the refined schemes (0 = choose by precision: 1e-4 for
                        BIE_FP32_IR, 5e-4 for BIE_FP16_IR and BIE_BF16_IR;
                        bie_solve_multi with more than 16 columns keeps no
                        recycled space and takes 2e-3 (FP16) and 1e-2 (BF16)) */
  int row_flip;      /* 1 (default): multiply the free-surface rows of A and b
                        by -1 so that the spectrum clusters at +1/2; the
                        solution is unchanged */
  int x0;            /* 0 (default): GMRES starts from zero.  1: the solution
                        buffer holds an initial guess on entry (omega for
                        bie_solve, bie_solve_b, bie_solve_psi and
                        bie_solve_host; gamma_out for bie_vs_normal_velocity),
                        e.g. the previous time step's; the first cycle then
                        starts from the full-accuracy residual of that guess
                        and rtol stays relative to ||b||.  bie_backward,
                        bie_solve_multi and the batched solver ignore it; the
                        evolution drivers set it themselves after their first
                        solve (the previous stage's solution is the guess) */
} bie_solve_opts;

typedef struct {
  int iters;         /* total Arnoldi steps (matrix-vector products) */
  int cycles;        /* GMRES cycles (= refinement steps for *_IR) */
  int converged;     /* 1 if rtol was met */
  double rel_resid;  /* final ||b - A omega|| / ||b|| (full-accuracy operator;
                        direct or updated, see rtol) */
} bie_solve_info;

/* Fill opts with the defaults listed above. */
void bie_default_opts(bie_solve_opts* opts);

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  Errors: BIE_ERR_ARG (out == NULL), BIE_ERR_CUDA. */
bie_status bie_create(bie_ctx** out, int device, void* cuda_stream);

/* Release the context and all library-owned device memory.  NULL is a no-op. */
void bie_destroy(bie_ctx* ctx);

/* Last error message of ctx ("" if none).  The string lives until the next
 * call on ctx.  Accepts NULL (returns a static message). */
const char* bie_last_error(const bie_ctx* ctx);

/* Load the boundaries (Sec. 2; Sec. 3.3 node layout).
 *   nb          number of boundaries including the free surface, nb >= 2
 *   M_host[k]   node count M_k >= 8 of boundary k, k = 0..nb-1
 *   zeta_dev    zeta_k(alpha_kl), double2[N]
 *   dzeta_dev   zeta_k'(alpha_kl), double2[N]
 *   d2zeta_dev  zeta_k''(alpha_kl), double2[N]
 *   zc_host     obstacle centres z_j (j = 2..nb-1), double2[nb-2], used by
 *               Phi_mv (eq. Phi:mv); may be NULL when nb == 2
 * The data are copied; node tables (e^{i zeta}, e^{-i zeta}, the diagonal limit
 * Im{zeta''/(2 zeta')}, the spectral derivative and Hilbert kernels of each
 * boundary) are prepared on the device.
 * Errors: BIE_ERR_ARG, BIE_ERR_GEOM (checked on a host copy: finite values,
 * zeta' != 0, distinct consecutive nodes, clockwise obstacles), BIE_ERR_OOM. */
bie_status bie_set_geometry(bie_ctx* ctx, int nb, const int* M_host,
                            const double* zeta_dev, const double* dzeta_dev,
                            const double* d2zeta_dev, const double* zc_host);

/* Background current V1 and circulations a_j, j = 2..nb-1 (eq. Phi:mv).
 * a_host has nb-2 entries (may be NULL when nb == 2).  Errors: BIE_ERR_STATE
 * (no geometry), BIE_ERR_ARG. */
bie_status bie_set_flow(bie_ctx* ctx, double V1, const double* a_host);

/* Assemble A (eq. lin:sys) in the storage of `precision` (a bie_precision).
 * Entries are computed once at ~48-bit accuracy (or FP64 for BIE_FP64); the
 * stored value of entry (m, l) is M_l times the Table-1 kernel value, minus 1
 * on obstacle diagonal blocks (the -E_k term times M_k); the weights 1/M_l and
 * the +-1/2 I are applied exactly by the matrix-vector product.  Storage is
 * row-major with a leading dimension of N rounded up to 64.
 * Errors: BIE_ERR_STATE, BIE_ERR_ARG, BIE_ERR_OOM. */
bie_status bie_assemble(bie_ctx* ctx, int precision);

/* Right-hand side of eq. Awb: b_0 = phi~ (surface), b_k = -psi_mv(zeta_k)
 * (solids), with psi_mv = V1 Im z + sum_j a_j (-ln|1 - e^{i(z - z_j)}|).
 *   phit_dev  phi~ at the surface nodes, double[M_0];  b_dev  double[N]. */
bie_status bie_rhs(bie_ctx* ctx, const double* phit_dev, double* b_dev);

/* y = A x with the assembled operator (eq. lin:sys), in the stored precision
 * `which`: 0 = low-precision inner storage (FP32/BF16/FP16 or FP64 for
 * BIE_FP64), 1 = full-accuracy storage (FP32 hi + lo, or FP64).
 *   x_dev, y_dev  double[N].  Errors: BIE_ERR_STATE if not assembled. */
bie_status bie_matvec(bie_ctx* ctx, int which, const double* x_dev, double* y_dev);

/* Products with several vectors at once on the tensor cores: Y_r = A X_r (A of
 * eq. lin:sys; the paper suggests block GMRES for several right-hand sides,
 * Sec. 7.4) for
 * r < nrhs with the low-precision inner storage (requires BIE_FP16_IR or
 * BIE_BF16_IR assembly): the sum over stored entries is a GEMM of the N x N
 * storage with the columns X_r / M_l (tcgen05 MMA, TMA-fed, FP32
 * accumulation), then the +-1/2 diagonal is added in FP64.  Each column is
 * scaled to unit maximum before rounding to the storage type, so the result
 * carries the storage's relative rounding (2^-11 FP16, 2^-8 BF16) like the
 * inner GMRES products.
 *   nrhs in [1, 64];  X_dev, Y_dev double[nrhs * N], column r at offset r N.
 * Synchronises the stream.  Errors: BIE_ERR_STATE (no FP16/BF16 storage or
 * adjoint storage), BIE_ERR_ARG, BIE_ERR_TIMEOUT (a bounded pipeline wait
 * expired). */
bie_status bie_matmat(bie_ctx* ctx, int nrhs, const double* X_dev, double* Y_dev);

/* Products with the FULL-accuracy operator (hi + lo storage, ~48 bits) on the
 * tensor cores: Y_r = A X_r (A of eq. lin:sys) for up to 64 columns, exact integer slices of
 * both operands (5 bits each, ten slices, row and column power-of-two
 * scales) multiplied as FP16 GEMMs whose FP32 accumulations are exact (at
 * most 16384 terms of size <= 2^10), combined in FP64; the truncated slice
 * pairs lie below 2^-50 of each row's scale.  The slices of the matrix are
 * built once per assembly.  Requires FP32/FP16/BF16-IR assembly and N <=
 * 16384.  X_dev, Y_dev double[nrhs * N] (column r at offset r N).
 * Synchronises the stream.  Errors: BIE_ERR_STATE, BIE_ERR_ARG, BIE_ERR_OOM,
 * BIE_ERR_TIMEOUT (a bounded pipeline wait expired). */
bie_status bie_matmat_full(bie_ctx* ctx, int nrhs, const double* X_dev, double* Y_dev);

/* Several right-hand sides on one assembled matrix (Sec. 3, eq. lin:sys, and
 * Sec. 4's normal velocity, for every column): nrhs independent GMRES-IR
 * solves that advance in lock step, each Arnoldi step one tensor-core product
 * (bie_matmat's) for all columns still iterating, with FP64 Gram-Schmidt and
 * Hessenberg per column; residuals and U use the hi + lo storage with all
 * columns in one pass over the matrix.  Each column reaches the accuracy of a
 * bie_solve with the same storage and options.  Requires BIE_FP16_IR or
 * BIE_BF16_IR assembly and bie_set_flow.
 *   nrhs        1..64
 *   rhs_kind    BIE_RHS_PHIT: rhs_dev holds phi~ (double[nrhs * M_0], column r
 *               at offset r M_0) and b follows eq. Awb; BIE_RHS_B: rhs_dev
 *               holds b itself (double[nrhs * N]), e.g. the auxiliary
 *               Dirichlet data of eq. pressure:d:prob from bie_pressure_rhs
 *   omega_dev   double[nrhs * N] (out)
 *   U_dev       double[nrhs * M_0] (out), or NULL to skip the normal velocity
 *               (it is the velocity of the flow set by bie_set_flow, so it only
 *               has that meaning for BIE_RHS_PHIT)
 *   opts        as bie_solve (restart <= 63); NULL = defaults
 *   infos       host array of nrhs bie_solve_info (out), or NULL
 * Synchronises the stream.  Errors: BIE_ERR_STATE (not assembled, no flow,
 * FP32/FP64 or adjoint storage), BIE_ERR_ARG, BIE_ERR_OOM, BIE_ERR_TIMEOUT
 * (a bounded pipeline wait expired), BIE_ERR_NAN, BIE_ERR_NOCONV (a column
 * missed rtol in max_cycles; omega and U are still written). */
#define BIE_RHS_PHIT 0
#define BIE_RHS_B 1
bie_status bie_solve_multi(bie_ctx* ctx, int nrhs, int rhs_kind, const double* rhs_dev,
                           double* omega_dev, double* U_dev, const bie_solve_opts* opts,
                           bie_solve_info* infos);

/* Right-hand side of the auxiliary Dirichlet problem for Phi_t - C(t) (Sec. 4,
 * eq. pressure:d:prob) from a solved state:
 *   b_0 = tau kappa - |grad phi|^2 / 2 - g eta   on the surface nodes,
 *   b_k = 0                                      on the solid boundaries,
 * with kappa = Im{zeta'' conj(zeta')}/|zeta'|^3 (the curvature of the
 * tau theta_alpha / s_alpha term of eq. phitileq), |grad phi|^2 =
 * (phi_alpha/s_alpha)^2 + U^2, phi_alpha = phi~_alpha (spectral) + Re{Phi_mv'
 * zeta'} (eq. d:phi:cyl) and eta = Im zeta_0 (rho = 1).
 *   phit_dev  double[M_0]: phi~ of the state;  U_dev double[M_0]: its normal
 *             velocity (bie_solve);  b_dev double[N] (out)
 * Needs bie_set_geometry and bie_set_flow.  Errors: BIE_ERR_STATE, BIE_ERR_ARG. */
bie_status bie_pressure_rhs(bie_ctx* ctx, const double* phit_dev, const double* U_dev, double tau,
                            double g, double* b_dev);

/* Phi~ = sum_j Phi_j of eq. w123 on every boundary node, from the fluid side
 * (Gamma_0^-, Gamma_k^+), by the Plemelj formula (Sec. 4).  For the omega of
 * a state this is phi~ + i psi~ on the boundaries; for omega^aux (bie_solve_b
 * with bie_pressure_rhs) its real part is Phi_t - C(t), whence the pressure
 * p / rho = -(Phi_t - C) - |grad phi|^2 / 2 - g y on the bottom and obstacles
 * (eq. press).  Re on Gamma_0 and Im on Gamma_k come from the operator
 * (full-accuracy storage), Im on Gamma_0 as the energy's psi, Re on Gamma_k
 * from double-float sums of Re / Im{zeta_l' 1/2 cot((zeta_l - zeta_m)/2)} with
 * the own boundary regularised by 1/2 cot((beta - alpha)/2) and the Hilbert
 * transform (symbol -i sgn k) taken spectrally.
 *   omega_dev  double[N];  phi_dev  double[2 N] (out, (re, im) per node)
 * Needs bie_assemble (the operator of eq. lin:sys, not the adjoint or App. B
 * storage).  Asynchronous on the context's stream.  Errors: BIE_ERR_STATE,
 * BIE_ERR_ARG, BIE_ERR_OOM. */
bie_status bie_boundary_potential(bie_ctx* ctx, const double* omega_dev, double* phi_dev);

/* Phi~(z) = sum_j Phi_j(z) of eq. w123 at n points z of the fluid: the
 * Helsing-Ojala ratio (eq. helsing:quad, App. F) applied to the boundary
 * values of bie_boundary_potential (Phi~ is analytic and single valued in
 * Omega), double-float sums, valid near the boundaries and far from them; a
 * target on a node returns the node's value.  For omega^aux the real part is
 * Phi_t - C(t), whence the pressure p / rho = -(Phi_t - C) - |u|^2 / 2 - g y
 * throughout the fluid (eq. press; u from bie_eval_velocity).
 *   omega_dev double[N];  z_dev double[2 n] (x, y per target, in Omega);
 *   phi_dev double[2 n] (out, (re, im) per target)
 * Needs bie_assemble (the operator of eq. lin:sys).  Asynchronous.  Errors:
 * BIE_ERR_STATE, BIE_ERR_ARG, BIE_ERR_OOM. */
bie_status bie_eval_potential(bie_ctx* ctx, const double* omega_dev, long long n,
                              const double* z_dev, double* phi_dev);

/* Solve eq. lin:sys for a given right-hand side b (double[N], device) with the
 * assembled storage, by the solver of bie_solve (same options and info);
 * omega_dev double[N] (out).  No normal velocity is formed.  Errors as
 * bie_solve. */
bie_status bie_solve_b(bie_ctx* ctx, const double* b_dev, double* omega_dev,
                       const bie_solve_opts* opts, bie_solve_info* info);

/* ---- App. B: psi prescribed on the solid boundaries ----------------------
 * Assemble the operator of eq. A:alt instead of eq. AB:cor: B (Table 1 entries
 * and the +-1/2 diagonal, no -E_k term) plus, for every obstacle k >= 2, the
 * column u_k <1_k, .> with u_k = phi_cyl(zeta_0 - z_k) on surface rows and
 * psi_cyl(zeta_j - z_k) on solid rows (phi_cyl = arg(1 - e^{iz}), psi_cyl =
 * -ln|1 - e^{iz}|).  Stored like bie_assemble (the u_k(m) times M_k added to
 * the columns of obstacle k).  Afterwards bie_solve, bie_backward and the
 * phi~ form of bie_solve_multi refuse the context (BIE_ERR_STATE) until
 * bie_assemble is called again; bie_solve_b and raw-b bie_solve_multi work.
 * Errors as bie_assemble. */
bie_status bie_assemble_psi(bie_ctx* ctx, int precision);

/* Solve the App. B system: b_0 = phi - V1 xi on the surface (phic_dev,
 * double[M_0]; phi given, V1 from bie_set_flow), b_k = psi - V1 eta_k on the
 * solid nodes (psi_dev, double[N - M_0], usually constant per boundary; psi
 * must be periodic).  Returns omega (double[N]), the circulations a_j =
 * <1_j, omega> in a_host (double[nb - 2], may be NULL) and, if U_dev is given,
 * the normal velocity of Phi = Phi~ + sum a_j Phi_cyl(z - z_j) + V1 z
 * (double[M_0]).  The a_j set by bie_set_flow are not used and not changed.
 * Synchronises the stream.  Errors: BIE_ERR_STATE (no bie_assemble_psi or
 * flow), BIE_ERR_ARG, solver errors (BIE_ERR_NOCONV still writes results). */
bie_status bie_solve_psi(bie_ctx* ctx, const double* phic_dev, const double* psi_dev,
                         double* omega_dev, double* U_dev, double* a_host,
                         const bie_solve_opts* opts, bie_solve_info* info);

/* ---- time evolution of the graph formulation (Sec. 2, eqs. graph:eta:t,
 * phitileq; xi = alpha) -------------------------------------------------- */

typedef struct {
  int steps;             /* RK4 steps taken */
  int solves;            /* systems of eq. lin:sys solved */
  long long gmres_iters; /* inner GMRES iterations over all solves */
  double max_rel_resid;  /* largest final relative residual */
} bie_evolve_info;

/* One right-hand-side evaluation: the surface block of the geometry is
 * replaced by the graph zeta_0 = alpha + i eta(alpha), alpha_m = 2 pi m / M_0
 * (zeta_0', zeta_0'' by FP64 spectral derivatives, Nyquist mode dropped), the
 * matrix assembled in `precision` and solved for phi~, and
 *   eta_t  = s_alpha U,
 *   phi~_t = (phi~_alpha/s_alpha) V + (U - d phi_mv/dn) U - |grad phi|^2/2
 *            - g eta + tau theta_alpha/s_alpha,     V = eta_alpha U,
 * with C(t) = 0 and rho = 1.  Bottom, obstacles, flow (V1, a_j) are those set
 * in the context; the context keeps the new surface, assembled.
 *   eta_dev, phit_dev        double[M_0] (in)
 *   eta_t_dev, phit_t_dev    double[M_0] (out)
 *   omega_dev, U_dev         double[N], double[M_0] (out, optional)
 * Synchronises the stream.  Errors: BIE_ERR_STATE, BIE_ERR_ARG, BIE_ERR_GEOM
 * (the new surface is invalid), solver errors. */
bie_status bie_graph_rhs(bie_ctx* ctx, const double* eta_dev, const double* phit_dev, double tau,
                         double g, int precision, const bie_solve_opts* opts, double* eta_t_dev,
                         double* phit_t_dev, double* omega_dev, double* U_dev);

/* nsteps classical RK4 steps of size dt on (eta, phi~) in place, with the
 * right-hand side of bie_graph_rhs; with filter != 0 the filter of eq. filter
 * acts on eta and phi~ at the end of every step (not in the stages).  If
 * energies_host is given it receives E (eq. E:formula, rho = 1) at t = 0, dt,
 * ..., nsteps dt (nsteps + 1 values; the final one costs one more solve).
 * Synchronises the stream.  Errors as bie_graph_rhs. */
bie_status bie_graph_evolve(bie_ctx* ctx, double* eta_dev, double* phit_dev, double dt, int nsteps,
                            double tau, double g, int filter, int precision,
                            const bie_solve_opts* opts, double* energies_host,
                            bie_evolve_info* info);

/* HLS (angle-arclength) formulation with P theta reconstruction (Sec. 2):
 * the surface is rebuilt from P theta (zero-mean tangent angle) by eq. CS:th
 * (C = P0[cos P theta], S = P0[sin P theta], P0 theta = arg(C - iS), s_alpha
 * = (C^2 + S^2)^(-1/2), zeta' = s_alpha e^{i theta}) and eq. xi:eta:recon
 * (zero-mean spectral antiderivatives, xi(0) = 0, P0[eta xi_alpha] = 0),
 * zeta'' = i theta_alpha zeta'.  bie_hls_curve writes that curve (double2
 * [M_0] each, optional) into the caller's buffers and the context.
 * bie_hls_rhs: (P theta)_t = P[(U_alpha + V theta_alpha)/s_alpha] (eq.
 * Pth:t) with V from eq. definitionOfV, its constant set by xi(0) = 0
 * (V(0) = U(0) eta_alpha(0)/xi_alpha(0)), and phi~_t of eq. phitileq (C = 0,
 * rho = 1).  bie_hls_evolve: RK4 steps as bie_graph_evolve, the filter of
 * eq. filter on P theta and phi~ at the end of each step when asked for.
 * Arguments, synchronisation and errors as the graph-formulation calls. */
bie_status bie_hls_curve(bie_ctx* ctx, const double* Ptheta_dev, double* zeta_dev,
                         double* dzeta_dev, double* d2zeta_dev);
bie_status bie_hls_rhs(bie_ctx* ctx, const double* Ptheta_dev, const double* phit_dev, double tau,
                       double g, int precision, const bie_solve_opts* opts, double* Ptheta_t_dev,
                       double* phit_t_dev, double* omega_dev, double* U_dev);
bie_status bie_hls_evolve(bie_ctx* ctx, double* Ptheta_dev, double* phit_dev, double dt, int nsteps,
                          double tau, double g, int filter, int precision,
                          const bie_solve_opts* opts, double* energies_host,
                          bie_evolve_info* info);

/* General driver: formulation BIE_FORM_GRAPH (y1 = eta, phit = phi~),
 * BIE_FORM_HLS (y1 = P theta, phit = phi~) or BIE_FORM_VS_GRAPH (y1 = eta,
 * phit = gamma_0: the vortex-sheet formulation of bie_vs_graph_rhs; no energy
 * monitor, energies_host must be NULL).  Integrator:
 *   BIE_INT_DP8   the eighth-order Dormand-Prince Runge-Kutta scheme of
 *                 Sec. 7.1 (12 stages, 12 right-hand sides per step), at the
 *                 fixed step dt;
 *   BIE_INT_RK4   classical fourth-order Runge-Kutta;
 *   BIE_INT_GBS8  an eighth-order Gragg-Bulirsch-Stoer step (explicit
 *                 midpoint rule with 2, 4, 6, 8 substeps and extrapolation in
 *                 (h/n)^2, 17 right-hand sides per step), an alternative.
 * Other arguments, synchronisation and errors as bie_graph_evolve. */
#define BIE_FORM_GRAPH 0
#define BIE_FORM_HLS 1
#define BIE_FORM_VS_GRAPH 2
#define BIE_INT_RK4 0
#define BIE_INT_GBS8 1
#define BIE_INT_DP8 2
bie_status bie_evolve(bie_ctx* ctx, int formulation, int integrator, double* y1_dev,
                      double* phit_dev, double dt, int nsteps, double tau, double g, int filter,
                      int precision, const bie_solve_opts* opts, double* energies_host,
                      bie_evolve_info* info);

/* Vortex-sheet formulation with xi = alpha (Sec. 4): state (eta, gamma_0).
 * U and gamma_1..N from eqs. lin:sys2 and U:from:gam:j (bie_vs_normal_velocity);
 * eta_t = s_alpha U; gamma_0,t from the block system of eqs. gam:t:final and
 * gam:t:aux (starred kernels, +1/2 on the surface and -1/2 on the solids, no
 * -E_k term; assembled on a private context) whose right-hand side uses W =
 * grad phi - gamma_0/(2 s_alpha) t on the surface (eq. dphi:W:gam; grad phi by
 * bie_boundary_velocity from omega_0 = -d^-1 gamma_0, omega_j = d^-1 gamma_j),
 * V = eta_alpha U, and F_00, F_k0 of eq. Fk:from:UV (FP64 sums over the
 * surface sources, Hilbert transform by the FP64 DFT); C(t) = 0, rho = 1.
 *   eta_dev, gamma0_dev double[M_0] (in); eta_t_dev, gamma0_t_dev double[M_0]
 *   (out); U_dev double[M_0] (out, optional).  Errors as bie_graph_rhs. */
bie_status bie_vs_graph_rhs(bie_ctx* ctx, const double* eta_dev, const double* gamma0_dev, double tau,
                            double g, int precision, const bie_solve_opts* opts, double* eta_t_dev,
                            double* gamma0_t_dev, double* U_dev);

/* Closest approach between different boundaries (the paper stops its runs
 * before the surface self-intersects or touches an obstacle, Sec. 7): the
 * minimum over nodes i of min_j |zeta_i - zeta_j| / h_i, j on the other
 * boundaries (nearest periodic image), h_i = |zeta'_i| 2 pi / M_k the local
 * node spacing.  *ratio_host gets it and *node_host (optional) the node i.
 * bie_set_min_separation(ctx, r) makes every evolution driver check this
 * before each step and stop with BIE_ERR_GEOM when it falls below r (0 turns
 * the check off; the default).  Errors: BIE_ERR_STATE, BIE_ERR_ARG. */
bie_status bie_min_separation(bie_ctx* ctx, double* ratio_host, int* node_host);
bie_status bie_set_min_separation(bie_ctx* ctx, double ratio);

/* Energy of eq. E:formula (Sec. 5.2) of a solved state on the context's
 * geometry and flow: the trapezoidal mean over the surface of tau s_alpha +
 * g eta^2 xi_alpha / 2 + psi phi_alpha / 2 plus sum_j a_j psi|_j / 2, with psi
 * on the surface = 1/2 H omega_0 - G_00 omega_0 + sum_j K_0j omega_j + psi_mv
 * (Table 1, imaginary parts; FP64 matrix-free over M_0 x N node pairs) and
 * psi|_j = <1_j, omega> (eq. psi:k).
 *   phit_dev double[M_0], omega_dev double[N] (its solution), *E_host (out).
 * Synchronises the stream.  Errors: BIE_ERR_STATE, BIE_ERR_ARG. */
bie_status bie_energy(bie_ctx* ctx, const double* phit_dev, const double* omega_dev, double tau,
                      double g, double* E_host);

/* The filter of eq. filter on one surface vector (double[M_0], in place):
 * Fourier mode k times exp(-36 (|k|/k_max)^36), k_max = M_0/2.  Errors:
 * BIE_ERR_STATE (no geometry), BIE_ERR_ARG. */
bie_status bie_filter(bie_ctx* ctx, double* x_dev);

/* Entries A[rows[i], cols[i]] of the assembled operator (Table 1, eq. lin:sys) as doubles, including
 * the 1/M_l weights, the +-1/2 diagonal and -E_k (for parity checks).
 *   n entries; rows_dev, cols_dev int64[n]; out_dev double[n];
 *   which as in bie_matvec. */
bie_status bie_sample_entries(bie_ctx* ctx, int which, long n, const long long* rows_dev,
                              const long long* cols_dev, double* out_dev);

/* Normal velocity (Sec. 3.4): U = [eq. d:phi:mv + sum_{j>=1} eq. d:phi:j
 * + eq. d:phi:0] / s_alpha on the M_0 surface nodes for a given density
 * omega, with omega_j' and H omega_0' taken spectrally (symbols ik and |k|,
 * Nyquist mode set to zero), and psi|_k = mean(omega_k), k >= 2 (eq. psi:k).
 *   omega_dev double[N]; U_dev double[M_0]; psi_dev double[nb-2] (may be NULL). */
bie_status bie_normal_velocity(bie_ctx* ctx, const double* omega_dev, double* U_dev,
                               double* psi_dev);

/* Velocity on the boundaries: Phi'(zeta_k(alpha_m)) = u - i v at every node,
 * from eq. phi:prime with s phi_n, s phi_s of eqs. dphij:dnk and dphij:dsk
 * (Sec. 5.1; gamma_0 = -omega_0', gamma_j = omega_j', eq. gam:def), the
 * limits taken from the fluid side.  On solid boundaries phi_n vanishes up to
 * the solve's accuracy.  These are the boundary data of the Helsing-Ojala
 * quadrature.
 *   omega_dev double[N] (e.g. from bie_solve);  f_dev double2[N] (u, -v). */
bie_status bie_boundary_velocity(bie_ctx* ctx, const double* omega_dev, double* f_dev);

/* Velocity u - i v = Phi'(z) at n points z of the fluid (Sec. 5.1, eq.
 * uv:phi:phi:t) for the densities omega_dev (double[N]).
 *   z_dev double2[n] targets;  uv_dev double2[n] output (u, -v).
 *   mode 0: trapezoidal Cauchy sums of eqs. Phi:j:prime / Phi:0:prime plus
 *           Phi_mv', in FP32 (accurate to ~1e-6 relative once a target is a
 *           few node spacings from every boundary);
 *   mode 1: Helsing-Ojala quadrature (eq. helsing:quad, App. F) over the
 *           boundary values, double-float sums, for every target (a target on
 *           a node returns the node value);
 *   mode 2: automatic: Helsing where the nearest boundary node is closer than
 *           near_spacings local node spacings (|zeta_l'| 2 pi / M_l), FP32 sums
 *           elsewhere.
 *   n_near_out (host, may be NULL) receives the number of Helsing targets;
 *   passing it synchronises the stream.
 * The boundary values are recomputed on each call (an O(N^2) pass). */
bie_status bie_eval_velocity(bie_ctx* ctx, const double* omega_dev, long long n,
                             const double* z_dev, double* uv_dev, int mode,
                             double near_spacings, long long* n_near_out);

/* One solve: b (eq. Awb) -> GMRES / GMRES-IR on the assembled A -> omega -> U.
 * Requires bie_assemble.  opts may be NULL (defaults); info may be NULL.
 *   phit_dev double[M_0]; omega_dev double[N]; U_dev double[M_0];
 *   psi_dev double[nb-2] (may be NULL).
 * Synchronises the context stream (convergence checks).  Returns
 * BIE_ERR_NOCONV if rtol was not met within max_cycles (outputs hold the last
 * iterate), BIE_ERR_NAN on a non-finite residual. */
bie_status bie_solve(bie_ctx* ctx, const double* phit_dev, double* omega_dev, double* U_dev,
                     double* psi_dev, const bie_solve_opts* opts, bie_solve_info* info);

/* Row partition of the stored operator over cooperating contexts, one per
 * GPU (the matrix construction "straightforward to parallelize on a cluster
 * using MPI", Sec. 3 summary of the algorithm; Sec. 7.4: the dense approach
 * "is easy to parallelize").  Part p of P stores rows [p R, min((p+1) R, N))
 * of the operator and of the surface U-matrix, R = 32 ceil(N / (32 P)); every
 * vector (b, omega, the Krylov basis, U) stays whole on every part.  Each
 * product runs on the local rows and an allgather through the caller's
 * exchange function rebuilds the whole result; the Gram-Schmidt, Givens and
 * update work then runs identically on every part, so all parts follow the
 * same iteration.
 *   exchange(user, op, count, elem_bytes, stream): op BIE_EXCH_ALLGATHER -
 *     stage_dev holds P segments of count elements of elem_bytes each; part p
 *     filled segment p; on return (its work enqueued on stream, or done) every
 *     segment must hold the owner's data on every part.  op
 *     BIE_EXCH_ALLREDUCE_SUM - the first count doubles of stage_dev are summed
 *     over the parts in place.  Return 0 on success.
 *   stage_dev, stage_bytes  a device buffer owned by the caller, at least
 *     8 P R bytes (bie_partition_rows reports R), used only inside exchange
 *     calls; it must stay valid while the partition is set.
 * nparts = 1 (fn may be NULL) restores the unpartitioned context.  Call after
 * bie_set_geometry (a new geometry keeps the partition; its R follows the new
 * N) and before bie_assemble.  On a partitioned context bie_assemble,
 * bie_matvec, bie_solve, bie_solve_b, bie_solve_host, bie_normal_velocity and
 * bie_backward follow the partition (bie_backward assembles the local rows of
 * S^T and adds the parts' U-matrix products V^T Nbar by the allreduce);
 * entry points that need no stored matrix (right-hand side, targets,
 * potentials, energy, filter) see whole vectors and work unchanged; the others
 * (bie_sample_entries, the App. B variant, the vortex-sheet route, the
 * several-column products and solves, the evolution drivers) return
 * BIE_ERR_STATE.  Every part must make the same calls with the same
 * arguments.  Errors: BIE_ERR_ARG (nparts < 1, part out
 * of range, null function or buffer for nparts > 1), BIE_ERR_STATE (no
 * geometry). */
#define BIE_EXCH_ALLGATHER 0
#define BIE_EXCH_ALLREDUCE_SUM 1
typedef int (*bie_exchange_fn)(void* user, int op, long long count, int elem_bytes, void* stream);
bie_status bie_set_partition(bie_ctx* ctx, int nparts, int part, void* stage_dev,
                             size_t stage_bytes, bie_exchange_fn exchange, void* user);

/* The local rows of a partitioned context: [*row0, *row1) and the rows per
 * part R (the exchange segment length).  Unpartitioned: 0, N, N. */
bie_status bie_partition_rows(const bie_ctx* ctx, int* row0, int* row1, long long* rows_per_part);

/* Normal velocity by the vortex-sheet formulation (Sec. 4): given the surface
 * vortex-sheet strength gamma_0, solve the solid-boundary system of eq.
 * lin:sys2 (the transposed kernels of eq. KG:tmat, weights 1/M_j of the
 * source boundary, diagonal -1/2) for gamma_1..gamma_N and evaluate U by eq.
 * U:from:gam:j.  An independent route to the same Dirichlet-Neumann map:
 * with gamma_0 = -omega_0' of a velocity-potential solve it returns the same U.
 *   gamma0_dev double[M_0] (device); U_dev double[M_0] (device);
 *   gamma_dev  double[N - M_0] (device, may be NULL): the solid strengths;
 *   precision  storage of the solid system (any bie_precision);
 *   opts, info as in bie_solve (row_flip is ignored: every diagonal sign is -1/2).
 * Requires bie_set_geometry + bie_set_flow; the velocity-potential storage is
 * not touched.  The solid system is assembled on the first call for a
 * geometry and precision (in a private sub-context) and reused.  Synchronises
 * the stream.  Returns BIE_ERR_NOCONV / BIE_ERR_NAN as bie_solve. */
bie_status bie_vs_normal_velocity(bie_ctx* ctx, const double* gamma0_dev, double* U_dev,
                                  double* gamma_dev, int precision, const bie_solve_opts* opts,
                                  bie_solve_info* info);

/* Outputs of bie_backward: DEVICE pointers, each may be NULL (not written).
 * Complex cotangents follow g = dJ/dRe u + i dJ/dIm u. */
typedef struct {
  double* g_zeta;    /* double2[N]: w.r.t. zeta_n, with zeta', zeta'' held fixed   */
  double* g_dzeta;   /* double2[N]: w.r.t. zeta'_n                                  */
  double* g_d2zeta;  /* double2[N]: w.r.t. zeta''_n                                 */
  double* g_zc;      /* double2[nb-2]: w.r.t. the centres z_j where they enter Phi_mv */
  double* g_phit;    /* double[M_0]: w.r.t. phi~                                     */
  double* g_node;    /* double2[N]: w.r.t. zeta_n when zeta' and zeta'' of every
                        boundary are the spectral derivatives (symbol ik, Nyquist
                        mode zero) of its nodes (of zeta - alpha on the surface and
                        bottom): g_zeta - D(g_dzeta - D g_d2zeta)                   */
  double* g_shape;   /* double[5(nb-2)]: w.r.t. (x_j, y_j, q_j, b_j, theta_j) of the
                        ellipse zeta_j = x_j + i y_j + e^{i theta_j}(q_j cos alpha -
                        i b_j sin alpha), its centre also moving z_j in Phi_mv      */
  double* lambda;    /* double[N]: the adjoint density, A^T lambda = dJ/domega       */
} bie_grads;

/* Backward pass of the solve for a functional J(U) of the normal velocity:
 * given gU = dJ/dU (double[M_0], device) at the densities omega_dev
 * (double[N], device, from bie_solve on this context), fills the requested
 * fields of *grads.  The paper has no adjoint; the pass differentiates eq.
 * lin:sys (Table 1, eq. Awb) and the U formula of Sec. 3.4 by hand:
 * omegabar = (dU/domega)^T gU, one solve of A^T lambda = omegabar (the
 * solver of bie_solve, with opts, on the transposed values stored in place of
 * A, in the precision of the last bie_assemble), then dJ = lambda.(db - dA
 * omega) + the explicit terms of U, contracted pair by pair without forming
 * dA (FP64 for BIE_FP64 storage, double-float otherwise).
 *   ellipses_host double[5(nb-2)] (x, y, q, b, theta per obstacle), needed
 *   only for g_shape (may be NULL otherwise).
 * Requires bie_assemble + bie_set_flow.  Afterwards the storage holds the
 * adjoint operator: bie_solve, bie_matvec and bie_sample_entries return
 * BIE_ERR_STATE until the next bie_assemble (bie_normal_velocity and further
 * backward passes still work).  Synchronises the stream.  Returns
 * BIE_ERR_NOCONV if the adjoint solve missed rtol (outputs from the last
 * iterate), BIE_ERR_ARG for null pointers or missing ellipse parameters. */
bie_status bie_backward(bie_ctx* ctx, const double* omega_dev, const double* gU_dev,
                        const double* ellipses_host, const bie_grads* grads,
                        const bie_solve_opts* opts, bie_solve_info* info);

/* ---------------------------------------------------------------------------
 * Batched solves: many independent problems of uneven size (the paper has no
 * batched driver; each problem is the system of eq. lin:sys and its U).
 * --------------------------------------------------------------------------- */
typedef struct bie_batch bie_batch;

/* Creates a batch on `device`.  cuda_stream (may be NULL): the caller's stream;
 * bie_batch_run orders its work after what is queued there and makes it wait
 * for the results.  The batch owns a private stream and eight auxiliary ones. */
bie_status bie_batch_create(bie_batch** out, int device, void* cuda_stream);
void bie_batch_destroy(bie_batch* b);
const char* bie_batch_last_error(const bie_batch* b);

/* Geometry and flow (Sec. 2, eq. Phi:mv) of problem p (0 <= p < 4096; problems are numbered
 * 0..nprob-1 without gaps), arguments as in bie_set_geometry and bie_set_flow
 * (device node arrays are copied; validation as there).  N = sum M_k <= 16384.
 * Synchronises the caller's stream.  Returns BIE_ERR_GEOM / BIE_ERR_ARG as the
 * single-problem calls do. */
bie_status bie_batch_set_problem(bie_batch* b, int p, int nb, const int* M_host,
                                 const double* zeta_dev, const double* dzeta_dev,
                                 const double* d2zeta_dev, const double* zc_host, double V1,
                                 const double* a_host);

/* Assemble, solve and evaluate U for every problem (eqs. lin:sys, Awb; Sec.
 * 3.4): node tables, assembly, right-hand side, GMRES-IR for all problems in
 * one cooperative kernel, normal velocity.  Arrays are DEVICE and packed
 * in problem order:
 *   phit_all  double[sum M_0,p]   omega_all double[sum N_p]   U_all double[sum M_0,p]
 * precision: BIE_FP32_IR, BIE_FP16_IR or BIE_BF16_IR (the storage of every
 * problem); opts as in bie_solve (restart <= 63), may be NULL; infos (host,
 * nprob entries, may be NULL) receive each problem's counts and residual.
 * The first run for a set of problems, pointers and options records the
 * sequence into a CUDA graph (after one direct run that allocates every
 * buffer); later runs replay it.  Synchronises.  Returns BIE_ERR_NOCONV if a
 * problem missed rtol, BIE_ERR_NAN on a non-finite residual, BIE_ERR_TIMEOUT
 * if a grid barrier of the solver gave up waiting (its wait is bounded). */
bie_status bie_batch_run(bie_batch* b, int nprob, const double* phit_all, double* omega_all,
                         double* U_all, int precision, const bie_solve_opts* opts,
                         bie_solve_info* infos);

/* The autotuner's choice: before the first run for a set of problem sizes
 * (and storage, restart), bie_batch_run times its solver kernel on those
 * problems for GEMV work units of 256 KB, 512 KB, 1 MB, 2 MB and 4 MB of
 * stored matrix (at least 32 rows each) and keeps the fastest.
 *   *unit_bytes    the chosen size (0 before the first run)
 *   candidate_ms   (may be NULL) float[5], the kernel times measured. */
bie_status bie_batch_tuning(const bie_batch* b, long long* unit_bytes, float* candidate_ms);

/* Stored-matrix bytes read by the residual products of the last bie_batch_run,
 * summed over its problems (each product reads N x ld entries of the hi + lo
 * pair, of the FP32 part alone, or of the FP16 / BF16 inner storage, by the
 * residual rule of bie_solve).  With the Arnoldi steps' reads (iters x N x ld
 * entries of the inner storage per problem) this is all the matrix traffic of
 * the solver kernel.  *bytes = 0 before the first run.  Errors: BIE_ERR_ARG. */
bie_status bie_batch_resid_bytes(const bie_batch* b, double* bytes);

/* Test of the solver's grid barrier: a cooperative launch of one CTA per SM
 * passes three barriers; the CTA numbered `stall` (>= 0) returns without
 * arriving, so the others' bounded waits (spin_limit polls) run out and set
 * the error flag.  stall < 0: no CTA stalls.  *passed_out = barriers passed
 * summed over CTAs, *err_out = the flag.  Returns BIE_ERR_TIMEOUT when the
 * flag is set. */
bie_status bie_test_grid_barrier(int device, unsigned spin_limit, int stall, int* passed_out,
                                 int* err_out);

/* End-to-end call on HOST buffers: copy the geometry and phi~ to the device,
 * set_geometry + set_flow + assemble(precision) + solve (eq. Awb, U of Sec. 3.4), copy omega, U and psi
 * back.  Shapes as in the device calls (zeta_host etc. double2[N], omega_host
 * double[N], U_host double[M_0], psi_host double[nb-2] or NULL).  Pinned host
 * memory gives the fastest copies.  Synchronises the stream before returning. */
bie_status bie_solve_host(bie_ctx* ctx, int nb, const int* M_host, const double* zeta_host,
                          const double* dzeta_host, const double* d2zeta_host,
                          const double* zc_host, double V1, const double* a_host,
                          const double* phit_host, int precision, const bie_solve_opts* opts,
                          double* omega_host, double* U_host, double* psi_host,
                          bie_solve_info* info);

/* Largest N = sum M_k that bie_normal_velocity_static accepts. */
#define BIE_STATIC_MAXN 8192

/* The normal velocity U and psi|_k, as bie_normal_velocity computes them, but
 * without a context and without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc or let a
 * library do so (an allocator that owns all device memory, a loop where an
 * allocation may stall, a host program whose other runtime owns the device
 * heap).  All scratch lives in one file-scope device array of fixed size
 * (about 6 MB, held by every GPU that loads the library until exit), which
 * limits N = sum M_k to BIE_STATIC_MAXN.
 *   nb, M_host, zeta_dev, dzeta_dev, d2zeta_dev, zc_host  as in bie_set_geometry
 *   V1, a_host   as in bie_set_flow;  omega_dev double[N]
 *   U_dev double[M_0];  psi_dev double[nb-2] (may be NULL)
 *   cuda_stream  the stream to enqueue on (NULL = legacy default stream); it
 *                must belong to the current device
 * The geometry is not validated (use bie_set_geometry for that).  Every call
 * shares the scratch array: calls that overlap on the GPU race and must be
 * serialised by the caller.  The array's device address belongs to the CUDA
 * context current at the call and is looked up on every call whose stream is
 * not being captured; a call on a capturing stream reuses the address of the
 * last uncaptured call on that device, so make one call before any capture.
 * Returns BIE_ERR_ARG for null pointers, nb out of range, M_k < 8,
 * N > BIE_STATIC_MAXN or a stream of another device; BIE_ERR_STATE for a
 * captured call with no earlier uncaptured one on the device; BIE_ERR_CUDA if
 * the address lookup or a launch fails.  Enqueues and returns without
 * synchronising. */
bie_status bie_normal_velocity_static(int nb, const int* M_host, const double* zeta_dev,
                                      const double* dzeta_dev, const double* d2zeta_dev,
                                      const double* zc_host, double V1, const double* a_host,
                                      const double* omega_dev, double* U_dev, double* psi_dev,
                                      void* cuda_stream);

/* Kernel timing (opt-in).  When profiling is on, the library brackets each of
 * its hot kernels with CUDA events on the context stream and accumulates the
 * durations; skipped (already-converged) Arnoldi launches are not counted.
 * The byte counts are the algorithmic matrix bytes of one product
 * (N^2 times the stored element size).  kernel_launches counts every kernel
 * the library launched since profiling was (re)enabled. */
typedef struct {
  int enabled;
  int n_gemv_inner;          /* products with the inner storage (low-precision, or
                                FP64): the Arnoldi steps and residuals updated
                                from the last increment in that storage */
  double ms_gemv_inner;
  double bytes_gemv_inner;   /* per product */
  int n_gemv_full;           /* full-accuracy residual products */
  double ms_gemv_full;
  double bytes_gemv_full;    /* per product */
  int n_assemble;
  double ms_assemble;
  int n_velocity;
  double ms_velocity;
  long long kernel_launches;
  int n_gemv_hi;             /* refinement residuals with the FP32 part only (early
                                ones, and ones updated from the last increment) */
  double ms_gemv_hi;
  double bytes_gemv_hi;      /* per product */
} bie_profile;

/* on != 0 enables profiling and resets the counters; 0 disables it. */
bie_status bie_set_profiling(bie_ctx* ctx, int on);

/* Synchronise the context stream and return the accumulated profile. */
bie_status bie_get_profile(bie_ctx* ctx, bie_profile* out);

#ifdef __cplusplus
}
#endif
#endif /* BIE_H */
