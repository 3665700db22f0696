/*
 * elrt.h - C ABI of the GB300 element-learning radiative-transfer library.
 *
 * Steady mono-energetic transport on the x-z plane (Sec. 2.1, eq. RT_PDE):
 *     s . grad u + sigma_e u - sigma_s int_S p(s, s') u(s') ds' = 0,   u = g on the inflow boundary,
 * discretised by Q_p spectral elements on LGL nodes, N uniform angular cells with p_a = 0, upwind DG
 * and its hybridisation (Sec. 2.2).  The library builds each element's in2out and in2sol operators
 * (eqs. hdg_local_i2u, hdg_local_i2o, ang_ave), solves the global skeleton system
 * (eq. hdg_global_mat) and recovers the mean intensity (Algorithm 1).
 *
 * Conventions shared by every entry point
 *   - Mesh: a uniform nx x nz grid of square elements of side h (km); element e = ix + nx*iz,
 *     ix along +x, iz along +z (up).  Node i = a + (p+1) b of an element sits at the LGL points
 *     (xi_a, xi_b) of the reference square [-1, 1]^2.
 *   - Angular cell k is the interval [k dth, (k+1) dth), dth = 2 pi / N, N a multiple of 4 (so no
 *     cell is tangent to a face).  sigma_s = omega * sigma_e with omega constant per element.
 *   - Faces of an element, in this order: bottom (-z), right (+x), top (+z), left (-x).
 *   - Skeleton DOFs of an element (n_in = n_out = 2 (p+1) N): per face, per face node m in the
 *     order of increasing coordinate along the face, the N/2 cells leaving (outflow) or entering
 *     (inflow) through that face in increasing k.  The inflow of an element through face F is the
 *     outflow of its neighbour through the opposite face, same nodes and cells, or boundary data.
 *   - Boundary inflow array (eq. for hat V_h^g, the projection P_M g): the four domain sides in
 *     the order bottom, right, top, left; nx faces (bottom/top) or nz faces (right/left) in the
 *     order of increasing coordinate; per face p+1 nodes; per node the N/2 entering cells in
 *     increasing k.  Length 2 (nx + nz) (p+1) N/2.
 *   - in2out: [E][n_out][n_in] row-major; in2sol (mean intensity): [E][(p+1)^2][n_in] row-major.
 *   - Pointers documented as "device" must be device (or managed) memory of the current CUDA
 *     device; "host" pointers are ordinary host memory.  The caller owns every buffer it passes;
 *     a context owns only its own workspace.
 *   - Every call is asynchronous on the context's stream unless it says it synchronises.
 *   - Errors: argument checks run on the host before any launch and return ELRT_EINVAL; CUDA
 *     failures return ELRT_ECUDA; elrt_last_error() gives a message.  No exception and no abort
 *     crosses this boundary.
 */
#ifndef ELRT_H
#define ELRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ELRT_OK = 0,
    ELRT_EINVAL = 1,      /* bad argument (checked on the host before any launch) */
    ELRT_ENOMEM = 2,      /* device allocation failed */
    ELRT_ESINGULAR = 3,   /* an element's local matrix had a zero pivot */
    ELRT_ENOCONV = 4,     /* iteration limit reached before the tolerance */
    ELRT_ETIMEOUT = 5,    /* a bounded device wait gave up */
    ELRT_ECUDA = 6,       /* a CUDA runtime call failed */
    ELRT_ENOTRAINED = 7   /* the network has no weights */
} elrt_status;

typedef enum {
    ELRT_ANG_FV0 = 0,     /* paper: P0 angular cells, cell-averaged direction and phase */
    ELRT_ANG_DO = 1       /* direction and phase sampled at cell centres */
} elrt_angular;

/* Local-solve modes.  "Refinement" below is iterative refinement whose residual -B^ - A X is formed
 * from the structured operator in float-float arithmetic (pairs of FP32 values, ~44 significant
 * bits, error-free TwoSum / FMA TwoProduct) with the running solution X also kept in float-float;
 * no FP64 instruction runs per matrix entry.  Measured: one sweep takes the FP32-level solution to a
 * maximum relative residual of ~2e-12 on the benchmark slab; two sweeps stay below 1e-12 on every
 * tested element. */
typedef enum {
    ELRT_LOCAL_FP64 = 0,     /* FP64 LU with partial pivoting on the CUDA cores (no refinement) */
    ELRT_LOCAL_FP32_IR = 1,  /* FP32 LU with partial pivoting on the CUDA cores, then float-float refinement */
    ELRT_LOCAL_TF32_IR = 2   /* LU without pivoting whose trailing updates run on the tensor cores as
                                3xTF32 (hi*hi + hi*lo + lo*hi of TF32 splits of the FP32 operands, FP32
                                accumulation: FP32-level factors), then float-float refinement */
} elrt_local_mode;

typedef enum { ELRT_F32 = 0, ELRT_F64 = 1 } elrt_dtype;

/* Operator used by the Arnoldi steps of the skeleton GMRES when in2out is FP32 (elrt_set_krylov_op). */
typedef enum { ELRT_KRYLOV_F32 = 0, ELRT_KRYLOV_F16 = 1 } elrt_krylov_op;

/* Element discretisation: degree p (1..10), N angular cells (4..32, multiple of 4), HG asymmetry g. */
typedef struct {
    int32_t p;
    int32_t n_angles;
    int32_t angular;   /* elrt_angular */
    double hg_g;       /* in [0, 1) */
} elrt_disc;

typedef struct elrt_ctx elrt_ctx;

typedef struct {
    int32_t refine_steps;      /* refinement steps taken (IR modes) */
    int32_t n_flagged;         /* elements whose status word is non-zero */
    double max_rel_residual;   /* max over elements of max|B^ + A X| / max|B^| after the last step */
} elrt_local_stats;

typedef struct {
    int32_t iterations;        /* Arnoldi steps in total */
    int32_t restarts;          /* completed restart cycles */
    int32_t converged;         /* 1 if the relative residual reached rtol */
    double rel_residual;       /* ||b - A x|| / ||b||, recomputed explicitly at exit */
} elrt_solve_stats;

/* ---------------------------------------------------------------- sizes and host-side tables */

/* Sizes of one element: nodes (p+1)^2, local unknowns (p+1)^2 N, inflow/outflow DOFs 2 (p+1) N,
 * and the length of the boundary inflow array of an nx x nz mesh.  -1 on an invalid disc. */
int64_t elrt_n_nodes(const elrt_disc* disc);
int64_t elrt_n_local(const elrt_disc* disc);
int64_t elrt_n_skel(const elrt_disc* disc);
int64_t elrt_n_inflow(const elrt_disc* disc, int32_t nx, int32_t nz);

/* LGL nodes (ascending) and weights of degree p into host arrays of p+1 doubles (Sec. 2.2.1:
 * Lagrange basis on the LGL points, which are also the quadrature points). */
elrt_status elrt_lgl(int32_t p, double* xi, double* w);

/* Phase coupling W[k][l] (host, N*N doubles, row-major) after dividing the scattering term by the
 * cell width: fv0 W_kl = (1/dth) int_k int_l p(t - t'), do W_kl = dth p(t_k - t_l), rows scaled
 * to sum to 1; p the HG function of Sec. 2.1 normalised on the circle. */
elrt_status elrt_phase_matrix(const elrt_disc* disc, double* W);

/* Physical coordinates (km) of the LGL nodes of every element: host arrays x, z of E (p+1)^2. */
elrt_status elrt_node_coords(const elrt_disc* disc, int32_t nx, int32_t nz, double h, double* x, double* z);

/* ---------------------------------------------------------------- context */

/* Creates a context for one discretisation on the current CUDA device.  `stream` is a
 * cudaStream_t (NULL: the legacy default stream).  Workspace is allocated on first use and grown
 * as needed; elrt_destroy frees it.  Not thread-safe: one host thread per context. */
elrt_status elrt_create(elrt_ctx** ctx, const elrt_disc* disc, void* stream);
elrt_status elrt_destroy(elrt_ctx* ctx);
elrt_status elrt_set_stream(elrt_ctx* ctx, void* stream);
/* Operator of the Arnoldi-step matvecs (and of the sweep preconditioner) of elrt_solve_global /
 * elrt_solve_field / elrt_solve_batch with FP32 in2out.  ELRT_KRYLOV_F32 (the default): the FP32
 * operator everywhere.  ELRT_KRYLOV_F16: each solve first writes an FP16 copy of in2out into the
 * context's workspace (2 bytes per entry) and builds the Krylov basis with it, while the
 * right-hand side and every restart residual use the FP32 operator, so the restarts still refine
 * the iterate to rtol in the FP32 system (restarted GMRES as the inner solver of a mixed-precision
 * iterative refinement; half the operator bytes per Arnoldi step).  A solve keeps the FP32
 * operator throughout when in2out holds an entry beyond +-6e4 or a non-finite one, and switches to
 * it when a restart cycle lowers the true residual by less than 10%.  The FP16 copy pays when the
 * solve is bound by its matvecs (plain GMRES, hundreds of steps); with the sweep preconditioner the
 * FP32 operator needs fewer restart cycles (benchmark slab: 12 steps in one cycle against 16 in
 * two, 12.1 against 15.6 ms).  FP64 operators ignore the setting.  ELRT_EINVAL on another value. */
elrt_status elrt_set_krylov_op(elrt_ctx* ctx, int32_t op);
/* CUDA-graph replay of the skeleton GMRES (on by default): each restart cycle -- restart residual,
 * convergence test on the device, restart-length Arnoldi steps, update -- is captured once per
 * solve and Arnoldi operator and replayed, with one host synchronisation per cycle instead of two
 * and no per-launch host cost.  The results are those of plain launches (the same kernels in the
 * same order); the one difference is that a stalled FP16 cycle switches the Arnoldi operator to
 * FP32 from the following cycle on, one cycle later.  Off (0) or while kernel timing is enabled:
 * plain launches. */
elrt_status elrt_set_graphs(elrt_ctx* ctx, int32_t on);

/* Preconditioner of the skeleton GMRES for FP32 in2out (elrt_set_precond).  ELRT_PRECOND_SWEEP (the
 * default): right preconditioning by upwind block Gauss-Seidel sweeps of the skeleton system
 * (I - A_int) z = r (eq. hdg_global_mat; Sec. 2.3 lists transport sweeps among the solvers of
 * radiative transfer), from z = 0, one sweep from each mesh corner in turn (bottom-left,
 * bottom-right, top-right, top-left): a sweep visits the elements in wavefront order from its
 * corner and recomputes the outflow of each element's two downwind faces (right and top from the
 * bottom-left corner, left and top from the bottom-right, left and bottom from the top-right,
 * right and bottom from the top-left) as z_F = r_F + A_i2o^K[F] z_in(K), with the inflow gathered
 * from the current z (the latest values written; zero before any).  With right preconditioning
 * GMRES still minimises the true residual, so the solution and the stopping test are those of
 * plain GMRES; the Arnoldi steps fall by an order of magnitude on the scattering workloads (each
 * then costs one application: every operator row read twice, on the Arnoldi operator
 * elrt_set_krylov_op selects).  ELRT_PRECOND_NONE: plain GMRES.  FP64 operators ignore the setting.  ELRT_EINVAL on
 * another value. */
typedef enum { ELRT_PRECOND_NONE = 0, ELRT_PRECOND_SWEEP = 1 } elrt_precond;
elrt_status elrt_set_precond(elrt_ctx* ctx, int32_t kind);
/* Products of the trailing updates of the TF32_IR local factorisation (elrt_set_lu_products).
 * ELRT_LU_PRODUCTS_AUTO (the default): 3xFP16 -- each operand as its FP16 rounding plus the FP16
 * rounding of the remainder, hi*hi + hi*lo + lo*hi accumulated in FP32, ~22-bit products like
 * 3xTF32 at half the tensor-core instructions -- for a batch chunk whose assembled entries all lie
 * in [0.25, 1024] and that has no source column, and 3xTF32 otherwise; the refinement re-solves of
 * such a chunk run their forward sweep in 3xFP16 too (each element's residual scaled by a power of
 * two into [0.5, 1)) and their backward sweep in 3xTF32.
 * ELRT_LU_PRODUCTS_TF32: 3xTF32 everywhere.  The refined operators meet the same accuracy either way.
 * ELRT_EINVAL on another value. */
typedef enum { ELRT_LU_PRODUCTS_AUTO = 0, ELRT_LU_PRODUCTS_TF32 = 1 } elrt_lu_products;
elrt_status elrt_set_lu_products(elrt_ctx* ctx, int32_t mode);
/* z = M r, the sweep preconditioner above applied once on the context's stream; synchronises.
 * in2out: device [E][n_out][n_in] FP32 (dtype ELRT_F32; ELRT_EINVAL otherwise); r, z: device
 * [E][n_out] FP32, distinct.  ELRT_ETIMEOUT (after a synchronisation) if a wait between elements
 * gave up. */
elrt_status elrt_apply_precond(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2out, int32_t dtype,
                               const float* r, float* z);
const char* elrt_status_str(elrt_status s);
const char* elrt_last_error(const elrt_ctx* ctx);   /* message of the last failing call (or "") */

/* ---------------------------------------------------------------- measurement */

/* Kernel timing.  While enabled, the context records CUDA events on its own stream around every
 * launch of its kernels and, at the next synchronisation inside a call, adds the elapsed times to
 * per-kernel totals.  elrt_profile_get returns the total milliseconds and the number of timed
 * launches of one kernel group ("assemble", "lu_factor_solve", "lu_resolve", "lu_tc_diag",
 * "lu_tc_rowcol", "lu_tc_update", "residual", "restrict", "status", "gemv", "krylov", "sweep",
 * "estimate"); unknown names give 0.  elrt_profile_work returns, for the same timed launches, the
 * algorithmic bytes (every operand read once and every result written once, at the width the
 * kernel stores it) and the useful flops the library counts for them (0 where a group has no
 * arithmetic worth counting); achieved bandwidth = bytes / time.  elrt_launch_count returns how
 * many kernels the context launched since creation or the last reset (whether or not timing is
 * on). */
elrt_status elrt_profile_enable(elrt_ctx* ctx, int32_t on);
elrt_status elrt_profile_reset(elrt_ctx* ctx);
elrt_status elrt_profile_get(elrt_ctx* ctx, const char* kernel, double* total_ms, int64_t* launches);
elrt_status elrt_profile_work(elrt_ctx* ctx, const char* kernel, double* bytes, double* flops);
int64_t elrt_launch_count(const elrt_ctx* ctx);

/* ---------------------------------------------------------------- local stage (Sec. 2.2.3) */

/* Element matrices of eq. hdg_local_mat, scaled to the reference element (Sec. 2.4.1: sigma -> h
 * sigma / 2) and divided by the cell width: A = B - C + M - S (device, [E][nu][nu] FP64) and the
 * right-hand sides -B^ (device, [E][nu][n_in] FP64).  kappa: device [E][(p+1)^2] FP64, km^-1 at
 * the nodes; omega: device [E]; h: element side (km), or per-element sides h_elem (device [E],
 * NULL to use h).  Provided for verification; the solve paths below never materialise A in FP64. */
elrt_status elrt_assemble(elrt_ctx* ctx, int64_t n_elems, double h, const double* h_elem,
                          const double* kappa, const double* omega, double* A, double* rhs);

/* in2out and in2sol of E elements (eqs. hdg_local_i2u, hdg_local_i2o, ang_ave):
 *   X = -(B - C + M - S)^{-1} B^,  in2out = R^o X,  in2sol = (1/N) sum_k X[(k, i), :].
 * mode: elrt_local_mode; out_dtype: elrt_dtype of in2out/in2sol (device buffers sized above).
 * refine_steps: float-float refinement sweeps for the IR modes (ignored for FP64; 0..8).
 * elem_status: device [E] int32 or NULL; per element 0 = ok, 1 = zero pivot, 2 = refinement
 * residual above 1e-10 after the last step, 4 = non-finite value.  stats (host, may be NULL)
 * synchronises the stream to fill it.  Inputs are checked on the device (kappa and h finite and
 * non-negative, h > 0, omega in [0, 1], kappa_hat = kappa h / 2 at most 1e30); a bad input makes
 * the call return ELRT_EINVAL after synchronising (the kernels still run on it, and every index
 * they form stays in range whatever the values). */
elrt_status elrt_build_local(elrt_ctx* ctx, int64_t n_elems, double h, const double* h_elem,
                             const double* kappa, const double* omega, int32_t mode,
                             int32_t refine_steps, int32_t out_dtype, void* in2out, void* in2sol,
                             int32_t* elem_status, elrt_local_stats* stats);

/* Optional extras of a local build with a volume source f (eq. RT_PDE with f != 0; eqs.
 * hdg_local_f2u_i2u and hdg_local_f2o_i2o: u_h = A_i2u u^_in + f_u on each element, with
 * f_u = (B - C + M - S)^{-1} [f] and its outflow trace f^_u = R^o f_u), and the full radiance
 * operator A_i2u for radiance recovery:
 *   source  device [E][N][(p+1)^2] FP64: f at node i averaged over angular cell k (row k, column i),
 *           km^-1 x radiance; the library scales it to the reference element like sigma (f h / 2)
 *           and weights it by the node's quadrature weight.  NULL: no source (f2o, f2m, f2u unused);
 *   f2o     device [E][n_out] FP64: f^_u (required with a source);
 *   f2m     device [E][(p+1)^2] FP64: the angular mean (1/N) sum_k f_u[(k, i)] (required with a source);
 *   f2u     device [E][nu] FP64: f_u itself, rows k (p+1)^2 + i, or NULL;
 *   in2rad  device [E][nu][n_in] in the build's out_dtype: A_i2u (rows k (p+1)^2 + i), or NULL.
 * The source is one more right-hand-side column of the element's solve (the matrix is factored
 * once) and is refined with the others. */
typedef struct {
    const double* source;
    double* f2o;
    double* f2m;
    double* f2u;
    void* in2rad;
} elrt_local_extras;

/* elrt_build_local with extras (NULL extras: identical to elrt_build_local).  ELRT_EINVAL if a
 * source is given without f2o and f2m. */
elrt_status elrt_build_local_ex(elrt_ctx* ctx, int64_t n_elems, double h, const double* h_elem,
                                const double* kappa, const double* omega, int32_t mode, int32_t refine_steps,
                                int32_t out_dtype, void* in2out, void* in2sol, const elrt_local_extras* extras,
                                int32_t* elem_status, elrt_local_stats* stats);

/* Same operators as elrt_build_local (modes ELRT_LOCAL_FP64 and ELRT_LOCAL_FP32_IR), for callers
 * that cannot allocate device memory: code running where cudaMalloc is not allowed or not wanted,
 * such as a host process whose device memory is owned and budgeted by another framework, a
 * real-time loop that must not allocate after start-up, or a plug-in that is handed buffers but
 * no allocator.  The paper has no counterpart; this is a library convenience.
 *   - It needs no context and allocates nothing: no cudaMalloc, cudaFree or other allocating call.
 *     Its scratch is one file-scope device array of ELRT_STATIC_SCRATCH_MIB MiB that every GPU
 *     which loads the library holds until the process exits.  The batch is processed in chunks
 *     that fit the array.  An element of nu = (p+1)^2 N unknowns and n_in = 2 (p+1) N inflow DOFs
 *     takes nu ld s + nu 4 + 76 bytes, plus nu n_in 8 in FP32_IR, where ld = nu + n_in rounded up
 *     to a multiple of 32 and s = 4 (FP32_IR) or 8 (FP64); 256 bytes of the array hold flags.
 *     ELRT_EINVAL is returned, before any launch, when one element does not fit the array or when
 *     its LU panel needs more than 227 KB of shared memory (nu beyond 1512 in FP32_IR, 1588 in
 *     FP64).
 *   - The first call on a device looks up the array's device address (once per device, with
 *     that device current); make that first call before any stream capture.
 *   - Every call on a device shares the array and leaves its contents behind; what must start
 *     at zero is cleared by each call.  Calls whose work overlaps on the GPU (other streams,
 *     other host threads) race on the array: serialise them.
 *   - The caller passes inputs and outputs exactly as for elrt_build_local; `stream` is a
 *     cudaStream_t (NULL: legacy default stream).  The call synchronises that stream at the end
 *     and returns ELRT_EINVAL for bad arguments or invalid kappa/omega/h, ELRT_ESINGULAR when some
 *     element met a zero pivot or produced a non-finite value (the other elements' operators are
 *     still written), ELRT_ECUDA on a CUDA failure.  It reports no statistics and no per-element
 *     status. */
#define ELRT_STATIC_SCRATCH_MIB 64
elrt_status elrt_build_local_static(const elrt_disc* disc, void* stream, int64_t n_elems, double h,
                                    const double* h_elem, const double* kappa, const double* omega, int32_t mode,
                                    int32_t refine_steps, int32_t out_dtype, void* in2out, void* in2sol);

/* ---------------------------------------------------------------- global stage (Sec. 2.3) */

/* y = (I - A_int) x on the skeleton of an nx x nz mesh: per element y_K = x_K - in2out_K x_in(K)
 * with the inflow gathered from the neighbours' outflow and zero on the domain boundary.
 * x, y: device [E][n_out] FP64; in2out: device, dtype elrt_dtype. */
elrt_status elrt_global_apply(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2out, int32_t dtype,
                              const double* x, double* y);

/* Solves eq. hdg_global_mat, sum_K (R^o_K - A_i2o^K) u^ = 0 with the boundary inflow moved to the
 * right-hand side, by restarted GMRES(restart) with classical Gram-Schmidt (FP32 basis and
 * restart <= 31: a second pass where the first removes more than 90% of ||w||^2; otherwise always
 * two passes), until ||b - A x|| <= rtol ||b|| (recomputed at every restart) or max_iter Arnoldi
 * steps.  FP64 in2out: FP64 vectors.  FP32 in2out: FP32 Krylov basis, float-float iterate,
 * right-hand side and restart residual, FP64 reductions; the Arnoldi steps use the operator that
 * elrt_set_krylov_op selects.
 * inflow: device boundary data (layout above); skeleton: device [E][n_out] FP64, read as the
 * initial guess if use_guess != 0, else zeroed; on return it holds the outflow DOFs.
 * Synchronises.  Returns ELRT_ENOCONV (stats filled, skeleton = last iterate) if not converged. */
elrt_status elrt_solve_global(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2out, int32_t dtype,
                              const double* inflow, double rtol, int32_t max_iter, int32_t restart,
                              int32_t use_guess, double* skeleton, elrt_solve_stats* stats);

/* Mean intensity u^m_K = in2sol_K x_in(K) (Algorithm 1 step 4 with eq. ang_ave), boundary inflow
 * included.  in2sol: device [E][(p+1)^2][n_in]; skeleton: device [E][n_out] FP64;
 * mean: device [E][(p+1)^2] FP64. */
elrt_status elrt_recover_mean(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2sol, int32_t dtype,
                              const double* skeleton, const double* inflow, double* mean);

/* The same with a volume source: elrt_solve_global_source solves eq. hdg_global_mat with the source
 * term, sum_K (R^o_K - A_i2o^K) u^ = sum_K f^_u^K, i.e. right-hand side A_bnd g + f2o (f2o: device
 * [E][n_out] FP64 from elrt_build_local_ex, NULL: no source); elrt_recover_mean_source adds the
 * source part of the mean, u^m_K = in2sol_K x_in(K) + f2m_K (f2m: device [E][(p+1)^2] FP64 or NULL).
 * Other arguments and behaviour as elrt_solve_global / elrt_recover_mean. */
elrt_status elrt_solve_global_source(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2out, int32_t dtype,
                                     const double* inflow, const double* f2o, double rtol, int32_t max_iter,
                                     int32_t restart, int32_t use_guess, double* skeleton, elrt_solve_stats* stats);
elrt_status elrt_recover_mean_source(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2sol, int32_t dtype,
                                     const double* f2m, const double* skeleton, const double* inflow, double* mean);

/* Radiance of every element (eq. hdg_local_f2u_i2u, Algorithm 1 step 4): u_K = A_i2u^K x_in(K) +
 * f_u^K, the inflow x_in(K) gathered from the skeleton solution and the boundary data.
 * in2rad: device [E][nu][n_in] (dtype) from elrt_build_local_ex; f2u: device [E][nu] FP64 or NULL
 * (no source); skeleton: device [E][n_out] FP64; u: device [E][nu] FP64, rows k (p+1)^2 + i.  The
 * learned local stage has no A_i2u (the network predicts in2out and in2sol only): radiance needs
 * the classical build. */
elrt_status elrt_recover_radiance(elrt_ctx* ctx, int32_t nx, int32_t nz, const void* in2rad, int32_t dtype,
                                  const double* f2u, const double* skeleton, const double* inflow, double* u);

/* ---------------------------------------------------------------- whole pipeline (Algorithm 1) */

/* One field: an nx x nz mesh of square elements of side h (km) with its coefficients and
 * boundary data (all device pointers, layouts as above). */
typedef struct {
    int32_t nx, nz;
    double h;
    const double* kappa;    /* [nx nz][(p+1)^2] km^-1 at the LGL nodes */
    const double* omega;    /* [nx nz] */
    const double* inflow;   /* boundary inflow, length elrt_n_inflow */
} elrt_field;

typedef struct elrt_net elrt_net;

typedef struct {
    int32_t mode;           /* elrt_local_mode of the classical local stage */
    int32_t refine_steps;   /* float-float refinement sweeps (IR modes) */
    double rtol;            /* GMRES relative residual */
    int32_t max_iter;
    int32_t restart;
    elrt_net* net;          /* non-NULL: learned local stage (elrt_build_local_learned) */
    double learned_tol;     /* its energy-balance fallback threshold */
} elrt_solve_opts;

typedef struct {
    elrt_local_stats local;
    elrt_solve_stats global;
    int64_t n_fallback;     /* learned stage: elements re-solved classically */
    double local_ms, global_ms;
} elrt_field_stats;

/* Algorithm 1 on one field: local operators (FP32 in2out / in2sol in the context's workspace),
 * skeleton GMRES, mean intensity.  mean: device [nx nz][(p+1)^2] FP64; skeleton: device
 * [nx nz][n_out] FP64 or NULL.  Synchronises; ELRT_ENOCONV if GMRES stopped at max_iter (the mean
 * of the last iterate is still written). */
elrt_status elrt_solve_field(elrt_ctx* ctx, const elrt_field* field, const elrt_solve_opts* opts, double* mean,
                             double* skeleton, elrt_field_stats* stats);

/* Many independent fields of uneven sizes and degrees in one call.  ctxs[k] (k < n_ctx) are
 * contexts of distinct discretisations; field f uses ctxs[field_ctx[f]].  Fields are processed in
 * waves whose operators fit in wave_bytes of device memory (0: 64 GiB): within a wave the local
 * stages of all fields that share a discretisation run as one batched build (one launch sequence),
 * then the skeleton solves run concurrently on up to `workers` streams (0: 8), each with its own
 * workspace.  means[f]: device [nx nz][(p+1)^2]; stats (host, may be NULL) [n_fields].
 * Synchronises; returns the first non-OK status (a wave in which a local stage fails is the last
 * one attempted; a field whose GMRES stops at max_iter still gets its mean). */
elrt_status elrt_solve_batch(elrt_ctx* const* ctxs, int32_t n_ctx, const elrt_field* fields, const int32_t* field_ctx,
                             int32_t n_fields, const elrt_solve_opts* opts, size_t wave_bytes, int32_t workers,
                             double* const* means, elrt_field_stats* stats);

/* ---------------------------------------------------------------- autotuning */

/* Launch parameters the library picks per discretisation, and an autotuner that measures them (the
 * paper has no counterpart: these are implementation choices of this library):
 *   local_chunk  elements per local-build chunk (0: as many as the workspace budget holds: an
 *                eighth of the device memory, at most 32 GB);
 *   lu_pairs     tensor-core LU schedule: 1 = panels in pairs, the second factored after a rank-64
 *                update of its rows and columns, the rest of the matrix updated by both with one
 *                rank-128 tensor-core update; 0 = panels one at a time with rank-64 updates;
 *   restart      GMRES restart length of solve calls that pass restart = 0 (default 12).
 * elrt_autotune builds the local operators of `field` (device inputs as elrt_solve_field) with
 * every candidate (local_chunk in {0, 512, 1024, ...} below the field's element count, lu_pairs in
 * {1, 0} for ELRT_LOCAL_TF32_IR), timing each by CUDA events (one warm-up, mean of two), keeps the
 * fastest, then solves the skeleton system to rtol with restart lengths {8, 12, 16, 20, 30} and
 * keeps the fastest converged one.  It allocates its own temporary operators (the field's in2out
 * and in2sol in FP32), synchronises, and leaves the context unchanged on failure.  With the
 * environment variable ELRT_TUNE_CACHE naming a file, each result is appended there as one text
 * line, and elrt_create applies the last line that matches the device and the discretisation. */
typedef struct {
    int64_t local_chunk;
    int32_t lu_pairs;
    int32_t restart;
    int32_t n_candidates;      /* configurations timed */
    double local_ms_default;   /* local build with the default parameters */
    double local_ms_best;      /* ... with the chosen ones */
    double solve_ms_default;   /* skeleton solve with restart 12 */
    double solve_ms_best;      /* ... with the chosen restart */
} elrt_tune_report;

elrt_status elrt_autotune(elrt_ctx* ctx, const elrt_field* field, int32_t mode, int32_t refine_steps,
                          double rtol, elrt_tune_report* report);
elrt_status elrt_get_tuning(const elrt_ctx* ctx, int64_t* local_chunk, int32_t* lu_pairs, int32_t* restart,
                            int32_t* tuned);
/* Sets the three parameters by hand (ELRT_EINVAL: local_chunk < 0, lu_pairs not 0/1, restart
 * outside 1..200). */
elrt_status elrt_set_tuning(elrt_ctx* ctx, int64_t local_chunk, int32_t lu_pairs, int32_t restart);

/* ---------------------------------------------------------------- element network (Sec. 2.4) */

/* The learned local solver of eq. param2sol: a fully connected network (Sec. 2.4.1)
 *     x_0 -> x_i = f(A_i x_{i-1} + b_i), i = 1..n_hidden (width units, f = GELU or ELU),
 *     output = A_out x_{n_hidden} + b_out  (linear),
 * mapping an element's coefficients to its (in2out, in2sol) = (A_i2o, A_i2m).  Input x_0: the
 * standardised log kappa_hat (or kappa_hat, desc.features) at the (p+1)^2 nodes and the standardised
 * albedo (Sec. 2.4.1 with sigma_s = omega sigma_e: one coefficient field plus the albedo),
 * zero-padded to a multiple of 64.  Output: the 2(p+1)N x 2(p+1)N in2out entries then the (p+1)^2 x 2(p+1)N in2sol entries,
 * each standardised by its training-set mean and standard deviation.  Weights are FP32 masters
 * with BF16 copies; every GEMM runs on tcgen05 (BF16 in, FP32 accumulate); training minimises the
 * mean absolute error with Adam (Sec. 3.1).  All calls are asynchronous on the network's stream
 * unless stated. */
typedef struct {
    int32_t p;            /* element discretisation the network is built for */
    int32_t n_angles;
    int32_t n_hidden;     /* hidden layers (0 = linear regression), <= 8 */
    int32_t width;        /* hidden width, a multiple of 64 */
    int32_t activation;   /* 0 GELU, 1 ELU */
    uint64_t seed;        /* initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from this seed */
    int32_t features;     /* node inputs before standardisation: 0 log(kappa_hat + 1e-12) (suits lognormal
                             coefficients), 1 kappa_hat itself (Sec. 2.4.1's nodal sigma) */
} elrt_net_desc;

typedef struct {
    int32_t epochs;
    int32_t batch;        /* a multiple of 64 */
    float lr;             /* Adam step size; divided by 10 after each third of the epochs */
    float beta1, beta2, eps;
    uint64_t seed;        /* sample order */
} elrt_train_opts;

elrt_status elrt_net_create(elrt_net** net, const elrt_net_desc* desc, void* stream);
elrt_status elrt_net_destroy(elrt_net* net);
elrt_status elrt_net_set_stream(elrt_net* net, void* stream);
const char* elrt_net_last_error(const elrt_net* net);
/* sizes: number of inputs before padding, padded input width, outputs, layers (hidden + 1), parameters */
elrt_status elrt_net_sizes(const elrt_net* net, int64_t* n_feat, int64_t* n_feat_pad, int64_t* n_out,
                           int32_t* n_layers, int64_t* n_params);

/* Host copies of layer l's parameters (l = 0 .. n_hidden; W is [out][in_pad] row-major):
 * what = 0 W, 1 b, 2 dW (last gradient), 3 db; dir = 0 read into host buf, 1 write from it (W, b).
 * Synchronises. */
elrt_status elrt_net_params(elrt_net* net, int32_t layer, int32_t what, int32_t dir, float* host_buf);

/* Checkpoint of a network (the paper has none: it trains once and exports the result): one
 * versioned little-endian binary file with everything training needs to resume bit-for-bit --
 * the description (p, N, n_hidden, width, activation, seed), the FP32 master weights and biases,
 * Adam's first and second moments, the Adam step counter and the input/output standardisation --
 * followed by a CRC-32 (IEEE 802.3) of all preceding bytes.  Layout: a 64-byte header (magic
 * "ELRTNET\0", u32 version 2, i32 p, n_angles, n_hidden, width, activation, u64 seed, i32
 * standardised, i64 Adam step, i64 count F of FP32 values, i32 features), F FP32 values (per layer: W
 * [out][in_pad], b, m(W), v(W), m(b), v(b); then input mean, input std [in_pad], output mean,
 * output std [n_out]), u32 CRC.  BF16 weight copies are rebuilt on load.
 * elrt_net_save synchronises the network's stream and writes `path` (through `path`.tmp and a
 * rename, so a reader never sees a half-written file); ELRT_EINVAL if the file cannot be written.
 * elrt_net_load creates a network from the file on the current device (stream as elrt_net_create);
 * ELRT_EINVAL, with no network created, if the file is missing, truncated, of another version, has
 * an invalid description, a size that does not match it, or a CRC mismatch.
 * elrt_net_file_info validates a file (header, size, CRC) and reports its description,
 * standardisation flag, Adam step and value count without touching a GPU (any pointer may be NULL). */
elrt_status elrt_net_save(elrt_net* net, const char* path);
elrt_status elrt_net_load(elrt_net** net, const char* path, void* stream);
elrt_status elrt_net_file_info(const char* path, elrt_net_desc* desc, int32_t* standardised, int64_t* adam_step,
                               int64_t* n_values);

/* Raw network on standardised features: x device [n][n_feat_pad] FP32 (rounded to BF16 on the
 * way in), y device [n][n_out] FP32 standardised outputs. */
elrt_status elrt_net_forward(elrt_net* net, int64_t n, const float* x, float* y);

/* One training step on a batch of n (a multiple of 64) standardised samples: forward, mean
 * absolute error against t (device [n][n_out] FP32), backward into the gradient buffers, and,
 * if lr > 0, an Adam update (step counter advanced) that also refreshes the BF16 weight copies
 * the GEMMs read.  loss (host, may be NULL) gets the batch MAE; synchronises when loss is given.
 * Device memory: the network keeps buffers for the last batch size it saw, n x (4 n_feat_pad +
 * 10 width n_hidden + 8 n_out) bytes (BF16 activations and their transposes, the output-layer
 * gradient and its transpose, FP32 targets), plus up to 8 x n x width x 4 bytes of FP32 partial
 * products when the output layer's input gradient is split along K because its output tiles
 * alone would not fill the GPU. */
elrt_status elrt_net_train_step(elrt_net* net, int64_t n, const float* x, const float* t, float lr, float* loss);

/* Training from physical data: kappa device [n][(p+1)^2] (km^-1 at the LGL nodes), omega [n],
 * h_elem [n] (element sides, km), labels in2out [n][n_in][n_in] and in2sol [n][(p+1)^2][n_in]
 * (FP32, e.g. from elrt_build_local).  Computes the input and output standardisation from this
 * set, then runs opts->epochs epochs of shuffled mini-batches.  epoch_loss (host, may be NULL)
 * receives the mean batch MAE of every epoch.  Synchronises. */
elrt_status elrt_net_fit(elrt_net* net, int64_t n, const double* kappa, const double* omega, const double* h_elem,
                         const float* in2out, const float* in2sol, const elrt_train_opts* opts, float* epoch_loss);

/* Learned in2out / in2sol (FP32, layouts as elrt_build_local) of n elements with side h (or
 * per-element h_elem).  ELRT_ENOTRAINED if the network has no standardisation yet. */
elrt_status elrt_net_infer(elrt_net* net, int64_t n, double h, const double* h_elem, const double* kappa,
                           const double* omega, float* in2out, float* in2sol);

/* Learned local stage with classical fallback (Sec. 2.4; the error indicator is an energy balance
 * that the exact local operators satisfy): network inference, then the per-element defect
 *     max_j | w_j |s.n|_j - sum_r w_r (s.n)_r A_i2o[r, j] - N sum_i w_i kappa_hat_i (1 - omega) A_i2m[i, j] |
 *           / (w_j |s.n|_j)
 * (exactly 0 for the classical operators), and the classical TF32-IR solve (one refinement sweep)
 * for every element whose defect exceeds tol.  estimate (device [n] FP32, may be NULL) receives the defects; n_fallback
 * (host, may be NULL) the number of re-solved elements.  ctx and net must share (p, N).
 * Synchronises. */
elrt_status elrt_build_local_learned(elrt_ctx* ctx, elrt_net* net, int64_t n, double h, const double* h_elem,
                                     const double* kappa, const double* omega, double tol, float* in2out,
                                     float* in2sol, float* estimate, int64_t* n_fallback);

#ifdef __cplusplus
}
#endif
#endif /* ELRT_H */
