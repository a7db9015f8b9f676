/*
 * pressure_projection.h -- C ABI of the GB300 pressure-projection library.
 *
 * The library solves the implicit pressure equation of the low-Mach
 * two-phase solver of Dalla Barba, Scapin, Rosti, Picano and Brandt,
 * "An interface capturing method for liquid-gas flows at low-Mach number"
 * (arXiv:2005.11806), Sec. 3.3 "Flow solver":
 *
 *   D(rho_f^{-1} G p) = (D u* - S_c) / dt             (Eq. lap_p)
 *   u^{n+1} = u* - dt rho_f^{-1} G p                 (Eq. corr)
 *
 * with Method III (Sec. 3.3.1, Eq. new_poisson, Algorithm 1): a
 * constant-coefficient recast solved iteratively, each pass calling the
 * eigenexpansion Poisson solver: a real FFT in x, a complex FFT in y (a
 * cosine transform with walls in y), and in z a tridiagonal solve per
 * (kx, ky) column (or the tensor-core eigenvector products of PP_MIXED_TC,
 * or the cosine transform of PP_ZSOLVE_COSINE for uniform z).
 *
 * Grid (Sec. 3): marker-and-cell, x periodic and y periodic or walled
 * (uniform spacing), z bounded by no-penetration walls (homogeneous Neumann
 * pressure), uniform or stretched.  Arrays are contiguous, x fastest:
 *   cell fields  (p, rho, S, phi)  [nz][ny][nx]
 *   u            [nz][ny][nx]      u[k][j][i] on the x-face at i - 1/2
 *   v            [nz][ny][nx]      v[k][j][i] on the y-face at j - 1/2
 *   w            [nz+1][ny][nx]    w[k][j][i] on the z-face k (0 and nz: walls)
 * With walls in y (bc[1] = PP_BC_WALL) v keeps its [nz][ny][nx] shape: row
 * j = 0 stands for both walls (y = 0 and y = ly); its input values are taken
 * as zero and it is returned as zero, like the wall planes of w.
 * The face density is the arithmetic mean of the two adjacent cells.  The
 * divergence target S is made compatible with the closed box by removing its
 * volume-weighted mean (S_c = S - <S>_V); p is returned with zero
 * volume-weighted mean.
 *
 * Pointers: every field pointer may be a device pointer or a host pointer
 * (pageable or pinned); the library tells them apart with
 * cudaPointerGetAttributes.  Host pointers are staged through device buffers
 * owned by the plan (allocated on the first call that needs them) with
 * copies on the plan's stream.  The caller owns every field buffer.
 * Errors: every call returns a pp_status and never aborts; on error the
 * output buffers are unspecified.  Plans are not thread-safe; calls on one
 * plan are serialised on its stream.
 */
#ifndef PRESSURE_PROJECTION_H
#define PRESSURE_PROJECTION_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PP_OK = 0,
    PP_ERR_INVALID_ARG = 1,   /* bad pointer, size, tolerance or dt */
    PP_ERR_UNSUPPORTED = 2,   /* grid size with a prime factor > 5, bad bc, or a call not
                                 built for walls in y */
    PP_ERR_NOT_CONVERGED = 3, /* maxit reached before the tolerance */
    PP_ERR_NUMERIC = 4,       /* NaN/Inf in the residual */
    PP_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    PP_ERR_OOM = 6,           /* device allocation failed */
    PP_ERR_TOO_LARGE = 7      /* grid needs more than the fixed no-allocation scratch */
} pp_status;

typedef enum { PP_BC_PERIODIC = 0, PP_BC_WALL = 1 } pp_bc;

typedef enum {
    PP_FP64 = 0,       /* every step in FP64 */
    PP_MIXED_FP32 = 1, /* x/y transforms in FP32; the residual is recomputed exactly in
                          FP64 every 40th pass and updated in FP32 in between (convergence
                          is only accepted on an exact residual); p is kept in FP64; the z
                          tridiagonal solve runs in FP32 on the well-conditioned (kx, ky)
                          columns (condition number <= 513) and in FP64 on the others,
                          the pinned zero mode among them */
    PP_MIXED_TC = 2,   /* as PP_MIXED_FP32, but the z solve is the eigenvector expansion
                          along z (x = V diag(1/(mu + lambda)) V^T W f) as BF16x3 split
                          products on the tensor cores with FP32 accumulation; nz <= 512 */
    PP_MIXED_Z64 = 3   /* as PP_MIXED_FP32, but every z column is solved with FP64
                          recurrences (values stored in FP32) */
} pp_precision;

/* Recast of the variable-coefficient Eq. lap_p into a constant-coefficient
 * iteration (Sec. 3.3.1).  All three are the same iteration
 *     L p^{s+1} = L p^s + r~ (D u^s - S_c) / dt,  u^s = u* - dt beta G p^s,
 * with a different scaling r~ of the residual:
 *   PP_METHOD_III: r~ = rho_c, the cell density (Eq. new_poisson; the default);
 *   PP_METHOD_I:   r~ = min rho over the grid (Eq. poisson_me1), and the
 *                  velocity is the modified correction of Eq. poisson_me2,
 *                  which uses the last and the second-to-last iterate;
 *   PP_METHOD_II:  r~ = 2 rho_min rho_max / (rho_min + rho_max), the
 *                  harmonic mean of the two phase densities taken as the
 *                  extremes of rho (Eq. poisson_laizet), then Eq. corr.
 * The stopping test is the relative norm of D u^s - S_c for all three, so
 * their pass counts compare. */
typedef enum { PP_METHOD_III = 0, PP_METHOD_I = 1, PP_METHOD_II = 2 } pp_method;

/* Solver of the z direction inside each constant-coefficient solve.
 *   PP_ZSOLVE_TRIDIAG: one tridiagonal (Thomas) solve per (kx, ky) column;
 *                      any z spacing (the default).
 *   PP_ZSOLVE_COSINE:  uniform z only: the z eigenbasis of the Neumann
 *                      second difference is cos(pi m (k + 1/2) / nz), so the
 *                      solve is a cosine transform along z (one complex FFT
 *                      of length nz per column), a divide by
 *                      lambda_x + lambda_y - (4/dz^2) sin^2(pi m / (2 nz))
 *                      with the (0, 0, 0) mode set to zero, and the inverse
 *                      transform.  FP64 plans, nz even. */
typedef enum { PP_ZSOLVE_TRIDIAG = 0, PP_ZSOLVE_COSINE = 1 } pp_zsolve;

typedef struct {
    int nx, ny, nz;        /* cells; nx, ny have prime factors in {2,3,5}; nx even;
                              ny even with walls in y */
    double lx, ly, lz;     /* domain lengths */
    const double* zfaces;  /* host, nz+1 finite, strictly increasing face coordinates, or
                              NULL (uniform); read during the call only.  Any other
                              values: PP_ERR_INVALID_ARG from every entry point that takes
                              a grid, before any CUDA call */
    int bc[3];             /* {PP_BC_PERIODIC, PP_BC_PERIODIC, PP_BC_WALL}, or walls in y:
                              {PP_BC_PERIODIC, PP_BC_WALL, PP_BC_WALL}.  With walls in y the
                              y transform is the cosine eigenbasis of the Neumann second
                              difference, cos(pi m (j + 1/2) / ny), eigenvalues
                              -(4/dy^2) sin^2(pi m / (2 ny)), computed by one complex FFT
                              of length ny; pressure_solve, pressure_correct (Methods I, II
                              and III), pressure_solve_adjoint, pressure_mixture_density, the
                              thermodynamic source (adiabatic y walls) and the predictor
                              (no-slip y walls) take them, and so do the allocation-free
                              solve and the batched entry points (per grid) */
    const double* yfaces;  /* host, ny+1 increasing face coordinates spanning ly, or NULL
                              (uniform y).  Walls in y only (PP_ERR_UNSUPPORTED otherwise),
                              2 <= ny <= 1024, any parity.  The y step of the eigenexpansion
                              solve is then the W-orthonormal eigenbasis V of the y part of L
                              (W^{-1} T, W = diag(dyf), T the symmetric second difference
                              with centre distances dyc), computed once on the host by Sturm
                              bisection and inverse iteration: forward V^T W f and back V c
                              as dense products per z plane (Sec. 3.3.1 needs homogeneous
                              conditions only).  pressure_solve, pressure_correct (Methods
                              I, II, III), pressure_solve_adjoint, pressure_mixture_density
                              and the thermodynamic source (pressure_p0_rate,
                              pressure_divergence_source) take it; the predictor returns
                              PP_ERR_UNSUPPORTED; PP_ERR_INVALID_ARG for faces that are not
                              finite, do not increase or do not span ly (1e-12 relative). */
} pp_grid;

typedef struct {
    int iters;             /* constant-coefficient solves performed (Algorithm 1's s) */
    double res0;           /* ||D u* - S_c||_2 */
    double res_final;      /* ||D u^{n+1} - S_c||_2 / res0 at exit */
    double res_l1_sum;     /* Algorithm 1's epsilon: sum over cells of |D u^{n+1} - S_c| */
    double mean_S_removed; /* <S>_V */
    int status;            /* pp_status of the iteration */
} pp_info;

typedef struct pp_plan_s* pp_plan;

/* Create a plan for one grid: eigenvalues, twiddles, z coefficients and the
 * inverse Thomas pivots are computed once; every workspace of the solves is
 * allocated here.  stream is a cudaStream_t (NULL = legacy default stream).
 * Follows Sec. 3 (grid) and Sec. 3.3.1 (homogeneous pressure BCs). */
pp_status pressure_plan_create(const pp_grid* grid, pp_precision prec, void* stream,
                               pp_plan* out);

pp_status pressure_plan_destroy(pp_plan plan);

/* Select the iteration of pressure_correct and pressure_solve_adjoint
 * (pp_method; plans start with PP_METHOD_III).  Method I on an FP64 plan
 * allocates one more FP64 cell field here (the last increment of p).
 * Returns PP_ERR_INVALID_ARG for an unknown method, PP_ERR_OOM when that
 * allocation fails. */
pp_status pressure_plan_set_method(pp_plan plan, int method);

/* Select the z solve (pp_zsolve; plans start with PP_ZSOLVE_TRIDIAG) of
 * every later solve on this plan.  PP_ZSOLVE_COSINE allocates its tables
 * (twiddles and eigenvalues of length nz) on first use.  Returns
 * PP_ERR_INVALID_ARG for an unknown value, PP_ERR_UNSUPPORTED unless the
 * plan is FP64 with uniform z faces (within 1e-12 relative) and even
 * nz <= 2048, PP_ERR_OOM when an allocation fails.  Both solves reach the
 * same discrete solution (Sec. 3.3.1: the eigenexpansion solve is exact). */
pp_status pressure_plan_set_zsolve(pp_plan plan, int zsolve);

/* Constant-coefficient solve by the eigenexpansion method (Sec. 3.3.1):
 * the zero-mean p with D G p = f - <f>_V.  f, p: cell fields. */
pp_status pressure_solve(pp_plan plan, const double* f, double* p, pp_info* info);

/* Eq. 22 with H replaced by the volume fraction Phi:
 * rho = rho_g phi + rho_l (1 - phi).  phi, rho: cell fields. */
pp_status pressure_mixture_density(pp_plan plan, const double* phi, double rho_g, double rho_l,
                                   double* rho);

/* ---- the divergence source from the thermodynamics --------------------
 * div(k grad T) is evaluated as D(k_f G T) on the MAC grid (second-order
 * central, Sec. 3.2): k_f is the arithmetic mean of the two cells of a face,
 * the z walls (and the y walls of a plan with walls in y) are adiabatic (no
 * heat flux), x (and otherwise y) periodic.
 *
 * Rate of the thermodynamic pressure, Eq. 30 (the discrete form of Eq.
 * final_p0):
 *   RP = (gamma / V_g) [ (gamma - 1)/gamma sum Phi div(k grad T) dV
 *                        - p0 sum Phi div(u) dV ],
 * with V_g = sum Phi dV (Eq. v_gas) and dV = dx dy dzf_k.
 * In: phi (gas volume fraction), kc (conductivity), T (temperature): cell
 * fields; u, v, w: faces (w wall planes are taken as zero); p0 and gamma.
 * Out: *rp, on the host; the call waits for the GPU.  PP_ERR_NUMERIC when
 * there is no gas (V_g = 0); PP_ERR_INVALID_ARG for gamma <= 0 or a
 * non-finite p0. */
pp_status pressure_p0_rate(pp_plan plan, const double* phi, const double* kc, const double* T,
                           const double* u, const double* v, const double* w, double p0,
                           double gamma, double* rp);

/* Sec. 3.3: (dp0/dt)^{n+1} extrapolated in time from RP^n and RP^{n-1},
 *   (1 + dt_new/dt_old) rp_n - (dt_new/dt_old) rp_nm1,
 * into *out (host arithmetic only).  PP_ERR_INVALID_ARG for non-positive
 * time steps. */
pp_status pressure_dp0dt_extrapolate(double rp_n, double rp_nm1, double dt_new, double dt_old,
                                     double* out);

/* Divergence source, Eq. 34:
 *   S = (1/p0) [ (gamma - 1)/gamma div(k grad T) - dp0dt / gamma ] Phi,
 * the S that pressure_correct takes.  In: phi, kc, T (cell fields), p0 != 0,
 * gamma > 0, dp0dt (the extrapolated rate).  Out: S (cell field).  Enqueued
 * on the plan's stream (waits only when S is a host pointer). */
pp_status pressure_divergence_source(pp_plan plan, const double* phi, const double* kc,
                                     const double* T, double p0, double gamma, double dp0dt,
                                     double* S);

/* ---- momentum predictor ------------------------------------------------
 * Eq. 29 (Adams-Bashforth):
 *   u* = u^n + dt_new [ (1 + r/2) RU^n - (r/2) RU^{n-1} ],  r = dt_new / dt_old,
 * forward Euler when ru_prev is NULL (the first step), with Eq. 32
 *   RU = -C(u) + (1/rho_f) [ div tau(mu, u) + f ] + g,
 * C(u) = div(u u) - u div(u) (central divergence form) and the
 * Newton-Stokes stress tau = mu [(grad u + grad u^T) - (2/3)(div u) I]
 * (Sec. 2).  Central second-order MAC differences: products and normal
 * stresses at cell centres, cross products and shear stresses at cell edges
 * (a velocity carried to an edge by the mean of its two values, mu by the
 * mean of the cells around the edge, rho_f by the mean of the face's two
 * cells); periodic x and y (or no-slip y walls on a plan with walls in y:
 * the wall row of v is read and written as zero, the wall shear of u and w
 * is taken over half a cell), no-slip z walls.  The surface-tension force of
 * the VOF model is out of scope: force (three face fields, or NULL) may
 * carry any body force, added to div tau.
 * In: u, v, w (faces of u^n; w wall planes zero), rho, mu (cell fields),
 * gravity[3], dt_new > 0, dt_old (> 0 with ru_prev), ru_prev[3] (RU^{n-1}
 * on the faces, or NULL).  Out: u_star[3] (u*, v*, w*; w wall planes zero),
 * ru_out[3] (RU^n for the next step, or NULL).  Device pointers only
 * (PP_ERR_INVALID_ARG otherwise); enqueued on the plan's stream.  Uses the
 * plan's workspace, so it must not overlap a pressure_correct on the same
 * plan. */
pp_status pressure_predictor(pp_plan plan, const double* u, const double* v, const double* w,
                             const double* rho, const double* mu, const double* const force[3],
                             const double gravity[3], double dt_new, double dt_old,
                             const double* const ru_prev[3], double* const u_star[3],
                             double* const ru_out[3]);

/* Method III projection (Algorithm 1, Sec. 3.3.1; Eqs. new_poisson, corr),
 * or Method I or II when pressure_plan_set_method selected one.
 * In: us, vs, ws (u*, faces; ws wall planes are taken as zero), rho (cell
 * density, > 0), S (divergence target, Eq. 34; may be NULL for zero), dt > 0,
 * p (cell field; used as the initial iterate when warm_start != 0).
 * Out: p (zero mean), u, v, w (u^{n+1}; w wall planes written as zero).
 * Stops when ||D u^s - S_c||_2 <= rtol ||D u* - S_c||_2 or after maxit
 * constant-coefficient solves (status PP_ERR_NOT_CONVERGED).  info may be
 * NULL: the call then returns without waiting for the GPU and the iteration
 * status stays on the device (read it later with pressure_last_info). */
pp_status pressure_correct(pp_plan plan, const double* us, const double* vs, const double* ws,
                           const double* rho, const double* S, double dt, double* p,
                           int warm_start, double* u, double* v, double* w, double rtol,
                           int maxit, pp_info* info);

/* Adjoint of the converged projection (Eqs. lap_p, corr differentiated at
 * the fixed point of Algorithm 1).  In: rho, p (the converged pressure of
 * the forward call with the same rho and dt), gu, gv, gw = dL/du^{n+1}.
 * Out: gus, gvs, gws = dL/du*, grho = dL/drho (cell field).  The transposed
 * system is solved by the same Method III loop.  Wall entries of gw (and,
 * with walls in y, the wall row j = 0 of gv) are ignored and those of gws
 * (and of gvs) are written as zero: they are not unknowns. */
pp_status pressure_solve_adjoint(pp_plan plan, const double* rho, const double* p, double dt,
                                 const double* gu, const double* gv, const double* gw,
                                 double* gus, double* gvs, double* gws, double* grho,
                                 double rtol, int maxit, pp_info* info);

/* Constant-coefficient FP64 solve (same result as pressure_solve on an FP64
 * plan) that allocates no device memory.  The paper has no counterpart: this
 * entry point serves callers that cannot call cudaMalloc, e.g. hosts whose
 * device memory belongs to an external pool or budget, or loops that must
 * not enter an allocator.  Working memory is one fixed 16 MiB device array
 * inside the library, held by every GPU that loads the library until the
 * process exits; grids whose spectral array, pivots and tables do not fit
 * return PP_ERR_TOO_LARGE (about 128 x 128 x 64 cells fit).  Grids are
 * periodic in x, periodic or walled in y (bc = {PERIODIC, PERIODIC, WALL}
 * or {PERIODIC, WALL, WALL}: the cosine y basis, ny even), walled in z, with
 * uniform y (yfaces NULL); nx even, nx and ny with prime factors in
 * {2, 3, 5} and at most 2048 (else PP_ERR_UNSUPPORTED); zfaces (host,
 * nz + 1 increasing values, or NULL) is
 * read during the call only.  f and p must be device pointers (host
 * pointers return PP_ERR_INVALID_ARG); the caller owns them.  Every table
 * is computed on the device, so the call copies nothing from the host: it
 * enqueues its kernels on `stream` (a cudaStream_t) and returns PP_OK
 * without waiting for the GPU.  No device-side status is reported: errors
 * found before the launches are returned, and the result is ready once the
 * stream reaches it.  The first call on a device looks up the array's
 * device address with that device current; make that first call before any
 * stream capture.  Calls on one device share its array and each overwrites
 * what the previous one left: calls that may overlap on the same device
 * (different streams) race and must be ordered by the caller.  Calls on
 * different devices use separate arrays. */
pp_status pressure_solve_noalloc(const pp_grid* grid, const double* f, double* p, void* stream);

/* ---- batched projections of independent grids -------------------------
 * Method III projections (Algorithm 1, Sec. 3.3.1) of ngrids independent
 * grids of different sizes, mixed precision only (PP_MIXED_FP32), solved
 * together (each grid periodic in x, periodic or walled in y with uniform
 * spacing, walled in z): each stage of a pass is one grouped launch over the tiles of all
 * grids, and one call is one CUDA graph launch holding the set-up, a
 * device-side while loop over passes (each grid stops at its own tolerance
 * or maxit; the loop ends when all have stopped) and the correction.
 * Creation allocates every workspace, computes every grid's tables, times
 * candidate tile sizes of the transform kernels on the batch and keeps the
 * fastest, and builds the graph.  Fields of all grids are packed: grid g's
 * cell fields start at element cell_offset[g] of every packed cell buffer,
 * its w field at wface_offset[g] of the packed w buffer
 * (pressure_batch_layout).  Packed buffers are device pointers.  The
 * correct call waits for the GPU and fills infos[ngrids] (may be NULL); it
 * returns PP_OK when every grid converged, else the first failing status. */
typedef struct pp_batch_s* pp_batch;

pp_status pressure_batch_create(const pp_grid* grids, int ngrids, pp_precision prec, void* stream,
                                pp_batch* out);
/* cell_offset, wface_offset: ngrids entries each (may be NULL); totals[2] =
 * packed cell and w lengths; tiles[2] = the tuner's elements-per-thread
 * choice for the x and y transform kernels. */
pp_status pressure_batch_layout(pp_batch batch, long long* cell_offset, long long* wface_offset,
                                long long* totals, int* tiles);
/* Eq. 22 over the packed cell fields of every grid (device pointers). */
pp_status pressure_batch_mixture_density(pp_batch batch, const double* phi, double rho_g, double rho_l,
                                         double* rho);
pp_status pressure_batch_correct(pp_batch batch, const double* us, const double* vs, const double* ws,
                                 const double* rho, const double* S, double dt, double* p, double* u,
                                 double* v, double* w, double rtol, int maxit, pp_info* infos);
pp_status pressure_batch_destroy(pp_batch batch);

/* Wait for the plan's stream and fill info from the last pressure_correct
 * or pressure_solve_adjoint call. */
pp_status pressure_last_info(pp_plan plan, pp_info* info);

/* Per-kernel timing (no counterpart in the paper: instrumentation of this
 * library).  When enabled, every kernel launch of the plan is bracketed by
 * CUDA events on the plan's stream; pressure_profile_read waits for the
 * stream and returns, per kernel name, the launch count and the summed
 * event-timed duration since the last enable.  The launch counter counts
 * the plan's own kernel launches whether or not timing is enabled.
 * out may be NULL to query the count; *n receives the number of entries. */
typedef struct {
    char name[32];
    long long launches;
    double total_ms;
} pp_kernel_time;

pp_status pressure_profile_enable(pp_plan plan, int enable);
pp_status pressure_profile_read(pp_plan plan, pp_kernel_time* out, int max_entries, int* n,
                                long long* total_launches);

const char* pressure_status_string(pp_status s);

#ifdef __cplusplus
}
#endif
#endif
