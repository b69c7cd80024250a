/*
 * sllbm.h -- C ABI of the GB300 semi-Lagrangian lattice Boltzmann (SLLBM) library.
 *
 * The library implements the fused pull-streaming + BGK-collision step of the SLLBM for
 * compressible flow of arXiv:1910.13918 (Sec. II): D2Q25 Hermite velocity set (Sec. II.B,
 * Table I), fourth-order equilibrium (Sec. II.A, Eqs. moments), a second population g for the
 * heat-capacity ratio (Sec. II.D), cell-wise Lagrange interpolation of order p <= 4 on
 * Gauss-Lobatto-Chebyshev support points (Sec. II.E, Eq. sl_streaming), and the lattice
 * Boltzmann equations of Eq. streaming_fg (Prandtl number 1, or another through the
 * quasi-equilibrium term of Sec. II.C), with the isothermal configuration of Sec. III.A as an
 * option, and the standard D2Q9 set that Sec. III.A compares D2Q25 with (isothermal).  It also
 * provides the adjoint of one step (D2Q25, Prandtl number 1), which the paper does not have.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an sllbm_status and never aborts or exits.  On failure the context's
 *   message (sllbm_last_error) says what went wrong.
 * - Pointers named *_dev are device pointers owned by the caller (for instance the data_ptr() of
 *   a CUDA tensor); they must stay valid until the enqueued work is done.  *_host pointers are
 *   host memory owned by the caller.
 * - All device work is enqueued on the CUDA stream given at creation (or by sllbm_set_stream).
 *   Functions that return host values synchronise that stream first.
 * - Vertex arrays are row-major [ny][nx] (x fastest).  A population field is
 *   [n_pop][25][ny][nx] with velocity index i = 5a + b, a (b) the D1Q5 index of the x (y)
 *   component in the order of Table I: 0, +sqrt(5-sqrt10), +sqrt(5+sqrt10), -sqrt(5-sqrt10),
 *   -sqrt(5+sqrt10).  Population 0 is f, population 1 is g.  With SLLBM_VEL_D2Q9 it is
 *   [1][9][ny][nx], i = 3a + b with the D1Q3 components 0, +sqrt3, -sqrt3.
 * - The stored state is the post-collision population field (the field the next step
 *   interpolates).  With SLLBM_PREC_F32 / SLLBM_PREC_BF16_STORE it is stored as deviations
 *   f - w_i and g - (2 C_v - D) w_i; with SLLBM_PREC_F64_PLAIN as full populations in double.
 * - The library owns the buffers it allocates internally (ping-pong state, departure tables,
 *   transposed stencils, reduction scratch) and frees them in sllbm_destroy.
 */
#ifndef SLLBM_H
#define SLLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SLLBM_OK = 0,
    SLLBM_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad enum)      */
    SLLBM_ERR_CUDA = 2,         /* a CUDA runtime call failed                               */
    SLLBM_ERR_OOM = 3,          /* device or host allocation failed                         */
    SLLBM_ERR_STATE = 4,        /* call order: e.g. step before precompute/init             */
    SLLBM_ERR_NEWTON = 5,       /* Newton inversion of the grid map did not converge        */
    SLLBM_ERR_UNSTABLE = 6,     /* a non-finite or non-positive density/temperature was seen */
    SLLBM_ERR_UNSUPPORTED = 7   /* order outside 1..4, unknown velocity set, ...            */
} sllbm_status;

typedef enum { SLLBM_BC_PERIODIC = 0, SLLBM_BC_ZERO_GRADIENT = 1 } sllbm_bc;
typedef enum { SLLBM_NODES_GLC = 0, SLLBM_NODES_EQUIDISTANT = 1 } sllbm_nodes;
typedef enum {
    SLLBM_MAP_IDENTITY = 0,
    /* x = xi + a sin(2 pi xi) sin(pi eta),  y = eta + a sin(pi xi) sin(2 pi eta),  a = map_param[0].
     * A boundary-preserving transformation of the reference box (cf. the transformed grid of
     * Sec. III.E); it needs the reference box [0, 2] x [0, 1] or any box it maps onto itself. */
    SLLBM_MAP_SINE = 1
} sllbm_map;
/* D2Q25: tensor product of the D1Q5 Gauss-Hermite rule (Sec. II.B, Table I), the method's set.
 * D2Q9: tensor product of the three-point rule (0, +-sqrt3; weights 2/3, 1/6, 1/6), with the same
 * fourth-order equilibrium (Sec. III.A); isothermal only (params.isothermal = 1, so cv = 1), plain
 * BGK (pr 0 or 1), no adjoint and no equilibrium VJP (UNSUPPORTED otherwise).  Its state is one
 * population in planar storage for every precision. */
typedef enum { SLLBM_VEL_D2Q25_HERMITE = 0, SLLBM_VEL_D2Q9 = 1, SLLBM_VEL_D3Q125 = 2 } sllbm_velset;
typedef enum {
    SLLBM_PREC_F32 = 0,         /* fused FP32 step, FP32 deviation storage                   */
    SLLBM_PREC_BF16_STORE = 1,  /* fused step with FP32 arithmetic and BF16 deviation storage */
    SLLBM_PREC_F64_PLAIN = 2    /* plain FP64 step on full populations (accuracy baseline)   */
} sllbm_prec;

/* Grid of nx_cells x ny_cells Lagrange cells of order `order` on the reference box
 * [x0,x1] x [y0,y1] (Sec. II.E).  Cells share their boundary vertices.  A periodic axis has
 * cells*order vertices, a zero-gradient axis cells*order + 1.  Enum fields are plain ints. */
typedef struct {
    int nx_cells, ny_cells, order;
    double x0, x1, y0, y1;
    int bc_x, bc_y;             /* sllbm_bc    */
    int nodes;                  /* sllbm_nodes */
    int map;                    /* sllbm_map   */
    double map_param[4];
} sllbm_grid_desc;

/* Time step, relaxation time tau = nu / (c_s^2 dt) + 1/2 (Sec. II.D), heat capacity C_v
 * (gamma = 1 + 1/C_v with R = 1; C_v = D/2 = 1 leaves g identically zero and the library then
 * carries f only), reference temperature T0 (must be 1: c_s^2 = R T0 = 1), precision, and the
 * Prandtl number pr (Sec. II.C, Eq. streaming_fg): 1 (or 0, which reads as 1) is plain BGK;
 * any other positive value adds (1/tau - 1/tau_Pr) f^qe, tau_Pr = (tau - 1/2)/Pr + 1/2, with the
 * quasi-equilibrium f^qe_i = w_i Q^neq : H^(3)(xi_i) / 3! of the non-equilibrium centred third
 * moment (and the same projection of g's own for g).  The adjoint covers Pr = 1 only.
 * isothermal = 1 evaluates the equilibrium at theta = 1 (the isothermal configuration of the
 * moving Taylor-Green vortex, Sec. III.A): mass and momentum are conserved, energy is not; it
 * requires cv = 1 (one population). */
typedef struct {
    int velset;                 /* sllbm_velset */
    double dt, tau, cv, T0;
    int prec;                   /* sllbm_prec   */
    double pr;                  /* Prandtl number; 0 or 1: plain BGK */
    int isothermal;             /* 1: equilibrium at theta = 1 (Sec. III.A); needs cv = 1 */
} sllbm_params;

typedef struct sllbm_ctx sllbm_ctx;  /* opaque, library-owned */

/* Create a context: validates the descriptors, builds the velocity set and support points in
 * FP64 on the host, allocates the state and tables on the current CUDA device.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  Errors: ARG, UNSUPPORTED, OOM, CUDA. */
sllbm_status sllbm_create(const sllbm_grid_desc* grid, const sllbm_params* params,
                          void* cuda_stream, sllbm_ctx** out);
sllbm_status sllbm_destroy(sllbm_ctx* ctx);
sllbm_status sllbm_set_stream(sllbm_ctx* ctx, void* cuda_stream);

/* Vertex counts per axis and number of populations carried (2, or 1 when C_v = 1). */
sllbm_status sllbm_grid_info(const sllbm_ctx* ctx, int* nx_vertices, int* ny_vertices, int* n_pop);

/* Bytes of one population field in the context's storage type: n_pop * 25 * ny * nx * elem. */
sllbm_status sllbm_state_bytes(const sllbm_ctx* ctx, size_t* bytes);

/* Physical vertex coordinates (Sec. II.E support points mapped by the grid transformation),
 * FP64, written to caller-owned device arrays of nx*ny doubles. */
sllbm_status sllbm_vertex_coords(sllbm_ctx* ctx, double* x_dev, double* y_dev);

/* Vertex quadrature weights A_v = integral of the shape function of vertex v over the domain
 * (with |det J| on transformed grids), FP64, nx*ny doubles.  sum_v A_v rho_v is the mass of the
 * interpolant (the m of Sec. III.E, mass conservation). */
sllbm_status sllbm_vertex_weights(sllbm_ctx* ctx, double* A_dev);

/* Departure points x_v - dt xi_i of every vertex and velocity (Eq. streaming_fg), folded into the
 * domain (periodic: wrap, zero-gradient: clamp), the containing cell, the local reference
 * coordinates (Newton inversion of the map in FP64 on transformed grids) and the Lagrange weights
 * of Eq. sl_streaming.  FP64 arithmetic on the GPU; FP32 (and FP64 for the plain step) tables.
 * Must precede sllbm_init_equilibrium/step/adjoint.  Errors: NEWTON, CUDA. */
sllbm_status sllbm_precompute_departures(sllbm_ctx* ctx);

/* Initial state: the equilibrium f^eq(rho, u, T) (Sec. II.A) and g^eq = (2 C_v - D) theta f^eq
 * (Sec. II.D) at every vertex.  rho, u, v, T: caller-owned device arrays of nx*ny doubles. */
sllbm_status sllbm_init_equilibrium(sllbm_ctx* ctx, const double* rho_dev, const double* u_dev,
                                    const double* v_dev, const double* T_dev);

/* Advance nsteps time steps: per step and vertex, interpolate the post-collision populations of
 * every velocity at its departure point (Eq. sl_streaming), take the moments (rho, rho u,
 * 2 rho E of Sec. II), relax toward the equilibrium with 1/tau (Eq. streaming_fg, Pr = 1) and
 * store the post-collision populations.  Enqueues only; returns without synchronising.  On grids
 * whose state (sllbm_state_bytes) is at most 64 MB, small enough for L2 and bound by launch
 * overhead, a call of 4 or more steps on a stream other than the legacy default stream replays
 * pairs of steps as a CUDA graph, captured at the first such call (the same launches with the
 * same parameters; the result is the same bit for bit). */
sllbm_status sllbm_step(sllbm_ctx* ctx, int nsteps);

/* One step as sllbm_step that also writes, per vertex, the moments its collision was evaluated
 * at: the density, velocity and temperature of the interpolated pre-collision populations (Sec.
 * II: rho = sum f, rho u = sum f xi, T from 2 rho E = sum f |xi|^2 + sum g; theta = T / T0).
 * BGK conserves them, so away from FP32 rounding they are the moments sllbm_moments returns for
 * the state the step produced -- the saved_moments of sllbm_adjoint_step (in the isothermal
 * configuration, whose collision does not keep the energy, they are the pre-collision ones).
 * moments_dev: caller-owned device FP32 [4][ny][nx] = (rho, u, v, theta), written by the step
 * kernels themselves (no second pass over the state).  D2Q25 only (else UNSUPPORTED); enqueues
 * only. */
sllbm_status sllbm_step_moments(sllbm_ctx* ctx, float* moments_dev);

/* Same step with host buffers: copies the state (sllbm_state_bytes bytes, dense layout) from
 * state_in_host to the device, advances nsteps, copies it back to state_out_host and
 * synchronises.  Pinned host memory gives the full link bandwidth. */
sllbm_status sllbm_step_host(sllbm_ctx* ctx, const void* state_in_host, void* state_out_host,
                             int nsteps);

/* Macroscopic fields of the current state: rho, u, v and T = theta T0 (FP32 device arrays of
 * nx*ny floats, any of them may be NULL), and optionally the FP64 sums
 * mass_energy_host[0] = sum_v A_v rho_v, mass_energy_host[1] = sum_v A_v rho_v E_v
 * (deterministic two-pass reduction; synchronises).  Returns SLLBM_ERR_UNSTABLE (after writing
 * the outputs) if any vertex has a non-finite or non-positive density or temperature. */
sllbm_status sllbm_moments(sllbm_ctx* ctx, float* rho_dev, float* u_dev, float* v_dev,
                           float* T_dev, double* mass_energy_host);

/* Checkpoint/resume: copy the current state to / from a caller-owned device buffer of
 * sllbm_state_bytes bytes in the dense layout [n_pop][25][ny][nx]. */
sllbm_status sllbm_get_state(sllbm_ctx* ctx, void* dst_dev);
sllbm_status sllbm_set_state(sllbm_ctx* ctx, const void* src_dev);

/* Adjoint of one step (not in the paper).  The step is s' = C(S s): S the interpolation of every
 * velocity plane, C the pointwise BGK collision.  Given lambda' = dJ/ds' (lambda_in, FP32
 * [2][25][ny][nx] dense, population g included even when C_v = 1) this writes
 * lambda = S^T J_C^T lambda' to lambda_out (same layout; must not alias lambda_in).  J_C is the
 * collision Jacobian at the pre-collision moments of that step, given as saved_moments
 * [4][ny][nx] FP32 = (rho, u, v, theta) -- exactly what sllbm_moments returns for the state the
 * step produced.  S^T is applied as a gather (pull) over precomputed transposed stencils: no
 * atomics, deterministic.  The first call builds the transposed stencils on the host and
 * allocates the context's scratch for J_C^T lambda' (25 FP32 pairs a vertex, with ghost cells on
 * uniform grids); later calls only enqueue.  A staging copy that does not land in time on uniform
 * grids makes the next sllbm_moments return SLLBM_ERR_CUDA, as for the step.  Works in every
 * precision mode (FP32 arithmetic); a context with Pr != 1 or the isothermal equilibrium gets
 * SLLBM_ERR_UNSUPPORTED. */
sllbm_status sllbm_adjoint_step(sllbm_ctx* ctx, const float* lambda_in_dev, float* lambda_out_dev,
                                const float* saved_moments_dev);

/* Vector-Jacobian product of the initial equilibrium with respect to the initial velocity:
 * du[v] = sum_i lambda0_f[i][v] d f_i^eq/du + lambda0_g[i][v] d g_i^eq/du at (rho0, u0, v0, T0)
 * (device FP64 arrays of nx*ny), and likewise dv.  lambda0: FP32 [2][25][ny][nx]; du, dv: FP32. */
sllbm_status sllbm_init_equilibrium_vjp(sllbm_ctx* ctx, const double* rho_dev, const double* u_dev,
                                        const double* v_dev, const double* T_dev,
                                        const float* lambda0_dev, float* du_dev, float* dv_dev);

/* Allocation-free moments and mass/energy sums.  The paper has no counterpart; this is for
 * callers that must not allocate device memory: code running inside a framework whose caching
 * allocator has reserved the device memory (a cudaMalloc beside it can fail or fragment),
 * latency-critical loops (cudaFree synchronises the whole device), or callers with a fixed memory
 * budget.  It computes what sllbm_moments computes, without a context:
 *   state_dev: FP32 deviation state in the dense layout of sllbm_get_state, [n_pop][25][ny][nx]
 *              with n_pop = 1 if cv == 1, else 2 (caller-owned, device);
 *   A_dev:     vertex weights (sllbm_vertex_weights, nx*ny doubles) or NULL to skip the sums;
 *   rho/u/v/T: FP32 outputs of nx*ny floats, each may be NULL;
 *   mass_energy_dev: two doubles on the device, written only if A_dev is given (required then,
 *              may be NULL otherwise).
 * Its reduction scratch is a file-scope device array of 1 MiB (the library keeps it on every GPU
 * that loads it until the process exits), so grids are limited to 16,777,216 vertices
 * (SLLBM_ERR_UNSUPPORTED beyond, checked before anything is launched).  Every call looks up that
 * array's device address on the current device (a host-side query, nothing cached), so a call
 * made after the device's context was rebuilt finds the array where it now is.  The first call
 * in a process may load the library's device code; make it before any stream capture.  All
 * calls share the array: calls that overlap on the GPU (other streams, other threads) race;
 * serialise them.  Synchronises cuda_stream; returns SLLBM_ERR_UNSTABLE like sllbm_moments. */
sllbm_status sllbm_moments_noalloc(const float* state_dev, int nx, int ny, double cv,
                                   const double* A_dev, float* rho_dev, float* u_dev, float* v_dev,
                                   float* T_dev, double* mass_energy_dev, void* cuda_stream);

/* Self-test of the bounded waits of the staging pipelines.  The paper has no counterpart: the
 * TMA-staged step kernels wait on mbarriers for their staged tiles with an iteration limit, so
 * that a copy that never lands makes sllbm_moments report SLLBM_ERR_CUDA ("a staging copy ...
 * timed out") instead of hanging the GPU.  This call runs that wait, with a short limit, on an
 * mbarrier nothing arrives on (no copy is involved) and returns SLLBM_OK if the wait ran out and
 * reported it, SLLBM_ERR_CUDA otherwise.  Enqueues one small kernel on cuda_stream and
 * synchronises it; allocates nothing (its flag is a device variable of the library). */
sllbm_status sllbm_selftest_bounded_wait(void* cuda_stream);

/* ------------------------------------------------------------------------------------------
 * 3D extension (the step the paper names as its next one): D3Q125, the tensor product of D1Q5
 * three times, on a uniform grid of hexahedral Lagrange cells of order 1..4 (Sec. II.E per axis),
 * with the same fourth-order equilibrium (Sec. II.A over index tuples in {x, y, z}^n), g^eq =
 * (2 C_v - 3) theta f^eq (Sec. II.D) and BGK (Eq. streaming_fg, Pr = 1).  params.velset =
 * SLLBM_VEL_D3Q125 with params.prec = SLLBM_PREC_F64_PLAIN (plain FP64 step on full populations)
 * or SLLBM_PREC_F32 (fused FP32 step: one launch per step, the state kept as FP32 deviations
 * (f - w, g - K w) side by side; get_state / set_state still exchange FP64 full populations);
 * pr 0 or 1, cv >= 3/2 (cv = 3/2 carries f only; isothermal = 1 needs it).  Population field
 * [n_pop][125][nz][ny][nx], velocity i = 25a + 5b + c (D1Q5 indices of the x, y, z components in
 * Table I order); vertex arrays [nz][ny][nx].  Conventions otherwise as above.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int nx_cells, ny_cells, nz_cells, order;
    double x0, x1, y0, y1, z0, z1;
    int bc_x, bc_y, bc_z;       /* sllbm_bc    */
    int nodes;                  /* sllbm_nodes */
} sllbm_grid3_desc;

typedef struct sllbm3d_ctx sllbm3d_ctx;  /* opaque, library-owned */

/* Create / destroy a 3D context.  Errors: ARG, UNSUPPORTED (other velocity set, precision,
 * Prandtl number, order), OOM, CUDA. */
sllbm_status sllbm3d_create(const sllbm_grid3_desc* grid, const sllbm_params* params,
                            void* cuda_stream, sllbm3d_ctx** out);
sllbm_status sllbm3d_destroy(sllbm3d_ctx* ctx);
/* Vertex counts per axis and populations carried. */
sllbm_status sllbm3d_grid_info(const sllbm3d_ctx* ctx, int* nx, int* ny, int* nz, int* n_pop);
/* Vertex coordinates, FP64 device arrays of nz*ny*nx doubles each. */
sllbm_status sllbm3d_vertex_coords(sllbm3d_ctx* ctx, double* x_dev, double* y_dev, double* z_dev);
/* Per-axis departure tables (stencil start and p+1 Lagrange weights per velocity component and
 * vertex, FP64).  Must precede init and step. */
sllbm_status sllbm3d_precompute_departures(sllbm3d_ctx* ctx);
/* Initial state: f^eq and g^eq of (rho, u, v, w, T) (device FP64 arrays of nz*ny*nx). */
sllbm_status sllbm3d_init_equilibrium(sllbm3d_ctx* ctx, const double* rho_dev, const double* u_dev,
                                      const double* v_dev, const double* w_dev, const double* T_dev);
/* Advance nsteps steps (pull interpolation of every velocity with the tensor-product Lagrange
 * basis, moments, BGK); enqueues only.  FP32 contexts of order 1 or 2 with an even number of x
 * vertices and at least 36 x 12 x 8 vertices take the sum-factorised step (three launches:
 * TMA-staged tiles that interpolate and sum the moments, a sweep that relaxes, a refresh of the
 * periodic images in the state's ghost cells); the others the one-launch gather step.  The
 * sum-factorised step keeps 2 ghost cells on every axis in its state and allocates 6 floats a
 * vertex of scratch at sllbm3d_precompute_departures. */
sllbm_status sllbm3d_step(sllbm3d_ctx* ctx, int nsteps);
/* Name of the kernel sllbm3d_step uses for this context ("stream3d" for the sum-factorised FP32
 * step, "gather_f32", "plain_f64"); valid after sllbm3d_precompute_departures. */
const char* sllbm3d_step_kernel_name(const sllbm3d_ctx* ctx);
/* rho, u, v, w, T of the current state (FP64 device arrays of nz*ny*nx, each may be NULL);
 * synchronises; SLLBM_ERR_UNSTABLE if a step or this call saw a non-positive or non-finite
 * density or temperature, SLLBM_ERR_CUDA if a staging copy of the sum-factorised step did not
 * land within its bounded wait. */
sllbm_status sllbm3d_moments(sllbm3d_ctx* ctx, double* rho_dev, double* u_dev, double* v_dev,
                             double* w_dev, double* T_dev);
/* Copy the state to / from a caller-owned device buffer of n_pop*125*nz*ny*nx doubles. */
sllbm_status sllbm3d_get_state(sllbm3d_ctx* ctx, double* dst_dev);
sllbm_status sllbm3d_set_state(sllbm3d_ctx* ctx, const double* src_dev);
const char* sllbm3d_last_error(const sllbm3d_ctx* ctx);

/* Name of the kernel the step uses for this context ("uniform_fused", "gather", "plain_f64"). */
const char* sllbm_step_kernel_name(const sllbm_ctx* ctx);

/* Number of kernel launches one call of sllbm_step(ctx, 1) enqueues. */
int sllbm_launches_per_step(const sllbm_ctx* ctx);

const char* sllbm_status_string(sllbm_status status);
const char* sllbm_last_error(const sllbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SLLBM_H */
