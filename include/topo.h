/*
 * topo.h -- C-ABI of the GB300 (sm_103a) homogenized-multigrid topology
 * optimisation hot path (arXiv 2201.12931, "Efficient hybrid topology
 * optimization using GPU and homogenization based multigrid approach").
 *
 * Problem: minimise the compliance c = f^T u subject to K(rho) u = f
 * (Sec. 2, Eq. topopt) on a structured grid of nx*ny*nz unit 8-node brick
 * elements with the SIMP modulus E(rho) = Emin + rho^p (E0 - Emin)
 * (Eq. K_mod read with K_min = (Emin/E0) K0).  The state equation is solved
 * by CG (Algorithm 1) preconditioned with a Jacobi-smoothed geometric
 * multigrid V-cycle (Algorithm 3) whose coarse operators are formed on the
 * fly from homogenized densities (Sec. 4.2.2, Sec. 6; optionally from
 * averaged moduli, or stored Galerkin element matrices, see
 * topo_params.homogenize); K.u is applied element by element from one
 * reference matrix K0 (Sec. 4.2.1).  Around the solve: compliance and
 * sensitivity, the density filter and its transpose, the OC update, the
 * paper's sensitivity filter with the OC step on the design's own volume,
 * passive (non-design) elements, and the design-dependent self-weight load.
 *
 * Conventions shared by every call
 *   - element id e = i + nx*(j + ny*k); node id n = i + (nx+1)*(j + (ny+1)*k);
 *     DOF 3*n + c, c = 0,1,2 for x,y,z (node-major, "interleaved").
 *   - "device pointer": memory of the CUDA device that was current when the
 *     handle was created (e.g. a torch CUDA tensor's data_ptr()).  The caller
 *     owns it; the library only borrows it for the duration of the call and
 *     keeps no reference.  Device pointers must be 8-byte aligned.
 *   - all GPU work is enqueued on the stream given to topo_create_grid.
 *     Calls that return host values (compliance, iteration counts, change)
 *     synchronise that stream before returning; the others return after
 *     enqueueing and the caller orders later use on the same stream.
 *   - errors are reported by the status code only (no exit, no trap); the
 *     message of the last failure is available from topo_last_error.  After
 *     TOPO_CUDA the handle may be unusable and should be destroyed.
 *   - a handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef TOPO_GB300_H
#define TOPO_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct topo_grid* topo_handle;

typedef enum {
    TOPO_OK = 0,
    TOPO_BADARG = 1,     /* invalid argument; nothing was enqueued            */
    TOPO_OOM = 2,        /* device allocation failed                          */
    TOPO_MAXITER = 3,    /* solver stopped at its iteration cap or stagnated; */
                         /* the best iterate and its residual are returned    */
    TOPO_BREAKDOWN = 4,  /* CG breakdown (p^T K p <= 0, NaN or Inf)           */
    TOPO_CUDA = 5        /* a CUDA runtime call failed                        */
} topo_status;

typedef enum {
    TOPO_FP64 = 0,       /* all vectors and arithmetic in FP64                */
    TOPO_MIXED = 1,      /* FP32 inner MGPCG inside FP64 iterative refinement */
    TOPO_MIXED_BF16 = 2, /* as TOPO_MIXED, V-cycle iterates stored in BF16 on */
                         /* all levels above the coarsest (FP32 arithmetic)  */
    TOPO_DF32 = 3,       /* step-level K.u and residual only (not a handle    */
                         /* precision): FP64 vectors and moduli, arithmetic  */
                         /* in double-FP32 pairs on the FP32 pipe -- the     */
                         /* outer residual of the mixed solves               */
    TOPO_FP32_TC = 4     /* step-level K.u, Jacobi sweep and residual only:   */
                         /* the FP32 operator with its element products on   */
                         /* the tensor cores (topo_params.tensor_cores)      */
} topo_precision;

/* Solver and material parameters.  Defaults from topo_default_params. */
typedef struct {
    double E0;          /* Young's modulus of solid material (1.0)                  */
    double Emin;        /* modulus of void (1e-9)                                   */
    double nu;          /* Poisson ratio (0.3), 0 <= nu < 0.5                       */
    double penal;       /* SIMP exponent p (3.0)                                    */
    int levels;         /* multigrid levels L >= 1; nx, ny, nz divisible by 2^(L-1) */
    int pre, post;      /* Jacobi sweeps before / after the coarse correction (2,2) */
    double omega;       /* Jacobi damping (0.35); must be < 2/5.318 for an SPD V-cycle */
    int precision;      /* topo_precision (TOPO_FP64)                               */
    double inner_tol;   /* residual reduction asked of each inner FP32 solve (1e-4);  */
                        /* the last one asks only for twice what is still missing */
    int inner_max_it;   /* iteration cap of each inner solve (500)                 */
    int max_refine;     /* cap on outer refinement steps (12)                      */
    int homogenize;     /* coarse operators (Sec. 4.2.2): 0 = SIMP of the mean of  */
                        /* the 8 children's densities (the paper's homogenization, */
                        /* default); 1 = mean of the children's moduli; 2 =       */
                        /* Galerkin P^T K P, stored as coarse element matrices    */
                        /* (576 FP64 + 576 FP32 values per coarse element, levels */
                        /* 1 .. L-1; not with TOPO_MIXED_BF16)                    */
    int graphs;         /* 1: each PCG iteration after the first is replayed from */
                        /* a CUDA graph captured once per handle and precision    */
                        /* (default); 0: direct launches.  Launch profiling       */
                        /* (topo_profile_enable) always launches directly         */
    int outer_residual; /* FP64-accurate residual r = f - K x of the refinement   */
                        /* loop of the mixed modes: 0 = double-FP32 kernel on the */
                        /* FP32 pipe, written straight into the FP32 right-hand  */
                        /* side of the inner solve (default); 1 = FP64 kernel     */
    int tensor_cores;   /* FP32 K.u, Jacobi sweeps and residuals of the inner     */
                        /* solve: 0 = modal kernel on the CUDA cores (default);   */
                        /* 1 = element products K0 (u_e - u_e0) on the tcgen05    */
                        /* tensor cores, TF32 operands split hi + lo (about 22    */
                        /* bits), FP32 accumulation in tensor memory              */
    int cg_check;       /* 0: the host reads r.r after batches of CG iterations   */
                        /* sized from the observed contraction rate (at most 8;   */
                        /* default); 1: after every iteration                     */
} topo_params;

/* Fills *p with the defaults listed above.  TOPO_BADARG if p is NULL. */
topo_status topo_default_params(topo_params* p);

/* Creates a grid of nx*ny*nz elements and allocates all device workspace
 * (vectors of every level; the dense coarsest-grid factor is allocated by the
 * first call that needs it).  `stream` is a cudaStream_t (NULL = legacy
 * default stream).  TOPO_BADARG: non-positive size, size not divisible by
 * 2^(levels-1), bad parameter, or 3 * (nx+1)(ny+1)(nz+1) >= 2^31 (the
 * operator kernels index nodal vectors with 32-bit integers: up to about
 * 715M nodes, e.g. 1152x768x768 elements, a mixed-precision handle of
 * roughly 220 GB).  Calls that need the coarsest-grid solve
 * (topo_solve_state, topo_vcycle) return TOPO_BADARG if that grid has more
 * than 12000 DOFs.
 * TOPO_OOM / TOPO_CUDA: allocation or device failure (no handle returned).
 * Alg. 4 "Initialize" and "Compute K0" (K0 by 2x2x2 Gauss quadrature). */
topo_status topo_create_grid(int nx, int ny, int nz, const topo_params* prm,
                             void* stream, topo_handle* out);

/* Frees the handle and all its device memory (synchronises its stream). */
topo_status topo_destroy_grid(topo_handle h);

/* Sets the physical (filtered) densities rho~ (device, nx*ny*nz FP64, values
 * in [0, 1]) and forms the per-level homogenized moduli (Sec. 4.2.2: coarse
 * density = mean of the 8 children) and the coarsest-grid factorisation.
 * The densities are copied; the pointer is not retained.  TOPO_BADARG for a
 * NULL pointer; values outside [0,1] or NaN make the next solve return
 * TOPO_BADARG. */
topo_status topo_set_density(topo_handle h, const double* rho_dev);

/* Sets Dirichlet DOFs and loads.  fixed_dev: device, 3*nodes uint8, nonzero
 * = DOF held at zero.  f_dev: device, 3*nodes FP64 nodal forces; entries at
 * fixed DOFs are ignored (taken as 0).  Coarse levels fix a DOF iff the
 * coincident fine-node DOF is fixed.  Resets the warm start to u = 0. */
topo_status topo_set_bc_loads(topo_handle h, const uint8_t* fixed_dev, const double* f_dev);

/* Solves K(rho~) u = f (Algorithm 1 with the V-cycle of Algorithm 3 as
 * preconditioner) to ||f - K u||_2 / ||f||_2 <= rel_tol, warm-started from
 * the previous solution of this handle.  In the mixed modes the FP64 outer
 * residual is recomputed after each inner FP32 solve (iterative refinement).
 * max_it caps the total number of inner CG iterations.  u_dev_out (device,
 * 3*nodes FP64) may be NULL.  iters_out / relres_out (host) may be NULL.
 * The FP64 outer residual of the mixed modes is computed by the double-FP32
 * kernel or the FP64 kernel (topo_params.outer_residual).
 * Returns TOPO_MAXITER with the best iterate when not converged, and
 * TOPO_BREAKDOWN when the problem is singular: a non-positive pivot of the
 * coarsest-grid factorisation (too few Dirichlet conditions: no iteration
 * runs and the warm start is returned with its FP64 residual), or
 * non-positive curvature or a non-finite value in CG (the step is not taken:
 * the last finite iterate and its FP64 residual are returned).  The message
 * is in topo_last_error; the handle stays usable (e.g. after
 * topo_set_bc_loads with a well-posed problem). */
topo_status topo_solve_state(topo_handle h, double rel_tol, int max_it,
                             double* u_dev_out, int* iters_out, double* relres_out);

/* Compliance and its sensitivity at the current solution (Eq. compliance
 * objective; Eq. sensitivity with the self-adjoint u* = u):
 *   C = sum_e E(rho~_e) u_e^T K0 u_e  (= f^T u at convergence), FP64 sum,
 *   dc_e = -p rho~_e^(p-1) (E0 - Emin) u_e^T K0 u_e.
 * C_out (host) may be NULL; dc_dev_out (device, nx*ny*nz FP64) may be NULL. */
topo_status topo_compliance_and_sensitivity(topo_handle h, double* C_out, double* dc_dev_out);

/* One state step from host memory (Sec. 4.2: the solver is called from the
 * host program with its own arrays, as the paper's mex interface is): copies
 * the physical density rho_host (host, nx*ny*nz FP64, x fastest; pinned for
 * an asynchronous copy, pageable works) to the device as topo_set_density
 * does, solves as topo_solve_state (from the handle's current solution:
 * topo_reset_solution first for a solve from zero), forms C and dc as
 * topo_compliance_and_sensitivity and copies dc to dc_host_out (host,
 * nx*ny*nz FP64; NULL = not copied).  C_out, iters_out, relres_out: host,
 * may be NULL.  Synchronises the handle's stream before returning; uses a
 * handle-owned device buffer for dc (no allocation per call).  Returns the
 * solve's status (TOPO_MAXITER / TOPO_BREAKDOWN with C and dc of the
 * returned iterate, as topo_solve_state describes), or TOPO_BADARG (NULL
 * rho, boundary conditions not set, density outside [0, 1]) / TOPO_CUDA. */
topo_status topo_state_step_host(topo_handle h, const double* rho_host, double rel_tol, int max_it,
                                 double* C_out, double* dc_host_out, int* iters_out, double* relres_out);

/* Density filter with the weights of Eqs. Neighbourhood / NB_dist
 * (w = r - |x_i - x_e| for element-centre distances below r, cut at the
 * domain boundary and normalised by the in-domain weight sum S_e):
 *   transpose = 0: out_e = sum_i w_ei in_i / S_e
 *   transpose = 1: out_i = sum_e w_ei in_e / S_e
 * in_dev, out_dev: device, nx*ny*nz FP64, must not overlap.  0 < r <= 6
 * (at most 905 neighbour offsets, staged in shared memory). */
topo_status topo_filter(topo_handle h, double r, const double* in_dev, double* out_dev,
                        int transpose);

/* Optimality-criteria update of the design variables x (Eqs. OCUp1, bisect,
 * read as the standard OC step with eta = 1/2, q = 1 and the density-filter
 * chain rule): dc~ = H^T dc, dv~ = H^T 1,
 *   x_new = clamp(x * (max(-dc~, 1e-30) / (lambda dv~))^(1/2), x - move, x + move) in [0,1],
 * lambda by bisection on [0, 1e9] until (l2-l1)/(l1+l2) <= 1e-9 such that
 * mean(H x_new) = volfrac.  rho_dev_inout: device, nx*ny*nz FP64 design x,
 * overwritten by x_new.  dc_dev: device dc/drho~ (from
 * topo_compliance_and_sensitivity).  change_out (host, may be NULL) receives
 * max |x_new - x|. */
topo_status topo_oc_update(topo_handle h, double r, double move, double volfrac,
                           double* rho_dev_inout, const double* dc_dev, double* change_out);

/* The paper's own filter (Eq. sensitivity filter): the design is the
 * physical density and its sensitivities are smoothed as
 *   out_e = sum_i w_ei rho_i dc_i / (max(gamma, rho_e) S_e),
 * w_ei = max(0, r - |x_i - x_e|) over the neighbourhood cut at the domain
 * boundary, S_e = sum_i w_ei (the weights of topo_filter).  rho_dev, dc_dev,
 * out_dev: device, nx*ny*nz FP64; out must not overlap the inputs.
 * 0 < r <= 6, gamma > 0 (the paper only asks for a small positive value; 1e-3 is typical),
 * else TOPO_BADARG. */
topo_status topo_sensitivity_filter(topo_handle h, double r, double gamma, const double* rho_dev,
                                    const double* dc_dev, double* out_dev);

/* OC update for designs without a density filter (the paper's loop with
 * the sensitivity filter): as topo_oc_update with dc~ = dc_dev (already
 * filtered) and dv~ = 1, the bisection matching mean(x_new) = volfrac.
 * passive_dev (device, nx*ny*nz bytes, may be NULL): 0 active element,
 * 1 passive solid (x_new = 1), 2 passive void (x_new = 0) -- the
 * non-design regions of Sec. 5, Examples 2 and 4; volfrac is then the
 * volume fraction of the active elements (TOPO_BADARG if there are none).
 * Other arguments, bounds, tolerance and errors as topo_oc_update. */
topo_status topo_oc_update_unfiltered(topo_handle h, double move, double volfrac, const uint8_t* passive_dev,
                                      double* rho_dev_inout, const double* dc_dev, double* change_out);

/* Design-dependent self-weight load (Sec. 5, Example 4: gravity load
 * proportional to the material present): element e carries the weight
 * w rho_e in -z, lumped 1/8 to each corner (the consistent load of a
 * constant body force on the trilinear brick):
 *   f_out = f_ext + sum_e rho_e g_e,  g_e = -(w/8) e_z at the 8 corners.
 * rho_dev: device, nx*ny*nz FP64; f_ext_dev: device 3*nodes FP64 or NULL
 * (zero); f_out_dev: device 3*nodes FP64, not overlapping f_ext.  No
 * Dirichlet masking here: pass f_out to topo_set_bc_loads. */
topo_status topo_gravity_load(topo_handle h, double w, const double* rho_dev, const double* f_ext_dev,
                              double* f_out_dev);

/* Adds the load term of the compliance sensitivity with the self-weight
 * load of topo_gravity_load: dc_e += 2 u_e^T g_e = -(w/4) * (sum of u_z at
 * the 8 corners of e), u the handle's current solution (from
 * topo_solve_state).  Call after topo_compliance_and_sensitivity, which
 * gives the stiffness term.  dc_dev_inout: device, nx*ny*nz FP64. */
topo_status topo_gravity_sensitivity(topo_handle h, double w, double* dc_dev_inout);

/* Message of the last failure on this handle ("" if none).  The string is
 * owned by the handle and valid until the next call on it.  With h == NULL
 * returns the message of the last failed topo_create_grid. */
const char* topo_last_error(topo_handle h);

/* ---------------------------------------------------------------------------
 * Step-level entry points.  Each runs one step of the hot path in isolation
 * so that it can be checked against the oracle; the solver uses the same
 * kernels.  Vectors are device, 3*nodes(level) FP64, node-major; `precision`
 * selects the FP64 kernel (TOPO_FP64), the FP32 kernel (TOPO_MIXED: inputs
 * rounded to FP32, result widened to FP64) or, for topo_apply_operator and
 * topo_residual, the double-FP32 kernel (TOPO_DF32: FP64 inputs split into
 * pairs of FP32 numbers, error-free sums and products of Knuth and Dekker,
 * result rounded to FP64; about 2^-44 relative to the element terms instead
 * of FP64's 2^-52), or, for topo_apply_operator, topo_jacobi_sweep and
 * topo_residual, the FP32 kernel with tensor-core element products
 * (TOPO_FP32_TC; TOPO_CUDA if a bounded wait on the tensor cores ran out).  TOPO_BADARG for a level outside [0, levels), a
 * precision the entry point does not offer, or NULL pointers.
 * ------------------------------------------------------------------------- */

/* Grid of a level: elements per axis (l = 0 is the fine grid). */
topo_status topo_level_dims(topo_handle h, int level, int* nx, int* ny, int* nz);

/* y = K_l u with Dirichlet identity rows (y = u at fixed DOFs, fixed u
 * excluded from free rows); K_l = sum_e E_l,e 2^l A_e^T K0 A_e (Sec. 4.2.1,
 * Sec. 4.2.2).  u_dev and y_dev must not overlap. */
topo_status topo_apply_operator(topo_handle h, int level, int precision,
                                const double* u_dev, double* y_dev);

/* One damped-Jacobi sweep u_out = u + omega D^-1 (f - K_l u) (Sec. 3.2,
 * damped Jacobi equation), D the diagonal of K_l. */
topo_status topo_jacobi_sweep(topo_handle h, int level, int precision,
                              const double* u_dev, const double* f_dev, double* u_out_dev);

/* r = f - K_l u (Eq. residual). */
topo_status topo_residual(topo_handle h, int level, int precision,
                          const double* u_dev, const double* f_dev, double* r_dev);

/* Restriction r_{l+1} = I_h^{2h} r_l: transpose of trilinear interpolation,
 * fixed DOFs masked on both levels (Sec. 3.2; restriction matrix of
 * Sec. 4.2.2, rows proportional to (1/4)[1 2 1]).  Output has 3*nodes(l+1). */
topo_status topo_restrict(topo_handle h, int level, const double* fine_dev, double* coarse_dev);

/* Prolongation and correction u_l += I_{2h}^h e_{l+1} (trilinear; no
 * correction at fixed DOFs) (Algorithm 3, "Prolongation correction"). */
topo_status topo_prolong_add(topo_handle h, int level, const double* coarse_dev, double* fine_dev);

/* Homogenized densities of a level (Sec. 4.2.2): out (device, elements of
 * level l, FP64). */
topo_status topo_level_density(topo_handle h, int level, double* rho_dev_out);

/* One V-cycle z = M^-1 r from z = 0 (Algorithm 3, the preconditioner of
 * Algorithm 1), with the direct coarsest solve.  precision: TOPO_FP64,
 * TOPO_MIXED (FP32 vectors and arithmetic) or TOPO_MIXED_BF16 (FP32
 * arithmetic, FP32 right-hand sides and residuals, smoother iterates and
 * prolongated corrections stored in BF16 on every level above the coarsest;
 * the level-0 result is FP32).  r and z: device FP64, 3*nodes each. */
topo_status topo_vcycle(topo_handle h, int precision, const double* r_dev, double* z_dev);

/* Statistics of the last topo_solve_state. */
typedef struct {
    int outer_steps;        /* FP64 residual evaluations after the first         */
    int inner_iters;        /* total CG iterations                               */
    double relres;          /* final FP64 ||f - K u|| / ||f||                   */
    double solve_ms;        /* wall time of the call (host clock, synchronised) */
    int status;             /* topo_status of the solve                          */
    int graph_replays;      /* CG iterations replayed from a captured CUDA graph */
} topo_solve_stats;

topo_status topo_get_stats(topo_handle h, topo_solve_stats* out);

/* Number of this library's kernel launches since the handle was created. */
topo_status topo_launch_count(topo_handle h, long long* out);

/* Sets the warm start of the next solve to u = 0 (no other state changes). */
topo_status topo_reset_solution(topo_handle h);

/* Kernel timing of the fine-level operator kernels.  With on != 0 every
 * fine-level launch of the element-by-element operator (K.u, Jacobi sweep,
 * first sweep from zero, residual) is bracketed by two CUDA events on the
 * handle's stream (up to 65536 launches; later launches are not recorded)
 * and previous records are cleared; on = 0 stops recording. */
topo_status topo_profile_enable(topo_handle h, int on);

/* Synchronises the stream and returns, for operator kind `mode` (0 = K.u,
 * 1 = Jacobi sweep, 2 = residual, 3 = first sweep from zero, 4 = K.p of CG
 * with the direction update p = z + beta p fused in, 5 = the first two
 * pre-smoothing sweeps from zero in one pass), the number of
 * recorded launches and their summed device time in milliseconds, split by
 * kernel precision: index 0 = FP64, 1 = FP32, 2 = FP32 arithmetic with BF16
 * iterates (V-cycle of TOPO_MIXED_BF16), 3 = double-FP32 (outer residual of
 * the mixed solves), 4 = FP32 with tensor-core element products -- arrays of
 * length 5. */
topo_status topo_profile_read(topo_handle h, int mode, long long* launches, double* total_ms);

/* Arithmetic peak of the CUDA cores, measured (instrumentation; no
 * counterpart in the paper): a full-occupancy grid of independent fused
 * multiply-add chains, timed with CUDA events on `stream` (cudaStream_t,
 * NULL = legacy default stream), best of three launches after a warm-up.
 * kind 0 = FP64 FMA, 1 = FP32 FMA, 2 = paired FP32 FMA (f32x2).  Returns
 * TFLOP/s (2 flops per FMA) in *tflops_out and the launch time in *ms_out.
 * Allocates and frees one small output buffer (8 blocks per SM x 256
 * threads x 8 bytes).  TOPO_BADARG for another kind or NULL outputs (message
 * from topo_last_error(NULL)), TOPO_OOM, TOPO_CUDA. */
topo_status topo_measure_peak(int kind, void* stream, double* tflops_out, double* ms_out);

/* Density filter for callers that cannot allocate GPU memory (no counterpart
 * in the paper).  Same result as topo_filter on a handle of the same grid,
 * without a handle: a framework whose caching allocator owns the device
 * memory, or a loop that must not stall on the device-wide synchronisation
 * of cudaMalloc/cudaFree, can call it at any point.  It calls no
 * cudaMalloc, cudaFree or other allocating routine; its scratch (weight sums,
 * divided input, neighbour table) lives in one statically sized array of
 * about 16 MiB that every GPU loading this library holds until the process
 * exits.  The first call on a device looks up that array's address (make it
 * before any stream capture).  Grids of at most 1,048,576 elements
 * (nx*ny*nz) and radii 0 < r <= 6; larger grids return TOPO_BADARG with a
 * message from topo_last_error(NULL).  in_dev/out_dev: device, nx*ny*nz FP64,
 * must not overlap; stream: cudaStream_t (NULL = legacy default stream).
 * All calls share the one array and leave their data in it: calls that can
 * overlap on the GPU (on different streams) race and must be ordered by the
 * caller.  Nothing in the array needs to start at zero. */
topo_status topo_filter_noalloc(int nx, int ny, int nz, double r, const double* in_dev, double* out_dev,
                                int transpose, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TOPO_GB300_H */
