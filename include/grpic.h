/*
 * grpic.h -- C ABI of the GB300 GRPIC library.
 *
 * One general-relativistic electromagnetic particle-in-cell timestep (Watson & Nishikawa,
 * "A Method for Incorporating General Relativity in Electromagnetic Particle-in-Cell Code",
 * arXiv:0904.0232) on one GPU: the B half-step, the per-particle gather + Kerr metric /
 * Christoffel + RK4 four-velocity push + curved-metric current deposit, the second B
 * half-step and the E step (Sec. 2.2, Fig. 1), followed by horizon / outer-boundary removal
 * and a counting sort of the particles by cell.
 *
 * Conventions shared by every call
 *   - Units: cell size 1 on all axes; x^4 = c t (Sec. 3); indices 1..4 of the paper are 0..3
 *     here (x, y, z, x^4).  The central mass sits at ((nx-1)/2, (ny-1)/2, (nz-1)/2).
 *   - Grid arrays are nz*ny*nx doubles, index (k*ny + j)*nx + i, three components back to
 *     back (3*nz*ny*nx doubles).  Prognostic field components and their Yee locations:
 *       d = F^{x4}, F^{y4}, F^{z4}  (contravariant; edges (i+1/2,j,k), (i,j+1/2,k), (i,j,k+1/2))
 *       b = F_{yz}, F_{zx}, F_{xy}  (covariant;     faces (i,j+1/2,k+1/2), (i+1/2,j,k+1/2),
 *                                                          (i+1/2,j+1/2,k))
 *       J = J^x, J^y, J^z          (contravariant current density, at the d locations)
 *     (Eq. 8 gives F^{4j} = E^j and F^{jk} = eps^{jkl} B^l for the contravariant tensor.)
 *   - Particle arrays are planar: x4 holds x^1[0..n), x^2[0..n), x^3[0..n), x^4[0..n); u4 the
 *     four-velocity u^1..u^4 (u^4 = c dt/dtau) alike.
 *   - Memory: every pointer argument is host memory unless the call's `mem` / flags argument
 *     says GRPIC_MEM_DEVICE, in which case it is device memory of the context's GPU.  The
 *     library copies inputs; outputs go to caller-owned buffers.  The caller keeps ownership
 *     of everything it passes.
 *   - Streams: all device work of a context is ordered on the stream given to grpic_create.
 *     Calls that return data synchronise that stream; grpic_step_async does not.
 *   - Errors: every call returns a grpic_status; nothing is thrown across the ABI.  Device-side
 *     faults (non-finite state, a particle moving a cell or more in one step) are recorded in a
 *     device status word and reported by the next synchronising call; grpic_last_error() gives
 *     a message.  After GRPIC_ERR_CFL or GRPIC_ERR_NONFINITE the state of the step is undefined.
 *   - Thread safety: a context is used by one host thread at a time.
 */
#ifndef GRPIC_H_
#define GRPIC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GRPIC_OK = 0,
  GRPIC_ERR_INVALID = 1,   /* bad argument, or a particle/field input the method cannot take */
  GRPIC_ERR_OOM = 2,       /* device allocation failed */
  GRPIC_ERR_CUDA = 3,      /* a CUDA call failed */
  GRPIC_ERR_CFL = 4,       /* c dt >= 1/sqrt(3) at create, or |dx^i| >= 1 cell in one step */
  GRPIC_ERR_NONFINITE = 5, /* NaN/Inf in particle state */
  GRPIC_ERR_TIMEOUT = 6,   /* a bounded wait gave up */
  GRPIC_ERR_AGAIN = 7,     /* serving: request not finished / not admitted yet */
  GRPIC_ERR_CAPACITY = 8,  /* more particles than the context's capacity */
  GRPIC_ERR_UNSTABLE = 9   /* serving: the request's box is too small for its hole (see grpic_submit) */
} grpic_status;

enum { GRPIC_FP64 = 0, GRPIC_FP32_MIXED = 1 };

enum {
  GRPIC_NO_GAMMA_IN_J = 1u,      /* deposit the plain Umeda flux, without the factor gamma of J = rho gamma v */
  GRPIC_LITERAL_HALF_STEPS = 2u, /* field update with each half-step explicit in its own start value (see below) */
  GRPIC_SINGLE_PUSH_KERNEL = 4u  /* FP32_MIXED: push every particle with the FP32-mixed code (no far-field
                                    path; see grpic_tuning); same policy, for comparison */
};

enum { GRPIC_MEM_HOST = 0, GRPIC_MEM_DEVICE = 1 };

/* grpic_load_particles flags: how u4 is given (bits 0-1) and where the arrays live (bit 4). */
enum {
  GRPIC_U_FULL = 0,          /* u4 holds u^1..u^4 as is */
  GRPIC_U_COV_SPATIAL = 1,   /* planes 0..2 hold covariant u_1..u_3; u^a is completed on the device */
  GRPIC_U_CONTRA_SPATIAL = 2,/* planes 0..2 hold u^1..u^3; u^4 is completed (needs g_44 < 0) */
  GRPIC_LOAD_DEVICE = 16     /* x4, u4, ids are device pointers */
};

/* Pipeline stages for grpic_stage (each is one row of the timestep).
 * Field time levels (Sec. 3: B is advanced in two half-steps around the push, E a full step):
 * the stored b lags d by half a step.  By default the update is time-centred: the first half
 * takes b^{n-1/2} to b^n = b^{n-1/2} - (dx^4/2) curl e(b^{n-1/2}, d^n) for the push; the second
 * gives b^{n+1/2} = b^{n-1/2} - dx^4 curl e(b^n, d^n); the E step evaluates the d-dependence of
 * the contravariant tensor at a midpoint predictor of d.  In Kerr-Schild coordinates e depends
 * on b (and h on d) through the shift, and the literal explicit form (GRPIC_LITERAL_HALF_STEPS:
 * each half-step b -= (dx^4/2) curl e(b, d) from its own start, E step explicit in d) is a
 * forward-Euler step of a centred advection term, which grows without bound. */
enum {
  GRPIC_STAGE_B_HALF = 0,       /* Sec. 3.1, Eq. 10: first B half-step */
  GRPIC_STAGE_ZERO_J = 1,       /* J <- 0 */
  GRPIC_STAGE_PUSH_DEPOSIT = 2, /* Sec. 3.3 + Sec. 4: RK4 push, curved deposit, removal flags */
  GRPIC_STAGE_E = 3,            /* Sec. 3.2, Eq. 12: d <- d + dx^4 (4 pi/c J - div F) */
  GRPIC_STAGE_SORT = 4,         /* counting sort by cell; drops removed particles */
  GRPIC_STAGE_B_HALF2 = 5       /* Sec. 3.1, Eq. 10: second B half-step */
};

/* Absorbing layers (the paper states no boundary condition for the fields).  Without them the
 * outer two index layers and the inside of r_excise are held at their values, which reflects
 * waves; with a rapidly rotating hole that reflection inside the horizon feeds a mode that grows
 * next to it, and where the metric at the box faces is far from flat the frozen faces feed one
 * there.  A layer relaxes the field toward a target: after the second B half-step and the E step
 * every advanced location with relaxation kappa > 0 takes F0 + (1 - kappa)(F - F0), kappa the
 * larger of the two layers' values there (r in FP64 at the location; s = the cell's distance in
 * cells to the nearest frozen layer, 1 for the first advanced cell).  The target F0 is the field
 * of the last grpic_set_fields / grpic_set_uniform_field call (zero before the first).  The inner
 * layer lies inside the horizon, so it acts on nothing that can reach the outside. */
typedef void* (*grpic_alloc_fn)(size_t bytes, void* user);
typedef void (*grpic_free_fn)(void* ptr, void* user);

typedef struct {
  int nx, ny, nz;        /* nodes per axis, each >= 8 */
  double m;              /* mass of the central object, in cells (Eq. 4), >= 0 */
  double a;              /* spin parameter, |a| <= m (Eqs. 4-6) */
  double c;              /* speed of light, cells per unit time */
  double dt;             /* time step; c dt < 1/sqrt(3) is required */
  int precision;         /* GRPIC_FP64 or GRPIC_FP32_MIXED */
  int quad_order;        /* Q of the Q x Q Gauss-Legendre rule of Eq. 18: 1, 2 or 3 (0 -> 2) */
  double r_excise;       /* fields at r < r_excise are frozen; <= 0 -> r_+ (the inside of the horizon) */
  unsigned flags;        /* GRPIC_NO_GAMMA_IN_J */
  int sort_interval;     /* counting sort every k steps (<= 0 -> 1) */
  int64_t max_particles; /* capacity per species (0 -> set by the first load) */
  double fp64_radius;    /* FP32_MIXED: where the FP32 estimate of r is below fp64_radius * m, the quartic,
                            the metric and the Christoffel contraction are evaluated in FP64 (0 -> 4;
                            negative -> never) */
  double absorb_inner;   /* absorbing layer inside the horizon (see below): relaxation per step at
                            r = r_excise, falling linearly to 0 at r = r_+; 0 -> none.  With it,
                            r_excise <= 0 means r_+/2.  In [0, 1] */
  double absorb_outer;   /* absorbing layer at the box faces: relaxation per step at the first advanced
                            cell, falling as ((W + 1 - s) / W)^2 to the s = W-th; 0 -> none.  In [0, 1] */
  int absorb_width;      /* W, in cells (<= 0 -> 8) */
  int z_origin;          /* this context's grid as planes z_origin .. z_origin + nz - 1 of a run whose grid has
                            nz_total planes (one z-slab of a run split across contexts, see
                            paper_0904_0232_gb300/slab.py): the hole sits at the run's centre, z_c =
                            (nz_total - 1)/2 - z_origin; the slab's edge planes are held like faces, so
                            a driver refreshes them from the neighbouring slabs.  0 with nz_total 0:
                            a whole grid.  An outer absorbing layer needs a whole grid */
  int nz_total;          /* planes of the whole run (0 -> nz) */
  grpic_alloc_fn alloc;  /* device allocator (NULL -> cudaMalloc); e.g. a PyTorch caching allocator */
  grpic_free_fn free_fn; /* matching free */
  void* alloc_user;      /* passed to alloc / free_fn */
} grpic_config;

typedef struct {
  int64_t steps;            /* timesteps taken */
  int64_t removed_horizon;  /* particles removed at r <= r_+ */
  int64_t removed_outer;    /* particles removed outside [1, n-2] */
  int64_t gamma_fallbacks;  /* Eq. 16 square-root argument < 0: gamma_1 = u^4/c used */
  int64_t fp64_evals;       /* FP32-mixed: metric evaluations promoted to FP64 (r < 4m region) */
  int64_t particle_steps;   /* particles advanced, summed over steps */
  int64_t n_alive[4];       /* particles per species after the last sort */
} grpic_stats;

typedef struct grpic_ctx grpic_ctx;

/* Create a context on the current CUDA device.  Validates the configuration (Courant:
 * c dt < 1/sqrt(3), Sec. 5), computes r_+ = m + sqrt(m^2 - a^2), and flags every field location
 * as advanced or excised (decided in FP64).  `stream` is a cudaStream_t (NULL = default stream).
 * Returns GRPIC_ERR_INVALID / GRPIC_ERR_CFL on bad input, GRPIC_ERR_OOM if allocation fails. */
grpic_status grpic_create(const grpic_config* cfg, void* stream, grpic_ctx** out);

/* Free all device memory of the context (stream-ordered) and the context itself. */
grpic_status grpic_destroy(grpic_ctx* ctx);

/* Set the prognostic field: d (3 planes, contravariant F^{i4}) and b (3 planes, covariant
 * F_{yz}, F_{zx}, F_{xy}) at their Yee locations (Sec. 3, Fig. 2).  FP32_MIXED rounds them. */
grpic_status grpic_set_fields(grpic_ctx* ctx, const double* d3, const double* b3, int mem);

/* Set a uniform contravariant field (Eq. 8: F^{4j} = E^j, F^{jk} = eps^{jkl} B^l) and convert
 * it to the prognostic components at every location with the metric there (Sec. 6 starts from
 * a uniform contravariant B_z). */
grpic_status grpic_set_uniform_field(grpic_ctx* ctx, const double E_contra[3], const double B_contra[3]);

/* Set J (3 planes); used to drive the E step on its own. */
grpic_status grpic_set_j(grpic_ctx* ctx, const double* J3, int mem);

/* Load (replace) the particles of one species (0..3): charge-to-mass ratio q/m of the push
 * (Eq. 15), macro-particle charge q_macro of the deposit (Sec. 4), n particles with planar
 * positions x4 and velocities u4 (see flags), and ids.  Positions must lie in [1, n_axis-2];
 * completed four-velocities are the future-directed root of g_mn u^m u^n = -c^2.
 * Returns GRPIC_ERR_INVALID for out-of-domain positions or an impossible completion,
 * GRPIC_ERR_CAPACITY if n exceeds max_particles. */
grpic_status grpic_load_particles(grpic_ctx* ctx, int species, double q_over_m, double q_macro, int64_t n,
                                  const double* x4, const double* u4, const uint32_t* ids, int flags);

/* Advance nsteps timesteps (Sec. 2.2 cycle: B half, push + deposit, B half, E; removal and
 * sort), then synchronise and report the device status. */
grpic_status grpic_step(grpic_ctx* ctx, int nsteps);

/* As grpic_step, without the final synchronisation; errors surface at the next grpic_sync. */
grpic_status grpic_step_async(grpic_ctx* ctx, int nsteps);

/* Run one stage of the timestep (GRPIC_STAGE_*), then synchronise.  Driving the stages by hand
 * leaves the removal to the caller: particles flagged by a GRPIC_STAGE_PUSH_DEPOSIT (r <= r_+ or
 * outside the grid) stay listed, at the position the push gave them, until GRPIC_STAGE_SORT. */
grpic_status grpic_stage(grpic_ctx* ctx, int stage);

/* Wait for the context's stream and report the device status. */
grpic_status grpic_sync(grpic_ctx* ctx);

/* Copy out the prognostic field and J (any pointer may be NULL).  The field tensor of Eq. 8
 * (Sec. 3) on the staggered lattice of Sec. 3, Fig. 2: d = contravariant (F^{x4}, F^{y4}, F^{z4})
 * on edges, b = covariant (F_{yz}, F_{zx}, F_{xy}) on faces, J = contravariant current of Sec. 4
 * at the d points; each (3, nz, ny, nx) float64, x fastest.  mem: GRPIC_MEM_HOST or
 * GRPIC_MEM_DEVICE for the destination.  FP32-mixed contexts widen their FP32 fields. */
grpic_status grpic_get_fields(grpic_ctx* ctx, double* d3, double* b3, double* J3, int mem);

/* The field in contravariant components (Eq. 8: F^{4j} = E^j, F^{jk} = eps^{jkl} B^l): d3 receives the
 * prognostic contravariant F^{i4} at the edges (as grpic_get_fields), h3 the contravariant (F^{yz},
 * F^{zx}, F^{xy}) at the b faces, converted from (b, d) as the E step converts them (the other
 * components brought to the face as the mean of their nearest points, the metric at the face; Sec. 3,
 * Eqs. 8 and 11); h3 is zero on the outer index layer.  Either pointer may be NULL; FP64, 3 planes each,
 * caller-owned, host or device memory by mem. */
grpic_status grpic_get_fields_contra(grpic_ctx* ctx, double* d3, double* h3, int mem);

/* A range of z-planes of one field, for a driver that splits one run into z-slabs across contexts
 * and exchanges the planes next to a neighbour's (not in the paper).  which: GRPIC_FIELD_D (the
 * contravariant F^{i4} of Eq. 12's update), GRPIC_FIELD_B (the covariant F_{yz}, F_{zx}, F_{xy} of
 * Eq. 10's), GRPIC_FIELD_J (the current density of Sec. 4); planes z0 .. z0 + nplanes - 1 of each of
 * the three components, FP64, component-major: buf[(q * nplanes + z - z0) * ny * nx + y * nx + x].
 * The current buffers, as grpic_get_fields / grpic_set_fields see them.  grpic_set_planes writes the
 * planes (FP32_MIXED rounds d and b) or, with add = 1, adds into them (J only).  buf is host or device
 * memory by mem; the caller owns it.  GRPIC_ERR_INVALID for a range outside the grid, an unknown
 * field or add on d or b. */
enum { GRPIC_FIELD_D = 0, GRPIC_FIELD_B = 1, GRPIC_FIELD_J = 2 };
grpic_status grpic_get_planes(grpic_ctx* ctx, int which, int z0, int nplanes, double* buf, int mem);
grpic_status grpic_set_planes(grpic_ctx* ctx, int which, int z0, int nplanes, const double* buf, int mem, int add);

/* Number of live particles of a species. */
grpic_status grpic_num_particles(grpic_ctx* ctx, int species, int64_t* n);

/* Particle state of Sec. 3.3 (positions x^a and four-velocities u^a advanced by Eqs. 13-16).
 * Copy out the live particles of a species in the library's (cell-sorted) order, with ids
 * (after grpic_step; after hand-driven stages, the particles listed since the last sort stage).
 * *n_inout: capacity of the caller's arrays on entry, particles written on return.
 * x^4 is returned as the particle's own clock coordinate. */
grpic_status grpic_get_particles(grpic_ctx* ctx, int species, int64_t* n_inout, double* x4, double* u4,
                                 uint32_t* ids, int mem);

grpic_status grpic_get_stats(grpic_ctx* ctx, grpic_stats* out);

/* Invariants of the particles' motion, evaluated in FP64 from the stored state of every live
 * particle: the normalisation g_mn u^m u^n = -c^2 of Eq. 7 (kept by the exact dynamics in any
 * field), and for a tracked subsample (ids divisible by 64) the change of the Killing energy
 * E = -u_4 and of the axial momentum L = u_phi = x u_y - y u_x (covariant components, position from
 * the centre; Eq. 3), both conserved along field-free orbits, since the last call with
 * set_baseline = 1.  Particles removed since the baseline are not compared.  The baseline buffers
 * are allocated by the context (sized by the largest id) and freed with it. */
typedef struct {
  int64_t n;           /* live particles evaluated */
  double norm_max;     /* max |g_mn u^m u^n + c^2| / c^2 */
  double norm_mean;
  int64_t tracked;     /* subsample particles present at the baseline and now */
  double energy_mean;  /* mean |E - E_0| / c over the tracked particles */
  double energy_max;
  double angmom_mean;  /* mean |L - L_0| / c (cells) */
  double angmom_max;
} grpic_invariants;
grpic_status grpic_get_invariants(grpic_ctx* ctx, int set_baseline, grpic_invariants* out);

/* Message for the last error on this context ("" if none); valid until the next call. */
const char* grpic_last_error(const grpic_ctx* ctx);

/* Name of a status code. */
const char* grpic_status_string(grpic_status s);

/* Tracing (not in the paper).  With profiling on, each stage is bracketed by CUDA events on
 * the context stream; grpic_get_profile returns, per GRPIC_STAGE_*, the accumulated device
 * milliseconds and the number of times the stage ran since the last reset (reset = 1 clears
 * after reading), plus the number of kernels the library has launched in total. */
grpic_status grpic_set_profiling(grpic_ctx* ctx, int on);
grpic_status grpic_get_profile(grpic_ctx* ctx, double times_ms[6], int64_t counts[6], int64_t* kernel_launches,
                               int reset);

/* Charge density at the nodes (Sec. 3.3 CIC weights, which det g = -1 makes trilinear) of the
 * particles as they stand: rho = sum q_macro W(x), or with with_gamma = 1 the time component of
 * J = rho gamma v (Sec. 4) over c, sum q_macro (u^4/c) W(x).  rho: ncell doubles in the field
 * layout (z-major, x fastest), host or device memory (mem).  Synchronises. */
grpic_status grpic_charge_density(grpic_ctx* ctx, int with_gamma, double* rho, int mem);

/* Gauss-law residual at the nodes, div E - 4 pi rho, with E^a = -d^a (= -F^{a4}) and backward
 * differences of the edge-centred d, rho from grpic_charge_density (no gamma).  With the
 * gamma-free deposit (GRPIC_NO_GAMMA_IN_J) in flat space it changes over a step by exactly
 * -4 pi times the deposit's 3-D continuity defect (zero for moves within a plane), a live check
 * of the current.  res (may be NULL): ncell doubles, host or device (mem); max_abs (may be
 * NULL): max |residual| over the nodes [2, n-3]^3.  Synchronises. */
grpic_status grpic_gauss_residual(grpic_ctx* ctx, double* res, int mem, double* max_abs);

/* Launch-shape choices of a context (not in the paper; what the autotuner chooses).
 * FP32_MIXED contexts tell "near" particles, R(x_n) < r_fp64 + |a| + 4 cells (some RK4 stage
 * or quadrature node of theirs may fall inside r < r_fp64, where the FP64 policy applies), from
 * "far" ones, which take an FP32-only code path.  Two ways to run that:
 *   split = 0: one launch per species; each warp takes the far-field code unless one of its
 *              particles is near, then the FP32-mixed code (near and far warps share the SMs)
 *   split = 1: a classification lists the near particles, a near-hole kernel pushes them (on a
 *              second, higher-priority stream if overlap = 1, else afterwards) and an FP32-only
 *              kernel pushes the rest
 *   far_min_blocks:     4, 5 or 6 resident 128-thread blocks per SM for the far-field (split = 1)
 *                       or per-warp (split = 0: 4 or 5) kernel at Q = 2 (register budget 128,
 *                       96, 80 per thread); other Q use fixed choices
 *   near_blocks_per_sm: persistent blocks per SM of the near-hole kernel (>= 1)
 *   sort_interval:      counting sort every k timesteps (>= 1)
 *   overlap:            split = 1 only, as above
 *   j_tile:             split = 0, Q = 2: 1 accumulates J per block in a shared-memory FP32 tile over
 *                       the nodes the block's particles can reach, added to the FP64 J once per node
 *   spread:             split = 0: G = 1, 2, 4, ... 64 maps blocks to particle chunks by a permutation of
 *                       groups of G consecutive chunks, spreading the near-hole (FP64-heavy) chunks over
 *                       the launch while each group keeps neighbouring cells together (larger G: more
 *                       L2 locality, less even FP64 load); 0 keeps them in order
 *   area_table:         split = 0, Q = 2, j_tile = 0 (with j_tile = 1 refused), FP32_MIXED (FP64 contexts
 *                       keep it and ignore it, like the other push shapes): 1 takes the face AREAs of Eq. 18
 *                       for far-field warps from per-cell polynomial fits of the integrand instead of
 *                       the Q x Q Gauss nodes, and raises the far-field radius to
 *                       max(r_fp64 + |a| + 4, 4 + (m / 4.5e-7)^(1/6)) cells, where the fits' weights
 *                       agree with the Q = 2 quadrature to a few 1e-9.  The fits (total degree 4 in the
 *                       cell fractions, 35 coefficients per cell and face orientation, the constant and
 *                       linear ones in FP32, the others in FP16: 256 bytes per cell) are allocated and
 *                       computed on the context's stream by the first
 *                       grpic_set_tuning that sets it (GRPIC_ERR_OOM if they do not fit) and kept
 *                       until grpic_destroy
 * grpic_set_tuning validates all fields (GRPIC_ERR_INVALID) and applies them from the next step. */
typedef struct {
  int far_min_blocks;
  int near_blocks_per_sm;
  int sort_interval;
  int overlap;
  int split;
  int j_tile;
  int spread;
  int area_table;
} grpic_tuning;
grpic_status grpic_set_tuning(grpic_ctx* ctx, const grpic_tuning* t);
grpic_status grpic_get_tuning(const grpic_ctx* ctx, grpic_tuning* t);

/* Measure the sustained fused-multiply-add rate of this GPU's CUDA cores (not the tensor
 * cores) with independent FMA chains in every lane: precision GRPIC_FP32_MIXED measures FP32,
 * GRPIC_FP64 measures FP64.  *flops_per_s counts an FMA as two operations.  Used as the
 * roofline denominator of the ALU-bound push. */
grpic_status grpic_probe_fma_peak(int precision, double* flops_per_s);

/* Self-check of the FP64 reciprocal, quotient and square root that the FP32-mixed policy uses
 * for its FP64 evaluations near the hole (one step of Newton's iteration for 1/x, of Heron's
 * for sqrt x, from the FP32 approximations; their results are rounded to FP32 afterwards).
 * Compares them on the current device with the IEEE operations over n log-uniform arguments in
 * [1e-8, 1e8] and returns the largest relative deviations: max_rel[0] 1/x, [1] y/x, [2] sqrt x. */
grpic_status grpic_check_newton64(int64_t n, double max_rel[3]);

/* Self-check of the integer-only FP32 -> FP64 widening and FP64 -> FP32 narrowing (round to
 * nearest even) that the FP32-mixed push uses instead of the hardware conversions (which run on
 * this GPU's FP64 pipe): over n pseudo-random bit patterns it counts, on the current device,
 * results that differ bit for bit from the hardware conversions -- mismatches[0] widening
 * (normal, infinite and NaN floats), mismatches[1] narrowing (doubles around and inside the
 * binary32 normal range, a quarter of them exact ties). */
grpic_status grpic_check_conversions(int64_t n, int64_t mismatches[2]);

/* Sort a particle set by cell without allocating any device memory.  The paper has no
 * counterpart: this is the library's counting sort offered to callers that cannot allocate at
 * the point of the call -- code running under a fixed, pre-reserved device-memory budget,
 * code called from inside an allocator or memory-pool callback (allocating would re-enter the
 * allocator), or loops that must never block in cudaMalloc/cudaFree.
 * x4, u4, ids: n particles on the current device, planar as elsewhere in this header (plane q
 * of x4 starts at x4 + q*n).  Outputs (caller-owned device memory of the same sizes, same plane
 * stride n): the particles whose position lies in [0, n_axis - 1) on every axis, ordered by
 * cell index (k*ny + j)*nx + i of floor(x), order within a cell unspecified; *n_out (a device
 * int64) receives how many were kept.  All work is ordered on `stream` (a cudaStream_t, NULL =
 * default stream); the call does not synchronise.
 * Scratch: one file-scope device array sized for grids of at most 262,144 cells (64^3), about
 * 2.1 MB, held by every GPU that loads this library until the process exits.  Larger grids
 * (nx*ny*nz > 262144) or n >= 2^31 return GRPIC_ERR_CAPACITY without touching the GPU.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Every call shares
 * the array and it keeps the last call's contents (each call clears the counts it uses), so
 * calls whose GPU work overlaps -- on different streams or from different host threads -- race.
 * The call makes no cudaMalloc/cudaFree or other allocating call. */
grpic_status grpic_sort_particles_static(int nx, int ny, int nz, int64_t n, const double* x4, const double* u4,
                                         const uint32_t* ids, double* x4_out, double* u4_out, uint32_t* ids_out,
                                         int64_t* n_out, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched engine: many independent contexts advanced together.  Each stage of the timestep
 * is one persistent launch over all (instance, work item) pairs read from a device table;
 * the per-step stage sequence is captured once in a CUDA graph and replayed.
 * Not in the paper: it runs the paper's cycle for several simulations at once.
 * ------------------------------------------------------------------------------------- */
typedef struct grpic_batch grpic_batch;

/* Group n contexts with the same precision, quadrature order and field-update form.  The
 * batch builds one device descriptor per instance and tables of (instance, work block) items
 * for every stage; each batched stage is one launch over such a table (persistent grid-stride
 * for the field and sort stages, one block per item for the push), and one step's stage sequence
 * is captured once in a CUDA graph on a stream the batch owns (`stream` is unused).  The
 * contexts stay owned by the caller and must outlive every grpic_batch_step and
 * grpic_batch_info of the batch; grpic_batch_destroy touches none of them (the batch keeps its own
 * copy of the first context's allocator).  The batch is built for the particle counts loaded at
 * creation (re-create it after loading more).  Every batched step sorts.  Returns
 * GRPIC_ERR_INVALID for mismatched contexts. */
grpic_status grpic_batch_create(grpic_ctx* const* ctxs, int n, void* stream, grpic_batch** out);

/* Advance every instance nsteps timesteps (graph replays), ordered after each context's pending
 * work; then synchronise and check every context's status (first error returned). */
grpic_status grpic_batch_step(grpic_batch* b, int nsteps);

/* Kernels launched per batched step, and the total number of work blocks in the stage tables. */
grpic_status grpic_batch_info(grpic_batch* b, int64_t* kernels_per_step, int64_t* work_blocks);

/* Persistent blocks per SM of the batch's launches (1..32, default 8; what the autotuner
 * chooses).  Takes effect at the next grpic_batch_step, which captures the graph again. */
grpic_status grpic_batch_set_blocks_per_sm(grpic_batch* b, int blocks_per_sm);

/* Status of one instance after the last grpic_batch_step (which returns the first instance error
 * but reads every instance's device status): GRPIC_OK, or the error that instance reported. */
grpic_status grpic_batch_ctx_status(const grpic_ctx* ctx);

grpic_status grpic_batch_destroy(grpic_batch* b);

/* ---------------------------------------------------------------------------------------
 * Serving: a request loop over whole simulation runs (not in the paper).  Requests are queued
 * by grpic_submit and admitted in arrival order when a slot is free and the run's device-memory
 * estimate fits the budget; each admitted run gets its own context whose plasma is generated on
 * the device; every grpic_server_tick advances all running runs by one timestep together (the
 * batched engine, rebuilt when the set of running runs changes) and retires the finished ones.
 * All runs of a server share precision, quadrature order and flags (those of the first request).
 * ------------------------------------------------------------------------------------- */
typedef struct grpic_server grpic_server;

typedef struct {
  grpic_config cfg;        /* grid, m, a, c, dt, precision, ... (the allocator fields are ignored) */
  double E_contra[3];      /* initial uniform field (Eq. 8) */
  double B_contra[3];
  int nspecies;            /* 1..4 species, co-located at start */
  double q_over_m[4];
  double q_macro[4];
  int ppc;                 /* particles per cell per species in the cells [1, n-3]^3 */
  double u_th;             /* thermal spread: covariant u_i from Maxwell-Juettner, theta = (u_th/c)^2 */
  double r_min;            /* no particles closer than r_min (Euclidean, cells) to the centre */
  uint64_t seed;           /* the plasma is a function of (seed, species, cell, slot) only */
  int nsteps;              /* timesteps to run */
} grpic_request;

enum { GRPIC_RUN_QUEUED = 0, GRPIC_RUN_RUNNING = 1, GRPIC_RUN_DONE = 2 };

/* hbm_budget: bytes of device memory the running runs may use together (their estimates);
 * max_slots: running runs at most; alloc/free/user: device allocator (NULL -> cudaMalloc). */
grpic_status grpic_server_create(size_t hbm_budget, int max_slots, grpic_alloc_fn alloc, grpic_free_fn free_fn,
                                 void* alloc_user, grpic_server** out);

/* Queue a run; *ticket identifies it.  GRPIC_ERR_CAPACITY if it could never fit the budget,
 * GRPIC_ERR_INVALID for a bad request or one whose precision/quadrature/flags differ.
 * GRPIC_ERR_UNSTABLE for a run longer than 40 light-crossing units (nsteps c dt > 40 cells) on a
 * grid whose faces lie where the metric is far from flat, f = 2m / R_face > 0.2 with R_face =
 * (min(nx, ny, nz) - 1) / 2: there the field update with its frozen outer layers (reading of the
 * paper's silent boundaries) grows a mode at the box edges, whatever the timestep, which after
 * ~100 steps accelerates the plasma past the one-cell step limit.  Short runs on such grids, runs
 * whose configuration has an outer absorbing layer (absorb_outer > 0) and every run on larger
 * grids are admitted. */
grpic_status grpic_submit(grpic_server* s, const grpic_request* req, uint64_t* ticket);

/* Admit what fits, advance every running run one timestep, retire finished runs.  A run whose
 * own step fails (non-finite state, a move of a cell or more) is retired with that status
 * (grpic_poll returns it); the others go on.  The tick itself fails only on a CUDA error.
 * *running / *queued (may be NULL) receive the counts after the tick. */
grpic_status grpic_server_tick(grpic_server* s, int* running, int* queued);

/* State of a run (GRPIC_RUN_*); once done, *ctx (may be NULL) borrows its context (fields,
 * particles, stats) until grpic_server_release. */
grpic_status grpic_poll(grpic_server* s, uint64_t ticket, int* state, grpic_ctx** ctx);
/* A run's context carries the invariant baseline of its initial plasma (set at admission), so
 * grpic_get_invariants(ctx, 0, ...) on a finished run gives the change over the whole run. */

/* Free a finished run's context and forget the ticket. */
grpic_status grpic_server_release(grpic_server* s, uint64_t ticket);

/* Device-memory estimate of a request's run (what admission charges against the budget). */
grpic_status grpic_request_bytes(const grpic_request* req, size_t* bytes);

grpic_status grpic_server_destroy(grpic_server* s);

#ifdef __cplusplus
}
#endif

#endif /* GRPIC_H_ */
