/*
 * sph.h -- C-ABI of libsph, the GB300-native SPH neighbour-interaction path.
 *
 * The operations follow Theuns, Chalk, Schaller & Gonnet 2015, "Swift:
 * task-based hydrodynamics and gravity for cosmological simulations":
 *   - cubic cells no smaller than the smoothing length, so that every neighbour
 *     of a particle lies in its own cell or an adjacent one (Sec. 3.1);
 *   - the density sum, Eq. 1, with h_i set so that a given weighted number of
 *     neighbours contributes (Sec. 2, after Eq. 2);
 *   - the pressure-gradient sum, Eq. 2, in the Gadget-2 form the paper adopts
 *     (Sec. 2), with signal-velocity artificial viscosity;
 *   - marching particles forward in time (Sec. 2).
 *
 * Conventions
 *   - Every pointer inside sph_particles is a DEVICE pointer owned by the caller
 *     (except for sph_step_host, which takes HOST pointers).  The library never
 *     frees caller memory.  Arrays are structure-of-arrays, length n, contiguous.
 *   - The library owns its scratch (cell arrays, sort buffers, packed FP32
 *     copies); it allocates it in sph_init / on first use and frees it in
 *     sph_destroy.
 *   - Every call enqueues its work on the stream given to sph_init and returns
 *     after the last launch, EXCEPT where a call documents a host read (the
 *     cell-grid size in sph_build_cells, the convergence count in sph_density,
 *     the time step in sph_step).
 *   - Calls return an sph_status.  No exception, abort or exit crosses the ABI.
 *     sph_last_error() gives a one-line message for the last failure.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_ERR_INVALID_ARG = 1,    /* null pointer, n < 0, bad parameter value      */
    SPH_ERR_CUDA = 2,           /* a CUDA runtime call failed (message kept)     */
    SPH_ERR_NOT_CONVERGED = 3,  /* h iteration hit max_h_iter; results valid for */
                                /* converged particles, last iterate for others  */
    SPH_ERR_H_EXCEEDS_CELL = 4, /* some h > box/3: no periodic cell grid with at */
                                /* least 3 cells per side can hold the support   */
    SPH_ERR_TIMEOUT = 5,        /* a bounded device-side wait ran out            */
    SPH_ERR_NAN = 6,            /* a non-finite input or result was detected     */
    SPH_ERR_STATE = 7,          /* call order violated (e.g. force before        */
                                /* density on the current positions)             */
    SPH_ERR_CAPACITY = 8,       /* a size limit was exceeded (adaptive cells:    */
                                /* more than 2^32 - 2 neighbour-list entries)    */
    SPH_ERR_PRECISION = 9       /* uniform grid: some converged h is below cell  */
                                /* side / SPH_FRAME_RATIO, where FP32 positions  */
                                /* relative to the cell centre cannot hold the   */
                                /* 1e-5 density tolerance (results are written;  */
                                /* use SPH_FLAG_ADAPTIVE for such h ranges)      */
} sph_status;

/* Largest cell side / h the uniform grid accepts (SPH_ERR_PRECISION beyond).  The
 * pair arithmetic takes positions relative to the cell centre in FP32: each
 * separation component is off by at most ~3.4 x 2^-24 L (the two positions, the
 * cell side and the shifted sum), which bounds the density error by ~2e-6 L/h when
 * every rounding points the same way; the roundings of the ~50 neighbours of a sum
 * are independent and partly cancel, and the largest error measured over clustered
 * fields is ~2e-8 L/h (2e-5 at L/h = 960).  At the limit that is ~1.3e-6. */
#define SPH_FRAME_RATIO 64

typedef struct sph_ctx sph_ctx; /* opaque, library-owned */

/* Flags for sph_params.flags */
#define SPH_FLAG_TIMING 1u /* record CUDA events around the pair kernels */
#define SPH_FLAG_NGB_HASH 2u /* density pass also writes a neighbour-set hash */
#define SPH_FLAG_AUTOTUNE 4u /* before the first density pass, time for each candidate
                                schedule (tile width 16/32 x cell factor 1.05/1.25/1.5;
                                with SPH_FLAG_ADAPTIVE: tile width x leaf size
                                64/128/256) the cell build, one density pass and one
                                force pass on the current particles and keep the
                                fastest; overrides tile_width and cell_factor
                                (leaf_max).  On the uniform grid it then times, at
                                that schedule, the staging with and without
                                SPH_FLAG_AXIS_SWEEP (build + density + force) and the
                                force pass in gather and symmetric form, and keeps
                                the faster of each (sph_stats.axis_sweep,
                                force_symmetric).  That first sph_density call also
                                writes the force outputs (ax..vsig) of the probes. */
#define SPH_FLAG_ADAPTIVE 8u /* adaptive cells (Sec. 3.1): the uniform grid becomes the
                                top level of an octree refined while a node holds more
                                than leaf_max particles; leaves are the work items,
                                each with a list of the leaves within reach.  Top
                                cells may number 1 or 2 per side (h < box/2).
                                For h spanning decades (clustered matter).  Builds read
                                tree sizes on the host, so sph_steps runs its steps
                                one by one instead of replaying a CUDA graph. */
#define SPH_FLAG_TREE_H_GUESS 16u /* with SPH_FLAG_ADAPTIVE: the first cell build
                                replaces every input h by an estimate from the number
                                density n of the smallest tree node around it that
                                holds at least 2 N_ngb particles, h = (3 N_ngb /
                                (4 pi n))^(1/3), so that the density iteration starts
                                near its root even where the input guess is off by
                                decades (it converges to the same h) */
#define SPH_FLAG_HPREDICT 32u /* sph_step / sph_steps start every step's density
                                iteration at the learned h guess (weights from
                                sph_hpredict_init / _load / _train) instead of at
                                the previous h; same root, same h_tol */
#define SPH_FLAG_AXIS_SWEEP 64u /* uniform grid: after each build, sort every cell's
                                particles along the 13 half-stencil directions (Sec. 3.1,
                                "sorting"); the pair passes then read a neighbour
                                cell in the order of the direction joining the two
                                cells and skip the particles whose projected distance
                                already exceeds the cutoff (exact: projected distance
                                <= distance).  Default off: the tile bounding-box test
                                alone prunes the same pairs */
#define SPH_FLAG_SYMMETRIC 128u /* uniform grid: the force pass evaluates each unordered pair
                                once (the paper's pair tasks update both cells, Sec. 3.1): one
                                warp per cell sums its own cell in gather form and the 13 cells
                                of a half stencil symmetrically, the far side's terms reduced
                                per source in a fixed order into per-direction slots that a
                                last pass adds up -- deterministic, no atomics on the sums.
                                Where some h needs the radius-2 stencil, and in individual
                                time-steps, the gather form runs.  SPH_FLAG_AUTOTUNE times both
                                forms and keeps the faster (sph_stats.force_symmetric) */
#define SPH_FLAG_BIN_LIMITER 256u /* sph_step_bins: time-step limiter with wake-up (Saitoh &
                                Makino 2009; the paper is silent on time-stepping): no pair
                                r_ij < max(h_i, h_j) with a particle whose step ends now is
                                left more than SPH_BIN_LIMIT_LEVELS bins apart, and a
                                sleeping particle whose raised bin's step ends earlier than
                                its own is woken (its step cut, its opening half kick
                                corrected) */
#define SPH_BIN_LIMIT_LEVELS 2  /* bins a neighbour may be coarser: steps within a factor 4 */

typedef struct {
    int64_t n;           /* particles; 0 <= n < 2^31                                  */
    double box_size;     /* periodic box side L (> 0)                                */
    float gamma;         /* adiabatic index of the ideal-gas EOS, P = (gamma-1) rho u */
    float n_ngb;         /* target weighted neighbour number N_ngb (Sec. 2)           */
    float h_tol;         /* converged when |N_w/N_ngb - 1| <= h_tol                   */
    float alpha_visc;    /* artificial-viscosity strength alpha                      */
    float cfl;           /* dt = cfl * min_i h_i / vsig_i                            */
    float cell_factor;   /* cell side >= cell_factor * max h  (>= 1)                  */
    int32_t max_h_iter;  /* cap on density passes after the last re-binning          */
    int32_t use_balsara; /* 1: viscosity scaled by the Balsara switch                */
    int32_t kernel;      /* 0: cubic spline (the only kernel)                        */
    uint32_t flags;      /* SPH_FLAG_*                                               */
    int32_t tile_width;  /* targets per warp work item: 16 (two cells per warp) or   */
                         /* 32 (one cell per warp); 0 = default (16)                 */
    int32_t n_boxes;     /* independent periodic boxes batched in one set (0 or 1:   */
                         /* a single box); every box has side box_size               */
    const int64_t *box_offsets; /* HOST, n_boxes + 1 entries, 0 = first <= ... <= */
                         /* last = n: box b owns particles [off[b], off[b+1]); each  */
                         /* box gets its own cell grid; NULL when n_boxes <= 1;      */
                         /* copied by sph_init                                       */
    int32_t leaf_max;    /* SPH_FLAG_ADAPTIVE: refine nodes holding more particles   */
                         /* than this (1..4096; 0 = default 64)                     */
    int64_t list_reserve; /* SPH_FLAG_ADAPTIVE, sph_steps: neighbour-list entries   */
                         /* reserved for the captured builds (>= 0; 0 = twice the  */
                         /* last host build's, at least 2^20); lists that outgrow  */
                         /* it return SPH_ERR_CAPACITY                              */
} sph_params;

/*
 * Particle arrays (caller-owned, device).  Inputs: x..h.  Outputs of the density
 * pass: h (converged), rho, P, c, f, divv, curl, n_ngb.  Outputs of the force pass:
 * ax, ay, az, dudt, vsig.  Units: box units for lengths, caller units otherwise.
 *   x, y, z    absolute positions (FP64), wrapped into [0, L) by sph_build_cells
 *   vx, vy, vz velocities (FP64)
 *   m          mass; u specific internal energy; h smoothing length = kernel
 *              support radius (W = 0 beyond h); on input h is the initial guess
 *   rho        density, Eq. 1 (self term included)
 *   P, c       pressure and sound speed from the ideal-gas EOS
 *   f          grad-h factor [1 + h/(3 rho) d rho/dh]^-1
 *   divv, curl velocity divergence and |curl| (SPH estimates at h_i)
 *   n_ngb      number of j != i with r_ij < h_i
 *   ax, ay, az hydrodynamic acceleration (pressure + viscosity)
 *   dudt       rate of change of u
 *   vsig       max signal velocity over the neighbours of i
 */
typedef struct {
    double *x, *y, *z;
    double *vx, *vy, *vz;
    float *m, *u, *h;
    float *rho, *P, *c, *f, *divv, *curl;
    int32_t *n_ngb;
    float *ax, *ay, *az, *dudt, *vsig;
} sph_particles;

/* Global quantities after a step (FP64 reductions, deterministic order). */
typedef struct {
    double momentum[3]; /* sum m v                                   */
    double e_kin;       /* sum m v^2 / 2                             */
    double e_th;        /* sum m u                                   */
    double dt_next;     /* cfl * min h/vsig from the new force pass  */
    int64_t u_floors;   /* kicks that drove u below 0 (clamped to 0) */
} sph_conserved;

/* Individual time-steps (sph_step_bins): deepest bin, and what one call reports. */
#define SPH_MAX_BINS 24
typedef struct {
    int64_t substeps;                    /* step ends visited (drift + update events)   */
    int64_t updates;                     /* particle updates: sum of active counts      */
    int64_t cfl_over;                    /* steps whose CFL step was below the smallest  */
                                         /* bin's, taken at the smallest bin anyway     */
    int64_t bin_count[SPH_MAX_BINS + 1]; /* particles per bin, for their last step      */
    int64_t limited;                     /* SPH_FLAG_BIN_LIMITER: starting steps whose  */
                                         /* bin the limiter raised above the CFL bin    */
    int64_t woken;                       /* SPH_FLAG_BIN_LIMITER: steps cut by wake-ups */
    int64_t limit_sweeps;                /* SPH_FLAG_BIN_LIMITER: limiter passes run    */
} sph_bin_stats;

/* Counters since the last sph_reset_stats (sph_get_stats synchronises the stream). */
typedef struct {
    int32_t nc;                /* cells per side of the grid of box 0                */
    int32_t rebuilds;          /* cell rebuilds forced by h growing past the cell    */
    int64_t n_cells;           /* cells of all boxes                                 */
    double cell_size;          /* cell side of box 0                                 */
    int64_t density_passes;    /* density-kernel launches                            */
    int64_t force_passes;      /* force-kernel launches                              */
    int64_t density_pairs;     /* directed pairs (i, j != i) with r_ij < h_i, summed */
                               /* over every density pass actually run               */
    int64_t density_targets;   /* active targets summed over density passes         */
    int64_t force_pairs;       /* directed pairs with r_ij < max(h_i, h_j)           */
    int64_t density_candidates;/* pair distance tests executed in density passes    */
    int64_t force_candidates;  /* pair distance tests executed in force passes      */
    double t_density_ms;       /* summed device time of density launches (TIMING)   */
    double t_force_ms;         /* summed device time of force launches (TIMING)     */
    double t_build_ms;         /* summed device time of cell builds (TIMING)        */
    int64_t kernel_launches;   /* libsph kernels launched                           */
    int32_t tile_width;        /* schedule in use: targets per tile (16 or 32)       */
    float cell_factor;         /* schedule in use: cell side / max h                 */
    int64_t graph_steps;       /* steps replayed from a captured graph (sph_steps)   */
    int32_t leaf_max;          /* adaptive cells: leaf size in use (0: uniform grid) */
    int64_t hp_samples;        /* learned h: (features, target) pairs collected so far */
    int64_t grav_passes;       /* gravity near-field launches (sph_gravity_p2p)       */
    int64_t grav_pairs;        /* gravity near-field pair interactions (j != i)        */
    double t_grav_ms;          /* summed device time of gravity launches (TIMING)     */
    int32_t force_symmetric;   /* force pass in use: 1 symmetric variant, 0 gather     */
    int32_t axis_sweep;        /* staging in use: 1 per-axis sorted sweep, 0 box test  */
    int64_t density_streamed;  /* density: sources read from the leaf lists, all tiles */
                               /* (adaptive cells; 0 on the uniform grid)             */
    int64_t density_staged;    /* density: of those, staged past the tile's box test   */
    int64_t force_streamed;    /* force: sources read (adaptive cells)                 */
    int64_t force_staged;      /* force: sources staged                                */
} sph_stats;

/* Fill *p with the defaults: gamma 5/3, n_ngb 48, h_tol 1e-4, alpha 0.8, cfl 0.1,
 * cell_factor 1.1, max_h_iter 30, use_balsara 1, kernel 0, flags 0, box 1,
 * tile_width 0 (default schedule). */
int sph_default_params(sph_params *p);

/* Create a context for up to p->n particles on CUDA device `device`, enqueuing on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  *ctx is set
 * to NULL on failure. */
int sph_init(sph_ctx **ctx, const sph_params *p, int device, void *cuda_stream);

/* Change the particle count (reallocates scratch if it grows). */
int sph_set_n(sph_ctx *ctx, int64_t n);

/* Sec. 3.1 cells: wrap positions into [0, L), choose nc = floor(L / (cell_factor *
 * max h)) (>= 3), key each particle by its cell ((iz*nc+iy)*nc+ix with
 * ix = floor(x * nc/L)) and its octant inside the cell (x, y, z at or above the
 * cell centre), stable LSD radix sort by that key, and permute x, y, z, vx, vy,
 * vz, m, u, h, the force outputs ax, ay, az, dudt, vsig and the density outputs
 * divv and n_ngb IN PLACE into cell order (rho, P, c, f and curl are left as they
 * are and are stale until sph_density).
 * The composite permutation since the first build (or since sph_reset_ids) is
 * kept: sph_get_permutation.  Host read: max h.
 * With SPH_FLAG_ADAPTIVE the grid is the top level (nc >= 1) of an octree keyed
 * by (top cell, Morton code inside it); the build also forms the leaves and their
 * neighbour lists (host reads: tree sizes, list total; the build inside sph_steps
 * has none).
 * Errors: SPH_ERR_H_EXCEEDS_CELL if max h > L/3 (adaptive: max h >= L/2);
 * SPH_ERR_CAPACITY if the lists would exceed 2^32 - 2 entries. */
int sph_build_cells(sph_ctx *ctx, sph_particles *parts);

/* Eq. 1 with the smoothing-length iteration: starting from parts->h, Newton steps
 * on N_w(h) = n_ngb (step clamped to [h/2, 2h]; a step leaving the bracket of the
 * root that the evaluations so far give is replaced by the bracket's geometric
 * middle) re-running only unconverged particles, until all satisfy
 * |N_w/N_ngb - 1| <= h_tol -- or their bracket is narrower than 2^-21 h, the
 * resolution of the FP32 sums -- or max_h_iter passes ran since the last
 * re-binning.  Rebuilds the cells (permuting the arrays again, restarting the
 * iteration) if some h outgrows its cell, at most 8 times per call
 * (SPH_ERR_NOT_CONVERGED beyond that).
 * Writes h, rho, P, c, f, divv, curl, n_ngb.  *iters_out (may be NULL) = passes
 * run.  Requires sph_build_cells on the current positions.  Host read: the
 * unconverged count after each pass.  On the uniform grid, SPH_ERR_PRECISION if a
 * converged h is below cell side / SPH_FRAME_RATIO (results are written, and the
 * state counts as having densities, so that sph_force may follow). */
int sph_density(sph_ctx *ctx, sph_particles *parts, int32_t *iters_out);

/* Eq. 2 (Gadget-2 form) with artificial viscosity over pairs r_ij < max(h_i, h_j).
 * Writes ax, ay, az, dudt, vsig.  Requires sph_density on the current state. */
int sph_force(sph_ctx *ctx, sph_particles *parts);

/* One kick-drift-kick step (the time integration of Sec. 2): kick v, u by dt/2
 * with the current a, du/dt; drift x by dt (FP64) and wrap; rebuild cells; density
 * and force on v, u predicted to the end of the step; kick by dt/2 with the new
 * rates; u is floored at 0.  If no force pass ran on the current state, one runs
 * first.  dt <= 0 selects the CFL step from the current vsig.  *dt_used and *out
 * (either may be NULL) receive the step taken and the conserved quantities.
 * SPH_ERR_NOT_CONVERGED (h iteration over its pass budget: those particles keep
 * their last iterate) and SPH_ERR_PRECISION do not stop the step: it completes and
 * returns the first of them at its end (also sph_steps, sph_step_bins and
 * sph_step_host).  Host read: dt and the reductions. */
int sph_step(sph_ctx *ctx, sph_particles *parts, double dt, double *dt_used, sph_conserved *out);

/* n_steps KDK steps (as sph_step) with no host synchronisation between them: the
 * step is captured once into a CUDA graph and replayed (SPH_FLAG_ADAPTIVE included:
 * the captured tree build keeps its sizes on the device, in arrays whose capacity
 * is fixed at entry -- the lists get twice the entries of the last host build, at
 * least 2^20; lists that outgrow that return SPH_ERR_CAPACITY, the step that met
 * it having done no pair work).  Differences from calling
 * sph_step n_steps times: dt lives on the device (dt <= 0: the CFL step of each
 * step's start, else the fixed dt); the cell grid of every box is fixed for the
 * run -- the grid of the previous run is kept while every box's max h is within
 * 1.8 of its cell side (and not far below), else it is planned again at entry
 * (cells stay correct while every h stays within twice the planned cell side;
 * beyond that the call returns SPH_ERR_H_EXCEEDS_CELL; adaptive cells: the top
 * grid is kept while its sides are >= 1.15 max h, else planned at that margin,
 * and stays correct while every h stays within its top cell side and within 1.15
 * of its leaf's largest h at the step's build -- a Newton step is cut back to
 * that limit, and SPH_ERR_H_EXCEEDS_CELL reported if a root lies beyond); each density
 * evaluation runs a fixed number of passes, min(max_h_iter, 6) -- passes after
 * convergence find no work -- and SPH_ERR_NOT_CONVERGED is returned if any
 * particle was still unconverged after them.  *out (may be NULL) receives the
 * conserved quantities after the last step; *dt_last (may be NULL) its dt.
 * n_steps = 0 only prepares (hydro pass if needed, plan, capture).  Synchronises
 * the stream at entry (max h, first dt) and at the end. */
int sph_steps(sph_ctx *ctx, sph_particles *parts, int32_t n_steps, double dt, double *dt_last,
              sph_conserved *out);

/* Individual time-steps: advances by dt_max with each particle on its own step
 * dt_max / 2^b, b in [0, n_bins] (0 <= n_bins <= SPH_MAX_BINS).  The paper is silent
 * on time-stepping; this is the power-of-two scheme of the Gadget-2 line its force
 * law comes from, each particle following the leapfrog of sph_step.  Time runs on
 * a grid of dt_max / 2^n_bins.  A particle starting a step at time s takes the
 * largest dt_max / 2^b not above its CFL step cfl h / vsig (b = n_bins, counted in
 * cfl_over, if even that is above it), made smaller until s is a multiple of it.
 * All particles open a step at 0 (half kick); at each later step end every particle
 * drifts, the cells are rebuilt, and the particles whose step ends there get the
 * density (h iteration) and force against all particles -- every particle's v and
 * u predicted to that time from the middle of its own step, v_half + a (t - t_mid),
 * the others keeping h, rho, P, c, f, Balsara B, a, du/dt and vsig from their last
 * update -- then their closing half kick, a new bin and, before dt_max, their
 * next opening half kick.  With SPH_FLAG_BIN_LIMITER the new bins (all of them at
 * 0) are then raised, in passes over the particles until none changes, to the
 * least fixed point of: a particle whose step ends now takes at least the largest
 * bin of its neighbours (r_ij < max(h_i, h_j), decided in FP64 from the positions)
 * minus SPH_BIN_LIMIT_LEVELS, a sleeping one at least the largest bin of its
 * neighbours whose step ends now minus SPH_BIN_LIMIT_LEVELS; a sleeping particle
 * whose raised bin's step, counted from the grid, ends at T' before its own step
 * end T is woken -- its step now ends at T', its opening half kick corrected by
 * (T' - T) / 2 -- and the others open their steps.  Each particle's step start and
 * end are kept as integers.  On return every particle is synchronised at dt_max with
 * current a, du/dt, vsig (n_bins = 0 is exactly sph_step with dt = dt_max).  Runs
 * a hydro pass first if the current state has none (or SPH_FLAG_AUTOTUNE has not
 * tuned yet).  *out and *stats may be NULL.  Errors as sph_step; on an error the
 * particles are left part-way through the interval.  Host reads at every step end. */
int sph_step_bins(sph_ctx *ctx, sph_particles *parts, double dt_max, int32_t n_bins, sph_conserved *out,
                  sph_bin_stats *stats);

/* Bin of every slot after the last sph_step_bins (device, int8, length n, the
 * current slot order). */
int sph_get_bins(sph_ctx *ctx, int8_t *dev_bins);

/* sph_step on HOST arrays (pinned memory recommended): copies x..h, vx..vz, m, u,
 * ax, ay, az, dudt, vsig to library-owned device buffers, steps, and copies every
 * array of *host_parts back (in the new cell order).  Includes the copies in the
 * call; synchronises the stream before returning. */
int sph_step_host(sph_ctx *ctx, sph_particles *host_parts, double dt, double *dt_used,
                  sph_conserved *out);

/* Composite permutation: dev_perm[k] (device, int64, length n) = index, in the
 * arrays given to the first sph_build_cells, of the particle now in slot k. */
int sph_get_permutation(sph_ctx *ctx, int64_t *dev_perm);

/* Forget the permutation: the next build numbers particles 0..n-1 afresh. */
int sph_reset_ids(sph_ctx *ctx);

/* Cell key of every slot (device, int32, length n) for the current grid (with
 * SPH_FLAG_ADAPTIVE: the top-level cell holding the slot). */
int sph_get_cell_keys(sph_ctx *ctx, int32_t *dev_keys);

/* Neighbour-set hash of the last density pass (needs SPH_FLAG_NGB_HASH): device,
 * uint64, length n: sum over j != i with r_ij < h_i of splitmix64(perm id of j). */
int sph_get_ngb_hash(sph_ctx *ctx, uint64_t *dev_hash);

/* ---------------------------------------------------------------------------
 * Learned initial smoothing lengths (not in the paper).  The h iteration above
 * (Sec. 2) may start from an MLP's guess instead of the previous h: 6 features per
 * particle (dt*divv_prev, log(n_ngb_prev/N_ngb), log(h_cell/h_prev),
 * log(count/N_ngb), log(h_prev/side), dt*vsig_prev/h_prev; "cell" = the
 * particle's cell, with SPH_FLAG_ADAPTIVE its leaf, h_cell the h of a uniform
 * medium of the cell's number density) -> 6-64-64-1 MLP with SiLU -> log(h/h_prev),
 * clamped to [log 1/2, log 1.2].  Weights BF16, activations BF16, accumulation
 * FP32; features and the target are normalised by means and standard deviations
 * stored with the weights.
 *   weights  w_bf16[SPH_HP_NBF16] = W1[64][6], W2[64][64] (row = output unit),
 *            W3[64]  (raw bfloat16 bits)
 *   floats   f32[SPH_HP_NF32] = b1[64], b2[64], b3, feature means[6], feature
 *            standard deviations[6], target mean, target standard deviation
 * All device arrays are caller-owned; features are row-major n x 6. */
#define SPH_HP_NBF16 4544
#define SPH_HP_NF32 143

/* Random (Glorot-uniform) weights from a seed; unit normalisation. */
int sph_hpredict_init(sph_ctx *ctx, uint64_t seed);
/* Weights and floats from HOST arrays (layout above). */
int sph_hpredict_load(sph_ctx *ctx, const uint16_t *w_bf16, const float *f32);
/* Current weights (BF16, as used for inference) and floats to HOST arrays. */
int sph_hpredict_save(sph_ctx *ctx, uint16_t *w_bf16, float *f32);
/* FP32 training state to a HOST array of SPH_HP_NPARAM floats: W1[64][6], b1[64],
 * W2[64][64], b2[64], W3[64], b3 (the BF16 weights are its rounding). */
#define SPH_HP_NPARAM 4673
int sph_hpredict_params(sph_ctx *ctx, float *params);
/* Features of the current state (after sph_build_cells, before sph_density; the
 * density/force outputs from the previous hydro pass are the "prev" inputs) with
 * time step dt, into dev_feats (n x 6); also remembers the current h as h_prev. */
int sph_hpredict_features(sph_ctx *ctx, sph_particles *parts, double dt, float *dev_feats);
/* Targets log(h / h_prev) of the remembered h_prev (after sph_density). */
int sph_hpredict_targets(sph_ctx *ctx, sph_particles *parts, float *dev_target);
/* Predictions log(h0 / h_prev) for n feature rows (BF16 tensor-core inference,
 * clamped to [log 1/2, log 1.2]) into dev_out. */
int sph_hpredict_eval(sph_ctx *ctx, const float *dev_feats, int64_t n, float *dev_out);
/* Train on n (features, target) pairs: `epochs` passes of ceil(n / 16384) Adam
 * steps (batch 16384, mean squared error of the normalised target, beta 0.9 /
 * 0.999).  Sample k of step s is row (s*16384 + k) mod n when seed = 0, else a
 * hash of (seed, s*16384 + k) mod n.  Initialises the weights (from seed, or 1)
 * if none were set; the normalisation comes from these samples unless it was
 * loaded.  *loss_out (host, may be NULL): loss of the last step.  Synchronises. */
int sph_hpredict_train(sph_ctx *ctx, const float *dev_feats, const float *dev_target, int64_t n,
                       int32_t epochs, float lr, uint64_t seed, float *loss_out);
/* Let sph_step append every step's (features, target) pairs to dev_feats (n x 6
 * per step) and dev_target until `capacity` rows are filled (a step that would
 * not fit is skipped); capacity 0 stops collecting.  Count: sph_stats.hp_samples. */
int sph_hpredict_collect(sph_ctx *ctx, float *dev_feats, float *dev_target, int64_t capacity);

/* Stable LSD radix sort of cell keys -- the sort sph_build_cells runs -- for callers
 * that cannot allocate device memory: code whose device memory is owned by another
 * framework's pool or reserved up front (so a cudaMalloc could fail or break its
 * accounting), or that must not allocate in the middle of a time step.  The paper
 * has no counterpart; it is a deployment convenience.
 *   keys_in   device uint32[n], read only, need not be sorted
 *   keys_out  device uint32[n], caller-owned: the input keys (all their bits) in
 *             ascending order of their low key_bits bits, equal ones in input order
 *   perm_out  device uint32[n], caller-owned: perm_out[k] = index in keys_in of
 *             the key now in slot k
 *   key_bits  significant low bits of every key, 1..32; bits above them take no
 *             part in the order
 * The three buffers must not overlap (an in-place sort is not supported):
 * overlapping ranges return SPH_ERR_INVALID_ARG before any GPU work.
 * The scratch is a fixed static device buffer of about 2.2 MB, held on every GPU
 * that loads the library until the process exits; n above SPH_SORT_STATIC_MAX_N
 * returns SPH_ERR_INVALID_ARG before any GPU work.  Nothing is allocated or freed.
 * Every call looks up the buffer's device address on the current device; the first
 * call on a device also loads the library's GPU code there (make it before any
 * stream capture).  Work is enqueued on `cuda_stream` (a cudaStream_t) on the
 * current device and the call returns without synchronising.  All calls share the
 * one buffer: calls whose GPU work overlaps (different streams, or several host
 * threads) race and must be serialised by the caller.  Returns SPH_OK,
 * SPH_ERR_INVALID_ARG or SPH_ERR_CUDA (no context, so no sph_last_error text):
 * SPH_ERR_CUDA also when a CUDA error from earlier work is still pending on entry
 * (it is left pending for its owner, and nothing is launched). */
#define SPH_SORT_STATIC_MAX_N 262144
int sph_sort_keys_static(const uint32_t *keys_in, uint32_t *keys_out, uint32_t *perm_out, int64_t n,
                         int32_t key_bits, void *cuda_stream);

/* Near-field gravity (Sec. 3.2, Eq. 3): the node-node tasks of the paper's tree walk
 * in which all particles of one node interact with all particles of a nearby node,
 * run on the cells of the current uniform grid.  For every particle i,
 *   a_i   = -G sum_j m_j (r_i - r_j) / (|r_i - r_j|^2 + eps^2)^(3/2)
 *   phi_i = -G sum_j m_j / (|r_i - r_j|^2 + eps^2)^(1/2)
 * over every j != i in i's own cell and the 26 cells adjacent to it (periodic, the
 * minimal-image separation; with 3 cells per side that is every particle of the
 * box).  eps is the Plummer softening length; eps = 0 is Eq. 3 as printed, and then
 * a pair at zero separation contributes nothing (below 1e-15 box units in FP32).  The far field (multipoles of
 * non-adjacent cells) is not computed.  Batched boxes: each box on its own grid.
 *   ax, ay, az  device FP32[n], caller-owned: the acceleration of every slot, in
 *               the current cell order (that of sph_build_cells)
 *   phi         device FP32[n] or NULL: the potential
 * FP32 arithmetic on the cell-relative positions of the last build, masses from m
 * at that build; the 27 cell sums of a particle are added with compensation.  A
 * separation component is off by up to ~3.5 x 2^-24 x cell side, so a softened
 * pair's force by at most m_j x that / eps^3, an unsoftened one by ~2 x that / r of
 * itself: close unsoftened pairs carry large relative errors.
 * Requires sph_build_cells on the current positions, uniform grid (SPH_ERR_STATE
 * otherwise, or with SPH_FLAG_ADAPTIVE); SPH_ERR_INVALID_ARG for eps < 0, non-finite
 * G or eps, or null outputs.  Asynchronous. */
int sph_gravity_p2p(sph_ctx *ctx, double G, double eps, float *ax, float *ay, float *az, float *phi);

/* Throughput of the plain FP32 FMA pipes on the current device: the ceiling of the
 * pair kernels, whose sums are not dense contractions (the tensor cores do not
 * apply).  Not in the paper; it measures the denominator of their roofline.  Runs
 * `reps` timed launches (after one untimed) of a kernel in which every thread
 * carries 16 independent FMA recurrences for `iters` rounds, 8 blocks of 256 threads
 * per SM, on `cuda_stream` (a cudaStream_t), and synchronises.  *tflops_out (host)
 * = 2 x FMAs / the fastest launch's CUDA-event time; *ms_out (may be NULL) = that
 * time.  Allocates nothing.  SPH_ERR_INVALID_ARG for iters < 1, reps < 1 or a null
 * tflops_out; SPH_ERR_CUDA if a CUDA call fails. */
int sph_fp32_peak(void *cuda_stream, int32_t iters, int32_t reps, double *tflops_out, float *ms_out);

int sph_get_stats(sph_ctx *ctx, sph_stats *s);
int sph_reset_stats(sph_ctx *ctx);
const char *sph_last_error(const sph_ctx *ctx);
void sph_destroy(sph_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
