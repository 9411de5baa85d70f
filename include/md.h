/*
 * md.h -- C ABI of the GB300 short-range molecular-dynamics library.
 *
 * The library integrates Newton's equations m r'' = F, F = -grad U (Eq. 1 of
 * arXiv:2109.10876, Sec. 2.1) for particles in orthorhombic periodic boxes,
 * with the Lennard-Jones pair potential of Eq. 2 truncated at r < r_cut
 * (Sec. 2.1.1), or its repulsive WCA form (r_cut = 2^(1/6) sigma, Sec. 4),
 * optional FENE bonds and a Langevin thermostat (Sec. 4), using cell binning
 * and Verlet lists with a skin, r_cell >= r_cut + r_skin (Sec. 2.1.2), and
 * velocity Verlet in two half steps (Fig. 1).
 *
 * Every step runs in hand-written sm_103a CUDA kernels; there is no CPU path.
 *
 * Conventions for every entry point:
 *   - Per-particle arrays use the component-major layout a[k * N + i]
 *     (k = 0, 1, 2 for x, y, z; N = total particles over all replicas),
 *     i.e. a (3, N) row-major array; particle i is the i-th particle the
 *     caller passed to md_set_state.
 *   - Array arguments may be device pointers or host pointers (pageable or
 *     pinned); the library copies through them and never keeps or frees them.
 *     The caller owns all memory it passes in.  The library owns everything it
 *     allocates (cells, lists, flags, its copy of the state) and frees it in
 *     md_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.
 *   - Argument errors are returned synchronously.  Errors found on the device
 *     (list overflow, non-finite values, broken bonds, fixed-point overflow)
 *     are latched in an error word and returned by the next synchronising
 *     call (md_get_stats, md_export_pairs, md_get_state, md_sync).
 *   - Units are reduced LJ units (Sec. 4: m = eps = sigma = 1 by default).
 */
#ifndef MD_GB300_H
#define MD_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_handle md_handle;

typedef enum {
    MD_OK = 0,
    MD_ERR_ARG = -1,            /* invalid argument or call order            */
    MD_ERR_CUDA = -2,           /* a CUDA runtime call failed                */
    MD_ERR_LIST_OVERFLOW = -3,  /* a particle had more neighbours than the list holds */
    MD_ERR_NONFINITE = -4,      /* a non-finite position, velocity or force  */
    MD_ERR_BOND_BROKEN = -5,    /* a FENE bond reached r >= R0               */
    MD_ERR_FIXED_OVERFLOW = -6, /* a pair force exceeded the fixed-point range */
    MD_ERR_TIMEOUT = -7,        /* a bounded device wait gave up             */
    MD_ERR_BOX_TOO_SMALL = -8,  /* a box edge is shorter than 2 (r_cut + r_skin) */
    MD_ERR_BOUNDS = -9          /* a device-side bounds check failed (checked build) */
} md_status;

/* md_params.potential.  MD_SOFT is the cosine push-off A (1 + cos(pi r / r_cut))
 * for r < r_cut, A = eps, r_cut = rc_over_sigma * sigma: a bounded repulsion
 * that separates overlapping beads when a polymer melt is prepared (the melt
 * of Sec. 4; the paper does not state its preparation).  MD_FP64 only, and
 * not covered by md_forward / md_backward. */
enum { MD_LJ = 0, MD_WCA = 1, MD_SOFT = 2 };
enum { MD_FP64 = 0, MD_FP32_FIXED = 1 };   /* md_params.precision */

/* Parameters of a set of independent replicas (n_replicas >= 1).  Replica r
 * holds particles [replica_offsets[r], replica_offsets[r+1]) of the arrays
 * passed to md_set_state.  All pointers here are HOST pointers, read during
 * md_create only. */
typedef struct {
    int32_t n_replicas;
    const int64_t *replica_offsets; /* n_replicas + 1, offsets[0] = 0           */
    const double *box;              /* 3 per replica: Lx, Ly, Lz                */
    const double *eps;              /* per replica, Eq. 2 epsilon               */
    const double *sigma;            /* per replica, Eq. 2 sigma                 */
    double rc_over_sigma;           /* cutoff in units of sigma (LJ fluid: 2.5);
                                       ignored for MD_WCA (2^(1/6)); MD_SOFT:
                                       its r_cut / sigma                        */
    double skin;                    /* Verlet skin r_skin (absolute)            */
    double dt;                      /* time step                                */
    double mass;                    /* particle mass                            */
    int32_t potential;              /* MD_LJ (shifted to 0 at r_cut), MD_WCA or
                                       MD_SOFT                                  */
    int32_t precision;              /* MD_FP32_FIXED or MD_FP64                 */
    double langevin_gamma;          /* 0 = NVE                                  */
    double kT;                      /* Langevin temperature                     */
    uint64_t seed;                  /* Langevin noise key (Philox4x32-10)       */
    double fene_K, fene_R0;         /* FENE bond constants                      */
    int64_t n_bonds;                /* FENE bonds                               */
    const int32_t *bonds;           /* 2 * n_bonds particle indices, or NULL    */
    int32_t list_capacity;          /* neighbours per particle, rounded up to a
                                       multiple of 32; 0 = automatic: sized
                                       from the mean density and grown until
                                       the list fits by md_build_neighbors,
                                       which the first md_step,
                                       md_compute_forces or md_get_checkpoint
                                       after md_set_state runs (synchronising
                                       once)                                    */
    int32_t reserved0;
    double angle_K;                 /* bending constant of the angle term       */
    int64_t n_angles;               /* angle triples                            */
    const int32_t *angles;          /* 3 * n_angles particle indices (a, b, c),
                                       b the middle bead, or NULL: the cosine
                                       term K (1 - cos theta) on the angle
                                       between b1 = x_b - x_a and b2 = x_c - x_b
                                       (Sec. 4 names a cosine-type term on
                                       triples without its form)                */
} md_params;

/* Counters and diagnostics (md_get_stats). */
typedef struct {
    int64_t steps;              /* steps integrated since md_set_state        */
    int64_t rebuilds;           /* neighbour-list builds since md_set_state   */
    int64_t list_entries;       /* sum of list lengths at the last build      */
    int32_t max_list_len;       /* longest list at the last build             */
    int32_t list_capacity;      /* current capacity per particle              */
    int32_t max_cell_occupancy; /* at the last build                          */
    int32_t error_word;         /* latched device error bits                  */
    int32_t ncell[3];           /* cell grid of replica 0                     */
    int32_t n_replicas;
    int64_t n_particles;
    int32_t n_tiles;            /* tiles of the last build (runs of cells along x) */
    int32_t max_halo;           /* largest tile halo (particles) at the last build */
    int32_t halo_capacity;      /* shared-memory halo capacity (particles)    */
    int32_t tile_size;          /* particles per tile the tiler aims at        */
    int64_t recoveries;         /* md_step overflows recovered (md_set_recovery) */
    int64_t bad_index;          /* checked build: the index that failed at bad_site */
    int32_t bad_site;           /* checked build: the first failing bounds check, else 0 */
} md_stats;

/* Create a handle for the replicas described by p (Sec. 2.1: cells of edge
 * >= r_cut + r_skin per box).  Synchronous.  Returns MD_ERR_BOX_TOO_SMALL when a
 * box edge is shorter than 2 (r_cut + r_skin), MD_ERR_ARG for inconsistent
 * parameters, MD_ERR_CUDA if device memory cannot be allocated.  *out is set to
 * NULL on failure. */
md_status md_create(const md_params *p, md_handle **out);

/* Free everything the handle owns.  Synchronises the device first.  No
 * passage of the paper: resource lifetime of this library. */
void md_destroy(md_handle *h);

/* Load positions x and velocities v, each (3, N) component-major FP64, into the
 * handle; positions are wrapped into [0, L).  These are the particle state
 * (r_i, v_i) that velocity Verlet advances (Fig. 1; Eq. 1).  Resets the step
 * counter, marks the neighbour list stale and the stored force invalid.  A
 * non-finite value latches MD_ERR_NONFINITE (reported by the next
 * synchronising call).  Asynchronous.  To resume a saved run exactly, use
 * md_set_checkpoint instead. */
md_status md_set_state(md_handle *h, const double *x, const double *v, void *stream);

/* Copy the current positions and velocities out, (3, N) FP64 each, in the
 * caller's particle order: the state (r_i, v_i) of Fig. 1 after the last
 * completed step.  Either pointer may be NULL.  Synchronises `stream` and
 * returns any latched device error. */
md_status md_get_state(md_handle *h, double *x, double *v, void *stream);

/* Save everything the next step depends on, so that a run can be stopped and
 * resumed exactly: positions x and velocities v ((3, N) FP64 each, as
 * md_get_state), the stored total force f ((3, N) FP64: the force of Fig. 1's
 * second half kick, which the next step's first half kick reuses, including
 * the Langevin term of Sec. 4's thermostatted runs), and the step counter
 * *step (host), which keys the Langevin noise.  Caller order; host or device
 * pointers, none NULL.  When the handle holds no stored force (no md_step
 * since the last md_set_state, md_build_neighbors or md_compute_forces) it is
 * evaluated now, as the next md_step would.  Synchronises `stream` and returns
 * any latched device error. */
md_status md_get_checkpoint(md_handle *h, double *x, double *v, double *f, int64_t *step, void *stream);

/* Restore a state saved by md_get_checkpoint: md_set_state(x, v), then the step
 * counter and the stored force, with the cells and the Verlet list built at x.
 * The following md_step continues the saved run: bit for bit in
 * MD_FP32_FIXED (its sums do not depend on when the list was built), to
 * rounding in MD_FP64, with the same Langevin noise in both.  MD_ERR_ARG for a
 * NULL pointer or step < 0.  Synchronises `stream`. */
md_status md_set_checkpoint(md_handle *h, const double *x, const double *v, const double *f, int64_t step,
                            void *stream);

/* Bin particles into cells with a counting sort and rebuild the Verlet list of
 * all pairs with |d| < r_cut + r_skin (Sec. 2.1.2), now, whatever the
 * displacement since the last build.  Asynchronous. */
md_status md_build_neighbors(md_handle *h, void *stream);

/* Evaluate the conservative forces (pair potential of Eq. 2 under r < r_cut,
 * plus FENE bonds and angle triples) at the current positions.  f_out (may be NULL) receives the
 * (3, N) FP64 forces in the caller's order; euw_out (may be NULL) receives
 * (U, K, W) per replica, 3 * n_replicas FP64: potential energy (pair energy
 * shifted to 0 at r_cut, plus FENE and angle terms), kinetic energy 1/2 m
 * sum v^2, and the virial sum over pairs of d_ij . f_ij (the angle term,
 * a function of the angle alone, has none).  Rebuilds the list first if particles
 * moved more than r_skin / 2 since the last build.  Asynchronous. */
md_status md_compute_forces(md_handle *h, double *f_out, double *euw_out, void *stream);

/* Advance nsteps velocity-Verlet steps (Fig. 1: half kick + drift, force,
 * half kick), rebuilding the cells and the Verlet list on the device whenever
 * some particle has moved more than r_skin / 2 since the last build.  If
 * thermo_every > 0, thermo_out receives (U, K, W) per replica after every
 * thermo_every-th step: floor(nsteps / thermo_every) records of 3 * n_replicas
 * FP64 each.  Asynchronous; device errors are latched. */
md_status md_step(md_handle *h, int32_t nsteps, int32_t thermo_every, double *thermo_out, void *stream);

/* Overflow recovery for md_step.  The Verlet list (Sec. 2.1.2) and each
 * tile's staged halo have fixed capacities; a rebuild that md_step runs on
 * the device can outgrow them when the system densifies.  With enable = 1,
 * md_step synchronises its stream at the start and the end of every call and,
 * if a rebuild inside the call overflowed, grows the capacity that overflowed
 * (also a list_capacity given at md_create), rebuilds the list from the state
 * at which that rebuild ran, and runs the rest of the call's steps; the result
 * equals an uninterrupted run with the larger capacity (bit for bit in
 * MD_FP32_FIXED), energy records included.  md_get_stats counts the
 * recoveries.  With enable = 0 (the default) md_step stays asynchronous and an
 * overflow is latched as MD_ERR_LIST_OVERFLOW: the call's remaining kernels
 * return at once and the error is reported by the next synchronising call. */
md_status md_set_recovery(md_handle *h, int32_t enable);

/* Self-test of the bounded device waits.  Every wait of the library's kernels
 * (the completion of a tile's bulk copies) gives up after a bounded number of
 * polls and latches MD_ERR_TIMEOUT instead of hanging the GPU.  This call
 * launches one block that waits, with the same code, on a barrier that
 * nothing completes, polling at most `polls` times (1..65536; each poll may
 * suspend the thread for a short, hardware-defined time), so that the error
 * path can be exercised: the next synchronising call returns MD_ERR_TIMEOUT,
 * and md_set_state (or md_set_checkpoint) clears it.  The paper has no
 * counterpart.  MD_ERR_ARG for polls outside 1..65536.  Asynchronous. */
md_status md_check_wait_timeout(md_handle *h, int32_t polls, void *stream);

/* Build flags of the loaded library: MD_BUILD_CHECKED for the checked build
 * (libmd_gb300_checked.so, compiled with -DMD_CHECKED), else 0.  In the
 * checked build every kernel checks the indices that the data layout keeps
 * in range by construction -- cell ids, bucket and destination slots,
 * particle ids, tile and halo-piece indices, candidate ranges, list entries
 * against the staged halo, the slots behind halo entries, bond and angle
 * partners.  A failed check latches MD_ERR_BOUNDS, with the first failing
 * site and index (md_stats.bad_site / bad_index, and the message of
 * md_last_error), and the access is replaced by a harmless one: nothing
 * traps, the context stays usable, and md_set_state clears the error.  It is
 * the device-side stand-in for a memory checker; the default build compiles
 * every check away.  No passage of the paper: a debugging aid of this
 * library. */
#define MD_BUILD_CHECKED 1
int md_build_flags(void);

/* Sites of the checked build's bounds checks (md_stats.bad_site). */
typedef enum {
    MD_SITE_BIN_CELL = 1,      /* binning: a particle's cell within its replica's cells */
    MD_SITE_SCATTER = 2,       /* counting sort: a bucket slot within its cell's slots  */
    MD_SITE_REORDER = 3,       /* re-sort: the particle id and the destination slot     */
    MD_SITE_TOPOLOGY = 4,      /* bond and angle partner ids                           */
    MD_SITE_TILE_WRITE = 5,    /* tiling: a tile's index within the tile table          */
    MD_SITE_PIECES = 6,        /* tiling: halo pieces within kMaxPieces and the slots   */
    MD_SITE_LIST_RANGE = 7,    /* list build: a candidate range within the halo         */
    MD_SITE_LIST_SELF = 8,     /* list build: the tile's own entries within the halo    */
    MD_SITE_FORCE_HALO = 9,    /* force kernels: a list entry within the staged halo    */
    MD_SITE_FORCE_OWN = 10,    /* force kernels: a particle's own halo entry            */
    MD_SITE_FORCE_SLOT = 11,   /* force kernels: the slot behind a halo entry           */
    MD_SITE_BOND_SLOT = 12,    /* force kernel: a bond or angle partner's slot          */
    MD_SITE_ADJ = 13           /* reverse pass: a list entry, particle id or slot       */
} md_check_site;

/* Self-test of the checked build's bounds checks: makes the checks of `site`
 * (an md_check_site) fail on purpose on their next evaluations, with the
 * index they see (which is in range), so that each site's failure path -- the
 * latch, the report, the harmless replacement access -- runs without a bad
 * access.
 * The next synchronising call that runs that site returns MD_ERR_BOUNDS;
 * md_set_state disarms it.  site 0 disarms it too.  MD_ERR_ARG in the default
 * build or for a site out of range.  Synchronises `stream`. */
md_status md_check_bounds_selftest(md_handle *h, int32_t site, void *stream);

/* Differentiable run (reverse-mode differentiation of the velocity-Verlet map
 * of Fig. 1; the paper itself has no gradients).  Advance nsteps NVE steps from
 * the current state, keeping (x, v) every ckpt_every steps in device memory the
 * handle owns, and write (U, K, W) per replica of the final state to euw_out
 * (3 * n_replicas FP64, host or device, may be NULL).  Pair potentials only:
 * returns MD_ERR_ARG for handles with FENE bonds, angle triples, a thermostat
 * or the push-off potential.
 * Synchronises `stream`. */
md_status md_forward(md_handle *h, int32_t nsteps, int32_t ckpt_every, double *euw_out, void *stream);

/* Reverse pass of the last md_forward (the adjoint of the velocity-Verlet map
 * of Fig. 1) for a loss L of its final state:
 *   dL_dx, dL_dv: the loss's gradients in the final positions and velocities,
 *                 (3, N) FP64 each in the caller's order, host or device, or
 *                 NULL (zero): a loss on the trajectory's end point itself,
 *                 such as a target structure or a displacement;
 *   dL_deuw:      (dL/dU, dL/dK, dL/dW) per replica, 3 * n_replicas FP64,
 *                 host or device, or NULL (zero): a loss on the final energies
 *                 and virial.
 * Writes dL/deps and dL/dsigma per replica (n_replicas FP64 each, host or
 * device): the derivative of the smooth flow, with r_cut = rc_over_sigma *
 * sigma moving with sigma (pairs crossing r_cut contribute jump terms that are
 * not included).  Recomputes each segment from its checkpoint; Hessian-vector
 * products and all adjoint sums in FP64.  Leaves the handle at the final state
 * of the recorded run (step counter and stats reset).  A device error latched
 * during the pass is returned as soon as it is seen (checked once per
 * segment), with the handle at a checkpoint's state: md_set_state before
 * further use.  Synchronises `stream`. */
md_status md_backward(md_handle *h, const double *dL_dx, const double *dL_dv, const double *dL_deuw,
                      double *dL_deps, double *dL_dsigma, void *stream);

/* Export the current Verlet pair set as pairs (i, j), i < j, in the caller's
 * particle numbering, in no particular order.  Writes at most `capacity` pairs
 * (2 * capacity int32) to pairs_out and the total count to *n_out (host).
 * Synchronises `stream`. */
md_status md_export_pairs(md_handle *h, int32_t *pairs_out, int64_t capacity, int64_t *n_out, void *stream);

/* Pick the tile size (particles per tile of the force and list kernels) by
 * timing trial_steps steps at each candidate: from the largest (128) down to
 * 64 in steps of 16, all of them, then halving while the steps get faster, down
 * to 8; the fastest is kept.  This is the GPU counterpart of the paper's tuning
 * of the HPX subnode count (Sec. 3.3, Sec. 4.2), which doubles the number of
 * subnodes until the elapsed time of a few steps stops falling.  Positions,
 * velocities, the stored force and the step counter are saved and restored,
 * so the trajectory goes on from where it was (bit for bit in
 * MD_FP32_FIXED, whose sums do not depend on the tiling); the rebuild
 * statistics restart.  Takes 9N doubles of extra device memory for the
 * duration of the call.  Writes the chosen size to *tile_max_out (host
 * pointer, may be NULL).  Synchronous. */
md_status md_autotune(md_handle *h, int32_t trial_steps, int32_t *tile_max_out, void *stream);

/* Set the tile size by hand (1..128 particles; a tile always holds at least
 * one whole cell, so cells fuller than the size make one-cell tiles).  The
 * next step, force or list call re-sorts and rebuilds the list on `stream`.
 * MD_ERR_ARG outside 1..128. */
md_status md_set_tile_size(md_handle *h, int32_t tile_size, void *stream);

/* Choose the Verlet-list form (Sec. 2.1.2): enable = 0 (the default) keeps
 * the full list, in which every pair is stored and evaluated from both of its
 * particles; enable = 1 switches to the half list of Newton's third law, in
 * which each pair is stored once (in the list of the particle that comes
 * first in the cell order) and its force is added to one particle and
 * subtracted from the other.  The partner's share goes through 64-bit integer
 * atomic adds into fixed-point force sums of 3 x (slots) int64 that the
 * handle allocates on the first enable and keeps until md_destroy; the
 * integration then runs as a second kernel.  Both forms give bit-identical
 * forces and trajectories: every pair force is rounded to the fixed point the
 * same way whichever end evaluates it, and the sums are exact.  Energies and
 * virials agree to FP32 rounding.  The next step, force or list call rebuilds
 * the list on `stream`.  MD_ERR_ARG for enable = 1 with MD_FP64, with FENE
 * bonds or angle triples; md_forward / md_backward need the full list and
 * return MD_ERR_ARG while the half list is on.  MD_ERR_CUDA if the sums cannot
 * be allocated. */
md_status md_set_half_list(md_handle *h, int32_t enable, void *stream);

/* Wait for all work on `stream` and return any latched device error. */
md_status md_sync(md_handle *h, void *stream);

/* Counters and latched errors; synchronises the device.  The counters are
 * those the paper reports for its runs (Sec. 4: steps, neighbour-list
 * rebuilds, neighbours per particle); the error word is this library's. */
md_status md_get_stats(md_handle *h, md_stats *out);

/* Section timers.  Sec. 4 of the paper splits the elapsed time of the
 * integrator loop into sections (Pair / Neigh / Integrate ...); here the
 * sections are the device-side cell sort + Verlet-list build chain
 * (MD_SECT_NEIGH, timed every step, whether or not it rebuilt), the fused
 * pair-force + velocity-Verlet kernel (MD_SECT_FORCE), and everything else in
 * md_step (MD_SECT_OTHER: the first half kick of a call, a force evaluation
 * when none is stored).  Timing uses CUDA events on the caller's stream. */
enum { MD_SECT_NEIGH = 0, MD_SECT_FORCE = 1, MD_SECT_OTHER = 2, MD_NSECT = 3 };

/* Enable (1) or disable (0) the section timers; enabling clears them. */
md_status md_set_timing(md_handle *h, int32_t enable);

/* Accumulated milliseconds and counts per section since md_set_timing(h, 1):
 * ms[MD_NSECT], counts[MD_NSECT] (host arrays, either may be NULL).
 * Synchronises the device. */
md_status md_get_timing(md_handle *h, double *ms, int64_t *counts);

/* Force evaluation that allocates nothing, for callers that cannot call
 * cudaMalloc: a host framework that owns every byte of device memory through
 * its own pool and forbids other allocators, or a process whose device memory
 * is already committed to a fixed budget.  The paper has no counterpart: it is
 * a convenience of this library.
 *
 * Computes only the non-bonded pair term of md_compute_forces (shifted LJ
 * when shift != 0, r < rc strict, minimum image in the orthorhombic box, FP32
 * pairs with 64-bit fixed-point sums or FP64), summed directly over all pairs
 * without cells or Verlet lists (O(n^2)), for ONE system of n particles.
 * FENE bonds and angle triples are not evaluated: for a system with bonded
 * terms the result differs from md_compute_forces.
 *   x      device, (3, n) FP64 positions      v     device, (3, n) or NULL (K = 0)
 *   box    host, 3 edges, each >= 2 rc        f_out device, (3, n) FP64 forces
 *   euw_out device, 3 FP64 (U, K, W) or NULL  err_msg/err_len optional host text buffer
 * Range: in MD_FP32_FIXED a pair closer than the fixed-point range allows
 * (|f| of one component near 2^21, r of about 0.44 sigma for LJ with eps = 1)
 * or two coincident particles make the force rows of both particles and the
 * U and W of euw_out NaN (K, from the velocities, is unaffected); the call
 * itself still returns MD_OK (it does not synchronise).
 * In MD_FP64 coincident particles give non-finite values.
 * Limits: 1 <= n <= 524288 (the fixed scratch), else MD_ERR_ARG with a message.
 * Scratch: a fixed 64 KB device array in the library, held by every GPU that
 * loads it until the process exits; every call shares it, so calls that
 * overlap on the GPU race.  Nothing is allocated or freed.  The first call on
 * a device looks up the scratch address with that device current and keeps
 * it for the life of the process (a cudaDeviceReset, which ends the primary
 * context, leaves a stale address: do not call this after one); make that
 * first call before any stream capture.  Asynchronous on `stream`. */
md_status md_compute_forces_noalloc(const double *x, const double *v, int64_t n, const double *box,
                                    double eps, double sigma, double rc, int32_t shift, int32_t precision,
                                    double mass, double *f_out, double *euw_out, char *err_msg,
                                    int32_t err_len, void *stream);

/* Text of the last error on this handle ("" if none).  Valid until the next
 * call.  No passage of the paper: error reporting of this library. */
const char *md_last_error(const md_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* MD_GB300_H */
