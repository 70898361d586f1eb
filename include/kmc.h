/*
 * kmc.h -- C ABI of libkmc, a GB300 (sm_103a) library for the per-time-step
 * collision step of the kinetic Monte Carlo hard-sphere gas described in
 * Howell et al., "Parallelization of Kinetic Theory Simulations" (arXiv:1310.3437).
 *
 * One time step (Sec. 2 "Initial Simulation Setup" and Sec. 3):
 *   1. particles are binned into cells (Sec. 2, grid of bins);
 *   2. every particle finds its closest collision partner by distance of closest
 *      approach among the particles of its own and the neighbouring cells
 *      (Sec. 2, the three criteria and the "closer partner replaces" rule);
 *   3. particles that chose each other collide (Sec. 2, mutual choice), repeated
 *      over the still-unmatched particles for up to max_rounds rounds;
 *   4. colliding pairs scatter isotropically in their centre-of-mass frame;
 *   5. all particles free-stream and the box boundaries are applied (Sec. 2,
 *      reflective or periodic walls; here also a moving piston).
 *
 * Conventions for every entry point:
 *   - Status: 0 (KMC_OK) or a negative KMC_E* code.  No C++ exception crosses
 *     this interface.  sim_last_error() gives a message for the last failure.
 *   - Asynchrony: work is enqueued on the CUDA stream given at creation and the
 *     call returns before it finishes.  sim_sync() waits and reports device-side
 *     errors (a buffer that overflowed, an exhausted random draw).
 *   - Pointers: arrays passed in or out may be device memory or host memory
 *     (pinned or pageable); the library copies with cudaMemcpyDefault.  The caller
 *     keeps ownership of everything it passes.  The library owns and frees its
 *     own buffers in sim_destroy / sim_group_destroy.
 *   - Layout: particle arrays are structure-of-arrays, indexed by particle id
 *     0..n-1.  Positions and velocities are IEEE-754 binary64.
 */
#ifndef KMC_H
#define KMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define KMC_OK 0
#define KMC_EINVAL (-1)    /* bad argument or parameter */
#define KMC_ENOMEM (-2)    /* device allocation failed */
#define KMC_ECUDA (-3)     /* a CUDA runtime call failed */
#define KMC_ETIMEOUT (-4)  /* a bounded device-side wait ran out: a tile of the cell
                              scan waited about a second for its predecessor's sum (the
                              step's results are void; sim_sync reports it) */
#define KMC_EOVERFLOW (-5) /* a buffer capacity was exceeded and could not grow */
#define KMC_ESTATE (-6)    /* call not allowed in the current state */
#define KMC_ERANDOM (-7)   /* 128 rejected sphere-point draws (probability ~1e-43) */

/* ---- boundary kinds per axis (Sec. 2: reflective or periodic box) -------- */
#define KMC_PERIODIC 0
#define KMC_REFLECT 1  /* walls at 0 and at the box end; on x the end wall may move */
#define KMC_ABSORB 2   /* absorptive walls (Sec. 2) at 0 and at the box end: a particle
                          whose end-of-step position lies beyond one (x < 0 or x > L)
                          leaves the gas: it keeps that position and its velocity, its
                          last partner becomes KMC_ABSORBED, and it is neither searched,
                          moved nor profiled again.  Live particles lie in [0, L]. */

/* ---- precision of the pair tests --------------------------------------- */
#define KMC_FP64 0          /* every pair test in binary64 */
#define KMC_GUARDED_FP32 1  /* binary32 pre-tests with proven guard bands, binary64
                               re-check of the survivors: identical pair lists */

/* ---- observables (sim_observe) ------------------------------------------
 * The paper writes its output after the particles are sorted into their bins
 * (Sec. 2, "Initial Simulation Setup") and only at a fixed interval of simulated
 * time, kept by a time-step counter (Sec. 3, "Algorithm Optimization"): here the
 * state, partners and candidate pairs describe the last completed step, per-step
 * counts are kept for every step, and the profiles every profile_every steps. */
#define KMC_OBS_STATE 1    /* 6 x n binary64 (x,y,z,vx,vy,vz) then n uint32 last
                              partner id (KMC_NONE if none): 52 n bytes */
#define KMC_OBS_PARTNERS 2 /* n uint32: partner id of each particle in the last
                              completed step, KMC_NONE if it did not collide */
#define KMC_OBS_COUNTS 3   /* kmc_step_counts records of the steps completed since
                              the previous COUNTS call (oldest first) */
#define KMC_OBS_PROFILES 4 /* profile snapshots taken since the previous PROFILES
                              call: per snapshot, profile_bins x 7 binary64 (count,
                              sum vx, vy, vz, sum vx^2, vy^2, vz^2 over the particles in
                              the gas with x in the bin).  The sums are exact fixed-point
                              sums rounded once; a bin holding a velocity component with
                              |v| >= 46341 (a square >= 2^31, beyond the fixed point's
                              range) has NaN for its six sums, its count stays exact */
#define KMC_OBS_EDGES 5    /* candidate pairs of the last completed step as uint32
                              (id_lo, id_hi) pairs, unordered list */
#define KMC_OBS_STEP 6     /* one uint64: absolute index of the next step */
#define KMC_OBS_LAUNCHES 7 /* one uint64: kernel launches enqueued for this simulation
                              (steps of its group included) */
#define KMC_OBS_PHASE_MS 8 /* 5 or 6 binary64 (as dst holds): milliseconds spent in the
                              sort, search, matching (exact test, lists, rounds,
                              scatter) and push phases while timing was on, the number
                              of timed steps, then the milliseconds of the main search
                              kernel alone (the one that searches the slow population:
                              row, cell or particle search), part of the search phase */
#define KMC_OBS_VMAX 9     /* one binary64: the largest particle speed of the current
                              state, sqrt(max ((vx*vx + vy*vy) + vz*vz)) over the particles
                              in the gas, each operation correctly rounded (0 for an
                              empty gas).  Sec. 2 derives the time step from the maximum
                              speed and Sec. 4 reduces it over all domains; here it sizes
                              the cells (d0 + 2 v_max dt) and the speed split */
#define KMC_OBS_DOMAINS 10 /* a decomposition (sim_create_domains): 2 x ndomains uint32,
                              the particles each domain owned in the last step, then
                              the ghosts it held (Sec. 4: the first phase's counts) */

#define KMC_NONE 0xFFFFFFFFu
#define KMC_ABSORBED 0xFFFFFFFEu /* last-partner value of a particle that has left
                                    through an absorbing wall (KMC_OBS_STATE; may be
                                    passed back to sim_create to resume) */

/* ---- flags (kmc_params.flags) --------------------------------------------- */
#define KMC_FLAG_NO_SPLIT 1u   /* never split fast particles into a second population
                                  (the speed split changes the work, never a result) */
#define KMC_FLAG_FORCE_SPLIT 2u /* split whenever possible, cycling the threshold through
                                  the trial values step by step (exercises the split) */
#define KMC_FLAG_PLANAR 4u     /* two-dimensional dynamics in the x-y plane (the paper's
                                  2D runs, Sec. 2 and Sec. 4: 8 neighbouring bins): every
                                  vz must be 0, z stays constant, scatter directions are
                                  isotropic in the plane (uniform on the unit circle, von
                                  Neumann's method from the same Philox draws).  Give the
                                  z axis an extent below 3 cells (one cell: a 9-cell
                                  stencil) and reflecting walls.  sim_create fails with
                                  KMC_EINVAL if a vz is not 0. */
#define KMC_FLAG_SCAN_WAIT_TEST 8u /* test of the failure path only: the cell scan's tiles
                                  wait for a status word that is never written, run into
                                  their bounded wait and sim_sync returns KMC_ETIMEOUT */

/* ---- search kernels (kmc_params.search_kernel) ----------------------------- */
#define KMC_SEARCH_AUTO 0      /* per step: warp-per-cell search when cells are well
                                  filled, the row search (binary32) or the
                                  thread-per-particle search (binary64) otherwise */
#define KMC_SEARCH_PARTICLE 1  /* one thread per particle, cell by cell */
#define KMC_SEARCH_CELL 2      /* one warp per cell, partners in lanes */
#define KMC_SEARCH_ROW 3       /* one lane per particle walking whole stencil rows as
                                  partner ranges (guarded binary32; binary64 uses
                                  KMC_SEARCH_CELL) */

/* Parameters of one simulation.  Zero-initialise, then set the fields. */
typedef struct kmc_params {
  uint32_t n;              /* particles, >= 1 */
  uint32_t flags;          /* 0 or KMC_FLAG_* bits */
  double box[3];           /* box extents L_x, L_y, L_z; particles live in [0, L) */
  int32_t bc[3];           /* KMC_PERIODIC, KMC_REFLECT or KMC_ABSORB per axis */
  int32_t max_rounds;      /* mutual-choice rounds per step, 1..4 (0 means 4) */
  double piston_x0;        /* reflecting x axis: upper wall at piston_x0 - piston_u*t */
  double piston_u;         /*   (set piston_x0 = box[0], piston_u = 0 for a fixed wall) */
  double d0;               /* collision diameter (effective radius sum), > 0 */
  double dt;               /* time step, > 0 */
  uint64_t seed;           /* Philox4x32-10 key of the scatter directions */
  uint64_t step0;          /* absolute index of the first step (resume) */
  int32_t precision;       /* KMC_FP64 or KMC_GUARDED_FP32 */
  int32_t profile_bins;    /* x-profile bins (0 = no profiles) */
  int32_t profile_every;   /* profile after every step s with (s+1) % every == 0 */
  int32_t stencil;         /* cells per search radius: 1 (27-cell search) or 2
                              (125 half-size cells); 0 means 1.  Never changes results. */
  double profile_range;    /* profiles cover x in [0, profile_range) */
  double cell_scale;       /* >= 1: cell size multiplier (occupancy knob); 0 means 1.
                              Never changes results. */
  uint32_t edge_cap;       /* initial candidate-pair capacity (0: automatic); grows on
                              demand at sim_sync */
  uint32_t history_cap;    /* step records kept for KMC_OBS_COUNTS (0: 4096) */
  uint32_t profile_cap;    /* profile snapshots kept for KMC_OBS_PROFILES (0: 64) */
  int32_t search_kernel;   /* KMC_SEARCH_AUTO (0), KMC_SEARCH_PARTICLE (1),
                              KMC_SEARCH_CELL (2) or KMC_SEARCH_ROW (3).
                              Never changes results. */
  double split_min_occ;    /* speed split only if the slow grid keeps at least this
                              many particles per cell on average (0: no floor).
                              Never changes results. */
} kmc_params;

/* One record per completed step (KMC_OBS_COUNTS). */
typedef struct kmc_step_counts {
  uint64_t step;            /* absolute step index */
  uint32_t collisions;      /* colliding pairs */
  uint32_t edges;           /* candidate pairs (before matching) */
  uint32_t round_pairs[4];  /* pairs matched in rounds 1..4 */
  uint32_t survivors;       /* pairs that passed the search pre-tests */
  uint32_t cells;           /* cells of the search grid */
  uint64_t pair_tests;      /* pair tests done by the search */
  uint64_t fast_tests;      /* the part of pair_tests done for the fast particles of the
                               speed split (the rest is the slow-population search) */
  uint32_t absorbed;        /* particles that left through absorbing walls this step */
  uint32_t live;            /* particles in the gas after the step */
} kmc_step_counts;

typedef struct kmc_sim kmc_sim;
typedef struct kmc_group kmc_group;

/* Create a simulation from an initial state (Sec. 2: particles initialised in a
 * box).  x..vz: n binary64 each, id order, host or device.  last: n uint32 last
 * collision partner ids or NULL (none).  stream: a cudaStream_t (NULL: the library
 * creates a stream of its own).  The arrays are copied; the caller keeps them.
 * Errors: KMC_EINVAL (bad parameter, particle outside the box), KMC_ENOMEM,
 * KMC_ECUDA.  On error *out is NULL. */
int sim_create(const kmc_params* p, const double* x, const double* y, const double* z,
               const double* vx, const double* vy, const double* vz, const uint32_t* last,
               void* stream, kmc_sim** out);

/* Create a mixture (Sec. 2: every particle carries a mass and an effective radius).
 * As sim_create, plus: species, n uint8 indices by particle id (host or device);
 * mass and radius, nspecies (1..256) binary64 values each in HOST memory.  A pair
 * (i, j) is in contact at radius[s_i] + radius[s_j]; p->d0 is the search reach and
 * must be at least 2 max(radius).  A collision keeps the centre-of-mass velocity
 * V = (m_a v_a + m_b v_b)/M and turns the relative velocity isotropically:
 * v_a' = V + (m_b/M) |g| n, v_b' = V - (m_a/M) |g| n (M = m_a + m_b, a the smaller
 * id; for equal power-of-two masses this is the single-species update bit for bit).
 * Profiles stay unweighted (counts and velocity sums over all species).
 * Errors: as sim_create, and KMC_EINVAL for a bad table, d0 < 2 max(radius) or a
 * species index >= nspecies. */
int sim_create_mixture(const kmc_params* p, const double* x, const double* y, const double* z,
                       const double* vx, const double* vy, const double* vz, const uint32_t* last,
                       const uint8_t* species, uint32_t nspecies, const double* mass,
                       const double* radius, void* stream, kmc_sim** out);

/* ---- device-side initial states (sim_create_init) ------------------------ */
#define KMC_INIT_MAXWELL 1     /* positions uniform in the box, velocity components
                                  i.i.d. N(0, sigma^2) (the equilibrium box and the
                                  piston tube) */
#define KMC_INIT_EQUAL_SPEED 2 /* positions uniform in the box, |v| = speed, direction
                                  uniform on the sphere (the paper's timing runs,
                                  Sec. 3 and Sec. 4) or, planar, on the circle */
#define KMC_INIT_BLAST 3       /* ids below n_hot uniform in the ball |x - center| <
                                  radius with N(0, sigma_hot^2) components, the others
                                  uniform in the box outside it with N(0, sigma^2) */

/* Initial-state descriptor.  Draws: Philox4x32-10 keyed by params.seed, counter
 * (id, 0xFFFFFFFF, k, 0xFFFFFFFF) -- the collision counter of step 2^64 - 1, which
 * no run reaches; blocks k = 0..127 for positions (53-bit uniforms, rejection for
 * the blast's ball), k = 128..191 for velocities (Marsaglia's polar method with a
 * logarithm built from +, -, *, /; directions as in the collision update).  Planar
 * (KMC_FLAG_PLANAR): z = box[2]/2, vz = 0.  The arrays depend only on (params,
 * descriptor), bit for bit, not on the GPU or the launch. */
typedef struct kmc_init {
  uint32_t kind;      /* KMC_INIT_* */
  uint32_t pad0;
  uint64_t n_hot;     /* BLAST: number of hot particles (ids 0..n_hot-1), <= n */
  double sigma;       /* MAXWELL, BLAST (outside): per-component standard deviation */
  double speed;       /* EQUAL_SPEED: the common speed */
  double sigma_hot;   /* BLAST (inside) */
  double center[3];   /* BLAST: ball centre; the ball must lie strictly inside the box */
  double radius;      /* BLAST: ball radius > 0 */
} kmc_init;

/* Create a simulation whose initial state is drawn on the device (no host arrays,
 * no host-to-device copy of the state): ids 0..n-1, no last partners.  Same
 * parameters, stream and ownership rules as sim_create.  Errors: KMC_EINVAL (bad
 * parameter or descriptor: unknown kind, negative or non-finite sigma/speed, a ball
 * not strictly inside the box, n_hot > n, BLAST with KMC_FLAG_PLANAR),
 * KMC_ERANDOM (a rejection loop ran out of its 64 attempts; probability below
 * 1e-20 per particle), KMC_ENOMEM, KMC_ECUDA.  On error *out is NULL. */
int sim_create_init(const kmc_params* p, const kmc_init* init, void* stream, kmc_sim** out);

/* Create a simulation decomposed into ndomains (1..64) equal slabs along x, the
 * domain decomposition of Sec. 4 ("Hybrid Simulations"), run on this GPU.  Domain k
 * owns the particles with X_k <= x < X_(k+1), X_k = k X / ndomains (X the box length,
 * or the larger of it and piston_x0 on a reflecting x axis), and holds as ghosts the
 * particles within the reach d0 + 2 v_max dt of its slab.  Every step runs the
 * paper's four communication phases between the domains: ghosts (with their counts),
 * the global v_max, the collision partners of ghosts in every matching round, and the
 * migration of particles that crossed a cut.  Results -- state, partners, candidate
 * pairs, step counts -- are bit for bit those of sim_create on the same input; the
 * decomposition changes the work, never a result.  sim_step, sim_sync, sim_observe
 * (STATE, PARTNERS, EDGES, COUNTS, STEP, VMAX, LAUNCHES, DOMAINS) and sim_destroy
 * apply; it cannot join a group and keeps no profiles.  The exchanges go through
 * id-indexed device buffers on this GPU (no inter-GPU transport).  Arguments as
 * sim_create.  Errors: KMC_EINVAL (as sim_create, and: ndomains outside 1..64, an
 * absorbing axis, profile_bins != 0), KMC_ENOMEM, KMC_ECUDA; sim_sync returns
 * KMC_EOVERFLOW if a domain's candidate-pair buffer overflowed (no regrowth: each
 * domain's buffer holds edge_cap pairs, by default one per particle).  Device memory: about ndomains times that of
 * sim_create, plus 4 ndomains + 70 bytes per particle. */
int sim_create_domains(const kmc_params* p, uint32_t ndomains, const double* x, const double* y,
                       const double* z, const double* vx, const double* vy, const double* vz,
                       const uint32_t* last, void* stream, kmc_sim** out);

/* Enqueue nsteps time steps (Sec. 2: sort, detect, collide, stream, boundaries).
 * Errors: KMC_ESTATE if the simulation belongs to a group, KMC_ECUDA. */
int sim_step(kmc_sim* s, uint32_t nsteps);

/* Wait for the enqueued steps.  If a candidate-pair buffer overflowed, it is grown
 * and the unfinished steps are re-run from the last completed step (results do not
 * change).  For a member of a group this is sim_group_sync of its group.
 * Errors: KMC_ERANDOM, KMC_EOVERFLOW, KMC_ENOMEM, KMC_ECUDA. */
int sim_sync(kmc_sim* s);

/* Copy an observable (KMC_OBS_*) into dst (host or device, dst_bytes long): the
 * paper's output (Sec. 2: after the sort; Sec. 3: at a fixed interval of simulated
 * time).  The copy is ordered after the enqueued steps; for a host dst the call
 * waits.  Returns the number of items written (records, snapshots, pairs, or 1) or
 * a negative status: KMC_EINVAL (unknown observable, dst too small), KMC_ENOMEM
 * (a staging buffer for a host dst), KMC_ECUDA. */
int64_t sim_observe(kmc_sim* s, int what, void* dst, size_t dst_bytes);

/* Diagnostics: with enable != 0, later sim_step calls launch the kernels one by one
 * (no CUDA graph) with CUDA events around each phase on the simulation's stream, and
 * wait for each step; KMC_OBS_PHASE_MS returns the accumulated times.  enable = 0
 * restores graph replay.  Results do not change. */
int sim_set_timing(kmc_sim* s, int enable);

/* Free the simulation (waits for its stream).  NULL is accepted. */
int sim_destroy(kmc_sim* s);

/* Message of the last failure on s (or of the last failed sim_create if s is
 * NULL).  Never NULL. */
const char* sim_last_error(const kmc_sim* s);

/* Device bytes sim_create would allocate for these parameters (admission control). */
size_t sim_bytes_required(const kmc_params* p);

/* X-profile of a particle state that allocates no device memory.  The paper has no
 * counterpart: it is an observable for callers that cannot call cudaMalloc (a host
 * application whose pool allocator owns all device memory, an in-situ analysis
 * step inside another code's time loop where an allocation would synchronise the
 * device, a tool handed only device pointers).  It returns the same bins x 7
 * binary64 values as KMC_OBS_PROFILES -- per x bin over [0, range): count, sum vx,
 * sum vy, sum vz, sum vx^2, sum vy^2, sum vz^2 -- for the n particles in the caller's
 * device arrays x, vx, vy, vz (any order), into the caller's device array out.
 * Limits: n < 2^31 (the fixed-point digit sums are int64); a bin holding a velocity
 * component with |v| >= 46341 (a square >= 2^31) gets NaN for its six sums, as in
 * KMC_OBS_PROFILES.  Scratch: a fixed array of 256 x 20 int64 counters (40,960
 * bytes) compiled into the library; every GPU that loads the library holds it until
 * the process exits.  bins above 256 (or below 1), range <= 0, n >= 2^31, NULL or
 * host pointers, memory of another device, or a stream of another device:
 * KMC_EINVAL, with a line on stderr.  The first call on a device, with that device
 * current, looks up the array's device address; make that first call before any
 * stream capture.  Calls share the array and it keeps the last call's contents
 * (each call clears the counters it uses first); calls that overlap on the GPU race
 * and return wrong sums, so order them on one stream.  Enqueued on stream; out is
 * valid after the stream synchronises.  Calls no cudaMalloc, cudaFree or
 * allocating library routine. */
int sim_profile_static(const double* x, const double* vx, const double* vy, const double* vz,
                       uint32_t n, int32_t bins, double range, double* out, void* stream);

/* ---- batching ------------------------------------------------------------ */
/* The paper runs one simulation per job, split over nodes (Sec. 4); a group is the
 * GPU's form of many independent jobs at once (no exchange between members, so
 * each member's results equal its run alone).
 * A group steps many simulations of uneven size with one launch per kernel for
 * all of them; the per-step launch sequence is captured in a CUDA graph.  All
 * members must share precision and stencil.  Members keep their own state and can
 * still be observed; sim_step on a member returns KMC_ESTATE.
 * Errors: KMC_EINVAL (empty, mixed precision, member already grouped). */
int sim_group_create(kmc_sim* const* sims, uint32_t count, void* stream, kmc_group** out);
/* Add or remove a member between steps (continuous batching). */
int sim_group_add(kmc_group* g, kmc_sim* s);
int sim_group_remove(kmc_group* g, kmc_sim* s);
/* Give member s a budget of nsteps more steps; a member with no steps left is
 * skipped by the group's launches. */
int sim_group_budget(kmc_group* g, kmc_sim* s, uint32_t nsteps);
/* Enqueue nsteps group steps (each member advances while its budget lasts). */
int sim_group_step(kmc_group* g, uint32_t nsteps);
/* Steps left in member s's budget (waits for the group's stream). */
int64_t sim_group_steps_left(kmc_group* g, kmc_sim* s);
/* Wait for the group's steps.  A member whose candidate-pair buffer overflowed was
 * skipped by the group's later steps: its buffer is grown and the steps it missed
 * since the previous sync run for it alone (within its budget), so that afterwards
 * every member stands where the group's steps took the others (results do not
 * change).  Errors: as sim_sync, for the worst member. */
int sim_group_sync(kmc_group* g);
int sim_group_destroy(kmc_group* g);

#ifdef __cplusplus
}
#endif

#endif /* KMC_H */
