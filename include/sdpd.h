/*
 * sdpd.h -- C ABI of the GB300 library for one time step of Smoothed
 * Dissipative Particle Dynamics (SDPD) integrated by Velocity Verlet and a
 * Shardlow-like pairwise fluctuation/dissipation sweep with the Metropolis
 * corrections of Faure & Stoltz, "Stable and accurate schemes for Smoothed
 * Dissipative Particle Dynamics".
 *
 * Conventions shared by every call:
 *  - Units are the caller's; kB is a parameter (1 in reduced units).
 *  - Arrays cross the boundary in particle-id order: particle k of the array
 *    given to sdpd_set_state has id k.  Positions and momenta are [N][3]
 *    row-major float64, internal energies [N] float64.
 *  - "on_device" = 1: the pointer is CUDA device memory of the current
 *    device; 0: host memory (pinned or pageable).
 *  - The caller owns every pointer it passes; the library copies from it and
 *    keeps nothing.  Device memory of the library is one workspace that the
 *    caller allocates (sdpd_workspace_bytes) and binds (sdpd_bind_workspace);
 *    the library calls no allocator.
 *  - Every call returns an int status (SDPD_OK = 0 or an SDPD_ERR_* code);
 *    errors found by device code are sticky and are returned by the next
 *    call that synchronises (sdpd_observables, sdpd_get_state, sdpd_sync).
 *  - Work is enqueued on the CUDA stream given to sdpd_create.  Only the
 *    calls documented as synchronising wait for it.
 */
#ifndef SDPD_H
#define SDPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SDPD_OK 0
#define SDPD_ERR_INVALID_ARG 1        /* a parameter is out of its domain */
#define SDPD_ERR_BOX_TOO_SMALL 2      /* fewer than 4 cells (even) of side >= h on an axis */
#define SDPD_ERR_NONPOSITIVE_ENERGY 3 /* sdpd_set_state got eps_i <= 0 or a non-finite value */
#define SDPD_ERR_NEGATIVE_ENERGY 4    /* the SSA scheme produced eps_i <= 0 (no rejection in SSA) */
#define SDPD_ERR_NAN 5                /* a non-finite momentum or energy was found */
#define SDPD_ERR_CUDA 6               /* a CUDA runtime call failed */
#define SDPD_ERR_TIMEOUT 7            /* a bounded device wait ran out */
#define SDPD_ERR_NO_WORKSPACE 8       /* no (or too small a) workspace is bound */
#define SDPD_ERR_CAPACITY 9           /* a fixed capacity without a fallback was exceeded (the
                                         gradient passes' neighbour-list rows of 160 entries;
                                         sdpd_density_static's static working memory) */
#define SDPD_ERR_NO_STATE 10          /* sdpd_step/get_state before sdpd_set_state */
#define SDPD_ERR_HOST_MEMORY 11       /* a host-side table could not be allocated */

/* smoothing kernels */
#define SDPD_KERNEL_CUBIC 0 /* cubic spline, Eq. (sdpd-cubic-w) */
#define SDPD_KERNEL_LUCY 1  /* Lucy: W = 105/(16 pi h^3)(1+3x)(1-x)^3, x = r/h */

/* fluctuation/dissipation schemes */
#define SDPD_SCHEME_SSA 0  /* Shardlow-like splitting, Section 3.2: every move accepted */
#define SDPD_SCHEME_AMS 1  /* approximate Metropolis, Section 3.3.3: energy bound only */
#define SDPD_SCHEME_EMS 2  /* exact Metropolis, Section 3.3.2: bound + ratio of Eq. (metropolis-ratio) */
#define SDPD_SCHEME_NONE 3 /* Velocity Verlet only (the paper's "Verlet" timing reference) */

/* arithmetic of the device path */
#define SDPD_FP64 0  /* every operation in float64 */
#define SDPD_MIXED 1 /* pair arithmetic in float32; eps, its updates and energy sums in float64 */

typedef struct sdpd_handle sdpd_t;

typedef struct {
  double kB;     /* Boltzmann constant */
  double eta;    /* shear viscosity eta > 0 (Section 2.2.2) */
  double zeta;   /* bulk viscosity, 0 <= zeta < 5 eta / 3 so both kappa are > 0 */
  double c_rho;  /* density coefficient of the ideal-gas entropy
                    S = C_K ln eps - c_rho ln rho (Eq. pg-eos); < 0 selects (K-1)/2 */
  int kernel;    /* SDPD_KERNEL_* */
  int scheme;    /* SDPD_SCHEME_* */
  int precision; /* SDPD_FP64 or SDPD_MIXED */
  int fd_only;   /* 1: skip Velocity Verlet, run the fluctuation/dissipation sweep
                    only (Section 4.1) */
  int theta;     /* multiple time step ratio (Section 4.2): one sweep with time
                    step theta*dt after each Verlet step whose count since
                    sdpd_set_state is a multiple of theta (however the steps
                    are split over sdpd_step calls); 1 = single step */
  int debug;     /* 1: reserve workspace for per-pair records (sdpd_debug_get) */
  int nc[3];     /* cells per axis; 0 = the largest even n with box/n >= h.  Else
                    an even n >= 4 with box/n >= h (SDPD_ERR_INVALID_ARG if odd
                    or < 4, SDPD_ERR_BOX_TOO_SMALL if box/n < h).  The cell grid
                    fixes the colouring and so the order of the sweep's pair
                    updates; any grid gives a valid sweep of Section 3.2. */
  int sweep_f32; /* float64 handles: 1 runs the fluctuation/dissipation sweep with
                    float32 pair arithmetic on the float64 state, as the mixed path
                    does (momenta and energies receive float32 increments; density,
                    Velocity Verlet and the gradients stay float64).  Ignored by
                    mixed handles. */
} sdpd_params;

/* Observables of the current state (Section 2.2: E and the total momentum
 * are the invariants of the dynamics).  All sums in float64. */
typedef struct {
  double E;          /* total energy sum_i eps_i + |p_i|^2 / (2m) */
  double E_int;      /* sum_i eps_i */
  double E_kin;      /* sum_i |p_i|^2 / (2m) */
  double P[3];       /* total momentum */
  double T_kin;      /* sum_i |p_i|^2 / (3 (N-1) m kB) */
  double T_int;      /* mean internal temperature (1/N) sum_i T(eps_i) */
  double eps_min;    /* smallest internal energy */
  int64_t n_pairs;   /* pair updates since the last counter reset */
  int64_t n_accept;
  int64_t n_reject_bound;      /* rejected by the energy bound, Eq. (energy-bound) */
  int64_t n_reject_metropolis; /* rejected by U > A of Eq. (metropolis-ratio) */
  int64_t fd_step;   /* fluctuation/dissipation sweeps done (the random-number step) */
  int64_t vv_step;   /* Velocity Verlet steps done */
  int status;        /* sticky device status (SDPD_OK or an error code) */
} sdpd_obs;

/* Create a handle for N particles in the periodic box [0,box[0]) x ... of the
 * paper's problem statement (Section 2.1: N particles of mass m, smoothing
 * length h; Section 4: ideal gas of particle size K, heat capacity
 * C_K = 3/2 (K-1) kB).  Host only: validates the parameters (K > 4/3 so that
 * d_ij < 1 in Eq. (sdpd-gamma-sigma); every box side gives an even number
 * >= 4 of cells of side >= h), chooses the cell grid and the workspace size.
 * stream: a cudaStream_t (NULL = the legacy default stream).
 * Errors: SDPD_ERR_INVALID_ARG, SDPD_ERR_BOX_TOO_SMALL, SDPD_ERR_HOST_MEMORY
 * (the per-cell tables, 4 + 4 + 16 bytes per cell, do not fit in host
 * memory).  *out is NULL on error. */
int sdpd_create(int64_t N, const double box[3], double m, double h, const sdpd_params* params,
                double K, void* stream, sdpd_t** out);

/* Bytes of device workspace the handle needs (256-byte aligned start). */
size_t sdpd_workspace_bytes(const sdpd_t* s);

/* Bind caller-allocated device memory of at least sdpd_workspace_bytes bytes
 * on the current device.  The library never frees it.  Uploads the cell
 * tables (asynchronous on the handle's stream).
 * Errors: SDPD_ERR_NO_WORKSPACE (NULL, too small or misaligned), SDPD_ERR_CUDA. */
int sdpd_bind_workspace(sdpd_t* s, void* device_ptr, size_t bytes);

/* Load a state (q[N][3], p[N][3], eps[N], float64, id order) and prepare it:
 * cell binning and sorting, then the densities of Eq. (sdpd-rho-v) and the
 * pressures of Section 2.1.2.  Positions outside [0, L) are wrapped.  Resets
 * the sweep counter (random-number step) to 0 and the pair counters.
 * Host pointers are copied before the call returns; device pointers are read
 * on the stream.  Errors: SDPD_ERR_NO_WORKSPACE, SDPD_ERR_NONPOSITIVE_ENERGY
 * (eps_i <= 0 or non-finite, checked on the host when on_device = 0, else
 * reported at the next synchronising call), SDPD_ERR_CUDA. */
int sdpd_set_state(sdpd_t* s, const double* q, const double* p, const double* eps, int on_device);

/* Copy the state back in id order (positions wrapped into [0, L)).
 * Synchronises the stream; returns the sticky device status. */
int sdpd_get_state(sdpd_t* s, double* q, double* p, double* eps, int on_device);

/* Advance nsteps Velocity Verlet steps of size dt (Eq. sdpd-verlet, entropies
 * fixed during the step, Section 3.1), each followed -- every theta steps --
 * by one fluctuation/dissipation sweep over all pairs r_ij < h with step
 * theta*dt (Sections 3.2-3.3).  The sweep visits the pairs in the colour
 * order of the library (8 cell-parity colours; within a colour the 2x2x2
 * cell blocks are independent; within a block pairs go by (rank difference,
 * lower rank), rank = position of the id among the block's particles)
 * and draws the pair's random numbers from Philox4x64-10 keyed by seed with
 * counter (sweep number, min id, max id, 0).  Any local density completes:
 * a particle with more than 160 neighbours has its forces summed from the
 * cells instead of its list, and a block with more than 256 particles, 2048
 * owned pairs or 255 dependency levels, or with a member of more than 160
 * neighbours, is swept pair by pair in the same order (slower, same
 * result; SDPD_DEBUG_BIG counts such blocks).  Asynchronous on the handle's
 * stream.
 * Errors: SDPD_ERR_INVALID_ARG (dt <= 0, nsteps < 0), SDPD_ERR_NO_STATE,
 * SDPD_ERR_CUDA; device errors are sticky. */
int sdpd_step(sdpd_t* s, double dt, int64_t nsteps, uint64_t seed);

/* Reduce the observables of the current state (float64) and copy them to
 * *out.  Synchronises the stream; returns out->status. */
int sdpd_observables(sdpd_t* s, sdpd_obs* out);

/* Wait for the stream; return the sticky device status. */
int sdpd_sync(sdpd_t* s);

/* Set / read the sweep counter (the random-number step), e.g. to resume a
 * run from a saved state: 20 steps equal 10 steps, sdpd_get_state,
 * sdpd_set_state, sdpd_set_fd_step(10), 10 steps. */
int sdpd_set_fd_step(sdpd_t* s, int64_t fd_step);
int64_t sdpd_get_fd_step(const sdpd_t* s);

/* Reset the pair counters of sdpd_obs. */
int sdpd_reset_counters(sdpd_t* s);

/* Number of CUDA kernels the handle has launched so far (a VV step launches
 * 8, a sweep 9 plus 5 when its schedule is rebuilt -- it is reused while the
 * positions do not change, as in FD-only runs -- sdpd_set_state 8,
 * sdpd_observables 2). */
int64_t sdpd_kernel_launches(const sdpd_t* s);

/* Per-stage timing with CUDA events recorded on the handle's stream around
 * every stage that sdpd_step launches.  Stages: 0 first kick + drift +
 * binning, 1 sort, 2 density + EOS, 3 second kick, 4 sweep schedule,
 * 5 sweep colours (8 launches per sweep); and of sdpd_vv_adjoint: 6 loading
 * a stored position (bin, sort, density), 7 pair pass A, 8 pair pass B,
 * 9 the elementwise steps between them.  sdpd_stage_times synchronises and
 * returns, per stage, the summed milliseconds and the number of kernel
 * launches since timing was enabled (arrays of n entries, n <= 10). */
#define SDPD_NSTAGES 10
int sdpd_enable_stage_timing(sdpd_t* s, int on);
int sdpd_stage_times(sdpd_t* s, double* ms, int64_t* launches, int n);

/* Histogram of the internal energies of the current state, for the
 * statistics of FD-only runs: the distribution of eps against the Gamma
 * marginal of Eq. (dist-analytic) and its error, Eq. (error-dist)
 * (Section 4.1).  With x_i = eps_i * scale and w = (hi - lo) / nbins, adds
 * to counts (device memory, nbins + 2 uint64 entries, owned by the caller):
 * counts[b] += #{i : lo + b w <= x_i < lo + (b + 1) w} for b < nbins
 * (b = floor((x - lo) / w) in float64, capped at nbins - 1),
 * counts[nbins] += #{x_i < lo}, counts[nbins + 1] += #{x_i >= hi or not
 * finite}.  Asynchronous on the handle's stream.  Errors:
 * SDPD_ERR_INVALID_ARG (nbins outside 1..4096, hi <= lo, non-finite bounds),
 * SDPD_ERR_NO_STATE. */
int sdpd_energy_histogram(sdpd_t* s, double lo, double hi, int nbins, double scale, unsigned long long* counts);

/* Debug read-outs (synchronising).  what:
 *  SDPD_DEBUG_ORDER   int64[N]   ids in storage order (Morton order of cells, then id)
 *  SDPD_DEBUG_CELLS   int32[N][3] cell of each particle, id order
 *  SDPD_DEBUG_RHO     double[N]  density rho_i, id order
 *  SDPD_DEBUG_FORCE   double[N][3] conservative force of Eq. (cons-forces) at the
 *                     current state, id order (computed on demand)
 *  SDPD_DEBUG_NCOUNT  int32[N]   number of neighbours j != i with r_ij < h, id order
 *  SDPD_DEBUG_PAIRS   sdpd_pair_rec[] of the last sweep (needs params.debug = 1),
 *                     one per pair in an order of the library's choosing
 *  SDPD_DEBUG_BIG     uint32[8]  per colour, the 2x2x2 cell blocks that the
 *                     latest sweep schedule left to the pair-by-pair sweep
 *                     (beyond its capacities: more than 256 particles, 2048
 *                     owned pairs or 255 dependency levels, or a member whose
 *                     neighbour list overflowed its row; Sections 3.2-3.3)
 * dst: host memory, cap = capacity in elements; *count receives the number
 * of elements written.  The capacity is checked before anything is copied.
 * Errors: SDPD_ERR_INVALID_ARG (unknown what or too small cap),
 * SDPD_ERR_NO_STATE, SDPD_ERR_HOST_MEMORY (staging buffers of N elements). */
#define SDPD_DEBUG_ORDER 0
#define SDPD_DEBUG_CELLS 1
#define SDPD_DEBUG_RHO 2
#define SDPD_DEBUG_FORCE 3
#define SDPD_DEBUG_NCOUNT 4
#define SDPD_DEBUG_PAIRS 5
#define SDPD_DEBUG_BIG 6

typedef struct {
  int64_t id_i, id_j; /* id_i < id_j */
  int32_t colour;     /* 0..7 */
  int32_t owner;      /* owner cell ox + nx (oy + ny oz) */
  int32_t decision;   /* 0 accept, 1 energy-bound reject, 2 Metropolis reject */
  int32_t level;      /* position of the pair in its block's dependency schedule */
  double margin;      /* EMS: a - ln U; otherwise the smaller new internal energy
                         (float64 on every path) */
  double margin_lo;   /* mixed EMS: the float32 estimate of a - ln U; otherwise = margin */
  double margin_tol;  /* mixed EMS: the bound on |margin_lo - margin| that decides when
                         the float64 value is evaluated; otherwise 0 */
} sdpd_pair_rec;

int sdpd_debug_get(sdpd_t* s, int what, void* dst, int64_t cap, int64_t* count);

/* Free the handle (not the workspace). */
void sdpd_destroy(sdpd_t* s);

/* Ensembles: many independent systems of uneven size and parameters stepped
 * together (the paper treats one system; independent replicas are how the
 * method is sampled in practice).  Each member is an ordinary handle with a
 * bound workspace and a loaded state, with stage timing off and debug off;
 * members may use multiple time steps (theta).  Members may share streams
 * (they then run one after the other) but not the ensemble's stream.
 * stream: the stream the ensemble launches on; NULL makes the ensemble create
 * a non-blocking stream of its own (sdpd_ensemble_stream returns it).
 * sdpd_ensemble_step advances every member by nsteps steps with its own seed
 * (seeds[i] for member i).  U = lcm(2, theta of every member) steps of all
 * members are captured once into one CUDA graph (forked from and joined into
 * the ensemble stream; the capture is redone when dt, the seeds, a
 * member's step count modulo its theta, its state buffer (after
 * sdpd_set_state or sdpd_autotune) or its launch shapes change) and the graph is replayed
 * nsteps/U times; the nsteps mod U last steps are enqueued directly.  Every
 * member's result is the same as stepping it alone.  The members' own
 * streams wait for the ensemble's work before later calls on them run.
 * Asynchronous.
 * Errors: SDPD_ERR_INVALID_ARG (bad or repeated member, a member on the
 * ensemble's stream, members' workspaces on different devices, timing or
 * debug on, U > 64), SDPD_ERR_NO_WORKSPACE, SDPD_ERR_CUDA,
 * SDPD_ERR_HOST_MEMORY. */
typedef struct sdpd_ensemble sdpd_ens_t;
int sdpd_ensemble_create(sdpd_t* const* members, int n, void* stream, sdpd_ens_t** out);
int sdpd_ensemble_step(sdpd_ens_t* e, double dt, int64_t nsteps, const uint64_t* seeds);
/* Chooses every member's launch shapes for the ensemble as a whole.  First
 * sdpd_autotune runs on every member alone (seeds[i], or 0 when seeds is
 * NULL).  Then the ensemble's graph is timed under each candidate
 * assignment: the defaults, the shapes each member chose alone, and each
 * colour-launch schedule given to every member (pair passes at 128 threads).
 * Each candidate gets one warm-up unit of U steps and then at least `steps`
 * timed steps, all from the saved states.  The fastest assignment is kept.
 * Shapes that win alone can lose when hundreds of members share the GPU,
 * which is why this second stage exists.  Every member's state and counters
 * are restored.  *ms_per_step (may be NULL) receives the ensemble's time
 * per step under the chosen shapes.  Synchronising.  Errors: those of
 * sdpd_autotune and sdpd_ensemble_step. */
int sdpd_ensemble_autotune(sdpd_ens_t* e, double dt, int64_t steps, const uint64_t* seeds, double* ms_per_step);
/* Kernel launches of the captured U-step graph (all members). */
int64_t sdpd_ensemble_kernel_nodes(const sdpd_ens_t* e);
/* The ensemble's stream (a cudaStream_t). */
void* sdpd_ensemble_stream(const sdpd_ens_t* e);
void sdpd_ensemble_destroy(sdpd_ens_t* e);

/* ---------------------------------------------------------------------------
 * Launch shapes and the autotuner (no counterpart in the paper: they choose
 * how the same arithmetic is mapped onto the GPU, never what it computes).
 * ------------------------------------------------------------------------- */

#define SDPD_FD_VARIANTS 5 /* block schedules of the sweep's colour launches */

typedef struct {
  int fd_variant;   /* blocks per warp x warps per thread block of the colour
                       launches: 0 (2 x 2), 1 (2 x 1), 2 (1 x 1), 3 (1 x 2),
                       4 (1 x 4); -1 = the precision's default (0 mixed,
                       1 float64).  Float64 handles take 1, 2 and 3 only (the
                       others need more than 48 KB of shared memory) */
  int pair_threads; /* threads per block of the density and force passes:
                       32, 64 or 128; 0 = 128 */
} sdpd_tuning;

/* Current launch shapes.  Errors: SDPD_ERR_INVALID_ARG. */
int sdpd_get_tuning(const sdpd_t* s, sdpd_tuning* out);

/* Sets the launch shapes used from the next launch on.  Results are
 * bitwise the same under every shape.  Errors: SDPD_ERR_INVALID_ARG. */
int sdpd_set_tuning(sdpd_t* s, const sdpd_tuning* t);

/* Measures the launch shapes on the loaded state and keeps the fastest:
 * first every colour-launch schedule (pair passes at 128 threads), then every
 * pair-pass block size with the best schedule.  Each candidate runs one
 * warm-up step and `steps` (1..1000) timed steps of dt from the same state,
 * timed with CUDA events on the handle's stream.  The loaded state, the step
 * counters, the random-number counter and the pair counters are restored
 * afterwards, so the next sdpd_step continues as if nothing had run (only
 * the per-pair debug records, when reserved, are those of the last trial).
 * best / ms_per_step (may be NULL) receive the chosen shapes and their time
 * per step.  Synchronising.  Errors: SDPD_ERR_INVALID_ARG, SDPD_ERR_NO_STATE,
 * SDPD_ERR_NO_WORKSPACE, SDPD_ERR_CUDA, or the sticky device status if the
 * state already carried an error. */
int sdpd_autotune(sdpd_t* s, double dt, int64_t steps, uint64_t seed, sdpd_tuning* best, double* ms_per_step);

/* ---------------------------------------------------------------------------
 * Gradients of the conservative dynamics with the sweeps frozen (reverse
 * mode; float64 handles without fd_only, else SDPD_ERR_INVALID_ARG).
 *
 * The differentiated map is nsteps steps x_{k+1} = VV(x_k) + D_k from the
 * loaded state (q^0, p^0, eps^0): one Velocity Verlet step, Eq.
 * (sdpd-verlet), with the entropies S_i = C_K ln eps_i - c_rho ln rho_i(q)
 * of the state at its start held fixed (Section 3.1: eps_i = E(S_i,
 * rho_i(q)) after the drift, pressures from Eq. (pg-eos)), then the
 * increments D_k of the momenta and internal energies that step k's
 * fluctuation/dissipation sweep (Sections 3.2-3.3, the handle's scheme and
 * theta) produced when the trajectory was recorded, held fixed: the sweep's
 * decisions and random numbers are frozen and so is its effect.  With
 * SDPD_SCHEME_NONE every D_k is zero and the map is Velocity Verlet alone.
 * The parameters differentiated are theta = (h, c_rho, C_K); kB, m and the
 * box are fixed.  Pair derivatives use the density gradient of Eq.
 * (gradient-rho) and dW/dh, dF/dh of the chosen kernel.  Cotangent and
 * increment arrays are device float64 in particle-id order: [N][3] for q
 * and p, [N] for eps.
 * ------------------------------------------------------------------------- */

/* Bytes of the tape for nsteps steps with a checkpoint every `every` steps:
 * ((ceil(nsteps/every) + max(1, min(every, nsteps))) * 56
 *  + max(1, nsteps) * 32 + 160) * N bytes plus a few KiB.
 * 0 for bad arguments (nsteps < 0, every < 1). */
size_t sdpd_tape_bytes(const sdpd_t* s, int64_t nsteps, int64_t every);

/* Runs nsteps full steps from the loaded state (Velocity Verlet, then the
 * sweep whenever sdpd_step would run one, random numbers keyed by seed) and
 * records on `tape` (device memory of at least sdpd_tape_bytes(s, nsteps,
 * every) bytes, 256-byte aligned, owned by the caller and kept unchanged
 * until the matching sdpd_vv_adjoint / sdpd_vv_replay calls are done) the
 * increments D_k of every step and the state at every `every`-th step and
 * at the end.  Each step's result is stored as before + D_k, which makes the
 * recorded trajectory the frozen map itself (it differs from sdpd_step's by
 * rounding only).  Leaves the handle at the final state; asynchronous.
 * Errors: SDPD_ERR_INVALID_ARG, SDPD_ERR_NO_STATE, SDPD_ERR_NO_WORKSPACE,
 * SDPD_ERR_CUDA. */
int sdpd_vv_record(sdpd_t* s, double dt, int64_t nsteps, int64_t every, uint64_t seed, void* tape,
                   size_t tape_bytes);

/* Reverse pass of the trajectory last recorded on this handle (`tape` and
 * `tape_bytes` as given to sdpd_vv_record).  Given the cotangents gq, gp,
 * geps of the final state (device; NULL = zero), writes those of the initial
 * state to gq0, gp0, geps0 (device) and of theta = (h, c_rho, C_K) to
 * gtheta[3] (host).  Positions between checkpoints are recomputed from the
 * tape (Verlet plus the stored increments), bit-identical to the recorded
 * run, so the result does not depend on `every`.  Uses the handle's
 * workspace and leaves the handle at the recorded final state again.
 * Synchronising; returns the sticky device status.  May be called again
 * with other cotangents.  Errors: SDPD_ERR_INVALID_ARG (no matching
 * record), SDPD_ERR_CAPACITY, SDPD_ERR_CUDA. */
int sdpd_vv_adjoint(sdpd_t* s, void* tape, size_t tape_bytes, const double* gq, const double* gp,
                    const double* geps, double* gq0, double* gp0, double* geps0, double gtheta[3]);

/* The frozen map of the last record, evaluated from the currently loaded
 * state: nsteps Velocity Verlet steps, each followed by the recorded
 * increments (no sweep runs).  From the recorded initial state it retraces
 * the recording bit for bit; from another state it is the map that
 * sdpd_vv_adjoint differentiates.  Asynchronous.  Errors:
 * SDPD_ERR_INVALID_ARG (no matching record), SDPD_ERR_NO_STATE. */
int sdpd_vv_replay(sdpd_t* s, const void* tape, size_t tape_bytes);

/* Copies the recorded increments of step `step` (0 <= step < nsteps):
 * momenta to dp [N][3] and energies to deps [N] (device, id order).
 * Asynchronous.  Errors: SDPD_ERR_INVALID_ARG. */
int sdpd_tape_increments(sdpd_t* s, const void* tape, size_t tape_bytes, int64_t step, double* dp, double* deps);

/* Virial pressure of the current state at its own energies,
 * P = (1/3V) [sum_i |p_i|^2/m + sum_{i<j} r_ij . F_ij] with the pair forces
 * of Eq. (cons-forces), into *value (host).  With gq, gp, geps (device, all
 * three or none) and gtheta (host) also its gradient with respect to q, p,
 * eps and theta = (h, c_rho, C_K) at fixed energies.  Synchronising; the
 * state is not changed.  Errors: SDPD_ERR_INVALID_ARG, SDPD_ERR_NO_STATE,
 * SDPD_ERR_CUDA. */
int sdpd_virial(sdpd_t* s, double* value, double* gq, double* gp, double* geps, double gtheta[3]);

/* Fused multiply-add throughput of the current device, measured -- the paper
 * has no counterpart; this is the denominator of the arithmetic rooflines of
 * the pair passes.  precision SDPD_MIXED: float32 FMA, SDPD_FP64: float64
 * FMA.  Runs 8 blocks of 256 threads per SM, each thread 8 independent FMA
 * chains, on `stream` (a cudaStream_t, NULL = legacy default stream), times
 * it with CUDA events after one warm-up launch and writes the achieved
 * FLOP/s (2 per FMA) to *flops.  Synchronising; allocates nothing.
 * Errors: SDPD_ERR_INVALID_ARG, SDPD_ERR_CUDA. */
int sdpd_fma_peak(int precision, void* stream, double* flops);

/* Density pass that allocates nothing -- the paper has no counterpart; this
 * is a service for callers that cannot allocate device memory themselves:
 * for example a plug-in that is handed raw device buffers by a host
 * application which owns every allocation on the device, or a code path
 * whose device-memory footprint has to be fixed before it runs.  Such a
 * caller cannot create the workspace that sdpd_bind_workspace expects.
 *
 * Computes rho_i = sum_j m W(r_ij) over j = 1..N (self term included) in
 * float64 for N particles at positions q[N][3] (device, float64; each
 * coordinate is wrapped periodically into [0, box) first, as sdpd_set_state
 * does) into rho[N] (device, float64), with the kernel
 * SDPD_KERNEL_CUBIC or SDPD_KERNEL_LUCY and the same neighbour rule as the
 * rest of the library (cells of side >= h, minimum image, r^2 < h^2).
 * Asynchronous on stream (a cudaStream_t, NULL = legacy default stream).
 *
 * The working memory (cell counts, cell starts, binned order: 1.25 MiB) is
 * one static array inside the library, held by every device that loads the
 * library until the process exits.  Limits: N <= 65536 and at most 65536
 * cells (box[d] / h, rounded down to an even number, multiplied over the
 * axes); larger inputs return SDPD_ERR_CAPACITY before any device work.
 * The first call on a device looks up the device address of that array
 * (one-time set-up, per device); make that first call before any stream
 * capture.  Every call reuses the same array and clears what must start at
 * zero; calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.  The function
 * calls no allocator.
 * Errors: SDPD_ERR_INVALID_ARG, SDPD_ERR_BOX_TOO_SMALL, SDPD_ERR_CAPACITY,
 * SDPD_ERR_CUDA. */
int sdpd_density_static(int64_t N, const double box[3], double m, double h, int kernel, const double* q,
                        double* rho, void* stream);

/* Static text for a status code. */
const char* sdpd_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* SDPD_H */
