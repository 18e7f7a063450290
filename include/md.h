/*
 * md.h -- C ABI of the GB300 (sm_103a) molecular-dynamics library.
 *
 * The library advances N classical particles in a cubic periodic box under a
 * truncated (and by default shifted) 12-6 Lennard-Jones pair potential, either
 * monatomic or as the Kob-Andersen A/B mixture, with the NVE velocity-Verlet
 * integrator.  This is the MD step of Colberg & Hoefling (arXiv:0912.3824):
 *   - Sec. 2.2: velocity Verlet, one thread per particle; cell binning by a
 *     parallel sort; a fixed-size Verlet neighbour list with a skin, rebuilt
 *     when the maximum particle displacement demands it; the force loop over
 *     the list; parallel reductions (maximum displacement, potential energy,
 *     temperature, centre-of-mass velocity, virial tensor); a periodic
 *     space-filling-curve reorder of the particles in memory;
 *   - Sec. 2.4: double-single arithmetic (a pair of floats, about 44 bits)
 *     for the velocity-Verlet update and for the summation of force
 *     contributions, while the pair forces themselves stay single precision;
 *   - Sec. 3: the 12-6 potential cut at r_c; Sec. 5: the Kob-Andersen
 *     parameters (sigma_AA=1, sigma_BB=0.88, sigma_AB=0.8, eps_AA=1,
 *     eps_BB=0.5, eps_AB=1.5, equal masses).
 * Several independent systems ("replicas", each with its own N and box) can
 * be advanced together by one handle; they share the potential and dt.
 *
 * Units are reduced Lennard-Jones units (sigma_AA, eps_AA, m).
 *
 * Conventions for every call:
 *   - Return value: MD_OK (0) or one of the MD_E_* codes below; the message of
 *     the last failure is available from md_last_error().
 *   - Host arrays passed in are owned by the caller and only read during the
 *     call (they are copied).  Host arrays passed out must be allocated by the
 *     caller with the stated size.
 *   - Per-particle host arrays are in the ORIGINAL particle order (the order
 *     given to md_create), replicas concatenated, whatever order the library
 *     keeps internally.  Vectors are [n][3] row-major float64.
 *   - Device memory: the library allocates no device memory.  The caller
 *     provides one workspace of md_workspace_size() bytes, 256-byte aligned,
 *     which must stay valid until md_destroy().  The library keeps
 *     pinned host staging buffers of its own.
 *   - All device work is issued on the CUDA stream given to md_create()
 *     (a cudaStream_t cast to void*; NULL = legacy default stream).
 *     md_step() returns without waiting for the GPU; the calls that return
 *     data (md_compute_forces, md_observables, md_get_state,
 *     md_get_neighbours, md_info, md_sync) wait for the stream.
 *   - Device-side failures (a neighbour list longer than the cap
 *     neigh_capacity_max, a non-finite value, a particle moving more than a
 *     quarter box in one step, an exhausted step-loop bound) stop the step
 *     loop at the end of the offending step, leave the positions at that
 *     step, and are reported by the next md_sync / md_observables / md_step.
 *     A list longer than the current capacity but within the cap is not a
 *     failure: the capacity grows on the device and the build is redone.
 */
#ifndef MD_GB300_H
#define MD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MD_OK           0
#define MD_E_INVAL      1  /* bad argument (sizes, box too small for the cutoff, dt <= 0 ...) */
#define MD_E_NOMEM      2  /* workspace smaller than md_workspace_size()                     */
#define MD_E_CUDA       3  /* a CUDA runtime call failed                                      */
#define MD_E_NONFINITE  4  /* a position became NaN or infinite                               */
#define MD_E_UNSTABLE   5  /* a particle moved more than a quarter box length in one step     */
#define MD_E_TIMEOUT    6  /* the device-side step loop exceeded its iteration bound          */
#define MD_E_CAPACITY   7  /* a neighbour list needed more than neigh_capacity_max entries    */
#define MD_E_BOUNDS     8  /* only in a library built with MD_CHECK_BOUNDS: a kernel index
                              left its array (the access was redirected to a valid one)     */

/* precision modes (Sec. 2.4) */
#define MD_PREC_FP64  0    /* everything in IEEE double                                        */
#define MD_PREC_MIXED 1    /* FP32 pair forces; double-single positions, velocities and
                              integration; compensated force summation; FP64 reductions   */
#define MD_PREC_FP32  2    /* everything in single precision (the paper's comparator)         */

typedef struct {
    int32_t n_species;        /* 1 or 2                                                        */
    int32_t shift;            /* 1 = truncated and shifted (V(r_c) = 0), 0 = truncated only    */
    double  eps[2][2];        /* epsilon_ab (symmetric)                                         */
    double  sigma[2][2];      /* sigma_ab (symmetric)                                           */
    double  rcut[2][2];       /* absolute cutoff r_c,ab (Kob-Andersen: 2.5 sigma_ab)            */
    double  mass[2];          /* mass per species                                               */
    double  dt;               /* time step, > 0                                                 */
    double  skin;             /* neighbour-list skin, >= 0 (default 0.3)                        */
    int32_t precision;        /* MD_PREC_*                                                      */
    int32_t neigh_capacity;   /* starting list entries per particle (rounded up to a multiple of
                                 8); 0 = derived from the density.  The list of Sec. 2.2 has a
                                 fixed size per particle; when a build finds a longer list the
                                 library raises the size on the device (to 1.25 times the
                                 longest list, rounded up to 8, at most neigh_capacity_max) and
                                 redoes the build, within the same md_step                     */
    int32_t sample_interval;  /* record observables every this many steps (>= 1)                */
    int32_t obs_capacity;     /* ring-buffer samples kept on the device (0 = 4096); also the
                                 number of newest steps the per-step potential-energy series
                                 keeps (md_epot_series)                                         */
    int32_t threads_per_particle; /* force-kernel lanes per particle: 0 = automatic (2 for MIXED
                                     and FP32, 4 for FP64), else a power of two in 1..32 (1..8
                                     with smooth_h > 0)                                          */
    int32_t use_graph;        /* 1 = md_step runs as one CUDA graph with the rebuild branch and
                                 the step loop decided on the device (default); 0 = plain
                                 stream launches, for debugging and per-kernel timing          */
    int32_t reorder;          /* cell order in memory: 1 = Morton curve (default), 2 = Hilbert
                                 curve (the paper's reorder, Sec. 2.2), 0 = x-fastest           */
    int32_t step_form;        /* blocks of the step kernel: 0 = automatic (form 2 when MIXED or
                                 FP32 at 1 or 2 lanes per particle needs more blocks than the
                                 GPU holds at once, else form 1), 1 = one block per chunk of
                                 particles, 2 = only the resident blocks, each sweeping a run of
                                 neighbouring chunks (MIXED or FP32 at 1 or 2 lanes only);
                                 the results are the same either way, bit for bit            */
    double  smooth_h;         /* h >= 0 of the smoothing of Sec. 4: every pair potential is
                                 multiplied by g(x) = x^4 / (1 + x^4), x = (r - r_c,ab) /
                                 (h sigma_ab), which makes it and its first two derivatives
                                 vanish at r_c; 0 = no smoothing (the paper uses h = 0.005).
                                 Not supported by md_forces_noalloc.                           */
    int32_t check_interval;   /* MD steps between the rebuild checks of md_step's CUDA graph:
                                 1, 2, 4, 8 or 16; 0 = automatic (4 below 262,144 particles, 1
                                 from there).  Between checks the rebuild decision adds a bound
                                 on how far particles can still move (speed and acceleration
                                 over the unchecked steps), so a longer interval rebuilds
                                 earlier; a check costs one conditional graph node           */
    int32_t neigh_capacity_max; /* cap on the list entries per particle (rounded up to 8): the
                                 workspace holds this many; 0 = twice the starting capacity.
                                 Only a list longer than the cap is an error (MD_E_CAPACITY);
                                 neigh_capacity_max = neigh_capacity keeps the size fixed     */
    int32_t step_budget;      /* 0 = automatic.  > 0: md_step's device loop stops with
                                 MD_E_TIMEOUT after this many step-kernel executions (its
                                 iteration bound; automatic = nsteps + 64), so the bounded-
                                 loop path can be exercised                                     */
    int32_t build_form;       /* neighbour build: 0 = automatic (one warp per cell when there
                                 are at least 8 cells per SM and at most 32 particles per cell
                                 on average, else one block per cell), 1 = one warp per cell,
                                 2 = one block per cell; the lists are the same either way     */
} md_params;

/* one sample of the reductions of Sec. 2.2, per replica */
typedef struct {
    int64_t step;             /* MD step index of the sample                                    */
    double  e_pot;            /* sum over pairs of V(r_ij)                                      */
    double  e_kin;            /* sum of m v^2 / 2                                               */
    double  virial;           /* sum over pairs of r_ij . F_ij                                  */
    double  w[6];             /* virial tensor xx, yy, zz, xy, xz, yz                           */
    double  p[3];             /* total momentum                                                 */
    double  max_disp;         /* largest displacement of the sample's positions from those of
                                 the last list build (over all replicas)                       */
    int64_t rebuilds;         /* neighbour-list builds so far (all replicas)                    */
} md_obs;

typedef struct {
    int64_t n_total;          /* particles over all replicas                                    */
    int32_t n_replicas;
    int32_t neigh_capacity;   /* list entries per particle in use (grows up to the cap)          */
    int32_t threads_per_particle;
    int32_t cells_per_edge;   /* of replica 0 (1 when the box holds fewer than 3 cells)         */
    int64_t step;             /* MD steps done since md_create                                  */
    int64_t rebuilds;         /* neighbour-list builds since md_create                          */
    int64_t kernel_launches;  /* library kernels executed on the device since md_create         */
    int32_t max_neighbours;   /* largest list length at the last build                          */
    int32_t status;           /* pending device status (MD_OK if none)                          */
    double  step_ms;          /* with use_graph = 0: summed CUDA-event time of the step kernel
                                 (pair forces + velocity-Verlet update, one launch per step)   */
    int64_t step_launches;    /* with use_graph = 0: step-kernel launches timed                 */
    double  rebuild_ms;       /* with use_graph = 0: summed time of the rebuild chains (sort,
                                 list build) launched when a check point asked for one         */
    int64_t rebuild_checks;   /* with use_graph = 0: rebuild chains launched                    */
    double  step_device_ms;   /* any mode: summed device duration of the step-kernel launches
                                 that advanced a step (first block start to last block end,
                                 read from the GPU's global timer)                              */
    int64_t step_device_launches; /* launches summed into step_device_ms (one per MD step)      */
    int32_t check_interval;   /* MD steps between rebuild checks, as resolved                   */
    int32_t neigh_capacity_max; /* the cap on neigh_capacity, as resolved                       */
    int64_t regrows;          /* list builds redone with a larger capacity since md_create      */
    int32_t build_form;       /* neighbour build in use: 1 = one warp per cell, 2 = one block   */
    int32_t step_form;        /* step-kernel blocks in use: 1 = one per chunk, 2 = resident
                                 blocks sweeping runs of chunks                                 */
} md_info_t;

typedef struct md_handle md_handle;

/* Fill p with the monatomic LJ defaults: eps = sigma = m = 1, r_c = 2.5,
 * shifted, dt = 0.005, skin = 0.3, MD_PREC_MIXED, sample_interval = 100,
 * use_graph = 1, reorder = 1.  Returns MD_OK, or MD_E_INVAL if p is NULL. */
int md_params_default(md_params *p);

/* Host-only: the order of the cells of replica 0 in memory.  rank[lin] (for
 * lin = x + nc (y + nc z), caller array of nc^3 entries, may be NULL) is the
 * position of cell (x, y, z) along the chosen curve; *cells_per_edge = nc.
 * Same argument checks as md_workspace_size. */
int md_cell_order(const md_params *p, int32_t n_replicas, const int64_t *n_per_replica, const double *box,
                  int32_t *rank, int32_t *cells_per_edge);

/* Device workspace needed for n_replicas systems with n_per_replica[r]
 * particles in cubic boxes of edge box[r].  Writes *bytes. */
int md_workspace_size(const md_params *p, int32_t n_replicas,
                      const int64_t *n_per_replica, const double *box, size_t *bytes);

/* Create a handle: the problem statement of Sec. 2.2 (N particles with
 * species, a periodic box, the pair potential of Sec. 3 with the parameters
 * in *p, the time step).  species[n_total] in {0, n_species-1} (checked on
 * the host: MD_E_INVAL otherwise); pos[n_total][3] (any real coordinates:
 * they are wrapped into [0, box)), vel[n_total][3], image[n_total][3] (may
 * be NULL = zeros).  Uploads the state, bins the particles and orders them
 * along the cell curve, builds the neighbour lists (growing the capacity up
 * to its cap if needed), evaluates the forces and records the step-0 sample.
 * Each box must exceed twice the largest cutoff plus skin.  workspace:
 * device memory of at least md_workspace_size() bytes, owned by the caller.
 * cuda_stream: a cudaStream_t or NULL.  Errors: MD_E_INVAL, MD_E_NOMEM,
 * MD_E_CUDA, MD_E_CAPACITY (a list longer than the cap at the first build).
 * On failure *h is NULL and nothing is left allocated. */
int md_create(md_handle **h, const md_params *p, int32_t n_replicas,
              const int64_t *n_per_replica, const double *box,
              const int32_t *species, const double *pos, const double *vel,
              const int32_t *image, void *workspace, size_t workspace_bytes,
              void *cuda_stream);

/* Advance every replica by nsteps >= 1 velocity-Verlet steps (Sec. 2.2),
 * rebuilding the neighbour lists whenever some particle has moved more than
 * skin/2 since the last build.  Asynchronous on the handle's stream. */
int md_step(md_handle *h, int64_t nsteps);

/* Scale all velocities of replica r by sqrt(T_target[r] / T_r), with
 * T_r = 2 E_kin,r / (3 N_r - 3)  (the exact rescale of Sec. 2.3). */
int md_rescale_velocities(md_handle *h, const double *T_target);

/* Andersen heat bath (Sec. 2.3): every particle of replica r receives a fresh
 * Maxwell-Boltzmann velocity at T_target[r] (host array [n_replicas], >= 0);
 * then the mass-weighted mean velocity of each replica is removed and its
 * velocities are rescaled so that 2 E_kin / (3 N_r - 3) = T_target[r] exactly
 * (all zero when N_r < 2 or T_target[r] = 0).  The random numbers are the
 * rand48 sequence (x_{k+1} = 0x5DEECE66D x_k + 0xB mod 2^48, seeded as
 * srand48(seed); deviate k = x_{k+1} / 2^48) shared out by leapfrogging:
 * particle i (original index over all replicas, of n_total) uses deviates
 * (4 event + j) n_total + i, j = 0..3, for three Box-Muller normals.  So a
 * collision is reproducible from (seed, event) and independent of the
 * particles' order in memory.  Call it every 1/(mu dt) steps with event =
 * 0, 1, 2, ... for a heat-bath collision rate mu.  Asynchronous on the
 * handle's stream.  MD_E_INVAL for a negative or non-finite target or a
 * negative event index.                                                       */
int md_andersen(md_handle *h, const double *T_target, uint64_t seed, int64_t event);

/* The force evaluation of Sec. 2.2 on its own: pair forces of the potential of
 * Sec. 3 (Kob-Andersen parameters of Sec. 5) over freshly built lists at the
 * current positions.  Outputs: the force on every particle f[n_total][3]
 * (may be NULL), the per-particle potential energy e[n_total] = half of each
 * pair energy (may be NULL), and per-replica totals[n_replicas] (may be NULL;
 * e_pot, virial, w are the force-kernel reductions, e_kin and p those of the
 * current velocities; max_disp is 0, the lists having just been rebuilt).
 * The state is not advanced.  Waits for the stream; returns any pending device status. */
int md_compute_forces(md_handle *h, double *f, double *e, md_obs *totals);

/* The reductions of Sec. 2.2 (potential energy, virial tensor, kinetic
 * energy, centre-of-mass momentum, maximum displacement), recorded on the
 * device every sample_interval steps.  Copies out the samples recorded since
 * the previous call, oldest first, as [sample][replica] records into the
 * caller's out[max_samples][n_replicas]; at most max_samples samples (the
 * newest are kept when more were recorded than the ring holds).  *n_samples
 * receives the number written.  Waits for the stream; returns any pending
 * device status. */
int md_observables(md_handle *h, md_obs *out, int32_t max_samples, int32_t *n_samples);

/* The potential energy of every replica at every MD step: Sec. 2.2 names the
 * potential-energy sum, with the maximum displacement, among the reductions
 * needed every step, so the step kernel sums the pair energies in the force
 * loop and reduces them (per block, then per replica in a fixed order, in
 * FP64) at every step; at sample steps the value equals the e_pot of the
 * md_observables record bit for bit.  The device keeps the newest
 * obs_capacity steps.  Copies out the steps recorded since the previous call,
 * oldest first (at most max_steps, the newest kept): steps[n] (the MD step of
 * each value; step 0 is the state given to md_create) and e_pot[n][n_replicas],
 * caller arrays.  *n_steps receives n.  Waits for the stream; returns any
 * pending device status.  MD_E_INVAL for a null pointer. */
int md_epot_series(md_handle *h, int64_t *steps, double *e_pot, int32_t max_steps, int32_t *n_steps);

/* Current positions (wrapped into [0, box)), velocities and image counters,
 * in the original order although the library keeps the particles sorted
 * along the cell curve (Sec. 2.2 reorder).  Caller arrays pos[n_total][3],
 * vel[n_total][3], image[n_total][3]; any may be NULL.  MIXED state is
 * returned as the double value of each double-single pair (Sec. 2.4).
 * Waits for the stream. */
int md_get_state(md_handle *h, double *pos, double *vel, int32_t *image);

/* Replace positions, velocities and images (original order, layouts as in
 * md_get_state; image may be NULL = zeros), then re-bin, rebuild the lists
 * (Sec. 2.2) and evaluate the forces; species stay those of md_create.
 * Non-finite values are not rejected here: the next md_step reports them as
 * MD_E_NONFINITE.  Asynchronous: the host arrays are staged through pinned
 * memory before the call returns. */
int md_set_state(md_handle *h, const double *pos, const double *vel, const int32_t *image);

/* Current neighbour lists, for inspection: counts[n_total] and
 * lists[n_total][kmax] of partner indices (original order; unused entries -1;
 * lists may be NULL).  Waits for the stream. */
int md_get_neighbours(md_handle *h, int32_t *counts, int32_t *lists, int32_t kmax);

/* Counters and settings of the handle.  Waits for the stream. */
int md_info(md_handle *h, md_info_t *out);

/* Wait for the stream and return the pending device status (MD_OK if none):
 * the failures that the device detects during the loop of Sec. 2.2 (list
 * overflow past the cap, non-finite or runaway positions, an exhausted loop
 * bound).  A status is reported once; the positions stay at the step where
 * it arose. */
int md_sync(md_handle *h);

/* Release the handle (not the workspace).  Waits for the stream. */
int md_destroy(md_handle *h);

/* Message of the last failure on h (never NULL).  With h = NULL: the message
 * of the calling thread's last failed md_forces_noalloc call, the one call
 * that takes no handle ("" after a success). */
const char *md_last_error(const md_handle *h);

/* Fixed name of a status code. */
const char *md_status_string(int code);

/* Largest particle count accepted by md_forces_noalloc(). */
#define MD_NOALLOC_MAX_N 1048576

/* Forces, per-particle energies and energy / virial totals of one periodic
 * configuration, computed without allocating any device memory.
 *
 * The paper has no counterpart to this call.  It exists for callers that may
 * not allocate device memory when they need forces: an out-of-memory handler
 * that must still evaluate a configuration after an allocation has failed, an
 * application whose memory manager owns the whole device and forbids
 * cudaMalloc / cudaFree outside its own pool (cudaFree also synchronises the
 * device), or code certified to allocate nothing after start-up.  It needs no
 * handle and no workspace.
 *
 * All arrays are DEVICE memory owned by the caller: species[n] (int32, in
 * [0, n_species)), pos[n][3] (float64, any real coordinates), force[n][3] (float64, out),
 * energy[n] (float64, out: half of each pair energy; may be NULL), totals[8]
 * (float64, out: E_pot, virial, W_xx, W_yy, W_zz, W_xy, W_xz, W_yz).  From *p
 * only the potential (n_species, eps, sigma, rcut, shift) and the precision
 * are used: MD_PREC_FP64 evaluates pairs in double, the other modes in single
 * precision on separations formed in double.  The sum runs directly over all
 * pairs (O(n^2) work), in a cubic box of edge `box` > 2 r_c,max.
 *
 * Scratch: a fixed 512 KiB area inside this library's device memory (the
 * per-block partial sums and a counter), present on every GPU that loads the
 * library until the process exits.  The first call on each device, with that
 * device current, looks up the area's address; make that first call before
 * any stream capture.  Every call uses the same area and resets the counter
 * itself; calls that overlap on the GPU (different streams, or unordered
 * calls from several threads) race on the area and give wrong totals.
 *
 * The scratch address is looked up once per device and kept: a device reset
 * (cudaDeviceReset) after the first call on that device is not supported.
 *
 * The species array is device memory, so the host cannot check it without a
 * copy: a code outside [0, n_species) is treated as the nearest valid species
 * for the pair parameters, the force and energy of that particle are written
 * as NaN, and all eight totals are NaN, so that bad input never passes as a
 * result.
 *
 * Cost: O(n^2) pair tests with the minimum image in FP64, in every precision
 * mode, so the time per call grows as n^2.  Measured on a GB300 (Kob-Andersen
 * mixture, density 1.2): 10 ms at n = 16,384, 154 ms at 65,536, 533 ms at
 * 131,072 (0.031 to 0.039 ns per ordered pair), so about 35 to 40 s at
 * n = MD_NOALLOC_MAX_N.
 *
 * Returns MD_OK, MD_E_INVAL (null pointer, n < 2, n > MD_NOALLOC_MAX_N, box
 * too small, bad parameters; the reason is in md_last_error(NULL)) or
 * MD_E_CUDA.  Asynchronous on cuda_stream (a cudaStream_t, NULL = legacy
 * default stream). */
int md_forces_noalloc(const md_params *p, int64_t n, double box, const int32_t *species,
                      const double *pos, double *force, double *energy, double *totals,
                      void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Time-correlation functions by the blocking scheme of Sec. 2.5.
 *
 * A correlator samples the state of one handle each time md_corr_sample is
 * called (the caller advances the handle by a fixed number of MD steps, the
 * sampling interval, between calls; sample index m = 0, 1, 2, ...).  Block n
 * (n = 0 .. k-1) holds at most l samples spaced l^n samples apart (it takes
 * the samples whose index is a multiple of l^n).  When a block becomes full
 * its first entry is correlated with each of the other l - 1 entries (lags
 * j l^n samples, j = 1 .. l-1) and then dropped.  Device memory: k l
 * snapshots of the unwrapped positions (FP64, 24 bytes per particle each).
 *
 * Correlated quantities, per species (all replicas pooled, an ensemble
 * average over independent systems), for a particle displacement d over the
 * lag: the mean-square displacement |d|^2 and the self intermediate
 * scattering function F_s = (1/n_q) sum_q cos(q . d) over the given
 * wavevectors (Sec. 5: F_s(q, t) = <rho_q(t) rho_-q(0)>, orientation
 * averaged; the paper uses |q| = 7.25 for the Kob-Andersen mixture).
 * |d|^2 is summed in FP64; the cosine is evaluated in FP32.
 * ------------------------------------------------------------------------- */
typedef struct md_corr md_corr;

/* Device workspace in bytes for a correlator over all particles of h:
 * 1 <= k, 2 <= l <= 32, 1 <= n_q <= 64, l^k < 9e15.  Host-only. */
int md_corr_workspace_size(const md_handle *h, int32_t k, int32_t l, int32_t n_q, size_t *bytes);

/* Create a correlator on h.  q: host array [n_q][3] of wavevectors (copied).
 * workspace: device memory, 256-byte aligned, caller-owned, at least
 * md_corr_workspace_size bytes, outliving the correlator.  Destroy the
 * correlator before its handle.  MD_E_INVAL / MD_E_NOMEM / MD_E_CUDA. */
int md_corr_create(md_corr **c, md_handle *h, int32_t k, int32_t l, int32_t n_q, const double *q,
                   void *workspace, size_t workspace_bytes);

/* Take the handle's current state as the next sample; launches the snapshot
 * and any correlation the insertion triggers, asynchronously on the handle's
 * stream. */
int md_corr_sample(md_corr *c);

/* Results so far, each array (host) of k (l-1) entries in the order (block n,
 * lag j): lags in samples (j l^n), number of time origins correlated, and per
 * species (second index 0 = A, 1 = B; arrays of 2 k (l-1)) the mean-square
 * displacement and F_s averaged over origins and particles; NaN where no
 * origin has been correlated yet or the species is absent.  Any pointer may
 * be NULL.  Synchronises the handle's stream. */
int md_corr_result(md_corr *c, int64_t *lags, double *msd, double *fs, int64_t *origins);

int md_corr_destroy(md_corr *c);

#ifdef __cplusplus
}
#endif

#endif /* MD_GB300_H */
