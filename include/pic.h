/*
 * pic.h -- C ABI of the GB300 implementation of the implicit 2D3V
 * particle-in-cell step of Petrov & Davis, "Parallelization of an implicit
 * algorithm for multi-dimensional particle-in-cell simulations".
 *
 * What one step computes (Section 3.3, "the PIC cycle"):
 *   1. the field solver: Eq. 4 for E^{n+1} at the nodes from the implicit
 *      source moments S (9 components) and dj (3) deposited at the end of the
 *      previous step, then Eq. 5 for H at the cell centres (E on nodes, H at
 *      cell centres, Section 2 last paragraph and Fig. 1);
 *   2. the forces: E^{n+1/2} and B gathered at every particle with linear
 *      (area) weights inside its cell (Section 3.3, last paragraph);
 *   3. the pusher: the particle's momentum equation (Eq. 2a) inverted with
 *      the electric field factored out, one push per step (Section 1, 2);
 *   4. the moments: rho, S and dj of Eq. 3 accumulated on the nodes at the
 *      new positions (Section 3.3, step 1), for the next field solve.
 *
 * Units are normalised: c = eps0 = mu0 = 1, so B = H; charge in e, mass in
 * m_e, u = p / (m c).  Lengths and times in any consistent unit (c/omega_r,
 * 1/omega_r).
 *
 * Grid: nx x ny cells of dx x dy.  y is periodic.  Along x the box is periodic
 * (nxn = nx node columns) or closed by absorbing walls (nxn = nx + 1 node
 * columns; columns 0 and nx lie on the walls, and a plane wave may be injected
 * at x = 0).  Host-side node arrays are planar per component and node-major:
 * component c of node (i, j) is element c*ny*nxn + j*nxn + i.  Cell arrays
 * (H) likewise with nx columns.
 *
 * Conventions for every call:
 *   - return value: PIC_OK (0) or a negative PIC_ERR_* code; the message of the
 *     last error of the calling thread is returned by pic_last_error();
 *   - all host pointers are owned by the caller and only read/written during
 *     the call; the library owns all device memory of a handle;
 *   - work is queued on the CUDA stream given in pic_config.cuda_stream (NULL
 *     means the legacy default stream); calls that return data to the host
 *     synchronise that stream first.  Errors of queued kernels surface at the
 *     next call that synchronises.
 *   - a handle is used by one host thread at a time.
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#if defined(__GNUC__)
#define PIC_API __attribute__((visibility("default")))
#else
#define PIC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_ERR_ARG (-1)       /* invalid argument or configuration */
#define PIC_ERR_OOM (-2)       /* device or host allocation failed */
#define PIC_ERR_CUDA (-3)      /* a CUDA runtime call or kernel failed */
#define PIC_ERR_TIMEOUT (-4)   /* a bounded device wait gave up */
#define PIC_ERR_STATE (-5)     /* call not valid in the handle's state */
#define PIC_ERR_CAPACITY (-6)  /* particle capacity exceeded */

#define PIC_BC_PERIODIC 0
#define PIC_BC_ABSORBING 1

#define PIC_FIELD_LITERAL 0  /* Eqs. 4-5 as printed: explicit curls, per-node 3x3 solve */
#define PIC_FIELD_CN 1       /* time-centred curls, iterative stencil solve: FP64 residual and
                                refinement around an FP32 BiCGSTAB (spectral preconditioner on
                                periodic power-of-two grids, block-Jacobi otherwise); with
                                absorbing walls the wall nodes are vacuum, their x rows take the
                                one-sided curl of H and their y, z rows a time-centred first-order
                                Mur condition (the laser enters through the x = 0 wall) */

/* Preconditioner of the CN solve's FP32 inner iterations.  JACOBI: the inverse
 * of each node's 3x3 diagonal block (any grid).  FFT: the spectral inverse of
 * the operator with the grid mean of S (periodic x, nx and ny powers of two),
 * or, in a box with walls (ny a power of two), the line preconditioner: FFT
 * along y, then per y-mode the exact block-tridiagonal solve along x with the
 * column means of S and the walls' Mur rows (the exact inverse in vacuum).
 * AUTO: the spectral preconditioner where it applies, else block-Jacobi (in
 * boxes with walls the line preconditioner needs fewer iterations but, per
 * application, about seven times the time of a block-Jacobi one). */
#define PIC_CN_PRECOND_AUTO 0
#define PIC_CN_PRECOND_JACOBI 1
#define PIC_CN_PRECOND_FFT 2

#define PIC_FP64 0
#define PIC_FP32 1

/* Deposit of the moments (Eq. 3).  ATOMIC: floating-point atomic sums, whose
 * last bits depend on the order the GPU adds them in.  DETERMINISTIC: every
 * corner contribution is rounded once to a 64-bit fixed-point number (scale
 * 2^-e per moment class rho / S / dj, e chosen from the weights loaded so
 * that no sum can overflow) and summed with integer additions, so the moments,
 * and everything computed from them, are bitwise the same from run to run.
 * The rounding adds at most 2^-(e+1) per contribution, about 1e-19 of the
 * class's total |weight| bound; FP32 partial sums of the FP32 form are formed
 * in a fixed order before the conversion. */
#define PIC_DEPOSIT_ATOMIC 0
#define PIC_DEPOSIT_DETERMINISTIC 1

/* Particle shape W for the gather and the deposit (Section 3.3, last
 * paragraph: polynomial shapes up to fourth order; the paper keeps linear).
 * LINEAR: the paper's area weighting over the particle's cell (4 nodes).
 * QUADRATIC, CUBIC, QUARTIC: the centred B-spline of degree n = 2, 3, 4 over
 * the (n + 1) x (n + 1) nodes nearest the particle (per axis node k at
 * distance x from the particle weighs B_n(x); e.g. n = 2: 3/4 - x^2 for
 * |x| <= 1/2, (3/2 - |x|)^2 / 2 for 1/2 <= |x| <= 3/2).  Along y and a periodic
 * x the nodes wrap; along a walled x a node beyond a wall gives its weight to
 * the wall node.  Not with pic_ionize or pic_batch_step. */
#define PIC_SHAPE_LINEAR 1
#define PIC_SHAPE_QUADRATIC 2
#define PIC_SHAPE_CUBIC 3
#define PIC_SHAPE_QUARTIC 4

#define PIC_MAX_SPECIES 8
#define PIC_MAX_TILE_CELLS 1024  /* tile_nx * tile_ny limit (each step sorts every tile by cell) */

typedef struct pic_t pic_t;

/* Run description (Section 3.2, "Initialization": grid, particles, fields = 0). */
typedef struct pic_config {
    int32_t nx, ny;            /* cells along x and y, >= 2 each */
    double dx, dy, dt;         /* cell size and time step, > 0 */
    int32_t bc_x;              /* PIC_BC_PERIODIC or PIC_BC_ABSORBING (y is always periodic) */
    int32_t field_mode;        /* PIC_FIELD_LITERAL or PIC_FIELD_CN (either bc_x) */
    int32_t precision;         /* PIC_FP64 or PIC_FP32 particle/field arithmetic */
    int32_t deposit;           /* PIC_DEPOSIT_ATOMIC or PIC_DEPOSIT_DETERMINISTIC */
    int32_t n_species;         /* 1 .. PIC_MAX_SPECIES */
    int32_t tile_nx, tile_ny;  /* particle-sort tile in cells (0 = 16); at most PIC_MAX_TILE_CELLS cells */
    double q[PIC_MAX_SPECIES]; /* species charge (units of e) */
    double m[PIC_MAX_SPECIES]; /* species mass (units of m_e), > 0 */
    /* incident plane wave at x = 0 of a walled box: E_pol(0,t) =
     * a0 sin(omega t) exp(-2 ln2 (t - t0)^2 / tau^2) for t >= 0 (tau <= 0: no envelope) */
    double laser_a0, laser_omega, laser_tau, laser_t0;
    int32_t laser_pol;         /* 0: E along y, 1: E along z */
    int32_t cn_max_iter;       /* CN solver cap on FP32 inner iterations, all refinements (0 = 400) */
    double cn_tol;             /* CN target of the FP64 relative residual (0 = 1e-12 FP64, 1e-10 FP32) */
    void *cuda_stream;         /* cudaStream_t to queue work on, or NULL */
    int64_t capacity[PIC_MAX_SPECIES]; /* particle capacity per species (0 = grow on load) */
    int32_t shape;             /* PIC_SHAPE_LINEAR (or 0), _QUADRATIC, _CUBIC or _QUARTIC */
    int32_t cn_precond;        /* CN preconditioner: PIC_CN_PRECOND_AUTO (0), _JACOBI or _FFT */
} pic_config;

/* FP64 global reductions of the current state (diagnostics). */
typedef struct pic_diag {
    double kinetic;            /* sum w m (gamma - 1) */
    double field;              /* 1/2 sum E^2 dA (nodes) + 1/2 sum H^2 dA (cells) */
    double total;              /* kinetic + field */
    double charge_grid;        /* sum over nodes of deposited rho dA */
    double charge_particles;   /* sum q w */
    int64_t count;             /* live particles, all species */
    int64_t removed;           /* particles removed at walls since init */
    int64_t step;              /* steps taken since init */
    double cn_residual;        /* last CN solve: relative FP64 residual |b - A x| / |b| reached */
    int32_t cn_iterations;     /* last CN solve: FP32 BiCGSTAB iterations, all refinements */
    int32_t flags;             /* bit 0: a particle moved farther than one tile in a step */
    int32_t cn_refinements;    /* last CN solve: FP64 refinement steps (FP32 inner solves) */
    int32_t full_regroups;     /* steps since init whose per-tile regroup fell back to the full sort */
} pic_diag;

/* Create a handle: validates cfg, allocates the grid, zero fields (Section 3.2 (3)). */
PIC_API int pic_init(const pic_config *cfg, pic_t **out);

/* Free every device and host resource of the handle.  NULL is accepted. */
PIC_API int pic_destroy(pic_t *h);

/* Append n particles of one species (Section 3.2 (2)): host FP64 arrays of
 * global positions (x in [0, nx dx), y in [0, ny dy)), u = p/(m c) and weight
 * w (particles per unit length in z; the node density of one particle is
 * w / node area).  Positions outside the box give PIC_ERR_ARG and load
 * nothing.  The species is then regrouped by tile (stable), and the moments
 * are re-deposited with the current B. */
PIC_API int pic_load_particles(pic_t *h, int species, int64_t n, const double *x, const double *y,
                       const double *ux, const double *uy, const double *uz, const double *w);

/* FP64 arrays of one species' particles: n and the six arrays of
 * pic_load_particles. */
typedef struct pic_species_data {
    int64_t n;
    const double *x, *y, *ux, *uy, *uz, *w;
} pic_species_data;

/* Append data[s] to species s for s = 0 .. nspecies - 1 (Section 3.2 (2);
 * nspecies <= the handle's species; n = 0 leaves a species as it is), all or
 * nothing: the same checks and the same resulting state as
 * pic_load_particles species by species, but an invalid particle in any
 * species gives PIC_ERR_ARG (naming the species and the particle) and loads
 * nothing.  Arrays may be page-locked host memory (read in place over the
 * CPU-GPU link), device memory, or pageable host memory (staged).  When every
 * species that receives particles is empty, one species' regroup (and, when
 * they are all the handle's particles, its deposit at rest) runs while the
 * next species' arrays are still being read.  The caller keeps ownership of
 * data and the arrays; none is retained after the call returns.  Errors:
 * PIC_ERR_ARG (NULL handle, data or array, nspecies out of range, negative
 * n), PIC_ERR_CAPACITY (more than 2^30 particles in a species), PIC_ERR_OOM,
 * PIC_ERR_CUDA. */
PIC_API int pic_load_species(pic_t *h, int nspecies, const pic_species_data *data);

/* Prefetch a later pic_load_species (no counterpart in the paper: it moves
 * the next inputs across the CPU-GPU link while the GPU works on the current
 * ones).  Starts copying data[s], s = 0 .. nspecies - 1, into device memory
 * the handle owns, on a copy stream of its own, and returns without waiting
 * for the copy; up to two prefetched loads wait at a time.  The arrays may be
 * page-locked host memory or device memory (copied asynchronously) or
 * pageable host memory (staged by the driver); they must stay valid and
 * unchanged until the matching pic_load_prefetched returns.  The device copy
 * (6 x 8 bytes per particle per slot) is kept for the next prefetch and freed
 * with the handle.  Errors: PIC_ERR_ARG (NULL handle, data or array, nspecies
 * out of range, negative n), PIC_ERR_STATE (two loads wait already),
 * PIC_ERR_OOM, PIC_ERR_CUDA. */
PIC_API int pic_prefetch_species(pic_t *h, int nspecies, const pic_species_data *data);

/* Load the oldest prefetched arrays: the handle's stream waits on the GPU for
 * their copy, then exactly pic_load_species on the device copies (the same
 * checks, result and errors).  PIC_ERR_STATE if nothing is prefetched. */
PIC_API int pic_load_prefetched(pic_t *h);

/* Remove every particle of every species (fields are kept; the moments become
 * zero).  PIC_ERR_ARG for a NULL handle, PIC_ERR_CUDA. */
PIC_API int pic_clear_particles(pic_t *h);

/* Advance nsteps PIC cycles (Section 3.3: field solve, forces, push,
 * moments), nsteps >= 0.  Asynchronous on the handle's stream: the literal
 * field solve runs on a second stream of the handle beside the previous
 * step's particle sort, ordered by events and joined back, so work queued on
 * the handle's stream afterwards (and any synchronisation of it) comes after
 * all of the step.  PIC_ERR_ARG (NULL handle, negative nsteps); device errors
 * of earlier steps are reported here (PIC_ERR_STATE for a broken invariant in
 * the checks build, PIC_ERR_TIMEOUT for a bounded wait that gave up,
 * PIC_ERR_CUDA) or at the next synchronising call. */
PIC_API int pic_step(pic_t *h, int nsteps);

/* Wait for all queued work of the handle and report any device error
 * (PIC_ERR_CUDA, PIC_ERR_TIMEOUT, PIC_ERR_STATE). */
PIC_API int pic_sync(pic_t *h);

/* Moments of Eq. 3 deposited for the next field solve (Section 3.3, step 1),
 * divided by the node area
 * (dA = dx dy, dA/2 on a wall column): rho [ny*nxn], S9 [9][ny*nxn] with
 * S_rc at plane 3r + c (row r = component of the current, column c =
 * component of E), dj3 [3][ny*nxn].  NULL skips an output.  Caller-owned
 * host buffers; synchronises the stream.  PIC_ERR_ARG, PIC_ERR_CUDA. */
PIC_API int pic_moments(pic_t *h, double *rho, double *S9, double *dj3);

/* E^n at the nodes [3][ny*nxn] and the stored H at the cell centres
 * [3][ny*nx] (H^{n+1/2} in literal mode, H^n in CN mode; the staggering of
 * Section 2 and Fig. 1).  NULL skips.  Caller-owned host buffers;
 * synchronises the stream.  PIC_ERR_ARG, PIC_ERR_CUDA. */
PIC_API int pic_fields(pic_t *h, double *E3, double *H3);

/* Overwrite E and/or H (layouts of pic_fields; NULL keeps the current one);
 * B at the nodes and the moments are recomputed from the new H.  No
 * counterpart in the paper (its fields start at zero, Section 3.2); used to
 * resume a saved run and by tests.  PIC_ERR_ARG, PIC_ERR_CUDA. */
PIC_API int pic_set_fields(pic_t *h, const double *E3, const double *H3);

/* Checkpoint form of one species' particles (no counterpart in the paper),
 * in the library's order: the linear cell index j*nx + i, the in-cell
 * offsets (ox, oy) in [0, 1), u and w, exactly as stored (FP32 form: widened
 * exactly to FP64).  Caller-owned host arrays of pic_particle_count()
 * entries; NULL skips an output.  PIC_ERR_ARG (NULL handle, species out of
 * range), PIC_ERR_OOM, PIC_ERR_CUDA. */
PIC_API int pic_save_particles(pic_t *h, int species, int32_t *cell, double *ox, double *oy, double *ux,
                               double *uy, double *uz, double *w);

/* Append n particles given in checkpoint form (no counterpart in the paper;
 * the arrays of pic_save_particles, in host, page-locked or device memory,
 * read during the call only), with the checks,
 * order and regroup of pic_load_particles: a cell outside [0, nx*ny), an
 * offset outside [0, 1) or a value not finite gives PIC_ERR_ARG and loads
 * nothing.  A run saved with pic_save_particles and pic_fields (and its step
 * count) and restored with pic_restore_particles, pic_set_fields and
 * pic_set_step continues bitwise in the FP64 form with the deterministic
 * deposit (each corner contribution is rounded to fixed point on its own, so
 * the moments re-deposited at rest are exactly the ones the step deposited);
 * the FP32 form continues to its rounding (its push sums a warp's
 * contributions in FP32 before the fixed-point rounding). */
PIC_API int pic_restore_particles(pic_t *h, int species, int64_t n, const int32_t *cell, const double *ox,
                                  const double *oy, const double *ux, const double *uy, const double *uz,
                                  const double *w);

/* Set the step counter (the laser source's time is step * dt), e.g. when
 * resuming a saved run (no counterpart in the paper).  PIC_ERR_ARG for a
 * NULL handle or a negative step. */
PIC_API int pic_set_step(pic_t *h, int64_t step);

/* Live particle count of one species into *n (synchronises the stream).
 * PIC_ERR_ARG (NULL handle or n, species out of range), PIC_ERR_CUDA. */
PIC_API int pic_particle_count(pic_t *h, int species, int64_t *n);

/* Particle order (what pic_get_particles returns): grouped by tile in
 * ascending tile order (tile = (cy / tile_ny) * ceil(nx / tile_nx) + cx / tile_nx),
 * inside a tile by cell in row-major order (cy, then cx).  After each step,
 * inside a cell, first the particles that were already in its tile, in their
 * previous order, then the ones that arrived from other tiles, in their
 * previous order (the stable sort of the previous order by (tile, cell,
 * arrived)); after a load, the stable sort by (tile, cell) of (current
 * particles, then the new ones).  Removed particles leave the sequence. */

/* Copy one species' particles to the host in the library's current order,
 * as global FP64 positions, u and w, plus the linear cell index j*nx + i.
 * Arrays must hold pic_particle_count() entries; NULL skips an output. */
PIC_API int pic_get_particles(pic_t *h, int species, double *x, double *y, double *ux, double *uy,
                      double *uz, double *w, int32_t *cell);

/* FP64 diagnostics of the current state (pic_diag): kinetic energy from the
 * particles' momenta (Eq. 2), field energy of E and H, deposited and particle
 * charge, counts.  The paper defines these quantities (Section 2) but prints
 * no such sums; they are this library's checks of a run.  Synchronises the
 * stream.  PIC_ERR_ARG, PIC_ERR_CUDA, and the device errors of pic_sync. */
PIC_API int pic_diagnostics(pic_t *h, pic_diag *out);

/* Per-kernel timing: when enabled, pic_step records CUDA events around each
 * kernel class on the handle's stream.  pic_timings returns the summed
 * milliseconds and launch counts since the last reset:
 * ms[0] particle step, ms[1] particle sort/regroup, ms[2] field solve,
 * ms[3] moments clear; launches[0..3] likewise; launches[4] all kernels. */
PIC_API int pic_set_timing(pic_t *h, int enabled);
PIC_API int pic_timings(pic_t *h, double ms[4], int64_t launches[5], int reset);

/* Allocation-free stable key sort (the paper has no counterpart: it is a service
 * of this library).  For callers that cannot call cudaMalloc -- code whose
 * device memory is owned by another allocator, such as a framework's caching
 * allocator that has reserved the device, and latency-critical loops where a
 * cudaMalloc/cudaFree would synchronise the device.
 *   keys:    device pointer, n 32-bit keys (read only);
 *   n:       0 .. PIC_NOALLOC_MAX_KEYS;
 *   max_key: the largest key value present (sets the number of 8-bit passes);
 *            keys above max_key are sorted only by their low bytes: perm is
 *            still a permutation of 0..n-1, but its order is unspecified;
 *   perm:    device pointer, n entries, written with the stable ascending
 *            order: perm[i] = index of the i-th key (equal keys keep their order);
 *   cuda_stream: cudaStream_t to queue the kernels on (NULL = legacy stream).
 * Allocates nothing: the scratch (about 16.3 MB for the key/value buffers, the
 * histogram and the scan sums) is one fixed array in the library's device image,
 * held by every GPU that loads the library until the process exits.  The first
 * call on a device looks up that array's device address (with the device
 * current) and caches it per device ordinal; make that first call before any
 * stream capture.  The cache assumes the device's primary context (the one the
 * CUDA runtime uses): after cudaDeviceReset, or with another context current
 * on that device, the cached address is stale and must not be used.
 * Every call shares the one array, so calls that overlap on the GPU (other
 * streams, other threads) race; serialise them.  Returns PIC_ERR_CAPACITY for
 * n > PIC_NOALLOC_MAX_KEYS, PIC_ERR_ARG for NULL pointers, PIC_ERR_CUDA if a
 * launch fails.  Asynchronous on the stream. */
#define PIC_NOALLOC_MAX_KEYS 1048576
PIC_API int pic_sort_keys_noalloc(const uint32_t *keys, int64_t n, uint32_t max_key, uint32_t *perm,
                                  void *cuda_stream);

/* Message of the calling thread's last error ("" if none). */
PIC_API const char *pic_last_error(void);

/* Optical field ionisation pass (the paper's targets ionise as the laser
 * arrives, Section 4 and Fig. 3; the paper states no rate).  Each chain moves
 * particles of species ion[c] to species target[c] (the next charge state;
 * Z = target's q, which must exceed ion's q by 1) and adds an electron with
 * the same position, u and weight to species electron[c].  A particle ionises
 * when u < P, with P = 1 - exp(-w dt), w the static ADK tunnelling rate of an
 * s-state held at its maximum above the field of that maximum,
 * w = |C|^2 Ip (K/F')^(2n*-1) exp(-K/(3F')), K = 2 (2 Ip)^(3/2), n* = Z/sqrt(2 Ip),
 * |C|^2 = 2^(2n*) / (n* Gamma(2n*)), F' = min(F, K/(3(2n*-1))), F = |E| at the
 * particle (E of the current time level, linear weights) -- all in atomic
 * units, converted with field_unit_au (the run's field unit in units of
 * 5.142e11 V/m) and time_unit_au (its time unit in units of 2.419e-17 s) --
 * and u the first output of Philox-4x64-10 at counter (index of the particle
 * in its species' order, ion species, step count, 0) and key (seed, 0), as
 * (out >> 11) 2^-53.  All decisions are taken before any particle moves; the
 * ionised particles leave their species (the others keep their order) and are
 * appended, chain by chain, to the target and electron species exactly as
 * stored (cell and in-cell offsets), re-ordered like a load; the moments are
 * redeposited before the next step.  Call between steps (after pic_step).
 *   p:          the chains (n_chains 1 .. PIC_MAX_SPECIES - 1; each ion species
 *               in one chain; ion, target and electron distinct), the units, the seed;
 *   n_ionized:  (may be NULL) transitions of this pass.
 * Allocates device staging for the ion species' particle counts (kept by the
 * handle).  PIC_ERR_ARG for a bad chain or unit, PIC_ERR_OOM, PIC_ERR_CUDA. */
typedef struct pic_ionization {
    int32_t n_chains;
    int32_t ion[PIC_MAX_SPECIES];
    int32_t target[PIC_MAX_SPECIES];
    int32_t electron[PIC_MAX_SPECIES];
    double ip_ev[PIC_MAX_SPECIES];     /* ionisation potential of the transition, eV */
    double field_unit_au;
    double time_unit_au;
    uint64_t seed;
} pic_ionization;
PIC_API int pic_ionize(pic_t *h, const pic_ionization *p, int64_t *n_ionized);

/* One binary-collision pass (the collisions the paper names with ionisation
 * as what drives its growing particle counts, Sections 4-5; it gives no
 * model).  Reading: Takizuka and Abe's binary model (J. Comput. Phys. 25,
 * 205, 1977) on u = p/(m c) as the velocity, with Nanbu and Yonemura's rule
 * for unequal weights.  For each entry (a[k], b[k]) in turn, cell by cell:
 * like particles (a == b) pair as (0,1), (2,3), ... in the species' order
 * (odd counts: the first three as (0,1), (1,2), (2,0) at half the variance);
 * unlike ones pair particle i of the species with more particles in the cell
 * (a on a tie) with particle i mod N_other of the other.  Per pair: relative
 * velocity g, reduced mass mu, density n_L (of the species, or the lower of
 * the two: sum of w over the cell's area), variance
 *   s2 = q1^2 q2^2 n_L ln_lambda kappa dt / (2 mu^2 |g|^3),
 * delta = sqrt(s2) sqrt(-2 ln(1 - v0)) cos(2 pi v1), phi = 2 pi v2, g rotated
 * by 2 atan(delta) about phi; u1 += m2/(m1+m2) dg if v3 < w2/max(w1,w2),
 * u2 -= m1/(m1+m2) dg if v3 < w1/max(w1,w2), with v0..v3 the outputs of
 * Philox-4x64-10 at counter (index in its species' order of the pair's first
 * particle, 16 + k, step, 1), key (seed, 0), as (out >> 11) 2^-53.  Only u
 * changes; the moments are redeposited at rest before their next use.
 *   kappa: r_e omega / c (the classical electron radius in the length unit
 *          c/omega; 2.21e-8 for omega of a 0.8 um laser), > 0.
 *   n_pairs (may be NULL): pairs processed.
 * PIC_ERR_ARG for a bad entry or parameter, PIC_ERR_OOM, PIC_ERR_CUDA. */
#define PIC_MAX_COLLISION_PAIRS 16
typedef struct pic_collisions {
    int32_t n_pairs;                            /* 1 .. PIC_MAX_COLLISION_PAIRS */
    int32_t a[PIC_MAX_COLLISION_PAIRS];         /* species of each entry */
    int32_t b[PIC_MAX_COLLISION_PAIRS];
    double ln_lambda;                           /* Coulomb logarithm, > 0 */
    double kappa;                               /* r_e omega / c, > 0 */
    uint64_t seed;
} pic_collisions;
PIC_API int pic_collide(pic_t *h, const pic_collisions *p, int64_t *n_pairs);

/* ------------------------------------------------------------------------
 * Serving: many independent runs on one GPU.  No counterpart in the paper
 * (which runs one job on many processors); it admits independent runs of
 * different sizes, for example laser-foil parameter scans, by device memory.
 *
 * A server owns a worker thread that drives the GPU.  Requests are admitted
 * in arrival order while a slot is free and the admitted runs' estimated
 * device bytes (pic_estimate_bytes) fit the budget; a request that does not
 * fit waits, one that can never fit fails at once.  Every admitted run gets
 * its own handle and CUDA stream; each scheduling round issues the next
 * steps of every admitted run, so the runs' kernels overlap on the device,
 * and runs that arrive meanwhile join at the next round.  A finished run's
 * diagnostics (and, if asked, its moments and fields) are copied to host
 * memory and its device memory is freed at once.
 * ------------------------------------------------------------------------ */

/* Device bytes a handle of this configuration holds with n_per_species[s]
 * particles loaded (NULL: none).  Needs no GPU. */
PIC_API int pic_estimate_bytes(const pic_config *cfg, const int64_t *n_per_species, uint64_t *bytes);

typedef struct pic_server pic_server;

typedef struct pic_server_config {
    uint64_t mem_budget;       /* device bytes for the admitted runs (0 = 80 % of the free memory at creation) */
    int32_t max_slots;         /* runs admitted at once (0 = 64) */
    int32_t steps_per_round;   /* steps issued per run per scheduling round (0 = 1) */
    int32_t batch_min_runs;    /* > 0: groups of at least this many runs of one form advance by one
                                  pic_batch_step; 0: every run steps on its own stream (default:
                                  measured faster, the streams interleave freely) */
} pic_server_config;

#define PIC_REQ_QUEUED 0
#define PIC_REQ_RUNNING 1
#define PIC_REQ_DONE 2
#define PIC_REQ_FAILED 3
#define PIC_REQ_CANCELLED 4

#define PIC_SUBMIT_KEEP_GRIDS 1    /* keep moments and fields for pic_server_result */

typedef struct pic_request_status {
    int32_t state;             /* PIC_REQ_* */
    int32_t error;             /* pic error code of a failed request */
    int64_t steps_done, steps_total;
    double t_submit, t_start, t_finish;  /* seconds on the server clock (pic_server_now); 0 = not yet */
    double particle_steps;     /* steps x mean live particle count, set when done */
    uint64_t device_bytes;     /* admission estimate */
} pic_request_status;

/* Create a server (the device current in the calling thread is the one it uses). */
PIC_API int pic_server_create(const pic_server_config *cfg, pic_server **out);

/* Stop the worker (runs in flight are abandoned) and free everything. */
PIC_API int pic_server_destroy(pic_server *srv);

/* Queue a run: cfg (cuda_stream is ignored; the server gives each run its
 * own stream), nsteps >= 0, one pic_species_data per species with arrays in
 * host memory (pageable or page-locked); the arrays are copied before the
 * call returns.  flags: PIC_SUBMIT_*.  *id identifies the
 * request.  Invalid configurations fail here with PIC_ERR_ARG. */
PIC_API int pic_server_submit(pic_server *srv, const pic_config *cfg, int32_t nsteps,
                              const pic_species_data *species, int32_t flags, int64_t *id);

PIC_API int pic_server_status(pic_server *srv, int64_t id, pic_request_status *out);

/* Results of a finished run: diagnostics, and with PIC_SUBMIT_KEEP_GRIDS the
 * moments and fields in pic_moments / pic_fields layout (NULL skips one).
 * PIC_ERR_STATE if the run has not finished. */
PIC_API int pic_server_result(pic_server *srv, int64_t id, pic_diag *diag, double *rho, double *S9, double *dj3,
                              double *E3, double *H3);

/* Forget a finished, failed or cancelled request and its host results. */
PIC_API int pic_server_release(pic_server *srv, int64_t id);

/* Self-test of the kernels' bounded waits (no counterpart in the paper):
 * one block arms an mbarrier for a transfer that never comes and waits on it
 * with the push's poll bound.  Returns PIC_ERR_TIMEOUT when the wait ran out
 * and the kernel returned its timeout status (the expected outcome; the
 * context stays usable), PIC_OK if the barrier completed, PIC_ERR_CUDA or
 * PIC_ERR_OOM on a failed launch or allocation.  *seconds (may be NULL) =
 * wall time of the call.  cuda_stream: the stream to run on (NULL = legacy
 * default stream). */
PIC_API int pic_selftest_wait(void *cuda_stream, double *seconds);

/* FP64 arithmetic rate of this GPU (no counterpart in the paper): the
 * denominator of the FP64 push's roofline, measured rather than derived from
 * unit counts.  Launches a kernel of independent FP64 fused multiply-add
 * chains on every SM (8 chains per thread, 8 blocks of 256 threads per SM;
 * each launch runs for a few tens of milliseconds), once to warm up and then
 * `repeats` times, each timed with CUDA events on cuda_stream (NULL = legacy
 * default stream); *tflops = the best launch's rate, counting an FMA as 2
 * flops.  Allocates 8 bytes per thread for the chains' results (freed before
 * returning).  PIC_ERR_ARG for NULL tflops or repeats < 1, PIC_ERR_OOM,
 * PIC_ERR_CUDA on a failed launch.  Synchronous. */
PIC_API int pic_probe_fp64_rate(void *cuda_stream, int repeats, double *tflops);

/* Cancel a request: a queued one leaves the queue at once, a running one
 * stops before its next step (its device memory and slot are freed at the end
 * of the worker's current round); either ends in PIC_REQ_CANCELLED with the
 * steps done so far and no results.  Other runs are not affected.
 * PIC_ERR_ARG for an unknown id, PIC_ERR_STATE if the request has already
 * finished, failed or been cancelled. */
PIC_API int pic_server_cancel(pic_server *srv, int64_t id);

/* Block until no request is queued or running, or timeout_s passes
 * (PIC_ERR_TIMEOUT). */
PIC_API int pic_server_wait_all(pic_server *srv, double timeout_s);

/* Seconds on the server's monotonic clock. */
PIC_API double pic_server_now(pic_server *srv);

/* Batched stepping of several runs (what the server uses).  A batch owns the
 * scratch of the batched launches: up to max_runs argument blocks in device
 * and page-locked host memory and the work-list prefixes.  pic_batch_step
 * advances n runs by nsteps: each run's field solve, regroup decision and
 * clears stay on its own stream, then ONE persistent push launch over the
 * (run, species, tile, segment run) work items of all n runs and ONE regroup
 * launch over all (run, tile, species) run on the batch's stream, joined to
 * the runs' streams by events.  The results equal per-run pic_step calls
 * (bitwise with PIC_DEPOSIT_DETERMINISTIC).  All runs of a call must share
 * precision and deposit mode; PIC_ERR_ARG otherwise. */
typedef struct pic_batch pic_batch;
PIC_API int pic_batch_create(int max_runs, void *cuda_stream, pic_batch **out);
PIC_API int pic_batch_destroy(pic_batch *b);
PIC_API int pic_batch_step(pic_batch *b, pic_t **runs, int n, int nsteps);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
