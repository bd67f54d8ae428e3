/*
 * bp.h -- C ABI of the GB300 two-body macro-ion particle-in-cell step.
 *
 * Method: An, Chen, Sheng, Zhang, "Modeling of bound electron effects in
 * particle-in-cell simulation" (arXiv 2208.08038).  A partially ionised
 * macro-ion is a two-body particle: a nucleus (q1, m1) and a combined bound
 * electron (q2, m2) joined by a modified Coulomb force (Sec. 2).  Each step
 * gathers the Yee-staggered E and B at both bodies, Boris-pushes both under
 * the external fields plus the internal field, deposits the charge-conserving
 * (Esirkepov, quadratic shape) current and advances Maxwell's equations with
 * Yee FDTD.  Every step runs in the library's own sm_103a kernels.
 *
 * Units are normalised: c = 1, lengths in 1/k0 (lambda0 = 2 pi), times in
 * 1/omega0, E in m_e c omega0 / e (so a0 = |E|), B in m_e omega0 / e,
 * densities in n_c, charges in e, masses in m_e.
 *
 * Memory: the context owns its device buffers and obtains them through the
 * caller's allocator (or cudaMalloc when none is given).  Every array passed
 * in is owned by the caller and is only read during the call; every
 * destination is owned by the caller.  Host pointers unless a function says
 * otherwise.  Row-major ("[n][3]" = three consecutive values per item).
 *
 * Errors: every function returns a bp_status.  Nothing crosses the ABI as an
 * exception.  Kernels report problems through a device status word that
 * bp_sync() returns; bp_last_error() gives a message for the last failure.
 *
 * Concurrency: a context is used by one host thread at a time; all its work
 * is issued on the stream given to bp_create.
 */
#ifndef BP_H
#define BP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bp_ctx bp_ctx;

typedef enum {
  BP_OK = 0,
  BP_ERR_ARG = -1,       /* invalid argument */
  BP_ERR_OOM = -2,       /* the allocator returned NULL */
  BP_ERR_CUDA = -3,      /* a CUDA runtime call failed */
  BP_ERR_CFL = -4,       /* dt violates the Courant limit or omega_b dt >= 2 */
  BP_ERR_NONFINITE = -5, /* a non-finite momentum was produced */
  BP_ERR_DOMAIN = -6,    /* a particle left the region its tile can handle */
  BP_ERR_TIMEOUT = -7,   /* a bounded device wait gave up */
  BP_ERR_IO = -8,        /* save/load file error or checksum mismatch */
  BP_ERR_STATE = -9      /* call not valid in the current state */
} bp_status;

enum { BP_PERIODIC = 0, BP_OPEN = 1 };
enum { BP_DEPOSIT_ATOMIC = 0, BP_DEPOSIT_SORTED = 1 };
enum { BP_TWO_BODY = 0, BP_FREE = 1 };
enum { BP_EX = 0, BP_EY, BP_EZ, BP_BX, BP_BY, BP_BZ, BP_JX, BP_JY, BP_JZ };

/* Device memory provider.  alloc(bytes, stream, user) returns device memory
 * usable on `stream` or NULL; free(ptr, stream, user) releases it.  Both are
 * called only from bp_create, bp_add_*, bp_load_particles, bp_set_*,
 * bp_forward_ckpt and bp_destroy -- never from bp_step. */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *user);
  void (*free)(void *ptr, void *stream, void *user);
  void *user;
} bp_allocator;

/* Grid.  The simulated axes are x, (y), (z); Yee stagger: E_x at (i+1/2, j, k),
 * E_y at (i, j+1/2, k), E_z at (i, j, k+1/2), B_x at (i, j+1/2, k+1/2), B_y at
 * (i+1/2, j, k+1/2), B_z at (i+1/2, j+1/2, k); J with E.  Open axes use Mur
 * first-order absorbing faces on the tangential E; periodic axes wrap.
 * Tiles are 16 cells (1D), 16 x 16 (2D), 8 x 8 x 8 (3D); n[a] must be a
 * multiple of the tile and the bit widths of n[0..2] may sum to at most 31. */
typedef struct {
  int dims;           /* 1, 2 or 3 */
  int64_t n[3];       /* cells per axis (1 on unused axes) */
  double dx[3];       /* cell size per axis */
  double dt;          /* time step; must satisfy dt < 1/sqrt(sum 1/dx^2) */
  int boundary[3];    /* BP_PERIODIC or BP_OPEN per axis */
  int deposit_mode;   /* BP_DEPOSIT_ATOMIC (FP32 shared atomics) or
                         BP_DEPOSIT_SORTED (integer fixed point: bit-exact reruns) */
  int tile[3];        /* 0, or the fixed tile size of the dimension */
} bp_grid_desc;

/* Species.  BP_TWO_BODY follows Sec. 2: q2 = -Zb, m2 = Zb, q1 = qc - q2,
 * m1 = mc - m2; omega_b[i] is the natural frequency of parameter index i,
 * mapped to the softening a_c by w_c^2 = |q1 q2| kappa / (m_r a_c^3)
 * (Sec. 3.1), kappa = r_e 2 pi / lambda0_m.  BP_FREE is a single body of
 * charge q and mass m.  weight: each macro-particle adds q * weight * S to
 * the charge density, S the quadratic shape (sums to 1). */
typedef struct {
  int kind;
  double Zb, qc, mc;
  double q, m;
  double weight;
  double lambda0_m;
  const double *omega_b; /* [n_omega], copied */
  int n_omega;
} bp_species_desc;

/* Laser launched by a current sheet on the x node plane ia: a sheet K
 * radiates E = -K/2 on either side, so J = -(2/dx) f(t, y, z) (times
 * cos(theta) for comp = 2) launches f forward, with
 *   f = a0 env(tau) prof(y, z) sin(omega tau + phase),  tau = t - (y - yc) sin(theta),
 *   env = exp(-2 ln2 (tau - t0)^2 / fwhm^2)            (fwhm > 0: intensity FWHM)
 *       = sin^2(pi tau / (2 ramp)) for 0 < tau < ramp, 1 after, 0 before  (fwhm = 0)
 *   prof = exp(-(((y - yc) cos(theta))^2 + (z - zc)^2) / waist^2)  (waist > 0), else 1.
 * comp 1 drives J_y (p-polarised in the x-y plane), comp 2 drives J_z. */
typedef struct {
  int comp;
  double a0, omega, theta, waist, fwhm, t0, ramp, phase;
  int64_t ia;
  double yc, zc;
} bp_laser_desc;

/* Create a context on the calling thread's current CUDA device.  stream is
 * a cudaStream_t (NULL: legacy default stream).  allocator may be NULL.
 * Source: Sec. 1 and Sec. 2 -- a PIC grid whose fields follow Maxwell's
 * equations with the macro-particles' currents as sources; Sec. 3.1 keeps the
 * vacuum permittivity in those equations.  (The Yee stagger, the Mur faces
 * and the tile shape are this library's choices; the paper fixes none.)
 * BP_ERR_ARG for a bad description, BP_ERR_CFL when dt breaks the Courant
 * limit, BP_ERR_OOM when the allocator fails; *out is set only on BP_OK. */
int bp_create(const bp_grid_desc *grid, const bp_allocator *allocator, void *stream, bp_ctx **out);
/* Release every device buffer of the context (through its allocator) and the
 * context itself; NULL is ignored.  (The paper has no counterpart: resource
 * release of this interface.) */
void bp_destroy(bp_ctx *ctx);
/* Text of the last failure of a call on ctx ("null context" for NULL),
 * valid until the next call on ctx.  (The paper has no counterpart.) */
const char *bp_last_error(const bp_ctx *ctx);

/* Add a species (Sec. 2: the two-body split q2 = -Zb e, m2 = Zb m_e,
 * q1 = qc - q2, m1 = mc - m2; Sec. 3.1: omega_b -> a_c).  *species_id
 * receives its index.  BP_ERR_ARG for a bad description, BP_ERR_CFL when
 * omega_b dt >= 2 (the leapfrog oscillation is then unstable). */
int bp_add_species(bp_ctx *ctx, const bp_species_desc *desc, int *species_id);

/* Load macro-particles from host arrays: ion positions x [n][dims] and
 * momenta u = p/(m c) [n][3] (NULL: at rest), parameter index per ion
 * param_idx [n] (NULL: all 0).  Two-body ions get the initial conditions of
 * Sec. 2: r1 = r2 = x, p1 + p2 = p_c, q1 v1 + q2 v2 = 0 (u1 = u2 = u for
 * neutral ions; non-relativistic split otherwise).  Particles are then
 * sorted by tile.  May be called once per species.  The arrays stay the
 * caller's and are not kept: page-locked arrays the device can address
 * (pinned or registered host memory) are read in place by the conversion
 * kernel; other host memory is copied through a device staging buffer.
 * Returns when the particles are on the device.  BP_ERR_NONFINITE for a
 * non-finite position or momentum, BP_ERR_DOMAIN for a position outside an
 * open grid or a param_idx out of range (the species then stays unloaded
 * and may be loaded again). */
int bp_load_particles(bp_ctx *ctx, int species_id, const double *x, const double *u,
                      const int32_t *param_idx, int64_t n);

/* Generate a medium on the device: ppc ions per cell over the cell box
 * [lo, hi), at seeded uniform in-cell positions and Gaussian momenta of
 * standard deviation sigma_u per component, with the counter-based
 * SplitMix64 streams that the input module of this package also implements
 * (ion g = cell rank * ppc + p takes uniforms 3g+a and normals 3g+a).
 * Source: Sec. 3.1 (a neutral medium of partially ionised atoms), with the
 * initial conditions of Sec. 2 applied to every ion as in bp_load_particles.
 * BP_ERR_STATE if the species is loaded, BP_ERR_ARG for an empty or
 * off-grid box. */
int bp_set_medium(bp_ctx *ctx, int species_id, const int64_t lo[3], const int64_t hi[3], int ppc,
                  uint64_t seed, double sigma_u);

/* Add a laser (see bp_laser_desc).  Source: Sec. 3.1 (an x-ray laser of
 * given wavelength and normalised amplitude a = |eE / (m_e omega c)|, normal
 * or oblique incidence) and Sec. 3.2 (a beam of given width, pulse length and
 * peak field, incident at an angle to the crystal axis).  The current-sheet
 * antenna is this library's launcher; the paper does not say how it injects.
 * At most 4 lasers (BP_ERR_ARG beyond, or for comp not 1 or 2). */
int bp_add_laser(bp_ctx *ctx, const bp_laser_desc *laser);

/* Probe: records field component comp (BP_EX..BP_JZ) at the given linear
 * node indices (i + nx (j + ny k)) after every step, up to capacity samples.
 * Source: Sec. 3.1 (group velocities and reflection phase shifts are read off
 * the simulated field at fixed points) and Sec. 3.2 (the transmitted E_x).
 * nodes [npts] is copied; BP_ERR_ARG for an index off the grid. */
int bp_add_probe(bp_ctx *ctx, int comp, const int64_t *nodes, int64_t npts, int64_t capacity,
                 int *probe_id);

/* Advance n_steps leapfrog steps (asynchronous on the context stream):
 *   B^n = B^{n-1/2} - dt/2 curl E^n; gather; internal field; Boris; drift;
 *   J^{n+1/2} (Esirkepov + antenna); B^{n+1/2}; E^{n+1} = E^n + dt (curl B - J).
 * Source: Sec. 2 -- the Boris equations for both bodies, each with the fields
 * at its own position plus the field of the modified Coulomb force
 * q1 q2 r / (4 pi eps0 (r^2 + a_c^2)^{3/2}), and the bodies' currents
 * q_{1,2} v_{1,2} / dV added to the total current that updates the fields;
 * Sec. 3.1 -- Maxwell's equations with the vacuum permittivity.  Returns
 * BP_ERR_ARG for n_steps < 0; kernel problems (a particle off its tile's
 * reach, a non-finite momentum) surface at the next bp_sync.  With two or
 * more steps and push timing off, the steps replay a CUDA graph of one step
 * (captured on first use and again whenever a launch argument has changed:
 * particle arrays, lasers, probes, parameters); single steps and timed steps
 * launch the same kernels directly, with the same results bit for bit. */
int bp_step(bp_ctx *ctx, int64_t n_steps);

/* Wait for the stream and return the device status word as a bp_status:
 * BP_ERR_DOMAIN, BP_ERR_NONFINITE or BP_ERR_TIMEOUT from the kernels,
 * BP_ERR_CUDA for a failed CUDA call.  (The paper has no counterpart:
 * completion and error reporting of this interface.) */
int bp_sync(bp_ctx *ctx);

/* Copy field component comp (nz*ny*nx floats, x fastest) to dst: a device
 * pointer when on_device != 0, else a host pointer.  Synchronous.  Source:
 * Sec. 3.1 and Sec. 3.2 read their results off the fields (the Fourier
 * transforms of E that show the refracted and the Bragg-scattered beams). */
int bp_read_field(bp_ctx *ctx, int comp, float *dst, int on_device);

/* (Source: as bp_read_field.)
 * Enqueue a read of field component comp, as it stands after the steps
 * enqueued so far, into caller-owned host memory dst (nz*ny*nx floats; page-
 * locked memory for the copy to run asynchronously).  Returns at once: the
 * field is first copied to one of two device snapshot buffers on the
 * context's stream, and the snapshot goes to dst on a side stream, so the
 * steps that follow overlap the transfer.  dst is valid after the next
 * bp_sync (which waits for every enqueued read).  The snapshot buffers
 * (2 * nz*ny*nx floats) are allocated at the first call; BP_ERR_OOM if they
 * cannot be. */
int bp_read_field_async(bp_ctx *ctx, int comp, float *dst);

/* Overwrite field component comp from src (nz*ny*nx floats; device pointer
 * when on_device != 0).  Synchronous.  Used to start from given fields.
 * (The paper has no counterpart: its runs start from zero fields.) */
int bp_write_field(bp_ctx *ctx, int comp, const float *src, int on_device);

/* Copy up to cap samples of probe probe_id ([samples][npts] floats) to host
 * dst; *n receives the number of samples recorded.  Source: as bp_add_probe.
 * BP_ERR_ARG for an unknown probe. */
int bp_read_probe(bp_ctx *ctx, int probe_id, float *dst, int64_t cap, int64_t *n);

/* Copy the bodies' states to host arrays in load order: x1, x2 positions
 * [n][3] (simulated axes reduced to the box for periodic axes; body 2 at
 * x1 - r), u1, u2 [n][3]; *n receives the number alive.  Any pointer may be
 * NULL.  Free particles fill x1, u1 only.  Source: Sec. 2 (each body has its
 * own position and momentum).  Synchronous. */
int bp_read_particles(bp_ctx *ctx, int species_id, double *x1, double *x2, double *u1, double *u2,
                      int64_t cap, int64_t *n);

/* Source: Sec. 3.2 (a crystal: ions placed periodically with crystal
 * constant d, the laser incident at an angle to the crystal axis), with the
 * initial conditions of Sec. 2.
 * Load a seeded lattice on the device: per_site ions at each of the n_sites
 * sites (sites [n_sites][D], FP64, lengths in 1/k0), ion g = site * per_site
 * + p at its site plus jitter * N(0, 1) per simulated axis (normals D g + a of
 * the jitter stream of seed) with momentum sigma_u * N(0, 1) per component
 * (normals 3 g + a of the momentum stream), split into the two bodies like
 * bp_load_particles; site_param [n_sites] (may be NULL) gives every ion of a
 * site that parameter index.  Load order = g.  The counter-based generator
 * is SplitMix64 (uniforms (z >> 11) 2^-53, Box-Muller normals), a published
 * definition the caller can evaluate on the host.  Synchronous;
 * BP_ERR_STATE if the species is loaded, BP_ERR_DOMAIN for an ion off the
 * grid. */
int bp_set_lattice(bp_ctx *ctx, int species_id, const double *sites, int64_t n_sites, int per_site, double jitter,
                   uint64_t seed, double sigma_u, const int32_t *site_param);

/* (The paper has no counterpart: checkpoint and restart of a run.)
 * Write the context's state to a file: the step counter, every species'
 * a_c values and particles (load ids, positions, momenta, parameter
 * indices, tile offsets), E and B, the status word.  bp_load reads it into a
 * context created with the same grid description and deposit mode and with
 * the same species added in the same order (lasers and probes are the loading
 * context's own); its species must not be loaded yet (bp_reset clears them).
 * Continuing from a loaded state gives the same fields as continuing the
 * saved run (bit-identical in the sorted deposit mode).  Host-endian binary
 * ending with the CRC-32 (zlib's convention: reflected polynomial
 * 0xEDB88320) of every byte before it, little-endian; synchronous.  bp_load
 * verifies the checksum before it changes anything: BP_ERR_IO for an
 * unreadable, truncated, corrupted or foreign file (the context is left as
 * it was), BP_ERR_ARG when the grid or the species differ. */
int bp_save(bp_ctx *ctx, const char *path);
int bp_load(bp_ctx *ctx, const char *path);

/* (Source: as bp_read_particles.)
 * Copy the states of the particles with load ids ids[0..n) (load order of
 * bp_load_particles / bp_set_medium, any order, repeats allowed) to host
 * arrays in the order of ids: x1, x2, u1, u2 [n][3] as bp_read_particles
 * (any may be NULL).  found[k] (may be NULL) receives 1 if particle ids[k]
 * is alive, else 0 (its rows are then 0).  A device search over the species'
 * particles (no host copy of the whole species); allocates scratch through
 * the context's allocator; synchronous.  BP_ERR_ARG for a negative id. */
int bp_read_particles_by_id(bp_ctx *ctx, int species_id, const int64_t *ids, int64_t n, double *x1, double *x2,
                            double *u1, double *u2, unsigned char *found);

/* Gauss-law residual R = div E - rho at every node, in FP64 on the device
 * (rho deposited in FP64 from the stored FP32 positions with the quadratic
 * shape).  dst holds nz*ny*nx doubles (device pointer if on_device).  (The
 * paper has no counterpart: a diagnostic of the discrete continuity that the
 * charge-conserving deposit of Sec. 2's body currents keeps, R^n = R^0.)
 * Allocates an FP64 scratch grid through the allocator on its first call
 * with a host dst (BP_ERR_OOM if that fails).  Synchronous. */
int bp_residual(bp_ctx *ctx, double *dst, int on_device);

/* bp_residual for callers that cannot have the library allocate device
 * memory during the call.  (The paper has no counterpart: this is an
 * interface for such callers.)  bp_residual obtains an FP64 scratch grid
 * through the context's allocator when dst is host memory; a thread that
 * does not own that allocator, or a run whose device memory is fully
 * committed, cannot allow that.  This entry point keeps the scratch in a
 * fixed array of the library's static device memory (32 MiB, present on
 * every GPU that loads the library until the process exits) and calls no
 * cudaMalloc, cudaFree or allocating routine.
 *   dst   host pointer to nz*ny*nx doubles, written with div E - rho.
 *   Grids of more than 4,194,304 nodes are rejected with BP_ERR_ARG.
 *   The context's device must be current (else BP_ERR_STATE).  The first
 *   call in each CUDA context looks up the array's device address
 *   (cudaGetSymbolAddress) and caches it under the context's id; make that
 *   first call before any stream capture.  A context destroyed and created
 *   again (cudaDeviceReset) has a new id, so its first call looks the
 *   address up afresh.
 *   All calls share the one array, which keeps the previous call's values
 *   (each call clears it first); calls that overlap on the GPU, from any
 *   contexts of the process, race on it.  Synchronous. */
int bp_residual_noalloc(bp_ctx *ctx, double *dst);

/* --- discrete adjoint -------------------------------------------------- */

/* Zero the fields, the step counter and the probe records, and unload the
 * particles (species and lasers stay; particle arrays are reused by the next
 * bp_load_particles).  (The paper has no counterpart: it restarts a run for
 * the adjoint's repeated forward passes.) */
int bp_reset(bp_ctx *ctx);

/* Replace the bound-electron frequencies omega_b[n] of a two-body species
 * (n = its n_omega); a_c follows from w_c^2 = |q1 q2| kappa / (m_r a_c^3).
 * Source: Sec. 3.1 (the natural frequency from the Taylor series of V_M).
 * BP_ERR_ARG for another n or a free species, BP_ERR_CFL for omega_b dt >= 2. */
int bp_set_omega(bp_ctx *ctx, int species_id, const double *omega_b, int n);

/* (The paper has no adjoint.  This checkpointed forward run and bp_backward
 * give gradients of a probe loss with respect to the natural frequencies of
 * Sec. 3.1 and the lattice sites of Sec. 3.2, through the discrete step of
 * Sec. 2.)
 * Run n_steps steps like bp_step (probes recorded), keeping the state before
 * every K-th step (E, B, particles, status) for the reverse pass.  Needs
 * BP_DEPOSIT_SORTED, whose bit-reproducible steps make the recomputation
 * exact. */
int bp_forward_ckpt(bp_ctx *ctx, int64_t n_steps, int K);

/* (Source: as bp_forward_ckpt.)
 * Reverse pass of the run of the last bp_forward_ckpt: for each segment,
 * newest first, restore its checkpoint, recompute its K steps storing every
 * step's state, then apply the transposed step K times (transposed Yee with
 * Mur faces, Esirkepov deposit transposed as a gather of the current adjoint,
 * reversed drift, Boris and modified-Coulomb force, gather transposed as a
 * deposit).  The loss gradient enters as dl_dprobe [n_steps][npts] (host,
 * FP32): dL/d(sample s of probe probe_id recorded by that run); the probe
 * must record an E component.  Outputs (host, FP64, reduced on the device in
 * a fixed order; either may be NULL):
 *   grad_omega [n_omega]        dL/d omega_b per parameter index of species_id
 *   grad_group [n_groups][dims] sum over the ions i of group g of dL/dx_i at
 *                               load time (both bodies start at x_i), with
 *                               group[n] the caller's group of each ion in
 *                               load order (e.g. its lattice site).
 * Afterwards the context holds an intermediate state: call bp_reset before
 * the next run. */
int bp_backward(bp_ctx *ctx, int probe_id, const float *dl_dprobe, int species_id, double *grad_omega,
                const int32_t *group, int64_t n_groups, double *grad_group);

/* Number of own-kernel launches issued since creation (for accounting).
 * (The paper has no counterpart; instrumentation.) */
int64_t bp_kernel_launches(const bp_ctx *ctx);

/* Per-kernel CUDA-event timing of the push/deposit launches: when enabled,
 * bp_step records events around each push launch (and launches directly,
 * not through the step graph); bp_push_time returns
 * the summed milliseconds and launch count since the last reset (bp_time_push
 * resets both, and the work counters of bp_push_work).  (The paper has no
 * counterpart; instrumentation.) */
int bp_time_push(bp_ctx *ctx, int enable);
int bp_push_time(bp_ctx *ctx, double *ms, int64_t *launches);

/* Work of the timed push launches since the last bp_time_push: *full
 * receives the number of particle pushes that gathered, kicked and deposited
 * (the whole step of Sec. 2), *quiet the number of co-moving neutral ions
 * that the quiet-tile pass only drifted (no field had reached their tiles, so
 * they carry no current).  Counted on the device only while timing is
 * enabled; synchronous.  (The paper has no counterpart; instrumentation.) */
int bp_push_work(bp_ctx *ctx, int64_t *full, int64_t *quiet);

/* Work of the field updates since the last call: *active_tiles receives the
 * tiles the field kernels updated, summed over the steps (on grids of 1024
 * tiles or more they skip tiles whose neighbourhood has never held a field
 * and receives no current: their E, B and J stay exactly zero), *steps the
 * steps counted; the count restarts at zero.  Smaller grids update every
 * tile and count nothing.  Synchronous.  (The paper has no counterpart;
 * instrumentation.) */
int bp_field_work(bp_ctx *ctx, int64_t *active_tiles, int64_t *steps);

/* (The paper has no counterpart: a resource limit of this implementation.)
 * Capacity of the sorted deposit's general-case record buffer, in records
 * (BP_DEPOSIT_SORTED only).  A particle whose positions change their nearest
 * node in a step (Esirkepov's five-node case) leaves a record that a
 * separate kernel adds to the fixed-point current; when a step has more
 * such particles than the capacity, the rest deposit in place.  Both paths
 * add the same integers, so the fields do not depend on the capacity.
 * n > 0 fixes the capacity (at least 1); n = 0 restores the default (one
 * record per 256 particles, at least 65,536).  Takes effect at the next
 * bp_step; returns BP_ERR_ARG for n < 0 or a context in atomic mode,
 * BP_ERR_OOM if the buffer cannot be allocated then. */
int bp_set_record_capacity(bp_ctx *ctx, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* BP_H */
