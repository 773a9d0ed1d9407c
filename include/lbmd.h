/*
 * lbmd.h -- C ABI of the GB300 (sm_103a) implementation of one time step of the
 * two-component D3Q19 Shan-Chen lattice Boltzmann fluid coupled to off-lattice point
 * particles by Ahlrichs-Duenweg friction and solvation forces, after Sega, Sbragaglia,
 * Kantorovich, Ivanov, "Mesoscale Structures at Complex Fluid-Fluid Interfaces: a Novel
 * Lattice Boltzmann / Molecular Dynamics Coupling" (arXiv:1306.0788).
 *
 * Conventions shared by every call
 *   Units      lattice units: spacing a = 1, lattice time step tau = 1 (Sec. 3).
 *   Lattice    nx * ny * nz nodes at integer positions, periodic in x, y and z.  Site
 *              index s = (z * ny + y) * nx + x (x fastest).
 *   Components 0 = A, 1 = B.
 *   D3Q19      velocity order i = 0; +x,-x,+y,-y,+z,-z; (+x+y),(-x-y),(+x-y),(-x+y),
 *              (+x+z),(-x-z),(+x-z),(-x+z), (+y+z),(-y-z),(+y-z),(-y+z)  (Eq. velo; the
 *              paper leaves the order within a shell free).  Weights 1/3, 1/18, 1/36
 *              (Eq. weights).
 *   Populations are exchanged as the post-streaming values f_zi(r, t) at a step
 *              boundary, layout [19][nz][ny][nx] per component, FP32.
 *   Particles  positions in [0, n) per axis (wrapped on input), given and returned in
 *              the caller's original order (index = particle id).
 *   Pointers   every pointer argument is caller-owned HOST memory, read or written
 *              before the call returns, unless the name ends in _dev.  The library owns
 *              all device memory it allocates; lbmd_destroy frees it.
 *   Streams    all device work of a context is issued on the stream given to
 *              lbmd_create (NULL = the legacy default stream).  Calls that return data
 *              to the host synchronise that stream.
 *   Errors     every int-returning call returns LBMD_OK (0) or a negative LBMD_E_* code;
 *              lbmd_last_error gives a message for the last failure of the context.
 *              Device-side failures (negative or non-finite density, broken bond,
 *              particle outside the box) are recorded in a device error word during
 *              lbmd_step and reported by the next call that synchronises (lbmd_sync,
 *              getters, lbmd_diagnostics); they are sticky until lbmd_clear_error.
 *   Threads    a context must not be used from two host threads at once.
 */
#ifndef LBMD_H
#define LBMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBMD_OK 0
#define LBMD_E_INVALID_ARG (-1)
#define LBMD_E_NOMEM (-2)
#define LBMD_E_CUDA (-3)
#define LBMD_E_NEGATIVE_DENSITY (-4) /* Sec. 3: large lambda can drive densities negative */
#define LBMD_E_NONFINITE (-5)
#define LBMD_E_TIMEOUT (-6)
#define LBMD_E_UNIMPLEMENTED (-7)
#define LBMD_E_BOND_BROKEN (-8) /* FENE bond stretched to or beyond R0 */
#define LBMD_E_STATE (-9)       /* call out of order (e.g. step before init_fluid) */
#define LBMD_E_PARTICLE_TOO_FAST (-10) /* md_substeps > 1: a particle crossed more than one cell in one step */
#define LBMD_E_DRIFT (-11) /* FP64 drift check: a conserved total moved beyond drift_tol (lbmd_params.diag_every) */

/* population storage: FP32, or 16-bit (IEEE half or bfloat16) holding the shifted value
 * f_zi - w_i rho0_z (lbmd_params.rho0_A / rho0_B); collisions always compute in FP32 and the
 * diagnostics in FP64 */
#define LBMD_STORAGE_FP32 0
#define LBMD_STORAGE_FP16_SHIFTED 1
#define LBMD_STORAGE_BF16_SHIFTED 2

/* collision operator (lbmd_params.collision) */
#define LBMD_COLLISION_BGK 0 /* every relaxation eigenvalue -1/tau_r; no fluid noise */
#define LBMD_COLLISION_MRT 1 /* Eq. MODES: per-mode eigenvalues, Gaussian mode noise at kT > 0 */

/* bonded interactions */
#define LBMD_BOND_FENE 2     /* U = -(k R0^2 / 2) ln(1 - (r/R0)^2) (Kremer-Grest form) */
#define LBMD_BOND_HARMONIC 3 /* U = (k/2) (r - d)^2 (Sec. 4.3, 4.4) */

/* warnings (bit mask) raised by lbmd_create / lbmd_set_types for the stability limits of
 * Sec. 3; they never fail a call */
#define LBMD_WARN_GAMMA_DT (1u << 0)   /* gamma dt / m not << 1 (here: > 0.5) */
#define LBMD_WARN_VISCOSITY (1u << 1)  /* eta/rho = c_s^2 (tau_r - 1/2) below 1e-3 */
#define LBMD_WARN_BOLTZMANN (1u << 2)  /* Bo = sqrt(kT / (rho c_s^2)) above 0.5 */
#define LBMD_WARN_ASYMMETRIC_G (1u << 3) /* g_AB != g_BA: no momentum guarantee (Sec. 2) */

#define LBMD_MAX_TYPES 8

typedef struct lbmd_ctx lbmd_ctx;

/* Model and numerics.  tau_r: BGK relaxation time (> 1/2); every relaxation eigenvalue
 * of the collision operator (Eq. collis, Eq. MODES) is -1/tau_r.  g_AB, g_BA: Shan-Chen
 * couplings of Eq. (SCforce) with psi = rho and g_AA = g_BB = 0; the lattice sum uses
 * the isotropy weights w_i.  kT: thermal energy of the particle noise (Eq. NEWTON).
 * dt: particle time step, must equal the lattice time step 1.  storage: LBMD_STORAGE_*.
 * rho0_A, rho0_B: shift reference of the 16-bit storages (ignored for FP32).  seed: key
 * of the counter-based particle and fluid noise.
 * collision: LBMD_COLLISION_BGK, or LBMD_COLLISION_MRT -- the collision of Eq. MODES in the
 * mode space of the orthogonal D3Q19 polynomials of Duenweg, Schiller and Ladd: the shear
 * modes relax with lambda_s = -1/tau_r, the bulk mode with lambda_bulk, each component's
 * momentum with lambda_mom (interdiffusion, mu = -(1/lambda_mom + 1/2)), the nine kinetic
 * modes with lambda_ghost, every eigenvalue in (-2, 0); at kT > 0 each mode receives
 * Gaussian noise with the amplitude that gives equipartition at temperature kT, the momentum
 * noise of A and B being one random number with opposite signs (Sec. 2).  The lambda_* are
 * ignored with BGK.
 * md_substeps: K >= 1 particle substeps per lattice step (Sec. 3: gamma dt / m << 1 and stiff
 * pair forces need a particle step below the lattice one): forces, momentum return and
 * particle update run K times with dt / K while the fluid fields of the step stay frozen,
 * and the collision takes the average momentum return.  K > 1 requires every particle to
 * stay within one cell of where the step started (else LBMD_E_PARTICLE_TOO_FAST); batches
 * take K = 1 only.
 * diag_every, drift_tol: the FP64 drift check.  The model conserves the total mass of each
 * component (the collision and the forcing term of the appendix have no zeroth moment) and
 * the total momentum of fluid and particles (Sec. 2: every force on a particle is returned to
 * the fluid, pair and bond forces act pairwise, the Shan-Chen forces cancel pairwise for
 * g_AB = g_BA).  With diag_every = K > 0, lbmd_step runs FP64 reductions on the device after
 * every step whose count is a multiple of K: M_A, M_B (sum of the populations) and the total
 * momentum P = sum_r j'(r) + sum_p m v_p, compared with the reference taken when the state was
 * last set (lbmd_init_fluid, lbmd_set_particles, lbmd_set_drift_reference).  The drifts are
 * |M_z - M_z,ref| / M_z,ref per component and |P - P_ref| / (M_A,ref + M_B,ref) (a velocity in
 * lattice units); when one exceeds drift_tol the device error word records it and the next
 * synchronising call returns LBMD_E_DRIFT (sticky, like the other device errors).  FP32 storage
 * drifts by about 1e-8 per step from rounding, so drift_tol is the caller's choice for its run
 * length and storage.  diag_every = 0 (the default) switches the check off; with diag_every > 0,
 * drift_tol must be finite and > 0.  The reductions read the populations once (152 B per site in
 * FP32): every K steps they cost about one density pass. */
typedef struct {
  int nx, ny, nz;
  double tau_r;
  double g_AB, g_BA;
  double kT;
  double dt;
  int storage;
  double rho0_A, rho0_B;
  uint64_t seed;
  int collision;
  double lambda_bulk, lambda_mom, lambda_ghost;
  int md_substeps;
  int diag_every;
  double drift_tol;
} lbmd_params;

/* Per particle type: kappa_A, kappa_B of Eq. (solvation_kappa), lambda_A, lambda_B of
 * Eq. (solvation_lambda), friction gamma of Eq. (NEWTON), mass. */
typedef struct {
  double kappa_A, kappa_B, lambda_A, lambda_B, gamma, mass;
} lbmd_ptype;

/* WCA pair parameters (Sec. 4.1): U = 4 eps [(sigma/r)^12 - (sigma/r)^6] for r < 2^(1/6) sigma. */
typedef struct {
  int type_i, type_j;
  double wca_eps, wca_sigma;
} lbmd_pair;

/* Create a context for an nx*ny*nz lattice on the current CUDA device.  stream: a
 * cudaStream_t (may be NULL).  Allocates both population buffers; fails with
 * LBMD_E_NOMEM if they do not fit.  *warnings (may be NULL) receives LBMD_WARN_* bits.
 * Errors: LBMD_E_INVALID_ARG for sizes < 1, tau_r <= 1/2, dt != 1, unknown storage,
 * negative rho0, unknown collision, an MRT eigenvalue outside (-2, 0), md_substeps outside
 * [1, 256], diag_every < 0, or diag_every > 0 with drift_tol not finite and > 0. */
int lbmd_create(const lbmd_params *params, void *stream, lbmd_ctx **out, unsigned *warnings);

/* Destroy a context and free its device memory (NULL is ignored). */
void lbmd_destroy(lbmd_ctx *ctx);

/* Particle types and WCA pairs.  ntypes in [1, LBMD_MAX_TYPES]; pairs not listed have no
 * WCA interaction; each listed pair applies to (i,j) and (j,i).  Copied before return. */
int lbmd_set_types(lbmd_ctx *ctx, int ntypes, const lbmd_ptype *types, int npairs,
                   const lbmd_pair *pairs, unsigned *warnings);

/* Screened Coulomb (Sec. 4.4): U = q_i q_j lB exp(-kappa_D r)/r for r < rc; lB = 0
 * switches it off.  rc must be below half the smallest box edge. */
int lbmd_set_debye_hueckel(lbmd_ctx *ctx, double lB, double kappa_D, double rc);

/* Initialise the fluid at equilibrium, f_zi = f^eq_i(rho_z, u) (Eq. feq), from host
 * arrays rhoA, rhoB [nz][ny][nx] (> 0) and u [nz][ny][nx][3] (NULL = at rest).  Resets
 * the step counter to 0. */
int lbmd_init_fluid(lbmd_ctx *ctx, const float *rhoA, const float *rhoB, const float *u);

/* Set / get the post-streaming populations of component comp (0 = A, 1 = B), host array
 * f [19][nz][ny][nx]. */
int lbmd_set_populations(lbmd_ctx *ctx, int comp, const float *f);
int lbmd_get_populations(lbmd_ctx *ctx, int comp, float *f);

/* Set the particles: n >= 0; x, v [n][3] doubles (positions wrapped into the box), type
 * [n] in [0, ntypes), q [n] charges (NULL = all zero).  Replaces all particles and bonds
 * stay as set (they refer to particle indices). */
int lbmd_set_particles(lbmd_ctx *ctx, int n, const double *x, const double *v, const int *type,
                       const double *q);

/* Bonds between particle indices pairs [nb][2]; kind LBMD_BOND_FENE (k, r = R0) or
 * LBMD_BOND_HARMONIC (k, r = d).  nb = 0 removes all bonds. */
int lbmd_set_bonds(lbmd_ctx *ctx, int nb, const int *pairs, int kind, double k, double r);

/* Advance nsteps >= 0 coupled steps (Sec. 2 and the appendix): Shan-Chen force, fluid-side
 * solvation force, coupling velocity, particle forces (friction + noise, solvation, WCA,
 * screened Coulomb, bonds), momentum return onto the 8 nodes of each particle's cell, BGK
 * collision with forcing and pull streaming for both components, particle update.
 * Asynchronous on the context stream; device errors surface at the next synchronising
 * call. */
int lbmd_step(lbmd_ctx *ctx, int nsteps);

/* Launch mode of lbmd_step (no counterpart in the paper: a property of the GPU code).  With
 * on != 0 (the default) lbmd_step takes its steps two at a time by replaying a CUDA graph of
 * two coupled steps, recorded at the first such call for the current buffers on a private
 * stream and launched into the context stream; an odd last step is launched directly.  The
 * results are bit-identical to on = 0, where every kernel is launched one by one; the graph
 * saves the launch latency that dominates small lattices.  The particle kernels read their noise
 * counter from a device-resident step base; the fluctuating MRT update gets its counter written
 * into its graph nodes before each replay (where those nodes are not recognised, the context
 * falls back to launches one by one).  Every setter (types, Debye-Hueckel,
 * fluid, populations, particles, bonds, profiling) drops the recorded graphs; recording
 * allocates nothing while it runs (the sub-stepping records are allocated first).  Returns
 * LBMD_E_INVALID_ARG for a NULL context; errors of recording surface at the next lbmd_step as
 * LBMD_E_CUDA. */
int lbmd_set_graphs(lbmd_ctx *ctx, int on);

/* How the lattice update reads the populations (no counterpart in the paper: a property of the
 * GPU code).  The Shan-Chen force of a node needs its neighbours' densities of the same step, so
 * the densities must exist before the update.  passes = 2: a density pass pulls every node's
 * populations and stores the densities, then the update pulls them again.  passes = 1: the
 * update of step t also forms the densities of step t + 1 from the values it has just computed
 * (streaming carries f*_i(r) to r + c_i, so the density of a node is the sum of what arrives
 * from its 19 sources); one short kernel finishes the nodes whose sources lie in another block
 * of the update (the x edges of each 32-column tile, the first and last row of each 8-row tile
 * and the first and last plane of each 16-plane chunk) by adding the partial sums the blocks
 * wrote -- or, on lattices too thin for them (tiles of 1-2 rows, one plane), by pulling their
 * populations -- and forms j' at the corners of the particles' cells for the next step's
 * coupling.  The one-pass update
 * reads the populations once per step instead of twice.  passes = 0 (the default) takes one
 * pass with FP32 storage on lattices of at least 16 x 152 x (blocks per SM) column-tile planes
 * (tiles of 32 x 8 columns: about 128^3 and up on 152 SMs), two passes otherwise (with 16-bit
 * storage the update is bound by instruction issue, not by the bytes the second pass reads).  Both give the
 * same step up to FP32 rounding order (the densities are sums in another order).  One pass
 * needs the BGK collision and md_substeps = 1 (else LBMD_E_INVALID_ARG for passes = 1).  Drops
 * the recorded graphs.  lbmd_get_lattice_passes returns the update the next step takes (1 or 2;
 * setting it up, the first time, allocates the partial-sum buffers) or a negative
 * LBMD_E_* code. */
int lbmd_set_lattice_passes(lbmd_ctx *ctx, int passes);
int lbmd_get_lattice_passes(lbmd_ctx *ctx);

/* Wait for the context stream; returns the first recorded device error, if any. */
int lbmd_sync(lbmd_ctx *ctx);
int lbmd_clear_error(lbmd_ctx *ctx);

/* Densities rhoA, rhoB [nz][ny][nx] and barycentric velocity u [nz][ny][nx][3]
 * (Eq. momentum_definition, u = (j' + g/2)/rho with the force of the last step's
 * collision) at the current step; any pointer may be NULL. */
int lbmd_get_fields(lbmd_ctx *ctx, float *rhoA, float *rhoB, float *u);

/* Particle positions x, velocities v and the total force f of the last step, each
 * [n][3] doubles in the caller's order; any pointer may be NULL. */
int lbmd_get_particles(lbmd_ctx *ctx, double *x, double *v, double *f);

/* Device-memory variants of the three getters above, for callers that keep the state on the
 * GPU (torch tensors, their own kernels): the same values in the same layouts -- rhoA, rhoB
 * [nz][ny][nx] and u [nz][ny][nx][3] FP32; f [19][nz][ny][nx] FP32 (the unshifted post-streaming
 * values of component comp); x, v, f [n][3] FP64 in the caller's particle order, n the count of
 * the last lbmd_set_particles -- written into caller-owned DEVICE buffers of the context's device,
 * with no copy through the host and no host synchronisation.  stream: a cudaStream_t of the caller
 * (NULL = the legacy default stream); the outputs are written after the context's queued steps and
 * after the work already queued on stream, and before any work queued on stream after the call
 * returns, so the caller may use them on stream at once.  Any output pointer may be NULL, except
 * f_dev of lbmd_get_populations_dev.  Each non-NULL pointer is checked before any launch: it must
 * be device (or managed) memory and, where the driver reports the allocation's extent, the stated
 * length from it must lie inside that allocation; otherwise LBMD_E_INVALID_ARG (nothing written).
 * A buffer carved from a larger allocation (a caching allocator's pool) is checked against that
 * whole allocation only: the caller must still pass buffers of the stated lengths.  These
 * calls do not synchronise, so device-side failures of earlier steps are reported by the next
 * call that does (lbmd_sync, the host getters, lbmd_diagnostics).  Errors: LBMD_E_INVALID_ARG,
 * LBMD_E_STATE (fluid not initialised), LBMD_E_CUDA.  The paper defines the fields (Sec. 2: the
 * densities, Eq. momentum_definition for u) but no interface to them. */
int lbmd_get_fields_dev(lbmd_ctx *ctx, float *rhoA_dev, float *rhoB_dev, float *u_dev, void *stream);
int lbmd_get_populations_dev(lbmd_ctx *ctx, int comp, float *f_dev, void *stream);
int lbmd_get_particles_dev(lbmd_ctx *ctx, double *x_dev, double *v_dev, double *f_dev, void *stream);

/* FP64 reductions on the device: out[0..1] = total mass of A and B, out[2..4] = fluid
 * momentum sum_r j'(r), out[5..7] = particle momentum sum m v. */
int lbmd_diagnostics(lbmd_ctx *ctx, double out[8]);

/* The FP64 drift check (lbmd_params.diag_every; appendix: mass; Sec. 2: momentum).
 * lbmd_set_drift_reference takes the current totals as the reference (enqueued on the context
 * stream; lbmd_init_fluid and lbmd_set_particles do the same when diag_every > 0,
 * lbmd_set_populations does not, so that a state changed by hand between steps is measured
 * against the run's start).
 * lbmd_get_drift synchronises and returns, for the last check, out[0] = its step count (-1: no
 * check yet), out[1], out[2] = the relative mass drift of A and B, out[3] = the momentum drift
 * per unit mass, out[4] = the number of checks since the reference was taken.  It does not
 * return LBMD_E_DRIFT itself (lbmd_sync does).  Errors: LBMD_E_INVALID_ARG, LBMD_E_STATE (fluid
 * not initialised), LBMD_E_CUDA. */
int lbmd_set_drift_reference(lbmd_ctx *ctx);
int lbmd_get_drift(lbmd_ctx *ctx, double out[5]);

/* Number of completed steps. */
int64_t lbmd_step_count(const lbmd_ctx *ctx);

/* Kernel timing of the lattice kernel: when enabled, lbmd_step brackets every launch of
 * the fused stream-collide kernel with CUDA events on the context stream;
 * lbmd_profile_read returns the summed milliseconds and the launch count since the last
 * reset (synchronises). */
int lbmd_profile_enable(lbmd_ctx *ctx, int on);
int lbmd_profile_read(lbmd_ctx *ctx, double *ms, int64_t *launches, int reset);

/* Number of kernel launches issued by lbmd_step so far (host-side count; a graph replay counts
 * the kernels it holds, the step counter's own one-thread kernels included). */
int64_t lbmd_launch_count(const lbmd_ctx *ctx);

/* Total mass of each component and fluid momentum -- the same FP64 sums as out[0..4] of
 * lbmd_diagnostics -- of a population array the caller already holds in device memory,
 * computed WITHOUT ALLOCATING any device memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- a serving loop that admits work
 * against a fixed device-memory budget and must not allocate once running, or code that runs
 * inside another framework that owns the device allocator.  The populations must already be in
 * the layout below (the host layout of lbmd_get_populations, FP32); the library's own
 * contexts keep theirs in another, internal layout and are not read by this call.
 *   f_dev    device pointer, FP32 [2][19][nz][ny][nx] (component A then B): 38 nx ny nz floats.
 *   out_dev  device pointer to 5 doubles: M_A, M_B, Px, Py, Pz.
 *   stream   cudaStream_t for both launches (NULL = legacy default stream); asynchronous.
 * Both pointers are checked before any launch: each must be device (or managed) memory and,
 * where the driver reports the allocation's extent, lie with its stated length inside one
 * allocation; otherwise LBMD_E_INVALID_ARG (no device access).
 * The per-block partial sums live in one file-scope static device array of 640 KiB
 * (16384 blocks x 5 doubles), which every GPU that loads the library holds until exit;
 * lattices above 2^27 sites (512^3) are rejected with LBMD_E_INVALID_ARG.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current, and so does the first call after the device's context was created again (after
 * cudaDeviceReset); make that first call before any stream capture.  Every call shares the
 * array: calls whose kernels overlap on the GPU (different streams, or different threads) race
 * on it and must be serialised by the caller.  Each call writes every partial it reads, so no
 * clearing is needed; the partials are summed in a fixed order (deterministic).  Errors:
 * LBMD_E_INVALID_ARG, LBMD_E_CUDA; lbmd_last_error(NULL) describes the last failure. */
int lbmd_fluid_moments_static(const float *f_dev, int nx, int ny, int nz, double *out_dev, void *stream);

/* Message of the last failure of ctx, or, if ctx is NULL, of the last failed call made without
 * a context (lbmd_create, lbmd_fluid_moments_static). */
const char *lbmd_last_error(const lbmd_ctx *ctx);

/* ==========================================================================================
 * Batches: many independent replicas (lattices with their particles, each with its own
 * parameters, sizes and step count) advanced together on one GPU.  Every kernel of the coupled
 * step runs once per step for all replicas of the batch (shared launches), the launches of a
 * step sequence are captured once in a CUDA graph, and replicas join and leave between calls
 * without recapture -- continuous batching.  A replica advances exactly as a context created
 * with lbmd_create would, and its results do not depend on the other replicas in the batch.
 *
 * Life cycle of a replica: lbmd_batch_add (admission: reserves its device memory against the
 * batch budget) -> lbmd_batch_set_types / lbmd_batch_set_debye_hueckel -> lbmd_batch_init_fluid
 * -> lbmd_batch_set_particles -> lbmd_batch_step (any number of calls, shared with the other
 * replicas) -> lbmd_batch_poll until its status is LBMD_SLOT_DONE -> getters ->
 * lbmd_batch_remove (frees its memory for the next replica).
 *
 * The paper defines the model of one system; batching, admission and the autotuner are not in
 * it.  Bonds (lbmd_set_bonds) are available in single contexts only.
 * ========================================================================================== */
typedef struct lbmd_batch lbmd_batch;

/* slot status reported by lbmd_batch_poll */
#define LBMD_SLOT_EMPTY 0  /* no replica */
#define LBMD_SLOT_ACTIVE 1 /* admitted, steps still to take (or fluid not initialised yet) */
#define LBMD_SLOT_DONE 2   /* took all the steps it asked for */
#define LBMD_SLOT_FAILED 3 /* stopped by a device error (lbmd_batch_slot_error gives the code) */

/* Create a batch on the current device.  mem_budget: bytes of device memory the replicas may
 * take (0 = 90 % of the free memory); storage: LBMD_STORAGE_* shared by every replica;
 * max_slots in [1, 65536]; stream: a cudaStream_t for all work of the batch, which must not be
 * the legacy default stream; NULL = the batch creates (and owns) a non-blocking stream.
 * Errors: LBMD_E_INVALID_ARG, LBMD_E_NOMEM, LBMD_E_CUDA (message: lbmd_batch_last_error(NULL)). */
int lbmd_batch_create(size_t mem_budget, int storage, int max_slots, void *stream, lbmd_batch **out);

/* Wait for the batch's work and free everything it holds (NULL is ignored). */
void lbmd_batch_destroy(lbmd_batch *batch);

/* Admit a replica: params as for lbmd_create (storage must be the batch's), np_max the most
 * particles it will hold, total_steps the steps it asks for.  Its device memory -- both
 * population buffers, densities, j', and its share of the particle and row arrays -- is
 * reserved against the budget; LBMD_E_NOMEM (nothing changed) when it does not fit or every
 * slot is taken: retry after lbmd_batch_remove.  *slot receives its slot index, *warnings
 * (may be NULL) LBMD_WARN_* bits.  The replica takes part in lbmd_batch_step once its fluid
 * is initialised. */
int lbmd_batch_add(lbmd_batch *batch, const lbmd_params *params, int np_max, int64_t total_steps, int *slot,
                   unsigned *warnings);

/* Free a replica's memory and slot (its results are gone; read them first). */
int lbmd_batch_remove(lbmd_batch *batch, int slot);

/* Per replica: as lbmd_set_types, lbmd_set_debye_hueckel, lbmd_init_fluid (resets the
 * replica's step count) and lbmd_set_particles (n <= np_max). */
int lbmd_batch_set_types(lbmd_batch *batch, int slot, int ntypes, const lbmd_ptype *types, int npairs,
                         const lbmd_pair *pairs, unsigned *warnings);
int lbmd_batch_set_debye_hueckel(lbmd_batch *batch, int slot, double lB, double kappa_D, double rc);
int lbmd_batch_init_fluid(lbmd_batch *batch, int slot, const float *rhoA, const float *rhoB, const float *u);
int lbmd_batch_set_particles(lbmd_batch *batch, int slot, int n, const double *x, const double *v,
                             const int *type, const double *q);

/* Advance every initialised replica by min(nsteps, steps it still asks for) coupled steps
 * (the step of lbmd_step), all replicas in the same launches.  Asynchronous on the batch
 * stream; a replica whose state fails on the device (negative or non-finite density, particle
 * out of range) stops at the end of that step while the others go on. */
int lbmd_batch_step(lbmd_batch *batch, int nsteps);

/* Wait for the batch's work; status (may be NULL) [max_slots] receives LBMD_SLOT_* per slot. */
int lbmd_batch_poll(lbmd_batch *batch, int *status);

/* LBMD_E_* code of a failed replica (LBMD_OK if none), and its step count, as of the last
 * call that waited for the batch (lbmd_batch_poll, getters); -1 / LBMD_E_INVALID_ARG for a
 * free slot. */
int lbmd_batch_slot_error(const lbmd_batch *batch, int slot);
int64_t lbmd_batch_step_count(const lbmd_batch *batch, int slot);

/* Per replica, as lbmd_get_populations, lbmd_get_fields, lbmd_get_particles and
 * lbmd_diagnostics (all wait for the batch stream). */
int lbmd_batch_get_populations(lbmd_batch *batch, int slot, int comp, float *f);
int lbmd_batch_get_fields(lbmd_batch *batch, int slot, float *rhoA, float *rhoB, float *u);
int lbmd_batch_get_particles(lbmd_batch *batch, int slot, double *x, double *v, double *f);
int lbmd_batch_diagnostics(lbmd_batch *batch, int slot, double out[8]);

/* The drift check of a replica whose lbmd_params.diag_every > 0, as lbmd_get_drift: out[5] = {step
 * of the last check (-1: none), mass drift of A, of B, momentum drift per unit mass, checks
 * since the reference}.  The reference is taken at the replica's first lbmd_batch_step after
 * lbmd_batch_init_fluid or lbmd_batch_set_particles; the check runs inside the step graphs after
 * every diag_every steps of the replica, and a drift beyond drift_tol stops the replica like any
 * device error (lbmd_batch_poll: LBMD_SLOT_FAILED; lbmd_batch_slot_error: LBMD_E_DRIFT).  Waits
 * for the batch stream.  Errors: LBMD_E_INVALID_ARG, LBMD_E_STATE (diag_every = 0). */
int lbmd_batch_get_drift(lbmd_batch *batch, int slot, double out[5]);

/* Launch shape of the two lattice kernels: the sites per tile (a multiple of 256 in
 * [256, 65536]), the persistent grid of the density pass and of the update (in [1, 64 x SM
 * count]), and the register budget of the update, collide_blocks = 3 (80 registers, three
 * blocks of 256 threads per SM) or 2 (up to 128 registers).  cfg[5] = {tile_sites,
 * grid_moments, grid_collide, collide_blocks, grid_particles}.  Results do not depend on it. */
int lbmd_batch_set_config(lbmd_batch *batch, int tile_sites, int grid_moments, int grid_collide,
                          int collide_blocks);
int lbmd_batch_get_config(const lbmd_batch *batch, int cfg[5]);

/* Autotuner: times the lattice kernels over the current replicas for tiles of 256, 1024 and
 * 4096 sites, density-pass grids of 2/3/4 blocks per SM and update variants (register budget
 * of 3 blocks per SM with grids of 1/2/3 blocks per SM, of 2 blocks per SM with 1/2), keeps
 * the fastest, and returns it in cfg[5] and the two kernel times in ms[2] (either may be
 * NULL).  The state of the replicas is unchanged.  Needs at least one initialised replica. */
int lbmd_batch_tune(lbmd_batch *batch, int cfg[5], double ms[2]);

/* Budget and use in bytes, number of occupied slots, slot count (any pointer may be NULL). */
int lbmd_batch_info(const lbmd_batch *batch, size_t *budget, size_t *used, int *occupied, int *max_slots);

/* Kernel launches issued by lbmd_batch_step so far (host-side count: 15 per step, 16 when the
 * batch holds replicas of both collisions; two more when a drift reference is taken). */
int64_t lbmd_batch_launch_count(const lbmd_batch *batch);

/* Message of the last failure of a batch call (NULL: of lbmd_batch_create). */
const char *lbmd_batch_last_error(const lbmd_batch *batch);

#ifdef __cplusplus
}
#endif
#endif /* LBMD_H */
