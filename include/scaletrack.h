/*
 * scaletrack.h - C ABI of the GB300 (sm_103a) per-particle Lagrangian step of a
 * two-way coupled Euler-Lagrange method (SCALE-TRACK, arXiv 2603.26691).
 *
 * The library advances point particles through a frozen, cell-centred fluid
 * velocity field on a periodic uniform grid and returns the momentum they
 * exchanged with the fluid as per-cell sources.  This follows the paper's
 * statement of the coupling problem (Sec. 2.5): the Lagrangian code is given
 * the domain geometry, the mesh and the Eulerian fields, and gives back
 * source terms.  One step of one particle:
 *   1. gather the fluid velocity u_p by trilinear interpolation of the
 *      cell-centred field (in place of the nearest-grid-point rule of
 *      Sec. 2.5);
 *   2. advance Newton's law (Sec. 2.1, Eqs. 9-10) under Stokes drag with
 *      relaxation time tau = rho_p d^2 / (18 mu), scaled by drag_scale, and
 *      gravity, with the exponential integrator (exact for frozen u_p):
 *        a = drag_scale / tau, w = u_p + g / a,
 *        v' = w + (v - w) e^{-a dt},
 *        x' = x + w dt + (v - w) (1 - e^{-a dt}) / a;
 *   3. wrap x' into the periodic box and relocate the particle to its new
 *      cell and chunk;
 *   4. deposit J = -m [(v' - v) - g dt] (the drag part of d(m u_p)/dt in the
 *      momentum source, Sec. 2.1 Eq. 11, with the sign of a gain for the
 *      fluid) whole into the cell that held the particle at the start of the
 *      step (Sec. 2.5).
 * Particles are kept as structures of arrays (Sec. 2.2) and reordered
 * periodically by a stable counting sort on a chunk-major key.
 *
 * Conventions for every call:
 *   - Every call returns st_status; nothing throws across the ABI.  After an
 *     error, st_last_error(h) gives a message; the handle stays usable
 *     unless the status is ST_ERR_CUDA from an asynchronous fault.
 *   - Pointers passed in are borrowed for the duration of the call only.
 *     Output buffers belong to the caller.  `on_device` = 1 means the
 *     pointer is CUDA device memory on the handle's device, 0 means host
 *     memory (pageable or pinned).
 *   - Work is ordered on the caller's CUDA stream (st_create_grid).  Calls
 *     that return data to the caller (st_get_*, st_invariants,
 *     st_num_particles) synchronise that stream; st_step, st_reorder,
 *     st_set_fluid and st_add_particles from device memory do not.
 *   - Cells are numbered c = i + nx * (j + ny * k).  Per-cell arrays of three
 *     components are component-major: out[q * ncell + c].  Particle arrays of
 *     three components are component-major too: xyz[q * count + p].
 *   - Fluid fields are cell-centred (centre of cell (i,j,k) at
 *     ((i + 1/2) h_x, (j + 1/2) h_y, (k + 1/2) h_z)), laid out u[k][j][i][3].
 */
#ifndef SCALETRACK_H
#define SCALETRACK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct st_ctx* st_handle;

/* Device-memory provider.  alloc returns device memory of at least `bytes`
 * bytes aligned to 256 bytes, or NULL; free releases it.  Both are called
 * from the thread that calls into the library; memory is used on the
 * handle's stream.  A NULL st_allocator pointer selects cudaMalloc/cudaFree. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} st_allocator;

typedef enum {
  ST_OK = 0,
  ST_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
  ST_ERR_OOM = 2,         /* the allocator returned NULL */
  ST_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  ST_ERR_STATE = 4,       /* call not valid in the handle's current state */
  ST_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  ST_ERR_NONFINITE = 6,   /* a field value, particle value or parameter is NaN/Inf */
  ST_ERR_OVERFLOW = 7     /* the source accumulator's range would be exceeded */
} st_status;

/* Storage and arithmetic of the particle state. */
typedef enum {
  ST_FP64 = 0,       /* x, y, z, u, v, w, d as FP64 (56 bytes per particle) */
  ST_MIXED_F32 = 1,  /* int32 cell + FP32 in-cell offset, FP32 velocity, FP32 d (32 B) */
  ST_MIXED_BF16V = 2 /* as ST_MIXED_F32 with the velocity stored in BF16 (26 B) */
} st_precision;

enum { ST_DTYPE_F32 = 0, ST_DTYPE_F64 = 1 };

/* Create a simulation on the current CUDA device: an nx x ny x nz periodic
 * grid over the box [0,Lx) x [0,Ly) x [0,Lz) (Sec. 2.5: the mesh and
 * geometry the Lagrangian solver needs).  chunk_edge B (power of two,
 * 1..32) sets the chunk of B^3 cells used as the major part of the ordering
 * key (chunks as particle-set partitions stored as structures of arrays,
 * Sec. 2.2).  1 <= n* <= 1024.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream).  Parameters start as rho_p = 1000, mu = 1.8e-5,
 * g = (0, 0, -9.81), drag_scale = 1, multiplicity = 1, reorder_every = 10.
 * The fluid starts at rest.  Errors: INVALID_ARG, OOM, CUDA. */
st_status st_create_grid(int nx, int ny, int nz, double Lx, double Ly, double Lz, int chunk_edge,
                         int precision, const st_allocator* allocator, void* stream, st_handle* out);

/* Release everything the handle owns.  Safe on NULL. */
void st_destroy(st_handle h);

/* Message for the last error on this handle ("" if none).  The string
 * belongs to the handle and lives until the next call on it. */
const char* st_last_error(st_handle h);

/* Change the CUDA stream later calls are ordered on. */
st_status st_set_stream(st_handle h, void* stream);

/* Wait for all work the handle has queued, the asynchronous transfers
 * (st_set_fluid_async, st_get_sources_async) included, and report pending
 * errors. */
st_status st_synchronize(st_handle h);

/* Physical parameters (Sec. 2.1): particle density rho_p > 0, fluid dynamic
 * viscosity mu > 0, gravity g[3], drag_scale alpha > 0 multiplying the
 * Stokes drag, parcel multiplicity w > 0 (particles lumped per parcel,
 * Sec. 3.2; it multiplies the mass in the source), and reorder_every K
 * (counting sort every K steps and before the first step; 0 = only on
 * st_reorder).  Errors: INVALID_ARG, NONFINITE. */
st_status st_set_params(st_handle h, double rho_p, double mu, const double g[3], double drag_scale,
                        double multiplicity, int reorder_every);

/* Physics variants.  The defaults (all 0) are the step described at the top
 * of this file.  The alternatives are the choices the paper itself makes:
 *   ST_GATHER_NGP: nearest grid point (Sec. 2.5) - the particle takes the
 *     value of the cell it is in;
 *   ST_INTEGRATOR_SEMI_IMPLICIT: semi-implicit Euler (Sec. 2.5), drag
 *     implicit in the new velocity and the position advanced with it,
 *       v' = (v + dt (a u_p + g)) / (1 + a dt),  x' = x + dt v';
 *   ST_DRAG_SCHILLER_NAUMANN: the drag correlation cited in Sec. 2.1,
 *     a = drag_scale f(Re) / tau with f = C_D Re / 24 = 1 + 0.15 Re^0.687
 *     for Re <= 1000 and 0.44 Re / 24 above, Re = rho_f |u_p - v| d / mu
 *     from the velocities at the start of the step (held over the step);
 *   ST_DEPOSIT_CIC: cloud in cell - J spread over the eight cells of the
 *     particle's trilinear stencil at the start of the step, with the
 *     trilinear weights (the transpose of the trilinear gather).
 * rho_f > 0 is the fluid density used in Re (only read by the
 * Schiller-Naumann drag).  Every combination runs on the sorted-particle
 * step kernel of mixed handles (a separate instance of it; the defaults keep
 * their own) and on the general kernels.  The adjoint (st_adjoint_*) needs
 * the default gather, integrator and drag, with either deposit.
 * Errors: INVALID_ARG, NONFINITE. */
enum { ST_GATHER_TRILINEAR = 0, ST_GATHER_NGP = 1 };
enum { ST_INTEGRATOR_EXPONENTIAL = 0, ST_INTEGRATOR_SEMI_IMPLICIT = 1 };
enum { ST_DRAG_STOKES = 0, ST_DRAG_SCHILLER_NAUMANN = 1 };
enum { ST_DEPOSIT_CELL = 0, ST_DEPOSIT_CIC = 1 };
st_status st_set_physics(st_handle h, int gather, int integrator, int drag, int deposit, double rho_f);

/* Copy in the cell-centred fluid velocity u[k][j][i][3] (dtype
 * ST_DTYPE_F32 or ST_DTYPE_F64) - the Eulerian state of Sec. 2.3 that the
 * Lagrangian step reads.  FP64 handles keep it in FP64, mixed handles in
 * FP32.  Errors: INVALID_ARG, NONFINITE (any NaN/Inf), CUDA. */
st_status st_set_fluid(st_handle h, const void* u, int dtype, int on_device);

/* Make room for `capacity` particles in total (optional; st_add_particles
 * grows geometrically otherwise).  Errors: INVALID_ARG, OOM. */
st_status st_reserve(st_handle h, int64_t capacity);

/* Append n particles (the Lagrangian phase's point particles of Sec. 2.1, each
 * with position, velocity and diameter; multiplicity and density come from
 * st_set_params): positions xyz[3][n] (any real values; wrapped into
 * the box), velocities vel[3][n] (NULL = at rest), diameters d[n] > 0,
 * optional ids[n] (NULL = consecutive from the number already held).  The
 * FP64 values are converted to the handle's storage.  The new particles
 * are unsorted until the next reorder.  Errors: INVALID_ARG (d <= 0),
 * NONFINITE, OOM, CUDA. */
st_status st_add_particles(st_handle h, int64_t n, const double* xyz, const double* vel,
                           const double* d, const uint32_t* ids, int on_device);

/* Number of particles held. */
st_status st_num_particles(st_handle h, int64_t* n);

/* Advance all particles nsteps steps of length dt > 0 through the current
 * fluid field (the fixed sub-steps per Eulerian step of Sec. 3.3), adding
 * each step's impulses to the per-cell source accumulator.  Runs the
 * counting sort first when it is due.  On mixed handles the step just before
 * a due sort writes the new state as 32-byte particle records for that
 * sort's gather; any other call that reads or changes the particles turns
 * them back first, so this is not visible through the ABI.  Asynchronous on
 * the stream.  Errors: INVALID_ARG, STATE (no fluid set), OVERFLOW, CUDA. */
st_status st_step(st_handle h, int nsteps, double dt);

/* Read the accumulated per-cell source: out[3][ncell] in FP64, the raw
 * impulse given to the fluid in each cell (kg m/s) summed over every step
 * since the last reset.  The momentum-source density of Sec. 2.1 Eq. 11 is
 * out / (V_cell * T) over the accumulation time T.  The accumulator is
 * exact fixed point (see the design notes), so the result does not depend
 * on thread scheduling.  reset = 1 clears it afterwards.  Synchronises.
 * Errors: INVALID_ARG, CUDA. */
st_status st_get_sources(st_handle h, double* out, int reset, int on_device);

/* The accumulated source as the exact fixed-point integers it is kept in:
 * words[3][ncell][4] (int64; component-major like st_get_sources) with
 * digits words[..][0..2] in [0, 2^32) below a signed top word [3], value =
 * sum_k words[k] 2^(32 k - E) kg m/s.  For summing several handles' sources
 * (for instance one per GPU) exactly and in no particular order: shift each
 * to the largest E and add the integers.  The carries are propagated in
 * place first (the accumulated value does not change).  Synchronises.
 * Errors: INVALID_ARG, CUDA. */
st_status st_get_sources_fixed(st_handle h, int64_t* words, int* E, int on_device);

/* Asynchronous host transfers, so that a loop of field in, step, sources
 * out keeps the GPU computing while data crosses the host link (the paper's
 * coupling, Sec. 2.3, overlaps the transfers with the particle step).  The
 * handle owns an upload and a download stream beside its compute stream and
 * a staging buffer for one field and two source fields (allocated at the
 * first call; freed by st_destroy).
 *
 * st_set_fluid_async: like st_set_fluid from host memory u (dtype as
 * there; pinned memory for the copy to overlap), but it returns once the
 * copy is queued.  The new field takes effect for the work queued after
 * this call (steps already queued keep the previous one).  The host must
 * leave u unchanged until the next call on the handle other than
 * st_get_sources_async, which waits for the copy and reads its scan: a
 * field with NaN or Inf is not taken and that call returns NONFINITE.
 *
 * st_get_sources_async: like st_get_sources to host memory out (pinned for
 * the copy to overlap), reset as there, but it returns once the conversion
 * and the copy are queued; out holds the sources after st_synchronize,
 * which waits for the compute, upload and download streams and reports any
 * pending error (NONFINITE from an upload, TIMEOUT from a device-side
 * wait).  Two staging buffers alternate, so two calls may be in flight; out
 * must stay valid and unread until then.
 *
 * In a loop of steps, queue the next step's field (st_set_fluid_async)
 * before this step's sources (st_get_sources_async): the upload then runs
 * beside the step instead of waiting behind the sources' download where the
 * two directions share a copy engine.
 * Errors: INVALID_ARG, NONFINITE, OOM, CUDA. */
st_status st_set_fluid_async(st_handle h, const void* u, int dtype);
st_status st_get_sources_async(st_handle h, double* out, int reset);

/* Stable counting sort of the particles now, by the chunk-major key of
 * their cell: chunk index (x fastest) times B^3 plus the Morton index of
 * the cell inside its chunk.  Particles with equal keys keep their order.
 * This keeps each chunk's particles together in the structure of arrays, the
 * spatially coherent particle sets of Sec. 2.2 (here chunks are blocks of
 * cells rather than the paper's redistributed particle sets).
 * Asynchronous.  Errors: OOM, CUDA. */
st_status st_reorder(st_handle h);

/* Copy out particles [first, first + count) in the current storage order:
 * absolute positions xyz[3][count] reconstructed in FP64 (mixed handles:
 * x = (i + offset) h), velocities vel[3][count], diameters d[count], ids.
 * Any output pointer may be NULL.  Synchronises.  Errors: INVALID_ARG, CUDA. */
st_status st_get_particles(st_handle h, int64_t first, int64_t count, double* xyz, double* vel,
                           double* d, uint32_t* ids, int on_device);

/* Cell index of particles [first, first + count) as int32 linear cell
 * numbers c = i + nx (j + ny k).  Synchronises. */
st_status st_get_cells(st_handle h, int64_t first, int64_t count, int32_t* cells, int on_device);

/* Particles per cell, counts[ncell], as of the last reorder (after a
 * reorder the particles of cell c occupy a contiguous range of the storage
 * order).  Errors: STATE if never sorted.  Synchronises. */
st_status st_get_cell_counts(st_handle h, int64_t* counts, int on_device);

/* Bounding boxes of the chunks (Sec. 2.2): a chunk is the set of particles in
 * the key range of its B^3 block of cells as of the last reorder, and its box
 * is the min and max of their current positions, each unwrapped to the
 * periodic image nearest the chunk's centre.  out[chunk][6] FP64 = {xmin,
 * ymin, zmin, xmax, ymax, zmax}, chunks numbered x fastest (the major part of
 * the ordering key); an empty chunk gets +inf for the minima and -inf for the
 * maxima.  Synchronises the handle's stream.  Errors: INVALID_ARG, STATE (not
 * sorted since particles were added or cleared), OOM, CUDA. */
st_status st_chunk_bounds(st_handle h, double* out, int on_device);

/* Global invariants in FP64: out = {particle count, P_x, P_y, P_z, S_x, S_y,
 * S_z, M} with P = sum_p m_p v_p, S = sum over cells of the accumulated
 * source and M = sum_p m_p.  With no fluid forcing beyond drag,
 * P(T) - P(0) - M g T + S = 0.  Synchronises. */
st_status st_invariants(st_handle h, double out[8]);

/* Remove all particles (the fluid, parameters and accumulated sources stay). */
st_status st_clear_particles(st_handle h);

/* Forward run for differentiation: advance all particles nsteps steps of
 * length dt (no reordering during the run), adding the impulses to the source
 * accumulator as st_step does, and keep checkpoints of positions and
 * velocities every checkpoint_every steps (FP64 handles: 6 x n x 8 bytes
 * each; mixed FP32-velocity handles: the cells, offsets and velocities, 28 x n
 * bytes, n rounded up to 64, stepped by the general mixed kernel in storage
 * order).  With Jtot the time-summed per-cell source, st_adjoint_backward then
 * returns the gradient of any loss L(Jtot).  The method has no adjoint in the
 * paper; this differentiates the step of Sec. 2.1 (Eqs. 9-11) as implemented
 * here: with the cell deposit the deposit cell is held fixed (its derivative
 * is zero almost everywhere); with the cloud-in-cell deposit (st_set_physics,
 * FP64 handles) its trilinear weights are differentiated as well.  The
 * trilinear gather, the exponential integrator and Stokes drag only.  On
 * mixed handles the adjoint runs in FP32 (see st_adjoint_backward).
 * Changing particles, parameters, the physics or the fluid, or reordering,
 * invalidates the recorded run.
 * Errors: STATE (BF16-velocity handle, microphysics on, other physics, the
 * cloud-in-cell deposit on a mixed handle, no particles), INVALID_ARG,
 * NONFINITE, OOM, CUDA. */
st_status st_adjoint_forward(st_handle h, int nsteps, double dt, int checkpoint_every);

/* Reverse sweep of the last st_adjoint_forward run, segment by segment from
 * the last checkpoint, recomputing each segment's states forward first.
 * lam[3][ncell] = dL/dJtot (host or device, lam_on_device).  Outputs (any may
 * be NULL; host or device per on_device): grad_d[n] = dL/dd per particle in
 * the current storage order, *grad_alpha = dL/d(drag_scale) (host pointer
 * always), grad_U[ncell][3] = dL/dU in the layout of st_set_fluid.  All sums
 * are formed in a fixed order or in exact fixed point, so results are
 * bit-reproducible.  Mixed handles: the reverse step runs in FP32 (lam
 * rounded to FP32, FP32 adjoints of position and velocity, each step's
 * dL/dd and dL/d(drag_scale) terms accumulated in FP64; the FP32 dL/dU
 * terms of particles in one warp that share a trilinear stencil summed in
 * FP32 in an order fixed by the stencils, each sum added exactly).
 * Synchronises.
 * Errors: STATE (no recorded run), INVALID_ARG, OOM, CUDA. */
st_status st_adjoint_backward(st_handle h, const double* lam, int lam_on_device, double* grad_d,
                              double* grad_alpha, double* grad_U, int on_device);

/* Two-way coupling parameters (Sec. 2.3 and 2.4): fluid density rho_f > 0
 * (kg/m^3, the cell's fluid mass is rho_f V), kinematic viscosity nu >= 0 of
 * the implicit diffusion step, Jacobi sweeps per interval (>= 0), particle
 * steps per coupling interval K (>= 1), and the extrapolator of the
 * extrapolator-corrector estimate (Eqs. 12-14): 0 zero, 1 constant, 2 linear.
 * Defaults: 1.2, 1e-3, 10, 5, 0.  Errors: INVALID_ARG, NONFINITE. */
st_status st_couple_params(st_handle h, double rho_f, double nu, int sweeps, int steps_per_interval,
                           int extrapolator);

/* Run nintervals coupling intervals of the asynchronous two-way coupling
 * (Sec. 2.3) on this GPU.  In interval n the particles take K steps of dt in
 * the frozen current field u^n (as st_step); the next field, computed from
 * u^n and the sources of earlier intervals only, is u* = u^n + S_est^n /
 * (rho_f V) per cell, then the Jacobi sweeps of (I - nu K dt Lap) u = u*
 * (7-point periodic Laplacian, from u*).  Both run on the handle's stream,
 * the fluid update ahead of the interval's steps: the lag of one interval
 * (the asynchrony of Sec. 2.3) is in the data, not in the scheduling.  S_est^n = S^{n-1} - S_ext^{n-1} + S_ext^n is the
 * estimate of the interval's source from the sources of earlier intervals
 * (reading of Sec. 2.4: the corrector removes the previous extrapolated part,
 * which keeps the fluid's total intake equal to the particles' output up to
 * the last, pending, interval).  At the interval's end the particles' source
 * S^n leaves the accumulator (so st_get_sources reads only what later
 * st_step calls deposit) and the new field becomes current.  The first
 * interval after st_set_fluid has no source history.  Returns once the last
 * interval's fluid update has finished; its particle steps may still run.
 * Errors: INVALID_ARG (nintervals < 0, dt <= 0), NONFINITE, STATE (no
 * fluid), OOM, CUDA, TIMEOUT. */
st_status st_couple_run(st_handle h, int nintervals, double dt);

/* The current fluid field as FP64 out[k][j][i][3] (the layout of st_set_fluid;
 * device or host pointer per on_device; synchronises the handle's stream).
 * Errors: INVALID_ARG, OOM, CUDA. */
st_status st_get_fluid(st_handle h, double* out, int on_device);

/* Sources given by the particles but not yet received by the fluid,
 * out[3][ncell] FP64: S^{N-1} - S_ext^{N-1} of the last coupling interval
 * plus what the accumulator holds now, so that particle momentum + rho_f V
 * sum(u) + sum(pending) - gravity impulse is conserved.  Synchronises the
 * handle's stream.  Errors: INVALID_ARG, OOM, CUDA. */
st_status st_get_pending_sources(st_handle h, double* out, int on_device);

/* Number of CUDA kernels this handle has launched since it was created (a
 * diagnostic for profiling: every kernel of the library counts once per
 * launch). */
st_status st_kernel_launches(st_handle h, int64_t* count);

/* Seeded synthetic particles (an input generator, not part of the method):
 * particles first .. first+count-1 of the counter-based SplitMix64 stream
 * `seed`, written as FP64 device arrays xyz[3][count], vel[3][count]
 * (uniform in [-vmax, vmax) per component, or zero when vmax == 0),
 * d[count] (inverse-transform sampled from qtable[nq + 1], a device array
 * of quantiles) and ids[count] = index.  The same definition is implemented
 * on the host by the package's input module.  Any output may be NULL.
 * Asynchronous.  Errors: INVALID_ARG, CUDA. */
st_status st_gen_particles(st_handle h, uint64_t seed, int64_t first, int64_t count, const double L[3],
                           double vmax, const double* qtable, int nq, double* xyz, double* vel, double* d,
                           uint32_t* ids);

/* Droplet microphysics (Sec. 2.1): each droplet also exchanges water vapour
 * and heat with the fluid,
 *   dm/dt = 2 pi D_v d rho_sat(T_f) (S_f - S_p),  S_f = rho_v / rho_sat(T_f),
 *           S_p = rho_sat(Tp) / rho_sat(T_f) (flat water at the droplet's
 *           temperature), i.e. dm/dt = 2 pi D_v d (rho_v - rho_sat(Tp));
 *   m C_p dTp/dt = pi Nu kappa_f d (T_f - Tp) + L dm/dt (the latent heat of
 *           condensed water warms the droplet, evaporation cools it; the
 *           paper prints the opposite sign, which would heat an evaporating
 *           droplet), Nu = 2 + 0.6 Re^(1/2) Pr^(1/3) (Ranz-Marshall) with
 *           Re = rho_f |u_p - v| d / mu;
 * and the fluid gains, in the cell that held the droplet at the start of the
 * step, the momentum -[(m' v' - m v) - m g dt] (Eq. 11 with the fluid's sign;
 * it reduces to the step's impulse when no mass moves), the vapour mass
 * -(m' - m) (the vapour source S_rho_v times V dt) and the energy
 * -C_p (m' Tp' - m Tp) (the energy source S_e times V dt).  rho_sat is the
 * saturation vapour density over flat water (Magnus form with the
 * Alduchov-Eskridge coefficients, over R_v T, R_v = 461.5 J/(kg K)).  Over a
 * step the droplet's diameter, slip and gathered fluid values are held,
 * rho_sat is linearised about the start temperature, the resulting linear
 * heat balance is solved exactly and the d^2 law (d(d^2)/dt = 8 D_v (rho_v -
 * rho_sat(Tp)) / rho_p) is integrated along that temperature path; a droplet
 * that would shrink below d_min keeps d_min.  Masses include the parcel
 * multiplicity; rho_p and the multiplicity come from st_set_params, rho_f
 * from st_set_physics.
 *
 * enable = 1 turns it on with vapour diffusivity D_v >= 0 (m^2/s), fluid
 * thermal conductivity kappa_f > 0 (W/(m K)), droplet specific heat cp_p > 0
 * (J/(kg K)), latent heat >= 0 (J/kg), Prandtl number > 0, d_min > 0 (m),
 * and T_init > 0 (K), the temperature of particles that have none yet (all
 * particles the first time, later additions every time); enable = 0 turns it
 * off (temperatures are kept).  While it is on, st_step runs the
 * microphysics step (FP64 or mixed handles; the default gather, integrator,
 * drag and deposit only, else ST_ERR_STATE; the fluid temperature and vapour
 * fields must be set).  The particle state adds a temperature (8 B FP64,
 * 4 B mixed) and the diameter is written every step.
 * Errors: INVALID_ARG, NONFINITE, OOM, CUDA. */
st_status st_set_microphysics(st_handle h, int enable, double D_v, double kappa_f, double cp_p, double latent_heat,
                              double prandtl, double d_min, double T_init);

/* The fluid temperature T[c] (K, > 0) and water vapour density rho_v[c]
 * (kg/m^3, >= 0) at cell centres, in the cell order of st_set_fluid (dtype
 * ST_DTYPE_F32 or ST_DTYPE_F64), gathered by the step like the velocity.
 * Copied in.  Errors: INVALID_ARG, NONFINITE, OOM, CUDA. */
st_status st_set_thermo(st_handle h, const void* T, const void* rho_v, int dtype, int on_device);

/* Particle temperatures (K) of particles [first, first + count) in the
 * current storage order: set from T[count] (microphysics on), or copied out
 * (synchronises).  Errors: STATE (microphysics never enabled), INVALID_ARG,
 * NONFINITE, OOM, CUDA. */
st_status st_set_temperatures(st_handle h, int64_t first, int64_t count, const double* T, int on_device);
st_status st_get_temperatures(st_handle h, int64_t first, int64_t count, double* T, int on_device);

/* What the fluid gained from the droplets' mass and heat transfer since the
 * last reset, out[2][ncell] FP64: the vapour mass (kg) and the energy (J) per
 * cell (the vapour and energy sources of Sec. 2.1 times V and the elapsed
 * time).  Summed exactly (carry-save integers), so the result does not
 * depend on thread scheduling.  reset = 1 clears them afterwards.
 * Synchronises.  Errors: INVALID_ARG, OOM, CUDA. */
st_status st_get_micro_sources(st_handle h, double* out, int reset, int on_device);

/* out = {sum_p m_p, sum_p C_p m_p Tp} in FP64 over the particles (for the
 * water and energy budgets: with the sources of st_get_micro_sources, mass +
 * vapour gained and C_p m T + energy gained stay constant).  Synchronises. */
st_status st_micro_invariants(st_handle h, double out[2]);

/* Chunked particle sets (Sec. 2.2: a GPU computes one chunk after another and
 * hides the transfer of a finished chunk behind the next one's computation),
 * for particle sets larger than device memory.  st_chunks_create turns the
 * handle (no resident particles) into one that keeps its particles as chunks
 * of chunk_particles (rounded up to a multiple of 64) in pinned host memory,
 * in the handle's own storage form (32 B per particle mixed, 56 B FP64, plus
 * a 4 B id), with three device slots of that capacity.  st_chunks_add appends
 * n particles (xyz[3][n], vel[3][n] or NULL, d[n]; ids continue from the
 * number already held) as ceil(n / C) new chunks, the last one possibly not
 * full.  st_chunks_step advances every particle nsteps steps of dt: chunk by
 * chunk in order, each copied in, sorted and stepped as resident particles
 * are (sorting every reorder_every steps), and copied back, with the copies of
 * the next and the previous chunk overlapping the computation on a second
 * stream; the sources go into the handle's accumulator (st_get_sources).
 * Positions and velocities equal those of the same particles stepped
 * resident; the sources equal a resident run's up to the FP32 rounding of the
 * run sums (their grouping depends on the storage order).  ms (NULL or 4
 * doubles) receives the wall time of the pass and the summed times of the
 * computations, uploads and downloads (CUDA events), which show the overlap.
 * st_chunks_get copies particles [first, first + count) of the chunks'
 * storage order to host arrays (positions in FP64 as st_get_particles).
 * st_chunks_count gives the particle and chunk counts.  While a handle holds
 * chunks, st_add_particles, st_reserve and enabling the microphysics are
 * refused (STATE) and st_step sees no particles.
 * Synchronous.  Errors: STATE, INVALID_ARG, OOM (device slots or pinned host
 * memory), CUDA. */
st_status st_chunks_create(st_handle h, int64_t chunk_particles);
st_status st_chunks_add(st_handle h, int64_t n, const double* xyz, const double* vel, const double* d, int on_device);
st_status st_chunks_step(st_handle h, int nsteps, double dt, double* ms);
st_status st_chunks_get(st_handle h, int64_t first, int64_t count, double* xyz, double* vel, double* d,
                        uint32_t* ids);
st_status st_chunks_count(st_handle h, int64_t* particles, int64_t* chunks);

/* Largest n that st_sort_keys_static accepts. */
#define ST_SORT_KEYS_STATIC_MAX_N (1 << 20)

/* Stable sort of n device keys for callers that cannot allocate device memory
 * (code running inside another framework's memory pool or arena, a process
 * whose allocations are made once at start-up and then frozen, or an
 * allocator callback that must not call back into the allocator).  The paper
 * has no counterpart; this is the ordering sort of st_reorder offered without
 * a handle and without allocation.
 *
 * Keys are compared on their low key_bits bits (1..32); equal keys keep their
 * input order.  Writes sorted_keys[n] (the input keys in sorted order) and
 * perm[n] (perm[r] = input index of the r-th key).  keys, sorted_keys and perm
 * are device pointers owned by the caller; keys is not modified; the outputs
 * must not overlap keys or each other.  Work is queued on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and the call returns without
 * waiting.
 *
 * All scratch memory is one static device array of 8.5 MiB; the call makes no
 * cudaMalloc, cudaFree or other allocating call.  Under CUDA's default lazy
 * module loading the array is created on a device when the library's sort
 * module is first used there (the first sort-related call on that device, by
 * this entry point or by a handle), so that first call may take device memory;
 * from then on the array lives on that device until the process exits and
 * later calls take no device memory.  n must not exceed
 * ST_SORT_KEYS_STATIC_MAX_N (2^20): larger n returns ST_ERR_INVALID_ARG
 * without doing any work.  The first call on a device looks up the array's
 * device address for that device; make that first call before any CUDA stream
 * capture.  Every call uses the same array, which keeps the previous call's
 * contents (its look-back words start zeroed with the module and afterwards
 * carry only earlier calls' tags; when the 30-bit tags would repeat, after
 * 2^27 calls on a device, the call clears them first), so calls whose work
 * overlaps on the GPU (other streams, other threads) race with each other:
 * order them on one stream or synchronise between them.  Its waits on other
 * thread blocks give up after one second; the call cannot report that (the
 * work runs after it returns), the output is then wrong, and
 * st_sort_keys_static_status reports it afterwards.
 * Errors: INVALID_ARG (n < 0, n > 2^20, key_bits outside 1..32, NULL pointer
 * with n > 0), CUDA. */
st_status st_sort_keys_static(const uint32_t* keys, int64_t n, int key_bits, uint32_t* sorted_keys,
                              uint32_t* perm, void* stream);

/* Whether a wait of an st_sort_keys_static call on the current device gave up
 * (its output is then wrong) since the last query.  Synchronises `stream`
 * (the stream the sorts were queued on; their work must have finished), reads
 * the flag the waits set in the static scratch array, and clears it.  Makes no
 * allocation.  Returns ST_OK, ST_ERR_TIMEOUT (a wait gave up) or ST_ERR_CUDA. */
st_status st_sort_keys_static_status(void* stream);

/* Kernel timers: CUDA events recorded around the library's own launches, on the stream each runs
 * on, summed per kind.  ST_TIMER_STEP: every particle step kernel (st_step, the adjoint's forward
 * steps and recomputation); ST_TIMER_SORT: a whole reorder (all of its kernels);
 * ST_TIMER_ADJOINT: the adjoint step kernel of st_adjoint_backward; ST_TIMER_FLUID: the coupled
 * fluid update of st_couple_run.  st_timers_enable(h, 1) clears and starts
 * recording, 0 stops it.  st_timers_read synchronises, writes the summed milliseconds and the
 * number of timed launches per kind (arrays of ST_TIMER_COUNT), and clears them if `reset`.
 * Recording costs two events per timed launch.  Errors: INVALID_ARG, CUDA. */
enum { ST_TIMER_STEP = 0, ST_TIMER_SORT = 1, ST_TIMER_ADJOINT = 2, ST_TIMER_FLUID = 3, ST_TIMER_COUNT = 4 };
st_status st_timers_enable(st_handle h, int on);
st_status st_timers_read(st_handle h, double* ms, int64_t* launches, int reset);

/* The FP64 and FP32 fused multiply-add rates of this GPU, in GFLOP/s (2 flops per FMA),
 * measured by short kernels of independent FMA chains with no memory traffic (about 0.1 s):
 * the peak that the FP64 step and the adjoint, which are bound by FP64 arithmetic, are
 * reported against.  Synchronises.  Errors: INVALID_ARG, OOM, CUDA. */
st_status st_probe_fma(st_handle h, double* fp64_gflops, double* fp32_gflops);

#ifdef __cplusplus
}
#endif
#endif
