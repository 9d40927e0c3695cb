/*
 * FP64 CPU oracle for the per-particle Lagrangian step of a two-way coupled
 * Euler-Lagrange method (SCALE-TRACK, arXiv 2603.26691).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the plain, slow, scalar reference
 * that the CUDA path is checked against.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library, and the library
 * never calls it.
 *
 * What it computes (each function cites the passage it follows):
 *   - Newton's second law for a particle (Sec. 2.1, Eqs. 9-10) with Stokes
 *     drag (relaxation time tau = rho_p d^2 / (18 mu)) and gravity, advanced
 *     by the exponential integrator, which is exact while the fluid velocity
 *     seen by the particle is frozen over the step;
 *   - the fluid velocity at the particle by trilinear interpolation of
 *     cell-centred values on a periodic uniform grid (used here in place of
 *     the nearest-grid-point rule of Sec. 2.5);
 *   - the momentum given to the fluid, J = -m [(v' - v) - g dt], which is the
 *     drag part of d(m u_p)/dt in the momentum source of Sec. 2.1, Eq. 11,
 *     deposited whole into the cell that holds the particle (Sec. 2.5) at the
 *     start of the step;
 *   - the chunk-major ordering key and a stable sort of particles by it
 *     (chunks organised as structures of arrays, Sec. 2.2);
 *   - global invariants (particle count, momentum, summed source, mass);
 *   - the hand-derived adjoint of the step for a loss on the time-summed
 *     source field;
 *   - droplet microphysics (Sec. 2.1): vapour mass transfer to or from a
 *     droplet and its heat balance with the latent heat, and the vapour-mass
 *     and energy sources they give the fluid;
 *   - the asynchronous two-way coupling of Sec. 2.3 on one device: the
 *     particles advance in a frozen fluid field while the fluid is updated
 *     from the sources of the previous coupling interval, estimated by the
 *     extrapolator-corrector method of Sec. 2.4 (Eqs. 12-14); the fluid
 *     update is an explicit momentum source followed by Jacobi sweeps of an
 *     implicit periodic diffusion step.
 *
 * Physics variants, selected in orc_grid: the nearest-grid-point gather and
 * semi-implicit Euler integrator the paper itself uses (Sec. 2.5), the
 * Schiller-Naumann drag correlation it cites (Sec. 2.1), and a cloud-in-cell
 * deposit (the transpose of the trilinear gather).  Pinned in
 * tests/test_physics_pins.py.
 *
 * Pins (tests/test_oracle_pins.py): closed-form and ODE-integrated
 * uniform-flow solutions, terminal velocity, exact reproduction of
 * trilinear functions, the momentum balance, brute-force deposit and sort
 * checks on tiny inputs, and central finite differences for the adjoint.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC.
 */
#ifndef SCALETRACK_ORACLE_H
#define SCALETRACK_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Grid, box and physical parameters.  Field and source arrays index cells
 * linearly as c = i + nx * (j + ny * k). */
typedef struct {
  int32_t n[3];        /* cells along x, y, z */
  int32_t chunk_edge;  /* B: cells per chunk edge (power of two) */
  double L[3];         /* periodic box lengths */
  double rho_p;        /* particle material density */
  double mu;           /* fluid dynamic viscosity */
  double g[3];         /* gravitational acceleration */
  double alpha;        /* drag scale multiplying the Stokes drag */
  double mult;         /* parcel multiplicity w (particles per parcel) */
  /* Physics variants (all 0 = trilinear gather, exponential integrator, Stokes drag, deposit
   * into the containing cell at the start of the step). */
  int32_t gather;      /* 0 trilinear on cell centres; 1 nearest grid point (Sec. 2.5) */
  int32_t integrator;  /* 0 exponential; 1 semi-implicit Euler (Sec. 2.5) */
  int32_t drag;        /* 0 Stokes; 1 Schiller-Naumann correlation (Sec. 2.1) */
  int32_t deposit;     /* 0 containing cell; 1 cloud-in-cell (transpose of the trilinear gather) */
  double rho_f;        /* fluid density in the particle Reynolds number (Schiller-Naumann only) */
} orc_grid;

/* Periodic wrap of one coordinate into [0, L). */
double orc_wrap(double x, double L);

/* Cell index (i, j, k) of a wrapped position. */
void orc_cell(const orc_grid* G, const double x[3], int32_t idx[3]);

/* The fluid velocity seen at x: trilinear interpolation of the cell-centred
 * field U[c][3], or (gather = 1) the value of the cell that holds x. */
void orc_gather(const orc_grid* G, const double* U, const double x[3], double up[3]);

/* Drag factor f = C_D Re / 24 of the Schiller-Naumann correlation at
 * particle Reynolds number Re (1 for Stokes drag at any Re). */
double orc_drag_factor(const orc_grid* G, double re);

/* One step of a particle of diameter d that sees the frozen fluid velocity
 * up: updates v and x in place (x not wrapped), by the exponential
 * integrator or (integrator = 1) semi-implicit Euler, with the drag factor
 * evaluated from the relative velocity at the start of the step. */
void orc_advance(const orc_grid* G, double d, const double up[3], double dt,
                 double x[3], double v[3]);

/* Add the impulse J of a particle at x (its start-of-step position) to
 * src[3][ncell]: whole into the cell that holds x, or (deposit = 1) spread
 * over the eight cells of its trilinear stencil with the gather's weights. */
void orc_deposit(const orc_grid* G, const double x[3], const double J[3], double* src);

/* Particle mass (parcel multiplicity included). */
double orc_mass(const orc_grid* G, double d);

/* One full step of one particle: start cell c0 (linear), gather, advance,
 * wrap, and the impulse J given to the fluid. */
void orc_particle_step(const orc_grid* G, const double* U, double dt, double d,
                       double x[3], double v[3], int64_t* c0, double J[3]);

/* nsteps steps of n particles (SoA pos[3][n], vel[3][n]) in the frozen field U.
 * Adds each step's impulses into src[3][ncell] in step-major, particle-index
 * order.  If trace != NULL it records the deposit cell of every particle and
 * step (trace[s*n + p]); if frozen != NULL the deposit cells are taken from
 * it instead of being computed (finite differences with the cell sequence
 * held fixed).  trace and frozen concern the containing-cell deposit; with
 * the cloud-in-cell deposit frozen must be NULL.  Returns 0, or -1 on bad
 * arguments. */
int orc_run(const orc_grid* G, const double* U, int64_t n, double* pos, double* vel,
            const double* d, int32_t nsteps, double dt, double* src,
            int64_t* trace, const int64_t* frozen);

/* Chunk-major ordering key of cell (i, j, k): chunk index (x fastest) times
 * B^3 plus the Morton (bit-interleaved, x lowest) index inside the chunk. */
uint32_t orc_key(const orc_grid* G, int32_t i, int32_t j, int32_t k);

/* Stable sort permutation: perm[r] = index of the r-th particle in key
 * order, ties kept in index order. */
void orc_sort_perm(int64_t n, const uint32_t* keys, int64_t* perm);

/* Particles per cell (counts[ncell]) for the wrapped positions pos[3][n]. */
void orc_cell_counts(const orc_grid* G, int64_t n, const double* pos, int64_t* counts);

/* Invariants: out = {count, P_x, P_y, P_z, sumJ_x, sumJ_y, sumJ_z, sum m}
 * with P = sum_p m_p v_p and sumJ = sum over cells of the source. */
void orc_invariants(const orc_grid* G, int64_t n, const double* vel, const double* d,
                    const double* src, double out[8]);

/* Adjoint of orc_run for a loss L(Jtot) with Jtot the time-summed source:
 * given lam[3][ncell] = dL/dJtot, returns dL/dd_p, dL/dalpha and
 * dL/dU (gradU[c][3], same layout as U).  With the containing-cell deposit
 * the deposit cells are treated as locally constant (the derivative that
 * exists almost everywhere); with the cloud-in-cell deposit the deposit
 * weights are differentiated as well (they are continuous in the position).
 * The forward trajectory is stored whole (no checkpointing).  pos0/vel0 are
 * not modified.  Trilinear gather, exponential integrator and Stokes drag
 * only, with either deposit.  Returns 0, -1 on bad arguments or other
 * physics, -2 on allocation failure. */
int orc_adjoint(const orc_grid* G, const double* U, int64_t n, const double* pos0,
                const double* vel0, const double* d, int32_t nsteps, double dt,
                const double* lam, double* grad_d, double* grad_alpha, double* gradU);

/* Bounding boxes of the chunks (Sec. 2.2): a chunk is the set of particles whose
 * cell, at the time of the last ordering (pos_sort[3][n]), lies in its B^3 block
 * of cells (numbered x fastest, as in orc_key); its box is the min and max of
 * the current positions pos_now[3][n], each unwrapped to the periodic image
 * nearest the chunk's centre.  out[chunk][6] = {xmin, ymin, zmin, xmax, ymax,
 * zmax}; an empty chunk gets {+inf, +inf, +inf, -inf, -inf, -inf}.  Returns
 * the number of chunks, or -1 on bad arguments. */
int64_t orc_chunk_bounds(const orc_grid* G, int64_t n, const double* pos_sort, const double* pos_now,
                         double* out);

/* Extrapolator-corrector estimate of the source of coupling interval n
 * (Sec. 2.4, Eqs. 12-14): S_est^n = S^{n-1} - S_ext^{n-1} + S_ext^n, where
 * S_ext^m extrapolates S^m from the sources before it: extrap 0 = zero (0),
 * 1 = constant (S^{m-1}), 2 = linear (2 S^{m-1} - S^{m-2}).  Reading: the
 * corrector removes the extrapolated part of the previous estimate; removing
 * the whole previous estimate, as printed, is not conservative over time.
 * s1, s2, s3 = S^{n-1}, S^{n-2}, S^{n-3} (NULL for an interval before the
 * first); m values each. */
void orc_ecm_estimate(int32_t extrap, int64_t m, const double* s1, const double* s2,
                      const double* s3, double* out);

/* Fluid update of one coupling interval of length dtc: u* = U + S / (rho_f V)
 * in every cell (S[3][ncell], the impulse given to the fluid; V the cell
 * volume), then `sweeps` Jacobi sweeps of the implicit diffusion step
 * (I - nu dtc Lap) u = u* with the 7-point periodic Laplacian, starting from
 * u*.  U[c][3] is updated in place.  Returns 0, or -1 / -2 on bad arguments
 * or allocation failure. */
int orc_fluid_update(const orc_grid* G, double* U, const double* S, double rho_f, double nu,
                     double dtc, int32_t sweeps);

/* Asynchronous two-way coupling (Sec. 2.3) of nint intervals of K particle
 * steps of dt: in interval n the particles advance K steps in the frozen
 * field u^n and deposit S^n, while the fluid becomes
 * u^{n+1} = F(u^n, S_est^n) (orc_fluid_update with the estimate of
 * orc_ecm_estimate, which uses only S^{n-1}, S^{n-2}, S^{n-3}).  U, pos and
 * vel are updated in place.  pending[3][ncell] receives the sources
 * deposited but not yet given to the fluid, S^{N-1} - S_ext^{N-1}, so that
 * particle momentum + fluid momentum + pending - gravity impulse is
 * conserved.  Returns 0, -1 on bad arguments, -2 on allocation failure. */
int orc_couple(const orc_grid* G, double* U, int64_t n, double* pos, double* vel, const double* d,
               int32_t nint, int32_t K, double dt, double rho_f, double nu, int32_t sweeps,
               int32_t extrap, double* pending);

/* Droplet microphysics parameters (Sec. 2.1). */
typedef struct {
  double D_v;      /* diffusivity of water vapour in the fluid (m^2/s) */
  double kappa_f;  /* thermal conductivity of the fluid (W/(m K)) */
  double cp_p;     /* specific heat capacity of the droplet (J/(kg K)) */
  double L;        /* latent heat of vaporization of water (J/kg) */
  double Pr;       /* Prandtl number of the fluid (Nusselt correlation) */
  double d_min;    /* diameter an evaporating droplet keeps at least (m) */
} orc_micro;

/* Saturation vapour density over flat water at T (K), kg/m^3 (Magnus form,
 * Alduchov-Eskridge coefficients, ideal gas with R_v = 461.5 J/(kg K)). */
double orc_rho_sat(double T);

/* d rho_sat / dT at T (K), from the same form. */
double orc_rho_sat_dT(double T);

/* Nusselt number (Ranz-Marshall: 2 + 0.6 Re^(1/2) Pr^(1/3)). */
double orc_nusselt(const orc_micro* M, double re);

/* One step of one droplet with motion, vapour mass transfer and heat transfer
 * (Sec. 2.1): x, v, d, Tp updated in place; c0 the start-of-step cell; J, dmass
 * and denergy the momentum, vapour mass and energy the fluid gains.  The step
 * is documented at its definition in oracle.c. */
void orc_micro_particle_step(const orc_grid* G, const orc_micro* M, const double* U, const double* Tf,
                             const double* rhov, double dt, double x[3], double v[3], double* d, double* Tp,
                             int64_t* c0, double J[3], double* dmass, double* denergy);

/* nsteps steps of n droplets with microphysics in the frozen fields U[c][3],
 * Tf[c] (K) and rhov[c] (kg/m^3); pos, vel, d and Tp updated in place; the
 * fluid's gains added, step-major in particle-index order, into src[3][ncell]
 * (momentum), msrc[ncell] (vapour mass) and esrc[ncell] (energy), each into
 * the start-of-step cell (any may be NULL).  The cell deposit only.  Returns
 * 0, or -1 on bad arguments. */
int orc_micro_run(const orc_grid* G, const orc_micro* M, const double* U, const double* Tf, const double* rhov,
                  int64_t n, double* pos, double* vel, double* d, double* Tp, int32_t nsteps, double dt,
                  double* src, double* msrc, double* esrc);

#ifdef __cplusplus
}
#endif
#endif
