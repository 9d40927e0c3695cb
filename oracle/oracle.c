/*
 * FP64 CPU oracle: plain scalar implementation of the per-particle
 * Lagrangian step.  TEST INFRASTRUCTURE ONLY (see oracle.h for the scope,
 * the citations and the pins).  Everything is double precision, evaluated in
 * the order written, with no fused multiply-add (built with
 * -ffp-contract=off).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double kPi = 3.14159265358979323846;

static double cell_size(const orc_grid* G, int ax) { return G->L[ax] / (double)G->n[ax]; }

static int64_t ncell_of(const orc_grid* G) {
  return (int64_t)G->n[0] * (int64_t)G->n[1] * (int64_t)G->n[2];
}

static int64_t linear_cell(const orc_grid* G, int32_t i, int32_t j, int32_t k) {
  return (int64_t)i + (int64_t)G->n[0] * ((int64_t)j + (int64_t)G->n[1] * (int64_t)k);
}

/* Periodic box: positions live in [0, L).  x - L floor(x / L) is the
 * periodic image; the two guards catch the cases where rounding lands the
 * result just outside [0, L). */
double orc_wrap(double x, double L) {
  double y = x - L * floor(x / L);
  if (y < 0.0) y = y + L;
  if (y >= L) y = 0.0;
  return y;
}

/* The cell holding a particle (Sec. 2.5: sources go to the cell containing
 * the particle): i = floor(x / h), clamped to the last cell. */
void orc_cell(const orc_grid* G, const double x[3], int32_t idx[3]) {
  for (int ax = 0; ax < 3; ++ax) {
    double h = cell_size(G, ax);
    int32_t i = (int32_t)floor(x[ax] / h);
    if (i < 0) i = 0;
    if (i > G->n[ax] - 1) i = G->n[ax] - 1;
    idx[ax] = i;
  }
}

static int32_t wrap_index(int32_t i, int32_t n) {
  int32_t r = i % n;
  return r < 0 ? r + n : r;
}

/* Trilinear interpolation of cell-centred values (centres at (i + 1/2) h):
 * s = x / h - 1/2, i0 = floor(s), f = s - i0; the value is the sum over the
 * eight corners (i0 + di, j0 + dj, k0 + dk), indices taken periodically, of
 * the corner value times prod over axes of (f if the offset is 1 else 1 - f).
 * The stencil (corner cells and weights) is shared with the cloud-in-cell
 * deposit, which is this map transposed. */
static void trilinear_stencil(const orc_grid* G, const double x[3], int64_t cells[8], double w[8]) {
  int32_t i0[3];
  double f[3];
  for (int ax = 0; ax < 3; ++ax) {
    double s = x[ax] / cell_size(G, ax) - 0.5;
    double fl = floor(s);
    i0[ax] = (int32_t)fl;
    f[ax] = s - fl;
  }
  int c = 0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        w[c] = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
        cells[c] = linear_cell(G, wrap_index(i0[0] + di, G->n[0]), wrap_index(i0[1] + dj, G->n[1]),
                               wrap_index(i0[2] + dk, G->n[2]));
        c = c + 1;
      }
}

/* Nearest grid point (Sec. 2.5): the particle takes the value of the cell it
 * is in. */
void orc_gather(const orc_grid* G, const double* U, const double x[3], double up[3]) {
  if (G->gather == 1) {
    int32_t idx[3];
    orc_cell(G, x, idx);
    int64_t c = linear_cell(G, idx[0], idx[1], idx[2]);
    for (int q = 0; q < 3; ++q) up[q] = U[3 * c + q];
    return;
  }
  int64_t cells[8];
  double w[8];
  trilinear_stencil(G, x, cells, w);
  up[0] = up[1] = up[2] = 0.0;
  for (int c = 0; c < 8; ++c)
    for (int q = 0; q < 3; ++q) up[q] = up[q] + w[c] * U[3 * cells[c] + q];
}

/* Drag correlation of Schiller and Naumann (cited in Sec. 2.1):
 *   C_D = 24 / Re (1 + 0.15 Re^0.687) for Re <= 1000, C_D = 0.44 above,
 * with the drag force 1/2 rho_f C_D (pi d^2 / 4) |u - v| (u - v).  Divided by
 * the mass rho_p pi d^3 / 6 this is (18 mu / (rho_p d^2)) (C_D Re / 24)
 * (u - v), i.e. Stokes drag times f = C_D Re / 24. */
double orc_drag_factor(const orc_grid* G, double re) {
  if (G->drag != 1) return 1.0;
  if (re <= 0.0) return 1.0;
  double cd = re <= 1000.0 ? 24.0 / re * (1.0 + 0.15 * pow(re, 0.687)) : 0.44;
  return cd * re / 24.0;
}

/* Newton's second law (Sec. 2.1, Eqs. 9-10) with drag and gravity:
 *   dx/dt = v,  dv/dt = alpha f (u_p - v) / tau + g,  tau = rho_p d^2 / (18 mu),
 * f the drag factor from the relative velocity at the start of the step
 * (Re = rho_f |u_p - v| d / mu), held over the step with u_p.
 * Exponential integrator: with a = alpha f / tau the solution is exact,
 *   w_t = u_p + g / a            (the velocity v relaxes towards)
 *   v'  = w_t + (v - w_t) e^{-a dt}
 *   x'  = x + w_t dt + (v - w_t) (1 - e^{-a dt}) / a
 * and 1 - e^{-a dt} is taken as -expm1(-a dt).
 * Semi-implicit Euler (Sec. 2.5): the drag implicit in the new velocity, the
 * position advanced with it,
 *   v'  = (v + dt (a u_p + g)) / (1 + a dt),   x' = x + dt v'. */
void orc_advance(const orc_grid* G, double d, const double up[3], double dt, double x[3],
                 double v[3]) {
  double tau = G->rho_p * d * d / (18.0 * G->mu);
  double f = 1.0;
  if (G->drag == 1) {
    double r0 = up[0] - v[0], r1 = up[1] - v[1], r2 = up[2] - v[2];
    double re = G->rho_f * sqrt(r0 * r0 + r1 * r1 + r2 * r2) * d / G->mu;
    f = orc_drag_factor(G, re);
  }
  double a = G->alpha * f / tau;
  if (G->integrator == 1) {
    for (int ax = 0; ax < 3; ++ax) {
      double vn = (v[ax] + dt * (a * up[ax] + G->g[ax])) / (1.0 + a * dt);
      x[ax] = x[ax] + dt * vn;
      v[ax] = vn;
    }
    return;
  }
  double E = exp(-a * dt);
  double E1 = -expm1(-a * dt);
  for (int ax = 0; ax < 3; ++ax) {
    double wt = up[ax] + G->g[ax] / a;
    double vn = wt + (v[ax] - wt) * E;
    double dx = wt * dt + (v[ax] - wt) * (E1 / a);
    x[ax] = x[ax] + dx;
    v[ax] = vn;
  }
}

/* Deposit of one particle's impulse: the cell containing the particle at the
 * start of the step (Sec. 2.5), or the eight cells of its trilinear stencil
 * with the gather's weights (cloud in cell). */
void orc_deposit(const orc_grid* G, const double x[3], const double J[3], double* src) {
  int64_t nc = ncell_of(G);
  if (G->deposit == 1) {
    int64_t cells[8];
    double w[8];
    trilinear_stencil(G, x, cells, w);
    for (int c = 0; c < 8; ++c)
      for (int ax = 0; ax < 3; ++ax) src[ax * nc + cells[c]] = src[ax * nc + cells[c]] + w[c] * J[ax];
    return;
  }
  int32_t idx[3];
  orc_cell(G, x, idx);
  int64_t c0 = linear_cell(G, idx[0], idx[1], idx[2]);
  for (int ax = 0; ax < 3; ++ax) src[ax * nc + c0] = src[ax * nc + c0] + J[ax];
}

/* Mass of a spherical particle, times the parcel multiplicity (Sec. 3.2
 * lumps identical droplets into parcels). */
double orc_mass(const orc_grid* G, double d) {
  return G->mult * G->rho_p * kPi * d * d * d / 6.0;
}

/* One step of one particle.  The impulse given to the fluid is the drag
 * part of the particle's momentum change (Sec. 2.1, Eq. 11, with the sign
 * that enters the fluid's momentum equation Eq. 2 as +S_u):
 *   J = -m [(v' - v) - g dt],
 * computed from the stored v' and v, and deposited into the start-of-step
 * cell c0. */
void orc_particle_step(const orc_grid* G, const double* U, double dt, double d, double x[3],
                       double v[3], int64_t* c0, double J[3]) {
  int32_t idx[3];
  double up[3], vold[3];
  orc_cell(G, x, idx);
  *c0 = linear_cell(G, idx[0], idx[1], idx[2]);
  orc_gather(G, U, x, up);
  vold[0] = v[0];
  vold[1] = v[1];
  vold[2] = v[2];
  orc_advance(G, d, up, dt, x, v);
  for (int ax = 0; ax < 3; ++ax) x[ax] = orc_wrap(x[ax], G->L[ax]);
  double m = orc_mass(G, d);
  for (int ax = 0; ax < 3; ++ax) J[ax] = -m * ((v[ax] - vold[ax]) - G->g[ax] * dt);
}

static int grid_ok(const orc_grid* G) {
  for (int ax = 0; ax < 3; ++ax) {
    if (G->n[ax] <= 0 || !(G->L[ax] > 0.0)) return 0;
  }
  if (G->gather < 0 || G->gather > 1 || G->integrator < 0 || G->integrator > 1 || G->drag < 0 ||
      G->drag > 1 || G->deposit < 0 || G->deposit > 1 || !(G->rho_f >= 0.0))
    return 0;
  return G->rho_p > 0.0 && G->mu > 0.0 && G->alpha > 0.0;
}

int orc_run(const orc_grid* G, const double* U, int64_t n, double* pos, double* vel,
            const double* d, int32_t nsteps, double dt, double* src, int64_t* trace,
            const int64_t* frozen) {
  if (!grid_ok(G) || n < 0 || nsteps < 0) return -1;
  if (frozen && G->deposit != 0) return -1;
  int64_t nc = ncell_of(G);
  for (int32_t s = 0; s < nsteps; ++s) {
    for (int64_t p = 0; p < n; ++p) {
      double x[3] = {pos[p], pos[n + p], pos[2 * n + p]};
      double v[3] = {vel[p], vel[n + p], vel[2 * n + p]};
      int64_t c0;
      double J[3];
      orc_particle_step(G, U, dt, d[p], x, v, &c0, J);
      if (frozen) c0 = frozen[(int64_t)s * n + p];
      if (trace) trace[(int64_t)s * n + p] = c0;
      if (src && G->deposit == 1) {
        double x0[3] = {pos[p], pos[n + p], pos[2 * n + p]};
        orc_deposit(G, x0, J, src);
      } else if (src) {
        for (int ax = 0; ax < 3; ++ax) src[ax * nc + c0] = src[ax * nc + c0] + J[ax];
      }
      pos[p] = x[0];
      pos[n + p] = x[1];
      pos[2 * n + p] = x[2];
      vel[p] = v[0];
      vel[n + p] = v[1];
      vel[2 * n + p] = v[2];
    }
  }
  return 0;
}

/* Chunk-major key: chunks are B^3 blocks of cells numbered x-fastest; inside
 * a chunk the cell's local coordinates are bit-interleaved (bit b of the
 * local x, y, z goes to bit 3b, 3b+1, 3b+2). */
uint32_t orc_key(const orc_grid* G, int32_t i, int32_t j, int32_t k) {
  int32_t B = G->chunk_edge;
  int32_t ncx = (G->n[0] + B - 1) / B;
  int32_t ncy = (G->n[1] + B - 1) / B;
  uint32_t chunk = (uint32_t)(i / B) + (uint32_t)ncx * ((uint32_t)(j / B) + (uint32_t)ncy * (uint32_t)(k / B));
  uint32_t li = (uint32_t)(i % B), lj = (uint32_t)(j % B), lk = (uint32_t)(k % B);
  uint32_t morton = 0;
  for (int b = 0; (1 << b) < B; ++b) {
    morton |= ((li >> b) & 1u) << (3 * b);
    morton |= ((lj >> b) & 1u) << (3 * b + 1);
    morton |= ((lk >> b) & 1u) << (3 * b + 2);
  }
  return chunk * (uint32_t)(B * B * B) + morton;
}

typedef struct {
  uint32_t key;
  int64_t idx;
} key_idx;

/* Ordering on (key, original index): sorting by it with any sort is a
 * stable sort by key. */
static int cmp_key_idx(const void* a, const void* b) {
  const key_idx* x = (const key_idx*)a;
  const key_idx* y = (const key_idx*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

void orc_sort_perm(int64_t n, const uint32_t* keys, int64_t* perm) {
  if (n <= 0) return;
  key_idx* t = (key_idx*)malloc((size_t)n * sizeof(key_idx));
  if (!t) return;
  for (int64_t p = 0; p < n; ++p) {
    t[p].key = keys[p];
    t[p].idx = p;
  }
  qsort(t, (size_t)n, sizeof(key_idx), cmp_key_idx);
  for (int64_t r = 0; r < n; ++r) perm[r] = t[r].idx;
  free(t);
}

void orc_cell_counts(const orc_grid* G, int64_t n, const double* pos, int64_t* counts) {
  int64_t nc = ncell_of(G);
  for (int64_t c = 0; c < nc; ++c) counts[c] = 0;
  for (int64_t p = 0; p < n; ++p) {
    double x[3] = {pos[p], pos[n + p], pos[2 * n + p]};
    int32_t idx[3];
    orc_cell(G, x, idx);
    counts[linear_cell(G, idx[0], idx[1], idx[2])] += 1;
  }
}

void orc_invariants(const orc_grid* G, int64_t n, const double* vel, const double* d,
                    const double* src, double out[8]) {
  int64_t nc = ncell_of(G);
  for (int q = 0; q < 8; ++q) out[q] = 0.0;
  out[0] = (double)n;
  for (int64_t p = 0; p < n; ++p) {
    double m = orc_mass(G, d[p]);
    out[1] = out[1] + m * vel[p];
    out[2] = out[2] + m * vel[n + p];
    out[3] = out[3] + m * vel[2 * n + p];
    out[7] = out[7] + m;
  }
  if (src) {
    for (int ax = 0; ax < 3; ++ax)
      for (int64_t c = 0; c < nc; ++c) out[4 + ax] = out[4 + ax] + src[ax * nc + c];
  }
}

/* Reverse-mode derivative of orc_run.  Per particle and step (forward):
 *   c0 = cell(x);  u_p = sum_corners W(f) U;  a = 18 mu alpha / (rho_p d^2)
 *   E = e^{-a dt};  E1 = 1 - E;  Q = E1 / a;  w_t = u_p + g / a
 *   v' = w_t E1 + v E;  x' = x + w_t (dt - Q) + v Q
 *   J = -m (v' - v - g dt),  m = mult rho_p pi d^3 / 6;  Jtot[c0] += J.
 * The backward sweep runs the chain rule through these lines in reverse,
 * with lam[c0] as the adjoint of J.  The periodic wrap is a translation
 * (derivative one) and the deposit cell is held fixed. */
int orc_adjoint(const orc_grid* G, const double* U, int64_t n, const double* pos0,
                const double* vel0, const double* d, int32_t nsteps, double dt,
                const double* lam, double* grad_d, double* grad_alpha, double* gradU) {
  /* the default physics, or the default physics with the cloud-in-cell deposit */
  const int cic = G->deposit == 1;
  if (!grid_ok(G) || G->gather != 0 || G->integrator != 0 || G->drag != 0 || G->deposit > 1 || n < 0 ||
      nsteps < 0)
    return -1;
  int64_t nc = ncell_of(G);
  for (int64_t c = 0; c < 3 * nc; ++c) gradU[c] = 0.0;
  *grad_alpha = 0.0;
  size_t per = (size_t)(nsteps > 0 ? nsteps : 1);
  double* tx = (double*)malloc(per * 3 * sizeof(double));
  double* tv = (double*)malloc(per * 3 * sizeof(double));
  int64_t* tc = (int64_t*)malloc(per * sizeof(int64_t));
  if (!tx || !tv || !tc) {
    free(tx);
    free(tv);
    free(tc);
    return -2;
  }
  for (int64_t p = 0; p < n; ++p) {
    /* forward sweep of this particle, storing the start-of-step states */
    double x[3] = {pos0[p], pos0[n + p], pos0[2 * n + p]};
    double v[3] = {vel0[p], vel0[n + p], vel0[2 * n + p]};
    for (int32_t s = 0; s < nsteps; ++s) {
      for (int ax = 0; ax < 3; ++ax) {
        tx[3 * s + ax] = x[ax];
        tv[3 * s + ax] = v[ax];
      }
      int64_t c0;
      double J[3];
      orc_particle_step(G, U, dt, d[p], x, v, &c0, J);
      tc[s] = c0;
    }
    /* backward sweep */
    double dp = d[p];
    double tau = G->rho_p * dp * dp / (18.0 * G->mu);
    double a = G->alpha / tau;
    double E = exp(-a * dt);
    double E1 = -expm1(-a * dt);
    double Q = E1 / a;
    double m = orc_mass(G, dp);
    double xb[3] = {0.0, 0.0, 0.0}; /* adjoint of the position after step s */
    double vb[3] = {0.0, 0.0, 0.0}; /* adjoint of the velocity after step s */
    double db = 0.0;
    double alphab = 0.0;
    for (int32_t s = nsteps - 1; s >= 0; --s) {
      const double* xs = &tx[3 * s];
      const double* vs = &tv[3 * s];
      /* recompute the step's intermediates */
      int32_t i0[3];
      double f[3], h[3];
      for (int ax = 0; ax < 3; ++ax) {
        h[ax] = cell_size(G, ax);
        double sx = xs[ax] / h[ax] - 0.5;
        double fl = floor(sx);
        i0[ax] = (int32_t)fl;
        f[ax] = sx - fl;
      }
      double up[3];
      orc_gather(G, U, xs, up);
      double wt[3], vn[3];
      for (int ax = 0; ax < 3; ++ax) {
        wt[ax] = up[ax] + G->g[ax] / a;
        vn[ax] = wt[ax] + (vs[ax] - wt[ax]) * E;
      }
      double Jb[3];
      double fdep[3] = {0.0, 0.0, 0.0}; /* derivative of lam . (deposit) in the stencil fractions */
      if (cic) {
        /* J spread with the trilinear weights of the start position: its adjoint is the weighted
         * sum of lam over the eight cells, and the weights' derivatives give lam . J terms */
        double J[3];
        for (int ax = 0; ax < 3; ++ax) J[ax] = -m * (vn[ax] - vs[ax] - G->g[ax] * dt);
        Jb[0] = Jb[1] = Jb[2] = 0.0;
        for (int dk = 0; dk < 2; ++dk)
          for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
              double wx = di ? f[0] : 1.0 - f[0];
              double wy = dj ? f[1] : 1.0 - f[1];
              double wz = dk ? f[2] : 1.0 - f[2];
              double w = wx * wy * wz;
              int64_t c = linear_cell(G, wrap_index(i0[0] + di, G->n[0]),
                                      wrap_index(i0[1] + dj, G->n[1]), wrap_index(i0[2] + dk, G->n[2]));
              double lj = 0.0;
              for (int q = 0; q < 3; ++q) {
                Jb[q] = Jb[q] + w * lam[q * nc + c];
                lj = lj + lam[q * nc + c] * J[q];
              }
              fdep[0] = fdep[0] + (di ? 1.0 : -1.0) * wy * wz * lj;
              fdep[1] = fdep[1] + wx * (dj ? 1.0 : -1.0) * wz * lj;
              fdep[2] = fdep[2] + wx * wy * (dk ? 1.0 : -1.0) * lj;
            }
      } else {
        int64_t c0 = tc[s];
        Jb[0] = lam[c0];
        Jb[1] = lam[nc + c0];
        Jb[2] = lam[2 * nc + c0];
      }
      /* J = -m (v' - v - g dt) */
      double mb = 0.0;
      double vnb[3], vsb[3];
      for (int ax = 0; ax < 3; ++ax) {
        vnb[ax] = vb[ax] - m * Jb[ax];
        vsb[ax] = m * Jb[ax];
        mb = mb - (vn[ax] - vs[ax] - G->g[ax] * dt) * Jb[ax];
      }
      /* v' = w_t E1 + v E ;  x' = x + w_t (dt - Q) + v Q */
      double wtb[3], ub[3];
      double Eb = 0.0, E1b = 0.0, Qb = 0.0, ab = 0.0;
      double xsb[3];
      for (int ax = 0; ax < 3; ++ax) {
        wtb[ax] = vnb[ax] * E1 + xb[ax] * (dt - Q);
        vsb[ax] = vsb[ax] + vnb[ax] * E + xb[ax] * Q;
        E1b = E1b + vnb[ax] * wt[ax];
        Eb = Eb + vnb[ax] * vs[ax];
        Qb = Qb + xb[ax] * (vs[ax] - wt[ax]);
        xsb[ax] = xb[ax];
        /* w_t = u_p + g / a */
        ub[ax] = wtb[ax];
        ab = ab - wtb[ax] * G->g[ax] / (a * a);
      }
      /* Q = E1 / a */
      E1b = E1b + Qb / a;
      ab = ab - Qb * E1 / (a * a);
      /* E = e^{-a dt}, E1 = 1 - e^{-a dt} */
      ab = ab + Eb * (-dt * E) + E1b * (dt * E);
      /* a = alpha * 18 mu / (rho_p d^2) */
      alphab = alphab + ab * a / G->alpha;
      db = db + ab * (-2.0 * a / dp);
      /* m = mult rho_p pi d^3 / 6 */
      db = db + mb * 3.0 * m / dp;
      /* u_p = sum_corners W(f) U[corner] */
      double fb[3] = {0.0, 0.0, 0.0};
      for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
          for (int di = 0; di < 2; ++di) {
            double wx = di ? f[0] : 1.0 - f[0];
            double wy = dj ? f[1] : 1.0 - f[1];
            double wz = dk ? f[2] : 1.0 - f[2];
            double w = wx * wy * wz;
            int64_t c = linear_cell(G, wrap_index(i0[0] + di, G->n[0]),
                                    wrap_index(i0[1] + dj, G->n[1]), wrap_index(i0[2] + dk, G->n[2]));
            double dot = 0.0;
            for (int q = 0; q < 3; ++q) {
              gradU[3 * c + q] = gradU[3 * c + q] + w * ub[q];
              dot = dot + U[3 * c + q] * ub[q];
            }
            fb[0] = fb[0] + (di ? 1.0 : -1.0) * wy * wz * dot;
            fb[1] = fb[1] + wx * (dj ? 1.0 : -1.0) * wz * dot;
            fb[2] = fb[2] + wx * wy * (dk ? 1.0 : -1.0) * dot;
          }
      for (int ax = 0; ax < 3; ++ax) {
        xb[ax] = xsb[ax] + (fb[ax] + fdep[ax]) / h[ax];
        vb[ax] = vsb[ax];
      }
    }
    grad_d[p] = db;
    *grad_alpha = *grad_alpha + alphab;
  }
  free(tx);
  free(tv);
  free(tc);
  return 0;
}

/* Extrapolation of S^m from the two sources before it (Sec. 2.4, Eqs. 14a-c). */
static double ecm_extrapolate(int32_t extrap, const double* prev1, const double* prev2, int64_t i) {
  double a = prev1 ? prev1[i] : 0.0;
  double b = prev2 ? prev2[i] : 0.0;
  if (extrap == 1) return a;
  if (extrap == 2) return 2.0 * a - b;
  return 0.0;
}

/* Sec. 2.4, Eqs. 12-13 with the reading stated in the header. */
void orc_ecm_estimate(int32_t extrap, int64_t m, const double* s1, const double* s2,
                      const double* s3, double* out) {
  for (int64_t i = 0; i < m; ++i) {
    double last = s1 ? s1[i] : 0.0;
    double ext_prev = ecm_extrapolate(extrap, s2, s3, i); /* estimate of S^{n-1} */
    double ext_now = ecm_extrapolate(extrap, s1, s2, i);  /* estimate of S^n */
    out[i] = last - ext_prev + ext_now;
  }
}

int orc_fluid_update(const orc_grid* G, double* U, const double* S, double rho_f, double nu,
                     double dtc, int32_t sweeps) {
  if (!grid_ok(G) || !(rho_f > 0.0) || nu < 0.0 || sweeps < 0) return -1;
  int64_t nc = ncell_of(G);
  double h[3] = {cell_size(G, 0), cell_size(G, 1), cell_size(G, 2)};
  double V = h[0] * h[1] * h[2];
  double lam[3];
  double lsum = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    lam[ax] = nu * dtc / (h[ax] * h[ax]);
    lsum = lsum + lam[ax];
  }
  double* ustar = (double*)malloc((size_t)nc * 3 * sizeof(double));
  double* next = (double*)malloc((size_t)nc * 3 * sizeof(double));
  if (!ustar || !next) {
    free(ustar);
    free(next);
    return -2;
  }
  /* explicit momentum source: the impulse S spread over the fluid mass of the cell */
  for (int64_t c = 0; c < nc; ++c)
    for (int q = 0; q < 3; ++q) {
      double add = S ? S[q * nc + c] / (rho_f * V) : 0.0;
      ustar[3 * c + q] = U[3 * c + q] + add;
      U[3 * c + q] = ustar[3 * c + q];
    }
  /* Jacobi: u_new = (u* + sum_ax lam_ax (u_old(+ax) + u_old(-ax))) / (1 + 2 sum lam) */
  for (int32_t it = 0; it < sweeps; ++it) {
    for (int32_t k = 0; k < G->n[2]; ++k)
      for (int32_t j = 0; j < G->n[1]; ++j)
        for (int32_t i = 0; i < G->n[0]; ++i) {
          int64_t c = linear_cell(G, i, j, k);
          int64_t nb[3][2] = {
              {linear_cell(G, wrap_index(i - 1, G->n[0]), j, k), linear_cell(G, wrap_index(i + 1, G->n[0]), j, k)},
              {linear_cell(G, i, wrap_index(j - 1, G->n[1]), k), linear_cell(G, i, wrap_index(j + 1, G->n[1]), k)},
              {linear_cell(G, i, j, wrap_index(k - 1, G->n[2])), linear_cell(G, i, j, wrap_index(k + 1, G->n[2]))}};
          for (int q = 0; q < 3; ++q) {
            double acc = ustar[3 * c + q];
            for (int ax = 0; ax < 3; ++ax)
              acc = acc + lam[ax] * (U[3 * nb[ax][0] + q] + U[3 * nb[ax][1] + q]);
            next[3 * c + q] = acc / (1.0 + 2.0 * lsum);
          }
        }
    memcpy(U, next, (size_t)nc * 3 * sizeof(double));
  }
  free(ustar);
  free(next);
  return 0;
}

int orc_couple(const orc_grid* G, double* U, int64_t n, double* pos, double* vel, const double* d,
               int32_t nint, int32_t K, double dt, double rho_f, double nu, int32_t sweeps,
               int32_t extrap, double* pending) {
  if (!grid_ok(G) || n < 0 || nint < 0 || K < 1 || !(dt > 0.0) || extrap < 0 || extrap > 2) return -1;
  int64_t m = 3 * ncell_of(G);
  /* the sources of the last three intervals, S^{n-1}, S^{n-2}, S^{n-3} */
  double* hist[3];
  double* cur = (double*)calloc((size_t)m, sizeof(double));
  double* est = (double*)calloc((size_t)m, sizeof(double));
  int ok = cur && est;
  for (int k = 0; k < 3; ++k) {
    hist[k] = (double*)calloc((size_t)m, sizeof(double));
    ok = ok && hist[k];
  }
  if (!ok) {
    free(cur);
    free(est);
    for (int k = 0; k < 3; ++k) free(hist[k]);
    return -2;
  }
  int32_t have = 0; /* intervals completed so far */
  for (int32_t it = 0; it < nint; ++it) {
    /* the estimate for interval it uses only the sources of earlier intervals */
    orc_ecm_estimate(extrap, m, have >= 1 ? hist[0] : NULL, have >= 2 ? hist[1] : NULL,
                     have >= 3 ? hist[2] : NULL, est);
    /* particles: K steps in the frozen field u^it, depositing S^it */
    memset(cur, 0, (size_t)m * sizeof(double));
    int r = orc_run(G, U, n, pos, vel, d, K, dt, cur, NULL, NULL);
    /* fluid: u^{it+1} from u^it and the estimate (independent of S^it, so the order of the two
     * halves does not matter) */
    if (r == 0) r = orc_fluid_update(G, U, est, rho_f, nu, (double)K * dt, sweeps);
    if (r != 0) {
      free(cur);
      free(est);
      for (int k = 0; k < 3; ++k) free(hist[k]);
      return r;
    }
    double* oldest = hist[2];
    hist[2] = hist[1];
    hist[1] = hist[0];
    hist[0] = oldest;
    memcpy(hist[0], cur, (size_t)m * sizeof(double));
    have = have + 1;
  }
  if (pending) {
    /* sum of S^n minus sum of S_est^n over the intervals run: S^{N-1} - S_ext^{N-1} */
    for (int64_t i = 0; i < m; ++i) {
      double last = have >= 1 ? hist[0][i] : 0.0;
      double ext_last = ecm_extrapolate(extrap, have >= 2 ? hist[1] : NULL, have >= 3 ? hist[2] : NULL, i);
      pending[i] = last - ext_last;
    }
  }
  free(cur);
  free(est);
  for (int k = 0; k < 3; ++k) free(hist[k]);
  return 0;
}

int64_t orc_chunk_bounds(const orc_grid* G, int64_t n, const double* pos_sort, const double* pos_now,
                         double* out) {
  if (!grid_ok(G) || n < 0 || G->chunk_edge < 1) return -1;
  int32_t B = G->chunk_edge;
  int32_t nc[3];
  for (int ax = 0; ax < 3; ++ax) nc[ax] = (G->n[ax] + B - 1) / B;
  int64_t nchunk = (int64_t)nc[0] * nc[1] * nc[2];
  for (int64_t c = 0; c < nchunk; ++c)
    for (int ax = 0; ax < 3; ++ax) {
      out[6 * c + ax] = INFINITY;
      out[6 * c + 3 + ax] = -INFINITY;
    }
  for (int64_t p = 0; p < n; ++p) {
    double xs[3] = {pos_sort[p], pos_sort[n + p], pos_sort[2 * n + p]};
    int32_t idx[3];
    orc_cell(G, xs, idx);
    int32_t ch[3] = {idx[0] / B, idx[1] / B, idx[2] / B};
    int64_t c = ch[0] + (int64_t)nc[0] * (ch[1] + (int64_t)nc[1] * ch[2]);
    for (int ax = 0; ax < 3; ++ax) {
      double h = cell_size(G, ax);
      double centre = ((double)ch[ax] * B + 0.5 * B) * h;
      double x = orc_wrap(pos_now[ax * n + p], G->L[ax]);
      /* nearest periodic image of x to the centre */
      double dx = x - centre;
      dx = dx - G->L[ax] * floor(dx / G->L[ax] + 0.5);
      double xu = centre + dx;
      if (xu < out[6 * c + ax]) out[6 * c + ax] = xu;
      if (xu > out[6 * c + 3 + ax]) out[6 * c + 3 + ax] = xu;
    }
  }
  return nchunk;
}

/* ---- droplet microphysics (Sec. 2.1): vapour mass transfer and heat transfer ---------------- */

/* Saturation vapour density over a flat water surface at temperature T (K):
 * rho_sat = e_s(T) / (R_v T) with the saturation vapour pressure of the Magnus
 * form, e_s = 610.94 Pa exp(17.625 t / (t + 243.04 K)), t = T - 273.15 K (the
 * coefficients Alduchov and Eskridge (1996) fitted over water), and the gas
 * constant of water vapour R_v = 461.5 J/(kg K). */
double orc_rho_sat(double T) {
  double t = T - 273.15;
  double es = 610.94 * exp(17.625 * t / (t + 243.04));
  return es / (461.5 * T);
}

/* Nusselt number of a sphere at particle Reynolds number Re: the Ranz-Marshall
 * correlation Nu = 2 + 0.6 Re^(1/2) Pr^(1/3) (the paper names the Nusselt
 * number without a correlation). */
double orc_nusselt(const orc_micro* M, double re) {
  return 2.0 + 0.6 * sqrt(re) * pow(M->Pr, 1.0 / 3.0);
}

/* A cell-centred scalar field F[c] at x: trilinear (or, gather = 1, the
 * containing cell's value), with the stencil of the velocity gather. */
static double scalar_gather(const orc_grid* G, const double* F, const double x[3]) {
  if (G->gather == 1) {
    int32_t idx[3];
    orc_cell(G, x, idx);
    return F[linear_cell(G, idx[0], idx[1], idx[2])];
  }
  int64_t cells[8];
  double w[8];
  trilinear_stencil(G, x, cells, w);
  double s = 0.0;
  for (int c = 0; c < 8; ++c) s = s + w[c] * F[cells[c]];
  return s;
}

/* d rho_sat / dT at T (K): rho_sat (d ln e_s / dT - 1 / T) with d ln e_s / dT =
 * 17.625 * 243.04 / (t + 243.04)^2 from the Magnus form above. */
double orc_rho_sat_dT(double T) {
  double t = T - 273.15;
  double a = t + 243.04;
  return orc_rho_sat(T) * (17.625 * 243.04 / (a * a) - 1.0 / T);
}

/* One step of one droplet with mass and heat transfer.  The rates come from the
 * state at the start of the step (position x, velocity v, diameter d,
 * temperature Tp) and the fluid values gathered at x (velocity u_p,
 * temperature T_f, vapour density rho_v), held over the step:
 *   - motion as orc_advance, with the drag of the start-of-step diameter;
 *   - mass (Sec. 2.1): dm/dt = 2 pi D_v d rho_sat (S_f - S_p) with S_f =
 *     rho_v / rho_sat(T_f) and S_p = rho_sat(Tp) / rho_sat(T_f) (a flat
 *     surface at the droplet's temperature), i.e. dm/dt = B (rho_v -
 *     rho_sat(Tp)), B = 2 pi D_v d; with m = rho_p pi d^3 / 6 per droplet
 *     this is d(d^2)/dt = 8 D_v (rho_v - rho_sat(Tp)) / rho_p;
 *   - heat (Sec. 2.1): m C_p dTp/dt = A (T_f - Tp) + L dm/dt, A = pi Nu kappa_f
 *     d (reading: the latent heat of the condensed mass warms the droplet and
 *     evaporation cools it; the printed equation has the opposite sign, which
 *     would heat an evaporating droplet), Nu from the start-of-step slip
 *     (Re = rho_f |u_p - v| d / mu);
 *   - the step (the paper gives none): with d, A, B frozen and rho_sat
 *     linearised about the start temperature T0, rho_sat(T) ~ r0 + s (T - T0),
 *     the heat balance is linear, dT/dt = -k (T - T*), and is advanced
 *     exactly; the d^2 law is integrated along the same temperature path:
 *       k = (A + L B s) / (m C_p),   x = k dt,
 *       delta = T* - T0 = (A (T_f - T0) + L B (rho_v - r0)) / (A + L B s),
 *       Tp' = T0 + delta x phi1(x),
 *       d'^2 = d^2 + (8 D_v / rho_p) dt [(rho_v - r0) - s delta x phi2(x)],
 *     with phi1(x) = (1 - e^{-x}) / x and phi2(x) = (1 - phi1(x)) / x (the
 *     time average of e^{-k t} over the step, and of the part of the
 *     temperature change not yet done).  These are the exact solution of the
 *     linearised equations written without cancellation.  The step is exact
 *     when the droplet stays at the fluid temperature (the d^2 law) and when no
 *     vapour moves (the temperature's exponential relaxation), and stable for
 *     steps much longer than the droplet's thermal time.  A droplet that would
 *     shrink below d_min keeps d_min;
 *   - what the fluid gains, into the start-of-step cell c0 (Sec. 2.1, Eq. 11
 *     and the vapour and energy sources, with the sign of a gain for the
 *     fluid): momentum J = -[(m' v' - m v) - m g dt], vapour mass -(m' - m),
 *     energy -C_p (m' Tp' - m Tp), evaluated as -[m (v' - v - g dt) + (m' - m)
 *     v'], -(m' - m) and -C_p [m (Tp' - Tp) + (m' - m) Tp'] with m' - m = c
 *     (d' - d)(d'^2 + d' d + d^2) and d' - d = (d'^2 - d^2) / (d' + d), so that
 *     no small difference is taken of large numbers.  Masses include the
 *     parcel multiplicity (c = w rho_p pi / 6); the per-droplet rates do not
 *     depend on it. */
void orc_micro_particle_step(const orc_grid* G, const orc_micro* M, const double* U, const double* Tf,
                             const double* rhov, double dt, double x[3], double v[3], double* d, double* Tp,
                             int64_t* c0, double J[3], double* dmass, double* denergy) {
  int32_t idx[3];
  double up[3], vold[3];
  orc_cell(G, x, idx);
  *c0 = linear_cell(G, idx[0], idx[1], idx[2]);
  orc_gather(G, U, x, up);
  double tf = scalar_gather(G, Tf, x);
  double rv = scalar_gather(G, rhov, x);
  double d0 = *d, T0 = *Tp;
  double r0 = up[0] - v[0], r1 = up[1] - v[1], r2 = up[2] - v[2];
  double re = G->rho_f * sqrt(r0 * r0 + r1 * r1 + r2 * r2) * d0 / G->mu;
  for (int ax = 0; ax < 3; ++ax) vold[ax] = v[ax];
  orc_advance(G, d0, up, dt, x, v);
  for (int ax = 0; ax < 3; ++ax) x[ax] = orc_wrap(x[ax], G->L[ax]);
  /* the linearised heat balance over the step */
  double nu = orc_nusselt(M, re);
  double md0 = G->rho_p * kPi * d0 * d0 * d0 / 6.0;
  double A = kPi * nu * M->kappa_f * d0;
  double B = 2.0 * kPi * M->D_v * d0;
  double rs = orc_rho_sat(T0);
  double sl = orc_rho_sat_dT(T0);
  double den = A + M->L * B * sl;
  double k = den / (md0 * M->cp_p);
  double delta = (A * (tf - T0) + M->L * B * (rv - rs)) / den;
  double xk = k * dt;
  double phi1 = -expm1(-xk) / xk;
  double phi2 = (1.0 - phi1) / xk;
  double T1 = T0 + delta * xk * phi1;
  /* the d^2 law along that temperature path */
  double dq = 8.0 * M->D_v * dt * ((rv - rs) - sl * delta * xk * phi2) / G->rho_p;
  double q = d0 * d0 + dq;
  double d1 = q > M->d_min * M->d_min ? sqrt(q) : M->d_min;
  double dd = q > M->d_min * M->d_min ? dq / (d1 + d0) : d1 - d0;
  double dm = G->mult * G->rho_p * kPi / 6.0 * dd * (d1 * d1 + d1 * d0 + d0 * d0);
  double m0 = orc_mass(G, d0);
  /* what the fluid gains */
  for (int ax = 0; ax < 3; ++ax) J[ax] = -(m0 * ((v[ax] - vold[ax]) - G->g[ax] * dt) + dm * v[ax]);
  *dmass = -dm;
  *denergy = -M->cp_p * (m0 * (T1 - T0) + dm * T1);
  *d = d1;
  *Tp = T1;
}

int orc_micro_run(const orc_grid* G, const orc_micro* M, const double* U, const double* Tf, const double* rhov,
                  int64_t n, double* pos, double* vel, double* d, double* Tp, int32_t nsteps, double dt,
                  double* src, double* msrc, double* esrc) {
  if (!grid_ok(G) || !M || n < 0 || nsteps < 0 || G->deposit != 0) return -1;
  if (!(M->D_v >= 0.0) || !(M->kappa_f > 0.0) || !(M->cp_p > 0.0) || !(M->Pr > 0.0) || !(M->d_min > 0.0))
    return -1;
  int64_t nc = ncell_of(G);
  for (int32_t s = 0; s < nsteps; ++s) {
    for (int64_t p = 0; p < n; ++p) {
      double x[3] = {pos[p], pos[n + p], pos[2 * n + p]};
      double v[3] = {vel[p], vel[n + p], vel[2 * n + p]};
      int64_t c0;
      double J[3], dm, de;
      orc_micro_particle_step(G, M, U, Tf, rhov, dt, x, v, &d[p], &Tp[p], &c0, J, &dm, &de);
      if (src)
        for (int ax = 0; ax < 3; ++ax) src[ax * nc + c0] = src[ax * nc + c0] + J[ax];
      if (msrc) msrc[c0] = msrc[c0] + dm;
      if (esrc) esrc[c0] = esrc[c0] + de;
      pos[p] = x[0];
      pos[n + p] = x[1];
      pos[2 * n + p] = x[2];
      vel[p] = v[0];
      vel[n + p] = v[1];
      vel[2 * n + p] = v[2];
    }
  }
  return 0;
}
