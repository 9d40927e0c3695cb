// Plain FP64 Lagrangian step: one particle per lane, 32 consecutive particles
// per warp.  Gather -> exponential integrator -> wrap/relocate -> impulse,
// then a warp-segmented reduction of the impulses over runs of equal
// start-of-step cell in storage order, committed to the exact fixed-point
// source accumulator.  The physics variants (nearest-grid-point gather,
// semi-implicit Euler, Schiller-Naumann drag, cloud-in-cell deposit) are
// uniform branches on the step's parameters.  GB300's FP64 rate is low, so this kernel is bound by
// FP64 arithmetic rather than by HBM.
#include "st_common.cuh"

namespace st {
namespace {

struct F64Args {
  F64State s;
  const D4* __restrict__ U;
  long long* __restrict__ acc;
  int64_t n;
  int64_t ncell;
  int nx, ny, nz;
  double L[3], invL[3], inv_h[3];
  double inv_ca;  // 1 / ca = rho_p / (18 mu alpha)
  StepParams p;
};

__device__ __forceinline__ double wrap_pos(double x, double L, double invL) {
  double y = x - L * floor(x * invL);
  if (y < 0.0) y += L;
  if (y >= L) y = 0.0;
  return y;
}

__device__ __forceinline__ D4 ld_cell(const D4* __restrict__ U, int64_t c) {
  const double2* p = reinterpret_cast<const double2*>(U + c);
  double2 a = __ldg(p), b = __ldg(p + 1);
  return D4{a.x, a.y, b.x, b.y};
}

__device__ __forceinline__ void lerp3(D4 a, D4 b, double f, double r[3]) {
  r[0] = fma(f, b.x - a.x, a.x);
  r[1] = fma(f, b.y - a.y, a.y);
  r[2] = fma(f, b.z - a.z, a.z);
}

// Schiller-Naumann drag factor f = C_D Re / 24: 1 + 0.15 Re^0.687 up to Re = 1000, 0.44 Re / 24 above
__device__ __forceinline__ double sn_factor(double re) {
  return re <= 1000.0 ? 1.0 + 0.15 * pow(re, 0.687) : (0.44 / 24.0) * re;
}

// Warp-segmented sum of J over runs of equal key (lanes in storage order), one commit per run.
__device__ __forceinline__ void deposit_runs(const F64Args& a, int lane, int key, double j0, double j1, double j2) {
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  const bool head = (lane == 0) || (prev != key);
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const unsigned above = lane == 31 ? 0u : (heads & ~((2u << lane) - 1u));
  const int end = above ? (__ffs(above) - 2) : 31;
  for (int off = 1; off < 32; off <<= 1) {
    double t0 = __shfl_down_sync(0xffffffffu, j0, off);
    double t1 = __shfl_down_sync(0xffffffffu, j1, off);
    double t2 = __shfl_down_sync(0xffffffffu, j2, off);
    if (lane + off <= end) {
      j0 += t0;
      j1 += t1;
      j2 += t2;
    }
  }
  if (a.acc && head && key >= 0) {
    acc_add_f64(a.acc + kAccWords * key, j0, a.p.E);
    acc_add_f64(a.acc + kAccWords * (a.ncell + key), j1, a.p.E);
    acc_add_f64(a.acc + kAccWords * (2 * a.ncell + key), j2, a.p.E);
  }
}

__global__ void __launch_bounds__(256) step_f64_kernel(const F64Args a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n3[3] = {a.nx, a.ny, a.nz};
  const int64_t row = a.nx, slab = (int64_t)a.nx * a.ny;
  for (int64_t base = warp * 32; base < a.n; base += nwarp * 32) {
    const int64_t p = base + lane;
    int key = -1;
    double J[3] = {0.0, 0.0, 0.0};
    int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    if (p < a.n) {
      double x[3], v[3];
      for (int q = 0; q < 3; ++q) {
        x[q] = a.s.x[q][p];
        v[q] = a.s.v[q][p];
      }
      const double d = a.s.d[p];
      // start-of-step cell and trilinear stencil on cell centres
      int c0[3];
      for (int q = 0; q < 3; ++q) {
        double sx = x[q] * a.inv_h[q];
        int i = (int)floor(sx);
        c0[q] = min(max(i, 0), n3[q] - 1);
        double s2 = sx - 0.5;
        double fl = floor(s2);
        int ii = (int)fl;
        f[q] = s2 - fl;
        i0[q] = ii < 0 ? ii + n3[q] : ii;
        i1[q] = ii + 1 >= n3[q] ? ii + 1 - n3[q] : ii + 1;
      }
      key = c0[0] + a.nx * (c0[1] + a.ny * c0[2]);
      double up[3];
      if (a.p.ngp) {
        // nearest grid point: the value of the cell holding the particle
        const D4 Uc = ld_cell(a.U, key);
        up[0] = Uc.x;
        up[1] = Uc.y;
        up[2] = Uc.z;
      } else {
        D4 U000 = ld_cell(a.U, i0[0] + row * i0[1] + slab * i0[2]);
        D4 U100 = ld_cell(a.U, i1[0] + row * i0[1] + slab * i0[2]);
        D4 U010 = ld_cell(a.U, i0[0] + row * i1[1] + slab * i0[2]);
        D4 U110 = ld_cell(a.U, i1[0] + row * i1[1] + slab * i0[2]);
        D4 U001 = ld_cell(a.U, i0[0] + row * i0[1] + slab * i1[2]);
        D4 U101 = ld_cell(a.U, i1[0] + row * i0[1] + slab * i1[2]);
        D4 U011 = ld_cell(a.U, i0[0] + row * i1[1] + slab * i1[2]);
        D4 U111 = ld_cell(a.U, i1[0] + row * i1[1] + slab * i1[2]);
        double r00[3], r10[3], r01[3], r11[3];
        lerp3(U000, U100, f[0], r00);
        lerp3(U010, U110, f[0], r10);
        lerp3(U001, U101, f[0], r01);
        lerp3(U011, U111, f[0], r11);
        for (int q = 0; q < 3; ++q) {
          const double r0 = fma(f[1], r10[q] - r00[q], r00[q]);
          const double r1 = fma(f[1], r11[q] - r01[q], r01[q]);
          up[q] = fma(f[2], r1 - r0, r0);
        }
      }
      // drag rate a = alpha f(Re) / tau, f = 1 for Stokes drag
      const double dd = d * d;
      // 1/a first (one division per particle: GB300 divides in FP64 by iteration), then a from it
      double inv_ra = dd * a.inv_ca;
      if (a.p.sn) {
        const double r0 = up[0] - v[0], r1 = up[1] - v[1], r2 = up[2] - v[2];
        inv_ra /= sn_factor(a.p.re_coef * sqrt(r0 * r0 + r1 * r1 + r2 * r2) * d);
      }
      const double ra = 1.0 / inv_ra;
      const double adt = ra * a.p.dt;
      const double m = a.p.mcoef * dd * d;
      if (a.p.semi) {
        // semi-implicit Euler: v' = (v + dt (a u_p + g)) / (1 + a dt), x' = x + dt v'
        const double inv_den = 1.0 / (1.0 + adt);
        for (int q = 0; q < 3; ++q) {
          const double vn = (v[q] + a.p.dt * (ra * up[q] + a.p.g[q])) * inv_den;
          const double xn = x[q] + a.p.dt * vn;
          J[q] = -m * ((vn - v[q]) - a.p.g[q] * a.p.dt);
          a.s.x[q][p] = wrap_pos(xn, a.L[q], a.invL[q]);
          a.s.v[q][p] = vn;
        }
      } else {
        // exponential integrator
        // 1 - e^{-a dt} from expm1; e^{-a dt} as its complement (absolute error ~1e-16, which is what
        // multiplies v - w), one FP64 exponential instead of two
        const double E1 = -expm1(-adt);
        const double E = 1.0 - E1;
        const double Qd = E1 * inv_ra;
        for (int q = 0; q < 3; ++q) {
          const double wt = up[q] + a.p.g[q] * inv_ra;
          const double vn = wt + (v[q] - wt) * E;
          const double xn = x[q] + (wt * a.p.dt + (v[q] - wt) * Qd);
          J[q] = -m * ((vn - v[q]) - a.p.g[q] * a.p.dt);
          a.s.x[q][p] = wrap_pos(xn, a.L[q], a.invL[q]);
          a.s.v[q][p] = vn;
        }
      }
    }
    if (!a.p.cic) {
      deposit_runs(a, lane, key, J[0], J[1], J[2]);
    } else {
      // cloud in cell: the eight cells of the start-of-step trilinear stencil, each its own pass of
      // runs over the warp (sorted particles share corners, so runs stay long)
      for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        const int kc = key < 0 ? -1 : (dx ? i1[0] : i0[0]) + a.nx * ((dy ? i1[1] : i0[1]) + a.ny * (dz ? i1[2] : i0[2]));
        deposit_runs(a, lane, kc, w * J[0], w * J[1], w * J[2]);
      }
    }
  }
}

}  // namespace

cudaError_t launch_step_f64(st_ctx* h, const StepParams& p) {
  return launch_step_f64_state(h, carve_f64(h->state.p, h->cap), (long long*)h->acc.p, p);
}

cudaError_t launch_step_f64_state(st_ctx* h, const F64State& s, long long* acc, const StepParams& p) {
  F64Args a;
  a.s = s;
  a.U = (const D4*)h->fluid.p;
  a.acc = acc;
  a.n = h->np;
  a.ncell = h->geo.ncell;
  a.nx = h->geo.n[0];
  a.ny = h->geo.n[1];
  a.nz = h->geo.n[2];
  for (int q = 0; q < 3; ++q) {
    a.L[q] = h->geo.L[q];
    a.invL[q] = 1.0 / h->geo.L[q];
    a.inv_h[q] = h->geo.inv_h[q];
  }
  a.p = p;
  a.inv_ca = 1.0 / p.ca;
  int64_t warps = (h->np + 31) / 32;
  int64_t blocks = (warps * 32 + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  step_f64_kernel<<<(int)blocks, 256, 0, h->stream>>>(a);
  h->launches += 1;
  return cudaGetLastError();
}

}  // namespace st
