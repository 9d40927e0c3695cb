// Lagrangian step with droplet microphysics (paper Sec. 2.1): besides moving under drag and gravity,
// each droplet exchanges water vapour with the fluid, dm/dt = 2 pi D_v d (rho_v - rho_sat(Tp)) (the
// mass-transfer equation with S_f = rho_v / rho_sat(T_f) and a flat surface at the droplet's
// temperature, S_p = rho_sat(Tp) / rho_sat(T_f)), and heat, m C_p dTp/dt = pi Nu kappa d (T_f - Tp)
// + L dm/dt (the latent heat of the condensed mass warms the droplet).  The fluid gains the momentum
// -[(m' v' - m v) - m g dt], the vapour -(m' - m) and the energy -C_p (m' Tp' - m Tp), each into the
// cell that held the droplet at the start of the step.
//
// The step holds d, the slip (for the Nusselt number, Ranz-Marshall 2 + 0.6 Re^(1/2) Pr^(1/3)) and
// the gathered fluid values over the step, linearises rho_sat about the start temperature T0 and
// solves the droplet's then linear heat balance exactly, with the d^2 law integrated along that
// temperature path:
//   k = (A + L B s) / (m C_p), x = k dt, A = pi Nu kappa d, B = 2 pi D_v d, s = drho_sat/dT(T0),
//   delta = (A (T_f - T0) + L B (rho_v - rho_sat(T0))) / (A + L B s),
//   Tp' = T0 + delta x phi1(x),   d'^2 = d^2 + (8 D_v / rho_p) dt [(rho_v - rho_sat(T0)) - s delta x phi2(x)],
// phi1(x) = (1 - e^-x) / x, phi2(x) = (1 - phi1(x)) / x; a droplet that would shrink below d_min keeps
// d_min.  The saturation density is the Magnus form with the coefficients Alduchov and Eskridge
// fitted over water, e_s = 610.94 Pa exp(17.625 t / (t + 243.04)), t in degC, over R_v T with
// R_v = 461.5 J/(kg K).
//
// Mixed handles keep the diameter and the temperature compensated: the per-step growth of a droplet is
// about 1e-7 of its diameter at dt = 5e-4 s, the size of one FP32 rounding step, and the per-step
// temperature change is often below the FP32 spacing at 285 K (3e-5 K), so FP32 values alone would
// round most of the transfer away.  Beside the FP32 diameter that every other kernel reads, each
// particle carries {T_hi, T_lo, d_lo, 0} (16 B): T = T_hi + T_lo and d = d + d_lo, each increment
// added with an error-free two-sum, so the stored state loses no increment.
//
// One particle per lane; the warp's lanes are reordered so that equal start cells are adjacent (an
// order fixed by the cells), the five gains are summed over each cell's lanes and each sum is added
// once to the exact accumulators: momentum to the fixed-point source accumulator,
// vapour and energy to a carry-save accumulator wide enough to need no exponent.  Only the default
// physics (trilinear gather, exponential integrator, Stokes drag, cell deposit).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "st_common.cuh"
#include "st_ptx.cuh"

namespace st {
namespace {

constexpr int kMicroThreads = 256;

// constants of the microphysics (per droplet; mcoef includes the parcel multiplicity)
template <class R>
struct MicroConst {
  R Dv, kappa, cp, L, nu_coef /* 0.6 Pr^(1/3) */, dmin, dq_coef /* 8 D_v / rho_p */;
  R mdrop /* rho_p pi / 6 */, mcoef /* mult rho_p pi / 6 */, re_coef /* rho_f / mu */;
};

__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ double em1(double x) { return expm1(x); }
__device__ __forceinline__ double sq(double x) { return sqrt(x); }
__device__ __forceinline__ double dv(double a, double b) { return a / b; }
// FP32: the hardware's approximate exponential and division (errors of a few units in the last place,
// for arguments of order one and divisors far from the FP32 range's ends), which the FP32 state's
// own rounding dominates; the step's increments enter the state through error-free sums
__device__ __forceinline__ float ex(float x) { return __expf(x); }
__device__ __forceinline__ float em1(float x) { return expm1f(x); }
__device__ __forceinline__ float sq(float x) { return sqrtf(x); }
__device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }

// saturation vapour density over flat water at T (K) and its temperature derivative
template <class R>
__device__ __forceinline__ void rho_sat(R T, R& rs, R& slope) {
  const R t = T - R(273.15);
  const R a = t + R(243.04);
  const R ia = dv(R(1), a), iT = dv(R(1), T);
  rs = R(610.94 / 461.5) * ex(R(17.625) * t * ia) * iT;
  slope = rs * (R(17.625 * 243.04) * ia * ia - iT);
}

// phi1(x) = (1 - e^-x) / x and phi2(x) = (1 - phi1) / x, x >= 0: their Taylor series below 1/4
// (alternating, error below the first dropped term, x^6 / 40320 < 6e-9), the closed forms above
template <class R>
__device__ __forceinline__ void phis(R x, R& p1, R& p2) {
  if (x < R(0.25)) {
    p2 = R(0.5) - x * (R(1.0 / 6) - x * (R(1.0 / 24) - x * (R(1.0 / 120) - x * (R(1.0 / 720) - x * R(1.0 / 5040)))));
    p1 = R(1) - x * p2;
  } else {
    const R ix = dv(R(1), x);
    p1 = -em1(-x) * ix;
    p2 = (R(1) - p1) * ix;
  }
}

// mass and heat over the step: the new diameter d1 (clamped at d_min) and its increment dd, the
// temperature increment dT, and the parcel's mass change dm
template <class R>
__device__ __forceinline__ bool transfer(const MicroConst<R>& c, R dt, R d0, R T0, R tf, R rv, R re, R& d1, R& dd,
                                        R& dT, R& dm) {
  const R nu = R(2) + c.nu_coef * sq(re);
  const R pi = R(3.14159265358979323846);
  const R A = pi * nu * c.kappa * d0;
  const R B = R(2) * pi * c.Dv * d0;
  R rs, sl;
  rho_sat(T0, rs, sl);
  const R den = A + c.L * B * sl;
  const R md0 = c.mdrop * d0 * d0 * d0;
  const R k = dv(den, md0 * c.cp);
  const R delta = dv(A * (tf - T0) + c.L * B * (rv - rs), den);
  const R x = k * dt;
  R p1, p2;
  phis(x, p1, p2);
  dT = delta * x * p1;
  const R dq = c.dq_coef * dt * ((rv - rs) - sl * delta * x * p2);
  const R q = d0 * d0 + dq;
  const bool clamped = !(q > c.dmin * c.dmin);
  if (!clamped) {
    d1 = sq(q);
    dd = dv(dq, d1 + d0);
  } else {
    d1 = c.dmin;
    dd = d1 - d0;
  }
  dm = c.mcoef * dd * (d1 * d1 + d1 * d0 + d0 * d0);
  return clamped;
}

// error-free a + b = s + e (Knuth's two-sum), and the renormalised pair of hi + lo
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) + x as a renormalised pair (|lo| <= half a unit of hi)
__device__ __forceinline__ void add_pair(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  e = __fadd_rn(e, lo);
  const float h2 = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(h2, s));
  hi = h2;
}

// ---- FP64 state -----------------------------------------------------------------------------------

struct F64Args {
  F64State s;
  double* __restrict__ T;
  const D4* __restrict__ U;
  const double2* __restrict__ th;  // (T_f, rho_v) per cell
  long long* __restrict__ acc;
  long long* __restrict__ macc;
  int64_t n, ncell;
  int nx, ny, nz;
  double L[3], invL[3], inv_h[3];
  double dt, inv_ca, g[3];
  int E;
  MicroConst<double> c;
};

__device__ __forceinline__ double wrap_pos(double x, double L, double invL) {
  double y = x - L * floor(x * invL);
  if (y < 0.0) y += L;
  if (y >= L) y = 0.0;
  return y;
}

__global__ void __launch_bounds__(kMicroThreads) micro_f64_kernel(const F64Args a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n3[3] = {a.nx, a.ny, a.nz};
  const int64_t row = a.nx, slab = (int64_t)a.nx * a.ny;
  for (int64_t base = warp * 32; base < a.n; base += nwarp * 32) {
    const int64_t p = base + lane;
    int key = -1;
    double gain[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (p < a.n) {
      double x[3], v[3];
      for (int q = 0; q < 3; ++q) {
        x[q] = a.s.x[q][p];
        v[q] = a.s.v[q][p];
      }
      const double d0 = a.s.d[p], T0 = a.T[p];
      int c0[3], i0[3], i1[3];
      double f[3];
      for (int q = 0; q < 3; ++q) {
        const double sx = x[q] * a.inv_h[q];
        c0[q] = min(max((int)floor(sx), 0), n3[q] - 1);
        const double s2 = sx - 0.5;
        const double fl = floor(s2);
        const int ii = (int)fl;
        f[q] = s2 - fl;
        i0[q] = ii < 0 ? ii + n3[q] : ii;
        i1[q] = ii + 1 >= n3[q] ? ii + 1 - n3[q] : ii + 1;
      }
      key = c0[0] + a.nx * (c0[1] + a.ny * c0[2]);
      // trilinear gather of the velocity and of (T_f, rho_v)
      double up[3] = {0.0, 0.0, 0.0}, tf = 0.0, rv = 0.0;
      for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
        const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        const int64_t c = (dx ? i1[0] : i0[0]) + row * (dy ? i1[1] : i0[1]) + slab * (dz ? i1[2] : i0[2]);
        const D4 u = a.U[c];
        const double2 t = a.th[c];
        up[0] += w * u.x;
        up[1] += w * u.y;
        up[2] += w * u.z;
        tf += w * t.x;
        rv += w * t.y;
      }
      const double r0 = up[0] - v[0], r1 = up[1] - v[1], r2 = up[2] - v[2];
      const double re = a.c.re_coef * sqrt(r0 * r0 + r1 * r1 + r2 * r2) * d0;
      // motion: the exponential integrator under Stokes drag of the start-of-step diameter
      const double inv_ra = d0 * d0 * a.inv_ca;
      const double ra = 1.0 / inv_ra;
      const double E1 = -expm1(-ra * a.dt);
      const double Em = 1.0 - E1;
      const double Qd = E1 * inv_ra;
      double vn[3];
      for (int q = 0; q < 3; ++q) {
        const double wt = up[q] + a.g[q] * inv_ra;
        vn[q] = wt + (v[q] - wt) * Em;
        const double xn = x[q] + (wt * a.dt + (v[q] - wt) * Qd);
        a.s.x[q][p] = wrap_pos(xn, a.L[q], a.invL[q]);
        a.s.v[q][p] = vn[q];
      }
      double d1, dd, dT, dm;
      transfer(a.c, a.dt, d0, T0, tf, rv, re, d1, dd, dT, dm);
      const double T1 = T0 + dT;
      a.s.d[p] = d1;
      a.T[p] = T1;
      const double m0 = a.c.mcoef * d0 * d0 * d0;
      for (int q = 0; q < 3; ++q) gain[q] = -(m0 * ((vn[q] - v[q]) - a.g[q] * a.dt) + dm * vn[q]);
      gain[3] = -dm;
      gain[4] = -a.c.cp * (m0 * (T1 - T0) + dm * T1);
    }
    const bool head = run_sums(lane, key, gain);
    if (head && key >= 0) {
      for (int q = 0; q < 3; ++q) acc_add_f64(a.acc + kAccWords * (q * a.ncell + key), gain[q], a.E);
      wide_add(a.macc + kWideWords * key, gain[3]);
      wide_add(a.macc + kWideWords * (a.ncell + key), gain[4]);
    }
  }
}

// ---- mixed state (int32 cell + FP32 offset, FP32 or BF16 velocity, FP32 diameter and temperature) --

struct MixedArgs {
  MixedState s;
  float4* __restrict__ ms;         // {T_hi, T_lo, d_lo, 0} per particle
  const float4* __restrict__ Up;   // velocity with kFluidPad ghost layers
  const float2* __restrict__ thp;  // (T_f, rho_v) with kFluidPad ghost layers
  long long* __restrict__ acc;
  long long* __restrict__ macc;
  float4* __restrict__ rec;        // the step before a sort: the new state as 32-byte records (else null)
  int64_t n, ncell;
  int nx, ny, nz;
  float inv_h[3];
  float dt, inv_ca, g[3], gdt[3];
  int E;
  MicroConst<float> c;
};

template <bool BF16>
__device__ __forceinline__ float load_v(const MixedArgs& a, int q, int64_t p) {
  if (BF16) return __bfloat162float(((const __nv_bfloat16*)a.s.v[q])[p]);
  return ((const float*)a.s.v[q])[p];
}

// whole cells carried by an offset o (cell units) from cell ci on an axis of n cells; the new offset
// in [0, 1)
__device__ __forceinline__ int relocate(float& o, int ci, int n) {
  const float fl = floorf(o);
  o = fminf(fmaxf(o - fl, 0.0f), 0.99999994f);
  // a move of less than one box length: one periodic correction (no 64-bit remainder)
  if (fabsf(fl) < 1048576.0f) {
    int k = ci + (int)fl;
    if (k >= n) k -= n;
    else if (k < 0) k += n;
    if ((unsigned)k < (unsigned)n) return k;
  }
  long long k = ((long long)ci + (long long)fl) % n;
  return (int)(k < 0 ? k + n : k);
}

// One particle of the mixed state: gather, motion, relocation, mass and heat transfer.  In: the
// packed cell, offsets, velocities (as FP32; BF16 handles' stored values), the diameter's high part and
// {T_hi, T_lo, d_lo, 0}.  Out: the same updated (velocities rounded to their stored precision), the
// start cell's index and the fluid's gains {momentum x, y, z, vapour mass, energy}.
template <bool BF16>
__device__ __forceinline__ void micro_particle(const MixedArgs& a, const int (&n3)[3], int px, int pxy, int32_t& cell,
                                               float (&xi)[3], float (&v)[3], float& dhi, float4& st, int& key,
                                               float (&gain)[5]) {
  const int ci[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
  const float d0 = dhi, T0 = st.x;  // the rates need only FP32 values
  key = ci[0] + a.nx * (ci[1] + a.ny * ci[2]);
  // stencil on cell centres from (cell, offset): offset >= 1/2 -> base cell, fraction o - 1/2
  float f[3];
  int b[3];
  for (int q = 0; q < 3; ++q) {
    const bool hi = xi[q] >= 0.5f;
    f[q] = xi[q] + (hi ? -0.5f : 0.5f);
    b[q] = ci[q] - (hi ? 0 : 1) + kFluidPad;
  }
  float up[3] = {0.0f, 0.0f, 0.0f}, tf = 0.0f, rv = 0.0f;
  // the padded field has fewer than 2^31 cells: 32-bit corner offsets from the base corner
  const int c0 = b[0] + px * b[1] + pxy * b[2];
  const float4* ub = a.Up + c0;
  const float2* tb = a.thp + c0;
  const float wx[2] = {1.0f - f[0], f[0]}, wy[2] = {1.0f - f[1], f[1]}, wz[2] = {1.0f - f[2], f[2]};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const float w = wx[dx] * wy[dy] * wz[dz];
    const int o = dx + px * dy + pxy * dz;
    const float4 u = __ldg(ub + o);
    const float2 t = __ldg(tb + o);
    up[0] = fmaf(w, u.x, up[0]);
    up[1] = fmaf(w, u.y, up[1]);
    up[2] = fmaf(w, u.z, up[2]);
    tf = fmaf(w, t.x, tf);
    rv = fmaf(w, t.y, rv);
  }
  const float r0 = up[0] - v[0], r1 = up[1] - v[1], r2 = up[2] - v[2];
  const float re = a.c.re_coef * sqrtf(fmaf(r0, r0, fmaf(r1, r1, r2 * r2))) * d0;
  // motion: the exponential integrator, then relocation of (cell, offset)
  const float inv_a = d0 * d0 * a.inv_ca;
  const float E1 = -expm1f(-a.dt / inv_a);
  const float Em = 1.0f - E1;
  const float Q = E1 * inv_a;
  float vn[3], jm[3];
  int nc[3];
  for (int q = 0; q < 3; ++q) {
    const float wt = fmaf(a.g[q], inv_a, up[q]);
    const float dvw = v[q] - wt;
    float vq = fmaf(dvw, Em, wt);
    if (BF16) {
      vq = __bfloat162float(__float2bfloat16_rn(vq));
      jm[q] = (vq - v[q]) - a.gdt[q];  // the stored change: the deposit balances the stored momentum
    } else {
      jm[q] = -fmaf(dvw, E1, a.gdt[q]);  // v' - v - g dt without subtracting the rounded v'
    }
    vn[q] = vq;
    float o = fmaf(fmaf(wt, a.dt, dvw * Q), a.inv_h[q], xi[q]);
    nc[q] = relocate(o, ci[q], n3[q]);
    xi[q] = o;
    v[q] = vq;
  }
  cell = pack_cell(nc[0], nc[1], nc[2]);
  float d1, dd, dT, dm;
  const bool clamped = transfer(a.c, a.dt, d0, T0, tf, rv, re, d1, dd, dT, dm);
  // the increments, added exactly to the compensated state; the clamp at d_min sets the diameter
  float dn = dhi, dl = st.z;
  if (clamped) {
    dd = (a.c.dmin - dhi) - dl;
    dn = a.c.dmin;
    dl = 0.0f;
  } else {
    add_pair(dn, dl, dd);
  }
  add_pair(st.x, st.y, dT);
  st.z = dl;
  dhi = dn;
  const float T1 = T0 + dT;
  const float m0 = a.c.mcoef * d0 * d0 * d0;
  for (int q = 0; q < 3; ++q) gain[q] = -(m0 * jm[q] + dm * vn[q]);
  gain[3] = -dm;
  gain[4] = -a.c.cp * (m0 * dT + dm * T1);  // dT: the increment the stored temperature took
}

// The group sums of the head lanes added to the exact accumulators, the commits spread over the lanes:
// the H heads' 5 H (value, cell) items in component-major order through the warp's staging buffer, one
// item per lane and round.  A round then runs one or two of the add routines on many lanes instead of
// all five on the few head lanes; the adds are exact, so the sums are the same.
__device__ __forceinline__ void micro_commit(const MixedArgs& a, GroupBuf<5>& b, int lane, bool head, int key,
                                             const float (&g)[5]) {
  const unsigned hm = __ballot_sync(0xffffffffu, head);
  const int H = __popc(hm);
  __syncwarp();  // the reordering's reads of the buffer are done
  if (head) {
    const int r = __popc(hm & ((1u << lane) - 1u));
#pragma unroll
    for (int q = 0; q < 5; ++q) b.g[q][r] = g[q];
    b.key[r] = key;
  }
  __syncwarp();
  // item i: component q = floor(i / H), head r = i - q H; (i + 1/2) / H lies at least 1/(2 H) >= 1/64
  // from an integer, far more than the reciprocal's rounding moves it
  const float inv_h = __frcp_rn((float)(H > 0 ? H : 1));
  for (int i = lane; i < 5 * H; i += 32) {
    const int q = (int)(((float)i + 0.5f) * inv_h);
    const int r = i - q * H;
    const float v = b.g[q][r];
    const int k = b.key[r];
    if (q < 3)
      acc_add_f32(a.acc + kAccWords * ((int64_t)q * a.ncell + k), v, a.E);
    else
      wide_add_f32(a.macc + kWideWords * ((int64_t)(q - 3) * a.ncell + k), v);
  }
}

template <bool BF16>
__global__ void __launch_bounds__(kMicroThreads) micro_mixed_kernel(const MixedArgs a) {
  __shared__ GroupBuf<5> perm[kMicroThreads / 32];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n3[3] = {a.nx, a.ny, a.nz};
  const int px = a.nx + 2 * kFluidPad, pxy = (a.nx + 2 * kFluidPad) * (a.ny + 2 * kFluidPad);
  for (int64_t base = warp * 32; base < a.n; base += nwarp * 32) {
    const int64_t p = base + lane;
    int key = -1;
    float gain[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (p < a.n) {
      int32_t cell = a.s.cell[p];
      float xi[3], v[3];
      for (int q = 0; q < 3; ++q) {
        xi[q] = a.s.xi[q][p];
        v[q] = load_v<BF16>(a, q, p);
      }
      float dhi = a.s.d[p];
      float4 st = a.ms[p];
      micro_particle<BF16>(a, n3, px, pxy, cell, xi, v, dhi, st, key, gain);
      a.s.cell[p] = cell;
      if (a.rec) {
        // the cells stay in the arrays (the sort's keys); the state goes out as one 32-byte record
        // for the sort's gather (BF16 velocities are exact in FP32)
        ptx::st_rec32(a.rec + 2 * p, ptx::Rec32{__int_as_float(cell), xi[0], xi[1], xi[2], v[0], v[1], v[2], dhi});
      } else {
        for (int q = 0; q < 3; ++q) {
          a.s.xi[q][p] = xi[q];
          if (BF16)
            ((__nv_bfloat16*)a.s.v[q])[p] = __float2bfloat16_rn(v[q]);
          else
            ((float*)a.s.v[q])[p] = v[q];
        }
        a.s.d[p] = dhi;
      }
      a.ms[p] = st;
    }
    GroupBuf<5>& gb = perm[threadIdx.x >> 5];
    group_by_key(gb, lane, key, gain);
    const bool head = run_sums(lane, key, gain) && key >= 0;
    micro_commit(a, gb, lane, head, key, gain);
  }
}

// ---- fields, temperatures, bookkeeping ------------------------------------------------------------

template <class S>
__global__ void thermo_pack_f64_kernel(const S* __restrict__ T, const S* __restrict__ rv, double2* __restrict__ out,
                                       int64_t ncell) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x)
    out[c] = make_double2((double)T[c], (double)rv[c]);
}

// (T, rho_v) into the ghost-padded float2 layout of the mixed velocity field (periodic ghosts)
template <class S>
__global__ void thermo_pack_padded_kernel(const S* __restrict__ T, const S* __restrict__ rv, float2* __restrict__ out,
                                          int nx, int ny, int nz) {
  const int px = nx + 2 * kFluidPad, py = ny + 2 * kFluidPad, pz = nz + 2 * kFluidPad;
  const int64_t m = (int64_t)px * py * pz;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < m; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % px), j = (int)((c / px) % py), k = (int)(c / ((int64_t)px * py));
    const int si = (i - kFluidPad + nx) % nx, sj = (j - kFluidPad + ny) % ny, sk = (k - kFluidPad + nz) % nz;
    const int64_t s = si + (int64_t)nx * (sj + (int64_t)ny * sk);
    out[c] = make_float2((float)T[s], (float)rv[s]);
  }
}

// min and max of T and of rho_v, and whether any value is not finite: out = bits of {max T, max rv,
// -min T, -min rv} as ordered integers (non-negative values compare like their bit patterns)
template <class S>
__global__ void thermo_scan_kernel(const S* __restrict__ T, const S* __restrict__ rv, int64_t n,
                                   unsigned long long* __restrict__ out, int* __restrict__ bad) {
  double mx[2] = {-1e300, -1e300}, mn[2] = {1e300, 1e300};
  int nf = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const double a = (double)T[c], b = (double)rv[c];
    if (!isfinite(a) || !isfinite(b)) nf = 1;
    mx[0] = fmax(mx[0], a);
    mx[1] = fmax(mx[1], b);
    mn[0] = fmin(mn[0], a);
    mn[1] = fmin(mn[1], b);
  }
  if (nf) atomicOr(bad, 1);
  // only the signs the checks need: T > 0 and rho_v >= 0 everywhere, and the largest rho_v
  if (mn[0] <= 0.0 || mn[1] < 0.0) atomicOr(bad, 2);
  if (mx[1] > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mx[1]));
}

template <class R>
__global__ void fill_kernel(R* __restrict__ p, int64_t n, R v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// a temperature as the mixed state's pair (hi, lo) with no diameter residual
__host__ __device__ inline float4 pack_temp(double T) {
  const float hi = (float)T;
  return make_float4(hi, (float)(T - (double)hi), 0.0f, 0.0f);
}

template <class R>
__global__ void gather_temp_kernel(const R* __restrict__ src, R* __restrict__ dst, const uint32_t* __restrict__ perm,
                                   int64_t n, const int* __restrict__ gate, int want) {
  if (gate && ((*gate != 0) ? 1 : 0) != want) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}

__global__ void temp_io_f64_kernel(double* __restrict__ T, int64_t first, int64_t n, double* __restrict__ out,
                                   const double* __restrict__ in) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (in)
      T[first + i] = in[i];
    else
      out[i] = T[first + i];
  }
}

// mixed: the temperature is T_hi + T_lo; setting it keeps the diameter residual
__global__ void temp_io_mixed_kernel(float4* __restrict__ ms, int64_t first, int64_t n, double* __restrict__ out,
                                     const double* __restrict__ in) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (in) {
      float4 v = pack_temp(in[i]);
      v.z = ms[first + i].z;
      ms[first + i] = v;
    } else {
      const float4 v = ms[first + i];
      out[i] = (double)v.x + (double)v.y;
    }
  }
}

// carry propagation of the carry-save accumulator: digits [0, 2^32) below a signed top word
__global__ void wide_normalize_kernel(long long* __restrict__ w, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    long long* v = w + i * kWideWords;
    long long carry = 0;
    for (int k = 0; k < kWideWords - 1; ++k) {
      const long long t = v[k] + carry;
      v[k] = t & 0xffffffffll;
      carry = t >> 32;  // arithmetic shift: floor division by 2^32
    }
    v[kWideWords - 1] += carry;
  }
}

// per-block partial sums of m and C_p m T (FP64), summed on the host in block order; mixed handles
// add the diameter residual and the temperature's low part
template <class R, class S>
__global__ void micro_sums_kernel(const R* __restrict__ d, const S* __restrict__ T, int64_t n, double mcoef,
                                  double cp, double* __restrict__ part) {
  __shared__ double s[2][kMicroThreads];
  double m = 0.0, e = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double dd, t;
    if constexpr (std::is_same<S, float4>::value) {
      const float4 v = T[i];
      dd = (double)d[i] + (double)v.z;
      t = (double)v.x + (double)v.y;
    } else {
      dd = (double)d[i];
      t = (double)T[i];
    }
    const double mi = mcoef * dd * dd * dd;
    m += mi;
    e += cp * mi * t;
  }
  s[0][threadIdx.x] = m;
  s[1][threadIdx.x] = e;
  __syncthreads();
  for (int off = kMicroThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      s[0][threadIdx.x] += s[0][threadIdx.x + off];
      s[1][threadIdx.x] += s[1][threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s[0][0];
    part[2 * blockIdx.x + 1] = s[1][0];
  }
}

int blocks_for(int64_t n, int cap = 152 * 16) {
  int64_t b = (n + kMicroThreads - 1) / kMicroThreads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

template <class R>
MicroConst<R> micro_const(const st_ctx* h) {
  MicroConst<R> c;
  const double pi = 3.14159265358979323846;
  c.Dv = (R)h->mi_Dv;
  c.kappa = (R)h->mi_kappa;
  c.cp = (R)h->mi_cp;
  c.L = (R)h->mi_L;
  c.nu_coef = (R)(0.6 * std::cbrt(h->mi_Pr));
  c.dmin = (R)h->mi_dmin;
  c.dq_coef = (R)(8.0 * h->mi_Dv / h->rho_p);
  c.mdrop = (R)(h->rho_p * pi / 6.0);
  c.mcoef = (R)(h->mult * h->rho_p * pi / 6.0);
  c.re_coef = (R)(h->rho_f_drag / h->mu);
  return c;
}

size_t temp_elem(const st_ctx* h) { return h->prec == ST_FP64 ? sizeof(double) : sizeof(float4); }

}  // namespace

cudaError_t launch_micro_step(st_ctx* h, const StepParams& p, bool records) {
  const int64_t warps = (h->np + 31) / 32;
  const int blocks = blocks_for(warps * 32);
  if (h->prec == ST_FP64) {
    F64Args a;
    a.s = carve_f64(h->state.p, h->cap);
    a.T = (double*)h->temp.p;
    a.U = (const D4*)h->fluid.p;
    a.th = (const double2*)h->thermo.p;
    a.acc = (long long*)h->acc.p;
    a.macc = (long long*)h->acc_micro.p;
    a.n = h->np;
    a.ncell = h->geo.ncell;
    a.nx = h->geo.n[0];
    a.ny = h->geo.n[1];
    a.nz = h->geo.n[2];
    for (int q = 0; q < 3; ++q) {
      a.L[q] = h->geo.L[q];
      a.invL[q] = 1.0 / h->geo.L[q];
      a.inv_h[q] = h->geo.inv_h[q];
      a.g[q] = p.g[q];
    }
    a.dt = p.dt;
    a.inv_ca = 1.0 / p.ca;
    a.E = p.E;
    a.c = micro_const<double>(h);
    micro_f64_kernel<<<blocks, kMicroThreads, 0, h->stream>>>(a);
  } else {
    const bool bf = h->prec == ST_MIXED_BF16V;
    MixedArgs a;
    a.s = carve_mixed(h->state.p, h->cap, bf);
    a.ms = (float4*)h->temp.p;
    a.Up = (const float4*)h->fluid_pad.p;
    a.thp = (const float2*)h->thermo.p;
    a.acc = (long long*)h->acc.p;
    a.macc = (long long*)h->acc_micro.p;
    a.rec = records ? (float4*)h->state_alt.p : nullptr;
    a.n = h->np;
    a.ncell = h->geo.ncell;
    a.nx = h->geo.n[0];
    a.ny = h->geo.n[1];
    a.nz = h->geo.n[2];
    for (int q = 0; q < 3; ++q) {
      a.inv_h[q] = (float)h->geo.inv_h[q];
      a.g[q] = (float)p.g[q];
      a.gdt[q] = (float)(p.g[q] * p.dt);
    }
    a.dt = (float)p.dt;
    a.inv_ca = (float)(1.0 / p.ca);
    a.E = p.E;
    a.c = micro_const<float>(h);
    if (bf)
      micro_mixed_kernel<true><<<blocks, kMicroThreads, 0, h->stream>>>(a);
    else
      micro_mixed_kernel<false><<<blocks, kMicroThreads, 0, h->stream>>>(a);
  }
  h->launches += 1;
  return cudaGetLastError();
}

st_status micro_prepare_step(st_ctx* h, double dt) {
  // one step can grow d^2 by at most 8 D_v rho_v,max dt / rho_p (rho_sat >= 0): the diameter bound
  // the momentum accumulator's exponent is chosen from
  const double grow = 8.0 * h->mi_Dv * h->rv_max * dt / h->rho_p;
  h->dmax = std::sqrt(h->dmax * h->dmax + grow);
  // each particle adds at most one digit to any word per step
  if (h->micro_adds + (double)h->np > 1073741824.0) {
    const int64_t m = 2 * h->geo.ncell;
    wide_normalize_kernel<<<blocks_for(m), kMicroThreads, 0, h->stream>>>((long long*)h->acc_micro.p, m);
    h->launches += 1;
    ST_TRY(cuda_check(h, cudaGetLastError(), "normalise microphysics sources"));
    h->micro_adds = 1.0;
  }
  h->micro_adds += (double)h->np;
  return ST_OK;
}

cudaError_t launch_gather_temp(st_ctx* h, const uint32_t* perm, const int* gate, int want) {
  if (!h->temp.p || !h->temp_alt.p) return cudaSuccess;
  const int b = blocks_for(h->np);
  if (h->prec == ST_FP64)
    gather_temp_kernel<double><<<b, kMicroThreads, 0, h->stream>>>((const double*)h->temp.p,
                                                                    (double*)h->temp_alt.p, perm, h->np, gate, want);
  else
    gather_temp_kernel<float4><<<b, kMicroThreads, 0, h->stream>>>((const float4*)h->temp.p,
                                                                    (float4*)h->temp_alt.p, perm, h->np, gate, want);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_fill_temp(st_ctx* h, int64_t first, int64_t n, double T) {
  if (!h->temp.p || n <= 0) return cudaSuccess;
  if (h->prec == ST_FP64)
    fill_kernel<double><<<blocks_for(n), kMicroThreads, 0, h->stream>>>((double*)h->temp.p + first, n, T);
  else
    fill_kernel<float4><<<blocks_for(n), kMicroThreads, 0, h->stream>>>((float4*)h->temp.p + first, n, pack_temp(T));
  h->launches += 1;
  return cudaGetLastError();
}

}  // namespace st

using namespace st;

namespace {
// the particle-temperature arrays (and the microphysics accumulator) sized for the handle's capacity;
// existing temperatures are kept
st_status ensure_micro_buffers(st_ctx* h) {
  const size_t esz = temp_elem(h);
  const size_t need = (size_t)std::max<int64_t>(h->cap, 64) * esz;
  if (h->temp.bytes < need) {
    Buf nt, na;
    ST_TRY(dev_alloc(h, nt, need));
    st_status s = dev_alloc(h, na, need);
    if (s != ST_OK) {
      dev_free(h, nt);
      return s;
    }
    if (h->temp.p && h->np > 0) {
      cudaError_t e = cudaMemcpyAsync(nt.p, h->temp.p, (size_t)h->np * esz, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) {
        dev_free(h, nt);
        dev_free(h, na);
        return cuda_check(h, e, "grow particle temperatures");
      }
    }
    dev_free(h, h->temp);
    dev_free(h, h->temp_alt);
    h->temp = nt;
    h->temp_alt = na;
  }
  if (!h->acc_micro.p) {
    ST_TRY(dev_alloc(h, h->acc_micro, (size_t)2 * h->geo.ncell * kWideWords * sizeof(long long)));
    ST_TRY(cuda_check(h, cudaMemsetAsync(h->acc_micro.p, 0, h->acc_micro.bytes, h->stream), "clear sources"));
    h->micro_adds = 0.0;
  }
  return ST_OK;
}
}  // namespace

namespace st {
st_status micro_grow(st_ctx* h) { return h->micro_on ? ensure_micro_buffers(h) : ST_OK; }
}  // namespace st

extern "C" {

st_status st_set_microphysics(st_handle h, int enable, double D_v, double kappa_f, double cp_p, double latent_heat,
                              double prandtl, double d_min, double T_init) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  ST_TRY(cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice"));
  if (!enable) {
    h->micro_on = false;
    return ST_OK;
  }
  // chunks carry the state without the particle temperatures
  if (h->chunks) return set_error(h, ST_ERR_STATE, "microphysics and chunks do not combine");
  const double v[7] = {D_v, kappa_f, cp_p, latent_heat, prandtl, d_min, T_init};
  for (double x : v)
    if (!std::isfinite(x)) return set_error(h, ST_ERR_NONFINITE, "non-finite microphysics parameter");
  if (!(D_v >= 0) || !(kappa_f > 0) || !(cp_p > 0) || !(latent_heat >= 0) || !(prandtl > 0) || !(d_min > 0) ||
      !(T_init > 0))
    return set_error(h, ST_ERR_INVALID_ARG,
                     "need D_v >= 0, kappa_f > 0, cp_p > 0, latent_heat >= 0, prandtl > 0, d_min > 0, T_init > 0");
  const bool was_on = h->micro_on;
  h->mi_Dv = D_v;
  h->mi_kappa = kappa_f;
  h->mi_cp = cp_p;
  h->mi_L = latent_heat;
  h->mi_Pr = prandtl;
  h->mi_dmin = d_min;
  h->mi_Tinit = T_init;
  const bool had_temps = h->temp.p != nullptr;
  ST_TRY(ensure_micro_buffers(h));
  h->micro_on = true;
  h->adj_ready = false;
  // particles that never had a temperature take T_init
  if (!was_on && !had_temps && h->np > 0) {
    ST_TRY(cuda_check(h, launch_fill_temp(h, 0, h->np, T_init), "particle temperatures"));
  }
  return ST_OK;
}

st_status st_set_thermo(st_handle h, const void* T, const void* rho_v, int dtype, int on_device) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  ST_TRY(cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice"));
  if (!T || !rho_v) return set_error(h, ST_ERR_INVALID_ARG, "T and rho_v are required");
  if (dtype != ST_DTYPE_F32 && dtype != ST_DTYPE_F64) return set_error(h, ST_ERR_INVALID_ARG, "bad dtype");
  const int64_t nc = h->geo.ncell;
  const size_t esz = dtype == ST_DTYPE_F64 ? 8 : 4;
  Buf tmp;
  const void* dT = T;
  const void* dR = rho_v;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, 2 * nc * esz));
    cudaError_t e = cudaMemcpyAsync(tmp.p, T, nc * esz, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char*)tmp.p + nc * esz, rho_v, nc * esz, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      dev_free(h, tmp);
      return cuda_check(h, e, "copy thermo fields");
    }
    dT = tmp.p;
    dR = (const char*)tmp.p + nc * esz;
  }
  const bool f64h = h->prec == ST_FP64;
  const size_t padded = (size_t)(h->geo.n[0] + 2 * kFluidPad) * (h->geo.n[1] + 2 * kFluidPad) *
                        (h->geo.n[2] + 2 * kFluidPad);
  st_status s = ensure(h, h->thermo, f64h ? (size_t)nc * sizeof(double2) : padded * sizeof(float2));
  unsigned long long* red = (unsigned long long*)h->red.p;
  int* bad = (int*)(red + 1);
  cudaError_t e = cudaSuccess;
  if (s == ST_OK) e = cudaMemsetAsync(red, 0, 16, h->stream);
  if (s == ST_OK && e == cudaSuccess) {
    const int b = blocks_for(nc, 152 * 4);
    if (dtype == ST_DTYPE_F64)
      thermo_scan_kernel<double><<<b, kMicroThreads, 0, h->stream>>>((const double*)dT, (const double*)dR, nc, red,
                                                                      bad);
    else
      thermo_scan_kernel<float><<<b, kMicroThreads, 0, h->stream>>>((const float*)dT, (const float*)dR, nc, red, bad);
    h->launches += 1;
    e = cudaGetLastError();
  }
  unsigned long long hb[2] = {0, 0};
  if (s == ST_OK && e == cudaSuccess) e = cudaMemcpyAsync(hb, red, 16, cudaMemcpyDeviceToHost, h->stream);
  if (s == ST_OK && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  const int flags = (int)(hb[1] & 0xffffffffull);
  if (s == ST_OK && e == cudaSuccess && flags == 0) {
    const int b = blocks_for(f64h ? nc : (int64_t)padded);
    if (f64h) {
      if (dtype == ST_DTYPE_F64)
        thermo_pack_f64_kernel<double><<<b, kMicroThreads, 0, h->stream>>>((const double*)dT, (const double*)dR,
                                                                            (double2*)h->thermo.p, nc);
      else
        thermo_pack_f64_kernel<float><<<b, kMicroThreads, 0, h->stream>>>((const float*)dT, (const float*)dR,
                                                                           (double2*)h->thermo.p, nc);
    } else {
      if (dtype == ST_DTYPE_F64)
        thermo_pack_padded_kernel<double><<<b, kMicroThreads, 0, h->stream>>>(
            (const double*)dT, (const double*)dR, (float2*)h->thermo.p, h->geo.n[0], h->geo.n[1], h->geo.n[2]);
      else
        thermo_pack_padded_kernel<float><<<b, kMicroThreads, 0, h->stream>>>(
            (const float*)dT, (const float*)dR, (float2*)h->thermo.p, h->geo.n[0], h->geo.n[1], h->geo.n[2]);
    }
    h->launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  dev_free(h, tmp);
  ST_TRY(s);
  ST_TRY(cuda_check(h, e, "set thermo fields"));
  if (flags & 1) return set_error(h, ST_ERR_NONFINITE, "thermo fields hold NaN or Inf");
  if (flags & 2) return set_error(h, ST_ERR_INVALID_ARG, "need T > 0 and rho_v >= 0 in every cell");
  h->rv_max = 0.0;
  if (hb[0]) std::memcpy(&h->rv_max, &hb[0], sizeof(double));
  h->thermo_set = true;
  return ST_OK;
}

st_status st_set_temperatures(st_handle h, int64_t first, int64_t count, const double* T, int on_device) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  ST_TRY(cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice"));
  if (!h->micro_on) return set_error(h, ST_ERR_STATE, "microphysics is off");
  if (first < 0 || count < 0 || first + count > h->np) return set_error(h, ST_ERR_INVALID_ARG, "range");
  if (count == 0) return ST_OK;
  if (!T) return set_error(h, ST_ERR_INVALID_ARG, "T is NULL");
  ST_TRY(materialize_state(h));
  Buf tmp;
  const double* src = T;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, (size_t)count * 8));
    cudaError_t e = cudaMemcpyAsync(tmp.p, T, (size_t)count * 8, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      dev_free(h, tmp);
      return cuda_check(h, e, "copy temperatures");
    }
    src = (const double*)tmp.p;
  }
  double mx = 0.0;
  int nf = 0;
  cudaError_t e = launch_maxabs(h, src, count, ST_DTYPE_F64, &mx, &nf);
  if (e == cudaSuccess && !nf) {
    if (h->prec == ST_FP64)
      temp_io_f64_kernel<<<blocks_for(count), kMicroThreads, 0, h->stream>>>((double*)h->temp.p, first, count,
                                                                              nullptr, src);
    else
      temp_io_mixed_kernel<<<blocks_for(count), kMicroThreads, 0, h->stream>>>((float4*)h->temp.p, first, count,
                                                                                nullptr, src);
    h->launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  dev_free(h, tmp);
  ST_TRY(cuda_check(h, e, "set temperatures"));
  if (nf) return set_error(h, ST_ERR_NONFINITE, "temperatures hold NaN or Inf");
  return ST_OK;
}

st_status st_get_temperatures(st_handle h, int64_t first, int64_t count, double* T, int on_device) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  ST_TRY(cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice"));
  if (!h->temp.p) return set_error(h, ST_ERR_STATE, "no particle temperatures (microphysics never enabled)");
  if (first < 0 || count < 0 || first + count > h->np) return set_error(h, ST_ERR_INVALID_ARG, "range");
  if (count == 0) return ST_OK;
  if (!T) return set_error(h, ST_ERR_INVALID_ARG, "T is NULL");
  Buf tmp;
  double* dst = T;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, (size_t)count * 8));
    dst = (double*)tmp.p;
  }
  if (h->prec == ST_FP64)
    temp_io_f64_kernel<<<blocks_for(count), kMicroThreads, 0, h->stream>>>((double*)h->temp.p, first, count, dst,
                                                                            nullptr);
  else
    temp_io_mixed_kernel<<<blocks_for(count), kMicroThreads, 0, h->stream>>>((float4*)h->temp.p, first, count, dst,
                                                                              nullptr);
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(T, dst, (size_t)count * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  return cuda_check(h, e, "get temperatures");
}

st_status st_get_micro_sources(st_handle h, double* out, int reset, int on_device) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  ST_TRY(cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice"));
  if (!out) return set_error(h, ST_ERR_INVALID_ARG, "out is NULL");
  const int64_t m = 2 * h->geo.ncell;
  Buf tmp;
  double* dst = out;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, (size_t)m * 8));
    dst = (double*)tmp.p;
  }
  cudaError_t e = cudaSuccess;
  if (h->acc_micro.p) {
    e = launch_wide_to_f64(h, (const long long*)h->acc_micro.p, dst, m);
    if (e == cudaSuccess && reset) {
      e = cudaMemsetAsync(h->acc_micro.p, 0, h->acc_micro.bytes, h->stream);
      h->micro_adds = 0.0;
    }
  } else {
    e = cudaMemsetAsync(dst, 0, (size_t)m * 8, h->stream);
  }
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dst, (size_t)m * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  return cuda_check(h, e, "get microphysics sources");
}

st_status st_micro_invariants(st_handle h, double out[2]) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  ST_TRY(cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice"));
  if (!out) return set_error(h, ST_ERR_INVALID_ARG, "out is NULL");
  out[0] = out[1] = 0.0;
  if (!h->temp.p || h->np == 0) return ST_OK;
  ST_TRY(materialize_state(h));
  const int b = blocks_for(h->np, 1024);
  double* part = (double*)h->red.p;  // 2 x 1024 doubles fit the 64 KiB reduction buffer
  const double mcoef = h->mult * h->rho_p * 3.14159265358979323846 / 6.0;
  if (h->prec == ST_FP64)
    micro_sums_kernel<double, double><<<b, kMicroThreads, 0, h->stream>>>(
        carve_f64(h->state.p, h->cap).d, (const double*)h->temp.p, h->np, mcoef, h->mi_cp, part);
  else
    micro_sums_kernel<float, float4><<<b, kMicroThreads, 0, h->stream>>>(
        carve_mixed(h->state.p, h->cap, h->prec == ST_MIXED_BF16V).d, (const float4*)h->temp.p, h->np, mcoef,
        h->mi_cp, part);
  h->launches += 1;
  std::vector<double> hp(2 * b);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, 2 * b * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  ST_TRY(cuda_check(h, e, "microphysics invariants"));
  for (int i = 0; i < b; ++i) {
    out[0] += hp[2 * i];
    out[1] += hp[2 * i + 1];
  }
  return ST_OK;
}

}  // extern "C"
