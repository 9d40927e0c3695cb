// Hand-written adjoint of the Lagrangian step (FP64 handles in FP64, mixed FP32-velocity handles in
// FP32), run backward through checkpointed segments with recomputation.
//
// For a loss L(Jtot) of the time-summed per-cell source, with
// lam = dL/dJtot given per cell, one reverse step of one particle runs the
// chain rule backward through the forward step
//   c0 = cell(x);  u_p = sum_corners W(f) U;  a = 18 mu alpha / (rho_p d^2)
//   E = e^{-a dt};  E1 = 1 - E;  Q = E1 / a;  w = u_p + g / a
//   v' = w E1 + v E;  x' = x + w (dt - Q) + v Q
//   J = -m (v' - v - g dt),  m = mult rho_p pi d^3 / 6,  Jtot[c0] += J
// with the deposit cell held fixed (its derivative is zero almost everywhere)
// and the periodic wrap a translation.  With the cloud-in-cell deposit
// (Jtot[corner] += W(f) J over the gather's stencil) the adjoint of J is the
// W-weighted sum of lam over the corners, and the weights' derivatives add
// lam_corner . J to the stencil-fraction adjoint beside the gather's term.  Per particle it carries the adjoints
// of x and v between steps and accumulates dL/dd; dL/dalpha is reduced
// per block in a fixed order; dL/dU is scattered through the transposed
// trilinear weights into an exact carry-save fixed-point accumulator, so
// every output is independent of thread scheduling.
#include "st_common.cuh"

namespace st {
namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjDirectGroups = 20;  // more distinct stencils than this in a warp: no grouping

struct AdjArgs {
  const double* __restrict__ x[3];   // state at the start of the step (tape)
  const double* __restrict__ v[3];
  const double* __restrict__ d;
  double* __restrict__ xb[3];        // adjoint of the state after the step (in), before it (out)
  double* __restrict__ vb[3];
  double* __restrict__ db;           // accumulated dL/dd
  double* __restrict__ ab_part;      // [gridDim.x] dL/dalpha partial sums, accumulated over steps
  const D4* __restrict__ U;
  const double* __restrict__ lam;    // [3][ncell]
  long long* __restrict__ Uw;        // [ncell][3][kWideWords] carry-save dL/dU
  int64_t n, ncell;
  int nx, ny, nz;
  double inv_h[3];
  double dt, ca, mcoef, alpha, g[3];
  double inv_ca, inv_alpha;  // 1 / ca, 1 / alpha
};

__device__ __forceinline__ D4 ld_cell(const D4* __restrict__ U, int64_t c) {
  const double2* p = reinterpret_cast<const double2*>(U + c);
  double2 a = __ldg(p), b = __ldg(p + 1);
  return D4{a.x, a.y, b.x, b.y};
}

// CIC: the cloud-in-cell deposit (else the containing cell)
template <bool CIC>
__global__ void __launch_bounds__(kAdjThreads) adjoint_step_kernel(const AdjArgs a) {
  const int n3[3] = {a.nx, a.ny, a.nz};
  double alphab_sum = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    double x[3], v[3], xb[3], vb[3];
    for (int q = 0; q < 3; ++q) {
      x[q] = a.x[q][p];
      v[q] = a.v[q][p];
      xb[q] = a.xb[q][p];
      vb[q] = a.vb[q][p];
    }
    const double d = a.d[p];
    // recompute the forward intermediates
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
    const int64_t key = c0[0] + (int64_t)a.nx * (c0[1] + (int64_t)a.ny * c0[2]);
    int64_t corner[8];
    D4 Uc[8];
    for (int k = 0; k < 8; ++k) {
      const int di = k & 1, dj = (k >> 1) & 1, dk = (k >> 2) & 1;
      corner[k] = (di ? i1[0] : i0[0]) + (int64_t)a.nx * ((dj ? i1[1] : i0[1]) + (int64_t)a.ny * (dk ? i1[2] : i0[2]));
      Uc[k] = ld_cell(a.U, corner[k]);
    }
    double up[3] = {0.0, 0.0, 0.0};
    double W[8];
    for (int k = 0; k < 8; ++k) {
      const int di = k & 1, dj = (k >> 1) & 1, dk = (k >> 2) & 1;
      W[k] = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
      up[0] += W[k] * Uc[k].x;
      up[1] += W[k] * Uc[k].y;
      up[2] += W[k] * Uc[k].z;
    }
    const double dd = d * d;
    // the reciprocals once (GB300 divides in FP64 by iteration): 1/a, 1/a^2, 1/d
    const double inv_ra = dd * a.inv_ca;
    const double ra = 1.0 / inv_ra;
    const double inv_ra2 = inv_ra * inv_ra;
    const double inv_d = 1.0 / d;
    const double E1 = -expm1(-ra * a.dt);
    const double E = 1.0 - E1;  // e^{-a dt} as the complement of expm1, as in the forward step
    const double Q = E1 * inv_ra;
    const double m = a.mcoef * dd * d;
    double wt[3], vn[3];
    for (int q = 0; q < 3; ++q) {
      wt[q] = up[q] + a.g[q] * inv_ra;
      vn[q] = wt[q] + (v[q] - wt[q]) * E;
    }
    // reverse sweep
    double Jb[3];
    double lj[CIC ? 8 : 1];  // cloud in cell: lam at each corner dotted with J
    if constexpr (CIC) {
      double J[3];
      for (int q = 0; q < 3; ++q) J[q] = -m * (vn[q] - v[q] - a.g[q] * a.dt);
      Jb[0] = Jb[1] = Jb[2] = 0.0;
      for (int k = 0; k < 8; ++k) {
        const double l0 = a.lam[corner[k]], l1 = a.lam[a.ncell + corner[k]], l2 = a.lam[2 * a.ncell + corner[k]];
        Jb[0] += W[k] * l0;
        Jb[1] += W[k] * l1;
        Jb[2] += W[k] * l2;
        lj[k] = l0 * J[0] + l1 * J[1] + l2 * J[2];
      }
    } else {
      Jb[0] = a.lam[key];
      Jb[1] = a.lam[a.ncell + key];
      Jb[2] = a.lam[2 * a.ncell + key];
    }
    double mb = 0.0, Eb = 0.0, E1b = 0.0, Qb = 0.0, ab = 0.0;
    double ub[3], vsb[3];
    for (int q = 0; q < 3; ++q) {
      const double vnb = vb[q] - m * Jb[q];
      vsb[q] = m * Jb[q] + vnb * E + xb[q] * Q;
      mb -= (vn[q] - v[q] - a.g[q] * a.dt) * Jb[q];
      const double wtb = vnb * E1 + xb[q] * (a.dt - Q);
      E1b += vnb * wt[q];
      Eb += vnb * v[q];
      Qb += xb[q] * (v[q] - wt[q]);
      ub[q] = wtb;
      ab -= wtb * a.g[q] * inv_ra2;
    }
    E1b += Qb * inv_ra;
    ab -= Qb * E1 * inv_ra2;
    ab += a.dt * E * (E1b - Eb);
    alphab_sum += ab * ra * a.inv_alpha;
    double dbv = a.db[p] + ab * (-2.0 * ra * inv_d) + mb * 3.0 * m * inv_d;
    a.db[p] = dbv;
    // transposed trilinear weights: dL/dU (each corner's weight times ub) and dL/df, the
    // derivative of the trilinear form of the corner values' dot products with ub (plus, for the
    // cloud-in-cell deposit, lam . J at the corner), taken separably (differences along one
    // axis, interpolated along the other two)
    double dot[8];
    for (int k = 0; k < 8; ++k) {
      dot[k] = Uc[k].x * ub[0] + Uc[k].y * ub[1] + Uc[k].z * ub[2];
      if constexpr (CIC) dot[k] += lj[k];
      long long* w = a.Uw + corner[k] * 3 * kWideWords;
      wide_add(w, W[k] * ub[0]);
      wide_add(w + kWideWords, W[k] * ub[1]);
      wide_add(w + 2 * kWideWords, W[k] * ub[2]);
    }
    // corner k = di + 2 dj + 4 dk; lerp(p, q, t) = p + t (q - p)
    auto lerp = [](double p0, double p1, double t) { return p0 + t * (p1 - p0); };
    double fb[3];
    {
      // d/df_x: x-differences at the four (dj, dk) edges, interpolated in y then z
      const double e00 = dot[1] - dot[0], e10 = dot[3] - dot[2], e01 = dot[5] - dot[4], e11 = dot[7] - dot[6];
      fb[0] = lerp(lerp(e00, e10, f[1]), lerp(e01, e11, f[1]), f[2]);
      // d/df_y: y-differences, interpolated in x then z
      const double g00 = dot[2] - dot[0], g10 = dot[3] - dot[1], g01 = dot[6] - dot[4], g11 = dot[7] - dot[5];
      fb[1] = lerp(lerp(g00, g10, f[0]), lerp(g01, g11, f[0]), f[2]);
      // d/df_z: z-differences, interpolated in x then y
      const double h00 = dot[4] - dot[0], h10 = dot[5] - dot[1], h01 = dot[6] - dot[2], h11 = dot[7] - dot[3];
      fb[2] = lerp(lerp(h00, h10, f[0]), lerp(h01, h11, f[0]), f[1]);
    }
    for (int q = 0; q < 3; ++q) {
      a.xb[q][p] = xb[q] + fb[q] * a.inv_h[q];
      a.vb[q][p] = vsb[q];
    }
  }
  // fixed-order block reduction of dL/dalpha
  __shared__ double sh[kAdjThreads / 32];
  double s = alphab_sum;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) t += sh[w];
    a.ab_part[blockIdx.x] += t;
  }
}

// ---- the FP32 adjoint of the mixed-precision step ----
//
// The same reverse sweep in FP32 on the mixed state: the tape gives the start-of-step cell, the
// offsets in it and the velocity; the trilinear stencil is the forward kernel's (base cell and
// fractions from the offset, corners read from the ghost-padded FP32 field), the deposit cell the
// start cell.  Position adjoints are per metre, as in the FP64 adjoint (the periodic wrap and the
// whole-cell carry are translations).  Each step's dL/dd and dL/dalpha contributions are FP32 and
// accumulate in FP64.  The dL/dU products of the particles of a warp that share a stencil are summed
// in FP32 (in an order fixed by the stencils, so the result is reproducible) and each sum is added
// exactly: one set of L2 reduction operations per distinct stencil instead of per particle.

struct AdjMixedArgs {
  MixedState tape;
  const float* __restrict__ d;
  float* __restrict__ xb[3];
  float* __restrict__ vb[3];
  double* __restrict__ db;
  double* __restrict__ ab_part;
  const float4* __restrict__ Up;     // ghost-padded field
  const float* __restrict__ lam;     // [3][ncell]
  long long* __restrict__ Uw;
  int64_t n, ncell;
  int nx, ny, nz;
  float inv_h[3];
  float dt, cadt, inv_ca, mcoef, g[3], gdt[3];
  double inv_alpha;
};

__global__ void __launch_bounds__(kAdjThreads) adjoint_mixed_kernel(const AdjMixedArgs a) {
  __shared__ GroupBuf<8> gb[kAdjThreads / 32];
  const int n3[3] = {a.nx, a.ny, a.nz};
  const int64_t row = a.nx + 2 * kFluidPad, slab = row * (a.ny + 2 * kFluidPad);
  const int lane = threadIdx.x & 31;
  GroupBuf<8>& b8 = gb[threadIdx.x >> 5];
  double alphab_sum = 0.0;
  // warp-uniform trip count: the dL/dU commits below are warp-collective
  for (int64_t wbase = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); wbase < a.n;
       wbase += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = wbase + lane;
    int key = -1;  // the stencil's lowest corner cell; -1: no particle on this lane
    float W[8], ub[3];
    if (p < a.n) {
      const int c = a.tape.cell[p];
      const int ci[3] = {cell_i(c), cell_j(c), cell_k(c)};
      float v[3], xb[3], vb[3], f[3];
      int i0[3], lo[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float o = a.tape.xi[q][p];
        v[q] = ((const float*)a.tape.v[q])[p];
        xb[q] = a.xb[q][p];
        vb[q] = a.vb[q][p];
        const bool up_half = o >= 0.5f;
        i0[q] = ci[q] - (up_half ? 0 : 1);  // -1 .. n - 1
        f[q] = o + (up_half ? -0.5f : 0.5f);
        lo[q] = i0[q] < 0 ? i0[q] + n3[q] : i0[q];
      }
      const float d = a.d[p];
      const int64_t cell_key = ci[0] + (int64_t)a.nx * (ci[1] + (int64_t)a.ny * ci[2]);
      key = lo[0] + a.nx * (lo[1] + a.ny * lo[2]);
      const float4* b = a.Up + (i0[0] + kFluidPad) + row * (i0[1] + kFluidPad) + slab * (i0[2] + kFluidPad);
      float4 Uc[8];
      float up[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int di = k & 1, dj = (k >> 1) & 1, dk = (k >> 2) & 1;
        Uc[k] = __ldg(b + di + row * dj + slab * dk);
        W[k] = (di ? f[0] : 1.0f - f[0]) * (dj ? f[1] : 1.0f - f[1]) * (dk ? f[2] : 1.0f - f[2]);
        up[0] = fmaf(W[k], Uc[k].x, up[0]);
        up[1] = fmaf(W[k], Uc[k].y, up[1]);
        up[2] = fmaf(W[k], Uc[k].z, up[2]);
      }
      const float dd = d * d;
      const float adt = a.cadt / dd;     // a dt
      const float inv_ra = dd * a.inv_ca;  // 1 / a
      const float ra = 1.0f / inv_ra;
      const float inv_ra2 = inv_ra * inv_ra;
      const float inv_d = 1.0f / d;
      const float E1 = -expm1f(-adt);
      const float E = 1.0f - E1;
      const float Q = E1 * inv_ra;
      const float m = a.mcoef * dd * d;
      float wt[3], vn[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        wt[q] = fmaf(a.g[q], inv_ra, up[q]);
        vn[q] = fmaf(v[q] - wt[q], E, wt[q]);
      }
      const float Jb[3] = {a.lam[cell_key], a.lam[a.ncell + cell_key], a.lam[2 * a.ncell + cell_key]};
      float mb = 0.0f, Eb = 0.0f, E1b = 0.0f, Qb = 0.0f, ab = 0.0f;
      float vsb[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float vnb = vb[q] - m * Jb[q];
        vsb[q] = fmaf(m, Jb[q], fmaf(vnb, E, xb[q] * Q));
        mb -= ((vn[q] - v[q]) - a.gdt[q]) * Jb[q];
        const float wtb = fmaf(vnb, E1, xb[q] * (a.dt - Q));
        E1b = fmaf(vnb, wt[q], E1b);
        Eb = fmaf(vnb, v[q], Eb);
        Qb = fmaf(xb[q], v[q] - wt[q], Qb);
        ub[q] = wtb;
        ab -= wtb * a.g[q] * inv_ra2;
      }
      E1b = fmaf(Qb, inv_ra, E1b);
      ab -= Qb * E1 * inv_ra2;
      ab = fmaf(a.dt * E, E1b - Eb, ab);
      alphab_sum += (double)(ab * ra) * a.inv_alpha;
      a.db[p] += (double)(ab * (-2.0f * ra * inv_d) + mb * 3.0f * m * inv_d);
      float dot[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) dot[k] = fmaf(Uc[k].x, ub[0], fmaf(Uc[k].y, ub[1], Uc[k].z * ub[2]));
      auto lerp = [](float p0, float p1, float t) { return fmaf(t, p1 - p0, p0); };
      float fb[3];
      {
        const float e00 = dot[1] - dot[0], e10 = dot[3] - dot[2], e01 = dot[5] - dot[4], e11 = dot[7] - dot[6];
        fb[0] = lerp(lerp(e00, e10, f[1]), lerp(e01, e11, f[1]), f[2]);
        const float g00 = dot[2] - dot[0], g10 = dot[3] - dot[1], g01 = dot[6] - dot[4], g11 = dot[7] - dot[5];
        fb[1] = lerp(lerp(g00, g10, f[0]), lerp(g01, g11, f[0]), f[2]);
        const float h00 = dot[4] - dot[0], h10 = dot[5] - dot[1], h01 = dot[6] - dot[2], h11 = dot[7] - dot[3];
        fb[2] = lerp(lerp(h00, h10, f[0]), lerp(h01, h11, f[0]), f[1]);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        a.xb[q][p] = fmaf(fb[q], a.inv_h[q], xb[q]);
        a.vb[q][p] = vsb[q];
      }
    }
    // dL/dU, each corner's FP32 product added exactly.  Where the warp's particles share stencils (sorted
    // storage, several particles per cell) they are first reordered so that equal stencils are adjacent
    // (they share all eight corners) and each corner's products are summed over the group
    auto corners_of = [&](int k0, int (&corner)[8]) {
      const int l0 = k0 < 0 ? 0 : k0 % a.nx, r = k0 < 0 ? 0 : k0 / a.nx;
      const int l1 = r % a.ny, l2 = r / a.ny;
      const int h0 = l0 + 1 == a.nx ? 0 : l0 + 1, h1 = l1 + 1 == a.ny ? 0 : l1 + 1, h2 = l2 + 1 == a.nz ? 0 : l2 + 1;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        corner[k] = ((k & 1) ? h0 : l0) + a.nx * ((((k >> 1) & 1) ? h1 : l1) + a.ny * (((k >> 2) & 1) ? h2 : l2));
    };
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const int groups = __popc(__ballot_sync(0xffffffffu, (grp & ((1u << lane) - 1u)) == 0u));
    int corner[8];
    if (groups > kAdjDirectGroups) {
      // few shared stencils: the reordering and the sums would cost more than they save
      if (key >= 0) {
        corners_of(key, corner);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          long long* w = a.Uw + (int64_t)corner[k] * 3 * kWideWords;
          wide_add_f32(w, W[k] * ub[0]);
          wide_add_f32(w + kWideWords, W[k] * ub[1]);
          wide_add_f32(w + 2 * kWideWords, W[k] * ub[2]);
        }
      }
      continue;
    }
    const int slot = key_group_slot(lane, grp);
    const int gkey = group_permute_key(b8.key, slot, lane, key);
    corners_of(gkey, corner);
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
      float g[8];
      const float uq = q == 0 ? ub[0] : (q == 1 ? ub[1] : ub[2]);  // no local-memory indexing
#pragma unroll
      for (int k = 0; k < 8; ++k) g[k] = key >= 0 ? W[k] * uq : 0.0f;
      group_permute(b8, slot, lane, g);
      const bool head = run_sums(lane, gkey, g);
      if (head && gkey >= 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) wide_add_f32(a.Uw + ((int64_t)corner[k] * 3 + q) * kWideWords, g[k]);
      }
    }
  }
  __shared__ double sh[kAdjThreads / 32];
  double s = alphab_sum;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) t += sh[w];
    a.ab_part[blockIdx.x] += t;
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// value of each carry-save accumulator in FP64: out[c][q]
// carry propagation: digits in [0, 2^32) below a signed top word
__device__ __forceinline__ void wide_carry(long long* v) {
  long long c = 0;
  for (int k = 0; k < kWideWords - 1; ++k) {
    const long long t = v[k] + c;
    v[k] = t & 0xffffffffll;
    c = t >> 32;
  }
  v[kWideWords - 1] += c;
}

__global__ void wide_to_f64_kernel(const long long* __restrict__ Uw, double* __restrict__ out, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    // sign and magnitude first: summing signed words (a normalised negative value is words near 2^32
    // below a top word of -1) would cancel
    long long v[kWideWords];
    for (int k = 0; k < kWideWords; ++k) v[k] = Uw[i * kWideWords + k];
    wide_carry(v);
    const bool neg = v[kWideWords - 1] < 0;
    if (neg) {
      for (int k = 0; k < kWideWords; ++k) v[k] = -v[k];
      wide_carry(v);
    }
    // non-negative terms, smallest first
    double s = 0.0;
    for (int k = 0; k < kWideWords; ++k) s += ldexp((double)v[k], 32 * k + kWideBase);
    out[i] = neg ? -s : s;
  }
}

}  // namespace

cudaError_t launch_adjoint_step(st_ctx* h, const AdjointStepArgs& s) {
  AdjArgs a;
  for (int q = 0; q < 3; ++q) {
    a.x[q] = s.x[q];
    a.v[q] = s.v[q];
    a.xb[q] = s.xb[q];
    a.vb[q] = s.vb[q];
    a.inv_h[q] = h->geo.inv_h[q];
    a.g[q] = h->g[q];
  }
  a.d = s.d;
  a.db = s.db;
  a.ab_part = s.ab_part;
  a.U = (const D4*)h->fluid.p;
  a.lam = s.lam;
  a.Uw = s.Uw;
  a.n = h->np;
  a.ncell = h->geo.ncell;
  a.nx = h->geo.n[0];
  a.ny = h->geo.n[1];
  a.nz = h->geo.n[2];
  a.dt = s.dt;
  a.ca = 18.0 * h->mu * h->alpha / h->rho_p;
  a.mcoef = h->mult * h->rho_p * 3.14159265358979323846 / 6.0;
  a.alpha = h->alpha;
  a.inv_ca = 1.0 / a.ca;
  a.inv_alpha = 1.0 / h->alpha;
  if (h->phys_deposit == ST_DEPOSIT_CIC)
    adjoint_step_kernel<true><<<kAdjBlocks, kAdjThreads, 0, h->stream>>>(a);
  else
    adjoint_step_kernel<false><<<kAdjBlocks, kAdjThreads, 0, h->stream>>>(a);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_adjoint_step_mixed(st_ctx* h, const AdjointMixedArgs& s) {
  AdjMixedArgs a;
  a.tape = s.tape;
  a.d = s.d;
  for (int q = 0; q < 3; ++q) {
    a.xb[q] = s.xb[q];
    a.vb[q] = s.vb[q];
    a.inv_h[q] = (float)h->geo.inv_h[q];
    a.g[q] = (float)h->g[q];
    a.gdt[q] = (float)(h->g[q] * s.dt);
  }
  a.db = s.db;
  a.ab_part = s.ab_part;
  a.Up = (const float4*)h->fluid_pad.p;
  a.lam = s.lam32;
  a.Uw = s.Uw;
  a.n = h->np;
  a.ncell = h->geo.ncell;
  a.nx = h->geo.n[0];
  a.ny = h->geo.n[1];
  a.nz = h->geo.n[2];
  const double ca = 18.0 * h->mu * h->alpha / h->rho_p;
  a.dt = (float)s.dt;
  a.cadt = (float)(ca * s.dt);
  a.inv_ca = (float)(1.0 / ca);
  a.mcoef = (float)(h->mult * h->rho_p * 3.14159265358979323846 / 6.0);
  a.inv_alpha = 1.0 / h->alpha;
  adjoint_mixed_kernel<<<kAdjBlocks, kAdjThreads, 0, h->stream>>>(a);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(st_ctx* h, const double* in, float* out, int64_t m) {
  int64_t b = (m + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  f64_to_f32_kernel<<<(int)b, 256, 0, h->stream>>>(in, out, m);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_wide_to_f64(st_ctx* h, const long long* Uw, double* out, int64_t m) {
  int64_t b = (m + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  wide_to_f64_kernel<<<(int)b, 256, 0, h->stream>>>(Uw, out, m);
  h->launches += 1;
  return cudaGetLastError();
}

}  // namespace st
