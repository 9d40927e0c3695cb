// Mixed-precision Lagrangian step: int32 packed cell + FP32 in-cell offset,
// FP32 (or BF16) velocity, FP32 diameter; FP32 arithmetic.  Each lane owns 4
// consecutive particles, so every particle array is read and written with
// 128-bit (BF16 velocity: 64-bit) coalesced accesses; a warp covers 128
// particles.  Impulses are reduced over runs of equal start-of-step cell in
// storage order (lane-local suffix sums, then a segmented suffix scan across
// lanes) and each run is committed once to the exact fixed-point accumulator.
// The physics variants (nearest-grid-point gather, semi-implicit Euler,
// Schiller-Naumann drag) are uniform branches; the cloud-in-cell deposit is a
// template instance that runs the run-sum once per stencil corner.
#include "st_common.cuh"

namespace st {
namespace {

struct MixedArgs {
  MixedState s;
  const float4* __restrict__ U;
  long long* __restrict__ acc;
  int64_t n;
  int64_t ncell;
  int nx, ny, nz;
  float inv_h[3];
  float dt, cadt, inv_ca, mcoef;
  float g[3], gdt[3];
  int E;
  int ngp, semi, sn;  // nearest-grid-point gather, semi-implicit Euler, Schiller-Naumann drag
  float re_coef;      // rho_f / mu
};

__device__ __forceinline__ void lerp3(float4 a, float4 b, float f, float r[3]) {
  r[0] = fmaf(f, b.x - a.x, a.x);
  r[1] = fmaf(f, b.y - a.y, a.y);
  r[2] = fmaf(f, b.z - a.z, a.z);
}

__device__ __forceinline__ void commit(const MixedArgs& a, int key, float j0, float j1, float j2) {
  acc_add_f32(a.acc + kAccWords * key, j0, a.E);
  acc_add_f32(a.acc + kAccWords * (a.ncell + key), j1, a.E);
  acc_add_f32(a.acc + kAccWords * (2 * a.ncell + key), j2, a.E);
}

template <bool BF16>
__device__ __forceinline__ void load_v(const MixedArgs& a, int q, int64_t p0, float v[4]) {
  if (BF16) {
    uint2 r = __ldcs((const uint2*)((const __nv_bfloat16*)a.s.v[q] + p0));
    __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162*>(&r.x);
    __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162*>(&r.y);
    float2 l = __bfloat1622float2(lo), h = __bfloat1622float2(hi);
    v[0] = l.x;
    v[1] = l.y;
    v[2] = h.x;
    v[3] = h.y;
  } else {
    float4 r = __ldcs((const float4*)((const float*)a.s.v[q] + p0));
    v[0] = r.x;
    v[1] = r.y;
    v[2] = r.z;
    v[3] = r.w;
  }
}

template <bool BF16>
__device__ __forceinline__ void store_v(const MixedArgs& a, int q, int64_t p0, float v[4]) {
  if (BF16) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
    uint2 r;
    r.x = *reinterpret_cast<unsigned*>(&lo);
    r.y = *reinterpret_cast<unsigned*>(&hi);
    __stcs((uint2*)((__nv_bfloat16*)a.s.v[q] + p0), r);
  } else {
    __stcs((float4*)((float*)a.s.v[q] + p0), make_float4(v[0], v[1], v[2], v[3]));
  }
}

// round a velocity to its stored precision
template <bool BF16>
__device__ __forceinline__ float stored(float v) {
  if (BF16) return __bfloat162float(__float2bfloat16_rn(v));
  return v;
}

// periodic index for a particle that moved more than a box length in one step (rare)
__device__ __noinline__ int wrap_index_slow(int ii, int n) {
  ii %= n;
  return ii < 0 ? ii + n : ii;
}

// cell index after a move of 2^22 cells or more in one step (rare); the offset is set here too
__device__ __noinline__ int relocate_far(float& o, int ci, int n) {
  const float fl = floorf(o);
  o = fmaxf(fminf(o - fl, 0.99999994f), 0.0f);
  long long k = ((long long)ci + (long long)fl) % n;
  return (int)(k < 0 ? k + n : k);
}

// Sums J over runs of equal key in the warp's 128 particles (4 consecutive per lane) and commits
// each run once to the fixed-point accumulator: lane-local suffix sums, then a segmented suffix
// scan across lanes.  Negative keys are skipped.
__device__ __forceinline__ void deposit_runs(const MixedArgs& a, int lane, const int key[4], const float J[4][3]) {
  // lane-local suffix sums S_j over the run that starts at j
  float S[4][3];
#pragma unroll
  for (int q = 0; q < 3; ++q) S[3][q] = J[3][q];
#pragma unroll
  for (int j = 2; j >= 0; --j) {
    const bool same = key[j] == key[j + 1];
#pragma unroll
    for (int q = 0; q < 3; ++q) S[j][q] = J[j][q] + (same ? S[j + 1][q] : 0.0f);
  }
  // first element of the run that ends the lane (the lane's tail run)
  const int tail = (key[2] != key[3]) ? 3 : (key[1] != key[2]) ? 2 : (key[0] != key[1]) ? 1 : 0;
  const bool all_same = tail == 0;
  // link to the next lane: its leading run continues this lane's trailing run
  const int nk0 = __shfl_down_sync(0xffffffffu, key[0], 1);
  const int nall = __shfl_down_sync(0xffffffffu, (int)all_same, 1);
  float A[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) A[q] = __shfl_down_sync(0xffffffffu, S[0][q], 1);
  const bool link = (lane < 31) && (nk0 == key[3]) && (key[3] >= 0);
  int B = (link && nall) ? 1 : 0;
#pragma unroll
  for (int q = 0; q < 3; ++q) A[q] = link ? A[q] : 0.0f;
  // segmented suffix scan R_l = A_l + B_l R_{l+1}
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    float t0 = __shfl_down_sync(0xffffffffu, A[0], off);
    float t1 = __shfl_down_sync(0xffffffffu, A[1], off);
    float t2 = __shfl_down_sync(0xffffffffu, A[2], off);
    int tb = __shfl_down_sync(0xffffffffu, B, off);
    if (lane + off > 31) {
      tb = 0;
      t0 = t1 = t2 = 0.0f;
    }
    if (B) {
      A[0] += t0;
      A[1] += t1;
      A[2] += t2;
    }
    B = B & tb;
  }
  const int pk3 = __shfl_up_sync(0xffffffffu, key[3], 1);
  const bool head_lane = (lane == 0) || (pk3 != key[0]);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool start = (j == 0) ? head_lane : (key[j] != key[j - 1]);
    if (start && key[j] >= 0) {
      const bool to_end = j == tail;  // only the tail run continues into the next lane
      commit(a, key[j], S[j][0] + (to_end ? A[0] : 0.0f), S[j][1] + (to_end ? A[1] : 0.0f),
             S[j][2] + (to_end ? A[2] : 0.0f));
    }
  }
}

// Schiller-Naumann drag factor f = C_D Re / 24: 1 + 0.15 Re^0.687 up to Re = 1000, 0.44 Re / 24 above
__device__ __forceinline__ float sn_factor(float re) {
  return re <= 1000.0f ? fmaf(0.15f, powf(re, 0.687f), 1.0f) : (0.44f / 24.0f) * re;
}

template <bool BF16, bool CIC>
__global__ void __launch_bounds__(256) step_mixed_kernel(const MixedArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n3[3] = {a.nx, a.ny, a.nz};
  for (int64_t base = warp * 128; base < a.n; base += nwarp * 128) {
    const int64_t p0 = base + lane * 4;
    int key[4] = {-1, -1, -1, -1};
    float J[4][3];
    for (int j = 0; j < 4; ++j) J[j][0] = J[j][1] = J[j][2] = 0.0f;
    // cloud-in-cell deposit: the start-of-step stencil's lower corner (periodic) and weights
    int sb[CIC ? 4 : 1][3];
    float sf[CIC ? 4 : 1][3];
    {
      // pull the next iteration's particle lines towards L2 while this one computes
      const int64_t pn = p0 + nwarp * 128;
      if (pn < a.n) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.s.cell + pn));
        for (int q = 0; q < 3; ++q) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.s.xi[q] + pn));
        for (int q = 0; q < 3; ++q)
          asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)a.s.v[q] + pn * (BF16 ? 2 : 4)));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.s.d + pn));
      }
    }
    if (p0 < a.n) {
      // ---- load (128-bit, streaming) ----
      int4 c4 = __ldcs((const int4*)(a.s.cell + p0));
      float4 x4[3];
      for (int q = 0; q < 3; ++q) x4[q] = __ldcs((const float4*)(a.s.xi[q] + p0));
      float v[3][4];
      for (int q = 0; q < 3; ++q) load_v<BF16>(a, q, p0, v[q]);
      float4 d4 = __ldcs((const float4*)(a.s.d + p0));
      int cell[4] = {c4.x, c4.y, c4.z, c4.w};
      float xi[3][4];
      for (int q = 0; q < 3; ++q) {
        xi[q][0] = x4[q].x;
        xi[q][1] = x4[q].y;
        xi[q][2] = x4[q].z;
        xi[q][3] = x4[q].w;
      }
      float dv[4] = {d4.x, d4.y, d4.z, d4.w};
      const int nvalid = (int)min((int64_t)4, a.n - p0);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j < nvalid) {
          const int ci[3] = {cell_i(cell[j]), cell_j(cell[j]), cell_k(cell[j])};
          key[j] = ci[0] + a.nx * (ci[1] + a.ny * ci[2]);
          // trilinear stencil from (cell, offset): centres at offset 1/2; the field carries
          // kFluidPad ghost layers, so corner indices ii and ii + 1 (ii in [-1, n-1]) need no wrap
          int i0[3];
          float f[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float o = xi[q][j];
            const bool hi = o >= 0.5f;
            i0[q] = ci[q] - (hi ? 0 : 1) + kFluidPad;
            f[q] = o + (hi ? -0.5f : 0.5f);
            if (CIC) {
              const int lo = i0[q] - kFluidPad;
              sb[CIC ? j : 0][q] = lo < 0 ? lo + n3[q] : lo;
              sf[CIC ? j : 0][q] = f[q];
            }
          }
          const int64_t row = a.nx + 2 * kFluidPad, slab = row * (a.ny + 2 * kFluidPad);
          float up[3];
          if (a.ngp) {
            // nearest grid point: the value of the cell holding the particle
            const float4 Uc = __ldg(a.U + (ci[0] + kFluidPad) + row * (ci[1] + kFluidPad) + slab * (ci[2] + kFluidPad));
            up[0] = Uc.x;
            up[1] = Uc.y;
            up[2] = Uc.z;
          } else {
            const float4* b = a.U + i0[0] + row * i0[1] + slab * i0[2];
            const float4 U000 = __ldg(b);
            const float4 U100 = __ldg(b + 1);
            const float4 U010 = __ldg(b + row);
            const float4 U110 = __ldg(b + row + 1);
            const float4 U001 = __ldg(b + slab);
            const float4 U101 = __ldg(b + slab + 1);
            const float4 U011 = __ldg(b + slab + row);
            const float4 U111 = __ldg(b + slab + row + 1);
            float r00[3], r10[3], r01[3], r11[3];
            lerp3(U000, U100, f[0], r00);
            lerp3(U010, U110, f[0], r10);
            lerp3(U001, U101, f[0], r01);
            lerp3(U011, U111, f[0], r11);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const float r0 = fmaf(f[1], r10[q] - r00[q], r00[q]);
              const float r1 = fmaf(f[1], r11[q] - r01[q], r01[q]);
              up[q] = fmaf(f[2], r1 - r0, r0);
            }
          }
          // drag rate a = alpha f(Re) / tau (f = 1 for Stokes drag); both integrators take the form
          // v' = w + (v - w) E, x' = x + w dt + (v - w) Q with w = u_p + g / a:
          //   exponential:         E = e^{-a dt},       Q = (1 - E) / a
          //   semi-implicit Euler: E = 1 / (1 + a dt),  Q = E dt  (x' = x + dt v')
          const float d = dv[j];
          const float dd = d * d;
          float adt = a.cadt / dd;       // a dt
          float inv_a = dd * a.inv_ca;   // 1 / a
          if (a.sn) {
            const float r0 = up[0] - v[0][j], r1 = up[1] - v[1][j], r2 = up[2] - v[2][j];
            const float fac = sn_factor(a.re_coef * sqrtf(fmaf(r0, r0, fmaf(r1, r1, r2 * r2))) * d);
            adt *= fac;
            inv_a /= fac;
          }
          float E, Q;
          if (a.semi) {
            E = 1.0f / (1.0f + adt);
            Q = E * a.dt;
          } else {
            const float E1 = -expm1f(-adt);  // 1 - e^{-a dt}
            E = 1.0f - E1;
            Q = E1 * inv_a;
          }
          const float m = a.mcoef * dd * d;
          int cn[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float wt = fmaf(a.g[q], inv_a, up[q]);
            const float dvw = v[q][j] - wt;
            const float vn = stored<BF16>(fmaf(dvw, E, wt));
            const float dx = fmaf(wt, a.dt, dvw * Q);
            // relocate: offset in cell units, carry whole cells into the index (k = round(o - 1/2)
            // by the 1.5 * 2^23 shift: no rounding or conversion instructions)
            float o = fmaf(dx, a.inv_h[q], xi[q][j]);
            int ii;
            if (__builtin_expect(fabsf(o) < 4194304.0f, 1)) {
              const float t = (o - 0.5f) + 12582912.0f;
              ii = ci[q] + (__float_as_int(t) - 0x4B400000);
              o = o - (t - 12582912.0f);
              if (o >= 1.0f) {  // on the upper face: offset 0 of the next cell
                o = 0.0f;
                ii += 1;
              }
              o = fmaxf(o, 0.0f);
              if (ii >= n3[q]) ii -= n3[q];
              else if (ii < 0) ii += n3[q];
              if (__builtin_expect((unsigned)ii >= (unsigned)n3[q], 0)) ii = wrap_index_slow(ii, n3[q]);
            } else {
              ii = relocate_far(o, ci[q], n3[q]);
            }
            cn[q] = ii;
            xi[q][j] = o;
            J[j][q] = -m * ((vn - v[q][j]) - a.gdt[q]);
            v[q][j] = vn;
          }
          cell[j] = pack_cell(cn[0], cn[1], cn[2]);
        }
      }
      // ---- store (128-bit, streaming) ----
      __stcs((int4*)(a.s.cell + p0), make_int4(cell[0], cell[1], cell[2], cell[3]));
      for (int q = 0; q < 3; ++q)
        __stcs((float4*)(a.s.xi[q] + p0), make_float4(xi[q][0], xi[q][1], xi[q][2], xi[q][3]));
      for (int q = 0; q < 3; ++q) store_v<BF16>(a, q, p0, v[q]);
    }
    // ---- deposit: runs of equal key over the warp's 128 particles (none without an accumulator:
    // the adjoint's recomputation) ----
    if (!a.acc) {
    } else if (!CIC) {
      deposit_runs(a, lane, key, J);
    } else {
      // cloud in cell: one pass of runs per stencil corner (sorted particles share corners)
#pragma unroll 1
      for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
        int kc[4];
        float Jc[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float* fj = sf[CIC ? j : 0];
          const int* bj = sb[CIC ? j : 0];
          const float w = (dx ? fj[0] : 1.0f - fj[0]) * (dy ? fj[1] : 1.0f - fj[1]) * (dz ? fj[2] : 1.0f - fj[2]);
          int ix = bj[0] + dx, iy = bj[1] + dy, iz = bj[2] + dz;
          ix = ix >= a.nx ? ix - a.nx : ix;
          iy = iy >= a.ny ? iy - a.ny : iy;
          iz = iz >= a.nz ? iz - a.nz : iz;
          kc[j] = key[j] < 0 ? -1 : ix + a.nx * (iy + a.ny * iz);
#pragma unroll
          for (int q = 0; q < 3; ++q) Jc[j][q] = w * J[j][q];
        }
        deposit_runs(a, lane, kc, Jc);
      }
    }
  }
}

}  // namespace

cudaError_t launch_step_mixed(st_ctx* h, const StepParams& p) {
  return launch_step_mixed_state(h, carve_mixed(h->state.p, h->cap, h->prec == ST_MIXED_BF16V), h->np,
                                 (long long*)h->acc.p, p);
}

cudaError_t launch_step_mixed_state(st_ctx* h, const MixedState& s, int64_t n, long long* acc, const StepParams& p) {
  MixedArgs a;
  bool bf = h->prec == ST_MIXED_BF16V;
  a.s = s;
  a.U = (const float4*)h->fluid_pad.p;
  a.acc = acc;
  a.n = n;
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
  a.cadt = (float)(p.ca * p.dt);
  a.inv_ca = (float)(1.0 / p.ca);
  a.mcoef = (float)p.mcoef;
  a.E = p.E;
  a.ngp = p.ngp;
  a.semi = p.semi;
  a.sn = p.sn;
  a.re_coef = (float)p.re_coef;
  int64_t warps = (n + 127) / 128;
  int64_t blocks = (warps * 32 + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  void (*kern)(const MixedArgs) = bf ? (p.cic ? step_mixed_kernel<true, true> : step_mixed_kernel<true, false>)
                                     : (p.cic ? step_mixed_kernel<false, true> : step_mixed_kernel<false, false>);
  kern<<<(int)blocks, 256, 0, h->stream>>>(a);
  h->launches += 1;
  return cudaGetLastError();
}

}  // namespace st
