// Mixed-precision Lagrangian step for sorted particles: a persistent,
// warp-specialised kernel fed by the Tensor Memory Accelerator.
//
// After the counting sort the particles of every aligned U^3 block of cells
// (U = min(B, 8); the Morton order inside a chunk makes each such block a
// contiguous key range) are contiguous in storage.  Each CTA owns a sequence of
// these units.  Per unit:
//   * a producer warp loads the unit's fluid tile - the U^3 cells plus a halo
//     of G cells - from the ghost-padded field with one 4-D TMA tensor copy
//     (double-buffered across units), and streams the unit's particle arrays
//     through a ring of shared-memory stages with 1-D bulk copies
//     (cp.async.bulk), signalling completion on mbarriers;
//   * consumer warps take 4 consecutive particles per lane from the stage,
//     gather the fluid velocity from the shared tile (8 LDS.128 with immediate
//     offsets; particles that drifted out of the tile read the padded field
//     from L2), advance and relocate them, store the new state with 128-bit
//     streaming stores, and reduce their impulses over runs of equal
//     start-of-step cell across the warp;
//   * each run is added once to the global carry-save fixed-point accumulator
//     with fire-and-forget integer atomic adds (exact and independent of the
//     order of the adds); sorted storage keeps runs long and the touched
//     accumulator lines hot in L2.
// The first step after a sort may also do that sort's payload gather (the GATHER instance): the sort
// leaves a permutation and the previous step's 32-byte records {cell, offsets | velocity, diameter}
// in the old order, and each consumer thread loads its own particles' records through the
// permutation with one 256-bit load each, asked of L2 by a prefetch one stage ahead (their ids come
// a stage ahead into registers and are stored in sorted order at the start of the stage they belong
// to; the diameters are stored as soon as the records arrive), then stores the new state in sorted
// order.  The separate gather would write the sorted arrays only for this step to read them back.
// Every wait is bounded: a wait that gives up sets an error flag and the CTA
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>

#include "st_common.cuh"
#include "st_ptx.cuh"

namespace st {
namespace {

using namespace ptx;

constexpr int kU = 8;                       // unit edge (cells)
constexpr int kG = 3;                       // fluid halo = padding of the field
constexpr int kTE = kU + 2 * kG;            // fluid tile edge (14)
constexpr int kConsumerWarps = 15;
constexpr int kT = kConsumerWarps * 128;    // particles per stage (1920)
constexpr int kStages = 2;
constexpr int kFluidBufs = 1;              // fluid tiles in flight (one reload bubble per unit)
constexpr int kR = 2;                      // deposit halo
constexpr int kDE = kU + 2 * kR;           // deposit tile edge (12)
constexpr int kDepositCells = kDE * kDE * kDE;  // 1728
constexpr int kScanLanes = 8;              // runs are chained across at most this many lanes
constexpr int kDirectRecords = 16;         // more run records than this per warp: commit in place
constexpr int kDigits = 3;                 // 15-bit digits per value in the shared deposit tile
constexpr int kDigitBits = 15;
constexpr int kDepShift = 51;              // shared tile units = global units * 2^kDepShift
constexpr int64_t kDepMaxCount = 65535;    // per-unit particles for which no digit word can overflow
constexpr int kThreads = (kConsumerWarps + 1) * 32;

constexpr int kFluidBytes = kTE * kTE * kTE * 16;          // 43904
constexpr int kStageBytes = kT * 32;                        // 61440 (FP32 layout; BF16 uses less)
constexpr int kDepositBytes = kDepositCells * 3 * kDigits * 4;  // 62208
constexpr int kSmemBytes = kFluidBufs * kFluidBytes + kDepositBytes + kStages * kStageBytes + 16 * 8;  // 229128

__device__ __forceinline__ void tma_load_tile(void* dst, const CUtensorMap* map, int c1, int c2, int c3,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(sptr(dst)),
      "l"(map), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(sptr(bar))
      : "memory");
}


__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

struct TmaArgs {
  MixedState s;
  const float4* __restrict__ Up;      // ghost-padded field [nz+2G][ny+2G][nx+2G]
  long long* __restrict__ acc;
  const uint32_t* __restrict__ cell_start;
  int* __restrict__ err;
  unsigned long long* __restrict__ acc_ctr;  // digits added to any accumulator word (global commits)
  unsigned* __restrict__ unit_ctr;           // next unit to hand out (zeroed before the launch)
  int64_t ncell;
  int nx, ny, nz;
  int nunits;                         // units of kU^3 cells in key order
  int logB, ncx, ncy;                 // chunk geometry for decoding a unit's origin
  float inv_h[3];
  float dt, cadt, inv_ca, mcoef;
  float g[3], gdt[3];
  int E;                              // global accumulator exponent
  float s1, s2;                       // s1 * s2 = 2^(E - kDepShift): global units -> deposit-tile units
  float4* __restrict__ rec;           // record output: two float4 per particle (see st_common.cuh)
  const uint32_t* __restrict__ perm;  // GATHER: storage index (old order) of each sorted position
  const float4* __restrict__ grec;    // GATHER: the records in the old order
  const uint32_t* __restrict__ ids_in;   // GATHER: ids in the old order
  uint32_t* __restrict__ ids_out;        // GATHER: ids in sorted order
  int ngp, semi, sn, cic;             // physics variants (the PHYS instance): nearest grid point,
  float re_coef;                      // semi-implicit Euler, Schiller-Naumann drag (Re = re_coef |u-v| d),
                                      // cloud-in-cell deposit
};

// de-interleave 3 bits per level (local x bit lowest)
__device__ __forceinline__ uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030c30c3u;
  v = (v | (v >> 4)) & 0x0300f00fu;
  v = (v | (v >> 8)) & 0xff0000ffu;
  v = (v | (v >> 16)) & 0x000003ffu;
  return v;
}

__device__ __forceinline__ void unit_origin(const TmaArgs& a, int u, int& ox, int& oy, int& oz) {
  const uint32_t key = (uint32_t)u * (kU * kU * kU);
  const uint32_t chunk = key >> (3 * a.logB);
  const uint32_t m = key & ((1u << (3 * a.logB)) - 1u);
  const int B = 1 << a.logB;
  const int cx = (int)(chunk % (uint32_t)a.ncx);
  const int cy = (int)((chunk / (uint32_t)a.ncx) % (uint32_t)a.ncy);
  const int cz = (int)(chunk / ((uint32_t)a.ncx * (uint32_t)a.ncy));
  ox = cx * B + (int)compact3(m);
  oy = cy * B + (int)compact3(m >> 1);
  oz = cz * B + (int)compact3(m >> 2);
}

template <bool BF16>
__device__ __forceinline__ int stage_bytes(int cnt) {
  return cnt * (BF16 ? 26 : 32);
}

// cell and offset of a coordinate that the fast relocation cannot take (rare): a move of 2^22 cells
// or more, or of more than one box length, in one step; the cell carried is floor(o) reduced
// periodically (fmodf is exact), the offset o - floor(o)
struct Relocated {
  int cell;
  float offset;
};
__device__ __noinline__ Relocated relocate_general(float o, int ci, int n) {
  if (!(fabsf(o) <= 3.0e38f)) return Relocated{ci, 0.5f};  // non-finite: keep the cell
  const float fl = floorf(o);
  int k = (ci + (int)fmodf(fl, (float)n)) % n;
  return Relocated{k < 0 ? k + n : k, fmaxf(fminf(o - fl, 0.99999994f), 0.0f)};
}

// two-lane FP32 arithmetic (one instruction for a register pair; round-to-nearest, no flush to
// zero, so each lane rounds exactly as the scalar operation would)
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long add_rm2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long dup2(float a) { return pack2(a, a); }
// lerp c0 + w (c1 - c0) on the (x, y) pair
__device__ __forceinline__ unsigned long long lerp2(unsigned long long w, unsigned long long c0, unsigned long long c1) {
  return fma2(w, sub2(c1, c0), c0);
}

// 1 - e^{-x} for a pair of arguments x >= 0 (*E = e^{-x}): the degree-5 Taylor polynomial in
// Horner form for x < 1/8 (truncation below 5e-8 relative), else 1 - 2^(-x log2 e); the polynomial
// as pair operations, the exponentials and the choice per lane
__device__ __forceinline__ unsigned long long one_minus_exp2(unsigned long long X, unsigned long long* E) {
  float x0, x1, a0, a1;
  unpack2(mul2(X, dup2(-1.4426950408889634f)), a0, a1);
  float ex0, ex1;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex0) : "f"(a0));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex1) : "f"(a1));
  unsigned long long S = fma2(X, dup2(1.0f / 120.0f), dup2(-1.0f / 24.0f));
  S = fma2(X, S, dup2(1.0f / 6.0f));
  S = fma2(X, S, dup2(-0.5f));
  S = fma2(X, S, dup2(1.0f));
  float s0, s1;
  unpack2(mul2(X, S), s0, s1);
  unpack2(X, x0, x1);
  const float r0 = x0 < 0.125f ? s0 : 1.0f - ex0;
  const float r1 = x1 < 0.125f ? s1 : 1.0f - ex1;
  *E = pack2(x0 < 0.125f ? 1.0f - r0 : ex0, x1 < 0.125f ? 1.0f - r1 : ex1);
  return pack2(r0, r1);
}

// trilinear interpolation of the 8 corner velocities (corner c_xyz, x fastest) at weights f: the
// x and y components as register pairs, z alone; the same operations and rounding per component
// as c0 + f (c1 - c0) applied along x, then y, then z
__device__ __forceinline__ void trilerp(const float4& c000, const float4& c100, const float4& c010,
                                        const float4& c110, const float4& c001, const float4& c101,
                                        const float4& c011, const float4& c111, float fx, float fy, float fz,
                                        float* up) {
  const unsigned long long FX = pack2(fx, fx), FY = pack2(fy, fy), FZ = pack2(fz, fz);
  const unsigned long long a = lerp2(FX, pack2(c000.x, c000.y), pack2(c100.x, c100.y));
  const unsigned long long b = lerp2(FX, pack2(c010.x, c010.y), pack2(c110.x, c110.y));
  const unsigned long long c = lerp2(FX, pack2(c001.x, c001.y), pack2(c101.x, c101.y));
  const unsigned long long d = lerp2(FX, pack2(c011.x, c011.y), pack2(c111.x, c111.y));
  const unsigned long long e = lerp2(FY, a, b), g = lerp2(FY, c, d);
  unpack2(lerp2(FZ, e, g), up[0], up[1]);
  const float az = fmaf(fx, c100.z - c000.z, c000.z), bz = fmaf(fx, c110.z - c010.z, c010.z);
  const float cz = fmaf(fx, c101.z - c001.z, c001.z), dz = fmaf(fx, c111.z - c011.z, c011.z);
  const float ez = fmaf(fy, bz - az, az), gz = fmaf(fy, dz - cz, cz);
  up[2] = fmaf(fz, gz - ez, ez);
}

// fluid velocity of a particle outside its unit's tile, from the ghost-padded field (L2); the same
// stencil and arithmetic as the tile path
__device__ __noinline__ float3 gather_padded(const float4* __restrict__ Up, int px, int pxy, int cell, float o0,
                                             float o1, float o2) {
  const int ci[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
  const float o[3] = {o0, o1, o2};
  int i0[3];
  float f[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const bool hi2 = o[q] >= 0.5f;
    i0[q] = ci[q] - (hi2 ? 0 : 1);
    f[q] = o[q] + (hi2 ? -0.5f : 0.5f);
  }
  const float4* g = Up + (i0[0] + kG) + (int64_t)px * (i0[1] + kG) + (int64_t)pxy * (i0[2] + kG);
  float up[3];
  trilerp(__ldg(g), __ldg(g + 1), __ldg(g + px), __ldg(g + px + 1), __ldg(g + pxy), __ldg(g + pxy + 1),
          __ldg(g + pxy + px), __ldg(g + pxy + px + 1), f[0], f[1], f[2], up);
  return make_float3(up[0], up[1], up[2]);
}

// nearest-grid-point value of a particle outside its unit's tile, from the ghost-padded field
__device__ __noinline__ float3 ngp_padded(const float4* __restrict__ Up, int px, int pxy, int cell) {
  const float4 u = __ldg(Up + (cell_i(cell) + kG) + (int64_t)px * (cell_j(cell) + kG) + (int64_t)pxy * (cell_k(cell) + kG));
  return make_float3(u.x, u.y, u.z);
}

// Schiller-Naumann drag factor f = C_D Re / 24: 1 + 0.15 Re^0.687 up to Re = 1000 (the power from
// the hardware base-2 logarithm and exponential), 0.44 Re / 24 above
__device__ __forceinline__ float sn_factor(float re) {
  float l, p;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(re));
  const float y = 0.687f * l;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p) : "f"(y));
  return re <= 1000.0f ? fmaf(0.15f, p, 1.0f) : (0.44f / 24.0f) * re;
}

// add round(r_q * 2^Es), q = 0, 1, 2, to the shared deposit-tile values of one cell, each kept as
// three signed digits in int32 words (w[0] + 2^15 w[kDepositCells] + 2^30 w[2 kDepositCells], the
// components kDigits kDepositCells words apart); s1 * s2 = 2^Es.  Each scaled value t
// (|t| < 2^45) is split exactly into balanced digits by round-to-nearest additions of
// 1.5 * 2^(23+b), which leave the nearest multiple of 2^b: t = 2^30 d2 + 2^15 d1 + d0 +
// (t - round(t)) with |d0|, |d1| <= 2^14 and |d2| <= 2^15.  Components 0 and 1 are split as a
// register pair.  Integer atomics make the sums exact and independent of the order of the adds.
__device__ __forceinline__ void digits1(float t, int& d0, int& d1, int& d2) {
  const float h = __fsub_rn(__fadd_rn(t, 0x1.8p53f), 0x1.8p53f);  // multiple of 2^30
  const float l = __fsub_rn(t, h);                                  // |l| <= 2^29, exact
  const float m = __fsub_rn(__fadd_rn(l, 0x1.8p38f), 0x1.8p38f);  // multiple of 2^15
  const float l2 = __fsub_rn(l, m);                                 // |l2| <= 2^14, exact
  d2 = __float_as_int(__fmaf_rn(h, 0x1p-30f, 12582912.0f)) - 0x4B400000;
  d1 = __float_as_int(__fmaf_rn(m, 0x1p-15f, 12582912.0f)) - 0x4B400000;
  d0 = __float_as_int(__fadd_rn(l2, 12582912.0f)) - 0x4B400000;
}
__device__ __forceinline__ void digits2(unsigned long long t, int* d0, int* d1, int* d2) {
  const unsigned long long C53 = pack2(0x1.8p53f, 0x1.8p53f), C38 = pack2(0x1.8p38f, 0x1.8p38f);
  const unsigned long long C23 = pack2(12582912.0f, 12582912.0f);
  const unsigned long long h = sub2(add2(t, C53), C53);
  const unsigned long long l = sub2(t, h);
  const unsigned long long m = sub2(add2(l, C38), C38);
  const unsigned long long l2 = sub2(l, m);
  float a, b;
  unpack2(fma2(h, pack2(0x1p-30f, 0x1p-30f), C23), a, b);
  d2[0] = __float_as_int(a) - 0x4B400000;
  d2[1] = __float_as_int(b) - 0x4B400000;
  unpack2(fma2(m, pack2(0x1p-15f, 0x1p-15f), C23), a, b);
  d1[0] = __float_as_int(a) - 0x4B400000;
  d1[1] = __float_as_int(b) - 0x4B400000;
  unpack2(add2(l2, C23), a, b);
  d0[0] = __float_as_int(a) - 0x4B400000;
  d0[1] = __float_as_int(b) - 0x4B400000;
}
__device__ __forceinline__ void dep_add3(int* w, float r0, float r1, float r2, float s1, float s2) {
  int d0[3], d1[3], d2[3];
  digits2(mul2(mul2(pack2(r0, r1), pack2(s1, s1)), pack2(s2, s2)), d0, d1, d2);
  digits1(__fmul_rn(__fmul_rn(r2, s1), s2), d0[2], d1[2], d2[2]);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    int* wq = w + q * (kDigits * kDepositCells);
    if (d0[q]) atomicAdd(wq, d0[q]);
    if (d1[q]) atomicAdd(wq + kDepositCells, d1[q]);
    if (d2[q]) atomicAdd(wq + 2 * kDepositCells, d2[q]);
  }
}

// one run record: into the shared deposit tile, or (start cell outside the tile, rare) straight to
// the global accumulator, counted for the carry-propagation decision
__device__ __forceinline__ void commit_record(const TmaArgs& a, int* dep, int kk, float r0, float r1, float r2) {
  if (__builtin_expect(kk < kDepositCells, 1)) {
    dep_add3(dep + kk, r0, r1, r2, a.s1, a.s2);
  } else {
    const int64_t c = kk - kDepositCells;
    acc_add_f32(a.acc + kAccWords * c, r0, a.E);
    acc_add_f32(a.acc + kAccWords * (a.ncell + c), r1, a.E);
    acc_add_f32(a.acc + kAccWords * (2 * a.ncell + c), r2, a.E);
    atomicAdd(a.acc_ctr, 1ull);
  }
}

// GATHER: the permutation entries of a lane's four sorted positions p0 .. p0 + 3 (p0 a multiple of
// 4), zeros when it owns none of them within [S, E) (then p0 may lie past the buffer)
__device__ __forceinline__ uint4 gather_perm(const TmaArgs& a, int64_t p0, int64_t S, int64_t E) {
  const bool any = p0 + 4 > S && p0 < E;
  return any ? __ldcs(reinterpret_cast<const uint4*>(a.perm + p0)) : make_uint4(0, 0, 0, 0);
}
// GATHER: the ids of the owned positions among p0 .. p0 + 3 through the permutation (0 elsewhere)
__device__ __forceinline__ uint4 gather_ids(const TmaArgs& a, uint4 pp, int64_t p0, int64_t S, int64_t E) {
  const uint32_t pj[4] = {pp.x, pp.y, pp.z, pp.w};
  uint32_t id[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) id[j] = (p0 + j >= S && p0 + j < E) ? __ldg(a.ids_in + pj[j]) : 0u;
  return make_uint4(id[0], id[1], id[2], id[3]);
}
// GATHER: store ids gathered for positions p0 .. p0 + 3 (the owned ones)
__device__ __forceinline__ void store_ids(const TmaArgs& a, uint4 id, int64_t p0, int64_t S, int64_t E) {
  if (p0 >= S && p0 + 4 <= E) {
    __stcs(reinterpret_cast<uint4*>(a.ids_out + p0), id);
  } else {
    const uint32_t v[4] = {id.x, id.y, id.z, id.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (p0 + j >= S && p0 + j < E) a.ids_out[p0 + j] = v[j];
  }
}
// GATHER: ask L2 for the records of the owned positions among p0 .. p0 + 3 (a stage before their
// loads)
__device__ __forceinline__ void gather_prefetch(const TmaArgs& a, uint4 pp, int64_t p0, int64_t S, int64_t E) {
  const uint32_t pj[4] = {pp.x, pp.y, pp.z, pp.w};
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (p0 + j >= S && p0 + j < E) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.grec + 2 * (int64_t)pj[j]));
}
// GATHER: the diameters of the owned positions among p0 .. p0 + 3, stored in sorted order as soon as
// their records arrive (a step does not change them)
__device__ __forceinline__ void store_d(const TmaArgs& a, const Rec32 (&r)[4], int64_t p0, int64_t S, int64_t E) {
  if (p0 >= S && p0 + 4 <= E) {
    __stcs(reinterpret_cast<float4*>(a.s.d + p0), make_float4(r[0].d, r[1].d, r[2].d, r[3].d));
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (p0 + j >= S && p0 + j < E) a.s.d[p0 + j] = r[j].d;
  }
}

template <bool BF16, bool PW2, bool REC, bool PHYS, bool GATHER>
__global__ void __maxnreg__(128) step_mixed_tma_kernel(const __grid_constant__ CUtensorMap fluid_map,
                                                                      const __grid_constant__ TmaArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float4* fluid = reinterpret_cast<float4*>(smem);                               // [kFluidBufs][kTE^3]
  int* dep = reinterpret_cast<int*>(smem + kFluidBufs * kFluidBytes);            // [3][kDigits][kDE^3]
  unsigned char* ring = smem + kFluidBufs * kFluidBytes + kDepositBytes;          // [kStages][kStageBytes]
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + kStages * kStageBytes);
  uint64_t* full = bars;                    // [kStages]   producer -> consumers (bytes landed)
  uint64_t* empty = bars + kStages;         // [kStages]   consumers -> producer (stage free)
  uint64_t* tile_full = bars + 2 * kStages;  // [2]        fluid tile landed
  uint64_t* tile_empty = tile_full + 2;      // [2]        consumers done with a fluid tile
  uint64_t* dep_done = tile_empty + 2;       // [1]        every consumer warp finished a unit's deposits
  uint64_t* flush_done = dep_done + 1;       // [1]        deposit tile flushed and cleared
  volatile int* unit_slot = reinterpret_cast<volatile int*>(flush_done + 1);  // [kFluidBufs] unit of a tile

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tile_full[b], 1);
      mbar_init(&tile_empty[b], kConsumerWarps);
    }
    mbar_init(dep_done, kConsumerWarps);
    mbar_init(flush_done, kConsumerWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 3 * kDigits * kDepositCells; i += blockDim.x) dep[i] = 0;
  __syncthreads();

  if (warp == kConsumerWarps) {
    // ================= producer =================
    if (lane == 0) {
      int loaded = 0;    // non-empty units whose fluid tile was issued
      int64_t gt = 0;    // particle stages issued
      // units are handed out one at a time from a global counter, so a CTA that starts late (its SM
      // busy with other work) simply takes fewer units
      for (;;) {
        const int u = (int)atomicAdd(a.unit_ctr, 1u);
        if (u >= a.nunits) break;
        const int64_t S = a.cell_start[(int64_t)u * (kU * kU * kU)];
        const int64_t E = a.cell_start[(int64_t)(u + 1) * (kU * kU * kU)];
        if (E <= S) continue;
        const int buf = loaded % kFluidBufs;
        if (loaded >= kFluidBufs && !mbar_wait(&tile_empty[buf], ((loaded / kFluidBufs) - 1) & 1)) {
          atomicOr(a.err, 1);
          return;
        }
        unit_slot[buf] = u;  // published to the consumers by the tile barrier's arrive
        int ox, oy, oz;
        unit_origin(a, u, ox, oy, oz);
        mbar_expect_tx(&tile_full[buf], kFluidBytes);
        tma_load_tile(fluid + buf * (kTE * kTE * kTE), &fluid_map, ox, oy, oz, &tile_full[buf]);
        ++loaded;
        const int64_t A = S & ~int64_t(7);
        const int64_t Z = (E + 7) & ~int64_t(7);
        for (int64_t t0 = A; t0 < Z; t0 += kT) {
          const int cnt = (int)min((int64_t)kT, Z - t0);
          const int st = (int)(gt % kStages);
          if (gt >= kStages && !mbar_wait(&empty[st], ((gt / kStages) - 1) & 1)) {
            atomicOr(a.err, 2);
            return;
          }
          unsigned char* dst = ring + st * kStageBytes;
          if (GATHER) {
            // the consumers load their particles themselves; the stage only serves as their scratch
            mbar_arrive(&full[st]);
            ++gt;
            continue;
          }
          mbar_expect_tx(&full[st], stage_bytes<BF16>(cnt));
          bulk_load(dst, a.s.cell + t0, cnt * 4, &full[st]);
          for (int q = 0; q < 3; ++q) bulk_load(dst + (1 + q) * kT * 4, a.s.xi[q] + t0, cnt * 4, &full[st]);
          const int vb = BF16 ? 2 : 4;
          for (int q = 0; q < 3; ++q)
            bulk_load(dst + 4 * kT * 4 + q * kT * vb, (const char*)a.s.v[q] + t0 * vb, cnt * vb, &full[st]);
          bulk_load(dst + 4 * kT * 4 + 3 * kT * vb, a.s.d + t0, cnt * 4, &full[st]);
          ++gt;
        }
      }
      // no more units: a tile phase without a copy, unit -1
      {
        const int buf = loaded % kFluidBufs;
        if (loaded >= kFluidBufs && !mbar_wait(&tile_empty[buf], ((loaded / kFluidBufs) - 1) & 1)) {
          atomicOr(a.err, 1);
          return;
        }
        unit_slot[buf] = -1;
        mbar_arrive(&tile_full[buf]);
      }
      // let the last copies land before the CTA can exit
      const int64_t first = gt > kStages ? gt - kStages : 0;
      for (int64_t k = first; k < gt; ++k) mbar_wait(&empty[k % kStages], (k / kStages) & 1);
    }
    return;
  }

  // ================= consumers =================
  const int ctid = threadIdx.x;  // 0 .. 32 kConsumerWarps - 1
  const int n3[3] = {a.nx, a.ny, a.nz};
  const int px = a.nx + 2 * kG, pxy = (a.nx + 2 * kG) * (a.ny + 2 * kG);
  int loaded = 0;
  int64_t gt = 0;
  for (;;) {
    const int buf = loaded % kFluidBufs;
    if (!mbar_wait(&tile_full[buf], (loaded / kFluidBufs) & 1)) {
      atomicOr(a.err, 4);
      return;
    }
    const int u = unit_slot[buf];
    if (u < 0) break;
    const int64_t S = a.cell_start[(int64_t)u * (kU * kU * kU)];
    const int64_t E = a.cell_start[(int64_t)(u + 1) * (kU * kU * kU)];
    const float4* tile = fluid + buf * (kTE * kTE * kTE);
    int uo[3];
    unit_origin(a, u, uo[0], uo[1], uo[2]);
    const bool use_tile = (E - S) <= kDepMaxCount;  // every digit word stays below 2^31
    const int64_t A = S & ~int64_t(7);
    const int64_t Z = (E + 7) & ~int64_t(7);
    const int L = 4 * ctid;
    // GATHER: the permutation entries of this stage and of the next, and this stage's ids, are
    // held in registers a stage ahead
    uint4 pcur = make_uint4(0, 0, 0, 0), pnext = make_uint4(0, 0, 0, 0), gid = make_uint4(0, 0, 0, 0);
    if constexpr (GATHER) {
      pcur = gather_perm(a, A + L, S, E);
      gid = gather_ids(a, pcur, A + L, S, E);
      pnext = gather_perm(a, A + kT + L, S, E);
    }
    for (int64_t t0 = A; t0 < Z; t0 += kT) {
      const int st = (int)(gt % kStages);
      if (!mbar_wait(&full[st], (gt / kStages) & 1)) {
        atomicOr(a.err, 8);
        return;
      }
      const unsigned char* src = ring + st * kStageBytes;
      const int64_t p0 = t0 + L;
      int cell[4];
      float xi[3][4], v[3][4], dv[4];
      if constexpr (GATHER) {
        // this stage's records through the permutation, one 256-bit load each (asked of L2 a stage
        // ago); positions outside the unit get harmless values and are neither stored nor deposited
        const int glo = (int)max((int64_t)0, min((int64_t)4, S - p0));
        const int ghi = (int)max((int64_t)0, min((int64_t)4, E - p0));
        const uint32_t pj[4] = {pcur.x, pcur.y, pcur.z, pcur.w};
        Rec32 r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          r[j] = (j >= glo && j < ghi) ? ld_rec32(a.grec + 2 * (int64_t)pj[j])
                                       : Rec32{0.0f, 0.5f, 0.5f, 0.5f, 0.0f, 0.0f, 0.0f, 1e-5f};
        // this stage's ids (loaded a stage ago) go out now; the next stage's come in, and its records
        // are asked for
        store_ids(a, gid, p0, S, E);
        if (t0 + kT < Z) {
          gather_prefetch(a, pnext, p0 + kT, S, E);
          gid = gather_ids(a, pnext, p0 + kT, S, E);
          pcur = pnext;
          pnext = gather_perm(a, p0 + 2 * kT, S, E);
        }
        store_d(a, r, p0, S, E);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          cell[j] = __float_as_int(r[j].c);
          xi[0][j] = r[j].x0;
          xi[1][j] = r[j].x1;
          xi[2][j] = r[j].x2;
          v[0][j] = r[j].v0;
          v[1][j] = r[j].v1;
          v[2][j] = r[j].v2;
          dv[j] = r[j].d;
        }
      } else {
        int4 c4 = *reinterpret_cast<const int4*>(src + L * 4);
        cell[0] = c4.x;
        cell[1] = c4.y;
        cell[2] = c4.z;
        cell[3] = c4.w;
        for (int q = 0; q < 3; ++q) {
          float4 x4 = *reinterpret_cast<const float4*>(src + (1 + q) * kT * 4 + L * 4);
          xi[q][0] = x4.x;
          xi[q][1] = x4.y;
          xi[q][2] = x4.z;
          xi[q][3] = x4.w;
        }
        if (BF16) {
          for (int q = 0; q < 3; ++q) {
            uint2 r = *reinterpret_cast<const uint2*>(src + 4 * kT * 4 + q * kT * 2 + L * 2);
            float2 l = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.x));
            float2 h = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&r.y));
            v[q][0] = l.x;
            v[q][1] = l.y;
            v[q][2] = h.x;
            v[q][3] = h.y;
          }
          float4 d4 = *reinterpret_cast<const float4*>(src + 4 * kT * 4 + 3 * kT * 2 + L * 4);
          dv[0] = d4.x;
          dv[1] = d4.y;
          dv[2] = d4.z;
          dv[3] = d4.w;
        } else {
          for (int q = 0; q < 3; ++q) {
            float4 r = *reinterpret_cast<const float4*>(src + 4 * kT * 4 + q * kT * 4 + L * 4);
            v[q][0] = r.x;
            v[q][1] = r.y;
            v[q][2] = r.z;
            v[q][3] = r.w;
          }
          float4 d4 = *reinterpret_cast<const float4*>(src + 7 * kT * 4 + L * 4);
          dv[0] = d4.x;
          dv[1] = d4.y;
          dv[2] = d4.z;
          dv[3] = d4.w;
        }
      }
      ++gt;

      // owned particles of this lane: [lo, hi) of 0..3 (the rest belong to neighbouring units
      // or lie past the unit); the others are computed too, without branches, from the unit's
      // origin cell so that every tile read stays in bounds, and neither stored nor deposited
      const int lo = (int)max((int64_t)0, min((int64_t)4, S - p0));
      const int hi = (int)max((int64_t)0, min((int64_t)4, E - p0));
      const int ucell = pack_cell(uo[0], uo[1], uo[2]);
      bool own[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        own[j] = (j >= lo) && (j < hi);
        if (!own[j]) cell[j] = ucell;
      }
      // ---- per particle: start cell relative to the unit, deposit key, fluid gather; then drag and
      // gravity (exponential integrator), relocation and exchanged momentum for two particles at
      // a time as FP32 register pairs.  A start cell within kR cells of the unit (the deposit tile)
      // has its whole stencil inside the fluid tile; the rest ("far" particles, rare) read the
      // padded field and commit to the global accumulator.
      int key[4];
      float J[4][3];
      unsigned vpk[3][2];  // BF16: the new velocities as packed pairs (particles 0-1, 2-3)
#pragma unroll
      for (int jp = 0; jp < 4; jp += 2) {
        int ci[2][3];
        float up[2][3];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int j = jp + e;
          ci[e][0] = cell_i(cell[j]);
          ci[e][1] = cell_j(cell[j]);
          ci[e][2] = cell_k(cell[j]);
          int rc[3], rb[3];
          float f[3];
          bool in_dep = true;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float o = xi[q][j];
            const bool hi2 = o >= 0.5f;
            f[q] = o + (hi2 ? -0.5f : 0.5f);
            int r = ci[e][q] - uo[q];  // periodic offset from the unit origin, valid within the tile
            if (PW2) {
              r = ((r + kR) & (n3[q] - 1)) - kR;
            } else {
              if (r >= n3[q] - kR) r -= n3[q];
              else if (r < kDE - kR - n3[q]) r += n3[q];
            }
            in_dep = in_dep && ((unsigned)(r + kR) < (unsigned)kDE);
            rc[q] = r;
            rb[q] = r - (hi2 ? 0 : 1);  // stencil base relative to the unit origin
          }
          const int tofs = in_dep ? (rb[0] + kG) + kTE * ((rb[1] + kG) + kTE * (rb[2] + kG)) : 0;
          key[j] = !own[j]                ? -1
                   : (in_dep && use_tile) ? (rc[0] + kR) + kDE * ((rc[1] + kR) + kDE * (rc[2] + kR))
                                          : kDepositCells + ci[e][0] + a.nx * (ci[e][1] + a.ny * ci[e][2]);
          if (PHYS && a.ngp) {
            // nearest grid point: the value of the start cell (inside the tile when in_dep)
            const float4 c = tile[in_dep ? (rc[0] + kG) + kTE * ((rc[1] + kG) + kTE * (rc[2] + kG)) : 0];
            up[e][0] = c.x;
            up[e][1] = c.y;
            up[e][2] = c.z;
            if (__builtin_expect(!in_dep, 0)) {
              const float3 g = ngp_padded(a.Up, px, pxy, cell[j]);
              up[e][0] = g.x;
              up[e][1] = g.y;
              up[e][2] = g.z;
            }
          } else {
            const float4* bb = tile + tofs;
            trilerp(bb[0], bb[1], bb[kTE], bb[kTE + 1], bb[kTE * kTE], bb[kTE * kTE + 1], bb[kTE * kTE + kTE],
                    bb[kTE * kTE + kTE + 1], f[0], f[1], f[2], up[e]);
            if (__builtin_expect(!in_dep, 0)) {
              const float3 g = gather_padded(a.Up, px, pxy, cell[j], xi[0][j], xi[1][j], xi[2][j]);
              up[e][0] = g.x;
              up[e][1] = g.y;
              up[e][2] = g.z;
            }
          }
        }
        // the integrator on the pair
        const unsigned long long D = pack2(dv[jp], dv[jp + 1]);
        const unsigned long long DD = mul2(D, D);
        float dd0, dd1;
        unpack2(DD, dd0, dd1);
        unsigned long long ADT = mul2(dup2(a.cadt), pack2(rcp_approx(dd0), rcp_approx(dd1)));
        unsigned long long INV_A = mul2(DD, dup2(a.inv_ca));
        unsigned long long EE, E1, Q;
        if (PHYS) {
          // drag rate a = alpha f(Re) / tau (f = 1 for Stokes drag), f from the start-of-step
          // relative velocity; both integrators take the form v' = w + (v - w) E,
          // x' = x + w dt + (v - w) Q with w = u_p + g / a:
          //   exponential:         E = e^{-a dt},       Q = (1 - E) / a
          //   semi-implicit Euler: E = 1 / (1 + a dt),  Q = E dt  (x' = x + dt v')
          if (a.sn) {
            float fac[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float r0 = up[e][0] - v[0][jp + e], r1 = up[e][1] - v[1][jp + e], r2 = up[e][2] - v[2][jp + e];
              fac[e] = sn_factor(a.re_coef * sqrtf(fmaf(r0, r0, fmaf(r1, r1, r2 * r2))) * dv[jp + e]);
            }
            ADT = mul2(ADT, pack2(fac[0], fac[1]));
            INV_A = mul2(INV_A, pack2(rcp_approx(fac[0]), rcp_approx(fac[1])));
          }
          if (a.semi) {
            float x0, x1;
            unpack2(ADT, x0, x1);
            const float e0 = rcp_approx(1.0f + x0), e1 = rcp_approx(1.0f + x1);
            EE = pack2(e0, e1);
            E1 = pack2(x0 * e0, x1 * e1);  // 1 - E = a dt / (1 + a dt)
            Q = mul2(EE, dup2(a.dt));
          } else {
            E1 = one_minus_exp2(ADT, &EE);
            Q = mul2(E1, INV_A);
          }
        } else {
          E1 = one_minus_exp2(ADT, &EE);
          Q = mul2(E1, INV_A);
        }
        const unsigned long long M = mul2(mul2(dup2(a.mcoef), DD), D);
        float oraw[2][3];
        int ii[2][3];
        bool bad[2] = {false, false};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const unsigned long long WT = fma2(dup2(a.g[q]), INV_A, pack2(up[0][q], up[1][q]));
          const unsigned long long V = pack2(v[q][jp], v[q][jp + 1]);
          const unsigned long long DVW = sub2(V, WT);
          float vn[2];
          unpack2(fma2(DVW, EE, WT), vn[0], vn[1]);
          if (BF16) {
            // the stored (rounded) velocity change, so that the deposit balances the particles'
            // momentum; the pair is rounded by one packing conversion, kept packed for the store
            float m0, m1;
            unpack2(M, m0, m1);
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(vn[0], vn[1]);
            vpk[q][jp >> 1] = *reinterpret_cast<const unsigned*>(&b2);
            vn[0] = __low2float(b2);
            vn[1] = __high2float(b2);
            J[jp][q] = -m0 * ((vn[0] - v[q][jp]) - a.gdt[q]);
            J[jp + 1][q] = -m1 * ((vn[1] - v[q][jp + 1]) - a.gdt[q]);
          } else {
            // v' - v = -(v - w) (1 - E), without the cancellation of subtracting the rounded v'
            unpack2(mul2(M, fma2(DVW, E1, dup2(a.gdt[q]))), J[jp][q], J[jp + 1][q]);
          }
          const unsigned long long DXV = fma2(WT, dup2(a.dt), mul2(DVW, Q));
          const unsigned long long O = fma2(DXV, dup2(a.inv_h[q]), pack2(xi[q][jp], xi[q][jp + 1]));
          // whole cells carried: floor(o) from an add of 1.5 * 2^23 rounded toward -inf (exact for
          // |o| < 2^22), so no conversion instructions; the offset o - floor(o) lies in [0, 1]
          const unsigned long long T = add_rm2(O, dup2(12582912.0f));
          float o[2], t[2], x[2];
          unpack2(O, o[0], o[1]);
          unpack2(T, t[0], t[1]);
          unpack2(sub2(O, sub2(T, dup2(12582912.0f))), x[0], x[1]);
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            oraw[e][q] = o[e];
            int k = (int)((unsigned)ci[e][q] + (unsigned)(__float_as_int(t[e]) - 0x4B400000));
            if (PW2) {
              k &= n3[q] - 1;  // any whole-cell move of fewer than 2^22 cells
              bad[e] = bad[e] || !(fabsf(o[e]) < 4194304.0f);
            } else {
              if (k >= n3[q]) k -= n3[q];
              else if (k < 0) k += n3[q];
              bad[e] = bad[e] || !(fabsf(o[e]) < 4194304.0f) || ((unsigned)k >= (unsigned)n3[q]);
            }
            ii[e][q] = k;
            xi[q][jp + e] = fminf(x[e], 0.99999994f);
            v[q][jp + e] = vn[e];
          }
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (__builtin_expect(bad[e], 0)) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const Relocated rl = relocate_general(oraw[e][q], ci[e][q], n3[q]);
              ii[e][q] = rl.cell;
              xi[q][jp + e] = rl.offset;
            }
          }
          cell[jp + e] = pack_cell(ii[e][0], ii[e][1], ii[e][2]);
        }
      }
      // ---- store the owned particles (128-bit when the lane owns all four) ----
      const bool all_own = own[0] && own[1] && own[2] && own[3];
      if (REC) {
        // the step before a sort: the cells to the structure of arrays (the sort's keys), the whole
        // state as 32-byte records {cell, offsets | velocity, diameter}, one 256-bit store per
        // particle (a full sector; the sort's gather then reads one sector per particle).  The
        // diameters are read again from the stage.  BF16 handles store the (BF16-exact) velocities
        // as FP32 in the record.
        const float4 d4 =
            *reinterpret_cast<const float4*>(src + (BF16 ? 4 * kT * 4 + 3 * kT * 2 : 7 * kT * 4) + L * 4);
        const float dj[4] = {d4.x, d4.y, d4.z, d4.w};
        if (all_own) __stcs((int4*)(a.s.cell + p0), make_int4(cell[0], cell[1], cell[2], cell[3]));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (!own[j]) continue;
          if (!all_own) a.s.cell[p0 + j] = cell[j];
          st_rec32(a.rec + 2 * (p0 + j),
                   Rec32{__int_as_float(cell[j]), xi[0][j], xi[1][j], xi[2][j], v[0][j], v[1][j], v[2][j], dj[j]});
        }
      } else if (all_own) {
        __stcs((int4*)(a.s.cell + p0), make_int4(cell[0], cell[1], cell[2], cell[3]));
        for (int q = 0; q < 3; ++q)
          __stcs((float4*)(a.s.xi[q] + p0), make_float4(xi[q][0], xi[q][1], xi[q][2], xi[q][3]));
        if (BF16) {
          for (int q = 0; q < 3; ++q) __stcs((uint2*)((__nv_bfloat16*)a.s.v[q] + p0), make_uint2(vpk[q][0], vpk[q][1]));
        } else {
          for (int q = 0; q < 3; ++q)
            __stcs((float4*)((float*)a.s.v[q] + p0), make_float4(v[q][0], v[q][1], v[q][2], v[q][3]));
        }
      } else {
        for (int j = 0; j < 4; ++j) {
          if (!own[j]) continue;
          a.s.cell[p0 + j] = cell[j];
          for (int q = 0; q < 3; ++q) {
            a.s.xi[q][p0 + j] = xi[q][j];
            if (BF16)
              ((__nv_bfloat16*)a.s.v[q])[p0 + j] = __float2bfloat16_rn(v[q][j]);
            else
              ((float*)a.s.v[q])[p0 + j] = v[q][j];
          }
        }
      }
      // ---- deposit: runs of equal key over the warp's 128 particles (lane-local suffix sums, then a
      // segmented suffix scan across lanes chains runs that span lanes).  compact = false keeps
      // the stage untouched (the records are committed where they are formed) ----
      auto deposit = [&](const int (&key)[4], const float (&J)[4][3], bool compact) {
        float Sx[4][3];
#pragma unroll
        for (int q = 0; q < 3; ++q) Sx[3][q] = J[3][q];
#pragma unroll
        for (int j = 2; j >= 0; --j) {
          const bool same = key[j] == key[j + 1];
#pragma unroll
          for (int q = 0; q < 3; ++q) Sx[j][q] = J[j][q] + (same ? Sx[j + 1][q] : 0.0f);
        }
        const int tail = (key[2] != key[3]) ? 3 : (key[1] != key[2]) ? 2 : (key[0] != key[1]) ? 1 : 0;
        const int nk0 = __shfl_down_sync(0xffffffffu, key[0], 1);
        const int nall = __shfl_down_sync(0xffffffffu, (int)(tail == 0), 1);
        float R[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) R[q] = __shfl_down_sync(0xffffffffu, Sx[0][q], 1);
        const int glane = lane & (kScanLanes - 1);
        const bool link = (glane < kScanLanes - 1) && (nk0 == key[3]) && (key[3] >= 0);
        int Bl = (link && nall) ? 1 : 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) R[q] = link ? R[q] : 0.0f;
        // the scan only matters where a run passes through a whole lane (often nowhere after drift)
        if (__any_sync(0xffffffffu, Bl)) {
#pragma unroll
          for (int off = 1; off < kScanLanes; off <<= 1) {
            float t0v = __shfl_down_sync(0xffffffffu, R[0], off);
            float t1v = __shfl_down_sync(0xffffffffu, R[1], off);
            float t2v = __shfl_down_sync(0xffffffffu, R[2], off);
            int tb = __shfl_down_sync(0xffffffffu, Bl, off);
            if (glane + off > kScanLanes - 1) {
              tb = 0;
              t0v = t1v = t2v = 0.0f;
            }
            if (Bl) {
              R[0] += t0v;
              R[1] += t1v;
              R[2] += t2v;
            }
            Bl &= tb;
          }
        }
        const int pk3 = __shfl_up_sync(0xffffffffu, key[3], 1);
        const bool head_lane = (glane == 0) || (pk3 != key[0]);
        // the run sums, one {J, key} record per run.  Few runs (after a sort): the records are packed
        // in (j, lane) order into the warp's own (already consumed) part of the stage - J in the cell
        // and first two offset arrays, the key in the third - and each lane takes one record at a
        // time, so the whole deposit is one pass.  Many runs (particles drifted away from their
        // sort-time cells): each lane commits its runs where they are, one pass per particle slot,
        // without the round trip through shared memory.
        bool starts[4];
        unsigned hms[4];
        int nh = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          starts[j] = ((j == 0) ? head_lane : (key[j] != key[j - 1])) && key[j] >= 0;
          hms[j] = __ballot_sync(0xffffffffu, starts[j]);
          nh += __popc(hms[j]);
        }
        const bool direct = !compact || nh > kDirectRecords;
        if (direct) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (starts[j]) {
              const bool to_end = j == tail;
              const float r0 = Sx[j][0] + (to_end ? R[0] : 0.0f);
              const float r1 = Sx[j][1] + (to_end ? R[1] : 0.0f);
              const float r2 = Sx[j][2] + (to_end ? R[2] : 0.0f);
              commit_record(a, dep, key[j], r0, r1, r2);
            }
          }
        } else {
          int* rj0 = reinterpret_cast<int*>(const_cast<unsigned char*>(src)) + warp * 128;
          int* rj1 = rj0 + kT;
          int* rj2 = rj0 + 2 * kT;
          int* rk = rj0 + 3 * kT;
          const unsigned lt_mask = (1u << lane) - 1u;
          int base = 0;
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (starts[j]) {
              const bool to_end = j == tail;
              const int slot = base + __popc(hms[j] & lt_mask);
              rj0[slot] = __float_as_int(Sx[j][0] + (to_end ? R[0] : 0.0f));
              rj1[slot] = __float_as_int(Sx[j][1] + (to_end ? R[1] : 0.0f));
              rj2[slot] = __float_as_int(Sx[j][2] + (to_end ? R[2] : 0.0f));
              rk[slot] = key[j];
            }
            base += __popc(hms[j]);
          }
          __syncwarp();
          for (int e = lane; e < nh; e += 32) {
            commit_record(a, dep, rk[e], __int_as_float(rj0[e]), __int_as_float(rj1[e]), __int_as_float(rj2[e]));
          }
          // the records were written through the generic proxy; order them before the producer's
          // next bulk copy into this stage
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
      };
      if (!(PHYS && a.cic)) {
        deposit(key, J, true);
      } else {
        // cloud in cell: J spread over the eight cells of the start-of-step trilinear stencil with
        // its weights, one pass per corner.  The start cells and offsets are read again
        // from the stage (still intact: every pass commits in place).  Corners inside the deposit
        // tile go there; the rest (start cells at the tile's edge or outside it, rare) go to the
        // global accumulator.
        const int4 c4 = *reinterpret_cast<const int4*>(src + L * 4);
        const int cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
          const int dl[3] = {c & 1, (c >> 1) & 1, c >> 2};
          int kc[4];
          float Jc[4][3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float4 o4 = *reinterpret_cast<const float4*>(src + (1 + q) * kT * 4 + L * 4);
            const float oj[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const bool lo = oj[j] < 0.5f;
              const float f = oj[j] + (lo ? 0.5f : -0.5f);
              const float w = dl[q] ? f : 1.0f - f;
              if (q == 0) {
                Jc[j][0] = w;
              } else {
                Jc[j][0] *= w;
              }
              // corner index along this axis relative to the start cell: -1, 0 or +1
              const int off = dl[q] - (lo ? 1 : 0);
              if (q == 0) kc[j] = off + 1;
              else if (q == 1) kc[j] += 3 * (off + 1);
              else kc[j] += 9 * (off + 1);
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float w = Jc[j][0];
            Jc[j][0] = w * J[j][0];
            Jc[j][1] = w * J[j][1];
            Jc[j][2] = w * J[j][2];
            const int ox = kc[j] % 3 - 1, oy = (kc[j] / 3) % 3 - 1, oz = kc[j] / 9 - 1;
            int k = -1;
            if (key[j] >= 0 && key[j] < kDepositCells) {
              const int kz = key[j] / (kDE * kDE), rem = key[j] - kz * (kDE * kDE);
              const int ky = rem / kDE, kx = rem - ky * kDE;
              const int bx = kx + ox, by = ky + oy, bz = kz + oz;
              if ((unsigned)bx < (unsigned)kDE && (unsigned)by < (unsigned)kDE && (unsigned)bz < (unsigned)kDE)
                k = bx + kDE * (by + kDE * bz);
            }
            if (k < 0 && key[j] >= 0) {  // the global accumulator, periodic corner index
              int gx = cell_i(cs[j]) + ox, gy = cell_j(cs[j]) + oy, gz = cell_k(cs[j]) + oz;
              gx = gx < 0 ? gx + n3[0] : (gx >= n3[0] ? gx - n3[0] : gx);
              gy = gy < 0 ? gy + n3[1] : (gy >= n3[1] ? gy - n3[1] : gy);
              gz = gz < 0 ? gz + n3[2] : (gz >= n3[2] ? gz - n3[2] : gz);
              k = kDepositCells + gx + a.nx * (gy + a.ny * gz);
            }
            kc[j] = k;
          }
          // each particle's corner straight into the tile: neighbouring particles of a cell sit in
          // different half-cells and so rarely share a corner cell, and run sums would only add
          // the cost of forming them
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (kc[j] >= 0) commit_record(a, dep, kc[j], Jc[j][0], Jc[j][1], Jc[j][2]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
    // all gathers of this unit are done: the producer may reuse its fluid buffer
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&tile_empty[buf]);
      mbar_arrive(dep_done);
    }
    // flush the deposit tile once every consumer warp has finished this unit
    if (!mbar_wait(dep_done, loaded & 1)) {
      atomicOr(a.err, 16);
      return;
    }
    for (int t = ctid; t < kDepositCells; t += kConsumerWarps * 32) {
      const int li = t % kDE, lj = (t / kDE) % kDE, lk = t / (kDE * kDE);
      int gi = uo[0] - kR + li, gj = uo[1] - kR + lj, gk = uo[2] - kR + lk;
      gi = gi < 0 ? gi + a.nx : (gi >= a.nx ? gi - a.nx : gi);
      gj = gj < 0 ? gj + a.ny : (gj >= a.ny ? gj - a.ny : gj);
      gk = gk < 0 ? gk + a.nz : (gk >= a.nz ? gk - a.nz : gk);
      const int64_t gc = gi + (int64_t)a.nx * (gj + (int64_t)a.ny * gk);
      for (int q = 0; q < 3; ++q) {
        int* w = dep + q * kDigits * kDepositCells + t;
        const long long val = (long long)w[0] + ((long long)w[kDepositCells] << kDigitBits) +
                              ((long long)w[2 * kDepositCells] << (2 * kDigitBits));
        if (val != 0) {
          w[0] = 0;
          w[kDepositCells] = 0;
          w[2 * kDepositCells] = 0;
          acc_add_mag(a.acc + kAccWords * (q * a.ncell + gc), (unsigned long long)(val < 0 ? -val : val), kDepShift,
                      val < 0);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(flush_done);
    if (!mbar_wait(flush_done, loaded & 1)) {
      atomicOr(a.err, 32);
      return;
    }
    ++loaded;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

bool tma_step_supported(const st_ctx* h) {
  if (h->prec == ST_FP64) return false;
  if (h->geo.B < kU) return false;
  for (int q = 0; q < 3; ++q)
    if (h->geo.n[q] % h->geo.B != 0 || h->geo.n[q] < kTE) return false;
  return h->fluid_pad.p != nullptr;
}

cudaError_t launch_step_mixed_tma(st_ctx* h, const StepParams& p, bool records, bool gather) {
  const bool bf = h->prec == ST_MIXED_BF16V;
  const bool phys = p.ngp || p.semi || p.sn || p.cic;
  if ((records || gather) && phys) return cudaErrorInvalidValue;
  if (records && gather) return cudaErrorInvalidValue;
  bool pw2 = true;
  for (int q = 0; q < 3; ++q) pw2 = pw2 && (h->geo.n[q] & (h->geo.n[q] - 1)) == 0;
  using Kern = void (*)(const CUtensorMap, const TmaArgs);
  static const Kern table[16] = {
      step_mixed_tma_kernel<false, false, false, false, false>, step_mixed_tma_kernel<false, true, false, false, false>,
      step_mixed_tma_kernel<false, false, false, true, false>,  step_mixed_tma_kernel<false, true, false, true, false>,
      step_mixed_tma_kernel<true, false, false, false, false>,  step_mixed_tma_kernel<true, true, false, false, false>,
      step_mixed_tma_kernel<true, false, false, true, false>,   step_mixed_tma_kernel<true, true, false, true, false>,
      step_mixed_tma_kernel<false, false, true, false, false>,  step_mixed_tma_kernel<false, true, true, false, false>,
      step_mixed_tma_kernel<true, false, true, false, false>,   step_mixed_tma_kernel<true, true, true, false, false>,
      step_mixed_tma_kernel<false, false, false, false, true>,  step_mixed_tma_kernel<false, true, false, false, true>,
      step_mixed_tma_kernel<true, false, false, false, true>,   step_mixed_tma_kernel<true, true, false, false, true>};
  constexpr int kAttrDevices = 64;
  // a kernel attribute is per device; atomic because handles may be driven from several host threads
  // (setting an attribute twice is harmless)
  static std::atomic<bool> attr_set[kAttrDevices][16];
  const int variant = gather    ? 12 + 2 * (int)bf + (int)pw2
                      : records ? 8 + 2 * (int)bf + (int)pw2
                                : 4 * (int)bf + 2 * (int)phys + (int)pw2;
  const Kern kern = table[variant];
  if (h->dev < 0 || h->dev >= kAttrDevices) return cudaErrorInvalidDevice;
  if (!attr_set[h->dev][variant].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set[h->dev][variant].store(true, std::memory_order_release);
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const int nx = h->geo.n[0], ny = h->geo.n[1], nz = h->geo.n[2];
  cuuint64_t dims[4] = {4, (cuuint64_t)(nx + 2 * kG), (cuuint64_t)(ny + 2 * kG), (cuuint64_t)(nz + 2 * kG)};
  cuuint64_t strides[3] = {16, (cuuint64_t)16 * (nx + 2 * kG), (cuuint64_t)16 * (nx + 2 * kG) * (ny + 2 * kG)};
  cuuint32_t box[4] = {4, kTE, kTE, kTE};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->fluid_pad.p, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TmaArgs a;
  a.s = carve_mixed(h->state.p, h->cap, bf);
  a.rec = records ? (float4*)h->state_alt.p : nullptr;
  // the deferred gather of the last sort: permutation, records (old order) and ids in, ids out
  a.perm = gather ? (const uint32_t*)h->vals[0].p : nullptr;
  a.grec = gather ? (const float4*)h->state_alt.p : nullptr;
  a.ids_in = gather ? (const uint32_t*)h->ids.p : nullptr;
  a.ids_out = gather ? (uint32_t*)h->ids_alt.p : nullptr;
  a.ngp = p.ngp;
  a.semi = p.semi;
  a.sn = p.sn;
  a.cic = p.cic;
  a.re_coef = (float)p.re_coef;
  a.Up = (const float4*)h->fluid_pad.p;
  a.acc = (long long*)h->acc.p;
  a.cell_start = (const uint32_t*)h->cell_start.p;
  a.err = (int*)h->flags.p;
  a.acc_ctr = (unsigned long long*)((char*)h->flags.p + kAccCounterOffset);
  a.unit_ctr = (unsigned*)((char*)h->flags.p + kUnitCounterOffset);
  {
    cudaError_t e = cudaMemsetAsync(a.unit_ctr, 0, sizeof(unsigned), h->stream);
    if (e != cudaSuccess) return e;
  }
  a.ncell = h->geo.ncell;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.nunits = (int)(h->nkeys / (kU * kU * kU));
  int logB = 0;
  while ((1 << logB) < h->geo.B) ++logB;
  a.logB = logB;
  a.ncx = nx / h->geo.B;
  a.ncy = ny / h->geo.B;
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
  {
    // 2^(E - kDepShift) as two representable factors; beyond +-250 every scaled impulse is 0 or
    // overflows the bound the exponent was chosen for, so clamping changes nothing
    const int Es = std::min(std::max(p.E - kDepShift, -250), 250);
    a.s1 = std::ldexp(1.0f, Es / 2);
    a.s2 = std::ldexp(1.0f, Es - Es / 2);
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev);
  int grid = sms > 0 ? sms : 152;
  if (grid > a.nunits) grid = a.nunits;
  kern<<<grid, kThreads, kSmemBytes, h->stream>>>(map, a);
  h->launches += 1;
  return cudaGetLastError();
}

}  // namespace st
