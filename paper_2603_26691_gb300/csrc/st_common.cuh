// Internal definitions shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "../../include/scaletrack.h"

namespace st {

constexpr int kMaxDim = 1024;       // cells per axis (10-bit fields of the packed cell)
constexpr int kAccBits = 96;        // a contribution at its bound maps to 2^96 in the accumulator
constexpr int kMaxRun = 128;        // particles folded into one committed run (warp x 4)
constexpr int kFluidPad = 3;        // ghost layers around the mixed-precision field

// Owned device allocation.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

// FP64 cell value padded to 32 bytes (x, y, z, 0).
struct alignas(16) D4 {
  double x, y, z, w;
};

// Grid geometry shared by the kernels.
struct Geometry {
  int n[3];
  double L[3];
  double h[3];
  double inv_h[3];
  int B;
  int64_t ncell;
};

}  // namespace st

namespace st {
struct ChunkStore;
struct Xfer;
}

struct st_ctx {
  int dev = 0;
  st::Geometry geo{};
  int prec = ST_FP64;
  st_allocator alloc{};
  bool have_alloc = false;
  cudaStream_t stream = nullptr;

  // physical parameters
  double rho_p = 1000.0, mu = 1.8e-5, g[3] = {0.0, 0.0, -9.81}, alpha = 1.0, mult = 1.0;
  int reorder_every = 10;
  // physics variants (st_set_physics): gather, integrator, drag law, deposit; all 0 by default
  int phys_gather = ST_GATHER_TRILINEAR, phys_integrator = ST_INTEGRATOR_EXPONENTIAL;
  int phys_drag = ST_DRAG_STOKES, phys_deposit = ST_DEPOSIT_CELL;
  double rho_f_drag = 1.2;  // fluid density in the particle Reynolds number

  // fluid: FP64 handles D4[ncell] (x, y, z, 0); mixed handles float4[ncell]
  st::Buf fluid;
  st::Buf fluid_pad;         // mixed handles: float4 field with kFluidPad ghost layers, periodic
  bool fluid_set = false;
  double umax = 0.0;

  // particle state (structure of arrays), capacity a multiple of 64
  int64_t np = 0, cap = 0;
  // FP64: x, y, z, vx, vy, vz, d (double[cap] each)
  // mixed: cell int32[cap], xi float[3][cap], v float[3][cap] (bf16[3][cap]), d float[cap]
  st::Buf state, state_alt;  // one block each; arrays carved at fixed offsets
  st::Buf ids, ids_alt;      // uint32[cap]
  double dmax = 0.0, vbound = 0.0;
  bool sorted = false;
  int steps_since_sort = 0;

  // sort
  uint32_t nkeys = 0;
  int key_bits = 0;
  st::Buf keys[2], vals[2], hist, scan_aux, cell_start;  // cell_start uint32[nkeys + 1]
  st::Buf lsort_aux;         // the neighbourhood sort's per-unit counts, offsets and totals
  int64_t sort_cap = 0;
  uint32_t sort_epoch = 0;   // tags the look-back words of each sort pass (no clearing between passes)
  // The step just before a due sort (mixed handles, sorted step kernel) writes the new state as
  // 32-byte records {cell, offsets | velocity, diameter} into state_alt and only the cells into
  // `state`; the sort gathers from the records.  Until then the offsets, velocities and
  // diameters in `state` are stale: every other reader calls materialize_state first.
  bool records_pending = false;
  // The sort's payload gather deferred to the next step (records_pending stays set): the sorted order
  // is the permutation in vals[0] (cell starts already updated), the state is still the records in
  // the old order and the ids in `ids`.  The next sorted step gathers; any other reader calls
  // materialize_state, which runs the gather.
  bool perm_pending = false;

  // kernel timers (st_timers_*): pending event pairs per kind, folded into sums on read
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[ST_TIMER_COUNT];
  double timer_ms[ST_TIMER_COUNT] = {0, 0, 0, 0};
  int64_t timer_count[ST_TIMER_COUNT] = {0, 0, 0, 0};

  // source accumulator: carry-save words [3][ncell][kAccWords] (int64), units of 2^-acc_E
  st::Buf acc;
  int acc_E = 0;             // value = integer * 2^-acc_E
  bool acc_empty = true;
  double acc_load = 0.0;     // bound on |accumulated integer| (in units of 1), for overflow control

  st::Buf red;               // small reduction scratch
  st::Buf flags;             // device error flags (bounded waits that gave up)

  // adjoint: checkpoints of (x, v) every adj_every steps of the last st_adjoint_forward
  st::Buf ckpt;
  int adj_nsteps = 0, adj_every = 0;
  double adj_dt = 0.0;
  bool adj_ready = false;
  // two-way coupling (st_couple_*): fluid master fields, source history
  double rho_f = 1.2, nu = 1e-3;
  int sweeps = 10, couple_K = 5, extrap = 0;
  int64_t couple_done = 0;   // coupling intervals whose source is in the history ring
  bool fl_valid = false;     // fl_cur holds the current field (mixed handles)
  st::Buf src_hist[4];       // S of the last intervals, FP64 [3][ncell]; interval n in slot n % 4
  st::Buf src_est;           // FP64 [3][ncell]
  st::Buf fl_cur, fl_next, fl_star, fl_tmp;  // fluid fields, float4 (mixed) or D4 (FP64) per cell
  st::Buf fluid_pad_next;    // mixed: the padded field of the next interval
  st::Buf umax_dev;          // max |u| of the next field (bits of a non-negative double)
  double* umax_host = nullptr;  // pinned
  cudaEvent_t ev_fluid = nullptr;  // the interval's fluid update done (its max |u| in umax_host)
  int64_t launches = 0;      // kernels launched by this handle

  // droplet microphysics (st_set_microphysics): vapour mass and heat transfer of Sec. 2.1
  bool micro_on = false;
  double mi_Dv = 2.5e-5, mi_kappa = 0.025, mi_cp = 4186.0, mi_L = 2.5e6, mi_Pr = 0.71, mi_dmin = 1e-7;
  double mi_Tinit = 293.15;
  st::Buf temp, temp_alt;    // particle temperatures (FP64 handles double[cap], mixed float[cap])
  st::Buf thermo;            // fluid temperature and vapour density per cell: double2[ncell] (FP64) or
                             // float2 with kFluidPad ghost layers (mixed)
  bool thermo_set = false;
  double rv_max = 0.0;       // largest vapour density of the field (bounds droplet growth per step)
  st::Buf acc_micro;         // exact sources [2][ncell][kWideWords]: vapour mass, energy the fluid gains
  double micro_adds = 0.0;   // digits added to any word of acc_micro since its last carry propagation

  // chunked particle sets (st_chunks_*): the chunks in pinned host memory and the device slots
  st::ChunkStore* chunks = nullptr;
  bool chunk_adding = false;  // st_chunks_add is importing through the resident path
  // asynchronous host transfers (st_set_fluid_async, st_get_sources_async): streams, staging buffers
  st::Xfer* xfer = nullptr;
  std::string err;
};

namespace st {

// ---- chunked particle sets (chunks.cu) ------------------------------------------------------
void chunk_store_free(st_ctx* h);

// ---- asynchronous host transfers (xfer.cu) --------------------------------------------------
void xfer_free(st_ctx* h);
cudaError_t xfer_sync(st_ctx* h);  // waits for the upload and download streams
// read the scan result of a pending asynchronous field upload (waits for it): the field's bound, or
// ST_ERR_NONFINITE when it was not taken; no-op without one
st_status settle_fluid(st_ctx* h);
// device error flags raised by bounded waits that gave up (reported and cleared)
st_status check_flags(st_ctx* h);

// ---- host helpers (st_api.cu) -------------------------------------------------------------
st_status set_error(st_ctx* h, st_status s, const std::string& msg);
st_status cuda_check(st_ctx* h, cudaError_t e, const char* what);
st_status dev_alloc(st_ctx* h, Buf& b, size_t bytes);
void dev_free(st_ctx* h, Buf& b);

#define ST_TRY(expr)                     \
  do {                                   \
    st_status _s = (expr);               \
    if (_s != ST_OK) return _s;          \
  } while (0)

#define ST_CUDA(h, expr) ST_TRY(cuda_check((h), (expr), #expr))
st_status ensure(st_ctx* h, Buf& b, size_t bytes);  // grow-only

// carve the state block
inline size_t state_bytes(int prec, int64_t cap) {
  if (prec == ST_FP64) return (size_t)cap * 7 * sizeof(double);
  size_t vb = (prec == ST_MIXED_BF16V) ? sizeof(__nv_bfloat16) : sizeof(float);
  return (size_t)cap * (sizeof(int32_t) + 3 * sizeof(float) + 3 * vb + sizeof(float));
}

struct F64State {
  double* x[3];
  double* v[3];
  double* d;
};

struct MixedState {
  int32_t* cell;
  float* xi[3];
  void* v[3];  // float* or __nv_bfloat16*
  float* d;
};

// the sort's spare buffer: room for the state, and on mixed handles for 32-byte particle records
inline size_t state_alt_bytes(int prec, int64_t cap) {
  const size_t b = state_bytes(prec, cap);
  return prec == ST_FP64 ? b : std::max(b, (size_t)cap * 32);
}

inline F64State carve_f64(void* base, int64_t cap) {
  F64State s;
  double* p = (double*)base;
  for (int q = 0; q < 3; ++q) s.x[q] = p + q * cap;
  for (int q = 0; q < 3; ++q) s.v[q] = p + (3 + q) * cap;
  s.d = p + 6 * cap;
  return s;
}

inline MixedState carve_mixed(void* base, int64_t cap, bool bf16) {
  MixedState s;
  char* p = (char*)base;
  s.cell = (int32_t*)p;
  p += cap * sizeof(int32_t);
  for (int q = 0; q < 3; ++q) {
    s.xi[q] = (float*)p;
    p += cap * sizeof(float);
  }
  size_t vb = bf16 ? sizeof(__nv_bfloat16) : sizeof(float);
  for (int q = 0; q < 3; ++q) {
    s.v[q] = (void*)p;
    p += cap * vb;
  }
  s.d = (float*)p;
  return s;
}

// ---- packed cell: i | j << 10 | k << 20 ---------------------------------------------------
__host__ __device__ inline int32_t pack_cell(int i, int j, int k) { return i | (j << 10) | (k << 20); }
__host__ __device__ inline int cell_i(int32_t c) { return c & 1023; }
__host__ __device__ inline int cell_j(int32_t c) { return (c >> 10) & 1023; }
__host__ __device__ inline int cell_k(int32_t c) { return (c >> 20) & 1023; }

// chunk-major key: chunk (x fastest) * B^3 + Morton(local), local x bit lowest
__host__ __device__ inline uint32_t spread3(uint32_t v) {
  // bit b of v -> bit 3b (v < 32)
  v &= 0x1f;
  v = (v | (v << 8)) & 0x0000f00fu;
  v = (v | (v << 4)) & 0x000c30c3u;
  v = (v | (v << 2)) & 0x00249249u;
  return v;
}

__host__ __device__ inline uint32_t chunk_key(int i, int j, int k, int B, int logB, int ncx, int ncy) {
  uint32_t ci = (uint32_t)i >> logB, cj = (uint32_t)j >> logB, ck = (uint32_t)k >> logB;
  uint32_t li = (uint32_t)i & (B - 1), lj = (uint32_t)j & (B - 1), lk = (uint32_t)k & (B - 1);
  uint32_t chunk = ci + (uint32_t)ncx * (cj + (uint32_t)ncy * ck);
  uint32_t morton = spread3(li) | (spread3(lj) << 1) | (spread3(lk) << 2);
  return (chunk << (3 * logB)) | morton;
}

// ---- exact fixed-point deposit -------------------------------------------------------------
// The per-cell source is an integer multiple of 2^-E per component, kept in carry-save form:
// kAccWords int64 words w[k] of signed 32-bit digits, value = sum_k w[k] 2^(32 k).  A
// contribution adds at most three digits with fire-and-forget atomic adds (no return value, so
// no round trip to L2 stalls the warp); integer addition is associative, so the sum is the same
// whatever order the contributions arrive in.  Each word absorbs 2^31 contributions before a
// normalisation pass (carry propagation) is needed; the host tracks that bound.

constexpr int kAccWords = 4;

// add sign * m * 2^s (m < 2^64, 0 <= s, s + 64 <= 32 * kAccWords + 32) to the words p[0..3]
__device__ __forceinline__ void acc_add_mag(long long* p, unsigned long long m, int s, bool neg) {
  if (m == 0) return;
  const int q = s >> 5, r = s & 31;
  const unsigned long long lo = m << r;
  const unsigned long long hi = r ? (m >> (64 - r)) : 0ull;
  long long d0 = (long long)(lo & 0xffffffffull), d1 = (long long)(lo >> 32), d2 = (long long)hi;
  if (neg) {
    d0 = -d0;
    d1 = -d1;
    d2 = -d2;
  }
  if (d0 && q < kAccWords) atomicAdd((unsigned long long*)&p[q], (unsigned long long)d0);
  if (d1 && q + 1 < kAccWords) atomicAdd((unsigned long long*)&p[q + 1], (unsigned long long)d1);
  if (d2 && q + 2 < kAccWords) atomicAdd((unsigned long long*)&p[q + 2], (unsigned long long)d2);
}

// add round(f * 2^E) (FP32 input; integer operations only) -- requires |f| 2^E < 2^100
__device__ __forceinline__ void acc_add_f32(long long* p, float f, int E) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t ex = (b >> 23) & 0xffu;
  unsigned long long man = b & 0x7fffffu;
  if (ex != 0) man |= 0x800000ull;
  int s = (int)(ex == 0 ? 1 : ex) - 150 + E;
  if (s < 0) {
    const int r = -s;
    man = r < 32 ? ((man + ((1ull << r) >> 1)) >> r) : 0ull;
    s = 0;
  }
  acc_add_mag(p, man, s, (b >> 31) != 0);
}

// add round(x * 2^E) (FP64 input; integer operations only) -- requires |x| 2^E < 2^100
__device__ __forceinline__ void acc_add_f64(long long* p, double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  unsigned long long man = b & 0xfffffffffffffull;
  if (ex != 0) man |= 1ull << 52;
  int s = (ex == 0 ? 1 : ex) - 1075 + E;
  if (s < 0) {
    const int r = -s;
    man = r < 64 ? ((man + ((1ull << r) >> 1)) >> r) : 0ull;
    s = 0;
  }
  acc_add_mag(p, man, s, (b >> 63) != 0);
}

// exact value of carry-save words as a 128-bit two's-complement integer (lo, hi)
__device__ __forceinline__ void acc_value(const long long* w, unsigned long long& lo, long long& hi) {
  long long c = 0;
  unsigned long long d[3];
  for (int k = 0; k < 3; ++k) {
    const long long t = w[k] + c;
    d[k] = (unsigned long long)t & 0xffffffffull;
    c = t >> 32;
  }
  const long long top = w[3] + c;
  lo = d[0] | (d[1] << 32);
  hi = (long long)d[2] + (long long)((unsigned long long)top << 32);
}

// a two's-complement 128-bit integer hi:lo as a double, through its sign and magnitude: summing the
// signed halves directly would cancel, losing a small negative value (hi = -1, lo close to 2^64)
__host__ __device__ __forceinline__ double i128_to_f64(unsigned long long lo, long long hi) {
  const bool neg = hi < 0;
  unsigned long long mlo = lo, mhi = (unsigned long long)hi;
  if (neg) {
    mlo = ~lo + 1ull;
    mhi = ~mhi + (mlo == 0 ? 1ull : 0ull);
  }
  const double m = (double)mhi * 0x1p64 + (double)mlo;
  return neg ? -m : m;
}

// 128-bit add with carry-out, used by the exact reductions (returns the old value from memory)
__device__ __forceinline__ void atomic_add_i128(unsigned long long* p, unsigned long long lo,
                                                unsigned long long hi) {
  unsigned long long carry = 0;
  if (lo) {
    unsigned long long old = atomicAdd(p, lo);
    carry = (old + lo < old) ? 1ull : 0ull;
  }
  unsigned long long hh = hi + carry;
  if (hh) atomicAdd(p + 1, hh);
}

// y = J * 2^E (exact), rounded to an integer, split into 64-bit words.
// Requires |J * 2^E| < 2^117.
__device__ __forceinline__ void f64_to_i128(double J, double scale, unsigned long long& lo,
                                            unsigned long long& hi) {
  double y = rint(J * scale);
  double yh = floor(y * 0x1p-64);
  double yl = y - yh * 0x1p64;
  lo = (unsigned long long)__double2ull_rz(yl);
  hi = (unsigned long long)(long long)yh;
}

// ---- launchers implemented in the other translation units --------------------------------
struct StepParams {
  double dt;
  double ca;       // a * d^2 = 18 mu alpha / rho_p
  double mcoef;    // m / d^3 = mult rho_p pi / 6
  double g[3];
  double scale;    // 2^E for the FP64 path
  int E;           // for the FP32 path
  // physics variants (nonzero = nearest grid point, semi-implicit Euler, Schiller-Naumann,
  // cloud-in-cell deposit) and rho_f / mu for the particle Reynolds number
  int ngp = 0, semi = 0, sn = 0, cic = 0;
  double re_coef = 0.0;
};

// every physics switch at its default (the sorted TMA step kernel implements only this)
inline bool default_physics(const st_ctx* h) {
  return h->phys_gather == ST_GATHER_TRILINEAR && h->phys_integrator == ST_INTEGRATOR_EXPONENTIAL &&
         h->phys_drag == ST_DRAG_STOKES && h->phys_deposit == ST_DEPOSIT_CELL;
}

cudaError_t launch_step_f64(st_ctx* h, const StepParams& p);
// the FP64 step on an explicit state; acc == nullptr skips the deposit (adjoint recomputation)
cudaError_t launch_step_f64_state(st_ctx* h, const F64State& s, long long* acc, const StepParams& p);

// ---- adjoint (adjoint.cu) ----------------------------------------------------------------------
constexpr int kWideWords = 8;     // carry-save accumulator: 8 words of 32-bit digits
constexpr int kWideBase = -160;   // weight of the lowest digit: 2^-160
constexpr int kAdjBlocks = 152 * 8;

// Carry-save accumulator: value = sum_i w[i] * 2^(32 i + kWideBase); each
// contribution adds 32-bit digits, so each int64 word absorbs 2^31 of them.
// an FP32 value into the same accumulator: its 24-bit significand spans at most two words
__device__ __forceinline__ void wide_add_f32(long long* w, float x) {
  if (x == 0.0f) return;
  const uint32_t b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xff);
  unsigned long long man = b & 0x7fffffu;
  if (ex != 0) man |= 1u << 23;                       // subnormals: man * 2^(1 - 150)
  const int s = (ex == 0 ? 1 : ex) - 150 - kWideBase;  // >= 11: every FP32 value is on the grid
  const int q = s >> 5, r = s & 31;
  const unsigned long long lo = man << r;  // < 2^55
  long long d0 = (long long)(lo & 0xffffffffull);
  long long d1 = (long long)(lo >> 32);
  if (b >> 31) {
    d0 = -d0;
    d1 = -d1;
  }
  if (d0 != 0 && q < kWideWords) atomicAdd((unsigned long long*)&w[q], (unsigned long long)d0);
  if (d1 != 0 && q + 1 < kWideWords) atomicAdd((unsigned long long*)&w[q + 1], (unsigned long long)d1);
}

__device__ __forceinline__ void wide_add(long long* w, double x) {
  if (x == 0.0) return;
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  unsigned long long man = b & 0xfffffffffffffull;
  if (ex != 0) man |= 1ull << 52;  // subnormals: man * 2^(1 - 1075)
  int s = (ex == 0 ? 1 : ex) - 1075 - kWideBase;  // bit position of man's lowest bit
  if (s < 0) {
    if (s <= -64) return;
    man = (man + ((1ull << (-s)) >> 1)) >> (-s);
    s = 0;
  }
  const int q = s >> 5, r = s & 31;
  const unsigned long long lo = man << r;                       // bits r .. 63
  const unsigned long long hi = r ? (man >> (64 - r)) : 0ull;   // bits 64 .. 84
  long long d0 = (long long)(lo & 0xffffffffull);
  long long d1 = (long long)(lo >> 32);
  long long d2 = (long long)hi;
  if (b >> 63) {
    d0 = -d0;
    d1 = -d1;
    d2 = -d2;
  }
  if (q < kWideWords) atomicAdd((unsigned long long*)&w[q], (unsigned long long)d0);
  if (q + 1 < kWideWords) atomicAdd((unsigned long long*)&w[q + 1], (unsigned long long)d1);
  if (q + 2 < kWideWords) atomicAdd((unsigned long long*)&w[q + 2], (unsigned long long)d2);
}

// ---- sums over a warp's lanes of equal key, before one exact commit per key ----

// sum of v over the run of equal key that starts at this lane (runs in lane order), for lanes that
// start a run (others: partial sums).  Every lane of the warp calls it.
template <class R, int K>
__device__ __forceinline__ bool run_sums(int lane, int key, R (&v)[K]) {
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  const bool head = (lane == 0) || (prev != key);
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const unsigned above = lane == 31 ? 0u : (heads & ~((2u << lane) - 1u));
  const int end = above ? (__ffs(above) - 2) : 31;
  for (int off = 1; off < 32; off <<= 1) {
    R t[K];
#pragma unroll
    for (int q = 0; q < K; ++q) t[q] = __shfl_down_sync(0xffffffffu, v[q], off);
    if (lane + off <= end) {
#pragma unroll
      for (int q = 0; q < K; ++q) v[q] += t[q];
    }
  }
  return head;
}

// The place of this lane when a warp's lanes are reordered so that equal keys are adjacent: groups in
// the order of their lowest lane, lanes inside a group in lane order.  A permutation of 0..31 that
// depends only on the keys, so sums formed over the reordered lanes are reproducible.  Particles that
// drifted from their sort-time cells put several keys into one warp in alternation; reordered, each
// distinct key is one run for run_sums and one commit.
__device__ __forceinline__ int key_group_slot(int lane, unsigned grp) {  // grp: the lanes of this lane's key
  const int leader = __ffs(grp) - 1;
  const int rank = __popc(grp & ((1u << lane) - 1u));
  const int size = leader == lane ? __popc(grp) : 0;
  int incl = size;  // inclusive prefix of the group sizes over the leaders, in lane order
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  return __shfl_sync(0xffffffffu, incl - size, leader) + rank;
}
__device__ __forceinline__ int key_group_slot(int lane, int key) {
  return key_group_slot(lane, (unsigned)__match_any_sync(0xffffffffu, key));
}

// per-warp staging of K values and the key for the reordering
template <int K>
struct GroupBuf {
  float g[K][32];
  int key[32];
};

// moves this lane's values to its slot and takes the values that land on this lane
template <int K>
__device__ __forceinline__ void group_permute(GroupBuf<K>& b, int slot, int lane, float (&v)[K]) {
  __syncwarp();  // the previous use's reads are done
#pragma unroll
  for (int q = 0; q < K; ++q) b.g[q][slot] = v[q];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = b.g[q][lane];
}
__device__ __forceinline__ int group_permute_key(int* keys, int slot, int lane, int key) {
  __syncwarp();
  keys[slot] = key;
  __syncwarp();
  return keys[lane];
}

// both at once, for a single use: afterwards equal keys are adjacent
template <int K>
__device__ __forceinline__ void group_by_key(GroupBuf<K>& b, int lane, int& key, float (&v)[K]) {
  const int slot = key_group_slot(lane, key);
  group_permute(b, slot, lane, v);
  key = group_permute_key(b.key, slot, lane, key);
}


struct AdjointStepArgs {
  const double* x[3];
  const double* v[3];
  const double* d;
  double* xb[3];
  double* vb[3];
  double* db;
  double* ab_part;
  const double* lam;
  long long* Uw;
  double dt;
};
cudaError_t launch_adjoint_step(st_ctx* h, const AdjointStepArgs& s);
// the FP32 adjoint of the mixed-precision step (FP32-velocity handles): the tape holds the state at
// the start of the step (cell, offsets, velocities; diameters in d), the adjoints of position and
// velocity are FP32 arrays, dL/dd and dL/dalpha accumulate in FP64, dL/dU goes into the same exact
// carry-save accumulator as the FP64 adjoint; lam32 = dL/dJtot per cell in FP32 [3][ncell]
struct AdjointMixedArgs {
  MixedState tape;
  const float* d;
  float* xb[3];
  float* vb[3];
  double* db;
  double* ab_part;
  const float* lam32;
  long long* Uw;
  double dt;
};
cudaError_t launch_adjoint_step_mixed(st_ctx* h, const AdjointMixedArgs& s);
cudaError_t launch_f64_to_f32(st_ctx* h, const double* in, float* out, int64_t m);
cudaError_t launch_wide_to_f64(st_ctx* h, const long long* Uw, double* out, int64_t m);
cudaError_t launch_step_mixed(st_ctx* h, const StepParams& p);
// the general mixed step on any state of the handle's capacity layout; acc = nullptr deposits nothing
cudaError_t launch_step_mixed_state(st_ctx* h, const MixedState& s, int64_t n, long long* acc, const StepParams& p);
bool tma_step_supported(const st_ctx* h);                               // step_mixed_tma.cu
// records = true (mixed handles, default physics): the new state goes out as 32-byte records into
// state_alt (plus the cells into the structure of arrays) for the sort that follows; see
// records_pending
// gather = true: the first step after a sort whose payload gather was deferred (perm_pending); it reads
// the records through the permutation and writes the sorted state, diameters and ids included
cudaError_t launch_step_mixed_tma(st_ctx* h, const StepParams& p, bool records, bool gather);  // step_mixed_tma.cu
cudaError_t launch_rescale_acc(st_ctx* h, int shift);
cudaError_t launch_normalize_acc(st_ctx* h);
// the particle steps of st_step (sort when due, accumulator bookkeeping, step kernel)
st_status run_steps(st_ctx* h, int nsteps, double dt);
// word-capacity bookkeeping of the carry-save accumulator, on the device: a counter (in the flags
// buffer) bounds the digits added to any word since the last carry propagation; before each step
// the propagation runs if the counter plus the step's worst case could overflow a word.  `add` is
// what the step adds for sure (its flushes, or its worst case when it does not count itself);
// kernels that add more (global commits of the sorted-step kernel) count them on the device.
cudaError_t launch_acc_maybe_normalize(st_ctx* h, double worst, double add);
cudaError_t reset_acc_counter(st_ctx* h);
constexpr size_t kAccCounterOffset = 64;   // bytes into the flags buffer: uint64 counter
constexpr size_t kAccFlagOffset = 72;      // int: 1 if the last check propagated carries
constexpr size_t kUnitCounterOffset = 80;  // uint32: next unit of the sorted-step kernel
constexpr size_t kFarFlagOffset = 84;      // int: the neighbourhood sort found a particle it cannot place
cudaError_t launch_acc_to_f64(st_ctx* h, double* out, int E);
cudaError_t launch_acc_sum(st_ctx* h, double out[3]);
cudaError_t launch_particle_sums(st_ctx* h, double out[4]);  // P_x, P_y, P_z, M
cudaError_t launch_maxabs(st_ctx* h, const void* p, int64_t n, int dtype, double* out_max, int* nonfinite);
// the same scan on `stream`, its 16-byte result {max bits, flag} left in dev_red and copied to host_red
// (pinned) asynchronously
cudaError_t launch_maxabs_on(st_ctx* h, const void* p, int64_t n, int dtype, cudaStream_t stream,
                             unsigned long long* dev_red, unsigned long long* host_red);
cudaError_t launch_particle_scan(st_ctx* h, const double* vel, const double* d, int64_t n, double* vmax,
                                 double* dmax, double* dmin, int* nonfinite);
cudaError_t launch_fluid_pack(st_ctx* h, const void* u, int dtype);
// the same, skipped on the device when *skip != 0
cudaError_t launch_fluid_pack_if(st_ctx* h, const void* u, int dtype, const int* skip);
cudaError_t launch_import(st_ctx* h, int64_t first, int64_t n, const double* xyz, const double* vel,
                          const double* d, const uint32_t* ids);
cudaError_t launch_export(st_ctx* h, int64_t first, int64_t n, double* xyz, double* vel, double* d,
                          uint32_t* ids, int32_t* cells);
cudaError_t launch_gen(st_ctx* h, uint64_t seed, int64_t first, int64_t count, const double L[3],
                       double vmax, const double* qtable, int nq, double* xyz, double* vel, double* d,
                       uint32_t* ids);
st_status sort_particles(st_ctx* h);                                       // sort.cu
// the neighbourhood sort (sort_local.cu): particles sorted before (h->sorted), mixed state, chunks
// of at least 8^3 cells dividing the grid.  It sets *far and leaves everything else untouched if a
// particle lies beyond the 26 units around its sort-time unit; otherwise it writes the sorted state
// (records or arrays, as sort_particles' own gather), the ids into ids_alt and the cell starts.
// lidx, lkey and perm are scratch of n entries, aux local_sort_aux_bytes(h).
bool local_sort_supported(const st_ctx* h);
size_t local_sort_aux_bytes(const st_ctx* h);
cudaError_t launch_local_sort(st_ctx* h, int* far, uint32_t* lidx, uint16_t* lkey, uint32_t* perm, void* aux);
// the structure of arrays current again if the last step left records for a sort (no-op otherwise)
st_status materialize_state(st_ctx* h);                                    // sort.cu
// whether a sort may leave its payload gather to the next step (mixed, sorted-step kernel, default
// physics, no microphysics, and the next step does not itself write records), and the bookkeeping
// once that step has gathered (ids swapped, nothing pending)
bool defer_gather(const st_ctx* h);                                        // sort.cu
void gather_step_done(st_ctx* h);                                          // sort.cu
// FP64 and FP32 FMA rates of this GPU (GFLOP/s), measured by FMA-chain kernels; synchronises
cudaError_t probe_fma_rates(st_ctx* h, double* fp64_gflops, double* fp32_gflops);  // util.cu
// timer marks around a launch of kind k on stream s (no-ops unless st_timers_enable is on); the
// end mark pairs with the last begin of the same kind
void timer_begin(st_ctx* h, int k, cudaStream_t s);                        // st_api.cu
void timer_end(st_ctx* h, int k, cudaStream_t s);                          // st_api.cu
cudaError_t launch_cell_counts(st_ctx* h, int64_t* counts);
// ---- droplet microphysics (micro.cu) -------------------------------------------------------------
// the step with vapour mass and heat transfer (default physics only; accumulators prepared)
// records (mixed handles): the new state as 32-byte records into state_alt (cells also into the arrays)
cudaError_t launch_micro_step(st_ctx* h, const StepParams& p, bool records = false);
// before a microphysics step: widen the diameter bound by the largest growth one step allows, and
// propagate the carries of the microphysics accumulator when the step could overflow a word
st_status micro_prepare_step(st_ctx* h, double dt);
// the sort's permutation applied to the particle temperatures (temp -> temp_alt); gate as the sort's
cudaError_t launch_gather_temp(st_ctx* h, const uint32_t* perm, const int* gate, int want);
// the temperatures of particles [first, first + n) set to `T` (new particles, enabling microphysics)
cudaError_t launch_fill_temp(st_ctx* h, int64_t first, int64_t n, double T);
// the temperature arrays grown to the handle's capacity (microphysics on), contents kept
st_status micro_grow(st_ctx* h);
cudaError_t launch_chunk_bounds(st_ctx* h, double* out);              // sort.cu

}  // namespace st
