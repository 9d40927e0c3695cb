// Stable counting sort of particles that were sorted before and have moved little since.
//
// The sort key is chunk-major with a Morton order inside the chunk, so every aligned block of
// 8^3 cells (a "unit") is a contiguous range of 512 keys, and after a sort the particles of a unit
// are contiguous in storage.  Between sorts a particle moves a few cells at most, so it ends up in
// its sort-time unit or in one of the 26 units around it.  The stable sort by the new key is then
// a stable sort by (destination unit, key inside the unit), ties kept in storage order, and it
// needs no global radix passes:
//   1. count: per source unit S (the particles of S's storage range), how many particles now lie
//      in each of the 27 units around S, and whether any lies farther away;
//   2. dest: per destination unit D, its 27 possible sources in storage order (increasing unit
//      index), the offset of each (S -> D) bucket inside D's incoming list, and D's total;
//   3. scan: the exclusive scan of the totals gives each D's range of the sorted storage;
//   4. scatter: per S, a stable partition of its particles into its 27 buckets, written as
//      (storage index, key inside D) entries into the incoming lists; each list is in storage
//      order because its buckets are;
//   5. rank: per D, a stable counting sort of the incoming list on the 9-bit key inside D (per-warp
//      counts, warp-order offsets, ranks from __match_any_sync), which gives the permutation of D's
//      range of the sorted storage and D's 512 cell starts.
// The payload (32-byte records from the step before the sort, or the arrays) is then gathered
// through the permutation by the sort's own gather, which serves both sorts.  Each warp works on a
// contiguous segment of a unit and reads it eight 32-element chunks at a time, so that loads overlap
// although the ranking itself is sequential.  If any particle lies farther than the 26 neighbouring
// units, a device flag set by the count makes steps 4 and 5 return at once, and the general radix
// sort, queued behind them with the opposite gate, runs instead; the host never waits.  Both leave
// the same permutation in the same buffer.
#include <cstdint>

#include "st_common.cuh"
#include "st_ptx.cuh"

namespace st {
namespace {

constexpr int kUE = 8;              // unit edge (cells)
constexpr int kUnitKeys = 512;      // keys per unit
constexpr int kDirs = 27;           // destination units around a source unit
constexpr int kCodes = kDirs + 1;   // + "farther away"
constexpr int kFar = kDirs;
constexpr int kLThreads = 256;             // count and scatter: one unit per block
constexpr int kLWarps = kLThreads / 32;
constexpr int kRThreads = 512;             // rank: one destination unit per block
constexpr int kRWarps = kRThreads / 32;
constexpr int kBatch = 8;                  // 32-element chunks a warp loads before ranking them

struct UnitGeo {
  int nu[3];          // units per axis
  int B, logB, ncx, ncy;
  int nunits;
};

// cell coordinate bits 0, 3, 6, ... of m packed together
__device__ __forceinline__ uint32_t demorton3(uint32_t m) {
  m &= 0x09249249u;
  m = (m | (m >> 2)) & 0x030c30c3u;
  m = (m | (m >> 4)) & 0x0300f00fu;
  m = (m | (m >> 8)) & 0xff0000ffu;
  m = (m | (m >> 16)) & 0x000003ffu;
  return m;
}

// unit coordinates (origin cell / 8) of unit u, the key range [512 u, 512 u + 512)
__device__ __forceinline__ void unit_coords(const UnitGeo& g, uint32_t u, int& x, int& y, int& z) {
  const uint32_t key = u * kUnitKeys;
  const uint32_t chunk = key >> (3 * g.logB);
  const uint32_t m = key & ((1u << (3 * g.logB)) - 1u);
  const int cx = (int)(chunk % (uint32_t)g.ncx);
  const int cy = (int)((chunk / (uint32_t)g.ncx) % (uint32_t)g.ncy);
  const int cz = (int)(chunk / ((uint32_t)g.ncx * (uint32_t)g.ncy));
  x = (cx * g.B + (int)demorton3(m)) / kUE;
  y = (cy * g.B + (int)demorton3(m >> 1)) / kUE;
  z = (cz * g.B + (int)demorton3(m >> 2)) / kUE;
}

__device__ __forceinline__ uint32_t unit_index(const UnitGeo& g, int x, int y, int z) {
  return chunk_key(x * kUE, y * kUE, z * kUE, g.B, g.logB, g.ncx, g.ncy) / kUnitKeys;
}

// step -1, 0 or +1 from unit coordinate s to t along an axis of nu units (periodic), or 2 if t is
// farther; with nu = 2 the other unit counts as +1, with nu = 1 every step is 0
__device__ __forceinline__ int axis_step(int s, int t, int nu) {
  if (t == s) return 0;
  int up = s + 1;
  if (up == nu) up = 0;
  if (t == up) return 1;
  int dn = s - 1;
  if (dn < 0) dn = nu - 1;
  return t == dn ? -1 : 2;
}

// bucket code of a particle of source unit (sx, sy, sz) now in packed cell c: the direction
// (dx + 1) + 3 (dy + 1) + 9 (dz + 1) of its unit, or kFar
__device__ __forceinline__ int code_of(const UnitGeo& g, int sx, int sy, int sz, int32_t c) {
  const int ax = axis_step(sx, cell_i(c) / kUE, g.nu[0]);
  const int ay = axis_step(sy, cell_j(c) / kUE, g.nu[1]);
  const int az = axis_step(sz, cell_k(c) / kUE, g.nu[2]);
  if (ax == 2 || ay == 2 || az == 2) return kFar;
  return (ax + 1) + 3 * (ay + 1) + 9 * (az + 1);
}

__device__ __forceinline__ int wrap_add(int a, int d, int n) {
  int r = a + d;
  if (r >= n) r -= n;
  if (r < 0) r += n;
  return r;
}

// a warp's share of [p0, p1) among `warps` warps: contiguous segments of a multiple of 32, in warp
// order
__device__ __forceinline__ void warp_segment(int64_t p0, int64_t p1, int w, int warps, int64_t& s0, int64_t& s1) {
  const int64_t m = p1 - p0;
  const int64_t seg = ((m + warps - 1) / warps + 31) & ~int64_t(31);
  s0 = min(p1, p0 + seg * w);
  s1 = min(p1, s0 + seg);
}

// 1. per source unit: particles per direction code, per warp segment (cntw[S][w][kCodes], the same
// segments as the scatter) and in all (cnt[S][kCodes]); any farther particle sets *far
__global__ void __launch_bounds__(kLThreads) usort_count_kernel(const int32_t* __restrict__ cell,
                                                                const uint32_t* __restrict__ cs_old, UnitGeo g,
                                                                uint32_t* __restrict__ cnt,
                                                                uint32_t* __restrict__ cntw, int* __restrict__ far) {
  __shared__ uint32_t wc[kLWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int S = blockIdx.x; S < g.nunits; S += gridDim.x) {
    wc[w][lane] = 0;
    const int64_t p0 = cs_old[(int64_t)S * kUnitKeys], p1 = cs_old[(int64_t)(S + 1) * kUnitKeys];
    int sx, sy, sz;
    unit_coords(g, (uint32_t)S, sx, sy, sz);
    int64_t s0, s1;
    warp_segment(p0, p1, w, kLWarps, s0, s1);
    __syncwarp();
    for (int64_t b = s0; b < s1; b += 32 * kBatch) {
      int32_t c[kBatch];
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const int64_t p = b + 32 * r + lane;
        c[r] = p < s1 ? __ldcs(cell + p) : -1;
      }
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const bool valid = c[r] >= 0;
        const int code = valid ? code_of(g, sx, sy, sz, c[r]) : 31;
        const unsigned peers = __match_any_sync(0xffffffffu, code);
        if (valid && lane == __ffs(peers) - 1) wc[w][code] += (uint32_t)__popc(peers);
        __syncwarp();
      }
    }
    __syncthreads();
    if (threadIdx.x < kCodes) {
      uint32_t t = 0;
      for (int ww = 0; ww < kLWarps; ++ww) {
        cntw[((int64_t)S * kLWarps + ww) * kCodes + threadIdx.x] = wc[ww][threadIdx.x];
        t += wc[ww][threadIdx.x];
      }
      cnt[(int64_t)S * kCodes + threadIdx.x] = t;
      if (threadIdx.x == kFar && t != 0) atomicOr(far, 1);
    }
    __syncthreads();
  }
}

// 2. per destination unit D: its sources S = D - d(k) in increasing unit index (their storage
// order), the offset rel[S][k] of bucket (S, k) inside D's incoming list, and D's total
__global__ void usort_dest_kernel(UnitGeo g, const uint32_t* __restrict__ cnt, uint32_t* __restrict__ rel,
                                  uint32_t* __restrict__ total) {
  for (int D = blockIdx.x * blockDim.x + threadIdx.x; D < g.nunits; D += gridDim.x * blockDim.x) {
    int x, y, z;
    unit_coords(g, (uint32_t)D, x, y, z);
    uint32_t src[kDirs];
    uint8_t ord[kDirs];
#pragma unroll 1
    for (int k = 0; k < kDirs; ++k) {
      const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
      src[k] = unit_index(g, wrap_add(x, -dx, g.nu[0]), wrap_add(y, -dy, g.nu[1]), wrap_add(z, -dz, g.nu[2]));
      // insertion into the order by source unit (stable; equal sources only arise on axes of one or
      // two units, where all but one of them have empty buckets)
      int j = k;
      while (j > 0 && src[ord[j - 1]] > src[k]) {
        ord[j] = ord[j - 1];
        --j;
      }
      ord[j] = (uint8_t)k;
    }
    uint32_t acc = 0;
#pragma unroll 1
    for (int r = 0; r < kDirs; ++r) {
      const int k = ord[r];
      rel[(int64_t)src[k] * kDirs + k] = acc;
      acc += cnt[(int64_t)src[k] * kCodes + k];
    }
    total[D] = acc;
  }
}

// 3. exclusive scan of the per-unit totals (one block): base[D], base[nunits] = the particle count
__global__ void __launch_bounds__(1024) usort_scan_kernel(const uint32_t* __restrict__ total, int nunits,
                                                          uint32_t* __restrict__ base) {
  __shared__ uint32_t part[1024];
  const int per = (nunits + 1023) / 1024;
  const int t0 = min((int)threadIdx.x * per, nunits), t1 = min(t0 + per, nunits);
  uint32_t s = 0;
  for (int i = t0; i < t1; ++i) s += total[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t acc = part[threadIdx.x] - s;
  for (int i = t0; i < t1; ++i) {
    base[i] = acc;
    acc += total[i];
  }
  if (threadIdx.x == 1023) base[nunits] = part[1023];
}

// 4. per source unit: stable partition into the 27 buckets, as (storage index, key inside the
// destination unit) entries of the destinations' incoming lists; each warp starts its buckets where
// the counts of the earlier warps' segments end
__global__ void __launch_bounds__(kLThreads) usort_scatter_kernel(const int32_t* __restrict__ cell,
                                                                  const uint32_t* __restrict__ cs_old, UnitGeo g,
                                                                  const uint32_t* __restrict__ cntw,
                                                                  const uint32_t* __restrict__ rel,
                                                                  const uint32_t* __restrict__ base,
                                                                  uint32_t* __restrict__ lidx,
                                                                  uint16_t* __restrict__ lkey,
                                                                  const int* __restrict__ far) {
  if (*far) return;
  __shared__ uint32_t wc[kLWarps][32];
  __shared__ uint32_t bb[kDirs];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int S = blockIdx.x; S < g.nunits; S += gridDim.x) {
    const int64_t p0 = cs_old[(int64_t)S * kUnitKeys], p1 = cs_old[(int64_t)(S + 1) * kUnitKeys];
    int sx, sy, sz;
    unit_coords(g, (uint32_t)S, sx, sy, sz);
    // each warp's start inside each bucket: the counts of the earlier warps
    if (lane < kDirs) {
      uint32_t acc = 0;
      for (int ww = 0; ww < w; ++ww) acc += cntw[((int64_t)S * kLWarps + ww) * kCodes + lane];
      wc[w][lane] = acc;
    }
    if (threadIdx.x < kDirs) {
      const int k = threadIdx.x;
      const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
      const uint32_t D =
          unit_index(g, wrap_add(sx, dx, g.nu[0]), wrap_add(sy, dy, g.nu[1]), wrap_add(sz, dz, g.nu[2]));
      bb[k] = base[D] + rel[(int64_t)S * kDirs + k];
    }
    int64_t s0, s1;
    warp_segment(p0, p1, w, kLWarps, s0, s1);
    __syncthreads();
    for (int64_t b = s0; b < s1; b += 32 * kBatch) {
      int32_t c[kBatch];
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const int64_t p = b + 32 * r + lane;
        c[r] = p < s1 ? __ldcs(cell + p) : -1;
      }
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const bool valid = c[r] >= 0;
        const int code = valid ? code_of(g, sx, sy, sz, c[r]) : 31;
        const unsigned peers = __match_any_sync(0xffffffffu, code);
        uint32_t before = 0;
        if (valid) before = wc[w][code];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wc[w][code] = before + (uint32_t)__popc(peers);
        __syncwarp();
        if (valid) {
          const uint32_t pos = bb[code] + before + (uint32_t)__popc(peers & lt);
          lidx[pos] = (uint32_t)(b + 32 * r + lane);
          lkey[pos] = (uint16_t)(chunk_key(cell_i(c[r]), cell_j(c[r]), cell_k(c[r]), g.B, g.logB, g.ncx, g.ncy) &
                                 (kUnitKeys - 1));
        }
      }
    }
    __syncthreads();
  }
}

// 5. per destination unit: stable counting sort of its incoming list by the key inside the unit:
// perm[b0 + r] = storage index of the r-th particle of the unit's sorted range, and the unit's cell
// starts
__global__ void __launch_bounds__(kRThreads) usort_rank_kernel(UnitGeo g, const uint32_t* __restrict__ base,
                                                               const uint32_t* __restrict__ lidx,
                                                               const uint16_t* __restrict__ lkey,
                                                               uint32_t* __restrict__ perm,
                                                               uint32_t* __restrict__ cell_start, int64_t n,
                                                               const int* __restrict__ far) {
  if (*far) return;
  __shared__ uint32_t wk[kRWarps][kUnitKeys];
  __shared__ uint32_t wsum[kRWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  if (blockIdx.x == 0 && threadIdx.x == 0) cell_start[(int64_t)g.nunits * kUnitKeys] = (uint32_t)n;
  for (int D = blockIdx.x; D < g.nunits; D += gridDim.x) {
    for (int k = lane; k < kUnitKeys; k += 32) wk[w][k] = 0;
    const int64_t b0 = base[D], b1 = base[D + 1];
    int64_t s0, s1;
    warp_segment(b0, b1, w, kRWarps, s0, s1);
    __syncwarp();
    for (int64_t b = s0; b < s1; b += 32 * kBatch) {
      uint32_t key[kBatch];
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const int64_t i = b + 32 * r + lane;
        key[r] = i < s1 ? (uint32_t)lkey[i] : 0xffffu;
      }
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const unsigned peers = __match_any_sync(0xffffffffu, key[r]);
        if (key[r] != 0xffffu && lane == __ffs(peers) - 1) wk[w][key[r]] += (uint32_t)__popc(peers);
        __syncwarp();
      }
    }
    __syncthreads();
    // one key per thread: its total over the warps, the exclusive scan over the 512 keys, then each
    // warp's start per key (key start + the counts of the earlier warps)
    const int k = threadIdx.x;
    uint32_t tot = 0;
    for (int ww = 0; ww < kRWarps; ++ww) tot += wk[ww][k];
    uint32_t inc = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t wbase = 0;
    for (int ww = 0; ww < w; ++ww) wbase += wsum[ww];
    const uint32_t st = wbase + inc - tot;
    cell_start[(int64_t)D * kUnitKeys + k] = (uint32_t)b0 + st;
    {
      uint32_t a = st;
      for (int ww = 0; ww < kRWarps; ++ww) {
        const uint32_t c = wk[ww][k];
        wk[ww][k] = a;
        a += c;
      }
    }
    __syncthreads();
    for (int64_t b = s0; b < s1; b += 32 * kBatch) {
      uint32_t key[kBatch], idx[kBatch];
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const int64_t i = b + 32 * r + lane;
        key[r] = i < s1 ? (uint32_t)lkey[i] : 0xffffu;
        idx[r] = i < s1 ? lidx[i] : 0u;
      }
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const bool valid = key[r] != 0xffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, key[r]);
        uint32_t before = 0;
        if (valid) before = wk[w][key[r]];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wk[w][key[r]] = before + (uint32_t)__popc(peers);
        __syncwarp();
        if (valid) perm[b0 + before + __popc(peers & lt)] = idx[r];
      }
    }
    __syncthreads();  // wk is reset for the next unit
  }
}

}  // namespace

bool local_sort_supported(const st_ctx* h) {
  if (h->prec == ST_FP64 || !h->sorted || h->np <= 0 || h->np >= (int64_t(1) << 32)) return false;
  if (h->geo.B < kUE) return false;
  for (int q = 0; q < 3; ++q)
    if (h->geo.n[q] % h->geo.B != 0) return false;
  return true;
}

size_t local_sort_aux_bytes(const st_ctx* h) {
  const size_t nunits = h->nkeys / kUnitKeys;
  return (nunits * (kCodes * (kLWarps + 1) + kDirs + 2) + 2) * sizeof(uint32_t);
}

cudaError_t launch_local_sort(st_ctx* h, int* far, uint32_t* lidx, uint16_t* lkey, uint32_t* perm, void* aux) {
  UnitGeo g;
  for (int q = 0; q < 3; ++q) g.nu[q] = h->geo.n[q] / kUE;
  g.B = h->geo.B;
  g.logB = 0;
  while ((1 << g.logB) < g.B) ++g.logB;
  g.ncx = h->geo.n[0] / g.B;
  g.ncy = h->geo.n[1] / g.B;
  g.nunits = (int)(h->nkeys / kUnitKeys);
  uint32_t* cnt = (uint32_t*)aux;
  uint32_t* cntw = cnt + (size_t)g.nunits * kCodes;
  uint32_t* rel = cntw + (size_t)g.nunits * kLWarps * kCodes;
  uint32_t* total = rel + (size_t)g.nunits * kDirs;
  uint32_t* base = total + g.nunits;
  const uint32_t* cs_old = (const uint32_t*)h->cell_start.p;
  const MixedState cur = carve_mixed(h->state.p, h->cap, h->prec == ST_MIXED_BF16V);
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemsetAsync(far, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int ublocks = std::min(g.nunits, 152 * 8);
  usort_count_kernel<<<ublocks, kLThreads, 0, s>>>(cur.cell, cs_old, g, cnt, cntw, far);
  usort_dest_kernel<<<(g.nunits + 127) / 128, 128, 0, s>>>(g, cnt, rel, total);
  usort_scan_kernel<<<1, 1024, 0, s>>>(total, g.nunits, base);
  usort_scatter_kernel<<<ublocks, kLThreads, 0, s>>>(cur.cell, cs_old, g, cntw, rel, base, lidx, lkey, far);
  // rank: as many blocks as are resident at once (its registers allow three of 512 threads per SM),
  // each taking every grid-th unit, so that no block waits for a second wave
  int sms = 152, per_sm = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, usort_rank_kernel, kRThreads, 0);
  const int rblocks = std::min(g.nunits, sms * std::max(per_sm, 1));
  usort_rank_kernel<<<rblocks, kRThreads, 0, s>>>(g, base, lidx, lkey, perm, (uint32_t*)h->cell_start.p, h->np,
                                                  far);
  h->launches += 5;
  return cudaGetLastError();
}

}  // namespace st
