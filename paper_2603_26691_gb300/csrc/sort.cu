// Stable counting sort of the particles by their chunk-major cell key.
//
// LSD radix sort of (key, slot) pairs with 8-bit digits.  One read of the keys counts every
// pass's digit totals; then each pass is a single sweep: a block takes the next tile of 4096
// keys in order, ranks them stably inside the tile (lanes of equal digit found with one
// __match_any_sync per 32 keys, prefix counts combined across warps in warp order), publishes its
// per-digit counts, places the tile in digit order in shared memory, adds the counts of all
// earlier tiles by looking back over their published words (decoupled look-back, a few tiles'
// words per round trip; each word holds a count and says whether it is the tile's own count or
// its inclusive prefix), and writes the tile out digit-run by digit-run so that the global
// writes coalesce.
// The first pass computes the keys from the particle state on the fly and uses the storage
// slot as the value.  The structure-of-arrays payload is then gathered once through the final
// permutation.  Equal keys keep their storage order, so the permutation is unique.
//
// Waits on other blocks are bounded: a look-back that gives up sets a device flag (reported as
// ST_ERR_TIMEOUT) and carries on, so no block can hang the grid.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <type_traits>
#include <vector>

#include "st_common.cuh"
#include "st_ptx.cuh"

namespace st {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kSortThreads * kItems;  // 4096 keys per tile
constexpr int kRadix = 256;
constexpr int kMaxPasses = 4;
constexpr uint32_t kLookSpinLimit = 1u << 22;
constexpr uint64_t kLookWaitNs = 1000000000ull;  // 1 s
constexpr int kLookWindow = 4;  // look-back words read per round trip
constexpr int kAttrDevices = 64;  // devices whose kernel attributes are tracked

// look-back word: epoch (30 bits) | kind (2 bits: 1 = the tile's own count, 2 = inclusive
// prefix) | count (32 bits).  A word whose epoch is not the pass's is empty.
constexpr unsigned long long kLookAgg = 1ull, kLookPrefix = 2ull;

struct KeyGeo {
  int n[3];
  double inv_h[3];
  int B, logB, ncx, ncy;
};

// key sources for the first pass
struct CellKeys {  // mixed precision: the packed cell of each slot
  const int32_t* __restrict__ cell;
  KeyGeo g;
  __device__ __forceinline__ uint32_t of_cell(int32_t c) const {
    return chunk_key(cell_i(c), cell_j(c), cell_k(c), g.B, g.logB, g.ncx, g.ncy);
  }
  __device__ __forceinline__ uint32_t operator()(int64_t i) const { return of_cell(cell[i]); }
  // the same key with the Morton spread of the local coordinates read from a 32-entry table
  // (tab[v] = spread3(v)): three table reads instead of the shift-and-mask sequences
  __device__ __forceinline__ uint32_t of_cell_tab(int32_t c, const uint32_t* tab) const {
    const uint32_t i = (uint32_t)cell_i(c), j = (uint32_t)cell_j(c), k = (uint32_t)cell_k(c);
    const uint32_t m = (uint32_t)g.B - 1u;
    const uint32_t chunk = (i >> g.logB) + (uint32_t)g.ncx * ((j >> g.logB) + (uint32_t)g.ncy * (k >> g.logB));
    const uint32_t morton = tab[(i & m) & 31u] | (tab[(j & m) & 31u] << 1) | (tab[(k & m) & 31u] << 2);
    return (chunk << (3 * g.logB)) | morton;
  }
};
struct PositionKeys {  // FP64: the cell of each position
  F64State s;
  KeyGeo g;
  __device__ __forceinline__ uint32_t operator()(int64_t i) const {
    int c[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) c[q] = min(max((int)floor(s.x[q][i] * g.inv_h[q]), 0), g.n[q] - 1);
    return chunk_key(c[0], c[1], c[2], g.B, g.logB, g.ncx, g.ncy);
  }
};
struct ArrayKeys {  // keys given by the caller
  const uint32_t* __restrict__ k;
  __device__ __forceinline__ uint32_t operator()(int64_t i) const { return k[i]; }
};

// the digit of pass p: bits [8p, 8p + 8) of the key, cut at key_bits (keys are compared on their
// low key_bits bits only)
__host__ __device__ __forceinline__ uint32_t digit_mask(int key_bits, int p) {
  const int b = key_bits - 8 * p;
  return b >= 8 ? 0xffu : (b <= 0 ? 0u : (1u << b) - 1u);
}

__device__ __forceinline__ uint64_t sort_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void store_look(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long load_look(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// A kernel given a gate runs only if *gate != 0: the general sort is queued behind the
// neighbourhood sort (sort_local.cu) and runs only when that one found a particle it cannot place.
__device__ __forceinline__ bool gated_off(const int* gate) { return gate != nullptr && *gate == 0; }

// every pass's digit totals in one read of the keys: each lane counts runs of equal digits over
// 16 consecutive keys and adds each run once to the block's counts
template <class Src>
__global__ void __launch_bounds__(kSortThreads) digit_totals_kernel(Src src, int64_t n, int key_bits,
                                                                     uint32_t* __restrict__ totals,
                                                                     const int* __restrict__ gate) {
  if (gated_off(gate)) return;
  const int passes = (key_bits + 7) / 8;
  __shared__ uint32_t cnt[kMaxPasses][kRadix];
  __shared__ uint32_t mtab[32];  // Morton spread table for keys from cells
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&cnt[0][0])[i] = 0;
  if (threadIdx.x < 32) mtab[threadIdx.x] = spread3(threadIdx.x);
  __syncthreads();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * kItems; base < n;
       base += nthreads * kItems) {
    uint32_t k[kItems];
    const int m = (int)min((int64_t)kItems, n - base);
    if constexpr (std::is_same<Src, CellKeys>::value || std::is_same<Src, ArrayKeys>::value) {
      // a thread's 16 consecutive words as four 16-byte loads (the arrays are 256-byte aligned)
      const uint32_t* w;
      if constexpr (std::is_same<Src, CellKeys>::value)
        w = reinterpret_cast<const uint32_t*>(src.cell);
      else
        w = src.k;
      if (m == kItems) {
#pragma unroll
        for (int r = 0; r < kItems; r += 4) {
          const uint4 q = __ldg(reinterpret_cast<const uint4*>(w + base + r));
          const uint32_t v4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if constexpr (std::is_same<Src, CellKeys>::value)
              k[r + e] = src.of_cell_tab((int32_t)v4[e], mtab);
            else
              k[r + e] = v4[e];
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < kItems; ++r) k[r] = r < m ? src(base + r) : 0u;
      }
    } else {
#pragma unroll
      for (int r = 0; r < kItems; ++r) k[r] = r < m ? src(base + r) : 0u;
    }
    for (int p = 0; p < passes; ++p) {
      const int sh = 8 * p;
      const uint32_t dm = digit_mask(key_bits, p);
      uint32_t cur = (k[0] >> sh) & dm, run = 1;
#pragma unroll
      for (int r = 1; r < kItems; ++r) {
        if (r >= m) break;
        const uint32_t d = (k[r] >> sh) & dm;
        if (d == cur) {
          ++run;
        } else {
          atomicAdd(&cnt[p][cur], run);
          cur = d;
          run = 1;
        }
      }
      atomicAdd(&cnt[p][cur], run);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t c = (&cnt[0][0])[i];
    if (c) atomicAdd(&totals[i], c);
  }
}

// exclusive scan of each pass's 256 digit totals (one block of 256 threads)
__global__ void digit_offsets_kernel(const uint32_t* __restrict__ totals, int passes, uint32_t* __restrict__ offs,
                                     const int* __restrict__ gate) {
  if (gated_off(gate)) return;
  __shared__ uint32_t s[kRadix];
  for (int p = 0; p < passes; ++p) {
    s[threadIdx.x] = totals[p * kRadix + threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      for (int d = 0; d < kRadix; ++d) {
        const uint32_t c = s[d];
        s[d] = acc;
        acc += c;
      }
    }
    __syncthreads();
    offs[p * kRadix + threadIdx.x] = s[threadIdx.x];
    __syncthreads();
  }
}

// shared memory of a pass: two staging buffers (each a key-or-cell array and a value array of a
// tile: the next tile lands in one while the current tile is ranked and written out through the
// other), per-warp digit counts, digit starts, two mbarriers, the tile numbers and the Morton
// spread table of the first pass
constexpr int kBufWords = 2 * kTile;
constexpr int kPassBlocksPerSM = 3;  // 3 x 75.8 KB of shared memory, 80 registers
constexpr size_t kPassSmem = 2 * kBufWords * 4 + kSortWarps * kRadix * 4 + 2 * kRadix * 4 + 2 * 8 + 2 * 8 + 32 * 4;

// one stable counting-sort pass over digit `shift / 8` (8 bits, fewer in the last pass: dmask), tiles
// taken in order.  BULK: the tile's input (the cell array in the first pass, else the keys and values)
// arrives by 1-D bulk copies issued one tile ahead; otherwise it is read with plain loads.
template <bool FIRST, bool BULK, class Src>
__global__ void __launch_bounds__(kSortThreads, kPassBlocksPerSM) onesweep_kernel(Src src, const uint32_t* __restrict__ kin,
                                                                 const uint32_t* __restrict__ vin,
                                                                 uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                                 int64_t n, int shift, uint32_t dmask, int64_t ntiles,
                                                                 const uint32_t* __restrict__ digit_offset,
                                                                 unsigned long long* __restrict__ look,
                                                                 unsigned long long epoch, unsigned* __restrict__ tile_ctr,
                                                                 int* __restrict__ err, const int* __restrict__ gate) {
  if (gated_off(gate)) return;
  extern __shared__ __align__(128) unsigned char sm[];
  uint32_t* bufs = reinterpret_cast<uint32_t*>(sm);                                   // [2][2][kTile]
  uint32_t (*wcnt)[kRadix] = reinterpret_cast<uint32_t (*)[kRadix]>(sm + 2 * kBufWords * 4);
  uint32_t* lstart = reinterpret_cast<uint32_t*>(sm + 2 * kBufWords * 4 + kSortWarps * kRadix * 4);
  uint32_t* gbase = lstart + kRadix;
  uint64_t* bar = reinterpret_cast<uint64_t*>(gbase + kRadix);
  int64_t* s_next = reinterpret_cast<int64_t*>(bar + 2);
  uint32_t* mtab = reinterpret_cast<uint32_t*>(s_next + 2);  // Morton spread table (first pass)
  if (FIRST && threadIdx.x < 32) mtab[threadIdx.x] = spread3(threadIdx.x);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned long long ep = epoch << 34;
  // bulk copy of tile t's input into buffer b (sizes rounded up to 4 words: the arrays' capacity
  // is a multiple of 64 slots, so the copy stays inside them)
  auto issue = [&](int64_t t, int b) {
    const int64_t cnt = min((int64_t)kTile, n - t * kTile);
    const uint32_t bytes = (uint32_t)(((cnt + 3) & ~int64_t(3)) * 4);
    uint32_t* dst = bufs + b * kBufWords;
    ptx::mbar_expect_tx(&bar[b], FIRST ? bytes : 2 * bytes);
    if constexpr (FIRST && BULK) {
      ptx::bulk_load(dst, reinterpret_cast<const uint32_t*>(src.cell) + t * kTile, bytes, &bar[b]);
    } else {
      ptx::bulk_load(dst, kin + t * kTile, bytes, &bar[b]);
      ptx::bulk_load(dst + kTile, vin + t * kTile, bytes, &bar[b]);
    }
  };
  if (threadIdx.x == 0) {
    if (BULK) {
      ptx::mbar_init(&bar[0], 1);
      ptx::mbar_init(&bar[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int64_t t = (int64_t)atomicAdd(tile_ctr, 1u);
    *s_next = t;
    if constexpr (BULK) {
      if (t < ntiles) issue(t, 0);
    }
  }
  __syncthreads();
  for (int it = 0;; ++it) {
    const int b = it & 1;
    uint32_t* kbuf = bufs + b * kBufWords;
    uint32_t* vbuf = kbuf + kTile;
    const int64_t tile = *s_next;
    for (int ww = 0; ww < kSortWarps; ++ww) wcnt[ww][threadIdx.x] = 0;
    __syncthreads();  // everyone has read the tile number
    if (tile >= ntiles) return;
    if (threadIdx.x == 0) {
      // take the next tile now and start its copy into the other buffer
      const int64_t t2 = (int64_t)atomicAdd(tile_ctr, 1u);
      *s_next = t2;
      if constexpr (BULK) {
        if (t2 < ntiles) issue(t2, b ^ 1);
      }
    }
    if (BULK && !ptx::mbar_wait(&bar[b], (it >> 1) & 1)) atomicOr(err, 128);
    // ---- load: warp w owns keys [w*512, (w+1)*512) of the tile in 16 rounds ----
    uint32_t key[kItems], val[kItems], rank[kItems];
    const int64_t start = tile * kTile + (int64_t)w * (kItems * 32);
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int64_t i = start + r * 32 + lane;
      const int li = w * (kItems * 32) + r * 32 + lane;
      if constexpr (BULK && FIRST) {
        key[r] = i < n ? src.of_cell_tab((int32_t)kbuf[li], mtab) : 0u;
        val[r] = (uint32_t)i;
      } else if constexpr (BULK) {
        key[r] = kbuf[li];
        val[r] = vbuf[li];
      } else if constexpr (FIRST) {
        key[r] = i < n ? src(i) : 0u;
        val[r] = (uint32_t)i;
      } else {
        key[r] = i < n ? kin[i] : 0u;
        val[r] = i < n ? vin[i] : 0u;
      }
    }
    __syncthreads();  // the staged input is in registers: the buffer takes the output next
    // ---- stable ranks inside the warp (one vote when all valid lanes hold the same digit) ----
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const bool valid = start + r * 32 + lane < n;
      const uint32_t dig = (key[r] >> shift) & dmask;
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      const uint32_t d0 = __shfl_sync(0xffffffffu, dig, vm ? __ffs(vm) - 1 : 0);
      // lanes holding the same digit (invalid lanes match only each other)
      unsigned peers;
      if (__all_sync(0xffffffffu, !valid || dig == d0))
        peers = valid ? vm : ~vm;
      else
        peers = __match_any_sync(0xffffffffu, valid ? dig : 0x100u);
      uint32_t before = 0;
      if (valid) before = wcnt[w][dig];
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) wcnt[w][dig] = before + __popc(peers);
      __syncwarp();
      rank[r] = valid ? before + __popc(peers & lt) : 0xffffffffu;
    }
    __syncthreads();
    // ---- per digit: offsets of the warps inside the tile, the tile's count (published) ----
    const int d = threadIdx.x;
    uint32_t tot = 0;
    for (int ww = 0; ww < kSortWarps; ++ww) {
      const uint32_t c = wcnt[ww][d];
      wcnt[ww][d] = tot;
      tot += c;
    }
    unsigned long long* my = look + tile * kRadix + d;
    store_look(my, ep | ((tile == 0 ? kLookPrefix : kLookAgg) << 32) | tot);
    // ---- tile-local start of each digit (exclusive scan of the tile's counts) ----
    lstart[d] = tot;
    __syncthreads();
    if (w == 0) {
      uint32_t c[8], s = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        c[k] = lstart[lane * 8 + k];
        s += c[k];
      }
      uint32_t x = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      uint32_t acc = x - s;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        lstart[lane * 8 + k] = acc;
        acc += c[k];
      }
    }
    __syncthreads();
    // ---- the tile in digit order in shared memory (needs only the tile's own counts) ----
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      if (rank[r] != 0xffffffffu) {
        const uint32_t dig = (key[r] >> shift) & dmask;
        const uint32_t lp = lstart[dig] + wcnt[w][dig] + rank[r];
        kbuf[lp] = key[r];
        vbuf[lp] = val[r];
      }
    }
    // ---- look back: the sum of this digit's counts over all earlier tiles.  The words of the
    // kLookWindow tiles before the first unread one are loaded together (one round trip) and
    // summed in order until a tile's inclusive prefix; a word not yet published ends the round
    // and the next round starts at it.
    uint32_t excl = 0;
    if (tile > 0) {
      int64_t t = tile - 1;
      uint64_t t0 = 0;
      uint32_t polls = 0;
      for (;;) {
        unsigned long long v[kLookWindow];
#pragma unroll
        for (int k = 0; k < kLookWindow; ++k) v[k] = t - k >= 0 ? load_look(look + (t - k) * kRadix + d) : 0ull;
        int k = 0;
        bool done = false;
#pragma unroll
        for (int q = 0; q < kLookWindow; ++q) {
          if (k == q && !done && t - q >= 0) {
            const unsigned long long kind = (v[q] >> 32) & 3ull;
            if ((v[q] >> 34) == epoch && kind != 0) {
              excl += (uint32_t)v[q];
              ++k;
              done = kind == kLookPrefix || t - q == 0;
            }
          }
        }
        if (done) break;
        if (k > 0) {
          t -= k;
          polls = 0;
          continue;
        }
        if (polls == 0) t0 = sort_ns();
        if (++polls >= kLookSpinLimit || ((polls & 31u) == 0 && sort_ns() - t0 > kLookWaitNs)) {
          atomicOr(err, 64);  // gave up: the output is wrong, the host reports a timeout
          break;
        }
      }
      store_look(my, ep | (kLookPrefix << 32) | (excl + tot));
    }
    gbase[d] = digit_offset[d] + excl;
    __syncthreads();
    const int cnt = (int)min((int64_t)kTile, n - tile * kTile);
    for (int lp = threadIdx.x; lp < cnt; lp += kSortThreads) {
      const uint32_t k = kbuf[lp];
      const uint32_t dig = (k >> shift) & dmask;
      const uint32_t dst = gbase[dig] + (uint32_t)lp - lstart[dig];
      kout[dst] = k;
      vout[dst] = vbuf[lp];
    }
    // this buffer receives the tile after next by bulk copy: order the generic-proxy accesses of
    // every thread before that async-proxy write
    if constexpr (BULK) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
}

// payload gather through the final permutation
__global__ void gather_f64_kernel(F64State src, F64State dst, const uint32_t* __restrict__ sid,
                                  uint32_t* __restrict__ did, const uint32_t* __restrict__ perm, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t p = perm[i];
    for (int q = 0; q < 3; ++q) {
      dst.x[q][i] = src.x[q][p];
      dst.v[q][i] = src.v[q][p];
    }
    dst.d[i] = src.d[p];
    did[i] = sid[p];
  }
}

// The payload gather from 32-byte particle records {cell, offsets | velocity, diameter} (written
// by the step before the sort): one 256-bit load, one sector, per particle instead of one sector per
// array.  BF16 handles' velocities are BF16-exact in the records.
template <bool BF16>
__device__ __forceinline__ void store_v4(void* v, int64_t o, float a, float b, float c, float d) {
  if (BF16) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 r;
    r.x = *reinterpret_cast<unsigned*>(&lo);
    r.y = *reinterpret_cast<unsigned*>(&hi);
    __stcs(reinterpret_cast<uint2*>((__nv_bfloat16*)v + o), r);
  } else {
    __stcs(reinterpret_cast<float4*>((float*)v + o), make_float4(a, b, c, d));
  }
}
template <bool BF16>
__device__ __forceinline__ void store_v1(void* v, int64_t i, float a) {
  if (BF16)
    ((__nv_bfloat16*)v)[i] = __float2bfloat16_rn(a);
  else
    ((float*)v)[i] = a;
}

template <bool BF16>
__global__ void gather_records_kernel(const float4* __restrict__ rec, MixedState dst, const uint32_t* __restrict__ sid,
                                      uint32_t* __restrict__ did, const uint32_t* __restrict__ perm, int64_t n,
                                      const int* __restrict__ gate) {
  if (gated_off(gate)) return;
  const int64_t n4 = n >> 2;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n4; g += (int64_t)gridDim.x * blockDim.x) {
    const uint4 pp = __ldg(reinterpret_cast<const uint4*>(perm) + g);
    const uint32_t p[4] = {pp.x, pp.y, pp.z, pp.w};
    ptx::Rec32 r[4];
    uint32_t id[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      r[k] = ptx::ld_rec32(rec + 2 * (int64_t)p[k]);
      id[k] = __ldg(sid + p[k]);
    }
    const int64_t o = g << 2;
    __stcs(reinterpret_cast<int4*>(dst.cell + o), make_int4(__float_as_int(r[0].c), __float_as_int(r[1].c),
                                                             __float_as_int(r[2].c), __float_as_int(r[3].c)));
    __stcs(reinterpret_cast<float4*>(dst.xi[0] + o), make_float4(r[0].x0, r[1].x0, r[2].x0, r[3].x0));
    __stcs(reinterpret_cast<float4*>(dst.xi[1] + o), make_float4(r[0].x1, r[1].x1, r[2].x1, r[3].x1));
    __stcs(reinterpret_cast<float4*>(dst.xi[2] + o), make_float4(r[0].x2, r[1].x2, r[2].x2, r[3].x2));
    store_v4<BF16>(dst.v[0], o, r[0].v0, r[1].v0, r[2].v0, r[3].v0);
    store_v4<BF16>(dst.v[1], o, r[0].v1, r[1].v1, r[2].v1, r[3].v1);
    store_v4<BF16>(dst.v[2], o, r[0].v2, r[1].v2, r[2].v2, r[3].v2);
    __stcs(reinterpret_cast<float4*>(dst.d + o), make_float4(r[0].d, r[1].d, r[2].d, r[3].d));
    __stcs(reinterpret_cast<uint4*>(did + o), make_uint4(id[0], id[1], id[2], id[3]));
  }
  // ragged tail
  for (int64_t i = (n4 << 2) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pi = perm[i];
    const ptx::Rec32 r = ptx::ld_rec32(rec + 2 * pi);
    dst.cell[i] = __float_as_int(r.c);
    dst.xi[0][i] = r.x0;
    dst.xi[1][i] = r.x1;
    dst.xi[2][i] = r.x2;
    store_v1<BF16>(dst.v[0], i, r.v0);
    store_v1<BF16>(dst.v[1], i, r.v1);
    store_v1<BF16>(dst.v[2], i, r.v2);
    dst.d[i] = r.d;
    did[i] = sid[pi];
  }
}

// Records back to the structure of arrays in place of a sort (the cells are already there).
template <bool BF16>
__global__ void records_to_soa_kernel(const float4* __restrict__ rec, MixedState dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = rec[2 * i], b = rec[2 * i + 1];
    dst.xi[0][i] = a.y;
    dst.xi[1][i] = a.z;
    dst.xi[2][i] = a.w;
    store_v1<BF16>(dst.v[0], i, b.x);
    store_v1<BF16>(dst.v[1], i, b.y);
    store_v1<BF16>(dst.v[2], i, b.z);
    dst.d[i] = b.w;
  }
}

// mixed-precision payload gather, 4 consecutive outputs per thread: one 16-byte load of the
// permutation, then every gathered load of the 4 particles in flight at once, then 128-bit
// (64-bit for BF16 velocities) coalesced stores
template <bool BF16>
__global__ void gather_mixed_kernel(MixedState src, MixedState dst, const uint32_t* __restrict__ sid,
                                    uint32_t* __restrict__ did, const uint32_t* __restrict__ perm, int64_t n,
                                    const int* __restrict__ gate) {
  if (gated_off(gate)) return;
  const int64_t n4 = n >> 2;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n4; g += (int64_t)gridDim.x * blockDim.x) {
    const uint4 pp = __ldg(reinterpret_cast<const uint4*>(perm) + g);
    const uint32_t p[4] = {pp.x, pp.y, pp.z, pp.w};
    int c[4];
    float x[3][4], v[3][4], d[4];
    uint32_t id[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      c[k] = __ldg(src.cell + p[k]);
      d[k] = __ldg(src.d + p[k]);
      id[k] = __ldg(sid + p[k]);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        x[q][k] = __ldg(src.xi[q] + p[k]);
        v[q][k] = BF16 ? __bfloat162float(__ldg((const __nv_bfloat16*)src.v[q] + p[k]))
                       : __ldg((const float*)src.v[q] + p[k]);
      }
    }
    const int64_t o = g << 2;
    __stcs(reinterpret_cast<int4*>(dst.cell + o), make_int4(c[0], c[1], c[2], c[3]));
    __stcs(reinterpret_cast<float4*>(dst.d + o), make_float4(d[0], d[1], d[2], d[3]));
    __stcs(reinterpret_cast<uint4*>(did + o), make_uint4(id[0], id[1], id[2], id[3]));
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      __stcs(reinterpret_cast<float4*>(dst.xi[q] + o), make_float4(x[q][0], x[q][1], x[q][2], x[q][3]));
      if (BF16) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[q][0], v[q][1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(v[q][2], v[q][3]);
        uint2 r;
        r.x = *reinterpret_cast<unsigned*>(&lo);
        r.y = *reinterpret_cast<unsigned*>(&hi);
        __stcs(reinterpret_cast<uint2*>((__nv_bfloat16*)dst.v[q] + o), r);
      } else {
        __stcs(reinterpret_cast<float4*>((float*)dst.v[q] + o), make_float4(v[q][0], v[q][1], v[q][2], v[q][3]));
      }
    }
  }
  // ragged tail
  for (int64_t i = (n4 << 2) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t pi = perm[i];
    dst.cell[i] = src.cell[pi];
    dst.d[i] = src.d[pi];
    did[i] = sid[pi];
    for (int q = 0; q < 3; ++q) {
      dst.xi[q][i] = src.xi[q][pi];
      if (BF16)
        ((__nv_bfloat16*)dst.v[q])[i] = ((const __nv_bfloat16*)src.v[q])[pi];
      else
        ((float*)dst.v[q])[i] = ((const float*)src.v[q])[pi];
    }
  }
}

// start[k] = first sorted position with key >= k, for k in [0, nkeys]: position i writes the keys
// in (key[i-1], key[i]] (one pass over the sorted keys; the keys after the last one are filled by
// cell_start_tail_kernel)
// start[k] = the first sorted position whose key is >= k, for every k up to the last key: each
// thread takes four consecutive sorted keys (one 16-byte load; the key arrays are 256-byte
// aligned) and the key before them
__global__ void cell_start_kernel(const uint32_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ start,
                                  const int* __restrict__ gate) {
  if (gated_off(gate)) return;
  const int64_t groups = (n + 3) >> 2;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = g << 2;
    uint32_t k4[4];
    if (i0 + 4 <= n) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(keys) + g);
      k4[0] = q.x;
      k4[1] = q.y;
      k4[2] = q.z;
      k4[3] = q.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) k4[e] = i0 + e < n ? keys[i0 + e] : 0u;
    }
    int64_t prev = i0 > 0 ? (int64_t)__ldg(keys + i0 - 1) : -1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (i0 + e < n) {
        const int64_t k1 = k4[e];
        for (int64_t k = prev + 1; k <= k1; ++k) start[k] = (uint32_t)(i0 + e);
        prev = k1;
      }
    }
  }
}

__global__ void cell_start_tail_kernel(const uint32_t* __restrict__ keys, int64_t n, uint32_t nkeys,
                                       uint32_t* __restrict__ start, const int* __restrict__ gate) {
  if (gated_off(gate)) return;
  const int64_t first = (int64_t)keys[n - 1] + 1;
  for (int64_t k = first + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= (int64_t)nkeys;
       k += (int64_t)gridDim.x * blockDim.x)
    start[k] = (uint32_t)n;
}

__global__ void cell_counts_kernel(const uint32_t* __restrict__ start, KeyGeo g, int64_t* __restrict__ counts) {
  int64_t ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(c % g.n[0]);
    int j = (int)((c / g.n[0]) % g.n[1]);
    int k = (int)(c / ((int64_t)g.n[0] * g.n[1]));
    uint32_t key = chunk_key(i, j, k, g.B, g.logB, g.ncx, g.ncy);
    counts[c] = (int64_t)start[key + 1] - (int64_t)start[key];
  }
}

// Bounding box of every chunk's particles (the particles of the chunk's key range in the sorted
// storage), each current position unwrapped to the periodic image nearest the chunk's centre:
// out[c][6] = {min x, y, z, max x, y, z}; +inf / -inf for an empty chunk.  One block per chunk at a
// time.  The extreme particles are found with exact integer keys - per axis the cell's offset from
// the chunk (moved by one box length when the cell is more than half a box from the chunk's
// centre) in the high half and the bits of the non-negative in-cell offset (mixed) in the low
// half, or the unwrapped FP64 position ordered as an integer (FP64 state) - and for the mixed
// state only the winners' positions are unwrapped in FP64, with the oracle's formula: min and max
// do not depend on the order of the reduction, and the FP64 work is per chunk, not per particle.
__device__ __forceinline__ long long ordered_bits(double x) {  // integer order = double order
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (long long)(0x8000000000000000ull - (unsigned long long)b);
}
__device__ __forceinline__ double from_ordered_bits(long long k) {
  return __longlong_as_double(k >= 0 ? k : (long long)(0x8000000000000000ull - (unsigned long long)k));
}

template <bool MIXED>
__global__ void __launch_bounds__(256) chunk_bounds_kernel(MixedState ms, F64State fs,
                                                          const uint32_t* __restrict__ start, KeyGeo g, double L0,
                                                          double L1, double L2, double h0, double h1, double h2,
                                                          int64_t nchunk, double* __restrict__ out) {
  __shared__ long long red[6][8];
  const double L[3] = {L0, L1, L2}, h[3] = {h0, h1, h2};
  const int64_t per = (int64_t)1 << (3 * g.logB);
  const long long kMax = 0x7fffffffffffffffll, kMin = -kMax - 1;
  for (int64_t c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const int cc[3] = {(int)(c % g.ncx), (int)((c / g.ncx) % g.ncy), (int)(c / ((int64_t)g.ncx * g.ncy))};
    long long lo[3] = {kMax, kMax, kMax}, hi[3] = {kMin, kMin, kMin};
    const int64_t S = start[c * per], E = start[(c + 1) * per];
    for (int64_t p = S + threadIdx.x; p < E; p += blockDim.x) {
      int idx[3];
      if (MIXED) {
        const int32_t cl = ms.cell[p];
        idx[0] = cell_i(cl);
        idx[1] = cell_j(cl);
        idx[2] = cell_k(cl);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        long long key;
        if (MIXED) {
          // offset of the cell from the chunk's first cell, moved to the image nearest the centre
          int r = idx[q] - cc[q] * g.B;
          if (2 * r - g.B >= g.n[q]) r -= g.n[q];
          else if (2 * r - g.B < -g.n[q]) r += g.n[q];
          key = ((long long)(r + (1 << 20)) << 32) | (long long)__float_as_uint(ms.xi[q][p]);
        } else {
          // FP64 positions: the unwrapped position itself, with the oracle's arithmetic
          const double cen = __dmul_rn((double)cc[q] * g.B + 0.5 * g.B, h[q]);
          double dx = __dsub_rn(fs.x[q][p], cen);
          dx = __dsub_rn(dx, __dmul_rn(L[q], floor(__dadd_rn(__ddiv_rn(dx, L[q]), 0.5))));
          key = ordered_bits(__dadd_rn(cen, dx));
        }
        lo[q] = min(lo[q], key);
        hi[q] = max(hi[q], key);
      }
    }
    long long v[6] = {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]};
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const long long t = __shfl_down_sync(0xffffffffu, v[k], o);
        v[k] = k < 3 ? min(v[k], t) : max(v[k], t);
      }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
      for (int k = 0; k < 6; ++k) red[k][w] = v[k];
    __syncthreads();
    if (threadIdx.x < 6) {
      const int k = threadIdx.x, q = k % 3;
      long long r = red[k][0];
      for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) r = k < 3 ? min(r, red[k][ww]) : max(r, red[k][ww]);
      double res;
      if (E <= S) {
        res = k < 3 ? INFINITY : -INFINITY;
      } else if (MIXED) {
        // the winner's position, unwrapped with the oracle's arithmetic
        int i = (int)((r >> 32) - (1 << 20)) + cc[q] * g.B;
        i = i < 0 ? i + g.n[q] : (i >= g.n[q] ? i - g.n[q] : i);
        const double x =
            __dmul_rn(__dadd_rn((double)i, (double)__uint_as_float((unsigned)(r & 0xffffffffll))), h[q]);
        const double centre = __dmul_rn((double)cc[q] * g.B + 0.5 * g.B, h[q]);
        double dx = __dsub_rn(x, centre);
        dx = __dsub_rn(dx, __dmul_rn(L[q], floor(__dadd_rn(__ddiv_rn(dx, L[q]), 0.5))));
        res = __dadd_rn(centre, dx);
      } else {
        res = from_ordered_bits(r);
      }
      out[6 * c + k] = res;
    }
    __syncthreads();
  }
}

KeyGeo key_geo(const st_ctx* h) {
  KeyGeo g;
  for (int q = 0; q < 3; ++q) {
    g.n[q] = h->geo.n[q];
    g.inv_h[q] = h->geo.inv_h[q];
  }
  g.B = h->geo.B;
  g.logB = 0;
  while ((1 << g.logB) < g.B) ++g.logB;
  g.ncx = (g.n[0] + g.B - 1) / g.B;
  g.ncy = (g.n[1] + g.B - 1) / g.B;
  return g;
}

int grid_for(int64_t n, int max_blocks = 152 * 16) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}


template <bool FIRST, bool BULK, class Src>
cudaError_t launch_pass(int64_t grid, cudaStream_t s, Src src, const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                        uint32_t* vout, int64_t n, int shift, uint32_t dmask, int64_t ntiles, const uint32_t* offs,
                        unsigned long long* look, uint32_t epoch, unsigned* tile_ctr, int* err, const int* gate) {
  // per instantiation and device (a kernel attribute is per device); atomic because the
  // allocation-free entry point may be called from several host threads at once (setting the
  // attribute twice is harmless)
  static std::atomic<bool> attr[kAttrDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kAttrDevices) return cudaErrorInvalidDevice;
  if (!attr[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(onesweep_kernel<FIRST, BULK, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPassSmem);
    if (e != cudaSuccess) return e;
    attr[dev].store(true, std::memory_order_release);
  }
  onesweep_kernel<FIRST, BULK, Src><<<(unsigned)grid, kSortThreads, kPassSmem, s>>>(
      src, kin, vin, kout, vout, n, shift, dmask, ntiles, offs, look, epoch, tile_ctr, err, gate);
  return cudaGetLastError();
}

// the passes of the stable sort of n keys of key_bits bits; the last pass writes kfinal / vfinal.
// Bulk copies read whole 16-byte groups, so they serve only arrays that are 16-byte aligned with
// capacity a multiple of 4 slots: the particle state's cell array (first pass, CellKeys) and,
// with bulk_rest, every intermediate key/value array.
template <class Src>
cudaError_t radix_passes(Src src, int64_t n, int key_bits, uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb,
                         uint32_t* kfinal, uint32_t* vfinal, uint32_t* totals, uint32_t* offs, unsigned* tile_ctr,
                         unsigned long long* look, uint32_t* epoch, int* err, int sms, cudaStream_t s,
                         int64_t* launches, bool bulk_rest, const int* gate = nullptr) {
  const int passes = (key_bits + 7) / 8;
  const int64_t ntiles = (n + kTile - 1) / kTile;
  cudaError_t e = cudaMemsetAsync(totals, 0, (size_t)kMaxPasses * kRadix * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tile_ctr, 0, kMaxPasses * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  digit_totals_kernel<Src><<<grid_for((n + kItems - 1) / kItems), kSortThreads, 0, s>>>(src, n, key_bits, totals,
                                                                                       gate);
  digit_offsets_kernel<<<1, kRadix, 0, s>>>(totals, passes, offs, gate);
  *launches += 2;
  int64_t grid = (int64_t)sms * kPassBlocksPerSM;
  if (grid > ntiles) grid = ntiles;
  const uint32_t* kin = nullptr;
  const uint32_t* vin = nullptr;
  for (int p = 0; p < passes; ++p) {
    // ping-pong so that the last pass lands in the final buffers
    const bool to_final = ((passes - 1 - p) % 2) == 0;
    uint32_t* kout = to_final ? kfinal : (kfinal == ka ? kb : ka);
    uint32_t* vout = to_final ? vfinal : (vfinal == va ? vb : va);
    *epoch = (*epoch + 1) & ((1u << 30) - 1);
    if (*epoch == 0) *epoch = 1;
    const uint32_t dm = digit_mask(key_bits, p);
    if (p == 0) {
      if constexpr (std::is_same<Src, CellKeys>::value)
        e = launch_pass<true, true, Src>(grid, s, src, nullptr, nullptr, kout, vout, n, 0, dm, ntiles, offs, look,
                                         *epoch, tile_ctr, err, gate);
      else
        e = launch_pass<true, false, Src>(grid, s, src, nullptr, nullptr, kout, vout, n, 0, dm, ntiles, offs, look,
                                          *epoch, tile_ctr, err, gate);
    } else if (bulk_rest) {
      e = launch_pass<false, true, ArrayKeys>(grid, s, ArrayKeys{nullptr}, kin, vin, kout, vout, n, 8 * p, dm, ntiles,
                                              offs + p * kRadix, look, *epoch, tile_ctr + p, err, gate);
    } else {
      e = launch_pass<false, false, ArrayKeys>(grid, s, ArrayKeys{nullptr}, kin, vin, kout, vout, n, 8 * p, dm, ntiles,
                                               offs + p * kRadix, look, *epoch, tile_ctr + p, err, gate);
    }
    if (e != cudaSuccess) return e;
    *launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kin = kout;
    vin = vout;
  }
  return cudaSuccess;
}

}  // namespace

static st_status run_deferred_gather(st_ctx* h);

st_status sort_particles(st_ctx* h) {
  const int64_t n = h->np;
  if (n == 0) return ST_OK;
  // a previous sort's gather still pending: the storage order it defined must be made real first
  if (h->perm_pending) ST_TRY(run_deferred_gather(h));
  if (n >= (int64_t(1) << 32)) return set_error(h, ST_ERR_INVALID_ARG, "sorting needs fewer than 2^32 particles");
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (h->sort_cap < h->cap) {
    size_t kb = (size_t)h->cap * sizeof(uint32_t);
    for (int b = 0; b < 2; ++b) {
      if (ensure(h, h->keys[b], kb) != ST_OK || ensure(h, h->vals[b], kb) != ST_OK) return ST_ERR_OOM;
    }
    h->sort_cap = h->cap;
  }
  // look-back words: one per tile and digit, cleared once per allocation (the epoch tells passes apart)
  const void* look_before = h->hist.p;
  if (ensure(h, h->hist, (size_t)ntiles * kRadix * sizeof(unsigned long long)) != ST_OK) return ST_ERR_OOM;
  if (ensure(h, h->scan_aux, (size_t)(2 * kMaxPasses * kRadix + kMaxPasses) * sizeof(uint32_t)) != ST_OK)
    return ST_ERR_OOM;
  if (ensure(h, h->cell_start, ((size_t)h->nkeys + 1) * sizeof(uint32_t)) != ST_OK) return ST_ERR_OOM;
  if (ensure(h, h->state_alt, state_alt_bytes(h->prec, h->cap)) != ST_OK) return ST_ERR_OOM;
  if (ensure(h, h->ids_alt, (size_t)h->cap * sizeof(uint32_t)) != ST_OK) return ST_ERR_OOM;
  if (h->hist.p != look_before || h->sort_epoch + kMaxPasses >= (1u << 30)) {
    // a new look-back buffer may hold anything, and once the 30-bit epoch tags are about to repeat
    // an old word could carry a current tag: clear the words so that no stale word carries an epoch
    cudaError_t ce = cudaMemsetAsync(h->hist.p, 0, h->hist.bytes, h->stream);
    if (ce != cudaSuccess) return cuda_check(h, ce, "clear look-back words");
    h->sort_epoch = 0;
  }

  KeyGeo g = key_geo(h);
  uint32_t* k0 = (uint32_t*)h->keys[0].p;
  uint32_t* v0 = (uint32_t*)h->vals[0].p;
  uint32_t* k1 = (uint32_t*)h->keys[1].p;
  uint32_t* v1 = (uint32_t*)h->vals[1].p;
  // particles sorted before and moved little since: the neighbourhood sort (sort_local.cu), with the
  // general sort's passes and cell starts queued behind it and gated on its "a particle moved too far"
  // flag.  Either leaves the permutation in v0; the payload gather below serves both.
  const int* gate = nullptr;
  if (local_sort_supported(h)) {
    if (ensure(h, h->lsort_aux, local_sort_aux_bytes(h)) != ST_OK) return ST_ERR_OOM;
    int* far = (int*)((char*)h->flags.p + kFarFlagOffset);
    cudaError_t le = launch_local_sort(h, far, v1, (uint16_t*)k1, v0, h->lsort_aux.p);
    if (le != cudaSuccess) return cuda_check(h, le, "neighbourhood sort");
    gate = far;
  }
  uint32_t* totals = (uint32_t*)h->scan_aux.p;
  uint32_t* offs = totals + kMaxPasses * kRadix;
  unsigned* tile_ctr = (unsigned*)(offs + kMaxPasses * kRadix);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev);
  if (sms <= 0) sms = 152;
  cudaError_t e;
  if (h->prec == ST_FP64) {
    PositionKeys src{carve_f64(h->state.p, h->cap), g};
    e = radix_passes(src, n, h->key_bits, k0, v0, k1, v1, k0, v0, totals, offs, tile_ctr,
                     (unsigned long long*)h->hist.p, &h->sort_epoch, (int*)h->flags.p, sms, h->stream, &h->launches,
                     true);
  } else {
    CellKeys src{(const int32_t*)h->state.p, g};
    e = radix_passes(src, n, h->key_bits, k0, v0, k1, v1, k0, v0, totals, offs, tile_ctr,
                     (unsigned long long*)h->hist.p, &h->sort_epoch, (int*)h->flags.p, sms, h->stream, &h->launches,
                     true, gate);
  }
  if (e != cudaSuccess) return cuda_check(h, e, "sort passes");
  // k0/v0 now hold the sorted keys and the permutation
  if (h->prec == ST_FP64) {
    gather_f64_kernel<<<grid_for(n), 256, 0, h->stream>>>(carve_f64(h->state.p, h->cap),
                                                          carve_f64(h->state_alt.p, h->cap), (const uint32_t*)h->ids.p,
                                                          (uint32_t*)h->ids_alt.p, v0, n);
  } else if (h->records_pending && defer_gather(h)) {
    // the next step is a sorted step that gathers through the permutation itself (GATHER instance)
    h->perm_pending = true;
  } else if (h->records_pending) {
    // the step before this sort left the state as records in state_alt: gather them back into
    // the (stale) structure of arrays; only the ids change buffers
    const bool bf = h->prec == ST_MIXED_BF16V;
    (bf ? gather_records_kernel<true> : gather_records_kernel<false>)<<<grid_for(n / 4 + 1), 256, 0, h->stream>>>(
        (const float4*)h->state_alt.p, carve_mixed(h->state.p, h->cap, bf), (const uint32_t*)h->ids.p,
        (uint32_t*)h->ids_alt.p, v0, n, nullptr);
  } else if (h->prec == ST_MIXED_F32) {
    gather_mixed_kernel<false><<<grid_for(n / 4 + 1), 256, 0, h->stream>>>(
        carve_mixed(h->state.p, h->cap, false), carve_mixed(h->state_alt.p, h->cap, false), (const uint32_t*)h->ids.p,
        (uint32_t*)h->ids_alt.p, v0, n, nullptr);
  } else {
    gather_mixed_kernel<true><<<grid_for(n / 4 + 1), 256, 0, h->stream>>>(
        carve_mixed(h->state.p, h->cap, true), carve_mixed(h->state_alt.p, h->cap, true), (const uint32_t*)h->ids.p,
        (uint32_t*)h->ids_alt.p, v0, n, nullptr);
  }
  cell_start_kernel<<<grid_for((n + 3) / 4), 256, 0, h->stream>>>(k0, n, (uint32_t*)h->cell_start.p, gate);
  cell_start_tail_kernel<<<grid_for((int64_t)h->nkeys + 1), 256, 0, h->stream>>>(k0, n, h->nkeys,
                                                                                   (uint32_t*)h->cell_start.p, gate);
  h->launches += h->perm_pending ? 2 : 3;  // gather + cell starts (two kernels)
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(h, e, "sort gather");
  if (h->perm_pending) return ST_OK;  // records and ids stay where they are until the gather
  // particle temperatures (microphysics), through the same permutation
  if (h->temp.p) {
    e = launch_gather_temp(h, v0, nullptr, 1);
    if (e != cudaSuccess) return cuda_check(h, e, "sort temperatures");
    std::swap(h->temp, h->temp_alt);
  }
  if (h->records_pending)
    h->records_pending = false;
  else
    std::swap(h->state, h->state_alt);
  std::swap(h->ids, h->ids_alt);
  return ST_OK;
}

// the payload gather a sort deferred: records (state_alt, old order) and ids through the permutation
// into the structure of arrays and ids_alt, as sort_particles would have done
static st_status run_deferred_gather(st_ctx* h) {
  const bool bf = h->prec == ST_MIXED_BF16V;
  (bf ? gather_records_kernel<true> : gather_records_kernel<false>)<<<grid_for(h->np / 4 + 1), 256, 0, h->stream>>>(
      (const float4*)h->state_alt.p, carve_mixed(h->state.p, h->cap, bf), (const uint32_t*)h->ids.p,
      (uint32_t*)h->ids_alt.p, (const uint32_t*)h->vals[0].p, h->np, nullptr);
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(h, e, "deferred sort gather");
  std::swap(h->ids, h->ids_alt);
  h->perm_pending = false;
  h->records_pending = false;
  return ST_OK;
}

bool defer_gather(const st_ctx* h) {
  return h->prec != ST_FP64 && !h->micro_on && default_physics(h) && tma_step_supported(h) &&
         h->reorder_every != 1 && h->np > 0;
}

void gather_step_done(st_ctx* h) {
  std::swap(h->ids, h->ids_alt);
  h->perm_pending = false;
  h->records_pending = false;
}

st_status materialize_state(st_ctx* h) {
  if (h->perm_pending) return run_deferred_gather(h);
  if (!h->records_pending) return ST_OK;
  const bool bf = h->prec == ST_MIXED_BF16V;
  (bf ? records_to_soa_kernel<true> : records_to_soa_kernel<false>)<<<grid_for(h->np), 256, 0, h->stream>>>(
      (const float4*)h->state_alt.p, carve_mixed(h->state.p, h->cap, bf), h->np);
  h->launches += 1;
  h->records_pending = false;
  return cuda_check(h, cudaGetLastError(), "records to arrays");
}

cudaError_t launch_chunk_bounds(st_ctx* h, double* out) {
  KeyGeo g = key_geo(h);
  const int64_t nchunk = (int64_t)g.ncx * g.ncy * ((h->geo.n[2] + g.B - 1) / g.B);
  const int grid = (int)std::min<int64_t>(nchunk, 152 * 8);
  const Geometry& G = h->geo;
  if (h->prec == ST_FP64)
    chunk_bounds_kernel<false><<<grid, 256, 0, h->stream>>>(MixedState{}, carve_f64(h->state.p, h->cap),
                                                            (const uint32_t*)h->cell_start.p, g, G.L[0], G.L[1],
                                                            G.L[2], G.h[0], G.h[1], G.h[2], nchunk, out);
  else
    chunk_bounds_kernel<true><<<grid, 256, 0, h->stream>>>(carve_mixed(h->state.p, h->cap, h->prec == ST_MIXED_BF16V),
                                                           F64State{}, (const uint32_t*)h->cell_start.p, g, G.L[0],
                                                           G.L[1], G.L[2], G.h[0], G.h[1], G.h[2], nchunk, out);
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_cell_counts(st_ctx* h, int64_t* counts) {
  KeyGeo g = key_geo(h);
  cell_counts_kernel<<<grid_for(h->geo.ncell), 256, 0, h->stream>>>((const uint32_t*)h->cell_start.p, g, counts);
  h->launches += 1;
  return cudaGetLastError();
}

}  // namespace st

// ---- the same stable sort for callers that cannot allocate device memory ----------------------
//
// Some callers cannot call cudaMalloc at all: code running inside another framework's memory
// pool or arena, a process whose allocations are made once at start-up and then frozen, or an
// allocator callback that must not re-enter the allocator.  st_sort_keys_static serves them:
// its scratch memory is one file-scope device array, so the call itself allocates nothing.
// Under CUDA's default lazy module loading the array comes into being on a device when this
// file's module is first used there (the first sort-related call on that device); it then lives
// until the process exits.

namespace st {
namespace {

constexpr int64_t kStaticMaxN = int64_t(1) << 20;  // keys per call (matches the header's limit)
constexpr int64_t kStaticTiles = kStaticMaxN / kTile;
// layout (32-bit words): ping-pong keys [N] | ping-pong values [N] | look-back words [2 T R] |
// digit totals [P R] | digit offsets [P R] | tile counters [P] | wait error word [1] (+ padding)
constexpr size_t kStaticLook = 2 * (size_t)kStaticMaxN;
constexpr size_t kStaticLookWords = 2 * (size_t)kStaticTiles * kRadix;  // 32-bit words of look-back
constexpr size_t kStaticTotals = kStaticLook + kStaticLookWords;
constexpr size_t kStaticErr = kStaticTotals + 2 * (size_t)kMaxPasses * kRadix + kMaxPasses;
constexpr size_t kStaticWords = kStaticErr + 4;
constexpr uint32_t kEpochSpan = 1u << 30;  // look-back epochs (30-bit tags)
constexpr uint32_t kEpochStep = 8;         // epochs reserved per call (at most kMaxPasses used)

}  // namespace
}  // namespace st

// The scratch array.  Host code must not use its name as an address: on the host the name
// refers to a host-side stand-in.  The device address comes from cudaGetSymbolAddress, once per
// device, below.  Device globals start zeroed, so no look-back word carries an epoch before use.
static __device__ __align__(256) uint32_t g_sort_scratch[st::kStaticWords];

namespace {
std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
uint32_t* g_scratch_addr[kMaxDevices] = {};
uint32_t g_scratch_epoch[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up on the first call per device)
// and that device's look-back epoch counter.
cudaError_t scratch_address(uint32_t** out, uint32_t** epoch) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (uint32_t*)p;
  }
  *out = g_scratch_addr[dev];
  *epoch = &g_scratch_epoch[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" st_status st_sort_keys_static(const uint32_t* keys, int64_t n, int key_bits, uint32_t* sorted_keys,
                                         uint32_t* perm, void* stream) {
  using namespace st;
  if (n < 0 || n > kStaticMaxN) return ST_ERR_INVALID_ARG;
  if (key_bits < 1 || key_bits > 32) return ST_ERR_INVALID_ARG;
  if (n == 0) return ST_OK;
  if (!keys || !sorted_keys || !perm) return ST_ERR_INVALID_ARG;
  uint32_t* base = nullptr;
  uint32_t* epoch = nullptr;
  if (scratch_address(&base, &epoch) != cudaSuccess) {
    cudaGetLastError();
    return ST_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* sk = base;
  uint32_t* sv = base + kStaticMaxN;
  unsigned long long* look = (unsigned long long*)(base + kStaticLook);
  uint32_t* totals = base + kStaticTotals;
  uint32_t* offs = totals + kMaxPasses * kRadix;
  unsigned* tile_ctr = offs + kMaxPasses * kRadix;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  int64_t launches = 0;
  // a look-back wait that gives up sets this word; it stays set until st_sort_keys_static_status
  // reads and clears it
  int* err = (int*)(base + kStaticErr);
  uint32_t ep;
  bool wrap = false;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ep = *epoch;
    if (ep + kEpochStep >= kEpochSpan) {
      // the 30-bit epoch tags would repeat: a word left by an old call could then carry the
      // current tag, so the look-back words start again from zero with the tags
      ep = 0;
      wrap = true;
    }
    *epoch = ep + kEpochStep;
  }
  cudaError_t e = cudaSuccess;
  if (wrap) e = cudaMemsetAsync(look, 0, kStaticLookWords * sizeof(uint32_t), s);
  if (e == cudaSuccess)
    e = radix_passes(ArrayKeys{keys}, n, key_bits, sk, sv, sorted_keys, perm, sorted_keys, perm, totals, offs,
                     tile_ctr, look, &ep, err, sms, s, &launches, false);
  return e == cudaSuccess ? ST_OK : ST_ERR_CUDA;
}

extern "C" st_status st_sort_keys_static_status(void* stream) {
  using namespace st;
  uint32_t* base = nullptr;
  uint32_t* epoch = nullptr;
  if (scratch_address(&base, &epoch) != cudaSuccess) {
    cudaGetLastError();
    return ST_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int* err = (int*)(base + kStaticErr);
  int f = 0;
  cudaError_t e = cudaMemcpyAsync(&f, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && f != 0) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ST_ERR_CUDA;
  }
  return f != 0 ? ST_ERR_TIMEOUT : ST_OK;
}
