// Stable counting sort of the particles by their chunk-major cell key.
//
// LSD radix sort of (key, slot) pairs with 8-bit digits; each pass is a
// stable counting sort in three phases: per-tile digit histograms (warp-
// aggregated shared-memory counts), one exclusive scan over the digit-major
// histogram matrix, and a scatter in which every element's rank among the
// equal digits of its tile comes from warp digit ballots and prefix counts combined
// across warps in warp order.  No phase waits on another block.  The
// structure-of-arrays payload is then gathered once through the final
// permutation.  Equal keys keep their storage order, so the permutation is
// unique.
#include <mutex>
#include <vector>

#include "st_common.cuh"

namespace st {
namespace {

constexpr int kSortThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kSortThreads * kItems;  // 4096 items per chunk
constexpr int kChunks = 16;
constexpr int64_t kBigTile = (int64_t)kTile * kChunks;  // 65536 items per tile (one CTA, chunks in order)
constexpr int kRadix = 256;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanBlock = kScanThreads * kScanItems;  // 2048

struct KeyGeo {
  int n[3];
  double inv_h[3];
  int B, logB, ncx, ncy;
};

__global__ void keys_f64_kernel(F64State s, int64_t n, KeyGeo g, uint32_t* __restrict__ keys,
                                uint32_t* __restrict__ vals) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int c[3];
    for (int q = 0; q < 3; ++q) {
      int i = (int)floor(s.x[q][p] * g.inv_h[q]);
      c[q] = min(max(i, 0), g.n[q] - 1);
    }
    keys[p] = chunk_key(c[0], c[1], c[2], g.B, g.logB, g.ncx, g.ncy);
    vals[p] = (uint32_t)p;
  }
}

__global__ void keys_mixed_kernel(const int32_t* __restrict__ cell, int64_t n, KeyGeo g, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = cell[p];
    keys[p] = chunk_key(cell_i(c), cell_j(c), cell_k(c), g.B, g.logB, g.ncx, g.ncy);
    vals[p] = (uint32_t)p;
  }
}

// lanes of the warp holding the same 8-bit digit (and the same validity): the intersection of one
// ballot per digit bit, a fixed cost whatever the number of distinct digits in the warp
__device__ __forceinline__ unsigned match_digit(uint32_t dig, bool valid) {
  unsigned m = __ballot_sync(0xffffffffu, valid);
  m = valid ? m : ~m;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (dig >> b) & 1u;
    const unsigned bb = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bb : ~bb;
  }
  return m;
}

// phase 1: digit histogram of each tile, stored digit-major: hist[d * ntiles + t]
__global__ void __launch_bounds__(kSortThreads) upsweep_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                                int64_t ntiles, uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[kRadix];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t = blockIdx.x;
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < kChunks; ++c) {
    const int64_t base = t * kBigTile + (int64_t)c * kTile;
    uint32_t k[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
      k[r] = i < n ? keys[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
      const bool valid = i < n;
      const uint32_t dig = (k[r] >> shift) & 0xffu;
      const unsigned peers = match_digit(dig, valid);
      if (valid && lane == __ffs(peers) - 1) atomicAdd(&cnt[dig], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + t] = cnt[threadIdx.x];
}

// exclusive scan, three kernels: block sums, scan of the block sums (one block,
// sequential over chunks with a carry), then block-local scans plus offsets
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    uint32_t s = lane < nw ? wsum[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) wsum[lane] = s;
  }
  __syncthreads();
  uint32_t before = (w > 0 ? wsum[w - 1] : 0u) + x - v;
  *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t m,
                                                                   uint32_t* __restrict__ bsum) {
  uint32_t s = 0;
  int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < m) s += in[base + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ uint32_t ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) scan_blocksums_kernel(uint32_t* __restrict__ bsum, int64_t nb) {
  uint32_t carry = 0;
  for (int64_t c = 0; c < nb; c += 1024) {
    int64_t i = c + threadIdx.x;
    uint32_t v = i < nb ? bsum[i] : 0u;
    uint32_t total;
    uint32_t ex = block_exclusive_scan(v, &total);
    if (i < nb) bsum[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t* __restrict__ in,
                                                                  uint32_t* __restrict__ out, int64_t m,
                                                                  const uint32_t* __restrict__ bsum) {
  uint32_t v[kScanItems];
  int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  uint32_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < m) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t ex = block_exclusive_scan(s, &total) + bsum[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < m) out[base + k] = ex;
    ex += v[k];
  }
}

// phase 3: stable scatter.  A tile is processed as kChunks chunks in order; in a chunk warp w
// owns items [w*512, (w+1)*512) in 16 coalesced rounds.  Ranks inside a round come from
// digit ballots + popc, across rounds from a per-warp running count, across warps from a prefix in
// warp order, and across chunks from per-digit running offsets.
__global__ void __launch_bounds__(kSortThreads) downsweep_kernel(const uint32_t* __restrict__ kin,
                                                                  const uint32_t* __restrict__ vin,
                                                                  uint32_t* __restrict__ kout,
                                                                  uint32_t* __restrict__ vout, int64_t n, int shift,
                                                                  int64_t ntiles, const uint32_t* __restrict__ offs) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t wcnt[kWarps][kRadix];
  __shared__ uint32_t base[kRadix];
  __shared__ uint32_t chunk_total[kRadix];
  const int64_t t = blockIdx.x;
  base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + t];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < kChunks; ++c) {
    const int64_t cstart = t * kBigTile + (int64_t)c * kTile;
    if (cstart >= n) break;
    for (int ww = 0; ww < kWarps; ++ww) wcnt[ww][threadIdx.x] = 0;
    __syncthreads();
    uint32_t key[kItems], val[kItems], rank[kItems];
    const int64_t start = cstart + (int64_t)w * (kItems * 32);
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int64_t i = start + r * 32 + lane;
      key[r] = i < n ? kin[i] : 0u;
      val[r] = i < n ? vin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int64_t i = start + r * 32 + lane;
      const bool valid = i < n;
      const uint32_t dig = (key[r] >> shift) & 0xffu;
      const unsigned peers = match_digit(dig, valid);
      uint32_t before = 0;
      if (valid) before = wcnt[w][dig];
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) wcnt[w][dig] = before + __popc(peers);
      __syncwarp();
      rank[r] = valid ? before + __popc(peers & lt) : 0xffffffffu;
    }
    __syncthreads();
    {
      uint32_t acc = 0;
      for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t cc = wcnt[ww][threadIdx.x];
        wcnt[ww][threadIdx.x] = acc;
        acc += cc;
      }
      chunk_total[threadIdx.x] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      if (rank[r] != 0xffffffffu) {
        const uint32_t dig = (key[r] >> shift) & 0xffu;
        const uint32_t dst = base[dig] + wcnt[w][dig] + rank[r];
        kout[dst] = key[r];
        vout[dst] = val[r];
      }
    }
    __syncthreads();
    base[threadIdx.x] += chunk_total[threadIdx.x];
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

// mixed-precision payload gather, 4 consecutive outputs per thread: one 16-byte load of the
// permutation, then every gathered load of the 4 particles in flight at once, then 128-bit
// (64-bit for BF16 velocities) coalesced stores
template <bool BF16>
__global__ void gather_mixed_kernel(MixedState src, MixedState dst, const uint32_t* __restrict__ sid,
                                    uint32_t* __restrict__ did, const uint32_t* __restrict__ perm, int64_t n) {
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
__global__ void cell_start_kernel(const uint32_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ start) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k1 = keys[i];
    const int64_t k0 = i > 0 ? (int64_t)keys[i - 1] : -1;
    for (int64_t k = k0 + 1; k <= k1; ++k) start[k] = (uint32_t)i;
  }
}

__global__ void cell_start_tail_kernel(const uint32_t* __restrict__ keys, int64_t n, uint32_t nkeys,
                                       uint32_t* __restrict__ start) {
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

cudaError_t exclusive_scan(st_ctx* h, const uint32_t* in, uint32_t* out, int64_t m) {
  int64_t nb = (m + kScanBlock - 1) / kScanBlock;
  uint32_t* bsum = (uint32_t*)h->scan_aux.p;
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, h->stream>>>(in, m, bsum);
  scan_blocksums_kernel<<<1, 1024, 0, h->stream>>>(bsum, nb);
  scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, h->stream>>>(in, out, m, bsum);
  h->launches += 3;
  return cudaGetLastError();
}

}  // namespace

st_status sort_particles(st_ctx* h) {
  const int64_t n = h->np;
  if (n == 0) return ST_OK;
  if (n >= (int64_t(1) << 32)) return set_error(h, ST_ERR_INVALID_ARG, "sorting needs fewer than 2^32 particles");
  const int64_t ntiles = (n + kBigTile - 1) / kBigTile;
  const int64_t hm = ntiles * kRadix;
  const int64_t nb = (hm + kScanBlock - 1) / kScanBlock;
  if (h->sort_cap < h->cap) {
    size_t kb = (size_t)h->cap * sizeof(uint32_t);
    for (int b = 0; b < 2; ++b) {
      if (ensure(h, h->keys[b], kb) != ST_OK || ensure(h, h->vals[b], kb) != ST_OK) return ST_ERR_OOM;
    }
    h->sort_cap = h->cap;
  }
  if (ensure(h, h->hist, (size_t)hm * 2 * sizeof(uint32_t)) != ST_OK) return ST_ERR_OOM;
  if (ensure(h, h->scan_aux, (size_t)(nb + 1) * sizeof(uint32_t)) != ST_OK) return ST_ERR_OOM;
  if (ensure(h, h->cell_start, ((size_t)h->nkeys + 1) * sizeof(uint32_t)) != ST_OK) return ST_ERR_OOM;
  if (ensure(h, h->state_alt, state_bytes(h->prec, h->cap)) != ST_OK) return ST_ERR_OOM;
  if (ensure(h, h->ids_alt, (size_t)h->cap * sizeof(uint32_t)) != ST_OK) return ST_ERR_OOM;

  KeyGeo g = key_geo(h);
  uint32_t* k0 = (uint32_t*)h->keys[0].p;
  uint32_t* v0 = (uint32_t*)h->vals[0].p;
  uint32_t* k1 = (uint32_t*)h->keys[1].p;
  uint32_t* v1 = (uint32_t*)h->vals[1].p;
  if (h->prec == ST_FP64)
    keys_f64_kernel<<<grid_for(n), 256, 0, h->stream>>>(carve_f64(h->state.p, h->cap), n, g, k0, v0);
  else
    keys_mixed_kernel<<<grid_for(n), 256, 0, h->stream>>>((const int32_t*)h->state.p, n, g, k0, v0);
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(h, e, "sort keys");
  uint32_t* hist = (uint32_t*)h->hist.p;
  uint32_t* offs = hist + hm;
  for (int shift = 0; shift < h->key_bits; shift += 8) {
    upsweep_kernel<<<(unsigned)ntiles, kSortThreads, 0, h->stream>>>(k0, n, shift, ntiles, hist);
    e = exclusive_scan(h, hist, offs, hm);
    if (e != cudaSuccess) return cuda_check(h, e, "sort scan");
    downsweep_kernel<<<(unsigned)ntiles, kSortThreads, 0, h->stream>>>(k0, v0, k1, v1, n, shift, ntiles, offs);
    h->launches += 2;  // upsweep + downsweep
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(h, e, "sort pass");
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  // k0/v0 now hold the sorted keys and the permutation
  if (h->prec == ST_FP64) {
    gather_f64_kernel<<<grid_for(n), 256, 0, h->stream>>>(carve_f64(h->state.p, h->cap),
                                                          carve_f64(h->state_alt.p, h->cap), (const uint32_t*)h->ids.p,
                                                          (uint32_t*)h->ids_alt.p, v0, n);
  } else if (h->prec == ST_MIXED_F32) {
    gather_mixed_kernel<false><<<grid_for(n / 4 + 1), 256, 0, h->stream>>>(
        carve_mixed(h->state.p, h->cap, false), carve_mixed(h->state_alt.p, h->cap, false), (const uint32_t*)h->ids.p,
        (uint32_t*)h->ids_alt.p, v0, n);
  } else {
    gather_mixed_kernel<true><<<grid_for(n / 4 + 1), 256, 0, h->stream>>>(
        carve_mixed(h->state.p, h->cap, true), carve_mixed(h->state_alt.p, h->cap, true), (const uint32_t*)h->ids.p,
        (uint32_t*)h->ids_alt.p, v0, n);
  }
  cell_start_kernel<<<grid_for(n), 256, 0, h->stream>>>(k0, n, (uint32_t*)h->cell_start.p);
  cell_start_tail_kernel<<<grid_for((int64_t)h->nkeys + 1), 256, 0, h->stream>>>(k0, n, h->nkeys,
                                                                                   (uint32_t*)h->cell_start.p);
  h->launches += 3;  // gather + cell starts (two kernels)
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(h, e, "sort gather");
  std::swap(h->state, h->state_alt);
  std::swap(h->ids, h->ids_alt);
  return ST_OK;
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
// The array is created when the library is loaded and lives on every GPU that loads the library
// until the process exits.

namespace st {
namespace {

constexpr int64_t kStaticMaxN = int64_t(1) << 20;  // keys per call (matches the header's limit)
constexpr int64_t kStaticTiles = kStaticMaxN / kBigTile;
constexpr int64_t kStaticHist = kStaticTiles * kRadix;
constexpr int64_t kStaticAux = (kStaticHist + kScanBlock - 1) / kScanBlock + 1;
// layout: index seeds [N] | ping-pong keys [N] | ping-pong values [N] | histograms [H] | offsets [H] | scan aux
constexpr size_t kStaticWords = (size_t)(3 * kStaticMaxN + 2 * kStaticHist + kStaticAux);

__global__ void iota_kernel(uint32_t* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)i;
}

// exclusive scan with caller-provided block-sum storage `aux` ((m + 2047) / 2048 + 1 words)
cudaError_t exclusive_scan_aux(const uint32_t* in, uint32_t* out, int64_t m, uint32_t* aux, cudaStream_t s) {
  int64_t nb = (m + kScanBlock - 1) / kScanBlock;
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, m, aux);
  scan_blocksums_kernel<<<1, 1024, 0, s>>>(aux, nb);
  scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, m, aux);
  return cudaGetLastError();
}

}  // namespace

}  // namespace st

// The scratch array.  Host code must not use its name as an address: on the host the name
// refers to a host-side stand-in.  The device address comes from cudaGetSymbolAddress, once per
// device, below.
static __device__ __align__(256) uint32_t g_sort_scratch[st::kStaticWords];

namespace {
std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
uint32_t* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up on the first call per device).
cudaError_t scratch_address(uint32_t** out) {
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
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return ST_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* seed = base;
  uint32_t* sk = base + kStaticMaxN;
  uint32_t* sv = base + 2 * kStaticMaxN;
  uint32_t* hist = base + 3 * kStaticMaxN;
  uint32_t* offs = hist + kStaticHist;
  uint32_t* aux = offs + kStaticHist;
  const int64_t ntiles = (n + kBigTile - 1) / kBigTile;
  const int passes = (key_bits + 7) / 8;
  iota_kernel<<<grid_for(n), 256, 0, s>>>(seed, n);
  // alternate between the caller's outputs and the scratch pair so that the last pass lands in the outputs
  const uint32_t* kin = keys;
  const uint32_t* vin = seed;
  for (int p = 0; p < passes; ++p) {
    bool to_out = ((passes - 1 - p) % 2) == 0;
    uint32_t* kout = to_out ? sorted_keys : sk;
    uint32_t* vout = to_out ? perm : sv;
    upsweep_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(kin, n, 8 * p, ntiles, hist);
    if (exclusive_scan_aux(hist, offs, ntiles * kRadix, aux, s) != cudaSuccess) return ST_ERR_CUDA;
    downsweep_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, 8 * p, ntiles, offs);
    if (cudaGetLastError() != cudaSuccess) return ST_ERR_CUDA;
    kin = kout;
    vin = vout;
  }
  return ST_OK;
}
