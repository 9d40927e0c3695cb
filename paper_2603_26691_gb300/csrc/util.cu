// Support kernels: argument scans, fluid packing, particle import/export,
// accumulator conversion and rescaling, invariant reductions, and the
// device-side twin of the seeded input generator.
#include <cmath>
#include <cstring>
#include <vector>

#include "st_common.cuh"

namespace st {

namespace {

constexpr int kThreads = 256;

int grid_for(int64_t n, int threads = kThreads, int max_blocks = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// ---- scans ----------------------------------------------------------------------------

template <typename T>
__global__ void maxabs_kernel(const T* __restrict__ p, int64_t n, unsigned long long* out_bits, int* flag) {
  double m = 0.0;
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)p[i];
    if (!isfinite(v)) bad = 1;
    else m = fmax(m, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out_bits, dbits(m));
    if (bad) atomicOr(flag, 1);
  }
}

__global__ void particle_scan_kernel(const double* __restrict__ xyz, const double* __restrict__ d, int64_t n,
                                     unsigned long long* dmax_bits, int* flag) {
  double m = 0.0;
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double di = d[i];
    if (!isfinite(xyz[i]) || !isfinite(xyz[n + i]) || !isfinite(xyz[2 * n + i]) || !isfinite(di)) bad |= 1;
    else if (!(di > 0.0)) bad |= 2;
    else m = fmax(m, di);
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(dmax_bits, dbits(m));
    if (bad) atomicOr(flag, bad);
  }
}

// ---- fluid packing -----------------------------------------------------------------------

template <typename T>
__global__ void pack_f64_kernel(const T* __restrict__ u, D4* __restrict__ out, int64_t ncell,
                                const int* __restrict__ skip = nullptr) {
  if (skip && *skip) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x)
    out[c] = D4{(double)u[3 * c], (double)u[3 * c + 1], (double)u[3 * c + 2], 0.0};
}

// FP32 field with P ghost layers on every side, filled periodically: padded cell (a, b, c)
// holds cell ((a - P) mod nx, (b - P) mod ny, (c - P) mod nz)
template <typename T>
__global__ void pack_f32_padded_kernel(const T* __restrict__ u, float4* __restrict__ out, int nx, int ny, int nz,
                                       int P, const int* __restrict__ skip = nullptr) {
  if (skip && *skip) return;
  const int64_t px = nx + 2 * P, py = ny + 2 * P, pz = nz + 2 * P;
  const int64_t total = px * py * pz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(t % px), b = (int)((t / px) % py), c = (int)(t / (px * py));
    int i = (a - P) % nx, j = (b - P) % ny, k = (c - P) % nz;
    i += i < 0 ? nx : 0;
    j += j < 0 ? ny : 0;
    k += k < 0 ? nz : 0;
    const int64_t s = i + (int64_t)nx * (j + (int64_t)ny * k);
    out[t] = make_float4((float)u[3 * s], (float)u[3 * s + 1], (float)u[3 * s + 2], 0.0f);
  }
}

// ---- particle import / export --------------------------------------------------------------

struct GeoArgs {
  int n[3];
  double L[3], invL[3], h[3], inv_h[3];
};

GeoArgs geo_args(const Geometry& G) {
  GeoArgs a;
  for (int q = 0; q < 3; ++q) {
    a.n[q] = G.n[q];
    a.L[q] = G.L[q];
    a.invL[q] = 1.0 / G.L[q];
    a.h[q] = G.h[q];
    a.inv_h[q] = G.inv_h[q];
  }
  return a;
}

__device__ __forceinline__ double wrap_pos(double x, double L, double invL) {
  double y = x - L * floor(x * invL);
  if (y < 0.0) y += L;
  if (y >= L) y = 0.0;
  return y;
}

__global__ void import_f64_kernel(F64State s, int64_t first, int64_t n, const double* __restrict__ xyz,
                                  const double* __restrict__ vel, const double* __restrict__ d,
                                  const uint32_t* __restrict__ ids, uint32_t* __restrict__ oid, GeoArgs g) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    for (int q = 0; q < 3; ++q) {
      s.x[q][first + p] = wrap_pos(xyz[q * n + p], g.L[q], g.invL[q]);
      s.v[q][first + p] = vel ? vel[q * n + p] : 0.0;
    }
    s.d[first + p] = d[p];
    oid[first + p] = ids ? ids[p] : (uint32_t)(first + p);
  }
}

__global__ void import_mixed_kernel(MixedState s, bool bf16, int64_t first, int64_t n, const double* __restrict__ xyz,
                                    const double* __restrict__ vel, const double* __restrict__ d,
                                    const uint32_t* __restrict__ ids, uint32_t* __restrict__ oid, GeoArgs g) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int idx[3];
    for (int q = 0; q < 3; ++q) {
      double x = wrap_pos(xyz[q * n + p], g.L[q], g.invL[q]);
      double s_ = x * g.inv_h[q];
      int i = (int)floor(s_);
      if (i > g.n[q] - 1) i = g.n[q] - 1;
      if (i < 0) i = 0;
      float xi = (float)(s_ - (double)i);
      if (xi >= 1.0f) {  // rounding reached the upper face: the particle belongs to the next cell
        xi = 0.0f;
        i = (i + 1 == g.n[q]) ? 0 : i + 1;
      }
      if (xi < 0.0f) xi = 0.0f;
      idx[q] = i;
      s.xi[q][first + p] = xi;
      double v = vel ? vel[q * n + p] : 0.0;
      if (bf16)
        ((__nv_bfloat16*)s.v[q])[first + p] = __double2bfloat16(v);
      else
        ((float*)s.v[q])[first + p] = (float)v;
    }
    s.cell[first + p] = pack_cell(idx[0], idx[1], idx[2]);
    s.d[first + p] = (float)d[p];
    oid[first + p] = ids ? ids[p] : (uint32_t)(first + p);
  }
}

__global__ void export_f64_kernel(F64State s, const uint32_t* __restrict__ sid, int64_t first, int64_t n,
                                  double* xyz, double* vel, double* d, uint32_t* ids, int32_t* cells, GeoArgs g) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t sp = first + p;
    int idx[3];
    for (int q = 0; q < 3; ++q) {
      double x = s.x[q][sp];
      if (xyz) xyz[q * n + p] = x;
      if (vel) vel[q * n + p] = s.v[q][sp];
      int i = (int)floor(x * g.inv_h[q]);
      idx[q] = min(max(i, 0), g.n[q] - 1);
    }
    if (d) d[p] = s.d[sp];
    if (ids) ids[p] = sid[sp];
    if (cells) cells[p] = idx[0] + g.n[0] * (idx[1] + g.n[1] * idx[2]);
  }
}

// ms (microphysics on): per particle {T_hi, T_lo, d_lo, 0}; the diameter is d + d_lo
__global__ void export_mixed_kernel(MixedState s, bool bf16, const uint32_t* __restrict__ sid, int64_t first,
                                    int64_t n, double* xyz, double* vel, double* d, uint32_t* ids, int32_t* cells,
                                    GeoArgs g, const float4* __restrict__ ms) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t sp = first + p;
    int32_t c = s.cell[sp];
    int idx[3] = {cell_i(c), cell_j(c), cell_k(c)};
    for (int q = 0; q < 3; ++q) {
      if (xyz) xyz[q * n + p] = ((double)idx[q] + (double)s.xi[q][sp]) * g.h[q];
      if (vel) {
        double v = bf16 ? (double)__bfloat162float(((const __nv_bfloat16*)s.v[q])[sp]) : (double)((const float*)s.v[q])[sp];
        vel[q * n + p] = v;
      }
    }
    if (d) d[p] = (double)s.d[sp] + (ms ? (double)ms[sp].z : 0.0);
    if (ids) ids[p] = sid[sp];
    if (cells) cells[p] = idx[0] + g.n[0] * (idx[1] + g.n[1] * idx[2]);
  }
}

// ---- accumulator ----------------------------------------------------------------------

__global__ void acc_to_f64_kernel(const long long* __restrict__ acc, double* __restrict__ out, int64_t m,
                                  double inv_scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long lo;
    long long hi;
    acc_value(acc + kAccWords * i, lo, hi);
    out[i] = i128_to_f64(lo, hi) * inv_scale;
  }
}

// carry propagation: rewrite every value with digits in [0, 2^32) below a signed top word (only
// when *flag is set, if a flag is given)
__global__ void normalize_kernel(long long* __restrict__ acc, int64_t m, const int* __restrict__ flag) {
  if (flag && *flag == 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    long long* w = acc + kAccWords * i;
    unsigned long long lo;
    long long hi;
    acc_value(w, lo, hi);
    w[0] = (long long)(lo & 0xffffffffull);
    w[1] = (long long)(lo >> 32);
    w[2] = (long long)((unsigned long long)hi & 0xffffffffull);
    w[3] = hi >> 32;
  }
}

// arithmetic right shift of every value by `sh` bits (1..120), rounding half up; also normalises
__global__ void rescale_kernel(long long* __restrict__ acc, int64_t m, int sh) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    long long* w = acc + kAccWords * i;
    unsigned long long lo;
    long long shi;
    acc_value(w, lo, shi);
    unsigned long long hi = (unsigned long long)shi;
    unsigned long long alo, ahi;
    if (sh - 1 < 64) {
      alo = 1ull << (sh - 1);
      ahi = 0;
    } else {
      alo = 0;
      ahi = 1ull << (sh - 1 - 64);
    }
    unsigned long long nlo = lo + alo;
    hi = hi + ahi + (nlo < lo ? 1ull : 0ull);
    lo = nlo;
    shi = (long long)hi;
    if (sh < 64) {
      lo = (lo >> sh) | (hi << (64 - sh));
      shi = shi >> sh;
    } else {
      lo = (unsigned long long)(shi >> (sh - 64));
      shi = shi >> 63;
    }
    w[0] = (long long)(lo & 0xffffffffull);
    w[1] = (long long)(lo >> 32);
    w[2] = (long long)((unsigned long long)shi & 0xffffffffull);
    w[3] = shi >> 32;
  }
}

// exact 128-bit sums of each component over all cells
__global__ void acc_sum_kernel(const long long* __restrict__ acc, int64_t ncell,
                               unsigned long long* __restrict__ out /* [3][2] */) {
  int q = blockIdx.y;
  unsigned long long lo = 0, hi = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long a;
    long long b;
    acc_value(acc + kAccWords * (q * ncell + c), a, b);
    unsigned long long n = lo + a;
    hi += (unsigned long long)b + (n < lo ? 1ull : 0ull);
    lo = n;
  }
  atomic_add_i128(out + 2 * q, lo, hi);
}

// FP64 partial sums of m v and m per block, combined on the host in block order
template <int PREC>
__global__ void particle_sums_kernel(F64State sf, MixedState sm, int64_t n, double mcoef, double* __restrict__ part) {
  double a[4] = {0, 0, 0, 0};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double d, v[3];
    if (PREC == ST_FP64) {
      d = sf.d[p];
      for (int q = 0; q < 3; ++q) v[q] = sf.v[q][p];
    } else if (PREC == ST_MIXED_F32) {
      d = (double)sm.d[p];
      for (int q = 0; q < 3; ++q) v[q] = (double)((const float*)sm.v[q])[p];
    } else {
      d = (double)sm.d[p];
      for (int q = 0; q < 3; ++q) v[q] = (double)__bfloat162float(((const __nv_bfloat16*)sm.v[q])[p]);
    }
    double m = mcoef * d * d * d;
    for (int q = 0; q < 3; ++q) a[q] += m * v[q];
    a[3] += m;
  }
  __shared__ double sh[4][kThreads / 32];
  for (int k = 0; k < 4; ++k) {
    double x = a[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double x = 0;
    for (int w = 0; w < kThreads / 32; ++w) x += sh[threadIdx.x][w];
    part[blockIdx.x * 4 + threadIdx.x] = x;
  }
}

// ---- seeded input generator (device twin of the package's input module) ----------------------

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gen_kernel(unsigned long long key, int64_t first, int64_t count, double L0, double L1, double L2,
                           double vmax, const double* __restrict__ qt, int qbits, double* xyz, double* vel,
                           double* d, uint32_t* ids) {
  const unsigned long long G = 0x9E3779B97F4A7C15ull;
  double L[3] = {L0, L1, L2};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < count; p += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long idx = (unsigned long long)(first + p);
    unsigned long long c0 = idx * 8ull + 1ull;
    if (xyz) {
      for (int q = 0; q < 3; ++q) {
        unsigned long long w = mix64(key + (c0 + q) * G);
        double u = (double)(w >> 11) * 0x1p-53;
        xyz[q * count + p] = __dmul_rn(L[q], u);
      }
    }
    if (d) {
      unsigned long long w = mix64(key + (c0 + 3) * G);
      unsigned long long seg = w >> (64 - qbits);
      double frac = (double)((w >> 11) & ((1ull << 37) - 1)) * 0x1p-37;
      double q0 = qt[seg];
      double dq = __dsub_rn(qt[seg + 1], q0);
      double t = __dmul_rn(frac, dq);
      d[p] = __dadd_rn(q0, t);
    }
    if (vel) {
      for (int q = 0; q < 3; ++q) {
        double v = 0.0;
        if (vmax != 0.0) {
          unsigned long long w = mix64(key + (c0 + 4 + q) * G);
          double u = (double)(w >> 11) * 0x1p-53;
          v = __dmul_rn(vmax, __dsub_rn(__dmul_rn(2.0, u), 1.0));
        }
        vel[q * count + p] = v;
      }
    }
    if (ids) ids[p] = (uint32_t)idx;
  }
}

unsigned long long mix64_host(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

cudaError_t launch_maxabs(st_ctx* h, const void* p, int64_t n, int dtype, double* out_max, int* nonfinite) {
  unsigned long long* bits = (unsigned long long*)h->red.p;
  int* flag = (int*)(bits + 1);
  cudaError_t e = cudaMemsetAsync(h->red.p, 0, 16, h->stream);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    if (dtype == ST_DTYPE_F64)
      maxabs_kernel<double><<<grid_for(n), kThreads, 0, h->stream>>>((const double*)p, n, bits, flag);
    else
      maxabs_kernel<float><<<grid_for(n), kThreads, 0, h->stream>>>((const float*)p, n, bits, flag);
    h->launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  unsigned long long hb[2];
  e = cudaMemcpyAsync(hb, h->red.p, 16, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  double m;
  memcpy(&m, &hb[0], 8);
  *out_max = m;
  *nonfinite = (int)(hb[1] & 0xffffffffu);
  return cudaSuccess;
}

cudaError_t launch_particle_scan(st_ctx* h, const double* xyz, const double* d, int64_t n, double* vmax, double* dmax,
                                 double* dmin, int* nonfinite) {
  unsigned long long* bits = (unsigned long long*)h->red.p;
  int* flag = (int*)(bits + 1);
  cudaError_t e = cudaMemsetAsync(h->red.p, 0, 16, h->stream);
  if (e != cudaSuccess) return e;
  particle_scan_kernel<<<grid_for(n), kThreads, 0, h->stream>>>(xyz, d, n, bits, flag);
  h->launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  unsigned long long hb[2];
  e = cudaMemcpyAsync(hb, h->red.p, 16, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  double m;
  memcpy(&m, &hb[0], 8);
  int f = (int)(hb[1] & 0xffffffffu);
  *vmax = 0.0;
  *dmax = m;
  *dmin = (f & 2) ? 0.0 : 1.0;  // only positivity is reported
  *nonfinite = f & 1;
  return cudaSuccess;
}

cudaError_t launch_fluid_pack(st_ctx* h, const void* u, int dtype) { return launch_fluid_pack_if(h, u, dtype, nullptr); }

cudaError_t launch_fluid_pack_if(st_ctx* h, const void* u, int dtype, const int* skip) {
  int64_t nc = h->geo.ncell;
  if (h->prec == ST_FP64) {
    if (dtype == ST_DTYPE_F64)
      pack_f64_kernel<double><<<grid_for(nc), kThreads, 0, h->stream>>>((const double*)u, (D4*)h->fluid.p, nc, skip);
    else
      pack_f64_kernel<float><<<grid_for(nc), kThreads, 0, h->stream>>>((const float*)u, (D4*)h->fluid.p, nc, skip);
  } else {
    const Geometry& G = h->geo;
    const int64_t tot = (int64_t)(G.n[0] + 2 * kFluidPad) * (G.n[1] + 2 * kFluidPad) * (G.n[2] + 2 * kFluidPad);
    if (dtype == ST_DTYPE_F64)
      pack_f32_padded_kernel<double><<<grid_for(tot), kThreads, 0, h->stream>>>(
          (const double*)u, (float4*)h->fluid_pad.p, G.n[0], G.n[1], G.n[2], kFluidPad, skip);
    else
      pack_f32_padded_kernel<float><<<grid_for(tot), kThreads, 0, h->stream>>>(
          (const float*)u, (float4*)h->fluid_pad.p, G.n[0], G.n[1], G.n[2], kFluidPad, skip);
  }
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_maxabs_on(st_ctx* h, const void* p, int64_t n, int dtype, cudaStream_t stream,
                             unsigned long long* dev_red, unsigned long long* host_red) {
  cudaError_t e = cudaMemsetAsync(dev_red, 0, 16, stream);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    int* flag = (int*)(dev_red + 1);
    if (dtype == ST_DTYPE_F64)
      maxabs_kernel<double><<<grid_for(n), kThreads, 0, stream>>>((const double*)p, n, dev_red, flag);
    else
      maxabs_kernel<float><<<grid_for(n), kThreads, 0, stream>>>((const float*)p, n, dev_red, flag);
    h->launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpyAsync(host_red, dev_red, 16, cudaMemcpyDeviceToHost, stream);
}

cudaError_t launch_import(st_ctx* h, int64_t first, int64_t n, const double* xyz, const double* vel, const double* d,
                          const uint32_t* ids) {
  GeoArgs g = geo_args(h->geo);
  if (h->prec == ST_FP64) {
    import_f64_kernel<<<grid_for(n), kThreads, 0, h->stream>>>(carve_f64(h->state.p, h->cap), first, n, xyz, vel, d,
                                                               ids, (uint32_t*)h->ids.p, g);
  } else {
    bool bf = h->prec == ST_MIXED_BF16V;
    import_mixed_kernel<<<grid_for(n), kThreads, 0, h->stream>>>(carve_mixed(h->state.p, h->cap, bf), bf, first, n,
                                                                 xyz, vel, d, ids, (uint32_t*)h->ids.p, g);
  }
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_export(st_ctx* h, int64_t first, int64_t n, double* xyz, double* vel, double* d, uint32_t* ids,
                          int32_t* cells) {
  GeoArgs g = geo_args(h->geo);
  if (h->prec == ST_FP64) {
    export_f64_kernel<<<grid_for(n), kThreads, 0, h->stream>>>(carve_f64(h->state.p, h->cap), (const uint32_t*)h->ids.p,
                                                               first, n, xyz, vel, d, ids, cells, g);
  } else {
    bool bf = h->prec == ST_MIXED_BF16V;
    export_mixed_kernel<<<grid_for(n), kThreads, 0, h->stream>>>(carve_mixed(h->state.p, h->cap, bf), bf,
                                                                 (const uint32_t*)h->ids.p, first, n, xyz, vel, d,
                                                                 ids, cells, g, (const float4*)h->temp.p);
  }
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_acc_to_f64(st_ctx* h, double* out, int E) {
  int64_t m = h->geo.ncell * 3;
  acc_to_f64_kernel<<<grid_for(m), kThreads, 0, h->stream>>>((const long long*)h->acc.p, out, m,
                                                             std::ldexp(1.0, -E));
  h->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_rescale_acc(st_ctx* h, int shift) {
  if (shift <= 0) return cudaSuccess;
  while (shift > 0) {
    int s = shift > 120 ? 120 : shift;
    int64_t m = h->geo.ncell * 3;
    rescale_kernel<<<grid_for(m), kThreads, 0, h->stream>>>((long long*)h->acc.p, m, s);
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    shift -= s;
  }
  return cudaSuccess;
}

cudaError_t launch_normalize_acc(st_ctx* h) {
  int64_t m = h->geo.ncell * 3;
  normalize_kernel<<<grid_for(m), kThreads, 0, h->stream>>>((long long*)h->acc.p, m, nullptr);
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? reset_acc_counter(h) : e;
}

// each int64 word takes digits of magnitude < 2^32: 2^31 of them cannot overflow it
__global__ void acc_decide_kernel(unsigned long long* __restrict__ ctr, int* __restrict__ flag, double worst,
                                  double add) {
  const double limit = 2147483648.0 - 1048576.0;
  unsigned long long c = *ctr;
  const int f = (double)c + worst > limit;
  if (f) c = 1;  // after propagation every word holds one digit
  *ctr = c + (unsigned long long)add;
  *flag = f;
}

cudaError_t launch_acc_maybe_normalize(st_ctx* h, double worst, double add) {
  unsigned long long* ctr = (unsigned long long*)((char*)h->flags.p + kAccCounterOffset);
  int* flag = (int*)((char*)h->flags.p + kAccFlagOffset);
  acc_decide_kernel<<<1, 1, 0, h->stream>>>(ctr, flag, worst, add);
  int64_t m = h->geo.ncell * 3;
  normalize_kernel<<<grid_for(m), kThreads, 0, h->stream>>>((long long*)h->acc.p, m, flag);
  h->launches += 2;
  return cudaGetLastError();
}

cudaError_t reset_acc_counter(st_ctx* h) {
  return cudaMemsetAsync((char*)h->flags.p + kAccCounterOffset, 0, sizeof(unsigned long long), h->stream);
}

cudaError_t launch_acc_sum(st_ctx* h, double out[3]) {
  unsigned long long* r = (unsigned long long*)h->red.p;
  cudaError_t e = cudaMemsetAsync(r, 0, 6 * 8, h->stream);
  if (e != cudaSuccess) return e;
  dim3 grid(grid_for(h->geo.ncell, kThreads, 1024), 3);
  acc_sum_kernel<<<grid, kThreads, 0, h->stream>>>((const long long*)h->acc.p, h->geo.ncell, r);
  h->launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  unsigned long long hb[6];
  e = cudaMemcpyAsync(hb, r, 48, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  double inv = std::ldexp(1.0, -h->acc_E);
  for (int q = 0; q < 3; ++q) out[q] = i128_to_f64(hb[2 * q], (long long)hb[2 * q + 1]) * inv;
  return cudaSuccess;
}

cudaError_t launch_particle_sums(st_ctx* h, double out[4]) {
  const int blocks = 1024;
  const double pi = 3.14159265358979323846;
  double mcoef = h->mult * h->rho_p * pi / 6.0;
  double* part = (double*)h->red.p;  // blocks * 4 doubles = 32 KB
  F64State sf{};
  MixedState sm{};
  if (h->prec == ST_FP64) {
    sf = carve_f64(h->state.p, h->cap);
    particle_sums_kernel<ST_FP64><<<blocks, kThreads, 0, h->stream>>>(sf, sm, h->np, mcoef, part);
  } else if (h->prec == ST_MIXED_F32) {
    sm = carve_mixed(h->state.p, h->cap, false);
    particle_sums_kernel<ST_MIXED_F32><<<blocks, kThreads, 0, h->stream>>>(sf, sm, h->np, mcoef, part);
  } else {
    sm = carve_mixed(h->state.p, h->cap, true);
    particle_sums_kernel<ST_MIXED_BF16V><<<blocks, kThreads, 0, h->stream>>>(sf, sm, h->np, mcoef, part);
  }
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  std::vector<double> hp(blocks * 4);
  e = cudaMemcpyAsync(hp.data(), part, blocks * 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 4; ++k) out[k] = 0.0;
  for (int b = 0; b < blocks; ++b)
    for (int k = 0; k < 4; ++k) out[k] += hp[b * 4 + k];
  return cudaSuccess;
}

cudaError_t launch_gen(st_ctx* h, uint64_t seed, int64_t first, int64_t count, const double L[3], double vmax,
                       const double* qtable, int nq, double* xyz, double* vel, double* d, uint32_t* ids) {
  unsigned long long key = mix64_host((unsigned long long)seed ^ 0x5DEECE66Dull);
  int qbits = 0;
  while ((1 << qbits) < nq) ++qbits;
  gen_kernel<<<grid_for(count, kThreads, 152 * 64), kThreads, 0, h->stream>>>(key, first, count, L[0], L[1], L[2],
                                                                             vmax, qtable, qbits, xyz, vel, d, ids);
  h->launches += 1;
  return cudaGetLastError();
}

// Arithmetic-rate probes: eight (FP64) or sixteen (FP32) independent FMA chains per thread, no
// memory traffic in the loop; the result is stored only if it equals an impossible value.
__global__ void fma64_probe_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-9 + k * 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += x[k];
  if (t == 12345.0) out[0] = t;
}
__global__ void fma32_probe_kernel(float* out, int iters, float a, float b) {
  float x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = threadIdx.x * 1e-6f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = fmaf(x[k], a, b);
  }
  float t = 0.0f;
#pragma unroll
  for (int k = 0; k < 16; ++k) t += x[k];
  if (t == 12345.0f) out[0] = t;
}

cudaError_t probe_fma_rates(st_ctx* h, double* fp64_gflops, double* fp32_gflops) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev);
  if (sms <= 0) sms = 152;
  const int blocks = sms * 8, threads = 256;
  Buf tmp;
  if (dev_alloc(h, tmp, 16) != ST_OK) return cudaErrorMemoryAllocation;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  const int it64 = 4000, it32 = 20000;
  if (e == cudaSuccess) {
    fma64_probe_kernel<<<blocks, threads, 0, h->stream>>>((double*)tmp.p, 50, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(e0, h->stream);
    fma64_probe_kernel<<<blocks, threads, 0, h->stream>>>((double*)tmp.p, it64, 0.999999, 1e-7);
    cudaEventRecord(e1, h->stream);
    e = cudaEventSynchronize(e1);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *fp64_gflops = 2.0 * 8 * (double)it64 * blocks * threads / (ms * 1e-3) / 1e9;
  if (e == cudaSuccess) {
    fma32_probe_kernel<<<blocks, threads, 0, h->stream>>>((float*)tmp.p, 50, 0.999999f, 1e-7f);
    cudaEventRecord(e0, h->stream);
    fma32_probe_kernel<<<blocks, threads, 0, h->stream>>>((float*)tmp.p, it32, 0.999999f, 1e-7f);
    cudaEventRecord(e1, h->stream);
    e = cudaEventSynchronize(e1);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *fp32_gflops = 2.0 * 16 * (double)it32 * blocks * threads / (ms * 1e-3) / 1e9;
  h->launches += 4;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(h, tmp);
  return e;
}

}  // namespace st
