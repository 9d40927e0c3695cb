// Asynchronous two-way coupling on one GPU (Sec. 2.3) with the extrapolator-corrector estimate of
// the Lagrangian source (Sec. 2.4, Eqs. 12-14).
//
// A coupling interval is K particle steps in a frozen fluid field u^n.  The next field
//   u* = u^n + S_est^n / (rho_f V),   then `sweeps` Jacobi sweeps of (I - nu dtc Lap) u = u*
// (7-point periodic Laplacian, dtc = K dt, starting from u*), where
//   S_est^n = S^{n-1} - S_ext^{n-1} + S_ext^n
// uses only the sources of earlier intervals (zero, constant or linear extrapolation of S^m from
// S^{m-1}, S^{m-2}), so it is computed before the interval's particle steps, in the same stream:
// on one GPU the persistent step kernel needs whole SMs, and fluid kernels running beside it cost
// it far more time than they take on their own.  At the end of the interval the particles' source
// S^n moves from the exact
// accumulator into a ring of the last four intervals' sources (FP64), the fields are swapped,
// and the next interval begins.  Jacobi sweeps are averages with positive weights, so they keep
// sum_c u_c (the fluid momentum) and never raise max |u|; max |u| of each new field is read back
// for the next interval's fixed-point exponent.
#include <algorithm>
#include <cmath>

#include "st_common.cuh"

namespace st {
namespace {

constexpr int kCoupleThreads = 256;

int cgrid(int64_t n) {
  int64_t b = (n + kCoupleThreads - 1) / kCoupleThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// S_ext^m from the two sources before it: 0 zero, 1 constant, 2 linear
__device__ __forceinline__ double extrapolate(int extrap, const double* p1, const double* p2, int64_t i) {
  const double a = p1 ? p1[i] : 0.0, b = p2 ? p2[i] : 0.0;
  return extrap == 1 ? a : extrap == 2 ? 2.0 * a - b : 0.0;
}

// est = S^{n-1} - S_ext^{n-1} + S_ext^n   (s1, s2, s3 = S^{n-1}, S^{n-2}, S^{n-3}, NULL if none)
__global__ void ecm_kernel(int extrap, const double* __restrict__ s1, const double* __restrict__ s2,
                           const double* __restrict__ s3, double* __restrict__ est, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const double last = s1 ? s1[i] : 0.0;
    est[i] = last - extrapolate(extrap, s2, s3, i) + extrapolate(extrap, s1, s2, i);
  }
}

// sources given out but not yet received by the fluid: S^{N-1} - S_ext^{N-1}, plus what the
// accumulator holds now (acc, FP64 [3][ncell], may be NULL)
__global__ void pending_kernel(int extrap, const double* __restrict__ s1, const double* __restrict__ s2,
                               const double* __restrict__ s3, const double* __restrict__ acc,
                               double* __restrict__ out, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const double last = s1 ? s1[i] : 0.0;
    out[i] = last - extrapolate(extrap, s2, s3, i) + (acc ? acc[i] : 0.0);
  }
}

// component access for the two field types
__device__ __forceinline__ double comp(const D4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : v.z; }
__device__ __forceinline__ float comp(const float4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : v.z; }
__device__ __forceinline__ D4 make3(double a, double b, double c, const D4*) { return D4{a, b, c, 0.0}; }
__device__ __forceinline__ float4 make3(float a, float b, float c, const float4*) { return make_float4(a, b, c, 0.0f); }

// u* = u + est / (rho_f V), in the field's precision
template <typename V, typename R>
__global__ void source_add_kernel(const V* __restrict__ u, const double* __restrict__ est, int64_t ncell,
                                  double inv_mass, V* __restrict__ ustar) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const V a = u[c];
    ustar[c] = make3(comp(a, 0) + (R)(est[c] * inv_mass), comp(a, 1) + (R)(est[ncell + c] * inv_mass),
                     comp(a, 2) + (R)(est[2 * ncell + c] * inv_mass), (const V*)nullptr);
  }
}

// one Jacobi sweep: out = (u* + sum_q lam_q (in(-q) + in(+q))) / (1 + 2 sum lam), periodic; one
// thread per cell of a row, rows on grid y (j) and z (k): no integer division
template <typename V, typename R>
__global__ void jacobi_kernel(const V* __restrict__ ustar, const V* __restrict__ in, V* __restrict__ out, int nx,
                              int ny, int nz, R lx, R ly, R lz, R inv_den) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= nx) return;
  const int64_t row = (int64_t)nx * (j + (int64_t)ny * k);
  const int64_t c = row + i;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const int64_t xm = row + (i > 0 ? i - 1 : nx - 1), xp = row + (i < nx - 1 ? i + 1 : 0);
  const int64_t ym = j > 0 ? c - sy : c + (int64_t)(ny - 1) * sy, yp = j < ny - 1 ? c + sy : c - (int64_t)(ny - 1) * sy;
  const int64_t zm = k > 0 ? c - sz : c + (int64_t)(nz - 1) * sz, zp = k < nz - 1 ? c + sz : c - (int64_t)(nz - 1) * sz;
  const V s = ustar[c], a = in[xm], b = in[xp], e = in[ym], f = in[yp], g = in[zm], hh = in[zp];
  R r[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    R acc = comp(s, q);
    acc = acc + lx * (comp(a, q) + comp(b, q));
    acc = acc + ly * (comp(e, q) + comp(f, q));
    acc = acc + lz * (comp(g, q) + comp(hh, q));
    r[q] = acc * inv_den;
  }
  out[c] = make3(r[0], r[1], r[2], (const V*)nullptr);
}

// padded FP32 field (P ghost layers, periodic) from the unpadded one; grid y, z = padded rows
__global__ void pad_kernel(const float4* __restrict__ u, float4* __restrict__ out, int nx, int ny, int nz, int P) {
  const int px = nx + 2 * P, py = ny + 2 * P;
  const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y, c = blockIdx.z;
  if (a >= px) return;
  int i = a - P, j = b - P, k = c - P;
  if (i < 0 || i >= nx) i = ((i % nx) + nx) % nx;  // ghost layers (the grid may be thinner than P)
  if (j < 0 || j >= ny) j = ((j % ny) + ny) % ny;
  if (k < 0 || k >= nz) k = ((k % nz) + nz) % nz;
  out[a + (int64_t)px * (b + (int64_t)py * c)] = u[i + (int64_t)nx * (j + (int64_t)ny * k)];
}

// the interior of the padded field; grid y, z = rows
__global__ void unpad_kernel(const float4* __restrict__ in, float4* __restrict__ u, int nx, int ny, int nz, int P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= nx) return;
  const int64_t px = nx + 2 * P, pxy = px * (ny + 2 * P);
  u[i + (int64_t)nx * (j + (int64_t)ny * k)] = in[(i + P) + px * (j + P) + pxy * (k + P)];
}

// max |component| over the field, as the bits of a non-negative double (ordered like the values)
template <typename V>
__global__ void field_maxabs_kernel(const V* __restrict__ u, int64_t ncell, unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const V a = u[c];
    m = fmax(m, fmax(fabs((double)comp(a, 0)), fmax(fabs((double)comp(a, 1)), fabs((double)comp(a, 2)))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// FP64 [ncell][3] copy of the field
template <typename V>
__global__ void field_out_kernel(const V* __restrict__ u, int64_t ncell, double* __restrict__ out) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const V a = u[c];
    out[3 * c] = (double)comp(a, 0);
    out[3 * c + 1] = (double)comp(a, 1);
    out[3 * c + 2] = (double)comp(a, 2);
  }
}

bool mixed(const st_ctx* h) { return h->prec != ST_FP64; }
size_t field_bytes(const st_ctx* h) { return (size_t)h->geo.ncell * (mixed(h) ? sizeof(float4) : sizeof(D4)); }

// buffers, stream and events of the coupling (allocated on first use)
st_status couple_resources(st_ctx* h) {
  const size_t fb = field_bytes(h), sb = (size_t)h->geo.ncell * 3 * sizeof(double);
  for (int k = 0; k < 4; ++k) {
    if (h->src_hist[k].bytes < sb) {
      ST_TRY(dev_alloc(h, h->src_hist[k], sb));
      ST_CUDA(h, cudaMemsetAsync(h->src_hist[k].p, 0, sb, h->stream));
    }
  }
  if (h->src_est.bytes < sb) ST_TRY(dev_alloc(h, h->src_est, sb));
  Buf* fields[] = {&h->fl_next, &h->fl_star, &h->fl_tmp};
  for (Buf* b : fields)
    if (b->bytes < fb) ST_TRY(dev_alloc(h, *b, fb));
  if (mixed(h)) {
    if (h->fl_cur.bytes < fb) ST_TRY(dev_alloc(h, h->fl_cur, fb));
    if (h->fluid_pad_next.bytes < h->fluid_pad.bytes) ST_TRY(dev_alloc(h, h->fluid_pad_next, h->fluid_pad.bytes));
  }
  if (h->umax_dev.bytes < 8) ST_TRY(dev_alloc(h, h->umax_dev, 8));
  if (!h->umax_host) ST_CUDA(h, cudaMallocHost((void**)&h->umax_host, sizeof(double)));
  if (!h->ev_fluid) ST_CUDA(h, cudaEventCreateWithFlags(&h->ev_fluid, cudaEventDisableTiming));
  return ST_OK;
}

// the current field as an unpadded array: FP64 handles keep it in `fluid`, mixed ones in fl_cur
// (extracted from the padded field on first use after st_set_fluid)
void* current_field(st_ctx* h) {
  if (!mixed(h)) return h->fluid.p;
  if (!h->fl_valid) {
    const Geometry& G = h->geo;
    const dim3 grid((G.n[0] + 127) / 128, G.n[1], G.n[2]);
    unpad_kernel<<<grid, 128, 0, h->stream>>>((const float4*)h->fluid_pad.p, (float4*)h->fl_cur.p, G.n[0], G.n[1],
                                              G.n[2], kFluidPad);
    h->launches += 1;
    h->fl_valid = true;
  }
  return h->fl_cur.p;
}

const double* hist_slot(const st_ctx* h, int64_t interval) {
  return interval >= 0 && interval < h->couple_done ? (const double*)h->src_hist[interval % 4].p : nullptr;
}

// fluid update of the current interval, on the handle's stream: fl_next = F(current, estimate)
template <typename V, typename R>
cudaError_t launch_fluid_update(st_ctx* h, const V* cur, double dt) {
  const Geometry& G = h->geo;
  const int64_t nc = G.ncell, m = 3 * nc;
  cudaStream_t s = h->stream;
  const int64_t n = h->couple_done;
  ecm_kernel<<<cgrid(m), kCoupleThreads, 0, s>>>(h->extrap, hist_slot(h, n - 1), hist_slot(h, n - 2),
                                                 hist_slot(h, n - 3), (double*)h->src_est.p, m);
  const double V_cell = G.h[0] * G.h[1] * G.h[2];
  source_add_kernel<V, R><<<cgrid(nc), kCoupleThreads, 0, s>>>(cur, (const double*)h->src_est.p, nc,
                                                               1.0 / (h->rho_f * V_cell), (V*)h->fl_star.p);
  const double dtc = (double)h->couple_K * dt;
  double lam[3], lsum = 0.0;
  for (int q = 0; q < 3; ++q) {
    lam[q] = h->nu * dtc / (G.h[q] * G.h[q]);
    lsum += lam[q];
  }
  const R inv_den = (R)(1.0 / (1.0 + 2.0 * lsum));
  int launches = 2;
  if (h->sweeps == 0) {
    cudaMemcpyAsync(h->fl_next.p, h->fl_star.p, field_bytes(h), cudaMemcpyDeviceToDevice, s);
  } else {
    // ping-pong between fl_tmp and fl_next so that the last sweep writes fl_next
    const V* in = (const V*)h->fl_star.p;
    for (int k = 0; k < h->sweeps; ++k) {
      V* out = ((h->sweeps - 1 - k) % 2 == 0) ? (V*)h->fl_next.p : (V*)h->fl_tmp.p;
      const dim3 grid((G.n[0] + 127) / 128, G.n[1], G.n[2]);
      jacobi_kernel<V, R><<<grid, 128, 0, s>>>((const V*)h->fl_star.p, in, out, G.n[0], G.n[1], G.n[2], (R)lam[0],
                                                (R)lam[1], (R)lam[2], inv_den);
      in = out;
      ++launches;
    }
  }
  if (mixed(h)) {
    const dim3 grid((G.n[0] + 2 * kFluidPad + 127) / 128, G.n[1] + 2 * kFluidPad, G.n[2] + 2 * kFluidPad);
    pad_kernel<<<grid, 128, 0, s>>>((const float4*)h->fl_next.p, (float4*)h->fluid_pad_next.p, G.n[0], G.n[1],
                                    G.n[2], kFluidPad);
    ++launches;
  }
  cudaMemsetAsync(h->umax_dev.p, 0, 8, s);
  field_maxabs_kernel<V><<<cgrid(nc), kCoupleThreads, 0, s>>>((const V*)h->fl_next.p, nc,
                                                              (unsigned long long*)h->umax_dev.p);
  cudaMemcpyAsync(h->umax_host, h->umax_dev.p, sizeof(double), cudaMemcpyDeviceToHost, s);
  h->launches += launches + 1;
  return cudaGetLastError();
}

}  // namespace
}  // namespace st

using namespace st;

st_status st_couple_params(st_handle h, double rho_f, double nu, int sweeps, int steps_per_interval,
                           int extrapolator) {
  if (!h) return ST_ERR_INVALID_ARG;
  if (!std::isfinite(rho_f) || !std::isfinite(nu)) return set_error(h, ST_ERR_NONFINITE, "non-finite parameter");
  if (!(rho_f > 0) || nu < 0 || sweeps < 0 || steps_per_interval < 1 || extrapolator < 0 || extrapolator > 2)
    return set_error(h, ST_ERR_INVALID_ARG,
                     "rho_f > 0, nu >= 0, sweeps >= 0, steps_per_interval >= 1, extrapolator in 0..2");
  h->rho_f = rho_f;
  h->nu = nu;
  h->sweeps = sweeps;
  h->couple_K = steps_per_interval;
  h->extrap = extrapolator;
  return ST_OK;
}

st_status st_couple_run(st_handle h, int nintervals, double dt) {
  if (!h) return ST_ERR_INVALID_ARG;
  if (nintervals < 0) return set_error(h, ST_ERR_INVALID_ARG, "nintervals < 0");
  if (!std::isfinite(dt)) return set_error(h, ST_ERR_NONFINITE, "dt is not finite");
  if (!(dt > 0)) return set_error(h, ST_ERR_INVALID_ARG, "dt must be > 0");
  if (nintervals == 0) return ST_OK;
  ST_TRY(couple_resources(h));
  for (int it = 0; it < nintervals; ++it) {
    void* cur = current_field(h);
    // the next field from the current one and the sources of earlier intervals (the previous
    // interval's source is already in the ring); the particles then read the current field only
    timer_begin(h, ST_TIMER_FLUID, h->stream);
    cudaError_t e = mixed(h) ? launch_fluid_update<float4, float>(h, (const float4*)cur, dt)
                             : launch_fluid_update<D4, double>(h, (const D4*)cur, dt);
    timer_end(h, ST_TIMER_FLUID, h->stream);
    ST_TRY(cuda_check(h, e, "fluid update"));
    ST_CUDA(h, cudaEventRecord(h->ev_fluid, h->stream));
    // the particles of this interval in the current field
    ST_TRY(run_steps(h, h->couple_K, dt));
    // their source moves into the ring and the accumulator starts empty
    double* slot = (double*)h->src_hist[h->couple_done % 4].p;
    ST_TRY(cuda_check(h, launch_acc_to_f64(h, slot, h->acc_E), "archive source"));
    ST_CUDA(h, cudaMemsetAsync(h->acc.p, 0, h->acc.bytes, h->stream));
    ST_CUDA(h, reset_acc_counter(h));
    h->acc_empty = true;
    h->acc_load = 0.0;
    // the next interval runs in the new field (its max |u|, read back, sets the next exponent; the
    // fluid update finished ahead of this interval's steps, so the wait does not drain the stream)
    ST_CUDA(h, cudaEventSynchronize(h->ev_fluid));
    h->umax = *h->umax_host;
    if (mixed(h)) {
      std::swap(h->fl_cur, h->fl_next);
      std::swap(h->fluid_pad, h->fluid_pad_next);
    } else {
      std::swap(h->fluid, h->fl_next);
    }
    h->couple_done += 1;
    h->adj_ready = false;
  }
  return ST_OK;
}

st_status st_get_fluid(st_handle h, double* out, int on_device) {
  if (!h) return ST_ERR_INVALID_ARG;
  if (!out) return set_error(h, ST_ERR_INVALID_ARG, "out is NULL");
  const int64_t nc = h->geo.ncell;
  const size_t bytes = (size_t)nc * 3 * sizeof(double);
  if (mixed(h) && h->fl_cur.bytes < field_bytes(h)) ST_TRY(dev_alloc(h, h->fl_cur, field_bytes(h)));
  Buf tmp;
  double* dst = out;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, bytes));
    dst = (double*)tmp.p;
  }
  void* cur = current_field(h);
  if (mixed(h))
    field_out_kernel<float4><<<cgrid(nc), kCoupleThreads, 0, h->stream>>>((const float4*)cur, nc, dst);
  else
    field_out_kernel<D4><<<cgrid(nc), kCoupleThreads, 0, h->stream>>>((const D4*)cur, nc, dst);
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  return cuda_check(h, e, "get fluid");
}

st_status st_get_pending_sources(st_handle h, double* out, int on_device) {
  if (!h) return ST_ERR_INVALID_ARG;
  if (!out) return set_error(h, ST_ERR_INVALID_ARG, "out is NULL");
  const int64_t m = 3 * h->geo.ncell;
  const size_t bytes = (size_t)m * sizeof(double);
  Buf tmp, accd;
  double* dst = out;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, bytes));
    dst = (double*)tmp.p;
  }
  st_status s = dev_alloc(h, accd, bytes);
  if (s != ST_OK) {
    dev_free(h, tmp);
    return s;
  }
  cudaError_t e = launch_acc_to_f64(h, (double*)accd.p, h->acc_E);
  const int64_t n = h->couple_done;
  if (e == cudaSuccess) {
    pending_kernel<<<cgrid(m), kCoupleThreads, 0, h->stream>>>(h->extrap, hist_slot(h, n - 1), hist_slot(h, n - 2),
                                                               hist_slot(h, n - 3), (const double*)accd.p, dst, m);
    h->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  dev_free(h, accd);
  return cuda_check(h, e, "get pending sources");
}
