// C ABI of the Lagrangian step: handle management, argument checks, memory,
// and the per-call orchestration of the kernels on the caller's stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "st_common.cuh"

namespace st {

st_status set_error(st_ctx* h, st_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

st_status cuda_check(st_ctx* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return ST_OK;
  return set_error(h, ST_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

st_status dev_alloc(st_ctx* h, Buf& b, size_t bytes) {
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) return ST_OK;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->have_alloc) {
    p = h->alloc.alloc(bytes, h->alloc.user);
    if (!p) return set_error(h, ST_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(h, ST_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
  }
  b.p = p;
  b.bytes = bytes;
  return ST_OK;
}

void dev_free(st_ctx* h, Buf& b) {
  if (!b.p) return;
  if (h->have_alloc) {
    h->alloc.free(b.p, h->alloc.user);
  } else {
    cudaFree(b.p);
  }
  b.p = nullptr;
  b.bytes = 0;
}

st_status ensure(st_ctx* h, Buf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return ST_OK;
  dev_free(h, b);
  return dev_alloc(h, b, bytes);
}

}  // namespace st

using namespace st;



static bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// Report (and clear) device-side error flags raised by bounded waits that gave up.
st_status st::check_flags(st_ctx* h) {
  int f = 0;
  cudaError_t e = cudaMemcpyAsync(&f, h->flags.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_check(h, e, "read error flags");
  if (f != 0) {
    cudaMemsetAsync(h->flags.p, 0, sizeof(int), h->stream);
    return set_error(h, ST_ERR_TIMEOUT, "a bounded device-side wait gave up (flags " + std::to_string(f) + ")");
  }
  return ST_OK;
}

// every call below first reads the result of a pending asynchronous field upload (st_set_fluid_async)
static st_status check_handle(st_handle h) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  cudaError_t e = cudaSetDevice(h->dev);
  ST_TRY(cuda_check(h, e, "cudaSetDevice"));
  return settle_fluid(h);
}

extern "C" {

st_status st_create_grid(int nx, int ny, int nz, double Lx, double Ly, double Lz, int chunk_edge,
                         int precision, const st_allocator* allocator, void* stream, st_handle* out) {
  if (!out) return ST_ERR_INVALID_ARG;
  *out = nullptr;
  int n[3] = {nx, ny, nz};
  double L[3] = {Lx, Ly, Lz};
  for (int q = 0; q < 3; ++q) {
    if (n[q] < 1 || n[q] > kMaxDim) return ST_ERR_INVALID_ARG;
    if (!std::isfinite(L[q])) return ST_ERR_NONFINITE;
    if (!(L[q] > 0.0)) return ST_ERR_INVALID_ARG;
  }
  if (chunk_edge < 1 || chunk_edge > 32 || (chunk_edge & (chunk_edge - 1))) return ST_ERR_INVALID_ARG;
  if (precision != ST_FP64 && precision != ST_MIXED_F32 && precision != ST_MIXED_BF16V) return ST_ERR_INVALID_ARG;
  if (allocator && (!allocator->alloc || !allocator->free)) return ST_ERR_INVALID_ARG;
  st_ctx* h = new (std::nothrow) st_ctx();
  if (!h) return ST_ERR_OOM;
  if (cudaGetDevice(&h->dev) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return ST_ERR_CUDA;
  }
  Geometry& G = h->geo;
  for (int q = 0; q < 3; ++q) {
    G.n[q] = n[q];
    G.L[q] = L[q];
    G.h[q] = L[q] / (double)n[q];
    G.inv_h[q] = (double)n[q] / L[q];
  }
  G.B = chunk_edge;
  G.ncell = (int64_t)nx * ny * nz;
  h->prec = precision;
  if (allocator) {
    h->alloc = *allocator;
    h->have_alloc = true;
  }
  h->stream = (cudaStream_t)stream;
  int logB = 0;
  while ((1 << logB) < chunk_edge) ++logB;
  int nc[3];
  for (int q = 0; q < 3; ++q) nc[q] = (n[q] + chunk_edge - 1) / chunk_edge;
  uint64_t nkeys = (uint64_t)nc[0] * nc[1] * nc[2] << (3 * logB);
  h->nkeys = (uint32_t)nkeys;
  int bits = 0;
  while ((1ull << bits) < nkeys) ++bits;
  h->key_bits = bits;
  st_status s = dev_alloc(h, h->acc, (size_t)G.ncell * 3 * kAccWords * sizeof(long long));
  if (s == ST_OK) s = dev_alloc(h, h->red, 64 * 1024);
  if (s == ST_OK) s = cuda_check(h, cudaMemsetAsync(h->acc.p, 0, h->acc.bytes, h->stream), "memset acc");
  if (precision == ST_FP64) {
    if (s == ST_OK) s = dev_alloc(h, h->fluid, (size_t)G.ncell * 4 * sizeof(double));
    if (s == ST_OK) s = cuda_check(h, cudaMemsetAsync(h->fluid.p, 0, h->fluid.bytes, h->stream), "memset fluid");
  } else {
    size_t padded = (size_t)(nx + 2 * kFluidPad) * (ny + 2 * kFluidPad) * (nz + 2 * kFluidPad);
    if (s == ST_OK) s = dev_alloc(h, h->fluid_pad, padded * 4 * sizeof(float));
    if (s == ST_OK)
      s = cuda_check(h, cudaMemsetAsync(h->fluid_pad.p, 0, h->fluid_pad.bytes, h->stream), "memset fluid");
  }
  if (s == ST_OK) s = dev_alloc(h, h->flags, 256);
  if (s == ST_OK) s = cuda_check(h, cudaMemsetAsync(h->flags.p, 0, 256, h->stream), "memset flags");
  if (s != ST_OK) {
    st_destroy(h);
    return s;
  }
  h->fluid_set = true;  // at rest until st_set_fluid
  h->umax = 0.0;
  *out = h;
  return ST_OK;
}

void st_destroy(st_handle h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  cudaStreamSynchronize(h->stream);
  chunk_store_free(h);  // its slot buffers first: the handle's own are freed below
  xfer_free(h);
  Buf* bufs[] = {&h->fluid, &h->fluid_pad, &h->flags, &h->ckpt, &h->state, &h->state_alt, &h->ids, &h->ids_alt,
                 &h->keys[0], &h->keys[1], &h->vals[0], &h->vals[1], &h->hist, &h->scan_aux, &h->cell_start, &h->lsort_aux,
                 &h->acc, &h->red, &h->src_hist[0], &h->src_hist[1], &h->src_hist[2], &h->src_hist[3],
                 &h->src_est, &h->fl_cur, &h->fl_next, &h->fl_star, &h->fl_tmp, &h->fluid_pad_next, &h->umax_dev,
                 &h->temp, &h->temp_alt, &h->thermo, &h->acc_micro};
  for (Buf* b : bufs) dev_free(h, *b);
  if (h->umax_host) cudaFreeHost(h->umax_host);
  if (h->ev_fluid) cudaEventDestroy(h->ev_fluid);
  for (int k = 0; k < ST_TIMER_COUNT; ++k)
    for (auto& pr : h->ev_pending[k]) {
      cudaEventDestroy(pr.first);
      if (pr.second) cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

const char* st_last_error(st_handle h) { return h ? h->err.c_str() : "null handle"; }

st_status st_set_stream(st_handle h, void* stream) {
  ST_TRY(check_handle(h));
  h->stream = (cudaStream_t)stream;
  return ST_OK;
}

st_status st_synchronize(st_handle h) {
  ST_TRY(check_handle(h));
  ST_CUDA(h, cudaStreamSynchronize(h->stream));
  ST_CUDA(h, xfer_sync(h));
  return check_flags(h);
}

st_status st_set_params(st_handle h, double rho_p, double mu, const double g[3], double drag_scale,
                        double multiplicity, int reorder_every) {
  ST_TRY(check_handle(h));
  if (!g) return set_error(h, ST_ERR_INVALID_ARG, "g is NULL");
  if (!std::isfinite(rho_p) || !std::isfinite(mu) || !finite3(g) || !std::isfinite(drag_scale) ||
      !std::isfinite(multiplicity))
    return set_error(h, ST_ERR_NONFINITE, "non-finite parameter");
  if (!(rho_p > 0) || !(mu > 0) || !(drag_scale > 0) || !(multiplicity > 0) || reorder_every < 0)
    return set_error(h, ST_ERR_INVALID_ARG, "rho_p, mu, drag_scale, multiplicity must be > 0, reorder_every >= 0");
  h->rho_p = rho_p;
  h->mu = mu;
  for (int q = 0; q < 3; ++q) h->g[q] = g[q];
  h->alpha = drag_scale;
  h->mult = multiplicity;
  h->reorder_every = reorder_every;
  h->adj_ready = false;
  return ST_OK;
}

extern "C++" {
namespace st {
static cudaEvent_t timer_event(st_ctx* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
void timer_begin(st_ctx* h, int k, cudaStream_t s) {
  if (!h->timing) return;
  cudaEvent_t e = timer_event(h);
  if (!e) return;
  cudaEventRecord(e, s);
  h->ev_pending[k].push_back({e, nullptr});
}
void timer_end(st_ctx* h, int k, cudaStream_t s) {
  if (!h->timing || h->ev_pending[k].empty() || h->ev_pending[k].back().second) return;
  cudaEvent_t e = timer_event(h);
  if (!e) return;
  cudaEventRecord(e, s);
  h->ev_pending[k].back().second = e;
}
static cudaError_t timers_fold(st_ctx* h) {
  for (int k = 0; k < ST_TIMER_COUNT; ++k) {
    for (auto& pr : h->ev_pending[k]) {
      if (pr.second) {
        cudaError_t e = cudaEventSynchronize(pr.second);
        if (e != cudaSuccess) return e;
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess) return e;
        h->timer_ms[k] += ms;
        h->timer_count[k] += 1;
        h->ev_pool.push_back(pr.second);
      }
      h->ev_pool.push_back(pr.first);
    }
    h->ev_pending[k].clear();
  }
  return cudaSuccess;
}
}  // namespace st
}  // extern "C++"

st_status st_timers_enable(st_handle h, int on) {
  ST_TRY(check_handle(h));
  ST_TRY(cuda_check(h, timers_fold(h), "timers"));
  for (int k = 0; k < ST_TIMER_COUNT; ++k) {
    h->timer_ms[k] = 0.0;
    h->timer_count[k] = 0;
  }
  h->timing = on != 0;
  return ST_OK;
}

st_status st_timers_read(st_handle h, double* ms, int64_t* launches, int reset) {
  ST_TRY(check_handle(h));
  if (!ms || !launches) return set_error(h, ST_ERR_INVALID_ARG, "ms and launches are required");
  ST_TRY(cuda_check(h, timers_fold(h), "timers"));
  for (int k = 0; k < ST_TIMER_COUNT; ++k) {
    ms[k] = h->timer_ms[k];
    launches[k] = h->timer_count[k];
    if (reset) {
      h->timer_ms[k] = 0.0;
      h->timer_count[k] = 0;
    }
  }
  return ST_OK;
}

st_status st_set_physics(st_handle h, int gather, int integrator, int drag, int deposit, double rho_f) {
  ST_TRY(check_handle(h));
  if (!std::isfinite(rho_f)) return set_error(h, ST_ERR_NONFINITE, "rho_f is not finite");
  if (gather < 0 || gather > 1 || integrator < 0 || integrator > 1 || drag < 0 || drag > 1 || deposit < 0 ||
      deposit > 1)
    return set_error(h, ST_ERR_INVALID_ARG, "unknown gather, integrator, drag or deposit");
  if (!(rho_f > 0)) return set_error(h, ST_ERR_INVALID_ARG, "rho_f must be > 0");
  h->phys_gather = gather;
  h->phys_integrator = integrator;
  h->phys_drag = drag;
  h->phys_deposit = deposit;
  h->rho_f_drag = rho_f;
  h->adj_ready = false;
  return ST_OK;
}

st_status st_set_fluid(st_handle h, const void* u, int dtype, int on_device) {
  ST_TRY(check_handle(h));
  if (!u) return set_error(h, ST_ERR_INVALID_ARG, "u is NULL");
  if (dtype != ST_DTYPE_F32 && dtype != ST_DTYPE_F64) return set_error(h, ST_ERR_INVALID_ARG, "bad dtype");
  size_t esz = dtype == ST_DTYPE_F64 ? 8 : 4;
  size_t bytes = (size_t)h->geo.ncell * 3 * esz;
  const void* src = u;
  Buf tmp;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, bytes));
    cudaError_t e = cudaMemcpyAsync(tmp.p, u, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      dev_free(h, tmp);
      return cuda_check(h, e, "copy fluid");
    }
    src = tmp.p;
  }
  double umax = 0.0;
  int nonfinite = 0;
  cudaError_t e = launch_maxabs(h, src, h->geo.ncell * 3, dtype, &umax, &nonfinite);
  if (e == cudaSuccess && !nonfinite) e = launch_fluid_pack(h, src, dtype);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  ST_TRY(cuda_check(h, e, "set fluid"));
  if (nonfinite) return set_error(h, ST_ERR_NONFINITE, "fluid field holds NaN or Inf");
  h->umax = umax;
  h->fluid_set = true;
  h->adj_ready = false;
  h->fl_valid = false;   // a coupled run starts from this field, with no source history
  h->couple_done = 0;
  return ST_OK;
}

static st_status grow(st_handle h, int64_t need) {
  if (need <= h->cap) return ST_OK;
  ST_TRY(materialize_state(h));
  int64_t cap = h->cap ? h->cap : 1024;
  while (cap < need) cap = cap + cap / 2 + 64;
  cap = (cap + 63) & ~int64_t(63);
  Buf ns, ni;
  // sized like the sort's spare buffer (room for 32-byte particle records on mixed handles): the
  // sort swaps the two, so either may be the one the step before a sort writes records into
  ST_TRY(dev_alloc(h, ns, state_alt_bytes(h->prec, cap)));
  st_status s = dev_alloc(h, ni, (size_t)cap * sizeof(uint32_t));
  if (s != ST_OK) {
    dev_free(h, ns);
    return s;
  }
  if (h->np > 0) {
    // copy each array of the old block to its place in the new one
    cudaError_t e = cudaSuccess;
    if (h->prec == ST_FP64) {
      for (int a = 0; a < 7 && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync((double*)ns.p + a * cap, (double*)h->state.p + a * h->cap, h->np * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->stream);
    } else {
      bool bf = h->prec == ST_MIXED_BF16V;
      MixedState o = carve_mixed(h->state.p, h->cap, bf), n = carve_mixed(ns.p, cap, bf);
      size_t vb = bf ? 2 : 4;
      e = cudaMemcpyAsync(n.cell, o.cell, h->np * 4, cudaMemcpyDeviceToDevice, h->stream);
      for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync(n.xi[q], o.xi[q], h->np * 4, cudaMemcpyDeviceToDevice, h->stream);
      for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync(n.v[q], o.v[q], h->np * vb, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(n.d, o.d, h->np * 4, cudaMemcpyDeviceToDevice, h->stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ni.p, h->ids.p, h->np * sizeof(uint32_t), cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      dev_free(h, ns);
      dev_free(h, ni);
      return cuda_check(h, e, "grow particle arrays");
    }
  }
  dev_free(h, h->state);
  dev_free(h, h->ids);
  dev_free(h, h->state_alt);
  dev_free(h, h->ids_alt);
  h->state = ns;
  h->ids = ni;
  h->cap = cap;
  return micro_grow(h);
}

st_status st_reserve(st_handle h, int64_t capacity) {
  ST_TRY(check_handle(h));
  if (capacity < 0 || capacity > (int64_t(1) << 34)) return set_error(h, ST_ERR_INVALID_ARG, "capacity out of range");
  // a handle with chunks keeps its buffers at the chunk capacity (they are the chunks' device slots)
  if (h->chunks) return set_error(h, ST_ERR_STATE, "the handle holds chunks");
  return grow(h, capacity);
}

st_status st_add_particles(st_handle h, int64_t n, const double* xyz, const double* vel, const double* d,
                           const uint32_t* ids, int on_device) {
  ST_TRY(check_handle(h));
  if (n < 0) return set_error(h, ST_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return ST_OK;
  if (!xyz || !d) return set_error(h, ST_ERR_INVALID_ARG, "xyz and d are required");
  if (h->chunks && !h->chunk_adding) return set_error(h, ST_ERR_STATE, "the handle holds chunks: st_chunks_add");
  if (h->np + n > (int64_t(1) << 34)) return set_error(h, ST_ERR_INVALID_ARG, "too many particles");
  ST_TRY(materialize_state(h));
  // stage host data on the device
  Buf tx, tv, td, ti;
  const double *dx = xyz, *dv = vel, *dd = d;
  const uint32_t* di = ids;
  auto cleanup = [&]() {
    dev_free(h, tx);
    dev_free(h, tv);
    dev_free(h, td);
    dev_free(h, ti);
  };
  if (!on_device) {
    st_status s = dev_alloc(h, tx, (size_t)n * 3 * 8);
    if (s == ST_OK && vel) s = dev_alloc(h, tv, (size_t)n * 3 * 8);
    if (s == ST_OK) s = dev_alloc(h, td, (size_t)n * 8);
    if (s == ST_OK && ids) s = dev_alloc(h, ti, (size_t)n * 4);
    cudaError_t e = cudaSuccess;
    if (s == ST_OK) e = cudaMemcpyAsync(tx.p, xyz, (size_t)n * 24, cudaMemcpyHostToDevice, h->stream);
    if (s == ST_OK && e == cudaSuccess && vel)
      e = cudaMemcpyAsync(tv.p, vel, (size_t)n * 24, cudaMemcpyHostToDevice, h->stream);
    if (s == ST_OK && e == cudaSuccess) e = cudaMemcpyAsync(td.p, d, (size_t)n * 8, cudaMemcpyHostToDevice, h->stream);
    if (s == ST_OK && e == cudaSuccess && ids)
      e = cudaMemcpyAsync(ti.p, ids, (size_t)n * 4, cudaMemcpyHostToDevice, h->stream);
    if (s == ST_OK) s = cuda_check(h, e, "copy particles");
    if (s != ST_OK) {
      cleanup();
      return s;
    }
    dx = (const double*)tx.p;
    dv = vel ? (const double*)tv.p : nullptr;
    dd = (const double*)td.p;
    di = ids ? (const uint32_t*)ti.p : nullptr;
  }
  double vmax = 0, dmax = 0, dmin = 0;
  int nonfinite = 0;
  cudaError_t e = launch_particle_scan(h, dx, dd, n, &vmax, &dmax, &dmin, &nonfinite);
  if (e == cudaSuccess && dv) {
    double vm = 0;
    int nf2 = 0;
    e = launch_maxabs(h, dv, n * 3, ST_DTYPE_F64, &vm, &nf2);
    vmax = vm;
    nonfinite |= nf2;
  }
  if (e != cudaSuccess) {
    cleanup();
    return cuda_check(h, e, "scan particles");
  }
  if (nonfinite) {
    cleanup();
    return set_error(h, ST_ERR_NONFINITE, "particle positions, velocities or diameters hold NaN or Inf");
  }
  if (!(dmin > 0.0)) {
    cleanup();
    return set_error(h, ST_ERR_INVALID_ARG, "diameters must be > 0");
  }
  st_status s = grow(h, h->np + n);
  if (s != ST_OK) {
    cleanup();
    return s;
  }
  e = launch_import(h, h->np, n, dx, dv, dd, di);
  // droplets added with microphysics on (or after it was on) start at its initial temperature
  if (e == cudaSuccess) e = launch_fill_temp(h, h->np, n, h->mi_Tinit);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cleanup();
  ST_TRY(cuda_check(h, e, "import particles"));
  h->np += n;
  h->dmax = std::max(h->dmax, dmax);
  h->vbound = std::max(h->vbound, vmax);
  h->sorted = false;
  h->adj_ready = false;
  return ST_OK;
}

st_status st_num_particles(st_handle h, int64_t* n) {
  ST_TRY(check_handle(h));
  if (!n) return set_error(h, ST_ERR_INVALID_ARG, "n is NULL");
  *n = h->np;
  return ST_OK;
}

st_status st_reorder(st_handle h) {
  ST_TRY(check_handle(h));
  timer_begin(h, ST_TIMER_SORT, h->stream);
  const st_status ss = sort_particles(h);
  timer_end(h, ST_TIMER_SORT, h->stream);
  ST_TRY(ss);
  h->adj_ready = false;
  h->sorted = true;
  h->steps_since_sort = 0;
  return ST_OK;
}

// Contributions one particle can make to one cell in one step: one, except that the cloud-in-cell
// stencil's two corners along an axis of a single cell are the same cell.
static double deposits_per_cell(const st_ctx* h) {
  if (h->phys_deposit != ST_DEPOSIT_CIC) return 1.0;
  double f = 1.0;
  for (int q = 0; q < 3; ++q) f *= h->geo.n[q] == 1 ? 2.0 : 1.0;
  return f;
}

// Choose the fixed-point exponent so that a committed run at its bound maps to
// at most 2^96 and the accumulated integer stays below 2^125.
static st_status prepare_accumulator(st_handle h, double dt, double adds_now, int* E_out) {
  const double pi = 3.14159265358979323846;
  double gn = std::sqrt(h->g[0] * h->g[0] + h->g[1] * h->g[1] + h->g[2] * h->g[2]);
  double tau_max = h->rho_p * h->dmax * h->dmax / (18.0 * h->mu);
  h->vbound = std::max(h->vbound, h->umax + gn * tau_max / h->alpha);
  double mmax = h->mult * h->rho_p * pi * h->dmax * h->dmax * h->dmax / 6.0;
  // |J| = m |v' - v - g dt| <= m (2 |v|max + |g| dt); with microphysics the mass change adds |m' - m| |v'|
  double jb = mmax * ((h->micro_on ? 3.0 : 2.0) * h->vbound + gn * dt) * 1.01 + 1e-300;
  double cb = jb * kMaxRun;
  int E = kAccBits - (int)std::ceil(std::log2(cb));
  if (!h->acc_empty && E < h->acc_E) {
    cudaError_t e = launch_rescale_acc(h, h->acc_E - E);
    ST_TRY(cuda_check(h, e, "rescale accumulator"));
    ST_TRY(cuda_check(h, reset_acc_counter(h), "reset accumulator counter"));
    h->acc_load = std::ldexp(h->acc_load, E - h->acc_E);
  }
  if (h->acc_empty || E < h->acc_E) h->acc_E = E;
  E = h->acc_E;
  // one step adds at most np * jb to any cell
  double add = (double)h->np * jb * std::ldexp(1.0, E) + 1.0;
  while (h->acc_load + add > 0x1p125) {
    cudaError_t e = launch_rescale_acc(h, 1);
    ST_TRY(cuda_check(h, e, "rescale accumulator"));
    ST_TRY(cuda_check(h, reset_acc_counter(h), "reset accumulator counter"));
    h->acc_E -= 1;
    E = h->acc_E;
    h->acc_load *= 0.5;
    add = (double)h->np * jb * std::ldexp(1.0, E) + 1.0;
  }
  h->acc_load += add;
  h->acc_empty = false;
  // each word takes at most one digit per contribution; a step adds at most one contribution per
  // particle to any cell, plus one per neighbouring unit's tile flush (at most 8)
  ST_TRY(cuda_check(h, launch_acc_maybe_normalize(h, deposits_per_cell(h) * (double)h->np + 8.0, adds_now),
                    "normalise accumulator"));
  *E_out = E;
  return ST_OK;
}

extern "C++" {
namespace st {
st_status run_steps(st_ctx* h, int nsteps, double dt) {
  ST_TRY(settle_fluid(h));
  if (nsteps < 0) return set_error(h, ST_ERR_INVALID_ARG, "nsteps < 0");
  if (!std::isfinite(dt)) return set_error(h, ST_ERR_NONFINITE, "dt is not finite");
  if (!(dt > 0)) return set_error(h, ST_ERR_INVALID_ARG, "dt must be > 0");
  if (!h->fluid_set) return set_error(h, ST_ERR_STATE, "no fluid field");
  if (h->micro_on && !h->thermo_set) return set_error(h, ST_ERR_STATE, "microphysics needs st_set_thermo first");
  if (h->micro_on && !default_physics(h))
    return set_error(h, ST_ERR_STATE, "microphysics runs with the default gather, integrator, drag and deposit only");
  const double pi = 3.14159265358979323846;
  for (int s = 0; s < nsteps; ++s) {
    if (h->np == 0) break;
    if (h->reorder_every > 0 && (!h->sorted || h->steps_since_sort >= h->reorder_every)) ST_TRY(st_reorder(h));
    // the sorted-step kernel adds one tile flush per covering unit (at most 8 per cell) and counts
    // its global commits itself; the other kernels may add one contribution per particle
    const bool tma = !h->micro_on && h->prec != ST_FP64 && h->sorted && tma_step_supported(h);
    // a sort is due before the next step: this step writes the state as records for its gather
    const bool records = tma && default_physics(h) && h->reorder_every > 0 &&
                         h->steps_since_sort + 1 >= h->reorder_every && h->state_alt.bytes >= (size_t)h->cap * 32;
    // a sort that deferred its payload gather: this step gathers, unless it is another kernel or
    // writes records itself (then the gather runs first)
    const bool gather = h->perm_pending && tma && default_physics(h) && !records;
    if (!gather) ST_TRY(materialize_state(h));
    if (h->micro_on) ST_TRY(micro_prepare_step(h, dt));
    int E = 0;
    ST_TRY(prepare_accumulator(h, dt, tma ? 8.0 : deposits_per_cell(h) * (double)h->np + 8.0, &E));
    StepParams p;
    p.dt = dt;
    p.ca = 18.0 * h->mu * h->alpha / h->rho_p;
    p.mcoef = h->mult * h->rho_p * pi / 6.0;
    for (int q = 0; q < 3; ++q) p.g[q] = h->g[q];
    p.E = E;
    p.scale = std::ldexp(1.0, E);
    p.ngp = h->phys_gather == ST_GATHER_NGP;
    p.semi = h->phys_integrator == ST_INTEGRATOR_SEMI_IMPLICIT;
    p.sn = h->phys_drag == ST_DRAG_SCHILLER_NAUMANN;
    p.cic = h->phys_deposit == ST_DEPOSIT_CIC;
    p.re_coef = h->rho_f_drag / h->mu;
    cudaError_t e;
    timer_begin(h, ST_TIMER_STEP, h->stream);
    if (h->micro_on) {
      // the step before a due sort leaves its output as records for the sort's gather
      const bool mrec = h->prec != ST_FP64 && h->reorder_every > 0 && h->steps_since_sort + 1 >= h->reorder_every &&
                        h->state_alt.bytes >= (size_t)h->cap * 32;
      e = launch_micro_step(h, p, mrec);
      if (e == cudaSuccess && mrec) h->records_pending = true;
    }
    else if (h->prec == ST_FP64)
      e = launch_step_f64(h, p);
    else if (tma) {
      e = launch_step_mixed_tma(h, p, records, gather);
      if (e == cudaSuccess && gather) gather_step_done(h);
      if (e == cudaSuccess && records) h->records_pending = true;
    }
    else
      e = launch_step_mixed(h, p);
    timer_end(h, ST_TIMER_STEP, h->stream);
    ST_TRY(cuda_check(h, e, "step kernel"));
    h->steps_since_sort += 1;
  }
  return ST_OK;
}
}  // namespace st
}  // extern "C++"

st_status st_step(st_handle h, int nsteps, double dt) {
  ST_TRY(check_handle(h));
  return run_steps(h, nsteps, dt);
}

st_status st_get_sources(st_handle h, double* out, int reset, int on_device) {
  ST_TRY(check_handle(h));
  if (!out) return set_error(h, ST_ERR_INVALID_ARG, "out is NULL");
  size_t bytes = (size_t)h->geo.ncell * 3 * sizeof(double);
  Buf tmp;
  double* dst = out;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, bytes));
    dst = (double*)tmp.p;
  }
  cudaError_t e = launch_acc_to_f64(h, dst, h->acc_E);
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(h->acc.p, 0, h->acc.bytes, h->stream);
  if (e == cudaSuccess && reset) e = reset_acc_counter(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  ST_TRY(cuda_check(h, e, "get sources"));
  ST_TRY(check_flags(h));
  if (reset) {
    h->acc_empty = true;
    h->acc_load = 0.0;
  }
  return ST_OK;
}

st_status st_get_sources_fixed(st_handle h, int64_t* words, int* E, int on_device) {
  ST_TRY(check_handle(h));
  if (!words || !E) return set_error(h, ST_ERR_INVALID_ARG, "words and E are required");
  // carries propagated in place (the value is unchanged), then the words copied out
  ST_TRY(cuda_check(h, launch_normalize_acc(h), "normalise sources"));
  cudaError_t e = cudaMemcpyAsync(words, h->acc.p, (size_t)h->geo.ncell * 3 * kAccWords * sizeof(long long),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  ST_TRY(cuda_check(h, e, "get fixed-point sources"));
  *E = h->acc_E;
  return check_flags(h);
}

st_status st_get_particles(st_handle h, int64_t first, int64_t count, double* xyz, double* vel, double* d,
                           uint32_t* ids, int on_device) {
  ST_TRY(check_handle(h));
  ST_TRY(materialize_state(h));
  if (first < 0 || count < 0 || first + count > h->np) return set_error(h, ST_ERR_INVALID_ARG, "range out of bounds");
  if (count == 0) return ST_OK;
  Buf tx, tv, td, ti;
  double *ox = xyz, *ov = vel, *od = d;
  uint32_t* oi = ids;
  st_status s = ST_OK;
  if (!on_device) {
    if (xyz) s = dev_alloc(h, tx, (size_t)count * 24);
    if (s == ST_OK && vel) s = dev_alloc(h, tv, (size_t)count * 24);
    if (s == ST_OK && d) s = dev_alloc(h, td, (size_t)count * 8);
    if (s == ST_OK && ids) s = dev_alloc(h, ti, (size_t)count * 4);
    ox = (double*)tx.p;
    ov = (double*)tv.p;
    od = (double*)td.p;
    oi = (uint32_t*)ti.p;
  }
  cudaError_t e = cudaSuccess;
  if (s == ST_OK) e = launch_export(h, first, count, ox, ov, od, oi, nullptr);
  if (s == ST_OK && !on_device) {
    if (e == cudaSuccess && xyz) e = cudaMemcpyAsync(xyz, ox, (size_t)count * 24, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && vel) e = cudaMemcpyAsync(vel, ov, (size_t)count * 24, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && d) e = cudaMemcpyAsync(d, od, (size_t)count * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && ids) e = cudaMemcpyAsync(ids, oi, (size_t)count * 4, cudaMemcpyDeviceToHost, h->stream);
  }
  if (s == ST_OK && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tx);
  dev_free(h, tv);
  dev_free(h, td);
  dev_free(h, ti);
  ST_TRY(s);
  return cuda_check(h, e, "get particles");
}

st_status st_get_cells(st_handle h, int64_t first, int64_t count, int32_t* cells, int on_device) {
  ST_TRY(check_handle(h));
  ST_TRY(materialize_state(h));
  if (!cells) return set_error(h, ST_ERR_INVALID_ARG, "cells is NULL");
  if (first < 0 || count < 0 || first + count > h->np) return set_error(h, ST_ERR_INVALID_ARG, "range out of bounds");
  if (count == 0) return ST_OK;
  Buf tc;
  int32_t* oc = cells;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tc, (size_t)count * 4));
    oc = (int32_t*)tc.p;
  }
  cudaError_t e = launch_export(h, first, count, nullptr, nullptr, nullptr, nullptr, oc);
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(cells, oc, (size_t)count * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tc);
  return cuda_check(h, e, "get cells");
}

st_status st_chunk_bounds(st_handle h, double* out, int on_device) {
  ST_TRY(check_handle(h));
  ST_TRY(materialize_state(h));
  if (!out) return set_error(h, ST_ERR_INVALID_ARG, "out is NULL");
  if (!h->sorted) return set_error(h, ST_ERR_STATE, "particles not sorted since the last change");
  const int B = h->geo.B;
  const int64_t nchunk =
      (int64_t)((h->geo.n[0] + B - 1) / B) * ((h->geo.n[1] + B - 1) / B) * ((h->geo.n[2] + B - 1) / B);
  const size_t bytes = (size_t)nchunk * 6 * sizeof(double);
  Buf tmp;
  double* dst = out;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, bytes));
    dst = (double*)tmp.p;
  }
  cudaError_t e = launch_chunk_bounds(h, dst);
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  return cuda_check(h, e, "chunk bounds");
}

st_status st_get_cell_counts(st_handle h, int64_t* counts, int on_device) {
  ST_TRY(check_handle(h));
  if (!counts) return set_error(h, ST_ERR_INVALID_ARG, "counts is NULL");
  if (!h->sorted && h->np > 0) return set_error(h, ST_ERR_STATE, "particles not sorted since the last change");
  size_t bytes = (size_t)h->geo.ncell * 8;
  Buf tmp;
  int64_t* dst = counts;
  if (!on_device) {
    ST_TRY(dev_alloc(h, tmp, bytes));
    dst = (int64_t*)tmp.p;
  }
  cudaError_t e = cudaSuccess;
  if (h->np == 0) {
    e = cudaMemsetAsync(dst, 0, bytes, h->stream);
  } else {
    e = launch_cell_counts(h, dst);
  }
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(counts, dst, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, tmp);
  return cuda_check(h, e, "cell counts");
}

st_status st_invariants(st_handle h, double out[8]) {
  ST_TRY(check_handle(h));
  ST_TRY(materialize_state(h));
  if (!out) return set_error(h, ST_ERR_INVALID_ARG, "out is NULL");
  double pm[4] = {0, 0, 0, 0}, s3[3] = {0, 0, 0};
  cudaError_t e = cudaSuccess;
  if (h->np > 0) e = launch_particle_sums(h, pm);
  if (e == cudaSuccess) e = launch_acc_sum(h, s3);
  ST_TRY(cuda_check(h, e, "invariants"));
  out[0] = (double)h->np;
  for (int q = 0; q < 3; ++q) out[1 + q] = pm[q];
  for (int q = 0; q < 3; ++q) out[4 + q] = s3[q];
  out[7] = pm[3];
  return ST_OK;
}


st_status st_clear_particles(st_handle h) {
  ST_TRY(check_handle(h));
  h->np = 0;
  h->records_pending = false;
  h->perm_pending = false;
  h->sorted = false;
  h->steps_since_sort = 0;
  h->dmax = 0.0;
  h->vbound = 0.0;
  h->adj_ready = false;
  return ST_OK;
}

static int64_t round64(int64_t n);
static cudaError_t copy_mixed7(const MixedState& dst, const MixedState& src, int64_t n, cudaStream_t st);

// The FP32 adjoint of a mixed FP32-velocity handle: like the FP64 one (segments from the last,
// each recomputed from its checkpoint with the general mixed kernel keeping the state at the start of
// every step, then reversed step by step), with FP32 adjoints of position and velocity.
static st_status adjoint_backward_mixed(st_handle h, const double* lam, int lam_on_device, double* grad_d,
                                        double* grad_alpha, double* grad_U, int on_device) {
  const int64_t n = h->np, nc = h->geo.ncell, cn = round64(n);
  const int C = h->adj_every, nsteps = h->adj_nsteps;
  const int K = (nsteps + C - 1) / C;
  const double pi = 3.14159265358979323846;
  const size_t sb = (size_t)28 * cn;  // one state: cell, offsets, velocities
  Buf blam, lam32, work, tape, adj, db, abp, Uw, tmp;
  auto cleanup = [&]() {
    for (Buf* b : {&blam, &lam32, &work, &tape, &adj, &db, &abp, &Uw, &tmp}) dev_free(h, *b);
  };
  st_status s = dev_alloc(h, work, state_bytes(ST_MIXED_F32, cn));
  if (s == ST_OK) s = dev_alloc(h, tape, (size_t)C * sb);
  if (s == ST_OK) s = dev_alloc(h, adj, (size_t)6 * cn * sizeof(float));
  if (s == ST_OK) s = dev_alloc(h, db, (size_t)cn * sizeof(double));
  if (s == ST_OK) s = dev_alloc(h, abp, (size_t)kAdjBlocks * sizeof(double));
  if (s == ST_OK) s = dev_alloc(h, Uw, (size_t)nc * 3 * kWideWords * sizeof(long long));
  if (s == ST_OK) s = dev_alloc(h, lam32, (size_t)3 * nc * sizeof(float));
  if (s == ST_OK && !lam_on_device) s = dev_alloc(h, blam, (size_t)3 * nc * sizeof(double));
  if (s == ST_OK && !on_device) s = dev_alloc(h, tmp, (size_t)3 * nc * sizeof(double));
  if (s != ST_OK) {
    cleanup();
    return s;
  }
  cudaError_t e = cudaSuccess;
  const double* dlam = lam;
  if (!lam_on_device) {
    e = cudaMemcpyAsync(blam.p, lam, (size_t)3 * nc * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    dlam = (const double*)blam.p;
  }
  if (e == cudaSuccess) e = launch_f64_to_f32(h, dlam, (float*)lam32.p, 3 * nc);
  if (e == cudaSuccess) e = cudaMemsetAsync(adj.p, 0, adj.bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(db.p, 0, db.bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(abp.p, 0, abp.bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(Uw.p, 0, Uw.bytes, h->stream);
  const MixedState st = carve_mixed(h->state.p, h->cap, false);
  MixedState ws = carve_mixed(work.p, cn, false);
  ws.d = st.d;
  float* A = (float*)adj.p;
  StepParams p;
  p.dt = h->adj_dt;
  p.ca = 18.0 * h->mu * h->alpha / h->rho_p;
  p.mcoef = h->mult * h->rho_p * pi / 6.0;
  for (int q = 0; q < 3; ++q) p.g[q] = h->g[q];
  p.E = 0;
  p.scale = 1.0;
  for (int seg = K - 1; seg >= 0 && e == cudaSuccess; --seg) {
    const int s0 = seg * C, s1 = std::min(nsteps, s0 + C);
    e = cudaMemcpyAsync(work.p, (char*)h->ckpt.p + (size_t)seg * sb, sb, cudaMemcpyDeviceToDevice, h->stream);
    for (int k = s0; k < s1 && e == cudaSuccess; ++k) {
      e = cudaMemcpyAsync((char*)tape.p + (size_t)(k - s0) * sb, work.p, sb, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess && k + 1 < s1) {
        timer_begin(h, ST_TIMER_STEP, h->stream);
        e = launch_step_mixed_state(h, ws, n, nullptr, p);
        timer_end(h, ST_TIMER_STEP, h->stream);
      }
    }
    for (int k = s1 - 1; k >= s0 && e == cudaSuccess; --k) {
      AdjointMixedArgs a;
      a.tape = carve_mixed((char*)tape.p + (size_t)(k - s0) * sb, cn, false);
      a.d = st.d;
      for (int q = 0; q < 3; ++q) {
        a.xb[q] = A + q * cn;
        a.vb[q] = A + (3 + q) * cn;
      }
      a.db = (double*)db.p;
      a.ab_part = (double*)abp.p;
      a.lam32 = (const float*)lam32.p;
      a.Uw = (long long*)Uw.p;
      a.dt = h->adj_dt;
      timer_begin(h, ST_TIMER_ADJOINT, h->stream);
      e = launch_adjoint_step_mixed(h, a);
      timer_end(h, ST_TIMER_ADJOINT, h->stream);
    }
  }
  std::vector<double> hab(kAdjBlocks);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hab.data(), abp.p, kAdjBlocks * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && grad_d)
    e = cudaMemcpyAsync(grad_d, db.p, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess && grad_U) {
    double* dst = on_device ? grad_U : (double*)tmp.p;
    e = launch_wide_to_f64(h, (const long long*)Uw.p, dst, 3 * nc);
    if (e == cudaSuccess && !on_device)
      e = cudaMemcpyAsync(grad_U, dst, (size_t)3 * nc * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cleanup();
  ST_TRY(cuda_check(h, e, "adjoint backward (FP32)"));
  if (grad_alpha) {
    double t = 0.0;
    for (int b = 0; b < kAdjBlocks; ++b) t += hab[b];
    *grad_alpha = t;
  }
  return ST_OK;
}

// the mixed state's first seven arrays (cell, offsets, velocities) at a stride of cap particles
static cudaError_t copy_mixed7(const MixedState& dst, const MixedState& src, int64_t n, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(dst.cell, src.cell, n * 4, cudaMemcpyDeviceToDevice, st);
  for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
    e = cudaMemcpyAsync(dst.xi[q], src.xi[q], n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst.v[q], src.v[q], n * 4, cudaMemcpyDeviceToDevice, st);
  }
  return e;
}

static int64_t round64(int64_t n) { return (n + 63) & ~int64_t(63); }

st_status st_adjoint_forward(st_handle h, int nsteps, double dt, int checkpoint_every) {
  ST_TRY(check_handle(h));
  if (h->prec == ST_MIXED_BF16V)
    return set_error(h, ST_ERR_STATE, "the adjoint needs an FP64 or an FP32-velocity handle");
  if (h->micro_on) return set_error(h, ST_ERR_STATE, "the adjoint does not cover the microphysics");
  if (h->prec != ST_FP64 && h->phys_deposit != ST_DEPOSIT_CELL)
    return set_error(h, ST_ERR_STATE, "the FP32 adjoint needs the deposit into the containing cell");
  if (h->phys_gather != ST_GATHER_TRILINEAR || h->phys_integrator != ST_INTEGRATOR_EXPONENTIAL ||
      h->phys_drag != ST_DRAG_STOKES)
    return set_error(h, ST_ERR_STATE,
                     "the adjoint needs the trilinear gather, the exponential integrator and Stokes drag");
  if (nsteps < 1 || checkpoint_every < 1) return set_error(h, ST_ERR_INVALID_ARG, "nsteps and checkpoint_every must be >= 1");
  if (!std::isfinite(dt)) return set_error(h, ST_ERR_NONFINITE, "dt is not finite");
  if (!(dt > 0)) return set_error(h, ST_ERR_INVALID_ARG, "dt must be > 0");
  if (h->np == 0) return set_error(h, ST_ERR_STATE, "no particles");
  const int64_t n = h->np;
  const int K = (nsteps + checkpoint_every - 1) / checkpoint_every;
  const bool mixed = h->prec != ST_FP64;
  if (mixed) ST_TRY(materialize_state(h));
  // checkpoints: x, v in FP64 (48 B per particle), or cell, offsets, velocities (28 B) at a stride of
  // n rounded up to 64
  const size_t ck_bytes = mixed ? (size_t)28 * round64(n) : (size_t)6 * n * sizeof(double);
  ST_TRY(ensure(h, h->ckpt, (size_t)K * ck_bytes));
  const double pi = 3.14159265358979323846;
  F64State s = carve_f64(h->state.p, h->cap);
  double* ck = (double*)h->ckpt.p;
  for (int step = 0; step < nsteps; ++step) {
    if (mixed && step % checkpoint_every == 0) {
      const MixedState slot = carve_mixed((char*)h->ckpt.p + (size_t)(step / checkpoint_every) * ck_bytes,
                                          round64(n), false);
      ST_TRY(cuda_check(h, copy_mixed7(slot, carve_mixed(h->state.p, h->cap, false), n, h->stream), "checkpoint"));
    } else if (step % checkpoint_every == 0) {
      double* slot = ck + (size_t)(step / checkpoint_every) * 6 * n;
      cudaError_t e = cudaSuccess;
      for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
        e = cudaMemcpyAsync(slot + q * n, s.x[q], n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(slot + (3 + q) * n, s.v[q], n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
      }
      ST_TRY(cuda_check(h, e, "checkpoint"));
    }
    int E = 0;
    ST_TRY(prepare_accumulator(h, dt, (double)h->np + 8.0, &E));
    StepParams p;
    p.dt = dt;
    p.ca = 18.0 * h->mu * h->alpha / h->rho_p;
    p.mcoef = h->mult * h->rho_p * pi / 6.0;
    for (int q = 0; q < 3; ++q) p.g[q] = h->g[q];
    p.E = E;
    p.scale = std::ldexp(1.0, E);
    p.cic = h->phys_deposit == ST_DEPOSIT_CIC;  // the other physics are the defaults here
    timer_begin(h, ST_TIMER_STEP, h->stream);
    // mixed handles: the general kernel in storage order, which the backward pass recomputes with
    const cudaError_t fe = mixed ? launch_step_mixed(h, p) : launch_step_f64(h, p);
    timer_end(h, ST_TIMER_STEP, h->stream);
    ST_TRY(cuda_check(h, fe, "adjoint forward step"));
  }
  h->adj_nsteps = nsteps;
  h->adj_every = checkpoint_every;
  h->adj_dt = dt;
  h->adj_ready = true;
  return ST_OK;
}

st_status st_adjoint_backward(st_handle h, const double* lam, int lam_on_device, double* grad_d, double* grad_alpha,
                              double* grad_U, int on_device) {
  ST_TRY(check_handle(h));
  if (!h->adj_ready) return set_error(h, ST_ERR_STATE, "no st_adjoint_forward run to differentiate");
  if (!lam) return set_error(h, ST_ERR_INVALID_ARG, "lam is NULL");
  if (h->prec != ST_FP64) return adjoint_backward_mixed(h, lam, lam_on_device, grad_d, grad_alpha, grad_U, on_device);
  const int64_t n = h->np, nc = h->geo.ncell;
  const int C = h->adj_every, nsteps = h->adj_nsteps;
  const int K = (nsteps + C - 1) / C;
  const double pi = 3.14159265358979323846;
  // scratch: lam, working state (x, v), tape of C states, adjoints, carry-save dL/dU
  Buf blam, work, tape, adj, abp, Uw, tmp;
  auto cleanup = [&]() {
    for (Buf* b : {&blam, &work, &tape, &adj, &abp, &Uw, &tmp}) dev_free(h, *b);
  };
  st_status s = dev_alloc(h, work, (size_t)6 * n * sizeof(double));
  if (s == ST_OK) s = dev_alloc(h, tape, (size_t)C * 6 * n * sizeof(double));
  if (s == ST_OK) s = dev_alloc(h, adj, (size_t)7 * n * sizeof(double));
  if (s == ST_OK) s = dev_alloc(h, abp, (size_t)kAdjBlocks * sizeof(double));
  if (s == ST_OK) s = dev_alloc(h, Uw, (size_t)nc * 3 * kWideWords * sizeof(long long));
  if (s == ST_OK && !lam_on_device) s = dev_alloc(h, blam, (size_t)3 * nc * sizeof(double));
  if (s == ST_OK && (!on_device)) s = dev_alloc(h, tmp, (size_t)(std::max<int64_t>(n, 3 * nc)) * sizeof(double));
  if (s != ST_OK) {
    cleanup();
    return s;
  }
  cudaError_t e = cudaSuccess;
  const double* dlam = lam;
  if (!lam_on_device) {
    e = cudaMemcpyAsync(blam.p, lam, (size_t)3 * nc * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    dlam = (const double*)blam.p;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(adj.p, 0, adj.bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(abp.p, 0, abp.bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(Uw.p, 0, Uw.bytes, h->stream);
  F64State st = carve_f64(h->state.p, h->cap);
  double* W = (double*)work.p;
  double* A = (double*)adj.p;
  F64State ws;
  for (int q = 0; q < 3; ++q) {
    ws.x[q] = W + q * n;
    ws.v[q] = W + (3 + q) * n;
  }
  ws.d = st.d;
  StepParams p;
  p.dt = h->adj_dt;
  p.ca = 18.0 * h->mu * h->alpha / h->rho_p;
  p.mcoef = h->mult * h->rho_p * pi / 6.0;
  for (int q = 0; q < 3; ++q) p.g[q] = h->g[q];
  p.E = 0;
  p.scale = 1.0;
  for (int seg = K - 1; seg >= 0 && e == cudaSuccess; --seg) {
    const int s0 = seg * C, s1 = std::min(nsteps, s0 + C);
    e = cudaMemcpyAsync(W, (double*)h->ckpt.p + (size_t)seg * 6 * n, (size_t)6 * n * sizeof(double),
                        cudaMemcpyDeviceToDevice, h->stream);
    // recompute the segment, keeping the state at the start of every step
    for (int k = s0; k < s1 && e == cudaSuccess; ++k) {
      double* slot = (double*)tape.p + (size_t)(k - s0) * 6 * n;
      e = cudaMemcpyAsync(slot, W, (size_t)6 * n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess && k + 1 < s1) {
        timer_begin(h, ST_TIMER_STEP, h->stream);
        e = launch_step_f64_state(h, ws, nullptr, p);
        timer_end(h, ST_TIMER_STEP, h->stream);
      }
    }
    // reverse sweep
    for (int k = s1 - 1; k >= s0 && e == cudaSuccess; --k) {
      const double* slot = (const double*)tape.p + (size_t)(k - s0) * 6 * n;
      AdjointStepArgs a;
      for (int q = 0; q < 3; ++q) {
        a.x[q] = slot + q * n;
        a.v[q] = slot + (3 + q) * n;
        a.xb[q] = A + q * n;
        a.vb[q] = A + (3 + q) * n;
      }
      a.d = st.d;
      a.db = A + 6 * n;
      a.ab_part = (double*)abp.p;
      a.lam = dlam;
      a.Uw = (long long*)Uw.p;
      a.dt = h->adj_dt;
      timer_begin(h, ST_TIMER_ADJOINT, h->stream);
      e = launch_adjoint_step(h, a);
      timer_end(h, ST_TIMER_ADJOINT, h->stream);
    }
  }
  // outputs
  std::vector<double> hab(kAdjBlocks);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hab.data(), abp.p, kAdjBlocks * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && grad_d) {
    if (on_device) {
      e = cudaMemcpyAsync(grad_d, A + 6 * n, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    } else {
      e = cudaMemcpyAsync(grad_d, A + 6 * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    }
  }
  if (e == cudaSuccess && grad_U) {
    double* dst = on_device ? grad_U : (double*)tmp.p;
    e = launch_wide_to_f64(h, (const long long*)Uw.p, dst, 3 * nc);
    if (e == cudaSuccess && !on_device)
      e = cudaMemcpyAsync(grad_U, dst, (size_t)3 * nc * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cleanup();
  ST_TRY(cuda_check(h, e, "adjoint backward"));
  if (grad_alpha) {
    double t = 0.0;
    for (int b = 0; b < kAdjBlocks; ++b) t += hab[b];
    *grad_alpha = t;
  }
  return ST_OK;
}

st_status st_probe_fma(st_handle h, double* fp64_gflops, double* fp32_gflops) {
  ST_TRY(check_handle(h));
  if (!fp64_gflops || !fp32_gflops) return set_error(h, ST_ERR_INVALID_ARG, "output pointers are required");
  return cuda_check(h, probe_fma_rates(h, fp64_gflops, fp32_gflops), "fma probe");
}

st_status st_kernel_launches(st_handle h, int64_t* count) {
  ST_TRY(check_handle(h));
  if (!count) return set_error(h, ST_ERR_INVALID_ARG, "count is NULL");
  *count = h->launches;
  return ST_OK;
}

st_status st_gen_particles(st_handle h, uint64_t seed, int64_t first, int64_t count, const double L[3], double vmax,
                           const double* qtable, int nq, double* xyz, double* vel, double* d, uint32_t* ids) {
  ST_TRY(check_handle(h));
  if (first < 0 || count < 0 || !L || nq < 1 || (d && !qtable)) return set_error(h, ST_ERR_INVALID_ARG, "bad arguments");
  if (!finite3(L) || !std::isfinite(vmax)) return set_error(h, ST_ERR_NONFINITE, "non-finite box or vmax");
  if (nq < 2 || (nq & (nq - 1)) != 0 || nq > (1 << 20)) return set_error(h, ST_ERR_INVALID_ARG, "nq must be a power of two in [2, 2^20]");
  if (count == 0) return ST_OK;
  cudaError_t e = launch_gen(h, seed, first, count, L, vmax, qtable, nq, xyz, vel, d, ids);
  return cuda_check(h, e, "generate particles");
}

}  // extern "C"
