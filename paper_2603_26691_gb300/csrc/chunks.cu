// Chunked particle sets (paper Sec. 2.2): the particles are held as chunks - structures of arrays of
// a fixed capacity - in pinned host memory, and the GPU computes one chunk after the other while the
// finished chunk's state goes back to the host and the next chunk's comes in.  This lets a particle
// set larger than device memory run on one GPU, with the transfers hidden behind the computation.
//
// Each chunk's state is one contiguous block in the device layout of a handle whose capacity is the
// chunk capacity C (cell | offsets | velocities | diameters, then the ids), so a chunk moves with two
// copies each way.  Three device slots rotate: while chunk k computes in its slot (the handle's own
// state buffers are bound to it, the chunk is sorted and stepped exactly as resident particles are),
// chunk k+1 is copied into the next slot and chunk k-1 out of the previous one, on an upload and a
// download stream of their own (the two directions of the host link run at once), ordered by
// events.  A particle's arithmetic does not depend on the other particles, so positions and
// velocities are those of a resident run; the sources of every chunk go into the handle's exact
// accumulator, whose sum does not depend on the order of the chunks.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "st_common.cuh"

namespace st {

struct ChunkStore {
  int64_t C = 0;                  // particles per chunk (a multiple of 64)
  std::vector<int64_t> count;     // particles in each chunk
  std::vector<char*> host;        // pinned: state block (state_bytes(prec, C)) then ids (4 C)
  size_t state_bytes_ = 0;
  Buf slot_state[3], slot_ids[3];  // device slots (slot 0 starts as the handle's own buffers)
  cudaStream_t up_s = nullptr, down_s = nullptr;
  cudaEvent_t up[3] = {}, done[3] = {}, down[3] = {}, t0 = nullptr, t1 = nullptr;
  double ms_compute = 0.0, ms_h2d = 0.0, ms_d2h = 0.0;
};

void chunk_store_free(st_ctx* h) {
  ChunkStore* cs = h->chunks;
  if (!cs) return;
  if (cs->up_s) cudaStreamSynchronize(cs->up_s);
  if (cs->down_s) cudaStreamSynchronize(cs->down_s);
  for (char* p : cs->host) cudaFreeHost(p);
  for (int s = 0; s < 3; ++s) {
    // slot buffers that are not (any longer) the handle's own
    Buf* own[4] = {&h->state, &h->state_alt, &h->ids, &h->ids_alt};
    bool owned = false;
    for (Buf* b : own) owned = owned || b->p == cs->slot_state[s].p;
    if (!owned) dev_free(h, cs->slot_state[s]);
    owned = false;
    for (Buf* b : own) owned = owned || b->p == cs->slot_ids[s].p;
    if (!owned) dev_free(h, cs->slot_ids[s]);
    for (cudaEvent_t e : {cs->up[s], cs->done[s], cs->down[s]})
      if (e) cudaEventDestroy(e);
  }
  if (cs->t0) cudaEventDestroy(cs->t0);
  if (cs->t1) cudaEventDestroy(cs->t1);
  if (cs->up_s) cudaStreamDestroy(cs->up_s);
  if (cs->down_s) cudaStreamDestroy(cs->down_s);
  delete cs;
  h->chunks = nullptr;
}

}  // namespace st

using namespace st;

namespace {

st_status chunk_check(st_handle h) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  ST_TRY(cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice"));
  if (!h->chunks) return set_error(h, ST_ERR_STATE, "no chunks (st_chunks_create first)");
  return ST_OK;
}

// bind slot s to the handle's working state (the buffers it computes in)
void bind_slot(st_ctx* h, int s) {
  ChunkStore* cs = h->chunks;
  h->state = cs->slot_state[s];
  h->ids = cs->slot_ids[s];
}

// the buffers that hold the chunk's state after it computed become slot s
void take_slot(st_ctx* h, int s) {
  ChunkStore* cs = h->chunks;
  cs->slot_state[s] = h->state;
  cs->slot_ids[s] = h->ids;
}

}  // namespace

extern "C" {

st_status st_chunks_create(st_handle h, int64_t chunk_particles) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  ST_TRY(cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice"));
  if (h->chunks) return set_error(h, ST_ERR_STATE, "chunks already created");
  if (h->np != 0) return set_error(h, ST_ERR_STATE, "the handle holds resident particles");
  if (h->micro_on) return set_error(h, ST_ERR_STATE, "chunks and microphysics do not combine");
  if (chunk_particles < 1 || chunk_particles > (int64_t(1) << 31))
    return set_error(h, ST_ERR_INVALID_ARG, "chunk_particles out of range");
  const int64_t C = (chunk_particles + 63) & ~int64_t(63);
  ChunkStore* cs = new (std::nothrow) ChunkStore();
  if (!cs) return ST_ERR_OOM;
  cs->C = C;
  cs->state_bytes_ = state_bytes(h->prec, C);
  h->chunks = cs;
  // the handle's own buffers at capacity C, sized like the sort's spare buffer so that any slot can
  // take the place of any other
  dev_free(h, h->state);
  dev_free(h, h->state_alt);
  dev_free(h, h->ids);
  dev_free(h, h->ids_alt);
  const size_t sb = state_alt_bytes(h->prec, C), ib = (size_t)C * sizeof(uint32_t);
  st_status s = dev_alloc(h, h->state, sb);
  if (s == ST_OK) s = dev_alloc(h, h->state_alt, sb);
  if (s == ST_OK) s = dev_alloc(h, h->ids, ib);
  if (s == ST_OK) s = dev_alloc(h, h->ids_alt, ib);
  h->cap = C;
  cs->slot_state[0] = h->state;
  cs->slot_ids[0] = h->ids;
  for (int k = 1; k < 3 && s == ST_OK; ++k) {
    s = dev_alloc(h, cs->slot_state[k], sb);
    if (s == ST_OK) s = dev_alloc(h, cs->slot_ids[k], ib);
  }
  cudaError_t e = cudaSuccess;
  if (s == ST_OK) e = cudaStreamCreateWithFlags(&cs->up_s, cudaStreamNonBlocking);
  if (s == ST_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs->down_s, cudaStreamNonBlocking);
  for (int k = 0; k < 3 && s == ST_OK && e == cudaSuccess; ++k) {
    e = cudaEventCreate(&cs->up[k]);
    if (e == cudaSuccess) e = cudaEventCreate(&cs->done[k]);
    if (e == cudaSuccess) e = cudaEventCreate(&cs->down[k]);
  }
  if (s == ST_OK && e == cudaSuccess) e = cudaEventCreate(&cs->t0);
  if (s == ST_OK && e == cudaSuccess) e = cudaEventCreate(&cs->t1);
  if (s == ST_OK) s = cuda_check(h, e, "chunk streams and events");
  if (s != ST_OK) {
    chunk_store_free(h);
    return s;
  }
  h->sorted = false;
  return ST_OK;
}

st_status st_chunks_add(st_handle h, int64_t n, const double* xyz, const double* vel, const double* d, int on_device) {
  ST_TRY(chunk_check(h));
  ChunkStore* cs = h->chunks;
  if (n < 0) return set_error(h, ST_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return ST_OK;
  if (!xyz || !d) return set_error(h, ST_ERR_INVALID_ARG, "xyz and d are required");
  int64_t total = 0;
  for (int64_t c : cs->count) total += c;
  if (total + n >= (int64_t(1) << 32)) return set_error(h, ST_ERR_INVALID_ARG, "ids run past 2^32");
  const int64_t C = cs->C;
  // pieces of up to C particles, packed contiguously on the device, imported through the handle's own
  // path into slot 0, then copied to a new chunk's pinned block
  Buf px, pv, pd, pi;
  auto cleanup = [&]() {
    dev_free(h, px);
    dev_free(h, pv);
    dev_free(h, pd);
    dev_free(h, pi);
  };
  st_status s = dev_alloc(h, px, (size_t)std::min(C, n) * 24);
  if (s == ST_OK && vel) s = dev_alloc(h, pv, (size_t)std::min(C, n) * 24);
  if (s == ST_OK) s = dev_alloc(h, pd, (size_t)std::min(C, n) * 8);
  if (s == ST_OK) s = dev_alloc(h, pi, (size_t)std::min(C, n) * 4);
  if (s != ST_OK) {
    cleanup();
    return s;
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  std::vector<uint32_t> idh((size_t)std::min(C, n));
  bind_slot(h, 0);
  for (int64_t f = 0; f < n && s == ST_OK; f += C) {
    const int64_t p = std::min(C, n - f);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
      e = cudaMemcpyAsync((double*)px.p + q * p, xyz + q * n + f, p * 8, kind, h->stream);
      if (e == cudaSuccess && vel) e = cudaMemcpyAsync((double*)pv.p + q * p, vel + q * n + f, p * 8, kind, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(pd.p, d + f, p * 8, kind, h->stream);
    for (int64_t i = 0; i < p; ++i) idh[i] = (uint32_t)(total + f + i);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pi.p, idh.data(), p * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    s = cuda_check(h, e, "stage chunk particles");
    if (s != ST_OK) break;
    h->np = 0;
    h->chunk_adding = true;
    s = st_add_particles(h, p, (const double*)px.p, vel ? (const double*)pv.p : nullptr, (const double*)pd.p,
                         (const uint32_t*)pi.p, 1);
    h->chunk_adding = false;
    if (s != ST_OK) break;
    char* blk = nullptr;
    e = cudaHostAlloc((void**)&blk, cs->state_bytes_ + (size_t)C * 4, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s = set_error(h, ST_ERR_OOM, "pinned host memory for a chunk");
      break;
    }
    e = cudaMemcpyAsync(blk, h->state.p, cs->state_bytes_, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(blk + cs->state_bytes_, h->ids.p, (size_t)C * 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      cudaFreeHost(blk);
      s = cuda_check(h, e, "chunk to host");
      break;
    }
    cs->host.push_back(blk);
    cs->count.push_back(p);
  }
  take_slot(h, 0);
  h->np = 0;
  h->sorted = false;
  cleanup();
  return s;
}

st_status st_chunks_count(st_handle h, int64_t* particles, int64_t* chunks) {
  ST_TRY(chunk_check(h));
  int64_t total = 0;
  for (int64_t c : h->chunks->count) total += c;
  if (particles) *particles = total;
  if (chunks) *chunks = (int64_t)h->chunks->count.size();
  return ST_OK;
}

st_status st_chunks_step(st_handle h, int nsteps, double dt, double* ms) {
  ST_TRY(chunk_check(h));
  ChunkStore* cs = h->chunks;
  if (nsteps < 0) return set_error(h, ST_ERR_INVALID_ARG, "nsteps < 0");
  if (!std::isfinite(dt) || !(dt > 0)) return set_error(h, ST_ERR_INVALID_ARG, "dt must be finite and > 0");
  const int64_t K = (int64_t)cs->count.size();
  if (K == 0 || nsteps == 0) return ST_OK;
  const size_t sb = cs->state_bytes_, ib = (size_t)cs->C * 4;
  cudaStream_t up = cs->up_s, down = cs->down_s, comp = h->stream;
  std::vector<cudaEvent_t> tev;  // per chunk: h2d start/end, compute start/end, d2h start/end
  auto ev = [&]() {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    tev.push_back(e);
    return e;
  };
  std::vector<cudaEvent_t> marks;
  cudaError_t e = cudaEventRecord(cs->t0, comp);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(up, cs->t0, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(down, cs->t0, 0);
  auto upload = [&](int64_t k) -> cudaError_t {
    const int s = (int)(k % 3);
    cudaError_t r = cudaSuccess;
    if (k >= 3) r = cudaStreamWaitEvent(up, cs->down[s], 0);  // chunk k-3's download left the slot
    cudaEvent_t a = ev(), b = ev();
    if (r == cudaSuccess) r = cudaEventRecord(a, up);
    if (r == cudaSuccess) r = cudaMemcpyAsync(cs->slot_state[s].p, cs->host[k], sb, cudaMemcpyHostToDevice, up);
    if (r == cudaSuccess) r = cudaMemcpyAsync(cs->slot_ids[s].p, cs->host[k] + sb, ib, cudaMemcpyHostToDevice, up);
    if (r == cudaSuccess) r = cudaEventRecord(b, up);
    if (r == cudaSuccess) r = cudaEventRecord(cs->up[s], up);
    marks.push_back(a);
    marks.push_back(b);
    return r;
  };
  if (e == cudaSuccess) e = upload(0);
  st_status st = cuda_check(h, e, "chunk upload");
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> comp_ev, d2h_ev;
  for (int64_t k = 0; k < K && st == ST_OK; ++k) {
    const int s = (int)(k % 3);
    if (k + 1 < K) {
      e = upload(k + 1);
      if ((st = cuda_check(h, e, "chunk upload")) != ST_OK) break;
    }
    // compute chunk k in slot s: the handle works on it as on resident particles
    e = cudaStreamWaitEvent(comp, cs->up[s], 0);
    if ((st = cuda_check(h, e, "chunk wait")) != ST_OK) break;
    bind_slot(h, s);
    h->np = cs->count[k];
    h->sorted = false;
    h->steps_since_sort = 0;
    h->records_pending = false;
    h->perm_pending = false;
    cudaEvent_t a = ev(), b = ev();
    cudaEventRecord(a, comp);
    st = run_steps(h, nsteps, dt);
    if (st == ST_OK) st = materialize_state(h);
    cudaEventRecord(b, comp);
    comp_ev.push_back({a, b});
    take_slot(h, s);
    if (st != ST_OK) break;
    e = cudaEventRecord(cs->done[s], comp);
    // chunk k back to its pinned block once computed
    if (e == cudaSuccess) e = cudaStreamWaitEvent(down, cs->done[s], 0);
    cudaEvent_t c = ev(), dd = ev();
    if (e == cudaSuccess) e = cudaEventRecord(c, down);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cs->host[k], cs->slot_state[s].p, sb, cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cs->host[k] + sb, cs->slot_ids[s].p, ib, cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess) e = cudaEventRecord(dd, down);
    if (e == cudaSuccess) e = cudaEventRecord(cs->down[s], down);
    d2h_ev.push_back({c, dd});
    st = cuda_check(h, e, "chunk download");
  }
  // the last download ends the pass (it follows every upload and computation through the events)
  if (st == ST_OK) e = cudaEventRecord(cs->t1, down);
  cudaError_t e1 = cudaStreamSynchronize(up);
  cudaError_t e2 = cudaStreamSynchronize(down);
  cudaError_t e3 = cudaStreamSynchronize(comp);
  if (st == ST_OK)
    st = cuda_check(h, e != cudaSuccess ? e : (e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)), "chunk pass");
  h->np = 0;
  h->sorted = false;
  if (st == ST_OK && ms) {
    float w = 0.0f;
    cudaEventElapsedTime(&w, cs->t0, cs->t1);
    double tc = 0, tu = 0, td = 0;
    float x;
    for (auto& pr : comp_ev)
      if (cudaEventElapsedTime(&x, pr.first, pr.second) == cudaSuccess) tc += x;
    for (size_t i = 0; i + 1 < marks.size(); i += 2)
      if (cudaEventElapsedTime(&x, marks[i], marks[i + 1]) == cudaSuccess) tu += x;
    for (auto& pr : d2h_ev)
      if (cudaEventElapsedTime(&x, pr.first, pr.second) == cudaSuccess) td += x;
    ms[0] = w;
    ms[1] = tc;
    ms[2] = tu;
    ms[3] = td;
  }
  for (cudaEvent_t t : tev) cudaEventDestroy(t);
  return st;
}

st_status st_chunks_get(st_handle h, int64_t first, int64_t count, double* xyz, double* vel, double* d,
                        uint32_t* ids) {
  ST_TRY(chunk_check(h));
  ChunkStore* cs = h->chunks;
  ST_TRY(cuda_check(h, cudaStreamSynchronize(cs->down_s), "chunk copies"));
  int64_t total = 0;
  for (int64_t c : cs->count) total += c;
  if (first < 0 || count < 0 || first + count > total) return set_error(h, ST_ERR_INVALID_ARG, "range out of bounds");
  const bool bf = h->prec == ST_MIXED_BF16V;
  int64_t base = 0, o = 0;
  for (size_t k = 0; k < cs->count.size() && o < count; ++k) {
    const int64_t cnt = cs->count[k];
    const int64_t lo = std::max(first, base), hi = std::min(first + count, base + cnt);
    for (int64_t g = lo; g < hi; ++g, ++o) {
      const int64_t i = g - base;
      char* blk = cs->host[k];
      const uint32_t* id = reinterpret_cast<const uint32_t*>(blk + cs->state_bytes_);
      if (ids) ids[o] = id[i];
      if (h->prec == ST_FP64) {
        const F64State fs = carve_f64(blk, cs->C);
        for (int q = 0; q < 3; ++q) {
          if (xyz) xyz[q * count + o] = fs.x[q][i];
          if (vel) vel[q * count + o] = fs.v[q][i];
        }
        if (d) d[o] = fs.d[i];
      } else {
        const MixedState ms = carve_mixed(blk, cs->C, bf);
        const int32_t c = ms.cell[i];
        const int idx[3] = {cell_i(c), cell_j(c), cell_k(c)};
        for (int q = 0; q < 3; ++q) {
          if (xyz) xyz[q * count + o] = ((double)idx[q] + (double)ms.xi[q][i]) * h->geo.h[q];
          if (vel) {
            float v;
            if (bf) {
              const uint16_t b = ((const uint16_t*)ms.v[q])[i];
              const uint32_t u = (uint32_t)b << 16;
              std::memcpy(&v, &u, 4);
            } else {
              v = ((const float*)ms.v[q])[i];
            }
            vel[q * count + o] = (double)v;
          }
        }
        if (d) d[o] = (double)ms.d[i];
      }
    }
    base += cnt;
  }
  return ST_OK;
}

}  // extern "C"
