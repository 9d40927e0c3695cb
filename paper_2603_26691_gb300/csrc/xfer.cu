// Asynchronous host transfers of the field and the sources.  The paper's coupling (Sec. 2.3) keeps the
// GPU computing while data moves between the host and the device; here a field upload and a source
// download run on streams of their own beside the particle step, ordered by events:
//   * st_set_fluid_async copies the host field into a device staging buffer on the upload stream,
//     scans it there (largest magnitude, non-finite values; the result is copied to pinned host
//     memory), and queues the padding into the step's field on the compute stream behind the work
//     already queued, so a step in flight keeps reading the previous field.  The host reads the scan
//     result at the next call that needs it (the next step, sort or synchronous call), normally long
//     after the copy finished; a field with NaN or Inf is not taken (its padding kernel skips) and that
//     call reports ST_ERR_NONFINITE.
//   * st_get_sources_async converts the exact accumulator into one of two device staging buffers on
//     the compute stream (and resets it when asked), and copies that buffer to the host on the
//     download stream while the next steps run.
//   * st_synchronize waits for both streams and the compute stream and reports any pending error.
#include <cstring>

#include "st_common.cuh"

namespace st {

struct Xfer {
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t up_done = nullptr, pack_done = nullptr, ready[2] = {}, out_done[2] = {};
  Buf fstage, sstage[2], red;              // red: {largest magnitude bits, non-finite flag} on the device
  unsigned long long* hred = nullptr;      // pinned host copy of red
  int next = 0;
  bool pending = false;  // an upload whose scan result the host has not read
};

void xfer_free(st_ctx* h) {
  Xfer* x = h->xfer;
  if (!x) return;
  if (x->up) cudaStreamSynchronize(x->up);
  if (x->down) cudaStreamSynchronize(x->down);
  dev_free(h, x->fstage);
  dev_free(h, x->sstage[0]);
  dev_free(h, x->sstage[1]);
  dev_free(h, x->red);
  if (x->hred) cudaFreeHost(x->hred);
  for (cudaEvent_t e : {x->up_done, x->pack_done, x->ready[0], x->ready[1], x->out_done[0], x->out_done[1]})
    if (e) cudaEventDestroy(e);
  if (x->up) cudaStreamDestroy(x->up);
  if (x->down) cudaStreamDestroy(x->down);
  delete x;
  h->xfer = nullptr;
}

st_status settle_fluid(st_ctx* h) {
  Xfer* x = h->xfer;
  if (!x || !x->pending) return ST_OK;
  x->pending = false;
  ST_TRY(cuda_check(h, cudaEventSynchronize(x->up_done), "field upload"));
  double m;
  std::memcpy(&m, &x->hred[0], 8);
  if (x->hred[1] & 0xffffffffu)
    return set_error(h, ST_ERR_NONFINITE, "the field given to st_set_fluid_async holds NaN or Inf (not taken)");
  h->umax = m;
  h->fluid_set = true;
  h->adj_ready = false;
  h->fl_valid = false;
  h->couple_done = 0;
  return ST_OK;
}

static st_status xfer_init(st_ctx* h) {
  if (h->xfer) return ST_OK;
  Xfer* x = new (std::nothrow) Xfer();
  if (!x) return ST_ERR_OOM;
  h->xfer = x;
  cudaError_t e = cudaStreamCreateWithFlags(&x->up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x->down, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&x->up_done, &x->pack_done, &x->ready[0], &x->ready[1], &x->out_done[0], &x->out_done[1]})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&x->hred, 16, cudaHostAllocDefault);
  st_status s = cuda_check(h, e, "transfer streams");
  if (s == ST_OK) s = dev_alloc(h, x->red, 16);
  if (s != ST_OK) xfer_free(h);
  return s;
}

cudaError_t xfer_sync(st_ctx* h) {
  if (!h->xfer) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(h->xfer->up);
  cudaError_t e2 = cudaStreamSynchronize(h->xfer->down);
  return e != cudaSuccess ? e : e2;
}

}  // namespace st

using namespace st;

namespace {
st_status xfer_check(st_handle h) {
  if (!h) return ST_ERR_INVALID_ARG;
  h->err.clear();
  return cuda_check(h, cudaSetDevice(h->dev), "cudaSetDevice");
}
}  // namespace

extern "C" {

st_status st_set_fluid_async(st_handle h, const void* u, int dtype) {
  ST_TRY(xfer_check(h));
  if (!u) return set_error(h, ST_ERR_INVALID_ARG, "u is NULL");
  if (dtype != ST_DTYPE_F32 && dtype != ST_DTYPE_F64) return set_error(h, ST_ERR_INVALID_ARG, "bad dtype");
  ST_TRY(settle_fluid(h));  // the previous upload's scan result first (its buffers are reused)
  ST_TRY(xfer_init(h));
  Xfer* x = h->xfer;
  const size_t bytes = (size_t)h->geo.ncell * 3 * (dtype == ST_DTYPE_F64 ? 8 : 4);
  if (x->fstage.bytes < bytes) {
    // nothing may still read the old staging buffer
    ST_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "staging buffer"));
    dev_free(h, x->fstage);
    ST_TRY(dev_alloc(h, x->fstage, bytes));
  }
  // the upload stream: after the previous padding consumed the staging buffer, copy, then scan
  cudaError_t e = cudaStreamWaitEvent(x->up, x->pack_done, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x->fstage.p, u, bytes, cudaMemcpyHostToDevice, x->up);
  if (e == cudaSuccess)
    e = launch_maxabs_on(h, x->fstage.p, h->geo.ncell * 3, dtype, x->up, (unsigned long long*)x->red.p, x->hred);
  if (e == cudaSuccess) e = cudaEventRecord(x->up_done, x->up);
  // the compute stream: the padding into the step's field behind the work already queued (skipped
  // when the scan found a non-finite value)
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, x->up_done, 0);
  if (e == cudaSuccess) e = launch_fluid_pack_if(h, x->fstage.p, dtype, (const int*)((unsigned long long*)x->red.p + 1));
  if (e == cudaSuccess) e = cudaEventRecord(x->pack_done, h->stream);
  ST_TRY(cuda_check(h, e, "field upload"));
  x->pending = true;
  return ST_OK;
}

st_status st_get_sources_async(st_handle h, double* out, int reset) {
  ST_TRY(xfer_check(h));
  if (!out) return set_error(h, ST_ERR_INVALID_ARG, "out is NULL");
  ST_TRY(xfer_init(h));
  Xfer* x = h->xfer;
  const size_t bytes = (size_t)h->geo.ncell * 3 * sizeof(double);
  const int b = x->next;
  if (x->sstage[b].bytes < bytes) {
    ST_TRY(cuda_check(h, cudaStreamSynchronize(x->down), "staging buffer"));
    dev_free(h, x->sstage[b]);
    ST_TRY(dev_alloc(h, x->sstage[b], bytes));
  }
  // the compute stream: once this staging buffer's previous download is done, convert (and reset)
  cudaError_t e = cudaStreamWaitEvent(h->stream, x->out_done[b], 0);
  if (e == cudaSuccess) e = launch_acc_to_f64(h, (double*)x->sstage[b].p, h->acc_E);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(h->acc.p, 0, h->acc.bytes, h->stream);
  if (e == cudaSuccess && reset) e = reset_acc_counter(h);
  if (e == cudaSuccess) e = cudaEventRecord(x->ready[b], h->stream);
  // the download stream: the copy to the host
  if (e == cudaSuccess) e = cudaStreamWaitEvent(x->down, x->ready[b], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, x->sstage[b].p, bytes, cudaMemcpyDeviceToHost, x->down);
  if (e == cudaSuccess) e = cudaEventRecord(x->out_done[b], x->down);
  ST_TRY(cuda_check(h, e, "source download"));
  if (reset) {
    h->acc_empty = true;
    h->acc_load = 0.0;
  }
  x->next ^= 1;
  return ST_OK;
}

}  // extern "C"
