// Inline-PTX wrappers shared by the kernels that stage data with the Tensor Memory Accelerator:
// shared-memory mbarriers (every wait bounded) and 1-D bulk copies global -> shared.
#pragma once

#include <stdint.h>

namespace st {
namespace ptx {

constexpr uint32_t kSpinLimit = 1u << 22;          // polls before a wait gives up
constexpr uint64_t kWaitLimitNs = 1000000000ull;   // or 1 s of wall time, whichever comes first

__device__ __forceinline__ uint32_t sptr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sptr(b)), "r"(tx) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(sptr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the phase with the given parity to complete: gives up after kWaitLimitNs of
// wall time or kSpinLimit polls, whichever comes first
static __device__ __noinline__ bool mbar_wait_slow(uint64_t* b, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kSpinLimit; i += 32) {
    for (int k = 0; k < 32; ++k)
      if (mbar_test(b, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  return mbar_test(b, parity) || mbar_wait_slow(b, parity);
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sptr(dst)),
               "l"(src), "r"(bytes), "r"(sptr(bar))
               : "memory");
}
// One 32-byte particle record {cell bits, offsets | velocity, diameter} as a single 256-bit
// global access (sm_100 and later; the address must be 32-byte aligned): one sector per particle.
struct Rec32 {
  float c, x0, x1, x2, v0, v1, v2, d;
};
__device__ __forceinline__ void st_rec32(void* p, const Rec32& r) {
  asm volatile("st.global.L1::no_allocate.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(r.c),
               "f"(r.x0), "f"(r.x1), "f"(r.x2), "f"(r.v0), "f"(r.v1), "f"(r.v2), "f"(r.d)
               : "memory");
}
__device__ __forceinline__ Rec32 ld_rec32(const void* p) {
  Rec32 r;
  asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(r.c), "=f"(r.x0), "=f"(r.x1), "=f"(r.x2), "=f"(r.v0), "=f"(r.v1), "=f"(r.v2), "=f"(r.d)
               : "l"(p));
  return r;
}

}  // namespace ptx
}  // namespace st
