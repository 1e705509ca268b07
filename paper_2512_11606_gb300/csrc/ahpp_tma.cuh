// TMA row gathers for the batched pull phases (sm_100+ tile::gather4).
//
// The query-minor state of a tile ([node][32 queries], 128 bytes per node) is
// described by a 2D tensor map (32 floats x rows, box 32 x 1).  One gather4
// fetches 4 arbitrary rows (4 x 128 B) into shared memory and signals an
// mbarrier, so the rows in flight live in shared memory instead of
// registers: a warp keeps two 32-entry stages (64 rows) in flight while it
// consumes earlier ones.  Every mbarrier wait is bounded.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "ahpp_internal.cuh"

namespace ahpp {

constexpr int kStage = 32;                      // entries per stage
constexpr int kStageBytes = kStage * 128;       // 32 rows of 128 B
constexpr unsigned int kMbarSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar), "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait (about two seconds of wall time) for the phase `parity` of
// bar; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (unsigned int i = 0; i < kMbarSpinLimit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 63u) == 63u && globaltimer_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

// 4 rows (y0..y3) of a [rows][32 floats] tensor into 512 contiguous bytes.
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* map, uint32_t y0,
                                            uint32_t y1, uint32_t y2, uint32_t y3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(map), "r"(0), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(bar)
      : "memory");
}

// Per-warp gather pipeline: two stage buffers and their mbarriers.
struct GatherPipe {
  float* buf;          // [2][kStage][32] in shared memory
  uint32_t bar[2];     // shared addresses of the two mbarriers
  uint32_t phase;      // bit b: parity to wait for on buffer b
};

// Issue one stage: entries [k0, k0 + n) with row indices idx (lane j holds
// entry j's index; lanes >= n hold 0, a valid row).  Warp-collective.
__device__ __forceinline__ void pipe_issue(GatherPipe& gp, int b, const CUtensorMap* map,
                                           uint32_t idx, uint32_t n, uint32_t lane) {
  const uint32_t ng = (n + 3) / 4;
  const uint32_t y0 = __shfl_sync(0xffffffffu, idx, (4 * lane) & 31);
  const uint32_t y1 = __shfl_sync(0xffffffffu, idx, (4 * lane + 1) & 31);
  const uint32_t y2 = __shfl_sync(0xffffffffu, idx, (4 * lane + 2) & 31);
  const uint32_t y3 = __shfl_sync(0xffffffffu, idx, (4 * lane + 3) & 31);
  if (lane == 0) mbar_expect(gp.bar[b], ng * 512u);
  __syncwarp();
  // the buffer was last read through the generic proxy; order those reads
  // before the async-proxy writes of the new stage
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane < ng)
    tma_gather4(smem_u32(gp.buf + b * kStage * 32 + lane * 4 * 32), map, y0, y1, y2, y3, gp.bar[b]);
}

// Wait for stage buffer b; false if the wait gave up (the error is recorded
// in *err and a second bounded wait lets the copies in flight land).
__device__ __forceinline__ bool pipe_wait(GatherPipe& gp, int b, unsigned int* err) {
  const uint32_t par = (gp.phase >> b) & 1u;
  bool ok = mbar_wait(gp.bar[b], par);
  if (!ok) {
    atomicOr(err, 2u);
    mbar_wait(gp.bar[b], par);
  }
  gp.phase ^= 1u << b;
  return ok;
}

}  // namespace ahpp
