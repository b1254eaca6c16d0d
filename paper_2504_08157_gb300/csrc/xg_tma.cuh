// xg_tma.cuh -- tensor-memory-accelerator (TMA) loads as inline PTX, and the
// host-side encoding of their tensor maps.
//
// A tensor map describes a tiled view of a global array (rank, extents,
// byte strides, box size); one thread issues cp.async.bulk.tensor for a box
// at given coordinates, the bytes land in shared memory and complete a
// transaction count on an mbarrier.  Rules these loads follow: the global
// base is 16-byte aligned, every stride a multiple of 16 bytes, the box's
// inner extent a multiple of 16 bytes, and the innermost coordinate of each
// load times the element size a multiple of 16 bytes (negative or
// out-of-range coordinates are allowed for loads and read zeros).  The maps
// cover this GPU's own memory only; no multicast.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

#include "xg_tc.cuh"

namespace xg {
namespace tma {

// the mbarrier at bar expects `bytes` more transaction bytes; this thread's
// arrival counts once
__device__ __forceinline__ void arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// the box of the 4-D map at coordinates (c0 innermost .. c3) into shared
// memory at dst; completes on the mbarrier at bar
__device__ __forceinline__ void load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                        uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy ones (a TMA load into a buffer that threads wrote)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tma

// Host: a 4-D FP32 tensor map over a [d3][d2][d1][d0] array (d0 contiguous)
// with box (b0, b1, b2, b3); zeros outside.  False when the driver entry
// point is missing or the encoding is refused (a stride or alignment rule).
bool encode_tma_4d_f32(CUtensorMap* map, const float* base, const uint64_t dims[4], const uint32_t box[4]);

}  // namespace xg
