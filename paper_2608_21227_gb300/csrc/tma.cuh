// tma.cuh -- Tensor Memory Accelerator (TMA) building blocks for sm_103a:
// tiled 2-D bulk loads into shared memory that complete on an mbarrier,
// bulk stores back to global memory, bulk-group waits, and the host-side
// tensor-map encoder (resolved through the runtime's driver entry point, so
// the library does not link libcuda).
//
// Alignment rules the callers guarantee: the tensor's base address and every
// row stride are multiples of 16 bytes, and the innermost coordinate of every
// copy times the element size is a multiple of 16 bytes.  A box load always
// delivers (and signals) the full box; elements outside the tensor read as 0.
// Stores clip at the tensor's edges.  A 128-byte-swizzled box must start on a
// 1024-byte boundary in shared memory.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "common.cuh"
#include "tc.cuh"

namespace nla {
namespace tma {

using tc::smem_u32;

NLA_DEV void load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}
NLA_DEV void store_2d(const CUtensorMap *map, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
NLA_DEV void commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// every committed store has finished reading shared memory
NLA_DEV void wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store has completed
NLA_DEV void wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
NLA_DEV void prefetch_map(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

NLA_DEV void expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
NLA_DEV void arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// barrier initialisation visible to the async proxy (TMA complete_tx)
NLA_DEV void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

}  // namespace tma

// Host: encode a 2-D tiled tensor map over a dim0 x dim1 array (dim0 contiguous,
// consecutive dim1 entries `stride_bytes` apart) with a box of box0 x box1
// elements.  Returns false when the driver rejects the layout.
bool tma_encode_2d(CUtensorMap *map, const void *base, int elem_bytes, uint64_t dim0, uint64_t dim1,
                   uint64_t stride_bytes, uint32_t box0, uint32_t box1, bool swizzle128);

}  // namespace nla
