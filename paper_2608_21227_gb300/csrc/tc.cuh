// tc.cuh -- 5th-generation tensor-core building blocks for sm_103a:
// tensor memory (TMEM) allocation, UMMA shared-memory and instruction
// descriptors, tcgen05.mma issue/commit, TMEM loads and stores, mbarrier waits.
//
// Operands live in shared memory in the canonical K-major layout without
// swizzle: a "core matrix" is 8 rows x 16 bytes stored as 8 consecutive 16-byte
// rows; core matrices adjacent along K are LBO bytes apart, 8-row groups are
// SBO bytes apart.  This file packs K-adjacent core matrices contiguously
// (LBO = 128) and 8-row groups one after another (SBO = 8 * row bytes), so
// element (r, k) of an operand with `rowbytes` bytes per row sits at
//   (r % 8) * 16 + (r / 8) * SBO + (k * es) % 16 + ((k * es) / 16) * 128.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace nla {
namespace tc {

NLA_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) of a K-major operand with `rowbytes` bytes per row.
NLA_DEV uint32_t kmajor_off(int r, int k, int es, int rowbytes) {
    const int kb = k * es;
    return (uint32_t)((r & 7) * 16 + (r >> 3) * (rowbytes * 8) + (kb & 15) + (kb >> 4) * 128);
}

// UMMA shared-memory descriptor: start address, LBO, SBO (bytes), version 1, no swizzle.
NLA_DEV uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// UMMA shared-memory descriptor of a K-major operand in the 128-byte-swizzled
// layout a TMA box with 128-byte rows produces: rows of 128 bytes, 8-row groups
// 1024 bytes apart (SBO), 16-byte chunks XOR-ed with (row & 7); the group base
// must be 1024-byte aligned.  Successive K steps advance the start address by
// their byte offset within the 128-byte row.
NLA_DEV uint64_t sdesc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Instruction descriptor: D = FP32, A and B of format `fmt` (kind::tf32: 2;
// kind::f16 with BF16 operands: 1), both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// ---- TMEM (one full warp executes alloc / dealloc)
NLA_DEV void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
NLA_DEV void tmem_relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
NLA_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
NLA_DEV void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
NLA_DEV void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
NLA_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- MMA issue (one thread): D[tmem] (+)= A[smem] * B[smem]
NLA_DEV void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
NLA_DEV void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
// D[tmem] (+)= A[tmem] * B[smem]: A's M rows in TMEM lanes 0..127, its K entries in
// consecutive 32-bit columns from a_tmem (kind::tf32: one entry per column).
NLA_DEV void mma_tf32_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t id, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
// arrive on the mbarrier once every previously issued MMA of this thread completed
NLA_DEV void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

// ---- mbarrier
NLA_DEV void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
NLA_DEV bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and kInfoTimeout in *info) when the budget runs out.
NLA_DEV bool mbar_wait(uint64_t *mbar, uint32_t parity, int *info) {
    if (mbar_try_wait(mbar, parity)) return true;
    unsigned long long t0 = global_ns();
    while (!mbar_try_wait(mbar, parity)) {
        if (global_ns() - t0 > kSpinBudgetNs) {
            if (info) atomicExch(info, kInfoTimeout);
            return false;
        }
    }
    return true;
}

// Warp-uniform bounded wait: lane 0 waits, the outcome is broadcast so the
// warp-collective TMEM loads that follow are executed by all lanes or none.
NLA_DEV bool mbar_wait_warp(uint64_t *mbar, uint32_t parity, int *info) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(mbar, parity, info) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Wait by every lane of a warp, with no warp shuffle on the way: each lane polls the
// phase itself; lane 0 alone keeps the time budget and, when it runs out, records
// kInfoTimeout and raises *abort (a shared-memory flag the other lanes poll too), so the
// whole warp gives up.  For loops whose per-stage latency matters.
NLA_DEV bool mbar_wait_lanes(uint64_t *mbar, uint32_t parity, int *info, volatile int *abort) {
    if (mbar_try_wait(mbar, parity)) return true;
    const bool leader = (threadIdx.x & 31) == 0;
    const unsigned long long t0 = leader ? global_ns() : 0ull;
    while (!mbar_try_wait(mbar, parity)) {
        if (*abort) return false;
        if (leader && global_ns() - t0 > kSpinBudgetNs) {
            if (info) atomicExch(info, kInfoTimeout);
            *abort = 1;
            return false;
        }
    }
    return true;
}

// ---- TMEM -> registers: this warp's 32 lanes, 16 consecutive 32-bit columns
NLA_DEV void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
NLA_DEV void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- registers -> TMEM: this warp's 32 lanes, 32 consecutive 32-bit columns from taddr
NLA_DEV void tmem_st32(uint32_t taddr, const float v[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
        "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
        "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
        "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
        "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
        "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
}
NLA_DEV void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- operand conversion (round to nearest; TF32 keeps 10 mantissa bits)
NLA_DEV uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
NLA_DEV uint16_t to_bf16(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

}  // namespace tc
}  // namespace nla
