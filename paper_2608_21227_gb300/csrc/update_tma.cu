// update_tma.cu -- FP32 trailing update (Algorithm 2, both sides) streamed
// through the Tensor Memory Accelerator.
//
// At band widths 16-64 an FP32 update pass reads (and the last one writes) the
// whole trailing matrix for 2*nb flops per element, so it is bound by HBM and
// by how many bytes each SM keeps in flight.  Every kernel here is one
// producer warp that streams tiles of X into a ring of shared-memory stages
// with TMA (completion on an mbarrier per stage) and consumer warps that work
// on each stage as it lands:
//
//   qr_proj       W = V^T X (QR side, reduction over rows).  A lane owns 4
//                 columns of a 128-column strip and 16 reflectors; per 4-row
//                 chunk, one 128-bit load of X per column and 16 broadcast
//                 128-bit loads of V feed 256 FMAs.
//   lq_proj       Y = X V (LQ side, reduction over columns).  A lane owns
//                 64/nb rows and all nb reflectors; per column, one load of X
//                 and nb/4 broadcast loads of V(c, :) feed 64 FMAs.
//   strip_update  X -= P Q^T (QR: P = V, Q = W'^T; LQ: P = Y', Q = V).  A lane
//                 keeps P(its 64/nb rows, :) in registers and streams columns;
//                 the producer writes each finished stage back with a TMA store.
//   qr_proj_tc    W = V^T X on the tensor cores (the default QR projection):
//                 tcgen05 kind::tf32 MMAs on the TMA boxes, FP32 accuracy from
//                 the three-term hi/lo split, accumulator in TMEM.
//
// The projections are split over the long dimension; the last block of each
// strip (atomic ticket, nobody waits) sums the partials in a fixed order and
// applies T (step 2 of Algorithm 2).
//
// X tiles are boxes of 32 rows (128 bytes) by `tc` columns with the 128-byte
// swizzle: column j of a box is a 128-byte row whose 16-byte chunk q is stored
// at chunk q ^ (j & 7), so a quarter warp reading chunk q of 8 consecutive
// columns, or chunks 0..7 of one column, touches 8 distinct bank groups.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "kernels.cuh"
#include "tma.cuh"

namespace nla {

// ------------------------------------------------------------------ host: tensor maps
bool tma_encode_2d(CUtensorMap *map, const void *base, int elem_bytes, uint64_t dim0, uint64_t dim1,
                   uint64_t stride_bytes, uint32_t box0, uint32_t box1, bool swizzle128) {
    // the driver entry point is the same for every device: looked up once (thread-safe)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        PFN_cuTensorMapEncodeTiled_v12000 f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        cudaGetLastError();
        return f;
    }();
    if (!encode || dim0 == 0 || dim1 == 0) return false;
    if (reinterpret_cast<uintptr_t>(base) % 16 || stride_bytes % 16) return false;
    const cuuint64_t dims[2] = {dim0, dim1};
    const cuuint64_t strides[1] = {stride_bytes};
    const cuuint32_t box[2] = {box0, box1};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = encode(map, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

constexpr int kBoxRows = 32;       // rows of an X box: 128 bytes of FP32
constexpr int kMaxStages = 8;
constexpr int kMaxSplitTma = 8;    // partial slabs (matches the tiled path's scratch layout)
constexpr int kMaxThreads = 288;   // producer + up to 8 consumer warps
constexpr size_t kTmaSmemLimit = 226 * 1024;  // dynamic bytes (the kernels' static shared memory is < 1 KB)

// Reflector entry of a unit lower-trapezoidal V: 1 on the diagonal, 0 above it.
NLA_DEV float unit_lower(int r, int k, float v) { return r > k ? v : (r == k ? 1.f : 0.f); }

NLA_DEV unsigned char *align1k(unsigned char *p) {
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// The block's abort flag as the warp sees it: lane 0 reads it and the value is broadcast,
// so a warp leaves its loop as a whole (the warp-collective operations after the loop
// then see every lane).
NLA_DEV bool abort_seen(const int *flag) { return __shfl_sync(0xffffffffu, *(volatile const int *)flag, 0) != 0; }

// Named barrier over the consumer warps (ids 1..; 0 is __syncthreads).
NLA_DEV void consumers_sync(int nc) { asm volatile("bar.sync 1, %0;" ::"r"(nc * 32) : "memory"); }

// Producer exit path: wait (bounded) until the last load issued into every
// stage has landed, so no copy is in flight when the block leaves.
NLA_DEV void drain_loads(uint64_t *full, int issued, int S, int *info) {
    for (int t = max(0, issued - S); t < issued; ++t) tc::mbar_wait(&full[t % S], (uint32_t)((t / S) & 1), info);
}

// Lane's RL floats of column j of a 32*RL-row X stage (RL boxes of 32 rows, tc
// columns each, 128-byte swizzle): rows RL*lane .. RL*lane + RL - 1.
template <int RL>
NLA_DEV float *xptr_rows(unsigned char *xs, int tcols, int j, int lane) {
    const int row = RL * lane, box = row >> 5, rib = row & 31;
    return reinterpret_cast<float *>(xs + (size_t)box * tcols * 128 + j * 128 + ((((rib >> 2) ^ (j & 7))) << 4) +
                                     (rib & 3) * 4);
}
template <int RL>
NLA_DEV void ld_rows(const float *p, float x[RL]) {
    if constexpr (RL == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
    } else if constexpr (RL == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        x[0] = v.x, x[1] = v.y;
    } else {
        x[0] = *p;
    }
}
template <int RL>
NLA_DEV void st_rows(float *p, const float x[RL]) {
    if constexpr (RL == 4)
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    else if constexpr (RL == 2)
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    else
        *p = x[0];
}

// ------------------------------------------------------------------ qr_proj
// Block (strip, s): partial W(:, strip) = V(rows of split s, :)^T X(rows, strip)
// over `nt` stages of BR*32 rows; last block of the strip: W' = T^T W -> fin
// (column-major by strip column: fin[c*NB + k]).
template <int NB>
__global__ void __launch_bounds__(kMaxThreads, 1)
qr_proj_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV, int M, int N,
               const float *__restrict__ Tm, int BR, int RW, int S, int Ms, float *part, float *fin,
               unsigned int *tickets, int *info) {
    pdl_wait();
    pdl_trigger();
    constexpr int RG = NB / 16;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], done[kMaxStages];
    __shared__ int sh_last, sh_abort;
    unsigned char *base = align1k(smem_raw);
    const int NC = RG * RW;
    const int xbytes = 128 * 128, vbytes = NB * 128;  // one 32-row box of X (128 columns) and of V
    const int stage = BR * (xbytes + vbytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c0 = blockIdx.x * 128, wc = min(128, N - c0);
    const int s = blockIdx.y, nsplit = gridDim.y;
    const int rbeg = s * Ms, rend = min(M, rbeg + Ms);
    const int th = BR * kBoxRows;
    const int nt = (rend - rbeg + th - 1) / th;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&done[i], NC);
        }
        sh_abort = 0;
        tma::fence_init();
        tma::prefetch_map(&tmX);
        tma::prefetch_map(&tmV);
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nt; ++t) {
                const int st = t % S;
                if (t >= S && !tc::mbar_wait(&done[st], (uint32_t)(((t / S) - 1) & 1), info)) {
                    sh_abort = 1;
                    break;
                }
                unsigned char *sb = base + (size_t)st * stage;
                tma::expect_tx(&full[st], (uint32_t)stage);
                const int r0 = rbeg + t * th;
                for (int bx = 0; bx < BR; ++bx) {
                    tma::load_2d(sb + bx * xbytes, &tmX, r0 + bx * kBoxRows, c0, &full[st]);
                    tma::load_2d(sb + BR * xbytes + bx * vbytes, &tmV, r0 + bx * kBoxRows, 0, &full[st]);
                }
                issued = t + 1;
            }
            drain_loads(full, issued, S, info);
        }
    } else {
        const int cw = warp - 1, rg = cw % RG, rw = cw / RG;
        float acc[16][4];
#pragma unroll
        for (int a = 0; a < 16; ++a)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[a][i] = 0.f;
        for (int t = 0; t < nt; ++t) {
            const int st = t % S;
            if (!tc::mbar_wait_warp(&full[st], (uint32_t)((t / S) & 1), info) || abort_seen(&sh_abort)) break;
            const unsigned char *sb = base + (size_t)st * stage;
            const int r0 = rbeg + t * th;  // trailing-matrix row of the stage's first row
            const bool diag_stage = r0 < NB;  // only the stage holding V's unit diagonal needs masking
            for (int q = rw; q < 8 * BR; q += RW) {
                const int bx = q >> 3, qq = q & 7;
                const unsigned char *xb = sb + bx * xbytes;
                float4 x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    x[i] = *reinterpret_cast<const float4 *>(xb + (lane + 32 * i) * 128 + ((qq ^ (lane & 7)) << 4));
                const float *vb = reinterpret_cast<const float *>(sb + BR * xbytes + bx * vbytes) + (16 * rg) * 32 + 4 * qq;
                if (!diag_stage) {
#pragma unroll
                    for (int a = 0; a < 16; ++a) {
                        const float4 v = *reinterpret_cast<const float4 *>(vb + a * 32);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float s4 = acc[a][i];
                            s4 = fmaf(v.x, x[i].x, s4);
                            s4 = fmaf(v.y, x[i].y, s4);
                            s4 = fmaf(v.z, x[i].z, s4);
                            acc[a][i] = fmaf(v.w, x[i].w, s4);
                        }
                    }
                } else {
                    const int rq = r0 + bx * kBoxRows + 4 * qq;
#pragma unroll
                    for (int a = 0; a < 16; ++a) {
                        float4 v = *reinterpret_cast<const float4 *>(vb + a * 32);
                        const int k = 16 * rg + a;
                        v.x = unit_lower(rq, k, v.x), v.y = unit_lower(rq + 1, k, v.y);
                        v.z = unit_lower(rq + 2, k, v.z), v.w = unit_lower(rq + 3, k, v.w);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float s4 = acc[a][i];
                            s4 = fmaf(v.x, x[i].x, s4);
                            s4 = fmaf(v.y, x[i].y, s4);
                            s4 = fmaf(v.z, x[i].z, s4);
                            acc[a][i] = fmaf(v.w, x[i].w, s4);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) tma::arrive(&done[st]);
        }
        // reduce the RW row groups in a fixed order into red[NB][128] (stage memory is free now)
        float *red = reinterpret_cast<float *>(base);
        consumers_sync(NC);
        for (int g = 0; g < RW; ++g) {
            if (rw == g) {
#pragma unroll
                for (int a = 0; a < 16; ++a)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float *p = red + (16 * rg + a) * 128 + lane + 32 * i;
                        *p = g == 0 ? acc[a][i] : *p + acc[a][i];
                    }
            }
            consumers_sync(NC);
        }
        for (int idx = tid - 32; idx < NB * 128; idx += NC * 32) {
            const int k = idx >> 7, c = idx & 127;
            if (c < wc) part[((size_t)s * NB + k) * N + c0 + c] = red[idx];
        }
    }
    __threadfence();
    __syncthreads();
    if (sh_abort) return;
    if (tid == 0) sh_last = atomicAdd(&tickets[blockIdx.x], 1u) == (unsigned)(nsplit - 1);
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    float *W = reinterpret_cast<float *>(base);
    for (int idx = tid; idx < NB * 128; idx += blockDim.x) {
        const int k = idx >> 7, c = idx & 127;
        float sum = 0.f;
        if (c < wc)
#pragma unroll
            for (int q = 0; q < kMaxSplitTma; ++q)  // (all partial loads in flight at once)
                if (q < nsplit) sum += __ldcg(part + ((size_t)q * NB + k) * N + c0 + c);
        W[idx] = sum;
    }
    __syncthreads();
    for (int idx = tid; idx < NB * wc; idx += blockDim.x) {
        const int k = idx % NB, c = idx / NB;
        float sum = 0.f;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j <= k) sum = fmaf(__ldg(Tm + j + (size_t)k * NB), W[j * 128 + c], sum);
        fin[(size_t)(c0 + c) * NB + k] = sum;
    }
    if (tid == 0) tickets[blockIdx.x] = 0u;
}

// ------------------------------------------------------------------ projections on the tensor cores
// QR side: W^T (128 strip columns x NB) = X_strip^T V; LQ side: Y (128 strip rows x NB)
// = X_strip V.  Both accumulate in TMEM with tcgen05 kind::tf32 MMAs (M = 128, K = 8 per
// instruction) and reach FP32 accuracy by the three-term split x = hi + lo (hi = x with
// the low 13 mantissa bits cleared, what the tensor core reads of an FP32 word; lo = x -
// hi, exact): x . v ~ hi_x (hi_v + lo_v) + lo_x hi_v -- the dropped lo_x lo_v term and the
// truncation of lo are below 2^-21 relative.  The first product runs as one MMA with
// N = 2 NB against the stacked operand [V_hi; V_lo] (its two halves of D are summed at
// the end), so a K step is two MMAs.
//
// Persistent blocks, one per SM: block b takes work items b, b + G, ... (item = strip x
// split of the reduction dimension) and streams their 32-deep K tiles through two rings:
//   landing ring (SL stages, deep): TMA boxes of X and V exactly as they arrive, so many
//                 bytes are in flight per SM whatever the converter and MMA latency;
//   operand ring (2 stages): what the MMAs read besides the landing tile -- the lo copy of
//                 X (QR side: the landing box is already the K-major operand, hi = the raw
//                 word) or hi and lo copies of X transposed to K-major (LQ side), and the
//                 stacked [V_hi; V_lo] with V's unit diagonal applied.
// Roles: warp 0 issues the TMA loads; warp 1 owns TMEM and one lane issues the MMAs (each
// tile's commits free its landing stage and its operand stage); warps 2..5 convert, then
// per item read the accumulator back (each warp its TMEM lane quadrant), write the split's
// partial and take a per-warp ticket: the last of the strip's 4 x nsplit arrivals sums the
// partials in split order and applies T (Algorithm 2, step 2).  Every wait is bounded.
constexpr int kTcWarps = 6;
constexpr int kLanding = 12;  // most landing stages
constexpr int kMaxOp = 6;     // most operand stages

NLA_DEV float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
NLA_DEV float4 tf32_lo4(float4 v) {
    return make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
}

// Shared-memory plan of the tensor-core projections (bytes).
__host__ __device__ constexpr int proj_land_bytes(int nb) { return 16384 + nb * 128; }
__host__ __device__ constexpr int proj_op_bytes(int side, int nb) { return (side == 0 ? 16384 : 32768) + 2 * nb * 128; }

template <int NB, int SIDE>
__global__ void __launch_bounds__(32 * kTcWarps, 1)
proj_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV, int M, int N,
               const float *__restrict__ Tm, int SL, int SO, int nsplit, int Ks, float *part, float *fin,
               unsigned int *tickets, int *info) {
    pdl_wait();
    pdl_trigger();
    constexpr uint32_t kCols = 2 * NB < 32 ? 32 : 2 * NB;  // TMEM columns (power of two >= 32)
    constexpr int LB = proj_land_bytes(NB), OB = proj_op_bytes(SIDE, NB);
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kLanding], lempty[kLanding], conv[kMaxOp], oempty[kMaxOp], accfull,
        accdone;
    __shared__ uint32_t tmem_base;
    __shared__ int sh_abort;
    unsigned char *base = align1k(smem_raw);
    unsigned char *ops = base + (size_t)SL * LB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // strip lines: QR -> columns of X, LQ -> rows; reduction dimension: the other one
    const int Lext = SIDE == 0 ? N : M, Kext = SIDE == 0 ? M : N;
    const int nstrip = (Lext + 127) / 128, nitems = nstrip * nsplit;
    if (tid == 0) {
        for (int i = 0; i < SL; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&lempty[i], 1);
        }
        for (int i = 0; i < SO; ++i) {
            tc::mbar_init(&conv[i], 4);
            tc::mbar_init(&oempty[i], 1);
        }
        tc::mbar_init(&accfull, 1);
        tc::mbar_init(&accdone, 1);
        sh_abort = 0;
        tma::fence_init();
        tma::prefetch_map(&tmX);
        tma::prefetch_map(&tmV);
    }
    if (warp == 1) {
        tc::tmem_alloc(&tmem_base, kCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    auto land = [&](int st) { return base + (size_t)st * LB; };
    auto opst = [&](int ot) { return ops + (size_t)ot * OB; };
    auto ktiles = [&](int it) {
        const int kb = (it % nsplit) * Ks;
        return (min(Kext, kb + Ks) - kb + 31) / 32;
    };

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int it = blockIdx.x; ok && it < nitems; it += gridDim.x) {
                const int l0 = (it / nsplit) * 128, kb = (it % nsplit) * Ks, nt = ktiles(it);
                for (int t = 0; t < nt; ++t, ++g) {
                    const int st = g % SL;
                    if (g >= SL && !tc::mbar_wait(&lempty[st], (uint32_t)(((g / SL) - 1) & 1), info)) {
                        sh_abort = 1;
                        ok = false;
                        break;
                    }
                    unsigned char *sb = land(st);
                    tma::expect_tx(&full[st], (uint32_t)LB);
                    const int k0 = kb + 32 * t;
                    if (SIDE == 0) {
                        tma::load_2d(sb, &tmX, k0, l0, &full[st]);            // 32 rows x 128 columns
                        tma::load_2d(sb + 16384, &tmV, k0, 0, &full[st]);     // V rows k0.., NB columns
                    } else {
                        for (int bx = 0; bx < 4; ++bx)                         // 128 rows x 32 columns
                            tma::load_2d(sb + bx * 4096, &tmX, l0 + 32 * bx, k0, &full[st]);
                        tma::load_2d(sb + 16384, &tmV, 0, k0, &full[st]);     // V^T: NB x 32 columns
                    }
                }
            }
            drain_loads(full, g, SL, info);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id2 = tc::idesc(2, 128, 2 * NB), id1 = tc::idesc(2, 128, NB);
            int g = 0;
            bool ok = true;
            for (int it = blockIdx.x; ok && it < nitems; it += gridDim.x) {
                const int nt = ktiles(it);
                for (int t = 0; t < nt; ++t, ++g) {
                    const int st = g % SL, ot = g % SO;
                    if (*(volatile int *)&sh_abort ||
                        !tc::mbar_wait(&conv[ot], (uint32_t)((g / SO) & 1), info)) {
                        sh_abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t o = tc::smem_u32(opst(ot));
                    // A_hi: the landing box (QR) or the transposed hi copy (LQ); A_lo; [V_hi; V_lo]
                    const uint32_t ah = SIDE == 0 ? tc::smem_u32(land(st)) : o;
                    const uint32_t al = SIDE == 0 ? o : o + 16384;
                    const uint32_t bv = o + (SIDE == 0 ? 16384 : 32768);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {  // 8 TF32 = 32 bytes of K per instruction
                        const uint32_t off = kk * 32;
                        tc::mma_tf32(tbase, tc::sdesc_sw128(ah + off), tc::sdesc_sw128(bv + off), id2,
                                     (t > 0 || kk > 0) ? 1u : 0u);
                        tc::mma_tf32(tbase, tc::sdesc_sw128(al + off), tc::sdesc_sw128(bv + off), id1, 1u);
                    }
                    tc::mma_commit(&lempty[st]);  // free once these MMAs have read them
                    tc::mma_commit(&oempty[ot]);
                }
                if (ok) tc::mma_commit(&accfull);  // this item's accumulator is complete
            }
            tc::mma_commit(&accdone);  // every issued MMA has completed
        }
        __syncwarp();
    } else {
        const int ct = tid - 64;  // 0..127
        const int q = warp & 3;   // TMEM lanes 32q .. 32q + 31 (the warp's quadrant)
        int g = 0, li = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++li) {
            const int strip = it / nsplit, sp = it % nsplit;
            const int l0 = strip * 128, lw = min(128, Lext - l0);
            const int kb = sp * Ks, nt = ktiles(it);
            bool ok = true;
            for (int t = 0; t < nt; ++t, ++g) {
                const int st = g % SL, ot = g % SO;
                if (!tc::mbar_wait_warp(&full[st], (uint32_t)((g / SL) & 1), info) ||
                    (g >= SO && !tc::mbar_wait_warp(&oempty[ot], (uint32_t)(((g / SO) - 1) & 1), info)) ||
                    abort_seen(&sh_abort)) {
                    ok = false;
                    break;
                }
                const int k0 = kb + 32 * t;  // reduction index of the tile's first entry
                unsigned char *sb = land(st), *ob = opst(ot);
                if (SIDE == 0) {
                    // lo copy of the X box (same K-major swizzled layout)
                    const float4 *xs = reinterpret_cast<const float4 *>(sb);
                    float4 *xl = reinterpret_cast<float4 *>(ob);
#pragma unroll 4
                    for (int e = ct; e < 1024; e += 128) xl[e] = tf32_lo4(xs[e]);
                    // V: entry (r, k) of the box is row k, 16-byte chunk (r/4) ^ (k & 7), word r % 4;
                    // unit diagonal applied (r == k: 1, r < k: 0), hi copy and lo stacked
                    const float4 *vs = reinterpret_cast<const float4 *>(sb + 16384);
                    float4 *vh = reinterpret_cast<float4 *>(ob + 16384);
                    float4 *vl = reinterpret_cast<float4 *>(ob + 16384 + NB * 128);
                    for (int e = ct; e < NB * 8; e += 128) {
                        float4 v = vs[e];
                        if (k0 < NB) {
                            const int k = e >> 3, rr = 4 * ((e & 7) ^ (k & 7)), r = k0 + rr;
                            v.x = unit_lower(r, k, v.x), v.y = unit_lower(r + 1, k, v.y);
                            v.z = unit_lower(r + 2, k, v.z), v.w = unit_lower(r + 3, k, v.w);
                        }
                        vh[e] = v;
                        vl[e] = tf32_lo4(v);
                    }
                } else {
                    // X (column-major boxes of 32 rows) -> K-major rows of 32 columns: row r,
                    // 16-byte chunk c4 ^ (r & 7) holds columns 4 c4 .. 4 c4 + 3
                    const int r = ct, box = r >> 5, rib = r & 31;
                    const unsigned char *xb = sb + box * 4096;
                    unsigned char *ah = ob + r * 128, *al = ob + 16384 + r * 128;
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4) {
                        float x4[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int j = 4 * c4 + i;
                            x4[i] = *reinterpret_cast<const float *>(xb + j * 128 + ((((rib >> 2) ^ (j & 7))) << 4) +
                                                                     (rib & 3) * 4);
                        }
                        const float4 v = make_float4(x4[0], x4[1], x4[2], x4[3]);
                        const int ch = (c4 ^ (r & 7)) << 4;
                        *reinterpret_cast<float4 *>(ah + ch) = v;
                        *reinterpret_cast<float4 *>(al + ch) = tf32_lo4(v);
                    }
                    // V^T box (column c: NB consecutive reflector entries) -> rows k of 32
                    // columns, unit diagonal applied (global column c: c == k -> 1, c < k -> 0)
                    const float *vs = reinterpret_cast<const float *>(sb + 16384);
                    unsigned char *vh = ob + 32768, *vl = ob + 32768 + NB * 128;
                    for (int e = ct; e < NB * 8; e += 128) {
                        const int k = e >> 3, c4 = e & 7;
                        float x4[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int j = 4 * c4 + i;
                            const float v = vs[j * NB + k];
                            x4[i] = k0 < NB ? unit_lower(k0 + j, k, v) : v;
                        }
                        const float4 v = make_float4(x4[0], x4[1], x4[2], x4[3]);
                        const int ch = k * 128 + ((c4 ^ (k & 7)) << 4);
                        *reinterpret_cast<float4 *>(vh + ch) = v;
                        *reinterpret_cast<float4 *>(vl + ch) = tf32_lo4(v);
                    }
                }
                tc::fence_async_smem();  // the copies -> visible to the tensor core
                __syncwarp();
                if (lane == 0) tma::arrive(&conv[ot]);
            }
            if (!ok) {
                if (lane == 0) sh_abort = 1;
                break;
            }
            // ---- epilogue of the item: this warp's 32 strip lines of the partial
            if (!tc::mbar_wait_warp(&accfull, (uint32_t)(li & 1), info)) {
                if (lane == 0) sh_abort = 1;
                break;
            }
            tc::fence_after_sync();
            const int line = 32 * q + lane;
#pragma unroll
            for (int c = 0; c < NB; c += 16) {
                float w1[16], w2[16];
                tc::tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)c, w1);
                tc::tmem_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(NB + c), w2);
                tc::tmem_wait_ld();
                if (line < lw) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) part[((size_t)sp * NB + c + k) * Lext + l0 + line] = w1[k] + w2[k];
                }
            }
            tc::fence_before_sync();  // (the next item's MMAs start only after this warp's next arrive)
            // per-warp ticket: the last of the strip's 4 x nsplit arrivals finishes the strip
            __threadfence();
            __syncwarp();
            unsigned last = 0;
            if (lane == 0) last = atomicAdd(&tickets[strip], 1u) == (unsigned)(4 * nsplit - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            if (!last) continue;
            __threadfence();
            for (int l = lane; l < lw; l += 32) {
                float w[NB];
#pragma unroll
                for (int k = 0; k < NB; ++k) w[k] = 0.f;
#pragma unroll 1
                for (int qq = 0; qq < nsplit; ++qq) {  // fixed split order; a split's NB loads in flight together
                    const float *pp = part + (size_t)qq * NB * Lext + l0 + l;
#pragma unroll
                    for (int k = 0; k < NB; ++k) w[k] += __ldcg(pp + (size_t)k * Lext);
                }
                // QR: W'(:, c) = T^T W(:, c) -> fin[c * NB + k];  LQ: Y'(i, :) = Y(i, :) T -> fin[k * M + i]
#pragma unroll 1
                for (int k = 0; k < NB; ++k) {
                    float s = 0.f;
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        if (j <= k) s = fmaf(__ldg(Tm + j + (size_t)k * NB), w[j], s);
                    if (SIDE == 0)
                        fin[(size_t)(l0 + l) * NB + k] = s;
                    else
                        fin[(size_t)k * M + l0 + l] = s;
                }
            }
            if (lane == 0) tickets[strip] = 0u;
        }
    }
    // every issued MMA completes before TMEM is released
    if (warp == 1) tc::mbar_wait_warp(&accdone, 0, info);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tbase, kCols);
}

// ------------------------------------------------------------------ lq_proj
// Block (strip, s): partial Y(strip rows, :) = X(strip rows, columns of split s) V
// over stages of tc columns; last block of the strip: Y' = Y T -> fin[k*M + i].
template <int NB>
__global__ void __launch_bounds__(kMaxThreads, 1)
lq_proj_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ, int M, int N,
               const float *__restrict__ Tm, int tcols, int NC, int S, int Ns, float *part, float *fin,
               unsigned int *tickets, int *info) {
    pdl_wait();
    pdl_trigger();
    constexpr int RL = 64 / NB, H = 32 * RL;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], done[kMaxStages];
    __shared__ int sh_last, sh_abort;
    unsigned char *base = align1k(smem_raw);
    const int xbytes = tcols * 128, qbytes = tcols * NB * 4;
    const int stage = RL * xbytes + qbytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.x * H, hr = min(H, M - i0);
    const int s = blockIdx.y, nsplit = gridDim.y;
    const int cbeg = s * Ns, cend = min(N, cbeg + Ns);
    const int nt = (cend - cbeg + tcols - 1) / tcols;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&done[i], NC);
        }
        sh_abort = 0;
        tma::fence_init();
        tma::prefetch_map(&tmX);
        tma::prefetch_map(&tmQ);
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nt; ++t) {
                const int st = t % S;
                if (t >= S && !tc::mbar_wait(&done[st], (uint32_t)(((t / S) - 1) & 1), info)) {
                    sh_abort = 1;
                    break;
                }
                unsigned char *sb = base + (size_t)st * stage;
                tma::expect_tx(&full[st], (uint32_t)stage);
                const int cb = cbeg + t * tcols;
                for (int bx = 0; bx < RL; ++bx) tma::load_2d(sb + bx * xbytes, &tmX, i0 + bx * kBoxRows, cb, &full[st]);
                tma::load_2d(sb + RL * xbytes, &tmQ, 0, cb, &full[st]);
                issued = t + 1;
            }
            drain_loads(full, issued, S, info);
        }
    } else {
        const int cw = warp - 1;
        float acc[RL][NB];
#pragma unroll
        for (int a = 0; a < RL; ++a)
#pragma unroll
            for (int k = 0; k < NB; ++k) acc[a][k] = 0.f;
        for (int t = 0; t < nt; ++t) {
            const int st = t % S;
            if (!tc::mbar_wait_warp(&full[st], (uint32_t)((t / S) & 1), info) || abort_seen(&sh_abort)) break;
            unsigned char *sb = base + (size_t)st * stage;
            const float *qs = reinterpret_cast<const float *>(sb + RL * xbytes);
            const int cb = cbeg + t * tcols;
            if (cb >= NB) {  // no column of this stage meets V's unit diagonal
#pragma unroll 2
                for (int j = cw; j < tcols; j += NC) {
                    float x[RL];
                    ld_rows<RL>(xptr_rows<RL>(sb, tcols, j, lane), x);
#pragma unroll
                    for (int k4 = 0; k4 < NB; k4 += 4) {
                        const float4 q = *reinterpret_cast<const float4 *>(qs + j * NB + k4);
#pragma unroll
                        for (int a = 0; a < RL; ++a) {
                            acc[a][k4] = fmaf(x[a], q.x, acc[a][k4]);
                            acc[a][k4 + 1] = fmaf(x[a], q.y, acc[a][k4 + 1]);
                            acc[a][k4 + 2] = fmaf(x[a], q.z, acc[a][k4 + 2]);
                            acc[a][k4 + 3] = fmaf(x[a], q.w, acc[a][k4 + 3]);
                        }
                    }
                }
            } else {
                for (int j = cw; j < tcols; j += NC) {
                    float x[RL];
                    ld_rows<RL>(xptr_rows<RL>(sb, tcols, j, lane), x);
                    const int c = cb + j;
#pragma unroll
                    for (int k4 = 0; k4 < NB; k4 += 4) {
                        float4 q = *reinterpret_cast<const float4 *>(qs + j * NB + k4);
                        q.x = unit_lower(c, k4, q.x), q.y = unit_lower(c, k4 + 1, q.y);
                        q.z = unit_lower(c, k4 + 2, q.z), q.w = unit_lower(c, k4 + 3, q.w);
#pragma unroll
                        for (int a = 0; a < RL; ++a) {
                            acc[a][k4] = fmaf(x[a], q.x, acc[a][k4]);
                            acc[a][k4 + 1] = fmaf(x[a], q.y, acc[a][k4 + 1]);
                            acc[a][k4 + 2] = fmaf(x[a], q.z, acc[a][k4 + 2]);
                            acc[a][k4 + 3] = fmaf(x[a], q.w, acc[a][k4 + 3]);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) tma::arrive(&done[st]);
        }
        // reduce the NC column groups in a fixed order into red[NB][H]
        float *red = reinterpret_cast<float *>(base);
        consumers_sync(NC);
        for (int g = 0; g < NC; ++g) {
            if (cw == g) {
#pragma unroll
                for (int a = 0; a < RL; ++a)
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        float *p = red + k * H + RL * lane + a;
                        *p = g == 0 ? acc[a][k] : *p + acc[a][k];
                    }
            }
            consumers_sync(NC);
        }
        for (int idx = tid - 32; idx < NB * H; idx += NC * 32) {
            const int k = idx / H, i = idx % H;
            if (i < hr) part[((size_t)s * NB + k) * M + i0 + i] = red[idx];
        }
    }
    __threadfence();
    __syncthreads();
    if (sh_abort) return;
    if (tid == 0) sh_last = atomicAdd(&tickets[blockIdx.x], 1u) == (unsigned)(nsplit - 1);
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    float *Y = reinterpret_cast<float *>(base);
    for (int idx = tid; idx < NB * H; idx += blockDim.x) {
        const int k = idx / H, i = idx % H;
        float sum = 0.f;
        if (i < hr)
#pragma unroll
            for (int q = 0; q < kMaxSplitTma; ++q)  // (all partial loads in flight at once)
                if (q < nsplit) sum += __ldcg(part + ((size_t)q * NB + k) * M + i0 + i);
        Y[idx] = sum;
    }
    __syncthreads();
    for (int idx = tid; idx < NB * H; idx += blockDim.x) {
        const int k = idx / H, i = idx % H;
        if (i >= hr) continue;
        float sum = 0.f;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j <= k) sum = fmaf(Y[j * H + i], __ldg(Tm + j + (size_t)k * NB), sum);
        fin[(size_t)k * M + i0 + i] = sum;
    }
    if (tid == 0) tickets[blockIdx.x] = 0u;
}

// ------------------------------------------------------------------ strip_update
// Persistent: block b takes work items b, b + G, ... (item = strip of 32*RL rows x one
// column chunk of Ns columns) and streams their tiles through one ring of S stages.
// Item: X(strip rows, chunk columns) -= P(strip rows, :) Q(cols, :)^T.
// SIDE 0 (QR): P = V (unit lower, column-major at Pv, ld ldp), Q = W'^T from
// fin[c*NB + k].  SIDE 1 (LQ): P = Y' at Pv[k*M + i] (ldp unused), Q = V
// stored by rows (unit lower in (c, k)).
template <int NB, int SIDE>
__global__ void __maxnreg__(128)
strip_update_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ, int M, int N,
                    const float *__restrict__ Pv, long ldp, int tcols, int NC, int S, int Ns, int moff, int *info) {
    pdl_wait();
    pdl_trigger();
    constexpr int RL = 64 / NB, H = 32 * RL;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], done[kMaxStages];
    __shared__ int sh_abort;
    unsigned char *base = align1k(smem_raw);
    const int xbytes = tcols * 128, qbytes = tcols * NB * 4;
    const int stage = RL * xbytes + qbytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nstrip = (M + H - 1) / H, ncs = (N + Ns - 1) / Ns, nitems = nstrip * ncs;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&done[i], NC);
        }
        sh_abort = 0;
        tma::fence_init();
        tma::prefetch_map(&tmX);
        tma::prefetch_map(&tmQ);
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0) {
            // ring entry t holds tile (row i0, column cb) until it is stored back
            int ti0[kMaxStages], tcb[kMaxStages];
            int g = 0, stored = 0;
            bool ok = true;
            for (int it = blockIdx.x; ok && it < nitems; it += gridDim.x) {
                const int i0 = (it / ncs) * H, cbeg = (it % ncs) * Ns, cend = min(N, cbeg + Ns);
                for (int cb = cbeg; cb < cend; cb += tcols, ++g) {
                    const int st = g % S;
                    unsigned char *sb = base + (size_t)st * stage;
                    if (g >= S) {
                        // write back the tile that used this stage, then reuse it
                        if (!tc::mbar_wait(&done[st], (uint32_t)(((g / S) - 1) & 1), info)) {
                            sh_abort = 1;
                            ok = false;
                            break;
                        }
                        for (int bx = 0; bx < RL; ++bx) tma::store_2d(&tmX, ti0[st] + bx * kBoxRows, tcb[st], sb + bx * xbytes);
                        tma::commit();
                        stored = g - S + 1;
                        tma::wait_read_all();
                    }
                    tma::expect_tx(&full[st], (uint32_t)stage);
                    for (int bx = 0; bx < RL; ++bx) tma::load_2d(sb + bx * xbytes, &tmX, i0 + bx * kBoxRows, cb, &full[st]);
                    tma::load_2d(sb + RL * xbytes, &tmQ, 0, cb, &full[st]);
                    ti0[st] = i0;
                    tcb[st] = cb;
                }
            }
            const int issued = g;
            for (int t = stored; ok && t < issued; ++t) {
                const int st = t % S;
                if (!tc::mbar_wait(&done[st], (uint32_t)((t / S) & 1), info)) {
                    sh_abort = 1;
                    ok = false;
                    break;
                }
                for (int bx = 0; bx < RL; ++bx)
                    tma::store_2d(&tmX, ti0[st] + bx * kBoxRows, tcb[st], base + (size_t)st * stage + bx * xbytes);
                tma::commit();
            }
            if (!ok) drain_loads(full, issued, S, info);
            tma::wait_all();
        }
    } else {
        const int cw = warp - 1;
        int g = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            const int i0 = (it / ncs) * H, cbeg = (it % ncs) * Ns, cend = min(N, cbeg + Ns);
            // P(lane's rows, :) in registers
            float p[RL][NB];
#pragma unroll
            for (int a = 0; a < RL; ++a) {
                const int i = i0 + RL * lane + a;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    float v = 0.f;
                    if (i < M) {
                        if constexpr (SIDE == 0)
                            v = unit_lower(moff + i, k, moff + i > k ? __ldg(Pv + i + (long)k * ldp) : 0.f);
                        else
                            v = __ldg(Pv + (size_t)k * M + i);
                    }
                    p[a][k] = v;
                }
            }
            bool ok = true;
            for (int cb = cbeg; cb < cend; cb += tcols, ++g) {
                const int st = g % S;
                if (!tc::mbar_wait_warp(&full[st], (uint32_t)((g / S) & 1), info) || abort_seen(&sh_abort)) {
                    ok = false;
                    break;
                }
                unsigned char *sb = base + (size_t)st * stage;
                const float *qs = reinterpret_cast<const float *>(sb + RL * xbytes);
                if (SIDE == 0 || moff + cb >= NB) {  // no column of this stage meets V's unit diagonal
#pragma unroll 2
                    for (int j = cw; j < tcols; j += NC) {
                        float *xp = xptr_rows<RL>(sb, tcols, j, lane);
                        float x[RL];
                        ld_rows<RL>(xp, x);
                        float d[RL][4];  // four independent partial sums per row: short FMA chains
#pragma unroll
                        for (int a = 0; a < RL; ++a) d[a][0] = d[a][1] = d[a][2] = d[a][3] = 0.f;
#pragma unroll
                        for (int k4 = 0; k4 < NB; k4 += 4) {
                            const float4 q = *reinterpret_cast<const float4 *>(qs + j * NB + k4);
#pragma unroll
                            for (int a = 0; a < RL; ++a) {
                                d[a][0] = fmaf(p[a][k4], q.x, d[a][0]);
                                d[a][1] = fmaf(p[a][k4 + 1], q.y, d[a][1]);
                                d[a][2] = fmaf(p[a][k4 + 2], q.z, d[a][2]);
                                d[a][3] = fmaf(p[a][k4 + 3], q.w, d[a][3]);
                            }
                        }
#pragma unroll
                        for (int a = 0; a < RL; ++a) x[a] -= (d[a][0] + d[a][1]) + (d[a][2] + d[a][3]);
                        st_rows<RL>(xp, x);
                    }
                } else {
                    for (int j = cw; j < tcols; j += NC) {
                        float *xp = xptr_rows<RL>(sb, tcols, j, lane);
                        float x[RL];
                        ld_rows<RL>(xp, x);
                        const int c = moff + cb + j;  // global column: V's unit diagonal
#pragma unroll
                        for (int k4 = 0; k4 < NB; k4 += 4) {
                            float4 q = *reinterpret_cast<const float4 *>(qs + j * NB + k4);
                            q.x = unit_lower(c, k4, q.x), q.y = unit_lower(c, k4 + 1, q.y);
                            q.z = unit_lower(c, k4 + 2, q.z), q.w = unit_lower(c, k4 + 3, q.w);
#pragma unroll
                            for (int a = 0; a < RL; ++a) {
                                x[a] = fmaf(-p[a][k4], q.x, x[a]);
                                x[a] = fmaf(-p[a][k4 + 1], q.y, x[a]);
                                x[a] = fmaf(-p[a][k4 + 2], q.z, x[a]);
                                x[a] = fmaf(-p[a][k4 + 3], q.w, x[a]);
                            }
                        }
                        st_rows<RL>(xp, x);
                    }
                }
                tc::fence_async_smem();  // this lane's shared-memory writes -> visible to the TMA store
                __syncwarp();
                if (lane == 0) tma::arrive(&done[st]);
            }
            if (!ok) break;
        }
    }
}

// ------------------------------------------------------------------ host launch
int splits_for(int nstrip, int units, int waves) {
    const int target = waves * device_sm_count();
    return std::max(1, std::min({(target + nstrip - 1) / std::max(nstrip, 1), kMaxSplitTma, units}));
}

// Launch shape of the TMA kernels, read from a trailing-update configuration:
//   tile    -> stage depth: 32-row boxes of the QR projection (tile / 32) and
//              columns per stage of the column-streaming kernels (tile);
//   threads -> consumer threads (the producer warp comes on top);
//   cpb     -> pipeline stages;
//   unroll  -> waves of blocks the long-dimension splits aim for.
struct TmaShape {
    int br, rw;  // qr_proj: 32-row boxes per stage, row-group warps
    int tc, nc;  // columns per stage, consumer warps
    int stages, waves;
};

int stage_bytes_qr(int nb, int tile) { return (tile / kBoxRows) * (128 * 128 + nb * 128); }
int stage_bytes_cols(int nb, int tile) { return (64 / nb) * tile * 128 + tile * nb * 4; }

TmaShape shape_of(int nb, const UpdCfg &c) {
    TmaShape sh;
    sh.br = c.tile / kBoxRows;
    sh.nc = c.threads / 32;
    sh.rw = sh.nc / (nb / 16);
    sh.tc = c.tile;
    sh.stages = c.cpb;
    sh.waves = c.unroll;
    return sh;
}

// Persistent launch of a tensor-core projection: one block per SM, the split count of
// the reduction dimension (<= 8) chosen so the items fill the grid's block slots best.
template <int NB, int SIDE>
cudaError_t proj_tc_launch(const CUtensorMap &mX, const CUtensorMap &mV, int M, int N, const float *Tm, float *part,
                           float *fin, const UpdScratch &sc, cudaStream_t st) {
    static PerDeviceOnce attr;
    allow_max_smem(proj_tc_kernel<NB, SIDE>, attr);
    constexpr int LB = proj_land_bytes(NB), OB = proj_op_bytes(SIDE, NB);
    // ring depths (landing, operand) and blocks per SM; NLA_PROJ_RING="SL,SO,B" overrides
    static const int3 ring = [] {
        int3 r = make_int3(0, 0, 0);
        if (const char *v = getenv("NLA_PROJ_RING")) sscanf(v, "%d,%d,%d", &r.x, &r.y, &r.z);
        return r;
    }();
    const int per_sm = ring.z > 0 ? std::min(ring.z, 4) : 1;
    const size_t budget = kTmaSmemLimit / per_sm - 1024;
    const int SO = std::max(2, std::min(kMaxOp, ring.y > 0 ? ring.y : 2));
    const int SL = std::max(2, std::min(kLanding, ring.x > 0 ? ring.x : (int)((budget - (size_t)SO * OB) / LB)));
    const size_t smem = (size_t)SL * LB + (size_t)SO * OB + 1024;
    const int Lext = SIDE == 0 ? N : M, Kext = SIDE == 0 ? M : N;
    const int nstrip = (Lext + 127) / 128, ktiles = (Kext + 31) / 32;
    const int G = device_sm_count() * per_sm;
    int nsplit = 1;
    double best = -1.0;
    for (int s = 1; s <= kMaxSplitTma && s <= ktiles; ++s) {
        const long items = (long)nstrip * s;
        const double eff = (double)items / ((double)((items + G - 1) / G) * G);  // busy fraction of block slots
        if (eff > best + 1e-9) {
            best = eff;
            nsplit = s;
        }
    }
    const int Ks = ((Kext + nsplit - 1) / nsplit + 31) / 32 * 32;
    nsplit = (Kext + Ks - 1) / Ks;
    const int grid = std::min(nstrip * nsplit, G);
    return launch_pdl(proj_tc_kernel<NB, SIDE>, dim3(grid), dim3(32 * kTcWarps), smem, st, mX, mV, M, N, Tm, SL, SO,
                      nsplit, Ks, part, fin, sc.tickets, sc.info);
}

bool proj_tc_enabled() {
    static const bool on = [] {  // NLA_PROJ_TC=0: the SIMT projections instead of the tensor-core ones
        const char *v = getenv("NLA_PROJ_TC");
        return !v || atoi(v) != 0;
    }();
    return on;
}

template <int NB>
cudaError_t left_proj_nb(float *X, long ldx, int M, int N, const float *V, long ldv, const float *Tm,
                         const TmaShape &sh, const UpdScratch &sc, cudaStream_t st) {
    float *part = reinterpret_cast<float *>(sc.work);
    float *fin = part + (size_t)kMaxSplitTma * 64 * std::max(M, N);
    CUtensorMap mX, mV;
    if (!tma_encode_2d(&mX, X, 4, M, N, ldx * 4, kBoxRows, 128, true) ||
        !tma_encode_2d(&mV, V, 4, M, NB, ldv * 4, kBoxRows, NB, false))
        return cudaErrorInvalidValue;
    // pass 1 (+ step 2): W' = T^T V^T X -- on the tensor cores (3xTF32) unless disabled
    const bool use_tc = proj_tc_enabled();
    CUtensorMap mVs;
    if (use_tc && tma_encode_2d(&mVs, V, 4, M, NB, ldv * 4, kBoxRows, NB, true)) {
        cudaError_t e = proj_tc_launch<NB, 0>(mX, mVs, M, N, Tm, part, fin, sc, st);
        if (e != cudaSuccess) return e;
    } else {
        static PerDeviceOnce attr;
        allow_max_smem(qr_proj_kernel<NB>, attr);
        const int th = sh.br * kBoxRows;
        const int stage = stage_bytes_qr(NB, th);
        const int nstrip = (N + 127) / 128;
        int nsplit = splits_for(nstrip, (M + th - 1) / th, sh.waves);
        const int Ms = ((M + nsplit - 1) / nsplit + th - 1) / th * th;
        nsplit = (M + Ms - 1) / Ms;
        const size_t smem = (size_t)sh.stages * stage + 1024;
        cudaError_t e = launch_pdl(qr_proj_kernel<NB>, dim3(nstrip, nsplit), dim3(32 * (sh.nc + 1)), smem, st, mX, mV,
                                   M, N, Tm, sh.br, sh.rw, sh.stages, Ms, part, fin, sc.tickets, sc.info);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Persistent grid of the strip update: as many blocks as the SMs hold (occupancy at
// this shared-memory size), items = (strips of H rows) x (column chunks); the chunk
// count is the one (at most `waves` chunks per block slot) whose items fill the block
// slots best, ties to fewer chunks.
template <typename K>
void strip_grid(K kernel, int M, int N, int H, const TmaShape &sh, size_t smem, int &grid, int &Ns) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * (sh.nc + 1), smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int slots = per_sm * device_sm_count();
    const int nstrip = (M + H - 1) / H, ntile = (N + sh.tc - 1) / sh.tc;
    const int maxc = std::max(1, std::min(ntile, (sh.waves * slots + nstrip - 1) / nstrip));
    int ncs = 1;
    double best = -1.0;
    for (int c = 1; c <= maxc; ++c) {
        const long items = (long)nstrip * c;
        const double eff = (double)items / ((double)((items + slots - 1) / slots) * slots);
        if (eff > best + 1e-9) {
            best = eff;
            ncs = c;
        }
    }
    static const bool all_items = [] {  // NLA_STRIP_GRID=1: one block per item instead of persistent blocks
        const char *v = getenv("NLA_STRIP_GRID");
        return v && atoi(v) != 0;
    }();
    if (all_items) ncs = std::max(1, std::min((sh.waves * device_sm_count() + nstrip - 1) / nstrip, ntile));
    Ns = ((N + ncs - 1) / ncs + sh.tc - 1) / sh.tc * sh.tc;
    ncs = (N + Ns - 1) / Ns;
    grid = all_items ? nstrip * ncs : std::min(nstrip * ncs, slots);
}

// pass 2 on rows [off, off + len) of the M x N trailing block: X -= V W'
template <int NB>
cudaError_t left_apply_nb(float *X, long ldx, int M, int N, const float *V, long ldv, int off, int len,
                          const TmaShape &sh, const UpdScratch &sc, cudaStream_t st) {
    if (len <= 0) return cudaSuccess;
    float *part = reinterpret_cast<float *>(sc.work);
    const float *fin = part + (size_t)kMaxSplitTma * 64 * std::max(M, N);
    float *Xo = X + off;
    const float *Vo = V + off;
    CUtensorMap mX2, mQ;
    if (!tma_encode_2d(&mX2, Xo, 4, len, N, ldx * 4, kBoxRows, sh.tc, true) ||
        !tma_encode_2d(&mQ, fin, 4, NB, N, NB * 4, NB, sh.tc, false))
        return cudaErrorInvalidValue;
    static PerDeviceOnce attr;
    allow_max_smem(strip_update_kernel<NB, 0>, attr);
    const size_t smem = (size_t)sh.stages * stage_bytes_cols(NB, sh.tc) + 1024;
    int grid = 0, Ns = 0;
    strip_grid(strip_update_kernel<NB, 0>, len, N, 32 * (64 / NB), sh, smem, grid, Ns);
    return launch_pdl(strip_update_kernel<NB, 0>, dim3(grid), dim3(32 * (sh.nc + 1)), smem, st, mX2, mQ, len, N,
                      Vo, ldv, sh.tc, sh.nc, sh.stages, Ns, off, sc.info);
}

template <int NB>
cudaError_t right_proj_nb(float *X, long ldx, int M, int N, const float *Vt, long ldvt, const float *Tm,
                          const TmaShape &sh, const UpdScratch &sc, cudaStream_t st) {
    float *part = reinterpret_cast<float *>(sc.work);
    float *fin = part + (size_t)kMaxSplitTma * 64 * std::max(M, N);
    CUtensorMap mX, mQ;
    // pass 1 (+ step 2): Y' = X V T -- on the tensor cores (3xTF32) unless disabled
    if (proj_tc_enabled() && tma_encode_2d(&mX, X, 4, M, N, ldx * 4, kBoxRows, 32, true) &&
        tma_encode_2d(&mQ, Vt, 4, NB, N, ldvt * 4, NB, 32, false))
        return proj_tc_launch<NB, 1>(mX, mQ, M, N, Tm, part, fin, sc, st);
    if (!tma_encode_2d(&mX, X, 4, M, N, ldx * 4, kBoxRows, sh.tc, true) ||
        !tma_encode_2d(&mQ, Vt, 4, NB, N, ldvt * 4, NB, sh.tc, false))
        return cudaErrorInvalidValue;
    constexpr int H = 32 * (64 / NB);
    const int stage = stage_bytes_cols(NB, sh.tc);
    const int nstrip = (M + H - 1) / H;
    const size_t smem = (size_t)sh.stages * stage + 1024;
    static PerDeviceOnce attr;
    allow_max_smem(lq_proj_kernel<NB>, attr);
    int nsplit = splits_for(nstrip, (N + sh.tc - 1) / sh.tc, sh.waves);
    const int Ns = ((N + nsplit - 1) / nsplit + sh.tc - 1) / sh.tc * sh.tc;
    nsplit = (N + Ns - 1) / Ns;
    return launch_pdl(lq_proj_kernel<NB>, dim3(nstrip, nsplit), dim3(32 * (sh.nc + 1)), smem, st, mX, mQ, M, N, Tm,
                      sh.tc, sh.nc, sh.stages, Ns, part, fin, sc.tickets, sc.info);
}

// pass 2 on columns [off, off + len) of the M x N trailing block: X -= Y' V^T
template <int NB>
cudaError_t right_apply_nb(float *X, long ldx, int M, int N, const float *Vt, long ldvt, int off, int len,
                           const TmaShape &sh, const UpdScratch &sc, cudaStream_t st, const float *fin_in) {
    if (len <= 0) return cudaSuccess;
    float *part = reinterpret_cast<float *>(sc.work);
    const float *fin = fin_in ? fin_in : part + (size_t)kMaxSplitTma * 64 * std::max(M, N);
    float *Xo = X + (long)off * ldx;
    const float *Vo = Vt + (long)off * ldvt;
    CUtensorMap mX, mQ;
    if (!tma_encode_2d(&mX, Xo, 4, M, len, ldx * 4, kBoxRows, sh.tc, true) ||
        !tma_encode_2d(&mQ, Vo, 4, NB, len, ldvt * 4, NB, sh.tc, false))
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)sh.stages * stage_bytes_cols(NB, sh.tc) + 1024;
    static PerDeviceOnce attr;
    allow_max_smem(strip_update_kernel<NB, 1>, attr);
    int grid = 0, Ns = 0;
    strip_grid(strip_update_kernel<NB, 1>, M, len, 32 * (64 / NB), sh, smem, grid, Ns);
    return launch_pdl(strip_update_kernel<NB, 1>, dim3(grid), dim3(32 * (sh.nc + 1)), smem, st, mX, mQ, M, len,
                      fin, 0L, sh.tc, sh.nc, sh.stages, Ns, off, sc.info);
}

}  // namespace

size_t tma_cfg_smem(int nb, const UpdCfg &c) {
    return (size_t)c.cpb * std::max(stage_bytes_qr(nb, c.tile), stage_bytes_cols(nb, c.tile)) + 1024;
}

bool tma_cfg_valid(int nb, const UpdCfg &c) {
    if (nb != 16 && nb != 32 && nb != 64) return false;
    if (c.tile != 32 && c.tile != 64 && c.tile != 128) return false;
    if (c.threads != 64 && c.threads != 128 && c.threads != 256) return false;
    if ((c.threads / 32) % (nb / 16)) return false;  // qr_proj: whole reflector groups of 16
    if (c.cpb != 2 && c.cpb != 4 && c.cpb != 8) return false;
    if (c.unroll != 1 && c.unroll != 2 && c.unroll != 4) return false;
    return tma_cfg_smem(nb, c) <= kTmaSmemLimit;
}

bool trail_tma_eligible(const float *X, long ldx, const float *V, long ldv, int nb, const UpdScratch &sc) {
    if (nb != 16 && nb != 32 && nb != 64) return false;
    if (!sc.work || !sc.tickets) return false;
    if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(V) % 16) return false;
    return ldx % 4 == 0 && ldv % 4 == 0;
}

cudaError_t trail_tma_project(int side, float *X, long ldx, int M, int N, const float *V, long ldv, int nb,
                              const float *Tm, const UpdCfg &c, const UpdScratch &sc, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (!trail_tma_eligible(X, ldx, V, ldv, nb, sc) || !tma_cfg_valid(nb, c)) return cudaErrorInvalidConfiguration;
    const TmaShape sh = shape_of(nb, c);
    if (side == 0) {
        switch (nb) {
            case 16: return left_proj_nb<16>(X, ldx, M, N, V, ldv, Tm, sh, sc, st);
            case 32: return left_proj_nb<32>(X, ldx, M, N, V, ldv, Tm, sh, sc, st);
            default: return left_proj_nb<64>(X, ldx, M, N, V, ldv, Tm, sh, sc, st);
        }
    }
    switch (nb) {
        case 16: return right_proj_nb<16>(X, ldx, M, N, V, ldv, Tm, sh, sc, st);
        case 32: return right_proj_nb<32>(X, ldx, M, N, V, ldv, Tm, sh, sc, st);
        default: return right_proj_nb<64>(X, ldx, M, N, V, ldv, Tm, sh, sc, st);
    }
}

cudaError_t trail_tma_apply(int side, float *X, long ldx, int M, int N, const float *V, long ldv, int nb, int off,
                            int len, const UpdCfg &c, const UpdScratch &sc, cudaStream_t st, const float *fin_in) {
    if (M <= 0 || N <= 0 || len <= 0) return cudaSuccess;
    if (!trail_tma_eligible(X, ldx, V, ldv, nb, sc) || !tma_cfg_valid(nb, c) || off % 4) return cudaErrorInvalidConfiguration;
    const TmaShape sh = shape_of(nb, c);
    if (side == 0) {
        switch (nb) {
            case 16: return left_apply_nb<16>(X, ldx, M, N, V, ldv, off, len, sh, sc, st);
            case 32: return left_apply_nb<32>(X, ldx, M, N, V, ldv, off, len, sh, sc, st);
            default: return left_apply_nb<64>(X, ldx, M, N, V, ldv, off, len, sh, sc, st);
        }
    }
    switch (nb) {
        case 16: return right_apply_nb<16>(X, ldx, M, N, V, ldv, off, len, sh, sc, st, fin_in);
        case 32: return right_apply_nb<32>(X, ldx, M, N, V, ldv, off, len, sh, sc, st, fin_in);
        default: return right_apply_nb<64>(X, ldx, M, N, V, ldv, off, len, sh, sc, st, fin_in);
    }
}

cudaError_t trail_tma(int side, float *X, long ldx, int M, int N, const float *V, long ldv, int nb, const float *Tm,
                      const UpdCfg &c, const UpdScratch &sc, cudaStream_t st) {
    cudaError_t e = trail_tma_project(side, X, ldx, M, N, V, ldv, nb, Tm, c, sc, st);
    if (e != cudaSuccess) return e;
    return trail_tma_apply(side, X, ldx, M, N, V, ldv, nb, 0, side == 0 ? M : N, c, sc, st);
}

}  // namespace nla
