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
//   lq_proj_tm    Y = X V on the tensor cores (the default LQ projection): the
//                 hi/lo rows of X go from the landed boxes to tensor memory
//                 (tcgen05.st) and feed the MMAs as their A operand there.
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
            if (!tc::mbar_wait_lanes(&full[st], (uint32_t)((t / S) & 1), info, &sh_abort) || sh_abort) break;
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

// ------------------------------------------------------------------ qr_proj on the tensor cores
// W^T (128 strip columns x NB) = X_strip^T V accumulated in TMEM by tcgen05.mma
// (kind::tf32, M = 128, K = 8 per instruction) over 32-row stages of X.
// FP32 accuracy from TF32 operands by the three-term split x = hi + lo,
// hi = x with the low 13 mantissa bits cleared (what the tensor core reads of an
// FP32 word), lo = x - hi (exact): x . v ~ hi_x hi_v + hi_x lo_v + lo_x hi_v, the
// dropped lo_x lo_v term and the truncation of lo are below 2^-21 relative.  The
// first two products are one MMA against [V_hi; V_lo] (N = 2 NB, the hi copy of X
// read once), the third a second MMA (N = NB) into its own accumulator; the
// epilogue adds the three parts.
// Roles: warp 0 issues the TMA loads of X and V (128-byte-swizzled boxes, which
// are the canonical K-major operand layout); warps 2..5 write the lo copies and
// mask V's unit diagonal; warp 1 owns TMEM and one lane issues the MMAs, each
// stage's commit freeing it for the producer; warps 2..5 read the accumulator
// back (each warp its TMEM lane quadrant).
constexpr int kTcWarps = 6;

NLA_DEV float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <int NB>
__global__ void __launch_bounds__(32 * kTcWarps, 1)
qr_proj_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV, int M, int N,
                  const float *__restrict__ Tm, int S, int Ms, float *part, float *fin, unsigned int *tickets,
                  int *info) {
    pdl_wait();
    pdl_trigger();
    // TMEM: D1 = hi x [V_hi | V_lo] (2 NB columns), D2 = lo x V_hi (NB columns)
    constexpr uint32_t kCols = 3 * NB <= 32 ? 32 : 3 * NB <= 64 ? 64 : 3 * NB <= 128 ? 128 : 256;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], conv[kMaxStages], empty[kMaxStages], accdone;
    __shared__ uint32_t tmem_base;
    __shared__ int sh_last, sh_abort;
    unsigned char *base = align1k(smem_raw);
    const int xbytes = 32 * 128 * 4, vbytes = NB * 128;  // one 32-row box of X (128 columns) and of V
    const int stage = 2 * xbytes + 2 * vbytes;          // hi and lo copies
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c0 = blockIdx.x * 128, wc = min(128, N - c0);
    const int sp = blockIdx.y, nsplit = gridDim.y;
    const int rbeg = sp * Ms, rend = min(M, rbeg + Ms);
    const int nt = (rend - rbeg + kBoxRows - 1) / kBoxRows;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&conv[i], 4);
            tc::mbar_init(&empty[i], 1);
        }
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
    auto xhi = [&](int st) { return base + (size_t)st * stage; };
    auto xlo = [&](int st) { return base + (size_t)st * stage + xbytes; };
    auto vhi = [&](int st) { return base + (size_t)st * stage + 2 * xbytes; };
    auto vlo = [&](int st) { return base + (size_t)st * stage + 2 * xbytes + vbytes; };

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nt; ++t) {
                const int st = t % S;
                if (t >= S && !tc::mbar_wait(&empty[st], (uint32_t)(((t / S) - 1) & 1), info)) {
                    sh_abort = 1;
                    break;
                }
                const int r0 = rbeg + t * kBoxRows;
                tma::expect_tx(&full[st], (uint32_t)(xbytes + vbytes));
                tma::load_2d(xhi(st), &tmX, r0, c0, &full[st]);
                tma::load_2d(vhi(st), &tmV, r0, 0, &full[st]);
                issued = t + 1;
            }
            drain_loads(full, issued, S, info);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // V_lo lies right after V_hi (NB rows of 128 bytes each): [V_hi; V_lo] is one B
            // operand of 2 NB rows, so the hi copy of X is read once per K step
            const uint32_t id2 = tc::idesc(2, 128, 2 * NB), id1 = tc::idesc(2, 128, NB);
            for (int t = 0; t < nt; ++t) {
                const int st = t % S;
                if (*(volatile int *)&sh_abort || !tc::mbar_wait(&conv[st], (uint32_t)((t / S) & 1), info)) {
                    sh_abort = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t ah = tc::smem_u32(xhi(st)), al = tc::smem_u32(xlo(st));
                const uint32_t bh = tc::smem_u32(vhi(st));
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {  // 8 TF32 = 32 bytes of K per instruction
                    const uint32_t off = kk * 32, acc = (t > 0 || kk > 0) ? 1u : 0u;
                    tc::mma_tf32(tbase, tc::sdesc_sw128(ah + off), tc::sdesc_sw128(bh + off), id2, acc);
                    tc::mma_tf32(tbase + 2 * NB, tc::sdesc_sw128(al + off), tc::sdesc_sw128(bh + off), id1, acc);
                }
                tc::mma_commit(&empty[st]);  // the stage is free once these MMAs have read it
            }
            tc::mma_commit(&accdone);  // every issued MMA has completed
        }
        __syncwarp();
    } else {
        // ---- warps 2..5: lo copies (and V's unit diagonal), then the epilogue
        const int ct = tid - 64;  // 0..127
        for (int t = 0; t < nt; ++t) {
            const int st = t % S;
            if (!tc::mbar_wait_lanes(&full[st], (uint32_t)((t / S) & 1), info, &sh_abort) || sh_abort) {
                sh_abort = 1;
                break;
            }
            const int r0 = rbeg + t * kBoxRows;  // trailing-matrix row of the stage's first row
            float *vh = reinterpret_cast<float *>(vhi(st));
            if (r0 < NB) {
                // V(r, k) with r <= k: 1 on the diagonal, 0 above (entry (r, k) of the box:
                // row k, 16-byte chunk (r/4) ^ (k & 7), word r % 4)
                for (int e = ct; e < NB * kBoxRows; e += 128) {
                    const int k = e / kBoxRows, rr = e % kBoxRows, r = r0 + rr;
                    if (r <= k) vh[k * 32 + ((((rr >> 2) ^ (k & 7))) << 2) + (rr & 3)] = r == k ? 1.f : 0.f;
                }
                asm volatile("bar.sync 2, 128;" ::: "memory");
            }
            const float4 *xs = reinterpret_cast<const float4 *>(xhi(st));
            float4 *xl = reinterpret_cast<float4 *>(xlo(st));
#pragma unroll 4
            for (int e = ct; e < xbytes / 16; e += 128) {
                const float4 v = xs[e];
                xl[e] = make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
            }
            const float4 *vs = reinterpret_cast<const float4 *>(vh);
            float4 *vl = reinterpret_cast<float4 *>(vlo(st));
            for (int e = ct; e < vbytes / 16; e += 128) {
                const float4 v = vs[e];
                vl[e] = make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
            }
            tc::fence_async_smem();  // the lo copies -> visible to the tensor core
            __syncwarp();
            if (lane == 0) tma::arrive(&conv[st]);
        }
        // epilogue: W^T rows of this warp's TMEM lane quadrant
        const bool ok = tc::mbar_wait_warp(&accdone, 0, info);
        tc::fence_after_sync();
        const int q = warp & 3;  // TMEM lanes 32q .. 32q + 31
        const int col = 32 * q + lane;
        if (ok && !*(volatile int *)&sh_abort) {
#pragma unroll
            for (int c = 0; c < NB; c += 16) {
                float w[16], wl[16], w2[16];  // hi.hi, hi.lo, lo.hi
                const uint32_t lb = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)c;
                tc::tmem_ld16(lb, w);
                tc::tmem_ld16(lb + NB, wl);
                tc::tmem_ld16(lb + 2 * NB, w2);
                tc::tmem_wait_ld();
                if (col < wc) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) part[((size_t)sp * NB + c + k) * N + c0 + col] = w[k] + (wl[k] + w2[k]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tbase, kCols);
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
            for (int qq = 0; qq < kMaxSplitTma; ++qq)  // (all partial loads in flight at once)
                if (qq < nsplit) sum += __ldcg(part + ((size_t)qq * NB + k) * N + c0 + c);
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

// ------------------------------------------------------------------ lq_proj
// Block (strip, s): partial Y(strip rows, :) = X(strip rows, columns of split s) V
// over stages of tc columns; last block of the strip: Y' = Y T -> fin[k*M + i].
// At NB = 16 the kernel is capped at 128 registers so three blocks of 160 threads share
// an SM (12 consumer warps instead of 8 hide the shared-memory latency of the FMA
// stream; 46.8 -> 44.4 ms of LQ-side update per 8192 SVD, no spills); the wider forms
// keep their 168.
template <int NB>
__global__ void __launch_bounds__(kMaxThreads, 1) __maxnreg__(NB == 16 ? 128 : 168)
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
            if (!tc::mbar_wait_lanes(&full[st], (uint32_t)((t / S) & 1), info, &sh_abort) || sh_abort) break;
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

// ------------------------------------------------------------------ lq_proj_tm
// Block (strip, s): partial Y(128 strip rows, :) = X(strip rows, columns of split s) V on
// the tensor cores (kind::tf32, M = 128 rows, N = NB, K = 8 columns per instruction) over
// stages of 32 columns; last block of the strip: Y' = Y T -> fin[k*M + i].
// The reduction runs over X's columns, which are strided in a column-major matrix, and a
// kind::tf32 operand in shared memory must be K-major; so the A operand goes through
// tensor memory instead.  Each converter warp owns 32 rows (its TMEM lane quadrant):
// lane i reads X(i, c) for the stage's 32 columns from the landed box (one 128-byte line
// per column, no bank conflict), splits it into hi + lo (the same three-term split as
// qr_proj_tc) and stores both to TMEM (tcgen05.st, 32 columns each); the box is free
// as soon as it has been read.  V(c, k) of the stage's columns comes from global memory
// (L2), masked to the unit lower form and written K-major as its hi and lo copies (B).
// Rings: kLqStages TMEM/B operand slots (freed by the MMA commit) behind an X ring
// sized to the shared memory (freed by the converters).
constexpr int kLqCols = 32;    // columns per stage
constexpr int kLqStages = 3;   // operand slots: 64 TMEM columns each (A hi, A lo)
constexpr int kLqXBox = kBoxRows * kLqCols * 4;  // one 32 x 32 box, no swizzle: 4 KB
constexpr int lq_tm_opnd_bytes(int nb) { return 2 * nb * 128; }

template <int NB>
__global__ void __launch_bounds__(32 * kTcWarps, 1)
lq_proj_tm_kernel(const __grid_constant__ CUtensorMap tmX, int M, int N, const float *__restrict__ Vt, long ldvt,
                  const float *__restrict__ Tm, int SX, int Ns, float *part, float *fin, unsigned int *tickets,
                  int *info) {
    pdl_wait();
    pdl_trigger();
    constexpr int H = 128;                            // rows per block = the MMA's M
    constexpr int kX = 4 * kLqXBox;                   // the stage's 128 rows
    constexpr int kB = NB * 128;                      // V^T of the stage's 32 columns (hi or lo)
    // At NB = 16 the accumulator is split like qr_proj_tc's (D1 = A_hi [V_hi; V_lo], 2 NB
    // columns; D2 = A_lo V_hi, NB columns: two MMAs per K step); the wider forms keep one
    // accumulator and three MMAs (the split one would not leave room for three slots).
    constexpr bool kStack = NB == 16;
    constexpr uint32_t kD = kStack ? 64 : (NB < 32 ? 32 : NB);  // TMEM columns of the accumulator(s)
    constexpr uint32_t kCols = 256;
    static_assert(kD + 64 * kLqStages <= 256, "TMEM budget: two blocks per SM");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t xfull[kMaxStages], xfree[kMaxStages], conv[kLqStages], ofree[kLqStages], accdone;
    __shared__ uint32_t tmem_base;
    __shared__ int sh_last, sh_abort;
    unsigned char *base = align1k(smem_raw);
    unsigned char *bring = base + (size_t)SX * kX;    // operand B slots (1024-byte aligned)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.x * H, hr = min(H, M - i0);
    const int s = blockIdx.y, nsplit = gridDim.y;
    const int cbeg = s * Ns, cend = min(N, cbeg + Ns);
    const int nt = (cend - cbeg + kLqCols - 1) / kLqCols;
    if (tid == 0) {
        for (int i = 0; i < SX; ++i) {
            tc::mbar_init(&xfull[i], 1);
            tc::mbar_init(&xfree[i], 4);
        }
        for (int i = 0; i < kLqStages; ++i) {
            tc::mbar_init(&conv[i], 4);
            tc::mbar_init(&ofree[i], 1);
        }
        tc::mbar_init(&accdone, 1);
        sh_abort = 0;
        tma::fence_init();
        tma::prefetch_map(&tmX);
    }
    if (warp == 1) {
        tc::tmem_alloc(&tmem_base, kCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    auto acol = [&](int o) { return kD + 64u * (uint32_t)o; };  // A hi at acol, A lo at acol + 32
    auto bhi = [&](int o) { return bring + (size_t)o * 2 * kB; };
    auto blo = [&](int o) { return bring + (size_t)o * 2 * kB + kB; };

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nt; ++t) {
                const int xs = t % SX;
                if (t >= SX && !tc::mbar_wait(&xfree[xs], (uint32_t)(((t / SX) - 1) & 1), info)) {
                    sh_abort = 1;
                    break;
                }
                unsigned char *xb = base + (size_t)xs * kX;
                tma::expect_tx(&xfull[xs], (uint32_t)kX);
                const int cb = cbeg + t * kLqCols;
                for (int bx = 0; bx < 4; ++bx) tma::load_2d(xb + bx * kLqXBox, &tmX, i0 + bx * kBoxRows, cb, &xfull[xs]);
                issued = t + 1;
            }
            drain_loads(xfull, issued, SX, info);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = tc::idesc(2, 128, NB), id2 = tc::idesc(2, 128, 2 * NB);
            for (int t = 0; t < nt; ++t) {
                const int o = t % kLqStages;
                if (*(volatile int *)&sh_abort || !tc::mbar_wait(&conv[o], (uint32_t)((t / kLqStages) & 1), info)) {
                    sh_abort = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t ah = tbase + acol(o), al = ah + 32;
                const uint32_t bh = tc::smem_u32(bhi(o)), bl = tc::smem_u32(blo(o));
#pragma unroll
                for (int kk = 0; kk < kLqCols / 8; ++kk) {  // 8 columns per instruction
                    const uint32_t off = kk * 32, acc = (t > 0 || kk > 0) ? 1u : 0u;
                    if constexpr (kStack) {  // B lo lies right after B hi: [V_hi; V_lo] is one operand
                        tc::mma_tf32_tmem_a(tbase, ah + 8 * kk, tc::sdesc_sw128(bh + off), id2, acc);
                        tc::mma_tf32_tmem_a(tbase + 2 * NB, al + 8 * kk, tc::sdesc_sw128(bh + off), id, acc);
                    } else {
                        tc::mma_tf32_tmem_a(tbase, ah + 8 * kk, tc::sdesc_sw128(bh + off), id, acc);
                        tc::mma_tf32_tmem_a(tbase, ah + 8 * kk, tc::sdesc_sw128(bl + off), id, 1u);
                        tc::mma_tf32_tmem_a(tbase, al + 8 * kk, tc::sdesc_sw128(bh + off), id, 1u);
                    }
                }
                tc::mma_commit(&ofree[o]);  // the operand slot is free once these MMAs have read it
            }
            tc::mma_commit(&accdone);
        }
        __syncwarp();
    } else {
        // ---- warps 2..5: rows 32q .. 32q + 31 of the strip (TMEM lane quadrant q = box q)
        const int q = warp & 3, ct = tid - 64;
        constexpr int kVe = NB * kLqCols / 128;  // V entries per thread and stage
        const uint32_t lane_base = tbase + ((uint32_t)(32 * q) << 16);
        // V of stage t, loaded a stage ahead (its L2 latency hides behind the previous stage):
        // entry (k, j) = V(cb + j, k), the address clamped into the split, the value masked to
        // the unit lower form after the load (no branch per load)
        float vraw[kVe];
        auto load_v = [&](int t) {
            const int cb = cbeg + t * kLqCols;
#pragma unroll
            for (int u = 0; u < kVe; ++u) {
                const int e = ct + 128 * u, j = e / NB, k = e % NB;
                vraw[u] = __ldg(Vt + k + (size_t)min(cb + j, cend - 1) * ldvt);
            }
        };
        if (nt > 0) load_v(0);
        for (int t = 0; t < nt; ++t) {
            const int xs = t % SX, o = t % kLqStages;
            const int cb = cbeg + t * kLqCols;
            float v[kVe];
#pragma unroll
            for (int u = 0; u < kVe; ++u) {
                const int e = ct + 128 * u, j = e / NB, k = e % NB, c = cb + j;
                v[u] = c < cend ? unit_lower(c, k, vraw[u]) : 0.f;
            }
            if (t + 1 < nt) load_v(t + 1);
            if (!tc::mbar_wait_lanes(&xfull[xs], (uint32_t)((t / SX) & 1), info, &sh_abort) || sh_abort) {
                sh_abort = 1;
                break;
            }
            float x[kLqCols], h[kLqCols];
            const float *xb = reinterpret_cast<const float *>(base + (size_t)xs * kX + q * kLqXBox);
#pragma unroll
            for (int c = 0; c < kLqCols; ++c) x[c] = xb[c * kBoxRows + lane];  // X(32q + lane, cb + c)
            __syncwarp();
            if (lane == 0) tma::arrive(&xfree[xs]);  // the box is read
            if (t >= kLqStages &&
                (!tc::mbar_wait_lanes(&ofree[o], (uint32_t)(((t / kLqStages) - 1) & 1), info, &sh_abort) ||
                 sh_abort)) {
                sh_abort = 1;
                break;
            }
            tc::fence_after_sync();
#pragma unroll
            for (int c = 0; c < kLqCols; ++c) {
                h[c] = tf32_hi(x[c]);
                x[c] -= h[c];
            }
            tc::tmem_st32(lane_base + acol(o), h);
            tc::tmem_st32(lane_base + acol(o) + 32, x);
            float *vh = reinterpret_cast<float *>(bhi(o));
            float *vl = reinterpret_cast<float *>(blo(o));
#pragma unroll
            for (int u = 0; u < kVe; ++u) {  // row k, 16-byte chunk (j/4) ^ (k & 7), word j % 4
                const int e = ct + 128 * u, j = e / NB, k = e % NB;
                const int w = k * 32 + (((j >> 2) ^ (k & 7)) << 2) + (j & 3);
                vh[w] = v[u];
                vl[w] = v[u] - tf32_hi(v[u]);
            }
            tc::tmem_wait_st();
            tc::fence_async_smem();  // the B copies -> visible to the tensor core
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tma::arrive(&conv[o]);
        }
        // epilogue: rows 32q .. 32q + 31 of the block from the accumulator's lane quadrant
        const bool ok = tc::mbar_wait_warp(&accdone, 0, info);
        tc::fence_after_sync();
        const int i = 32 * q + lane;
        if (ok && !*(volatile int *)&sh_abort) {
#pragma unroll
            for (int c = 0; c < NB; c += 16) {
                float y[16], yl[16], y2[16];
                tc::tmem_ld16(lane_base + (uint32_t)c, y);
                if constexpr (kStack) {  // hi.hi + (hi.lo + lo.hi)
                    tc::tmem_ld16(lane_base + (uint32_t)(NB + c), yl);
                    tc::tmem_ld16(lane_base + (uint32_t)(2 * NB + c), y2);
                }
                tc::tmem_wait_ld();
                if constexpr (kStack) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) y[k] += yl[k] + y2[k];
                }
                if (i < hr) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) part[((size_t)s * NB + c + k) * M + i0 + i] = y[k];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tbase, kCols);
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
            for (int qq = 0; qq < kMaxSplitTma; ++qq)  // (all partial loads in flight at once)
                if (qq < nsplit) sum += __ldcg(part + ((size_t)qq * NB + k) * M + i0 + i);
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
// Block (strip, cs): X(strip rows, columns of split cs) -= P(strip rows, :) Q(cols, :)^T.
// SIDE 0 (QR): P = V (unit lower, column-major at Pv, ld ldp), Q = W'^T from
// fin[c*NB + k].  SIDE 1 (LQ): P = Y' at Pv[k*M + i] (ldp unused), Q = V
// stored by rows (unit lower in (c, k)).
template <int NB, int SIDE>
__global__ void __launch_bounds__(kMaxThreads, 1)
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
    const int i0 = blockIdx.x * H;
    const int cbeg = blockIdx.y * Ns, cend = min(N, cbeg + Ns);
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
            int issued = 0, stored = 0;
            bool ok = true;
            for (int t = 0; t < nt && ok; ++t) {
                const int st = t % S;
                unsigned char *sb = base + (size_t)st * stage;
                if (t >= S) {
                    // write back the tile that used this stage, then reuse it
                    if (!tc::mbar_wait(&done[st], (uint32_t)(((t / S) - 1) & 1), info)) {
                        sh_abort = 1;
                        ok = false;
                        break;
                    }
                    const int cbo = cbeg + (t - S) * tcols;
                    for (int bx = 0; bx < RL; ++bx) tma::store_2d(&tmX, i0 + bx * kBoxRows, cbo, sb + bx * xbytes);
                    tma::commit();
                    stored = t - S + 1;
                    tma::wait_read_all();
                }
                tma::expect_tx(&full[st], (uint32_t)stage);
                const int cb = cbeg + t * tcols;
                for (int bx = 0; bx < RL; ++bx) tma::load_2d(sb + bx * xbytes, &tmX, i0 + bx * kBoxRows, cb, &full[st]);
                tma::load_2d(sb + RL * xbytes, &tmQ, 0, cb, &full[st]);
                issued = t + 1;
            }
            for (int t = stored; ok && t < issued; ++t) {
                const int st = t % S;
                if (!tc::mbar_wait(&done[st], (uint32_t)((t / S) & 1), info)) {
                    sh_abort = 1;
                    ok = false;
                    break;
                }
                const int cbo = cbeg + t * tcols;
                for (int bx = 0; bx < RL; ++bx)
                    tma::store_2d(&tmX, i0 + bx * kBoxRows, cbo, base + (size_t)st * stage + bx * xbytes);
                tma::commit();
            }
            if (!ok) drain_loads(full, issued, S, info);
            tma::wait_all();
        }
    } else {
        const int cw = warp - 1;
        // P(lane's rows, :) in registers
        float p[RL][NB];
#pragma unroll
        for (int a = 0; a < RL; ++a) {
            const int i = i0 + RL * lane + a;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                float v = 0.f;
                if (i < M) {
                    // (SIDE 0: the entries on and above V's diagonal hold R, inside the panel's
                    // storage: loaded like the rest and masked, so the 64 loads carry no branch)
                    if constexpr (SIDE == 0)
                        v = unit_lower(moff + i, k, __ldg(Pv + i + (long)k * ldp));
                    else
                        v = __ldg(Pv + (size_t)k * M + i);
                }
                p[a][k] = v;
            }
        }
        for (int t = 0; t < nt; ++t) {
            const int st = t % S;
            if (!tc::mbar_wait_lanes(&full[st], (uint32_t)((t / S) & 1), info, &sh_abort) || sh_abort) break;
            unsigned char *sb = base + (size_t)st * stage;
            const float *qs = reinterpret_cast<const float *>(sb + RL * xbytes);
            const int cb = cbeg + t * tcols;
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

// NLA_PROJ_TC: which projections run on the tensor cores (bit 0: QR side, bit 1: LQ
// side; default both; 0: both on the SIMT kernels).
bool proj_tc(int side) {
    static const int mask = [] {
        const char *v = getenv("NLA_PROJ_TC");
        return v ? (atoi(v) & 3) : 3;
    }();
    return (mask >> side) & 1;
}
// Pipeline depth of the tensor-core projection: 3 stages measured best at 8192 (deeper
// rings cost blocks per SM); NLA_TC_STAGES overrides.
int tc_stages(int stage_bytes) {
    static const int sforce = [] {
        const char *v = getenv("NLA_TC_STAGES");
        return v ? atoi(v) : 0;
    }();
    return std::max(2, std::min({sforce > 0 ? sforce : 3, kMaxStages, (200 * 1024) / stage_bytes}));
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
    CUtensorMap mVs;
    if (proj_tc(0) && tma_encode_2d(&mVs, V, 4, M, NB, ldv * 4, kBoxRows, NB, true)) {
        static PerDeviceOnce attr;
        allow_max_smem(qr_proj_tc_kernel<NB>, attr);
        const int stage = 2 * (32 * 128 * 4) + 2 * NB * 128;
        const int S = tc_stages(stage);
        const int nstrip = (N + 127) / 128;
        int nsplit = splits_for(nstrip, (M + kBoxRows - 1) / kBoxRows, sh.waves);
        const int Ms = ((M + nsplit - 1) / nsplit + kBoxRows - 1) / kBoxRows * kBoxRows;
        nsplit = (M + Ms - 1) / Ms;
        const size_t smem = (size_t)S * stage + 1024;
        cudaError_t e = launch_pdl(qr_proj_tc_kernel<NB>, dim3(nstrip, nsplit), dim3(32 * kTcWarps), smem, st, mX, mVs,
                                   M, N, Tm, S, Ms, part, fin, sc.tickets, sc.info);
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
    constexpr int H = 32 * (64 / NB);
    const int stage = stage_bytes_cols(NB, sh.tc);
    const int nstrip = (len + H - 1) / H;
    int ncs = std::max(1, std::min((sh.waves * device_sm_count() + nstrip - 1) / nstrip, (N + sh.tc - 1) / sh.tc));
    const int Ns = ((N + ncs - 1) / ncs + sh.tc - 1) / sh.tc * sh.tc;
    ncs = (N + Ns - 1) / Ns;
    const size_t smem = (size_t)sh.stages * stage + 1024;
    return launch_pdl(strip_update_kernel<NB, 0>, dim3(nstrip, ncs), dim3(32 * (sh.nc + 1)), smem, st, mX2, mQ, len, N,
                      Vo, ldv, sh.tc, sh.nc, sh.stages, Ns, off, sc.info);
}

template <int NB>
cudaError_t right_proj_nb(float *X, long ldx, int M, int N, const float *Vt, long ldvt, const float *Tm,
                          const TmaShape &sh, const UpdScratch &sc, cudaStream_t st) {
    float *part = reinterpret_cast<float *>(sc.work);
    float *fin = part + (size_t)kMaxSplitTma * 64 * std::max(M, N);
    CUtensorMap mX, mQ;
    if (!tma_encode_2d(&mX, X, 4, M, N, ldx * 4, kBoxRows, sh.tc, true) ||
        !tma_encode_2d(&mQ, Vt, 4, NB, N, ldvt * 4, NB, sh.tc, false))
        return cudaErrorInvalidValue;
    // pass 1 (+ step 2): Y' = X V T -- on the tensor cores (3xTF32, A through TMEM) unless disabled
    CUtensorMap mXt;
    if (proj_tc(1) && tma_encode_2d(&mXt, X, 4, M, N, ldx * 4, kBoxRows, kLqCols, false)) {
        static PerDeviceOnce attr_tm;
        allow_max_smem(lq_proj_tm_kernel<NB>, attr_tm);
        // X ring: what two blocks per SM leave beside the operand slots
        const int sx = std::max(2, std::min(kMaxStages, (int)((108 * 1024 - kLqStages * lq_tm_opnd_bytes(NB)) /
                                                              (4 * kLqXBox))));
        const int nstrip = (M + 127) / 128;
        int nsplit = splits_for(nstrip, (N + kLqCols - 1) / kLqCols, sh.waves);
        const int Ns = ((N + nsplit - 1) / nsplit + kLqCols - 1) / kLqCols * kLqCols;
        nsplit = (N + Ns - 1) / Ns;
        const size_t smem = (size_t)sx * 4 * kLqXBox + (size_t)kLqStages * lq_tm_opnd_bytes(NB) + 1024;
        return launch_pdl(lq_proj_tm_kernel<NB>, dim3(nstrip, nsplit), dim3(32 * kTcWarps), smem, st, mXt, M, N, Vt,
                          ldvt, Tm, sx, Ns, part, fin, sc.tickets, sc.info);
    }
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
    constexpr int H = 32 * (64 / NB);
    const int stage = stage_bytes_cols(NB, sh.tc);
    const int nstrip = (M + H - 1) / H;
    const size_t smem = (size_t)sh.stages * stage + 1024;
    static PerDeviceOnce attr;
    allow_max_smem(strip_update_kernel<NB, 1>, attr);
    int ncs = std::max(1, std::min((sh.waves * device_sm_count() + nstrip - 1) / nstrip, (len + sh.tc - 1) / sh.tc));
    const int Ns = ((len + ncs - 1) / ncs + sh.tc - 1) / sh.tc * sh.tc;
    ncs = (len + Ns - 1) / Ns;
    return launch_pdl(strip_update_kernel<NB, 1>, dim3(nstrip, ncs), dim3(32 * (sh.nc + 1)), smem, st, mX, mQ, M, len,
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
