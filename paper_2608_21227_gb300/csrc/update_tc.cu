// update_tc.cu -- mixed-precision trailing update on the 5th-generation tensor
// cores: FP64 matrix, TF32 or BF16 operands (or their compensated three-product
// forms TF32X3 / BF16X3), FP32 accumulation in TMEM, exact power-of-two scaling of
// the converted operands (the trailing update of Algorithm 2 with the
// mixed-precision form of the contraction).
//
// Two launches per side (as in the SIMT path): step 1 on a grid of
// (128-wide strips) x (splits of the reduction dimension), the last block of a
// strip applying T; step 3 on a 2-D grid of 128 x 128 output tiles.
// QR side (strips of 128 columns of X):
//   1. W^T (128 x nbp) = X_strip^T V, accumulated over 32-row tiles.  Each tile
//      of X is scaled per column by 2^-e (e = exponent of the column's largest
//      magnitude in that tile), rounded to TF32/BF16 and multiplied on the
//      tensor cores into one of two TMEM accumulators; the previous tile's
//      accumulator is read back and added, unscaled, into FP32 registers while
//      the next multiply runs.
//   2. W' = T^T W per column in FP32; W' is scaled per column and rounded.
//   3. For each 128-row tile: D = V_tile W' on the tensor cores, then the
//      epilogue reads D from TMEM row by row and subtracts it, rescaled, from
//      X in FP64 (coalesced: one thread per row).
// LQ side (one block per 128-row strip): the same with rows and columns
// exchanged (Y = X_strip V, Y' = Y T, X_strip -= Y' V^T), scaling per row.
//
// Panel factorisation, T and the matrix stay FP64; only the two products are
// on the tensor cores.  Every wait is bounded; TMEM is freed on every path.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "../../include/nla.h"
#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace nla {

bool trail_tc_available() { return true; }

size_t trail_tc_scratch_bytes(int M, int N, int nb) {
    (void)M;
    (void)N;
    (void)nb;
    return 256;
}

namespace {

constexpr int kTcThreads = 256;   // 8 warps
constexpr int kStrip = 128;       // strip width = UMMA M
constexpr int kKt = 32;           // rows (QR) / columns (LQ) of X per step-1 tile
constexpr int kTmemCols = 256;    // self-test accumulator columns

// Operand types.  The compensated forms (TF32X3, BF16X3) split each scaled FP32
// operand v into hi = round(v) and lo = round(v - hi) in the operand type and form
// every product from three MMAs, hi*hi + hi*lo + lo*hi (the lo*lo term and lo's own
// rounding are below u^2 relative; Ootomo & Yokota 2022), so each product keeps about
// twice the operand type's significand bits.
template <int PREC>
struct Prec;
template <>
struct Prec<NLA_UPD_TF32> {
    static constexpr int es = 4;
    static constexpr uint32_t fmt = 2;
    static constexpr bool split = false;
    NLA_DEV static float round(float v) { return __uint_as_float(tc::to_tf32(v)); }
    NLA_DEV static void put(unsigned char *base, uint32_t off, float v) {
        *reinterpret_cast<uint32_t *>(base + off) = tc::to_tf32(v);
    }
    NLA_DEV static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) { tc::mma_tf32(d, a, b, id, acc); }
};
template <>
struct Prec<NLA_UPD_BF16> {
    static constexpr int es = 2;
    static constexpr uint32_t fmt = 1;
    static constexpr bool split = false;
    NLA_DEV static float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    NLA_DEV static void put(unsigned char *base, uint32_t off, float v) {
        *reinterpret_cast<uint16_t *>(base + off) = tc::to_bf16(v);
    }
    NLA_DEV static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) { tc::mma_bf16(d, a, b, id, acc); }
};
template <>
struct Prec<NLA_UPD_TF32X3> : Prec<NLA_UPD_TF32> {
    static constexpr bool split = true;
};
template <>
struct Prec<NLA_UPD_BF16X3> : Prec<NLA_UPD_BF16> {
    static constexpr bool split = true;
};

// Store operand v at byte offset `off` of the hi tile (and, for the compensated
// forms, its remainder at the same offset of the lo tile).
template <int PREC>
NLA_DEV void put_op(unsigned char *hi, unsigned char *lo, uint32_t off, float v) {
    using P = Prec<PREC>;
    P::put(hi, off, v);
    if constexpr (P::split) P::put(lo, off, v - P::round(v));
}

// power-of-two scale exponent: x * 2^-e lies in [0.5, 1) for the largest |x|
NLA_DEV int scale_exp(double mx) {
    if (!(mx > 0.0) || !isfinite(mx)) return 0;
    int e;
    frexp(mx, &e);
    return e;
}

// GB300's FP64 pipe issues a small fraction of the FP32/integer rate, so the
// per-element scaling and conversions below work on the IEEE bit patterns with
// integer instructions.  An FP64 x = (-1)^s 1.m 2^(E-1023) (biased exponent E of
// 11 bits, 52-bit m) is normal or zero throughout (subnormal inputs read as 0).
// Biased exponent of |x| (0 for zero); the scale exponent of a set of values is
// max(E) - 1022 (the frexp exponent of the largest).
NLA_DEV int f64_biased_exp(double x) { return (int)(((uint32_t)__double2hiint(x) >> 20) & 0x7FFu); }
// Scale exponent of a tile line for the step-1 accumulation: kNoExp marks a line whose
// entries are all zero (it adds nothing to the product).
constexpr int kNoExp = -100000;
NLA_DEV int tile_exp_from_biased(int emax) { return emax > 0 ? emax - 1022 : kNoExp; }
// 2^k for k <= 0 (0 below FP32's range); the power-of-two factors of the running sums.
NLA_DEV float exp2_nonpos(int k) { return k < -149 ? 0.f : ldexpf(1.f, k); }
// x * 2^-e as FP32 (exact scaling; the mantissa is truncated to FP32's 23 bits, far
// below the TF32/BF16 rounding that follows); results below FP32's normal range are 0.
NLA_DEV float f64_scaled_to_f32(double x, int e) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int E = (int)((hi >> 20) & 0x7FFu);
    const int fe = E - 1023 + 127 - e;
    const uint32_t sign = hi & 0x80000000u;
    if (E == 0 || fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);  // beyond FP32 (or not finite)
    const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    return __uint_as_float(sign | ((uint32_t)fe << 23) | mant);
}
// v * 2^e as FP64 (exact while the result is a normal FP64 number); FP32 zeros and
// subnormals give 0, results below FP64's normal range give a signed 0, results above
// it (or an infinite / NaN v) a signed infinity.
NLA_DEV double f32_scaled_to_f64(float v, int e) {
    const uint32_t b = __float_as_uint(v);
    const int E8 = (int)((b >> 23) & 0xFFu);
    const uint32_t sign = b & 0x80000000u;
    if (E8 == 0) return 0.0;
    const int E11 = E8 - 127 + 1023 + e;
    if (E11 <= 0) return __hiloint2double((int)sign, 0);
    if (E8 == 255 || E11 >= 2047) return __hiloint2double((int)(sign | 0x7FF00000u), 0);
    const uint32_t hi = sign | ((uint32_t)E11 << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

struct TcShared {
    uint64_t mbar[3];
    uint32_t tmem_base;
    int fail;
    int last_bar, last_parity;  // most recent commit (drained before TMEM is freed after a failure)
};

// Before freeing TMEM after a failed wait: one more bounded wait for the last
// committed group of MMAs (called by one thread).
NLA_DEV void drain_after_failure(TcShared *sh) {
    if (sh->fail && sh->last_bar >= 0) tc::mbar_wait(&sh->mbar[sh->last_bar], sh->last_parity, nullptr);
}

// Issue the MMAs of one product over kbytes of K, 32 K-bytes each (one thread).
template <int PREC>
NLA_DEV void issue1(uint32_t d, const unsigned char *A, int arowbytes, const unsigned char *B, int browbytes,
                    int kbytes, uint32_t id, bool accumulate_first) {
    const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
    for (int kk = 0; kk < kbytes / 32; ++kk) {
        uint64_t ad = tc::sdesc(a0 + kk * 256, 128, 8 * arowbytes);
        uint64_t bd = tc::sdesc(b0 + kk * 256, 128, 8 * browbytes);
        Prec<PREC>::mma(d, ad, bd, id, (kk > 0 || accumulate_first) ? 1u : 0u);
    }
}
// D (+)= A B^T; the compensated forms add the hi*lo and lo*hi products (Al, Bl: lo tiles).
template <int PREC>
NLA_DEV void issue(uint32_t d, const unsigned char *A, const unsigned char *Al, int arowbytes, const unsigned char *B,
                   const unsigned char *Bl, int browbytes, int kbytes, uint32_t id, bool accumulate_first) {
    issue1<PREC>(d, A, arowbytes, B, browbytes, kbytes, id, accumulate_first);
    if constexpr (Prec<PREC>::split) {
        issue1<PREC>(d, A, arowbytes, Bl, browbytes, kbytes, id, true);
        issue1<PREC>(d, Al, arowbytes, B, browbytes, kbytes, id, true);
    }
}

// ---------------------------------------------------------------- self-test
// D (128 x N, row-major FP32) = A (128 x K) * B (K x N), operands rounded to PREC.
template <int PREC>
__global__ void __launch_bounds__(128) tc_selftest_kernel(const float *A, const float *B, float *D, int K, int N,
                                                          int *info) {
    extern __shared__ __align__(1024) unsigned char sm[];
    using P = Prec<PREC>;
    const int rowbytes = K * P::es;
    unsigned char *As = sm;                          // 128 rows x K
    unsigned char *Bs = sm + 128 * rowbytes;         // N rows x K (B^T)
    TcShared *sh = reinterpret_cast<TcShared *>(Bs + (size_t)N * rowbytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(&sh->tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&sh->mbar[0], 1);
        sh->fail = 0;
        sh->last_bar = -1;
    }
    for (int idx = tid; idx < 128 * K; idx += blockDim.x) {
        int r = idx / K, k = idx % K;
        P::put(As, tc::kmajor_off(r, k, P::es, rowbytes), A[r * K + k]);
    }
    for (int idx = tid; idx < N * K; idx += blockDim.x) {
        int n = idx / K, k = idx % K;
        P::put(Bs, tc::kmajor_off(n, k, P::es, rowbytes), B[k * N + n]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = sh->tmem_base;
    if (tid == 0) {
        issue1<PREC>(tbase, As, rowbytes, Bs, rowbytes, rowbytes, tc::idesc(P::fmt, 128, N), false);
        tc::mma_commit(&sh->mbar[0]);
        sh->last_bar = 0;
        sh->last_parity = 0;
    }
    if (!tc::mbar_wait_warp(&sh->mbar[0], 0, info) && lane == 0) sh->fail = 1;
    tc::fence_after_sync();
    __syncthreads();
    if (!sh->fail) {
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tc::tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + c, v);
            tc::tmem_wait_ld();
            for (int i = 0; i < 16; ++i) D[(32 * warp + lane) * N + c + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) drain_after_failure(sh);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

// ---------------------------------------------------------------- step 1 (both sides)
// Block (strip, split) accumulates the partial W^T (QR side: strip columns x
// reflectors, reduction over rows [sbeg, send)) or Y (LQ side: strip rows x
// reflectors, reduction over columns) from 32-wide tiles scaled per strip
// line by 2^-e, rounded and multiplied on the tensor cores; the previous
// tile's TMEM accumulator is read back (unscaled) into FP32 registers while
// the next multiply runs.  The last block of the strip (atomic ticket) sums
// the partials and applies T (QR: W' = T^T W; LQ: Y' = Y T), storing FP32.
template <int PREC, int SIDE>
__global__ void __launch_bounds__(kTcThreads)
tc_w_kernel(const double *__restrict__ X, long ldx, int M, int N, const double *__restrict__ V, long ldv, int nb,
            int nbp, const double *__restrict__ Tm, int Ls, float *part, int *pexp, float *fin, int *finexp,
            unsigned int *tickets, int *info) {
    using P = Prec<PREC>;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ int sh_last;
    const int es = P::es, rb1 = kKt * es;
    constexpr int nsp = P::split ? 2 : 1;                    // hi (and lo) copies of each tile
    unsigned char *A1 = sm;                                  // 2 x [128 x kKt]  X tile (strip line x K)
    unsigned char *B1 = A1 + 2 * kStrip * rb1;               // 2 x [64 x kKt]   V tile (reflector x K)
    unsigned char *A1l = B1 + 2 * 64 * rb1;                  // lo copies (compensated forms)
    unsigned char *B1l = A1l + (nsp - 1) * 2 * kStrip * rb1;
    int *ex1 = reinterpret_cast<int *>(B1l + (nsp - 1) * 2 * 64 * rb1);  // 2 x 128
    int *lmax = ex1 + 2 * kStrip;                            // 2 x 128 biased exponents
    TcShared *sh = reinterpret_cast<TcShared *>(lmax + 2 * kStrip);
    float *Wsh = reinterpret_cast<float *>(sm);              // reused after the MMAs: nbp x 128
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hh = warp >> 2;
    // strip lines: QR -> columns of X, LQ -> rows of X; reduction dimension: the other one
    const int L0 = blockIdx.x * kStrip;
    const int Lext = SIDE == 0 ? N : M, Kext = SIDE == 0 ? M : N;
    const int lw = min(kStrip, Lext - L0);
    const int s = blockIdx.y, S = gridDim.y;
    const int kbeg = s * Ls, kend = min(Kext, kbeg + Ls);
    if (warp == 0) {
        tc::tmem_alloc(&sh->tmem_base, 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&sh->mbar[0], 1);
        tc::mbar_init(&sh->mbar[1], 1);
        sh->fail = 0;
        sh->last_bar = -1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = sh->tmem_base;
    const uint32_t id1 = tc::idesc(P::fmt, 128, nbp);
    const int half = nbp / 2;
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
    int erun = kNoExp;  // acc holds the line's partial W scaled by 2^-erun
    const int m = tid & (kStrip - 1), h = tid >> 7;  // loader: strip line m, K entries h*16 .. h*16+15
    const int ntiles = (kend - kbeg + kKt - 1) / kKt;
    for (int t = 0; t <= ntiles; ++t) {
        const int buf = t & 1;
        if (t < ntiles) {
            const int k0 = kbeg + t * kKt;
            double xv[16];
            if (SIDE == 0) {
                // lanes over the tile's 32 rows, warp w over strip columns 16w .. 16w+15:
                // coalesced column segments; the column's scale from a warp-wide max
                const int kk = k0 + lane;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int mc = warp * 16 + c;
                    xv[c] = (mc < lw && kk < kend) ? X[kk + (long)(L0 + mc) * ldx] : 0.0;
                }
            } else {
                int emx = 0;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int kk = k0 + h * 16 + i;
                    const double v = (m < lw && kk < kend) ? X[(L0 + m) + (long)kk * ldx] : 0.0;
                    xv[i] = v;
                    emx = max(emx, f64_biased_exp(v));
                }
                lmax[h * kStrip + m] = emx;
            }
            for (int idx = tid; idx < nbp * kKt; idx += blockDim.x) {
                int n, k;
                if (SIDE == 0) {
                    k = idx % kKt, n = idx / kKt;
                } else {
                    n = idx % nbp, k = idx / nbp;
                }
                const int g = k0 + k;
                double v = 0.0;
                if (n < nb && g < kend) {
                    if (SIDE == 0)
                        v = g > n ? V[g + (long)n * ldv] : (g == n ? 1.0 : 0.0);
                    else
                        v = g > n ? V[n + (long)g * ldv] : (g == n ? 1.0 : 0.0);
                }
                put_op<PREC>(B1 + buf * 64 * rb1, B1l + buf * 64 * rb1, tc::kmajor_off(n, k, es, rb1),
                             f64_scaled_to_f32(v, 0));
            }
            if (SIDE == 0) {
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int mc = warp * 16 + c;
                    const int e = tile_exp_from_biased(__reduce_max_sync(0xffffffffu, f64_biased_exp(xv[c])));
                    if (lane == 0) ex1[buf * kStrip + mc] = e;
                    put_op<PREC>(A1 + buf * kStrip * rb1, A1l + buf * kStrip * rb1, tc::kmajor_off(mc, lane, es, rb1),
                                 f64_scaled_to_f32(xv[c], e));
                }
            } else {
                __syncthreads();
                const int e = tile_exp_from_biased(max(lmax[m], lmax[kStrip + m]));
                if (h == 0) ex1[buf * kStrip + m] = e;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    put_op<PREC>(A1 + buf * kStrip * rb1, A1l + buf * kStrip * rb1,
                                 tc::kmajor_off(m, h * 16 + i, es, rb1), f64_scaled_to_f32(xv[i], e));
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                issue<PREC>(tbase + buf * 64, A1 + buf * kStrip * rb1, A1l + buf * kStrip * rb1, rb1,
                            B1 + buf * 64 * rb1, B1l + buf * 64 * rb1, rb1, rb1, id1, false);
                tc::mma_commit(&sh->mbar[buf]);
                sh->last_bar = buf;
                sh->last_parity = (t >> 1) & 1;
            }
        }
        if (t > 0) {
            const int pb = (t - 1) & 1;
            const bool ok = tc::mbar_wait_warp(&sh->mbar[pb], ((t - 1) >> 1) & 1, info);
            if (!ok && lane == 0) sh->fail = 1;
            tc::fence_after_sync();
            // the tile's product is scaled by 2^-et per line; the running sum is kept
            // scaled by 2^-erun (erun = the largest et so far), so no factor leaves
            // FP32's range whatever the exponents of X
            // (ok is warp-uniform: the TMEM loads below are warp-collective, so every lane
            // executes them; a line whose tile is all zero adds its product with factor 0)
            const int et = ex1[pb * kStrip + 32 * q + lane];
            if (ok) {
                float sc = 0.f;
                if (et != kNoExp) {
                    if (et > erun) {
                        const float r = exp2_nonpos(erun - et);
#pragma unroll
                        for (int i = 0; i < 32; ++i) acc[i] *= r;
                        erun = et;
                    }
                    sc = exp2_nonpos(et - erun);
                }
                for (int c = 0; c < half; c += 16) {
                    float v[16];
                    tc::tmem_ld16(tbase + pb * 64 + hh * half + c + ((uint32_t)(32 * q) << 16), v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[c + i] += v[i] * sc;
                }
            }
            tc::fence_before_sync();
        }
        __syncthreads();
        if (sh->fail) break;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) drain_after_failure(sh);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 128);
    if (sh->fail) return;
    // ---- partial of this split; the last block of the strip finishes
    const int line = 32 * q + lane;
    for (int i = 0; i < half; ++i)
        if (line < lw) part[((size_t)s * nbp + hh * half + i) * Lext + L0 + line] = acc[i];
    if (hh == 0 && line < lw) pexp[(size_t)s * Lext + L0 + line] = erun;
    __threadfence();
    __syncthreads();
    if (tid == 0) sh_last = atomicAdd(&tickets[blockIdx.x], 1u) == (unsigned)(S - 1);
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // the line's common exponent: the largest of its splits' (kNoExp: all zero)
    int *lexp = reinterpret_cast<int *>(Wsh + (size_t)nbp * kStrip);
    if (tid < kStrip) {
        int em = kNoExp;
#pragma unroll
        for (int qq = 0; qq < 8; ++qq)
            if (qq < S && tid < lw) em = max(em, __ldcg(pexp + (size_t)qq * Lext + L0 + tid));
        lexp[tid] = em;
        if (tid < lw) finexp[L0 + tid] = em == kNoExp ? 0 : em;
    }
    __syncthreads();
    for (int idx = tid; idx < nbp * kStrip; idx += blockDim.x) {
        const int l = idx % kStrip, k = idx / kStrip;
        float sum = 0.f;
        if (l < lw && lexp[l] != kNoExp)
#pragma unroll
            for (int qq = 0; qq < 8; ++qq)  // (S <= 8 splits; all partial loads in flight at once)
                if (qq < S) {
                    const int es_ = __ldcg(pexp + (size_t)qq * Lext + L0 + l);
                    if (es_ != kNoExp)
                        sum += __ldcg(part + ((size_t)qq * nbp + k) * Lext + L0 + l) * exp2_nonpos(es_ - lexp[l]);
                }
        Wsh[k * kStrip + l] = sum;
    }
    __syncthreads();
    for (int i = 0; i < half; ++i) {
        const int kk = hh * half + i;
        float v = 0.f;
        // QR: W'(kk) = sum_{k <= kk} T(k, kk) W(k);  LQ: Y'(kk) = sum_{k <= kk} Y(k) T(k, kk) -- same form
        if (kk < nb)
            for (int k = 0; k <= kk; ++k) v += (float)Tm[k + (long)kk * nb] * Wsh[k * kStrip + line];
        if (line < lw) fin[(size_t)kk * Lext + L0 + line] = v;
    }
    if (tid == 0) tickets[blockIdx.x] = 0u;
}

// ---------------------------------------------------------------- step 3 (both sides)
// Block (strip, tile) forms one 128 x 128 product on the tensor cores and
// subtracts it from X in FP64.  QR: D = V(rows) W'(strip columns); LQ:
// D = Y'(strip rows) V(columns)^T.  W' / Y' are scaled per strip line by a
// power of two before rounding; the scale is undone in the epilogue.
template <int PREC, int SIDE>
__global__ void __launch_bounds__(kTcThreads)
tc_x_kernel(double *__restrict__ X, long ldx, int M, int N, const double *__restrict__ V, long ldv, int nb, int nbp,
            const float *__restrict__ fin, const int *__restrict__ finexp, int *info) {
    using P = Prec<PREC>;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int es = P::es, rb3 = nbp * es;
    constexpr int nsp = P::split ? 2 : 1;
    unsigned char *Aop = sm;                         // [128 x nbp]
    unsigned char *Bop = Aop + kStrip * rb3;         // [128 x nbp]
    unsigned char *Aopl = Bop + kStrip * rb3;        // lo copies (compensated forms)
    unsigned char *Bopl = Aopl + (nsp - 1) * kStrip * rb3;
    int *exs = reinterpret_cast<int *>(Bopl + (nsp - 1) * kStrip * rb3);  // 128 strip-line exponents
    float *lmax = reinterpret_cast<float *>(exs + kStrip);    // 2 x 128
    TcShared *sh = reinterpret_cast<TcShared *>(lmax + 2 * kStrip);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hh = warp >> 2;
    const int Lext = SIDE == 0 ? N : M;
    const int L0 = blockIdx.x * kStrip, lw = min(kStrip, Lext - L0);  // strip lines
    const int T0 = blockIdx.y * kStrip;                               // tile along the other dimension
    const int Text = SIDE == 0 ? M : N, tw = min(kStrip, Text - T0);
    if (warp == 0) {
        tc::tmem_alloc(&sh->tmem_base, 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&sh->mbar[0], 1);
        sh->fail = 0;
        sh->last_bar = -1;
    }
    // W' / Y' strip block: line l, reflector k; scale per line
    {
        const int l = tid & (kStrip - 1), hf = tid >> 7;
        float mx = 0.f;
        for (int k = hf; k < nbp; k += 2) mx = fmaxf(mx, fabsf(l < lw && k < nb ? fin[(size_t)k * Lext + L0 + l] : 0.f));
        lmax[hf * kStrip + l] = mx;
        __syncthreads();
        // fin holds W' / Y' scaled by 2^-finexp per line (step 1); rescaled here so the
        // line's largest entry lies in [0.5, 1) before rounding, both undone in the epilogue
        const int e = scale_exp((double)fmaxf(lmax[l], lmax[kStrip + l]));
        if (hf == 0) exs[l] = e + (l < lw ? finexp[L0 + l] : 0);
        // QR: B operand rows = strip columns (N dim), K = reflectors; LQ: A operand rows = strip rows
        unsigned char *dst = SIDE == 0 ? Bop : Aop;
        unsigned char *dstl = SIDE == 0 ? Bopl : Aopl;
        for (int k = hf; k < nbp; k += 2) {
            const float v = (l < lw && k < nb) ? fin[(size_t)k * Lext + L0 + l] : 0.f;
            put_op<PREC>(dst, dstl, tc::kmajor_off(l, k, es, rb3), ldexpf(v, -e));
        }
    }
    // V block of this tile: QR -> rows T0.. of V (A operand); LQ -> V(T0 + n, k) (B operand)
    for (int idx = tid; idx < kStrip * nbp; idx += blockDim.x) {
        int r, k;
        if (SIDE == 0) {
            r = idx % kStrip, k = idx / kStrip;
        } else {
            k = idx % nbp, r = idx / nbp;
        }
        const int g = T0 + r;
        double v = 0.0;
        if (k < nb && r < tw) {
            if (SIDE == 0)
                v = g > k ? V[g + (long)k * ldv] : (g == k ? 1.0 : 0.0);
            else
                v = g > k ? V[k + (long)g * ldv] : (g == k ? 1.0 : 0.0);
        }
        put_op<PREC>(SIDE == 0 ? Aop : Bop, SIDE == 0 ? Aopl : Bopl, tc::kmajor_off(r, k, es, rb3),
                     f64_scaled_to_f32(v, 0));
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = sh->tmem_base;
    if (tid == 0) {
        issue<PREC>(tbase, Aop, Aopl, rb3, Bop, Bopl, rb3, rb3, tc::idesc(P::fmt, 128, 128), false);
        tc::mma_commit(&sh->mbar[0]);
        sh->last_bar = 0;
        sh->last_parity = 0;
    }
    const bool ok = tc::mbar_wait_warp(&sh->mbar[0], 0, info);
    if (!ok && lane == 0) sh->fail = 1;
    tc::fence_after_sync();
    if (ok) {
        // D row = MMA row (QR: X row T0 + row; LQ: strip row L0 + row); D column = MMA column
        const int row = 32 * q + lane;
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tc::tmem_ld16(tbase + hh * 64 + c + ((uint32_t)(32 * q) << 16), v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = hh * 64 + c + i;
                if (SIDE == 0) {
                    if (row < tw && col < lw) {
                        double *px = X + (T0 + row) + (long)(L0 + col) * ldx;
                        *px -= f32_scaled_to_f64(v[i], exs[col]);
                    }
                } else {
                    if (row < lw && col < tw) {
                        double *px = X + (L0 + row) + (long)(T0 + col) * ldx;
                        *px -= f32_scaled_to_f64(v[i], exs[row]);
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) drain_after_failure(sh);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 128);
}

size_t tc_w_smem(int es, int nsp) {
    const size_t rb1 = (size_t)kKt * es;
    return std::max((size_t)nsp * (2 * kStrip * rb1 + 2 * 64 * rb1) + 2 * kStrip * 4 + 2 * kStrip * 8 +
                        sizeof(TcShared) + 64,
                    (size_t)64 * kStrip * 4 + kStrip * 4 + 64);
}
size_t tc_x_smem(int es, int nbp, int nsp) {
    return (size_t)nsp * 2 * kStrip * nbp * es + kStrip * 4 + 2 * kStrip * 4 + sizeof(TcShared) + 64;
}

template <int PREC, int SIDE>
cudaError_t launch_tc(double *X, long ldx, int M, int N, const double *V, long ldv, int nb, const double *Tm,
                      const UpdScratch &sc, int *info, cudaStream_t st) {
    const int nbp = nb <= 32 ? 32 : 64;
    const int es = Prec<PREC>::es, nsp = Prec<PREC>::split ? 2 : 1;
    static PerDeviceOnce a1, a3;
    allow_max_smem(tc_w_kernel<PREC, SIDE>, a1);
    allow_max_smem(tc_x_kernel<PREC, SIDE>, a3);
    const int Lext = SIDE == 0 ? N : M, Kext = SIDE == 0 ? M : N;
    const int nblk = (Lext + kStrip - 1) / kStrip;
    int S = (3 * device_sm_count() + nblk - 1) / nblk;
    S = std::max(1, std::min({S, 8, (Kext + kKt - 1) / kKt}));
    int Ls = ((Kext + S - 1) / S + kKt - 1) / kKt * kKt;
    S = (Kext + Ls - 1) / Ls;
    // scratch (FP64-element workspace of 10 * 64 * max(M, N) entries): 8 partial slabs of
    // W / Y, the finished W' / Y', then the partials' and the result's line exponents
    const size_t L = (size_t)std::max(M, N);
    float *part = reinterpret_cast<float *>(sc.work);
    float *fin = part + (size_t)8 * 64 * L;
    int *pexp = reinterpret_cast<int *>(fin + (size_t)64 * L);
    int *finexp = pexp + (size_t)8 * L;
    tc_w_kernel<PREC, SIDE><<<dim3(nblk, S), kTcThreads, tc_w_smem(es, nsp), st>>>(X, ldx, M, N, V, ldv, nb, nbp, Tm, Ls,
                                                                             part, pexp, fin, finexp, sc.tickets, info);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int Text = SIDE == 0 ? M : N;
    tc_x_kernel<PREC, SIDE><<<dim3(nblk, (Text + kStrip - 1) / kStrip), kTcThreads, tc_x_smem(es, nbp, nsp), st>>>(
        X, ldx, M, N, V, ldv, nb, nbp, fin, finexp, info);
    return cudaGetLastError();
}

// Element-wise check of the two conversions (nla_scale_selftest).
__global__ void scale_selftest_kernel(int n, const double *x, const int *ex, float *f, const float *v, const int *ev,
                                      double *d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    f[i] = f64_scaled_to_f32(x[i], ex[i]);
    d[i] = f32_scaled_to_f64(v[i], ev[i]);
}

}  // namespace

cudaError_t trail_tc(int side, double *X, long ldx, int M, int N, const double *V, long ldv, int nb, const double *Tm,
                     int prec, const UpdScratch &sc, int *info, cudaStream_t st) {
    if (M <= 0 || N <= 0 || nb <= 0) return cudaSuccess;
    if (nb > 64 || !sc.work || !sc.tickets) return cudaErrorInvalidValue;
    if (prec == NLA_UPD_TF32)
        return side == 0 ? launch_tc<NLA_UPD_TF32, 0>(X, ldx, M, N, V, ldv, nb, Tm, sc, info, st)
                         : launch_tc<NLA_UPD_TF32, 1>(X, ldx, M, N, V, ldv, nb, Tm, sc, info, st);
    if (prec == NLA_UPD_BF16)
        return side == 0 ? launch_tc<NLA_UPD_BF16, 0>(X, ldx, M, N, V, ldv, nb, Tm, sc, info, st)
                         : launch_tc<NLA_UPD_BF16, 1>(X, ldx, M, N, V, ldv, nb, Tm, sc, info, st);
    if (prec == NLA_UPD_TF32X3)
        return side == 0 ? launch_tc<NLA_UPD_TF32X3, 0>(X, ldx, M, N, V, ldv, nb, Tm, sc, info, st)
                         : launch_tc<NLA_UPD_TF32X3, 1>(X, ldx, M, N, V, ldv, nb, Tm, sc, info, st);
    if (prec == NLA_UPD_BF16X3)
        return side == 0 ? launch_tc<NLA_UPD_BF16X3, 0>(X, ldx, M, N, V, ldv, nb, Tm, sc, info, st)
                         : launch_tc<NLA_UPD_BF16X3, 1>(X, ldx, M, N, V, ldv, nb, Tm, sc, info, st);
    return cudaErrorInvalidValue;
}

cudaError_t trail_left_tc(double *X, long ldx, int M, int N, const double *Vp, long ldv, int nb, const double *Tm,
                          int prec, const UpdScratch &sc, int *info, cudaStream_t st) {
    return trail_tc(0, X, ldx, M, N, Vp, ldv, nb, Tm, prec, sc, info, st);
}

cudaError_t trail_right_tc(double *X, long ldx, int M, int N, const double *Vt, long ldvt, int nb, const double *Tm,
                           int prec, const UpdScratch &sc, int *info, cudaStream_t st) {
    return trail_tc(1, X, ldx, M, N, Vt, ldvt, nb, Tm, prec, sc, info, st);
}

}  // namespace nla

extern "C" nla_status nla_tc_selftest(int prec, int K, int N, const float *dA, const float *dB, float *dD, int *dInfo,
                                      nla_stream_t stream) {
    if ((prec != NLA_UPD_TF32 && prec != NLA_UPD_BF16) || K < 16 || K > 128 || K % 16 || N < 16 || N > 256 ||
        N % 16 || !dA || !dB || !dD || !dInfo)
        return NLA_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int es = prec == NLA_UPD_TF32 ? 4 : 2;
    const size_t smem = (size_t)(128 + N) * K * es + sizeof(nla::TcShared) + 64;
    cudaMemsetAsync(dInfo, 0, sizeof(int), st);
    if (prec == NLA_UPD_TF32) {
        cudaFuncSetAttribute(nla::tc_selftest_kernel<NLA_UPD_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
        nla::tc_selftest_kernel<NLA_UPD_TF32><<<1, 128, smem, st>>>(dA, dB, dD, K, N, dInfo);
    } else {
        cudaFuncSetAttribute(nla::tc_selftest_kernel<NLA_UPD_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
        nla::tc_selftest_kernel<NLA_UPD_BF16><<<1, 128, smem, st>>>(dA, dB, dD, K, N, dInfo);
    }
    return cudaGetLastError() == cudaSuccess ? NLA_OK : NLA_ERR_CUDA;
}

extern "C" nla_status nla_scale_selftest(int n, const double *dX, const int *dEx, float *dF, const float *dV,
                                         const int *dEv, double *dD, nla_stream_t stream) {
    if (n < 0 || (n > 0 && (!dX || !dEx || !dF || !dV || !dEv || !dD))) return NLA_ERR_ARG;
    if (n == 0) return NLA_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    nla::scale_selftest_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, dX, dEx, dF, dV, dEv, dD);
    return cudaGetLastError() == cudaSuccess ? NLA_OK : NLA_ERR_CUDA;
}
