// update_tc.cu -- mixed-precision trailing update on the 5th-generation tensor
// cores: FP64 matrix, TF32 or BF16 operands, FP32 accumulation in TMEM, exact
// power-of-two scaling of the converted operands (the trailing update of
// Algorithm 2 with the mixed-precision form of the contraction).
//
// QR side (one block per 128-column strip of X):
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
constexpr int kTmemCols = 256;    // D1 x 2 (64 columns each) + D3 (128 columns)

template <int PREC>
struct Prec;
template <>
struct Prec<NLA_UPD_TF32> {
    static constexpr int es = 4;
    static constexpr uint32_t fmt = 2;
    NLA_DEV static void put(unsigned char *base, uint32_t off, float v) {
        *reinterpret_cast<uint32_t *>(base + off) = tc::to_tf32(v);
    }
    NLA_DEV static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) { tc::mma_tf32(d, a, b, id, acc); }
};
template <>
struct Prec<NLA_UPD_BF16> {
    static constexpr int es = 2;
    static constexpr uint32_t fmt = 1;
    NLA_DEV static void put(unsigned char *base, uint32_t off, float v) {
        *reinterpret_cast<uint16_t *>(base + off) = tc::to_bf16(v);
    }
    NLA_DEV static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) { tc::mma_bf16(d, a, b, id, acc); }
};

// power-of-two scale exponent: x * 2^-e lies in [0.5, 1) for the largest |x|
NLA_DEV int scale_exp(double mx) {
    if (!(mx > 0.0) || !isfinite(mx)) return 0;
    int e;
    frexp(mx, &e);
    return e;
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

// Issue `count` MMAs of 32 K-bytes each (one thread).
template <int PREC>
NLA_DEV void issue(uint32_t d, const unsigned char *A, int arowbytes, const unsigned char *B, int browbytes,
                   int kbytes, uint32_t id, bool accumulate_first) {
    const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
    for (int kk = 0; kk < kbytes / 32; ++kk) {
        uint64_t ad = tc::sdesc(a0 + kk * 256, 128, 8 * arowbytes);
        uint64_t bd = tc::sdesc(b0 + kk * 256, 128, 8 * browbytes);
        Prec<PREC>::mma(d, ad, bd, id, (kk > 0 || accumulate_first) ? 1u : 0u);
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
        issue<PREC>(tbase, As, rowbytes, Bs, rowbytes, rowbytes, tc::idesc(P::fmt, 128, N), false);
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

// ---------------------------------------------------------------- QR side
template <int PREC>
__global__ void __launch_bounds__(kTcThreads, 1)
trail_left_tc_kernel(double *__restrict__ X, long ldx, int M, int N, const double *__restrict__ V, long ldv, int nb,
                     int nbp, const double *__restrict__ Tm, int *info) {
    using P = Prec<PREC>;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int es = P::es;
    const int rb1 = kKt * es;     // step-1 operand row bytes (K = 32 rows of X)
    const int rb3 = nbp * es;     // step-3 operand row bytes (K = nbp reflectors)
    unsigned char *A1 = sm;                                  // 2 x [128 x kKt]   X^T tiles
    unsigned char *B1 = A1 + 2 * kStrip * rb1;               // 2 x [nbp x kKt]   V tiles (as B^T)
    unsigned char *A3 = B1 + 2 * 64 * rb1;                   // [128 x nbp]       V row tile
    unsigned char *B3 = A3 + kStrip * rb3;                   // [128 x nbp]       W'^T (as B^T)
    float *Wsh = reinterpret_cast<float *>(B3 + kStrip * rb3);  // nbp x 128
    float *Tsh = Wsh + 64 * kStrip;                          // nbp x nbp (column-major)
    int *ex1 = reinterpret_cast<int *>(Tsh + 64 * 64);       // 2 x 128 tile-column exponents
    int *ex3 = ex1 + 2 * kStrip;                             // 128 W' column exponents
    double *cmax = reinterpret_cast<double *>(ex3 + kStrip); // 2 x 128 partial maxima
    TcShared *sh = reinterpret_cast<TcShared *>(cmax + 2 * kStrip);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hh = warp >> 2;  // TMEM lane quarter, column half
    const int c0 = blockIdx.x * kStrip, wc = min(kStrip, N - c0);
    if (warp == 0) {
        tc::tmem_alloc(&sh->tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) tc::mbar_init(&sh->mbar[i], 1);
        sh->fail = 0;
        sh->last_bar = -1;
    }
    for (int idx = tid; idx < nbp * nbp; idx += blockDim.x) {
        int i = idx % nbp, k = idx / nbp;
        Tsh[idx] = (i < nb && k < nb) ? (float)Tm[i + (long)k * nb] : 0.f;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = sh->tmem_base;
    const uint32_t id1 = tc::idesc(P::fmt, 128, nbp), id3 = tc::idesc(P::fmt, 128, 128);
    const int half = nbp / 2;  // accumulator columns per thread

    // ---------------- step 1: W^T = X_strip^T V
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
    const int m = tid & (kStrip - 1), h = tid >> 7;  // loader: strip column m, rows h*16 .. h*16+15
    const int ntiles = (M + kKt - 1) / kKt;
    for (int t = 0; t <= ntiles; ++t) {
        const int buf = t & 1;
        if (t < ntiles) {
            const int r0 = t * kKt;
            double xv[16];
            double mx = 0.0;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int r = r0 + h * 16 + i;
                xv[i] = (m < wc && r < M) ? X[r + (long)(c0 + m) * ldx] : 0.0;
                mx = fmax(mx, fabs(xv[i]));
            }
            cmax[h * kStrip + m] = mx;
            for (int idx = tid; idx < nbp * kKt; idx += blockDim.x) {
                const int k = idx % kKt, n = idx / kKt, gr = r0 + k;
                double v = 0.0;
                if (n < nb && gr < M) v = gr > n ? V[gr + (long)n * ldv] : (gr == n ? 1.0 : 0.0);
                P::put(B1 + buf * 64 * rb1, tc::kmajor_off(n, k, es, rb1), (float)v);
            }
            __syncthreads();
            const int e = scale_exp(fmax(cmax[m], cmax[kStrip + m]));
            if (h == 0) ex1[buf * kStrip + m] = e;
#pragma unroll
            for (int i = 0; i < 16; ++i)
                P::put(A1 + buf * kStrip * rb1, tc::kmajor_off(m, h * 16 + i, es, rb1), (float)ldexp(xv[i], -e));
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                issue<PREC>(tbase + buf * 64, A1 + buf * kStrip * rb1, rb1, B1 + buf * 64 * rb1, rb1, rb1, id1, false);
                tc::mma_commit(&sh->mbar[buf]);
                sh->last_bar = buf;
                sh->last_parity = (t >> 1) & 1;
            }
        }
        if (t > 0) {  // drain tile t-1 while tile t multiplies
            const int pb = (t - 1) & 1;
            const bool ok = tc::mbar_wait_warp(&sh->mbar[pb], ((t - 1) >> 1) & 1, info);
            if (!ok && lane == 0) sh->fail = 1;
            tc::fence_after_sync();
            const int col = 32 * q + lane;
            const float sc = ldexpf(1.f, ex1[pb * kStrip + col]);
            for (int c = 0; ok && c < half; c += 16) {
                float v[16];
                tc::tmem_ld16(tbase + pb * 64 + hh * half + c + ((uint32_t)(32 * q) << 16), v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[c + i] += v[i] * sc;
            }
            tc::fence_before_sync();
        }
        __syncthreads();
        if (sh->fail) break;
    }
    // ---------------- step 2: W' = T^T W (per strip column), scale, round
    const int col = 32 * q + lane;
    if (!sh->fail) {
        for (int i = 0; i < half; ++i) Wsh[(hh * half + i) * kStrip + col] = acc[i];
        __syncthreads();
        double mx = 0.0;
        for (int i = 0; i < half; ++i) {
            const int kk = hh * half + i;
            float s = 0.f;
            for (int k = 0; k <= kk; ++k) s += Tsh[k + kk * nbp] * Wsh[k * kStrip + col];
            acc[i] = s;
            mx = fmax(mx, fabs((double)s));
        }
        cmax[hh * kStrip + col] = mx;
        __syncthreads();
        const int e = scale_exp(fmax(cmax[col], cmax[kStrip + col]));
        if (hh == 0) ex3[col] = e;
        for (int i = 0; i < half; ++i)
            P::put(B3, tc::kmajor_off(col, hh * half + i, es, rb3), ldexpf(acc[i], -e));
    }
    __syncthreads();
    // ---------------- step 3: X_strip -= V W', 128 rows at a time
    const int nrt = (M + kStrip - 1) / kStrip;
    for (int t = 0; t < nrt && !sh->fail; ++t) {
        const int r0 = t * kStrip;
        for (int idx = tid; idx < kStrip * nbp; idx += blockDim.x) {
            const int r = idx % kStrip, k = idx / kStrip, gr = r0 + r;
            double v = 0.0;
            if (k < nb && gr < M) v = gr > k ? V[gr + (long)k * ldv] : (gr == k ? 1.0 : 0.0);
            P::put(A3, tc::kmajor_off(r, k, es, rb3), (float)v);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            issue<PREC>(tbase + 128, A3, rb3, B3, rb3, rb3, id3, false);
            tc::mma_commit(&sh->mbar[2]);
            sh->last_bar = 2;
            sh->last_parity = t & 1;
        }
        if (!tc::mbar_wait_warp(&sh->mbar[2], t & 1, info)) {
            if (lane == 0) sh->fail = 1;
        } else {
            tc::fence_after_sync();
            const int r = r0 + 32 * q + lane;
            for (int c = 0; c < 64; c += 16) {
                float v[16];
                tc::tmem_ld16(tbase + 128 + hh * 64 + c + ((uint32_t)(32 * q) << 16), v);
                tc::tmem_wait_ld();
                if (r < M) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int cc = hh * 64 + c + i;
                        if (cc < wc) {
                            double *px = X + r + (long)(c0 + cc) * ldx;
                            *px -= ldexp((double)v[i], ex3[cc]);
                        }
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) drain_after_failure(sh);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

// ---------------------------------------------------------------- LQ side
template <int PREC>
__global__ void __launch_bounds__(kTcThreads, 1)
trail_right_tc_kernel(double *__restrict__ X, long ldx, int M, int N, const double *__restrict__ Vt, long ldvt, int nb,
                      int nbp, const double *__restrict__ Tm, int *info) {
    using P = Prec<PREC>;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int es = P::es;
    const int rb1 = kKt * es, rb3 = nbp * es;
    unsigned char *A1 = sm;                                  // 2 x [128 x kKt]   X tiles (rows x cols)
    unsigned char *B1 = A1 + 2 * kStrip * rb1;               // 2 x [nbp x kKt]   V tiles (as B^T)
    unsigned char *A3 = B1 + 2 * 64 * rb1;                   // [128 x nbp]       Y' (rows x reflectors)
    unsigned char *B3 = A3 + kStrip * rb3;                   // [128 x nbp]       V tile (as B^T = V rows)
    float *Ysh = reinterpret_cast<float *>(B3 + kStrip * rb3);  // nbp x 128
    float *Tsh = Ysh + 64 * kStrip;
    int *ex1 = reinterpret_cast<int *>(Tsh + 64 * 64);
    int *ex3 = ex1 + 2 * kStrip;
    double *rmax = reinterpret_cast<double *>(ex3 + kStrip);
    TcShared *sh = reinterpret_cast<TcShared *>(rmax + 2 * kStrip);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hh = warp >> 2;
    const int i0 = blockIdx.x * kStrip, hr = min(kStrip, M - i0);
    if (warp == 0) {
        tc::tmem_alloc(&sh->tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) tc::mbar_init(&sh->mbar[i], 1);
        sh->fail = 0;
        sh->last_bar = -1;
    }
    for (int idx = tid; idx < nbp * nbp; idx += blockDim.x) {
        int i = idx % nbp, k = idx / nbp;
        Tsh[idx] = (i < nb && k < nb) ? (float)Tm[i + (long)k * nb] : 0.f;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = sh->tmem_base;
    const uint32_t id1 = tc::idesc(P::fmt, 128, nbp), id3 = tc::idesc(P::fmt, 128, 128);
    const int half = nbp / 2;

    // ---------------- step 1: Y = X_strip V
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
    const int m = tid & (kStrip - 1), h = tid >> 7;  // loader: strip row m, columns h*16 .. h*16+15
    const int ntiles = (N + kKt - 1) / kKt;
    for (int t = 0; t <= ntiles; ++t) {
        const int buf = t & 1;
        if (t < ntiles) {
            const int cb = t * kKt;
            double xv[16];
            double mx = 0.0;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = cb + h * 16 + i;
                xv[i] = (m < hr && c < N) ? X[(i0 + m) + (long)c * ldx] : 0.0;
                mx = fmax(mx, fabs(xv[i]));
            }
            rmax[h * kStrip + m] = mx;
            for (int idx = tid; idx < nbp * kKt; idx += blockDim.x) {
                const int n = idx % nbp, k = idx / nbp, gc = cb + k;
                double v = 0.0;
                if (n < nb && gc < N) v = gc > n ? Vt[n + (long)gc * ldvt] : (gc == n ? 1.0 : 0.0);
                P::put(B1 + buf * 64 * rb1, tc::kmajor_off(n, k, es, rb1), (float)v);
            }
            __syncthreads();
            const int e = scale_exp(fmax(rmax[m], rmax[kStrip + m]));
            if (h == 0) ex1[buf * kStrip + m] = e;
#pragma unroll
            for (int i = 0; i < 16; ++i)
                P::put(A1 + buf * kStrip * rb1, tc::kmajor_off(m, h * 16 + i, es, rb1), (float)ldexp(xv[i], -e));
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (tid == 0) {
                issue<PREC>(tbase + buf * 64, A1 + buf * kStrip * rb1, rb1, B1 + buf * 64 * rb1, rb1, rb1, id1, false);
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
            const int row = 32 * q + lane;
            const float sc = ldexpf(1.f, ex1[pb * kStrip + row]);
            for (int c = 0; ok && c < half; c += 16) {
                float v[16];
                tc::tmem_ld16(tbase + pb * 64 + hh * half + c + ((uint32_t)(32 * q) << 16), v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[c + i] += v[i] * sc;
            }
            tc::fence_before_sync();
        }
        __syncthreads();
        if (sh->fail) break;
    }
    // ---------------- step 2: Y' = Y T (per strip row), scale, round
    const int row = 32 * q + lane;
    if (!sh->fail) {
        for (int i = 0; i < half; ++i) Ysh[(hh * half + i) * kStrip + row] = acc[i];
        __syncthreads();
        double mx = 0.0;
        for (int i = 0; i < half; ++i) {
            const int kk = hh * half + i;
            float s = 0.f;
            for (int k = 0; k <= kk; ++k) s += Ysh[k * kStrip + row] * Tsh[k + kk * nbp];
            acc[i] = s;
            mx = fmax(mx, fabs((double)s));
        }
        rmax[hh * kStrip + row] = mx;
        __syncthreads();
        const int e = scale_exp(fmax(rmax[row], rmax[kStrip + row]));
        if (hh == 0) ex3[row] = e;
        for (int i = 0; i < half; ++i)
            P::put(A3, tc::kmajor_off(row, hh * half + i, es, rb3), ldexpf(acc[i], -e));
    }
    __syncthreads();
    // ---------------- step 3: X_strip -= Y' V^T, 128 columns at a time
    const int nct = (N + kStrip - 1) / kStrip;
    for (int t = 0; t < nct && !sh->fail; ++t) {
        const int cb = t * kStrip;
        for (int idx = tid; idx < kStrip * nbp; idx += blockDim.x) {
            const int k = idx % nbp, n = idx / nbp, gc = cb + n;
            double v = 0.0;
            if (k < nb && gc < N) v = gc > k ? Vt[k + (long)gc * ldvt] : (gc == k ? 1.0 : 0.0);
            P::put(B3, tc::kmajor_off(n, k, es, rb3), (float)v);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            issue<PREC>(tbase + 128, A3, rb3, B3, rb3, rb3, id3, false);
            tc::mma_commit(&sh->mbar[2]);
            sh->last_bar = 2;
            sh->last_parity = t & 1;
        }
        if (!tc::mbar_wait_warp(&sh->mbar[2], t & 1, info)) {
            if (lane == 0) sh->fail = 1;
        } else {
            tc::fence_after_sync();
            const int r = i0 + row;
            const int e = ex3[row];
            for (int c = 0; c < 64; c += 16) {
                float v[16];
                tc::tmem_ld16(tbase + 128 + hh * 64 + c + ((uint32_t)(32 * q) << 16), v);
                tc::tmem_wait_ld();
                if (row < hr) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int cc = cb + hh * 64 + c + i;
                        if (cc < N) {
                            double *px = X + r + (long)cc * ldx;
                            *px -= ldexp((double)v[i], e);
                        }
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) drain_after_failure(sh);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

size_t tc_smem_bytes(int es, int nbp) {
    const size_t rb1 = (size_t)kKt * es, rb3 = (size_t)nbp * es;
    return 2 * kStrip * rb1 + 2 * 64 * rb1 + 2 * kStrip * rb3 + (size_t)64 * kStrip * 4 + 64 * 64 * 4 +
           3 * kStrip * 4 + 2 * kStrip * 8 + sizeof(TcShared) + 64;
}

template <int PREC>
cudaError_t launch_tc(int side, double *X, long ldx, int M, int N, const double *V, long ldv, int nb,
                      const double *Tm, int *info, cudaStream_t st) {
    const int nbp = nb <= 32 ? 32 : 64;
    const size_t smem = tc_smem_bytes(Prec<PREC>::es, nbp);
    if (side == 0) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(trail_left_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            attr = true;
        }
        trail_left_tc_kernel<PREC><<<(N + kStrip - 1) / kStrip, kTcThreads, smem, st>>>(X, ldx, M, N, V, ldv, nb, nbp,
                                                                                        Tm, info);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(trail_right_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            attr = true;
        }
        trail_right_tc_kernel<PREC><<<(M + kStrip - 1) / kStrip, kTcThreads, smem, st>>>(X, ldx, M, N, V, ldv, nb, nbp,
                                                                                         Tm, info);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t trail_tc(int side, double *X, long ldx, int M, int N, const double *V, long ldv, int nb, const double *Tm,
                     int prec, int *info, cudaStream_t st) {
    if (M <= 0 || N <= 0 || nb <= 0) return cudaSuccess;
    if (nb > 64) return cudaErrorInvalidValue;
    if (prec == NLA_UPD_TF32) return launch_tc<NLA_UPD_TF32>(side, X, ldx, M, N, V, ldv, nb, Tm, info, st);
    if (prec == NLA_UPD_BF16) return launch_tc<NLA_UPD_BF16>(side, X, ldx, M, N, V, ldv, nb, Tm, info, st);
    return cudaErrorInvalidValue;
}

cudaError_t trail_left_tc(double *X, long ldx, int M, int N, const double *Vp, long ldv, int nb, const double *Tm,
                          int prec, int *info, cudaStream_t st) {
    return trail_tc(0, X, ldx, M, N, Vp, ldv, nb, Tm, prec, info, st);
}

cudaError_t trail_right_tc(double *X, long ldx, int M, int N, const double *Vt, long ldvt, int nb, const double *Tm,
                           int prec, int *info, cudaStream_t st) {
    return trail_tc(1, X, ldx, M, N, Vt, ldvt, nb, Tm, prec, info, st);
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
