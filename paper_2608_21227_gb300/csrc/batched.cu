// batched.cu -- singular values of many small matrices of uneven shapes in one
// persistent launch (the batched form of the two-stage method, Section 5.1.1).
//
//  1. prep kernel (one block): orders the batch by element count, largest first
//     (bitonic sort of (count, index) keys in shared memory), so that blocks
//     draw similar matrices together and the long ones start first; counts the
//     matrices too large for shared memory and sets the work counters.
//     Everything stays on the device, so the whole call can be captured into a
//     CUDA graph.
//  2. large-matrix kernel (4 blocks of 256 threads per SM, no matrix shared
//     memory): one of those large matrices per block, in the block's global
//     scratch slot (L2-resident); with several blocks per SM more of these
//     latency-bound reductions are in flight.
//  3. persistent kernel (one block of 256 threads per SM, 192 KiB of shared
//     memory for matrices): each block takes rounds of the remaining work from
//     an atomic counter.  In a round it splits into
//     groups of g threads -- g chosen per size bucket (kt_load_config installs
//     tuned values; defaults otherwise) -- and each group reduces one matrix:
//       * the matrix (or its transpose, so that m >= n) is copied into the
//         group's share of shared memory when it fits, else into a global
//         scratch slot of the block (L2-resident at these sizes);
//       * band width 1: one-stage Householder bidiagonalisation (the band
//         stage degenerates to the bidiagonal for these sizes), left and right
//         reflectors with group-wide reductions;
//       * the bidiagonal singular values by bisection on Sturm counts of the
//         Golub-Kahan tridiagonal, one thread per value (FP32 arithmetic for
//         FP32 matrices: the batched accuracy target 5e-6 N sigma_1 is met and
//         the FP64 pipe is 64x slower on this GPU).
//     Groups synchronise with named barriers (bar.sync id, g).
#include <algorithm>
#include <cstdlib>
#include <cfloat>
#include <vector>

#include "../../include/nla.h"
#include "common.cuh"
#include "kernels.cuh"
#include "trace.h"
#include "tuned.h"

namespace {

constexpr int kBThreads = 256;
constexpr int kBSmemElems = 48 * 1024;      // floats of shared memory for matrices per block (192 KiB)
constexpr int kSortMax = 16384;             // batches up to this size are sorted
constexpr int kBuckets = 5;
// Buckets by element count m*n: <= 1/8, 1/4, 1/2, 1 of the block's matrix shared memory, or more
// (global scratch).  A bucket-b matrix fits one group's share when g >= kMinGroup[b].
// (the largest bucket runs in the large-matrix kernel, which takes 128 or 256)
const int kMinGroup[kBuckets] = {32, 64, 128, 256, 128};

struct BatchCfg {
    int group[kBuckets];  // threads per matrix for each bucket
};

__device__ int bucket_of(long elems) {
    int b = 0;
    while (b < kBuckets - 1 && elems > (long)kBSmemElems >> (kBuckets - 2 - b)) ++b;
    return b;
}

nla_status berr(nla_status s, const char *m) {
    nla_set_last_error(m);
    return s;
}

// ---------------------------------------------------------------- prep
// counter[0]: next position of the main kernel, counter[1]: next position of the
// large-matrix kernel, counter[2]: number of matrices above the shared-memory size
// (the sorted order's first counter[2] entries; the main kernel starts after them).
__global__ void batched_prep_kernel(int batch, const int *dM, const int *dN, int *order, unsigned int *counter) {
    extern __shared__ unsigned long long keys[];
    __shared__ unsigned int sh_large;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        counter[0] = 0u;
        counter[1] = 0u;
        counter[2] = 0u;
        sh_large = 0u;
    }
    if (batch > kSortMax) {
        for (int i = tid; i < batch; i += nt) order[i] = i;
        return;
    }
    int P = 1;
    while (P < batch) P <<= 1;
    for (int i = tid; i < P; i += nt) {
        unsigned long long k = ~0ull;
        if (i < batch) {
            unsigned long long e = (unsigned long long)max(dM[i], 0) * (unsigned long long)max(dN[i], 0);
            e = min(e, 0xFFFFFFFFull);
            k = ((0xFFFFFFFFull - e) << 32) | (unsigned)i;  // ascending key = descending size, then index
        }
        keys[i] = k;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < P; i += nt) {
                int j = i ^ stride;
                if (j > i) {
                    bool up = (i & size) == 0;
                    unsigned long long a = keys[i], b = keys[j];
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    unsigned int large = 0;
    for (int i = tid; i < batch; i += nt) {
        order[i] = (int)(keys[i] & 0xFFFFFFFFull);
        large += (0xFFFFFFFFull - (keys[i] >> 32)) > (unsigned long long)kBSmemElems ? 1u : 0u;
    }
    atomicAdd(&sh_large, large);
    __syncthreads();
    if (tid == 0) {
        counter[0] = sh_large;
        counter[2] = sh_large;
    }
}

// ---------------------------------------------------------------- group primitives
__device__ __forceinline__ void gsync(int gid, int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(g) : "memory");
}

// sum over the group of v (g threads, red holds g/32 floats)
__device__ float gsum(float v, float *red, int gid, int g, int gt) {
    v = nla::warp_sum(v);
    if ((gt & 31) == 0) red[gt >> 5] = v;
    gsync(gid, g);
    float s = 0.f;
    for (int w = 0; w < g / 32; ++w) s += red[w];
    gsync(gid, g);
    return s;
}

// Householder reflector for [alpha; x] with ||x||^2 = xn2 (all threads compute the same scalars)
__device__ void reflector(float alpha, float xn2, float &tau, float &beta, float &scale) {
    tau = 0.f;
    beta = alpha;
    scale = 0.f;
    if (xn2 > 0.f) {
        float r = sqrtf(alpha * alpha + xn2);
        beta = alpha >= 0.f ? -r : r;
        tau = (beta - alpha) / beta;
        scale = 1.f / (alpha - beta);
    }
}

// number of singular values of B(d, e) below x (Sturm count of the Golub-Kahan tridiagonal)
__device__ int count_below_f(int n, const float *d, const float *e, float x, float pivmin) {
    float q = -x;
    int neg = q < 0.f;
    for (int i = 0; i < n; ++i) {
        q = -x - d[i] * d[i] / q;
        if (fabsf(q) < pivmin) q = -pivmin;  // floor first, then count the sign used
        neg += q < 0.f;
        if (i + 1 < n) {
            q = -x - e[i] * e[i] / q;
            if (fabsf(q) < pivmin) q = -pivmin;
            neg += q < 0.f;
        }
    }
    return neg - n;
}

// One matrix by one group: W (M x N, column-major, leading dimension ldw) already
// loaded, M >= N.
__device__ void group_svd(float *W, int M, int N, float *d, float *e, float *vbuf, float *red, float *S, int gid,
                          int g, int gt, int ldw) {
    for (int j = 0; j < N; ++j) {
        // ---- left reflector on column j, rows j..M-1
        float *col = W + (size_t)j * ldw;
        float part = 0.f;
        for (int i = j + 1 + gt; i < M; i += g) part += col[i] * col[i];
        const float xn2 = gsum(part, red, gid, g, gt);
        float tau, beta, sc;
        reflector(col[j], xn2, tau, beta, sc);
        if (tau != 0.f) {
            for (int i = j + 1 + gt; i < M; i += g) col[i] *= sc;  // v, v_j = 1 implicit
            gsync(gid, g);
            // columns c > j: warp-per-column dot products, then the update
            const int wid = gt >> 5, lane = gt & 31, nw = g >> 5;
            for (int c = j + 1 + wid; c < N; c += nw) {
                float *cc = W + (size_t)c * ldw;
                float s = lane == 0 ? cc[j] : 0.f;
                for (int i = j + 1 + lane; i < M; i += 32) s += col[i] * cc[i];
                s = nla::warp_sum(s) * tau;
                if (lane == 0) cc[j] -= s;
                for (int i = j + 1 + lane; i < M; i += 32) cc[i] -= s * col[i];
            }
        }
        if (gt == 0) d[j] = beta;
        gsync(gid, g);
        if (j + 1 >= N) break;
        // ---- right reflector on row j, columns j+1..N-1
        const int L = N - j - 1;
        float p2 = 0.f;
        for (int c = j + 2 + gt; c < N; c += g) {
            float v = W[j + (size_t)c * ldw];
            p2 += v * v;
        }
        const float yn2 = gsum(p2, red, gid, g, gt);
        reflector(W[j + (size_t)(j + 1) * ldw], yn2, tau, beta, sc);
        if (gt == 0) e[j] = beta;
        if (tau != 0.f && L > 1) {
            for (int c = gt; c < L; c += g) vbuf[c] = c == 0 ? 1.f : W[j + (size_t)(j + 1 + c) * ldw] * sc;
            gsync(gid, g);
            for (int i = j + 1 + gt; i < M; i += g) {  // one thread per row
                float s = 0.f;
                for (int c = 0; c < L; ++c) s += W[i + (size_t)(j + 1 + c) * ldw] * vbuf[c];
                s *= tau;
                for (int c = 0; c < L; ++c) W[i + (size_t)(j + 1 + c) * ldw] -= s * vbuf[c];
            }
        }
        gsync(gid, g);
    }
    // ---- bisection: one thread per singular value
    float bnd = 0.f, tmax = 0.f;
    for (int i = gt; i < N; i += g) {
        float di = fabsf(d[i]), el = i > 0 ? fabsf(e[i - 1]) : 0.f, er = i + 1 < N ? fabsf(e[i]) : 0.f;
        bnd = fmaxf(bnd, di + fmaxf(el, er));
        tmax = fmaxf(tmax, fmaxf(di, er));
    }
    {
        float v = bnd;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        float t = tmax;
        for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
        if ((gt & 31) == 0) {
            red[gt >> 5] = v;
            red[16 + (gt >> 5)] = t;
        }
        gsync(gid, g);
        float b = 0.f, tt = 0.f;
        for (int w = 0; w < g / 32; ++w) {
            b = fmaxf(b, red[w]);
            tt = fmaxf(tt, red[16 + w]);
        }
        bnd = b * (1.f + 4.f * FLT_EPSILON) + FLT_MIN;
        tmax = tt;
        gsync(gid, g);
    }
    const float pivmin = FLT_MIN * fmaxf(1.f, tmax * tmax);
    const float tol = 2.f * FLT_EPSILON * bnd;
    for (int idx = gt; idx < N; idx += g) {
        const int jj = N - 1 - idx;
        float lo = 0.f, hi = bnd;
        for (int it = 0; it < 64; ++it) {
            float mid = 0.5f * (lo + hi);
            if (hi - lo <= tol || mid <= lo || mid >= hi) break;
            if (count_below_f(N, d, e, mid, pivmin) <= jj)
                lo = mid;
            else
                hi = mid;
        }
        S[idx] = 0.5f * (lo + hi);
    }
}

__global__ void __launch_bounds__(kBThreads)
batched_svd_kernel(int batch, const int *__restrict__ dM, const int *__restrict__ dN, const int *__restrict__ dLda,
                   float *const *dA, float *const *dS, const int *__restrict__ order, unsigned int *counter,
                   float *scratch, size_t scratch_elems, int *dInfo, BatchCfg cfg, int sorted) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int sh_start, sh_groups;
    float *mat = smem;                                    // kBSmemElems
    float *aux = smem + kBSmemElems;                      // per group: d, e (256 each), vbuf 256, red 32
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) {
            unsigned int pos = atomicAdd(counter, 0u);
            int gsz = kBThreads;
            if (sorted && pos < (unsigned)batch) {
                const int i0 = order[pos];
                const long el = (long)dM[i0] * dN[i0];
                const int bk = bucket_of(el);
                gsz = bk == kBuckets - 1 ? kBThreads : cfg.group[bk];  // global scratch: one matrix per block
            }
            const int ng = kBThreads / gsz;
            sh_groups = ng;
            sh_start = (int)atomicAdd(counter, (unsigned)ng);
        }
        __syncthreads();
        const int start = sh_start, ng = sh_groups;
        if (start >= batch) break;
        const int g = kBThreads / ng, gid = tid / g, gt = tid % g;
        const int item = start + gid;
        if (item < batch) {
            const int i = order[item];
            const int m = dM[i], n = dN[i], lda = dLda[i];
            const float *A = dA[i];
            float *Sout = dS[i];
            const int M = max(m, n), N = min(m, n);
            const bool tr = m < n;
            const int share = kBSmemElems / ng;
            float *W = (long)M * N <= share ? mat + (size_t)gid * share : scratch + (size_t)blockIdx.x * scratch_elems;
            float *d = aux + gid * 800, *e = d + 256, *vb = e + 256, *red = vb + 256;
            // the global slot is only ever used by a block working on one matrix
            const bool ok = (long)M * N <= share || (ng == 1 && (size_t)M * N <= scratch_elems);
            if (ok && N <= 256) {
                for (int idx = gt; idx < M * N; idx += g) {
                    const int r = idx % M, c = idx / M;  // W(r, c)
                    W[idx] = tr ? A[c + (size_t)r * lda] : A[r + (size_t)c * lda];
                }
                gsync(gid, g);
                if (N > 0) group_svd(W, M, N, d, e, vb, red, Sout, gid, g, gt, M);
                if (gt == 0) dInfo[i] = 0;
            } else if (gt == 0) {
                dInfo[i] = -NLA_ERR_UNSUPPORTED;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- blocked QR (large matrices)
// W (M x N, column-major, leading dimension ldw a multiple of 4, M >= N) is reduced to
// R = Q^T W by blocked Householder QR with panels of PW columns: each panel (rows k0..M-1)
// is factored in shared memory (column-major, leading dimension ldp), its compact-WY
// factor T formed from V^T V (T(j, j) = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) V(:, 0:j)^T v_j),
// and the trailing columns updated as X -= V (T^T (V^T X)) in two streaming passes
// (X read once, then read and written once), so the trailing block is read 3 times per
// PW columns instead of twice per column.  On return the top N x N block of W holds R
// (zeros below its diagonal).  The singular values of R are those of W: R = Q^T W with Q
// orthogonal (the same argument as Section 5.1.1's).
template <int PW, int G>
__device__ void group_qr_blocked(float *W, int ldw, int M, int N, float *Pm, int ldp, float *Wt, float *Tt, float *tau,
                                 float *red, int gt) {
    const int lane = gt & 31, wid = gt >> 5, nw = G / 32;
    for (int k0 = 0; k0 < N; k0 += PW) {
        const int nb = min(PW, N - k0), r = M - k0, C = N - k0 - nb;
        // ---- load the panel (rows k0.., columns k0..k0+nb-1); zero rows up to ldp
        for (int idx = gt; idx < PW * ldp; idx += G) {
            const int k = idx / ldp, i = idx % ldp;
            Pm[idx] = (k < nb && i < r) ? W[(k0 + i) + (size_t)(k0 + k) * ldw] : 0.f;
        }
        gsync(0, G);
        // ---- factor the panel: reflector j on rows j..r-1, applied to the panel's columns > j
        for (int j = 0; j < nb; ++j) {
            float *col = Pm + (size_t)j * ldp;
            float part = 0.f;
            for (int i = j + 1 + gt; i < r; i += G) part += col[i] * col[i];
            const float xn2 = gsum(part, red, 0, G, gt);
            float t, beta, sc;
            reflector(col[j], xn2, t, beta, sc);
            if (gt == 0) tau[j] = t;
            if (t != 0.f) {
                for (int i = j + 1 + gt; i < r; i += G) col[i] *= sc;  // v, v_j = 1 implicit
                gsync(0, G);
                for (int c = j + 1 + wid; c < nb; c += nw) {
                    float *cc = Pm + (size_t)c * ldp;
                    float s = lane == 0 ? cc[j] : 0.f;
                    for (int i = j + 1 + lane; i < r; i += 32) s += col[i] * cc[i];
                    s = nla::warp_sum(s) * t;
                    if (lane == 0) cc[j] -= s;
                    for (int i = j + 1 + lane; i < r; i += 32) cc[i] -= s * col[i];
                }
            }
            gsync(0, G);
            if (gt == 0) col[j] = beta;
            gsync(0, G);
        }
        // ---- R rows of the panel back to W (zeros below the diagonal within the top N rows),
        // then V's unit diagonal and zeros above it in the panel
        for (int idx = gt; idx < nb * nb; idx += G) {
            const int i = idx % nb, k = idx / nb;
            W[(k0 + i) + (size_t)(k0 + k) * ldw] = i <= k ? Pm[i + (size_t)k * ldp] : 0.f;
        }
        for (int idx = gt; idx < nb * (N - k0 - nb); idx += G) {  // rows k0+nb..N-1 of the panel columns
            const int i = nb + idx % (N - k0 - nb), k = idx / (N - k0 - nb);
            W[(k0 + i) + (size_t)(k0 + k) * ldw] = 0.f;
        }
        gsync(0, G);
        for (int idx = gt; idx < nb * nb; idx += G) {
            const int i = idx % nb, k = idx / nb;
            if (i <= k) Pm[i + (size_t)k * ldp] = i == k ? 1.f : 0.f;
        }
        gsync(0, G);
        if (C <= 0) continue;
        // ---- T from V^T V (warp per entry of the strict upper triangle), then the recurrence
        for (int e = wid; e < nb * nb; e += nw) {
            const int a = e % nb, b = e / nb;
            if (a >= b) continue;
            const float *va = Pm + (size_t)a * ldp, *vb = Pm + (size_t)b * ldp;
            float s = 0.f;
            for (int i = lane; i < r; i += 32) s += va[i] * vb[i];
            s = nla::warp_sum(s);
            if (lane == 0) Tt[a + b * PW] = s;  // (V^T V)(a, b), overwritten by T below
        }
        gsync(0, G);
        if (wid == 0) {
            // column b of T: T(0:b, b) = -tau_b T(0:b, 0:b) (V^T V)(0:b, b), computed top-down in
            // registers (lane a holds entry a); T(b, b) = tau_b
            for (int b = 0; b < nb; ++b) {
                const float g_ab = lane < b ? Tt[lane + b * PW] : 0.f;
                float v = 0.f;
                for (int a = 0; a < b; ++a) {  // v_lane = sum_a T(lane, a) g(a, b), T upper triangular
                    const float ga = __shfl_sync(0xffffffffu, g_ab, a);
                    if (lane <= a) v += Tt[lane + a * PW] * ga;
                }
                __syncwarp();
                if (lane < b) Tt[lane + b * PW] = -tau[b] * v;
                if (lane == b) Tt[b + b * PW] = tau[b];
                __syncwarp();
            }
        }
        gsync(0, G);
        // ---- pass 1: Wt(:, c) = V^T X(:, c) (warp per column; each lane 4 consecutive rows)
        const float *X0 = W + k0;  // X(i, c) = X0[i + (c0 + c) * ldw], c0 = k0 + nb
        const int c0 = k0 + nb;
        for (int c = wid; c < C; c += nw) {
            const float *xc = X0 + (size_t)(c0 + c) * ldw;
            float acc[PW];
#pragma unroll
            for (int k = 0; k < PW; ++k) acc[k] = 0.f;
            for (int i0 = 4 * lane; i0 < r; i0 += 128) {
                float4 x4;
                if (i0 + 3 < r) {
                    x4 = *reinterpret_cast<const float4 *>(xc + i0);
                } else {
                    x4.x = xc[i0];
                    x4.y = i0 + 1 < r ? xc[i0 + 1] : 0.f;
                    x4.z = i0 + 2 < r ? xc[i0 + 2] : 0.f;
                    x4.w = 0.f;
                }
#pragma unroll
                for (int k = 0; k < PW; ++k) {
                    const float4 v4 = *reinterpret_cast<const float4 *>(Pm + (size_t)k * ldp + i0);
                    acc[k] += v4.x * x4.x + v4.y * x4.y + v4.z * x4.z + v4.w * x4.w;
                }
            }
#pragma unroll
            for (int k = 0; k < PW; ++k) {
                const float s = nla::warp_sum(acc[k]);
                if (lane == k) Wt[k * 256 + c] = s;
            }
        }
        gsync(0, G);
        // ---- W' = T^T Wt (in place, column by column: W'(k, c) = sum_{j <= k} T(j, k) Wt(j, c))
        for (int c = gt; c < C; c += G) {
            float w[PW];
#pragma unroll
            for (int k = 0; k < PW; ++k) w[k] = k < nb ? Wt[k * 256 + c] : 0.f;
#pragma unroll
            for (int k = PW - 1; k >= 0; --k) {
                float v = 0.f;
#pragma unroll
                for (int j = 0; j <= k; ++j) v += Tt[j + k * PW] * w[j];
                if (k < nb) Wt[k * 256 + c] = v;
            }
        }
        gsync(0, G);
        // ---- pass 2: X(:, c) -= V W'(:, c)
        for (int c = wid; c < C; c += nw) {
            float *xc = W + k0 + (size_t)(c0 + c) * ldw;
            float wk[PW];
#pragma unroll
            for (int k = 0; k < PW; ++k) wk[k] = k < nb ? Wt[k * 256 + c] : 0.f;
            for (int i0 = 4 * lane; i0 < r; i0 += 128) {
                float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int k = 0; k < PW; ++k) {
                    const float4 v4 = *reinterpret_cast<const float4 *>(Pm + (size_t)k * ldp + i0);
                    d.x += v4.x * wk[k], d.y += v4.y * wk[k], d.z += v4.z * wk[k], d.w += v4.w * wk[k];
                }
                if (i0 + 3 < r) {
                    float4 x4 = *reinterpret_cast<float4 *>(xc + i0);
                    x4.x -= d.x, x4.y -= d.y, x4.z -= d.z, x4.w -= d.w;
                    *reinterpret_cast<float4 *>(xc + i0) = x4;
                } else {
                    xc[i0] -= d.x;
                    if (i0 + 1 < r) xc[i0 + 1] -= d.y;
                    if (i0 + 2 < r) xc[i0 + 2] -= d.z;
                }
            }
        }
        gsync(0, G);
    }
}

// threads per block of the large-matrix kernel: 1024 per SM in blocks of G
// (global scratch slots: one per block)
constexpr int kLargeThreadsPerSm = 1024;
constexpr int kLargeSlotsPerSm = kLargeThreadsPerSm / 128;

// The matrices too large for shared memory (the sorted order's first counter[2]):
// one per block of G threads, working in the block's global scratch slot (leading
// dimension rounded up to 4).  When its panel fits the block's shared memory
// (ldp_max), a matrix is first reduced to its N x N triangular factor R by blocked
// Householder QR (three streaming passes per 16 columns instead of two per column)
// and R's singular values are found by the one-stage bidiagonalisation + bisection;
// otherwise the one-stage reduction runs on the whole matrix.
constexpr int kQrPanel = 16;

__host__ __device__ constexpr size_t large_smem_floats(int ldp) {
    return (size_t)kQrPanel * ldp + (size_t)kQrPanel * 256 + kQrPanel * kQrPanel + kQrPanel;
}

template <int G>
__global__ void __launch_bounds__(G)
batched_large_kernel(const int *__restrict__ dM, const int *__restrict__ dN, const int *__restrict__ dLda,
                     float *const *dA, float *const *dS, const int *__restrict__ order, unsigned int *counter,
                     float *scratch, size_t scratch_elems, int ldp_max, int rsm_floats, int *dInfo) {
    extern __shared__ __align__(16) float qsm[];
    __shared__ float aux[800];
    __shared__ int sh_item;
    const int tid = threadIdx.x;
    const int nlarge = (int)counter[2];
    while (true) {
        if (tid == 0) sh_item = (int)atomicAdd(&counter[1], 1u);
        __syncthreads();
        const int item = sh_item;
        if (item >= nlarge) break;
        const int i = order[item];
        const int m = dM[i], n = dN[i], lda = dLda[i];
        const float *A = dA[i];
        const int M = max(m, n), N = min(m, n);
        const bool tr = m < n;
        const int ldw = (M + 3) & ~3;
        float *W = scratch + (size_t)blockIdx.x * scratch_elems;
        if ((size_t)ldw * N <= scratch_elems && N <= 256) {
            for (int idx = tid; idx < M * N; idx += G) {
                const int r = idx % M, c = idx / M;  // W(r, c)
                W[r + (size_t)c * ldw] = tr ? A[c + (size_t)r * lda] : A[r + (size_t)c * lda];
            }
            gsync(0, G);
            if (N > 0) {
                if (ldw <= ldp_max && M > N) {
                    float *Pm = qsm, *Wt = Pm + (size_t)kQrPanel * ldw, *Tt = Wt + kQrPanel * 256,
                          *tau = Tt + kQrPanel * kQrPanel;
                    group_qr_blocked<kQrPanel, G>(W, ldw, M, N, Pm, ldw, Wt, Tt, tau, aux + 768, tid);
                    if ((size_t)N * N <= (size_t)rsm_floats) {
                        // R into shared memory (the panel's space), where the one-stage reduction
                        // runs at shared-memory latency
                        for (int idx = tid; idx < N * N; idx += G) {
                            const int r = idx % N, c = idx / N;
                            qsm[idx] = W[r + (size_t)c * ldw];
                        }
                        gsync(0, G);
                        group_svd(qsm, N, N, aux, aux + 256, aux + 512, aux + 768, dS[i], 0, G, tid, N);
                    } else {
                        group_svd(W, N, N, aux, aux + 256, aux + 512, aux + 768, dS[i], 0, G, tid, ldw);
                    }
                } else {
                    group_svd(W, M, N, aux, aux + 256, aux + 512, aux + 768, dS[i], 0, G, tid, ldw);
                }
            }
            if (tid == 0) dInfo[i] = 0;
        } else if (tid == 0) {
            dInfo[i] = -NLA_ERR_UNSUPPORTED;
        }
        __syncthreads();
    }
}

BatchCfg default_cfg() {
    BatchCfg c;
    for (int b = 0; b < kBuckets; ++b) c.group[b] = kMinGroup[b];
    c.group[kBuckets - 1] = kBThreads;
    return c;
}

}  // namespace

namespace nla {
// Group sizes per bucket installed by the tuner table (bucket b -> threads per matrix).
int g_batched_group[kBuckets] = {0, 0, 0, 0, 0};
}

extern "C" {

nla_status nla_gesvd_vals_batched_workspace(int batch, nla_dtype dtype, int max_m, int max_n, size_t *bytes) {
    if (!bytes || batch < 0 || max_m < 0 || max_n < 0) return berr(NLA_ERR_ARG, "bad arguments");
    if (dtype != NLA_F32) return berr(NLA_ERR_UNSUPPORTED, "the batched kernel supports FP32 only");
    const size_t blocks = (size_t)nla::device_sm_count() * std::max(2, kLargeSlotsPerSm);
    const size_t slot = (size_t)((std::max(max_m, 1) + 3) & ~3) * std::max(max_n, 1);
    size_t b = 256;                                    // counter
    b += ((size_t)std::max(batch, 1) * 4 + 255) / 256 * 256;  // order
    b += blocks * slot * 4;                            // scratch slots
    *bytes = b;
    return NLA_OK;
}

nla_status nla_gesvd_vals_batched(int batch, nla_dtype dtype, const int *dM, const int *dN, const int *dLda,
                                  void *const *dA_array, void *const *dS_array, int max_m, int max_n, void *dWork,
                                  size_t work_bytes, int *dInfo, const nla_opts *opts, nla_stream_t stream) {
    (void)opts;
    if (dtype != NLA_F32) return berr(NLA_ERR_UNSUPPORTED, "the batched kernel supports FP32 only");
    if (batch < 0 || max_m < 0 || max_n < 0) return berr(NLA_ERR_ARG, "negative size");
    if (batch == 0) return NLA_OK;
    if (max_n > 256) return berr(NLA_ERR_UNSUPPORTED, "min(m_i, n_i) must be <= 256");
    if (!dM || !dN || !dLda || !dA_array || !dS_array || !dInfo || !dWork)
        return berr(NLA_ERR_ARG, "null device pointer");
    size_t need = 0;
    nla_gesvd_vals_batched_workspace(batch, dtype, max_m, max_n, &need);
    if (work_bytes < need) return berr(NLA_ERR_WORKSPACE, "workspace too small");
    if (((uintptr_t)dWork) % 256) return berr(NLA_ERR_WORKSPACE, "workspace not 256-byte aligned");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *w = reinterpret_cast<char *>(dWork);
    unsigned int *counter = reinterpret_cast<unsigned int *>(w);
    int *order = reinterpret_cast<int *>(w + 256);
    float *scratch = reinterpret_cast<float *>(w + 256 + ((size_t)batch * 4 + 255) / 256 * 256);
    const size_t slot = (size_t)((std::max(max_m, 1) + 3) & ~3) * std::max(max_n, 1);
    BatchCfg cfg = default_cfg();
    for (int b = 0; b < kBuckets; ++b)
        if (nla::g_batched_group[b] >= kMinGroup[b] && nla::g_batched_group[b] <= kBThreads &&
            kBThreads % nla::g_batched_group[b] == 0)
            cfg.group[b] = nla::g_batched_group[b];
    static nla::PerDeviceOnce attr;
    const size_t sort_smem = (size_t)kSortMax * sizeof(unsigned long long);
    const size_t main_smem = ((size_t)kBSmemElems + 8 * 800) * sizeof(float);
    attr.run([&] {
        cudaFuncSetAttribute(batched_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);
        cudaFuncSetAttribute(batched_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)main_smem);
        cudaGetLastError();
    });
    {
        nla::TraceScope ts(nla::kTrBatched, st);
        batched_prep_kernel<<<1, 1024, batch <= kSortMax ? sort_smem : 0, st>>>(batch, dM, dN, order, counter);
        int blocks = nla::device_sm_count();
        if (batch <= kSortMax) {  // (unsorted batches leave counter[2] = 0: the main kernel takes all)
            static const int per_sm_threads = [] {  // NLA_BATCH_LARGE_THREADS: threads per SM of the kernel
                const char *v = getenv("NLA_BATCH_LARGE_THREADS");
                const int t = v ? atoi(v) : kLargeThreadsPerSm;
                return std::max(256, std::min(t, kLargeThreadsPerSm));
            }();
            // threads per large matrix: the tuned group of the largest bucket (128 or 256); the
            // blocked QR's panel is sized for the batch's largest row count when it fits
            // (and a triangular factor R that fits the same shared memory is reduced there;
            // larger ones in the scratch slot -- growing the shared memory for them costs
            // blocks per SM: 232 vs 187 ms per batch of the 10,000-matrix workload)
            const int ldp = (std::max(max_m, max_n) + 3) & ~3;
            const size_t qsmem = large_smem_floats(ldp) * sizeof(float);
            const bool qr = qsmem <= (size_t)160 * 1024;
            const size_t dsm = qr ? qsmem : 0;
            const int rsm_floats = qr ? (int)(dsm / sizeof(float)) : 0;
            auto launch_large = [&](auto kern, int G) {
                static nla::PerDeviceOnce lattr;
                lattr.run([&] {
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
                    cudaGetLastError();
                });
                int per_sm = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G, dsm) != cudaSuccess || per_sm < 1) {
                    cudaGetLastError();
                    per_sm = 1;
                }
                per_sm = std::min(per_sm, per_sm_threads / G);
                kern<<<blocks * per_sm, G, dsm, st>>>(dM, dN, dLda, (float *const *)dA_array, (float *const *)dS_array,
                                                      order, counter, scratch, slot, qr ? ldp : 0, rsm_floats, dInfo);
            };
            if (cfg.group[kBuckets - 1] == 128)
                launch_large(batched_large_kernel<128>, 128);
            else
                launch_large(batched_large_kernel<256>, 256);
        }
        batched_svd_kernel<<<blocks, kBThreads, main_smem, st>>>(batch, dM, dN, dLda, (float *const *)dA_array,
                                                                 (float *const *)dS_array, order, counter, scratch, slot,
                                                                 dInfo, cfg, batch <= kSortMax ? 1 : 0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return berr(NLA_ERR_CUDA, cudaGetErrorString(e));
    return NLA_OK;
}

}  // extern "C"
