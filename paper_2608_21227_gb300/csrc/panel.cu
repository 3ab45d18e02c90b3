// panel.cu -- Householder panel factorisation (the GEQRT/TSQRT step of
// Algorithm 1: "QR sweep" on a tile column, "LQ sweep" on a tile row).
//
// One cooperative launch factors an M x nb panel (nb <= 64).  The panel is
// split into row chunks, one per block, held in shared memory for the whole
// factorisation, so the panel is read from and written to global memory once.
// Column j needs one grid-wide reduction: every block contributes partial sums
// of ||x||^2 and of x . a_c for the columns c > j right of it (x = column j
// below the diagonal), the partials meet in global memory behind a counter
// barrier, and each block then finishes the reflector redundantly and updates
// its own rows.  The dot products are taken before beta is known, using
// v = [1; x / (alpha - beta)] so that v . a_c = a_jc + (x . a_c) / (alpha - beta);
// that is what makes one barrier per column enough.
//
// After the last column a second reduction forms G = V^T V and block 0 builds
// the compact-WY factor T (H_1 ... H_nb = I - V T V^T, T upper triangular,
// T_jj = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) G(0:j, j)), which the trailing
// update (Algorithm 2) consumes.
//
// Householder convention (LAPACK-style): beta = -sign(alpha) ||[alpha; x]||,
// sign(0) = +1, tau = (beta - alpha) / beta; a zero x gives tau = 0, H = I.
// Norms and the cross-block sums are FP64 in every precision mode.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace nla {

constexpr int kPanelThreads = 256;
constexpr int kNbMax = 64;
constexpr int kPanelRowsTarget = 256;  // rows per block when the panel is long enough

size_t panel_part_doubles(int P) {
    return (size_t)2 * P * (kNbMax + 1) + (size_t)P * kNbMax * kNbMax + 2 * kNbMax;
}

int device_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int panel_max_ctas() { return device_sm_count(); }

template <typename T>
__global__ void __launch_bounds__(kPanelThreads)
panel_kernel(T *__restrict__ P, long rs, long cs, int M, int nb, int R, T *__restrict__ tau,
             T *__restrict__ Tm, unsigned int *bar, double *part, int *info) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);  // R x nb, column c at S + c*R
    // G = V^T V and T (nb x nb each, row-major, ld nb) after the panel rows
    double *Gs = reinterpret_cast<double *>(smem_raw + (((size_t)R * nb * sizeof(T) + 15) & ~(size_t)15));
    double *Ts = Gs + (size_t)nb * nb;
    __shared__ double red[kNbMax + 1];
    __shared__ double rowv[kNbMax + 1];
    __shared__ T wcoef[kNbMax + 1];
    __shared__ double sh_tau, sh_beta, sh_scale;
    __shared__ int sh_fail;

    const int p = blockIdx.x, nP = gridDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int r0 = p * R;
    const int nr = max(0, min(M, r0 + R) - r0);
    const int kmax = min(nb, M);
    double *colpart = part;                                    // [2][nP][kNbMax+1]
    double *gpart = part + (size_t)2 * nP * (kNbMax + 1);      // [nP][kNbMax*kNbMax]
    double *rowbuf = gpart + (size_t)nP * kNbMax * kNbMax;     // [2][kNbMax]

    if (tid == 0) sh_fail = 0;
    if (p == 0)
        for (int j = kmax + tid; j < nb; j += blockDim.x) tau[j] = T(0);

    // ---- load the block's rows of the panel into shared memory
    if (cs == 1) {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int c = idx % nb, rr = idx / nb;
            S[(size_t)c * R + rr] = P[(long)(r0 + rr) * rs + c];
        }
    } else {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int rr = idx % nr, c = idx / nr;
            S[(size_t)c * R + rr] = P[(long)(r0 + rr) * rs + (long)c * cs];
        }
    }
    __syncthreads();

    for (int j = 0; j < kmax; ++j) {
        const int buf = j & 1;
        const int nitem = nb - j;  // item 0: ||x||^2; item t > 0: x . a_{j+t}
        const int rr_lo = max(0, j + 1 - r0);
        double *cp = colpart + ((size_t)buf * nP + p) * (kNbMax + 1);
        const T *xj = S + (size_t)j * R;
        for (int it = warp; it < nitem; it += nwarps) {
            if (it == 0) {
                T s = T(0);
                for (int rr = rr_lo + lane; rr < nr; rr += 32) s += xj[rr] * xj[rr];
                s = warp_sum(s);
                if (lane == 0) cp[0] = (double)s;
            } else {
                const T *ac = S + (size_t)(j + it) * R;
                T s = T(0);
                for (int rr = rr_lo + lane; rr < nr; rr += 32) s += xj[rr] * ac[rr];
                s = warp_sum(s);
                if (lane == 0) cp[it] = (double)s;
            }
        }
        if (j >= r0 && j < r0 + nr)
            for (int c = j + tid; c < nb; c += blockDim.x)
                rowbuf[buf * kNbMax + (c - j)] = (double)S[(size_t)c * R + (j - r0)];
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            atomicAdd(bar, 1u);
            if (!spin_until_geq(bar, (unsigned)(j + 1) * (unsigned)nP, info, 32)) sh_fail = 1;
            __threadfence();
        }
        __syncthreads();
        if (sh_fail) return;

        // fixed-order sum of the partials (deterministic across runs): each item is
        // split over `sub` threads whose independent loads are in flight together
        {
            const int sub = nitem <= 32 ? 8 : 4;  // 256 threads cover up to 64 items
            const int it = tid / sub, part = tid % sub;
            double s = 0.0;
            if (it < nitem) {
                const double *base = colpart + (size_t)buf * nP * (kNbMax + 1) + it;
#pragma unroll 8
                for (int q = part; q < nP; q += sub) s += ld_cg(base + (size_t)q * (kNbMax + 1));
            }
            for (int o = sub >> 1; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, sub);
            if (it < nitem && part == 0) {
                red[it] = s;
                rowv[it] = ld_cg(rowbuf + buf * kNbMax + it);
            }
        }
        __syncthreads();
        if (tid == 0) {
            double alpha = rowv[0], xn2 = red[0];
            double tj = 0.0, beta = alpha, scale = 0.0;
            if (xn2 > 0.0) {
                double r = sqrt(alpha * alpha + xn2);
                beta = alpha >= 0.0 ? -r : r;
                tj = (beta - alpha) / beta;
                scale = 1.0 / (alpha - beta);
            }
            sh_tau = tj;
            sh_beta = beta;
            sh_scale = scale;
            if (p == 0) tau[j] = (T)tj;
        }
        __syncthreads();
        const double tj = sh_tau, sc = sh_scale;
        for (int it = 1 + tid; it < nitem; it += blockDim.x) wcoef[it] = (T)(tj * (rowv[it] + sc * red[it]));
        __syncthreads();
        if (tj != 0.0) {
            const T scT = (T)sc;
            for (int rr = rr_lo + tid; rr < nr; rr += blockDim.x) {
                T v = S[(size_t)j * R + rr] * scT;  // reflector entry v_r
                for (int c = j + 1; c < nb; ++c) S[(size_t)c * R + rr] -= v * wcoef[c - j];
                S[(size_t)j * R + rr] = v;
            }
            if (j >= r0 && j < r0 + nr) {  // row j itself: v_j = 1
                for (int c = j + 1 + tid; c < nb; c += blockDim.x) S[(size_t)c * R + (j - r0)] -= wcoef[c - j];
                if (tid == 0) S[(size_t)j * R + (j - r0)] = (T)sh_beta;
            }
        }
        __syncthreads();
    }

    // ---- write the factored rows back
    if (cs == 1) {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int c = idx % nb, rr = idx / nb;
            P[(long)(r0 + rr) * rs + c] = S[(size_t)c * R + rr];
        }
    } else {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int rr = idx % nr, c = idx / nr;
            P[(long)(r0 + rr) * rs + (long)c * cs] = S[(size_t)c * R + rr];
        }
    }

    // ---- partial Gram matrix G(i, k) = v_i . v_k (i < k) over this block's rows.
    // v_c has an implicit 1 in row c and zeros above it.
    double *gp = gpart + (size_t)p * kNbMax * kNbMax;
    for (int it = warp; it < nb * nb; it += nwarps) {
        int i = it / nb, k = it % nb;
        if (i >= k || k >= kmax) continue;
        T s = T(0);
        for (int rr = (k > r0 ? ((k - r0) & ~31) : 0) + lane; rr < nr; rr += 32) {  // rows below k only
            const int r = r0 + rr;
            if (r < k) continue;
            const T vk = (r == k) ? T(1) : S[(size_t)k * R + rr];
            s += S[(size_t)i * R + rr] * vk;  // r >= k > i: stored tail
        }
        s = warp_sum(s);
        if (lane == 0) gp[i * kNbMax + k] = (double)s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(bar, 1u);

    if (p == 0) {
        if (tid == 0 && !spin_until_geq(bar, (unsigned)(kmax + 1) * (unsigned)nP, info)) sh_fail = 1;
        __syncthreads();
        if (sh_fail) return;
        for (int it = tid; it < nb * nb; it += blockDim.x) {
            int i = it / nb, k = it % nb;
            double s = 0.0;
            if (i < k && k < kmax)
                for (int q = 0; q < nP; ++q) s += ld_cg(gpart + (size_t)q * kNbMax * kNbMax + i * kNbMax + k);
            Gs[i * nb + k] = s;
            Ts[i * nb + k] = 0.0;
        }
        __syncthreads();
        for (int k = 0; k < nb; ++k) {
            double tk = (k < kmax) ? (double)tau[k] : 0.0;
            double t = 0.0;
            if (tid < k)
                for (int q = tid; q < k; ++q) t += Ts[tid * nb + q] * Gs[q * nb + k];
            __syncthreads();
            if (tid < k) Ts[tid * nb + k] = -tk * t;
            if (tid == k) Ts[k * nb + k] = tk;
            __syncthreads();
        }
        for (int it = tid; it < nb * nb; it += blockDim.x) {
            int i = it % nb, k = it / nb;
            Tm[i + (size_t)k * nb] = (T)Ts[i * nb + k];
        }
    }
    // ---- the last block out resets the counters for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned int prev = atomicAdd(bar + 1, 1u);
        if (prev == (unsigned)nP - 1) {
            atomicExch(bar, 0u);
            atomicExch(bar + 1, 0u);
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------ cluster variant
// Same algorithm with the panel spread over one thread-block cluster (up to 16
// blocks on one GPC): the per-column partial sums live in each block's shared
// memory, are read by every block through distributed shared memory, and the
// hardware cluster barrier replaces the global counter barrier.
template <typename T>
__global__ void __launch_bounds__(kPanelThreads)
panel_cluster_kernel(T *__restrict__ P, long rs, long cs, int M, int nb, int R, T *__restrict__ tau,
                     T *__restrict__ Tm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int p = (int)cluster.block_rank(), nP = (int)cluster.num_blocks();
    T *S = reinterpret_cast<T *>(smem_raw);  // R x nb
    double *Gs = reinterpret_cast<double *>(smem_raw + (((size_t)R * nb * sizeof(T) + 15) & ~(size_t)15));
    double *Ts = Gs + (size_t)nb * nb;
    __shared__ double cpart[2][kNbMax + 1];  // this block's partial sums, double-buffered by column parity
    __shared__ double rowb[2][kNbMax + 1];   // row j (owner block only)
    __shared__ T wcoef[kNbMax + 1];
    __shared__ double sh_tau, sh_beta, sh_scale;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int r0 = p * R;
    const int nr = max(0, min(M, r0 + R) - r0);
    const int kmax = min(nb, M);
    if (p == 0)
        for (int j = kmax + tid; j < nb; j += blockDim.x) tau[j] = T(0);
    if (cs == 1) {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int c = idx % nb, rr = idx / nb;
            S[(size_t)c * R + rr] = P[(long)(r0 + rr) * rs + c];
        }
    } else {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int rr = idx % nr, c = idx / nr;
            S[(size_t)c * R + rr] = P[(long)(r0 + rr) * rs + (long)c * cs];
        }
    }
    __syncthreads();
    for (int j = 0; j < kmax; ++j) {
        const int buf = j & 1;
        const int nitem = nb - j;
        const int rr_lo = max(0, j + 1 - r0);
        const T *xj = S + (size_t)j * R;
        for (int it = warp; it < nitem; it += nwarps) {
            double sacc;
            if (it == 0) {
                T s2 = T(0);
                for (int rr = rr_lo + lane; rr < nr; rr += 32) s2 += xj[rr] * xj[rr];
                sacc = (double)warp_sum(s2);
            } else {
                const T *ac = S + (size_t)(j + it) * R;
                T s1 = T(0);
                for (int rr = rr_lo + lane; rr < nr; rr += 32) s1 += xj[rr] * ac[rr];
                sacc = (double)warp_sum(s1);
            }
            if (lane == 0) cpart[buf][it] = sacc;
        }
        const int owner = j / R;
        if (p == owner)
            for (int c = j + tid; c < nb; c += blockDim.x) rowb[buf][c - j] = (double)S[(size_t)c * R + (j - r0)];
        cluster.sync();
        // warp 0: fixed-order sum over the cluster's blocks (every remote load in
        // flight at once), the reflector in the panel's precision, and the update
        // coefficients w_c = tau (a_jc + x . a_c / (alpha - beta)) = tau v . a_c
        if (warp == 0) {
            const int i0 = lane, i1 = lane + 32;  // items: nitem <= kNbMax = 64
            double s0 = 0.0, s1 = 0.0, w0 = 0.0, w1 = 0.0;
            {
                double v0[16], v1[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    v0[q] = 0.0;
                    v1[q] = 0.0;
                    if (q < nP) {
                        const double *cp = cluster.map_shared_rank(&cpart[buf][0], q);
                        if (i0 < nitem) v0[q] = cp[i0];
                        if (i1 < nitem) v1[q] = cp[i1];
                    }
                }
                const double *rb = cluster.map_shared_rank(&rowb[buf][0], owner);
                if (i0 < nitem) w0 = rb[i0];
                if (i1 < nitem) w1 = rb[i1];
#pragma unroll
                for (int q = 0; q < 16; ++q) s0 += v0[q], s1 += v1[q];
            }
            const T alpha = (T)__shfl_sync(0xffffffffu, w0, 0), xn2 = (T)__shfl_sync(0xffffffffu, s0, 0);
            T tj = T(0), beta = alpha, scale = T(0);
            if (xn2 > T(0)) {
                const T r = sqrt(alpha * alpha + xn2);
                beta = alpha >= T(0) ? -r : r;
                tj = (beta - alpha) / beta;
                scale = T(1) / (alpha - beta);
            }
            if (lane == 0) {
                sh_tau = (double)tj;
                sh_beta = (double)beta;
                sh_scale = (double)scale;
                if (p == 0) tau[j] = tj;
            }
            if (i0 >= 1 && i0 < nitem) wcoef[i0] = tj * ((T)w0 + scale * (T)s0);
            if (i1 < nitem) wcoef[i1] = tj * ((T)w1 + scale * (T)s1);
        }
        __syncthreads();
        const double tj = sh_tau, sc = sh_scale;
        if (tj != 0.0) {
            const T scT = (T)sc;
            for (int rr = rr_lo + tid; rr < nr; rr += blockDim.x) {
                T v = S[(size_t)j * R + rr] * scT;
                for (int c = j + 1; c < nb; ++c) S[(size_t)c * R + rr] -= v * wcoef[c - j];
                S[(size_t)j * R + rr] = v;
            }
            if (p == owner) {
                for (int c = j + 1 + tid; c < nb; c += blockDim.x) S[(size_t)c * R + (j - r0)] -= wcoef[c - j];
                if (tid == 0) S[(size_t)j * R + (j - r0)] = (T)sh_beta;
            }
        }
        __syncthreads();
    }
    if (cs == 1) {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int c = idx % nb, rr = idx / nb;
            P[(long)(r0 + rr) * rs + c] = S[(size_t)c * R + rr];
        }
    } else {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int rr = idx % nr, c = idx / nr;
            P[(long)(r0 + rr) * rs + (long)c * cs] = S[(size_t)c * R + rr];
        }
    }
    // partial Gram matrix of this block's rows into its own Gs
    for (int it = warp; it < nb * nb; it += nwarps) {
        int i = it / nb, k = it % nb;
        T sacc = T(0);
        if (i < k && k < kmax) {
            for (int rr = (k > r0 ? ((k - r0) & ~31) : 0) + lane; rr < nr; rr += 32) {  // rows below k only
                const int r = r0 + rr;
                if (r < k) continue;
                const T vk = (r == k) ? T(1) : S[(size_t)k * R + rr];
                sacc += S[(size_t)i * R + rr] * vk;
            }
            sacc = warp_sum(sacc);
        }
        if (lane == 0) Gs[i * nb + k] = (double)sacc;
    }
    cluster.sync();
    if (p == 0) {
        for (int it = tid; it < nb * nb; it += blockDim.x) {
            int i = it / nb, k = it % nb;
            double sum = 0.0;
            if (i < k && k < kmax)
                for (int q = 0; q < nP; ++q) sum += cluster.map_shared_rank(Gs, q)[it];
            Ts[it] = sum;  // the summed Gram matrix (read below as G)
        }
    }
    cluster.sync();  // every remote read is done: blocks may leave after this point
    if (p != 0) return;
    // T from G = Ts (summed Gram), built in Gs (no longer read remotely)
    for (int it = tid; it < nb * nb; it += blockDim.x) Gs[it] = 0.0;
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        double tk = (k < kmax) ? (double)tau[k] : 0.0;
        double t = 0.0;
        if (tid < k)
            for (int q = tid; q < k; ++q) t += Gs[tid * nb + q] * Ts[q * nb + k];
        __syncthreads();
        if (tid < k) Gs[tid * nb + k] = -tk * t;
        if (tid == k) Gs[k * nb + k] = tk;
        __syncthreads();
    }
    for (int it = tid; it < nb * nb; it += blockDim.x) {
        int i = it % nb, k = it / nb;
        Tm[i + (size_t)k * nb] = (T)Gs[i * nb + k];
    }
}

// ------------------------------------------------------------------ TSQR variant
// Communication-avoiding panel: each block of the cluster factors its own rows
// (local Householder QR, block barriers only), block 0 factors the stacked
// triangular factors, every block forms its rows of the explicit Q1 = Q(:, 0:nb),
// and the compact-WY pair (V, T) of the Householder QR of the whole panel is
// recovered from Q1 by an LU factorisation without pivoting (Householder
// reconstruction): with Sigma = diag(+-1) chosen on the fly so that every pivot
// has magnitude >= 1,
//     Q1 - [Sigma; 0] = V U,   T = -U Sigma V1^{-T},   R := Sigma R,
// since I - V T V^T has first columns Q1 Sigma (V1 = top nb x nb block of V).
// Four cluster barriers per panel instead of one per column.

// Householder QR of the rows x cols column-major block A (column c at A + c*ld)
// by one thread block: reflector tails overwrite the strictly lower part, R the
// upper part, tau[cols].  Warp 0 forms each reflector; each warp then applies it
// to the columns it owns.
template <typename T>
__device__ void block_house_qr(T *A, int ld, int rows, int cols, T *tau, T *sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < cols; ++j) {
        if (warp == 0) {
            T *x = A + (size_t)j * ld;
            if (j > 0) {  // finish the previous column: v = x / (alpha - beta), R entry = beta
                T *xp = A + (size_t)(j - 1) * ld;
                const T s0 = sc[1];
                for (int r = j + lane; r < rows; r += 32) xp[r] *= s0;
                if (lane == 0) xp[j - 1] = sc[2];
            }
            T s2 = T(0);
            for (int r = j + 1 + lane; r < rows; r += 32) s2 += x[r] * x[r];
            s2 = warp_sum(s2);
            if (lane == 0) {
                const T alpha = x[j];
                T tj = T(0), beta = alpha, scale = T(0);
                if (s2 > T(0)) {
                    const T rr = sqrt(alpha * alpha + s2);
                    beta = alpha >= T(0) ? -rr : rr;
                    tj = (beta - alpha) / beta;
                    scale = T(1) / (alpha - beta);
                }
                tau[j] = tj;
                sc[0] = tj;
                sc[1] = tj != T(0) ? scale : T(0);
                sc[2] = tj != T(0) ? beta : alpha;
            }
        }
        __syncthreads();
        const T tj = sc[0], scale = sc[1];
        if (tj != T(0)) {
            const T *x = A + (size_t)j * ld;
            for (int c = j + 1 + warp; c < cols; c += nw) {
                T *a = A + (size_t)c * ld;
                T d = T(0);
                for (int r = j + 1 + lane; r < rows; r += 32) d += x[r] * a[r];
                d = warp_sum(d);
                const T w = tj * (a[j] + scale * d);
                for (int r = j + 1 + lane; r < rows; r += 32) a[r] -= w * scale * x[r];
                __syncwarp();
                if (lane == 0) a[j] -= w;
            }
        }
        __syncthreads();
    }
    if (warp == 0 && cols > 0) {
        T *xp = A + (size_t)(cols - 1) * ld;
        const T s0 = sc[1];
        for (int r = cols + lane; r < rows; r += 32) xp[r] *= s0;
        if (lane == 0) xp[cols - 1] = sc[2];
    }
    __syncthreads();
}

// Q <- H_0 H_1 ... H_{k-1} Q for the reflectors stored in V (unit lower, rows x k,
// column c at V + c*ldv) and tau; Q is rows x cols (column c at Q + c*ldq).  Each
// warp owns whole columns of Q, so no barrier is needed between reflectors.
template <typename T>
__device__ void block_apply_q(const T *V, int ldv, const T *tau, int k, T *Q, int ldq, int rows, int cols) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < cols; c += nw) {
        T *q = Q + (size_t)c * ldq;
        for (int i = k - 1; i >= 0; --i) {
            const T ti = tau[i];
            if (ti == T(0)) continue;
            const T *v = V + (size_t)i * ldv;
            T d = T(0);
            for (int r = i + 1 + lane; r < rows; r += 32) d += v[r] * q[r];
            d = warp_sum(d) + q[i];
            const T w = ti * d;
            for (int r = i + 1 + lane; r < rows; r += 32) q[r] -= w * v[r];
            __syncwarp();
            if (lane == 0) q[i] -= w;
            __syncwarp();
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kPanelThreads)
panel_tsqr_kernel(T *__restrict__ P, long rs, long cs, int M, int nb, int R, T *__restrict__ tau,
                  T *__restrict__ Tm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int p = (int)cluster.block_rank(), nP = (int)cluster.num_blocks();
    const int ZR = nP * nb;  // rows of the stacked triangular factors
    T *S = reinterpret_cast<T *>(smem_raw);  // R x nb: local rows, then local V / R
    T *Qb = S + (size_t)R * nb;              // R x nb: local rows of Q1, then of V
    T *Z = Qb + (size_t)R * nb;              // ZR x nb (block 0): stacked R's -> top V / R
    T *Qt = Z + (size_t)ZR * nb;             // ZR x nb (block 0): explicit top Q
    T *U = Qt + (size_t)ZR * nb;             // nb x nb (column-major), LU upper factor
    T *taul = U + (size_t)nb * nb;           // nb local taus
    T *taut = taul + kNbMax;                 // nb top taus
    T *sg = taut + kNbMax;                   // nb signs
    T *sc = sg + kNbMax;                     // 4 scratch scalars
    const int tid = threadIdx.x;
    const int r0 = p * R;
    const int nr = max(0, min(M, r0 + R) - r0);  // >= nb (host guarantees)
    // ---- load this block's rows
    if (cs == 1) {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            const int c = idx % nb, rr = idx / nb;
            S[(size_t)c * R + rr] = P[(long)(r0 + rr) * rs + c];
        }
    } else {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            const int rr = idx % nr, c = idx / nr;
            S[(size_t)c * R + rr] = P[(long)(r0 + rr) * rs + (long)c * cs];
        }
    }
    __syncthreads();
    // ---- 1. local QR
    block_house_qr<T>(S, R, nr, nb, taul, sc);
    cluster.sync();  // every R_q ready
    // ---- 2. block 0: QR of the stacked R's and the explicit top Q
    if (p == 0) {
        for (int idx = tid; idx < ZR * nb; idx += blockDim.x) {
            const int c = idx / ZR, zr = idx % ZR, q = zr / nb, i = zr % nb;
            T v = T(0);
            if (i <= c) v = cluster.map_shared_rank(S, q)[(size_t)c * R + i];
            Z[(size_t)c * ZR + zr] = v;
            Qt[(size_t)c * ZR + zr] = zr == c ? T(1) : T(0);
        }
        __syncthreads();
        block_house_qr<T>(Z, ZR, ZR, nb, taut, sc);
        block_apply_q<T>(Z, ZR, taut, nb, Qt, ZR, ZR, nb);
    }
    cluster.sync();  // Qt ready
    // ---- 3. local rows of Q1 = Q_p [Qt(p*nb : p*nb+nb, :); 0]
    {
        const T *qt = cluster.map_shared_rank(Qt, 0);
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            const int c = idx / nr, rr = idx % nr;
            Qb[(size_t)c * R + rr] = rr < nb ? qt[(size_t)c * ZR + p * nb + rr] : T(0);
        }
        __syncthreads();
        block_apply_q<T>(S, R, taul, nb, Qb, R, nr, nb);
    }
    // ---- 4. block 0: LU without pivoting of Q1(0:nb, :) - Sigma (one warp, nb <= 64)
    if (p == 0) {
        if (tid < 32) {
            const int lane = tid;
            for (int i = 0; i < nb; ++i) {
                // pivot column i: rows i..nb-1 already updated by steps < i
                const T a = Qb[(size_t)i * R + i];
                const T s = a >= T(0) ? T(-1) : T(1);  // -sign(a), sign(0) = +1
                const T piv = a - s;
                if (lane == 0) {
                    sg[i] = s;
                    Qb[(size_t)i * R + i] = piv;
                }
                __syncwarp();
                const T inv = T(1) / piv;
                for (int k = i + 1 + lane; k < nb; k += 32) Qb[(size_t)i * R + k] *= inv;  // L(k, i)
                __syncwarp();
                // trailing update of rows i+1.., columns i+1..
                for (int c = i + 1; c < nb; ++c) {
                    const T u = Qb[(size_t)c * R + i];
                    for (int k = i + 1 + lane; k < nb; k += 32) Qb[(size_t)c * R + k] -= Qb[(size_t)i * R + k] * u;
                }
                __syncwarp();
            }
            // U (upper, incl. diagonal) to its own array
            for (int idx = lane; idx < nb * nb; idx += 32) {
                const int c = idx / nb, i = idx % nb;
                U[(size_t)c * nb + i] = i <= c ? Qb[(size_t)c * R + i] : T(0);
            }
        }
        __syncthreads();
    }
    cluster.sync();  // U, Sigma ready
    // ---- 5. V rows = Q1 rows U^{-1} (block 0: rows >= nb; rows < nb hold L1 from the LU)
    {
        const T *Uu = U;
        if (p != 0) {  // local copy of block 0's U (this block's Z is unused)
            const T *Ur = cluster.map_shared_rank(U, 0);
            for (int idx = tid; idx < nb * nb; idx += blockDim.x) Z[idx] = Ur[idx];
            __syncthreads();
            Uu = Z;
        }
        const int rbeg = (p == 0) ? nb : 0;
        for (int rr = rbeg + tid; rr < nr; rr += blockDim.x) {
            for (int i = 0; i < nb; ++i) {
                T x = Qb[(size_t)i * R + rr];
                for (int j = 0; j < i; ++j) x -= Qb[(size_t)j * R + rr] * Uu[(size_t)i * nb + j];
                Qb[(size_t)i * R + rr] = x / Uu[(size_t)i * nb + i];
            }
        }
        __syncthreads();
    }
    // ---- 6. write back: V below the diagonal, Sigma R on and above it (block 0)
    if (cs == 1) {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            const int c = idx % nb, rr = idx / nb, r = r0 + rr;
            T v;
            if (r > c)
                v = Qb[(size_t)c * R + rr];
            else
                v = sg[r] * Z[(size_t)c * ZR + r];
            P[(long)r * rs + c] = v;
        }
    } else {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            const int rr = idx % nr, c = idx / nr, r = r0 + rr;
            T v;
            if (r > c)
                v = Qb[(size_t)c * R + rr];
            else
                v = sg[r] * Z[(size_t)c * ZR + r];
            P[(long)r * rs + (long)c * cs] = v;
        }
    }
    // ---- 7. block 0: T = -U Sigma V1^{-T} (upper triangular), tau = diag(T).
    // Row rr of T solves V1 x = -(U Sigma)(rr, :)^T (V1 unit lower = L1 in Qb).
    if (p == 0) {
        for (int rr = tid; rr < nb; rr += blockDim.x) {
            for (int i = 0; i < nb; ++i) {
                T x = T(0);
                if (i >= rr) {
                    x = -U[(size_t)i * nb + rr] * sg[i];
                    for (int j = rr; j < i; ++j) x -= Qb[(size_t)j * R + i] * Tm[rr + (size_t)j * nb];
                }
                Tm[rr + (size_t)i * nb] = x;
            }
            tau[rr] = Tm[rr + (size_t)rr * nb];
        }
    }
    cluster.sync();  // remote reads of every block's shared memory are done
}

// Cluster size and rows per block for the TSQR panel, or 0 when it does not apply:
// 2..16 blocks of <= 512 rows, every block at least nb rows, everything in shared memory.
template <typename T>
static int tsqr_plan(int M, int nb, int &R, size_t &dyn) {
    static bool init = false;
    static size_t max_dyn = 0;
    static bool sched[5] = {false, false, false, false, false};
    if (!init) {
        init = true;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, panel_tsqr_kernel<T>) == cudaSuccess && (size_t)optin > fa.sharedSizeBytes)
            max_dyn = (size_t)optin - fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(panel_tsqr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dyn) !=
                cudaSuccess ||
            cudaFuncSetAttribute(panel_tsqr_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess)
            max_dyn = 0;
        for (int k = 1; k < 5 && max_dyn > 0; ++k) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(1u << k);
            cfg.blockDim = dim3(kPanelThreads);
            cfg.dynamicSmemBytes = max_dyn;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 1u << k;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int ncl = 0;
            sched[k] = cudaOccupancyMaxActiveClusters(&ncl, panel_tsqr_kernel<T>, &cfg) == cudaSuccess && ncl >= 1;
        }
        cudaGetLastError();
    }
    static const int mode = [] {  // NLA_PANEL_TSQR=0 disables this variant
        const char *v = getenv("NLA_PANEL_TSQR");
        return v ? atoi(v) : 1;
    }();
    if (!mode || nb > kNbMax || M < 2 * nb) return 0;
    for (int k = 1; k < 5; ++k) {
        const int C = 1 << k;
        if (!sched[k]) continue;
        const int r = (M + C - 1) / C;
        if (r > 512 && k < 4) continue;        // prefer <= 512 rows per block
        if (M - (C - 1) * r < nb) break;       // the last block needs nb rows
        const size_t zr = (size_t)C * nb;
        const size_t elems = 2 * (size_t)r * nb + 2 * zr * nb + (size_t)nb * nb + 3 * kNbMax + 4;
        const size_t d = elems * sizeof(T);
        if (d > max_dyn) continue;
        R = r;
        dyn = d;
        return C;
    }
    return 0;
}

// Cluster size and rows per block for an M x nb panel, or 0 if it does not fit one cluster.
// Which cluster sizes the device can schedule (one block per SM at the largest
// dynamic shared memory) is asked once; smaller allocations schedule as well.
template <typename T>
static int cluster_plan(int M, int nb, int &R, size_t &dyn) {
    static bool init = false;
    static size_t max_dyn = 0;
    static bool sched[5] = {false, false, false, false, false};  // cluster sizes 1, 2, 4, 8, 16
    if (!init) {
        init = true;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, panel_cluster_kernel<T>) == cudaSuccess && (size_t)optin > fa.sharedSizeBytes)
            max_dyn = (size_t)optin - fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dyn) !=
                cudaSuccess ||
            cudaFuncSetAttribute(panel_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess)
            max_dyn = 0;
        for (int k = 0; k < 5 && max_dyn > 0; ++k) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(1u << k);
            cfg.blockDim = dim3(kPanelThreads);
            cfg.dynamicSmemBytes = max_dyn;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 1u << k;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int ncl = 0;
            sched[k] = cudaOccupancyMaxActiveClusters(&ncl, panel_cluster_kernel<T>, &cfg) == cudaSuccess && ncl >= 1;
        }
        cudaGetLastError();
    }
    int k0 = 0;
    while (k0 < 4 && (1 << k0) * kPanelRowsTarget < M) ++k0;  // smallest size with <= 256 rows per block
    static const int force = [] {  // NLA_PANEL_CLUSTER: cluster size to use where it fits (0: grid kernel)
        const char *v = getenv("NLA_PANEL_CLUSTER");
        return v ? atoi(v) : -1;
    }();
    if (force == 0) return 0;
    int best = 0;
    for (int k = 0; k < 5; ++k) {
        if (!sched[k]) continue;
        if (force > 0 && (1 << k) != force) continue;
        const int C = 1 << k;
        const int r = (M + C - 1) / C;
        const size_t d = (((size_t)r * nb * sizeof(T) + 15) & ~(size_t)15) + (size_t)2 * nb * nb * sizeof(double);
        if (d > max_dyn) continue;
        best = C;
        R = r;
        dyn = d;
        if (k >= k0) break;  // the smallest fitting size at or above the target, else the largest that fits
    }
    return best;
}

template <typename T>
cudaError_t panel_factor(T *P, long rs, long cs, int M, int nb, T *tau, T *Tm, const PanelCtl &ctl,
                         cudaStream_t st) {
    if (M <= 0 || nb <= 0) return cudaSuccess;
    if (nb > kNbMax) return cudaErrorInvalidValue;
    {  // preferred: TSQR + Householder reconstruction in one cluster (four cluster barriers)
        int R = 0;
        size_t dyn = 0;
        const int C = tsqr_plan<T>(M, nb, R, dyn);
        if (C > 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(kPanelThreads);
            cfg.dynamicSmemBytes = dyn;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cudaError_t e = cudaLaunchKernelEx(&cfg, panel_tsqr_kernel<T>, P, rs, cs, M, nb, R, tau, Tm);
            if (e == cudaSuccess) return e;
            cudaGetLastError();
        }
    }
    {  // next: one thread-block cluster, one cluster barrier per column
        int R = 0;
        size_t dyn = 0;
        const int C = cluster_plan<T>(M, nb, R, dyn);
        if (C > 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(kPanelThreads);
            cfg.dynamicSmemBytes = dyn;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cudaError_t e = cudaLaunchKernelEx(&cfg, panel_cluster_kernel<T>, P, rs, cs, M, nb, R, tau, Tm);
            if (e == cudaSuccess) return e;
            cudaGetLastError();  // fall back to the grid-wide version
        }
    }
    static size_t max_dyn = 0;
    static bool attr_set = false;
    if (!attr_set) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, panel_kernel<T>);
        max_dyn = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dyn);
        attr_set = true;
    }
    const int maxP = panel_max_ctas();
    int Pn = std::max(1, std::min(maxP, (M + kPanelRowsTarget - 1) / kPanelRowsTarget));
    const size_t gt_bytes = (size_t)2 * nb * nb * sizeof(double) + 16;
    if (max_dyn <= gt_bytes) return cudaErrorInvalidConfiguration;
    size_t rows_fit = (max_dyn - gt_bytes) / ((size_t)nb * sizeof(T));
    if (rows_fit == 0) return cudaErrorInvalidConfiguration;
    int R = (M + Pn - 1) / Pn;
    if ((size_t)R > rows_fit) {
        Pn = (int)((M + rows_fit - 1) / rows_fit);
        if (Pn > maxP) return cudaErrorInvalidConfiguration;
        R = (M + Pn - 1) / Pn;
    }
    Pn = (M + R - 1) / R;  // no empty blocks
    size_t dyn = (((size_t)R * nb * sizeof(T) + 15) & ~(size_t)15) + (size_t)2 * nb * nb * sizeof(double);

    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Pn);
    cfg.blockDim = dim3(kPanelThreads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, panel_kernel<T>, P, rs, cs, M, nb, R, tau, Tm, ctl.bar, ctl.part,
                              ctl.info);
}

template cudaError_t panel_factor<double>(double *, long, long, int, int, double *, double *,
                                          const PanelCtl &, cudaStream_t);
template cudaError_t panel_factor<float>(float *, long, long, int, int, float *, float *,
                                         const PanelCtl &, cudaStream_t);

}  // namespace nla
