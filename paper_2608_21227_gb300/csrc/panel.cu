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
// This grid variant takes norms and cross-block sums in FP64 in every precision
// mode; the cluster variant below takes them in the panel's own precision (FP64 for
// the FP64 and mixed-precision paths, FP32 for the plain FP32 path).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace nla {

constexpr int kPanelThreads = 256;
constexpr int kNbMax = 64;
constexpr int kPanelRowsTarget = 256;  // rows per block when the panel is long enough

size_t panel_part_doubles(int P) {
    return (size_t)2 * P * (kNbMax + 1) + (size_t)P * kNbMax * kNbMax + 2 * kNbMax;
}

int current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return dev;
}

int device_sm_count() {
    static PerDeviceValue<int> sms;
    return sms.get([] {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, std::max(current_device(), 0)) != cudaSuccess)
            cudaGetLastError();
        return n > 0 ? n : 1;
    });
}

int panel_max_ctas() { return device_sm_count(); }

// Off by default: at 8192 it measured 182.8 vs 181.9 ms per SVD (the launch gaps
// between the stage-1 kernels are not where the time goes); NLA_PDL=1 enables it.
bool pdl_enabled() {
    static const bool on = [] {
        const char *v = getenv("NLA_PDL");
        return v && atoi(v) != 0;
    }();
    return on;
}

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
// blocks on one GPC).  Per column each block pushes its partial sums (and the
// owner block row j) into every block's shared memory over distributed shared
// memory and arrives on every block's mbarrier; a block waits only on its own
// barrier, so the exchange costs one remote write latency instead of a
// cluster-wide barrier plus remote reads.
constexpr int kClusterThreads = 512;

NLA_DEV uint32_t cluster_addr(const void *local, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc::smem_u32(local)), "r"(rank));
    return r;
}
NLA_DEV void mbar_arrive_remote(uint32_t cluster_mbar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_mbar) : "memory");
}
NLA_DEV bool mbar_try_wait_cluster(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc::smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One element global -> shared as an asynchronous copy (completed by cp.async.wait_all).
template <typename T>
NLA_DEV void cp_async_4or8(T *dst_smem, const T *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(tc::smem_u32(dst_smem)), "l"(src),
                 "n"((int)sizeof(T))
                 : "memory");
}

// Dot product of two columns over rows [lo, hi) of the block, four independent
// partial sums per lane, then a warp reduction.
template <typename T>
NLA_DEV T warp_dot(const T *x, const T *y, int lo, int hi, int lane) {
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int r = lo + lane;
    for (; r + 96 < hi; r += 128) {
        a0 += x[r] * y[r];
        a1 += x[r + 32] * y[r + 32];
        a2 += x[r + 64] * y[r + 64];
        a3 += x[r + 96] * y[r + 96];
    }
    for (; r < hi; r += 32) a0 += x[r] * y[r];
    return warp_sum((a0 + a1) + (a2 + a3));
}

template <typename T>
__global__ void __launch_bounds__(kClusterThreads)
panel_cluster_kernel(T *__restrict__ P, long rs, long cs, int M, int nb, int R, T *__restrict__ tau,
                     T *__restrict__ Tm, int *info) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int p = (int)cluster.block_rank(), nP = (int)cluster.num_blocks();
    T *S = reinterpret_cast<T *>(smem_raw);  // R x nb
    // Per column j the blocks exchange nb partial sums over their rows below j:
    //   item 0            ||x||^2                     (x = column j below row j)
    //   item t in 1..nb-1-j   x . a_{j+t}             (trailing columns)
    //   item nb-j+i, i < j    x . v_i                 (finished reflectors: G(i, j))
    // and the owner of row j pushes row j at the same positions (a_j,j+t and v_i[j]).
    __shared__ T inbox[2][16][kNbMax];  // by column parity and source block
    __shared__ T rowin[2][kNbMax];
    __shared__ T mypart[kNbMax];
    __shared__ T wcoef[kNbMax];
    __shared__ T taus[kNbMax];  // block 0: tau_j, for T after the column loop
    // block 0: T(i, k), i <= k, at Tsh[i + k*nb] and G(i, k) = v_i . v_k, i < k, transposed
    // into the strictly lower part, at Tsh[k + i*nb]
    __shared__ T Tsh[kNbMax * kNbMax];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ T sh_tau, sh_beta, sh_scale;
    __shared__ int sh_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int r0 = p * R;
    const int nr = max(0, min(M, r0 + R) - r0);
    const int kmax = min(nb, M);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], nP);
        tc::mbar_init(&mbar[1], nP);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh_abort = 0;
    }
    if (p == 0) {
        for (int j = kmax + tid; j < nb; j += blockDim.x) tau[j] = T(0);
        for (int i = tid; i < nb * nb; i += blockDim.x) Tsh[i] = T(0);
    }
    // the block's rows into shared memory: every copy in flight at once (one memory latency)
    if (cs == 1) {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int c = idx % nb, rr = idx / nb;
            cp_async_4or8(&S[(size_t)c * R + rr], &P[(long)(r0 + rr) * rs + c]);
        }
    } else {
        for (int idx = tid; idx < nr * nb; idx += blockDim.x) {
            int rr = idx % nr, c = idx / nr;
            cp_async_4or8(&S[(size_t)c * R + rr], &P[(long)(r0 + rr) * rs + (long)c * cs]);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    cluster.sync();  // every block's barriers are initialised before the first remote arrive
    for (int j = 0; j < kmax; ++j) {
        const int buf = j & 1;
        const int ntr = nb - j;  // items 0 .. ntr-1: norm and trailing columns; ntr .. nb-1: G(i, j)
        const int rr_lo = max(0, j + 1 - r0);
        const T *xj = S + (size_t)j * R;
        for (int it = warp; it < nb; it += nwarps) {
            const int col = it < ntr ? j + it : it - ntr;
            const T d = warp_dot<T>(xj, S + (size_t)col * R, rr_lo, nr, lane);
            if (lane == 0) mypart[it] = d;
        }
        __syncthreads();
        // push this block's partials (and row j, by its owner) to every block of the cluster
        const int owner = j / R;
        for (int idx = tid; idx < nP * nb; idx += blockDim.x) {
            const int q = idx / nb, it = idx % nb;
            cluster.map_shared_rank(&inbox[buf][p][0], q)[it] = mypart[it];
            if (p == owner) {
                const int col = it < ntr ? j + it : it - ntr;
                cluster.map_shared_rank(&rowin[buf][0], q)[it] = S[(size_t)col * R + (j - r0)];
            }
        }
        __syncthreads();  // all of this block's pushes precede its arrivals
        if (tid < nP) mbar_arrive_remote(cluster_addr(&mbar[buf], tid));
        // warp 0: wait for every block's partials, sum them in a fixed order, form the
        // reflector, the coefficients w_c = tau v . a_c and (block 0) column j of T
        if (warp == 0) {
            if (lane == 0 && !sh_abort) {
                const uint32_t par = (uint32_t)((j >> 1) & 1);
                if (!mbar_try_wait_cluster(&mbar[buf], par)) {
                    const unsigned long long t0 = global_ns();
                    while (!mbar_try_wait_cluster(&mbar[buf], par)) {
                        if (global_ns() - t0 > kSpinBudgetNs) {
                            if (info) atomicExch(info, kInfoTimeout);
                            sh_abort = 1;
                            break;
                        }
                    }
                }
            }
            __syncwarp();  // lane 0's acquire orders the warp's reads below
            const int i0 = lane, i1 = lane + 32;  // nb <= kNbMax = 64
            T s0 = T(0), s1 = T(0), w0 = T(0), w1 = T(0);
#pragma unroll
            for (int q = 0; q < 16; ++q) {  // (the cluster size as a predicate: the loads issue together)
                if (q < nP && i0 < nb) s0 += inbox[buf][q][i0];
                if (q < nP && i1 < nb) s1 += inbox[buf][q][i1];
            }
            if (i0 < nb) w0 = rowin[buf][i0];
            if (i1 < nb) w1 = rowin[buf][i1];
            const T alpha = __shfl_sync(0xffffffffu, w0, 0), xn2 = __shfl_sync(0xffffffffu, s0, 0);
            T tj = T(0), beta = alpha, scale = T(0);
            if (xn2 > T(0)) {
                if constexpr (sizeof(T) == 4) {  // a few ulp, far inside the FP32 path's tolerance
                    const float q = alpha * alpha + xn2;
                    const float r = q * rsqrtf(q);
                    beta = alpha >= 0.f ? -r : r;
                    tj = __fdividef(beta - alpha, beta);
                    scale = __fdividef(1.f, alpha - beta);
                } else {
                    const T r = sqrt(alpha * alpha + xn2);
                    beta = alpha >= T(0) ? -r : r;
                    tj = (beta - alpha) / beta;
                    scale = T(1) / (alpha - beta);
                }
            }
            if (lane == 0) {
                sh_tau = tj;
                sh_beta = beta;
                sh_scale = scale;
                if (p == 0) {
                    tau[j] = tj;
                    taus[j] = tj;
                }
            }
            if (i0 >= 1 && i0 < ntr) wcoef[i0] = tj * (w0 + scale * s0);
            if (i1 < ntr) wcoef[i1] = tj * (w1 + scale * s1);
            if (p == 0) {  // G(i, j) = v_i . v_j = v_i[j] + x . v_i / (alpha - beta), i < j; T after the loop
                if (i0 >= ntr && i0 < nb) Tsh[j + (i0 - ntr) * nb] = w0 + scale * s0;
                if (i1 >= ntr && i1 < nb) Tsh[j + (i1 - ntr) * nb] = w1 + scale * s1;
            }
        }
        __syncthreads();
        const T tj = sh_tau, scT = sh_scale;
        if (tj != T(0)) {
            // columns in blocks of 16: the coefficients in registers, then independent updates
            // (all 16 entries of a row are loaded before any is stored back: the loads then
            // issue together instead of waiting on possibly aliasing stores)
            for (int cb = j + 1; cb < nb; cb += 16) {
                const int nc = min(16, nb - cb);
                T wr[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) wr[u] = u < nc ? wcoef[cb + u - j] : T(0);
                for (int rr = rr_lo + tid; rr < nr; rr += blockDim.x) {
                    T *row = S + (size_t)cb * R + rr;
                    const T v = S[(size_t)j * R + rr] * scT;
                    T xr[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) xr[u] = u < nc ? row[(size_t)u * R] : T(0);
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (u < nc) row[(size_t)u * R] = xr[u] - v * wr[u];
                }
            }
            for (int rr = rr_lo + tid; rr < nr; rr += blockDim.x) S[(size_t)j * R + rr] *= scT;
            if (p == owner) {
                for (int c = j + 1 + tid; c < nb; c += blockDim.x) S[(size_t)c * R + (j - r0)] -= wcoef[c - j];
                if (tid == 0) S[(size_t)j * R + (j - r0)] = sh_beta;
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
    if (p == 0) {
        // T(0:k, k) = -tau_k T(0:k, 0:k) G(0:k, k), T(k, k) = tau_k -- one warp, column by column
        if (warp == 0) {
            // lane i (and i + 32) forms T(i, kk) = -tau_kk sum_{i <= q < kk} T(i, q) G(q, kk); the
            // q loop is unrolled in blocks of 16 with the range as a predicate
            for (int kk = 0; kk < kmax; ++kk) {
                const T tk = taus[kk];
                for (int i = lane; i < kk; i += 32) {
                    T t = T(0);
                    for (int q0 = i & ~15; q0 < kk; q0 += 16) {
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int q = q0 + u;
                            const T tv = q < nb ? Tsh[i + q * nb] : T(0), gv = q < nb ? Tsh[kk + q * nb] : T(0);
                            t = (q >= i && q < kk) ? fma(tv, gv, t) : t;  // T(i, q) G(q, kk)
                        }
                    }
                    Tsh[i + kk * nb] = -tk * t;
                }
                if (lane == 0) Tsh[kk + kk * nb] = tk;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int idx = tid; idx < nb * nb; idx += blockDim.x) Tm[idx] = (idx % nb) <= (idx / nb) ? Tsh[idx] : T(0);
    }
    cluster.sync();  // no block leaves while another may still write to its shared memory
}

// ------------------------------------------------------------------ register-resident cluster variant
// The same factorisation with each thread holding its panel rows in registers
// (thread t of block p owns rows r0 + t + 512 q, q < RP; nb = NB fixed).  With
// column indices instead of item indices, the partial sums of column j are
//   x . a_c over rows below j, for every column c:
//   c == j: ||x||^2;  c > j: x . a_c (trailing);  c < j: x . v_c (finished reflector c),
// so one product per owned entry gives them all.  Per column: products and a warp
// reduce-scatter in registers, per-warp sums into shared memory, a block barrier;
// warp 0 adds the warps, pushes the block's sums (and row j, by its owner) to every
// block over DSMEM, arrives on their barriers, waits for its own, forms beta / tau
// and the coefficients; a block barrier; every thread updates its own rows.  Two
// block barriers per column and no shared-memory pass over the panel.

// Sum v[0..NB-1] over the warp's lanes, leaving the sum of column (NB == 32 ? lane
// : lane >> 1) in the return value: halving exchanges (upper lanes keep the upper half).
template <typename T, int NB>
NLA_DEV T warp_reduce_scatter(T (&v)[NB], int lane) {
#pragma unroll
    for (int h = NB / 2, o = 16; h >= 1; h /= 2, o /= 2) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    if (NB == 16) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

// Asynchronous store into another block's shared memory that completes as bytes on
// that block's mbarrier (release at cluster scope); addresses from cluster_addr.
NLA_DEV void st_async_remote(uint32_t addr, float v, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(addr), "f"(v),
                 "r"(mbar)
                 : "memory");
}
NLA_DEV void st_async_remote(uint32_t addr, double v, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(addr), "d"(v),
                 "r"(mbar)
                 : "memory");
}
// This block's arrival on its own barrier, announcing the bytes the phase waits for.
NLA_DEV void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

template <typename T, int NB>
NLA_DEV T select_col(const T (&a)[NB], int j) {
    T x = T(0);
#pragma unroll
    for (int c = 0; c < NB; ++c) x = c == j ? a[c] : x;
    return x;
}

template <typename T, int NB, int RP>
__global__ void __launch_bounds__(kClusterThreads, 1)
panel_reg_kernel(T *__restrict__ P, long rs, long cs, int M, int R, T *__restrict__ tau, T *__restrict__ Tm,
                 int *info) {
    pdl_wait();
    pdl_trigger();
    static_assert(NB == 16 || NB == 32, "NB");
    cg::cluster_group cluster = cg::this_cluster();
    const int p = (int)cluster.block_rank(), nP = (int)cluster.num_blocks();
    constexpr int kWarps = kClusterThreads / 32;
    __shared__ T red[kWarps][NB];   // per-warp column sums
    __shared__ T inbox[2][16][NB];  // by column parity and source block
    __shared__ T rowin[2][NB];
    __shared__ T myrow[NB];
    __shared__ T wcoef[NB];  // tau (v . a_c) for c > j, 0 otherwise
    __shared__ T taus[NB];
    // block 0: T(i, k), i <= k, at Tsh[i + k*NB]; G(i, k) = v_i . v_k, i < k, at Tsh[k + i*NB]
    __shared__ T Tsh[NB * NB];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ T sh_scale, sh_beta;
    __shared__ int sh_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = p * R;
    const int nr = max(0, min(M, r0 + R) - r0);
    const int kmax = min(NB, M);
    if (tid == 0) {
        // one arrival per phase (this block's expect_tx); the other blocks' partial sums
        // and the owner's row j complete it as transaction bytes
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh_abort = 0;
    }
    if (p == 0) {
        for (int j = kmax + tid; j < NB; j += blockDim.x) tau[j] = T(0);
        for (int i = tid; i < NB * NB; i += blockDim.x) Tsh[i] = T(0);
    }
    T a[RP][NB];
    // a row whose NB entries are contiguous and 16-byte aligned (the LQ panel: rs = ldx,
    // cs = 1) moves as 16-byte vectors
    const bool vec = cs == 1 && (rs * (long)sizeof(T)) % 16 == 0 && reinterpret_cast<uintptr_t>(P) % 16 == 0;
#pragma unroll
    for (int q = 0; q < RP; ++q) {
        const int rr = tid + kClusterThreads * q;
        if (vec && rr < nr) {
            if constexpr (sizeof(T) == 4) {
                const float4 *src = reinterpret_cast<const float4 *>(P + (long)(r0 + rr) * rs);
#pragma unroll
                for (int u = 0; u < NB / 4; ++u) {
                    const float4 f = src[u];
                    a[q][4 * u] = f.x, a[q][4 * u + 1] = f.y, a[q][4 * u + 2] = f.z, a[q][4 * u + 3] = f.w;
                }
            } else {
                const double2 *src = reinterpret_cast<const double2 *>(P + (long)(r0 + rr) * rs);
#pragma unroll
                for (int u = 0; u < NB / 2; ++u) {
                    const double2 f = src[u];
                    a[q][2 * u] = f.x, a[q][2 * u + 1] = f.y;
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < NB; ++c) a[q][c] = rr < nr ? P[(long)(r0 + rr) * rs + (long)c * cs] : T(0);
        }
    }
    cluster.sync();  // every block's barriers are initialised before the first remote arrive
    for (int j = 0; j < kmax; ++j) {
        const int buf = j & 1;
        T prod[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) prod[c] = T(0);
#pragma unroll
        for (int q = 0; q < RP; ++q) {
            const int rr = tid + kClusterThreads * q;
            const T x = (rr < nr && r0 + rr > j) ? select_col<T, NB>(a[q], j) : T(0);
#pragma unroll
            for (int c = 0; c < NB; ++c) prod[c] = fma(x, a[q][c], prod[c]);
        }
        const T wsum = warp_reduce_scatter<T, NB>(prod, lane);
        if (NB == 32 || (lane & 1) == 0) red[warp][NB == 32 ? lane : lane >> 1] = wsum;
        if (j >= r0 && j < r0 + nr) {  // the owner of row j publishes it
            const int rr = j - r0;
            if (tid == rr % kClusterThreads) {
#pragma unroll
                for (int q = 0; q < RP; ++q)
                    if (q == rr / kClusterThreads) {
#pragma unroll
                        for (int c = 0; c < NB; ++c) myrow[c] = a[q][c];
                    }
            }
        }
        __syncthreads();
        if (warp == 0) {
            const bool owner = j >= r0 && j < r0 + nr;
            if (lane == 0) mbar_arrive_expect_tx(&mbar[buf], (uint32_t)((nP + 1) * NB * sizeof(T)));
            // lane l pushes column c = l mod NB to blocks l / NB, l / NB + 32 / NB, ...
            const int c = lane % NB;
            T sblk = T(0);
#pragma unroll
            for (int w = 0; w < kWarps; ++w) sblk += red[w][c];
            const T rv = owner ? myrow[c] : T(0);
            for (int q = lane / NB; q < nP; q += 32 / NB) {
                const uint32_t mb = cluster_addr(&mbar[buf], q);
                st_async_remote(cluster_addr(&inbox[buf][p][c], q), sblk, mb);
                if (owner) st_async_remote(cluster_addr(&rowin[buf][c], q), rv, mb);
            }
            if (lane == 0 && !sh_abort) {
                const uint32_t par = (uint32_t)((j >> 1) & 1);
                if (!mbar_try_wait_cluster(&mbar[buf], par)) {
                    const unsigned long long t0 = global_ns();
                    while (!mbar_try_wait_cluster(&mbar[buf], par)) {
                        if (global_ns() - t0 > kSpinBudgetNs) {
                            if (info) atomicExch(info, kInfoTimeout);
                            sh_abort = 1;
                            break;
                        }
                    }
                }
            }
            __syncwarp();  // lane 0's acquire orders the warp's reads below
            T sc_ = T(0), wc_ = T(0);
            if (lane < NB) {
                // unrolled over the largest cluster with the size as a predicate: the loads
                // issue together instead of one load-to-add latency per block
#pragma unroll
                for (int q = 0; q < 16; ++q) sc_ += q < nP ? inbox[buf][q][lane] : T(0);
                wc_ = rowin[buf][lane];
            }
            const T alpha = __shfl_sync(0xffffffffu, wc_, j), xn2 = __shfl_sync(0xffffffffu, sc_, j);
            T tj = T(0), beta = alpha, scale = T(0);
            if (xn2 > T(0)) {
                if constexpr (sizeof(T) == 4) {  // a few ulp, far inside the FP32 path's tolerance
                    const float q = alpha * alpha + xn2;
                    const float r = q * rsqrtf(q);
                    beta = alpha >= 0.f ? -r : r;
                    tj = __fdividef(beta - alpha, beta);
                    scale = __fdividef(1.f, alpha - beta);
                } else {
                    const T r = sqrt(alpha * alpha + xn2);
                    beta = alpha >= T(0) ? -r : r;
                    tj = (beta - alpha) / beta;
                    scale = T(1) / (alpha - beta);
                }
            }
            if (lane < NB) {
                const T vdot = wc_ + scale * sc_;  // v . a_c (c > j) or G(c, j) = v_c . v_j (c < j)
                wcoef[lane] = lane > j ? tj * vdot : T(0);
                if (p == 0 && lane < j) Tsh[j + lane * NB] = vdot;
            }
            if (lane == 0) {
                sh_scale = scale;
                sh_beta = beta;
                taus[j] = tj;
                if (p == 0) tau[j] = tj;
            }
        }
        __syncthreads();
        const T tj = taus[j];
        if (tj != T(0)) {
            const T scl = sh_scale, bt = sh_beta;
            T w[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) w[c] = wcoef[c];
#pragma unroll
            for (int q = 0; q < RP; ++q) {
                const int rr = tid + kClusterThreads * q, gr = r0 + rr;
                if (rr < nr && gr >= j) {
                    // rows below j: a_c -= v w_c with v = x / (alpha - beta), and v into column j;
                    // row j: a_c -= w_c (v_j = 1), beta into column j
                    const T v = gr > j ? select_col<T, NB>(a[q], j) * scl : T(1);
#pragma unroll
                    for (int c = 0; c < NB; ++c) a[q][c] = c == j ? (gr > j ? v : bt) : fma(-v, w[c], a[q][c]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RP; ++q) {
        const int rr = tid + kClusterThreads * q;
        if (rr < nr) {
            if (vec) {
                if constexpr (sizeof(T) == 4) {
                    float4 *dst = reinterpret_cast<float4 *>(P + (long)(r0 + rr) * rs);
#pragma unroll
                    for (int u = 0; u < NB / 4; ++u)
                        dst[u] = make_float4(a[q][4 * u], a[q][4 * u + 1], a[q][4 * u + 2], a[q][4 * u + 3]);
                } else {
                    double2 *dst = reinterpret_cast<double2 *>(P + (long)(r0 + rr) * rs);
#pragma unroll
                    for (int u = 0; u < NB / 2; ++u) dst[u] = make_double2(a[q][2 * u], a[q][2 * u + 1]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < NB; ++c) P[(long)(r0 + rr) * rs + (long)c * cs] = a[q][c];
            }
        }
    }
    if (p == 0) {
        __syncthreads();
        // T(0:k, k) = -tau_k T(0:k, 0:k) G(0:k, k), T(k, k) = tau_k -- one warp, column by column
        if (warp == 0) {
            // lane i forms T(i, kk) = -tau_kk sum_{i <= q < kk} T(i, q) G(q, kk); the q loop is
            // unrolled over the whole width with the range as a predicate, so its loads issue at once
            for (int kk = 0; kk < kmax; ++kk) {
                const T tk = taus[kk];
                if (lane < kk) {
                    T t = T(0);
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        const T tv = Tsh[lane + q * NB], gv = Tsh[kk + q * NB];  // T(i, q), G(q, kk)
                        t = (q >= lane && q < kk) ? fma(tv, gv, t) : t;
                    }
                    Tsh[lane + kk * NB] = -tk * t;
                }
                if (lane == 0) Tsh[kk + kk * NB] = tk;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int idx = tid; idx < NB * NB; idx += blockDim.x) Tm[idx] = (idx % NB) <= (idx / NB) ? Tsh[idx] : T(0);
    }
    cluster.sync();  // no block leaves while another may still write to its shared memory
}

// Cluster size and rows per block for an M x nb panel, or 0 if it does not fit one cluster.
// Which cluster sizes the device can schedule (one block per SM at the largest
// dynamic shared memory) is asked once; smaller allocations schedule as well.
struct ClusterCaps {
    size_t max_dyn = 0;
    bool sched[5] = {false, false, false, false, false};  // cluster sizes 1, 2, 4, 8, 16
};

template <typename T>
static int cluster_plan(int M, int nb, int &R, size_t &dyn) {
    static PerDeviceValue<ClusterCaps> caps_dev;
    const ClusterCaps caps = caps_dev.get([] {
        ClusterCaps c;
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, std::max(current_device(), 0));
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, panel_cluster_kernel<T>) == cudaSuccess && (size_t)optin > fa.sharedSizeBytes)
            c.max_dyn = (size_t)optin - fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.max_dyn) !=
                cudaSuccess ||
            cudaFuncSetAttribute(panel_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess)
            c.max_dyn = 0;
        for (int k = 0; k < 5 && c.max_dyn > 0; ++k) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(1u << k);
            cfg.blockDim = dim3(kClusterThreads);
            cfg.dynamicSmemBytes = c.max_dyn;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 1u << k;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int ncl = 0;
            c.sched[k] = cudaOccupancyMaxActiveClusters(&ncl, panel_cluster_kernel<T>, &cfg) == cudaSuccess && ncl >= 1;
        }
        cudaGetLastError();
        return c;
    });
    const size_t max_dyn = caps.max_dyn;
    const bool *sched = caps.sched;
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
        const size_t d = (size_t)r * nb * sizeof(T);
        if (d > max_dyn) continue;
        best = C;
        R = r;
        dyn = d;
        if (k >= k0) break;  // the smallest fitting size at or above the target, else the largest that fits
    }
    return best;
}

// Register-resident cluster panel for the shapes it is built for (nb 16 or 32, one
// row per thread: at most 512 rows per block); cudaErrorNotSupported otherwise.
// NLA_PANEL_REG=0 keeps the shared-memory variant.
template <typename T, int NB, int RP>
cudaError_t panel_reg_launch_nb(T *P, long rs, long cs, int M, int R, int C, T *tau, T *Tm, int *info,
                                cudaStream_t st) {
    static PerDeviceOnce attr;
    attr.run([] {
        cudaFuncSetAttribute(panel_reg_kernel<T, NB, RP>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaGetLastError();
    });
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, panel_reg_kernel<T, NB, RP>, P, rs, cs, M, R, tau, Tm, info);
}

template <typename T>
cudaError_t panel_reg_launch(T *P, long rs, long cs, int M, int nb, int R, int C, T *tau, T *Tm, int *info,
                             cudaStream_t st) {
    static const bool on = [] {
        const char *v = getenv("NLA_PANEL_REG");
        return !v || atoi(v) != 0;
    }();
    if (!on || C > 16) return cudaErrorNotSupported;
    const int rp = (R + kClusterThreads - 1) / kClusterThreads;
    if constexpr (sizeof(T) == 4) {
        // (two or more rows per thread spill at the 128-register limit of 512 threads)
        if (nb == 16 && rp == 1) return panel_reg_launch_nb<T, 16, 1>(P, rs, cs, M, R, C, tau, Tm, info, st);
        if (nb == 32 && rp == 1) return panel_reg_launch_nb<T, 32, 1>(P, rs, cs, M, R, C, tau, Tm, info, st);
    } else {
        if (nb == 16 && rp == 1) return panel_reg_launch_nb<T, 16, 1>(P, rs, cs, M, R, C, tau, Tm, info, st);
    }
    return cudaErrorNotSupported;
}

template <typename T>
cudaError_t panel_factor(T *P, long rs, long cs, int M, int nb, T *tau, T *Tm, const PanelCtl &ctl,
                         cudaStream_t st) {
    if (M <= 0 || nb <= 0) return cudaSuccess;
    if (nb > kNbMax) return cudaErrorInvalidValue;
    {  // preferred: one thread-block cluster, no global barrier
        int R = 0;
        size_t dyn = 0;
        const int C = cluster_plan<T>(M, nb, R, dyn);
        if (C > 0) {
            // rows in registers: one row per thread, so the smallest cluster with at
            // most 512 rows per block (fewer blocks, fewer exchanges per column)
            int Cr = 1;
            while (Cr < 16 && (long)Cr * kClusterThreads < M) Cr *= 2;
            const int Rr = (M + Cr - 1) / Cr;
            cudaError_t e = Rr <= kClusterThreads ? panel_reg_launch<T>(P, rs, cs, M, nb, Rr, Cr, tau, Tm, ctl.info, st)
                                                  : cudaErrorNotSupported;
            if (e == cudaSuccess) return e;
            cudaGetLastError();  // not available for this shape: shared-memory variant
        }
        if (C > 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(kClusterThreads);
            cfg.dynamicSmemBytes = dyn;
            cfg.stream = st;
            cudaLaunchAttribute attr[2];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[1].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = pdl_enabled() ? 2 : 1;
            cudaError_t e = cudaLaunchKernelEx(&cfg, panel_cluster_kernel<T>, P, rs, cs, M, nb, R, tau, Tm, ctl.info);
            if (e == cudaSuccess) return e;
            cudaGetLastError();  // fall back to the grid-wide version
        }
    }
    static PerDeviceValue<size_t> grid_dyn;
    const size_t max_dyn = grid_dyn.get([] {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, std::max(current_device(), 0));
        cudaFuncAttributes fa;
        size_t md = 0;
        if (cudaFuncGetAttributes(&fa, panel_kernel<T>) == cudaSuccess)
            md = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)md);
        cudaGetLastError();
        return md;
    });
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
