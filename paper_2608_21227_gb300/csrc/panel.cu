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
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace nla {

constexpr int kPanelThreads = 256;
constexpr int kNbMax = 64;
constexpr int kPanelRowsTarget = 128;  // rows per block when the panel is long enough

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
    __shared__ double wcoef[kNbMax + 1];
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
                double s = 0.0;
                for (int rr = rr_lo + lane; rr < nr; rr += 32) {
                    double x = (double)xj[rr];
                    s += x * x;
                }
                s = warp_sum(s);
                if (lane == 0) cp[0] = s;
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
            if (!spin_until_geq(bar, (unsigned)(j + 1) * (unsigned)nP, info)) sh_fail = 1;
            __threadfence();
        }
        __syncthreads();
        if (sh_fail) return;

        // fixed-order sum of the partials: deterministic across runs
        for (int it = tid; it < nitem; it += blockDim.x) {
            double s = 0.0;
            for (int q = 0; q < nP; ++q) s += ld_cg(colpart + ((size_t)buf * nP + q) * (kNbMax + 1) + it);
            red[it] = s;
            rowv[it] = ld_cg(rowbuf + buf * kNbMax + it);
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
        for (int it = 1 + tid; it < nitem; it += blockDim.x) wcoef[it] = tj * (rowv[it] + sc * red[it]);
        __syncthreads();
        if (tj != 0.0) {
            const T scT = (T)sc;
            for (int rr = rr_lo + tid; rr < nr; rr += blockDim.x) {
                T v = S[(size_t)j * R + rr] * scT;  // reflector entry v_r
                for (int c = j + 1; c < nb; ++c) S[(size_t)c * R + rr] -= v * (T)wcoef[c - j];
                S[(size_t)j * R + rr] = v;
            }
            if (j >= r0 && j < r0 + nr) {  // row j itself: v_j = 1
                for (int c = j + 1 + tid; c < nb; c += blockDim.x) S[(size_t)c * R + (j - r0)] -= (T)wcoef[c - j];
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
        double s = 0.0;
        for (int rr = lane; rr < nr; rr += 32) {
            int r = r0 + rr;
            if (r < k) continue;
            double vk = (r == k) ? 1.0 : (double)S[(size_t)k * R + rr];
            double vi = (double)S[(size_t)i * R + rr];  // r >= k > i: stored tail
            s += vi * vk;
        }
        s = warp_sum(s);
        if (lane == 0) gp[i * kNbMax + k] = s;
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

template <typename T>
cudaError_t panel_factor(T *P, long rs, long cs, int M, int nb, T *tau, T *Tm, const PanelCtl &ctl,
                         cudaStream_t st) {
    if (M <= 0 || nb <= 0) return cudaSuccess;
    if (nb > kNbMax) return cudaErrorInvalidValue;
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
