// update.cu -- blocked trailing-matrix update (the UNMQR/TSMQR step of
// Algorithm 1, whose GPU kernel is Algorithm 2), FP64 and FP32 SIMT paths.
//
// QR side:  X <- (I - V T V^T)^T X = X - V (T^T (V^T X))      (X below/right of a tile column)
// LQ side:  X <- X (I - V T V^T)   = X - ((X V) T) V^T        (X below a tile row)
//
// As in Algorithm 2, one block owns a strip of the trailing matrix -- 32*cpb
// columns on the QR side, 32*cpb rows on the LQ side -- over its whole extent,
// so the reflector block is applied in three steps without a grid-wide
// reduction: (1) W = V^T X_strip accumulated over tiles of `tile` rows staged
// through shared memory (Algorithm 2's reflector dot products, here all nb at
// once), (2) W <- T^T W with the compact-WY factor, (3) X_strip -= V W, tile by
// tile.  V is unit lower trapezoidal: its implicit unit diagonal and zero upper
// part are substituted while staging, so the panel's stored R is never read
// as reflector data.  Accumulation is in the matrix type.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace nla {

constexpr int kMaxItems = 32;     // W entries held in registers per thread
constexpr size_t kSmemLimit = 226 * 1024;

static size_t left_smem(int elem, int nb, int th, int w) {
    return (size_t)elem * ((size_t)th * (nb + 1) + (size_t)th * (w + 1) + (size_t)nb * w);
}
static size_t right_smem(int elem, int nb, int th, int h) {
    return (size_t)elem * ((size_t)th * h + (size_t)th * nb + (size_t)nb * h);
}

// Generic kernels (below): any band width 1..64; W entries strided over the block.
static bool generic_cfg_valid(int side, int elem, int nb, const UpdCfg &c, size_t *smem_bytes) {
    if (nb < 1 || nb > 64) return false;
    if (c.threads < 32 || c.threads > 1024 || c.threads % 32) return false;
    if (c.cpb < 1 || c.cpb > 8 || c.tile < 1 || c.tile > 256) return false;
    if (c.unroll != 1 && c.unroll != 2 && c.unroll != 4) return false;
    const int w = 32 * c.cpb;
    const long items = (long)nb * w;
    if (items % c.threads) return false;  // every thread owns the same number of W entries
    const long per = items / c.threads;
    if (per < 1 || per > kMaxItems) return false;
    if ((long)c.tile * w < c.threads) return false;  // phase-3 tile must cover the block
    size_t sm = side == 0 ? left_smem(elem, nb, c.tile, w) : right_smem(elem, nb, c.tile, w);
    if (sm > kSmemLimit) return false;
    if (smem_bytes) *smem_bytes = sm;
    return true;
}

// Band widths divisible by 4 use the register-tiled kernels (update_tiled.cu);
// others the generic kernels here.
// FP32 at band widths 16, 32, 64 runs the TMA-streamed kernels; everything
// else the register-tiled (nb % 4 == 0) or generic SIMT kernels.
bool tma_band(int elem, int nb) { return elem == 4 && (nb == 16 || nb == 32 || nb == 64); }

bool upd_cfg_valid(int side, int elem, int nb, const UpdCfg &c, size_t *smem_bytes) {
    if (tma_band(elem, nb)) {
        if (!tma_cfg_valid(nb, c)) return false;
        if (smem_bytes) *smem_bytes = tma_cfg_smem(nb, c);
        return true;
    }
    if (nb % 4 == 0) {
        if (!tiled_r(nb, c)) return false;
        size_t sm = tiled_smem(side, elem, nb, c.tile, 32 * c.cpb);
        if (sm > kSmemLimit) return false;
        if (smem_bytes) *smem_bytes = sm;
        return true;
    }
    return generic_cfg_valid(side, elem, nb, c, smem_bytes);
}

// -------------------------------------------------------------------- QR side
template <typename T, int U>
__global__ void trail_left_kernel(T *__restrict__ X, long ldx, int M, int N, const T *__restrict__ V,
                                  long ldv, int nb, const T *__restrict__ Tm, int th, int w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldvs = nb + 1, ldxs = w + 1;
    T *Vs = reinterpret_cast<T *>(smem_raw);  // th x nb  (row r at Vs + r*ldvs)
    T *Xs = Vs + (size_t)th * ldvs;          // th x w   (row r at Xs + r*ldxs)
    T *Ws = Xs + (size_t)th * ldxs;          // nb x w   (row k at Ws + k*w)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int c0 = blockIdx.x * w;
    const int wc = min(w, N - c0);
    const int items = nb * w / nt;

    T acc[kMaxItems];
#pragma unroll
    for (int i = 0; i < kMaxItems; ++i) acc[i] = T(0);

    // (1) W = V^T X_strip
    for (int r0 = 0; r0 < M; r0 += th) {
        const int rows = min(th, M - r0);
        for (int idx = tid; idx < th * nb; idx += nt) {
            int r = idx % th, k = idx / th, gr = r0 + r;
            T v = T(0);
            if (r < rows) v = gr > k ? V[gr + (long)k * ldv] : (gr == k ? T(1) : T(0));
            Vs[r * ldvs + k] = v;
        }
        for (int idx = tid; idx < th * w; idx += nt) {
            int r = idx % th, c = idx / th;
            Xs[r * ldxs + c] = (r < rows && c < wc) ? X[(r0 + r) + (long)(c0 + c) * ldx] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kMaxItems; ++i) {
            if (i < items) {
                const int it = tid + i * nt, k = it / w, c = it % w;
                T s = acc[i];
#pragma unroll U
                for (int r = 0; r < rows; ++r) s += Vs[r * ldvs + k] * Xs[r * ldxs + c];
                acc[i] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < kMaxItems; ++i)
        if (i < items) {
            const int it = tid + i * nt;
            Ws[it] = acc[i];  // it = k*w + c
        }
    __syncthreads();
    // (2) W <- T^T W : W'(i, c) = sum_{k <= i} T(k, i) W(k, c)
#pragma unroll
    for (int i = 0; i < kMaxItems; ++i)
        if (i < items) {
            const int it = tid + i * nt, ii = it / w, c = it % w;
            T s = T(0);
            for (int k = 0; k <= ii; ++k) s += Tm[k + (long)ii * nb] * Ws[k * w + c];
            acc[i] = s;
        }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kMaxItems; ++i)
        if (i < items) Ws[tid + i * nt] = acc[i];
    __syncthreads();
    // (3) X_strip -= V W'
    for (int r0 = 0; r0 < M; r0 += th) {
        const int rows = min(th, M - r0);
        for (int idx = tid; idx < th * nb; idx += nt) {
            int r = idx % th, k = idx / th, gr = r0 + r;
            T v = T(0);
            if (r < rows) v = gr > k ? V[gr + (long)k * ldv] : (gr == k ? T(1) : T(0));
            Vs[r * ldvs + k] = v;
        }
        __syncthreads();
        for (int idx = tid; idx < th * w; idx += nt) {
            int r = idx % th, c = idx / th;
            if (r < rows && c < wc) {
                T s = T(0);
#pragma unroll 4
                for (int k = 0; k < nb; ++k) s += Vs[r * ldvs + k] * Ws[k * w + c];
                T *px = X + (r0 + r) + (long)(c0 + c) * ldx;
                *px = *px - s;
            }
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------- LQ side
template <typename T, int U>
__global__ void trail_right_kernel(T *__restrict__ X, long ldx, int M, int N, const T *__restrict__ Vt,
                                   long ldvt, int nb, const T *__restrict__ Tm, int th, int h) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);  // th cols x h rows (col c at Xs + c*h)
    T *Vs = Xs + (size_t)th * h;             // th x nb (row c at Vs + c*nb)
    T *Ys = Vs + (size_t)th * nb;            // nb x h  (col k at Ys + k*h)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int i0 = blockIdx.x * h;
    const int hr = min(h, M - i0);
    const int items = nb * h / nt;

    T acc[kMaxItems];
#pragma unroll
    for (int i = 0; i < kMaxItems; ++i) acc[i] = T(0);

    // (1) Y = X_strip V
    for (int cb = 0; cb < N; cb += th) {
        const int cols = min(th, N - cb);
        for (int idx = tid; idx < th * h; idx += nt) {
            int i = idx % h, c = idx / h;
            Xs[c * h + i] = (i < hr && c < cols) ? X[(i0 + i) + (long)(cb + c) * ldx] : T(0);
        }
        for (int idx = tid; idx < th * nb; idx += nt) {
            int k = idx % nb, c = idx / nb, gc = cb + c;
            T v = T(0);
            if (c < cols) v = gc > k ? Vt[k + (long)gc * ldvt] : (gc == k ? T(1) : T(0));
            Vs[c * nb + k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
            if (q < items) {
                const int it = tid + q * nt, i = it % h, k = it / h;
                T s = acc[q];
#pragma unroll U
                for (int c = 0; c < cols; ++c) s += Xs[c * h + i] * Vs[c * nb + k];
                acc[q] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q)
        if (q < items) Ys[tid + q * nt] = acc[q];  // it = k*h + i
    __syncthreads();
    // (2) Y <- Y T : Y'(i, k) = sum_{j <= k} Y(i, j) T(j, k)
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q)
        if (q < items) {
            const int it = tid + q * nt, i = it % h, k = it / h;
            T s = T(0);
            for (int j = 0; j <= k; ++j) s += Ys[j * h + i] * Tm[j + (long)k * nb];
            acc[q] = s;
        }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q)
        if (q < items) Ys[tid + q * nt] = acc[q];
    __syncthreads();
    // (3) X_strip -= Y' V^T
    for (int cb = 0; cb < N; cb += th) {
        const int cols = min(th, N - cb);
        for (int idx = tid; idx < th * nb; idx += nt) {
            int k = idx % nb, c = idx / nb, gc = cb + c;
            T v = T(0);
            if (c < cols) v = gc > k ? Vt[k + (long)gc * ldvt] : (gc == k ? T(1) : T(0));
            Vs[c * nb + k] = v;
        }
        __syncthreads();
        for (int idx = tid; idx < th * h; idx += nt) {
            int i = idx % h, c = idx / h;
            if (i < hr && c < cols) {
                T s = T(0);
#pragma unroll 4
                for (int k = 0; k < nb; ++k) s += Ys[k * h + i] * Vs[c * nb + k];
                T *px = X + (i0 + i) + (long)(cb + c) * ldx;
                *px = *px - s;
            }
        }
        __syncthreads();
    }
}

template <typename T, int U>
static cudaError_t launch_left(T *X, long ldx, int M, int N, const T *V, long ldv, int nb, const T *Tm,
                               const UpdCfg &c, size_t smem, cudaStream_t st) {
    static PerDeviceOnce attr;
    attr.run([] {
        cudaFuncSetAttribute(trail_left_kernel<T, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
        cudaGetLastError();
    });
    const int w = 32 * c.cpb;
    dim3 grid((N + w - 1) / w);
    trail_left_kernel<T, U><<<grid, c.threads, smem, st>>>(X, ldx, M, N, V, ldv, nb, Tm, c.tile, w);
    return cudaGetLastError();
}

template <typename T, int U>
static cudaError_t launch_right(T *X, long ldx, int M, int N, const T *Vt, long ldvt, int nb,
                                const T *Tm, const UpdCfg &c, size_t smem, cudaStream_t st) {
    static PerDeviceOnce attr;
    attr.run([] {
        cudaFuncSetAttribute(trail_right_kernel<T, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
        cudaGetLastError();
    });
    const int h = 32 * c.cpb;
    dim3 grid((M + h - 1) / h);
    trail_right_kernel<T, U><<<grid, c.threads, smem, st>>>(X, ldx, M, N, Vt, ldvt, nb, Tm, c.tile, h);
    return cudaGetLastError();
}

// Largest block the compiled kernel can launch (its register use bounds it); -1 when
// it cannot be asked (no CUDA device in this process): the launch itself then decides.
template <typename K>
static int max_threads_of(K kernel) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return fa.maxThreadsPerBlock;
}

template <typename T>
static int max_threads(int side, int unroll) {
    static std::mutex mu;  // (thread limits are per architecture, not per device)
    static int cache[2][3] = {{-1, -1, -1}, {-1, -1, -1}};
    std::lock_guard<std::mutex> lk(mu);
    int u = unroll == 1 ? 0 : unroll == 2 ? 1 : 2;
    int &v = cache[side][u];
    if (v < 0) {
        int q;
        if (side == 0)
            q = u == 0 ? max_threads_of(trail_left_kernel<T, 1>)
                       : u == 1 ? max_threads_of(trail_left_kernel<T, 2>) : max_threads_of(trail_left_kernel<T, 4>);
        else
            q = u == 0 ? max_threads_of(trail_right_kernel<T, 1>)
                       : u == 1 ? max_threads_of(trail_right_kernel<T, 2>) : max_threads_of(trail_right_kernel<T, 4>);
        if (q < 0) return 1024;  // unknown (not cached)
        v = q;
    }
    return v;
}

bool upd_cfg_launchable(int side, int elem, int nb, const UpdCfg &c) {
    size_t sm;
    if (!upd_cfg_valid(side, elem, nb, c, &sm)) return false;
    if (tma_band(elem, nb)) return true;  // <= 288 threads, within the kernels' launch bounds
    if (nb % 4 == 0) return c.threads <= tiled_max_threads(side, elem, tiled_r(nb, c), c.unroll);
    int mt = elem == 8 ? max_threads<double>(side, c.unroll) : max_threads<float>(side, c.unroll);
    return c.threads <= mt;
}

// A launchable register-tiled configuration (nb % 4 == 0) for FP32 calls whose
// buffers do not meet the TMA alignment rules.
static UpdCfg tiled_for(int side, int elem, int nb, const UpdCfg &c) {
    if (tiled_r(nb, c) && tiled_smem(side, elem, nb, c.tile, 32 * c.cpb) <= kSmemLimit &&
        c.threads <= tiled_max_threads(side, elem, tiled_r(nb, c), c.unroll))
        return c;
    const int tiles[] = {64, 32, 128, 16};
    for (int cpb : {2, 1, 4})
        for (int threads = 128; threads <= 512; threads += 64)
            for (int tile : tiles) {
                const UpdCfg t{tile, threads, cpb, 1};
                if (tiled_r(nb, t) && tiled_smem(side, elem, nb, tile, 32 * cpb) <= kSmemLimit &&
                    threads <= tiled_max_threads(side, elem, tiled_r(nb, t), 1))
                    return t;
            }
    return c;
}

template <typename T>
cudaError_t trail_left(T *X, long ldx, int M, int N, const T *Vp, long ldv, int nb, const T *Tm,
                       const UpdCfg &c, const UpdScratch &sc, cudaStream_t st) {
    if (M <= 0 || N <= 0 || nb <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if (tma_band(4, nb)) {
            if (!tma_cfg_valid(nb, c)) return cudaErrorInvalidConfiguration;
            if (trail_tma_eligible(X, ldx, Vp, ldv, nb, sc)) return trail_tma(0, X, ldx, M, N, Vp, ldv, nb, Tm, c, sc, st);
            return trail_tiled<T>(0, X, ldx, M, N, Vp, ldv, nb, Tm, tiled_for(0, 4, nb, c), sc, st);
        }
    }
    if (nb % 4 == 0) {
        if (!upd_cfg_launchable(0, (int)sizeof(T), nb, c)) return cudaErrorInvalidConfiguration;
        return trail_tiled<T>(0, X, ldx, M, N, Vp, ldv, nb, Tm, c, sc, st);
    }
    size_t smem = 0;
    if (!generic_cfg_valid(0, (int)sizeof(T), nb, c, &smem)) return cudaErrorInvalidConfiguration;
    if (c.threads > max_threads<T>(0, c.unroll)) return cudaErrorInvalidConfiguration;
    switch (c.unroll) {
        case 1: return launch_left<T, 1>(X, ldx, M, N, Vp, ldv, nb, Tm, c, smem, st);
        case 2: return launch_left<T, 2>(X, ldx, M, N, Vp, ldv, nb, Tm, c, smem, st);
        default: return launch_left<T, 4>(X, ldx, M, N, Vp, ldv, nb, Tm, c, smem, st);
    }
}

template <typename T>
cudaError_t trail_right(T *X, long ldx, int M, int N, const T *Vt, long ldvt, int nb, const T *Tm,
                        const UpdCfg &c, const UpdScratch &sc, cudaStream_t st) {
    if (M <= 0 || N <= 0 || nb <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if (tma_band(4, nb)) {
            if (!tma_cfg_valid(nb, c)) return cudaErrorInvalidConfiguration;
            if (trail_tma_eligible(X, ldx, Vt, ldvt, nb, sc))
                return trail_tma(1, X, ldx, M, N, Vt, ldvt, nb, Tm, c, sc, st);
            return trail_tiled<T>(1, X, ldx, M, N, Vt, ldvt, nb, Tm, tiled_for(1, 4, nb, c), sc, st);
        }
    }
    if (nb % 4 == 0) {
        if (!upd_cfg_launchable(1, (int)sizeof(T), nb, c)) return cudaErrorInvalidConfiguration;
        return trail_tiled<T>(1, X, ldx, M, N, Vt, ldvt, nb, Tm, c, sc, st);
    }
    size_t smem = 0;
    if (!generic_cfg_valid(1, (int)sizeof(T), nb, c, &smem)) return cudaErrorInvalidConfiguration;
    if (c.threads > max_threads<T>(1, c.unroll)) return cudaErrorInvalidConfiguration;
    switch (c.unroll) {
        case 1: return launch_right<T, 1>(X, ldx, M, N, Vt, ldvt, nb, Tm, c, smem, st);
        case 2: return launch_right<T, 2>(X, ldx, M, N, Vt, ldvt, nb, Tm, c, smem, st);
        default: return launch_right<T, 4>(X, ldx, M, N, Vt, ldvt, nb, Tm, c, smem, st);
    }
}

template cudaError_t trail_left<double>(double *, long, int, int, const double *, long, int,
                                        const double *, const UpdCfg &, const UpdScratch &, cudaStream_t);
template cudaError_t trail_left<float>(float *, long, int, int, const float *, long, int, const float *,
                                       const UpdCfg &, const UpdScratch &, cudaStream_t);
template cudaError_t trail_right<double>(double *, long, int, int, const double *, long, int,
                                         const double *, const UpdCfg &, const UpdScratch &, cudaStream_t);
template cudaError_t trail_right<float>(float *, long, int, int, const float *, long, int,
                                        const float *, const UpdCfg &, const UpdScratch &, cudaStream_t);

}  // namespace nla
