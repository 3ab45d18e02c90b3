// update_tiled.cu -- register-tiled trailing update (Algorithm 2, both sides),
// the main FP64 / FP32 SIMT path.  Same three steps as update.cu
// (W = V^T X_strip, W <- T^T W, X_strip -= V W'), with the work of each step
// tiled for the FMA pipes:
//
//   threads = (w/4 column groups) x (nb/R reflector groups); thread (cg, rg)
//   owns 4 strip columns (QR side) / 4 strip rows (LQ side) and R reflectors.
//   Step 1: for every staged row (column) of X the thread does R x 4 FMAs from
//           one 128-bit shared load of X and R reflector values that the whole
//           warp shares (broadcast).
//   Step 3: the thread updates sub-blocks of 4 x 4 entries of the staged X
//           tile; per reflector one 128-bit load of W' and one broadcast
//           128-bit load of V (stored k-major) feed 16 FMAs.
//
// QR side: X tiles are staged row-major with an XOR swizzle of the 4-column
// group by (row & 7), so that both the column-wise staging stores and the
// row-wise 128-bit reads are free of bank conflicts.  LQ side: X tiles are
// staged column-major (the strip rows are contiguous), which needs no swizzle.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace nla {

constexpr size_t kTiledSmemLimit = 227 * 1024;

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    NLA_DEV static void ld(const float *p, float v[4]) {
        float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    }
    NLA_DEV static void st(float *p, const float v[4]) { *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]); }
};
template <>
struct Vec4<double> {
    NLA_DEV static void ld(const double *p, double v[4]) {
        double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
    NLA_DEV static void st(double *p, const double v[4]) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
};

// Swizzled position of X(r, c) in a row-major tile with w columns.
NLA_DEV int swz(int r, int c, int w) { return r * w + ((((c >> 2) ^ (r & 7))) << 2) + (c & 3); }

size_t tiled_smem(int side, int elem, int nb, int th, int w) {
    (void)side;
    return (size_t)elem * ((size_t)th * w + (size_t)th * (nb + 4) + (size_t)nb * w);
}

// R = reflectors per thread, or 0 if (nb, threads, cpb, tile, unroll) do not tile.
int tiled_r(int nb, const UpdCfg &c) {
    if (nb < 4 || nb > 64 || nb % 4) return 0;
    if (c.threads < 32 || c.threads > 1024 || c.threads % 32) return 0;
    if (c.cpb != 1 && c.cpb != 2 && c.cpb != 4 && c.cpb != 8) return 0;  // swizzle needs 2^k column groups
    if (c.unroll != 1 && c.unroll != 2 && c.unroll != 4) return 0;
    const int w = 32 * c.cpb, ncg = w / 4;
    if (c.threads % ncg) return 0;
    const int nrg = c.threads / ncg;
    if (nb % nrg) return 0;
    const int R = nb / nrg;
    if (R != 1 && R != 2 && R != 4 && R != 8) return 0;
    if (c.tile < 4 || c.tile > 256 || c.tile % (4 * nrg)) return 0;  // step-3 rows per thread: multiple of 4
    return R;
}

// -------------------------------------------------------------------- QR side
template <typename T, int R, int U>
__global__ void trail_left_tiled(T *__restrict__ X, long ldx, int M, int N, const T *__restrict__ V, long ldv, int nb,
                 const T *__restrict__ Tm, int th, int w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldv_s = nb + 4;
    T *Xs = reinterpret_cast<T *>(smem_raw);  // th x w, swizzled
    T *Vs = Xs + (size_t)th * w;             // step 1: th x (nb+4) row-major; step 3: nb x th (k-major)
    T *Ws = Vs + (size_t)th * ldv_s;         // nb x w row-major
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ncg = w >> 2, cg = tid % ncg, rg = tid / ncg, nrg = nt / ncg;
    const int c0 = blockIdx.x * w, wc = min(w, N - c0);

    T acc[R][4];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    // ---- step 1: W = V^T X_strip
    for (int r0 = 0; r0 < M; r0 += th) {
        const int rows = min(th, M - r0);
        for (int idx = tid; idx < th * w; idx += nt) {
            int r = idx % th, c = idx / th;
            Xs[swz(r, c, w)] = (r < rows && c < wc) ? X[(r0 + r) + (long)(c0 + c) * ldx] : T(0);
        }
        for (int idx = tid; idx < th * nb; idx += nt) {
            int r = idx % th, k = idx / th, gr = r0 + r;
            T v = T(0);
            if (r < rows) v = gr > k ? V[gr + (long)k * ldv] : (gr == k ? T(1) : T(0));
            Vs[r * ldv_s + k] = v;
        }
        __syncthreads();
#pragma unroll U
        for (int r = 0; r < rows; ++r) {
            T x[4];
            Vec4<T>::ld(Xs + swz(r, 4 * cg, w), x);
            const T *vr = Vs + r * ldv_s + R * rg;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const T vi = vr[i];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += vi * x[j];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < R; ++i) Vec4<T>::st(Ws + (R * rg + i) * w + 4 * cg, acc[i]);
    __syncthreads();
    // ---- step 2: W <- T^T W
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int kk = R * rg + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        for (int k = 0; k <= kk; ++k) {
            const T t = Tm[k + (long)kk * nb];
            T wv[4];
            Vec4<T>::ld(Ws + k * w + 4 * cg, wv);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += t * wv[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < R; ++i) Vec4<T>::st(Ws + (R * rg + i) * w + 4 * cg, acc[i]);
    __syncthreads();
    // ---- step 3: X_strip -= V W'
    const int rpt = th / nrg;  // rows per thread, multiple of 4
    for (int r0 = 0; r0 < M; r0 += th) {
        const int rows = min(th, M - r0);
        for (int idx = tid; idx < th * w; idx += nt) {
            int r = idx % th, c = idx / th;
            Xs[swz(r, c, w)] = (r < rows && c < wc) ? X[(r0 + r) + (long)(c0 + c) * ldx] : T(0);
        }
        for (int idx = tid; idx < th * nb; idx += nt) {
            int r = idx % th, k = idx / th, gr = r0 + r;
            T v = T(0);
            if (r < rows) v = gr > k ? V[gr + (long)k * ldv] : (gr == k ? T(1) : T(0));
            Vs[k * th + r] = v;  // k-major
        }
        __syncthreads();
        for (int rb = rg * rpt; rb < rg * rpt + rpt; rb += 4) {
            T s[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int j = 0; j < 4; ++j) s[a][j] = T(0);
#pragma unroll U
            for (int k = 0; k < nb; ++k) {
                T v[4], wv[4];
                Vec4<T>::ld(Vs + k * th + rb, v);
                Vec4<T>::ld(Ws + k * w + 4 * cg, wv);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int j = 0; j < 4; ++j) s[a][j] += v[a] * wv[j];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T *p = Xs + swz(rb + a, 4 * cg, w);
                T x[4];
                Vec4<T>::ld(p, x);
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] -= s[a][j];
                Vec4<T>::st(p, x);
            }
        }
        __syncthreads();
        for (int idx = tid; idx < th * w; idx += nt) {
            int r = idx % th, c = idx / th;
            if (r < rows && c < wc) X[(r0 + r) + (long)(c0 + c) * ldx] = Xs[swz(r, c, w)];
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------- LQ side
template <typename T, int R, int U>
__global__ void trail_right_tiled(T *__restrict__ X, long ldx, int M, int N, const T *__restrict__ Vt, long ldvt, int nb,
                  const T *__restrict__ Tm, int th, int h) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldv_s = nb + 4;
    T *Xs = reinterpret_cast<T *>(smem_raw);  // th columns x h rows, column-major (col c at Xs + c*h)
    T *Vs = Xs + (size_t)th * h;             // step 1: th x (nb+4) (row c = V(c, :)); step 3: nb x th (k-major)
    T *Ys = Vs + (size_t)th * ldv_s;         // nb x h (col k at Ys + k*h)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ncg = h >> 2, cg = tid % ncg, rg = tid / ncg, nrg = nt / ncg;
    const int i0 = blockIdx.x * h, hr = min(h, M - i0);

    T acc[R][4];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    // ---- step 1: Y = X_strip V   (acc[i][j] = Y(4cg + j, R rg + i))
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
            Vs[c * ldv_s + k] = v;
        }
        __syncthreads();
#pragma unroll U
        for (int c = 0; c < cols; ++c) {
            T x[4];
            Vec4<T>::ld(Xs + c * h + 4 * cg, x);
            const T *vc = Vs + c * ldv_s + R * rg;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const T vi = vc[i];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += vi * x[j];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < R; ++i) Vec4<T>::st(Ys + (R * rg + i) * h + 4 * cg, acc[i]);
    __syncthreads();
    // ---- step 2: Y <- Y T : Y'(r, kk) = sum_{k <= kk} Y(r, k) T(k, kk)
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int kk = R * rg + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        for (int k = 0; k <= kk; ++k) {
            const T t = Tm[k + (long)kk * nb];
            T yv[4];
            Vec4<T>::ld(Ys + k * h + 4 * cg, yv);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += t * yv[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < R; ++i) Vec4<T>::st(Ys + (R * rg + i) * h + 4 * cg, acc[i]);
    __syncthreads();
    // ---- step 3: X_strip -= Y' V^T  (thread: rows 4cg..4cg+3, columns rg*cpt .. +cpt)
    const int cpt = th / nrg;
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
            Vs[k * th + c] = v;  // k-major
        }
        __syncthreads();
        for (int cbl = rg * cpt; cbl < rg * cpt + cpt; cbl += 4) {
            T s[4][4];  // s[column a][row j]
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int j = 0; j < 4; ++j) s[a][j] = T(0);
#pragma unroll U
            for (int k = 0; k < nb; ++k) {
                T v[4], yv[4];
                Vec4<T>::ld(Vs + k * th + cbl, v);
                Vec4<T>::ld(Ys + k * h + 4 * cg, yv);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int j = 0; j < 4; ++j) s[a][j] += v[a] * yv[j];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T *p = Xs + (cbl + a) * h + 4 * cg;
                T x[4];
                Vec4<T>::ld(p, x);
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] -= s[a][j];
                Vec4<T>::st(p, x);
            }
        }
        __syncthreads();
        for (int idx = tid; idx < th * h; idx += nt) {
            int i = idx % h, c = idx / h;
            if (i < hr && c < cols) X[(i0 + i) + (long)(cb + c) * ldx] = Xs[c * h + i];
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------- dispatch
template <typename T, int R, int U>
static cudaError_t run_tiled(int side, T *X, long ldx, int M, int N, const T *V, long ldv, int nb, const T *Tm,
                             const UpdCfg &c, size_t smem, cudaStream_t st) {
    const int w = 32 * c.cpb;
    if (side == 0) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(trail_left_tiled<T, R, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kTiledSmemLimit);
            attr = true;
        }
        trail_left_tiled<T, R, U><<<(N + w - 1) / w, c.threads, smem, st>>>(X, ldx, M, N, V, ldv, nb, Tm, c.tile, w);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(trail_right_tiled<T, R, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kTiledSmemLimit);
            attr = true;
        }
        trail_right_tiled<T, R, U><<<(M + w - 1) / w, c.threads, smem, st>>>(X, ldx, M, N, V, ldv, nb, Tm, c.tile, w);
    }
    return cudaGetLastError();
}

template <typename T, int R>
static cudaError_t run_tiled_u(int side, T *X, long ldx, int M, int N, const T *V, long ldv, int nb, const T *Tm,
                               const UpdCfg &c, size_t smem, cudaStream_t st) {
    switch (c.unroll) {
        case 1: return run_tiled<T, R, 1>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, st);
        case 2: return run_tiled<T, R, 2>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, st);
        default: return run_tiled<T, R, 4>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, st);
    }
}

template <typename T>
cudaError_t trail_tiled(int side, T *X, long ldx, int M, int N, const T *V, long ldv, int nb, const T *Tm,
                        const UpdCfg &c, cudaStream_t st) {
    const int R = tiled_r(nb, c);
    if (!R) return cudaErrorInvalidConfiguration;
    const size_t smem = tiled_smem(side, (int)sizeof(T), nb, c.tile, 32 * c.cpb);
    if (smem > kTiledSmemLimit) return cudaErrorInvalidConfiguration;
    switch (R) {
        case 1: return run_tiled_u<T, 1>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, st);
        case 2: return run_tiled_u<T, 2>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, st);
        case 4: return run_tiled_u<T, 4>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, st);
        default: return run_tiled_u<T, 8>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, st);
    }
}

template <typename T, int R, int U>
static int max_threads_one(int side) {
    cudaFuncAttributes fa;
    cudaError_t e = side == 0 ? cudaFuncGetAttributes(&fa, trail_left_tiled<T, R, U>)
                              : cudaFuncGetAttributes(&fa, trail_right_tiled<T, R, U>);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return fa.maxThreadsPerBlock;
}

template <typename T, int R>
static int max_threads_r(int side, int u) {
    return u == 1 ? max_threads_one<T, R, 1>(side) : u == 2 ? max_threads_one<T, R, 2>(side) : max_threads_one<T, R, 4>(side);
}

int tiled_max_threads(int side, int elem, int R, int unroll) {
    static int cache[2][2][4][3];
    static bool init = false;
    if (!init) {
        for (auto &a : cache)
            for (auto &b : a)
                for (auto &c : b)
                    for (int &d : c) d = -1;
        init = true;
    }
    const int ri = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : 3, ui = unroll == 1 ? 0 : unroll == 2 ? 1 : 2;
    int &v = cache[side][elem == 8 ? 0 : 1][ri][ui];
    if (v < 0) {
        if (elem == 8)
            v = R == 1 ? max_threads_r<double, 1>(side, unroll) : R == 2 ? max_threads_r<double, 2>(side, unroll)
              : R == 4 ? max_threads_r<double, 4>(side, unroll) : max_threads_r<double, 8>(side, unroll);
        else
            v = R == 1 ? max_threads_r<float, 1>(side, unroll) : R == 2 ? max_threads_r<float, 2>(side, unroll)
              : R == 4 ? max_threads_r<float, 4>(side, unroll) : max_threads_r<float, 8>(side, unroll);
    }
    return v;
}

template cudaError_t trail_tiled<double>(int, double *, long, int, int, const double *, long, int, const double *,
                                         const UpdCfg &, cudaStream_t);
template cudaError_t trail_tiled<float>(int, float *, long, int, int, const float *, long, int, const float *,
                                        const UpdCfg &, cudaStream_t);

}  // namespace nla
