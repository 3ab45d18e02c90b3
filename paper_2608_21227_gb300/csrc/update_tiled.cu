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
// Two launches per side keep every SM busy: step 1 runs on a grid of
// (strips) x (splits of the long dimension, about three waves in all) and the
// last block of each strip -- chosen by an atomic ticket, so nothing waits --
// reduces the partial sums and applies T (step 2); step 3 runs on a full 2-D
// grid of (tile x strip) blocks.
//
// QR side: X tiles are staged row-major with an XOR swizzle of the 4-column
// group by (row & 7), so that both the column-wise staging stores and the
// row-wise 128-bit reads are free of bank conflicts.  LQ side: X tiles are
// staged column-major (the strip rows are contiguous), which needs no swizzle.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace nla {

constexpr size_t kTiledSmemLimit = 226 * 1024;  // dynamic bytes; the kernels' static shared memory fits in the rest

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
// Step 1 (+ step 2 in the last block of each strip): block (cb, s) accumulates
// the partial W = V^T X over rows [s*Ms, (s+1)*Ms) of strip cb and stores it;
// the last block of the strip to finish (atomic ticket) sums the S partials,
// applies T^T and stores W' for step 3.
template <typename T, int R, int U>
__global__ void left_w_kernel(const T *__restrict__ X, long ldx, int M, int N, const T *__restrict__ V, long ldv,
                              int nb, const T *__restrict__ Tm, int th, int w, int Ms, T *part, T *fin,
                              unsigned int *tickets) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int sh_last;
    const int ldv_s = nb + 4;
    T *Xs = reinterpret_cast<T *>(smem_raw);  // th x w, swizzled
    T *Vs = Xs + (size_t)th * w;             // th x (nb+4) row-major
    T *Ws = Vs + (size_t)th * ldv_s;         // nb x w row-major
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ncg = w >> 2, cg = tid % ncg, rg = tid / ncg;
    const int c0 = blockIdx.x * w, wc = min(w, N - c0);
    const int s = blockIdx.y, S = gridDim.y;
    const int rbeg = s * Ms, rend = min(M, rbeg + Ms);

    T acc[R][4];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int r0 = rbeg; r0 < rend; r0 += th) {
        const int rows = min(th, rend - r0);
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
            T x[4], v[R];
            Vec4<T>::ld(Xs + swz(r, 4 * cg, w), x);
            const T *vr = Vs + r * ldv_s + R * rg;
            if constexpr (R % 4 == 0) {
#pragma unroll
                for (int i = 0; i < R; i += 4) Vec4<T>::ld(vr + i, v + i);
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) v[i] = vr[i];
            }
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += v[i] * x[j];
        }
        __syncthreads();
    }
    // store the partial W (nb x N slab of this split)
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * cg + j;
            if (c < wc) part[((size_t)s * nb + R * rg + i) * N + c0 + c] = acc[i][j];
        }
    __threadfence();
    __syncthreads();
    if (tid == 0) sh_last = atomicAdd(&tickets[blockIdx.x], 1u) == (unsigned)(S - 1);
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // ---- step 2 (last block of the strip): W = sum of partials; W' = T^T W
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * cg + j;
            T sum = T(0);
            if (c < wc)
                for (int q = 0; q < S; ++q) sum += __ldcg(part + ((size_t)q * nb + R * rg + i) * N + c0 + c);
            acc[i][j] = sum;
        }
#pragma unroll
    for (int i = 0; i < R; ++i) Vec4<T>::st(Ws + (R * rg + i) * w + 4 * cg, acc[i]);
    __syncthreads();
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
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * cg + j;
            if (c < wc) fin[(size_t)kk * N + c0 + c] = acc[i][j];
        }
    }
    if (tid == 0) tickets[blockIdx.x] = 0u;  // ready for the next launch
}

// Step 3: block (cb, rb) updates the th x w tile X(rb, cb) -= V(rb, :) W'(:, cb).
template <typename T, int U>
__global__ void left_x_kernel(T *__restrict__ X, long ldx, int M, int N, const T *__restrict__ V, long ldv, int nb,
                              int th, int w, const T *__restrict__ fin) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);  // th x w, swizzled
    T *Vs = Xs + (size_t)th * w;             // nb x th, k-major
    T *Ws = Vs + (size_t)th * (nb + 4);      // nb x w
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ncg = w >> 2, cg = tid % ncg, rg = tid / ncg, nrg = nt / ncg;
    const int c0 = blockIdx.x * w, wc = min(w, N - c0);
    const int r0 = blockIdx.y * th, rows = min(th, M - r0);
    for (int idx = tid; idx < th * w; idx += nt) {
        int r = idx % th, c = idx / th;
        Xs[swz(r, c, w)] = (r < rows && c < wc) ? X[(r0 + r) + (long)(c0 + c) * ldx] : T(0);
    }
    for (int idx = tid; idx < th * nb; idx += nt) {
        int r = idx % th, k = idx / th, gr = r0 + r;
        T v = T(0);
        if (r < rows) v = gr > k ? V[gr + (long)k * ldv] : (gr == k ? T(1) : T(0));
        Vs[k * th + r] = v;
    }
    for (int idx = tid; idx < nb * w; idx += nt) {
        int c = idx % w, k = idx / w;
        Ws[k * w + c] = c < wc ? fin[(size_t)k * N + c0 + c] : T(0);
    }
    __syncthreads();
    const int rpt = th / nrg;  // rows per thread, a multiple of 4
    for (int rb = rg * rpt; rb < rg * rpt + rpt; rb += 4) {
        T sacc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < 4; ++j) sacc[a][j] = T(0);
#pragma unroll U
        for (int k = 0; k < nb; ++k) {
            T v[4], wv[4];
            Vec4<T>::ld(Vs + k * th + rb, v);
            Vec4<T>::ld(Ws + k * w + 4 * cg, wv);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int j = 0; j < 4; ++j) sacc[a][j] += v[a] * wv[j];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            T *p = Xs + swz(rb + a, 4 * cg, w);
            T x[4];
            Vec4<T>::ld(p, x);
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] -= sacc[a][j];
            Vec4<T>::st(p, x);
        }
    }
    __syncthreads();
    for (int idx = tid; idx < th * w; idx += nt) {
        int r = idx % th, c = idx / th;
        if (r < rows && c < wc) X[(r0 + r) + (long)(c0 + c) * ldx] = Xs[swz(r, c, w)];
    }
}

// -------------------------------------------------------------------- LQ side
// Step 1 (+2): block (rb, s) accumulates Y = X V over columns [s*Ns, (s+1)*Ns)
// of the h-row strip rb; the last block sums the partials and stores Y' = Y T.
template <typename T, int R, int U>
__global__ void right_w_kernel(const T *__restrict__ X, long ldx, int M, int N, const T *__restrict__ Vt, long ldvt,
                               int nb, const T *__restrict__ Tm, int th, int h, int Ns, T *part, T *fin,
                               unsigned int *tickets) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int sh_last;
    const int ldv_s = nb + 4;
    T *Xs = reinterpret_cast<T *>(smem_raw);  // th columns x h rows, column-major
    T *Vs = Xs + (size_t)th * h;             // th x (nb+4): row c = V(c, :)
    T *Ys = Vs + (size_t)th * ldv_s;         // nb x h
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ncg = h >> 2, cg = tid % ncg, rg = tid / ncg;
    const int i0 = blockIdx.x * h, hr = min(h, M - i0);
    const int s = blockIdx.y, S = gridDim.y;
    const int cbeg = s * Ns, cend = min(N, cbeg + Ns);

    T acc[R][4];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int cb = cbeg; cb < cend; cb += th) {
        const int cols = min(th, cend - cb);
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
            T x[4], v[R];
            Vec4<T>::ld(Xs + c * h + 4 * cg, x);
            const T *vc = Vs + c * ldv_s + R * rg;
            if constexpr (R % 4 == 0) {
#pragma unroll
                for (int i = 0; i < R; i += 4) Vec4<T>::ld(vc + i, v + i);
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) v[i] = vc[i];
            }
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += v[i] * x[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = 4 * cg + j;
            if (r < hr) part[((size_t)s * nb + R * rg + i) * M + i0 + r] = acc[i][j];
        }
    __threadfence();
    __syncthreads();
    if (tid == 0) sh_last = atomicAdd(&tickets[blockIdx.x], 1u) == (unsigned)(S - 1);
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = 4 * cg + j;
            T sum = T(0);
            if (r < hr)
                for (int q = 0; q < S; ++q) sum += __ldcg(part + ((size_t)q * nb + R * rg + i) * M + i0 + r);
            acc[i][j] = sum;
        }
#pragma unroll
    for (int i = 0; i < R; ++i) Vec4<T>::st(Ys + (R * rg + i) * h + 4 * cg, acc[i]);
    __syncthreads();
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
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = 4 * cg + j;
            if (r < hr) fin[(size_t)kk * M + i0 + r] = acc[i][j];
        }
    }
    if (tid == 0) tickets[blockIdx.x] = 0u;
}

// Step 3: block (rb, cbk) updates the h x th tile X(rb, cbk) -= Y'(rb, :) V(cbk, :)^T.
template <typename T, int U>
__global__ void right_x_kernel(T *__restrict__ X, long ldx, int M, int N, const T *__restrict__ Vt, long ldvt, int nb,
                               int th, int h, const T *__restrict__ fin) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);  // th columns x h rows
    T *Vs = Xs + (size_t)th * h;             // nb x th, k-major
    T *Ys = Vs + (size_t)th * (nb + 4);      // nb x h
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ncg = h >> 2, cg = tid % ncg, rg = tid / ncg, nrg = nt / ncg;
    const int i0 = blockIdx.x * h, hr = min(h, M - i0);
    const int cb = blockIdx.y * th, cols = min(th, N - cb);
    for (int idx = tid; idx < th * h; idx += nt) {
        int i = idx % h, c = idx / h;
        Xs[c * h + i] = (i < hr && c < cols) ? X[(i0 + i) + (long)(cb + c) * ldx] : T(0);
    }
    for (int idx = tid; idx < th * nb; idx += nt) {
        int k = idx % nb, c = idx / nb, gc = cb + c;
        T v = T(0);
        if (c < cols) v = gc > k ? Vt[k + (long)gc * ldvt] : (gc == k ? T(1) : T(0));
        Vs[k * th + c] = v;
    }
    for (int idx = tid; idx < nb * h; idx += nt) {
        int i = idx % h, k = idx / h;
        Ys[k * h + i] = i < hr ? fin[(size_t)k * M + i0 + i] : T(0);
    }
    __syncthreads();
    const int cpt = th / nrg;
    for (int cbl = rg * cpt; cbl < rg * cpt + cpt; cbl += 4) {
        T sacc[4][4];  // [column a][row j]
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < 4; ++j) sacc[a][j] = T(0);
#pragma unroll U
        for (int k = 0; k < nb; ++k) {
            T v[4], yv[4];
            Vec4<T>::ld(Vs + k * th + cbl, v);
            Vec4<T>::ld(Ys + k * h + 4 * cg, yv);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int j = 0; j < 4; ++j) sacc[a][j] += v[a] * yv[j];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            T *p = Xs + (cbl + a) * h + 4 * cg;
            T x[4];
            Vec4<T>::ld(p, x);
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] -= sacc[a][j];
            Vec4<T>::st(p, x);
        }
    }
    __syncthreads();
    for (int idx = tid; idx < th * h; idx += nt) {
        int i = idx % h, c = idx / h;
        if (i < hr && c < cols) X[(i0 + i) + (long)(cb + c) * ldx] = Xs[c * h + i];
    }
}

// -------------------------------------------------------------------- dispatch
constexpr int kMaxSplit = 8;

// partial slabs, the projection's W' / Y', and room for the mixed path's line exponents
size_t tiled_scratch_elems(int M, int N) { return (size_t)(kMaxSplit + 2) * 64 * (size_t)std::max(std::max(M, N), 1); }
size_t tiled_tickets(int M, int N) { return (size_t)std::max(M, N) / 32 + 2; }

// number of splits of the long dimension L for `nblk` strips: about three waves
static int split_count(int L, int th, int nblk) {
    int S = (3 * device_sm_count() + nblk - 1) / std::max(nblk, 1);
    S = std::max(1, std::min({S, kMaxSplit, (L + th - 1) / th}));
    return S;
}

template <typename T, int R, int U>
static cudaError_t run_tiled(int side, T *X, long ldx, int M, int N, const T *V, long ldv, int nb, const T *Tm,
                             const UpdCfg &c, size_t smem, const UpdScratch &sc, cudaStream_t st) {
    const int w = 32 * c.cpb, th = c.tile;
    T *part = reinterpret_cast<T *>(sc.work);
    T *fin = part + (size_t)kMaxSplit * 64 * std::max(M, N);
    if (side == 0) {
        static PerDeviceOnce a1, a3;
        allow_max_smem(left_w_kernel<T, R, U>, a1);
        allow_max_smem(left_x_kernel<T, U>, a3);
        const int nblk = (N + w - 1) / w;
        int S = split_count(M, th, nblk);
        const int Ms = ((M + S - 1) / S + th - 1) / th * th;
        S = (M + Ms - 1) / Ms;
        left_w_kernel<T, R, U><<<dim3(nblk, S), c.threads, smem, st>>>(X, ldx, M, N, V, ldv, nb, Tm, th, w, Ms, part,
                                                                       fin, sc.tickets);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        left_x_kernel<T, U><<<dim3(nblk, (M + th - 1) / th), c.threads, smem, st>>>(X, ldx, M, N, V, ldv, nb, th, w,
                                                                                   fin);
    } else {
        static PerDeviceOnce a1, a3;
        allow_max_smem(right_w_kernel<T, R, U>, a1);
        allow_max_smem(right_x_kernel<T, U>, a3);
        const int nblk = (M + w - 1) / w;
        int S = split_count(N, th, nblk);
        const int Ns = ((N + S - 1) / S + th - 1) / th * th;
        S = (N + Ns - 1) / Ns;
        right_w_kernel<T, R, U><<<dim3(nblk, S), c.threads, smem, st>>>(X, ldx, M, N, V, ldv, nb, Tm, th, w, Ns, part,
                                                                        fin, sc.tickets);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        right_x_kernel<T, U><<<dim3(nblk, (N + th - 1) / th), c.threads, smem, st>>>(X, ldx, M, N, V, ldv, nb, th, w,
                                                                                    fin);
    }
    return cudaGetLastError();
}

template <typename T, int R>
static cudaError_t run_tiled_u(int side, T *X, long ldx, int M, int N, const T *V, long ldv, int nb, const T *Tm,
                               const UpdCfg &c, size_t smem, const UpdScratch &sc, cudaStream_t st) {
    switch (c.unroll) {
        case 1: return run_tiled<T, R, 1>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, sc, st);
        case 2: return run_tiled<T, R, 2>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, sc, st);
        default: return run_tiled<T, R, 4>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, sc, st);
    }
}

template <typename T>
cudaError_t trail_tiled(int side, T *X, long ldx, int M, int N, const T *V, long ldv, int nb, const T *Tm,
                        const UpdCfg &c, const UpdScratch &sc, cudaStream_t st) {
    const int R = tiled_r(nb, c);
    if (!R || !sc.work || !sc.tickets) return cudaErrorInvalidConfiguration;
    const size_t smem = tiled_smem(side, (int)sizeof(T), nb, c.tile, 32 * c.cpb);
    if (smem > kTiledSmemLimit) return cudaErrorInvalidConfiguration;
    switch (R) {
        case 1: return run_tiled_u<T, 1>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, sc, st);
        case 2: return run_tiled_u<T, 2>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, sc, st);
        case 4: return run_tiled_u<T, 4>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, sc, st);
        default: return run_tiled_u<T, 8>(side, X, ldx, M, N, V, ldv, nb, Tm, c, smem, sc, st);
    }
}

// Largest block the compiled kernel can launch; 1024 (not cached) when it cannot be
// asked because this process has no CUDA device.
template <typename K>
static int kernel_max_threads(K kernel, bool &known) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
        cudaGetLastError();
        known = false;
        return 1024;
    }
    return fa.maxThreadsPerBlock;
}

template <typename T, int R, int U>
static int max_threads_one(int side, bool &known) {
    if (side == 0)
        return std::min(kernel_max_threads(left_w_kernel<T, R, U>, known), kernel_max_threads(left_x_kernel<T, U>, known));
    return std::min(kernel_max_threads(right_w_kernel<T, R, U>, known), kernel_max_threads(right_x_kernel<T, U>, known));
}

template <typename T, int R>
static int max_threads_r(int side, int u, bool &known) {
    return u == 1 ? max_threads_one<T, R, 1>(side, known)
           : u == 2 ? max_threads_one<T, R, 2>(side, known) : max_threads_one<T, R, 4>(side, known);
}

int tiled_max_threads(int side, int elem, int R, int unroll) {
    // a kernel's thread limit (from its register count) is the same on every device of
    // this architecture: cached once, under a lock
    static std::mutex mu;
    static int cache[2][2][4][3];
    static bool init = false;
    std::lock_guard<std::mutex> lk(mu);
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
        bool known = true;
        int q;
        if (elem == 8)
            q = R == 1 ? max_threads_r<double, 1>(side, unroll, known) : R == 2 ? max_threads_r<double, 2>(side, unroll, known)
              : R == 4 ? max_threads_r<double, 4>(side, unroll, known) : max_threads_r<double, 8>(side, unroll, known);
        else
            q = R == 1 ? max_threads_r<float, 1>(side, unroll, known) : R == 2 ? max_threads_r<float, 2>(side, unroll, known)
              : R == 4 ? max_threads_r<float, 4>(side, unroll, known) : max_threads_r<float, 8>(side, unroll, known);
        if (!known) return q;
        v = q;
    }
    return v;
}

template cudaError_t trail_tiled<double>(int, double *, long, int, int, const double *, long, int, const double *,
                                         const UpdCfg &, const UpdScratch &, cudaStream_t);
template cudaError_t trail_tiled<float>(int, float *, long, int, int, const float *, long, int, const float *,
                                        const UpdCfg &, const UpdScratch &, cudaStream_t);

}  // namespace nla
