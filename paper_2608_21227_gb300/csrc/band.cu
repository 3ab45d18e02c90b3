// band.cu -- input staging, band extraction and stage 2 (band -> bidiagonal).
//
// Band storage (entries with -b <= j - i <= 2b): A(i, j) at AB[(2b + i - j) + j*ldab],
// ldab >= 3b + 1.  Stage 1 leaves an upper band 0 <= j - i <= b; the extra b
// rows below and b rows above hold the bulges created while chasing.
//
// Bulge chasing (Section 5.1.1: band -> bidiagonal by orthogonal
// transformations that keep the singular values intact).  Sweep s makes row s
// bidiagonal.  Its block step k (k = 0, 1, ...) applies
//   right:  a reflector on columns c0..c1 = s+kb+1 .. s+(k+1)b that zeroes row
//           tr (tr = s for k = 0, s+(k-1)b+1 otherwise) beyond column c0; it is
//           applied to rows tr..c1 and fills the block below the diagonal;
//   left:   a reflector on rows c0..r1 = c0 .. s+(k+1)b that zeroes column c0
//           below the diagonal; it is applied to columns c0..s+(k+2)b and fills
//           row c0 beyond the band, which the right reflector of step k+1
//           removes.
// Fill that one sweep leaves behind (the rest of each triangular bulge) is
// exactly what the next sweep's reflectors at the same position remove.  Block
// step k of sweep s touches rows s+(k-1)b+1 .. s+(k+1)b only, so it is
// independent of every step >= k+3 of sweep s-1: sweeps run concurrently,
// one per block, each waiting (bounded spin) until its predecessor has
// finished three more steps.
#include <algorithm>
#include <cstdlib>
#include <climits>

#include "common.cuh"
#include "kernels.cuh"

namespace nla {

// ------------------------------------------------------------------ copies
template <typename T>
__global__ void copy_kernel(const T *__restrict__ A, long lda, int m, int n, T *__restrict__ B, long ldb) {
    long total = (long)m * n;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        long j = idx / m, i = idx % m;
        B[i + j * ldb] = A[i + j * lda];
    }
}

// B (n x m) = A^T via 32 x 32 shared-memory tiles
template <typename T>
__global__ void transpose_kernel(const T *__restrict__ A, long lda, int m, int n, T *__restrict__ B, long ldb) {
    __shared__ T tile[32][33];
    int bi = blockIdx.x * 32, bj = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int i = bi + threadIdx.x, j = bj + y;
        if (i < m && j < n) tile[y][threadIdx.x] = A[i + (long)j * lda];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int j = bj + threadIdx.x, i = bi + y;  // B(j, i) = A(i, j)
        if (i < m && j < n) B[j + (long)i * ldb] = tile[threadIdx.x][y];
    }
}

template <typename T>
cudaError_t copy_matrix(const T *A, long lda, int m, int n, T *B, long ldb, bool transpose, cudaStream_t st) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (!transpose) {
        long total = (long)m * n;
        int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
        copy_kernel<T><<<blocks, 256, 0, st>>>(A, lda, m, n, B, ldb);
    } else {
        dim3 grid((m + 31) / 32, (n + 31) / 32);
        transpose_kernel<T><<<grid, dim3(32, 8), 0, st>>>(A, lda, m, n, B, ldb);
    }
    return cudaGetLastError();
}

template <typename T>
__global__ void band_extract_kernel(const T *__restrict__ A, long lda, int n, int b, T *__restrict__ AB,
                                    long ldab) {
    const int j = blockIdx.x;
    if (j >= n) return;
    for (int q = threadIdx.x; q < ldab; q += blockDim.x) {
        int i = q - 2 * b + j;  // storage row q holds A(i, j)
        T v = T(0);
        if (q >= b && q <= 2 * b && i >= 0) v = A[i + (long)j * lda];
        AB[q + (long)j * ldab] = v;
    }
}

template <typename T>
cudaError_t band_extract(const T *A, long lda, int n, int b, T *AB, long ldab, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    band_extract_kernel<T><<<n, 128, 0, st>>>(A, lda, n, b, AB, ldab);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ bulge chasing
constexpr int kChaseThreads = 128;  // >= 2b - 1 rows / columns per reflector application

size_t band2bd_scratch_bytes(int n) { return (size_t)std::max(n, 1) * sizeof(int); }

template <typename T>
struct Band {
    T *AB;
    long ldab;
    int b2;  // 2b
    NLA_DEV T *at(int i, int j) const { return AB + (b2 + i - j) + (long)j * ldab; }
};

// Householder reflector of the vector held in v[0..L-1] (shared memory), built by
// one warp: v becomes [1; x / (alpha - beta)], *tau and *beta are set.
template <typename T>
NLA_DEV void warp_reflector(T *v, int L, T *tau_out, T *beta_out) {
    const int lane = threadIdx.x & 31;
    T s = T(0);
    for (int i = 1 + lane; i < L; i += 32) s += v[i] * v[i];
    s = warp_sum(s);
    T alpha = v[0];
    T tau = T(0), beta = alpha, scale = T(0);
    if (s > T(0)) {
        T r = sqrt(alpha * alpha + s);
        beta = alpha >= T(0) ? -r : r;
        tau = (beta - alpha) / beta;
        scale = T(1) / (alpha - beta);
    }
    __syncwarp();
    for (int i = 1 + lane; i < L; i += 32) v[i] = (tau != T(0)) ? v[i] * scale : T(0);
    __syncwarp();
    if (lane == 0) {
        v[0] = T(1);
        *tau_out = tau;
        *beta_out = beta;
    }
}

// One block step (right + left reflector) of sweep s at position k, on a
// shared-memory copy of its window.  The window is the box rows [tr, r1] x
// columns [c0, cend]; only its two sub-boxes that the step reads or writes are
// moved: R = rows [tr, c1] x columns [c0, c1] and L = rows [c0, r1] x columns
// [c0, cend] (c1 = r1).  W(i, j) = W[(i - tr) + (j - c0) * ldw].
template <typename T>
NLA_DEV void chase_step(const Band<T> &A, int n, int b, int s, int k, T *W, int ldw, T *v, T *sh) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int c0 = s + k * b + 1;
    const int tr = (k == 0) ? s : s + (k - 1) * b + 1;
    const int c1 = min(s + (k + 1) * b, n - 1);  // == r1
    const int cend = min(s + (k + 2) * b, n - 1);
    const int L = c1 - c0 + 1;                  // right reflector length == left reflector length
    const int hR = c1 - tr + 1;                 // rows of R
    const int wL = cend - c0 + 1;               // columns of L
    const int top = c0 - tr;                    // rows of R above L
    // ---- load: columns of R (rows tr..c1) and the columns of L right of R (rows c0..c1)
    for (int idx = tid; idx < hR * L; idx += nt) {
        int i = idx % hR, j = idx / hR;
        W[i + j * ldw] = __ldcg(A.at(tr + i, c0 + j));
    }
    for (int idx = tid; idx < L * (wL - L); idx += nt) {
        int i = idx % L, j = L + idx / L;
        W[top + i + j * ldw] = __ldcg(A.at(c0 + i, c0 + j));
    }
    __syncthreads();
    // ---- right reflector on columns c0..c1 from row tr
    if (L >= 2) {
        for (int j = tid; j < L; j += nt) v[j] = W[0 + j * ldw];
        __syncthreads();
        if (tid < 32) warp_reflector<T>(v, L, sh, sh + 1);
        __syncthreads();
        const T tau = sh[0];
        if (tau != T(0)) {
            if (tid == 0) W[0] = sh[1];
            for (int j = 1 + tid; j < L; j += nt) W[j * ldw] = T(0);
            for (int i = 1 + tid; i < hR; i += nt) {  // one thread per row
                T w = T(0);
                for (int j = 0; j < L; ++j) w += W[i + j * ldw] * v[j];
                w *= tau;
                for (int j = 0; j < L; ++j) W[i + j * ldw] -= w * v[j];
            }
        }
        __syncthreads();
    }
    // ---- left reflector on rows c0..c1 from column c0
    if (L >= 2) {
        for (int i = tid; i < L; i += nt) v[i] = W[top + i];
        __syncthreads();
        if (tid < 32) warp_reflector<T>(v, L, sh, sh + 1);
        __syncthreads();
        const T tau = sh[0];
        if (tau != T(0)) {
            if (tid == 0) W[top] = sh[1];
            for (int i = 1 + tid; i < L; i += nt) W[top + i] = T(0);
            for (int j = 1 + tid; j < wL; j += nt) {  // one thread per column
                T *col = W + top + j * ldw;
                T w = T(0);
                for (int i = 0; i < L; ++i) w += v[i] * col[i];
                w *= tau;
                for (int i = 0; i < L; ++i) col[i] -= w * v[i];
            }
        }
        __syncthreads();
    }
    // ---- store R and the part of L right of R
    for (int idx = tid; idx < hR * L; idx += nt) {
        int i = idx % hR, j = idx / hR;
        __stcg(A.at(tr + i, c0 + j), W[i + j * ldw]);
    }
    for (int idx = tid; idx < L * (wL - L); idx += nt) {
        int i = idx % L, j = L + idx / L;
        __stcg(A.at(c0 + i, c0 + j), W[top + i + j * ldw]);
    }
}

template <typename T>
__global__ void __launch_bounds__(kChaseThreads)
band2bd_kernel(T *AB, long ldab, int n, int b, int *progress, int *info) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldw = 2 * b + 1;
    T *W = reinterpret_cast<T *>(smem_raw);  // (2b+1) x 2b window
    T *v = W + (size_t)ldw * 2 * b;          // reflector, <= b entries
    T *sh = v + 64;                          // tau, beta
    __shared__ int sh_fail;
    const int tid = threadIdx.x;
    Band<T> A{AB, ldab, 2 * b};
    const int nsweeps = n - 2;
    if (tid == 0) sh_fail = 0;
    __syncthreads();

    for (int s = blockIdx.x; s < nsweeps; s += gridDim.x) {
        for (int k = 0;; ++k) {
            const int c0 = s + k * b + 1;
            if (c0 > n - 1) break;
            if (s > 0) {
                if (tid == 0 && !spin_until_geq(&progress[s - 1], k + 3, info)) sh_fail = 1;
                __syncthreads();
                if (sh_fail) return;
            }
            chase_step<T>(A, n, b, s, k, W, ldw, v, sh);
            __threadfence();
            __syncthreads();
            if (tid == 0) st_release(&progress[s], k + 1);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(&progress[s], INT_MAX);
    }
}

// ------------------------------------------------------------------ grouped bulge chasing
// A block runs a group of G consecutive sweeps s0 .. s0+G-1, one warp per
// sweep, on a window of band columns held in shared memory (columns stored
// circularly, the same 3b+1 storage rows per column).  At wavefront step tau,
// warp i performs block step k = tau - 2i of its sweep in two halves -- every
// warp's right reflector, a barrier, every warp's left reflector, a barrier.
// With sweeps two block steps apart, half-steps that share an entry then run
// in the order of the sequential chase and concurrent ones are disjoint (the
// one entry that steps (s, k+2) and (s+1, k) share is written by the former's
// right reflector before the latter's left one); a whole-step schedule would
// need three steps between sweeps.  Columns that no sweep of the group will
// touch again are written back to global memory and announced in done[group]
// ("every column < value is final"); the next group waits (bounded spin) until
// the columns it loads are final.  The window spans at most (2G-1) b + G + 1
// columns.
template <typename T>
struct Win {
    T *w;
    int ldw, wc, b2;
    NLA_DEV T &at(int i, int j) const { return w[(b2 + i - j) + (j % wc) * ldw]; }
    // Column j's storage shifted so that element (i, j) is col(j)[i].
    NLA_DEV T *col(int j) const { return w + (size_t)(j % wc) * ldw + b2 - j; }
    // Column j0 + c from j0's slot (0 <= c < wc): one compare instead of a division.
    NLA_DEV T *col_from(int slot0, int j0, int c) const {
        int sl = slot0 + c;
        sl -= sl >= wc ? wc : 0;
        return w + (size_t)sl * ldw + b2 - (j0 + c);
    }
};

// Householder scalars of (alpha, x) with ||x||^2 = xn2: beta, tau = (beta - alpha) / beta
// and 1 / (alpha - beta).  FP32 uses the fast reciprocal square root and division
// (a few ulp, far inside the FP32 path's tolerance); FP64 the correctly rounded ones.
template <typename T>
NLA_DEV void house_scalars(T alpha, T xn2, T &beta, T &tau, T &scale) {
    tau = T(0), beta = alpha, scale = T(0);
    if (xn2 > T(0)) {
        if constexpr (sizeof(T) == 4) {
            const float q = alpha * alpha + xn2;
            const float r = q * rsqrtf(q);
            beta = alpha >= 0.f ? -r : r;
            tau = __fdividef(beta - alpha, beta);
            scale = __fdividef(1.f, alpha - beta);
        } else {
            const T r = sqrt(alpha * alpha + xn2);
            beta = alpha >= T(0) ? -r : r;
            tau = (beta - alpha) / beta;
            scale = T(1) / (alpha - beta);
        }
    }
}

// One block step (right + left reflector) of sweep s at position k by one warp;
// sl0 = window slot of column c0 = s + k b + 1.  B = the band width when it is a
// compile-time constant (<= 32: the reflector and the lane's row or column are then
// held in registers, every load issues at once and nothing is reloaded), 0 otherwise.
template <typename T, int B>
NLA_DEV void warp_chase_step(const Win<T> &W, int n, int b, int s, int k, int sl0, T *v, int part) {
    const int lane = threadIdx.x & 31;
    const int c0 = s + k * b + 1;
    const int tr = (k == 0) ? s : s + (k - 1) * b + 1;
    const int c1 = min(s + (k + 1) * b, n - 1);
    const int cend = min(s + (k + 2) * b, n - 1);
    const int L = c1 - c0 + 1;
    if (L < 2) return;
    constexpr int UB = (B > 0 && B <= 32) ? B : 1;
    T xa, xb, xn2, alpha, tau, beta, scale;
    if (part == 1) goto left;
    // ---- right reflector on columns c0..c1 from row tr, applied to rows tr+1..c1
    // (lane c < 32 holds entry (tr, c0 + c); L <= 64 for the generic form)
    xa = lane < L ? W.col_from(sl0, c0, lane)[tr] : T(0);
    xb = lane + 32 < L ? W.col_from(sl0, c0, lane + 32)[tr] : T(0);
    xn2 = warp_sum((lane > 0 ? xa * xa : T(0)) + xb * xb);
    alpha = __shfl_sync(0xffffffffu, xa, 0);
    house_scalars<T>(alpha, xn2, beta, tau, scale);
    if (tau != T(0)) {
        if (lane < L) {
            v[lane] = lane == 0 ? T(1) : xa * scale;
            W.col_from(sl0, c0, lane)[tr] = lane == 0 ? beta : T(0);
        }
        if (lane + 32 < L) {
            v[lane + 32] = xb * scale;
            W.col_from(sl0, c0, lane + 32)[tr] = T(0);
        }
        __syncwarp();
        if (B > 0 && B <= 32 && L == B) {
            T vr[UB];
#pragma unroll
            for (int c = 0; c < UB; ++c) vr[c] = v[c];
            // apply to the lane's row held in xr (columns c0 .. c0 + B - 1)
            auto apply_row = [&](T(&xr)[UB]) {
                T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
                for (int c = 0; c < UB; c += 4) {
                    d0 += xr[c] * vr[c];
                    if (c + 1 < UB) d1 += xr[c + 1] * vr[c + 1];
                    if (c + 2 < UB) d2 += xr[c + 2] * vr[c + 2];
                    if (c + 3 < UB) d3 += xr[c + 3] * vr[c + 3];
                }
                const T w = tau * ((d0 + d1) + (d2 + d3));
#pragma unroll
                for (int c = 0; c < UB; ++c) xr[c] -= w * vr[c];
            };
            if (sl0 + B <= W.wc) {
                // the B columns sit in consecutive slots: entry (i, c0 + c) is
                // base[i + c (ldw - 1)], constant offsets from one address per lane
                constexpr int LDW1 = ((3 * UB + 2) & ~1) - 1;
                T *base = W.w + (size_t)sl0 * W.ldw + W.b2 - c0;
                for (int i = tr + 1 + lane; i <= c1; i += 32) {  // one lane per row
                    T *rp = base + i;
                    T xr[UB];
#pragma unroll
                    for (int c = 0; c < UB; ++c) xr[c] = rp[c * LDW1];
                    apply_row(xr);
#pragma unroll
                    for (int c = 0; c < UB; ++c) rp[c * LDW1] = xr[c];
                }
            } else {
                for (int i = tr + 1 + lane; i <= c1; i += 32) {
                    T xr[UB];
#pragma unroll
                    for (int c = 0; c < UB; ++c) xr[c] = W.col_from(sl0, c0, c)[i];
                    apply_row(xr);
#pragma unroll
                    for (int c = 0; c < UB; ++c) W.col_from(sl0, c0, c)[i] = xr[c];
                }
            }
        } else {
            for (int i = tr + 1 + lane; i <= c1; i += 32) {  // one lane per row
                T w = T(0);
                for (int c = 0; c < L; ++c) w += W.col_from(sl0, c0, c)[i] * v[c];
                w *= tau;
                for (int c = 0; c < L; ++c) W.col_from(sl0, c0, c)[i] -= w * v[c];
            }
        }
        __syncwarp();
    }
    if (part == 0) return;
left:
    // ---- left reflector on rows c0..c1 from column c0, applied to columns c0+1..cend
    T *clw = W.col_from(sl0, c0, 0) + c0;  // clw[r] = entry (c0 + r, c0)
    xa = lane < L ? clw[lane] : T(0);
    xb = lane + 32 < L ? clw[lane + 32] : T(0);
    xn2 = warp_sum((lane > 0 ? xa * xa : T(0)) + xb * xb);
    alpha = __shfl_sync(0xffffffffu, xa, 0);
    house_scalars<T>(alpha, xn2, beta, tau, scale);
    if (tau != T(0)) {
        if (lane < L) {
            v[lane] = lane == 0 ? T(1) : xa * scale;
            clw[lane] = lane == 0 ? beta : T(0);
        }
        if (lane + 32 < L) {
            v[lane + 32] = xb * scale;
            clw[lane + 32] = T(0);
        }
        __syncwarp();
        if (B > 0 && B <= 32 && L == B) {
            T vr[UB];
#pragma unroll
            for (int r = 0; r < UB; ++r) vr[r] = v[r];
            for (int j = c0 + 1 + lane; j <= cend; j += 32) {  // one lane per column
                T *cj = W.col_from(sl0, c0, j - c0) + c0;
                T xr[UB];
#pragma unroll
                for (int r = 0; r < UB; ++r) xr[r] = cj[r];
                T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
                for (int r = 0; r < UB; r += 4) {
                    d0 += xr[r] * vr[r];
                    if (r + 1 < UB) d1 += xr[r + 1] * vr[r + 1];
                    if (r + 2 < UB) d2 += xr[r + 2] * vr[r + 2];
                    if (r + 3 < UB) d3 += xr[r + 3] * vr[r + 3];
                }
                const T w = tau * ((d0 + d1) + (d2 + d3));
#pragma unroll
                for (int r = 0; r < UB; ++r) cj[r] = xr[r] - w * vr[r];
            }
        } else {
            for (int j = c0 + 1 + lane; j <= cend; j += 32) {  // one lane per column
                T *cj = W.col_from(sl0, c0, j - c0);
                T w = T(0);
                for (int r = 0; r < L; ++r) w += v[r] * cj[c0 + r];
                w *= tau;
                for (int r = 0; r < L; ++r) cj[c0 + r] -= w * v[r];
            }
        }
        __syncwarp();
    }
}

// Window of the group [s0, s0+g) at wavefront step tau: columns [lo, hi].  lo
// is the first column any unfinished sweep will still touch (a sweep that has
// not started yet will start at column s+1), hi the last column a running
// sweep touches now.  active = some sweep of the group is unfinished.
constexpr int kLag = 2;  // block steps between consecutive sweeps of a group

NLA_DEV void group_need(int n, int b, int s0, int g, int tau, int &lo, int &hi, bool &active) {
    // c0 of sweep i at step tau - kLag i decreases with i, so the last started sweep
    // (i_ls) holds the lowest column in use and the first unfinished one (i_f) the
    // highest; sweeps with s >= n - 2 do not run.
    lo = n;
    hi = -1;
    active = false;
    const int gv = min(g, n - 2 - s0);
    if (gv <= 0) return;
    const int ils = min(gv - 1, tau / kLag);
    const int num = s0 + tau * b + 2 - n, den = kLag * b - 1;
    const int ifst = num <= 0 ? 0 : (num + den - 1) / den;
    if (ifst <= ils) {
        active = true;
        lo = s0 + ils + (tau - kLag * ils) * b + 1;
        hi = min(s0 + ifst + (tau - kLag * ifst + 2) * b, n - 1);
    }
    if (ils + 1 < gv) {
        active = true;
        lo = min(lo, s0 + ils + 2);
    }
}

// One element global -> shared without a register round trip (LDGSTS): every copy a
// lane issues is in flight at once; cp_async_wait_all() completes the lane's copies.
template <typename T>
NLA_DEV void cp_async_elem(T *dst_smem, const T *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
                 "l"(src), "n"((int)sizeof(T))
                 : "memory");
}
NLA_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Mover warp: copy band columns j0..j1 (3b+1 storage rows each) between global
// memory and the window.  With the compact layout (ldab = 3b+1) the columns are
// one contiguous run in global memory: lanes walk it element by element (coalesced);
// otherwise column by column.  Loads are asynchronous copies that all issue before
// the one wait (a single memory latency per call); write-backs keep eight loads from
// the window in flight before their stores.
template <typename T, bool LOAD, int B>
NLA_DEV void mover_copy(const Win<T> &W, const Band<T> &A, int n, int b, int j0, int j1, int lane) {
    const int h = 3 * b + 1;
    if (LOAD) {
        if (B > 0 && A.ldab == (long)(3 * B + 1)) {
            constexpr int H = 3 * B + 1;
            const T *g = A.AB + (long)j0 * H;
            const int tot = (j1 - j0 + 1) * H;
            const int sl0 = j0 % W.wc;
            for (int e = lane; e < tot; e += 32) {
                int sl = sl0 + e / H;
                sl -= sl >= W.wc ? W.wc : 0;
                cp_async_elem(W.w + (size_t)sl * W.ldw + (e % H), g + e);
            }
        } else {
            for (int j = j0; j <= j1; ++j) {
                T *cw = W.col(j);
                for (int q = lane; q < h; q += 32) {
                    const int i = j + q - 2 * b;
                    if (i >= 0 && i < n) cp_async_elem(cw + i, A.at(i, j));
                }
            }
        }
        cp_async_wait_all();
        return;
    }
    if (B > 0 && A.ldab == (long)(3 * B + 1)) {
        constexpr int H = 3 * B + 1;
        T *g = A.AB + (long)j0 * H;
        const int tot = (j1 - j0 + 1) * H;
        const int sl0 = j0 % W.wc;
        for (int base = 0; base < tot; base += 32 * 8) {
            T r[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = base + u * 32 + lane;
                if (e < tot) {
                    int sl = sl0 + e / H;
                    sl -= sl >= W.wc ? W.wc : 0;
                    r[u] = W.w[(size_t)sl * W.ldw + (e % H)];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = base + u * 32 + lane;
                if (e < tot) __stcg(g + e, r[u]);
            }
        }
        return;
    }
    for (int j = j0; j <= j1; ++j) {
        const T *cw = W.col(j);
        for (int q = lane; q < h; q += 32) {
            const int i = j + q - 2 * b;
            if (i >= 0 && i < n) __stcg(A.at(i, j), cw[i]);
        }
    }
}

// Bounded spin of a chase warp on the window's "loaded up to" column.
NLA_DEV bool wait_loaded(volatile int *sh_hi, int hi, volatile int *sh_abort, int *info) {
    if (*sh_hi >= hi) return true;
    const unsigned long long t0 = global_ns();
    while (*sh_hi < hi) {
        __nanosleep(40);  // leave the issue slots to the mover warp
        if (*sh_abort) return false;
        if (global_ns() - t0 > kSpinBudgetNs) {
            if (info) atomicExch(info, kInfoTimeout);
            *sh_abort = 1;
            return false;
        }
    }
    return true;
}

// Block = G chase warps + a flusher warp (warp G) + a loader warp (warp G+1).
// The chase warps run the group's sweeps on the window in lockstep (named
// barrier 1 after each half-step) and never touch global memory.  The flusher
// writes back columns the group will not touch again and announces them in
// done[group]; the loader brings in, up to `pf` steps ahead, the columns the
// previous group has released.  The window holds columns [flushed + 1, loaded]
// in wc >= (2G - 1) b + G + 1 + pf b circular slots.
template <typename T, int B>
__global__ void band2bd_group_kernel(T *AB, long ldab, int n, int b, int G, int wc, int pf, int *done, int *info) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // chase progress, loaded-up-to column, flushed-up-to column, loader finished, abort flag
    __shared__ int sh_tau, sh_hi, sh_fl, sh_ldone, sh_abort;
    const int ldw = (3 * b + 2) & ~1;  // even: lanes walking a row hit distinct banks
    Win<T> W{reinterpret_cast<T *>(smem_raw), ldw, wc, 2 * b};
    T *vbase = W.w + (size_t)wc * ldw;  // 64 entries per chase warp
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    Band<T> A{AB, ldab, 2 * b};
    const int nsweeps = n - 2;
    const int ngroups = (nsweeps + G - 1) / G;
    volatile int *vtau = &sh_tau, *vhi = &sh_hi, *vfl = &sh_fl, *vldone = &sh_ldone, *vabort = &sh_abort;
    if (tid == 0) sh_abort = 0;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int s0 = grp * G, g = min(G, nsweeps - s0);
        int lo0, hi0;
        bool act0;
        group_need(n, b, s0, g, 0, lo0, hi0, act0);
        if (tid == 0) {
            sh_tau = 0;
            sh_hi = lo0 - 1;
            sh_fl = lo0 - 1;
            sh_ldone = 0;
        }
        __syncthreads();
        if (*vabort) break;
        if (warp < G) {
            // ---------------- chase warps
            T *v = vbase + warp * 64;
            int wslot = 0;  // window slot of this warp's current c0 (advanced by b per step)
            // the loaded-up-to column this warp last observed (and fenced after): columns up
            // to it are in the window and stay there while any sweep of the group needs them
            int seen = -1;
            for (int tau = 0;; ++tau) {
                int lo, hi;
                bool active;
                group_need(n, b, s0, g, tau, lo, hi, active);
                if (!active) break;
                const int s = s0 + warp, k = tau - kLag * warp;
                const bool mine = warp < g && k >= 0 && s + k * b + 1 <= n - 1;  // this warp steps now
                bool ok = true;
                const int need = min(s + (k + 2) * b, n - 1);  // last column of this warp's footprint
                if (mine && need > seen) {  // not yet observed loaded: wait for it
                    int hv = 0;
                    if (lane == 0) {
                        ok = wait_loaded(vhi, need, vabort, info);
                        hv = *vhi;
                    }
                    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                    hv = __shfl_sync(0xffffffffu, hv, 0);
                    __threadfence_block();
                    if (ok) seen = hv;
                }
                if (ok && mine) {
                    {
                        if (k == 0) {
                            wslot = (s + 1) % wc;
                        } else {
                            wslot += b;
                            if (wslot >= wc) wslot -= wc;
                        }
                        warp_chase_step<T, B>(W, n, b, s, k, wslot, v, 0);  // right reflector
                    }
                }
                // the right reflectors of this step all precede every left reflector:
                // with sweeps two steps apart that is the order the sequential chase needs
                asm volatile("bar.sync 1, %0;" ::"r"(32 * G) : "memory");
                if (ok && mine) warp_chase_step<T, B>(W, n, b, s, k, wslot, v, 1);  // left reflector
                asm volatile("bar.sync 1, %0;" ::"r"(32 * G) : "memory");
                if (*vabort) break;
                if (warp == 0 && lane == 0) {
                    __threadfence_block();
                    *vtau = tau + 1;
                }
            }
        } else if (warp == G) {
            // ---------------- flusher
            int flushed = lo0 - 1;
            unsigned idle = 32;  // backoff while there is nothing to write back
            for (;;) {
                if (*vabort) break;
                const int t = *vtau;  // steps < t are complete
                __threadfence_block();
                int lo, hi;
                bool active;
                group_need(n, b, s0, g, t, lo, hi, active);
                if (!active) {  // the group is done: every loaded column is final
                    if (lane == 0) {
                        const unsigned long long t0 = global_ns();
                        while (!*vldone && !*vabort) {
                            __nanosleep(64);
                            if (global_ns() - t0 > kSpinBudgetNs) {
                                if (info) atomicExch(info, kInfoTimeout);
                                *vabort = 1;
                            }
                        }
                    }
                    __syncwarp();
                    __threadfence_block();
                    if (*vabort) break;
                    const int fin = *vhi;
                    if (fin > flushed) mover_copy<T, false, B>(W, A, n, b, flushed + 1, fin, lane);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) st_release(&done[grp], INT_MAX);
                    break;
                }
                const int fin = lo - 1;  // columns <= fin are final
                if (fin > flushed) {
                    mover_copy<T, false, B>(W, A, n, b, flushed + 1, fin, lane);
                    flushed = fin;
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) {
                        st_release(&done[grp], flushed + 1);
                        *vfl = flushed;  // the loader may reuse these slots now
                    }
                    idle = 32;
                } else {
                    __nanosleep(idle);
                    idle = min(idle * 2, 64u);
                }
            }
        } else {
            // ---------------- loader
            int loaded = lo0 - 1;
            int have = grp > 0 ? 0 : INT_MAX;  // columns < have are final in the previous group
            unsigned idle = 32;  // backoff while nothing new can be loaded
            for (;;) {
                if (*vabort) break;
                const int t = *vtau;
                __threadfence_block();
                int lo, hi;
                bool active;
                group_need(n, b, s0, g, t, lo, hi, active);
                if (!active) break;
                // the columns steps t .. t + pf need, within the window's capacity
                int lt, want;
                bool at;
                group_need(n, b, s0, g, t + pf, lt, want, at);
                want = max(want, hi);
                want = min(want, *vfl + wc);
                __threadfence_block();
                bool worked = false;
                if (want > loaded) {
                    if (have - 1 < want) {  // (never for group 0)
                        if (hi > loaded && have < hi + 1) {
                            // the current step cannot start without its columns: wait for those
                            if (lane == 0 && !spin_until_geq(&done[grp - 1], hi + 1, info, 64)) *vabort = 1;
                            __syncwarp();
                            if (*vabort) break;
                        }
                        // every lane acquires, so that its own copies below see what the previous
                        // group wrote; the smallest value seen is final for all of them
                        have = __reduce_min_sync(0xffffffffu, ld_acquire(&done[grp - 1]));
                    }
                    const int avail = min(want, have - 1);
                    if (avail > loaded) {
                        mover_copy<T, true, B>(W, A, n, b, loaded + 1, avail, lane);
                        loaded = avail;
                        __syncwarp();
                        __threadfence_block();
                        if (lane == 0) *vhi = loaded;
                        worked = true;
                    }
                }
                if (worked) {
                    idle = 32;
                } else {
                    __nanosleep(idle);
                    idle = min(idle * 2, 64u);
                }
            }
            __syncwarp();
            __threadfence_block();
            if (lane == 0) *vldone = 1;
        }
        __syncthreads();
    }
}

// Sweeps per block group and prefetch depth that fit the shared-memory window
// (G = 0: none fits).
static int chase_group_size(int b, int elem, size_t budget, int gmax, int &pf) {
    const size_t ldw = (size_t)((3 * b + 2) & ~1);
    for (int G = gmax; G >= 1; --G)
        for (int p : {4, 2, 1}) {
            const size_t wc = (size_t)(kLag * G - 1) * b + G + 1 + (size_t)p * b;
            if (wc * ldw * elem + (size_t)G * 64 * elem <= budget) {
                pf = p;
                return G;
            }
        }
    pf = 0;
    return 0;
}

template <typename T>
__global__ void bidiag_extract_kernel(const T *__restrict__ AB, long ldab, int n, int b, double *d, double *e) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        d[i] = (double)AB[2 * b + (long)i * ldab];
        if (i + 1 < n) e[i] = (double)AB[(2 * b - 1) + (long)(i + 1) * ldab];
    }
}

template <typename T>
cudaError_t band2bd(T *AB, long ldab, int n, int b, double *d, double *e, void *scratch, int *info,
                    cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int *progress = reinterpret_cast<int *>(scratch);
    const int nsweeps = n - 2;
    const size_t kGroupBudget = 200 * 1024;
    // Sweeps per block: FP32 up to 16 (the occupancy check below lowers it to what one
    // SM holds), FP64 4 -- an FP64 block step is bound by the SM's small FP64 pipe, so
    // more sweeps per SM slow every step down (measured at n = 256, 2048 and 8192).
    // NLA_CHASE_GROUP overrides it (0: one sweep per block on the global band).
    static const int gset = [] {
        const char *v = getenv("NLA_CHASE_GROUP");
        return v ? atoi(v) : (sizeof(T) == 8 ? 4 : 16);
    }();
    auto kern = b == 16 ? band2bd_group_kernel<T, 16>
                : b == 32 ? band2bd_group_kernel<T, 32>
                : b == 64 ? band2bd_group_kernel<T, 64> : band2bd_group_kernel<T, 0>;
    static PerDeviceOnce gattr;
    gattr.run([&] {
        for (auto k : {band2bd_group_kernel<T, 0>, band2bd_group_kernel<T, 16>, band2bd_group_kernel<T, 32>,
                       band2bd_group_kernel<T, 64>})
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGroupBudget);
        cudaGetLastError();
    });
    // the largest G (<= the requested one) whose block -- G chase warps + 2 movers, its
    // window -- is resident on every SM (registers, shared memory), cached per device and
    // band width (16, 32, 64; other widths are asked every call)
    auto pick_group = [&](int &G, int &pf) {
        G = 0;
        pf = 0;
        for (int gmax = std::min(gset, 30); gmax >= 1; --gmax) {
            int p2 = 0;
            const int g2 = chase_group_size(b, (int)sizeof(T), kGroupBudget, gmax, p2);
            if (g2 < 1) break;
            const int wc2 = (kLag * g2 - 1) * b + g2 + 1 + p2 * b;
            const size_t sm2 = (size_t)wc2 * ((3 * b + 2) & ~1) * sizeof(T) + (size_t)g2 * 64 * sizeof(T);
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 32 * (g2 + 2), sm2) == cudaSuccess && nb >= 1) {
                G = g2;
                pf = p2;
                break;
            }
            cudaGetLastError();
            gmax = std::min(gmax, g2);
        }
    };
    static PerDeviceValue<int2> gcache[4];
    const int ci = b == 16 ? 1 : b == 32 ? 2 : b == 64 ? 3 : 0;
    int G = 0, pf = 0;
    if (gset > 0 && ci > 0) {
        const int2 gp = gcache[ci].get([&] {
            int g = 0, p = 0;
            pick_group(g, p);
            return make_int2(g, p);
        });
        G = gp.x;
        pf = gp.y;
    } else if (gset > 0) {
        pick_group(G, pf);
    }
    if (nsweeps > 0 && b > 1 && G >= 1) {
        const int ngroups = (nsweeps + G - 1) / G;
        cudaError_t err = cudaMemsetAsync(progress, 0, sizeof(int) * (size_t)ngroups, st);
        if (err != cudaSuccess) return err;
        const int wc = (kLag * G - 1) * b + G + 1 + pf * b;
        const size_t smem = (size_t)wc * ((3 * b + 2) & ~1) * sizeof(T) + (size_t)G * 64 * sizeof(T);
        const int grid = std::min(ngroups, device_sm_count());
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(32 * (G + 2));
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        err = cudaLaunchKernelEx(&cfg, kern, AB, ldab, n, b, G, wc, pf, progress, info);
        if (err != cudaSuccess) return err;
    } else if (nsweeps > 0 && b > 1) {
        cudaError_t err = cudaMemsetAsync(progress, 0, sizeof(int) * (size_t)nsweeps, st);
        if (err != cudaSuccess) return err;
        static PerDeviceOnce smem_attr;
        smem_attr.run([] {
            cudaFuncSetAttribute(band2bd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(((size_t)129 * 128 + 64 + 8) * sizeof(T)));
            cudaGetLastError();
        });
        int grid = std::min(nsweeps, device_sm_count());
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kChaseThreads);
        cfg.dynamicSmemBytes = ((size_t)(2 * b + 1) * 2 * b + 64 + 8) * sizeof(T);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        err = cudaLaunchKernelEx(&cfg, band2bd_kernel<T>, AB, ldab, n, b, progress, info);
        if (err != cudaSuccess) return err;
    }
    bidiag_extract_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(AB, ldab, n, b, d, e);
    return cudaGetLastError();
}

#define NLA_INST(T)                                                                                       \
    template cudaError_t copy_matrix<T>(const T *, long, int, int, T *, long, bool, cudaStream_t);      \
    template cudaError_t band_extract<T>(const T *, long, int, int, T *, long, cudaStream_t);           \
    template cudaError_t band2bd<T>(T *, long, int, int, double *, double *, void *, int *, cudaStream_t);
NLA_INST(double)
NLA_INST(float)
#undef NLA_INST

}  // namespace nla
