// bdsvd.cu -- stage 3: singular values of the upper bidiagonal B(d, e).
//
// Section 5.1.1 ends the reduction at "diagonal form"; here the bidiagonal's
// singular values are found by bisection, which is data-parallel (one thread
// per singular value) where QR iteration is sequential.  The eigenvalues of
// the 2n x 2n Golub-Kahan tridiagonal TGK (zero diagonal, off-diagonals
// d_0, e_0, d_1, e_1, ..., d_{n-1}) are +-sigma_i, so for x > 0 the number of
// singular values below x is negcount(TGK - x I) - n, where negcount counts
// the negative pivots of the LDL^T factorisation of TGK - x I (Sylvester's law
// of inertia): q_1 = -x, q_i = -x - t_{i-1}^2 / q_{i-1}.  A pivot that is
// exactly zero is replaced by -pivmin.  All arithmetic is FP64.
//
// Thread i brackets the i-th largest value in [lo, hi] starting from
// [0, max_i(|d_i| + max(|e_{i-1}|, |e_i|))] (Gershgorin on TGK) and halves the
// bracket until its width is below the resolution of the output type
// relative to that bound (2^-52 for FP64 output, 2^-27 for FP32 output).
#include <cfloat>

#include "common.cuh"
#include "kernels.cuh"

namespace nla {

constexpr int kBisectThreads = 128;

NLA_DEV int count_below(int n, const double *__restrict__ d, const double *__restrict__ e, double x,
                        double pivmin) {
    double q = -x;
    int neg = q < 0.0;
    for (int i = 0; i < n; ++i) {
        if (fabs(q) < pivmin) q = -pivmin;
        double di = __ldg(d + i);
        q = -x - (di * di) / q;
        neg += q < 0.0;
        if (i + 1 < n) {
            if (fabs(q) < pivmin) q = -pivmin;
            double ei = __ldg(e + i);
            q = -x - (ei * ei) / q;
            neg += q < 0.0;
        }
    }
    return neg - n;
}

template <typename T>
__global__ void __launch_bounds__(kBisectThreads)
bisect_kernel(int n, const double *__restrict__ d, const double *__restrict__ e, T *__restrict__ S,
              double rel_tol) {
    __shared__ double sh_bound, sh_tmax;
    // Gershgorin bound and the largest squared off-diagonal, per block
    double bnd = 0.0, tmax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double di = fabs(d[i]);
        double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i + 1 < n ? fabs(e[i]) : 0.0;
        bnd = fmax(bnd, di + fmax(el, er));
        tmax = fmax(tmax, fmax(di, er));
    }
    bnd = warp_max(bnd);
    tmax = warp_max(tmax);
    __shared__ double wb[32], wt[32];
    if ((threadIdx.x & 31) == 0) {
        wb[threadIdx.x >> 5] = bnd;
        wt[threadIdx.x >> 5] = tmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0, t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            b = fmax(b, wb[w]);
            t = fmax(t, wt[w]);
        }
        sh_bound = b;
        sh_tmax = t;
    }
    __syncthreads();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const double bound = sh_bound * (1.0 + 4.0 * DBL_EPSILON) + DBL_MIN;
    const double pivmin = DBL_MIN * fmax(1.0, sh_tmax * sh_tmax);
    const double tol = rel_tol * bound;
    const int j = n - 1 - idx;  // idx-th largest == j-th smallest
    double lo = 0.0, hi = bound;
    for (int it = 0; it < 128; ++it) {
        double mid = 0.5 * (lo + hi);
        if (hi - lo <= tol || mid <= lo || mid >= hi) break;
        if (count_below(n, d, e, mid, pivmin) <= j)
            lo = mid;
        else
            hi = mid;
    }
    S[idx] = (T)(0.5 * (lo + hi));
}

template <typename T>
cudaError_t bdsvd_bisect(int n, const double *d, const double *e, T *S, int *info, cudaStream_t st) {
    (void)info;
    if (n <= 0) return cudaSuccess;
    const double rel_tol = sizeof(T) == 8 ? 2.0 * DBL_EPSILON : 0x1p-27;
    bisect_kernel<T><<<(n + kBisectThreads - 1) / kBisectThreads, kBisectThreads, 0, st>>>(n, d, e, S, rel_tol);
    return cudaGetLastError();
}

template cudaError_t bdsvd_bisect<double>(int, const double *, const double *, double *, int *, cudaStream_t);
template cudaError_t bdsvd_bisect<float>(int, const double *, const double *, float *, int *, cudaStream_t);

}  // namespace nla
