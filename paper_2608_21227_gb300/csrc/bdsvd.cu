// bdsvd.cu -- stage 3: singular values of the upper bidiagonal B(d, e).
//
// Section 5.1.1 ends the reduction at "diagonal form"; here the bidiagonal's
// singular values are found by bisection, which is data-parallel (one thread
// per singular value) where QR iteration is sequential.  The eigenvalues of
// the 2n x 2n Golub-Kahan tridiagonal TGK (zero diagonal, off-diagonals
// t = d_0, e_0, d_1, e_1, ..., d_{n-1}) are +-sigma_i, so for x > 0 the number
// of singular values below x is negcount(TGK - x I) - n, where negcount counts
// the negative pivots of the LDL^T factorisation of TGK - x I (Sylvester's law
// of inertia): q_1 = -x, q_i = -x - t_{i-1}^2 / q_{i-1}; a pivot smaller than
// pivmin in magnitude is replaced by -pivmin before its sign is counted, so the
// count stays monotone in x.
//
// GB300's FP64 pipe issues a small fraction of the FP32 rate, and an IEEE FP64
// division costs many FP64 issue slots, so the search is split:
//   prep:   B is scaled by a power of two so its Gershgorin bound is <= 1
//           (exact), and the squares t_i^2 are stored once in FP64 and FP32;
//   coarse: multisection with FP32 Sturm counts.  A group of 8 lanes owns one
//           value and counts at 8 interior points of its bracket per round, so
//           a round shrinks the bracket 9-fold where bisection halves it.  An
//           FP32 count is the exact count of a matrix whose entries differ
//           relatively by a few FP32 rounding errors, so it can only misplace
//           values within a few 2^-24 of x (the scaled bound is 1).  For FP32
//           output that is the answer: the reduction before it has the same
//           absolute error level.  For FP64 output the coarse bracket stops at
//           2^-16 and is widened by 2^-18 on both sides, which keeps the value
//           inside it;
//   fine:   (FP64 output) multisection with FP64 counts to 2^-51 of the bound,
//           kl lanes per value (kl = 1, plain bisection, for large n; more lanes
//           when few values would leave most SMs idle).  The FP64 count forms 1/q from an FP32 estimate
//           and two Newton-Raphson corrections r <- r + r (1 - q r) (quadratic
//           convergence: ~2^-22 -> 2^-44 -> below FP64 rounding), i.e. four
//           FMAs instead of a division.
#include <cfloat>

#include "common.cuh"
#include "kernels.cuh"

namespace nla {

constexpr int kBisectThreads = 32;  // fine phase: one warp per block spreads the FP64 work over all SMs
constexpr int kMsLanes = 8;         // points per multisection round (one lane each)
constexpr int kMsThreads = 128;
constexpr double kPivminFine = 0x1p-100;   // pivot floor of the FP64 counts (scaled problem)
constexpr float kPivminCoarse = 0x1p-60f;  // pivot floor of the FP32 counts

size_t bdsvd_scratch_bytes(int n) {
    const size_t m = (size_t)(n > 0 ? 2 * n : 1);
    return 256 + m * sizeof(double) + ((m * sizeof(float) + 255) / 256) * 256 + (size_t)(n > 0 ? n : 1) * 8;
}

// One block: Gershgorin bound, power-of-two scale, squared scaled off-diagonals.
__global__ void bd_prep_kernel(int n, const double *__restrict__ d, const double *__restrict__ e, double *hdr,
                               double *t2, float *t2f) {
    __shared__ double wb[32];
    __shared__ double sh_scale;
    double bnd = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double di = fabs(d[i]);
        double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i + 1 < n ? fabs(e[i]) : 0.0;
        bnd = fmax(bnd, di + fmax(el, er));
    }
    bnd = warp_max(bnd);
    if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = bnd;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, wb[w]);
        int ex = 0;
        if (b > 0.0) frexp(b, &ex);  // b * 2^-ex in [0.5, 1)
        sh_scale = ldexp(1.0, -ex);
        hdr[0] = sh_scale;
        hdr[1] = b;
    }
    __syncthreads();
    const double s = sh_scale;
    for (int i = threadIdx.x; i < 2 * n - 1; i += blockDim.x) {
        double t = (i & 1) ? e[i >> 1] : d[i >> 1];
        t *= s;
        t2[i] = t * t;
        t2f[i] = (float)(t * t);
    }
}

NLA_DEV int count_coarse(int n2, const float *__restrict__ t2f, float x) {
    float q = -x;
    int neg = q < 0.f;
    for (int i = 0; i < n2; ++i) {
        q = -x - __fdividef(__ldg(t2f + i), q);
        if (fabsf(q) < kPivminCoarse) q = -kPivminCoarse;  // floor first, then count the sign used
        neg += q < 0.f;
    }
    return neg;
}

NLA_DEV double recip_nr(double q) {
    double r = (double)__fdividef(1.f, (float)q);  // ~2^-22 relative
    double h = fma(-q, r, 1.0);
    r = fma(r, h, r);  // ~2^-44
    h = fma(-q, r, 1.0);
    return fma(r, h, r);  // FP64 rounding level
}

NLA_DEV int count_fine(int n2, const double *__restrict__ t2, double x) {
    double q = -x;
    int neg = q < 0.0;
    for (int i = 0; i < n2; ++i) {
        q = fma(-__ldg(t2 + i), recip_nr(q), -x);
        if (fabs(q) < kPivminFine) q = -kPivminFine;
        neg += q < 0.0;
    }
    return neg;
}

// Multisection with FP32 counts on [0, 1]: group g of kMsLanes lanes finds the
// g-th largest value.  Invariant: count(lo) - n <= j < count(hi) - n, i.e. the
// j-th smallest value lies in [lo, hi).  Each round every lane counts at its
// own interior point; the bracket becomes the first interval of consecutive
// points over which the count passes j.
template <typename T>
__global__ void __launch_bounds__(kMsThreads)
coarse_kernel(int n, const double *__restrict__ hdr, const float *__restrict__ t2f, float stop,
              float2 *__restrict__ br, T *__restrict__ S) {
    const int idx = (blockIdx.x * blockDim.x + threadIdx.x) / kMsLanes;
    const int l = threadIdx.x % kMsLanes;
    const int gbase = (threadIdx.x & 31) & ~(kMsLanes - 1);
    const unsigned gmask = ((1u << kMsLanes) - 1) << gbase;
    if (idx >= n) return;  // uniform over the group
    const int n2 = 2 * n - 1;
    const int j = n - 1 - idx;
    const float frac = (float)(l + 1) * (1.0f / (kMsLanes + 1));
    float lo = 0.f, hi = 1.f;
    for (int round = 0; round < 64 && hi - lo > stop; ++round) {
        const float x = fmaf(hi - lo, frac, lo);
        const bool below = count_coarse(n2, t2f, x) - n <= j;
        const unsigned m = (__ballot_sync(gmask, below) >> gbase) & ((1u << kMsLanes) - 1);
        const int f = __ffs(~m) - 1;  // first point whose count passes j; kMsLanes if none
        const float xf = __shfl_sync(gmask, x, gbase + min(f, kMsLanes - 1));
        const float xp = __shfl_sync(gmask, x, gbase + max(f - 1, 0));
        if (f < kMsLanes) hi = xf;
        if (f > 0) lo = xp;
    }
    if (l == 0) {
        if (S)
            S[idx] = (T)(0.5 * ((double)lo + (double)hi) / hdr[0]);
        else
            br[idx] = make_float2(lo, hi);
    }
}

// FP64 search from the widened coarse bracket: a group of kl lanes (a power of two,
// kl <= 32) per value counts at kl interior points per round (kl = 1: bisection).
// Few values leave most SMs idle, so the host gives each value more lanes then.
template <typename T>
__global__ void __launch_bounds__(kBisectThreads)
fine_kernel(int n, const double *__restrict__ hdr, const double *__restrict__ t2, const float2 *__restrict__ br,
            T *__restrict__ S, double fine_tol, int kl) {
    const int idx = (blockIdx.x * blockDim.x + threadIdx.x) / kl;
    const int l = threadIdx.x % kl;
    const int gbase = (threadIdx.x & 31) & ~(kl - 1);
    const unsigned gmask = (kl == 32 ? 0xffffffffu : ((1u << kl) - 1)) << gbase;
    if (idx >= n) return;  // uniform over the group
    const double s = hdr[0];
    const int n2 = 2 * n - 1;
    const int j = n - 1 - idx;  // idx-th largest == j-th smallest; counts below x are negcount - n
    const float2 b = br[idx];
    double dlo = fmax(0.0, (double)b.x - 0x1p-18), dhi = fmin(1.0, (double)b.y + 0x1p-18);
    const double frac = (double)(l + 1) / (double)(kl + 1);
    for (int it = 0; it < 80; ++it) {
        const double x = fma(dhi - dlo, frac, dlo);
        // stop at the tolerance or when the points no longer separate (FP64 spacing)
        const bool done = dhi - dlo <= fine_tol || !(x > dlo && x < dhi);
        if (__any_sync(gmask, done)) break;
        const bool below = count_fine(n2, t2, x) - n <= j;
        const unsigned full = gmask >> gbase;
        const unsigned m = (__ballot_sync(gmask, below) >> gbase) & full;
        const int f = m == full ? kl : __ffs(~m) - 1;  // first point whose count passes j; kl if none
        const double xf = __shfl_sync(gmask, x, gbase + min(f, kl - 1));
        const double xp = __shfl_sync(gmask, x, gbase + max(f - 1, 0));
        if (f < kl) dhi = xf;
        if (f > 0) dlo = xp;
    }
    if (l == 0) S[idx] = (T)(0.5 * (dlo + dhi) / s);
}

template <typename T>
cudaError_t bdsvd_bisect(int n, const double *d, const double *e, T *S, void *scratch, int *info, cudaStream_t st) {
    (void)info;
    if (n <= 0) return cudaSuccess;
    char *w = reinterpret_cast<char *>(scratch);
    double *hdr = reinterpret_cast<double *>(w);
    double *t2 = reinterpret_cast<double *>(w + 256);
    float *t2f = reinterpret_cast<float *>(w + 256 + (size_t)2 * n * sizeof(double));
    float2 *br = reinterpret_cast<float2 *>(w + 256 + (size_t)2 * n * sizeof(double) +
                                            (((size_t)2 * n * sizeof(float) + 255) / 256) * 256);
    bd_prep_kernel<<<1, 1024, 0, st>>>(n, d, e, hdr, t2, t2f);
    const int cblocks = (int)(((long)n * kMsLanes + kMsThreads - 1) / kMsThreads);
    if (sizeof(T) == 4) {
        coarse_kernel<T><<<cblocks, kMsThreads, 0, st>>>(n, hdr, t2f, 0x1p-23f, nullptr, S);
        return cudaGetLastError();
    }
    coarse_kernel<T><<<cblocks, kMsThreads, 0, st>>>(n, hdr, t2f, 0x1p-16f, br, nullptr);
    // lanes per value: the largest power of two <= 32 that keeps n * kl / 32 warps
    // within one per SM sub-partition (the FP64 count is bound by that pipe)
    const long slots = 4L * device_sm_count() * 32;
    int kl = 1;
    while (kl < 32 && (long)n * kl * 2 <= slots) kl *= 2;
    const long fthreads = (long)n * kl;
    fine_kernel<T><<<(int)((fthreads + kBisectThreads - 1) / kBisectThreads), kBisectThreads, 0, st>>>(
        n, hdr, t2, br, S, 0x1p-51, kl);
    return cudaGetLastError();
}

template cudaError_t bdsvd_bisect<double>(int, const double *, const double *, double *, void *, int *, cudaStream_t);
template cudaError_t bdsvd_bisect<float>(int, const double *, const double *, float *, void *, int *, cudaStream_t);

}  // namespace nla
