/*
 * nla.h -- singular values of dense real matrices on one GB300 (sm_103a).
 *
 * The library computes the singular values of a dense m x n matrix by the
 * two-stage reduction of the paper's Section 5.1.1 (Fig. 3, Algorithm 1):
 *   stage 1  dense -> upper band of width b by tiled Householder QR / LQ panels
 *            (GEQRT/TSQRT-style panel factorisation, Algorithm 1 steps
 *            "QR sweep" / "LQ sweep") and a blocked trailing update
 *            (UNMQR/TSMQR, Algorithm 2);
 *   stage 2  band -> bidiagonal by bulge chasing (Section 5.1.1, Fig. 3);
 *   stage 3  bidiagonal -> singular values (Section 5.1.1: "finally to ...
 *            diagonal form"), here by Sturm-count bisection.
 * Every step keeps the singular values intact because it applies orthogonal
 * transformations only (Section 5.1.1).
 *
 * Conventions shared by every call:
 *   - Pointers named d* are DEVICE pointers owned by the caller; pointers named
 *     h* are host pointers.  The library never allocates device memory on
 *     these paths: scratch comes from the caller's workspace (dWork).
 *   - Matrices are column-major with leading dimension lda >= rows.  A
 *     row-major PyTorch tensor of shape (r, c) passed as-is is the column-major
 *     c x r matrix A^T, which has the same singular values.
 *   - All work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and the call returns without synchronising.
 *   - Argument errors are returned synchronously and nothing is enqueued.
 *     Device-side outcomes go to the int pointed to by dInfo after the stream
 *     completes: 0 = success, > 0 = number of values that did not converge,
 *     < 0 = -(nla_status) of a device-side failure (e.g. -NLA_ERR_TIMEOUT when
 *     a bounded inter-block wait gave up; the results are then undefined but
 *     the context stays usable).
 *   - m == 0 or n == 0 is a successful no-op.
 *   - NaN or Inf entries give undefined singular values; no error is promised.
 *   - nla_last_error() returns a thread-local message for the last non-OK
 *     status returned on the calling thread.
 */
#ifndef NLA_H
#define NLA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *nla_stream_t; /* a cudaStream_t */

typedef enum {
    NLA_OK = 0,
    NLA_ERR_ARG = 1,         /* invalid argument */
    NLA_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in nla_last_error) */
    NLA_ERR_CONFIG = 3,      /* the launch configuration is not valid for this problem */
    NLA_ERR_WORKSPACE = 4,   /* workspace too small or misaligned */
    NLA_ERR_TIMEOUT = 5,     /* a bounded inter-block wait gave up (device side) */
    NLA_ERR_NOCONV = 6,      /* an iteration hit its cap */
    NLA_ERR_UNSUPPORTED = 7  /* problem outside the sizes this build supports */
} nla_status;

typedef enum { NLA_F64 = 0, NLA_F32 = 1 } nla_dtype;

/* Operand precision of the trailing update (Algorithm 2).  NATIVE computes in
 * the matrix dtype.  TF32 / BF16 round the (power-of-two column-scaled)
 * operands to that type and run the contraction on the tensor cores with FP32
 * accumulation; the matrix itself stays in its dtype, and panel
 * factorisation, bulge chasing and the singular-value solve are unchanged.
 * TF32X3 / BF16X3 are the compensated forms: each operand is split into a
 * rounded high part and a rounded remainder and every product is formed from
 * three tensor-core products (hi*hi + hi*lo + lo*hi), which keeps about twice
 * the operand type's precision at three times the tensor-core work (the
 * contraction is memory-bound either way).  All four need an FP64 matrix. */
typedef enum {
    NLA_UPD_NATIVE = 0,
    NLA_UPD_TF32 = 1,
    NLA_UPD_BF16 = 2,
    NLA_UPD_TF32X3 = 3,
    NLA_UPD_BF16X3 = 4
} nla_update;

/* Launch configuration of the trailing-update kernels (Algorithm 2's tunable
 * parameters, Section 5.2 search-space table, re-expressed for this GPU):
 *   band            b  : band width = panel width (the pipeline parameter);
 *   tile            th : rows (QR side) / columns (LQ side) of X staged per step;
 *   threads            : threads per block (multiple of 32, <= 1024);
 *   cols_per_block  cpb: the block owns 32*cpb columns (QR side) or rows (LQ
 *                        side) of the trailing matrix;
 *   unroll          u  : unroll factor of the reduction loop over the staged tile.
 * A field <= 0 means "use the tuned or default value". */
typedef struct {
    int band;
    int tile;
    int threads;
    int cols_per_block;
    int unroll;
} nla_cfg;

typedef struct {
    nla_update update;  /* trailing-update operand precision */
    const nla_cfg *cfg; /* NULL = tuned table (kt_load_config) else defaults */
    int preserve_a;     /* nonzero: A is copied to the workspace and left intact */
} nla_opts;

/* ---------------------------------------------------------------- whole SVD */

/* Workspace bytes needed by nla_gesvd_vals for this problem and options.
 * Returns NLA_ERR_CONFIG (and sets no size) when opts->cfg names trailing-update
 * parameters that are not a valid launch configuration for the band used --
 * the same check nla_gesvd_vals makes before enqueuing anything. */
nla_status nla_gesvd_vals_workspace(int m, int n, nla_dtype dtype, const nla_opts *opts,
                                    size_t *bytes);

/* Singular values of the column-major m x n matrix dA (dtype elements, lda >= m)
 * by the whole two-stage method (Section 5.1.1, Fig. 3; Algorithm 1 for stage 1,
 * Algorithm 2 for its trailing updates).
 * dS receives min(m, n) values in descending order, in dtype.  dA is
 * overwritten unless opts->preserve_a (or m < n, where A^T is formed in the
 * workspace and dA is left intact).  dWork: >= nla_gesvd_vals_workspace bytes,
 * 256-byte aligned.  dInfo: one device int (see conventions). */
nla_status nla_gesvd_vals(int m, int n, nla_dtype dtype, void *dA, int lda, void *dS,
                          void *dWork, size_t work_bytes, int *dInfo,
                          const nla_opts *opts, nla_stream_t stream);

/* Batched singular values of `batch` independent FP32 matrices of uneven
 * shapes in one call (the batched form of the method of Section 5.1.1): a sort
 * kernel, a kernel for the matrices above 48K elements (one per block, several
 * blocks per SM, global scratch) and a persistent kernel for the rest (shared
 * memory).  dM, dN, dLda: DEVICE int arrays of shapes and leading dimensions;
 * dA_array / dS_array: DEVICE arrays of device pointers; matrix i is column
 * major m_i x n_i and is read, not modified; dS_array[i] receives
 * min(m_i, n_i) values, descending.  max_m, max_n bound every m_i, n_i
 * (min(max_m, max_n) <= 256).  dInfo: `batch` device ints (0 = success,
 * -NLA_ERR_UNSUPPORTED for a matrix the kernel cannot hold).  Matrices are
 * ordered by size on the device and reduced by groups of threads whose size
 * per size bucket comes from the tuned table (kt_load_config) or defaults.
 * Nothing is read from the host at run time, so the call can be captured in
 * a CUDA graph and replayed.  Only NLA_F32 is supported.  The workspace holds
 * the sort keys and one max_m x max_n scratch slot per block of the large-
 * matrix kernel (4 per SM). */
nla_status nla_gesvd_vals_batched_workspace(int batch, nla_dtype dtype, int max_m, int max_n,
                                            size_t *bytes);
nla_status nla_gesvd_vals_batched(int batch, nla_dtype dtype, const int *dM, const int *dN,
                                  const int *dLda, void *const *dA_array, void *const *dS_array,
                                  int max_m, int max_n, void *dWork, size_t work_bytes, int *dInfo,
                                  const nla_opts *opts, nla_stream_t stream);

/* The launch configuration nla_gesvd_vals would use for this problem (after
 * opts->cfg overrides, the tuned table and the defaults, and the adjustment
 * to the band width actually used); side 0 = QR-side update, 1 = LQ side. */
nla_status nla_plan_cfg(int m, int n, nla_dtype dtype, const nla_opts *opts, int side, nla_cfg *out);

/* ---------------------------------------------------------------- stages */

/* Stage 1 (Algorithm 1): reduce the column-major m x n matrix dA (m >= n) to
 * upper band form of width `band` in place.  On return the band
 * (entries with 0 <= j - i <= band) holds the band matrix; the QR reflectors
 * are stored below the diagonal of each panel column block and the LQ
 * reflectors to the right of the band in each panel row block.  dTauQ, dTauP
 * (dtype, ceil(n/band)*band entries each, may be NULL) receive the reflector
 * scalars tau.  Returns NLA_ERR_ARG if m < n. */
nla_status nla_gebrd_band_workspace(int m, int n, int band, nla_dtype dtype,
                                    const nla_opts *opts, size_t *bytes);
nla_status nla_gebrd_band(int m, int n, int band, nla_dtype dtype, void *dA, int lda,
                          void *dTauQ, void *dTauP, void *dWork, size_t work_bytes,
                          int *dInfo, const nla_opts *opts, nla_stream_t stream);

/* Copy the upper band (0 <= j - i <= band) of the column-major n x n matrix dA
 * into compact band storage dAB (dtype, ldab >= 3*band + 1): entry (i, j)
 * with -band <= j - i <= 2*band lives at dAB[(2*band + i - j) + j*ldab]; rows
 * outside the upper band are zeroed (room for the bulges of stage 2). */
nla_status nla_band_extract(int n, int band, nla_dtype dtype, const void *dA, int lda,
                            void *dAB, int ldab, nla_stream_t stream);

/* Stage 2 (Section 5.1.1, Fig. 3: band to bidiagonal): reduce the upper band
 * matrix in dAB (layout of nla_band_extract, overwritten) to upper bidiagonal
 * form by Householder bulge chasing; dD (n) and dE (n-1) receive the FP64
 * diagonal and superdiagonal.  dWork: >= nla_band2bd_workspace bytes (the
 * sweeps' progress counters; the library allocates nothing on this path). */
nla_status nla_band2bd_workspace(int n, int band, nla_dtype dtype, size_t *bytes);
nla_status nla_band2bd(int n, int band, nla_dtype dtype, void *dAB, int ldab, double *dD,
                       double *dE, void *dWork, size_t work_bytes, int *dInfo,
                       const nla_opts *opts, nla_stream_t stream);

/* nla_band2bd without a workspace, for callers that cannot allocate device
 * memory: a plug-in running inside a host framework whose memory manager owns
 * the whole device and forbids allocations outside it, code that must never
 * synchronise the device (cudaMalloc and cudaFree may), and programs with a
 * fixed device-memory budget set at start-up.  The paper has no counterpart;
 * this is a library convenience.  Same arguments, layout and results as
 * nla_band2bd, but the sweep-progress scratch is a fixed array inside the
 * library (65536 ints = 256 KiB per GPU that loads the library, held until the
 * process exits), so n may not exceed 65536 (NLA_ERR_UNSUPPORTED otherwise).
 * It allocates nothing: the first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current -- make that first
 * call before any stream capture.  Every call clears the counters it uses on
 * its stream; all calls share the one array, so calls that could overlap on
 * the GPU (unordered streams) race and must not be issued. */
nla_status nla_band2bd_noalloc(int n, int band, nla_dtype dtype, void *dAB, int ldab, double *dD,
                               double *dE, int *dInfo, nla_stream_t stream);

/* Stage 3 (Section 5.1.1: bidiagonal to diagonal form, i.e. the singular
 * values): singular values of the upper bidiagonal (dD, dE) by bisection on
 * Sturm counts of the Golub-Kahan tridiagonal (coarse steps with FP32 counts,
 * final steps with FP64 counts); dS receives n values descending, converted to
 * dtype, accurate to the output type's resolution of the bidiagonal's
 * Gershgorin bound.  dWork: >= nla_bdsvd_vals_workspace bytes, 256-aligned. */
nla_status nla_bdsvd_vals_workspace(int n, size_t *bytes);
nla_status nla_bdsvd_vals(int n, const double *dD, const double *dE, void *dS, nla_dtype dtype,
                          void *dWork, size_t work_bytes, int *dInfo, nla_stream_t stream);

/* ---------------------------------------------------------------- tracing */

/* Per-kernel-class timing (the tuner's timing observer, paper Section 4.2,
 * made available to callers).  While enabled, every kernel the library
 * launches is bracketed by a pair of CUDA events recorded on the launching
 * stream; nla_trace_read synchronises those events and returns, per kernel
 * class, the number of launches and their summed device time.  Classes:
 * "panel_qr", "panel_lq", "trail_left", "trail_right", "stage_copy",
 * "band_extract", "band2bd", "bisect", "batched".  Tracing adds two event
 * records per launch; it is off by default. */
typedef struct {
    const char *name;   /* static string owned by the library */
    int launches;
    double total_ms;
} nla_trace_entry;
nla_status nla_trace_enable(int on);
/* Fills up to max_entries entries and returns how many classes were seen. */
int nla_trace_read(nla_trace_entry *out, int max_entries);
void nla_trace_reset(void);

/* ---------------------------------------------------------------- diagnostics */

/* One 128 x N x K product D = A B on this GPU's tensor cores, the building
 * block of the TF32 / BF16 trailing update (prec = NLA_UPD_TF32 or
 * NLA_UPD_BF16): dA is 128 x K and dB is K x N, row-major FP32 (rounded to the
 * operand type on the device), dD receives 128 x N row-major FP32.  K a
 * multiple of 16 in [16, 128], N a multiple of 16 in [16, 256].  Lets a caller
 * check the tensor-core path of its device in isolation. */
nla_status nla_tc_selftest(int prec, int K, int N, const float *dA, const float *dB, float *dD,
                           int *dInfo, nla_stream_t stream);

/* The two exact power-of-two conversions of the TF32 / BF16 trailing update's
 * scaling step (the "column scaling" of the mixed-precision form), element by
 * element, so a caller can check them on edge values: for i < n,
 *   dF[i] = dX[i] * 2^-dEx[i] as FP32, its significand truncated to FP32's 24
 *           bits; 0 (signed) below FP32's normal range, +-inf at or above 2^128
 *           (FP64 subnormal inputs read as 0);
 *   dD[i] = dV[i] * 2^dEv[i] as FP64 (exact); 0 for FP32 zeros and subnormals,
 *           a signed 0 below FP64's normal range, +-inf above it.
 * All pointers are device arrays of n entries.  Asynchronous on `stream`. */
nla_status nla_scale_selftest(int n, const double *dX, const int *dEx, float *dF, const float *dV,
                              const int *dEv, double *dD, nla_stream_t stream);

/* Pipe microbenchmarks (no counterpart in the paper): the peaks the kernels'
 * rooflines are measured against.  kind 0: FP32 FMA (blocks x 256 threads, 8
 * independent chains of `iters` FMAs per thread: 2 * 8 * iters flops a thread);
 * kind 1: the same with FP64 FMAs; kind 2: tensor cores, kind::tf32 (one block
 * of 128 threads per entry of `blocks`, one thread issuing `iters` MMAs of
 * 128 x 256 x 8: 524288 flops each; launch at most one block per SM).  dOut:
 * a device buffer of blocks * 256 elements of the kind's type (never written in
 * practice); dInfo: device int (-NLA_ERR_TIMEOUT if a wait gave up).  The caller
 * times the launch on `stream` (CUDA events). */
nla_status nla_pipe_selftest(int kind, int blocks, int iters, void *dOut, int *dInfo, nla_stream_t stream);

/* Failure-detection self-test (no counterpart in the paper): one block waits,
 * with a budget of budget_us microseconds, on something that never happens --
 * mode 0: a global flag that nothing sets (the inter-block spin every
 * cooperative kernel of the library uses); mode 1: an mbarrier phase that never
 * completes (the stage barriers of the TMA / tensor-core kernels).  The wait
 * gives up, the kernel writes -NLA_ERR_TIMEOUT to *dInfo and returns, and the
 * context stays usable.  budget_us in [1, 2000000]; returns NLA_ERR_ARG
 * otherwise.  Asynchronous on `stream`. */
nla_status nla_wait_selftest(int mode, int budget_us, int *dInfo, nla_stream_t stream);

/* Message for the last non-OK status returned on this thread. */
const char *nla_last_error(void);

/* Library version string. */
const char *nla_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NLA_H */
