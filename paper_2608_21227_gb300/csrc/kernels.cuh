// kernels.cuh -- launch wrappers for every device kernel of the library.
// Each returns cudaSuccess or the launch error; all work goes on `st`.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace nla {

// ---------------------------------------------------------------- panel
// Householder factorisation of an M x nb panel whose element (r, c) lives at
// P[r*rs + c*cs] (QR panel: rs = 1, cs = lda; LQ panel seen transposed:
// rs = lda, cs = 1).  Reflector tails overwrite the strictly lower part,
// R the upper part; tau (nb) and the compact-WY factor T (nb x nb, column
// major, upper triangular, ld nb) are written in the panel's type.
struct PanelCtl {
    unsigned int *bar;   // 2 counters (barrier, exit); zero before first use
    double *part;        // >= panel_part_doubles(P) doubles of scratch
    int *info;           // device info word (timeout reporting)
};
size_t panel_part_doubles(int P);
int panel_max_ctas();    // cooperative CTAs usable by the panel kernel
template <typename T>
cudaError_t panel_factor(T *P, long rs, long cs, int M, int nb, T *tau, T *Tm,
                         const PanelCtl &ctl, cudaStream_t st);

// ---------------------------------------------------------------- trailing update
struct UpdCfg {
    int tile, threads, cpb, unroll;
};
// Scratch of the register-tiled update: partial sums and W' / Y'
// (tiled_scratch_elems elements of the matrix type) and one ticket counter per
// strip (tiled_tickets; zero before the first launch, left zero after each).
struct UpdScratch {
    void *work;
    unsigned int *tickets;
    int *info = nullptr;  // device info word: a bounded wait that gives up records a timeout here
};
size_t tiled_scratch_elems(int M, int N);
size_t tiled_tickets(int M, int N);
// Validity of a configuration for the SIMT trailing-update kernels
// (side 0 = QR/left, 1 = LQ/right); elem = bytes per element.
bool upd_cfg_valid(int side, int elem, int nb, const UpdCfg &c, size_t *smem_bytes);
// upd_cfg_valid plus the device check that the compiled kernel's register use
// admits c.threads threads per block (needs a CUDA device).
bool upd_cfg_launchable(int side, int elem, int nb, const UpdCfg &c);

// Register-tiled kernels (update_tiled.cu): reflectors per thread R for a
// configuration, or 0 if it does not tile; their shared-memory bytes; the
// largest block the compiled instance admits.
int tiled_r(int nb, const UpdCfg &c);
size_t tiled_smem(int side, int elem, int nb, int th, int w);
int tiled_max_threads(int side, int elem, int R, int unroll);
template <typename T>
cudaError_t trail_tiled(int side, T *X, long ldx, int M, int N, const T *V, long ldv, int nb, const T *Tm,
                        const UpdCfg &c, const UpdScratch &sc, cudaStream_t st);

// TMA-streamed FP32 kernels (update_tma.cu): band widths 16, 32, 64; X, V
// 16-byte aligned with leading dimensions divisible by 4; same scratch as the
// register-tiled path.  side 0 = QR (V column-major at V, ld ldv), side 1 = LQ
// (V(c, k) at V[k + c*ldv]).  Their configuration reads (tile, threads, cpb,
// unroll) as (stage depth, consumer threads, pipeline stages, waves of blocks).
bool tma_cfg_valid(int nb, const UpdCfg &c);
size_t tma_cfg_smem(int nb, const UpdCfg &c);
bool trail_tma_eligible(const float *X, long ldx, const float *V, long ldv, int nb, const UpdScratch &sc);
cudaError_t trail_tma(int side, float *X, long ldx, int M, int N, const float *V, long ldv, int nb, const float *Tm,
                      const UpdCfg &c, const UpdScratch &sc, cudaStream_t st);
// The same in two parts: the projection (step 1 + T, into the scratch) and the
// update of rows [off, off + len) (side 0) / columns [off, off + len) (side 1) of
// the M x N block; off a multiple of 4.
cudaError_t trail_tma_project(int side, float *X, long ldx, int M, int N, const float *V, long ldv, int nb,
                              const float *Tm, const UpdCfg &c, const UpdScratch &sc, cudaStream_t st);
// fin_in (side 1 only): Y' to apply instead of the one trail_tma_project left in the scratch.
cudaError_t trail_tma_apply(int side, float *X, long ldx, int M, int N, const float *V, long ldv, int nb, int off,
                            int len, const UpdCfg &c, const UpdScratch &sc, cudaStream_t st,
                            const float *fin_in = nullptr);

// QR side: X (M x N at X, ldx) <- (I - V T V^T)^T X, V = unit lower M x nb at Vp (ldv).
template <typename T>
cudaError_t trail_left(T *X, long ldx, int M, int N, const T *Vp, long ldv, int nb,
                       const T *Tm, const UpdCfg &c, const UpdScratch &sc, cudaStream_t st);
// LQ side: X (M x N) <- X (I - V T V^T), V = unit lower N x nb stored transposed:
// V(c, k) = Vt[k + c*ldvt].
template <typename T>
cudaError_t trail_right(T *X, long ldx, int M, int N, const T *Vt, long ldvt, int nb,
                        const T *Tm, const UpdCfg &c, const UpdScratch &sc, cudaStream_t st);

// Mixed precision (FP64 matrix, TF32 or BF16 tensor-core contraction).
// prec: 1 = TF32, 2 = BF16; a bounded wait that gives up writes to *info.
cudaError_t trail_left_tc(double *X, long ldx, int M, int N, const double *Vp, long ldv, int nb,
                          const double *Tm, int prec, const UpdScratch &sc, int *info, cudaStream_t st);
cudaError_t trail_right_tc(double *X, long ldx, int M, int N, const double *Vt, long ldvt,
                           int nb, const double *Tm, int prec, const UpdScratch &sc, int *info, cudaStream_t st);
size_t trail_tc_scratch_bytes(int M, int N, int nb);
bool trail_tc_available();

// ---------------------------------------------------------------- copies
template <typename T>
cudaError_t copy_matrix(const T *A, long lda, int m, int n, T *B, long ldb, bool transpose,
                        cudaStream_t st);
template <typename T>
cudaError_t band_extract(const T *A, long lda, int n, int b, T *AB, long ldab, cudaStream_t st);

// ---------------------------------------------------------------- stage 2 / 3
size_t band2bd_scratch_bytes(int n);
template <typename T>
cudaError_t band2bd(T *AB, long ldab, int n, int b, double *d, double *e, void *scratch,
                    int *info, cudaStream_t st);
size_t bdsvd_scratch_bytes(int n);
template <typename T>
cudaError_t bdsvd_bisect(int n, const double *d, const double *e, T *S, void *scratch, int *info,
                         cudaStream_t st);

int device_sm_count();

}  // namespace nla
