/*
 * kt.h -- the library's auto-tuner (paper Section 3.1 and Section 4).
 *
 * The tuner searches the launch configurations of the trailing-update
 * kernels (Algorithm 2) and the band width of the pipeline (Algorithm 1's
 * only pipeline parameter, Section 5.2), minimising measured runtime:
 *     x* = argmin_{x in X} f(K_x)                       (Eq. 1)
 * over the space X of valid configurations (Section 3.1; the space's constraints
 * are the library's launch rule, kt_cfg_valid).  As in the paper
 * (Section 4.1, 4.2): every configuration's input is restored from a pristine
 * copy before each run (deep copy), one untimed warm-up run precedes the
 * timed runs, runtimes come from CUDA events on the launching stream, output
 * is verified against the default configuration's, and a configuration that
 * fails to launch or verify is recorded and skipped.  Kernel parameters are
 * tuned per band width; the band width is chosen at pipeline level
 * (Section 5.2: pipeline vs kernel parameters): KT_GESVD times the whole SVD per
 * band, each side with its own best cached kernel configuration (installed as a
 * temporary table while it runs, so other threads calling nla_gesvd_vals then see
 * it), and verifies every candidate's singular values against the default
 * configuration's.
 *
 * Search space (per band width b in {16, 32, 64}):
 *   tile {16, 32, 64, 128} x threads {64, 128, ..., 1024} x
 *   cols_per_block {1, 2, 4, 8} x unroll {1, 2, 4}       (768 points per band,
 *   2304 in all), ordered lexicographically by (band, tile, threads, cpb, unroll).
 *
 * A learned cost model (KT_MODEL_TOPK) ranks the valid space with a small MLP
 * (3 hidden layers of 128 ReLU units, FP32) trained on the GPU by the
 * library's own kernels on runtimes from earlier sweeps; only the top
 * fraction is benchmarked and the best measured configuration returned.
 * Exhaustive search remains available and is the judge of the model's picks.
 *
 * All calls run synchronously on the current CUDA device and allocate their
 * own buffers (tuning is not a hot path).  Returned statuses follow nla.h.
 */
#ifndef KT_H
#define KT_H

#include "nla.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { KT_EXHAUSTIVE = 0, KT_MODEL_TOPK = 1, KT_RANDOM = 2 } kt_strategy;

/* What Eq. 1 minimises: the runtime (milliseconds, CUDA events) or the energy one
 * launch draws (millijoules, from the device's NVML energy counter; see the energy
 * observer below). */
typedef enum { KT_TIME = 0, KT_ENERGY = 1 } kt_objective;

/* What is tuned: one trailing-update launch at panel step 0 (full size) of
 * the QR side or the LQ side, or the whole pipeline (band width only). */
typedef enum { KT_TRAIL_LEFT = 0, KT_TRAIL_RIGHT = 1, KT_GESVD = 2 } kt_kernel;

typedef struct {
    kt_kernel kernel;
    int m, n;          /* problem size (m >= n for the trailing-update kernels) */
    nla_dtype dtype;
    nla_update update; /* must be NLA_UPD_NATIVE for the SIMT trailing-update kernels */
    int band;          /* band width to tune the kernel for; 0 = every band of the space */
    int reps;          /* timed runs per configuration (median taken); 0 = 5 */
    int objective;     /* kt_objective; KT_ENERGY is supported for the kernel level (the
                          *_ms fields of the result then hold millijoules per launch) */
} kt_problem;

typedef struct {
    nla_cfg best;          /* x* of Eq. 1 (ties: lexicographically smallest) */
    double best_ms;        /* its median runtime */
    double median_ms;      /* median over all evaluated valid configurations */
    double default_ms;     /* the default configuration (band 32, tile 64, threads 128, cpb 2,
                              unroll 1): at kernel level its launch at this size (at the tuned
                              band when problem->band is set, else at band 32); for KT_GESVD
                              the whole SVD with every field of it explicit */
    int evaluated;         /* configurations timed (or read from the cache) */
    int valid;             /* configurations of the space valid for this problem */
    int failed;            /* configurations that failed to launch or verify */
    nla_cfg best_lq;       /* KT_GESVD: the LQ side's configuration of the best point (best is
                              the QR side's, with the band); zero for the kernel level */
} kt_result;

/* Number of points of the search space (2304) and the index-th point. */
int kt_space_size(void);
nla_status kt_space_get(int index, nla_cfg *out);

/* The sample KT_RANDOM draws: k distinct indices of 0..count-1 by a partial
 * Fisher-Yates shuffle driven by SplitMix64 (Steele, Lea & Flood 2014) from
 * `seed` (host only; exported so the sample can be checked). */
nla_status kt_random_subset(int count, int k, unsigned long long seed, int *out);

/* 1 if cfg is a valid launch configuration of the kernel for dtype, else 0
 * (KT_GESVD: valid for both sides).  The rule is the library's launch contract,
 * not a property of the method: the register-tiled kernels (FP64, and band
 * widths divisible by 4) need the block to tile the 32*cpb-wide strip into
 * 4-column groups and the band into groups of 1, 2, 4 or 8 reflectors, a staged
 * tile of whole 4-row sub-blocks per thread, at most 227 KiB of shared memory
 * and no more threads than the compiled kernels allow on the current device;
 * the TMA-streamed FP32 kernels (band 16/32/64) read the fields as (band, stage
 * depth 32/64/128, consumer threads 64/128/256 in whole 16-reflector groups,
 * stages 2/4/8, waves 1/2/4) within 226 KiB of shared memory.  Without a CUDA
 * device only the shape and shared-memory parts are checked.  For a problem
 * with min(m, n) >= band, nla_gesvd_vals and its workspace query return
 * NLA_ERR_CONFIG for exactly the configurations this rejects (KT_GESVD). */
int kt_cfg_valid(kt_kernel kernel, nla_dtype dtype, const nla_cfg *cfg);

/* Tune.  strategy KT_EXHAUSTIVE times every valid point; KT_RANDOM times a
 * uniformly random fraction budget_frac of the valid points (SplitMix64 from
 * `seed`, partial Fisher-Yates); KT_MODEL_TOPK times the budget_frac fraction
 * ranked best by the MLP stored at model_path (kt_mlp_train).  cache_path (may
 * be NULL): CSV of measurements; existing rows for the same problem (and
 * objective) are reused (an interrupted sweep resumes) and new rows appended.
 *
 * KT_GESVD (whole SVD, timed end to end and verified against the default
 * configuration's singular values): KT_EXHAUSTIVE picks the band width, each
 * band running each side's best configuration found in the cache (kernel-level
 * sweeps); KT_MODEL_TOPK and KT_RANDOM tune the pipeline jointly (the paper's
 * full-pipeline optimisation, Section 5.2 and Section 6) over every (band, QR-
 * side configuration, LQ-side configuration) triple: the model ranks a triple
 * by the sum over all stage-1 steps of its two update launches' predicted
 * runtimes at that step's trailing-block size; the random strategy samples the
 * triples uniformly.  Their budget is budget_frac of the joint space, at most 64
 * end-to-end runs; with the model, each band's default-kernel point is among
 * them and calibrates what the band costs besides its updates (panels, chase,
 * bisection), which the model does not predict. */
nla_status kt_tune(const kt_problem *problem, kt_strategy strategy, double budget_frac,
                   const char *cache_path, const char *model_path, unsigned long long seed,
                   kt_result *out);

/* Install a table of best configurations written by kt_write_table (or by
 * hand) -- the tuner's results put to use (Section 5.2: the tuned kernel
 * configurations and the pipeline-level band width); nla_gesvd_vals consults
 * it whenever opts->cfg is NULL, matching
 * dtype, update precision and side and taking the entry nearest in log size;
 * side-2 entries set the batched kernel's threads per matrix (cfg.band) for
 * size bucket m (0..4).  path NULL clears the table. */
nla_status kt_load_config(const char *path);

/* Append the best configuration of a finished tuning to a table file:
 * side 0 = QR-side update, 1 = LQ-side update, 2 = batched bucket m. */
nla_status kt_write_table(const char *path, int side, int m, int n, nla_dtype dtype,
                          nla_update update, const nla_cfg *cfg, double ms);

/* ---------------------------------------------------------------- energy observer */

/* The tuner's energy observer (the paper's observers for an energy objective,
 * Section 3.1, Section 6): reads, never changes, the GPU's total energy counter
 * through NVML, opened at run time (libnvidia-ml.so.1, or the library named by
 * the NLA_NVML_LIB environment variable, or by kt_energy_open).  The counter is
 * in millijoules since the driver loaded; it advances in coarse steps, so the
 * tuner measures energy over a window of at least 200 ms of repeated launches
 * and divides by their count.  Returns NLA_ERR_UNSUPPORTED when NVML or the
 * counter is unavailable. */
nla_status kt_energy_open(const char *nvml_path);
/* Counter of the current CUDA device (matched to NVML by PCI bus id). */
nla_status kt_energy_read(unsigned long long *millijoules);
/* Counter of NVML device `index`. */
nla_status kt_energy_read_index(unsigned int index, unsigned long long *millijoules);

/* ---------------------------------------------------------------- cost model */

/* Feature vector of a configuration (KT_MLP_FEATURES floats): one-hot kernel
 * (3), log2 of band, tile, threads, cols_per_block, unroll, m, n, one-hot
 * dtype (2), one-hot update (3). */
#define KT_MLP_FEATURES 15
nla_status kt_features(kt_kernel kernel, int m, int n, nla_dtype dtype, nla_update update,
                       const nla_cfg *cfg, float *out);

/* Train the MLP on the GPU with the library's kernels: X (rows x
 * KT_MLP_FEATURES, host, row-major), y (rows, host, the target log runtime).
 * Weights are initialised from `seed` (He-uniform), inputs are standardised
 * with the training set's mean and standard deviation, loss = MSE, Adam
 * (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8), minibatches of `batch` rows
 * drawn in a SplitMix64 shuffle per epoch.  The trained model (weights +
 * standardisation) is written to model_path.  final_loss (may be NULL)
 * receives the last epoch's mean training loss. */
nla_status kt_mlp_train(const float *X, const float *y, int rows, int epochs, int batch, float lr,
                        unsigned long long seed, const char *model_path, float *final_loss);

/* Predict log runtimes for `rows` feature vectors (host arrays) with the
 * model at model_path; inference runs on the GPU. */
nla_status kt_mlp_predict(const char *model_path, const float *X, int rows, float *y_out);

/* One forward + backward pass of the MLP on device buffers, for gradient
 * checks: params (device, the packed W1,b1,...,W4,b4 in FP32, W row-major
 * out x in), X (device, rows x KT_MLP_FEATURES, already standardised), y
 * (device, rows); grads (device, same packing as params) receives dL/dparams
 * of the mean squared error; pred (device, rows) the predictions. */
size_t kt_mlp_param_count(void);
nla_status kt_mlp_forward_backward(const float *dParams, const float *dX, const float *dY, int rows,
                                   float *dPred, float *dGrads, void *dWork, size_t work_bytes,
                                   nla_stream_t stream);
size_t kt_mlp_work_bytes(int rows);

/* One Adam step on device buffers (count parameters), step number t >= 1. */
nla_status kt_mlp_adam_step(float *dParams, const float *dGrads, float *dM, float *dV, size_t count,
                            int t, float lr, nla_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* KT_H */
