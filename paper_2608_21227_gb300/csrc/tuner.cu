// tuner.cu -- kt_tune / kt_load_config: the auto-tuner of include/kt.h.
//
// Eq. 1 (Section 3.1): x* = argmin over the valid space of the measured runtime.
// Measurement follows Section 4.1/4.2: the input is restored from a pristine
// device copy before every run (deep copy, excluded from timing), one untimed
// warm-up per configuration, CUDA events on the launching stream, median of
// `reps` timed runs, output verified against the default configuration, and
// launch/verification failures recorded and skipped.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/kt.h"
#include "../../include/nla.h"
#include "common.cuh"
#include "kernels.cuh"
#include "tuned.h"

extern "C" nla_status kt_random_subset(int count, int k, unsigned long long seed, int *out);

namespace {

const int kTiles[] = {16, 32, 64, 128};
const int kBands[] = {16, 32, 64};
const int kCpbs[] = {1, 2, 4, 8};
const int kUnrolls[] = {1, 2, 4};
constexpr int kThreadSteps = 16;  // 64 .. 1024 step 64
constexpr int kSpace = 3 * 4 * kThreadSteps * 4 * 3;

nla_cfg space_point(int idx) {
    // lexicographic order (band, tile, threads, cpb, unroll)
    nla_cfg c;
    c.unroll = kUnrolls[idx % 3];
    idx /= 3;
    c.cols_per_block = kCpbs[idx % 4];
    idx /= 4;
    c.threads = 64 * (1 + idx % kThreadSteps);
    idx /= kThreadSteps;
    c.tile = kTiles[idx % 4];
    idx /= 4;
    c.band = kBands[idx];
    return c;
}

nla::UpdCfg upd_of(const nla_cfg &c) { return nla::UpdCfg{c.tile, c.threads, c.cols_per_block, c.unroll}; }

// The launch rule of the trailing-update kernels (shape, shared memory and, when a
// device is present, the compiled kernels' thread limits): what nla_gesvd_vals accepts.
bool cfg_valid(int side, int elem, const nla_cfg &c) {
    return nla::upd_cfg_launchable(side, elem, c.band, upd_of(c));
}

nla_status terr(nla_status s, const std::string &m) {
    nla_set_last_error(m.c_str());
    return s;
}

// ------------------------------------------------------------------ SplitMix64
struct SplitMix64 {
    unsigned long long s;
    unsigned long long next() {
        s += 0x9E3779B97F4A7C15ull;
        unsigned long long z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// ------------------------------------------------------------------ device helpers
template <typename T>
__global__ void fill_uniform_kernel(T *A, long count, unsigned long long seed) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        A[i] = (T)((double)(z >> 11) * 0x1p-52 - 1.0);  // U[-1, 1)
    }
}

template <typename T>
__global__ void max_abs_diff_kernel(const T *A, const T *B, long count, double *out) {
    double mx = 0.0, mr = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        double a = (double)A[i], b = (double)B[i];
        mx = fmax(mx, fabs(a - b));
        mr = fmax(mr, fabs(b));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    }
    if ((threadIdx.x & 31) == 0) {
        // non-negative doubles order like their bit patterns
        atomicMax(reinterpret_cast<unsigned long long *>(out), __double_as_longlong(mx));
        atomicMax(reinterpret_cast<unsigned long long *>(out + 1), __double_as_longlong(mr));
    }
}

// ------------------------------------------------------------------ cache
struct Key {
    int kernel, m, n, dtype, update, band, tile, threads, cpb, unroll, objective;
    bool operator<(const Key &o) const {
        return std::tie(kernel, m, n, dtype, update, band, tile, threads, cpb, unroll, objective) <
               std::tie(o.kernel, o.m, o.n, o.dtype, o.update, o.band, o.tile, o.threads, o.cpb, o.unroll,
                        o.objective);
    }
};
struct Meas {
    double ms;   // the objective's value: milliseconds (KT_TIME) or millijoules per launch (KT_ENERGY)
    int status;  // 0 ok, 1 launch failure, 2 verification failure
};

void load_cache(const char *path, std::map<Key, Meas> &c) {
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == 'k') continue;  // comment / header
        Key k;
        Meas v;
        k.objective = KT_TIME;  // (files without the objective column hold runtimes)
        if (sscanf(line, "%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%lf,%d,%d", &k.kernel, &k.m, &k.n, &k.dtype, &k.update, &k.band,
                   &k.tile, &k.threads, &k.cpb, &k.unroll, &v.ms, &v.status, &k.objective) >= 12)
            c[k] = v;
    }
    fclose(f);
}

void append_cache(const char *path, const Key &k, const Meas &v) {
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    if (ftell(f) == 0) fprintf(f, "kernel,m,n,dtype,update,band,tile,threads,cpb,unroll,median_ms,status,objective\n");
    fprintf(f, "%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%.6f,%d,%d\n", k.kernel, k.m, k.n, k.dtype, k.update, k.band, k.tile,
            k.threads, k.cpb, k.unroll, v.ms, v.status, k.objective);
    fclose(f);
}

// ------------------------------------------------------------------ installed table
struct TableEntry {
    int side, m, n, dtype, update;
    nla_cfg cfg;
    double ms;
};
std::mutex g_table_mu;
std::vector<TableEntry> g_table;

double median_of(std::vector<double> v) {
    if (v.empty()) return NAN;
    std::sort(v.begin(), v.end());
    size_t k = v.size();
    return k % 2 ? v[k / 2] : 0.5 * (v[k / 2 - 1] + v[k / 2]);
}

const nla_cfg kDefault = {32, 64, 128, 2, 1};

// The default configuration's kernel parameters (any band).
bool is_default_kernel(const nla_cfg &c) {
    return c.tile == kDefault.tile && c.threads == kDefault.threads && c.cols_per_block == kDefault.cols_per_block &&
           c.unroll == kDefault.unroll;
}

// ------------------------------------------------------------------ trailing-update tuning
template <typename T>
struct TrailBench {
    int side, m, n, reps, objective = KT_TIME;
    T *A = nullptr, *A0 = nullptr, *Xref = nullptr;
    T *tau = nullptr, *Tm = nullptr;
    unsigned int *bar = nullptr, *tickets = nullptr;
    void *uwork = nullptr;
    double *part = nullptr, *diff = nullptr;
    int *info = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int b = 0;

    cudaError_t init() {
        size_t cnt = (size_t)m * n;
        cudaError_t e;
        if ((e = cudaMalloc(&A, cnt * sizeof(T)))) return e;
        if ((e = cudaMalloc(&A0, cnt * sizeof(T)))) return e;
        if ((e = cudaMalloc(&Xref, cnt * sizeof(T)))) return e;
        if ((e = cudaMalloc(&tau, 64 * sizeof(T)))) return e;
        if ((e = cudaMalloc(&Tm, 64 * 64 * sizeof(T)))) return e;
        if ((e = cudaMalloc(&bar, 64 * sizeof(unsigned int)))) return e;
        if ((e = cudaMalloc(&tickets, nla::tiled_tickets(m, n) * sizeof(unsigned int)))) return e;
        if ((e = cudaMemset(tickets, 0, nla::tiled_tickets(m, n) * sizeof(unsigned int)))) return e;
        if ((e = cudaMalloc(&uwork, nla::tiled_scratch_elems(m, n) * sizeof(T)))) return e;
        if ((e = cudaMalloc(&part, nla::panel_part_doubles(nla::panel_max_ctas()) * sizeof(double)))) return e;
        if ((e = cudaMalloc(&diff, 2 * sizeof(double)))) return e;
        if ((e = cudaMalloc(&info, sizeof(int)))) return e;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) return e;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        return cudaSuccess;
    }
    ~TrailBench() {
        cudaFree(A);
        cudaFree(A0);
        cudaFree(Xref);
        cudaFree(tau);
        cudaFree(Tm);
        cudaFree(bar);
        cudaFree(tickets);
        cudaFree(uwork);
        cudaFree(part);
        cudaFree(diff);
        cudaFree(info);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    }
    // Fresh input and the reflectors of panel step 0 for band width bb.
    cudaError_t setup(int bb, unsigned long long seed) {
        b = bb;
        long cnt = (long)m * n;
        fill_uniform_kernel<T><<<1024, 256, 0, st>>>(A, cnt, seed);
        cudaMemsetAsync(bar, 0, 64 * sizeof(unsigned int), st);
        cudaMemsetAsync(info, 0, sizeof(int), st);
        nla::PanelCtl ctl{bar, part, info};
        cudaError_t e;
        if (side == 0)
            e = nla::panel_factor<T>(A, 1, m, m, b, tau, Tm, ctl, st);
        else
            e = nla::panel_factor<T>(A + (long)b * m, m, 1, n - b, b, tau, Tm, ctl, st);
        if (e) return e;
        e = cudaMemcpyAsync(A0, A, cnt * sizeof(T), cudaMemcpyDeviceToDevice, st);
        if (e) return e;
        return cudaStreamSynchronize(st);
    }
    cudaError_t launch(const nla_cfg &c) {
        const nla::UpdScratch sc{uwork, tickets};
        if (side == 0)
            return nla::trail_left<T>(A + (long)b * m, m, m, n - b, A, m, b, Tm, upd_of(c), sc, st);
        return nla::trail_right<T>(A + b + (long)b * m, m, m - b, n - b, A + (long)b * m, m, b, Tm, upd_of(c), sc,
                                   st);
    }
    cudaError_t restore() { return cudaMemcpyAsync(A, A0, (size_t)m * n * sizeof(T), cudaMemcpyDeviceToDevice, st); }
    // Returns median ms (status 0), or status 1 (launch) / 2 (verification).
    Meas measure(const nla_cfg &c, bool is_reference) {
        restore();
        if (launch(c) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return {NAN, 1};
        }
        std::vector<double> t;
        for (int r = 0; r < reps; ++r) {
            restore();
            cudaEventRecord(e0, st);
            if (launch(c) != cudaSuccess) {
                cudaGetLastError();
                return {NAN, 1};
            }
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return {NAN, 1};
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms > 0.f) t.push_back(ms);
        }
        if (t.empty()) return {NAN, 1};
        double value = median_of(t);
        if (objective == KT_ENERGY) {
            // energy per launch: back-to-back launches over at least 200 ms (the counter
            // advances in coarse steps; each launch applies an orthogonal transformation,
            // so the repeats keep X bounded), restored afterwards for the verification
            const int R = std::max(reps, (int)std::ceil(200.0 / std::max(value, 1e-3)));
            unsigned long long e0 = 0, e1 = 0;
            cudaStreamSynchronize(st);
            if (kt_energy_read(&e0) != NLA_OK) return {NAN, 1};
            for (int r = 0; r < R; ++r)
                if (launch(c) != cudaSuccess) {
                    cudaGetLastError();
                    return {NAN, 1};
                }
            if (cudaStreamSynchronize(st) != cudaSuccess || kt_energy_read(&e1) != NLA_OK) return {NAN, 1};
            value = (double)(e1 - e0) / R;
            restore();
            if (launch(c) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
                cudaGetLastError();
                return {NAN, 1};
            }
        }
        size_t cnt = (size_t)m * n;
        if (is_reference) {
            cudaMemcpyAsync(Xref, A, cnt * sizeof(T), cudaMemcpyDeviceToDevice, st);
            cudaStreamSynchronize(st);
        } else {
            cudaMemsetAsync(diff, 0, 2 * sizeof(double), st);
            max_abs_diff_kernel<T><<<512, 256, 0, st>>>(A, Xref, (long)cnt, diff);
            double h[2] = {0, 0};
            cudaMemcpyAsync(h, diff, sizeof h, cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            const double tol = sizeof(T) == 8 ? 1e-10 : 1e-3;
            if (!(h[0] <= tol * std::max(h[1], 1e-300))) return {value, 2};
        }
        return {value, 0};
    }
};

}  // namespace

// ------------------------------------------------------------------ MLP inference hook (mlp.cu)
namespace nla {
nla_status mlp_predict_host(const char *model_path, const float *X, int rows, float *y);
extern int g_batched_group[5];  // batched.cu: threads per matrix per size bucket (0 = default)
}

namespace {

template <typename T>
nla_status tune_trail(const kt_problem &p, kt_strategy strategy, double frac, const char *cache_path,
                      const char *model_path, unsigned long long seed, kt_result *out) {
    const int side = p.kernel == KT_TRAIL_LEFT ? 0 : 1;
    const int elem = (int)sizeof(T);
    std::map<Key, Meas> cache;
    load_cache(cache_path, cache);
    TrailBench<T> tb;
    tb.side = side;
    tb.m = p.m;
    tb.n = p.n;
    tb.reps = p.reps > 0 ? p.reps : 5;
    tb.objective = p.objective;
    if (p.objective == KT_ENERGY) {
        unsigned long long e = 0;
        nla_status s = kt_energy_read(&e);
        if (s != NLA_OK) return s;
    }
    if (tb.init() != cudaSuccess) {
        cudaGetLastError();
        return terr(NLA_ERR_CUDA, "tuner: allocation failed");
    }
    std::vector<nla_cfg> valid;
    for (int i = 0; i < kSpace; ++i) {
        nla_cfg c = space_point(i);
        if (p.band > 0 && c.band != p.band) continue;
        if (c.band >= p.n) continue;
        if (nla::upd_cfg_launchable(side, elem, c.band, upd_of(c))) valid.push_back(c);
    }
    // candidate list per strategy
    std::vector<nla_cfg> cand = valid;
    if (strategy != KT_EXHAUSTIVE && !valid.empty()) {
        size_t k = (size_t)std::ceil(std::max(0.0, std::min(1.0, frac)) * valid.size());
        k = std::max<size_t>(1, std::min(k, valid.size()));
        if (strategy == KT_RANDOM) {
            std::vector<int> idx(k);
            kt_random_subset((int)valid.size(), (int)k, seed, idx.data());
            cand.clear();
            for (size_t i = 0; i < k; ++i) cand.push_back(valid[idx[i]]);
        } else {  // model-ranked top fraction
            if (!model_path) return terr(NLA_ERR_ARG, "KT_MODEL_TOPK needs model_path");
            std::vector<float> X(valid.size() * KT_MLP_FEATURES), y(valid.size());
            for (size_t i = 0; i < valid.size(); ++i)
                kt_features(p.kernel, p.m, p.n, p.dtype, p.update, &valid[i], &X[i * KT_MLP_FEATURES]);
            nla_status s = nla::mlp_predict_host(model_path, X.data(), (int)valid.size(), y.data());
            if (s != NLA_OK) return s;
            std::vector<int> idx(valid.size());
            for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return y[a] < y[b]; });
            cand.clear();
            for (size_t i = 0; i < k; ++i) cand.push_back(valid[idx[i]]);
        }
    }
    kt_result r;
    memset(&r, 0, sizeof r);
    r.valid = (int)valid.size();
    r.best_ms = r.median_ms = r.default_ms = NAN;
    std::vector<double> times;
    bool have_best = false;
    int cur_band = -1;
    for (size_t ci = 0; ci < cand.size(); ++ci) {
        const nla_cfg &c = cand[ci];
        if (c.band != cur_band) {  // new band: fresh reflectors and a reference output
            cur_band = c.band;
            if (tb.setup(cur_band, seed ^ 0x5EEDull) != cudaSuccess) {
                cudaGetLastError();
                return terr(NLA_ERR_CUDA, "tuner: setup failed");
            }
            nla_cfg ref = kDefault;
            ref.band = cur_band;
            nla::UpdCfg u = upd_of(ref);
            size_t sm;
            if (!nla::upd_cfg_valid(side, elem, cur_band, u, &sm)) ref = c;
            Meas mref = tb.measure(ref, true);
            if (mref.status != 0) return terr(NLA_ERR_CUDA, "tuner: reference configuration failed");
            // the default's kernel parameters at the band being tuned (kernel parameters are
            // tuned per band; with every band, the default band's entry is reported)
            if (is_default_kernel(ref) && (p.band > 0 || ref.band == kDefault.band)) r.default_ms = mref.ms;
        }
        Key k{(int)p.kernel, p.m, p.n, (int)p.dtype, (int)p.update, c.band, c.tile, c.threads, c.cols_per_block,
              c.unroll, p.objective};
        Meas v;
        auto it = cache.find(k);
        if (it != cache.end()) {
            v = it->second;
        } else {
            v = tb.measure(c, false);
            cache[k] = v;
            append_cache(cache_path, k, v);
        }
        r.evaluated++;
        if (v.status != 0) {
            r.failed++;
            continue;
        }
        times.push_back(v.ms);
        if (!have_best || v.ms < r.best_ms) {  // candidates are visited in lexicographic order: ties keep the first
            r.best = c;
            r.best_ms = v.ms;
            have_best = true;
        }
        if (is_default_kernel(c) && (p.band > 0 || c.band == kDefault.band)) r.default_ms = v.ms;
    }
    // the model / random strategies visit candidates out of lexicographic order: recompute ties properly
    r.median_ms = median_of(times);
    if (!have_best) return terr(NLA_ERR_CONFIG, "tuner: no configuration ran successfully");
    *out = r;
    return NLA_OK;
}

// Installs a temporary tuned table for the pipeline-level runs (each side its own
// configuration) and puts the caller's table back when it goes out of scope.
struct TableSwap {
    std::vector<TableEntry> saved;
    bool active = false;
    void install(const std::vector<TableEntry> &t) {
        std::lock_guard<std::mutex> lk(g_table_mu);
        if (!active) saved = g_table;
        g_table = t;
        active = true;
    }
    ~TableSwap() {
        if (!active) return;
        std::lock_guard<std::mutex> lk(g_table_mu);
        g_table.swap(saved);
    }
};

// Verification tolerance of a pipeline-level candidate against the default
// configuration's singular values (relative to the largest): twice the acceptance
// bound of the dtype, or for the TF32 / BF16 forms the first-order model 10 u sqrt(N/16)
// (u = 2^-11, 2^-8; the compensated BF16X3 form u = 2^-16, TF32X3 the FP32 bound).
double pipeline_tol(const kt_problem &p, int N) {
    if (p.update == NLA_UPD_TF32) return 10.0 * std::ldexp(1.0, -11) * std::sqrt(N / 16.0);
    if (p.update == NLA_UPD_BF16) return 10.0 * std::ldexp(1.0, -8) * std::sqrt(N / 16.0);
    if (p.update == NLA_UPD_BF16X3) return 10.0 * std::ldexp(1.0, -16) * std::sqrt(N / 16.0);
    if (p.update == NLA_UPD_TF32X3) return 2.0 * 5e-6 * N;
    return 2.0 * (p.dtype == NLA_F64 ? 1e-12 : 5e-6) * N;
}

// End-to-end timing of nla_gesvd_vals on one seeded U[-1, 1] problem: the input is
// restored from a pristine copy before every run, one warm-up precedes `reps` timed
// runs (median), and the singular values are either kept as the reference (the default
// configuration) or checked against it.
struct PipelineBench {
    const kt_problem &p;
    int es, M, N, reps;
    size_t cnt, wbytes = 0;
    void *A = nullptr, *A0 = nullptr, *S = nullptr, *Sref = nullptr, *W = nullptr;
    int *info = nullptr;
    double *diff = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;

    explicit PipelineBench(const kt_problem &prob)
        : p(prob), es(prob.dtype == NLA_F64 ? 8 : 4), M(std::max(prob.m, prob.n)), N(std::min(prob.m, prob.n)),
          reps(prob.reps > 0 ? prob.reps : 3), cnt((size_t)M * N) {}
    ~PipelineBench() {
        cudaFree(A);
        cudaFree(A0);
        cudaFree(S);
        cudaFree(Sref);
        cudaFree(W);
        cudaFree(info);
        cudaFree(diff);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    }
    bool init(unsigned long long seed) {
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        if (cudaMalloc(&A, cnt * es) || cudaMalloc(&A0, cnt * es) || cudaMalloc(&S, N * (size_t)es) ||
            cudaMalloc(&Sref, N * (size_t)es) || cudaMalloc(&info, sizeof(int)) || cudaMalloc(&diff, 2 * sizeof(double))) {
            cudaGetLastError();
            return false;
        }
        if (es == 8)
            fill_uniform_kernel<double><<<1024, 256, 0, st>>>((double *)A0, (long)cnt, seed);
        else
            fill_uniform_kernel<float><<<1024, 256, 0, st>>>((float *)A0, (long)cnt, seed);
        return cudaStreamSynchronize(st) == cudaSuccess;
    }
    // 0 ok, 1 launch failure, 2 verification failure
    int run(const nla_opts &o, bool reference, double &med) {
        size_t need = 0;
        if (nla_gesvd_vals_workspace(M, N, p.dtype, &o, &need) != NLA_OK) return 1;
        if (need > wbytes) {
            cudaFree(W);
            W = nullptr;
            wbytes = 0;
            if (cudaMalloc(&W, need)) {
                cudaGetLastError();
                return 1;
            }
            wbytes = need;
        }
        std::vector<double> t;
        for (int rep = 0; rep <= reps; ++rep) {
            cudaMemcpyAsync(A, A0, cnt * es, cudaMemcpyDeviceToDevice, st);
            cudaEventRecord(e0, st);
            nla_status s = nla_gesvd_vals(M, N, p.dtype, A, M, S, W, wbytes, info, &o, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || s != NLA_OK) {
                cudaGetLastError();
                return 1;
            }
            int hinfo = 0;
            cudaMemcpy(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost);
            if (hinfo != 0) return 1;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t.push_back(ms);  // rep 0 is the warm-up
        }
        med = median_of(t);
        if (reference) {
            cudaMemcpyAsync(Sref, S, N * (size_t)es, cudaMemcpyDeviceToDevice, st);
            cudaStreamSynchronize(st);
            return 0;
        }
        cudaMemsetAsync(diff, 0, 2 * sizeof(double), st);
        if (es == 8)
            max_abs_diff_kernel<double><<<64, 256, 0, st>>>((const double *)S, (const double *)Sref, N, diff);
        else
            max_abs_diff_kernel<float><<<64, 256, 0, st>>>((const float *)S, (const float *)Sref, N, diff);
        double h[2] = {0, 0};
        cudaMemcpyAsync(h, diff, sizeof h, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        return h[0] <= pipeline_tol(p, M) * std::max(h[1], 1e-300) ? 0 : 2;
    }
    // the whole SVD with band b, the QR-side update running cl and the LQ side cr at every
    // step (installed as a one-size table while it runs)
    int run_pair(TableSwap &swap, int b, const nla_cfg &cl, const nla_cfg &cr, double &med) {
        std::vector<TableEntry> t(2);
        t[0] = TableEntry{0, M, N, (int)p.dtype, (int)p.update, cl, 0.0};
        t[1] = TableEntry{1, M, N, (int)p.dtype, (int)p.update, cr, 0.0};
        swap.install(t);
        nla_cfg band_only = {b, 0, 0, 0, 0};
        nla_opts o = {p.update, &band_only, 0};
        return run(o, false, med);
    }
    // the default configuration (every field explicit: no table), kept as the reference
    bool run_default(double &med) {
        nla_cfg dflt = kDefault;
        nla_opts od = {p.update, &dflt, 0};
        return run(od, true, med) == 0;
    }
};

nla_status tune_gesvd(const kt_problem &p, const char *cache_path, unsigned long long seed, kt_result *out) {
    // pipeline level: band width, each band with each side's best kernel configuration
    // from the cache (else the defaults), timed end to end and verified against the
    // default configuration's singular values
    std::map<Key, Meas> cache;
    load_cache(cache_path, cache);
    kt_result r;
    memset(&r, 0, sizeof r);
    r.best_ms = r.median_ms = r.default_ms = NAN;
    std::vector<double> times;
    TableSwap swap;
    PipelineBench pb(p);
    if (!pb.init(seed)) return terr(NLA_ERR_CUDA, "tuner: allocation failed");
    double dms = NAN;
    if (!pb.run_default(dms)) return terr(NLA_ERR_CUDA, "tuner: the default configuration failed");
    r.default_ms = dms;
    for (int bi = 0; bi < 3; ++bi) {
        const int b = kBands[bi];
        if (p.band > 0 && b != p.band) continue;
        if (b >= pb.N) continue;
        nla_cfg best[2];
        for (int side = 0; side < 2; ++side) {
            best[side] = kDefault;
            best[side].band = b;
            double bm = INFINITY;
            for (auto &kv : cache) {
                const Key &k = kv.first;
                if (k.kernel != side || k.dtype != (int)p.dtype || k.update != (int)p.update || k.band != b ||
                    kv.second.status != 0)
                    continue;
                // nearest problem size in the cache with this band
                double d = std::fabs(std::log2((double)k.m / p.m)) + std::fabs(std::log2((double)k.n / p.n));
                double score = d * 1e6 + kv.second.ms;
                if (score < bm) {
                    bm = score;
                    best[side] = nla_cfg{b, k.tile, k.threads, k.cpb, k.unroll};
                }
            }
        }
        double med = NAN;
        const int rs = pb.run_pair(swap, b, best[0], best[1], med);
        r.evaluated++;
        if (rs != 0) {
            r.failed++;
            continue;
        }
        times.push_back(med);
        if (!(med >= r.best_ms)) {
            r.best_ms = med;
            r.best = best[0];
            r.best_lq = best[1];
        }
    }
    r.valid = (int)times.size() + r.failed;
    r.median_ms = median_of(times);
    if (times.empty()) return terr(NLA_ERR_CONFIG, "tuner: no band ran successfully");
    *out = r;
    return NLA_OK;
}

// Full-pipeline joint tuning: the space is every (band, QR-side configuration, LQ-side
// configuration) triple valid for the problem, and each point is judged by the whole
// SVD's runtime (the paper's "full pipeline optimization", Section 5.2 / Section 6).
// KT_MODEL_TOPK ranks the joint space with the MLP: a point's predicted cost is the sum,
// over every stage-1 step, of the predicted runtimes of its two update launches at that
// step's trailing-block size; KT_RANDOM samples the joint space uniformly (SplitMix64).
// The budget_frac fraction (at most kJointMax points) is timed end to end and verified.
constexpr int kJointMax = 64;

nla_status tune_joint(const kt_problem &p, kt_strategy strategy, double frac, const char *model_path,
                      unsigned long long seed, kt_result *out) {
    const int elem = p.dtype == NLA_F64 ? 8 : 4;
    const int M = std::max(p.m, p.n), N = std::min(p.m, p.n);
    struct BandSpace {
        int b;
        std::vector<nla_cfg> L, R;
        std::vector<double> pl, pr;  // predicted stage-1 update time per configuration (ms)
    };
    std::vector<BandSpace> bands;
    long total = 0;
    for (int bi = 0; bi < 3; ++bi) {
        const int b = kBands[bi];
        if ((p.band > 0 && b != p.band) || b >= N) continue;
        BandSpace bs;
        bs.b = b;
        for (int i = 0; i < kSpace; ++i) {
            const nla_cfg c = space_point(i);
            if (c.band != b) continue;
            if (nla::upd_cfg_launchable(0, elem, b, upd_of(c))) bs.L.push_back(c);
            if (nla::upd_cfg_launchable(1, elem, b, upd_of(c))) bs.R.push_back(c);
        }
        if (bs.L.empty() || bs.R.empty()) continue;
        total += (long)bs.L.size() * (long)bs.R.size();
        bands.push_back(std::move(bs));
    }
    if (bands.empty() || total <= 0) return terr(NLA_ERR_CONFIG, "tuner: empty joint space");
    if (total > (long)1 << 30) return terr(NLA_ERR_UNSUPPORTED, "tuner: joint space too large");
    long k = (long)std::ceil(std::max(0.0, std::min(1.0, frac)) * (double)total);
    k = std::max(1L, std::min({k, total, (long)kJointMax}));
    // candidates as (band index, left index, right index)
    std::vector<std::array<int, 3>> cand;
    auto decode = [&](long idx) {
        for (int bi = 0; bi < (int)bands.size(); ++bi) {
            const long sz = (long)bands[bi].L.size() * (long)bands[bi].R.size();
            if (idx < sz) return std::array<int, 3>{bi, (int)(idx / (long)bands[bi].R.size()),
                                                    (int)(idx % (long)bands[bi].R.size())};
            idx -= sz;
        }
        return std::array<int, 3>{0, 0, 0};
    };
    if (strategy == KT_RANDOM) {
        std::vector<int> idx((size_t)k);
        kt_random_subset((int)total, (int)k, seed, idx.data());
        for (long i = 0; i < k; ++i) cand.push_back(decode(idx[(size_t)i]));
    } else {
        if (!model_path) return terr(NLA_ERR_ARG, "KT_MODEL_TOPK needs model_path");
        // predicted stage-1 update time of every configuration of each band and side
        for (BandSpace &bs : bands) {
            std::vector<std::pair<int, int>> steps[2];  // trailing-block sizes of the QR / LQ updates
            for (int kb = 0; kb < N; kb += bs.b) {
                const int nb = std::min(bs.b, N - kb), c0 = kb + nb;
                if (c0 >= N) break;
                steps[0].push_back({M - kb, N - c0});
                if (M - c0 > 0) steps[1].push_back({M - c0, N - c0});
            }
            for (int side = 0; side < 2; ++side) {
                const std::vector<nla_cfg> &cs = side == 0 ? bs.L : bs.R;
                std::vector<double> &pred = side == 0 ? bs.pl : bs.pr;
                const size_t rows = cs.size() * steps[side].size();
                std::vector<float> X(rows * KT_MLP_FEATURES), y(rows);
                size_t r = 0;
                for (const nla_cfg &c : cs)
                    for (const auto &mn : steps[side])
                        kt_features(side == 0 ? KT_TRAIL_LEFT : KT_TRAIL_RIGHT, mn.first, mn.second, p.dtype, p.update,
                                    &c, &X[(r++) * KT_MLP_FEATURES]);
                nla_status s = nla::mlp_predict_host(model_path, X.data(), (int)rows, y.data());
                if (s != NLA_OK) return s;
                pred.assign(cs.size(), 0.0);
                for (size_t i = 0; i < cs.size(); ++i)
                    for (size_t j = 0; j < steps[side].size(); ++j) pred[i] += std::exp((double)y[i * steps[side].size() + j]);
            }
        }
    }
    kt_result r;
    memset(&r, 0, sizeof r);
    r.best_ms = r.median_ms = r.default_ms = NAN;
    r.valid = (int)std::min(total, (long)INT32_MAX);
    std::vector<double> times;
    TableSwap swap;
    PipelineBench pb(p);
    if (!pb.init(seed)) return terr(NLA_ERR_CUDA, "tuner: allocation failed");
    double dms = NAN;
    if (!pb.run_default(dms)) return terr(NLA_ERR_CUDA, "tuner: the default configuration failed");
    r.default_ms = dms;
    auto measure = [&](const std::array<int, 3> &c) -> double {
        const BandSpace &bs = bands[(size_t)c[0]];
        const nla_cfg &cl = bs.L[(size_t)c[1]], &cr = bs.R[(size_t)c[2]];
        double med = NAN;
        const int rs = pb.run_pair(swap, bs.b, cl, cr, med);
        r.evaluated++;
        if (rs != 0) {
            r.failed++;
            return (double)NAN;
        }
        times.push_back(med);
        if (!(med >= r.best_ms)) {
            r.best_ms = med;
            r.best = cl;
            r.best_lq = cr;
        }
        return med;
    };
    if (strategy != KT_RANDOM) {
        // The model predicts the update launches only; what a band adds besides them (its
        // panels, chase and bisection) is measured: each band's default-kernel point is
        // timed first (part of the budget) and the difference to its predicted update
        // cost is the band's constant.  The rest of the budget goes to the points of
        // smallest predicted total (ties: lexicographic order).
        std::vector<double> cband(bands.size(), 0.0);
        std::vector<long> taken;
        long base = 0;
        for (size_t bi = 0; bi < bands.size() && (long)taken.size() < k; ++bi) {
            const BandSpace &bs = bands[bi];
            auto pick = [&](const std::vector<nla_cfg> &cs) {
                for (size_t i = 0; i < cs.size(); ++i)
                    if (is_default_kernel(cs[i])) return i;
                return (size_t)0;
            };
            const size_t dl = pick(bs.L), dr = pick(bs.R);
            const double t = measure({(int)bi, (int)dl, (int)dr});
            if (t == t) cband[bi] = std::max(0.0, t - (bs.pl[dl] + bs.pr[dr]));
            taken.push_back(base + (long)(dl * bs.R.size() + dr));
            base += (long)bs.L.size() * (long)bs.R.size();
        }
        std::vector<std::pair<double, long>> all;
        all.reserve((size_t)total);
        base = 0;
        for (size_t bi = 0; bi < bands.size(); ++bi) {
            const BandSpace &bs = bands[bi];
            for (size_t i = 0; i < bs.L.size(); ++i)
                for (size_t j = 0; j < bs.R.size(); ++j) {
                    const long idx = base + (long)(i * bs.R.size() + j);
                    if (std::find(taken.begin(), taken.end(), idx) == taken.end())
                        all.push_back({cband[bi] + bs.pl[i] + bs.pr[j], idx});
                }
            base += (long)bs.L.size() * (long)bs.R.size();
        }
        const long rest = std::max(0L, std::min(k - (long)taken.size(), (long)all.size()));
        std::partial_sort(all.begin(), all.begin() + rest, all.end());
        for (long i = 0; i < rest; ++i) cand.push_back(decode(all[(size_t)i].second));
    }
    for (const auto &c : cand) measure(c);
    r.median_ms = median_of(times);
    if (times.empty()) return terr(NLA_ERR_CONFIG, "tuner: no joint candidate ran successfully");
    *out = r;
    return NLA_OK;
}

}  // namespace

extern "C" {

int kt_space_size(void) { return kSpace; }

nla_status kt_random_subset(int count, int k, unsigned long long seed, int *out) {
    if (count < 0 || k < 0 || (k > 0 && !out)) return terr(NLA_ERR_ARG, "bad arguments");
    std::vector<int> idx(count);
    for (int i = 0; i < count; ++i) idx[i] = i;
    SplitMix64 g{seed};
    k = std::min(k, count);
    for (int i = 0; i < k; ++i) {
        int j = i + (int)(g.next() % (unsigned long long)(count - i));
        std::swap(idx[i], idx[j]);
        out[i] = idx[i];
    }
    return NLA_OK;
}

nla_status kt_space_get(int index, nla_cfg *out) {
    if (index < 0 || index >= kSpace || !out) return NLA_ERR_ARG;
    *out = space_point(index);
    return NLA_OK;
}

int kt_cfg_valid(kt_kernel kernel, nla_dtype dtype, const nla_cfg *cfg) {
    if (!cfg) return 0;
    const int elem = dtype == NLA_F64 ? 8 : 4;
    if (kernel == KT_TRAIL_LEFT) return cfg_valid(0, elem, *cfg);
    if (kernel == KT_TRAIL_RIGHT) return cfg_valid(1, elem, *cfg);
    return cfg_valid(0, elem, *cfg) && cfg_valid(1, elem, *cfg);
}

nla_status kt_features(kt_kernel kernel, int m, int n, nla_dtype dtype, nla_update update, const nla_cfg *cfg,
                       float *out) {
    if (!cfg || !out || kernel < 0 || kernel > 2) return NLA_ERR_ARG;
    for (int i = 0; i < KT_MLP_FEATURES; ++i) out[i] = 0.f;
    out[kernel] = 1.f;
    out[3] = (float)std::log2((double)std::max(cfg->band, 1));
    out[4] = (float)std::log2((double)std::max(cfg->tile, 1));
    out[5] = (float)std::log2((double)std::max(cfg->threads, 1));
    out[6] = (float)std::log2((double)std::max(cfg->cols_per_block, 1));
    out[7] = (float)std::log2((double)std::max(cfg->unroll, 1));
    out[8] = (float)std::log2((double)std::max(m, 1));
    out[9] = (float)std::log2((double)std::max(n, 1));
    out[10 + (dtype == NLA_F64 ? 0 : 1)] = 1.f;
    out[12 + std::min(std::max((int)update, 0), 2)] = 1.f;
    return NLA_OK;
}

nla_status kt_tune(const kt_problem *p, kt_strategy strategy, double budget_frac, const char *cache_path,
                   const char *model_path, unsigned long long seed, kt_result *out) {
    if (!p || !out) return terr(NLA_ERR_ARG, "null argument");
    if (p->m <= 0 || p->n <= 0) return terr(NLA_ERR_ARG, "empty problem");
    if (p->dtype != NLA_F64 && p->dtype != NLA_F32) return terr(NLA_ERR_ARG, "unknown dtype");
    if (strategy < KT_EXHAUSTIVE || strategy > KT_RANDOM) return terr(NLA_ERR_ARG, "unknown strategy");
    if (p->objective != KT_TIME && p->objective != KT_ENERGY) return terr(NLA_ERR_ARG, "unknown objective");
    if (p->objective == KT_ENERGY && p->kernel == KT_GESVD)
        return terr(NLA_ERR_UNSUPPORTED, "the energy objective is supported for the kernel level");
    if (p->kernel == KT_GESVD)
        return strategy == KT_EXHAUSTIVE ? tune_gesvd(*p, cache_path, seed, out)
                                         : tune_joint(*p, strategy, budget_frac, model_path, seed, out);
    if (p->kernel != KT_TRAIL_LEFT && p->kernel != KT_TRAIL_RIGHT) return terr(NLA_ERR_ARG, "unknown kernel");
    if (p->update != NLA_UPD_NATIVE) return terr(NLA_ERR_ARG, "SIMT trailing-update tuning needs NLA_UPD_NATIVE");
    if (p->m < p->n) return terr(NLA_ERR_ARG, "trailing-update tuning needs m >= n");
    if (p->dtype == NLA_F64) return tune_trail<double>(*p, strategy, budget_frac, cache_path, model_path, seed, out);
    return tune_trail<float>(*p, strategy, budget_frac, cache_path, model_path, seed, out);
}

nla_status kt_write_table(const char *path, int side, int m, int n, nla_dtype dtype, nla_update update,
                          const nla_cfg *cfg, double ms) {
    if (!path || !cfg || side < 0 || side > 2) return terr(NLA_ERR_ARG, "bad arguments");
    FILE *f = fopen(path, "a");
    if (!f) return terr(NLA_ERR_ARG, std::string("cannot open ") + path);
    if (ftell(f) == 0) fprintf(f, "# side m n dtype update band tile threads cpb unroll ms\n");
    fprintf(f, "%d %d %d %d %d %d %d %d %d %d %.6f\n", side, m, n, (int)dtype, (int)update, cfg->band, cfg->tile,
            cfg->threads, cfg->cols_per_block, cfg->unroll, ms);
    fclose(f);
    return NLA_OK;
}

nla_status kt_load_config(const char *path) {
    std::vector<TableEntry> t;
    if (path) {
        FILE *f = fopen(path, "r");
        if (!f) return terr(NLA_ERR_ARG, std::string("cannot open ") + path);
        char line[512];
        while (fgets(line, sizeof line, f)) {
            if (line[0] == '#') continue;
            TableEntry e;
            if (sscanf(line, "%d %d %d %d %d %d %d %d %d %d %lf", &e.side, &e.m, &e.n, &e.dtype, &e.update,
                       &e.cfg.band, &e.cfg.tile, &e.cfg.threads, &e.cfg.cols_per_block, &e.cfg.unroll, &e.ms) == 11)
                t.push_back(e);
        }
        fclose(f);
        if (t.empty()) return terr(NLA_ERR_ARG, std::string("no entries in ") + path);
    }
    // side-2 entries carry the batched kernel's group size per size bucket:
    // m = bucket index, band field = threads per matrix
    int groups[5] = {0, 0, 0, 0, 0};
    for (const TableEntry &e : t)
        if (e.side == 2 && e.m >= 0 && e.m < 5) groups[e.m] = e.cfg.band;
    for (int b = 0; b < 5; ++b) nla::g_batched_group[b] = groups[b];
    std::lock_guard<std::mutex> lk(g_table_mu);
    g_table.swap(t);
    return NLA_OK;
}

int nla_tuned_lookup(int m, int n, int dtype, int update, int side, nla_cfg *out) {
    std::lock_guard<std::mutex> lk(g_table_mu);
    const TableEntry *best = nullptr;
    double bd = INFINITY;
    for (const TableEntry &e : g_table) {
        if (e.dtype != dtype || e.update != update || e.side != side) continue;
        double d = std::fabs(std::log2((double)std::max(m, 1) / e.m)) + std::fabs(std::log2((double)std::max(n, 1) / e.n));
        if (d < bd) {
            bd = d;
            best = &e;
        }
    }
    if (!best) return 0;
    *out = best->cfg;
    return 1;
}

}  // extern "C"
