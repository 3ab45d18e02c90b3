// api.cu -- the C ABI declared in include/nla.h: argument checking, workspace
// carving, configuration lookup and the host-side loop of Algorithm 1.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/nla.h"
#include "common.cuh"
#include "kernels.cuh"
#include "trace.h"
#include "tuned.h"

namespace {

thread_local std::string g_last_error;

nla_status fail(nla_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

nla_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorInvalidConfiguration ? NLA_ERR_CONFIG : NLA_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define NLA_CUDA(call, what)                          \
    do {                                              \
        cudaError_t _e = (call);                      \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// A kernel launch bracketed by the tracing events of its class.
#define NLA_LAUNCH(cls, st, call, what)               \
    do {                                              \
        cudaError_t _e;                               \
        {                                             \
            nla::TraceScope _ts(cls, st);             \
            _e = (call);                              \
        }                                             \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves typed regions out of the caller's workspace (or only sizes them when base == nullptr).
struct Carver {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

const nla_cfg kDefaultCfg = {32, 64, 128, 2, 1};

// Resolve the configuration: explicit opts->cfg fields, else the tuned table,
// else the defaults; band is clamped to [1, min(64, N)].
nla_cfg resolve_cfg(int m, int n, nla_dtype dt, const nla_opts *opts, int side_hint) {
    nla_cfg c = kDefaultCfg;
    nla_cfg tuned;
    int upd = opts ? (int)opts->update : 0;
    // the compensated forms run the TF32 / BF16 kernels with three products: their tuned
    // band is the base form's
    if (upd == NLA_UPD_TF32X3) upd = NLA_UPD_TF32;
    if (upd == NLA_UPD_BF16X3) upd = NLA_UPD_BF16;
    if (nla_tuned_lookup(m, n, (int)dt, upd, side_hint, &tuned)) c = tuned;
    if (opts && opts->cfg) {
        const nla_cfg *u = opts->cfg;
        if (u->band > 0) c.band = u->band;
        if (u->tile > 0) c.tile = u->tile;
        if (u->threads > 0) c.threads = u->threads;
        if (u->cols_per_block > 0) c.cols_per_block = u->cols_per_block;
        if (u->unroll > 0) c.unroll = u->unroll;
    }
    return c;
}

struct Stage1Plan {
    int b;
    nla::UpdCfg left, right;
    int update;  // nla_update
    // per-step configurations: the tuned table's entry for each step's trailing block
    // (set when the caller fixed no update parameters and a table is installed)
    bool adaptive = false;
    nla_dtype dt = NLA_F64;
};

struct Stage1Bufs {
    unsigned int *bar;
    unsigned int *tickets;  // strip tickets of the tiled update (cleared per call)
    size_t nticket;
    void *upd_work;         // partial sums / W' of the tiled update
    double *part;
    void *tauq, *taup, *Tq, *Tp;
    void *tc_scratch;
    size_t tc_bytes;
};

size_t elem_size(nla_dtype dt) { return dt == NLA_F64 ? 8 : 4; }

void carve_stage1(Carver &cv, int M, int N, nla_dtype dt, int b, int update, Stage1Bufs &s) {
    size_t es = elem_size(dt);
    s.bar = cv.take<unsigned int>(64);
    s.nticket = nla::tiled_tickets(M, N);
    s.tickets = cv.take<unsigned int>(s.nticket);
    s.upd_work = cv.take<char>(es * nla::tiled_scratch_elems(M, N));
    s.part = cv.take<double>(nla::panel_part_doubles(nla::panel_max_ctas()));
    s.tauq = cv.take<char>(es * 64);
    s.taup = cv.take<char>(es * 64);
    s.Tq = cv.take<char>(es * 64 * 64);
    s.Tp = cv.take<char>(es * 64 * 64);
    s.tc_bytes = update != NLA_UPD_NATIVE ? nla::trail_tc_scratch_bytes(M, N, b) : 0;
    s.tc_scratch = s.tc_bytes ? cv.take<char>(s.tc_bytes) : nullptr;
}

nla_status check_upd(const Stage1Plan &p, int elem) {
    if (p.update != NLA_UPD_NATIVE) return NLA_OK;
    if (!nla::upd_cfg_launchable(0, elem, p.b, p.left))
        return fail(NLA_ERR_CONFIG, "trailing-update config (tile %d, threads %d, cpb %d, unroll %d) invalid for band %d",
                    p.left.tile, p.left.threads, p.left.cpb, p.left.unroll, p.b);
    if (!nla::upd_cfg_launchable(1, elem, p.b, p.right))
        return fail(NLA_ERR_CONFIG, "LQ trailing-update config (tile %d, threads %d, cpb %d, unroll %d) invalid for band %d",
                    p.right.tile, p.right.threads, p.right.cpb, p.right.unroll, p.b);
    return NLA_OK;
}

void step_cfgs(const Stage1Plan &p, int Mt, int Nt, nla::UpdCfg &l, nla::UpdCfg &r);

template <typename T>
nla_status run_stage1(T *X, long ldx, int M, int N, const Stage1Plan &p, const Stage1Bufs &bufs,
                      T *tauq_all, T *taup_all, int *dInfo, cudaStream_t st) {
    const int b = p.b;
    nla::PanelCtl ctl{bufs.bar, bufs.part, dInfo};
    const nla::UpdScratch usc{bufs.upd_work, bufs.tickets, dInfo};
    for (int kb = 0; kb < N; kb += b) {
        const int nb = std::min(b, N - kb);
        T *tq = tauq_all ? tauq_all + kb : reinterpret_cast<T *>(bufs.tauq);
        T *tp = taup_all ? taup_all + kb : reinterpret_cast<T *>(bufs.taup);
        T *Tq = reinterpret_cast<T *>(bufs.Tq), *Tp = reinterpret_cast<T *>(bufs.Tp);
        // QR sweep: factor the tile column, then update the trailing columns
        T *panel = X + kb + (long)kb * ldx;
        NLA_LAUNCH(nla::kTrPanelQR, st, nla::panel_factor<T>(panel, 1, ldx, M - kb, nb, tq, Tq, ctl, st), "QR panel");
        const int c0 = kb + nb;
        if (c0 >= N) break;
        nla::UpdCfg cfl, cfr, unused;
        step_cfgs(p, M - kb, N - c0, cfl, unused);
        step_cfgs(p, M - c0, N - c0, unused, cfr);
        if constexpr (sizeof(T) == 8) {
            if (p.update != NLA_UPD_NATIVE) {
                NLA_LAUNCH(nla::kTrTrailLeft, st, nla::trail_left_tc(X + kb + (long)c0 * ldx, ldx, M - kb, N - c0, panel, ldx, nb, Tq,
                                            p.update, usc, dInfo, st),
                         "QR trailing update (tensor core)");
            } else {
                NLA_LAUNCH(nla::kTrTrailLeft, st, nla::trail_left<T>(X + kb + (long)c0 * ldx, ldx, M - kb, N - c0, panel, ldx, nb, Tq,
                                            cfl, usc, st),
                         "QR trailing update");
            }
        } else {
            NLA_LAUNCH(nla::kTrTrailLeft, st, nla::trail_left<T>(X + kb + (long)c0 * ldx, ldx, M - kb, N - c0, panel, ldx, nb, Tq, cfl,
                                        usc, st),
                     "QR trailing update");
        }
        // LQ sweep: factor the tile row right of the diagonal tile, update below it
        T *rowp = X + kb + (long)c0 * ldx;  // element (kb, c0); panel(r, c) = rowp[c + r*ldx]
        NLA_LAUNCH(nla::kTrPanelLQ, st, nla::panel_factor<T>(rowp, ldx, 1, N - c0, nb, tp, Tp, ctl, st), "LQ panel");
        if (M - c0 > 0) {
            T *Xr = X + c0 + (long)c0 * ldx;
            if constexpr (sizeof(T) == 8) {
                if (p.update != NLA_UPD_NATIVE) {
                    NLA_LAUNCH(nla::kTrTrailRight, st, nla::trail_right_tc(Xr, ldx, M - c0, N - c0, rowp, ldx, nb, Tp, p.update, usc, dInfo, st),
                             "LQ trailing update (tensor core)");
                    continue;
                }
            }
            NLA_LAUNCH(nla::kTrTrailRight, st, nla::trail_right<T>(Xr, ldx, M - c0, N - c0, rowp, ldx, nb, Tp, cfr, usc, st),
                     "LQ trailing update");
        }
    }
    return NLA_OK;
}

// A valid update configuration for band nb when the requested one does not fit
// (small or odd band widths): widest block first, one 32-column strip.
nla::UpdCfg fallback_upd(int side, int elem, int nb, nla::UpdCfg c) {
    size_t sm;
    if (nla::upd_cfg_launchable(side, elem, nb, c)) return c;
    (void)sm;
    const int tiles[] = {64, 32, 16, 128, 8, 4};
    const int cpbs[] = {2, 1, 4};
    for (int cpb : cpbs)
        for (int threads = 128; threads <= 1024; threads += 32)
            for (int tile : tiles) {
                nla::UpdCfg t{tile, threads, cpb, 1};
                if (nla::upd_cfg_launchable(side, elem, nb, t)) return t;
            }
    for (int threads = 96; threads >= 32; threads -= 32)
        for (int tile : tiles) {
            nla::UpdCfg t{tile, threads, 1, 1};
            if (nla::upd_cfg_launchable(side, elem, nb, t)) return t;
        }
    return c;
}

Stage1Plan make_plan(int M, int N, nla_dtype dt, const nla_opts *opts, int band_override) {
    nla_cfg cl = resolve_cfg(M, N, dt, opts, 0);
    nla_cfg cr = resolve_cfg(M, N, dt, opts, 1);
    Stage1Plan p;
    p.b = band_override > 0 ? band_override : cl.band;
    p.b = std::max(1, std::min({p.b, 64, std::max(N, 1)}));
    p.left = {cl.tile, cl.threads, cl.cols_per_block, cl.unroll};
    p.right = {cr.tile, cr.threads, cr.cols_per_block, cr.unroll};
    p.update = opts ? (int)opts->update : 0;
    const nla_cfg *u = opts ? opts->cfg : nullptr;
    const bool explicit_upd = u && (u->tile > 0 || u->threads > 0 || u->cols_per_block > 0 || u->unroll > 0);
    if (!explicit_upd) {  // defaults / tuned entries adapt to the band actually used
        const int es = (int)elem_size(dt);
        p.left = fallback_upd(0, es, p.b, p.left);
        p.right = fallback_upd(1, es, p.b, p.right);
        nla_cfg probe;
        p.adaptive = p.update == NLA_UPD_NATIVE && nla_tuned_lookup(M, N, (int)dt, 0, 0, &probe);
        p.dt = dt;
    }
    return p;
}

// The update configurations of one stage-1 step whose trailing block is Mt x Nt: the
// tuned entry nearest to that size (kernel-level parameters only; the band stays the
// plan's), made valid for the band.
void step_cfgs(const Stage1Plan &p, int Mt, int Nt, nla::UpdCfg &l, nla::UpdCfg &r) {
    l = p.left;
    r = p.right;
    if (!p.adaptive) return;
    const int es = (int)elem_size(p.dt);
    nla_cfg t;
    if (nla_tuned_lookup(Mt, Nt, (int)p.dt, 0, 0, &t)) l = fallback_upd(0, es, p.b, {t.tile, t.threads, t.cols_per_block, t.unroll});
    if (nla_tuned_lookup(Mt, Nt, (int)p.dt, 0, 1, &t)) r = fallback_upd(1, es, p.b, {t.tile, t.threads, t.cols_per_block, t.unroll});
}

nla_status check_common(nla_dtype dt, const nla_opts *opts) {
    if (dt != NLA_F64 && dt != NLA_F32) return fail(NLA_ERR_ARG, "unknown dtype %d", (int)dt);
    if (opts && (opts->update < NLA_UPD_NATIVE || opts->update > NLA_UPD_BF16X3))
        return fail(NLA_ERR_ARG, "unknown update precision %d", (int)opts->update);
    if (opts && opts->update != NLA_UPD_NATIVE && dt != NLA_F64)
        return fail(NLA_ERR_ARG, "TF32/BF16 trailing updates are defined for FP64 matrices");
    if (opts && opts->update != NLA_UPD_NATIVE && !nla::trail_tc_available())
        return fail(NLA_ERR_UNSUPPORTED, "tensor-core trailing update not available in this build");
    return NLA_OK;
}

struct GesvdLayout {
    Stage1Bufs s1;
    void *Aw;
    long ldw;
    void *AB;
    long ldab;
    void *prog;
    void *bd;  // bisection scratch
    double *d, *e;
    size_t bytes;
};

GesvdLayout gesvd_layout(char *base, int m, int n, nla_dtype dt, const nla_opts *opts, const Stage1Plan &p) {
    const int M = std::max(m, n), N = std::min(m, n);
    const bool need_copy = (m < n) || (opts && opts->preserve_a);
    size_t es = elem_size(dt);
    GesvdLayout L;
    Carver cv{base};
    carve_stage1(cv, M, N, dt, p.b, p.update, L.s1);
    L.ldw = (long)align_up((size_t)std::max(M, 1), 32);
    L.Aw = need_copy ? cv.take<char>(es * L.ldw * N) : nullptr;
    L.ldab = 3 * p.b + 1;
    L.AB = cv.take<char>(es * L.ldab * std::max(N, 1));
    L.prog = cv.take<char>(nla::band2bd_scratch_bytes(N));
    L.bd = cv.take<char>(nla::bdsvd_scratch_bytes(N));
    L.d = cv.take<double>(std::max(N, 1));
    L.e = cv.take<double>(std::max(N, 1));
    L.bytes = align_up(cv.off, 256);
    return L;
}

template <typename T>
nla_status gesvd_impl(int m, int n, nla_dtype dt, T *dA, int lda, T *dS, const GesvdLayout &L,
                      const Stage1Plan &p, const nla_opts *opts, int *dInfo, cudaStream_t st) {
    const int M = std::max(m, n), N = std::min(m, n);
    const bool transpose = m < n;
    const bool need_copy = transpose || (opts && opts->preserve_a);
    NLA_CUDA(cudaMemsetAsync(L.s1.bar, 0, 64 * sizeof(unsigned int), st), "memset control");
    NLA_CUDA(cudaMemsetAsync(L.s1.tickets, 0, L.s1.nticket * sizeof(unsigned int), st), "memset tickets");
    NLA_CUDA(cudaMemsetAsync(dInfo, 0, sizeof(int), st), "memset info");
    T *X = dA;
    long ldx = lda;
    if (need_copy) {
        X = reinterpret_cast<T *>(L.Aw);
        ldx = L.ldw;
        NLA_LAUNCH(nla::kTrStageCopy, st, nla::copy_matrix<T>(dA, lda, m, n, X, ldx, transpose, st), "input staging");
    }
    nla_status s = run_stage1<T>(X, ldx, M, N, p, L.s1, nullptr, nullptr, dInfo, st);
    if (s != NLA_OK) return s;
    T *AB = reinterpret_cast<T *>(L.AB);
    NLA_LAUNCH(nla::kTrBandExtract, st, nla::band_extract<T>(X, ldx, N, p.b, AB, L.ldab, st), "band extract");
    NLA_LAUNCH(nla::kTrBand2bd, st, nla::band2bd<T>(AB, L.ldab, N, p.b, L.d, L.e, L.prog, dInfo, st), "bulge chase");
    NLA_LAUNCH(nla::kTrBisect, st, nla::bdsvd_bisect<T>(N, L.d, L.e, dS, L.bd, dInfo, st), "bidiagonal singular values");
    (void)dt;
    return NLA_OK;
}

}  // namespace

extern "C" {

const char *nla_last_error(void) { return g_last_error.c_str(); }

void nla_set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

const char *nla_version(void) { return "nla-gb300 0.1 (sm_103a)"; }

nla_status nla_gesvd_vals_workspace(int m, int n, nla_dtype dtype, const nla_opts *opts, size_t *bytes) {
    if (!bytes) return fail(NLA_ERR_ARG, "bytes is NULL");
    nla_status s = check_common(dtype, opts);
    if (s != NLA_OK) return s;
    if (m < 0 || n < 0) return fail(NLA_ERR_ARG, "negative size %d x %d", m, n);
    const int M = std::max(m, n), N = std::min(m, n);
    Stage1Plan p = make_plan(M, N, dtype, opts, 0);
    s = check_upd(p, (int)elem_size(dtype));
    if (s != NLA_OK) return s;
    *bytes = gesvd_layout(nullptr, m, n, dtype, opts, p).bytes;
    return NLA_OK;
}

nla_status nla_gesvd_vals(int m, int n, nla_dtype dtype, void *dA, int lda, void *dS, void *dWork,
                          size_t work_bytes, int *dInfo, const nla_opts *opts, nla_stream_t stream) {
    nla_status s = check_common(dtype, opts);
    if (s != NLA_OK) return s;
    if (m < 0 || n < 0) return fail(NLA_ERR_ARG, "negative size %d x %d", m, n);
    if (m == 0 || n == 0) return NLA_OK;
    if (!dA || !dS || !dInfo) return fail(NLA_ERR_ARG, "null device pointer");
    if (lda < std::max(m, 1)) return fail(NLA_ERR_ARG, "lda %d < m %d", lda, m);
    if (((uintptr_t)dWork) % 256) return fail(NLA_ERR_WORKSPACE, "workspace not 256-byte aligned");
    const int M = std::max(m, n), N = std::min(m, n);
    Stage1Plan p = make_plan(M, N, dtype, opts, 0);
    s = check_upd(p, (int)elem_size(dtype));
    if (s != NLA_OK) return s;
    GesvdLayout L = gesvd_layout(reinterpret_cast<char *>(dWork), m, n, dtype, opts, p);
    if (!dWork || work_bytes < L.bytes)
        return fail(NLA_ERR_WORKSPACE, "workspace %zu bytes < required %zu", work_bytes, L.bytes);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (dtype == NLA_F64)
        return gesvd_impl<double>(m, n, dtype, (double *)dA, lda, (double *)dS, L, p, opts, dInfo, st);
    return gesvd_impl<float>(m, n, dtype, (float *)dA, lda, (float *)dS, L, p, opts, dInfo, st);
}

nla_status nla_plan_cfg(int m, int n, nla_dtype dtype, const nla_opts *opts, int side, nla_cfg *out) {
    if (!out || (side != 0 && side != 1)) return fail(NLA_ERR_ARG, "bad arguments");
    nla_status s = check_common(dtype, opts);
    if (s != NLA_OK) return s;
    if (m < 0 || n < 0) return fail(NLA_ERR_ARG, "negative size");
    const int M = std::max(m, n), N = std::min(m, n);
    Stage1Plan p = make_plan(M, N, dtype, opts, 0);
    const nla::UpdCfg &u = side == 0 ? p.left : p.right;
    *out = nla_cfg{p.b, u.tile, u.threads, u.cpb, u.unroll};
    return NLA_OK;
}

nla_status nla_gebrd_band_workspace(int m, int n, int band, nla_dtype dtype, const nla_opts *opts,
                                    size_t *bytes) {
    if (!bytes) return fail(NLA_ERR_ARG, "bytes is NULL");
    nla_status s = check_common(dtype, opts);
    if (s != NLA_OK) return s;
    if (m < n || n < 0) return fail(NLA_ERR_ARG, "gebrd_band needs m >= n >= 0 (got %d x %d)", m, n);
    Stage1Plan p = make_plan(m, n, dtype, opts, band);
    s = check_upd(p, (int)elem_size(dtype));
    if (s != NLA_OK) return s;
    Stage1Bufs b;
    Carver cv{nullptr};
    carve_stage1(cv, m, n, dtype, p.b, p.update, b);
    *bytes = align_up(cv.off, 256);
    return NLA_OK;
}

nla_status nla_gebrd_band(int m, int n, int band, nla_dtype dtype, void *dA, int lda, void *dTauQ,
                          void *dTauP, void *dWork, size_t work_bytes, int *dInfo, const nla_opts *opts,
                          nla_stream_t stream) {
    nla_status s = check_common(dtype, opts);
    if (s != NLA_OK) return s;
    if (m < n || n < 0) return fail(NLA_ERR_ARG, "gebrd_band needs m >= n >= 0 (got %d x %d)", m, n);
    if (band < 1 || band > 64) return fail(NLA_ERR_ARG, "band %d outside [1, 64]", band);
    if (n == 0) return NLA_OK;
    if (!dA || !dInfo) return fail(NLA_ERR_ARG, "null device pointer");
    if (lda < std::max(m, 1)) return fail(NLA_ERR_ARG, "lda %d < m %d", lda, m);
    if (((uintptr_t)dWork) % 256) return fail(NLA_ERR_WORKSPACE, "workspace not 256-byte aligned");
    Stage1Plan p = make_plan(m, n, dtype, opts, band);
    s = check_upd(p, (int)elem_size(dtype));
    if (s != NLA_OK) return s;
    Stage1Bufs b;
    Carver cv{reinterpret_cast<char *>(dWork)};
    carve_stage1(cv, m, n, dtype, p.b, p.update, b);
    if (!dWork || work_bytes < align_up(cv.off, 256))
        return fail(NLA_ERR_WORKSPACE, "workspace %zu bytes < required %zu", work_bytes, align_up(cv.off, 256));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    NLA_CUDA(cudaMemsetAsync(b.bar, 0, 64 * sizeof(unsigned int), st), "memset control");
    NLA_CUDA(cudaMemsetAsync(b.tickets, 0, b.nticket * sizeof(unsigned int), st), "memset tickets");
    NLA_CUDA(cudaMemsetAsync(dInfo, 0, sizeof(int), st), "memset info");
    if (dtype == NLA_F64)
        return run_stage1<double>((double *)dA, lda, m, n, p, b, (double *)dTauQ, (double *)dTauP, dInfo, st);
    return run_stage1<float>((float *)dA, lda, m, n, p, b, (float *)dTauQ, (float *)dTauP, dInfo, st);
}

nla_status nla_band_extract(int n, int band, nla_dtype dtype, const void *dA, int lda, void *dAB, int ldab,
                            nla_stream_t stream) {
    if (dtype != NLA_F64 && dtype != NLA_F32) return fail(NLA_ERR_ARG, "unknown dtype %d", (int)dtype);
    if (n < 0 || band < 1 || band > 64) return fail(NLA_ERR_ARG, "bad n %d or band %d", n, band);
    if (n == 0) return NLA_OK;
    if (!dA || !dAB) return fail(NLA_ERR_ARG, "null device pointer");
    if (lda < n || ldab < 3 * band + 1) return fail(NLA_ERR_ARG, "lda %d < n or ldab %d < 3*band+1", lda, ldab);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (dtype == NLA_F64)
        NLA_LAUNCH(nla::kTrBandExtract, st, nla::band_extract<double>((const double *)dA, lda, n, band, (double *)dAB, ldab, st), "band extract");
    else
        NLA_LAUNCH(nla::kTrBandExtract, st, nla::band_extract<float>((const float *)dA, lda, n, band, (float *)dAB, ldab, st), "band extract");
    return NLA_OK;
}

nla_status nla_band2bd_workspace(int n, int band, nla_dtype dtype, size_t *bytes) {
    (void)band;
    (void)dtype;
    if (!bytes || n < 0) return fail(NLA_ERR_ARG, "bad arguments");
    *bytes = align_up(nla::band2bd_scratch_bytes(n), 256);
    return NLA_OK;
}

nla_status nla_band2bd(int n, int band, nla_dtype dtype, void *dAB, int ldab, double *dD, double *dE, void *dWork,
                       size_t work_bytes, int *dInfo, const nla_opts *opts, nla_stream_t stream) {
    (void)opts;
    if (dtype != NLA_F64 && dtype != NLA_F32) return fail(NLA_ERR_ARG, "unknown dtype %d", (int)dtype);
    if (n < 0 || band < 1 || band > 64) return fail(NLA_ERR_ARG, "bad n %d or band %d", n, band);
    if (n == 0) return NLA_OK;
    if (!dAB || !dD || !dE || !dInfo) return fail(NLA_ERR_ARG, "null device pointer");
    if (ldab < 3 * band + 1) return fail(NLA_ERR_ARG, "ldab %d < 3*band+1", ldab);
    if (!dWork || work_bytes < nla::band2bd_scratch_bytes(n))
        return fail(NLA_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    NLA_CUDA(cudaMemsetAsync(dInfo, 0, sizeof(int), st), "memset info");
    if (dtype == NLA_F64)
        NLA_LAUNCH(nla::kTrBand2bd, st, nla::band2bd<double>((double *)dAB, ldab, n, band, dD, dE, dWork, dInfo, st), "bulge chase");
    else
        NLA_LAUNCH(nla::kTrBand2bd, st, nla::band2bd<float>((float *)dAB, ldab, n, band, dD, dE, dWork, dInfo, st), "bulge chase");
    return NLA_OK;
}

nla_status nla_bdsvd_vals_workspace(int n, size_t *bytes) {
    if (!bytes || n < 0) return fail(NLA_ERR_ARG, "bad arguments");
    *bytes = align_up(nla::bdsvd_scratch_bytes(n), 256);
    return NLA_OK;
}

nla_status nla_bdsvd_vals(int n, const double *dD, const double *dE, void *dS, nla_dtype dtype, void *dWork,
                          size_t work_bytes, int *dInfo, nla_stream_t stream) {
    if (dtype != NLA_F64 && dtype != NLA_F32) return fail(NLA_ERR_ARG, "unknown dtype %d", (int)dtype);
    if (n < 0) return fail(NLA_ERR_ARG, "negative n");
    if (n == 0) return NLA_OK;
    if (!dD || !dS || !dInfo || (n > 1 && !dE)) return fail(NLA_ERR_ARG, "null device pointer");
    if (!dWork || work_bytes < nla::bdsvd_scratch_bytes(n) || ((uintptr_t)dWork) % 256)
        return fail(NLA_ERR_WORKSPACE, "workspace too small or misaligned");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    NLA_CUDA(cudaMemsetAsync(dInfo, 0, sizeof(int), st), "memset info");
    if (dtype == NLA_F64)
        NLA_LAUNCH(nla::kTrBisect, st, nla::bdsvd_bisect<double>(n, dD, dE, (double *)dS, dWork, dInfo, st), "bisection");
    else
        NLA_LAUNCH(nla::kTrBisect, st, nla::bdsvd_bisect<float>(n, dD, dE, (float *)dS, dWork, dInfo, st), "bisection");
    return NLA_OK;
}

}  // extern "C"
