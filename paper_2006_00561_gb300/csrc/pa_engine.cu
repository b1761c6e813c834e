// pa_engine.cu -- host side of the C ABI declared in include/pa.h.
//
// The engine validates a run's configuration, lays the run out in the
// caller's device workspace, builds the per-step host tables (beta schedule,
// Metropolis thresholds, Eq. 3 weights) in IEEE double, and enqueues the
// kernels of pa_sweep.cu / pa_resample.cu on the caller's stream.  It never
// allocates device memory.
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <array>
#include <new>
#include <vector>

#include "pa_internal.cuh"

using pa::RunDev;
using pa::DevState;

struct pa_run {
    pa_config cfg;
    cudaStream_t stream;
    RunDev d;
    int sweep_grid;
    std::vector<uint32_t> thr;
    std::vector<double> beta, dbeta, dtab;
    std::vector<uint32_t> dsel;
    uint32_t ndist;  // weight tables of the fixed schedule
    // the fixed schedule, kept to undo the per-step overrides of pa_resample_to
    std::vector<uint32_t> thr_fixed, dsel_fixed;
    std::vector<double> beta_fixed, dbeta_fixed;
    std::vector<double> dyn_table[2];  // host copies of the two dynamic weight slots
    DevState init_state;
    cudaStream_t cap_stream;
    cudaGraphExec_t graph;
    size_t hist_bytes;  // accum (16 B) + histogram
    // kernel timing
    bool prof;
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> ev_pool;
    std::vector<Pending> pending;
    int64_t prof_n[4];
    double prof_ms[4];
    uint32_t load_R;  // source of the population size written by pa_load
    // pa_step_stream: a range's sweeps are done / the last copy is done
    cudaEvent_t ev_range, ev_copied;
    // pa_resample_begin has run the counts and scan; the gather waits for
    // pa_resample_finish
    bool gather_pending;
};

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    int64_t N, bins, nrows, NW, nwords, stride, cap, tiles, ndist;
    size_t mn_cum, mn_tiles;
    size_t state, obs, thr, beta, dbeta, dsel, dtab, accum, tabn, tabF, desc, coup, ebin[2], mag[2],
        counts, offsets, srcmap, srcmap2, spins[2], total;
};

// beta_i = beta0 + (beta_max - beta0) * i / K (constant step, Sec. 3).
double beta_of(const pa_config* c, int32_t i) {
    return c->beta0 + ((c->beta_max - c->beta0) * (double)i) / (double)c->K;
}

// floor(2^32 exp(-beta dE)): u < T accepts with probability exp(-beta dE).
uint64_t threshold_of(double beta, int32_t dE) {
    const double x = -(beta * (double)dE);
    return (uint64_t)std::floor(std::exp(x) * 4294967296.0);
}

// exp(-|dbeta| 4 j): Eq. 3 weight of the level j steps away from the reference
// level (lowest occupied when cooling, highest when heating).
double weight_of(double dbeta, int64_t j) { return std::exp(-(std::fabs(dbeta) * (double)(4 * j))); }

int64_t ipow(int64_t a, int b) {
    int64_t r = 1;
    for (int i = 0; i < b; ++i) r *= a;
    return r;
}

int validate(const pa_config* c) {
    if (!c) return PA_ERR_INVALID_ARG;
    if (c->dim != 2 && c->dim != 3) return PA_ERR_INVALID_ARG;
    if (c->L < 2) return PA_ERR_INVALID_ARG;
    if (c->L & 1) return PA_ERR_ODD_L;
    if (c->layout != PA_LAYOUT_INT8 && c->layout != PA_LAYOUT_PACKED) return PA_ERR_INVALID_ARG;
    if (c->model != PA_MODEL_FERRO && c->model != PA_MODEL_PMJ) return PA_ERR_INVALID_ARG;
    if (c->K < 1 || c->theta < 0) return PA_ERR_INVALID_ARG;
    if (c->init != PA_INIT_RANDOM && c->init != PA_INIT_GROUND) return PA_ERR_INVALID_ARG;
    if (c->init == PA_INIT_GROUND && c->model != PA_MODEL_FERRO) return PA_ERR_INVALID_ARG;
    if (c->resample != PA_RESAMPLE_NEAREST && c->resample != PA_RESAMPLE_POISSON &&
        c->resample != PA_RESAMPLE_MULTINOMIAL)
        return PA_ERR_INVALID_ARG;
    if (c->reserved != 0) return PA_ERR_INVALID_ARG;
    if (c->instance_id < 0 || c->instance_id >= (1 << 28)) return PA_ERR_INVALID_ARG;
    if (c->R0 < 1 || c->R0 > (int64_t(1) << 31)) return PA_ERR_INVALID_ARG;
    if (!std::isfinite(c->beta0) || !std::isfinite(c->beta_max) || c->beta0 < 0.0 ||
        c->beta_max < 0.0)
        return PA_ERR_INVALID_ARG;
    if (c->capacity != 0 && (c->capacity < c->R0 || c->capacity > (int64_t(1) << 31)))
        return PA_ERR_INVALID_ARG;
    if (!pa::sweep_supported(c->layout, c->dim, c->L)) return PA_ERR_UNSUPPORTED;
    return PA_OK;
}

// Poisson(1) distribution function scaled to 32 bits: the probabilities
// e^-1 / m! by the recurrence p_m = p_{m-1} / m, accumulated in order of m,
// each partial sum truncated to floor(2^32 P); the table ends at the first
// entry that saturates at 2^32 - 1.
int poisson1_table(uint32_t* T, int cap) {
    double p = std::exp(-1.0);
    double acc = 0.0;
    int m = 0;
    while (m < cap) {
        acc = acc + p;
        const double scaled = std::floor(std::ldexp(acc, 32));
        const bool top = !(scaled < 4294967295.0);
        T[m] = top ? 0xffffffffu : (uint32_t)scaled;
        ++m;
        if (top) break;
        p = p / (double)m;
    }
    return m;
}

// Schedule and deduplicated weight tables (one per distinct dbeta bit pattern).
void schedule(const pa_config* c, int64_t bins, std::vector<double>& beta,
              std::vector<double>& dbeta, std::vector<uint32_t>& dsel, std::vector<double>* dtab,
              int64_t* ndist) {
    beta.assign(c->K + 1, 0.0);
    dbeta.assign(c->K + 1, 0.0);
    dsel.assign(c->K + 1, 0u);
    for (int32_t i = 0; i <= c->K; ++i) beta[i] = beta_of(c, i);
    std::vector<double> uniq;
    for (int32_t i = 1; i <= c->K; ++i) {
        dbeta[i] = beta[i] - beta[i - 1];
        const double mag = std::fabs(dbeta[i]);  // tables depend on |dbeta| only
        size_t j = 0;
        while (j < uniq.size() && std::memcmp(&uniq[j], &mag, sizeof(double)) != 0) ++j;
        if (j == uniq.size()) uniq.push_back(mag);
        dsel[i] = (uint32_t)j;
    }
    if (uniq.empty()) uniq.push_back(0.0);
    *ndist = (int64_t)uniq.size();
    if (dtab) {
        dtab->assign((size_t)(uniq.size() * bins), 0.0);
        for (size_t u = 0; u < uniq.size(); ++u)
            for (int64_t j = 0; j < bins; ++j) (*dtab)[u * bins + j] = weight_of(uniq[u], j);
    }
}

int make_layout(const pa_config* c, Layout* Lo, std::vector<double>* beta, std::vector<double>* dbeta,
                std::vector<uint32_t>* dsel, std::vector<double>* dtab) {
    int rc = validate(c);
    if (rc) return rc;
    Layout& l = *Lo;
    l.N = ipow(c->L, c->dim);
    l.bins = (int64_t)c->dim * l.N / 2 + 1;
    l.nrows = c->dim == 2 ? c->L : (int64_t)c->L * c->L;
    l.NW = (c->L + 31) / 32;
    l.nwords = l.nrows * l.NW;
    l.stride = c->layout == PA_LAYOUT_PACKED ? (l.nwords * 4 + 15) / 16 * 16 : (l.N + 15) / 16 * 16;
    l.cap = c->capacity > 0 ? c->capacity
                            : c->R0 + 16 * (int64_t)std::ceil(std::sqrt((double)c->R0)) + 1024;
    if (l.cap > (int64_t(1) << 31)) return PA_ERR_INVALID_ARG;
    l.tiles = (l.cap + pa::RS_TILE - 1) / pa::RS_TILE;
    std::vector<double> b, db;
    std::vector<uint32_t> ds;
    schedule(c, l.bins, beta ? *beta : b, dbeta ? *dbeta : db, dsel ? *dsel : ds, dtab, &l.ndist);
    const size_t K1 = (size_t)c->K + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    l.state = take(256);
    l.obs = take(K1 * sizeof(pa_obs));
    l.thr = take(K1 * 16);
    l.beta = take(K1 * 8);
    l.dbeta = take(K1 * 8);
    l.dsel = take(K1 * 4);
    l.dtab = take((size_t)((l.ndist + 2) * l.bins * 8));  // + two dynamic slots
    l.accum = take(16 + (size_t)l.bins * 4);
    l.tabn = take((size_t)l.bins * 4);
    l.tabF = take((size_t)l.bins * 4);
    l.desc = take((size_t)l.tiles * 8);
    l.mn_cum = l.mn_tiles = 0;
    if (c->resample == PA_RESAMPLE_MULTINOMIAL) {
        l.mn_cum = take((size_t)l.cap * 8);
        l.mn_tiles = take((size_t)(l.tiles + 1) * 8);
    }
    if (c->model == PA_MODEL_PMJ)
        l.coup = take(c->layout == PA_LAYOUT_PACKED ? (size_t)(c->dim * l.nwords * 4)
                                                    : (size_t)(l.N * c->dim));
    else
        l.coup = 0;
    for (int b2 = 0; b2 < 2; ++b2) l.ebin[b2] = take((size_t)l.cap * 4);
    for (int b2 = 0; b2 < 2; ++b2) l.mag[b2] = take((size_t)l.cap * 4);
    l.counts = take((size_t)l.cap * 4);
    l.offsets = take((size_t)l.cap * 4);
    l.srcmap = take((size_t)l.cap * 4);
    l.srcmap2 = take((size_t)l.cap * 4);
    for (int b2 = 0; b2 < 2; ++b2) l.spins[b2] = take((size_t)(l.cap * l.stride));
    l.total = off;
    return PA_OK;
}

#define CK(call)                                   \
    do {                                           \
        if ((call) != cudaSuccess) return PA_ERR_CUDA; \
    } while (0)

int sticky_to_code(uint32_t bits) {
    if (bits & pa::ST_TIMEOUT) return PA_ERR_TIMEOUT;
    if (bits & pa::ST_CAPACITY) return PA_ERR_CAPACITY;
    if (bits & pa::ST_INVARIANT) return PA_ERR_INVARIANT;
    if (bits & pa::ST_EMPTY) return PA_ERR_EMPTY;
    if (bits & pa::ST_DONE) return PA_ERR_DONE;
    return PA_OK;
}

int read_state(pa_run* r, DevState* out) {
    CK(cudaStreamSynchronize(r->stream));
    CK(cudaMemcpy(out, r->d.st, sizeof(DevState), cudaMemcpyDeviceToHost));
    return PA_OK;
}

cudaEvent_t take_event(pa_run* r) {
    if (!r->ev_pool.empty()) {
        cudaEvent_t e = r->ev_pool.back();
        r->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launches one kernel; brackets it with events when timing is on and the
// launch goes to the run's own stream (not into a graph capture).
template <class F>
int timed(pa_run* r, cudaStream_t s, int kind, F&& launch) {
    if (!r->prof || s != r->stream) {
        CK(launch());
        return PA_OK;
    }
    cudaEvent_t a = take_event(r), b = take_event(r);
    if (!a || !b) return PA_ERR_CUDA;
    CK(cudaEventRecord(a, s));
    CK(launch());
    CK(cudaEventRecord(b, s));
    r->pending.push_back({kind, a, b});
    return PA_OK;
}

int enqueue_sweep(pa_run* r, cudaStream_t s, int32_t nsweeps) {
    CK(cudaMemsetAsync(r->d.accum, 0, r->hist_bytes, s));
    int rc = timed(r, s, 2, [&] { return pa::launch_sweep(r->d, nsweeps, r->sweep_grid, s); });
    if (rc) return rc;
    return timed(r, s, 3, [&] { return pa::launch_obs(r->d, nsweeps, s); });
}

int enqueue_resample(pa_run* r, cudaStream_t s) {
    int rc = timed(r, s, 0, [&] { return pa::launch_tau(r->d, s); });
    if (rc) return rc;
    return timed(r, s, 1, [&] {
        if (r->cfg.resample == PA_RESAMPLE_MULTINOMIAL) {
            const cudaError_t e = pa::launch_multinomial(r->d, s);
            if (e != cudaSuccess) return e;
        }
        return pa::launch_resample(r->d, s);
    });
}

// Metropolis thresholds of the three dE classes at beta, and the mask of the
// classes that always accept.
void thresholds_into(double beta, uint32_t* t4) {
    uint32_t full = 0;
    for (int c = 0; c < 3; ++c) {
        const uint64_t T = threshold_of(beta, 4 * (c + 1));
        if (T >= 4294967296ull) {
            full |= 1u << c;
            t4[c] = 0xffffffffu;
        } else {
            t4[c] = (uint32_t)T;
        }
    }
    t4[3] = full;
}

// Moves step i of the schedule to inverse temperature b, with temperature step
// b - beta[i-1]: the thresholds, beta and dbeta of step i are replaced, and its
// weight table goes to dynamic slot i & 1 unless the fixed schedule already
// has this exact step.  Host copies first, then stream-ordered uploads.
int set_step(pa_run* r, uint32_t i, double b, cudaStream_t s) {
    RunDev& d = r->d;
    r->beta[i] = b;
    thresholds_into(b, &r->thr[(size_t)i * 4]);
    if (i >= 1) {
        r->dbeta[i] = b - r->beta[i - 1];
        if (r->dbeta[i] == r->dbeta_fixed[i]) {
            r->dsel[i] = r->dsel_fixed[i];
        } else {
            std::vector<double>& t = r->dyn_table[i & 1];
            t.resize((size_t)d.bins);
            for (int64_t j = 0; j < d.bins; ++j) t[j] = weight_of(r->dbeta[i], j);
            r->dsel[i] = r->ndist + (i & 1);
            CK(cudaMemcpyAsync((void*)(d.dtab + (size_t)r->dsel[i] * d.bins), t.data(),
                               (size_t)d.bins * 8, cudaMemcpyHostToDevice, s));
        }
        CK(cudaMemcpyAsync((void*)(d.dbeta + i), &r->dbeta[i], 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync((void*)(d.dsel + i), &r->dsel[i], 4, cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemcpyAsync((void*)(d.beta + i), &r->beta[i], 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void*)(d.thr + (size_t)i * 4), &r->thr[(size_t)i * 4], 16,
                       cudaMemcpyHostToDevice, s));
    return PA_OK;
}

// Step i at beta_i; step i + 1 keeps its fixed beta, with its temperature step
// taken from beta_i.
int move_step(pa_run* r, uint32_t i, double b, cudaStream_t s) {
    int rc = set_step(r, i, b, s);
    if (rc == PA_OK && i + 1 <= (uint32_t)r->cfg.K) rc = set_step(r, i + 1, r->beta_fixed[i + 1], s);
    return rc;
}

int enqueue_step(pa_run* r, cudaStream_t s) {
    int rc = enqueue_resample(r, s);
    if (rc) return rc;
    return enqueue_sweep(r, s, r->cfg.theta);
}

}  // namespace

extern "C" {

int pa_poisson1_table(uint32_t* T, int32_t cap) {
    if (!T || cap < 1) return PA_ERR_INVALID_ARG;
    uint32_t full[pa::P1_MAX];
    const int n = poisson1_table(full, pa::P1_MAX);
    for (int m = 0; m < n && m < cap; ++m) T[m] = full[m];
    return n;
}

int64_t pa_num_bins(int32_t dim, int32_t L) {
    if ((dim != 2 && dim != 3) || L < 1) return 0;
    return (int64_t)dim * ipow(L, dim) / 2 + 1;
}

size_t pa_workspace_size(const pa_config* cfg) {
    Layout l;
    if (make_layout(cfg, &l, nullptr, nullptr, nullptr, nullptr)) return 0;
    return l.total;
}

int pa_tables(const pa_config* cfg, int32_t step, uint64_t T[3], double* D, int64_t bins) {
    int rc = validate(cfg);
    if (rc) return rc;
    if (step < 0 || step > cfg->K || !T) return PA_ERR_INVALID_ARG;
    const double b = beta_of(cfg, step);
    for (int c = 0; c < 3; ++c) T[c] = threshold_of(b, 4 * (c + 1));
    if (D && step >= 1) {
        const double db = b - beta_of(cfg, step - 1);
        for (int64_t j = 0; j < bins; ++j) D[j] = weight_of(db, j);
    }
    return PA_OK;
}

int pa_init(const pa_config* cfg, void* ws, size_t bytes, void* stream, pa_run** out) {
    if (!out) return PA_ERR_INVALID_ARG;
    *out = nullptr;
    Layout l;
    std::vector<double> beta, dbeta, dtab;
    std::vector<uint32_t> dsel;
    int rc = make_layout(cfg, &l, &beta, &dbeta, &dsel, &dtab);
    if (rc) return rc;
    if (!ws || ((uintptr_t)ws % ALIGN) != 0 || bytes < l.total) return PA_ERR_WORKSPACE;

    pa_run* r = new (std::nothrow) pa_run();
    if (!r) return PA_ERR_INVALID_ARG;
    r->cfg = *cfg;
    r->stream = (cudaStream_t)stream;
    r->beta = beta;
    r->dbeta = dbeta;
    r->dsel = dsel;
    r->dtab = dtab;
    r->ndist = (uint32_t)l.ndist;
    r->cap_stream = nullptr;
    r->graph = nullptr;
    r->ev_range = r->ev_copied = nullptr;
    r->prof = false;
    for (int k = 0; k < 4; ++k) {
        r->prof_n[k] = 0;
        r->prof_ms[k] = 0.0;
    }
    r->load_R = 0;
    r->thr.assign((size_t)(cfg->K + 1) * 4, 0u);
    for (int32_t i = 0; i <= cfg->K; ++i) thresholds_into(beta[i], &r->thr[(size_t)i * 4]);
    r->thr_fixed = r->thr;
    r->dsel_fixed = r->dsel;
    r->beta_fixed = r->beta;
    r->dbeta_fixed = r->dbeta;

    uint8_t* base = (uint8_t*)ws;
    RunDev& d = r->d;
    std::memset(&d, 0, sizeof(d));
    d.st = (DevState*)(base + l.state);
    for (int b2 = 0; b2 < 2; ++b2) {
        d.spins[b2] = base + l.spins[b2];
        d.ebin[b2] = (uint32_t*)(base + l.ebin[b2]);
        d.mag[b2] = (int32_t*)(base + l.mag[b2]);
    }
    d.counts = (uint32_t*)(base + l.counts);
    d.offsets = (uint32_t*)(base + l.offsets);
    d.srcmap = (uint32_t*)(base + l.srcmap);
    d.srcmap2 = (uint32_t*)(base + l.srcmap2);
    d.accum = (unsigned long long*)(base + l.accum);
    d.hist = (uint32_t*)(base + l.accum + 16);
    d.tab_n = (uint32_t*)(base + l.tabn);
    d.tab_F = (uint32_t*)(base + l.tabF);
    d.thr = (const uint32_t*)(base + l.thr);
    d.dtab = (const double*)(base + l.dtab);
    d.dsel = (const uint32_t*)(base + l.dsel);
    d.beta = (const double*)(base + l.beta);
    d.dbeta = (const double*)(base + l.dbeta);
    d.desc = (unsigned long long*)(base + l.desc);
    d.obs = (pa_obs*)(base + l.obs);
    if (cfg->model == PA_MODEL_PMJ) {
        if (cfg->layout == PA_LAYOUT_PACKED) d.jpk = (uint32_t*)(base + l.coup);
        else d.j8 = (int8_t*)(base + l.coup);
    }
    d.seed = cfg->seed;
    d.coupling_seed = cfg->coupling_seed;
    d.one = 1u;
    d.slot_lo = 0u;
    d.slot_hi = 0xffffffffu;
    d.theta = cfg->theta;
    d.init = cfg->init;
    d.resample = cfg->resample;
    d.p1_len = (uint32_t)poisson1_table(d.p1, pa::P1_MAX);
    for (int k = 0; k < 10; ++k) {
        d.rk0[k] = (uint32_t)cfg->seed + (uint32_t)k * 0x9E3779B9u;
        d.rk1[k] = (uint32_t)(cfg->seed >> 32) + (uint32_t)k * 0xBB67AE85u;
    }
    d.instance = (uint32_t)cfg->instance_id;
    d.dim = cfg->dim;
    d.L = cfg->L;
    d.layout = cfg->layout;
    d.model = cfg->model;
    d.K = cfg->K;
    d.N = l.N;
    d.bins = l.bins;
    d.stride = (uint32_t)l.stride;
    d.nwords = (uint32_t)l.nwords;
    d.cap = (uint32_t)l.cap;
    d.cap_alloc = (uint32_t)l.cap;
    d.R0 = (uint32_t)cfg->R0;
    d.tiles = (uint32_t)l.tiles;
    d.mn_cum = l.mn_cum ? (unsigned long long*)(base + l.mn_cum) : nullptr;
    d.mn_tiles = l.mn_tiles ? (unsigned long long*)(base + l.mn_tiles) : nullptr;
    r->hist_bytes = 16 + (size_t)l.bins * 4;

    r->sweep_grid = pa::sweep_grid(d);
    if (r->sweep_grid <= 0) {
        delete r;
        return PA_ERR_CUDA;
    }

    std::memset(&r->init_state, 0, sizeof(DevState));
    r->init_state.R = (uint32_t)cfg->R0;
    // ln Omega of the protocol: N ln 2 states at beta0 = 0, or the two ground
    // states of energy -dim N near T = 0
    if (cfg->init == PA_INIT_GROUND)
        r->init_state.lnZ = std::log(2.0) + cfg->beta0 * (double)((int64_t)cfg->dim * l.N);
    else
        r->init_state.lnZ = (double)l.N * std::log(2.0);
    cudaStream_t s = r->stream;
    const size_t K1 = (size_t)cfg->K + 1;
    bool ok = cudaMemcpyAsync(d.st, &r->init_state, sizeof(DevState), cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemsetAsync(d.desc, 0, (size_t)l.tiles * 8, s) == cudaSuccess &&
              cudaMemsetAsync(d.obs, 0, K1 * sizeof(pa_obs), s) == cudaSuccess &&
              cudaMemsetAsync(d.counts, 0, (size_t)l.cap * 4, s) == cudaSuccess &&
              cudaMemsetAsync(d.offsets, 0, (size_t)l.cap * 4, s) == cudaSuccess &&
              cudaMemsetAsync(d.srcmap, 0, (size_t)l.cap * 4, s) == cudaSuccess &&
              cudaMemsetAsync(d.srcmap2, 0, (size_t)l.cap * 4, s) == cudaSuccess &&
              cudaMemsetAsync(d.tab_n, 0, (size_t)l.bins * 4, s) == cudaSuccess &&
              cudaMemsetAsync(d.tab_F, 0, (size_t)l.bins * 4, s) == cudaSuccess &&
              cudaMemcpyAsync((void*)d.thr, r->thr.data(), K1 * 16, cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemcpyAsync((void*)d.beta, r->beta.data(), K1 * 8, cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemcpyAsync((void*)d.dbeta, r->dbeta.data(), K1 * 8, cudaMemcpyHostToDevice,
                              s) == cudaSuccess &&
              cudaMemcpyAsync((void*)d.dsel, r->dsel.data(), K1 * 4, cudaMemcpyHostToDevice, s) ==
                  cudaSuccess &&
              cudaMemcpyAsync((void*)d.dtab, r->dtab.data(), r->dtab.size() * 8,
                              cudaMemcpyHostToDevice, s) == cudaSuccess &&
              pa::launch_init(d, s) == cudaSuccess && enqueue_sweep(r, s, 0) == PA_OK;
    if (!ok) {
        delete r;
        return PA_ERR_CUDA;
    }
    *out = r;
    return PA_OK;
}

int pa_resample(pa_run* r) {
    if (!r || r->gather_pending) return PA_ERR_INVALID_ARG;
    return enqueue_resample(r, r->stream);
}

int pa_sweep(pa_run* r, int32_t nsweeps) {
    if (!r || nsweeps < 0 || r->gather_pending) return PA_ERR_INVALID_ARG;
    return enqueue_sweep(r, r->stream, nsweeps);
}

int pa_step(pa_run* r) {
    if (!r || r->gather_pending) return PA_ERR_INVALID_ARG;
    return enqueue_step(r, r->stream);
}

int pa_resample_begin(pa_run* r) {
    if (!r || r->gather_pending) return PA_ERR_INVALID_ARG;
    int rc = timed(r, r->stream, 0, [&] { return pa::launch_tau(r->d, r->stream); });
    if (rc) return rc;
    rc = timed(r, r->stream, 1, [&] {
        if (r->cfg.resample == PA_RESAMPLE_MULTINOMIAL) {
            const cudaError_t e = pa::launch_multinomial(r->d, r->stream);
            if (e != cudaSuccess) return e;
        }
        return pa::launch_resample_scan(r->d, r->stream);
    });
    if (rc) return rc;
    r->gather_pending = true;
    return PA_OK;
}

int pa_resample_finish(pa_run* r, int32_t nseg, const int64_t* seg_src, const int64_t* seg_len) {
    if (!r || !r->gather_pending || nseg < 1 || nseg > pa::MAX_SEGMENTS || !seg_src || !seg_len)
        return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    pa::SegList segs;
    segs.n = (uint32_t)nseg;
    int64_t at = 0;
    for (int32_t q = 0; q < nseg; ++q) {
        if (seg_len[q] < 0 || seg_src[q] < 0 || seg_src[q] + seg_len[q] > (int64_t)st.R)
            return PA_ERR_INVALID_ARG;
        segs.dst[q] = (uint32_t)at;
        segs.src[q] = (uint32_t)seg_src[q];
        at += seg_len[q];
    }
    if (at != (int64_t)st.R) return PA_ERR_INVALID_ARG;
    segs.dst[nseg] = (uint32_t)at;
    rc = timed(r, r->stream, 1, [&] { return pa::launch_remap_gather(r->d, segs, r->stream); });
    if (rc) return rc;
    r->gather_pending = false;
    return PA_OK;
}

int pa_step_stream(pa_run* r, void* host_dst, size_t bytes, int32_t chunks, void* copy_stream,
                   int64_t* R_out) {
    if (!r || !host_dst || !copy_stream || chunks < 1 || chunks > 64 || r->gather_pending)
        return PA_ERR_INVALID_ARG;
    const cudaStream_t copy = (cudaStream_t)copy_stream;
    const RunDev& d = r->d;
    if (copy == r->stream || bytes < (size_t)d.cap * d.stride) return PA_ERR_INVALID_ARG;
    if (!r->ev_range) CK(cudaEventCreateWithFlags(&r->ev_range, cudaEventDisableTiming));
    if (!r->ev_copied) CK(cudaEventCreateWithFlags(&r->ev_copied, cudaEventDisableTiming));
    int rc = enqueue_resample(r, r->stream);
    if (rc) return rc;
    // the host needs R_i and the buffer that holds the new population
    DevState st;
    rc = read_state(r, &st);
    if (rc) return rc;
    if (st.status) return sticky_to_code(st.status);
    if (st.R > d.cap) return PA_ERR_CAPACITY;
    if (R_out) *R_out = st.R;
    CK(cudaMemsetAsync(d.accum, 0, r->hist_bytes, r->stream));
    const uint8_t* src = d.spins[st.cur];
    uint8_t* out = (uint8_t*)host_dst;
    for (int32_t c = 0; c < chunks; ++c) {
        // range bounds are multiples of 32 (32-replica warps of the
        // replica-sliced kernel); the last range ends at R
        const uint32_t lo = (uint32_t)((uint64_t)st.R * c / chunks) & ~31u;
        const uint32_t hi =
            c + 1 == chunks ? st.R : (uint32_t)((uint64_t)st.R * (c + 1) / chunks) & ~31u;
        if (hi <= lo) continue;
        RunDev dd = d;
        dd.slot_lo = lo;
        dd.slot_hi = hi;
        rc = timed(r, r->stream, 2,
                   [&] { return pa::launch_sweep(dd, r->cfg.theta, r->sweep_grid, r->stream); });
        if (rc) return rc;
        CK(cudaEventRecord(r->ev_range, r->stream));
        CK(cudaStreamWaitEvent(copy, r->ev_range, 0));
        CK(cudaMemcpyAsync(out + (size_t)lo * d.stride, src + (size_t)lo * d.stride,
                           (size_t)(hi - lo) * d.stride, cudaMemcpyDeviceToHost, copy));
    }
    rc = timed(r, r->stream, 3, [&] { return pa::launch_obs(d, r->cfg.theta, r->stream); });
    if (rc) return rc;
    CK(cudaEventRecord(r->ev_copied, copy));
    CK(cudaStreamWaitEvent(r->stream, r->ev_copied, 0));
    return PA_OK;
}

int64_t pa_bench_philox_threads(void) { return (int64_t)pa::philox_rate_threads(); }

int pa_bench_philox(uint64_t seed, int32_t halfsweeps, void* out, int64_t out_words, void* stream) {
    const int64_t need = pa::philox_rate_threads();
    if (!out || halfsweeps < 1 || need <= 0 || out_words < need) return PA_ERR_INVALID_ARG;
    CK(pa::launch_philox_rate(seed, (uint32_t)halfsweeps, (uint32_t*)out, (cudaStream_t)stream));
    return PA_OK;
}

int pa_debug(pa_run* r, uint32_t flags) {
    if (!r || (flags & ~PA_DEBUG_WITHHOLD_PREFIX)) return PA_ERR_INVALID_ARG;
    r->d.debug = flags;
    return PA_OK;
}

int pa_run_steps(pa_run* r, int32_t nsteps) {
    if (!r || nsteps < 0 || r->gather_pending) return PA_ERR_INVALID_ARG;
    if (!r->graph) {
        if (!r->cap_stream) CK(cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_step(r, r->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(r->cap_stream, &g);
        if (rc || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : PA_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&r->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            r->graph = nullptr;
            return PA_ERR_CUDA;
        }
    }
    for (int32_t i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(r->graph, r->stream));
    return PA_OK;
}

int pa_status(pa_run* r) {
    if (!r) return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    return sticky_to_code(st.status);
}

int pa_observables(pa_run* r, pa_obs* out) {
    if (!r || !out) return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    CK(cudaMemcpy(out, r->d.obs + st.step, sizeof(pa_obs), cudaMemcpyDeviceToHost));
    return sticky_to_code(st.status);
}

int pa_observables_history(pa_run* r, int32_t first, int32_t n, pa_obs* out) {
    if (!r || !out || first < 0 || n < 0 || (int64_t)first + n > (int64_t)r->cfg.K + 1)
        return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    if (n) CK(cudaMemcpy(out, r->d.obs + first, (size_t)n * sizeof(pa_obs), cudaMemcpyDeviceToHost));
    return sticky_to_code(st.status);
}

int64_t pa_dump_size(pa_run* r, int32_t what) {
    if (!r) return -1;
    DevState st;
    if (read_state(r, &st)) return -1;
    const RunDev& d = r->d;
    switch (what) {
        case PA_DUMP_SPINS: return (int64_t)st.R * d.N;
        case PA_DUMP_SPINS_RAW: return (int64_t)st.R * d.stride;
        case PA_DUMP_EBIN:
        case PA_DUMP_MAG: return (int64_t)st.R * 4;
        case PA_DUMP_HIST:
        case PA_DUMP_TAB_N:
        case PA_DUMP_TAB_F: return d.bins * 4;
        case PA_DUMP_COUNTS:
        case PA_DUMP_OFFSETS: return (int64_t)st.R_prev * 4;
        case PA_DUMP_COUPLINGS: return d.N * d.dim;
        case PA_DUMP_STATE: return (int64_t)sizeof(pa_state);
        default: return -1;
    }
}

int pa_dump(pa_run* r, int32_t what, void* dst, size_t bytes) {
    if (!r || !dst) return PA_ERR_INVALID_ARG;
    const int64_t need = pa_dump_size(r, what);
    if (need < 0 || (int64_t)bytes < need) return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    const RunDev& d = r->d;
    const int NW = (d.L + 31) / 32;
    switch (what) {
        case PA_DUMP_SPINS: {
            std::vector<uint8_t> raw((size_t)st.R * d.stride);
            if (!raw.empty())
                CK(cudaMemcpy(raw.data(), d.spins[st.cur], raw.size(), cudaMemcpyDeviceToHost));
            int8_t* o = (int8_t*)dst;
            for (uint32_t rep = 0; rep < st.R; ++rep) {
                const uint8_t* p = raw.data() + (size_t)rep * d.stride;
                int8_t* q = o + (size_t)rep * d.N;
                if (d.layout == PA_LAYOUT_INT8) {
                    std::memcpy(q, p, (size_t)d.N);
                } else {
                    const uint32_t* w = (const uint32_t*)p;
                    for (int64_t s = 0; s < d.N; ++s) {
                        const int64_t row = s / d.L, x = s % d.L;
                        const uint32_t bit = (w[row * NW + x / 32] >> (x % 32)) & 1u;
                        q[s] = bit ? (int8_t)-1 : (int8_t)1;
                    }
                }
            }
            break;
        }
        case PA_DUMP_SPINS_RAW:
            if (need) CK(cudaMemcpy(dst, d.spins[st.cur], (size_t)need, cudaMemcpyDeviceToHost));
            break;
        case PA_DUMP_EBIN:
            if (need) CK(cudaMemcpy(dst, d.ebin[st.cur], (size_t)need, cudaMemcpyDeviceToHost));
            break;
        case PA_DUMP_MAG:
            if (need) CK(cudaMemcpy(dst, d.mag[st.cur], (size_t)need, cudaMemcpyDeviceToHost));
            break;
        case PA_DUMP_HIST: CK(cudaMemcpy(dst, d.hist, (size_t)need, cudaMemcpyDeviceToHost)); break;
        case PA_DUMP_TAB_N: CK(cudaMemcpy(dst, d.tab_n, (size_t)need, cudaMemcpyDeviceToHost)); break;
        case PA_DUMP_TAB_F: CK(cudaMemcpy(dst, d.tab_F, (size_t)need, cudaMemcpyDeviceToHost)); break;
        case PA_DUMP_COUNTS:
            if (need) CK(cudaMemcpy(dst, d.counts, (size_t)need, cudaMemcpyDeviceToHost));
            break;
        case PA_DUMP_OFFSETS:
            if (need) CK(cudaMemcpy(dst, d.offsets, (size_t)need, cudaMemcpyDeviceToHost));
            break;
        case PA_DUMP_COUPLINGS: {
            int8_t* o = (int8_t*)dst;
            if (d.model != PA_MODEL_PMJ) {
                std::memset(o, 1, (size_t)need);
            } else if (d.layout == PA_LAYOUT_INT8) {
                CK(cudaMemcpy(o, d.j8, (size_t)need, cudaMemcpyDeviceToHost));
            } else {
                std::vector<uint32_t> pk((size_t)d.dim * d.nwords);
                CK(cudaMemcpy(pk.data(), d.jpk, pk.size() * 4, cudaMemcpyDeviceToHost));
                for (int64_t s = 0; s < d.N; ++s)
                    for (int dd = 0; dd < d.dim; ++dd) {
                        const int64_t row = s / d.L, x = s % d.L;
                        const uint32_t bit =
                            (pk[(size_t)dd * d.nwords + row * NW + x / 32] >> (x % 32)) & 1u;
                        o[s * d.dim + dd] = bit ? (int8_t)-1 : (int8_t)1;
                    }
            }
            break;
        }
        case PA_DUMP_STATE: {
            pa_state ps;
            ps.step = st.step;
            ps.R = st.R;
            ps.R_prev = st.R_prev;
            ps.kref = st.kref;
            ps.sweeps_done = (int64_t)st.sweeps_done;
            ps.status_bits = st.status;
            ps.lnQ = st.lnQ;
            ps.lnZ = st.lnZ;
            ps.S = st.S;
            ps.N = d.N;
            ps.bins = d.bins;
            ps.stride = d.stride;
            ps.capacity = d.cap;
            ps.parity = st.negbonds & 1u;
            ps.sources = (int64_t)st.sources;
            std::memcpy(dst, &ps, sizeof(ps));
            break;
        }
        default: return PA_ERR_INVALID_ARG;
    }
    return PA_OK;
}

int pa_dump_range(pa_run* r, int32_t what, int64_t first, int64_t count, void* dst,
                  size_t bytes) {
    if (!r || !dst || first < 0 || count < 0) return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    const RunDev& d = r->d;
    const int NW = (d.L + 31) / 32;
    int64_t limit = st.R, elem = 4;
    const uint8_t* src = nullptr;
    switch (what) {
        case PA_DUMP_SPINS: elem = d.N; src = d.spins[st.cur]; break;
        case PA_DUMP_SPINS_RAW: elem = d.stride; src = d.spins[st.cur]; break;
        case PA_DUMP_EBIN: src = (const uint8_t*)d.ebin[st.cur]; break;
        case PA_DUMP_MAG: src = (const uint8_t*)d.mag[st.cur]; break;
        case PA_DUMP_COUNTS: limit = st.R_prev; src = (const uint8_t*)d.counts; break;
        case PA_DUMP_OFFSETS: limit = st.R_prev; src = (const uint8_t*)d.offsets; break;
        default: return PA_ERR_INVALID_ARG;
    }
    if (first + count > limit || (int64_t)bytes < count * elem) return PA_ERR_INVALID_ARG;
    if (count == 0) return PA_OK;
    if (what != PA_DUMP_SPINS) {
        const size_t per = what == PA_DUMP_SPINS_RAW ? d.stride : 4;
        CK(cudaMemcpy(dst, src + (size_t)first * per, (size_t)count * per, cudaMemcpyDeviceToHost));
        return PA_OK;
    }
    std::vector<uint8_t> raw((size_t)count * d.stride);
    CK(cudaMemcpy(raw.data(), src + (size_t)first * d.stride, raw.size(), cudaMemcpyDeviceToHost));
    int8_t* o = (int8_t*)dst;
    for (int64_t rep = 0; rep < count; ++rep) {
        const uint8_t* p = raw.data() + (size_t)rep * d.stride;
        int8_t* q = o + (size_t)rep * d.N;
        if (d.layout == PA_LAYOUT_INT8) {
            std::memcpy(q, p, (size_t)d.N);
        } else {
            const uint32_t* w = (const uint32_t*)p;
            for (int64_t s = 0; s < d.N; ++s) {
                const int64_t row = s / d.L, x = s % d.L;
                q[s] = ((w[row * NW + x / 32] >> (x % 32)) & 1u) ? (int8_t)-1 : (int8_t)1;
            }
        }
    }
    return PA_OK;
}

int pa_load(pa_run* r, int32_t what, const void* src, int64_t count, size_t bytes) {
    if (!r || !src || count < 1 || count > (int64_t)r->d.cap || r->gather_pending)
        return PA_ERR_INVALID_ARG;
    const RunDev& d = r->d;
    if (what != PA_DUMP_SPINS && what != PA_DUMP_SPINS_RAW) return PA_ERR_INVALID_ARG;
    const int64_t per = what == PA_DUMP_SPINS ? d.N : d.stride;
    if ((int64_t)bytes < count * per) return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    uint8_t* dst = d.spins[st.cur];
    if (what == PA_DUMP_SPINS_RAW) {
        CK(cudaMemcpyAsync(dst, src, (size_t)(count * d.stride), cudaMemcpyHostToDevice, r->stream));
    } else {
        std::vector<uint8_t> stage((size_t)(count * d.stride), 0);
        const int8_t* in = (const int8_t*)src;
        const int NW = (d.L + 31) / 32;
        for (int64_t rep = 0; rep < count; ++rep) {
            const int8_t* p = in + rep * d.N;
            uint8_t* q = stage.data() + rep * d.stride;
            if (d.layout == PA_LAYOUT_INT8) {
                for (int64_t s2 = 0; s2 < d.N; ++s2) {
                    if (p[s2] != 1 && p[s2] != -1) return PA_ERR_INVALID_ARG;
                    q[s2] = (uint8_t)p[s2];
                }
            } else {
                uint32_t* w = (uint32_t*)q;
                for (int64_t s2 = 0; s2 < d.N; ++s2) {
                    if (p[s2] != 1 && p[s2] != -1) return PA_ERR_INVALID_ARG;
                    if (p[s2] < 0) w[(s2 / d.L) * NW + (s2 % d.L) / 32] |= 1u << ((s2 % d.L) % 32);
                }
            }
        }
        CK(cudaMemcpyAsync(dst, stage.data(), stage.size(), cudaMemcpyHostToDevice, r->stream));
        CK(cudaStreamSynchronize(r->stream));
    }
    r->load_R = (uint32_t)count;
    CK(cudaMemcpyAsync((uint8_t*)d.st + offsetof(DevState, R), &r->load_R, 4,
                       cudaMemcpyHostToDevice, r->stream));
    return enqueue_sweep(r, r->stream, 0);
}

// Checkpoint layout: header | records [step+1] | spins [R][stride] | levels [R]
// | magnetisations [R] | histogram [bins].  The couplings are not stored: they
// follow from the configuration.
struct CkptHeader {
    char magic[8];
    uint32_t version, pad;
    pa_config cfg;
    DevState st;
    uint64_t R, bins, stride, nrec;
    double beta_step;  // beta of the current step (differs from the schedule after pa_resample_to)
};

static const char kCkptMagic[8] = {'P', 'A', 'G', 'B', '3', '0', '0', '2'};

int64_t pa_checkpoint_size(pa_run* r) {
    if (!r) return -1;
    DevState st;
    if (read_state(r, &st)) return -1;
    const RunDev& d = r->d;
    return (int64_t)sizeof(CkptHeader) + (int64_t)(st.step + 1) * (int64_t)sizeof(pa_obs) +
           (int64_t)st.R * ((int64_t)d.stride + 8) + d.bins * 4;
}

int pa_checkpoint(pa_run* r, void* dst, size_t bytes) {
    if (!r || !dst || r->gather_pending) return PA_ERR_INVALID_ARG;
    const int64_t need = pa_checkpoint_size(r);
    if (need < 0 || (int64_t)bytes < need) return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    if (st.status) return sticky_to_code(st.status);
    const RunDev& d = r->d;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 2;
    h.cfg = r->cfg;
    h.st = st;
    h.R = st.R;
    h.bins = (uint64_t)d.bins;
    h.stride = d.stride;
    h.nrec = (uint64_t)st.step + 1;
    h.beta_step = r->beta[st.step];
    uint8_t* o = (uint8_t*)dst;
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    CK(cudaMemcpy(o, d.obs, h.nrec * sizeof(pa_obs), cudaMemcpyDeviceToHost));
    o += h.nrec * sizeof(pa_obs);
    if (st.R) {
        CK(cudaMemcpy(o, d.spins[st.cur], (size_t)st.R * d.stride, cudaMemcpyDeviceToHost));
        o += (size_t)st.R * d.stride;
        CK(cudaMemcpy(o, d.ebin[st.cur], (size_t)st.R * 4, cudaMemcpyDeviceToHost));
        o += (size_t)st.R * 4;
        CK(cudaMemcpy(o, d.mag[st.cur], (size_t)st.R * 4, cudaMemcpyDeviceToHost));
        o += (size_t)st.R * 4;
    }
    CK(cudaMemcpy(o, d.hist, (size_t)d.bins * 4, cudaMemcpyDeviceToHost));
    return PA_OK;
}

int pa_restore(pa_run* r, const void* src, size_t bytes) {
    if (!r || !src || bytes < sizeof(CkptHeader) || r->gather_pending) return PA_ERR_INVALID_ARG;
    CkptHeader h;
    std::memcpy(&h, src, sizeof(h));
    const RunDev& d = r->d;
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 2) return PA_ERR_INVALID_ARG;
    if (std::memcmp(&h.cfg, &r->cfg, sizeof(pa_config)) != 0) return PA_ERR_INVALID_ARG;
    if (h.bins != (uint64_t)d.bins || h.stride != d.stride || h.R > d.cap ||
        h.nrec != (uint64_t)h.st.step + 1 || h.st.step > (uint32_t)r->cfg.K)
        return PA_ERR_INVALID_ARG;
    const size_t need = sizeof(h) + h.nrec * sizeof(pa_obs) + h.R * (h.stride + 8) + h.bins * 4;
    if (bytes < need) return PA_ERR_INVALID_ARG;
    DevState now;
    int rc = read_state(r, &now);
    if (rc) return rc;
    // the run's own lookback epoch keeps counting; the population goes to buffer 0
    DevState st = h.st;
    st.cur = 0;
    st.src = 0;
    st.epoch = now.epoch;
    st.tile_counter = 0;
    st.tau_done = 0;
    st.active = 0;
    st.status = 0;
    r->init_state = st;
    const uint8_t* in = (const uint8_t*)src + sizeof(h);
    CK(cudaMemcpy(d.obs, in, h.nrec * sizeof(pa_obs), cudaMemcpyHostToDevice));
    in += h.nrec * sizeof(pa_obs);
    if (h.R) {
        CK(cudaMemcpy(d.spins[0], in, h.R * d.stride, cudaMemcpyHostToDevice));
        in += h.R * d.stride;
        CK(cudaMemcpy(d.ebin[0], in, h.R * 4, cudaMemcpyHostToDevice));
        in += h.R * 4;
        CK(cudaMemcpy(d.mag[0], in, h.R * 4, cudaMemcpyHostToDevice));
        in += h.R * 4;
    }
    CK(cudaMemcpy(d.hist, in, h.bins * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.st, &r->init_state, sizeof(DevState), cudaMemcpyHostToDevice));
    // back to the fixed schedule, then the checkpointed step's own beta
    const size_t K1 = (size_t)r->cfg.K + 1;
    r->thr = r->thr_fixed;
    r->dsel = r->dsel_fixed;
    r->beta = r->beta_fixed;
    r->dbeta = r->dbeta_fixed;
    CK(cudaMemcpy((void*)d.thr, r->thr.data(), K1 * 16, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)d.beta, r->beta.data(), K1 * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)d.dbeta, r->dbeta.data(), K1 * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)d.dsel, r->dsel.data(), K1 * 4, cudaMemcpyHostToDevice));
    if (h.beta_step != r->beta_fixed[h.st.step]) {
        rc = move_step(r, h.st.step, h.beta_step, r->stream);
        if (rc) return rc;
        CK(cudaStreamSynchronize(r->stream));
    }
    return PA_OK;
}

// Histogram overlap of the population with its reweighting to beta + dbeta:
// sum_k min(H_k / R, H_k w_k / sum_j H_j w_j), sums over k ascending.
static double overlap_of(const std::vector<uint32_t>& H, int64_t R, double dbeta) {
    const bool heating = dbeta < 0.0;
    const int64_t bins = (int64_t)H.size();
    int64_t kref = -1;
    if (heating) {
        for (int64_t k = bins - 1; k >= 0; --k)
            if (H[k]) {
                kref = k;
                break;
            }
    } else {
        for (int64_t k = 0; k < bins; ++k)
            if (H[k]) {
                kref = k;
                break;
            }
    }
    if (kref < 0 || R < 1) return 0.0;
    double sw = 0.0;
    for (int64_t k = 0; k < bins; ++k) {
        const int64_t j = heating ? kref - k : k - kref;
        if (j >= 0 && H[k]) sw = sw + (double)H[k] * weight_of(dbeta, j);
    }
    double a = 0.0;
    for (int64_t k = 0; k < bins; ++k) {
        const int64_t j = heating ? kref - k : k - kref;
        if (j < 0 || !H[k]) continue;
        const double p = (double)H[k] / (double)R;
        const double q = ((double)H[k] * weight_of(dbeta, j)) / sw;
        a = a + (p < q ? p : q);
    }
    return a;
}

int pa_adaptive_beta(pa_run* r, double target, double beta_end, double* beta_next) {
    if (!r || !beta_next || !std::isfinite(target) || !std::isfinite(beta_end) || beta_end < 0.0)
        return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    if (st.status) return sticky_to_code(st.status);
    std::vector<uint32_t> H((size_t)r->d.bins);
    CK(cudaMemcpy(H.data(), r->d.hist, H.size() * 4, cudaMemcpyDeviceToHost));
    const double beta = r->beta[st.step];
    const double span = beta_end - beta;
    if (span == 0.0 || overlap_of(H, st.R, span) >= target) {
        *beta_next = span == 0.0 ? beta : beta_end;
        return PA_OK;
    }
    double lo = 0.0, hi = std::fabs(span);
    const double sgn = span < 0.0 ? -1.0 : 1.0;
    for (int it = 0; it < 60; ++it) {
        const double mid = lo + (hi - lo) * 0.5;
        if (overlap_of(H, st.R, sgn * mid) >= target) lo = mid;
        else hi = mid;
    }
    *beta_next = beta + sgn * lo;
    return PA_OK;
}

int pa_resample_to(pa_run* r, double beta_next) {
    if (!r || !std::isfinite(beta_next) || beta_next < 0.0 || r->gather_pending)
        return PA_ERR_INVALID_ARG;
    DevState st;
    int rc = read_state(r, &st);
    if (rc) return rc;
    if (st.step + 1 > (uint32_t)r->cfg.K) return PA_ERR_DONE;
    rc = move_step(r, st.step + 1, beta_next, r->stream);
    if (rc) return rc;
    return enqueue_resample(r, r->stream);
}

int pa_profile(pa_run* r, int32_t enable) {
    if (!r) return PA_ERR_INVALID_ARG;
    r->prof = enable != 0;
    return PA_OK;
}

int pa_profile_read(pa_run* r, int64_t launches[4], double ms[4], int32_t reset) {
    if (!r) return PA_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(r->stream));
    for (const auto& p : r->pending) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, p.a, p.b));
        r->prof_n[p.kind] += 1;
        r->prof_ms[p.kind] += t;
        r->ev_pool.push_back(p.a);
        r->ev_pool.push_back(p.b);
    }
    r->pending.clear();
    for (int k = 0; k < 4; ++k) {
        if (launches) launches[k] = r->prof_n[k];
        if (ms) ms[k] = r->prof_ms[k];
        if (reset) {
            r->prof_n[k] = 0;
            r->prof_ms[k] = 0.0;
        }
    }
    return PA_OK;
}

void pa_free(pa_run* r) {
    if (!r) return;
    for (const auto& p : r->pending) {
        r->ev_pool.push_back(p.a);
        r->ev_pool.push_back(p.b);
    }
    for (cudaEvent_t e : r->ev_pool) cudaEventDestroy(e);
    if (r->ev_range) cudaEventDestroy(r->ev_range);
    if (r->ev_copied) cudaEventDestroy(r->ev_copied);
    if (r->graph) cudaGraphExecDestroy(r->graph);
    if (r->cap_stream) cudaStreamDestroy(r->cap_stream);
    delete r;
}

const char* pa_strerror(int code) {
    switch (code) {
        case PA_OK: return "ok";
        case PA_ERR_INVALID_ARG: return "invalid argument";
        case PA_ERR_ODD_L: return "L must be even for the checkerboard update";
        case PA_ERR_UNSUPPORTED: return "no compiled kernel for this (dim, L, layout)";
        case PA_ERR_CAPACITY: return "population exceeded the configured capacity";
        case PA_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        case PA_ERR_CUDA: return "CUDA runtime error";
        case PA_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
        case PA_ERR_DONE: return "annealing schedule already finished";
        case PA_ERR_EMPTY: return "population died out";
        case PA_ERR_INVARIANT: return "device invariant failed (histogram sum != R)";
        default: return "unknown error";
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched form
// ---------------------------------------------------------------------------
struct pa_batch {
    std::vector<pa_run*> runs;
    cudaStream_t stream;
    pa::BatchDev bd;
    struct Cls {
        int layout, dim, L, model;
        std::vector<uint32_t> ids;
        pa::BatchSweepArgs args;
        pa::RunDev proto;
        int warps, grid;
        cudaStream_t stream;  // the class's branch of a step (fork / join)
        cudaEvent_t done;
    };
    std::vector<Cls> cls;
    std::vector<pa::RunDev> mn_runs;  // runs on multinomial draws (their draws launch per run)
    cudaEvent_t fork;
    cudaStream_t cap_stream;
    cudaGraphExec_t graph;
    int64_t steps_left;
    // phase timing of steps enqueued by pa_batch_step while profiling is on:
    // events before the reweight, the resample, the sweeps, the observables
    // and after them
    bool prof;
    std::vector<std::array<cudaEvent_t, 5>> pending;
    std::vector<cudaEvent_t> ev_pool;
    int64_t prof_steps;
    double prof_ms[4];
};

namespace {
size_t batch_layout(int32_t nruns, size_t off[5]) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    off[0] = take((size_t)nruns * sizeof(pa::RunDev));     // runs
    off[1] = take((size_t)(nruns + 1) * 4);                 // tile_base
    off[2] = take((size_t)(nruns + 1) * 4);                 // counters
    off[3] = take((size_t)nruns * 4);                       // run ids by class
    off[4] = take((size_t)(2 * nruns) * 4);                 // slot bases
    return o;
}

// Slots per claim: the largest power of two <= 32 that still leaves about
// four claims per resident warp, so small classes spread over the GPU.
uint32_t auto_chunk(uint32_t total_slots, int grid, int warps) {
    uint32_t chunk = 32;
    const uint64_t want = 4ull * (uint64_t)grid * (uint64_t)warps;
    while (chunk > 1 && (uint64_t)(total_slots / chunk) < want) chunk >>= 1;
    return chunk;
}

cudaEvent_t batch_event(pa_batch* b) {
    if (!b->ev_pool.empty()) {
        cudaEvent_t e = b->ev_pool.back();
        b->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int enqueue_batch_launches(pa_batch* b, cudaStream_t s, bool timing,
                           const std::array<cudaEvent_t, 5>& ev);

// One batched step: reweight and resample of every run on s, then the sweep
// classes as parallel branches (fork / join through events), then the
// observables of every run on s.  With phase timing on (and s the batch's own
// stream) the phases are bracketed by pooled events.
int enqueue_batch_step(pa_batch* b, cudaStream_t s) {
    std::array<cudaEvent_t, 5> ev{};
    const bool timing = b->prof && s == b->stream;
    int got = 0;
    if (timing) {
        for (; got < 5; ++got) {
            ev[got] = batch_event(b);
            if (!ev[got]) break;
        }
    }
    int rc = timing && got < 5 ? PA_ERR_CUDA : enqueue_batch_launches(b, s, timing, ev);
    if (timing) {
        if (rc == PA_OK) {
            b->pending.push_back(ev);
        } else {
            for (int k = 0; k < got; ++k) b->ev_pool.push_back(ev[k]);
        }
    }
    return rc;
}

int enqueue_batch_launches(pa_batch* b, cudaStream_t s, bool timing,
                           const std::array<cudaEvent_t, 5>& ev) {
    auto mark = [&](int k) { return timing ? cudaEventRecord(ev[k], s) : cudaSuccess; };
    CK(mark(0));
    CK(pa::launch_tau_batched(b->bd, s));
    CK(mark(1));
    for (const auto& d : b->mn_runs) CK(pa::launch_multinomial(d, s));
    CK(pa::launch_resample_batched(b->bd, s));
    CK(mark(2));
    if (b->cls.size() == 1) {
        const auto& c = b->cls[0];
        CK(pa::launch_sweep_batched(c.args, c.proto, c.warps, c.grid, s));
    } else {
        CK(cudaEventRecord(b->fork, s));
        for (const auto& c : b->cls) {
            CK(cudaStreamWaitEvent(c.stream, b->fork, 0));
            CK(pa::launch_sweep_batched(c.args, c.proto, c.warps, c.grid, c.stream));
            CK(cudaEventRecord(c.done, c.stream));
        }
        for (const auto& c : b->cls) CK(cudaStreamWaitEvent(s, c.done, 0));
    }
    CK(mark(3));
    CK(pa::launch_obs_batched(b->bd, s));
    CK(mark(4));
    return PA_OK;
}

void batch_release(pa_batch* b) {
    for (const auto& ev : b->pending)
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (auto& c : b->cls) {
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// Shared body of pa_batch_init (steps_left == nullptr: each run's remaining
// steps read from the device, then the uploads are waited for) and
// pa_batch_init_async (remaining steps given by the caller, nothing waited for).
int batch_init(pa_run* const* runs, int32_t nruns, const int32_t* steps_left, void* ws,
               size_t bytes, void* stream, pa_batch** out);
}  // namespace

extern "C" {

size_t pa_batch_workspace_size(int32_t nruns) {
    if (nruns < 1) return 0;
    size_t off[5];
    return batch_layout(nruns, off);
}

int pa_batch_init(pa_run* const* runs, int32_t nruns, void* ws, size_t bytes, void* stream,
                  pa_batch** out) {
    return batch_init(runs, nruns, nullptr, ws, bytes, stream, out);
}

int pa_batch_init_async(pa_run* const* runs, int32_t nruns, const int32_t* steps_left, void* ws,
                        size_t bytes, void* stream, pa_batch** out) {
    if (!steps_left) return PA_ERR_INVALID_ARG;
    return batch_init(runs, nruns, steps_left, ws, bytes, stream, out);
}

}  // extern "C"

namespace {
int batch_init(pa_run* const* runs, int32_t nruns, const int32_t* steps_left, void* ws,
               size_t bytes, void* stream, pa_batch** out) {
    if (!out || !runs || nruns < 1) return PA_ERR_INVALID_ARG;
    *out = nullptr;
    size_t off[5];
    const size_t need = batch_layout(nruns, off);
    if (!ws || ((uintptr_t)ws % ALIGN) != 0 || bytes < need) return PA_ERR_WORKSPACE;
    pa_batch* b = new (std::nothrow) pa_batch();
    if (!b) return PA_ERR_INVALID_ARG;
    b->stream = (cudaStream_t)stream;
    b->cap_stream = nullptr;
    b->graph = nullptr;
    b->fork = nullptr;
    b->steps_left = INT64_MAX;
    b->prof = false;
    b->prof_steps = 0;
    for (double& m : b->prof_ms) m = 0.0;
    std::vector<pa::RunDev> h_runs;
    std::vector<uint32_t> tile_base(1, 0u);
    for (int32_t i = 0; i < nruns; ++i) {
        pa_run* r = runs[i];
        if (!r || r->gather_pending) {
            batch_release(b);
            return PA_ERR_INVALID_ARG;
        }
        for (int32_t j = 0; j < i; ++j)
            if (runs[j] == r) {
                batch_release(b);
                return PA_ERR_INVALID_ARG;
            }
        int64_t left = 0;
        if (steps_left) {
            if (steps_left[i] < 0 || steps_left[i] > r->cfg.K) {
                batch_release(b);
                return PA_ERR_INVALID_ARG;
            }
            left = steps_left[i];
        } else {
            DevState st;
            if (read_state(r, &st) != PA_OK) {
                batch_release(b);
                return PA_ERR_CUDA;
            }
            left = (int64_t)r->cfg.K - (int64_t)st.step;
        }
        if (left < b->steps_left) b->steps_left = left;
        b->runs.push_back(r);
        h_runs.push_back(r->d);
        tile_base.push_back(tile_base.back() + r->d.tiles);
    }
    // classes: one sweep kernel instantiation per (layout, dim, L, model)
    for (int32_t i = 0; i < nruns; ++i) {
        const pa::RunDev& d = h_runs[i];
        size_t c = 0;
        while (c < b->cls.size() &&
               !(b->cls[c].layout == d.layout && b->cls[c].dim == d.dim && b->cls[c].L == d.L &&
                 b->cls[c].model == d.model))
            ++c;
        if (c == b->cls.size()) {
            pa_batch::Cls k;
            k.layout = d.layout;
            k.dim = d.dim;
            k.L = d.L;
            k.model = d.model;
            k.proto = d;
            k.warps = pa::l64_batched_applies(d) ? pa::l64_block_warps(d) : 4;
            k.stream = nullptr;
            k.done = nullptr;
            b->cls.push_back(k);
        }
        b->cls[c].ids.push_back((uint32_t)i);
    }
    std::vector<uint32_t> ids, bases;
    uint8_t* base = (uint8_t*)ws;
    pa::RunDev* d_runs = (pa::RunDev*)(base + off[0]);
    uint32_t* d_tile_base = (uint32_t*)(base + off[1]);
    uint32_t* d_counters = (uint32_t*)(base + off[2]);
    uint32_t* d_ids = (uint32_t*)(base + off[3]);
    uint32_t* d_bases = (uint32_t*)(base + off[4]);
    for (size_t c = 0; c < b->cls.size(); ++c) {
        auto& k = b->cls[c];
        const size_t id0 = ids.size(), base0 = bases.size();
        uint32_t slots = 0;
        for (uint32_t i : k.ids) {
            ids.push_back(i);
            bases.push_back(slots);
            slots += (h_runs[i].cap + 31u) / 32u * 32u;
        }
        bases.push_back(slots);
        k.args.runs = d_runs;
        k.args.run_ids = d_ids + id0;
        k.args.slot_base = d_bases + base0;
        k.args.n = (uint32_t)k.ids.size();
        k.args.total_slots = slots;
        k.args.counter = d_counters + 1 + c;
        k.grid = pa::batched_sweep_grid(k.proto, k.warps);
        if (k.grid <= 0 || cudaStreamCreateWithFlags(&k.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&k.done, cudaEventDisableTiming) != cudaSuccess) {
            batch_release(b);
            return PA_ERR_CUDA;
        }
        k.args.chunk = auto_chunk(slots, k.grid, k.warps);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        batch_release(b);
        return PA_ERR_CUDA;
    }
    b->bd.runs = d_runs;
    b->bd.nruns = (uint32_t)nruns;
    b->bd.tile_base = d_tile_base;
    b->bd.total_tiles = tile_base.back();
    b->bd.any_poisson = 0;
    b->bd.any_multinomial = 0;
    for (const auto& h : h_runs) {
        if (h.resample == PA_RESAMPLE_POISSON) b->bd.any_poisson = 1;
        if (h.resample == PA_RESAMPLE_MULTINOMIAL) {
            b->bd.any_multinomial = 1;
            b->mn_runs.push_back(h);
        }
    }
    b->bd.counters = d_counters;
    b->bd.ncounters = (uint32_t)(1 + b->cls.size());
    cudaStream_t s = b->stream;
    const bool ok =
        cudaMemcpyAsync(d_runs, h_runs.data(), h_runs.size() * sizeof(pa::RunDev),
                        cudaMemcpyHostToDevice, s) == cudaSuccess &&
        cudaMemcpyAsync(d_tile_base, tile_base.data(), tile_base.size() * 4, cudaMemcpyHostToDevice,
                        s) == cudaSuccess &&
        cudaMemsetAsync(d_counters, 0, (size_t)(nruns + 1) * 4, s) == cudaSuccess &&
        cudaMemcpyAsync(d_ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice, s) ==
            cudaSuccess &&
        cudaMemcpyAsync(d_bases, bases.data(), bases.size() * 4, cudaMemcpyHostToDevice, s) ==
            cudaSuccess &&
        (steps_left || cudaStreamSynchronize(s) == cudaSuccess);
    if (!ok) {
        batch_release(b);
        return PA_ERR_CUDA;
    }
    *out = b;
    return PA_OK;
}
}  // namespace

extern "C" {

int pa_batch_profile(pa_batch* b, int32_t enable) {
    if (!b) return PA_ERR_INVALID_ARG;
    b->prof = enable != 0;
    return PA_OK;
}

int pa_batch_profile_read(pa_batch* b, int64_t* steps, double ms[4], int32_t reset) {
    if (!b) return PA_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(b->stream));
    for (const auto& ev : b->pending) {
        for (int k = 0; k < 4; ++k) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
            b->prof_ms[k] += t;
        }
        b->prof_steps += 1;
        for (cudaEvent_t e : ev) b->ev_pool.push_back(e);
    }
    b->pending.clear();
    if (steps) *steps = b->prof_steps;
    for (int k = 0; k < 4; ++k) {
        if (ms) ms[k] = b->prof_ms[k];
        if (reset) b->prof_ms[k] = 0.0;
    }
    if (reset) b->prof_steps = 0;
    return PA_OK;
}

int pa_batch_step(pa_batch* b) {
    if (!b) return PA_ERR_INVALID_ARG;
    if (b->steps_left <= 0) return PA_ERR_DONE;
    const int rc = enqueue_batch_step(b, b->stream);
    if (rc == PA_OK) --b->steps_left;
    return rc;
}

int pa_batch_run_steps(pa_batch* b, int32_t nsteps) {
    if (!b || nsteps < 0) return PA_ERR_INVALID_ARG;
    if (nsteps > b->steps_left) return PA_ERR_DONE;
    if (!b->graph) {
        if (!b->cap_stream) CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_batch_step(b, b->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (rc || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : PA_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            b->graph = nullptr;
            return PA_ERR_CUDA;
        }
    }
    for (int32_t i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(b->graph, b->stream));
    b->steps_left -= nsteps;
    return PA_OK;
}

int pa_batch_sync(pa_batch* b) {
    if (!b) return PA_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(b->stream));
    int worst = PA_OK;
    for (pa_run* r : b->runs) {
        const int rc = pa_status(r);
        if (rc != PA_OK && worst == PA_OK) worst = rc;
    }
    return worst;
}

int pa_batch_num_classes(pa_batch* b) { return b ? (int)b->cls.size() : PA_ERR_INVALID_ARG; }

int pa_batch_class_info(pa_batch* b, int32_t c, int32_t info[8]) {
    if (!b || !info || c < 0 || c >= (int32_t)b->cls.size()) return PA_ERR_INVALID_ARG;
    const auto& k = b->cls[c];
    info[0] = k.layout;
    info[1] = k.dim;
    info[2] = k.L;
    info[3] = k.model;
    info[4] = (int32_t)k.ids.size();
    info[5] = k.warps;
    info[6] = (int32_t)k.args.total_slots;
    info[7] = (int32_t)k.args.chunk;
    return PA_OK;
}

int pa_batch_set_shape(pa_batch* b, int32_t c, int32_t warps, int32_t chunk) {
    if (!b || c < 0 || c >= (int32_t)b->cls.size()) return PA_ERR_INVALID_ARG;
    if (chunk < 0 || chunk > 32 || (chunk & (chunk - 1))) return PA_ERR_INVALID_ARG;
    auto& k = b->cls[c];
    int w = warps == 0 ? k.warps : warps;
    if (pa::l64_batched_applies(k.proto)) {
        if (w != pa::l64_block_warps(k.proto)) return PA_ERR_INVALID_ARG;
    } else if ((w != 2 && w != 4 && w != 8) || !pa::batched_warps_valid(k.proto, w)) {
        return PA_ERR_INVALID_ARG;
    }
    const int grid = pa::batched_sweep_grid(k.proto, w);
    if (grid <= 0) return PA_ERR_CUDA;
    k.warps = w;
    k.grid = grid;
    k.args.chunk = chunk ? (uint32_t)chunk : auto_chunk(k.args.total_slots, grid, w);
    if (b->graph) {  // the captured step used the old shape
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return PA_OK;
}

void pa_batch_free(pa_batch* b) {
    if (!b) return;
    batch_release(b);
}

}  // extern "C"
