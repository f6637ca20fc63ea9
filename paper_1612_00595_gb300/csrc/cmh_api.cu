// Host side of the chromh C ABI (include/chromh.h).
//
// A model owns: the signals and the predicted-variance buffer V (row-major
// [station][pitch], pitch a multiple of 64 samples), two event stores used
// alternately by consecutive sweeps, the partition tables, and a CUDA graph
// of one sweep (re-bin + one phase launch per colour + bookkeeping) that
// cmh_run_sweeps replays.  Every kernel reads the sweep number from device
// memory, so one captured graph serves every sweep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <vector>

#include "chromh.h"
#include "cmh_common.cuh"

using namespace cmh;

namespace {

constexpr uint64_t kCkptMagic = 0x31484d4f52484343ULL;  // "CCHROMH1"
constexpr int kCkptVersion = 3;

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return CMH_OK;
    if (e == cudaErrorMemoryAllocation) return CMH_ERR_OOM;
    return CMH_ERR_CUDA;
}

#define CK(expr)                                 \
    do {                                         \
        cudaError_t e_ = (expr);                 \
        if (e_ != cudaSuccess) return cuda_err(e_); \
    } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

namespace cmh {

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

}  // namespace cmh

struct cmh_model {
    cmh_params p{};
    Geo g{};
    Dev d{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void*> allocs;        // freed at destroy
    std::vector<void*> part_allocs;   // freed when re-partitioned
    FlatList flat{};
    long long flat_cap = 0;
    double* off_lp = nullptr;         // latent arrival offsets: their log prior (device scalar)
    double* partial = nullptr;
    int n_partial = 0;
    bool partitioned = false;
    double grid_L = 0.0, sx0 = 0.0, sy0 = 0.0;
    int shift_mode = 0;
    long long sweeps = 0;             // host mirror of the device sweep counter
    long long launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int timing = 0;
    int sweep_grid = 0;               // CTAs of the persistent sweep kernel (0: colour by colour)
    long long part_gen = 0;           // partitions and birth tables set so far (a batch refuses a model changed since)
    double* bt_mass = nullptr;        // learned birth table (owned)
    double* bt_cdf = nullptr;
    float* bt_tab = nullptr;
    float* bt_mag = nullptr;
    double phase_ms = 0.0;
    long long phase_launches = 0;
    int latched = 0;
    long long trace_cap = 0;
    long long n0 = 0;
    // asynchronous state reads: the flat list written by the flatten kernel
    // straight into mapped pinned host memory, plus the log-density and
    // statistics, in stream order
    struct ReadSlot {
        unsigned char* host = nullptr;   // x, y, t, m [cap] doubles, id [cap], logp, stats [kStats], n
        long long cap = 0;
        cudaEvent_t ev = nullptr;
        bool pending = false;
        long long sweeps = 0, launches = 0, phase_launches = 0;
        double phase_ms = 0.0;
    } rs[2];

    template <typename T>
    cudaError_t alloc(T** ptr, size_t count, bool partition_scope = false) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) return e;
        (partition_scope ? part_allocs : allocs).push_back(q);
        *ptr = (T*)q;
        return cudaSuccess;
    }

    void drop_graph() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        graph_exec = nullptr;
        graph = nullptr;
    }

    void free_partition() {
        drop_graph();
        for (void* q : part_allocs) cudaFree(q);
        part_allocs.clear();
    }
};

namespace {

// exact upper bound of how many stations lie within `radius` of any point:
// all of them are within 2 * radius of one of them
int max_within(const std::vector<double>& sx, const std::vector<double>& sy, double radius) {
    const size_t n = sx.size();
    int best = 0;
    const double r2 = 4.0 * radius * radius;
    for (size_t i = 0; i < n; ++i) {
        int c = 0;
        for (size_t j = 0; j < n; ++j) {
            const double dx = sx[i] - sx[j], dy = sy[i] - sy[j];
            c += dx * dx + dy * dy < r2;
        }
        best = std::max(best, c);
    }
    return best;
}

int check_status(cmh_model* m) {
    if (m->latched) return m->latched;
    int st = 0;
    CK(cudaMemcpyAsync(&st, m->d.status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (st) m->latched = st;
    return st;
}

// the store holding the current events between sweeps
int cur_buf(const cmh_model* m) { return (int)((m->sweeps + 1) & 1); }

int upload_sweep(cmh_model* m, long long s) {
    CK(cudaMemcpyAsync(m->d.sweep, &s, sizeof(long long), cudaMemcpyHostToDevice, m->stream));
    return CMH_OK;
}

// events of the current store -> flat list (device), count on the host
int flatten_current(cmh_model* m, int* n_host) {
    int dummy = 0;
    CK(launch_flatten(m->g, m->d, cur_buf(m), m->flat, m->stream, &dummy));
    m->launches += dummy;
    CK(cudaMemcpyAsync(n_host, m->flat.n, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return CMH_OK;
}

double host_log_prior(const cmh_params& p, const double* x, const double* y, const double* t,
                      const double* mm, long long n) {
    double lp = -p.Lambda;
    for (long long i = 0; i < n; ++i) {
        if (!(x[i] >= 0.0 && x[i] < p.W && y[i] >= 0.0 && y[i] < p.W && t[i] >= 0.0 && t[i] < p.T &&
              mm[i] >= 2.0))
            return -INFINITY;
        lp += std::log(p.Lambda) - std::log(p.W * p.W * p.T) - (mm[i] - 2.0);
    }
    return lp;
}

// V from the flat list, then prior (host) + likelihood (device) in float64
int synth_and_logdensity(cmh_model* m, int n_flat, double* out) {
    int l = 0;
    CK(launch_vsynth(m->g, m->d, m->flat, m->stream, &l));
    CK(launch_loglik(m->g, m->d, m->partial, m->n_partial, m->stream));
    l += 1;
    m->launches += l;
    std::vector<double> part(m->n_partial);
    std::vector<double> hx(n_flat), hy(n_flat), ht(n_flat), hm(n_flat);
    CK(cudaMemcpyAsync(part.data(), m->partial, sizeof(double) * m->n_partial, cudaMemcpyDeviceToHost, m->stream));
    if (n_flat) {
        CK(cudaMemcpyAsync(hx.data(), m->flat.x, sizeof(double) * n_flat, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaMemcpyAsync(hy.data(), m->flat.y, sizeof(double) * n_flat, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaMemcpyAsync(ht.data(), m->flat.t, sizeof(double) * n_flat, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaMemcpyAsync(hm.data(), m->flat.m, sizeof(double) * n_flat, cudaMemcpyDeviceToHost, m->stream));
    }
    double olp = 0.0;   // latent arrival offsets: sum of their log N(delta; 0, sig_a^2)
    if (m->flat.off && m->g.n_st > 0) {
        CK(launch_offset_prior(m->g, m->d, m->flat, m->off_lp, m->stream));
        m->launches += 1;
        CK(cudaMemcpyAsync(&olp, m->off_lp, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    }
    CK(cudaStreamSynchronize(m->stream));
    double ll = 0.0;
    for (double v : part) ll += v;
    *out = host_log_prior(m->p, hx.data(), hy.data(), ht.data(), hm.data(), n_flat) + olp + ll;
    CK(cudaMemcpyAsync(m->d.logp, out, sizeof(double), cudaMemcpyHostToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return CMH_OK;
}

int validate_params(const cmh_params* p) {
    if (!p) return CMH_ERR_ARG;
    const double pos[] = {p->W, p->T, p->Lambda, p->v, p->tau, p->t_s, p->noise_var, p->f_hz, p->R_max,
                          p->sig_xy, p->sig_t, p->sig_m};
    for (double v : pos)
        if (!finite_pos(v)) return CMH_ERR_ARG;
    if (!std::isfinite(p->alpha) || !std::isfinite(p->beta_att)) return CMH_ERR_ARG;
    if (!(p->p_birth > 0.0 && p->p_death > 0.0 && p->p_birth + p->p_death < 1.0)) return CMH_ERR_ARG;
    if (!(p->p_pair >= 0.0 && p->p_birth + p->p_death + p->p_pair <= 1.0)) return CMH_ERR_ARG;
    // latent arrival times and the arrival-time move
    if (!(std::isfinite(p->sig_a) && p->sig_a >= 0.0 && std::isfinite(p->p_arr) && p->p_arr >= 0.0))
        return CMH_ERR_ARG;
    if (!(p->p_birth + p->p_death + p->p_pair + p->p_arr <= 1.0)) return CMH_ERR_ARG;
    if (p->p_arr > 0.0 && !(p->sig_a > 0.0 && finite_pos(p->sig_da))) return CMH_ERR_ARG;
    if (p->k_per_phase < 1 || p->k_per_phase > kMaxK) return CMH_ERR_ARG;
    if (p->dtype != CMH_F32 && p->dtype != CMH_F64) return CMH_ERR_ARG;
    if (p->likelihood != 0 && !(p->likelihood == 1 && p->dtype == CMH_F32)) return CMH_ERR_ARG;
    if (p->ev_capacity < 0 || p->frozen_capacity < 0 || p->max_events < 0) return CMH_ERR_ARG;
    if (p->stage_samples < -1 || (p->schedule != 0 && p->schedule != 1) || p->ctas_per_sm < 0 || p->ctas_per_sm > 3)
        return CMH_ERR_ARG;
    // the float32 kernel of joint moves (and the one of latent arrival
    // offsets) reads the windows from global memory under the variance reading
    if ((p->p_pair > 0.0 || p->sig_a > 0.0) && p->dtype == CMH_F32 && (p->stage_samples != 0 || p->likelihood != 0))
        return CMH_ERR_ARG;
    if (p->block_threads != 0 && (p->block_threads < 64 || p->block_threads > 512 || p->block_threads % 32))
        return CMH_ERR_ARG;
    const double nw = std::llround(p->t_s * p->f_hz);
    if (nw < 1 || nw > 1e8) return CMH_ERR_ARG;
    return CMH_OK;
}

int bin_flat_into_current(cmh_model* m, int n_flat) {
    // the flat list becomes the "previous" store of a pseudo sweep s+1; its
    // re-bin writes the store sweep s will read
    const long long s = m->sweeps;
    Store src = m->d.st[s & 1];
    if (n_flat) {
        CK(cudaMemcpyAsync(src.x, m->flat.x, sizeof(double) * n_flat, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(src.y, m->flat.y, sizeof(double) * n_flat, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(src.t, m->flat.t, sizeof(double) * n_flat, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(src.m, m->flat.m, sizeof(double) * n_flat, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(src.id, m->flat.id, sizeof(unsigned long long) * n_flat, cudaMemcpyDeviceToDevice,
                           m->stream));
        if (src.off && m->flat.off)
            CK(cudaMemcpyAsync(src.off, m->flat.off, sizeof(double) * (size_t)n_flat * m->g.n_st,
                               cudaMemcpyDeviceToDevice, m->stream));
    }
    int rc = upload_sweep(m, s + 1);
    if (rc) return rc;
    int l = 0;
    CK(launch_rebin(m->g, m->d, n_flat, m->stream, &l));
    m->launches += l;
    rc = upload_sweep(m, s);
    if (rc) return rc;
    return check_status(m);
}

int capture_graph(cmh_model* m) {
    m->drop_graph();
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    int l = 0;
    cudaError_t e = launch_rebin(m->g, m->d, -1, m->stream, &l);
    if (m->sweep_grid > 0) {
        if (e == cudaSuccess) e = launch_sweep32(m->g, m->d, m->sweep_grid, m->stream);
    } else {
        for (int c = 0; c < m->g.n_colours && e == cudaSuccess; ++c) e = launch_phase(m->g, m->d, c, m->stream);
    }
    if (e == cudaSuccess) e = launch_sweep_end(m->g, m->d, m->stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(m->stream, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_err(e);
    }
    CK(e2);
    m->graph = graph;
    CK(cudaGraphInstantiate(&m->graph_exec, graph, 0));
    return CMH_OK;
}

int launches_per_sweep(const cmh_model* m) { return 3 + (m->sweep_grid > 0 ? 1 : m->g.n_colours) + 1; }

// grow the flat list to `cap` events, keeping its first n_keep
int ensure_flat(cmh_model* m, long long cap, int n_keep) {
    if (cap <= m->flat_cap) return CMH_OK;
    FlatList nf{};
    void* q[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    const size_t sz[6] = {sizeof(double), sizeof(double), sizeof(double), sizeof(double),
                          sizeof(unsigned long long), sizeof(int)};
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaMalloc(&q[i], sz[i] * (i == 5 ? 1 : (size_t)cap));
    if (e != cudaSuccess) {
        for (void* x : q) if (x) cudaFree(x);
        return cuda_err(e);
    }
    nf.x = (double*)q[0]; nf.y = (double*)q[1]; nf.t = (double*)q[2]; nf.m = (double*)q[3];
    nf.id = (unsigned long long*)q[4]; nf.n = (int*)q[5];
    void* old[6] = {m->flat.x, m->flat.y, m->flat.t, m->flat.m, m->flat.id, m->flat.n};
    for (int i = 0; i < 6; ++i) {
        const size_t bytes = sz[i] * (i == 5 ? 1 : (size_t)n_keep);
        if (bytes) CK(cudaMemcpyAsync(q[i], old[i], bytes, cudaMemcpyDeviceToDevice, m->stream));
    }
    CK(cudaStreamSynchronize(m->stream));
    for (void* x : old) {
        auto it = std::find(m->allocs.begin(), m->allocs.end(), x);
        if (it != m->allocs.end()) m->allocs.erase(it);
        cudaFree(x);
    }
    for (void* x : q) m->allocs.push_back(x);
    if (m->flat.off) {   // latent arrival offsets: rows of n_st, the first n_keep kept
        const size_t row = (size_t)std::max(m->g.n_st, 1);
        double* no = nullptr;
        e = cudaMalloc(&no, sizeof(double) * row * (size_t)cap);
        if (e != cudaSuccess) return cuda_err(e);
        m->allocs.push_back(no);
        CK(cudaMemsetAsync(no, 0, sizeof(double) * row * (size_t)cap, m->stream));
        if (n_keep)
            CK(cudaMemcpyAsync(no, m->flat.off, sizeof(double) * row * (size_t)n_keep, cudaMemcpyDeviceToDevice,
                               m->stream));
        CK(cudaStreamSynchronize(m->stream));
        auto it = std::find(m->allocs.begin(), m->allocs.end(), (void*)m->flat.off);
        if (it != m->allocs.end()) m->allocs.erase(it);
        cudaFree(m->flat.off);
        nf.off = no;
    }
    m->flat = nf;
    m->flat_cap = cap;
    return CMH_OK;
}

}  // namespace

extern "C" {

const char* cmh_strerror(int code) {
    switch (code) {
        case CMH_OK: return "ok";
        case CMH_ERR_ARG: return "invalid argument";
        case CMH_ERR_GEOMETRY: return "R_max too large for the colour pattern of this grid";
        case CMH_ERR_NONFINITE: return "non-finite signal sample or event coordinate";
        case CMH_ERR_OOM: return "device allocation failed";
        case CMH_ERR_CAPACITY: return "a fixed capacity (events, blanket, arrivals) was exceeded";
        case CMH_ERR_TIMEOUT: return "a bounded device wait gave up";
        case CMH_ERR_CUDA: return "CUDA runtime error";
        case CMH_ERR_STATE: return "call out of order or error latched";
        default: return "unknown error";
    }
}

int cmh_create_model(const cmh_event* init_events, int64_t n_events, const cmh_station* stations,
                     int32_t n_stations, const void* signals, int64_t n_samples, int64_t row_pitch,
                     cmh_dtype sig_dtype, int32_t signals_on_device, const cmh_params* p, void* cuda_stream,
                     cmh_model** out) {
    (void)cudaGetLastError();   // an earlier call's failed launch must not be reported here
    if (!out) return CMH_ERR_ARG;
    *out = nullptr;
    int rc = validate_params(p);
    if (rc) return rc;
    if (n_events < 0 || (n_events > 0 && !init_events) || n_stations < 0 || (n_stations > 0 && !stations) ||
        n_samples < 1 || row_pitch < n_samples || (n_stations > 0 && !signals) ||
        (sig_dtype != CMH_F32 && sig_dtype != CMH_F64))
        return CMH_ERR_ARG;
    if (n_samples > (1LL << 30)) return CMH_ERR_ARG;
    for (int64_t i = 0; i < n_events; ++i) {
        const cmh_event& e = init_events[i];
        if (!std::isfinite(e.x) || !std::isfinite(e.y) || !std::isfinite(e.t) || !std::isfinite(e.m))
            return CMH_ERR_NONFINITE;
        if (!(e.x >= 0.0 && e.x < p->W && e.y >= 0.0 && e.y < p->W && e.t >= 0.0 && e.t < p->T && e.m >= 2.0))
            return CMH_ERR_ARG;
    }
    for (int32_t j = 0; j < n_stations; ++j)
        if (!std::isfinite(stations[j].x) || !std::isfinite(stations[j].y)) return CMH_ERR_NONFINITE;

    cmh_model* m = new (std::nothrow) cmh_model();
    if (!m) return CMH_ERR_OOM;
    m->p = *p;
    if (m->p.ev_capacity == 0) m->p.ev_capacity = 128;
    if (m->p.frozen_capacity == 0) m->p.frozen_capacity = 64;
    if (m->p.block_threads == 0) m->p.block_threads = 256;
    if (m->p.max_events == 0) m->p.max_events = 4 * (n_events + (int64_t)std::ceil(p->Lambda)) + 4096;
    if (m->p.max_events < n_events) { delete m; return CMH_ERR_ARG; }
    m->n0 = n_events;

    auto fail = [&](int code) {
        cmh_destroy(m);
        return code;
    };
    if (cuda_stream) {
        m->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(cuda_err(e));
        m->own_stream = true;
    }
    Geo& g = m->g;
    g.W = p->W; g.T = p->T; g.Lambda = p->Lambda; g.v = p->v; g.alpha = p->alpha; g.beta_att = p->beta_att;
    g.tau = p->tau; g.noise_var = p->noise_var; g.f_hz = p->f_hz; g.R_max = p->R_max;
    g.p_birth = p->p_birth; g.p_death = p->p_death; g.sig_xy = p->sig_xy; g.sig_t = p->sig_t; g.sig_m = p->sig_m;
    g.p_pair = p->p_pair;
    g.sig_a = p->sig_a;
    g.p_arr = p->p_arr;
    g.sig_da = p->sig_da;
    g.log_pb = std::log(p->p_birth);
    g.log_pd = std::log(p->p_death);
    g.log_Lambda = std::log(p->Lambda);
    g.log_WWT = std::log(p->W * p->W * p->T);
    g.log_T = std::log(p->T);
    g.n_w = (int)std::llround(p->t_s * p->f_hz);
    g.k = p->k_per_phase;
    g.commit = p->commit ? 1 : 0;
    g.n_st = n_stations;
    g.n_samp = n_samples;
    g.pitch = (n_samples + 63) / 64 * 64;
    g.seed = p->seed;
    g.ev_cap = m->p.ev_capacity;
    g.frz_cap = m->p.frozen_capacity;
    g.f32 = p->dtype == CMH_F32;
    g.threads = m->p.block_threads;
    g.dep_wait_limit = kDepWaitLimitDefault;
    g.hold_cell = -1;
    g.count_unique = m->timing && g.f32 ? 1 : 0;
    g.max_events = m->p.max_events;
    g.fv_f = (float)(p->f_hz / p->v);
    g.mean_mode = p->likelihood == 1;
    const double pw = g.mean_mode ? 1.0 : 2.0;
    g.apow_f = (float)pw;
    g.syn0_f = g.mean_mode ? 0.f : (float)p->noise_var;
    g.inv_noise_f = (float)(1.0 / p->noise_var);
    g.twoftau_f = (float)(pw / (p->f_hz * p->tau));
    g.kap_f = (float)(pw * 1.4426950408889634074 / (p->f_hz * p->tau));
    for (int e = 0; e < 4; ++e) g.rho_f[e] = (float)std::exp2(-(double)g.kap_f * e);
    g.alpha_f = (float)p->alpha;
    g.beta_f = (float)p->beta_att;
    g.R_f = (float)p->R_max;
    g.noise_f = (float)p->noise_var;
    g.f_f = (float)p->f_hz;
    g.tau_f = (float)p->tau;
    g.v_f = (float)p->v;
    g.Tf = p->T * p->f_hz;
    g.TfK = (int)std::floor(g.Tf);
    g.lb0 = g.log_Lambda - g.log_WWT + 2.0;
    g.Cb0 = g.log_Lambda - g.log_WWT + g.log_T + g.log_pd - g.log_pb;
    g.lLWT = g.log_Lambda - g.log_WWT;
    g.lpdpb = g.log_pd - g.log_pb;
    g.bt_on = 0;
    if (g.ev_cap < g.k + 1) return fail(CMH_ERR_ARG);

    Dev& d = m->d;
    const size_t esz = g.f32 ? sizeof(float) : sizeof(double);
    std::vector<double> hx(n_stations), hy(n_stations);
    std::vector<float> hxf(n_stations), hyf(n_stations);
    for (int j = 0; j < n_stations; ++j) {
        hx[j] = stations[j].x;
        hy[j] = stations[j].y;
        hxf[j] = (float)hx[j];
        hyf[j] = (float)hy[j];
    }
    double *stx = nullptr, *sty = nullptr;
    cudaError_t e;
    if ((e = m->alloc(&stx, n_stations)) || (e = m->alloc(&sty, n_stations))) return fail(cuda_err(e));
    d.stx = stx;
    d.sty = sty;
    float *stxf = nullptr, *styf = nullptr;
    if ((e = m->alloc(&stxf, n_stations)) || (e = m->alloc(&styf, n_stations))) return fail(cuda_err(e));
    d.stxf = stxf;
    d.styf = styf;
    unsigned char *sig = nullptr, *V = nullptr;
    if ((e = m->alloc(&sig, (size_t)n_stations * g.pitch * esz)) ||
        (e = m->alloc(&V, (size_t)n_stations * g.pitch * esz)))
        return fail(cuda_err(e));
    d.sig = sig;
    d.V = V;
    int* nonfinite = nullptr;
    if ((e = m->alloc(&d.status, 1)) || (e = m->alloc(&d.sweep, 1)) || (e = m->alloc(&d.shift, 2)) ||
        (e = m->alloc(&d.logp, 1)) || (e = m->alloc(&d.stats, kStats)) || (e = m->alloc(&nonfinite, 1)))
        return fail(cuda_err(e));
    double* log_n = nullptr;
    if ((e = m->alloc(&log_n, g.ev_cap + 2))) return fail(cuda_err(e));
    d.log_n = log_n;
    m->n_partial = 1216;
    if ((e = m->alloc(&m->partial, m->n_partial))) return fail(cuda_err(e));
    m->flat_cap = m->p.max_events;
    if ((e = m->alloc(&m->flat.x, m->flat_cap)) || (e = m->alloc(&m->flat.y, m->flat_cap)) ||
        (e = m->alloc(&m->flat.t, m->flat_cap)) || (e = m->alloc(&m->flat.m, m->flat_cap)) ||
        (e = m->alloc(&m->flat.id, m->flat_cap)) || (e = m->alloc(&m->flat.n, 1)))
        return fail(cuda_err(e));
    if (g.sig_a > 0.0) {
        // latent arrival offsets of the flat list, 0 to start with
        const size_t cnt = (size_t)m->flat_cap * (size_t)std::max(n_stations, 1);
        if ((e = m->alloc(&m->flat.off, cnt)) || (e = m->alloc(&m->off_lp, 1))) return fail(cuda_err(e));
        if ((e = cudaMemsetAsync(m->flat.off, 0, sizeof(double) * cnt, m->stream))) return fail(cuda_err(e));
    }

    std::vector<double> ln(g.ev_cap + 2);
    ln[0] = -INFINITY;
    for (int i = 1; i < g.ev_cap + 2; ++i) ln[i] = std::log((double)i);
    cudaStream_t s = m->stream;
    if ((e = cudaMemcpyAsync(log_n, ln.data(), sizeof(double) * ln.size(), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(stx, hx.data(), sizeof(double) * n_stations, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(sty, hy.data(), sizeof(double) * n_stations, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(stxf, hxf.data(), sizeof(float) * n_stations, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(styf, hyf.data(), sizeof(float) * n_stations, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemsetAsync(d.status, 0, sizeof(int), s)) || (e = cudaMemsetAsync(nonfinite, 0, sizeof(int), s)) ||
        (e = cudaMemsetAsync(d.sweep, 0, sizeof(long long), s)) ||
        (e = cudaMemsetAsync(d.stats, 0, sizeof(unsigned long long) * kStats, s)) ||
        (e = cudaMemsetAsync(d.V, 0, (size_t)n_stations * g.pitch * esz, s)))
        return fail(cuda_err(e));

    // signals: copy (and convert) into the padded device buffer
    if (n_stations > 0) {
        const size_t ssz = sig_dtype == CMH_F32 ? sizeof(float) : sizeof(double);
        const void* src = signals;
        void* staged = nullptr;
        if (!signals_on_device) {
            e = cudaMalloc(&staged, (size_t)n_stations * n_samples * ssz);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(staged, n_samples * ssz, signals, row_pitch * ssz, n_samples * ssz, n_stations,
                                      cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                if (staged) cudaFree(staged);
                return fail(cuda_err(e));
            }
            src = staged;
        }
        e = launch_convert_signals(src, sig_dtype == CMH_F32, signals_on_device ? row_pitch : n_samples, sig,
                                   g.f32, g.pitch, n_stations, n_samples, nonfinite, s);
        m->launches += 1;
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (staged) cudaFree(staged);
        if (e != cudaSuccess) return fail(cuda_err(e));
        int bad = 0;
        if ((e = cudaMemcpy(&bad, nonfinite, sizeof(int), cudaMemcpyDeviceToHost))) return fail(cuda_err(e));
        if (bad) return fail(CMH_ERR_NONFINITE);
    }
    // initial events -> flat list -> V and the log-density
    {
        std::vector<double> ex(n_events), ey(n_events), et(n_events), em(n_events);
        std::vector<unsigned long long> id(n_events);
        for (int64_t i = 0; i < n_events; ++i) {
            ex[i] = init_events[i].x; ey[i] = init_events[i].y; et[i] = init_events[i].t; em[i] = init_events[i].m;
            id[i] = (unsigned long long)i;
        }
        const int n = (int)n_events;
        if ((e = cudaMemcpyAsync(m->flat.x, ex.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(m->flat.y, ey.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(m->flat.t, et.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(m->flat.m, em.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(m->flat.id, id.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(m->flat.n, &n, sizeof(int), cudaMemcpyHostToDevice, s)))
            return fail(cuda_err(e));
        double lp = 0.0;
        rc = synth_and_logdensity(m, n, &lp);
        if (rc) return fail(rc);
    }
    *out = m;
    return CMH_OK;
}

int cmh_partition_and_color(cmh_model* m, const cmh_grid* grid, int32_t shift_mode, double sx, double sy,
                            int32_t* n_colors_out) {
    (void)cudaGetLastError();   // an earlier call's failed launch must not be reported here
    if (!m || !grid) return CMH_ERR_ARG;
    if (m->latched) return CMH_ERR_STATE;
    const double L = grid->L;
    if (!finite_pos(L) || (shift_mode != 0 && shift_mode != 1)) return CMH_ERR_ARG;
    if (shift_mode == 0 && !(sx >= 0.0 && sx < L && sy >= 0.0 && sy < L)) return CMH_ERR_ARG;
    const int P = (int)std::ceil(2.0 * m->p.R_max / L) + 1;
    if (P * P > kMaxColours) return CMH_ERR_GEOMETRY;
    const double ncell_axis = std::floor(m->p.W / L) + 2;
    if (ncell_axis * ncell_axis > (double)(1 << 20)) return CMH_ERR_ARG;

    // current events -> flat list (the model's own order)
    int n_flat = (int)m->n0;
    if (m->partitioned) {
        int rc = flatten_current(m, &n_flat);
        if (rc) return rc;
        m->n0 = n_flat;   // until binned again, the flat list is the state
    }
    m->free_partition();
    m->partitioned = false;
    if (m->g.bt_on && (L / m->g.bt_hx + 4.0) * (L / m->g.bt_hy + 4.0) > 256.0) return CMH_ERR_ARG;

    Geo& g = m->g;
    g.L = L;
    g.invL_f = (float)(1.0 / L);
    g.shift_mode = shift_mode;
    g.sx_static = shift_mode == 0 ? sx : 0.0;
    g.sy_static = shift_mode == 0 ? sy : 0.0;
    g.ncx = g.ncy = (int)ncell_axis;
    g.n_cells = g.ncx * g.ncy;
    g.period = P;
    g.n_colours = P * P;
    g.max_rpc = ((g.ncx + P - 1) / P) * ((g.ncy + P - 1) / P);
    // capacities that depend on the station geometry (exact bounds)
    std::vector<double> hx(g.n_st), hy(g.n_st);
    if (g.n_st) {
        CK(cudaMemcpy(hx.data(), m->d.stx, sizeof(double) * g.n_st, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(hy.data(), m->d.sty, sizeof(double) * g.n_st, cudaMemcpyDeviceToHost));
    }
    const double Rm = m->p.R_max * 1.0001 + 1e-3;
    g.arr_cap = std::max(1, max_within(hx, hy, m->p.R_max));
    g.blk_cap = std::max(1, std::min(g.n_st, max_within(hx, hy, L * std::sqrt(0.5) + Rm)));
    g.store_cap = m->p.max_events + (long long)g.n_cells * g.k;
    if (g.store_cap > (1LL << 31) - 1) return CMH_ERR_ARG;
    if (n_flat > m->p.max_events) return CMH_ERR_CAPACITY;   // the new store could not hold them
    {
        int rc = ensure_flat(m, g.store_cap, n_flat);
        if (rc) return rc;
    }
    g.stage_cap = 0;
    // a step touches the old and new arrivals of one event, or of two with the
    // joint move of a pair
    g.task_cap = std::max(32, (g.p_pair > 0.0 ? 4 : 2) * g.arr_cap);
    g.spill = 0;
    g.spill_bytes = 0;
    // float32 regions whose arrival caches and lists do not fit in shared
    // memory keep those in a global slot per CTA
    if (g.f32 && phase32_smem_bytes(g) > 227 * 1024) {
        g.spill = 1;
        g.spill_bytes = (long long)phase32_spill_bytes(g);
    }
    if (g.f32) CK(choose_stage_cap(g, m->p.stage_samples));
    if ((g.f32 ? phase32_smem_bytes(g) : phase_smem_bytes(g)) > 227 * 1024) return CMH_ERR_CAPACITY;
    if (g.f32)
        CK(prepare_phase32(g));
    else
        CK(prepare_kernels(g));
    CK(prepare_rebin(g));
    m->sweep_grid = 0;
    if (g.f32 && m->p.schedule == 0) CK(sweep32_grid(g, m->p.ctas_per_sm, &m->sweep_grid));

    Dev& d = m->d;
    cudaError_t e;
    for (int b = 0; b < 2; ++b) {
        Store& S = d.st[b];
        if ((e = m->alloc(&S.x, g.store_cap, true)) || (e = m->alloc(&S.y, g.store_cap, true)) ||
            (e = m->alloc(&S.t, g.store_cap, true)) || (e = m->alloc(&S.m, g.store_cap, true)) ||
            (e = m->alloc(&S.id, g.store_cap, true)) || (e = m->alloc(&S.start, g.n_cells, true)) ||
            (e = m->alloc(&S.count, g.n_cells, true)) || (e = m->alloc(&S.cap, g.n_cells, true)) ||
            (e = m->alloc(&S.total, 1, true)))
            return cuda_err(e);
        S.off = nullptr;
        if (g.sig_a > 0.0) {   // latent arrival offsets, a row of n_st per store slot
            const size_t cnt = (size_t)g.store_cap * (size_t)std::max(g.n_st, 1);
            if ((e = m->alloc(&S.off, cnt, true))) return cuda_err(e);
            CK(cudaMemsetAsync(S.off, 0, sizeof(double) * cnt, m->stream));
        }
        CK(cudaMemsetAsync(S.count, 0, sizeof(int) * g.n_cells, m->stream));
        CK(cudaMemsetAsync(S.start, 0, sizeof(int) * g.n_cells, m->stream));
        CK(cudaMemsetAsync(S.total, 0, sizeof(int), m->stream));
    }
    if ((e = m->alloc(&d.colour_count, kMaxColours, true)) ||
        (e = m->alloc(&d.colour_cells, (size_t)g.n_colours * g.max_rpc, true)) ||
        (e = m->alloc(&d.fill, g.n_cells, true)) || (e = m->alloc(&d.ncell, g.store_cap, true)) ||
        (e = m->alloc(&d.cell_col, g.n_cells, true)) || (e = m->alloc(&d.colour_off, kMaxColours + 1, true)) ||
        (e = m->alloc(&d.queue, 1, true)) || (e = m->alloc(&d.done, g.n_cells, true)) ||
        (e = m->alloc(&d.region_dlp, g.n_cells, true)) || (e = m->alloc(&d.flat_off, g.n_cells + 1, true)))
        return cuda_err(e);
    {
        // blanket candidates: a cell's region is [s + (i-1) L, s + i L) per axis
        // (clipped to the domain) for a shift s in [0, L), so it lies inside
        // [(i-1) L, (i+1) L]; the stations within R_max (with room for the
        // kernel's float test and its margin) of that box
        std::vector<int> off(g.n_cells + 1), idx;
        const double Rc = m->p.R_max * 1.001 + 1.0, W = m->p.W;
        for (int c = 0; c < g.n_cells; ++c) {
            const int cx = c % g.ncx, cy = c / g.ncx;
            const double x0 = std::max(0.0, (cx - 1) * L), x1 = std::min(W, (cx + 1) * L);
            const double y0 = std::max(0.0, (cy - 1) * L), y1 = std::min(W, (cy + 1) * L);
            off[c] = (int)idx.size();
            for (int j = 0; j < g.n_st; ++j) {
                const double dx = hx[j] < x0 ? x0 - hx[j] : (hx[j] > x1 ? hx[j] - x1 : 0.0);
                const double dy = hy[j] < y0 ? y0 - hy[j] : (hy[j] > y1 ? hy[j] - y1 : 0.0);
                if (dx * dx + dy * dy < Rc * Rc) idx.push_back(j);
            }
        }
        off[g.n_cells] = (int)idx.size();
        int *doff = nullptr, *didx = nullptr;
        if ((e = m->alloc(&doff, off.size(), true)) || (e = m->alloc(&didx, idx.size(), true))) return cuda_err(e);
        CK(cudaMemcpy(doff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
        if (!idx.empty()) CK(cudaMemcpy(didx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice));
        d.bl_off = doff;
        d.bl_idx = didx;
    }
    if (g.spill) {
        // one slot per CTA that may run a region at once: every region of a
        // colour (colour-by-colour launch) or every resident CTA (persistent)
        int dev = 0, n_sm = 1;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
        const size_t slots = (size_t)std::max(g.max_rpc, 3 * n_sm);
        if ((e = m->alloc(&d.spill_buf, slots * (size_t)g.spill_bytes, true))) return cuda_err(e);
    } else {
        d.spill_buf = nullptr;
    }
    CK(cudaMemsetAsync(d.done, 0, sizeof(long long) * g.n_cells, m->stream));
    CK(cudaMemsetAsync(d.colour_off, 0, sizeof(int) * (kMaxColours + 1), m->stream));
    CK(cudaMemsetAsync(d.fill, 0, sizeof(int) * g.n_cells, m->stream));
    CK(cudaMemsetAsync(d.region_dlp, 0, sizeof(double) * g.n_cells, m->stream));
    CK(cudaMemsetAsync(d.colour_count, 0, sizeof(int) * kMaxColours, m->stream));
    if (m->trace_cap > 0) CK(cudaMemsetAsync(d.trace, 0, sizeof(cmh_trace) * m->trace_cap, m->stream));

    m->grid_L = L;
    m->shift_mode = shift_mode;
    m->sx0 = sx;
    m->sy0 = sy;
    int rc = bin_flat_into_current(m, n_flat);
    if (rc) return rc;
    m->partitioned = true;
    m->part_gen += 1;
    if (n_colors_out) *n_colors_out = g.n_colours;
    return CMH_OK;
}

int cmh_run_sweeps(cmh_model* m, int64_t n) {
    if (!m || n < 0) return CMH_ERR_ARG;
    if (!m->partitioned || m->latched) return CMH_ERR_STATE;
    if (n == 0) return CMH_OK;
    if (m->timing) {
        std::vector<cudaEvent_t> ev;
        ev.reserve((size_t)(2 * n * m->g.n_colours));
        int rc = CMH_OK;
        for (int64_t i = 0; i < n && rc == CMH_OK; ++i) {
            int l = 0;
            cudaError_t e = launch_rebin(m->g, m->d, -1, m->stream, &l);
            // one timed launch per colour phase, or one per sweep (persistent)
            const int n_launch = m->sweep_grid > 0 ? 1 : m->g.n_colours;
            for (int c = 0; c < n_launch && e == cudaSuccess; ++c) {
                cudaEvent_t a, b;
                cudaEventCreate(&a);
                cudaEventCreate(&b);
                ev.push_back(a);
                ev.push_back(b);
                cudaEventRecord(a, m->stream);
                e = m->sweep_grid > 0 ? launch_sweep32(m->g, m->d, m->sweep_grid, m->stream)
                                      : launch_phase(m->g, m->d, c, m->stream);
                cudaEventRecord(b, m->stream);
            }
            if (e == cudaSuccess) e = launch_sweep_end(m->g, m->d, m->stream);
            if (e != cudaSuccess) rc = cuda_err(e);
            m->launches += launches_per_sweep(m);
            m->sweeps += 1;
        }
        cudaError_t e = cudaStreamSynchronize(m->stream);
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) m->phase_ms += ms;
            m->phase_launches += 1;
        }
        for (cudaEvent_t x : ev) cudaEventDestroy(x);
        if (rc) return rc;
        return cuda_err(e);
    }
    if (!m->graph_exec) {
        int rc = capture_graph(m);
        if (rc) return rc;
    }
    for (int64_t i = 0; i < n; ++i) CK(cudaGraphLaunch(m->graph_exec, m->stream));
    m->launches += n * launches_per_sweep(m);
    m->sweeps += n;
    return CMH_OK;
}

int cmh_sync(cmh_model* m) {
    if (!m) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    return check_status(m);
}

int cmh_read_state(cmh_model* m, cmh_event* out, uint64_t* ids_out, int64_t cap, int64_t* n_out,
                   double* log_density_out, cmh_stats* stats_out) {
    if (!m || cap < 0 || (cap > 0 && !out)) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    int rc = check_status(m);
    if (rc) return rc;
    int n = (int)m->n0;
    if (m->partitioned) {
        rc = flatten_current(m, &n);
        if (rc) return rc;
    }
    if (n_out) *n_out = n;
    const int64_t nc = std::min<int64_t>(cap, n);
    if (nc > 0) {
        std::vector<double> x(nc), y(nc), t(nc), mm(nc);
        CK(cudaMemcpy(x.data(), m->flat.x, sizeof(double) * nc, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(y.data(), m->flat.y, sizeof(double) * nc, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(t.data(), m->flat.t, sizeof(double) * nc, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(mm.data(), m->flat.m, sizeof(double) * nc, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nc; ++i) out[i] = cmh_event{x[i], y[i], t[i], mm[i]};
        if (ids_out) CK(cudaMemcpy(ids_out, m->flat.id, sizeof(uint64_t) * nc, cudaMemcpyDeviceToHost));
    }
    if (log_density_out) CK(cudaMemcpy(log_density_out, m->d.logp, sizeof(double), cudaMemcpyDeviceToHost));
    if (stats_out) {
        unsigned long long st[kStats];
        CK(cudaMemcpy(st, m->d.stats, sizeof(st), cudaMemcpyDeviceToHost));
        std::memset(stats_out, 0, sizeof(*stats_out));
        for (int i = 0; i < 3; ++i) {
            stats_out->proposed[i] = st[i];
            stats_out->evaluated[i] = st[3 + i];
            stats_out->accepted[i] = st[6 + i];
        }
        stats_out->sweeps = m->sweeps;
        stats_out->n_events = n;
        stats_out->phase_ms = m->phase_ms;
        stats_out->phase_launches = m->phase_launches;
        stats_out->kernel_launches = m->launches;
        stats_out->priced_samples = st[9];
        stats_out->rewritten_samples = st[10];
        stats_out->spill_bytes = m->partitioned && m->g.spill ? m->g.spill_bytes : 0;
        for (int i = 0; i < 3; ++i) stats_out->pair[i] = st[11 + i];
        for (int i = 0; i < 3; ++i) stats_out->arrival[i] = st[14 + i];
        stats_out->unique_samples = st[17];
    }
    return CMH_OK;
}

int cmh_set_arrival_offsets(cmh_model* m, const double* off, int64_t n_events, int32_t n_stations) {
    (void)cudaGetLastError();   // an earlier call's failed launch must not be reported here
    if (!m || n_events < 0 || (n_events > 0 && n_stations > 0 && !off)) return CMH_ERR_ARG;
    if (!m->flat.off || n_stations != m->g.n_st || n_events != m->n0) return CMH_ERR_ARG;
    if (m->partitioned || m->latched) return CMH_ERR_STATE;
    const size_t cnt = (size_t)n_events * (size_t)n_stations;
    for (size_t q = 0; q < cnt; ++q)
        if (!std::isfinite(off[q])) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    if (cnt) CK(cudaMemcpy(m->flat.off, off, sizeof(double) * cnt, cudaMemcpyHostToDevice));
    // V with the shifted arrivals, and the log-density with the offsets' prior
    double lp = 0.0;
    return synth_and_logdensity(m, (int)n_events, &lp);
}

int cmh_read_arrival_offsets(cmh_model* m, double* out, int64_t cap, int64_t* n_out) {
    if (!m || cap < 0 || (cap > 0 && !out)) return CMH_ERR_ARG;
    if (!m->flat.off) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    int rc = check_status(m);
    if (rc) return rc;
    int n = (int)m->n0;
    if (m->partitioned) {
        rc = flatten_current(m, &n);
        if (rc) return rc;
    }
    if (n_out) *n_out = n;
    const int64_t nc = std::min<int64_t>(cap, n);
    if (nc > 0 && m->g.n_st > 0)
        CK(cudaMemcpy(out, m->flat.off, sizeof(double) * (size_t)nc * m->g.n_st, cudaMemcpyDeviceToHost));
    return CMH_OK;
}

int cmh_log_density(cmh_model* m, double* out) {
    if (!m || !out) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    int rc = check_status(m);
    if (rc) return rc;
    int n = (int)m->n0;
    if (m->partitioned) {
        rc = flatten_current(m, &n);
        if (rc) return rc;
    }
    return synth_and_logdensity(m, n, out);
}

int cmh_set_trace(cmh_model* m, int64_t capacity) {
    if (!m || capacity < 0) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    m->drop_graph();
    if (m->d.trace) {
        cudaFree(m->d.trace);
        auto it = std::find(m->allocs.begin(), m->allocs.end(), (void*)m->d.trace);
        if (it != m->allocs.end()) m->allocs.erase(it);
        m->d.trace = nullptr;
    }
    m->trace_cap = capacity;
    m->d.trace_cap = capacity;
    m->d.trace_sweep0 = m->sweeps;
    if (capacity > 0) {
        cudaError_t e = m->alloc(&m->d.trace, capacity);
        if (e) return cuda_err(e);
        CK(cudaMemsetAsync(m->d.trace, 0, sizeof(cmh_trace) * capacity, m->stream));
    }
    return CMH_OK;
}

int cmh_read_trace(cmh_model* m, cmh_trace* out, int64_t cap, int64_t* n_out) {
    if (!m || cap < 0 || (cap > 0 && !out)) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    std::vector<cmh_trace> all(m->trace_cap);
    if (m->trace_cap) CK(cudaMemcpy(all.data(), m->d.trace, sizeof(cmh_trace) * m->trace_cap, cudaMemcpyDeviceToHost));
    int64_t n = 0;
    for (const cmh_trace& r : all) {
        if (!r.written) continue;
        if (n < cap) out[n] = r;
        ++n;
    }
    if (n_out) *n_out = n;
    return CMH_OK;
}

int cmh_test_hold_region(cmh_model* m, int32_t cell, uint32_t wait_limit) {
    if (!m) return CMH_ERR_ARG;
    if (!m->partitioned || !m->g.f32 || m->sweep_grid <= 0) return CMH_ERR_STATE;
    if (cell < -1 || cell >= m->g.n_cells) return CMH_ERR_ARG;
    m->g.hold_cell = cell;
    m->g.dep_wait_limit = wait_limit ? wait_limit : kDepWaitLimitDefault;
    m->drop_graph();   // the captured sweep holds the old constants
    return CMH_OK;
}

int cmh_set_timing(cmh_model* m, int32_t enable) {
    if (!m) return CMH_ERR_ARG;
    m->timing = enable ? 1 : 0;
    // timed sweeps also count each region phase's unique window samples; the
    // captured graph (untimed sweeps) keeps the constants it was captured with
    m->g.count_unique = m->timing && m->g.f32 ? 1 : 0;
    return CMH_OK;
}

int cmh_read_shift(cmh_model* m, double* sx, double* sy) {
    if (!m || !sx || !sy) return CMH_ERR_ARG;
    if (!m->partitioned) return CMH_ERR_STATE;
    double s[2];
    CK(cudaMemcpyAsync(s, m->d.shift, sizeof(s), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    *sx = s[0];
    *sy = s[1];
    return CMH_OK;
}

namespace {
struct CkptHeader {
    uint64_t magic;
    int32_t version, shift_mode;
    cmh_params p;
    int64_t n_st, n_samp, sweeps, n_events;
    double L, sx, sy, logp;
    uint64_t stats[kStats];
    int32_t partitioned, pad;
};
}  // namespace

int cmh_checkpoint(cmh_model* m, void* buf, size_t* len) {
    if (!m || !len) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    int rc = check_status(m);
    if (rc) return rc;
    int n = (int)m->n0;
    if (m->partitioned) {
        rc = flatten_current(m, &n);
        if (rc) return rc;
    }
    const size_t orow = m->flat.off ? sizeof(double) * (size_t)m->g.n_st : 0;   // latent offsets per event
    const size_t need = sizeof(CkptHeader) + (size_t)n * (4 * sizeof(double) + sizeof(uint64_t) + orow);
    if (!buf) { *len = need; return CMH_OK; }
    if (*len < need) { *len = need; return CMH_ERR_ARG; }
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kCkptMagic;
    h.version = kCkptVersion;
    h.shift_mode = m->shift_mode;
    h.p = m->p;
    h.n_st = m->g.n_st;
    h.n_samp = m->g.n_samp;
    h.sweeps = m->sweeps;
    h.n_events = n;
    h.L = m->grid_L;
    h.sx = m->sx0;
    h.sy = m->sy0;
    h.partitioned = m->partitioned;
    CK(cudaMemcpy(&h.logp, m->d.logp, sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(h.stats, m->d.stats, sizeof(h.stats), cudaMemcpyDeviceToHost));
    unsigned char* q = (unsigned char*)buf;
    std::memcpy(q, &h, sizeof(h));
    q += sizeof(h);
    if (n) {
        CK(cudaMemcpy(q, m->flat.x, sizeof(double) * n, cudaMemcpyDeviceToHost)); q += sizeof(double) * n;
        CK(cudaMemcpy(q, m->flat.y, sizeof(double) * n, cudaMemcpyDeviceToHost)); q += sizeof(double) * n;
        CK(cudaMemcpy(q, m->flat.t, sizeof(double) * n, cudaMemcpyDeviceToHost)); q += sizeof(double) * n;
        CK(cudaMemcpy(q, m->flat.m, sizeof(double) * n, cudaMemcpyDeviceToHost)); q += sizeof(double) * n;
        CK(cudaMemcpy(q, m->flat.id, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost)); q += sizeof(uint64_t) * n;
        if (orow) CK(cudaMemcpy(q, m->flat.off, orow * n, cudaMemcpyDeviceToHost));
    }
    *len = need;
    return CMH_OK;
}

int cmh_restore(cmh_model* m, const void* buf, size_t len) {
    (void)cudaGetLastError();   // an earlier call's failed launch must not be reported here
    if (!m || !buf || len < sizeof(CkptHeader)) return CMH_ERR_ARG;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kCkptMagic || h.version != kCkptVersion) return CMH_ERR_ARG;
    if (h.n_st != m->g.n_st || h.n_samp != m->g.n_samp || h.n_events < 0 || h.n_events > m->flat_cap ||
        h.p.dtype != m->p.dtype || h.p.seed != m->p.seed || (h.p.sig_a > 0.0) != (m->p.sig_a > 0.0))
        return CMH_ERR_ARG;
    const size_t orow = m->flat.off ? sizeof(double) * (size_t)m->g.n_st : 0;
    const size_t need = sizeof(CkptHeader) + (size_t)h.n_events * (4 * sizeof(double) + sizeof(uint64_t) + orow);
    if (len < need) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(m->stream));
    const int n = (int)h.n_events;
    const unsigned char* q = (const unsigned char*)buf + sizeof(h);
    const double* x = (const double*)q;
    const double* y = x + n;
    const double* t = y + n;
    const double* mm = t + n;
    for (int i = 0; i < n; ++i)
        if (!(x[i] >= 0.0 && x[i] < m->p.W && y[i] >= 0.0 && y[i] < m->p.W && t[i] >= 0.0 && t[i] < m->p.T &&
              mm[i] >= 2.0))
            return CMH_ERR_ARG;
    CK(cudaMemcpy(m->flat.x, x, sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->flat.y, y, sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->flat.t, t, sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->flat.m, mm, sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->flat.id, mm + n, sizeof(uint64_t) * n, cudaMemcpyHostToDevice));
    if (orow && n)
        CK(cudaMemcpy(m->flat.off, (const unsigned char*)(mm + n) + sizeof(uint64_t) * n, orow * n,
                      cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->flat.n, &n, sizeof(int), cudaMemcpyHostToDevice));
    double lp = 0.0;
    int rc = synth_and_logdensity(m, n, &lp);
    if (rc) return rc;
    CK(cudaMemcpy(m->d.logp, &h.logp, sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d.stats, h.stats, sizeof(h.stats), cudaMemcpyHostToDevice));
    m->latched = 0;
    CK(cudaMemset(m->d.status, 0, sizeof(int)));
    m->free_partition();
    m->partitioned = false;
    m->sweeps = h.sweeps;
    m->n0 = n;
    rc = upload_sweep(m, h.sweeps);
    if (rc) return rc;
    if (h.partitioned) {
        cmh_grid gr{h.L};
        // the flat list already holds the events: partition bins it
        rc = cmh_partition_and_color(m, &gr, h.shift_mode, h.sx, h.sy, nullptr);
        if (rc) return rc;
    }
    return CMH_OK;
}

void cmh_destroy(cmh_model* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    m->free_partition();
    for (void* q : m->allocs) cudaFree(q);
    m->allocs.clear();
    if (m->bt_mass) cudaFree(m->bt_mass);
    if (m->bt_cdf) cudaFree(m->bt_cdf);
    if (m->bt_tab) cudaFree(m->bt_tab);
    if (m->bt_mag) cudaFree(m->bt_mag);
    for (auto& r : m->rs) {
        if (r.host) cudaFreeHost(r.host);
        if (r.ev) cudaEventDestroy(r.ev);
    }
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

namespace {
// byte offsets inside a read slot of capacity cap
inline size_t rs_off_id(long long cap) { return (size_t)cap * 4 * sizeof(double); }
inline size_t rs_off_logp(long long cap) { return rs_off_id(cap) + (size_t)cap * sizeof(unsigned long long); }
inline size_t rs_off_stats(long long cap) { return rs_off_logp(cap) + sizeof(double); }
inline size_t rs_off_n(long long cap) { return rs_off_stats(cap) + kStats * sizeof(unsigned long long); }
inline size_t rs_off_status(long long cap) { return rs_off_n(cap) + sizeof(int); }
inline size_t rs_bytes(long long cap) { return rs_off_n(cap) + 16; }
}  // namespace

int cmh_read_state_async(cmh_model* m, int32_t slot) {
    if (!m || slot < 0 || slot > 1) return CMH_ERR_ARG;
    if (!m->partitioned) return CMH_ERR_STATE;
    if (m->latched) return m->latched;
    (void)cudaGetLastError();
    cmh_model::ReadSlot& r = m->rs[slot];
    if (r.pending) CK(cudaEventSynchronize(r.ev));   // its previous request is still being read
    r.pending = false;
    if (!r.ev) CK(cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming));
    if (r.cap < m->flat_cap) {
        if (r.host) CK(cudaFreeHost(r.host));
        r.host = nullptr;
        r.cap = 0;
        if (cudaHostAlloc((void**)&r.host, rs_bytes(m->flat_cap), cudaHostAllocMapped) != cudaSuccess) {
            r.host = nullptr;
            return CMH_ERR_OOM;
        }
        r.cap = m->flat_cap;
    }
    unsigned char* dev = nullptr;
    CK(cudaHostGetDevicePointer((void**)&dev, r.host, 0));
    FlatList f;
    f.x = (double*)dev;
    f.y = f.x + r.cap;
    f.t = f.y + r.cap;
    f.m = f.t + r.cap;
    f.id = (unsigned long long*)(dev + rs_off_id(r.cap));
    f.n = (int*)(dev + rs_off_n(r.cap));
    f.off = nullptr;   // offsets are read by cmh_read_arrival_offsets
    int l = 0;
    CK(launch_flatten(m->g, m->d, cur_buf(m), f, m->stream, &l));
    CK(cudaMemcpyAsync(r.host + rs_off_logp(r.cap), m->d.logp, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(r.host + rs_off_stats(r.cap), m->d.stats, kStats * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(r.host + rs_off_status(r.cap), m->d.status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaEventRecord(r.ev, m->stream));
    m->launches += l;
    r.sweeps = m->sweeps;
    r.launches = m->launches;
    r.phase_launches = m->phase_launches;
    r.phase_ms = m->phase_ms;
    r.pending = true;
    return CMH_OK;
}

int cmh_read_state_fetch(cmh_model* m, int32_t slot, cmh_event* out, uint64_t* ids_out, int64_t cap,
                         int64_t* n_out, double* log_density_out, cmh_stats* stats_out) {
    if (!m || slot < 0 || slot > 1 || cap < 0 || (cap > 0 && !out)) return CMH_ERR_ARG;
    cmh_model::ReadSlot& r = m->rs[slot];
    if (!r.pending) return CMH_ERR_STATE;
    CK(cudaEventSynchronize(r.ev));
    // the device status as of the request (the stream may hold later work)
    const int st_dev = *(volatile int*)(r.host + rs_off_status(r.cap));
    if (st_dev && !m->latched) m->latched = st_dev;
    if (m->latched) {
        r.pending = false;
        return m->latched;
    }
    const int n = *(volatile int*)(r.host + rs_off_n(r.cap));
    if (n_out) *n_out = n;
    if (!out && cap == 0 && !ids_out && !log_density_out && !stats_out) return CMH_OK;   // a query of n
    const int64_t nc = std::min<int64_t>(cap, n);
    const double* x = (const double*)r.host;
    for (int64_t i = 0; i < nc; ++i) out[i] = cmh_event{x[i], x[r.cap + i], x[2 * r.cap + i], x[3 * r.cap + i]};
    if (ids_out && nc > 0) std::memcpy(ids_out, r.host + rs_off_id(r.cap), sizeof(uint64_t) * nc);
    if (log_density_out) std::memcpy(log_density_out, r.host + rs_off_logp(r.cap), sizeof(double));
    if (stats_out) {
        const unsigned long long* st = (const unsigned long long*)(r.host + rs_off_stats(r.cap));
        std::memset(stats_out, 0, sizeof(*stats_out));
        for (int i = 0; i < 3; ++i) {
            stats_out->proposed[i] = st[i];
            stats_out->evaluated[i] = st[3 + i];
            stats_out->accepted[i] = st[6 + i];
        }
        stats_out->sweeps = r.sweeps;
        stats_out->n_events = n;
        stats_out->phase_ms = r.phase_ms;
        stats_out->phase_launches = r.phase_launches;
        stats_out->kernel_launches = r.launches;
        stats_out->priced_samples = st[9];
        stats_out->rewritten_samples = st[10];
        stats_out->spill_bytes = m->g.spill ? m->g.spill_bytes : 0;
        for (int i = 0; i < 3; ++i) stats_out->pair[i] = st[11 + i];
        for (int i = 0; i < 3; ++i) stats_out->arrival[i] = st[14 + i];
        stats_out->unique_samples = st[17];
    }
    r.pending = false;
    return CMH_OK;
}

int cmh_philox4x64(const uint64_t* ctr, const uint64_t* key, uint64_t* out, int64_t n) {
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return CMH_ERR_ARG;
    if (n == 0) return CMH_OK;
    unsigned long long *dc = nullptr, *dk = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dc, sizeof(uint64_t) * 4 * n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(uint64_t) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint64_t) * 4 * n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint64_t) * 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, sizeof(uint64_t) * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox_test(dc, dk, dout, n, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint64_t) * 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return cuda_err(e);
}

}  // extern "C"

namespace cmh {
Geo cmh_model_geo(const cmh_model* m) { return m->g; }
Dev cmh_model_dev(const cmh_model* m) { return m->d; }
}  // namespace cmh

// ---------------------------------------------------------------------------
// learned birth component
// ---------------------------------------------------------------------------
extern "C" int cmh_set_birth_table(cmh_model* m, const float* tab, int32_t nx, int32_t ny, int32_t nt,
                                   double mix) {
    if (!m) return CMH_ERR_ARG;
    if (m->latched) return CMH_ERR_STATE;
    if (nx == 0) {   // back to uniform births
        m->g.bt_on = 0;
        m->g.bt_mag_on = 0;
        m->part_gen += 1;
        m->drop_graph();
        return CMH_OK;
    }
    if (!m->g.f32 || !tab || nx < 1 || ny < 1 || nt < 1 || !(mix > 0.0 && mix < 1.0)) return CMH_ERR_ARG;
    const long long np = (long long)nx * ny;
    if (np * nt > (1LL << 31)) return CMH_ERR_ARG;
    // pixels a region's range may span (one pixel of margin each way)
    if (m->partitioned) {
        const double px = m->grid_L / (m->p.W / nx) + 4.0, py = m->grid_L / (m->p.W / ny) + 4.0;
        if (px * py > 256.0) return CMH_ERR_ARG;
    }
    // per pixel: mass and cdf, running sums in index order in float64
    std::vector<double> mass(np), cdf((size_t)(np * nt));
    for (long long q = 0; q < np; ++q) {
        double run = 0.0;
        for (int b = 0; b < nt; ++b) {
            const double v = (double)tab[q * nt + b];
            if (!(v >= 0.0) || std::isinf(v)) return CMH_ERR_NONFINITE;
            run += v;
            cdf[q * nt + b] = run;
        }
        mass[q] = run;
        for (int b = 0; b < nt; ++b) cdf[q * nt + b] = run > 0.0 ? cdf[q * nt + b] / run : 0.0;
    }
    CK(cudaStreamSynchronize(m->stream));
    if (m->bt_mass) cudaFree(m->bt_mass);
    if (m->bt_cdf) cudaFree(m->bt_cdf);
    if (m->bt_tab) cudaFree(m->bt_tab);
    if (m->bt_mag) cudaFree(m->bt_mag);
    m->bt_mass = m->bt_cdf = nullptr;
    m->bt_tab = m->bt_mag = nullptr;
    m->g.bt_on = 0;
    m->g.bt_mag_on = 0;
    m->part_gen += 1;
    m->drop_graph();   // the captured sweep holds the old parameters
    if (cudaMalloc(&m->bt_mass, sizeof(double) * np) || cudaMalloc(&m->bt_cdf, sizeof(double) * np * nt) ||
        cudaMalloc(&m->bt_tab, sizeof(float) * np * nt))
        return CMH_ERR_OOM;
    CK(cudaMemcpy(m->bt_mass, mass.data(), sizeof(double) * np, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->bt_cdf, cdf.data(), sizeof(double) * np * nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->bt_tab, tab, sizeof(float) * np * nt, cudaMemcpyHostToDevice));
    Geo& g = m->g;
    g.bt_on = 1;
    g.bt_nx = nx;
    g.bt_ny = ny;
    g.bt_nt = nt;
    g.bt_mix = mix;
    g.bt_hx = m->p.W / (double)nx;
    g.bt_hy = m->p.W / (double)ny;
    g.bt_dt = m->p.T / (double)nt;
    g.bt_pixarea = g.bt_hx * g.bt_hy;
    g.bt_ihx = 1.0 / g.bt_hx;
    g.bt_ihy = 1.0 / g.bt_hy;
    g.bt_idt = 1.0 / g.bt_dt;
    m->d.bt_mass = m->bt_mass;
    m->d.bt_cdf = m->bt_cdf;
    m->d.bt_tab = m->bt_tab;
    m->drop_graph();   // the captured sweep holds the old parameters
    return CMH_OK;
}

extern "C" int cmh_set_birth_magnitude(cmh_model* m, const float* centre, double half_width) {
    if (!m) return CMH_ERR_ARG;
    if (m->latched) return CMH_ERR_STATE;
    if (!centre) {   // back to magnitudes from the prior
        m->g.bt_mag_on = 0;
        m->part_gen += 1;
        m->drop_graph();
        return CMH_OK;
    }
    if (!m->g.bt_on) return CMH_ERR_STATE;
    if (!(half_width > 0.0) || std::isinf(half_width)) return CMH_ERR_ARG;
    const long long n = (long long)m->g.bt_nx * m->g.bt_ny * m->g.bt_nt;
    for (long long i = 0; i < n; ++i)
        if (!std::isfinite(centre[i])) return CMH_ERR_NONFINITE;
    CK(cudaStreamSynchronize(m->stream));
    m->g.bt_mag_on = 0;
    m->part_gen += 1;
    m->drop_graph();   // the captured sweep holds the old parameters
    if (!m->bt_mag && cudaMalloc(&m->bt_mag, sizeof(float) * n) != cudaSuccess) {
        m->bt_mag = nullptr;
        return CMH_ERR_OOM;
    }
    CK(cudaMemcpy(m->bt_mag, centre, sizeof(float) * n, cudaMemcpyHostToDevice));
    m->d.bt_mag = m->bt_mag;
    m->g.bt_h = half_width;
    m->g.bt_h2 = 2.0 * half_width;
    m->g.bt_ih2 = 1.0 / (2.0 * half_width);
    m->g.bt_mag_on = 1;
    return CMH_OK;
}

// ---------------------------------------------------------------------------
// autotuning of the launch configuration
// ---------------------------------------------------------------------------
extern "C" int cmh_autotune(cmh_model* m, int32_t trial_sweeps, cmh_tuning* out) {
    if (!m || !out || trial_sweeps < 1) return CMH_ERR_ARG;
    if (!m->partitioned || m->latched) return CMH_ERR_STATE;
    if (!m->g.f32) return CMH_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    size_t len = 0;
    int rc = cmh_checkpoint(m, nullptr, &len);
    if (rc) return rc;
    std::vector<unsigned char> ck(len);
    if ((rc = cmh_checkpoint(m, ck.data(), &len))) return rc;
    const cmh_params keep = m->p;
    const long long launches0 = m->launches;
    struct Cand { int schedule, stage, ctas; };
    const Cand cands[] = {{1, 0, 0}, {1, -1, 0}, {0, 0, 3}, {0, 0, 2}, {0, 0, 1}, {0, -1, 0}};
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    double best = -1.0;
    int best_i = -1;
    for (const Cand& c : cands) {
        const int i = out->n_tried++;
        out->tried_schedule[i] = c.schedule;
        out->tried_stage[i] = c.stage;
        out->tried_ctas[i] = c.ctas;
        out->tried_ms[i] = -1.0;
        m->p = keep;
        m->p.schedule = c.schedule;
        m->p.stage_samples = c.stage;
        m->p.ctas_per_sm = c.ctas;
        if ((keep.p_pair > 0.0 || keep.sig_a > 0.0) && c.stage != 0) continue;   // no staging with these moves
        if (cmh_restore(m, ck.data(), len) != CMH_OK) continue;   // does not fit: skip it
        if (cmh_run_sweeps(m, 1) != CMH_OK) continue;             // warm-up (and graph capture)
        cudaEventRecord(a, m->stream);
        if (cmh_run_sweeps(m, trial_sweeps) != CMH_OK) continue;
        cudaEventRecord(b, m->stream);
        if (cudaEventSynchronize(b) != cudaSuccess || check_status(m) != CMH_OK) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        out->tried_ms[i] = ms / trial_sweeps;
        if (best < 0.0 || out->tried_ms[i] < best) {
            best = out->tried_ms[i];
            best_i = i;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    m->p = keep;
    if (best_i >= 0) {
        m->p.schedule = out->tried_schedule[best_i];
        m->p.stage_samples = out->tried_stage[best_i];
        m->p.ctas_per_sm = out->tried_ctas[best_i];
    }
    m->latched = 0;
    if ((rc = cmh_restore(m, ck.data(), len))) return rc;
    m->launches = launches0;   // the trials are not part of the chain
    out->schedule = m->p.schedule;
    out->stage_samples = m->p.stage_samples;
    out->ctas_per_sm = m->p.ctas_per_sm;
    out->ms_per_sweep = best;
    return best_i >= 0 ? CMH_OK : CMH_ERR_STATE;
}

// ---------------------------------------------------------------------------
// batches of independent models
// ---------------------------------------------------------------------------
// Models are grouped by how many of their region CTAs fit on an SM (the
// shared memory one region needs): each group gets its own persistent launch
// with its own queue and shared-memory size, and the groups run concurrently
// (forked branches of the sweep's graph) between the common re-binning and
// sweep-end launches.
struct BatchGroup {
    Geo* G = nullptr;
    Dev* D = nullptr;
    int* item_tab = nullptr;
    int* queue = nullptr;
    int n = 0, n_col = 0, grid = 0;
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

struct cmh_batch {
    std::vector<cmh_model*> models;
    std::vector<long long> gens;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Geo* G = nullptr;
    Dev* D = nullptr;
    int* blk_off = nullptr;
    int n = 0, n_blocks = 0, max_ev_cap = 0;
    std::vector<BatchGroup> groups;
    cudaEvent_t fork = nullptr, finished = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    void release() {
        if (stream) cudaStreamSynchronize(stream);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (BatchGroup& q : groups) {
            for (void* x : {(void*)q.G, (void*)q.D, (void*)q.item_tab, (void*)q.queue})
                if (x) cudaFree(x);
            if (q.stream) cudaStreamDestroy(q.stream);
            if (q.done) cudaEventDestroy(q.done);
        }
        for (void* x : {(void*)G, (void*)D, (void*)blk_off})
            if (x) cudaFree(x);
        if (fork) cudaEventDestroy(fork);
        if (finished) cudaEventDestroy(finished);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};


extern "C" int cmh_batch_create(cmh_model* const* models, int32_t n_models, void* cuda_stream, cmh_batch** out) {
    (void)cudaGetLastError();   // an earlier call's failed launch must not be reported here
    if (!out || !models || n_models < 1) return CMH_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n_models; ++i) {
        const cmh_model* m = models[i];
        if (!m) return CMH_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (models[j] == m) return CMH_ERR_ARG;   // each model once
        if (!m->partitioned || m->latched) return CMH_ERR_STATE;
        if (!m->g.f32 || m->g.stage_cap != 0 || m->g.ev_cap > 512 || m->g.p_pair > 0.0 || m->g.sig_a > 0.0)
            return CMH_ERR_ARG;
    }
    cmh_batch* b = new cmh_batch;
    auto fail = [&](int rc) {
        b->release();
        delete b;
        return rc;
    };
    b->n = n_models;
    b->models.assign(models, models + n_models);
    b->stream = (cudaStream_t)cuda_stream;
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(CMH_ERR_CUDA);
        b->own_stream = true;
    }
    int dev = 0, per_sm = 0, reserved = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev))
        return fail(CMH_ERR_CUDA);
    std::vector<Geo> hg(n_models);
    std::vector<Dev> hd(n_models);
    std::vector<int> off(n_models + 1, 0);
    std::vector<int> fit(n_models);
    for (int i = 0; i < n_models; ++i) {
        cmh_model* m = models[i];
        if (cudaStreamSynchronize(m->stream) != cudaSuccess) return fail(CMH_ERR_CUDA);
        hg[i] = m->g;
        hd[i] = m->d;
        b->gens.push_back(m->part_gen);
        off[i + 1] = off[i] + rebin_blocks(m->g);
        b->max_ev_cap = std::max(b->max_ev_cap, m->g.ev_cap);
        const size_t sm = phase32_smem_bytes(m->g);
        if (sm > 227 * 1024) return fail(CMH_ERR_CAPACITY);
        if (m->g.mean_mode != models[0]->g.mean_mode) return fail(CMH_ERR_ARG);   // one likelihood reading per batch
        // region CTAs of this model that fit on one SM (static shared memory ~2 KB)
        fit[i] = std::max(1, std::min(3, (int)(per_sm / (sm + 2048 + (size_t)reserved))));
    }
    b->n_blocks = off[n_models];
    if (cudaMalloc(&b->G, sizeof(Geo) * n_models) || cudaMalloc(&b->D, sizeof(Dev) * n_models) ||
        cudaMalloc(&b->blk_off, sizeof(int) * (n_models + 1)))
        return fail(CMH_ERR_OOM);
    if (cudaMemcpy(b->G, hg.data(), sizeof(Geo) * n_models, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->D, hd.data(), sizeof(Dev) * n_models, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->blk_off, off.data(), sizeof(int) * (n_models + 1), cudaMemcpyHostToDevice))
        return fail(CMH_ERR_CUDA);
    if (prepare_rebin_batch(b->max_ev_cap)) return fail(CMH_ERR_CUDA);
    // a group's sweep lasts as long as its slowest instance's colour chain:
    // the work queue takes instances by an estimate of their region cost
    // (events per region x blanket stations), largest first, so the longest
    // chains start first (each model's own chain does not depend on the order)
    std::vector<double> cost(n_models);
    for (int i = 0; i < n_models; ++i) {
        const cmh_model* m = models[i];
        const double per_region = (double)std::max<long long>(m->n0, 1) / std::max(1, hg[i].n_cells);
        cost[i] = (per_region + hg[i].k) * hg[i].blk_cap * (hg[i].spill ? 2.0 : 1.0);
    }
    std::vector<int> order(n_models);
    for (int i = 0; i < n_models; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    for (int f = 3; f >= 1; --f) {   // groups: 3, 2, then 1 resident region per SM
        std::vector<Geo> gg;
        std::vector<Dev> gd;
        BatchGroup q;
        for (int i : order)
            if (fit[i] == f) {
                gg.push_back(hg[i]);
                gd.push_back(hd[i]);
                q.n_col = std::max(q.n_col, hg[i].n_colours);
                q.smem = std::max(q.smem, phase32_smem_bytes(hg[i]));
            }
        if (gg.empty()) continue;
        q.n = (int)gg.size();
        b->groups.push_back(q);
        BatchGroup& r = b->groups.back();
        if (cudaMalloc(&r.G, sizeof(Geo) * r.n) || cudaMalloc(&r.D, sizeof(Dev) * r.n) ||
            cudaMalloc(&r.item_tab, sizeof(int) * ((size_t)r.n_col * r.n + 1)) || cudaMalloc(&r.queue, sizeof(int)))
            return fail(CMH_ERR_OOM);
        if (cudaMemcpy(r.G, gg.data(), sizeof(Geo) * r.n, cudaMemcpyHostToDevice) ||
            cudaMemcpy(r.D, gd.data(), sizeof(Dev) * r.n, cudaMemcpyHostToDevice))
            return fail(CMH_ERR_CUDA);
        if (prepare_sweep32_batch(r.smem, &r.grid)) return fail(CMH_ERR_CUDA);
        if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) ||
            cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming))
            return fail(CMH_ERR_CUDA);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) ||
        cudaEventCreateWithFlags(&b->finished, cudaEventDisableTiming))
        return fail(CMH_ERR_CUDA);
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(CMH_ERR_CUDA);
    cudaError_t e = launch_rebin_batch(b->G, b->D, b->blk_off, b->n, b->n_blocks, b->max_ev_cap, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    for (BatchGroup& r : b->groups) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(r.stream, b->fork, 0);
        if (e == cudaSuccess)
            e = launch_sweep32_batch(hg[0].mean_mode != 0, r.G, r.D, r.n, r.n_col, r.item_tab, r.queue, r.smem, r.grid,
                                     r.stream);
        if (e == cudaSuccess) e = cudaEventRecord(r.done, r.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, r.done, 0);
    }
    if (e == cudaSuccess) e = launch_sweep_end_batch(b->G, b->D, b->n, b->stream);
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &b->graph);
    if (e != cudaSuccess || e2 != cudaSuccess) return fail(CMH_ERR_CUDA);
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return fail(CMH_ERR_CUDA);
    *out = b;
    return CMH_OK;
}

extern "C" int cmh_batch_run_sweeps(cmh_batch* b, int64_t n) {
    if (!b || n < 0) return CMH_ERR_ARG;
    for (int i = 0; i < b->n; ++i) {
        const cmh_model* m = b->models[i];
        if (m->latched || !m->partitioned || m->part_gen != b->gens[i]) return CMH_ERR_STATE;
    }
    if (n == 0) return CMH_OK;
    for (int i = 0; i < b->n; ++i)   // the models' own queued work first
        CK(cudaStreamSynchronize(b->models[i]->stream));
    for (int64_t s = 0; s < n; ++s) CK(cudaGraphLaunch(b->exec, b->stream));
    // later calls on a model's own stream wait for these sweeps
    CK(cudaEventRecord(b->finished, b->stream));
    for (int i = 0; i < b->n; ++i) {
        cmh_model* m = b->models[i];
        CK(cudaStreamWaitEvent(m->stream, b->finished, 0));
        m->sweeps += n;
        m->launches += n * (4 + 2 * (long long)b->groups.size());   // re-binning, sweep end; plan + phase per group
    }
    return CMH_OK;
}

extern "C" int cmh_batch_sync(cmh_batch* b) {
    if (!b) return CMH_ERR_ARG;
    CK(cudaStreamSynchronize(b->stream));
    int rc = CMH_OK;
    for (int i = 0; i < b->n; ++i) {
        const int st = check_status(b->models[i]);
        if (st && rc == CMH_OK) rc = st;
    }
    return rc;
}

extern "C" int cmh_batch_groups(const cmh_batch* b, int32_t* n_groups, int32_t* models_per_group,
                                int32_t* grid_per_group, int32_t cap) {
    if (!b || !n_groups || cap < 0) return CMH_ERR_ARG;
    *n_groups = (int32_t)b->groups.size();
    for (int i = 0; i < (int)b->groups.size() && i < cap; ++i) {
        if (models_per_group) models_per_group[i] = b->groups[i].n;
        if (grid_per_group) grid_per_group[i] = b->groups[i].grid;
    }
    return CMH_OK;
}

extern "C" void cmh_batch_destroy(cmh_batch* b) {
    if (!b) return;
    b->release();
    delete b;
}
