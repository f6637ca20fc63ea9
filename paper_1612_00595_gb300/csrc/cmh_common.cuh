// Internal definitions shared by the chromh CUDA translation units.
//
// Precision policy:
//  * event coordinates, the partition and every proposal are float64 and use
//    explicitly rounded intrinsics (__dadd_rn, __dmul_rn, __ddiv_rn,
//    __dsqrt_rn) where a result decides an integer (a cell, a window start)
//    or a coordinate, so no fused multiply-add changes them;
//  * per-sample likelihood terms are float64 (replay mode) or float32 with
//    compensated sums (throughput mode);
//  * the log acceptance ratio and the running log-density are float64.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "chromh.h"

namespace cmh {

constexpr int kMaxColours = 16;
constexpr int kMaxK = 4095;
constexpr unsigned kDepWaitLimitDefault = 1u << 22;   // polls of a neighbour's done stamp (~0.5 s)
// proposed[3], evaluated[3], accepted[3], priced samples, rewritten samples,
// joint moves of a pair: proposed, evaluated, accepted; arrival-time moves:
// proposed, evaluated, accepted; unique window samples (float32 form, while
// count_unique is set)
constexpr int kStats = 18;

// model, partition and launch constants; passed by value to every kernel
struct Geo {
    double W, T, Lambda, v, alpha, beta_att, tau, noise_var, f_hz, R_max, L;
    double p_birth, p_death, sig_xy, sig_t, sig_m;
    double p_pair;      // joint move of a pair of events (float64 form only)
    // latent arrival times (float64 form only): offsets ~ N(0, sig_a^2) per
    // (event, reached station) when sig_a > 0; the arrival-time move's share
    // and step
    double sig_a, p_arr, sig_da;
    // logs computed once on the host
    double log_pb, log_pd, log_Lambda, log_WWT, log_T;
    int n_w, k, commit, shift_mode;
    double sx_static, sy_static;
    int ncx, ncy, n_cells, period, n_colours, max_rpc;
    int n_st;
    long long n_samp, pitch;
    unsigned long long seed;
    int ev_cap, blk_cap, frz_cap, arr_cap;
    int stage_cap;      // floats per shared-memory staging buffer of the float32 phase (0: none)
    int task_cap;       // stations one float32 step may touch (old and new arrivals)
    // float32 regions too large for shared memory: their event arrival caches
    // and station arrival lists live in a global scratch slot per CTA
    int spill;
    long long spill_bytes;   // bytes of one slot
    long long store_cap, max_events;
    int f32;
    int threads;
    int count_unique;   // float32 form: count the union of each region phase's priced windows (stats[17])
    // float32 persistent sweep: polls a region makes of each lower-colour
    // neighbour's done stamp before it gives up (CMH_ERR_TIMEOUT); and a test
    // hook: the region of cell hold_cell (-1: none) runs its phase but never
    // announces it, so that its neighbours' bounded waits run out
    unsigned dep_wait_limit;
    int hold_cell;
    // float32 form of the model constants (host-computed)
    float invL_f;      // 1 / L
    float fv_f;        // f / v
    // likelihood reading: 0 = arrivals add (A g)^2 to the variance of a
    // zero-mean sample (V buffer = variance), 1 = they add A g to its mean
    // (V buffer = mean; the variance is the noise's).  p = 2 or 1 is the power
    // of the envelope that an arrival contributes.
    int mean_mode;
    float apow_f;      // p
    float syn0_f;      // the predicted quantity without arrivals: noise variance, or 0
    float inv_noise_f; // 1 / noise variance (mean reading)
    float twoftau_f;   // p / (f tau)
    float kap_f;       // p log2(e) / (f tau): per-sample decay of log2 of a contribution
    float rho_f[4];    // 2^(-kap e), e = 0..3 (rho_f[0] = 1)
    float alpha_f, beta_f, R_f, noise_f, f_f, tau_f, v_f;
    double Tf;         // T f
    int TfK;           // floor(T f)
    double lb0;        // log Lambda - log(W^2 T) + 2: log beta(m) = lb0 - m
    double Cb0;        // log Lambda - log(W^2 T) + log T + log p_d - log p_b (+ log area per region)
    double lLWT;       // log Lambda - log(W^2 T)
    double lpdpb;      // log p_d - log p_b
    // learned birth component (bt_on == 0: uniform births only): weights over
    // bt_nx x bt_ny pixels of [0,W)^2 and bt_nt time bins of [0,T)
    int bt_on, bt_nx, bt_ny, bt_nt;
    double bt_mix, bt_hx, bt_hy, bt_dt, bt_pixarea;
    double bt_ihx, bt_ihy, bt_idt;   // 1 / bt_hx, 1 / bt_hy, 1 / bt_dt
    // learned magnitudes (bt_mag_on == 0: table births draw m from the prior):
    // a table birth at an entry draws m uniform on [lo, lo + 2h), lo = max(2, centre - h)
    int bt_mag_on;
    double bt_h, bt_h2, bt_ih2;      // h, 2h, 1 / (2h)
};

// one event store (structure of arrays) with per-cell slices
struct Store {
    double *x, *y, *t, *m;
    unsigned long long* id;
    int *start, *count, *cap;   // [n_cells]
    int* total;                 // number of events
    double* off;                // latent arrival offsets [store_cap][n_st] (nullptr without them)
};

struct Dev {
    Store st[2];                // sweep s works on st[s & 1]
    long long* sweep;           // device sweep counter
    double* shift;              // [2] current (sx, sy)
    int* colour_count;          // [n_colours]
    int* colour_cells;          // [n_colours][max_rpc]
    int* fill;                  // [n_cells] events counted into each new cell (cleared by the scan)
    int* ncell;                 // [store_cap] new cell of the event at each position of the old store
    int* cell_col;              // [n_cells] colour of each live cell of the current sweep, -1 if not live
    int* colour_off;            // [n_colours + 1] first queue item of each colour (persistent sweep)
    int* queue;                 // next queue item (persistent sweep)
    long long* done;            // [n_cells] last sweep + 1 whose phase the cell's region has finished
    int* flat_off;              // [n_cells + 1] first flat-list position of each cell (flattening scratch)
    const int* bl_off;          // [n_cells + 1] blanket candidates of each cell: the stations that may lie
    const int* bl_idx;          //   within R_max of its region under any shift, in station order
    double* region_dlp;         // [n_cells] log-density change of the current sweep
    double* logp;               // running log-density
    int* status;                // latched CMH_ERR_* (0 = fine)
    unsigned long long* stats;  // [kStats]
    cmh_trace* trace;
    long long trace_cap, trace_sweep0;
    const void* sig;            // [n_st][pitch] float or double
    void* V;                    // [n_st][pitch] predicted variance
    const double* stx;
    const double* sty;
    const float* stxf;          // float copies of the station coordinates
    const float* styf;
    const double* log_n;        // [ev_cap + 2] log(n) table, computed on the host
    unsigned char* spill_buf;   // [CTA slots][spill_bytes] (float32 regions with spill)
    const double* bt_mass;      // [pixel] table mass of each pixel (learned birth component)
    const double* bt_cdf;       // [pixel][bin] running sum of the pixel's weights / its mass
    const float* bt_tab;        // [pixel][bin] the table's weights as given
    const float* bt_mag;        // [pixel][bin] centre of the learned magnitude window
};

// --------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11): ten rounds of two 64x64->128-bit
// products with the multipliers below, xor with the odd words and the key,
// key bumped by the Weyl increments.
// --------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64(unsigned long long c[4], unsigned long long k0,
                                           unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

// uniform doubles from the top 53 bits: [0,1) and (0,1]
__device__ __forceinline__ double u01(unsigned long long w) {
    return __dmul_rn((double)(w >> 11), 1.0 / 9007199254740992.0);
}
__device__ __forceinline__ double u01o(unsigned long long w) {
    return __dmul_rn((double)((w >> 11) + 1ULL), 1.0 / 9007199254740992.0);
}
// uniform integer in [0, n) from the low 32 bits
__device__ __forceinline__ int pick32(unsigned long long w, int n) {
    return (int)(((w & 0xffffffffULL) * (unsigned long long)n) >> 32);
}

// cell index along one axis: floor((x - s) / L) + 1
__device__ __forceinline__ int cell_axis(double x, double s, double L) {
    return (int)floor(__ddiv_rn(__dsub_rn(x, s), L)) + 1;
}

__device__ __forceinline__ int cell_of(const Geo& g, double sx, double sy, double x, double y) {
    int ix = cell_axis(x, sx, g.L), iy = cell_axis(y, sy, g.L);
    if (ix < 0 || ix >= g.ncx || iy < 0 || iy >= g.ncy) return -1;
    return iy * g.ncx + ix;
}

// [x0, x1) x [y0, y1) of a cell, clipped to the domain
__device__ __forceinline__ void cell_rect(const Geo& g, double sx, double sy, int cell, double r[4]) {
    int ix = cell % g.ncx, iy = cell / g.ncx;
    double x0 = __dadd_rn(sx, __dmul_rn((double)(ix - 1), g.L));
    double x1 = __dadd_rn(sx, __dmul_rn((double)ix, g.L));
    double y0 = __dadd_rn(sy, __dmul_rn((double)(iy - 1), g.L));
    double y1 = __dadd_rn(sy, __dmul_rn((double)iy, g.L));
    r[0] = x0 < 0.0 ? 0.0 : x0;
    r[1] = x1 > g.W ? g.W : x1;
    r[2] = y0 < 0.0 ? 0.0 : y0;
    r[3] = y1 > g.W ? g.W : y1;
}

__device__ __forceinline__ double dist_rn(double x, double y, double xs, double ys) {
    double dx = __dsub_rn(x, xs), dy = __dsub_rn(y, ys);
    return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// the shift of one sweep: Philox stream 1 at counter (sweep, 0, 0, 0)
__device__ __forceinline__ void sweep_shift(const Geo& g, long long sweep, double* sx, double* sy) {
    if (g.shift_mode == 1) {
        unsigned long long c[4] = {(unsigned long long)sweep, 0ULL, 0ULL, 0ULL};
        philox4x64(c, g.seed, 1ULL);
        *sx = __dmul_rn(u01(c[0]), g.L);
        *sy = __dmul_rn(u01(c[1]), g.L);
    } else {
        *sx = g.sx_static;
        *sy = g.sy_static;
    }
}

__device__ __forceinline__ void latch(int* status, int code) { atomicCAS(status, 0, code); }

// --------------------------------------------------------------------------
// float32 form of an arrival, shared by every kernel that builds or changes
// the float32 variance buffer, so that the variance an event adds at a station
// is the same bit pattern wherever it is computed (a pure function of the
// event's float64 master and the station).  Every float operation is
// explicitly rounded (no contraction differences between translation units).
// The reach test and the window start have margins ~10x their worst-case
// float32 error and fall back to the exact float64 expressions inside them,
// so both integer decisions equal the float64 definition's.
// --------------------------------------------------------------------------
constexpr float kMarginR = 2e-3f;   // km
constexpr float kMarginK = 2e-3f;   // samples

// the exact float64 decisions, out of line: they run only inside the margins
static __device__ __noinline__ bool reach_exact(double x, double y, double xs, double ys, double R) {
    return dist_rn(x, y, xs, ys) < R;
}
static __device__ __noinline__ int k0_exact(double x, double y, double t, double xs, double ys, double v, double f) {
    const double a = __dadd_rn(t, __ddiv_rn(dist_rn(x, y, xs, ys), v));
    return (int)ceil(__dmul_rn(a, f));
}
// the same with a latent arrival offset dl (s): ceil(((t + d / v) + dl) f)
static __device__ __noinline__ int k0_exact_lat(double x, double y, double t, double xs, double ys, double v,
                                                double f, double dl) {
    const double a = __dadd_rn(__dadd_rn(t, __ddiv_rn(dist_rn(x, y, xs, ys), v)), dl);
    return (int)ceil(__dmul_rn(a, f));
}

// per-event float32 terms: K = floor(t f), ph = t f - K, mf = m
__device__ __forceinline__ void event_terms32(const Geo& g, double t, double m, int& K, float& ph, float& mf) {
    const double tf = __dmul_rn(t, g.f_hz);
    const double fk = floor(tf);
    K = (int)fk;
    ph = (float)__dsub_rn(tf, fk);
    mf = (float)m;
}

// float32 distance of an event from a station
__device__ __forceinline__ float dist32(double x, double y, double xs, double ys) {
    const float dx = (float)__dsub_rn(x, xs), dy = (float)__dsub_rn(y, ys);
    return __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
}

// reach of a station: d < R_max, d the float32 distance returned in dist
__device__ __forceinline__ bool reach32(const Geo& g, double x, double y, double xs, double ys, float& dist) {
    const float d = dist32(x, y, xs, ys);
    dist = d;
    if (d < g.R_f - kMarginR) return true;
    if (d > g.R_f + kMarginR) return false;
    return reach_exact(x, y, xs, ys, g.R_max);
}

// first sample k0 and E0 = log2 of the variance added at k0 of an arrival at
// float32 distance d; dl is the latent arrival offset (s), 0 without latent
// arrivals (a constant 0 compiles the offset away).  The offset enters in
// float32 as dl f samples; within the margin the exact float64 start decides.
__device__ __forceinline__ void window32(const Geo& g, double x, double y, double t, int K, float ph, float mf,
                                         double xs, double ys, float d, double dl, int& k0, float& E0) {
    float q = __fadd_rn(ph, __fmul_rn(d, g.fv_f));   // arrival x f - K
    if (dl != 0.0) q = __fadd_rn(q, (float)__dmul_rn(dl, g.f_hz));
    if (fabsf(__fsub_rn(q, rintf(q))) < kMarginK)
        k0 = dl != 0.0 ? k0_exact_lat(x, y, t, xs, ys, g.v, g.f_hz, dl) : k0_exact(x, y, t, xs, ys, g.v, g.f_hz);
    else
        k0 = K + (int)ceilf(q);
    const float lnA2 = __fmul_rn(g.apow_f, __fsub_rn(__fmul_rn(g.alpha_f, mf), __fmul_rn(g.beta_f, d)));
    const float frac = __fsub_rn((float)(k0 - K), q);      // k0 - arrival x f, in [0, 1)
    E0 = __fmul_rn(1.4426950408889634f, __fsub_rn(lnA2, __fmul_rn(frac, g.twoftau_f)));
}

// reach, first sample k0 and E0 = log2 of the variance added at k0
__device__ __forceinline__ bool arrival32c(const Geo& g, double x, double y, double t, int K, float ph, float mf,
                                           double xs, double ys, int& k0, float& E0, double dl = 0.0) {
    float d;
    if (!reach32(g, x, y, xs, ys, d)) return false;
    window32(g, x, y, t, K, ph, mf, xs, ys, d, dl, k0, E0);
    return true;
}

// latent offset drawn from its prior N(0, sig_a^2) for station j and the
// step's e-th changed event: Philox stream 0 at counter (sweep, cell, step,
// 16 + 2 j + e), a Box-Muller cosine from words 0 and 1 rounded to 2^-20
// (as the walk offsets), the sign from bit 0 of word 2
static __device__ __noinline__ double draw_offset(const Geo& g, long long sweep, int cell, int step, int j, int e) {
    unsigned long long c[4] = {(unsigned long long)sweep, (unsigned long long)cell, (unsigned long long)step,
                               16ULL + 2ULL * (unsigned long long)j + (unsigned long long)e};
    philox4x64(c, g.seed, 0ULL);
    const double r = __dsqrt_rn(__dmul_rn(-2.0, log(u01o(c[0]))));
    const double th = __dmul_rn(6.283185307179586, u01(c[1]));
    double z = __dmul_rn(rint(__dmul_rn(fabs(__dmul_rn(r, cos(th))), 1048576.0)), 1.0 / 1048576.0);
    if (c[2] & 1ULL) z = -z;
    return __dmul_rn(g.sig_a, z);
}

// log N(v; 0, sig_a^2)
__device__ __forceinline__ double log_off_prior1(const Geo& g, double v) {
    const double s2 = __dmul_rn(g.sig_a, g.sig_a);
    return __dsub_rn(__dmul_rn(-0.5, log(__dmul_rn(2.0 * M_PI, s2))), __ddiv_rn(__dmul_rn(v, v), __dmul_rn(2.0, s2)));
}

// 2^x by the SFU (relative error ~2^-22); inline PTX so that every kernel
// evaluates the same instruction
__device__ __forceinline__ float ex2_sfu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// float32 variance an arrival (window start k0, E0 = log2 of the variance at
// k0) adds at sample k, for k in its window.  Samples are grouped in fours
// (k4 = k & ~3): the SFU evaluates the group's base 2^(E0 - kap (k4 - k0))
// and the sample multiplies it by rho[k - k4] = 2^(-kap (k - k4)), constants
// computed once on the host.  Every kernel evaluates exactly this, so a
// group's four values can be produced from one SFU result.
__device__ __forceinline__ float arr_base32(const Geo& g, float E0, int k0, int k4) {
    return ex2_sfu(__fsub_rn(E0, __fmul_rn(g.kap_f, (float)(k4 - k0))));
}
__device__ __forceinline__ float arr_var32(const Geo& g, float E0, int k0, int k) {
    return __fmul_rn(arr_base32(g, E0, k0, k & ~3), g.rho_f[k & 3]);
}

// log(1 + x) for x >= -1/2: the Taylor series x - x^2/2 + ... + x^7/7 for
// |x| < 1/16 (truncation < 3e-11 relative), else the SFU log of 1 + x
// (1 + x is within 1.2e-7 relative when x >= -1/2)
__device__ __forceinline__ float log1p_fast(float x) {
    if (fabsf(x) < 0.0625f) {
        float p = 1.f / 7.f;
        p = fmaf(p, x, -1.f / 6.f);
        p = fmaf(p, x, 1.f / 5.f);
        p = fmaf(p, x, -1.f / 4.f);
        p = fmaf(p, x, 1.f / 3.f);
        p = fmaf(p, x, -0.5f);
        p = fmaf(p, x, 1.f);
        return p * x;
    }
    return __logf(1.f + x);
}

// a flat event list in device memory (canonical order)
struct FlatList {
    double *x, *y, *t, *m;
    unsigned long long* id;
    int* n;
    double* off;                // [cap][n_st] latent arrival offsets, or nullptr (not copied)
};

// host-side launchers (defined in the .cu files)
// a model's geometry and device buffers (for the learned-proposal code)
Geo cmh_model_geo(const cmh_model* m);
Dev cmh_model_dev(const cmh_model* m);

// raise a kernel's dynamic shared-memory limit to at least `bytes`, never
// lowering it (the attribute is shared by every model of the process)
cudaError_t raise_smem_limit(const void* func, size_t bytes);
cudaError_t launch_rebin(const Geo& g, const Dev& d, int init_n, cudaStream_t s, int* launches);
// a batch of independent instances (device arrays of their Geo and Dev)
int rebin_blocks(const Geo& g);
cudaError_t prepare_rebin_batch(int max_ev_cap);
cudaError_t launch_rebin_batch(const Geo* G, const Dev* D, const int* blk_off, int n_inst, int n_blocks,
                               int max_ev_cap, cudaStream_t s);
cudaError_t prepare_sweep32_batch(size_t smem_bytes, int* grid);
cudaError_t launch_sweep32_batch(bool mean, const Geo* G, const Dev* D, int n_inst, int n_col, int* item_tab, int* queue,
                                 size_t smem_bytes, int grid, cudaStream_t s);
cudaError_t launch_sweep_end_batch(const Geo* G, const Dev* D, int n_inst, cudaStream_t s);
cudaError_t prepare_rebin(const Geo& g);
cudaError_t launch_phase(const Geo& g, const Dev& d, int colour, cudaStream_t s);
cudaError_t launch_phase32(const Geo& g, const Dev& d, int colour, cudaStream_t s);
size_t phase32_smem_bytes(const Geo& g);
size_t phase32_spill_bytes(const Geo& g);   // bytes of one CTA's global slot if the region spills
cudaError_t prepare_phase32(const Geo& g);
cudaError_t choose_stage_cap(Geo& g, int requested);
cudaError_t sweep32_grid(const Geo& g, int ctas_per_sm, int* grid);
cudaError_t launch_sweep32(const Geo& g, const Dev& d, int grid, cudaStream_t s);
cudaError_t launch_sweep_end(const Geo& g, const Dev& d, cudaStream_t s);
size_t phase_smem_bytes(const Geo& g);
cudaError_t launch_vsynth(const Geo& g, const Dev& d, const FlatList& f, cudaStream_t s, int* launches);
cudaError_t launch_flatten(const Geo& g, const Dev& d, int buf, const FlatList& f, cudaStream_t s, int* launches);
cudaError_t prepare_kernels(const Geo& g);
cudaError_t launch_loglik(const Geo& g, const Dev& d, double* partial, int n_part, cudaStream_t s);
// latent arrival offsets of a flat list: zero the entries of stations an event
// does not reach, and write sum log N(delta; 0, sig_a^2) over the others to *out
cudaError_t launch_offset_prior(const Geo& g, const Dev& d, const FlatList& f, double* out, cudaStream_t s);
cudaError_t launch_convert_signals(const void* src, int src_f32, long long src_pitch, void* dst,
                                   int dst_f32, long long dst_pitch, int n_st, long long n_samp,
                                   int* nonfinite, cudaStream_t s);
cudaError_t launch_philox_test(const unsigned long long* ctr, const unsigned long long* key,
                               unsigned long long* out, long long n, cudaStream_t s);

}  // namespace cmh
