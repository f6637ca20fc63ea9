// Colour-phase kernel, float32 throughput form (Algorithm "Chromatic MH with
// Static Coloring": every region of one colour runs k MH steps in parallel
// with the other regions fixed).  One CTA per region.
//
// Precision.  The state stays float64 (the event masters), but within a
// phase every per-step test runs in float32:
//   * "does the event reach station j" (distance < R_max),
//   * "which sample does its window start at" (ceil(arrival x f)),
//   * "is the moved event still in the region / domain / time range".
// Each float32 test has a margin about 10x its worst-case rounding error; a
// value inside the margin is decided by the exact float64 expression of the
// float64 master coordinates instead (out-of-line functions).  So every
// integer decision is the one the float64 definition gives, while the float64
// pipe (64-cycle dependent latency, 1/64 of the float32 rate on this part) is
// used for little more than the accept decision.  Per-sample likelihood terms
// are float32, summed in groups of four and compensated (Kahan) per thread,
// reduced across threads in float-float (TwoSum) and finished in float64.
//
// Schedule.  Warp 0 manages: while warps 1.. price step i it prepares step
// i+1 (decode, reach, tasks), assuming step i is rejected (the common case),
// then decides step i; after an accepted step it prepares step i+1 again.
// Each blanket station keeps the list of arrivals that cover it (neighbouring
// regions' and the region's own, tagged by owner), updated on every commit,
// so preparing a step never scans the region's events and re-synthesising V
// reads one list.
//
// Staging (optional, the STAGE instantiation).  Having prepared step i+1,
// warp 0 copies its station windows of s and V into shared memory with bulk
// copies (cp.async.bulk, completion counted on an mbarrier; two buffers
// alternate by step parity), and the workers price from shared memory.  After
// an accepted step, V is re-written, fenced for the async proxy, and the next
// step's copies are issued again.  Every mbarrier wait is bounded.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "cmh_common.cuh"

namespace cmh {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float kDr = 2e-3f;   // km: margin of the region tests
constexpr float kDm = 1e-5f;   // magnitude units: margin of the m >= 2 test
constexpr int kThreads32 = 288;
constexpr int kUnroll = 2;     // float4 groups whose loads a pricing thread issues together
constexpr int kFrozen = -2;    // owner tag of an arrival from a neighbouring region
constexpr int kMinBlocks32 = 3;   // resident CTAs per SM the kernel is built for
constexpr int kMaxPix = 256;      // pixels of the learned birth table a region's range may span
static_assert(kThreads32 <= 512, "the decision reduces the worker warps' partials in a four-level tree");
constexpr int kTree0 = kThreads32 > 256 ? 8 : 4;
constexpr unsigned kWaitLimit = 1u << 24;   // bounded mbarrier waits
constexpr int kIv = 8;            // disjoint priced intervals kept per blanket station (unique-sample count)

struct A32 {            // arrival of an own event at a blanket slot (the event's cache)
    int slot, k0;
    float E0;
    int pad;
};

struct SA {             // an entry of a station's arrival list
    int k0;
    float E0;           // log2 of the variance added at sample k0
    int own;            // physical slot of the own event, or kFrozen
    int pad;
};

struct D32 {            // state-independent part of one MH step
    double bx, by, bt, bm, blb;   // birth: float64 candidate and its log beta; move: float64 offsets
                                  // (arrival-time move: bx, the step of the offset)
    double blq;                   // birth: log Lambda - log(W^2 T) - log q_b(candidate) (magnitude factor out)
    float xr, yr, ph, mf;         // birth: relative form; move: offsets dx, dy, dt (s), dm
    float logu;
    unsigned pickw;
    int type, bK, bvalid;
    int exch;           // joint move of a pair: exchange the two locations (else a common offset)
    unsigned pick2;     // joint move of a pair: the second event among the others
};

struct T32 {            // one station whose variance the proposal changes
    int row, slot, lo, hi;
    int has_o, has_n, k0o, k0n;
    float E0o, E0n;
    int skip;           // owner whose arrival leaves the station (-1: none)
    int u0;             // first float4 group of this task in the step's flat range
};

struct T32X {           // joint move of a pair: the second event's arrivals at the task's station
    int pair;           // 0: a one-event task
    int exch;           // the pair exchanges its locations (else a common offset)
    int has_o2, has_n2, k0o2, k0n2, skip2;
    float E0o2, E0n2;
};

struct P32 {            // an event: float64 master, float32 terms, region-relative position
    double x, y, t, m;
    double lq;          // log Lambda - log(W^2 T) - log q_b at the event (birth / death Hastings term)
    float xr, yr, ph, mf;
    int K, pad;
};

// everything a CTA keeps in shared memory: pointers into the dynamic buffer
// and the scalars of the region and of the two step buffers
struct Sm {
    double *mx, *my, *mt, *mm;
    unsigned long long* eid;
    float *exr, *eyr;
    int *enarr, *order, *freel;
    A32* earr;
    double *tabB, *tabD;
    double* elq;        // [ev_cap] lq of each own event (see P32)
    double* pcum;       // [kMaxPix] running table mass over the region's pixel range
    int* pidx;          // [kMaxPix] pixel index of each entry
    int* bsta;
    double *bx, *by;
    int* scnt;          // entries of each station's arrival list
    SA* sarr;           // [blk_cap][scap]
    D32* draws;
    A32* cand;          // [2][arr_cap]
    A32* cand2;         // [2][arr_cap] the second candidate of a joint move
    T32* tasks;         // [2][task_cap]
    T32X* tasksx;       // [2][task_cap] with joint moves (p_pair > 0), else null
    double *nx, *ny, *nt;
    float *nph, *nmf;
    int* nK;
    int* tsoff;         // [2][task_cap] staging offset of each task's window (floats), -1: global
    float* stage_s;     // [2][scap] staged signal windows
    float* stage_v;     // [2][scap] staged variance windows
    int scap;           // floats per staging buffer (0: no staging)
    int2* uiv;          // [blk_cap][kIv] disjoint windows priced at each blanket station this phase
    int* un;            // [blk_cap] intervals held in uiv
    // latent arrival offsets (sig_a > 0), else null: the offset of each entry
    // of an own event's arrival cache, of each candidate arrival, and the
    // store index of each loaded neighbouring event
    double* aoff;       // [ev_cap][arr_cap]
    double* coff;       // [2][arr_cap]
    double* coff2;      // [2][arr_cap] the second candidate of a joint move
    int* nsrc;          // [ev_cap]
    long long sweep;
    unsigned long long bar[2];   // mbarrier of each staging buffer
    int ph[2], on[2];   // parity of its pending completion; copies in flight
    double rect[4], X0, Y0, sx, sy, region_dlp;
    float rl[4];        // region in relative coordinates: x lo, x hi, y lo, y hi
    int cell, n_own, n_free, n_blk, err, acc;
    double lop0, lopi;  // latent offsets: log N(v; 0, sig_a^2) = lop0 - v^2 lopi
    double bt_G;        // table mass inside the region (learned birth component)
    double lq_unif;     // lq of the uniform birth alone: log(Lambda area / W^2)
    double qu;          // density of the uniform birth in space-time: 1 / (area T)
    double qmu;         // (1 - mix) qu: the uniform component's share of the mixture density
    double bt_in;       // 1 / (pixel area x bt_G x bin width): table weight -> q_net
    int bt_np, bt_last; // pixel entries; last entry with mass
    int valid[2], idx[2], type[2], ncand[2], ntask[2], units[2], width[2];
    double thr[2];      // accept iff the log-likelihood change exceeds this (log u minus the other terms of log alpha)
    float thrf[2];      // thr rounded to float32: the decision away from it needs no float64
    double dlp[2];      // log-prior change of the step
    int nb_start[64], nb_cnt[64], nb_off[65];   // neighbouring cells of the region (prologue)
    P32 c[2];           // candidate of each step buffer
    P32 c2[2];          // joint move of a pair: the second candidate
    int idx2[2], ncand2[2];
    int ai[2];          // arrival-time move: the entry of the event's arrival cache it steps
    int warp_cnt[32];
    float2 redf[32];
    // statistics of this CTA: proposed[3], evaluated[3], accepted[3], priced
    // samples, re-synthesised samples, unique window samples, joint moves
    // proposed, evaluated, accepted, arrival-time moves proposed, evaluated,
    // accepted (thread 0)
    unsigned long long cnt[18];
};

// carve the dynamic shared buffer; returns its size (base may be null).  With
// g.spill the event arrival caches and the station arrival lists come from
// the CTA's global slot gbase instead, and *gbytes receives their size.
__host__ __device__ inline size_t layout32(const Geo& g, Sm* S, unsigned char* base, unsigned char* gbase = nullptr,
                                           size_t* gbytes = nullptr) {
    size_t o = 0, go = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += (bytes + 15) & ~size_t(15);
        return base + r;
    };
    auto gtake = [&](size_t bytes) {
        if (!g.spill) return take(bytes);
        size_t r = go;
        go += (bytes + 15) & ~size_t(15);
        return gbase + r;
    };
    const size_t E = g.ev_cap, B = g.blk_cap;
    double *mx = (double*)take(8 * E), *my = (double*)take(8 * E), *mt = (double*)take(8 * E),
           *mm = (double*)take(8 * E);
    unsigned long long* eid = (unsigned long long*)take(8 * E);
    float *exr = (float*)take(4 * E), *eyr = (float*)take(4 * E);
    int *enarr = (int*)take(4 * E), *order = (int*)take(4 * E), *freel = (int*)take(4 * E);
    A32* earr = (A32*)gtake(sizeof(A32) * E * g.arr_cap);
    double *tabB = (double*)take(8 * (E + 1)), *tabD = (double*)take(8 * (E + 1));
    double* elq = (double*)take(8 * E);
    double* pcum = (double*)take(8 * kMaxPix);
    int* pidx = (int*)take(4 * kMaxPix);
    int* bsta = (int*)take(4 * B);
    double *bx = (double*)take(8 * B), *by = (double*)take(8 * B);
    int* scnt = (int*)take(4 * B);
    SA* sarr = (SA*)gtake(sizeof(SA) * B * g.frz_cap);
    D32* draws = (D32*)take(sizeof(D32) * (size_t)g.k);
    A32* cand = (A32*)take(sizeof(A32) * 2 * (size_t)g.arr_cap);
    A32* cand2 = (A32*)take(sizeof(A32) * 2 * (size_t)g.arr_cap);
    T32* tasks = (T32*)take(sizeof(T32) * 2 * (size_t)g.task_cap);
    const bool lat = g.sig_a > 0.0;
    T32X* tasksx = (g.p_pair > 0.0 || lat) ? (T32X*)take(sizeof(T32X) * 2 * (size_t)g.task_cap) : nullptr;
    double *nx = (double*)take(8 * E), *ny = (double*)take(8 * E), *nt = (double*)take(8 * E);
    float *nph = (float*)take(4 * E), *nmf = (float*)take(4 * E);
    int* nK = (int*)take(4 * E);
    int* tsoff = (int*)take(4 * 2 * (size_t)g.task_cap);
    int2* uiv = (int2*)gtake(sizeof(int2) * B * kIv);
    int* un = (int*)gtake(4 * B);
    const size_t scap = (size_t)g.stage_cap;
    float* stage_s = scap ? (float*)take(4 * 2 * scap) : nullptr;
    float* stage_v = scap ? (float*)take(4 * 2 * scap) : nullptr;
    double* aoff = lat ? (double*)gtake(8 * E * g.arr_cap) : nullptr;
    double* coff = lat ? (double*)take(8 * 2 * (size_t)g.arr_cap) : nullptr;
    double* coff2 = lat ? (double*)take(8 * 2 * (size_t)g.arr_cap) : nullptr;
    int* nsrc = lat ? (int*)take(4 * E) : nullptr;
    if (S) {
        S->aoff = aoff;
        S->coff = coff;
        S->coff2 = coff2;
        S->nsrc = nsrc;
        S->uiv = uiv;
        S->un = un;
        S->tsoff = tsoff;
        S->stage_s = stage_s;
        S->stage_v = stage_v;
        S->scap = (int)scap;
        S->mx = mx; S->my = my; S->mt = mt; S->mm = mm; S->eid = eid; S->exr = exr; S->eyr = eyr;
        S->enarr = enarr; S->order = order; S->freel = freel; S->earr = earr;
        S->tabB = tabB; S->tabD = tabD; S->elq = elq; S->pcum = pcum; S->pidx = pidx; S->bsta = bsta; S->bx = bx; S->by = by;
        S->scnt = scnt; S->sarr = sarr; S->draws = draws; S->cand = cand; S->cand2 = cand2; S->tasks = tasks; S->tasksx = tasksx;
        S->nx = nx; S->ny = ny; S->nt = nt; S->nph = nph; S->nmf = nmf; S->nK = nK;
    }
    if (gbytes) *gbytes = go;
    return o;
}

__device__ __forceinline__ void kahan_add32(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__device__ __forceinline__ float2 ff_add32(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb);
    const float lo = a.y + b.y + e;
    const float hi = s + lo;
    return make_float2(hi, lo - (hi - s));
}

// 1/x by the SFU (relative error ~1 ulp)
__device__ __forceinline__ float rcp_sfu(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- bulk copies and mbarriers (inline PTX) ---------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// one arrival that also announces `bytes` of transactions to come
__device__ __forceinline__ void mbar_arm(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the phase with this parity to complete, at most kWaitLimit tries
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (unsigned i = 0; i < kWaitLimit; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// global -> shared bulk copy (both addresses 16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// uniform in (0, 1] from the top 32 bits, as a float (relative precision
// 2^-24 even for small values, so its log is accurate to ~6e-8)
__device__ __forceinline__ float u32o(unsigned long long w) {
    return (float)((w >> 32) + 1ULL) * (1.0f / 4294967296.0f);
}

// 2 - log(u), u = ((w >> 11) + 1) 2^-53 in (0, 1]: the magnitude of a birth
// (m - 2 ~ Exp(1)).  u = mant 2^(e-53) with mant in [1, 2): the exponent part
// is exact, log2(mant) is float32 (absolute error ~1e-7).
__device__ __forceinline__ double mag_from_u53(unsigned long long w) {
    const unsigned long long v = (w >> 11) + 1ULL;   // 1 .. 2^53
    const int e = 63 - __clzll((long long)v);        // v in [2^e, 2^(e+1))
    const unsigned m24 = e >= 23 ? (unsigned)(v >> (e - 23)) : (unsigned)(v << (23 - e));
    const float lm = log2f((float)m24 * (1.0f / 8388608.0f));
    return 2.0 + 0.69314718055994530942 * (double)(53 - e) - (double)(0.69314718f * lm);
}

// region-relative position and float32 terms of a float64 event
__device__ __forceinline__ void to_rel(const Geo& g, double X0, double Y0, P32& e) {
    e.xr = (float)__dsub_rn(e.x, X0);
    e.yr = (float)__dsub_rn(e.y, Y0);
    event_terms32(g, e.t, e.m, e.K, e.ph, e.mf);
}

// the exact float64 region / range test of a candidate (the oracle's)
__device__ __noinline__ bool inside_exact(const Geo& g, double sx, double sy, int cell, double x, double y, double t,
                                          double m) {
    return x >= 0.0 && x < g.W && y >= 0.0 && y < g.W && cell_of(g, sx, sy, x, y) == cell && t >= 0.0 && t < g.T &&
           m >= 2.0;
}

// ---- learned birth component (float64, explicitly rounded: the same values
// as the oracle's plain float64 C) -------------------------------------------
// pixel range that may overlap [r0, r1) along one axis (one pixel of margin)
__device__ __forceinline__ void bt_range(double r0, double r1, double h, int n, int& i0, int& i1) {
    const int a = (int)__ddiv_rn(r0, h) - 1, b = (int)__ddiv_rn(r1, h) + 1;
    i0 = a < 0 ? 0 : a;
    i1 = b > n - 1 ? n - 1 : b;
}

__device__ __forceinline__ double bt_overlap(double r0, double r1, double h, int i) {
    const double p0 = __dmul_rn((double)i, h), p1 = __dmul_rn((double)(i + 1), h);
    const double lo = p0 > r0 ? p0 : r0, hi = p1 < r1 ? p1 : r1;
    return hi > lo ? __dsub_rn(hi, lo) : 0.0;
}

// table mass of pixel (ix, iy) inside the region rect r
__device__ __forceinline__ double bt_weight(const Geo& g, const Dev& d, const double* r, int ix, int iy) {
    const double ox = bt_overlap(r[0], r[1], g.bt_hx, ix), oy = bt_overlap(r[2], r[3], g.bt_hy, iy);
    return __dmul_rn(d.bt_mass[(long long)iy * g.bt_nx + ix], __ddiv_rn(__dmul_rn(ox, oy), g.bt_pixarea));
}

// lq at (x, y, t): log Lambda - log(W^2 T) - log[(1 - mix) / (area T) + mix q_net],
// q_net = table weight of (pixel, bin) / (pixel area x region mass x bin
// width).  A density term of the float32 path: the pixel and bin come from
// reciprocal products, the weight is the table's own float and the logarithm
// is taken in float32 (error ~1e-7 against the float64 form); the sum into
// log alpha stays float64.  The sampling itself (learned_birth) is exact.
__device__ __noinline__ double bt_lq(const Geo& g, const Dev& d, const Sm& S, double x, double y, double t,
                                     double m) {
    double qn = 0.0;
    if (S.bt_G > 0.0) {
        int ix = (int)(x * g.bt_ihx), iy = (int)(y * g.bt_ihy), b = (int)(t * g.bt_idt);
        ix = ix < 0 ? 0 : (ix > g.bt_nx - 1 ? g.bt_nx - 1 : ix);
        iy = iy < 0 ? 0 : (iy > g.bt_ny - 1 ? g.bt_ny - 1 : iy);
        b = b < 0 ? 0 : (b > g.bt_nt - 1 ? g.bt_nt - 1 : b);
        const long long q = ((long long)iy * g.bt_nx + ix) * g.bt_nt + b;
        qn = (double)__ldg(d.bt_tab + q) * S.bt_in;
        if (g.bt_mag_on) {
            // the learned component draws m on its entry's window: q_win(m) / p(m)
            const double lo = fmax(2.0, __dsub_rn((double)__ldg(d.bt_mag + q), g.bt_h));
            qn = (m >= lo && m < __dadd_rn(lo, g.bt_h2)) ? qn * g.bt_ih2 * (double)expf((float)(m - 2.0)) : 0.0;
        }
    }
    return g.lLWT - (double)logf((float)(S.qmu + g.bt_mix * qn));
}

// a birth from the learned component: pixel by its share of the region's
// table mass (word w_pix), position uniform in pixel and region (w_x and the
// third Philox block of the step), time bin by the pixel's cdf, time uniform
// in the bin, and with learned magnitudes m uniform on the drawn entry's
// window (word 3 of the third block); returns whether it drew m
__device__ __noinline__ bool learned_birth(const Geo& g, const Dev& d, const Sm& S, long long sweep, int cell,
                                           int st, unsigned long long w_pix, unsigned long long w_x, P32& e) {
    unsigned long long c2[4] = {(unsigned long long)sweep, (unsigned long long)cell, (unsigned long long)st, 2ULL};
    philox4x64(c2, g.seed, 0ULL);
    const double target = __dmul_rn(u01(w_pix), S.bt_G);
    int lo = 0, hi = S.bt_np - 1;   // first entry whose running mass exceeds target
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (S.pcum[mid] > target) hi = mid; else lo = mid + 1;
    }
    const int j = S.pcum[lo] > target ? lo : S.bt_last;
    const int px = S.pidx[j] % g.bt_nx, py = S.pidx[j] / g.bt_nx;
    const double xa = __dmul_rn((double)px, g.bt_hx), xb = __dmul_rn((double)(px + 1), g.bt_hx);
    const double ya = __dmul_rn((double)py, g.bt_hy), yb = __dmul_rn((double)(py + 1), g.bt_hy);
    const double lx = xa > S.rect[0] ? xa : S.rect[0], hx = xb < S.rect[1] ? xb : S.rect[1];
    const double ly = ya > S.rect[2] ? ya : S.rect[2], hy = yb < S.rect[3] ? yb : S.rect[3];
    e.x = __dadd_rn(lx, __dmul_rn(u01(w_x), __dsub_rn(hx, lx)));
    e.y = __dadd_rn(ly, __dmul_rn(u01(c2[0]), __dsub_rn(hy, ly)));
    const double* cd = d.bt_cdf + (long long)S.pidx[j] * g.bt_nt;
    const double ub = u01(c2[1]);
    int b0 = 0, b1 = g.bt_nt - 1;   // first bin whose cdf exceeds ub (the last one otherwise)
    while (b0 < b1) {
        const int mid = (b0 + b1) >> 1;
        if (cd[mid] > ub) b1 = mid; else b0 = mid + 1;
    }
    e.t = __dadd_rn(__dmul_rn((double)b0, g.bt_dt), __dmul_rn(u01(c2[2]), g.bt_dt));
    if (!g.bt_mag_on) return false;
    const double mlo = fmax(2.0, __dsub_rn((double)d.bt_mag[(long long)S.pidx[j] * g.bt_nt + b0], g.bt_h));
    e.m = __dadd_rn(mlo, __dmul_rn(u01(c2[3]), g.bt_h2));
    return true;
}

// a candidate event at (x, y, t, m) (float64 master; xr, yr its position
// relative to the region's cell origin in float32): its float32 terms, and
// whether it lies in the region, the domain, [0, T) and m >= 2 -- decided in
// float32 away from the edges, by the exact float64 test within kDr / kDm
__device__ __forceinline__ int cand_of(const Geo& g, const Sm& S, double x, double y, double t, double m, float xr,
                                       float yr, P32& c) {
    c.x = x; c.y = y; c.t = t; c.m = m;
    event_terms32(g, c.t, c.m, c.K, c.ph, c.mf);
    c.xr = xr;
    c.yr = yr;
    const bool xin = c.xr >= S.rl[0] + kDr && c.xr < S.rl[1] - kDr;
    const bool yin = c.yr >= S.rl[2] + kDr && c.yr < S.rl[3] - kDr;
    const bool xout = c.xr < S.rl[0] - kDr || c.xr >= S.rl[1] + kDr;
    const bool yout = c.yr < S.rl[2] - kDr || c.yr >= S.rl[3] + kDr;
    const bool tin = c.K >= 1 && c.K + 2 <= g.TfK;
    const bool min_ = c.mf >= 2.f + kDm;
    const bool mout = c.mf < 2.f - kDm;
    if (xout || yout || mout) return 0;
    if (xin && yin && tin && min_) return 1;
    const int v = inside_exact(g, S.sx, S.sy, S.cell, c.x, c.y, c.t, c.m);
    if (v) to_rel(g, S.X0, S.Y0, c);
    return v;
}

// candidate arrivals of event e (lanes of warp 0 over blanket slots),
// compacted in slot order into out; with latent arrivals each one's offset
// goes to oo: kept from the event old_ps it replaces where that one reached
// the station (its arrival cache, slot-sorted, is searched), else drawn from
// the prior with the counter of step `step` and changed event `which`
template <bool LAT>
__device__ __forceinline__ int cand_arrivals(const Geo& g, const Sm& S, int step, const P32& e, int which,
                                             int old_ps, A32* out, double* oo) {
    const int lane = threadIdx.x & 31, n_blk = S.n_blk;
    int n = 0;
    for (int b0 = 0; b0 < n_blk; b0 += 32) {
        const int b = b0 + lane;
        int k0 = 0;
        float E0 = 0.f, dd = 0.f;
        double dl = 0.0;
        const bool r = b < n_blk && reach32(g, e.x, e.y, S.bx[b], S.by[b], dd);
        if (r) {
            if (LAT) {
                bool kept = false;
                if (old_ps >= 0) {
                    const A32* L = S.earr + old_ps * g.arr_cap;
                    int lo = 0, hi = S.enarr[old_ps];
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (L[mid].slot < b) lo = mid + 1; else hi = mid;
                    }
                    if (lo < S.enarr[old_ps] && L[lo].slot == b) {
                        dl = S.aoff[old_ps * g.arr_cap + lo];
                        kept = true;
                    }
                }
                if (!kept) dl = draw_offset(g, S.sweep, S.cell, step, S.bsta[b], which);
            }
            window32(g, e.x, e.y, e.t, e.K, e.ph, e.mf, S.bx[b], S.by[b], dd, dl, k0, E0);
        }
        const unsigned bal = __ballot_sync(FULL, r);
        const int pos = n + __popc(bal & ((1u << lane) - 1));
        if (r && pos < g.arr_cap) {
            out[pos] = A32{b, k0, E0, 0};
            if (LAT) oo[pos] = dl;
        }
        n += __popc(bal);
    }
    return n;
}

__device__ __forceinline__ void clear_p32(P32& c) {
    c.x = c.y = c.t = c.m = 0.0;
    c.xr = c.yr = c.ph = c.mf = 0.f;
    c.K = 0;
    c.pad = 0;
    c.lq = 0.0;
}

// ---------------------------------------------------------------------------
// preparation of one step (all lanes of warp 0): decode the proposal against
// the current state, find the stations the candidate reaches, and merge the
// old and new arrivals into tasks (one per station whose variance changes)
// in step buffer sl; with STAGE, start the bulk copies of the task windows.
// A joint move of a pair is prepared by prepare_pair (its own function, so
// that its registers do not weigh on the steps of one event).
// ---------------------------------------------------------------------------
template <bool STAGE, bool LAT>
__device__ __noinline__ void prepare_step(const Geo& g, const Dev& d, Sm& S, int step, int sl) {
    const int lane = threadIdx.x & 31;
    if (STAGE) {
        // copies of an earlier preparation of this buffer may still be in
        // flight: let them land before the buffer is reused
        if (lane == 0 && S.on[sl]) {
            if (!mbar_wait(&S.bar[sl], (unsigned)S.ph[sl])) S.err = CMH_ERR_TIMEOUT;
            S.ph[sl] ^= 1;
            S.on[sl] = 0;
        }
        __syncwarp();
    }
    const D32& dr = S.draws[step];
    const int n_own = S.n_own;
    A32* cd = S.cand + sl * g.arr_cap;
    T32* tk = S.tasks + sl * g.task_cap;
    int valid = 0, idx = -1, ps = -1;
    P32 c;
    clear_p32(c);
    if (dr.type == 0) {
        valid = dr.bvalid;
        c.x = dr.bx; c.y = dr.by; c.t = dr.bt; c.m = dr.bm;
        c.xr = dr.xr; c.yr = dr.yr; c.ph = dr.ph; c.mf = dr.mf; c.K = dr.bK;
        c.lq = dr.blq;
    } else if (n_own > 0) {
        idx = pick32(dr.pickw, n_own);
        ps = S.order[idx];
        if (dr.type == 1) {
            valid = 1;
        } else {
            // the float64 state the move proposes (the float64 offsets of the
            // draw), its float32 terms and region-relative position
            valid = cand_of(g, S, __dadd_rn(S.mx[ps], dr.bx), __dadd_rn(S.my[ps], dr.by),
                            __dadd_rn(S.mt[ps], dr.bt), __dadd_rn(S.mm[ps], dr.bm), S.exr[ps] + dr.xr,
                            S.eyr[ps] + dr.yr, c);
        }
    }
    int ncand = 0;
    double* co = LAT ? S.coff + sl * g.arr_cap : nullptr;
    if (valid && dr.type != 1) {
        ncand = cand_arrivals<LAT>(g, S, step, c, 0, dr.type == 0 ? -1 : ps, cd, co);
    }
    __syncwarp();
    if (lane == 0) {
        int err = ncand > g.arr_cap ? CMH_ERR_CAPACITY : 0;
        int ntask = 0, units = 0, width = 0;
        if (valid && !err) {
            // merge the old event's arrivals and the candidate's, by slot
            const A32* oa = (ps >= 0 && dr.type != 0) ? S.earr + ps * g.arr_cap : nullptr;
            const int no = oa ? S.enarr[ps] : 0;
            const int nnw = dr.type != 1 ? ncand : 0;
            int io = 0, in = 0;
            while (io < no || in < nnw) {
                const int so = io < no ? oa[io].slot : 1 << 30;
                const int sn = in < nnw ? cd[in].slot : 1 << 30;
                if (ntask >= g.task_cap) {
                    err = CMH_ERR_CAPACITY;
                    break;
                }
                T32 T;
                T.slot = so < sn ? so : sn;
                T.row = S.bsta[T.slot];
                T.has_o = so <= sn;
                T.has_n = sn <= so;
                T.k0o = T.k0n = 0;
                T.E0o = T.E0n = 0.f;
                T.skip = dr.type == 0 ? -1 : ps;
                int lo = 1 << 30, hi = -1;
                if (T.has_o) {
                    const A32 A = oa[io++];
                    T.k0o = A.k0; T.E0o = A.E0;
                    lo = min(lo, A.k0);
                    hi = max(hi, A.k0 + g.n_w);
                }
                if (T.has_n) {
                    const A32 A = cd[in++];
                    T.k0n = A.k0; T.E0n = A.E0;
                    lo = min(lo, A.k0);
                    hi = max(hi, A.k0 + g.n_w);
                }
                lo = max(lo, 0);
                hi = (long long)hi > g.n_samp ? (int)g.n_samp : hi;
                T.lo = lo;
                T.hi = hi;
                if (lo < hi) {
                    T.u0 = units;   // float4 groups [lo/4, ceil(hi/4)) continue the flat range
                    units += ((hi + 3) >> 2) - (lo >> 2);
                    width += hi - lo;
                    tk[ntask++] = T;
                }
            }
        }
        if (STAGE && !err && ntask > 0) {
            // stage the windows that fit (in task order) into this step's buffer
            int* so = S.tsoff + sl * g.task_cap;
            int used = 0;
            unsigned bytes = 0;
            for (int ti = 0; ti < ntask; ++ti) {
                const int w4 = ((tk[ti].hi + 3) & ~3) - (tk[ti].lo & ~3);
                so[ti] = -1;
                if (used + w4 <= S.scap) {
                    so[ti] = used;
                    used += w4;
                    bytes += 8u * (unsigned)w4;
                }
            }
            if (bytes) {
                mbar_arm(&S.bar[sl], bytes);
                for (int ti = 0; ti < ntask; ++ti) {
                    if (so[ti] < 0) continue;
                    const int lo4 = tk[ti].lo & ~3;
                    const unsigned nb = 4u * (unsigned)(((tk[ti].hi + 3) & ~3) - lo4);
                    const size_t off = (size_t)tk[ti].row * g.pitch + lo4;
                    bulk_g2s(S.stage_s + sl * S.scap + so[ti], (const float*)d.sig + off, nb, &S.bar[sl]);
                    bulk_g2s(S.stage_v + sl * S.scap + so[ti], (const float*)d.V + off, nb, &S.bar[sl]);
                }
                S.on[sl] = 1;
            }
        }
        if (err) S.err = err;
        if (valid && !err) {
            // the state-dependent terms of log alpha, so that the decision is
            // one comparison with the log-likelihood change
            double thr, dlp;
            if (dr.type == 0) {
                thr = (double)dr.logu - (dr.blq + S.tabB[n_own]);
                dlp = dr.blb;
            } else if (dr.type == 1) {
                thr = (double)dr.logu - (S.tabD[n_own] - S.elq[ps]);
                dlp = S.mm[ps] - g.lb0;
            } else {
                const double dm = __dsub_rn(c.m, S.mm[ps]);
                thr = (double)dr.logu + dm;
                dlp = -dm;
            }
            S.thr[sl] = thr;
            S.thrf[sl] = (float)thr;
            S.dlp[sl] = dlp;
        }
        S.valid[sl] = valid && !err;
        S.ntask[sl] = ntask;
        S.units[sl] = units;
        S.width[sl] = width;
        S.idx[sl] = idx;
        S.type[sl] = dr.type;
        S.ncand[sl] = ncand;
        S.c[sl] = c;
    }
    __syncwarp();
}

// preparation of a joint move of a pair (all lanes of warp 0; no staging):
// the ordered pair (idx, idx2), then either the exchange of their locations
// (each keeps its time and magnitude) or one common offset; both candidates
// must lie in the region.  The two events' old arrivals and the two
// candidates' are merged by slot; the second event's go to the task's
// extension record, one task per disjoint stretch of a station's windows.
template <bool LAT>
__device__ __noinline__ void prepare_pair(const Geo& g, Sm& S, int step, int sl) {
    const int lane = threadIdx.x & 31;
    const D32& dr = S.draws[step];
    const int n_own = S.n_own;
    A32* cd = S.cand + sl * g.arr_cap;
    A32* cd2 = S.cand2 + sl * g.arr_cap;
    T32* tk = S.tasks + sl * g.task_cap;
    int valid = 0, idx = -1, ps = -1, idx2 = -1, ps2 = -1;
    P32 c, c2;
    clear_p32(c);
    clear_p32(c2);
    if (n_own >= 2) {
        idx = pick32(dr.pickw, n_own);
        const int j = pick32(dr.pick2, n_own - 1);
        idx2 = j + (j >= idx ? 1 : 0);
        ps = S.order[idx];
        ps2 = S.order[idx2];
        if (dr.exch) {
            valid = cand_of(g, S, S.mx[ps2], S.my[ps2], S.mt[ps], S.mm[ps], S.exr[ps2], S.eyr[ps2], c) &&
                    cand_of(g, S, S.mx[ps], S.my[ps], S.mt[ps2], S.mm[ps2], S.exr[ps], S.eyr[ps], c2);
        } else {
            valid = cand_of(g, S, __dadd_rn(S.mx[ps], dr.bx), __dadd_rn(S.my[ps], dr.by),
                            __dadd_rn(S.mt[ps], dr.bt), __dadd_rn(S.mm[ps], dr.bm), S.exr[ps] + dr.xr,
                            S.eyr[ps] + dr.yr, c) &&
                    cand_of(g, S, __dadd_rn(S.mx[ps2], dr.bx), __dadd_rn(S.my[ps2], dr.by),
                            __dadd_rn(S.mt[ps2], dr.bt), __dadd_rn(S.mm[ps2], dr.bm), S.exr[ps2] + dr.xr,
                            S.eyr[ps2] + dr.yr, c2);
        }
    }
    int ncand = 0, ncand2 = 0;
    if (valid) {
        ncand = cand_arrivals<LAT>(g, S, step, c, 0, ps, cd, LAT ? S.coff + sl * g.arr_cap : nullptr);
        ncand2 = cand_arrivals<LAT>(g, S, step, c2, 1, ps2, cd2, LAT ? S.coff2 + sl * g.arr_cap : nullptr);
    }
    __syncwarp();
    if (lane == 0) {
        int err = (ncand > g.arr_cap || ncand2 > g.arr_cap) ? CMH_ERR_CAPACITY : 0;
        int ntask = 0, units = 0, width = 0;
        if (valid && !err) {
            T32X* tx = S.tasksx + sl * g.task_cap;
            const A32* L[4] = {S.earr + ps * g.arr_cap, S.earr + ps2 * g.arr_cap, cd, cd2};
            const int nl[4] = {S.enarr[ps], S.enarr[ps2], ncand, ncand2};
            int il[4] = {0, 0, 0, 0};
            for (;;) {
                int slot = 1 << 30;
                for (int q = 0; q < 4; ++q)
                    if (il[q] < nl[q] && L[q][il[q]].slot < slot) slot = L[q][il[q]].slot;
                if (slot == 1 << 30) break;
                T32 T;
                T32X X;
                T.slot = slot;
                T.row = S.bsta[slot];
                T.skip = ps;
                T.has_o = T.has_n = 0;
                T.k0o = T.k0n = 0;
                T.E0o = T.E0n = 0.f;
                X.pair = 1;
                X.exch = dr.exch;
                X.skip2 = ps2;
                X.has_o2 = X.has_n2 = X.k0o2 = X.k0n2 = 0;
                X.E0o2 = X.E0n2 = 0.f;
                int ws[4], nws = 0;   // window starts at this station, in start order
                for (int q = 0; q < 4; ++q) {
                    if (il[q] >= nl[q] || L[q][il[q]].slot != slot) continue;
                    const A32 A = L[q][il[q]++];
                    if (q == 0) { T.has_o = 1; T.k0o = A.k0; T.E0o = A.E0; }
                    if (q == 1) { X.has_o2 = 1; X.k0o2 = A.k0; X.E0o2 = A.E0; }
                    if (q == 2) { T.has_n = 1; T.k0n = A.k0; T.E0n = A.E0; }
                    if (q == 3) { X.has_n2 = 1; X.k0n2 = A.k0; X.E0n2 = A.E0; }
                    int w = nws++;
                    for (; w > 0 && ws[w - 1] > A.k0; --w) ws[w] = ws[w - 1];
                    ws[w] = A.k0;
                }
                // the two events may be far apart in time: one task per
                // disjoint stretch of the windows' union, not their hull
                for (int a = 0; a < nws && !err;) {
                    int lo = ws[a];
                    int hi = ws[a] + g.n_w;
                    for (++a; a < nws && ws[a] <= hi; ++a) hi = max(hi, ws[a] + g.n_w);
                    if (ntask >= g.task_cap) {
                        err = CMH_ERR_CAPACITY;
                        break;
                    }
                    lo = max(lo, 0);
                    hi = (long long)hi > g.n_samp ? (int)g.n_samp : hi;
                    if (lo < hi) {
                        T.lo = lo;
                        T.hi = hi;
                        T.u0 = units;   // float4 groups [lo/4, ceil(hi/4)) continue the flat range
                        units += ((hi + 3) >> 2) - (lo >> 2);
                        width += hi - lo;
                        tx[ntask] = X;
                        tk[ntask++] = T;
                    }
                }
                if (err) break;
            }
        }
        if (err) S.err = err;
        if (valid && !err) {
            // symmetric proposal: the two events' prior ratio, the change of
            // their magnitudes (0 for an exchange)
            const double dm = __dadd_rn(__dsub_rn(c.m, S.mm[ps]), __dsub_rn(c2.m, S.mm[ps2]));
            const double thr = (double)dr.logu + dm;
            S.thr[sl] = thr;
            S.thrf[sl] = (float)thr;
            S.dlp[sl] = -dm;
        }
        S.valid[sl] = valid && !err;
        S.ntask[sl] = ntask;
        S.units[sl] = units;
        S.width[sl] = width;
        S.idx[sl] = idx;
        S.type[sl] = dr.type;
        S.ncand[sl] = ncand;
        S.c[sl] = c;
        S.idx2[sl] = idx2;
        S.ncand2[sl] = ncand2;
        S.c2[sl] = c2;
    }
    __syncwarp();
}

// preparation of an arrival-time move (all lanes of warp 0; latent offsets,
// no staging): one entry of an event's arrival cache (in slot order: the
// stations it reaches in index order), its offset stepped; the event's
// arrivals become the candidate's with that one's window recomputed, and
// the one station whose variance changes is the step's only task
__device__ __noinline__ void prepare_arrival(const Geo& g, Sm& S, int step, int sl) {
    const int lane = threadIdx.x & 31;
    const D32& dr = S.draws[step];
    const int n_own = S.n_own;
    A32* cd = S.cand + sl * g.arr_cap;
    double* co = S.coff + sl * g.arr_cap;
    T32* tk = S.tasks + sl * g.task_cap;
    int valid = 0, idx = -1, ps = -1, ai = -1, na = 0;
    P32 c;
    clear_p32(c);
    if (n_own > 0) {
        idx = pick32(dr.pickw, n_own);
        ps = S.order[idx];
        na = S.enarr[ps];
        if (na > 0) {
            ai = pick32(dr.pick2, na);
            c.x = S.mx[ps]; c.y = S.my[ps]; c.t = S.mt[ps]; c.m = S.mm[ps];
            event_terms32(g, c.t, c.m, c.K, c.ph, c.mf);
            c.xr = S.exr[ps];
            c.yr = S.eyr[ps];
            valid = 1;
        }
    }
    if (valid) {
        for (int a = lane; a < na; a += 32) {
            A32 A = S.earr[ps * g.arr_cap + a];
            double dl = S.aoff[ps * g.arr_cap + a];
            if (a == ai) {
                dl = __dadd_rn(dl, dr.bx);
                const double xs = S.bx[A.slot], ys = S.by[A.slot];
                window32(g, c.x, c.y, c.t, c.K, c.ph, c.mf, xs, ys, dist32(c.x, c.y, xs, ys), dl, A.k0, A.E0);
            }
            cd[a] = A;
            co[a] = dl;
        }
    }
    __syncwarp();
    if (lane == 0) {
        int ntask = 0, units = 0, width = 0;
        if (valid) {
            const A32 O = S.earr[ps * g.arr_cap + ai], N = cd[ai];
            T32 T;
            T.slot = O.slot;
            T.row = S.bsta[O.slot];
            T.has_o = T.has_n = 1;
            T.k0o = O.k0; T.E0o = O.E0;
            T.k0n = N.k0; T.E0n = N.E0;
            T.skip = ps;
            const int lo = max(min(O.k0, N.k0), 0);
            const long long h = (long long)max(O.k0, N.k0) + g.n_w;
            const int hi = h > g.n_samp ? (int)g.n_samp : (int)h;
            T.lo = lo;
            T.hi = hi;
            if (lo < hi) {
                T.u0 = 0;   // float4 groups [lo/4, ceil(hi/4))
                units = ((hi + 3) >> 2) - (lo >> 2);
                width = hi - lo;
                tk[ntask++] = T;
            }
            // symmetric step of one offset: its prior ratio
            const double a = S.aoff[ps * g.arr_cap + ai], b = co[ai];
            const double s2 = __dmul_rn(g.sig_a, g.sig_a);
            const double dlp = __ddiv_rn(__dsub_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(2.0, s2));
            const double thr = (double)dr.logu - dlp;
            S.thr[sl] = thr;
            S.thrf[sl] = (float)thr;
            S.dlp[sl] = dlp;
        }
        S.valid[sl] = valid;
        S.ntask[sl] = ntask;
        S.units[sl] = units;
        S.width[sl] = width;
        S.idx[sl] = idx;
        S.type[sl] = dr.type;
        S.ncand[sl] = na;
        S.c[sl] = c;
        S.ai[sl] = ai;
    }
    __syncwarp();
}

// the preparation of step `step` into buffer sl, by the kind of its move
template <bool STAGE, bool PAIR, bool LAT>
__device__ __forceinline__ void prepare(const Geo& g, const Dev& d, Sm& S, int step, int sl) {
    const int type = S.draws[step].type;
    if (PAIR && type == 3) prepare_pair<LAT>(g, S, step, sl);
    else if (LAT && type == 4) prepare_arrival(g, S, step, sl);
    else prepare_step<STAGE, LAT>(g, d, S, step, sl);
}

// the change of the log-likelihood over one float4 group of samples
// k4 .. k4+3 of task T (samples outside [T.lo, T.hi) or either window add 0):
// the four terms summed in order
template <bool MEAN, bool PAIR>
__device__ __forceinline__ float group_terms(const Geo& g, const Sm& S, const T32& T, const T32X* X, int k4,
                                             float4 s4, float4 v4) {
    // one SFU evaluation per arrival for the whole group (see arr_var32)
    const float bo = T.has_o ? arr_base32(g, T.E0o, T.k0o, k4) : 0.f;
    const float bn = T.has_n ? arr_base32(g, T.E0n, T.k0n, k4) : 0.f;
    // joint move of a pair: the second event's old and new arrivals
    const bool pr = PAIR && X->pair;
    const float bo2 = pr && X->has_o2 ? arr_base32(g, X->E0o2, X->k0o2, k4) : 0.f;
    const float bn2 = pr && X->has_n2 ? arr_base32(g, X->E0n2, X->k0n2, k4) : 0.f;
    const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
    const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
    float term[4], cnv[4], cnv2[4];
    unsigned need = 0;   // samples whose V' is rebuilt from the arrivals that stay
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int kk = k4 + e;
        const bool io = T.has_o && (unsigned)(kk - T.k0o) < (unsigned)g.n_w;
        const bool inn = T.has_n && (unsigned)(kk - T.k0n) < (unsigned)g.n_w;
        // the same per-sample values the variance synthesis adds, so the
        // priced change is the change written to V on accept
        const float co = io ? __fmul_rn(bo, g.rho_f[e]) : 0.f;
        const float cn = inn ? __fmul_rn(bn, g.rho_f[e]) : 0.f;
        float dd = cn - co;
        cnv[e] = cn;
        cnv2[e] = 0.f;
        if (pr) {
            const bool io2 = X->has_o2 && (unsigned)(kk - X->k0o2) < (unsigned)g.n_w;
            const bool in2 = X->has_n2 && (unsigned)(kk - X->k0n2) < (unsigned)g.n_w;
            const float co2 = io2 ? __fmul_rn(bo2, g.rho_f[e]) : 0.f;
            const float cn2 = in2 ? __fmul_rn(bn2, g.rho_f[e]) : 0.f;
            cnv2[e] = cn2;
            // pair the terms that nearly cancel: an exchange puts each event
            // where the other was, a common offset moves each a little
            dd = X->exch ? __fadd_rn(__fsub_rn(cn, co2), __fsub_rn(cn2, co))
                         : __fadd_rn(__fsub_rn(cn, co), __fsub_rn(cn2, co2));
        }
        term[e] = 0.f;
        if (MEAN && kk < T.hi && dd != 0.f) {
            // additive reading: (d (s - mu) - d^2 / 2) / noise, mu = vv
            term[e] = __fmul_rn(g.inv_noise_f, __fsub_rn(__fmul_rn(dd, __fsub_rn(sv[e], vv[e])),
                                                         __fmul_rn(0.5f, __fmul_rn(dd, dd))));
        } else if (!MEAN && kk < T.hi && dd != 0.f) {
            const float V = vv[e], sm = sv[e];
            const float Vp = V + dd;
            if (Vp < 0.5f * V) {
                need |= 1u << e;   // the changed arrival dominates V
            } else {
                // log(V'/V) - s^2 d / (V V'), one reciprocal (explicitly
                // rounded, so every build of this code gives the same bits)
                const float inv = rcp_sfu(__fmul_rn(V, Vp));
                const float x = __fmul_rn(__fmul_rn(dd, Vp), inv);
                const float q = __fmul_rn(__fmul_rn(sm, sm), __fmul_rn(dd, inv));
                term[e] = __fmul_rn(-0.5f, __fsub_rn(log1p_fast(x), q));
            }
        }
    }
    if (need) {
        // V' of the flagged samples from the arrivals that stay on this
        // station (list order, compensated), one SFU evaluation per
        // arrival for the group; the candidate's own arrival last
        float a2[4], c2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            a2[e] = g.syn0_f;
            c2[e] = 0.f;
        }
        const SA* L = S.sarr + T.slot * g.frz_cap;
        const int nl = S.scnt[T.slot];
        for (int o = 0; o < nl; ++o) {
            const SA A = L[o];
            if (A.own == T.skip || (pr && A.own == X->skip2) || (unsigned)(k4 + 3 - A.k0) >= (unsigned)(g.n_w + 3))
                continue;
            const float base = arr_base32(g, A.E0, A.k0, k4);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (((need >> e) & 1u) && (unsigned)(k4 + e - A.k0) < (unsigned)g.n_w)
                    kahan_add32(a2[e], c2[e], __fmul_rn(base, g.rho_f[e]));
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (!((need >> e) & 1u)) continue;
            if (cnv[e] != 0.f) kahan_add32(a2[e], c2[e], cnv[e]);
            if (cnv2[e] != 0.f) kahan_add32(a2[e], c2[e], cnv2[e]);
            const float V = vv[e], sm = sv[e];
            const float Vr = a2[e] - c2[e];
            const float q = __fmul_rn(__fmul_rn(sm, sm), __fsub_rn(rcp_sfu(Vr), rcp_sfu(V)));
            term[e] = __fmul_rn(-0.5f, __fadd_rn(__logf(__fdividef(Vr, V)), q));
        }
    }
    return __fadd_rn(__fadd_rn(__fadd_rn(term[0], term[1]), term[2]), term[3]);
}

// ---------------------------------------------------------------------------
// pricing of step buffer sl by warps 1..: the change of the Gaussian
// log-likelihood over the float4 groups of all tasks (one flat range; each
// thread issues the loads of kUnroll groups before computing them), one
// float-float partial per warp in S.redf.  PAIR: the tasks of a joint move
// of a pair (the second event's arrivals in their extension records)
// ---------------------------------------------------------------------------
template <bool STAGE, bool MEAN, bool PAIR>
__device__ __forceinline__ void price_tasks(const Geo& g, const Dev& d, Sm& S, int sl) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const T32* tk = S.tasks + sl * g.task_cap;
    const int U = S.units[sl], ntask = S.ntask[sl];
    const int wt = threadIdx.x - 32, nwk = blockDim.x - 32;
    const int* so = S.tsoff + sl * g.task_cap;
    const float* ss = STAGE ? S.stage_s + sl * S.scap : nullptr;
    const float* sv_ = STAGE ? S.stage_v + sl * S.scap : nullptr;
    if (STAGE && S.on[sl] && !mbar_wait(&S.bar[sl], (unsigned)S.ph[sl])) atomicCAS(&S.err, 0, CMH_ERR_TIMEOUT);
    float acc = 0.f, comp = 0.f;
    for (int u0 = wt; u0 < U; u0 += nwk * kUnroll) {
        float4 s4[kUnroll], v4[kUnroll];
        int ti_[kUnroll], k_[kUnroll];
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
            const int u = u0 + r * nwk;
            ti_[r] = -1;
            k_[r] = 0;
            if (u < U) {
                int ti = 0;
                while (ti + 1 < ntask && u >= tk[ti + 1].u0) ++ti;
                const T32& T = tk[ti];
                const int k = ((T.lo >> 2) + (u - T.u0)) << 2;
                ti_[r] = ti;
                k_[r] = k;
                const int o = STAGE ? so[ti] : -1;
                if (STAGE && o >= 0) {
                    s4[r] = *reinterpret_cast<const float4*>(ss + o + (k - (T.lo & ~3)));
                    v4[r] = *reinterpret_cast<const float4*>(sv_ + o + (k - (T.lo & ~3)));
                } else {
                    s4[r] = __ldg(reinterpret_cast<const float4*>((const float*)d.sig + (size_t)T.row * g.pitch + k));
                    v4[r] = *reinterpret_cast<const float4*>((const float*)d.V + (size_t)T.row * g.pitch + k);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
            if (ti_[r] < 0) continue;
            const T32X* X = PAIR ? S.tasksx + sl * g.task_cap + ti_[r] : nullptr;
            kahan_add32(acc, comp, group_terms<MEAN, PAIR>(g, S, tk[ti_[r]], X, k_[r], s4[r], v4[r]));
        }
    }
    float2 v = make_float2(acc, -comp);
    for (int o = 16; o > 0; o >>= 1) {
        float2 w2;
        w2.x = __shfl_xor_sync(FULL, v.x, o);
        w2.y = __shfl_xor_sync(FULL, v.y, o);
        v = ff_add32(v, w2);
    }
    if (lane == 0) S.redf[wid] = v;
}

// every task of a step belongs to a joint move of a pair or none does: a
// kernel with joint moves prices the other steps with the one-event loop
template <bool STAGE, bool MEAN, bool PAIR>
__device__ __forceinline__ void price_step(const Geo& g, const Dev& d, Sm& S, int sl) {
    if (PAIR && S.type[sl] == 3) price_tasks<STAGE, MEAN, true>(g, d, S, sl);
    else price_tasks<STAGE, MEAN, false>(g, d, S, sl);
}

// add the window [lo, hi) priced at blanket slot `slot` to the slot's disjoint
// intervals (one thread): every interval it overlaps or touches is merged
// into it; with no room left it is counted on its own (an upper bound)
__device__ __forceinline__ void iv_add(Sm& S, int slot, int lo, int hi) {
    int2* L = S.uiv + slot * kIv;
    const int n = S.un[slot];
    int w = 0;
    for (int i = 0; i < n; ++i) {
        const int2 a = L[i];
        if (a.x <= hi && lo <= a.y) {
            lo = min(lo, a.x);
            hi = max(hi, a.y);
        } else {
            L[w++] = a;
        }
    }
    if (w < kIv) L[w++] = make_int2(lo, hi);
    else S.cnt[11] += (unsigned long long)(hi - lo);
    S.un[slot] = w;
}

// the decision of step `step` held in buffer sl (lane 0 of warp 0): count it,
// record it, and on a commit update the region's event bookkeeping; rm / put
// receive the event whose arrivals leave / join the station lists (-1: none).
// t is the float-float sum of the step's partial log-likelihood changes.
template <bool PAIR, bool LAT>
__device__ __forceinline__ int decide_lane0(const Geo& g, const Dev& d, Sm& S, long long sweep, int cell, int step,
                                         int sl, float2 t, int valid, int& rm, int& put, int& rm2, int& put2) {
    const int type = S.type[sl], n_own = S.n_own, idx = S.idx[sl];
    const D32& dr = S.draws[step];
    // counters: birth, death, move in [0..8]; the joint move of a pair in
    // [12..14]; the arrival-time move in [15..17]
    const int ext = (LAT && type == 4) ? 15 : 12;
    const int c_prop = (!(PAIR || LAT) || type < 3) ? type : ext,
              c_eval = (!(PAIR || LAT) || type < 3) ? 3 + type : ext + 1,
              c_acc = (!(PAIR || LAT) || type < 3) ? 6 + type : ext + 2;
    ++S.cnt[c_prop];
    double dll = 0.0, la = -INFINITY, dlp = 0.0;
    int acc = 0;
    if (valid) {
        ++S.cnt[c_eval];
        if (g.count_unique) {
            const T32* tk = S.tasks + sl * g.task_cap;
            for (int ti = 0; ti < S.ntask[sl]; ++ti) iv_add(S, tk[ti].slot, tk[ti].lo, tk[ti].hi);
        }
        S.cnt[9] += (unsigned long long)S.width[sl];
        // float32 first: its gap to the threshold errs by < 3e-7
        // (|t.x| + |thr|), so outside 1e-5 of that it decides as
        // float64 would; inside, float64 decides
        const float gap = (t.x + t.y) - S.thrf[sl];
        const float tol = 1e-5f * (fabsf(t.x) + fabsf(S.thrf[sl])) + 1e-30f;
        if (gap > tol || gap < -tol) {
            acc = gap > 0.f;
            if (acc || d.trace) dll = (double)t.x + (double)t.y;
        } else {
            dll = (double)t.x + (double)t.y;
            acc = dll > S.thr[sl];
        }
        dlp = S.dlp[sl];
        if (d.trace) la = dll + ((double)dr.logu - S.thr[sl]);
    }
    if (d.trace) {
        const long long slot = ((sweep - d.trace_sweep0) * g.n_cells + cell) * (long long)g.k + step;
        if (slot >= 0 && slot < d.trace_cap) {
            cmh_trace& R = d.trace[slot];
            R.sweep = (int)sweep; R.cell = cell; R.step = step; R.type = type;
            R.evaluated = valid; R.accepted = acc; R.n_before = n_own; R.written = 1;
            R.dll = dll; R.log_alpha = la;
        }
    }
    const int do_commit = acc && g.commit;
    if (acc) ++S.cnt[c_acc];
    if (do_commit) {
        S.cnt[10] += (unsigned long long)S.width[sl];
        // latent offsets drawn from (or dropped to) their prior cancel from
        // log alpha but change the log-density: the candidates' offsets in,
        // the replaced events' out (an arrival-time move's are in dlp)
        double dlo = 0.0;
        if (LAT && type != 4) {
            auto rowsum = [&](const double* row, int n) {
                double q = 0.0;
                for (int a = 0; a < n; ++a) q += row[a] * row[a];
                return (double)n * S.lop0 - q * S.lopi;
            };
            const int p1 = idx >= 0 ? S.order[idx] : -1;
            if (type != 1) dlo += rowsum(S.coff + sl * g.arr_cap, S.ncand[sl]);
            if (type != 0) dlo -= rowsum(S.aoff + p1 * g.arr_cap, S.enarr[p1]);
            if (type == 3) {
                const int p2 = S.order[S.idx2[sl]];
                dlo += rowsum(S.coff2 + sl * g.arr_cap, S.ncand2[sl]) - rowsum(S.aoff + p2 * g.arr_cap, S.enarr[p2]);
            }
        }
        S.region_dlp += dll + dlp + dlo;
        if (type == 1) {
            const int ps = S.order[idx];
            rm = ps;
            for (int q = idx; q + 1 < n_own; ++q) S.order[q] = S.order[q + 1];
            S.freel[S.n_free++] = ps;
            S.n_own = n_own - 1;
        } else if (type == 0) {
            const int ps = S.freel[--S.n_free];
            S.eid[ps] = ((unsigned long long)(sweep + 1) << 32) | ((unsigned long long)cell << 12) |
                        (unsigned long long)step;
            S.order[n_own] = ps;
            S.n_own = n_own + 1;
            put = ps;
        } else {
            rm = put = S.order[idx];
            if (PAIR && type == 3) rm2 = put2 = S.order[S.idx2[sl]];
        }
    }
    return do_commit;
}

// remove the arrivals of own event ps from its stations' lists, keeping the
// order (the 32 lanes of a warp: entries in chunks of 32, kept ones compacted
// by ballot; a chunk is read before any of it is written, and writes land at
// or before the positions read)
__device__ __forceinline__ void lists_remove_warp(const Geo& g, Sm& S, int ps) {
    const int lane = threadIdx.x & 31;
    const int na = S.enarr[ps];
    for (int a = 0; a < na; ++a) {
        const int b = S.earr[ps * g.arr_cap + a].slot;
        SA* L = S.sarr + b * g.frz_cap;
        const int n = S.scnt[b];
        int w = 0;
        for (int c = 0; c < n; c += 32) {
            const int i = c + lane;
            SA e = {0, 0.f, 0, 0};
            if (i < n) e = L[i];
            const bool keep = i < n && e.own != ps;
            const unsigned bal = __ballot_sync(FULL, keep);
            __syncwarp();
            if (keep) L[w + __popc(bal & ((1u << lane) - 1))] = e;
            w += __popc(bal);
            __syncwarp();
        }
        if (lane == 0) S.scnt[b] = w;
        __syncwarp();
    }
}

// append the arrivals A[0..na) of own event ps to their stations' lists
__device__ __forceinline__ void lists_add(const Geo& g, Sm& S, int ps, const A32* A, int na) {
    for (int a = 0; a < na; ++a) {
        const int b = A[a].slot;
        const int n = S.scnt[b];
        if (n >= g.frz_cap) {
            S.err = CMH_ERR_CAPACITY;
            return;
        }
        S.sarr[b * g.frz_cap + n] = SA{A[a].k0, A[a].E0, ps, 0};
        S.scnt[b] = n + 1;
    }
}

// a committed candidate c (arrivals cd[0..ncd), their latent offsets co or
// null) of a step of type `type` becomes own event ps (one thread): its
// master, density term, relative position and arrival cache, and its
// arrivals join the station lists
__device__ __forceinline__ void put_event(const Geo& g, const Dev& d, Sm& S, const P32& c, const A32* cd, int ncd,
                                          int type, int ps, const double* co) {
    S.mx[ps] = c.x; S.my[ps] = c.y; S.mt[ps] = c.t; S.mm[ps] = c.m;
    // a move's own log alpha has no position term: the moved event's term
    // (for a later death) is taken here (an arrival-time move keeps it)
    if (type != 4) S.elq[ps] = type == 0 ? c.lq : (g.bt_on ? bt_lq(g, d, S, c.x, c.y, c.t, c.m) : S.lq_unif);
    S.exr[ps] = c.xr; S.eyr[ps] = c.yr;
    for (int a = 0; a < ncd; ++a) S.earr[ps * g.arr_cap + a] = cd[a];
    if (co)
        for (int a = 0; a < ncd; ++a) S.aoff[ps * g.arr_cap + a] = co[a];
    S.enarr[ps] = ncd;
    lists_add(g, S, ps, cd, ncd);
}

// re-synthesise V over the windows of buffer sl's tasks from the station
// lists (threads rt of rn): groups of four samples, one SFU evaluation per
// arrival and group, compensated sums in list order
__device__ __forceinline__ void resynth(const Geo& g, const Dev& d, const Sm& S, int sl, int rt, int rn) {
    const T32* tk = S.tasks + sl * g.task_cap;
    for (int ti = 0; ti < S.ntask[sl]; ++ti) {
        const T32& T = tk[ti];
        const SA* L = S.sarr + T.slot * g.frz_cap;
        const int nl = S.scnt[T.slot];
        float* vrow = (float*)d.V + (size_t)T.row * g.pitch;
        for (int k4 = ((T.lo >> 2) + rt) << 2; k4 < T.hi; k4 += rn << 2) {
            float a2[4], c2[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                a2[e] = g.syn0_f;
                c2[e] = 0.f;
            }
            for (int o = 0; o < nl; ++o) {
                const SA A = L[o];
                if ((unsigned)(k4 + 3 - A.k0) >= (unsigned)(g.n_w + 3)) continue;
                const float base = arr_base32(g, A.E0, A.k0, k4);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if ((unsigned)(k4 + e - A.k0) < (unsigned)g.n_w)
                        kahan_add32(a2[e], c2[e], __fmul_rn(base, g.rho_f[e]));
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (k4 + e >= T.lo && k4 + e < T.hi) vrow[k4 + e] = a2[e] - c2[e];
        }
    }
}

// the mbarriers of the staging buffers, once per CTA (their phase bits carry
// over from one region to the next; every region leaves no copy in flight)
template <bool STAGE>
__device__ __forceinline__ void init_staging(Sm& S) {
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            S.ph[b] = 0;
            S.on[b] = 0;
            if (STAGE) mbar_init(&S.bar[b], 1);
        }
        if (STAGE) fence_async_shared();   // the initialised barriers are visible to the async proxy
    }
}

// one colour phase of one region, in two parts (every thread of the CTA).
// region_begin: what does not depend on the neighbouring regions' state --
// the region's rectangle, its own events, the acceptance constants, the
// blanket stations, the own events' arrival caches and the k steps' random
// draws; a kernel whose regions wait for their lower-colour neighbours runs
// it before that wait.  Returns false (uniformly) after latching an error.
template <bool STAGE, bool LAT>
__device__ __forceinline__ bool region_begin(const Geo& g, const Dev& d, int cell, long long sweep, Sm& S,
                                             unsigned char* smem) {
    const Store St = d.st[sweep & 1];
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    const int ix = cell % g.ncx, iy = cell / g.ncx;
    const int start = St.start[cell], n0 = St.count[cell];
    (void)ix;
    (void)iy;
    (void)start;
    if (tid == 0) {
        layout32(g, &S, smem, g.spill ? d.spill_buf + (size_t)blockIdx.x * (size_t)g.spill_bytes : nullptr);
        S.cell = cell;
        S.sweep = sweep;
        if (LAT) {   // the offsets' prior, its constant part once per region
            const double s2 = __dmul_rn(g.sig_a, g.sig_a);
            S.lop0 = __dmul_rn(-0.5, log(__dmul_rn(2.0 * M_PI, s2)));
            S.lopi = __ddiv_rn(1.0, __dmul_rn(2.0, s2));
        }
        S.sx = d.shift[0];
        S.sy = d.shift[1];
        cell_rect(g, S.sx, S.sy, cell, S.rect);
        S.X0 = __dadd_rn(S.sx, __dmul_rn((double)(ix - 1), g.L));
        S.Y0 = __dadd_rn(S.sy, __dmul_rn((double)(iy - 1), g.L));
        S.rl[0] = (float)(S.rect[0] - S.X0);
        S.rl[1] = (float)(S.rect[1] - S.X0);
        S.rl[2] = (float)(S.rect[2] - S.Y0);
        S.rl[3] = (float)(S.rect[3] - S.Y0);
        S.err = (n0 + g.k > g.ev_cap) ? CMH_ERR_CAPACITY : 0;
        S.n_own = n0;
        S.n_free = g.ev_cap - n0;
        S.region_dlp = 0.0;
        S.acc = 0;
    }
    if (tid < 18) S.cnt[tid] = 0;
    // only thread 0 has S.err initialised yet: the others would read what an
    // earlier CTA left in this shared memory
    if (__syncthreads_or(tid == 0 && S.err != 0)) {
        if (tid == 0) latch(d.status, S.err);
        return false;
    }
    const double X0 = S.X0, Y0 = S.Y0;
    // ---- own events: masters, relative position, free list ----------------------
    for (int i = tid; i < g.ev_cap; i += nthr) {
        if (i < n0) {
            const double x = St.x[start + i], y = St.y[start + i];
            S.mx[i] = x; S.my[i] = y; S.mt[i] = St.t[start + i]; S.mm[i] = St.m[start + i];
            S.exr[i] = (float)__dsub_rn(x, X0);
            S.eyr[i] = (float)__dsub_rn(y, Y0);
            S.eid[i] = St.id[start + i];
            S.order[i] = i;
        } else {
            S.freel[g.ev_cap - 1 - i] = i;   // pops give the lowest free slot first
        }
    }
    // ---- acceptance constants: the count terms of birth / death by event
    // count; the position terms (log beta - log q_b) per candidate / event ----
    {
        for (int n = tid; n <= g.ev_cap; n += nthr) {
            S.tabB[n] = g.lpdpb - d.log_n[n + 1];
            S.tabD[n] = n > 0 ? -g.lpdpb + d.log_n[n] : 0.0;
        }
        if (tid == 0) {
            const double area = __dmul_rn(__dsub_rn(S.rect[1], S.rect[0]), __dsub_rn(S.rect[3], S.rect[2]));
            S.qu = __ddiv_rn(1.0, __dmul_rn(area, g.T));
            S.lq_unif = __dsub_rn(g.lLWT, log(S.qu));
            S.qmu = (1.0 - g.bt_mix) * S.qu;
            S.bt_G = 0.0;
            S.bt_in = 0.0;
            S.bt_np = 0;
            S.bt_last = -1;
        }
        if (g.bt_on) {
            // the region's pixels in (iy, ix) order: masses in parallel, then
            // their running sum in that order by one thread
            int x0, x1, y0, y1;
            bt_range(S.rect[0], S.rect[1], g.bt_hx, g.bt_nx, x0, x1);
            bt_range(S.rect[2], S.rect[3], g.bt_hy, g.bt_ny, y0, y1);
            const int wx = x1 - x0 + 1, np = wx * (y1 - y0 + 1), npc = np < kMaxPix ? np : kMaxPix;
            for (int k = tid; k < npc; k += nthr) {
                const int px = x0 + k % wx, py = y0 + k / wx;
                S.pcum[k] = bt_weight(g, d, S.rect, px, py);
                S.pidx[k] = py * g.bt_nx + px;
            }
            __syncthreads();
            if (tid == 0) {
                if (np > kMaxPix) S.err = CMH_ERR_CAPACITY;
                double run = 0.0;
                for (int k = 0; k < npc; ++k) {
                    const double a = S.pcum[k];
                    run = __dadd_rn(run, a);
                    if (a > 0.0) S.bt_last = k;
                    S.pcum[k] = run;
                }
                S.bt_np = npc;
                S.bt_G = run;
                S.bt_in = run > 0.0 ? 1.0 / (g.bt_pixarea * run * g.bt_dt) : 0.0;
            }
        }
    }
    // ---- blanket: stations within R_max of the region (float test, margin) ----
    // among the cell's candidates (a superset, in station order); warp w scans
    // a contiguous chunk of them and chunks are concatenated in order, so the
    // blanket lists stations by index
    {
        const float r0 = (float)S.rect[0], r1 = (float)S.rect[1], r2 = (float)S.rect[2], r3 = (float)S.rect[3];
        const float Rm = g.R_f * 1.0001f + 1e-3f;
        const int* cand = d.bl_idx + d.bl_off[cell];
        const int n_cand = d.bl_off[cell + 1] - d.bl_off[cell];
        const int chunk = (n_cand + nw - 1) / nw;
        const int j0 = wid * chunk, j1 = min(n_cand, j0 + chunk);
        auto in_blanket = [&](int q) {
            const int j = cand[q];
            const float fx = d.stxf[j], fy = d.styf[j];
            const float dx = fx < r0 ? r0 - fx : (fx > r1 ? fx - r1 : 0.f);
            const float dy = fy < r2 ? r2 - fy : (fy > r3 ? fy - r3 : 0.f);
            return dx * dx + dy * dy < Rm * Rm;
        };
        int cnt = 0;
        for (int j = j0 + lane; j - lane < j1; j += 32) cnt += __popc(__ballot_sync(FULL, j < j1 && in_blanket(j)));
        if (lane == 0) S.warp_cnt[wid] = cnt;
        __syncthreads();
        int pos = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) pos += S.warp_cnt[w];
            total += S.warp_cnt[w];
        }
        for (int j = j0 + lane; j - lane < j1; j += 32) {
            const bool in = j < j1 && in_blanket(j);
            const unsigned bal = __ballot_sync(FULL, in);
            const int p = pos + __popc(bal & ((1u << lane) - 1));
            if (in && p < g.blk_cap) {
                const int st = cand[j];
                S.bsta[p] = st;
                S.bx[p] = d.stx[st];
                S.by[p] = d.sty[st];
            }
            pos += __popc(bal);
        }
        if (tid == 0) {
            if (total > g.blk_cap) S.err = CMH_ERR_CAPACITY;
            S.n_blk = min(total, g.blk_cap);
        }
        __syncthreads();
    }
    const int n_blk = S.n_blk;
    if (g.count_unique)
        for (int b = tid; b < n_blk; b += nthr) S.un[b] = 0;
    // position terms of the own events (the death Hastings term)
    for (int i = tid; i < n0; i += nthr)
        S.elq[i] = g.bt_on ? bt_lq(g, d, S, S.mx[i], S.my[i], S.mt[i], S.mm[i]) : S.lq_unif;
    // ---- arrival cache of the own events (warp per event, lanes over slots) -----
    for (int i = wid; i < n0; i += nw) {
        int K;
        float ph, mf;
        event_terms32(g, S.mt[i], S.mm[i], K, ph, mf);
        int na = 0;
        for (int b0 = 0; b0 < n_blk; b0 += 32) {
            const int b = b0 + lane;
            int k0 = 0;
            float E0 = 0.f, dd = 0.f;
            double dl = 0.0;   // latent offset of (event, station) from the store's row
            const bool r = b < n_blk && reach32(g, S.mx[i], S.my[i], S.bx[b], S.by[b], dd);
            if (r) {
                if (LAT) dl = St.off[(size_t)(start + i) * g.n_st + S.bsta[b]];
                window32(g, S.mx[i], S.my[i], S.mt[i], K, ph, mf, S.bx[b], S.by[b], dd, dl, k0, E0);
            }
            const unsigned bal = __ballot_sync(FULL, r);
            const int p = na + __popc(bal & ((1u << lane) - 1));
            if (r && p < g.arr_cap) {
                S.earr[i * g.arr_cap + p] = A32{b, k0, E0, 0};
                if (LAT) S.aoff[i * g.arr_cap + p] = dl;
            }
            na += __popc(bal);
        }
        if (lane == 0) {
            if (na > g.arr_cap) atomicCAS(&S.err, 0, CMH_ERR_CAPACITY);
            S.enarr[i] = min(na, g.arr_cap);
        }
    }
    // ---- the k steps' random draws (Philox stream 0, counter (sweep, cell, step, 0|1))
    const unsigned long long thr_b = (unsigned long long)ceil(g.p_birth * 9007199254740992.0);
    const unsigned long long thr_d = (unsigned long long)ceil(__dadd_rn(g.p_birth, g.p_death) * 9007199254740992.0);
    const double cp = __dadd_rn(__dadd_rn(g.p_birth, g.p_death), g.p_pair);
    const unsigned long long thr_p = (unsigned long long)ceil(cp * 9007199254740992.0);
    const unsigned long long thr_a = LAT ? (unsigned long long)ceil(__dadd_rn(cp, g.p_arr) * 9007199254740992.0) : 0ULL;
    // one warp, warp 1, draws them: the float64 of the walk offsets (~250
    // float64 instructions, each holding its sub-partition's float64 pipe for
    // ~64 cycles whatever the number of active lanes) then runs on a
    // sub-partition whose float64 pipe no manager warp (warp 0 of every
    // resident CTA: the decisions) uses
    for (int st = wid == 1 ? lane : g.k; st < g.k; st += 32) {
        unsigned long long c0[4] = {(unsigned long long)sweep, (unsigned long long)cell, (unsigned long long)st, 0ULL};
        unsigned long long c1[4] = {(unsigned long long)sweep, (unsigned long long)cell, (unsigned long long)st, 1ULL};
        philox4x64(c0, g.seed, 0ULL);
        philox4x64(c1, g.seed, 0ULL);
        D32 D;
        const unsigned long long u53 = c0[0] >> 11;   // u < p  <=>  u53 < p 2^53 (rounded up)
        D.type = u53 < thr_b ? 0 : (u53 < thr_d ? 1 : (u53 < thr_p ? 3 : ((LAT && u53 < thr_a) ? 4 : 2)));
        // joint move of a pair: the second pick from word 7, the exchange
        // when bit 36 of word 1 is clear
        D.pick2 = (unsigned)(c1[3] & 0xffffffffULL);
        D.exch = ((c0[1] >> 36) & 1ULL) == 0ULL;
        D.pickw = (unsigned)(c0[1] & 0xffffffffULL);
        D.logu = __logf(u32o(c1[2]));
        D.bvalid = 0;
        D.bK = 0;
        D.bx = D.by = D.bt = D.bm = D.blb = D.blq = 0.0;
        if (D.type == 0) {
            P32 e;
            bool drew_m = false;
            if (g.bt_on && S.bt_last >= 0 && u01(c1[3]) < g.bt_mix) {
                drew_m = learned_birth(g, d, S, sweep, cell, st, c0[2], c0[3], e);
            } else {
                e.x = __dadd_rn(S.rect[0], __dmul_rn(u01(c0[2]), __dsub_rn(S.rect[1], S.rect[0])));
                e.y = __dadd_rn(S.rect[2], __dmul_rn(u01(c0[3]), __dsub_rn(S.rect[3], S.rect[2])));
                e.t = __dmul_rn(u01(c1[0]), g.T);
            }
            if (!drew_m) e.m = mag_from_u53(c1[1]);
            D.blq = g.bt_on ? bt_lq(g, d, S, e.x, e.y, e.t, e.m) : S.lq_unif;
            to_rel(g, X0, Y0, e);
            D.bx = e.x; D.by = e.y; D.bt = e.t; D.bm = e.m;
            D.blb = g.lb0 - e.m;
            D.xr = e.xr; D.yr = e.yr; D.ph = e.ph; D.mf = e.mf; D.bK = e.K;
            // inside [r0, r1) x [r2, r3) by construction up to rounding at the
            // edges: decide in float32 away from them, exactly near them
            const bool sure = e.xr >= S.rl[0] + kDr && e.xr < S.rl[1] - kDr && e.yr >= S.rl[2] + kDr &&
                              e.yr < S.rl[3] - kDr && e.K >= 1 && e.K + 2 <= g.TfK;
            D.bvalid = sure || inside_exact(g, S.sx, S.sy, cell, e.x, e.y, e.t, e.m);
        } else if (D.type == 2 || D.type == 3 || D.type == 4) {
            // the walk offset in float64 (a joint move's common offset too),
            // the same definition as the float64
            // form (Box-Muller, each Gaussian rounded to 2^-20, signs from
            // word 1): the float64 candidate is then the one the exact chain
            // proposes, not one a float32 rounding away from it, so the
            // float32 terms price the same candidate (an arrival's first
            // sample can change for a candidate a millimetre away).  Computed
            // here, for all k steps at once, off the step chain.
            const double r1 = __dsqrt_rn(__dmul_rn(-2.0, log(u01o(c0[2]))));
            const double th1 = __dmul_rn(6.283185307179586, u01(c0[3]));
            const double r2 = __dsqrt_rn(__dmul_rn(-2.0, log(u01o(c1[0]))));
            const double th2 = __dmul_rn(6.283185307179586, u01(c1[1]));
            const double z[4] = {__dmul_rn(r1, cos(th1)), __dmul_rn(r1, sin(th1)), __dmul_rn(r2, cos(th2)),
                                 __dmul_rn(r2, sin(th2))};
            // (the arrival-time move steps its offset by sig_da times the first)
            const double sg[4] = {D.type == 4 ? g.sig_da : g.sig_xy, g.sig_xy, g.sig_t, g.sig_m};
            double o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                double q = __dmul_rn(rint(__dmul_rn(fabs(z[i]), 1048576.0)), 1.0 / 1048576.0);
                if ((c0[1] >> (32 + i)) & 1ULL) q = -q;
                o[i] = __dmul_rn(sg[i], q);
            }
            D.bx = o[0]; D.by = o[1]; D.bt = o[2]; D.bm = o[3];
            D.xr = (float)o[0]; D.yr = (float)o[1]; D.ph = (float)o[2]; D.mf = (float)o[3];
        } else {
            D.xr = D.yr = D.ph = D.mf = 0.f;
        }
        S.draws[st] = D;
    }
    if (__syncthreads_or(S.err != 0)) {
        if (tid == 0) latch(d.status, S.err);
        return false;
    }
    return true;

}

// region_rest: the station arrival lists (the neighbouring regions' events,
// read once they have finished this sweep, then the own events), the k MH
// steps and the write-back of the region's events.  MEAN: the additive
// likelihood reading (a kernel per reading, so each pricing loop is compiled
// for its own)
template <bool STAGE, bool MEAN, bool PAIR, bool LAT>
__device__ __forceinline__ void region_rest(const Geo& g, const Dev& d, int cell, long long sweep, Sm& S) {
    const Store St = d.st[sweep & 1];
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    const int ix = cell % g.ncx, iy = cell / g.ncx;
    const int start = St.start[cell], n0 = S.n_own;
    const int n_blk = S.n_blk;
    // ---- station lists: arrivals of the neighbouring cells (other colours) in
    // (cell, id) order, then the region's own events in id order
    for (int b = tid; b < n_blk; b += nthr) S.scnt[b] = 0;
    {
        // the neighbouring cells' slices in one round, then their events in
        // batches of up to ev_cap, in (cell, id) order
        const int P1 = g.period - 1, side = 2 * P1 + 1, n_nb = side * side;
        if (tid < n_nb) {
            const int jx = ix - P1 + tid % side, jy = iy - P1 + tid / side;
            int s0 = 0, nn = 0;
            if (jx >= 0 && jy >= 0 && jx < g.ncx && jy < g.ncy && jy * g.ncx + jx != cell) {
                s0 = St.start[jy * g.ncx + jx];
                nn = St.count[jy * g.ncx + jx];
            }
            S.nb_start[tid] = s0;
            S.nb_cnt[tid] = nn;
        }
        __syncthreads();
        if (tid == 0) {
            int off = 0;
            for (int q = 0; q < n_nb; ++q) {
                S.nb_off[q] = off;
                off += S.nb_cnt[q];
            }
            S.nb_off[n_nb] = off;
        }
        __syncthreads();
        const int total = S.nb_off[n_nb];
        for (int b0 = 0; b0 < total; b0 += g.ev_cap) {
            const int nn = min(g.ev_cap, total - b0);
            for (int i = tid; i < nn; i += nthr) {
                const int gi = b0 + i;
                int q = 0;
                while (S.nb_off[q + 1] <= gi) ++q;
                const int src = S.nb_start[q] + (gi - S.nb_off[q]);
                const double t = St.t[src];
                S.nx[i] = St.x[src];
                S.ny[i] = St.y[src];
                S.nt[i] = t;
                if (LAT) S.nsrc[i] = src;
                event_terms32(g, t, St.m[src], S.nK[i], S.nph[i], S.nmf[i]);
            }
            __syncthreads();
            for (int b = wid; b < n_blk; b += nw) {
                int nf = S.scnt[b];
                for (int i0 = 0; i0 < nn; i0 += 32) {
                    const int i = i0 + lane;
                    int k0 = 0;
                    float E0 = 0.f, dd = 0.f;
                    const bool r = i < nn && reach32(g, S.nx[i], S.ny[i], S.bx[b], S.by[b], dd);
                    if (r) {
                        const double dl = LAT ? St.off[(size_t)S.nsrc[i] * g.n_st + S.bsta[b]] : 0.0;
                        window32(g, S.nx[i], S.ny[i], S.nt[i], S.nK[i], S.nph[i], S.nmf[i], S.bx[b], S.by[b], dd, dl,
                                 k0, E0);
                    }
                    const unsigned bal = __ballot_sync(FULL, r);
                    const int p = nf + __popc(bal & ((1u << lane) - 1));
                    if (r && p < g.frz_cap) S.sarr[b * g.frz_cap + p] = SA{k0, E0, kFrozen, 0};
                    nf += __popc(bal);
                }
                __syncwarp();
                if (lane == 0) {
                    if (nf > g.frz_cap) atomicCAS(&S.err, 0, CMH_ERR_CAPACITY);
                    S.scnt[b] = min(nf, g.frz_cap);
                }
                __syncwarp();
            }
            __syncthreads();   // this batch fully consumed
        }
    }
    __syncthreads();
    for (int b = wid; b < n_blk; b += nw) {
        int nf = S.scnt[b];
        for (int q0 = 0; q0 < n0; q0 += 32) {
            const int q = q0 + lane;
            bool hit = false;
            SA A = {0, 0.f, q, 0};
            if (q < n0)
                for (int a = 0; a < S.enarr[q]; ++a)
                    if (S.earr[q * g.arr_cap + a].slot == b) {
                        hit = true;
                        A.k0 = S.earr[q * g.arr_cap + a].k0;
                        A.E0 = S.earr[q * g.arr_cap + a].E0;
                    }
            const unsigned bal = __ballot_sync(FULL, hit);
            const int p = nf + __popc(bal & ((1u << lane) - 1));
            if (hit && p < g.frz_cap) S.sarr[b * g.frz_cap + p] = A;
            nf += __popc(bal);
        }
        __syncwarp();
        if (lane == 0) {
            if (nf > g.frz_cap) atomicCAS(&S.err, 0, CMH_ERR_CAPACITY);
            S.scnt[b] = min(nf, g.frz_cap);
        }
        __syncwarp();
    }
    if (wid == 0) prepare<STAGE, PAIR, LAT>(g, d, S, 0, 0);
    __syncthreads();
    for (int step = 0; step < g.k; ++step) {
        const int sl = step & 1;
        const int valid = S.valid[sl];
        // ================ prepare step+1 (warp 0) || price step (warps 1..) =========
        if (wid == 0) {
            if (step + 1 < g.k) prepare<STAGE, PAIR, LAT>(g, d, S, step + 1, sl ^ 1);   // assumes a rejection
        } else if (valid) {
            // (this buffer is refilled by bulk copies only after two more
            // barriers: these generic reads come first)
            price_step<STAGE, MEAN, PAIR>(g, d, S, sl);
        }
        // errors are set before a barrier and read through its OR, so every
        // thread leaves the loop at the same point
        if (__syncthreads_or(S.err != 0)) break;
        // ================ decision (warp 0; float64 on lane 0) =====================
        if (wid == 0) {
            // partials of warps 1..7 in lanes 1..7: a three-level tree
            float2 t = (valid && lane > 0 && lane < nw) ? S.redf[lane] : make_float2(0.f, 0.f);
            for (int o = kTree0; o > 0; o >>= 1) {
                float2 w2;
                w2.x = __shfl_xor_sync(FULL, t.x, o);
                w2.y = __shfl_xor_sync(FULL, t.y, o);
                t = ff_add32(t, w2);
            }
            int rm = -1, put = -1;   // event leaving its station lists / event (re)joining them
            int rm2 = -1, put2 = -1; // the second event of a joint move
            if (lane == 0) {
                if (STAGE && S.on[sl]) {   // this buffer's copies have landed (the workers waited)
                    if (!mbar_wait(&S.bar[sl], (unsigned)S.ph[sl])) S.err = CMH_ERR_TIMEOUT;
                    S.ph[sl] ^= 1;
                    S.on[sl] = 0;
                }
                S.acc = decide_lane0<PAIR, LAT>(g, d, S, sweep, cell, step, sl, t, valid, rm, put, rm2, put2);
            }
            // the removed or moved event's arrivals leave their station lists
            // (all lanes), then the new arrivals join (lane 0)
            rm = __shfl_sync(FULL, rm, 0);
            put = __shfl_sync(FULL, put, 0);
            if (rm >= 0) lists_remove_warp(g, S, rm);
            if (PAIR) {   // the second event of a joint move
                rm2 = __shfl_sync(FULL, rm2, 0);
                if (rm2 >= 0) lists_remove_warp(g, S, rm2);
            }
            if (lane == 0 && put >= 0)
                put_event(g, d, S, S.c[sl], S.cand + sl * g.arr_cap, S.ncand[sl], S.type[sl], put,
                          LAT ? S.coff + sl * g.arr_cap : nullptr);
            if (PAIR && lane == 0 && put2 >= 0)
                put_event(g, d, S, S.c2[sl], S.cand2 + sl * g.arr_cap, S.ncand2[sl], S.type[sl], put2,
                          LAT ? S.coff2 + sl * g.arr_cap : nullptr);
        }
        if (__syncthreads_or(S.err != 0)) break;
        // ================ commit: re-synthesise V on the touched windows ============
        // The prepared next step assumed a rejection and is prepared again.
        // Without staging that only reads shared memory, so warp 0 does it
        // while the workers re-synthesise V; with staging its bulk copies
        // read V, so it follows the re-synthesis.
        if (S.acc) {
            const int rt = STAGE ? tid : tid - 32, rn = STAGE ? nthr : nthr - 32;
            if (!STAGE && wid == 0) {
                if (step + 1 < g.k) prepare<STAGE, PAIR, LAT>(g, d, S, step + 1, sl ^ 1);
            } else {
                resynth(g, d, S, sl, rt, rn);
            }
            if (STAGE) {
                fence_async_global();   // the new V is visible to the next bulk copies
                __syncthreads();
                if (wid == 0 && step + 1 < g.k) prepare<STAGE, PAIR, LAT>(g, d, S, step + 1, sl ^ 1);
            }
            if (__syncthreads_or(S.err != 0)) break;
        }
    }
    __syncthreads();
    if (STAGE && tid == 0)
        for (int b = 0; b < 2; ++b)
            if (S.on[b]) {   // copies still in flight after an early exit: let them land
                if (!mbar_wait(&S.bar[b], (unsigned)S.ph[b])) S.err = CMH_ERR_TIMEOUT;
                S.on[b] = 0;
            }
    if (__syncthreads_or(S.err != 0)) {
        if (tid == 0) latch(d.status, S.err);
        return;
    }
    const int n_fin = S.n_own;
    for (int i = tid; i < n_fin; i += nthr) {
        const int ps = S.order[i];
        St.x[start + i] = S.mx[ps];
        St.y[start + i] = S.my[ps];
        St.t[start + i] = S.mt[ps];
        St.m[start + i] = S.mm[ps];
        St.id[start + i] = S.eid[ps];
    }
    if (LAT) {
        // offset rows of the written events: 0 but at the stations they reach
        for (size_t q = tid; q < (size_t)n_fin * g.n_st; q += nthr) St.off[(size_t)start * g.n_st + q] = 0.0;
        __syncthreads();
        for (int i = wid; i < n_fin; i += nw) {
            const int ps = S.order[i];
            for (int a = lane; a < S.enarr[ps]; a += 32)
                St.off[(size_t)(start + i) * g.n_st + S.bsta[S.earr[ps * g.arr_cap + a].slot]] =
                    S.aoff[ps * g.arr_cap + a];
        }
    }
    if (tid == 0) {
        St.count[cell] = n_fin;
        d.region_dlp[cell] = S.region_dlp;
        for (int t = 0; t < 11; ++t)
            if (S.cnt[t]) atomicAdd(&d.stats[t], S.cnt[t]);
        for (int t = 0; t < 3; ++t) {   // joint moves of a pair, arrival-time moves: proposed, evaluated, accepted
            if (S.cnt[12 + t]) atomicAdd(&d.stats[11 + t], S.cnt[12 + t]);
            if (S.cnt[15 + t]) atomicAdd(&d.stats[14 + t], S.cnt[15 + t]);
        }
        if (g.count_unique) {
            unsigned long long u = S.cnt[11];
            for (int b = 0; b < S.n_blk; ++b)
                for (int j = 0; j < S.un[b]; ++j) u += (unsigned long long)(S.uiv[b * kIv + j].y - S.uiv[b * kIv + j].x);
            if (u) atomicAdd(&d.stats[17], u);
        }
    }
}


// both parts, for kernels without dependency waits
template <bool STAGE, bool MEAN, bool PAIR, bool LAT>
__device__ __forceinline__ void region_phase(const Geo& g, const Dev& d, int cell, long long sweep, Sm& S,
                                             unsigned char* smem) {
    if (region_begin<STAGE, LAT>(g, d, cell, sweep, S, smem)) region_rest<STAGE, MEAN, PAIR, LAT>(g, d, cell, sweep, S);
}

// one colour phase: a CTA per region of the colour
template <bool STAGE, bool MEAN, bool PAIR, bool LAT>
__global__ void __launch_bounds__(kThreads32, kMinBlocks32) phase32_kernel(const __grid_constant__ Geo g,
                                                                           const __grid_constant__ Dev d, int colour) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    if ((int)blockIdx.x >= d.colour_count[colour]) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Sm S;
    init_staging<STAGE>(S);
    region_phase<STAGE, MEAN, PAIR, LAT>(g, d, d.colour_cells[colour * g.max_rpc + blockIdx.x], sweep, S, smem);
}

__device__ __forceinline__ long long ld_acquire(const long long* p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(long long* p, long long v) {
    asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}


// All colour phases of one sweep in one persistent launch.  Regions are
// taken from a queue in colour order (colour 0's regions first, each
// colour's in its list order); a region waits only until its neighbouring
// regions of lower colours have finished this sweep (the regions whose
// blankets share stations with its own), then runs its phase.  A region of
// a higher colour waits for it in turn, so every region sees its
// neighbours' state exactly as in the colour-by-colour schedule, and the
// results do not depend on the order in which CTAs take regions.  Every
// region a CTA waits for was taken earlier by a CTA that is running, so the
// waits end; they are bounded all the same (CMH_ERR_TIMEOUT).
template <bool STAGE, bool MEAN, bool PAIR, bool LAT>
__global__ void __launch_bounds__(kThreads32, kMinBlocks32) sweep32_kernel(const __grid_constant__ Geo g,
                                                                           const __grid_constant__ Dev d) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Sm S;
    __shared__ int s_cell, s_run;
    __shared__ long long s_sweep;
    init_staging<STAGE>(S);
    for (;;) {
        // thread 0 takes the next region and broadcasts it (-1: none left)
        if (threadIdx.x == 0) {
            const int total = d.colour_off[g.n_colours];
            const int it = *(volatile int*)d.status ? total : atomicAdd(d.queue, 1);
            int colour = 0, cell = -1;
            if (it < total) {
                while (colour + 1 < g.n_colours && it >= d.colour_off[colour + 1]) ++colour;
                cell = d.colour_cells[colour * g.max_rpc + (it - d.colour_off[colour])];
            }
            s_cell = cell;
            s_sweep = *d.sweep;
            s_run = colour;
        }
        __syncthreads();
        const int cell = s_cell;
        if (cell < 0) break;
        const long long sweep = s_sweep, stamp = sweep + 1;
        const int colour_taken = s_run;
        // the part of the region's phase that needs no neighbour runs while
        // the lower-colour neighbours may still be running theirs
        const bool begun = region_begin<STAGE, LAT>(g, d, cell, sweep, S, smem);
        if (threadIdx.x == 0) {
            const int colour = colour_taken;
            const int P1 = g.period - 1, ix = cell % g.ncx, iy = cell / g.ncx;
            for (int jy = iy - P1; jy <= iy + P1; ++jy)
                for (int jx = ix - P1; jx <= ix + P1; ++jx) {
                    if (jx < 0 || jy < 0 || jx >= g.ncx || jy >= g.ncy) continue;
                    const int nb = jy * g.ncx + jx;
                    const int c = d.cell_col[nb];
                    if (nb == cell || c < 0 || c >= colour) continue;
                    unsigned n = 0;
                    while (ld_acquire(d.done + nb) < stamp && !*(volatile int*)d.status) {
                        if (++n >= g.dep_wait_limit) {
                            latch(d.status, CMH_ERR_TIMEOUT);
                            break;
                        }
                        __nanosleep(128);
                    }
                }
            if (STAGE) fence_async_global();   // the neighbours' V writes before any bulk copy of them
            s_run = begun && *(volatile int*)d.status == 0;
        }
        __syncthreads();
        if (s_run) region_rest<STAGE, MEAN, PAIR, LAT>(g, d, cell, sweep, S);
        __syncthreads();
        if (threadIdx.x == 0 && cell != g.hold_cell) {
            __threadfence();
            st_release(d.done + cell, stamp);
        }
    }
}

// ---- a batch of independent instances ------------------------------------
// The queue holds every instance's regions in colour order across instances:
// item_tab[c * n_inst + i] is the first item of (colour c, instance i) and
// item_tab[n_col * n_inst] the number of items.  Dependencies stay inside an
// instance (lower colours come earlier in the queue), so the argument of the
// single-instance kernel carries over.
__global__ void __launch_bounds__(1024) batch_plan(const Geo* G, const Dev* D, int n_inst, int n_col, int* item_tab,
                                                   int* queue) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int n = n_col * n_inst, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int e = base + threadIdx.x;
        int v = 0;
        if (e < n) {
            const int c = e / n_inst, i = e % n_inst;
            if (c < G[i].n_colours && *(volatile int*)D[i].status == 0) v = D[i].colour_count[c];
        }
        int x = v;   // block inclusive scan
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = lane < nwarp ? s_warp[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nwarp) s_warp[lane] = w;
        }
        __syncthreads();
        const int excl = s_carry + (wid ? s_warp[wid - 1] : 0) + x - v;
        if (e < n) item_tab[e] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        item_tab[n] = s_carry;
        *queue = 0;
    }
}

template <bool MEAN>
__global__ void __launch_bounds__(kThreads32, kMinBlocks32) sweep32_batch(const Geo* G, const Dev* D, int n_inst,
                                                                          int n_col, const int* item_tab,
                                                                          int* queue) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Sm S;
    __shared__ int s_inst, s_cell, s_col, s_run;
    __shared__ long long s_sweep;
    init_staging<false>(S);
    for (;;) {
        if (threadIdx.x == 0) {
            const int n = n_col * n_inst, total = item_tab[n];
            const int it = atomicAdd(queue, 1);
            int inst = -1, col = 0, cell = -1;
            if (it < total) {
                int lo = 0, hi = n - 1;   // largest entry whose first item is <= it
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (item_tab[mid] <= it) lo = mid; else hi = mid - 1;
                }
                col = lo / n_inst;
                inst = lo % n_inst;
                cell = D[inst].colour_cells[col * G[inst].max_rpc + (it - item_tab[lo])];
                s_sweep = *D[inst].sweep;
            }
            s_inst = inst;
            s_cell = cell;
            s_col = col;
        }
        __syncthreads();
        const int inst = s_inst, cell = s_cell;
        if (inst < 0) break;
        const Geo& g = G[inst];
        const Dev& d = D[inst];
        const long long sweep = s_sweep, stamp = sweep + 1;
        const bool begun = region_begin<false, false>(g, d, cell, sweep, S, smem);
        if (threadIdx.x == 0) {
            const int colour = s_col;
            const int P1 = g.period - 1, ix = cell % g.ncx, iy = cell / g.ncx;
            for (int jy = iy - P1; jy <= iy + P1; ++jy)
                for (int jx = ix - P1; jx <= ix + P1; ++jx) {
                    if (jx < 0 || jy < 0 || jx >= g.ncx || jy >= g.ncy) continue;
                    const int nb = jy * g.ncx + jx;
                    const int c = d.cell_col[nb];
                    if (nb == cell || c < 0 || c >= colour) continue;
                    unsigned k = 0;
                    while (ld_acquire(d.done + nb) < stamp && !*(volatile int*)d.status) {
                        if (++k >= g.dep_wait_limit) {
                            latch(d.status, CMH_ERR_TIMEOUT);
                            break;
                        }
                        __nanosleep(128);
                    }
                }
            s_run = begun && *(volatile int*)d.status == 0;
        }
        __syncthreads();
        if (s_run) region_rest<false, MEAN, false, false>(g, d, cell, sweep, S);
        __syncthreads();
        if (threadIdx.x == 0 && cell != g.hold_cell) {
            __threadfence();
            st_release(d.done + cell, stamp);
        }
    }
}

}  // namespace

size_t phase32_smem_bytes(const Geo& g) { return layout32(g, nullptr, nullptr); }

size_t phase32_spill_bytes(const Geo& g) {
    Geo h = g;
    h.spill = 1;
    size_t go = 0;
    layout32(h, nullptr, nullptr, nullptr, &go);
    return go;
}

cudaError_t prepare_sweep32_batch(size_t smem_bytes, int* grid) {
    cudaError_t e = raise_smem_limit((const void*)sweep32_batch<false>, smem_bytes);
    if (e == cudaSuccess) e = raise_smem_limit((const void*)sweep32_batch<true>, smem_bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 1, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep32_batch<false>, kThreads32, smem_bytes)))
        return e;
    *grid = std::max(1, n_sm * std::max(1, std::min(per_sm, kMinBlocks32)));
    return cudaSuccess;
}

cudaError_t launch_sweep32_batch(bool mean, const Geo* G, const Dev* D, int n_inst, int n_col, int* item_tab,
                                 int* queue,
                                 size_t smem_bytes, int grid, cudaStream_t s) {
    batch_plan<<<1, 1024, 0, s>>>(G, D, n_inst, n_col, item_tab, queue);
    if (mean)
        sweep32_batch<true><<<grid, kThreads32, smem_bytes, s>>>(G, D, n_inst, n_col, item_tab, queue);
    else
        sweep32_batch<false><<<grid, kThreads32, smem_bytes, s>>>(G, D, n_inst, n_col, item_tab, queue);
    return cudaGetLastError();
}

// staging capacity (samples per buffer): 0 for `requested` 0 (no staging);
// `requested` rounded down to a multiple of 4 when positive; for -1, one
// arrival window (a move's shift included), cut down to what keeps the CTAs
// of one colour phase resident in a single wave (at most kMinBlocks32 per SM;
// none when fewer than 64 samples fit).  Windows that do not fit are read
// from global memory.
cudaError_t choose_stage_cap(Geo& g, int requested) {
    g.stage_cap = 0;
    if (requested == 0 || g.p_pair > 0.0 || g.sig_a > 0.0) return cudaSuccess;
    if (requested > 0) {
        g.stage_cap = requested & ~3;
        return cudaSuccess;
    }
    int dev = 0, per_sm = 0, reserved = 0, n_sm = 1, optin = 0;
    cudaError_t e;
    cudaFuncAttributes fa;
    if ((e = cudaGetDevice(&dev)) ||
        (e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) ||
        (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) ||
        (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) ||
        (e = cudaFuncGetAttributes(&fa, phase32_kernel<true, false, false, false>)))
        return e;
    const int resident = std::min(kMinBlocks32, std::max(1, (g.max_rpc + n_sm - 1) / std::max(1, n_sm)));
    const long long dyn = (long long)layout32(g, nullptr, nullptr);
    long long budget = (long long)per_sm / resident - reserved - (long long)fa.sharedSizeBytes - dyn;
    budget = std::min(budget, (long long)optin - (long long)fa.sharedSizeBytes - dyn);
    const long long want = (((long long)g.n_w + 3) & ~3LL) + 64;
    long long cap = budget > 0 ? (budget / 16) & ~3LL : 0;
    if (cap > want) cap = want;
    g.stage_cap = cap >= 64 ? (int)cap : 0;
    return cudaSuccess;
}

// the kernels of a model: one per staging x likelihood reading, the
// instantiation with joint moves of a pair (no staging, variance reading),
// and the one with latent arrival offsets and the arrival-time move (joint
// moves too), so that kernels without them carry none of their code
const void* sweep32_func(const Geo& g) {
    if (g.sig_a > 0.0) return (const void*)sweep32_kernel<false, false, true, true>;
    if (g.p_pair > 0.0) return (const void*)sweep32_kernel<false, false, true, false>;
    if (g.stage_cap > 0)
        return g.mean_mode ? (const void*)sweep32_kernel<true, true, false, false> : (const void*)sweep32_kernel<true, false, false, false>;
    return g.mean_mode ? (const void*)sweep32_kernel<false, true, false, false> : (const void*)sweep32_kernel<false, false, false, false>;
}

const void* phase32_func(const Geo& g) {
    if (g.sig_a > 0.0) return (const void*)phase32_kernel<false, false, true, true>;
    if (g.p_pair > 0.0) return (const void*)phase32_kernel<false, false, true, false>;
    if (g.stage_cap > 0)
        return g.mean_mode ? (const void*)phase32_kernel<true, true, false, false> : (const void*)phase32_kernel<true, false, false, false>;
    return g.mean_mode ? (const void*)phase32_kernel<false, true, false, false> : (const void*)phase32_kernel<false, false, false, false>;
}

cudaError_t prepare_phase32(const Geo& g) {
    const int bytes = (int)phase32_smem_bytes(g);
    cudaError_t e;
    const bool mn = g.mean_mode;
    if (g.sig_a > 0.0 || g.p_pair > 0.0) {
        if ((e = raise_smem_limit(phase32_func(g), bytes)) || (e = raise_smem_limit(sweep32_func(g), bytes))) return e;
        return cudaSuccess;
    }
    if ((e = raise_smem_limit(mn ? (const void*)phase32_kernel<false, true, false, false> : (const void*)phase32_kernel<false, false, false, false>,
                              bytes)) ||
        (e = raise_smem_limit(mn ? (const void*)phase32_kernel<true, true, false, false> : (const void*)phase32_kernel<true, false, false, false>,
                              bytes)) ||
        (e = raise_smem_limit(mn ? (const void*)sweep32_kernel<false, true, false, false> : (const void*)sweep32_kernel<false, false, false, false>,
                              bytes)) ||
        (e = raise_smem_limit(mn ? (const void*)sweep32_kernel<true, true, false, false> : (const void*)sweep32_kernel<true, false, false, false>,
                              bytes)))
        return e;
    return cudaSuccess;
}
cudaError_t sweep32_grid(const Geo& g, int ctas_per_sm, int* grid) {
    int dev = 0, n_sm = 1, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)))
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep32_func(g), kThreads32, phase32_smem_bytes(g))))
        return e;
    per_sm = std::max(1, std::min(per_sm, kMinBlocks32));
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    *grid = std::max(1, std::min(n_sm * per_sm, g.n_colours * g.max_rpc));
    return cudaSuccess;
}

cudaError_t launch_sweep32(const Geo& g, const Dev& d, int grid, cudaStream_t s) {
    const size_t smem = phase32_smem_bytes(g);
    if (g.sig_a > 0.0)
        sweep32_kernel<false, false, true, true><<<grid, kThreads32, smem, s>>>(g, d);
    else if (g.p_pair > 0.0)
        sweep32_kernel<false, false, true, false><<<grid, kThreads32, smem, s>>>(g, d);
    else if (g.stage_cap > 0)
        g.mean_mode ? sweep32_kernel<true, true, false, false><<<grid, kThreads32, smem, s>>>(g, d)
                    : sweep32_kernel<true, false, false, false><<<grid, kThreads32, smem, s>>>(g, d);
    else
        g.mean_mode ? sweep32_kernel<false, true, false, false><<<grid, kThreads32, smem, s>>>(g, d)
                    : sweep32_kernel<false, false, false, false><<<grid, kThreads32, smem, s>>>(g, d);
    return cudaGetLastError();
}
cudaError_t launch_phase32(const Geo& g, const Dev& d, int colour, cudaStream_t s) {
    const size_t smem = phase32_smem_bytes(g);
    if (g.sig_a > 0.0)
        phase32_kernel<false, false, true, true><<<g.max_rpc, kThreads32, smem, s>>>(g, d, colour);
    else if (g.p_pair > 0.0)
        phase32_kernel<false, false, true, false><<<g.max_rpc, kThreads32, smem, s>>>(g, d, colour);
    else if (g.stage_cap > 0)
        g.mean_mode ? phase32_kernel<true, true, false, false><<<g.max_rpc, kThreads32, smem, s>>>(g, d, colour)
                    : phase32_kernel<true, false, false, false><<<g.max_rpc, kThreads32, smem, s>>>(g, d, colour);
    else
        g.mean_mode ? phase32_kernel<false, true, false, false><<<g.max_rpc, kThreads32, smem, s>>>(g, d, colour)
                    : phase32_kernel<false, false, false, false><<<g.max_rpc, kThreads32, smem, s>>>(g, d, colour);
    return cudaGetLastError();
}

}  // namespace cmh
