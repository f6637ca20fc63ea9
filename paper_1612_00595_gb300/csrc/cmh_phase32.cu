// Colour-phase kernel, float32 throughput form (Algorithm "Chromatic MH with
// Static Coloring": every region of one colour runs k MH steps in parallel
// with the other regions fixed).  One CTA per region.
//
// The state stays float64 (the event masters), but within a phase every
// per-step test runs in float32 on cell-relative coordinates:
//   * "does the event reach station j" (distance < R_max),
//   * "which sample does its window start at" (ceil(arrival x f)),
//   * "is the moved event still in the region / domain / time range".
// Each float32 test has a margin about 10x its worst-case rounding error; a
// value inside the margin is decided by the exact float64 expression of the
// float64 master coordinates instead.  So every integer decision is the one
// the float64 definition gives, while the float64 pipe (1/64 of the float32
// rate on this part) is used only for the accept decision and for master
// updates on accept.  Per-sample likelihood terms are float32 with Kahan sums
// per thread, float-float (TwoSum) warp-shuffle reductions and a float64
// result.
#include <cuda_runtime.h>
#include <math.h>

#include "cmh_common.cuh"

namespace cmh {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float kDr = 2e-3f;   // km: margin of the region tests
constexpr float kDm = 1e-5f;   // magnitude units: margin of the m >= 2 test
constexpr int kThreads32 = 256;
constexpr int kMaxTasks32 = 64;

struct A32 {            // arrival of an event at a blanket slot
    int slot, k0;
    float E0;           // log2 of the variance added at sample k0
    int pad;
};

struct F32a {           // an arrival in a list (frozen neighbours, others of a task)
    int k0;
    float E0;
};

struct D32 {            // state-independent part of one MH step
    double bx, by, bt, bm, blb;   // birth: float64 candidate and its log beta
    float xr, yr, ph, mf;         // birth: relative form; move: offsets dx, dy, dt (s), dm
    float logu;
    unsigned pickw;
    int type, bK, bvalid, pad;
};

struct T32 {            // one station whose variance the proposal changes
    int row, slot, lo, hi;
    int has_o, has_n, k0o, k0n;
    float E0o, E0n;
    int oth0, noth;
};

struct L32 {
    size_t mx, my, mt, mm, id, xr, yr, ph, mf, K, narr, arr, order, freel, tabB, tabD;
    size_t bsta, bx, by, fcnt, farr, draws, cand, tasks, pool;
    size_t nx, ny, nt, nmm, nxr, nyr, nph, nmf, nK, total;
    int pool_cap;
    __host__ __device__ L32(const Geo& g) {
        pool_cap = g.ev_cap + g.frz_cap;
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 15) & ~size_t(15); return r; };
        const size_t E = g.ev_cap;
        mx = take(8 * E); my = take(8 * E); mt = take(8 * E); mm = take(8 * E); id = take(8 * E);
        xr = take(4 * E); yr = take(4 * E); ph = take(4 * E); mf = take(4 * E); K = take(4 * E);
        narr = take(4 * E);
        arr = take(sizeof(A32) * E * g.arr_cap);
        order = take(4 * E); freel = take(4 * E);
        tabB = take(8 * (E + 1)); tabD = take(8 * (E + 1));
        bsta = take(4 * (size_t)g.blk_cap);
        bx = take(8 * (size_t)g.blk_cap); by = take(8 * (size_t)g.blk_cap);
        fcnt = take(4 * (size_t)g.blk_cap);
        farr = take(sizeof(F32a) * (size_t)g.blk_cap * g.frz_cap);
        draws = take(sizeof(D32) * (size_t)g.k);
        cand = take(sizeof(A32) * (size_t)g.arr_cap);
        tasks = take(sizeof(T32) * kMaxTasks32);
        pool = take(sizeof(F32a) * (size_t)pool_cap);
        // one neighbouring cell's events at a time (frozen arrivals)
        nx = take(8 * E); ny = take(8 * E); nt = take(8 * E); nmm = take(8 * E);
        nxr = take(4 * E); nyr = take(4 * E); nph = take(4 * E); nmf = take(4 * E); nK = take(4 * E);
        total = o;
    }
};

// an event in cell-relative float form plus its float64 master
struct P32 {
    float xr, yr, ph, mf;
    int K;
    double x, y, t, m;
};

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

// ordered append across the block (see cmh_sweep.cu)
__device__ __forceinline__ int block_append32(bool flag, int* s_warp, int* s_base) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(FULL, flag);
    if (lane == 0) s_warp[wid] = __popc(bal);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < nw; ++w) {
        const int c = s_warp[w];
        if (w < wid) before += c;
        all += c;
    }
    const int pos = *s_base + before + __popc(bal & ((1u << lane) - 1));
    __syncthreads();
    if (threadIdx.x == 0) *s_base += all;
    __syncthreads();
    return pos;
}

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

// relative float form of a float64 event (region tests) and its float32 terms
__device__ __forceinline__ void to_rel(const Geo& g, double X0, double Y0, double x, double y, double t, double m,
                                       float& xr, float& yr, float& ph, float& mf, int& K) {
    xr = (float)__dsub_rn(x, X0);
    yr = (float)__dsub_rn(y, Y0);
    event_terms32(g, t, m, K, ph, mf);
}

__global__ void __launch_bounds__(kThreads32, 3) phase32_kernel(Geo g, Dev d, int colour) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    if ((int)blockIdx.x >= d.colour_count[colour]) return;
    const int cell = d.colour_cells[colour * g.max_rpc + blockIdx.x];
    const Store S = d.st[sweep & 1];
    const double sx = d.shift[0], sy = d.shift[1];
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int ix = cell % g.ncx, iy = cell / g.ncx;

    extern __shared__ __align__(16) unsigned char smem[];
    const L32 Lo(g);
    double* mx = (double*)(smem + Lo.mx);
    double* my = (double*)(smem + Lo.my);
    double* mt = (double*)(smem + Lo.mt);
    double* mm = (double*)(smem + Lo.mm);
    unsigned long long* eid = (unsigned long long*)(smem + Lo.id);
    float* exr = (float*)(smem + Lo.xr);
    float* eyr = (float*)(smem + Lo.yr);
    float* eph = (float*)(smem + Lo.ph);
    float* emf = (float*)(smem + Lo.mf);
    int* eK = (int*)(smem + Lo.K);
    int* enarr = (int*)(smem + Lo.narr);
    A32* earr = (A32*)(smem + Lo.arr);
    int* order = (int*)(smem + Lo.order);
    int* freel = (int*)(smem + Lo.freel);
    double* tabB = (double*)(smem + Lo.tabB);
    double* tabD = (double*)(smem + Lo.tabD);
    int* bsta = (int*)(smem + Lo.bsta);
    double* bx = (double*)(smem + Lo.bx);
    double* by = (double*)(smem + Lo.by);
    int* fcnt = (int*)(smem + Lo.fcnt);
    F32a* farr = (F32a*)(smem + Lo.farr);
    D32* draws = (D32*)(smem + Lo.draws);
    A32* cand = (A32*)(smem + Lo.cand);
    T32* tasks = (T32*)(smem + Lo.tasks);
    F32a* pool = (F32a*)(smem + Lo.pool);
    double* nx = (double*)(smem + Lo.nx);
    double* ny = (double*)(smem + Lo.ny);
    double* nt = (double*)(smem + Lo.nt);
    double* nmm = (double*)(smem + Lo.nmm);
    float* nxr = (float*)(smem + Lo.nxr);
    float* nyr = (float*)(smem + Lo.nyr);
    float* nph = (float*)(smem + Lo.nph);
    float* nmf = (float*)(smem + Lo.nmf);
    int* nK = (int*)(smem + Lo.nK);

    __shared__ double s_rect[4], s_X0, s_Y0, s_region_dlp;
    __shared__ float s_rl[4];   // region in relative coordinates: x lo, x hi, y lo, y hi
    __shared__ int s_n_own, s_n_free, s_n_blk, s_err, s_valid, s_idx, s_type, s_ncand, s_ntask, s_acc;
    __shared__ int s_warp[32], s_base;
    __shared__ float2 s_redf[32];
    __shared__ P32 s_cand;

    const int start = S.start[cell], n0 = S.count[cell];
    if (tid == 0) {
        cell_rect(g, sx, sy, cell, s_rect);
        s_X0 = __dadd_rn(sx, __dmul_rn((double)(ix - 1), g.L));
        s_Y0 = __dadd_rn(sy, __dmul_rn((double)(iy - 1), g.L));
        s_rl[0] = (float)(s_rect[0] - s_X0);
        s_rl[1] = (float)(s_rect[1] - s_X0);
        s_rl[2] = (float)(s_rect[2] - s_Y0);
        s_rl[3] = (float)(s_rect[3] - s_Y0);
        s_err = (n0 + g.k > g.ev_cap) ? CMH_ERR_CAPACITY : 0;
        s_n_own = n0;
        s_n_free = g.ev_cap - n0;
        s_base = 0;
        s_region_dlp = 0.0;
    }
    __syncthreads();
    if (s_err) {
        if (tid == 0) latch(d.status, s_err);
        return;
    }
    const double X0 = s_X0, Y0 = s_Y0;
    // ---- own events: masters, relative form, free list --------------------------
    for (int i = tid; i < g.ev_cap; i += nthr) {
        if (i < n0) {
            const double x = S.x[start + i], y = S.y[start + i], t = S.t[start + i], m = S.m[start + i];
            mx[i] = x; my[i] = y; mt[i] = t; mm[i] = m;
            eid[i] = S.id[start + i];
            to_rel(g, X0, Y0, x, y, t, m, exr[i], eyr[i], eph[i], emf[i], eK[i]);
            order[i] = i;
        } else {
            freel[g.ev_cap - 1 - i] = i;
        }
    }
    // ---- acceptance constants: log(beta / q_b) = log(Lambda area / W^2) ----------
    {
        const double area = (s_rect[1] - s_rect[0]) * (s_rect[3] - s_rect[2]);
        const double Cb = g.Cb0 + (double)logf((float)area);
        for (int n = tid; n <= g.ev_cap; n += nthr) {
            tabB[n] = Cb - d.log_n[n + 1];
            tabD[n] = n > 0 ? -Cb + d.log_n[n] : 0.0;
        }
    }
    // ---- blanket: stations within R_max of the region (float test, margin) ------
    {
        const float r0 = (float)s_rect[0], r1 = (float)s_rect[1], r2 = (float)s_rect[2], r3 = (float)s_rect[3];
        const float Rm = g.R_f * 1.0001f + 1e-3f;
        for (int base = 0; base < g.n_st; base += nthr) {
            const int j = base + tid;
            bool in = false;
            if (j < g.n_st) {
                const float fx = d.stxf[j], fy = d.styf[j];
                const float dx = fx < r0 ? r0 - fx : (fx > r1 ? fx - r1 : 0.f);
                const float dy = fy < r2 ? r2 - fy : (fy > r3 ? fy - r3 : 0.f);
                in = dx * dx + dy * dy < Rm * Rm;
            }
            const int pos = block_append32(in, s_warp, &s_base);
            if (in) {
                if (pos < g.blk_cap) {
                    const double xs = d.stx[j], ys = d.sty[j];
                    bsta[pos] = j;
                    bx[pos] = xs;
                    by[pos] = ys;
                } else {
                    atomicCAS(&s_err, 0, CMH_ERR_CAPACITY);
                }
            }
        }
        __syncthreads();
        if (tid == 0) s_n_blk = min(s_base, g.blk_cap);
        __syncthreads();
    }
    const int n_blk = s_n_blk;
    // ---- arrival cache of the own events -----------------------------------------
    for (int i = tid; i < n0; i += nthr) {
        int na = 0;
        for (int b = 0; b < n_blk; ++b) {
            int k0;
            float E0;
            if (arrival32c(g, mx[i], my[i], mt[i], eK[i], eph[i], emf[i], bx[b], by[b], k0, E0)) {
                if (na < g.arr_cap) earr[i * g.arr_cap + na] = A32{b, k0, E0, 0};
                ++na;
            }
        }
        if (na > g.arr_cap) atomicCAS(&s_err, 0, CMH_ERR_CAPACITY);
        enarr[i] = min(na, g.arr_cap);
    }
    // ---- frozen arrivals: neighbouring cells (other colours), in (cell, id) order -
    for (int b = tid; b < n_blk; b += nthr) fcnt[b] = 0;
    {
        const int P1 = g.period - 1;
        for (int jy = iy - P1; jy <= iy + P1; ++jy) {
            for (int jx = ix - P1; jx <= ix + P1; ++jx) {
                if (jx < 0 || jy < 0 || jx >= g.ncx || jy >= g.ncy) continue;
                const int oc = jy * g.ncx + jx;
                if (oc == cell) continue;
                const int s0 = S.start[oc], nn = S.count[oc];
                if (nn == 0) continue;
                __syncthreads();   // previous cell's list fully consumed
                if (nn > g.ev_cap) {
                    if (tid == 0) s_err = CMH_ERR_CAPACITY;
                    break;
                }
                for (int i = tid; i < nn; i += nthr) {
                    const double x = S.x[s0 + i], y = S.y[s0 + i], t = S.t[s0 + i], m = S.m[s0 + i];
                    nx[i] = x; ny[i] = y; nt[i] = t; nmm[i] = m;
                    to_rel(g, X0, Y0, x, y, t, m, nxr[i], nyr[i], nph[i], nmf[i], nK[i]);
                }
                __syncthreads();
                for (int b = tid; b < n_blk; b += nthr) {
                    int nf = fcnt[b];
                    for (int i = 0; i < nn; ++i) {
                        int k0;
                        float E0;
                        if (arrival32c(g, nx[i], ny[i], nt[i], nK[i], nph[i], nmf[i], bx[b], by[b], k0, E0)) {
                            if (nf < g.frz_cap) farr[b * g.frz_cap + nf] = F32a{k0, E0};
                            ++nf;
                        }
                    }
                    if (nf > g.frz_cap) atomicCAS(&s_err, 0, CMH_ERR_CAPACITY);
                    fcnt[b] = min(nf, g.frz_cap);
                }
            }
        }
    }
    // ---- the k steps' random draws (Philox stream 0, counter (sweep, cell, step, 0|1))
    const unsigned long long thr_b = (unsigned long long)ceil(g.p_birth * 9007199254740992.0);
    const unsigned long long thr_d = (unsigned long long)ceil(__dadd_rn(g.p_birth, g.p_death) * 9007199254740992.0);
    for (int st = tid; st < g.k; st += nthr) {
        unsigned long long c0[4] = {(unsigned long long)sweep, (unsigned long long)cell, (unsigned long long)st, 0ULL};
        unsigned long long c1[4] = {(unsigned long long)sweep, (unsigned long long)cell, (unsigned long long)st, 1ULL};
        philox4x64(c0, g.seed, 0ULL);
        philox4x64(c1, g.seed, 0ULL);
        D32 D;
        const unsigned long long u53 = c0[0] >> 11;   // u < p  <=>  u53 < p 2^53 (p 2^53 rounded up)
        D.type = u53 < thr_b ? 0 : (u53 < thr_d ? 1 : 2);
        D.pickw = (unsigned)(c0[1] & 0xffffffffULL);
        D.logu = __logf(u32o(c1[2]));
        D.bvalid = 0;
        D.bK = 0;
        D.bx = D.by = D.bt = D.bm = D.blb = 0.0;
        if (D.type == 0) {
            const double x = __dadd_rn(s_rect[0], __dmul_rn(u01(c0[2]), __dsub_rn(s_rect[1], s_rect[0])));
            const double y = __dadd_rn(s_rect[2], __dmul_rn(u01(c0[3]), __dsub_rn(s_rect[3], s_rect[2])));
            const double t = __dmul_rn(u01(c1[0]), g.T);
            const double m = mag_from_u53(c1[1]);
            D.bx = x; D.by = y; D.bt = t; D.bm = m;
            D.blb = g.lb0 - m;
            D.bvalid = x >= 0.0 && x < g.W && y >= 0.0 && y < g.W && cell_of(g, sx, sy, x, y) == cell &&
                       t >= 0.0 && t < g.T && m >= 2.0;
            to_rel(g, X0, Y0, x, y, t, m, D.xr, D.yr, D.ph, D.mf, D.bK);
        } else if (D.type == 2) {
            const float u2 = (float)(c0[3] >> 40) * (1.0f / 16777216.0f);
            const float u4 = (float)(c1[1] >> 40) * (1.0f / 16777216.0f);
            const float r1 = sqrtf(-2.f * __logf(u32o(c0[2]))), r2 = sqrtf(-2.f * __logf(u32o(c1[0])));
            float s1, co1, s2, co2;
            __sincosf(6.2831853071795865f * u2, &s1, &co1);
            __sincosf(6.2831853071795865f * u4, &s2, &co2);
            float z[4] = {r1 * co1, r1 * s1, r2 * co2, r2 * s2};
            const float sg[4] = {(float)g.sig_xy, (float)g.sig_xy, (float)g.sig_t, (float)g.sig_m};
            for (int i = 0; i < 4; ++i) {
                float q = rintf(fabsf(z[i]) * 1048576.f) * (1.f / 1048576.f);
                if ((c0[1] >> (32 + i)) & 1ULL) q = -q;
                z[i] = sg[i] * q;
            }
            D.xr = z[0]; D.yr = z[1]; D.ph = z[2]; D.mf = z[3];
        } else {
            D.xr = D.yr = D.ph = D.mf = 0.f;
        }
        draws[st] = D;
    }
    __syncthreads();
    if (s_err) {
        if (tid == 0) latch(d.status, s_err);
        return;
    }

    unsigned long long n_prop[3] = {0, 0, 0}, n_eval[3] = {0, 0, 0}, n_acc[3] = {0, 0, 0};
    unsigned long long n_priced = 0, n_rewritten = 0;

    for (int step = 0; step < g.k; ++step) {
        // ===================== control (warp 0) =====================
        if (wid == 0) {
            const D32& dr = draws[step];
            const int n_own = s_n_own;
            int valid = 0, idx = -1, ps = -1;
            P32 c;
            c.xr = c.yr = c.ph = c.mf = 0.f;
            c.K = 0;
            c.x = c.y = c.t = c.m = 0.0;
            if (dr.type == 0) {
                valid = dr.bvalid;
                c.xr = dr.xr; c.yr = dr.yr; c.ph = dr.ph; c.mf = dr.mf; c.K = dr.bK;
                c.x = dr.bx; c.y = dr.by; c.t = dr.bt; c.m = dr.bm;
            } else if (n_own > 0) {
                idx = pick32(dr.pickw, n_own);
                ps = order[idx];
                if (dr.type == 1) {
                    valid = 1;
                } else {
                    // masters of the candidate (what the state becomes on accept), their
                    // float32 terms, and region-relative coordinates for the region test
                    c.x = __dadd_rn(mx[ps], (double)dr.xr);
                    c.y = __dadd_rn(my[ps], (double)dr.yr);
                    c.t = __dadd_rn(mt[ps], (double)dr.ph);
                    c.m = __dadd_rn(mm[ps], (double)dr.mf);
                    event_terms32(g, c.t, c.m, c.K, c.ph, c.mf);
                    c.xr = exr[ps] + dr.xr;
                    c.yr = eyr[ps] + dr.yr;
                    // region, domain, time, magnitude: float test, exact inside the margins
                    const bool xin = c.xr >= s_rl[0] + kDr && c.xr < s_rl[1] - kDr;
                    const bool yin = c.yr >= s_rl[2] + kDr && c.yr < s_rl[3] - kDr;
                    const bool xout = c.xr < s_rl[0] - kDr || c.xr >= s_rl[1] + kDr;
                    const bool yout = c.yr < s_rl[2] - kDr || c.yr >= s_rl[3] + kDr;
                    const bool tin = c.K >= 1 && c.K + 2 <= g.TfK;
                    const bool min_ = c.mf >= 2.f + kDm;
                    const bool mout = c.mf < 2.f - kDm;
                    if (xout || yout || mout) {
                        valid = 0;
                    } else if (xin && yin && tin && min_) {
                        valid = 1;
                    } else {
                        valid = c.x >= 0.0 && c.x < g.W && c.y >= 0.0 && c.y < g.W &&
                                cell_of(g, sx, sy, c.x, c.y) == cell && c.t >= 0.0 && c.t < g.T && c.m >= 2.0;
                        if (valid) to_rel(g, X0, Y0, c.x, c.y, c.t, c.m, c.xr, c.yr, c.ph, c.mf, c.K);
                    }
                }
            }
            // candidate arrivals, lanes over blanket slots, compacted in slot order
            int ncand = 0;
            if (valid && dr.type != 1) {
                for (int b0 = 0; b0 < n_blk; b0 += 32) {
                    const int b = b0 + lane;
                    int k0 = 0;
                    float E0 = 0.f;
                    const bool r = b < n_blk && arrival32c(g, c.x, c.y, c.t, c.K, c.ph, c.mf, bx[b], by[b], k0, E0);
                    const unsigned bal = __ballot_sync(FULL, r);
                    const int pos = ncand + __popc(bal & ((1u << lane) - 1));
                    if (r && pos < g.arr_cap) cand[pos] = A32{b, k0, E0, 0};
                    ncand += __popc(bal);
                }
            }
            __syncwarp();
            int err = ncand > g.arr_cap ? CMH_ERR_CAPACITY : 0;
            int ntask = 0, npool = 0;
            if (valid && !err) {
                const A32* oa = (ps >= 0 && dr.type != 0) ? earr + ps * g.arr_cap : nullptr;
                const int no = oa ? enarr[ps] : 0;
                const int nnw = dr.type != 1 ? ncand : 0;
                int io = 0, in = 0;
                while (io < no || in < nnw) {
                    const int so = io < no ? oa[io].slot : 1 << 30;
                    const int sn = in < nnw ? cand[in].slot : 1 << 30;
                    if (ntask >= kMaxTasks32) { err = CMH_ERR_CAPACITY; break; }
                    T32 T;
                    T.slot = so < sn ? so : sn;
                    T.row = bsta[T.slot];
                    T.has_o = so <= sn;
                    T.has_n = sn <= so;
                    T.k0o = T.k0n = 0;
                    T.E0o = T.E0n = 0.f;
                    int lo = 1 << 30, hi = -1;
                    if (T.has_o) {
                        const A32 A = oa[io++];
                        T.k0o = A.k0; T.E0o = A.E0;
                        lo = min(lo, A.k0);
                        hi = max(hi, A.k0 + g.n_w);
                    }
                    if (T.has_n) {
                        const A32 A = cand[in++];
                        T.k0n = A.k0; T.E0n = A.E0;
                        lo = min(lo, A.k0);
                        hi = max(hi, A.k0 + g.n_w);
                    }
                    lo = max(lo, 0);
                    hi = (long long)hi > g.n_samp ? (int)g.n_samp : hi;
                    T.lo = lo;
                    T.hi = hi;
                    T.oth0 = npool;
                    T.noth = 0;
                    if (lo < hi) {
                        if (lane == 0) tasks[ntask] = T;
                        ++ntask;
                    }
                }
                __syncwarp();
                // others lists of every task: own events except the changed one, then
                // frozen neighbours, each covering part of [lo, hi), in order
                for (int ti = 0; ti < ntask && !err; ++ti) {
                    const int slot = tasks[ti].slot, lo = tasks[ti].lo, hi = tasks[ti].hi;
                    const int o0 = npool;
                    for (int q0 = 0; q0 < n_own; q0 += 32) {
                        const int q = q0 + lane;
                        bool hit = false;
                        F32a A = {0, 0.f};
                        if (q < n_own) {
                            const int p2 = order[q];
                            if (p2 != ps) {
                                for (int a = 0; a < enarr[p2]; ++a) {
                                    const A32& B = earr[p2 * g.arr_cap + a];
                                    if (B.slot == slot && B.k0 + g.n_w > lo && B.k0 < hi) {
                                        hit = true;
                                        A = F32a{B.k0, B.E0};
                                    }
                                }
                            }
                        }
                        const unsigned bal = __ballot_sync(FULL, hit);
                        const int pos = npool + __popc(bal & ((1u << lane) - 1));
                        if (hit && pos < Lo.pool_cap) pool[pos] = A;
                        npool += __popc(bal);
                    }
                    for (int a0 = 0; a0 < fcnt[slot]; a0 += 32) {
                        const int a = a0 + lane;
                        bool hit = false;
                        F32a A = {0, 0.f};
                        if (a < fcnt[slot]) {
                            A = farr[slot * g.frz_cap + a];
                            hit = A.k0 + g.n_w > lo && A.k0 < hi;
                        }
                        const unsigned bal = __ballot_sync(FULL, hit);
                        const int pos = npool + __popc(bal & ((1u << lane) - 1));
                        if (hit && pos < Lo.pool_cap) pool[pos] = A;
                        npool += __popc(bal);
                    }
                    if (npool > Lo.pool_cap) err = CMH_ERR_CAPACITY;
                    if (lane == 0) {
                        tasks[ti].oth0 = o0;
                        tasks[ti].noth = min(npool, Lo.pool_cap) - o0;
                    }
                }
            }
            if (lane == 0) {
                s_err = err;
                s_valid = valid;
                s_idx = idx;
                s_type = dr.type;
                s_ncand = ncand;
                s_ntask = ntask;
                s_cand = c;
            }
        }
        __syncthreads();
        if (s_err) break;
        const int valid = s_valid, ntask = s_ntask;

        // ===================== pricing (all threads) =====================
        if (valid) {
            float acc = 0.f, comp = 0.f;
            for (int ti = 0; ti < ntask; ++ti) {
                const T32& T = tasks[ti];
                const float* srow = (const float*)d.sig + (size_t)T.row * g.pitch;
                const float* vrow = (const float*)d.V + (size_t)T.row * g.pitch;
                for (int q = (T.lo >> 2) + tid; (q << 2) < T.hi; q += nthr) {
                    const int k = q << 2;
                    const float4 s4 = __ldg(reinterpret_cast<const float4*>(srow + k));
                    const float4 v4 = *reinterpret_cast<const float4*>(vrow + k);
                    const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
                    const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int kk = k + e;
                        const int ro = kk - T.k0o, rn = kk - T.k0n;
                        const bool io = T.has_o && (unsigned)ro < (unsigned)g.n_w;
                        const bool inn = T.has_n && (unsigned)rn < (unsigned)g.n_w;
                        // the same per-sample values the variance synthesis adds, so the
                        // priced change is the change written to V on accept
                        const float co = io ? arr_var32(g, T.E0o, ro) : 0.f;
                        const float cn = inn ? arr_var32(g, T.E0n, rn) : 0.f;
                        const float dd = cn - co;
                        if (kk < T.hi && dd != 0.f) {
                            const float V = vv[e], s = sv[e];
                            const float Vp = V + dd;
                            float term;
                            if (Vp < 0.5f * V) {
                                // the changed arrival dominates V: rebuild V' from the others
                                float a2 = g.noise_f, c2 = 0.f;
                                for (int o = 0; o < T.noth; ++o) {
                                    const F32a A = pool[T.oth0 + o];
                                    const int r = kk - A.k0;
                                    if ((unsigned)r < (unsigned)g.n_w) kahan_add32(a2, c2, arr_var32(g, A.E0, r));
                                }
                                if (inn) kahan_add32(a2, c2, cn);
                                const float Vr = a2 - c2;
                                term = logf(Vr / V) + s * s * (1.f / Vr - 1.f / V);
                            } else {
                                term = log1pf(dd / V) - s * s * dd / (V * Vp);
                            }
                            kahan_add32(acc, comp, -0.5f * term);
                        }
                    }
                }
            }
            float2 v = make_float2(acc, -comp);
            for (int o = 16; o > 0; o >>= 1) {
                float2 w2;
                w2.x = __shfl_xor_sync(FULL, v.x, o);
                w2.y = __shfl_xor_sync(FULL, v.y, o);
                v = ff_add32(v, w2);
            }
            if (lane == 0) s_redf[wid] = v;
            __syncthreads();
        }

        // ===================== decision (thread 0, float64) =====================
        if (tid == 0) {
            const int type = s_type, n_own = s_n_own;
            const D32& dr = draws[step];
            ++n_prop[type];
            double dll = 0.0, la = -INFINITY, dlp = 0.0;
            int acc = 0;
            if (valid) {
                ++n_eval[type];
                for (int ti = 0; ti < ntask; ++ti) n_priced += (unsigned long long)(tasks[ti].hi - tasks[ti].lo);
                float2 t = s_redf[0];
                for (int w = 1; w < (nthr >> 5); ++w) t = ff_add32(t, s_redf[w]);
                dll = (double)t.x + (double)t.y;
                if (type == 0) {
                    la = dll + tabB[n_own];
                    dlp = dr.blb;
                } else if (type == 1) {
                    la = dll + tabD[n_own];
                    dlp = mm[order[s_idx]] - g.lb0;
                } else {
                    const double dm = __dsub_rn(s_cand.m, mm[order[s_idx]]);
                    la = dll - dm;
                    dlp = -dm;
                }
                acc = (double)dr.logu < la;
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
            if (acc) ++n_acc[type];
            if (do_commit) {
                for (int ti = 0; ti < ntask; ++ti) n_rewritten += (unsigned long long)(tasks[ti].hi - tasks[ti].lo);
                s_region_dlp += dll + dlp;
                const P32 c = s_cand;
                int ps;
                if (type == 1) {
                    ps = order[s_idx];
                    for (int q = s_idx; q + 1 < n_own; ++q) order[q] = order[q + 1];
                    freel[s_n_free++] = ps;
                    s_n_own = n_own - 1;
                } else {
                    if (type == 0) {
                        ps = freel[--s_n_free];
                        eid[ps] = ((unsigned long long)(sweep + 1) << 32) | ((unsigned long long)cell << 12) |
                                  (unsigned long long)step;
                        order[n_own] = ps;
                        s_n_own = n_own + 1;
                    } else {
                        ps = order[s_idx];
                    }
                    mx[ps] = c.x; my[ps] = c.y; mt[ps] = c.t; mm[ps] = c.m;
                    exr[ps] = c.xr; eyr[ps] = c.yr; eph[ps] = c.ph; emf[ps] = c.mf; eK[ps] = c.K;
                    for (int a = 0; a < s_ncand; ++a) earr[ps * g.arr_cap + a] = cand[a];
                    enarr[ps] = s_ncand;
                }
            }
            s_acc = do_commit;
        }
        __syncthreads();

        // ===================== commit: re-synthesise V on the touched windows ======
        if (s_acc) {
            const bool has_new_type = s_type != 1;
            for (int ti = 0; ti < ntask; ++ti) {
                const T32& T = tasks[ti];
                const bool has_new = has_new_type && T.has_n;
                float* vrow = (float*)d.V + (size_t)T.row * g.pitch;
                for (int kk = T.lo + tid; kk < T.hi; kk += nthr) {
                    float a2 = g.noise_f, c2 = 0.f;
                    for (int o = 0; o < T.noth; ++o) {
                        const F32a A = pool[T.oth0 + o];
                        const int r = kk - A.k0;
                        if ((unsigned)r < (unsigned)g.n_w) kahan_add32(a2, c2, arr_var32(g, A.E0, r));
                    }
                    if (has_new) {
                        const int r = kk - T.k0n;
                        if ((unsigned)r < (unsigned)g.n_w) kahan_add32(a2, c2, arr_var32(g, T.E0n, r));
                    }
                    vrow[kk] = a2 - c2;
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    if (s_err) {
        if (tid == 0) latch(d.status, s_err);
        return;
    }
    const int n_fin = s_n_own;
    for (int i = tid; i < n_fin; i += nthr) {
        const int ps = order[i];
        S.x[start + i] = mx[ps];
        S.y[start + i] = my[ps];
        S.t[start + i] = mt[ps];
        S.m[start + i] = mm[ps];
        S.id[start + i] = eid[ps];
    }
    if (tid == 0) {
        S.count[cell] = n_fin;
        d.region_dlp[cell] = s_region_dlp;
        for (int t = 0; t < 3; ++t) {
            if (n_prop[t]) atomicAdd(&d.stats[t], n_prop[t]);
            if (n_eval[t]) atomicAdd(&d.stats[3 + t], n_eval[t]);
            if (n_acc[t]) atomicAdd(&d.stats[6 + t], n_acc[t]);
        }
        if (n_priced) atomicAdd(&d.stats[9], n_priced);
        if (n_rewritten) atomicAdd(&d.stats[10], n_rewritten);
    }
}

}  // namespace

size_t phase32_smem_bytes(const Geo& g) { return L32(g).total; }

cudaError_t prepare_phase32(const Geo& g) {
    return cudaFuncSetAttribute(phase32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)phase32_smem_bytes(g));
}

cudaError_t launch_phase32(const Geo& g, const Dev& d, int colour, cudaStream_t s) {
    phase32_kernel<<<g.max_rpc, kThreads32, phase32_smem_bytes(g), s>>>(g, d, colour);
    return cudaGetLastError();
}

}  // namespace cmh
