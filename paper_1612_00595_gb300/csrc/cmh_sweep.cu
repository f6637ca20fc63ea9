// Colour-phase kernel of chromatic Metropolis-Hastings in float64 (the replay
// form that reproduces the CPU oracle step for step; the float32 throughput
// form is cmh_phase32.cu), plus the predicted-variance synthesis and the
// log-density reduction.  (Algorithm "Chromatic MH with Static Coloring": for
// one colour, every region of that colour runs k MH steps in parallel with
// all other regions fixed.)
//
// One CTA per region of the active colour.  Within a CTA:
//   * warp 0 is the control warp: it decodes each step's proposal (birth,
//     death, Gaussian move, and with p_pair > 0 the joint move of a pair of
//     events; §Generative Model of Seismic Signals, the MH moves), finds the
//     stations the proposal reaches and makes the float64 accept decision
//     (MH rule, §Background);
//   * all warps price the proposal: the change of the Gaussian
//     log-likelihood over the samples whose variance changes (§Generative
//     Model: zero-mean diagonal Gaussian with variance = noise + arriving
//     signals' variances), reduced with warp shuffles;
//   * on accept all warps re-synthesise the predicted variance V over the
//     touched windows from the arrivals that cover them.
// Same-colour regions have disjoint Markov blankets (the partition guarantees
// it), so no two CTAs of a launch touch the same station row of V.
#include <cuda_runtime.h>
#include <math.h>

#include "cmh_common.cuh"

namespace cmh {

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct EvArr {          // one arrival of an own event at a blanket station
    int slot, k0;       // blanket slot, first sample of the window
    double af, lnA2;    // arrival time x f, 2 (alpha m - beta_att d)
};

struct Arr {            // an arrival in a list (frozen neighbours, others of a task)
    int k0, pad;
    double af, lnA2;
};

struct Draw {           // state-independent part of one MH step
    double a[4];        // birth: candidate (x, y, t, m); move, pair: signed offsets; arrival: a[0] the step
    double logu;        // log of the accept uniform, (0, 1]
    unsigned pickw;     // low word for the event pick
    unsigned pickw2;    // joint move: low word for the second event's pick
    int type;           // 0 birth, 1 death, 2 move, 3 joint move of a pair, 4 arrival-time move
    int bvalid;         // birth candidate inside region, time and magnitude range
    int sub;            // joint move: 0 exchange of locations, 1 common offset
    int pad;
};

struct Task {           // one station whose variance the proposal changes
    int row, slot, lo, hi;
    int has_o, has_n, k0o, k0n;
    int oth0;           // others list: [oth0, oth0 + noth) in the pool
    int noth;
    int has_o2, has_n2, k0o2, k0n2;   // joint move: the second event's old and new arrivals
    double afo, lnA2o, afn, lnA2n, rm1d;
    double afo2, lnA2o2, afn2, lnA2n2;
};

// shared-memory layout of the phase kernel (host computes the size)
struct Layout {
    size_t ev_x, ev_y, ev_t, ev_m, ev_id, ev_narr, ev_arr, order, freel;
    size_t b_sta, b_x, b_y, f_cnt, f_arr, draws, cand, tasks, pool, eoff, coff, total;
    int task_cap;       // a task per distinct blanket slot of the changed arrivals
    int pool_cap;
    __host__ __device__ Layout(const Geo& g) {
        const int lists = g.p_pair > 0.0 ? 4 : 2;   // old and new arrivals of one or two events
        task_cap = g.blk_cap < lists * g.arr_cap ? g.blk_cap : lists * g.arr_cap;
        if (task_cap < 1) task_cap = 1;
        pool_cap = (g.ev_cap + g.frz_cap) * (lists / 2);
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 15) & ~size_t(15); return r; };
        ev_x = take(sizeof(double) * g.ev_cap);
        ev_y = take(sizeof(double) * g.ev_cap);
        ev_t = take(sizeof(double) * g.ev_cap);
        ev_m = take(sizeof(double) * g.ev_cap);
        ev_id = take(sizeof(unsigned long long) * g.ev_cap);
        ev_narr = take(sizeof(int) * g.ev_cap);
        ev_arr = take(sizeof(EvArr) * (size_t)g.ev_cap * g.arr_cap);
        order = take(sizeof(int) * g.ev_cap);
        freel = take(sizeof(int) * g.ev_cap);
        b_sta = take(sizeof(int) * g.blk_cap);
        b_x = take(sizeof(double) * g.blk_cap);
        b_y = take(sizeof(double) * g.blk_cap);
        f_cnt = take(sizeof(int) * g.blk_cap);
        f_arr = take(sizeof(Arr) * (size_t)g.blk_cap * g.frz_cap);
        draws = take(sizeof(Draw) * g.k);
        cand = take(sizeof(EvArr) * 2 * g.arr_cap);   // the candidate's arrivals; a pair's second at arr_cap
        tasks = take(sizeof(Task) * task_cap);
        pool = take(sizeof(Arr) * (size_t)pool_cap);
        // latent arrival offsets by blanket slot: own events' [ev_cap][blk_cap],
        // the candidates' [2][blk_cap] (0 where not reached)
        const size_t lat = g.sig_a > 0.0 ? 1 : 0;
        eoff = take(sizeof(double) * (size_t)g.ev_cap * g.blk_cap * lat);
        coff = take(sizeof(double) * 2 * (size_t)g.blk_cap * lat);
        total = o;
    }
};

// arrival of an event at a station: a = t + d/v, plus the latent offset
// delta of that (event, station) when arrivals are latent (sig_a > 0)
__device__ __forceinline__ bool arrival(const Geo& g, double x, double y, double t, double m, double xs,
                                        double ys, int& k0, double& af, double& lnA2, double delta = 0.0) {
    const double dd = dist_rn(x, y, xs, ys);
    if (!(dd < g.R_max)) return false;
    double a = __dadd_rn(t, __ddiv_rn(dd, g.v));
    if (g.sig_a > 0.0) a = __dadd_rn(a, delta);
    af = __dmul_rn(a, g.f_hz);
    k0 = (int)ceil(af);
    lnA2 = 2.0 * (g.alpha * m - g.beta_att * dd);
    return true;
}

// variance added at sample k by an arrival (float64 form)
__device__ __forceinline__ double arr_c64(const Geo& g, double af, double lnA2, int k) {
    return exp(lnA2 - ((double)k - af) * (2.0 / (g.f_hz * g.tau)));
}

// log(1 + x): for |x| < 1/16 the Taylor series sum (-1)^(n+1) x^n / n through
// n = 13 in Horner form (truncation below |x|^14 / 14, under 2e-18 relative),
// else the library's log1p.  Most priced samples lie in an arrival's tail,
// where x = d / V is small.
__device__ __forceinline__ double log1p_series64(double x) {
    if (fabs(x) < 0.0625) {
        double p = 1.0 / 13.0;
        p = fma(p, x, -1.0 / 12.0);
        p = fma(p, x, 1.0 / 11.0);
        p = fma(p, x, -1.0 / 10.0);
        p = fma(p, x, 1.0 / 9.0);
        p = fma(p, x, -1.0 / 8.0);
        p = fma(p, x, 1.0 / 7.0);
        p = fma(p, x, -1.0 / 6.0);
        p = fma(p, x, 1.0 / 5.0);
        p = fma(p, x, -1.0 / 4.0);
        p = fma(p, x, 1.0 / 3.0);
        p = fma(p, x, -0.5);
        p = fma(p, x, 1.0);
        return p * x;
    }
    return log1p(x);
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// ordered append across the block: returns the position of this thread's
// element among the flagged ones of this pass; *total (shared) is advanced
__device__ __forceinline__ int block_append(bool flag, int* s_warp, int* s_base) {
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

__global__ void __launch_bounds__(512, 1) phase_kernel(Geo g, Dev d, int colour) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    if ((int)blockIdx.x >= d.colour_count[colour]) return;
    const int cell = d.colour_cells[colour * g.max_rpc + blockIdx.x];
    const Store S = d.st[sweep & 1];
    const double sx = d.shift[0], sy = d.shift[1];
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5;

    extern __shared__ __align__(16) unsigned char smem[];
    const Layout Lo(g);
    double* ex = (double*)(smem + Lo.ev_x);
    double* ey = (double*)(smem + Lo.ev_y);
    double* et = (double*)(smem + Lo.ev_t);
    double* em = (double*)(smem + Lo.ev_m);
    unsigned long long* eid = (unsigned long long*)(smem + Lo.ev_id);
    int* enarr = (int*)(smem + Lo.ev_narr);
    EvArr* earr = (EvArr*)(smem + Lo.ev_arr);
    int* order = (int*)(smem + Lo.order);
    int* freel = (int*)(smem + Lo.freel);
    int* bsta = (int*)(smem + Lo.b_sta);
    double* bx = (double*)(smem + Lo.b_x);
    double* by = (double*)(smem + Lo.b_y);
    int* fcnt = (int*)(smem + Lo.f_cnt);
    Arr* farr = (Arr*)(smem + Lo.f_arr);
    Draw* draws = (Draw*)(smem + Lo.draws);
    EvArr* cand = (EvArr*)(smem + Lo.cand);
    Task* tasks = (Task*)(smem + Lo.tasks);
    Arr* pool = (Arr*)(smem + Lo.pool);
    double* eoff = (double*)(smem + Lo.eoff);
    double* coff = (double*)(smem + Lo.coff);
    const bool lat = g.sig_a > 0.0;   // latent arrival offsets

    __shared__ double s_rect[4];
    __shared__ double s_log_area, s_dll, s_region_dlp;
    __shared__ double s_c[4], s_c2[4];
    __shared__ int s_n_own, s_n_free, s_n_blk, s_err, s_valid, s_idx, s_type, s_ncand, s_ntask, s_acc;
    __shared__ int s_idx2, s_ncand2, s_aslot;
    __shared__ int s_warp[32], s_base;
    __shared__ double s_redd[32];

    const int start = S.start[cell], n0 = S.count[cell];
    if (tid == 0) {
        cell_rect(g, sx, sy, cell, s_rect);
        s_log_area = log(__dmul_rn(__dsub_rn(s_rect[1], s_rect[0]), __dsub_rn(s_rect[3], s_rect[2])));
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
    // own events (physical slots 0..n0-1, order = identity), free list
    for (int i = tid; i < g.ev_cap; i += nthr) {
        if (i < n0) {
            ex[i] = S.x[start + i];
            ey[i] = S.y[start + i];
            et[i] = S.t[start + i];
            em[i] = S.m[start + i];
            eid[i] = S.id[start + i];
            order[i] = i;
        } else {
            freel[g.ev_cap - 1 - i] = i;  // pop from the top gives the lowest slot first
        }
    }
    // blanket: stations within R_max of the region (float32 test with a margin;
    // a superset is harmless, every reach test below is exact float64)
    {
        const float r0 = (float)s_rect[0], r1 = (float)s_rect[1], r2 = (float)s_rect[2], r3 = (float)s_rect[3];
        const float Rm = (float)g.R_max * 1.0001f + 1e-3f;
        for (int base = 0; base < g.n_st; base += nthr) {
            const int j = base + tid;
            bool in = false;
            double xs = 0.0, ys = 0.0;
            if (j < g.n_st) {
                xs = d.stx[j];
                ys = d.sty[j];
                const float fx = (float)xs, fy = (float)ys;
                const float dx = fx < r0 ? r0 - fx : (fx > r1 ? fx - r1 : 0.f);
                const float dy = fy < r2 ? r2 - fy : (fy > r3 ? fy - r3 : 0.f);
                in = dx * dx + dy * dy < Rm * Rm;
            }
            const int pos = block_append(in, s_warp, &s_base);
            if (in) {
                if (pos < g.blk_cap) {
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
    // own events' latent offsets by blanket slot (every station an own event
    // reaches is in the blanket)
    if (lat) {
        for (int q = tid; q < n0 * n_blk; q += nthr) {
            const int i = q / n_blk, b = q - i * n_blk;
            eoff[i * g.blk_cap + b] = S.off[(size_t)(start + i) * g.n_st + bsta[b]];
        }
        __syncthreads();
    }
    // arrival cache of the own events
    for (int i = tid; i < n0; i += nthr) {
        int na = 0;
        for (int b = 0; b < n_blk; ++b) {
            int k0;
            double af, lnA2;
            if (arrival(g, ex[i], ey[i], et[i], em[i], bx[b], by[b], k0, af, lnA2,
                        lat ? eoff[i * g.blk_cap + b] : 0.0)) {
                if (na < g.arr_cap) {
                    EvArr& A = earr[i * g.arr_cap + na];
                    A.slot = b; A.k0 = k0; A.af = af; A.lnA2 = lnA2;
                }
                ++na;
            }
        }
        if (na > g.arr_cap) atomicCAS(&s_err, 0, CMH_ERR_CAPACITY);
        enarr[i] = na;
    }
    // frozen arrivals: events of the neighbouring cells (other colours) that
    // reach each blanket station, in (cell, id) order
    for (int b = tid; b < n_blk; b += nthr) {
        const int ix = cell % g.ncx, iy = cell / g.ncx, P1 = g.period - 1;
        int nf = 0;
        for (int jy = iy - P1; jy <= iy + P1; ++jy) {
            if (jy < 0 || jy >= g.ncy) continue;
            for (int jx = ix - P1; jx <= ix + P1; ++jx) {
                if (jx < 0 || jx >= g.ncx) continue;
                const int oc = jy * g.ncx + jx;
                if (oc == cell) continue;
                const int s0 = S.start[oc], n = S.count[oc];
                for (int i = 0; i < n; ++i) {
                    int k0;
                    double af, lnA2;
                    if (arrival(g, S.x[s0 + i], S.y[s0 + i], S.t[s0 + i], S.m[s0 + i], bx[b], by[b], k0, af, lnA2,
                                lat ? S.off[(size_t)(s0 + i) * g.n_st + bsta[b]] : 0.0)) {
                        if (nf < g.frz_cap) {
                            Arr& A = farr[b * g.frz_cap + nf];
                            A.k0 = k0; A.af = af; A.lnA2 = lnA2;
                        }
                        ++nf;
                    }
                }
            }
        }
        if (nf > g.frz_cap) atomicCAS(&s_err, 0, CMH_ERR_CAPACITY);
        fcnt[b] = min(nf, g.frz_cap);
    }
    // the k steps' random draws and their state-independent decoding
    for (int st = tid; st < g.k; st += nthr) {
        unsigned long long w[8];
        unsigned long long c0[4] = {(unsigned long long)sweep, (unsigned long long)cell, (unsigned long long)st, 0ULL};
        philox4x64(c0, g.seed, 0ULL);
        unsigned long long c1[4] = {(unsigned long long)sweep, (unsigned long long)cell, (unsigned long long)st, 1ULL};
        philox4x64(c1, g.seed, 0ULL);
        for (int i = 0; i < 4; ++i) { w[i] = c0[i]; w[4 + i] = c1[i]; }
        Draw D;
        const double u = u01(w[0]);
        const double cd = __dadd_rn(g.p_birth, g.p_death), cp = __dadd_rn(cd, g.p_pair);
        const double ca = __dadd_rn(cp, g.p_arr);
        D.type = u < g.p_birth ? 0 : (u < cd ? 1 : (u < cp ? 3 : (u < ca ? 4 : 2)));
        D.pickw = (unsigned)(w[1] & 0xffffffffULL);
        D.pickw2 = (unsigned)(w[7] & 0xffffffffULL);
        D.sub = (int)((w[1] >> 36) & 1ULL);
        D.logu = log(u01o(w[6]));
        D.bvalid = 0;
        if (D.type == 0) {
            const double x = __dadd_rn(s_rect[0], __dmul_rn(u01(w[2]), __dsub_rn(s_rect[1], s_rect[0])));
            const double y = __dadd_rn(s_rect[2], __dmul_rn(u01(w[3]), __dsub_rn(s_rect[3], s_rect[2])));
            const double t = __dmul_rn(u01(w[4]), g.T);
            const double m = __dsub_rn(2.0, log(u01o(w[5])));
            D.a[0] = x; D.a[1] = y; D.a[2] = t; D.a[3] = m;
            D.bvalid = x >= 0.0 && x < g.W && y >= 0.0 && y < g.W && cell_of(g, sx, sy, x, y) == cell &&
                       t >= 0.0 && t < g.T && m >= 2.0;
        } else if (D.type == 2 || D.type == 3 || D.type == 4) {
            const double r1 = __dsqrt_rn(__dmul_rn(-2.0, log(u01o(w[2]))));
            const double th1 = __dmul_rn(6.283185307179586, u01(w[3]));
            const double r2 = __dsqrt_rn(__dmul_rn(-2.0, log(u01o(w[4]))));
            const double th2 = __dmul_rn(6.283185307179586, u01(w[5]));
            double z[4] = {__dmul_rn(r1, cos(th1)), __dmul_rn(r1, sin(th1)), __dmul_rn(r2, cos(th2)),
                           __dmul_rn(r2, sin(th2))};
            // the arrival-time move steps its offset by sig_da times the first Gaussian
            const double sig[4] = {D.type == 4 ? g.sig_da : g.sig_xy, g.sig_xy, g.sig_t, g.sig_m};
            for (int i = 0; i < 4; ++i) {
                double q = __dmul_rn(rint(__dmul_rn(fabs(z[i]), 1048576.0)), 1.0 / 1048576.0);
                if ((w[1] >> (32 + i)) & 1ULL) q = -q;
                D.a[i] = __dmul_rn(sig[i], q);
            }
        } else {
            D.a[0] = D.a[1] = D.a[2] = D.a[3] = 0.0;
        }
        draws[st] = D;
    }
    __syncthreads();
    if (s_err) {
        if (tid == 0) latch(d.status, s_err);
        return;
    }

    unsigned long long n_prop[5] = {0, 0, 0, 0, 0}, n_eval[5] = {0, 0, 0, 0, 0}, n_acc[5] = {0, 0, 0, 0, 0};
    unsigned long long n_priced = 0, n_rewritten = 0;   // sample terms (thread 0's tally)

    for (int step = 0; step < g.k; ++step) {
        // ---------------- control: decode, reach, tasks (warp 0) ----------------
        if (wid == 0) {
            const Draw dr = draws[step];
            const int n_own = s_n_own;
            int valid = 0, idx = -1, ncand = 0, idx2 = -1, ncand2 = 0, aslot = -1;
            double cx = 0.0, cy = 0.0, ct = 0.0, cm = 0.0;
            double cx2 = 0.0, cy2 = 0.0, ct2 = 0.0, cm2 = 0.0;   // joint move: the second event
            if (dr.type == 0) {
                valid = dr.bvalid;
                cx = dr.a[0]; cy = dr.a[1]; ct = dr.a[2]; cm = dr.a[3];
            } else if (dr.type == 3) {
                // joint move of an ordered pair of distinct events: exchange of
                // their locations (each keeps its time and magnitude), or one
                // common offset for both
                if (n_own >= 2) {
                    idx = pick32(dr.pickw, n_own);
                    const int j = pick32(dr.pickw2, n_own - 1);
                    idx2 = j + (j >= idx ? 1 : 0);
                    const int p1 = order[idx], p2 = order[idx2];
                    if (dr.sub == 0) {
                        cx = ex[p2]; cy = ey[p2]; ct = et[p1]; cm = em[p1];
                        cx2 = ex[p1]; cy2 = ey[p1]; ct2 = et[p2]; cm2 = em[p2];
                    } else {
                        cx = __dadd_rn(ex[p1], dr.a[0]);
                        cy = __dadd_rn(ey[p1], dr.a[1]);
                        ct = __dadd_rn(et[p1], dr.a[2]);
                        cm = __dadd_rn(em[p1], dr.a[3]);
                        cx2 = __dadd_rn(ex[p2], dr.a[0]);
                        cy2 = __dadd_rn(ey[p2], dr.a[1]);
                        ct2 = __dadd_rn(et[p2], dr.a[2]);
                        cm2 = __dadd_rn(em[p2], dr.a[3]);
                    }
                    valid = cx >= 0.0 && cx < g.W && cy >= 0.0 && cy < g.W &&
                            cell_of(g, sx, sy, cx, cy) == cell && ct >= 0.0 && ct < g.T && cm >= 2.0 &&
                            cx2 >= 0.0 && cx2 < g.W && cy2 >= 0.0 && cy2 < g.W &&
                            cell_of(g, sx, sy, cx2, cy2) == cell && ct2 >= 0.0 && ct2 < g.T && cm2 >= 2.0;
                }
            } else if (dr.type == 4) {
                // arrival-time move: one of the stations an event reaches
                // (its arrival list is in station order), its offset stepped
                if (n_own > 0) {
                    idx = pick32(dr.pickw, n_own);
                    const int ps = order[idx];
                    const int na = enarr[ps];
                    if (na > 0) {
                        aslot = earr[ps * g.arr_cap + pick32(dr.pickw2, na)].slot;
                        cx = ex[ps]; cy = ey[ps]; ct = et[ps]; cm = em[ps];
                        valid = 1;
                    }
                }
            } else if (n_own > 0) {
                idx = pick32(dr.pickw, n_own);
                if (dr.type == 1) {
                    valid = 1;
                } else {
                    const int ps = order[idx];
                    cx = __dadd_rn(ex[ps], dr.a[0]);
                    cy = __dadd_rn(ey[ps], dr.a[1]);
                    ct = __dadd_rn(et[ps], dr.a[2]);
                    cm = __dadd_rn(em[ps], dr.a[3]);
                    valid = cx >= 0.0 && cx < g.W && cy >= 0.0 && cy < g.W &&
                            cell_of(g, sx, sy, cx, cy) == cell && ct >= 0.0 && ct < g.T && cm >= 2.0;
                }
            }
            // latent offset of candidate e at blanket slot b (0 where it does not
            // reach): kept from the event it replaces where that one reached b,
            // else drawn from the prior
            auto cand_offset = [&](int e, int old_ps, double x, double y, int b) -> double {
                if (!(dist_rn(x, y, bx[b], by[b]) < g.R_max)) return 0.0;
                if (old_ps >= 0 && dist_rn(ex[old_ps], ey[old_ps], bx[b], by[b]) < g.R_max)
                    return eoff[old_ps * g.blk_cap + b];
                return draw_offset(g, sweep, cell, step, bsta[b], e);
            };
            if (valid && dr.type != 1) {
                const int old1 = dr.type == 0 ? -1 : order[idx];
                for (int b0 = 0; b0 < n_blk; b0 += 32) {
                    const int b = b0 + lane;
                    int k0 = 0;
                    double af = 0.0, lnA2 = 0.0, dl = 0.0;
                    if (lat && b < n_blk) {
                        if (dr.type == 4) {
                            dl = eoff[old1 * g.blk_cap + b];
                            if (b == aslot) dl = __dadd_rn(dl, dr.a[0]);
                        } else {
                            dl = cand_offset(0, old1, cx, cy, b);
                        }
                        coff[b] = dl;
                    }
                    const bool r = b < n_blk && arrival(g, cx, cy, ct, cm, bx[b], by[b], k0, af, lnA2, dl);
                    const unsigned bal = __ballot_sync(FULL, r);
                    const int pos = ncand + __popc(bal & ((1u << lane) - 1));
                    if (r && pos < g.arr_cap) {
                        EvArr& A = cand[pos];
                        A.slot = b; A.k0 = k0; A.af = af; A.lnA2 = lnA2;
                    }
                    ncand += __popc(bal);
                }
            }
            if (valid && dr.type == 3) {
                EvArr* cand2 = cand + g.arr_cap;
                const int old2 = order[idx2];
                for (int b0 = 0; b0 < n_blk; b0 += 32) {
                    const int b = b0 + lane;
                    int k0 = 0;
                    double af = 0.0, lnA2 = 0.0, dl = 0.0;
                    if (lat && b < n_blk) {
                        dl = cand_offset(1, old2, cx2, cy2, b);
                        coff[g.blk_cap + b] = dl;
                    }
                    const bool r = b < n_blk && arrival(g, cx2, cy2, ct2, cm2, bx[b], by[b], k0, af, lnA2, dl);
                    const unsigned bal = __ballot_sync(FULL, r);
                    const int pos = ncand2 + __popc(bal & ((1u << lane) - 1));
                    if (r && pos < g.arr_cap) {
                        EvArr& A = cand2[pos];
                        A.slot = b; A.k0 = k0; A.af = af; A.lnA2 = lnA2;
                    }
                    ncand2 += __popc(bal);
                }
            }
            __syncwarp();
            if (lane == 0) {
                int err = (ncand > g.arr_cap || ncand2 > g.arr_cap) ? CMH_ERR_CAPACITY : 0;
                int nt = 0, npool = 0;
                if (valid && !err && dr.type == 3) {
                    // merge the four slot-sorted lists: the two events' old
                    // arrivals and their candidates'
                    const int p1 = order[idx], p2 = order[idx2];
                    const EvArr* La[4] = {earr + p1 * g.arr_cap, earr + p2 * g.arr_cap, cand, cand + g.arr_cap};
                    const int Na[4] = {enarr[p1], enarr[p2], ncand, ncand2};
                    int hd[4] = {0, 0, 0, 0};
                    while (!err) {
                        int sl = 1 << 30;
                        for (int q = 0; q < 4; ++q)
                            if (hd[q] < Na[q] && La[q][hd[q]].slot < sl) sl = La[q][hd[q]].slot;
                        if (sl == 1 << 30) break;
                        if (nt >= Lo.task_cap) { err = CMH_ERR_CAPACITY; break; }
                        Task& T = tasks[nt];
                        T.slot = sl;
                        T.row = bsta[sl];
                        T.has_o = T.has_o2 = T.has_n = T.has_n2 = 0;
                        T.rm1d = 0.0;
                        long long lo = 1LL << 40, hi = -1;
                        for (int q = 0; q < 4; ++q) {
                            if (!(hd[q] < Na[q] && La[q][hd[q]].slot == sl)) continue;
                            const EvArr& A = La[q][hd[q]++];
                            if (q == 0) { T.has_o = 1; T.k0o = A.k0; T.afo = A.af; T.lnA2o = A.lnA2; }
                            if (q == 1) { T.has_o2 = 1; T.k0o2 = A.k0; T.afo2 = A.af; T.lnA2o2 = A.lnA2; }
                            if (q == 2) { T.has_n = 1; T.k0n = A.k0; T.afn = A.af; T.lnA2n = A.lnA2; }
                            if (q == 3) { T.has_n2 = 1; T.k0n2 = A.k0; T.afn2 = A.af; T.lnA2n2 = A.lnA2; }
                            lo = min(lo, (long long)A.k0);
                            hi = max(hi, (long long)A.k0 + g.n_w);
                        }
                        if (lo < 0) lo = 0;
                        if (hi > g.n_samp) hi = g.n_samp;
                        T.lo = (int)lo;
                        T.hi = (int)hi;
                        if (lo >= hi) continue;  // every window after the record
                        // the other arrivals covering [lo, hi): own events but
                        // the pair, then frozen neighbours
                        T.oth0 = npool;
                        const int n_own2 = s_n_own;
                        for (int q = 0; q < n_own2 && !err; ++q) {
                            const int pq = order[q];
                            if (pq == p1 || pq == p2) continue;
                            for (int a = 0; a < enarr[pq]; ++a) {
                                const EvArr& A = earr[pq * g.arr_cap + a];
                                if (A.slot != T.slot) continue;
                                if (A.k0 + g.n_w <= lo || A.k0 >= hi) continue;
                                if (npool >= Lo.pool_cap) { err = CMH_ERR_CAPACITY; break; }
                                Arr& B = pool[npool++];
                                B.k0 = A.k0; B.af = A.af; B.lnA2 = A.lnA2;
                            }
                        }
                        for (int a = 0; a < fcnt[T.slot] && !err; ++a) {
                            const Arr& A = farr[T.slot * g.frz_cap + a];
                            if (A.k0 + g.n_w <= lo || A.k0 >= hi) continue;
                            if (npool >= Lo.pool_cap) { err = CMH_ERR_CAPACITY; break; }
                            pool[npool++] = A;
                        }
                        T.noth = npool - T.oth0;
                        ++nt;
                    }
                } else if (valid && !err) {
                    // merge the old event's arrivals and the candidate's, by slot
                    const int ps = idx >= 0 ? order[idx] : -1;
                    const EvArr* oa = ps >= 0 && dr.type != 0 ? earr + ps * g.arr_cap : nullptr;
                    const int no = oa ? enarr[ps] : 0;
                    const int nn = dr.type != 1 ? ncand : 0;
                    int io = 0, in = 0;
                    while ((io < no || in < nn) && !err) {
                        const int so = io < no ? oa[io].slot : 1 << 30;
                        const int sn = in < nn ? cand[in].slot : 1 << 30;
                        if (nt >= Lo.task_cap) { err = CMH_ERR_CAPACITY; break; }
                        Task& T = tasks[nt];
                        T.slot = so < sn ? so : sn;
                        T.row = bsta[T.slot];
                        T.has_o = so <= sn;
                        T.has_n = sn <= so;
                        T.has_o2 = T.has_n2 = 0;
                        long long lo = 1LL << 40, hi = -1;
                        if (T.has_o) {
                            const EvArr& A = oa[io++];
                            T.k0o = A.k0; T.afo = A.af; T.lnA2o = A.lnA2;
                            lo = min(lo, (long long)A.k0);
                            hi = max(hi, (long long)A.k0 + g.n_w);
                        }
                        if (T.has_n) {
                            const EvArr& A = cand[in++];
                            T.k0n = A.k0; T.afn = A.af; T.lnA2n = A.lnA2;
                            lo = min(lo, (long long)A.k0);
                            hi = max(hi, (long long)A.k0 + g.n_w);
                        }
                        if (T.has_o && T.has_n) {
                            // c_new / c_old is constant over the overlap of the two windows
                            T.rm1d = expm1((T.lnA2n - T.lnA2o) + (T.afo - T.afn) * (-2.0 / (g.f_hz * g.tau)));
                        } else {
                            T.rm1d = 0.0;
                        }
                        if (lo < 0) lo = 0;
                        if (hi > g.n_samp) hi = g.n_samp;
                        T.lo = (int)lo;
                        T.hi = (int)hi;
                        if (lo >= hi) continue;  // window entirely after the record
                        // the other arrivals covering [lo, hi) at this station:
                        // own events except the changed one, then frozen neighbours
                        T.oth0 = npool;
                        const int n_own2 = s_n_own;
                        for (int q = 0; q < n_own2 && !err; ++q) {
                            const int p2 = order[q];
                            if (p2 == ps) continue;
                            for (int a = 0; a < enarr[p2]; ++a) {
                                const EvArr& A = earr[p2 * g.arr_cap + a];
                                if (A.slot != T.slot) continue;
                                if (A.k0 + g.n_w <= lo || A.k0 >= hi) continue;
                                if (npool >= Lo.pool_cap) { err = CMH_ERR_CAPACITY; break; }
                                Arr& B = pool[npool++];
                                B.k0 = A.k0; B.af = A.af; B.lnA2 = A.lnA2;
                            }
                        }
                        for (int a = 0; a < fcnt[T.slot] && !err; ++a) {
                            const Arr& A = farr[T.slot * g.frz_cap + a];
                            if (A.k0 + g.n_w <= lo || A.k0 >= hi) continue;
                            if (npool >= Lo.pool_cap) { err = CMH_ERR_CAPACITY; break; }
                            pool[npool++] = A;
                        }
                        T.noth = npool - T.oth0;
                        ++nt;
                    }
                }
                s_err = err;
                s_valid = valid;
                s_idx = idx;
                s_idx2 = idx2;
                s_aslot = aslot;
                s_type = dr.type;
                s_ncand = ncand;
                s_ncand2 = ncand2;
                s_ntask = nt;
                s_c[0] = cx; s_c[1] = cy; s_c[2] = ct; s_c[3] = cm;
                s_c2[0] = cx2; s_c2[1] = cy2; s_c2[2] = ct2; s_c2[3] = cm2;
            }
        }
        __syncthreads();
        if (s_err) break;
        const int valid = s_valid, ntask = s_ntask;

        // ---------------- pricing: all threads ----------------
        if (valid) {
            {
                double acc = 0.0;
                // a thread's samples are nthr apart: an arrival's contribution
                // at the next one is this one times rstep (one exp at the
                // first sample inside the window, then a product per sample)
                const double rstep = exp(-(double)nthr * (2.0 / (g.f_hz * g.tau)));
                if (s_type == 3) {
                    // joint move: on every sample inside one of the four
                    // windows, the resident variance changed by the two
                    // candidates' contributions less the two old ones (each a
                    // running envelope product along the thread's samples);
                    // where the change removes more than half of it, the new
                    // variance summed from scratch instead
                    for (int ti = 0; ti < ntask; ++ti) {
                        const Task& T = tasks[ti];
                        const double* srow = (const double*)d.sig + (size_t)T.row * g.pitch;
                        const double* vrow = (const double*)d.V + (size_t)T.row * g.pitch;
                        double co = -1.0, co2 = -1.0, cn = -1.0, cn2 = -1.0;   // < 0: not started
                        for (int kk = T.lo + tid; kk < T.hi; kk += nthr) {
                            const bool io = T.has_o && (unsigned)(kk - T.k0o) < (unsigned)g.n_w;
                            const bool io2 = T.has_o2 && (unsigned)(kk - T.k0o2) < (unsigned)g.n_w;
                            const bool in1 = T.has_n && (unsigned)(kk - T.k0n) < (unsigned)g.n_w;
                            const bool in2 = T.has_n2 && (unsigned)(kk - T.k0n2) < (unsigned)g.n_w;
                            if (io) co = co < 0.0 ? arr_c64(g, T.afo, T.lnA2o, kk) : co * rstep;
                            if (io2) co2 = co2 < 0.0 ? arr_c64(g, T.afo2, T.lnA2o2, kk) : co2 * rstep;
                            if (in1) cn = cn < 0.0 ? arr_c64(g, T.afn, T.lnA2n, kk) : cn * rstep;
                            if (in2) cn2 = cn2 < 0.0 ? arr_c64(g, T.afn2, T.lnA2n2, kk) : cn2 * rstep;
                            if (!(io || io2 || in1 || in2)) continue;
                            double dd = 0.0;
                            if (in1) dd += cn;
                            if (in2) dd += cn2;
                            if (io) dd -= co;
                            if (io2) dd -= co2;
                            const double V = vrow[kk], sv = __ldg(srow + kk);
                            const double Vp = V + dd;
                            if (Vp < 0.5 * V) {
                                double a2 = g.noise_var;
                                for (int o = 0; o < T.noth; ++o) {
                                    const Arr& A = pool[T.oth0 + o];
                                    if ((unsigned)(kk - A.k0) < (unsigned)g.n_w) a2 += arr_c64(g, A.af, A.lnA2, kk);
                                }
                                if (in1) a2 += arr_c64(g, T.afn, T.lnA2n, kk);
                                if (in2) a2 += arr_c64(g, T.afn2, T.lnA2n2, kk);
                                acc += -0.5 * (log(a2 / V) + sv * sv * (1.0 / a2 - 1.0 / V));
                            } else {
                                const double inv = 1.0 / (V * Vp);   // one division for both terms
                                acc += -0.5 * (log1p_series64(dd * Vp * inv) - sv * sv * dd * inv);
                            }
                        }
                    }
                } else
                for (int ti = 0; ti < ntask; ++ti) {
                    const Task& T = tasks[ti];
                    const double* srow = (const double*)d.sig + (size_t)T.row * g.pitch;
                    const double* vrow = (const double*)d.V + (size_t)T.row * g.pitch;
                    double co = -1.0, cn = -1.0;   // running contributions (< 0: not started)
                    for (int kk = T.lo + tid; kk < T.hi; kk += nthr) {
                        const int ro = kk - T.k0o, rn = kk - T.k0n;
                        const bool io = T.has_o && (unsigned)ro < (unsigned)g.n_w;
                        const bool inn = T.has_n && (unsigned)rn < (unsigned)g.n_w;
                        // each running value advances on every sample of its own window
                        if (io) co = co < 0.0 ? arr_c64(g, T.afo, T.lnA2o, kk) : co * rstep;
                        if (inn) cn = cn < 0.0 ? arr_c64(g, T.afn, T.lnA2n, kk) : cn * rstep;
                        double dd = 0.0;
                        if (io)
                            dd = inn ? co * T.rm1d : -co;
                        else if (inn)
                            dd = cn;
                        if (dd != 0.0) {
                            const double V = vrow[kk], s = __ldg(srow + kk);
                            const double Vp = V + dd;
                            if (Vp < 0.5 * V) {
                                double a2 = g.noise_var;
                                for (int o = 0; o < T.noth; ++o) {
                                    const Arr& A = pool[T.oth0 + o];
                                    const int r = kk - A.k0;
                                    if ((unsigned)r < (unsigned)g.n_w) a2 += arr_c64(g, A.af, A.lnA2, kk);
                                }
                                if (inn) a2 += arr_c64(g, T.afn, T.lnA2n, kk);
                                acc += -0.5 * (log(a2 / V) + s * s * (1.0 / a2 - 1.0 / V));
                            } else {
                                const double inv = 1.0 / (V * Vp);   // one division for both terms
                                acc += -0.5 * (log1p_series64(dd * Vp * inv) - s * s * dd * inv);
                            }
                        }
                    }
                }
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
                if (lane == 0) s_redd[wid] = acc;
                __syncthreads();
                if (tid == 0) {
                    double t = 0.0;
                    for (int w = 0; w < (nthr >> 5); ++w) t += s_redd[w];
                    s_dll = t;
                }
            }
        }

        // ---------------- decision (thread 0) ----------------
        if (tid == 0) {
            const int type = s_type;
            const int n_own = s_n_own;
            const Draw& dr = draws[step];
            ++n_prop[type];
            double dll = 0.0, la = -INFINITY, dlp = 0.0;
            int acc = 0;
            if (valid) {
                ++n_eval[type];
                for (int ti = 0; ti < s_ntask; ++ti) n_priced += (unsigned long long)(tasks[ti].hi - tasks[ti].lo);
                dll = s_dll;
                const double cm = s_c[3];
                if (type == 0) {
                    const double lb = g.log_Lambda - g.log_WWT - (cm - 2.0);
                    const double lq = -s_log_area - g.log_T - (cm - 2.0);
                    dlp = lb;
                    la = dll + dlp - lq + g.log_pd - d.log_n[n_own + 1] - g.log_pb;
                } else if (type == 1) {
                    const double me = em[order[s_idx]];
                    const double lb = g.log_Lambda - g.log_WWT - (me - 2.0);
                    const double lq = -s_log_area - g.log_T - (me - 2.0);
                    dlp = -lb;
                    la = dll + dlp + lq + g.log_pb - g.log_pd + d.log_n[n_own];
                } else if (type == 4) {
                    // symmetric step of one offset: its prior ratio
                    const double a = eoff[order[s_idx] * g.blk_cap + s_aslot], b = coff[s_aslot];
                    const double s2 = __dmul_rn(g.sig_a, g.sig_a);
                    dlp = __ddiv_rn(__dsub_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(2.0, s2));
                    la = dll + dlp;
                } else if (type == 3) {
                    // symmetric proposal: the prior ratio of the two events
                    const double me1 = em[order[s_idx]], me2 = em[order[s_idx2]];
                    const double lb1n = g.log_Lambda - g.log_WWT - (cm - 2.0);
                    const double lb1o = g.log_Lambda - g.log_WWT - (me1 - 2.0);
                    const double lb2n = g.log_Lambda - g.log_WWT - (s_c2[3] - 2.0);
                    const double lb2o = g.log_Lambda - g.log_WWT - (me2 - 2.0);
                    dlp = (lb1n - lb1o) + (lb2n - lb2o);
                    la = dll + dlp;
                } else {
                    const double me = em[order[s_idx]];
                    const double lb_new = g.log_Lambda - g.log_WWT - (cm - 2.0);
                    const double lb_old = g.log_Lambda - g.log_WWT - (me - 2.0);
                    dlp = lb_new - lb_old;
                    la = dll + dlp;
                }
                acc = dr.logu < la;
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
            int do_commit = acc && g.commit;
            if (do_commit) {
                ++n_acc[type];
                for (int ti = 0; ti < s_ntask; ++ti) n_rewritten += (unsigned long long)(tasks[ti].hi - tasks[ti].lo);
                // latent offsets drawn from (or dropped to) their prior cancel
                // from the ratio but still change the log-density
                double dlo = 0.0;
                if (lat) {
                    auto rowsum = [&](const double* row, const EvArr* L, int n) {
                        double t = 0.0;
                        for (int a = 0; a < n; ++a) t += log_off_prior1(g, row[L[a].slot]);
                        return t;
                    };
                    const int p1 = s_idx >= 0 ? order[s_idx] : -1;
                    if (type == 0) {
                        dlo = rowsum(coff, cand, s_ncand);
                    } else if (type == 1) {
                        dlo = -rowsum(eoff + p1 * g.blk_cap, earr + p1 * g.arr_cap, enarr[p1]);
                    } else if (type == 2) {
                        dlo = rowsum(coff, cand, s_ncand) - rowsum(eoff + p1 * g.blk_cap, earr + p1 * g.arr_cap, enarr[p1]);
                    } else if (type == 3) {
                        const int p2 = order[s_idx2];
                        dlo = (rowsum(coff, cand, s_ncand) -
                               rowsum(eoff + p1 * g.blk_cap, earr + p1 * g.arr_cap, enarr[p1])) +
                              (rowsum(coff + g.blk_cap, cand + g.arr_cap, s_ncand2) -
                               rowsum(eoff + p2 * g.blk_cap, earr + p2 * g.arr_cap, enarr[p2]));
                    }
                }
                s_region_dlp += dll + dlp + dlo;
                if (type == 0) {
                    const int ps = freel[--s_n_free];
                    ex[ps] = s_c[0]; ey[ps] = s_c[1]; et[ps] = s_c[2]; em[ps] = s_c[3];
                    eid[ps] = ((unsigned long long)(sweep + 1) << 32) | ((unsigned long long)cell << 12) |
                              (unsigned long long)step;
                    for (int a = 0; a < s_ncand; ++a) earr[ps * g.arr_cap + a] = cand[a];
                    enarr[ps] = s_ncand;
                    if (lat)
                        for (int b = 0; b < n_blk; ++b) eoff[ps * g.blk_cap + b] = coff[b];
                    order[n_own] = ps;
                    s_n_own = n_own + 1;
                } else if (type == 1) {
                    const int ps = order[s_idx];
                    for (int q = s_idx; q + 1 < n_own; ++q) order[q] = order[q + 1];
                    freel[s_n_free++] = ps;
                    s_n_own = n_own - 1;
                } else {
                    const int ps = order[s_idx];
                    ex[ps] = s_c[0]; ey[ps] = s_c[1]; et[ps] = s_c[2]; em[ps] = s_c[3];
                    for (int a = 0; a < s_ncand; ++a) earr[ps * g.arr_cap + a] = cand[a];
                    enarr[ps] = s_ncand;
                    if (lat)
                        for (int b = 0; b < n_blk; ++b) eoff[ps * g.blk_cap + b] = coff[b];
                    if (type == 3) {
                        const int p2 = order[s_idx2];
                        ex[p2] = s_c2[0]; ey[p2] = s_c2[1]; et[p2] = s_c2[2]; em[p2] = s_c2[3];
                        for (int a = 0; a < s_ncand2; ++a) earr[p2 * g.arr_cap + a] = cand[g.arr_cap + a];
                        enarr[p2] = s_ncand2;
                        if (lat)
                            for (int b = 0; b < n_blk; ++b) eoff[p2 * g.blk_cap + b] = coff[g.blk_cap + b];
                    }
                }
            } else if (acc) {
                ++n_acc[type];
            }
            s_acc = do_commit;
        }
        __syncthreads();

        // ---------------- commit: re-synthesise V over the touched windows ----------------
        if (s_acc) {
            const int type = s_type;
            for (int ti = 0; ti < ntask; ++ti) {
                const Task& T = tasks[ti];
                const bool has_new = type != 1 && T.has_n;
                const bool has_new2 = type == 3 && T.has_n2;
                {
                    double* vrow = (double*)d.V + (size_t)T.row * g.pitch;
                    for (int kk = T.lo + tid; kk < T.hi; kk += nthr) {
                        double a2 = g.noise_var;
                        for (int o = 0; o < T.noth; ++o) {
                            const Arr& A = pool[T.oth0 + o];
                            const int r = kk - A.k0;
                            if ((unsigned)r < (unsigned)g.n_w) a2 += arr_c64(g, A.af, A.lnA2, kk);
                        }
                        if (has_new) {
                            const int r = kk - T.k0n;
                            if ((unsigned)r < (unsigned)g.n_w) a2 += arr_c64(g, T.afn, T.lnA2n, kk);
                        }
                        if (has_new2) {
                            const int r = kk - T.k0n2;
                            if ((unsigned)r < (unsigned)g.n_w) a2 += arr_c64(g, T.afn2, T.lnA2n2, kk);
                        }
                        vrow[kk] = a2;
                    }
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
    // write the region's events back in order (ids stay sorted)
    const int n_fin = s_n_own;
    for (int i = tid; i < n_fin; i += nthr) {
        const int ps = order[i];
        S.x[start + i] = ex[ps];
        S.y[start + i] = ey[ps];
        S.t[start + i] = et[ps];
        S.m[start + i] = em[ps];
        S.id[start + i] = eid[ps];
    }
    if (lat) {
        // offsets rows of the written events: 0 but at the blanket stations
        for (int q = tid; q < n_fin * g.n_st; q += nthr) S.off[(size_t)start * g.n_st + q] = 0.0;
        __syncthreads();
        for (int q = tid; q < n_fin * n_blk; q += nthr) {
            const int i = q / n_blk, b = q - i * n_blk;
            S.off[(size_t)(start + i) * g.n_st + bsta[b]] = eoff[order[i] * g.blk_cap + b];
        }
    }
    if (tid == 0) {
        S.count[cell] = n_fin;
        d.region_dlp[cell] = s_region_dlp;
        for (int t = 0; t < 3; ++t) {
            if (n_prop[t]) atomicAdd(&d.stats[t], n_prop[t]);
            if (n_eval[t]) atomicAdd(&d.stats[3 + t], n_eval[t]);
            if (n_acc[t]) atomicAdd(&d.stats[6 + t], n_acc[t]);
        }
        if (n_prop[3]) atomicAdd(&d.stats[11], n_prop[3]);
        if (n_eval[3]) atomicAdd(&d.stats[12], n_eval[3]);
        if (n_acc[3]) atomicAdd(&d.stats[13], n_acc[3]);
        if (n_prop[4]) atomicAdd(&d.stats[14], n_prop[4]);
        if (n_eval[4]) atomicAdd(&d.stats[15], n_eval[4]);
        if (n_acc[4]) atomicAdd(&d.stats[16], n_acc[4]);
        if (n_priced) atomicAdd(&d.stats[9], n_priced);
        if (n_rewritten) atomicAdd(&d.stats[10], n_rewritten);
    }
}

__device__ __forceinline__ void sweep_end_body(const Geo& g, const Dev& d) {
    if (*d.status) return;
    __shared__ double s_part[32];
    double acc = 0.0;
    // fixed assignment and fixed tree: the sum does not depend on scheduling
    for (int c = threadIdx.x; c < g.n_cells; c += blockDim.x) {
        acc += d.region_dlp[c];
        d.region_dlp[c] = 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        *d.logp += t;
        *d.sweep += 1;
    }
}

__global__ void sweep_end(const __grid_constant__ Geo g, const __grid_constant__ Dev d) { sweep_end_body(g, d); }

// one block per instance of a batch
__global__ void sweep_end_batch(const Geo* G, const Dev* D) { sweep_end_body(G[blockIdx.x], D[blockIdx.x]); }

// ---------------------------------------------------------------------------
// predicted-variance synthesis: V_j[k] = noise + sum of the variances of the
// arrivals covering sample k, for every station (one block per station).
// Events come from a flat list (fx, fy, ft, fm)[0, *n) in canonical order;
// arrivals are gathered in list order, kSynthArr per pass, and applied tile
// by tile in that order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
constexpr int kSynthThreads = 256;
constexpr int kSynthArr = 512;
constexpr int kSynthTile = kSynthThreads * 8;

template <bool F32>
__global__ void __launch_bounds__(kSynthThreads) vsynth_kernel(Geo g, Dev d, const double* fx, const double* fy,
                                                               const double* ft, const double* fm, const int* n_ptr,
                                                               const double* foff) {
    const int j = blockIdx.x;
    const int n = *n_ptr;
    const double xs = d.stx[j], ys = d.sty[j];
    __shared__ int s_k0[kSynthArr];
    __shared__ double s_af[kSynthArr], s_ln[kSynthArr];
    __shared__ float s_E0[kSynthArr];
    __shared__ int s_tl[kSynthArr];
    __shared__ int s_warp[32], s_base, s_cnt, s_nt;
    int base = 0;
    bool first = true;
    while (true) {
        if (threadIdx.x == 0) s_base = 0;
        __syncthreads();
        while (base < n) {
            const int idx = base + threadIdx.x;
            int k0 = 0;
            double af = 0.0, ln = 0.0;
            float E0 = 0.f;
            bool r = false;
            if (idx < n) {
                if (F32) {
                    int K;
                    float ph, mf;
                    event_terms32(g, ft[idx], fm[idx], K, ph, mf);
                    r = foff ? arrival32c(g, fx[idx], fy[idx], ft[idx], K, ph, mf, xs, ys, k0, E0,
                                          foff[(size_t)idx * g.n_st + j])
                             : arrival32c(g, fx[idx], fy[idx], ft[idx], K, ph, mf, xs, ys, k0, E0);
                } else {
                    r = arrival(g, fx[idx], fy[idx], ft[idx], fm[idx], xs, ys, k0, af, ln,
                                foff ? foff[(size_t)idx * g.n_st + j] : 0.0);
                }
            }
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            if (r) atomicAdd(&s_cnt, 1);
            __syncthreads();
            if (s_base + s_cnt > kSynthArr) break;   // full: apply, then resume here
            const int pos = block_append(r, s_warp, &s_base);
            if (r) {
                s_k0[pos] = k0;
                s_af[pos] = af;
                s_ln[pos] = ln;
                s_E0[pos] = E0;
            }
            base += blockDim.x;
        }
        __syncthreads();
        const int na = s_base;
        for (long long t0 = 0; t0 < g.n_samp; t0 += kSynthTile) {
            const long long t1 = min((long long)g.n_samp, t0 + kSynthTile);
            if (threadIdx.x == 0) s_nt = 0;
            __syncthreads();
            for (int a0 = 0; a0 < na; a0 += blockDim.x) {
                const int a = a0 + threadIdx.x;
                const bool hit = a < na && s_k0[a] < t1 && (long long)s_k0[a] + g.n_w > t0;
                const int pos = block_append(hit, s_warp, &s_nt);
                if (hit) s_tl[pos] = a;
            }
            const int nt = s_nt;
            for (long long k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
                if (F32) {
                    float* vrow = (float*)d.V + (size_t)j * g.pitch;
                    float a2 = first ? g.syn0_f : vrow[k], c2 = 0.f;
                    for (int q = 0; q < nt; ++q) {
                        const int a = s_tl[q];
                        const int r = (int)(k - s_k0[a]);
                        if ((unsigned)r < (unsigned)g.n_w) kahan_add(a2, c2, arr_var32(g, s_E0[a], s_k0[a], (int)k));
                    }
                    vrow[k] = a2 - c2;
                } else {
                    double* vrow = (double*)d.V + (size_t)j * g.pitch;
                    double a2 = first ? g.noise_var : vrow[k];
                    for (int q = 0; q < nt; ++q) {
                        const int a = s_tl[q];
                        const int r = (int)(k - s_k0[a]);
                        if ((unsigned)r < (unsigned)g.n_w) a2 += arr_c64(g, s_af[a], s_ln[a], (int)k);
                    }
                    vrow[k] = a2;
                }
            }
            __syncthreads();
        }
        first = false;
        if (base >= n) break;
    }
}

// the flat list of store `buf` (cells in index order, events in their
// order): first each cell's position, an exclusive prefix of the counts (one
// block), then a warp per cell copies its events (lanes over events)
__global__ void __launch_bounds__(1024) flatten_scan(Geo g, Dev d, int buf, int* n_out) {
    const Store S = d.st[buf];
    __shared__ int s_warp[32], s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < g.n_cells; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int n = c < g.n_cells ? S.count[c] : 0;
        int x = n;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) before += s_warp[w];
            all += s_warp[w];
        }
        if (c < g.n_cells) d.flat_off[c] = s_base + before + x - n;
        __syncthreads();
        if (threadIdx.x == 0) s_base += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.flat_off[g.n_cells] = s_base;
        *n_out = s_base;
    }
}

__global__ void __launch_bounds__(256) flatten_copy(Geo g, Dev d, int buf, double* fx, double* fy, double* ft,
                                                    double* fm, unsigned long long* fid, double* foff) {
    const Store S = d.st[buf];
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= g.n_cells) return;
    const int n = S.count[c], s0 = S.start[c], off = d.flat_off[c];
    for (int i = lane; i < n; i += 32) {
        fx[off + i] = S.x[s0 + i];
        fy[off + i] = S.y[s0 + i];
        ft[off + i] = S.t[s0 + i];
        fm[off + i] = S.m[s0 + i];
        fid[off + i] = S.id[s0 + i];
    }
    if (foff && S.off)   // latent arrival offsets: the cell's rows, lanes over entries
        for (long long q = lane; q < (long long)n * g.n_st; q += 32)
            foff[(size_t)off * g.n_st + q] = S.off[(size_t)s0 * g.n_st + q];
}

// latent arrival offsets of a flat list: entries of stations an event does
// not reach are set to 0; the others' log N(delta; 0, sig_a^2) summed in a
// fixed order (thread-strided, then a tree) into *out.  One block.
__global__ void __launch_bounds__(256) offprior_kernel(Geo g, Dev d, const double* fx, const double* fy,
                                                       double* foff, const int* n_ptr, double* out) {
    __shared__ double s_part[256];
    const long long tot = (long long)(*n_ptr) * g.n_st;
    double acc = 0.0;
    for (long long q = threadIdx.x; q < tot; q += blockDim.x) {
        const long long i = q / g.n_st;
        const int j = (int)(q - i * g.n_st);
        if (dist_rn(fx[i], fy[i], d.stx[j], d.sty[j]) < g.R_max) acc += log_off_prior1(g, foff[q]);
        else foff[q] = 0.0;
    }
    s_part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s_part[threadIdx.x] += s_part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s_part[0];
}

// sum over all stations and samples of log N(s; 0, V) (or, with the additive
// reading in float32, log N(s; mu, noise) with mu in the V buffer): per-block
// partials
template <bool F32>
__global__ void loglik_kernel(Geo g, Dev d, double* partial) {
    __shared__ double s_part[32];
    double acc = 0.0;
    const long long total = (long long)g.n_st * g.n_samp;
    const double half_log_2pi = 0.91893853320467274178;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = i / g.n_samp, k = i - j * g.n_samp;
        if (F32) {
            const float s = ((const float*)d.sig)[j * g.pitch + k];
            const float V = ((const float*)d.V)[j * g.pitch + k];
            if (g.mean_mode) {
                const float r = s - V;
                acc += (double)(-0.5f * r * r * g.inv_noise_f) - 0.5 * log(g.noise_var) - half_log_2pi;
            } else {
                acc += (double)(-0.5f * logf(V) - s * s / (2.f * V)) - half_log_2pi;
            }
        } else {
            const double s = ((const double*)d.sig)[j * g.pitch + k];
            const double V = ((const double*)d.V)[j * g.pitch + k];
            acc += -half_log_2pi - 0.5 * log(V) - s * s / (2.0 * V);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void convert_kernel(const void* src, int src_f32, long long src_pitch, void* dst, int dst_f32,
                               long long dst_pitch, int n_st, long long n_samp, int* nonfinite) {
    const long long total = (long long)n_st * dst_pitch;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = i / dst_pitch, k = i - j * dst_pitch;
        double v = 0.0;
        if (k < n_samp) {
            v = src_f32 ? (double)((const float*)src)[j * src_pitch + k] : ((const double*)src)[j * src_pitch + k];
            if (!isfinite(v)) atomicExch(nonfinite, 1);
        }
        if (dst_f32) ((float*)dst)[i] = (float)v;
        else ((double*)dst)[i] = v;
    }
}

__global__ void philox_test_kernel(const unsigned long long* ctr, const unsigned long long* key,
                                   unsigned long long* out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    philox4x64(c, key[0], key[1]);
    for (int q = 0; q < 4; ++q) out[4 * i + q] = c[q];
}

}  // namespace

size_t phase_smem_bytes(const Geo& g) { return Layout(g).total; }

cudaError_t launch_phase(const Geo& g, const Dev& d, int colour, cudaStream_t s) {
    if (g.f32) return launch_phase32(g, d, colour, s);
    const size_t smem = phase_smem_bytes(g);
    phase_kernel<<<g.max_rpc, g.threads, smem, s>>>(g, d, colour);
    return cudaGetLastError();
}

cudaError_t launch_sweep_end_batch(const Geo* G, const Dev* D, int n_inst, cudaStream_t s) {
    sweep_end_batch<<<n_inst, 1024, 0, s>>>(G, D);
    return cudaGetLastError();
}

cudaError_t launch_sweep_end(const Geo& g, const Dev& d, cudaStream_t s) {
    sweep_end<<<1, 1024, 0, s>>>(g, d);
    return cudaGetLastError();
}

cudaError_t launch_vsynth(const Geo& g, const Dev& d, const FlatList& f, cudaStream_t s, int* launches) {
    if (g.n_st == 0) return cudaSuccess;
    if (g.f32) vsynth_kernel<true><<<g.n_st, kSynthThreads, 0, s>>>(g, d, f.x, f.y, f.t, f.m, f.n, f.off);
    else vsynth_kernel<false><<<g.n_st, kSynthThreads, 0, s>>>(g, d, f.x, f.y, f.t, f.m, f.n, f.off);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_flatten(const Geo& g, const Dev& d, int buf, const FlatList& f, cudaStream_t s, int* launches) {
    flatten_scan<<<1, 1024, 0, s>>>(g, d, buf, f.n);
    flatten_copy<<<(g.n_cells + 7) / 8, 256, 0, s>>>(g, d, buf, f.x, f.y, f.t, f.m, f.id, f.off);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t prepare_kernels(const Geo& g) {
    const size_t smem = phase_smem_bytes(g);
    return raise_smem_limit((const void*)phase_kernel, smem);
}

cudaError_t launch_offset_prior(const Geo& g, const Dev& d, const FlatList& f, double* out, cudaStream_t s) {
    offprior_kernel<<<1, 256, 0, s>>>(g, d, f.x, f.y, f.off, f.n, out);
    return cudaGetLastError();
}

cudaError_t launch_loglik(const Geo& g, const Dev& d, double* partial, int n_part, cudaStream_t s) {
    if (g.f32) loglik_kernel<true><<<n_part, 256, 0, s>>>(g, d, partial);
    else loglik_kernel<false><<<n_part, 256, 0, s>>>(g, d, partial);
    return cudaGetLastError();
}

cudaError_t launch_convert_signals(const void* src, int src_f32, long long src_pitch, void* dst, int dst_f32,
                                   long long dst_pitch, int n_st, long long n_samp, int* nonfinite,
                                   cudaStream_t s) {
    if (n_st == 0) return cudaSuccess;
    convert_kernel<<<1216, 256, 0, s>>>(src, src_f32, src_pitch, dst, dst_f32, dst_pitch, n_st, n_samp, nonfinite);
    return cudaGetLastError();
}

cudaError_t launch_philox_test(const unsigned long long* ctr, const unsigned long long* key,
                               unsigned long long* out, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    philox_test_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(ctr, key, out, n);
    return cudaGetLastError();
}

}  // namespace cmh
