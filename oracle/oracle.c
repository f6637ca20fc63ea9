/*
 * CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain float64 C,
 * compiled with -ffp-contract=off so that every + - * / sqrt is a single
 * correctly rounded IEEE operation.  Parity: pinned by tests/test_oracle_*.py
 * (closed forms, exact enumeration and detailed balance on lattice worlds,
 * prior-only chains, brute-force differences, numpy's Philox).
 *
 * Model (§Generative Model of Seismic Signals, with the attenuating,
 * finite-reach extension that §Partitioning the World names as the case where
 * a spatial partition is natural):
 *   event e = (x, y, t, m) in [0,W)^2 x [0,T) x [2, inf)
 *   prior: Poisson process with intensity beta(e) = Lambda/(W^2 T) exp(-(m-2));
 *          log-density  -Lambda + sum_i log beta(e_i)
 *   arrival at station j: a = t + d/v + delta_j  (d = distance; with
 *          sig_a > 0 a latent delta_j ~ N(0, sig_a^2) per reached station,
 *          otherwise delta_j = 0: the deterministic arrival)
 *   the event reaches station j iff d < R_max
 *   variance added at sample k (time k/f): (A g(k/f - a))^2 for
 *          k in [ceil(a f), ceil(a f) + n_w), A = exp(alpha m - beta_att d),
 *          g(u) = exp(-u / tau)
 *   s_jk ~ N(0, V_jk), V_jk = noise_var + sum of the variances above
 * or, with the additive-mean reading (likelihood = 1), each arrival adds
 * A g(k/f - a) to the mean: s_jk ~ N(mu_jk, noise_var), mu_jk = that sum
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Planted mistakes for the pin tests (tests/test_oracle_mutants.py build the
 * oracle with -DORC_MUTANT=n and check that some pin fails):
 *   1: birth ratio uses 1/(n+2) for the reverse death;  2: death drops log q_b;
 *   3: an arrival adds its standard deviation instead of its variance;
 *   4: a move ignores the prior ratio;
 *   5: the birth and death terms use the uniform density although births
 *      come from the mixture with a learned table;
 *   6: with learned magnitudes, the learned component's density keeps the
 *      prior magnitude law although it draws m from its window;
 *   7: the joint move of a pair ignores the prior ratio;
 *   8: the arrival-time move ignores the prior ratio of its offset;
 *   9: offsets of stations an event newly reaches are set to 0 instead of
 *      drawn from their prior.
 * 0 (the default) is the oracle itself. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

/* an event; with latent arrival times also the offsets delta of the na
 * stations it reaches (sta[] increasing) */
#define ORC_MAXA 128
typedef struct {
    double x, y, t, m;
    uint64_t id;
    int32_t na;
    int32_t sta[ORC_MAXA];
    double off[ORC_MAXA];
} ev_t;

struct orc_world {
    orc_params p;
    int32_t n_st;
    double* st;          /* [n_st][2], owned copy */
    const void* sig;     /* [n_st][pitch], caller-owned */
    int32_t f32;
    int64_t n_samp, pitch;
    /* learned birth component (none when bt_nx == 0): a weight table over
     * pixels (bt_nx x bt_ny over [0,W)^2) and time bins (bt_nt over [0,T)) */
    int32_t bt_nx, bt_ny, bt_nt;
    double bt_mix, bt_hx, bt_hy, bt_dt, bt_pixarea;
    double* bt_mass;     /* [pixel] sum of the pixel's weights */
    double* bt_cdf;      /* [pixel][bin] running sum of its weights / mass */
    /* magnitudes of the learned component (none when NULL: m - 2 ~ Exp(1) as
     * for uniform births): a birth at (pixel, bin) draws m uniform on
     * [lo, lo + 2h), lo = max(2, centre - h) */
    float* bt_mag;       /* [pixel][bin] window centre, owned copy */
    double bt_h;
};

struct orc_set { ev_t* e; int64_t n, cap; };

/* ------------------------------------------------------------------------
 * Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Round: two 64x64->128 products of the counter's
 * even words with fixed multipliers, the high halves xored with the odd words
 * and the key, the key bumped by the Weyl constants between rounds.
 * ---------------------------------------------------------------------- */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform in [0,1) from the top 53 bits */
static double u01(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }
/* uniform in (0,1] */
static double u01o(uint64_t w) { return (double)((w >> 11) + 1) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, n) from the low 32 bits */
static int64_t pick(uint64_t w, int64_t n) { return (int64_t)(((w & 0xffffffffULL) * (uint64_t)n) >> 32); }

/* twelve 64-bit words of one MH step: counter (c0, c1, c2, 0|1|2), key
 * (seed, stream); the third block is used only by learned births */
static void step_words(const orc_world* w, uint64_t stream, uint64_t c0, uint64_t c1, uint64_t c2,
                       uint64_t out[12]) {
    uint64_t key[2] = { w->p.seed, stream };
    uint64_t ctr[4] = { c0, c1, c2, 0 };
    orc_philox4x64(ctr, key, out);
    ctr[3] = 1;
    orc_philox4x64(ctr, key, out + 4);
    ctr[3] = 2;
    orc_philox4x64(ctr, key, out + 8);
}

/* ------------------------------------------------------------------------
 * world and event sets
 * ---------------------------------------------------------------------- */
orc_world* orc_world_new(const orc_params* p, const double* stations, int32_t n_st,
                         const void* signals, int32_t signals_f32, int64_t n_samp, int64_t pitch) {
    orc_world* w = (orc_world*)calloc(1, sizeof(orc_world));
    w->p = *p;
    w->n_st = n_st;
    w->st = (double*)malloc(sizeof(double) * 2 * (size_t)(n_st > 0 ? n_st : 1));
    if (n_st > 0) memcpy(w->st, stations, sizeof(double) * 2 * (size_t)n_st);
    w->sig = signals;
    w->f32 = signals_f32;
    w->n_samp = n_samp;
    w->pitch = pitch;
    if (p->sig_a > 0.0) {
        /* an event's reached stations lie within 2 R_max of one another, so
         * no event reaches more than the largest such neighbourhood */
        for (int32_t j = 0; j < n_st; ++j) {
            int32_t c = 0;
            for (int32_t k = 0; k < n_st; ++k) {
                const double dx = w->st[2 * j] - w->st[2 * k], dy = w->st[2 * j + 1] - w->st[2 * k + 1];
                if (sqrt(dx * dx + dy * dy) < 2.0 * p->R_max) ++c;
            }
            if (c > ORC_MAXA) { orc_world_free(w); return NULL; }
        }
    }
    return w;
}

void orc_world_free(orc_world* w) {
    if (!w) return;
    free(w->st);
    free(w->bt_mass);
    free(w->bt_cdf);
    free(w->bt_mag);
    free(w);
}

/* The learned component of the birth proposal (a mixture with the uniform
 * birth, mixing weight mix): tab[(iy * nx + ix) * nt + b] >= 0 is the weight
 * of pixel (ix, iy) of side (W/nx, W/ny) and time bin b of length T/nt.
 * Sums run in index order in float64.  nx == 0 removes the component. */
int orc_set_birth_table(orc_world* w, const float* tab, int32_t nx, int32_t ny, int32_t nt, double mix) {
    free(w->bt_mass);
    free(w->bt_cdf);
    free(w->bt_mag);
    w->bt_mass = NULL;
    w->bt_cdf = NULL;
    w->bt_mag = NULL;
    w->bt_nx = w->bt_ny = w->bt_nt = 0;
    if (nx == 0) return 0;
    if (nx < 1 || ny < 1 || nt < 1 || !(mix > 0.0 && mix < 1.0) || !tab) return -1;
    const int64_t np = (int64_t)nx * ny;
    w->bt_mass = (double*)malloc(sizeof(double) * (size_t)np);
    w->bt_cdf = (double*)malloc(sizeof(double) * (size_t)(np * nt));
    for (int64_t q = 0; q < np; ++q) {
        double run = 0.0;
        for (int32_t b = 0; b < nt; ++b) {
            const double v = (double)tab[q * nt + b];
            if (!(v >= 0.0) || isinf(v)) return -1;
            run += v;
            w->bt_cdf[q * nt + b] = run;
        }
        w->bt_mass[q] = run;
        for (int32_t b = 0; b < nt; ++b) w->bt_cdf[q * nt + b] = run > 0.0 ? w->bt_cdf[q * nt + b] / run : 0.0;
    }
    w->bt_nx = nx;
    w->bt_ny = ny;
    w->bt_nt = nt;
    w->bt_mix = mix;
    w->bt_hx = w->p.W / (double)nx;
    w->bt_hy = w->p.W / (double)ny;
    w->bt_dt = w->p.T / (double)nt;
    w->bt_pixarea = w->bt_hx * w->bt_hy;
    return 0;
}

/* Magnitudes of the learned component: centre[(iy * nx + ix) * nt + b]
 * (finite) for the table's pixels and bins, window half-width h > 0; NULL
 * returns to magnitudes from the prior.  Needs a table; a new table drops
 * them. */
int orc_set_birth_magnitude(orc_world* w, const float* centre, double h) {
    free(w->bt_mag);
    w->bt_mag = NULL;
    if (!centre) return 0;
    if (!w->bt_nx || !(h > 0.0) || isinf(h)) return -1;
    const int64_t n = (int64_t)w->bt_nx * w->bt_ny * w->bt_nt;
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(centre[i])) return -1;
    w->bt_mag = (float*)malloc(sizeof(float) * (size_t)n);
    memcpy(w->bt_mag, centre, sizeof(float) * (size_t)n);
    w->bt_h = h;
    return 0;
}

static double sig_at(const orc_world* w, int32_t j, int64_t k) {
    if (w->f32) return (double)((const float*)w->sig)[(int64_t)j * w->pitch + k];
    return ((const double*)w->sig)[(int64_t)j * w->pitch + k];
}

orc_set* orc_set_new(const double* ev, const uint64_t* ids, int64_t n) {
    orc_set* s = (orc_set*)calloc(1, sizeof(orc_set));
    s->cap = n > 16 ? n : 16;
    s->e = (ev_t*)malloc(sizeof(ev_t) * (size_t)s->cap);
    s->n = n;
    for (int64_t i = 0; i < n; ++i) {
        s->e[i].x = ev[4 * i]; s->e[i].y = ev[4 * i + 1];
        s->e[i].t = ev[4 * i + 2]; s->e[i].m = ev[4 * i + 3];
        s->e[i].id = ids ? ids[i] : (uint64_t)i;
        s->e[i].na = 0;
    }
    return s;
}

static void fill_offsets(const orc_world* w, ev_t* e, const double* row);

orc_set* orc_set_new_w(const orc_world* w, const double* ev, const uint64_t* ids, const double* off,
                       int64_t n) {
    orc_set* s = orc_set_new(ev, ids, n);
    for (int64_t i = 0; i < n; ++i) fill_offsets(w, &s->e[i], off ? off + (size_t)i * (size_t)w->n_st : NULL);
    return s;
}

void orc_set_offsets(const orc_world* w, const orc_set* s, double* off) {
    memset(off, 0, sizeof(double) * (size_t)s->n * (size_t)w->n_st);
    for (int64_t i = 0; i < s->n; ++i)
        for (int32_t k = 0; k < s->e[i].na; ++k) off[(size_t)i * (size_t)w->n_st + s->e[i].sta[k]] = s->e[i].off[k];
}
int64_t orc_set_size(const orc_set* s) { return s->n; }
void orc_set_get(const orc_set* s, double* ev, uint64_t* ids) {
    for (int64_t i = 0; i < s->n; ++i) {
        ev[4 * i] = s->e[i].x; ev[4 * i + 1] = s->e[i].y;
        ev[4 * i + 2] = s->e[i].t; ev[4 * i + 3] = s->e[i].m;
        if (ids) ids[i] = s->e[i].id;
    }
}
void orc_set_free(orc_set* s) {
    if (!s) return;
    free(s->e);
    free(s);
}

static void to_ev(const double* a, ev_t* e) {
    e->x = a[0]; e->y = a[1]; e->t = a[2]; e->m = a[3]; e->id = 0; e->na = 0;
}

static int reaches(const orc_world* w, const ev_t* e, int32_t j) {
    double dx = e->x - w->st[2 * j];
    double dy = e->y - w->st[2 * j + 1];
    return sqrt(dx * dx + dy * dy) < w->p.R_max;
}

/* with latent arrivals: the offsets of the stations e reaches, from a dense
 * row (NULL: 0) */
static void fill_offsets(const orc_world* w, ev_t* e, const double* row) {
    e->na = 0;
    if (!(w->p.sig_a > 0.0)) return;
    for (int32_t j = 0; j < w->n_st; ++j)
        if (reaches(w, e, j)) {
            e->sta[e->na] = j;
            e->off[e->na] = row ? row[j] : 0.0;
            ++e->na;
        }
}

/* offset of e at station j (0 if none is held) */
static double offset_at(const ev_t* e, int32_t j) {
    for (int32_t k = 0; k < e->na; ++k)
        if (e->sta[k] == j) return e->off[k];
    return 0.0;
}

/* log N(delta; 0, sig_a^2) summed over e's offsets (0 without latent arrivals) */
static double log_off_prior(const orc_world* w, const ev_t* e) {
    if (!(w->p.sig_a > 0.0)) return 0.0;
    const double s2 = w->p.sig_a * w->p.sig_a;
    double lp = 0.0;
    for (int32_t k = 0; k < e->na; ++k)
        lp += -0.5 * log(2.0 * M_PI * s2) - e->off[k] * e->off[k] / (2.0 * s2);
    return lp;
}

/* ------------------------------------------------------------------------
 * likelihood pieces (§Generative Model: the observed signal is a zero-mean
 * diagonal Gaussian whose per-sample variance is the noise variance plus the
 * variances of the arriving event signals)
 * ---------------------------------------------------------------------- */
typedef struct { int reach; int64_t k0; double a, amp; } arr_t;

/* arrival of event e at station j: a = t + d/v (the mean of the
 * arrival-time distribution of §Event Detections) plus, with latent arrival
 * times, the event's offset at j */
static arr_t arrival_of(const orc_world* w, const ev_t* e, int32_t j) {
    arr_t r;
    double dx = e->x - w->st[2 * j];
    double dy = e->y - w->st[2 * j + 1];
    double d = sqrt(dx * dx + dy * dy);
    r.reach = d < w->p.R_max;
    r.a = e->t + d / w->p.v;
    if (w->p.sig_a > 0.0) r.a += offset_at(e, j);
    r.k0 = (int64_t)ceil(r.a * w->p.f_hz);
    r.amp = exp(w->p.alpha * e->m - w->p.beta_att * d);
    return r;
}

/* what this arrival adds at sample k to the predicted quantity: the variance
 * (A e^{-u/tau})^2 of the zero-mean sample, or with the additive-mean
 * reading the mean A e^{-u/tau} */
static double arr_var(const orc_world* w, const arr_t* r, int64_t k) {
    if (!r->reach || k < r->k0 || k >= r->k0 + w->p.n_w) return 0.0;
    double u = (double)k / w->p.f_hz - r->a;
    double sd = r->amp * exp(-u / w->p.tau);
    if (w->p.likelihood) return sd;
    return ORC_MUTANT == 3 ? sd : sd * sd;
}

/* the predicted quantity with no arrival: the noise variance, or mean 0 */
static double pred_base(const orc_world* w) { return w->p.likelihood ? 0.0 : w->p.noise_var; }

static double log_normal0(double s, double V) {
    return -0.5 * log(2.0 * M_PI * V) - s * s / (2.0 * V);
}

/* log density of sample s given the predicted quantity P */
static double log_lik_sample(const orc_world* w, double s, double P) {
    if (!w->p.likelihood) return log_normal0(s, P);
    const double r = s - P;
    return -0.5 * log(2.0 * M_PI * w->p.noise_var) - r * r / (2.0 * w->p.noise_var);
}

void orc_variance(const orc_world* w, const double* ev, int64_t n, int32_t j,
                  int64_t k0, int64_t k1, double* out) {
    arr_t* ar = (arr_t*)malloc(sizeof(arr_t) * (size_t)(n > 0 ? n : 1));
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
        ev_t e; to_ev(ev + 4 * i, &e);
        arr_t a = arrival_of(w, &e, j);
        if (a.reach) ar[na++] = a;
    }
    for (int64_t k = k0; k < k1; ++k) {
        double V = pred_base(w);
        for (int64_t i = 0; i < na; ++i) V += arr_var(w, &ar[i], k);
        out[k - k0] = V;
    }
    free(ar);
}

double orc_log_likelihood_off(const orc_world* w, const double* ev, const double* off, int64_t n) {
    double total = 0.0;
    ev_t* es = (ev_t*)malloc(sizeof(ev_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        to_ev(ev + 4 * i, &es[i]);
        fill_offsets(w, &es[i], off ? off + (size_t)i * (size_t)w->n_st : NULL);
    }
    arr_t* ar = (arr_t*)malloc(sizeof(arr_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t j = 0; j < w->n_st; ++j) {
        int64_t na = 0;
        for (int64_t i = 0; i < n; ++i) {
            arr_t a = arrival_of(w, &es[i], j);
            if (a.reach) ar[na++] = a;
        }
        for (int64_t k = 0; k < w->n_samp; ++k) {
            double V = pred_base(w);
            for (int64_t i = 0; i < na; ++i) V += arr_var(w, &ar[i], k);
            total += log_lik_sample(w, sig_at(w, j, k), V);
        }
    }
    free(ar);
    free(es);
    return total;
}

double orc_log_likelihood(const orc_world* w, const double* ev, int64_t n) {
    return orc_log_likelihood_off(w, ev, NULL, n);
}

/* ------------------------------------------------------------------------
 * prior (§Generative Model, "Event prior"): Poisson count, uniform location
 * and time; magnitude 2 + Exp(1).  Written as a Poisson-process density:
 * -Lambda + sum log beta(e).  Lattice mode restricts coordinates to a grid
 * and beta to point masses (used only by the enumeration tests).
 * ---------------------------------------------------------------------- */
static int lat_index(double v, double v0, double dv, int32_t n) {
    double f = (v - v0) / dv;
    double r = rint(f);
    if (fabs(f - r) > 1e-9 || r < 0 || r >= n) return -1;
    return (int)r;
}

static double lat_log_wm(const orc_params* p, int im) {
    double z = 0.0;
    for (int i = 0; i < p->lat_nm; ++i) z += exp(-(p->lat_m0 + i * p->lat_dm - 2.0));
    return -(p->lat_m0 + im * p->lat_dm - 2.0) - log(z);
}

static double log_beta(const orc_world* w, const ev_t* e) {
    const orc_params* p = &w->p;
    if (p->lattice) {
        int ix = lat_index(e->x, p->lat_x0, p->lat_dx, p->lat_nx);
        int iy = lat_index(e->y, p->lat_y0, p->lat_dy, p->lat_ny);
        int it = lat_index(e->t, p->lat_t0, p->lat_dt, p->lat_nt);
        int im = lat_index(e->m, p->lat_m0, p->lat_dm, p->lat_nm);
        if (ix < 0 || iy < 0 || it < 0 || im < 0) return -INFINITY;
        return log(p->Lambda) - log((double)p->lat_nx * p->lat_ny) - log((double)p->lat_nt)
               + lat_log_wm(p, im);
    }
    if (!(e->x >= 0.0 && e->x < p->W && e->y >= 0.0 && e->y < p->W &&
          e->t >= 0.0 && e->t < p->T && e->m >= 2.0))
        return -INFINITY;
    return log(p->Lambda) - log(p->W * p->W * p->T) - (e->m - 2.0);
}

double orc_log_prior_off(const orc_world* w, const double* ev, const double* off, int64_t n) {
    double lp = -w->p.Lambda;
    for (int64_t i = 0; i < n; ++i) {
        ev_t e; to_ev(ev + 4 * i, &e);
        fill_offsets(w, &e, off ? off + (size_t)i * (size_t)w->n_st : NULL);
        lp += log_beta(w, &e) + log_off_prior(w, &e);
    }
    return lp;
}

double orc_log_prior(const orc_world* w, const double* ev, int64_t n) {
    return orc_log_prior_off(w, ev, NULL, n);
}

/* ------------------------------------------------------------------------
 * log-likelihood change of one proposal: the event own[old_idx] (if any) is
 * replaced by cand (if any); context = own + oth.  Plain definition: for every
 * station and sample whose predicted value changes, the difference of the two
 * Gaussian log-densities of the sample (§Generative Model, Observed Signals),
 * the predicted values P (old) and P' (new) summed from scratch.
 *
 * The difference is written out term by term rather than as a subtraction of
 * two log-densities.  Where a large signal is unexplained, s^2 / 2V is large
 * (1e5 and more) at both P and P', and subtracting the two rounded terms loses
 * digits the difference needs; written out, the two forms are equal:
 *   variance reading:  log N(s; 0, P') - log N(s; 0, P)
 *                        = -1/2 log(P'/P) + s^2 D / (2 P P')
 *   mean reading:      log N(s; P', s2) - log N(s; P, s2)
 *                        = D ((s - P) + (s - P')) / (2 s2)
 * with D = P' - P the change of the changed events' own contributions
 * (arr_change), not the difference of the two sums.
 * ---------------------------------------------------------------------- */

/* is sample k inside the window of arrival r */
static int covers(const orc_world* w, const arr_t* r, int64_t k) {
    return r->reach && k >= r->k0 && k < r->k0 + w->p.n_w;
}

static double dist_to(const orc_world* w, const ev_t* e, int32_t j) {
    double dx = e->x - w->st[2 * j];
    double dy = e->y - w->st[2 * j + 1];
    return sqrt(dx * dx + dy * dy);
}

/* change at sample k of station j of what one event adds to the predicted
 * value when it goes from eo (arrival ao) to en (arrival an); either may be
 * NULL (birth, death).  Where both windows cover k the two contributions are
 * the same envelope shape, A e^{-u/tau} with A = e^{alpha m - beta d} and
 * u = k/f - a (squared in the variance reading), so their ratio is the same
 * at every such sample:
 *   c_new / c_old = exp(q [alpha (m' - m) - beta (d' - d) + (a' - a) / tau]),
 * q = 2 (variance) or 1 (mean).  The change is then c_old (e^E - 1), E taken
 * from the coordinate changes: d' - d = (d'^2 - d^2) / (d' + d) with
 * d'^2 - d^2 = (x' - x)(x' + x - 2 x_j) + (y' - y)(y' + y - 2 y_j), and
 * a' - a = (t' - t) + (d' - d) / v plus the change of the offset at j with
 * latent arrivals.  A small move then subtracts no two nearly equal numbers. */
static double arr_change(const orc_world* w, const ev_t* eo, const arr_t* ao, const ev_t* en,
                         const arr_t* an, int32_t j, int64_t k) {
    const int io = eo && covers(w, ao, k), in = en && covers(w, an, k);
    if (!io && !in) return 0.0;
    if (!io) return arr_var(w, an, k);
    if (!in) return -arr_var(w, ao, k);
    const double xj = w->st[2 * j], yj = w->st[2 * j + 1];
    const double d_o = dist_to(w, eo, j), d_n = dist_to(w, en, j);
    const double dsq = (en->x - eo->x) * (en->x + eo->x - 2.0 * xj) +
                       (en->y - eo->y) * (en->y + eo->y - 2.0 * yj);
    const double dd = d_n + d_o > 0.0 ? dsq / (d_n + d_o) : 0.0;
    double da = (en->t - eo->t) + dd / w->p.v;
    if (w->p.sig_a > 0.0) da += offset_at(en, j) - offset_at(eo, j);
    const double q = (w->p.likelihood || ORC_MUTANT == 3) ? 1.0 : 2.0;   /* the power arr_var takes */
    const double E = q * (w->p.alpha * (en->m - eo->m) - w->p.beta_att * dd + da / w->p.tau);
    return arr_var(w, ao, k) * expm1(E);
}

/* the difference of the two log-densities of sample s, written out as above */
static double delta_sample(const orc_world* w, double s, double P_old, double P_new, double D) {
    if (w->p.likelihood)
        return D * ((s - P_old) + (s - P_new)) / (2.0 * w->p.noise_var);
    return -0.5 * log(P_new / P_old) + s * s * D / (2.0 * P_old * P_new);
}

static double delta_ll2(const orc_world* w, const ev_t* own, int64_t n_own, const ev_t* oth,
                        int64_t n_oth, int64_t old_idx, const ev_t* cand) {
    double total = 0.0;
    int64_t cap = n_own + n_oth;
    arr_t* ar = (arr_t*)malloc(sizeof(arr_t) * (size_t)(cap > 0 ? cap : 1));
    for (int32_t j = 0; j < w->n_st; ++j) {
        arr_t ao = { 0, 0, 0.0, 0.0 }, an = { 0, 0, 0.0, 0.0 };
        if (old_idx >= 0) ao = arrival_of(w, &own[old_idx], j);
        if (cand) an = arrival_of(w, cand, j);
        if (!ao.reach && !an.reach) continue;
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        if (ao.reach) { if (ao.k0 < lo) lo = ao.k0; if (ao.k0 + w->p.n_w > hi) hi = ao.k0 + w->p.n_w; }
        if (an.reach) { if (an.k0 < lo) lo = an.k0; if (an.k0 + w->p.n_w > hi) hi = an.k0 + w->p.n_w; }
        if (lo < 0) lo = 0;
        if (hi > w->n_samp) hi = w->n_samp;
        if (lo >= hi) continue;
        int64_t na = 0;
        for (int64_t i = 0; i < n_own; ++i) {
            if (i == old_idx) continue;
            arr_t a = arrival_of(w, &own[i], j);
            if (a.reach) ar[na++] = a;
        }
        for (int64_t i = 0; i < n_oth; ++i) {
            arr_t a = arrival_of(w, &oth[i], j);
            if (a.reach) ar[na++] = a;
        }
        for (int64_t k = lo; k < hi; ++k) {
            double base = pred_base(w);
            for (int64_t i = 0; i < na; ++i) base += arr_var(w, &ar[i], k);
            double V_old = base + arr_var(w, &ao, k);
            double V_new = base + arr_var(w, &an, k);
            double D = arr_change(w, old_idx >= 0 ? &own[old_idx] : NULL, &ao, cand, &an, j, k);
            if (ORC_MUTANT == 10)
                total += log_lik_sample(w, sig_at(w, j, k), V_new) - log_lik_sample(w, sig_at(w, j, k), V_old);
            else
                total += delta_sample(w, sig_at(w, j, k), V_old, V_new, D);
        }
    }
    free(ar);
    return total;
}

double orc_delta_loglik(const orc_world* w, const double* ev, int64_t n,
                        int64_t old_idx, const double* cand) {
    ev_t* own = (ev_t*)malloc(sizeof(ev_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) to_ev(ev + 4 * i, &own[i]);
    ev_t c;
    if (cand) to_ev(cand, &c);
    double d = delta_ll2(w, own, n, NULL, 0, old_idx, cand ? &c : NULL);
    free(own);
    return d;
}

/* log-likelihood change of a joint move: own[i1] and own[i2] become c1 and
 * c2.  Same plain definition: at every station one of the four events
 * reaches, over the span of their windows, the difference of the two
 * Gaussian log-densities written out as in delta_sample, D the sum of the two
 * events' own changes. */
static double delta_ll_pair(const orc_world* w, const ev_t* own, int64_t n_own, const ev_t* oth,
                            int64_t n_oth, int64_t i1, int64_t i2, const ev_t* c1, const ev_t* c2) {
    double total = 0.0;
    int64_t cap = n_own + n_oth;
    arr_t* ar = (arr_t*)malloc(sizeof(arr_t) * (size_t)(cap > 0 ? cap : 1));
    for (int32_t j = 0; j < w->n_st; ++j) {
        arr_t ch[4];
        ch[0] = arrival_of(w, &own[i1], j);
        ch[1] = arrival_of(w, &own[i2], j);
        ch[2] = arrival_of(w, c1, j);
        ch[3] = arrival_of(w, c2, j);
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        for (int q = 0; q < 4; ++q) {
            if (!ch[q].reach) continue;
            if (ch[q].k0 < lo) lo = ch[q].k0;
            if (ch[q].k0 + w->p.n_w > hi) hi = ch[q].k0 + w->p.n_w;
        }
        if (lo == INT64_MAX) continue;
        if (lo < 0) lo = 0;
        if (hi > w->n_samp) hi = w->n_samp;
        if (lo >= hi) continue;
        int64_t na = 0;
        for (int64_t i = 0; i < n_own; ++i) {
            if (i == i1 || i == i2) continue;
            arr_t a = arrival_of(w, &own[i], j);
            if (a.reach) ar[na++] = a;
        }
        for (int64_t i = 0; i < n_oth; ++i) {
            arr_t a = arrival_of(w, &oth[i], j);
            if (a.reach) ar[na++] = a;
        }
        for (int64_t k = lo; k < hi; ++k) {
            double base = pred_base(w);
            for (int64_t i = 0; i < na; ++i) base += arr_var(w, &ar[i], k);
            double V_old = base + arr_var(w, &ch[0], k) + arr_var(w, &ch[1], k);
            double V_new = base + arr_var(w, &ch[2], k) + arr_var(w, &ch[3], k);
            double D = arr_change(w, &own[i1], &ch[0], c1, &ch[2], j, k) +
                       arr_change(w, &own[i2], &ch[1], c2, &ch[3], j, k);
            total += delta_sample(w, sig_at(w, j, k), V_old, V_new, D);
        }
    }
    free(ar);
    return total;
}

/* ------------------------------------------------------------------------
 * spatial partition (§Partitioning the World, in two spatial dimensions):
 * square cells of side L whose boundaries are shifted by (sx, sy);
 * cell index ix = floor((x - sx)/L) + 1.  Cells whose indices differ by a
 * multiple of the period p = ceil(2 R_max / L) + 1 in both axes share a colour;
 * their nearest points are >= (p-1) L >= 2 R_max apart, so no station lies
 * within R_max of both: same-colour regions have disjoint Markov blankets.
 * ---------------------------------------------------------------------- */
int32_t orc_period(const orc_world* w) { return (int32_t)ceil(2.0 * w->p.R_max / w->p.L) + 1; }

void orc_grid_dims(const orc_world* w, int32_t* ncx, int32_t* ncy) {
    int32_t n = (int32_t)floor(w->p.W / w->p.L) + 2;
    *ncx = n;
    *ncy = n;
}

int32_t orc_cell_of(const orc_world* w, double sx, double sy, double x, double y) {
    int32_t ncx, ncy;
    orc_grid_dims(w, &ncx, &ncy);
    int32_t ix = (int32_t)floor((x - sx) / w->p.L) + 1;
    int32_t iy = (int32_t)floor((y - sy) / w->p.L) + 1;
    if (ix < 0 || ix >= ncx || iy < 0 || iy >= ncy) return -1;
    return iy * ncx + ix;
}

void orc_cell_rect(const orc_world* w, double sx, double sy, int32_t cell, double* r4) {
    int32_t ncx, ncy;
    orc_grid_dims(w, &ncx, &ncy);
    int32_t ix = cell % ncx, iy = cell / ncx;
    double x0 = sx + (double)(ix - 1) * w->p.L, x1 = sx + (double)ix * w->p.L;
    double y0 = sy + (double)(iy - 1) * w->p.L, y1 = sy + (double)iy * w->p.L;
    if (x0 < 0.0) x0 = 0.0;
    if (y0 < 0.0) y0 = 0.0;
    if (x1 > w->p.W) x1 = w->p.W;
    if (y1 > w->p.W) y1 = w->p.W;
    r4[0] = x0; r4[1] = x1; r4[2] = y0; r4[3] = y1;
}

int32_t orc_colour_of(const orc_world* w, int32_t cell) {
    int32_t ncx, ncy, p = orc_period(w);
    orc_grid_dims(w, &ncx, &ncy);
    int32_t ix = cell % ncx, iy = cell / ncx;
    return (ix % p) + p * (iy % p);
}

/* §Chromatic MH with Dynamic Coloring: a uniform offset in [0, L) per axis,
 * drawn from Philox stream 1 at counter (sweep, 0, 0, 0) */
void orc_shift(const orc_world* w, int64_t sweep, double* sx, double* sy) {
    uint64_t key[2] = { w->p.seed, 1 };
    uint64_t ctr[4] = { (uint64_t)sweep, 0, 0, 0 };
    uint64_t out[4];
    orc_philox4x64(ctr, key, out);
    *sx = u01(out[0]) * w->p.L;
    *sy = u01(out[1]) * w->p.L;
}

static int cell_live(const double* r) { return r[1] > r[0] && r[3] > r[2]; }

void orc_blankets(const orc_world* w, double sx, double sy, uint8_t* member) {
    int32_t ncx, ncy;
    orc_grid_dims(w, &ncx, &ncy);
    for (int32_t c = 0; c < ncx * ncy; ++c) {
        double r[4];
        orc_cell_rect(w, sx, sy, c, r);
        for (int32_t j = 0; j < w->n_st; ++j) {
            uint8_t in = 0;
            if (cell_live(r)) {
                double xs = w->st[2 * j], ys = w->st[2 * j + 1];
                double dx = 0.0, dy = 0.0;
                if (xs < r[0]) dx = r[0] - xs; else if (xs > r[1]) dx = xs - r[1];
                if (ys < r[2]) dy = r[2] - ys; else if (ys > r[3]) dy = ys - r[3];
                in = sqrt(dx * dx + dy * dy) < w->p.R_max;
            }
            member[(int64_t)c * w->n_st + j] = in;
        }
    }
}

/* ------------------------------------------------------------------------
 * proposals (§Generative Model, the MH moves: birth from a uniform
 * distribution, death of an existing event, Gaussian location move), restricted
 * to one region as in Algorithm "Chromatic MH with Static Coloring".
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t cell;          /* -1: whole domain (serial sampler) */
    double r[4];           /* x0, x1, y0, y1 of the region within the domain */
    double sx, sy;
    double G;              /* learned component: table mass inside the region */
} region_t;

/* pixel range that may overlap [r0, r1) along one axis of pixel side h (one
 * pixel of margin each way: pixels that do not overlap weigh nothing) */
static void pix_range(double r0, double r1, double h, int32_t n, int32_t* i0, int32_t* i1) {
    int32_t a = (int32_t)(r0 / h) - 1, b = (int32_t)(r1 / h) + 1;
    *i0 = a < 0 ? 0 : a;
    *i1 = b > n - 1 ? n - 1 : b;
}

/* overlap of pixel i (side h) with [r0, r1) */
static double pix_overlap(double r0, double r1, double h, int32_t i) {
    const double p0 = (double)i * h, p1 = (double)(i + 1) * h;
    const double lo = p0 > r0 ? p0 : r0, hi = p1 < r1 ? p1 : r1;
    return hi > lo ? hi - lo : 0.0;
}

/* table mass of pixel (ix, iy) inside the region: M_p |p n R| / |p| */
static double pix_weight(const orc_world* w, const region_t* g, int32_t ix, int32_t iy) {
    const double ox = pix_overlap(g->r[0], g->r[1], w->bt_hx, ix);
    const double oy = pix_overlap(g->r[2], g->r[3], w->bt_hy, iy);
    return w->bt_mass[(int64_t)iy * w->bt_nx + ix] * ((ox * oy) / w->bt_pixarea);
}

/* the region's table mass, summed over its pixel range in (iy, ix) order */
static void region_bt(const orc_world* w, region_t* g) {
    g->G = 0.0;
    if (!w->bt_nx) return;
    int32_t x0, x1, y0, y1;
    pix_range(g->r[0], g->r[1], w->bt_hx, w->bt_nx, &x0, &x1);
    pix_range(g->r[2], g->r[3], w->bt_hy, w->bt_ny, &y0, &y1);
    for (int32_t iy = y0; iy <= y1; ++iy)
        for (int32_t ix = x0; ix <= x1; ++ix) g->G += pix_weight(w, g, ix, iy);
}

/* window start of the learned magnitude at table entry q */
static double mag_lo(const orc_world* w, int64_t q) { return fmax(2.0, (double)w->bt_mag[q] - w->bt_h); }

/* table entry (pixel, bin) that (x, y, t) falls in */
static int64_t bt_entry(const orc_world* w, double x, double y, double t) {
    int32_t ix = (int32_t)floor(x / w->bt_hx), iy = (int32_t)floor(y / w->bt_hy), b = (int32_t)floor(t / w->bt_dt);
    if (ix > w->bt_nx - 1) ix = w->bt_nx - 1;
    if (iy > w->bt_ny - 1) iy = w->bt_ny - 1;
    if (b > w->bt_nt - 1) b = w->bt_nt - 1;
    return ((int64_t)iy * w->bt_nx + ix) * w->bt_nt + b;
}

/* density of the learned component at (x, y, t), magnitude factor left out:
 * the pixel's mass share of the region over the pixel area, times the time
 * bin's share of the pixel over the bin length */
static double q_net(const orc_world* w, const region_t* g, double x, double y, double t) {
    if (!(g->G > 0.0)) return 0.0;
    int32_t ix = (int32_t)floor(x / w->bt_hx), iy = (int32_t)floor(y / w->bt_hy), b = (int32_t)floor(t / w->bt_dt);
    if (ix > w->bt_nx - 1) ix = w->bt_nx - 1;
    if (iy > w->bt_ny - 1) iy = w->bt_ny - 1;
    if (b > w->bt_nt - 1) b = w->bt_nt - 1;
    const int64_t q = (int64_t)iy * w->bt_nx + ix;
    const double* c = w->bt_cdf + q * w->bt_nt;
    const double share = c[b] - (b > 0 ? c[b - 1] : 0.0);
    return w->bt_mass[q] * share / (w->bt_pixarea * g->G * w->bt_dt);
}

static int in_region(const orc_world* w, const region_t* g, const ev_t* e) {
    const orc_params* p = &w->p;
    if (!(e->x >= 0.0 && e->x < p->W && e->y >= 0.0 && e->y < p->W)) return 0;
    if (g->cell < 0) return 1;
    return orc_cell_of(w, g->sx, g->sy, e->x, e->y) == g->cell;
}

static int in_time_mag(const orc_world* w, const ev_t* e) {
    if (w->p.lattice) {
        const orc_params* p = &w->p;
        return lat_index(e->t, p->lat_t0, p->lat_dt, p->lat_nt) >= 0 &&
               lat_index(e->m, p->lat_m0, p->lat_dm, p->lat_nm) >= 0 &&
               lat_index(e->x, p->lat_x0, p->lat_dx, p->lat_nx) >= 0 &&
               lat_index(e->y, p->lat_y0, p->lat_dy, p->lat_ny) >= 0;
    }
    return e->t >= 0.0 && e->t < w->p.T && e->m >= 2.0;
}

/* xy lattice points of a region, in row-major order */
static int64_t lat_points(const orc_world* w, const region_t* g, int64_t want, double* xy) {
    const orc_params* p = &w->p;
    int64_t c = 0;
    for (int iy = 0; iy < p->lat_ny; ++iy)
        for (int ix = 0; ix < p->lat_nx; ++ix) {
            ev_t e = { p->lat_x0 + ix * p->lat_dx, p->lat_y0 + iy * p->lat_dy, 0.0, 2.0, 0 };
            if (!in_region(w, g, &e)) continue;
            if (c == want && xy) { xy[0] = e.x; xy[1] = e.y; }
            ++c;
        }
    return c;
}

/* log of the birth proposal density (mass in lattice mode) at e: uniform on
 * cell n D x [0, T) with m - 2 ~ Exp(1), or its mixture with the learned
 * component (same magnitude law) */
static double log_qb(const orc_world* w, const region_t* g, const ev_t* e) {
    const orc_params* p = &w->p;
    if (p->lattice) {
        double nr = (double)lat_points(w, g, -1, NULL);
        return -log(nr) - log((double)p->lat_nt) - log((double)p->lat_nm);
    }
    double area = (g->r[1] - g->r[0]) * (g->r[3] - g->r[2]);
    if (!w->bt_nx || !(g->G > 0.0) || ORC_MUTANT == 5) return -log(area) - log(p->T) - (e->m - 2.0);
    const double qu = 1.0 / (area * p->T);
    if (!w->bt_mag)   /* both components draw m from the prior */
        return log((1.0 - w->bt_mix) * qu + w->bt_mix * q_net(w, g, e->x, e->y, e->t)) - (e->m - 2.0);
    /* the learned component draws m uniform on its entry's window */
    const double pm = exp(-(e->m - 2.0));
    double qm = 0.0;
    if (ORC_MUTANT == 6) {
        qm = pm;
    } else {
        const double lo = mag_lo(w, bt_entry(w, e->x, e->y, e->t));
        if (e->m >= lo && e->m < lo + 2.0 * w->bt_h) qm = 1.0 / (2.0 * w->bt_h);
    }
    return log((1.0 - w->bt_mix) * qu * pm + w->bt_mix * q_net(w, g, e->x, e->y, e->t) * qm);
}

/* a learned birth candidate: pixel by its share of the region's table mass,
 * uniform inside pixel n region, time bin by the pixel's cdf, uniform inside
 * the bin, and with magnitudes the magnitude uniform on the drawn entry's
 * window (words: pixel wd[2], x wd[3], y wd[8], bin wd[9], t wd[10], m
 * wd[11]); returns whether it drew the magnitude */
static int learned_birth(const orc_world* w, const region_t* g, const uint64_t* wd, ev_t* c) {
    int32_t x0, x1, y0, y1;
    pix_range(g->r[0], g->r[1], w->bt_hx, w->bt_nx, &x0, &x1);
    pix_range(g->r[2], g->r[3], w->bt_hy, w->bt_ny, &y0, &y1);
    const double target = u01(wd[2]) * g->G;
    double run = 0.0;
    int32_t px = -1, py = -1, lastx = -1, lasty = -1;
    for (int32_t iy = y0; iy <= y1; ++iy)
        for (int32_t ix = x0; ix <= x1; ++ix) {
            const double a = pix_weight(w, g, ix, iy);
            if (a <= 0.0) continue;
            run += a;
            lastx = ix;
            lasty = iy;
            if (px < 0 && run > target) { px = ix; py = iy; }
        }
    if (px < 0) { px = lastx; py = lasty; }   /* target reached the total by rounding */
    const double xa = (double)px * w->bt_hx, xb = (double)(px + 1) * w->bt_hx;
    const double ya = (double)py * w->bt_hy, yb = (double)(py + 1) * w->bt_hy;
    const double lx = xa > g->r[0] ? xa : g->r[0], hx = xb < g->r[1] ? xb : g->r[1];
    const double ly = ya > g->r[2] ? ya : g->r[2], hy = yb < g->r[3] ? yb : g->r[3];
    c->x = lx + u01(wd[3]) * (hx - lx);
    c->y = ly + u01(wd[8]) * (hy - ly);
    const double* cd = w->bt_cdf + ((int64_t)py * w->bt_nx + px) * w->bt_nt;
    const double ub = u01(wd[9]);
    int32_t b = 0;
    while (b < w->bt_nt - 1 && !(cd[b] > ub)) ++b;
    c->t = (double)b * w->bt_dt + u01(wd[10]) * w->bt_dt;
    if (!w->bt_mag) return 0;
    c->m = mag_lo(w, ((int64_t)py * w->bt_nx + px) * w->bt_nt + b) + u01(wd[11]) * (2.0 * w->bt_h);
    return 1;
}

/* Gaussian magnitude of a Box-Muller pair, rounded to a multiple of 2^-20 so
 * that platform differences in log/cos/sin below that grain cannot change a
 * coordinate; the sign comes from an independent bit, so the offset is
 * exactly symmetric. */
static double qgauss(double z) { return rint(fabs(z) * 1048576.0) * (1.0 / 1048576.0); }

typedef struct { int32_t type, valid; int64_t idx, idx2; int32_t slot; ev_t cand, cand2; } prop_t;

/* Philox counter of one step: key (seed, stream), counter (c0, c1, c2, .) */
typedef struct { uint64_t stream, c0, c1, c2; } ctr_t;

/* offset drawn from its prior N(0, sig_a^2) for station j and the step's
 * e-th changed event: one Philox block at counter word 16 + 2 j + e, a
 * Box-Muller cosine from its words 0 and 1 rounded like the walk offsets,
 * the sign from bit 0 of word 2 */
static double draw_offset(const orc_world* w, const ctr_t* c, int32_t j, int e) {
    uint64_t key[2] = { w->p.seed, c->stream };
    uint64_t ctr[4] = { c->c0, c->c1, c->c2, 16 + 2 * (uint64_t)j + (uint64_t)e };
    uint64_t o[4];
    orc_philox4x64(ctr, key, o);
    double z = qgauss(sqrt(-2.0 * log(u01o(o[0]))) * cos(2.0 * M_PI * u01(o[1])));
    if (o[2] & 1) z = -z;
    return w->p.sig_a * z;
}

/* offsets of an event that moves from `old` (NULL: a birth) to c's
 * coordinates: a station reached before and after keeps its offset, a newly
 * reached one draws it from the prior, one no longer reached drops it.  The
 * draws come from the prior, so their density cancels against the prior's
 * in every Hastings ratio. */
static void relocate(const orc_world* w, const ev_t* old, ev_t* c, const ctr_t* ctr, int e) {
    c->na = 0;
    if (!(w->p.sig_a > 0.0)) return;
    int32_t h = 0;
    for (int32_t j = 0; j < w->n_st; ++j) {
        if (!reaches(w, c, j)) continue;
        while (old && h < old->na && old->sta[h] < j) ++h;
        c->sta[c->na] = j;
        if (old && h < old->na && old->sta[h] == j) c->off[c->na] = old->off[h];
        else c->off[c->na] = ORC_MUTANT == 9 ? 0.0 : draw_offset(w, ctr, j, e);
        ++c->na;
    }
}

/* offset of a random-walk step: on a lattice one grid step along one of the
 * four axes (direction from wd[2]); otherwise independent Gaussians of
 * scales (sig_xy, sig_xy, sig_t, sig_m) by Box-Muller from wd[2..5], signs
 * from bits 32..35 of wd[1] */
static void walk_offset(const orc_world* w, const uint64_t* wd, double off[4]) {
    const orc_params* p = &w->p;
    off[0] = off[1] = off[2] = off[3] = 0.0;
    if (p->lattice) {
        int64_t dir = pick(wd[2], 8);
        double step = (dir & 1) ? -1.0 : 1.0;
        const double d[4] = { p->lat_dx, p->lat_dy, p->lat_dt, p->lat_dm };
        off[dir >> 1] = step * d[dir >> 1];
        return;
    }
    double r1 = sqrt(-2.0 * log(u01o(wd[2]))), th1 = 2.0 * M_PI * u01(wd[3]);
    double r2 = sqrt(-2.0 * log(u01o(wd[4]))), th2 = 2.0 * M_PI * u01(wd[5]);
    double z[4] = { qgauss(r1 * cos(th1)), qgauss(r1 * sin(th1)),
                    qgauss(r2 * cos(th2)), qgauss(r2 * sin(th2)) };
    for (int i = 0; i < 4; ++i)
        if ((wd[1] >> (32 + i)) & 1) z[i] = -z[i];
    off[0] = p->sig_xy * z[0];
    off[1] = p->sig_xy * z[1];
    off[2] = p->sig_t * z[2];
    off[3] = p->sig_m * z[3];
}

static prop_t decode_coords(const orc_world* w, const region_t* g, const uint64_t* wd,
                            const ev_t* own, int64_t n_own, int64_t n_total);

/* one step's proposal: coordinates, then the latent offsets the candidates
 * carry */
static prop_t decode(const orc_world* w, const region_t* g, const uint64_t* wd, const ctr_t* ctr,
                     const ev_t* own, int64_t n_own, int64_t n_total) {
    prop_t q = decode_coords(w, g, wd, own, n_own, n_total);
    if (!q.valid || !(w->p.sig_a > 0.0)) return q;
    if (q.type == 0) relocate(w, NULL, &q.cand, ctr, 0);
    else if (q.type == 2) relocate(w, &own[q.idx], &q.cand, ctr, 0);
    else if (q.type == 3) {
        relocate(w, &own[q.idx], &q.cand, ctr, 0);
        relocate(w, &own[q.idx2], &q.cand2, ctr, 1);
    }
    return q;
}

static prop_t decode_coords(const orc_world* w, const region_t* g, const uint64_t* wd,
                            const ev_t* own, int64_t n_own, int64_t n_total) {
    const orc_params* p = &w->p;
    prop_t q;
    memset(&q, 0, sizeof(q));
    double u = u01(wd[0]);
    const double cb = p->p_birth, cd = cb + p->p_death, cp = cd + p->p_pair, ca = cp + p->p_arr;
    q.type = u < cb ? 0 : (u < cd ? 1 : (u < cp ? 3 : (u < ca ? 4 : 2)));
    q.idx = -1;
    q.idx2 = -1;
    q.slot = -1;
    if (q.type == 0) {
        if (p->lattice) {
            if (n_total >= p->lat_nmax) return q;
            int64_t nr = lat_points(w, g, -1, NULL);
            if (nr == 0) return q;
            double xy[2];
            lat_points(w, g, pick(wd[2], nr), xy);
            q.cand.x = xy[0]; q.cand.y = xy[1];
            q.cand.t = p->lat_t0 + (double)pick(wd[3], p->lat_nt) * p->lat_dt;
            q.cand.m = p->lat_m0 + (double)pick(wd[4], p->lat_nm) * p->lat_dm;
        } else if (w->bt_nx && g->G > 0.0 && u01(wd[7]) < w->bt_mix) {
            if (!learned_birth(w, g, wd, &q.cand)) q.cand.m = 2.0 - log(u01o(wd[5]));
        } else {
            q.cand.x = g->r[0] + u01(wd[2]) * (g->r[1] - g->r[0]);
            q.cand.y = g->r[2] + u01(wd[3]) * (g->r[3] - g->r[2]);
            q.cand.t = u01(wd[4]) * p->T;
            q.cand.m = 2.0 - log(u01o(wd[5]));
        }
        q.valid = in_region(w, g, &q.cand) && in_time_mag(w, &q.cand);
        return q;
    }
    if (q.type == 4) {
        /* arrival-time move (§MH moves, "Arrival Time Move"): event i from
         * wd[1], one of the stations it reaches from wd[7], its offset moved
         * by sig_da times a Gaussian (Box-Muller cosine of wd[2], wd[3],
         * rounded, sign from bit 32 of wd[1]) */
        if (n_own == 0) return q;
        q.idx = pick(wd[1], n_own);
        const ev_t* e = &own[q.idx];
        if (e->na == 0) return q;
        q.slot = (int32_t)pick(wd[7], e->na);
        double z = qgauss(sqrt(-2.0 * log(u01o(wd[2]))) * cos(2.0 * M_PI * u01(wd[3])));
        if ((wd[1] >> 32) & 1) z = -z;
        q.cand = *e;
        q.cand.off[q.slot] += p->sig_da * z;
        q.valid = 1;
        return q;
    }
    if (q.type == 3) {
        /* joint move (§MH moves, "Joint Events Move"): an ordered pair of
         * distinct events, i from wd[1] and j from wd[7] among the others.
         * Bit 36 of wd[1] clear: the pair's other mode under the station
         * geometry, the two events exchanging their locations while each
         * keeps its origin time and magnitude (stations equidistant from the
         * two see the same arrivals); set: both shifted by one common
         * random-walk offset. */
        if (n_own < 2) return q;
        q.idx = pick(wd[1], n_own);
        const int64_t j = pick(wd[7], n_own - 1);
        q.idx2 = j + (j >= q.idx ? 1 : 0);
        q.cand = own[q.idx];
        q.cand2 = own[q.idx2];
        if (((wd[1] >> 36) & 1) == 0) {
            q.cand.x = own[q.idx2].x; q.cand.y = own[q.idx2].y;
            q.cand2.x = own[q.idx].x; q.cand2.y = own[q.idx].y;
        } else {
            double off[4];
            walk_offset(w, wd, off);
            q.cand.x += off[0]; q.cand.y += off[1]; q.cand.t += off[2]; q.cand.m += off[3];
            q.cand2.x += off[0]; q.cand2.y += off[1]; q.cand2.t += off[2]; q.cand2.m += off[3];
        }
        q.valid = in_region(w, g, &q.cand) && in_time_mag(w, &q.cand) &&
                  in_region(w, g, &q.cand2) && in_time_mag(w, &q.cand2);
        return q;
    }
    if (n_own == 0) return q;
    q.idx = pick(wd[1], n_own);
    if (q.type == 1) { q.valid = 1; return q; }
    q.cand = own[q.idx];
    double off[4];
    walk_offset(w, wd, off);
    q.cand.x += off[0];
    q.cand.y += off[1];
    q.cand.t += off[2];
    q.cand.m += off[3];
    q.valid = in_region(w, g, &q.cand) && in_time_mag(w, &q.cand);
    return q;
}

/* log acceptance ratio (MH, §Background / Algorithm "Serial Metropolis
 * Hastings"): log pi(x') - log pi(x) + log q(x | x') - log q(x' | x), with
 * pi the Poisson-process posterior and the proposal restricted to the region.
 *   birth:  dll + log beta(c) - log q_b(c) + log p_d - log(n+1) - log p_b
 *   death:  dll - log beta(e) + log q_b(e) + log p_b - log p_d + log n
 *   move:   dll + log beta(c) - log beta(e)        (symmetric offset)
 *   pair:   dll + sum over the two of log beta(c) - log beta(e): the exchange
 *           is its own inverse, the common offset is symmetric, and the
 *           ordered pair is drawn with probability 1/(n (n-1)) both ways
 *   arrival: dll + log N(delta'; 0, sig_a^2) - log N(delta; 0, sig_a^2)
 *           (symmetric step of one offset)
 * Latent offsets drawn from their prior (a birth's, those of stations a
 * moved event newly reaches) and those dropped (a death's, stations no longer
 * reached) have proposal density equal to their prior density, so their
 * terms cancel from every ratio above.
 */
static double log_alpha_of(const orc_world* w, const region_t* g, const prop_t* q,
                           const ev_t* own, int64_t n_own, const ev_t* oth, int64_t n_oth,
                           double* dll_out, double* dlp_out) {
    const orc_params* p = &w->p;
    double dll, dlp, la, dlo = 0.0;
    if (q->type == 0) {
        dll = delta_ll2(w, own, n_own, oth, n_oth, -1, &q->cand);
        dlp = log_beta(w, &q->cand);
        la = dll + dlp - log_qb(w, g, &q->cand) + log(p->p_death)
             - log((double)(n_own + (ORC_MUTANT == 1 ? 2 : 1))) - log(p->p_birth);
        dlo = log_off_prior(w, &q->cand);
    } else if (q->type == 1) {
        const ev_t* e = &own[q->idx];
        dll = delta_ll2(w, own, n_own, oth, n_oth, q->idx, NULL);
        dlp = -log_beta(w, e);
        la = dll + dlp + (ORC_MUTANT == 2 ? 0.0 : log_qb(w, g, e)) + log(p->p_birth) - log(p->p_death)
             + log((double)n_own);
        dlo = -log_off_prior(w, e);
    } else if (q->type == 3) {
        dll = delta_ll_pair(w, own, n_own, oth, n_oth, q->idx, q->idx2, &q->cand, &q->cand2);
        dlp = (log_beta(w, &q->cand) - log_beta(w, &own[q->idx])) +
              (log_beta(w, &q->cand2) - log_beta(w, &own[q->idx2]));
        la = dll + (ORC_MUTANT == 7 ? 0.0 : dlp);
        dlo = (log_off_prior(w, &q->cand) - log_off_prior(w, &own[q->idx])) +
              (log_off_prior(w, &q->cand2) - log_off_prior(w, &own[q->idx2]));
    } else if (q->type == 4) {
        /* symmetric offset step: the prior ratio of the one offset */
        dll = delta_ll2(w, own, n_own, oth, n_oth, q->idx, &q->cand);
        const double s2 = p->sig_a * p->sig_a, a = own[q->idx].off[q->slot], b = q->cand.off[q->slot];
        dlp = (a * a - b * b) / (2.0 * s2);
        la = dll + (ORC_MUTANT == 8 ? 0.0 : dlp);
    } else {
        dll = delta_ll2(w, own, n_own, oth, n_oth, q->idx, &q->cand);
        dlp = log_beta(w, &q->cand) - log_beta(w, &own[q->idx]);
        la = dll + (ORC_MUTANT == 4 ? 0.0 : dlp);
        dlo = log_off_prior(w, &q->cand) - log_off_prior(w, &own[q->idx]);
    }
    /* offsets drawn from their prior cancel against it in la (births, the
     * stations a moved event newly reaches); the log-density change still
     * counts them */
    *dll_out = dll;
    *dlp_out = dlp + dlo;
    return la;
}

/* ------------------------------------------------------------------------
 * region runner: k MH steps on the region's own events with the others fixed
 * ---------------------------------------------------------------------- */
typedef struct { ev_t* e; int64_t n, cap; } vec_t;

static void vec_push(vec_t* v, const ev_t* e) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 16;
        v->e = (ev_t*)realloc(v->e, sizeof(ev_t) * (size_t)v->cap);
    }
    v->e[v->n++] = *e;
}

static void apply(vec_t* own, const prop_t* q, uint64_t new_id) {
    if (q->type == 0) {
        ev_t e = q->cand;
        e.id = new_id;
        vec_push(own, &e);
    } else if (q->type == 1) {
        for (int64_t i = q->idx; i + 1 < own->n; ++i) own->e[i] = own->e[i + 1];
        own->n--;
    } else {
        uint64_t id = own->e[q->idx].id;
        own->e[q->idx] = q->cand;
        own->e[q->idx].id = id;
        if (q->type == 3) {
            id = own->e[q->idx2].id;
            own->e[q->idx2] = q->cand2;
            own->e[q->idx2].id = id;
        }
    }
}

/* one MH step; stream/c0/c1/c2 select the Philox counter */
static void mh_step(const orc_world* w, const region_t* g, vec_t* own, const ev_t* oth, int64_t n_oth,
                    int64_t n_total_other, uint64_t stream, uint64_t c0, uint64_t c1, uint64_t c2,
                    uint64_t new_id, orc_trace* tr, double* dlogp) {
    uint64_t wd[12];
    step_words(w, stream, c0, c1, c2, wd);
    const ctr_t ctr = { stream, c0, c1, c2 };
    prop_t q = decode(w, g, wd, &ctr, own->e, own->n, own->n + n_total_other);
    double dll = 0.0, dlp = 0.0, la = -INFINITY;
    int acc = 0;
    if (tr) {
        tr->type = q.type;
        tr->n_before = (int32_t)own->n;
        tr->evaluated = q.valid;
    }
    if (q.valid) {
        la = log_alpha_of(w, g, &q, own->e, own->n, oth, n_oth, &dll, &dlp);
        acc = log(u01o(wd[6])) < la;
    }
    if (tr) {
        tr->accepted = acc;
        tr->dll = dll;
        tr->log_alpha = la;
    }
    if (acc && w->p.commit) {
        apply(own, &q, new_id);
        *dlogp += dll + dlp;
    }
}

double orc_log_alpha_off(const orc_world* w, double sx, double sy, int32_t cell,
                         const double* ev, const double* off, int64_t n, int32_t type, int64_t idx,
                         int32_t station, const double* cand, const double* cand_off, int32_t* valid) {
    region_t g;
    g.cell = cell; g.sx = sx; g.sy = sy;
    if (cell < 0) { g.r[0] = 0.0; g.r[1] = w->p.W; g.r[2] = 0.0; g.r[3] = w->p.W; }
    else orc_cell_rect(w, sx, sy, cell, g.r);
    region_bt(w, &g);
    vec_t own = { 0, 0, 0 }, oth = { 0, 0, 0 };
    for (int64_t i = 0; i < n; ++i) {
        ev_t e; to_ev(ev + 4 * i, &e);
        fill_offsets(w, &e, off ? off + (size_t)i * (size_t)w->n_st : NULL);
        e.id = (uint64_t)i;
        if (cell < 0 || orc_cell_of(w, sx, sy, e.x, e.y) == cell) vec_push(&own, &e);
        else vec_push(&oth, &e);
    }
    prop_t q;
    memset(&q, 0, sizeof(q));
    q.type = type;
    q.idx = idx;
    q.slot = -1;
    q.valid = 1;
    if (type != 0 && (idx < 0 || idx >= own.n)) q.valid = 0;
    if (type == 4) {
        if (q.valid) {
            q.cand = own.e[idx];
            for (int32_t k = 0; k < q.cand.na; ++k)
                if (q.cand.sta[k] == station) q.slot = k;
            if (q.slot < 0 || !cand_off) q.valid = 0;
            else q.cand.off[q.slot] = cand_off[0];
        }
    } else {
        if (cand) {
            to_ev(cand, &q.cand);
            fill_offsets(w, &q.cand, cand_off);
        }
        if (type == 0 && w->p.lattice && n >= w->p.lat_nmax) q.valid = 0;
        if (type != 1 && q.valid) q.valid = in_region(w, &g, &q.cand) && in_time_mag(w, &q.cand);
    }
    double la = -INFINITY, dll, dlp;
    if (q.valid) la = log_alpha_of(w, &g, &q, own.e, own.n, oth.e, oth.n, &dll, &dlp);
    *valid = q.valid;
    free(own.e);
    free(oth.e);
    return la;
}

double orc_log_alpha(const orc_world* w, double sx, double sy, int32_t cell,
                     const double* ev, int64_t n, int32_t type, int64_t idx,
                     const double* cand, int32_t* valid) {
    return orc_log_alpha_off(w, sx, sy, cell, ev, NULL, n, type, idx, -1, cand, NULL, valid);
}

double orc_log_alpha_pair(const orc_world* w, double sx, double sy, int32_t cell,
                          const double* ev, int64_t n, int64_t i, int64_t j,
                          const double* cand1, const double* cand2, int32_t* valid) {
    region_t g;
    g.cell = cell; g.sx = sx; g.sy = sy;
    if (cell < 0) { g.r[0] = 0.0; g.r[1] = w->p.W; g.r[2] = 0.0; g.r[3] = w->p.W; }
    else orc_cell_rect(w, sx, sy, cell, g.r);
    region_bt(w, &g);
    vec_t own = { 0, 0, 0 }, oth = { 0, 0, 0 };
    for (int64_t q = 0; q < n; ++q) {
        ev_t e; to_ev(ev + 4 * q, &e);
        fill_offsets(w, &e, NULL);
        e.id = (uint64_t)q;
        if (cell < 0 || orc_cell_of(w, sx, sy, e.x, e.y) == cell) vec_push(&own, &e);
        else vec_push(&oth, &e);
    }
    prop_t q;
    memset(&q, 0, sizeof(q));
    q.type = 3;
    q.idx = i;
    q.idx2 = j;
    to_ev(cand1, &q.cand);
    to_ev(cand2, &q.cand2);
    fill_offsets(w, &q.cand, NULL);
    fill_offsets(w, &q.cand2, NULL);
    q.valid = i >= 0 && i < own.n && j >= 0 && j < own.n && i != j &&
              in_region(w, &g, &q.cand) && in_time_mag(w, &q.cand) &&
              in_region(w, &g, &q.cand2) && in_time_mag(w, &q.cand2);
    double la = -INFINITY, dll, dlp;
    if (q.valid) la = log_alpha_of(w, &g, &q, own.e, own.n, oth.e, oth.n, &dll, &dlp);
    *valid = q.valid;
    free(own.e);
    free(oth.e);
    return la;
}

/* ------------------------------------------------------------------------
 * Serial MH (Algorithm "Serial Metropolis Hastings"): the whole domain is one
 * region; Philox stream 2, counter (step, 0, 0, 0|1).
 * ---------------------------------------------------------------------- */
int orc_run_serial(const orc_world* w, orc_set* s, int64_t step0, int64_t n_steps,
                   orc_trace* trace, int64_t trace_cap, int64_t* n_trace, double* dlogp) {
    region_t g;
    g.cell = -1; g.sx = 0.0; g.sy = 0.0;
    g.r[0] = 0.0; g.r[1] = w->p.W; g.r[2] = 0.0; g.r[3] = w->p.W;
    region_bt(w, &g);
    vec_t own = { s->e, s->n, s->cap };
    double acc_lp = 0.0;
    int64_t nt = 0;
    for (int64_t i = 0; i < n_steps; ++i) {
        int64_t step = step0 + i;
        orc_trace* tr = (trace && nt < trace_cap) ? &trace[nt] : NULL;
        if (tr) {
            memset(tr, 0, sizeof(*tr));
            tr->sweep = (int32_t)(step >> 31);
            tr->cell = -1;
            tr->step = (int32_t)(step & 0x7fffffff);
        }
        uint64_t new_id = 0x8000000000000000ULL | (uint64_t)step;
        mh_step(w, &g, &own, NULL, 0, 0, 2, (uint64_t)step, 0, 0, new_id, tr, &acc_lp);
        ++nt;
    }
    s->e = own.e; s->n = own.n; s->cap = own.cap;
    if (n_trace) *n_trace = nt;
    if (dlogp) *dlogp = acc_lp;
    return 0;
}

/* ------------------------------------------------------------------------
 * Chromatic MH (Algorithm "Chromatic MH with Static Coloring"; with
 * shift_mode = 1 the boundaries move by a fresh uniform offset before every
 * sweep, §Chromatic MH with Dynamic Coloring).  Within a sweep the colours run
 * in order 0..p^2-1; the regions of one colour are independent and may run on
 * several threads.  Region r runs k steps with Philox stream 0, counter
 * (sweep, r, step, 0|1).  Births get id (sweep+1) << 32 | r << 12 | step,
 * which keeps every region's events sorted by id.
 * ---------------------------------------------------------------------- */
static int cmp_cell_id(const void* a, const void* b) {
    const int64_t* x = (const int64_t*)a;
    const int64_t* y = (const int64_t*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if ((uint64_t)x[1] != (uint64_t)y[1]) return (uint64_t)x[1] < (uint64_t)y[1] ? -1 : 1;
    return 0;
}

int orc_run_chromatic(const orc_world* w, orc_set* s, int64_t sweep0, int64_t n_sweeps,
                      int32_t shift_mode, double sx_static, double sy_static,
                      orc_trace* trace, int64_t trace_cap, int64_t* n_trace,
                      int32_t n_threads, double* dlogp) {
    int32_t ncx, ncy;
    orc_grid_dims(w, &ncx, &ncy);
    const int32_t nc = ncx * ncy, per = orc_period(w), ncol = per * per;
    const int32_t k = w->p.k_per_phase;
    if (2.0 * w->p.R_max > (double)(per - 1) * w->p.L) return -1;
    if (k >= 4096 || nc >= (1 << 20)) return -2;
    vec_t* cells = (vec_t*)calloc((size_t)nc, sizeof(vec_t));
    int32_t* regs = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
    double* reg_lp = (double*)malloc(sizeof(double) * (size_t)nc);
    double total_lp = 0.0;
    int64_t nt = 0;
    int rc = 0;
    for (int64_t sw = sweep0; sw < sweep0 + n_sweeps; ++sw) {
        double sx = sx_static, sy = sy_static;
        if (shift_mode == 1) orc_shift(w, sw, &sx, &sy);
        /* bin events into cells, each cell sorted by id */
        int64_t* key = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(s->n > 0 ? s->n : 1));
        for (int64_t i = 0; i < s->n; ++i) {
            int32_t c = orc_cell_of(w, sx, sy, s->e[i].x, s->e[i].y);
            if (c < 0) { rc = -3; free(key); goto done; }
            key[3 * i] = c;
            key[3 * i + 1] = (int64_t)s->e[i].id;
            key[3 * i + 2] = i;
        }
        qsort(key, (size_t)s->n, sizeof(int64_t) * 3, cmp_cell_id);
        for (int32_t c = 0; c < nc; ++c) cells[c].n = 0;
        for (int64_t i = 0; i < s->n; ++i) vec_push(&cells[key[3 * i]], &s->e[key[3 * i + 2]]);
        free(key);

        for (int32_t col = 0; col < ncol; ++col) {
            int32_t nr = 0;
            for (int32_t c = 0; c < nc; ++c) {
                double r[4];
                orc_cell_rect(w, sx, sy, c, r);
                if (orc_colour_of(w, c) == col && cell_live(r)) regs[nr++] = c;
            }
            int64_t tbase = nt;
            int use_threads = (n_threads > 1 && !w->p.lattice) ? n_threads : 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(use_threads)
#endif
            for (int32_t ri = 0; ri < nr; ++ri) {
                int32_t c = regs[ri];
                region_t g;
                g.cell = c; g.sx = sx; g.sy = sy;
                orc_cell_rect(w, sx, sy, c, g.r);
                region_bt(w, &g);
                /* the region's Markov blanket: events of cells within per-1 */
                vec_t oth = { 0, 0, 0 };
                int32_t ix = c % ncx, iy = c / ncx;
                for (int32_t jy = iy - (per - 1); jy <= iy + (per - 1); ++jy)
                    for (int32_t jx = ix - (per - 1); jx <= ix + (per - 1); ++jx) {
                        if (jx < 0 || jy < 0 || jx >= ncx || jy >= ncy) continue;
                        int32_t cc = jy * ncx + jx;
                        if (cc == c) continue;
                        for (int64_t i = 0; i < cells[cc].n; ++i) vec_push(&oth, &cells[cc].e[i]);
                    }
                double lp = 0.0;
                /* lattice cap on the total count (lattice mode runs regions in order) */
                int64_t n_other_world = 0;
                if (w->p.lattice)
                    for (int32_t cc = 0; cc < nc; ++cc)
                        if (cc != c) n_other_world += cells[cc].n;
                for (int32_t st = 0; st < k; ++st) {
                    int64_t ti = tbase + (int64_t)ri * k + st;
                    orc_trace* tr = (trace && ti < trace_cap) ? &trace[ti] : NULL;
                    if (tr) {
                        memset(tr, 0, sizeof(*tr));
                        tr->sweep = (int32_t)sw;
                        tr->cell = c;
                        tr->step = st;
                    }
                    uint64_t new_id = ((uint64_t)(sw + 1) << 32) | ((uint64_t)c << 12) | (uint64_t)st;
                    mh_step(w, &g, &cells[c], oth.e, oth.n, n_other_world, 0,
                            (uint64_t)sw, (uint64_t)c, (uint64_t)st, new_id, tr, &lp);
                }
                free(oth.e);
                reg_lp[ri] = lp;
            }
            for (int32_t ri = 0; ri < nr; ++ri) total_lp += reg_lp[ri];
            nt += (int64_t)nr * k;
        }
        /* flatten back, cell order then id */
        int64_t n_new = 0;
        for (int32_t c = 0; c < nc; ++c) n_new += cells[c].n;
        if (n_new > s->cap) {
            s->cap = n_new + 16;
            s->e = (ev_t*)realloc(s->e, sizeof(ev_t) * (size_t)s->cap);
        }
        s->n = 0;
        for (int32_t c = 0; c < nc; ++c)
            for (int64_t i = 0; i < cells[c].n; ++i) s->e[s->n++] = cells[c].e[i];
    }
done:
    for (int32_t c = 0; c < nc; ++c) free(cells[c].e);
    free(cells);
    free(regs);
    free(reg_lp);
    if (n_trace) *n_trace = nt;
    if (dlogp) *dlogp = total_lp;
    return rc;
}
