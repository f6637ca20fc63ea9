/*
 * CPU oracle for spatially partitioned chromatic Metropolis-Hastings on the
 * toy seismic model.  TEST INFRASTRUCTURE ONLY: it is used by tests/, by
 * __graft_entry__.smoke() and by bench.py's CPU-baseline leg, never by the
 * library.  It shares no code with the CUDA path.
 *
 * What it computes (all in float64, plain loops, no blocking or fusion):
 *   - the model's log-density (event prior, Gaussian signal likelihood whose
 *     per-sample variance is noise plus the arriving signals' variances)
 *     -- §Generative Model of Seismic Signals, the joint P(e, a, s);
 *   - the change of the log-likelihood for one birth / death / move proposal,
 *     and for the joint move of a pair of events, as the difference of two
 *     sums of Gaussian log-densities;
 *   - Serial Metropolis-Hastings (Algorithm "Serial Metropolis Hastings");
 *   - Chromatic MH with static colouring and with dynamic colouring
 *     (Algorithm "Chromatic Metropolis Hastings with Static Coloring", and
 *     §Chromatic MH with Dynamic Coloring: a uniform boundary shift per sweep);
 *   - the spatial partition, its colouring and the regions' station blankets
 *     (§Partitioning the World);
 *   - Philox4x64-10 (Salmon et al., SC'11), the counter-based generator both
 *     sides implement from its published definition.
 */
#ifndef CHROMH_ORACLE_H
#define CHROMH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double W, T, Lambda, v, alpha, beta_att, tau, t_s, noise_var, f_hz, R_max, L;
    double p_birth, p_death, sig_xy, sig_t, sig_m;
    int32_t n_w;          /* samples per arrival window (t_s * f_hz) */
    int32_t k_per_phase;  /* MH steps per region per colour phase */
    uint64_t seed;
    int32_t commit;       /* 1: apply accepted proposals; 0: price only */
    /* lattice mode (exact-enumeration tests): coordinates on a finite grid */
    int32_t lattice;
    int32_t lat_nx, lat_ny, lat_nt, lat_nm, lat_nmax;
    int32_t likelihood;   /* 0: arrivals add to the variance of a zero-mean sample;
                             1: they add to its mean, the variance is the noise's */
    double lat_x0, lat_dx, lat_y0, lat_dy, lat_t0, lat_dt, lat_m0, lat_dm;
    /* probability of the joint move of a pair of the region's events (§MH
     * moves, "Joint Events Move"); proposals with u in [p_birth + p_death,
     * p_birth + p_death + p_pair) take it, the Gaussian move keeps the rest */
    double p_pair;
    /* latent arrival times (§Generative Model, Event Detections): the arrival
     * of an event at a station it reaches is t + d/v + delta with delta ~
     * N(0, sig_a^2), one latent delta per (event, reached station); sig_a = 0
     * is the deterministic model (no latent offsets).  p_arr is the share of
     * steps that propose the arrival-time move (one delta changed by a
     * Gaussian of scale sig_da; §MH moves, "Arrival Time Move"); it follows
     * p_pair in the proposal mix */
    double sig_a, p_arr, sig_da;
} orc_params;

typedef struct {
    int32_t sweep, cell, step, type;   /* type: 0 birth, 1 death, 2 move, 3 pair, 4 arrival */
    int32_t evaluated, accepted, n_before, pad;
    double dll, log_alpha;
} orc_trace;

typedef struct orc_world orc_world;
typedef struct orc_set orc_set;

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

orc_world* orc_world_new(const orc_params* p, const double* stations, int32_t n_st,
                         const void* signals, int32_t signals_f32, int64_t n_samp, int64_t pitch);
void orc_world_free(orc_world* w);
/* learned birth component: weights tab[(iy * nx + ix) * nt + b] over pixels of
 * [0,W)^2 and time bins of [0,T), mixing weight mix in (0, 1); nx == 0
 * removes it.  Returns 0, or -1 for bad arguments. */
int orc_set_birth_table(orc_world* w, const float* tab, int32_t nx, int32_t ny, int32_t nt, double mix);
int orc_set_birth_magnitude(orc_world* w, const float* centre, double half_width);

orc_set* orc_set_new(const double* ev, const uint64_t* ids, int64_t n);
int64_t orc_set_size(const orc_set* s);
void orc_set_get(const orc_set* s, double* ev, uint64_t* ids);
void orc_set_free(orc_set* s);

double orc_log_prior(const orc_world* w, const double* ev, int64_t n);
double orc_log_likelihood(const orc_world* w, const double* ev, int64_t n);
/* V at station j for samples [k0, k1) under event set ev (definition). */
void orc_variance(const orc_world* w, const double* ev, int64_t n, int32_t j,
                  int64_t k0, int64_t k1, double* out);
/* The same with latent arrival offsets: off is a dense [n][n_st] array of
 * the events' offsets (entries of stations an event does not reach are
 * ignored; NULL: all 0).  The prior adds log N(delta; 0, sig_a^2) for every
 * (event, reached station) when sig_a > 0. */
double orc_log_prior_off(const orc_world* w, const double* ev, const double* off, int64_t n);
double orc_log_likelihood_off(const orc_world* w, const double* ev, const double* off, int64_t n);
/* Log-likelihood change when event old_idx of ev is removed (-1: none) and
 * cand is added (NULL: none). */
double orc_delta_loglik(const orc_world* w, const double* ev, int64_t n,
                        int64_t old_idx, const double* cand);

/* partition */
int32_t orc_period(const orc_world* w);
void orc_grid_dims(const orc_world* w, int32_t* ncx, int32_t* ncy);
int32_t orc_cell_of(const orc_world* w, double sx, double sy, double x, double y);
void orc_cell_rect(const orc_world* w, double sx, double sy, int32_t cell, double* r4);
int32_t orc_colour_of(const orc_world* w, int32_t cell);
void orc_shift(const orc_world* w, int64_t sweep, double* sx, double* sy);
/* blanket membership as a dense [n_cells][n_st] 0/1 matrix */
void orc_blankets(const orc_world* w, double sx, double sy, uint8_t* member);

/* log acceptance ratio of one explicit proposal restricted to region `cell`
 * (cell = -1: the serial sampler over the whole domain). type 0 birth of
 * cand, 1 death of the idx-th event of the region, 2 move of it to cand.
 * *valid = 0 when the proposal is rejected without evaluation. */
double orc_log_alpha(const orc_world* w, double sx, double sy, int32_t cell,
                     const double* ev, int64_t n, int32_t type, int64_t idx,
                     const double* cand, int32_t* valid);

/* log acceptance ratio of one explicit joint move: the i-th and j-th events
 * of the region (i != j) become cand1 and cand2. */
double orc_log_alpha_pair(const orc_world* w, double sx, double sy, int32_t cell,
                          const double* ev, int64_t n, int64_t i, int64_t j,
                          const double* cand1, const double* cand2, int32_t* valid);

/* log acceptance ratio of one explicit proposal with latent offsets: as
 * orc_log_alpha for types 0-2 (off, cand_off: dense offsets of the events
 * and of the candidate, NULL = 0), and type 4, the arrival-time move of the
 * idx-th event of the region at station `station` to the offset cand_off[0]. */
double orc_log_alpha_off(const orc_world* w, double sx, double sy, int32_t cell,
                         const double* ev, const double* off, int64_t n, int32_t type, int64_t idx,
                         int32_t station, const double* cand, const double* cand_off, int32_t* valid);
/* event sets with their latent offsets (dense [n][n_st], NULL = 0): the set
 * keeps the offsets of the stations each event reaches */
orc_set* orc_set_new_w(const orc_world* w, const double* ev, const uint64_t* ids, const double* off,
                       int64_t n);
void orc_set_offsets(const orc_world* w, const orc_set* s, double* off);

/* samplers; return 0 on success */
int orc_run_serial(const orc_world* w, orc_set* s, int64_t step0, int64_t n_steps,
                   orc_trace* trace, int64_t trace_cap, int64_t* n_trace, double* dlogp);
int orc_run_chromatic(const orc_world* w, orc_set* s, int64_t sweep0, int64_t n_sweeps,
                      int32_t shift_mode, double sx, double sy,
                      orc_trace* trace, int64_t trace_cap, int64_t* n_trace,
                      int32_t n_threads, double* dlogp);

#ifdef __cplusplus
}
#endif
#endif
