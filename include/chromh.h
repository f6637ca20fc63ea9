/*
 * chromh -- chromatic Metropolis-Hastings with dynamic spatial partitioning
 * for the toy seismic event model, on one GB300 (sm_103a).
 *
 * The calls follow the paper's inference problem (Song & Moore, "Parallel
 * Chromatic MCMC with Spatial Partitioning", §Generative Model of Seismic
 * Signals): from the noisy signals recorded at the stations, infer how many
 * events there were and where and when each happened:
 *   cmh_create_model         events, stations, signals -> model
 *   cmh_partition_and_color  region grid + boundary shift (§Partitioning the
 *                            World; §Chromatic MH with Dynamic Coloring)
 *   cmh_run_sweeps           n sweeps of Algorithm "Chromatic MH with Static
 *                            Coloring" (a fresh shift per sweep when dynamic)
 *   cmh_read_state           the current event hypothesis and log-density
 *
 * Model (all lengths km, times s):
 *   event (x, y, t, m) in [0,W)^2 x [0,T) x [2, inf), Poisson prior with mean
 *   count Lambda, uniform location and time, m - 2 ~ Exp(1);
 *   arrival at a station at distance d: a = t + d / v; reach iff d < R_max;
 *   at sample k (time k / f_hz, k in [ceil(a f), ceil(a f) + t_s f)) the
 *   station's variance grows by (exp(alpha m - beta_att d) exp(-(k/f - a)/tau))^2;
 *   each sample s ~ N(0, noise_var + sum of those variances).
 * Options (cmh_params): the additive reading (likelihood = 1: arrivals add
 * the enveloped amplitude to the sample's mean, float32), latent arrival
 * times (sig_a > 0: a = t + d / v + delta, delta ~ N(0, sig_a^2) per event and
 * reached station) and the joint move of a pair (p_pair), both in either
 * precision under the variance reading.
 *
 * Conventions for every call:
 *   - return 0 (CMH_OK) or a negative CMH_ERR_* code; nothing throws across
 *     the ABI; cmh_strerror() names the code;
 *   - a model is driven by one host thread at a time;
 *   - device-side errors (a capacity exceeded inside a kernel) are latched in
 *     the model and returned by the next call that synchronises
 *     (cmh_read_state, cmh_sync, ...); once latched the model refuses work;
 *   - all device work is ordered on the model's CUDA stream.
 */
#ifndef CHROMH_H
#define CHROMH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CMH_OK 0
#define CMH_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, non-finite parameter) */
#define CMH_ERR_GEOMETRY (-2)  /* R_max too large for the colour pattern of the grid */
#define CMH_ERR_NONFINITE (-3) /* a signal sample or event coordinate is NaN/Inf */
#define CMH_ERR_OOM (-4)       /* device allocation failed */
#define CMH_ERR_CAPACITY (-5)  /* a fixed capacity (events, blanket, arrivals) was exceeded */
#define CMH_ERR_TIMEOUT (-6)   /* a bounded device wait gave up */
#define CMH_ERR_CUDA (-7)      /* a CUDA runtime call failed */
#define CMH_ERR_STATE (-8)     /* call out of order (e.g. run before partition) or error latched */

typedef struct cmh_model cmh_model;

/* one event: epicentre (km), origin time (s), magnitude */
typedef struct { double x, y, t, m; } cmh_event;
/* one station (km) */
typedef struct { double x, y; } cmh_station;

typedef enum { CMH_F64 = 0, CMH_F32 = 1 } cmh_dtype;

typedef struct {
    /* model (see the header comment) */
    double W, T, Lambda, v, alpha, beta_att, tau, t_s, noise_var, f_hz, R_max;
    /* proposal mix and random-walk steps (km, s, magnitude units) */
    double p_birth, p_death, sig_xy, sig_t, sig_m;
    int32_t k_per_phase;   /* MH steps per region per colour phase (1..4095) */
    int32_t commit;        /* 1: accepted proposals change the state; 0: price only */
    uint64_t seed;         /* key of every Philox stream */
    cmh_dtype dtype;       /* arithmetic of per-sample terms: CMH_F64 (replay) or CMH_F32 */
    int32_t ev_capacity;   /* max events one region may hold in a phase; 0: 128 */
    int32_t frozen_capacity; /* max arrivals listed per blanket station in a phase
                                (neighbouring regions', plus the region's own in the
                                float32 form); 0: 64 */
    int32_t block_threads; /* threads per region CTA (64..512, multiple of 32); 0: 256 */
    int32_t stage_samples; /* float32 form: samples per shared-memory buffer into which the
                              station windows of the next step are staged by bulk copies
                              while the current step is priced; 0: no staging (windows are
                              read from global memory); -1: one window, cut down to what
                              keeps three CTAs resident per SM; > 0: that many (rounded
                              down to a multiple of 4) */
    int32_t schedule;      /* float32 form: 0 = one persistent launch per sweep in which each
                              region waits only for its neighbouring regions of lower colours
                              (same results as colour by colour, shorter tails); 1 = one launch
                              per colour phase.  The float64 form always runs colour by colour */
    int32_t ctas_per_sm;   /* schedule 0: resident CTAs per SM of the persistent launch
                              (1..3; 0: as many as fit, at most 3) */
    int32_t likelihood;    /* 0: an arrival adds (A g(u))^2 to the variance of a zero-mean
                              sample (the default reading); 1 (CMH_F32 only): it adds A g(u)
                              to the sample's mean and the variance is noise_var (the
                              additive reading) */
    int64_t max_events;    /* capacity of the whole event store; 0: 4 (n0 + Lambda) + 4096 */
    double p_pair;         /* probability of the joint move of a pair of the
                              region's events (§MH moves, "Joint Events Move"); a step whose
                              uniform falls in [p_birth + p_death, p_birth + p_death + p_pair)
                              takes it, the Gaussian move keeps the rest.  The ordered pair
                              (i, j), i != j, is drawn uniformly; then with probability 1/2
                              the two exchange their locations (each keeps its origin time and
                              magnitude: the other mode for stations near the pair's
                              perpendicular bisector), else both shift by one common Gaussian
                              offset of the move's scales.  0 (the default) turns it off;
                              p_birth + p_death + p_pair <= 1.  In CMH_F32 it needs the
                              variance reading without staging (likelihood 0, stage_samples
                              0; else CMH_ERR_ARG), and a batch refuses it */
    /* Latent arrival times (§Generative Model, Event Detections: the
     * arrival is Gaussian around t + d/v).  sig_a > 0 gives every (event, station it
     * reaches) a latent offset delta ~ N(0, sig_a^2), the arrival being t + d/v +
     * delta; births draw the offsets from that prior, a moved event keeps the offsets
     * of the stations it still reaches and draws those of newly reached ones.  p_arr
     * is the share of the arrival-time move (§MH moves: one offset of one event moved
     * by a Gaussian of scale sig_da); it follows p_pair in the mix
     * (p_birth + p_death + p_pair + p_arr <= 1).  sig_a = 0 (the default): arrivals
     * are deterministic and p_arr must be 0.  Offsets start at 0 unless set by
     * cmh_set_arrival_offsets.  The offsets are float64 in both precisions; in
     * CMH_F32 they enter a window's float32 start as delta f samples (the
     * exact float64 start decides within the margin) and need the variance
     * reading without staging (likelihood 0, stage_samples 0; else
     * CMH_ERR_ARG), and a batch refuses them. */
    double sig_a, p_arr, sig_da;
} cmh_params;

/* region grid: squares of side L anchored at the origin, shifted by (sx, sy) */
typedef struct { double L; } cmh_grid;

typedef struct {
    uint64_t proposed[3];   /* by move type: 0 birth, 1 death, 2 move */
    uint64_t evaluated[3];  /* proposals that were priced (not rejected outright) */
    uint64_t accepted[3];
    int64_t sweeps;         /* sweeps run so far */
    int64_t n_events;
    double phase_ms;        /* summed device time of the colour-phase kernels while timing
                               is enabled (cmh_set_timing), CUDA events on the model stream */
    int64_t phase_launches; /* colour-phase kernels counted in phase_ms */
    int64_t kernel_launches;/* all kernels this model launched */
    uint64_t priced_samples;    /* station samples priced over all evaluated proposals */
    uint64_t rewritten_samples; /* station samples whose variance was re-synthesised */
    int64_t spill_bytes;    /* float32 regions too large for shared memory: bytes of the global
                               slot per CTA holding their arrival caches and lists (0: none) */
    uint64_t pair[3];       /* joint moves of a pair (p_pair): proposed, evaluated, accepted */
    uint64_t arrival[3];    /* arrival-time moves (p_arr): proposed, evaluated, accepted */
    uint64_t unique_samples;/* float32 form, counted only while timing is enabled
                               (cmh_set_timing): per region and colour phase, the samples of
                               the union of the windows its evaluated proposals priced at each
                               station, summed over regions (the samples a phase first touches) */
} cmh_stats;

/* one record per MH step (optional, cmh_set_trace) */
typedef struct {
    int32_t sweep, cell, step, type;   /* type: 0 birth, 1 death, 2 move, 3 joint move of a pair,
                                          4 arrival-time move */
    int32_t evaluated, accepted, n_before, written;
    double dll;        /* log-likelihood change of the proposal (0 if not evaluated) */
    double log_alpha;  /* log acceptance ratio (-inf if not evaluated) */
} cmh_trace;

/*
 * Build a model from an initial event hypothesis (the paper starts from the
 * empty set: n_events = 0 is valid), the stations and their signals.
 *   init_events  [n_events] host array (may be NULL when n_events == 0)
 *   stations     [n_stations] host array, n_stations >= 0
 *   signals      row-major [n_stations][row_pitch] samples of type sig_dtype;
 *                host memory, or device memory when signals_on_device != 0
 *                (then ordered after work already on cuda_stream)
 *   n_samples    samples per station (>= 1), row_pitch >= n_samples (elements)
 *   p            model parameters (copied)
 *   cuda_stream  cudaStream_t all device work of the model is ordered on;
 *                NULL: the model creates and owns a non-blocking stream
 * The library copies every input (FP64 signals are rounded to FP32 when
 * p->dtype == CMH_F32) and synthesises the predicted-variance buffer.
 * Errors: CMH_ERR_ARG, CMH_ERR_NONFINITE (signals or events), CMH_ERR_OOM,
 * CMH_ERR_CUDA.  *out is NULL on error.
 */
int cmh_create_model(const cmh_event* init_events, int64_t n_events,
                     const cmh_station* stations, int32_t n_stations,
                     const void* signals, int64_t n_samples, int64_t row_pitch,
                     cmh_dtype sig_dtype, int32_t signals_on_device,
                     const cmh_params* p, void* cuda_stream, cmh_model** out);

/*
 * Partition the event space into squares of side grid->L and colour them
 * (§Partitioning the World): cells whose indices differ by the period
 * P = ceil(2 R_max / L) + 1 share a colour (P^2 colours, 4 when
 * R_max <= L/2), so same-colour regions have disjoint Markov blankets.
 *   shift_mode 0: boundaries fixed at offset (sx, sy), 0 <= sx, sy < L
 *                 (Algorithm "Chromatic MH with Static Coloring")
 *   shift_mode 1: a fresh uniform offset in [0, L)^2 before every sweep, drawn
 *                 from Philox (§Chromatic MH with Dynamic Coloring); sx, sy ignored
 * Bins the current events into the cells.  May be called again (new grid).
 * *n_colors_out (may be NULL) receives P^2.
 * Errors: CMH_ERR_ARG, CMH_ERR_GEOMETRY (P^2 > 16), CMH_ERR_OOM, CMH_ERR_CAPACITY.
 */
int cmh_partition_and_color(cmh_model* m, const cmh_grid* grid, int32_t shift_mode,
                            double sx, double sy, int32_t* n_colors_out);

/*
 * Enqueue n >= 0 sweeps on the model's stream and return (asynchronous).
 * A sweep: (re)bin events into the shifted cells, then for each colour in
 * order one launch in which every region of that colour runs k_per_phase MH
 * steps (birth / death / move) on its own events with all others fixed.
 * Errors: CMH_ERR_STATE (no partition yet, or an error is latched), CMH_ERR_CUDA.
 */
int cmh_run_sweeps(cmh_model* m, int64_t n);

/*
 * Synchronise and copy the current events out.
 *   out [cap] host array (may be NULL when cap == 0); ids_out [cap] or NULL
 *   *n_out receives the number of events (even when it exceeds cap)
 *   *log_density_out (may be NULL): running log-density (prior + likelihood)
 *   *stats_out (may be NULL)
 * Events are ordered by region, then by id.  Returns a latched device error.
 */
int cmh_read_state(cmh_model* m, cmh_event* out, uint64_t* ids_out, int64_t cap,
                   int64_t* n_out, double* log_density_out, cmh_stats* stats_out);

/*
 * Latent arrival offsets (sig_a > 0; §Generative Model, Event Detections).
 * cmh_set_arrival_offsets: before the first cmh_partition_and_color, set the
 *   offsets of the initial events: off [n_events][n_stations] host array,
 *   row i for the i-th event given to cmh_create_model, column j for station
 *   j; entries of stations an event does not reach (distance >= R_max) are
 *   ignored and read back as 0.  The predicted variance and the running
 *   log-density (whose prior then includes log N(delta; 0, sig_a^2) per
 *   offset) are recomputed.
 * cmh_read_arrival_offsets: synchronise and copy the current events' offsets
 *   out, rows in cmh_read_state's order: out [cap][n_stations] (may be NULL
 *   when cap == 0); *n_out receives the number of events.
 * Errors: CMH_ERR_ARG (null pointers, sizes that do not match the model,
 * non-finite offsets, or a model without latent arrivals), CMH_ERR_STATE
 * (set after partitioning, or an error is latched), CMH_ERR_CUDA.
 */
int cmh_set_arrival_offsets(cmh_model* m, const double* off, int64_t n_events, int32_t n_stations);
int cmh_read_arrival_offsets(cmh_model* m, double* out, int64_t cap, int64_t* n_out);

/*
 * Asynchronous state reads (two slots), so that a caller can read every
 * sweep's state while the next sweep runs.
 * cmh_read_state_async: enqueues on the model's stream, after the sweeps
 *   enqueued so far, the copy of the events, running log-density, statistics
 *   and device status into slot 0 or 1 (model-owned pinned host memory the
 *   flattening kernel writes directly); returns without waiting.  A slot
 *   with an unfetched request is waited for first.  Needs a partition
 *   (CMH_ERR_STATE).
 * cmh_read_state_fetch: waits for the slot's request only, then fills the
 *   outputs as cmh_read_state would for the state at the request.  With
 *   out == ids_out == log_density_out == stats_out == NULL and cap == 0 it
 *   only reports *n_out and leaves the request to be fetched.  CMH_ERR_STATE
 *   if the slot holds no request; a device error latched by the sweeps
 *   before the request is returned.
 */
int cmh_read_state_async(cmh_model* m, int32_t slot);
int cmh_read_state_fetch(cmh_model* m, int32_t slot, cmh_event* out, uint64_t* ids_out, int64_t cap,
                         int64_t* n_out, double* log_density_out, cmh_stats* stats_out);

/* Wait for the model's stream; return a latched device error if any. */
int cmh_sync(cmh_model* m);

/*
 * Recompute the log-density from scratch on the device: the variance buffer
 * is re-synthesised from the events, then prior + Gaussian log-likelihood are
 * summed in float64.  Also resets the running log-density to that value.
 */
int cmh_log_density(cmh_model* m, double* out);

/*
 * Keep one cmh_trace record per MH step of the next sweeps, up to `capacity`
 * records (0 disables).  Records are indexed by (sweep, cell, step).
 */
int cmh_set_trace(cmh_model* m, int64_t capacity);
/* Copy the written trace records (ordered by sweep, cell, step). */
int cmh_read_trace(cmh_model* m, cmh_trace* out, int64_t cap, int64_t* n_out);

/* 1: launch sweeps without a CUDA graph and time every colour-phase kernel
 * with CUDA events on the model stream (summed into cmh_stats.phase_ms). */
int cmh_set_timing(cmh_model* m, int32_t enable);

/* Current shift (sx, sy) of the partition. */
int cmh_read_shift(cmh_model* m, double* sx, double* sy);

/*
 * Serialise the sampler state (parameters, grid, sweep counter, events with
 * ids, running log-density) into buf.  With buf == NULL only *len is set.
 * Errors: CMH_ERR_ARG (buffer too small: *len holds the size needed).
 */
int cmh_checkpoint(cmh_model* m, void* buf, size_t* len);
/* Restore a checkpoint into a model built over the same stations and
 * signals; re-synthesises the variance buffer.  Errors: CMH_ERR_ARG (corrupt
 * or mismatched checkpoint). */
int cmh_restore(cmh_model* m, const void* buf, size_t len);

void cmh_destroy(cmh_model* m);
const char* cmh_strerror(int code);

/* ---- batches of independent models (same library, float32 form) -----------
 * A batch sweeps many independent models together: one sweep of every model
 * per step, the re-binning of all models in three launches, and every
 * region of every model in persistent launches fed by device work queues
 * (colour order across models; a region waits only for its own model's
 * neighbouring regions of lower colours), captured in one CUDA graph.
 * Models are grouped by how many of their region CTAs fit on an SM (3, 2 or
 * 1, from the shared memory a region needs); each group has its own queue
 * and launch, and the groups run concurrently.  The chains are the ones
 * cmh_run_sweeps gives each model alone.
 *
 * cmh_batch_create: models[0..n_models) must be distinct, partitioned, of
 *   dtype CMH_F32 and one likelihood reading, without staging (stage_samples
 *   0), joint moves (p_pair 0) or latent arrival offsets (sig_a 0), and with
 *   ev_capacity <= 512 (CMH_ERR_ARG otherwise; CMH_ERR_STATE for an unpartitioned or
 *   failed model).  The batch refers to the models (it does not own them)
 *   and to their current partitions; cuda_stream may be NULL (the batch
 *   creates its own).  Destroy the batch before its models.
 * cmh_batch_run_sweeps: enqueues n sweeps of every model on the batch's
 *   stream and returns; later calls on a model's own stream wait for them.
 *   CMH_ERR_STATE if a model failed, was re-partitioned or had its birth
 *   table set or removed since the batch was made.  Each model's state, statistics and sweep count advance as if
 *   cmh_run_sweeps(model, n) had run.
 * cmh_batch_sync: waits for the batch's sweeps; a device-side error of a
 *   model is latched in that model and the first one is returned.
 * cmh_batch_groups: the number of groups and, for the first `cap`, their
 *   models and persistent-launch CTAs.
 */
/* ---- learned birth proposal --------------------------------------------------
 * cmh_set_birth_table makes the birth proposal a mixture (float32 form): with
 * probability mix (0 < mix < 1) a birth comes from the table, otherwise it is
 * uniform in the region as before.  tab[(iy * nx + ix) * nt + b] >= 0 (host
 * memory, copied) weights pixel (ix, iy) of side (W/nx, W/ny) and time bin b
 * of length T/nt.  A table birth in a region picks a pixel by its share of
 * the region's table mass (pixel mass times the fraction of the pixel inside
 * the region), a position uniform in pixel and region, a time bin by the
 * pixel's weights and a time uniform in the bin; the magnitude is drawn as
 * for uniform births.  The birth and death Hastings terms carry the mixture
 * density, so the chain still targets the posterior (the prior, without
 * stations).  The sampling runs in explicitly rounded float64; the density
 * term of log alpha uses the table's float weight and a float32 logarithm
 * (about 1e-7 absolute), like the other float32 terms of the sweep.  A region's pixel range may span at most 256 pixels
 * ((L nx / W + 4)(L ny / W + 4) <= 256).  nx == 0 removes the table.
 * Errors: CMH_ERR_ARG (float64 model, bad sizes or mix), CMH_ERR_NONFINITE
 * (a negative or non-finite weight), CMH_ERR_OOM. */
int cmh_set_birth_table(cmh_model* m, const float* tab, int32_t nx, int32_t ny, int32_t nt, double mix);

/* cmh_set_birth_magnitude: learned magnitudes for the table births.
 * centre[(iy * nx + ix) * nt + b] (host, copied, finite; the shape of the
 * table set last) is the centre of entry (ix, iy, b); a table birth at that
 * entry draws m uniform on [lo, lo + 2 h), lo = max(2, centre - h), h =
 * half_width > 0, from word 3 of the step's third Philox block (float64,
 * explicitly rounded).  The mixture density in log alpha becomes
 * (1 - mix) q_unif p(m) + mix q_net q_win(m), p the magnitude prior.
 * centre == NULL returns to magnitudes from the prior; a new table drops
 * them.  Errors: CMH_ERR_STATE (no table), CMH_ERR_ARG (half_width),
 * CMH_ERR_NONFINITE, CMH_ERR_OOM. */
int cmh_set_birth_magnitude(cmh_model* m, const float* centre, double half_width);

/* ---- the network behind the learned birth proposal ----------------------------
 * A 1-D convolutional network maps a tile of 8 x 8 stations (100 km apart,
 * 800 km) x 256 samples (features log1p(s^2), layout [window][sample][station])
 * to 4101 outputs: 4096 logits over the tile's 64 x 64 pixels (12.5 km,
 * row-major from the tile origin), one "no event" logit, the mean and log sd
 * of the event's origin time relative to the window start (s) and of its
 * magnitude.  Products on the tensor cores in BF16 with FP32 accumulation;
 * FP32 parameters (cmh_net_param_count floats) with BF16 copies.
 *
 * cmh_net_create: max_batch windows per call (1..4096); seeded initialisation.
 * cmh_net_get_params / set_params: the FP32 parameters (host arrays).
 * cmh_net_forward: outputs [batch][4101] for host features [batch][256][64].
 * cmh_net_gradients: the gradient of the mean loss (cross-entropy over the
 *   4097 classes, Gaussian negative log-likelihood of time and magnitude for
 *   labels < 4096) with respect to every parameter, and the loss.
 * cmh_net_train: `steps` AdamW steps on batches simulated on the GPU from the
 *   generative model of `geometry` (its noise, attenuation, envelope, speed):
 *   stations jittered by 25 km around an 8 x 8 grid, half the windows with one
 *   event (origin time in [-15 s, window end)); *loss_out = the last batch's.
 * cmh_net_birth_table: slides the network over a float32 model's signals:
 *   n_tiles tiles (tiles[t*64 + s] = the model's station index of tile
 *   station s, row-major from the tile origin tile_origin[2t], [2t+1] in km),
 *   windows every hop_s seconds; each window adds its pixel probabilities
 *   times its time Gaussian's mass per bin to table[(iy*nx + ix)*nt + b]
 *   (pixels of side W/nx, W/ny, nt bins over [0,T)), for cmh_set_birth_table;
 *   magnitude (may be NULL) receives the same weights' mean predicted
 *   magnitude per entry (3 where no weight was added), for
 *   cmh_set_birth_magnitude.
 */
typedef struct cmh_net cmh_net;
int64_t cmh_net_param_count(void);
int cmh_net_create(int32_t max_batch, uint64_t seed, void* cuda_stream, cmh_net** out);
void cmh_net_destroy(cmh_net* n);
int cmh_net_get_params(cmh_net* n, float* out);
int cmh_net_set_params(cmh_net* n, const float* in);
int cmh_net_forward(cmh_net* n, const float* features, int32_t batch, float* out);
int cmh_net_gradients(cmh_net* n, const float* features, const int32_t* label, const float* t_label,
                      const float* m_label, int32_t batch, float* grads, double* loss);
int cmh_net_train(cmh_net* n, const cmh_model* geometry, int32_t steps, int32_t batch, double lr, double* loss_out);
int cmh_net_birth_table(cmh_net* n, cmh_model* m, const int32_t* tiles, const double* tile_origin, int32_t n_tiles,
                        int32_t nx, int32_t ny, int32_t nt, double hop_s, float* table, float* magnitude);

/* ---- autotuning ------------------------------------------------------------
 * cmh_autotune times, from a checkpoint of the model, trial_sweeps sweeps of
 * each launch configuration the float32 form offers (colour by colour or
 * persistent; staging off or automatic; 1-3 CTAs per SM for the persistent
 * launch), keeps the fastest in the model's parameters and restores the
 * checkpoint, so the chain continues as if no trial had run.  Needs a
 * partitioned CMH_F32 model (CMH_ERR_ARG / CMH_ERR_STATE otherwise). */
typedef struct {
    int32_t schedule, stage_samples, ctas_per_sm;   /* the choice */
    double ms_per_sweep;                            /* its trial time */
    int32_t n_tried;
    int32_t tried_schedule[16], tried_stage[16], tried_ctas[16];
    double tried_ms[16];                            /* -1: the configuration does not fit */
} cmh_tuning;
int cmh_autotune(cmh_model* m, int32_t trial_sweeps, cmh_tuning* out);

typedef struct cmh_batch cmh_batch;
int cmh_batch_create(cmh_model* const* models, int32_t n_models, void* cuda_stream, cmh_batch** out);
int cmh_batch_run_sweeps(cmh_batch* b, int64_t n);
int cmh_batch_sync(cmh_batch* b);
int cmh_batch_groups(const cmh_batch* b, int32_t* n_groups, int32_t* models_per_group, int32_t* grid_per_group,
                     int32_t cap);
void cmh_batch_destroy(cmh_batch* b);

/*
 * Sum over rows r < n_rows and samples k < n_samples of the Gaussian
 * log-density log N(signals[r][k]; 0, variance[r][k]), for callers that cannot
 * allocate device memory: applications whose memory manager owns the whole
 * GPU, hooks that must not trigger the device synchronisation an allocation
 * may cause, plugins in processes that forbid allocations outside their
 * framework.  The paper has no counterpart; it is the likelihood reduction of
 * cmh_log_density applied to caller-owned buffers.
 *   signals, variance  device pointers, row-major [n_rows][row_pitch] of dtype
 *                      (caller-owned, read only)
 *   out                host pointer; receives the sum (float64 accumulation)
 *   cuda_stream        stream the two kernels and the 8-byte read-back are
 *                      ordered on (NULL: legacy default stream); the call
 *                      synchronises it before returning
 * Allocates nothing: the partial sums live in a fixed 64 KB device array
 * that every GPU loading the library keeps until exit.  The first call on a
 * device looks that array's address up (cudaGetSymbolAddress) and keeps it;
 * make that first call before any stream capture begins.  The address
 * belongs to the device's context: after cudaDeviceReset the next call sees
 * the new context and looks it up again.  Every call reuses the same array
 * and leaves its sums there: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Errors: CMH_ERR_ARG (null pointer, n_samples < 1, row_pitch < n_samples,
 * unknown dtype), CMH_ERR_CAPACITY (n_rows > 8191, the array's limit),
 * CMH_ERR_CUDA.
 */
int cmh_gaussian_loglik_noalloc(const void* signals, const void* variance, int32_t n_rows,
                                int64_t n_samples, int64_t row_pitch, cmh_dtype dtype, double* out,
                                void* cuda_stream);

/*
 * Test hook for the bounded waits of the persistent float32 sweep (schedule 0):
 * from the next cmh_run_sweeps on, the region of cell `cell` runs its colour
 * phase but never announces that it has finished, so every higher-colour
 * neighbour waiting for it gives up after `wait_limit` polls (0: the default,
 * about half a second) and the sweep latches CMH_ERR_TIMEOUT, which the next
 * synchronising call returns; the model then refuses further work
 * (CMH_ERR_STATE) and must be destroyed.  No kernel is left waiting: every
 * wait is bounded and the others end as soon as the error is latched.
 * cell = -1 turns the hook off.  The paper has no counterpart.
 * Errors: CMH_ERR_ARG (null model, cell outside -1..n_cells-1),
 * CMH_ERR_STATE (not partitioned, float64 form, or colour-by-colour schedule).
 */
int cmh_test_hold_region(cmh_model* m, int32_t cell, uint32_t wait_limit);

/*
 * Measured throughput of the current device's special-function unit (ex2,
 * lg2, rcp: the per-sample exponential, logarithm and reciprocal of the
 * float32 pricing) and of its float32 FMA pipe, the denominators of the
 * roofline's arithmetic terms beside the HBM bandwidth.  The paper has no
 * counterpart: it is a measurement, not part of the method.
 *   mufu_ops_per_s   host pointer; receives MUFU operations per second
 *   fma_flops_per_s  host pointer; receives float32 flops per second (2 per FMA)
 *   cuda_stream      stream the timed kernels run on (NULL: legacy default)
 * Best of three timed launches each, after a warm-up, with CUDA events;
 * synchronises the stream.  Allocates nothing.
 * Errors: CMH_ERR_ARG (null pointer), CMH_ERR_CUDA.
 */
int cmh_measure_alu_peaks(double* mufu_ops_per_s, double* fma_flops_per_s, void* cuda_stream);

/*
 * Test hook: n Philox4x64-10 blocks computed by a device kernel.
 * ctr [n][4], key [2], out [n][4] host arrays.
 */
int cmh_philox4x64(const uint64_t* ctr, const uint64_t* key, uint64_t* out, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* CHROMH_H */
