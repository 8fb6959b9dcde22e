/*
 * gaps.h - C interface of the GB300 (sm_103a) parton-shower library.
 *
 * The library generates hard events, showers them with the dipole-shower
 * max-veto algorithm (Seymour & Sule, arXiv:2511.19633, Section 2 and Fig. 1)
 * with initial- and final-state dipoles (Appendix B), the PDF-ratio veto for
 * backward initial-state evolution (Appendix A), Catani-Seymour recoil
 * kinematics (Appendix B.2-B.5) and the MC@NLO-like matching for on-shell Z
 * production (Appendix C), and computes per-event observables and weighted
 * histograms (Section 4.1). One event per CUDA thread.
 *
 * Conventions shared by every entry point:
 *   - Four-vectors are (E, px, py, pz) in GeV, metric (+,-,-,-).
 *   - Incoming partons carry their physical momenta and crossed colour tags
 *     (an incoming quark holds an anticolour tag), so that partons i and k
 *     form a dipole when col[i] == acol[k] or acol[i] == col[k].
 *   - pp events: slot 0 = parton from beam 1 (+z), slot 1 = beam 2 (-z),
 *     slot 2 = the Z boson (flavour 23), then final-state partons.
 *     e+e- events: slot 0 = quark, slot 1 = antiquark, then emissions.
 *   - Flavours: 21 gluon, 1..5 d u s c b, negative = antiquark, 23 = Z.
 *   - Random numbers: Philox-4x32-10 (Salmon et al., SC'11) with key =
 *     (seed_lo, seed_hi) and counter = (event_lo, event_hi, draw_lo, draw_hi);
 *     event k of a seed is identical whatever the chunking or launch shape.
 *   - Every call is asynchronous on the given stream (a cudaStream_t passed
 *     as void*, NULL = legacy default stream). Return values report argument
 *     and launch errors; errors found on the device (capacity, iteration cap,
 *     non-finite values) are stored per event in `status` and counted by
 *     gaps_get_stats, which synchronises the stream.
 *   - Device buffers are owned by the caller; the library owns its copy of
 *     the PDF grid, its bound tables, its counters and, for GAPS_MIXED, a
 *     working set of nmax partons per resident thread (allocated by the
 *     first mixed gaps_shower call; about 132 B x nmax x resident threads),
 *     or with GAPS_SCHED_WAVE one per event of ev->capacity (about
 *     132 B x nmax + 160 B per event).
 */
#ifndef GAPS_H
#define GAPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes (0 or negative) */
#define GAPS_OK                0
#define GAPS_ERR_INVALID_ARG  -1
#define GAPS_ERR_CAPACITY     -2   /* an event reached nmax partons */
#define GAPS_ERR_ITER_CAP     -3   /* an event exceeded the step cap */
#define GAPS_ERR_NUMERIC      -4   /* a non-finite scale or weight */
#define GAPS_ERR_CUDA         -5   /* a CUDA runtime call failed */
#define GAPS_ERR_NO_DEVICE    -6

/* processes (Section 4.1; e+e- as in GAPS 1) */
#define GAPS_EE_QQ       0   /* e+e- -> Z/gamma* -> q qbar, final-state shower */
#define GAPS_PP_Z_LO     1   /* pp -> Z at LO, initial- and final-state shower */
#define GAPS_PP_Z_NLO    2   /* pp -> Z, S and H events of Appendix C.4 */
#define GAPS_PP_LL       3   /* pp -> Z/gamma* -> e- e+ at LO with the Z/gamma
                                interference (the process GAPS 2 provides besides
                                on-shell Z production, Sec. 4.1): dilepton mass in
                                [mll_lo, mll_hi] by a Breit-Wigner map; records hold
                                the beams in slots 0, 1 and e-, e+ in slots 2, 3 */

/* arithmetic of the shower */
#define GAPS_FP64        0   /* all FP64; matches the reference per event */
#define GAPS_MIXED       1   /* FP32 trials, PDF and bounds; FP64 kinematics */

/* launch schedules of the shower */
#define GAPS_SCHED_PER_EVENT  0   /* one thread per event, run to completion */
#define GAPS_SCHED_PERSISTENT 1   /* persistent grid, finished lanes take the next event */
#define GAPS_SCHED_WARP       2   /* GAPS_MIXED only: persistent grid, one event per warp
                                     in shared memory, the lanes share its trials */
#define GAPS_SCHED_WAVE       3   /* GAPS_MIXED only: wavefront passes, one kernel per phase
                                     (end tables, veto cycles, emissions) over lists of
                                     live events, then the persistent grid for the events
                                     still live; identical events to GAPS_SCHED_PERSISTENT */

/* per-event status values; negative values are the error codes above */
#define GAPS_STATUS_ACTIVE 0
#define GAPS_STATUS_DONE   1

/* PDF grid geometry: value = x f(x, Q^2), layout [GAPS_PDF_NFL][NX][NQ],
 * flavour order g d u s c b dbar ubar sbar cbar bbar; nodes uniform in ln x
 * over [GAPS_PDF_XMIN, GAPS_PDF_XMAX] and in ln Q^2 over [Q2MIN, Q2MAX].
 * Bilinear interpolation in (ln x, ln Q^2); zero outside (Appendix B.6). */
#define GAPS_PDF_NFL   11
#define GAPS_PDF_NX    100
#define GAPS_PDF_NQ    50
#define GAPS_PDF_XMIN  1e-6
#define GAPS_PDF_XMAX  (1.0 - 1e-6)
#define GAPS_PDF_Q2MIN 0.5
#define GAPS_PDF_Q2MAX (13600.0 * 13600.0)

#define GAPS_NOBS      8     /* per-event observables, see gaps_observables */
#define GAPS_NHIST     6     /* histograms per process family */
#define GAPS_HIST_BINS 66    /* per histogram: underflow, 64 bins, overflow */

typedef struct gaps_ctx gaps_ctx;  /* opaque, owned by the library */

/* Mixed batch (config field n_mix > 0): the batch holds several processes
 * and one launch showers them all (Section 3 on heterogeneous batches). The
 * paper does not say how events are assigned; here event `id` belongs to the
 * first row whose cumulative fraction exceeds the uniform of Philox block
 * (seed, id, draw 2^62), words 0 and 1 (the last row takes the remainder),
 * and is then exactly event `id` of a one-process context with that row's
 * process, sqrt_s and t_cut and the same other settings. */
#define GAPS_MAX_MIX 4
typedef struct {
    int process;          /* GAPS_EE_QQ, GAPS_PP_Z_LO, GAPS_PP_Z_NLO or GAPS_PP_LL */
    double sqrt_s;        /* GeV */
    double t_cut;         /* GeV^2 */
    double fraction;      /* share of the events, > 0; the shares sum to 1 */
} gaps_mix_row;

/* Configuration, copied by gaps_init. */
typedef struct {
    int process;          /* GAPS_EE_QQ, GAPS_PP_Z_LO, GAPS_PP_Z_NLO or GAPS_PP_LL */
    int precision;        /* GAPS_FP64 or GAPS_MIXED */
    int nf;               /* active flavours for g -> q qbar (5) */
    int nmax_partons;     /* capacity per event, 4..128 */
    double sqrt_s;        /* collider energy, GeV */
    double alpha_s_mz;    /* alpha_s(m_Z^2); one-loop running with 5 flavours */
    double t_cut;         /* shower cutoff on t = pT^2, GeV^2, >= GAPS_PDF_Q2MIN */
    double p_s;           /* probability of an S event in GAPS_PP_Z_NLO, in (0,1) */
    uint64_t seed;        /* Philox key */
    const float* pdf_grid;/* host pointer to the PDF grid (pp processes), copied */
    int block_size;       /* threads per block for the shower, 0 = library default */
    int schedule;         /* GAPS_SCHED_PER_EVENT, GAPS_SCHED_PERSISTENT or GAPS_SCHED_WARP */
    int blocks_per_sm;    /* persistent schedule: resident blocks per SM, 0 = default */
    int refill_period;    /* GAPS_MIXED: idle lanes take new events at most every
                             this many cycles (compaction period), 0 = 1 */
    int emit_batch;       /* GAPS_MIXED: accepted emissions of a warp are built
                             together once this many lanes wait (or after 4x
                             this many cycles), 1..32, 0 = 1 */
    int n_mix;            /* 0: one process (the fields above); 1..GAPS_MAX_MIX:
                             mixed batch of these rows, which replace process,
                             sqrt_s and t_cut above */
    gaps_mix_row mix[GAPS_MAX_MIX];
    int trial_mode;       /* GAPS_TRIALS_*: how the overestimate trials of a cycle are
                             drawn; KEEP and SELECT only with GAPS_MIXED and
                             GAPS_SCHED_PERSISTENT or GAPS_SCHED_WAVE, VETOMAX only
                             with GAPS_MIXED and GAPS_SCHED_PERSISTENT; any other
                             combination or value is GAPS_ERR_INVALID_ARG */
    double mll_lo, mll_hi;  /* GAPS_PP_LL (also as a row of a mixed batch): dilepton
                             mass window in GeV, 0 < mll_lo < mll_hi <= sqrt_s */
    int max_cycles;       /* veto cycles an event may take before it ends with
                             GAPS_ERR_ITER_CAP, 0 = 200000, at most 1e9 */
    int wave_passes;      /* GAPS_SCHED_WAVE: passes before the persistent grid takes
                             the remaining live events, 0 = 24, at most 4096 */
    int wave_cycles;      /* GAPS_SCHED_WAVE: veto cycles of one event in one pass
                             before it waits for the next pass, 0 = 64, 1..1e6 */
    int wave_veto_blocks_per_sm; /* GAPS_SCHED_WAVE: resident blocks of block_size
                             threads per SM of the veto kernel, which sets its
                             register budget (2: 128, 3: 80, 4: 64 registers a
                             thread); 0 = 2, else 2..4 */
} gaps_config;

/* Trial schemes (gaps_config.trial_mode). All three give the same
 * distributions (Sec. 2): every channel's overestimate is a Poisson process
 * in ln t with a constant rate while its dipole end's record is unchanged.
 *   REDRAW  every channel of every end draws a trial each cycle and the
 *           largest wins (max-veto, Fig. 1 as printed; the FP64 path's order)
 *   KEEP    max-veto keeping the losing trials: after a veto only the
 *           winner's channel draws again, after an emission only the ends
 *           whose record changed (the kept trial is the channel's first point
 *           below the scale the event continues from)
 *   SELECT  generate-select (the alternative named in Sec. 2's footnote):
 *           one trial from the summed rate of the channels active at the
 *           current scale, restarted at each channel's maximum scale as it
 *           is passed, and the channel chosen with probability rate / sum
 *   VETOMAX veto-max (Sec. 2): every channel runs its own veto algorithm to
 *           its first accepted point, the largest wins; the accepted points
 *           are kept while their end's record is unchanged. Persistent
 *           schedule only; the plain bounds (a learned proposal is not used) */
#define GAPS_TRIALS_REDRAW 0
#define GAPS_TRIALS_KEEP 1
#define GAPS_TRIALS_SELECT 2
#define GAPS_TRIALS_VETOMAX 3

/* Event records: structure of arrays in device memory, caller-owned, event
 * index fastest so that a warp's loads are coalesced. `capacity` is the
 * allocated number of events (row stride) and `nmax` the slots per event. */
typedef struct {
    uint64_t capacity;
    int nmax;
    double* p;        /* [4][nmax][capacity] momenta */
    int32_t* flav;    /* [nmax][capacity] */
    int32_t* col;     /* [nmax][capacity] colour tag (crossed for incoming) */
    int32_t* acol;    /* [nmax][capacity] anticolour tag */
    int32_t* npart;   /* [capacity] partons in the record */
    int32_t* status;  /* [capacity] GAPS_STATUS_* or a negative error code */
    int32_t* n_emit;  /* [capacity] accepted emissions */
    double* weight;   /* [capacity] event weight, pb (may be negative for H) */
    double* t;        /* [capacity] current evolution scale */
    double* eta;      /* [2][capacity] momentum fractions of slots 0 and 1 */
    uint64_t* draw;   /* [capacity] next Philox block of the event's stream */
} gaps_events;

/* Weighted histograms in device memory, caller-owned and zeroed by the
 * caller: sumw and sumw2 are [GAPS_NHIST][GAPS_HIST_BINS] doubles, or
 * [n_mix][GAPS_NHIST][GAPS_HIST_BINS] for a mixed batch (one set per row);
 * the binning of each histogram is returned by gaps_hist_binning. */
typedef struct {
    double* sumw;
    double* sumw2;
} gaps_hists;

/* Counters accumulated over all gaps_shower calls of a context. */
typedef struct {
    uint64_t events;      /* events finished */
    uint64_t steps;       /* max-veto cycles (Fig. 1) */
    uint64_t trials;      /* dipole-channel trials with a non-zero overestimate */
    uint64_t isr_trials;  /* of which with an initial-state emitter */
    uint64_t vetoes;      /* rejected winners */
    uint64_t accepts;     /* accepted emissions */
    uint64_t violations;  /* acceptance weights above one (overestimate failures) */
    uint64_t err_capacity, err_iter_cap, err_numeric;
    uint64_t lane_steps;  /* active lanes summed over warp steps (divergence) */
    uint64_t warp_steps;  /* warp steps x 32 */
    uint64_t rebuilds;    /* GAPS_MIXED: warp-cooperative colour-end table rebuilds */
    uint64_t mlp_tiles;   /* GAPS_MIXED: 16-row network evaluations of the learned proposal */
} gaps_stats;

/* Creates a context on the current CUDA device: validates `cfg`, copies the
 * PDF grid and builds the certified PDF-ratio bound tables of Appendix A.2
 * (reading: a strict bound replaces the paper's percentile fit).
 * Returns GAPS_ERR_INVALID_ARG for a bad configuration (process, sqrt_s,
 * t_cut below the grid, nmax out of range, missing grid for pp), and
 * GAPS_ERR_NO_DEVICE / GAPS_ERR_CUDA on device errors; *out is set only on
 * success. */
int gaps_init(gaps_ctx** out, const gaps_config* cfg);

/* Hard events (Appendix C.1-C.4; e+e- from the textbook LO formula):
 * fills records first_event .. first_event + n - 1 into slots 0 .. n-1 of
 * `ev` (n <= ev->capacity), sets status ACTIVE, draw = 0 and the starting
 * scale t = s (power shower, Appendix C.4). */
int gaps_generate_hard(gaps_ctx* ctx, uint64_t first_event, uint64_t n,
                       const gaps_events* ev, void* stream);

/* Shower (Section 2, Fig. 1; Appendices A-B): evolves every ACTIVE record
 * among the first n until its winner scale falls below t_cut. Records are
 * read and written in place; first_event must be the value given to
 * gaps_generate_hard (it keys the random streams). GAPS_FP64 reproduces the
 * FP64 reference evaluation bit for bit; GAPS_MIXED runs the trials, PDF and
 * acceptance in FP32 with FP64 kinematics on a persistent grid with live-event
 * refill, and agrees with it in distribution. Returns GAPS_ERR_CUDA if the
 * working set cannot be allocated. */
int gaps_shower(gaps_ctx* ctx, uint64_t first_event, uint64_t n,
                const gaps_events* ev, void* stream);

/* Shower without any device allocation, for callers that cannot allocate
 * device memory themselves (code embedded in a host application that owns all
 * device allocations, or whose device footprint is fixed before it runs).
 * The paper has no counterpart: it is the GAPS_MIXED persistent shower of
 * gaps_shower, run with 64 blocks of 128 threads and emission batch 8, with
 * every piece of scratch memory held in device arrays of the library itself:
 * a working set for at most 32 partons per event (37.7 MB), the work counter,
 * the statistics and copies of the PDF grid and its bound tables (38.0 MB in
 * all). Every GPU that loads the library keeps these arrays until the process
 * exits. It needs no context: `cfg` is read as in gaps_init and the caller
 * still passes the event records, written by gaps_generate_hard or an
 * equivalent. cfg's precision, schedule and launch fields (block size, blocks
 * per SM, refill period, emission batch) are ignored. Results are identical to
 * gaps_shower with GAPS_MIXED and the plain bounds for the same events (a
 * learned proposal is never used here).
 *   - Rejects ev->nmax above 32 (or different from cfg->nmax_partons) and
 *     any invalid configuration with GAPS_ERR_INVALID_ARG.
 *   - The first call on a device looks up the arrays' device addresses; make
 *     that first call before any stream capture.
 *   - When cfg->pdf_grid is set (every pp process) the call rebuilds the bound
 *     tables on the host, copies them and the grid into the library's arrays
 *     and synchronises `stream` before the launch (the tables' host copy lives
 *     in the call).
 *   - When stats != NULL it synchronises `stream` after the launch and
 *     returns this call's counters.
 *   - All calls share the same arrays (the counters are cleared by each
 *     call): calls that overlap on the GPU, from any stream or thread, race. */
int gaps_shower_static(const gaps_config* cfg, uint64_t first_event, uint64_t n,
                       const gaps_events* ev, gaps_stats* stats, void* stream);

/* ---- learned initial-state proposal --------------------------------------
 * The overestimate of every initial-state channel (Appendix A.2) is made
 * piecewise constant over GAPS_ISR_BINS bins of zeta, the coordinate in which
 * z is sampled; bin heights come from a 4 -> 64 -> 64 -> 1 ReLU network with
 * inputs (ln eta, ln(s/t_c), bin centre in zeta, class of dipole type, channel
 * and flavour), evaluated with BF16 weights and FP32 accumulation. The
 * heights are calibrated on sampled states, not certified: the acceptance
 * weight of every winner (accepted or vetoed) is checked, and a weight above
 * one is counted as a violation and sends the event back to the plain
 * certified bound from the scale before that cycle. A zero violation count
 * shows that the heights held wherever a winner landed; the result is the
 * plain algorithm's only where they bound the ratio over the whole bin, which
 * the histogram tests check statistically.
 * Parameter layout (FP32): W1 [64][4], b1 [64], W2 [64][64], b2 [64], W3 [64],
 * b3. */
#define GAPS_MLP_PARAMS  4545
#define GAPS_ISR_BINS    8
/* classes of (dipole type, channel, emitter flavour): for IF (0..21) and II
 * (22..43): q <- q for the ten quark PDF indices 1..10 (d u s c b, then the
 * antiquarks), g <- q for the same ten, g <- g, q <- g */
#define GAPS_ISR_CLASSES 44
/* buckets of eta for the calibration margins: upper edges eta = 1e-5, 1e-4,
 * 1e-3, 1e-2, 0.1, 0.4, 0.7 (compared on the network input ln(eta)/7 + 1) */
#define GAPS_ISR_ETA_BINS 8

/* Runs the GAPS_MIXED shower with the plain bounds and logs the initial-state
 * colour ends met at every rebuild of an event's end table, each with
 * probability keep_fraction in (0, 1] (decided by a hash of the event id, its
 * parton count and the end, so that a bounded log samples the whole run):
 * states is a device array [capacity][4] of {eta, s, dipole type (2 IF,
 * 3 II), PDF index of the emitter}; *count (device) is incremented per
 * logged end, also past capacity. Requires one pp process and GAPS_MIXED. */
int gaps_collect_isr_states(gaps_ctx* ctx, uint64_t first_event, uint64_t n,
                            const gaps_events* ev, float keep_fraction, float* states,
                            uint64_t capacity, uint64_t* count, void* stream);

/* Training targets of the learned bound: for each logged state, channel and
 * bin (16 rows per state, row = state * 16 + channel * 8 + bin) the network
 * inputs features[row][4] and targets[row] = ln(max(r, 1e-6)), with r the
 * largest acceptance ratio over 33 zeta points of the bin (its edges included) and 64 log-spaced scales in
 * [t_c, t_kin]. Device arrays. */
int gaps_isr_targets(gaps_ctx* ctx, const float* states, uint64_t n_states,
                     float* features, float* targets, void* stream);

/* Installs a trained network (host array of GAPS_MLP_PARAMS floats, copied)
 * and the calibration margins added to its output, a host array
 * log_margins[GAPS_ISR_CLASSES][GAPS_ISR_ETA_BINS][GAPS_ISR_BINS] (copied):
 * the height of bin m of class c at eta bucket b is
 * min(1, exp(NN + log_margins[c][b][m])), rounded up to a power 2^(-k/16).
 * Later GAPS_MIXED showers of the context use them. params == NULL returns
 * to the plain bounds. Non-finite values give GAPS_ERR_INVALID_ARG. A network
 * and its margins are calibrated for the hadronic process whose states they
 * were fitted on; installed for another process, heights can fall below the
 * ratio and the shower then counts violations. */
int gaps_set_learned_proposal(gaps_ctx* ctx, const float* params, const float* log_margins);

/* The whole training pipeline of the learned proposal behind one call, on the
 * context's device and stream (the build's own addition to the method; the
 * paper's initial-state overestimate is a fitted PDF-ratio bound, App. A.2):
 *   1. collect: the plain GAPS_MIXED shower of n_events events from
 *      first_event logs initial-state colour ends (gaps_collect_isr_states),
 *      kept with a fraction set by a pilot run of 2^14 events so that about
 *      0.95 x capacity states are logged over the whole range;
 *   2. the states are sorted into a canonical order (dipole type, PDF index,
 *      eta, s), so that the network does not depend on the logging order;
 *   3. targets (gaps_isr_targets), floored at target_floor;
 *   4. training (gaps_mlp_train) from a Philox-seeded He initialisation:
 *      steps/2 Adam steps at lr, steps/4 at 0.3 lr, the rest at 0.1 lr;
 *   5. held-out states from holdout_events events at holdout_first (up to
 *      holdout_capacity), sorted and with targets the same way;
 *   6. calibration with the shower's BF16 inference numerics: per (class, eta
 *      bucket, bin) cell, margin = max(target - network) over the rows of
 *      both sets + ln(1 + slack) where the cell has min_rows rows, else 30
 *      (height 1, the plain bound);
 *   7. install (gaps_set_learned_proposal).
 * The context must hold one pp process with GAPS_MIXED. The call allocates
 * and frees its own scratch (event records for chunks of 2^19 events,
 * states, rows) and synchronises the stream. params_out
 * (GAPS_MLP_PARAMS floats) and log_margins_out (GAPS_ISR_CLASSES x
 * GAPS_ISR_ETA_BINS x GAPS_ISR_BINS floats) are host arrays that receive the
 * installed proposal when not NULL. Returns GAPS_ERR_INVALID_ARG for a bad
 * configuration, GAPS_ERR_CUDA on device errors. */
typedef struct {
    uint64_t first_event, n_events, capacity;
    uint64_t holdout_first, holdout_events, holdout_capacity;
    uint64_t steps;       /* Adam steps in all (>= 4) */
    float lr, tau;        /* learning rate; expectile of the loss, in (0, 1) */
    uint64_t seed;        /* initialisation and minibatches */
    float slack;          /* relative margin above the calibration maximum, >= 0 */
    uint32_t min_rows;    /* rows a calibration cell needs */
    float target_floor;   /* smallest target (log of the ratio) */
} gaps_learn_config;

typedef struct {
    uint64_t states, rows, holdout_states;
    float loss_first, loss_last;      /* minibatch loss of the first and last step */
    uint32_t cells_calibrated;        /* cells with a learned margin */
    float mean_bin_height;            /* mean calibrated height over the training rows */
    float fit_rmse;                   /* rms of network - target over the training rows */
} gaps_learn_report;

int gaps_train_learned_proposal(gaps_ctx* ctx, const gaps_learn_config* cfg, float* params_out,
                                float* log_margins_out, gaps_learn_report* report, void* stream);

/* The paper's fitted PDF-ratio overestimate (App. A.2) as a comparison mode
 * of the mixed-precision shower; the plain shower's bound is certified
 * instead (it bounds the ratio on the whole grid).
 * gaps_collect_pdf_ratios: runs the GAPS_MIXED shower of events first_event ..
 *   first_event + n - 1 with the certified bounds and logs the PDF ratios it
 *   evaluates for winners, x' f(x') / (eta f(eta)) of initial-state channels
 *   (times (t - m^2)/t for a heavy quark) and of final-initial spectators,
 *   each with probability keep_fraction (a hash of event and Philox counter
 *   decides): samples[capacity][4] (device) = {numerator table index,
 *   denominator table index, eta, ratio}; *count (device) counts past
 *   capacity.
 * gaps_fit_pdf_ratios: host arrays; per (numerator, denominator) transition
 *   the nearest-rank 99th and 99.99th percentiles of the sampled ratios,
 *   fit[12][12][2] (0 without samples).
 * gaps_set_pdf_ratio_fit: installs a fit (host array, copied; NULL returns to
 *   the certified bounds). Later GAPS_MIXED showers of the context use
 *   max(P99, P99.99 eta) per transition (eq. pdfmax) and P99.99 sqrt(eta) for
 *   a gluon from the summed quarks, which holds the u and d parents of eq.
 *   pdfmax_ud; transitions without samples keep the certified bound. It is not
 *   a strict bound: acceptance weights above one are counted as violations in
 *   gaps_stats (and accepted). FP64 contexts ignore it. */
int gaps_collect_pdf_ratios(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev,
                            float keep_fraction, float* samples, uint64_t capacity, uint64_t* count,
                            void* stream);
int gaps_fit_pdf_ratios(const float* samples, uint64_t n, float* fit);
int gaps_set_pdf_ratio_fit(gaps_ctx* ctx, const float* fit);

/* Violation log (device arrays, caller-owned; log == NULL switches it off):
 * every acceptance weight above one of the GAPS_MIXED shower appends 8 floats
 * to log[capacity][8] and increments *count (also past capacity): with the
 * learned bounds {eta, s, t, w, class, bin, z, zeta}; with the plain bounds
 * (the fitted PDF-ratio overestimate, or FP32 rounding at the edge of a
 * certified bound) {eta, s, t, w, -1 - (8 dipole type + channel), -1, z, 0},
 * dipole type 0 FF, 1 FI, 2 IF, 3 II and channel 0..6 as in the kernels
 * (final state: 0 q -> qg, 1 g -> gg, 2 g -> qqbar; initial state, backward:
 * 3 a quark stays a quark, 4 a quark becomes a gluon, 5 a gluon stays a
 * gluon, 6 a gluon becomes a quark). */
int gaps_set_violation_log(gaps_ctx* ctx, float* log, uint64_t capacity, uint64_t* count);

/* Network kernels (device arrays; features [n][4]):
 * gaps_mlp_loss_grad: expectile loss mean w (y - t)^2, w = tau below the
 *   target and 1 - tau above, and its gradient [GAPS_MLP_PARAMS] (FP32).
 * gaps_mlp_forward: outputs [n], FP32 (bf16 = 0) or the BF16 tensor-core
 *   numerics of the shower (bf16 = 1).
 * gaps_mlp_train: `steps` Adam steps (lr, beta 0.9/0.999) on minibatches of
 *   256 rows drawn with replacement (Philox, seed), updating params and the
 *   moment buffers m, v in place; loss_history[k] = batch loss of step
 *   k * history_every when not NULL. */
int gaps_mlp_loss_grad(const float* params, const float* features, const float* targets,
                       uint64_t n, float tau, float* grad, float* loss, void* stream);
int gaps_mlp_forward(const float* params, const float* features, uint64_t n, int bf16,
                     float* out, void* stream);
int gaps_mlp_train(float* params, float* adam_m, float* adam_v, const float* features,
                   const float* targets, uint64_t n, uint64_t steps, float lr, float tau,
                   uint64_t seed, float* loss_history, int history_every, void* stream);

/* Observables (Section 4.1) of records first_event .. first_event + n - 1
 * (the event ids pick the rows of a mixed batch): writes
 * obs[GAPS_NOBS][capacity] (device) and, when hists != NULL, adds every
 * event with status DONE to the histograms (of its row).
 * Clustering and event shapes run in FP64 for GAPS_FP64 contexts and in FP32
 * for GAPS_MIXED ones (the Z observables always in FP64).
 *   e+e-: 0 1-T, 1 y23, 2 y34 (Durham), 3 final partons, 4 emissions
 *   pp  : 0 Z pT, 1 Z rapidity, 2 Z phi (0 without emission), 3 anti-kT
 *         R=0.4 jets with pT > 5 GeV and |eta| < 5, 4 leading jet pT,
 *         5 leading jet eta, 6 final partons, 7 emissions */
int gaps_observables(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev,
                     double* obs, const gaps_hists* hists, void* stream);

/* The whole path over events first_event .. first_event + n - 1 in chunks of
 * ev->capacity: per chunk the hard process, the shower and the observables
 * (into obs_dev [GAPS_NOBS][capacity], device, may be NULL), the histograms
 * when hists != NULL and, when obs_host != NULL (pinned host memory,
 * [GAPS_NOBS][n], requires obs_dev), a copy of every event's observables.
 * The launches of all chunks are captured into one CUDA graph on a stream of
 * the context and launched on `stream` (asynchronous; the legacy default
 * stream is allowed). A later call with the same n and capacity updates the
 * graph's parameters in place instead of instantiating it again. Not to be
 * called while `stream` or the context's other calls are being captured.
 * With GAPS_MIXED and GAPS_SCHED_WAVE and two or more chunks the context
 * allocates a second slot (records and observables like `ev` and obs_dev, and
 * a second wavefront working set, about 100 GB for 2^22 events of 128 slots)
 * and the graph runs the odd chunks there on a second stream, concurrently
 * with the even ones in `ev`; obs_host and the histograms are the same, but
 * after the call `ev` and obs_dev hold only the even chunks' records and
 * observables. When that memory cannot be allocated the chunks run one after
 * another as without it. */
int gaps_process(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev,
                 double* obs_dev, double* obs_host, const gaps_hists* hists, void* stream);

/* Duration in ms of each chunk's shower in the last gaps_process call, timed
 * by events recorded inside its graph; waits for that call to finish. Writes
 * at most max_chunks values and returns how many (>= 0), or an error code. */
int gaps_process_shower_ms(gaps_ctx* ctx, float* ms, int max_chunks);

/* Binning of histogram h (0 .. GAPS_NHIST-1, or 0 .. n_mix * GAPS_NHIST - 1
 * over the rows of a mixed batch) of the context's process:
 * lo, hi, number of regular bins (<= 64), observable index and whether the
 * observable is binned in log10. Returns GAPS_ERR_INVALID_ARG for bad h. */
int gaps_hist_binning(const gaps_ctx* ctx, int h, double* lo, double* hi,
                      int* nbins, int* obs_index, int* log10_axis);

/* Synchronises `stream` and copies the accumulated counters. */
int gaps_get_stats(gaps_ctx* ctx, gaps_stats* out, void* stream);

/* Zeroes the counters (asynchronously on `stream`). */
int gaps_reset_stats(gaps_ctx* ctx, void* stream);

/* Static description of a return code; never NULL. */
const char* gaps_error_string(int code);

/* Frees the context and its device memory. NULL is ignored. */
void gaps_destroy(gaps_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GAPS_H */
