// C ABI of the shower library (include/gaps.h): configuration checks, the
// library-owned device state (PDF grid, certified bound tables, counters) and
// the launches of the hard-process, shower and observable kernels.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "gmath.cuh"

namespace gaps {
cudaError_t launch_generate_hard(const DevParams&, const DevEvents&, uint64_t, uint64_t, int, cudaStream_t);
cudaError_t launch_shower_fp64(const DevParams&, const DevEvents&, uint64_t, uint64_t, int, int,
                               unsigned long long*, cudaStream_t);
void workset_carve(void* base, int lanes, int nmax, WorkSet& W);
cudaError_t launch_shower_mixed(const DevParams&, const DevEvents&, const WorkSet&, const LearnedCfg&, uint64_t,
                                uint64_t, int, int, int, int, int, int, unsigned long long*, cudaStream_t);
cudaError_t launch_isr_targets(const DevParams&, int, const float4*, uint64_t, float*, float*, cudaStream_t);
cudaError_t mixed_kernels_init();
cudaError_t launch_mlp_image(const float* params, void* image, cudaStream_t stream);
size_t mlp_image_bytes();
cudaError_t launch_shower_warp(const DevParams&, const DevEvents&, const LearnedCfg&, uint64_t, uint64_t, int, int,
                               int, int, unsigned long long*, cudaStream_t);
cudaError_t launch_shower_wave(const DevParams&, const DevEvents&, const WorkSet&, const WaveSet&, const LearnedCfg&,
                               uint64_t, uint64_t, int, int, int, int, int, int, int, int, int, cudaStream_t);
cudaError_t launch_observables(const DevParams&, const DevEvents&, uint64_t, uint64_t, double*,
                               const HistSet&, double*, double*, int, int, cudaStream_t);
cudaError_t observables_init();
cudaError_t sort_states(float4*, uint64_t, cudaStream_t);
cudaError_t floor_values(float*, uint64_t, float, cudaStream_t);
cudaError_t mlp_init(float*, uint64_t, cudaStream_t);
cudaError_t calibration_init(int*, unsigned*, cudaStream_t);
cudaError_t calibration_accumulate(const float*, const float*, const float*, uint64_t, int*, unsigned*,
                                   cudaStream_t);
cudaError_t calibration_margins(const int*, const unsigned*, unsigned, float, float, float*, unsigned*,
                                cudaStream_t);
cudaError_t calibration_stats(const float*, const float*, const float*, uint64_t, const float*, double*,
                              cudaStream_t);
}  // namespace gaps

using namespace gaps;

struct gaps_ctx {
  gaps_config cfg;
  int device = 0;
  int n_sm = 0;
  float* d_grid = nullptr;
  double* d_tables = nullptr;  // umax [12][100], sufmax [12][101], lmin [12][100]
  unsigned long long* d_counters = nullptr;  // C_NCOUNTERS + 1 (work counter)
  DevParams P;
  HistSet H;   // binning per row (one row for one process)
  int q_independent = 0;     // every Q^2 column of the grid is identical
  void* d_work = nullptr;    // mixed-precision working set
  size_t work_bytes = 0;
  void* d_wave = nullptr;    // wavefront schedule: working set with one lane per event, then its state
  size_t wave_bytes = 0;
  uint64_t wave_cap = 0;
  float* d_mlp = nullptr;    // learned-proposal network (FP32 parameters)
  void* d_mlp_image = nullptr;  // its BF16 weight image for the shower
  int learned = 0;
  float* vlog = nullptr;     // caller's violation log (device), capacity, counter
  uint64_t vcap = 0;
  uint64_t* vcount = nullptr;
  // gaps_process: capture stream and the instantiated graph of the last call
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_n = 0, graph_cap = 0;
  std::vector<cudaEvent_t> shower_ev;  // start/stop of each chunk's shower in the graph
  int graph_chunks = 0;
  // gaps_process with the wavefront schedule: a second slot (event records,
  // observables, working set) for every other chunk, run on a second stream so
  // that the tail of one chunk's shower overlaps the next chunk
  void* d_slot2 = nullptr;   // records and observables of the second slot
  size_t slot2_bytes = 0;
  gaps_events ev2{};
  double* obs2 = nullptr;
  void* d_wave2 = nullptr;   // its wavefront working set and state
  size_t wave_bytes2 = 0;
  uint64_t wave_cap2 = 0;
  cudaStream_t cap_stream2 = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

namespace gaps {

// Per-node extrema of the grid over Q^2 and their suffix maxima in x: the
// ingredients of the certified PDF-ratio bound (index 11 = sum of the ten
// quark and antiquark densities). `out` holds kBoundTableDoubles values:
// umax [12][NX], sufmax [12][NX+1], lmin [12][NX].
//
// Heavy-quark thresholds (App. A.2): a c, b, cbar or bbar table whose nodes
// vanish for every x on all Q^2 nodes up to k0 and are positive above has its
// mass on node k0; for it lmin is the minimum over the nodes above k0 and
// first[f][ix] the value on node k0 + 1 (the tables of the measure
// correction's bound). thr / m2 (when not NULL, [12]) receive k0 (-1: none)
// and the mass squared, exp(ln Q2min + k0 dlq).
void build_bound_tables(const float* g, double* out, int* thr, double* m2) {
  const int NX = GAPS_PDF_NX, NQ = GAPS_PDF_NQ;
  double* umax = out;
  double* sufmax = umax + 12 * NX;
  double* lmin = sufmax + 12 * (NX + 1);
  double* first = lmin + 12 * NX;
  auto node = [&](int f, int ix, int iq) -> double {
    if (f < 11) return (double)g[((size_t)f * NX + ix) * NQ + iq];
    double s = 0.0;
    for (int k = 1; k <= 10; ++k) s += (double)g[((size_t)k * NX + ix) * NQ + iq];
    return s;
  };
  auto threshold = [&](int f) -> int {
    if (f != 4 && f != 5 && f != 9 && f != 10) return -1;
    int k0 = -1;
    for (int iq = 0; iq < NQ; ++iq) {
      bool zero = true;
      for (int ix = 0; ix < NX && zero; ++ix) zero = node(f, ix, iq) == 0.0;
      if (!zero) break;
      k0 = iq;
    }
    if (k0 < 0 || k0 >= NQ - 1) return -1;
    for (int iq = k0 + 1; iq < NQ; ++iq)
      for (int ix = 0; ix < NX; ++ix)
        if (!(node(f, ix, iq) > 0.0)) return -1;
    return k0;
  };
  const double lqmin = gm_log(GAPS_PDF_Q2MIN);
  const double dlq = (gm_log(GAPS_PDF_Q2MAX) - lqmin) / (GAPS_PDF_NQ - 1);
  for (int f = 0; f < 12; ++f) {
    const int k0 = f < 11 ? threshold(f) : -1;
    if (thr) thr[f] = k0;
    if (m2) m2[f] = k0 >= 0 ? gm_exp(lqmin + (double)k0 * dlq) : 0.0;
    for (int ix = 0; ix < NX; ++ix) {
      first[f * NX + ix] = k0 >= 0 ? node(f, ix, k0 + 1) : 0.0;
      double mx = node(f, ix, 0), mn = 0.0;
      for (int iq = 1; iq < NQ; ++iq) {
        double v = node(f, ix, iq);
        if (v > mx) mx = v;
      }
      for (int iq = k0 + 1; iq < NQ; ++iq) {
        double v = node(f, ix, iq);
        if (iq == k0 + 1 || v < mn) mn = v;
      }
      umax[f * NX + ix] = mx;
      lmin[f * NX + ix] = mn;
    }
    sufmax[f * (NX + 1) + NX] = 0.0;
    for (int ix = NX - 1; ix >= 0; --ix) {
      double a = umax[f * NX + ix], b = sufmax[f * (NX + 1) + ix + 1];
      sufmax[f * (NX + 1) + ix] = a > b ? a : b;
    }
  }
}

// the device tables of a context or call: pointers into one array of
// kBoundTableDoubles values and the thresholds of the host grid
void set_bound_tables(DevParams& P, const double* t, const float* host_grid) {
  P.umax = t;
  P.sufmax = t + 12 * GAPS_PDF_NX;
  P.lmin = t + 12 * GAPS_PDF_NX + 12 * (GAPS_PDF_NX + 1);
  P.first = t + 12 * GAPS_PDF_NX + 12 * (GAPS_PDF_NX + 1) + 12 * GAPS_PDF_NX;
  std::vector<double> tmp(kBoundTableDoubles);
  if (host_grid) {
    build_bound_tables(host_grid, tmp.data(), P.thr, P.m2);
  } else {
    for (int f = 0; f < 12; ++f) { P.thr[f] = -1; P.m2[f] = 0.0; }
  }
}

// GAPS_OK or GAPS_ERR_INVALID_ARG for a configuration (no device work)
// the one-process configuration of row r of a mixed batch
gaps_config row_config(const gaps_config& c, int r) {
  gaps_config k = c;
  k.n_mix = 0;
  k.process = c.mix[r].process;
  k.sqrt_s = c.mix[r].sqrt_s;
  k.t_cut = c.mix[r].t_cut;
  return k;
}

int validate_config(const gaps_config& c) {
  if (c.n_mix < 0 || c.n_mix > GAPS_MAX_MIX) return GAPS_ERR_INVALID_ARG;
  if (c.n_mix > 0) {
    double sum = 0.0;
    for (int r = 0; r < c.n_mix; ++r) {
      const double f = c.mix[r].fraction;
      if (!(f > 0.0) || !std::isfinite(f)) return GAPS_ERR_INVALID_ARG;
      sum += f;
      const int rc = validate_config(row_config(c, r));
      if (rc != GAPS_OK) return rc;
    }
    return std::fabs(sum - 1.0) <= 1e-9 ? GAPS_OK : GAPS_ERR_INVALID_ARG;
  }
  if (c.process < GAPS_EE_QQ || c.process > GAPS_PP_LL) return GAPS_ERR_INVALID_ARG;
  if (c.process == GAPS_PP_LL &&
      !(c.mll_lo > 0.0 && c.mll_lo < c.mll_hi && c.mll_hi <= c.sqrt_s && std::isfinite(c.mll_hi)))
    return GAPS_ERR_INVALID_ARG;
  if (c.precision != GAPS_FP64 && c.precision != GAPS_MIXED) return GAPS_ERR_INVALID_ARG;
  if (!(c.sqrt_s > 0.0) || !std::isfinite(c.sqrt_s)) return GAPS_ERR_INVALID_ARG;
  if (c.process != GAPS_EE_QQ && !(c.sqrt_s > 91.1876 && c.sqrt_s <= 13600.0)) return GAPS_ERR_INVALID_ARG;
  if (!(c.t_cut >= GAPS_PDF_Q2MIN) || !std::isfinite(c.t_cut)) return GAPS_ERR_INVALID_ARG;
  if (!(c.alpha_s_mz > 0.0 && c.alpha_s_mz < 1.0)) return GAPS_ERR_INVALID_ARG;
  if (c.nf < 1 || c.nf > 5) return GAPS_ERR_INVALID_ARG;
  if (c.nmax_partons < 4 || c.nmax_partons > 128) return GAPS_ERR_INVALID_ARG;
  if (c.process == GAPS_PP_Z_NLO && !(c.p_s > 0.0 && c.p_s < 1.0)) return GAPS_ERR_INVALID_ARG;
  if (c.process != GAPS_EE_QQ && !c.pdf_grid) return GAPS_ERR_INVALID_ARG;
  if (c.block_size < 0 || c.block_size > 1024 || (c.block_size % 32) != 0) return GAPS_ERR_INVALID_ARG;
  if (c.schedule != GAPS_SCHED_PER_EVENT && c.schedule != GAPS_SCHED_PERSISTENT && c.schedule != GAPS_SCHED_WARP &&
      c.schedule != GAPS_SCHED_WAVE)
    return GAPS_ERR_INVALID_ARG;
  if ((c.schedule == GAPS_SCHED_WARP || c.schedule == GAPS_SCHED_WAVE) && c.precision != GAPS_MIXED)
    return GAPS_ERR_INVALID_ARG;
  if (c.wave_passes < 0 || c.wave_passes > 4096) return GAPS_ERR_INVALID_ARG;
  if (c.wave_cycles < 0 || c.wave_cycles > 1000000) return GAPS_ERR_INVALID_ARG;
  if (c.wave_veto_blocks_per_sm != 0 && (c.wave_veto_blocks_per_sm < 2 || c.wave_veto_blocks_per_sm > 4))
    return GAPS_ERR_INVALID_ARG;
  if (c.trial_mode != GAPS_TRIALS_REDRAW && c.trial_mode != GAPS_TRIALS_KEEP && c.trial_mode != GAPS_TRIALS_SELECT &&
      c.trial_mode != GAPS_TRIALS_VETOMAX)
    return GAPS_ERR_INVALID_ARG;
  if (c.trial_mode == GAPS_TRIALS_VETOMAX && (c.precision != GAPS_MIXED || c.schedule != GAPS_SCHED_PERSISTENT))
    return GAPS_ERR_INVALID_ARG;
  if (c.trial_mode != GAPS_TRIALS_REDRAW &&
      (c.precision != GAPS_MIXED || (c.schedule != GAPS_SCHED_PERSISTENT && c.schedule != GAPS_SCHED_WAVE)))
    return GAPS_ERR_INVALID_ARG;
  if (c.blocks_per_sm < 0 || c.blocks_per_sm > 64) return GAPS_ERR_INVALID_ARG;
  if (c.refill_period < 0 || c.refill_period > 1000000) return GAPS_ERR_INVALID_ARG;
  if (c.emit_batch < 0 || c.emit_batch > 32) return GAPS_ERR_INVALID_ARG;
  if (c.max_cycles < 0 || c.max_cycles > 1000000000) return GAPS_ERR_INVALID_ARG;
  if (c.precision == GAPS_MIXED && c.block_size != 0 && c.block_size != 64 && c.block_size != 128 &&
      c.block_size != 256)
    return GAPS_ERR_INVALID_ARG;
  // one-loop running must stay below its pole down to the cutoff
  const double beta0 = (33.0 - 2.0 * 5.0) / (12.0 * 3.14159265358979323846);
  double den = 1.0 + c.alpha_s_mz * beta0 * gm_log(c.t_cut / (91.1876 * 91.1876));
  if (!(den > 0.0)) return GAPS_ERR_INVALID_ARG;
  if (c.pdf_grid) {
    const size_t gsz = (size_t)GAPS_PDF_NFL * GAPS_PDF_NX * GAPS_PDF_NQ;
    for (size_t q = 0; q < gsz; ++q)
      if (!std::isfinite(c.pdf_grid[q]) || c.pdf_grid[q] < 0.0f) return GAPS_ERR_INVALID_ARG;
    // heavy-quark thresholds: the measure correction is built into the FP64
    // kernels and the mixed-precision trials of the kept and redrawn schemes
    std::vector<double> tmp(kBoundTableDoubles);
    int thr[12];
    build_bound_tables(c.pdf_grid, tmp.data(), thr, nullptr);
    bool heavy = false;
    for (int f = 0; f < 12; ++f) heavy = heavy || thr[f] >= 0;
    if (heavy && c.precision == GAPS_MIXED &&
        (c.schedule == GAPS_SCHED_WARP || c.trial_mode == GAPS_TRIALS_SELECT || c.trial_mode == GAPS_TRIALS_VETOMAX))
      return GAPS_ERR_INVALID_ARG;
  }
  return GAPS_OK;
}

// scalar parameters of a configuration (device pointers left unset)
void fill_params(const gaps_config& c, DevParams& P) {
  if (c.n_mix > 0) {
    // row 0 fills the scalar fields; each row its own process-dependent part
    fill_params(row_config(c, 0), P);
    double cum = 0.0;
    for (int r = 0; r < c.n_mix; ++r) {
      DevParams Q;
      fill_params(row_config(c, r), Q);
      P.rows[r] = Q.rows[0];
      cum += c.mix[r].fraction;  // summed in row order, as the selection compares
      P.cum[r] = cum;
    }
    P.n_rows = c.n_mix;
    return;
  }
  const double beta0 = (33.0 - 2.0 * 5.0) / (12.0 * 3.14159265358979323846);
  double den = 1.0 + c.alpha_s_mz * beta0 * gm_log(c.t_cut / (91.1876 * 91.1876));
  P.process = c.process;
  P.trial_mode = c.trial_mode;
  P.max_steps = c.max_cycles > 0 ? c.max_cycles : kMaxSteps;
  P.fit_on = 0;
  for (int a = 0; a < 12; ++a)
    for (int b = 0; b < 12; ++b) P.fit[a][b][0] = P.fit[a][b][1] = 0.0f;
  // images of the dilepton mass window under m^2 = m_Z^2 + m_Z Gamma_Z tan(2 pi r)
  {
    const double mg = kMZ * kGZ, mz2 = kMZ * kMZ;
    const double lo = c.mll_lo > 0.0 ? c.mll_lo : 66.0, hi = c.mll_hi > 0.0 ? c.mll_hi : 116.0;
    P.ll_rlo = std::atan((lo * lo - mz2) / mg) / kGmTwoPi;
    P.ll_rhi = std::atan((hi * hi - mz2) / mg) / kGmTwoPi;
  }
  P.nf = c.nf;
  P.nmax = c.nmax_partons;
  P.sqrt_s = c.sqrt_s;
  P.s_had = c.sqrt_s * c.sqrt_s;
  P.t_cut = c.t_cut;
  P.as_mz = c.alpha_s_mz;
  P.beta0 = beta0;
  P.as_over = c.alpha_s_mz / den;  // alpha_s(t_cut), the overestimate of Appendix A.2
  P.p_s = c.p_s;
  P.seed = c.seed;
  P.lxmin = gm_log(GAPS_PDF_XMIN);
  P.dlx = (gm_log(GAPS_PDF_XMAX) - P.lxmin) / (GAPS_PDF_NX - 1);
  P.lqmin = gm_log(GAPS_PDF_Q2MIN);
  P.dlq = (gm_log(GAPS_PDF_Q2MAX) - P.lqmin) / (GAPS_PDF_NQ - 1);
  P.n_rows = 1;
  P.rows[0] = RowParams{P.process, P.sqrt_s, P.s_had, P.t_cut, P.as_over};
  P.cum[0] = 1.0;
  for (int r = 1; r < kMaxRows; ++r) { P.rows[r] = P.rows[0]; P.cum[r] = 1.0; }
}

// 1 when every Q^2 column of the grid is identical
int grid_q_independent(const float* g) {
  if (!g) return 1;
  const size_t gsz = (size_t)GAPS_PDF_NFL * GAPS_PDF_NX * GAPS_PDF_NQ;
  for (size_t q = 0; q < gsz; q += GAPS_PDF_NQ)
    for (int iq = 1; iq < GAPS_PDF_NQ; ++iq)
      if (g[q + iq] != g[q]) return 0;
  return 1;
}

}  // namespace gaps

namespace {

int cuda_fail(cudaError_t e) { return e == cudaSuccess ? GAPS_OK : GAPS_ERR_CUDA; }

bool events_ok(const gaps_ctx* c, const gaps_events* ev, uint64_t n) {
  if (!ev || !ev->p || !ev->flav || !ev->col || !ev->acol || !ev->npart || !ev->status ||
      !ev->n_emit || !ev->weight || !ev->t || !ev->eta || !ev->draw)
    return false;
  if (n > ev->capacity) return false;
  if (ev->nmax != c->cfg.nmax_partons) return false;
  return true;
}

DevEvents dev_events(const gaps_events* ev) {
  DevEvents E;
  E.cap = ev->capacity; E.nmax = ev->nmax; E.p = ev->p; E.flav = ev->flav; E.col = ev->col;
  E.acol = ev->acol; E.npart = ev->npart; E.status = ev->status; E.n_emit = ev->n_emit;
  E.weight = ev->weight; E.t = ev->t; E.eta = ev->eta; E.draw = ev->draw;
  return E;
}

void set_hist_defs(int process, HistDef& H) {
  const double pi = 3.14159265358979323846;
  if (process == GAPS_EE_QQ) {
    // 1-T, log10 y23, log10 y34, final partons, emissions, log10(1-T)
    const double lo[6] = {0.0, -5.0, -5.0, -0.5, -0.5, -4.0};
    const double hi[6] = {0.5, 0.0, 0.0, 63.5, 63.5, 0.0};
    const int nb[6] = {50, 50, 50, 64, 64, 40}, ob[6] = {0, 1, 2, 3, 4, 0}, lg[6] = {0, 1, 1, 0, 0, 1};
    for (int h = 0; h < 6; ++h) { H.lo[h] = lo[h]; H.hi[h] = hi[h]; H.nb[h] = nb[h]; H.obs[h] = ob[h]; H.logx[h] = lg[h]; }
  } else {
    // log10 Z pT, Z y, Z phi, jets, log10 leading-jet pT, final partons
    const double lo[6] = {-1.0, -6.0, -pi, -0.5, 0.5, -0.5};
    const double hi[6] = {3.0, 6.0, pi, 15.5, 3.5, 127.5};
    const int nb[6] = {40, 48, 32, 16, 30, 64}, ob[6] = {0, 1, 2, 3, 4, 6}, lg[6] = {1, 0, 0, 0, 1, 0};
    for (int h = 0; h < 6; ++h) { H.lo[h] = lo[h]; H.hi[h] = hi[h]; H.nb[h] = nb[h]; H.obs[h] = ob[h]; H.logx[h] = lg[h]; }
  }
}

}  // namespace

extern "C" {

const char* gaps_error_string(int code) {
  switch (code) {
    case GAPS_OK: return "ok";
    case GAPS_ERR_INVALID_ARG: return "invalid argument";
    case GAPS_ERR_CAPACITY: return "an event exceeded its parton capacity";
    case GAPS_ERR_ITER_CAP: return "an event exceeded the shower step cap";
    case GAPS_ERR_NUMERIC: return "non-finite scale or weight";
    case GAPS_ERR_CUDA: return "CUDA runtime error";
    case GAPS_ERR_NO_DEVICE: return "no CUDA device";
    default: return "unknown error";
  }
}

int gaps_init(gaps_ctx** out, const gaps_config* cfg) {
  if (!out || !cfg) return GAPS_ERR_INVALID_ARG;
  const gaps_config& c = *cfg;
  int vrc = validate_config(c);
  if (vrc != GAPS_OK) return vrc;

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return GAPS_ERR_NO_DEVICE;
  gaps_ctx* ctx = new (std::nothrow) gaps_ctx();
  if (!ctx) return GAPS_ERR_CUDA;
  ctx->cfg = c;
  ctx->cfg.pdf_grid = nullptr;
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  int rc = GAPS_OK;
  do {
    const size_t gsz = (size_t)GAPS_PDF_NFL * GAPS_PDF_NX * GAPS_PDF_NQ;
    if ((rc = cuda_fail(cudaMalloc(&ctx->d_grid, gsz * sizeof(float))))) break;
    std::vector<float> zero;
    const float* g = c.pdf_grid;
    if (!g) { zero.assign(gsz, 0.0f); g = zero.data(); }
    if ((rc = cuda_fail(cudaMemcpy(ctx->d_grid, g, gsz * sizeof(float), cudaMemcpyHostToDevice)))) break;
    ctx->q_independent = grid_q_independent(g);
    std::vector<double> tables(kBoundTableDoubles);
    build_bound_tables(g, tables.data());
    if ((rc = cuda_fail(cudaMalloc(&ctx->d_tables, tables.size() * sizeof(double))))) break;
    if ((rc = cuda_fail(cudaMemcpy(ctx->d_tables, tables.data(), tables.size() * sizeof(double),
                                   cudaMemcpyHostToDevice)))) break;
    if ((rc = cuda_fail(cudaMalloc(&ctx->d_counters, (C_NCOUNTERS + 1) * sizeof(unsigned long long))))) break;
    if ((rc = cuda_fail(cudaMemset(ctx->d_counters, 0, (C_NCOUNTERS + 1) * sizeof(unsigned long long))))) break;
    if ((rc = cuda_fail(mixed_kernels_init()))) break;
    if ((rc = cuda_fail(observables_init()))) break;
  } while (false);
  if (rc != GAPS_OK) {
    gaps_destroy(ctx);
    return rc;
  }
  DevParams& P = ctx->P;
  fill_params(c, P);
  P.grid = ctx->d_grid;
  set_bound_tables(P, ctx->d_tables, c.pdf_grid);
  P.counters = ctx->d_counters;
  for (int r = 0; r < P.n_rows; ++r) set_hist_defs(P.rows[r].process, ctx->H.h[r]);
  *out = ctx;
  return GAPS_OK;
}

int gaps_generate_hard(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev,
                       void* stream) {
  if (!ctx || !events_ok(ctx, ev, n)) return GAPS_ERR_INVALID_ARG;
  return cuda_fail(launch_generate_hard(ctx->P, dev_events(ev), first_event, n,
                                       ctx->cfg.precision == GAPS_MIXED ? 1 : 0, (cudaStream_t)stream));
}

namespace {
// working set of the mixed-precision shower for the context's launch shape
// (allocated on first use)
int ensure_workset(gaps_ctx* ctx, int& blocks, int& bs, WorkSet& W) {
  const gaps_config& c = ctx->cfg;
  bs = c.block_size > 0 ? c.block_size : 128;
  int per_sm = c.blocks_per_sm > 0 ? c.blocks_per_sm : 4;
  blocks = ctx->n_sm * per_sm;
  int lanes = blocks * bs;
  // the kernels index the working set with 32-bit element offsets
  if ((size_t)lanes * 4 * (size_t)c.nmax_partons >= ((size_t)1 << 31)) return GAPS_ERR_INVALID_ARG;
  size_t need = workset_bytes(lanes, c.nmax_partons);
  if (need > ctx->work_bytes) {
    if (ctx->d_work) cudaFree(ctx->d_work);
    ctx->d_work = nullptr;
    ctx->work_bytes = 0;
    if (cudaMalloc(&ctx->d_work, need) != cudaSuccess) return GAPS_ERR_CUDA;
    ctx->work_bytes = need;
  }
  workset_carve(ctx->d_work, lanes, c.nmax_partons, W);
  return GAPS_OK;
}

// working set and state of the wavefront schedule for `cap` events
// (allocated on first use, grown when a larger capacity comes)
constexpr int kWavePassesDefault = 24;
constexpr int kWaveCyclesDefault = 64;  // veto cycles of one event in one pass
int ensure_wave(gaps_ctx* ctx, uint64_t cap, WorkSet& W, WaveSet& V, int slot = 0) {
  const int nmax = ctx->cfg.nmax_partons;
  // the kernels index the working set with unsigned 32-bit element offsets
  if (cap * 4 * (uint64_t)nmax >= ((uint64_t)1 << 32) || cap >= ((uint64_t)1 << 31)) return GAPS_ERR_INVALID_ARG;
  void*& mem = slot ? ctx->d_wave2 : ctx->d_wave;
  size_t& bytes = slot ? ctx->wave_bytes2 : ctx->wave_bytes;
  uint64_t& have = slot ? ctx->wave_cap2 : ctx->wave_cap;
  const size_t wb = (workset_bytes((int)cap, nmax) + 255) / 256 * 256;
  const size_t need = wb + wave_state_bytes(cap);
  if (need > bytes || cap > have) {
    if (mem) cudaFree(mem);
    mem = nullptr;
    bytes = 0;
    have = 0;
    if (cudaMalloc(&mem, need) != cudaSuccess) {
      cudaGetLastError();
      return GAPS_ERR_CUDA;
    }
    bytes = need;
    have = cap;
  }
  workset_carve(mem, (int)cap, nmax, W);
  wave_state_carve((char*)mem + wb, cap, V);
  return GAPS_OK;
}

int shower_wave(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev, const LearnedCfg& Lc,
                void* stream, int slot = 0) {
  const gaps_config& c = ctx->cfg;
  WorkSet W;
  WaveSet V;
  const int rc = ensure_wave(ctx, ev->capacity, W, V, slot);
  if (rc != GAPS_OK) return rc;
  const int bs = c.block_size > 0 ? c.block_size : 128;
  const int per_sm = c.blocks_per_sm > 0 ? c.blocks_per_sm : 4;
  const int passes = c.wave_passes > 0 ? c.wave_passes : kWavePassesDefault;
  const int cycles = c.wave_cycles > 0 ? c.wave_cycles : kWaveCyclesDefault;
  // the veto kernel runs best with 128 registers a thread (no spills)
  const int veto_per_sm = c.wave_veto_blocks_per_sm > 0 ? c.wave_veto_blocks_per_sm : 2;
  return cuda_fail(launch_shower_wave(ctx->P, dev_events(ev), W, V, Lc, first_event, n, passes, cycles,
                                      ctx->n_sm * per_sm, ctx->n_sm * veto_per_sm, bs, ctx->n_sm, c.refill_period,
                                      c.emit_batch, ctx->q_independent, (cudaStream_t)stream));
}

int shower_mixed(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev, const LearnedCfg& Lc,
                 void* stream) {
  const gaps_config& c = ctx->cfg;
  int blocks, bs;
  WorkSet W;
  const int rc = ensure_workset(ctx, blocks, bs, W);
  if (rc != GAPS_OK) return rc;
  return cuda_fail(launch_shower_mixed(ctx->P, dev_events(ev), W, Lc, first_event, n, blocks, bs, ctx->n_sm,
                                       c.refill_period, c.emit_batch, ctx->q_independent,
                                       ctx->d_counters + C_NCOUNTERS, (cudaStream_t)stream));
}
}  // namespace

namespace {
// gaps_shower; slot 1: the second wavefront slot of gaps_process
int shower_impl(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev, void* stream, int slot) {
  const gaps_config& c = ctx->cfg;
  if (c.precision == GAPS_MIXED) {
    LearnedCfg Lc{};
    bool any_pp = false;
    for (int r = 0; r < ctx->P.n_rows; ++r) any_pp = any_pp || ctx->P.rows[r].process != GAPS_EE_QQ;
    // veto-max runs every channel's veto with the plain bounds
    Lc.learned = ctx->learned && ctx->d_mlp && any_pp && c.trial_mode != GAPS_TRIALS_VETOMAX;
    Lc.mlp = ctx->d_mlp;
    Lc.image = ctx->d_mlp_image;
    Lc.vlog = reinterpret_cast<float4*>(ctx->vlog);
    Lc.vcount = reinterpret_cast<unsigned long long*>(ctx->vcount);
    Lc.vcap = ctx->vcap;
    if (c.schedule == GAPS_SCHED_WARP) {
      const int bs = c.block_size > 0 ? c.block_size : 128;
      const int per_sm = c.blocks_per_sm > 0 ? c.blocks_per_sm : 2;
      return cuda_fail(launch_shower_warp(ctx->P, dev_events(ev), Lc, first_event, n, ctx->n_sm * per_sm, bs,
                                          per_sm, ctx->q_independent, ctx->d_counters + C_NCOUNTERS,
                                          (cudaStream_t)stream));
    }
    if (c.schedule == GAPS_SCHED_WAVE) return shower_wave(ctx, first_event, n, ev, Lc, stream, slot);
    return shower_mixed(ctx, first_event, n, ev, Lc, stream);
  }
  int bs = c.block_size > 0 ? c.block_size : 128;
  int pblocks = 0;
  if (c.schedule == GAPS_SCHED_PERSISTENT) {
    int per_sm = c.blocks_per_sm > 0 ? c.blocks_per_sm : 4;
    pblocks = ctx->n_sm * per_sm;
  }
  return cuda_fail(launch_shower_fp64(ctx->P, dev_events(ev), first_event, n, bs, pblocks,
                                      ctx->d_counters + C_NCOUNTERS, (cudaStream_t)stream));
}
}  // namespace

int gaps_shower(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev, void* stream) {
  if (!ctx || !events_ok(ctx, ev, n)) return GAPS_ERR_INVALID_ARG;
  return shower_impl(ctx, first_event, n, ev, stream, 0);
}

int gaps_collect_isr_states(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev,
                            float keep_fraction, float* states, uint64_t capacity, uint64_t* count,
                            void* stream) {
  if (!ctx || !events_ok(ctx, ev, n) || !states || !count) return GAPS_ERR_INVALID_ARG;
  if (!(keep_fraction > 0.0f && keep_fraction <= 1.0f)) return GAPS_ERR_INVALID_ARG;
  if (ctx->cfg.n_mix > 0 || ctx->cfg.process == GAPS_EE_QQ || ctx->cfg.precision != GAPS_MIXED)
    return GAPS_ERR_INVALID_ARG;
  LearnedCfg Lc{};
  Lc.collect = reinterpret_cast<float4*>(states);
  Lc.collect_count = reinterpret_cast<unsigned long long*>(count);
  Lc.collect_cap = capacity;
  Lc.collect_keep = keep_fraction >= 1.0f ? 0xFFFFFFFFu : (uint32_t)((double)keep_fraction * 4294967296.0);
  return shower_mixed(ctx, first_event, n, ev, Lc, stream);
}

int gaps_isr_targets(gaps_ctx* ctx, const float* states, uint64_t n_states, float* features, float* targets,
                     void* stream) {
  if (!ctx || !states || !features || !targets) return GAPS_ERR_INVALID_ARG;
  if (ctx->cfg.n_mix > 0 || ctx->cfg.process == GAPS_EE_QQ) return GAPS_ERR_INVALID_ARG;
  return cuda_fail(launch_isr_targets(ctx->P, ctx->q_independent, reinterpret_cast<const float4*>(states),
                                      n_states, features, targets, (cudaStream_t)stream));
}

int gaps_set_learned_proposal(gaps_ctx* ctx, const float* params, const float* log_margins) {
  if (!ctx) return GAPS_ERR_INVALID_ARG;
  if (!params) {
    ctx->learned = 0;
    return GAPS_OK;
  }
  if (!log_margins) return GAPS_ERR_INVALID_ARG;
  constexpr int nm = GAPS_ISR_CLASSES * GAPS_ISR_ETA_BINS * GAPS_ISR_BINS;
  for (int q = 0; q < GAPS_MLP_PARAMS; ++q)
    if (!std::isfinite(params[q])) return GAPS_ERR_INVALID_ARG;
  for (int q = 0; q < nm; ++q)
    if (!std::isfinite(log_margins[q])) return GAPS_ERR_INVALID_ARG;
  // device image: parameters, then the margins
  const size_t pbytes = (size_t)GAPS_MLP_PARAMS * sizeof(float);
  if (!ctx->d_mlp && cudaMalloc(&ctx->d_mlp, pbytes + nm * sizeof(float)) != cudaSuccess) return GAPS_ERR_CUDA;
  if (cudaMemcpy(ctx->d_mlp, params, pbytes, cudaMemcpyHostToDevice) != cudaSuccess) return GAPS_ERR_CUDA;
  if (cudaMemcpy(ctx->d_mlp + GAPS_MLP_PARAMS, log_margins, nm * sizeof(float), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return GAPS_ERR_CUDA;
  if (!ctx->d_mlp_image && cudaMalloc(&ctx->d_mlp_image, mlp_image_bytes()) != cudaSuccess) return GAPS_ERR_CUDA;
  if (launch_mlp_image(ctx->d_mlp, ctx->d_mlp_image, nullptr) != cudaSuccess) return GAPS_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return GAPS_ERR_CUDA;
  ctx->learned = 1;
  return GAPS_OK;
}

}  // extern "C"

namespace {

// device scratch of the training pipeline, freed on every return path
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  T* get(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return (T*)p;
  }
};

// event records of `cap` events with nmax slots, carved from one allocation
bool alloc_events(Scratch& sc, uint64_t cap, int nmax, gaps_events& ev) {
  ev.capacity = cap;
  ev.nmax = nmax;
  ev.p = sc.get<double>(4 * (size_t)nmax * cap);
  ev.flav = sc.get<int32_t>((size_t)nmax * cap);
  ev.col = sc.get<int32_t>((size_t)nmax * cap);
  ev.acol = sc.get<int32_t>((size_t)nmax * cap);
  ev.npart = sc.get<int32_t>(cap);
  ev.status = sc.get<int32_t>(cap);
  ev.n_emit = sc.get<int32_t>(cap);
  ev.weight = sc.get<double>(cap);
  ev.t = sc.get<double>(cap);
  ev.eta = sc.get<double>(2 * cap);
  ev.draw = sc.get<uint64_t>(cap);
  return ev.p && ev.flav && ev.col && ev.acol && ev.npart && ev.status && ev.n_emit && ev.weight && ev.t &&
         ev.eta && ev.draw;
}

uint64_t pow2_at_least(uint64_t n) {
  uint64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

// Showers n events from `first` in chunks and logs up to `capacity` states
// (kept with a fraction from a pilot run), sorted canonically; then the
// training rows. Returns the number of states, or a negative error code.
int64_t collect_rows(gaps_ctx* ctx, Scratch& sc, const gaps_events& ev, uint64_t first, uint64_t n,
                     uint64_t capacity, float floor, float*& feats, float*& targ, cudaStream_t st) {
  const uint64_t chunk = ev.capacity;
  uint64_t* d_count = sc.get<uint64_t>(1);
  if (!d_count) return GAPS_ERR_CUDA;
  // pilot: states per event with every state kept
  const uint64_t pilot = n < (1u << 14) ? n : (1u << 14);
  float* probe = sc.get<float>(4 * pilot * 64);
  if (!probe) return GAPS_ERR_CUDA;
  if (cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st) != cudaSuccess) return GAPS_ERR_CUDA;
  int rc = gaps_generate_hard(ctx, first - pilot, pilot, &ev, st);
  if (rc == GAPS_OK) rc = gaps_collect_isr_states(ctx, first - pilot, pilot, &ev, 1.0f, probe, pilot * 64, d_count, st);
  if (rc != GAPS_OK) return rc;
  uint64_t h_count = 0;
  if (cudaMemcpyAsync(&h_count, d_count, sizeof h_count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GAPS_ERR_CUDA;
  double per_event = (double)h_count / (double)(pilot ? pilot : 1);
  if (per_event < 1.0) per_event = 1.0;
  double keep = 0.95 * (double)capacity / (per_event * (double)n);
  if (keep > 1.0) keep = 1.0;
  if (!(keep > 0.0)) keep = 1e-9;
  const uint64_t cap2 = pow2_at_least(capacity);
  float* states = sc.get<float>(4 * cap2);
  if (!states) return GAPS_ERR_CUDA;
  if (cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st) != cudaSuccess) return GAPS_ERR_CUDA;
  for (uint64_t f0 = 0; f0 < n; f0 += chunk) {
    const uint64_t m = n - f0 < chunk ? n - f0 : chunk;
    rc = gaps_generate_hard(ctx, first + f0, m, &ev, st);
    if (rc == GAPS_OK) rc = gaps_collect_isr_states(ctx, first + f0, m, &ev, (float)keep, states, capacity, d_count, st);
    if (rc != GAPS_OK) return rc;
  }
  if (cudaMemcpyAsync(&h_count, d_count, sizeof h_count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GAPS_ERR_CUDA;
  const uint64_t m = h_count < capacity ? h_count : capacity;
  if (sort_states(reinterpret_cast<float4*>(states), m, st) != cudaSuccess) return GAPS_ERR_CUDA;
  feats = sc.get<float>(4 * 16 * m);
  targ = sc.get<float>(16 * m);
  if (!feats || !targ) return GAPS_ERR_CUDA;
  rc = gaps_isr_targets(ctx, states, m, feats, targ, st);
  if (rc != GAPS_OK) return rc;
  if (floor_values(targ, 16 * m, floor, st) != cudaSuccess) return GAPS_ERR_CUDA;
  return (int64_t)m;
}

}  // namespace

extern "C" {

int gaps_train_learned_proposal(gaps_ctx* ctx, const gaps_learn_config* lc, float* params_out,
                                float* log_margins_out, gaps_learn_report* report, void* stream) {
  if (!ctx || !lc) return GAPS_ERR_INVALID_ARG;
  const gaps_config& c = ctx->cfg;
  if (c.n_mix > 0 || c.process == GAPS_EE_QQ || c.precision != GAPS_MIXED) return GAPS_ERR_INVALID_ARG;
  if (lc->n_events == 0 || lc->capacity == 0 || lc->holdout_events == 0 || lc->holdout_capacity == 0 ||
      lc->steps < 4 || !(lc->lr > 0.0f) || !(lc->tau > 0.0f && lc->tau < 1.0f) || !(lc->slack >= 0.0f) ||
      !std::isfinite(lc->target_floor) || lc->first_event < (1u << 14) || lc->holdout_first < (1u << 14) ||
      lc->capacity > (1ull << 28) || lc->holdout_capacity > (1ull << 28))
    return GAPS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc;
  const uint64_t chunk = lc->n_events < (1u << 19) ? (lc->n_events < (1u << 14) ? (1u << 14) : lc->n_events)
                                                   : (1u << 19);
  gaps_events ev;
  if (!alloc_events(sc, chunk, c.nmax_partons, ev)) return GAPS_ERR_CUDA;
  // the collection runs the plain bound whatever the context holds
  const int had_learned = ctx->learned;
  ctx->learned = 0;
  float *feats = nullptr, *targ = nullptr, *hf = nullptr, *ht = nullptr;
  int64_t m = collect_rows(ctx, sc, ev, lc->first_event, lc->n_events, lc->capacity, lc->target_floor, feats, targ, st);
  int64_t mh = m < 0 ? m
                     : collect_rows(ctx, sc, ev, lc->holdout_first, lc->holdout_events, lc->holdout_capacity,
                                    lc->target_floor, hf, ht, st);
  ctx->learned = had_learned;
  if (m < 0) return (int)m;
  if (mh < 0) return (int)mh;
  if (m == 0) return GAPS_ERR_INVALID_ARG;  // nothing to train on
  const uint64_t rows = 16 * (uint64_t)m, hrows = 16 * (uint64_t)mh;
  // training
  float* P = sc.get<float>(GAPS_MLP_PARAMS);
  float* am = sc.get<float>(GAPS_MLP_PARAMS);
  float* av = sc.get<float>(GAPS_MLP_PARAMS);
  float* hist = sc.get<float>(lc->steps + 1);
  if (!P || !am || !av || !hist) return GAPS_ERR_CUDA;
  if (mlp_init(P, lc->seed, st) != cudaSuccess) return GAPS_ERR_CUDA;
  if (cudaMemsetAsync(am, 0, GAPS_MLP_PARAMS * sizeof(float), st) != cudaSuccess ||
      cudaMemsetAsync(av, 0, GAPS_MLP_PARAMS * sizeof(float), st) != cudaSuccess ||
      cudaMemsetAsync(hist, 0, (lc->steps + 1) * sizeof(float), st) != cudaSuccess)
    return GAPS_ERR_CUDA;
  const uint64_t phase[3] = {lc->steps / 2, lc->steps / 4, lc->steps - lc->steps / 2 - lc->steps / 4};
  const float lrs[3] = {lc->lr, lc->lr * 0.3f, lc->lr * 0.1f};
  uint64_t done = 0;
  for (int k = 0; k < 3; ++k) {
    const int rc = gaps_mlp_train(P, am, av, feats, targ, rows, phase[k], lrs[k], lc->tau, lc->seed + k, hist + done, 1,
                                  st);
    if (rc != GAPS_OK) return rc;
    done += phase[k];
  }
  // calibration: BF16 outputs of both sets, the largest gap per cell
  constexpr int ncell = GAPS_ISR_CLASSES * GAPS_ISR_ETA_BINS * GAPS_ISR_BINS;
  float* out = sc.get<float>(rows);
  float* hout = sc.get<float>(hrows);
  int* gap = sc.get<int>(ncell);
  unsigned* cnt = sc.get<unsigned>(ncell + 1);
  float* margins = sc.get<float>(ncell);
  double* sums = sc.get<double>(2);
  if (!out || !hout || !gap || !cnt || !margins || !sums) return GAPS_ERR_CUDA;
  int rc = gaps_mlp_forward(P, feats, rows, 1, out, st);
  if (rc == GAPS_OK && hrows) rc = gaps_mlp_forward(P, hf, hrows, 1, hout, st);
  if (rc != GAPS_OK) return rc;
  if (calibration_init(gap, cnt, st) != cudaSuccess ||
      cudaMemsetAsync(cnt + ncell, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(sums, 0, 2 * sizeof(double), st) != cudaSuccess ||
      calibration_accumulate(feats, targ, out, rows, gap, cnt, st) != cudaSuccess ||
      calibration_accumulate(hf, ht, hout, hrows, gap, cnt, st) != cudaSuccess ||
      calibration_margins(gap, cnt, lc->min_rows, lc->slack, 30.0f, margins, cnt + ncell, st) != cudaSuccess ||
      calibration_stats(feats, targ, out, rows, margins, sums, st) != cudaSuccess)
    return GAPS_ERR_CUDA;
  std::vector<float> hp(GAPS_MLP_PARAMS), hm(ncell);
  std::vector<float> hh(lc->steps);
  unsigned seen = 0;
  double hs[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(hp.data(), P, hp.size() * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(hm.data(), margins, hm.size() * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(hh.data(), hist, hh.size() * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&seen, cnt + ncell, sizeof seen, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GAPS_ERR_CUDA;
  rc = gaps_set_learned_proposal(ctx, hp.data(), hm.data());
  if (rc != GAPS_OK) return rc;
  if (params_out) std::memcpy(params_out, hp.data(), hp.size() * sizeof(float));
  if (log_margins_out) std::memcpy(log_margins_out, hm.data(), hm.size() * sizeof(float));
  if (report) {
    report->states = (uint64_t)m;
    report->rows = rows;
    report->holdout_states = (uint64_t)mh;
    report->loss_first = hh.empty() ? 0.0f : hh.front();
    report->loss_last = hh.empty() ? 0.0f : hh.back();
    report->cells_calibrated = seen;
    report->mean_bin_height = (float)(hs[0] / (double)rows);
    report->fit_rmse = (float)std::sqrt(hs[1] / (double)rows);
  }
  return GAPS_OK;
}

int gaps_collect_pdf_ratios(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev,
                            float keep_fraction, float* samples, uint64_t capacity, uint64_t* count,
                            void* stream) {
  if (!ctx || !events_ok(ctx, ev, n) || !samples || !count) return GAPS_ERR_INVALID_ARG;
  if (!(keep_fraction > 0.0f && keep_fraction <= 1.0f)) return GAPS_ERR_INVALID_ARG;
  if (ctx->cfg.precision != GAPS_MIXED) return GAPS_ERR_INVALID_ARG;
  LearnedCfg Lc{};
  Lc.rlog = reinterpret_cast<float4*>(samples);
  Lc.rcount = reinterpret_cast<unsigned long long*>(count);
  Lc.rcap = capacity;
  Lc.rkeep = keep_fraction >= 1.0f ? 0xFFFFFFFFu : (uint32_t)((double)keep_fraction * 4294967296.0);
  // the certified bounds, whatever fit the context holds
  const int fit_on = ctx->P.fit_on;
  ctx->P.fit_on = 0;
  const int rc = shower_mixed(ctx, first_event, n, ev, Lc, stream);
  ctx->P.fit_on = fit_on;
  return rc;
}

int gaps_fit_pdf_ratios(const float* samples, uint64_t n, float* fit) {
  if ((!samples && n) || !fit) return GAPS_ERR_INVALID_ARG;
  std::vector<std::vector<float>> by(12 * 12);
  for (uint64_t i = 0; i < n; ++i) {
    const float* r = samples + 4 * i;
    const int num = (int)r[0], den = (int)r[1];
    if (num < 0 || num > 11 || den < 0 || den > 11 || !std::isfinite(r[3])) return GAPS_ERR_INVALID_ARG;
    if (r[3] > 0.0f) by[num * 12 + den].push_back(r[3]);
  }
  // nearest-rank percentiles: the smallest sample with at least p of the
  // samples at or below it
  auto pct = [](std::vector<float>& v, double p) -> float {
    size_t k = (size_t)std::ceil(p * (double)v.size());
    if (k < 1) k = 1;
    std::nth_element(v.begin(), v.begin() + (k - 1), v.end());
    return v[k - 1];
  };
  for (int q = 0; q < 144; ++q) {
    std::vector<float>& v = by[q];
    fit[2 * q] = v.empty() ? 0.0f : pct(v, 0.99);
    fit[2 * q + 1] = v.empty() ? 0.0f : pct(v, 0.9999);
  }
  return GAPS_OK;
}

int gaps_set_pdf_ratio_fit(gaps_ctx* ctx, const float* fit) {
  if (!ctx) return GAPS_ERR_INVALID_ARG;
  if (!fit) {
    ctx->P.fit_on = 0;
    return GAPS_OK;
  }
  for (int q = 0; q < 288; ++q)
    if (!std::isfinite(fit[q]) || fit[q] < 0.0f) return GAPS_ERR_INVALID_ARG;
  for (int a = 0; a < 12; ++a)
    for (int b = 0; b < 12; ++b)
      for (int k = 0; k < 2; ++k) ctx->P.fit[a][b][k] = fit[(a * 12 + b) * 2 + k];
  ctx->P.fit_on = 1;
  return GAPS_OK;
}

int gaps_set_violation_log(gaps_ctx* ctx, float* log, uint64_t capacity, uint64_t* count) {
  if (!ctx || (log && !count)) return GAPS_ERR_INVALID_ARG;
  ctx->vlog = log;
  ctx->vcap = log ? capacity : 0;
  ctx->vcount = log ? count : nullptr;
  return GAPS_OK;
}

int gaps_observables(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev, double* obs,
                     const gaps_hists* hists, void* stream) {
  if (!ctx || !events_ok(ctx, ev, n)) return GAPS_ERR_INVALID_ARG;
  if (hists && (!hists->sumw || !hists->sumw2)) return GAPS_ERR_INVALID_ARG;
  return cuda_fail(launch_observables(ctx->P, dev_events(ev), first_event, n, obs, ctx->H,
                                      hists ? hists->sumw : nullptr, hists ? hists->sumw2 : nullptr,
                                      ctx->cfg.precision == GAPS_MIXED, ctx->n_sm, (cudaStream_t)stream));
}

namespace {
void free_slot2(gaps_ctx* ctx) {
  if (ctx->d_slot2) cudaFree(ctx->d_slot2);
  if (ctx->d_wave2) cudaFree(ctx->d_wave2);
  ctx->d_slot2 = ctx->d_wave2 = nullptr;
  ctx->slot2_bytes = ctx->wave_bytes2 = 0;
  ctx->wave_cap2 = 0;
  ctx->ev2 = gaps_events{};
  ctx->obs2 = nullptr;
}

// The second slot of gaps_process for records like `ev` (library-owned
// records, observables and a wavefront working set), its stream and the
// fork/join events. Returns false, holding nothing, when the memory is not
// there: the call then runs its chunks one after another.
bool ensure_slot2(gaps_ctx* ctx, const gaps_events* ev) {
  const uint64_t cap = ev->capacity;
  const int nmax = ev->nmax;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t need = al(4 * (size_t)nmax * cap * sizeof(double)) + 3 * al((size_t)nmax * cap * sizeof(int32_t)) +
                      3 * al(cap * sizeof(int32_t)) + 4 * al(cap * sizeof(double)) + al(cap * sizeof(uint64_t)) +
                      al((size_t)GAPS_NOBS * cap * sizeof(double));
  if (!ctx->d_slot2 || ctx->slot2_bytes < need || ctx->ev2.capacity != cap || ctx->ev2.nmax != nmax) {
    free_slot2(ctx);
    if (cudaMalloc(&ctx->d_slot2, need) != cudaSuccess) {
      cudaGetLastError();
      ctx->d_slot2 = nullptr;
      return false;
    }
    ctx->slot2_bytes = need;
    char* q = (char*)ctx->d_slot2;
    auto take = [&](size_t b) { char* r = q; q += al(b); return r; };
    gaps_events& e = ctx->ev2;
    e.capacity = cap;
    e.nmax = nmax;
    e.p = (double*)take(4 * (size_t)nmax * cap * sizeof(double));
    e.flav = (int32_t*)take((size_t)nmax * cap * sizeof(int32_t));
    e.col = (int32_t*)take((size_t)nmax * cap * sizeof(int32_t));
    e.acol = (int32_t*)take((size_t)nmax * cap * sizeof(int32_t));
    e.npart = (int32_t*)take(cap * sizeof(int32_t));
    e.status = (int32_t*)take(cap * sizeof(int32_t));
    e.n_emit = (int32_t*)take(cap * sizeof(int32_t));
    e.weight = (double*)take(cap * sizeof(double));
    e.t = (double*)take(cap * sizeof(double));
    e.eta = (double*)take(2 * cap * sizeof(double));
    e.draw = (uint64_t*)take(cap * sizeof(uint64_t));
    ctx->obs2 = (double*)take((size_t)GAPS_NOBS * cap * sizeof(double));
  }
  WorkSet W;
  WaveSet V;
  if (ensure_wave(ctx, cap, W, V, 1) != GAPS_OK) {
    free_slot2(ctx);
    return false;
  }
  if (!ctx->cap_stream2 && cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->cap_stream2 = nullptr;
    return false;
  }
  if (!ctx->fork_ev && cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess) return false;
  if (!ctx->join_ev && cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming) != cudaSuccess) return false;
  return true;
}
}  // namespace

int gaps_process(gaps_ctx* ctx, uint64_t first_event, uint64_t n, const gaps_events* ev, double* obs_dev,
                 double* obs_host, const gaps_hists* hists, void* stream) {
  if (!ctx || !ev || ev->capacity == 0) return GAPS_ERR_INVALID_ARG;
  if (obs_host && !obs_dev) return GAPS_ERR_INVALID_ARG;
  if (n == 0) return GAPS_OK;
  const uint64_t cap = ev->capacity;
  if (!events_ok(ctx, ev, n < cap ? n : cap)) return GAPS_ERR_INVALID_ARG;
  // everything the launches need is allocated before the capture
  if (ctx->cfg.precision == GAPS_MIXED && ctx->cfg.schedule == GAPS_SCHED_PERSISTENT) {
    int blocks, bs;
    WorkSet W;
    const int rc = ensure_workset(ctx, blocks, bs, W);
    if (rc != GAPS_OK) return rc;
  }
  if (ctx->cfg.precision == GAPS_MIXED && ctx->cfg.schedule == GAPS_SCHED_WAVE) {
    WorkSet W;
    WaveSet V;
    const int rc = ensure_wave(ctx, cap, W, V);
    if (rc != GAPS_OK) return rc;
  }
  if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return GAPS_ERR_CUDA;
  const uint64_t chunks = (n + cap - 1) / cap;
  if (chunks > 1u << 20) return GAPS_ERR_INVALID_ARG;
  while (ctx->shower_ev.size() < 2 * chunks) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return GAPS_ERR_CUDA;
    ctx->shower_ev.push_back(e);
  }
  // with the wavefront schedule, odd chunks run in a second slot on a second
  // stream (events are independent; counters and histograms are atomics)
  const bool two = chunks >= 2 && ctx->cfg.precision == GAPS_MIXED && ctx->cfg.schedule == GAPS_SCHED_WAVE &&
                   ensure_slot2(ctx, ev);
  cudaStream_t cs = ctx->cap_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GAPS_ERR_CUDA;
  int rc = GAPS_OK;
  if (two && (cudaEventRecord(ctx->fork_ev, cs) != cudaSuccess ||
              cudaStreamWaitEvent(ctx->cap_stream2, ctx->fork_ev, 0) != cudaSuccess))
    rc = GAPS_ERR_CUDA;
  for (uint64_t f0 = 0, k = 0; f0 < n && rc == GAPS_OK; f0 += cap, ++k) {
    const uint64_t m = n - f0 < cap ? n - f0 : cap;
    const int slot = two ? (int)(k & 1) : 0;
    cudaStream_t s = slot ? ctx->cap_stream2 : cs;
    const gaps_events* e = slot ? &ctx->ev2 : ev;
    double* od = slot && obs_dev ? ctx->obs2 : obs_dev;
    rc = gaps_generate_hard(ctx, first_event + f0, m, e, s);
    if (rc == GAPS_OK && cudaEventRecordWithFlags(ctx->shower_ev[2 * k], s, cudaEventRecordExternal) != cudaSuccess)
      rc = GAPS_ERR_CUDA;
    if (rc == GAPS_OK) rc = shower_impl(ctx, first_event + f0, m, e, s, slot);
    if (rc == GAPS_OK &&
        cudaEventRecordWithFlags(ctx->shower_ev[2 * k + 1], s, cudaEventRecordExternal) != cudaSuccess)
      rc = GAPS_ERR_CUDA;
    if (rc == GAPS_OK) rc = gaps_observables(ctx, first_event + f0, m, e, od, hists, s);
    if (rc == GAPS_OK && obs_host &&
        cudaMemcpy2DAsync(obs_host + f0, n * sizeof(double), od, cap * sizeof(double), m * sizeof(double),
                          GAPS_NOBS, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = GAPS_ERR_CUDA;
  }
  if (two && rc == GAPS_OK &&
      (cudaEventRecord(ctx->join_ev, ctx->cap_stream2) != cudaSuccess ||
       cudaStreamWaitEvent(cs, ctx->join_ev, 0) != cudaSuccess))
    rc = GAPS_ERR_CUDA;
  cudaGraph_t g = nullptr;
  const cudaError_t end = cudaStreamEndCapture(cs, &g);
  if (rc == GAPS_OK && (end != cudaSuccess || !g)) rc = GAPS_ERR_CUDA;
  if (rc != GAPS_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  // same chunking as the last call: update the parameters in place
  bool updated = false;
  if (ctx->graph && ctx->graph_n == n && ctx->graph_cap == cap) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(ctx->graph, g, &info) == cudaSuccess;
    if (!updated) cudaGetLastError();
  }
  if (!updated) {
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    if (cudaGraphInstantiate(&ctx->graph, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      ctx->graph = nullptr;
      return GAPS_ERR_CUDA;
    }
    ctx->graph_n = n;
    ctx->graph_cap = cap;
  }
  cudaGraphDestroy(g);
  ctx->graph_chunks = (int)chunks;
  return cuda_fail(cudaGraphLaunch(ctx->graph, (cudaStream_t)stream));
}

int gaps_process_shower_ms(gaps_ctx* ctx, float* ms, int max_chunks) {
  if (!ctx || !ms || max_chunks < 0) return GAPS_ERR_INVALID_ARG;
  const int k = ctx->graph_chunks < max_chunks ? ctx->graph_chunks : max_chunks;
  for (int c = 0; c < k; ++c) {
    if (cudaEventSynchronize(ctx->shower_ev[2 * c + 1]) != cudaSuccess) return GAPS_ERR_CUDA;
    if (cudaEventElapsedTime(&ms[c], ctx->shower_ev[2 * c], ctx->shower_ev[2 * c + 1]) != cudaSuccess)
      return GAPS_ERR_CUDA;
  }
  return k;
}

int gaps_hist_binning(const gaps_ctx* ctx, int h, double* lo, double* hi, int* nbins, int* obs_index,
                      int* log10_axis) {
  if (!ctx || h < 0 || h >= GAPS_NHIST * ctx->P.n_rows) return GAPS_ERR_INVALID_ARG;
  const HistDef& H = ctx->H.h[h / GAPS_NHIST];
  h %= GAPS_NHIST;
  if (lo) *lo = H.lo[h];
  if (hi) *hi = H.hi[h];
  if (nbins) *nbins = H.nb[h];
  if (obs_index) *obs_index = H.obs[h];
  if (log10_axis) *log10_axis = H.logx[h];
  return GAPS_OK;
}

int gaps_get_stats(gaps_ctx* ctx, gaps_stats* out, void* stream) {
  if (!ctx || !out) return GAPS_ERR_INVALID_ARG;
  unsigned long long h[C_NCOUNTERS];
  cudaError_t e = cudaMemcpyAsync(h, ctx->d_counters, sizeof h, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return GAPS_ERR_CUDA;
  out->events = h[C_EVENTS]; out->steps = h[C_STEPS]; out->trials = h[C_TRIALS];
  out->isr_trials = h[C_ISR_TRIALS]; out->vetoes = h[C_VETOES]; out->accepts = h[C_ACCEPTS];
  out->violations = h[C_VIOLATIONS]; out->err_capacity = h[C_ERR_CAP];
  out->err_iter_cap = h[C_ERR_ITER]; out->err_numeric = h[C_ERR_NUM];
  out->lane_steps = h[C_LANE_STEPS]; out->warp_steps = h[C_WARP_STEPS];
  out->rebuilds = h[C_REBUILDS]; out->mlp_tiles = h[C_MLP_TILES];
  return GAPS_OK;
}

int gaps_reset_stats(gaps_ctx* ctx, void* stream) {
  if (!ctx) return GAPS_ERR_INVALID_ARG;
  return cuda_fail(cudaMemsetAsync(ctx->d_counters, 0, C_NCOUNTERS * sizeof(unsigned long long),
                                   (cudaStream_t)stream));
}

void gaps_destroy(gaps_ctx* ctx) {
  if (!ctx) return;
  if (ctx->d_grid) cudaFree(ctx->d_grid);
  if (ctx->d_tables) cudaFree(ctx->d_tables);
  if (ctx->d_counters) cudaFree(ctx->d_counters);
  if (ctx->d_work) cudaFree(ctx->d_work);
  if (ctx->d_wave) cudaFree(ctx->d_wave);
  if (ctx->d_mlp) cudaFree(ctx->d_mlp);
  if (ctx->d_mlp_image) cudaFree(ctx->d_mlp_image);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  free_slot2(ctx);
  if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  for (cudaEvent_t e : ctx->shower_ev) cudaEventDestroy(e);
  delete ctx;
}

}  // extern "C"
