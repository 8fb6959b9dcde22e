// Shared device definitions of the GB300 shower library: parameters, event
// record view, Philox-4x32-10, PDF interpolation and its certified ratio
// bound, running coupling and the dipole-shower helpers of Appendix B.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gaps.h"

namespace gaps {

constexpr double kPi = 3.14159265358979323846;
constexpr double kCF = 4.0 / 3.0, kCA = 3.0, kTR = 0.5, kNc = 3.0;
constexpr double kMZ = 91.1876, kGZ = 2.4952;
constexpr double kSin2W = 0.2312, kGF = 1.16638e-5, kAlphaEM = 1.0 / 128.9;
constexpr double kGeV2pb = 0.3893794e9;
constexpr int kNX = GAPS_PDF_NX, kNQ = GAPS_PDF_NQ;
constexpr double kXMin = GAPS_PDF_XMIN, kXMax = GAPS_PDF_XMAX;
constexpr double kQ2Min = GAPS_PDF_Q2MIN, kQ2Max = GAPS_PDF_Q2MAX;
constexpr uint64_t kHardDrawBase = 0x8000000000000000ull;
constexpr int kMaxSteps = 200000;  // default of gaps_config.max_cycles

// counters in the device stats block (uint64 each)
enum Counter {
  C_EVENTS = 0, C_STEPS, C_TRIALS, C_ISR_TRIALS, C_VETOES, C_ACCEPTS, C_VIOLATIONS,
  C_ERR_CAP, C_ERR_ITER, C_ERR_NUM, C_LANE_STEPS, C_WARP_STEPS, C_REBUILDS, C_MLP_TILES, C_NCOUNTERS
};

// the process-dependent part of the parameters (one row of a mixed batch)
struct RowParams {
  int process;
  double sqrt_s, s_had, t_cut, as_over;
};
constexpr int kMaxRows = GAPS_MAX_MIX;
constexpr uint64_t kMixDraw = 0x4000000000000000ull;

struct DevParams {
  int process, nf, nmax;
  double sqrt_s, s_had, t_cut, as_mz, as_over, beta0, p_s;
  int trial_mode;              // GAPS_TRIALS_* (KEEP and SELECT: mixed lane kernel only)
  int max_steps;               // veto cycles per event before GAPS_ERR_ITER_CAP
  double ll_rlo, ll_rhi;       // GAPS_PP_LL: the mass window's images under the Breit-Wigner map
  int n_rows;                  // 1: one process; > 1: mixed batch
  RowParams rows[kMaxRows];    // row 0 = the fields above for one process
  double cum[kMaxRows];        // cumulative fractions, summed in row order
  uint64_t seed;
  const float* grid;      // [11][100][50] x f
  const double* umax;     // [12][100] max over Q^2 nodes (index 11 = sum of quarks)
  const double* sufmax;   // [12][101] suffix max over x nodes of umax
  const double* lmin;     // [12][100] min over Q^2 nodes (above the threshold of a heavy flavour)
  const double* first;    // [12][100] node value on the first Q^2 node above a heavy flavour's threshold
  int thr[12];            // Q^2 node of a heavy flavour's mass (c, b, cbar, bbar), -1: no threshold
  double m2[12];          // that mass squared (the node's Q^2), 0 without a threshold
  // the paper's percentile-fitted PDF-ratio overestimate (App. A.2, eqs.
  // pdfmax and pdfmax_ud) in place of the certified bound (mixed precision):
  // fit[num][den] = {99th, 99.99th percentile}; a transition without samples
  // (99.99th percentile 0) keeps the certified bound
  int fit_on;
  float fit[12][12][2];
  double lxmin, dlx, lqmin, dlq;
  unsigned long long* counters;  // [C_NCOUNTERS]
};

// per-lane working set of the mixed-precision persistent shower
struct WorkSet {
  double* p;
  uint32_t* tag;
  float4* end;
  float4* trial;         // kept trials {ln t, R_z} of both channels per end [lanes][2 nmax]
  float4* aux;           // the veto's inputs per end {s, eta, emitter tag, partner tag} [lanes][2 nmax]
  float* tmx;            // per end the larger of its two kept trials' ln t (NaN: draws next cycle),
                         // [lanes][tmx_stride(nmax)]: the scan of a veto cycle reads only these
  float4* lkey;          // learned proposal: network inputs of the last evaluation [lanes][4 ends]
  unsigned char* lcode;  // learned proposal: 8-bit bin-height codes [lanes][4 ends][2][8]
  int lanes;
};

// floats per lane of WorkSet::tmx: 2 nmax rounded up to a multiple of four, so
// that four consecutive ends load as one aligned float4
__host__ __device__ constexpr unsigned tmx_stride(int nmax) { return (unsigned)(2 * nmax + 3) & ~3u; }

// bytes of a working set of `lanes` lanes (workset_carve's layout)
constexpr size_t workset_bytes(int lanes, int nmax) {
  return (size_t)lanes * nmax * (4 * sizeof(double) + sizeof(uint32_t) + 6 * sizeof(float4)) +
         (size_t)lanes * tmx_stride(nmax) * sizeof(float) + (size_t)lanes * (64 + 4 * sizeof(float4));
}

// State of the wavefront schedule (GAPS_SCHED_WAVE): per event of a chunk,
// structure of arrays in library-owned device memory, beside a working set
// (WorkSet) with one lane per event.
struct WaveSet {
  float* lnT;               // [cap] ln of the current evolution scale
  int* n;                   // [cap] partons in the event
  int* n_emit;              // [cap] accepted emissions
  int* status;              // [cap] GAPS_STATUS_* or an error code
  int* steps;               // [cap] veto cycles so far
  int* flags;               // [cap] bit 0: learned bounds active; bit 1: write the record
                            // back; bit 2: write the status back only; bit 3: an emission
                            // is parked; bits 8..15: mix row
  int* keep;                // [cap] ends that may keep their trials at the next rebuild (-1: none)
  int* chg;                 // [cap] slots the last emission changed, emitter | spectator << 8 |
                            // new << 16, or -1: the next rebuild recomputes every end
  double* eta;              // [2][cap] momentum fractions of slots 0 and 1
  uint64_t* draw;           // [cap] next Philox block of the event's stream
  unsigned char* pend;      // [cap][kWavePendBytes] the parked emission of the pass
  uint32_t* list;           // [4][cap] live events of even / odd passes, (unused), rebuilds
  float4* mlpq;             // [cap][4 ends][3] initial-state ends for the dense network pass
  uint32_t* mlpi;           // [4 cap] the pass's queue of those ends: 4 event + end
  unsigned long long* ctl;  // [8] lengths of the lists, work counter of the veto pass
  uint64_t cap;
};
constexpr int kWavePendBytes = 64;
enum WaveList { WL_LIVE0 = 0, WL_LIVE1 = 1, WL_REBUILD = 3, WL_GRAB = 4, WL_MLP = 5, WL_NCTL = 8 };
// entries of a rebuild warp's network-queue buffer in shared memory (one
// atomic on the queue length per flush)
constexpr int kMlpBuf = 64;
// WaveSet::flags bits
constexpr int kWaveParked = 8;
// events of the live list a veto warp takes with one atomic on the work counter
constexpr int kWaveGrab = 32;
size_t wave_state_bytes(uint64_t cap);
void wave_state_carve(void* base, uint64_t cap, WaveSet& V);

// learned initial-state proposal and sample collection of one launch
struct LearnedCfg {
  int learned;                    // use the learned bin heights
  const float* mlp;               // FP32 parameters, then the margins [44][8][8], device
  const void* image;              // BF16 weight image of the network (global memory, read through L1)
  float4* collect;                // logged initial-state ends {eta, s, type, pdf index}
  unsigned long long* collect_count;
  uint64_t collect_cap;
  uint32_t collect_keep;          // a state is logged when its 32-bit hash is below this
  float4* vlog;                   // violations of the learned bound: 2 float4 per entry
  unsigned long long* vcount;
  uint64_t vcap;
  float4* rlog;                   // logged PDF ratios {numerator index, denominator index, eta, ratio}
  unsigned long long* rcount;
  uint64_t rcap;
  uint32_t rkeep;                 // a ratio is logged when its 32-bit hash is below this
};

// host helpers shared by the entry points (api.cu); none allocates memory
constexpr int kBoundTableDoubles = 12 * GAPS_PDF_NX + 12 * (GAPS_PDF_NX + 1) + 12 * GAPS_PDF_NX + 12 * GAPS_PDF_NX;
// heavy-quark trials of the measure dt/(t - m^2) end at m^2 (1 + kHqFloor)
constexpr double kHqFloor = 1e-3;
void build_bound_tables(const float* grid, double* out, int* thr = nullptr, double* m2 = nullptr);
void set_bound_tables(DevParams& P, const double* dev_tables, const float* host_grid);
int validate_config(const gaps_config& c);
void fill_params(const gaps_config& c, DevParams& P);
int grid_q_independent(const float* grid);

// histogram binning of one process family
struct HistDef {
  double lo[GAPS_NHIST], hi[GAPS_NHIST];
  int nb[GAPS_NHIST], obs[GAPS_NHIST], logx[GAPS_NHIST];
};
struct HistSet {
  HistDef h[GAPS_MAX_MIX];
};

struct DevEvents {
  uint64_t cap;
  int nmax;
  double* p;
  int32_t* flav;
  int32_t* col;
  int32_t* acol;
  int32_t* npart;
  int32_t* status;
  int32_t* n_emit;
  double* weight;
  double* t;
  double* eta;
  uint64_t* draw;

  __device__ __forceinline__ double& P(int mu, int slot, uint64_t e) const {
    return p[((uint64_t)mu * nmax + slot) * cap + e];
  }
  __device__ __forceinline__ int32_t& F(int slot, uint64_t e) const { return flav[(uint64_t)slot * cap + e]; }
  __device__ __forceinline__ int32_t& C(int slot, uint64_t e) const { return col[(uint64_t)slot * cap + e]; }
  __device__ __forceinline__ int32_t& A(int slot, uint64_t e) const { return acol[(uint64_t)slot * cap + e]; }
};

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// (top 53 bits of hi:lo + 0.5) * 2^-53, in (0, 1)
__device__ __forceinline__ double u01(uint32_t lo, uint32_t hi) {
  uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
  return ((double)(w >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

struct Rng {
  uint32_t k0, k1, e0, e1;
  uint64_t draw;
  __device__ __forceinline__ void init(uint64_t seed, uint64_t event, uint64_t d) {
    k0 = (uint32_t)seed; k1 = (uint32_t)(seed >> 32);
    e0 = (uint32_t)event; e1 = (uint32_t)(event >> 32);
    draw = d;
  }
  __device__ __forceinline__ void next2(double& a, double& b) {
    uint32_t w[4];
    philox(e0, e1, (uint32_t)draw, (uint32_t)(draw >> 32), k0, k1, w);
    draw += 1;
    a = u01(w[0], w[1]);
    b = u01(w[2], w[3]);
  }
};

// row of event `id` in a mixed batch: the first row whose cumulative fraction
// exceeds the uniform of block (seed, id, 2^62), the last one otherwise
__device__ __forceinline__ int mix_row(const DevParams& P, uint64_t id) {
  if (P.n_rows <= 1) return 0;
  Rng r;
  r.init(P.seed, id, kMixDraw);
  double u, unused;
  r.next2(u, unused);
  for (int k = 0; k + 1 < P.n_rows; ++k)
    if (u < P.cum[k]) return k;
  return P.n_rows - 1;
}

// copy of the parameters with the process-dependent fields of row r
__device__ __forceinline__ void apply_row(DevParams& Q, int r) {
  const RowParams& R = Q.rows[r];
  Q.process = R.process;
  Q.sqrt_s = R.sqrt_s;
  Q.s_had = R.s_had;
  Q.t_cut = R.t_cut;
  Q.as_over = R.as_over;
}

// ---------------------------------------------------------------------------
// flavours
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pdf_index(int fl) {
  if (fl == 21) return 0;
  if (fl >= 1 && fl <= 5) return fl;
  if (fl <= -1 && fl >= -5) return 5 - fl;
  return -1;
}

__device__ __forceinline__ double dot4(const double a[4], const double b[4]) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

}  // namespace gaps
