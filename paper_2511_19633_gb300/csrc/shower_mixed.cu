// Mixed-precision persistent shower (Section 2 / Fig. 1 and Appendices A-B
// of arXiv:2511.19633; the partitioning of Section 3.1 becomes live-event
// refill). FP32 in the trial loop, the PDF interpolation, the bounds and the
// acceptance weight; FP64 for dipole invariants, emission kinematics and the
// II Lorentz kick. With the trials of Fig. 1 redrawn every cycle
// (GAPS_TRIALS_REDRAW) the random stream is the FP64 kernel's (one Philox
// block per dipole-end channel in canonical order, two after a winner), so
// most events follow the same history; kept trials (the default) and
// generate-select draw fewer blocks. In every mode the histograms agree with
// the FP64 ones within statistics.
//
// Layout: every lane of the persistent grid owns a lane-major working set in
// global memory (each event contiguous, so a lane walks its own cache lines):
//   p      f64 [L][nmax][4]     momenta
//   tag    u32 [L][nmax]        flavour | colour << 8 | anticolour << 16
//   end    f32x4 [L][2 nmax]    the event's colour ends in canonical order
//                               (emitter ascending, colour side first):
//                               {1/c0, 1/c1, ln t_kin, partner slot (-1: none)}
//   trial  f32x4 [L][2 nmax]    kept trials {ln t, R_z} of both channels
//   aux    f32x4 [L][2 nmax]    per end: {s, eta, tag of the emitter, tag of the
//                               partner}, the veto's inputs as of the last rebuild
//   lcode  u8 [L][4][2][8], lkey f32x4 [L][4]: the learned proposal's bin
//          heights of the initial-state ends and the inputs they came from
// `end` caches the inverse overestimate coefficients of the end's channels
// (< 0: channel absent, 0: no phase space) and is rebuilt after every
// accepted emission.
//
// Learned initial-state proposal: for the ends of the two incoming partons
// the overestimate of each channel is made piecewise constant in 8 bins of
// zeta, the coordinate in which z is sampled (the cumulative of Pover over
// the z range at t_c). Bin m carries U_m = min(1, exp(NN + margin)), rounded
// up to a power 2^(-k/16), where the
// network NN (4 -> 64 -> 64 -> 1, BF16 tensor cores) bounds the acceptance
// ratio r = w / (alpha_s ratio) over the bin and every t in [t_c, t_kin].
// The channel's coefficient becomes c * mean(U), the bin is chosen from R_z,
// and the weight is divided by U_m. A weight above one is counted as a
// violation; the event then continues with the plain bounds from the scale
// before that cycle. Lanes whose event has finished take new events in warp-aggregated
// batches, at most every `period` cycles.
#include <mutex>

#include "physics_fp64.cuh"
#include "mlp_infer.cuh"

namespace gaps {

namespace {

constexpr int kSmNX = GAPS_PDF_NX;

struct SmemPdf {
  float xf[12][kSmNX];      // Q^2-independent grids: x f per flavour (11 = sum of quarks)
  float umax[12][kSmNX];
  float sufmax[12][kSmNX + 1];
  float lmin[12][kSmNX];
  // heavy-quark thresholds (App. A.2): node values above the mass and the
  // mass squared (0: no threshold)
  float first[12][kSmNX];
  float m2[12];
  // per row of a mixed batch: ln t_c, alpha_s(t_c) / 2 pi, pp process
  float lnTc[kMaxRows], asOver2pi[kMaxRows];
  int pp[kMaxRows];
};

__device__ __forceinline__ void load_rows(SmemPdf& S, const DevParams& P) {
  if (threadIdx.x < kMaxRows) {
    const RowParams& R = P.rows[threadIdx.x < P.n_rows ? threadIdx.x : 0];
    S.lnTc[threadIdx.x] = (float)gm_log(R.t_cut);
    S.asOver2pi[threadIdx.x] = (float)(R.as_over / (2.0 * kPi));
    S.pp[threadIdx.x] = R.process != GAPS_EE_QQ;
  }
}

struct MixedCtx {
  DevParams P;
  DevEvents E;
  WorkSet W;
  LearnedCfg Lc;
  uint64_t first, n;
  unsigned long long* next;
  int q_independent;   // grid equal for every Q^2 node: use the staged x table
  int period;          // refill at most every `period` cycles
  int emit_batch;      // build parked emissions once this many lanes of a warp wait
  int emit_wait;       // ... or after this many cycles
  float lnTc, asOver2pi, lxminf, dlxf, lqminf, dlqf;
  // wavefront schedule: per-event state, parity of the pass (its live list),
  // veto cycles an event may take in one pass
  WaveSet V;
  int wave_par;
  int wave_budget;
};

__device__ __forceinline__ float u24(uint32_t w) { return ((float)(w >> 8) + 0.5f) * (1.0f / 16777216.0f); }

__device__ __forceinline__ uint32_t pack_tag(int fl, int c, int a) {
  return ((uint32_t)(fl & 0xff)) | ((uint32_t)(c & 0xff) << 8) | ((uint32_t)(a & 0xff) << 16);
}
__device__ __forceinline__ int tag_fl(uint32_t t) { return (int)(int8_t)(t & 0xff); }
__device__ __forceinline__ int tag_col(uint32_t t) { return (int)((t >> 8) & 0xff); }
__device__ __forceinline__ int tag_acol(uint32_t t) { return (int)((t >> 16) & 0xff); }

struct Lane {
  uint64_t ev;      // record index in the caller's arrays
  int n, n_emit, status, steps;
  int row;          // row of a mixed batch
  int slot;         // index of the event's learned bin heights (the lane's global index)
  bool learned_ok;  // learned bounds active for this event
  float lnT;        // ln of the current evolution scale
  double eta0, eta1;
  uint64_t draw;
};

// ---- FP32 PDF -------------------------------------------------------------
__device__ __forceinline__ bool loc_x(const MixedCtx& M, float x, int& ix, float& fx) {
  if (!(x >= (float)kXMin && x <= (float)kXMax)) return false;
  // ln x to full FP32 precision above x = 1/2: in the last cell the density
  // falls linearly in ln x to zero at x_max = 1 - 1e-6, and the fast
  // logarithm's absolute error (about 2^-21) is then comparable with the
  // distance to x_max, which could break the certified ratio bound there
  const float lx = x > 0.5f ? logf(x) : __logf(x);
  float u = (lx - M.lxminf) / M.dlxf;
  ix = (int)floorf(u);
  ix = min(max(ix, 0), kNX - 2);
  fx = u - (float)ix;
  return true;
}

// out of line: one copy for all call sites (instruction-cache footprint)
__device__ __noinline__ float pdf32(const MixedCtx& M, const SmemPdf& S, int f, float x, float q2) {
  if (f < 0 || f > 11) return 0.0f;
  int ix;
  float fx;
  if (!loc_x(M, x, ix, fx)) return 0.0f;
  if (!(q2 >= (float)kQ2Min && q2 <= (float)kQ2Max)) return 0.0f;
  if (M.q_independent) return (1.0f - fx) * S.xf[f][ix] + fx * S.xf[f][ix + 1];
  float u = (__logf(q2) - M.lqminf) / M.dlqf;
  int iq = min(max((int)floorf(u), 0), kNQ - 2);
  float fq = u - (float)iq;
  auto node = [&](int xx, int qq) -> float {
    if (f < 11) return __ldg(&M.P.grid[((size_t)f * kNX + xx) * kNQ + qq]);
    float s = 0.0f;
    for (int k = 1; k <= 10; ++k) s += __ldg(&M.P.grid[((size_t)k * kNX + xx) * kNQ + qq]);
    return s;
  };
  float lo = (1.0f - fx) * node(ix, iq) + fx * node(ix + 1, iq);
  float hi = (1.0f - fx) * node(ix, iq + 1) + fx * node(ix + 1, iq + 1);
  return lo * (1.0f - fq) + hi * fq;
}

__device__ __noinline__ float bound32(const MixedCtx& M, const SmemPdf& S, int num, int den, float eta) {
  if (num < 0 || num > 11 || den < 0 || den > 11) return 0.0f;
  if (M.P.fit_on && den < 11 && M.P.fit[num][den][1] > 0.0f) {
    // the paper's fitted overestimate (App. A.2): max(P99, P99.99 eta), or
    // P99.99 sqrt(eta) for a gluon from the quarks (its u and d parents)
    const float p99 = M.P.fit[num][den][0], p9999 = M.P.fit[num][den][1];
    if (!(eta >= (float)kXMin && eta <= (float)kXMax)) return 0.0f;
    return (num == 11 && den == 0) ? p9999 * sqrtf(eta) : fmaxf(p99, p9999 * eta);
  }
  int ix;
  float fx;
  if (!loc_x(M, eta, ix, fx)) return 0.0f;
  float uin = (1.0f - fx) * S.umax[num][ix] + fx * S.umax[num][ix + 1];
  float un = fmaxf(uin, S.sufmax[num][ix + 1]);
  float ld = (1.0f - fx) * S.lmin[den][ix] + fx * S.lmin[den][ix + 1];
  if (!(ld > 0.0f)) return 0.0f;
  if (S.m2[den] > 0.0f) {
    // heavy denominator with a threshold: bound of the ratio times (t - m^2)/t
    const float fd = (1.0f - fx) * S.first[den][ix] + fx * S.first[den][ix + 1];
    if (!(fd > 0.0f)) return 0.0f;
    return un * fmaxf(M.dlqf / fd, 1.0f / ld) * 1.0001f;
  }
  // relative slack for the rounding of the FP32 interpolation
  return un / ld * 1.0001f;
}

// Mass squared of the heavy-quark measure of end q's channels: an incoming c
// or b whose density has a threshold (both its channels, q <- q and q <- g,
// draw in dt/(t - m^2)); 0 for every other end.
__device__ __forceinline__ float end_m2(const SmemPdf& S, const float4& aux, int q, int row) {
  if (q >= 4 || !S.pp[row]) return 0.0f;
  const int fe = pdf_index(tag_fl(__float_as_uint(aux.z)));
  return fe > 0 ? S.m2[fe] : 0.0f;
}

// ln of a channel's next trial scale below t_max: t_max R^(1/c) in the
// measure dt/t, or m^2 + (t_max - m^2) R^(1/c) in dt/(t - m^2) for a heavy
// quark (m2 > 0), -infinity below the heavy channel's floor m^2 (1 + 1e-3)
__device__ __forceinline__ float trial_lnt(float lnTmax, float ic, float lnR, float m2) {
  if (!(m2 > 0.0f)) return fmaf(lnR, ic, lnTmax);
  const float t = m2 + (__expf(lnTmax) - m2) * __expf(lnR * ic);
  return t > m2 * (1.0f + (float)kHqFloor) ? __logf(t) : -INFINITY;
}

// ---- FP32 kinematic limits and overestimate shapes -------------------------
__device__ __forceinline__ bool zlim32(int type, float t, float s, float eta, float& zm, float& delta) {
  float e;
  if (type == kFF) e = 4.0f * t / s;
  else if (type == kFI) e = 4.0f * t / s * eta / (1.0f - eta);
  else if (type == kIF) e = 4.0f * t * eta / (s * (1.0f - eta));
  else e = 4.0f * t * eta / (s * (1.0f - eta) * (1.0f - eta));
  float D = 1.0f - e;
  if (!(D > 0.0f)) return false;
  float sq = sqrtf(D);
  if (type == kFF || type == kFI) { delta = 0.5f * e / (1.0f + sq); zm = delta; }
  else { delta = 0.5f * (1.0f - eta) * e / (1.0f + sq); zm = eta + delta; }
  return true;
}

__device__ __forceinline__ float tkin32(int type, float s, float eta) {
  if (type == kFF) return 0.25f * s;
  if (type == kFI || type == kIF) return 0.25f * s * (1.0f - eta) / eta;
  return 0.25f * s * (1.0f - eta) * (1.0f - eta) / eta;
}

__device__ __forceinline__ float shape_int32(int sh, float zm, float delta) {
  float zp = 1.0f - delta;
  switch (sh) {
    case kSoft: return __logf((1.0f - zm) / delta);
    case kFlat: return zp - zm;
    case kBoth: return __logf(zp / zm) + __logf((1.0f - zm) / delta);
    default: return __logf(zp / zm);
  }
}

__device__ __forceinline__ void shape_sample32(int sh, float zm, float delta, float R, float& z, float& omz) {
  float zp = 1.0f - delta;
  switch (sh) {
    case kSoft:
      omz = (1.0f - zm) * __expf(R * __logf(delta / (1.0f - zm)));
      z = 1.0f - omz;
      break;
    case kFlat:
      z = zm + R * (zp - zm);
      omz = 1.0f - z;
      break;
    case kBoth: {
      float lm = __logf(zm / (1.0f - zm)), lp = __logf(zp / delta);
      float em = __expf(-(lm + R * (lp - lm)));
      z = 1.0f / (1.0f + em);
      omz = em / (1.0f + em);
      break;
    }
    default:
      z = zm * __expf(R * __logf(zp / zm));
      omz = 1.0f - z;
      break;
  }
}

__device__ __forceinline__ float shape_val32(int sh, float coef, float z, float omz) {
  switch (sh) {
    case kSoft: return coef / omz;
    case kFlat: return coef;
    case kBoth: return coef / (z * omz);
    default: return coef / z;
  }
}

// ---- working-set access ------------------------------------------------------
// Lane-major: each lane's event is contiguous (a slot's four momentum
// components in 32 bytes, the end table in 2 nmax x 16 bytes), so the trial
// loop walks its own cache lines and the cooperative rebuild reads one
// event's lines. Unsigned 32-bit element indices: lanes x 4 nmax < 2^32
// (checked by the launcher).
struct WS {
  const WorkSet& W;
  int lane, nmax;
  __device__ __forceinline__ double& P(int mu, int slot) const {
    return W.p[((unsigned)lane * (unsigned)nmax + (unsigned)slot) * 4u + (unsigned)mu];
  }
  __device__ __forceinline__ uint32_t& T(int slot) const {
    return W.tag[(unsigned)lane * (unsigned)nmax + (unsigned)slot];
  }
  __device__ __forceinline__ float4& End(int q) const {
    return W.end[(unsigned)lane * (unsigned)(2 * nmax) + (unsigned)q];
  }
  // kept trials of end q: {ln t, R_z} of channel 0, then of channel 1; a NaN
  // ln t of channel 0 marks an end whose channels draw in the next cycle
  __device__ __forceinline__ float4& Trial(int q) const {
    return W.trial[(unsigned)lane * (unsigned)(2 * nmax) + (unsigned)q];
  }
  __device__ __forceinline__ float4& Aux(int q) const {
    return W.aux[(unsigned)lane * (unsigned)(2 * nmax) + (unsigned)q];
  }
  // the larger ln t of end q's two kept trials (NaN with the mark above)
  __device__ __forceinline__ float& Tmx(int q) const {
    return W.tmx[(unsigned)lane * tmx_stride(nmax) + (unsigned)q];
  }
  // ends q0 .. q0 + 3 (q0 a multiple of four)
  __device__ __forceinline__ float4 Tmx4(int q0) const {
    return *reinterpret_cast<const float4*>(W.tmx + (unsigned)lane * tmx_stride(nmax) + (unsigned)q0);
  }
  // writes end q's kept trials and their maximum
  __device__ __forceinline__ void SetTrial(int q, const float4& tr) const {
    Trial(q) = tr;
    Tmx(q) = tr.z > tr.x ? tr.z : tr.x;
  }
  // marks end q: its channels draw in the next cycle
  __device__ __forceinline__ void MarkTrial(int q) const {
    Trial(q).x = __uint_as_float(0x7fc00000u);
    Tmx(q) = __uint_as_float(0x7fc00000u);
  }
  static constexpr bool kTrials = true;
};

// one event per warp, in shared memory (the warp-per-event kernel)
struct WSS {
  double* p;        // [4][nmax]
  uint32_t* tag;    // [nmax]
  float4* end;      // [2 nmax]
  float4* aux;      // [2 nmax]
  int nmax;
  __device__ __forceinline__ double& P(int mu, int slot) const { return p[mu * nmax + slot]; }
  __device__ __forceinline__ uint32_t& T(int slot) const { return tag[slot]; }
  __device__ __forceinline__ float4& End(int q) const { return end[q]; }
  __device__ __forceinline__ float4& Aux(int q) const { return aux[q]; }
  static constexpr bool kTrials = false;  // no kept trials in this schedule
};
// 32-bit words of one warp's tag staging in the lane kernels: the event's
// tags, then the colour-partner table (2 x 256 bytes: the slot owning each
// colour tag, then each anticolour tag; 0xff none)
__host__ __device__ constexpr int tag_stage_words(int nmax) { return nmax + 128; }
// bytes of the per-warp tag staging of a block (16-byte multiple)
__host__ __device__ constexpr size_t tag_stage_bytes(int warps, int nmax) {
  return ((size_t)warps * tag_stage_words(nmax) * sizeof(uint32_t) + 15) / 16 * 16;
}

// bytes of one warp's event in shared memory
__host__ __device__ constexpr size_t wss_bytes(int nmax) {
  return (size_t)nmax * (4 * sizeof(double) + sizeof(uint32_t) + 4 * sizeof(float4));
}

// colour partner of end (i, side) among the event's tags (shared memory)
__device__ __forceinline__ int find_partner_tags(const uint32_t* tg, int n, int i, int side, int tag) {
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    const uint32_t t = tg[m];
    if (side == 0 ? (tag_acol(t) == tag) : (tag_col(t) == tag)) return m;
  }
  return -1;
}

// the same from the partner table of unique tags (own: the slot of each
// colour tag, then of each anticolour tag)
__device__ __forceinline__ int partner_from_table(const unsigned char* own, int i, int side, int tag) {
  const int m = own[side == 0 ? 256 + tag : tag];
  return (m == 0xff || m == i) ? -1 : m;
}

template <class W>
__device__ __forceinline__ int find_partner(const W& w, int n, int i, int side, int tag) {
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    uint32_t t = w.T(m);
    if (side == 0 ? (tag_acol(t) == tag) : (tag_col(t) == tag)) return m;
  }
  return -1;
}

// class of an initial-state end and channel for the learned bound: 22 per
// dipole type (IF, II): q<-q and g<-q for each quark table index, g<-g, q<-g
__device__ __forceinline__ int isr_class(int type, int ch, int fl_emitter) {
  const int base = type == kII ? 22 : 0;
  const int fi = pdf_index(fl_emitter);
  if (ch == 3) return base + (fi - 1);
  if (ch == 4) return base + 10 + (fi - 1);
  return base + (ch == 5 ? 20 : 21);
}

// network inputs: ln eta, ln(s / t_c), the bin's centre in zeta, the class
__device__ __forceinline__ void mlp_features(float eta, float s, float tc, int bin, int cls, float* f) {
  f[0] = __logf(eta) * (1.0f / 7.0f) + 1.0f;
  f[1] = __logf(s / tc) * 0.1f - 1.0f;
  f[2] = 2.0f * ((float)bin + 0.5f) * 0.125f - 1.0f;
  f[3] = (float)cls * (1.0f / 21.5f) - 1.0f;
}

// channel_over's overestimate in FP32: the same shapes, and coefficients equal
// to the FP64 ones rounded to float (2 C_F is the exact double of C_F, n_f T_R
// / 2 = n_f / 4 is exact), without FP64 instructions, which run at 1/64 of
// the FP32 rate here
__device__ __forceinline__ void channel_over32(int ch, int type, int nf, int& shape, float& coef) {
  constexpr float cf = (float)kCF, ca = (float)kCA, tr = (float)kTR;
  switch (ch) {
    case 0: shape = kSoft; coef = 2.0f * cf; break;
    case 1: shape = kSoft; coef = ca; break;
    case 2: shape = kFlat; coef = (float)nf * tr * 0.5f; break;
    case 3: shape = kSoft; coef = 2.0f * cf; break;
    case 4: shape = type == kIF ? kSoft : kFlat; coef = tr; break;
    case 5: shape = kBoth; coef = ca; break;
    default: shape = type == kIF ? kBoth : kInv; coef = cf; break;
  }
}

struct IsrEval {
  float r, x, omx, u, omu, v, sumF;
  float fr;       // the PDF ratio F(eta/x)/F(eta) (corrected for a heavy quark)
  int num, den;   // its table indices
  bool ok;
};

// Acceptance ratio r = kernel J x / Pover * PDF ratio / bound of an
// initial-state winner (Appendix B.4/B.5), with (1-z) given directly; the
// cycle's weight is alpha_s(t)/alpha_s(t_c) * r. ok = false outside the map.
__device__ IsrEval isr_eval32(const MixedCtx& M, const SmemPdf& S, int type, int ch, int fl_i, float eta, float s,
                              float tw, float z, float omz, float pover) {
  IsrEval e;
  e.ok = false;
  e.r = 0.0f; e.x = 1.0f; e.omx = 0.0f; e.u = 0.0f; e.omu = 1.0f; e.v = 0.0f; e.sumF = 0.0f;
  e.fr = 0.0f; e.num = 0; e.den = 0;
  const float r = tw / s;
  float J;
  if (type == kIF) {
    const float q = omz + r;
    const float disc = 1.0f - 4.0f * r * z * omz / (q * q);
    if (!(disc >= 0.0f)) return e;
    e.x = 2.0f * z * omz / (q * (1.0f + sqrtf(disc)));
    e.u = e.x * r / omz;
    e.omu = 1.0f - e.u;
    if (!(e.omu > 0.0f)) return e;
    e.omx = omz / e.omu;
    J = 1.0f / (e.x * e.omu + e.u * e.omx);
  } else {
    e.x = z * omz / (omz + r);
    e.omx = (omz * omz + r) / (omz + r);
    e.v = e.x * r / omz;
    if (!(e.omx - e.v > 0.0f)) return e;
    J = 1.0f / z;
  }
  if (!(e.x > eta)) return e;
  const float x = e.x, omx = e.omx;
  const float soft = (type == kIF) ? (omx + e.u) : omx;
  float kk;
  if (ch == 3) kk = (float)kCF * (2.0f / soft - (1.0f + x));
  else if (ch == 4) kk = (float)kTR * (1.0f - 2.0f * x * omx);
  else if (ch == 5) kk = (float)kCA * (1.0f / soft + omx / x - 1.0f + x * omx);
  else kk = (float)kCF * 0.5f * (x + 2.0f * omx / x);
  int num, den;
  isr_pdf_indices(ch, fl_i, num, den);
  const float B = bound32(M, S, num, den, eta);
  const float F0 = pdf32(M, S, den, eta, tw);
  const float F1 = pdf32(M, S, num, eta / x, tw);
  if (ch == 6) e.sumF = F1;
  float Fratio = F0 > 0.0f ? F1 / F0 : 0.0f;
  if (ch == 3 || ch == 4) {
    const float m2 = S.m2[pdf_index(fl_i)];
    if (m2 > 0.0f) Fratio *= (tw - m2) / tw;  // heavy-quark measure correction
  }
  e.r = B > 0.0f ? kk * J * x / pover * Fratio / B : 0.0f;
  e.fr = Fratio;
  e.num = num;
  e.den = den;
  e.ok = true;
  return e;
}

// Cached record of colour end q = 2 slot + side of an event: {1/c0, 1/c1,
// ln t_kin, partner} (partner -1: no dipole on this side), and in aux_out the
// veto's inputs {s, eta, emitter tag, partner tag}.
template <class W>
__device__ float4 end_record(const MixedCtx& M, const SmemPdf& S, const W& w, const uint32_t* tg,
                             const unsigned char* own, int n, float eta0, float eta1, int row, int q,
                             float& s_out, float& eta_out, int& type_out, float4& aux_out) {
  type_out = -1;
  aux_out = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const bool pp = S.pp[row] != 0;
  const int i = q >> 1, side = q & 1;
  const uint32_t ti = tg[i];
  const int tag = side == 0 ? tag_col(ti) : tag_acol(ti);
  const int k = !tag ? -1 : (own ? partner_from_table(own, i, side, tag) : find_partner_tags(tg, n, i, side, tag));
  if (k < 0) return make_float4(-1.0f, -1.0f, 0.0f, __int_as_float(-1));
  const int fi = tag_fl(ti);
  const bool ini = pp && i < 2, ink = pp && k < 2;
  const int type = ini ? (ink ? kII : kIF) : (ink ? kFI : kFF);
  double pi[4], pk[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) { pi[mu] = w.P(mu, i); pk[mu] = w.P(mu, k); }
  const float s = (float)(2.0 * dot4(pi, pk));  // FP64: near-collinear invariant
  float eta = 0.0f;
  if (type == kFI) eta = k == 0 ? eta0 : eta1;
  if (type == kIF || type == kII) eta = i == 0 ? eta0 : eta1;
  s_out = s;
  eta_out = eta;
  type_out = type;
  aux_out = make_float4(s, eta, __uint_as_float(ti), __uint_as_float(tg[k]));
  const int first = ini ? (fi == 21 ? 5 : 3) : (fi == 21 ? 1 : 0);
  const int nch = (!ini && fi != 21) ? 1 : 2;
  const float tc = __expf(S.lnTc[row]);
  const float tk = tkin32(type, s, eta);
  float zm, delta;
  const bool ok = tk > tc && zlim32(type, tc, s, eta, zm, delta);
  float ic[2] = {0.0f, -1.0f};
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (c >= nch) continue;
    ic[c] = 0.0f;
    if (!ok) continue;
    const int ch = first + c;
    int shape;
    float coefd;
    channel_over32(ch, type, M.P.nf, shape, coefd);
    float B = 1.0f;
    if (type == kFI) {
      const int f = pdf_index(tag_fl(tg[k]));
      B = bound32(M, S, f, f, eta);
    } else if (type == kIF || type == kII) {
      int num, den;
      isr_pdf_indices(ch, fi, num, den);
      B = bound32(M, S, num, den, eta);
    }
    const float cc = S.asOver2pi[row] * B * (float)coefd * shape_int32(shape, zm, delta);
    ic[c] = cc > 0.0f ? 1.0f / cc : 0.0f;
  }
  return make_float4(ic[0], ic[1], __logf(tk), __int_as_float(k));
}

// Learned bin heights of an event slot, 8-bit codes: height = 2^(-k/16)
// (k < 255), rounded up from the network's value so that it stays a bound.
// Slot-major, [slot][4 ends][2 channels][8 bins] bytes and [slot][4 ends]
// keys: in the lane kernel the slots are the global lanes (working set in
// global memory, read through L1), in the warp kernel the block's warps
// (shared memory).
struct LearnedSmem {
  unsigned char* code;   // NULL without the learned proposal
  const float* dec;      // [256] decoded heights (shared memory)
  float4* key;           // {eta, s, class code, -} of the last evaluation per end
  __device__ __forceinline__ unsigned char* at(int q, int c, int slot) const {
    return code + (size_t)slot * 64 + (q * 2 + c) * 8;
  }
  __device__ __forceinline__ float4& keyat(int q, int slot) const { return key[(size_t)slot * 4 + q]; }
};

__device__ __forceinline__ int height_code(float U) {
  // smallest k with 2^(-k/16) >= U, i.e. floor(-16 log2 U), clamped to [0, 254]
  if (!(U < 1.0f)) return 0;
  const float k = floorf(-16.0f * __log2f(U));
  return k < 0.0f ? 0 : (k > 254.0f ? 254 : (int)k);
}

// Writes end q's record. With kept trials (keep_ends >= 0) an end among the
// first keep_ends whose record (rates, maximum scale, partner) is unchanged
// keeps its trials: each channel's trials are a Poisson process in ln t with
// that rate, and the kept trial lies below the scale the event continues from.
// Every other end draws in the next cycle.
template <class W>
__device__ __forceinline__ void set_end(const W& w, int q, const float4& rec, int keep_ends) {
  if constexpr (W::kTrials) {
    if (keep_ends < 0) {
      // trials are not kept
    } else if (q < keep_ends) {
      const float4 old = w.End(q);
      if (__float_as_uint(old.x) == __float_as_uint(rec.x) && __float_as_uint(old.y) == __float_as_uint(rec.y) &&
          __float_as_uint(old.z) == __float_as_uint(rec.z) && __float_as_uint(old.w) == __float_as_uint(rec.w))
        return;
      w.MarkTrial(q);
    } else {
      w.MarkTrial(q);
    }
  }
  w.End(q) = rec;
}

// The warp evaluates the learned bound of up to four initial-state ends. Lane
// j (0..3) describes end j: eta, s, dipole type, emitter flavour, t_c of its
// row, and where its heights go (slot_j, end q_j); bit j of `eval` selects the
// ends to evaluate. Rows r = lane and lane + 32 of the staging hold end r / 16,
// channel (r / 8) % 2, bin r % 8: one 16-row tensor-core tile per end. Writes
// the ends' 8-bit height codes and keys and returns on lane j the coefficient
// scales of end j's two channels, 8 / the sum of its heights.
__device__ __noinline__ void learned_heights(const MixedCtx& M, const MlpSmem& mlp, const LearnedSmem& ls,
                                             float (*stage)[4], float* ustage, unsigned eval, float tc,
                                             float isr_eta, float isr_s, int isr_type, int fl_i, int slot_j, int q_j,
                                             int lane_id, float& scale0, float& scale1, bool four = false) {
  int cls_j[2];  // margin row: (class, eta bucket)
  // the end's two continuous inputs, once per end (lane j < 4), as
  // mlp_features forms them
  float fe[4];
  {
    const float eta_c = lane_id < 4 ? isr_eta : 1.0f, s_c = lane_id < 4 ? isr_s : 1.0f, tc_c = lane_id < 4 ? tc : 1.0f;
    mlp_features(eta_c, s_c, tc_c, 0, 0, fe);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int r = lane_id + 32 * j, e = r >> 4, c = (r >> 3) & 1, m = r & 7;
    const float f0 = __shfl_sync(0xffffffffu, fe[0], e);
    const float f1 = __shfl_sync(0xffffffffu, fe[1], e);
    const int type_e = __shfl_sync(0xffffffffu, isr_type, e);
    const int fl_e = __shfl_sync(0xffffffffu, fl_i, e);
    cls_j[j] = 0;
    if ((eval >> e) & 1u) {
      const int cls = isr_class(type_e, (fl_e == 21 ? 5 : 3) + c, fl_e);
      float f[4];
      mlp_features(1.0f, 1.0f, 1.0f, m, cls, f);  // the bin and class inputs
      *reinterpret_cast<float4*>(stage[r]) = make_float4(f0, f1, f[2], f[3]);
      cls_j[j] = cls * kEtaBins + eta_bucket(f0);
    }
  }
  // calibration margins of (class, eta bucket, bin), after the parameters,
  // loaded before the tiles
  float mg[2] = {0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int r = lane_id + 32 * j;
    if ((eval >> (r >> 4)) & 1u) mg[j] = __ldg(&M.Lc.mlp[kMlpParams + cls_j[j] * kIsrBins + (r & 7)]);
  }
  __syncwarp();
  if (four) {
    // all four tiles, two at a time (rows of unselected ends are unused)
    mlp_tiles<2>(mlp, stage, ustage);
    mlp_tiles<2>(mlp, stage + 32, ustage + 32);
  } else {
    for (int tile = 0; tile < 4; ++tile)
      if ((eval >> tile) & 1u) mlp_tile(mlp, stage + 16 * tile, ustage + 16 * tile);
  }
  __syncwarp();
  float tot[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int r = lane_id + 32 * j, e = r >> 4, c = (r >> 3) & 1, m = r & 7;
    const int slot_e = __shfl_sync(0xffffffffu, slot_j, e);
    const int q_e = __shfl_sync(0xffffffffu, q_j, e);
    float U = 0.0f;
    int hc = 0;
    if ((eval >> e) & 1u) {
      hc = height_code(__expf(ustage[r] + mg[j]));
      U = ls.dec[hc];
    }
    // the channel's eight codes, gathered by its first lane into one 8-byte store
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const uint32_t v = (uint32_t)__shfl_sync(0xffffffffu, hc, (lane_id & ~7) + b) & 0xffu;
      if (b < 4) lo |= v << (8 * b);
      else hi |= v << (8 * (b - 4));
    }
    if (m == 0 && ((eval >> e) & 1u)) *reinterpret_cast<uint2*>(ls.at(q_e, c, slot_e)) = make_uint2(lo, hi);
    // the channel's sum over its 8 bins, in bin order (the order the veto sums them)
    float t = 0.0f;
#pragma unroll
    for (int b = 0; b < 8; ++b) t += __shfl_sync(0xffffffffu, U, (lane_id & ~7) + b);
    tot[j] = t;
  }
  // end e = lane (0..3): rows 16 e + 8 c + m, held by lanes 16 (e % 2) + 8 c + m in row set e / 2
  const int base = (lane_id & 1) * 16;
  const float t00 = __shfl_sync(0xffffffffu, tot[0], base), t01 = __shfl_sync(0xffffffffu, tot[1], base);
  const float t10 = __shfl_sync(0xffffffffu, tot[0], base + 8), t11 = __shfl_sync(0xffffffffu, tot[1], base + 8);
  const float tc0 = (lane_id & 2) ? t01 : t00, tc1 = (lane_id & 2) ? t11 : t10;
  scale0 = tc0 > 0.0f ? 8.0f / tc0 : 0.0f;
  scale1 = tc1 > 0.0f ? 8.0f / tc1 : 0.0f;
  if (lane_id < 4 && ((eval >> lane_id) & 1u))
    ls.keyat(q_j, slot_j) = make_float4(isr_eta, isr_s, (float)(isr_type * 32 + pdf_index(fl_i)), 0.0f);
}

// The whole warp rebuilds the colour-end table of the event held by lane
// `src` (one end per lane), after an emission or a refill of that lane. With
// the learned proposal the warp then evaluates the network for those of the
// (up to four) initial-state ends whose inputs changed since their last
// evaluation: 2 channels x 8 bins = one 16-row tile per end, two rows per
// lane for the inputs and the bin heights. The body is inlined into the
// wavefront's rebuild kernel (a call there costs parameter and register
// traffic through local memory) and called out of line elsewhere
// (rebuild_coop: one copy in each of the larger kernels' code).
template <class W>
__device__ __forceinline__ int rebuild_body(const MixedCtx& M, const SmemPdf& S, const MlpSmem& mlp,
                                            const LearnedSmem& ls, float (*stage)[4], float* ustage,
                                            const W& w, uint32_t* tg, bool stage_tags, int slot, uint64_t ev_src,
                                            int n, double eta0, double eta1, int row, bool learned_src,
                                            int keep_ends, int lane_id, bool defer = false,
                                            unsigned* defer_mask = nullptr, float4* deferred = nullptr,
                                            float4* isr_plain = nullptr, int chg = -1) {
  // the event's tags in shared memory, and (lane kernels) the table of the
  // slot owning each colour and anticolour tag, so that an end finds its
  // partner in one lookup; with a tag held by two partons (not a leading-
  // colour event) every end scans the tags instead, as the table cannot give
  // the first match
  const float eta0f = (float)eta0, eta1f = (float)eta1;  // the veto's FP32 momentum fractions
  unsigned char* own = nullptr;
  if (stage_tags) {
    own = reinterpret_cast<unsigned char*>(tg + M.P.nmax);
    uint32_t* ow = reinterpret_cast<uint32_t*>(own);
    for (int k = lane_id; k < 128; k += 32) ow[k] = 0xffffffffu;
    for (int m = lane_id; m < n; m += 32) tg[m] = w.T(m);
    __syncwarp();
    for (int m = lane_id; m < n; m += 32) {
      const uint32_t t = tg[m];
      if (tag_col(t)) own[tag_col(t)] = (unsigned char)m;
      if (tag_acol(t)) own[256 + tag_acol(t)] = (unsigned char)m;
    }
    __syncwarp();
    bool dup = false;
    for (int m = lane_id; m < n; m += 32) {
      const uint32_t t = tg[m];
      dup = dup || (tag_col(t) && own[tag_col(t)] != m) || (tag_acol(t) && own[256 + tag_acol(t)] != m);
    }
    if (__any_sync(0xffffffffu, dup)) own = nullptr;
  }
  const bool pp = S.pp[row] != 0;
  // the learned state of the initial-state ends, loaded before the records
  // are built: the inputs of the last evaluation and the record it gave
  float4 key = make_float4(-1.0f, -1.0f, -1.0f, 0.0f), old_isr = key;
  if (pp && lane_id < 4 && lane_id < 2 * n && M.Lc.learned && learned_src) {
    key = ls.keyat(lane_id, slot);
    old_isr = w.End(lane_id);
  }
  float4 isr_rec = make_float4(-1.0f, -1.0f, 0.0f, __int_as_float(-1));
  float isr_s = 0.0f, isr_eta = 0.0f;
  int isr_type = -1;
  for (int q = lane_id; q < 2 * n; q += 32) {
    if (chg >= 0 && !(pp && q < 4) && q < keep_ends) {
      // an end whose parton and colour partner the last emission left alone
      // keeps its record (the same bits a recomputation gives): its inputs
      // are the two momenta, the tags and the momentum fraction of an
      // initial-state parton among them, and the emission changed only the
      // emitter, the spectator and the new parton, whose ends and partners'
      // ends take the new colour line
      const int ci = chg & 0xff, ck = (chg >> 8) & 0xff, cj = (chg >> 16) & 0xff;
      const int a = q >> 1;
      if (a != ci && a != ck && a != cj) {
        const int side = q & 1;
        const uint32_t ta = tg[a];
        const int tag = side == 0 ? tag_col(ta) : tag_acol(ta);
        const int p = !tag ? -1 : (own ? partner_from_table(own, a, side, tag) : find_partner_tags(tg, n, a, side, tag));
        if (p != ci && p != ck && p != cj) continue;
      }
    }
    float s_, eta_;
    int type_;
    float4 aux;
    const float4 rec = end_record(M, S, w, tg, own, n, eta0f, eta1f, row, q, s_, eta_, type_, aux);
    w.Aux(q) = aux;
    if (pp && q < 4) { isr_rec = rec; isr_s = s_; isr_eta = eta_; isr_type = type_; }
    else set_end(w, q, rec, keep_ends);
  }
  if (!pp) return 0;
  // lanes 0..3 hold the ends of the incoming partons
  const bool mine = lane_id < 4 && lane_id < 2 * n;
  const bool valid = mine && isr_type >= 0 && isr_rec.x > 0.0f && isr_rec.y > 0.0f &&
                     (isr_type == kIF || isr_type == kII);
  const int fl_i = mine ? tag_fl(tg[lane_id >> 1]) : 0;
  // training-state sampling: a hash of (event, partons, end) decides, so
  // that a bounded log covers the whole run uniformly
  bool keep = false;
  if (valid && M.Lc.collect) {
    uint64_t h = (M.first + ev_src) * 0x9E3779B97F4A7C15ull ^ ((uint64_t)n << 8 | (uint64_t)lane_id);
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    keep = (uint32_t)(h >> 32) < M.Lc.collect_keep || M.Lc.collect_keep == 0xFFFFFFFFu;
  }
  if (keep) {
    const unsigned long long at = atomicAdd(M.Lc.collect_count, 1ull);
    if (at < M.Lc.collect_cap)
      M.Lc.collect[at] = make_float4(isr_eta, isr_s, (float)isr_type, (float)pdf_index(fl_i));
  }
  const bool use = valid && M.Lc.learned && learned_src;
  // inputs of the end; the heights are reused while they are unchanged
  const float code = (float)(isr_type * 32 + pdf_index(fl_i));
  const bool need = use && !(key.x == isr_eta && key.y == isr_s && key.z == code);
  const unsigned eval = __ballot_sync(0xffffffffu, need) & 0xFu;
  float scale0 = 0.0f, scale1 = 0.0f;  // 8 / sum of the new heights (lanes 0..3)
  if (defer) *defer_mask = eval;
  if (eval && defer) {
    // the wavefront's dense network pass evaluates these ends; their records
    // and trials are finished there
    if (need) *deferred = make_float4(isr_eta, isr_s, __int_as_float(isr_type), __int_as_float(fl_i));
  } else if (eval) {
    learned_heights(M, mlp, ls, stage, ustage, eval, __expf(S.lnTc[row]), isr_eta, isr_s, isr_type, fl_i, slot,
                    lane_id, lane_id, scale0, scale1);
  }
  if (mine) {
    if (use) {
      // the coefficient scale c * mean(U): new heights, or the unchanged
      // inputs' record of the last evaluation (the same product)
      if (need && defer) {
        *isr_plain = isr_rec;  // scaled by the dense pass
      } else if (need) {
        isr_rec.x *= scale0;
        isr_rec.y *= scale1;
      } else {
        isr_rec.x = old_isr.x;
        isr_rec.y = old_isr.y;
      }
    } else if (ls.code) {
      // every other initial-state end proposes with height 1 in all bins (the
      // plain bound): a winner from it reads these codes, and its rate was not
      // rescaled
      for (int c = 0; c < 2; ++c) *reinterpret_cast<uint2*>(ls.at(lane_id, c, slot)) = make_uint2(0u, 0u);
      ls.keyat(lane_id, slot) = make_float4(-1.0f, -1.0f, -1.0f, 0.0f);
    }
    // an end whose network inputs changed draws anew (with kept trials)
    set_end(w, lane_id, isr_rec, (need && keep_ends >= 0) ? 0 : keep_ends);
  }
  __syncwarp();
  return defer ? 0 : __popc(eval);
}

template <class W>
__device__ __noinline__ int rebuild_coop(const MixedCtx& M, const SmemPdf& S, const MlpSmem& mlp,
                                         const LearnedSmem& ls, float (*stage)[4], float* ustage,
                                         const W& w, uint32_t* tg, bool stage_tags, int slot, uint64_t ev_src,
                                         int n, double eta0, double eta1, int row, bool learned_src,
                                         int keep_ends, int lane_id) {
  return rebuild_body(M, S, mlp, ls, stage, ustage, w, tg, stage_tags, slot, ev_src, n, eta0, eta1, row,
                      learned_src, keep_ends, lane_id);
}

struct Emission {
  int kind;  // 0: build the emission, 1: only rebuild the end table (learned-bound fallback)
  int bi, k, bside, ch, type, new_fl_i, fl_j;
  float z, omz, tw;
  double Rphi;
  uint32_t ti;
};

// FP64 reciprocal and reciprocal square root for the mixed kernel's
// kinematics: an FP32 estimate refined by two Newton-Raphson steps
// (relative error (2^-23)^4 before rounding, i.e. an ulp of FP64), a few
// instructions each instead of the library's division sequences. For normal
// arguments within the FP32 range, which every invariant here is.
__device__ __forceinline__ double rcp64(double x) {
  double r = (double)__frcp_rn((float)x);
  r = r * fma(-x, r, 2.0);
  r = r * fma(-x, r, 2.0);
  return r;
}
__device__ __forceinline__ double rsqrt64(double x) {
  double r = (double)rsqrtf((float)x);
  r = r * fma(-0.5 * x * r, r, 1.5);
  r = r * fma(-0.5 * x * r, r, 1.5);
  return r;
}

// Transverse basis of a dipole (as in physics_fp64.cuh) with one reciprocal
// per divisor: the mixed-precision kernel needs FP64 accuracy here, not the
// FP64 kernel's operation-for-operation agreement with the reference, and
// every FP64 division is a long instruction sequence.
__device__ __noinline__ void transverse_basis_mixed(const double P[4], const double K[4], double e1[4],
                                                    double e2[4]) {
  const double iPK = rcp64(dot4(P, K));
  const double N1 = 1.0 + 2.0 * P[1] * K[1] * iPK;
  const double N2 = 1.0 + 2.0 * P[2] * K[2] * iPK;
  const double N3 = 1.0 + 2.0 * P[3] * K[3] * iPK;
  int a = 1;
  double Na = N1;
  if (N2 > Na) { a = 2; Na = N2; }
  if (N3 > Na) { a = 3; Na = N3; }
  int b;
  if (a == 1) b = (N3 > N2) ? 3 : 2;
  else if (a == 2) b = (N3 > N1) ? 3 : 1;
  else b = (N2 > N1) ? 2 : 1;
  const double ina = rsqrt64(Na);
  const double ka = K[a] * iPK, pa = P[a] * iPK, kb = K[b] * iPK, pb = P[b] * iPK;
  double e2p[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) e1[mu] = ((mu == a ? 1.0 : 0.0) + ka * P[mu] + pa * K[mu]) * ina;
  const double e1b = e1[b];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) e2p[mu] = (mu == b ? 1.0 : 0.0) + kb * P[mu] + pb * K[mu] - e1b * e1[mu];
  const double in2 = rsqrt64(-dot4(e2p, e2p));
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) e2[mu] = e2p[mu] * in2;
}

// Appendix B.4 and B.5 maps as in physics_fp64.cuh, with one reciprocal per
// divisor (FP64 accuracy without the FP64 kernel's operation order)
__device__ __forceinline__ bool if_map_mixed(double r, double z, double omz, double& x, double& omx, double& u,
                                             double& omu) {
  const double iq = rcp64(omz + r);
  const double disc = 1.0 - 4.0 * r * z * omz * iq * iq;
  if (!(disc >= 0.0)) return false;
  const double sq = disc > 0.0 ? disc * rsqrt64(disc) : 0.0;
  x = 2.0 * z * omz * iq * rcp64(1.0 + sq);
  u = x * r * rcp64(omz);
  omu = 1.0 - u;
  if (!(omu > 0.0)) return false;
  omx = omz * rcp64(omu);
  return true;
}

__device__ __forceinline__ bool ii_map_mixed(double r, double z, double omz, double& x, double& omx, double& v) {
  const double iq = rcp64(omz + r);
  x = z * omz * iq;
  omx = (omz * omz + r) * iq;
  v = x * r * rcp64(omz);
  return omx - v > 0.0;
}

// Accepted emission: FP64 kinematics (Appendix B maps, II Lorentz kick) and
// colour update; the warp then rebuilds the event's end table cooperatively.
// Kept out of line: it runs on the parked lanes of a warp only.
template <class W>
__device__ __noinline__ bool emit(const MixedCtx& M, const W& w, Lane& L, const Emission& em) {
  const int bi = em.bi, k = em.k, bside = em.bside, ch = em.ch, type = em.type;
  const int new_fl_i = em.new_fl_i, fl_j = em.fl_j;
  const float z = em.z, omz = em.omz, tw = em.tw;
  const double Rphi = em.Rphi;
  const uint32_t ti = em.ti;
  double Pm[4], K[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) { Pm[mu] = w.P(mu, bi); K[mu] = w.P(mu, k); }
  const double sd = 2.0 * dot4(Pm, K);
  // ---- FP64 emission kinematics ----
  const double t = (double)tw;
  // the smaller of z, 1-z carries the FP32 sample's relative precision; the
  // other is formed in FP64 so that z + (1-z) = 1 and the maps conserve momentum
  const double zd = omz < 0.5f ? 1.0 - (double)omz : (double)z;
  const double omzd = omz < 0.5f ? (double)omz : 1.0 - (double)z;
  double e1v[4], e2v[4];
  transverse_basis_mixed(Pm, K, e1v, e2v);
  double cph, sph;
  gm_sincos2pi(Rphi, cph, sph);
  const double st = t * rsqrt64(t);
  double kt[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) kt[mu] = st * (cph * e1v[mu] + sph * e2v[mu]);
  const int j = L.n;
  // the maps as p_i' = a1 p_i + b1 p_k + c1 k_T, p_k' = a2 p_i + b2 p_k + c2 k_T,
  // p_j = a3 p_i + b3 p_k + c3 k_T (Appendix B), then one store of each
  double a1, b1, c1, a2, b2, c2, a3, b3, c3;
  double eta_f = 1.0;  // factor of eta of the incoming slot `eta_slot`
  int eta_slot = -1;
  double xd = 1.0, omxd = 0.0, vd = 0.0;
  const double isd = rcp64(sd);
  if (type == kFF || type == kFI) {
    const double yd = t * rcp64(zd * omzd * sd);  // y (FF) or rho (FI)
    a1 = zd; b1 = yd * omzd; c1 = 1.0;
    a3 = omzd; b3 = yd * zd; c3 = -1.0;
    a2 = 0.0; c2 = 0.0;
    if (type == kFF) {
      b2 = 1.0 - yd;
    } else {
      b2 = 1.0 + yd;
      eta_slot = k;
      eta_f = b2;
    }
  } else if (type == kIF) {
    double ud, omud;
    if (!if_map_mixed(t * isd, zd, omzd, xd, omxd, ud, omud)) return false;
    const double ixd = rcp64(xd);
    a1 = ixd; b1 = 0.0; c1 = 0.0;
    a3 = omud * omxd * ixd; b3 = ud; c3 = -1.0;
    a2 = ud * omxd * ixd; b2 = omud; c2 = 1.0;
    eta_slot = bi;
    eta_f = ixd;
  } else {
    if (!ii_map_mixed(t * isd, zd, omzd, xd, omxd, vd)) return false;
    const double ixd = rcp64(xd);
    a1 = ixd; b1 = 0.0; c1 = 0.0;
    a3 = (omxd - vd) * ixd; b3 = vd; c3 = -1.0;
    a2 = 0.0; b2 = 1.0; c2 = 0.0;
    eta_slot = bi;
    eta_f = ixd;
  }
  double pi2[4], pk2[4], pj[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    pi2[mu] = a1 * Pm[mu] + b1 * K[mu] + c1 * kt[mu];
    pk2[mu] = a2 * Pm[mu] + b2 * K[mu] + c2 * kt[mu];
    pj[mu] = a3 * Pm[mu] + b3 * K[mu] + c3 * kt[mu];
  }
  if (type == kII) {
    // Lorentz kick of every final-state parton but j (Appendix B.5)
    double Kp[4], Kn[4], KK[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      Kp[mu] = Pm[mu] + K[mu];
      Kn[mu] = (pi2[mu] + K[mu]) - pj[mu];
      KK[mu] = Kp[mu] + Kn[mu];
    }
    const double iKK2 = 2.0 * rcp64(dot4(KK, KK)), iKp2 = 2.0 * rcp64(dot4(Kp, Kp));
    for (int m = 2; m < L.n; ++m) {
      double q[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) q[mu] = w.P(mu, m);
      const double a = dot4(KK, q) * iKK2, b = dot4(Kp, q) * iKp2;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) w.P(mu, m) = q[mu] - a * KK[mu] + b * Kn[mu];
    }
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    w.P(mu, bi) = pi2[mu];
    w.P(mu, k) = pk2[mu];
    w.P(mu, j) = pj[mu];
  }
  if (eta_slot == 0) L.eta0 *= eta_f;
  else if (eta_slot == 1) L.eta1 *= eta_f;

  // colours
  const int T = 100 + L.n;
  int ci = tag_col(ti), ai = tag_acol(ti), cj = 0, aj = 0;
  if (ch == 0 || ch == 1 || ch == 3 || ch == 5) {
    if (bside == 0) { cj = ci; aj = T; ci = T; }
    else { aj = ai; cj = T; ai = T; }
  } else if (ch == 2) {
    aj = ai; cj = 0; ai = 0;
  } else if (ch == 4) {
    if (ai != 0) { ci = T; aj = T; cj = 0; }
    else { ai = T; cj = T; aj = 0; }
  } else {
    int A = ci, Bt = ai;
    if (new_fl_i > 0) { ci = 0; ai = Bt; cj = A; aj = 0; }
    else { ci = A; ai = 0; cj = 0; aj = Bt; }
  }
  w.T(bi) = pack_tag(new_fl_i, ci, ai);
  w.T(j) = pack_tag(fl_j, cj, aj);
  L.n += 1;
  L.n_emit += 1;
  return true;
}

static_assert(sizeof(Emission) <= kWavePendBytes, "parked emission exceeds its slot");

// logs a sampled PDF ratio of a winner (the paper's data for its fitted
// overestimate, App. A.2); the sample is decided by a hash of (event, draw)
__device__ __noinline__ void log_ratio(const MixedCtx& M, uint64_t id, uint64_t draw, int num, int den, float eta,
                                       float ratio) {
  uint64_t h = id * 0x9E3779B97F4A7C15ull ^ (draw * 0xD6E8FEB86659FD93ull);
  h ^= h >> 31;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 29;
  if (!((uint32_t)(h >> 32) < M.Lc.rkeep || M.Lc.rkeep == 0xFFFFFFFFu)) return;
  const unsigned long long at = atomicAdd(M.Lc.rcount, 1ull);
  if (at < M.Lc.rcap) M.Lc.rlog[at] = make_float4((float)num, (float)den, eta, ratio);
}

// a weight above one met with the plain bounds (the fitted PDF-ratio
// overestimate, or rounding at the edge of a certified bound): logged with
// class -1 - (8 type + channel) and bin -1
__device__ __noinline__ void log_plain_violation(const MixedCtx& M, float eta, float s, float tw, float w, int type,
                                                 int ch, float z) {
  if (!M.Lc.vlog) return;
  const unsigned long long at = atomicAdd(M.Lc.vcount, 1ull);
  if (at < M.Lc.vcap) {
    M.Lc.vlog[2 * at] = make_float4(eta, s, tw, w);
    M.Lc.vlog[2 * at + 1] = make_float4(-1.0f - (float)(8 * type + ch), -1.0f, z, 0.0f);
  }
}

struct Counters32 {
  unsigned long long steps = 0, trials = 0, isr_trials = 0, vetoes = 0, accepts = 0, violations = 0;
};

// The cycle after its trials (Fig. 1): the winner (best = ln t, end bq,
// channel bch, z draw bRz; bq < 0: no trial) against the cutoff, the veto
// and, when accepted, the parked emission. L.draw is past the trial draws.
// Returns the new status.
template <class W>
__device__ int step_veto(const MixedCtx& M, const SmemPdf& S, const LearnedSmem& ls, const W& w, Lane& L,
                         uint64_t id, Counters32& cnt, Emission& pend, bool& parked, float best, int bq, int bch,
                         float bRz) {
  const bool pp = S.pp[L.row] != 0;
  const float lnTc = S.lnTc[L.row];
  cnt.steps += 1;
  const uint32_t k0 = (uint32_t)M.P.seed, k1 = (uint32_t)(M.P.seed >> 32);
  const uint32_t e0 = (uint32_t)id, e1 = (uint32_t)(id >> 32);
  int bi = -1, bside = 0, k = -1;
  if (bq >= 0) {
    bi = bq >> 1;
    bside = bq & 1;
    k = __float_as_int(w.End(bq).w);
  }
  if (bi < 0 || best < lnTc) return GAPS_STATUS_DONE;
  uint32_t o1[4], o2[4];
  philox(e0, e1, (uint32_t)L.draw, (uint32_t)(L.draw >> 32), k0, k1, o1);
  philox(e0, e1, (uint32_t)(L.draw + 1), (uint32_t)((L.draw + 1) >> 32), k0, k1, o2);
  L.draw += 2;
  const float Rveto = u24(o1[1]);
  const float Rfl = u24(o2[1]);
  const float lnT_before = L.lnT;
  L.lnT = best;
  const float tw = __expf(best);

  // the winner's dipole: its invariant, momentum fraction and tags as the
  // last rebuild of the end table stored them (momenta, tags and eta change
  // only in emissions, which are followed by a rebuild)
  const float4 ax = w.Aux(bq);
  const uint32_t ti = __float_as_uint(ax.z);
  const int fl_i = tag_fl(ti);
  const bool ini = pp && bi < 2;
  const bool ink = pp && k < 2;
  const int type = ini ? (ink ? kII : kIF) : (ink ? kFI : kFF);
  const int ch = (ini ? (fl_i == 21 ? 5 : 3) : (fl_i == 21 ? 1 : 0)) + bch;
  const float s = ax.x;
  const float eta = ax.y;
  int shape;
  float coef;
  channel_over32(ch, type, M.P.nf, shape, coef);
  float zm, delta;
  zlim32(type, __expf(lnTc), s, eta, zm, delta);
  // learned bounds: pick the bin from R_z, then zeta inside it
  const bool learned_end = M.Lc.learned && L.learned_ok && ini;
  float zeta = bRz, Um = 1.0f;
  int mbin = -1;
  if (learned_end) {
    float U[8], tot = 0.0f;
    const uint2 kc = *reinterpret_cast<const uint2*>(ls.at(bq, bch, L.slot));
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      U[m] = ls.dec[((m < 4 ? kc.x : kc.y) >> (8 * (m & 3))) & 0xffu];
      tot += U[m];
    }
    const float target = bRz * tot;
    float acc = 0.0f;
    int mb = 7;  // when no earlier bin is reached, acc = U[0] + ... + U[6]
    for (int m = 0; m < 7; ++m) {
      if (target < acc + U[m]) { mb = m; break; }
      acc += U[m];
    }
    Um = U[mb];
    mbin = mb;
    float frac = Um > 0.0f ? (target - acc) / Um : 0.5f;
    frac = fminf(fmaxf(frac, 0.0f), 0.99999994f);
    zeta = ((float)mb + frac) * 0.125f;
  }
  float z, omz;
  shape_sample32(shape, zm, delta, zeta, z, omz);
  float zm_t, delta_t;
  if (!zlim32(type, tw, s, eta, zm_t, delta_t) || !(omz > delta_t) || !(z > zm_t)) {
    cnt.vetoes += 1;
    return GAPS_STATUS_ACTIVE;
  }
  const float pover = shape_val32(shape, coef, z, omz);
  const float as_t = (float)M.P.as_mz / (1.0f + (float)M.P.as_mz * (float)M.P.beta0 * __logf(tw / (float)(kMZ * kMZ)));
  const float as_ratio = as_t / (S.asOver2pi[L.row] * 2.0f * (float)kPi);
  float w8 = 0.0f, y = 0.0f, rho = 0.0f, x = 1.0f, omx = 0.0f, u = 0.0f, omu = 1.0f, v = 0.0f;
  int new_fl_i = fl_i, fl_j = 21;
  float sumF = 0.0f, B = 1.0f;
  if (type == kFF) {
    y = tw / (z * omz * s);
    float den = omz + z * y, kk;
    if (ch == 0) kk = (float)kCF * (2.0f / den - (1.0f + z));
    else if (ch == 1) kk = (float)kCA * 0.5f * (2.0f / den - 2.0f + z * omz);
    else kk = M.P.nf * (float)kTR * 0.5f * (1.0f - 2.0f * z * omz);
    w8 = as_ratio * (1.0f - y) * kk / pover;
  } else if (type == kFI) {
    rho = tw / (z * omz * s);
    x = 1.0f / (1.0f + rho);
    omx = rho / (1.0f + rho);
    float den = omz + omx, kk;
    if (ch == 0) kk = (float)kCF * (2.0f / den - (1.0f + z));
    else if (ch == 1) kk = (float)kCA * 0.5f * (2.0f / den - 2.0f + z * omz);
    else kk = M.P.nf * (float)kTR * 0.5f * (1.0f - 2.0f * z * omz);
    int f = pdf_index(tag_fl(__float_as_uint(ax.w)));
    B = bound32(M, S, f, f, eta);
    float F1 = pdf32(M, S, f, eta * (1.0f + rho), tw);
    float F0 = pdf32(M, S, f, eta, tw);
    float ratio = F0 > 0.0f ? x * F1 / F0 : 0.0f;
    w8 = as_ratio * kk / pover * ratio / B;
    if (M.Lc.rlog) log_ratio(M, id, L.draw, f, f, eta, F0 > 0.0f ? F1 / F0 : 0.0f);
  } else {
    const IsrEval ev = isr_eval32(M, S, type, ch, fl_i, eta, s, tw, z, omz, pover);
    if (!ev.ok) { cnt.vetoes += 1; return GAPS_STATUS_ACTIVE; }
    x = ev.x; omx = ev.omx; u = ev.u; omu = ev.omu; v = ev.v; sumF = ev.sumF;
    w8 = as_ratio * ev.r / Um;
    if (M.Lc.rlog) log_ratio(M, id, L.draw, ev.num, ev.den, eta, ev.fr);
    if (ch == 4) { new_fl_i = 21; fl_j = -fl_i; }
    if (ch == 5) { new_fl_i = 21; fl_j = 21; }
  }
  if (!isfinite(w8)) return GAPS_ERR_NUMERIC;
  if (w8 > 1.0f) {
    cnt.violations += 1;
    if (learned_end) {
      if (M.Lc.vlog) {
        const unsigned long long at = atomicAdd(M.Lc.vcount, 1ull);
        if (at < M.Lc.vcap) {
          M.Lc.vlog[2 * at] = make_float4(eta, s, tw, w8);
          M.Lc.vlog[2 * at + 1] = make_float4((float)isr_class(type, ch, fl_i), (float)mbin, z, zeta);
        }
      }
      // the learned bound failed here: continue the event with the plain
      // bounds from the scale before this cycle
      L.learned_ok = false;
      L.lnT = lnT_before;
      pend = Emission{1, bi, k, bside, ch, type, new_fl_i, fl_j, z, omz, tw, u01(o1[2], o1[3]), ti};
      parked = true;
      return GAPS_STATUS_ACTIVE;
    }
    log_plain_violation(M, eta, s, tw, w8, type, ch, z);
  }
  if (!(Rveto < w8)) { cnt.vetoes += 1; return GAPS_STATUS_ACTIVE; }

  if (ch == 2) {
    int f = 1 + (int)floorf(Rfl * M.P.nf);
    if (f > M.P.nf) f = M.P.nf;
    new_fl_i = f; fl_j = -f;
  } else if (ch == 6) {
    float target = Rfl * sumF, acc = 0.0f;
    int pick = 10;
    for (int f = 1; f <= 10; ++f) {
      acc += pdf32(M, S, f, eta / x, tw);
      if (target < acc) { pick = f; break; }
    }
    int fl = pick <= 5 ? pick : -(pick - 5);
    new_fl_i = fl; fl_j = fl;
  }
  if (L.n >= M.P.nmax) return GAPS_ERR_CAPACITY;

  // accepted: the emission is built later, together with the other parked
  // lanes of the warp (see the kernel loop)
  pend = Emission{0, bi, k, bside, ch, type, new_fl_i, fl_j, z, omz, tw, u01(o1[2], o1[3]), ti};
  parked = true;
  return GAPS_STATUS_ACTIVE;
}

// ---- veto-max (Sec. 2: each emission channel runs its own veto algorithm to
// its first accepted point, and the largest accepted scale wins) ----------
struct ChannelWeight {
  float w, z, omz, x, sumF;
  int ch, type, k, new_fl_i, fl_j;
  uint32_t ti;
  bool ok;  // inside the true z range and the map's domain
};

// Acceptance weight of a trial of end q, channel c at scale tw with z draw
// Rz, with the plain bounds: the arithmetic of the max-veto winner's weight.
template <class W>
__device__ __noinline__ ChannelWeight channel_weight(const MixedCtx& M, const SmemPdf& S, const W& w, const Lane& L,
                                                     int q, int c, float tw, float Rz) {
  ChannelWeight r;
  r.ok = false;
  r.w = 0.0f;
  const bool pp = S.pp[L.row] != 0;
  const float lnTc = S.lnTc[L.row];
  const int bi = q >> 1;
  r.k = __float_as_int(w.End(q).w);
  const float4 ax = w.Aux(q);
  r.ti = __float_as_uint(ax.z);
  const int fl_i = tag_fl(r.ti);
  const bool ini = pp && bi < 2, ink = pp && r.k < 2;
  r.type = ini ? (ink ? kII : kIF) : (ink ? kFI : kFF);
  r.ch = (ini ? (fl_i == 21 ? 5 : 3) : (fl_i == 21 ? 1 : 0)) + c;
  r.new_fl_i = fl_i;
  r.fl_j = 21;
  r.x = 1.0f;
  r.sumF = 0.0f;
  const float s = ax.x, eta = ax.y;
  int shape;
  float coef;
  channel_over32(r.ch, r.type, M.P.nf, shape, coef);
  float zm, delta;
  zlim32(r.type, __expf(lnTc), s, eta, zm, delta);
  shape_sample32(shape, zm, delta, Rz, r.z, r.omz);
  const float z = r.z, omz = r.omz;
  float zm_t, delta_t;
  if (!zlim32(r.type, tw, s, eta, zm_t, delta_t) || !(omz > delta_t) || !(z > zm_t)) return r;
  const float pover = shape_val32(shape, coef, z, omz);
  const float as_t = (float)M.P.as_mz / (1.0f + (float)M.P.as_mz * (float)M.P.beta0 * __logf(tw / (float)(kMZ * kMZ)));
  const float as_ratio = as_t / (S.asOver2pi[L.row] * 2.0f * (float)kPi);
  const int ch = r.ch;
  if (r.type == kFF) {
    const float y = tw / (z * omz * s);
    const float den = omz + z * y;
    float kk;
    if (ch == 0) kk = (float)kCF * (2.0f / den - (1.0f + z));
    else if (ch == 1) kk = (float)kCA * 0.5f * (2.0f / den - 2.0f + z * omz);
    else kk = M.P.nf * (float)kTR * 0.5f * (1.0f - 2.0f * z * omz);
    r.w = as_ratio * (1.0f - y) * kk / pover;
  } else if (r.type == kFI) {
    const float rho = tw / (z * omz * s);
    const float x = 1.0f / (1.0f + rho), omx = rho / (1.0f + rho);
    const float den = omz + omx;
    float kk;
    if (ch == 0) kk = (float)kCF * (2.0f / den - (1.0f + z));
    else if (ch == 1) kk = (float)kCA * 0.5f * (2.0f / den - 2.0f + z * omz);
    else kk = M.P.nf * (float)kTR * 0.5f * (1.0f - 2.0f * z * omz);
    const int f = pdf_index(tag_fl(__float_as_uint(ax.w)));
    const float B = bound32(M, S, f, f, eta);
    const float F1 = pdf32(M, S, f, eta * (1.0f + rho), tw);
    const float F0 = pdf32(M, S, f, eta, tw);
    const float ratio = F0 > 0.0f ? x * F1 / F0 : 0.0f;
    r.w = as_ratio * kk / pover * ratio / B;
  } else {
    const IsrEval ev = isr_eval32(M, S, r.type, ch, fl_i, eta, s, tw, z, omz, pover);
    if (!ev.ok) return r;
    r.x = ev.x;
    r.sumF = ev.sumF;
    r.w = as_ratio * ev.r;
    if (ch == 4) { r.new_fl_i = 21; r.fl_j = -fl_i; }
    if (ch == 5) { r.new_fl_i = 21; r.fl_j = 21; }
  }
  r.ok = true;
  return r;
}

// One cycle of veto-max: the marked ends' channels first run their own veto
// algorithms from the event's scale to their first accepted points (kept, as
// kept trials are, while the end's record is unchanged); the largest accepted
// point is the emission. Trial blocks use word 1 for t, word 3 for z and
// word 2 for the acceptance; the emission then draws one block for the
// flavour choice and the azimuth.
template <class W>
__device__ int step_vetomax(const MixedCtx& M, const SmemPdf& S, const W& w, Lane& L, uint64_t id, Counters32& cnt,
                            Emission& pend, bool& parked) {
  const bool pp = S.pp[L.row] != 0;
  const float lnTc = S.lnTc[L.row];
  const uint32_t k0 = (uint32_t)M.P.seed, k1 = (uint32_t)(M.P.seed >> 32);
  const uint32_t e0 = (uint32_t)id, e1 = (uint32_t)(id >> 32);
  cnt.steps += 1;
  float best = -INFINITY, bRz = 0.5f;
  int bq = -1, bch = 0;
  uint64_t d = L.draw;
  const int ne = 2 * L.n;
#pragma unroll 1
  for (int q = 0; q < ne; ++q) {
    float4 tr = w.Trial(q);
    if (isnan(tr.x)) {
      tr = make_float4(-INFINITY, 0.5f, -INFINITY, 0.5f);
      const float4 rec = w.End(q);
      if (__float_as_int(rec.w) >= 0) {
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
          const float ic = c == 0 ? rec.x : rec.y;
          if (ic < 0.0f) continue;  // channel absent for this emitter
          float lnT = fminf(L.lnT, rec.z), lt = -INFINITY, rz = 0.5f;
#pragma unroll 1
          while (lnT > lnTc && ic > 0.0f) {
            const uint64_t dd = d++;
            uint32_t out[4];
            philox(e0, e1, (uint32_t)dd, (uint32_t)(dd >> 32), k0, k1, out);
            cnt.trials += 1;
            if (pp && q < 4) cnt.isr_trials += 1;
            const float t1 = fmaf(__logf(u24(out[1])), ic, lnT);
            if (!(t1 > lnTc)) break;
            const ChannelWeight cw = channel_weight(M, S, w, L, q, c, __expf(t1), u24(out[3]));
            if (cw.ok && cw.w > 1.0f) {
              cnt.violations += 1;
              log_plain_violation(M, w.Aux(q).y, w.Aux(q).x, __expf(t1), cw.w, cw.type, cw.ch, cw.z);
            }
            if (cw.ok && u24(out[2]) < cw.w) {
              lt = t1;
              rz = u24(out[3]);
              break;
            }
            cnt.vetoes += 1;
            lnT = t1;
          }
          if (c == 0) { tr.x = lt; tr.y = rz; }
          else { tr.z = lt; tr.w = rz; }
        }
      }
      w.SetTrial(q, tr);
    }
    if (tr.x > best) { best = tr.x; bq = q; bch = 0; bRz = tr.y; }
    if (tr.z > best) { best = tr.z; bq = q; bch = 1; bRz = tr.w; }
  }
  L.draw = d;
  if (bq < 0 || !(best > lnTc)) return GAPS_STATUS_DONE;
  // the winner was accepted when its channel ran: the emission
  L.lnT = best;
  const float tw = __expf(best);
  const ChannelWeight cw = channel_weight(M, S, w, L, bq, bch, tw, bRz);
  uint32_t o[4];
  const uint64_t dd = L.draw++;
  philox(e0, e1, (uint32_t)dd, (uint32_t)(dd >> 32), k0, k1, o);
  const float Rfl = u24(o[1]);
  int new_fl_i = cw.new_fl_i, fl_j = cw.fl_j;
  const float4 ax = w.Aux(bq);
  const float eta = ax.y;
  if (cw.ch == 2) {
    int f = 1 + (int)floorf(Rfl * M.P.nf);
    if (f > M.P.nf) f = M.P.nf;
    new_fl_i = f; fl_j = -f;
  } else if (cw.ch == 6) {
    float target = Rfl * cw.sumF, acc = 0.0f;
    int pick = 10;
    for (int f = 1; f <= 10; ++f) {
      acc += pdf32(M, S, f, eta / cw.x, tw);
      if (target < acc) { pick = f; break; }
    }
    const int fl = pick <= 5 ? pick : -(pick - 5);
    new_fl_i = fl; fl_j = fl;
  }
  if (L.n >= M.P.nmax) return GAPS_ERR_CAPACITY;
  pend = Emission{0, bq >> 1, cw.k, bq & 1, cw.ch, cw.type, new_fl_i, fl_j, cw.z, cw.omz, tw, u01(o[2], o[3]), cw.ti};
  parked = true;
  return GAPS_STATUS_ACTIVE;
}


// Generate-select (the alternative to max-veto in Sec. 2's footnote): the
// superposition of every channel's overestimate process is a Poisson process
// in ln t whose rate is the sum R of the rates of the channels active at that
// scale (a channel is active below its end's maximum scale); a point of it
// belongs to a channel with probability rate / R. One trial is drawn from R
// at the current scale; when it falls below the next maximum scale of an
// inactive channel, the process restarts there with that channel added (no
// memory). Inline: out of line, its reference arguments would keep the trial
// loop's running maximum in local memory on every path.
__device__ __forceinline__ void select_trial(const WS& w, int ne, float lnT, float lnTc, bool pp, uint32_t e0,
                                          uint32_t e1, uint32_t k0, uint32_t k1, uint64_t& d, Counters32& cnt,
                                          float& best, int& bq, int& bch, float& bRz) {
  float t0 = lnT;
  // every pass either gives the trial or moves t0 down to the next distinct
  // maximum scale: at most 2 ne + 1 passes
  for (int pass = 0; pass <= 2 * ne && t0 > lnTc; ++pass) {
    float R = 0.0f, t1 = -INFINITY;
#pragma unroll 1
    for (int q = 0; q < ne; ++q) {
      const float4 rec = w.End(q);
      if (__float_as_int(rec.w) < 0) continue;  // no dipole on this side
      if (rec.z >= t0) {
        if (rec.x > 0.0f) R += __frcp_rn(rec.x);
        if (rec.y > 0.0f) R += __frcp_rn(rec.y);
      } else if (rec.x > 0.0f || rec.y > 0.0f) {
        t1 = fmaxf(t1, rec.z);
      }
    }
    if (R > 0.0f) {
      const uint64_t dd = d++;
      uint32_t out[4];
      philox(e0, e1, (uint32_t)dd, (uint32_t)(dd >> 32), k0, k1, out);
      cnt.trials += 1;
      const float lt = t0 + __logf(u24(out[1])) / R;
      if (lt >= t1) {
        // the channel, in canonical order, with the same partial sums as R
        const float target = u24(out[2]) * R;
        float acc = 0.0f;
        int sq = -1, sc = 0;
#pragma unroll 1
        for (int q = 0; q < ne && sq < 0; ++q) {
          const float4 rec = w.End(q);
          if (__float_as_int(rec.w) < 0 || rec.z < t0) continue;
          if (rec.x > 0.0f) {
            acc += __frcp_rn(rec.x);
            bq = q; bch = 0;  // the last active channel, should rounding leave target >= acc
            if (target < acc) { sq = q; sc = 0; continue; }
          }
          if (rec.y > 0.0f) {
            acc += __frcp_rn(rec.y);
            bq = q; bch = 1;
            if (target < acc) { sq = q; sc = 1; }
          }
        }
        if (sq >= 0) { bq = sq; bch = sc; }
        if (pp && bq < 4) cnt.isr_trials += 1;  // emitter in slot 0 or 1
        best = lt;
        bRz = u24(out[3]);
        return;
      }
    }
    t0 = t1;  // nothing above the next maximum scale: continue from there
  }
}

// One max-veto cycle of the lane's event: one overestimate trial per channel
// of every colour end in canonical order, then step_veto. With kept trials
// only the ends marked by the last rebuild draw, and after a veto only the
// winner's channel: every channel's trials are a Poisson process in ln t, so
// when the winner at t_w is vetoed, each other channel's trial is the first
// point of its process below t_w.
__device__ int step_mixed(const MixedCtx& M, const SmemPdf& S, const LearnedSmem& ls, const WS& w, Lane& L,
                          uint64_t id, Counters32& cnt, Emission& pend, bool& parked) {
  const bool pp = S.pp[L.row] != 0;
  const float lnTc = S.lnTc[L.row];
  const uint32_t k0 = (uint32_t)M.P.seed, k1 = (uint32_t)(M.P.seed >> 32);
  const uint32_t e0 = (uint32_t)id, e1 = (uint32_t)(id >> 32);
  const bool cache = M.P.trial_mode == GAPS_TRIALS_KEEP;
  float best = -INFINITY;
  int bq = -1, bch = 0;
  float bRz = 0.5f;
  const int ne = 2 * L.n;  // ends q = 2 slot + side, canonical order
  uint64_t d = L.draw;
  const bool select = M.P.trial_mode == GAPS_TRIALS_SELECT;
  if (select) select_trial(w, ne, L.lnT, lnTc, pp, e0, e1, k0, k1, d, cnt, best, bq, bch, bRz);
  // the ends' trials: the scan reads each end's larger trial scale, four ends
  // per load (one aligned float4 of the per-end maxima); only ends a rebuild
  // marked (NaN) draw, one by one in canonical order; redrawing every cycle,
  // every end draws. One copy of the drawing code (instruction-cache
  // footprint). The winning end's trials are read once at the end.
  const int nq = select ? 0 : ne;
#pragma unroll 1
  for (int q0 = 0; q0 < nq; q0 += 4) {
    float m4[4];
    if (cache) {
      const float4 v = w.Tmx4(q0);
      m4[0] = v.x; m4[1] = v.y; m4[2] = v.z; m4[3] = v.w;
    }
    bool draws = !cache;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (q0 + j >= nq) m4[j] = -INFINITY;  // past the event's ends
      else if (cache) draws = draws || isnan(m4[j]);
    }
    if (draws) {
#pragma unroll 1
      for (int q = q0; q < q0 + 4 && q < nq; ++q) {
        if (cache && !isnan(w.Tmx(q))) continue;  // kept
        float4 tr = make_float4(-INFINITY, 0.5f, -INFINITY, 0.5f);
        const float4 rec = w.End(q);
        if (__float_as_int(rec.w) >= 0) {  // a dipole on this side
          const float lnTmax = fminf(L.lnT, rec.z);
          const bool live = lnTmax > lnTc;
          const float m2 = q < 4 ? end_m2(S, w.Aux(q), q, L.row) : 0.0f;
#pragma unroll 1
          for (int c = 0; c < 2; ++c) {
            const float ic = c == 0 ? rec.x : rec.y;  // 1/c
            if (ic < 0.0f) continue;  // channel absent for this emitter
            const uint64_t dd = d++;
            if (!(live && ic > 0.0f)) continue;
            uint32_t out[4];
            philox(e0, e1, (uint32_t)dd, (uint32_t)(dd >> 32), k0, k1, out);
            cnt.trials += 1;
            if (pp && q < 4) cnt.isr_trials += 1;  // emitter in slot 0 or 1
            const float lt = trial_lnt(lnTmax, ic, __logf(u24(out[1])), m2);  // ln(t_max R^(1/c))
            if (c == 0) { tr.x = lt; tr.y = u24(out[3]); }
            else { tr.z = lt; tr.w = u24(out[3]); }
          }
        }
        w.SetTrial(q, tr);  // with redraw, the cycle's trials (read back below)
        m4[q - q0] = tr.z > tr.x ? tr.z : tr.x;
      }
    }
    // the largest wins, the earlier end on ties (and channel 0 within an end)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (m4[j] > best) { best = m4[j]; bq = q0 + j; }
  }
  if (!select && bq >= 0) {
    const float4 tr = w.Trial(bq);
    bch = tr.z > tr.x ? 1 : 0;
    bRz = bch ? tr.w : tr.y;
  }
  L.draw = d;
  const int st = step_veto(M, S, ls, w, L, id, cnt, pend, parked, best, bq, bch, bRz);
  if (cache && st == GAPS_STATUS_ACTIVE && !parked && bq >= 0) {
    // vetoed: the winner's channel draws its next trial below t_w = L.lnT
    const float4 rec = w.End(bq);
    const float ic = bch == 0 ? rec.x : rec.y;
    const float lnTmax = fminf(L.lnT, rec.z);
    float lt = -INFINITY, rz = 0.5f;
    const uint64_t dd = L.draw++;
    if (lnTmax > lnTc && ic > 0.0f) {
      uint32_t out[4];
      philox(e0, e1, (uint32_t)dd, (uint32_t)(dd >> 32), k0, k1, out);
      cnt.trials += 1;
      if (pp && bq < 4) cnt.isr_trials += 1;
      const float m2 = bq < 4 ? end_m2(S, w.Aux(bq), bq, L.row) : 0.0f;
      lt = trial_lnt(lnTmax, ic, __logf(u24(out[1])), m2);
      rz = u24(out[3]);
    }
    float4 tr = w.Trial(bq);
    if (bch == 0) { tr.x = lt; tr.y = rz; } else { tr.z = lt; tr.w = rz; }
    w.SetTrial(bq, tr);
  }
  return st;
}

__device__ __noinline__ void load_event(const MixedCtx& M, const WS& w, const LearnedSmem& ls, Lane& L,
                                       uint64_t e) {
  const DevEvents& E = M.E;
  L.ev = e;
  L.status = E.status[e];
  L.n = E.npart[e];
  L.n_emit = E.n_emit[e];
  L.steps = 0;
  L.eta0 = E.eta[e];
  L.eta1 = E.eta[E.cap + e];
  L.draw = E.draw[e];
  L.lnT = __logf((float)E.t[e]);
  L.learned_ok = true;
  L.row = mix_row(M.P, M.first + e);
  if (ls.key)
    for (int q = 0; q < 4; ++q) ls.keyat(q, L.slot) = make_float4(-1.0f, -1.0f, -1.0f, 0.0f);
  if (L.status != GAPS_STATUS_ACTIVE) return;
  if (L.n < 2 || L.n > M.P.nmax) { L.status = GAPS_ERR_NUMERIC; return; }
  for (int s = 0; s < L.n; ++s) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) w.P(mu, s) = E.P(mu, s, e);
    w.T(s) = pack_tag(E.F(s, e), E.C(s, e), E.A(s, e));
  }
}

// with_record: the event's partons were loaded into the working set (an event
// that was not active when loaded only has its scalars written back)
__device__ __noinline__ void store_event(const MixedCtx& M, const WS& w, const Lane& L, bool with_record = true) {
  const DevEvents& E = M.E;
  const uint64_t e = L.ev;
  if (with_record && L.n >= 2 && L.n <= M.P.nmax) {
    for (int s = 0; s < L.n; ++s) {
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) E.P(mu, s, e) = w.P(mu, s);
      uint32_t t = w.T(s);
      E.F(s, e) = tag_fl(t);
      E.C(s, e) = tag_col(t);
      E.A(s, e) = tag_acol(t);
    }
    E.npart[e] = L.n;
  }
  E.n_emit[e] = L.n_emit;
  E.status[e] = L.status;
  E.t[e] = (double)__expf(L.lnT);
  E.eta[e] = L.eta0;
  E.eta[E.cap + e] = L.eta1;
  E.draw[e] = L.draw;
}

// Shared memory of the mixed-precision kernels besides the PDF tables: per
// warp the tags of the event being rebuilt and, with the learned proposal, 64
// rows of network inputs and outputs, then the height decode table (dynamic
// shared memory; the network's weight image stays in global memory, read
// through L1).
struct MixedSmem {
  uint32_t* tag_stage;
  float (*stage)[64][4];
  float (*ustage)[64];
  LearnedSmem ls;
};

// Fills the block's PDF tables and decode table (the caller synchronises).
// Dynamic shared memory: the warps' tag staging, then with the learned
// proposal the height decode table and, for kernels that evaluate the
// network inside a rebuild (with_stage), the warps' 64-row tile staging.
__device__ __forceinline__ void mixed_prologue(const MixedCtx& M, SmemPdf& S, unsigned char* dyn, MixedSmem& D,
                                               bool with_stage) {
  const int nw = blockDim.x >> 5;
  D.tag_stage = reinterpret_cast<uint32_t*>(dyn);
  unsigned char* learned_smem = dyn + tag_stage_bytes(nw, M.P.nmax);
  D.stage = nullptr;
  D.ustage = nullptr;
  D.ls.code = nullptr;
  D.ls.dec = nullptr;
  D.ls.key = nullptr;
  if (M.Lc.learned) {
    float* dec = reinterpret_cast<float*>(learned_smem);
    D.ls.dec = dec;
    D.ls.code = M.W.lcode;
    D.ls.key = M.W.lkey;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) dec[k] = k < 255 ? exp2f(-(float)k * 0.0625f) : 0.0f;
    if (with_stage) {
      unsigned char* st = learned_smem + 256 * sizeof(float);
      D.stage = reinterpret_cast<float(*)[64][4]>(st);
      D.ustage = reinterpret_cast<float(*)[64]>(st + (size_t)nw * 64 * 4 * sizeof(float));
    }
  }
  for (int q = threadIdx.x; q < 12 * kSmNX; q += blockDim.x) {
    int f = q / kSmNX, ix = q % kSmNX;
    S.umax[f][ix] = (float)M.P.umax[q];
    S.lmin[f][ix] = (float)M.P.lmin[q];
    float xf = 0.0f;
    if (f < 11) xf = M.P.grid[((size_t)f * kNX + ix) * kNQ];
    else for (int k = 1; k <= 10; ++k) xf += M.P.grid[((size_t)k * kNX + ix) * kNQ];
    S.xf[f][ix] = xf;
  }
  for (int q = threadIdx.x; q < 12 * (kSmNX + 1); q += blockDim.x)
    S.sufmax[q / (kSmNX + 1)][q % (kSmNX + 1)] = (float)M.P.sufmax[q];
  for (int q = threadIdx.x; q < 12 * kSmNX; q += blockDim.x) S.first[q / kSmNX][q % kSmNX] = (float)M.P.first[q];
  if (threadIdx.x < 12) S.m2[threadIdx.x] = (float)M.P.m2[threadIdx.x];
  load_rows(S, M.P);
}

// dynamic shared memory of a mixed-precision block of `block_size` threads
// (mixed_prologue's layout)
__host__ __device__ constexpr size_t mixed_dyn_bytes(int block_size, int nmax, bool learned, bool with_stage) {
  return tag_stage_bytes(block_size / 32, nmax) +
         (learned ? 256 * sizeof(float) + (with_stage ? (size_t)(block_size / 32) * 64 * 5 * sizeof(float) : 0)
                  : 0);
}

// ---- wavefront schedule: per-event lane state in the WaveSet arrays -------
__device__ __forceinline__ void wave_load(const MixedCtx& M, Lane& L, uint64_t e) {
  const WaveSet& V = M.V;
  L.ev = e;
  L.slot = (int)e;
  L.n = V.n[e];
  L.n_emit = V.n_emit[e];
  L.status = V.status[e];
  L.steps = V.steps[e];
  L.eta0 = V.eta[e];
  L.eta1 = V.eta[V.cap + e];
  L.draw = V.draw[e];
  L.lnT = V.lnT[e];
  const int f = V.flags[e];
  L.learned_ok = (f & 1) != 0;
  L.row = (f >> 8) & 0xff;
}

__device__ __forceinline__ void wave_store(const MixedCtx& M, const Lane& L) {
  const WaveSet& V = M.V;
  const uint64_t e = L.ev;
  V.n[e] = L.n;
  V.n_emit[e] = L.n_emit;
  V.status[e] = L.status;
  V.steps[e] = L.steps;
  V.eta[e] = L.eta0;
  V.eta[V.cap + e] = L.eta1;
  V.draw[e] = L.draw;
  V.lnT[e] = L.lnT;
  V.flags[e] = (V.flags[e] & ~1) | (L.learned_ok ? 1 : 0);
}

// Appends e to list `which` for every lane with `want` (one atomic per warp);
// all 32 lanes call it.
__device__ __forceinline__ void wave_append(const MixedCtx& M, int which, bool want, uint64_t e, int lane_id) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane_id == leader) base = atomicAdd(&M.V.ctl[which], (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) M.V.list[(size_t)which * M.V.cap + base + __popc(m & ((1u << lane_id) - 1u))] = (uint32_t)e;
}

// counters: warp sums, one atomic per warp and counter
__device__ __forceinline__ void flush_counters(const MixedCtx& M, const Counters32& cnt, unsigned long long finished,
                                               unsigned long long err_cap, unsigned long long err_iter,
                                               unsigned long long err_num, unsigned long long lane_steps,
                                               unsigned long long warp_steps, unsigned long long rebuilds,
                                               unsigned long long mlp_tiles, int lane_id) {
  unsigned long long v[14] = {finished, cnt.steps, cnt.trials, cnt.isr_trials, cnt.vetoes, cnt.accepts,
                              cnt.violations, err_cap, err_iter, err_num, lane_steps, warp_steps, rebuilds,
                              mlp_tiles};
  const int idx[14] = {C_EVENTS, C_STEPS, C_TRIALS, C_ISR_TRIALS, C_VETOES, C_ACCEPTS, C_VIOLATIONS,
                       C_ERR_CAP, C_ERR_ITER, C_ERR_NUM, C_LANE_STEPS, C_WARP_STEPS, C_REBUILDS, C_MLP_TILES};
#pragma unroll 1
  for (int q = 0; q < 14; ++q) {
    unsigned long long x = v[q];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane_id == 0 && x) atomicAdd(&M.P.counters[idx[q]], x);
  }
}

// The persistent mixed-precision shower. MINB sets the register tier:
// 256-thread blocks x MINB per SM (128, 80 or 64 registers per thread).
// WAVE = false: lane g owns working-set lane g and takes events 0 .. n-1 of
// the chunk from the work counter (records loaded and stored by the kernel).
// WAVE = true: the wavefront schedule's final pass; the lanes take the events
// of the live list, whose working-set lanes and end tables the wavefront
// passes left ready, and write their state back to the WaveSet arrays.
template <int MINB, bool WAVE, bool VMAX = false>
__global__ void __launch_bounds__(256, MINB) k_shower_mixed(const __grid_constant__ MixedCtx M) {
  __shared__ SmemPdf S;
  extern __shared__ __align__(16) unsigned char dyn_lane_smem[];
  MixedSmem D;
  mixed_prologue(M, S, dyn_lane_smem, D, true);
  const MlpSmem& mlp_s = *reinterpret_cast<const MlpSmem*>(M.Lc.image);
  const LearnedSmem& ls = D.ls;
  __syncthreads();

  const int lane_id = threadIdx.x & 31;
  const int gl = blockIdx.x * blockDim.x + threadIdx.x;
  const int warp_id = threadIdx.x >> 5;
  // the events of this launch: 0 .. n-1, or the live list of the wavefront
  const uint32_t* live = WAVE ? M.V.list + (size_t)M.wave_par * M.V.cap : nullptr;
  const uint64_t n_work = WAVE ? M.V.ctl[M.wave_par] : M.n;
  unsigned long long* work = WAVE ? &M.V.ctl[WL_GRAB] : M.next;
  Lane L;
  L.slot = gl;
  L.ev = 0;
  L.n = 0;
  L.row = 0;
  L.learned_ok = false;
  L.eta0 = L.eta1 = 0.0;
  bool active = false;
  bool exhausted = false;
  Counters32 cnt;
  unsigned long long finished = 0, err_cap = 0, err_iter = 0, err_num = 0;
  unsigned long long lane_steps = 0, warp_steps = 0;
  unsigned long long rebuilds = 0, mlp_tiles = 0;  // warp-uniform
  int since_refill = M.period;
  bool parked = false;
  Emission pend;
  int since_flush = 0;
  // ends keep their trials (max-veto) or accepted points (veto-max) while
  // their records are unchanged
  const bool cache = M.P.trial_mode == GAPS_TRIALS_KEEP || VMAX;
  while (true) {
    // warp-aggregated refill of idle lanes
    unsigned idle = __ballot_sync(0xffffffffu, !active);
    if (idle && !exhausted && since_refill >= M.period) {
      since_refill = 0;
      int cnt_idle = __popc(idle);
      unsigned long long base = 0;
      if (lane_id == 0) base = atomicAdd(work, (unsigned long long)cnt_idle);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= n_work) exhausted = true;
      bool loaded = false;
      if (!active) {
        int rank = __popc(idle & ((1u << lane_id) - 1u));
        uint64_t e = base + rank;
        if (e < n_work) {
          if (WAVE) {
            wave_load(M, L, live[e]);
            active = L.status == GAPS_STATUS_ACTIVE;
          } else {
            load_event(M, WS{M.W, L.slot, M.P.nmax}, ls, L, e);
            if (L.status == GAPS_STATUS_ACTIVE) active = loaded = true;
            else { store_event(M, WS{M.W, L.slot, M.P.nmax}, L, false); finished += 1; }
          }
        }
      }
      // cooperative end tables of the freshly loaded events
      __syncwarp();  // the loads above are visible to the whole warp
      unsigned todo = __ballot_sync(0xffffffffu, loaded);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int n_src = __shfl_sync(0xffffffffu, L.n, src);
        const double e0 = __shfl_sync(0xffffffffu, L.eta0, src), e1 = __shfl_sync(0xffffffffu, L.eta1, src);
        const bool lok = __shfl_sync(0xffffffffu, L.learned_ok ? 1 : 0, src) != 0;
        const int row_src = __shfl_sync(0xffffffffu, L.row, src);
        const uint64_t ev_src = __shfl_sync(0xffffffffu, L.ev, src);
        const int slot_src = __shfl_sync(0xffffffffu, L.slot, src);
        mlp_tiles += rebuild_coop(M, S, mlp_s, ls, D.stage[warp_id], D.ustage[warp_id],
                                  WS{M.W, slot_src, M.P.nmax}, D.tag_stage + warp_id * tag_stage_words(M.P.nmax), true,
                                  slot_src, ev_src, n_src, e0, e1, row_src, lok, cache ? 0 : -1, lane_id);
        rebuilds += 1;
      }
      __syncwarp();
    }
    unsigned act = __ballot_sync(0xffffffffu, active);
    if (act == 0) {
      if (exhausted) break;
      since_refill = M.period;
      continue;
    }
    since_refill += 1;
    // build the parked emissions when enough lanes wait, when no active lane
    // could take another step, or after the longest allowed wait
    const unsigned pk = __ballot_sync(0xffffffffu, parked);
    since_flush += 1;
    if (pk && (__popc(pk) >= M.emit_batch || pk == act || since_flush >= M.emit_wait)) {
      since_flush = 0;
      bool done_emit = false;
      int keep = -1;  // ends of the emitting lane that may keep their trials
      if (parked) {
        parked = false;
        if (pend.kind == 1) {
          // plain rebuild after a learned-bound violation: the event goes on
          // from the scale before that cycle, and every end draws again
          done_emit = true;
          keep = cache ? 0 : -1;
        } else {
          done_emit = emit(M, WS{M.W, L.slot, M.P.nmax}, L, pend);
          if (done_emit) {
            cnt.accepts += 1;
            keep = cache ? 2 * (L.n - 1) : -1;  // the ends that existed before
          } else {
            cnt.vetoes += 1;  // the map failed: the winner's end draws again
            if (cache) WS{M.W, L.slot, M.P.nmax}.MarkTrial(2 * pend.bi + pend.bside);
          }
        }
      }
      __syncwarp();  // the emissions above are visible to the whole warp
      unsigned todo = __ballot_sync(0xffffffffu, done_emit);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int n_src = __shfl_sync(0xffffffffu, L.n, src);
        const double e0 = __shfl_sync(0xffffffffu, L.eta0, src), e1 = __shfl_sync(0xffffffffu, L.eta1, src);
        const bool lok = __shfl_sync(0xffffffffu, L.learned_ok ? 1 : 0, src) != 0;
        const int row_src = __shfl_sync(0xffffffffu, L.row, src);
        const uint64_t ev_src = __shfl_sync(0xffffffffu, L.ev, src);
        const int keep_src = __shfl_sync(0xffffffffu, keep, src);
        const int slot_src = __shfl_sync(0xffffffffu, L.slot, src);
        mlp_tiles += rebuild_coop(M, S, mlp_s, ls, D.stage[warp_id], D.ustage[warp_id],
                                  WS{M.W, slot_src, M.P.nmax}, D.tag_stage + warp_id * tag_stage_words(M.P.nmax), true,
                                  slot_src, ev_src, n_src, e0, e1, row_src, lok, keep_src, lane_id);
        rebuilds += 1;
      }
      __syncwarp();
    }
    lane_steps += __popc(__ballot_sync(0xffffffffu, active && !parked));
    warp_steps += 32;
    if (active && !parked) {
      int st = VMAX ? step_vetomax(M, S, WS{M.W, L.slot, M.P.nmax}, L, M.first + L.ev, cnt, pend, parked)
                    : step_mixed(M, S, ls, WS{M.W, L.slot, M.P.nmax}, L, M.first + L.ev, cnt,
                                                     pend, parked);
      if (++L.steps >= M.P.max_steps && st == GAPS_STATUS_ACTIVE) st = GAPS_ERR_ITER_CAP;
      if (st != GAPS_STATUS_ACTIVE) {
        L.status = st;
        if (WAVE) wave_store(M, L);
        else store_event(M, WS{M.W, L.slot, M.P.nmax}, L);
        active = false;
        finished += 1;
        if (st == GAPS_ERR_CAPACITY) err_cap += 1;
        else if (st == GAPS_ERR_ITER_CAP) err_iter += 1;
        else if (st == GAPS_ERR_NUMERIC) err_num += 1;
      }
    }
  }
  flush_counters(M, cnt, finished, err_cap, err_iter, err_num, lane_id == 0 ? lane_steps : 0ull,
                 lane_id == 0 ? warp_steps : 0ull, lane_id == 0 ? rebuilds : 0ull, lane_id == 0 ? mlp_tiles : 0ull,
                 lane_id);
}

// ---------------------------------------------------------------------------
// Wavefront schedule (GAPS_SCHED_WAVE). The persistent kernel above mixes
// every phase of an event's evolution in one warp: trial scans, vetoes, FP64
// emissions, end-table rebuilds with network tiles and refills, so the lanes
// of a warp diverge and the code of all phases competes for the instruction
// cache. The wavefront schedule runs the same per-event steps in passes,
// each phase as its own kernel over a list of events (the paper's
// kernel-per-step structure, Sec. 3, with live-event lists in place of its
// partitioning):
//   ends  one warp per event of the rebuild list: the cooperative end-table
//         rebuild, with the learned proposal's network tiles;
//   veto  persistent lanes over the live list: max-veto cycles of one event
//         until an emission is accepted (parked), the event ends, or the pass's
//         cycle budget is used up (the event stays live);
//   emit  one thread per parked emission: the FP64 maps and the colour update;
//         the event joins the next rebuild list and the next live list.
// After the fixed number of passes the remaining live events finish in the
// persistent kernel above (WAVE = true). Every event takes the same steps
// with the same random numbers as in the persistent kernel, so the two
// schedules give identical events. The working set has one lane per event of
// the chunk (lane = event index), so no state moves between the kernels.
// ---------------------------------------------------------------------------

// Records of the chunk into the working set and the WaveSet arrays; active
// events start the live list and the rebuild list.
__global__ void k_wave_init(const __grid_constant__ MixedCtx M) {
  LearnedSmem ls;
  ls.code = M.Lc.learned ? M.W.lcode : nullptr;
  ls.key = M.Lc.learned ? M.W.lkey : nullptr;
  ls.dec = nullptr;
  const int lane_id = threadIdx.x & 31;
  const bool cache = M.P.trial_mode == GAPS_TRIALS_KEEP;
  unsigned long long finished = 0, err_num = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // whole warps iterate together (the appends are warp-collective)
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < M.n; b += stride) {
    const uint64_t e = b + lane_id;
    bool live = false;
    if (e < M.n) {
      Lane L;
      L.slot = (int)e;
      load_event(M, WS{M.W, (int)e, M.P.nmax}, ls, L, e);
      live = L.status == GAPS_STATUS_ACTIVE;
      // bit 1: the record was loaded and is written back; bit 2: only the
      // status changed (a record that could not be read)
      const int wb = live ? 2 : (L.status != M.E.status[e] ? 4 : 0);
      M.V.flags[e] = 1 | wb | (L.row << 8);
      M.V.keep[e] = cache ? 0 : -1;
      M.V.chg[e] = -1;
      wave_store(M, L);
      if (!live) {
        finished += 1;
        if (L.status == GAPS_ERR_NUMERIC) err_num += 1;
      }
    }
    wave_append(M, WL_LIVE0, live, e, lane_id);
    wave_append(M, WL_REBUILD, live, e, lane_id);
  }
  Counters32 cnt;
  flush_counters(M, cnt, finished, 0, 0, err_num, 0, 0, 0, 0, lane_id);
}

// The trials of the ends a rebuild marked (kept-trial scheme), drawn by the
// warp together, one end per lane: the same Philox blocks, in the same
// canonical order, as the first cycle's trial loop would draw them one by one
// (each end's first counter is the event's counter plus a warp prefix sum of
// the draws of the marked ends before it), so the events are unchanged and
// the cycle that follows only scans. Returns the event's counter after the
// draws (every lane).
__device__ __forceinline__ uint64_t draw_marked_ends(const MixedCtx& M, const SmemPdf& S, const WS& w, uint64_t id,
                                                     int n, int row, float lnT, uint64_t d, int lane_id,
                                                     Counters32& cnt, unsigned defer_mask, uint64_t& defer_off) {
  const unsigned full = 0xffffffffu;
  const bool pp = S.pp[row] != 0;
  const float lnTc = S.lnTc[row];
  const uint32_t k0 = (uint32_t)M.P.seed, k1 = (uint32_t)(M.P.seed >> 32);
  const uint32_t e0 = (uint32_t)id, e1 = (uint32_t)(id >> 32);
  const int ne = 2 * n;
  for (int q0 = 0; q0 < ne; q0 += 32) {
    const int q = q0 + lane_id;
    bool marked = false;
    float4 rec = make_float4(-1.0f, -1.0f, 0.0f, __int_as_float(-1));
    int nd = 0;  // Philox blocks of this end: one per channel present
    if (q < ne) {
      marked = isnan(w.Tmx(q));
      if (marked) {
        rec = w.End(q);
        if (__float_as_int(rec.w) >= 0) nd = (rec.x >= 0.0f ? 1 : 0) + (rec.y >= 0.0f ? 1 : 0);
      }
    }
    int inc = nd;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(full, inc, off);
      if (lane_id >= off) inc += t;
    }
    const int tot = __shfl_sync(full, inc, 31);
    if (marked && q < 4 && ((defer_mask >> q) & 1u)) {
      // the dense network pass draws this end's trials from here
      defer_off = d + (uint64_t)(inc - nd);
      marked = false;
    }
    if (marked) {
      float4 tr = make_float4(-INFINITY, 0.5f, -INFINITY, 0.5f);
      if (__float_as_int(rec.w) >= 0) {
        uint64_t dd = d + (uint64_t)(inc - nd);
        const float lnTmax = fminf(lnT, rec.z);
        const bool live = lnTmax > lnTc;
        const float m2 = q < 4 ? end_m2(S, w.Aux(q), q, row) : 0.0f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float ic = c == 0 ? rec.x : rec.y;  // 1/c
          if (ic < 0.0f) continue;                  // channel absent for this emitter
          const uint64_t dc = dd++;
          if (!(live && ic > 0.0f)) continue;
          uint32_t out[4];
          philox(e0, e1, (uint32_t)dc, (uint32_t)(dc >> 32), k0, k1, out);
          cnt.trials += 1;
          if (pp && q < 4) cnt.isr_trials += 1;
          const float lt = trial_lnt(lnTmax, ic, __logf(u24(out[1])), m2);
          if (c == 0) { tr.x = lt; tr.y = u24(out[3]); }
          else { tr.z = lt; tr.w = u24(out[3]); }
        }
      }
      w.SetTrial(q, tr);
    }
    d += (uint64_t)tot;
  }
  return d;
}

// L2 prefetch of the rows a rebuild reads (one line per lane): the event's
// scalars, its first 16 partons' momenta and tags, and its first 32 ends'
// records, veto inputs and trial maxima. Addresses inside the arrays only.
__device__ __forceinline__ void prefetch_event_rows(const MixedCtx& M, uint32_t e, int lane_id) {
  const WaveSet& V = M.V;
  const WorkSet& W = M.W;
  const char* a = nullptr;
  // momenta and end rows are both nmax x 32 bytes: lines past a short row are skipped
  const size_t row_bytes = (size_t)M.P.nmax * 32;
  const size_t row_p = (size_t)e * row_bytes, row_e = (size_t)e * row_bytes;
  switch (lane_id) {
    case 0: a = (const char*)(V.flags + e); break;
    case 1: a = (const char*)(V.n + e); break;
    case 2: a = (const char*)(V.keep + e); break;
    case 3: a = (const char*)(V.chg + e); break;
    case 4: a = (const char*)(V.eta + e); break;
    case 5: a = (const char*)(V.eta + V.cap + e); break;
    case 6: a = (const char*)(V.lnT + e); break;
    case 7: a = (const char*)(V.draw + e); break;
    case 8: case 9: case 10: case 11:
      if (128 * (size_t)(lane_id - 8) < row_bytes) a = (const char*)W.p + row_p + 128 * (lane_id - 8);
      break;
    case 12: a = (const char*)(W.tag + (size_t)e * M.P.nmax); break;
    case 13: case 14: case 15: case 16:
      if (128 * (size_t)(lane_id - 13) < row_bytes) a = (const char*)W.end + row_e + 128 * (lane_id - 13);
      break;
    case 17: case 18: case 19: case 20:
      if (128 * (size_t)(lane_id - 17) < row_bytes) a = (const char*)W.aux + row_e + 128 * (lane_id - 17);
      break;
    case 21: a = (const char*)(W.tmx + (size_t)e * tmx_stride(M.P.nmax)); break;
    default: break;
  }
  if (a) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// One warp per event of the rebuild list: the end table, then (kept trials)
// the trials of the ends it marked. Also clears, for the passes after it, the
// lists this pass's later kernels fill.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_wave_ends(const __grid_constant__ MixedCtx M) {
  __shared__ SmemPdf S;
  extern __shared__ __align__(16) unsigned char dyn_lane_smem[];
  const uint64_t count = M.V.ctl[WL_REBUILD];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    M.V.ctl[WL_LIVE0 + (M.wave_par ^ 1)] = 0;  // the next pass's live list
    M.V.ctl[WL_GRAB] = 0;
  }
  // blocks past the list's last warp leave before loading their tables
  if ((uint64_t)blockIdx.x * (blockDim.x >> 5) >= count) return;
  MixedSmem D;
  const bool with_stage = M.P.trial_mode != GAPS_TRIALS_KEEP;
  mixed_prologue(M, S, dyn_lane_smem, D, with_stage);
  const MlpSmem& mlp_s = *reinterpret_cast<const MlpSmem*>(M.Lc.image);
  __syncthreads();
  const int lane_id = threadIdx.x & 31, warp_id = threadIdx.x >> 5;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const bool cache = M.P.trial_mode == GAPS_TRIALS_KEEP;
  // the warp's buffer of initial-state ends for the network pass (with the
  // learned proposal and kept trials), after the prologue's shared memory
  uint32_t* mbuf = reinterpret_cast<uint32_t*>(
                       dyn_lane_smem + mixed_dyn_bytes(blockDim.x, M.P.nmax, M.Lc.learned != 0, with_stage)) +
                   warp_id * kMlpBuf;
  int mfill = 0;  // warp-uniform
  auto mflush = [&]() {
    __syncwarp();
    unsigned long long base = 0;
    if (lane_id == 0) base = atomicAdd(&M.V.ctl[WL_MLP], (unsigned long long)mfill);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int j = lane_id; j < mfill; j += 32) M.V.mlpi[base + j] = mbuf[j];
    __syncwarp();
    mfill = 0;
  };
  unsigned long long rebuilds = 0, mlp_tiles = 0;
  Counters32 cnt;
  // the list two events ahead, so that the next event's rows can be brought
  // into L2 while this one is rebuilt (its loads are a chain of dependent
  // misses: scalars, tags, momenta, records)
  const uint32_t* rl = M.V.list + (size_t)WL_REBUILD * M.V.cap;
  const uint64_t i0 = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp_id;
  uint32_t e_a = i0 < count ? rl[i0] : 0u, e_b = i0 + nw < count ? rl[i0 + nw] : 0u;
  for (uint64_t i = i0; i < count; i += nw) {
    const uint64_t e = e_a;
    e_a = e_b;
    e_b = i + 2 * nw < count ? rl[i + 2 * nw] : 0u;
    if (i + nw < count) prefetch_event_rows(M, e_a, lane_id);
    const int flags = M.V.flags[e], n = M.V.n[e], row = (flags >> 8) & 0xff;
    const WS w{M.W, (int)e, M.P.nmax};
    unsigned defer_mask = 0;
    float4 deferred = make_float4(0.0f, 0.0f, 0.0f, 0.0f), plain = deferred;
    mlp_tiles += rebuild_body(M, S, mlp_s, D.ls, D.stage[warp_id], D.ustage[warp_id], w,
                              D.tag_stage + warp_id * tag_stage_words(M.P.nmax), true, (int)e, e, n, M.V.eta[e],
                              M.V.eta[M.V.cap + e], row, (flags & 1) != 0, M.V.keep[e], lane_id, cache, &defer_mask,
                              &deferred, &plain, M.V.chg[e]);
    rebuilds += 1;
    if (cache) {
      uint64_t off = 0;
      const uint64_t d = draw_marked_ends(M, S, w, M.first + e, n, row, M.V.lnT[e], M.V.draw[e], lane_id, cnt,
                                          defer_mask, off);
      __syncwarp();  // every lane has read the old counter
      if (lane_id == 0) M.V.draw[e] = d;
      // initial-state ends whose network inputs changed: their inputs in the
      // event's own slots, their index to the warp's buffer for the network
      // pass's queue
      const bool mine = lane_id < 4 && ((defer_mask >> lane_id) & 1u);
      const unsigned m = __ballot_sync(0xffffffffu, mine) & 0xFu;
      if (mine) {
        float4* q = M.V.mlpq + 3 * (4 * e + lane_id);
        q[0] = plain;
        q[1] = deferred;
        q[2] = make_float4(__uint_as_float((uint32_t)e), __int_as_float(lane_id | (row << 8)),
                           __uint_as_float((uint32_t)off), __uint_as_float((uint32_t)(off >> 32)));
      }
      if (m) {
        const int k = __popc(m);
        if (mfill + k > kMlpBuf) mflush();
        if (mine) mbuf[mfill + __popc(m & ((1u << lane_id) - 1u))] = (uint32_t)(4 * e + lane_id);
        mfill += k;
      }
    }
  }
  if (mfill) mflush();
  flush_counters(M, cnt, 0, 0, 0, 0, 0, 0, lane_id == 0 ? rebuilds : 0ull, lane_id == 0 ? mlp_tiles : 0ull,
                 lane_id);
}

// The dense network pass of the learned proposal: four queued initial-state
// ends per warp iteration (one 16-row tile each), from whatever events the
// rebuild pass queued them. Each end gets its height codes and key, its
// record scaled by c * mean(U), and its two trials drawn at the Philox
// counters the rebuild pass reserved for it, as the persistent kernel's
// inline evaluation and first trial loop would give them.
__global__ void __launch_bounds__(256, 2) k_wave_mlp(const __grid_constant__ MixedCtx M) {
  // the pass's queue of initial-state ends, four per warp step
  const uint64_t count = M.V.ctl[WL_MLP];
  if ((uint64_t)blockIdx.x * (blockDim.x >> 5) * 4 >= count) return;  // nothing queued for this block
  __shared__ float dec[256];
  __shared__ __align__(16) float stage_s[8][64][4];
  __shared__ float ustage_s[8][64];
  __shared__ float lnTc[kMaxRows];
  __shared__ __align__(16) unsigned char wimg[kMlpSmemBytes];  // the network's BF16 image
  {
    const uint4* src = reinterpret_cast<const uint4*>(M.Lc.image);
    uint4* dst = reinterpret_cast<uint4*>(wimg);
    for (int k = threadIdx.x; k < (int)(kMlpSmemBytes / 16); k += blockDim.x) dst[k] = src[k];
  }
  for (int k = threadIdx.x; k < 256; k += blockDim.x) dec[k] = k < 255 ? exp2f(-(float)k * 0.0625f) : 0.0f;
  if (threadIdx.x < kMaxRows) {
    const RowParams& R = M.P.rows[threadIdx.x < M.P.n_rows ? threadIdx.x : 0];
    lnTc[threadIdx.x] = (float)gm_log(R.t_cut);
  }
  __syncthreads();
  LearnedSmem ls;
  ls.code = M.W.lcode;
  ls.key = M.W.lkey;
  ls.dec = dec;
  const MlpSmem& mlp_s = *reinterpret_cast<const MlpSmem*>(wimg);
  const int lane_id = threadIdx.x & 31, warp_id = threadIdx.x >> 5;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint32_t k0 = (uint32_t)M.P.seed, k1 = (uint32_t)(M.P.seed >> 32);
  Counters32 cnt;
  unsigned long long tiles = 0;
  for (uint64_t g = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp_id; 4 * g < count; g += nw) {
    const uint64_t j = 4 * g + lane_id;
    const bool have = lane_id < 4 && j < count;
    float4 plain = make_float4(0.0f, 0.0f, 0.0f, 0.0f), in = plain, tag = plain;
    if (have) {
      const uint32_t idx = M.V.mlpi[j];
      const float4* qe = M.V.mlpq + 3 * (uint64_t)idx;  // slot (event idx / 4, end idx % 4)
      plain = qe[0];
      in = qe[1];
      tag = qe[2];
    }
    const unsigned eval = __ballot_sync(0xffffffffu, have) & 0xFu;
    const int e = (int)__float_as_uint(tag.x), qq = __float_as_int(tag.y) & 0xff, row = __float_as_int(tag.y) >> 8;
    const float tc = have ? __expf(lnTc[row]) : 1.0f;
    float scale0 = 0.0f, scale1 = 0.0f;
    learned_heights(M, mlp_s, ls, stage_s[warp_id], ustage_s[warp_id], eval, tc, in.x, in.y, __float_as_int(in.z),
                    __float_as_int(in.w), e, qq, lane_id, scale0, scale1, true);
    tiles += __popc(eval);
    if (have) {
      const WS w{M.W, e, M.P.nmax};
      float4 rec = plain;
      rec.x *= scale0;
      rec.y *= scale1;
      w.End(qq) = rec;
      // the end's trials, channel by channel, from its reserved counter
      uint64_t dd = ((uint64_t)__float_as_uint(tag.w) << 32) | (uint64_t)__float_as_uint(tag.z);
      const uint64_t id = M.first + (uint64_t)e;
      const uint32_t e0 = (uint32_t)id, e1 = (uint32_t)(id >> 32);
      const float lnTmax = fminf(M.V.lnT[e], rec.z);
      const bool live = lnTmax > lnTc[row];
      // heavy-quark measure of an incoming c or b (its two channels)
      const int fe = pdf_index(tag_fl(__float_as_uint(w.Aux(qq).z)));
      const float m2 = fe > 0 ? (float)M.P.m2[fe] : 0.0f;
      float4 tr = make_float4(-INFINITY, 0.5f, -INFINITY, 0.5f);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float ic = c == 0 ? rec.x : rec.y;
        if (ic < 0.0f) continue;
        const uint64_t dc = dd++;
        if (!(live && ic > 0.0f)) continue;
        uint32_t out[4];
        philox(e0, e1, (uint32_t)dc, (uint32_t)(dc >> 32), k0, k1, out);
        cnt.trials += 1;
        cnt.isr_trials += 1;
        const float lt = trial_lnt(lnTmax, ic, __logf(u24(out[1])), m2);
        if (c == 0) { tr.x = lt; tr.y = u24(out[3]); }
        else { tr.z = lt; tr.w = u24(out[3]); }
      }
      w.SetTrial(qq, tr);
    }
    __syncwarp();
  }
  flush_counters(M, cnt, 0, 0, 0, 0, 0, 0, 0, lane_id == 0 ? tiles : 0ull, lane_id);
}

// Persistent lanes over the live list: each lane runs max-veto cycles of one
// event until it parks an emission, ends, or uses up the pass's budget, then
// takes the next event.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_wave_veto(const __grid_constant__ MixedCtx M) {
  __shared__ SmemPdf S;
  extern __shared__ __align__(16) unsigned char dyn_lane_smem[];
  const uint64_t n_work = M.V.ctl[M.wave_par];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    M.V.ctl[WL_REBUILD] = 0;  // filled by this pass's emissions
    M.V.ctl[WL_MLP] = 0;      // filled by the next pass's rebuilds
  }
  // blocks with more lanes than the list has events leave before loading their tables
  if ((uint64_t)blockIdx.x * blockDim.x >= n_work) return;
  MixedSmem D;
  mixed_prologue(M, S, dyn_lane_smem, D, false);
  const LearnedSmem& ls = D.ls;
  __syncthreads();
  const int lane_id = threadIdx.x & 31;
  const uint32_t* live = M.V.list + (size_t)M.wave_par * M.V.cap;
  const int next_live = WL_LIVE0 + (M.wave_par ^ 1);
  Lane L;
  L.slot = 0;
  L.ev = 0;
  L.n = 0;
  L.row = 0;
  L.learned_ok = false;
  bool active = false, exhausted = false, parked = false;
  int cycles = 0, since_refill = M.period;
  // the warp's share of the live list: [gnext, gend), kWaveGrab events taken
  // with one atomic on the work counter (warp-uniform)
  uint64_t gnext = 0, gend = 0;
  Emission pend;
  Counters32 cnt;
  unsigned long long finished = 0, err_cap = 0, err_iter = 0, err_num = 0, lane_steps = 0, warp_steps = 0;
  while (true) {
    const unsigned idle = __ballot_sync(0xffffffffu, !active);
    if (idle && since_refill >= M.period && !(exhausted && gnext >= gend)) {
      since_refill = 0;
      if (gnext >= gend) {
        unsigned long long base = 0;
        if (lane_id == 0) base = atomicAdd(&M.V.ctl[WL_GRAB], (unsigned long long)kWaveGrab);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_work) {
          exhausted = true;
          gnext = gend = n_work;
        } else {
          gnext = base;
          gend = base + kWaveGrab < n_work ? base + kWaveGrab : n_work;
        }
      }
      const uint64_t i = gnext + __popc(idle & ((1u << lane_id) - 1u));
      if (!active && i < gend) {
        wave_load(M, L, live[i]);
        active = true;
        cycles = 0;
      }
      const uint64_t take = (uint64_t)__popc(idle);
      gnext = gnext + take < gend ? gnext + take : gend;
    }
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (act == 0) {
      if (exhausted && gnext >= gend) break;
      since_refill = M.period;
      continue;
    }
    since_refill += 1;
    lane_steps += __popc(act);
    warp_steps += 32;
    bool to_next = false;
    if (active) {
      int st = step_mixed(M, S, ls, WS{M.W, L.slot, M.P.nmax}, L, M.first + L.ev, cnt, pend,
                                              parked);
      if (++L.steps >= M.P.max_steps && st == GAPS_STATUS_ACTIVE) st = GAPS_ERR_ITER_CAP;
      ++cycles;
      if (st != GAPS_STATUS_ACTIVE) {
        L.status = st;
        finished += 1;
        if (st == GAPS_ERR_CAPACITY) err_cap += 1;
        else if (st == GAPS_ERR_ITER_CAP) err_iter += 1;
        else if (st == GAPS_ERR_NUMERIC) err_num += 1;
        wave_store(M, L);
        active = false;
      } else if (parked) {
        // the emission (or the plain rebuild after a learned-bound
        // violation) is built by the emission pass
        parked = false;
        *reinterpret_cast<Emission*>(M.V.pend + L.ev * kWavePendBytes) = pend;
        wave_store(M, L);
        M.V.flags[L.ev] |= kWaveParked;  // the emission pass takes it from the live list
        active = false;
      } else if (cycles >= M.wave_budget) {
        wave_store(M, L);  // continues in the next pass
        to_next = true;
        active = false;
      }
    }
    wave_append(M, next_live, to_next, L.ev, lane_id);
  }
  flush_counters(M, cnt, finished, err_cap, err_iter, err_num, lane_id == 0 ? lane_steps : 0ull,
                 lane_id == 0 ? warp_steps : 0ull, 0, 0, lane_id);
}

// One thread per event of the pass's live list; those the veto pass parked
// an emission for get the FP64 kinematics and colours of the persistent
// kernel's flush, then join the next live list and, when their end table
// changed, the rebuild list.
__global__ void __launch_bounds__(128) k_wave_emit(const __grid_constant__ MixedCtx M) {
  const uint64_t count = M.V.ctl[M.wave_par];
  const uint32_t* live = M.V.list + (size_t)M.wave_par * M.V.cap;
  if ((uint64_t)blockIdx.x * blockDim.x >= count) return;
  const int lane_id = threadIdx.x & 31;
  const bool cache = M.P.trial_mode == GAPS_TRIALS_KEEP;
  const int next_live = WL_LIVE0 + (M.wave_par ^ 1);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  Counters32 cnt;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < count; b += stride) {
    const uint64_t i = b + lane_id;
    bool have = false, rebuild = false;
    uint64_t e = 0;
    if (i < count) {
      e = live[i];
      const int f = M.V.flags[e];
      have = (f & kWaveParked) != 0;
      if (have) M.V.flags[e] = f & ~kWaveParked;
    }
    if (have) {
      Lane L;
      wave_load(M, L, e);
      const Emission em = *reinterpret_cast<const Emission*>(M.V.pend + e * kWavePendBytes);
      int keep = -1, chg = -1;
      if (em.kind == 1) {
        rebuild = true;
        keep = cache ? 0 : -1;
      } else if (emit(M, WS{M.W, (int)e, M.P.nmax}, L, em)) {
        cnt.accepts += 1;
        rebuild = true;
        keep = cache ? 2 * (L.n - 1) : -1;
        // the partons the emission moved: emitter, spectator and the new one
        // (an initial-initial emission kicks every final parton: all ends)
        if (em.type != kII) chg = em.bi | (em.k << 8) | ((L.n - 1) << 16);
      } else {
        cnt.vetoes += 1;  // the map failed: the winner's end draws again
        if (cache) WS{M.W, (int)e, M.P.nmax}.MarkTrial(2 * em.bi + em.bside);
      }
      M.V.keep[e] = keep;
      M.V.chg[e] = chg;
      wave_store(M, L);
    }
    wave_append(M, WL_REBUILD, rebuild, e, lane_id);
    wave_append(M, next_live, have, e, lane_id);
  }
  flush_counters(M, cnt, 0, 0, 0, 0, 0, 0, 0, 0, lane_id);
}

// The working set and the WaveSet arrays back into the caller's records.
__global__ void k_wave_final(const __grid_constant__ MixedCtx M) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M.n; e += stride) {
    const int f = M.V.flags[e];
    if (!(f & 6)) continue;
    Lane L;
    wave_load(M, L, e);
    store_event(M, WS{M.W, (int)e, M.P.nmax}, L, (f & 2) != 0);
  }
}


// ---------------------------------------------------------------------------
// Warp-per-event persistent shower (GAPS_SCHED_WARP). Each warp owns one event
// at a time, held in shared memory. The lanes share the event's colour ends in
// the trial generation, one end per lane per round; a warp prefix sum gives
// every trial the Philox draw of its place in the canonical order, and the
// winner is a warp arg-max with ties to the earlier trial, as in the
// lane-per-event kernel. Lane 0 runs the veto and builds an accepted emission;
// the warp then rebuilds the end table together. Every trial, veto and
// emission uses the lane-per-event kernel's arithmetic, so the two schedules
// give identical events.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t wss_stride(int nmax) { return (wss_bytes(nmax) + 15) / 16 * 16; }

__device__ __forceinline__ WSS warp_event_smem(unsigned char* base, int nmax) {
  WSS w;
  w.nmax = nmax;
  w.p = reinterpret_cast<double*>(base);
  w.end = reinterpret_cast<float4*>(base + (size_t)nmax * 4 * sizeof(double));
  w.aux = reinterpret_cast<float4*>(base + (size_t)nmax * (4 * sizeof(double) + 2 * sizeof(float4)));
  w.tag = reinterpret_cast<uint32_t*>(base + (size_t)nmax * (4 * sizeof(double) + 4 * sizeof(float4)));
  return w;
}

// every lane fills the same Lane; the slots are loaded by the lanes together
__device__ void load_event_warp(const MixedCtx& M, const WSS& w, const LearnedSmem& ls, Lane& L, uint64_t e,
                                int lane_id) {
  const DevEvents& E = M.E;
  L.ev = e;
  L.status = E.status[e];
  L.n = E.npart[e];
  L.n_emit = E.n_emit[e];
  L.steps = 0;
  L.eta0 = E.eta[e];
  L.eta1 = E.eta[E.cap + e];
  L.draw = E.draw[e];
  L.lnT = __logf((float)E.t[e]);
  L.learned_ok = true;
  L.row = mix_row(M.P, M.first + e);
  if (ls.key && lane_id < 4) ls.keyat(lane_id, L.slot) = make_float4(-1.0f, -1.0f, -1.0f, 0.0f);
  if (L.status != GAPS_STATUS_ACTIVE) return;
  if (L.n < 2 || L.n > M.P.nmax) { L.status = GAPS_ERR_NUMERIC; return; }
  for (int s = lane_id; s < L.n; s += 32) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) w.P(mu, s) = E.P(mu, s, e);
    w.T(s) = pack_tag(E.F(s, e), E.C(s, e), E.A(s, e));
  }
}

__device__ void store_event_warp(const MixedCtx& M, const WSS& w, const Lane& L, int lane_id) {
  const DevEvents& E = M.E;
  const uint64_t e = L.ev;
  if (L.n >= 2 && L.n <= M.P.nmax) {
    for (int s = lane_id; s < L.n; s += 32) {
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) E.P(mu, s, e) = w.P(mu, s);
      const uint32_t t = w.T(s);
      E.F(s, e) = tag_fl(t);
      E.C(s, e) = tag_col(t);
      E.A(s, e) = tag_acol(t);
    }
    if (lane_id == 0) E.npart[e] = L.n;
  }
  if (lane_id == 0) {
    E.n_emit[e] = L.n_emit;
    E.status[e] = L.status;
    E.t[e] = (double)__expf(L.lnT);
    E.eta[e] = L.eta0;
    E.eta[E.cap + e] = L.eta1;
    E.draw[e] = L.draw;
  }
}

// lane 0's Lane to every lane of the warp
__device__ __forceinline__ void broadcast_lane(Lane& L) {
  const unsigned full = 0xffffffffu;
  L.n = __shfl_sync(full, L.n, 0);
  L.n_emit = __shfl_sync(full, L.n_emit, 0);
  L.status = __shfl_sync(full, L.status, 0);
  L.steps = __shfl_sync(full, L.steps, 0);
  L.learned_ok = __shfl_sync(full, L.learned_ok ? 1 : 0, 0) != 0;
  L.lnT = __shfl_sync(full, L.lnT, 0);
  L.eta0 = __shfl_sync(full, L.eta0, 0);
  L.eta1 = __shfl_sync(full, L.eta1, 0);
  L.draw = __shfl_sync(full, L.draw, 0);
}

// The trials of one cycle, shared by the lanes. Returns the winner in
// (best, bq, bch, bRz) on every lane and the Philox draw after the trials.
__device__ __forceinline__ uint64_t warp_trials(const MixedCtx& M, const SmemPdf& S, const WSS& w,
                                                const Lane& L, int lane_id, Counters32& cnt, float& best, int& bq,
                                                int& bch, float& bRz, unsigned long long& lane_steps,
                                                unsigned long long& warp_steps) {
  const unsigned full = 0xffffffffu;
  const bool pp = S.pp[L.row] != 0;
  const float lnTc = S.lnTc[L.row];
  const uint64_t id = M.first + L.ev;
  const uint32_t k0 = (uint32_t)M.P.seed, k1 = (uint32_t)(M.P.seed >> 32);
  const uint32_t e0 = (uint32_t)id, e1 = (uint32_t)(id >> 32);
  best = -INFINITY;
  int bidx = 0x7fffffff;  // 2 q + c of the winner in canonical order
  bRz = 0.5f;
  uint64_t d = L.draw;
  const int ne = 2 * L.n;
  for (int q0 = 0; q0 < ne; q0 += 32) {
    const int q = q0 + lane_id;
    float4 rec = make_float4(-1.0f, -1.0f, 0.0f, __int_as_float(-1));
    int nd = 0;  // draws of this end: one per channel present
    if (q < ne) {
      rec = w.End(q);
      if (__float_as_int(rec.w) >= 0) nd = (rec.x >= 0.0f ? 1 : 0) + (rec.y >= 0.0f ? 1 : 0);
    }
    int inc = nd;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(full, inc, off);
      if (lane_id >= off) inc += t;
    }
    const int tot = __shfl_sync(full, inc, 31);
    if (nd > 0) {
      uint64_t dd = d + (uint64_t)(inc - nd);
      const float lnTmax = fminf(L.lnT, rec.z);
      const bool live = lnTmax > lnTc;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float ic = c == 0 ? rec.x : rec.y;  // 1/c
        if (ic < 0.0f) continue;  // channel absent for this emitter
        const uint64_t dc = dd++;
        if (!(live && ic > 0.0f)) continue;
        uint32_t out[4];
        philox(e0, e1, (uint32_t)dc, (uint32_t)(dc >> 32), k0, k1, out);
        cnt.trials += 1;
        if (pp && q < 4) cnt.isr_trials += 1;
        const float lt = fmaf(__logf(u24(out[1])), ic, lnTmax);
        if (lt > best) { best = lt; bidx = 2 * q + c; bRz = u24(out[3]); }
      }
    }
    d += (uint64_t)tot;
    if (lane_id == 0) {
      lane_steps += (unsigned long long)min(32, ne - q0);
      warp_steps += 32;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(full, best, off);
    const int oi = __shfl_xor_sync(full, bidx, off);
    const float oz = __shfl_xor_sync(full, bRz, off);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; bRz = oz; }
  }
  bq = bidx == 0x7fffffff ? -1 : (bidx >> 1);
  bch = bidx & 1;
  return d;
}

template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_shower_warp(const __grid_constant__ MixedCtx M) {
  __shared__ SmemPdf S;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int nw = blockDim.x >> 5;
  const int lane_id = threadIdx.x & 31, warp_id = threadIdx.x >> 5;
  const size_t ev_bytes = (size_t)nw * wss_stride(M.P.nmax);
  const WSS w = warp_event_smem(dyn_smem + (size_t)warp_id * wss_stride(M.P.nmax), M.P.nmax);
  // learned proposal after the events: staging and heights (the network's
  // weight image stays in global memory)
  unsigned char* lbase = dyn_smem + ev_bytes;
  const MlpSmem& mlp_s = *reinterpret_cast<const MlpSmem*>(M.Lc.image);
  float(*stage)[64][4] = reinterpret_cast<float(*)[64][4]>(lbase);
  float(*ustage)[64] = reinterpret_cast<float(*)[64]>(lbase + (size_t)nw * 64 * 4 * sizeof(float));
  LearnedSmem ls;  // one slot of heights per warp, in shared memory
  ls.code = nullptr;
  ls.dec = nullptr;
  ls.key = nullptr;
  if (M.Lc.learned) {
    unsigned char* hb = lbase + (size_t)nw * 64 * 5 * sizeof(float);
    float* dec = reinterpret_cast<float*>(hb);
    ls.dec = dec;
    ls.code = hb + 256 * sizeof(float);
    ls.key = reinterpret_cast<float4*>(ls.code + (size_t)nw * 64);
    for (int k = threadIdx.x; k < 256; k += blockDim.x) dec[k] = k < 255 ? exp2f(-(float)k * 0.0625f) : 0.0f;
  }
  for (int q = threadIdx.x; q < 12 * kSmNX; q += blockDim.x) {
    int f = q / kSmNX, ix = q % kSmNX;
    S.umax[f][ix] = (float)M.P.umax[q];
    S.lmin[f][ix] = (float)M.P.lmin[q];
    float xf = 0.0f;
    if (f < 11) xf = M.P.grid[((size_t)f * kNX + ix) * kNQ];
    else for (int k = 1; k <= 10; ++k) xf += M.P.grid[((size_t)k * kNX + ix) * kNQ];
    S.xf[f][ix] = xf;
  }
  for (int q = threadIdx.x; q < 12 * (kSmNX + 1); q += blockDim.x)
    S.sufmax[q / (kSmNX + 1)][q % (kSmNX + 1)] = (float)M.P.sufmax[q];
  for (int q = threadIdx.x; q < 12 * kSmNX; q += blockDim.x) S.first[q / kSmNX][q % kSmNX] = (float)M.P.first[q];
  if (threadIdx.x < 12) S.m2[threadIdx.x] = (float)M.P.m2[threadIdx.x];
  load_rows(S, M.P);
  __syncthreads();

  Lane L;
  L.slot = warp_id;
  Counters32 cnt;
  unsigned long long finished = 0, err_cap = 0, err_iter = 0, err_num = 0;
  unsigned long long lane_steps = 0, warp_steps = 0, rebuilds = 0, mlp_tiles = 0;
  bool active = false;
  while (true) {
    if (!active) {
      unsigned long long e = 0;
      if (lane_id == 0) e = atomicAdd(M.next, 1ull);
      e = __shfl_sync(0xffffffffu, e, 0);
      if (e >= M.n) break;
      load_event_warp(M, w, ls, L, e, lane_id);
      __syncwarp();
      if (L.status != GAPS_STATUS_ACTIVE) {
        store_event_warp(M, w, L, lane_id);
        finished += lane_id == 0 ? 1 : 0;
        if (lane_id == 0 && L.status == GAPS_ERR_NUMERIC) err_num += 1;
        __syncwarp();
        continue;
      }
      active = true;
      mlp_tiles += rebuild_coop(M, S, mlp_s, ls, stage[warp_id], ustage[warp_id], w, w.tag, false, warp_id, L.ev,
                                L.n, L.eta0, L.eta1, L.row, L.learned_ok, -1, lane_id);
      rebuilds += 1;
    }
    float best, bRz;
    int bq, bch;
    const uint64_t d = warp_trials(M, S, w, L, lane_id, cnt, best, bq, bch, bRz, lane_steps, warp_steps);
    int st = GAPS_STATUS_ACTIVE;
    bool done_emit = false;
    if (lane_id == 0) {
      L.draw = d;
      Emission pend;
      bool parked = false;
      st = step_veto(M, S, ls, w, L, M.first + L.ev, cnt, pend, parked, best, bq, bch, bRz);
      if (++L.steps >= M.P.max_steps && st == GAPS_STATUS_ACTIVE) st = GAPS_ERR_ITER_CAP;
      if (st == GAPS_STATUS_ACTIVE && parked) {
        if (pend.kind == 1) {
          done_emit = true;  // plain rebuild after a learned-bound violation
        } else {
          done_emit = emit(M, w, L, pend);
          if (done_emit) cnt.accepts += 1;
          else cnt.vetoes += 1;
        }
      }
      L.status = st;
    }
    broadcast_lane(L);
    st = L.status;
    done_emit = __shfl_sync(0xffffffffu, done_emit ? 1 : 0, 0) != 0;
    __syncwarp();  // lane 0's writes to the event are visible to the warp
    if (st != GAPS_STATUS_ACTIVE) {
      store_event_warp(M, w, L, lane_id);
      active = false;
      if (lane_id == 0) {
        finished += 1;
        if (st == GAPS_ERR_CAPACITY) err_cap += 1;
        else if (st == GAPS_ERR_ITER_CAP) err_iter += 1;
        else if (st == GAPS_ERR_NUMERIC) err_num += 1;
      }
      __syncwarp();
      continue;
    }
    if (done_emit) {
      mlp_tiles += rebuild_coop(M, S, mlp_s, ls, stage[warp_id], ustage[warp_id], w, w.tag, false, warp_id, L.ev,
                                L.n, L.eta0, L.eta1, L.row, L.learned_ok, -1, lane_id);
      rebuilds += 1;
    }
  }
  unsigned long long v[14] = {finished, cnt.steps, cnt.trials, cnt.isr_trials, cnt.vetoes, cnt.accepts,
                              cnt.violations, err_cap, err_iter, err_num, lane_steps, warp_steps,
                              lane_id == 0 ? rebuilds : 0ull, lane_id == 0 ? mlp_tiles : 0ull};
  const int idx[14] = {C_EVENTS, C_STEPS, C_TRIALS, C_ISR_TRIALS, C_VETOES, C_ACCEPTS, C_VIOLATIONS,
                       C_ERR_CAP, C_ERR_ITER, C_ERR_NUM, C_LANE_STEPS, C_WARP_STEPS, C_REBUILDS, C_MLP_TILES};
#pragma unroll 1
  for (int q = 0; q < 14; ++q) {
    unsigned long long x = v[q];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane_id == 0 && x) atomicAdd(&M.P.counters[idx[q]], x);
  }
}

}  // namespace

void workset_carve(void* base, int lanes, int nmax, WorkSet& W) {
  char* p = (char*)base;
  W.lanes = lanes;
  W.p = (double*)p;
  p += (size_t)lanes * nmax * 4 * sizeof(double);
  W.end = (float4*)p;
  p += (size_t)lanes * nmax * 2 * sizeof(float4);
  W.trial = (float4*)p;
  p += (size_t)lanes * nmax * 2 * sizeof(float4);
  W.aux = (float4*)p;
  p += (size_t)lanes * nmax * 2 * sizeof(float4);
  W.tmx = (float*)p;
  p += (size_t)lanes * tmx_stride(nmax) * sizeof(float);
  W.lkey = (float4*)p;
  p += (size_t)lanes * 4 * sizeof(float4);
  W.lcode = (unsigned char*)p;
  p += (size_t)lanes * 64;
  W.tag = (uint32_t*)p;
}


namespace {

// Targets of the learned bound (the "teacher"): for every logged initial-state
// end, channel and zeta bin, the largest acceptance ratio r over 33 zeta points
// of the bin and 64 scales t log-spaced over [t_c, t_kin] (both ends), as ln(max(r, 1e-6)),
// with the network's input features of the row.
constexpr int kTeacherZ = 32, kTeacherT = 64;
__global__ void k_isr_targets(const __grid_constant__ MixedCtx M, const float4* states, uint64_t n_states, float* feats, float* targets) {
  __shared__ SmemPdf S;
  for (int q = threadIdx.x; q < 12 * kSmNX; q += blockDim.x) {
    int f = q / kSmNX, ix = q % kSmNX;
    S.umax[f][ix] = (float)M.P.umax[q];
    S.lmin[f][ix] = (float)M.P.lmin[q];
    float xf = 0.0f;
    if (f < 11) xf = M.P.grid[((size_t)f * kNX + ix) * kNQ];
    else for (int k = 1; k <= 10; ++k) xf += M.P.grid[((size_t)k * kNX + ix) * kNQ];
    S.xf[f][ix] = xf;
  }
  for (int q = threadIdx.x; q < 12 * (kSmNX + 1); q += blockDim.x)
    S.sufmax[q / (kSmNX + 1)][q % (kSmNX + 1)] = (float)M.P.sufmax[q];
  for (int q = threadIdx.x; q < 12 * kSmNX; q += blockDim.x) S.first[q / kSmNX][q % kSmNX] = (float)M.P.first[q];
  if (threadIdx.x < 12) S.m2[threadIdx.x] = (float)M.P.m2[threadIdx.x];
  __syncthreads();
  const uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_states * 16) return;
  const float4 st = states[row / 16];
  const int c = (int)((row / 8) % 2), m = (int)(row % 8);
  const float eta = st.x, s = st.y;
  const int type = (int)st.z, fidx = (int)st.w;
  const int fl_i = fidx == 0 ? 21 : (fidx <= 5 ? fidx : -(fidx - 5));
  const int ch = (fl_i == 21 ? 5 : 3) + c;
  const float tc = __expf(M.lnTc);
  float f[4];
  mlp_features(eta, s, tc, m, isr_class(type, ch, fl_i), f);
  for (int k = 0; k < 4; ++k) feats[4 * row + k] = f[k];
  int shape;
  float coefd;
  channel_over32(ch, type, M.P.nf, shape, coefd);
  float zm, delta;
  float best = 0.0f;
  const float tk = tkin32(type, s, eta);
  if (tk > tc && zlim32(type, tc, s, eta, zm, delta)) {
    const float ltc = __logf(tc), ltk = __logf(tk);
    for (int a = 0; a <= kTeacherZ; ++a) {
      const float zeta = ((float)m + (float)a * (1.0f / kTeacherZ)) * 0.125f;
      float z, omz;
      shape_sample32(shape, zm, delta, fminf(zeta, 0.99999994f), z, omz);
      const float pover = shape_val32(shape, (float)coefd, z, omz);
      for (int b = 0; b < kTeacherT; ++b) {
        // log-spaced, both ends included: the ratio is often largest at t_c
        const float t = __expf(ltc + (ltk - ltc) * (float)b * (1.0f / (kTeacherT - 1)));
        float zm_t, delta_t;
        if (!zlim32(type, t, s, eta, zm_t, delta_t) || !(omz > delta_t) || !(z > zm_t)) continue;
        const IsrEval ev = isr_eval32(M, S, type, ch, fl_i, eta, s, t, z, omz, pover);
        if (ev.ok) best = fmaxf(best, ev.r);
      }
    }
  }
  targets[row] = __logf(fmaxf(best, 1e-6f));
}

}  // namespace

cudaError_t launch_isr_targets(const DevParams& P, int q_independent, const float4* states, uint64_t n_states,
                               float* feats, float* targets, cudaStream_t stream) {
  if (n_states == 0) return cudaSuccess;
  MixedCtx M;
  M.P = P;
  M.q_independent = q_independent;
  M.lnTc = (float)gm_log(P.t_cut);
  M.asOver2pi = (float)(P.as_over / (2.0 * kPi));
  M.lxminf = (float)P.lxmin; M.dlxf = (float)P.dlx; M.lqminf = (float)P.lqmin; M.dlqf = (float)P.dlq;
  const uint64_t rows = n_states * 16;
  k_isr_targets<<<(unsigned)((rows + 127) / 128), 128, 0, stream>>>(M, states, n_states, feats, targets);
  return cudaGetLastError();
}

constexpr int kWarpKernelMaxDyn = 200 * 1024;

// Opt-in for the dynamic shared memory of the mixed-precision kernels (the
// learned proposal's, up to 64 KB; the warp-per-event kernel's events, up to
// 200 KB) on the current device; called when a context is created.
template <class K>
cudaError_t opt_in(K kernel, int bytes, cudaError_t e) {
  return e == cudaSuccess ? cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) : e;
}

cudaError_t mixed_kernels_init() {
  const int bytes = 64 * 1024;
  cudaError_t e = cudaSuccess;
  e = opt_in(k_shower_mixed<2, false>, bytes, e);
  e = opt_in(k_shower_mixed<3, false>, bytes, e);
  e = opt_in(k_shower_mixed<4, false>, bytes, e);
  e = opt_in(k_shower_mixed<2, true>, bytes, e);
  e = opt_in(k_shower_mixed<3, true>, bytes, e);
  e = opt_in(k_shower_mixed<4, true>, bytes, e);
  e = opt_in(k_shower_mixed<2, false, true>, bytes, e);
  e = opt_in(k_shower_mixed<3, false, true>, bytes, e);
  e = opt_in(k_shower_mixed<4, false, true>, bytes, e);
  e = opt_in(k_wave_ends<2>, bytes, e);
  e = opt_in(k_wave_ends<3>, bytes, e);
  e = opt_in(k_wave_ends<4>, bytes, e);
  e = opt_in(k_wave_veto<2>, bytes, e);
  e = opt_in(k_wave_veto<3>, bytes, e);
  e = opt_in(k_wave_veto<4>, bytes, e);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_shower_warp<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWarpKernelMaxDyn);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_shower_warp<128, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWarpKernelMaxDyn);
  return e;
}

// shared memory of a warp-per-event block of `block_size` threads
size_t warp_kernel_smem(int block_size, int nmax, bool learned) {
  const size_t nw = (size_t)block_size / 32;
  size_t b = nw * wss_stride(nmax);
  if (learned) b += nw * 64 * 5 * sizeof(float) + 256 * sizeof(float) + nw * 64 + nw * 4 * sizeof(float4);
  return b;
}

cudaError_t launch_shower_warp(const DevParams& P, const DevEvents& E, const LearnedCfg& Lc, uint64_t first,
                               uint64_t n, int blocks, int block_size, int blocks_per_sm, int q_independent,
                               unsigned long long* next, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  MixedCtx M;
  M.P = P; M.E = E; M.Lc = Lc; M.first = first; M.n = n; M.next = next;
  M.q_independent = q_independent;
  M.period = 1;
  M.emit_batch = 1;
  M.emit_wait = 4;
  M.lnTc = (float)gm_log(P.t_cut);
  M.asOver2pi = (float)(P.as_over / (2.0 * kPi));
  M.lxminf = (float)P.lxmin; M.dlxf = (float)P.dlx; M.lqminf = (float)P.lqmin; M.dlqf = (float)P.dlq;
  const size_t dyn = warp_kernel_smem(block_size, P.nmax, Lc.learned != 0);
  if (dyn > (size_t)kWarpKernelMaxDyn) return cudaErrorInvalidValue;
  cudaError_t err = cudaMemsetAsync(next, 0, sizeof(unsigned long long), stream);
  if (err != cudaSuccess) return err;
  if (blocks <= 0) return cudaErrorInvalidValue;
  if (block_size < 32 || block_size > 256 || block_size % 32) return cudaErrorInvalidValue;
  // register tier: three or more resident blocks of at most 128 threads get
  // the tighter budget, anything else up to 255 registers per thread
  if (blocks_per_sm >= 3 && block_size <= 128) k_shower_warp<128, 3><<<blocks, block_size, dyn, stream>>>(M);
  else k_shower_warp<256, 1><<<blocks, block_size, dyn, stream>>>(M);
  return cudaGetLastError();
}

namespace {
MixedCtx mixed_ctx(const DevParams& P, const DevEvents& E, const WorkSet& W, const LearnedCfg& Lc, uint64_t first,
                   uint64_t n, int period, int emit_batch, int q_independent, unsigned long long* next) {
  MixedCtx M;
  M.P = P; M.E = E; M.W = W; M.Lc = Lc; M.first = first; M.n = n; M.next = next;
  M.q_independent = q_independent;
  M.period = period < 1 ? 1 : period;
  M.emit_batch = emit_batch < 1 ? 1 : (emit_batch > 32 ? 32 : emit_batch);
  M.emit_wait = 4 * M.emit_batch;
  M.lnTc = (float)gm_log(P.t_cut);
  M.asOver2pi = (float)(P.as_over / (2.0 * kPi));
  M.lxminf = (float)P.lxmin; M.dlxf = (float)P.dlx; M.lqminf = (float)P.lqmin; M.dlqf = (float)P.dlq;
  M.V = WaveSet{};
  M.wave_par = 0;
  M.wave_budget = 0;
  return M;
}

// register tier of a launch: the resident threads per SM it asks for
int mixed_tier(int blocks, int block_size, int sm_count) {
  const int threads_per_sm = blocks * block_size / max(1, sm_count);
  return threads_per_sm <= 512 ? 2 : (threads_per_sm <= 768 ? 3 : 4);
}

template <bool WAVE, bool VMAX = false>
void launch_persistent(const MixedCtx& M, int tier, int blocks, int block_size, size_t dyn, cudaStream_t stream) {
  if (tier == 2) k_shower_mixed<2, WAVE, VMAX><<<blocks, block_size, dyn, stream>>>(M);
  else if (tier == 3) k_shower_mixed<3, WAVE, VMAX><<<blocks, block_size, dyn, stream>>>(M);
  else k_shower_mixed<4, WAVE, VMAX><<<blocks, block_size, dyn, stream>>>(M);
}
}  // namespace

cudaError_t launch_shower_mixed(const DevParams& P, const DevEvents& E, const WorkSet& W, const LearnedCfg& Lc,
                                uint64_t first, uint64_t n, int blocks, int block_size, int sm_count, int period,
                                int emit_batch, int q_independent, unsigned long long* next,
                                cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const MixedCtx M = mixed_ctx(P, E, W, Lc, first, n, period, emit_batch, q_independent, next);
  cudaError_t err = cudaMemsetAsync(next, 0, sizeof(unsigned long long), stream);
  if (err != cudaSuccess) return err;
  // learned proposal: per-warp staging, height decode table, 64 bytes of
  // height codes per lane
  const size_t dyn = mixed_dyn_bytes(block_size, P.nmax, Lc.learned != 0, true);
  const int tier = mixed_tier(blocks, block_size, sm_count);
  if (P.trial_mode == GAPS_TRIALS_VETOMAX) launch_persistent<false, true>(M, tier, blocks, block_size, dyn, stream);
  else launch_persistent<false>(M, tier, blocks, block_size, dyn, stream);
  return cudaGetLastError();
}

// Per-event state of the wavefront schedule for `cap` events: sizes and
// carve (every array 256-byte aligned).
namespace {
size_t al256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace

size_t wave_state_bytes(uint64_t cap) {
  return al256(cap * sizeof(float)) + 7 * al256(cap * sizeof(int)) + al256(2 * cap * sizeof(double)) +
         al256(cap * sizeof(uint64_t)) + al256(cap * (size_t)kWavePendBytes) + al256(4 * cap * sizeof(uint32_t)) +
         al256(12 * cap * sizeof(float4)) + al256(4 * cap * sizeof(uint32_t)) +
         al256(WL_NCTL * sizeof(unsigned long long));
}

void wave_state_carve(void* base, uint64_t cap, WaveSet& V) {
  char* p = (char*)base;
  auto take = [&](size_t b) { char* q = p; p += al256(b); return q; };
  V.cap = cap;
  V.lnT = (float*)take(cap * sizeof(float));
  V.n = (int*)take(cap * sizeof(int));
  V.n_emit = (int*)take(cap * sizeof(int));
  V.status = (int*)take(cap * sizeof(int));
  V.steps = (int*)take(cap * sizeof(int));
  V.flags = (int*)take(cap * sizeof(int));
  V.keep = (int*)take(cap * sizeof(int));
  V.chg = (int*)take(cap * sizeof(int));
  V.eta = (double*)take(2 * cap * sizeof(double));
  V.draw = (uint64_t*)take(cap * sizeof(uint64_t));
  V.pend = (unsigned char*)take(cap * (size_t)kWavePendBytes);
  V.list = (uint32_t*)take(4 * cap * sizeof(uint32_t));
  V.mlpq = (float4*)take(12 * cap * sizeof(float4));
  V.mlpi = (uint32_t*)take(4 * cap * sizeof(uint32_t));
  V.ctl = (unsigned long long*)take(WL_NCTL * sizeof(unsigned long long));
}

// The wavefront schedule over events first .. first + n - 1 (records 0 .. n-1):
// `passes` passes of (ends, veto, emit), the last rebuilds, the persistent
// kernel over the events still live, and the records written back. W has one
// lane per event (W.lanes >= n), V is carved for at least n events.
cudaError_t launch_shower_wave(const DevParams& P, const DevEvents& E, const WorkSet& W, const WaveSet& V,
                               const LearnedCfg& Lc, uint64_t first, uint64_t n, int passes, int budget,
                               int blocks, int veto_blocks, int block_size, int sm_count, int period,
                               int emit_batch, int q_independent, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  if (n > V.cap || (uint64_t)W.lanes < n || passes < 0 || budget < 1) return cudaErrorInvalidValue;
  MixedCtx M = mixed_ctx(P, E, W, Lc, first, n, period, emit_batch, q_independent, nullptr);
  M.V = V;
  M.wave_budget = budget;
  cudaError_t err = cudaMemsetAsync(V.ctl, 0, WL_NCTL * sizeof(unsigned long long), stream);
  if (err != cudaSuccess) return err;
  // dynamic shared memory: the rebuild kernel evaluates the network itself
  // only when it redraws (with kept trials the network pass does), the veto
  // kernel only decodes heights, the persistent kernel does both
  const bool learned = Lc.learned != 0;
  const bool keep = P.trial_mode == GAPS_TRIALS_KEEP;
  const size_t dyn_ends = mixed_dyn_bytes(block_size, P.nmax, learned, !keep) +
                          (learned && keep ? (size_t)(block_size / 32) * kMlpBuf * sizeof(uint32_t) : 0);
  const size_t dyn_veto = mixed_dyn_bytes(block_size, P.nmax, learned, false);
  const size_t dyn = mixed_dyn_bytes(block_size, P.nmax, learned, true);
  const int tier = mixed_tier(blocks, block_size, sm_count);
  // the veto kernel's own residency (its register budget)
  const int veto_tier = mixed_tier(veto_blocks, block_size, sm_count);
  // grid-stride kernels: enough warps to cover the SMs several times
  const int flat_blocks = sm_count * 16;
  k_wave_init<<<flat_blocks, 128, 0, stream>>>(M);
  for (int w = 0; w <= passes; ++w) {
    M.wave_par = w & 1;
    if (tier == 2) k_wave_ends<2><<<blocks, block_size, dyn_ends, stream>>>(M);
    else if (tier == 3) k_wave_ends<3><<<blocks, block_size, dyn_ends, stream>>>(M);
    else k_wave_ends<4><<<blocks, block_size, dyn_ends, stream>>>(M);
    if (Lc.learned) k_wave_mlp<<<sm_count * 2, 256, 0, stream>>>(M);
    if (w == passes) break;  // the last rebuilds, then the persistent kernel
    if (veto_tier == 2) k_wave_veto<2><<<veto_blocks, block_size, dyn_veto, stream>>>(M);
    else if (veto_tier == 3) k_wave_veto<3><<<veto_blocks, block_size, dyn_veto, stream>>>(M);
    else k_wave_veto<4><<<veto_blocks, block_size, dyn_veto, stream>>>(M);
    k_wave_emit<<<flat_blocks, 128, 0, stream>>>(M);
  }
  // the remaining events: a tail of long showers, run like the veto kernel
  launch_persistent<true>(M, veto_tier, veto_blocks, block_size, dyn, stream);
  k_wave_final<<<flat_blocks, 128, 0, stream>>>(M);
  return cudaGetLastError();
}

}  // namespace gaps

// ---------------------------------------------------------------------------
// Allocation-free entry point. Some callers cannot allocate device memory:
// code that runs inside a host that owns every allocation (an embedding
// framework with its own pool, or a plugin that must not grow the process's
// device footprint), or code whose memory is fixed before it starts. For them
// the mixed-precision shower runs with every piece of its scratch memory in
// file-scope device arrays: the per-lane working set of 64 blocks x 128 threads
// for at most 32 partons per event (37.7 MB), the work counter, the
// statistics, and copies of the PDF grid and its bound tables. Every GPU that
// loads the library holds these arrays until the process exits.
// ---------------------------------------------------------------------------
namespace gaps {
namespace {

constexpr int kStaticBlocks = 64, kStaticThreads = 128;
constexpr int kStaticLanes = kStaticBlocks * kStaticThreads;
constexpr int kStaticMaxNmax = 32;
// the carve of workset_carve for the static launch shape (a record with fewer
// parton slots carves less)
constexpr size_t kStaticWorkBytes = workset_bytes(kStaticLanes, kStaticMaxNmax);
static __device__ __align__(256) unsigned char g_static_work[kStaticWorkBytes];
static __device__ __align__(256) float g_static_grid[GAPS_PDF_NFL * GAPS_PDF_NX * GAPS_PDF_NQ];
static __device__ __align__(256) double g_static_tables[kBoundTableDoubles];
static __device__ __align__(256) unsigned long long g_static_counters[C_NCOUNTERS + 1];

// device addresses of the arrays, looked up once per device
struct StaticAddrs {
  void* work;
  float* grid;
  double* tables;
  unsigned long long* counters;
  bool ready;
};
constexpr int kStaticMaxDevices = 64;
StaticAddrs g_static_addrs[kStaticMaxDevices];
std::mutex g_static_mutex;

int static_addresses(int dev, StaticAddrs& out) {
  std::lock_guard<std::mutex> lock(g_static_mutex);
  StaticAddrs& a = g_static_addrs[dev];
  if (!a.ready) {
    if (cudaGetSymbolAddress(&a.work, g_static_work) != cudaSuccess) return GAPS_ERR_CUDA;
    if (cudaGetSymbolAddress((void**)&a.grid, g_static_grid) != cudaSuccess) return GAPS_ERR_CUDA;
    if (cudaGetSymbolAddress((void**)&a.tables, g_static_tables) != cudaSuccess) return GAPS_ERR_CUDA;
    if (cudaGetSymbolAddress((void**)&a.counters, g_static_counters) != cudaSuccess) return GAPS_ERR_CUDA;
    a.ready = true;
  }
  out = a;
  return GAPS_OK;
}

}  // namespace
}  // namespace gaps

extern "C" int gaps_shower_static(const gaps_config* cfg, uint64_t first_event, uint64_t n,
                                  const gaps_events* ev, gaps_stats* stats, void* stream) {
  using namespace gaps;
  if (!cfg || !ev) return GAPS_ERR_INVALID_ARG;
  gaps_config c = *cfg;  // always the persistent mixed-precision shower
  c.precision = GAPS_MIXED;
  c.schedule = GAPS_SCHED_PERSISTENT;
  if (validate_config(c) != GAPS_OK) return GAPS_ERR_INVALID_ARG;
  if (!ev->p || !ev->flav || !ev->col || !ev->acol || !ev->npart || !ev->status || !ev->n_emit ||
      !ev->weight || !ev->t || !ev->eta || !ev->draw)
    return GAPS_ERR_INVALID_ARG;
  if (n > ev->capacity || ev->nmax != cfg->nmax_partons) return GAPS_ERR_INVALID_ARG;
  if (ev->nmax > kStaticMaxNmax) return GAPS_ERR_INVALID_ARG;  // beyond the static working set
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GAPS_ERR_NO_DEVICE;
  if (dev < 0 || dev >= kStaticMaxDevices) return GAPS_ERR_INVALID_ARG;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GAPS_ERR_CUDA;
  StaticAddrs a;
  int rc = static_addresses(dev, a);
  if (rc != GAPS_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  DevParams P;
  fill_params(c, P);
  int q_independent = 1;
  if (cfg->pdf_grid) {
    double tables[kBoundTableDoubles];
    build_bound_tables(cfg->pdf_grid, tables);
    q_independent = grid_q_independent(cfg->pdf_grid);
    const size_t gbytes = sizeof(float) * GAPS_PDF_NFL * GAPS_PDF_NX * GAPS_PDF_NQ;
    if (cudaMemcpyAsync(a.grid, cfg->pdf_grid, gbytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return GAPS_ERR_CUDA;
    if (cudaMemcpyAsync(a.tables, tables, sizeof tables, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return GAPS_ERR_CUDA;
    // `tables` lives on this stack frame: wait for the copy before returning
    if (cudaStreamSynchronize(st) != cudaSuccess) return GAPS_ERR_CUDA;
  }
  // the counters keep the previous call's values: start from zero
  if (cudaMemsetAsync(a.counters, 0, sizeof(unsigned long long) * (C_NCOUNTERS + 1), st) != cudaSuccess)
    return GAPS_ERR_CUDA;
  P.grid = a.grid;
  set_bound_tables(P, a.tables, cfg->pdf_grid);
  P.counters = a.counters;
  DevEvents E;
  E.cap = ev->capacity; E.nmax = ev->nmax; E.p = ev->p; E.flav = ev->flav; E.col = ev->col;
  E.acol = ev->acol; E.npart = ev->npart; E.status = ev->status; E.n_emit = ev->n_emit;
  E.weight = ev->weight; E.t = ev->t; E.eta = ev->eta; E.draw = ev->draw;
  WorkSet W;
  workset_carve(a.work, kStaticLanes, ev->nmax, W);
  LearnedCfg plain{};
  if (launch_shower_mixed(P, E, W, plain, first_event, n, kStaticBlocks, kStaticThreads, n_sm, 1, 8,
                          q_independent, a.counters + C_NCOUNTERS, st) != cudaSuccess)
    return GAPS_ERR_CUDA;
  if (stats) {
    unsigned long long h[C_NCOUNTERS];
    if (cudaMemcpyAsync(h, a.counters, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return GAPS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GAPS_ERR_CUDA;
    stats->events = h[C_EVENTS]; stats->steps = h[C_STEPS]; stats->trials = h[C_TRIALS];
    stats->isr_trials = h[C_ISR_TRIALS]; stats->vetoes = h[C_VETOES]; stats->accepts = h[C_ACCEPTS];
    stats->violations = h[C_VIOLATIONS]; stats->err_capacity = h[C_ERR_CAP];
    stats->err_iter_cap = h[C_ERR_ITER]; stats->err_numeric = h[C_ERR_NUM];
    stats->lane_steps = h[C_LANE_STEPS]; stats->warp_steps = h[C_WARP_STEPS];
    stats->rebuilds = h[C_REBUILDS]; stats->mlp_tiles = h[C_MLP_TILES];
  }
  return GAPS_OK;
}
