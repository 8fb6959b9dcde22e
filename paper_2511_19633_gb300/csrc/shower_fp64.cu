// FP64 max-veto dipole shower (Section 2, Fig. 1; Appendices A and B of
// arXiv:2511.19633), one event per thread, evolving the caller's SoA record
// in place. Compiled without FMA contraction (-fmad=false) so that every
// event reproduces a plain FP64 CPU evaluation to rounding of libm calls.
//
// Launch forms:
//   k_shower_fp64     one thread per event, runs each event to completion
//                     (the paper's layout without partitioning);
//   k_shower_fp64_pq  persistent grid: a thread takes the next unstarted
//                     event from a global counter as soon as its event
//                     finishes (live-event refill instead of the paper's
//                     thrust::partition, Section 3.1).
#include "physics_fp64.cuh"

namespace gaps {
namespace {

struct Counters {
  unsigned long long steps = 0, trials = 0, isr_trials = 0, vetoes = 0, accepts = 0, violations = 0;
};

struct Winner {
  int i, k, side, ch, type, shape;
  double t, Rz, coef, zm, delta, s, eta, B;
  double m2;  // heavy-quark measure dt/(t - m2) of the trial, 0: dt/t
};

// One max-veto cycle for event e. Returns the new status (ACTIVE, DONE or an
// error code). n, t, eta0/eta1, draw live in registers of the caller.
__device__ int shower_step(const DevParams& P, const DevEvents& E, uint64_t e, int& n, double& t,
                           double& eta0, double& eta1, Rng& rng, int& n_emit, Counters& cnt) {
  cnt.steps += 1;
  Winner best;
  best.t = -1.0;
  best.i = -1;
  best.m2 = 0.0;
  for (int i = 0; i < n; ++i) {
    int ci = E.C(i, e), ai = E.A(i, e);
    if (ci == 0 && ai == 0) continue;
    int fi = E.F(i, e);
    bool ini = (P.process != GAPS_EE_QQ) && i < 2;
    for (int side = 0; side < 2; ++side) {
      int tag = side == 0 ? ci : ai;
      if (tag == 0) continue;
      int k = -1;
      for (int m = 0; m < n; ++m) {
        if (m == i) continue;
        if (side == 0 ? (E.A(m, e) == tag) : (E.C(m, e) == tag)) { k = m; break; }
      }
      if (k < 0) continue;
      bool ink = (P.process != GAPS_EE_QQ) && k < 2;
      int type = ini ? (ink ? kII : kIF) : (ink ? kFI : kFF);
      double pi[4], pk[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) { pi[mu] = E.P(mu, i, e); pk[mu] = E.P(mu, k, e); }
      double s = 2.0 * dot4(pi, pk);
      double eta = 0.0;
      if (type == kFI) eta = (k == 0) ? eta0 : eta1;
      if (type == kIF || type == kII) eta = (i == 0) ? eta0 : eta1;
      int first = ini ? (fi == 21 ? 5 : 3) : (fi == 21 ? 1 : 0);
      int nch = (!ini && fi != 21) ? 1 : 2;
      for (int c = 0; c < nch; ++c) {
        int ch = first + c;
        double Rt, Rz;
        rng.next2(Rt, Rz);
        double tmax = fmin(t, t_kin_max(type, s, eta));
        if (!(tmax > P.t_cut)) continue;
        // heavy-quark measure correction (App. A.2): an incoming c or b with a
        // threshold draws its q <- q and q <- g trials in dt/(t - m_q^2), down to
        // m_q^2 (1 + kHqFloor)
        double mq2 = 0.0;
        if ((type == kIF || type == kII) && (ch == 3 || ch == 4)) {
          const int fe = pdf_index(fi);
          if (fe >= 0 && P.thr[fe] >= 0) mq2 = P.m2[fe];
        }
        if (mq2 > 0.0 && !(tmax > mq2 * (1.0 + kHqFloor))) continue;
        double zm, delta;
        if (!z_limits(type, P.t_cut, s, eta, zm, delta)) continue;
        int shape;
        double coef;
        channel_over(ch, type, P.nf, shape, coef);
        double B = 1.0;
        if (type == kFI) {
          int f = pdf_index(E.F(k, e));
          B = pdf_ratio_bound(P, f, f, eta);
        } else if (type == kIF || type == kII) {
          int num, den;
          isr_pdf_indices(ch, fi, num, den);
          B = pdf_ratio_bound(P, num, den, eta);
        }
        if (!(B > 0.0)) continue;
        double cc = P.as_over / (2.0 * kPi) * B * coef * shape_integral(shape, zm, delta);
        if (!(cc > 0.0)) continue;
        cnt.trials += 1;
        if (type == kIF || type == kII) cnt.isr_trials += 1;
        double tt = mq2 > 0.0 ? mq2 + (tmax - mq2) * gm_exp(gm_log(Rt) / cc) : tmax * gm_exp(gm_log(Rt) / cc);
        if (mq2 > 0.0 && !(tt > mq2 * (1.0 + kHqFloor))) continue;  // below the channel's floor
        if (tt > best.t) {
          best.i = i; best.k = k; best.side = side; best.ch = ch; best.type = type;
          best.t = tt; best.Rz = Rz; best.shape = shape; best.coef = coef;
          best.zm = zm; best.delta = delta; best.s = s; best.eta = eta; best.B = B; best.m2 = mq2;
        }
      }
    }
  }
  if (best.i < 0 || best.t < P.t_cut) return GAPS_STATUS_DONE;
  if (!isfinite(best.t)) return GAPS_ERR_NUMERIC;
  double Rveto, Rphi, Rfl, Rcol;
  rng.next2(Rveto, Rphi);
  rng.next2(Rfl, Rcol);
  const double tw = best.t;
  t = tw;

  double z, omz;
  shape_sample(best.shape, best.zm, best.delta, best.Rz, z, omz);
  double zm_t, delta_t;
  if (!z_limits(best.type, tw, best.s, best.eta, zm_t, delta_t) || !(omz > delta_t) || !(z > zm_t)) {
    cnt.vetoes += 1;
    return GAPS_STATUS_ACTIVE;
  }
  double pover = shape_value(best.shape, best.coef, z, omz);
  double as_ratio = alpha_s(P, tw) / P.as_over;
  const int type = best.type, ch = best.ch, bi = best.i, bk = best.k;
  const double s = best.s;
  int fl_i = E.F(bi, e);
  double w = 0.0;
  double y = 0.0, rho = 0.0, x = 1.0, omx = 0.0, u = 0.0, omu = 1.0, v = 0.0;
  int new_fl_i = fl_i, fl_j = 21;
  double sumF = 0.0;
  if (type == kFF) {
    y = tw / (z * omz * s);
    double k;
    double den = omz + z * y;
    if (ch == 0) k = kCF * (2.0 / den - (1.0 + z));
    else if (ch == 1) k = kCA / 2.0 * (2.0 / den - 2.0 + z * omz);
    else k = P.nf * kTR / 2.0 * (1.0 - 2.0 * z * omz);
    w = as_ratio * (1.0 - y) * k / pover;
  } else if (type == kFI) {
    rho = tw / (z * omz * s);
    x = 1.0 / (1.0 + rho);
    omx = rho / (1.0 + rho);
    double k;
    double den = omz + omx;
    if (ch == 0) k = kCF * (2.0 / den - (1.0 + z));
    else if (ch == 1) k = kCA / 2.0 * (2.0 / den - 2.0 + z * omz);
    else k = P.nf * kTR / 2.0 * (1.0 - 2.0 * z * omz);
    int f = pdf_index(E.F(bk, e));
    double eta = best.eta;
    double F1 = pdf_xf(P, f, eta * (1.0 + rho), tw);
    double F0 = pdf_xf(P, f, eta, tw);
    double ratio = (F0 > 0.0) ? x * F1 / F0 : 0.0;
    w = as_ratio * k / pover * ratio / best.B;
  } else {
    double r = tw / s;
    double J;
    if (type == kIF) {
      if (!if_map(r, z, omz, x, omx, u, omu)) { cnt.vetoes += 1; return GAPS_STATUS_ACTIVE; }
      J = 1.0 / (x * omu + u * omx);
    } else {
      if (!ii_map(r, z, omz, x, omx, v)) { cnt.vetoes += 1; return GAPS_STATUS_ACTIVE; }
      J = 1.0 / z;
    }
    double eta = best.eta;
    if (!(x > eta)) { cnt.vetoes += 1; return GAPS_STATUS_ACTIVE; }
    double k;
    double soft = (type == kIF) ? (omx + u) : omx;
    if (ch == 3) k = kCF * (2.0 / soft - (1.0 + x));
    else if (ch == 4) k = kTR * (1.0 - 2.0 * x * omx);
    else if (ch == 5) k = kCA * (1.0 / soft + omx / x - 1.0 + x * omx);
    else k = kCF / 2.0 * (x + 2.0 * omx / x);
    int num, den;
    isr_pdf_indices(ch, fl_i, num, den);
    double F0 = pdf_xf(P, den, eta, tw);
    double F1;
    if (ch == 6) {
      F1 = 0.0;
      for (int f = 1; f <= 10; ++f) F1 += pdf_xf(P, f, eta / x, tw);
      sumF = F1;
    } else {
      F1 = pdf_xf(P, num, eta / x, tw);
    }
    double Fratio = (F0 > 0.0) ? F1 / F0 : 0.0;
    if (best.m2 > 0.0) Fratio = Fratio * ((tw - best.m2) / tw);  // heavy-quark measure correction
    w = as_ratio * k * J * x / pover * Fratio / best.B;
    if (ch == 4) { new_fl_i = 21; fl_j = -fl_i; }
    if (ch == 5) { new_fl_i = 21; fl_j = 21; }
  }
  if (!isfinite(w)) return GAPS_ERR_NUMERIC;
  if (w > 1.0) cnt.violations += 1;
  if (!(Rveto < w)) { cnt.vetoes += 1; return GAPS_STATUS_ACTIVE; }

  // accepted: flavours
  if (ch == 2) {
    int f = 1 + (int)floor(Rfl * P.nf);
    if (f > P.nf) f = P.nf;
    new_fl_i = f; fl_j = -f;
  } else if (ch == 6) {
    double target = Rfl * sumF, acc = 0.0;
    int pick = 10;
    for (int f = 1; f <= 10; ++f) {
      acc += pdf_xf(P, f, best.eta / x, tw);
      if (target < acc) { pick = f; break; }
    }
    int fl = pick <= 5 ? pick : -(pick - 5);
    new_fl_i = fl; fl_j = fl;
  }
  if (n >= P.nmax) return GAPS_ERR_CAPACITY;

  // kinematics
  double Pm[4], K[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) { Pm[mu] = E.P(mu, bi, e); K[mu] = E.P(mu, bk, e); }
  double e1[4], e2[4];
  transverse_basis(Pm, K, e1, e2);
  double st = sqrt(tw), cph, sph;
  gm_sincos2pi(Rphi, cph, sph);  // phi = 2 pi R_phi
  double kt[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) kt[mu] = st * (cph * e1[mu] + sph * e2[mu]);
  const int j = n;
  double pj[4];
  if (type == kFF) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      E.P(mu, bi, e) = z * Pm[mu] + (y * omz) * K[mu] + kt[mu];
      pj[mu] = omz * Pm[mu] + (y * z) * K[mu] - kt[mu];
      E.P(mu, bk, e) = (1.0 - y) * K[mu];
    }
  } else if (type == kFI) {
    double xinv = 1.0 + rho;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      E.P(mu, bi, e) = z * Pm[mu] + (omz * rho) * K[mu] + kt[mu];
      pj[mu] = omz * Pm[mu] + (z * rho) * K[mu] - kt[mu];
      E.P(mu, bk, e) = xinv * K[mu];
    }
    if (bk == 0) eta0 = eta0 * xinv; else eta1 = eta1 * xinv;
  } else if (type == kIF) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      E.P(mu, bi, e) = Pm[mu] / x;
      pj[mu] = (omu * omx / x) * Pm[mu] + u * K[mu] - kt[mu];
      E.P(mu, bk, e) = (u * omx / x) * Pm[mu] + omu * K[mu] + kt[mu];
    }
    if (bi == 0) eta0 = eta0 / x; else eta1 = eta1 / x;
  } else {
    double pa[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      pa[mu] = Pm[mu] / x;
      E.P(mu, bi, e) = pa[mu];
      pj[mu] = ((omx - v) / x) * Pm[mu] + v * K[mu] - kt[mu];
    }
    if (bi == 0) eta0 = eta0 / x; else eta1 = eta1 / x;
    // Lorentz kick of all other final-state particles (eq. IIkinematics3)
    double Kp[4], Kn[4], KK[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      Kp[mu] = Pm[mu] + K[mu];
      Kn[mu] = (pa[mu] + K[mu]) - pj[mu];
      KK[mu] = Kp[mu] + Kn[mu];
    }
    double KK2 = dot4(KK, KK), Kp2 = dot4(Kp, Kp);
    for (int m = 2; m < n; ++m) {
      double q[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) q[mu] = E.P(mu, m, e);
      double a = 2.0 * dot4(KK, q) / KK2;
      double b = 2.0 * dot4(Kp, q) / Kp2;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) E.P(mu, m, e) = q[mu] - a * KK[mu] + b * Kn[mu];
    }
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) E.P(mu, j, e) = pj[mu];

  // colours: new tag 100 + slot of j
  int T = 100 + n;
  int ci = E.C(bi, e), ai = E.A(bi, e);
  int cj = 0, aj = 0;
  if (ch == 0 || ch == 1 || ch == 3 || ch == 5) {
    if (best.side == 0) { cj = ci; aj = T; ci = T; }
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
  E.C(bi, e) = ci; E.A(bi, e) = ai; E.F(bi, e) = new_fl_i;
  E.C(j, e) = cj; E.A(j, e) = aj; E.F(j, e) = fl_j;
  n += 1;
  n_emit += 1;
  cnt.accepts += 1;
  return GAPS_STATUS_ACTIVE;
}

// warp-aggregated counter flush; every lane of the warp must call it
__device__ __forceinline__ void flush_counters(const DevParams& P, const Counters& c,
                                               unsigned long long finished) {
  __syncwarp();
  unsigned long long v[7] = {finished, c.steps, c.trials, c.isr_trials, c.vetoes, c.accepts, c.violations};
  const int idx[7] = {C_EVENTS, C_STEPS, C_TRIALS, C_ISR_TRIALS, C_VETOES, C_ACCEPTS, C_VIOLATIONS};
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    unsigned long long x = v[q];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&P.counters[idx[q]], x);
  }
}

__device__ __forceinline__ void count_error(const DevParams& P, int st) {
  if (st == GAPS_ERR_CAPACITY) atomicAdd(&P.counters[C_ERR_CAP], 1ull);
  else if (st == GAPS_ERR_ITER_CAP) atomicAdd(&P.counters[C_ERR_ITER], 1ull);
  else if (st == GAPS_ERR_NUMERIC) atomicAdd(&P.counters[C_ERR_NUM], 1ull);
}

// run event e to completion; returns its final status
__device__ int run_event(const DevParams& P0, const DevEvents& E, uint64_t e, uint64_t id, Counters& cnt) {
  int st = E.status[e];
  if (st != GAPS_STATUS_ACTIVE) return st;
  DevParams P = P0;  // the event's row of a mixed batch
  if (P0.n_rows > 1) apply_row(P, mix_row(P0, id));
  int n = E.npart[e];
  if (n < 2 || n > P.nmax) {  // not a record written by the hard-process kernel
    E.status[e] = GAPS_ERR_NUMERIC;
    count_error(P, GAPS_ERR_NUMERIC);
    return GAPS_ERR_NUMERIC;
  }
  double t = E.t[e];
  double eta0 = E.eta[e], eta1 = E.eta[E.cap + e];
  int n_emit = E.n_emit[e];
  Rng rng;
  rng.init(P.seed, id, E.draw[e]);
  int steps = 0;
  while (st == GAPS_STATUS_ACTIVE) {
    st = shower_step(P, E, e, n, t, eta0, eta1, rng, n_emit, cnt);
    if (++steps >= P.max_steps && st == GAPS_STATUS_ACTIVE) st = GAPS_ERR_ITER_CAP;
  }
  E.npart[e] = n;
  E.t[e] = t;
  E.eta[e] = eta0;
  E.eta[E.cap + e] = eta1;
  E.n_emit[e] = n_emit;
  E.draw[e] = rng.draw;
  E.status[e] = st;
  if (st < 0) count_error(P, st);
  return st;
}

__global__ void k_shower_fp64(DevParams P, DevEvents E, uint64_t first, uint64_t n) {
  uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Counters cnt;
  unsigned long long fin = 0;
  if (e < n) {
    run_event(P, E, e, first + e, cnt);
    fin = 1;
  }
  flush_counters(P, cnt, fin);
}

// persistent form: each thread pulls event indices from *next until n
__global__ void k_shower_fp64_pq(DevParams P, DevEvents E, uint64_t first, uint64_t n,
                                 unsigned long long* next) {
  Counters cnt;
  unsigned long long fin = 0;
  while (true) {
    unsigned long long e = atomicAdd(next, 1ull);
    if (e >= n) break;
    run_event(P, E, e, first + e, cnt);
    fin += 1;
  }
  flush_counters(P, cnt, fin);
}

}  // namespace

cudaError_t launch_shower_fp64(const DevParams& P, const DevEvents& E, uint64_t first, uint64_t n,
                               int block_size, int persistent_blocks, unsigned long long* next,
                               cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  int bs = block_size > 0 ? block_size : 128;
  if (persistent_blocks > 0 && next) {
    cudaError_t err = cudaMemsetAsync(next, 0, sizeof(unsigned long long), stream);
    if (err != cudaSuccess) return err;
    k_shower_fp64_pq<<<persistent_blocks, bs, 0, stream>>>(P, E, first, n, next);
  } else {
    unsigned grid = (unsigned)((n + bs - 1) / bs);
    k_shower_fp64<<<grid, bs, 0, stream>>>(P, E, first, n);
  }
  return cudaGetLastError();
}

}  // namespace gaps
