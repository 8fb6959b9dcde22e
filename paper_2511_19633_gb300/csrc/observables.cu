// Per-event observables (Section 4.1 of arXiv:2511.19633; e+e- event shapes
// as in GAPS 1) and weighted histograms. One thread per event; the clustering
// works on a thread-local copy of the final-state momenta. Histograms are
// privatised per block in shared memory and merged with global atomics.
#include "physics_fp64.cuh"

namespace gaps {


namespace {

constexpr int kMaxFinal = 128;

template <typename R>
__device__ __forceinline__ R norm3(const R* p) {
  return sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
}

// thrust: all 2^(n-1) subsets for n <= 12 (total momentum is zero), otherwise
// the exact construction from candidate axes p_i x p_j with the four sign
// choices of i and j
template <typename R>
__device__ R thrust(const R (*ps)[4], int n) {
  R sum = 0;
  for (int i = 0; i < n; ++i) sum += norm3(ps[i]);
  if (n < 2 || !(sum > R(0))) return R(1);
  R best = 0;
  if (n <= 12) {
    for (uint32_t m = 0; m < (1u << (n - 1)); ++m) {
      R v0 = 0, v1 = 0, v2 = 0;
      for (int i = 0; i < n; ++i)
        if ((m >> i) & 1u) { v0 += ps[i][1]; v1 += ps[i][2]; v2 += ps[i][3]; }
      R l = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      best = fmax(best, l);
    }
  } else {
    for (int i = 0; i < n; ++i) {
      for (int j = i + 1; j < n; ++j) {
        R ax0 = ps[i][2] * ps[j][3] - ps[i][3] * ps[j][2];
        R ax1 = ps[i][3] * ps[j][1] - ps[i][1] * ps[j][3];
        R ax2 = ps[i][1] * ps[j][2] - ps[i][2] * ps[j][1];
        R b0 = 0, b1 = 0, b2 = 0;
        for (int k = 0; k < n; ++k) {
          if (k == i || k == j) continue;
          R d = ps[k][1] * ax0 + ps[k][2] * ax1 + ps[k][3] * ax2;
          if (d > R(0)) { b0 += ps[k][1]; b1 += ps[k][2]; b2 += ps[k][3]; }
        }
        for (int si = 0; si < 2; ++si) {
          for (int sj = 0; sj < 2; ++sj) {
            R v0 = b0, v1 = b1, v2 = b2;
            if (si) { v0 += ps[i][1]; v1 += ps[i][2]; v2 += ps[i][3]; }
            if (sj) { v0 += ps[j][1]; v1 += ps[j][2]; v2 += ps[j][3]; }
            R l = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
            best = fmax(best, l);
          }
        }
      }
    }
  }
  return R(2) * best / sum;
}

template <typename R>
__device__ __forceinline__ void erase(R (*ps)[4], int& m, int at) {
  for (int q = at; q < m - 1; ++q)
    for (int mu = 0; mu < 4; ++mu) ps[q][mu] = ps[q + 1][mu];
  m -= 1;
}

// Durham clustering, E-scheme; y23, y34 = smallest y_ij when 3 -> 2, 4 -> 3
template <typename R>
__device__ void durham(R (*ps)[4], int m, R& y23, R& y34) {
  R evis = 0;
  for (int i = 0; i < m; ++i) evis += ps[i][0];
  y23 = 0; y34 = 0;
  while (m > 1) {
    R ymin = R(INFINITY);
    int bi = -1, bj = -1;
    for (int i = 0; i < m; ++i) {
      for (int j = i + 1; j < m; ++j) {
        R ni = norm3(ps[i]), nj = norm3(ps[j]);
        R omc;  // 1 - cos(theta_ij)
        if constexpr (sizeof(R) == 8) {
          omc = R(1) - (ps[i][1] * ps[j][1] + ps[i][2] * ps[j][2] + ps[i][3] * ps[j][3]) / (ni * nj);
        } else {
          // |n_i - n_j|^2 / 2 keeps the relative precision for collinear pairs
          R d0 = ps[i][1] / ni - ps[j][1] / nj, d1 = ps[i][2] / ni - ps[j][2] / nj,
            d2 = ps[i][3] / ni - ps[j][3] / nj;
          omc = R(0.5) * (d0 * d0 + d1 * d1 + d2 * d2);
        }
        R emin = fmin(ps[i][0], ps[j][0]);
        R y = R(2) * emin * emin * omc / (evis * evis);
        if (y < ymin) { ymin = y; bi = i; bj = j; }
      }
    }
    if (m == 3) y23 = ymin;
    if (m == 4) y34 = ymin;
    for (int mu = 0; mu < 4; ++mu) ps[bi][mu] += ps[bj][mu];
    erase(ps, m, bj);
  }
}

// Pseudo-jet layout: FP64 keeps (E, px, py, pz); FP32 keeps the light-cone
// components (E + pz, px, py, E - pz), formed in FP64 from the event record,
// so that rapidities near the beam axis keep their relative precision (E-scheme
// recombination adds both forms componentwise).
template <typename R>
__device__ __forceinline__ void jet_kin(const R* p, R& pt2, R& y, R& phi) {
  pt2 = p[1] * p[1] + p[2] * p[2];
  if constexpr (sizeof(R) == 8) y = R(0.5) * log((p[0] + p[3]) / (p[0] - p[3]));
  else y = R(0.5) * log(p[0] / p[3]);
  phi = atan2(p[2], p[1]);
}

template <typename R>
__device__ __forceinline__ R jet_pz(const R* p) {
  if constexpr (sizeof(R) == 8) return p[3];
  else return R(0.5) * (p[0] - p[3]);
}

// anti-kT distance of pseudo-jets i, j from their cached kinematics
template <typename R>
__device__ __forceinline__ R akt_dij(const R* pt2, const R* y, const R* phi, int i, int j, R R2) {
  R dphi = fabs(phi[i] - phi[j]);
  if (dphi > R(kPi)) dphi = R(2.0 * kPi) - dphi;
  R dr2 = (y[i] - y[j]) * (y[i] - y[j]) + dphi * dphi;
  return fmin(R(1) / pt2[i], R(1) / pt2[j]) * dr2 / R2;
}

// nearest neighbour of i among j > i
template <typename R>
__device__ __forceinline__ void akt_nn(const R* pt2, const R* y, const R* phi, int m, int i, R R2, R* nnd, int* nnj) {
  R best = R(INFINITY);
  int bj = -1;
  for (int j = i + 1; j < m; ++j) {
    R d = akt_dij(pt2, y, phi, i, j, R2);
    if (d < best) { best = d; bj = j; }
  }
  nnd[i] = best;
  nnj[i] = bj;
}

// anti-kT R (Cacciari, Salam, Soyez 2008), E-scheme, rapidity-azimuth
// distance. Nearest-neighbour bookkeeping (O(n^2)); the minimum is searched
// in the order of a full scan (beam distance of i, then pairs (i, j > i)), so
// the clustering sequence equals the brute-force one. Reports the number of
// jets with pT > 5 GeV and |eta| < 5 and the leading one's pT and eta.
template <typename R>
__device__ void antikt(R (*ps)[4], int m, R Rj, int& njets, R& lead, R& lead_eta) {
  R pt2[kMaxFinal], y[kMaxFinal], phi[kMaxFinal], nnd[kMaxFinal];
  int nnj[kMaxFinal];
  int w = 0;
  for (int i = 0; i < m; ++i) {
    if (ps[i][1] * ps[i][1] + ps[i][2] * ps[i][2] > R(0)) {
      for (int mu = 0; mu < 4; ++mu) ps[w][mu] = ps[i][mu];
      ++w;
    }
  }
  m = w;
  const R R2 = Rj * Rj;
  for (int i = 0; i < m; ++i) jet_kin(ps[i], pt2[i], y[i], phi[i]);
  for (int i = 0; i < m; ++i) akt_nn(pt2, y, phi, m, i, R2, nnd, nnj);
  njets = 0;
  lead = 0;
  lead_eta = 0;
  while (m > 0) {
    R dmin = R(INFINITY);
    int bi = -1, bj = -1;
    for (int i = 0; i < m; ++i) {
      R diB = R(1) / pt2[i];
      if (diB < dmin) { dmin = diB; bi = i; bj = -1; }
      if (nnd[i] < dmin) { dmin = nnd[i]; bi = i; bj = nnj[i]; }
    }
    int gone;
    if (bj < 0) {
      R jpt = sqrt(ps[bi][1] * ps[bi][1] + ps[bi][2] * ps[bi][2]);
      R jeta = asinh(jet_pz(ps[bi]) / jpt);
      if (jpt > R(5) && fabs(jeta) < R(5)) {
        njets += 1;
        if (jpt > lead) { lead = jpt; lead_eta = jeta; }
      }
      gone = bi;
    } else {
      for (int mu = 0; mu < 4; ++mu) ps[bi][mu] += ps[bj][mu];
      gone = bj;
    }
    // remove `gone`, keeping the order of the others
    for (int q = gone; q < m - 1; ++q) {
      for (int mu = 0; mu < 4; ++mu) ps[q][mu] = ps[q + 1][mu];
      pt2[q] = pt2[q + 1]; y[q] = y[q + 1]; phi[q] = phi[q + 1];
      nnd[q] = nnd[q + 1]; nnj[q] = nnj[q + 1];
    }
    m -= 1;
    for (int i = 0; i < m; ++i)
      if (nnj[i] > gone) nnj[i] -= 1;
    if (bj >= 0) jet_kin(ps[bi], pt2[bi], y[bi], phi[bi]);
    // refresh the neighbours that pointed at a changed or removed pseudo-jet
    for (int i = 0; i < m; ++i) {
      bool stale = (bj >= 0 && (i == bi || nnj[i] == bi)) || nnj[i] == gone;
      if (bj >= 0 && i < bi && !stale) {
        // a merged pseudo-jet may become i's nearest neighbour, or displace one
        R d = akt_dij(pt2, y, phi, i, bi, R2);
        if (d < nnd[i] || (d == nnd[i] && bi < nnj[i])) { nnd[i] = d; nnj[i] = bi; }
      }
      if (stale) akt_nn(pt2, y, phi, m, i, R2, nnd, nnj);
    }
  }
}

__device__ __forceinline__ int bin_of(const HistDef& H, int h, double v) {
  if (H.logx[h]) {
    if (!(v > 0.0)) return 0;
    v = log10(v);
  }
  if (!(v >= H.lo[h])) return 0;
  double f = (v - H.lo[h]) / (H.hi[h] - H.lo[h]);
  int b = (int)floor(f * H.nb[h]);
  if (b >= H.nb[h]) return H.nb[h] + 1;
  return b + 1;
}

// R = double for per-event parity (GAPS_FP64), float for mixed-precision contexts
template <typename R>
__global__ void k_observables(DevParams P, DevEvents E, uint64_t first, uint64_t n, double* obs, HistSet Hs,
                              double* sumw, double* sumw2) {
  // shared: per row of the batch, sumw then sumw2 [GAPS_NHIST][GAPS_HIST_BINS]
  extern __shared__ double sh[];
  __shared__ HistDef sH[kMaxRows];
  __shared__ int s_pp[kMaxRows];
  constexpr int kSet = GAPS_NHIST * GAPS_HIST_BINS;
  const bool fill = sumw != nullptr;
  if (threadIdx.x < P.n_rows) {
    sH[threadIdx.x] = Hs.h[threadIdx.x];
    s_pp[threadIdx.x] = P.rows[threadIdx.x].process != GAPS_EE_QQ;
  }
  if (fill)
    for (int q = threadIdx.x; q < 2 * kSet * P.n_rows; q += blockDim.x) sh[q] = 0.0;
  __syncthreads();
  uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    const int row = mix_row(P, first + e);
    const HistDef& H = sH[row];
    double* hw = sh + 2 * kSet * row;
    double* hw2 = hw + kSet;
    double o[GAPS_NOBS];
    for (int q = 0; q < GAPS_NOBS; ++q) o[q] = 0.0;
    R ps[kMaxFinal][4];
    int np = E.npart[e];
    int m = 0;
    const bool pp = s_pp[row] != 0;
    double z0 = 0.0, z1 = 0.0, z2 = 0.0, z3 = 0.0;  // the colourless final state: Z, or e- e+
    for (int i = 0; i < np && m < kMaxFinal; ++i) {
      if (pp && i < 2) continue;
      const int fl = E.F(i, e);
      if (fl == 23 || fl == 11 || fl == -11) {
        z0 += E.P(0, i, e); z1 += E.P(1, i, e); z2 += E.P(2, i, e); z3 += E.P(3, i, e);
        continue;
      }
      if (sizeof(R) == 4 && pp) {
        const double en = E.P(0, i, e), pz = E.P(3, i, e);
        ps[m][0] = (R)(en + pz);
        ps[m][1] = (R)E.P(1, i, e);
        ps[m][2] = (R)E.P(2, i, e);
        ps[m][3] = (R)(en - pz);
      } else {
        for (int mu = 0; mu < 4; ++mu) ps[m][mu] = (R)E.P(mu, i, e);
      }
      ++m;
    }
    if (!pp) {
      o[0] = 1.0 - (double)thrust(ps, m);
      o[3] = (double)m;
      o[4] = (double)E.n_emit[e];
      R y23, y34;
      durham(ps, m, y23, y34);
      o[1] = y23;
      o[2] = y34;
    } else {
      double pt = sqrt(z1 * z1 + z2 * z2);
      o[0] = pt;
      o[1] = 0.5 * log((z0 + z3) / (z0 - z3));
      o[2] = pt > 0.0 ? atan2(z2, z1) : 0.0;
      o[6] = (double)m;
      o[7] = (double)E.n_emit[e];
      int cnt = 0;
      R lead = 0, lead_eta = 0;
      antikt(ps, m, R(0.4), cnt, lead, lead_eta);
      o[3] = (double)cnt;
      o[4] = lead;
      o[5] = lead_eta;
    }
    if (obs)
      for (int q = 0; q < GAPS_NOBS; ++q) obs[(uint64_t)q * E.cap + e] = o[q];
    if (fill && E.status[e] == GAPS_STATUS_DONE) {
      double w = E.weight[e];
      for (int h = 0; h < GAPS_NHIST; ++h) {
        int b = bin_of(H, h, o[H.obs[h]]);
        atomicAdd(&hw[h * GAPS_HIST_BINS + b], w);
        atomicAdd(&hw2[h * GAPS_HIST_BINS + b], w * w);
      }
    }
  }
  if (fill) {
    __syncthreads();
    for (int q = threadIdx.x; q < kSet * P.n_rows; q += blockDim.x) {
      const int r = q / kSet, k = q % kSet;
      const double a = sh[2 * kSet * r + k], b = sh[2 * kSet * r + kSet + k];
      if (a != 0.0) atomicAdd(&sumw[q], a);
      if (b != 0.0) atomicAdd(&sumw2[q], b);
    }
  }
}

}  // namespace

cudaError_t launch_observables(const DevParams& P, const DevEvents& E, uint64_t first, uint64_t n, double* obs,
                               const HistSet& H, double* sumw, double* sumw2, int fp32, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  int bs = 64;
  unsigned grid = (unsigned)((n + bs - 1) / bs);
  size_t shm = sumw ? 2 * (size_t)P.n_rows * GAPS_NHIST * GAPS_HIST_BINS * sizeof(double) : 0;
  if (fp32) k_observables<float><<<grid, bs, shm, stream>>>(P, E, first, n, obs, H, sumw, sumw2);
  else k_observables<double><<<grid, bs, shm, stream>>>(P, E, first, n, obs, H, sumw, sumw2);
  return cudaGetLastError();
}

}  // namespace gaps
