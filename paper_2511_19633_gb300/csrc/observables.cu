// Per-event observables (Section 4.1 of arXiv:2511.19633; e+e- event shapes
// as in GAPS 1) and weighted histograms. One thread per event; the clustering
// works on a thread-local copy of the final-state momenta. Histograms are
// privatised per block in shared memory and merged with global atomics.
#include "physics_fp64.cuh"

namespace gaps {


namespace {

constexpr int kMaxFinal = 128;

__device__ __forceinline__ double norm3(const double* p) {
  return sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
}

// thrust: all 2^(n-1) subsets for n <= 12 (total momentum is zero), otherwise
// the exact construction from candidate axes p_i x p_j with the four sign
// choices of i and j
__device__ double thrust(const double (*ps)[4], int n) {
  double sum = 0.0;
  for (int i = 0; i < n; ++i) sum += norm3(ps[i]);
  if (n < 2 || !(sum > 0.0)) return 1.0;
  double best = 0.0;
  if (n <= 12) {
    for (uint32_t m = 0; m < (1u << (n - 1)); ++m) {
      double v0 = 0.0, v1 = 0.0, v2 = 0.0;
      for (int i = 0; i < n; ++i)
        if ((m >> i) & 1u) { v0 += ps[i][1]; v1 += ps[i][2]; v2 += ps[i][3]; }
      double l = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      best = fmax(best, l);
    }
  } else {
    for (int i = 0; i < n; ++i) {
      for (int j = i + 1; j < n; ++j) {
        double ax0 = ps[i][2] * ps[j][3] - ps[i][3] * ps[j][2];
        double ax1 = ps[i][3] * ps[j][1] - ps[i][1] * ps[j][3];
        double ax2 = ps[i][1] * ps[j][2] - ps[i][2] * ps[j][1];
        double b0 = 0.0, b1 = 0.0, b2 = 0.0;
        for (int k = 0; k < n; ++k) {
          if (k == i || k == j) continue;
          double d = ps[k][1] * ax0 + ps[k][2] * ax1 + ps[k][3] * ax2;
          if (d > 0.0) { b0 += ps[k][1]; b1 += ps[k][2]; b2 += ps[k][3]; }
        }
        for (int si = 0; si < 2; ++si) {
          for (int sj = 0; sj < 2; ++sj) {
            double v0 = b0, v1 = b1, v2 = b2;
            if (si) { v0 += ps[i][1]; v1 += ps[i][2]; v2 += ps[i][3]; }
            if (sj) { v0 += ps[j][1]; v1 += ps[j][2]; v2 += ps[j][3]; }
            double l = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
            best = fmax(best, l);
          }
        }
      }
    }
  }
  return 2.0 * best / sum;
}

__device__ __forceinline__ void erase(double (*ps)[4], int& m, int at) {
  for (int q = at; q < m - 1; ++q)
    for (int mu = 0; mu < 4; ++mu) ps[q][mu] = ps[q + 1][mu];
  m -= 1;
}

// Durham clustering, E-scheme; y23, y34 = smallest y_ij when 3 -> 2, 4 -> 3
__device__ void durham(double (*ps)[4], int m, double& y23, double& y34) {
  double evis = 0.0;
  for (int i = 0; i < m; ++i) evis += ps[i][0];
  y23 = 0.0; y34 = 0.0;
  while (m > 1) {
    double ymin = __longlong_as_double(0x7ff0000000000000ll);
    int bi = -1, bj = -1;
    for (int i = 0; i < m; ++i) {
      for (int j = i + 1; j < m; ++j) {
        double ni = norm3(ps[i]), nj = norm3(ps[j]);
        double cth = (ps[i][1] * ps[j][1] + ps[i][2] * ps[j][2] + ps[i][3] * ps[j][3]) / (ni * nj);
        double emin = fmin(ps[i][0], ps[j][0]);
        double y = 2.0 * emin * emin * (1.0 - cth) / (evis * evis);
        if (y < ymin) { ymin = y; bi = i; bj = j; }
      }
    }
    if (m == 3) y23 = ymin;
    if (m == 4) y34 = ymin;
    for (int mu = 0; mu < 4; ++mu) ps[bi][mu] += ps[bj][mu];
    erase(ps, m, bj);
  }
}

__device__ __forceinline__ void jet_kin(const double* p, double& pt2, double& y, double& phi) {
  pt2 = p[1] * p[1] + p[2] * p[2];
  y = 0.5 * log((p[0] + p[3]) / (p[0] - p[3]));
  phi = atan2(p[2], p[1]);
}

// anti-kT R (Cacciari, Salam, Soyez 2008), E-scheme; jets written over ps,
// returns their number
__device__ int antikt(double (*ps)[4], int m, double R, double (*jets)[4]) {
  // drop particles without transverse momentum
  int w = 0;
  for (int i = 0; i < m; ++i) {
    if (ps[i][1] * ps[i][1] + ps[i][2] * ps[i][2] > 0.0) {
      for (int mu = 0; mu < 4; ++mu) ps[w][mu] = ps[i][mu];
      ++w;
    }
  }
  m = w;
  int nj = 0;
  const double kPiL = kPi;
  while (m > 0) {
    double dmin = __longlong_as_double(0x7ff0000000000000ll);
    int bi = -1, bj = -1;
    for (int i = 0; i < m; ++i) {
      double pti2, yi, phii;
      jet_kin(ps[i], pti2, yi, phii);
      double diB = 1.0 / pti2;
      if (diB < dmin) { dmin = diB; bi = i; bj = -1; }
      for (int j = i + 1; j < m; ++j) {
        double ptj2, yj, phij;
        jet_kin(ps[j], ptj2, yj, phij);
        double dphi = fabs(phii - phij);
        if (dphi > kPiL) dphi = 2.0 * kPiL - dphi;
        double dr2 = (yi - yj) * (yi - yj) + dphi * dphi;
        double dij = fmin(1.0 / pti2, 1.0 / ptj2) * dr2 / (R * R);
        if (dij < dmin) { dmin = dij; bi = i; bj = j; }
      }
    }
    if (bj < 0) {
      for (int mu = 0; mu < 4; ++mu) jets[nj][mu] = ps[bi][mu];
      ++nj;
      erase(ps, m, bi);
    } else {
      for (int mu = 0; mu < 4; ++mu) ps[bi][mu] += ps[bj][mu];
      erase(ps, m, bj);
    }
  }
  return nj;
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

__global__ void k_observables(DevParams P, DevEvents E, uint64_t n, double* obs, HistDef H,
                              double* sumw, double* sumw2) {
  extern __shared__ double sh[];
  double* hw = sh;
  double* hw2 = sh + GAPS_NHIST * GAPS_HIST_BINS;
  const bool fill = sumw != nullptr;
  if (fill) {
    for (int q = threadIdx.x; q < 2 * GAPS_NHIST * GAPS_HIST_BINS; q += blockDim.x) sh[q] = 0.0;
    __syncthreads();
  }
  uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    double o[GAPS_NOBS];
    for (int q = 0; q < GAPS_NOBS; ++q) o[q] = 0.0;
    double ps[kMaxFinal][4];
    double jets[kMaxFinal][4];
    int np = E.npart[e];
    int m = 0;
    bool pp = P.process != GAPS_EE_QQ;
    for (int i = 0; i < np && m < kMaxFinal; ++i) {
      if (pp && i < 2) continue;
      if (E.F(i, e) == 23) continue;
      for (int mu = 0; mu < 4; ++mu) ps[m][mu] = E.P(mu, i, e);
      ++m;
    }
    if (!pp) {
      o[0] = 1.0 - thrust(ps, m);
      o[3] = (double)m;
      o[4] = (double)E.n_emit[e];
      durham(ps, m, o[1], o[2]);
    } else {
      double z0 = E.P(0, 2, e), z1 = E.P(1, 2, e), z2 = E.P(2, 2, e), z3 = E.P(3, 2, e);
      double pt = sqrt(z1 * z1 + z2 * z2);
      o[0] = pt;
      o[1] = 0.5 * log((z0 + z3) / (z0 - z3));
      o[2] = pt > 0.0 ? atan2(z2, z1) : 0.0;
      o[6] = (double)m;
      o[7] = (double)E.n_emit[e];
      int nj = antikt(ps, m, 0.4, jets);
      int cnt = 0;
      double lead = 0.0, lead_eta = 0.0;
      for (int q = 0; q < nj; ++q) {
        double jpt = sqrt(jets[q][1] * jets[q][1] + jets[q][2] * jets[q][2]);
        double jeta = asinh(jets[q][3] / jpt);
        if (jpt > 5.0 && fabs(jeta) < 5.0) {
          cnt += 1;
          if (jpt > lead) { lead = jpt; lead_eta = jeta; }
        }
      }
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
    for (int q = threadIdx.x; q < GAPS_NHIST * GAPS_HIST_BINS; q += blockDim.x) {
      if (hw[q] != 0.0) atomicAdd(&sumw[q], hw[q]);
      if (hw2[q] != 0.0) atomicAdd(&sumw2[q], hw2[q]);
    }
  }
}

}  // namespace

cudaError_t launch_observables(const DevParams& P, const DevEvents& E, uint64_t n, double* obs,
                               const HistDef& H, double* sumw, double* sumw2, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  int bs = 64;
  unsigned grid = (unsigned)((n + bs - 1) / bs);
  size_t shm = sumw ? 2 * GAPS_NHIST * GAPS_HIST_BINS * sizeof(double) : 0;
  k_observables<<<grid, bs, shm, stream>>>(P, E, n, obs, H, sumw, sumw2);
  return cudaGetLastError();
}

}  // namespace gaps
