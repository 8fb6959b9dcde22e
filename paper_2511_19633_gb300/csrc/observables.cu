// Per-event observables (Section 4.1 of arXiv:2511.19633; e+e- event shapes
// as in GAPS 1) and weighted histograms. Each warp takes groups of 32
// events: per-event scalar work (the colourless final state, the boson
// kinematics, the output and the histogram bins) runs with one lane per
// event; the clusterings run one event at a time with the event's final-state
// momenta in the warp's shared memory and the lanes sharing the pair scans and
// the thrust candidates. Every value is formed with the same operations, in
// the same order, as a plain one-thread evaluation, and every minimum is taken
// in the order of a plain scan (lowest index on ties), so the results do not
// depend on the number of lanes. Histograms are privatised per block in shared
// memory and merged with global atomics.
#include "physics_fp64.cuh"

namespace gaps {


namespace {

constexpr int kMaxFinal = 128;
constexpr int kObsWords = kMaxFinal / 32;
constexpr int kObsWarps = 8;  // warps per block, each on its own group of events
constexpr unsigned kFull = 0xffffffffu;
static_assert(GAPS_NOBS == 8, "the kernel writes eight observables per event");

// one warp's event: coloured final state (pseudo-jets), their anti-kT
// kinematics and nearest neighbours
template <typename R>
struct ObsWarp {
  R ps[kMaxFinal][4];
  R pt2[kMaxFinal], y[kMaxFinal], phi[kMaxFinal], nnd[kMaxFinal];
  int nnj[kMaxFinal];
  uint32_t am[kObsWords];  // remaining pseudo-jets (the pair scans index it by word)
};

template <typename R>
__device__ __forceinline__ R norm3(const R* p) {
  return sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
}

// warp-wide lexicographic minimum of (v, k); v is never NaN
template <typename R>
__device__ __forceinline__ void warp_argmin(R& v, int& k) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const R ov = __shfl_xor_sync(kFull, v, off);
    const int ok = __shfl_xor_sync(kFull, k, off);
    if (ov < v || (ov == v && ok < k)) { v = ov; k = ok; }
  }
}

template <typename R>
__device__ __forceinline__ R warp_fmax(R v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

// bits of word w of an index mask that stand for indices above i
__device__ __forceinline__ uint32_t above(int i, int w) {
  const int lo = 32 * w;
  if (i < lo) return kFull;
  if (i >= lo + 31) return 0u;
  return kFull << (i - lo + 1);
}

// thrust: all 2^(n-1) subsets for n <= 12 (total momentum is zero), otherwise
// the exact construction from candidate axes p_i x p_j with the four sign
// choices of i and j; the lanes share the candidates, the maximum is exact
template <typename R>
__device__ __forceinline__ R thrust(const ObsWarp<R>& W, int n, int lane) {
  R sum = 0;
  for (int i = 0; i < n; ++i) sum += norm3(W.ps[i]);
  if (n < 2 || !(sum > R(0))) return R(1);
  R best = 0;
  if (n <= 12) {
    for (uint32_t m = lane; m < (1u << (n - 1)); m += 32) {
      R v0 = 0, v1 = 0, v2 = 0;
      for (int i = 0; i < n; ++i)
        if ((m >> i) & 1u) { v0 += W.ps[i][1]; v1 += W.ps[i][2]; v2 += W.ps[i][3]; }
      R l = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      best = fmax(best, l);
    }
  } else {
    for (int i = 0; i < n; ++i) {
      for (int j = i + 1 + lane; j < n; j += 32) {
        const R* pi = W.ps[i];
        const R* pj = W.ps[j];
        R ax0 = pi[2] * pj[3] - pi[3] * pj[2];
        R ax1 = pi[3] * pj[1] - pi[1] * pj[3];
        R ax2 = pi[1] * pj[2] - pi[2] * pj[1];
        R b0 = 0, b1 = 0, b2 = 0;
        for (int k = 0; k < n; ++k) {
          if (k == i || k == j) continue;
          R d = W.ps[k][1] * ax0 + W.ps[k][2] * ax1 + W.ps[k][3] * ax2;
          if (d > R(0)) { b0 += W.ps[k][1]; b1 += W.ps[k][2]; b2 += W.ps[k][3]; }
        }
        for (int si = 0; si < 2; ++si) {
          for (int sj = 0; sj < 2; ++sj) {
            R v0 = b0, v1 = b1, v2 = b2;
            if (si) { v0 += pi[1]; v1 += pi[2]; v2 += pi[3]; }
            if (sj) { v0 += pj[1]; v1 += pj[2]; v2 += pj[3]; }
            R l = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
            best = fmax(best, l);
          }
        }
      }
    }
  }
  best = warp_fmax(best);
  return R(2) * best / sum;
}

// Durham clustering, E-scheme; y23, y34 = smallest y_ij when 3 -> 2, 4 -> 3.
// Each step takes the smallest y_ij over the remaining pairs in row-major
// order of the pair (lowest i, then lowest j, on ties); a merged pair keeps
// the slot of i, and j leaves.
template <typename R>
__device__ __forceinline__ void durham(ObsWarp<R>& W, int m, int lane, R& y23, R& y34) {
  R evis = 0;
  for (int i = 0; i < m; ++i) evis += W.ps[i][0];
  y23 = 0; y34 = 0;
  if (lane < kObsWords)
    W.am[lane] = m >= 32 * (lane + 1) ? kFull : (m > 32 * lane ? (1u << (m - 32 * lane)) - 1u : 0u);
  __syncwarp();
  while (m > 1) {
    R ymin = R(INFINITY);
    int key = INT_MAX;
#pragma unroll
    for (int k = 0; k < kObsWords; ++k) {
      const int i = 32 * k + lane;
      if (!((W.am[k] >> lane) & 1u)) continue;
      const R ni = norm3(W.ps[i]);
      for (int w = i >> 5; w < kObsWords; ++w) {
        uint32_t bits = W.am[w] & above(i, w);
        while (bits) {
          const int j = 32 * w + __ffs(bits) - 1;
          bits &= bits - 1;
          R nj = norm3(W.ps[j]);
          R omc;  // 1 - cos(theta_ij)
          if constexpr (sizeof(R) == 8) {
            omc = R(1) - (W.ps[i][1] * W.ps[j][1] + W.ps[i][2] * W.ps[j][2] + W.ps[i][3] * W.ps[j][3]) / (ni * nj);
          } else {
            // |n_i - n_j|^2 / 2 keeps the relative precision for collinear pairs
            R d0 = W.ps[i][1] / ni - W.ps[j][1] / nj, d1 = W.ps[i][2] / ni - W.ps[j][2] / nj,
              d2 = W.ps[i][3] / ni - W.ps[j][3] / nj;
            omc = R(0.5) * (d0 * d0 + d1 * d1 + d2 * d2);
          }
          R emin = fmin(W.ps[i][0], W.ps[j][0]);
          R yij = R(2) * emin * emin * omc / (evis * evis);
          if (yij < ymin) { ymin = yij; key = i * kMaxFinal + j; }
        }
      }
    }
    warp_argmin(ymin, key);
    if (key == INT_MAX) break;  // no finite y_ij (degenerate momenta)
    const int bi = key / kMaxFinal, bj = key % kMaxFinal;
    if (m == 3) y23 = ymin;
    if (m == 4) y34 = ymin;
    __syncwarp();
    if (lane < 4) W.ps[bi][lane] += W.ps[bj][lane];
    if (lane == 0) W.am[bj >> 5] &= ~(1u << (bj & 31));
    m -= 1;
    __syncwarp();
  }
}

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

// nearest remaining neighbour of i among j > i (lowest j on ties)
template <typename R>
__device__ __forceinline__ void akt_nn(ObsWarp<R>& W, int i, R R2) {
  R best = R(INFINITY);
  int bj = -1;
  for (int w = i >> 5; w < kObsWords; ++w) {
    uint32_t bits = W.am[w] & above(i, w);
    while (bits) {
      const int j = 32 * w + __ffs(bits) - 1;
      bits &= bits - 1;
      R d = akt_dij(W.pt2, W.y, W.phi, i, j, R2);
      if (d < best) { best = d; bj = j; }
    }
  }
  W.nnd[i] = best;
  W.nnj[i] = bj;
}

// anti-kT R (Cacciari, Salam, Soyez 2008), E-scheme, rapidity-azimuth
// distance, over the m0 pseudo-jets of W.ps (those with zero transverse
// momentum are left out). Nearest-neighbour bookkeeping (O(n^2)): every
// remaining pseudo-jet keeps its nearest neighbour among the later ones, and
// each step takes the smallest of all beam and neighbour distances in the
// order of a full scan (beam distance of i, then its neighbour, i ascending),
// so the clustering sequence equals the brute-force one. Reports the number
// of jets with pT > 5 GeV and |eta| < 5 and the leading one's pT and eta.
template <typename R>
__device__ __forceinline__ void antikt(ObsWarp<R>& W, int m0, int lane, R Rj, int& njets, R& lead, R& lead_eta) {
  int m = 0;
#pragma unroll
  for (int k = 0; k < kObsWords; ++k) {
    const int i = 32 * k + lane;
    const bool keep = i < m0 && W.ps[i][1] * W.ps[i][1] + W.ps[i][2] * W.ps[i][2] > R(0);
    const uint32_t bits = __ballot_sync(kFull, keep);
    m += __popc(bits);
    if (keep) jet_kin(W.ps[i], W.pt2[i], W.y[i], W.phi[i]);
    if (lane == 0) W.am[k] = bits;
  }
  const R R2 = Rj * Rj;
  __syncwarp();
#pragma unroll
  for (int k = 0; k < kObsWords; ++k)
    if ((W.am[k] >> lane) & 1u) akt_nn(W, 32 * k + lane, R2);
  __syncwarp();
  njets = 0;
  lead = 0;
  lead_eta = 0;
  while (m > 0) {
    R dmin = R(INFINITY);
    int key = INT_MAX;  // 2 i for the beam distance of i, 2 i + 1 for its neighbour
#pragma unroll
    for (int k = 0; k < kObsWords; ++k) {
      if (!((W.am[k] >> lane) & 1u)) continue;
      const int i = 32 * k + lane;
      R diB = R(1) / W.pt2[i];
      if (diB < dmin) { dmin = diB; key = 2 * i; }
      if (W.nnd[i] < dmin) { dmin = W.nnd[i]; key = 2 * i + 1; }
    }
    warp_argmin(dmin, key);
    if (key == INT_MAX) break;  // no finite distance (cannot happen for pT > 0)
    const int bi = key >> 1;
    const int bj = (key & 1) ? W.nnj[bi] : -1;
    int gone;
    __syncwarp();
    if (bj < 0) {
      R jpt = sqrt(W.ps[bi][1] * W.ps[bi][1] + W.ps[bi][2] * W.ps[bi][2]);
      R jeta = asinh(jet_pz(W.ps[bi]) / jpt);
      if (jpt > R(5) && fabs(jeta) < R(5)) {
        njets += 1;
        if (jpt > lead) { lead = jpt; lead_eta = jeta; }
      }
      gone = bi;
    } else {
      if (lane < 4) W.ps[bi][lane] += W.ps[bj][lane];
      __syncwarp();
      if (lane == 0) jet_kin(W.ps[bi], W.pt2[bi], W.y[bi], W.phi[bi]);
      gone = bj;
    }
    if (lane == 0) W.am[gone >> 5] &= ~(1u << (gone & 31));
    m -= 1;
    __syncwarp();
    // refresh the neighbours that pointed at a changed or removed pseudo-jet
#pragma unroll
    for (int k = 0; k < kObsWords; ++k) {
      if (!((W.am[k] >> lane) & 1u)) continue;
      const int i = 32 * k + lane;
      const int nj = W.nnj[i];
      const bool stale = (bj >= 0 && (i == bi || nj == bi)) || nj == gone;
      if (bj >= 0 && i < bi && !stale) {
        // a merged pseudo-jet may become i's nearest neighbour, or displace one
        R d = akt_dij(W.pt2, W.y, W.phi, i, bi, R2);
        if (d < W.nnd[i] || (d == W.nnd[i] && bi < nj)) { W.nnd[i] = d; W.nnj[i] = bi; }
      }
      if (stale) akt_nn(W, i, R2);
    }
    __syncwarp();
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

// R = double for per-event parity (GAPS_FP64), float for mixed-precision
// contexts. Each warp takes groups of 32 consecutive events (group g of the
// grid's warps, then steps by their count). Per group: the lanes scan their
// own events' records for the colourless final state (lane = event), the
// warp clusters the events one after the other (lane = pseudo-jet), and the
// lanes form, write and histogram their events' observables (lane = event),
// so the per-event FP64 work (boson kinematics, binning) runs once per event.
template <typename R>
__global__ void __launch_bounds__(kObsWarps * 32, sizeof(R) == 4 ? 4 : 2)
    k_observables(DevParams P, DevEvents E, uint64_t first, uint64_t n, double* obs, HistSet Hs, double* sumw,
                  double* sumw2) {
  // shared: the warps' events, then per row of the batch sumw and sumw2
  // [GAPS_NHIST][GAPS_HIST_BINS]
  extern __shared__ __align__(16) unsigned char obs_smem[];
  ObsWarp<R>* Wa = reinterpret_cast<ObsWarp<R>*>(obs_smem);
  double* sh = reinterpret_cast<double*>(Wa + kObsWarps);
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
  const int lane = threadIdx.x & 31;
  ObsWarp<R>& W = Wa[threadIdx.x >> 5];
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t stride = (uint64_t)gridDim.x * kObsWarps * 32;
  for (uint64_t g0 = ((uint64_t)blockIdx.x * kObsWarps + (threadIdx.x >> 5)) * 32; g0 < n; g0 += stride) {
    // --- lane = event: the colourless final state (Z, or e- e+) and the
    // number of coloured partons, in a plain scan of the record that stops
    // at the kMaxFinal-th coloured parton
    const uint64_t el = g0 + lane;
    const bool live = el < n;
    int row = 0, np = 0, mc = 0;
    bool pp = false;
    double z0 = 0.0, z1 = 0.0, z2 = 0.0, z3 = 0.0;
    if (live) {
      row = mix_row(P, first + el);
      pp = s_pp[row] != 0;
      np = E.npart[el];
      for (int i = pp ? 2 : 0; i < np && mc < kMaxFinal; ++i) {
        const int fl = E.F(i, el);
        if (fl == 23 || fl == 11 || fl == -11) {
          z0 += E.P(0, i, el); z1 += E.P(1, i, el); z2 += E.P(2, i, el); z3 += E.P(3, i, el);
        } else {
          ++mc;
        }
      }
    }
    // --- lane = pseudo-jet: cluster the group's events one by one; lane k
    // keeps event k's results
    R ra = 0, rb = 0, rc = 0;
    int rn = 0;
    const int ng = n - g0 < 32 ? (int)(n - g0) : 32;
    for (int k = 0; k < ng; ++k) {
      const uint64_t e = g0 + k;
      const bool ppk = __shfl_sync(kFull, (int)pp, k) != 0;
      const int npk = __shfl_sync(kFull, np, k);
      int m = 0;
      for (int base = ppk ? 2 : 0; base < npk && m < kMaxFinal; base += 32) {
        const int i = base + lane;
        int fl = 0;
        if (i < npk) fl = E.F(i, e);
        const bool coloured = i < npk && !(fl == 23 || fl == 11 || fl == -11);
        const uint32_t cm = __ballot_sync(kFull, coloured);
        const int at = m + __popc(cm & lt);
        if (coloured && at < kMaxFinal) {
          R* q = W.ps[at];
          if (sizeof(R) == 4 && ppk) {
            const double en = E.P(0, i, e), pz = E.P(3, i, e);
            q[0] = (R)(en + pz);
            q[1] = (R)E.P(1, i, e);
            q[2] = (R)E.P(2, i, e);
            q[3] = (R)(en - pz);
          } else {
            for (int mu = 0; mu < 4; ++mu) q[mu] = (R)E.P(mu, i, e);
          }
        }
        m = min(m + __popc(cm), kMaxFinal);
      }
      __syncwarp();
      R a, b, c;
      int cnt = 0;
      if (!ppk) {
        a = thrust(W, m, lane);
        durham(W, m, lane, b, c);
      } else {
        antikt(W, m, lane, R(0.4), cnt, a, b);
        c = 0;
      }
      if (lane == k) { ra = a; rb = b; rc = c; rn = cnt; }
      __syncwarp();
    }
    if (!live) continue;
    // --- lane = event: observables, their output and the histograms (the
    // observables stay in named registers: an array picked by H.obs[h] would
    // be placed in local memory)
    const double nem = (double)E.n_emit[el];
    double o0, o1, o2, o3, o4, o5 = 0.0, o6 = 0.0, o7 = 0.0;
    if (!pp) {
      o0 = 1.0 - (double)ra;
      o1 = rb;
      o2 = rc;
      o3 = (double)mc;
      o4 = nem;
    } else {
      double pt = sqrt(z1 * z1 + z2 * z2);
      o0 = pt;
      o1 = 0.5 * log((z0 + z3) / (z0 - z3));
      o2 = pt > 0.0 ? atan2(z2, z1) : 0.0;
      o3 = (double)rn;
      o4 = ra;
      o5 = rb;
      o6 = (double)mc;
      o7 = nem;
    }
    if (obs) {
      double* out = obs + el;
      const uint64_t c = E.cap;
      out[0] = o0; out[c] = o1; out[2 * c] = o2; out[3 * c] = o3;
      out[4 * c] = o4; out[5 * c] = o5; out[6 * c] = o6; out[7 * c] = o7;
    }
    if (fill && E.status[el] == GAPS_STATUS_DONE) {
      const HistDef& H = sH[row];
      double* hw = sh + 2 * kSet * row;
      double* hw2 = hw + kSet;
      const double w = E.weight[el];
#pragma unroll
      for (int h = 0; h < GAPS_NHIST; ++h) {
        const int oi = H.obs[h];
        const double v = oi == 0 ? o0 : oi == 1 ? o1 : oi == 2 ? o2 : oi == 3 ? o3
                       : oi == 4 ? o4 : oi == 5 ? o5 : oi == 6 ? o6 : o7;
        const int bin = bin_of(H, h, v);
        atomicAdd(&hw[h * GAPS_HIST_BINS + bin], w);
        atomicAdd(&hw2[h * GAPS_HIST_BINS + bin], w * w);
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

template <typename R>
size_t observables_smem(int n_rows, bool fill) {
  return kObsWarps * sizeof(ObsWarp<R>) +
         (fill ? 2 * (size_t)n_rows * GAPS_NHIST * GAPS_HIST_BINS * sizeof(double) : 0);
}

}  // namespace

// Opt-in for the observables kernels' dynamic shared memory (the warps'
// events and a mixed batch's histograms); called when a context is created.
cudaError_t observables_init() {
  cudaError_t e = cudaFuncSetAttribute(k_observables<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)observables_smem<float>(kMaxRows, true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_observables<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)observables_smem<double>(kMaxRows, true));
  return e;
}

cudaError_t launch_observables(const DevParams& P, const DevEvents& E, uint64_t first, uint64_t n, double* obs,
                               const HistSet& H, double* sumw, double* sumw2, int fp32, int sm_count,
                               cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const uint64_t blocks_needed = (n + 32 * kObsWarps - 1) / (32 * kObsWarps);
  const uint64_t resident = (uint64_t)max(1, sm_count) * (fp32 ? 4 : 2);
  const unsigned grid = (unsigned)min(blocks_needed, resident);
  const bool fill = sumw != nullptr;
  if (fp32)
    k_observables<float><<<grid, kObsWarps * 32, observables_smem<float>(P.n_rows, fill), stream>>>(
        P, E, first, n, obs, H, sumw, sumw2);
  else
    k_observables<double><<<grid, kObsWarps * 32, observables_smem<double>(P.n_rows, fill), stream>>>(
        P, E, first, n, obs, H, sumw, sumw2);
  return cudaGetLastError();
}

}  // namespace gaps
