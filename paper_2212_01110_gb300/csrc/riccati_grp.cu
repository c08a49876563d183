// Chain-region Riccati passes with three cooperating warps per chain.
//
// Same data flow as the staged chain kernels (each chain step's factors are
// copied into shared memory one step ahead by bulk asynchronous copies, two
// stage buffers per chain), but the GEMVs of a step are split over the three
// warps of the chain's group -- columns of [Abar | B]^T q, then d, then the
// rows of q (backward); the rows of x^c and the entries of u (forward) --
// with a named barrier between phases.  One warp per chain left each SM
// sub-partition issuing from a single instruction stream (issue-bound at
// about 2,000 instructions per step); three warps cut that per-warp stream
// by three at the same shared-memory footprint, and put FP64 work on every
// sub-partition.
#include <algorithm>

#include "kernels.cuh"
#include "spock_internal.h"
#include "tma.cuh"

namespace spock {

constexpr int kGrpWarps = 3;
constexpr int kGrpThreads = 32 * kGrpWarps;
constexpr int kMaxGroups = 4;

template <typename S>
struct GrpLayout {
  uint32_t gB, nbB, xB, uB, ktB, stageB, groupB;
};

template <typename S>
__host__ __device__ inline GrpLayout<S> grp_layout_bwd(const KP<S>& p) {
  GrpLayout<S> L;
  L.gB = p.gstride * sizeof(S);
  L.nbB = p.nbstride * sizeof(S);
  L.xB = p.xs * sizeof(S);
  L.uB = p.us * sizeof(S);
  L.ktB = p.ktstride * sizeof(S);
  L.stageB = L.gB + L.nbB + 2 * L.xB + L.uB;  // G | NB | xbar_k | ubar_k | xbar_leaf
  L.groupB = 2 * L.stageB + 3 * kVecPad * sizeof(S) + 16;
  return L;
}
template <typename S>
__host__ __device__ inline GrpLayout<S> grp_layout_fwd(const KP<S>& p) {
  GrpLayout<S> L;
  L.gB = p.gstride * sizeof(S);
  L.nbB = p.nbstride * sizeof(S);
  L.xB = p.xs * sizeof(S);
  L.uB = p.us * sizeof(S);
  L.ktB = p.ktstride * sizeof(S);
  L.stageB = L.ktB + L.gB + L.uB;  // Kt | Gf | d_k
  L.groupB = 2 * L.stageB + 2 * kVecPad * sizeof(S) + 16;
  return L;
}

// Group-uniform bounded wait: every thread polls; the outcome is agreed on
// through shared memory so that all warps of the group take the same path.
__device__ __forceinline__ bool grp_wait(uint64_t* bar, uint32_t parity, int* vote, int sub, int lane, int bar_id) {
  const bool ok = __all_sync(kFull, mbar_wait(bar, parity));
  if (lane == 0) vote[sub] = ok ? 1 : 0;
  named_bar(bar_id, kGrpThreads);
  const bool all = vote[0] && vote[1] && vote[2];
  named_bar(bar_id, kGrpThreads);  // votes read before they are rewritten
  return all;
}

template <typename S, int SLG>
__global__ void __launch_bounds__(kGrpThreads* kMaxGroups) k_bwd_chain_grp(KP<S> p) {
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxGroups][2];
  __shared__ int votes[kMaxGroups][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = w / kGrpWarps, sub = w % kGrpWarps;
  const int ngb = blockDim.x / kGrpThreads;
  const int gg = blockIdx.x * ngb + g, ng = gridDim.x * ngb;
  const int bar_id = 1 + g;
  const int nx = p.nx, nu = p.nu, ncol = nx + nu;
  const GrpLayout<S> Ly = grp_layout_bwd(p);
  unsigned char* base = smem + (size_t)g * Ly.groupB;
  S* stg[2] = {reinterpret_cast<S*>(base), reinterpret_cast<S*>(base + Ly.stageB)};
  S* vq = reinterpret_cast<S*>(base + 2 * Ly.stageB);
  S* vh = vq + kVecPad;
  S* vd = vh + kVecPad;
  uint64_t* bar = bars[g];
  const bool leader = (sub == 0 && lane == 0);
  if (leader) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  named_bar(bar_id, kGrpThreads);
  const int Lc = p.N - p.chain_stage;
  const int nch = gg < p.n_chains ? (p.n_chains - gg + ng - 1) / ng : 0;
  const int nsteps = nch * Lc;
  auto issue = [&](int j) {
    const int ci = gg + (j / Lc) * ng;
    const int t = p.N - 1 - (j % Lc);
    const int k = p.stage_begin[t] + ci, c = p.stage_begin[t + 1] + ci;
    S* dst = stg[j & 1];
    const bool first = (t == p.N - 1);
    fence_proxy_async();
    mbar_expect_tx(&bar[j & 1], Ly.gB + Ly.nbB + Ly.xB + Ly.uB + (first ? Ly.xB : 0u));
    bulk_g2s(dst, p.Gb + (int64_t)(c - 1) * p.gstride, Ly.gB, &bar[j & 1]);
    bulk_g2s(dst + p.gstride, p.NB + (int64_t)k * p.nbstride, Ly.nbB, &bar[j & 1]);
    bulk_g2s(dst + p.gstride + p.nbstride, p.xbar + (int64_t)k * p.xs, Ly.xB, &bar[j & 1]);
    bulk_g2s(dst + p.gstride + p.nbstride + p.xs, p.ubar + (int64_t)k * p.us, Ly.uB, &bar[j & 1]);
    if (first) bulk_g2s(dst + p.gstride + p.nbstride + p.xs + p.us, p.xbar + (int64_t)c * p.xs, Ly.xB, &bar[j & 1]);
  };
  uint32_t phase0 = 0, phase1 = 0;
  if (nsteps > 0 && leader) issue(0);
  for (int j = 0; j < nsteps; ++j) {
    const int ci = gg + (j / Lc) * ng;
    const int t = p.N - 1 - (j % Lc);
    const int k = p.stage_begin[t] + ci;
    if (j + 1 < nsteps && leader) issue(j + 1);
    uint32_t& ph = (j & 1) ? phase1 : phase0;
    const uint32_t par = ph;
    const bool ok = grp_wait(&bar[j & 1], par, votes[g], sub, lane, bar_id);
    ph ^= 1u;
    if (!ok) {  // flag, drain the group's copies in flight (bounded), leave together
      if (leader) {
        atomicExch(p.err, 1);
        mbar_wait(&bar[j & 1], par);
        if (j + 1 < nsteps) mbar_wait(&bar[(j + 1) & 1], (j & 1) ? phase0 : phase1);
      }
      return;
    }
    const S* G = stg[j & 1];
    const S* NBk = G + p.gstride;
    const S* xb = NBk + p.nbstride;
    const S* ub = xb + p.xs;
    if (t == p.N - 1) {
      const S* xl = ub + p.us;
      for (int r = sub * 32 + lane; r < nx; r += kGrpThreads) vq[r] = -xl[r];
      named_bar(bar_id, kGrpThreads);
    }
    // phase A: h = [Abar | B]^T q, columns split over the three warps
    {
      S h[SLG];
#pragma unroll
      for (int s = 0; s < SLG; ++s) h[s] = S(0);
#pragma unroll 4
      for (int r = 0; r < nx; ++r) {
        const S qr = vq[r];
        const S* row = G + r * ncol;
#pragma unroll
        for (int s = 0; s < SLG; ++s) {
          const int col = sub * 32 + lane + s * kGrpThreads;
          if (col < ncol) h[s] += row[col] * qr;
        }
      }
#pragma unroll
      for (int s = 0; s < SLG; ++s) {
        const int col = sub * 32 + lane + s * kGrpThreads;
        if (col < ncol) vh[col] = h[s];
      }
    }
    named_bar(bar_id, kGrpThreads);
    // phase B: d = Rt^-1 (ubar - B^T q)
    {
      const S* Ri = NBk + 2 * nu * nx;  // symmetric: read column-wise
      for (int a = sub * 32 + lane; a < nu; a += kGrpThreads) {
        S acc = 0;
        for (int b = 0; b < nu; ++b) acc += Ri[b * nu + a] * (ub[b] - vh[nx + b]);
        vd[a] = acc;
        p.d[(int64_t)k * p.us + a] = acc;
      }
    }
    named_bar(bar_id, kGrpThreads);
    // phase C: q = K^T (d - ubar) + W d - xbar + Abar^T q = C^T d - K^T ubar - xbar
    // + Abar^T q (C = K + W^T), rows split over the warps
    {
      const S* Km = NBk;
      const S* Cm = NBk + nu * nx;
      S qn[SLG];
#pragma unroll
      for (int s = 0; s < SLG; ++s) {
        const int r = sub * 32 + lane + s * kGrpThreads;
        qn[s] = (r < nx) ? vh[r] - xb[r] : S(0);
      }
#pragma unroll 4
      for (int b = 0; b < nu; ++b) {
        const S db = vd[b];
        const S u = ub[b];
        const S* kr = Km + b * nx;
        const S* cr = Cm + b * nx;
#pragma unroll
        for (int s = 0; s < SLG; ++s) {
          const int r = sub * 32 + lane + s * kGrpThreads;
          if (r < nx) qn[s] = fma(-kr[r], u, fma(cr[r], db, qn[s]));   // two FMAs, no add
        }
      }
      // every warp has finished reading vq in phase A (barrier above)
#pragma unroll
      for (int s = 0; s < SLG; ++s) {
        const int r = sub * 32 + lane + s * kGrpThreads;
        if (r < nx) {
          vq[r] = qn[s];
          if (t == p.chain_stage) p.q[(int64_t)k * p.xs + r] = qn[s];
        }
      }
    }
    named_bar(bar_id, kGrpThreads);  // stage j&1 free, vq complete
  }
}

template <typename S, int SLG>
__global__ void __launch_bounds__(kGrpThreads* kMaxGroups) k_fwd_chain_grp(KP<S> p, S* __restrict__ zo) {
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxGroups][2];
  __shared__ int votes[kMaxGroups][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = w / kGrpWarps, sub = w % kGrpWarps;
  const int ngb = blockDim.x / kGrpThreads;
  const int gg = blockIdx.x * ngb + g, ng = gridDim.x * ngb;
  const int bar_id = 1 + g;
  const int nx = p.nx, nu = p.nu, ncol = nx + nu;
  const GrpLayout<S> Ly = grp_layout_fwd(p);
  unsigned char* base = smem + (size_t)g * Ly.groupB;
  S* stg[2] = {reinterpret_cast<S*>(base), reinterpret_cast<S*>(base + Ly.stageB)};
  S* vw = reinterpret_cast<S*>(base + 2 * Ly.stageB);  // (x; d)
  uint64_t* bar = bars[g];
  const bool leader = (sub == 0 && lane == 0);
  if (leader) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  named_bar(bar_id, kGrpThreads);
  const int Lc = p.N - p.chain_stage;
  const int nch = gg < p.n_chains ? (p.n_chains - gg + ng - 1) / ng : 0;
  const int nsteps = nch * Lc;
  // output slots of 32: [0, xslots) rows of x^c, then entries of u^k; slot i
  // belongs to warp i % 3, so every warp runs one kind of loop per slot
  const int xslots = (nx + 31) / 32, nslots = xslots + (nu + 31) / 32;
  auto issue = [&](int j) {
    const int ci = gg + (j / Lc) * ng;
    const int t = p.chain_stage + (j % Lc);
    const int k = p.stage_begin[t] + ci, c = p.stage_begin[t + 1] + ci;
    S* dst = stg[j & 1];
    fence_proxy_async();
    mbar_expect_tx(&bar[j & 1], Ly.ktB + Ly.gB + Ly.uB);
    bulk_g2s(dst, p.Kt + (int64_t)k * p.ktstride, Ly.ktB, &bar[j & 1]);
    bulk_g2s(dst + p.ktstride, p.Gf + (int64_t)(c - 1) * p.gstride, Ly.gB, &bar[j & 1]);
    bulk_g2s(dst + p.ktstride + p.gstride, p.d + (int64_t)k * p.us, Ly.uB, &bar[j & 1]);
  };
  uint32_t phase0 = 0, phase1 = 0;
  if (nsteps > 0 && leader) issue(0);
  for (int j = 0; j < nsteps; ++j) {
    const int ci = gg + (j / Lc) * ng;
    const int t = p.chain_stage + (j % Lc);
    const int k = p.stage_begin[t] + ci, c = p.stage_begin[t + 1] + ci;
    if (j + 1 < nsteps && leader) issue(j + 1);
    if (t == p.chain_stage) {  // state at the top of the chain
      for (int r = sub * 32 + lane; r < nx; r += kGrpThreads) {
        if (k == 0) {
          vw[r] = p.x0[r];
          zo[p.zx[0] + r] = p.x0[r];
        } else {
          vw[r] = zo[p.zx[k] + r];
        }
      }
    }
    uint32_t& ph = (j & 1) ? phase1 : phase0;
    const uint32_t par = ph;
    const bool ok = grp_wait(&bar[j & 1], par, votes[g], sub, lane, bar_id);
    ph ^= 1u;
    if (!ok) {
      if (leader) {
        atomicExch(p.err, 1);
        mbar_wait(&bar[j & 1], par);
        if (j + 1 < nsteps) mbar_wait(&bar[(j + 1) & 1], (j & 1) ? phase0 : phase1);
      }
      return;
    }
    const S* Kt = stg[j & 1];
    const S* Gf = Kt + p.ktstride;
    const S* dk = Gf + p.gstride;
    for (int a = sub * 32 + lane; a < nu; a += kGrpThreads) vw[nx + a] = dk[a];
    named_bar(bar_id, kGrpThreads);
    S res[SLG];
    int idx[SLG];
#pragma unroll
    for (int s = 0; s < SLG; ++s) {
      const int slot = sub + s * kGrpWarps;
      res[s] = S(0);
      idx[s] = -1;
      if (slot < xslots) {  // x^c_r = sum_j Gf[j][r] w_j
        const int r = slot * 32 + lane;
        if (r < nx) {
          S acc = 0;
#pragma unroll 4
          for (int jj = 0; jj < ncol; ++jj) acc += Gf[jj * nx + r] * vw[jj];
          res[s] = acc;
          idx[s] = r;
        }
      } else if (slot < nslots) {  // u_a = d_a + sum_r Kt[r][a] x_r
        const int a = (slot - xslots) * 32 + lane;
        if (a < nu) {
          S acc = vw[nx + a];
#pragma unroll 4
          for (int r = 0; r < nx; ++r) acc += Kt[r * nu + a] * vw[r];
          res[s] = acc;
          idx[s] = nx + a;
        }
      }
    }
    named_bar(bar_id, kGrpThreads);  // every warp has read vw
    const int64_t zxc = p.zx[c], zuk = p.zu[k];
#pragma unroll
    for (int s = 0; s < SLG; ++s) {
      const int i = idx[s];
      if (i >= 0 && i < nx) {
        zo[zxc + i] = res[s];
        vw[i] = res[s];
      } else if (i >= nx) {
        zo[zuk + (i - nx)] = res[s];
      }
    }
    named_bar(bar_id, kGrpThreads);  // stage j&1 free, vw holds x^c
  }
}

static size_t grp_max_smem() {
  static size_t v = 0;
  if (!v) {
    int dev = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    v = (size_t)b;
  }
  return v;
}
static int grp_sms() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  }
  return v;
}

template <typename S>
bool grp_chain_fits(const KP<S>& p) {
  const size_t avail = grp_max_smem() - 2048;
  return grp_layout_bwd(p).groupB <= avail && grp_layout_fwd(p).groupB <= avail;
}

template <typename S, int SLG>
static int launch_bwd_chain_grp_slg(const KP<S>& p, cudaStream_t st) {
  const GrpLayout<S> Ly = grp_layout_bwd(p);
  int ngb = (int)std::min<size_t>(kMaxGroups, (grp_max_smem() - 2048) / Ly.groupB);
  ngb = std::max(1, ngb);
  const size_t bytes = (size_t)ngb * Ly.groupB;
  static size_t granted = 0;
  if (bytes > granted) {
    cudaFuncSetAttribute(k_bwd_chain_grp<S, SLG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    granted = bytes;
  }
  const int grid = std::max(1, std::min(grp_sms(), (p.n_chains + ngb - 1) / ngb));
  k_bwd_chain_grp<S, SLG><<<grid, kGrpThreads * ngb, bytes, st>>>(p);
  return 1;
}
template <typename S, int SLG>
static int launch_fwd_chain_grp_slg(const KP<S>& p, S* zo, cudaStream_t st) {
  const GrpLayout<S> Ly = grp_layout_fwd(p);
  int ngb = (int)std::min<size_t>(kMaxGroups, (grp_max_smem() - 2048) / Ly.groupB);
  ngb = std::max(1, ngb);
  const size_t bytes = (size_t)ngb * Ly.groupB;
  static size_t granted = 0;
  if (bytes > granted) {
    cudaFuncSetAttribute(k_fwd_chain_grp<S, SLG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    granted = bytes;
  }
  const int grid = std::max(1, std::min(grp_sms(), (p.n_chains + ngb - 1) / ngb));
  k_fwd_chain_grp<S, SLG><<<grid, kGrpThreads * ngb, bytes, st>>>(p, zo);
  return 1;
}

// SLG: output slots of 96 per warp group (ncol <= 96: 1, else 2).  For the
// forward pass the slots are per warp: ceil(nx/32) + ceil(nu/32) <= 6 -> 2.
template <typename S>
int launch_bwd_chain_grp(const KP<S>& p, cudaStream_t st) {
  return (p.nx + p.nu <= kGrpThreads) ? launch_bwd_chain_grp_slg<S, 1>(p, st) : launch_bwd_chain_grp_slg<S, 2>(p, st);
}
template <typename S>
int launch_fwd_chain_grp(const KP<S>& p, S* zo, cudaStream_t st) {
  const int nslots = (p.nx + 31) / 32 + (p.nu + 31) / 32;
  return (nslots <= kGrpWarps) ? launch_fwd_chain_grp_slg<S, 1>(p, zo, st) : launch_fwd_chain_grp_slg<S, 2>(p, zo, st);
}

template bool grp_chain_fits<double>(const KP<double>&);
template bool grp_chain_fits<float>(const KP<float>&);
template int launch_bwd_chain_grp<double>(const KP<double>&, cudaStream_t);
template int launch_bwd_chain_grp<float>(const KP<float>&, cudaStream_t);
template int launch_fwd_chain_grp<double>(const KP<double>&, double*, cudaStream_t);
template int launch_fwd_chain_grp<float>(const KP<float>&, float*, cudaStream_t);

}  // namespace spock
