// Riccati passes (Algorithm 2) with every node's factors staged in shared
// memory by bulk asynchronous copies, one step ahead of their use.
//
// Chain region (one warp per chain, persistent grid, double-buffered):
//   while the warp computes chain step j from stage buffer j&1, the copy of
//   step j+1 -- [Abar^c | B^c] (or its transpose for the forward pass), the
//   node block [K | K + W^T | Rt^-1] (or K^T) and the node's vectors -- is in
//   flight into the other buffer, so the GEMVs never wait on DRAM; the
//   costate q (backward) or state x (forward) of the chain stays in shared
//   memory from step to step.
// Branching stages (one block per node, one warp per child): the children's
//   blocks and the node block are fetched with one bulk copy each, then the
//   children's contributions are computed in parallel and combined.
// Bounded waits: a wait that exceeds kWaitLimit polls sets *p.err, drains the
// copies the warp has in flight (again bounded) and returns.
#include <algorithm>
#include <vector>

#include "batch.cuh"
#include "kernels.cuh"
#include "spock_internal.h"
#include "tma.cuh"

namespace spock {

// ---------------------------------------------------------------------------
// shared-memory GEMV pieces (lanes over outputs, reduction in registers)
// ---------------------------------------------------------------------------

// h += G^T q, G = nx x ncol row-major in shared memory.
template <typename S, int SL>
__device__ __forceinline__ void sm_GTq(const S* G, const S* q, int nx, int ncol, int lane, S (&h)[SL]) {
#pragma unroll 4
  for (int r = 0; r < nx; ++r) {
    const S qr = q[r];
    const S* row = G + r * ncol;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int col = 32 * s + lane;
      if (col < ncol) h[s] += row[col] * qr;
    }
  }
}

// From h (summed over children) and the node block in shared memory: d^k, q^k.
// vh, vg, vd, vq are per-warp shared vectors; ub, xb the node's ubar, xbar.
template <typename S, int SL>
__device__ __forceinline__ void sm_node_bwd(const KP<S>& p, int k, const S (&h)[SL], const S* NBk, const S* xb,
                                            const S* ub, S* vh, S* vg, S* vd, S* vq, int lane) {
  const int nx = p.nx, nu = p.nu, ncol = nx + nu;
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int col = 32 * s + lane;
    if (col < ncol) vh[col] = h[s];
  }
  __syncwarp();
  for (int b = lane; b < nu; b += 32) vg[b] = ub[b] - vh[nx + b];
  __syncwarp();
  const S* Km = NBk;
  const S* Cm = NBk + nu * nx;      // K + W^T
  const S* Ri = NBk + 2 * nu * nx;  // symmetric: read column-wise for conflict-free lanes
  for (int a = lane; a < nu; a += 32) {
    S acc = 0;
    for (int b = 0; b < nu; ++b) acc += Ri[b * nu + a] * vg[b];
    vd[a] = acc;
    p.d[(int64_t)k * p.us + a] = acc;
  }
  __syncwarp();
  S qn[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int r = 32 * s + lane;
    qn[s] = (r < nx) ? vh[r] - xb[r] : S(0);
  }
  // q += K^T (d - ubar) + W d = C^T d - K^T ubar
#pragma unroll 4
  for (int b = 0; b < nu; ++b) {
    const S db = vd[b];
    const S u = ub[b];
    const S* kr = Km + b * nx;
    const S* cr = Cm + b * nx;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int r = 32 * s + lane;
      if (r < nx) qn[s] = fma(-kr[r], u, fma(cr[r], db, qn[s]));   // two FMAs, no add
    }
  }
  __syncwarp();
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int r = 32 * s + lane;
    if (r < nx) vq[r] = qn[s];
  }
  __syncwarp();
}

// u^k = K^k x^k + d^k (Kt = K^T, nx x nu, shared); vw = (x; d) on entry.
template <typename S>
__device__ __forceinline__ void sm_node_fwd(const KP<S>& p, int k, const S* Kt, const S* vw, S* __restrict__ zo,
                                            int lane) {
  const int nx = p.nx, nu = p.nu;
  const int64_t zu = p.zu[k];
  for (int a = lane; a < nu; a += 32) {
    S acc = vw[nx + a];
#pragma unroll 4
    for (int r = 0; r < nx; ++r) acc += Kt[r * nu + a] * vw[r];
    zo[zu + a] = acc;
  }
}

// x^c = Gf^T-layout product: x^c_r = sum_j Gf[j][r] w_j (Gf ncol x nx, shared).
template <typename S, int SL>
__device__ __forceinline__ void sm_child_fwd(const S* Gf, const S* w, int nx, int ncol, int lane, S (&x)[SL]) {
#pragma unroll
  for (int s = 0; s < SL; ++s) x[s] = S(0);
#pragma unroll 4
  for (int j = 0; j < ncol; ++j) {
    const S wj = w[j];
    const S* row = Gf + j * nx;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int r = 32 * s + lane;
      if (r < nx) x[s] += row[r] * wj;
    }
  }
}

__device__ __forceinline__ void flag_timeout(int32_t* err, int lane) {
  if (lane == 0 && err) atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// chain kernels
// ---------------------------------------------------------------------------
constexpr int kMaxChainWarps = 8;

template <typename S>
struct ChainLayout {
  uint32_t gB, nbB, xB, uB, ktB, stageB, warpB;
};

template <typename S>
__host__ __device__ inline ChainLayout<S> chain_layout_bwd(const KP<S>& p) {
  ChainLayout<S> L;
  L.gB = p.gstride * sizeof(S);
  L.nbB = p.nbstride * sizeof(S);
  L.xB = p.xs * sizeof(S);
  L.uB = p.us * sizeof(S);
  L.ktB = p.ktstride * sizeof(S);
  L.stageB = L.gB + L.nbB + 2 * L.xB + L.uB;  // G | NB | xbar_k | ubar_k | xbar_leaf
  L.warpB = 2 * L.stageB + 4 * kVecPad * sizeof(S);
  return L;
}

template <typename S>
__host__ __device__ inline ChainLayout<S> chain_layout_fwd(const KP<S>& p) {
  ChainLayout<S> L;
  L.gB = p.gstride * sizeof(S);
  L.nbB = p.nbstride * sizeof(S);
  L.xB = p.xs * sizeof(S);
  L.uB = p.us * sizeof(S);
  L.ktB = p.ktstride * sizeof(S);
  L.stageB = L.ktB + L.gB + L.uB;  // Kt | Gf | d_k
  L.warpB = 2 * L.stageB + 1 * kVecPad * sizeof(S);
  return L;
}

// Bodies shared by the single-problem and the batched kernels: block `bid`
// of `nblk` for problem p; every warp owns `slotB` bytes of shared memory
// (at least its layout's warpB).
template <typename S, int SL>
__device__ __forceinline__ void bwd_chain_tma_body(const KP<S>& p, int bid, int nblk, uint32_t slotB) {
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxChainWarps][2];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int gw = bid * wpb + wl, nw = nblk * wpb;
  const int nx = p.nx, ncol = p.nx + p.nu;
  const ChainLayout<S> Ly = chain_layout_bwd(p);
  unsigned char* base = smem + (size_t)wl * slotB;
  S* stg[2] = {reinterpret_cast<S*>(base), reinterpret_cast<S*>(base + Ly.stageB)};
  S* vq = reinterpret_cast<S*>(base + 2 * Ly.stageB);
  S* vh = vq + kVecPad;
  S* vg = vh + kVecPad;
  S* vd = vg + kVecPad;
  uint64_t* bar = bars[wl];
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncwarp();
  const int Lc = p.N - p.chain_stage;  // steps per chain
  const int ldim = p.n_chains > 0 ? (p.n_chains - gw + nw - 1) / nw : 0;
  const int nsteps = gw < p.n_chains ? ldim * Lc : 0;
  auto issue = [&](int j) {
    const int ci = gw + (j / Lc) * nw;
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
  if (nsteps > 0 && lane == 0) issue(0);
  for (int j = 0; j < nsteps; ++j) {
    const int ci = gw + (j / Lc) * nw;
    const int t = p.N - 1 - (j % Lc);
    const int k = p.stage_begin[t] + ci;
    if (j + 1 < nsteps && lane == 0) issue(j + 1);
    uint32_t& ph = (j & 1) ? phase1 : phase0;
    const uint32_t par = ph;
    const bool ok = __all_sync(kFull, mbar_wait(&bar[j & 1], par));
    ph ^= 1u;
    if (!ok) {  // flag, then drain this warp's copies in flight (bounded) and leave
      flag_timeout(p.err, lane);
      mbar_wait(&bar[j & 1], par);
      if (j + 1 < nsteps) mbar_wait(&bar[(j + 1) & 1], (j & 1) ? phase0 : phase1);
      return;
    }
    const S* G = stg[j & 1];
    const S* NBk = G + p.gstride;
    const S* xb = NBk + p.nbstride;
    const S* ub = xb + p.xs;
    if (t == p.N - 1) {
      const S* xl = ub + p.us;
      for (int r = lane; r < nx; r += 32) vq[r] = -xl[r];
      __syncwarp();
    }
    S h[SL];
#pragma unroll
    for (int s = 0; s < SL; ++s) h[s] = S(0);
    sm_GTq<S, SL>(G, vq, nx, ncol, lane, h);
    __syncwarp();
    sm_node_bwd<S, SL>(p, k, h, NBk, xb, ub, vh, vg, vd, vq, lane);
    if (t == p.chain_stage)
      for (int r = lane; r < nx; r += 32) p.q[(int64_t)k * p.xs + r] = vq[r];
    __syncwarp();
  }
}

template <typename S, int SL>
__global__ void __launch_bounds__(32 * kMaxChainWarps) k_bwd_chain_tma(KP<S> p) {
  bwd_chain_tma_body<S, SL>(p, blockIdx.x, gridDim.x, chain_layout_bwd(p).warpB);
}

template <typename S, int SL>
__device__ __forceinline__ void fwd_chain_tma_body(const KP<S>& p, S* __restrict__ zo, int bid, int nblk,
                                                   uint32_t slotB) {
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxChainWarps][2];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int gw = bid * wpb + wl, nw = nblk * wpb;
  const int nx = p.nx, ncol = p.nx + p.nu;
  const ChainLayout<S> Ly = chain_layout_fwd(p);
  unsigned char* base = smem + (size_t)wl * slotB;
  S* stg[2] = {reinterpret_cast<S*>(base), reinterpret_cast<S*>(base + Ly.stageB)};
  S* vw = reinterpret_cast<S*>(base + 2 * Ly.stageB);
  uint64_t* bar = bars[wl];
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncwarp();
  const int Lc = p.N - p.chain_stage;
  const int ldim = p.n_chains > 0 ? (p.n_chains - gw + nw - 1) / nw : 0;
  const int nsteps = gw < p.n_chains ? ldim * Lc : 0;
  auto issue = [&](int j) {
    const int ci = gw + (j / Lc) * nw;
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
  if (nsteps > 0 && lane == 0) issue(0);
  for (int j = 0; j < nsteps; ++j) {
    const int ci = gw + (j / Lc) * nw;
    const int t = p.chain_stage + (j % Lc);
    const int k = p.stage_begin[t] + ci, c = p.stage_begin[t + 1] + ci;
    if (j + 1 < nsteps && lane == 0) issue(j + 1);
    if (t == p.chain_stage) {  // state at the top of the chain
      if (k == 0) {
        for (int r = lane; r < nx; r += 32) {
          vw[r] = p.x0[r];
          zo[p.zx[0] + r] = p.x0[r];
        }
      } else {
        for (int r = lane; r < nx; r += 32) vw[r] = zo[p.zx[k] + r];
      }
    }
    uint32_t& ph = (j & 1) ? phase1 : phase0;
    const uint32_t par = ph;
    const bool ok = __all_sync(kFull, mbar_wait(&bar[j & 1], par));
    ph ^= 1u;
    if (!ok) {  // flag, then drain this warp's copies in flight (bounded) and leave
      flag_timeout(p.err, lane);
      mbar_wait(&bar[j & 1], par);
      if (j + 1 < nsteps) mbar_wait(&bar[(j + 1) & 1], (j & 1) ? phase0 : phase1);
      return;
    }
    const S* Kt = stg[j & 1];
    const S* Gf = Kt + p.ktstride;
    const S* dk = Gf + p.gstride;
    for (int a = lane; a < p.nu; a += 32) vw[nx + a] = dk[a];
    __syncwarp();
    sm_node_fwd<S>(p, k, Kt, vw, zo, lane);
    S x[SL];
    sm_child_fwd<S, SL>(Gf, vw, nx, ncol, lane, x);
    __syncwarp();
    const int64_t zx = p.zx[c];
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int r = 32 * s + lane;
      if (r < nx) {
        zo[zx + r] = x[s];
        vw[r] = x[s];
      }
    }
    __syncwarp();
  }
}

template <typename S, int SL>
__global__ void __launch_bounds__(32 * kMaxChainWarps) k_fwd_chain_tma(KP<S> p, S* __restrict__ zo) {
  fwd_chain_tma_body<S, SL>(p, zo, blockIdx.x, gridDim.x, chain_layout_fwd(p).warpB);
}

// ---------------------------------------------------------------------------
// branching-stage kernels: one block per node, warp w takes children w, w+NW..
// ---------------------------------------------------------------------------
constexpr int kMaxStageWarps = 8;

template <typename S>
__host__ __device__ inline uint32_t stage_smem_bwd(const KP<S>& p, int nwarps) {
  // per warp: G buffer + q + h partial; node: NB | xbar | ubar + vh, vg, vd, vq
  return (uint32_t)(nwarps * (p.gstride + 2 * kVecPad) + p.nbstride + p.xs + p.us + 4 * kVecPad) * sizeof(S);
}
template <typename S>
__host__ __device__ inline uint32_t stage_smem_fwd(const KP<S>& p, int nwarps) {
  // per warp: Gf buffer; node: Kt | d + vw
  return (uint32_t)(nwarps * p.gstride + p.ktstride + p.us + kVecPad) * sizeof(S);
}

template <typename S, int SL>
__device__ __forceinline__ void bwd_stage_tma_body(const KP<S>& p, int t, int node) {
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStageWarps + 1];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int nx = p.nx, nu = p.nu, ncol = nx + nu;
  const int k = p.stage_begin[t] + node;
  const int c0 = p.ch_begin[k], m = p.ch_count[k];
  S* Gw = reinterpret_cast<S*>(smem) + (size_t)wl * (p.gstride + 2 * kVecPad);
  S* qw = Gw + p.gstride;
  S* hw = qw + kVecPad;
  S* NBk = reinterpret_cast<S*>(smem) + (size_t)NW * (p.gstride + 2 * kVecPad);
  S* xb = NBk + p.nbstride;
  S* ub = xb + p.xs;
  S* vh = ub + p.us;
  S* vg = vh + kVecPad;
  S* vd = vg + kVecPad;
  S* vq = vd + kVecPad;
  if (threadIdx.x == 0) {
    for (int i = 0; i <= NW; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t gB = p.gstride * sizeof(S);
  if (threadIdx.x == 0) {  // node block, consumed by warp 0 after the children
    mbar_expect_tx(&bars[NW], (p.nbstride + p.xs + p.us) * sizeof(S));
    bulk_g2s(NBk, p.NB + (int64_t)k * p.nbstride, p.nbstride * sizeof(S), &bars[NW]);
    bulk_g2s(xb, p.xbar + (int64_t)k * p.xs, p.xs * sizeof(S), &bars[NW]);
    bulk_g2s(ub, p.ubar + (int64_t)k * p.us, p.us * sizeof(S), &bars[NW]);
  }
  S h[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) h[s] = S(0);
  uint32_t ph = 0;
  bool ok = true;
  for (int j = wl; j < m; j += NW) {
    const int c = c0 + j;
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bars[wl], gB);
      bulk_g2s(Gw, p.Gb + (int64_t)(c - 1) * p.gstride, gB, &bars[wl]);
    }
    const S* qsrc = (c >= p.nl) ? p.xbar + (int64_t)c * p.xs : p.q + (int64_t)c * p.xs;
    const S sg = (c >= p.nl) ? S(-1) : S(1);
    for (int r = lane; r < nx; r += 32) qw[r] = sg * qsrc[r];
    ok = __all_sync(kFull, mbar_wait(&bars[wl], ph));
    if (!ok) {
      mbar_wait(&bars[wl], ph);  // drain the copy in flight (bounded)
      break;
    }
    ph ^= 1u;
    __syncwarp();
    sm_GTq<S, SL>(Gw, qw, nx, ncol, lane, h);
    __syncwarp();
  }
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int col = 32 * s + lane;
    if (col < ncol) hw[col] = h[s];
  }
  if (!ok) flag_timeout(p.err, lane);
  __syncthreads();
  if (wl != 0) return;
  bool okn = __all_sync(kFull, mbar_wait(&bars[NW], 0));
  if (!okn) {
    flag_timeout(p.err, lane);
    mbar_wait(&bars[NW], 0);
    return;
  }
  S hs[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int col = 32 * s + lane;
    hs[s] = S(0);
    if (col < ncol)
      for (int w = 0; w < NW; ++w)
        hs[s] += (reinterpret_cast<S*>(smem) + (size_t)w * (p.gstride + 2 * kVecPad) + p.gstride + kVecPad)[col];
  }
  sm_node_bwd<S, SL>(p, k, hs, NBk, xb, ub, vh, vg, vd, vq, lane);
  for (int r = lane; r < nx; r += 32) p.q[(int64_t)k * p.xs + r] = vq[r];
  (void)nu;
}

template <typename S, int SL>
__global__ void __launch_bounds__(32 * kMaxStageWarps) k_bwd_stage_tma(KP<S> p, int t) {
  bwd_stage_tma_body<S, SL>(p, t, blockIdx.x);
}

template <typename S, int SL>
__device__ __forceinline__ void fwd_stage_tma_body(const KP<S>& p, int t, S* __restrict__ zo, int node) {
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bars[kMaxStageWarps + 1];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int nx = p.nx, ncol = p.nx + p.nu;
  const int k = p.stage_begin[t] + node;
  const int c0 = p.ch_begin[k], m = p.ch_count[k];
  S* Gw = reinterpret_cast<S*>(smem) + (size_t)wl * p.gstride;
  S* Kt = reinterpret_cast<S*>(smem) + (size_t)NW * p.gstride;
  S* dk = Kt + p.ktstride;
  S* vw = dk + p.us;
  if (threadIdx.x == 0) {
    for (int i = 0; i <= NW; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t gB = p.gstride * sizeof(S);
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bars[NW], (p.ktstride + p.us) * sizeof(S));
    bulk_g2s(Kt, p.Kt + (int64_t)k * p.ktstride, p.ktstride * sizeof(S), &bars[NW]);
    bulk_g2s(dk, p.d + (int64_t)k * p.us, p.us * sizeof(S), &bars[NW]);
  }
  if (lane == 0 && wl < m) {  // first child of each warp, fetched while u^k is computed
    mbar_expect_tx(&bars[wl], gB);
    bulk_g2s(Gw, p.Gf + (int64_t)(c0 + wl - 1) * p.gstride, gB, &bars[wl]);
  }
  bool ok = true;
  if (wl == 0) {
    if (k == 0) {
      for (int r = lane; r < nx; r += 32) {
        vw[r] = p.x0[r];
        zo[p.zx[0] + r] = p.x0[r];
      }
    } else {
      for (int r = lane; r < nx; r += 32) vw[r] = zo[p.zx[k] + r];
    }
    ok = __all_sync(kFull, mbar_wait(&bars[NW], 0));
    if (ok) {
      for (int a = lane; a < p.nu; a += 32) vw[nx + a] = dk[a];
      __syncwarp();
      sm_node_fwd<S>(p, k, Kt, vw, zo, lane);
    } else {
      flag_timeout(p.err, lane);
      mbar_wait(&bars[NW], 0);
    }
  }
  __syncthreads();
  uint32_t ph = 0;
  for (int j = wl; j < m; j += NW) {
    const int c = c0 + j;
    if (j != wl && lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bars[wl], gB);
      bulk_g2s(Gw, p.Gf + (int64_t)(c - 1) * p.gstride, gB, &bars[wl]);
    }
    const bool okc = __all_sync(kFull, mbar_wait(&bars[wl], ph));
    if (!okc) {
      flag_timeout(p.err, lane);
      mbar_wait(&bars[wl], ph);
      return;
    }
    ph ^= 1u;
    S x[SL];
    sm_child_fwd<S, SL>(Gw, vw, nx, ncol, lane, x);
    const int64_t zx = p.zx[c];
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int r = 32 * s + lane;
      if (r < nx) zo[zx + r] = x[s];
    }
    __syncwarp();
  }
  (void)ok;
}

template <typename S, int SL>
__global__ void __launch_bounds__(32 * kMaxStageWarps) k_fwd_stage_tma(KP<S> p, int t, S* __restrict__ zo) {
  fwd_stage_tma_body<S, SL>(p, t, zo, blockIdx.x);
}

// ---------------------------------------------------------------------------
// batched staged kernels: block -> (instance, block) from the launch's map;
// chain warps own slotB bytes each (the largest layout of the batch); stage
// blocks take one node of the instance's stage m.stage[i]
// ---------------------------------------------------------------------------
template <typename S, int SL>
__global__ void __launch_bounds__(32 * kMaxChainWarps) k_bwd_chain_tma_b(const BInst<S>* __restrict__ bi, BMap m,
                                                                        uint32_t slotB) {
  const int i = m.inst[blockIdx.x];
  const KP<S> p = bi[i].kp;
  bwd_chain_tma_body<S, SL>(p, blockIdx.x - m.base[i], m.cnt[i], slotB);
}
template <typename S, int SL>
__global__ void __launch_bounds__(32 * kMaxChainWarps) k_fwd_chain_tma_b(const BInst<S>* __restrict__ bi, BMap m,
                                                                        uint32_t slotB) {
  const int i = m.inst[blockIdx.x];
  const KP<S> p = bi[i].kp;
  fwd_chain_tma_body<S, SL>(p, bi[i].TVt, blockIdx.x - m.base[i], m.cnt[i], slotB);
}
template <typename S, int SL>
__global__ void __launch_bounds__(32 * kMaxStageWarps) k_bwd_stage_tma_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const KP<S> p = bi[i].kp;
  bwd_stage_tma_body<S, SL>(p, m.stage[i], blockIdx.x - m.base[i]);
}
template <typename S, int SL>
__global__ void __launch_bounds__(32 * kMaxStageWarps) k_fwd_stage_tma_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const KP<S> p = bi[i].kp;
  fwd_stage_tma_body<S, SL>(p, m.stage[i], bi[i].TVt, blockIdx.x - m.base[i]);
}

// ---------------------------------------------------------------------------
// launch plan
// ---------------------------------------------------------------------------
static size_t max_dyn_smem() {
  static size_t v = 0;
  if (!v) {
    int dev = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    v = (size_t)b;
  }
  return v;
}
static int num_sms() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  }
  return v;
}

// Raises the kernel's dynamic shared-memory limit when needed (once per size).
template <typename F>
static void allow_smem(F* fn, size_t bytes, size_t& granted) {
  if (bytes > granted) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    granted = bytes;
  }
}

// The staged chain kernels hold two steps per warp in shared memory, which
// bounds the warps per SM.  FP64 arithmetic runs on one unit per SM
// sub-partition (a quarter of the SM's FP64 rate each, measured), so the FP64
// instance is used only when at least four warps fit; otherwise the
// direct-load kernels, with many more resident warps, are faster.
template <typename S>
bool tma_chain_fits(const KP<S>& p) {
  const size_t avail = max_dyn_smem() - 1024;
  const size_t need_warps = sizeof(S) == 8 ? 4 : 1;
  return (size_t)chain_layout_bwd(p).warpB * need_warps <= avail &&
         (size_t)chain_layout_fwd(p).warpB * need_warps <= avail;
}
template <typename S>
bool tma_stage_fits(const KP<S>& p) {
  return (size_t)stage_smem_bwd(p, 1) <= max_dyn_smem() - 1024 && (size_t)stage_smem_fwd(p, 1) <= max_dyn_smem() - 1024;
}

template <typename S, int SL>
int launch_bwd_chain_tma(const KP<S>& p, cudaStream_t st) {
  const ChainLayout<S> Ly = chain_layout_bwd(p);
  int wpb = (int)std::min<size_t>(kMaxChainWarps, (max_dyn_smem() - 1024) / Ly.warpB);
  wpb = std::max(1, wpb);
  const size_t bytes = (size_t)wpb * Ly.warpB;
  static size_t granted = 0;
  allow_smem(k_bwd_chain_tma<S, SL>, bytes, granted);
  int grid = std::min(num_sms(), (p.n_chains + wpb - 1) / wpb);
  k_bwd_chain_tma<S, SL><<<grid, 32 * wpb, bytes, st>>>(p);
  return 1;
}

template <typename S, int SL>
int launch_fwd_chain_tma(const KP<S>& p, S* zo, cudaStream_t st) {
  const ChainLayout<S> Ly = chain_layout_fwd(p);
  int wpb = (int)std::min<size_t>(kMaxChainWarps, (max_dyn_smem() - 1024) / Ly.warpB);
  wpb = std::max(1, wpb);
  const size_t bytes = (size_t)wpb * Ly.warpB;
  static size_t granted = 0;
  allow_smem(k_fwd_chain_tma<S, SL>, bytes, granted);
  int grid = std::min(num_sms(), (p.n_chains + wpb - 1) / wpb);
  k_fwd_chain_tma<S, SL><<<grid, 32 * wpb, bytes, st>>>(p, zo);
  return 1;
}

template <typename S, int SL>
int launch_bwd_stage_tma(const KP<S>& p, int t, int cnt, int max_children, cudaStream_t st) {
  int nwp = std::min(max_children, kMaxStageWarps);
  while (nwp > 1 && stage_smem_bwd(p, nwp) > max_dyn_smem() - 1024) --nwp;
  const size_t bytes = stage_smem_bwd(p, nwp);
  static size_t granted = 0;
  allow_smem(k_bwd_stage_tma<S, SL>, bytes, granted);
  k_bwd_stage_tma<S, SL><<<cnt, 32 * nwp, bytes, st>>>(p, t);
  return 1;
}

template <typename S, int SL>
int launch_fwd_stage_tma(const KP<S>& p, int t, int cnt, int max_children, S* zo, cudaStream_t st) {
  int nwp = std::min(max_children, kMaxStageWarps);
  while (nwp > 1 && stage_smem_fwd(p, nwp) > max_dyn_smem() - 1024) --nwp;
  const size_t bytes = stage_smem_fwd(p, nwp);
  static size_t granted = 0;
  allow_smem(k_fwd_stage_tma<S, SL>, bytes, granted);
  k_fwd_stage_tma<S, SL><<<cnt, 32 * nwp, bytes, st>>>(p, t, zo);
  return 1;
}

// Shape of the staged kernels for a batch: warps per chain block and the
// per-warp slot (largest layout over the instances), warps per stage block
// and the stage blocks' shared memory.  Returns false if some instance's
// layout does not fit.
template <typename S>
bool tma_batch_shape(const std::vector<KP<S>>& kps, int max_children, TmaBatchShape& sh) {
  uint32_t wb = 0, wf = 0;
  for (const KP<S>& p : kps) {
    wb = std::max(wb, chain_layout_bwd(p).warpB);
    wf = std::max(wf, chain_layout_fwd(p).warpB);
  }
  const size_t avail = max_dyn_smem() - 1024;
  if (wb == 0 || wf == 0 || wb > avail || wf > avail) return false;
  sh.slot_bwd = wb;
  sh.slot_fwd = wf;
  sh.wpb_bwd = (int)std::min<size_t>(kMaxChainWarps, avail / wb);
  sh.wpb_fwd = (int)std::min<size_t>(kMaxChainWarps, avail / wf);
  int nwb = std::max(1, std::min(max_children, kMaxStageWarps)), nwf = nwb;
  auto smem_b = [&](int nw) {
    uint32_t v = 0;
    for (const KP<S>& p : kps) v = std::max(v, stage_smem_bwd(p, nw));
    return v;
  };
  auto smem_f = [&](int nw) {
    uint32_t v = 0;
    for (const KP<S>& p : kps) v = std::max(v, stage_smem_fwd(p, nw));
    return v;
  };
  while (nwb > 1 && smem_b(nwb) > avail) --nwb;
  while (nwf > 1 && smem_f(nwf) > avail) --nwf;
  if (smem_b(nwb) > avail || smem_f(nwf) > avail) return false;
  sh.nw_stage_bwd = nwb;
  sh.nw_stage_fwd = nwf;
  sh.smem_stage_bwd = smem_b(nwb);
  sh.smem_stage_fwd = smem_f(nwf);
  return true;
}

template <typename S, int SL>
static void riccati_tma_b_sl(int which, const BInst<S>* bi, const BMap& m, int nblocks, const TmaBatchShape& sh,
                             cudaStream_t st) {
  static size_t g0 = 0, g1 = 0, g2 = 0, g3 = 0;
  if (which == 0) {
    const size_t bytes = (size_t)sh.wpb_bwd * sh.slot_bwd;
    allow_smem(k_bwd_chain_tma_b<S, SL>, bytes, g0);
    k_bwd_chain_tma_b<S, SL><<<nblocks, 32 * sh.wpb_bwd, bytes, st>>>(bi, m, sh.slot_bwd);
  } else if (which == 1) {
    allow_smem(k_bwd_stage_tma_b<S, SL>, sh.smem_stage_bwd, g1);
    k_bwd_stage_tma_b<S, SL><<<nblocks, 32 * sh.nw_stage_bwd, sh.smem_stage_bwd, st>>>(bi, m);
  } else if (which == 2) {
    allow_smem(k_fwd_stage_tma_b<S, SL>, sh.smem_stage_fwd, g2);
    k_fwd_stage_tma_b<S, SL><<<nblocks, 32 * sh.nw_stage_fwd, sh.smem_stage_fwd, st>>>(bi, m);
  } else {
    const size_t bytes = (size_t)sh.wpb_fwd * sh.slot_fwd;
    allow_smem(k_fwd_chain_tma_b<S, SL>, bytes, g3);
    k_fwd_chain_tma_b<S, SL><<<nblocks, 32 * sh.wpb_fwd, bytes, st>>>(bi, m, sh.slot_fwd);
  }
}

template <typename S>
void launch_riccati_tma_b(int which, const BInst<S>* bi, const BMap& m, int nblocks, int SL, const TmaBatchShape& sh,
                          cudaStream_t st) {
  if (nblocks <= 0) return;
  switch (SL) {
    case 1: riccati_tma_b_sl<S, 1>(which, bi, m, nblocks, sh, st); break;
    case 2: riccati_tma_b_sl<S, 2>(which, bi, m, nblocks, sh, st); break;
    case 3: riccati_tma_b_sl<S, 3>(which, bi, m, nblocks, sh, st); break;
    default: riccati_tma_b_sl<S, 4>(which, bi, m, nblocks, sh, st); break;
  }
}
template bool tma_batch_shape<double>(const std::vector<KP<double>>&, int, TmaBatchShape&);
template bool tma_batch_shape<float>(const std::vector<KP<float>>&, int, TmaBatchShape&);
template void launch_riccati_tma_b<double>(int, const BInst<double>*, const BMap&, int, int, const TmaBatchShape&,
                                           cudaStream_t);
template void launch_riccati_tma_b<float>(int, const BInst<float>*, const BMap&, int, int, const TmaBatchShape&,
                                          cudaStream_t);

#define SPOCK_TMA_INST(S, SL)                                                                    \
  template int launch_bwd_chain_tma<S, SL>(const KP<S>&, cudaStream_t);                          \
  template int launch_fwd_chain_tma<S, SL>(const KP<S>&, S*, cudaStream_t);                      \
  template int launch_bwd_stage_tma<S, SL>(const KP<S>&, int, int, int, cudaStream_t);           \
  template int launch_fwd_stage_tma<S, SL>(const KP<S>&, int, int, int, S*, cudaStream_t);
SPOCK_TMA_INST(double, 1)
SPOCK_TMA_INST(double, 2)
SPOCK_TMA_INST(double, 3)
SPOCK_TMA_INST(double, 4)
SPOCK_TMA_INST(float, 1)
SPOCK_TMA_INST(float, 2)
SPOCK_TMA_INST(float, 3)
SPOCK_TMA_INST(float, 4)
template bool tma_chain_fits<double>(const KP<double>&);
template bool tma_chain_fits<float>(const KP<float>&);
template bool tma_stage_fits<double>(const KP<double>&);
template bool tma_stage_fits<float>(const KP<float>&);

}  // namespace spock
