// Online projection on the tree dynamics S1 (Algorithm 2) with the factors
// of Algorithm 1 (factor.cpp).
//
// Backward pass, for every nonleaf node i from stage N-1 to 0, with
// q^j = -xbar^j at the leaves:
//   d^i = Rt^-1 (ubar^i - sum_c B^cT q^c)
//   q^i = K^iT (d^i - ubar^i) - xbar^i + W^i d^i + sum_c Abar^cT q^c
// (W^i = sum_c Abar^cT P^c B^c gathers the P^c B^c d^i terms of the paper's
// recursion).  Forward pass from x^0 = x:
//   u^i = K^i x^i + d^i,   x^c = A^c x^i + B^c u^i = Abar^c x^i + B^c d^i.
//
// GB300 mapping.  One warp owns one node at a time.  Every factor is read
// exactly once per pass, with lanes over output entries so that each warp
// load instruction reads a contiguous row segment (coalesced) and the
// reduction index runs through registers; the small vectors (q, x, d, ubar)
// live in per-warp shared memory so any lane can broadcast-read any entry.
//   * chain kernels: below the "chain stage" every node has one child
//     (4096 chains of 15 nodes for the 62,805-node tree), so one warp walks
//     a whole chain, carrying q (backward) or x (forward) in shared memory
//     with no grid-wide synchronisation;
//   * stage kernels: above it (branching stages) one launch per stage, one
//     warp per node, children's q / parent's x exchanged through global
//     memory between launches.
// The backward layout [Abar^c | B^c] (nx x (nx+nu), row-major) serves
// h = [Abar^c | B^c]^T q^c; the forward layout is its transpose so that
// x^c = [Abar^c | B^c] (x; d) is again lanes-over-outputs.
#include <cstdlib>

#include "batch.cuh"
#include "kernels.cuh"
#include "spock_internal.h"

namespace spock {

template <typename S>
struct WarpVecs {
  S* q;  // [nx]     costate of the child being absorbed / result
  S* h;  // [nx+nu]  accumulated [Abar | B]^T q over the children
  S* u;  // [nu]     ubar of the node
  S* g;  // [nu]     ubar - sum B^T q
  S* d;  // [nu]
  S* w;  // [nx+nu]  forward input (x; d)
};

// h += [Abar | B]^T q  for one child; G is nx x ncol row-major.
template <typename S, int SL>
__device__ __forceinline__ void acc_GTq(const S* __restrict__ G, const S* q, int nx, int ncol, int lane,
                                        S (&h)[SL]) {
#pragma unroll 8
  for (int r = 0; r < nx; ++r) {
    const S qr = q[r];
    const S* row = G + (int64_t)r * ncol;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int col = 32 * s + lane;
      if (col < ncol) h[s] += __ldg(row + col) * qr;
    }
  }
}

// Node part of the backward step: from h (sum over children) compute d^k and
// q^k (into v.q); d^k is also stored for the forward pass.
template <typename S, int SL>
__device__ __forceinline__ void node_bwd(const KP<S>& p, int k, const S (&h)[SL], WarpVecs<S>& v, int lane) {
  const int nx = p.nx, nu = p.nu, ncol = nx + nu;
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int col = 32 * s + lane;
    if (col < ncol) v.h[col] = h[s];
  }
  const S* ub = p.ubar + (int64_t)k * p.us;
  for (int b = lane; b < nu; b += 32) v.u[b] = ub[b];
  __syncwarp();
  for (int b = lane; b < nu; b += 32) v.g[b] = v.u[b] - v.h[nx + b];
  __syncwarp();
  const S* __restrict__ Km = p.NB + (int64_t)k * p.nbstride;
  const S* __restrict__ Wt = Km + (int64_t)nu * nx;
  const S* __restrict__ Ri = Km + 2 * (int64_t)nu * nx;
  for (int a = lane; a < nu; a += 32) {
    S acc = 0;
    for (int b = 0; b < nu; ++b) acc += __ldg(Ri + a * nu + b) * v.g[b];
    v.d[a] = acc;
    p.d[(int64_t)k * p.us + a] = acc;
  }
  __syncwarp();
  S qn[SL];
  const S* xb = p.xbar + (int64_t)k * p.xs;
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int r = 32 * s + lane;
    qn[s] = (r < nx) ? v.h[r] - xb[r] : S(0);
  }
#pragma unroll 4
  for (int b = 0; b < nu; ++b) {
    const S db = v.d[b];
    const S dmu = db - v.u[b];
    const S* kr = Km + (int64_t)b * nx;
    const S* wr = Wt + (int64_t)b * nx;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int r = 32 * s + lane;
      if (r < nx) qn[s] += __ldg(kr + r) * dmu + __ldg(wr + r) * db;
    }
  }
  __syncwarp();
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int r = 32 * s + lane;
    if (r < nx) v.q[r] = qn[s];
  }
  __syncwarp();
}

// Node part of the forward step: v.w[0..nx) holds x^k; computes u^k and
// writes it; leaves (x^k; d^k) in v.w.
template <typename S>
__device__ __forceinline__ void node_fwd(const KP<S>& p, int k, WarpVecs<S>& v, S* __restrict__ zo, int lane) {
  const int nx = p.nx, nu = p.nu;
  for (int a = lane; a < nu; a += 32) v.w[nx + a] = p.d[(int64_t)k * p.us + a];
  __syncwarp();
  const S* __restrict__ Kt = p.Kt + (int64_t)k * p.ktstride;
  const int64_t zu = p.zu[k];
  for (int a = lane; a < nu; a += 32) {
    S acc = v.w[nx + a];
#pragma unroll 8
    for (int r = 0; r < nx; ++r) acc += __ldg(Kt + (int64_t)r * nu + a) * v.w[r];
    zo[zu + a] = acc;
  }
}

// x^c = [Abar^c | B^c] (x; d) for one child, Gf = ncol x nx row-major.
template <typename S, int SL>
__device__ __forceinline__ void child_fwd(const S* __restrict__ Gf, const S* w, int nx, int ncol, int lane,
                                          S (&x)[SL]) {
#pragma unroll
  for (int s = 0; s < SL; ++s) x[s] = S(0);
#pragma unroll 8
  for (int j = 0; j < ncol; ++j) {
    const S wj = w[j];
    const S* row = Gf + (int64_t)j * nx;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int r = 32 * s + lane;
      if (r < nx) x[s] += __ldg(row + r) * wj;
    }
  }
}

#define SPOCK_WARP_VECS(S)                                           \
  __shared__ S sm_q[kWarpsPerBlock][kVecPad];                        \
  __shared__ S sm_h[kWarpsPerBlock][kVecPad];                        \
  __shared__ S sm_u[kWarpsPerBlock][kVecPad];                        \
  __shared__ S sm_g[kWarpsPerBlock][kVecPad];                        \
  __shared__ S sm_d[kWarpsPerBlock][kVecPad];                        \
  __shared__ S sm_w[kWarpsPerBlock][kVecPad];                        \
  const int wl_ = threadIdx.x >> 5;                                  \
  WarpVecs<S> v{sm_q[wl_], sm_h[wl_], sm_u[wl_], sm_g[wl_], sm_d[wl_], sm_w[wl_]};

// ---------------------------------------------------------------------------
// backward, chain region: warp per chain, leaves up to the chain stage
// ---------------------------------------------------------------------------
template <typename S, int SL>
__device__ __forceinline__ void bwd_chain_body(const KP<S>& p, int bid, int nblk) {
  if (p.skip && *p.skip) return;
  SPOCK_WARP_VECS(S)
  const int lane = threadIdx.x & 31;
  const int gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  const int nx = p.nx, ncol = p.nx + p.nu;
  for (int ci = gw; ci < p.n_chains; ci += nw) {
    const int leaf = p.stage_begin[p.N] + ci;
    for (int r = lane; r < nx; r += 32) v.q[r] = -p.xbar[(int64_t)leaf * p.xs + r];
    __syncwarp();
    int k = -1;
    for (int t = p.N - 1; t >= p.chain_stage; --t) {
      k = p.stage_begin[t] + ci;
      const int c = p.stage_begin[t + 1] + ci;
      S h[SL];
#pragma unroll
      for (int s = 0; s < SL; ++s) h[s] = S(0);
      acc_GTq<S, SL>(p.Gb + (int64_t)(c - 1) * p.gstride, v.q, nx, ncol, lane, h);
      __syncwarp();
      node_bwd<S, SL>(p, k, h, v, lane);
    }
    for (int r = lane; r < nx; r += 32) p.q[(int64_t)k * p.xs + r] = v.q[r];
    __syncwarp();
  }
}

template <typename S, int SL>
__global__ void __launch_bounds__(128) k_bwd_chain(KP<S> p) {
  bwd_chain_body<S, SL>(p, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// backward, one branching stage: warp per node
// ---------------------------------------------------------------------------
template <typename S, int SL>
__device__ __forceinline__ void bwd_stage_body(const KP<S>& p, int t, int bid, int nblk) {
  if (p.skip && *p.skip) return;
  SPOCK_WARP_VECS(S)
  const int lane = threadIdx.x & 31;
  const int gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  const int nx = p.nx, ncol = p.nx + p.nu;
  const int b0 = p.stage_begin[t], cnt = p.stage_begin[t + 1] - b0;
  for (int idx = gw; idx < cnt; idx += nw) {
    const int k = b0 + idx;
    const int c0 = p.ch_begin[k], m = p.ch_count[k];
    S h[SL];
#pragma unroll
    for (int s = 0; s < SL; ++s) h[s] = S(0);
    for (int j = 0; j < m; ++j) {
      const int c = c0 + j;
      if (c >= p.nl) {
        for (int r = lane; r < nx; r += 32) v.q[r] = -p.xbar[(int64_t)c * p.xs + r];
      } else {
        for (int r = lane; r < nx; r += 32) v.q[r] = p.q[(int64_t)c * p.xs + r];
      }
      __syncwarp();
      acc_GTq<S, SL>(p.Gb + (int64_t)(c - 1) * p.gstride, v.q, nx, ncol, lane, h);
      __syncwarp();
    }
    node_bwd<S, SL>(p, k, h, v, lane);
    for (int r = lane; r < nx; r += 32) p.q[(int64_t)k * p.xs + r] = v.q[r];
    __syncwarp();
  }
}

template <typename S, int SL>
__global__ void __launch_bounds__(128) k_bwd_stage(KP<S> p, int t) {
  bwd_stage_body<S, SL>(p, t, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// forward, one branching stage: warp per node
// ---------------------------------------------------------------------------
template <typename S, int SL>
__device__ __forceinline__ void fwd_stage_body(const KP<S>& p, int t, S* __restrict__ zo, int bid, int nblk) {
  if (p.skip && *p.skip) return;
  SPOCK_WARP_VECS(S)
  const int lane = threadIdx.x & 31;
  const int gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  const int nx = p.nx, ncol = p.nx + p.nu;
  const int b0 = p.stage_begin[t], cnt = p.stage_begin[t + 1] - b0;
  for (int idx = gw; idx < cnt; idx += nw) {
    const int k = b0 + idx;
    if (k == 0) {
      for (int r = lane; r < nx; r += 32) {
        v.w[r] = p.x0[r];
        zo[p.zx[0] + r] = p.x0[r];
      }
    } else {
      for (int r = lane; r < nx; r += 32) v.w[r] = zo[p.zx[k] + r];
    }
    __syncwarp();
    node_fwd<S>(p, k, v, zo, lane);
    __syncwarp();
    const int c0 = p.ch_begin[k], m = p.ch_count[k];
    for (int j = 0; j < m; ++j) {
      const int c = c0 + j;
      S x[SL];
      child_fwd<S, SL>(p.Gf + (int64_t)(c - 1) * p.gstride, v.w, nx, ncol, lane, x);
      const int64_t zx = p.zx[c];
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        const int r = 32 * s + lane;
        if (r < nx) zo[zx + r] = x[s];
      }
    }
    __syncwarp();
  }
}

template <typename S, int SL>
__global__ void __launch_bounds__(128) k_fwd_stage(KP<S> p, int t, S* __restrict__ zo) {
  fwd_stage_body<S, SL>(p, t, zo, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// forward, chain region: warp per chain, chain stage down to the leaves
// ---------------------------------------------------------------------------
template <typename S, int SL>
__device__ __forceinline__ void fwd_chain_body(const KP<S>& p, S* __restrict__ zo, int bid, int nblk) {
  if (p.skip && *p.skip) return;
  SPOCK_WARP_VECS(S)
  const int lane = threadIdx.x & 31;
  const int gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  const int nx = p.nx, ncol = p.nx + p.nu;
  for (int ci = gw; ci < p.n_chains; ci += nw) {
    const int top = p.stage_begin[p.chain_stage] + ci;
    if (top == 0) {
      for (int r = lane; r < nx; r += 32) {
        v.w[r] = p.x0[r];
        zo[p.zx[0] + r] = p.x0[r];
      }
    } else {
      for (int r = lane; r < nx; r += 32) v.w[r] = zo[p.zx[top] + r];
    }
    __syncwarp();
    for (int t = p.chain_stage; t < p.N; ++t) {
      const int k = p.stage_begin[t] + ci;
      const int c = p.stage_begin[t + 1] + ci;
      node_fwd<S>(p, k, v, zo, lane);
      __syncwarp();
      S x[SL];
      child_fwd<S, SL>(p.Gf + (int64_t)(c - 1) * p.gstride, v.w, nx, ncol, lane, x);
      __syncwarp();
      const int64_t zx = p.zx[c];
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        const int r = 32 * s + lane;
        if (r < nx) {
          zo[zx + r] = x[s];
          v.w[r] = x[s];
        }
      }
      __syncwarp();
    }
  }
}

template <typename S, int SL>
__global__ void __launch_bounds__(128) k_fwd_chain(KP<S> p, S* __restrict__ zo) {
  fwd_chain_body<S, SL>(p, zo, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// launcher: the whole S1 projection (prep kernel already ran)
// ---------------------------------------------------------------------------
// bulk-copy pipelined variants (riccati_tma.cu)
template <typename S>
bool tma_chain_fits(const KP<S>& p);
template <typename S>
bool tma_stage_fits(const KP<S>& p);
template <typename S, int SL>
int launch_bwd_chain_tma(const KP<S>& p, cudaStream_t st);
template <typename S, int SL>
int launch_fwd_chain_tma(const KP<S>& p, S* zo, cudaStream_t st);
template <typename S, int SL>
int launch_bwd_stage_tma(const KP<S>& p, int t, int cnt, int max_children, cudaStream_t st);
template <typename S, int SL>
int launch_fwd_stage_tma(const KP<S>& p, int t, int cnt, int max_children, S* zo, cudaStream_t st);

template <typename S>
bool grp_chain_fits(const KP<S>& p);
template <typename S>
int launch_bwd_chain_grp(const KP<S>& p, cudaStream_t st);
template <typename S>
int launch_fwd_chain_grp(const KP<S>& p, S* zo, cudaStream_t st);

// Kernel family for the chain region: "grp" (three warps per chain, staged),
// "tma" (one warp per chain, staged) or "direct" (one warp per chain, loads
// straight from global memory); the branching stages use the staged
// block-per-node kernels unless "direct".  Default (measured on the
// 62,805-node tree): forward pass "grp"; backward pass "tma" (FP32) -- its
// node update keeps only one warp busy, so splitting it over three warps
// loses more at the barriers than it gains -- and "direct" for FP64 where
// the staged variant fits too few warps per SM (tma_chain_fits).
// SPOCK_RICCATI_KERNELS forces one family everywhere (the tests cover each).
enum ChainFamily { CF_AUTO = -1, CF_GRP = 0, CF_TMA = 1, CF_DIRECT = 2 };
constexpr int kStagedMaxNodes = 2048;  // FP64 stages with more nodes use the direct kernels
static int chain_family() {
  const char* e = getenv("SPOCK_RICCATI_KERNELS");
  if (!e || !e[0]) return CF_AUTO;
  if (e[0] == 'd') return CF_DIRECT;
  if (e[0] == 't') return CF_TMA;
  if (e[0] == 'g') return CF_GRP;
  return CF_AUTO;
}

// Launches both passes; ev (optional, 3 events) is recorded after the
// backward chain kernel, the backward stage kernels and the forward stage
// kernels.  Returns the number of kernels launched.
template <typename S, int SL>
int riccati_passes_sl(const KP<S>& p, const std::vector<int32_t>& stage_begin,
                      const std::vector<int32_t>& stage_maxch, S* zo, cudaStream_t st, cudaEvent_t* ev) {
  const int cs = p.chain_stage;
  const int fam = chain_family();
  const bool grp_ok = fam != CF_DIRECT && fam != CF_TMA && grp_chain_fits(p);
  const bool bwd_grp = fam == CF_GRP && grp_ok;
  const bool fwd_grp = (fam == CF_GRP || fam == CF_AUTO) && grp_ok;
  const bool tma_chain = fam != CF_DIRECT && tma_chain_fits(p);
  const bool tma_stage = fam != CF_DIRECT && tma_stage_fits(p);
  int launches = 0;
  if (p.n_chains > 0 && cs < p.N) {
    if (bwd_grp) {
      launches += launch_bwd_chain_grp<S>(p, st);
    } else if (tma_chain) {
      launches += launch_bwd_chain_tma<S, SL>(p, st);
    } else {
      const int grid = (p.n_chains + kWarpsPerBlock - 1) / kWarpsPerBlock;
      k_bwd_chain<S, SL><<<grid, 128, 0, st>>>(p);
      ++launches;
    }
  }
  if (ev) record_event(ev[0], st);
  // Branching stages: the staged block-per-node kernels cut the latency of
  // every stage in FP32 (measured); in FP64 a stage with many nodes runs
  // better on the direct warp-per-node kernels, which keep far more warps
  // resident (FP64 needs one per SM sub-partition).
  auto staged = [&](int cnt) { return tma_stage && (sizeof(S) == 4 || cnt < kStagedMaxNodes); };
  for (int t = cs - 1; t >= 0; --t) {
    const int cnt = stage_begin[t + 1] - stage_begin[t];
    if (staged(cnt)) {
      launches += launch_bwd_stage_tma<S, SL>(p, t, cnt, stage_maxch[t], st);
    } else {
      k_bwd_stage<S, SL><<<(cnt + kWarpsPerBlock - 1) / kWarpsPerBlock, 128, 0, st>>>(p, t);
      ++launches;
    }
  }
  if (ev) record_event(ev[1], st);
  for (int t = 0; t < cs; ++t) {
    const int cnt = stage_begin[t + 1] - stage_begin[t];
    if (staged(cnt)) {
      launches += launch_fwd_stage_tma<S, SL>(p, t, cnt, stage_maxch[t], zo, st);
    } else {
      k_fwd_stage<S, SL><<<(cnt + kWarpsPerBlock - 1) / kWarpsPerBlock, 128, 0, st>>>(p, t, zo);
      ++launches;
    }
  }
  if (ev) record_event(ev[2], st);
  if (p.n_chains > 0 && cs < p.N) {
    if (fwd_grp) {
      launches += launch_fwd_chain_grp<S>(p, zo, st);
    } else if (tma_chain) {
      launches += launch_fwd_chain_tma<S, SL>(p, zo, st);
    } else {
      const int grid = (p.n_chains + kWarpsPerBlock - 1) / kWarpsPerBlock;
      k_fwd_chain<S, SL><<<grid, 128, 0, st>>>(p, zo);
      ++launches;
    }
  }
  return launches;
}

template <typename S>
int launch_riccati(const KP<S>& p, const std::vector<int32_t>& stage_begin, const std::vector<int32_t>& stage_maxch,
                   S* zo, cudaStream_t st, cudaEvent_t* ev) {
  const int sl = (p.nx + p.nu + 31) / 32;
  switch (sl) {
    case 1: return riccati_passes_sl<S, 1>(p, stage_begin, stage_maxch, zo, st, ev);
    case 2: return riccati_passes_sl<S, 2>(p, stage_begin, stage_maxch, zo, st, ev);
    case 3: return riccati_passes_sl<S, 3>(p, stage_begin, stage_maxch, zo, st, ev);
    default: return riccati_passes_sl<S, 4>(p, stage_begin, stage_maxch, zo, st, ev);
  }
}

// ---------------------------------------------------------------------------
// batched: direct kernels over the block map of the launch (chains of every
// instance, or one stage of every instance: stage[i] from the map)
// ---------------------------------------------------------------------------
template <typename S, int SL>
__global__ void __launch_bounds__(128) k_bwd_chain_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const KP<S> p = bi[i].kp;
  bwd_chain_body<S, SL>(p, blockIdx.x - m.base[i], m.cnt[i]);
}
template <typename S, int SL>
__global__ void __launch_bounds__(128) k_bwd_stage_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const KP<S> p = bi[i].kp;
  bwd_stage_body<S, SL>(p, m.stage[i], blockIdx.x - m.base[i], m.cnt[i]);
}
template <typename S, int SL>
__global__ void __launch_bounds__(128) k_fwd_stage_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const KP<S> p = bi[i].kp;
  fwd_stage_body<S, SL>(p, m.stage[i], bi[i].TVt, blockIdx.x - m.base[i], m.cnt[i]);
}
template <typename S, int SL>
__global__ void __launch_bounds__(128) k_fwd_chain_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const KP<S> p = bi[i].kp;
  fwd_chain_body<S, SL>(p, bi[i].TVt, blockIdx.x - m.base[i], m.cnt[i]);
}

template <typename S>
void launch_riccati_b(int which, const BInst<S>* bi, const BMap& m, int nblocks, int SL, cudaStream_t st) {
  if (nblocks <= 0) return;
#define SPOCK_RB(L)                                                                    \
  case L:                                                                              \
    if (which == 0) k_bwd_chain_b<S, L><<<nblocks, 128, 0, st>>>(bi, m);              \
    else if (which == 1) k_bwd_stage_b<S, L><<<nblocks, 128, 0, st>>>(bi, m);         \
    else if (which == 2) k_fwd_stage_b<S, L><<<nblocks, 128, 0, st>>>(bi, m);         \
    else k_fwd_chain_b<S, L><<<nblocks, 128, 0, st>>>(bi, m);                         \
    break;
  switch (SL) {
    SPOCK_RB(1) SPOCK_RB(2) SPOCK_RB(3)
    default: SPOCK_RB(4)
  }
#undef SPOCK_RB
}
template void launch_riccati_b<double>(int, const BInst<double>*, const BMap&, int, int, cudaStream_t);
template void launch_riccati_b<float>(int, const BInst<float>*, const BMap&, int, int, cudaStream_t);

template int launch_riccati<double>(const KP<double>&, const std::vector<int32_t>&, const std::vector<int32_t>&,
                                    double*, cudaStream_t, cudaEvent_t*);
template int launch_riccati<float>(const KP<float>&, const std::vector<int32_t>&, const std::vector<int32_t>&,
                                   float*, cudaStream_t, cudaEvent_t*);

}  // namespace spock
