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
#include "riccati_body.cuh"
#include "spock_internal.h"

namespace spock {

template <typename S, int SL>
__global__ void __launch_bounds__(128) k_bwd_chain(KP<S> p) {
  bwd_chain_body<S, SL>(p, blockIdx.x, gridDim.x);
}

template <typename S, int SL>
__global__ void __launch_bounds__(128) k_bwd_stage(KP<S> p, int t) {
  bwd_stage_body<S, SL>(p, t, blockIdx.x, gridDim.x);
}

template <typename S, int SL>
__global__ void __launch_bounds__(128) k_fwd_stage(KP<S> p, int t, S* __restrict__ zo) {
  fwd_stage_body<S, SL>(p, t, zo, blockIdx.x, gridDim.x);
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
// FP64 stages with at least this many nodes use the direct kernels (many
// resident warps keep the FP64 pipe busy): 1,024 in the backward pass, 2,048
// in the forward pass (on the 62,805-node tree the stage of 1,024 nodes with
// four children each took 0.174 vs 0.213 ms per T of backward stages on the
// direct kernel, but 0.211 vs 0.184 ms of forward stages);
// SPOCK_STAGED_MAX_NODES overrides both.
inline int staged_max_nodes(bool backward) {
  static int v = [] {
    const char* e = getenv("SPOCK_STAGED_MAX_NODES");
    return e ? atoi(e) : -1;
  }();
  return v >= 0 ? v : (backward ? 1024 : 2048);
}
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
  auto staged = [&](int cnt, bool bwd) {
    return tma_stage && (sizeof(S) == 4 || cnt < staged_max_nodes(bwd));
  };
  for (int t = cs - 1; t >= 0; --t) {
    const int cnt = stage_begin[t + 1] - stage_begin[t];
    if (staged(cnt, true)) {
      launches += launch_bwd_stage_tma<S, SL>(p, t, cnt, stage_maxch[t], st);
    } else {
      k_bwd_stage<S, SL><<<(cnt + kWarpsPerBlock - 1) / kWarpsPerBlock, 128, 0, st>>>(p, t);
      ++launches;
    }
  }
  if (ev) record_event(ev[1], st);
  for (int t = 0; t < cs; ++t) {
    const int cnt = stage_begin[t + 1] - stage_begin[t];
    if (staged(cnt, false)) {
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
