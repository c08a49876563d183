// Single-block solves.  One thread block of 128 threads runs Algorithm 3 for
// one instance, from the first evaluation of T to termination: the same
// bodies as the multi-block kernels (ops_body.cuh, riccati_body.cuh,
// rounds_body.cuh) called as block 0 of 1, the phases separated by block
// barriers instead of kernel launches, the SuperMann decision taken by
// thread 0 between them.  A launch with one block per instance solves a
// whole batch in one persistent launch: no host decisions, no graph
// replays, no grid-wide phase boundaries.  Meant for small instances, whose
// iterations are otherwise bound by launch and phase latency.
#include <cstdint>

#include "batch.cuh"
#include "kernels.cuh"
#include "ops_body.cuh"
#include "riccati_body.cuh"
#include "rounds_body.cuh"
#include "spock_internal.h"

namespace spock {

// T(Vt) -> TVt with the residual statistics (direction d), in one block.
template <typename S, int J, int SL>
__device__ __forceinline__ void cta_eval(const KP<S>& p, const BInst<S>& b) {
  const int64_t nz = p.n_z;
  lstar_body<S, LS_PREP, J>(p, 0, 1, b.Vt + nz, b.Vt, b.TVt);
  __syncthreads();
  const bool chains = p.n_chains > 0 && p.chain_stage < p.N;
  if (chains) {
    bwd_chain_body<S, SL>(p, 0, 1);
    __syncthreads();
  }
  for (int t = p.chain_stage - 1; t >= 0; --t) {
    bwd_stage_body<S, SL>(p, t, 0, 1);
    __syncthreads();
  }
  for (int t = 0; t < p.chain_stage; ++t) {
    fwd_stage_body<S, SL>(p, t, b.TVt, 0, 1);
    __syncthreads();
  }
  if (chains) {
    fwd_chain_body<S, SL>(p, b.TVt, 0, 1);
    __syncthreads();
  }
  dual_fused_body<S, true, J>(p, 0, 1, b.Vt, b.TVt, b.Vt + nz, b.TVt + nz, b.d, b.pd);
  __syncthreads();
  reduce_stats_body(b.pd, 1, nullptr, 0, b.stats, p.skip);
  __syncthreads();
}

// Block i solves instance i: T of the starting point, then rounds until the
// state says done or max_rounds rounds have run.  `trace` (or NULL) records
// the SuperMann branches of a single-instance solve.
template <typename S, int J, int SL, int MEM>
__global__ void __launch_bounds__(128) k_solve_cta(const BInst<S>* __restrict__ bi, int64_t max_rounds,
                                                   int32_t* trace) {
  const BInst<S>& b = bi[blockIdx.x];
  const KP<S> p = b.kp;
  SmState* st = b.st;
  cta_eval<S, J, SL>(p, b);
  for (int64_t r = 0; r < max_rounds; ++r) {
    if (threadIdx.x == 0) round_decide_body(st, b.stats, trace);
    __syncthreads();
    // an accepted point is committed even when the decision ends the solve:
    // the returned pair is the last accepted (v, T(v))
    round_commit_body<S, MEM>(st, b.V, b.TV, b.Vt, b.TVt, b.MR, b.D, b.n_v, b.ld, b.paa, 0, 1);
    __syncthreads();
    if (*reinterpret_cast<volatile int32_t*>(&st->done)) break;
    round_aa_solve_body(st, b.paa, 1);
    __syncthreads();
    round_point_body<S, MEM>(st, b.V, b.TV, b.Vt, b.TVt, b.d, b.D, b.n_v, b.ld, 0, 1);
    __syncthreads();
    cta_eval<S, J, SL>(p, b);
  }
}

// Lane layouts: nx + nu <= 30 (J = SL = 1) or <= 62 (J = SL = 2); Anderson
// memory 0, 3 (the paper's) or 5.
bool cta_supported(int nx, int nu, int mem) {
  return nx + nu <= 62 && (mem == 0 || mem == 3 || mem == 5);
}

template <typename S>
void launch_solve_cta(const BInst<S>* bi, int n_inst, int max_nxu, int mem, int64_t max_rounds, int32_t* trace,
                      cudaStream_t st) {
  const bool small = max_nxu <= 30;
#define SPOCK_CTA(M)                                                                              \
  if (small) k_solve_cta<S, 1, 1, M><<<n_inst, 128, 0, st>>>(bi, max_rounds, trace);            \
  else k_solve_cta<S, 2, 2, M><<<n_inst, 128, 0, st>>>(bi, max_rounds, trace);
  if (mem == 0) {
    SPOCK_CTA(0)
  } else if (mem == 3) {
    SPOCK_CTA(3)
  } else {
    SPOCK_CTA(5)
  }
#undef SPOCK_CTA
}

template void launch_solve_cta<double>(const BInst<double>*, int, int, int, int64_t, int32_t*, cudaStream_t);
template void launch_solve_cta<float>(const BInst<float>*, int, int, int, int64_t, int32_t*, cudaStream_t);

}  // namespace spock
