// Device-driven iteration of Algorithm 3 (SPOCK).
//
// The buffers are fixed: (V, TV) the accepted iterate and T of it, (Vt, TVt)
// the point being evaluated and T of it, d the direction, the Anderson columns.
// Each round: k_round_decide reads the statistics of the last evaluation and
// the state, takes the SuperMann decision of Algorithm 3 (same readings as
// supermann.cu) and writes this round's orders; k_round_commit copies an
// accepted (Vt, TVt) into (V, TV) and in the
// same pass writes the new Anderson column and its Gram row; k_round_aa_solve
// solves for gamma; k_round_point forms the next evaluation point in Vt
// (v + d with the Anderson direction, v + tau d, the K2 point, or the relaxed
// step); then T(Vt) is evaluated.  No decision is taken on the host, so a
// run of rounds can be captured in a CUDA graph and replayed.
#include <cmath>

#include "batch.cuh"
#include "kernels.cuh"
#include "rounds_body.cuh"
#include "supermann.cuh"

namespace spock {

__global__ void k_round_decide(SmState* st, const double* __restrict__ stats_t, int32_t* trace) {
  if (threadIdx.x != 0) return;
  round_decide_body(st, stats_t, trace);
}

template <typename S, int MEM>
__global__ void __launch_bounds__(256, 4) k_round_commit(SmState* st, S* __restrict__ V, S* __restrict__ TV,
                                                         const S* __restrict__ Vt, const S* __restrict__ TVt,
                                                         S* __restrict__ MR, S* __restrict__ D, int64_t n,
                                                         int64_t ld, double* __restrict__ partials) {
  round_commit_body<S, MEM>(st, V, TV, Vt, TVt, MR, D, n, ld, partials, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_round_aa_solve(SmState* st, const double* __restrict__ partials,
                                                        int nblocks) {
  round_aa_solve_body(st, partials, nblocks);
}

template <typename S, int MEM>
__global__ void __launch_bounds__(256) k_round_point(const SmState* __restrict__ st, const S* __restrict__ V,
                                                     const S* __restrict__ TV, S* __restrict__ Vt,
                                                     const S* __restrict__ TVt, S* __restrict__ d,
                                                     const S* __restrict__ D, int64_t n, int64_t ld) {
  round_point_body<S, MEM>(st, V, TV, Vt, TVt, d, D, n, ld, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// batched rounds
// ---------------------------------------------------------------------------
template <typename S>
__global__ void k_round_decide_b(const BInst<S>* __restrict__ bi, int n_inst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_inst) round_decide_body(bi[i].st, bi[i].stats, nullptr);
}
template <typename S, int MEM>
__global__ void __launch_bounds__(256, 4) k_round_commit_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const BInst<S>& b = bi[i];
  round_commit_body<S, MEM>(b.st, b.V, b.TV, b.Vt, b.TVt, b.MR, b.D, b.n_v, b.ld, b.paa,
                            blockIdx.x - m.base[i], m.cnt[i]);
}
template <typename S>
__global__ void __launch_bounds__(256) k_round_aa_solve_b(const BInst<S>* __restrict__ bi) {
  const BInst<S>& b = bi[blockIdx.x];
  round_aa_solve_body(b.st, b.paa, b.nb_vec);
}
template <typename S, int MEM>
__global__ void __launch_bounds__(256) k_round_point_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const BInst<S>& b = bi[i];
  round_point_body<S, MEM>(b.st, b.V, b.TV, b.Vt, b.TVt, b.d, b.D, b.n_v, b.ld, blockIdx.x - m.base[i],
                           m.cnt[i]);
}

void launch_round_decide(SmState* st, const double* stats_t, int32_t* trace, cudaStream_t s) {
  k_round_decide<<<1, 32, 0, s>>>(st, stats_t, trace);
}
void launch_round_aa_solve(SmState* st, const double* partials, int nblocks, cudaStream_t s) {
  k_round_aa_solve<<<1, 256, 0, s>>>(st, partials, nblocks);
}

template <typename S>
void launch_round_commit(SmState* st, S* V, S* TV, const S* Vt, const S* TVt, S* MR, S* D,
                         int64_t n, int64_t ld, int mem, double* partials, int grid, cudaStream_t s) {
  switch (mem) {
#define SPOCK_RC(M) \
  case M: k_round_commit<S, M><<<grid, 256, 0, s>>>(st, V, TV, Vt, TVt, MR, D, n, ld, partials); break;
    SPOCK_RC(0) SPOCK_RC(1) SPOCK_RC(2) SPOCK_RC(3) SPOCK_RC(4) SPOCK_RC(5) SPOCK_RC(6) SPOCK_RC(7) SPOCK_RC(8)
    SPOCK_RC(9) SPOCK_RC(10) SPOCK_RC(11) SPOCK_RC(12) SPOCK_RC(13) SPOCK_RC(14) SPOCK_RC(15) SPOCK_RC(16)
#undef SPOCK_RC
    default: break;
  }
}
template <typename S>
void launch_round_point(SmState* st, const S* V, const S* TV, S* Vt, const S* TVt, S* d, const S* D, int64_t n,
                        int64_t ld, int mem, int grid, cudaStream_t s) {
  switch (mem) {
#define SPOCK_RP(M) case M: k_round_point<S, M><<<grid, 256, 0, s>>>(st, V, TV, Vt, TVt, d, D, n, ld); break;
    SPOCK_RP(0) SPOCK_RP(1) SPOCK_RP(2) SPOCK_RP(3) SPOCK_RP(4) SPOCK_RP(5) SPOCK_RP(6) SPOCK_RP(7) SPOCK_RP(8)
    SPOCK_RP(9) SPOCK_RP(10) SPOCK_RP(11) SPOCK_RP(12) SPOCK_RP(13) SPOCK_RP(14) SPOCK_RP(15) SPOCK_RP(16)
#undef SPOCK_RP
    default: break;
  }
}

template <typename S>
void launch_round_decide_b(const BInst<S>* bi, int n_inst, cudaStream_t st) {
  k_round_decide_b<S><<<(n_inst + 63) / 64, 64, 0, st>>>(bi, n_inst);
}
template <typename S>
void launch_round_aa_solve_b(const BInst<S>* bi, int n_inst, cudaStream_t st) {
  k_round_aa_solve_b<S><<<n_inst, 256, 0, st>>>(bi);
}
template <typename S>
void launch_round_commit_b(const BInst<S>* bi, const BMap& m, int nblocks, int mem, cudaStream_t st) {
  switch (mem) {
#define SPOCK_RC(M) case M: k_round_commit_b<S, M><<<nblocks, 256, 0, st>>>(bi, m); break;
    SPOCK_RC(0) SPOCK_RC(1) SPOCK_RC(2) SPOCK_RC(3) SPOCK_RC(4) SPOCK_RC(5) SPOCK_RC(6) SPOCK_RC(7) SPOCK_RC(8)
    SPOCK_RC(9) SPOCK_RC(10) SPOCK_RC(11) SPOCK_RC(12) SPOCK_RC(13) SPOCK_RC(14) SPOCK_RC(15) SPOCK_RC(16)
#undef SPOCK_RC
    default: break;
  }
}
template <typename S>
void launch_round_point_b(const BInst<S>* bi, const BMap& m, int nblocks, int mem, cudaStream_t st) {
  switch (mem) {
#define SPOCK_RP(M) case M: k_round_point_b<S, M><<<nblocks, 256, 0, st>>>(bi, m); break;
    SPOCK_RP(0) SPOCK_RP(1) SPOCK_RP(2) SPOCK_RP(3) SPOCK_RP(4) SPOCK_RP(5) SPOCK_RP(6) SPOCK_RP(7) SPOCK_RP(8)
    SPOCK_RP(9) SPOCK_RP(10) SPOCK_RP(11) SPOCK_RP(12) SPOCK_RP(13) SPOCK_RP(14) SPOCK_RP(15) SPOCK_RP(16)
#undef SPOCK_RP
    default: break;
  }
}
#define SPOCK_RB_INST(S)                                                                          \
  template void launch_round_decide_b<S>(const BInst<S>*, int, cudaStream_t);                     \
  template void launch_round_aa_solve_b<S>(const BInst<S>*, int, cudaStream_t);                   \
  template void launch_round_commit_b<S>(const BInst<S>*, const BMap&, int, int, cudaStream_t);   \
  template void launch_round_point_b<S>(const BInst<S>*, const BMap&, int, int, cudaStream_t);
SPOCK_RB_INST(double)
SPOCK_RB_INST(float)
#undef SPOCK_RB_INST

template void launch_round_commit<double>(SmState*, double*, double*, const double*, const double*, double*,
                                          double*, int64_t, int64_t, int, double*, int, cudaStream_t);
template void launch_round_commit<float>(SmState*, float*, float*, const float*, const float*, float*, float*,
                                         int64_t, int64_t, int, double*, int, cudaStream_t);
template void launch_round_point<double>(SmState*, const double*, const double*, double*, const double*, double*,
                                         const double*, int64_t, int64_t, int, int, cudaStream_t);
template void launch_round_point<float>(SmState*, const float*, const float*, float*, const float*, float*,
                                        const float*, int64_t, int64_t, int, int, cudaStream_t);

}  // namespace spock
