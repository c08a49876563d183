// SuperMann decisions (Algorithm 3) and Anderson directions (Sec.
// "Anderson's acceleration") on the device.
//
// Readings of Algorithm 3 implemented here:
//  * each iteration first has r = v - T(v), omega = ||r||_M and xi; the
//    termination test, then the Anderson update with c = r, then K0 or the
//    line search; after K1 the trial residual is reused;
//  * rho = omega~^2 - rho_coef <r~, v~ - v>_M with rho_coef = 1 (SuperMann's
//    averagedness 1/2 of a firmly nonexpansive T times 2);
//  * the line search stops after max_backtracks reductions with tau = 0,
//    i.e. the relaxed step v - lambda r (K2 with v~ = v);
//  * Anderson memory m counts difference columns; gamma solves the normal
//    equations of min ||M^R gamma - c|| in FP64 by Cholesky; if the Gram
//    matrix is numerically singular the oldest columns are left out of
//    that solve.
// Scalars are FP64 in every precision mode; vectors follow the mode.
#include <cmath>

#include "kernels.cuh"
#include "supermann.cuh"

namespace spock {

__device__ void trace_put(SmState* st, int32_t* trace, int branch, int nb) {
  if (st->record_trace && trace && st->k < st->max_iter) {
    trace[2 * st->k] = branch;
    trace[2 * st->k + 1] = nb;
  }
}

__global__ void k_sm_after_eval(SmState* st, const double* __restrict__ stats, int32_t* trace) {
  if (threadIdx.x != 0) return;
  const double om2 = stats[ST_RZ2] + stats[ST_RE2] - 2.0 * st->alpha * stats[ST_RE_LRZ];
  const double omega = sqrt(fmax(om2, 0.0));
  const double xi = fmax(stats[ST_XIP], stats[ST_XID]);
  if (!st->initialized) {
    st->zeta = omega;
    st->omega_safe = omega;
    st->xi0 = xi;
    if (!(st->tol > 0.0)) st->tol = fmax(st->eps_abs, st->eps_rel * xi);  // tol > 0: given by the host
    st->best_xi = xi;
    st->best_k = 0;
    st->initialized = 1;
  }
  st->omega = omega;
  st->xi = xi;
  if (xi < 0.5 * st->best_xi) {
    st->best_xi = xi;
    st->best_k = st->k;
  }
  if (!isfinite(om2) || !isfinite(xi)) {
    st->action = A_NUMERICAL;
  } else if (xi <= st->tol) {
    st->action = A_DONE;
  } else if (st->k >= st->max_iter) {
    st->action = A_MAXIT;
  } else if (st->stall_window > 0 && st->k - st->best_k > st->stall_window && xi <= 30.0 * st->tol) {
    // no halving of xi for stall_window iterations close to the tolerance:
    // the FP32 operator's rounding floor, hand over to FP64
    st->action = A_STALL;
  } else if (omega <= st->c0 * st->zeta) {
    st->action = A_K0;  // blind step v + d; zeta_{k+1} = omega_k
    st->zeta = omega;
    trace_put(st, trace, 0, 0);
    st->n_k0++;
    st->k++;
  } else {
    st->action = A_LS;
    st->tau = 1.0;
    st->nb = 0;
  }
}

__global__ void k_sm_line_search(SmState* st, const double* __restrict__ stats, int32_t* trace) {
  if (threadIdx.x != 0) return;
  const double om2 = stats[ST_RZ2] + stats[ST_RE2] - 2.0 * st->alpha * stats[ST_RE_LRZ];
  const double omt = sqrt(fmax(om2, 0.0));
  st->omega_t = omt;
  if (!isfinite(om2)) {
    st->action = A_NUMERICAL;
    return;
  }
  const double omega = st->omega;
  if (omega <= st->omega_safe && omt <= st->c1 * omega) {
    st->action = A_K1;  // educated step: accept v~
    st->omega_safe = omt + pow(st->c2, (double)st->k);
    trace_put(st, trace, 1, st->nb);
    st->n_k1++;
    st->k++;
    return;
  }
  // <r~, v~ - v>_M = tau <r~, d>_M,  <a, b>_M = a.b - alpha (<L a_z, b_eta> + <a_eta, L b_z>)
  const double rdM = stats[ST_RD] - st->alpha * (stats[ST_LRZ_DE] + stats[ST_RE_LDZ]);
  const double rho = om2 - st->rho_coef * st->tau * rdM;
  st->rho = rho;
  if (rho >= st->sigma * omt * omega && omt > 0.0) {
    st->action = A_K2;  // safeguard step: projection on the separating hyperplane
    st->coef = st->lam * rho / (omt * omt);
    trace_put(st, trace, 2, st->nb);
    st->n_k2++;
    st->k++;
    return;
  }
  st->nb++;
  st->n_back++;
  st->tau *= st->beta;
  if (st->nb >= st->max_back) {
    st->action = A_CAP;
    trace_put(st, trace, 3, st->nb);
    st->n_cap++;
    st->k++;
  } else {
    st->action = A_RETRY;
  }
}

void sm_init_state(SmState* st_dev, const SmState& h, cudaStream_t s) {
  cudaMemcpyAsync(st_dev, &h, sizeof(SmState), cudaMemcpyHostToDevice, s);
}
void launch_sm_after_eval(SmState* st, const double* stats, int32_t* trace, cudaStream_t s) {
  k_sm_after_eval<<<1, 32, 0, s>>>(st, stats, trace);
}
void launch_sm_line_search(SmState* st, const double* stats, int32_t* trace, cudaStream_t s) {
  k_sm_line_search<<<1, 32, 0, s>>>(st, stats, trace);
}

// ---------------------------------------------------------------------------
// Anderson
// ---------------------------------------------------------------------------
// Streaming kernels move 16 bytes per load (float4 / double2); every vector
// and every Anderson column starts on a 256-byte boundary (column stride
// `ld` padded by the host), so only the tail of a vector is scalar.
template <typename S>
struct Pack;
template <>
struct Pack<float> {
  using T = float4;
  static constexpr int N = 4;
};
template <>
struct Pack<double> {
  using T = double2;
  static constexpr int N = 2;
};
template <typename S>
__device__ __forceinline__ S& pk(typename Pack<S>::T& v, int e) {
  return reinterpret_cast<S*>(&v)[e];
}
template <typename S>
__device__ __forceinline__ typename Pack<S>::T ldp(const S* p, int64_t q) {
  return reinterpret_cast<const typename Pack<S>::T*>(p)[q];
}
template <typename S>
__device__ __forceinline__ void stp(S* p, int64_t q, const typename Pack<S>::T& v) {
  reinterpret_cast<typename Pack<S>::T*>(p)[q] = v;
}
// Block partials: [0, cnt) = <M^R_j, M^R_slot>, [kMaxMemory, kMaxMemory+cnt)
// = <M^R_j, r> (j over the stored slots, the new column included).
template <typename S, int CNT>
__global__ void __launch_bounds__(256, 4) k_aa_update(const S* __restrict__ v, const S* __restrict__ Tv,
                                                      const S* __restrict__ vp, const S* __restrict__ Tvp,
                                                      S* __restrict__ MR, S* __restrict__ D, int64_t n, int64_t ld,
                                                      int slot, double* __restrict__ partials) {
  // Writes column `slot` of M^R and of D = M^P - M^R and accumulates
  // <M^R_j, new column> and <M^R_j, r>: terms in the working precision, one
  // pack at a time, added into FP64 per pack.  CNT (stored columns, the new
  // one included) is a template parameter so the accumulators stay in
  // registers.
  constexpr int NP = Pack<S>::N;
  using PT = typename Pack<S>::T;
  double gr[CNT], rh[CNT];
#pragma unroll
  for (int j = 0; j < CNT; ++j) gr[j] = rh[j] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t npack = n / NP;
  S* mrs = MR + (int64_t)slot * ld;
  S* ds = D + (int64_t)slot * ld;
  for (int64_t q = gt; q < npack; q += stride) {
    PT a = ldp(v, q), b = ldp(Tv, q), c = ldp(vp, q), e = ldp(Tvp, q);
    PT rr, dc, dd;
#pragma unroll
    for (int t = 0; t < NP; ++t) {
      pk<S>(rr, t) = pk<S>(a, t) - pk<S>(b, t);
      pk<S>(dc, t) = pk<S>(rr, t) - (pk<S>(c, t) - pk<S>(e, t));
      pk<S>(dd, t) = (pk<S>(a, t) - pk<S>(c, t)) - pk<S>(dc, t);
    }
    stp(mrs, q, dc);
    stp(ds, q, dd);
#pragma unroll
    for (int j = 0; j < CNT; ++j) {
      PT col = (j == slot) ? dc : ldp(MR + (int64_t)j * ld, q);
      S g = 0, h = 0;
#pragma unroll
      for (int t = 0; t < NP; ++t) {
        g += pk<S>(col, t) * pk<S>(dc, t);
        h += pk<S>(col, t) * pk<S>(rr, t);
      }
      gr[j] += (double)g;
      rh[j] += (double)h;
    }
  }
  for (int64_t i = npack * NP + gt; i < n; i += stride) {  // tail
    const S r = v[i] - Tv[i];
    const S dc = r - (vp[i] - Tvp[i]);
    mrs[i] = dc;
    ds[i] = (v[i] - vp[i]) - dc;
#pragma unroll
    for (int j = 0; j < CNT; ++j) {
      const S c = (j == slot) ? dc : MR[(int64_t)j * ld + i];
      gr[j] += (double)(c * dc);
      rh[j] += (double)(c * r);
    }
  }
  __shared__ double red[8][2 * kMaxMemory];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < CNT; ++j) {
    const double a = warp_sum(gr[j]), b = warp_sum(rh[j]);
    if (lane == 0) {
      red[w][j] = a;
      red[w][kMaxMemory + j] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * kMaxMemory) {
    const int j = threadIdx.x % kMaxMemory;
    double s = 0.0;
    if (j < CNT)
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s += red[ww][threadIdx.x];
    partials[(int64_t)blockIdx.x * 2 * kMaxMemory + threadIdx.x] = s;
  }
}

// Reduces the partials, updates the Gram matrix and solves for gamma.
// order[] lists the stored slots from newest to oldest.
struct SlotOrder {
  int32_t s[kMaxMemory];
};

__global__ void __launch_bounds__(256) k_aa_solve(SmState* st, const double* __restrict__ partials, int nblocks,
                                                  int slot, int cnt, SlotOrder order) {
  // 256 threads: value t % 32 of the block partials, blocks t / 32, t / 32 + 8, ...
  __shared__ double part[8][2 * kMaxMemory];
  __shared__ double sums[2 * kMaxMemory];
  const int t = threadIdx.x;
  {
    const int val = t & 31, grp = t >> 5;
    double s = 0.0;
    for (int b = grp; b < nblocks; b += 8) s += partials[(int64_t)b * 2 * kMaxMemory + val];
    part[grp][val] = s;
  }
  __syncthreads();
  if (t < 2 * kMaxMemory) {
    double s = 0.0;
    for (int g = 0; g < 8; ++g) s += part[g][t];
    sums[t] = s;
  }
  __syncthreads();
  if (t != 0) return;
  const int M = kMaxMemory;
  for (int j = 0; j < cnt; ++j) {
    st->G[slot * M + j] = sums[j];
    st->G[j * M + slot] = sums[j];
    st->rhs[j] = sums[M + j];
  }
  for (int j = 0; j < M; ++j) st->gamma[j] = 0.0;
  // Cholesky on the newest `use` columns; drop the oldest ones while the
  // Gram matrix is numerically singular.
  st->aa_dropped = 0;
  for (int use = cnt; use >= 1; --use) {
    double Lm[kMaxMemory * kMaxMemory];
    double maxd = 0.0;
    for (int a = 0; a < use; ++a) maxd = fmax(maxd, st->G[order.s[a] * M + order.s[a]]);
    bool ok = maxd > 0.0;
    for (int a = 0; a < use && ok; ++a) {
      for (int b = 0; b <= a; ++b) {
        double s = st->G[order.s[a] * M + order.s[b]];
        for (int c = 0; c < b; ++c) s -= Lm[a * M + c] * Lm[b * M + c];
        if (a == b) {
          if (!(s > 1e-13 * maxd)) { ok = false; break; }
          Lm[a * M + a] = sqrt(s);
        } else {
          Lm[a * M + b] = s / Lm[b * M + b];
        }
      }
    }
    if (!ok) {
      st->aa_dropped++;
      continue;
    }
    double y[kMaxMemory];
    for (int a = 0; a < use; ++a) {
      double s = st->rhs[order.s[a]];
      for (int c = 0; c < a; ++c) s -= Lm[a * M + c] * y[c];
      y[a] = s / Lm[a * M + a];
    }
    for (int a = use - 1; a >= 0; --a) {
      double s = y[a];
      for (int c = a + 1; c < use; ++c) s -= Lm[c * M + a] * y[c];
      y[a] = s / Lm[a * M + a];
    }
    for (int a = 0; a < use; ++a) st->gamma[order.s[a]] = y[a];
    break;
  }
}

template <typename S, int CNT>
static void aa_update_cnt(const S* v, const S* Tv, const S* vp, const S* Tvp, S* MR, S* D, int64_t n, int64_t ld,
                          int slot, double* partials, int grid, cudaStream_t s) {
  k_aa_update<S, CNT><<<grid, 256, 0, s>>>(v, Tv, vp, Tvp, MR, D, n, ld, slot, partials);
}

template <typename S>
void launch_aa_update(SmState* st, const S* v, const S* Tv, const S* vp, const S* Tvp, S* MR, S* D, int64_t n,
                      int64_t ld, int slot, int cnt, int order[kMaxMemory], double* partials, int grid,
                      cudaStream_t s) {
  switch (cnt) {
#define SPOCK_AA_CASE(C) \
  case C: aa_update_cnt<S, C>(v, Tv, vp, Tvp, MR, D, n, ld, slot, partials, grid, s); break;
    SPOCK_AA_CASE(1) SPOCK_AA_CASE(2) SPOCK_AA_CASE(3) SPOCK_AA_CASE(4) SPOCK_AA_CASE(5) SPOCK_AA_CASE(6)
    SPOCK_AA_CASE(7) SPOCK_AA_CASE(8) SPOCK_AA_CASE(9) SPOCK_AA_CASE(10) SPOCK_AA_CASE(11) SPOCK_AA_CASE(12)
    SPOCK_AA_CASE(13) SPOCK_AA_CASE(14) SPOCK_AA_CASE(15) SPOCK_AA_CASE(16)
#undef SPOCK_AA_CASE
    default: return;
  }
  SlotOrder o;
  for (int j = 0; j < kMaxMemory; ++j) o.s[j] = order[j];
  k_aa_solve<<<1, 256, 0, s>>>(st, partials, grid, slot, cnt, o);
}

template <typename S, int CNT>
__global__ void __launch_bounds__(256) k_aa_direction(const SmState* __restrict__ st, const S* __restrict__ v,
                                                      const S* __restrict__ Tv, const S* __restrict__ D, int64_t n,
                                                      int64_t ld, S* __restrict__ d, S* __restrict__ vt) {
  constexpr int NP = Pack<S>::N;
  using PT = typename Pack<S>::T;
  S g[CNT > 0 ? CNT : 1];
#pragma unroll
  for (int j = 0; j < CNT; ++j) g[j] = (S)st->gamma[j];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t npack = n / NP;
  for (int64_t q = gt; q < npack; q += stride) {
    PT a = ldp(v, q), b = ldp(Tv, q), dd;
#pragma unroll
    for (int t = 0; t < NP; ++t) pk<S>(dd, t) = pk<S>(b, t) - pk<S>(a, t);
#pragma unroll
    for (int j = 0; j < CNT; ++j) {
      PT c = ldp(D + (int64_t)j * ld, q);
#pragma unroll
      for (int t = 0; t < NP; ++t) pk<S>(dd, t) -= g[j] * pk<S>(c, t);
    }
    PT w;
#pragma unroll
    for (int t = 0; t < NP; ++t) pk<S>(w, t) = pk<S>(a, t) + pk<S>(dd, t);
    stp(d, q, dd);
    stp(vt, q, w);
  }
  for (int64_t i = npack * NP + gt; i < n; i += stride) {
    S di = Tv[i] - v[i];
#pragma unroll
    for (int j = 0; j < CNT; ++j) di -= g[j] * D[(int64_t)j * ld + i];
    d[i] = di;
    vt[i] = v[i] + di;
  }
}

template <typename S>
__global__ void __launch_bounds__(256) k_ls_point(const SmState* __restrict__ st, const S* __restrict__ v,
                                                  const S* __restrict__ d, S* __restrict__ vt, int64_t n) {
  const S tau = (S)st->tau;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int NP = Pack<S>::N;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, npack = n / NP;
  for (int64_t q = gt; q < npack; q += stride) {
    typename Pack<S>::T a = ldp(v, q), b = ldp(d, q);
#pragma unroll
    for (int t = 0; t < NP; ++t) pk<S>(a, t) += tau * pk<S>(b, t);
    stp(vt, q, a);
  }
  for (int64_t i = npack * NP + gt; i < n; i += stride) vt[i] = v[i] + tau * d[i];
}

template <typename S>
__global__ void __launch_bounds__(256) k_k2_point(const SmState* __restrict__ st, const S* __restrict__ v,
                                                  const S* __restrict__ vt, const S* __restrict__ Tvt,
                                                  S* __restrict__ vn, int64_t n) {
  const S c = (S)st->coef;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int NP = Pack<S>::N;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, npack = n / NP;
  for (int64_t q = gt; q < npack; q += stride) {
    typename Pack<S>::T a = ldp(v, q), b = ldp(vt, q), e = ldp(Tvt, q);
#pragma unroll
    for (int t = 0; t < NP; ++t) pk<S>(a, t) -= c * (pk<S>(b, t) - pk<S>(e, t));
    stp(vn, q, a);
  }
  for (int64_t i = npack * NP + gt; i < n; i += stride) vn[i] = v[i] - c * (vt[i] - Tvt[i]);
}

template <typename S>
__global__ void __launch_bounds__(256) k_km_point(const SmState* __restrict__ st, const S* __restrict__ v,
                                                  const S* __restrict__ Tv, S* __restrict__ vn, int64_t n) {
  const S c = (S)st->lam;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int NP = Pack<S>::N;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, npack = n / NP;
  for (int64_t q = gt; q < npack; q += stride) {
    typename Pack<S>::T a = ldp(v, q), b = ldp(Tv, q);
#pragma unroll
    for (int t = 0; t < NP; ++t) pk<S>(a, t) -= c * (pk<S>(a, t) - pk<S>(b, t));
    stp(vn, q, a);
  }
  for (int64_t i = npack * NP + gt; i < n; i += stride) vn[i] = v[i] - c * (v[i] - Tv[i]);
}

template <typename S>
void launch_aa_direction(const SmState* st, const S* v, const S* Tv, const S* D, int64_t n, int64_t ld, int cnt,
                         S* d, S* vt, int grid, cudaStream_t s) {
  switch (cnt) {
#define SPOCK_DIR_CASE(C) \
  case C: k_aa_direction<S, C><<<grid, 256, 0, s>>>(st, v, Tv, D, n, ld, d, vt); break;
    SPOCK_DIR_CASE(0) SPOCK_DIR_CASE(1) SPOCK_DIR_CASE(2) SPOCK_DIR_CASE(3) SPOCK_DIR_CASE(4) SPOCK_DIR_CASE(5)
    SPOCK_DIR_CASE(6) SPOCK_DIR_CASE(7) SPOCK_DIR_CASE(8) SPOCK_DIR_CASE(9) SPOCK_DIR_CASE(10) SPOCK_DIR_CASE(11)
    SPOCK_DIR_CASE(12) SPOCK_DIR_CASE(13) SPOCK_DIR_CASE(14) SPOCK_DIR_CASE(15) SPOCK_DIR_CASE(16)
#undef SPOCK_DIR_CASE
    default: break;
  }
}
template <typename S>
void launch_ls_point(const SmState* st, const S* v, const S* d, S* vt, int64_t n, int grid, cudaStream_t s) {
  k_ls_point<S><<<grid, 256, 0, s>>>(st, v, d, vt, n);
}
template <typename S>
void launch_k2_point(const SmState* st, const S* v, const S* vt, const S* Tvt, S* vn, int64_t n, int grid,
                     cudaStream_t s) {
  k_k2_point<S><<<grid, 256, 0, s>>>(st, v, vt, Tvt, vn, n);
}
template <typename S>
void launch_km_point(const SmState* st, const S* v, const S* Tv, S* vn, int64_t n, int grid, cudaStream_t s) {
  k_km_point<S><<<grid, 256, 0, s>>>(st, v, Tv, vn, n);
}

#define SPOCK_INST(S)                                                                                         \
  template void launch_aa_update<S>(SmState*, const S*, const S*, const S*, const S*, S*, S*, int64_t,       \
                                    int64_t, int, int, int*, double*, int, cudaStream_t);                     \
  template void launch_aa_direction<S>(const SmState*, const S*, const S*, const S*, int64_t, int64_t, int,   \
                                       S*, S*, int, cudaStream_t);                                            \
  template void launch_ls_point<S>(const SmState*, const S*, const S*, S*, int64_t, int, cudaStream_t);       \
  template void launch_k2_point<S>(const SmState*, const S*, const S*, const S*, S*, int64_t, int,            \
                                   cudaStream_t);                                                             \
  template void launch_km_point<S>(const SmState*, const S*, const S*, S*, int64_t, int, cudaStream_t);
SPOCK_INST(double)
SPOCK_INST(float)

}  // namespace spock
