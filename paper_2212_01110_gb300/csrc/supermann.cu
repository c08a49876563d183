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
    st->tol = fmax(st->eps_abs, st->eps_rel * xi);
    st->initialized = 1;
  }
  st->omega = omega;
  st->xi = xi;
  if (!isfinite(om2) || !isfinite(xi)) {
    st->action = A_NUMERICAL;
  } else if (xi <= st->tol) {
    st->action = A_DONE;
  } else if (st->k >= st->max_iter) {
    st->action = A_MAXIT;
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
// Block partials: [0, cnt) = <M^R_j, M^R_slot>, [kMaxMemory, kMaxMemory+cnt)
// = <M^R_j, r> (j over the stored slots, the new column included).
template <typename S>
__global__ void __launch_bounds__(256) k_aa_update(const S* __restrict__ v, const S* __restrict__ Tv,
                                                   const S* __restrict__ vp, const S* __restrict__ Tvp,
                                                   S* __restrict__ MR, S* __restrict__ D, int64_t n, int slot,
                                                   int cnt, double* __restrict__ partials) {
  // Dot products: terms in the working precision, summed over chunks of 8
  // grid-stride steps in S, then accumulated in FP64.
  double gr[kMaxMemory], rh[kMaxMemory];
  S cg[kMaxMemory], cr[kMaxMemory];
#pragma unroll
  for (int j = 0; j < kMaxMemory; ++j) {
    gr[j] = rh[j] = 0.0;
    cg[j] = cr[j] = S(0);
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int chunk = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const S r = v[i] - Tv[i];
    const S dc = r - (vp[i] - Tvp[i]);
    const S dv = v[i] - vp[i];
    MR[(int64_t)slot * n + i] = dc;
    D[(int64_t)slot * n + i] = dv - dc;
#pragma unroll
    for (int j = 0; j < kMaxMemory; ++j) {
      if (j < cnt) {
        const S c = (j == slot) ? dc : MR[(int64_t)j * n + i];
        cg[j] += c * dc;
        cr[j] += c * r;
      }
    }
    if (++chunk == 8) {
      chunk = 0;
#pragma unroll
      for (int j = 0; j < kMaxMemory; ++j) {
        if (j < cnt) {
          gr[j] += (double)cg[j];
          rh[j] += (double)cr[j];
          cg[j] = cr[j] = S(0);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kMaxMemory; ++j) {
    if (j < cnt) {
      gr[j] += (double)cg[j];
      rh[j] += (double)cr[j];
    }
  }
  __shared__ double red[8][2 * kMaxMemory];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kMaxMemory; ++j) {
    if (j < cnt) {
      const double a = warp_sum(gr[j]), b = warp_sum(rh[j]);
      if (lane == 0) {
        red[w][j] = a;
        red[w][kMaxMemory + j] = b;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * kMaxMemory) {
    const int j = threadIdx.x % kMaxMemory;
    double s = 0.0;
    if (j < cnt)
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s += red[ww][threadIdx.x];
    partials[(int64_t)blockIdx.x * 2 * kMaxMemory + threadIdx.x] = s;
  }
}

// Reduces the partials, updates the Gram matrix and solves for gamma.
// order[] lists the stored slots from newest to oldest.
struct SlotOrder {
  int32_t s[kMaxMemory];
};

__global__ void k_aa_solve(SmState* st, const double* __restrict__ partials, int nblocks, int slot, int cnt,
                           SlotOrder order) {
  __shared__ double sums[2 * kMaxMemory];
  const int t = threadIdx.x;
  if (t < 2 * kMaxMemory) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * 2 * kMaxMemory + t];
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

template <typename S>
void launch_aa_update(SmState* st, const S* v, const S* Tv, const S* vp, const S* Tvp, S* MR, S* D, int64_t n,
                      int slot, int cnt, int order[kMaxMemory], double* partials, int grid, cudaStream_t s) {
  k_aa_update<S><<<grid, 256, 0, s>>>(v, Tv, vp, Tvp, MR, D, n, slot, cnt, partials);
  SlotOrder o;
  for (int j = 0; j < kMaxMemory; ++j) o.s[j] = order[j];
  k_aa_solve<<<1, 64, 0, s>>>(st, partials, grid, slot, cnt, o);
}

template <typename S>
__global__ void __launch_bounds__(256) k_aa_direction(const SmState* __restrict__ st, const S* __restrict__ v,
                                                      const S* __restrict__ Tv, const S* __restrict__ D, int64_t n,
                                                      int cnt, S* __restrict__ d, S* __restrict__ vt) {
  S g[kMaxMemory];
#pragma unroll
  for (int j = 0; j < kMaxMemory; ++j) g[j] = (j < cnt) ? (S)st->gamma[j] : S(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const S vi = v[i];
    S di = -(vi - Tv[i]);
#pragma unroll
    for (int j = 0; j < kMaxMemory; ++j)
      if (j < cnt) di -= g[j] * D[(int64_t)j * n + i];
    d[i] = di;
    vt[i] = vi + di;
  }
}

template <typename S>
__global__ void __launch_bounds__(256) k_ls_point(const SmState* __restrict__ st, const S* __restrict__ v,
                                                  const S* __restrict__ d, S* __restrict__ vt, int64_t n) {
  const S tau = (S)st->tau;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) vt[i] = v[i] + tau * d[i];
}

template <typename S>
__global__ void __launch_bounds__(256) k_k2_point(const SmState* __restrict__ st, const S* __restrict__ v,
                                                  const S* __restrict__ vt, const S* __restrict__ Tvt,
                                                  S* __restrict__ vn, int64_t n) {
  const S c = (S)st->coef;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    vn[i] = v[i] - c * (vt[i] - Tvt[i]);
}

template <typename S>
__global__ void __launch_bounds__(256) k_km_point(const SmState* __restrict__ st, const S* __restrict__ v,
                                                  const S* __restrict__ Tv, S* __restrict__ vn, int64_t n) {
  const S c = (S)st->lam;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    vn[i] = v[i] - c * (v[i] - Tv[i]);
}

template <typename S>
void launch_aa_direction(const SmState* st, const S* v, const S* Tv, const S* D, int64_t n, int cnt, S* d, S* vt,
                         int grid, cudaStream_t s) {
  k_aa_direction<S><<<grid, 256, 0, s>>>(st, v, Tv, D, n, cnt, d, vt);
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
  template void launch_aa_update<S>(SmState*, const S*, const S*, const S*, const S*, S*, S*, int64_t, int,  \
                                    int, int*, double*, int, cudaStream_t);                                   \
  template void launch_aa_direction<S>(const SmState*, const S*, const S*, const S*, int64_t, int, S*, S*,    \
                                       int, cudaStream_t);                                                    \
  template void launch_ls_point<S>(const SmState*, const S*, const S*, S*, int64_t, int, cudaStream_t);       \
  template void launch_k2_point<S>(const SmState*, const S*, const S*, const S*, S*, int64_t, int,            \
                                   cudaStream_t);                                                             \
  template void launch_km_point<S>(const SmState*, const S*, const S*, S*, int64_t, int, cudaStream_t);
SPOCK_INST(double)
SPOCK_INST(float)

}  // namespace spock
