// Gradient of the optimal cost V* = s^0* with respect to x0, the diagonals of
// Q, R, Q_N and the dynamics A, B, from a converged pair (z*, eta*).
//
// At the saddle point of  s^0 + lambda^T (G z_1 - h) + mu^T M z_2 + <eta, Lz>
// - g*(eta)  (the splitting of Sec. "Operator splitting" with the dynamics
// G z_1 = h of S1 and the kernel M z_2 = 0 of S2 dualised), z-stationarity
// gives G^T lambda = -(L* eta*)_{z_1}, and dV*/dtheta is the partial
// derivative of the Lagrangian (envelope theorem).  Writing w = L* eta*,
// the x-rows of G^T lambda = -w_{z_1} give, from the leaves up,
//   lambda^j = -w_x^j (leaves),
//   lambda^i = sum_c A^cT lambda^c - w_x^i
//            = sum_c Abar^cT lambda^c - K^iT (sum_c B^cT lambda^c) - w_x^i
// (A^c = Abar^c - B^c K^i), i.e. the Riccati backward GEMV on the stored
// [Abar^c | B^c] blocks followed by a K^T product.  Then
//   dV/dx0 = -lambda^0, dV/dA^c = -lambda^c x^anc(c)T, dV/dB^c = -lambda^c u^anc(c)T,
//   dV/dQ^c_kk = eta*_{c,Qx,k} x^anc_k / (2 sqrt Q^c_kk)  (likewise R, Q_N).
#include "kernels.cuh"
#include "spock_internal.h"

namespace spock {

// lambda for the nonleaf nodes of stage t (warp per node); lam has stride xs.
template <typename S, int SL>
__global__ void __launch_bounds__(128) k_lambda_stage(KP<S> p, int t, const S* __restrict__ w, S* __restrict__ lam) {
  __shared__ S lv[kWarpsPerBlock][kVecPad];
  __shared__ S hv[kWarpsPerBlock][kVecPad];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nx = p.nx, nu = p.nu, ncol = nx + nu;
  const int b0 = p.stage_begin[t], cnt = p.stage_begin[t + 1] - b0;
  S* lc = lv[wl];
  S* hs = hv[wl];
  for (int idx = gw; idx < cnt; idx += nw) {
    const int k = b0 + idx;
    const NodeDesc D = p.desc[k];
    S h[SL];
#pragma unroll
    for (int s = 0; s < SL; ++s) h[s] = S(0);
    for (int j = 0; j < D.m; ++j) {
      const int c = D.c0 + j;
      if (c >= p.nl) {
        const int64_t zxc = p.desc[c].zx;
        for (int r = lane; r < nx; r += 32) lc[r] = -w[zxc + r];
      } else {
        for (int r = lane; r < nx; r += 32) lc[r] = lam[(int64_t)c * p.xs + r];
      }
      __syncwarp();
      const S* G = p.Gb + (int64_t)(c - 1) * p.gstride;
      for (int r = 0; r < nx; ++r) {
        const S lr = lc[r];
#pragma unroll
        for (int s = 0; s < SL; ++s) {
          const int col = 32 * s + lane;
          if (col < ncol) h[s] += G[(int64_t)r * ncol + col] * lr;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int col = 32 * s + lane;
      if (col < ncol) hs[col] = h[s];
    }
    __syncwarp();
    const S* Km = p.NB + (int64_t)k * p.nbstride;  // K: nu x nx
    for (int r = lane; r < nx; r += 32) {
      S acc = hs[r] - w[D.zx + r];
      for (int b = 0; b < nu; ++b) acc -= Km[b * nx + r] * hs[nx + b];
      lam[(int64_t)k * p.xs + r] = acc;
    }
    __syncwarp();
  }
}

// Gradients (FP64 outputs in the caller's node numbering), warp per node.
template <typename S>
__global__ void __launch_bounds__(128) k_gradients(KP<S> p, const S* __restrict__ z, const S* __restrict__ eta,
                                                   const S* __restrict__ w, const S* __restrict__ lam,
                                                   double* gx0, double* gA, double* gB, double* gQ, double* gR,
                                                   double* gQN) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nx = p.nx, nu = p.nu;
  for (int k = gw; k < p.n; k += nw) {
    const NodeDesc D = p.desc[k];
    const int64_t u = D.user;
    // lambda^k (leaves: -w_x)
    auto lamk = [&](int r) -> double {
      return k < p.nl ? (double)lam[(int64_t)k * p.xs + r] : -(double)w[D.zx + r];
    };
    if (k == 0 && gx0)
      for (int r = lane; r < nx; r += 32) gx0[r] = -lamk(r);
    if (k > 0) {
      if (gA)
        for (int e = lane; e < nx * nx; e += 32) {
          const int r = e / nx, c = e % nx;
          gA[u * nx * nx + e] = -lamk(r) * (double)z[D.zxp + c];
        }
      if (gB)
        for (int e = lane; e < nx * nu; e += 32) {
          const int r = e / nu, c = e % nu;
          gB[u * nx * nu + e] = -lamk(r) * (double)z[D.zup + c];
        }
      if (gQ)
        for (int r = lane; r < nx; r += 32)
          gQ[u * nx + r] = (double)eta[D.enr + r] * (double)z[D.zxp + r] / (2.0 * (double)p.qs[(int64_t)k * nx + r]);
      if (gR)
        for (int r = lane; r < nu; r += 32)
          gR[u * nu + r] =
              (double)eta[D.enr + nx + r] * (double)z[D.zup + r] / (2.0 * (double)p.rs[(int64_t)k * nu + r]);
    }
    if (k >= p.nl && gQN)
      for (int r = lane; r < nx; r += 32)
        gQN[u * nx + r] =
            (double)eta[D.elf + nx + r] * (double)z[D.zx + r] / (2.0 * (double)p.qns[(int64_t)k * nx + r]);
  }
}

// Multipliers of the dynamics for a right-hand side -w_1: the solution of
// G^T lambda = -w_{z_1} by the tree recursion above (leaves lambda = -w_x,
// not stored); lam [nonleaf][xs].
template <typename S>
int launch_lambda(const KP<S>& p, const std::vector<int32_t>& stage_begin, const S* w, S* lam, int max_blocks,
                  cudaStream_t st) {
  const int sl = (p.nx + p.nu + 31) / 32;
  int launches = 0;
  for (int t = p.N - 1; t >= 0; --t) {
    const int cnt = stage_begin[t + 1] - stage_begin[t];
    const int grid = std::max(1, std::min((cnt + kWarpsPerBlock - 1) / kWarpsPerBlock, max_blocks));
    switch (sl) {
      case 1: k_lambda_stage<S, 1><<<grid, 128, 0, st>>>(p, t, w, lam); break;
      case 2: k_lambda_stage<S, 2><<<grid, 128, 0, st>>>(p, t, w, lam); break;
      case 3: k_lambda_stage<S, 3><<<grid, 128, 0, st>>>(p, t, w, lam); break;
      default: k_lambda_stage<S, 4><<<grid, 128, 0, st>>>(p, t, w, lam); break;
    }
    ++launches;
  }
  return launches;
}
template int launch_lambda<double>(const KP<double>&, const std::vector<int32_t>&, const double*, double*, int,
                                   cudaStream_t);
template int launch_lambda<float>(const KP<float>&, const std::vector<int32_t>&, const float*, float*, int,
                                  cudaStream_t);

template <typename S>
int launch_gradient(const KP<S>& p, const std::vector<int32_t>& stage_begin, const S* z, const S* eta, const S* w,
                    S* lam, double* gx0, double* gA, double* gB, double* gQ, double* gR, double* gQN, int max_blocks,
                    cudaStream_t st) {
  const int launches = launch_lambda<S>(p, stage_begin, w, lam, max_blocks, st);
  const int grid = std::max(1, std::min((p.n + kWarpsPerBlock - 1) / kWarpsPerBlock, max_blocks));
  k_gradients<S><<<grid, 128, 0, st>>>(p, z, eta, w, lam, gx0, gA, gB, gQ, gR, gQN);
  return launches + 1;
}

template int launch_gradient<double>(const KP<double>&, const std::vector<int32_t>&, const double*, const double*,
                                     const double*, double*, double*, double*, double*, double*, double*, double*,
                                     int, cudaStream_t);
template int launch_gradient<float>(const KP<float>&, const std::vector<int32_t>&, const float*, const float*,
                                    const float*, float*, double*, double*, double*, double*, double*, double*, int,
                                    cudaStream_t);

}  // namespace spock
