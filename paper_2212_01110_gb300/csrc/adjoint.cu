// Adjoint of the CP fixed point (implicit differentiation of v* = T(v*)):
// the kernels of the adjoint solve (I - J^T) w = (g, 0) by restarted GMRES
// and of the gradient of phi(z*) = <g, z*> in the problem data (FP64).
//
// J is the Jacobian of T (Eq. (chambolle-pock-operator)) at the converged
// pair.  With A the Jacobian of prox_{alpha f} (identity on s^0, the
// projection on the null space of the dynamics on z_1, proj_S2 on z_2; it
// does not depend on the point) and B = I - D(wbar / alpha) that of
// prox_{alpha g*} (D the Jacobian of proj_S3 at wbar / alpha,
// wbar = eta* + alpha L z*), both symmetric,
//   J^T (wz, weta) = (p - alpha L* q,  q - alpha L p),
//   q = B weta,  p = A (wz + 2 alpha L* q).
// A is applied by the prox-of-f kernels with alpha = 0 and x0 = 0 (the
// homogeneous Riccati pass), L and L* by the operator kernels; this file
// holds B, the vector steps and the gradient assembly.
#include <algorithm>

#include "kernels.cuh"
#include "spock_internal.h"

namespace spock {

// out = x - D x on one translated SOC block (SOC + sh, sh = (0, .., 1/2, -1/2),
// SOC = {(v, t): ||v|| <= t}) of `dim` entries, D the Jacobian of the
// projection at y = wbar / alpha - sh:
//   ||v|| <= t: D = I;   ||v|| <= -t: D = 0;   otherwise, with vh = v / ||v||
//   and s = t / ||v||:  (D x)_v = ((1 + s) x_v - s vh (vh'x_v) + vh x_t) / 2,
//                       (D x)_t = (vh'x_v + x_t) / 2.
template <int J>
__device__ __forceinline__ void soc_jac_block(const double* __restrict__ wb, const double* __restrict__ x,
                                              double* __restrict__ out, int dim, double ial, int lane) {
  double yv[J], xv[J];
  double s2 = 0.0, tl = 0.0, xtl = 0.0;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int e = lane + 32 * j;
    yv[j] = xv[j] = 0.0;
    if (e < dim) {
      double y = wb[e] * ial;
      if (e == dim - 2) y -= 0.5;
      if (e == dim - 1) y += 0.5;
      yv[j] = y;
      xv[j] = x[e];
      if (e < dim - 1) s2 += y * y;
      else {
        tl = y;
        xtl = xv[j];
      }
    }
  }
  s2 = warp_sum(s2);
  const double t = __shfl_sync(kFull, tl, (dim - 1) & 31);
  const double xt = __shfl_sync(kFull, xtl, (dim - 1) & 31);
  const double nv = sqrt(s2);
  if (nv <= t) {
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (lane + 32 * j < dim) out[lane + 32 * j] = 0.0;
    return;
  }
  if (nv <= -t) {
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (lane + 32 * j < dim) out[lane + 32 * j] = xv[j];
    return;
  }
  const double inv = 1.0 / nv, s = t * inv;
  double a = 0.0;
#pragma unroll
  for (int j = 0; j < J; ++j)
    if (lane + 32 * j < dim - 1) a += yv[j] * inv * xv[j];
  a = warp_sum(a);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int e = lane + 32 * j;
    if (e < dim - 1) {
      const double vh = yv[j] * inv;
      out[e] = xv[j] - 0.5 * ((1.0 + s) * xv[j] - s * vh * a + vh * xt);
    } else if (e == dim - 1) {
      out[e] = xv[j] - 0.5 * (a + xt);
    }
  }
}

// out = B x = x - D(wbar / alpha) x, warp per node, block by block of Eq.
// (S3-def): the y block of (K^i)* = R^{2m}_+ x R (D = 0/1 on the orthant
// entries, 1 on the free one), the R_+ row s - b'y, the boxes, the cones.
template <int J>
__global__ void __launch_bounds__(128) k_cone_jac(KP<double> p, const double* __restrict__ wbar,
                                                  const double* __restrict__ x, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const double ial = p.inv_alpha;
  const int nx = p.nx, nu = p.nu;
  for (int k = gw; k < p.n; k += nw) {
    const int64_t enl = p.desc[k].enl, enr = p.desc[k].enr, elf = p.desc[k].elf;
    const int m = p.desc[k].m;
    if (k < p.nl) {
      for (int e = lane; e < 2 * m + 2; e += 32) {
        const int64_t i = enl + e;
        const bool d_one = (e == 2 * m) || (wbar[i] * ial > 0.0);
        out[i] = d_one ? 0.0 : x[i];
      }
      const int64_t ea = enl + 2 * m + 2;
      for (int e = lane; e < nx + nu; e += 32) {
        const double y = wbar[ea + e] * ial;
        const double lo = e < nx ? p.xlo[(int64_t)k * nx + e] : p.ulo[(int64_t)k * nu + (e - nx)];
        const double hi = e < nx ? p.xhi[(int64_t)k * nx + e] : p.uhi[(int64_t)k * nu + (e - nx)];
        out[ea + e] = (y > lo && y < hi) ? 0.0 : x[ea + e];
      }
    } else {
      for (int e = lane; e < nx; e += 32) {
        const double y = wbar[elf + e] * ial;
        out[elf + e] = (y > p.xlo[(int64_t)k * nx + e] && y < p.xhi[(int64_t)k * nx + e]) ? 0.0 : x[elf + e];
      }
      soc_jac_block<J>(wbar + elf + nx, x + elf + nx, out + elf + nx, nx + 2, ial, lane);
    }
    if (k > 0) soc_jac_block<J>(wbar + enr, x + enr, out + enr, nx + nu + 2, ial, lane);
  }
}

// out = y + a x
__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, const double* __restrict__ y,
                       double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = y[i] + a * x[i];
}

// ---------------------------------------------------------------------------
// restarted GMRES on (I - J^T) w = (g, 0): the Krylov basis is a set of
// vectors of length nz + ne with stride ld (FP64), built by classical
// Gram-Schmidt with one reorthogonalisation; dot products are reduced in a
// fixed order (block partials, then one block), so runs are deterministic.
// ---------------------------------------------------------------------------
constexpr int kGmresMaxBasis = 32;    // basis vectors per dot-product launch
constexpr int kGmresMaxRestart = 128; // basis vectors of one axpy launch

// u = x - J^T x from the parts of J^T x: (pz - alpha t, q - alpha Lp)
__global__ void k_jt_residual(int64_t nz, int64_t ne, double alpha, const double* __restrict__ pz,
                              const double* __restrict__ t, const double* __restrict__ q,
                              const double* __restrict__ Lp, const double* __restrict__ x, double* __restrict__ u) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nz + ne;
       i += (int64_t)gridDim.x * blockDim.x)
    u[i] = x[i] - (i < nz ? pz[i] - alpha * t[i] : q[i - nz] - alpha * Lp[i - nz]);
}

// partials[block][j] = sum over the block's entries of u . V_j, j < k
// (k <= kGmresMaxRestart), in chunks of 32 basis vectors held in registers.
// With kdev, k is *kdev + k (the basis size of a captured Arnoldi step).
__global__ void __launch_bounds__(256) k_dots(int64_t n, const double* __restrict__ u, const double* __restrict__ V,
                                              int64_t ld, int k, const int* __restrict__ kdev,
                                              double* __restrict__ partials) {
  if (kdev) k += *kdev;
  __shared__ double red[8][kGmresMaxBasis];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c0 = 0; c0 < k; c0 += kGmresMaxBasis) {
    const int kc = min(kGmresMaxBasis, k - c0);
    const double* Vc = V + (int64_t)c0 * ld;
    double acc[kGmresMaxBasis];
#pragma unroll
    for (int j = 0; j < kGmresMaxBasis; ++j) acc[j] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const double ui = u[i];
#pragma unroll
      for (int j = 0; j < kGmresMaxBasis; ++j)
        if (j < kc) acc[j] = fma(ui, Vc[(int64_t)j * ld + i], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < kGmresMaxBasis; ++j) {
      if (j < kc) {
        const double v = warp_sum(acc[j]);
        if (lane == 0) red[w][j] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x < kc) {
      double sum = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) sum += red[ww][threadIdx.x];
      partials[(int64_t)blockIdx.x * kGmresMaxRestart + c0 + threadIdx.x] = sum;
    }
    __syncthreads();
  }
}

// out[j] = sum_b partials[b][j], j < k (one block, fixed order)
__global__ void k_dots_reduce(int nblocks, int k, const int* __restrict__ kdev, const double* __restrict__ partials,
                              double* __restrict__ out) {
  if (kdev) k += *kdev;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * kGmresMaxRestart + j];
    out[j] = s;
  }
}

// u += sign * sum_{j < k} h_j V_j  (h on the device, k <= kGmresMaxRestart;
// with kdev, k is *kdev + k)
__global__ void k_axpy_many(int64_t n, double* __restrict__ u, const double* __restrict__ V, int64_t ld, int k,
                            const int* __restrict__ kdev, const double* __restrict__ h, double sign) {
  if (kdev) k += *kdev;
  __shared__ double hs[kGmresMaxRestart];
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = sign * h[j];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = u[i];
    for (int j = 0; j < k; ++j) v = fma(hs[j], V[(int64_t)j * ld + i], v);
    u[i] = v;
  }
}

// v = a u
__global__ void k_scale(int64_t n, double a, const double* __restrict__ u, double* __restrict__ v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = a * u[i];
}

// The next basis vector of a captured Arnoldi step: V_{k+1} = vin = u / ||u||
// with k = *kdev and ||u||^2 = *norm2 (0 when the norm vanishes)
__global__ void k_next_basis(int64_t n, const double* __restrict__ u, const double* __restrict__ norm2,
                             const int* __restrict__ kdev, double* __restrict__ V, int64_t ld,
                             double* __restrict__ vin) {
  const double nn = *norm2;
  const double a = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  double* vk1 = V + (int64_t)(*kdev + 1) * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = a * u[i];
    vk1[i] = v;
    vin[i] = v;
  }
}

__global__ void k_inc(int* kdev) { *kdev += 1; }

// red[0] = max |b - u|, red[1] = max |x| (bit patterns of non-negative
// doubles), r = b - u written out; b = (g, 0)
__global__ void k_true_residual(int64_t nz, int64_t ntot, const double* __restrict__ g, const double* __restrict__ u,
                                const double* __restrict__ x, double* __restrict__ r, unsigned long long* red) {
  double rmax = 0.0, xmax = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ntot; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = (i < nz ? g[i] : 0.0) - u[i];
    r[i] = ri;
    rmax = fmax(rmax, fabs(ri));
    xmax = fmax(xmax, fabs(x[i]));
  }
  rmax = warp_max(rmax);
  xmax = warp_max(xmax);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(red, (unsigned long long)__double_as_longlong(rmax));
    atomicMax(red + 1, (unsigned long long)__double_as_longlong(xmax));
  }
}

// Gradients of phi from the adjoint quantities (outputs in the caller's node
// numbering; entries of nodes where a quantity does not exist are left 0):
//   mu:  G^T mu = r_1 - p_1 (lam_mu for nonleaf nodes; leaves mu = -negy_x)
//   nu = alpha lambda, G^T lambda = -(L* eta*)_1 (lam_env; leaves -wenv_x)
//   g_x0 = mu^0,  g_A^c = nu^c p_x^anc' + mu^c x*^anc',  g_B^c likewise with u,
//   g_Q^c_k = alpha (q_{c,Qx,k} x*^anc_k - eta*_{c,Qx,k} p_{x^anc,k}) / (2 sqrt Q^c_k),
//   g_R, g_QN likewise (rows R^1/2 u^anc, Q_N^1/2 x^j).
__global__ void __launch_bounds__(128) k_adj_gradients(KP<double> p, const double* __restrict__ z,
                                                       const double* __restrict__ eta, const double* __restrict__ q,
                                                       const double* __restrict__ pv,
                                                       const double* __restrict__ lam_mu,
                                                       const double* __restrict__ negy,
                                                       const double* __restrict__ lam_env,
                                                       const double* __restrict__ wenv, double* gx0, double* gA,
                                                       double* gB, double* gQ, double* gR, double* gQN) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nx = p.nx, nu = p.nu;
  const double al = p.alpha;
  for (int k = gw; k < p.n; k += nw) {
    const NodeDesc D = p.desc[k];
    const int64_t u = D.user;
    auto mu = [&](int r) { return k < p.nl ? lam_mu[(int64_t)k * p.xs + r] : -negy[D.zx + r]; };
    auto nu_ = [&](int r) { return al * (k < p.nl ? lam_env[(int64_t)k * p.xs + r] : -wenv[D.zx + r]); };
    if (k == 0 && gx0)
      for (int r = lane; r < nx; r += 32) gx0[r] = mu(r);
    if (k > 0) {
      if (gA)
        for (int e = lane; e < nx * nx; e += 32) {
          const int r = e / nx, c = e % nx;
          gA[u * nx * nx + e] = nu_(r) * pv[D.zxp + c] + mu(r) * z[D.zxp + c];
        }
      if (gB)
        for (int e = lane; e < nx * nu; e += 32) {
          const int r = e / nu, c = e % nu;
          gB[u * nx * nu + e] = nu_(r) * pv[D.zup + c] + mu(r) * z[D.zup + c];
        }
      if (gQ)
        for (int r = lane; r < nx; r += 32)
          gQ[u * nx + r] = al * (q[D.enr + r] * z[D.zxp + r] - eta[D.enr + r] * pv[D.zxp + r]) /
                           (2.0 * p.qs[(int64_t)k * nx + r]);
      if (gR)
        for (int r = lane; r < nu; r += 32)
          gR[u * nu + r] = al * (q[D.enr + nx + r] * z[D.zup + r] - eta[D.enr + nx + r] * pv[D.zup + r]) /
                           (2.0 * p.rs[(int64_t)k * nu + r]);
    }
    if (k >= p.nl && gQN)
      for (int r = lane; r < nx; r += 32)
        gQN[u * nx + r] = al * (q[D.elf + nx + r] * z[D.zx + r] - eta[D.elf + nx + r] * pv[D.zx + r]) /
                          (2.0 * p.qns[(int64_t)k * nx + r]);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_cone_jac(const KP<double>& p, const double* wbar, const double* x, double* out, int grid,
                     cudaStream_t st) {
  const int J = (p.nx + p.nu + 2 + 31) / 32;
  switch (J) {
    case 1: k_cone_jac<1><<<grid, 128, 0, st>>>(p, wbar, x, out); break;
    case 2: k_cone_jac<2><<<grid, 128, 0, st>>>(p, wbar, x, out); break;
    case 3: k_cone_jac<3><<<grid, 128, 0, st>>>(p, wbar, x, out); break;
    case 4: k_cone_jac<4><<<grid, 128, 0, st>>>(p, wbar, x, out); break;
    default: k_cone_jac<5><<<grid, 128, 0, st>>>(p, wbar, x, out); break;
  }
}

void launch_axpy(int64_t n, double a, const double* x, const double* y, double* out, int grid, cudaStream_t st) {
  k_axpy<<<grid, 256, 0, st>>>(n, a, x, y, out);
}

void launch_jt_residual(int64_t nz, int64_t ne, double alpha, const double* pz, const double* t, const double* q,
                        const double* Lp, const double* x, double* u, int grid, cudaStream_t st) {
  k_jt_residual<<<grid, 256, 0, st>>>(nz, ne, alpha, pz, t, q, Lp, x, u);
}

// out[j] = u . V_j for j < k (k <= 128; plus *kdev when kdev is given) in
// two launches; partials holds grid x 128 doubles
void launch_dots(int64_t n, const double* u, const double* V, int64_t ld, int k, const int* kdev, double* partials,
                 double* out, int grid, cudaStream_t st) {
  k_dots<<<grid, 256, 0, st>>>(n, u, V, ld, k, kdev, partials);
  k_dots_reduce<<<1, kGmresMaxRestart, 0, st>>>(grid, k, kdev, partials, out);
}

void launch_axpy_many(int64_t n, double* u, const double* V, int64_t ld, int k, const int* kdev, const double* h,
                      double sign, int grid, cudaStream_t st) {
  k_axpy_many<<<grid, 256, 0, st>>>(n, u, V, ld, k, kdev, h, sign);
}

void launch_next_basis(int64_t n, const double* u, const double* norm2, int* kdev, double* V, int64_t ld,
                       double* vin, int grid, cudaStream_t st) {
  k_next_basis<<<grid, 256, 0, st>>>(n, u, norm2, kdev, V, ld, vin);
  k_inc<<<1, 1, 0, st>>>(kdev);
}

void launch_scale(int64_t n, double a, const double* u, double* v, int grid, cudaStream_t st) {
  k_scale<<<grid, 256, 0, st>>>(n, a, u, v);
}

void launch_true_residual(int64_t nz, int64_t ntot, const double* g, const double* u, const double* x, double* r,
                          unsigned long long* red, int grid, cudaStream_t st) {
  k_true_residual<<<grid, 256, 0, st>>>(nz, ntot, g, u, x, r, red);
}

void launch_adj_gradients(const KP<double>& p, const double* z, const double* eta, const double* q,
                          const double* pv, const double* lam_mu, const double* negy, const double* lam_env,
                          const double* wenv, double* gx0, double* gA, double* gB, double* gQ, double* gR,
                          double* gQN, int grid, cudaStream_t st) {
  k_adj_gradients<<<grid, 128, 0, st>>>(p, z, eta, q, pv, lam_mu, negy, lam_env, wenv, gx0, gA, gB, gQ, gR, gQN);
}

}  // namespace spock
