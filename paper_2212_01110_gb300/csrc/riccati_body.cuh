// Device bodies of the direct Riccati kernels (riccati.cu), shared with the
// single-block solve kernel (cta.cu): every body works for block `bid` of
// `nblk` blocks of one problem.
#pragma once

#include <cstdint>

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
  const S* __restrict__ Cm = Km + (int64_t)nu * nx;   // K + W^T
  const S* __restrict__ Ri = Km + 2 * (int64_t)nu * nx;
  for (int a = lane; a < nu; a += 32) {
    S acc = 0;
    // Rtilde^-1 is stored exactly symmetric: lane a reads column a (row a),
    // consecutive lanes consecutive addresses
    for (int b = 0; b < nu; ++b) acc += __ldg(Ri + b * nu + a) * v.g[b];
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
  // q += K^T (d - ubar) + W d = C^T d - K^T ubar
#pragma unroll 4
  for (int b = 0; b < nu; ++b) {
    const S db = v.d[b];
    const S ub = v.u[b];
    const S* kr = Km + (int64_t)b * nx;
    const S* cr = Cm + (int64_t)b * nx;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int r = 32 * s + lane;
      if (r < nx) qn[s] = fma(-__ldg(kr + r), ub, fma(__ldg(cr + r), db, qn[s]));   // two FMAs, no add
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

// Per-warp vectors of at most nx + nu <= 32 SL entries (the lane slots of
// the body's instance).
#define SPOCK_WARP_VECS(S)                                           \
  constexpr int kVP_ = 32 * SL + 8;                                  \
  __shared__ S sm_q[kWarpsPerBlock][kVP_];                           \
  __shared__ S sm_h[kWarpsPerBlock][kVP_];                           \
  __shared__ S sm_u[kWarpsPerBlock][kVP_];                           \
  __shared__ S sm_g[kWarpsPerBlock][kVP_];                           \
  __shared__ S sm_d[kWarpsPerBlock][kVP_];                           \
  __shared__ S sm_w[kWarpsPerBlock][kVP_];                           \
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

}  // namespace spock
