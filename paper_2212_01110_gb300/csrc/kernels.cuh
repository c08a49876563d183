// Device-side building blocks of the CP operator T (Eq.
// (chambolle-pock-operator)) for the tree layout of spock_internal.h.
//
// Mapping: one warp per tree node for the vector work (every block of z and
// eta belongs to exactly one node), lanes over the entries of the node's
// blocks.  Vectors are in the caller's layout (offset tables per node), the
// Riccati factors and scratch in breadth-first ("internal") order.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace spock {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;        // 128-thread blocks for the warp-per-node kernels
constexpr int kVecPad = 136;             // per-warp shared vector length (>= kMaxDim + 2)

// Residual statistics accumulated by the dual / primal-statistics kernels.
enum Stat : int {
  ST_RZ2 = 0,      // sum r_z^2
  ST_RE2 = 1,      // sum r_eta^2
  ST_RE_LRZ = 2,   // sum r_eta . (L r_z)
  ST_XIP = 3,      // max |r_z / alpha - L* r_eta|
  ST_XID = 4,      // max |r_eta / alpha - L r_z|
  ST_RD = 5,       // sum r . d              (line search, d = direction)
  ST_LRZ_DE = 6,   // sum (L r_z) . d_eta
  ST_RE_LDZ = 7,   // sum r_eta . (L d_z)
};

// Everything a warp needs to locate node k's blocks in z and eta, in one
// 128-byte record (one memory round trip instead of a chain of table loads).
struct alignas(16) NodeDesc {
  int64_t zx, zu, zz2, zs, ztau;   // x^k, u^k, z2 block, s^k, tau^k in z
  int64_t enl, enr, elf;           // nonleaf / nonroot / leaf block of k in eta
  int64_t zxp, zup;                // x and u of the parent in z
  int64_t es;                      // eta row holding s^k: enl + 2m + 1 (nonleaf) or elf + 2 nx (leaf)
  int32_t par, m, c0, user;        // parent, number of children, first child, caller's node id
  int64_t enr_c0, es_c0;           // enr and es of the first child (-1 at leaves)
};
static_assert(sizeof(NodeDesc) == 128, "NodeDesc must be 128 bytes");

// A warp reads a NodeDesc as 32 four-byte words, one per lane (one coalesced
// 128-byte load that can be issued a node ahead), and broadcasts the fields
// with shuffles.  Word positions of the fields:
enum NodeWord : int {
  NW_ZX = 0, NW_ZU = 2, NW_ZZ2 = 4, NW_ZS = 6, NW_ZTAU = 8, NW_ENL = 10, NW_ENR = 12, NW_ELF = 14,
  NW_ZXP = 16, NW_ZUP = 18, NW_ES = 20, NW_PAR = 22, NW_M = 23, NW_C0 = 24, NW_USER = 25,
  NW_ENR_C0 = 26, NW_ES_C0 = 28
};
static_assert(offsetof(NodeDesc, zz2) == 4 * NW_ZZ2 && offsetof(NodeDesc, es) == 4 * NW_ES &&
                  offsetof(NodeDesc, m) == 4 * NW_M && offsetof(NodeDesc, c0) == 4 * NW_C0 &&
                  offsetof(NodeDesc, enr_c0) == 4 * NW_ENR_C0 && offsetof(NodeDesc, es_c0) == 4 * NW_ES_C0,
              "NodeDesc word positions");

struct NodeF {
  int64_t zx, zu, zz2, zs, ztau, enl, enr, elf, zxp, zup, es, enr_c0, es_c0;
  int32_t m, c0;
};

__device__ __forceinline__ uint32_t desc_word(const NodeDesc* desc, int64_t k, int lane) {
  return __ldg(reinterpret_cast<const uint32_t*>(desc + k) + lane);
}
__device__ __forceinline__ int64_t desc_i64(uint32_t w, int i) {
  const uint32_t lo = __shfl_sync(0xffffffffu, w, i), hi = __shfl_sync(0xffffffffu, w, i + 1);
  return (int64_t)(((uint64_t)hi << 32) | (uint64_t)lo);
}
__device__ __forceinline__ NodeF node_fields(uint32_t w) {
  NodeF f;
  f.zx = desc_i64(w, NW_ZX);
  f.zu = desc_i64(w, NW_ZU);
  f.zz2 = desc_i64(w, NW_ZZ2);
  f.zs = desc_i64(w, NW_ZS);
  f.ztau = desc_i64(w, NW_ZTAU);
  f.enl = desc_i64(w, NW_ENL);
  f.enr = desc_i64(w, NW_ENR);
  f.elf = desc_i64(w, NW_ELF);
  f.zxp = desc_i64(w, NW_ZXP);
  f.zup = desc_i64(w, NW_ZUP);
  f.es = desc_i64(w, NW_ES);
  f.enr_c0 = desc_i64(w, NW_ENR_C0);
  f.es_c0 = desc_i64(w, NW_ES_C0);
  f.m = (int32_t)__shfl_sync(0xffffffffu, w, NW_M);
  f.c0 = (int32_t)__shfl_sync(0xffffffffu, w, NW_C0);
  return f;
}

template <typename S>
struct KP {
  const NodeDesc* __restrict__ desc;
  int32_t n, nl, nx, nu, N, chain_stage, n_chains;
  int64_t n_z, n_eta;
  S alpha;
  S inv_alpha;        // 1 / alpha (multiplications instead of FP64 divisions)
  // per-node strides (elements), padded to 16 bytes for bulk copies
  int32_t xs, us;                     // xbar / q, ubar / d
  int32_t gstride, nbstride, ktstride;  // Gb and Gf, NB, Kt
  int32_t* err;                       // pipeline timeout flag (device)
  const int32_t* skip;                // nonzero: the solve has finished, kernels return at once
  const int32_t* __restrict__ parent;
  const int32_t* __restrict__ ch_begin;
  const int32_t* __restrict__ ch_count;
  const int32_t* __restrict__ stage_begin;   // device copy [N + 2]
  const int64_t* __restrict__ zx;
  const int64_t* __restrict__ zu;
  const int64_t* __restrict__ zz2;
  const int64_t* __restrict__ zs;
  const int64_t* __restrict__ ztau;
  const int64_t* __restrict__ enl;
  const int64_t* __restrict__ enr;
  const int64_t* __restrict__ elf;
  const S* __restrict__ Gb;
  const S* __restrict__ Gf;
  const S* __restrict__ NB;
  const S* __restrict__ Kt;
  const S* __restrict__ qs;
  const S* __restrict__ rs;
  const S* __restrict__ qns;
  const S* __restrict__ xlo;
  const S* __restrict__ xhi;
  const S* __restrict__ ulo;
  const S* __restrict__ uhi;
  const S* __restrict__ av;
  const S* __restrict__ prob;
  const S* __restrict__ s2inv;   // per nonleaf node: 1 / (a^2 + 3), 1 / (a^2 + 3 + m)
  S* __restrict__ xbar;
  S* __restrict__ ubar;
  S* __restrict__ q;
  S* __restrict__ d;
  const S* __restrict__ x0;
  // general form (gen != 0): constraint rows and leading dimensions, and the
  // per-node matrices of L in column-major (c) and transposed (t) layouts
  int32_t gen, nc, ncN, ldc, ldxu, ldx, ldu, ldcn, cst;
  const S* __restrict__ gc;
  const S* __restrict__ gt;
  const S* __restrict__ fqc;
  const S* __restrict__ fqt;
  const S* __restrict__ frc;
  const S* __restrict__ frt;
  const S* __restrict__ fnc;
  const S* __restrict__ fnt;
  const S* __restrict__ gnc;
  const S* __restrict__ gnt;
  const S* __restrict__ clo;
  const S* __restrict__ chi;
  // risk measures of the general form (per nonleaf node): rows of y, orthant
  // rows of K, offsets of b and of the S2 projector, their values
  int32_t max_nz2;
  const int32_t* __restrict__ rny;
  const int32_t* __restrict__ rkp;
  const int64_t* __restrict__ rboff;
  const int64_t* __restrict__ rpoff;
  const S* __restrict__ rb;
  const S* __restrict__ rpi;
};

// Records `ev` on `st`; while `st` is being captured into a graph the record
// becomes an event-record node (timing of every replay), otherwise a plain
// record.
inline void record_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  else cudaEventRecord(ev, st);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
// Sum over lanes [0, n) of v (zero on the other lanes), returned to every
// lane: ceil(log2 n) adds instead of five (n = 1 is a broadcast of lane 0).
template <typename S>
__device__ __forceinline__ S lanes_sum(S v, int n) {
  for (int o = 1; o < n && o < 32; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
  return __shfl_sync(kFull, v, 0);
}
// Sum of the values held by lanes a and b (different lanes), to every lane.
template <typename S>
__device__ __forceinline__ S two_lanes_sum(S v, int a, int b) {
  return __shfl_sync(kFull, v, a) + __shfl_sync(kFull, v, b);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Working-precision math with the precision fixed by the argument type (no
// promotion of FP32 arguments to the FP64 pipe).
__device__ __forceinline__ float vabs(float v) { return fabsf(v); }
__device__ __forceinline__ double vabs(double v) { return fabs(v); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float vsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double vsqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float vrsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double vrsqrt(double v) { return rsqrt(v); }

template <typename S>
__device__ __forceinline__ S clampv(S v, S lo, S hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Statistics accumulator: sums in FP64.  Terms are first summed in the
// working precision S.  FP64: every lane adds its node sums to its own FP64
// accumulator, and the block store reduces across lanes.  FP32: every
// kFlushNodesF32 nodes (and at the end) the warp reduces its lanes' FP32
// sums with shuffles and lane 0 alone adds them in FP64.  Every FP64
// operation costs a 64-cycle slot of its sub-partition's FP64 pipe per warp
// instruction on GB300, whatever the number of active lanes, so the FP32
// kernels keep FP64 work to ~16 warp instructions per 32 nodes.
struct StatAcc {
  double s[8];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = 0.0;
  }
};
constexpr int kFlushNodesF32 = 32;
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
template <typename S>
struct NodeAcc {
  S s[8];
  int nodes;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = S(0);
    nodes = 0;
  }
  // all lanes of the warp call it
  __device__ __forceinline__ void flush(StatAcc& a) {
    if (sizeof(S) == 4) {
      const bool lead = (threadIdx.x & 31) == 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const bool mx = (i == 3 || i == 4);
        const float v = mx ? warp_max_f((float)s[i]) : warp_sum((float)s[i]);
        if (lead) a.s[i] = mx ? fmax(a.s[i], (double)v) : a.s[i] + (double)v;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (i == 3 || i == 4) a.s[i] = fmax(a.s[i], (double)s[i]);
        else a.s[i] += (double)s[i];
      }
    }
    zero();
  }
  // end of a node: flush when due
  __device__ __forceinline__ void node_done(StatAcc& a) {
    // FP64 terms are summed in FP64 already: one flush at the end of the
    // kernel; FP32 terms are flushed into FP64 every kFlushNodesF32 nodes
    if (sizeof(S) == 4 && ++nodes == kFlushNodesF32) flush(a);
  }
};

// Reduces the statistics of a block (after the final flush) and writes row
// `row` of the partials.  Sums for sums, maxima for ST_XIP / ST_XID.  With
// LEAD (FP32 kernels) lane 0 of every warp already holds its warp's totals.
template <bool LEAD>
__device__ __forceinline__ void block_stats_store(StatAcc& a, double* partials, int row) {
  __shared__ double red[kWarpsPerBlock][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    double v = a.s[i];
    if (!LEAD) v = (i == ST_XIP || i == ST_XID) ? warp_max(v) : warp_sum(v);
    if (lane == 0) red[w][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int i = threadIdx.x;
    double v = red[0][i];
    for (int k = 1; k < kWarpsPerBlock; ++k)
      v = (i == ST_XIP || i == ST_XID) ? fmax(v, red[k][i]) : v + red[k][i];
    partials[(int64_t)row * 8 + i] = v;
  }
}

}  // namespace spock
