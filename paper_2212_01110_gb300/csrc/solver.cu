// Host side of libspock: problem setup (layout, Algorithm 1, uploads), the
// evaluation of T as a sequence of kernel launches, the driver loop of
// Algorithm 3 whose decisions are taken on the device (supermann.cu), the
// vanilla CP loop and the C ABI of include/spock.h.
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <exception>
#include <mutex>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "batch.cuh"
#include "kernels.cuh"
#include "general.h"
#include "spock_internal.h"
#include "supermann.cuh"

namespace spock {

// launchers defined in ops.cu / riccati.cu
template <typename S>
void launch_prep(const KP<S>& p, const S* z, const S* eta, S* zo, int max_blocks, cudaStream_t st);
template <typename S>
void launch_dual(const KP<S>& p, int mode, bool stats, const S* z, const S* zp, const S* eta, S* out,
                 const S* dir, double* partials, int grid, cudaStream_t st);
template <typename S>
void launch_lstar(const KP<S>& p, const S* eta, S* zout, int grid, cudaStream_t st);
void launch_reduce_stats(const double* pd, int nd, const double* pp, int np, double* out, cudaStream_t st,
                         const int32_t* skip = nullptr);
template <typename S>
int launch_riccati(const KP<S>& p, const std::vector<int32_t>& stage_begin, const std::vector<int32_t>& stage_maxch,
                   S* zo, cudaStream_t st, cudaEvent_t* ev);

enum { DM_APPLY_L_ = 0, DM_PROXG_ = 1, DM_DUAL_ = 2 };

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

struct SpockError : std::runtime_error {
  int code;
  SpockError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CUDA_TRY(x)                                                                               \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess)                                                                        \
      throw SpockError(e_ == cudaErrorMemoryAllocation ? SPOCK_ERR_OOM : SPOCK_ERR_CUDA,          \
                       std::string(#x) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const SpockError& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(SPOCK_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(SPOCK_ERR_CUDA, e.what());
  }
}

// A kernel whose bounded wait on a bulk copy gave up sets *P.err; report it
// (and clear the flag) after the work on `st` has completed.
static void check_device_flag(Problem& P, cudaStream_t st) {
  int32_t h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, P.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (h) {
    CUDA_TRY(cudaMemsetAsync(P.err, 0, sizeof(int32_t), st));
    CUDA_TRY(cudaStreamSynchronize(st));
    throw SpockError(SPOCK_ERR_CUDA, "a kernel's bounded wait for a bulk copy timed out");
  }
}

static void check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw SpockError(SPOCK_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// in-solve timing of the kernel groups of T (CUDA events on the solve stream)
// ---------------------------------------------------------------------------
struct Profiler {
  static constexpr int kGroups = 7, kSlots = 64;
  bool on = false;
  std::vector<cudaEvent_t> ev;
  int used = 0, n = 0;
  double acc[kGroups] = {0, 0, 0, 0, 0, 0, 0};
  ~Profiler() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  void start() {
    if (ev.empty()) {
      ev.resize((size_t)kSlots * (kGroups + 1));
      for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
    }
    used = n = 0;
    for (double& a : acc) a = 0.0;
    on = true;
  }
  cudaEvent_t* slot() {
    if (used == kSlots) harvest();
    return &ev[(size_t)(used++) * (kGroups + 1)];
  }
  // Graph replays: slots 0..k-1 were recorded by the rounds that ran.
  void harvest_first(int k) {
    used = std::min(k, used);
    harvest();
  }
  void harvest() {
    for (int s = 0; s < used; ++s) {
      cudaEvent_t* e = &ev[(size_t)s * (kGroups + 1)];
      CUDA_TRY(cudaEventSynchronize(e[kGroups]));
      for (int g = 0; g < kGroups; ++g) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, e[g], e[g + 1]));
        acc[g] += ms;
      }
    }
    n += used;
    used = 0;
  }
};

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct Workspace {
  int prec = 0;
  int64_t n_v = 0;
  int64_t ld = 0;  // column stride of the Anderson buffers
  int mem = -1;
  void* v[3] = {nullptr, nullptr, nullptr};
  void* Tv[3] = {nullptr, nullptr, nullptr};
  double* stats = nullptr;  // [3][8]
  void* d = nullptr;
  void* MR = nullptr;
  void* D = nullptr;
  void* zero_eta = nullptr;
  double* pd = nullptr;
  double* paa = nullptr;
  int grid_d = 0, grid_v = 0;
  SmState* st = nullptr;
  int32_t* trace = nullptr;
  int trace_cap = 0;
  int32_t* h_action = nullptr;  // pinned
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Profiler prof;
  int64_t launches = 0;
  // device-driven rounds: internal stream, cached graph of kRounds rounds
  cudaStream_t stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double g_alpha = 0.0;
  int g_trace = -1, g_launches_per_round = 0;
  int32_t* h_done = nullptr;  // pinned
  void* cta_bi = nullptr;      // instance view of the single-block solve (device)
  std::vector<void*> allocs;
  ~Workspace() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (stream) cudaStreamDestroy(stream);
    if (h_done) cudaFreeHost(h_done);
    for (void* p : allocs) cudaFree(p);
    if (h_action) cudaFreeHost(h_action);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  void* alloc(size_t bytes) {
    void* p = nullptr;
    CUDA_TRY(cudaMalloc(&p, bytes > 0 ? bytes : 16));
    allocs.push_back(p);
    return p;
  }
};

Problem::~Problem() {
  delete ws64;
  delete ws32;
  for (void* p : allocations) cudaFree(p);
  if (adj_pinned) cudaFreeHost(adj_pinned);
}

static int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 132;
}

template <typename S>
static Workspace*& ws_slot(Problem& P) {
  return sizeof(S) == 8 ? P.ws64 : P.ws32;
}

template <typename S>
static Workspace* get_ws_impl(Problem& P, int mem) {
  Workspace*& w = ws_slot<S>(P);
  if (w && w->mem >= mem) return w;
  delete w;
  w = nullptr;
  auto* ws = new Workspace();
  try {
    ws->prec = sizeof(S) == 8 ? SPOCK_FP64 : SPOCK_FP32;
    ws->n_v = P.off.n_z + P.off.n_eta;
    ws->mem = mem;
    const size_t vb = sizeof(S) * (size_t)ws->n_v;
    for (int i = 0; i < 3; ++i) {
      ws->v[i] = ws->alloc(vb);
      ws->Tv[i] = ws->alloc(vb);
    }
    ws->stats = (double*)ws->alloc(3 * 8 * sizeof(double));
    ws->d = ws->alloc(vb);
    ws->ld = (ws->n_v + 63) / 64 * 64;  // column stride: 256-byte aligned columns
    const size_t cb = sizeof(S) * (size_t)ws->ld;
    ws->MR = ws->alloc(cb * (size_t)(mem > 0 ? mem : 1));
    ws->D = ws->alloc(cb * (size_t)(mem > 0 ? mem : 1));
    ws->zero_eta = ws->alloc(sizeof(double) * (size_t)P.off.n_eta);
    CUDA_TRY(cudaMemset(ws->zero_eta, 0, sizeof(double) * (size_t)P.off.n_eta));
    const int sms = sm_count();
    // one wave of the fused dual kernel (fewer end-of-block statistics
    // reductions): the box form's FP64 kernel holds 238 registers (two
    // resident 128-thread blocks per SM), the others at most 128 (four)
    const int per_sm = (sizeof(S) == 8 && !P.general) ? 2 : 4;
    ws->grid_d = std::min((P.tree.n + kWarpsPerBlock - 1) / kWarpsPerBlock, sms * per_sm);
    ws->grid_d = std::max(ws->grid_d, 1);
    ws->grid_v = sms * 4;
    ws->pd = (double*)ws->alloc(sizeof(double) * 8 * ws->grid_d);
    ws->paa = (double*)ws->alloc(sizeof(double) * 2 * kMaxMemory * ws->grid_v);
    ws->st = (SmState*)ws->alloc(sizeof(SmState));
    CUDA_TRY(cudaMallocHost(&ws->h_action, sizeof(int32_t) * 4));
    CUDA_TRY(cudaMallocHost(&ws->h_done, sizeof(int32_t) * 4));
    CUDA_TRY(cudaStreamCreateWithFlags(&ws->stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreate(&ws->e0));
    CUDA_TRY(cudaEventCreate(&ws->e1));
  } catch (...) {
    delete ws;
    throw;
  }
  w = ws;
  return ws;
}

// ---------------------------------------------------------------------------
// kernel parameters
// ---------------------------------------------------------------------------
template <typename S>
static const DevFactors<S>& factors(const Problem& P);
template <>
const DevFactors<double>& factors<double>(const Problem& P) { return P.f64; }
template <>
const DevFactors<float>& factors<float>(const Problem& P) { return P.f32; }

template <typename S>
static KP<S> make_kp(const Problem& P, double alpha, const int32_t* stage_begin_dev) {
  const DevFactors<S>& f = factors<S>(P);
  KP<S> k;
  k.desc = P.idx.desc;
  k.n = P.tree.n;
  k.nl = P.tree.n_nonleaf;
  k.nx = P.nx;
  k.nu = P.nu;
  k.N = P.tree.N;
  k.chain_stage = P.tree.chain_stage;
  k.n_chains = P.tree.chain_stage < P.tree.N
                   ? P.tree.stage_begin[P.tree.chain_stage + 1] - P.tree.stage_begin[P.tree.chain_stage]
                   : 0;
  k.n_z = P.off.n_z;
  k.n_eta = P.off.n_eta;
  k.alpha = (S)alpha;
  k.inv_alpha = (S)(1.0 / alpha);
  k.parent = P.idx.parent;
  k.ch_begin = P.idx.ch_begin;
  k.ch_count = P.idx.ch_count;
  k.stage_begin = stage_begin_dev;
  k.zx = P.idx.zx;
  k.zu = P.idx.zu;
  k.zz2 = P.idx.zz2;
  k.zs = P.idx.zs;
  k.ztau = P.idx.ztau;
  k.enl = P.idx.enl;
  k.enr = P.idx.enr;
  k.elf = P.idx.elf;
  k.Gb = f.Gb;
  k.Gf = f.Gf;
  k.NB = f.NB;
  k.Kt = f.Kt;
  k.qs = f.qs;
  k.rs = f.rs;
  k.qns = f.qns;
  k.xlo = f.xlo;
  k.xhi = f.xhi;
  k.ulo = f.ulo;
  k.uhi = f.uhi;
  k.av = f.av;
  k.prob = f.prob;
  k.s2inv = f.s2inv;
  k.xbar = f.xbar;
  k.ubar = f.ubar;
  k.q = f.q;
  k.d = f.d;
  k.x0 = f.x0;
  k.xs = f.xs;
  k.us = f.us;
  k.gstride = f.gstride;
  k.nbstride = f.nbstride;
  k.ktstride = f.ktstride;
  k.err = P.err;
  k.skip = nullptr;
  const GenDims& g = P.gd;
  k.gen = P.general ? 1 : 0;
  k.nc = g.nc;
  k.ncN = g.ncN;
  k.ldc = g.ldc;
  k.ldxu = g.ldxu;
  k.ldx = g.ldx;
  k.ldu = g.ldu;
  k.ldcn = g.ldcn;
  k.cst = g.cst;
  k.gc = f.gc;
  k.gt = f.gt;
  k.fqc = f.fqc;
  k.fqt = f.fqt;
  k.frc = f.frc;
  k.frt = f.frt;
  k.fnc = f.fnc;
  k.fnt = f.fnt;
  k.gnc = f.gnc;
  k.gnt = f.gnt;
  k.clo = f.clo;
  k.chi = f.chi;
  k.max_nz2 = g.max_nz2;
  k.rny = P.idx.rny;
  k.rkp = P.idx.rkp;
  k.rboff = P.idx.rboff;
  k.rpoff = P.idx.rpoff;
  k.rb = f.rb;
  k.rpi = f.rpi;
  return k;
}

// One instance's view for the batched and single-block kernels.
template <typename S>
static BInst<S> make_binst(Problem& P, Workspace* ws, double alpha) {
  BInst<S> b;
  b.kp = make_kp<S>(P, alpha, P.idx.stage_begin);
  b.kp.skip = &ws->st->done;
  b.st = ws->st;
  b.V = (S*)ws->v[0];
  b.TV = (S*)ws->Tv[0];
  b.Vt = (S*)ws->v[2];
  b.TVt = (S*)ws->Tv[2];
  b.d = (S*)ws->d;
  b.MR = (S*)ws->MR;
  b.D = (S*)ws->D;
  b.stats = ws->stats;
  b.pd = ws->pd;
  b.paa = ws->paa;
  b.n_v = ws->n_v;
  b.ld = ws->ld;
  b.nb_node = 1;
  b.nb_vec = 1;
  return b;
}


static double default_alpha(const Problem& P, double alpha) { return alpha > 0.0 ? alpha : 0.99 / P.normL; }

// ---------------------------------------------------------------------------
// conversion kernels (user FP64 buffers <-> working precision)
// ---------------------------------------------------------------------------
template <typename D, typename S>
__global__ void k_convert(const S* __restrict__ in, D* __restrict__ out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (D)in[i];
}
template <typename D, typename S>
static void convert(const S* in, D* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
  k_convert<D, S><<<grid, 256, 0, st>>>(in, out, n);
}

// ---------------------------------------------------------------------------
// T and its residual statistics
// ---------------------------------------------------------------------------
struct Ctx {
  Problem* P;
  Workspace* ws;
  double alpha;
  cudaStream_t st;
  int32_t* stage_dev;
};

template <typename S>
static void eval_T(const Ctx& c, const S* v, S* Tv, const S* dir, double* stats, const int32_t* skip = nullptr) {
  Problem& P = *c.P;
  Workspace* ws = c.ws;
  KP<S> kp = make_kp<S>(P, c.alpha, c.stage_dev);
  kp.skip = skip;
  const int64_t nz = P.off.n_z;
  const int maxb = sm_count() * 16;
  cudaEvent_t* ev = (ws && ws->prof.on) ? ws->prof.slot() : nullptr;
  if (ev) record_event(ev[0], c.st);
  launch_prep<S>(kp, v, v + nz, Tv, maxb, c.st);
  if (ev) record_event(ev[1], c.st);
  int launches = 2 + launch_riccati<S>(kp, P.tree.stage_begin, P.tree.stage_maxch, Tv, c.st, ev ? ev + 2 : nullptr);
  if (ev) record_event(ev[5], c.st);
  launch_dual<S>(kp, DM_DUAL_, stats != nullptr, v, Tv, v + nz, Tv + nz, dir, ws ? ws->pd : nullptr,
                 ws ? ws->grid_d : std::min((P.tree.n + 3) / 4, maxb), c.st);
  if (ev) record_event(ev[6], c.st);
  if (stats) {  // the dual kernel left the dual and primal statistics in pd
    launch_reduce_stats(ws->pd, ws->grid_d, nullptr, 0, stats, c.st, skip);
    launches += 1;
  }
  if (ev) record_event(ev[7], c.st);
  if (ws) ws->launches += launches;
  check_launch();
}

// ---------------------------------------------------------------------------
// Algorithm 3 driver
// ---------------------------------------------------------------------------
// One run of Algorithm 3 in precision S.  tol_given > 0 replaces the
// tolerance max(eps_abs, eps_rel xi_0) (FP64 continuation of an FP32 run);
// stall_window > 0 stops with A_STALL when xi has not halved for that many
// iterations.  *final_action receives the last decision.
template <typename S>
static int solve_host(Problem& P, const double* x0_dev, const spock_settings& s, double* z_dev, double* eta_dev,
                      int warm, spock_info* info, cudaStream_t st, double tol_given, int stall_window,
                      int* final_action_out) {
  const int mem = std::max(0, std::min<int>(s.memory, kMaxMemory));
  Workspace* ws = get_ws_impl<S>(P, mem);
  const DevFactors<S>& f = factors<S>(P);
  const int64_t nz = P.off.n_z, nv = ws->n_v;
  Ctx c{&P, ws, default_alpha(P, s.alpha), st, P.idx.stage_begin};
  S* V[3];
  S* TV[3];
  for (int i = 0; i < 3; ++i) {
    V[i] = (S*)ws->v[i];
    TV[i] = (S*)ws->Tv[i];
  }
  S* d = (S*)ws->d;
  S* MR = (S*)ws->MR;
  S* Dm = (S*)ws->D;
  // inputs
  convert<S, double>(x0_dev, f.x0, P.nx, st);
  if (warm) {
    convert<S, double>(z_dev, V[0], nz, st);
    convert<S, double>(eta_dev, V[0] + nz, P.off.n_eta, st);
  } else {
    CUDA_TRY(cudaMemsetAsync(V[0], 0, sizeof(S) * nv, st));
  }
  if (mem > 0) {
    CUDA_TRY(cudaMemsetAsync(MR, 0, sizeof(S) * ws->ld * mem, st));
    CUDA_TRY(cudaMemsetAsync(Dm, 0, sizeof(S) * ws->ld * mem, st));
  }
  const int max_iter = std::max(0, s.max_iter);
  int32_t* trace_dev = nullptr;
  if (s.trace && max_iter > 0) {
    if (ws->trace_cap < max_iter) {
      ws->trace = (int32_t*)ws->alloc(sizeof(int32_t) * 2 * (size_t)max_iter);
      ws->trace_cap = max_iter;
    }
    trace_dev = ws->trace;
    CUDA_TRY(cudaMemsetAsync(trace_dev, 0xff, sizeof(int32_t) * 2 * (size_t)max_iter, st));
  }
  SmState h{};
  h.alpha = c.alpha;
  h.eps_abs = s.eps_abs;
  h.eps_rel = s.eps_rel;
  h.c0 = s.c0;
  h.c1 = s.c1;
  h.c2 = s.c2;
  h.beta = s.beta;
  h.sigma = s.sigma;
  h.lam = s.lambda;
  h.rho_coef = s.rho_coef;
  h.max_iter = max_iter;
  h.max_back = std::max(0, s.max_backtracks);
  h.mem = mem;
  h.record_trace = trace_dev != nullptr;
  h.tol = tol_given;
  h.stall_window = stall_window;
  sm_init_state(ws->st, h, st);
  ws->launches = 0;
  if (s.profile) ws->prof.start();
  else ws->prof.on = false;
  double* stats[3] = {ws->stats, ws->stats + 8, ws->stats + 16};
  CUDA_TRY(cudaEventRecord(ws->e0, st));
  int cur = 0, prev = 1, trial = 2;
  int nT = 0;
  eval_T<S>(c, V[cur], TV[cur], nullptr, stats[cur]);
  ++nT;
  bool have_prev = false;
  int stored = 0, next_slot = 0;
  int final_action = A_NONE;
  auto read_action = [&]() -> int {
    CUDA_TRY(cudaMemcpyAsync(ws->h_action, &ws->st->action, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (ws->prof.on) ws->prof.harvest();
    return ws->h_action[0];
  };
  for (;;) {
    launch_sm_after_eval(ws->st, stats[cur], trace_dev, st);
    ws->launches += 1;
    const int act = read_action();
    if (act == A_DONE || act == A_MAXIT || act == A_NUMERICAL || act == A_STALL) {
      final_action = act;
      break;
    }
    int cnt = 0;
    if (have_prev && mem > 0) {
      const int slot = next_slot;
      next_slot = (next_slot + 1) % mem;
      stored = std::min(stored + 1, mem);
      cnt = stored;
      int order[kMaxMemory];
      for (int j = 0; j < kMaxMemory; ++j) order[j] = 0;
      for (int j = 0; j < cnt; ++j) order[j] = ((slot - j) % mem + mem) % mem;
      launch_aa_update<S>(ws->st, V[cur], TV[cur], V[prev], TV[prev], MR, Dm, nv, ws->ld, slot, cnt, order,
                          ws->paa, ws->grid_v, st);
      ws->launches += 2;
    }
    launch_aa_direction<S>(ws->st, V[cur], TV[cur], Dm, nv, ws->ld, cnt, d, V[trial], ws->grid_v, st);
    ws->launches += 1;
    check_launch();
    if (act == A_K0) {
      eval_T<S>(c, V[trial], TV[trial], nullptr, stats[trial]);
      ++nT;
      const int old_prev = prev;
      prev = cur;
      cur = trial;
      trial = old_prev;
    } else {
      bool numerical = false;
      for (;;) {
        eval_T<S>(c, V[trial], TV[trial], d, stats[trial]);
        ++nT;
        launch_sm_line_search(ws->st, stats[trial], trace_dev, st);
        ws->launches += 1;
        const int la = read_action();
        if (la == A_K1) {
          const int old_prev = prev;
          prev = cur;
          cur = trial;
          trial = old_prev;
          break;
        }
        if (la == A_K2 || la == A_CAP) {
          if (la == A_K2) {
            launch_k2_point<S>(ws->st, V[cur], V[trial], TV[trial], V[prev], nv, ws->grid_v, st);
          } else {
            launch_km_point<S>(ws->st, V[cur], TV[cur], V[prev], nv, ws->grid_v, st);
          }
          ws->launches += 1;
          eval_T<S>(c, V[prev], TV[prev], nullptr, stats[prev]);
          ++nT;
          const int newcur = prev;
          prev = cur;
          cur = newcur;
          break;
        }
        if (la == A_NUMERICAL) {
          numerical = true;
          break;
        }
        launch_ls_point<S>(ws->st, V[cur], d, V[trial], nv, ws->grid_v, st);
        ws->launches += 1;
      }
      if (numerical) {
        final_action = A_NUMERICAL;
        break;
      }
    }
    have_prev = true;
  }
  CUDA_TRY(cudaEventRecord(ws->e1, st));
  // outputs: T(v) of the final iterate
  convert<double, S>(TV[cur], z_dev, nz, st);
  convert<double, S>(TV[cur] + nz, eta_dev, P.off.n_eta, st);
  check_launch();
  SmState fin;
  CUDA_TRY(cudaMemcpyAsync(&fin, ws->st, sizeof(SmState), cudaMemcpyDeviceToHost, st));
  if (trace_dev)
    CUDA_TRY(cudaMemcpyAsync(s.trace, trace_dev, sizeof(int32_t) * 2 * (size_t)max_iter, cudaMemcpyDeviceToHost,
                             st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (ws->prof.on) ws->prof.harvest();
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ws->e0, ws->e1);
  if (final_action_out) *final_action_out = final_action;
  int status = final_action == A_DONE ? SPOCK_OK
                                      : ((final_action == A_MAXIT || final_action == A_STALL) ? SPOCK_MAX_ITER
                                                                                              : SPOCK_ERR_NUMERICAL);
  if (info) {
    info->status = status;
    info->iterations = fin.k;
    info->n_T = nT;
    info->n_K0 = fin.n_k0;
    info->n_K1 = fin.n_k1;
    info->n_K2 = fin.n_k2;
    info->n_cap = fin.n_cap;
    info->n_backtracks = fin.n_back;
    info->xi = fin.xi;
    info->xi0 = fin.xi0;
    info->alpha = c.alpha;
    info->solve_ms = ms;
    info->n_launches = (int32_t)ws->launches;
    info->n_timed = ws->prof.on ? ws->prof.n : 0;
    for (int g = 0; g < Profiler::kGroups; ++g) info->t_group_ms[g] = ws->prof.on ? ws->prof.acc[g] : 0.0;
    info->fp64_iterations = sizeof(S) == 8 ? fin.k : 0;
    info->certified = sizeof(S) == 8 ? 1 : 0;
    info->xi_fp32 = sizeof(S) == 8 ? NAN : fin.xi;
  }
  ws->prof.on = false;
  check_device_flag(P, st);
  if (status == SPOCK_ERR_NUMERICAL) return fail(status, "non-finite residual during the iteration");
  return status;
}

// ---------------------------------------------------------------------------
// Algorithm 3, device-driven: fixed rounds replayed from a CUDA graph
// ---------------------------------------------------------------------------
constexpr int kRounds = 8;  // rounds per graph launch (one host check per launch)

template <typename S>
static int solve_graph(Problem& P, const double* x0_dev, const spock_settings& s, double* z_dev, double* eta_dev,
                       int warm, spock_info* info, cudaStream_t user_st, double tol_given, int stall_window,
                       int* final_action_out, bool cta = false) {
  const int mem = std::max(0, std::min<int>(s.memory, kMaxMemory));
  Workspace* ws = get_ws_impl<S>(P, mem);
  const DevFactors<S>& f = factors<S>(P);
  const int64_t nz = P.off.n_z, nv = ws->n_v;
  cudaStream_t st = ws->stream;
  CUDA_TRY(cudaStreamSynchronize(user_st));  // inputs produced on the caller's stream
  const double alpha = default_alpha(P, s.alpha);
  Ctx c{&P, ws, alpha, st, P.idx.stage_begin};
  S* V = (S*)ws->v[0];
  S* TV = (S*)ws->Tv[0];
  S* Vt = (S*)ws->v[2];
  S* TVt = (S*)ws->Tv[2];
  S* d = (S*)ws->d;
  S* MR = (S*)ws->MR;
  S* Dm = (S*)ws->D;
  double* stats_t = ws->stats;
  convert<S, double>(x0_dev, f.x0, P.nx, st);
  if (warm) {
    convert<S, double>(z_dev, Vt, nz, st);
    convert<S, double>(eta_dev, Vt + nz, P.off.n_eta, st);
  } else {
    CUDA_TRY(cudaMemsetAsync(Vt, 0, sizeof(S) * nv, st));
  }
  CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(S) * nv, st));
  const int max_iter = std::max(0, s.max_iter);
  int32_t* trace_dev = nullptr;
  if (s.trace && max_iter > 0) {
    if (ws->trace_cap < max_iter) {
      ws->trace = (int32_t*)ws->alloc(sizeof(int32_t) * 2 * (size_t)max_iter);
      ws->trace_cap = max_iter;
      if (ws->gexec) {
        cudaGraphExecDestroy(ws->gexec);
        ws->gexec = nullptr;
      }
    }
    trace_dev = ws->trace;
    CUDA_TRY(cudaMemsetAsync(trace_dev, 0xff, sizeof(int32_t) * 2 * (size_t)max_iter, st));
  }
  SmState h{};
  h.alpha = alpha;
  h.eps_abs = s.eps_abs;
  h.eps_rel = s.eps_rel;
  h.c0 = s.c0;
  h.c1 = s.c1;
  h.c2 = s.c2;
  h.beta = s.beta;
  h.sigma = s.sigma;
  h.lam = s.lambda;
  h.rho_coef = s.rho_coef;
  h.max_iter = max_iter;
  h.max_back = std::max(0, s.max_backtracks);
  h.mem = mem;
  h.record_trace = trace_dev != nullptr;
  h.tol = tol_given;
  h.stall_window = stall_window;
  h.pending = P_INIT;
  h.n_T = 1;
  sm_init_state(ws->st, h, st);
  const int32_t* skip = &ws->st->done;
  // the graph of kRounds rounds (captured once per workspace and settings)
  const int grid_v = ws->grid_v;
  auto round = [&](cudaStream_t s2) {
    Ctx c2 = c;
    c2.st = s2;
    launch_round_decide(ws->st, stats_t, trace_dev, s2);
    launch_round_commit<S>(ws->st, V, TV, Vt, TVt, MR, Dm, nv, ws->ld, mem, ws->paa, grid_v, s2);
    launch_round_aa_solve(ws->st, ws->paa, grid_v, s2);
    launch_round_point<S>(ws->st, V, TV, Vt, TVt, d, Dm, nv, ws->ld, mem, grid_v, s2);
    const int64_t before = ws->launches;
    eval_T<S>(c2, Vt, TVt, d, stats_t, skip);
    return 4 + (int)(ws->launches - before);
  };
  ws->launches = 0;
  const int64_t max_rounds = (int64_t)(max_iter + 1) * (h.max_back + 3) + 2;
  if (cta) {  // the whole solve in one block (cta.cu): one launch
    const BInst<S> hb = make_binst<S>(P, ws, alpha);
    if (!ws->cta_bi) ws->cta_bi = ws->alloc(sizeof(BInst<S>));
    CUDA_TRY(cudaMemcpyAsync(ws->cta_bi, &hb, sizeof(hb), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));  // hb lives on this stack frame
    CUDA_TRY(cudaEventRecord(ws->e0, st));
    launch_solve_cta<S>((const BInst<S>*)ws->cta_bi, 1, P.nx + P.nu, mem, max_rounds, trace_dev, st);
    check_launch();
    ws->launches = 1;
  } else {
    CUDA_TRY(cudaEventRecord(ws->e0, st));
    eval_T<S>(c, Vt, TVt, nullptr, stats_t, nullptr);  // T(v0); also sets kernel attributes outside capture
    const int64_t launches0 = ws->launches;
    const char* fam = getenv("SPOCK_RICCATI_KERNELS");
    const int trace_key = (trace_dev ? 1 : 0) + 2 * (s.profile ? 1 : 0) +
                          4 * (fam && fam[0] ? (int)(unsigned char)fam[0] : 0);
    if (s.profile) ws->prof.start();  // event slot r is recorded by round r of every replay
    if (!ws->gexec || ws->g_alpha != alpha || ws->g_trace != trace_key) {
      if (ws->gexec) {
        cudaGraphExecDestroy(ws->gexec);
        ws->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      int per = 0;
      for (int r = 0; r < kRounds; ++r) per = round(st);
      CUDA_TRY(cudaStreamEndCapture(st, &g));
      cudaError_t e = cudaGraphInstantiate(&ws->gexec, g, 0);
      cudaGraphDestroy(g);
      CUDA_TRY(e);
      ws->g_alpha = alpha;
      ws->g_trace = trace_key;
      ws->g_launches_per_round = per;
    }
    int64_t launches = launches0;
    int64_t rounds = 0;
    int32_t rounds_done = 0;
    for (;;) {
      CUDA_TRY(cudaGraphLaunch(ws->gexec, st));
      rounds += kRounds;
      launches += (int64_t)kRounds * ws->g_launches_per_round;
      CUDA_TRY(cudaMemcpyAsync(ws->h_done, &ws->st->done, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaMemcpyAsync(ws->h_done + 1, &ws->st->rounds, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaStreamSynchronize(st));
      if (s.profile) {  // rounds that evaluated T in this replay: the first (rounds now - rounds before)
        const int ran = ws->h_done[1] - rounds_done - (ws->h_done[0] ? 1 : 0);
        ws->prof.used = kRounds;
        ws->prof.harvest_first(std::max(0, std::min(ran, kRounds)));
      }
      rounds_done = ws->h_done[1];
      if (ws->h_done[0] || rounds > max_rounds) break;
    }
    ws->launches = launches;
  }
  const int64_t launches = ws->launches;
  CUDA_TRY(cudaEventRecord(ws->e1, st));
  convert<double, S>(TV, z_dev, nz, st);
  convert<double, S>(TV + nz, eta_dev, P.off.n_eta, st);
  check_launch();
  SmState fin;
  CUDA_TRY(cudaMemcpyAsync(&fin, ws->st, sizeof(SmState), cudaMemcpyDeviceToHost, st));
  if (trace_dev)
    CUDA_TRY(cudaMemcpyAsync(s.trace, trace_dev, sizeof(int32_t) * 2 * (size_t)max_iter, cudaMemcpyDeviceToHost,
                             st));
  CUDA_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ws->e0, ws->e1);
  const int final_action = fin.done ? fin.action : A_MAXIT;
  if (final_action_out) *final_action_out = final_action;
  const int status = final_action == A_DONE ? SPOCK_OK
                                            : ((final_action == A_MAXIT || final_action == A_STALL)
                                                   ? SPOCK_MAX_ITER
                                                   : SPOCK_ERR_NUMERICAL);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = status;
    info->iterations = fin.k;
    info->n_T = fin.n_T;
    info->n_K0 = fin.n_k0;
    info->n_K1 = fin.n_k1;
    info->n_K2 = fin.n_k2;
    info->n_cap = fin.n_cap;
    info->n_backtracks = fin.n_back;
    info->xi = fin.xi;
    info->xi0 = fin.xi0;
    info->alpha = alpha;
    info->solve_ms = ms;
    info->n_launches = (int32_t)std::min<int64_t>(launches, INT32_MAX);
    info->fp64_iterations = sizeof(S) == 8 ? fin.k : 0;
    info->certified = sizeof(S) == 8 ? 1 : 0;
    info->xi_fp32 = sizeof(S) == 8 ? NAN : fin.xi;
    info->n_timed = ws->prof.on ? ws->prof.n : 0;
    for (int g = 0; g < Profiler::kGroups; ++g) info->t_group_ms[g] = ws->prof.on ? ws->prof.acc[g] : 0.0;
  }
  ws->prof.on = false;
  check_device_flag(P, st);
  if (status == SPOCK_ERR_NUMERICAL) return fail(status, "non-finite residual during the iteration");
  return status;
}

// Device-driven rounds replayed from a CUDA graph, or -- for small problems
// (at most kCtaAutoNodes nodes, nx + nu <= 62, Anderson memory 0, 3 or 5, no
// profiling) -- the whole solve in one single-block launch (cta.cu).
// SPOCK_DRIVER = host / graph / cta selects the host-driven loop (one host
// decision per SuperMann step), the graph or the single block.
constexpr int kCtaAutoNodes = 64;
template <typename S>
static int solve_impl(Problem& P, const double* x0_dev, const spock_settings& s, double* z_dev, double* eta_dev,
                      int warm, spock_info* info, cudaStream_t st, double tol_given = 0.0, int stall_window = 0,
                      int* final_action_out = nullptr) {
  const char* drv = getenv("SPOCK_DRIVER");
  if (drv && drv[0] == 'h')
    return solve_host<S>(P, x0_dev, s, z_dev, eta_dev, warm, info, st, tol_given, stall_window, final_action_out);
  const int mem = std::max(0, std::min<int>(s.memory, kMaxMemory));
  const bool cta_ok = cta_supported(P.nx, P.nu, mem) && !s.profile && !P.general;
  const bool cta = cta_ok && (drv && drv[0] == 'c' ? true : (!(drv && drv[0]) && P.tree.n <= kCtaAutoNodes));
  return solve_graph<S>(P, x0_dev, s, z_dev, eta_dev, warm, info, st, tol_given, stall_window, final_action_out,
                        cta);
}

template <typename S>
static int cp_impl(Problem& P, const double* x0_dev, int k, double alpha, double* z_dev, double* eta_dev,
                   double* xi_out, cudaStream_t st) {
  Workspace* ws = get_ws_impl<S>(P, 0);
  const DevFactors<S>& f = factors<S>(P);
  const int64_t nz = P.off.n_z;
  Ctx c{&P, ws, default_alpha(P, alpha), st, P.idx.stage_begin};
  S* a = (S*)ws->v[0];
  S* b = (S*)ws->v[1];
  convert<S, double>(x0_dev, f.x0, P.nx, st);
  convert<S, double>(z_dev, a, nz, st);
  convert<S, double>(eta_dev, a + nz, P.off.n_eta, st);
  for (int i = 0; i < k; ++i) {
    eval_T<S>(c, a, b, nullptr, (i == k - 1 && xi_out) ? ws->stats : nullptr);
    std::swap(a, b);
  }
  convert<double, S>(a, z_dev, nz, st);
  convert<double, S>(a + nz, eta_dev, P.off.n_eta, st);
  check_launch();
  if (xi_out) {
    if (k > 0) {
      double h[8];
      CUDA_TRY(cudaMemcpyAsync(h, ws->stats, sizeof(h), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaStreamSynchronize(st));
      *xi_out = std::max(h[ST_XIP], h[ST_XID]);
    } else {
      *xi_out = NAN;
    }
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  check_device_flag(P, st);
  return SPOCK_OK;
}

// ---------------------------------------------------------------------------
// batches: every kernel of a round launched once for all instances
// (batch.cuh); kBatchRounds rounds captured in one CUDA graph
// ---------------------------------------------------------------------------
constexpr int kBatchRounds = 8;
constexpr int kVecElemsPerThread = 16;   // commit / point kernels of the batch

// Device copy of a block map: inst[nblocks] | base[n] | cnt[n] | stage[n].
struct DevMap {
  int32_t* buf = nullptr;
  int nblocks = 0;
  BMap view(int n) const { return BMap{buf, buf + nblocks, buf + nblocks + n, buf + nblocks + 2 * n}; }
};

struct Batch {
  int32_t tag = TAG_BATCH;
  std::vector<Problem*> probs;
  cudaStream_t main = nullptr;
  // plan of the batched launches for one precision, node tile and memory
  int p_prec = -1, p_mem = -1, p_tile = -1, p_fam = -1;
  std::vector<void*> p_ws;
  std::vector<double> p_alpha;
  void* bi_dev = nullptr;  // BInst<S>[n]
  DevMap node, vec, chain_b, chain_f;
  std::vector<DevMap> bwd_lv, fwd_lv;  // branching stages, one map per level
  int fam = 0;                         // Riccati kernels: 0 direct, 1 staged (bulk copies)
  TmaBatchShape tsh;
  int J = 1, SL = 1;
  int launches_per_eval = 0;
  // graph of kBatchRounds rounds
  cudaGraphExec_t gexec = nullptr;
  double g_alpha = -1.0;
  int g_launches = 0;
  int tuned_tile[2] = {0, 0};  // node tile (nodes per warp) picked by the autotuner, per precision
  int tuned_fam[2] = {-1, -1};  // Riccati kernel family picked by the autotuner, per precision
  int tuned_cta[2] = {0, 0};     // 1: the single-block persistent solve was faster
  SmState** st_ptrs = nullptr;
  int32_t* done_dev = nullptr;
  int32_t* done_host = nullptr;  // pinned
  void* tab_dev = nullptr;       // pointer / length tables of the batched copies
  void* tab_host = nullptr;      // pinned
  size_t tab_bytes = 0;
  SmState* st_stage = nullptr;   // staging of the instances' states
  int st_stage_n = 0;
  std::vector<int32_t*> bufs;
  void free_plan() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    for (auto b : bufs) cudaFree(b);
    bufs.clear();
    if (bi_dev) cudaFree(bi_dev);
    bi_dev = nullptr;
    bwd_lv.clear();
    fwd_lv.clear();
    p_prec = p_mem = p_tile = p_fam = -1;
    p_ws.clear();
    p_alpha.clear();
  }
  ~Batch() {
    free_plan();
    if (main) cudaStreamDestroy(main);
    if (st_ptrs) cudaFree(st_ptrs);
    if (done_dev) cudaFree(done_dev);
    if (done_host) cudaFreeHost(done_host);
    if (tab_dev) cudaFree(tab_dev);
    if (tab_host) cudaFreeHost(tab_host);
    if (st_stage) cudaFree(st_stage);
  }
  // uploads one block map from per-instance block counts (and stages)
  DevMap make_map(const std::vector<int>& cnt, const std::vector<int>& stage) {
    const int n = (int)cnt.size();
    DevMap m;
    std::vector<int32_t> h;
    std::vector<int32_t> base(n), cn(n), stg(n);
    int total = 0;
    for (int i = 0; i < n; ++i) {
      base[i] = total;
      cn[i] = cnt[i];
      stg[i] = stage.empty() ? -1 : stage[i];
      total += cnt[i];
    }
    h.reserve((size_t)total + 3 * n);
    for (int i = 0; i < n; ++i)
      for (int b = 0; b < cnt[i]; ++b) h.push_back(i);
    h.insert(h.end(), base.begin(), base.end());
    h.insert(h.end(), cn.begin(), cn.end());
    h.insert(h.end(), stg.begin(), stg.end());
    CUDA_TRY(cudaMalloc(&m.buf, sizeof(int32_t) * h.size()));
    bufs.push_back(m.buf);
    CUDA_TRY(cudaMemcpy(m.buf, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice));
    m.nblocks = total;
    return m;
  }
};

__global__ void k_gather_done(SmState* const* __restrict__ sts, int n, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sts[i]->done;
}

// Block maps and instance views for the batched launches.  tile = nodes per
// warp of the node kernels (the autotuned tile shape); the vector kernels
// take kVecElemsPerThread elements per thread; the Riccati passes use the
// direct kernels (fam 0: one warp per chain / node) or the staged ones
// (fam 1: chain blocks of wpb warps, one block per branching node; falls
// back to direct if a layout does not fit).
template <typename S>
static void batch_plan(Batch& B, const std::vector<Workspace*>& wss, const std::vector<double>& alphas, int mem,
                       int tile, int fam) {
  std::vector<void*> ws_now(wss.begin(), wss.end());
  if (B.p_prec == (int)sizeof(S) && B.p_mem == mem && B.p_tile == tile && B.p_fam == fam && B.p_ws == ws_now &&
      B.p_alpha == alphas)
    return;
  B.free_plan();
  const int n = (int)B.probs.size();
  std::vector<BInst<S>> h(n);
  std::vector<int> cn(n), cv(n);
  int max_cs = 0, max_ch = 1;
  B.J = 1;
  B.SL = 1;
  for (int i = 0; i < n; ++i) {
    Problem& P = *B.probs[i];
    Workspace* ws = wss[i];
    BInst<S>& b = h[i];
    b = make_binst<S>(P, ws, alphas[i]);
    const int nn = P.tree.n;
    b.nb_node = std::max(1, std::min(ws->grid_d, (nn + kWarpsPerBlock * tile - 1) / (kWarpsPerBlock * tile)));
    const int64_t per_block = (int64_t)256 * kVecElemsPerThread;
    b.nb_vec = (int)std::max<int64_t>(1, std::min<int64_t>(ws->grid_v, (ws->n_v + per_block - 1) / per_block));
    cn[i] = b.nb_node;
    cv[i] = b.nb_vec;
    max_cs = std::max(max_cs, (int)P.tree.chain_stage);
    for (int t = 0; t < P.tree.chain_stage; ++t) max_ch = std::max(max_ch, (int)P.tree.stage_maxch[t]);
    B.J = std::max(B.J, (P.nx + P.nu + 2 + 31) / 32);
    B.SL = std::max(B.SL, (P.nx + P.nu + 31) / 32);
  }
  CUDA_TRY(cudaMalloc(&B.bi_dev, sizeof(BInst<S>) * n));
  CUDA_TRY(cudaMemcpy(B.bi_dev, h.data(), sizeof(BInst<S>) * n, cudaMemcpyHostToDevice));
  B.fam = fam;
  if (B.fam == 1) {
    std::vector<KP<S>> kps(n);
    for (int i = 0; i < n; ++i) kps[i] = h[i].kp;
    if (!tma_batch_shape<S>(kps, max_ch, B.tsh)) B.fam = 0;
  }
  const int cw_b = B.fam == 1 ? B.tsh.wpb_bwd : kWarpsPerBlock;  // chains per chain block
  const int cw_f = B.fam == 1 ? B.tsh.wpb_fwd : kWarpsPerBlock;
  const int npb = B.fam == 1 ? 1 : kWarpsPerBlock;                // branching nodes per stage block
  std::vector<int> ccb(n), ccf(n);
  for (int i = 0; i < n; ++i) {
    const KP<S>& k = h[i].kp;
    const bool chains = k.n_chains > 0 && k.chain_stage < k.N;
    ccb[i] = chains ? (k.n_chains + cw_b - 1) / cw_b : 0;
    ccf[i] = chains ? (k.n_chains + cw_f - 1) / cw_f : 0;
  }
  B.node = B.make_map(cn, {});
  B.vec = B.make_map(cv, {});
  B.chain_b = B.make_map(ccb, {});
  B.chain_f = B.make_map(ccf, {});
  for (int L = 0; L < max_cs; ++L) {  // backward: level L is stage cs_i - 1 - L of instance i
    std::vector<int> cnt(n, 0), stg(n, -1);
    for (int i = 0; i < n; ++i) {
      const Tree& t = B.probs[i]->tree;
      const int st = t.chain_stage - 1 - L;
      if (st >= 0) {
        stg[i] = st;
        cnt[i] = (t.stage_begin[st + 1] - t.stage_begin[st] + npb - 1) / npb;
      }
    }
    B.bwd_lv.push_back(B.make_map(cnt, stg));
  }
  for (int L = 0; L < max_cs; ++L) {  // forward: level L is stage L
    std::vector<int> cnt(n, 0), stg(n, -1);
    for (int i = 0; i < n; ++i) {
      const Tree& t = B.probs[i]->tree;
      if (L < t.chain_stage) {
        stg[i] = L;
        cnt[i] = (t.stage_begin[L + 1] - t.stage_begin[L] + npb - 1) / npb;
      }
    }
    B.fwd_lv.push_back(B.make_map(cnt, stg));
  }
  B.launches_per_eval = 5 + 2 * max_cs;
  B.p_prec = (int)sizeof(S);
  B.p_mem = mem;
  B.p_tile = tile;
  B.p_fam = fam;
  B.p_ws = ws_now;
  B.p_alpha = alphas;
}

// One T evaluation of every instance: Vt -> TVt with statistics (direction d).
template <typename S>
static void batch_eval(Batch& B, cudaStream_t st) {
  const int n = (int)B.probs.size();
  const BInst<S>* bi = (const BInst<S>*)B.bi_dev;
  launch_node_ops_b<S>(0, bi, B.node.view(n), B.node.nblocks, n, B.J, st);
  if (B.fam == 1) {
    launch_riccati_tma_b<S>(0, bi, B.chain_b.view(n), B.chain_b.nblocks, B.SL, B.tsh, st);
    for (const DevMap& m : B.bwd_lv) launch_riccati_tma_b<S>(1, bi, m.view(n), m.nblocks, B.SL, B.tsh, st);
    for (const DevMap& m : B.fwd_lv) launch_riccati_tma_b<S>(2, bi, m.view(n), m.nblocks, B.SL, B.tsh, st);
    launch_riccati_tma_b<S>(3, bi, B.chain_f.view(n), B.chain_f.nblocks, B.SL, B.tsh, st);
  } else {
    launch_riccati_b<S>(0, bi, B.chain_b.view(n), B.chain_b.nblocks, B.SL, st);
    for (const DevMap& m : B.bwd_lv) launch_riccati_b<S>(1, bi, m.view(n), m.nblocks, B.SL, st);
    for (const DevMap& m : B.fwd_lv) launch_riccati_b<S>(2, bi, m.view(n), m.nblocks, B.SL, st);
    launch_riccati_b<S>(3, bi, B.chain_f.view(n), B.chain_f.nblocks, B.SL, st);
  }
  launch_node_ops_b<S>(1, bi, B.node.view(n), B.node.nblocks, n, B.J, st);
  launch_node_ops_b<S>(3, bi, B.node.view(n), 0, n, B.J, st);
  check_launch();
}

// Per-instance copies of a batch in one launch each: pointer tables on the
// device, blockIdx.y over instances, x-blocks and threads over the entries.
template <typename D, typename S>
__global__ void k_convert_many(const D* const* __restrict__ in, S* const* __restrict__ out,
                               const int64_t* __restrict__ len, int count) {
  for (int i = blockIdx.y; i < count; i += gridDim.y) {
    const D* a = in[i];
    S* b = out[i];
    const int64_t m = len[i];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
      b[e] = a ? (S)a[e] : S(0);   // a NULL source zero-fills
  }
}
// SmState scatter / gather between per-instance states and a staging array.
__global__ void k_states_many(SmState* const* __restrict__ per, SmState* __restrict__ staging, int count,
                              int to_instances) {
  constexpr int W = (int)(sizeof(SmState) / sizeof(int32_t));
  const int64_t total = (int64_t)count * W;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / W), w = (int)(t % W);
    int32_t* a = reinterpret_cast<int32_t*>(per[i]) + w;
    int32_t* b = reinterpret_cast<int32_t*>(staging + i) + w;
    if (to_instances) *a = *b;
    else *b = *a;
  }
}
static_assert(sizeof(SmState) % sizeof(int32_t) == 0, "SmState is copied as 32-bit words");

// Uploads the pointer/length tables of one batched copy (device scratch of
// the batch, grown on demand) and launches it.
template <typename D, typename S>
static void copy_many(Batch& B, const std::vector<const D*>& in, const std::vector<S*>& out,
                      const std::vector<int64_t>& len, cudaStream_t st) {
  const int n = (int)in.size();
  if (n == 0) return;
  const size_t bytes = (size_t)n * (2 * sizeof(void*) + sizeof(int64_t));
  if (B.tab_bytes < bytes) {
    if (B.tab_dev) cudaFree(B.tab_dev);
    if (B.tab_host) cudaFreeHost(B.tab_host);
    B.tab_dev = nullptr;
    B.tab_host = nullptr;
    CUDA_TRY(cudaMalloc(&B.tab_dev, bytes));
    CUDA_TRY(cudaMallocHost(&B.tab_host, bytes));
    B.tab_bytes = bytes;
  }
  CUDA_TRY(cudaStreamSynchronize(st));  // the pinned table of the previous copy is free again
  char* h = (char*)B.tab_host;
  std::memcpy(h, in.data(), n * sizeof(void*));
  std::memcpy(h + n * sizeof(void*), out.data(), n * sizeof(void*));
  std::memcpy(h + 2 * n * sizeof(void*), len.data(), n * sizeof(int64_t));
  CUDA_TRY(cudaMemcpyAsync(B.tab_dev, h, bytes, cudaMemcpyHostToDevice, st));
  char* d = (char*)B.tab_dev;
  int64_t mx = 1;
  for (int64_t l : len) mx = std::max(mx, l);
  const dim3 grid((unsigned)std::min<int64_t>((mx + 255) / 256, 64), (unsigned)std::min(n, 65535));
  k_convert_many<D, S><<<grid, 256, 0, st>>>((const D* const*)d, (S* const*)(d + n * sizeof(void*)),
                                             (const int64_t*)(d + 2 * n * sizeof(void*)), n);
  check_launch();
}

// Host states -> every instance's device state (to_instances) or back, with
// one staging copy and one scatter / gather launch.
static void batch_states(Batch& B, const std::vector<Workspace*>& wss, SmState* host, bool to_instances,
                         cudaStream_t st) {
  const int n = (int)wss.size();
  if (B.st_stage_n < n) {
    if (B.st_stage) cudaFree(B.st_stage);
    B.st_stage = nullptr;
    CUDA_TRY(cudaMalloc(&B.st_stage, sizeof(SmState) * n));
    B.st_stage_n = n;
  }
  std::vector<SmState*> ptrs(n);
  for (int i = 0; i < n; ++i) ptrs[i] = wss[i]->st;
  CUDA_TRY(cudaMemcpyAsync(B.st_ptrs, ptrs.data(), sizeof(SmState*) * n, cudaMemcpyHostToDevice, st));
  constexpr int W = (int)(sizeof(SmState) / sizeof(int32_t));
  const int blocks = (int)std::min<int64_t>(((int64_t)n * W + 255) / 256, 1024);
  if (to_instances) {
    CUDA_TRY(cudaMemcpyAsync(B.st_stage, host, sizeof(SmState) * n, cudaMemcpyHostToDevice, st));
    k_states_many<<<blocks, 256, 0, st>>>(B.st_ptrs, B.st_stage, n, 1);
  } else {
    k_states_many<<<blocks, 256, 0, st>>>(B.st_ptrs, B.st_stage, n, 0);
    CUDA_TRY(cudaMemcpyAsync(host, B.st_stage, sizeof(SmState) * n, cudaMemcpyDeviceToHost, st));
  }
  check_launch();
  CUDA_TRY(cudaStreamSynchronize(st));  // host buffer and pointer table in use until here
}

// Puts every instance at its starting point: Vt = v0 (cold: 0, warm: the
// caller's (z, eta)), d = 0, fresh SuperMann state -- a handful of launches
// for the whole batch.
template <typename S>
static void batch_init(Batch& B, const std::vector<Workspace*>& wss, const std::vector<double>& alphas,
                       const spock_settings& s, int mem, const double* const* x0, double* const* z,
                       double* const* eta, int warm) {
  const int n = (int)B.probs.size();
  cudaStream_t st = B.main;
  std::vector<const double*> src;
  std::vector<S*> dst;
  std::vector<int64_t> len;
  for (int i = 0; i < n; ++i) {  // x0 and the starting points (NULL source: zeros)
    Problem& P = *B.probs[i];
    Workspace* ws = wss[i];
    S* Vt = (S*)ws->v[2];
    src.push_back(x0[i]);
    dst.push_back(factors<S>(P).x0);
    len.push_back(P.nx);
    src.push_back(warm ? z[i] : nullptr);
    dst.push_back(Vt);
    len.push_back(P.off.n_z);
    src.push_back(warm ? eta[i] : nullptr);
    dst.push_back(Vt + P.off.n_z);
    len.push_back(P.off.n_eta);
    src.push_back(nullptr);
    dst.push_back((S*)ws->d);
    len.push_back(ws->n_v);
  }
  copy_many<double, S>(B, src, dst, len, st);
  std::vector<SmState> hs(n);
  for (int i = 0; i < n; ++i) {
    SmState& h = hs[i];
    h = SmState{};
    h.alpha = alphas[i];
    h.eps_abs = s.eps_abs;
    h.eps_rel = s.eps_rel;
    h.c0 = s.c0;
    h.c1 = s.c1;
    h.c2 = s.c2;
    h.beta = s.beta;
    h.sigma = s.sigma;
    h.lam = s.lambda;
    h.rho_coef = s.rho_coef;
    h.max_iter = std::max(0, s.max_iter);
    h.max_back = std::max(0, s.max_backtracks);
    h.mem = mem;
    h.pending = P_INIT;
    h.n_T = 1;
  }
  batch_states(B, wss, hs.data(), true, st);
}

// Autotuner of the batch.  Candidates: the work-list kernels with node tile
// 1, 2, 4, 8 or 16 (nodes per warp of the node kernels) and the direct or
// staged Riccati family, and -- when every instance fits it -- the
// single-block persistent solve (cta.cu).  Each candidate runs the
// evaluation of T at the starting points and kTuneRounds rounds from the
// same state; the fastest is cached per batch and precision.
// SPOCK_BATCH_TILE fixes the tile, SPOCK_RICCATI_KERNELS = direct / tma the
// family, SPOCK_BATCH_MODE = list / cta the mode.
constexpr int kTuneRounds = 4;
struct BatchCfg {
  int tile, fam;
  bool cta;
};

template <typename S>
static void batch_rounds_direct(Batch& B, int mem, int rounds) {
  const int n = (int)B.probs.size();
  const BInst<S>* bi = (const BInst<S>*)B.bi_dev;
  batch_eval<S>(B, B.main);
  for (int r = 0; r < rounds; ++r) {
    launch_round_decide_b<S>(bi, n, B.main);
    launch_round_commit_b<S>(bi, B.vec.view(n), B.vec.nblocks, mem, B.main);
    launch_round_aa_solve_b<S>(bi, n, B.main);
    launch_round_point_b<S>(bi, B.vec.view(n), B.vec.nblocks, mem, B.main);
    batch_eval<S>(B, B.main);
  }
}

static int batch_max_nxu(const Batch& B) {
  int v = 0;
  for (const Problem* P : B.probs) v = std::max(v, P->nx + P->nu);
  return v;
}

template <typename S>
static BatchCfg batch_tune(Batch& B, const std::vector<Workspace*>& wss, const std::vector<double>& alphas, int mem,
                           const spock_settings& s, const double* const* x0, double* const* z,
                           double* const* eta, int warm) {
  std::vector<int> tiles = {1, 2, 4, 8, 16}, fams = {0, 1};
  const char* env = getenv("SPOCK_BATCH_TILE");
  if (env && env[0]) {
    const int t = atoi(env);
    if (t == 1 || t == 2 || t == 4 || t == 8 || t == 16) tiles = {t};
  }
  const char* ek = getenv("SPOCK_RICCATI_KERNELS");
  if (ek && ek[0] == 'd') fams = {0};
  if (ek && ek[0] == 't') fams = {1};
  bool cta_ok = true;
  for (const Problem* P : B.probs) cta_ok = cta_ok && cta_supported(P->nx, P->nu, mem);
  bool try_list = true;
  const char* em = getenv("SPOCK_BATCH_MODE");
  if (em && em[0] == 'l') cta_ok = false;
  if (em && em[0] == 'c' && cta_ok) try_list = false;
  const bool cacheable = tiles.size() > 1 && fams.size() > 1 && !(em && em[0]);
  const int pi = sizeof(S) == 8 ? 0 : 1;
  if (cacheable && B.tuned_tile[pi] > 0) return {B.tuned_tile[pi], B.tuned_fam[pi], B.tuned_cta[pi] != 0};
  cudaEvent_t a, b;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  float best = 1e30f;
  BatchCfg pick{tiles[0], fams[0], false};
  auto timed = [&](auto&& run) {
    batch_init<S>(B, wss, alphas, s, mem, x0, z, eta, warm);
    CUDA_TRY(cudaEventRecord(a, B.main));
    run();
    CUDA_TRY(cudaEventRecord(b, B.main));
    CUDA_TRY(cudaEventSynchronize(b));
    check_launch();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  };
  if (try_list) {
    for (int fam : fams) {
      for (int tile : tiles) {
        batch_plan<S>(B, wss, alphas, mem, tile, fam);
        if (B.fam != fam) continue;  // staged layout does not fit
        timed([&] { batch_rounds_direct<S>(B, mem, 1); });  // warm-up
        const float ms = timed([&] { batch_rounds_direct<S>(B, mem, kTuneRounds); });
        if (ms < best) {
          best = ms;
          pick = {tile, fam, false};
        }
      }
    }
  }
  if (cta_ok) {
    batch_plan<S>(B, wss, alphas, mem, pick.tile, pick.fam);
    const int n = (int)B.probs.size(), nxu = batch_max_nxu(B);
    const BInst<S>* bi = (const BInst<S>*)B.bi_dev;
    timed([&] { launch_solve_cta<S>(bi, n, nxu, mem, 1, nullptr, B.main); });  // warm-up
    const float ms = timed([&] { launch_solve_cta<S>(bi, n, nxu, mem, kTuneRounds, nullptr, B.main); });
    if (ms < best) {
      best = ms;
      pick.cta = true;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (cacheable) {
    B.tuned_tile[pi] = pick.tile;
    B.tuned_fam[pi] = pick.fam;
    B.tuned_cta[pi] = pick.cta ? 1 : 0;
  }
  return pick;
}

template <typename S>
static int batch_solve(Batch& B, const double* const* x0, const spock_settings& s, double* const* z,
                       double* const* eta, int warm, spock_info* infos) {
  const int n = (int)B.probs.size();
  const int mem = std::max(0, std::min<int>(s.memory, kMaxMemory));
  const int max_iter = std::max(0, s.max_iter);
  std::vector<Workspace*> wss(n);
  std::vector<double> alphas(n);
  CUDA_TRY(cudaSetDevice(B.probs[0]->device));
  for (int i = 0; i < n; ++i) {
    Problem& P = *B.probs[i];
    wss[i] = get_ws_impl<S>(P, mem);
    alphas[i] = default_alpha(P, s.alpha);
  }
  const BatchCfg cfg = batch_tune<S>(B, wss, alphas, mem, s, x0, z, eta, warm);
  batch_plan<S>(B, wss, alphas, mem, cfg.tile, cfg.fam);
  batch_init<S>(B, wss, alphas, s, mem, x0, z, eta, warm);
  const BInst<S>* bi = (const BInst<S>*)B.bi_dev;
  const int64_t max_rounds = (int64_t)(max_iter + 1) * (std::max(0, s.max_backtracks) + 3) + 2;
  // the graph of kBatchRounds rounds (the plan, hence the graph, is rebuilt
  // when precision, memory, tile or workspaces change)
  const double a_key = s.alpha > 0 ? s.alpha : 0.0;
  if (!cfg.cta && (!B.gexec || B.g_alpha != a_key)) {
    if (B.gexec) {
      cudaGraphExecDestroy(B.gexec);
      B.gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(B.main, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < kBatchRounds; ++r) {
      launch_round_decide_b<S>(bi, n, B.main);
      launch_round_commit_b<S>(bi, B.vec.view(n), B.vec.nblocks, mem, B.main);
      launch_round_aa_solve_b<S>(bi, n, B.main);
      launch_round_point_b<S>(bi, B.vec.view(n), B.vec.nblocks, mem, B.main);
      batch_eval<S>(B, B.main);
    }
    k_gather_done<<<(n + 127) / 128, 128, 0, B.main>>>(B.st_ptrs, n, B.done_dev);
    check_launch();
    CUDA_TRY(cudaStreamEndCapture(B.main, &g));
    cudaError_t e = cudaGraphInstantiate(&B.gexec, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e);
    B.g_alpha = a_key;
    B.g_launches = kBatchRounds * (4 + B.launches_per_eval) + 1;
  }
  {
    std::vector<SmState*> h(n);
    for (int i = 0; i < n; ++i) h[i] = wss[i]->st;
    CUDA_TRY(cudaMemcpy(B.st_ptrs, h.data(), sizeof(SmState*) * n, cudaMemcpyHostToDevice));
  }
  int64_t rounds = 0, graph_launches = 0;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  CUDA_TRY(cudaEventRecord(e0, B.main));
  if (cfg.cta) {  // one persistent launch: every instance solved by its own block
    launch_solve_cta<S>(bi, n, batch_max_nxu(B), mem, max_rounds, nullptr, B.main);
    check_launch();
  } else {
    batch_eval<S>(B, B.main);  // T of the starting points
  }
  for (; !cfg.cta;) {
    CUDA_TRY(cudaGraphLaunch(B.gexec, B.main));
    rounds += kBatchRounds;
    ++graph_launches;
    CUDA_TRY(cudaMemcpyAsync(B.done_host, B.done_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, B.main));
    CUDA_TRY(cudaStreamSynchronize(B.main));
    bool all = true;
    for (int i = 0; i < n; ++i) all = all && B.done_host[i];
    if (all || rounds > max_rounds) break;
  }
  CUDA_TRY(cudaEventRecord(e1, B.main));
  CUDA_TRY(cudaStreamSynchronize(B.main));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int64_t total_launches = cfg.cta ? 1 : B.launches_per_eval + graph_launches * B.g_launches;
  int status = SPOCK_OK;
  std::vector<SmState> fin(n);
  {
    std::vector<const S*> src;
    std::vector<double*> dst;
    std::vector<int64_t> len;
    for (int i = 0; i < n; ++i) {
      Problem& P = *B.probs[i];
      const S* TV = (const S*)wss[i]->Tv[0];
      src.push_back(TV);
      dst.push_back(z[i]);
      len.push_back(P.off.n_z);
      src.push_back(TV + P.off.n_z);
      dst.push_back(eta[i]);
      len.push_back(P.off.n_eta);
    }
    copy_many<S, double>(B, src, dst, len, B.main);
    batch_states(B, wss, fin.data(), false, B.main);
  }
  for (int i = 0; i < n; ++i) {
    const SmState& f = fin[i];
    const int act = f.done ? f.action : A_MAXIT;
    const int si = act == A_DONE ? SPOCK_OK : ((act == A_MAXIT || act == A_STALL) ? SPOCK_MAX_ITER : SPOCK_ERR_NUMERICAL);
    if (si == SPOCK_ERR_NUMERICAL) status = SPOCK_ERR_NUMERICAL;
    else if (si == SPOCK_MAX_ITER && status == SPOCK_OK) status = SPOCK_MAX_ITER;
    if (infos) {
      spock_info& I = infos[i];
      std::memset(&I, 0, sizeof(I));
      I.status = si;
      I.iterations = f.k;
      I.n_T = f.n_T;
      I.n_K0 = f.n_k0;
      I.n_K1 = f.n_k1;
      I.n_K2 = f.n_k2;
      I.n_cap = f.n_cap;
      I.n_backtracks = f.n_back;
      I.xi = f.xi;
      I.xi0 = f.xi0;
      I.alpha = alphas[i];
      I.solve_ms = ms;  // the whole batch
      I.n_launches = (int32_t)std::min<int64_t>(total_launches, INT32_MAX);  // the whole batch
      I.certified = sizeof(S) == 8 ? 1 : 0;
      I.fp64_iterations = sizeof(S) == 8 ? f.k : 0;
      I.xi_fp32 = sizeof(S) == 8 ? NAN : f.xi;
    }
    check_device_flag(*B.probs[i], B.main);
  }
  if (status == SPOCK_ERR_NUMERICAL) return fail(status, "non-finite residual in a batch instance");
  return status;
}

int fp64_fma_rate(int iters, double* tflops, cudaStream_t st);
template <typename S>
int launch_lambda(const KP<S>& p, const std::vector<int32_t>& stage_begin, const S* w, S* lam, int max_blocks,
                  cudaStream_t st);
void launch_cone_jac(const KP<double>& p, const double* wbar, const double* x, double* out, int grid,
                     cudaStream_t st);
void launch_axpy(int64_t n, double a, const double* x, const double* y, double* out, int grid, cudaStream_t st);
void launch_jt_residual(int64_t nz, int64_t ne, double alpha, const double* pz, const double* t, const double* q,
                        const double* Lp, const double* x, double* u, int grid, cudaStream_t st);
void launch_dots(int64_t n, const double* u, const double* V, int64_t ld, int k, const int* kdev, double* partials,
                 double* out, int grid, cudaStream_t st);
void launch_axpy_many(int64_t n, double* u, const double* V, int64_t ld, int k, const int* kdev, const double* h,
                      double sign, int grid, cudaStream_t st);
void launch_next_basis(int64_t n, const double* u, const double* norm2, int* kdev, double* V, int64_t ld,
                       double* vin, int grid, cudaStream_t st);
void launch_scale(int64_t n, double a, const double* u, double* v, int grid, cudaStream_t st);
void launch_true_residual(int64_t nz, int64_t ntot, const double* g, const double* u, const double* x, double* r,
                          unsigned long long* red, int grid, cudaStream_t st);
void launch_adj_gradients(const KP<double>& p, const double* z, const double* eta, const double* q,
                          const double* pv, const double* lam_mu, const double* negy, const double* lam_env,
                          const double* wenv, double* gx0, double* gA, double* gB, double* gQ, double* gR,
                          double* gQN, int grid, cudaStream_t st);

template <typename S>
int launch_gradient(const KP<S>& p, const std::vector<int32_t>& stage_begin, const S* z, const S* eta, const S* w,
                    S* lam, double* gx0, double* gA, double* gB, double* gQ, double* gR, double* gQN, int max_blocks,
                    cudaStream_t st);

template <typename S>
static int grad_impl(Problem& P, const double* z, const double* eta, double* gx0, double* gA, double* gB,
                     double* gQ, double* gR, double* gQN, cudaStream_t st) {
  if (P.general) return fail(SPOCK_ERR_UNSUPPORTED, "gradients: box constraints and diagonal costs only");
  Workspace* ws = get_ws_impl<S>(P, 0);
  const DevFactors<S>& f = factors<S>(P);
  const int64_t nz = P.off.n_z, ne = P.off.n_eta;
  const size_t n = (size_t)P.tree.n;
  S* zs = (S*)ws->v[0];
  S* es = zs + nz;
  S* w = (S*)ws->Tv[0];
  convert<S, double>(z, zs, nz, st);
  convert<S, double>(eta, es, ne, st);
  KP<S> kp = make_kp<S>(P, default_alpha(P, 0.0), P.idx.stage_begin);
  const int maxb = sm_count() * 16;
  launch_lstar<S>(kp, es, w, std::min((P.tree.n + 3) / 4, maxb), st);  // w = L* eta
  const int nx = P.nx, nu = P.nu;
  if (gA) CUDA_TRY(cudaMemsetAsync(gA, 0, sizeof(double) * n * nx * nx, st));
  if (gB) CUDA_TRY(cudaMemsetAsync(gB, 0, sizeof(double) * n * nx * nu, st));
  if (gQ) CUDA_TRY(cudaMemsetAsync(gQ, 0, sizeof(double) * n * nx, st));
  if (gR) CUDA_TRY(cudaMemsetAsync(gR, 0, sizeof(double) * n * nu, st));
  if (gQN) CUDA_TRY(cudaMemsetAsync(gQN, 0, sizeof(double) * n * nx, st));
  launch_gradient<S>(kp, P.tree.stage_begin, zs, es, w, f.q, gx0, gA, gB, gQ, gR, gQN, maxb, st);
  check_launch();
  CUDA_TRY(cudaStreamSynchronize(st));
  return SPOCK_OK;
}

// Adjoint of the CP fixed point (implicit differentiation of v* = T(v*)):
// w = J^T w + (g, 0) iterated from w = 0, J the Jacobian of T at the
// converged pair (z, eta); then the gradient of <g, z*> in x0, A, B and the
// diagonals of Q, R, Q_N (adjoint.cu).  One iteration: q = B w_eta (cone
// Jacobians), t = L* q, r = w_z + 2 alpha t, p = A r (the prox-of-f kernels
// with alpha = 0 and x0 = 0: the homogeneous Riccati pass and proj_S2),
// L p, then w = (p - alpha t + g, q - alpha L p).
static int adjoint_impl(Problem& P, const double* z, const double* eta, const double* gz, int max_iter, double tol,
                        double* gx0, double* gA, double* gB, double* gQ, double* gR, double* gQN,
                        int32_t* iters_out, double* res_out, cudaStream_t st) {
  if (P.general) return fail(SPOCK_ERR_UNSUPPORTED, "adjoint: box constraints and diagonal costs only");
  Workspace* ws = get_ws_impl<double>(P, 0);
  // the inputs were produced on the caller's stream; the solve runs on the
  // workspace's own stream (a CUDA graph cannot be captured on the legacy
  // default stream) and is synchronised before returning
  CUDA_TRY(cudaStreamSynchronize(st));
  st = ws->stream;
  const int64_t nz = P.off.n_z, ne = P.off.n_eta, ntot = nz + ne;
  const size_t n = (size_t)P.tree.n, nx = (size_t)P.nx, nu = (size_t)P.nu;
  const size_t xs = (size_t)P.f64.xs;
  // restarted GMRES(m): basis of m + 1 vectors, Hessenberg columns and dot
  // partials on the device.  m = 100, fewer when the basis would take more
  // than a quarter of the free device memory (at least 10); fixed at the
  // first call.
  const int gvec = sm_count() * 4;
  const size_t ldv = ((size_t)ntot + 31) / 32 * 32;
  if (!P.adj) {
    size_t fr = 0, tot = 0;
    CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    const size_t fit = fr / 4 / (ldv * sizeof(double));
    P.adj_restart = (int)std::max<size_t>(10, std::min<size_t>(100, fit > 1 ? fit - 1 : 1));
  }
  const int m = P.adj_restart;
  const size_t len = (size_t)ntot + 3 * (size_t)ne + 6 * (size_t)nz + 2 * n * xs + xs + 2 +
                     (size_t)(m + 1) * ldv + 3 * (size_t)ntot + (size_t)gvec * 128 + 3 * (size_t)(m + 1) + 8;
  if (!P.adj) {
    CUDA_TRY(cudaMalloc(&P.adj, sizeof(double) * len));
    P.allocations.push_back(P.adj);
  }
  const size_t nh = 2 * (size_t)(m + 1) + 1;   // Hessenberg column, second pass, norm
  if (!P.adj_pinned) CUDA_TRY(cudaMallocHost(&P.adj_pinned, sizeof(double) * nh));
  double* w = P.adj;
  double* wbar = w + ntot;
  double* q = wbar + ne;
  double* Lp = q + ne;
  double* t = Lp + ne;
  double* r = t + nz;
  double* pv = r + nz;
  double* g = pv + nz;
  double* negy = g + nz;
  double* wenv = negy + nz;
  double* lam_mu = wenv + nz;
  double* lam_env = lam_mu + n * xs;
  double* zero_x0 = lam_env + n * xs;
  unsigned long long* red = reinterpret_cast<unsigned long long*>(zero_x0 + xs);
  double* V = zero_x0 + xs + 2;        // basis, stride ldv
  double* u = V + (size_t)(m + 1) * ldv;
  double* res = u + ntot;              // true residual b - (I - J^T) w
  double* part = res + ntot;           // dot partials [gvec][128]
  // [m + 1] Hessenberg column, [m + 1] its second Gram-Schmidt pass, [1] norm;
  // then [m + 1] the solution of the small least-squares problem
  double* hdev = part + (size_t)gvec * 128;
  double* hdev2 = hdev + (m + 1);
  double* hnorm = hdev2 + (m + 1);
  double* ydev = hnorm + 1;
  double* vin = ydev + (m + 1) + 1;    // the current basis vector (input of the captured step)
  int* kdev = reinterpret_cast<int*>(ydev + (m + 1));   // basis index of the captured step
  const double alpha = default_alpha(P, 0.0);
  KP<double> kp = make_kp<double>(P, alpha, P.idx.stage_begin);
  KP<double> kA = kp;   // Jacobian of prox_{alpha f}: no shift of s^0, x0 = 0
  kA.alpha = 0.0;
  kA.inv_alpha = 0.0;
  kA.x0 = zero_x0;
  const int maxb = sm_count() * 16;
  const int gnode = std::min((P.tree.n + 3) / 4, maxb);
  CUDA_TRY(cudaMemsetAsync(zero_x0, 0, sizeof(double) * xs, st));
  // wbar = eta + alpha L z (the point of prox_{alpha g*} at the fixed point)
  launch_dual<double>(kp, DM_APPLY_L_, false, z, nullptr, nullptr, Lp, nullptr, nullptr, gnode, st);
  launch_axpy(ne, alpha, Lp, eta, wbar, gvec, st);
  if (gz) {
    CUDA_TRY(cudaMemcpyAsync(g, gz, sizeof(double) * nz, cudaMemcpyDeviceToDevice, st));
  } else {
    const double one = 1.0;
    CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(double) * nz, st));
    CUDA_TRY(cudaMemcpyAsync(g, &one, sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));   // the host value `one` goes out of scope
  }
  CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(double) * ntot, st));
  const double* zero_eta = (const double*)ws->zero_eta;
  auto jt_parts = [&](const double* x) {   // q, t, r, p, L p of J^T x
    launch_cone_jac(kp, wbar, x + nz, q, gnode, st);
    launch_lstar<double>(kp, q, t, gnode, st);
    launch_axpy(nz, 2.0 * alpha, t, x, r, gvec, st);
    launch_prep<double>(kA, r, zero_eta, pv, maxb, st);
    launch_riccati<double>(kA, P.tree.stage_begin, P.tree.stage_maxch, pv, st, nullptr);
    launch_dual<double>(kp, DM_APPLY_L_, false, pv, nullptr, nullptr, Lp, nullptr, nullptr, gnode, st);
  };
  auto apply_op = [&](const double* x, double* out) {   // out = (I - J^T) x
    jt_parts(x);
    launch_jt_residual(nz, ne, alpha, pv, t, q, Lp, x, out, gvec, st);
  };
  auto dots = [&](const double* a, int k, double* out_dev, std::vector<double>& out_host) {
    launch_dots(ntot, a, V, (int64_t)ldv, k, nullptr, part, out_dev, gvec, st);
    out_host.resize(k);
    CUDA_TRY(cudaMemcpyAsync(out_host.data(), out_dev, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  };
  // true residual res = b - (I - J^T) w and its max norm against max |w|
  double rinf = INFINITY, winf = 0.0;
  auto true_residual = [&]() {
    apply_op(w, u);
    CUDA_TRY(cudaMemsetAsync(red, 0, 2 * sizeof(unsigned long long), st));
    launch_true_residual(nz, ntot, g, u, w, res, red, gvec, st);
    unsigned long long h[2];
    CUDA_TRY(cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    std::memcpy(&rinf, &h[0], sizeof(double));
    std::memcpy(&winf, &h[1], sizeof(double));
    if (!std::isfinite(rinf)) throw SpockError(SPOCK_ERR_NUMERICAL, "the adjoint solve diverged");
  };
  int it = 0;   // applications of J^T inside the Arnoldi steps
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gam(m + 1), hv, y(m);
  const double* hh = P.adj_pinned;
  // one Arnoldi step, captured once and replayed: u = (I - J^T) vin; two
  // classical Gram-Schmidt passes against V_0 .. V_k (k = *kdev); ||u||^2;
  // the coefficients copied to pinned host memory; V_{k+1} = vin = u / ||u||
  cudaGraphExec_t step = nullptr;
  {
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    apply_op(vin, u);
    launch_dots(ntot, u, V, (int64_t)ldv, 1, kdev, part, hdev, gvec, st);
    launch_axpy_many(ntot, u, V, (int64_t)ldv, 1, kdev, hdev, -1.0, gvec, st);
    launch_dots(ntot, u, V, (int64_t)ldv, 1, kdev, part, hdev2, gvec, st);
    launch_axpy_many(ntot, u, V, (int64_t)ldv, 1, kdev, hdev2, -1.0, gvec, st);
    launch_dots(ntot, u, u, 0, 1, nullptr, part, hnorm, gvec, st);   // ||u||^2 (V stride 0: u itself)
    cudaMemcpyAsync(P.adj_pinned, hdev, sizeof(double) * nh, cudaMemcpyDeviceToHost, st);
    launch_next_basis(ntot, u, hnorm, kdev, V, (int64_t)ldv, vin, gvec, st);
    CUDA_TRY(cudaStreamEndCapture(st, &g));
    const cudaError_t e = cudaGraphInstantiate(&step, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e);
  }
  struct StepGuard {
    cudaGraphExec_t& s;
    ~StepGuard() {
      if (s) cudaGraphExecDestroy(s);
    }
  } step_guard{step};
  true_residual();
  while (!(rinf <= tol * std::max(1.0, winf)) && it < max_iter) {
    // v_0 = res / ||res||
    CUDA_TRY(cudaMemcpyAsync(V, res, sizeof(double) * ntot, cudaMemcpyDeviceToDevice, st));
    dots(res, 1, hdev, hv);
    const double beta = std::sqrt(std::max(hv[0], 0.0));
    if (!(beta > 0.0)) break;
    launch_scale(ntot, 1.0 / beta, res, V, gvec, st);
    CUDA_TRY(cudaMemcpyAsync(vin, V, sizeof(double) * ntot, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemsetAsync(kdev, 0, sizeof(int), st));
    std::fill(gam.begin(), gam.end(), 0.0);
    gam[0] = beta;
    const double thr = tol * std::max(1.0, winf);
    int k = 0;
    for (; k < m && it < max_iter; ++k) {
      CUDA_TRY(cudaGraphLaunch(step, st));
      CUDA_TRY(cudaStreamSynchronize(st));
      ++it;
      const double hn = std::sqrt(std::max(hh[2 * (size_t)(m + 1)], 0.0));
      for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = hh[i] + hh[(size_t)(m + 1) + i];
      H[(size_t)(k + 1) * m + k] = hn;
      // Givens rotations on the new column
      for (int i = 0; i < k; ++i) {
        const double a = H[(size_t)i * m + k], b = H[(size_t)(i + 1) * m + k];
        H[(size_t)i * m + k] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[(size_t)k * m + k], b = H[(size_t)(k + 1) * m + k];
      const double rr = std::hypot(a, b);
      cs[k] = rr > 0.0 ? a / rr : 1.0;
      sn[k] = rr > 0.0 ? b / rr : 0.0;
      H[(size_t)k * m + k] = rr;
      H[(size_t)(k + 1) * m + k] = 0.0;
      gam[k + 1] = -sn[k] * gam[k];
      gam[k] = cs[k] * gam[k];
      if (std::fabs(gam[k + 1]) <= thr || !(hn > 0.0)) {
        ++k;
        break;
      }
    }
    // w += V y, H(0:k, 0:k) y = gam(0:k)
    for (int i = k - 1; i >= 0; --i) {
      double sum = gam[i];
      for (int c = i + 1; c < k; ++c) sum -= H[(size_t)i * m + c] * y[c];
      y[i] = H[(size_t)i * m + i] != 0.0 ? sum / H[(size_t)i * m + i] : 0.0;
    }
    CUDA_TRY(cudaMemcpyAsync(ydev, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
    launch_axpy_many(ntot, w, V, (int64_t)ldv, k, nullptr, ydev, 1.0, gvec, st);
    CUDA_TRY(cudaStreamSynchronize(st));   // y is a host buffer
    true_residual();
  }
  const double diff = rinf, mag = winf;
  // data derivatives from the final w
  jt_parts(w);
  launch_axpy(nz, -1.0, r, pv, negy, gvec, st);                    // negy = p - r
  launch_lambda<double>(kp, P.tree.stage_begin, negy, lam_mu, maxb, st);
  launch_lstar<double>(kp, eta, wenv, gnode, st);                  // wenv = L* eta
  launch_lambda<double>(kp, P.tree.stage_begin, wenv, lam_env, maxb, st);
  if (gA) CUDA_TRY(cudaMemsetAsync(gA, 0, sizeof(double) * n * nx * nx, st));
  if (gB) CUDA_TRY(cudaMemsetAsync(gB, 0, sizeof(double) * n * nx * nu, st));
  if (gQ) CUDA_TRY(cudaMemsetAsync(gQ, 0, sizeof(double) * n * nx, st));
  if (gR) CUDA_TRY(cudaMemsetAsync(gR, 0, sizeof(double) * n * nu, st));
  if (gQN) CUDA_TRY(cudaMemsetAsync(gQN, 0, sizeof(double) * n * nx, st));
  launch_adj_gradients(kp, z, eta, q, pv, lam_mu, negy, lam_env, wenv, gx0, gA, gB, gQ, gR, gQN, gnode, st);
  check_launch();
  CUDA_TRY(cudaStreamSynchronize(st));
  check_device_flag(P, st);
  if (iters_out) *iters_out = it;
  if (res_out) *res_out = diff / std::max(1.0, mag);
  return diff <= tol * std::max(1.0, mag) ? SPOCK_OK : SPOCK_MAX_ITER;
}

// ---------------------------------------------------------------------------
// problem creation
// ---------------------------------------------------------------------------
template <typename T>
static T* upload(Problem& P, const std::vector<T>& h) {
  void* p = nullptr;
  CUDA_TRY(cudaMalloc(&p, sizeof(T) * std::max<size_t>(h.size(), 1)));
  P.allocations.push_back(p);
  if (!h.empty()) CUDA_TRY(cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return (T*)p;
}
template <typename S>
static S* dalloc(Problem& P, size_t n) {
  void* p = nullptr;
  CUDA_TRY(cudaMalloc(&p, sizeof(S) * std::max<size_t>(n, 1)));
  P.allocations.push_back(p);
  return (S*)p;
}

static int32_t pad16(int64_t elems, size_t elt) {
  const int64_t a = (int64_t)(16 / elt);
  return (int32_t)((elems + a - 1) / a * a);
}

template <typename S>
static void upload_factors(Problem& P, DevFactors<S>& f, const std::vector<double>& Gb,
                           const std::vector<double>& Gf, const std::vector<double>& NB,
                           const std::vector<double>& Kt, const std::vector<std::vector<double>>& par,
                           const GenHost* gen) {
  auto cast = [](const std::vector<double>& v) {
    std::vector<S> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (S)v[i];
    return o;
  };
  // blocks of `len` entries re-laid out with a padded stride
  auto padded = [](const std::vector<double>& v, size_t len, size_t stride) {
    const size_t cnt = len ? v.size() / len : 0;
    std::vector<S> o(cnt * stride, S(0));
    for (size_t b = 0; b < cnt; ++b)
      for (size_t i = 0; i < len; ++i) o[b * stride + i] = (S)v[b * len + i];
    return o;
  };
  const int nx = P.nx, nu = P.nu, ncol = nx + nu;
  f.xs = pad16(nx, sizeof(S));
  f.us = pad16(nu, sizeof(S));
  f.gstride = pad16((int64_t)nx * ncol, sizeof(S));
  f.nbstride = pad16(2 * (int64_t)nu * nx + (int64_t)nu * nu, sizeof(S));
  f.ktstride = pad16((int64_t)nx * nu, sizeof(S));
  f.Gb = upload(P, padded(Gb, (size_t)nx * ncol, f.gstride));
  f.Gf = upload(P, padded(Gf, (size_t)nx * ncol, f.gstride));
  f.NB = upload(P, padded(NB, 2 * (size_t)nu * nx + (size_t)nu * nu, f.nbstride));
  f.Kt = upload(P, padded(Kt, (size_t)nx * nu, f.ktstride));
  f.qs = upload(P, cast(par[0]));
  f.rs = upload(P, cast(par[1]));
  f.qns = upload(P, cast(par[2]));
  f.xlo = upload(P, cast(par[3]));
  f.xhi = upload(P, cast(par[4]));
  f.ulo = upload(P, cast(par[5]));
  f.uhi = upload(P, cast(par[6]));
  f.av = upload(P, cast(par[7]));
  f.prob = upload(P, cast(par[8]));
  const Tree& t = P.tree;
  {  // reciprocals of the Sherman-Morrison closed form of proj_S2 (one pair per node)
    std::vector<S> inv(2 * (size_t)t.n, S(0));
    for (int32_t k = 0; k < t.n_nonleaf; ++k) {
      const double a = par[7][k], c = a * a + 3.0;
      inv[2 * (size_t)k] = (S)(1.0 / c);
      inv[2 * (size_t)k + 1] = (S)(1.0 / (c + t.ch_count[k]));
    }
    f.s2inv = upload(P, inv);
  }
  if (gen) {
    f.gc = upload(P, cast(gen->gc));
    f.gt = upload(P, cast(gen->gt));
    f.fqc = upload(P, cast(gen->fqc));
    f.fqt = upload(P, cast(gen->fqt));
    f.frc = upload(P, cast(gen->frc));
    f.frt = upload(P, cast(gen->frt));
    f.fnc = upload(P, cast(gen->fnc));
    f.fnt = upload(P, cast(gen->fnt));
    f.gnc = upload(P, cast(gen->gnc));
    f.gnt = upload(P, cast(gen->gnt));
    // infinite bounds stay infinite in FP32 as well
    f.clo = upload(P, cast(gen->clo));
    f.chi = upload(P, cast(gen->chi));
    f.rb = upload(P, cast(gen->rb));
    f.rpi = upload(P, cast(gen->rpi));
  }
  f.xbar = dalloc<S>(P, (size_t)t.n * f.xs);
  f.ubar = dalloc<S>(P, (size_t)t.n_nonleaf * f.us);
  f.q = dalloc<S>(P, (size_t)t.n * f.xs);
  f.d = dalloc<S>(P, (size_t)t.n_nonleaf * f.us);
  f.x0 = dalloc<S>(P, (size_t)P.nx);
}

static bool all_finite(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

static int noalloc_scratch(int dev, double** out);

// General-form inputs of problem_create (user numbering; see
// spock_problem_create_general).
struct GenInput {
  bool dense = false;
  const spock_risk* risk = nullptr;   // nullptr: AV@R with parameter a
  int32_t nc = 0, ncN = 0;
  const double *Gx = nullptr, *Gu = nullptr, *cmin = nullptr, *cmax = nullptr;
  const double *GN = nullptr, *cNmin = nullptr, *cNmax = nullptr;
};

// Box form (gi == nullptr): diagonal Q, R, QN and boxes xmin..umax.  General
// form (gi != nullptr): Q, R, QN dense or diagonal as gi->dense says, the
// constraint rows of gi; xmin..umax are not read.
static int problem_create(const Tree& tree, int32_t nx, int32_t nu, const double* A, const double* B,
                          const double* Q, const double* R, const double* QN, const double* a, const double* xmin,
                          const double* xmax, const double* umin, const double* umax, const GenInput* gi,
                          spock_problem** out) {
  if (!A || !B || !Q || !R || !QN || (!a && !(gi && gi->risk)) || !out)
    return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
  if (!gi && (!xmin || !xmax || !umin || !umax)) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
  if (gi && (!gi->Gx || !gi->Gu || !gi->cmin || !gi->cmax || !gi->GN || !gi->cNmin || !gi->cNmax))
    return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
  if (nx < 1 || nu < 1 || nx + nu > kMaxDim)
    return fail(SPOCK_ERR_INVALID_ARG, "need nx >= 1, nu >= 1, nx + nu <= 128");
  if (gi && (gi->nc < 1 || gi->nc > kMaxDim || gi->ncN < 1 || gi->ncN > kMaxDim))
    return fail(SPOCK_ERR_INVALID_ARG, "need 1 <= nc, ncN <= 128");
  const int32_t n = tree.n;
  const size_t nn = (size_t)n;
  // validation (user numbering)
  if (!all_finite(A + (size_t)nx * nx, (nn - 1) * nx * nx) || !all_finite(B + (size_t)nx * nu, (nn - 1) * nx * nu))
    return fail(SPOCK_ERR_NUMERICAL, "non-finite dynamics");
  if (gi) {
    const size_t qsz = gi->dense ? (size_t)nx * nx : (size_t)nx, rsz = gi->dense ? (size_t)nu * nu : (size_t)nu;
    if (!all_finite(Q, nn * qsz) || !all_finite(R, nn * rsz) || !all_finite(QN, nn * qsz) ||
        !all_finite(gi->Gx, nn * gi->nc * nx) || !all_finite(gi->Gu, nn * gi->nc * nu) ||
        !all_finite(gi->GN, nn * gi->ncN * nx))
      return fail(SPOCK_ERR_NUMERICAL, "non-finite cost or constraint matrices");
    for (int32_t u = 0; u < n && !gi->risk; ++u)
      if (tree.int_of[u] < tree.n_nonleaf && !(a[u] >= 0.0 && a[u] <= 1.0))
        return fail(SPOCK_ERR_INVALID_ARG, "AV@R parameter must be in [0, 1]");
  }
  for (int32_t u = 0; u < n && !gi; ++u) {
    const int32_t k = tree.int_of[u];
    const bool nonroot = k > 0, leaf = k >= tree.n_nonleaf, nonleaf = !leaf;
    for (int r = 0; r < nx; ++r) {
      if (nonroot && !(Q[(size_t)u * nx + r] > 0.0 && std::isfinite(Q[(size_t)u * nx + r])))
        return fail(SPOCK_ERR_NOT_POSDEF, "Q must be positive and finite");
      if (leaf && !(QN[(size_t)u * nx + r] > 0.0 && std::isfinite(QN[(size_t)u * nx + r])))
        return fail(SPOCK_ERR_NOT_POSDEF, "QN must be positive and finite");
      const double lo = xmin[(size_t)u * nx + r], hi = xmax[(size_t)u * nx + r];
      if (std::isnan(lo) || std::isnan(hi) || lo > hi) return fail(SPOCK_ERR_INVALID_ARG, "xmin > xmax");
    }
    for (int r = 0; r < nu; ++r) {
      if (nonroot && !(R[(size_t)u * nu + r] > 0.0 && std::isfinite(R[(size_t)u * nu + r])))
        return fail(SPOCK_ERR_NOT_POSDEF, "R must be positive and finite");
      if (nonleaf) {
        const double lo = umin[(size_t)u * nu + r], hi = umax[(size_t)u * nu + r];
        if (std::isnan(lo) || std::isnan(hi) || lo > hi) return fail(SPOCK_ERR_INVALID_ARG, "umin > umax");
      }
    }
    if (nonleaf && !(a[u] >= 0.0 && a[u] <= 1.0)) return fail(SPOCK_ERR_INVALID_ARG, "AV@R parameter must be in [0, 1]");
  }
  auto* P = new Problem();
  try {
    CUDA_TRY(cudaGetDevice(&P->device));
    P->tree = tree;
    P->nx = nx;
    P->nu = nu;
    const Tree& t = P->tree;
    const int nl = t.n_nonleaf, ncol = nx + nu;
    int threads = (int)std::thread::hardware_concurrency();
    if (threads <= 0) threads = 4;
    GenHost gh;
    if (gi) {
      std::string err;
      const int rc = build_general(t, nx, nu, gi->dense, Q, R, QN, a, gi->risk, gi->nc, gi->Gx, gi->Gu, gi->cmin,
                                   gi->cmax, gi->ncN, gi->GN, gi->cNmin, gi->cNmax, threads, gh, err);
      if (rc != SPOCK_OK) {
        delete P;
        return fail(rc, err);
      }
      P->general = true;
      P->gd = gh.d;
      build_offsets(P->tree, nx, nu, gi->nc, gi->ncN, &gh.ny_user, P->off);
    } else {
      P->gd.nc = nx + nu;
      P->gd.ncN = nx;
      build_offsets(P->tree, nx, nu, nx + nu, nx, nullptr, P->off);
    }
    // internal-order dynamics
    std::vector<double> Ai(nn * nx * nx), Bi(nn * nx * nu);
    for (int32_t k = 1; k < n; ++k) {
      const int32_t u = t.user_of[k];
      std::memcpy(&Ai[(size_t)k * nx * nx], A + (size_t)u * nx * nx, sizeof(double) * nx * nx);
      std::memcpy(&Bi[(size_t)k * nx * nu], B + (size_t)u * nx * nu, sizeof(double) * nx * nu);
    }
    std::vector<double> Gb, NB;
    const auto t0 = std::chrono::steady_clock::now();
    if (!riccati_factor(t, nx, nu, Ai, Bi, Gb, NB, threads)) {
      delete P;
      return fail(SPOCK_ERR_NUMERICAL, "Cholesky of I + sum B'PB failed");
    }
    P->factor_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!all_finite(Gb.data(), Gb.size()) || !all_finite(NB.data(), NB.size())) {
      delete P;
      return fail(SPOCK_ERR_NUMERICAL, "non-finite Riccati factors");
    }
    // forward layouts: transpose of [Abar | B], and K^T
    std::vector<double> Gf(Gb.size()), Kt((size_t)nl * nx * nu);
    const size_t gsz = (size_t)nx * ncol, nbsz = 2 * (size_t)nu * nx + (size_t)nu * nu;
    for (int32_t c = 1; c < n; ++c) {
      const double* g = &Gb[(size_t)(c - 1) * gsz];
      double* h = &Gf[(size_t)(c - 1) * gsz];
      for (int r = 0; r < nx; ++r)
        for (int j = 0; j < ncol; ++j) h[(size_t)j * nx + r] = g[(size_t)r * ncol + j];
    }
    for (int32_t k = 0; k < nl; ++k)
      for (int r = 0; r < nu; ++r)
        for (int q = 0; q < nx; ++q) Kt[(size_t)k * nx * nu + (size_t)q * nu + r] = NB[(size_t)k * nbsz + (size_t)r * nx + q];
    // node parameters (internal order)
    std::vector<std::vector<double>> par(9);
    par[0].assign(nn * nx, 0.0);
    par[1].assign(nn * nu, 0.0);
    par[2].assign(nn * nx, 0.0);
    par[3].assign(nn * nx, 0.0);
    par[4].assign(nn * nx, 0.0);
    par[5].assign(nn * nu, 0.0);
    par[6].assign(nn * nu, 0.0);
    par[7].assign(nn, 0.0);
    par[8].assign(nn, 1.0);
    for (int32_t k = 0; k < n; ++k) {
      const int32_t u = t.user_of[k];
      if (gi) {   // general form: the box-form arrays stay zero
        if (k < nl && a) par[7][k] = a[u];
        par[8][k] = t.prob[k];
        continue;
      }
      for (int r = 0; r < nx; ++r) {
        if (k > 0) par[0][(size_t)k * nx + r] = std::sqrt(Q[(size_t)u * nx + r]);
        if (k >= nl) par[2][(size_t)k * nx + r] = std::sqrt(QN[(size_t)u * nx + r]);
        par[3][(size_t)k * nx + r] = xmin[(size_t)u * nx + r];
        par[4][(size_t)k * nx + r] = xmax[(size_t)u * nx + r];
      }
      for (int r = 0; r < nu; ++r) {
        if (k > 0) par[1][(size_t)k * nu + r] = std::sqrt(R[(size_t)u * nu + r]);
        if (k < nl) {
          par[5][(size_t)k * nu + r] = umin[(size_t)u * nu + r];
          par[6][(size_t)k * nu + r] = umax[(size_t)u * nu + r];
        }
      }
      if (k < nl) par[7][k] = a[u];
      par[8][k] = t.prob[k];
    }
    // ||L||^2 as the largest block norm (remark after the definition of L)
    double best = std::max(0.5, std::max(gh.normL2_xu, gh.normL2_ys));
    for (int32_t k = 0; k < nl && !gi; ++k) {
      const int c0 = t.ch_begin[k], m = t.ch_count[k];
      for (int r = 0; r < nx && !gi; ++r) {
        double s = 1.0;
        for (int j = 0; j < m; ++j) s += par[0][(size_t)(c0 + j) * nx + r] * par[0][(size_t)(c0 + j) * nx + r];
        best = std::max(best, s);
      }
      for (int r = 0; r < nu && !gi; ++r) {
        double s = 1.0;
        for (int j = 0; j < m; ++j) s += par[1][(size_t)(c0 + j) * nu + r] * par[1][(size_t)(c0 + j) * nu + r];
        best = std::max(best, s);
      }
      double b2 = 1.0;
      for (int j = 0; j < m; ++j) b2 += t.prob[c0 + j] * t.prob[c0 + j];
      const double bb = std::sqrt(b2);
      best = std::max(best, (2.0 + b2 + bb * std::sqrt(b2 + 4.0)) / 2.0);
    }
    for (int32_t k = nl; k < n && !gi; ++k)
      for (int r = 0; r < nx; ++r) best = std::max(best, 1.0 + par[2][(size_t)k * nx + r] * par[2][(size_t)k * nx + r]);
    P->normL = std::sqrt(best);
    // device index
    P->idx.parent = upload(*P, t.parent);
    P->idx.ch_begin = upload(*P, t.ch_begin);
    P->idx.ch_count = upload(*P, t.ch_count);
    P->idx.sib = upload(*P, t.sib);
    P->idx.zx = upload(*P, P->off.zx);
    P->idx.zu = upload(*P, P->off.zu);
    P->idx.zz2 = upload(*P, P->off.zz2);
    P->idx.zs = upload(*P, P->off.zs);
    P->idx.ztau = upload(*P, P->off.ztau);
    P->idx.enl = upload(*P, P->off.enl);
    P->idx.enr = upload(*P, P->off.enr);
    P->idx.elf = upload(*P, P->off.elf);
    upload_factors<double>(*P, P->f64, Gb, Gf, NB, Kt, par, gi ? &gh : nullptr);
    upload_factors<float>(*P, P->f32, Gb, Gf, NB, Kt, par, gi ? &gh : nullptr);
    if (gi) {
      P->idx.rny = upload(*P, gh.rny);
      P->idx.rkp = upload(*P, gh.rkp);
      P->idx.rboff = upload(*P, gh.rboff);
      P->idx.rpoff = upload(*P, gh.rpoff);
    }
    P->idx.stage_begin = upload(*P, t.stage_begin);
    {
      std::vector<NodeDesc> dh(nn);
      const Offsets& o = P->off;
      for (int32_t k = 0; k < n; ++k) {
        NodeDesc& q = dh[k];
        std::memset(&q, 0, sizeof(q));
        q.zx = o.zx[k];
        q.zu = o.zu[k];
        q.zz2 = o.zz2[k];
        q.zs = o.zs[k];
        q.ztau = o.ztau[k];
        q.enl = o.enl[k];
        q.enr = o.enr[k];
        q.elf = o.elf[k];
        q.par = t.parent[k];
        q.m = t.ch_count[k];
        q.c0 = t.ch_begin[k];
        q.user = t.user_of[k];
        q.zxp = k > 0 ? o.zx[t.parent[k]] : -1;
        q.zup = k > 0 ? o.zu[t.parent[k]] : -1;
        q.es = k < nl ? o.enl[k] + (gi ? gh.rny[k] : 2 * t.ch_count[k] + 1) : o.elf[k] + P->gd.ncN + nx;
      }
      for (int32_t k = 0; k < n; ++k) {
        dh[k].enr_c0 = t.ch_count[k] > 0 ? dh[t.ch_begin[k]].enr : -1;
        dh[k].es_c0 = t.ch_count[k] > 0 ? dh[t.ch_begin[k]].es : -1;
      }
      P->idx.desc = upload(*P, dh);
    }
    P->err = upload(*P, std::vector<int32_t>(1, 0));
    CUDA_TRY(cudaDeviceSynchronize());
    // device address of the fixed scratch array of spock_prox_f_noalloc_dev,
    // looked up here (where allocating is allowed) so that the lookup, and
    // any module loading it triggers, never happens inside that entry point
    double* scratch = nullptr;
    const int rc = noalloc_scratch(P->device, &scratch);
    if (rc != SPOCK_OK) {
      delete P;
      return rc;
    }
  } catch (const SpockError& e) {
    delete P;
    return fail(e.code, e.what());
  }
  *out = reinterpret_cast<spock_problem*>(P);
  return SPOCK_OK;
}

}  // namespace spock

// ===========================================================================
// C ABI
// ===========================================================================
using namespace spock;

static Problem* as_problem(void* h) {
  Problem* p = reinterpret_cast<Problem*>(h);
  return (p && p->tag == TAG_PROBLEM) ? p : nullptr;
}
static const Tree* as_tree(const void* h) {
  const Tree* t = reinterpret_cast<const Tree*>(h);
  return (t && t->tag == TAG_TREE) ? t : nullptr;
}

extern "C" {

int spock_default_settings(spock_settings* s) {
  if (!s) return fail(SPOCK_ERR_INVALID_ARG, "settings is NULL");
  s->eps_abs = 1e-6;
  s->eps_rel = 1e-6;
  s->alpha = 0.0;
  s->memory = 3;
  s->c0 = s->c1 = s->c2 = 0.99;
  s->beta = 0.5;
  s->sigma = 0.1;
  s->lambda = 1.0;
  s->rho_coef = 1.0;
  s->max_iter = 100000;
  s->max_backtracks = 30;
  s->precision = SPOCK_FP64;
  s->trace = nullptr;
  s->profile = 0;
  s->fp64_tail = 1;
  s->stall_window = 2000;   // near the tolerance the FP32 iteration can take ~500 iterations to halve xi
  return SPOCK_OK;
}

int spock_tree_create(int32_t n_nodes, const int32_t* anc, const double* prob, spock_tree** out) {
  return guarded([&]() -> int {
    if (!out) return fail(SPOCK_ERR_INVALID_ARG, "out is NULL");
    auto* t = new Tree();
    int rc = build_tree(n_nodes, anc, prob, *t);
    if (rc != SPOCK_OK) {
      delete t;
      return rc;
    }
    *out = reinterpret_cast<spock_tree*>(t);
    return SPOCK_OK;
  });
}

int spock_tree_create_abs(int32_t n_nodes, const int32_t* anc, const double* pi, spock_tree** out) {
  return guarded([&]() -> int {
    if (!out || !anc || !pi) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    if (n_nodes < 2) return fail(SPOCK_ERR_INVALID_ARG, "tree needs at least 2 nodes");
    if (anc[0] != -1) return fail(SPOCK_ERR_BAD_TREE, "anc[0] must be -1 (node 0 is the root)");
    std::vector<double> p((size_t)n_nodes, 1.0);
    for (int32_t i = 0; i < n_nodes; ++i)
      if (!(pi[i] > 0.0) || !std::isfinite(pi[i]))
        return fail(SPOCK_ERR_INVALID_ARG, "absolute probabilities must be positive and finite");
    for (int32_t i = 1; i < n_nodes; ++i) {
      if (anc[i] < 0 || anc[i] >= n_nodes || anc[i] == i)
        return fail(SPOCK_ERR_BAD_TREE, "anc[" + std::to_string(i) + "] out of range");
      p[(size_t)i] = pi[i] / pi[anc[i]];   // p^i = pi^i / pi^anc(i)
    }
    auto* t = new Tree();
    int rc = build_tree(n_nodes, anc, p.data(), *t);
    if (rc != SPOCK_OK) {
      delete t;
      return rc;
    }
    *out = reinterpret_cast<spock_tree*>(t);
    return SPOCK_OK;
  });
}

int spock_tree_info(const spock_tree* tree, int32_t* n_nodes, int32_t* horizon, int32_t* n_nonleaf) {
  const Tree* t = as_tree(tree);
  if (!t) return fail(SPOCK_ERR_INVALID_ARG, "not a tree handle");
  if (n_nodes) *n_nodes = t->n;
  if (horizon) *horizon = t->N;
  if (n_nonleaf) *n_nonleaf = t->n_nonleaf;
  return SPOCK_OK;
}

int spock_problem_create(const spock_tree* tree, int32_t nx, int32_t nu, const double* A, const double* B,
                         const double* Q, const double* R, const double* QN, const double* a, const double* xmin,
                         const double* xmax, const double* umin, const double* umax, int32_t flags,
                         spock_problem** out) {
  return guarded([&]() -> int {
    const Tree* t = as_tree(tree);
    if (!t) return fail(SPOCK_ERR_INVALID_ARG, "not a tree handle");
    if (flags & ~SPOCK_DENSE_COST) return fail(SPOCK_ERR_UNSUPPORTED, "unknown flag");
    if (!(flags & SPOCK_DENSE_COST))
      return problem_create(*t, nx, nu, A, B, Q, R, QN, a, xmin, xmax, umin, umax, nullptr, out);
    // dense costs with the box constraints: the general form with Gamma = I
    if (!xmin || !xmax || !umin || !umax) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    if (nx < 1 || nu < 1 || nx + nu > kMaxDim)
      return fail(SPOCK_ERR_INVALID_ARG, "need nx >= 1, nu >= 1, nx + nu <= 128");
    const size_t n = (size_t)t->n, nc = (size_t)nx + nu;
    std::vector<double> Gx(n * nc * nx, 0.0), Gu(n * nc * nu, 0.0), cmin(n * nc), cmax(n * nc);
    std::vector<double> GN(n * nx * nx, 0.0);
    for (size_t u = 0; u < n; ++u) {
      for (int r = 0; r < nx; ++r) {
        Gx[(u * nc + r) * nx + r] = 1.0;
        GN[(u * nx + r) * nx + r] = 1.0;
        cmin[u * nc + r] = xmin[u * nx + r];
        cmax[u * nc + r] = xmax[u * nx + r];
      }
      for (int r = 0; r < nu; ++r) {
        Gu[(u * nc + nx + r) * nu + r] = 1.0;
        cmin[u * nc + nx + r] = umin[u * nu + r];
        cmax[u * nc + nx + r] = umax[u * nu + r];
      }
    }
    GenInput gi;
    gi.dense = true;
    gi.risk = nullptr;
    gi.nc = (int32_t)nc;
    gi.ncN = nx;
    gi.Gx = Gx.data();
    gi.Gu = Gu.data();
    gi.cmin = cmin.data();
    gi.cmax = cmax.data();
    gi.GN = GN.data();
    gi.cNmin = xmin;
    gi.cNmax = xmax;
    return problem_create(*t, nx, nu, A, B, Q, R, QN, a, nullptr, nullptr, nullptr, nullptr, &gi, out);
  });
}

int spock_problem_create_general(const spock_tree* tree, int32_t nx, int32_t nu, const double* A,
                                 const double* B, const double* Q, const double* R, const double* QN,
                                 const double* a, const spock_risk* risk, int32_t nc, const double* Gx,
                                 const double* Gu, const double* cmin, const double* cmax, int32_t ncN,
                                 const double* GN, const double* cNmin, const double* cNmax, int32_t flags,
                                 spock_problem** out) {
  return guarded([&]() -> int {
    const Tree* t = as_tree(tree);
    if (!t) return fail(SPOCK_ERR_INVALID_ARG, "not a tree handle");
    if (flags & ~SPOCK_DENSE_COST) return fail(SPOCK_ERR_UNSUPPORTED, "unknown flag");
    GenInput gi;
    gi.dense = (flags & SPOCK_DENSE_COST) != 0;
    gi.risk = risk;
    gi.nc = nc;
    gi.ncN = ncN;
    gi.Gx = Gx;
    gi.Gu = Gu;
    gi.cmin = cmin;
    gi.cmax = cmax;
    gi.GN = GN;
    gi.cNmin = cNmin;
    gi.cNmax = cNmax;
    return problem_create(*t, nx, nu, A, B, Q, R, QN, a, nullptr, nullptr, nullptr, nullptr, &gi, out);
  });
}

int spock_problem_info(const spock_problem* p, int64_t* n_z, int64_t* n_eta, double* norm_L, double* factor_seconds) {
  Problem* P = as_problem((void*)p);
  if (!P) return fail(SPOCK_ERR_INVALID_ARG, "not a problem handle");
  if (n_z) *n_z = P->off.n_z;
  if (n_eta) *n_eta = P->off.n_eta;
  if (norm_L) *norm_L = P->normL;
  if (factor_seconds) *factor_seconds = P->factor_seconds;
  return SPOCK_OK;
}

// FP32 iteration with FP64 certification and FP64 tail: the FP32 run stops
// at its tolerance, its iteration cap, or stagnation; its result T32(v) (in
// the FP64 output buffers) warm-starts an FP64 run with the same tolerance
// (from the FP32 run's xi_0), whose first evaluation of T is the FP64
// certificate -- zero FP64 iterations when the FP32 result already meets it.
static int solve_mixed(Problem& P, const double* x0_dev, const spock_settings& s, double* z_dev, double* eta_dev,
                       int warm, spock_info* info, cudaStream_t st) {
  spock_info i32{};
  int act32 = A_NONE;
  int rc = solve_impl<float>(P, x0_dev, s, z_dev, eta_dev, warm, &i32, st, 0.0, s.fp64_tail ? s.stall_window : 0,
                             &act32);
  if (rc < 0 || !s.fp64_tail) {
    if (info) *info = i32;
    return rc;
  }
  spock_settings s64 = s;
  s64.max_iter = std::max(0, s.max_iter - i32.iterations);
  s64.trace = nullptr;
  const double tol = std::max(s.eps_abs, s.eps_rel * i32.xi0);
  spock_info i64{};
  rc = solve_impl<double>(P, x0_dev, s64, z_dev, eta_dev, 1, &i64, st, tol, 0, nullptr);
  if (info) {
    *info = i64;
    info->iterations = i32.iterations + i64.iterations;
    info->n_T = i32.n_T + i64.n_T;
    info->n_K0 = i32.n_K0 + i64.n_K0;
    info->n_K1 = i32.n_K1 + i64.n_K1;
    info->n_K2 = i32.n_K2 + i64.n_K2;
    info->n_cap = i32.n_cap + i64.n_cap;
    info->n_backtracks = i32.n_backtracks + i64.n_backtracks;
    info->xi0 = i32.xi0;
    info->solve_ms = i32.solve_ms + i64.solve_ms;
    info->n_launches = i32.n_launches + i64.n_launches;
    info->n_timed = i32.n_timed + i64.n_timed;
    for (int g = 0; g < 7; ++g) info->t_group_ms[g] = i32.t_group_ms[g] + i64.t_group_ms[g];
    info->fp64_iterations = i64.iterations;
    info->certified = 1;
    info->xi_fp32 = i32.xi;
  }
  return rc;
}

static int solve_dev_impl(Problem* P, const double* x0_dev, const spock_settings* settings, double* z_dev,
                          double* eta_dev, int32_t warm, spock_info* info, cudaStream_t st) {
  spock_settings s;
  spock_default_settings(&s);
  if (settings) s = *settings;
  if (!x0_dev || !z_dev || !eta_dev) return fail(SPOCK_ERR_INVALID_ARG, "NULL buffer");
  if (s.memory < 0 || s.memory > kMaxMemory) return fail(SPOCK_ERR_INVALID_ARG, "memory must be in 0..16");
  if (!(s.eps_abs > 0) || !(s.eps_rel >= 0)) return fail(SPOCK_ERR_INVALID_ARG, "tolerances must be positive");
  if (s.max_iter < 0 || s.max_backtracks < 0) return fail(SPOCK_ERR_INVALID_ARG, "negative cap");
  if (s.alpha > 0 && s.alpha * P->normL >= 1.0) return fail(SPOCK_ERR_INVALID_ARG, "alpha ||L|| must be < 1");
  CUDA_TRY(cudaSetDevice(P->device));
  int rc;
  if (s.precision == SPOCK_FP64) rc = solve_impl<double>(*P, x0_dev, s, z_dev, eta_dev, warm, info, st);
  else if (s.precision == SPOCK_FP32) rc = solve_mixed(*P, x0_dev, s, z_dev, eta_dev, warm, info, st);
  else return fail(SPOCK_ERR_INVALID_ARG, "unknown precision");
  if (info && rc >= 0) info->n_L = 2 * info->n_T;   // L z and L z+ in every evaluation of T
  return rc;
}

// Root box check on a host copy of x0.
static int root_box_ok(const Problem& P, const double* x0, cudaStream_t st, bool x0_on_device) {
  std::vector<double> h(P.nx);
  if (x0_on_device) {
    CUDA_TRY(cudaMemcpyAsync(h.data(), x0, sizeof(double) * P.nx, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  } else {
    std::memcpy(h.data(), x0, sizeof(double) * P.nx);
  }
  if (P.general) {   // the root's constraint rows involve u^0: only finiteness is checked
    for (int r = 0; r < P.nx; ++r)
      if (!std::isfinite(h[r])) return fail(SPOCK_ERR_NUMERICAL, "x0 is not finite");
    return SPOCK_OK;
  }
  std::vector<double> lo(P.nx), hi(P.nx);
  CUDA_TRY(cudaMemcpy(lo.data(), P.f64.xlo, sizeof(double) * P.nx, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(hi.data(), P.f64.xhi, sizeof(double) * P.nx, cudaMemcpyDeviceToHost));
  for (int r = 0; r < P.nx; ++r) {
    if (!std::isfinite(h[r])) return fail(SPOCK_ERR_NUMERICAL, "x0 is not finite");
    if (h[r] < lo[r] || h[r] > hi[r]) return fail(SPOCK_ERR_INVALID_ARG, "x0 violates the box of the root node");
  }
  return SPOCK_OK;
}

int spock_solve_dev(spock_problem* p, const double* x0_dev, const spock_settings* settings, double* z_dev,
                    double* eta_dev, int32_t warm, spock_info* info, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P) return fail(SPOCK_ERR_INVALID_ARG, "not a problem handle");
    if (!x0_dev) return fail(SPOCK_ERR_INVALID_ARG, "x0 is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = root_box_ok(*P, x0_dev, st, true);
    if (rc != SPOCK_OK) return rc;
    return solve_dev_impl(P, x0_dev, settings, z_dev, eta_dev, warm, info, st);
  });
}

// Device staging buffers of the host-buffer entry points (allocated once per
// problem, reused by every call).
static void host_io_buffers(Problem& P, double** dx0, double** dz, double** de) {
  if (!P.io_x0) {
    CUDA_TRY(cudaMalloc(&P.io_x0, sizeof(double) * P.nx));
    P.allocations.push_back(P.io_x0);
    CUDA_TRY(cudaMalloc(&P.io_z, sizeof(double) * P.off.n_z));
    P.allocations.push_back(P.io_z);
    CUDA_TRY(cudaMalloc(&P.io_eta, sizeof(double) * P.off.n_eta));
    P.allocations.push_back(P.io_eta);
  }
  *dx0 = P.io_x0;
  *dz = P.io_z;
  *de = P.io_eta;
}

int spock_solve(spock_problem* p, const double* x0, const spock_settings* settings, double* z_io, double* eta_io,
                int32_t warm, spock_info* info) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P) return fail(SPOCK_ERR_INVALID_ARG, "not a problem handle");
    if (!x0 || !z_io || !eta_io) return fail(SPOCK_ERR_INVALID_ARG, "NULL buffer");
    CUDA_TRY(cudaSetDevice(P->device));
    int rc = root_box_ok(*P, x0, nullptr, false);
    if (rc != SPOCK_OK) return rc;
    const int64_t nz = P->off.n_z, ne = P->off.n_eta;
    double *dx0 = nullptr, *dz = nullptr, *de = nullptr;
    host_io_buffers(*P, &dx0, &dz, &de);
    CUDA_TRY(cudaMemcpy(dx0, x0, sizeof(double) * P->nx, cudaMemcpyHostToDevice));
    if (warm) {
      CUDA_TRY(cudaMemcpy(dz, z_io, sizeof(double) * nz, cudaMemcpyHostToDevice));
      CUDA_TRY(cudaMemcpy(de, eta_io, sizeof(double) * ne, cudaMemcpyHostToDevice));
    }
    rc = solve_dev_impl(P, dx0, settings, dz, de, warm, info, nullptr);
    if (rc == SPOCK_OK || rc == SPOCK_MAX_ITER) {
      CUDA_TRY(cudaMemcpy(z_io, dz, sizeof(double) * nz, cudaMemcpyDeviceToHost));
      CUDA_TRY(cudaMemcpy(eta_io, de, sizeof(double) * ne, cudaMemcpyDeviceToHost));
    }
    return rc;
  });
}

int spock_cp_step_dev(spock_problem* p, const double* x0_dev, int32_t k, double alpha, int32_t precision,
                      double* z_dev, double* eta_dev, double* xi_out, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P) return fail(SPOCK_ERR_INVALID_ARG, "not a problem handle");
    if (!x0_dev || !z_dev || !eta_dev || k < 0) return fail(SPOCK_ERR_INVALID_ARG, "NULL buffer or k < 0");
    if (alpha > 0 && alpha * P->normL >= 1.0) return fail(SPOCK_ERR_INVALID_ARG, "alpha ||L|| must be < 1");
    CUDA_TRY(cudaSetDevice(P->device));
    cudaStream_t st = (cudaStream_t)stream;
    int rc = root_box_ok(*P, x0_dev, st, true);
    if (rc != SPOCK_OK) return rc;
    if (precision == SPOCK_FP64) return cp_impl<double>(*P, x0_dev, k, alpha, z_dev, eta_dev, xi_out, st);
    if (precision == SPOCK_FP32) return cp_impl<float>(*P, x0_dev, k, alpha, z_dev, eta_dev, xi_out, st);
    return fail(SPOCK_ERR_INVALID_ARG, "unknown precision");
  });
}

int spock_cp_step(spock_problem* p, const double* x0, int32_t k, double alpha, int32_t precision, double* z_io,
                  double* eta_io, double* xi_out) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P) return fail(SPOCK_ERR_INVALID_ARG, "not a problem handle");
    if (!x0 || !z_io || !eta_io) return fail(SPOCK_ERR_INVALID_ARG, "NULL buffer");
    CUDA_TRY(cudaSetDevice(P->device));
    const int64_t nz = P->off.n_z, ne = P->off.n_eta;
    double *dx0 = nullptr, *dz = nullptr, *de = nullptr;
    host_io_buffers(*P, &dx0, &dz, &de);
    CUDA_TRY(cudaMemcpy(dx0, x0, sizeof(double) * P->nx, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(dz, z_io, sizeof(double) * nz, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(de, eta_io, sizeof(double) * ne, cudaMemcpyHostToDevice));
    int rc = spock_cp_step_dev(p, dx0, k, alpha, precision, dz, de, xi_out, nullptr);
    if (rc != SPOCK_OK) return rc;
    CUDA_TRY(cudaMemcpy(z_io, dz, sizeof(double) * nz, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(eta_io, de, sizeof(double) * ne, cudaMemcpyDeviceToHost));
    return SPOCK_OK;
  });
}

// ---- operator-level entry points (FP64, device buffers) --------------------
static KP<double> op_kp(Problem* P, double alpha) {
  return make_kp<double>(*P, default_alpha(*P, alpha), P->idx.stage_begin);
}

int spock_apply_L_dev(spock_problem* p, const double* z, double* eta_out, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !z || !eta_out) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(P->device));
    KP<double> kp = op_kp(P, 0.0);
    const int grid = std::min((P->tree.n + 3) / 4, sm_count() * 16);
    launch_dual<double>(kp, DM_APPLY_L_, false, z, nullptr, nullptr, eta_out, nullptr, nullptr, grid,
                        (cudaStream_t)stream);
    check_launch();
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return SPOCK_OK;
  });
}

int spock_apply_Lt_dev(spock_problem* p, const double* eta, double* z_out, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !eta || !z_out) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(P->device));
    KP<double> kp = op_kp(P, 0.0);
    const int grid = std::min((P->tree.n + 3) / 4, sm_count() * 16);
    launch_lstar<double>(kp, eta, z_out, grid,
                          (cudaStream_t)stream);
    check_launch();
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return SPOCK_OK;
  });
}

int spock_prox_f_dev(spock_problem* p, const double* x0_dev, double alpha, const double* z, double* z_out,
                     void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !x0_dev || !z || !z_out) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(P->device));
    cudaStream_t st = (cudaStream_t)stream;
    Workspace* ws = get_ws_impl<double>(*P, 0);
    KP<double> kp = op_kp(P, alpha);
    CUDA_TRY(cudaMemcpyAsync(P->f64.x0, x0_dev, sizeof(double) * P->nx, cudaMemcpyDeviceToDevice, st));
    launch_prep<double>(kp, z, (const double*)ws->zero_eta, z_out, sm_count() * 16, st);
    launch_riccati<double>(kp, P->tree.stage_begin, P->tree.stage_maxch, z_out, st, nullptr);
    check_launch();
    CUDA_TRY(cudaStreamSynchronize(st));
    check_device_flag(*P, st);
    return SPOCK_OK;
  });
}

int spock_prox_gconj_dev(spock_problem* p, double alpha, const double* eta, double* eta_out, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !eta || !eta_out) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(P->device));
    KP<double> kp = op_kp(P, alpha);
    const int grid = std::min((P->tree.n + 3) / 4, sm_count() * 16);
    launch_dual<double>(kp, DM_PROXG_, false, nullptr, nullptr, eta, eta_out, nullptr, nullptr, grid,
                        (cudaStream_t)stream);
    check_launch();
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return SPOCK_OK;
  });
}

int spock_T_dev(spock_problem* p, const double* x0_dev, double alpha, const double* z, const double* eta,
                double* z_out, double* eta_out, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !x0_dev || !z || !eta || !z_out || !eta_out) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(P->device));
    cudaStream_t st = (cudaStream_t)stream;
    KP<double> kp = op_kp(P, alpha);
    CUDA_TRY(cudaMemcpyAsync(P->f64.x0, x0_dev, sizeof(double) * P->nx, cudaMemcpyDeviceToDevice, st));
    launch_prep<double>(kp, z, eta, z_out, sm_count() * 16, st);
    launch_riccati<double>(kp, P->tree.stage_begin, P->tree.stage_maxch, z_out, st, nullptr);
    launch_dual<double>(kp, DM_DUAL_, false, z, z_out, eta, eta_out, nullptr, nullptr,
                        std::min((P->tree.n + 3) / 4, sm_count() * 16), st);
    check_launch();
    CUDA_TRY(cudaStreamSynchronize(st));
    check_device_flag(*P, st);
    return SPOCK_OK;
  });
}

int spock_grad_dev(spock_problem* p, const double* z, const double* eta, int32_t precision, double* g_x0,
                   double* g_A, double* g_B, double* g_Q, double* g_R, double* g_QN, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !z || !eta) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(P->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == SPOCK_FP64) return grad_impl<double>(*P, z, eta, g_x0, g_A, g_B, g_Q, g_R, g_QN, st);
    if (precision == SPOCK_FP32) return grad_impl<float>(*P, z, eta, g_x0, g_A, g_B, g_Q, g_R, g_QN, st);
    return fail(SPOCK_ERR_INVALID_ARG, "unknown precision");
  });
}

int spock_grad(spock_problem* p, const double* z, const double* eta, int32_t precision, double* g_x0, double* g_A,
               double* g_B, double* g_Q, double* g_R, double* g_QN) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !z || !eta) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(cudaSetDevice(P->device));
    const size_t n = (size_t)P->tree.n, nx = (size_t)P->nx, nu = (size_t)P->nu;
    double *dx0 = nullptr, *dz = nullptr, *de = nullptr;
    host_io_buffers(*P, &dx0, &dz, &de);
    if (!P->io_grad) {   // gradient outputs, allocated once per problem
      const size_t len = nx + n * nx * nx + n * nx * nu + 2 * n * nx + n * nu;
      CUDA_TRY(cudaMalloc(&P->io_grad, sizeof(double) * len));
      P->allocations.push_back(P->io_grad);
    }
    double* gx0 = P->io_grad;
    double* gA = gx0 + nx;
    double* gB = gA + n * nx * nx;
    double* gQ = gB + n * nx * nu;
    double* gR = gQ + n * nx;
    double* gQN = gR + n * nu;
    CUDA_TRY(cudaMemcpy(dz, z, sizeof(double) * P->off.n_z, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(de, eta, sizeof(double) * P->off.n_eta, cudaMemcpyHostToDevice));
    const int rc = spock_grad_dev(p, dz, de, precision, g_x0 ? gx0 : nullptr, g_A ? gA : nullptr,
                                  g_B ? gB : nullptr, g_Q ? gQ : nullptr, g_R ? gR : nullptr,
                                  g_QN ? gQN : nullptr, nullptr);
    if (rc != SPOCK_OK) return rc;
    const struct { double* host; const double* dev; size_t len; } outs[] = {
        {g_x0, gx0, nx}, {g_A, gA, n * nx * nx}, {g_B, gB, n * nx * nu},
        {g_Q, gQ, n * nx}, {g_R, gR, n * nu}, {g_QN, gQN, n * nx}};
    for (const auto& o : outs)
      if (o.host) CUDA_TRY(cudaMemcpy(o.host, o.dev, sizeof(double) * o.len, cudaMemcpyDeviceToHost));
    return SPOCK_OK;
  });
}

int spock_fp64_fma_rate(int32_t iters, double* tflops, void* stream) {
  return guarded([&]() -> int {
    if (iters < 1 || !tflops) return fail(SPOCK_ERR_INVALID_ARG, "need iters >= 1 and an output");
    return fp64_fma_rate(iters, tflops, (cudaStream_t)stream);
  });
}

int spock_adjoint_dev(spock_problem* p, const double* z, const double* eta, const double* g_z, int32_t max_iter,
                      double tol, double* g_x0, double* g_A, double* g_B, double* g_Q, double* g_R, double* g_QN,
                      int32_t* iterations, double* residual, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !z || !eta) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    if (max_iter < 1 || !(tol > 0.0)) return fail(SPOCK_ERR_INVALID_ARG, "need max_iter >= 1 and tol > 0");
    CUDA_TRY(cudaSetDevice(P->device));
    return adjoint_impl(*P, z, eta, g_z, max_iter, tol, g_x0, g_A, g_B, g_Q, g_R, g_QN, iterations, residual,
                        (cudaStream_t)stream);
  });
}

int spock_batch_create(int32_t n, spock_problem* const* problems, spock_batch** out) {
  return guarded([&]() -> int {
    if (n < 1 || !problems || !out) return fail(SPOCK_ERR_INVALID_ARG, "need n >= 1 problems and an out pointer");
    auto* B = new Batch();
    try {
      for (int i = 0; i < n; ++i) {
        Problem* P = as_problem(problems[i]);
        if (!P) {
          delete B;
          return fail(SPOCK_ERR_INVALID_ARG, "not a problem handle in the batch");
        }
        if (P->general) {
          delete B;
          return fail(SPOCK_ERR_UNSUPPORTED, "batches take box-form problems only");
        }
        for (Problem* q : B->probs)
          if (q == P) {
            delete B;
            return fail(SPOCK_ERR_INVALID_ARG, "a problem appears twice in the batch (instances need their own problem)");
          }
        B->probs.push_back(P);
      }
      CUDA_TRY(cudaSetDevice(B->probs[0]->device));
      CUDA_TRY(cudaStreamCreateWithFlags(&B->main, cudaStreamNonBlocking));
      CUDA_TRY(cudaMalloc(&B->st_ptrs, sizeof(SmState*) * n));
      CUDA_TRY(cudaMalloc(&B->done_dev, sizeof(int32_t) * n));
      CUDA_TRY(cudaMallocHost(&B->done_host, sizeof(int32_t) * n));
    } catch (...) {
      delete B;
      throw;
    }
    *out = reinterpret_cast<spock_batch*>(B);
    return SPOCK_OK;
  });
}

int spock_batch_solve_dev(spock_batch* batch, const double* const* x0_dev, const spock_settings* settings,
                          double* const* z_dev, double* const* eta_dev, int32_t warm, spock_info* infos) {
  return guarded([&]() -> int {
    Batch* B = reinterpret_cast<Batch*>(batch);
    if (!B || B->tag != TAG_BATCH || !x0_dev || !z_dev || !eta_dev)
      return fail(SPOCK_ERR_INVALID_ARG, "NULL argument or not a batch handle");
    spock_settings s;
    spock_default_settings(&s);
    if (settings) s = *settings;
    if (s.memory < 0 || s.memory > kMaxMemory) return fail(SPOCK_ERR_INVALID_ARG, "memory must be in 0..16");
    if (!(s.eps_abs > 0) || !(s.eps_rel >= 0)) return fail(SPOCK_ERR_INVALID_ARG, "tolerances must be positive");
    if (s.max_iter < 0 || s.max_backtracks < 0) return fail(SPOCK_ERR_INVALID_ARG, "negative cap");
    for (size_t i = 0; i < B->probs.size(); ++i) {
      if (!x0_dev[i] || !z_dev[i] || !eta_dev[i]) return fail(SPOCK_ERR_INVALID_ARG, "NULL instance buffer");
      if (s.alpha > 0 && s.alpha * B->probs[i]->normL >= 1.0)
        return fail(SPOCK_ERR_INVALID_ARG, "alpha ||L|| must be < 1 for every instance");
      int rc = root_box_ok(*B->probs[i], x0_dev[i], nullptr, true);
      if (rc != SPOCK_OK) return rc;
    }
    CUDA_TRY(cudaSetDevice(B->probs[0]->device));
    int rc;
    if (s.precision == SPOCK_FP64) rc = batch_solve<double>(*B, x0_dev, s, z_dev, eta_dev, warm, infos);
    else if (s.precision == SPOCK_FP32) rc = batch_solve<float>(*B, x0_dev, s, z_dev, eta_dev, warm, infos);
    else return fail(SPOCK_ERR_INVALID_ARG, "unknown precision");
    if (infos && rc >= 0)
      for (size_t i = 0; i < B->probs.size(); ++i) infos[i].n_L = 2 * infos[i].n_T;
    return rc;
  });
}

int spock_batch_solve(spock_batch* batch, const double* const* x0, const spock_settings* settings,
                      double* const* z_io, double* const* eta_io, int32_t warm, spock_info* infos) {
  return guarded([&]() -> int {
    Batch* B = reinterpret_cast<Batch*>(batch);
    if (!B || B->tag != TAG_BATCH || !x0 || !z_io || !eta_io)
      return fail(SPOCK_ERR_INVALID_ARG, "NULL argument or not a batch handle");
    const size_t n = B->probs.size();
    for (size_t i = 0; i < n; ++i)
      if (!x0[i] || !z_io[i] || !eta_io[i]) return fail(SPOCK_ERR_INVALID_ARG, "NULL instance buffer");
    CUDA_TRY(cudaSetDevice(B->probs[0]->device));
    // every instance is a distinct problem: its own staging buffers serve
    std::vector<const double*> dx0(n);
    std::vector<double*> dz(n), de(n);
    for (size_t i = 0; i < n; ++i) {
      Problem& P = *B->probs[i];
      double *a = nullptr, *b = nullptr, *c = nullptr;
      host_io_buffers(P, &a, &b, &c);
      CUDA_TRY(cudaMemcpyAsync(a, x0[i], sizeof(double) * P.nx, cudaMemcpyHostToDevice, B->main));
      if (warm) {
        CUDA_TRY(cudaMemcpyAsync(b, z_io[i], sizeof(double) * P.off.n_z, cudaMemcpyHostToDevice, B->main));
        CUDA_TRY(cudaMemcpyAsync(c, eta_io[i], sizeof(double) * P.off.n_eta, cudaMemcpyHostToDevice, B->main));
      }
      dx0[i] = a;
      dz[i] = b;
      de[i] = c;
    }
    CUDA_TRY(cudaStreamSynchronize(B->main));
    const int rc = spock_batch_solve_dev(batch, dx0.data(), settings, dz.data(), de.data(), warm, infos);
    if (rc == SPOCK_OK || rc == SPOCK_MAX_ITER) {
      for (size_t i = 0; i < n; ++i) {
        const Problem& P = *B->probs[i];
        CUDA_TRY(cudaMemcpyAsync(z_io[i], dz[i], sizeof(double) * P.off.n_z, cudaMemcpyDeviceToHost, B->main));
        CUDA_TRY(cudaMemcpyAsync(eta_io[i], de[i], sizeof(double) * P.off.n_eta, cudaMemcpyDeviceToHost,
                                 B->main));
      }
      CUDA_TRY(cudaStreamSynchronize(B->main));
    }
    return rc;
  });
}

int spock_problem_clone(const spock_problem* base, spock_problem** out) {
  return guarded([&]() -> int {
    Problem* B = const_cast<Problem*>(reinterpret_cast<const Problem*>(base));
    if (!B || B->tag != TAG_PROBLEM || !out) return fail(SPOCK_ERR_INVALID_ARG, "not a problem handle");
    while (B->base) B = B->base;   // clones of clones share the original
    CUDA_TRY(cudaSetDevice(B->device));
    auto* C = new Problem();
    try {
      C->device = B->device;
      C->tree = B->tree;
      C->off = B->off;
      C->nx = B->nx;
      C->nu = B->nu;
      C->normL = B->normL;
      C->general = B->general;
      C->gd = B->gd;
      C->idx = B->idx;      // read-only index arrays, shared
      C->f64 = B->f64;      // data and factors, shared
      C->f32 = B->f32;
      const Tree& t = C->tree;
      auto scratch = [&](auto& f, auto zero) {
        using S = decltype(zero);
        f.xbar = dalloc<S>(*C, (size_t)t.n * f.xs);
        f.ubar = dalloc<S>(*C, (size_t)t.n_nonleaf * f.us);
        f.q = dalloc<S>(*C, (size_t)t.n * f.xs);
        f.d = dalloc<S>(*C, (size_t)t.n_nonleaf * f.us);
        f.x0 = dalloc<S>(*C, (size_t)C->nx);
      };
      scratch(C->f64, 0.0);
      scratch(C->f32, 0.0f);
      C->err = upload(*C, std::vector<int32_t>(1, 0));
      CUDA_TRY(cudaDeviceSynchronize());
    } catch (...) {
      delete C;
      throw;
    }
    C->base = B;
    B->n_clones++;
    *out = reinterpret_cast<spock_problem*>(C);
    return SPOCK_OK;
  });
}

void spock_free(void* handle) {
  if (!handle) return;
  const int32_t tag = *reinterpret_cast<const int32_t*>(handle);
  if (tag == TAG_TREE) {
    delete reinterpret_cast<Tree*>(handle);
  } else if (tag == TAG_PROBLEM) {
    Problem* P = reinterpret_cast<Problem*>(handle);
    if (P->n_clones > 0) {   // clones still use its device data: delete it with the last one
      P->free_pending = true;
      return;
    }
    Problem* B = P->base;
    delete P;
    if (B && --B->n_clones == 0 && B->free_pending) delete B;
  } else if (tag == TAG_BATCH) {
    delete reinterpret_cast<Batch*>(handle);
  }
}

const char* spock_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ===========================================================================
// Allocation-free variant of spock_prox_f_dev
// ===========================================================================
// For callers that must not allocate device memory on the call path (a
// real-time control loop with a fixed memory budget, or code that runs while
// another component owns the allocator): the scratch of prox_{alpha f} (the
// Riccati vectors xbar, ubar, q, d and an all-zero dual vector) lives in the
// fixed-size device array below instead of problem- or workspace-owned
// buffers.  Every GPU that loads this library holds the array until the
// process exits.
namespace spock {

constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;  // 8 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on `dev` (the current device).  Host
// code must not use the symbol itself: on the host it names a stand-in, not
// device memory.  Looked up once per device, by the first spock_problem_create
// on that device.
static int noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SPOCK_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(SPOCK_ERR_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SPOCK_OK;
}

}  // namespace spock

extern "C" int spock_prox_f_noalloc_dev(spock_problem* p, const double* x0_dev, double alpha, const double* z,
                                        double* z_out, void* stream) {
  return guarded([&]() -> int {
    Problem* P = as_problem(p);
    if (!P || !x0_dev || !z || !z_out) return fail(SPOCK_ERR_INVALID_ARG, "NULL argument");
    const Tree& t = P->tree;
    const size_t nxb = (size_t)t.n * P->f64.xs, nub = (size_t)t.n_nonleaf * P->f64.us;
    const size_t need = 2 * nxb + 2 * nub + (size_t)P->off.n_eta;
    if (need > kNoAllocScratchDoubles)
      return fail(SPOCK_ERR_INVALID_ARG, "problem too large for spock_prox_f_noalloc_dev: needs " +
                                             std::to_string(need) + " doubles of scratch, the fixed array holds " +
                                             std::to_string(kNoAllocScratchDoubles));
    CUDA_TRY(cudaSetDevice(P->device));
    double* scratch = nullptr;
    int rc = noalloc_scratch(P->device, &scratch);   // cached at problem creation
    if (rc != SPOCK_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    KP<double> kp = op_kp(P, alpha);
    kp.x0 = x0_dev;   // read in place: no buffer owned by the problem is written
    kp.xbar = scratch;
    kp.q = scratch + nxb;
    kp.ubar = scratch + 2 * nxb;
    kp.d = scratch + 2 * nxb + nub;
    double* zero_eta = scratch + 2 * nxb + 2 * nub;
    // the array keeps the previous call's contents: the dual input must be zero
    CUDA_TRY(cudaMemsetAsync(zero_eta, 0, sizeof(double) * (size_t)P->off.n_eta, st));
    launch_prep<double>(kp, z, zero_eta, z_out, sm_count() * 16, st);
    launch_riccati<double>(kp, P->tree.stage_begin, P->tree.stage_maxch, z_out, st, nullptr);
    check_launch();
    CUDA_TRY(cudaStreamSynchronize(st));
    check_device_flag(*P, st);
    return SPOCK_OK;
  });
}
