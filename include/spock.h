/*
 * spock.h -- C ABI of the GB300 SPOCK library (libspock.so).
 *
 * SPOCK solves the multistage risk-averse optimal control problem (RAOCP)
 * of arXiv 2212.01110 on a scenario tree: the Chambolle-Pock (CP) operator
 * T of Eq. (chambolle-pock-operator) applied to the splitting
 * min f(z) + g(Lz) of Sec. "Operator splitting", accelerated by SuperMann
 * with Anderson directions (Algorithm 3).  Every step of the iteration runs
 * in this library's CUDA kernels on one GPU.
 *
 * Conventions common to every entry point
 * ---------------------------------------
 *  - Return value: 0 (SPOCK_OK) on success, > 0 for a non-fatal outcome of a
 *    solve, < 0 for an error (see spock_status).  On error, out-parameters
 *    are left untouched and spock_last_error() describes the failure.
 *    No C++ exception crosses this boundary.
 *  - All host arrays are read during the call only; the library copies what
 *    it keeps.  Device pointers ("_dev" entry points) must point to memory of
 *    the current CUDA device and stay valid until the call returns; those
 *    calls are ordered on the given stream (cudaStream_t passed as void*,
 *    NULL = legacy default stream) and return after the stream has
 *    completed the work, except where stated.
 *  - Node ids are the caller's ("user") ids 0..n-1 with node 0 the root.
 *    Children of a node are ordered by increasing user id.
 *  - A handle is used by one host thread at a time.
 *
 * Layout of the primal vector z (length n_z) and the dual vector eta
 * (length n_eta), Sec. "Operator splitting" with box constraints
 * (Gamma = I in Eq. (constraints)) and AV@R risks
 * (Sec. "Conic representation of risk measures"); m_i = #children of i:
 *   z   = [ s^0,
 *           x^i (nx) for every node i in user order,
 *           u^i (nu) for every nonleaf i in user order,
 *           (y^i (2 m_i + 1), tau^c (m_i), s^c (m_i)) for every nonleaf i in
 *             user order, c running over the children of i ]
 *   eta = [ (y^i (2 m_i + 1), s^i - b^iT y^i (1), x^i (nx), u^i (nu))
 *             for every nonleaf i,
 *           (Q^c^1/2 x^anc(c) (nx), R^c^1/2 u^anc(c) (nu), tau^c/2, tau^c/2)
 *             for every nonroot c,
 *           (x^j (nx), Q_N^j^1/2 x^j (nx), s^j/2, s^j/2) for every leaf j ]
 *   with b^i = (p^ch(i), 0_{m_i}, 1) built from conditional probabilities.
 */
#ifndef SPOCK_H
#define SPOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spock_status {
  SPOCK_OK = 0,
  SPOCK_MAX_ITER = 1,          /* iteration cap reached; buffers hold T(v) of the last iterate */
  SPOCK_ERR_INVALID_ARG = -1,  /* NULL pointer, size out of range, x0 outside its box, ... */
  SPOCK_ERR_BAD_TREE = -2,     /* ancestor array is not a tree with all leaves at one stage */
  SPOCK_ERR_NOT_POSDEF = -3,   /* a cost weight is not positive */
  SPOCK_ERR_NUMERICAL = -4,    /* NaN/Inf in inputs or during the iteration */
  SPOCK_ERR_CUDA = -5,         /* a CUDA runtime call failed */
  SPOCK_ERR_OOM = -6,          /* device or host allocation failed */
  SPOCK_ERR_UNSUPPORTED = -7   /* option not implemented by this build */
} spock_status;

typedef enum spock_precision {
  SPOCK_FP64 = 0,  /* every vector and factor in double precision */
  SPOCK_FP32 = 1   /* operator T in single precision (factors rounded from the
                      FP64 Algorithm 1), residual, M-norms, Anderson Gram and
                      least squares accumulated/solved in double */
} spock_precision;

typedef struct spock_tree spock_tree;
typedef struct spock_problem spock_problem;
typedef struct spock_batch spock_batch;

/* Settings of Algorithm 3.  spock_default_settings() fills the defaults. */
typedef struct spock_settings {
  double eps_abs;       /* stop when xi <= max(eps_abs, eps_rel * xi_0)      (1e-6) */
  double eps_rel;       /*                                                    (1e-6) */
  double alpha;         /* CP step; <= 0 selects 0.99 / ||L||                  (0)    */
  int32_t memory;       /* Anderson memory m (difference columns), 0..16      (3)    */
  double c0, c1, c2;    /* SuperMann K0/K1 constants, in [0, 1)               (0.99) */
  double beta;          /* line-search reduction, (0, 1)                      (0.5)  */
  double sigma;         /* K2 acceptance, (0, 1)                              (0.1)  */
  double lambda;        /* K2 relaxation, (0, 2)                              (1.0)  */
  double rho_coef;      /* coefficient of <r~, v~ - v>_M in rho               (1.0)  */
  int32_t max_iter;     /* SuperMann iteration cap                            (100000) */
  int32_t max_backtracks; /* line-search cap; at the cap tau = 0             (30)   */
  int32_t precision;    /* spock_precision                                   (FP64) */
  int32_t* trace;       /* optional host array of 2*max_iter int32: per iteration
                           (branch, backtracks), branch 0=K0 1=K1 2=K2 3=cap  (NULL) */
  int32_t profile;      /* nonzero: time the kernel groups of every T evaluation
                           with CUDA events on the solve's stream (info.t_*)  (0)    */
  int32_t fp64_tail;    /* SPOCK_FP32 only: when the FP32 iteration meets the
                           tolerance, certify it with one FP64 evaluation of T,
                           and continue in FP64 (warm start, Anderson memory
                           reset) until the FP64 residual meets it too; also
                           taken when FP32 stagnates                       (1)    */
  int32_t stall_window; /* FP32 stagnation: no halving of xi in this many
                           iterations while xi <= 30 x tolerance hands over
                           to FP64 (0 = never)                             (2000)  */
} spock_settings;

/* Outcome of a solve. */
typedef struct spock_info {
  int32_t status;       /* spock_status of the solve */
  int32_t iterations;   /* SuperMann iterations k */
  int32_t n_T;          /* evaluations of the CP operator T */
  int32_t n_K0, n_K1, n_K2, n_cap, n_backtracks;
  double xi;            /* termination residual xi at the returned pair */
  double xi0;           /* xi at the initial point */
  double alpha;         /* CP step used */
  double solve_ms;      /* device time of the solve (CUDA events) */
  int32_t n_launches;   /* kernels launched by the solve */
  int32_t n_timed;      /* T evaluations timed when settings.profile != 0 */
  /* summed device time (ms) of the kernel groups of the timed T evaluations:
     [0] zbar = z - alpha L* eta and proj_S2, [1] Riccati backward, chain
     region, [2] Riccati backward, branching stages, [3] Riccati forward,
     branching stages, [4] Riccati forward, chain region, [5] L and
     prox_{alpha g*} (dual update, with the residual statistics accumulated
     in the same pass), [6] reduction of the statistics */
  double t_group_ms[7];
  int32_t fp64_iterations; /* SPOCK_FP32 with fp64_tail: iterations run in FP64 */
  int32_t certified;       /* 1 if the returned pair's xi was computed in FP64 */
  double xi_fp32;          /* xi reported by the FP32 iteration when it stopped */
  int32_t n_L;             /* applications of L (the x-axis of Fig. 1): two per
                              evaluation of T -- L z and L z+, from which the
                              dual update L(2 z+ - z) and the residual's L r_z
                              are formed in the same pass */
} spock_info;

/* Fills *s with the defaults listed above.  Returns SPOCK_ERR_INVALID_ARG
   if s is NULL. */
int spock_default_settings(spock_settings* s);

/*
 * spock_tree_create -- scenario tree of Sec. "Scenario trees".
 *   n_nodes : number of nodes, >= 2.
 *   anc     : [n_nodes] ancestor of each node; anc[0] = -1 (root), others
 *             in [0, n_nodes).  All leaves must lie at the same stage N >= 1.
 *   prob    : [n_nodes] conditional probability p^i = pi^i / pi^anc(i) of
 *             each nonroot node (prob[0] ignored); positive, summing to 1
 *             over the children of each node within 1e-9.
 *   out     : receives the new handle (free with spock_free).
 * Errors: SPOCK_ERR_INVALID_ARG (NULL pointer, n_nodes < 2, bad
 * probabilities), SPOCK_ERR_BAD_TREE (not a tree / uneven leaf depth).
 * Host only; no GPU work.
 */
int spock_tree_create(int32_t n_nodes, const int32_t* anc, const double* prob,
                      spock_tree** out);

/*
 * spock_tree_create_abs -- as spock_tree_create, with the absolute
 * probability pi^i of every node (Sec. "Scenario trees": pi^i is the
 * probability of reaching node i; pi[0] is the root's, normally 1).  The
 * conditional probabilities p^i = pi^i / pi^anc(i) are formed here, so the
 * children of every node must carry their parent's probability in total
 * (within 1e-9 relative).  Errors as spock_tree_create; non-positive or
 * non-finite pi is SPOCK_ERR_INVALID_ARG.  Host only; no GPU work.
 */
int spock_tree_create_abs(int32_t n_nodes, const int32_t* anc, const double* pi, spock_tree** out);

/* Number of nodes, horizon N and number of nonleaf nodes of a tree. */
int spock_tree_info(const spock_tree* tree, int32_t* n_nodes, int32_t* horizon,
                    int32_t* n_nonleaf);

/*
 * spock_problem_create -- RAOCP data on a tree (Sec. "Multistage nested
 * risk-averse OCPs"), with diagonal costs and box constraints, and the
 * offline factorisation of the projection on the dynamics (Algorithm 1, in
 * FP64 on the host).  All arrays are host arrays indexed by user node id;
 * entries of nodes where a quantity does not exist are ignored.
 *   nx, nu    : state / input dimension, 1 <= nx, nu and nx + nu <= 128.
 *   A         : [n][nx][nx] row-major, A^i of the edge into node i (Eq.
 *               (finite-horizon-evolution-2)); A[0] ignored.
 *   B         : [n][nx][nu] row-major, B^i; B[0] ignored.
 *   Q         : [n][nx] diagonal of Q^i (> 0), stage cost of the edge into i.
 *   R         : [n][nu] diagonal of R^i (> 0).
 *   QN        : [n][nx] diagonal of the terminal weight Q_N^j (> 0), leaves.
 *   a         : [n] AV@R parameter of each nonleaf node, in [0, 1].
 *   xmin,xmax : [n][nx] state box of every node (xmin <= xmax).
 *   umin,umax : [n][nu] input box of every nonleaf node.
 *   flags     : 0, or SPOCK_DENSE_COST: Q, R, QN are then full symmetric
 *               positive definite matrices [n][nx][nx], [n][nu][nu],
 *               [n][nx][nx] (row-major), as in spock_problem_create_general,
 *               and the problem runs on the general-form kernels with the
 *               box rows as constraint matrices Gamma = I.
 *   out       : receives the handle; it owns a copy of the data, the FP64
 *               factors (and their FP32 copies) in device memory.
 * The current CUDA device at creation is used for every later call.
 * Errors: INVALID_ARG, NOT_POSDEF, NUMERICAL (non-finite input), CUDA, OOM,
 * UNSUPPORTED (unknown flag).
 */
#define SPOCK_DENSE_COST 1
int spock_problem_create(const spock_tree* tree, int32_t nx, int32_t nu,
                         const double* A, const double* B, const double* Q,
                         const double* R, const double* QN, const double* a,
                         const double* xmin, const double* xmax,
                         const double* umin, const double* umax,
                         int32_t flags, spock_problem** out);

/*
 * spock_problem_create_general -- RAOCP data in the paper's general form:
 * constraints Gamma_x^i x^i + Gamma_u^i u^i in C^i (nonleaf i) and
 * Gamma_N^j x^j in C_N^j (leaf j) of Eq. (constraints), with C^i, C_N^j
 * boxes, and quadratic costs with full matrices (Sec. "Quadratic costs").
 * The rows of L (definition of L) become per-node matrix-vector products:
 *   nonleaf block:  (y^i, s^i - b'y^i, Gamma_x^i x^i + Gamma_u^i u^i)   nc rows
 *   nonroot block:  (Q^i^1/2 x^anc, R^i^1/2 u^anc, tau^i/2, tau^i/2)
 *   leaf block:     (Gamma_N^j x^j, Q_N^j^1/2 x^j, s^j/2, s^j/2)         ncN rows
 * where M^1/2 is the upper Cholesky factor F of M (F'F = M; any factor gives
 * the same cost ||F x||^2 = x'Mx, this one is the library's).  Eta is laid out
 * as for spock_problem_create with nc (nonleaf) and ncN (leaf) constraint
 * rows in place of the nx + nu and nx box rows.  ||L|| is the largest norm
 * of the per-node blocks (remark after the definition of L): the largest
 * eigenvalue of Gamma^i'Gamma^i + sum_c blockdiag(Q^c, R^c), resp.
 * Gamma_N'Gamma_N + Q_N, found by power iteration and certified as an upper
 * bound by a Cholesky factorisation of (lambda (1 + 1e-9) I - M) on the host.
 *   A, B, a     : as spock_problem_create (a is read only where risk is NULL).
 *   risk        : NULL (AV@R with parameter a at every nonleaf node), or [n]
 *                 per node (caller's numbering; leaves ignored) a coherent
 *                 risk measure in the conic form of Sec. "Conic representation
 *                 of risk measures", Eq. (dual_risk): rho[Z] = min { y'b :
 *                 E'y = Z, F'y = 0, y in K* } with K = R^kp_+ x {0}^(ny - kp).
 *                 Then y^i has ny entries, S2^i = ker [[E'  -I  -I], [F'  0  0]]
 *                 (projected with the dense projector I - M'(MM')^-1 M, formed
 *                 on the host: M must have full row rank, i.e. F full column
 *                 rank), and (K^i)* = R^kp_+ x R^(ny - kp) in S3.  Needs
 *                 ny + 2 m <= 160 per node.  With risk NULL the AV@R
 *                 projection on S2 is the closed form (any m).  z_2 of node i is (y^i [ny],
 *                 tau^[i] [m], s^[i] [m]) and its nonleaf eta block
 *                 (y^i [ny], s^i - b'y^i, constraint rows [nc]).
 *   Q, R, QN    : with flags & SPOCK_DENSE_COST: [n][nx][nx], [n][nu][nu],
 *                 [n][nx][nx] symmetric positive definite (row-major; the
 *                 upper triangle is read); otherwise diagonals [n][nx],
 *                 [n][nu], [n][nx] (> 0).
 *   nc          : constraint rows per nonleaf node, 1 <= nc <= 128.
 *   Gx, Gu      : [n][nc][nx], [n][nc][nu] row-major Gamma_x^i, Gamma_u^i
 *                 (read at nonleaf nodes).
 *   cmin, cmax  : [n][nc] bounds of C^i (cmin <= cmax; +-inf allowed).
 *   ncN         : constraint rows per leaf, 1 <= ncN <= 128.
 *   GN          : [n][ncN][nx] row-major Gamma_N^j (read at leaves).
 *   cNmin,cNmax : [n][ncN] bounds of C_N^j.
 *   flags       : 0 or SPOCK_DENSE_COST.
 * Every entry point that takes a problem accepts a general one except
 * spock_grad(_dev), spock_adjoint_dev (their formulas are written for
 * diagonal costs and box constraints) and spock_batch_create: these return
 * SPOCK_ERR_UNSUPPORTED.  Solves never use the single-block solve kernel.
 * Errors: INVALID_ARG, NOT_POSDEF (a cost matrix is not positive
 * definite), NUMERICAL, CUDA, OOM, UNSUPPORTED (unknown flag).
 */
typedef struct spock_risk {
  int32_t ny;        /* rows of y^i, >= 1 */
  int32_t n_nu;      /* columns of F^i, >= 0 */
  int32_t kp;        /* 0 <= kp <= ny: K^i = R^kp_+ x {0}^(ny - kp) */
  const double* b;   /* [ny] */
  const double* E;   /* [ny][m] row-major, m = the node's number of children */
  const double* F;   /* [ny][n_nu] row-major; may be NULL when n_nu = 0 */
} spock_risk;

int spock_problem_create_general(const spock_tree* tree, int32_t nx, int32_t nu,
                                 const double* A, const double* B, const double* Q,
                                 const double* R, const double* QN, const double* a,
                                 const spock_risk* risk,
                                 int32_t nc, const double* Gx, const double* Gu,
                                 const double* cmin, const double* cmax,
                                 int32_t ncN, const double* GN,
                                 const double* cNmin, const double* cNmax,
                                 int32_t flags, spock_problem** out);

/*
 * spock_problem_clone -- a problem with the same tree, data and offline
 * factors as `base`, sharing base's device copies of them (read-only), with
 * its own iterate, scratch and workspace buffers.  The paper has no
 * counterpart: it serves batches of instances that differ only in x0 (the
 * batched "family" form): spock_batch_create accepts the clones as distinct
 * instances, and each launch then reads a family's factors from HBM once and
 * from L2 for the other members.  A clone of a clone shares the original.
 * Freeing the base while clones exist defers its deletion to the last clone.
 * Errors: INVALID_ARG, CUDA, OOM.
 */
int spock_problem_clone(const spock_problem* base, spock_problem** out);

/* Sizes of z and eta, ||L|| (closed form, remark after the definition of L)
   and the seconds spent in Algorithm 1. */
int spock_problem_info(const spock_problem* p, int64_t* n_z, int64_t* n_eta,
                       double* norm_L, double* factor_seconds);

/*
 * spock_solve -- Algorithm 3 (SPOCK) from (z, eta), host buffers.
 *   x0       : [nx] initial state (must satisfy the root's box).
 *   settings : NULL for the defaults.
 *   z_io     : [n_z]  in: initial z if warm != 0; out: z of T(v) at termination.
 *   eta_io   : [n_eta] likewise for eta.
 *   warm     : 0 = cold start from v = 0 (inputs of z_io/eta_io ignored).
 *   info     : optional outcome.
 * Copies inputs to the device and results back inside the call.  Returns
 * SPOCK_OK on convergence, SPOCK_MAX_ITER at the iteration cap (outputs
 * written in both cases), or an error.
 * Execution: the SuperMann decisions are taken on the device; rounds of
 * (decision, Anderson update, next point, evaluation of T) are replayed from
 * a CUDA graph, or -- for problems of at most 64 nodes with nx + nu <= 62,
 * memory 0, 3 or 5 and no profiling -- the whole solve runs in one
 * single-block launch.  The environment variable SPOCK_DRIVER = graph /
 * cta / host forces the graph, the single block (if the problem fits) or a
 * host-driven loop.
 */
int spock_solve(spock_problem* p, const double* x0, const spock_settings* settings,
                double* z_io, double* eta_io, int32_t warm, spock_info* info);

/* As spock_solve with device buffers x0_dev [nx], z_dev [n_z], eta_dev
   [n_eta] (FP64) on stream `stream`. */
int spock_solve_dev(spock_problem* p, const double* x0_dev, const spock_settings* settings,
                    double* z_dev, double* eta_dev, int32_t warm, spock_info* info,
                    void* stream);

/*
 * spock_cp_step -- k iterations of the vanilla CP method v <- T(v)
 * (Eq. (chambolle-pock-operator)) on host buffers z_io [n_z], eta_io
 * [n_eta] (in: v_0, out: v_k).  xi_out (optional) receives xi of the pair
 * (v_{k-1}, v_k) (Sec. "The Chambolle-Pock method").  precision as in
 * spock_settings; alpha <= 0 selects 0.99/||L||.
 */
int spock_cp_step(spock_problem* p, const double* x0, int32_t k, double alpha,
                  int32_t precision, double* z_io, double* eta_io, double* xi_out);

/* Device-buffer variant of spock_cp_step. */
int spock_cp_step_dev(spock_problem* p, const double* x0_dev, int32_t k, double alpha,
                      int32_t precision, double* z_dev, double* eta_dev, double* xi_out,
                      void* stream);

/*
 * Operator-level entry points (device buffers, FP64, ordered on `stream`;
 * alpha <= 0 selects 0.99/||L||).  They expose the steps of T one by one:
 *   spock_apply_L_dev      eta_out = L z             (definition of L)
 *   spock_apply_Lt_dev     z_out   = L* eta          (adjoint, Sec. "Notation")
 *   spock_prox_f_dev       z_out   = prox_{alpha f}(z): s^0 - alpha, proj_S1 on
 *                          z_1 (Algorithm 2 with the factors of Algorithm 1),
 *                          proj_S2 on z_2 (Sec. "Proximal operator of f")
 *   spock_prox_gconj_dev   eta_out = prox_{alpha g*}(eta)
 *                                  = eta - alpha proj_S3(eta / alpha)
 *   spock_T_dev            (z_out, eta_out) = T(z, eta)
 * Output buffers must not alias inputs.
 */
int spock_apply_L_dev(spock_problem* p, const double* z, double* eta_out, void* stream);
int spock_apply_Lt_dev(spock_problem* p, const double* eta, double* z_out, void* stream);
int spock_prox_f_dev(spock_problem* p, const double* x0_dev, double alpha, const double* z,
                     double* z_out, void* stream);
int spock_prox_gconj_dev(spock_problem* p, double alpha, const double* eta, double* eta_out,
                         void* stream);
int spock_T_dev(spock_problem* p, const double* x0_dev, double alpha, const double* z,
                const double* eta, double* z_out, double* eta_out, void* stream);

/*
 * spock_prox_f_noalloc_dev -- spock_prox_f_dev without any allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run (a control loop with a fixed
 * memory budget, or code executing while another component owns the device
 * allocator).  It computes exactly what spock_prox_f_dev computes, but the
 * scratch vectors of the Riccati passes and the zero dual vector live in a
 * fixed, file-scope device array of 2^20 doubles (8 MiB) that every GPU which
 * loads the library holds until the process exits; x0_dev is read in place.
 * It calls no cudaMalloc or cudaFree.  The array's device address is looked
 * up by spock_problem_create (which allocates anyway), so the array is
 * brought onto the device there, before the first call of this function.
 *   Limit: 2 (n nx' + n_nonleaf nu') + n_eta <= 2^20 with nx', nu' the
 *   dimensions rounded up to even numbers; larger problems are
 *   rejected with SPOCK_ERR_INVALID_ARG and a message giving both sizes.
 *   All calls share the one array: calls that overlap on the GPU (other
 *   streams, other host threads) race and must be serialised by the caller.
 *   No buffer owned by the problem is written (except its error flag when a
 *   kernel reports a failure), so calls on one problem from other entry
 *   points do not race with it through the problem's buffers.
 *   The call synchronises `stream` before it returns (to read the kernels'
 *   error flag), so it cannot be captured into a CUDA graph.
 * Arguments, layout and other errors as spock_prox_f_dev.
 */
int spock_prox_f_noalloc_dev(spock_problem* p, const double* x0_dev, double alpha, const double* z,
                             double* z_out, void* stream);

/*
 * spock_grad_dev -- gradient of the optimal cost V* = s^0 with respect to
 * the problem data, from a converged pair (z, eta) = T(v*) (device buffers,
 * FP64, layout as above), e.g. the output of spock_solve_dev.
 * Method: at the saddle point of the Lagrangian
 *   s^0 + lambda^T (G z_1 - h) + mu^T M z_2 + <eta, L z> - g*(eta)
 * of the splitting (Sec. "Operator splitting": G z_1 = h the dynamics of S1,
 * M z_2 = 0 the kernel of S2, g* the conjugate of g of Eq. (g)), the
 * multipliers of the dynamics solve G^T lambda = -(L* eta)_{z_1} (one tree
 * recursion from the leaves on the stored [Abar | B] blocks) and the
 * derivative of V* in each datum is the Lagrangian's partial derivative
 * (envelope theorem):
 *   g_x0 = -lambda^0, g_A[c] = -lambda^c x^anc(c)T, g_B[c] = -lambda^c u^anc(c)T,
 *   g_Q[c][k] = eta_{c,Qx,k} x^anc(c)_k / (2 sqrt Q^c_kk), g_R likewise,
 *   g_QN[j][k] = eta_{j,QNx,k} x^j_k / (2 sqrt QN^j_kk).
 * Outputs (device, FP64, caller's node numbering; any may be NULL):
 *   g_x0 [nx], g_A [n][nx][nx], g_B [n][nx][nu], g_Q [n][nx], g_R [n][nu],
 *   g_QN [n][nx]; entries of nodes where a quantity does not exist are 0.
 * precision: SPOCK_FP64 or SPOCK_FP32 (arithmetic and factors of that
 * precision; inputs rounded).  Accuracy follows the accuracy of (z, eta).
 */
int spock_grad_dev(spock_problem* p, const double* z, const double* eta, int32_t precision, double* g_x0,
                   double* g_A, double* g_B, double* g_Q, double* g_R, double* g_QN, void* stream);

/*
 * spock_adjoint_dev -- gradient of phi(z*) = <g, z*> for any linear function
 * of the solution (g_z = NULL: phi = s^0, the optimal cost V*) with respect
 * to the problem data, by implicit differentiation of the CP fixed point
 * v* = T(v*) of Eq. (chambolle-pock-operator): the adjoint equation
 * (I - J^T) w = (g, 0) is solved by restarted GMRES(m) from w = 0 (m = 100,
 * or fewer -- at least 10 -- when the basis would take more than a quarter of
 * the free device memory at the first call; classical Gram-Schmidt with one
 * reorthogonalisation, deterministic reductions), J the
 * Jacobian of T at the converged pair (z, eta) (device buffers, FP64, e.g.
 * the output of spock_solve_dev).  J^T
 * is applied with the library's kernels: the Jacobians of the cone
 * projections of S3 at eta + alpha L z, L*, the Jacobian of prox_{alpha f}
 * (the homogeneous Riccati pass of Algorithm 2 and proj_S2) and L.  Then
 *   d phi/d x0    = mu^0,
 *   d phi/d A^c   = nu^c p_x^anc(c)T + mu^c x*^anc(c)T,  B^c likewise with u,
 *   d phi/d Q^c_kk = alpha (q_{c,Qx,k} x*^anc_k - eta_{c,Qx,k} p_{x^anc,k})
 *                    / (2 sqrt Q^c_kk),  R^c and Q_N^j likewise,
 * with q = B w_eta, r = w_z + 2 alpha L* q, p = (Jacobian of prox_f) r, mu and
 * nu the multipliers of the dynamics for r - p and for -alpha L* eta (tree
 * recursions on the stored factors).  For phi = s^0 the result equals
 * spock_grad_dev's (envelope theorem); for other phi (a component of the
 * first input u^0, say) it is the derivative of the solution map.
 *   g_z        : [n_z] device, the gradient of phi in z (NULL: e_{s^0}).
 *   max_iter, tol : the solve stops when the residual of the adjoint
 *                equation max|(g, 0) - (I - J^T) w| <= tol max(1, max|w|)
 *                (the true residual, checked at every restart; inside a
 *                cycle the GMRES residual estimate ends it early), or after
 *                max_iter applications of J^T.
 *   outputs    : as spock_grad_dev (device, FP64, caller's numbering, any
 *                may be NULL); iterations, residual (optional host pointers)
 *                receive the applications of J^T and the final relative
 *                residual.
 * Returns SPOCK_OK when the tolerance is met, SPOCK_MAX_ITER at the cap
 * (gradients written), SPOCK_ERR_NUMERICAL if the iteration diverges (the
 * fixed point must be one where T is differentiable and I - J^T invertible
 * on the data's directions).  Uses the problem's Riccati scratch: not
 * concurrent with solves on the same problem.  Device vectors (the Krylov
 * basis: m + 1 vectors of n_z + n_eta doubles, and about 12 more) are
 * allocated on the first call and kept by the problem.  Runs on the
 * problem's own stream after synchronising `stream` (one Arnoldi step is
 * captured into a CUDA graph and replayed).  Blocking.
 */
int spock_adjoint_dev(spock_problem* p, const double* z, const double* eta, const double* g_z, int32_t max_iter,
                      double tol, double* g_x0, double* g_A, double* g_B, double* g_Q, double* g_R, double* g_QN,
                      int32_t* iterations, double* residual, void* stream);

/*
 * spock_grad -- spock_grad_dev with host buffers: z [n_z] and eta [n_eta]
 * are copied to the device, the gradients (same layout as spock_grad_dev)
 * copied back into the non-NULL host outputs.  Device buffers for the
 * outputs are allocated on the first call and kept by the problem.
 * Blocking; errors as spock_grad_dev.
 */
int spock_grad(spock_problem* p, const double* z, const double* eta, int32_t precision, double* g_x0,
               double* g_A, double* g_B, double* g_Q, double* g_R, double* g_QN);

/*
 * spock_batch_create -- a batch of independent problems (any trees, depths,
 * nx, nu) solved together by spock_batch_solve_dev.  The problems stay owned
 * by the caller and must outlive the batch; a problem may belong to one
 * batch at a time and appears in it once (SPOCK_ERR_INVALID_ARG otherwise:
 * every instance needs its own iterate buffers).  n >= 1.
 */
int spock_batch_create(int32_t n, spock_problem* const* problems, spock_batch** out);

/*
 * spock_batch_solve_dev -- Algorithm 3 on every problem of the batch.
 * All instances advance together, round by round (decision, Anderson
 * update, next point, evaluation of T): each kernel of a round is launched
 * once for the whole batch, its blocks mapped to (instance, block of that
 * instance) by tables built once per batch, so a round costs the same
 * number of launches for 1 or 10,000 instances.  A fixed number of rounds
 * is captured into one CUDA graph; finished instances skip their work; the
 * host only reads the done flags after each graph launch.  When every
 * instance has nx + nu <= 62 (memory 0, 3 or 5), a second mode solves the
 * whole batch in one persistent launch, one thread block per instance; the
 * autotuner times both (SPOCK_BATCH_MODE = list / cta forces one).
 * Autotuner (before the first solve in a precision): the node tile of the
 * vector kernels (nodes per warp: 1, 2, 4, 8 or 16), the Riccati kernel
 * family (direct or staged) and the mode, each candidate timed over the
 * first evaluation of T and four rounds.  info.solve_ms and info.n_launches
 * describe the whole batch.
 *   x0_dev, z_dev, eta_dev : host arrays of n device pointers (FP64), per
 *     instance as in spock_solve_dev.
 *   settings : shared by all instances (alpha <= 0: each instance's own
 *     0.99/||L||); precision SPOCK_FP64 or SPOCK_FP32 (no FP64 tail here).
 *   infos    : optional host array of n outcomes.
 * Returns SPOCK_OK if every instance converged, SPOCK_MAX_ITER if some hit
 * the iteration cap (outputs written for all), or an error.  Blocking.
 */
int spock_batch_solve_dev(spock_batch* batch, const double* const* x0_dev, const spock_settings* settings,
                          double* const* z_dev, double* const* eta_dev, int32_t warm, spock_info* infos);

/*
 * spock_batch_solve -- spock_batch_solve_dev with host buffers: x0[i] [nx_i],
 * z_io[i] [n_z,i], eta_io[i] [n_eta,i] (host arrays of n host pointers, FP64).
 * The inputs are copied into each problem's device staging buffers (the
 * ones spock_solve uses; allocated on first use and kept by the problem),
 * the solutions copied back on SPOCK_OK and SPOCK_MAX_ITER.  Blocking.
 */
int spock_batch_solve(spock_batch* batch, const double* const* x0, const spock_settings* settings,
                      double* const* z_io, double* const* eta_io, int32_t warm, spock_info* infos);

/*
 * spock_fp64_fma_rate -- measures the FP64 fused multiply-add throughput of
 * the current device (TFLOP/s, two flops per FMA): the ALU roofline of the
 * SPOCK_FP64 path.  The paper has no counterpart; it is a measurement
 * utility.  Kernels of 4 or 8 blocks of 256 threads per SM, each thread
 * running 8 or 16 independent FMA chains (8 `iters` FMAs per thread), timed
 * with CUDA events on `stream` after a warm-up launch each; the best of the
 * four is returned.  Blocking.  Errors: INVALID_ARG (iters < 1 or NULL
 * output), CUDA, OOM.
 */
int spock_fp64_fma_rate(int32_t iters, double* tflops, void* stream);

/* Frees a handle returned by any *_create call; NULL is a no-op. */
void spock_free(void* handle);

/* Description of the last error raised on the calling thread ("" if none). */
const char* spock_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPOCK_H */
