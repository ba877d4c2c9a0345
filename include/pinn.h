/*
 * pinn.h - C ABI of the GB300 PINN loss + gradient library (libpinn.so).
 *
 * The library computes, on one GPU, the physics-informed loss of a tanh MLP
 * over a batch of collocation points and its gradient with respect to the
 * network parameters, plus a fused Adam update.  What is computed follows the
 * paper (arXiv 2604.15645):
 *   - MLP layers f = W g + b, g = tanh(f), final layer linear (Sec. 2.2, Eqs. 4-6);
 *   - random Fourier features gamma(x) = [cos(xB), sin(xB)], B frozen (Sec. 2.6.1, Eq. 14);
 *   - random weight factorisation W = diag(exp(s)) V on every layer (Sec. 2.6.2, Eq. 15);
 *   - composite MSE loss, each term the mean over its own point set (Sec. 2.3,
 *     Eqs. 10-13) weighted by lambda_pde, lambda_ic, lambda_bc (Sec. 2.6.4, Eq. 17);
 *   - residuals of viscous Burgers (Sec. 4.3 with a viscosity term), steady
 *     incompressible Navier-Stokes (Sec. 4.4) and TE Maxwell, eps = mu = 1 (Sec. 4.8);
 *   - Adam (Sec. 2.6.5).
 * Input derivatives, which the paper takes with autograd, are carried as
 * per-point jets (value plus derivative rows) through every layer, and the
 * parameter gradient comes from a hand-written adjoint of those jets.
 *
 * Conventions for every entry point:
 *   - All pointers named d_* are DEVICE pointers owned by the caller; the library
 *     never frees them.  Host pointers are read during the call only.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *     void*; NULL = legacy default stream).  A call returns once the work is
 *     queued.
 *   - Argument errors are detected on the host and returned synchronously
 *     without queuing work.  Numerical faults found on the device (a non-finite
 *     loss, or a kernel wait that ran past its bound) are latched in a device
 *     status word and reported by pinn_status_poll().
 *   - After pinn_create() no call allocates device memory except the option
 *     setters that say so (pinn_set_periodic keeps its matrix; with pinn_set_graph
 *     the first call of each argument set captures and instantiates a CUDA graph):
 *     the caller provides the workspace (size from pinn_workspace_bytes()).
 *     Calls that do allocate return PINN_ERR_OOM when an allocation fails.
 *   - Every call that launches work must be made with the device the handle was
 *     created on current; otherwise it returns PINN_ERR_INVALID_ARG.
 *   - A handle is not thread-safe; one handle per host thread.
 */
#ifndef PINN_H
#define PINN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PINN_API __attribute__((visibility("default")))
#else
#define PINN_API
#endif

#define PINN_MAX_HIDDEN 16
#define PINN_LOSS_TERMS 8

typedef enum {
  PINN_OK = 0,
  PINN_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or spec field        */
  PINN_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement        */
  PINN_ERR_CUDA = 3,          /* a CUDA runtime/driver call failed                  */
  PINN_ERR_WORKSPACE = 4,     /* workspace smaller than pinn_workspace_bytes()      */
  PINN_ERR_NONFINITE = 5,     /* device saw a NaN/Inf loss (latched)                */
  PINN_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired (latched)       */
  PINN_ERR_OOM = 7            /* a host or device allocation the call makes failed  */
} pinn_status;

typedef enum {
  PINN_FP32 = 0,   /* jet GEMMs in FP32 on CUDA cores                            */
  PINN_TF32 = 1,   /* jet GEMMs on tensor cores, TF32 inputs, FP32 accumulation;
                      forward / adjoint add both truncation remainders (3 MMAs)  */
  PINN_BF16 = 2    /* jet GEMMs on tensor cores, BF16 inputs, FP32 accumulation  */
} pinn_precision;

typedef enum {
  PINN_BURGERS_1D = 0,     /* inputs (x,t),   output u;          r = u_t + u u_x - nu u_xx  */
  PINN_NS_STEADY_2D = 1,   /* inputs (x,y),   outputs (u,v,p);   momentum x, y + continuity */
  PINN_MAXWELL_TE_2D = 2,  /* inputs (x,y,t), outputs (Ez,Hx,Hy); TE curl equations       */
  PINN_ADVECTION_1D = 3,   /* inputs (x,t),   output u;          r = u_t + c u_x, c = nu (Sec. 4.1)      */
  PINN_ALLEN_CAHN_1D = 4   /* inputs (x,t),   output u;  r = u_t - nu u_xx + 5u^3 - 5u (Sec. 4.2)         */
} pinn_pde;

/* Network description (pinn_create).  d_in and d_out follow from `pde`
 * (Burgers 2->1, Navier-Stokes 2->3, Maxwell 3->3). */
typedef struct {
  int32_t pde;                       /* pinn_pde                                          */
  int32_t n_hidden;                  /* L, number of tanh layers, 1..PINN_MAX_HIDDEN      */
  int32_t widths[PINN_MAX_HIDDEN];   /* widths[0..L-1], each 1..2048                      */
  int32_t ff_m;                      /* Fourier frequencies m (embedding width 2m), 0=none */
  int32_t rwf;                       /* 1: every layer is W = diag(exp(s)) V (Eq. 15)     */
  int32_t precision;                 /* pinn_precision of the hidden-layer jet GEMMs      */
  int32_t flags;                     /* PINN_FLAG_* bits, 0 = defaults                    */
} pinn_spec;

/* pinn_spec.flags: run every jet GEMM on CUDA cores even where tcgen05 kernels
 * apply (the many-network autotuner picks per network between the two). */
#define PINN_FLAG_CUDA_CORES 1

/* pinn_spec.flags, BF16 only: split the weights into BF16 high and low halves for
 * the value rows only.  By default the tensor-core forward adds W_lo . A on every jet
 * row (two full MMAs plus the value-row low half).  With this flag the derivative
 * rows use W_hi alone, which makes the forward 1.25 instead of 2.25 MMAs per K step
 * at a larger derivative-row error.  Use it where the BF16 error budget allows:
 * the Navier-Stokes cavity networks stay near 1e-2, while Burgers networks whose
 * residual terms cancel need the full split. */
#define PINN_FLAG_BF16_VALUE_SPLIT 4
/* (flag value 2 is reserved) */

/* pinn_spec.flags, kernel variants (same results up to rounding; the many-network
 * autotuner picks among them per network shape):
 *   PINN_FLAG_UNFUSED_ADJOINT  run every layer's adjoint and weight gradient as two
 *                              kernels even where the fused kernel applies (BF16,
 *                              fan-out <= 256);
 *   PINN_FLAG_DW_ROWS_128      weight-gradient tiles of 128 output rows (default: 256
 *                              rows, two accumulators sharing each staged operand, for
 *                              layers with more than 256 outputs). */
#define PINN_FLAG_UNFUSED_ADJOINT 8
#define PINN_FLAG_DW_ROWS_128 16

/* Loss weights and the PDE coefficient (nu for Burgers; 1/Re for Navier-Stokes;
 * ignored for Maxwell). */
typedef struct {
  double nu;
  double lambda_pde, lambda_ic, lambda_bc;
} pinn_problem;

/* One batch of collocation points.  Coordinates are SoA FP32 device arrays
 * [d_in][n] (coordinate-major, n contiguous); targets are [d_out][n].  Bit c of a
 * mask constrains output c on that set.  A set with n = 0 or mask = 0 adds no
 * term.  Pointers of empty sets may be NULL. */
typedef struct {
  const float* x_res; int64_t n_res;
  const float* x_ic;  const float* g_ic; int64_t n_ic; uint32_t ic_mask;
  const float* x_bc;  const float* g_bc; int64_t n_bc; uint32_t bc_mask;
} pinn_batch;

typedef struct pinn_handle pinn_handle;

/* Validate `spec`, compute the packed parameter layout and allocate the handle
 * (host metadata plus a 256-byte device status word).  The parameter vector is
 * packed per layer l = 1..L+1 as  V_l [fan_out x fan_in, row-major] | s_l [fan_out]
 * (only if rwf) | b_l [fan_out];  the first fan_in is 2m with Fourier features,
 * else d_in.  Returns PINN_ERR_INVALID_ARG for a bad spec. */
PINN_API pinn_status pinn_create(const pinn_spec* spec, pinn_handle** out);

/* Free the handle and its status word.  NULL is accepted. */
PINN_API pinn_status pinn_destroy(pinn_handle* h);

/* Number of FP32 entries P in the packed parameter (and gradient) vector. */
PINN_API pinn_status pinn_param_count(const pinn_handle* h, int64_t* P);

/* Bytes of device workspace one call on a batch of these sizes needs (jets of
 * every layer, adjoints, split reduction partials).  With point chunking
 * (pinn_set_chunk_points) it is the size of one chunk's pass plus a small staging
 * area, independent of the batch size beyond one chunk. */
PINN_API pinn_status pinn_workspace_bytes(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc,
                                 size_t* bytes);

/* Point chunking: process a batch in consecutive chunks of at most `points`
 * collocation points (rounded up to a multiple of 64; 0 = one pass over the whole
 * batch, the default).  Points are taken in the order interior, initial, boundary.
 * Each chunk runs the whole forward and reverse sweep; loss sums and the gradient
 * accumulate over chunks in a fixed order, with every mean normalised by the
 * batch's full point counts, so the result equals the one-pass result up to
 * rounding and is deterministic.  Peak workspace then stays at one chunk's size for
 * any batch.  Negative `points` is PINN_ERR_INVALID_ARG. */
PINN_API pinn_status pinn_set_chunk_points(pinn_handle* h, int64_t points);

/* Shard of a larger batch (data parallelism without a collective in the library):
 * normalise every mean by these global point counts instead of the batch's own, so a
 * call on one slice of the points returns that slice's share of each loss term and of
 * the gradient.  Summing the shares over the slices (for instance an all-reduce the
 * caller performs across ranks) gives the whole batch's loss and gradient, up to
 * rounding.  All zero switches it off.  Negative counts are PINN_ERR_INVALID_ARG; a
 * later call on a batch larger than the counts is PINN_ERR_INVALID_ARG, and with
 * temporal causality on it is PINN_ERR_UNSUPPORTED (the weights need every segment). */
PINN_API pinn_status pinn_set_global_counts(pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc);

/* CUDA-graph replay (on = 1; 0 = off, the default).  With it on, pinn_loss,
 * pinn_loss_grad, pinn_loss_grad_ff and pinn_loss_grad_terms capture their whole launch
 * sequence into a CUDA graph on the first call (on a stream the handle owns) and
 * replay it on the caller's stream while every argument (pointers, sizes, problem
 * values, stream) and every handle setting stays the same; any change captures
 * again.  The result is the same as without the graph; the host cost of a step drops
 * to one graph launch.  Calls with phase profiling on (pinn_set_profiling) run
 * without the graph.  Capture or instantiation failures return PINN_ERR_CUDA. */
PINN_API pinn_status pinn_set_graph(pinn_handle* h, int on);

/* *held = 1 if the handle currently holds an instantiated CUDA graph (pinn_set_graph),
 * else 0.  An inspection hook with no counterpart in the paper. */
PINN_API pinn_status pinn_graph_held(const pinn_handle* h, int32_t* held);

/* Hidden-layer activation: PINN_ACT_TANH (the default, Eq. 5) or PINN_ACT_SINE, the
 * periodic activation sin(omega0 z) of Sec. 2.6 (Table 1), in every hidden layer.
 * A sine network keeps each hidden layer's pre-activation jets for the adjoint (one
 * more FP32 [w_l][4 N] array per layer, counted by pinn_workspace_bytes), because
 * the sign of cos(omega0 z) cannot be recovered from the stored sin.  BF16 sine
 * networks run their hidden jet GEMMs on tcgen05 tensor cores (separate adjoint and
 * weight-gradient kernels); TF32 sine networks compute in FP32 on CUDA cores.
 * Unknown `act`, or omega0 not finite and > 0: PINN_ERR_INVALID_ARG. */
#define PINN_ACT_TANH 0
#define PINN_ACT_SINE 1
PINN_API pinn_status pinn_set_activation(pinn_handle* h, int act, double omega0);

/* Temporal causality (Sec. 2.6.8, Eqs. 20-21) for time-dependent problems: the time
 * domain [t0, t1] is cut into `segments` equal segments (1..32; 0 switches it off);
 * an interior point at time t belongs to segment floor((t - t0)/(t1 - t0) * M),
 * clamped.  The PDE term becomes L_pde = (1/M) sum_i omega_i L^i, with L^i the mean
 * squared residual (summed over equations) of segment i's points, omega_1 = 1 and
 * omega_i = exp(-eps sum_{k<i} L^k).  The weights are evaluated from the current
 * parameters and held constant in the gradient (stop-gradient); each call computes
 * them with an extra output-layer pass before the seeds.  Time is input 1 (x, t) or
 * input 2 (Maxwell x, y, t); the steady Navier-Stokes problem is
 * PINN_ERR_UNSUPPORTED.  Causality with point chunking is PINN_ERR_UNSUPPORTED
 * (the weights need every segment first). */
PINN_API pinn_status pinn_set_causal(pinn_handle* h, int segments, double eps, double t0, double t1);

/* The weights omega_i of the last loss call with causality on, FP64 device [segments]. */
PINN_API pinn_status pinn_causal_weights(pinn_handle* h, double* d_weights, void* stream);

/* Register the frozen Fourier-feature matrix B, FP32 device [d_in][m] (Eq. 14).
 * Required before any loss call when ff_m > 0.  The pointer is kept, not copied. */
PINN_API pinn_status pinn_set_ff_matrix(pinn_handle* h, const float* d_B);

/* Strict periodic input map (Sec. 2.6.3, Eq. 16) for a network with ff_m = d_in:
 * the input is mapped to [cos(2 pi x_k / P_k) for k..., sin(2 pi x_k / P_k) for k...],
 * i.e. the Fourier embedding with B = diag(2 pi / P) held by the handle (a device
 * copy is made here; no pinn_set_ff_matrix needed).  This is the paper's map up to
 * the order of the first layer's input columns (the paper interleaves cos and sin per
 * input).  `periods` is a host array [d_in] of finite values > 0; anything else, or
 * ff_m != d_in, is PINN_ERR_INVALID_ARG.  pinn_set_ff_matrix switches back to a
 * caller-owned B. */
PINN_API pinn_status pinn_set_periodic(pinn_handle* h, const double* periods);

/* pinn_loss_grad plus the gradient with respect to the input map: with a Fourier
 * matrix, d_grad_ff receives dL/dB, FP32 device [d_in][m] (Eq. 14 treated as
 * trainable); with the periodic map it receives dL/dP, FP32 device [d_in], the
 * gradient with respect to the periods (the paper trains P_t).  It is computed from
 * the adjoint of the input jets, W_1^T Zbar_1, by CUDA-core kernels after the first
 * layer's weight gradient; FP64 block partials are summed in a fixed order.  With
 * point chunking it accumulates over chunks like the parameter gradient.  A network
 * without Fourier features, or d_grad_ff NULL, is PINN_ERR_INVALID_ARG. */
PINN_API pinn_status pinn_loss_grad_ff(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch,
                                       const float* d_params, void* d_ws, size_t ws_bytes, double* d_loss_terms,
                                       float* d_grad, float* d_grad_ff, void* stream);

/* Loss only: the composite MSE loss of Sec. 2.3 (Eqs. 10-13) with the weights of
 * Sec. 2.6.4 (Eq. 17), over the network of Sec. 2.2 (Eqs. 4-6) with the optional
 * Fourier embedding (Eq. 14) and weight factorisation (Eq. 15); each residual is the
 * PDE of `spec.pde` (Sec. 4.1-4.4, 4.8) evaluated from the input derivatives that
 * the paper takes by autograd (Sec. 2.3).  d_loss_terms receives PINN_LOSS_TERMS
 * doubles:
 *   [0] total = lambda_pde*L_pde + lambda_ic*L_ic + lambda_bc*L_bc
 *   [1] L_pde (sum over equations)  [2..4] L_pde per equation (unused = 0)
 *   [5] L_ic   [6] L_bc   [7] 0
 * d_params: FP32 [P] in the packed layout of pinn_create.  d_ws: at least
 * pinn_workspace_bytes(), 256-byte aligned, caller-owned; its contents on entry do
 * not matter.  d_loss_terms: FP64 device [8], overwritten.  Errors: NULL pointers,
 * a misaligned workspace, an empty batch, masks naming missing outputs or a missing
 * Fourier matrix are PINN_ERR_INVALID_ARG; a workspace smaller than needed is
 * PINN_ERR_WORKSPACE; a launch failure is PINN_ERR_CUDA.  Nothing is queued on error. */
PINN_API pinn_status pinn_loss(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch,
                      const float* d_params, void* d_ws, size_t ws_bytes,
                      double* d_loss_terms, void* stream);

/* Loss (as pinn_loss) and its gradient dL/dtheta with respect to every packed
 * parameter: the paper obtains it by differentiating the autograd input derivatives
 * once more (Sec. 2.3, double backward); here it comes from the hand-written adjoint
 * of the jets, then the factorisation's chain rule dV = exp(s) dW,
 * ds_i = sum_j dW_ij W_ij (Eq. 15).  d_grad: FP32 device [P], packed like d_params,
 * overwritten.  Reductions over points are ordered and done in FP64, so repeated
 * calls on the same inputs give bitwise identical results.  Workspace, ownership and
 * errors as pinn_loss; a NULL d_grad is PINN_ERR_INVALID_ARG. */
PINN_API pinn_status pinn_loss_grad(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch,
                           const float* d_params, void* d_ws, size_t ws_bytes,
                           double* d_loss_terms, float* d_grad, void* stream);

/* Per-term gradients for loss balancing (Sec. 2.6.4): the loss as pinn_loss_grad
 * (d_loss_terms, weighted total with prob's lambdas), and in d_grad_terms FP32
 * [3][P] the unweighted gradients dL_pde/dtheta, dL_ic/dtheta, dL_bc/dtheta
 * (overwritten).  One forward sweep feeds three reverse sweeps, each seeded with
 * weight 1 on its term and 0 on the others; so sum_i lambda_i d_grad_terms[i] equals
 * pinn_loss_grad's gradient up to rounding.  Workspace and chunking as
 * pinn_loss_grad. */
PINN_API pinn_status pinn_loss_grad_terms(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch,
                                          const float* d_params, void* d_ws, size_t ws_bytes,
                                          double* d_loss_terms, float* d_grad_terms, void* stream);

/* Loss-balancing weights (Sec. 2.6.4, Eqs. 18-19), on the device: the L2 norms
 * n_i = |d_grad_terms[i]| (FP64, fixed reduction order) go to d_norms [3] (may be
 * NULL); if `update`, lambda_hat_i = (n_pde + n_ic + n_bc) / (n_i + eps) and
 * d_lambda[i] = alpha d_lambda[i] + (1 - alpha) lambda_hat_i, for i in (pde, ic, bc)
 * with n_i > 0 (a term without points keeps its weight).  d_lambda: FP64 device [3],
 * in/out.  The paper updates with alpha = 0.9 and eps = 1e-9 every 1000 steps: the
 * caller picks the steps with `update`.  alpha outside [0, 1] or negative eps is
 * PINN_ERR_INVALID_ARG. */
PINN_API pinn_status pinn_loss_balance(pinn_handle* h, const float* d_grad_terms, double* d_lambda, double* d_norms,
                                       double alpha, double eps, int update, void* stream);

/* ---- L-BFGS refinement (Sec. 2.6.5, Eqs. 22-26) ----------------------------------
 * A pinn_lbfgs keeps the last `history` pairs s_k = theta_{k+1} - theta_k,
 * y_k = g_{k+1} - g_k on the device (2 history P floats plus five P-vectors, allocated
 * by pinn_lbfgs_create).  The direction p = -H g is the two-loop recursion (initial
 * matrix gamma I, gamma = s.y / y.y of the newest pair), with every scalar an FP64
 * fixed-order reduction kept on the device. */
typedef struct pinn_lbfgs pinn_lbfgs;
PINN_API pinn_status pinn_lbfgs_create(pinn_handle* h, int history, pinn_lbfgs** out);   /* history 1..64 */
PINN_API pinn_status pinn_lbfgs_destroy(pinn_lbfgs* lb);
/* Forget the pairs and the cached gradient (e.g. after the parameters were changed
 * outside pinn_lbfgs_step). */
PINN_API pinn_status pinn_lbfgs_reset(pinn_lbfgs* lb);
/* One step: the direction from the history, a backtracking line search (Eq. 26)
 * taking the first lambda in 1, 1/2, 1/4, ... (at most 30 trials) with
 * L(theta + lambda p) <= L(theta) + 1e-4 lambda g.p (the last trial is taken if none
 * passes), the gradient at the new point, and the new pair when s.y > 0.  A
 * non-descent direction restarts from -g with an empty history.  d_params is
 * updated in place; *loss_out (host, may be NULL) receives the new loss and
 * *backtracks_out (host, may be NULL) the number of halvings.  Synchronises
 * `stream` once per line-search trial to read the loss. */
PINN_API pinn_status pinn_lbfgs_step(pinn_lbfgs* lb, const pinn_problem* prob, const pinn_batch* batch,
                                     float* d_params, void* d_ws, size_t ws_bytes, double* loss_out,
                                     int* backtracks_out, void* stream);
/* Test hooks: p = -H g from the current history (d_g, d_p device [P]); append a pair. */
PINN_API pinn_status pinn_lbfgs_direction(pinn_lbfgs* lb, const float* d_g, float* d_p, void* stream);
PINN_API pinn_status pinn_lbfgs_push_pair(pinn_lbfgs* lb, const float* d_s, const float* d_y, void* stream);

/* One Adam step in place over n entries (Sec. 2.6.5): m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, theta -= lr * (m/(1-b1^step)) / (sqrt(v/(1-b2^step)) + eps).
 * step is 1-based.  All four arrays FP32 device [n]. */
PINN_API pinn_status pinn_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t n,
                           int64_t step, float lr, float beta1, float beta2, float eps, void* stream);

/* Synchronise `stream`, then read and clear the device status word: PINN_OK,
 * PINN_ERR_NONFINITE or PINN_ERR_TIMEOUT. */
PINN_API pinn_status pinn_status_poll(pinn_handle* h, void* stream);

/* Last error message recorded on the handle (never NULL). */
PINN_API const char* pinn_last_error(const pinn_handle* h);

/* Static name of a status code. */
PINN_API const char* pinn_status_string(pinn_status s);

/* Phase profiler.  While enabled, every loss call brackets each launch group
 * with CUDA events on the caller's stream (no synchronisation inside the call).
 * Phases: 0 RWF weights, 1 input embedding / first layer, 2 forward jet GEMMs,
 * 3 output layer + residual + loss, 4 weight-gradient GEMMs, 5 adjoint GEMMs,
 * 6 reductions and finalisation, 7 other, 8 fused adjoint + weight-gradient GEMMs
 * (pinn_layer_engines, engine 2).  At most 16384 event pairs are kept between reads;
 * later ones are dropped (and counted in launches of the last phase as -1). */
#define PINN_PROF_PHASES 9
PINN_API pinn_status pinn_set_profiling(pinn_handle* h, int enable);

/* Synchronise on the recorded events, then return per phase the summed GPU time
 * in milliseconds and the number of kernel launches since the last read, and
 * reset the record.  Both arrays have PINN_PROF_PHASES entries. */
PINN_API pinn_status pinn_profile_read(pinn_handle* h, double* ms, int64_t* launches);

/* Number of hidden layers whose jet GEMMs run on tcgen05 tensor cores for a batch
 * of these sizes (the rest run on CUDA cores), written to *n. */
PINN_API pinn_status pinn_tensor_core_layers(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc,
                                             int32_t* n);

/* The engine of every hidden layer's jet GEMMs for a batch of these sizes, written to
 * engines[0..L-1]: 0 CUDA cores; 1 tensor cores (separate forward, adjoint and
 * weight-gradient kernels); 2 tensor cores with the layer's adjoint and weight
 * gradient fused into one kernel (BF16, fan-out <= 256, every layer but the first). */
PINN_API pinn_status pinn_layer_engines(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc,
                                        int32_t* engines);

/* Self-test of the tensor-core GEMM core (no PINN arithmetic): FP32 output, all
 * device pointers.  "Tile-major" is the library's jet-matrix layout: a logical
 * [R][C] matrix stored as [C/256][R][256].
 *   kind 0: D = A B (+ A2 B when d_A2 != NULL), A, A2 [M][K] row-major, B [K][N]
 *           and D [M][N] tile-major (the forward / adjoint layout); N % 256 == 0.
 *   kind 1: D = A B^T, A [M][K] and B [N][K] tile-major (the weight-gradient
 *           layout), D [M][N] row-major; K % 256 == 0.
 *   kinds 0, 1: BF16 inputs (kind::f16 MMA); kind 3: the kind-1 layout with FP32
 *           inputs that the tensor cores read as TF32 (kind::tf32 MMA).  Kind 2
 *           (TF32 with an MN-major operand) returns PINN_ERR_UNSUPPORTED.
 * M, N, K multiples of 8.  Synchronises `stream`; returns PINN_ERR_TIMEOUT if a
 * bounded device wait expired.  No counterpart in the paper: a test hook. */
PINN_API pinn_status pinn_tc_selftest(int kind, int M, int N, int K, const void* d_A, const void* d_A2,
                                      const void* d_B, float* d_D, void* stream);

/* Test hook for failure detection, with no counterpart in the paper: the kind-0 BF16
 * self-test GEMM (d_A [M][K] row-major, d_B [K][N] tile-major, d_D [M][N] FP32;
 * N % 256 == 0, M and K multiples of 8) launched with its MMA-issuing thread first
 * waiting on an mbarrier that no thread ever arrives on, with every wait bounded by
 * wait_us microseconds (1..2,000,000).  The wait expires, the kernel latches
 * PINN_ERR_TIMEOUT in h's status word, stops its other roles, waits (bounded) for its
 * own copies in flight, frees its tensor memory and returns; d_D is left partly or
 * wholly unwritten.  Asynchronous on `stream`; pinn_status_poll(h) then reports
 * PINN_ERR_TIMEOUT and clears it, and the context stays usable. */
PINN_API pinn_status pinn_debug_wait_expiry(pinn_handle* h, int M, int N, int K, const void* d_A, const void* d_B,
                                            float* d_D, int64_t wait_us, void* stream);

/* ---- many independent networks in one training step --------------------------------
 * A pinn_multi holds one network handle per spec (uneven widths, depths and point
 * counts allowed).  pinn_multi_train_step runs, for every network, the loss and
 * gradient of its own batch and problem (as pinn_loss_grad), then one Adam step
 * (Sec. 2.6.5) over the concatenation of all parameter vectors.  The first call with
 * a given set of buffers captures the whole step in a CUDA graph; later calls replay
 * it, updating only the Adam scalars.  By default each network's launch sequence runs
 * on one of up to 32 parallel worker streams.  With pinn_multi_set_grouped(m, 1) the
 * step runs all networks level by level instead: at each layer level one grouped
 * tcgen05 launch per kernel variant covers that level's tensor-core GEMMs of every
 * network (each GEMM with the CTAs and work split of its own launch, so the results
 * are bitwise those of separate launches), and the other launches of the level run on
 * the worker streams.  Parameters, gradients and Adam moments are single FP32
 * device vectors laid out by pinn_multi_param_offsets (network i owns
 * [offsets[i], offsets[i+1])).  d_loss receives PINN_LOSS_TERMS doubles per network.
 * The workspace (pinn_multi_workspace_bytes) serves both GEMM engines, so
 * pinn_multi_set_engine / pinn_multi_autotune never require a new one.  Not
 * thread-safe; the graph keeps the buffers it was captured with alive by address. */
typedef struct pinn_multi pinn_multi;

PINN_API pinn_status pinn_multi_create(const pinn_spec* specs, int32_t n_nets, pinn_multi** out);
PINN_API pinn_status pinn_multi_destroy(pinn_multi* m);
/* n_nets + 1 offsets into the concatenated parameter vector. */
PINN_API pinn_status pinn_multi_param_offsets(const pinn_multi* m, int64_t* offsets);
PINN_API pinn_status pinn_multi_workspace_bytes(pinn_multi* m, const pinn_batch* batches, size_t* bytes);
PINN_API pinn_status pinn_multi_set_ff_matrix(pinn_multi* m, int32_t net, const float* d_B);
/* Kernel configuration of network `net` (same results up to rounding):
 *   0 tcgen05, fused adjoint + weight gradient where it applies (the default);
 *   1 CUDA-core GEMMs;
 *   2 tcgen05 with separate adjoint and weight-gradient kernels (PINN_FLAG_UNFUSED_ADJOINT);
 *   3 as 2 with 128-row weight-gradient tiles (PINN_FLAG_DW_ROWS_128).
 * Anything else is PINN_ERR_INVALID_ARG. */
PINN_API pinn_status pinn_multi_set_config(pinn_multi* m, int32_t net, int32_t config);
PINN_API pinn_status pinn_multi_get_config(const pinn_multi* m, int32_t net, int32_t* config);
/* cuda_cores = 1 forces the CUDA-core GEMMs for network `net` (configuration 1), 0 the
 * default tcgen05 configuration 0. */
PINN_API pinn_status pinn_multi_set_engine(pinn_multi* m, int32_t net, int32_t cuda_cores);
PINN_API pinn_status pinn_multi_get_engine(const pinn_multi* m, int32_t net, int32_t* cuda_cores);
/* on = 1: grouped launches per layer level, as above; on = 0 (the default): each
 * network's launch sequence (pinn_loss_grad's launches) on its worker stream, the
 * networks side by side.  Both give bitwise the same step.  The grouped step keeps a
 * level's data of all networks in flight at once, where the per-network sequences
 * read each layer's input while the layer below has just left it in L2, and it waits
 * for the slowest network at every level: on the 64-network Burgers family it is the
 * slower of the two on one GB300 (measured).  A change takes effect
 * with the next pinn_multi_train_step, which captures a new graph.  A bounded wait
 * that expires inside a grouped launch is reported (PINN_ERR_TIMEOUT, through
 * pinn_multi_status_poll) on the network whose GEMM the waiting CTA was running. */
PINN_API pinn_status pinn_multi_set_grouped(pinn_multi* m, int32_t on);
PINN_API pinn_status pinn_multi_get_grouped(const pinn_multi* m, int32_t* on);
/* One training step (1-based `step`); asynchronous on `stream` except for graph
 * (re)capture on the first call with new buffers, which also synchronises `stream`
 * and may allocate (the grouped launches' device table). */
PINN_API pinn_status pinn_multi_train_step(pinn_multi* m, const pinn_problem* probs, const pinn_batch* batches,
                                           float* d_params, float* d_grad, float* d_m, float* d_v, int64_t step,
                                           float lr, float beta1, float beta2, float eps, void* d_ws,
                                           size_t ws_bytes, double* d_loss, void* stream);
/* Times every kernel configuration that applies to a network (keyed by width, depth,
 * power-of-two point bucket and precision), selects the fastest, and reads / writes
 * the choices as a JSON object in `cache_path` (NULL: no file).  Runs eagerly and
 * synchronises.  The training step spreads the networks over up to 32 worker
 * streams, longest first by estimated jet-GEMM work. */
PINN_API pinn_status pinn_multi_autotune(pinn_multi* m, const pinn_problem* probs, const pinn_batch* batches,
                                         const float* d_params, void* d_ws, size_t ws_bytes, double* d_loss,
                                         float* d_grad, const char* cache_path, void* stream);
PINN_API pinn_status pinn_multi_status_poll(pinn_multi* m, void* stream);
PINN_API const char* pinn_multi_last_error(const pinn_multi* m);

/* Test hook: the tanh used by the BF16 epilogues, t = tanh(z) and tp = 1 - tanh(z)^2,
 * computed from e = exp(-2|z|) as t = sign(z)(1-e)/(1+e), tp = 4e/(1+e)^2, for n
 * FP32 device values.  Asynchronous on `stream`.  No counterpart in the paper. */
PINN_API pinn_status pinn_tanh_selftest(int64_t n, const float* d_z, float* d_t, float* d_tp, void* stream);

/* Size of the scratch array compiled into the library for pinn_loss_grad_static. */
#define PINN_STATIC_WS_BYTES ((size_t)64 << 20)

/* Loss and gradient exactly as pinn_loss_grad, for callers that cannot allocate
 * device memory (code in host callbacks or real-time loops where an allocation may
 * block or fail, plug-ins whose host runtime owns the memory pool, processes with a
 * memory budget fixed at start-up) and so cannot provide a workspace.  The paper
 * has no counterpart: this is a library-interface convenience.
 *   - Scratch is a 64 MiB (PINN_STATIC_WS_BYTES) file-scope __device__ array inside
 *     libpinn.so; every GPU that loads the library holds it until process exit.
 *   - A batch whose pinn_workspace_bytes() exceeds that size is rejected with
 *     PINN_ERR_WORKSPACE (message in pinn_last_error) and nothing is queued.
 *   - The call allocates nothing (no cudaMalloc/cudaFree or allocating library call).
 *     It always launches eagerly: a handle with pinn_set_graph on captures no graph
 *     here (capturing and instantiating one would allocate), and the graph it may
 *     hold for its other calls is left as it is.
 *   - The handle's device must be current (else PINN_ERR_INVALID_ARG).  Every call
 *     looks up the array's device address on it (cudaGetSymbolAddress, no
 *     allocation), so a device whose context was reset gets the new address.  The
 *     first call on a device, and the first after such a reset, makes the CUDA
 *     runtime load the library's device code there, which reserves the array: make
 *     that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents; every value
 *     a call reads is written earlier in the same call.  Calls whose GPU work
 *     overlaps (e.g. on two streams) race on the array. */
PINN_API pinn_status pinn_loss_grad_static(pinn_handle* h, const pinn_problem* prob, const pinn_batch* batch,
                                           const float* d_params, double* d_loss_terms, float* d_grad,
                                           void* stream);

/* Library version string. */
PINN_API const char* pinn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PINN_H */
