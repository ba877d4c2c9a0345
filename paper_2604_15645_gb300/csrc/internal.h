// Internal declarations of libpinn: handle, workspace plan and kernel launchers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/pinn.h"

namespace pinn {

struct TcBatch;   // grouped tensor-core launches (tc.h)

// Jet rows per point: r=0 value, r=1,2 first derivatives, r=3 either a
// second-order row (Burgers d2/dx2, Navier-Stokes Laplacian) or a third first
// derivative (Maxwell d/dt).  The column layout (tiles of 64 points, blocked by
// row) is described in jet.cuh.
constexpr int R = 4;
// Points are padded to a multiple of this (one 256-column tile).
constexpr int PT_ALIGN = 64;

enum JetMode : int {
  JET_BURGERS = 0,  // rows [u, d/dx, d/dt, d2/dx2]; second-order set S = {x}
  JET_NS = 1,       // rows [u, d/dx, d/dy, Laplacian]; S = {x, y}
  JET_MAXWELL = 2   // rows [u, d/dx, d/dy, d/dt]; no second-order row
};

struct LayerPlan {
  int fin = 0, fout = 0;
  int64_t off_V = 0, off_s = -1, off_b = 0;   // offsets into the packed parameter vector
  // workspace offsets (bytes)
  size_t w32 = 0;      // W fp32 [fout][fin]
  size_t wc = 0;       // W in compute type [fout][fin]
  size_t wtc = 0;      // W^T in compute type [fin][fout]
  size_t wt32 = 0;     // W^T fp32 [fin][fout]
  size_t wlo = 0;      // W - hi(W) in the compute type [fout][fin] (second half of the split weight)
  size_t wtlo = 0;     // its transpose [fin][fout] (TF32 adjoint)
  size_t dwpart = 0;   // dW split partials fp32 [nsplit][fout][fin]
  size_t dbpart = 0;   // db partials fp32 [nbpart][fout]
  int nsplit = 1;
};

struct Plan {
  int64_t n_res = 0, n_ic = 0, n_bc = 0;
  int64_t ncols = 0;   // 4 (n_res + n_ic + n_bc): columns of real points
  int64_t NP = 0;      // points padded to PT_ALIGN
  int64_t NC = 0;      // 4 NP
  int es = 4;          // bytes per element of the compute type (2 bf16, 4 fp32/tf32)
  bool lo = false;     // BF16 / TF32: value rows also keep a low half in Alo
  int lo_es = 2;       // bytes per low-half element (BF16 2, TF32 4)
  size_t A[PINN_MAX_HIDDEN + 1] = {};   // A_l^T [w_l][NC] compute type, l = 0..L (A_0 only with FF)
  size_t Alo[PINN_MAX_HIDDEN + 1] = {}; // low half of the value rows, tile-major [NP/64][w_l][64]
  size_t Z[PINN_MAX_HIDDEN + 1] = {};   // sine activation only: pre-activations Z_l^T [w_l][NC] FP32
  size_t Zbar[2] = {};                  // ping-pong adjoints [w_max][NC] compute type
  size_t losspart = 0;                  // per-block loss partials, double [nloss_blocks][8]
  size_t segpart = 0;                   // causality: per-block segment sums [nloss_blocks][CAUSAL_MAX][4]
  size_t ffpart = 0;                    // Fourier features: dL/dB block partials, double [m][FFG_BLOCKS][d_in]
  int nloss_blocks = 0;
  int nbpart = 0;                       // column chunks of the bias/first-layer reductions
  size_t total = 0;
};

}  // namespace pinn

// Everything a captured step depends on: the call's arguments and the handle's
// settings.  Zero-filled before use so that memcmp also covers the padding.
struct pinn_graph_key {
  int kind;                  // 0 loss, 1 loss+grad, 2 loss+grad+input map, 3 per-term grads
  pinn_problem prob;
  pinn_batch batch;
  const void* params; void* ws; size_t ws_bytes; void* loss; void* grad; void* out2;
  int64_t chunk_points;
  int global_counts; int64_t g_res, g_ic, g_bc;
  int causal_M; double causal_eps, causal_t0, causal_t1;
  int act; float omega0;
  const float* ff_B; int periodic; double periods[3];
  void* stream;
};

struct pinn_handle {
  pinn_spec spec{};
  int d_in = 0, d_out = 0, L = 0;
  int jet_mode = 0;
  int first_gemm = 0;        // index of the first hidden layer computed by a GEMM (0 with FF, 1 without)
  int64_t P = 0;
  int w_max = 0;
  pinn::LayerPlan layers[PINN_MAX_HIDDEN + 1];
  const float* ff_B = nullptr;
  int* d_status = nullptr;   // device status word (bit 0 nonfinite, bit 1 timeout)
  double* d_scratch = nullptr;  // small device scratch (loss balancing; causal weights), allocated at create
  int causal_M = 0;          // temporal causality: segments (0 off), decay, time domain
  double causal_eps = 0.0, causal_t0 = 0.0, causal_t1 = 1.0;
  int device = 0;
  int sm_count = 0;
  int64_t chunk_points = 0;  // 0: one pass; else points per chunk (multiple of 64)
  bool global_counts = false; // normalise the means by these counts (a shard of a larger batch)
  int64_t g_res = 0, g_ic = 0, g_bc = 0;
  float* d_periodic_B = nullptr;   // periodic input map: owned diag(2 pi / P) [d_in][d_in]
  bool periodic = false;     // ff_B is d_periodic_B; the input-map gradient is dL/dP
  double periods[3] = {0, 0, 0};
  // CUDA-graph replay of whole calls (pinn_set_graph): the last captured call and its key
  bool graph_on = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  pinn_graph_key graph_key{};
  int act = PINN_ACT_TANH;   // hidden activation; sine keeps Z and runs on CUDA cores
  pinn::TcBatch* tc_batch = nullptr;   // set: tensor-core GEMMs are collected for a grouped launch
  float omega0 = 1.f;
  char err[512] = {0};
  // phase profiler (pinn_set_profiling)
  bool prof = false;
  int prof_n = 0;
  int prof_dropped = 0;
  cudaEvent_t* prof_ev = nullptr;   // 2 * PROF_MAX events
  int* prof_phase = nullptr;
  int* prof_launches = nullptr;
};

namespace pinn {

pinn_status make_plan(const pinn_handle* h, int64_t n_res, int64_t n_ic, int64_t n_bc, Plan* plan);

// ---- kernel launchers (defined in the .cu files) ------------------------------------
struct RwfArgs {
  const float* params; char* ws; int L1; int rwf; int prec;
  int fin[PINN_MAX_HIDDEN + 1], fout[PINN_MAX_HIDDEN + 1];
  int64_t offV[PINN_MAX_HIDDEN + 1], offs[PINN_MAX_HIDDEN + 1];
  size_t w32[PINN_MAX_HIDDEN + 1], wc[PINN_MAX_HIDDEN + 1], wtc[PINN_MAX_HIDDEN + 1];
  size_t wt32[PINN_MAX_HIDDEN + 1], wlo[PINN_MAX_HIDDEN + 1], wtlo[PINN_MAX_HIDDEN + 1];
};
void launch_rwf_prep(const RwfArgs& a, cudaStream_t st);

void launch_embed_ff(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                     int64_t n_bc, int d_in, const float* B, int m, int jet_mode, void* A0, void* A0lo, int64_t NP,
                     int prec, cudaStream_t st);

void launch_first_layer(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                        int64_t n_bc, int d_in, const float* W, const float* b, int fout, int jet_mode, void* A1,
                        void* A1lo, int64_t NP, int prec, float omega0, float* Z1, cudaStream_t st);

struct EpiArgs {
  const float* bias;      // fwd: bias of this layer [M]
  void* out;              // fwd: A_l^T, adj: Zbar_{l-1}^T (compute type)
  void* alo_out;          // fwd, BF16: low half of A_l's value rows [M][NP] (else nullptr)
  const void* alo_in;     // fwd, CUDA-core BF16 path: low half of the input's value rows [K][NP]
  const void* ain;        // adj: A_{l-1}^T (compute type), the output jet of the layer below
  const void* ain_lo;     // adj, BF16: low half of its value rows [NP/64][M][64] (t = hi + lo)
  void* out_pm;           // TF32 tensor-core path: point-major copy of `out`, [NC][M] FP32 (nullptr = none)
  int jet_mode;
  // sine activation (CUDA-core path): fwd writes the pre-activation jets to zout,
  // adj reads them from zin ([M][NC] FP32, tile-major); act 0 = tanh.
  int act;
  float omega0;
  float* zout;
  const float* zin;
  // tensor-core forward / adjoint: visit the column tiles last to first, so a kernel
  // starts on the tiles its predecessor touched last (still in L2)
  int reverse;
  // adjoint only: bias-gradient partials of the layer whose pre-activation adjoint
  // this epilogue writes ([part][M][1 + dterms]; nullptr = not fused), and for a
  // first layer on raw coordinates the coordinate terms of its dW (dterms = d_in).
  float* dbpart;
  int dterms;
  const float* x_res; const float* x_ic; const float* x_bc;
  int64_t n_res, n_ic, n_bc;
};

// D[M][4 NP] = Aop[M][K] Bop[K][4 NP] (+ epilogue), Aop row-major ld=K (FP32 weights),
// Bop row-major (activations in the compute type).
void launch_simt_gemm_fwd(const float* Aop, const void* Bop, int M, int K, int64_t NP, const EpiArgs& e, int prec,
                          cudaStream_t st);
void launch_simt_gemm_adj(const float* Aop, const void* Bop, int M, int K, int64_t NP, const EpiArgs& e, int prec,
                          cudaStream_t st);
// out[M][4 NP] = Aop[M][K] Bop[K][4 NP] with no epilogue (the input-jet adjoint W_1^T Zbar_1).
void launch_simt_gemm_lin(const float* Aop, const void* Bop, int M, int K, int64_t NP, void* out, int prec,
                          cudaStream_t st);
// part[s][M][N] = sum_{k in split s} Aop[m][k] Bop[n][k]; Aop/Bop row-major with ld = NC.
// a_fp32 / b_fp32 select float storage, else the compute type.
void launch_simt_gemm_dw(const void* Aop, bool a_fp32, const void* Bop, bool b_fp32, int M, int N, int64_t NC,
                         int nsplit, float* part, int prec, cudaStream_t st);

struct OutArgs {
  const void* AL;        // A_L^T [w][NC] compute type
  const void* ALlo;      // BF16: low half of A_L's value rows [w][NP] (else nullptr)
  const float* W;        // output weights fp32 [d_out][w]
  const float* b;        // output bias [d_out]
  const float* g_ic; const float* g_bc;   // targets [d_out][n]
  uint32_t ic_mask, bc_mask;
  int64_t n_res, n_ic, n_bc, NP, NC;
  int w, d_out, pde, jet_mode;
  float nu;
  float k_pde, k_ic, k_bc;  // 2 lambda / N per set (adjoint seed scale)
  int want_grad;
  // temporal causality (Sec. 2.6.8): segment of an interior point from its time input
  int segments;          // 0: off
  const float* x_res;    // interior coordinates [d_in][n_res] (for the time input)
  int t_index;           // which input is time
  float t0, tinv;        // segment = floor((t - t0) * tinv), tinv = M / (t1 - t0)
  double* segpart;       // phase 1: per-block segment sums [nblocks][CAUSAL_MAX][4] (3 equations + count)
  const float* seg_scale;  // phase 2: per-segment seed scale lambda omega_i / (M N_i), replacing k_pde
  float* dwpart;         // output-layer dW partials [nblocks][d_out][w] (per block, fixed order)
  float* dbpart;         // output-layer bias partials [d_out][nblocks]
  float* dbhid;          // last hidden layer's bias partials [w][nblocks] (value rows of Zbar_L), or nullptr
  void* Zbar;            // Zbar_L^T [w][NC] compute type
  const float* ZL;       // sine activation: Z_L^T [w][NC] FP32 for the adjoint (else nullptr)
  int reverse;           // visit the point tiles last to first
  float omega0;
  double* losspart;      // [nblocks][8]
  int* status;
};
// Output layer, residuals, loss partials and (want_grad) the adjoint seeds, Zbar_L
// and the output layer's dW and bias partials, one block per 64-point tile stride.
// dL/dB of the Fourier embedding (Eq. 14) from the input-jet adjoint Abar_0 [2m][NC]
// (compute type): per-block FP64 partials, then an ordered sum into out [d_in][m]
// (accumulating when `accumulate`), or, for the periodic map (Eq. 16, B = diag(2 pi/P)),
// out[k] = dL/dP_k = -(2 pi / P_k^2) dL/dB_kk.
constexpr int FFG_BLOCKS = 32;
void launch_ff_grad(const void* Abar0, const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res,
                    int64_t n_ic, int64_t n_bc, int d_in, const float* B, int m, int jet_mode, int64_t NP,
                    double* part, int prec, cudaStream_t st);
void launch_ff_grad_final(const double* part, int d_in, int m, bool periodic, const double* periods, int accumulate,
                          float* out, cudaStream_t st);
cudaError_t launch_out_loss(const OutArgs& a, int prec, int nblocks, cudaStream_t st);
int out_loss_blocks(int64_t n_points);
// The output/loss kernel with A_L staged by TMA (BF16 tanh networks, last hidden width
// <= 512) runs two blocks per SM; its block count (the number of loss, dW and bias
// partials) is out_loss_tma_blocks.
bool out_loss_tma_ok(int prec, int act, int w);
int out_loss_tma_blocks(int64_t n_points, int sm_count);

// Bias gradient partials of a layer from its pre-activation adjoint (value rows
// only), plus, for a first layer applied to raw coordinates, the coordinate terms
// of dW.  part [M][nbpart][1 + d_in_terms].  `fp32_in` reads the adjoint as FP32.
void launch_row_reduce(const void* Zbar, bool fp32_in, int M, int64_t NP, int64_t n_res, int64_t n_ic, int64_t n_bc,
                       int nbpart, const float* x_res, const float* x_ic, const float* x_bc, int d_in_terms,
                       int jet_mode, float* part, int prec, cudaStream_t st);

struct FinalizeArgs {
  const float* params; float* grad; char* ws; int L1; int rwf;
  int fin[PINN_MAX_HIDDEN + 1], fout[PINN_MAX_HIDDEN + 1];
  int64_t offV[PINN_MAX_HIDDEN + 1], offs[PINN_MAX_HIDDEN + 1], offb[PINN_MAX_HIDDEN + 1];
  size_t w32[PINN_MAX_HIDDEN + 1], dwpart[PINN_MAX_HIDDEN + 1], dbpart[PINN_MAX_HIDDEN + 1];
  int nsplit[PINN_MAX_HIDDEN + 1];
  int nbpart_l[PINN_MAX_HIDDEN + 1];   // bias partial count per layer
  int dbstride[PINN_MAX_HIDDEN + 1];   // floats per (part, row) in dbpart: 1, or 1 + d_in for a raw-coordinate first layer
  int first_raw;                        // 1: layer 0 takes raw coordinates (its dW comes from dbpart too)
  int nbpart;
  int accumulate;                       // 1: add into grad (later point chunks) instead of overwriting
};
void launch_finalize_grad(const FinalizeArgs& a, cudaStream_t st);
// acc: 5 running FP64 sums carried across point chunks (first: start from zero;
// last: normalise by the full counts and write `out`, else store the sums in acc).
void launch_finalize_loss(const double* losspart, int nblocks, int64_t n_res, int64_t n_ic, int64_t n_bc,
                          double lam_pde, double lam_ic, double lam_bc, double* out, double* acc, int first, int last,
                          int* status, cudaStream_t st);
// Loss balancing (Sec. 2.6.4): L2 norms of the three term gradients [3][P] (FP64,
// fixed order), lambda_hat_i = sum_j |g_j| / (|g_i| + eps) over the terms whose gradient
// is nonzero, and (update) lambda = alpha lambda + (1 - alpha) lambda_hat.
// part: 3 x 64 doubles of scratch.
void launch_loss_balance(const float* g, int64_t P, double* lambda, double* norms, double alpha, double eps,
                         int update, double* part, cudaStream_t st);
// Temporal causality (Sec. 2.6.8, Eqs. 20-21): segment losses from the output/loss
// kernel's segment partials (fixed order), the weights omega_i (written to omega), the
// causally weighted loss terms (out[8], with the IC/BC terms from losspart) and the
// per-segment seed scales lam_seed omega_i / (M N_i) (scale, for the second pass).
constexpr int CAUSAL_MAX = 32;
void launch_finalize_causal(const double* segpart, const double* losspart, int nblocks, int M, double eps,
                            int64_t n_ic, int64_t n_bc, double lam_pde, double lam_ic, double lam_bc, double lam_seed,
                            double* out, double* omega, float* scale, int* status, cudaStream_t st);
// Ordered compaction of S split partials [S][n] into S2 [S2][n] (out may not alias in).
void launch_sum_splits(const float* in, float* out, int S, int S2, int64_t n, cudaStream_t st);
constexpr int OUT_SUM_SLOTS = 16;   // output-layer dW partials after compaction
// Tile-major [w][NC] FP32 -> point-major [NC][w] (TF32 tensor-core operand layout).
void launch_to_point_major(const void* src, void* dst, int w, int64_t NC, cudaStream_t st);

void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, cudaStream_t st);

// pinn_loss_grad without CUDA-graph capture or replay, whatever pinn_set_graph says
// (the launch sequence only; it allocates nothing).
pinn_status loss_grad_eager(pinn_handle* h, const pinn_problem* prob, const pinn_batch* b, const float* d_params,
                            void* d_ws, size_t ws_bytes, double* d_loss, float* d_grad, void* stream);

// The stages of one whole-batch loss + gradient pass (the launch sequence of
// pinn_loss_grad split where the many-network step interleaves networks): the
// prologue (RWF weights, input jets), forward levels 0 .. staged_forward_levels()-1
// (one hidden GEMM each), the output/loss stage, backward levels 0 .. L-1 (hidden
// layer L-1 first), and the gradient finalisation.  Run in that order on one stream
// they enqueue exactly pinn_loss_grad's launches.  staged_create validates like
// pinn_loss_grad and refuses point chunking (PINN_ERR_UNSUPPORTED).
struct StagedPass;
pinn_status staged_create(pinn_handle* h, const pinn_problem* prob, const pinn_batch* b, const float* d_params,
                          void* d_ws, size_t ws_bytes, double* d_loss, float* d_grad, StagedPass** out);
void staged_destroy(StagedPass* sp);
int staged_forward_levels(const StagedPass* sp);
pinn_status staged_prologue(StagedPass* sp, cudaStream_t st);
pinn_status staged_forward(StagedPass* sp, int level, cudaStream_t st);
pinn_status staged_output(StagedPass* sp, cudaStream_t st);
pinn_status staged_backward(StagedPass* sp, int level, cudaStream_t st);
pinn_status staged_finalize(StagedPass* sp, cudaStream_t st);

}  // namespace pinn
