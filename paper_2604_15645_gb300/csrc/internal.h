// Internal declarations of libpinn: handle, workspace plan and kernel launchers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/pinn.h"

namespace pinn {

// Jet rows per interior point.  Column 4p+r of every activation matrix holds
// row r of point p: r=0 value, r=1,2 first derivatives, r=3 either a second-order
// row (Burgers d2/dx2, Navier-Stokes Laplacian) or a third first derivative
// (Maxwell d/dt).  Initial/boundary points take one (value) column each, after
// all interior columns.
constexpr int R = 4;
// Column tiles are multiples of this; the jet matrices are padded to it.
constexpr int COL_ALIGN = 256;

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
  size_t wlo = 0;      // BF16 only: W - bf16(W) rounded to bf16 [fout][fin] (second half of the split weight)
  size_t dwpart = 0;   // dW split partials fp32 [nsplit][fout][fin]
  size_t dbpart = 0;   // db partials fp32 [nbpart][fout]
  int nsplit = 1;
};

struct Plan {
  int64_t n_res = 0, n_ic = 0, n_bc = 0;
  int64_t ncols = 0;   // 4 n_res + n_ic + n_bc
  int64_t NC = 0;      // ncols padded to COL_ALIGN
  int es = 4;          // bytes per element of the compute type (2 bf16, 4 fp32/tf32)
  size_t A[PINN_MAX_HIDDEN + 1] = {};   // A_l^T [w_l][NC] compute type, l = 0..L (A_0 only with FF)
  size_t Z[PINN_MAX_HIDDEN + 1] = {};   // Z_l^T [w_l][NC] compute type, l = 1..L
  size_t Zbar[2] = {};                  // ping-pong adjoints [w_max][NC] compute type
  size_t Ubar = 0;                      // output seeds [d_out][NC] fp32
  size_t losspart = 0;                  // per-block loss partials, double [nloss_blocks][8]
  int nloss_blocks = 0;
  int nbpart = 0;                       // column chunks of the bias/first-layer reductions
  size_t total = 0;
};

}  // namespace pinn

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
  int device = 0;
  int sm_count = 0;
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
  size_t wt32[PINN_MAX_HIDDEN + 1], wlo[PINN_MAX_HIDDEN + 1];
};
void launch_rwf_prep(const RwfArgs& a, cudaStream_t st);

void launch_embed_ff(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                     int64_t n_bc, int d_in, const float* B, int m, int jet_mode, void* A0, int64_t NC, int prec,
                     cudaStream_t st);

void launch_first_layer(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                        int64_t n_bc, int d_in, const float* W, const float* b, int fout, int jet_mode, void* A1,
                        void* Z1, int64_t NC, int prec, cudaStream_t st);

struct EpiArgs {
  const float* bias;      // fwd: bias of this layer [M]
  void* out;              // fwd: A_l^T, adj: Zbar_{l-1}^T (compute type)
  void* zout;             // fwd: Z_l^T (compute type)
  const void* zin;        // adj: Z_{l-1}^T (compute type)
  int64_t n_res4;         // 4 n_res: columns below it are jet columns
  int64_t ncols;          // valid columns
  int jet_mode;
  // adjoint only: bias-gradient partials of the layer whose pre-activation adjoint
  // this epilogue writes ([part][M][1 + dterms]; nullptr = not fused), and for a
  // first layer on raw coordinates the coordinate terms of its dW (dterms = d_in).
  float* dbpart;
  int dterms;
  const float* x_res; const float* x_ic; const float* x_bc;
  int64_t n_res, n_ic, n_bc;
};

// D[M][N] = Aop[M][K] Bop[K][N] (+ epilogue), Aop row-major ld=K (FP32 weights),
// Bop row-major ld=NC (activations in the compute type).
void launch_simt_gemm_fwd(const float* Aop, const void* Bop, int M, int K, int64_t NC, const EpiArgs& e, int prec,
                          cudaStream_t st);
void launch_simt_gemm_adj(const float* Aop, const void* Bop, int M, int K, int64_t NC, const EpiArgs& e, int prec,
                          cudaStream_t st);
// part[s][M][N] = sum_{k in split s} Aop[m][k] Bop[n][k]; Aop/Bop row-major with ld = NC.
// a_fp32 / b_fp32 select float storage, else the compute type.
void launch_simt_gemm_dw(const void* Aop, bool a_fp32, const void* Bop, bool b_fp32, int M, int N, int64_t NC,
                         int nsplit, float* part, int prec, cudaStream_t st);

struct OutArgs {
  const void* AL;        // A_L^T [w][NC] compute type
  const void* ZL;        // Z_L^T [w][NC] compute type
  const float* W;        // output weights fp32 [d_out][w]
  const float* b;        // output bias [d_out]
  const float* g_ic; const float* g_bc;   // targets [d_out][n]
  uint32_t ic_mask, bc_mask;
  int64_t n_res, n_ic, n_bc, NC;
  int w, d_out, pde, jet_mode;
  float nu;
  float k_pde, k_ic, k_bc;  // 2 lambda / N per set (adjoint seed scale)
  int want_grad;
  float* Ubar;           // [d_out][NC]
  void* Zbar;            // Zbar_L^T [w][NC] compute type
  double* losspart;      // [nblocks][8]
  int* status;
};
void launch_out_loss(const OutArgs& a, int prec, int nblocks, cudaStream_t st);
// Output-layer weight gradient dW_out[c][f] = sum_col Ubar[c][col] A_L[f][col],
// partials [nchunks][d_out][w].
void launch_dw_out(const void* AL, const float* Ubar, int w, int d_out, int64_t NC, int nchunks, float* part,
                   int prec, cudaStream_t st);
int out_loss_blocks(int64_t n_points);

// Bias gradient partials of a layer from its pre-activation adjoint (value
// columns only), plus, for a first layer applied to raw coordinates, the
// coordinate terms of dW.  part [nbpart][M][1 + d_in_terms].
void launch_row_reduce(const void* Zbar, int M, int64_t NC, int64_t n_res, int64_t ncols, int nbpart,
                       const float* x_res, const float* x_ic, const float* x_bc, int64_t n_ic, int64_t n_bc,
                       int d_in_terms, int jet_mode, float* part, int prec, cudaStream_t st);

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
};
void launch_finalize_grad(const FinalizeArgs& a, cudaStream_t st);
void launch_finalize_loss(const double* losspart, int nblocks, int64_t n_res, int64_t n_ic, int64_t n_bc,
                          double lam_pde, double lam_ic, double lam_bc, double* out, int* status, cudaStream_t st);
void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, cudaStream_t st);

}  // namespace pinn
