// Tensor-core (tcgen05 / TMA) jet GEMMs for sm_103a.
#pragma once

#include "internal.h"

namespace pinn {

// Called once from pinn_create: resolves the driver entry point used to build
// TMA tensor maps.
void tc_init(pinn_handle* h);
// True when hidden layer li (0-based weight layer) runs on tensor cores.
bool tc_layer_supported(const pinn_handle* h, int li, int64_t NC);
// Bias partials per column tile written by the fused adjoint epilogue.
constexpr int TC_DB_PARTS = 2;   // bias partials per 64-point tile (epilogue warps per lane quadrant)
constexpr int TC_BN = 256;
// Number of K (column) splits of the tensor-core weight-gradient GEMM.
int tc_dw_splits(const pinn_handle* h, int fout, int fin, int64_t NC);

// Z = (W_hi + W_lo) A + W_hi A_lo (+ bias, tanh jet): W_hi, W_lo [fout][fin] BF16 (K-major),
// A^T [fin][NC], A_lo [fin][NC/4] the low half of A's value rows.
pinn_status tc_gemm_fwd(pinn_handle* h, const void* W, const void* Wlo, const void* A, const void* Alo, int fout,
                        int fin, int64_t NC, const EpiArgs& e, cudaStream_t st);
// Abar = W^T Zbar (tanh-jet adjoint epilogue): WT [fin][fout], Zbar^T [fout][NC].
pinn_status tc_gemm_adj(pinn_handle* h, const void* WT, const void* Zbar, int fin, int fout, int64_t NC,
                        const EpiArgs& e, cudaStream_t st);
// part[s] = Zbar^T A over column split s: Zbar^T [fout][NC], A^T [fin][NC] (both K-major).
pinn_status tc_gemm_dw(pinn_handle* h, const void* Zbar, const void* A, int fout, int fin, int64_t NC, int nsplit,
                       float* part, cudaStream_t st);

}  // namespace pinn
