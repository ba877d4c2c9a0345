// Tensor-core (tcgen05 / TMA) jet GEMMs for sm_103a.
#pragma once

#include <cuda.h>

#include "internal.h"

namespace pinn {

// Called once from pinn_create: resolves the driver entry point used to build
// TMA tensor maps.
void tc_init(pinn_handle* h);
// 3-D TMA tensor map over a tile-major jet matrix [ntiles][rows][tcols] (BF16, or FP32
// when fp32), box [1][box_rows][box_cols], 128-byte swizzle, zero fill out of bounds.
// False if the driver entry point is missing or the encoding fails.
bool tc_map3(CUtensorMap* m, const void* base, bool fp32, uint64_t tcols, uint64_t rows, uint64_t ntiles,
             uint32_t box_cols, uint32_t box_rows);
// True when hidden layer li (0-based weight layer) runs on tensor cores.
bool tc_layer_supported(const pinn_handle* h, int li, int64_t NC);
// Bias partials per column tile written by the fused adjoint epilogue.
constexpr int TC_DB_PARTS = 2;   // bias partials per 64-point tile (epilogue warps per lane quadrant)
constexpr int TC_BN = 256;
// Number of K (column) splits of the tensor-core weight-gradient GEMM.
int tc_dw_splits(const pinn_handle* h, int fout, int fin, int64_t NC);

// Forward (+ bias, tanh jet), W_hi, W_lo [fout][fin] (K-major).
//   BF16: Z = (W_hi + W_lo) A + W_hi A_lo, A^T [fin][NC] tile-major, A_lo [fin][NC/4]
//         the low half of A's value rows.
//   TF32: Z = (W_hi + W_lo) A + W_hi (A - tf32(A)), A point-major [NC][fin]; Alo unused;
//         the epilogue also writes e.out_pm (point-major A_l) when set.
pinn_status tc_gemm_fwd(pinn_handle* h, const void* W, const void* Wlo, const void* A, const void* Alo, int fout,
                        int fin, int64_t NC, const EpiArgs& e, cudaStream_t st);
// Abar = W^T Zbar (tanh-jet adjoint epilogue), WT [fin][fout].
//   BF16: Zbar^T [fout][NC] tile-major, high halves only (WTlo unused).
//   TF32: (WT_hi + WT_lo) Zbar + WT_hi (Zbar - tf32(Zbar)), Zbar point-major [NC][fout];
//         the epilogue also writes e.out_pm when set.
pinn_status tc_gemm_adj(pinn_handle* h, const void* WT, const void* WTlo, const void* Zbar, int fin, int fout,
                        int64_t NC, const EpiArgs& e, cudaStream_t st);
// part[s] = Zbar^T A over column split s: Zbar^T [fout][NC], A^T [fin][NC] (both K-major).
pinn_status tc_gemm_dw(pinn_handle* h, const void* Zbar, const void* A, int fout, int fin, int64_t NC, int nsplit,
                       float* part, cudaStream_t st);

// Fused adjoint + weight gradient (BF16, hidden layer li >= 1 on tensor cores with
// fan-out <= 256): one kernel computes Abar = W^T Zbar with the tanh-jet adjoint
// epilogue (as tc_gemm_adj) and dW^T = A_{l-1} Zbar^T, written as tc_adjdw_splits()
// partials [nsplit][fout][fin] (as tc_gemm_dw).  Ain is A_{l-1}^T [fin][NC] tile-major.
bool tc_adjdw_supported(const pinn_handle* h, int li, int64_t NC);
int tc_adjdw_splits(const pinn_handle* h, int fin, int64_t NC);
pinn_status tc_gemm_adjdw(pinn_handle* h, const void* WT, const void* Zbar, const void* Ain, int fin, int fout,
                          int64_t NC, const EpiArgs& e, float* dwpart, int nsplit, cudaStream_t st);

// ---- grouped launches ---------------------------------------------------------------
// A batch collects the tensor-core GEMMs that attached handles would launch and issues
// them as grouped launches, one per kernel variant: each GEMM keeps the CTA count and
// work split of its own launch (so its results are bitwise those of that launch), and
// the CTAs of all GEMMs share one grid, the GEMMs with the most work first.  Each
// grouped launch reads its GEMMs' tensor maps and parameters from a device table.
struct TcBatch;
TcBatch* tc_batch_create();
void tc_batch_destroy(TcBatch* b);
// Routes the tensor-core launches of h into b (nullptr: launch them directly again).
void tc_batch_attach(pinn_handle* h, TcBatch* b);
// Forgets the collected GEMMs and the table built so far.
void tc_batch_reset(TcBatch* b);
// Makes room for `entries` table entries on the device (cudaMalloc: not under capture).
pinn_status tc_batch_reserve(TcBatch* b, size_t entries);
// Issues the GEMMs collected since the last flush on st (errors are reported on h).
// The launches read table entries that tc_batch_upload writes: upload before the
// launches run (for a captured graph: after the capture, before the first replay).
pinn_status tc_batch_flush(TcBatch* b, pinn_handle* h, cudaStream_t st);
// Copies the table to the device (synchronous).
pinn_status tc_batch_upload(TcBatch* b);
// Grouped launches issued since the last reset.
int tc_batch_launches(const TcBatch* b);

}  // namespace pinn
