// Per-point tanh jet rules shared by every GPU epilogue.
//
// A hidden layer applies g = tanh(f) elementwise (Sec. 2.2, Eq. 5).  With the
// input derivatives carried as jet rows, the chain rule gives, per feature,
//   a   = t,  a_k = t' z_k,  a_L = t'' * sum_{k in S} z_k^2 + t' z_L,
// with t = tanh(z), t' = 1 - t^2 = (1-t)(1+t), t'' = -2 t t', and S the directions
// of the second-order row (Burgers {x}, Navier-Stokes {x, y}).  Maxwell's fourth
// row is a plain first derivative (d/dt).  The adjoint (reverse mode through the
// same formulas, t''' = t'(6 t^2 - 2)) is
//   zbar_L = abar_L t'
//   zbar_k = abar_k t' + [k in S] 2 abar_L t'' z_k
//   zbar   = abar t' + sum_k abar_k t'' z_k + abar_L (t''' sum_{k in S} z_k^2 + t'' z_L).
#pragma once

#include "internal.h"

namespace pinn {

__device__ __forceinline__ float tanh_exact(float x) { return tanhf(x); }

__device__ __forceinline__ void jet_fwd(const float z[4], float a[4], int mode) {
  const float t = tanh_exact(z[0]);
  const float tp = (1.f - t) * (1.f + t);
  a[0] = t;
  a[1] = tp * z[1];
  a[2] = tp * z[2];
  if (mode == JET_MAXWELL) {
    a[3] = tp * z[3];
  } else {
    const float tpp = -2.f * t * tp;
    const float q = z[1] * z[1] + (mode == JET_NS ? z[2] * z[2] : 0.f);
    a[3] = fmaf(tpp, q, tp * z[3]);
  }
}

__device__ __forceinline__ void jet_adj(const float z[4], const float ab[4], float zb[4], int mode) {
  const float t = tanh_exact(z[0]);
  const float tp = (1.f - t) * (1.f + t);
  const float tpp = -2.f * t * tp;
  if (mode == JET_MAXWELL) {
    zb[1] = ab[1] * tp;
    zb[2] = ab[2] * tp;
    zb[3] = ab[3] * tp;
    zb[0] = fmaf(ab[0], tp, tpp * (ab[1] * z[1] + ab[2] * z[2] + ab[3] * z[3]));
  } else {
    const bool ns = (mode == JET_NS);
    const float tppp = tp * (6.f * t * t - 2.f);
    const float q = z[1] * z[1] + (ns ? z[2] * z[2] : 0.f);
    zb[3] = ab[3] * tp;
    zb[1] = fmaf(ab[1], tp, 2.f * ab[3] * tpp * z[1]);
    zb[2] = ns ? fmaf(ab[2], tp, 2.f * ab[3] * tpp * z[2]) : ab[2] * tp;
    zb[0] = fmaf(ab[0], tp, tpp * (ab[1] * z[1] + ab[2] * z[2])) + ab[3] * fmaf(tppp, q, tpp * z[3]);
  }
}

// Value-only column (initial/boundary point).
__device__ __forceinline__ float val_fwd(float z) { return tanh_exact(z); }
__device__ __forceinline__ float val_adj(float z, float ab) {
  const float t = tanh_exact(z);
  return ab * (1.f - t) * (1.f + t);
}

// ---- element type helpers ---------------------------------------------------------
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

}  // namespace pinn
