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
// The epilogues evaluate it from the layer's output jet a instead of z: substituting
// z_k = a_k / t' and z_L = (a_L - t'' sum z_k^2) / t', every 1/t' cancels
// (t'''/t' - t''^2/t'^2 = -2), leaving, with t = a and t' = (1 - t)(1 + t),
//   zbar_L = abar_L t'
//   zbar_k = abar_k t' - [k in S] 4 abar_L t a_k
//   zbar   = abar t' - 2 t sum_k abar_k a_k - 2 abar_L (sum_{k in S} a_k^2 + t a_L).
// So the forward stores A only (it feeds the next layer and the weight gradient
// anyway), not Z.
#pragma once

#include <cstring>

#include "internal.h"

namespace pinn {

__device__ __forceinline__ float tanh_exact(float x) { return tanhf(x); }

// tanh and its derivative from the exponential form: with e = exp(-2|z|),
//   tanh z = sign(z) (1 - e) / (1 + e),   tanh' z = sech^2 z = 4 e / (1 + e)^2.
// One fast exponential and one fast reciprocal; both t and t' keep a relative
// error of a few 1e-7 for every z, including saturated units where 1 - t^2 would
// cancel.  Used by the BF16 path, whose storage rounding is ~4e-3.
__device__ __forceinline__ void tanh_fast(float z, float& t, float& tp) {
  const float e = __expf(-2.f * fabsf(z));
  const float r = __fdividef(1.f, 1.f + e);
  t = copysignf((1.f - e) * r, z);
  tp = 4.f * e * r * r;
}

template <bool FAST>
__device__ __forceinline__ void tanh_pair(float z, float& t, float& tp) {
  if (FAST) {
    tanh_fast(z, t, tp);
  } else {
    t = tanh_exact(z);
    tp = (1.f - t) * (1.f + t);
  }
}

template <bool FAST = false>
__device__ __forceinline__ void jet_fwd(const float z[4], float a[4], int mode) {
  float t, tp;
  tanh_pair<FAST>(z[0], t, tp);
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

// The same adjoint from the output jet a (see the header comment); no tanh evaluation.
__device__ __forceinline__ void jet_adj_a(const float a[4], const float ab[4], float zb[4], int mode) {
  const float t = a[0];
  const float tp = (1.f - t) * (1.f + t);
  if (mode == JET_MAXWELL) {
    zb[1] = ab[1] * tp;
    zb[2] = ab[2] * tp;
    zb[3] = ab[3] * tp;
    zb[0] = fmaf(ab[0], tp, -2.f * t * (ab[1] * a[1] + ab[2] * a[2] + ab[3] * a[3]));
  } else {
    const bool ns = (mode == JET_NS);
    const float q = a[1] * a[1] + (ns ? a[2] * a[2] : 0.f);
    const float t4 = 4.f * ab[3] * t;
    zb[3] = ab[3] * tp;
    zb[1] = fmaf(ab[1], tp, -t4 * a[1]);
    zb[2] = ns ? fmaf(ab[2], tp, -t4 * a[2]) : ab[2] * tp;
    zb[0] = fmaf(ab[0], tp, -2.f * (t * (ab[1] * a[1] + ab[2] * a[2]) + ab[3] * fmaf(t, a[3], q)));
  }
}

// ---- periodic activation sin(omega z) ----------------------------------------------
// The sine activation (periodic activation function, Sec. 2.6) uses the same jet rule
// with t = sin(w z), t' = w cos(w z), t'' = -w^2 sin(w z), t''' = -w^3 cos(w z).  Its
// adjoint cannot be written in A alone (the sign of cos is lost in sin), so sine
// layers keep their pre-activation jets Z and evaluate the adjoint from z:
//   zbar_L = abar_L t'
//   zbar_k = abar_k t' + [k in S] 2 abar_L t'' z_k
//   zbar   = abar t' + t'' sum_k abar_k z_k + abar_L (t''' sum_{k in S} z_k^2 + t'' z_L),
// and for Maxwell's first-order fourth row zbar = abar t' + t'' sum_k abar_k z_k.
__device__ __forceinline__ void jet_fwd_sine(const float z[4], float a[4], int mode, float w) {
  float s, c;
  sincosf(w * z[0], &s, &c);
  const float tp = w * c;
  a[0] = s;
  a[1] = tp * z[1];
  a[2] = tp * z[2];
  if (mode == JET_MAXWELL) {
    a[3] = tp * z[3];
  } else {
    const float tpp = -w * w * s;
    const float q = z[1] * z[1] + (mode == JET_NS ? z[2] * z[2] : 0.f);
    a[3] = fmaf(tpp, q, tp * z[3]);
  }
}

__device__ __forceinline__ void jet_adj_sine(const float z[4], const float ab[4], float zb[4], int mode, float w) {
  float s, c;
  sincosf(w * z[0], &s, &c);
  const float tp = w * c, tpp = -w * w * s, tppp = -w * w * tp;
  if (mode == JET_MAXWELL) {
    zb[1] = ab[1] * tp;
    zb[2] = ab[2] * tp;
    zb[3] = ab[3] * tp;
    zb[0] = fmaf(ab[0], tp, tpp * (ab[1] * z[1] + ab[2] * z[2] + ab[3] * z[3]));
  } else {
    const bool ns = (mode == JET_NS);
    const float q = z[1] * z[1] + (ns ? z[2] * z[2] : 0.f);
    const float t2 = 2.f * ab[3] * tpp;
    zb[3] = ab[3] * tp;
    zb[1] = fmaf(ab[1], tp, t2 * z[1]);
    zb[2] = ns ? fmaf(ab[2], tp, t2 * z[2]) : ab[2] * tp;
    // sum_k abar_k z_k over the two first-order rows, plus abar_L's second-order terms
    const float g1 = ab[1] * z[1] + ab[2] * z[2];
    zb[0] = fmaf(ab[0], tp, fmaf(tpp, g1, ab[3] * fmaf(tppp, q, tpp * z[3])));
  }
}

// ---- geometry of the jet matrices ------------------------------------------------------
// Every point (interior, initial, boundary, padding) owns four columns.  Points are
// grouped in tiles of 64; inside a 256-column tile the columns are blocked by jet
// row: [64 values | 64 first rows | 64 second rows | 64 fourth rows].  Column of
// row r of point p:  256 * (p / 64) + 64 * r + p % 64.  Interior points come
// first, then initial, then boundary points, then padding up to a multiple of 64.
// Initial/boundary points only have a value row: their three derivative rows are
// zero and stay exactly zero through every layer (and so do their adjoints).
constexpr int TILE_PTS = 64;
constexpr int TILE_COLS = 256;

__host__ __device__ __forceinline__ int64_t jcol(int64_t p, int r) {
  return ((p >> 6) << 8) + ((int64_t)r << 6) + (p & 63);
}

// Storage is tile-major: a jet matrix with w feature rows is [NP/64][w][256], so
// the 256 columns of one tile and one feature are contiguous and a whole tile
// (w x 256) is one contiguous block.  Element offset of (feature f, column c):
__host__ __device__ __forceinline__ int64_t toff(int64_t f, int64_t c, int64_t w) {
  return (((c >> 8) * w + f) << 8) + (c & 255);
}
// The BF16 low half of the value rows is [NP/64][w][64]; offset of (f, point p):
__host__ __device__ __forceinline__ int64_t loff(int64_t f, int64_t p, int64_t w) {
  return (((p >> 6) * w + f) << 6) + (p & 63);
}

enum PointSet : int { SET_RES = 0, SET_IC = 1, SET_BC = 2, SET_PAD = 3 };

__device__ __forceinline__ int point_set(int64_t p, int64_t n_res, int64_t n_ic, int64_t n_bc, int64_t& idx) {
  if (p < n_res) { idx = p; return SET_RES; }
  if (p < n_res + n_ic) { idx = p - n_res; return SET_IC; }
  if (p < n_res + n_ic + n_bc) { idx = p - n_res - n_ic; return SET_BC; }
  idx = 0;
  return SET_PAD;
}

// Coordinate j of point p (0 for padding).
__device__ __forceinline__ float point_coord(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res,
                                             int64_t n_ic, int64_t n_bc, int64_t p, int j) {
  int64_t idx;
  const int s = point_set(p, n_res, n_ic, n_bc, idx);
  if (s == SET_RES) return x_res[(int64_t)j * n_res + idx];
  if (s == SET_IC) return x_ic[(int64_t)j * n_ic + idx];
  if (s == SET_BC) return x_bc[(int64_t)j * n_bc + idx];
  return 0.f;
}

// Input direction of jet row r (1..3), or -1 for a second-order row.
__device__ __forceinline__ int row_dir(int mode, int r) { return (mode == JET_MAXWELL || r < 3) ? r - 1 : -1; }

// TF32 keeps the top 19 bits of an FP32 value (1 sign, 8 exponent, 10 mantissa);
// the tensor cores read FP32 operands that way.  The remainder x - trunc(x) is exact
// in FP32 and is the low half the TF32 path adds back where precision matters.
__host__ __device__ __forceinline__ float tf32_trunc(float x) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  u &= 0xFFFFE000u;
  float y;
  memcpy(&y, &u, 4);
  return y;
#endif
}

// ---- element type helpers ---------------------------------------------------------
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T>
__device__ __forceinline__ void store4(T* p, const float v[4]);
template <>
__device__ __forceinline__ void store4<float>(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16* p, const float v[4]) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t*>(&lo);
  u.y = *reinterpret_cast<uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(p) = u;
}
template <typename T>
__device__ __forceinline__ void load4(const T* p, float v[4]);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float v[4]) {
  float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void load4<__nv_bfloat16>(const __nv_bfloat16* p, float v[4]) {
  uint2 u = *reinterpret_cast<const uint2*>(p);
  __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162*>(&u.x);
  __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162*>(&u.y);
  float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

}  // namespace pinn
