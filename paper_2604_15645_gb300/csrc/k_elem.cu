// Bandwidth-bound kernels of the PINN step: RWF weight preparation, the input
// embedding jets, the output layer with the PDE residual / loss / adjoint seed,
// per-row reductions, the ordered FP64 finalisation, and Adam.
#include <cmath>

#include "internal.h"
#include "jet.cuh"

namespace pinn {

// ------------------------------------------------------------------------------------
// RWF (Sec. 2.7.2, Eq. 15): W_l = diag(exp(s_l)) V_l for l = 1..L+1, written as an FP32
// master copy and its transpose, a copy in the compute type with its transpose
// (operands of the tensor-core GEMMs), and the rounding remainder W - round(W) in
// the compute type (the low half of the two-term BF16 weight used by the forward
// GEMM).  blockIdx.y selects the layer.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void k_rwf_prep(RwfArgs a) {
  const int l = blockIdx.y;
  const int fin = a.fin[l], fout = a.fout[l];
  const int64_t n = (int64_t)fin * fout;
  const float* V = a.params + a.offV[l];
  const float* s = a.rwf ? a.params + a.offs[l] : nullptr;
  float* W32 = reinterpret_cast<float*>(a.ws + a.w32[l]);
  T* Wc = reinterpret_cast<T*>(a.ws + a.wc[l]);
  T* WTc = reinterpret_cast<T*>(a.ws + a.wtc[l]);
  float* WT32 = reinterpret_cast<float*>(a.ws + a.wt32[l]);
  T* Wlo = reinterpret_cast<T*>(a.ws + a.wlo[l]);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / fin), j = (int)(idx % fin);
    float w = V[idx];
    if (s) w *= expf(s[i]);
    W32[idx] = w;
    const T wh = from_f<T>(w);
    Wc[idx] = wh;
    Wlo[idx] = from_f<T>(w - to_f<T>(wh));
    WTc[(int64_t)j * fout + i] = wh;
    WT32[(int64_t)j * fout + i] = w;
  }
}

void launch_rwf_prep(const RwfArgs& a, cudaStream_t st) {
  dim3 grid(128, a.L1);
  if (a.prec == PINN_BF16) k_rwf_prep<__nv_bfloat16><<<grid, 256, 0, st>>>(a);
  else k_rwf_prep<float><<<grid, 256, 0, st>>>(a);
}

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

// ------------------------------------------------------------------------------------
// Fourier-feature input jets (Sec. 2.7.1, Eq. 14): phi_j = sum_i x_i B_ij,
// gamma = [cos phi, sin phi].  Row k (direction d): d cos = -sin phi B_dj,
// d sin = cos phi B_dj; second-order row: -cos phi sum_{k in S} B_kj^2 (and -sin
// for the sine block).  One thread per (feature j < m, column group).
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void k_embed_ff(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                           int64_t n_bc, int d_in, const float* B, int m, int mode, T* A0, int64_t NC) {
  const int j = blockIdx.y;
  const int64_t ngroups = NC / 4;
  float Bj[3] = {0.f, 0.f, 0.f};
  for (int i = 0; i < d_in; ++i) Bj[i] = B[(int64_t)i * m + j];
  const float q = (mode == JET_MAXWELL) ? 0.f : (Bj[0] * Bj[0] + (mode == JET_NS ? Bj[1] * Bj[1] : 0.f));
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c0 = 4 * g;
    float vc[4], vs[4];
    if (c0 < 4 * n_res) {
      const int64_t p = g;
      float phi = 0.f;
      for (int i = 0; i < d_in; ++i) phi = fmaf(x_res[(int64_t)i * n_res + p], Bj[i], phi);
      float sn, cs;
      sincosf(phi, &sn, &cs);
      vc[0] = cs; vs[0] = sn;
      for (int r = 1; r < 4; ++r) {
        const int d = row_dir(mode, r);
        if (d >= 0) { vc[r] = -sn * Bj[d]; vs[r] = cs * Bj[d]; }
        else { vc[r] = -cs * q; vs[r] = -sn * q; }
      }
    } else {
      for (int r = 0; r < 4; ++r) {
        const ColPoint cp = classify_col(c0 + r, n_res, n_ic, n_bc);
        if (cp.set == 3) { vc[r] = 0.f; vs[r] = 0.f; continue; }
        float phi = 0.f;
        for (int i = 0; i < d_in; ++i) phi = fmaf(coord(x_res, x_ic, x_bc, n_res, n_ic, n_bc, cp, i), Bj[i], phi);
        sincosf(phi, &vs[r], &vc[r]);
      }
    }
    store4<T>(A0 + (int64_t)j * NC + c0, vc);
    store4<T>(A0 + (int64_t)(m + j) * NC + c0, vs);
  }
}

void launch_embed_ff(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                     int64_t n_bc, int d_in, const float* B, int m, int mode, void* A0, int64_t NC, int prec,
                     cudaStream_t st) {
  const int64_t ngroups = NC / 4;
  dim3 grid((unsigned)std::min<int64_t>((ngroups + 255) / 256, 4096), m);
  if (prec == PINN_BF16)
    k_embed_ff<__nv_bfloat16><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, B, m, mode,
                                                    (__nv_bfloat16*)A0, NC);
  else
    k_embed_ff<float><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, B, m, mode, (float*)A0, NC);
}

// ------------------------------------------------------------------------------------
// First hidden layer on raw coordinates (no Fourier features): z = W x + b on the
// value row, z_k = W[:, d_k] on first-derivative rows, 0 on the second-order row
// (the input has no curvature); then the tanh jet rule.  Writes A_1 and Z_1.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void k_first_layer(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                              int64_t n_bc, int d_in, const float* W, const float* b, int fout, int mode, T* A1,
                              T* Z1, int64_t NC) {
  const int f = blockIdx.y;
  const int64_t ngroups = NC / 4;
  float Wf[3] = {0.f, 0.f, 0.f};
  for (int i = 0; i < d_in; ++i) Wf[i] = W[(int64_t)f * d_in + i];
  const float bf = b[f];
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c0 = 4 * g;
    float z[4], a[4];
    if (c0 < 4 * n_res) {
      float v = bf;
      for (int i = 0; i < d_in; ++i) v = fmaf(Wf[i], x_res[(int64_t)i * n_res + g], v);
      z[0] = v;
      for (int r = 1; r < 4; ++r) {
        const int d = row_dir(mode, r);
        z[r] = d >= 0 ? Wf[d] : 0.f;
      }
      jet_fwd(z, a, mode);
    } else {
      for (int r = 0; r < 4; ++r) {
        const ColPoint cp = classify_col(c0 + r, n_res, n_ic, n_bc);
        if (cp.set == 3) { z[r] = 0.f; a[r] = 0.f; continue; }
        float v = bf;
        for (int i = 0; i < d_in; ++i) v = fmaf(Wf[i], coord(x_res, x_ic, x_bc, n_res, n_ic, n_bc, cp, i), v);
        z[r] = v;
        a[r] = val_fwd(v);
      }
    }
    store4<T>(A1 + (int64_t)f * NC + c0, a);
    store4<T>(Z1 + (int64_t)f * NC + c0, z);
  }
}

void launch_first_layer(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                        int64_t n_bc, int d_in, const float* W, const float* b, int fout, int mode, void* A1,
                        void* Z1, int64_t NC, int prec, cudaStream_t st) {
  const int64_t ngroups = NC / 4;
  dim3 grid((unsigned)std::min<int64_t>((ngroups + 255) / 256, 4096), fout);
  if (prec == PINN_BF16)
    k_first_layer<__nv_bfloat16><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, W, b, fout, mode,
                                                       (__nv_bfloat16*)A1, (__nv_bfloat16*)Z1, NC);
  else
    k_first_layer<float><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, W, b, fout, mode,
                                               (float*)A1, (float*)Z1, NC);
}

// ------------------------------------------------------------------------------------
// Output layer (Sec. 2.2, Eq. 6: linear, no activation) + PDE residual + loss
// partials + adjoint seed.  One thread per column group (one interior point, or up
// to four initial/boundary points).  Loss partial sums are reduced per block in
// FP64 and written per block; the cross-block sum happens in finalize (ordered).
// ------------------------------------------------------------------------------------
constexpr int OUT_THREADS = 128;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;
}

template <typename T, int D, bool FAST>
__global__ void __launch_bounds__(OUT_THREADS) k_out_loss(OutArgs a) {
  extern __shared__ float sW[];   // [d_out][w]
  const int w = a.w;
  for (int i = threadIdx.x; i < D * w; i += blockDim.x) sW[i] = a.W[i];
  __syncthreads();
  const T* AL = reinterpret_cast<const T*>(a.AL);
  T* Zb = reinterpret_cast<T*>(a.Zbar);
  const int64_t ngroups = a.NC / 4;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c0 = 4 * g;
    float U[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 4; ++r) U[c][r] = 0.f;
#pragma unroll 4
    for (int f = 0; f < w; ++f) {
      float v[4];
      load4<T>(AL + (int64_t)f * a.NC + c0, v);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float wc = sW[c * w + f];
#pragma unroll
        for (int r = 0; r < 4; ++r) U[c][r] = fmaf(wc, v[r], U[c][r]);
      }
    }
    float Ub[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 4; ++r) Ub[c][r] = 0.f;
    const bool interior = c0 < 4 * a.n_res;
    if (interior) {
#pragma unroll
      for (int c = 0; c < D; ++c) U[c][0] += a.b[c];
      const float k = a.k_pde, nu = a.nu;
      if (a.pde == PINN_BURGERS_1D) {
        // rows [u, u_x, u_t, u_xx]
        const float r = U[0][2] + U[0][0] * U[0][1] - nu * U[0][3];
        acc[0] += (double)r * r;
        const float g2 = 2.f * k * r;
        Ub[0][0] = g2 * U[0][1]; Ub[0][1] = g2 * U[0][0]; Ub[0][2] = g2; Ub[0][3] = -nu * g2;
      } else if (a.pde == PINN_NS_STEADY_2D) {
        // outputs u, v, p; rows [value, d/dx, d/dy, Laplacian]
        const float u = U[0][0], v = U[1][0];
        const float r1 = u * U[0][1] + v * U[0][2] + U[2][1] - nu * U[0][3];
        const float r2 = u * U[1][1] + v * U[1][2] + U[2][2] - nu * U[1][3];
        const float r3 = U[0][1] + U[1][2];
        acc[0] += (double)r1 * r1; acc[1] += (double)r2 * r2; acc[2] += (double)r3 * r3;
        const float g1 = 2.f * k * r1, g2 = 2.f * k * r2, g3 = 2.f * k * r3;
        Ub[0][0] = g1 * U[0][1] + g2 * U[1][1];
        Ub[1][0] = g1 * U[0][2] + g2 * U[1][2];
        Ub[0][1] = g1 * u + g3; Ub[0][2] = g1 * v; Ub[0][3] = -nu * g1;
        Ub[1][1] = g2 * u; Ub[1][2] = g2 * v + g3; Ub[1][3] = -nu * g2;
        Ub[2][1] = g1; Ub[2][2] = g2;
      } else {
        // outputs Ez, Hx, Hy; rows [value, d/dx, d/dy, d/dt]
        const float r1 = U[0][3] - (U[2][1] - U[1][2]);
        const float r2 = U[1][3] + U[0][2];
        const float r3 = U[2][3] - U[0][1];
        acc[0] += (double)r1 * r1; acc[1] += (double)r2 * r2; acc[2] += (double)r3 * r3;
        const float g1 = 2.f * k * r1, g2 = 2.f * k * r2, g3 = 2.f * k * r3;
        Ub[0][3] = g1; Ub[2][1] = -g1; Ub[1][2] = g1;
        Ub[1][3] = g2; Ub[0][2] = g2;
        Ub[2][3] = g3; Ub[0][1] = -g3;
      }
    } else {
      for (int r = 0; r < 4; ++r) {
        const ColPoint cp = classify_col(c0 + r, a.n_res, a.n_ic, a.n_bc);
        if (cp.set == 3) continue;
        const bool ic = cp.set == 1;
        const uint32_t mask = ic ? a.ic_mask : a.bc_mask;
        const float* g = ic ? a.g_ic : a.g_bc;
        const int64_t n = ic ? a.n_ic : a.n_bc;
        const float k = ic ? a.k_ic : a.k_bc;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          U[c][r] += a.b[c];
          if (mask >> c & 1u) {
            const float e = U[c][r] - g[(int64_t)c * n + cp.idx];
            acc[ic ? 3 : 4] += (double)e * e;
            Ub[c][r] = 2.f * k * e;
          }
        }
      }
    }
    if (!a.want_grad) continue;
#pragma unroll
    for (int c = 0; c < D; ++c) store4<float>(a.Ubar + (int64_t)c * a.NC + c0, Ub[c]);
    // abar_L = Ubar W_out (rank <= 3), then the tanh-jet adjoint with Z_L.
    const T* ZL = reinterpret_cast<const T*>(a.ZL);
#pragma unroll 4
    for (int f = 0; f < w; ++f) {
      float ab[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float wc = sW[c * w + f];
#pragma unroll
        for (int r = 0; r < 4; ++r) ab[r] = fmaf(wc, Ub[c][r], ab[r]);
      }
      float z[4], zb[4];
      load4<T>(ZL + (int64_t)f * a.NC + c0, z);
      if (interior) {
        jet_adj<FAST>(z, ab, zb, a.jet_mode);
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          zb[r] = (c0 + r < a.n_res * 4 + a.n_ic + a.n_bc) ? val_adj<FAST>(z[r], ab[r]) : 0.f;
      }
      store4<T>(Zb + (int64_t)f * a.NC + c0, zb);
    }
  }
  __shared__ double sh[OUT_THREADS / 32];
  for (int i = 0; i < 5; ++i) {
    const double s = block_sum_d(acc[i], sh);
    if (threadIdx.x == 0) a.losspart[(int64_t)blockIdx.x * 8 + i] = s;
  }
}

int out_loss_blocks(int64_t ngroups) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((ngroups + OUT_THREADS - 1) / OUT_THREADS, 1184));
}

void launch_out_loss(const OutArgs& a, int prec, int nblocks, cudaStream_t st) {
  const size_t smem = sizeof(float) * a.d_out * a.w;
  if (prec == PINN_BF16) {
    if (a.d_out == 1) k_out_loss<__nv_bfloat16, 1, true><<<nblocks, OUT_THREADS, smem, st>>>(a);
    else k_out_loss<__nv_bfloat16, 3, true><<<nblocks, OUT_THREADS, smem, st>>>(a);
  } else {
    if (a.d_out == 1) k_out_loss<float, 1, false><<<nblocks, OUT_THREADS, smem, st>>>(a);
    else k_out_loss<float, 3, false><<<nblocks, OUT_THREADS, smem, st>>>(a);
  }
}

// ------------------------------------------------------------------------------------
// Output-layer weight gradient: dW_out[c][f] = sum over columns of Ubar[c][col] A_L[f][col].
// One warp per (feature row f, column chunk), coalesced along columns; partials
// [chunk][d_out][w] reduced in FP64 by the finalisation.
// ------------------------------------------------------------------------------------
template <typename T, int D>
__global__ void k_dw_out(const T* AL, const float* Ubar, int w, int64_t NC, int nchunks, float* part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * (blockDim.x >> 5) + warp;
  if (f >= w) return;
  const int chunk = blockIdx.y;
  const int64_t noct = NC / 8;
  const int64_t per = (noct + nchunks - 1) / nchunks;
  const int64_t o0 = chunk * per, o1 = min(noct, o0 + per);
  float acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = 0.f;
  const T* rowp = AL + (int64_t)f * NC;
#pragma unroll 2
  for (int64_t o = o0 + lane; o < o1; o += 32) {
    float v[4], u[4];
    load4<T>(rowp + 8 * o, v);
    load4<T>(rowp + 8 * o + 4, u);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float g[4], h[4];
      load4<float>(Ubar + (int64_t)c * NC + 8 * o, g);
      load4<float>(Ubar + (int64_t)c * NC + 8 * o + 4, h);
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[c] = fmaf(g[r], v[r], fmaf(h[r], u[r], acc[c]));
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    float s = acc[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[((int64_t)chunk * D + c) * w + f] = s;
  }
}

void launch_dw_out(const void* AL, const float* Ubar, int w, int d_out, int64_t NC, int nchunks, float* part,
                   int prec, cudaStream_t st) {
  dim3 grid((w + 7) / 8, nchunks);
  if (prec == PINN_BF16) {
    if (d_out == 1) k_dw_out<__nv_bfloat16, 1><<<grid, 256, 0, st>>>((const __nv_bfloat16*)AL, Ubar, w, NC, nchunks, part);
    else k_dw_out<__nv_bfloat16, 3><<<grid, 256, 0, st>>>((const __nv_bfloat16*)AL, Ubar, w, NC, nchunks, part);
  } else {
    if (d_out == 1) k_dw_out<float, 1><<<grid, 256, 0, st>>>((const float*)AL, Ubar, w, NC, nchunks, part);
    else k_dw_out<float, 3><<<grid, 256, 0, st>>>((const float*)AL, Ubar, w, NC, nchunks, part);
  }
}

// ------------------------------------------------------------------------------------
// Row reductions over a pre-activation adjoint Zbar^T [M][NC]: the bias gradient
// (value columns only) and, for a first layer applied to raw coordinates, the
// coordinate part of dW: dW_ij = sum_value zbar x_j + sum_{rows k with direction j} zbar_k.
// One warp per (row, column chunk); partials [chunk][M][1 + d_in_terms].
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void row_group(const float v[4], int64_t c0, int64_t n_res, int64_t n_ic, int64_t n_bc,
                                          const float* x_res, const float* x_ic, const float* x_bc, int dterms,
                                          int mode, float acc[4]) {
  if (c0 < 4 * n_res) {
    const int64_t g = c0 >> 2;
    acc[0] += v[0];
    for (int j = 0; j < dterms; ++j) acc[1 + j] = fmaf(v[0], x_res[(int64_t)j * n_res + g], acc[1 + j]);
    if (dterms) {
      for (int r = 1; r < 4; ++r) {
        const int d = row_dir(mode, r);
        if (d >= 0) acc[1 + d] += v[r];
      }
    }
  } else {
    for (int r = 0; r < 4; ++r) {
      const ColPoint cp = classify_col(c0 + r, n_res, n_ic, n_bc);
      if (cp.set == 3) continue;
      acc[0] += v[r];
      for (int j = 0; j < dterms; ++j)
        acc[1 + j] = fmaf(v[r], coord(x_res, x_ic, x_bc, n_res, n_ic, n_bc, cp, j), acc[1 + j]);
    }
  }
}

template <typename T>
__global__ void k_row_reduce(const T* Zb, int M, int64_t NC, int64_t n_res, int64_t ncols, int nbpart,
                             const float* x_res, const float* x_ic, const float* x_bc, int64_t n_ic, int64_t n_bc,
                             int dterms, int mode, float* part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + warp;
  if (row >= M) return;
  const int chunk = blockIdx.y;
  const int64_t noct = NC / 8;                          // 8-column units
  const int64_t per = (noct + nbpart - 1) / nbpart;
  const int64_t o0 = chunk * per, o1 = min(noct, o0 + per);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const T* rowp = Zb + (int64_t)row * NC;
#pragma unroll 4
  for (int64_t o = o0 + lane; o < o1; o += 32) {
    float v[4], u[4];
    load4<T>(rowp + 8 * o, v);
    load4<T>(rowp + 8 * o + 4, u);
    row_group<T>(v, 8 * o, n_res, n_ic, n_bc, x_res, x_ic, x_bc, dterms, mode, acc);
    row_group<T>(u, 8 * o + 4, n_res, n_ic, n_bc, x_res, x_ic, x_bc, dterms, mode, acc);
  }
  for (int j = 0; j <= dterms; ++j) {
    float s = acc[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[((int64_t)chunk * M + row) * (1 + dterms) + j] = s;
  }
}

void launch_row_reduce(const void* Zbar, int M, int64_t NC, int64_t n_res, int64_t ncols, int nbpart,
                       const float* x_res, const float* x_ic, const float* x_bc, int64_t n_ic, int64_t n_bc,
                       int dterms, int mode, float* part, int prec, cudaStream_t st) {
  dim3 grid((M + 7) / 8, nbpart);
  if (prec == PINN_BF16)
    k_row_reduce<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)Zbar, M, NC, n_res, ncols, nbpart, x_res,
                                                      x_ic, x_bc, n_ic, n_bc, dterms, mode, part);
  else
    k_row_reduce<float><<<grid, 256, 0, st>>>((const float*)Zbar, M, NC, n_res, ncols, nbpart, x_res, x_ic, x_bc,
                                              n_ic, n_bc, dterms, mode, part);
}

// ------------------------------------------------------------------------------------
// Ordered FP64 reduction of the split partials, then the RWF chain rule
// (Eq. 15): dV = exp(s) dW, ds_i = sum_j dW_ij W_ij, plus db.  One block per
// (output row, layer).
// ------------------------------------------------------------------------------------
// Deterministic block sum of N doubles per thread (fixed assignment and order).
template <int N>
__device__ __forceinline__ void block_sum_n(double v[N], double (*sh)[N]) {
  for (int k = 0; k < N; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < N; ++k) sh[threadIdx.x >> 5][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      for (int k = 0; k < N; ++k) v[k] += sh[w][k];
}

__global__ void k_finalize_grad(FinalizeArgs a) {
  const int l = blockIdx.y, i = blockIdx.x;
  const int fin = a.fin[l], fout = a.fout[l];
  if (i >= fout) return;
  const bool raw = (l == 0 && a.first_raw);
  const float* W = reinterpret_cast<const float*>(a.ws + a.w32[l]) + (int64_t)i * fin;
  const float* dbp = reinterpret_cast<const float*>(a.ws + a.dbpart[l]);
  const int dbs = a.dbstride[l];
  const int nbp = a.nbpart_l[l];
  const float es = a.rwf ? expf(a.params[a.offs[l] + i]) : 1.f;
  __shared__ double sh[32][5];
  // v[0]: sum_j dW_ij W_ij (RWF scale gradient), v[1]: bias, v[2..4]: raw-coordinate dW
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int p = threadIdx.x; p < nbp; p += blockDim.x) {
    const float* q = dbp + ((int64_t)p * fout + i) * dbs;
    v[1] += (double)q[0];
    if (raw)
      for (int j = 0; j < fin && j < 3; ++j) v[2 + j] += (double)q[1 + j];
  }
  if (!raw) {
    const float* part = reinterpret_cast<const float*>(a.ws + a.dwpart[l]);
    const int ns = a.nsplit[l];
    const int64_t sstride = (int64_t)fout * fin;
    if ((fin & 3) == 0) {
      for (int j4 = threadIdx.x * 4; j4 < fin; j4 += blockDim.x * 4) {
        double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
        const float* q = part + (int64_t)i * fin + j4;
#pragma unroll 4
        for (int s = 0; s < ns; ++s) {
          const float4 x = *reinterpret_cast<const float4*>(q + s * sstride);
          d0 += (double)x.x; d1 += (double)x.y; d2 += (double)x.z; d3 += (double)x.w;
        }
        const double dd[4] = {d0, d1, d2, d3};
        for (int k = 0; k < 4; ++k) {
          a.grad[a.offV[l] + (int64_t)i * fin + j4 + k] = (float)(dd[k] * es);
          v[0] += dd[k] * (double)W[j4 + k];
        }
      }
    } else {
      for (int j = threadIdx.x; j < fin; j += blockDim.x) {
        double dW = 0.0;
        for (int s = 0; s < ns; ++s) dW += (double)part[s * sstride + (int64_t)i * fin + j];
        a.grad[a.offV[l] + (int64_t)i * fin + j] = (float)(dW * es);
        v[0] += dW * (double)W[j];
      }
    }
  }
  block_sum_n<5>(v, sh);
  if (threadIdx.x == 0) {
    if (raw) {
      for (int j = 0; j < fin && j < 3; ++j) {
        a.grad[a.offV[l] + (int64_t)i * fin + j] = (float)(v[2 + j] * es);
        v[0] += v[2 + j] * (double)W[j];
      }
    }
    if (a.rwf) a.grad[a.offs[l] + i] = (float)v[0];
    a.grad[a.offb[l] + i] = (float)v[1];
  }
}

void launch_finalize_grad(const FinalizeArgs& a, cudaStream_t st) {
  int maxout = 1;
  for (int l = 0; l < a.L1; ++l) maxout = std::max(maxout, a.fout[l]);
  dim3 grid(maxout, a.L1);
  k_finalize_grad<<<grid, 128, 0, st>>>(a);
}

__global__ void k_finalize_loss(const double* part, int nblocks, int64_t n_res, int64_t n_ic, int64_t n_bc,
                                double lam_pde, double lam_ic, double lam_bc, double* out, int* status) {
  __shared__ double sh[5][256];
  double s[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int i = 0; i < 5; ++i) s[i] += part[(int64_t)b * 8 + i];
  for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] = s[i];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] += sh[i][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double e0 = n_res ? sh[0][0] / n_res : 0.0, e1 = n_res ? sh[1][0] / n_res : 0.0,
                 e2 = n_res ? sh[2][0] / n_res : 0.0;
    const double lic = n_ic ? sh[3][0] / n_ic : 0.0, lbc = n_bc ? sh[4][0] / n_bc : 0.0;
    const double lpde = e0 + e1 + e2;
    const double tot = lam_pde * lpde + lam_ic * lic + lam_bc * lbc;
    out[0] = tot; out[1] = lpde; out[2] = e0; out[3] = e1; out[4] = e2; out[5] = lic; out[6] = lbc; out[7] = 0.0;
    if (!isfinite(tot)) atomicOr(status, 1);
  }
}

void launch_finalize_loss(const double* part, int nblocks, int64_t n_res, int64_t n_ic, int64_t n_bc, double lam_pde,
                          double lam_ic, double lam_bc, double* out, int* status, cudaStream_t st) {
  k_finalize_loss<<<1, 256, 0, st>>>(part, nblocks, n_res, n_ic, n_bc, lam_pde, lam_ic, lam_bc, out, status);
}

// ------------------------------------------------------------------------------------
// Adam (Sec. 2.7.5), bias-corrected, in place.
// ------------------------------------------------------------------------------------
__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

void launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048));
  k_adam<<<blocks, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
}

}  // namespace pinn

// Test hook: the fast tanh pair used by the BF16 epilogues, elementwise.
namespace {
__global__ void k_tanh_selftest(int64_t n, const float* z, float* t, float* tp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float a, b;
    pinn::tanh_fast(z[i], a, b);
    t[i] = a;
    tp[i] = b;
  }
}
}  // namespace

extern "C" PINN_API pinn_status pinn_tanh_selftest(int64_t n, const float* d_z, float* d_t, float* d_tp,
                                                   void* stream) {
  if (n < 0 || (n && (!d_z || !d_t || !d_tp))) return PINN_ERR_INVALID_ARG;
  if (n == 0) return PINN_OK;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_tanh_selftest<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, d_z, d_t, d_tp);
  return cudaGetLastError() == cudaSuccess ? PINN_OK : PINN_ERR_CUDA;
}
