// Bandwidth-bound kernels of the PINN step: RWF weight preparation, the input
// embedding jets, the output layer with the PDE residual / loss / adjoint seed,
// per-row reductions, the ordered FP64 finalisation, and Adam.
#include <cmath>

#include <cuda.h>

#include "internal.h"
#include "jet.cuh"
#include "ptx.cuh"
#include "tc.h"

namespace pinn {

// ------------------------------------------------------------------------------------
// RWF (Sec. 2.6.2, Eq. 15): W_l = diag(exp(s_l)) V_l for l = 1..L+1, written as an FP32
// master copy and its transpose, a copy in the compute type with its transpose
// (operands of the tensor-core GEMMs), and the rounding remainder W - round(W) in
// the compute type (the low half of the two-term BF16 weight used by the forward
// GEMM).  blockIdx.y selects the layer.
// ------------------------------------------------------------------------------------
// One 32 x 32 tile of layer blockIdx.y per block iteration: the row-major outputs are
// stored straight from the loads, the transposed ones through a shared-memory tile, so
// every store of a warp is one contiguous row segment (a store per element at stride
// fout would scatter each warp's writes over 32 rows).
constexpr int RWF_T = 32;

template <typename T>
__device__ __forceinline__ void rwf_split(float w, int prec, T& wh, T& wl) {
  // high / low halves of the weight in the compute type (BF16 rounding; TF32 truncation)
  const float whf = (prec == PINN_TF32) ? tf32_trunc(w) : to_f<T>(from_f<T>(w));
  wh = from_f<T>(whf);
  wl = from_f<T>(w - whf);
}

template <typename T>
__global__ void __launch_bounds__(256) k_rwf_prep(RwfArgs a) {
  __shared__ float tw[RWF_T][RWF_T + 1];
  const int l = blockIdx.y;
  const int fin = a.fin[l], fout = a.fout[l];
  const int tj_n = (fin + RWF_T - 1) / RWF_T, ntiles = tj_n * ((fout + RWF_T - 1) / RWF_T);
  const float* V = a.params + a.offV[l];
  const float* s = a.rwf ? a.params + a.offs[l] : nullptr;
  float* W32 = reinterpret_cast<float*>(a.ws + a.w32[l]);
  T* Wc = reinterpret_cast<T*>(a.ws + a.wc[l]);
  T* WTc = reinterpret_cast<T*>(a.ws + a.wtc[l]);
  float* WT32 = reinterpret_cast<float*>(a.ws + a.wt32[l]);
  T* Wlo = reinterpret_cast<T*>(a.ws + a.wlo[l]);
  T* WTlo = reinterpret_cast<T*>(a.ws + a.wtlo[l]);
  const int tx = threadIdx.x % RWF_T, ty = threadIdx.x / RWF_T;   // 32 x 8 threads
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = (t / tj_n) * RWF_T, j0 = (t % tj_n) * RWF_T;
    for (int r = ty; r < RWF_T; r += 256 / RWF_T) {
      const int i = i0 + r, j = j0 + tx;
      float w = 0.f;
      if (i < fout && j < fin) {
        const int64_t idx = (int64_t)i * fin + j;
        w = V[idx];
        if (s) w *= expf(s[i]);
        T wh, wl;
        rwf_split<T>(w, a.prec, wh, wl);
        W32[idx] = w;
        Wc[idx] = wh;
        Wlo[idx] = wl;
      }
      tw[r][tx] = w;
    }
    __syncthreads();
    for (int r = ty; r < RWF_T; r += 256 / RWF_T) {
      const int j = j0 + r, i = i0 + tx;
      if (i < fout && j < fin) {
        const float w = tw[tx][r];
        T wh, wl;
        rwf_split<T>(w, a.prec, wh, wl);
        const int64_t tidx = (int64_t)j * fout + i;
        WT32[tidx] = w;
        WTc[tidx] = wh;
        WTlo[tidx] = wl;
      }
    }
    __syncthreads();
  }
}

void launch_rwf_prep(const RwfArgs& a, cudaStream_t st) {
  int tiles = 1;
  for (int l = 0; l < a.L1; ++l)
    tiles = std::max(tiles, ((a.fin[l] + RWF_T - 1) / RWF_T) * ((a.fout[l] + RWF_T - 1) / RWF_T));
  dim3 grid(std::min(tiles, 1024), a.L1);
  if (a.prec == PINN_BF16) k_rwf_prep<__nv_bfloat16><<<grid, 256, 0, st>>>(a);
  else k_rwf_prep<float><<<grid, 256, 0, st>>>(a);
}

// Low half of a value-row entry stored in BF16: v - bf16(v), itself rounded to BF16.
template <int LO>
__device__ __forceinline__ void store_lo4(void* base, int64_t off, const float v[4]) {
  if (LO) {
    float lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) lo[k] = v[k] - __bfloat162float(__float2bfloat16_rn(v[k]));
    store4<__nv_bfloat16>(reinterpret_cast<__nv_bfloat16*>(base) + off, lo);
  }
}

// ------------------------------------------------------------------------------------
// Fourier-feature input jets (Sec. 2.6.1, Eq. 14): phi_j = sum_i x_i B_ij,
// gamma = [cos phi, sin phi].  Row k (direction d): d cos = -sin phi B_dj,
// d sin = cos phi B_dj; second-order row: -cos phi sum_{k in S} B_kj^2 (and -sin
// for the sine block).  Initial/boundary points get their value row only.  A thread
// takes four consecutive points (one vector store per jet row) and EMB_F features,
// so each point's set and coordinates are looked up once for all of them.  The BF16
// path uses the fast sincos: its absolute error (about 1e-6 for the phases of the
// Fourier features) is far below the BF16 rounding of the stored jets.
// ------------------------------------------------------------------------------------
constexpr int EMB_F = 4;

template <typename T, int LO>
__global__ void k_embed_ff(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                           int64_t n_bc, int d_in, const float* B, int m, int mode, T* A0, void* A0lo, int64_t NP) {
  const int j0 = blockIdx.y * EMB_F;
  const int64_t wA = 2 * (int64_t)m;   // rows of A_0
  for (int64_t p0 = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); p0 < NP;
       p0 += 4 * (int64_t)gridDim.x * blockDim.x) {
    int set[4];
    float x[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int64_t idx;
      set[k] = point_set(p0 + k, n_res, n_ic, n_bc, idx);
#pragma unroll
      for (int i = 0; i < 3; ++i)
        x[k][i] = (i < d_in) ? point_coord(x_res, x_ic, x_bc, n_res, n_ic, n_bc, p0 + k, i) : 0.f;
    }
    const int64_t c0 = jcol(p0, 0);
    for (int j = j0; j < min(j0 + EMB_F, m); ++j) {
      float Bj[3] = {0.f, 0.f, 0.f};
      for (int i = 0; i < d_in; ++i) Bj[i] = B[(int64_t)i * m + j];
      const float q = (mode == JET_MAXWELL) ? 0.f : (Bj[0] * Bj[0] + (mode == JET_NS ? Bj[1] * Bj[1] : 0.f));
      float vc[4][4], vs[4][4];   // [row][point]
#pragma unroll
      for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int r = 0; r < 4; ++r) { vc[r][k] = 0.f; vs[r][k] = 0.f; }
        if (set[k] != SET_PAD) {
          const float phi = fmaf(x[k][2], Bj[2], fmaf(x[k][1], Bj[1], x[k][0] * Bj[0]));
          float sn, cs;
          if (LO) __sincosf(phi, &sn, &cs);
          else sincosf(phi, &sn, &cs);
          vc[0][k] = cs; vs[0][k] = sn;
          if (set[k] == SET_RES) {
#pragma unroll
            for (int r = 1; r < 4; ++r) {
              const int d = row_dir(mode, r);
              if (d >= 0) { vc[r][k] = -sn * Bj[d]; vs[r][k] = cs * Bj[d]; }
              else { vc[r][k] = -cs * q; vs[r][k] = -sn * q; }
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        store4<T>(A0 + toff(j, c0 + 64 * r, wA), vc[r]);
        store4<T>(A0 + toff(m + j, c0 + 64 * r, wA), vs[r]);
      }
      if (LO) {
        store_lo4<LO>(A0lo, loff(j, p0, wA), vc[0]);
        store_lo4<LO>(A0lo, loff(m + j, p0, wA), vs[0]);
      }
    }
  }
}

void launch_embed_ff(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                     int64_t n_bc, int d_in, const float* B, int m, int mode, void* A0, void* A0lo, int64_t NP,
                     int prec, cudaStream_t st) {
  dim3 grid((unsigned)std::min<int64_t>((NP / 4 + 255) / 256, 4096), (m + EMB_F - 1) / EMB_F);
  if (prec == PINN_BF16)
    k_embed_ff<__nv_bfloat16, 1><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, B, m, mode,
                                                       (__nv_bfloat16*)A0, A0lo, NP);
  else
    k_embed_ff<float, 0><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, B, m, mode,
                                               (float*)A0, nullptr, NP);
}

// ------------------------------------------------------------------------------------
// First hidden layer on raw coordinates (no Fourier features): z = W x + b on the
// value row, z_k = W[:, d_k] on the first-derivative rows of interior points, 0 on
// the second-order row (the input has no curvature); then the activation's jet rule.
// Writes A_1 (and its value-row low half), and for the sine activation Z_1 (FP32).
// ------------------------------------------------------------------------------------
template <typename T, int LO, bool SINE>
__global__ void k_first_layer(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                              int64_t n_bc, int d_in, const float* W, const float* b, int fout, int mode, T* A1,
                              void* A1lo, int64_t NP, float omega0, float* Z1) {
  const int f = blockIdx.y;
  float Wf[3] = {0.f, 0.f, 0.f};
  for (int i = 0; i < d_in; ++i) Wf[i] = W[(int64_t)f * d_in + i];
  const float bf = b[f];

  for (int64_t p0 = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); p0 < NP;
       p0 += 4 * (int64_t)gridDim.x * blockDim.x) {
    float aa[4][4], zs[4][4];   // [row][point]
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t p = p0 + k;
      int64_t idx;
      const int set = point_set(p, n_res, n_ic, n_bc, idx);
      float z[4] = {bf, 0.f, 0.f, 0.f}, a[4];
      for (int i = 0; i < d_in; ++i) z[0] = fmaf(Wf[i], point_coord(x_res, x_ic, x_bc, n_res, n_ic, n_bc, p, i), z[0]);
      if (set == SET_RES) {
#pragma unroll
        for (int r = 1; r < 4; ++r) {
          const int d = row_dir(mode, r);
          z[r] = d >= 0 ? Wf[d] : 0.f;
        }
      }
      if constexpr (SINE) jet_fwd_sine(z, a, mode, omega0);
      else jet_fwd<(LO == 1)>(z, a, mode);
#pragma unroll
      for (int r = 0; r < 4; ++r) { aa[r][k] = a[r]; zs[r][k] = z[r]; }
    }
    const int64_t c0 = jcol(p0, 0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      store4<T>(A1 + toff(f, c0 + 64 * r, fout), aa[r]);
      if constexpr (SINE) store4<float>(Z1 + toff(f, c0 + 64 * r, fout), zs[r]);
    }
    if (LO) store_lo4<LO>(A1lo, loff(f, p0, fout), aa[0]);
  }
}

void launch_first_layer(const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res, int64_t n_ic,
                        int64_t n_bc, int d_in, const float* W, const float* b, int fout, int mode, void* A1,
                        void* A1lo, int64_t NP, int prec, float omega0, float* Z1, cudaStream_t st) {
  dim3 grid((unsigned)std::min<int64_t>((NP / 4 + 255) / 256, 4096), fout);
  if (prec == PINN_BF16) {
    if (Z1)
      k_first_layer<__nv_bfloat16, 1, true><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, W, b,
                                                                  fout, mode, (__nv_bfloat16*)A1, A1lo, NP, omega0, Z1);
    else
      k_first_layer<__nv_bfloat16, 1, false><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, W, b,
                                                                   fout, mode, (__nv_bfloat16*)A1, A1lo, NP, omega0,
                                                                   nullptr);
  } else {
    if (Z1)
      k_first_layer<float, 0, true><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, W, b, fout,
                                                          mode, (float*)A1, nullptr, NP, omega0, Z1);
    else
      k_first_layer<float, 0, false><<<grid, 256, 0, st>>>(x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, W, b, fout,
                                                           mode, (float*)A1, nullptr, NP, omega0, nullptr);
  }
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

// Compensated FP32 accumulation (Knuth's TwoSum): s + c tracks the exact sum of
// the added values to about 2^-48 relative, using the FP32 pipe; it is turned into
// FP64 once per thread, so the FP64 work of the final reductions stays small.
struct Acc2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Residual and seed for one point from its output jets U[c][r] (bias included).
// k: the interior seed scale (k_pde, or the point's causal segment scale); rr: the
// point's squared residual per equation (interior points); lacc (FP64, or FP32 for a
// few points at a time) gathers the squared errors per loss term.
template <int D, typename LT>
__device__ __forceinline__ void point_residual(const OutArgs& a, int set, int64_t idx, float k, float U[3][4],
                                               float Ub[3][4], LT lacc[5], float rr[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) Ub[c][r] = 0.f;
  rr[0] = rr[1] = rr[2] = 0.f;
  if (set == SET_RES) {
    const float nu = a.nu;
    if (a.pde == PINN_BURGERS_1D) {
      // rows [u, u_x, u_t, u_xx]
      const float r = U[0][2] + U[0][0] * U[0][1] - nu * U[0][3];
      lacc[0] += (LT)r * r; rr[0] = r * r;
      const float g2 = 2.f * k * r;
      Ub[0][0] = g2 * U[0][1]; Ub[0][1] = g2 * U[0][0]; Ub[0][2] = g2; Ub[0][3] = -nu * g2;
    } else if (a.pde == PINN_ADVECTION_1D) {
      // u_t + c u_x with c = nu (Sec. 4.1)
      const float r = fmaf(nu, U[0][1], U[0][2]);
      lacc[0] += (LT)r * r; rr[0] = r * r;
      const float g2 = 2.f * k * r;
      Ub[0][1] = nu * g2; Ub[0][2] = g2;
    } else if (a.pde == PINN_ALLEN_CAHN_1D) {
      // u_t - eps u_xx + 5 u^3 - 5 u with eps = nu (Sec. 4.2)
      const float u = U[0][0];
      const float r = U[0][2] - nu * U[0][3] + 5.f * u * (u * u - 1.f);
      lacc[0] += (LT)r * r; rr[0] = r * r;
      const float g2 = 2.f * k * r;
      Ub[0][0] = g2 * (15.f * u * u - 5.f); Ub[0][2] = g2; Ub[0][3] = -nu * g2;
    } else if (a.pde == PINN_NS_STEADY_2D) {
      // outputs u, v, p; rows [value, d/dx, d/dy, Laplacian]
      const float u = U[0][0], v = U[1 % D][0];
      const float r1 = u * U[0][1] + v * U[0][2] + U[2 % D][1] - nu * U[0][3];
      const float r2 = u * U[1 % D][1] + v * U[1 % D][2] + U[2 % D][2] - nu * U[1 % D][3];
      const float r3 = U[0][1] + U[1 % D][2];
      lacc[0] += (LT)r1 * r1; lacc[1] += (LT)r2 * r2; lacc[2] += (LT)r3 * r3;
      rr[0] = r1 * r1; rr[1] = r2 * r2; rr[2] = r3 * r3;
      const float g1 = 2.f * k * r1, g2 = 2.f * k * r2, g3 = 2.f * k * r3;
      Ub[0][0] = g1 * U[0][1] + g2 * U[1 % D][1];
      Ub[1 % D][0] = g1 * U[0][2] + g2 * U[1 % D][2];
      Ub[0][1] = g1 * u + g3; Ub[0][2] = g1 * v; Ub[0][3] = -nu * g1;
      Ub[1 % D][1] = g2 * u; Ub[1 % D][2] = g2 * v + g3; Ub[1 % D][3] = -nu * g2;
      Ub[2 % D][1] = g1; Ub[2 % D][2] = g2;
    } else {
      // outputs Ez, Hx, Hy; rows [value, d/dx, d/dy, d/dt]
      const float r1 = U[0][3] - (U[2 % D][1] - U[1 % D][2]);
      const float r2 = U[1 % D][3] + U[0][2];
      const float r3 = U[2 % D][3] - U[0][1];
      lacc[0] += (LT)r1 * r1; lacc[1] += (LT)r2 * r2; lacc[2] += (LT)r3 * r3;
      rr[0] = r1 * r1; rr[1] = r2 * r2; rr[2] = r3 * r3;
      const float g1 = 2.f * k * r1, g2 = 2.f * k * r2, g3 = 2.f * k * r3;
      Ub[0][3] = g1; Ub[2 % D][1] = -g1; Ub[1 % D][2] = g1;
      Ub[1 % D][3] = g2; Ub[0][2] = g2;
      Ub[2 % D][3] = g3; Ub[0][1] = -g3;
    }
  } else if (set != SET_PAD) {
    const bool ic = set == SET_IC;
    const uint32_t mask = ic ? a.ic_mask : a.bc_mask;
    const float* gt = ic ? a.g_ic : a.g_bc;
    const int64_t n = ic ? a.n_ic : a.n_bc;
    const float k = ic ? a.k_ic : a.k_bc;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (mask >> c & 1u) {
        const float err = U[c][0] - gt[(int64_t)c * n + idx];
        lacc[ic ? 3 : 4] += (LT)err * err;
        Ub[c][0] = 2.f * k * err;
      }
    }
  }
}

// Cache hints for the two passes over A_L: the second read is its last use, and the
// adjoint Zbar_L is written once and read by the next kernel, so neither should push
// the first pass's A_L lines out of L2 before the second pass re-reads them.
template <typename T> __device__ __forceinline__ void load4_last(const T* p, float v[4]);
template <> __device__ __forceinline__ void load4_last<float>(const float* p, float v[4]) {
  const float4 q = __ldlu(reinterpret_cast<const float4*>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <> __device__ __forceinline__ void load4_last<__nv_bfloat16>(const __nv_bfloat16* p, float v[4]) {
  const uint2 u = __ldlu(reinterpret_cast<const uint2*>(p));
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename T> __device__ __forceinline__ void store4_stream(T* p, const float v[4]);
template <> __device__ __forceinline__ void store4_stream<float>(float* p, const float v[4]) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}
template <> __device__ __forceinline__ void store4_stream<__nv_bfloat16>(__nv_bfloat16* p, const float v[4]) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 u;
  u.x = *reinterpret_cast<const uint32_t*>(&lo);
  u.y = *reinterpret_cast<const uint32_t*>(&hi);
  __stcs(reinterpret_cast<uint2*>(p), u);
}

// One block per 64-point tile (grid-stride).  Warp w takes points 16w..16w+15;
// lane = 8 * pg + sl: point group pg (4 consecutive points) and feature slice sl
// (features sl, sl+8, ...).  The 8 slices of a point group combine their partial
// outputs with three xor-shuffles; every slice then holds the group's outputs.
template <typename T, int D, bool FAST, bool SINE>
__global__ void __launch_bounds__(OUT_THREADS) k_out_loss(OutArgs a) {
  // [d_out][w] weights, then [warps][d_out][w] dW accumulators, then [warps][w] bias
  // accumulators of the last hidden layer
  extern __shared__ float sW[];
  const int w = a.w;
  float* sdw = sW + D * w;
  float* sdb = sdw + (OUT_THREADS / 32) * D * w;
  for (int i = threadIdx.x; i < D * w; i += blockDim.x) sW[i] = a.W[i];
  for (int i = threadIdx.x; i < (OUT_THREADS / 32) * (D + 1) * w; i += blockDim.x) sdw[i] = 0.f;
  __syncthreads();
  const T* AL = reinterpret_cast<const T*>(a.AL);
  const __nv_bfloat16* ALlo = reinterpret_cast<const __nv_bfloat16*>(a.ALlo);
  T* Zb = reinterpret_cast<T*>(a.Zbar);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pg = lane >> 3, sl = lane & 7;
  const int q0 = 16 * warp + 4 * pg;               // first of this thread's 4 points in the tile
  const int64_t ntiles = a.NP / TILE_PTS;
  Acc2 acc[5];   // compensated FP32 running sums (FP64 is a slow pipe on this part)
  float dbo[3] = {0.f, 0.f, 0.f};                 // output bias gradient (value-row seeds)
  // temporal causality, first pass: this block's segment sums (3 equations + count),
  // accumulated by one thread over the tile's points in a fixed order
  __shared__ double segacc[CAUSAL_MAX][4];
  __shared__ int s_seg[TILE_PTS];
  __shared__ float s_rr[TILE_PTS][3];
  if (a.segpart)
    for (int i = threadIdx.x; i < CAUSAL_MAX * 4; i += blockDim.x) segacc[i / 4][i % 4] = 0.0;
  for (int64_t T0i = blockIdx.x; T0i < ntiles; T0i += gridDim.x) {
    const int64_t T0 = a.reverse ? ntiles - 1 - T0i : T0i;
    const int64_t cb = T0 * TILE_COLS + q0;        // column of row 0 of the first point
    const int64_t p0 = T0 * TILE_PTS + q0;
    float U[4][3][4];                              // [point][output][row]
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) U[j][c][r] = 0.f;
#pragma unroll 2
    for (int f = sl; f < w; f += 8) {
      const T* row = AL + toff(f, cb, w);
      float v[4][4];                               // [row][point]
#pragma unroll
      for (int r = 0; r < 4; ++r) load4<T>(row + 64 * r, v[r]);
      if (ALlo) {
        float lo[4];
        load4<__nv_bfloat16>(ALlo + loff(f, p0, w), lo);
#pragma unroll
        for (int j = 0; j < 4; ++j) v[0][j] += lo[j];
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float wc = sW[c * w + f];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) U[j][c][r] = fmaf(wc, v[r][j], U[j][c][r]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float x = U[j][c][r];
          x += __shfl_xor_sync(0xffffffffu, x, 1);
          x += __shfl_xor_sync(0xffffffffu, x, 2);
          x += __shfl_xor_sync(0xffffffffu, x, 4);
          U[j][c][r] = x;
        }
    float Ub[4][3][4];
    float lacc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int segj[4];
    float rrj[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t idx;
      const int set = point_set(p0 + j, a.n_res, a.n_ic, a.n_bc, idx);
      if (set != SET_PAD) {
#pragma unroll
        for (int c = 0; c < D; ++c) U[j][c][0] += a.b[c];
      }
      float kp = a.k_pde;
      segj[j] = -1;
      if (a.segments && set == SET_RES) {
        const float tt = a.x_res[(int64_t)a.t_index * a.n_res + idx];
        segj[j] = min(a.segments - 1, max(0, (int)floorf((tt - a.t0) * a.tinv)));
        if (a.seg_scale) kp = a.seg_scale[segj[j]];
      }
      point_residual<D>(a, set, idx, kp, U[j], Ub[j], lacc, rrj[j]);
    }
    if (sl == 0)
      for (int i = 0; i < 5; ++i) acc[i].add(lacc[i]);
    if (a.segpart) {   // uniform over the block
      if (sl == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          s_seg[q0 + j] = segj[j];
          s_rr[q0 + j][0] = rrj[j][0]; s_rr[q0 + j][1] = rrj[j][1]; s_rr[q0 + j][2] = rrj[j][2];
        }
      __syncthreads();
      if (threadIdx.x == 0)
        for (int q = 0; q < TILE_PTS; ++q)
          if (s_seg[q] >= 0) {
            double* sa = segacc[s_seg[q]];
            sa[0] += s_rr[q][0]; sa[1] += s_rr[q][1]; sa[2] += s_rr[q][2]; sa[3] += 1.0;
          }
      __syncthreads();
    }
    if (!a.want_grad) continue;
    if (sl == 0) {
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) dbo[c] += Ub[j][c][0];
    }
    // A_L read again (from L2) for the output layer's dW[c][f] = sum over the tile's
    // columns of Ubar[c] A_L[f], and for abar_L = Ubar W_out (rank <= 3) followed by
    // the tanh-jet adjoint written in A_L.  Every lane runs every pass (the dW sum
    // shuffles across the warp); a slice past the width reads feature w-1 and
    // discards what it computed.
#pragma unroll 2
    for (int f0 = 0; f0 < w; f0 += 8) {
      const bool live = f0 + sl < w;
      const int f = live ? f0 + sl : w - 1;
      float av[4][4], zb[4][4];                    // [row][point]
      {
        const T* arow = AL + toff(f, cb, w);
#pragma unroll
        for (int r = 0; r < 4; ++r) load4_last<T>(arow + 64 * r, av[r]);
        if (ALlo) {
          float lo[4];
          load4<__nv_bfloat16>(ALlo + loff(f, p0, w), lo);
#pragma unroll
          for (int j = 0; j < 4; ++j) av[0][j] += lo[j];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
          float g = 0.f;
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) g = fmaf(Ub[j][c][r], av[r][j], g);
          g += __shfl_xor_sync(0xffffffffu, g, 8);    // the warp's four point groups
          g += __shfl_xor_sync(0xffffffffu, g, 16);
          if (pg == 0 && live) sdw[(warp * D + c) * w + f] += g;
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float ab[4] = {0.f, 0.f, 0.f, 0.f}, zz[4], o[4];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const float wc = sW[c * w + f];
#pragma unroll
          for (int r = 0; r < 4; ++r) ab[r] = fmaf(wc, Ub[j][c][r], ab[r]);
        }
        if constexpr (SINE) {   // the adjoint is evaluated from the pre-activation jets
#pragma unroll
          for (int r = 0; r < 4; ++r) zz[r] = a.ZL[toff(f, cb + 64 * r + j, w)];
          jet_adj_sine(zz, ab, o, a.jet_mode, a.omega0);
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r) zz[r] = av[r][j];
          jet_adj_a(zz, ab, o, a.jet_mode);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) zb[r][j] = o[r];
      }
      T* zbrow = Zb + toff(f, cb, w);
      if (live)
#pragma unroll
        for (int r = 0; r < 4; ++r) store4_stream<T>(zbrow + 64 * r, zb[r]);
      if (a.dbhid) {   // the last hidden layer's bias gradient: value rows of Zbar_L
        float s = (zb[0][0] + zb[0][1]) + (zb[0][2] + zb[0][3]);
        s += __shfl_xor_sync(0xffffffffu, s, 8);
        s += __shfl_xor_sync(0xffffffffu, s, 16);
        if (pg == 0 && live) sdb[warp * w + f] += s;
      }
    }
  }
  __shared__ double sh[OUT_THREADS / 32];
  for (int i = 0; i < 5; ++i) {
    const double s = block_sum_d(acc[i].value(), sh);
    if (threadIdx.x == 0) a.losspart[(int64_t)blockIdx.x * 8 + i] = s;
  }
  if (a.segpart) {
    __syncthreads();
    for (int i = threadIdx.x; i < CAUSAL_MAX * 4; i += blockDim.x)
      a.segpart[(int64_t)blockIdx.x * CAUSAL_MAX * 4 + i] = segacc[i / 4][i % 4];
  }
  if (!a.want_grad) return;
  // block partials of the output layer's dW (warps summed in a fixed order) and bias
  __syncthreads();
  for (int i = threadIdx.x; i < D * w; i += blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < OUT_THREADS / 32; ++k) s += sdw[k * D * w + i];
    a.dwpart[(int64_t)blockIdx.x * D * w + i] = s;
  }
  if (a.dbhid)
    for (int i = threadIdx.x; i < w; i += blockDim.x) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < OUT_THREADS / 32; ++k) s += sdb[k * w + i];
      a.dbhid[(int64_t)i * gridDim.x + blockIdx.x] = s;
    }
  for (int c = 0; c < D; ++c) {
    float v = dbo[c];
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    __shared__ float shb[OUT_THREADS / 32];
    __syncthreads();
    if (lane == 0) shb[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int k = 0; k < OUT_THREADS / 32; ++k) t += shb[k];
      a.dbpart[(int64_t)c * gridDim.x + blockIdx.x] = t;
    }
  }
}

int out_loss_blocks(int64_t NP) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(NP / TILE_PTS, 4096));
}

// ------------------------------------------------------------------------------------
// The same output layer, residual, loss and adjoint seed for BF16 tanh networks
// (hidden width <= 512), with A_L staged through shared memory by TMA instead of
// register-limited global loads.  A producer warp streams each 64-point tile's A_L
// in chunks of 32 features (four 128-byte swizzled boxes, one per jet row, plus the
// value-row low half) through a three-stage ring: once for the output jets and the
// residual, and once more (an L2 hit) for the output layer's dW, the adjoint
// abar_L = Ubar W_out and its tanh-jet adjoint.  Four consumer warps use the same
// lane mapping as k_out_loss (point group pg = lane / 8, feature slice sl = lane % 8);
// the swizzle spreads a warp's eight features over all banks.  Results (loss and
// segment partials, dW, bias partials, Zbar_L) and their summation order per block
// are those of k_out_loss.  The consumers read the ring with ordinary shared loads
// (generic proxy) and the producer refills it with bulk copies (async proxy): the
// mbarrier's release/acquire orders only the generic proxy, so every consumer fences
// the proxies (fence.proxy.async) after its last read of a slot and before releasing
// it; without the fence a refill could overwrite a slot under reads still in flight
// (measured: loss changes of 1e-5 to 1e-4 relative at width 512 that depended on
// what else was in L2).
// ------------------------------------------------------------------------------------
constexpr int OT_CONS = 128;                     // consumer threads (4 warps)
constexpr int OT_THREADS = OT_CONS + 32;         // + the producer warp
constexpr int OT_FC = 32;                        // features per chunk
constexpr int OT_ROWB = OT_FC * 128;             // one jet-row box: 32 features x 64 points x 2 B = 4 KB
constexpr int OT_STAGE = 5 * OT_ROWB;            // four jet rows + the value-row low half: 20 KB
constexpr int OT_STAGES = 3;
constexpr uint64_t OT_WAIT_NS = 2000000000ull;

__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 1, %0;" ::"n"(OT_CONS) : "memory"); }
// Named barrier over the four consumer warps that also ANDs a predicate over them, so
// that a failed (bounded) wait in any warp makes every warp leave the loop together.
__device__ __forceinline__ bool cons_sync_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(OT_CONS)
      : "memory");
  return r != 0;
}

// Four BF16 values of (feature fi, points q0..q0+3) of a 128-byte swizzled box row.
__device__ __forceinline__ void ot_load4(const uint8_t* box, int fi, int q0, float v[4]) {
  const int chunk = (q0 >> 3) ^ (fi & 7);
  const uint2 u = *reinterpret_cast<const uint2*>(box + fi * 128 + chunk * 16 + (q0 & 7) * 2);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ double cons_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  cons_sync();
  if (l == 0) sh[w] = v;
  cons_sync();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < OT_CONS / 32; ++i) s += sh[i];
  return s;
}

// D outputs, jet rule MODE and the presence of the value-row low half (LO) are
// compile-time, and the width is a multiple of the 32-feature chunk: the unrolled
// per-feature loops carry no branches, so their loads and arithmetic interleave.
template <int D, int MODE, bool LO>
__global__ void __launch_bounds__(OT_THREADS) k_out_loss_tma(const __grid_constant__ CUtensorMap mapA,
                                                            const __grid_constant__ CUtensorMap mapLo, OutArgs a) {
  extern __shared__ uint8_t ot_raw[];
  // 1024-byte aligned by offsetting the shared array itself (not through an integer
  // round trip), so the compiler keeps every access below in the shared window
  uint8_t* ring = ot_raw + ((1024u - (smem_u32(ot_raw) & 1023u)) & 1023u);
  const int w = a.w;
  float* sW = reinterpret_cast<float*>(ring + OT_STAGES * OT_STAGE);   // [D][w] output weights
  float* sdw = sW + D * w;                                            // [4 warps][D][w] dW accumulators
  float* sdb = sdw + (OT_CONS / 32) * D * w;                          // [4 warps][w] hidden bias accumulators
  const int bar_off = (OT_STAGES * OT_STAGE + (int)sizeof(float) * (D * w + (OT_CONS / 32) * (D + 1) * w) + 7) & ~7;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + bar_off);
  uint64_t* empty = full + OT_STAGES;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + OT_STAGES);
  __shared__ double segacc[CAUSAL_MAX][4];
  __shared__ int s_seg[TILE_PTS];
  __shared__ float s_rr[TILE_PTS][3];
  __shared__ double sh[OT_CONS / 32];
  __shared__ float shb[OT_CONS / 32];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OT_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], OT_CONS);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < D * w; i += blockDim.x) sW[i] = a.W[i];
  for (int i = threadIdx.x; i < (OT_CONS / 32) * (D + 1) * w; i += blockDim.x) sdw[i] = 0.f;
  if (a.segpart)
    for (int i = threadIdx.x; i < CAUSAL_MAX * 4; i += blockDim.x) segacc[i / 4][i % 4] = 0.0;
  __syncthreads();

  const int64_t ntiles = a.NP / TILE_PTS;
  const int nchunks = w / OT_FC;
  const int passes = a.want_grad ? 2 : 1;

  if (warp == OT_CONS / 32) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed[OT_STAGES] = {0, 0, 0};
      for (int64_t T0i = blockIdx.x; T0i < ntiles && !*abort_flag; T0i += gridDim.x) {
        const int T0 = (int)(a.reverse ? ntiles - 1 - T0i : T0i);
        for (int pass = 0; pass < passes && !*abort_flag; ++pass)
          for (int k = 0; k < nchunks; ++k) {
            if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.status, OT_WAIT_NS)) break;
            uint8_t* sb = ring + stage * OT_STAGE;
            mbar_expect_tx(&full[stage], (LO ? 5 : 4) * OT_ROWB);
            armed[stage] = (int)phase + 1;
#pragma unroll
            for (int r = 0; r < 4; ++r) tma_load_3d(sb + r * OT_ROWB, &mapA, &full[stage], 64 * r, OT_FC * k, T0);
            if constexpr (LO) tma_load_3d(sb + 4 * OT_ROWB, &mapLo, &full[stage], 0, OT_FC * k, T0);
            if (++stage == OT_STAGES) { stage = 0; phase ^= 1; }
          }
      }
      // every load this thread issued lands before the block may exit (bounded)
      for (int s = 0; s < OT_STAGES; ++s)
        if (armed[s]) {
          const uint64_t t0 = gtimer();
          while (!mbar_try(&full[s], (uint32_t)(armed[s] - 1)) && gtimer() - t0 < OT_WAIT_NS) {}
        }
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  const __nv_bfloat16* ALlo = reinterpret_cast<const __nv_bfloat16*>(a.ALlo);
  (void)ALlo;
  __nv_bfloat16* Zb = reinterpret_cast<__nv_bfloat16*>(a.Zbar);
  const int pg = lane >> 3, sl = lane & 7;
  const int q0 = 16 * warp + 4 * pg;
  // squared errors: FP32 per tile (four points), compensated FP32 across tiles, FP64
  // only in the block's final sum (FP64 is a slow pipe on this part)
  Acc2 acc[5];
  float dbo[3] = {0.f, 0.f, 0.f};
  int stage = 0;
  uint32_t phase = 0;
  bool ok = true;
  // A failed bounded wait leaves the chunk loop in that warp only; the ANDed barrier
  // after each pass makes every consumer warp leave the tile loop together, so no named
  // barrier is left waiting for a warp that has gone.
  for (int64_t T0i = blockIdx.x; T0i < ntiles; T0i += gridDim.x) {
    const int64_t T0 = a.reverse ? ntiles - 1 - T0i : T0i;
    const int64_t cb = T0 * TILE_COLS + q0;
    const int64_t p0 = T0 * TILE_PTS + q0;
    float U[4][3][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) U[j][c][r] = 0.f;
    for (int k = 0; k < nchunks; ++k) {
      if (!mbar_wait(&full[stage], phase, abort_flag, a.status, OT_WAIT_NS)) { ok = false; break; }
      const uint8_t* sb = ring + stage * OT_STAGE;
#pragma unroll
      for (int e = 0; e < OT_FC / 8; ++e) {
        const int fi = sl + 8 * e, f = OT_FC * k + fi;
        float v[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) ot_load4(sb + r * OT_ROWB, fi, q0 & 63, v[r]);
        if constexpr (LO) {
          float l4[4];
          ot_load4(sb + 4 * OT_ROWB, fi, q0 & 63, l4);
#pragma unroll
          for (int j = 0; j < 4; ++j) v[0][j] += l4[j];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const float wc = sW[c * w + f];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) U[j][c][r] = fmaf(wc, v[r][j], U[j][c][r]);
        }
      }
      fence_proxy_async_smem();   // these reads before the producer's next bulk copy into the slot
      mbar_arrive(&empty[stage]);
      if (++stage == OT_STAGES) { stage = 0; phase ^= 1; }
    }
    ok = cons_sync_and(ok);
    if (!ok) break;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float x = U[j][c][r];
          x += __shfl_xor_sync(0xffffffffu, x, 1);
          x += __shfl_xor_sync(0xffffffffu, x, 2);
          x += __shfl_xor_sync(0xffffffffu, x, 4);
          U[j][c][r] = x;
        }
    float Ub[4][3][4];
    float lacc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int segj[4];
    float rrj[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t idx;
      const int set = point_set(p0 + j, a.n_res, a.n_ic, a.n_bc, idx);
      if (set != SET_PAD) {
#pragma unroll
        for (int c = 0; c < D; ++c) U[j][c][0] += a.b[c];
      }
      float kp = a.k_pde;
      segj[j] = -1;
      if (a.segments && set == SET_RES) {
        const float tt = a.x_res[(int64_t)a.t_index * a.n_res + idx];
        segj[j] = min(a.segments - 1, max(0, (int)floorf((tt - a.t0) * a.tinv)));
        if (a.seg_scale) kp = a.seg_scale[segj[j]];
      }
      point_residual<D>(a, set, idx, kp, U[j], Ub[j], lacc, rrj[j]);
    }
    if (sl == 0)
      for (int i = 0; i < 5; ++i) acc[i].add(lacc[i]);
    if (a.segpart) {
      if (sl == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          s_seg[q0 + j] = segj[j];
          s_rr[q0 + j][0] = rrj[j][0]; s_rr[q0 + j][1] = rrj[j][1]; s_rr[q0 + j][2] = rrj[j][2];
        }
      cons_sync();
      if (threadIdx.x == 0)
        for (int q = 0; q < TILE_PTS; ++q)
          if (s_seg[q] >= 0) {
            double* sa = segacc[s_seg[q]];
            sa[0] += s_rr[q][0]; sa[1] += s_rr[q][1]; sa[2] += s_rr[q][2]; sa[3] += 1.0;
          }
      cons_sync();
    }
    if (!a.want_grad) continue;
    if (sl == 0) {
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) dbo[c] += Ub[j][c][0];
    }
    for (int k = 0; k < nchunks; ++k) {
      if (!mbar_wait(&full[stage], phase, abort_flag, a.status, OT_WAIT_NS)) { ok = false; break; }
      const uint8_t* sb = ring + stage * OT_STAGE;
#pragma unroll
      for (int e = 0; e < OT_FC / 8; ++e) {
        const int fi = sl + 8 * e;
        const int f = OT_FC * k + fi;
        float av[4][4], zb[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) ot_load4(sb + r * OT_ROWB, fi, q0 & 63, av[r]);
        if constexpr (LO) {
          float l4[4];
          ot_load4(sb + 4 * OT_ROWB, fi, q0 & 63, l4);
#pragma unroll
          for (int j = 0; j < 4; ++j) av[0][j] += l4[j];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
          float g = 0.f;
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) g = fmaf(Ub[j][c][r], av[r][j], g);
          g += __shfl_xor_sync(0xffffffffu, g, 8);
          g += __shfl_xor_sync(0xffffffffu, g, 16);
          if (pg == 0) sdw[(warp * D + c) * w + f] += g;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float ab[4] = {0.f, 0.f, 0.f, 0.f}, zz[4], o[4];
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const float wc = sW[c * w + f];
#pragma unroll
            for (int r = 0; r < 4; ++r) ab[r] = fmaf(wc, Ub[j][c][r], ab[r]);
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) zz[r] = av[r][j];
          jet_adj_a(zz, ab, o, MODE);
#pragma unroll
          for (int r = 0; r < 4; ++r) zb[r][j] = o[r];
        }
        __nv_bfloat16* zbrow = Zb + toff(f, cb, w);
#pragma unroll
        for (int r = 0; r < 4; ++r) store4_stream<__nv_bfloat16>(zbrow + 64 * r, zb[r]);
        if (a.dbhid) {
          float s = (zb[0][0] + zb[0][1]) + (zb[0][2] + zb[0][3]);
          s += __shfl_xor_sync(0xffffffffu, s, 8);
          s += __shfl_xor_sync(0xffffffffu, s, 16);
          if (pg == 0) sdb[warp * w + f] += s;
        }
      }
      fence_proxy_async_smem();   // these reads before the producer's next bulk copy into the slot
      mbar_arrive(&empty[stage]);
      if (++stage == OT_STAGES) { stage = 0; phase ^= 1; }
    }
    ok = cons_sync_and(ok);
    if (!ok) break;
  }
  for (int i = 0; i < 5; ++i) {
    const double s = cons_sum_d(acc[i].value(), sh);
    if (threadIdx.x == 0) a.losspart[(int64_t)blockIdx.x * 8 + i] = s;
  }
  if (a.segpart) {
    cons_sync();
    for (int i = threadIdx.x; i < CAUSAL_MAX * 4; i += OT_CONS)
      a.segpart[(int64_t)blockIdx.x * CAUSAL_MAX * 4 + i] = segacc[i / 4][i % 4];
  }
  if (!a.want_grad) return;
  cons_sync();
  for (int i = threadIdx.x; i < D * w; i += OT_CONS) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < OT_CONS / 32; ++k) s += sdw[k * D * w + i];
    a.dwpart[(int64_t)blockIdx.x * D * w + i] = s;
  }
  if (a.dbhid)
    for (int i = threadIdx.x; i < w; i += OT_CONS) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < OT_CONS / 32; ++k) s += sdb[k * w + i];
      a.dbhid[(int64_t)i * gridDim.x + blockIdx.x] = s;
    }
  for (int c = 0; c < D; ++c) {
    float v = dbo[c];
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    cons_sync();
    if (lane == 0) shb[warp] = v;
    cons_sync();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int k = 0; k < OT_CONS / 32; ++k) t += shb[k];
      a.dbpart[(int64_t)c * gridDim.x + blockIdx.x] = t;
    }
  }
}

// Whether the TMA-staged output kernel applies: BF16 tanh networks whose last hidden
// layer is at most 512 wide and a multiple of 32 features.
bool out_loss_tma_ok(int prec, int act, int w) {
  return prec == PINN_BF16 && act == PINN_ACT_TANH && w <= 512 && w % OT_FC == 0;
}

int out_loss_tma_blocks(int64_t NP, int sm_count) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(NP / TILE_PTS, 2 * (int64_t)std::max(sm_count, 1)));
}

static size_t ot_smem(int w, int d_out) {
  return (size_t)OT_STAGES * OT_STAGE + 1024 +
         sizeof(float) * (size_t)w * (d_out * (1 + OT_CONS / 32) + OT_CONS / 32) + 8 + 8 * 2 * OT_STAGES + 16;
}

template <int D, int MODE, bool LO>
cudaError_t out_loss_tma_launch(const CUtensorMap& ma, const CUtensorMap& ml, const OutArgs& a, int nblocks,
                                cudaStream_t st) {
  auto kern = k_out_loss_tma<D, MODE, LO>;
  const size_t smem = ot_smem(a.w, D);
  static size_t reserved = 0;
  if (smem > reserved) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    reserved = smem;
  }
  kern<<<nblocks, OT_THREADS, smem, st>>>(ma, ml, a);
  return cudaGetLastError();
}

// Returns cudaErrorNotSupported (nothing launched) when the tensor maps cannot be built.
cudaError_t launch_out_loss_tma(const OutArgs& a, int nblocks, cudaStream_t st) {
  CUtensorMap ma, ml;
  const uint64_t nt = (uint64_t)(a.NP / TILE_PTS);
  if (!tc_map3(&ma, a.AL, false, TILE_COLS, (uint64_t)a.w, nt, 64, OT_FC)) return cudaErrorNotSupported;
  ml = ma;
  if (a.ALlo && !tc_map3(&ml, a.ALlo, false, TILE_PTS, (uint64_t)a.w, nt, 64, OT_FC)) return cudaErrorNotSupported;
  const bool lo = a.ALlo != nullptr;
  if (a.d_out == 1 && a.jet_mode == JET_BURGERS)
    return lo ? out_loss_tma_launch<1, JET_BURGERS, true>(ma, ml, a, nblocks, st)
              : out_loss_tma_launch<1, JET_BURGERS, false>(ma, ml, a, nblocks, st);
  if (a.d_out == 3 && a.jet_mode == JET_NS)
    return lo ? out_loss_tma_launch<3, JET_NS, true>(ma, ml, a, nblocks, st)
              : out_loss_tma_launch<3, JET_NS, false>(ma, ml, a, nblocks, st);
  if (a.d_out == 3 && a.jet_mode == JET_MAXWELL)
    return lo ? out_loss_tma_launch<3, JET_MAXWELL, true>(ma, ml, a, nblocks, st)
              : out_loss_tma_launch<3, JET_MAXWELL, false>(ma, ml, a, nblocks, st);
  return cudaErrorNotSupported;
}

// ------------------------------------------------------------------------------------
// The output layer, residual, loss and adjoint seed for BF16 tanh networks whose last
// hidden layer is at most 256 wide, with the three contractions of width d_out on
// warp-level tensor-core MMAs (m16n8k16, BF16 operands, FP32 accumulation):
//   U     = W_out A_L           (rows: W_hi in MMA rows c, W_lo in rows 8 + c)
//   dW    = Ubar A_L^T          (rows: Ubar_hi in c, Ubar_lo in 8 + c)
//   Abar  = W_out^T Ubar        (k-slots: W_hi.Ubar_hi, W_lo.Ubar_hi, W_hi.Ubar_lo)
// The hi/lo splits make the products accurate to about 2^-16 relative, like the FP32
// weights and seeds of k_out_loss_tma.  tcgen05's smallest M is 64 and would leave 61
// of 64 accumulator lanes idle for d_out = 3; these MMAs keep the fragments in
// registers beside the residual and jet arithmetic.  The A_L chunks arrive through
// the same TMA ring (each slot released after a proxy fence, as there); the ldmatrix fragments the weight gradient reads from them are
// exactly the activations the tanh-jet adjoint needs for the same (feature, point)
// pairs.  The four warps stmatrix their adjoints into one staging chunk laid out like
// the load boxes, which leaves as four bulk tensor stores (per-lane 32-byte stores
// touch 32 lines per instruction and cost a fifth of the kernel).  Warp w (of four)
// owns points 16 w .. 16 w + 15 of every 64-point tile.  A failed bounded wait in any
// warp is ANDed over the warps at the next barrier, so they all leave together.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ldsm4(uint32_t addr, uint32_t r[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void ldsm4_t(uint32_t addr, uint32_t r[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void stsm4(uint32_t addr, const uint32_t r[4]) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(r[0]), "r"(r[1]),
               "r"(r[2]), "r"(r[3])
               : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

constexpr int OM_MAXW = 256;
constexpr int OM_SCRATCH = 3584;                  // per warp: U gather and seed fragments
constexpr int OM_STAGE_OUT = 4 * OT_ROWB;         // one chunk of Zbar_L (4 jet-row boxes), 16 KB
static_assert(4 * OM_SCRATCH <= OM_STAGE_OUT, "the seed scratch fits in the output staging");

// dynamic shared memory after the ring (byte offsets from the ring's start)
struct OmLayout {
  int stg, wa, wf, dw, db, bar, total;
  __host__ __device__ OmLayout(int w, int d) {
    stg = OT_STAGES * OT_STAGE;                   // Zbar_L chunk for the bulk store (1024-aligned, swizzled like
                                                  // the load boxes); between the passes, the per-warp seed scratch
    wa = stg + OM_STAGE_OUT;                      // W_hi / W_lo rows: bf16 [16][w + 8]
    wf = wa + 32 * (w + 8);                       // W^T fragments: u32 [w / 16][32 lanes][4]
    dw = wf + 32 * w;                             // dW accumulators: float [4 warps][d][w + 8]
    db = dw + 16 * d * (w + 8);                   // hidden-bias accumulators: float [4 warps][w]
    bar = db + 16 * w;                            // 2 OT_STAGES mbarriers + the abort flag
    total = bar + 16 * OT_STAGES + 16;
  }
};


template <int D, int MODE, bool LO>
__global__ void __launch_bounds__(OT_THREADS, 2) k_out_loss_mma(const __grid_constant__ CUtensorMap mapA,
                                                            const __grid_constant__ CUtensorMap mapLo,
                                                            const __grid_constant__ CUtensorMap mapZ, OutArgs a) {
  constexpr int NB = LO ? 5 : 4;                  // staged boxes per chunk: four jet rows (+ the low half)
  extern __shared__ uint8_t om_raw[];
  uint8_t* ring = om_raw + ((1024u - (smem_u32(om_raw) & 1023u)) & 1023u);
  const int w = a.w;
  const int was = w + 8;                          // sWA row stride (elements): conflict-free A fragments
  const OmLayout lay(w, D);
  __nv_bfloat16* sWA = reinterpret_cast<__nv_bfloat16*>(ring + lay.wa);
  uint32_t* sWf = reinterpret_cast<uint32_t*>(ring + lay.wf);
  float* sdw = reinterpret_cast<float*>(ring + lay.dw);
  float* sdb = reinterpret_cast<float*>(ring + lay.db);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + lay.bar);
  uint64_t* empty = full + OT_STAGES;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + OT_STAGES);
  __shared__ double segacc[CAUSAL_MAX][4];
  __shared__ int s_seg[TILE_PTS];
  __shared__ float s_rr[TILE_PTS][3];
  __shared__ double sh[OT_CONS / 32];
  __shared__ float shb[OT_CONS / 32];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OT_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], OT_CONS);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  // weights as MMA operands: W_hi rows c, W_lo rows 8 + c (zero elsewhere), and the
  // W^T fragments of every 16-feature m-tile with k-slots (W_hi, W_lo, W_hi)
  for (int i = threadIdx.x; i < 16 * was; i += blockDim.x) {
    const int row = i / was, f = i - row * was;
    float v = 0.f;
    if (f < w && (row & 7) < D) {
      const float x = a.W[(row & 7) * w + f];
      const float hi = __bfloat162float(__float2bfloat16_rn(x));
      v = row < 8 ? hi : x - hi;
    }
    sWA[i] = __float2bfloat16_rn(v);
  }
  for (int i = threadIdx.x; i < (w / 16) * 32; i += blockDim.x) {
    const int mt = i >> 5, l = i & 31, g = l >> 2, t = l & 3;
    auto wk = [&](int f, int k) -> float {     // W^T with k-slots
      const int c = k % D, part = k / D;
      if (part > 2) return 0.f;
      const float x = a.W[c * w + f];
      const float hi = __bfloat162float(__float2bfloat16_rn(x));
      return part == 1 ? x - hi : hi;
    };
    const int f0 = 16 * mt + g;
    uint32_t q[4];
    q[0] = pack_bf16(wk(f0, 2 * t), wk(f0, 2 * t + 1));
    q[1] = pack_bf16(wk(f0 + 8, 2 * t), wk(f0 + 8, 2 * t + 1));
    q[2] = pack_bf16(wk(f0, 2 * t + 8), wk(f0, 2 * t + 9));
    q[3] = pack_bf16(wk(f0 + 8, 2 * t + 8), wk(f0 + 8, 2 * t + 9));
#pragma unroll
    for (int j = 0; j < 4; ++j) sWf[4 * i + j] = q[j];
  }
  for (int i = threadIdx.x; i < 4 * D * (w + 8) + 4 * w; i += blockDim.x) sdw[i] = 0.f;   // sdw and sdb
  if (a.segpart)
    for (int i = threadIdx.x; i < CAUSAL_MAX * 4; i += blockDim.x) segacc[i / 4][i % 4] = 0.0;
  __syncthreads();

  const int64_t ntiles = a.NP / TILE_PTS;
  const int nchunks = w / OT_FC;
  const int passes = a.want_grad ? 2 : 1;

  if (warp == OT_CONS / 32) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed[OT_STAGES] = {};
      // the consumers' order: chunk k of the previous tile's second pass, then chunk k of
      // this tile's first pass, so every first-pass (DRAM) load leads its use by a
      // second-pass chunk
      bool live = true;
      auto load_chunk = [&](int k, int T) {
        if (!live || !mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.status, OT_WAIT_NS)) { live = false; return; }
        uint8_t* sb = ring + stage * OT_STAGE;
        mbar_expect_tx(&full[stage], NB * OT_ROWB);
        armed[stage] = (int)phase + 1;
#pragma unroll
        for (int r = 0; r < 4; ++r) tma_load_3d(sb + r * OT_ROWB, &mapA, &full[stage], 64 * r, OT_FC * k, T);
        if constexpr (LO) tma_load_3d(sb + 4 * OT_ROWB, &mapLo, &full[stage], 0, OT_FC * k, T);
        if (++stage == OT_STAGES) { stage = 0; phase ^= 1; }
      };
      int prevT = -1;
      for (int64_t T0i = blockIdx.x; live; T0i += gridDim.x) {
        const bool cur = T0i < ntiles;
        const bool prev = prevT >= 0;
        if (!cur && !prev) break;
        const int Tc = cur ? (int)(a.reverse ? ntiles - 1 - T0i : T0i) : 0;
        for (int k = 0; k < nchunks; ++k) {
          if (prev) load_chunk(k, prevT);
          if (cur) load_chunk(k, Tc);
        }
        prevT = (cur && passes == 2) ? Tc : -1;
      }
      for (int s = 0; s < OT_STAGES; ++s)
        if (armed[s]) {
          const uint64_t t0 = gtimer();
          while (!mbar_try(&full[s], (uint32_t)(armed[s] - 1)) && gtimer() - t0 < OT_WAIT_NS) {}
        }
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  const int g = lane >> 2, t = lane & 3;
  const int p0 = 16 * warp;                        // this warp's first point in a tile
  const int ck = p0 >> 3;                          // its first 16-byte chunk in a box row
  uint8_t* scr = ring + lay.stg + warp * OM_SCRATCH;
  float* sU = reinterpret_cast<float*>(scr);                                  // [16 points][D][4]
  __nv_bfloat16* sUd = reinterpret_cast<__nv_bfloat16*>(scr + 768);          // [hi/lo][4 rows][D][16 points]
  uint8_t* sUb = scr + 1536;                                                   // [4 rows][16 points][16 k] bf16
  const uint32_t stg = smem_u32(ring + lay.stg);                              // Zbar_L chunk staging
  const uint32_t sWA_u = smem_u32(sWA);
  const uint32_t sUd_u = smem_u32(sUd);
  const uint32_t sUb_u = smem_u32(sUb);
  float* sdw_w = sdw + warp * D * (w + 8);
  float* sdb_w = sdb + warp * w;
  Acc2 acc[5];
  float dbo[3] = {0.f, 0.f, 0.f};
  int stage = 0;
  uint32_t phase = 0;
  bool ok = true;
  // ldmatrix row address inside a box for (feature fi in the chunk, 16-byte point chunk c)
  auto box_row = [&](uint32_t box, int fi, int c) { return box + fi * 128 + ((c ^ (fi & 7)) << 4); };
  const int lm = lane >> 3, li = lane & 7;

  // Software pipeline over this block's tiles: in each round, chunk k of the previous
  // tile's second pass is followed by chunk k of the current tile's first pass.  A failed
  // bounded wait skips the work but still reaches the next ANDed barrier.
  int64_t prevT = -1;                              // the tile whose second pass is pending
  uint32_t ua[4][4], ub[4][2][2];                  // its seed fragments
  for (int64_t T0i = blockIdx.x;; T0i += gridDim.x) {
    const bool cur = T0i < ntiles;
    const bool prev = prevT >= 0;
    if (!cur && !prev) break;
    const int64_t Tc = cur ? (a.reverse ? ntiles - 1 - T0i : T0i) : 0;
    float acc1[NB][2][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc1[b][j][e] = 0.f;
    for (int k = 0; k < nchunks; ++k) {
      if (prev) {
      // ---------------- pass 2, chunk k of the previous tile: dW, Abar = W^T Ubar, its tanh-jet
      // adjoint, Zbar_L
      if (ok) ok = mbar_wait(&full[stage], phase, abort_flag, a.status, OT_WAIT_NS);
      // the staging is free once the previous chunk's bulk store has read it
      if (threadIdx.x == 0) bulk_wait_read0();
      ok = cons_sync_and(ok);
      if (!ok) break;   // (uniform: every consumer thread leaves the tile loop)
      const uint32_t sb = smem_u32(ring + stage * OT_STAGE);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int f0 = OT_FC * k + 16 * s;
        // A_L of features f0 .. f0 + 15 at the warp's points: matrices (features +0, points
        // +0), (+0, +8), (+8, +0), (+8, +8), each thread (feature g, points 2t, 2t + 1)
        uint32_t L[NB][4];
        const int fi = 16 * s + 8 * (lm >> 1) + li, c = ck + (lm & 1);
#pragma unroll
        for (int b = 0; b < NB; ++b) ldsm4(box_row(sb + b * OT_ROWB, fi, c), L[b]);
        // weight gradient of these 16 features (two n-tiles), K = the warp's points
        float dacc[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
          for (int e = 0; e < 4; ++e) dacc[nt][e] = 0.f;
#pragma unroll
          for (int b = 0; b < NB; ++b) mma_bf16_16816(dacc[nt], ua[b < 4 ? b : 0], L[b][2 * nt], L[b][2 * nt + 1]);
        }
        if (g < D) {
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            float* d = sdw_w + g * (w + 8) + f0 + 8 * nt + 2 * t;
            d[0] += dacc[nt][0] + dacc[nt][2];
            d[1] += dacc[nt][1] + dacc[nt][3];
          }
        }
        // the adjoint of the 16 features at the warp's 16 points x 4 rows
        uint32_t wfr[4];
        {
          const uint4 q = *reinterpret_cast<const uint4*>(sWf + 4 * ((f0 / 16) * 32 + lane));
          wfr[0] = q.x; wfr[1] = q.y; wfr[2] = q.z; wfr[3] = q.w;
        }
        float adj[4][2][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int e = 0; e < 4; ++e) adj[r][j][e] = 0.f;
            mma_bf16_16816(adj[r][j], wfr, ub[r][j][0], ub[r][j][1]);
          }
        // tanh-jet adjoint per (feature f0 + 8 fh + g, point p0 + 8 j + 2 t + e)
        uint32_t zp[2][4][2];
        float dbs[2] = {0.f, 0.f};
#pragma unroll
        for (int fh = 0; fh < 2; ++fh)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            float zo[2][4];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              float av[4], ab[4];
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const uint32_t u = L[r][2 * fh + j];
                av[r] = e ? bf16_hi(u) : bf16_lo(u);
                ab[r] = adj[r][j][2 * fh + e];
              }
              if constexpr (LO) {
                const uint32_t u = L[NB - 1][2 * fh + j];
                av[0] += e ? bf16_hi(u) : bf16_lo(u);
              }
              jet_adj_a(av, ab, zo[e], MODE);
              dbs[fh] += zo[e][0];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) zp[fh][r][j] = pack_bf16(zo[0][r], zo[1][r]);
          }
        // into the chunk's staging boxes (the load boxes' swizzled layout), at the rows
        // and 16-byte chunks this warp's ldmatrix read
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const uint32_t v[4] = {zp[0][r][0], zp[0][r][1], zp[1][r][0], zp[1][r][1]};
          stsm4(box_row(stg + r * OT_ROWB, fi, c), v);
        }
        if (a.dbhid) {
#pragma unroll
          for (int fh = 0; fh < 2; ++fh) {
            float x = dbs[fh];
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if (t == 0) sdb_w[f0 + 8 * fh + g] += x;
          }
        }
      }
      // the chunk's Zbar_L (32 features x 4 rows x 64 points) as four bulk tensor stores
      fence_proxy_async_smem();
      cons_sync();
      if (threadIdx.x == 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) tma_store_3d(&mapZ, ring + lay.stg + r * OT_ROWB, 64 * r, OT_FC * k, (int)prevT);
        bulk_commit();
      }
      mbar_arrive(&empty[stage]);
      if (++stage == OT_STAGES) { stage = 0; phase ^= 1; }
          }
      if (cur) {
      // ---------------- pass 1, chunk k of this tile: U = W_out A_L for this warp's 16 points
      if (ok) ok = mbar_wait(&full[stage], phase, abort_flag, a.status, OT_WAIT_NS);
      if (ok) {
      const uint32_t sb = smem_u32(ring + stage * OT_STAGE);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int f0 = OT_FC * k + 16 * s;
        uint32_t af[4];
        const uint32_t wa = sWA_u + 2 * (f0 + 2 * t);
        af[0] = lds32(wa + 2 * g * was);
        af[1] = lds32(wa + 2 * (g + 8) * was);
        af[2] = lds32(wa + 2 * g * was + 16);
        af[3] = lds32(wa + 2 * (g + 8) * was + 16);
        // B fragments (k = features, n = points) through the transposing load:
        // matrices (features +0/+8, points +0/+8) in the order n-tile 0 (k lo, k hi), n-tile 1
        const int fi = 16 * s + 8 * (lm & 1) + li, c = ck + (lm >> 1);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          uint32_t r[4];
          ldsm4_t(box_row(sb + b * OT_ROWB, fi, c), r);
          mma_bf16_16816(acc1[b][0], af, r[0], r[1]);
          mma_bf16_16816(acc1[b][1], af, r[2], r[3]);
        }
      }
      fence_proxy_async_smem();   // these reads before the producer's next bulk copy into the slot
      mbar_arrive(&empty[stage]);
      if (++stage == OT_STAGES) { stage = 0; phase ^= 1; }
      }
      }
    }
    // (a failed first-pass wait is not uniform: it reaches the ANDed barrier below)
    if (!cur) break;
    // every warp is through its first pass, and the last bulk store has read the staging
    // (the seed scratch below shares it)
    if (threadIdx.x == 0) bulk_wait_read0();
    ok = cons_sync_and(ok);
    if (!ok) break;

    // ---------------- U to the point lanes, residual, seeds
    if (g < D) {
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            float u = acc1[b][j][e] + acc1[b][j][2 + e];
            if constexpr (LO) {
              if (b == 0) u += acc1[NB - 1][j][e] + acc1[NB - 1][j][2 + e];
            }
            const int q = 8 * j + 2 * t + e;
            sU[(q * D + g) * 4 + b] = u;
          }
    }
    __syncwarp();
    float rr[3] = {0.f, 0.f, 0.f};
    int seg = -1;
    if (lane < 16) {
      const int q = lane;
      float U[3][4], Ub[3][4];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) U[c][r] = c < D ? sU[(q * D + c) * 4 + r] : 0.f;
      int64_t idx;
      const int set = point_set(Tc * TILE_PTS + p0 + q, a.n_res, a.n_ic, a.n_bc, idx);
      if (set != SET_PAD) {
#pragma unroll
        for (int c = 0; c < D; ++c) U[c][0] += a.b[c];
      }
      float kp = a.k_pde;
      if (a.segments && set == SET_RES) {
        const float tt = a.x_res[(int64_t)a.t_index * a.n_res + idx];
        seg = min(a.segments - 1, max(0, (int)floorf((tt - a.t0) * a.tinv)));
        if (a.seg_scale) kp = a.seg_scale[seg];
      }
      float lacc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      point_residual<D>(a, set, idx, kp, U, Ub, lacc, rr);
#pragma unroll
      for (int i = 0; i < 5; ++i) acc[i].add(lacc[i]);
      if (a.want_grad) {
#pragma unroll
        for (int c = 0; c < D; ++c) dbo[c] += Ub[c][0];
        // seed fragments: Ubar_hi / Ubar_lo per (row, output) over the warp's points,
        // and per (row, point) the 16 k-slots (Ubar_hi, Ubar_hi, Ubar_lo, zeros)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float kv[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) kv[i] = 0.f;
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const __nv_bfloat16 hb = __float2bfloat16_rn(Ub[c][r]);
            const float hi = __bfloat162float(hb);
            const float lo = Ub[c][r] - hi;
            sUd[((0 * 4 + r) * D + c) * 16 + q] = hb;
            sUd[((1 * 4 + r) * D + c) * 16 + q] = __float2bfloat16_rn(lo);
            kv[c] = hi;
            kv[D + c] = hi;
            kv[2 * D + c] = lo;
          }
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) pk[i] = pack_bf16(kv[2 * i], kv[2 * i + 1]);
          uint4* dst = reinterpret_cast<uint4*>(sUb + (r * 16 + q) * 32);
          dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
      }
    }
    if (a.segpart) {   // uniform over the block
      if (lane < 16) {
        s_seg[p0 + lane] = seg;
        s_rr[p0 + lane][0] = rr[0]; s_rr[p0 + lane][1] = rr[1]; s_rr[p0 + lane][2] = rr[2];
      }
      cons_sync();
      if (threadIdx.x == 0)
        for (int q = 0; q < TILE_PTS; ++q)
          if (s_seg[q] >= 0) {
            double* sa = segacc[s_seg[q]];
            sa[0] += s_rr[q][0]; sa[1] += s_rr[q][1]; sa[2] += s_rr[q][2]; sa[3] += 1.0;
          }
      cons_sync();
    }
    if (a.want_grad) {
    __syncwarp();
    // weight-gradient A fragments (rows: Ubar_hi c, Ubar_lo 8 + c; k = the row's 16 points)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const bool live = g < D;
      const uint32_t hrow = sUd_u + 2 * (((0 * 4 + r) * D + (live ? g : 0)) * 16 + 2 * t);
      const uint32_t lrow = sUd_u + 2 * (((1 * 4 + r) * D + (live ? g : 0)) * 16 + 2 * t);
      ua[r][0] = live ? lds32(hrow) : 0u;
      ua[r][1] = live ? lds32(lrow) : 0u;
      ua[r][2] = live ? lds32(hrow + 16) : 0u;
      ua[r][3] = live ? lds32(lrow + 16) : 0u;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t kc = sUb_u + (r * 16 + 8 * j + g) * 32 + 4 * t;   // point 8 j + g, k-slots 2t, 2t+1 (+8)
        ub[r][j][0] = lds32(kc);
        ub[r][j][1] = lds32(kc + 16);
      }
    }
    __syncwarp();   // the scratch is the store staging from here on
    }

    prevT = a.want_grad ? Tc : -1;
  }
  if (threadIdx.x == 0) bulk_wait0();   // every bulk store has completed
  for (int i = 0; i < 5; ++i) {
    const double s = cons_sum_d(acc[i].value(), sh);
    if (threadIdx.x == 0) a.losspart[(int64_t)blockIdx.x * 8 + i] = s;
  }
  if (a.segpart) {
    cons_sync();
    for (int i = threadIdx.x; i < CAUSAL_MAX * 4; i += OT_CONS)
      a.segpart[(int64_t)blockIdx.x * CAUSAL_MAX * 4 + i] = segacc[i / 4][i % 4];
  }
  if (!a.want_grad) return;
  cons_sync();
  for (int i = threadIdx.x; i < D * w; i += OT_CONS) {
    const int c = i / w, f = i - c * w;
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < OT_CONS / 32; ++k) s += sdw[(k * D + c) * (w + 8) + f];
    a.dwpart[(int64_t)blockIdx.x * D * w + i] = s;
  }
  if (a.dbhid)
    for (int i = threadIdx.x; i < w; i += OT_CONS) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < OT_CONS / 32; ++k) s += sdb[k * w + i];
      a.dbhid[(int64_t)i * gridDim.x + blockIdx.x] = s;
    }
  for (int c = 0; c < D; ++c) {
    float v = dbo[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    cons_sync();
    if (lane == 0) shb[warp] = v;
    cons_sync();
    if (threadIdx.x == 0) {
      float tsum = 0.f;
      for (int k = 0; k < OT_CONS / 32; ++k) tsum += shb[k];
      a.dbpart[(int64_t)c * gridDim.x + blockIdx.x] = tsum;
    }
  }
}

// Whether the MMA output kernel applies: BF16 tanh networks whose last hidden layer is
// at most 256 wide and a multiple of 32 features.
bool out_loss_mma_ok(int prec, int act, int w) {
  return prec == PINN_BF16 && act == PINN_ACT_TANH && w <= OM_MAXW && w % OT_FC == 0;
}

template <int D, int MODE, bool LO>
cudaError_t out_loss_mma_launch(const CUtensorMap& ma, const CUtensorMap& ml, const CUtensorMap& mz, const OutArgs& a,
                                int nblocks, cudaStream_t st) {
  auto kern = k_out_loss_mma<D, MODE, LO>;
  const size_t smem = (size_t)OmLayout(a.w, D).total + 1024;
  static size_t reserved = 0;
  if (smem > reserved) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    reserved = smem;
  }
  kern<<<nblocks, OT_THREADS, smem, st>>>(ma, ml, mz, a);
  return cudaGetLastError();
}

cudaError_t launch_out_loss_mma(const OutArgs& a, int nblocks, cudaStream_t st) {
  CUtensorMap ma, ml, mz;
  const uint64_t nt = (uint64_t)(a.NP / TILE_PTS);
  if (!tc_map3(&ma, a.AL, false, TILE_COLS, (uint64_t)a.w, nt, 64, OT_FC)) return cudaErrorNotSupported;
  // Zbar_L has A_L's layout: the same boxes serve the bulk stores (loss-only calls store nothing)
  mz = ma;
  if (a.want_grad && !tc_map3(&mz, a.Zbar, false, TILE_COLS, (uint64_t)a.w, nt, 64, OT_FC)) return cudaErrorNotSupported;
  ml = ma;
  if (a.ALlo && !tc_map3(&ml, a.ALlo, false, TILE_PTS, (uint64_t)a.w, nt, 64, OT_FC)) return cudaErrorNotSupported;
  const bool lo = a.ALlo != nullptr;
  if (a.d_out == 1 && a.jet_mode == JET_BURGERS)
    return lo ? out_loss_mma_launch<1, JET_BURGERS, true>(ma, ml, mz, a, nblocks, st)
              : out_loss_mma_launch<1, JET_BURGERS, false>(ma, ml, mz, a, nblocks, st);
  if (a.d_out == 3 && a.jet_mode == JET_NS)
    return lo ? out_loss_mma_launch<3, JET_NS, true>(ma, ml, mz, a, nblocks, st)
              : out_loss_mma_launch<3, JET_NS, false>(ma, ml, mz, a, nblocks, st);
  if (a.d_out == 3 && a.jet_mode == JET_MAXWELL)
    return lo ? out_loss_mma_launch<3, JET_MAXWELL, true>(ma, ml, mz, a, nblocks, st)
              : out_loss_mma_launch<3, JET_MAXWELL, false>(ma, ml, mz, a, nblocks, st);
  return cudaErrorNotSupported;
}


template <typename T, int D, bool FAST, bool SINE>
cudaError_t out_loss_launch(const OutArgs& a, int nblocks, size_t smem, cudaStream_t st) {
  auto kern = k_out_loss<T, D, FAST, SINE>;
  // weights + per-warp dW accumulators: up to 120 KB for 2048-wide, 3-output networks
  static size_t reserved = 48 * 1024;
  if (smem > reserved) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    reserved = smem;
  }
  kern<<<nblocks, OUT_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_out_loss(const OutArgs& a, int prec, int nblocks, cudaStream_t st) {
  if (!a.ZL && out_loss_mma_ok(prec, PINN_ACT_TANH, a.w)) {
    const cudaError_t e = launch_out_loss_mma(a, nblocks, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (!a.ZL && out_loss_tma_ok(prec, PINN_ACT_TANH, a.w)) {
    const cudaError_t e = launch_out_loss_tma(a, nblocks, st);
    if (e != cudaErrorNotSupported) return e;
  }
  const size_t smem = sizeof(float) * a.w * (a.d_out * (1 + OUT_THREADS / 32) + OUT_THREADS / 32);
  // the sine adjoint (from stored pre-activations) is a separate instantiation, so the
  // tanh kernels carry none of its registers
  if (a.ZL) {
    if (prec == PINN_BF16)
      return a.d_out == 1 ? out_loss_launch<__nv_bfloat16, 1, true, true>(a, nblocks, smem, st)
                          : out_loss_launch<__nv_bfloat16, 3, true, true>(a, nblocks, smem, st);
    return a.d_out == 1 ? out_loss_launch<float, 1, false, true>(a, nblocks, smem, st)
                        : out_loss_launch<float, 3, false, true>(a, nblocks, smem, st);
  }
  if (prec == PINN_BF16)
    return a.d_out == 1 ? out_loss_launch<__nv_bfloat16, 1, true, false>(a, nblocks, smem, st)
                        : out_loss_launch<__nv_bfloat16, 3, true, false>(a, nblocks, smem, st);
  return a.d_out == 1 ? out_loss_launch<float, 1, false, false>(a, nblocks, smem, st)
                      : out_loss_launch<float, 3, false, false>(a, nblocks, smem, st);
}


// ------------------------------------------------------------------------------------
// Row reductions over a pre-activation adjoint Zbar^T [M][NC]: the bias gradient
// (value columns only) and, for a first layer applied to raw coordinates, the
// coordinate part of dW: dW_ij = sum_value zbar x_j + sum_{rows k with direction j} zbar_k.
// One warp per (row, column chunk); partials [chunk][M][1 + d_in_terms].
// ------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------
// Row reductions over a pre-activation adjoint Zbar^T [M][NC]: the bias gradient
// (value rows; padding and derivative rows of initial/boundary points are zero) and,
// for a first layer applied to raw coordinates, the coordinate part of dW:
// dW_ij = sum_points zbar x_j + sum_{rows k with direction j} zbar_k.
// One warp per (row, chunk of points), one lane per point; partials
// [M][nbpart][1 + dterms] in a fixed order (deterministic).
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void k_row_reduce(const T* Zb, int M, int64_t NP, int64_t n_res, int64_t n_ic, int64_t n_bc, int nbpart,
                             const float* x_res, const float* x_ic, const float* x_bc, int dterms, int mode,
                             float* part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + warp;
  if (row >= M) return;
  const int chunk = blockIdx.y;
  const int64_t per = (NP + nbpart - 1) / nbpart;
  const int64_t p0 = chunk * per, p1 = min(NP, p0 + per);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int64_t p = p0 + lane; p < p1; p += 32) {
    const float v0 = to_f<T>(Zb[toff(row, jcol(p, 0), M)]);
    acc[0] += v0;
    if (dterms) {
      for (int j = 0; j < dterms; ++j)
        acc[1 + j] = fmaf(v0, point_coord(x_res, x_ic, x_bc, n_res, n_ic, n_bc, p, j), acc[1 + j]);
      for (int r = 1; r < 4; ++r) {
        const int d = row_dir(mode, r);
        if (d >= 0) acc[1 + d] += to_f<T>(Zb[toff(row, jcol(p, r), M)]);
      }
    }
  }
  for (int j = 0; j <= dterms; ++j) {
    float s = acc[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[((int64_t)row * nbpart + chunk) * (1 + dterms) + j] = s;
  }
}

void launch_row_reduce(const void* Zbar, bool fp32_in, int M, int64_t NP, int64_t n_res, int64_t n_ic, int64_t n_bc,
                       int nbpart, const float* x_res, const float* x_ic, const float* x_bc, int dterms, int mode,
                       float* part, int prec, cudaStream_t st) {
  dim3 grid((M + 7) / 8, nbpart);
  if (prec == PINN_BF16 && !fp32_in)
    k_row_reduce<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)Zbar, M, NP, n_res, n_ic, n_bc, nbpart,
                                                      x_res, x_ic, x_bc, dterms, mode, part);
  else
    k_row_reduce<float><<<grid, 256, 0, st>>>((const float*)Zbar, M, NP, n_res, n_ic, n_bc, nbpart, x_res, x_ic,
                                              x_bc, dterms, mode, part);
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

__device__ __forceinline__ void put_grad(const FinalizeArgs& a, int64_t idx, float v) {
  a.grad[idx] = a.accumulate ? a.grad[idx] + v : v;
}

// Each block is bound by memory latency, not bandwidth: its threads keep 8 partial
// loads in flight (the splits of a row then take a few memory latencies instead of
// one per split), the bias partials are read as float4, and 128-thread blocks at
// most 40 registers keep the whole grid resident in one wave.
constexpr int FIN_THREADS = 128;
constexpr int FIN_UNROLL = 8;

__global__ void __launch_bounds__(FIN_THREADS, 12) k_finalize_grad(FinalizeArgs a) {
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
  {
    Acc2 ab[4];
    if (!raw && (nbp & 3) == 0) {
      // one row's bias partials are contiguous: float4 p4 = t, t + T, ..., each
      // summed in element order
      const float4* q4 = reinterpret_cast<const float4*>(dbp + (int64_t)i * nbp);
      const int n4 = nbp >> 2, T = blockDim.x;
      // batches of four loads in flight, the last one predicated (same order of adds)
      for (int p4 = threadIdx.x; p4 < n4; p4 += 4 * T) {
        float4 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = (p4 + u * T < n4) ? __ldcs(q4 + p4 + u * T) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (p4 + u * T < n4) { ab[0].add(x[u].x); ab[0].add(x[u].y); ab[0].add(x[u].z); ab[0].add(x[u].w); }
      }
    } else {
      for (int p = threadIdx.x; p < nbp; p += blockDim.x) {
        const float* q = dbp + ((int64_t)i * nbp + p) * dbs;
        ab[0].add(q[0]);
        if (raw)
          for (int j = 0; j < fin && j < 3; ++j) ab[1 + j].add(q[1 + j]);
      }
    }
    v[1] = ab[0].value();
    for (int j = 0; j < 3; ++j) v[2 + j] = ab[1 + j].value();
  }
  if (!raw) {
    const float* part = reinterpret_cast<const float*>(a.ws + a.dwpart[l]);
    const int ns = a.nsplit[l];
    const int64_t sstride = (int64_t)fout * fin;
    if ((fin & 3) == 0 && fin / 4 <= (int)blockDim.x) {
      // G thread groups each sum every G-th split of the same float4 column; the
      // groups are then combined in a fixed order (deterministic).
      __shared__ double shd[FIN_THREADS][4];
      const int ncol4 = fin / 4;
      const int G = blockDim.x / ncol4;
      const int q = threadIdx.x % ncol4, g = threadIdx.x / ncol4;
      double d[4] = {0.0, 0.0, 0.0, 0.0};
      if (g < G) {
        const float* base = part + (int64_t)i * fin + 4 * q;
        Acc2 a0, a1, a2, a3;
        // splits g, g + G, g + 2G, ... in that order; the loads of FIN_UNROLL splits
        // are issued before any of them is added (the partials are read once: streaming),
        // and the remaining splits form one more batch, predicated, instead of a chain
        // of single loads each waiting for the one before
        int s = g;
        for (; s + (FIN_UNROLL - 1) * G < ns; s += FIN_UNROLL * G) {
          float4 x[FIN_UNROLL];
#pragma unroll
          for (int u = 0; u < FIN_UNROLL; ++u)
            x[u] = __ldcs(reinterpret_cast<const float4*>(base + (int64_t)(s + u * G) * sstride));
#pragma unroll
          for (int u = 0; u < FIN_UNROLL; ++u) { a0.add(x[u].x); a1.add(x[u].y); a2.add(x[u].z); a3.add(x[u].w); }
        }
        if (s < ns) {
          float4 x[FIN_UNROLL - 1];
#pragma unroll
          for (int u = 0; u < FIN_UNROLL - 1; ++u)
            if (s + u * G < ns) x[u] = __ldcs(reinterpret_cast<const float4*>(base + (int64_t)(s + u * G) * sstride));
#pragma unroll
          for (int u = 0; u < FIN_UNROLL - 1; ++u)
            if (s + u * G < ns) { a0.add(x[u].x); a1.add(x[u].y); a2.add(x[u].z); a3.add(x[u].w); }
        }
        d[0] = a0.value(); d[1] = a1.value(); d[2] = a2.value(); d[3] = a3.value();
      }
      for (int k = 0; k < 4; ++k) shd[threadIdx.x][k] = d[k];
      __syncthreads();
      if (g == 0) {
        for (int gg = 1; gg < G; ++gg)
          for (int k = 0; k < 4; ++k) d[k] += shd[gg * ncol4 + q][k];
        for (int k = 0; k < 4; ++k) {
          put_grad(a, a.offV[l] + (int64_t)i * fin + 4 * q + k, (float)(d[k] * es));
          v[0] += d[k] * (double)W[4 * q + k];
        }
      }
    } else if ((fin & 3) == 0) {
      for (int j4 = threadIdx.x * 4; j4 < fin; j4 += blockDim.x * 4) {
        Acc2 a0, a1, a2, a3;
        const float* q = part + (int64_t)i * fin + j4;
#pragma unroll 4
        for (int s = 0; s < ns; ++s) {
          const float4 x = *reinterpret_cast<const float4*>(q + s * sstride);
          a0.add(x.x); a1.add(x.y); a2.add(x.z); a3.add(x.w);
        }
        const double dd[4] = {a0.value(), a1.value(), a2.value(), a3.value()};
        for (int k = 0; k < 4; ++k) {
          put_grad(a, a.offV[l] + (int64_t)i * fin + j4 + k, (float)(dd[k] * es));
          v[0] += dd[k] * (double)W[j4 + k];
        }
      }
    } else {
      for (int j = threadIdx.x; j < fin; j += blockDim.x) {
        Acc2 acc;
        for (int s = 0; s < ns; ++s) acc.add(part[s * sstride + (int64_t)i * fin + j]);
        const double dW = acc.value();
        put_grad(a, a.offV[l] + (int64_t)i * fin + j, (float)(dW * es));
        v[0] += dW * (double)W[j];
      }
    }
  }
  block_sum_n<5>(v, sh);
  if (threadIdx.x == 0) {
    if (raw) {
      for (int j = 0; j < fin && j < 3; ++j) {
        put_grad(a, a.offV[l] + (int64_t)i * fin + j, (float)(v[2 + j] * es));
        v[0] += v[2 + j] * (double)W[j];
      }
    }
    if (a.rwf) put_grad(a, a.offs[l] + i, (float)v[0]);
    put_grad(a, a.offb[l] + i, (float)v[1]);
  }
}

void launch_finalize_grad(const FinalizeArgs& a, cudaStream_t st) {
  int maxout = 1;
  for (int l = 0; l < a.L1; ++l) maxout = std::max(maxout, a.fout[l]);
  dim3 grid(maxout, a.L1);
  k_finalize_grad<<<grid, FIN_THREADS, 0, st>>>(a);
}

__global__ void k_finalize_loss(const double* part, int nblocks, int64_t n_res, int64_t n_ic, int64_t n_bc,
                                double lam_pde, double lam_ic, double lam_bc, double* out, double* acc, int first,
                                int last, int* status) {
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
    double t[5];
    for (int i = 0; i < 5; ++i) t[i] = (first ? 0.0 : acc[i]) + sh[i][0];
    if (!last) {
      for (int i = 0; i < 5; ++i) acc[i] = t[i];
      return;
    }
    // each term is a mean over its own set (Eqs. 10-12), summed over equations
    const double e0 = n_res ? t[0] / n_res : 0.0, e1 = n_res ? t[1] / n_res : 0.0, e2 = n_res ? t[2] / n_res : 0.0;
    const double lic = n_ic ? t[3] / n_ic : 0.0, lbc = n_bc ? t[4] / n_bc : 0.0;
    const double lpde = e0 + e1 + e2;
    const double tot = lam_pde * lpde + lam_ic * lic + lam_bc * lbc;
    out[0] = tot; out[1] = lpde; out[2] = e0; out[3] = e1; out[4] = e2; out[5] = lic; out[6] = lbc; out[7] = 0.0;
    if (!isfinite(tot)) atomicOr(status, 1);
  }
}

void launch_finalize_loss(const double* part, int nblocks, int64_t n_res, int64_t n_ic, int64_t n_bc, double lam_pde,
                          double lam_ic, double lam_bc, double* out, double* acc, int first, int last, int* status,
                          cudaStream_t st) {
  k_finalize_loss<<<1, 256, 0, st>>>(part, nblocks, n_res, n_ic, n_bc, lam_pde, lam_ic, lam_bc, out, acc, first, last,
                                     status);
}

// ------------------------------------------------------------------------------------
// Temporal causality (Sec. 2.6.8, Eqs. 20-21).  Thread (i, e) sums segment i's
// equation-e partials over the blocks in order; thread 0 then forms the segment
// losses L^i = sum_e S_ie / N_i, omega_1 = 1, omega_i = exp(-eps sum_{k<i} L^k), the
// weighted PDE term (1/M) sum_i omega_i L^i (and per equation), and the seed scales.
// ------------------------------------------------------------------------------------
__global__ void k_finalize_causal(const double* segpart, const double* losspart, int nblocks, int M, double eps,
                                  int64_t n_ic, int64_t n_bc, double lam_pde, double lam_ic, double lam_bc,
                                  double lam_seed, double* out, double* omega, float* scale, int* status) {
  __shared__ double S[CAUSAL_MAX][4];
  __shared__ double ib[2];
  const int t = threadIdx.x;
  if (t < M * 4) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += segpart[(int64_t)b * CAUSAL_MAX * 4 + t];
    S[t / 4][t % 4] = s;
  } else if (t >= 128 && t < 130) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += losspart[(int64_t)b * 8 + 3 + (t - 128)];
    ib[t - 128] = s;
  }
  __syncthreads();
  if (t != 0) return;
  double cum = 0.0, pe[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < M; ++i) {
    const double n = S[i][3];
    const double w = exp(-eps * cum);             // omega_i from the segments before i
    double Li = 0.0;
    for (int e = 0; e < 3; ++e) {
      const double le = n > 0.0 ? S[i][e] / n : 0.0;
      pe[e] += w * le / M;
      Li += le;
    }
    cum += Li;
    omega[i] = w;
    scale[i] = n > 0.0 ? (float)(lam_seed * w / (M * n)) : 0.f;
  }
  const double lic = n_ic ? ib[0] / n_ic : 0.0, lbc = n_bc ? ib[1] / n_bc : 0.0;
  const double lpde = pe[0] + pe[1] + pe[2];
  const double tot = lam_pde * lpde + lam_ic * lic + lam_bc * lbc;
  out[0] = tot; out[1] = lpde; out[2] = pe[0]; out[3] = pe[1]; out[4] = pe[2]; out[5] = lic; out[6] = lbc; out[7] = 0.0;
  if (!isfinite(tot)) atomicOr(status, 1);
}

void launch_finalize_causal(const double* segpart, const double* losspart, int nblocks, int M, double eps,
                            int64_t n_ic, int64_t n_bc, double lam_pde, double lam_ic, double lam_bc, double lam_seed,
                            double* out, double* omega, float* scale, int* status, cudaStream_t st) {
  k_finalize_causal<<<1, 256, 0, st>>>(segpart, losspart, nblocks, M, eps, n_ic, n_bc, lam_pde, lam_ic, lam_bc,
                                       lam_seed, out, omega, scale, status);
}

// ------------------------------------------------------------------------------------
// Gradient of the input map.  The Fourier embedding (Eq. 14) has, per feature j with
// phi = sum_e x_e B_ej, c = cos phi, s = sin phi, the jets  value [c, s];  row of
// direction d [-s B_dj, c B_dj];  second-order row [-c q, -s q], q = sum_{k in S} B_kj^2.
// Their derivatives with respect to B_ej (dphi/dB_ej = x_e):
//   value            [-s x_e, c x_e]
//   direction d      [-c x_e B_dj - s [d=e],  -s x_e B_dj + c [d=e]]
//   second order     [s x_e q - 2 c B_ej [e in S],  -c x_e q - 2 s B_ej [e in S]]
// dL/dB_ej = sum over points and rows of Abar_0 (the adjoint of these jets) times them.
// Grid (FFG_BLOCKS, m): block (b, j) reduces its points' terms for feature j in FP64.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void k_ff_grad(const T* __restrict__ Abar, const float* x_res, const float* x_ic, const float* x_bc,
                          int64_t n_res, int64_t n_ic, int64_t n_bc, int d_in, const float* B, int m, int mode,
                          int64_t NP, double* part) {
  const int j = blockIdx.y;
  float Bj[3] = {0.f, 0.f, 0.f};
  for (int i = 0; i < d_in; ++i) Bj[i] = B[(int64_t)i * m + j];
  const float q = (mode == JET_MAXWELL) ? 0.f : (Bj[0] * Bj[0] + (mode == JET_NS ? Bj[1] * Bj[1] : 0.f));
  const int64_t wA = 2 * (int64_t)m;
  double g[3] = {0.0, 0.0, 0.0};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < NP; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx;
    const int set = point_set(p, n_res, n_ic, n_bc, idx);
    if (set == SET_PAD) continue;
    float x[3] = {0.f, 0.f, 0.f};
    float phi = 0.f;
    for (int i = 0; i < d_in; ++i) {
      x[i] = point_coord(x_res, x_ic, x_bc, n_res, n_ic, n_bc, p, i);
      phi = fmaf(x[i], Bj[i], phi);
    }
    float sn, cs;
    sincosf(phi, &sn, &cs);
    const int nr = (set == SET_RES) ? 4 : 1;   // initial/boundary points carry the value row only
    float ac[4], as[4];
    for (int r = 0; r < nr; ++r) {
      ac[r] = to_f<T>(Abar[toff(j, jcol(p, r), wA)]);
      as[r] = to_f<T>(Abar[toff(m + j, jcol(p, r), wA)]);
    }
    for (int e = 0; e < d_in; ++e) {
      float ge = (cs * as[0] - sn * ac[0]) * x[e];
      for (int r = 1; r < nr; ++r) {
        const int d = row_dir(mode, r);
        if (d >= 0) {
          ge += ac[r] * (-cs * x[e] * Bj[d] - (d == e ? sn : 0.f)) + as[r] * (-sn * x[e] * Bj[d] + (d == e ? cs : 0.f));
        } else {
          const bool in_s = (e == 0) || (mode == JET_NS && e == 1);
          ge += ac[r] * (sn * x[e] * q - (in_s ? 2.f * cs * Bj[e] : 0.f)) +
                as[r] * (-cs * x[e] * q - (in_s ? 2.f * sn * Bj[e] : 0.f));
        }
      }
      g[e] += (double)ge;
    }
  }
  __shared__ double sh[8];
  for (int e = 0; e < d_in; ++e) {
    const double v = block_sum_d(g[e], sh);
    if (threadIdx.x == 0) part[((int64_t)j * gridDim.x + blockIdx.x) * d_in + e] = v;
  }
}

void launch_ff_grad(const void* Abar0, const float* x_res, const float* x_ic, const float* x_bc, int64_t n_res,
                    int64_t n_ic, int64_t n_bc, int d_in, const float* B, int m, int jet_mode, int64_t NP,
                    double* part, int prec, cudaStream_t st) {
  dim3 grid(FFG_BLOCKS, m);
  if (prec == PINN_BF16)
    k_ff_grad<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)Abar0, x_res, x_ic, x_bc, n_res, n_ic, n_bc,
                                                   d_in, B, m, jet_mode, NP, part);
  else
    k_ff_grad<float><<<grid, 256, 0, st>>>((const float*)Abar0, x_res, x_ic, x_bc, n_res, n_ic, n_bc, d_in, B, m,
                                           jet_mode, NP, part);
}

struct PeriodFactors { double f[3]; };

// Ordered FP64 sum of the block partials; one thread per output entry.
__global__ void k_ff_grad_final(const double* part, int d_in, int m, int periodic, PeriodFactors pf, int accumulate,
                                float* out) {
  const int n = periodic ? d_in : d_in * m;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int e = periodic ? t : t / m, j = periodic ? t : t % m;
    double s = 0.0;
    for (int b = 0; b < FFG_BLOCKS; ++b) s += part[((int64_t)j * FFG_BLOCKS + b) * d_in + e];
    if (periodic) s *= pf.f[e];
    out[t] = accumulate ? (float)((double)out[t] + s) : (float)s;
  }
}

void launch_ff_grad_final(const double* part, int d_in, int m, bool periodic, const double* periods, int accumulate,
                          float* out, cudaStream_t st) {
  PeriodFactors pf{{0.0, 0.0, 0.0}};
  if (periodic)   // B_kk = 2 pi / P_k, so dB_kk/dP_k = -2 pi / P_k^2
    for (int k = 0; k < d_in; ++k) pf.f[k] = -2.0 * 3.14159265358979323846 / (periods[k] * periods[k]);
  const int n = periodic ? d_in : d_in * m;
  k_ff_grad_final<<<(n + 255) / 256, 256, 0, st>>>(part, d_in, m, periodic ? 1 : 0, pf, accumulate, out);
}

// ------------------------------------------------------------------------------------
// Loss balancing (Sec. 2.6.4, Eqs. 18-19).  Stage 1: per (block, term) sums of squares;
// stage 2 (one thread): the norms in a fixed order, then the weights.
// ------------------------------------------------------------------------------------
constexpr int LB_BLOCKS = 64;
__global__ void k_sumsq(const float* __restrict__ g, int64_t P, double* part) {
  const int term = blockIdx.y;
  const float* x = g + (int64_t)term * P;
  Acc2 acc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    acc.add(x[i] * x[i]);
  __shared__ double sh[256 / 32];
  const double s = block_sum_d(acc.value(), sh);
  if (threadIdx.x == 0) part[term * LB_BLOCKS + blockIdx.x] = s;
}
__global__ void k_balance(const double* part, double* lambda, double* norms, double alpha, double eps, int update) {
  if (threadIdx.x != 0) return;
  double n[3], sum = 0.0;
  for (int t = 0; t < 3; ++t) {
    double s = 0.0;
    for (int b = 0; b < LB_BLOCKS; ++b) s += part[t * LB_BLOCKS + b];
    n[t] = sqrt(s);
    sum += n[t];
    if (norms) norms[t] = n[t];
  }
  if (!update) return;
  for (int t = 0; t < 3; ++t) {
    if (n[t] == 0.0) continue;   // a term without points keeps its weight
    const double hat = sum / (n[t] + eps);
    lambda[t] = alpha * lambda[t] + (1.0 - alpha) * hat;
  }
}
void launch_loss_balance(const float* g, int64_t P, double* lambda, double* norms, double alpha, double eps,
                         int update, double* part, cudaStream_t st) {
  k_sumsq<<<dim3(LB_BLOCKS, 3), 256, 0, st>>>(g, P, part);
  k_balance<<<1, 32, 0, st>>>(part, lambda, norms, alpha, eps, update);
}

// ------------------------------------------------------------------------------------
// Ordered partial-sum compaction: in [S][n] -> out [S2][n], slot k summing splits
// k*ceil(S/S2) .. in order (compensated), so the finalisation reads S2 splits.
// ------------------------------------------------------------------------------------
__global__ void k_sum_splits(const float* __restrict__ in, float* __restrict__ out, int S, int S2, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= n) return;
  const int per = (S + S2 - 1) / S2;
  const int s0 = k * per, s1 = min(S, s0 + per);
  Acc2 acc;
  for (int s = s0; s < s1; ++s) acc.add(in[(int64_t)s * n + i]);
  out[(int64_t)k * n + i] = (float)acc.value();
}

void launch_sum_splits(const float* in, float* out, int S, int S2, int64_t n, cudaStream_t st) {
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)S2);
  k_sum_splits<<<grid, 256, 0, st>>>(in, out, S, S2, n);
}

// ------------------------------------------------------------------------------------
// Tile-major [w][NC] FP32 -> point-major [NC][w] (the TF32 tensor-core operand layout),
// through a padded shared-memory tile of 32 features x 64 columns; both sides coalesced.
// ------------------------------------------------------------------------------------
__global__ void k_to_point_major(const float* __restrict__ src, float* __restrict__ dst, int w, int64_t NC) {
  __shared__ float t[32][65];
  const int64_t c0 = (int64_t)blockIdx.x * 64;   // 64 columns inside one 256-column tile
  const int f0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // 256 threads: 64 x 4
  for (int fy = ty; fy < 32; fy += 4) {
    const int f = f0 + fy;
    t[fy][tx] = f < w ? src[toff(f, c0 + tx, w)] : 0.f;
  }
  __syncthreads();
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;   // 32 x 8
  for (int cy = ly; cy < 64; cy += 8)
    if (f0 + lx < w) dst[(c0 + cy) * w + f0 + lx] = t[lx][cy];
}

void launch_to_point_major(const void* src, void* dst, int w, int64_t NC, cudaStream_t st) {
  dim3 grid((unsigned)(NC / 64), (unsigned)((w + 31) / 32));
  k_to_point_major<<<grid, 256, 0, st>>>((const float*)src, (float*)dst, w, NC);
}


// ------------------------------------------------------------------------------------
// Adam (Sec. 2.6.5), bias-corrected, in place.
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

const void* adam_kernel() { return reinterpret_cast<const void*>(&k_adam); }

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
