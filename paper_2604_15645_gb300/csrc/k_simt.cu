// CUDA-core jet GEMMs: the FP32 path, and the fallback for shapes the tensor-core
// kernels do not take.  Same data layout as the tensor-core path (tile-major jet
// matrices, see jet.cuh); every thread owns whole points, so the jet rule and its
// adjoint are applied locally.
#include "internal.h"
#include "jet.cuh"

namespace pinn {

namespace {

constexpr int BM = 64, BN = TILE_COLS, BK = 16, THREADS = 256;

template <typename T>
__device__ __forceinline__ void load_vec8(const T* p, float v[8]);
template <>
__device__ __forceinline__ void load_vec8<float>(const float* p, float v[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <>
__device__ __forceinline__ void load_vec8<__nv_bfloat16>(const __nv_bfloat16* p, float v[8]) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
    v[2 * i] = f.x; v[2 * i + 1] = f.y;
  }
}


// One block per (64 features, one 256-column tile = 64 points).  Thread (ty, tx)
// owns features 4ty..4ty+3 and points 4tx..4tx+3 of the tile, i.e. the columns
// 64 r + 4 tx + j of all four jet rows r, so the jet rule is thread-local.
// EPI 0: forward (bias on value rows, activation jet, writes A and the BF16 low half;
//        with the sine activation also the pre-activation jets Z)
// EPI 1: adjoint (reads A_{l-1}, or Z_{l-1} for sine, the jet adjoint, writes Zbar_{l-1})
// EPI 2: linear adjoint (writes W^T Zbar itself: the adjoint of the input jets)
template <typename T, int EPI, bool SINE>
__global__ void __launch_bounds__(THREADS) k_simt_gemm(const float* __restrict__ Aop, const T* __restrict__ Bop,
                                                       const __nv_bfloat16* __restrict__ Blo, int M, int K,
                                                       int64_t NP, EpiArgs e) {
  constexpr bool FAST = sizeof(T) == 2;
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  const int m0 = blockIdx.y * BM;
  const int64_t tile = blockIdx.x;
  const int64_t n0 = tile * BN;
  float acc[4][16];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < K; k0 += BK) {
    {  // A tile: 64 rows x 16 k, 4 per thread
      const int i = t >> 2, kk = (t & 3) * 4;
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + i, k = k0 + kk + q;
        As[kk + q][i] = (m < M && k < K) ? Aop[(int64_t)m * K + k] : 0.f;
      }
    }
    {  // B tile: 16 k x 256 columns, 16 per thread (value columns add the low half)
      const int kk = t >> 4, c = (t & 15) * 16;
      float v[16];
      if (k0 + kk < K) {
        load_vec8<T>(Bop + toff(k0 + kk, n0 + c, K), v);
        load_vec8<T>(Bop + toff(k0 + kk, n0 + c, K) + 8, v + 8);
        if (Blo && c < TILE_PTS) {
          float lo[16];
          load_vec8<__nv_bfloat16>(Blo + loff(k0 + kk, tile * TILE_PTS + c, K), lo);
          load_vec8<__nv_bfloat16>(Blo + loff(k0 + kk, tile * TILE_PTS + c, K) + 8, lo + 8);
          for (int q = 0; q < 16; ++q) v[q] += lo[q];
        }
      } else {
        for (int q = 0; q < 16; ++q) v[q] = 0.f;
      }
      for (int q = 0; q < 16; ++q) Bs[kk][c + q] = v[q];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float a[4] = {a4.x, a4.y, a4.z, a4.w};
      float b[16];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][64 * r + 4 * tx]);
        b[4 * r] = b4.x; b[4 * r + 1] = b4.y; b[4 * r + 2] = b4.z; b[4 * r + 3] = b4.w;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  T* out = reinterpret_cast<T*>(e.out);
  for (int i = 0; i < 4; ++i) {
    const int f = m0 + ty * 4 + i;
    if (f >= M) continue;
    float o[4][4], zz[4][4];   // [row][point]
    if (EPI == 1 && SINE) {   // sine: the pre-activation jets of the layer below
      const float* zr = e.zin + toff(f, n0 + 4 * tx, M);
      for (int r = 0; r < 4; ++r) load4<float>(zr + 64 * r, zz[r]);
    } else if (EPI == 1) {   // tanh: the output jet of the layer below (value row: hi + lo for BF16)
      const T* ar = reinterpret_cast<const T*>(e.ain) + toff(f, n0 + 4 * tx, M);
      for (int r = 0; r < 4; ++r) load4<T>(ar + 64 * r, zz[r]);
      if (sizeof(T) == 2 && e.ain_lo) {
        float lo[4];
        load4<__nv_bfloat16>(reinterpret_cast<const __nv_bfloat16*>(e.ain_lo) + loff(f, tile * TILE_PTS + 4 * tx, M), lo);
        for (int j = 0; j < 4; ++j) zz[0][j] += lo[j];
      }
    }
    const float bias = (EPI == 0) ? e.bias[f] : 0.f;
    for (int j = 0; j < 4; ++j) {
      float z[4], a[4], ab[4];
      for (int r = 0; r < 4; ++r) {
        if (EPI == 0) z[r] = acc[i][4 * r + j] + (r == 0 ? bias : 0.f);
        else { z[r] = zz[r][j]; ab[r] = acc[i][4 * r + j]; }
      }
      if (EPI == 2) {
        for (int r = 0; r < 4; ++r) o[r][j] = acc[i][4 * r + j];
      } else if (EPI == 0) {
        if constexpr (SINE) {
          jet_fwd_sine(z, a, e.jet_mode, e.omega0);
          for (int r = 0; r < 4; ++r) zz[r][j] = z[r];
        } else {
          jet_fwd<FAST>(z, a, e.jet_mode);
        }
        for (int r = 0; r < 4; ++r) o[r][j] = a[r];
      } else {
        if constexpr (SINE) jet_adj_sine(z, ab, a, e.jet_mode, e.omega0);
        else jet_adj_a(z, ab, a, e.jet_mode);
        for (int r = 0; r < 4; ++r) o[r][j] = a[r];
      }
    }
    if (EPI == 0 && SINE) {
      float* zrow = e.zout + toff(f, n0 + 4 * tx, M);
      for (int r = 0; r < 4; ++r) store4<float>(zrow + 64 * r, zz[r]);
    }
    T* orow = out + toff(f, n0 + 4 * tx, M);
    for (int r = 0; r < 4; ++r) store4<T>(orow + 64 * r, o[r]);
    if (EPI == 0) {
      if (sizeof(T) == 2 && e.alo_out) {
        __nv_bfloat16* lo = reinterpret_cast<__nv_bfloat16*>(e.alo_out) + loff(f, tile * TILE_PTS + 4 * tx, M);
        for (int j = 0; j < 4; ++j)
          lo[j] = __float2bfloat16_rn(o[0][j] - __bfloat162float(__float2bfloat16_rn(o[0][j])));
      }
    }
  }
}

// Split-K weight gradient: part[s][m][n] = sum_{k in split s} Aop[m][k] Bop[n][k].
constexpr int DBM = 64, DBN = 64, DBK = 32;

template <typename TA, typename TB>
__global__ void __launch_bounds__(THREADS) k_simt_dw(const TA* __restrict__ Aop, const TB* __restrict__ Bop, int M,
                                                     int N, int64_t NC, int64_t kchunk, float* __restrict__ part) {
  __shared__ float As[DBK][DBM + 4];
  __shared__ float Bs[DBK][DBN + 4];
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  const int m0 = blockIdx.y * DBM, nn0 = blockIdx.x * DBN;
  const int s = blockIdx.z;
  const int64_t kb = (int64_t)s * kchunk, ke = min(NC, kb + kchunk);
  // A split sums up to NC / nsplit jet columns (hundreds of thousands at a million
  // points): each DBK-column block is summed on its own, and the block sums are added
  // to the running total with Kahan compensation, so the rounding error stays near
  // that of a DBK-term sum instead of growing with the split's length.
  float acc[4][4], comp[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = comp[i][j] = 0.f;
  for (int64_t k0 = kb; k0 < ke; k0 += DBK) {
    const int i = t >> 2, kk = (t & 3) * 8;   // 64 rows x 32 k, 8 per thread
    {
      float v[8];
      if (m0 + i < M) load_vec8<TA>(Aop + toff(m0 + i, k0 + kk, M), v);
      else
        for (int q = 0; q < 8; ++q) v[q] = 0.f;
      for (int q = 0; q < 8; ++q) As[kk + q][i] = v[q];
    }
    {
      float v[8];
      if (nn0 + i < N) load_vec8<TB>(Bop + toff(nn0 + i, k0 + kk, N), v);
      else
        for (int q = 0; q < 8; ++q) v[q] = 0.f;
      for (int q = 0; q < 8; ++q) Bs[kk + q][i] = v[q];
    }
    __syncthreads();
    float blk[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) blk[p][q] = 0.f;
#pragma unroll
    for (int k = 0; k < DBK; ++k) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
      const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) blk[p][q] = fmaf(a[p], b[q], blk[p][q]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {   // Kahan: acc + blk with the lost low part kept in comp
        const float y = blk[p][q] - comp[p][q];
        const float t = acc[p][q] + y;
        comp[p][q] = (t - acc[p][q]) - y;
        acc[p][q] = t;
      }
    __syncthreads();
  }
  for (int p = 0; p < 4; ++p) {
    const int m = m0 + ty * 4 + p;
    if (m >= M) continue;
    for (int q = 0; q < 4; ++q) {
      const int n = nn0 + tx * 4 + q;
      if (n < N) part[((int64_t)s * M + m) * N + n] = acc[p][q];
    }
  }
}

}  // namespace

void launch_simt_gemm_fwd(const float* Aop, const void* Bop, int M, int K, int64_t NP, const EpiArgs& e, int prec,
                          cudaStream_t st) {
  dim3 grid((unsigned)(NP / TILE_PTS), (M + BM - 1) / BM);
  if (prec == PINN_BF16) {
    if (e.act)
      k_simt_gemm<__nv_bfloat16, 0, true><<<grid, THREADS, 0, st>>>(Aop, (const __nv_bfloat16*)Bop,
                                                                    (const __nv_bfloat16*)e.alo_in, M, K, NP, e);
    else
      k_simt_gemm<__nv_bfloat16, 0, false><<<grid, THREADS, 0, st>>>(Aop, (const __nv_bfloat16*)Bop,
                                                                     (const __nv_bfloat16*)e.alo_in, M, K, NP, e);
  } else {
    if (e.act)
      k_simt_gemm<float, 0, true><<<grid, THREADS, 0, st>>>(Aop, (const float*)Bop, nullptr, M, K, NP, e);
    else
      k_simt_gemm<float, 0, false><<<grid, THREADS, 0, st>>>(Aop, (const float*)Bop, nullptr, M, K, NP, e);
  }
}

void launch_simt_gemm_adj(const float* Aop, const void* Bop, int M, int K, int64_t NP, const EpiArgs& e, int prec,
                          cudaStream_t st) {
  dim3 grid((unsigned)(NP / TILE_PTS), (M + BM - 1) / BM);
  if (prec == PINN_BF16) {
    if (e.act)
      k_simt_gemm<__nv_bfloat16, 1, true><<<grid, THREADS, 0, st>>>(Aop, (const __nv_bfloat16*)Bop, nullptr, M, K,
                                                                    NP, e);
    else
      k_simt_gemm<__nv_bfloat16, 1, false><<<grid, THREADS, 0, st>>>(Aop, (const __nv_bfloat16*)Bop, nullptr, M, K,
                                                                     NP, e);
  } else {
    if (e.act)
      k_simt_gemm<float, 1, true><<<grid, THREADS, 0, st>>>(Aop, (const float*)Bop, nullptr, M, K, NP, e);
    else
      k_simt_gemm<float, 1, false><<<grid, THREADS, 0, st>>>(Aop, (const float*)Bop, nullptr, M, K, NP, e);
  }
}

void launch_simt_gemm_lin(const float* Aop, const void* Bop, int M, int K, int64_t NP, void* out, int prec,
                          cudaStream_t st) {
  dim3 grid((unsigned)(NP / TILE_PTS), (M + BM - 1) / BM);
  EpiArgs e{};
  e.out = out;
  if (prec == PINN_BF16)
    k_simt_gemm<__nv_bfloat16, 2, false><<<grid, THREADS, 0, st>>>(Aop, (const __nv_bfloat16*)Bop, nullptr, M, K,
                                                                   NP, e);
  else
    k_simt_gemm<float, 2, false><<<grid, THREADS, 0, st>>>(Aop, (const float*)Bop, nullptr, M, K, NP, e);
}

void launch_simt_gemm_dw(const void* Aop, bool a_fp32, const void* Bop, bool b_fp32, int M, int N, int64_t NC,
                         int nsplit, float* part, int prec, cudaStream_t st) {
  int64_t kchunk = (NC + nsplit - 1) / nsplit;
  kchunk = (kchunk + DBK - 1) / DBK * DBK;
  dim3 grid((N + DBN - 1) / DBN, (M + DBM - 1) / DBM, nsplit);
  const bool bf = (prec == PINN_BF16);
  if (!bf || (a_fp32 && b_fp32)) {
    k_simt_dw<float, float><<<grid, THREADS, 0, st>>>((const float*)Aop, (const float*)Bop, M, N, NC, kchunk, part);
  } else if (a_fp32) {
    k_simt_dw<float, __nv_bfloat16><<<grid, THREADS, 0, st>>>((const float*)Aop, (const __nv_bfloat16*)Bop, M, N, NC,
                                                             kchunk, part);
  } else {
    k_simt_dw<__nv_bfloat16, __nv_bfloat16><<<grid, THREADS, 0, st>>>(
        (const __nv_bfloat16*)Aop, (const __nv_bfloat16*)Bop, M, N, NC, kchunk, part);
  }
}

}  // namespace pinn
