// Tensor-core jet GEMMs for sm_103a: tcgen05.mma with operands staged in shared
// memory by TMA (cp.async.bulk.tensor, 128-byte swizzle) and FP32 accumulators in
// tensor memory, read back with tcgen05.ld for the fused epilogues.
//
// Data layout (shared with the CUDA-core path): every activation-like matrix is
// feature-major, [features][NC] with NC jet columns, and the four jet rows of an
// interior point are adjacent columns.  The three GEMMs of a hidden layer are
//   forward  Z^T[fout][NC]    = W[fout][fin]   . A^T[fin][NC]       (B operand MN-major)
//   adjoint  Abar^T[fin][NC]  = W^T[fin][fout] . Zbar^T[fout][NC]   (B operand MN-major)
//   weights  dW[fout][fin]    = Zbar^T[fout][NC] . (A^T[fin][NC])^T (both K-major, split over NC)
// so a 128-row accumulator tile puts one feature in each TMEM lane and 256
// consecutive jet columns in its columns: each epilogue thread owns one feature of
// 64 whole points and applies the tanh jet rule (or its adjoint) without any
// cross-thread exchange.
//
// Warp roles per CTA (576 threads, one CTA per SM, persistent over tiles):
//   warp 0      TMA producer (one lane)
//   warp 1      TMEM allocator + MMA issuer (one lane)
//   warps 2-17  epilogue; warp w reads TMEM lanes 32*(w%4) .. +31, columns
//               64*((w-2)/4) .. +63 of the 256-column accumulator
// Two accumulator buffers of 256 columns let the epilogue of one tile overlap the
// MMAs of the next.  Every mbarrier wait is bounded (global timer); on expiry the
// CTA latches PINN_ERR_TIMEOUT in the status word, stops issuing work, waits for
// its own copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>

#include "jet.cuh"
#include "tc.h"

namespace pinn {

namespace {

constexpr int BM = 128;          // accumulator rows (TMEM lanes)
constexpr int BN = 256;          // accumulator columns per buffer
constexpr int EPI_WARPS = 16;    // four warps per TMEM lane quadrant, each on a quarter of the columns
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s bound on any single wait

enum TcMode { TC_FWD = 0, TC_ADJ = 1, TC_DW = 2, TC_STORE = 3 };

// ---- PTX wrappers -------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when another role aborted or the bound expired (then the
// abort flag and the device status word are set).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try(bar, parity)) return true;
    if ((spin & 63) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > WAIT_NS) {
        *abort_flag = 1;
        atomicOr(status, 2);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
template <bool TF32>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, float v[16]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Bulk tensor store shared -> global (asynchronous proxy) and its group bookkeeping.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05), 128-byte swizzle, version 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;   // SWIZZLE_128B
  return d;
}
// Instruction descriptor: FP32 accumulate, A/B format (1 = BF16, 2 = TF32),
// A K-major, B K-major (b_mn = 0) or MN-major (b_mn = 1), N = BN, M = BM.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t b_mn) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (b_mn << 16) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

struct TcParams {
  int M;               // valid accumulator rows (features, or dW rows)
  int N;               // valid columns (NC for fwd/adj/store, fin for dW)
  int K;               // reduction length (fin / fout for fwd / adj, NC for dW)
  int m_tiles, n_tiles, k_iters;
  int nsplit, kps;     // dW: K splits and K iterations per split
  int64_t NC;          // leading dimension of feature-major matrices
  EpiArgs e;
  float* out32;        // dW partials / selftest output
  int* status;
};

template <bool TF32, int MODE, bool SPLIT>
struct Cfg {
  static constexpr int ES = TF32 ? 4 : 2;
  static constexpr int BKE = 128 / ES;            // K elements per stage (one 128-byte swizzle row)
  static constexpr int UK = TF32 ? 8 : 16;        // K per MMA instruction
  static constexpr int A_BYTES = BM * 128;        // 16 KB
  static constexpr int B_BYTES = BN * 128;        // 32 KB
  static constexpr int STAGE = A_BYTES * (SPLIT ? 2 : 1) + B_BYTES;
  // Epilogues that write jet matrices stage each 32-row x 16-column chunk in shared
  // memory and store it with a bulk tensor copy (double-buffered per warp).
  static constexpr bool STAGED = (MODE == TC_FWD || MODE == TC_ADJ);
  static constexpr int STG_BYTES = 32 * 16 * ES;                        // one chunk of one array
  static constexpr int STAGING = STAGED ? EPI_WARPS * 2 * 2 * STG_BYTES : 0;
  static constexpr int STAGES = STAGED ? (SPLIT ? 2 : 3) : (SPLIT ? 3 : 4);
  static constexpr bool B_MN = (MODE != TC_DW);
  static constexpr int BOXN = 128 / ES;           // MN-major box width (columns)
  static constexpr int NBOX = BN / BOXN;
  static constexpr int BOX_BYTES = BOXN * 0 + BKE * 128;   // one MN-major box: BKE rows of 128 bytes
  static constexpr size_t SMEM = (size_t)STAGES * STAGE + STAGING + 1024 /*align*/ + 256 /*barriers*/;
};

template <typename T>
__device__ __forceinline__ void store16(T* p, const float v[16]);
template <>
__device__ __forceinline__ void store16<float>(float* p, const float v[16]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    reinterpret_cast<float4*>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
template <>
__device__ __forceinline__ void store16<__nv_bfloat16>(__nv_bfloat16* p, const float v[16]) {
  uint32_t u[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    u[i] = *reinterpret_cast<uint32_t*>(&h);
  }
  reinterpret_cast<uint4*>(p)[0] = make_uint4(u[0], u[1], u[2], u[3]);
  reinterpret_cast<uint4*>(p)[1] = make_uint4(u[4], u[5], u[6], u[7]);
}
// 16 elements as raw 128-bit words (8 registers for BF16), converted on use.
template <typename T>
struct Raw16 {
  uint4 w[sizeof(T) * 16 / 16];
};
template <typename T>
__device__ __forceinline__ void load_raw16(const T* p, Raw16<T>& r) {
#pragma unroll
  for (int i = 0; i < (int)(sizeof(r.w) / sizeof(uint4)); ++i) r.w[i] = reinterpret_cast<const uint4*>(p)[i];
}
__device__ __forceinline__ void unpack16(const Raw16<__nv_bfloat16>& r, float v[16]) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const uint32_t w[4] = {r.w[i].x, r.w[i].y, r.w[i].z, r.w[i].w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[j]));
      v[8 * i + 2 * j] = f.x;
      v[8 * i + 2 * j + 1] = f.y;
    }
  }
}
__device__ __forceinline__ void unpack16(const Raw16<float>& r, float v[16]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[4 * i] = __uint_as_float(r.w[i].x); v[4 * i + 1] = __uint_as_float(r.w[i].y);
    v[4 * i + 2] = __uint_as_float(r.w[i].z); v[4 * i + 3] = __uint_as_float(r.w[i].w);
  }
}

template <typename T>
__device__ __forceinline__ void load16(const T* p, float v[16]);
template <>
__device__ __forceinline__ void load16<float>(const float* p, float v[16]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 q = reinterpret_cast<const float4*>(p)[i];
    v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
  }
}
template <>
__device__ __forceinline__ void load16<__nv_bfloat16>(const __nv_bfloat16* p, float v[16]) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const uint4 q = reinterpret_cast<const uint4*>(p)[i];
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[j]));
      v[8 * i + 2 * j] = f.x;
      v[8 * i + 2 * j + 1] = f.y;
    }
  }
}

// ---- the kernel -----------------------------------------------------------------------
template <bool TF32, int MODE, bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapA2,
              const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapO1,
              const __grid_constant__ CUtensorMap mapO2, const TcParams p) {
  using C = Cfg<TF32, MODE, SPLIT>;
  using T = typename std::conditional<TF32, float, __nv_bfloat16>::type;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* staging = smem + C::STAGES * C::STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(staging + C::STAGING);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;
  uint64_t* acc_empty = acc_full + 2;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(acc_empty + 2);
  volatile int* inflight = abort_flag + 1;             // [STAGES]: parity+1 of an armed, unconsumed stage
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(const_cast<int*>(inflight + C::STAGES));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      inflight[s] = 0;
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 32 * EPI_WARPS);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {   // allocate 2 x 256 TMEM columns (whole warp)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int total = p.m_tiles * p.n_tiles * (MODE == TC_DW ? p.nsplit : 1);
  auto coords = [&](int t, int& mb, int& nb, int& k0, int& k1) {
    mb = t % p.m_tiles;
    int r = t / p.m_tiles;
    nb = r % p.n_tiles;
    if (MODE == TC_DW) {
      const int s = r / p.n_tiles;
      k0 = s * p.kps;
      k1 = min(p.k_iters, k0 + p.kps);
    } else {
      k0 = 0;
      k1 = p.k_iters;
    }
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
        int mb, nb, k0, k1;
        coords(t, mb, nb, k0, k1);
        for (int kb = k0; kb < k1; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, p.status)) break;
          uint8_t* sa = smem + stage * C::STAGE;
          uint8_t* sa2 = sa + C::A_BYTES;
          uint8_t* sb = sa + C::A_BYTES * (SPLIT ? 2 : 1);
          mbar_expect_tx(&full[stage], C::STAGE);
          inflight[stage] = (int)phase + 1;
          const int kx = kb * C::BKE;
          tma_load_2d(sa, &mapA, &full[stage], kx, mb * BM);
          if (SPLIT) tma_load_2d(sa2, &mapA2, &full[stage], kx, mb * BM);
          if (C::B_MN) {
#pragma unroll
            for (int j = 0; j < C::NBOX; ++j)
              tma_load_2d(sb + j * C::BOX_BYTES, &mapB, &full[stage], nb * BN + j * C::BOXN, kx);
          } else {
            tma_load_2d(sb, &mapB, &full[stage], kx, nb * BN);
          }
          if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(TF32 ? 2u : 1u, C::B_MN ? 1u : 0u);
      int stage = 0;
      uint32_t phase = 0;
      int local = 0;
      for (int t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++local) {
        int mb, nb, k0, k1;
        coords(t, mb, nb, k0, k1);
        const int buf = local & 1;
        if (!mbar_wait(&acc_empty[buf], ((local >> 1) & 1) ^ 1, abort_flag, p.status)) break;
        tc_fence_after();
        const uint32_t d = tmem_base + buf * BN;
        bool ok = true;
        for (int kb = k0; kb < k1; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.status)) { ok = false; break; }
          inflight[stage] = 0;
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * C::STAGE);
          const uint32_t sa2 = sa + C::A_BYTES;
          const uint32_t sb = sa + C::A_BYTES * (SPLIT ? 2 : 1);
#pragma unroll
          for (int kk = 0; kk < C::BKE / C::UK; ++kk) {
            const uint64_t ad = make_desc(sa + kk * 32, 16, 1024);
            const uint64_t bd = C::B_MN ? make_desc(sb + kk * C::UK * 128, C::BOX_BYTES, 1024)
                                        : make_desc(sb + kk * 32, 16, 1024);
            tc_mma<TF32>(d, ad, bd, idesc, (kb > k0 || kk > 0) ? 1u : 0u);
            if (SPLIT) tc_mma<TF32>(d, make_desc(sa2 + kk * 32, 16, 1024), bd, idesc, 1u);
          }
          tc_commit(&empty[stage]);
          if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        tc_commit(&acc_full[buf]);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    constexpr bool FAST = !TF32;
    constexpr int PARTS = EPI_WARPS / 4;       // column parts per tile
    constexpr int CPP = BN / 16 / PARTS;       // 16-column chunks per part
    const int quad = warp & 3;                 // TMEM lane quadrant this warp may read
    const int part = (warp - 2) >> 2;          // which quarter of the tile's columns
    const int row = quad * 32 + lane;
    T* stg = reinterpret_cast<T*>(staging + (warp - 2) * (2 * 2 * C::STG_BYTES));   // [buf][array][32][16]
    uint32_t nstore = 0;
    int local = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++local) {
      int mb, nb, k0, k1;
      coords(t, mb, nb, k0, k1);
      const int buf = local & 1;
      if (!mbar_wait(&acc_full[buf], (local >> 1) & 1, abort_flag, p.status)) break;
      tc_fence_after();
      const int m = mb * BM + row;
      const int row0 = mb * BM + quad * 32;    // first row of this warp's 32-row slab
      const bool mvalid = m < p.M;
      const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + buf * BN;
      const float bias = (MODE == TC_FWD && mvalid) ? p.e.bias[m] : 0.f;
      float dbacc[4] = {0.f, 0.f, 0.f, 0.f};
      float v[2][16];
      Raw16<T> zr[2];
      const T* zrow = (MODE == TC_ADJ) ? reinterpret_cast<const T*>(p.e.zin) + (int64_t)m * p.NC : nullptr;
      if (MODE == TC_ADJ && mvalid) load_raw16<T>(zrow + (int64_t)nb * BN + part * CPP * 16, zr[0]);
      tmem_ld16_issue(taddr + part * CPP * 16, v[0]);
      tmem_wait_ld();
#pragma unroll
      for (int cc = 0; cc < CPP; ++cc) {
        const int c = part * CPP + cc;
        const int64_t col0 = (int64_t)nb * BN + c * 16;
        float* cur = v[cc & 1];
        float z[16];
        if (MODE == TC_ADJ) unpack16(zr[cc & 1], z);
        if (cc + 1 < CPP) {                    // prefetch the next chunk
          if (MODE == TC_ADJ && mvalid) load_raw16<T>(zrow + col0 + 16, zr[(cc + 1) & 1]);
          tmem_ld16_issue(taddr + (c + 1) * 16, v[(cc + 1) & 1]);
        }
        if (C::STAGED) {
          float o[16];
          if (MODE == TC_FWD) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const int64_t col = col0 + 4 * g;
              float* zz = &cur[4 * g];
              if (col < p.e.n_res4) {
                zz[0] += bias;
                jet_fwd<FAST>(zz, &o[4 * g], p.e.jet_mode);
              } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                  if (col + r < p.e.ncols) { zz[r] += bias; o[4 * g + r] = val_fwd<FAST>(zz[r]); }
                  else { zz[r] = 0.f; o[4 * g + r] = 0.f; }
                }
              }
            }
          } else {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const int64_t col = col0 + 4 * g;
              if (col < p.e.n_res4) {
                jet_adj<FAST>(&z[4 * g], &cur[4 * g], &o[4 * g], p.e.jet_mode);
              } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                  o[4 * g + r] = (col + r < p.e.ncols) ? val_adj<FAST>(z[4 * g + r], cur[4 * g + r]) : 0.f;
              }
            }
            if (p.e.dbpart && mvalid) {
              // bias gradient (value columns) and, for a first layer on raw
              // coordinates, the coordinate terms of its weight gradient
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                const int64_t col = col0 + 4 * g;
                if (col < p.e.n_res4) {
                  dbacc[0] += o[4 * g];
                  if (p.e.dterms) {
                    const int64_t pt = col >> 2;
                    for (int jj = 0; jj < p.e.dterms; ++jj)
                      dbacc[1 + jj] = fmaf(o[4 * g], p.e.x_res[(int64_t)jj * p.e.n_res + pt], dbacc[1 + jj]);
                    for (int r = 1; r < 4; ++r) {
                      const int d = row_dir(p.e.jet_mode, r);
                      if (d >= 0) dbacc[1 + d] += o[4 * g + r];
                    }
                  }
                } else {
                  for (int r = 0; r < 4; ++r) {
                    const ColPoint cp = classify_col(col + r, p.e.n_res, p.e.n_ic, p.e.n_bc);
                    if (cp.set == 3) continue;
                    dbacc[0] += o[4 * g + r];
                    for (int jj = 0; jj < p.e.dterms; ++jj)
                      dbacc[1 + jj] = fmaf(o[4 * g + r],
                                           coord(p.e.x_res, p.e.x_ic, p.e.x_bc, p.e.n_res, p.e.n_ic, p.e.n_bc, cp, jj),
                                           dbacc[1 + jj]);
                  }
                }
              }
            }
          }
          // stage this warp's 32 x 16 chunk(s) and store them with one bulk copy each
          const int sb = nstore & 1;
          if (nstore >= 2) {
            if (lane == 0) bulk_wait_read1();   // the copy that used this buffer has read it
            __syncwarp();
          }
          T* s0 = stg + (sb * 2 + 0) * (32 * 16);
          T* s1 = stg + (sb * 2 + 1) * (32 * 16);
          store16<T>(s0 + lane * 16, o);
          if (MODE == TC_FWD) store16<T>(s1 + lane * 16, cur);
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            if (row0 < p.M) {
              tma_store_2d(&mapO1, s0, (int)col0, row0);
              if (MODE == TC_FWD) tma_store_2d(&mapO2, s1, (int)col0, row0);
            }
            bulk_commit();   // one group per chunk (possibly empty) keeps the buffer parity exact
          }
          ++nstore;
        } else if (mvalid) {
          if (MODE == TC_DW) {
            const int split = t / (p.m_tiles * p.n_tiles);
            float* dst = p.out32 + ((int64_t)split * p.M + m) * p.N;
            if (col0 + 16 <= p.N && (p.N & 3) == 0) {
              store16<float>(dst + col0, cur);
            } else {
              for (int j = 0; j < 16; ++j)
                if (col0 + j < p.N) dst[col0 + j] = cur[j];
            }
          } else {   // TC_STORE
            store16<float>(p.out32 + (int64_t)m * p.NC + col0, cur);
          }
        }
        if (cc + 1 < CPP) tmem_wait_ld();
      }
      if (MODE == TC_ADJ && p.e.dbpart && mvalid) {
        float* dst = p.e.dbpart + ((int64_t)(nb * PARTS + part) * p.M + m) * (1 + p.e.dterms);
        for (int jj = 0; jj <= p.e.dterms; ++jj) dst[jj] = dbacc[jj];
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[buf]);
    }
    if (C::STAGED && lane == 0) bulk_wait_all();   // bulk stores done before the CTA exits
  }

  // ---- teardown: wait (bounded) for copies still in flight, free TMEM ----------------
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    for (int s = 0; s < C::STAGES; ++s) {
      const int f = inflight[s];
      if (f) {
        const uint64_t t0 = gtimer();
        while (!mbar_try(&full[s], (uint32_t)(f - 1)) && gtimer() - t0 < WAIT_NS) {}
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * BN));
  }
}

// ---- host side ------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// 2-D tensor map over a row-major matrix [rows][cols] (cols contiguous), box
// [box_rows][box_cols], 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap* m, const void* base, bool tf32, uint64_t cols, uint64_t rows, uint32_t box_cols,
              uint32_t box_rows) {
  if (!g_encode) return false;
  const uint32_t es = tf32 ? 4 : 2;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * es};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Output map for the staged bulk stores: [rows][cols], box 32 rows x 16 columns,
// no swizzle (the staging buffer is plain row-major).
bool make_store_map(CUtensorMap* m, const void* base, bool tf32, uint64_t cols, uint64_t rows) {
  if (!g_encode) return false;
  const uint32_t es = tf32 ? 4 : 2;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * es};
  cuuint32_t box[2] = {16, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <bool TF32, int MODE, bool SPLIT>
pinn_status launch(pinn_handle* h, const CUtensorMap& a, const CUtensorMap& a2, const CUtensorMap& b,
                   const CUtensorMap& o1, const CUtensorMap& o2, const TcParams& p, int grid, cudaStream_t st) {
  using C = Cfg<TF32, MODE, SPLIT>;
  auto kern = k_tc_gemm<TF32, MODE, SPLIT>;
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM) != cudaSuccess) {
      snprintf(h->err, sizeof(h->err), "tcgen05 kernel: cannot reserve %zu bytes of shared memory", C::SMEM);
      return PINN_ERR_CUDA;
    }
    attr_set = true;
  }
  kern<<<grid, THREADS, C::SMEM, st>>>(a, a2, b, o1, o2, p);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(h->err, sizeof(h->err), "tcgen05 kernel launch: %s", cudaGetErrorString(e));
    return PINN_ERR_CUDA;
  }
  return PINN_OK;
}

int grid_for(const pinn_handle* h, int tiles) { return std::max(1, std::min(tiles, std::max(h->sm_count, 1))); }

}  // namespace

void tc_init(pinn_handle* h) {
  (void)h;
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
}

bool tc_layer_supported(const pinn_handle* h, int li, int64_t NC) {
  (void)li;
  if (!g_encode || h->spec.precision != PINN_BF16) return false;
  if (NC % BN) return false;
  const int fin = h->layers[li].fin, fout = h->layers[li].fout;
  // TMA row strides must be multiples of 16 bytes: fin and fout multiples of 8 (bf16).
  return (fin % 8 == 0) && (fout % 8 == 0) && fin >= 16 && fout >= 16;
}

int tc_dw_splits(const pinn_handle* h, int fout, int fin, int64_t NC) {
  const int tiles = ((fout + BM - 1) / BM) * ((fin + BN - 1) / BN);
  const int k_iters = (int)((NC + 63) / 64);
  int ns = std::max(1, (std::max(h->sm_count, 1) + tiles - 1) / tiles);
  ns = std::min(ns, k_iters);
  const int kps = (k_iters + ns - 1) / ns;
  return (k_iters + kps - 1) / kps;   // no empty split
}

namespace {

TcParams base_params(int M, int N, int K, int64_t NC, int kblock, int* status) {
  TcParams p{};
  p.M = M; p.N = N; p.K = K; p.NC = NC;
  p.m_tiles = (M + BM - 1) / BM;
  p.n_tiles = (N + BN - 1) / BN;
  p.k_iters = (K + kblock - 1) / kblock;
  p.nsplit = 1; p.kps = p.k_iters;
  p.status = status;
  return p;
}

pinn_status map_err(pinn_handle* h, const char* what) {
  snprintf(h->err, sizeof(h->err), "cuTensorMapEncodeTiled failed for %s", what);
  return PINN_ERR_CUDA;
}

}  // namespace

pinn_status tc_gemm_fwd(pinn_handle* h, const void* W, const void* Wlo, const void* A, int fout, int fin, int64_t NC,
                        const EpiArgs& e, cudaStream_t st) {
  CUtensorMap ma, ma2, mb;
  if (!make_map(&ma, W, false, fin, fout, 64, BM) || !make_map(&ma2, Wlo, false, fin, fout, 64, BM))
    return map_err(h, "forward weights");
  if (!make_map(&mb, A, false, NC, fin, 64, 64)) return map_err(h, "forward activations");
  CUtensorMap o1, o2;
  if (!make_store_map(&o1, e.out, false, NC, fout) || !make_store_map(&o2, e.zout, false, NC, fout))
    return map_err(h, "forward outputs");
  TcParams p = base_params(fout, (int)NC, fin, NC, 64, h->d_status);
  p.e = e;
  return launch<false, TC_FWD, true>(h, ma, ma2, mb, o1, o2, p, grid_for(h, p.m_tiles * p.n_tiles), st);
}

pinn_status tc_gemm_adj(pinn_handle* h, const void* WT, const void* Zbar, int fin, int fout, int64_t NC,
                        const EpiArgs& e, cudaStream_t st) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, WT, false, fout, fin, 64, BM)) return map_err(h, "adjoint weights");
  if (!make_map(&mb, Zbar, false, NC, fout, 64, 64)) return map_err(h, "adjoint input");
  CUtensorMap o1;
  if (!make_store_map(&o1, e.out, false, NC, fin)) return map_err(h, "adjoint output");
  TcParams p = base_params(fin, (int)NC, fout, NC, 64, h->d_status);
  p.e = e;
  return launch<false, TC_ADJ, false>(h, ma, ma, mb, o1, o1, p, grid_for(h, p.m_tiles * p.n_tiles), st);
}

pinn_status tc_gemm_dw(pinn_handle* h, const void* Zbar, const void* A, int fout, int fin, int64_t NC, int nsplit,
                       float* part, cudaStream_t st) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, Zbar, false, NC, fout, 64, BM)) return map_err(h, "weight-gradient adjoint");
  if (!make_map(&mb, A, false, NC, fin, 64, BN)) return map_err(h, "weight-gradient activations");
  TcParams p = base_params(fout, fin, (int)NC, NC, 64, h->d_status);
  p.nsplit = nsplit;
  p.kps = (p.k_iters + nsplit - 1) / nsplit;
  if ((p.k_iters + p.kps - 1) / p.kps != nsplit) {
    snprintf(h->err, sizeof(h->err), "weight-gradient split plan mismatch");
    return PINN_ERR_INVALID_ARG;
  }
  p.out32 = part;
  return launch<false, TC_DW, false>(h, ma, ma, mb, mb, mb, p, grid_for(h, p.m_tiles * p.n_tiles * nsplit), st);
}

}  // namespace pinn

// Raw tensor-core GEMM of the library's two operand layouts, FP32 output, for
// testing the MMA core in isolation (no epilogue).
extern "C" PINN_API pinn_status pinn_tc_selftest(int kind, int M, int N, int K, const void* d_A, const void* d_A2,
                                                 const void* d_B, float* d_D, void* stream) {
  using namespace pinn;
  if (!d_A || !d_B || !d_D || M < 1 || N < 1 || K < 1 || (kind != 0 && kind != 1)) return PINN_ERR_INVALID_ARG;
  if (K % 8 || M % 8 || N % 8) return PINN_ERR_INVALID_ARG;
  if (kind == 0 && N % BN) return PINN_ERR_INVALID_ARG;
  pinn_handle h;
  tc_init(&h);
  if (!g_encode) return PINN_ERR_UNSUPPORTED;
  if (cudaGetDevice(&h.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h.sm_count, cudaDevAttrMultiProcessorCount, h.device) != cudaSuccess)
    return PINN_ERR_CUDA;
  int* status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return PINN_ERR_CUDA;
  cudaMemsetAsync(status, 0, sizeof(int), (cudaStream_t)stream);
  CUtensorMap ma, ma2, mb;
  pinn_status r = PINN_OK;
  if (kind == 0) {
    // D[M][N] = A[M][K] . B[K][N]   (B stored K x N, N contiguous: MN-major)
    if (!make_map(&ma, d_A, false, K, M, 64, BM) || !make_map(&ma2, d_A2 ? d_A2 : d_A, false, K, M, 64, BM) ||
        !make_map(&mb, d_B, false, N, K, 64, 64)) {
      r = PINN_ERR_CUDA;
    } else {
      TcParams p = base_params(M, N, K, N, 64, status);
      p.out32 = d_D;
      if (d_A2)
        r = launch<false, TC_STORE, true>(&h, ma, ma2, mb, mb, mb, p, grid_for(&h, p.m_tiles * p.n_tiles),
                                          (cudaStream_t)stream);
      else
        r = launch<false, TC_STORE, false>(&h, ma, ma, mb, mb, mb, p, grid_for(&h, p.m_tiles * p.n_tiles),
                                           (cudaStream_t)stream);
    }
  } else {
    // D[M][N] = A[M][K] . B[N][K]^T   (both K contiguous: K-major)
    if (!make_map(&ma, d_A, false, K, M, 64, BM) || !make_map(&mb, d_B, false, K, N, 64, BN)) {
      r = PINN_ERR_CUDA;
    } else {
      TcParams p = base_params(M, N, K, N, 64, status);
      p.out32 = d_D;
      r = launch<false, TC_DW, false>(&h, ma, ma, mb, mb, mb, p, grid_for(&h, p.m_tiles * p.n_tiles),
                                      (cudaStream_t)stream);
    }
  }
  int st = 0;
  if (r == PINN_OK) {
    if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
      r = PINN_ERR_CUDA;
    else if (st & 2)
      r = PINN_ERR_TIMEOUT;
  }
  cudaFree(status);
  return r;
}
