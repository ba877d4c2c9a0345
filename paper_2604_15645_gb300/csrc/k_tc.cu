// Tensor-core jet GEMMs for sm_103a: tcgen05.mma with operands staged in shared
// memory by TMA (cp.async.bulk.tensor, 128-byte swizzle) and FP32 accumulators in
// tensor memory, read back with tcgen05.ld for the fused epilogues.
//
// Data layout (shared with the CUDA-core path): every jet matrix is tile-major,
// [NC/256][features][256]: a tile holds 64 points, its 256 columns blocked by jet
// row ([values | d1 | d2 | d2nd], see jet.cuh).  The three GEMMs of a hidden layer are
//   forward  Z^T[fout][NC]    = W[fout][fin]   . A^T[fin][NC]       (B operand MN-major)
//   adjoint  Abar^T[fin][NC]  = W^T[fin][fout] . Zbar^T[fout][NC]   (B operand MN-major)
//   weights  dW[fout][fin]    = Zbar^T[fout][NC] . (A^T[fin][NC])^T (both K-major, split over NC)
// so a 128-row accumulator tile puts one feature in each TMEM lane and the 256
// columns of one point tile in its columns: each epilogue thread owns one feature
// of whole points and applies the tanh jet rule (or its adjoint) without any
// cross-thread exchange.  On the BF16 path the forward also adds the low half of
// the weights (all columns) and of the input's value rows (the 64 value columns).
//
// TF32 (kind::tf32) reads both operands K-major only, so its forward and adjoint take
// the jets from a point-major copy [NC][features] (written by the epilogue of the
// layer before) and add both truncation remainders: W_hi B + W_lo B + W_hi B_lo, with
// B_lo = B - tf32(B) computed in shared memory by two converter warps.
//
// Warp roles per CTA (320 threads, 384 with converters, one CTA per SM, persistent):
//   warp 0     TMA producer (one lane)
//   warp 1     TMEM allocator + MMA issuer (one lane)
//   warps 2-9  epilogue; warp w reads TMEM lanes 32*(w%4) .. +31 and handles the
//              points 32*((w-2)/4) .. +31 of the tile, 16 at a time
//   warps 10-11 (TF32 forward / adjoint only) B_lo converters
// Two accumulator buffers of 256 columns let the epilogue of one tile overlap the
// MMAs of the next.  Every mbarrier wait is bounded (global timer); on expiry the
// CTA latches PINN_ERR_TIMEOUT in the status word, stops issuing work, waits for
// its own copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <new>
#include <vector>

#include "jet.cuh"
#include "ptx.cuh"
#include "tc.h"

namespace pinn {

namespace {

constexpr int BM = 128;          // accumulator rows (TMEM lanes)
constexpr int BN = 256;          // accumulator columns per buffer
constexpr int EPI_WARPS = 8;     // two warps per TMEM lane quadrant, each on 32 of a tile's 64 points
constexpr uint64_t WAIT_NS = 2000000000ull;   // default bound on any single wait: 2 s

enum TcMode { TC_FWD = 0, TC_ADJ = 1, TC_DW = 2, TC_STORE = 3 };

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
// A K-major, B K-major (b_mn = 0) or MN-major (b_mn = 1), N columns, M = BM.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t b_mn, uint32_t n = BN) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (b_mn << 16) | ((n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
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
  int wlo_values_only; // forward: W_lo . B on the 64 value columns only (PINN_FLAG_BF16_VALUE_SPLIT)
  uint64_t wait_ns;    // bound on every mbarrier wait (WAIT_NS)
  int stall;           // test hook: the MMA issuer first waits on a barrier nothing arrives on
};

// One GEMM of a grouped launch: its tensor maps (the GEMM kernel's four, or the fused
// adjoint's three), its parameters, and the blocks of the grouped grid it owns.  Each
// GEMM keeps the CTA count and work split it has when launched alone.
struct TcGroupEntry {   // 128-byte aligned (CUtensorMap)
  CUtensorMap map[4];
  TcParams p;
  int block0;   // first block of the grouped grid that runs this GEMM
  int grid;     // its block count
};

// Orders this thread's later TMA reads of the entry's tensor maps after the writes that
// put them in global memory (the table is rewritten by the host between captures).
__device__ __forceinline__ void acquire_maps(const TcGroupEntry& g, int nmaps) {
  for (int i = 0; i < nmaps; ++i)
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&g.map[i]) : "memory");
}

// The entry that owns block b: the last one whose first block is <= b (block0 ascends).
__device__ __forceinline__ int group_of_block(const TcGroupEntry* __restrict__ tab, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].block0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Where a CTA sits in the launch: the hardware indices of a single launch (read where
// used, as a plain kernel would), or its share of a grouped launch.
struct SingleGrid {
  __device__ __forceinline__ int bx() const { return (int)blockIdx.x; }
  __device__ __forceinline__ int gdim() const { return (int)gridDim.x; }
};
struct GroupShare {
  int b, g;
  __device__ __forceinline__ int bx() const { return b; }
  __device__ __forceinline__ int gdim() const { return g; }
};

template <bool TF32, int MODE, bool SPLIT>
struct Cfg {
  static constexpr int ES = TF32 ? 4 : 2;
  static constexpr int BKE = 128 / ES;            // K elements per stage (one 128-byte swizzle row)
  static constexpr int UK = TF32 ? 8 : 16;        // K per MMA instruction
  static constexpr int A_BYTES = BM * 128;        // 16 KB
  static constexpr int B_BYTES = BN * 128;        // 32 KB
  // TF32 forward / adjoint: B from the point-major copy (K-major, 2-D map), its low
  // half computed in shared memory (one B-sized buffer).
  static constexpr bool KPM = TF32 && (MODE == TC_FWD || MODE == TC_ADJ);
  static constexpr int BLOC_BYTES = KPM ? B_BYTES : 0;
  static constexpr int CVT_WARPS = KPM ? 2 : 0;
  static constexpr int NTHREADS = 64 + 32 * (EPI_WARPS + CVT_WARPS);
  // BF16 forward: low half of the input's value rows, 64 MN-major columns per stage.
  static constexpr bool VLO = (MODE == TC_FWD) && !TF32;
  static constexpr int BLO_BYTES = VLO ? TILE_PTS * 128 : 0;   // 8 KB
  static constexpr int STAGE = A_BYTES * (SPLIT ? 2 : 1) + B_BYTES + BLO_BYTES;
  static constexpr int STAGES = (MODE == TC_FWD || SPLIT) ? 3 : 4;
  static_assert(STAGES * STAGE + BLOC_BYTES + 1024 + 256 <= 227 * 1024, "shared memory budget");
  static constexpr bool B_MN = (MODE != TC_DW) && !KPM;
  static constexpr int BOXN = 128 / ES;           // MN-major box width (columns)
  static constexpr int NBOX = BN / BOXN;
  static constexpr int BOX_BYTES = BKE * 128;     // one MN-major box: BKE rows of 128 bytes
  static constexpr size_t SMEM = (size_t)STAGES * STAGE + BLOC_BYTES + 1024 /*align*/ + 256 /*barriers*/;
};

// Point-major copy [NC][M] of one thread's 8 points x 4 rows of feature m: column
// c0 + 64 r + i.  Lanes hold consecutive features, so each store instruction writes
// 128 contiguous bytes.
__device__ __forceinline__ void store_pm8(float* pm, int64_t c0, int M, int m, const float v[4][8]) {
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i) pm[(c0 + 64 * r + i) * M + m] = v[r][i];
}

// ---- the kernel -----------------------------------------------------------------------
// SINE (BF16 forward / adjoint): the periodic activation sin(w0 z) instead of tanh.  Its
// adjoint cannot be written in the activations (the sign of cos is lost), so the
// forward epilogue also stores the pre-activation jets Z (FP32) and the adjoint
// epilogue evaluates the rule from them.
// The body runs as CTA grid.bx() of grid.gdim() CTAs over the GEMM that p and the maps
// describe: the whole grid of a single launch, or one GEMM's share of a grouped launch.
template <bool TF32, int MODE, bool SPLIT, bool SINE, typename Grid>
__device__ __forceinline__ void tc_gemm_body(const CUtensorMap* mapA, const CUtensorMap* mapA2,
                                             const CUtensorMap* mapB, const CUtensorMap* mapBlo, const TcParams& p,
                                             const Grid grid) {
  using C = Cfg<TF32, MODE, SPLIT>;
  using T = typename std::conditional<TF32, float, __nv_bfloat16>::type;
  // weight gradient with 256-row tiles: two 128-row accumulators (TMEM columns 0..255 and
  // 256..511) share each staged B operand, so the B rows are read once for 256 output
  // rows; one work item fills both accumulators (no double buffering across items)
  constexpr bool DW2 = (MODE == TC_DW) && SPLIT;
  constexpr int MROWS = DW2 ? 2 * BM : BM;                // output rows per work item
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned by offsetting the shared array itself (an integer round trip would
  // hide the address space and turn every shared access below into a generic one)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* blo = smem + C::STAGES * C::STAGE;          // TF32 B_lo buffer (BLOC_BYTES)
  uint64_t* full = reinterpret_cast<uint64_t*>(blo + C::BLOC_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* lo_full = acc_empty + 2;                  // converter -> MMA: B_lo ready
  uint64_t* lo_empty = lo_full + 1;                   // MMA -> converter: B_lo consumed
  uint64_t* never = lo_empty + 1;                     // test hook (p.stall): no thread arrives on it
  volatile int* abort_flag = reinterpret_cast<volatile int*>(never + 1);
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
    mbar_init(lo_full, 1);
    mbar_init(lo_empty, 1);
    mbar_init(never, 1);
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
    if (MODE != TC_DW && p.e.reverse) t = total - 1 - t;   // same tiles, last column tile first
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
      for (int t = grid.bx(); t < total && !*abort_flag; t += grid.gdim()) {
        int mb, nb, k0, k1;
        coords(t, mb, nb, k0, k1);
        for (int kb = k0; kb < k1; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, p.status, p.wait_ns)) break;
          uint8_t* sa = smem + stage * C::STAGE;
          uint8_t* sa2 = sa + C::A_BYTES;
          uint8_t* sb = sa + C::A_BYTES * (SPLIT ? 2 : 1);
          mbar_expect_tx(&full[stage], C::STAGE);
          inflight[stage] = (int)phase + 1;
          const int kx = kb * C::BKE;
          if (C::KPM) {
            // A: weights [M][K]; B: point-major jets [NC][K], columns nb*BN.. (both 2-D, K-major)
            tma_load_2d(sa, mapA, &full[stage], kx, mb * BM);
            if (SPLIT) tma_load_2d(sa2, mapA2, &full[stage], kx, mb * BM);
            tma_load_2d(sb, mapB, &full[stage], kx, nb * BN);
          } else if (C::B_MN) {
            // A: weights [M][K] (2-D); B: jet tile nb, rows kx..kx+BKE (3-D, tile-major)
            tma_load_2d(sa, mapA, &full[stage], kx, mb * BM);
            if (SPLIT) tma_load_2d(sa2, mapA2, &full[stage], kx, mb * BM);
#pragma unroll
            for (int j = 0; j < C::NBOX; ++j)
              tma_load_3d(sb + j * C::BOX_BYTES, mapB, &full[stage], j * C::BOXN, kx, nb);
            if (C::VLO) {
#pragma unroll
              for (int j = 0; j < TILE_PTS / C::BOXN; ++j)
                tma_load_3d(sb + C::B_BYTES + j * C::BOX_BYTES, mapBlo, &full[stage], j * C::BOXN, kx, nb);
            }
          } else {
            // weight gradient: K runs over jet columns, 256 / BKE K-blocks per tile
            constexpr int KPT = TILE_COLS / C::BKE;
            const int tz = kb / KPT, tx = (kb % KPT) * C::BKE;
            tma_load_3d(sa, mapA, &full[stage], tx, mb * MROWS, tz);
            if (DW2) tma_load_3d(sa2, mapA, &full[stage], tx, mb * MROWS + BM, tz);
            tma_load_3d(sb, mapB, &full[stage], tx, nb * BN, tz);
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
      uint32_t phase = 0, lo_phase = 0;
      int local = 0;
      // test hook: a dependency that is never satisfied, so the bounded wait expires and
      // the whole CTA takes the abort path (status bit 1, teardown below)
      const bool stalled = p.stall && !mbar_wait(never, 0, abort_flag, p.status, p.wait_ns);
      for (int t = grid.bx(); t < total && !*abort_flag && !stalled; t += grid.gdim(), ++local) {
        int mb, nb, k0, k1;
        coords(t, mb, nb, k0, k1);
        const int buf = DW2 ? 0 : local & 1;
        const uint32_t par = DW2 ? ((uint32_t)local & 1) : ((uint32_t)(local >> 1) & 1);
        if (!mbar_wait(&acc_empty[buf], par ^ 1, abort_flag, p.status, p.wait_ns)) break;
        tc_fence_after();
        const uint32_t d = tmem_base + buf * BN;
        bool ok = true;
        for (int kb = k0; kb < k1; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.status, p.wait_ns)) { ok = false; break; }
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
            if constexpr (DW2) {
              // the second 128 output rows, same B operand, into TMEM columns 256..511
              tc_mma<TF32>(d + BN, make_desc(sa2 + kk * 32, 16, 1024), bd, idesc, (kb > k0 || kk > 0) ? 1u : 0u);
            } else if (SPLIT) {
              // low half of the weights: D += W_lo . A on every column, or on the value columns
              constexpr uint32_t idesc_v = make_idesc(TF32 ? 2u : 1u, C::B_MN ? 1u : 0u, TILE_PTS);
              tc_mma<TF32>(d, make_desc(sa2 + kk * 32, 16, 1024), bd, p.wlo_values_only ? idesc_v : idesc, 1u);
            }
            if (C::VLO) {
              // low half of the input's value rows: D[:, 0:64] += W_hi . A_lo
              constexpr uint32_t idesc64 = make_idesc(TF32 ? 2u : 1u, 1u, TILE_PTS);
              tc_mma<TF32>(d, ad, make_desc(sb + C::B_BYTES + kk * C::UK * 128, C::BOX_BYTES, 1024), idesc64, 1u);
            }
          }
          if (C::KPM) {
            // TF32: D += W_hi . B_lo once the converters have written B_lo
            if (!mbar_wait(lo_full, lo_phase, abort_flag, p.status, p.wait_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sbl = smem_u32(blo);
#pragma unroll
            for (int kk = 0; kk < C::BKE / C::UK; ++kk)
              tc_mma<TF32>(d, make_desc(sa + kk * 32, 16, 1024), make_desc(sbl + kk * 32, 16, 1024), idesc, 1u);
            tc_commit(lo_empty);
            lo_phase ^= 1;
          }
          tc_commit(&empty[stage]);
          if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        tc_commit(&acc_full[buf]);
      }
    }
  } else if (C::KPM && warp >= 2 + EPI_WARPS) {
    // ---------------------------------------------------------------- TF32 B_lo converters
    // B_lo = B - tf32(B), elementwise over the stage's B tile (layout-agnostic), into
    // the single B_lo buffer once the MMAs of the previous stage have released it.
    const int ct = threadIdx.x - 32 * (2 + EPI_WARPS);
    int stage = 0;
    uint32_t phase = 0, lo_phase = 0;
    for (int t = grid.bx(); t < total && !*abort_flag; t += grid.gdim()) {
      int mb, nb, k0, k1;
      coords(t, mb, nb, k0, k1);
      bool ok = true;
      for (int kb = k0; kb < k1; ++kb) {
        bool got = mbar_wait(&full[stage], phase, abort_flag, p.status, p.wait_ns) &&
                   mbar_wait(lo_empty, lo_phase ^ 1, abort_flag, p.status, p.wait_ns);
        // both converter warps meet at named barrier 1 below: decide together whether to go on
        {
          uint32_t r;
          asm volatile(
              "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
              : "=r"(r)
              : "r"((uint32_t)got), "n"(32 * C::CVT_WARPS)
              : "memory");
          got = r != 0;
        }
        if (!got) { ok = false; break; }
        const float4* src = reinterpret_cast<const float4*>(smem + stage * C::STAGE + C::A_BYTES * (SPLIT ? 2 : 1));
        float4* dst = reinterpret_cast<float4*>(blo);
        // latency-bound: keep 16 shared-memory loads in flight per thread
        constexpr int U = 16, STRIDE = 32 * (C::CVT_WARPS > 0 ? C::CVT_WARPS : 1);
        static_assert((C::B_BYTES / 16) % (U * STRIDE) == 0, "converter batches cover the tile");
        for (int i0 = ct; i0 < C::B_BYTES / 16; i0 += U * STRIDE) {
          float4 x[U];
#pragma unroll
          for (int u = 0; u < U; ++u) x[u] = src[i0 + u * STRIDE];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            x[u].x -= tf32_trunc(x[u].x); x[u].y -= tf32_trunc(x[u].y);
            x[u].z -= tf32_trunc(x[u].z); x[u].w -= tf32_trunc(x[u].w);
            dst[i0 + u * STRIDE] = x[u];
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
        asm volatile("bar.sync 1, %0;" ::"n"(32 * C::CVT_WARPS) : "memory");
        if (ct == 0) mbar_arrive(lo_full);
        lo_phase ^= 1;
        if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
      }
      if (!ok) break;
    }
  } else if (warp < 2 + EPI_WARPS) {
    // ---------------------------------------------------------------- epilogue
    // Warp part `part` of a lane quadrant handles points 32 part .. 32 part + 31 of the
    // tile in units of UPTS points; a unit is the four UPTS-column chunks at columns
    // pc + 64 r (jet row r), so every thread holds whole points of its feature.  A unit
    // row is one full 32-byte sector (16 BF16 or 8 FP32 values): partial-sector stores
    // would make L2 fetch the sector first.  FP32 units are small enough to double-buffer
    // the TMEM loads; in the adjoint the next unit's Z rows are always loaded one unit
    // ahead (the layer-below activations the adjoint is written in).
    constexpr bool FAST = !TF32;
    constexpr int PARTS = EPI_WARPS / 4;                 // warps per lane quadrant
    constexpr int UPTS = TF32 ? 8 : 16;                  // points per unit
    constexpr int UNITS = TILE_PTS / (UPTS * PARTS);     // units per warp and tile
    constexpr bool PIPE = TF32;                          // double-buffered TMEM loads
    static_assert(PARTS * UNITS * UPTS == TILE_PTS && UNITS % 2 == 0, "epilogue units cover a 64-point tile");
    constexpr int ZW = (int)sizeof(T) * UPTS / 4;        // 32-bit words of one Z row of a unit
    const int quad = warp & 3;
    const int part = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    auto unit_col = [&](int u) { return part * (UNITS * UPTS) + UPTS * u; };

    constexpr int ZR = 4;                                // jet rows loaded per unit
    uint32_t znext[ZR][ZW];                              // adjoint: A rows of the next unit
    auto load_z = [&](int t_, int u_) {
      int mb_, nb_, k0_, k1_;
      coords(t_, mb_, nb_, k0_, k1_);
      const int m_ = mb_ * BM + row;
      if (m_ < p.M) {
        const T* zr = reinterpret_cast<const T*>(p.e.ain) + toff(m_, (int64_t)nb_ * BN, p.M) + unit_col(u_);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if constexpr (UPTS == 8) ld8raw(zr + 64 * r, znext[r]);
          else ld_global_256(zr + 64 * r, znext[r]);
        }
      }
    };
    if constexpr (MODE == TC_ADJ && !SINE) {
      if (grid.bx() < total) load_z(grid.bx(), 0);
    }

    int local = 0;
    for (int t = grid.bx(); t < total; t += grid.gdim(), ++local) {
      int mb, nb, k0, k1;
      coords(t, mb, nb, k0, k1);
      const int buf = DW2 ? 0 : local & 1;
      if (!mbar_wait(&acc_full[buf], DW2 ? ((uint32_t)local & 1) : ((uint32_t)(local >> 1) & 1), abort_flag,
                     p.status, p.wait_ns)) break;
      tc_fence_after();
      for (int half = 0; half < (DW2 ? 2 : 1); ++half) {
      const int m = mb * MROWS + half * BM + row;
      const bool mvalid = m < p.M;
      const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) + (DW2 ? half : buf) * BN;
      float db[4] = {0.f, 0.f, 0.f, 0.f};

      auto issue = [&](int u, float (&v)[4][UPTS]) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if constexpr (UPTS == 8) tmem_ld8_issue(tbase + unit_col(u) + 64 * r, v[r]);
          else tmem_ld16_issue(tbase + unit_col(u) + 64 * r, v[r]);
        }
      };
      auto process = [&](int u, float (&v)[4][UPTS]) {
        uint32_t zw[ZR][ZW];
        if constexpr (MODE == TC_ADJ && !SINE) {
#pragma unroll
          for (int r = 0; r < ZR; ++r)
#pragma unroll
            for (int j = 0; j < ZW; ++j) zw[r][j] = znext[r][j];
          if (u + 1 < UNITS) load_z(t, u + 1);
          else if (t + grid.gdim() < total) load_z(t + grid.gdim(), 0);
        }
        if (!mvalid) return;
        const int pc = unit_col(u);                                   // first point of the unit in its tile
        const int64_t cbase = toff(m, (int64_t)nb * BN, p.M) + pc;    // tile nb, row m
        if constexpr (MODE == TC_FWD) {
          const float bias = p.e.bias[m];
#pragma unroll
          for (int i = 0; i < UPTS; ++i) v[0][i] += bias;
          if constexpr (SINE) {
            // the pre-activation jets for the adjoint, FP32 [M][NC] tile-major
            float* zo = p.e.zout + cbase;
#pragma unroll
            for (int r = 0; r < 4; ++r) st_f32<UPTS>(zo + 64 * r, v[r]);
          }
#pragma unroll
          for (int i = 0; i < UPTS; ++i) {
            float z[4] = {v[0][i], v[1][i], v[2][i], v[3][i]}, a[4];
            if constexpr (SINE) jet_fwd_sine(z, a, p.e.jet_mode, p.e.omega0);
            else jet_fwd<FAST>(z, a, p.e.jet_mode);
#pragma unroll
            for (int r = 0; r < 4; ++r) v[r][i] = a[r];
          }
          T* ao = reinterpret_cast<T*>(p.e.out) + cbase;
#pragma unroll
          for (int r = 0; r < 4; ++r) st_row(ao + 64 * r, v[r]);
          if constexpr (TF32) {
            if (p.e.out_pm) store_pm8(reinterpret_cast<float*>(p.e.out_pm), (int64_t)nb * BN + pc, p.M, m, v);
          }
          if (!TF32 && p.e.alo_out) {
            // low half of the value rows for the next forward (BF16 rounding remainder)
            float lo[UPTS];
#pragma unroll
            for (int i = 0; i < UPTS; ++i) lo[i] = v[0][i] - __bfloat162float(__float2bfloat16_rn(v[0][i]));
            st_row(reinterpret_cast<T*>(p.e.alo_out) + loff(m, (int64_t)nb * TILE_PTS, p.M) + pc, lo);
          }
        } else if constexpr (MODE == TC_ADJ) {
          if constexpr (SINE) {
            // the rule from the stored pre-activation jets z of the layer below
            const float* zr = p.e.zin + cbase;
#pragma unroll
            for (int h8 = 0; h8 < UPTS / 8; ++h8) {
              uint32_t zz[4][8];
#pragma unroll
              for (int r = 0; r < 4; ++r) ld_global_256(zr + 64 * r + 8 * h8, zz[r]);
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                float z[4] = {__uint_as_float(zz[0][i]), __uint_as_float(zz[1][i]), __uint_as_float(zz[2][i]),
                              __uint_as_float(zz[3][i])};
                const int k = 8 * h8 + i;
                float ab[4] = {v[0][k], v[1][k], v[2][k], v[3][k]}, zb[4];
                jet_adj_sine(z, ab, zb, p.e.jet_mode, p.e.omega0);
#pragma unroll
                for (int r = 0; r < 4; ++r) v[r][k] = zb[r];
              }
            }
          } else {
#pragma unroll
            for (int i = 0; i < UPTS; ++i) {
              float av[4];
#pragma unroll
              for (int r = 0; r < 4; ++r) av[r] = raw_elem<T>(zw[r], i);
              float ab[4] = {v[0][i], v[1][i], v[2][i], v[3][i]}, zb[4];
              jet_adj_a(av, ab, zb, p.e.jet_mode);
#pragma unroll
              for (int r = 0; r < 4; ++r) v[r][i] = zb[r];
            }
          }
          T* zbo = reinterpret_cast<T*>(p.e.out) + cbase;
#pragma unroll
          for (int r = 0; r < 4; ++r) st_row(zbo + 64 * r, v[r]);
          if constexpr (TF32) {
            if (p.e.out_pm) store_pm8(reinterpret_cast<float*>(p.e.out_pm), (int64_t)nb * BN + pc, p.M, m, v);
          }
          if (p.e.dbpart) {
            // bias gradient of the layer below (value rows) and, for a first layer on
            // raw coordinates, the coordinate terms of its weight gradient
#pragma unroll
            for (int i = 0; i < UPTS; ++i) db[0] += v[0][i];
            if (p.e.dterms) {
              const int64_t p0 = (int64_t)nb * TILE_PTS + pc;
              const int nd = (p.e.jet_mode == JET_MAXWELL) ? 3 : 2;   // rows 1..nd are first derivatives
#pragma unroll
              for (int i = 0; i < UPTS; ++i) {
                const int64_t pp = p0 + i;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                  if (j >= p.e.dterms) break;
                  float x = point_coord(p.e.x_res, p.e.x_ic, p.e.x_bc, p.e.n_res, p.e.n_ic, p.e.n_bc, pp, j);
                  db[1 + j] = fmaf(v[0][i], x, db[1 + j]);
                  if (j < nd) db[1 + j] += v[1 + j][i];
                }
              }
            }
          }
        } else if constexpr (MODE == TC_DW) {
          const int split = t / (p.m_tiles * p.n_tiles);
          float* dst = p.out32 + ((int64_t)split * p.M + m) * p.N;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int64_t col0 = (int64_t)nb * BN + pc + 64 * r;
            if (col0 + UPTS <= p.N && (p.N & 7) == 0) {
              st_f32<UPTS>(dst + col0, v[r]);
            } else {
              for (int j = 0; j < UPTS; ++j)
                if (col0 + j < p.N) dst[col0 + j] = v[r][j];
            }
          }
        } else {   // TC_STORE
#pragma unroll
          for (int r = 0; r < 4; ++r) st_f32<UPTS>(p.out32 + cbase + 64 * r, v[r]);
        }
      };

      if constexpr (PIPE) {
        float va[4][UPTS], vb[4][UPTS];
        issue(0, va);
        tmem_wait_ld();
#pragma unroll 1
        for (int u = 0; u < UNITS; u += 2) {
          issue(u + 1, vb);
          process(u, va);
          tmem_wait_ld();
          if (u + 2 < UNITS) issue(u + 2, va);
          process(u + 1, vb);
          if (u + 2 < UNITS) tmem_wait_ld();
        }
      } else {
#pragma unroll 1
        for (int u = 0; u < UNITS; ++u) {
          float va[4][UPTS];
          issue(u, va);
          tmem_wait_ld();
          process(u, va);
        }
      }
      if (MODE == TC_ADJ && mvalid && p.e.dbpart) {
        float* dst = p.e.dbpart + ((int64_t)m * (p.n_tiles * PARTS) + nb * PARTS + part) * (1 + p.e.dterms);
        dst[0] = db[0];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (j < p.e.dterms) dst[1 + j] = db[1 + j];
      }
      }   // half
      tc_fence_before();
      mbar_arrive(&acc_empty[buf]);
    }
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

template <bool TF32, int MODE, bool SPLIT, bool SINE = false>
__global__ void __launch_bounds__(Cfg<TF32, MODE, SPLIT>::NTHREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapA2,
              const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapBlo,
              const __grid_constant__ TcParams p) {
  tc_gemm_body<TF32, MODE, SPLIT, SINE>(&mapA, &mapA2, &mapB, &mapBlo, p, SingleGrid{});
}

// Grouped launch: the GEMMs of several networks (or layers) side by side, each entry of
// the device table holding one GEMM's tensor maps and parameters and its block range.
template <bool TF32, int MODE, bool SPLIT, bool SINE = false>
__global__ void __launch_bounds__(Cfg<TF32, MODE, SPLIT>::NTHREADS, 1)
    k_tc_gemm_group(const TcGroupEntry* __restrict__ tab, const int n) {
  const TcGroupEntry& g = tab[group_of_block(tab, n, (int)blockIdx.x)];
  acquire_maps(g, 4);
  tc_gemm_body<TF32, MODE, SPLIT, SINE>(&g.map[0], &g.map[1], &g.map[2], &g.map[3], g.p,
                                        GroupShare{(int)blockIdx.x - g.block0, g.grid});
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

// 3-D tensor map over a tile-major jet matrix [ntiles][rows][tcols] (tcols = 256 for
// jet matrices, 64 for value-row low halves), box [1][box_rows][box_cols], 128-byte
// swizzle, zero fill out of bounds.
bool make_map3(CUtensorMap* m, const void* base, bool tf32, uint64_t tcols, uint64_t rows, uint64_t ntiles,
               uint32_t box_cols, uint32_t box_rows) {
  if (!g_encode) return false;
  const uint32_t es = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {tcols, rows, ntiles};
  cuuint64_t strides[2] = {tcols * es, tcols * rows * es};
  cuuint32_t box[3] = {box_cols, box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool tc_map3(CUtensorMap* m, const void* base, bool fp32, uint64_t tcols, uint64_t rows, uint64_t ntiles,
             uint32_t box_cols, uint32_t box_rows) {
  return make_map3(m, base, fp32, tcols, rows, ntiles, box_cols, box_rows);
}

namespace {

// Reserves the dynamic shared memory of kernel `kern` once per kernel.
template <typename K>
pinn_status reserve_smem(pinn_handle* h, K kern, size_t bytes, bool& done, const char* what) {
  if (done) return PINN_OK;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    cudaGetLastError();   // do not leave the failure for the next launch to report
    snprintf(h->err, sizeof(h->err), "%s: cannot reserve %zu bytes of shared memory", what, bytes);
    return PINN_ERR_CUDA;
  }
  done = true;
  return PINN_OK;
}

pinn_status launch_check(pinn_handle* h, const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return PINN_OK;
  snprintf(h->err, sizeof(h->err), "%s launch: %s", what, cudaGetErrorString(e));
  return PINN_ERR_CUDA;
}

// Grouped launch of n table entries (blocks in all) of one GEMM kernel variant.
template <bool TF32, int MODE, bool SPLIT, bool SINE>
pinn_status launch_group(pinn_handle* h, const TcGroupEntry* d_tab, int n, int blocks, cudaStream_t st) {
  using C = Cfg<TF32, MODE, SPLIT>;
  auto kern = k_tc_gemm_group<TF32, MODE, SPLIT, SINE>;
  static bool attr_set = false;   // per instantiation
  pinn_status s = reserve_smem(h, kern, C::SMEM, attr_set, "grouped tcgen05 kernel");
  if (s) return s;
  kern<<<blocks, C::NTHREADS, C::SMEM, st>>>(d_tab, n);
  return launch_check(h, "grouped tcgen05 kernel");
}

pinn_status launch_adjdw_group(pinn_handle* h, const TcGroupEntry* d_tab, int n, int blocks, cudaStream_t st);

}  // namespace

// Tensor-core GEMMs collected from several handles (tc_batch_attach) and issued as
// grouped launches: one per kernel variant, the GEMMs with the most work first.
struct TcBatch {
  using GroupFn = pinn_status (*)(pinn_handle*, const TcGroupEntry*, int, int, cudaStream_t);
  struct Item {
    GroupFn fn;
    TcGroupEntry e;
    double work;   // tiles x K iterations: the order of the grouped grid
  };
  std::vector<Item> pending;
  std::vector<TcGroupEntry> table;   // every issued entry, in device-table order
  TcGroupEntry* d_table = nullptr;
  size_t capacity = 0;               // entries d_table holds
  int launches = 0;
};

namespace {

pinn_status batch_add(TcBatch* b, TcBatch::GroupFn fn, const CUtensorMap* maps, int nmaps, const TcParams& p,
                      int grid) {
  TcBatch::Item it{};
  it.fn = fn;
  for (int i = 0; i < nmaps; ++i) it.e.map[i] = maps[i];
  it.e.p = p;
  it.e.grid = grid;
  it.work = (double)p.m_tiles * p.n_tiles * std::max(p.k_iters, 1);
  b->pending.push_back(it);
  return PINN_OK;
}

template <bool TF32, int MODE, bool SPLIT, bool SINE = false>
pinn_status launch(pinn_handle* h, const CUtensorMap& a, const CUtensorMap& a2, const CUtensorMap& b,
                   const CUtensorMap& blo, const TcParams& p, int grid, cudaStream_t st) {
  if (h->tc_batch) {
    const CUtensorMap maps[4] = {a, a2, b, blo};
    return batch_add(h->tc_batch, &launch_group<TF32, MODE, SPLIT, SINE>, maps, 4, p, grid);
  }
  using C = Cfg<TF32, MODE, SPLIT>;
  auto kern = k_tc_gemm<TF32, MODE, SPLIT, SINE>;
  static bool attr_set = false;   // per instantiation
  pinn_status s = reserve_smem(h, kern, C::SMEM, attr_set, "tcgen05 kernel");
  if (s) return s;
  kern<<<grid, C::NTHREADS, C::SMEM, st>>>(a, a2, b, blo, p);
  return launch_check(h, "tcgen05 kernel");
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
  if (!g_encode || h->spec.precision == PINN_FP32 || (h->spec.flags & PINN_FLAG_CUDA_CORES)) return false;
  // the tensor-core epilogues carry the tanh jet, and (BF16) the sine jet
  if (h->act != PINN_ACT_TANH && !(h->act == PINN_ACT_SINE && h->spec.precision == PINN_BF16)) return false;
  if (NC % BN) return false;
  const int fin = h->layers[li].fin, fout = h->layers[li].fout;
  // TMA row strides must be multiples of 16 bytes: fin and fout multiples of 8 elements.
  return (fin % 8 == 0) && (fout % 8 == 0) && fin >= 16 && fout >= 16;
}

// Weight-gradient tiles have 256 output rows (two accumulators sharing B) when the
// layer has more than 256 outputs, else (or with PINN_FLAG_DW_ROWS_128) 128.  At 256
// outputs the 256-row tile is a single work item per column split, and two 128-row
// items per split balance better (measured: 0.063 -> 0.059 ms at the 6x256 cavity, and
// half as many split partials for the finalisation to sum).
static int dw_rows(const pinn_handle* h, int fout) {
  return (fout > 2 * BM && !(h->spec.flags & PINN_FLAG_DW_ROWS_128)) ? 2 * BM : BM;
}

int tc_dw_splits(const pinn_handle* h, int fout, int fin, int64_t NC) {
  const int tiles = ((fout + dw_rows(h, fout) - 1) / dw_rows(h, fout)) * ((fin + BN - 1) / BN);
  const int kblock = (h->spec.precision == PINN_TF32) ? 32 : 64;
  const int k_iters = (int)((NC + kblock - 1) / kblock);
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
  p.wait_ns = WAIT_NS;
  p.stall = 0;
  return p;
}

pinn_status map_err(pinn_handle* h, const char* what) {
  snprintf(h->err, sizeof(h->err), "cuTensorMapEncodeTiled failed for %s", what);
  return PINN_ERR_CUDA;
}

}  // namespace

namespace {

template <bool TF32>
pinn_status fwd_impl(pinn_handle* h, const void* W, const void* Wlo, const void* A, const void* Alo, int fout, int fin,
                     int64_t NC, const EpiArgs& e, cudaStream_t st) {
  using C = Cfg<TF32, TC_FWD, true>;
  CUtensorMap ma, ma2, mb, mlo;
  const uint64_t nt = (uint64_t)(NC / TILE_COLS);
  if (!make_map(&ma, W, TF32, fin, fout, C::BKE, BM) || !make_map(&ma2, Wlo, TF32, fin, fout, C::BKE, BM))
    return map_err(h, "forward weights");
  if (TF32) {
    // point-major jets [NC][fin], K-major boxes of BKE features x BN columns
    if (!make_map(&mb, A, true, fin, (uint64_t)NC, C::BKE, BN)) return map_err(h, "forward activations");
    mlo = mb;
  } else {
    if (!make_map3(&mb, A, false, TILE_COLS, fin, nt, C::BOXN, C::BKE)) return map_err(h, "forward activations");
    if (!make_map3(&mlo, Alo, false, TILE_PTS, fin, nt, C::BOXN, C::BKE))
      return map_err(h, "forward value-row low half");
  }
  TcParams p = base_params(fout, (int)NC, fin, NC, C::BKE, h->d_status);
  p.e = e;
  p.wlo_values_only = (!TF32 && (h->spec.flags & PINN_FLAG_BF16_VALUE_SPLIT)) ? 1 : 0;
  const int grid = grid_for(h, p.m_tiles * p.n_tiles);
  if constexpr (!TF32)
    if (h->act == PINN_ACT_SINE) return launch<TF32, TC_FWD, true, true>(h, ma, ma2, mb, mlo, p, grid, st);
  return launch<TF32, TC_FWD, true>(h, ma, ma2, mb, mlo, p, grid, st);
}

template <bool TF32>
pinn_status adj_impl(pinn_handle* h, const void* WT, const void* WTlo, const void* Zbar, int fin, int fout,
                     int64_t NC, const EpiArgs& e, cudaStream_t st) {
  // TF32: split weights and the point-major adjoint with its low half (three MMAs);
  // BF16: high halves only.
  constexpr bool SPLIT = TF32;
  using C = Cfg<TF32, TC_ADJ, SPLIT>;
  CUtensorMap ma, ma2, mb;
  if (!make_map(&ma, WT, TF32, fout, fin, C::BKE, BM)) return map_err(h, "adjoint weights");
  ma2 = ma;
  if (TF32) {
    if (!make_map(&ma2, WTlo, true, fout, fin, C::BKE, BM)) return map_err(h, "adjoint weights (low half)");
    if (!make_map(&mb, Zbar, true, fout, (uint64_t)NC, C::BKE, BN)) return map_err(h, "adjoint input");
  } else {
    if (!make_map3(&mb, Zbar, false, TILE_COLS, fout, (uint64_t)(NC / TILE_COLS), C::BOXN, C::BKE))
      return map_err(h, "adjoint input");
  }
  TcParams p = base_params(fin, (int)NC, fout, NC, C::BKE, h->d_status);
  p.e = e;
  const int grid = grid_for(h, p.m_tiles * p.n_tiles);
  if constexpr (!TF32)
    if (h->act == PINN_ACT_SINE) return launch<TF32, TC_ADJ, SPLIT, true>(h, ma, ma2, mb, mb, p, grid, st);
  return launch<TF32, TC_ADJ, SPLIT>(h, ma, ma2, mb, mb, p, grid, st);
}

template <bool TF32>
pinn_status dw_impl(pinn_handle* h, const void* Zbar, const void* A, int fout, int fin, int64_t NC, int nsplit,
                    float* part, cudaStream_t st) {
  using C = Cfg<TF32, TC_DW, false>;   // (the 256-row variant stages the same boxes, twice for A)
  const bool two = dw_rows(h, fout) > BM;
  CUtensorMap ma, mb;
  const uint64_t nt = (uint64_t)(NC / TILE_COLS);
  if (!make_map3(&ma, Zbar, TF32, TILE_COLS, fout, nt, C::BKE, BM)) return map_err(h, "weight-gradient adjoint");
  if (!make_map3(&mb, A, TF32, TILE_COLS, fin, nt, C::BKE, BN)) return map_err(h, "weight-gradient activations");
  TcParams p = base_params(fout, fin, (int)NC, NC, C::BKE, h->d_status);
  if (two) p.m_tiles = (fout + 2 * BM - 1) / (2 * BM);
  p.nsplit = nsplit;
  p.kps = (p.k_iters + nsplit - 1) / nsplit;
  if ((p.k_iters + p.kps - 1) / p.kps != nsplit) {
    snprintf(h->err, sizeof(h->err), "weight-gradient split plan mismatch");
    return PINN_ERR_INVALID_ARG;
  }
  p.out32 = part;
  const int grid = grid_for(h, p.m_tiles * p.n_tiles * nsplit);
  if (two) return launch<TF32, TC_DW, true>(h, ma, ma, mb, mb, p, grid, st);
  return launch<TF32, TC_DW, false>(h, ma, ma, mb, mb, p, grid, st);
}

}  // namespace

pinn_status tc_gemm_fwd(pinn_handle* h, const void* W, const void* Wlo, const void* A, const void* Alo, int fout,
                        int fin, int64_t NC, const EpiArgs& e, cudaStream_t st) {
  if (h->spec.precision == PINN_TF32) return fwd_impl<true>(h, W, Wlo, A, Alo, fout, fin, NC, e, st);
  return fwd_impl<false>(h, W, Wlo, A, Alo, fout, fin, NC, e, st);
}

pinn_status tc_gemm_adj(pinn_handle* h, const void* WT, const void* WTlo, const void* Zbar, int fin, int fout,
                        int64_t NC, const EpiArgs& e, cudaStream_t st) {
  if (h->spec.precision == PINN_TF32) return adj_impl<true>(h, WT, WTlo, Zbar, fin, fout, NC, e, st);
  return adj_impl<false>(h, WT, WTlo, Zbar, fin, fout, NC, e, st);
}

pinn_status tc_gemm_dw(pinn_handle* h, const void* Zbar, const void* A, int fout, int fin, int64_t NC, int nsplit,
                       float* part, cudaStream_t st) {
  if (h->spec.precision == PINN_TF32) return dw_impl<true>(h, Zbar, A, fout, fin, NC, nsplit, part, st);
  return dw_impl<false>(h, Zbar, A, fout, fin, NC, nsplit, part, st);
}

// ==== fused adjoint + weight gradient (BF16, fan-out <= 256) ==========================
//
// For a hidden layer whose adjoint and weight gradient both run on tensor cores, the
// two GEMMs read the same two arrays for the same column tile: Zbar_l^T [fout][NC]
// and A_{l-1}^T [fin][NC].  One persistent kernel does both per work unit (fin
// m-tile mb, column tile nb):
//   adjoint  Abar^T[mb rows][256 cols] = W^T[mb rows][fout] . Zbar^T[fout][256 cols]
//            (MN-major B), then the activation-form tanh-jet adjoint in the epilogue
//   weights  dW^T[mb rows][fout] += A_{l-1}^T[mb rows][256 cols] . Zbar^T[fout][256 cols]^T
//            (both K-major over the columns), accumulated in tensor memory across all
//            of the CTA's column tiles and written once as its split partial.
// Every CTA keeps one m-tile (the grid is a multiple of the m-tile count), so its dW
// slab stays in tensor memory: 256 columns for the adjoint accumulator (single
// buffer; the epilogue copies it to registers and releases it at once) plus up to
// 256 for dW^T.  The A_{l-1} tile is staged by TMA in shared memory (two buffers)
// and serves both the dW MMAs and the epilogue, which reads it from there instead of
// global memory.  Zbar is read once from HBM per column tile (the m-tile CTAs of a
// column tile run side by side, the second read hits L2), A once, Zbar_{l-1} written
// once: the separate weight-gradient pass and its re-reads are gone.
//
// Warp roles (352 threads): 0 stage producer (W^T chunk + Zbar chunk), 1 TMEM
// allocator + MMA issuer, 2-9 epilogue, 10 A-tile producer.
namespace {

constexpr int FZ_EPI = EPI_WARPS;
constexpr int FZ_NT = 64 + 32 * FZ_EPI + 32;
constexpr int FZ_WB = BM * 128;                  // W^T chunk [128 fin][64 fout]       16 KB
constexpr int FZ_BOX = 64 * 128;                 // Zbar box [64 fout][64 cols]         8 KB
constexpr int FZ_ZB = 4 * FZ_BOX;                // Zbar chunk [64 fout][256 cols]     32 KB
constexpr int FZ_STAGE = FZ_WB + FZ_ZB;          // 48 KB
constexpr int FZ_STAGES = 2;
constexpr int FZ_ABOX = BM * 128;                // A box [128 fin][64 cols]           16 KB
constexpr int FZ_AT = 4 * FZ_ABOX;               // A_{l-1} tile [128 fin][256 cols]   64 KB
constexpr int FZ_ABUF = 2;
constexpr size_t FZ_SMEM = (size_t)FZ_STAGES * FZ_STAGE + (size_t)FZ_ABUF * FZ_AT + 1024 + 256;
static_assert(FZ_SMEM <= 227 * 1024, "fused adjoint: shared memory budget");
constexpr int FZ_DW_COL = BN;                    // dW^T accumulator: TMEM columns 256..511

template <typename Grid>
__device__ __forceinline__ void tc_adjdw_body(const CUtensorMap* mapW, const CUtensorMap* mapZ,
                                              const CUtensorMap* mapA, const TcParams& p, const Grid grid) {
  using T = __nv_bfloat16;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned by offsetting the shared array itself (an integer round trip would
  // hide the address space and turn every shared access below into a generic one)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* abase = smem + FZ_STAGES * FZ_STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(abase + FZ_ABUF * FZ_AT);
  uint64_t* empty = full + FZ_STAGES;
  uint64_t* acc_full = empty + FZ_STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* a_full = acc_empty + 1;
  uint64_t* a_empty = a_full + FZ_ABUF;
  uint64_t* dw_full = a_empty + FZ_ABUF;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(dw_full + 1);
  volatile int* inflight = abort_flag + 1;              // [FZ_STAGES]
  volatile int* a_inflight = inflight + FZ_STAGES;      // [FZ_ABUF]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(const_cast<int*>(a_inflight + FZ_ABUF));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < FZ_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      inflight[s] = 0;
    }
    for (int b = 0; b < FZ_ABUF; ++b) {
      mbar_init(&a_full[b], 1);
      mbar_init(&a_empty[b], 1 + 32 * FZ_EPI);   // the dW MMAs' commit + every epilogue thread
      a_inflight[b] = 0;
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 32 * FZ_EPI);
    mbar_init(dw_full, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int total = p.m_tiles * p.n_tiles;
  auto coords = [&](int t, int& mb, int& nb) {
    if (p.e.reverse) t = total - 1 - t;
    mb = t % p.m_tiles;
    nb = t / p.m_tiles;
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- stage producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int t = grid.bx(); t < total && !*abort_flag; t += grid.gdim()) {
        int mb, nb;
        coords(t, mb, nb);
        for (int kb = 0; kb < p.k_iters; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, p.status, p.wait_ns)) break;
          uint8_t* sw = smem + stage * FZ_STAGE;
          uint8_t* sz = sw + FZ_WB;
          mbar_expect_tx(&full[stage], FZ_STAGE);
          inflight[stage] = (int)phase + 1;
          tma_load_2d(sw, mapW, &full[stage], kb * 64, mb * BM);
#pragma unroll
          for (int j = 0; j < 4; ++j) tma_load_3d(sz + j * FZ_BOX, mapZ, &full[stage], j * 64, kb * 64, nb);
          if (++stage == FZ_STAGES) { stage = 0; phase ^= 1; }
        }
      }
    }
  } else if (warp == 2 + FZ_EPI) {
    // ---------------------------------------------------------------- A-tile producer
    if (lane == 0) {
      int local = 0;
      for (int t = grid.bx(); t < total && !*abort_flag; t += grid.gdim(), ++local) {
        int mb, nb;
        coords(t, mb, nb);
        const int ab = local & 1;
        const uint32_t aph = (uint32_t)(local >> 1) & 1;
        if (!mbar_wait(&a_empty[ab], aph ^ 1, abort_flag, p.status, p.wait_ns)) break;
        mbar_expect_tx(&a_full[ab], FZ_AT);
        a_inflight[ab] = (int)aph + 1;
        uint8_t* at = abase + ab * FZ_AT;
#pragma unroll
        for (int j = 0; j < 4; ++j) tma_load_3d(at + j * FZ_ABOX, mapA, &a_full[ab], j * 64, mb * BM, nb);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc_adj = make_idesc(1u, 1u, BN);   // W^T . Zbar, B MN-major, N = 256
      constexpr uint32_t idesc_dw = make_idesc(1u, 0u, 64);    // A_{l-1} . Zbar chunk^T, both K-major, N = 64
      const uint32_t d_adj = tmem_base;
      const uint32_t d_dw = tmem_base + FZ_DW_COL;
      int stage = 0;
      uint32_t phase = 0;
      int local = 0;
      bool ok = true;
      for (int t = grid.bx(); t < total && !*abort_flag && ok; t += grid.gdim(), ++local) {
        const int ab = local & 1;
        if (!mbar_wait(&a_full[ab], (uint32_t)(local >> 1) & 1, abort_flag, p.status, p.wait_ns)) { ok = false; break; }
        a_inflight[ab] = 0;
        tc_fence_after();
        const uint32_t sa_t = smem_u32(abase + ab * FZ_AT);
        for (int kb = 0; kb < p.k_iters; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.status, p.wait_ns)) { ok = false; break; }
          inflight[stage] = 0;
          tc_fence_after();
          const uint32_t sw = smem_u32(smem + stage * FZ_STAGE);
          const uint32_t sz = sw + FZ_WB;
          // weight gradient of this 64-row fout chunk: dW^T[:, 64 kb ..] += A_tile . Zbar_chunk^T
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc_mma<false>(d_dw + 64 * kb, make_desc(sa_t + j * FZ_ABOX + kk * 32, 16, 1024),
                            make_desc(sz + j * FZ_BOX + kk * 32, 16, 1024), idesc_dw,
                            (local > 0 || j > 0 || kk > 0) ? 1u : 0u);
          if (kb == 0) {
            // the single adjoint accumulator: wait until the epilogue has copied out the last tile
            if (!mbar_wait(acc_empty, ((uint32_t)local & 1) ^ 1, abort_flag, p.status, p.wait_ns)) { ok = false; break; }
            tc_fence_after();
          }
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            tc_mma<false>(d_adj, make_desc(sw + kk * 32, 16, 1024), make_desc(sz + kk * 16 * 128, FZ_BOX, 1024),
                          idesc_adj, (kb > 0 || kk > 0) ? 1u : 0u);
          tc_commit(&empty[stage]);
          if (++stage == FZ_STAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        tc_commit(&a_empty[ab]);
        tc_commit(acc_full);
      }
      if (ok && !*abort_flag) tc_commit(dw_full);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    constexpr int PARTS = FZ_EPI / 4;
    constexpr int UPTS = 16;
    constexpr int UNITS = TILE_PTS / (UPTS * PARTS);   // 2
    const int quad = warp & 3;
    const int part = (warp - 2) >> 2;
    const int rr = quad * 32 + lane;                    // accumulator row = feature within the m-tile
    auto unit_col = [&](int u) { return part * (UNITS * UPTS) + UPTS * u; };
    const uint32_t tq = tmem_base + ((uint32_t)(quad * 32) << 16);
    int local = 0;
    int mb_cta = 0;
    for (int t = grid.bx(); t < total; t += grid.gdim(), ++local) {
      int mb, nb;
      coords(t, mb, nb);
      mb_cta = mb;
      if (!mbar_wait(acc_full, (uint32_t)local & 1, abort_flag, p.status, p.wait_ns)) break;
      tc_fence_after();
      float v[UNITS][4][UPTS];
#pragma unroll
      for (int u = 0; u < UNITS; ++u)
#pragma unroll
        for (int r = 0; r < 4; ++r) tmem_ld16_issue(tq + unit_col(u) + 64 * r, v[u][r]);
      tmem_wait_ld();
      tc_fence_before();
      mbar_arrive(acc_empty);            // the next tile's adjoint MMAs may overwrite it now
      const int ab = local & 1;
      if (!mbar_wait(&a_full[ab], (uint32_t)(local >> 1) & 1, abort_flag, p.status, p.wait_ns)) break;
      const uint8_t* at = abase + ab * FZ_AT;
      const int m = mb * BM + rr;
      const bool mvalid = m < p.M;
      float db[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int pc = unit_col(u);
#pragma unroll
        for (int h8 = 0; h8 < UPTS / 8; ++h8) {
          // A_{l-1} of 8 points x 4 jet rows from the swizzled tile: row rr of box r,
          // 16-byte chunk (pc + 8 h8) / 8 XOR (rr mod 8)
          uint32_t aw[4][4];
          const int chunk = ((pc + 8 * h8) >> 3) ^ (rr & 7);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const uint32_t addr = smem_u32(at + r * FZ_ABOX + rr * 128 + chunk * 16);
            asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(aw[r][0]), "=r"(aw[r][1]), "=r"(aw[r][2]), "=r"(aw[r][3])
                         : "r"(addr));
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            float av[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) av[r] = raw_elem<T>(aw[r], i);
            float abr[4] = {v[u][0][8 * h8 + i], v[u][1][8 * h8 + i], v[u][2][8 * h8 + i], v[u][3][8 * h8 + i]};
            float zb[4];
            jet_adj_a(av, abr, zb, p.e.jet_mode);
#pragma unroll
            for (int r = 0; r < 4; ++r) v[u][r][8 * h8 + i] = zb[r];
          }
        }
        if (mvalid) {
          const int64_t cbase = toff(m, (int64_t)nb * BN, p.M) + pc;
          T* zbo = reinterpret_cast<T*>(p.e.out) + cbase;
#pragma unroll
          for (int r = 0; r < 4; ++r) st_row(zbo + 64 * r, v[u][r]);
          if (p.e.dbpart) {
#pragma unroll
            for (int i = 0; i < UPTS; ++i) db[0] += v[u][0][i];
            if (p.e.dterms) {
              const int64_t p0 = (int64_t)nb * TILE_PTS + pc;
              const int nd = (p.e.jet_mode == JET_MAXWELL) ? 3 : 2;
#pragma unroll
              for (int i = 0; i < UPTS; ++i) {
                const int64_t pp = p0 + i;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                  if (j >= p.e.dterms) break;
                  float x = point_coord(p.e.x_res, p.e.x_ic, p.e.x_bc, p.e.n_res, p.e.n_ic, p.e.n_bc, pp, j);
                  db[1 + j] = fmaf(v[u][0][i], x, db[1 + j]);
                  if (j < nd) db[1 + j] += v[u][1 + j][i];
                }
              }
            }
          }
        }
      }
      // done with this A tile: its ordinary shared loads ordered before the next bulk copy
      // into the buffer (the mbarrier orders the generic proxy only)
      fence_proxy_async_smem();
      mbar_arrive(&a_empty[ab]);
      if (mvalid && p.e.dbpart) {
        float* dst = p.e.dbpart + ((int64_t)m * (p.n_tiles * PARTS) + nb * PARTS + part) * (1 + p.e.dterms);
        dst[0] = db[0];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (j < p.e.dterms) dst[1 + j] = db[1 + j];
      }
    }
    // this CTA's dW^T slab (its m-tile rows x all fout) as split partial (CTA index) / m_tiles
    if (local > 0 && !*abort_flag && mbar_wait(dw_full, 0, abort_flag, p.status, p.wait_ns)) {
      tc_fence_after();
      const int m = mb_cta * BM + rr;
      const int split = grid.bx() / p.m_tiles;
      const int f0 = part * 128;
      for (int c = 0; c < 128; c += 16) {
        if (f0 + c >= p.K) break;
        float d[16];
        tmem_ld16_issue(tq + FZ_DW_COL + f0 + c, d);
        tmem_wait_ld();
        if (m < p.M) {
          float* dst = p.out32 + ((int64_t)split * p.K + f0 + c) * p.M + m;
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (f0 + c + i < p.K) dst[(int64_t)i * p.M] = d[i];
        }
      }
    }
  }

  // ---- teardown: wait (bounded) for copies still in flight, free TMEM ----------------
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    for (int s = 0; s < FZ_STAGES; ++s) {
      const int f = inflight[s];
      if (f) {
        const uint64_t t0 = gtimer();
        while (!mbar_try(&full[s], (uint32_t)(f - 1)) && gtimer() - t0 < WAIT_NS) {}
      }
    }
    for (int b = 0; b < FZ_ABUF; ++b) {
      const int f = a_inflight[b];
      if (f) {
        const uint64_t t0 = gtimer();
        while (!mbar_try(&a_full[b], (uint32_t)(f - 1)) && gtimer() - t0 < WAIT_NS) {}
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

__global__ void __launch_bounds__(FZ_NT, 1)
    k_tc_adjdw(const __grid_constant__ CUtensorMap mapW, const __grid_constant__ CUtensorMap mapZ,
               const __grid_constant__ CUtensorMap mapA, const __grid_constant__ TcParams p) {
  tc_adjdw_body(&mapW, &mapZ, &mapA, p, SingleGrid{});
}

__global__ void __launch_bounds__(FZ_NT, 1) k_tc_adjdw_group(const TcGroupEntry* __restrict__ tab, const int n) {
  const TcGroupEntry& g = tab[group_of_block(tab, n, (int)blockIdx.x)];
  acquire_maps(g, 3);
  tc_adjdw_body(&g.map[0], &g.map[1], &g.map[2], g.p, GroupShare{(int)blockIdx.x - g.block0, g.grid});
}

int adjdw_grid(const pinn_handle* h, int fin, int64_t NC) {
  const int mt = (fin + BM - 1) / BM;
  const int tiles = mt * (int)(NC / TILE_COLS);
  const int per = std::max(1, std::max(h->sm_count, 1) / mt) * mt;   // a multiple of the m-tile count
  return std::max(mt, std::min(tiles, per));
}

}  // namespace

bool tc_adjdw_supported(const pinn_handle* h, int li, int64_t NC) {
  if (h->spec.precision != PINN_BF16 || li < 1 || !tc_layer_supported(h, li, NC)) return false;
  if (h->spec.flags & PINN_FLAG_UNFUSED_ADJOINT) return false;
  if (h->act != PINN_ACT_TANH) return false;   // the fused epilogue carries the tanh jet only
  return h->layers[li].fout <= BN;   // the dW^T slab fits beside the adjoint accumulator
}

int tc_adjdw_splits(const pinn_handle* h, int fin, int64_t NC) {
  return adjdw_grid(h, fin, NC) / ((fin + BM - 1) / BM);
}

pinn_status tc_gemm_adjdw(pinn_handle* h, const void* WT, const void* Zbar, const void* Ain, int fin, int fout,
                          int64_t NC, const EpiArgs& e, float* dwpart, int nsplit, cudaStream_t st) {
  CUtensorMap mw, mz, ma;
  const uint64_t nt = (uint64_t)(NC / TILE_COLS);
  if (!make_map(&mw, WT, false, fout, fin, 64, BM)) return map_err(h, "fused adjoint weights");
  if (!make_map3(&mz, Zbar, false, TILE_COLS, fout, nt, 64, 64)) return map_err(h, "fused adjoint input");
  if (!make_map3(&ma, Ain, false, TILE_COLS, fin, nt, 64, BM)) return map_err(h, "fused adjoint activations");
  TcParams p = base_params(fin, (int)NC, fout, NC, 64, h->d_status);
  p.e = e;
  p.out32 = dwpart;
  const int grid = adjdw_grid(h, fin, NC);
  if (grid / p.m_tiles != nsplit || grid > p.m_tiles * p.n_tiles) {
    snprintf(h->err, sizeof(h->err), "fused adjoint: split plan mismatch");
    return PINN_ERR_INVALID_ARG;
  }
  p.nsplit = nsplit;
  if (h->tc_batch) {
    const CUtensorMap maps[3] = {mw, mz, ma};
    return batch_add(h->tc_batch, &launch_adjdw_group, maps, 3, p, grid);
  }
  static bool attr_set = false;
  pinn_status s = reserve_smem(h, k_tc_adjdw, FZ_SMEM, attr_set, "fused adjoint kernel");
  if (s) return s;
  k_tc_adjdw<<<grid, FZ_NT, FZ_SMEM, st>>>(mw, mz, ma, p);
  return launch_check(h, "fused adjoint");
}

namespace {

pinn_status launch_adjdw_group(pinn_handle* h, const TcGroupEntry* d_tab, int n, int blocks, cudaStream_t st) {
  static bool attr_set = false;
  pinn_status s = reserve_smem(h, k_tc_adjdw_group, FZ_SMEM, attr_set, "grouped fused adjoint kernel");
  if (s) return s;
  k_tc_adjdw_group<<<blocks, FZ_NT, FZ_SMEM, st>>>(d_tab, n);
  return launch_check(h, "grouped fused adjoint");
}

}  // namespace

TcBatch* tc_batch_create() { return new (std::nothrow) TcBatch(); }

void tc_batch_destroy(TcBatch* b) {
  if (!b) return;
  if (b->d_table) cudaFree(b->d_table);
  delete b;
}

void tc_batch_attach(pinn_handle* h, TcBatch* b) { h->tc_batch = b; }

void tc_batch_reset(TcBatch* b) {
  b->pending.clear();
  b->table.clear();
  b->launches = 0;
}

pinn_status tc_batch_reserve(TcBatch* b, size_t entries) {
  if (entries <= b->capacity) return PINN_OK;
  if (b->d_table) cudaFree(b->d_table);
  b->d_table = nullptr;
  b->capacity = 0;
  if (cudaMalloc(&b->d_table, entries * sizeof(TcGroupEntry)) != cudaSuccess) {
    cudaGetLastError();
    return PINN_ERR_CUDA;
  }
  b->capacity = entries;
  return PINN_OK;
}

pinn_status tc_batch_flush(TcBatch* b, pinn_handle* h, cudaStream_t st) {
  // one grouped launch per kernel variant, in the order the variants first appeared
  std::vector<TcBatch::GroupFn> fns;
  for (const TcBatch::Item& it : b->pending)
    if (std::find(fns.begin(), fns.end(), it.fn) == fns.end()) fns.push_back(it.fn);
  pinn_status s = PINN_OK;
  for (TcBatch::GroupFn fn : fns) {
    std::vector<const TcBatch::Item*> items;
    for (const TcBatch::Item& it : b->pending)
      if (it.fn == fn) items.push_back(&it);
    // the GEMMs with the most work first, so that the small ones fill the tail
    std::stable_sort(items.begin(), items.end(),
                     [](const TcBatch::Item* x, const TcBatch::Item* y) { return x->work > y->work; });
    const size_t off = b->table.size();
    if (off + items.size() > b->capacity) {
      snprintf(h->err, sizeof(h->err), "grouped launch table full (%zu entries)", b->capacity);
      s = PINN_ERR_INVALID_ARG;
      break;
    }
    int blocks = 0;
    for (const TcBatch::Item* it : items) {
      TcGroupEntry e = it->e;
      e.block0 = blocks;
      blocks += e.grid;
      b->table.push_back(e);
    }
    s = fn(h, b->d_table + off, (int)items.size(), blocks, st);
    if (s) break;
    ++b->launches;
  }
  b->pending.clear();
  return s;
}

pinn_status tc_batch_upload(TcBatch* b) {
  if (b->table.empty()) return PINN_OK;
  if (cudaMemcpy(b->d_table, b->table.data(), b->table.size() * sizeof(TcGroupEntry), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    cudaGetLastError();
    return PINN_ERR_CUDA;
  }
  return PINN_OK;
}

int tc_batch_launches(const TcBatch* b) { return b->launches; }

}  // namespace pinn

// Raw tensor-core GEMM of the library's two operand layouts, FP32 output, for
// testing the MMA core in isolation (no epilogue).
namespace {
template <bool TF32>
pinn_status selftest_impl(pinn_handle* h, int layout, int M, int N, int K, const void* d_A, const void* d_A2,
                          const void* d_B, float* d_D, int* status, cudaStream_t st, uint64_t wait_ns = 0,
                          int stall = 0) {
  using namespace pinn;
  CUtensorMap ma, ma2, mb;
  if (layout == 0) {
    // D = A B: A [M][K] row-major, B [K][N] and D [M][N] in the tile-major jet layout
    using C = Cfg<TF32, TC_STORE, false>;
    if (!make_map(&ma, d_A, TF32, K, M, C::BKE, BM) || !make_map(&ma2, d_A2 ? d_A2 : d_A, TF32, K, M, C::BKE, BM) ||
        !make_map3(&mb, d_B, TF32, TILE_COLS, K, N / TILE_COLS, C::BOXN, C::BKE))
      return PINN_ERR_CUDA;
    TcParams p = base_params(M, N, K, N, C::BKE, status);
    p.out32 = d_D;
    if (wait_ns) p.wait_ns = wait_ns;
    p.stall = stall;
    const int grid = grid_for(h, p.m_tiles * p.n_tiles);
    if (d_A2) return launch<TF32, TC_STORE, true>(h, ma, ma2, mb, mb, p, grid, st);
    return launch<TF32, TC_STORE, false>(h, ma, ma, mb, mb, p, grid, st);
  }
  // D = A B^T: A [M][K] and B [N][K] in the tile-major layout (K over jet columns), D [M][N]
  using C = Cfg<TF32, TC_DW, false>;
  if (!make_map3(&ma, d_A, TF32, TILE_COLS, M, K / TILE_COLS, C::BKE, BM) ||
      !make_map3(&mb, d_B, TF32, TILE_COLS, N, K / TILE_COLS, C::BKE, BN))
    return PINN_ERR_CUDA;
  TcParams p = base_params(M, N, K, N, C::BKE, status);
  p.out32 = d_D;
  return launch<TF32, TC_DW, false>(h, ma, ma, mb, mb, p, grid_for(h, p.m_tiles * p.n_tiles), st);
}
}  // namespace

extern "C" PINN_API pinn_status pinn_tc_selftest(int kind, int M, int N, int K, const void* d_A, const void* d_A2,
                                                 const void* d_B, float* d_D, void* stream) {
  using namespace pinn;
  if (!d_A || !d_B || !d_D || M < 1 || N < 1 || K < 1 || kind < 0 || kind > 3) return PINN_ERR_INVALID_ARG;
  const int layout = kind & 1;
  const bool tf32 = (kind & 2) != 0;
  if (tf32 && layout == 0) return PINN_ERR_UNSUPPORTED;   // kind::tf32 takes K-major operands only
  if (K % 8 || M % 8 || N % 8) return PINN_ERR_INVALID_ARG;
  if (layout == 0 && N % TILE_COLS) return PINN_ERR_INVALID_ARG;
  if (layout == 1 && K % TILE_COLS) return PINN_ERR_INVALID_ARG;
  pinn_handle h;
  tc_init(&h);
  if (!g_encode) return PINN_ERR_UNSUPPORTED;
  if (cudaGetDevice(&h.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h.sm_count, cudaDevAttrMultiProcessorCount, h.device) != cudaSuccess)
    return PINN_ERR_CUDA;
  int* status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return PINN_ERR_CUDA;
  cudaMemsetAsync(status, 0, sizeof(int), (cudaStream_t)stream);
  pinn_status r = tf32 ? selftest_impl<true>(&h, layout, M, N, K, d_A, d_A2, d_B, d_D, status, (cudaStream_t)stream)
                       : selftest_impl<false>(&h, layout, M, N, K, d_A, d_A2, d_B, d_D, status, (cudaStream_t)stream);
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

extern "C" PINN_API pinn_status pinn_debug_wait_expiry(pinn_handle* h, int M, int N, int K, const void* d_A,
                                                       const void* d_B, float* d_D, int64_t wait_us, void* stream) {
  using namespace pinn;
  if (!h || !d_A || !d_B || !d_D || M < 1 || N < 1 || K < 1 || wait_us < 1 || wait_us > 2000000)
    return PINN_ERR_INVALID_ARG;
  if (K % 8 || M % 8 || N % TILE_COLS) return PINN_ERR_INVALID_ARG;
  if (!g_encode) return PINN_ERR_UNSUPPORTED;
  // the kind-0 BF16 GEMM with its MMA issuer waiting first on a barrier that nothing
  // arrives on: the wait expires after wait_us, and the kernel latches the timeout in
  // the handle's status word and returns through its abort path
  return selftest_impl<false>(h, 0, M, N, K, d_A, nullptr, d_B, d_D, h->d_status, (cudaStream_t)stream,
                              (uint64_t)wait_us * 1000ull, 1);
}
