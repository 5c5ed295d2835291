// Tensor-core GEMM for sm_103a: tcgen05.mma with TMEM accumulators, operands
// staged by TMA (cp.async.bulk.tensor) into 128-byte-swizzled shared memory.
//
//   C[b][m][n] = alpha * sum_k A[b][m][k] * B[b][n][k] (+ beta * C)
//   (or stored transposed, C[b][n][m], when the caller asks for it)
//
// Both operands are K-major ("TN"), which is the layout every contraction of
// the FT-CCSD S kernel is packed into.  Persistent CTAs (one per SM) walk
// 128 x BN output tiles (BN = 32, 64, 128 or 256, the narrowest covering N):
//   warp 0 / lane 0   TMA producer (multi-stage ring of shared-memory stages)
//   warp 1            TMEM allocation (2 x BN columns), MMA issuer (one thread,
//                     tcgen05.mma kind::tf32 or kind::f16)
//   warps 2-9         epilogue: tcgen05.ld 32 lanes x 32 columns, scale, store
//                     through a shared-memory transpose, overlapping the next
//                     tile's main loop (double-buffered accumulator)
// BF16X3 keeps a two-way bf16 split of each operand (x = hi + lo) and issues
// hi*hi + hi*lo + lo*hi into the same FP32 accumulator.
//
// Every mbarrier wait is bounded (about two seconds of clock64); on expiry the
// thread records an error code in *err and leaves its loop, so the block
// always reaches the TMEM release and exits.
#include <atomic>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "ftcc_internal.h"

namespace ftcc {
namespace {

constexpr int kBM = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false (and flags *err) after
// ~2^32 cycles, or at once if another thread already flagged an error.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023u) == 0) {
      if (*reinterpret_cast<volatile int*>(err) != 0) return false;
      if (clock64() - t0 > (1LL << 32)) {
        atomicCAS(err, 0, code);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(1) << 16) |
         (static_cast<uint64_t>(1024 >> 4) << 32) | (static_cast<uint64_t>(1) << 46) |
         (static_cast<uint64_t>(2) << 61);
}


__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Output block of the epilogue: 32 rows x 32 FP32 columns from shared memory
// (128-byte swizzle) to C[c2][c1][c0..c0+31] through the TMA unit; rows and
// columns beyond the tensor's extent are not written.  `add` makes it a
// reduce-add into C (C += block) performed in L2.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                             bool add) {
  if (add)
    asm volatile(
        "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
  else
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// the TMA unit has finished reading this thread's earlier bulk-store sources
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... and finished writing them
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the TMA unit
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Instruction descriptor for an M = 128 x N = bn tile.
__host__ __device__ constexpr uint32_t instr_desc_n(uint32_t fmt, uint32_t bn) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((bn >> 3) << 17) | ((uint32_t(kBM) >> 4) << 24);
}

constexpr int kEpiWarps = 8;   // two epilogue warps per TMEM lane quadrant, one per column half
constexpr int kGemmThreads = 32 * (2 + kEpiWarps);

template <int KIND, int BN>
struct TcCfg {
  static constexpr int kOps = KIND == GEMM_TF32 ? 1 : 2;                       // hi (and lo) halves
  static constexpr int kABytes = 128 * 128;                                     // 128 rows x 128 B
  static constexpr int kBBytes = BN * 128;                                      // BN rows x 128 B
  static constexpr int kStageBytes = kOps * (kABytes + kBBytes);
  static constexpr int kStages = (192 * 1024) / kStageBytes > 6 ? 6 : (192 * 1024) / kStageBytes;
  static constexpr int kKElems = KIND == GEMM_TF32 ? 32 : 64;                  // elements per 128-byte row
  static constexpr uint32_t kTmemCols = 2 * BN;                                // double-buffered accumulator
  static constexpr int kEpiBytes = kEpiWarps * 32 * 33 * 4;                   // epilogue staging
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256 + kEpiBytes;
};

constexpr int kGroupM = 8;   // tile raster: groups of 8 row tiles swept across all column tiles

// Persistent warp-specialised GEMM.  CTA = 10 warps:
//   warp 0        TMA producer over a ring of kStages shared-memory stages
//   warp 1        TMEM owner and MMA issuer (one thread), two accumulators
//   warps 2..9    epilogue; warp w drains TMEM lanes 32 (w % 4) .. + 31 of
//                 column half (w - 2) / 4 of the tile (all columns when BN = 32)
// Tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...; the accumulator of tile
// i is buffer i % 2, so tile i's epilogue overlaps tile i+1's main loop.
template <int KIND, int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                   const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB2,
                   float* __restrict__ C, int M, int N, int K, long long ldc, long long sc, int a_batched,
                   int b_batched, float alpha, float beta, int batch, int splits, int kc, float* __restrict__ W,
                   int trans, const __grid_constant__ CUtensorMap mC, int cmode, int* err) {
  using Cfg = TcCfg<KIND, BN>;
  constexpr int S = Cfg::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * Cfg::kStageBytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  float* epi = reinterpret_cast<float*>(smem + S * Cfg::kStageBytes + 256);   // 8 x 32 x 33 staging
  // bulk-store staging (same region, 1024-byte aligned): 8 blocks of 32 x 128 bytes
  float4* bulk = reinterpret_cast<float4*>(smem + S * Cfg::kStageBytes + 1024);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int mt = (M + kBM - 1) / kBM;
  const int nt = (N + BN - 1) / BN;
  const long long per_batch = static_cast<long long>(mt) * nt;
  const long long per_split = per_batch * batch;
  const long long tiles = per_split * splits;   // split-K: each split sums kc K steps into W
  const int nk = (K + Cfg::kKElems - 1) / Cfg::kKElems;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], kEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(Cfg::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  // tile t -> (split, batch, row tile, column tile) with grouped rasterisation
  auto decode = [&](long long t, int& sp, int& b, int& m0, int& n0) {
    sp = static_cast<int>(t / per_split);
    t -= static_cast<long long>(sp) * per_split;
    b = static_cast<int>(t / per_batch);
    const long long r = t - static_cast<long long>(b) * per_batch;
    const long long group = r / (static_cast<long long>(kGroupM) * nt);
    const int first = static_cast<int>(group * kGroupM);
    const int gsize = min(kGroupM, mt - first);
    const long long in = r - group * kGroupM * nt;
    m0 = (first + static_cast<int>(in % gsize)) * kBM;
    n0 = static_cast<int>(in / gsize) * BN;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      uint32_t it = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        int sp, b, m0, n0;
        decode(t, sp, b, m0, n0);
        const int ca = a_batched ? b : 0, cb = b_batched ? b : 0;
        const int kt0 = sp * kc, kt1 = min(nk, kt0 + kc);
        for (int kt = kt0; kt < kt1; ++kt, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          if (it >= static_cast<uint32_t>(S) && !mbar_wait(&empty[s], ph ^ 1u, err, DEVERR_TMA_TIMEOUT)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], Cfg::kStageBytes);
          uint8_t* st = smem + s * Cfg::kStageBytes;
          const int kc = kt * Cfg::kKElems;
          tma_load_3d(st, &mA, &full[s], kc, m0, ca);
          tma_load_3d(st + Cfg::kABytes, &mB, &full[s], kc, n0, cb);
          if (KIND == GEMM_BF16X3) {
            tma_load_3d(st + Cfg::kABytes + Cfg::kBBytes, &mA2, &full[s], kc, m0, ca);
            tma_load_3d(st + 2 * Cfg::kABytes + Cfg::kBBytes, &mB2, &full[s], kc, n0, cb);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      constexpr uint32_t idesc = instr_desc_n(KIND == GEMM_TF32 ? 2u : 1u, BN);
      uint32_t it = 0, local = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++local) {
        const uint32_t acc = local & 1u, use = local >> 1;
        if (local >= 2 && !mbar_wait(&tempty[acc], (use - 1) & 1u, err, DEVERR_MMA_TIMEOUT)) break;
        fence_after_sync();
        const uint32_t d = tmem + acc * BN;
        int sp, b, m0, n0;
        decode(t, sp, b, m0, n0);
        const int kt0 = sp * kc, kt1 = min(nk, kt0 + kc);
        for (int kt = kt0; kt < kt1; ++kt, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          if (!mbar_wait(&full[s], ph, err, DEVERR_MMA_TIMEOUT)) {
            ok = false;
            break;
          }
          fence_after_sync();
          const uint32_t a0 = smem_u32(smem + s * Cfg::kStageBytes);
          const uint32_t b0 = a0 + Cfg::kABytes;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {   // four 32-byte K slices per 128-byte row
            const uint64_t da = smem_desc(a0 + kk * 32);
            const uint64_t db = smem_desc(b0 + kk * 32);
            const uint32_t accum = (kt > kt0 || kk > 0) ? 1u : 0u;
            if (KIND == GEMM_TF32) {
              mma_tf32(d, da, db, idesc, accum);
            } else {
              const uint64_t da2 = smem_desc(b0 + Cfg::kBBytes + kk * 32);
              const uint64_t db2 = smem_desc(b0 + Cfg::kBBytes + Cfg::kABytes + kk * 32);
              mma_f16(d, da, db, idesc, accum);   // hi * hi
              mma_f16(d, da, db2, idesc, 1u);     // hi * lo
              mma_f16(d, da2, db, idesc, 1u);     // lo * hi
            }
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&tfull[acc]);
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31
    const int q = warp & 3;                                  // TMEM lane quadrant of this warp
    const int half = (warp - 2) >> 2;                        // column half of the tile
    constexpr int kHalf = BN >= 64 ? BN / 2 : BN;            // columns per epilogue warp
    const int c_lo = BN >= 64 ? half * kHalf : 0;
    const bool idle = BN < 64 && half == 1;                  // narrow tiles: one warp per quadrant
    uint32_t local = 0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++local) {
      const uint32_t acc = local & 1u, use = local >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[acc], use & 1u, err, DEVERR_EPI_TIMEOUT));
      if (!ok) break;
      fence_after_sync();
      int sp, b, m0, n0;
      decode(t, sp, b, m0, n0);
      const bool part = splits > 1;   // split-K partial: dense [split][batch][M][N] in W, no beta
      float* cbase = part ? W + (static_cast<long long>(sp) * batch + b) * M * static_cast<long long>(N)
                          : C + static_cast<long long>(b) * sc;
      const long long ldo = part ? N : ldc;
      const float bta = part ? 0.0f : beta;
      float* stg = epi + (warp - 2) * (32 * 33);   // this warp's 32 x 32 staging block, row stride 33
      if (idle) {
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
        continue;
      }
#pragma unroll 1
      for (int c = c_lo; c < c_lo + kHalf; c += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + acc * BN + static_cast<uint32_t>(c), r);
        if (c + 32 >= c_lo + kHalf) {   // this warp's part drained: the MMA warp may reuse it
          fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[acc]);
        }
        if (n0 + c >= N) continue;
        if (cmode != 0) {
          // cmode 1: C = alpha AB; cmode 2: C += alpha AB.  Thread = row: its
          // 32 columns go to one 128-byte row of the block, 16-byte chunk j
          // at position j ^ (row % 8) (the TMA 128-byte swizzle), so the
          // eight threads of each quarter-warp store hit distinct banks.
          const int row0 = m0 + q * 32;
          if (row0 >= M) continue;
          float4* blk = bulk + (warp - 2) * (32 * 8);
          if (lane == 0) bulk_wait_read();   // the previous block has left this buffer
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 8; ++j)
            blk[lane * 8 + (j ^ (lane & 7))] =
                make_float4(alpha * __uint_as_float(r[4 * j]), alpha * __uint_as_float(r[4 * j + 1]),
                            alpha * __uint_as_float(r[4 * j + 2]), alpha * __uint_as_float(r[4 * j + 3]));
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) tma_store_3d(&mC, blk, n0 + c, row0, b, cmode == 2);
          continue;
        }
        if (trans && !part) {
          // C stored transposed: lanes are rows m, contiguous in memory
          const int row = m0 + q * 32 + lane;
          float* pc = cbase + row;
          const int ncol = min(32, N - (n0 + c));
          if (row < M) {
            if (bta == 0.0f) {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < ncol) pc[static_cast<long long>(n0 + c + j) * ldc] = alpha * __uint_as_float(r[j]);
            } else {
              float old[32];
#pragma unroll
              for (int j = 0; j < 32; ++j) old[j] = j < ncol ? pc[static_cast<long long>(n0 + c + j) * ldc] : 0.0f;
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < ncol) pc[static_cast<long long>(n0 + c + j) * ldc] = alpha * __uint_as_float(r[j]) + bta * old[j];
            }
          }
          continue;
        }
        // transpose through shared memory: thread = row while staging,
        // lane = column while storing, so every store (and the beta load) is
        // one contiguous 128-byte row segment
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int col = n0 + c + lane;
        const int nrow = min(32, M - (m0 + q * 32));
        float* p0 = cbase + static_cast<long long>(m0 + q * 32) * ldo + col;
        if (col < N) {
          if (bta == 0.0f) {
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr)
              if (rr < nrow) p0[rr * ldo] = alpha * stg[rr * 33 + lane];
          } else {
            // all 32 loads of the old values in flight before the first store
            float old[32];
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) old[rr] = rr < nrow ? p0[rr * ldo] : 0.0f;
#pragma unroll
            for (int rr = 0; rr < 32; ++rr)
              if (rr < nrow) p0[rr * ldo] = alpha * stg[rr * 33 + lane] + bta * old[rr];
          }
        }
        __syncwarp();
      }
    }
    if (cmode != 0 && lane == 0) bulk_wait_all();   // every bulk store of this warp has landed
    __syncwarp();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kTmemCols) : "memory");
  }
}

// C[b][m][n] = sum_s W[s][b][m][n] (+ beta C): the split-K reduction, fixed order.
__global__ void tc_splitk_reduce(const float* __restrict__ W, float* __restrict__ C, long long ldc, long long sc, int M,
                                 int N, int batch, int splits, float beta, int trans) {
  const long long mn = static_cast<long long>(M) * N;
  const long long total = mn * batch;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long b = e / mn;
    const long long r = e - b * mn;
    const long long m = r / N, n = r - m * N;
    float acc = 0.0f;
    for (int s = 0; s < splits; ++s) acc += W[static_cast<long long>(s) * total + e];
    float* c = C + b * sc + (trans ? n * ldc + m : m * ldc + n);
    *c = (beta == 0.0f) ? acc : acc + beta * *c;
  }
}

std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};

bool get_encode() {
  if (g_encode.load()) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr)
    return false;
  g_encode.store(reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn));   // (idempotent under a race)
  return true;
}

// 3D tiled map over [batch][rows][K] (K innermost), 128-byte swizzle, box of
// 128 bytes x 128 rows x 1.  Out-of-range elements load as zero.
bool make_map(CUtensorMap* m, const void* base, bool bf16, long long K, long long rows, long long ld,
              long long bstride, int batch, int box_rows) {
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(bstride > 0 ? batch : 1)};
  const long long bs = bstride > 0 ? bstride : rows * ld;
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld * es), static_cast<cuuint64_t>(bs * es)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(128 / es), static_cast<cuuint32_t>(box_rows), 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = g_encode.load()(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                        const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3D tiled map over C [batch][M][N] (N innermost, row stride ldc, batch stride
// sc), box of 32 columns x 32 rows x 1, 128-byte swizzle: the epilogue's bulk
// stores.  False when the layout breaks a TMA rule (16-byte aligned base and
// strides); the epilogue then stores element by element.
bool make_cmap(CUtensorMap* m, void* C, int M, int N, long long ldc, long long sc, int batch) {
  if (reinterpret_cast<uintptr_t>(C) % 16 != 0 || ldc % 4 != 0 || ldc < N) return false;
  if (batch > 1 && (sc % 4 != 0 || sc < static_cast<long long>(M) * ldc)) return false;
  const long long bs = batch > 1 ? sc : static_cast<long long>(M) * ldc;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(M), static_cast<cuuint64_t>(batch)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ldc * 4), static_cast<cuuint64_t>(((bs * 4 + 15) / 16) * 16)};
  cuuint32_t box[3] = {32u, 32u, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  return g_encode.load()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIND, int BN>
cudaError_t launch_tc(const GemmArgs& g, int* dev_err, cudaStream_t st) {
  const bool bf = (KIND == GEMM_BF16X3);
  CUtensorMap mA, mB, mA2, mB2;
  if (!make_map(&mA, g.A, bf, g.K, g.M, g.lda, g.sa, g.batch, kBM)) return cudaErrorInvalidValue;
  if (!make_map(&mB, g.B, bf, g.K, g.N, g.ldb, g.sb, g.batch, BN)) return cudaErrorInvalidValue;
  if (bf) {
    if (!make_map(&mA2, g.A2, bf, g.K, g.M, g.lda, g.sa, g.batch, kBM)) return cudaErrorInvalidValue;
    if (!make_map(&mB2, g.B2, bf, g.K, g.N, g.ldb, g.sb, g.batch, BN)) return cudaErrorInvalidValue;
  } else {
    mA2 = mA;
    mB2 = mB;
  }
  constexpr int smem = TcCfg<KIND, BN>::kSmem;
  // (set once per instantiation; host threads driving distinct contexts may
  // race here, and both the attribute call and the SM count are idempotent)
  static std::atomic<bool> attr_set{false};
  if (!attr_set.load()) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<KIND, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set.store(true);
  }
  static std::atomic<int> sms_cached{0};
  int sms = sms_cached.load();
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
    sms_cached.store(sms);
  }
  const long long tiles = static_cast<long long>((g.M + kBM - 1) / kBM) * ((g.N + BN - 1) / BN) * g.batch;
  const int nk = (g.K + TcCfg<KIND, BN>::kKElems - 1) / TcCfg<KIND, BN>::kKElems;
  // split K when the output tiles cannot fill half the SMs and the K loop is long
  int splits = 1;
  const long long outer = static_cast<long long>(g.M) * g.N * g.batch;
  if (g.split > 0) {
    splits = std::min(g.split, std::max(1, nk));   // a tuned choice
  } else if (g.work && tiles * 2 < sms && nk >= 8) {
    splits = static_cast<int>(std::min<long long>((sms + tiles - 1) / tiles, nk / 4));
    splits = std::min(splits, 32);
  }
  if (!g.work) splits = 1;
  while (splits > 1 && static_cast<size_t>(splits) * outer * sizeof(float) > g.work_bytes) --splits;
  const int kc = (nk + splits - 1) / splits;
  splits = (nk + kc - 1) / kc;
  const int grid = static_cast<int>(std::min<long long>(tiles * splits, sms));
  // bulk (TMA) output stores for row-major outputs written in one pass with
  // beta 0 (store) or 1 (reduce-add)
  CUtensorMap mC = mA;
  int cmode = 0;
  if (splits == 1 && !g.trans && (g.beta == 0.0 || g.beta == 1.0) &&
      make_cmap(&mC, g.C, g.M, g.N, g.ldc, g.sc, g.batch))
    cmode = g.beta == 0.0 ? 1 : 2;
  gemm_tc_kernel<KIND, BN><<<grid, kGemmThreads, smem, st>>>(mA, mB, mA2, mB2, static_cast<float*>(g.C), g.M, g.N, g.K, g.ldc,
                                                    g.sc, g.sa > 0 ? 1 : 0, g.sb > 0 ? 1 : 0,
                                                    static_cast<float>(g.alpha), static_cast<float>(g.beta), g.batch,
                                                    splits, kc, static_cast<float*>(g.work), g.trans, mC, cmode, dev_err);
  if (splits > 1) {
    const int blocks = static_cast<int>(std::min<long long>((outer + 255) / 256, 152LL * 8));
    tc_splitk_reduce<<<blocks, 256, 0, st>>>(static_cast<const float*>(g.work), static_cast<float*>(g.C), g.ldc, g.sc,
                                             g.M, g.N, g.batch, splits, static_cast<float>(g.beta), g.trans);
  }
  return cudaGetLastError();
}

}  // namespace

bool tma_available() { return get_encode(); }

cudaError_t gemm_tc(int kind, const GemmArgs& g, int* dev_err, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.K <= 0) return cudaErrorInvalidValue;
  if (!get_encode()) return cudaErrorNotSupported;
  if (g.batch > 65535) return cudaErrorInvalidValue;
  // tile width: the narrowest of 32 / 64 / 128 / 256 columns that covers N (tcgen05 with
  // M = 128 takes N in steps of 16 up to 256)
  const int bn = g.bn ? g.bn : (g.N <= 32 ? 32 : (g.N <= 64 ? 64 : (g.N <= 128 ? 128 : 256)));
  if (bn != 32 && bn != 64 && bn != 128 && bn != 256) return cudaErrorInvalidValue;
  if (kind == GEMM_TF32) {
    switch (bn) {
      case 32: return launch_tc<GEMM_TF32, 32>(g, dev_err, st);
      case 64: return launch_tc<GEMM_TF32, 64>(g, dev_err, st);
      case 128: return launch_tc<GEMM_TF32, 128>(g, dev_err, st);
      default: return launch_tc<GEMM_TF32, 256>(g, dev_err, st);
    }
  }
  if (kind == GEMM_BF16X3) {
    switch (bn) {
      case 32: return launch_tc<GEMM_BF16X3, 32>(g, dev_err, st);
      case 64: return launch_tc<GEMM_BF16X3, 64>(g, dev_err, st);
      case 128: return launch_tc<GEMM_BF16X3, 128>(g, dev_err, st);
      default: return launch_tc<GEMM_BF16X3, 256>(g, dev_err, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace ftcc
