// Trailing update of the FP32 fronts on the 5th-generation tensor cores.
//
// C[t0:f, t0:f] -= L21 U12 with K = the panel width (<= 64), one 128 x 128
// output tile per CTA.  FP32 accuracy is kept with the three-term TF32 split:
// every operand x = x_hi + x_lo with x_hi = x rounded to TF32 and
// x_lo = x - x_hi rounded to TF32, and D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// is accumulated in FP32 in tensor memory by tcgen05.mma (kind::tf32).  The
// dropped A_lo B_lo term and the rounding of x_lo are at FP32 rounding level.
//
// Operands are staged by the CTA's threads into shared memory in the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// K-adjacent cores 128 bytes apart (leading byte offset), 8-row groups
// (K/4) * 128 bytes apart (stride byte offset).  One thread issues the MMAs
// and commits them to an mbarrier; the eight warps then read the accumulator
// with tcgen05.ld (warp w: lanes of quadrant w % 4, columns of half w / 4)
// and subtract it from C (coalesced: one lane per row).  mbarrier waits are
// bounded: on timeout the kernel raises an error flag, releases its tensor
// memory and returns.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "kernels.h"

namespace h2sp {
namespace {

constexpr int kTcM = 128, kTcN = 128, kTcK = 64;
constexpr int kTcThreads = 256;
constexpr uint32_t kTcCols = 256;                          // two 128-column FP32 accumulators
constexpr int kTileFloats = kTcM * kTcK;                   // 8192 floats = 32 KB per operand tile
constexpr uint32_t kLbo = 128;                             // K-adjacent core matrices
constexpr uint32_t kSbo = (kTcK / 4) * 128;                // 8-row groups (2048 bytes)
constexpr uint32_t kWaitCap = 1u << 24;                    // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((kLbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((kSbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}

// kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kTcN >> 3) << 17) |
                            (uint32_t(kTcM >> 4) << 24);

// v = hi + lo with hi = v rounded to nearest TF32 and lo = v - hi (exact in
// FP32, |lo| <= 2^-12 |v|), itself rounded to TF32 (error <= 2^-24 |v|).
__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ void split_tf32(float v, float &hi, float &lo) {
  hi = __uint_as_float(to_tf32(v));
  lo = __uint_as_float(to_tf32(v - hi));
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ bool wait_phase(uint32_t mbar_addr, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitCap; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(done)
        : "r"(mbar_addr), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void sync_for_tensor_cores() {
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
}

// One CTA: a 128-row tile of the trailing block against a range of 128-column
// tiles.  The A tile (hi / lo) stays in shared memory; B tiles and the two
// TMEM accumulators alternate, so staging tile i + 1 and the epilogue of tile
// i overlap the asynchronous MMAs.
// With kb > 0 (an inner step of the blocked LU) only the columns left in the
// step's kb-wide outer block, [t0, min(J + kb, s)) with J = kb floor(j0 / kb),
// are updated; the columns after the block wait for the block's rank-kb update.
// With sym (block Cholesky) the B operand is L21^T: column n of the tile is
// row t0 + n of the panel columns, staged like the A tile.
__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_tc(const FrontDev *__restrict__ fr, int j0,
                                                          float *__restrict__ fronts, int *__restrict__ err,
                                                          int splits, int tile_lo, int tile_hi, int partial_only,
                                                          int kb, int sym) {
  const FrontDev F = fr[blockIdx.z];
  if (j0 >= F.s) return;
  const int jb = min(kTcK, F.s - j0);
  if (partial_only && jb == kTcK) return;  // full panels are done by k_gemm_tc_tma
  const int t0 = j0 + jb;
  const int nrest = F.f - t0;
  const int ncols = kb > 0 ? min(nrest, min((j0 / kb) * kb + kb, F.s) - t0) : nrest;
  const int rb = blockIdx.y * kTcM;
  if (rb >= nrest || ncols <= 0) return;
  // this launch covers column tiles [tile_lo, tile_hi) of the trailing block
  const int ntiles = min((ncols + kTcN - 1) / kTcN, tile_hi) - tile_lo;
  if (ntiles <= 0) return;
  const int per = (ntiles + splits - 1) / splits;
  const int c_lo = tile_lo + blockIdx.x * per, c_hi = min(tile_lo + ntiles, c_lo + per);
  if (c_lo >= c_hi) return;
  float *A = fronts + F.off;
  const int64_t ld = F.ld;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char *sAh = smraw, *sAl = smraw + 4 * kTileFloats;
  unsigned char *sBh[2] = {smraw + 8 * kTileFloats, smraw + 16 * kTileFloats};
  unsigned char *sBl[2] = {smraw + 12 * kTileFloats, smraw + 20 * kTileFloats};
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ksteps = (jb + 7) / 8;

  // Element e of a tile in the canonical layout sits at word e when
  // row = (e >> 9) * 8 + ((e & 31) >> 2) and k = ((e >> 5) & 15) * 4 + (e & 3):
  // stores are linear (conflict-free), a warp loads 4 K-steps x 8 rows.
  constexpr int kIters = kTcM * kTcK / kTcThreads;
  {
    float v[kIters];
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int e = tid + it * kTcThreads;
      const int m = (e >> 9) * 8 + ((e & 31) >> 2), k = ((e >> 5) & 15) * 4 + (e & 3);
      const int r = rb + m;
      v[it] = (k < jb && r < nrest) ? A[(t0 + r) + int64_t(j0 + k) * ld] : 0.f;
    }
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int e = tid + it * kTcThreads;
      float hi, lo;
      split_tf32(v[it], hi, lo);
      reinterpret_cast<float *>(sAh)[e] = hi;
      reinterpret_cast<float *>(sAl)[e] = lo;
    }
  }
  // B (the U12 rows, K contiguous in memory): a warp reads 8 K-values of 4
  // columns (four full 32-byte sectors); the shared stores are at most
  // two-way conflicted.
  auto stage_b = [&](int ct, int buf) {
    const int cb = ct * kTcN;
    float v[kIters];
    if (sym) {
      // same canonical layout as A: element e is (n, k) of the tile, stored at word e
#pragma unroll
      for (int it = 0; it < kIters; ++it) {
        const int e = tid + it * kTcThreads;
        const int n = (e >> 9) * 8 + ((e & 31) >> 2), k = ((e >> 5) & 15) * 4 + (e & 3);
        const int c = cb + n;
        v[it] = (k < jb && c < ncols) ? A[(t0 + c) + int64_t(j0 + k) * ld] : 0.f;
      }
      float *bh = reinterpret_cast<float *>(sBh[buf]), *bl = reinterpret_cast<float *>(sBl[buf]);
#pragma unroll
      for (int it = 0; it < kIters; ++it) {
        const int e = tid + it * kTcThreads;
        float hi, lo;
        split_tf32(v[it], hi, lo);
        bh[e] = hi;
        bl[e] = lo;
      }
      return;
    }
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int e = tid + it * kTcThreads;
      const int ln = e & 31, wv = e >> 5;
      const int k = (ln & 7) + 8 * (wv & 7), n = (ln >> 3) + 4 * (wv >> 3);
      const int c = cb + n;
      v[it] = (k < jb && c < ncols) ? A[(j0 + k) + int64_t(t0 + c) * ld] : 0.f;
    }
    float *bh = reinterpret_cast<float *>(sBh[buf]), *bl = reinterpret_cast<float *>(sBl[buf]);
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int e = tid + it * kTcThreads;
      const int ln = e & 31, wv = e >> 5;
      const int k = (ln & 7) + 8 * (wv & 7), n = (ln >> 3) + 4 * (wv >> 3);
      const int w = (n >> 3) * (kSbo / 4) + (k >> 2) * (kLbo / 4) + (n & 7) * 4 + (k & 3);
      float hi, lo;
      split_tf32(v[it], hi, lo);
      bh[w] = hi;
      bl[w] = lo;
    }
  };
  auto issue = [&](uint32_t tmem, int buf) {
    const uint32_t ah0 = smem_u32(sAh), al0 = smem_u32(sAl), bh0 = smem_u32(sBh[buf]), bl0 = smem_u32(sBl[buf]);
    const uint32_t acc = tmem + uint32_t(buf) * kTcN;
    for (int kk = 0; kk < ksteps; ++kk) {
      const uint32_t koff = uint32_t(kk) * 2 * kLbo;  // 8 TF32 = two K-adjacent cores
      const uint64_t ah = smem_desc(ah0 + koff), al = smem_desc(al0 + koff);
      const uint64_t bh = smem_desc(bh0 + koff), bl = smem_desc(bl0 + koff);
      mma_tf32(acc, ah, bh, kk > 0 ? 1u : 0u);
      mma_tf32(acc, ah, bl, 1u);
      mma_tf32(acc, al, bh, 1u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&mbar[buf])));
  };

  stage_b(c_lo, 0);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  sync_for_tensor_cores();
  const uint32_t tmem = tmem_base;
  if (tid == 0) issue(tmem, 0);
  uint32_t parity[2] = {0u, 0u};
  bool ok = true;
  int pending = -1;  // buffer of a group issued but not yet waited for
  const int q = warp & 3, half = warp >> 2;  // TMEM lane quadrant, column half of the epilogue
  for (int it = 0; c_lo + it < c_hi; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    const int ct = c_lo + it;
    pending = -1;
    if (ct + 1 < c_hi) {
      stage_b(ct + 1, nxt);  // the buffer's previous MMA finished before the last epilogue
      sync_for_tensor_cores();
      if (tid == 0) issue(tmem, nxt);
      pending = nxt;
    }
    // this thread's 64 C values (one row), read while the MMAs run; all loads
    // are issued before any store
    const int row = rb + q * 32 + lane;
    const int cb = ct * kTcN + half * 64;
    float *Crow = A + (t0 + row) + int64_t(t0 + cb) * ld;
    const int ncol = row < nrest ? min(64, ncols - cb) : 0;
    float cv[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) cv[j] = j < ncol ? Crow[int64_t(j) * ld] : 0.f;
    const bool w = wait_phase(smem_u32(&mbar[cur]), parity[cur]);
    parity[cur] ^= 1u;
    ok = __syncthreads_and(w ? 1 : 0) != 0;  // one decision for the whole CTA
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + uint32_t(cur * kTcN + half * 64 + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int j = 0; j < 32; ++j) cv[c0 + j] -= __uint_as_float(v[j]);
    }
#pragma unroll
    for (int j = 0; j < 64; ++j)
      if (j < ncol) Crow[int64_t(j) * ld] = cv[j];
    // accumulator `cur` and B buffer `cur` are free for tile it + 2
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (!ok) {
    if (tid == 0) atomicOr(err, 4);
    // give the group still in flight a bounded chance to finish before TMEM is released
    if (pending >= 0) wait_phase(smem_u32(&mbar[pending]), parity[pending]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// TMA helpers (2D tiles of an FP32 front: x = row, y = column)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
// C += box (FP32 add in L2), same completion as a store
__device__ __forceinline__ void tma_reduce_add_2d(const void *tmap, int x, int y, uint32_t src) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   tmap),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_store_2d(const void *tmap, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tmap), "r"(x),
               "r"(y), "r"(src)
               : "memory");
}

// The update with a full panel (jb = 64): the C tile moves by TMA (one
// 128 x 128 FP32 box in, one out, per column tile) instead of 128 scalar
// accesses per thread, so the load/store queues carry only the B operand.
// Per column tile: the C load is requested first, the threads stage B
// (hi / lo), one thread issues the MMAs, the epilogue subtracts the
// accumulator from the tile in shared memory, and the tile is stored back
// asynchronously while the next one starts.  Shared memory: A hi/lo, B hi/lo
// and the C tile, 192 KB.
__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_tc_tma(const FrontDev *__restrict__ fr, int j0,
                                                              float *__restrict__ fronts, int *__restrict__ err,
                                                              int splits, int tile_lo, int tile_hi,
                                                              const uint8_t *__restrict__ maps) {
  const FrontDev F = fr[blockIdx.z];
  if (j0 >= F.s || F.s - j0 < kTcK) return;  // full panels only
  const int jb = kTcK;
  const int t0 = j0 + jb;
  const int nrest = F.f - t0;
  const int rb = blockIdx.y * kTcM;
  if (rb >= nrest) return;
  const int ntiles = min((nrest + kTcN - 1) / kTcN, tile_hi) - tile_lo;
  if (ntiles <= 0) return;
  const int per = (ntiles + splits - 1) / splits;
  const int c_lo = tile_lo + blockIdx.x * per, c_hi = min(tile_lo + ntiles, c_lo + per);
  if (c_lo >= c_hi) return;
  const void *tmap = maps + size_t(blockIdx.z) * kTmapBytes;
  float *A = fronts + F.off;
  const int64_t ld = F.ld;
  extern __shared__ __align__(1024) unsigned char smraw[];
  float *sAh = reinterpret_cast<float *>(smraw), *sAl = sAh + kTileFloats;
  float *sBh = sAl + kTileFloats, *sBl = sBh + kTileFloats;
  float *sC = sBl + kTileFloats;  // 128 x 128, column-major (TMA box order)
  __shared__ __align__(8) uint64_t bar_mma, bar_c;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kIters = kTcM * kTcK / kTcThreads;
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
    const int e = tid + it * kTcThreads;
    const int m = (e >> 9) * 8 + ((e & 31) >> 2), k = ((e >> 5) & 15) * 4 + (e & 3);
    const int r = rb + m;
    const float v = r < nrest ? A[(t0 + r) + int64_t(j0 + k) * ld] : 0.f;
    float hi, lo;
    split_tf32(v, hi, lo);
    sAh[e] = hi;
    sAl[e] = lo;
  }
  auto stage_b = [&](int ct) {
    const int cb = ct * kTcN;
    float v[kIters];
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int e = tid + it * kTcThreads;
      const int ln = e & 31, wv = e >> 5;
      const int k = (ln & 7) + 8 * (wv & 7), n = (ln >> 3) + 4 * (wv >> 3);
      const int c = cb + n;
      v[it] = c < nrest ? A[(j0 + k) + int64_t(t0 + c) * ld] : 0.f;
    }
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int e = tid + it * kTcThreads;
      const int ln = e & 31, wv = e >> 5;
      const int k = (ln & 7) + 8 * (wv & 7), n = (ln >> 3) + 4 * (wv >> 3);
      const int w = (n >> 3) * (kSbo / 4) + (k >> 2) * (kLbo / 4) + (n & 7) * 4 + (k & 3);
      float hi, lo;
      split_tf32(v[it], hi, lo);
      sBh[w] = hi;
      sBl[w] = lo;
    }
  };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(uint32_t(kTcN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_mma)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_c)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  uint32_t ph_mma = 0u, ph_c = 0u;
  bool ok = true, mma_pending = false, c_pending = false;
  const int q = warp & 3, half = warp >> 2;
  for (int ct = c_lo; ct < c_hi; ++ct) {
    const int x = t0 + rb, y = t0 + ct * kTcN;
    if (tid == 0) {
      // the previous tile's store has read the shared tile
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar_c)),
                   "r"(uint32_t(kTcM * kTcN * 4))
                   : "memory");
      tma_load_2d(smem_u32(sC), tmap, x, y, smem_u32(&bar_c));
    }
    c_pending = true;
    stage_b(ct);  // the previous tile's MMAs completed before its epilogue
    sync_for_tensor_cores();
    if (tid == 0) {
      const uint32_t ah0 = smem_u32(sAh), al0 = smem_u32(sAl), bh0 = smem_u32(sBh), bl0 = smem_u32(sBl);
      for (int kk = 0; kk < kTcK / 8; ++kk) {
        const uint32_t koff = uint32_t(kk) * 2 * kLbo;
        const uint64_t ah = smem_desc(ah0 + koff), al = smem_desc(al0 + koff);
        const uint64_t bh = smem_desc(bh0 + koff), bl = smem_desc(bl0 + koff);
        mma_tf32(tmem, ah, bh, kk > 0 ? 1u : 0u);
        mma_tf32(tmem, ah, bl, 1u);
        mma_tf32(tmem, al, bh, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&bar_mma)));
    }
    mma_pending = true;
    const bool w1 = wait_phase(smem_u32(&bar_mma), ph_mma);
    const bool w2 = wait_phase(smem_u32(&bar_c), ph_c);
    ok = __syncthreads_and((w1 && w2) ? 1 : 0) != 0;
    if (!ok) {
      // a wait gave up: keep track of what may still be in flight
      mma_pending = !w1;
      c_pending = !w2;
      break;
    }
    ph_mma ^= 1u;
    ph_c ^= 1u;
    mma_pending = c_pending = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int row = q * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + uint32_t(half * 64 + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      float *col = sC + (half * 64 + c0) * kTcM + row;
#pragma unroll
      for (int j = 0; j < 32; ++j) col[j * kTcM] -= __uint_as_float(v[j]);
    }
    // the tile goes back asynchronously; TMEM and the B tile are free
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      tma_store_2d(tmap, x, y, smem_u32(sC));
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(err, 4);
    // bounded waits for what may still target this CTA's memory
    if (mma_pending) wait_phase(smem_u32(&bar_mma), ph_mma);
    if (c_pending) wait_phase(smem_u32(&bar_c), ph_c);
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(kTcN)));
}

// ---- packed operands and the warp-specialised block-end update ----
constexpr int kPkK = 16;                          // K values per packed chunk
constexpr int kPkTile = kTcM * kPkK;              // floats per hi (or lo) array: 2048 = 8 KB
constexpr uint32_t kPkSbo = (kPkK / 4) * 128;     // 8-row groups of a packed array (512 bytes)
constexpr int kWsStages = 5;                      // chunks in flight (32 KB each)
constexpr int kWsHalf = 64;                       // columns of one C half-tile moved by TMA
constexpr int kWsCFloats = kTcM * kWsHalf;        // one C half-tile in shared memory: 32 KB
static_assert(kPackTileFloats == int64_t(kPackChunks) * 2 * kPkTile, "packed tile size");

__device__ __forceinline__ uint64_t smem_desc_pk(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((kLbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((kPkSbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Word w of a packed 128 x 16 array holds element (m, k) (m = row of A or
// column of B, k = K index): 8-row x 4-K core matrices of 128 bytes, K-adjacent
// cores 128 bytes apart, 8-row groups 512 bytes apart.
__device__ __forceinline__ void pk_coords(int w, int &m, int &k) {
  m = ((w >> 7) << 3) | ((w >> 2) & 7);
  k = (((w >> 5) & 3) << 2) | (w & 3);
}

// L21 of the outer block [j0, j0 + jb): rows [t0, f), t0 = j0 + jb, one CTA
// per 128-row tile and 16-wide K chunk; zero beyond the front and beyond jb.
constexpr int kPkPer = kPkTile / 256;  // elements per thread of a chunk
__global__ void __launch_bounds__(256) k_pack_a(const FrontDev *__restrict__ fr, int j0, int kb,
                                                const float *__restrict__ fronts, float *__restrict__ pack) {
  const FrontDev F = fr[blockIdx.y];
  if (j0 >= F.s) return;
  const int jb = min(kb, F.s - j0), t0 = j0 + jb, nrest = F.f - t0;
  const int rt = blockIdx.x / kPackChunks, q = blockIdx.x % kPackChunks;
  if (rt * kTcM >= nrest || q * kPkK >= jb) return;
  const float *A = fronts + F.off;
  const int64_t ld = F.ld;
  float *dst = pack + (int64_t(F.pack_off) + rt) * kPackTileFloats + int64_t(2 * q) * kPkTile;
  float v[kPkPer];
#pragma unroll
  for (int it = 0; it < kPkPer; ++it) {
    const int w = threadIdx.x + it * 256;
    int m, k;
    pk_coords(w, m, k);
    const int r = rt * kTcM + m, kk = q * kPkK + k;
    v[it] = (r < nrest && kk < jb) ? A[(t0 + r) + int64_t(j0 + kk) * ld] : 0.f;
  }
#pragma unroll
  for (int it = 0; it < kPkPer; ++it) {
    const int w = threadIdx.x + it * 256;
    float hi, lo;
    split_tf32(v[it], hi, lo);
    dst[w] = hi;
    dst[kPkTile + w] = lo;
  }
}

// U12 (rows [j0, j0 + jb)) of the trailing-block column tiles [ct_lo, ct_hi),
// one CTA per tile and chunk.
__global__ void __launch_bounds__(256) k_pack_b(const FrontDev *__restrict__ fr, int j0, int kb,
                                                const float *__restrict__ fronts, float *__restrict__ pack, int ct_lo,
                                                int ct_hi) {
  const FrontDev F = fr[blockIdx.y];
  if (j0 >= F.s) return;
  const int jb = min(kb, F.s - j0), t0 = j0 + jb, nrest = F.f - t0;
  const int ct = ct_lo + int(blockIdx.x) / kPackChunks, q = blockIdx.x % kPackChunks;
  if (ct >= ct_hi || ct * kTcN >= nrest || q * kPkK >= jb) return;
  const float *A = fronts + F.off;
  const int64_t ld = F.ld;
  float *dst = pack + (int64_t(F.pack_off) + ct) * kPackTileFloats + int64_t(2 * q) * kPkTile;
  float v[kPkPer];
#pragma unroll
  for (int it = 0; it < kPkPer; ++it) {
    const int w = threadIdx.x + it * 256;
    int n, k;
    pk_coords(w, n, k);
    const int c = ct * kTcN + n, kk = q * kPkK + k;
    v[it] = (c < nrest && kk < jb) ? A[(j0 + kk) + int64_t(t0 + c) * ld] : 0.f;
  }
#pragma unroll
  for (int it = 0; it < kPkPer; ++it) {
    const int w = threadIdx.x + it * 256;
    float hi, lo;
    split_tf32(v[it], hi, lo);
    dst[w] = hi;
    dst[kPkTile + w] = lo;
  }
}

// ---- the BF16 block-end operands (block Cholesky, H2SP_BF16_CHOL) ----
// A 128-row tile of L21 (K = the block's columns, <= 256) scaled by 2^-e,
// e = the exponent of the tile's largest |entry| (frexp), and rounded to BF16,
// in the canonical K-major layout of kind::f16: per 64-deep K chunk, 8-row
// groups 1024 bytes apart, K-adjacent 8 x 8 core matrices 128 bytes apart
// (chunk q at byte 16384 q).  The exponent (an int) follows at byte 65536 of
// the tile's slot.  One CTA per tile and front.
constexpr int kBfK = 64;                            // K per chunk
constexpr uint32_t kBfSbo = (kBfK / 8) * 128;       // 8-row groups: 1024 bytes
constexpr int kBfChunkBytes = kTcM * kBfK * 2;      // 16 KB
constexpr int kBfExpFloat = 4 * kBfChunkBytes / 4;  // float index of the exponent (byte 65536)
static_assert(kBfChunkBytes == 2 * kPkTile * 4, "a BF16 chunk has the bytes of a TF32 hi/lo chunk pair");

__device__ __forceinline__ uint64_t smem_desc_bf(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((kLbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((kBfSbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// kind::f16, D = F32, A = B = BF16, both K-major, M = 128, N = 128
constexpr uint32_t kIdescBf = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kTcN >> 3) << 17) |
                              (uint32_t(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kIdescBf), "r"(accumulate));
}

// The exponent e (frexp) of the largest |entry| of rows [r0, r0 + rows) x
// columns [j0, j0 + jb) of a column-major array (0 for an all-zero tile), on
// every thread of a 256-thread CTA; thread 0 also stores it at *out.
__device__ int tile_exponent(const float *__restrict__ A, int64_t ld, int r0, int rows, int j0, int jb, int *out) {
  __shared__ float red[8];
  __shared__ int s_e;
  const int tid = threadIdx.x;
  float mx = 0.f;
  for (int e = tid; e < kTcM * jb; e += 256) {
    const int m = e % kTcM, k = e / kTcM;
    if (m < rows) mx = fmaxf(mx, fabsf(A[(r0 + m) + int64_t(j0 + k) * ld]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t = fmaxf(t, red[i]);
    int ex = 0;
    if (t > 0.f && isfinite(t)) frexpf(t, &ex);
    s_e = ex;
    *out = ex;
  }
  __syncthreads();
  return s_e;
}

__global__ void __launch_bounds__(256) k_pack_bf16(const FrontDev *__restrict__ fr, int j0, int kb,
                                                   const float *__restrict__ fronts, float *__restrict__ pack) {
  const FrontDev F = fr[blockIdx.y];
  if (j0 >= F.s) return;
  const int jb = min(kb, F.s - j0), t0 = j0 + jb, nrest = F.f - t0;
  const int rt = blockIdx.x;
  if (rt * kTcM >= nrest) return;  // uniform over the CTA
  const float *A = fronts + F.off;
  const int64_t ld = F.ld;
  float *slot = pack + (int64_t(F.pack_off) + rt) * kPackTileFloats;
  const int tid = threadIdx.x;
  const int r0 = t0 + rt * kTcM;
  const int s_e = tile_exponent(A, ld, r0, nrest - rt * kTcM, j0, jb, reinterpret_cast<int *>(slot) + kBfExpFloat);
  const float sc = ldexpf(1.f, -s_e);
  // units of 8 consecutive K values of one row: one 16-byte store each
  unsigned char *dst = reinterpret_cast<unsigned char *>(slot);
  const int nunit = kTcM * (kLuOuterBlock / 8);
  for (int u = tid; u < nunit; u += 256) {
    const int m = u % kTcM, kcg = u / kTcM;  // row, global K core (8 values)
    const int q = kcg / (kBfK / 8), kc = kcg % (kBfK / 8);
    const bool row_ok = rt * kTcM + m < nrest;
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      float v[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int k = kcg * 8 + 2 * h + t;
        v[t] = (row_ok && k < jb) ? A[(r0 + m) + int64_t(j0 + k) * ld] * sc : 0.f;
      }
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[0], v[1]);
      w[h] = *reinterpret_cast<const uint32_t *>(&b2);
    }
    const int g = m / 8, r = m % 8;
    const size_t off = size_t(q) * kBfChunkBytes + size_t((g * (kBfK / 8) + kc) * 8 + r) * 16;
    *reinterpret_cast<uint4 *>(dst + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// The two-term split (H2SP_BF16X3_CHOL): with the tile's scale 2^-e as above,
// x 2^-e = hi + lo + O(2^-17 |x 2^-e|), hi = bf16(x 2^-e), lo = bf16(x 2^-e - hi).
// Layout of the TF32 operands: per 32-deep K chunk q a hi and a lo 128 x 32
// array (8 KB each, chunk q at float 4096 q); word w of an array holds the
// BF16 pair of K values 2k, 2k + 1 of element (m, k) = pk_coords(w).  The
// exponent follows the eight chunks at float kBf2ExpFloat.
constexpr int kBf2K = 32;
constexpr int kBf2ExpFloat = (kLuOuterBlock / kBf2K) * 2 * kPkTile;
static_assert(kBf2ExpFloat < kPackTileFloats, "exponent inside the tile slot");

__global__ void __launch_bounds__(256) k_pack_bf16x2(const FrontDev *__restrict__ fr, int j0, int kb,
                                                     const float *__restrict__ fronts, float *__restrict__ pack) {
  const FrontDev F = fr[blockIdx.y];
  if (j0 >= F.s) return;
  const int jb = min(kb, F.s - j0), t0 = j0 + jb, nrest = F.f - t0;
  const int rt = blockIdx.x;
  if (rt * kTcM >= nrest) return;  // uniform over the CTA
  const float *A = fronts + F.off;
  const int64_t ld = F.ld;
  float *slot = pack + (int64_t(F.pack_off) + rt) * kPackTileFloats;
  const int r0 = t0 + rt * kTcM, rows = nrest - rt * kTcM;
  const int ex = tile_exponent(A, ld, r0, rows, j0, jb, reinterpret_cast<int *>(slot) + kBf2ExpFloat);
  const float sc = ldexpf(1.f, -ex);
  uint32_t *dst = reinterpret_cast<uint32_t *>(slot);
  const int nq = (jb + kBf2K - 1) / kBf2K;
  for (int u = threadIdx.x; u < nq * kPkTile; u += 256) {
    const int q = u / kPkTile, w = u % kPkTile;
    int m, kw;
    pk_coords(w, m, kw);
    const int k = q * kBf2K + 2 * kw;
    float v[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) v[t] = (m < rows && k + t < jb) ? A[(r0 + m) + int64_t(j0 + k + t) * ld] * sc : 0.f;
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 l2 =
        __floats2bfloat162_rn(v[0] - __bfloat162float(h2.x), v[1] - __bfloat162float(h2.y));
    dst[q * 2 * kPkTile + w] = *reinterpret_cast<const uint32_t *>(&h2);
    dst[q * 2 * kPkTile + kPkTile + w] = *reinterpret_cast<const uint32_t *>(&l2);
  }
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
// named barrier of the epilogue warps, with an AND over the threads' votes
constexpr int kWsEpiWarps = 16;
__device__ __forceinline__ bool epi_bar_and(bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"(int(v)), "n"(kWsEpiWarps * 32));
  return r != 0;
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kWsEpiWarps * 32) : "memory"); }

constexpr int kWsThreads = (kWsEpiWarps + 2) * 32;  // sixteen epilogue warps, a copy warp and an MMA warp

// Block-end update C[t0:f, t0:f] -= L21 U12 (K = jb <= 256) from packed
// operands.  Warp 16 streams the (A, B) chunk pairs of the CTA's tiles through
// kWsStages shared-memory stages with bulk copies, refilling a stage once the
// MMAs that read it have finished; warp 17 issues the MMAs of each chunk as
// soon as it lands, into one of two TMEM accumulators (alternating by tile).  Warps
// 0-15 prefetch their rows of the next C tile (a row and 32 columns per
// thread) into registers while its MMAs run, then subtract the finished
// accumulator and store (one lane per row: coalesced), and hand the
// accumulator back.  Every wait is bounded; on
// timeout the kernel raises the error flag, waits (bounded) for its copies and
// MMAs in flight, releases TMEM and returns.
// MODE 0: FP32 operands as TF32 hi/lo pairs, three kind::tf32 MMAs per K step;
// MODE 1: BF16 operands (k_pack_bf16), one kind::f16 MMA per K step;
// MODE 2: BF16 hi/lo pairs (k_pack_bf16x2), three kind::f16 MMAs per K step.
template <int MODE>
__global__ void __launch_bounds__(kWsThreads, 1) k_gemm_tc_ws(const FrontDev *__restrict__ fr, int j0, int kb,
                                                             float *__restrict__ fronts, int *__restrict__ err,
                                                             int splits, int tile_lo, int tile_hi,
                                                             const float *__restrict__ apack,
                                                             const float *__restrict__ bpack, int lower,
                                                             const uint8_t *__restrict__ maps64) {
  const FrontDev F = fr[blockIdx.z];
  if (j0 >= F.s) return;
  const int jb = min(kb, F.s - j0);
  const int t0 = j0 + jb;
  const int nrest = F.f - t0;
  const int rb = blockIdx.y * kTcM;
  if (rb >= nrest) return;
  const int ntiles = min((nrest + kTcN - 1) / kTcN, tile_hi) - tile_lo;
  if (ntiles <= 0) return;
  const int per = (ntiles + splits - 1) / splits;
  // lower (block Cholesky): the column tiles up to the diagonal tile only
  const int tile_end = lower ? min(tile_lo + ntiles, int(blockIdx.y) + 1) : tile_lo + ntiles;
  const int c_lo = tile_lo + blockIdx.x * per, c_hi = min(tile_end, c_lo + per);
  if (c_lo >= c_hi) return;
  const int nt = c_hi - c_lo;
  // K chunks: 16 TF32 values (hi and lo arrays), 64 BF16 values or 32 BF16
  // values (hi and lo arrays), 16 KB per operand in each case
  const int nq = MODE == 1 ? (jb + kBfK - 1) / kBfK : MODE == 2 ? (jb + kBf2K - 1) / kBf2K : (jb + kPkK - 1) / kPkK;
  const int G = nt * nq;  // chunk steps of this CTA
  float *A = fronts + F.off;
  const int64_t ld = F.ld;
  extern __shared__ __align__(1024) unsigned char smraw[];
  float *stage0 = reinterpret_cast<float *>(smraw);  // kWsStages x (Ah, Al, Bh, Bl)
  float *sC = stage0 + kWsStages * 4 * kPkTile;      // two C half-tiles (TMA epilogue)
  __shared__ __align__(8) uint64_t full[kWsStages], empty[kWsStages], accf[2], acce[2], cfull[2];
  // The C tiles move by TMA when the tile origin's row t0 + rb sits on a
  // 16-byte boundary (the tensor maps' rule for the innermost coordinate);
  // otherwise the epilogue threads load and store C themselves.
  const bool use_tma = maps64 != nullptr && (t0 & 3) == 0;
  const void *tmap = use_tma ? static_cast<const void *>(maps64 + size_t(blockIdx.z) * kTmapBytes) : nullptr;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(uint32_t(2 * kTcN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < kWsStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(1));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&accf[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&cfull[i])), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const float *Ab = apack + (int64_t(F.pack_off) + blockIdx.y) * kPackTileFloats;
  const float *Bb = bpack + int64_t(F.pack_off) * kPackTileFloats;
  constexpr uint32_t kHalfBytes = 2 * kPkTile * 4;  // a hi and a lo array (or a BF16 chunk): 16 KB
  // BF16 operands carry one power-of-two scale per tile: the product of the
  // row tile's and the column tile's goes back on in the epilogue
  auto tile_scale = [&](int ct) -> float {
    if constexpr (MODE != 0) {
      constexpr int xf = MODE == 1 ? kBfExpFloat : kBf2ExpFloat;
      const int ea = reinterpret_cast<const int *>(Ab)[xf];
      const int eb = reinterpret_cast<const int *>(Bb + int64_t(ct) * kPackTileFloats)[xf];
      return ldexpf(1.f, ea + eb);
    } else {
      (void)ct;
      return 1.f;
    }
  };
  constexpr int kStageFloats = 4 * kPkTile;

  __shared__ volatile int s_consumed;  // chunks whose copies the MMA warp has waited for
  if (tid == 0) s_consumed = 0;
  __syncthreads();
  if (warp == kWsEpiWarps) {
    // ---- copy producer ----
    if (lane == 0) {
      int issued = 0;
      for (int g = 0; g < G; ++g) {
        const int st = g % kWsStages, i = g / nq, q = g % nq;
        if (g >= kWsStages) {
          // the MMAs of chunk g - kWsStages (same stage) have finished
          const bool w = !abort_flag && wait_phase(smem_u32(&empty[st]), uint32_t(((g - kWsStages) / kWsStages) & 1));
          if (!w) {
            abort_flag = 1;
            break;
          }
        }
        const float *a = Ab + int64_t(q) * 2 * kPkTile;
        const float *b = Bb + int64_t(c_lo + i) * kPackTileFloats + int64_t(q) * 2 * kPkTile;
        const uint32_t dst = smem_u32(stage0 + st * kStageFloats);
        const uint32_t mb = smem_u32(&full[st]);
        mbar_expect_tx(mb, 2 * kHalfBytes);
        bulk_copy_g2s(dst, a, kHalfBytes, mb);
        bulk_copy_g2s(dst + kHalfBytes, b, kHalfBytes, mb);
        ++issued;
      }
      if (abort_flag) {
        atomicOr(err, 4);
        // bounded waits for the copies still writing this CTA's shared memory
        for (int g = s_consumed; g < issued; ++g)
          wait_phase(smem_u32(&full[g % kWsStages]), uint32_t((g / kWsStages) & 1));
      }
    }
  } else if (warp == kWsEpiWarps + 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int last_mma = -1;
      bool ok = true;
      for (int g = 0; g < G && ok; ++g) {
        const int st = g % kWsStages, i = g / nq, q = g % nq, a = i & 1;
        if (abort_flag || !wait_phase(smem_u32(&full[st]), uint32_t((g / kWsStages) & 1))) {
          ok = false;
          break;
        }
        s_consumed = g + 1;
        if (q == 0 && i >= 2 && !wait_phase(smem_u32(&acce[a]), uint32_t(((i - 2) >> 1) & 1))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t base = smem_u32(stage0 + st * kStageFloats);
        const uint32_t ah0 = base, al0 = base + kPkTile * 4, bh0 = base + 2 * kPkTile * 4, bl0 = base + 3 * kPkTile * 4;
        const uint32_t acc = tmem + uint32_t(a * kTcN);
        if constexpr (MODE == 2) {
          // the TF32 pairs' layout, K = 16 BF16 values per MMA (32 bytes: the same cores)
#pragma unroll
          for (int kk = 0; kk < kBf2K / 16; ++kk) {
            const uint32_t koff = uint32_t(kk) * 2 * kLbo;
            const uint64_t ah = smem_desc_pk(ah0 + koff), al = smem_desc_pk(al0 + koff);
            const uint64_t bh = smem_desc_pk(bh0 + koff), bl = smem_desc_pk(bl0 + koff);
            mma_bf16(acc, ah, bh, (q > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(acc, ah, bl, 1u);
            mma_bf16(acc, al, bh, 1u);
          }
        } else if constexpr (MODE == 1) {
          // A at the stage's first 16 KB, B at the second; K = 16 per MMA
          const uint32_t b0 = base + uint32_t(kBfChunkBytes);
          (void)al0, (void)bh0, (void)bl0;
#pragma unroll
          for (int kk = 0; kk < kBfK / 16; ++kk) {
            const uint32_t koff = uint32_t(kk) * 2 * kLbo;
            mma_bf16(acc, smem_desc_bf(ah0 + koff), smem_desc_bf(b0 + koff), (q > 0 || kk > 0) ? 1u : 0u);
          }
        } else {
#pragma unroll
          for (int kk = 0; kk < kPkK / 8; ++kk) {
            const uint32_t koff = uint32_t(kk) * 2 * kLbo;
            const uint64_t ah = smem_desc_pk(ah0 + koff), al = smem_desc_pk(al0 + koff);
            const uint64_t bh = smem_desc_pk(bh0 + koff), bl = smem_desc_pk(bl0 + koff);
            mma_tf32(acc, ah, bh, (q > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(acc, ah, bl, 1u);
            mma_tf32(acc, al, bh, 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&empty[st])));
        last_mma = g;
        if (q == nq - 1)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&accf[a])));
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(err, 4);
        if (last_mma >= 0)
          wait_phase(smem_u32(&empty[last_mma % kWsStages]), uint32_t((last_mma / kWsStages) & 1));
      }
    }
  } else if (use_tma) {
    // ---- epilogue warps with TMA: per tile two 128 x 64 halves of C pass
    // through sC[h]; thread (q4, qc) owns row q4 * 32 + lane and columns
    // qc * 16 .. + 15 of each half.  Thread 0 issues every TMA operation: the
    // load of half h of the next tile goes out as soon as the store of half h
    // of this tile has read sC[h], so it runs under the next tile's MMAs.
    const int q4 = warp & 3, qc = warp >> 2;
    const int row = q4 * 32 + lane;
    const int x = t0 + rb;
    auto load_half = [&](int ct, int h) {
      const uint32_t mb = smem_u32(&cfull[h]);
      mbar_expect_tx(mb, uint32_t(kWsCFloats * 4));
      tma_load_2d(smem_u32(sC + h * kWsCFloats), tmap, x, t0 + ct * kTcN + h * kWsHalf, mb);
    };
    if (tid == 0) {
      load_half(c_lo, 0);
      load_half(c_lo, 1);
    }
    int loads_issued = 2, loads_done = 0;  // thread 0's count of C halves requested / consumed
    for (int i = 0; i < nt; ++i) {
      const int a = i & 1, ct = c_lo + i;
      const bool w = !abort_flag && wait_phase(smem_u32(&accf[a]), uint32_t((i >> 1) & 1));
      if (!epi_bar_and(w)) {
        if (tid == 0) abort_flag = 1, atomicOr(err, 4);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      bool ok = true;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool wc = !abort_flag && wait_phase(smem_u32(&cfull[h]), uint32_t(i & 1));
        if (!epi_bar_and(wc)) {
          ok = false;
          break;
        }
        if (tid == 0) ++loads_done;
        uint32_t v[16];
        const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16) + uint32_t(a * kTcN + h * kWsHalf + qc * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        float *col = sC + h * kWsCFloats + (qc * 16) * kTcM + row;  // box order: rows fastest
        const float scl = tile_scale(ct);
#pragma unroll
        for (int j = 0; j < 16; ++j) col[j * kTcM] -= scl * __uint_as_float(v[j]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_bar();
        if (tid == 0) {
          tma_store_2d(tmap, x, t0 + ct * kTcN + h * kWsHalf, smem_u32(sC + h * kWsCFloats));
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          if (i + 1 < nt) {
            // sC[h] is read by the store before it is refilled
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            load_half(ct + 1, h);
            ++loads_issued;
          }
        }
      }
      if (!ok) {
        if (tid == 0) abort_flag = 1, atomicOr(err, 4);
        break;
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      if (tid == 0) mbar_arrive(smem_u32(&acce[a]));  // the accumulator is free again
    }
    if (tid == 0) {
      // bounded waits for the C loads still writing sC, then for the stores
      for (int g = loads_done; g < loads_issued; ++g) wait_phase(smem_u32(&cfull[g & 1]), uint32_t((g >> 1) & 1));
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
  } else {
    // ---- epilogue warps without TMA: thread (q4, qc) owns row q4 * 32 + lane, columns qc * 32 .. + 31 ----
    const int q4 = warp & 3, qc = warp >> 2;
    const int row = rb + q4 * 32 + lane;
    for (int i = 0; i < nt; ++i) {
      const int a = i & 1, ct = c_lo + i;
      const int cb = ct * kTcN + qc * 32;
      float *Crow = A + (t0 + row) + int64_t(t0 + cb) * ld;
      const int ncol = row < nrest ? min(32, nrest - cb) : 0;
      float cv[32];
      {
        const float *p = Crow;  // one pointer, bumped by ld (not 32 live addresses)
#pragma unroll
        for (int j = 0; j < 32; ++j, p += ld) cv[j] = j < ncol ? *p : 0.f;
      }
      const bool w = !abort_flag && wait_phase(smem_u32(&accf[a]), uint32_t((i >> 1) & 1));
      if (!epi_bar_and(w)) {
        if (tid == 0) abort_flag = 1, atomicOr(err, 4);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16) + uint32_t(a * kTcN + qc * 32 + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const float scl = tile_scale(ct);
#pragma unroll
        for (int j = 0; j < 16; ++j) cv[c0 + j] -= scl * __uint_as_float(v[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      epi_bar();
      if (tid == 0) mbar_arrive(smem_u32(&acce[a]));  // the accumulator is free again
      {
        float *p = Crow;
#pragma unroll
        for (int j = 0; j < 32; ++j, p += ld)
          if (j < ncol) *p = cv[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(2 * kTcN)));
}

// ---- the block-end update with 128 x 256 output tiles ----
// The same update as k_gemm_tc_ws (three-term TF32 products; C -= L21 U12
// from the packed A and B, or with `lower` the block Cholesky's lower
// triangle C -= L21 L21^T with B = A's pack), with the column tiles taken in
// pairs: one kind::tf32 MMA of N = 256 per K step reads two packed 128-row
// B tiles laid one after the other in shared memory (their 8-row groups
// continue at the same stride), so each staged byte of A serves twice the
// products.  A pair whose second tile lies past the last column tile (or,
// with `lower`, past the diagonal tile) is a single tile with the N = 128 MMA.
// S 48 KB operand stages, two 256-column TMEM accumulators (all 512
// columns), and the C tile through TMA in 64-column quarters.  RED = false
// (three stages): C is loaded, the product subtracted and C stored back
// through two alternating buffers, quarter s + 2 requested as soon as the
// store of quarter s has read its buffer.  RED = true (four stages): the
// negated product goes out as a TMA reduce-add into C (one FP32 addition in
// L2, the rounding of C - product) through one buffer, so the epilogue never
// waits for C and the freed buffer buys a fourth operand stage.  Every wait
// is bounded, as in k_gemm_tc_ws.
constexpr int kWdStages = 3;     // with the load / store epilogue
constexpr int kWdStagesRed = 4;  // with the reduce-add epilogue (one C buffer)
constexpr int kWdStageFloats = 6 * kPkTile;  // A hi, A lo, B hi x 2 tiles, B lo x 2 tiles: 48 KB
constexpr uint32_t kIdescWide = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(256 >> 3) << 17) |
                                (uint32_t(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_tf32_i(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

template <bool RED, int S>
__global__ void __launch_bounds__(kWsThreads, 1) k_gemm_tc_wide(const FrontDev *__restrict__ fr, int j0, int kb,
                                                               float *__restrict__ fronts, int *__restrict__ err,
                                                               int splits, int tile_lo, int tile_hi,
                                                               const float *__restrict__ apack,
                                                               const float *__restrict__ bpack, int lower,
                                                               const uint8_t *__restrict__ maps64) {
  const FrontDev F = fr[blockIdx.z];
  if (j0 >= F.s) return;
  const int jb = min(kb, F.s - j0);
  const int t0 = j0 + jb;
  const int nrest = F.f - t0;
  const int rb = blockIdx.y * kTcM;
  if (rb >= nrest) return;
  // column tiles [tile_lo, tend) (with `lower`, up to the diagonal tile), taken in pairs
  const int tend_all = min((nrest + kTcN - 1) / kTcN, tile_hi);
  const int tend = lower ? min(tend_all, int(blockIdx.y) + 1) : tend_all;
  if (tend <= tile_lo) return;
  const int npair = (tend - tile_lo + 1) / 2;
  const int per = (npair + splits - 1) / splits;
  const int p_lo = blockIdx.x * per, p_hi = min(npair, p_lo + per);
  if (p_lo >= p_hi) return;
  const int np = p_hi - p_lo;
  const int nq = (jb + kPkK - 1) / kPkK;
  const int G = np * nq;
  auto pair_tile = [&](int i) { return tile_lo + 2 * (p_lo + i); };
  auto pair_wide = [&](int i) { return pair_tile(i) + 1 < tend; };
  float *A = fronts + F.off;
  const int64_t ld = F.ld;
  extern __shared__ __align__(1024) unsigned char smraw[];
  float *stage0 = reinterpret_cast<float *>(smraw);
  float *sC = stage0 + S * kWdStageFloats;  // 128 x 64 C quarters: two (RED: one)
  __shared__ __align__(8) uint64_t full[S], empty[S], accf[2], acce[2], cfull[2];
  const bool use_tma = maps64 != nullptr && (t0 & 3) == 0;
  const void *tmap = use_tma ? static_cast<const void *>(maps64 + size_t(blockIdx.z) * kTmapBytes) : nullptr;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ volatile int s_consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(uint32_t(4 * kTcN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(1));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&accf[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&cfull[i])), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    s_consumed = 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const float *Ab = apack + (int64_t(F.pack_off) + blockIdx.y) * kPackTileFloats;
  const float *Bb = bpack + int64_t(F.pack_off) * kPackTileFloats;
  constexpr uint32_t kArr = kPkTile * 4;  // one 128 x 16 hi (or lo) array: 8 KB

  if (warp == kWsEpiWarps) {
    // ---- copy producer ----
    if (lane == 0) {
      int issued = 0;
      for (int g = 0; g < G; ++g) {
        const int st = g % S, i = g / nq, q = g % nq;
        if (g >= S) {
          const bool w = !abort_flag && wait_phase(smem_u32(&empty[st]), uint32_t(((g - S) / S) & 1));
          if (!w) {
            abort_flag = 1;
            break;
          }
        }
        const int c0 = pair_tile(i);
        const bool wide = pair_wide(i);
        const float *a = Ab + int64_t(q) * 2 * kPkTile;
        const float *b0 = Bb + int64_t(c0) * kPackTileFloats + int64_t(q) * 2 * kPkTile;
        const float *b1 = b0 + kPackTileFloats;
        const uint32_t dst = smem_u32(stage0 + st * kWdStageFloats);
        const uint32_t mb = smem_u32(&full[st]);
        mbar_expect_tx(mb, 2 * kArr + (wide ? 4 : 2) * kArr);
        bulk_copy_g2s(dst, a, 2 * kArr, mb);                       // A hi, A lo
        bulk_copy_g2s(dst + 2 * kArr, b0, kArr, mb);               // B hi, tile c0
        if (wide) bulk_copy_g2s(dst + 3 * kArr, b1, kArr, mb);     // B hi, tile c0 + 1
        bulk_copy_g2s(dst + 4 * kArr, b0 + kPkTile, kArr, mb);     // B lo, tile c0
        if (wide) bulk_copy_g2s(dst + 5 * kArr, b1 + kPkTile, kArr, mb);  // B lo, tile c0 + 1
        ++issued;
      }
      if (abort_flag) {
        atomicOr(err, 4);
        for (int g = s_consumed; g < issued; ++g)
          wait_phase(smem_u32(&full[g % S]), uint32_t((g / S) & 1));
      }
    }
  } else if (warp == kWsEpiWarps + 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int last_mma = -1;
      bool ok = true;
      for (int g = 0; g < G && ok; ++g) {
        const int st = g % S, i = g / nq, q = g % nq, a = i & 1;
        if (abort_flag || !wait_phase(smem_u32(&full[st]), uint32_t((g / S) & 1))) {
          ok = false;
          break;
        }
        s_consumed = g + 1;
        if (q == 0 && i >= 2 && !wait_phase(smem_u32(&acce[a]), uint32_t(((i - 2) >> 1) & 1))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t base = smem_u32(stage0 + st * kWdStageFloats);
        const uint32_t ah0 = base, al0 = base + kArr, bh0 = base + 2 * kArr, bl0 = base + 4 * kArr;
        const uint32_t acc = tmem + uint32_t(a * 2 * kTcN);
        const uint32_t idesc = pair_wide(i) ? kIdescWide : kIdesc;
#pragma unroll
        for (int kk = 0; kk < kPkK / 8; ++kk) {
          const uint32_t koff = uint32_t(kk) * 2 * kLbo;
          const uint64_t ah = smem_desc_pk(ah0 + koff), al = smem_desc_pk(al0 + koff);
          const uint64_t bh = smem_desc_pk(bh0 + koff), bl = smem_desc_pk(bl0 + koff);
          mma_tf32_i(acc, ah, bh, idesc, (q > 0 || kk > 0) ? 1u : 0u);
          mma_tf32_i(acc, ah, bl, idesc, 1u);
          mma_tf32_i(acc, al, bh, idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&empty[st])));
        last_mma = g;
        if (q == nq - 1)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&accf[a])));
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(err, 4);
        if (last_mma >= 0)
          wait_phase(smem_u32(&empty[last_mma % S]), uint32_t((last_mma / S) & 1));
      }
    }
  } else if (use_tma && RED) {
    // ---- epilogue by TMA reduce-add: slot s = quarter (s & 3) of pair (s >> 2), buffer s & 1 ----
    const int q4 = warp & 3, qc = warp >> 2;
    const int row = q4 * 32 + lane;
    const int x = t0 + rb;
    bool ok = true;
    for (int i = 0; i < np && ok; ++i) {
      const int a = i & 1;
      const bool w = !abort_flag && wait_phase(smem_u32(&accf[a]), uint32_t((i >> 1) & 1));
      if (!epi_bar_and(w)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int nqq = pair_wide(i) ? 4 : 2;
      for (int qq = 0; qq < nqq; ++qq) {
        const int sl = 4 * i + qq, buf = 0;
        uint32_t v[16];
        const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16) + uint32_t(a * 2 * kTcN + qq * kWsHalf + qc * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (sl >= 1) {
          // the reduce of the previous quarter has read the (single) buffer
          if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          epi_bar();
        }
        float *col = sC + buf * kWsCFloats + (qc * 16) * kTcM + row;
#pragma unroll
        for (int j = 0; j < 16; ++j) col[j * kTcM] = -__uint_as_float(v[j]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_bar();
        if (tid == 0) {
          tma_reduce_add_2d(tmap, x, t0 + pair_tile(i) * kTcN + qq * kWsHalf, smem_u32(sC + buf * kWsCFloats));
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      if (tid == 0) mbar_arrive(smem_u32(&acce[a]));
    }
    if (!ok && tid == 0) abort_flag = 1, atomicOr(err, 4);
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  } else if (use_tma) {
    // ---- epilogue with TMA: slot s = quarter (s & 3) of pair (s >> 2), 64 columns, buffer s & 1 ----
    const int q4 = warp & 3, qc = warp >> 2;
    const int row = q4 * 32 + lane;
    const int x = t0 + rb;
    const int nslot = 4 * (np - 1) + (pair_wide(np - 1) ? 4 : 2);
    auto slot_col = [&](int sl) { return t0 + pair_tile(sl >> 2) * kTcN + (sl & 3) * kWsHalf; };
    auto load_slot = [&](int sl) {
      const uint32_t mb = smem_u32(&cfull[sl & 1]);
      mbar_expect_tx(mb, uint32_t(kWsCFloats * 4));
      tma_load_2d(smem_u32(sC + (sl & 1) * kWsCFloats), tmap, x, slot_col(sl), mb);
    };
    if (tid == 0) {
      load_slot(0);
      if (nslot > 1) load_slot(1);
    }
    int loads_issued = min(2, nslot), loads_done = 0;
    bool ok = true;
    for (int i = 0; i < np && ok; ++i) {
      const int a = i & 1;
      const bool w = !abort_flag && wait_phase(smem_u32(&accf[a]), uint32_t((i >> 1) & 1));
      if (!epi_bar_and(w)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int nqq = pair_wide(i) ? 4 : 2;
      for (int qq = 0; qq < nqq; ++qq) {
        const int sl = 4 * i + qq, buf = sl & 1;
        const bool wc = !abort_flag && wait_phase(smem_u32(&cfull[buf]), uint32_t((sl >> 1) & 1));
        if (!epi_bar_and(wc)) {
          ok = false;
          break;
        }
        if (tid == 0) ++loads_done;
        uint32_t v[16];
        const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16) + uint32_t(a * 2 * kTcN + qq * kWsHalf + qc * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        float *col = sC + buf * kWsCFloats + (qc * 16) * kTcM + row;
#pragma unroll
        for (int j = 0; j < 16; ++j) col[j * kTcM] -= __uint_as_float(v[j]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_bar();
        if (tid == 0) {
          tma_store_2d(tmap, x, slot_col(sl), smem_u32(sC + buf * kWsCFloats));
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          if (sl + 2 < nslot) {
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            load_slot(sl + 2);
            ++loads_issued;
          }
        }
      }
      if (!ok) break;
      asm volatile("tcgen05.fence::before_thread_sync;");
      if (tid == 0) mbar_arrive(smem_u32(&acce[a]));
    }
    if (!ok && tid == 0) abort_flag = 1, atomicOr(err, 4);
    if (tid == 0) {
      for (int g = loads_done; g < loads_issued; ++g) wait_phase(smem_u32(&cfull[g & 1]), uint32_t((g >> 1) & 1));
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
  } else {
    // ---- epilogue without TMA: thread (q4, qc) owns row q4 * 32 + lane, columns qc * 32 .. + 31 of each tile ----
    const int q4 = warp & 3, qc = warp >> 2;
    const int row = rb + q4 * 32 + lane;
    for (int i = 0; i < np; ++i) {
      const int a = i & 1;
      const bool w = !abort_flag && wait_phase(smem_u32(&accf[a]), uint32_t((i >> 1) & 1));
      if (!epi_bar_and(w)) {
        if (tid == 0) abort_flag = 1, atomicOr(err, 4);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int nh = pair_wide(i) ? 2 : 1;
      for (int hh = 0; hh < nh; ++hh) {
        const int ct = pair_tile(i) + hh;
        const int cb = ct * kTcN + qc * 32;
        float *Crow = A + (t0 + row) + int64_t(t0 + cb) * ld;
        const int ncol = row < nrest ? min(32, nrest - cb) : 0;
        float cv[32];
        {
          const float *pp = Crow;
#pragma unroll
          for (int j = 0; j < 32; ++j, pp += ld) cv[j] = j < ncol ? *pp : 0.f;
        }
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 16) {
          uint32_t v[16];
          const uint32_t taddr =
              tmem + (uint32_t(q4 * 32) << 16) + uint32_t(a * 2 * kTcN + hh * kTcN + qc * 32 + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int j = 0; j < 16; ++j) cv[c0 + j] -= __uint_as_float(v[j]);
        }
        float *pp = Crow;
#pragma unroll
        for (int j = 0; j < 32; ++j, pp += ld)
          if (j < ncol) *pp = cv[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      epi_bar();
      if (tid == 0) mbar_arrive(smem_u32(&acce[a]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(4 * kTcN)));
}

// Whole-wave split count: each CTA takes ceil(ct / splits) column tiles of one
// row tile; the launch lasts about ceil(CTAs / slots) such ranges (plus the
// A staging, `lead` tiles), minimised over whole waves.
int wave_splits(int rt, int ct, int nfront, int slots, double lead) {
  int splits = 1;
  double best = 1e300;
  for (int sp = 1; sp <= ct; ++sp) {
    const int per = (ct + sp - 1) / sp;
    if (sp > 1 && (ct + sp - 2) / (sp - 1) == per) continue;  // same range length, more CTAs
    const double waves = double((int64_t(rt) * nfront * sp + slots - 1) / slots);
    const double cost = waves * (per + lead);
    if (cost < best - 1e-9) best = cost, splits = sp;
  }
  return splits;
}

}  // namespace

size_t gemm_tc_smem() { return size_t(24) * kTileFloats + 1024; }

cudaError_t launch_gemm_tc(const FrontDev *fr, int j0, int nfront, int max_f, float *fronts, int *err,
                           cudaStream_t s, int tile_lo, int tile_hi, int sm_budget, const uint8_t *maps,
                           bool any_full, bool any_partial) {
  if (cudaError_t ea = smem_attr((const void *)k_gemm_tc, int(gemm_tc_smem())); ea != cudaSuccess) return ea;
  if (cudaError_t ea = smem_attr((const void *)k_gemm_tc_tma, int(gemm_tc_smem())); ea != cudaSuccess) return ea;
  const int rest = max_f - j0 - 1;
  if (rest <= 0) return cudaSuccess;
  const int rt = (rest + kTcM - 1) / kTcM;
  const int ct = std::min((rest + kTcN - 1) / kTcN, tile_hi) - tile_lo;
  if (ct <= 0) return cudaSuccess;
  // One CTA per SM (shared memory).  Each CTA takes a contiguous range of
  // ceil(ct / splits) column tiles of one row tile; the launch lasts about
  // ceil(CTAs / SMs) such ranges (plus the A staging, ~0.3 tile), so splits
  // is chosen to minimise that over whole waves.
  const int splits = wave_splits(rt, ct, nfront, std::max(sm_budget, 1), 0.3);
  dim3 g(splits, rt, nfront);
  if (maps != nullptr) {
    if (any_full)
      k_gemm_tc_tma<<<g, kTcThreads, gemm_tc_smem(), s>>>(fr, j0, fronts, err, splits, tile_lo, tile_hi, maps);
    if (any_partial)
      k_gemm_tc<<<g, kTcThreads, gemm_tc_smem(), s>>>(fr, j0, fronts, err, splits, tile_lo, tile_hi, 1, 0, 0);
  } else {
    k_gemm_tc<<<g, kTcThreads, gemm_tc_smem(), s>>>(fr, j0, fronts, err, splits, tile_lo, tile_hi, 0, 0, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc_inner(const FrontDev *fr, int j0, int kb, int nfront, int max_f, float *fronts, int *err,
                                 cudaStream_t s, int sm_budget, int sym) {
  if (cudaError_t ea = smem_attr((const void *)k_gemm_tc, int(gemm_tc_smem())); ea != cudaSuccess) return ea;
  const int rest = max_f - j0 - 1;
  const int cols = (j0 / kb) * kb + kb - (j0 + kTcK);  // columns left in the outer block (at most)
  if (rest <= 0 || cols <= 0) return cudaSuccess;
  const int rt = (rest + kTcM - 1) / kTcM;
  const int ct = (cols + kTcN - 1) / kTcN;
  const int splits = wave_splits(rt, ct, nfront, std::max(sm_budget, 1), 0.3);
  dim3 g(splits, rt, nfront);
  k_gemm_tc<<<g, kTcThreads, gemm_tc_smem(), s>>>(fr, j0, fronts, err, splits, 0, ct, 0, kb, sym);
  return cudaGetLastError();
}

cudaError_t launch_pack_a(const FrontDev *fr, int j0, int kb, int nfront, int max_f, const float *fronts, float *apack,
                          cudaStream_t s) {
  const int rest = max_f - j0 - 1;
  if (rest <= 0 || nfront == 0) return cudaSuccess;
  k_pack_a<<<dim3(((rest + kTcM - 1) / kTcM) * kPackChunks, nfront), 256, 0, s>>>(fr, j0, kb, fronts, apack);
  return cudaGetLastError();
}

cudaError_t launch_pack_bf16(const FrontDev *fr, int j0, int kb, int nfront, int max_f, const float *fronts,
                             float *pack, cudaStream_t s, int mode) {
  const int rest = max_f - j0 - 1;
  if (rest <= 0 || nfront == 0) return cudaSuccess;
  const dim3 g((rest + kTcM - 1) / kTcM, nfront);
  if (mode == 2)
    k_pack_bf16x2<<<g, 256, 0, s>>>(fr, j0, kb, fronts, pack);
  else
    k_pack_bf16<<<g, 256, 0, s>>>(fr, j0, kb, fronts, pack);
  return cudaGetLastError();
}

cudaError_t launch_pack_b(const FrontDev *fr, int j0, int kb, int nfront, int max_f, const float *fronts, float *bpack,
                          int ct_lo, int ct_hi, cudaStream_t s) {
  const int rest = max_f - j0 - 1;
  if (rest <= 0 || nfront == 0) return cudaSuccess;
  const int nct = std::min((rest + kTcN - 1) / kTcN, ct_hi) - ct_lo;
  if (nct <= 0) return cudaSuccess;
  k_pack_b<<<dim3(nct * kPackChunks, nfront), 256, 0, s>>>(fr, j0, kb, fronts, bpack, ct_lo, ct_hi);
  return cudaGetLastError();
}

size_t gemm_ws_smem() { return (size_t(kWsStages) * 4 * kPkTile + 2 * size_t(kWsCFloats)) * sizeof(float) + 1024; }

cudaError_t launch_gemm_tc_ws(const FrontDev *fr, int j0, int kb, int nfront, int max_f, float *fronts, int *err,
                              cudaStream_t s, int tile_lo, int tile_hi, int sm_budget, const uint8_t *maps,
                              const float *apack, const float *bpack, int lower, int max_tiles,
                              const uint8_t *maps64, int bf16) {
  const void *kern = bf16 == 2 ? (const void *)k_gemm_tc_ws<2>
                     : bf16 == 1 ? (const void *)k_gemm_tc_ws<1>
                                 : (const void *)k_gemm_tc_ws<0>;
  if (cudaError_t ea = smem_attr(kern, int(gemm_ws_smem())); ea != cudaSuccess) return ea;
  (void)maps;
  if (apack == nullptr || bpack == nullptr) return cudaErrorInvalidValue;
  const int rest = max_f - j0 - 1;
  if (rest <= 0) return cudaSuccess;
  const int rt = (rest + kTcM - 1) / kTcM;
  const int ct = std::min((rest + kTcN - 1) / kTcN, tile_hi) - tile_lo;
  if (ct <= 0) return cudaSuccess;
  // a CTA's first tile costs about one more tile (set-up, first copies and C)
  int splits = wave_splits(rt, ct, nfront, std::max(sm_budget, 1), 1.0);
  // a cap on the column tiles of one CTA keeps CTAs short, so that the SMs
  // turn over often (work on a higher-priority stream gets them sooner)
  if (max_tiles > 0) splits = std::max(splits, std::min(ct, (ct + max_tiles - 1) / max_tiles));
  dim3 g(splits, rt, nfront);
  if (bf16 == 2)
    k_gemm_tc_ws<2><<<g, kWsThreads, gemm_ws_smem(), s>>>(fr, j0, kb, fronts, err, splits, tile_lo, tile_hi, apack,
                                                          bpack, lower, maps64);
  else if (bf16 == 1)
    k_gemm_tc_ws<1><<<g, kWsThreads, gemm_ws_smem(), s>>>(fr, j0, kb, fronts, err, splits, tile_lo, tile_hi, apack,
                                                          bpack, lower, maps64);
  else
    k_gemm_tc_ws<0><<<g, kWsThreads, gemm_ws_smem(), s>>>(fr, j0, kb, fronts, err, splits, tile_lo, tile_hi, apack,
                                                          bpack, lower, maps64);
  return cudaGetLastError();
}

size_t gemm_wide_smem(bool reduce) {
  return reduce ? (size_t(kWdStagesRed) * kWdStageFloats + size_t(kWsCFloats)) * sizeof(float) + 1024
                : (size_t(kWdStages) * kWdStageFloats + 2 * size_t(kWsCFloats)) * sizeof(float) + 1024;
}

cudaError_t launch_gemm_tc_wide(const FrontDev *fr, int j0, int kb, int nfront, int max_f, float *fronts, int *err,
                                cudaStream_t s, int tile_lo, int tile_hi, int sm_budget, const float *apack,
                                const float *bpack, int lower, int max_tiles, const uint8_t *maps64, int reduce) {
  const void *kern = reduce ? (const void *)k_gemm_tc_wide<true, kWdStagesRed>
                            : (const void *)k_gemm_tc_wide<false, kWdStages>;
  if (cudaError_t ea = smem_attr(kern, int(gemm_wide_smem(reduce != 0))); ea != cudaSuccess) return ea;
  if (apack == nullptr || bpack == nullptr) return cudaErrorInvalidValue;
  const int rest = max_f - j0 - 1;
  if (rest <= 0) return cudaSuccess;
  const int rt = (rest + kTcM - 1) / kTcM;
  const int ct = std::min((rest + kTcN - 1) / kTcN, tile_hi) - tile_lo;
  if (ct <= 0) return cudaSuccess;
  const int npair = (ct + 1) / 2;
  int splits = wave_splits(rt, npair, nfront, std::max(sm_budget, 1), 1.0);
  if (max_tiles > 0) {
    const int max_pairs = std::max(1, max_tiles / 2);
    splits = std::max(splits, std::min(npair, (npair + max_pairs - 1) / max_pairs));
  }
  dim3 g(splits, rt, nfront);
  if (reduce)
    k_gemm_tc_wide<true, kWdStagesRed><<<g, kWsThreads, gemm_wide_smem(true), s>>>(
        fr, j0, kb, fronts, err, splits, tile_lo, tile_hi, apack, bpack, lower, maps64);
  else
    k_gemm_tc_wide<false, kWdStages><<<g, kWsThreads, gemm_wide_smem(false), s>>>(
        fr, j0, kb, fronts, err, splits, tile_lo, tile_hi, apack, bpack, lower, maps64);
  return cudaGetLastError();
}

// One TMA descriptor per FP32 front: 2D, rows x columns, leading dimension
// ld (16-byte multiple), 128 x 128 boxes, zero fill outside the front.
cudaError_t make_front_tmaps(const Front *fronts, int n, const float *base, uint8_t *maps_dev, int box_cols) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (encode == nullptr) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || fn == nullptr || q != cudaDriverEntryPointSuccess) return e != cudaSuccess ? e : cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  static_assert(sizeof(CUtensorMap) == kTmapBytes, "tensor map size");
  std::vector<CUtensorMap> maps(std::max(n, 1));
  for (int k = 0; k < n; ++k) {
    const Front &F = fronts[k];
    const cuuint64_t dims[2] = {cuuint64_t(std::max(F.f, 1)), cuuint64_t(std::max(F.f, 1))};
    const cuuint64_t strides[1] = {cuuint64_t(F.ld) * sizeof(float)};
    const cuuint32_t box[2] = {cuuint32_t(kTcM), cuuint32_t(box_cols)};
    const cuuint32_t es[2] = {1, 1};
    CUresult r = encode(&maps[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base + F.off), dims, strides,
                        box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaMemcpy(maps_dev, maps.data(), sizeof(CUtensorMap) * size_t(n), cudaMemcpyHostToDevice);
}

}  // namespace h2sp
