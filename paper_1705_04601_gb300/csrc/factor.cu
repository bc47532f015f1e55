// Block LU of the sparse S and the triangular solves (multifrontal form).
//
// The paper factors S with a sparse direct solver (§5.3-5.4).  Here S is
// eliminated supernode by supernode in the nested-dissection order built on
// the host; each supernode owns a dense front
//       F = [F11 F12; F21 F22]   (s + b rows: supernode rows, then boundary rows)
// that receives its blocks of S and the contribution blocks of its children.
// A front is factored by a right-looking blocked LU that stops after its s
// supernode columns, with partial pivoting restricted to the supernode rows:
//   panel      : columns [j0, j0+jb), rows [j0, f), pivots searched in [j0, s)
//   swap+trsm  : the panel's row swaps on the other columns, U12 = L^-1 A12
//   gemm       : trailing update A22 -= L21 U12
// The trailing block left in F22 is the contribution block, added into the
// parent front (extend-add).  All fronts of one elimination level (one depth
// of the closure clusters) are processed by the same launches.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include <cooperative_groups.h>

#include "kernels.h"

namespace h2sp {
namespace {

// |x| with the sign bit cleared (-0 becomes +0, which the bit-pattern argmax needs)
template <typename T>
__device__ __forceinline__ T tabs(T x) {
  return fabs(x);
}

template <typename TS, typename T>
__global__ void k_assemble(const AItem *__restrict__ items, const TS *__restrict__ S, T *__restrict__ F) {
  const AItem it = items[blockIdx.x];
  const int n = it.rows * it.cols;
  const TS *src = S + it.src;
  T *dst = F + it.dst;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = i % it.rows, c = i / it.rows;
    dst[r + int64_t(c) * it.ld] = T(src[i]);
  }
}

constexpr int kPanelThreads = 512;

template <typename T, int NB>
__global__ void __launch_bounds__(kPanelThreads) k_panel(const FrontDev *__restrict__ fr, int j0, T *__restrict__ fronts,
                                                         int32_t *__restrict__ piv, int32_t *__restrict__ swaps,
                                                         int *__restrict__ err) {
  const FrontDev F = fr[blockIdx.x];
  if (j0 >= F.s) return;
  const int jb = min(NB, F.s - j0);
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  __shared__ T urow[NB];
  __shared__ T redv[kPanelThreads / 32];
  __shared__ int redi[kPanelThreads / 32];
  __shared__ int s_p;
  __shared__ T s_pv;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int j = 0; j < jb; ++j) {
    const int col = j0 + j;
    T *Acol = A + int64_t(col) * ld;
    T bv = T(-1);
    int bi = INT_MAX;
    for (int r = col + tid; r < F.s; r += nt) {
      const T v = tabs(Acol[r]);
      if (v > bv) bv = v, bi = r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) bv = ov, bi = oi;
    }
    if (lane == 0) redv[wid] = bv, redi[wid] = bi;
    __syncthreads();
    if (tid == 0) {
      T v = redv[0];
      int i = redi[0];
      for (int w = 1; w < (nt >> 5); ++w)
        if (redv[w] > v || (redv[w] == v && redi[w] < i)) v = redv[w], i = redi[w];
      if (i == INT_MAX) {  // every candidate is NaN
        i = col;
        atomicOr(err, 2);
      }
      s_p = i;
      piv[F.piv_off + col] = i;
      const T pv = A[i + int64_t(col) * ld];
      s_pv = pv;
      if (pv == T(0)) atomicOr(err, 1);
    }
    __syncthreads();
    const int p = s_p;
    if (p != col)
      for (int c = j0 + tid; c < j0 + jb; c += nt) {
        T *a = A + int64_t(c) * ld;
        const T t = a[col];
        a[col] = a[p];
        a[p] = t;
      }
    __syncthreads();
    for (int c = col + 1 + tid; c < j0 + jb; c += nt) urow[c - j0] = A[col + int64_t(c) * ld];
    __syncthreads();
    const T pv = s_pv;
    if (pv != T(0)) {
      const T inv = T(1) / pv;
      for (int r = col + 1 + tid; r < F.f; r += nt) {
        const T l = Acol[r] * inv;
        Acol[r] = l;
        for (int c = col + 1; c < j0 + jb; ++c) A[r + int64_t(c) * ld] -= l * urow[c - j0];
      }
    }
    __syncthreads();
  }
  // net row movement of this panel: the swaps compose to new_row[r] = old_row[src[r]]
  if (tid == 0) {
    int32_t *sw = swaps + int64_t(blockIdx.x) * (1 + 2 * kMaxSwapRows);
    int nr = 0;
    int32_t *rows = sw + 1, *src = sw + 1 + kMaxSwapRows;
    for (int j = 0; j < jb; ++j) {
      const int a = j0 + j, b = piv[F.piv_off + a];
      if (a == b) continue;
      int ia = -1, ib = -1;
      for (int q = 0; q < nr; ++q) {
        if (rows[q] == a) ia = q;
        if (rows[q] == b) ib = q;
      }
      if (ia < 0) rows[nr] = a, src[nr] = a, ia = nr++;
      if (ib < 0) rows[nr] = b, src[nr] = b, ib = nr++;
      const int32_t t = src[ia];
      src[ia] = src[ib];
      src[ib] = t;
    }
    sw[0] = nr;
  }
}

constexpr int kClusterPanelThreads = 512;
constexpr int kMaxPanelCluster = 16;
constexpr int kPanelRowsPerThread = 4;  // rows per CTA <= 4 * 512 (shared memory allows ~800)

__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Panel factorization by one thread-block cluster per front.  The panel rows
// [j0, f) are split into C contiguous chunks, one per CTA, held in shared
// memory for the whole panel; thread t owns local rows t, t + 512, ...
// Rows are not moved while the panel is factored (logical pivoting).  Per
// column j:
//   A  column j of every live row receives the update of pivot j - 1;
//   B  each CTA finds its best live supernode row of column j (exact ties to
//      the lowest row) and pushes (value, row index, row) into a mailbox slot
//      of every CTA of the cluster (remote shared-memory stores);
//   -  cluster barrier, split: after arriving, the CTA applies the deferred
//      update of pivot j - 1 to columns j+1.. of its live rows, then waits;
//   C  every warp reduces the C candidates of its own mailbox: pivot row p;
//      the pivot row's columns > j are brought up to date from the previous
//      pivot row, its owner retires it, and the multipliers of column j are
//      formed.
// The mailbox alternates between two slots; a slot is rewritten only after
// every CTA has passed the barrier of the column that read it.  At the end
// each CTA turns the pivot sequence into LAPACK's sequential row interchanges
// and writes its rows to their final positions.
template <typename T, int NB>
__global__ void __launch_bounds__(kClusterPanelThreads) k_panel_cluster(const FrontDev *__restrict__ fr, int j0,
                                                                        T *__restrict__ fronts, int32_t *__restrict__ piv,
                                                                        int32_t *__restrict__ swaps, int *__restrict__ err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = int(cluster.num_blocks());
  const int rank = int(cluster.block_rank());
  const int fi = blockIdx.x / C;
  const FrontDev F = fr[fi];
  if (j0 >= F.s) return;  // uniform over the cluster: no barrier is ever entered
  const int jb = min(NB, F.s - j0);
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  const int R = F.f - j0;
  const int per = (R + C - 1) / C;
  const int r_lo = j0 + rank * per;
  const int nr = max(0, min(F.f, r_lo + per) - r_lo);
  extern __shared__ __align__(16) unsigned char smraw[];
  T *P = reinterpret_cast<T *>(smraw);                        // [NB][per], column c at P + c * per
  int32_t *dest = reinterpret_cast<int32_t *>(P + NB * per);  // [per] final row of each local row
  unsigned char *done = reinterpret_cast<unsigned char *>(dest + per);  // [per] retired pivot rows
  __shared__ T mb_row[2][kMaxPanelCluster][NB];  // mailbox: candidate rows, values, row indices
  __shared__ T mb_v[2][kMaxPanelCluster];
  __shared__ int mb_i[2][kMaxPanelCluster];
  __shared__ T urow[2][NB];  // up-to-date pivot rows of the last two columns
  __shared__ T stage[kClusterPanelThreads / 32][NB];  // each warp's candidate row
  __shared__ T redv[kClusterPanelThreads / 32];
  __shared__ int redi[kClusterPanelThreads / 32];
  __shared__ int hist[NB];
  __shared__ int32_t lrow[2 * NB], lsrc[2 * NB];
  __shared__ int nswap;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < nr * jb; e += nt) {
    const int i = e % nr, c = e / nr;
    P[c * per + i] = A[(r_lo + i) + int64_t(j0 + c) * ld];
  }
  for (int i = tid; i < per; i += nt) done[i] = 0, dest[i] = r_lo + i;
  const int i_hi = max(0, min(F.s, r_lo + nr) - r_lo);  // local supernode rows
  T lmul[kPanelRowsPerThread];  // multipliers of the last pivot for this thread's rows
#pragma unroll
  for (int k = 0; k < kPanelRowsPerThread; ++k) lmul[k] = T(0);
  T u_next = T(0);  // the last pivot row's entry in the current column
  // every CTA of the cluster is running (and its mailbox exists) past this point
  cluster.sync();
  for (int j = 0; j < jb; ++j) {
    const int buf = j & 1;
    // A: pivot j - 1 on column j, and this thread's candidate
    T bv = T(-1);
    int bi = INT_MAX;
#pragma unroll
    for (int k = 0; k < kPanelRowsPerThread; ++k) {
      const int i = tid + k * nt;
      if (i >= nr) break;
      if (i < i_hi && done[i]) continue;
      T v = P[j * per + i];
      if (j > 0) {
        v -= lmul[k] * u_next;
        P[j * per + i] = v;
      }
      if (i < i_hi) {
        const T a = tabs(v);
        if (a > bv) bv = a, bi = r_lo + i;
      }
    }
    // B: warp candidates, each staged with its row (the owner may update the
    // row in shared memory during the barrier), then the CTA candidate
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) bv = ov, bi = oi;
    }
    __syncwarp();
    {
      const int wl = (bi == INT_MAX) ? -1 : bi - r_lo;
      for (int c = lane; c < jb; c += 32) stage[wid][c] = wl >= 0 ? P[c * per + wl] : T(0);
    }
    if (lane == 0) redv[wid] = bv, redi[wid] = bi;
    __syncthreads();
    int ww = lane;
    {
      T v = lane < (nt >> 5) ? redv[lane] : T(-1);
      int i = lane < (nt >> 5) ? redi[lane] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        const int ow = __shfl_xor_sync(0xffffffffu, ww, o);
        if (ov > v || (ov == v && oi < i)) v = ov, i = oi, ww = ow;
      }
      bv = v;
      bi = i;
    }
    for (int e = tid; e < C * (jb + 2); e += nt) {
      const int q = e / (jb + 2), c = e % (jb + 2);
      if (c < jb) {
        cluster.map_shared_rank(&mb_row[buf][rank][0], q)[c] = stage[ww][c];
      } else if (c == jb) {
        *cluster.map_shared_rank(&mb_v[buf][rank], q) = bv;
      } else {
        *cluster.map_shared_rank(&mb_i[buf][rank], q) = bi;
      }
    }
    cluster_arrive_release();
    // deferred: pivot j - 1 on columns j+1 .. jb-1 of the live rows
    if (j > 0) {
      const T *u = urow[(j - 1) & 1];
#pragma unroll
      for (int k = 0; k < kPanelRowsPerThread; ++k) {
        const int i = tid + k * nt;
        if (i >= nr) break;
        if (i < i_hi && done[i]) continue;
        const T l = lmul[k];
        for (int c = j + 1; c < jb; ++c) P[c * per + i] -= l * u[c];
      }
    }
    cluster_wait_acquire();
    // C: the pivot of column j from the mailbox
    T v = lane < C ? mb_v[buf][lane] : T(-1);
    int i = lane < C ? mb_i[buf][lane] : INT_MAX;
    int w = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      const int ow = __shfl_xor_sync(0xffffffffu, w, o);
      if (ov > v || (ov == v && oi < i)) v = ov, i = oi, w = ow;
    }
    int p = i;
    T pv, lprev = T(0);
    const T *prow;
    if (p == INT_MAX) {
      // no finite candidate: keep the sequence a permutation with the lowest
      // not-yet-pivoted supernode row; the factorization reports the failure
      if (tid == 0 && rank == 0) atomicOr(err, 2);
      p = j0;
      bool used = true;
      while (used) {
        used = false;
        for (int q = 0; q < j; ++q)
          if (hist[q] == p) used = true, ++p;
      }
      prow = nullptr;
      pv = T(0);
    } else {
      prow = &mb_row[buf][w][0];
      pv = prow[j];
      if (j > 0) lprev = prow[j - 1];
    }
    if (tid == 0) hist[j] = p;
    // up-to-date pivot row: columns > j still lack the update of pivot j - 1
    if (j + 1 < jb) {
      if (prow != nullptr) {
        u_next = prow[j + 1] - (j > 0 ? lprev * urow[(j - 1) & 1][j + 1] : T(0));
        if (wid == 0)
          for (int c = j + 1 + lane; c < jb; c += 32)
            urow[buf][c] = prow[c] - (j > 0 ? lprev * urow[(j - 1) & 1][c] : T(0));
      } else {
        u_next = T(0);
        if (wid == 0)
          for (int c = j + 1 + lane; c < jb; c += 32) urow[buf][c] = T(0);
      }
    }
    if (p >= r_lo && p < r_lo + nr && (p - r_lo) % nt == tid) done[p - r_lo] = 1;
    if (pv == T(0)) {
      if (tid == 0 && rank == 0) atomicOr(err, 1);
#pragma unroll
      for (int k = 0; k < kPanelRowsPerThread; ++k) lmul[k] = T(0);
    } else {
      const T inv = T(1) / pv;
#pragma unroll
      for (int k = 0; k < kPanelRowsPerThread; ++k) {
        const int ii = tid + k * nt;
        lmul[k] = T(0);
        if (ii >= nr) break;
        if (ii < i_hi && done[ii]) continue;
        const T l = P[j * per + ii] * inv;
        P[j * per + ii] = l;
        lmul[k] = l;
      }
    }
  }
  __syncthreads();
  // LAPACK-style interchanges from the pivot sequence, and where every row goes
  if (tid == 0) {
    int n = 0;  // touched positions: position lrow[q] currently holds physical row lsrc[q]
    for (int j = 0; j < jb; ++j) {
      const int col = j0 + j, p = hist[j];
      int ip = -1, ic = -1;
      for (int q = 0; q < n; ++q) {
        if (lsrc[q] == p) ip = q;
        if (lrow[q] == col) ic = q;
      }
      const int pos_p = ip >= 0 ? lrow[ip] : p;  // untouched rows sit at their own position
      if (rank == 0) piv[F.piv_off + col] = pos_p;
      if (pos_p == col) continue;
      if (ic < 0) lrow[n] = col, lsrc[n] = col, ic = n++;
      if (ip < 0) lrow[n] = p, lsrc[n] = p, ip = n++;
      const int32_t t = lsrc[ic];
      lsrc[ic] = lsrc[ip];
      lsrc[ip] = t;
    }
    nswap = n;
    if (rank == 0) {
      int32_t *sw = swaps + int64_t(fi) * (1 + 2 * kMaxSwapRows);
      for (int q = 0; q < n; ++q) sw[1 + q] = lrow[q], sw[1 + kMaxSwapRows + q] = lsrc[q];
      sw[0] = n;
    }
  }
  __syncthreads();
  for (int q = tid; q < nswap; q += nt) {
    const int src = lsrc[q];
    if (src >= r_lo && src < r_lo + nr) dest[src - r_lo] = lrow[q];
  }
  __syncthreads();
  for (int e = tid; e < nr * jb; e += nt) {
    const int i = e % nr, c = e / nr;
    A[dest[i] + int64_t(j0 + c) * ld] = P[c * per + i];
  }
  // no CTA may exit while others can still write into its mailbox
  cluster.sync();
}

// Argmax over a warp: the largest value, ties to the lowest index; lanes
// without a candidate pass (anything, INT_MAX).  Every lane gets the result
// (value -1 and INT_MAX when no lane has a candidate).  Values are absolute
// values (non-negative, never NaN); for FP32 their bit patterns order like
// the values, so two hardware warp reductions do it.
template <typename T>
__device__ __forceinline__ void warp_argmax(T &v, int &i) {
  if constexpr (sizeof(T) == 4) {
    const unsigned key = i != INT_MAX ? __float_as_uint(v) : 0u;
    const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
    const int imin = __reduce_min_sync(0xffffffffu, (i != INT_MAX && key == kmax) ? i : INT_MAX);
    v = imin != INT_MAX ? __uint_as_float(kmax) : T(-1);
    i = imin;
  } else {
    if (i == INT_MAX) v = T(-1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) v = ov, i = oi;
    }
  }
}

constexpr int kRegPanelThreads = 384;
constexpr int kRegPanelRows = 2;  // panel rows per thread, held in registers
constexpr int kRegPanelMaxRows = kRegPanelThreads * kRegPanelRows;

// Tile-pivoted FP32 panel (the FP32 preconditioner's option): the pivot of
// column j0 + j is searched only among the rows of the panel's jb x jb
// diagonal tile, so no search or row exchange reaches below the tile.
// Step 1, one CTA per front: LU of the tile with partial pivoting among its
// rows (first maximum on ties), in shared memory; LAPACK ipiv and the step's
// swap list as k_panel_reg writes them.  Step 2 (k_panel_tile_l21): the rows
// below, L21 = A21 U11^-1.
constexpr int kTileThreads = 256;

template <int NB>
__global__ void __launch_bounds__(kTileThreads) k_panel_tile_diag(const FrontDev *__restrict__ fr, int j0,
                                                                  float *__restrict__ fronts,
                                                                  int32_t *__restrict__ piv,
                                                                  int32_t *__restrict__ swaps, int *__restrict__ err) {
  const FrontDev F = fr[blockIdx.x];
  if (j0 >= F.s) return;  // uniform over the CTA
  const int jb = min(NB, F.s - j0);
  float *A = fronts + F.off;
  const int64_t ld = F.ld;
  __shared__ float T[NB * NB];  // tile, column-major, ld NB
  __shared__ int perm[NB];      // tile row (relative to j0) now at each position
  __shared__ int s_p;
  __shared__ float s_inv;
  const int tid = threadIdx.x;
  for (int e = tid; e < jb * jb; e += kTileThreads) {
    const int r = e % jb, c = e / jb;
    T[r + c * NB] = A[(j0 + r) + int64_t(j0 + c) * ld];
  }
  for (int r = tid; r < jb; r += kTileThreads) perm[r] = r;
  __syncthreads();
  for (int j = 0; j < jb; ++j) {
    if (tid < 32) {
      // first row of largest modulus among rows j .. jb-1 of column j
      float best = -1.0f;
      int bi = jb;
      for (int r = j + tid; r < jb; r += 32) {
        const float v = fabsf(T[r + j * NB]);
        if (v > best) best = v, bi = r;  // rows visited in increasing order per lane
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
      }
      if (tid == 0) {
        if (bi >= jb) bi = j;  // no comparable candidate (NaN column): keep the row
        s_p = bi;
        piv[F.piv_off + j0 + j] = j0 + bi;
        const int t = perm[j];
        perm[j] = perm[bi];
        perm[bi] = t;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != j)
      for (int c = tid; c < jb; c += kTileThreads) {
        const float t = T[j + c * NB];
        T[j + c * NB] = T[p + c * NB];
        T[p + c * NB] = t;
      }
    __syncthreads();
    if (tid == 0) {
      const float pv = T[j + j * NB];
      if (pv == 0.0f) atomicOr(err, 1);
      s_inv = pv != 0.0f ? 1.0f / pv : 0.0f;
    }
    __syncthreads();
    const float inv = s_inv;
    for (int r = j + 1 + tid; r < jb; r += kTileThreads) T[r + j * NB] *= inv;
    __syncthreads();
    const int m = jb - j - 1;
    for (int e = tid; e < m * m; e += kTileThreads) {
      const int r = j + 1 + e % m, c = j + 1 + e / m;
      T[r + c * NB] -= T[r + j * NB] * T[j + c * NB];
    }
    __syncthreads();
  }
  for (int e = tid; e < jb * jb; e += kTileThreads) {
    const int r = e % jb, c = e / jb;
    A[(j0 + r) + int64_t(j0 + c) * ld] = T[r + c * NB];
  }
  if (tid == 0) {
    int32_t *sw = swaps + int64_t(blockIdx.x) * (1 + 2 * kMaxSwapRows);
    int n = 0;
    for (int r = 0; r < jb; ++r)
      if (perm[r] != r) {
        sw[1 + n] = j0 + r;
        sw[1 + kMaxSwapRows + n] = j0 + perm[r];
        ++n;
      }
    sw[0] = n;
  }
}

// Step 2: rows j0 + jb .. f of the panel columns, L21 = A21 U11^-1.  Each CTA
// inverts U11 in shared memory (back substitution, one column per thread),
// then each thread takes one row: the row in registers, one column of
// U11^-1 per output element.  grid = (row chunks of kL21Rows, fronts).
constexpr int kL21Rows = 64;

template <int NB>
__global__ void __launch_bounds__(kL21Rows) k_panel_tile_l21(const FrontDev *__restrict__ fr, int j0,
                                                             float *__restrict__ fronts) {
  static_assert(NB == kL21Rows, "one thread per column of U11 while inverting it");
  const FrontDev F = fr[blockIdx.y];
  if (j0 >= F.s) return;
  const int jb = min(NB, F.s - j0);
  const int row0 = j0 + jb + int(blockIdx.x) * kL21Rows;
  if (row0 >= F.f) return;  // uniform over the CTA
  float *A = fronts + F.off;
  const int64_t ld = F.ld;
  __shared__ float U[NB * NB];   // U11, column-major, ld NB; zero outside the upper jb x jb tile
  __shared__ float Ui[NB * NB];  // U11^-1 (upper); zero columns from jb on
  for (int e = threadIdx.x; e < NB * NB; e += kL21Rows) {
    const int r = e % NB, c = e / NB;
    U[e] = (r < jb && c < jb && r <= c) ? A[(j0 + r) + int64_t(j0 + c) * ld] : 0.0f;
  }
  __syncthreads();
  {
    const int c = int(threadIdx.x);  // U11 x = e_c, rows c down to 0
    for (int r = NB - 1; r > c; --r) Ui[r + c * NB] = 0.0f;
    if (c < jb) {
      const float d = U[c + c * NB];
      Ui[c + c * NB] = d != 0.0f ? 1.0f / d : 0.0f;
      for (int r = c - 1; r >= 0; --r) {
        float acc = 0.0f;
        for (int k = r + 1; k <= c; ++k) acc += U[r + k * NB] * Ui[k + c * NB];
        const float dr = U[r + r * NB];
        Ui[r + c * NB] = dr != 0.0f ? -acc / dr : 0.0f;
      }
    } else {
      for (int r = c; r >= 0; --r) Ui[r + c * NB] = 0.0f;
    }
  }
  __syncthreads();
  const int row = row0 + int(threadIdx.x);
  if (row >= F.f) return;
  float a[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) a[k] = k < jb ? A[row + int64_t(j0 + k) * ld] : 0.0f;
#pragma unroll 1
  for (int c = 0; c < jb; ++c) {
    const float *ui = Ui + c * NB;
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < NB; ++k) acc += a[k] * ui[k];
    A[row + int64_t(j0 + c) * ld] = acc;
  }
}

// Panel factorization with the rows in registers, by one thread-block cluster
// per front.  Thread t of CTA q holds rows r_lo(q) + t and r_lo(q) + t + 384,
// NB values each, in a shifting frame: at column j, slot 0 holds column j,
// slot c column j + c, and the multipliers l_0 .. l_{j-1} of the row fill the
// last j slots.  Per column: every warp stages its best live supernode row,
// one barrier, the CTA candidate (value, row index, pivot value, row) is
// pushed into a mailbox slot of every CTA of the cluster, a cluster barrier,
// then every thread reduces the C candidates of its own mailbox (exact ties
// to the lowest row), retires the pivot row if it holds it, and updates its
// live rows while shifting them by one slot: x[c] = x[c+1] - l u[c] with
// l = x[0] / pivot and u the pivot row's columns j+1.., and x[NB-1] = l.
// Rows are never moved during the panel (logical pivoting); at the end the
// pivot sequence becomes LAPACK's sequential interchanges (piv) and every row
// is written once to its final position.
template <typename T, int NB>
__global__ void __launch_bounds__(kRegPanelThreads, 1) k_panel_reg(const FrontDev *__restrict__ fr, int j0,
                                                                   T *__restrict__ fronts, int32_t *__restrict__ piv,
                                                                   int32_t *__restrict__ swaps, int *__restrict__ err) {
  namespace cg = cooperative_groups;
  static_assert(kRegPanelRows == 2, "the staging below names rows 0 and 1");
  static_assert(NB % 4 == 0 && NB <= 64, "panel width");
  constexpr int NW = kRegPanelThreads / 32;
  constexpr int VE = 16 / int(sizeof(T));  // elements per 16-byte vector
  cg::cluster_group cluster = cg::this_cluster();
  const int C = int(cluster.num_blocks());
  const int rank = int(cluster.block_rank());
  const int fi = blockIdx.x / C;
  const FrontDev F = fr[fi];
  if (j0 >= F.s) return;  // uniform over the cluster
  const int jb = min(NB, F.s - j0);
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  const int R = F.f - j0;
  const int per = (R + C - 1) / C;
  const int r_lo = j0 + rank * per;
  const int nr = max(0, min(F.f, r_lo + per) - r_lo);
  extern __shared__ __align__(16) unsigned char smraw[];
  int32_t *pos_of = reinterpret_cast<int32_t *>(smraw);  // [R] final position of each panel row
  int32_t *at_pos = pos_of + R;                          // [R] row now at each position
  unsigned char *touched = reinterpret_cast<unsigned char *>(at_pos + R);  // [R]
  __shared__ __align__(16) T mb_row[2][kMaxPanelCluster][NB];  // mailbox: pivot candidates' columns j+1..
  __shared__ T mb_v[2][kMaxPanelCluster], mb_pv[2][kMaxPanelCluster];
  __shared__ int mb_i[2][kMaxPanelCluster];
  __shared__ __align__(16) T stage[NW][NB];
  __shared__ T stage_pv[NW];
  __shared__ T redv[NW];
  __shared__ int redi[NW];
  __shared__ int hist[NB];
  __shared__ int32_t lrow[2 * NB], lsrc[2 * NB];
  __shared__ int nswap;
  const int tid = threadIdx.x, nt = kRegPanelThreads, lane = tid & 31, wid = tid >> 5;

  T x[kRegPanelRows][NB];
  int ret[kRegPanelRows];  // -2: no row, -1: live, >= 0: column at which it became a pivot
  bool sn[kRegPanelRows];  // supernode row (pivot candidate)
#pragma unroll
  for (int k = 0; k < kRegPanelRows; ++k) {
    const int i = tid + k * nt;
    ret[k] = i < nr ? -1 : -2;
    sn[k] = i < nr && r_lo + i < F.s;
    const T *src = A + (r_lo + i) + int64_t(j0) * ld;
#pragma unroll
    for (int c = 0; c < NB; ++c) x[k][c] = (i < nr && c < jb) ? src[int64_t(c) * ld] : T(0);
  }
  // every CTA of the cluster is running (its mailbox exists) past this point
  cluster.sync();
  for (int j = 0; j < jb; ++j) {
    const int buf = j & 1;
    // this thread's best live supernode row (the lower row wins ties)
    T bv = T(-1);
    int bi = INT_MAX, bk = -1;
#pragma unroll
    for (int k = 0; k < kRegPanelRows; ++k)
      if (ret[k] == -1 && sn[k]) {
        const T a = tabs(x[k][0]);
        if (a > bv) bv = a, bi = r_lo + tid + k * nt, bk = k;
      }
    const int my_bi = bi;
    warp_argmax(bv, bi);
    // the owner stages the warp candidate: slots 1.. (columns j+1..) and the pivot value
    if (bi != INT_MAX && my_bi == bi) {
      T *st = stage[wid];
      if (bk == 0) {
        stage_pv[wid] = x[0][0];
#pragma unroll
        for (int c = 0; c < NB; c += VE) {
          if constexpr (VE == 4) {
            *reinterpret_cast<float4 *>(st + c) =
                make_float4(x[0][c + 1], x[0][c + 2], x[0][c + 3], c + 4 < NB ? x[0][(c + 4) % NB] : T(0));
          } else {
            *reinterpret_cast<double2 *>(st + c) = make_double2(x[0][c + 1], c + 2 < NB ? x[0][(c + 2) % NB] : T(0));
          }
        }
      } else {
        stage_pv[wid] = x[kRegPanelRows - 1][0];
#pragma unroll
        for (int c = 0; c < NB; c += VE) {
          constexpr int K = kRegPanelRows - 1;
          if constexpr (VE == 4) {
            *reinterpret_cast<float4 *>(st + c) =
                make_float4(x[K][c + 1], x[K][c + 2], x[K][c + 3], c + 4 < NB ? x[K][(c + 4) % NB] : T(0));
          } else {
            *reinterpret_cast<double2 *>(st + c) = make_double2(x[K][c + 1], c + 2 < NB ? x[K][(c + 2) % NB] : T(0));
          }
        }
      }
    }
    if (lane == 0) redv[wid] = bv, redi[wid] = bi;
    __syncthreads();
    int ww;
    {
      T v = lane < NW ? redv[lane] : T(-1);
      int i = lane < NW ? redi[lane] : INT_MAX;
      const int mine = i;
      warp_argmax(v, i);
      ww = __ffs(__ballot_sync(0xffffffffu, i != INT_MAX && mine == i)) - 1;  // the winning warp
      bv = v;
      bi = i;
    }
    // push, one warp per target CTA, one 16-byte store per lane: columns
    // beyond the panel (and the multiplier slots) go out as zeros
    const int ulen = jb - j - 1;
    for (int q = wid; q < C; q += NW) {
      if (lane < NB / VE) {
        const int c = lane * VE;
        T *dst = cluster.map_shared_rank(&mb_row[buf][rank][0], q) + c;
        if constexpr (VE == 4) {
          float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
          if (bi != INT_MAX) s = *reinterpret_cast<const float4 *>(&stage[ww < 0 ? 0 : ww][c]);
          s.x = c < ulen ? s.x : 0.f;
          s.y = c + 1 < ulen ? s.y : 0.f;
          s.z = c + 2 < ulen ? s.z : 0.f;
          s.w = c + 3 < ulen ? s.w : 0.f;
          *reinterpret_cast<float4 *>(dst) = s;
        } else {
          double2 s = make_double2(0.0, 0.0);
          if (bi != INT_MAX) s = *reinterpret_cast<const double2 *>(&stage[ww < 0 ? 0 : ww][c]);
          s.x = c < ulen ? s.x : 0.0;
          s.y = c + 1 < ulen ? s.y : 0.0;
          *reinterpret_cast<double2 *>(dst) = s;
        }
      } else if (lane == NB / VE) {
        *cluster.map_shared_rank(&mb_v[buf][rank], q) = bv;
      } else if (lane == NB / VE + 1) {
        *cluster.map_shared_rank(&mb_i[buf][rank], q) = bi;
      } else if (lane == NB / VE + 2) {
        *cluster.map_shared_rank(&mb_pv[buf][rank], q) = bi != INT_MAX ? stage_pv[ww < 0 ? 0 : ww] : T(0);
      }
    }
    cluster_arrive_release();
    cluster_wait_acquire();
    // the pivot of column j, and the CTA whose mailbox slot holds it
    T v = lane < C ? mb_v[buf][lane] : T(-1);
    int p = lane < C ? mb_i[buf][lane] : INT_MAX;
    const int mine = p;
    warp_argmax(v, p);
    const int w = __ffs(__ballot_sync(0xffffffffu, p != INT_MAX && mine == p)) - 1;
    T pv;
    if (p == INT_MAX) {
      // no finite candidate: keep the sequence a permutation with the lowest
      // not-yet-pivoted supernode row; the factorization reports the failure
      if (tid == 0 && rank == 0) atomicOr(err, 2);
      p = j0;
      bool used = true;
      while (used) {
        used = false;
        for (int q = 0; q < j; ++q)
          if (hist[q] == p) used = true, ++p;
      }
      pv = T(0);
    } else {
      pv = mb_pv[buf][w];
    }
    if (tid == 0) hist[j] = p;
#pragma unroll
    for (int k = 0; k < kRegPanelRows; ++k)
      if (ret[k] == -1 && r_lo + tid + k * nt == p) ret[k] = j;
    if (pv == T(0) && tid == 0 && rank == 0) atomicOr(err, 1);
    const T inv = pv != T(0) ? T(1) / pv : T(0);
    const T *u = &mb_row[buf][w < 0 ? 0 : w][0];  // no pivot: multipliers are 0 anyway
#pragma unroll
    for (int k = 0; k < kRegPanelRows; ++k) {
      if (ret[k] != -1) continue;
      const T l = x[k][0] * inv;
#pragma unroll
      for (int c = 0; c < NB; c += VE) {
        if constexpr (VE == 4) {
          const float4 q = *reinterpret_cast<const float4 *>(u + c);
          x[k][c] = x[k][c + 1] - l * q.x;
          x[k][c + 1] = x[k][c + 2] - l * q.y;
          x[k][c + 2] = x[k][c + 3] - l * q.z;
          if (c + 4 < NB) x[k][c + 3] = x[k][(c + 4) % NB] - l * q.w;
        } else {
          const double2 q = *reinterpret_cast<const double2 *>(u + c);
          x[k][c] = x[k][c + 1] - l * q.x;
          if (c + 2 < NB) x[k][c + 1] = x[k][(c + 2) % NB] - l * q.y;
        }
      }
      x[k][NB - 1] = l;
    }
  }
  // LAPACK's sequential interchanges from the pivot sequence (positions and
  // rows relative to j0); every CTA computes them for its own rows
  for (int r = tid; r < R; r += nt) pos_of[r] = r, at_pos[r] = r, touched[r] = 0;
  __syncthreads();
  if (tid == 0) {
    int n = 0;
    for (int j = 0; j < jb; ++j) {
      const int pr = hist[j] - j0, pp = pos_of[pr];
      if (rank == 0) piv[F.piv_off + j0 + j] = j0 + pp;
      if (pp == j) continue;
      const int rc = at_pos[j];
      at_pos[j] = pr;
      at_pos[pp] = rc;
      pos_of[pr] = j;
      pos_of[rc] = pp;
      if (!touched[j]) touched[j] = 1, lrow[n++] = j;
      if (!touched[pp]) touched[pp] = 1, lrow[n++] = pp;
    }
    for (int q = 0; q < n; ++q) lsrc[q] = at_pos[lrow[q]];
    nswap = n;
    if (rank == 0) {
      int32_t *sw = swaps + int64_t(fi) * (1 + 2 * kMaxSwapRows);
      for (int q = 0; q < n; ++q) sw[1 + q] = j0 + lrow[q], sw[1 + kMaxSwapRows + q] = j0 + lsrc[q];
      sw[0] = n;
    }
  }
  __syncthreads();
  // every row once to its final position: multipliers, and the U part of pivot rows
#pragma unroll
  for (int k = 0; k < kRegPanelRows; ++k) {
    if (ret[k] == -2) continue;
    const int i = tid + k * nt;
    T *dst = A + (j0 + pos_of[r_lo + i - j0]) + int64_t(j0) * ld;
    const int jr = ret[k] >= 0 ? ret[k] : jb;  // columns < jr hold multipliers
#pragma unroll
    for (int s = 0; s < NB; ++s) {
      if (s < jb - jr) dst[int64_t(jr + s) * ld] = x[k][s];            // U: column jr + s
      if (s >= NB - jr) dst[int64_t(s - (NB - jr)) * ld] = x[k][s];     // L: column s - (NB - jr)
    }
  }
  // no CTA exits while another may still read its mailbox
  cluster.sync();
}

template <typename T, int NB>
__global__ void __launch_bounds__(256) k_swap_trsm(const FrontDev *__restrict__ fr, int j0, T *__restrict__ fronts,
                                                   const int32_t *__restrict__ swaps, int part, int w) {
  const FrontDev F = fr[blockIdx.y];
  if (j0 >= F.s) return;
  const int jb = min(NB, F.s - j0);
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  __shared__ T L[NB * NB];
  __shared__ int32_t srow[kMaxSwapRows], ssrc[kMaxSwapRows];
  const int32_t *sw = swaps + int64_t(blockIdx.y) * (1 + 2 * kMaxSwapRows);
  const int nsw = sw[0];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < nsw; i += blockDim.x) srow[i] = sw[1 + i], ssrc[i] = sw[1 + kMaxSwapRows + i];
  for (int i = tid; i < jb * jb; i += blockDim.x) {
    const int r = i % jb, c = i / jb;
    L[r + c * NB] = A[(j0 + r) + int64_t(j0 + c) * ld];
  }
  __syncthreads();
  constexpr int kPer = (kMaxSwapRows + 31) / 32;
  // part 0: every column but the panel's; part 1: the w columns after the
  // panel (what the next panel needs); part 2: the others; part 3 (an inner
  // step of the blocked LU, w = the outer block width): the columns of the
  // panel's outer block [J, min(J + w, s)), J = w floor(j0 / w)
  const int t0 = j0 + jb;
  int c_begin = part == 1 ? t0 : 0, c_end = part == 1 ? min(F.f, t0 + w) : F.f;
  if (part == 3) c_begin = (j0 / w) * w, c_end = min(c_begin + w, F.s);
  for (int c = c_begin + blockIdx.x * 8 + wid; c < c_end; c += gridDim.x * 8) {
    if (c >= j0 && c < t0) continue;
    if (part == 2 && c >= t0 && c < t0 + w) continue;
    T *Ac = A + int64_t(c) * ld;
    if (nsw > 0) {
      T v[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int e = lane + 32 * q;
        if (e < nsw) v[q] = Ac[ssrc[e]];
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int e = lane + 32 * q;
        if (e < nsw) Ac[srow[e]] = v[q];
      }
      __syncwarp();
    }
    if (c >= j0 + jb) {
      T x0 = (lane < jb) ? Ac[j0 + lane] : T(0);
      T x1 = (NB > 32 && lane + 32 < jb) ? Ac[j0 + 32 + lane] : T(0);
      for (int i = 0; i < jb; ++i) {
        const T xi = __shfl_sync(0xffffffffu, i < 32 ? x0 : x1, i & 31);
        if (lane > i && lane < jb) x0 -= L[lane + i * NB] * xi;
        if (NB > 32 && lane + 32 > i && lane + 32 < jb) x1 -= L[lane + 32 + i * NB] * xi;
      }
      if (lane < jb) Ac[j0 + lane] = x0;
      if (NB > 32 && lane + 32 < jb) Ac[j0 + 32 + lane] = x1;
    }
  }
}

// Block end of the blocked FP32 LU for the outer block [J, J + jbo), jbo =
// min(KB, s - J): the block's panels interchanged rows only inside the block,
// so every other column now takes their interchanges (panel by panel, in
// order), and the columns after the block also take U12 = L11^-1 A12 on rows
// [J, J + jbo), L11 the block's unit lower triangle.  A warp takes kBlkCols
// adjacent columns, lane l holding rows J + l + 32 i (i < KB / 32) of each in
// registers; L11 passes through shared memory one 64-column block at a time
// (zero above the diagonal and below row jbo, so the updates need no row
// tests), each value read once for all the warp's columns.
// trsm = 1: columns [t0 + c_lo, t0 + c_hi) clipped to f (t0 = J + jbo);
// trsm = 0: interchanges only, columns [c_lo, min(c_hi, J)).
constexpr int kBlkCols = 4;                    // columns per warp
constexpr int kBlkCtaCols = 8 * kBlkCols;      // columns per CTA (eight warps)
template <int KB>
__global__ void __launch_bounds__(256, 3) k_blk_swap_trsm(const FrontDev *__restrict__ fr, int J, float *__restrict__ fronts,
                                                      const int32_t *__restrict__ swaps, int64_t swap_stride, int c_lo,
                                                      int c_hi, int trsm) {
  static_assert(KB % 64 == 0 && KB <= 256, "outer block");
  constexpr int NR = KB / 32;
  constexpr int CW = kBlkCols;
  const int fi = blockIdx.y;
  const FrontDev F = fr[fi];
  if (J >= F.s) return;
  const int jbo = min(KB, F.s - J);
  const int t0 = J + jbo;
  float *A = fronts + F.off;
  const int64_t ld = F.ld;
  int lo, hi;
  if (trsm) {
    if (c_lo >= F.f - t0) return;
    lo = t0 + c_lo;
    hi = c_hi >= F.f - t0 ? F.f : t0 + c_hi;
  } else {
    lo = c_lo;
    hi = min(c_hi, J);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lo + int(blockIdx.x) * kBlkCtaCols >= hi) return;  // uniform over the CTA
  const int cw = lo + blockIdx.x * kBlkCtaCols + warp * CW;  // this warp's first column
  const int npan = (jbo + 63) / 64;
  constexpr int kPer = (kMaxSwapRows + 31) / 32;
  // one gather and one scatter round per panel for all the warp's columns
  const int ncw = max(0, min(CW, hi - cw));
  for (int i = 0; i < npan; ++i) {
    const int32_t *sw = swaps + int64_t(((J / 64) + i) & 7) * swap_stride + int64_t(fi) * (1 + 2 * kMaxSwapRows);
    const int n = sw[0];
    if (n <= 0) continue;
    int srow[kPer], ssrc[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = lane + 32 * q;
      srow[q] = e < n ? sw[1 + e] : 0;
      ssrc[q] = e < n ? sw[1 + kMaxSwapRows + e] : 0;
    }
    float v[CW][kPer];
#pragma unroll
    for (int j = 0; j < CW; ++j)
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (j < ncw && lane + 32 * q < n) v[j][q] = A[ssrc[q] + int64_t(cw + j) * ld];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < CW; ++j)
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (j < ncw && lane + 32 * q < n) A[srow[q] + int64_t(cw + j) * ld] = v[j][q];
    __syncwarp();
  }
  if (!trsm) return;
  extern __shared__ float Ls[];  // [64][KB]: column kl of the current 64-column block of L11, rows 0..KB-1
  float x[CW][NR];
#pragma unroll
  for (int j = 0; j < CW; ++j)
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int row = 32 * i + lane;
      x[j][i] = (cw + j < hi && row < jbo) ? A[(J + row) + int64_t(cw + j) * ld] : 0.f;
    }
#pragma unroll
  for (int b = 0; b < KB / 64; ++b) {
    if (b >= npan) break;  // uniform
    const int kb0 = 64 * b, kbn = min(64, jbo - kb0);
    __syncthreads();  // the previous block of L11 has been used
    for (int e = threadIdx.x; e < 64 * KB; e += blockDim.x) {
      const int kl = e / KB, row = e % KB;
      Ls[e] = (kl < kbn && row > kb0 + kl && row < jbo) ? A[(J + row) + int64_t(J + kb0 + kl) * ld] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      for (int kl2 = 0; kl2 < 32; ++kl2) {
        const int kl = 32 * h + kl2;
        if (kl >= kbn) break;  // uniform
        float xk[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) xk[j] = __shfl_sync(0xffffffffu, x[j][2 * b + h], kl2);
        const float *Lk = Ls + kl * KB + lane;
#pragma unroll
        for (int i = 2 * b + h; i < NR; ++i) {
          const float l = Lk[32 * i];
#pragma unroll
          for (int j = 0; j < CW; ++j) x[j][i] -= l * xk[j];
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < CW; ++j) {
    if (cw + j >= hi) break;
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int row = 32 * i + lane;
      if (row < jbo) A[(J + row) + int64_t(cw + j) * ld] = x[j][i];
    }
  }
}

// trailing update: A[t0:f, t0:f] -= A[t0:f, j0:j0+jb] * A[j0:j0+jb, t0:f], t0 = j0 + jb.
// Thread (tr, tc) owns rows tr + RT*i and columns tc + CT*j of the tile, so a
// warp touches consecutive rows of C (coalesced).  The operand tiles are
// stored permuted in shared memory -- row tr + RT*i of the A tile at
// tr*TM + i -- so each thread reads its TM (TN) values as 16-byte vectors.
// The C tile is prefetched into the accumulators while the operands are staged.
// sym = 1 (block Cholesky): only tiles that reach the lower triangle, and the
// B operand is L21^T, read from the panel columns of the rows [t0, f).
template <typename T, int BM, int BN, int TM, int TN, int NB>
__global__ void __launch_bounds__(256) k_gemm_update(const FrontDev *__restrict__ fr, int j0, T *__restrict__ fronts,
                                                     int c_lo, int c_hi, int sym) {
  constexpr int RT = BM / TM, CT = BN / TN;  // thread grid over the tile (rows fastest)
  constexpr int PA = BM + 16 / int(sizeof(T)), PB = BN + 16 / int(sizeof(T));  // padded rows, 16-byte aligned
  constexpr int VA = 16 / int(sizeof(T));    // elements per 16-byte vector
  const FrontDev F = fr[blockIdx.z];
  if (j0 >= F.s) return;
  const int jb = min(NB, F.s - j0);
  const int t0 = j0 + jb;
  const int nrest = F.f - t0;
  const int ncol = min(nrest, c_hi);  // trailing columns [c_lo, ncol) of this launch
  const int rb = blockIdx.y * BM, cb = c_lo + blockIdx.x * BN;
  if (rb >= nrest || cb >= ncol) return;
  if (sym && cb >= rb + BM) return;  // strictly above the diagonal
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sA = reinterpret_cast<T *>(smraw);  // [NB][PA]
  T *sB = sA + NB * PA;                   // [NB][PB]
  const int tid = threadIdx.x;
  const int tr = tid % RT, tc = tid / RT;
  T acc[TM][TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int c = cb + tc + CT * j;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int r = rb + tr + RT * i;
      acc[i][j] = (c < ncol && r < nrest) ? A[(t0 + r) + int64_t(t0 + c) * ld] : T(0);
    }
  }
  // operand tiles: all loads of a pass are issued before any store (fixed trip counts)
  constexpr int kIA = NB * BM / 256, kIB = NB * BN / 256;
  {
    T v[kIA];
#pragma unroll
    for (int it = 0; it < kIA; ++it) {
      const int e = tid + it * 256;
      const int i = e % BM, k = e / BM;  // tile row i = (i % RT) + RT * (i / RT)
      const int r = rb + i;
      v[it] = (k < jb && r < nrest) ? A[(t0 + r) + int64_t(j0 + k) * ld] : T(0);
    }
#pragma unroll
    for (int it = 0; it < kIA; ++it) {
      const int e = tid + it * 256;
      const int i = e % BM, k = e / BM;
      sA[k * PA + (i % RT) * TM + i / RT] = v[it];
    }
  }
  {
    T v[kIB];
#pragma unroll
    for (int it = 0; it < kIB; ++it) {
      const int e = tid + it * 256;
      // U12 rows (K contiguous), or L21 rows (columns of the tile contiguous)
      const int k = sym ? e / BN : e % NB, j = sym ? e % BN : e / NB;
      const int c = cb + j;
      v[it] = (k < jb && c < ncol) ? (sym ? A[(t0 + c) + int64_t(j0 + k) * ld] : A[(j0 + k) + int64_t(t0 + c) * ld])
                                   : T(0);
    }
#pragma unroll
    for (int it = 0; it < kIB; ++it) {
      const int e = tid + it * 256;
      const int k = sym ? e / BN : e % NB, j = sym ? e % BN : e / NB;
      sB[k * PB + (j % CT) * TN + j / CT] = v[it];
    }
  }
  __syncthreads();
  for (int k = 0; k < jb; ++k) {
    T a[TM], b[TN];
    const T *pa = sA + k * PA + tr * TM;
    const T *pb = sB + k * PB + tc * TN;
#pragma unroll
    for (int v = 0; v < TM; v += VA) {
      if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(pa + v);
        a[v] = q.x, a[v + 1] = q.y, a[v + 2] = q.z, a[v + 3] = q.w;
      } else {
        const double2 q = *reinterpret_cast<const double2 *>(pa + v);
        a[v] = q.x, a[v + 1] = q.y;
      }
    }
#pragma unroll
    for (int v = 0; v < TN; v += VA) {
      if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(pb + v);
        b[v] = q.x, b[v + 1] = q.y, b[v + 2] = q.z, b[v + 3] = q.w;
      } else {
        const double2 q = *reinterpret_cast<const double2 *>(pb + v);
        b[v] = q.x, b[v + 1] = q.y;
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] -= a[i] * b[j];
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int c = cb + tc + CT * j;
    if (c >= ncol) continue;
    T *Cc = A + int64_t(t0 + c) * ld + t0;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int r = rb + tr + RT * i;
      if (r < nrest) Cc[r] = acc[i][j];
    }
  }
}

template <typename T>
__global__ void k_extend_add(const FrontDev *__restrict__ fr_all, int lo, const int32_t *__restrict__ map,
                             T *__restrict__ fronts, int lower) {
  const FrontDev F = fr_all[lo + blockIdx.z];
  if (F.parent < 0 || F.b == 0) return;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  if (i0 >= F.b || j0 >= F.b || (lower && i0 + 31 < j0)) return;
  const FrontDev P = fr_all[F.parent];
  const int32_t *mp = map + F.map_off;
  const T *C = fronts + F.off + int64_t(F.s) * F.ld + F.s;
  T *Pa = fronts + P.off;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int i = i0 + (e & 31), j = j0 + (e >> 5);
    if (i < F.b && j < F.b && (!lower || i >= j)) atomicAdd(&Pa[mp[i] + int64_t(mp[j]) * P.ld], C[i + int64_t(j) * F.ld]);
  }
}

__global__ void k_make_perm(const FrontDev *__restrict__ fr, const int32_t *__restrict__ piv, int32_t *__restrict__ perm,
                            int smem_cap) {
  const FrontDev F = fr[blockIdx.x];
  extern __shared__ int32_t sp[];
  int32_t *P = perm + F.piv_off;
  const int32_t *pv = piv + F.piv_off;
  const bool sm = F.s <= smem_cap;
  int32_t *W = sm ? sp : P;
  for (int i = threadIdx.x; i < F.s; i += blockDim.x) W[i] = i;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = 0; j < F.s; ++j) {
      const int p = pv[j];
      if (p != j) {
        const int32_t t = W[j];
        W[j] = W[p];
        W[p] = t;
      }
    }
  __syncthreads();
  if (sm)
    for (int i = threadIdx.x; i < F.s; i += blockDim.x) P[i] = W[i];
}

// ---------------- triangular solves ----------------
constexpr int kBS = kSolveBlock;
constexpr int kMaxRhs = 16;
constexpr int kRowsPerCta = 128;

template <typename T>
__global__ void k_fwd_gather(const FrontDev *__restrict__ fr, const int32_t *__restrict__ perm,
                             const int32_t *__restrict__ idx, const T *__restrict__ y, int64_t ldy, int nrhs,
                             T *__restrict__ work, const int64_t *__restrict__ work_off, int lo) {
  const FrontDev F = fr[blockIdx.y];
  T *W = work + work_off[lo + blockIdx.y];
  const int32_t *ix = idx + F.idx_off;
  const int32_t *pm = perm + F.piv_off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F.f; i += gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; ++r) W[i + int64_t(r) * F.f] = (i < F.s) ? y[ix[pm[i]] + r * ldy] : T(0);
}

template <typename T>
__global__ void k_fwd_scatter(const FrontDev *__restrict__ fr, const int32_t *__restrict__ idx, T *__restrict__ y,
                              int64_t ldy, int nrhs, const T *__restrict__ work, const T *__restrict__ zbuf,
                              const int64_t *__restrict__ work_off, int lo) {
  const FrontDev F = fr[blockIdx.y];
  const T *W = work + work_off[lo + blockIdx.y];
  const T *Z = zbuf + work_off[lo + blockIdx.y];
  const int32_t *ix = idx + F.idx_off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F.f; i += gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; ++r) {
      if (i < F.s)
        y[ix[i] + r * ldy] = Z[i + int64_t(r) * F.f];
      else
        atomicAdd(&y[ix[i] + r * ldy], W[i + int64_t(r) * F.f]);
    }
}

// Inverses of the kBS x kBS diagonal blocks of L11 (unit lower) and U11
// (upper) of every front, so that each column-block step of a triangular
// solve is a dense product instead of a sequential substitution.
template <typename T>
__global__ void __launch_bounds__(kBS) k_invert_diag(const FrontDev *__restrict__ fr, const T *__restrict__ fronts,
                                                     T *__restrict__ dinv) {
  const FrontDev F = fr[blockIdx.y];
  const int q = blockIdx.x;
  const int c0 = q * kBS;
  if (c0 >= F.s) return;
  const int cb = min(kBS, F.s - c0);
  __shared__ T D[kBS * kBS];
  const T *A = fronts + F.off;
  for (int e = threadIdx.x; e < cb * cb; e += blockDim.x) {
    const int r = e % cb, c = e / cb;
    D[r + c * kBS] = A[(c0 + r) + int64_t(c0 + c) * F.ld];
  }
  __syncthreads();
  T *Li = dinv + F.dinv_off + int64_t(q) * 2 * kBS * kBS;
  T *Ui = Li + kBS * kBS;
  const int c = threadIdx.x;  // one column of each inverse per thread
  if (c < cb) {
    // L X = e_c (unit lower): rows c.. cb-1
    for (int r = 0; r < c; ++r) Li[r + c * kBS] = T(0);
    Li[c + c * kBS] = T(1);
    for (int r = c + 1; r < cb; ++r) {
      T acc = T(0);
      for (int k = c; k < r; ++k) acc += D[r + k * kBS] * Li[k + c * kBS];
      Li[r + c * kBS] = -acc;
    }
    // U X = e_c (upper): rows c down to 0
    for (int r = cb - 1; r > c; --r) Ui[r + c * kBS] = T(0);
    Ui[c + c * kBS] = T(1) / D[c + c * kBS];
    for (int r = c - 1; r >= 0; --r) {
      T acc = T(0);
      for (int k = r + 1; k <= c; ++k) acc += D[r + k * kBS] * Ui[k + c * kBS];
      Ui[r + c * kBS] = -acc / D[r + r * kBS];
    }
  }
}

// x = Dinv (cb x cb) * W[c0:c0+cb] into shared memory (every CTA of the step computes it)
template <typename T>
__device__ void diag_apply(const T *Dinv, const T *W, int64_t ldw, int c0, int cb, int nrhs, T *sD, T *sW, T *sX) {
  const int tid = threadIdx.x;
  for (int e = tid; e < kBS * kBS; e += blockDim.x) sD[e] = Dinv[e];
  for (int e = tid; e < cb * nrhs; e += blockDim.x) {
    const int r = e % cb, c = e / cb;
    sW[r + c * kBS] = W[(c0 + r) + int64_t(c) * ldw];
  }
  __syncthreads();
  for (int e = tid; e < cb * nrhs; e += blockDim.x) {
    const int r = e % cb, c = e / cb;
    T acc = T(0);
#pragma unroll 8
    for (int k = 0; k < cb; ++k) acc += sD[r + k * kBS] * sW[k + c * kBS];
    sX[r + c * kBS] = acc;
  }
  __syncthreads();
}

// rows [row0, min(row0 + kStepRows, r_hi)) of W -= A[rows, c0:c0+cb] * sX.
// Four threads share a row, each a quarter of the cb columns; the partial sums
// meet in shared memory (sRed may alias the inverted block, no longer needed).
constexpr int kStepThreads = 256, kStepRows = 64;
template <typename T>
__device__ void slab_update(const T *A, int64_t ld, T *W, int64_t ldw, int row0, int r_hi, int c0, int cb, int nrhs,
                            const T *sX, T *sRed) {
  const int tid = threadIdx.x;
  const int rl = tid % kStepRows, qq = tid / kStepRows;
  const int r = row0 + rl;
  constexpr int kQ = kBS / (kStepThreads / kStepRows);
  const int q0 = qq * kQ, q1 = min(cb, q0 + kQ);
  T acc[kMaxRhs];
#pragma unroll
  for (int c = 0; c < kMaxRhs; ++c) acc[c] = T(0);
  if (r < r_hi) {
#pragma unroll 4
    for (int q = q0; q < q1; ++q) {
      const T a = A[r + int64_t(c0 + q) * ld];
#pragma unroll
      for (int c = 0; c < kMaxRhs; ++c)
        if (c < nrhs) acc[c] += a * sX[q + c * kBS];
    }
  }
  __syncthreads();  // sRed aliases the inverted block: every thread is done with it
#pragma unroll
  for (int c = 0; c < kMaxRhs; ++c)
    if (c < nrhs) sRed[(qq * kStepRows + rl) * kMaxRhs + c] = acc[c];
  __syncthreads();
  if (qq == 0 && r < r_hi)
    for (int c = 0; c < nrhs; ++c) {
      T t = T(0);
#pragma unroll
      for (int g = 0; g < kStepThreads / kStepRows; ++g) t += sRed[(g * kStepRows + rl) * kMaxRhs + c];
      W[r + int64_t(c) * ldw] -= t;
    }
}

// forward step of column block [c0, c0+cb): x = Linv W_c0 -> Z; rows below -= L x
template <typename T>
__global__ void __launch_bounds__(kStepThreads) k_fwd_step(const FrontDev *__restrict__ fr, int c0,
                                                           const T *__restrict__ fronts, const T *__restrict__ dinv,
                                                           int nrhs, T *__restrict__ work, T *__restrict__ zbuf,
                                                           const int64_t *__restrict__ work_off, int lo) {
  const FrontDev F = fr[blockIdx.y];
  if (c0 >= F.s) return;
  const int cb = min(kBS, F.s - c0);
  const int r0 = c0 + cb + int(blockIdx.x) * kStepRows;
  if (blockIdx.x > 0 && r0 >= F.f) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sD = reinterpret_cast<T *>(smraw);
  T *sW = sD + kBS * kBS, *sX = sW + kBS * kMaxRhs;
  T *W = work + work_off[lo + blockIdx.y];
  const T *Li = dinv + F.dinv_off + int64_t(c0 / kBS) * 2 * kBS * kBS;
  diag_apply<T>(Li, W, F.f, c0, cb, nrhs, sD, sW, sX);
  if (blockIdx.x == 0) {
    T *Z = zbuf + work_off[lo + blockIdx.y];
    for (int e = threadIdx.x; e < cb * nrhs; e += blockDim.x) {
      const int r = e % cb, c = e / cb;
      Z[(c0 + r) + int64_t(c) * F.f] = sX[r + c * kBS];
    }
  }
  slab_update<T>(fronts + F.off, F.ld, W, F.f, r0, F.f, c0, cb, nrhs, sX, sD);
}

// backward step of column block [c0, c0+cb): x = Uinv W_c0 -> Z; rows above -= U x
template <typename T>
__global__ void __launch_bounds__(kStepThreads) k_bwd_step(const FrontDev *__restrict__ fr, int c0,
                                                           const T *__restrict__ fronts, const T *__restrict__ dinv,
                                                           int nrhs, T *__restrict__ work, T *__restrict__ zbuf,
                                                           const int64_t *__restrict__ work_off, int lo) {
  const FrontDev F = fr[blockIdx.y];
  if (c0 >= F.s) return;
  const int cb = min(kBS, F.s - c0);
  const int r0 = int(blockIdx.x) * kStepRows;
  if (blockIdx.x > 0 && r0 >= c0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sD = reinterpret_cast<T *>(smraw);
  T *sW = sD + kBS * kBS, *sX = sW + kBS * kMaxRhs;
  T *W = work + work_off[lo + blockIdx.y];
  const T *Ui = dinv + F.dinv_off + int64_t(c0 / kBS) * 2 * kBS * kBS + kBS * kBS;
  diag_apply<T>(Ui, W, F.f, c0, cb, nrhs, sD, sW, sX);
  if (blockIdx.x == 0) {
    T *Z = zbuf + work_off[lo + blockIdx.y];
    for (int e = threadIdx.x; e < cb * nrhs; e += blockDim.x) {
      const int r = e % cb, c = e / cb;
      Z[(c0 + r) + int64_t(c) * F.f] = sX[r + c * kBS];
    }
  }
  slab_update<T>(fronts + F.off, F.ld, W, F.f, r0, c0, c0, cb, nrhs, sX, sD);
}

// The rectangular products of the sweeps that do not lie on the block chain:
//   mode 0 (backward, before the sweep): W[0:s]  -= U12 W[s:f]   (U12 = rows [0, s), columns [s, f))
//   mode 1 (forward, after the sweep):   W[s:f]  -= L21 Z[0:s]   (L21 = rows [s, f), columns [0, s))
// Two output rows per thread and a 256-wide K chunk per CTA (blockIdx.y).
// The chunk's X values are staged in shared memory with the right-hand sides
// of one k contiguous, so a thread reads them as 16-byte vectors shared by its
// two rows; eight matrix loads per row are in flight.  Partial sums over the
// chunks are added atomically.
constexpr int kU12Chunk = 256;
constexpr int kRectRows = 2 * kRowsPerCta;  // output rows per CTA
template <typename T>
__global__ void __launch_bounds__(kRowsPerCta) k_rect_update(const FrontDev *__restrict__ fr, const T *__restrict__ fronts,
                                                             int nrhs, T *__restrict__ work, const T *__restrict__ zbuf,
                                                             const int64_t *__restrict__ work_off, int lo, int mode) {
  constexpr int VE = 16 / int(sizeof(T));  // right-hand sides per 16-byte vector
  const FrontDev F = fr[blockIdx.z];
  const int r_lo = mode ? F.s : 0, r_hi = mode ? F.f : F.s;
  const int kk_lo = mode ? 0 : F.s, kk_hi = mode ? F.s : F.f;
  const int k_lo = kk_lo + int(blockIdx.y) * kU12Chunk;
  const int rb = r_lo + int(blockIdx.x) * kRectRows;
  if (F.b == 0 || rb >= r_hi || k_lo >= kk_hi) return;
  const int k_hi = min(kk_hi, k_lo + kU12Chunk);
  __shared__ __align__(16) T sX[kU12Chunk * kMaxRhs];  // sX[q * kMaxRhs + c]
  T *W = work + work_off[lo + blockIdx.z];
  const T *X = (mode ? zbuf : work) + work_off[lo + blockIdx.z];
  const int kb = k_hi - k_lo;
  for (int e = threadIdx.x; e < kU12Chunk * kMaxRhs; e += blockDim.x) {
    const int q = e % kU12Chunk, c = e / kU12Chunk;
    sX[q * kMaxRhs + c] = (q < kb && c < nrhs) ? X[(k_lo + q) + int64_t(c) * F.f] : T(0);
  }
  __syncthreads();
  const int r0 = rb + int(threadIdx.x), r1 = r0 + kRowsPerCta;
  if (r0 >= r_hi) return;
  const bool has1 = r1 < r_hi;
  T acc0[kMaxRhs], acc1[kMaxRhs];
#pragma unroll
  for (int c = 0; c < kMaxRhs; ++c) acc0[c] = acc1[c] = T(0);
  const T *A0 = fronts + F.off + r0;
  const T *A1 = fronts + F.off + (has1 ? r1 : r0);
  constexpr int U = 8;
  for (int q0 = 0; q0 < kb; q0 += U) {
    T a0[U], a1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool in = q0 + u < kb;
      a0[u] = in ? A0[int64_t(k_lo + q0 + u) * F.ld] : T(0);
      a1[u] = (in && has1) ? A1[int64_t(k_lo + q0 + u) * F.ld] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const T *xq = sX + (q0 + u) * kMaxRhs;
#pragma unroll
      for (int c = 0; c < kMaxRhs; c += VE) {
        T xv[VE];
        if constexpr (VE == 4) {
          const float4 v = *reinterpret_cast<const float4 *>(xq + c);
          xv[0] = v.x, xv[1] = v.y, xv[2] = v.z, xv[3] = v.w;
        } else {
          const double2 v = *reinterpret_cast<const double2 *>(xq + c);
          xv[0] = v.x, xv[1] = v.y;
        }
#pragma unroll
        for (int j = 0; j < VE; ++j) {
          acc0[c + j] += a0[u] * xv[j];
          acc1[c + j] += a1[u] * xv[j];
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kMaxRhs; ++c)
    if (c < nrhs) {
      atomicAdd(&W[r0 + int64_t(c) * F.f], -acc0[c]);
      if (has1) atomicAdd(&W[r1 + int64_t(c) * F.f], -acc1[c]);
    }
}

template <typename T>
__global__ void k_bwd_gather(const FrontDev *__restrict__ fr, const int32_t *__restrict__ idx, const T *__restrict__ y,
                             int64_t ldy, int nrhs, T *__restrict__ work, const int64_t *__restrict__ work_off, int lo) {
  const FrontDev F = fr[blockIdx.y];
  T *W = work + work_off[lo + blockIdx.y];
  const int32_t *ix = idx + F.idx_off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F.f; i += gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; ++r) W[i + int64_t(r) * F.f] = y[ix[i] + r * ldy];
}

template <typename T>
__global__ void k_bwd_scatter(const FrontDev *__restrict__ fr, const int32_t *__restrict__ idx, T *__restrict__ y,
                              int64_t ldy, int nrhs, const T *__restrict__ zbuf, const int64_t *__restrict__ work_off,
                              int lo) {
  const FrontDev F = fr[blockIdx.y];
  const T *W = zbuf + work_off[lo + blockIdx.y];
  const int32_t *ix = idx + F.idx_off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F.s; i += gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; ++r) y[ix[i] + r * ldy] = W[i + int64_t(r) * F.f];
}

inline int cdiv(int64_t a, int64_t b) { return int((a + b - 1) / b); }

inline int num_sms() { return device_sms(); }


// ---------------- flag-synchronised block sweeps ----------------
// One launch per elimination level and direction replaces the kBS-column
// step launches.  Work items are row blocks: (front, b) for the supernode
// rows of kBS-row blocks b and b+1 (forward) or b and b-1 (backward), and in
// the forward sweep (front, -(q+1)) for the q-th kBS-row block of the
// boundary rows.  A CTA takes items in ticket order and accumulates,
// left-looking, the contributions of the solution blocks it depends on as
// their flags appear:
//   forward,  block b : w_b -= sum_{b' < b} L[b, b'] z_{b'},  z_b = L_bb^-1 w_b
//   boundary, block q : w_q -= sum_{b'}    L[q, b'] z_{b'}   (added to y later)
//   backward, block b : w_b -= sum_{b' > b} U[b, b'] x_{b'},  x_b = U_bb^-1 w_b
// The two blocks of an item share the external contributions; the second
// then takes the first's solution inside the CTA, so a hop between CTAs
// (flag, release / acquire, reload) happens once per two blocks.  Each block
// is published as soon as it is solved (release store of the launch's
// epoch).  An item depends only on items with smaller tickets, which are held
// by running or finished CTAs of the same cooperative launch, so every wait
// ends; each wait is still bounded (ChainArgs::spin_cap polls, 2^22 unless
// the handle sets another), after which the CTA raises an error flag and
// leaves.
constexpr int kChainThreads = 256;
constexpr int kChainSub = 2;                          // row blocks per supernode item
constexpr int kChainPre = kBS * kBS / kChainThreads;  // values of one 64 x 64 block per thread

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// bounded wait of thread 0 for flag == epoch (at most spin_cap polls); the
// verdict is shared through *s_ok
__device__ __forceinline__ bool chain_wait(const int *flag, int epoch, uint32_t spin_cap, int *err, int *s_ok) {
  if (threadIdx.x == 0) {
    int okv = 1;
    uint32_t n = 0;
    while (ld_acquire_gpu(flag) != epoch) {
      if (++n > spin_cap) {
        okv = 0;
        atomicOr(err, 4);
        break;
      }
      __nanosleep(32);
    }
    *s_ok = okv;
  }
  __syncthreads();
  return *s_ok != 0;
}

template <typename T, bool Fwd>
__global__ void __launch_bounds__(kChainThreads) k_chain(const FrontDev *__restrict__ fr, const int2 *__restrict__ items,
                                                         int nitems, int *__restrict__ ticket,
                                                         const T *__restrict__ fronts, const T *__restrict__ dinv,
                                                         int nrhs, T *__restrict__ work, T *__restrict__ zbuf,
                                                         const int64_t *__restrict__ work_off, int *__restrict__ flags,
                                                         int epoch, int *__restrict__ err, int wait_epoch,
                                                         uint32_t spin_cap) {
  __shared__ __align__(16) T sL[kChainSub * kBS * kBS];  // blocks of L / U for both sub-blocks, column-major
  __shared__ __align__(16) T sZ[kBS * kMaxRhs];           // a solution block, sZ[k * kMaxRhs + c]
  __shared__ int s_item, s_ok;
  const int tid = threadIdx.x, row = tid & (kBS - 1), g = tid >> 6;  // right-hand sides g, g+4, g+8, g+12
  for (;;) {
    __syncthreads();  // s_item, sL, sZ free
    if (tid == 0) s_item = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_item;
    if (t >= nitems) return;
    const int2 it = items[t];
    const FrontDev F = fr[it.x];
    const T *A = fronts + F.off;
    T *W = work + work_off[it.x];
    T *Z = zbuf + work_off[it.x];
    const int64_t lda = F.ld, ld = F.f;  // front matrix / work vectors
    const bool sn = it.y >= 0;
    const int nbs = (F.s + kBS - 1) / kBS;
    const int fbase = int(F.dinv_off / (2 * kBS * kBS));
    // the item's row blocks: sub u is block blk[u] (boundary items: one block of boundary rows)
    int nsub, blk[kChainSub], r0[kChainSub], rb[kChainSub];
    if (sn) {
      nsub = Fwd ? min(kChainSub, nbs - it.y) : min(kChainSub, it.y + 1);
#pragma unroll
      for (int u = 0; u < kChainSub; ++u) {
        blk[u] = Fwd ? it.y + u : it.y - u;
        r0[u] = blk[u] * kBS;
        rb[u] = u < nsub ? min(kBS, F.s - r0[u]) : 0;
      }
    } else {
      nsub = 1;
      blk[0] = -1;
      r0[0] = F.s + (-it.y - 1) * kBS;
      rb[0] = min(kBS, F.f - r0[0]);
#pragma unroll
      for (int u = 1; u < kChainSub; ++u) blk[u] = -1, r0[u] = 0, rb[u] = 0;
    }
    // external dependencies, in the order they are published
    const int b_first = Fwd ? 0 : nbs - 1;
    const int nblk = Fwd ? (sn ? it.y : nbs) : (nbs - 1 - it.y);
    T acc[kChainSub][4];
#pragma unroll
    for (int u = 0; u < kChainSub; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = g + 4 * q;
        acc[u][q] = (row < rb[u] && c < nrhs) ? W[(r0[u] + row) + int64_t(c) * ld] : T(0);
      }
    T pre[kChainSub][kChainPre];
    auto load_block = [&](int bp) {
      const int c0 = bp * kBS, kb = min(kBS, F.s - c0);
#pragma unroll
      for (int u = 0; u < kChainSub; ++u)
#pragma unroll
        for (int e = 0; e < kChainPre; ++e) {
          const int idx = tid + e * kChainThreads, k = idx / kBS, rr = idx % kBS;
          pre[u][e] = (rr < rb[u] && k < kb) ? A[(r0[u] + rr) + int64_t(c0 + k) * lda] : T(0);
        }
    };
    // the item's own inverted diagonal blocks and the block coupling its two
    // sub-blocks do not depend on any other item: request them now, so that
    // they are not on the chain's critical path
    T preD[kChainSub][kChainPre], preI[kChainPre];
    if (sn) {
#pragma unroll
      for (int u = 0; u < kChainSub; ++u) {
        const T *Di = dinv + F.dinv_off + int64_t(max(blk[u], 0)) * 2 * kBS * kBS + (Fwd ? 0 : kBS * kBS);
#pragma unroll
        for (int e = 0; e < kChainPre; ++e) {
          const int idx = tid + e * kChainThreads, rr = idx % kBS, k = idx / kBS;
          preD[u][e] = (u < nsub && rr < rb[u] && k < rb[u]) ? Di[rr + k * kBS] : T(0);
        }
      }
      const int c0 = max(blk[0], 0) * kBS;
#pragma unroll
      for (int e = 0; e < kChainPre; ++e) {
        const int idx = tid + e * kChainThreads, k = idx / kBS, rr = idx % kBS;
        preI[e] = (nsub > 1 && rr < rb[1] && k < rb[0]) ? A[(r0[1] + rr) + int64_t(c0 + k) * lda] : T(0);
      }
    }
    bool ok = true;
    if (nblk > 0) load_block(b_first);
    for (int s = 0; s < nblk; ++s) {
      const int bp = Fwd ? s : nbs - 1 - s;
      __syncthreads();  // the previous block's sL / sZ are consumed
#pragma unroll
      for (int u = 0; u < kChainSub; ++u)
#pragma unroll
        for (int e = 0; e < kChainPre; ++e) sL[u * kBS * kBS + tid + e * kChainThreads] = pre[u][e];
      if (s + 1 < nblk) load_block(Fwd ? bp + 1 : bp - 1);  // in flight during the wait
      if (!chain_wait(&flags[fbase + bp], wait_epoch, spin_cap, err, &s_ok)) {
        ok = false;
        break;
      }
      const int kb = min(kBS, F.s - bp * kBS);
      for (int e = tid; e < kBS * kMaxRhs; e += kChainThreads) {
        const int k = e % kBS, c = e / kBS;
        sZ[k * kMaxRhs + c] = (k < kb && c < nrhs) ? __ldcg(&Z[(bp * kBS + k) + int64_t(c) * ld]) : T(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < kBS; ++k) {
        T a[kChainSub];
#pragma unroll
        for (int u = 0; u < kChainSub; ++u) a[u] = sL[u * kBS * kBS + k * kBS + row];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T z = sZ[k * kMaxRhs + g + 4 * q];
#pragma unroll
          for (int u = 0; u < kChainSub; ++u) acc[u][q] -= a[u] * z;
        }
      }
    }
    if (!ok) return;  // uniform: every thread saw s_ok == 0
    if (!sn) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = g + 4 * q;
        if (row < rb[0] && c < nrhs) W[(r0[0] + row) + int64_t(c) * ld] = acc[0][q];
      }
      continue;
    }
    // the item's own blocks: solve, publish, and hand the solution to the next sub-block
#pragma unroll
    for (int u = 0; u < kChainSub; ++u) {
      if (u >= nsub) break;
      if (u > 0) {
        // acc[u] -= (L or U)[block u, block u-1] * (solution of block u-1, still in sZ)
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kChainPre; ++e) sL[tid + e * kChainThreads] = preI[e];
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kBS; ++k) {
          const T a = sL[k * kBS + row];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[u][q] -= a * sZ[k * kMaxRhs + g + 4 * q];
        }
      }
      // x = D^-1 w with the inverted kBS x kBS block
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kChainPre; ++e) sL[tid + e * kChainThreads] = preD[u][e];
#pragma unroll
      for (int q = 0; q < 4; ++q) sZ[row * kMaxRhs + g + 4 * q] = row < rb[u] ? acc[u][q] : T(0);
      __syncthreads();
      T x[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
      for (int k = 0; k < kBS; ++k) {
        const T a = sL[k * kBS + row];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] += a * sZ[k * kMaxRhs + g + 4 * q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = g + 4 * q;
        if (row < rb[u] && c < nrhs) Z[(r0[u] + row) + int64_t(c) * ld] = x[q];
      }
      __syncthreads();  // every Z store issued; sZ free
      if (tid == 0) {
        __threadfence();
        st_release_gpu(&flags[fbase + blk[u]], epoch);
      }
      // keep this block's solution in sZ for the next sub-block
#pragma unroll
      for (int q = 0; q < 4; ++q) sZ[row * kMaxRhs + g + 4 * q] = row < rb[u] ? x[q] : T(0);
    }
  }
}

template <typename T, bool Fwd>
int chain_grid(int nitems) {
  static int per_sm = -1;
  if (per_sm < 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chain<T, Fwd>, kChainThreads, 0) != cudaSuccess || n <= 0)
      n = 1;
    per_sm = n;
    cudaGetLastError();
  }
  return std::max(1, std::min(nitems, per_sm * num_sms()));
}

template <typename T, bool Fwd>
cudaError_t launch_chain(const FrontDev *fr, const ChainArgs &ca, int li, const T *fronts, const T *dinv, int nrhs,
                         T *work, T *zbuf, const int64_t *work_off, cudaStream_t s) {
  const int off = Fwd ? ca.fwd_off[li] : ca.bwd_off[li];
  const int n = Fwd ? ca.fwd_n[li] : ca.bwd_n[li];
  if (n == 0) return cudaSuccess;
  const int2 *items = ca.items + off;
  int *ticket = ca.tickets + 2 * li + (Fwd ? 0 : 1);
  int epoch = ca.epoch, wait_epoch = ca.wait_epoch;
  uint32_t spin_cap = ca.spin_cap;
  void *args[] = {(void *)&fr, (void *)&items, (void *)&n, (void *)&ticket, (void *)&fronts, (void *)&dinv,
                  (void *)&nrhs, (void *)&work, (void *)&zbuf, (void *)&work_off, (void *)&ca.flags, (void *)&epoch,
                  (void *)&ca.err, (void *)&wait_epoch, (void *)&spin_cap};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_chain<T, Fwd>), dim3(chain_grid<T, Fwd>(n)),
                                     dim3(kChainThreads), args, 0, s);
}



template <typename T>
struct GemmCfg;
template <>
struct GemmCfg<double> {
  static constexpr int BM = 64, BN = 64, TM = 4, TN = 4;
};
template <>
struct GemmCfg<float> {
  static constexpr int BM = 128, BN = 128, TM = 8, TN = 8;
};

// Cluster size for a panel of R rows: the smallest C (rows per CTA near 512)
// that fits the shared-memory budget, up to the largest cluster this device
// schedules with that budget; 0 means "use the single-CTA kernel".
template <typename T, int NB>
size_t panel_smem_bytes(int per) {
  return sizeof(T) * size_t(NB) * per + sizeof(int32_t) * size_t(per) + size_t(per) + 16;
}

// Largest cluster the register-resident panel kernel can run with (16 or 8;
// 0 if none), for a panel of up to kRegPanelMaxRows rows per CTA.
template <typename T, int NB>
size_t reg_panel_smem_bytes(int R) {
  return size_t(R) * (2 * sizeof(int32_t) + 1) + 16;
}

template <typename T, int NB>
int reg_panel_cluster_max() {
  static int cmax = -1;
  if (cmax < 0) {
    auto k = k_panel_reg<T, NB>;
    const size_t smem = reg_panel_smem_bytes<T, NB>(kRegPanelMaxRows * kMaxPanelCluster);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cmax = 0;
    for (int c : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(c));
      cfg.blockDim = dim3(kRegPanelThreads);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = unsigned(c);
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n > 0) {
        cmax = c;
        break;
      }
    }
    cudaGetLastError();
  }
  return cmax;
}

template <typename T, int NB>
int panel_cluster_size(int R) {
  constexpr size_t kSmemCap = 200 * 1024;
  static int cmax = -1;
  if (cmax < 0) {
    auto k = k_panel_cluster<T, NB>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemCap));
    cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cmax = 0;
    for (int c : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(c));
      cfg.blockDim = dim3(kClusterPanelThreads);
      cfg.dynamicSmemBytes = kSmemCap;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = unsigned(c);
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n > 0) {
        cmax = c;
        break;
      }
    }
    cudaGetLastError();
  }
  if (cmax <= 0 || R <= 0) return 0;
  const size_t row_bytes = sizeof(T) * NB + sizeof(int32_t) + 1;
  const int cap_rows = int((kSmemCap - 16) / row_bytes);
  const int need = (R + cap_rows - 1) / cap_rows;  // clusters smaller than this do not fit
  if (need > cmax) return 0;
  int C = std::min(cmax, std::max(need, (R + 511) / 512));
  int c2 = 1;
  while (c2 < C) c2 <<= 1;
  return c2 <= cmax ? c2 : C;}

}  // namespace

template <typename TS, typename T>
cudaError_t launch_assemble(const AItem *items, int64_t n, const TS *S, T *fronts, cudaStream_t s, Prof *prof,
                            double bytes) {
  if (n == 0) return cudaSuccess;
  const size_t e0 = prof->begin();
  k_assemble<TS, T><<<unsigned(n), 128, 0, s>>>(items, S, fronts);
  prof->end(P_ASSEMBLE, 1, e0, bytes);
  return cudaGetLastError();
}

// Outer block width of the blocked FP32 LU (four 64-column panels).
constexpr int kLuOuter = kLuOuterBlock;

// The FP32 fronts are factored in outer blocks of kLuOuter columns (with
// tensor cores and TMA descriptors); H2SP_LU=step keeps one trailing update
// per 64-column panel.
inline bool blocked_lu_enabled() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_LU");
    v = (e && std::strcmp(e, "step") == 0) ? 0 : 1;
  }
  return v == 1;
}

// FP32 panels with the pivot search restricted to the diagonal tile
// (H2SP_PANEL=tile); partial pivoting over the supernode rows otherwise.
inline bool tile_panel_enabled() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_PANEL");
    v = (e && std::strcmp(e, "tile") == 0) ? 1 : 0;
  }
  return v == 1;
}

// The FP32 trailing update runs on the tensor cores (three-term TF32 split);
// H2SP_GEMM=simt selects the CUDA-core kernel instead.
inline bool use_tensor_core_gemm() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_GEMM");
    v = (e && std::strcmp(e, "simt") == 0) ? 0 : 1;
  }
  return v == 1;
}

// The FP32 block LU's block-end update: 128 x 256 tiles with the C update by
// TMA reduce-add (k_gemm_tc_wide, four operand stages); H2SP_GEMM_WIDE=load
// loads and stores C instead, H2SP_GEMM_WIDE=0 keeps the 128 x 128 tiles.
inline int wide_lu_mode() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_GEMM_WIDE");
    v = (e && std::strcmp(e, "0") == 0) ? 0 : (e && std::strcmp(e, "load") == 0) ? 1 : 2;
  }
  return v;
}


// Step j0 of the blocked LU of every front of a level: panel (columns
// [j0, j0 + NB), partial pivoting over the supernode rows), row interchanges
// and U12 = L11^-1 A12, then A22 -= L21 U12.  With look-ahead the trailing
// update is split: the first column tile (which holds the next panel) goes
// first, then the next panel is factored on the high-priority side stream
// while the remaining columns are updated on the main stream.
template <typename T>
cudaError_t launch_lu_level(const FrontDev *fr, const Front *host_fr, int nfront, int max_s, int max_f, T *fronts,
                            int32_t *piv, int32_t *swaps, int *err, cudaStream_t s, const LuAsync *la, Prof *prof,
                            const uint8_t *maps, float *pack, const uint8_t *maps64) {
  constexpr int NB = LuCfg<T>::NB;
  using G = GemmCfg<T>;
  auto gemm = k_gemm_update<T, G::BM, G::BN, G::TM, G::TN, NB>;
  const size_t gsmem = sizeof(T) * NB * (G::BM + G::BN + 2 * (16 / sizeof(T)));
  if (cudaError_t ea = smem_attr((const void *)gemm, int(gsmem)); ea != cudaSuccess) return ea;
  bool tc = false;
  if constexpr (std::is_same<T, float>::value) tc = use_tensor_core_gemm();
  const int W = tc ? kTcTile : G::BN;  // width of the first column tile (holds the next panel)
  static_assert(G::BN >= NB, "the first column tile must cover the next panel");
  const int nsm = num_sms();

  // the interchanges of step j0 go to half (j0 / NB) & 1 of the swaps buffer: the
  // next panel writes the other half while this step's remaining columns are
  // still being interchanged on the low-priority stream
  const size_t swap_stride = size_t(nfront) * (1 + 2 * kMaxSwapRows);
  int slot_mask = 1;  // swap-list slots in use: 2 (one panel step ahead) or 8 (two outer blocks of 4 panels)
  auto panel = [&](int j0, cudaStream_t st, int *cl) -> cudaError_t {
    int32_t *swp = swaps + size_t((j0 / NB) & slot_mask) * swap_stride;
    double fpanel = 0.0;
    if (prof->timing)
      for (int k = 0; k < nfront; ++k) {
        const Front &F = host_fr[k];
        if (j0 >= F.s) continue;
        const double jb = std::min(NB, F.s - j0), rows = F.f - j0;
        fpanel += rows * jb * jb;  // scaling + rank-1 updates inside the panel
      }
    const size_t e0 = prof->begin(st);
    const int R = max_f - j0;
    if constexpr (std::is_same<T, float>::value) {
      if (tile_panel_enabled()) {
        *cl = nfront;
        k_panel_tile_diag<NB><<<nfront, kTileThreads, 0, st>>>(fr, j0, fronts, piv, swp, err);
        const int chunks = std::max(1, cdiv(R - 1, kL21Rows));
        k_panel_tile_l21<NB><<<dim3(unsigned(chunks), unsigned(nfront)), kL21Rows, 0, st>>>(fr, j0, fronts);
        prof->end(P_PANEL, 2, e0, fpanel, st);
        return cudaGetLastError();
      }
    }
    const int creg = reg_panel_cluster_max<T, NB>();
    const int C = (creg > 0 && R <= kRegPanelMaxRows * creg) ? 0 : panel_cluster_size<T, NB>(R);
    if (creg > 0 && R <= kRegPanelMaxRows * creg) {
      // rows in registers: one row per thread where the cluster allows, else two
      int cr = std::max(1, cdiv(R, kRegPanelThreads));
      if (cr > creg) cr = cdiv(R, kRegPanelMaxRows);
      *cl = cr * nfront;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(nfront * cr));
      cfg.blockDim = dim3(kRegPanelThreads);
      cfg.dynamicSmemBytes = reg_panel_smem_bytes<T, NB>(R);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = unsigned(cr);
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaError_t le = cudaLaunchKernelEx(&cfg, k_panel_reg<T, NB>, fr, j0, fronts, piv, swp, err);
      if (le != cudaSuccess) return le;
    } else if (C > 0) {
      *cl = C * nfront;
      const int per = (R + C - 1) / C;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(nfront * C));
      cfg.blockDim = dim3(kClusterPanelThreads);
      cfg.dynamicSmemBytes = panel_smem_bytes<T, NB>(per);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = unsigned(C);
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaError_t le = cudaLaunchKernelEx(&cfg, k_panel_cluster<T, NB>, fr, j0, fronts, piv, swp, err);
      if (le != cudaSuccess) return le;
    } else {
      *cl = nfront;
      k_panel<T, NB><<<nfront, kPanelThreads, 0, st>>>(fr, j0, fronts, piv, swp, err);
    }
    prof->end(P_PANEL, 1, e0, fpanel, st);
    return cudaSuccess;
  };
  // A22[:, c_lo:c_hi] -= L21 U12[:, c_lo:c_hi] (columns relative to the trailing block), on stream us
  auto update = [&](int j0, int c_lo, int c_hi, int sm_budget, cudaStream_t us) -> cudaError_t {
    const int rest = max_f - j0 - 1;
    if (rest <= 0 || c_lo >= std::min(rest, c_hi)) return cudaSuccess;
    double fgemm = 0.0;
    if (prof->timing)
      for (int k = 0; k < nfront; ++k) {
        const Front &F = host_fr[k];
        if (j0 >= F.s) continue;
        const double jb = std::min(NB, F.s - j0);
        const int nrest = F.f - j0 - int(jb);
        const double cols = std::max(0, std::min(nrest, c_hi) - c_lo);
        fgemm += 2.0 * nrest * cols * jb;  // algorithmic flops
      }
    const size_t e0 = prof->begin(us);
    if (tc) {
      if constexpr (std::is_same<T, float>::value) {
        const int thi = c_hi >= (INT_MAX - kTcTile) ? INT_MAX : c_hi / kTcTile;
        bool any_full = false, any_partial = false;
        for (int k = 0; k < nfront; ++k) {
          const int left = host_fr[k].s - j0;
          if (left >= NB) any_full = true;
          else if (left > 0) any_partial = true;
        }
        cudaError_t ge = launch_gemm_tc(fr, j0, nfront, max_f, fronts, err, us, c_lo / kTcTile, thi, sm_budget,
                                        maps, any_full, any_partial);
        if (ge != cudaSuccess) return ge;
      }
    } else {
      const int ncol = std::min(rest, c_hi) - c_lo;
      dim3 g(cdiv(ncol, G::BN), cdiv(rest, G::BM), nfront);
      gemm<<<g, 256, gsmem, us>>>(fr, j0, fronts, c_lo, c_hi, 0);
    }
    prof->end(P_GEMM, 1, e0, fgemm, us);
    return cudaSuccess;
  };

  const bool ahead = la != nullptr && la->side != nullptr && la->rest != nullptr && la->next != nullptr &&
                     la->panel != nullptr && la->done != nullptr;
  int panel_ctas = 0;
  cudaError_t e = cudaSuccess;
  if constexpr (std::is_same<T, float>::value && NB == 64) {
    if (tc && maps != nullptr && pack != nullptr && blocked_lu_enabled()) {
      // ---- blocked LU: outer blocks of KB columns = KB / NB panels ----
      constexpr int KB = kLuOuter;
      slot_mask = 7;
      // packed operands: two L21 buffers (by block parity) and one U12 buffer,
      // each kPackTileFloats per 128-row tile of the level's fronts
      int64_t pack_tiles = 0;
      for (int k = 0; k < nfront; ++k) pack_tiles += cdiv(host_fr[k].f, kTcTile);
      const int64_t pack_stride = pack_tiles * kPackTileFloats;
      cudaStream_t ms = ahead ? la->side : s;  // panels, inner steps, the next block's columns
      cudaStream_t rs = ahead ? la->rest : s;  // the rest of each block-end update
      cudaEvent_t done_ev[2] = {ahead ? la->panel : nullptr, ahead ? la->done : nullptr};
      if (ahead) {
        if ((e = cudaEventRecord(la->next, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(ms, la->next, 0)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(rs, la->next, 0)) != cudaSuccess) return e;
      }
      if (cudaError_t ea = smem_attr((const void *)k_blk_swap_trsm<KB>, int(sizeof(float) * 64 * KB));
          ea != cudaSuccess)
        return ea;
      auto fl_trsm = [&](int j0, int lo_col, int hi_col) {  // U12 flops of a panel step over a column range
        double f = 0.0;
        if (prof->timing)
          for (int k = 0; k < nfront; ++k) {
            const Front &F = host_fr[k];
            if (j0 >= F.s) continue;
            const double jb = std::min(NB, F.s - j0);
            f += jb * jb * std::max(0, std::min(hi_col, F.s) - std::max(lo_col, j0 + int(jb)));
          }
        return f;
      };
      // block end, over the columns [t0 + lo, t0 + hi) of the trailing block
      // (and, with left, the interchanges of the columns before the block)
      float *apack[2] = {pack, pack + pack_stride};
      float *bpack = pack + 2 * pack_stride;
      auto block_end = [&](int J, int lo, int hi, bool left, int budget, cudaStream_t st) -> cudaError_t {
        double ft = 0.0, fg = 0.0, fp = 0.0;
        int wcols = 0;
        for (int k = 0; k < nfront; ++k) {
          const Front &F = host_fr[k];
          if (J >= F.s) continue;
          const int jbo = std::min(KB, F.s - J), t0 = J + jbo, nrest = F.f - t0;
          const int cols = std::max(0, std::min(nrest, hi) - lo);
          wcols = std::max(wcols, cols);
          ft += 0.5 * double(jbo) * jbo * cols;
          fg += 2.0 * double(jbo) * nrest * cols;  // algorithmic flops of the rank-jbo update
          fp += 12.0 * double(jbo) * cols;         // the U12 pack: 4 bytes read, 8 written per element
        }
        size_t e0 = prof->begin(st);
        if (left && J > 0)
          k_blk_swap_trsm<KB><<<dim3(cdiv(J, kBlkCtaCols), nfront), 256, 0, st>>>(fr, J, fronts, swaps,
                                                                                  int64_t(swap_stride), 0, J, 0);
        if (wcols > 0)
          k_blk_swap_trsm<KB><<<dim3(cdiv(wcols, kBlkCtaCols), nfront), 256, sizeof(float) * 64 * KB, st>>>(
              fr, J, fronts, swaps, int64_t(swap_stride), lo, hi, 1);
        prof->end(P_TRSM, (left && J > 0 ? 1 : 0) + (wcols > 0 ? 1 : 0), e0, ft, st);
        if (wcols <= 0) return cudaGetLastError();
        const int tlo = lo / kTcTile, thi = hi >= (INT_MAX - kTcTile) ? INT_MAX : hi / kTcTile;
        e0 = prof->begin(st);
        cudaError_t ge = launch_pack_b(fr, J, KB, nfront, max_f, fronts, bpack, tlo, thi, st);
        prof->end(P_GEMM_INNER, 1, e0, fp, st);
        e0 = prof->begin(st);
        if (ge == cudaSuccess)
          ge = wide_lu_mode() != 0
                   ? launch_gemm_tc_wide(fr, J, KB, nfront, max_f, fronts, err, st, tlo, thi, budget,
                                         apack[(J / KB) & 1], bpack, /*lower=*/0, 0, maps64, wide_lu_mode() == 2)
                   : launch_gemm_tc_ws(fr, J, KB, nfront, max_f, fronts, err, st, tlo, thi, budget, maps,
                                       apack[(J / KB) & 1], bpack, 0, 0, maps64);
        prof->end(P_GEMM, 1, e0, fg, st);
        return ge != cudaSuccess ? ge : cudaGetLastError();
      };
      const int nblk = cdiv(max_s, KB);
      if ((e = panel(0, ms, &panel_ctas)) != cudaSuccess) return e;
      for (int b = 0; b < nblk; ++b) {
        const int J = b * KB;
        for (int i = 0; i < KB / NB; ++i) {
          const int jp = J + i * NB;
          if (jp >= max_s) break;
          if (i > 0 && (e = panel(jp, ms, &panel_ctas)) != cudaSuccess) return e;
          {
            const int32_t *sw = swaps + size_t((jp / NB) & slot_mask) * swap_stride;
            const size_t e0 = prof->begin(ms);
            k_swap_trsm<T, NB><<<dim3(cdiv(KB, 8), nfront), 256, 0, ms>>>(fr, jp, fronts, sw, 3, KB);
            prof->end(P_TRSM, 1, e0, fl_trsm(jp, J, J + KB), ms);
          }
          if (i + 1 < KB / NB) {
            double fgemm = 0.0;
            if (prof->timing)
              for (int k = 0; k < nfront; ++k) {
                const Front &F = host_fr[k];
                if (jp >= F.s) continue;
                const int jb = std::min(NB, F.s - jp), nrest = F.f - jp - jb;
                const int cols = std::max(0, std::min(J + KB, F.s) - (jp + jb));
                fgemm += double(sizeof(float)) * (2.0 * nrest * cols + double(jb) * (nrest + cols));
              }
            const size_t e0 = prof->begin(ms);
            if ((e = launch_gemm_tc_inner(fr, jp, KB, nfront, max_f, fronts, err, ms, nsm)) != cudaSuccess) return e;
            prof->end(P_GEMM_INNER, 1, e0, fgemm, ms);
          }
        }
        const bool more = J + KB < max_s;
        if ((e = launch_pack_a(fr, J, KB, nfront, max_f, fronts, apack[b & 1], ms)) != cudaSuccess) return e;
        if (ahead) {
          // the rest of the block end goes to the low-priority stream as soon
          // as the block's panels are done; the next block's columns stay here
          if ((e = cudaEventRecord(la->next, ms)) != cudaSuccess) return e;
          if ((e = cudaStreamWaitEvent(rs, la->next, 0)) != cudaSuccess) return e;
          if ((e = block_end(J, KB, INT_MAX, true, std::max(nsm - panel_ctas, nsm / 2), rs)) != cudaSuccess) return e;
          if ((e = cudaEventRecord(done_ev[b & 1], rs)) != cudaSuccess) return e;
          // the previous block's rest covered these columns
          if (b > 0 && (e = cudaStreamWaitEvent(ms, done_ev[(b - 1) & 1], 0)) != cudaSuccess) return e;
          if ((e = block_end(J, 0, KB, false, nsm, ms)) != cudaSuccess) return e;
        } else {
          if ((e = block_end(J, 0, INT_MAX, true, nsm, s)) != cudaSuccess) return e;
        }
        if (more && (e = panel(J + KB, ms, &panel_ctas)) != cudaSuccess) return e;
      }
      if (ahead) {
        if ((e = cudaStreamWaitEvent(ms, done_ev[(nblk - 1) & 1], 0)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(la->next, ms)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, la->next, 0)) != cudaSuccess) return e;
      }
      return cudaGetLastError();
    }
  }
  e = panel(0, s, &panel_ctas);
  if (e != cudaSuccess) return e;
  for (int j0 = 0; j0 < max_s; j0 += NB) {
    double ftrsm = 0.0;
    if (prof->timing)
      for (int k = 0; k < nfront; ++k) {
        const Front &F = host_fr[k];
        if (j0 >= F.s) continue;
        const double jb = std::min(NB, F.s - j0), rest = F.f - j0 - jb;
        ftrsm += jb * jb * rest;  // U12 = L^-1 A12
      }
    const int32_t *sw = swaps + size_t((j0 / NB) & 1) * swap_stride;  // this step's interchanges
    const bool more = j0 + NB < max_s;
    auto swap_trsm = [&](int part, cudaStream_t st) {
      const size_t e0 = prof->begin(st);
      const int span = part == 1 ? W : max_f;
      const int ncol_blocks = std::min(cdiv(span, 8), 4096);
      k_swap_trsm<T, NB><<<dim3(ncol_blocks, nfront), 256, 0, st>>>(fr, j0, fronts, sw, part, W);
      const double share = std::min(1.0, double(W) / std::max(max_f, 1));
      prof->end(P_TRSM, 1, e0, part == 0 ? ftrsm : part == 1 ? ftrsm * share : ftrsm * (1.0 - share), st);
    };
    if (more && ahead) {
      // the next panel's columns first; the other columns' interchanges and
      // U12 move to the low-priority stream, ahead of the rest of the update
      swap_trsm(1, s);
      if ((e = update(j0, 0, W, nsm, s)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(la->next, s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(la->side, la->next, 0)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(la->rest, la->next, 0)) != cudaSuccess) return e;
      if ((e = panel(j0 + NB, la->side, &panel_ctas)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(la->panel, la->side)) != cudaSuccess) return e;
      swap_trsm(2, la->rest);
      if ((e = update(j0, W, INT_MAX, std::max(nsm - panel_ctas, nsm / 2), la->rest)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(la->done, la->rest)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(s, la->panel, 0)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(s, la->done, 0)) != cudaSuccess) return e;
    } else {
      swap_trsm(0, s);
      if ((e = update(j0, 0, INT_MAX, nsm, s)) != cudaSuccess) return e;
      if (more && (e = panel(j0 + NB, s, &panel_ctas)) != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extend_add_impl(const FrontDev *fr_all, int lo, int nfront, int max_b, const int32_t *map,
                                   T *fronts, cudaStream_t s, Prof *prof, double elems, bool lower) {
  if (nfront == 0 || max_b == 0) return cudaSuccess;
  dim3 g(cdiv(max_b, 32), cdiv(max_b, 32), nfront);
  const size_t e0 = prof->begin();
  k_extend_add<T><<<g, 256, 0, s>>>(fr_all, lo, map, fronts, lower ? 1 : 0);
  prof->end(P_EXTEND, 1, e0, elems);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gemm_update_sym(const FrontDev *fr, int j0, int nfront, int max_f, T *fronts, cudaStream_t s) {
  constexpr int NB = LuCfg<T>::NB;
  using G = GemmCfg<T>;
  auto gemm = k_gemm_update<T, G::BM, G::BN, G::TM, G::TN, NB>;
  const size_t gsmem = sizeof(T) * NB * (G::BM + G::BN + 2 * (16 / sizeof(T)));
  if (cudaError_t ea = smem_attr((const void *)gemm, int(gsmem)); ea != cudaSuccess) return ea;
  const int rest = max_f - j0 - 1;
  if (rest <= 0 || nfront == 0) return cudaSuccess;
  dim3 g(cdiv(rest, G::BN), cdiv(rest, G::BM), nfront);
  gemm<<<g, 256, gsmem, s>>>(fr, j0, fronts, 0, INT_MAX, 1);
  return cudaGetLastError();
}

bool use_tensor_core_gemm_host() { return use_tensor_core_gemm(); }

template <typename T>
cudaError_t launch_make_perm(const FrontDev *fr, int nfront, int max_s, const int32_t *piv, int32_t *perm,
                             cudaStream_t s, Prof *prof) {
  if (nfront == 0) return cudaSuccess;
  const int cap = 40 * 1024;  // entries staged in shared memory (160 KB)
  const size_t smem = sizeof(int32_t) * size_t(std::min(max_s, cap));
  if (cudaError_t ea = smem_attr((const void *)k_make_perm, int(sizeof(int32_t) * cap)); ea != cudaSuccess) return ea;
  const size_t e0 = prof->begin();
  k_make_perm<<<nfront, 256, smem, s>>>(fr, piv, perm, std::min(max_s, cap));
  prof->end(P_OTHER, 1, e0, 0.0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_invert_diag(const FrontDev *fr, int nfront, int max_s, const T *fronts, T *dinv, cudaStream_t s,
                               Prof *prof) {
  if (nfront == 0 || max_s == 0) return cudaSuccess;
  const size_t e0 = prof->begin();
  k_invert_diag<T><<<dim3(cdiv(max_s, kBS), nfront), kBS, 0, s>>>(fr, fronts, dinv);
  prof->end(P_OTHER, 1, e0, 0.0);
  return cudaGetLastError();
}

constexpr int kLogdetThreads = 256;

// One CTA per front: sum of log|u_jj| over the pivot block (the diagonal of
// U11 left in place by the LU) and the parity of the block's interchanges
// (piv[j] != j) and negative pivots; det F11 = (-1)^interchanges prod u_jj.
template <typename T>
__global__ void __launch_bounds__(kLogdetThreads) k_logdet_front(const FrontDev *__restrict__ fr,
                                                                 const T *__restrict__ fronts,
                                                                 const int32_t *__restrict__ piv,
                                                                 double *__restrict__ lsum, int *__restrict__ flips) {
  const FrontDev F = fr[blockIdx.x];
  double acc = 0.0;
  int odd = 0;
  for (int j = threadIdx.x; j < F.s; j += kLogdetThreads) {
    const double u = double(fronts[F.off + int64_t(j) * F.ld + j]);
    acc += log(fabs(u));
    odd ^= int(u < 0.0) ^ int(piv[F.piv_off + j] != j);
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    odd ^= __shfl_xor_sync(0xffffffffu, odd, o);
  }
  __shared__ double sa[kLogdetThreads / 32];
  __shared__ int so[kLogdetThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = acc;
    so[threadIdx.x >> 5] = odd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    int p = 0;
    for (int w = 0; w < kLogdetThreads / 32; ++w) {
      t += sa[w];
      p ^= so[w];
    }
    lsum[blockIdx.x] = t;
    flips[blockIdx.x] = p;
  }
}

// One warp per independent system: its fronts' sums, lanes strided, then a
// butterfly (every lane ends with the same value).
__global__ void __launch_bounds__(kLogdetThreads) k_logdet_sys(const int32_t *__restrict__ sys_ptr,
                                                               const int32_t *__restrict__ sys_front,
                                                               const double *__restrict__ lsum,
                                                               const int *__restrict__ flips, int nsys,
                                                               double *__restrict__ out, int32_t *__restrict__ sign) {
  const int w = blockIdx.x * (kLogdetThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nsys) return;  // uniform across the warp
  double acc = 0.0;
  int odd = 0;
  for (int i = sys_ptr[w] + lane; i < sys_ptr[w + 1]; i += 32) {
    const int f = sys_front[i];
    acc += lsum[f];
    odd ^= flips[f];
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    odd ^= __shfl_xor_sync(0xffffffffu, odd, o);
  }
  if (lane == 0) {
    out[w] = acc;
    sign[w] = odd ? -1 : 1;
  }
}

template <typename T>
cudaError_t launch_logdet(const FrontDev *fr, int nfront, const T *fronts, const int32_t *piv, const int32_t *sys_ptr,
                          const int32_t *sys_front, int nsys, double *lsum, int *flips, double *out, int32_t *sign,
                          cudaStream_t s, Prof *prof) {
  if (nsys <= 0) return cudaSuccess;
  const size_t e0 = prof->begin();
  if (nfront > 0) k_logdet_front<T><<<nfront, kLogdetThreads, 0, s>>>(fr, fronts, piv, lsum, flips);
  k_logdet_sys<<<cdiv(nsys, kLogdetThreads / 32), kLogdetThreads, 0, s>>>(sys_ptr, sys_front, lsum, flips, nsys, out,
                                                                          sign);
  prof->end(P_OTHER, nfront > 0 ? 2 : 1, e0, 0.0);
  return cudaGetLastError();
}

template <typename T>
size_t step_smem() {
  const size_t bytes = sizeof(T) * (kBS * kBS + 2 * kBS * kMaxRhs);
  smem_attr((const void *)k_fwd_step<T>, int(bytes));
  smem_attr((const void *)k_bwd_step<T>, int(bytes));
  return bytes;
}

template <typename T>
cudaError_t launch_solve_fwd_level_impl(const FrontDev *fr, int lo, int nfront, int max_s, int max_f, const T *fronts,
                                        const T *dinv, const int32_t *perm, const int32_t *idx, T *y, int64_t ldy,
                                        int nrhs, T *work, T *zbuf, const int64_t *work_off, cudaStream_t s,
                                        Prof *prof, double bytes, const ChainArgs *ca, int li) {
  if (nfront == 0) return cudaSuccess;
  const FrontDev *frl = fr + lo;
  const size_t e0 = prof->begin();
  int nl = 2;
  k_fwd_gather<T><<<dim3(cdiv(max_f, 256), nfront), 256, 0, s>>>(frl, perm, idx, y, ldy, nrhs, work, work_off, lo);
  if (ca != nullptr) {
    cudaError_t ce = launch_chain<T, true>(fr, *ca, li, fronts, dinv, nrhs, work, zbuf, work_off, s);
    if (ce != cudaSuccess) return ce;
    // the boundary rows take the whole L21 Z product after the chain
    k_rect_update<T><<<dim3(cdiv(std::max(max_f - 1, 1), kRectRows), cdiv(max_s, kU12Chunk), nfront), kRowsPerCta, 0,
                       s>>>(frl, fronts, nrhs, work, zbuf, work_off, lo, 1);
    nl += 2;
  } else
  for (int c0 = 0; c0 < max_s; c0 += kBS) {
    const int rest = max_f - c0 - 1;
    const int nb = std::max(1, cdiv(std::max(rest, 1), kStepRows));
    k_fwd_step<T><<<dim3(nb, nfront), kStepThreads, step_smem<T>(), s>>>(frl, c0, fronts, dinv, nrhs, work, zbuf,
                                                                       work_off, lo);
    ++nl;
  }
  k_fwd_scatter<T><<<dim3(cdiv(max_f, 256), nfront), 256, 0, s>>>(frl, idx, y, ldy, nrhs, work, zbuf, work_off, lo);
  prof->end(P_SOLVE, nl, e0, bytes);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_bwd_level_impl(const FrontDev *fr, int lo, int nfront, int max_s, int max_f, const T *fronts,
                                        const T *dinv, const int32_t *idx, T *y, int64_t ldy, int nrhs, T *work,
                                        T *zbuf, const int64_t *work_off, cudaStream_t s, Prof *prof, double bytes,
                                        const ChainArgs *ca, int li) {
  if (nfront == 0) return cudaSuccess;
  const FrontDev *frl = fr + lo;
  const size_t e0 = prof->begin();
  int nl = 3;
  k_bwd_gather<T><<<dim3(cdiv(max_f, 256), nfront), 256, 0, s>>>(frl, idx, y, ldy, nrhs, work, work_off, lo);
  k_rect_update<T><<<dim3(cdiv(max_s, kRectRows), cdiv(std::max(max_f - 1, 1), kU12Chunk), nfront), kRowsPerCta, 0,
                     s>>>(frl, fronts, nrhs, work, zbuf, work_off, lo, 0);
  const int last = ((max_s - 1) / kBS) * kBS;
  if (ca != nullptr) {
    cudaError_t ce = launch_chain<T, false>(fr, *ca, li, fronts, dinv, nrhs, work, zbuf, work_off, s);
    if (ce != cudaSuccess) return ce;
    ++nl;
  } else
  for (int c0 = last; c0 >= 0; c0 -= kBS) {
    const int nb = std::max(1, cdiv(c0, kStepRows));
    k_bwd_step<T><<<dim3(nb, nfront), kStepThreads, step_smem<T>(), s>>>(frl, c0, fronts, dinv, nrhs, work, zbuf,
                                                                       work_off, lo);
    ++nl;
  }
  k_bwd_scatter<T><<<dim3(cdiv(max_s, 256), nfront), 256, 0, s>>>(frl, idx, y, ldy, nrhs, zbuf, work_off, lo);
  prof->end(P_SOLVE, nl, e0, bytes);
  return cudaGetLastError();
}

template cudaError_t launch_assemble<double, double>(const AItem *, int64_t, const double *, double *, cudaStream_t,
                                                     Prof *, double);
template cudaError_t launch_assemble<float, double>(const AItem *, int64_t, const float *, double *, cudaStream_t,
                                                    Prof *, double);
template cudaError_t launch_lu_level<double>(const FrontDev *, const Front *, int, int, int, double *, int32_t *, int32_t *,
                                           int *, cudaStream_t, const LuAsync *, Prof *,
                                           const uint8_t *, float *, const uint8_t *);
template cudaError_t launch_make_perm<double>(const FrontDev *, int, int, const int32_t *, int32_t *, cudaStream_t, Prof *);
template cudaError_t launch_extend_add_impl<double>(const FrontDev *, int, int, int, const int32_t *, double *, cudaStream_t,
                                                  Prof *, double, bool);
template cudaError_t launch_gemm_update_sym<double>(const FrontDev *, int, int, int, double *, cudaStream_t);
template cudaError_t launch_gemm_update_sym<float>(const FrontDev *, int, int, int, float *, cudaStream_t);
template cudaError_t launch_invert_diag<double>(const FrontDev *, int, int, const double *, double *, cudaStream_t, Prof *);
template cudaError_t launch_logdet<double>(const FrontDev *, int, const double *, const int32_t *, const int32_t *,
                                           const int32_t *, int, double *, int *, double *, int32_t *, cudaStream_t,
                                           Prof *);
template cudaError_t launch_logdet<float>(const FrontDev *, int, const float *, const int32_t *, const int32_t *,
                                          const int32_t *, int, double *, int *, double *, int32_t *, cudaStream_t,
                                          Prof *);
template cudaError_t launch_solve_fwd_level_impl<double>(const FrontDev *, int, int, int, int, const double *, const double *,
                                                       const int32_t *, const int32_t *, double *, int64_t, int, double *,
                                                       double *, const int64_t *, cudaStream_t, Prof *, double,
                                                       const ChainArgs *, int);
template cudaError_t launch_solve_bwd_level_impl<double>(const FrontDev *, int, int, int, int, const double *, const double *,
                                                       const int32_t *, double *, int64_t, int, double *, double *,
                                                       const int64_t *, cudaStream_t, Prof *, double,
                                                       const ChainArgs *, int);
template cudaError_t launch_assemble<double, float>(const AItem *, int64_t, const double *, float *, cudaStream_t,
                                                    Prof *, double);
template cudaError_t launch_assemble<float, float>(const AItem *, int64_t, const float *, float *, cudaStream_t, Prof *,
                                                   double);
template cudaError_t launch_lu_level<float>(const FrontDev *, const Front *, int, int, int, float *, int32_t *, int32_t *,
                                           int *, cudaStream_t, const LuAsync *, Prof *,
                                           const uint8_t *, float *, const uint8_t *);
template cudaError_t launch_make_perm<float>(const FrontDev *, int, int, const int32_t *, int32_t *, cudaStream_t, Prof *);
template cudaError_t launch_extend_add_impl<float>(const FrontDev *, int, int, int, const int32_t *, float *, cudaStream_t,
                                                  Prof *, double, bool);
template cudaError_t launch_invert_diag<float>(const FrontDev *, int, int, const float *, float *, cudaStream_t, Prof *);
template cudaError_t launch_solve_fwd_level_impl<float>(const FrontDev *, int, int, int, int, const float *, const float *,
                                                       const int32_t *, const int32_t *, float *, int64_t, int, float *,
                                                       float *, const int64_t *, cudaStream_t, Prof *, double,
                                                       const ChainArgs *, int);
template cudaError_t launch_solve_bwd_level_impl<float>(const FrontDev *, int, int, int, int, const float *, const float *,
                                                       const int32_t *, float *, int64_t, int, float *, float *,
                                                       const int64_t *, cudaStream_t, Prof *, double,
                                                       const ChainArgs *, int);

}  // namespace h2sp
