// Applies of U^T and V (the products of Eq. main_uv used in Eq. sp0), the
// VBR product with S, the FP64 H^2 matrix-vector product of Definition 4.9,
// and the small vector kernels of the iterative solves (§5.5).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "kernels.h"

namespace h2sp {
namespace {

constexpr int kRhs = 16;  // right-hand sides handled per kernel pass

// Q^T applied to X_l(t); basis rows go to the next level, non-basis rows to S space
// T is the precision of Q, the vectors and the sums: FP64 for the applies
// of the API, FP32 inside the FP32 preconditioner.
template <typename T>
__global__ void __launch_bounds__(64) k_apply_qt(const ApItem *__restrict__ items, const T *__restrict__ Q,
                                                 const T *__restrict__ x, int64_t ldx, T *__restrict__ ys,
                                                 int64_t ldys, T *__restrict__ xn, int64_t ldxn, int nrhs) {
  const ApItem it = items[blockIdx.x];
  __shared__ T sx[kMaxBlock * kRhs];
  const int m = it.m;
  for (int e = threadIdx.x; e < m * nrhs; e += blockDim.x) {
    const int j = e % m, r = e / m;
    sx[j + r * kMaxBlock] = x[it.xin + j + r * ldx];
  }
  __syncthreads();
  const T *Qt = Q + it.q;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    T acc[kRhs];
#pragma unroll
    for (int r = 0; r < kRhs; ++r) acc[r] = T(0);
    for (int j = 0; j < m; ++j) {
      const T q = Qt[j + int64_t(i) * m];
#pragma unroll
      for (int r = 0; r < kRhs; ++r)
        if (r < nrhs) acc[r] += q * sx[j + r * kMaxBlock];
    }
    if (i < it.kp) {
      if (it.xout >= 0)
        for (int r = 0; r < nrhs; ++r) xn[it.xout + i + r * ldxn] = acc[r];
    } else {
      for (int r = 0; r < nrhs; ++r) ys[it.yout + (i - it.kp) + r * ldys] = acc[r];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(64) k_apply_q(const ApItem *__restrict__ items, const T *__restrict__ Q,
                                                const T *__restrict__ xn, int64_t ldxn,
                                                const T *__restrict__ ys, int64_t ldys, T *__restrict__ x,
                                                int64_t ldx, int nrhs) {
  const ApItem it = items[blockIdx.x];
  __shared__ T sz[kMaxBlock * kRhs];
  const int m = it.m;
  for (int e = threadIdx.x; e < m * nrhs; e += blockDim.x) {
    const int j = e % m, r = e / m;
    T v = T(0);
    if (j < it.kp) {
      if (it.xout >= 0) v = xn[it.xout + j + r * ldxn];
    } else {
      v = ys[it.yout + (j - it.kp) + r * ldys];
    }
    sz[j + r * kMaxBlock] = v;
  }
  __syncthreads();
  const T *Qt = Q + it.q;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    T acc[kRhs];
#pragma unroll
    for (int r = 0; r < kRhs; ++r) acc[r] = T(0);
    for (int j = 0; j < m; ++j) {
      const T q = Qt[i + int64_t(j) * m];
#pragma unroll
      for (int r = 0; r < kRhs; ++r)
        if (r < nrhs) acc[r] += q * sz[j + r * kMaxBlock];
    }
    for (int r = 0; r < nrhs; ++r) x[it.xin + i + r * ldx] = acc[r];
  }
}

// k_apply_qt / k_apply_q for levels whose blocks exceed kMaxBlock rows: the
// input slab (m x nrhs, leading dimension ms = the level's largest m) sits in
// dynamic shared memory; each thread computes rows i, i + 128, ...
template <typename T>
__global__ void __launch_bounds__(128) k_apply_qt_large(const ApItem *__restrict__ items, const T *__restrict__ Q,
                                                        const T *__restrict__ x, int64_t ldx, T *__restrict__ ys,
                                                        int64_t ldys, T *__restrict__ xn, int64_t ldxn, int nrhs,
                                                        int ms) {
  const ApItem it = items[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw_a[];
  T *sx = reinterpret_cast<T *>(smraw_a);
  const int m = it.m;
  for (int e = threadIdx.x; e < m * nrhs; e += blockDim.x) {
    const int j = e % m, r = e / m;
    sx[j + r * ms] = x[it.xin + j + r * ldx];
  }
  __syncthreads();
  const T *Qt = Q + it.q;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    T acc[kRhs];
#pragma unroll
    for (int r = 0; r < kRhs; ++r) acc[r] = T(0);
    for (int j = 0; j < m; ++j) {
      const T q = Qt[j + int64_t(i) * m];
#pragma unroll
      for (int r = 0; r < kRhs; ++r)
        if (r < nrhs) acc[r] += q * sx[j + r * ms];
    }
    if (i < it.kp) {
      if (it.xout >= 0)
        for (int r = 0; r < nrhs; ++r) xn[it.xout + i + r * ldxn] = acc[r];
    } else {
      for (int r = 0; r < nrhs; ++r) ys[it.yout + (i - it.kp) + r * ldys] = acc[r];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_apply_q_large(const ApItem *__restrict__ items, const T *__restrict__ Q,
                                                       const T *__restrict__ xn, int64_t ldxn,
                                                       const T *__restrict__ ys, int64_t ldys, T *__restrict__ x,
                                                       int64_t ldx, int nrhs, int ms) {
  const ApItem it = items[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw_a[];
  T *sz = reinterpret_cast<T *>(smraw_a);
  const int m = it.m;
  for (int e = threadIdx.x; e < m * nrhs; e += blockDim.x) {
    const int j = e % m, r = e / m;
    T v = T(0);
    if (j < it.kp) {
      if (it.xout >= 0) v = xn[it.xout + j + r * ldxn];
    } else {
      v = ys[it.yout + (j - it.kp) + r * ldys];
    }
    sz[j + r * ms] = v;
  }
  __syncthreads();
  const T *Qt = Q + it.q;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    T acc[kRhs];
#pragma unroll
    for (int r = 0; r < kRhs; ++r) acc[r] = T(0);
    for (int j = 0; j < m; ++j) {
      const T q = Qt[i + int64_t(j) * m];
#pragma unroll
      for (int r = 0; r < kRhs; ++r)
        if (r < nrhs) acc[r] += q * sz[j + r * ms];
    }
    for (int r = 0; r < nrhs; ++r) x[it.xin + i + r * ldx] = acc[r];
  }
}

template <typename T>
__global__ void k_copy_rows(const int64_t *__restrict__ src_row, const int64_t *__restrict__ dst_row,
                            const int32_t *__restrict__ len, const T *__restrict__ src, int64_t lds,
                            T *__restrict__ dst, int64_t ldd, int nrhs) {
  const int64_t s0 = src_row[blockIdx.x], d0 = dst_row[blockIdx.x];
  const int n = len[blockIdx.x];
  for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) {
    const int i = e % n, r = e / n;
    dst[d0 + i + r * ldd] = src[s0 + i + r * lds];
  }
}

template <typename TS>
__global__ void __launch_bounds__(128) k_spmv(const int64_t *__restrict__ brow_ptr, const int32_t *__restrict__ bcol,
                                              const int64_t *__restrict__ val_off, const int64_t *__restrict__ node_off,
                                              const TS *__restrict__ vals, const double *__restrict__ x, int64_t ldx,
                                              double *__restrict__ y, int64_t ldy, int nrhs) {
  const int i = blockIdx.x;
  const int64_t r0 = node_off[i];
  const int di = int(node_off[i + 1] - r0);
  __shared__ double sx[64 * kRhs];
  for (int rb = 0; rb < di; rb += blockDim.x) {
    const int row = rb + threadIdx.x;
    double acc[kRhs];
#pragma unroll
    for (int r = 0; r < kRhs; ++r) acc[r] = 0.0;
    for (int64_t z = brow_ptr[i]; z < brow_ptr[i + 1]; ++z) {
      const int j = bcol[z];
      const int64_t c0 = node_off[j];
      const int dj = int(node_off[j + 1] - c0);
      const TS *blk = vals + val_off[z];
      for (int cb = 0; cb < dj; cb += 64) {
        const int nc = min(64, dj - cb);
        __syncthreads();
        for (int e = threadIdx.x; e < nc * nrhs; e += blockDim.x) {
          const int c = e % nc, r = e / nc;
          sx[c + r * 64] = x[c0 + cb + c + r * ldx];
        }
        __syncthreads();
        if (row < di)
          for (int c = 0; c < nc; ++c) {
            const double a = double(blk[row + int64_t(cb + c) * di]);
#pragma unroll
            for (int r = 0; r < kRhs; ++r)
              if (r < nrhs) acc[r] += a * sx[c + r * 64];
          }
      }
    }
    if (row < di)
      for (int r = 0; r < nrhs; ++r) y[r0 + row + r * ldy] = acc[r];
  }
}

// ---------------- H^2 product (Definition 4.9) ----------------
// FP64 multiply-adds are the throughput limit of these kernels (GB300's FP64
// pipe), so idle lanes cost directly.  A CTA of 64 threads computes one
// cluster's rows; when the cluster has at most 32 (16) rows, the threads form
// 2 (4) groups that split the right-hand sides, so every lane carries rows.
// Each thread keeps 16 / G independent accumulators (one per right-hand side
// it owns) and reads the vector entries straight from global memory (the
// lanes of a warp read the same entry).
constexpr int kMvThreads = 64;

__device__ __forceinline__ int mv_groups(int rows) { return rows <= 16 ? 4 : (rows <= 32 ? 2 : 1); }

// acc[q] += sum_j A[i + j * lda] * X[j + (g + G q) * ldx] for j < nj
template <int G>
__device__ __forceinline__ void mv_accumulate(double *acc, const double *__restrict__ A, int64_t lda, int i, int nj,
                                              const double *__restrict__ X, int64_t ldx, int g, int nrhs) {
  constexpr int NQ = kRhs / G;
  for (int j = 0; j < nj; ++j) {
    const double a = A[i + int64_t(j) * lda];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int c = g + G * q;
      if (c < nrhs) acc[q] += a * X[j + int64_t(c) * ldx];
    }
  }
}

// y_t = R_t y^_t + sum_{s near t} C_ts x_s
template <int G>
__device__ __forceinline__ void leaf_out_body(const H2Dev &h, int lf, const double *__restrict__ x, int64_t ldx,
                                              const double *__restrict__ yh, int64_t ldh, double *__restrict__ y,
                                              int64_t ldy, int nrhs) {
  constexpr int P = kMvThreads / G, NQ = kRhs / G;
  const int t = h.leaf0 + lf;
  const int n = int(h.size[t]), k = h.rank[t];
  const int i = threadIdx.x % P, g = threadIdx.x / P;
  if (i >= n) return;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  mv_accumulate<G>(acc, h.leaf_basis + h.leaf_basis_off[lf], n, i, k, yh + h.xh_off[t], ldh, g, nrhs);
  for (int64_t z = h.near_ptr[lf]; z < h.near_ptr[lf + 1]; ++z) {
    const int s = h.near_col[z];
    mv_accumulate<G>(acc, h.near_block + h.near_off[z], n, i, int(h.size[s]), x + h.begin[s], ldx, g, nrhs);
  }
  const int64_t b0 = h.begin[t];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int c = g + G * q;
    if (c < nrhs) y[b0 + i + c * ldy] = acc[q];
  }
}

__global__ void __launch_bounds__(kMvThreads, 10) k_h2_leaf_out(H2Dev h, const double *__restrict__ x, int64_t ldx,
                                                            const double *__restrict__ yh, int64_t ldh,
                                                            double *__restrict__ y, int64_t ldy, int nrhs) {
  const int lf = h.leaf_order ? h.leaf_order[blockIdx.x] : int(blockIdx.x);
  const int n = int(h.size[h.leaf0 + lf]);
  switch (mv_groups(n)) {
    case 4: leaf_out_body<4>(h, lf, x, ldx, yh, ldh, y, ldy, nrhs); break;
    case 2: leaf_out_body<2>(h, lf, x, ldx, yh, ldh, y, ldy, nrhs); break;
    default: leaf_out_body<1>(h, lf, x, ldx, yh, ldh, y, ldy, nrhs); break;
  }
}

// leaf_out_body for leaves of more than kMvThreads points: rows r0 + tid, all
// right-hand sides per thread
__device__ __forceinline__ void leaf_out_rows(const H2Dev &h, int lf, int r0, const double *__restrict__ x,
                                              int64_t ldx, const double *__restrict__ yh, int64_t ldh,
                                              double *__restrict__ y, int64_t ldy, int nrhs) {
  const int t = h.leaf0 + lf;
  const int n = int(h.size[t]), k = h.rank[t];
  const int i = r0 + int(threadIdx.x);
  if (i >= n) return;
  double acc[kRhs];
#pragma unroll
  for (int q = 0; q < kRhs; ++q) acc[q] = 0.0;
  mv_accumulate<1>(acc, h.leaf_basis + h.leaf_basis_off[lf], n, i, k, yh + h.xh_off[t], ldh, 0, nrhs);
  for (int64_t z = h.near_ptr[lf]; z < h.near_ptr[lf + 1]; ++z) {
    const int s = h.near_col[z];
    mv_accumulate<1>(acc, h.near_block + h.near_off[z], n, i, int(h.size[s]), x + h.begin[s], ldx, 0, nrhs);
  }
  const int64_t b0 = h.begin[t];
#pragma unroll
  for (int q = 0; q < kRhs; ++q)
    if (q < nrhs) y[b0 + i + q * ldy] = acc[q];
}

// close blocks of the leaves leaf_order[first ..]: more than kMvThreads points each
__global__ void __launch_bounds__(kMvThreads) k_h2_leaf_out_large(H2Dev h, int first, const double *__restrict__ x,
                                                                  int64_t ldx, const double *__restrict__ yh,
                                                                  int64_t ldh, double *__restrict__ y, int64_t ldy,
                                                                  int nrhs) {
  const int lf = h.leaf_order[first + int(blockIdx.x)];
  const int n = int(h.size[h.leaf0 + lf]);
  for (int r0 = 0; r0 < n; r0 += kMvThreads) leaf_out_rows(h, lf, r0, x, ldx, yh, ldh, y, ldy, nrhs);
}

// y^_t = sum_{s in Far(t)} D_ts x^_s
template <int G>
__device__ __forceinline__ void couple_body(const H2Dev &h, int t, const double *__restrict__ xh,
                                            double *__restrict__ yh, int64_t ldh, int nrhs) {
  constexpr int P = kMvThreads / G, NQ = kRhs / G;
  const int kt = h.rank[t];
  const int i = threadIdx.x % P, g = threadIdx.x / P;
  if (i >= kt) return;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  for (int64_t z = h.far_ptr[t]; z < h.far_ptr[t + 1]; ++z) {
    const int s = h.far_col[z];
    mv_accumulate<G>(acc, h.coupling + h.coupling_off[z], kt, i, h.rank[s], xh + h.xh_off[s], ldh, g, nrhs);
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int c = g + G * q;
    if (c < nrhs) yh[h.xh_off[t] + i + c * ldh] = acc[q];
  }
}

__global__ void __launch_bounds__(kMvThreads, 10) k_h2_couple(H2Dev h, const double *__restrict__ xh,
                                                          double *__restrict__ yh, int64_t ldh, int nrhs) {
  const int t = h.couple_order ? h.couple_order[blockIdx.x] : int(blockIdx.x);
  switch (mv_groups(h.rank[t])) {
    case 4: couple_body<4>(h, t, xh, yh, ldh, nrhs); break;
    case 2: couple_body<2>(h, t, xh, yh, ldh, nrhs); break;
    default: couple_body<1>(h, t, xh, yh, ldh, nrhs); break;
  }
}

// ---- the same products for few right-hand sides (nrhs <= 4) ----
// With one right-hand side the kernels above give each thread one row and a
// serial chain of dependent FMAs, one global load per step.  Here a CTA of
// kNwThreads threads takes one block row (a leaf's close blocks, or a
// cluster's couplings) with several threads per row: thread (i, ph) of a
// row pad RP (32, 64 or 128 rows) sums the columns j = ph, ph + PH, ...
// (PH = kNwThreads / RP) with two independent accumulator sets, so a warp
// reads 32 consecutive rows of a column per load (coalesced) and keeps
// several loads in flight; the vector entries are read from global memory
// (every lane of a warp reads the same one).  The PH partial sums of a row
// are added in shared memory at the end, in a fixed order.
constexpr int kNwThreads = 256;

__device__ __forceinline__ int nw_rowpad(int rows) { return rows <= 32 ? 32 : (rows <= 64 ? 64 : 128); }

// acc0/acc1[r] += sum over this thread's columns j of A[i + j lda] X[j + r ldx]
template <int NR>
__device__ __forceinline__ void nw_accumulate(double (&acc0)[NR], double (&acc1)[NR], const double *__restrict__ A,
                                              int64_t lda, int i, int nc, const double *__restrict__ X, int64_t ldx,
                                              int ph, int PH, int nrhs) {
  int j = ph;
  for (; j + PH < nc; j += 2 * PH) {
    const double a0 = A[i + int64_t(j) * lda], a1 = A[i + int64_t(j + PH) * lda];
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) {
        acc0[r] += a0 * X[j + int64_t(r) * ldx];
        acc1[r] += a1 * X[j + PH + int64_t(r) * ldx];
      }
  }
  if (j < nc) {
    const double a0 = A[i + int64_t(j) * lda];
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) acc0[r] += a0 * X[j + int64_t(r) * ldx];
  }
}

// sum of the PH partials of each row (thread ph = 0 of row i receives it)
template <int NR>
__device__ __forceinline__ void nw_reduce(double (&acc0)[NR], const double (&acc1)[NR], int i, int ph, int RP,
                                          int PH, double *red) {
#pragma unroll
  for (int r = 0; r < NR; ++r) red[threadIdx.x + r * kNwThreads] = acc0[r] + acc1[r];
  __syncthreads();
  if (ph == 0)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double v = 0.0;
      for (int q = 0; q < PH; ++q) v += red[q * RP + i + r * kNwThreads];
      acc0[r] = v;
    }
}

// y_t = R_t y^_t + sum_{s near t} C_ts x_s for leaves of at most 128 points
template <int NR>
__global__ void __launch_bounds__(kNwThreads) k_h2_leaf_out_nw(H2Dev h, const double *__restrict__ x, int64_t ldx,
                                                             const double *__restrict__ yh, int64_t ldh,
                                                             double *__restrict__ y, int64_t ldy, int nrhs) {
  const int lf = h.leaf_order ? h.leaf_order[blockIdx.x] : int(blockIdx.x);
  const int t = h.leaf0 + lf;
  const int n = int(h.size[t]), k = h.rank[t];
  const int RP = nw_rowpad(n), PH = kNwThreads / RP;
  const int i = threadIdx.x % RP, ph = threadIdx.x / RP;
  __shared__ double red[kNwThreads * NR];
  double acc0[NR], acc1[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc0[r] = acc1[r] = 0.0;
  if (i < n) {
    nw_accumulate<NR>(acc0, acc1, h.leaf_basis + h.leaf_basis_off[lf], n, i, k, yh + h.xh_off[t], ldh, ph, PH, nrhs);
    for (int64_t z = h.near_ptr[lf]; z < h.near_ptr[lf + 1]; ++z) {
      const int s = h.near_col[z];
      nw_accumulate<NR>(acc0, acc1, h.near_block + h.near_off[z], n, i, int(h.size[s]), x + h.begin[s], ldx, ph, PH,
                        nrhs);
    }
  }
  nw_reduce<NR>(acc0, acc1, i, ph, RP, PH, red);
  if (ph == 0 && i < n) {
    const int64_t b0 = h.begin[t];
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) y[b0 + i + r * ldy] = acc0[r];
  }
}

// y^_t = sum_{s in Far(t)} D_ts x^_s
template <int NR>
__global__ void __launch_bounds__(kNwThreads) k_h2_couple_nw(H2Dev h, const double *__restrict__ xh,
                                                           double *__restrict__ yh, int64_t ldh, int nrhs) {
  const int t = h.couple_order ? h.couple_order[blockIdx.x] : int(blockIdx.x);
  const int kt = h.rank[t];
  const int RP = nw_rowpad(kt), PH = kNwThreads / RP;
  const int i = threadIdx.x % RP, ph = threadIdx.x / RP;
  __shared__ double red[kNwThreads * NR];
  double acc0[NR], acc1[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc0[r] = acc1[r] = 0.0;
  if (i < kt)
    for (int64_t z = h.far_ptr[t]; z < h.far_ptr[t + 1]; ++z) {
      const int s = h.far_col[z];
      nw_accumulate<NR>(acc0, acc1, h.coupling + h.coupling_off[z], kt, i, h.rank[s], xh + h.xh_off[s], ldh, ph, PH,
                        nrhs);
    }
  nw_reduce<NR>(acc0, acc1, i, ph, RP, PH, red);
  if (ph == 0 && i < kt)
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) yh[h.xh_off[t] + i + r * ldh] = acc0[r];
}

// y^_c += T_c y^_parent for the clusters [lo, hi) of one depth
template <int G>
__device__ __forceinline__ void down_body(const H2Dev &h, int c, double *__restrict__ yh, int64_t ldh, int nrhs) {
  constexpr int P = kMvThreads / G, NQ = kRhs / G;
  const int p = h.parent[c];
  const int kc = h.rank[c];
  const int i = threadIdx.x % P, g = threadIdx.x / P;
  if (i >= kc) return;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  mv_accumulate<G>(acc, h.transfer + h.transfer_off[c], kc, i, h.rank[p], yh + h.xh_off[p], ldh, g, nrhs);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int r = g + G * q;
    if (r < nrhs) yh[h.xh_off[c] + i + r * ldh] += acc[q];
  }
}

__global__ void __launch_bounds__(kMvThreads) k_h2_down(H2Dev h, int lo, double *__restrict__ yh, int64_t ldh,
                                                        int nrhs) {
  const int c = lo + blockIdx.x;
  switch (mv_groups(h.rank[c])) {
    case 4: down_body<4>(h, c, yh, ldh, nrhs); break;
    case 2: down_body<2>(h, c, yh, ldh, nrhs); break;
    default: down_body<1>(h, c, yh, ldh, nrhs); break;
  }
}

// acc[q] += sum_j A[j + i * lda] * X[j + (g + G q) * ldx]   (A transposed)
template <int G>
__device__ __forceinline__ void mv_accumulate_t(double *acc, const double *__restrict__ A, int64_t lda, int i, int nj,
                                                const double *__restrict__ X, int64_t ldx, int g, int nrhs) {
  constexpr int NQ = kRhs / G;
  const double *a = A + int64_t(i) * lda;
  for (int j = 0; j < nj; ++j) {
    const double av = a[j];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int c = g + G * q;
      if (c < nrhs) acc[q] += av * X[j + int64_t(c) * ldx];
    }
  }
}

// x^_t = E_t^T x_t for the leaves
template <int G>
__device__ __forceinline__ void leaf_up_body(const H2Dev &h, int lf, const double *__restrict__ x, int64_t ldx,
                                             double *__restrict__ xh, int64_t ldh, int nrhs) {
  constexpr int P = kMvThreads / G, NQ = kRhs / G;
  const int t = h.leaf0 + lf;
  const int n = int(h.size[t]), k = h.rank[t];
  const int i = threadIdx.x % P, g = threadIdx.x / P;
  if (i >= k) return;
  const double *E = h.col_leaf_basis ? h.col_leaf_basis + h.col_leaf_basis_off[lf] : h.leaf_basis + h.leaf_basis_off[lf];
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  mv_accumulate_t<G>(acc, E, n, i, n, x + h.begin[t], ldx, g, nrhs);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int c = g + G * q;
    if (c < nrhs) xh[h.xh_off[t] + i + c * ldh] = acc[q];
  }
}

__global__ void __launch_bounds__(kMvThreads) k_h2_leaf_up(H2Dev h, const double *__restrict__ x, int64_t ldx,
                                                           double *__restrict__ xh, int64_t ldh, int nrhs) {
  switch (mv_groups(h.rank[h.leaf0 + blockIdx.x])) {
    case 4: leaf_up_body<4>(h, blockIdx.x, x, ldx, xh, ldh, nrhs); break;
    case 2: leaf_up_body<2>(h, blockIdx.x, x, ldx, xh, ldh, nrhs); break;
    default: leaf_up_body<1>(h, blockIdx.x, x, ldx, xh, ldh, nrhs); break;
  }
}

// x^_p = sum_c T'_c^T x^_c over the sons of p (clusters [lo, hi) of one depth)
template <int G>
__device__ __forceinline__ void up_body(const H2Dev &h, const int32_t *__restrict__ child_start,
                                        const int32_t *__restrict__ child_cnt, int p, double *__restrict__ xh,
                                        int64_t ldh, int nrhs) {
  constexpr int P = kMvThreads / G, NQ = kRhs / G;
  const int kp = h.rank[p];
  const int i = threadIdx.x % P, g = threadIdx.x / P;
  if (i >= kp) return;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  for (int c = child_start[p]; c < child_start[p] + child_cnt[p]; ++c) {
    const int kc = h.rank[c];
    const double *T = h.col_transfer ? h.col_transfer + h.col_transfer_off[c] : h.transfer + h.transfer_off[c];
    mv_accumulate_t<G>(acc, T, kc, i, kc, xh + h.xh_off[c], ldh, g, nrhs);
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int r = g + G * q;
    if (r < nrhs) xh[h.xh_off[p] + i + r * ldh] = acc[q];
  }
}

__global__ void __launch_bounds__(kMvThreads) k_h2_up(H2Dev h, const int32_t *__restrict__ child_start,
                                                      const int32_t *__restrict__ child_cnt, int lo,
                                                      double *__restrict__ xh, int64_t ldh, int nrhs) {
  const int p = lo + blockIdx.x;
  switch (mv_groups(h.rank[p])) {
    case 4: up_body<4>(h, child_start, child_cnt, p, xh, ldh, nrhs); break;
    case 2: up_body<2>(h, child_start, child_cnt, p, xh, ldh, nrhs); break;
    default: up_body<1>(h, child_start, child_cnt, p, xh, ldh, nrhs); break;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// per (segment, column): ||b - y||^2 over the segment's rows (y == nullptr: ||b||^2);
// r = b - y is stored when r != nullptr.  grid = (chunks, segments, columns)
__global__ void __launch_bounds__(256) k_residual(const double *__restrict__ b, int64_t ldb, const double *__restrict__ y,
                                                  int64_t ldy, double *__restrict__ r, int64_t ldr,
                                                  const int64_t *__restrict__ seg_ptr, int nrhs,
                                                  double *__restrict__ norms2) {
  const int seg = blockIdx.y, c = blockIdx.z;
  const int64_t lo = seg_ptr[seg], hi = seg_ptr[seg + 1];
  __shared__ double red[8];
  double part = 0.0;
  for (int64_t i = lo + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < hi; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = b[i + c * ldb] - (y ? y[i + c * ldy] : 0.0);
    if (r) r[i + c * ldr] = v;
    part += v * v;
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(&norms2[int64_t(seg) * nrhs + c], t);
  }
}

// out[i * nrhs + c] = <V_i[:, c], W[:, c]> for the first nv blocks V_i (block stride ldv * nrhs)
__global__ void __launch_bounds__(256) k_block_dots(const double *__restrict__ V, int64_t ldv, int64_t vstride, int nv,
                                                    const double *__restrict__ W, int64_t ldw, int64_t n, int nrhs,
                                                    double *__restrict__ out) {
  const int i = blockIdx.y % nv, c = blockIdx.y / nv;
  const double *v = V + i * vstride + c * ldv;
  const double *w = W + c * ldw;
  __shared__ double red[8];
  double part = 0.0;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
    part += v[r] * w[r];
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) t += red[q];
    atomicAdd(&out[int64_t(i) * nrhs + c], t);
  }
}

// W[:, c] += sum_i coef[i * nrhs + c] * V_i[:, c]   (coef on the device)
__global__ void k_block_axpy(const double *__restrict__ V, int64_t ldv, int64_t vstride, int nv,
                             const double *__restrict__ coef, double *__restrict__ W, int64_t ldw, int64_t n) {
  const int c = blockIdx.y;
  const int nrhs = gridDim.y;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    double acc = W[r + c * ldw];
    for (int i = 0; i < nv; ++i) acc += coef[int64_t(i) * nrhs + c] * V[i * vstride + c * ldv + r];
    W[r + c * ldw] = acc;
  }
}

// X[:, c] *= s[c]
__global__ void k_col_scale(double *__restrict__ X, int64_t ldx, const double *__restrict__ sc, int64_t n) {
  const int c = blockIdx.y;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
    X[r + c * ldx] *= sc[c];
}

__global__ void k_axpy(const double *__restrict__ d, int64_t ldd, double *__restrict__ x, int64_t ldx, int64_t n) {
  const int c = blockIdx.y;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i + c * ldx] += d[i + c * ldd];
}

template <typename A, typename B>
__global__ void k_cast(const A *__restrict__ a, int64_t lda, B *__restrict__ b, int64_t ldb, int64_t n) {
  const int c = blockIdx.y;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i + c * ldb] = B(a[i + c * lda]);
}

inline unsigned grid_for(int64_t n, int per = 256) {
  return unsigned(std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 4 * device_sms())));
}

}  // namespace

template <typename T>
cudaError_t launch_apply_qt(const ApItem *items, int n, const T *Q, const T *x, int64_t ldx, T *ys, int64_t ldys, T *xn,
                            int64_t ldxn, int nrhs, cudaStream_t s, int max_m) {
  if (n == 0) return cudaSuccess;
  if (max_m > kMaxBlock) {
    const size_t smem = sizeof(T) * size_t(max_m) * kRhs;
    if (cudaError_t ea = smem_attr((const void *)k_apply_qt_large<T>, int(smem)); ea != cudaSuccess) return ea;
    for (int r0 = 0; r0 < nrhs; r0 += kRhs)
      k_apply_qt_large<T><<<n, 128, smem, s>>>(items, Q, x + r0 * ldx, ldx, ys + r0 * ldys, ldys,
                                               xn ? xn + r0 * ldxn : nullptr, ldxn, std::min(kRhs, nrhs - r0), max_m);
    return cudaGetLastError();
  }
  for (int r0 = 0; r0 < nrhs; r0 += kRhs)
    k_apply_qt<T><<<n, 64, 0, s>>>(items, Q, x + r0 * ldx, ldx, ys + r0 * ldys, ldys, xn ? xn + r0 * ldxn : nullptr,
                                   ldxn, std::min(kRhs, nrhs - r0));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_q(const ApItem *items, int n, const T *Q, const T *xn, int64_t ldxn, const T *ys, int64_t ldys,
                           T *x, int64_t ldx, int nrhs, cudaStream_t s, int max_m) {
  if (n == 0) return cudaSuccess;
  if (max_m > kMaxBlock) {
    const size_t smem = sizeof(T) * size_t(max_m) * kRhs;
    if (cudaError_t ea = smem_attr((const void *)k_apply_q_large<T>, int(smem)); ea != cudaSuccess) return ea;
    for (int r0 = 0; r0 < nrhs; r0 += kRhs)
      k_apply_q_large<T><<<n, 128, smem, s>>>(items, Q, xn ? xn + r0 * ldxn : nullptr, ldxn, ys + r0 * ldys, ldys,
                                              x + r0 * ldx, ldx, std::min(kRhs, nrhs - r0), max_m);
    return cudaGetLastError();
  }
  for (int r0 = 0; r0 < nrhs; r0 += kRhs)
    k_apply_q<T><<<n, 64, 0, s>>>(items, Q, xn ? xn + r0 * ldxn : nullptr, ldxn, ys + r0 * ldys, ldys, x + r0 * ldx,
                                  ldx, std::min(kRhs, nrhs - r0));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_rows(const int64_t *src_row, const int64_t *dst_row, const int32_t *len, int n, const T *src,
                             int64_t lds, T *dst, int64_t ldd, int nrhs, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_copy_rows<T><<<n, 128, 0, s>>>(src_row, dst_row, len, src, lds, dst, ldd, nrhs);
  return cudaGetLastError();
}

#define H2SP_APPLY_INSTANTIATE(T)                                                                                      \
  template cudaError_t launch_apply_qt<T>(const ApItem *, int, const T *, const T *, int64_t, T *, int64_t, T *,       \
                                          int64_t, int, cudaStream_t, int);                                            \
  template cudaError_t launch_apply_q<T>(const ApItem *, int, const T *, const T *, int64_t, const T *, int64_t, T *,  \
                                         int64_t, int, cudaStream_t, int);                                             \
  template cudaError_t launch_copy_rows<T>(const int64_t *, const int64_t *, const int32_t *, int, const T *, int64_t, \
                                           T *, int64_t, int, cudaStream_t);
H2SP_APPLY_INSTANTIATE(double)
H2SP_APPLY_INSTANTIATE(float)
#undef H2SP_APPLY_INSTANTIATE

template <typename TS>
cudaError_t launch_spmv(const int64_t *brow_ptr, const int32_t *bcol, const int64_t *val_off, const int64_t *node_off,
                        int nnodes, const TS *vals, const double *x, int64_t ldx, double *y, int64_t ldy, int nrhs,
                        cudaStream_t s) {
  if (nnodes == 0) return cudaSuccess;
  for (int r0 = 0; r0 < nrhs; r0 += kRhs)
    k_spmv<TS><<<nnodes, 128, 0, s>>>(brow_ptr, bcol, val_off, node_off, vals, x + r0 * ldx, ldx, y + r0 * ldy, ldy,
                                      std::min(kRhs, nrhs - r0));
  return cudaGetLastError();
}

template cudaError_t launch_spmv<double>(const int64_t *, const int32_t *, const int64_t *, const int64_t *, int,
                                         const double *, const double *, int64_t, double *, int64_t, int,
                                         cudaStream_t);
template cudaError_t launch_spmv<float>(const int64_t *, const int32_t *, const int64_t *, const int64_t *, int,
                                        const float *, const double *, int64_t, double *, int64_t, int, cudaStream_t);

cudaError_t launch_h2_matvec(const H2Dev &h, const int32_t *level_ptr_host, const int32_t *child_start,
                             const int32_t *child_cnt, int depth, const double *x, int64_t ldx, double *y,
                             int64_t ldy, int nrhs, double *xh, double *yh, int64_t ldh, cudaStream_t s) {
  const int nleaf = level_ptr_host[depth + 1] - level_ptr_host[depth];
  const int ncl = level_ptr_host[depth + 1];
  for (int r0 = 0; r0 < nrhs; r0 += kRhs) {
    const int nr = std::min(kRhs, nrhs - r0);
    const double *xr = x + r0 * ldx;
    double *yr = y + r0 * ldy;
    k_h2_leaf_up<<<nleaf, kMvThreads, 0, s>>>(h, xr, ldx, xh, ldh, nr);
    for (int d = depth - 1; d >= 0; --d) {
      const int lo = level_ptr_host[d], hi = level_ptr_host[d + 1];
      k_h2_up<<<hi - lo, kMvThreads, 0, s>>>(h, child_start, child_cnt, lo, xh, ldh, nr);
    }
    const bool narrow = nr <= 4 && h.max_leaf <= 128;
    if (narrow && nr == 1)
      k_h2_couple_nw<1><<<ncl, kNwThreads, 0, s>>>(h, xh, yh, ldh, nr);
    else if (narrow)
      k_h2_couple_nw<4><<<ncl, kNwThreads, 0, s>>>(h, xh, yh, ldh, nr);
    else
      k_h2_couple<<<ncl, kMvThreads, 0, s>>>(h, xh, yh, ldh, nr);
    for (int d = 1; d <= depth; ++d) {
      const int lo = level_ptr_host[d], hi = level_ptr_host[d + 1];
      k_h2_down<<<hi - lo, kMvThreads, 0, s>>>(h, lo, yh, ldh, nr);
    }
    const int nlarge = h.nleaf_large;
    if (narrow && nr == 1) {
      k_h2_leaf_out_nw<1><<<nleaf, kNwThreads, 0, s>>>(h, xr, ldx, yh, ldh, yr, ldy, nr);
    } else if (narrow) {
      k_h2_leaf_out_nw<4><<<nleaf, kNwThreads, 0, s>>>(h, xr, ldx, yh, ldh, yr, ldy, nr);
    } else {
      if (nleaf > nlarge) k_h2_leaf_out<<<nleaf - nlarge, kMvThreads, 0, s>>>(h, xr, ldx, yh, ldh, yr, ldy, nr);
      if (nlarge > 0)
        k_h2_leaf_out_large<<<nlarge, kMvThreads, 0, s>>>(h, nleaf - nlarge, xr, ldx, yh, ldh, yr, ldy, nr);
    }
  }
  return cudaGetLastError();
}

// Workspace of h2sp_h2_matvec_static: the two coefficient vectors of the
// upward and downward passes live in this file-scope device array, so that
// entry point allocates nothing.  Every GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) double g_h2_static_scratch[kStaticScratchElems];

cudaError_t static_scratch_address(double **out) {
  // cudaGetSymbolAddress gives the device address of the array for the
  // current device; the host-side name itself is not a device pointer.
  static std::mutex mu;
  static double *addr[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_h2_static_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = static_cast<double *>(p);
  }
  *out = addr[dev];
  return cudaSuccess;
}

cudaError_t launch_residual(const double *b, int64_t ldb, const double *y, int64_t ldy, double *r, int64_t ldr,
                            const int64_t *seg_ptr, int nseg, int64_t n, int nrhs, double *norms2, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(norms2, 0, sizeof(double) * nrhs * nseg, s);
  if (e != cudaSuccess) return e;
  const unsigned chunks = unsigned(std::max<int64_t>(1, std::min<int64_t>(64, (n / std::max(nseg, 1) + 4095) / 4096)));
  k_residual<<<dim3(chunks, nseg, nrhs), 256, 0, s>>>(b, ldb, y, ldy, r, ldr, seg_ptr, nrhs, norms2);
  return cudaGetLastError();
}

cudaError_t launch_colnorm2(const double *x, int64_t ldx, const int64_t *seg_ptr, int nseg, int64_t n, int nrhs,
                            double *norms2, cudaStream_t s) {
  return launch_residual(x, ldx, nullptr, 0, nullptr, 0, seg_ptr, nseg, n, nrhs, norms2, s);
}

cudaError_t launch_block_dots(const double *V, int64_t ldv, int64_t vstride, int nv, const double *W, int64_t ldw,
                              int64_t n, int nrhs, double *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * nv * nrhs, s);
  if (e != cudaSuccess) return e;
  k_block_dots<<<dim3(std::max(1u, grid_for(n) / 4), nv * nrhs), 256, 0, s>>>(V, ldv, vstride, nv, W, ldw, n, nrhs,
                                                                               out);
  return cudaGetLastError();
}

cudaError_t launch_block_axpy(const double *V, int64_t ldv, int64_t vstride, int nv, const double *coef, double *W,
                              int64_t ldw, int64_t n, int nrhs, cudaStream_t s) {
  k_block_axpy<<<dim3(grid_for(n), nrhs), 256, 0, s>>>(V, ldv, vstride, nv, coef, W, ldw, n);
  return cudaGetLastError();
}

cudaError_t launch_col_scale(double *X, int64_t ldx, const double *sc, int64_t n, int nrhs, cudaStream_t s) {
  k_col_scale<<<dim3(grid_for(n), nrhs), 256, 0, s>>>(X, ldx, sc, n);
  return cudaGetLastError();
}

cudaError_t launch_axpy(const double *d, int64_t ldd, double *x, int64_t ldx, int64_t n, int nrhs, cudaStream_t s) {
  k_axpy<<<dim3(grid_for(n), nrhs), 256, 0, s>>>(d, ldd, x, ldx, n);
  return cudaGetLastError();
}

cudaError_t launch_cast_d2f(const double *a, int64_t lda, float *b, int64_t ldb, int64_t n, int nrhs, cudaStream_t s) {
  k_cast<double, float><<<dim3(grid_for(n), nrhs), 256, 0, s>>>(a, lda, b, ldb, n);
  return cudaGetLastError();
}

cudaError_t launch_cast_f2d(const float *a, int64_t lda, double *b, int64_t ldb, int64_t n, int nrhs, cudaStream_t s) {
  k_cast<float, double><<<dim3(grid_for(n), nrhs), 256, 0, s>>>(a, lda, b, ldb, n);
  return cudaGetLastError();
}

}  // namespace h2sp
