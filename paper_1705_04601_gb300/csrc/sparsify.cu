// Sparsification kernels: the per-level steps of §2.1-2.3 built from the H^2
// parameters as in §4.2-4.3.  The Householder completions, the stacked bases
// and the coupling projections are FP64 (U and V orthogonal to FP64
// accuracy); the close-block products and everything stored into S are FP64,
// or FP32 when S only feeds an FP32 preconditioner.
//
//   k_householder : Q_t = [Q^b | Q^perp] and Rr_t from W_t (orthogonal
//                   completion of the cluster basis, §4.2), one CTA per cluster.
//   k_stack_w     : W_p = [Rr_c T_c] stacked over the sons c (nested bases).
//   k_coupling    : Rr_p D_pq Rrc_q^T into the next level's close block (Eq. cl1).
//   k_transform   : Y = QL^T X QR on close blocks (Eq. cl0) and on the
//                   cross-level panels, split at the basis / non-basis
//                   boundary and scattered into S or the next level (§2.2).
//
// Blocks of at most 64 x 64 are staged whole in shared memory, one CTA per
// item.  Larger blocks (up to kMaxLargeBlock: 3D leaves, upper levels stacked
// from up to eight sons) take k_householder_large, which keeps Q in its
// global output, and k_transform_large, which streams the block and the Q
// factors from global memory and keeps one 16-column slab of the product in
// shared memory.  A level's small items come first in its lists; each group
// is one launch.
#include <cstdint>

#include "internal.h"
#include "kernels.h"

namespace h2sp {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the CTA; every thread receives the total
__device__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// Householder QR of W (m x k) with LAPACK's conventions and the square
// completion Q = H_0 H_1 ... H_{k'-1} I_m.
__global__ void __launch_bounds__(kThreads) k_householder(const QItem *__restrict__ items, int n_items,
                                                          const double *__restrict__ w_in,
                                                          const double *__restrict__ w_buf,
                                                          double *__restrict__ Qout, double *__restrict__ Rout) {
  // persistent: each CTA walks the work list with a stride of the grid
  for (int ib = blockIdx.x; ib < n_items; ib += gridDim.x) {
  const QItem it = items[ib];
  const int m = it.m, k = it.k, kp = min(m, k);
  extern __shared__ double sm[];
  double *A = sm;              // m x k, ld m
  double *Q = A + m * k;       // m x m, ld m
  double *tau = Q + m * m;     // kp
  double *red = tau + kMaxRank + 1;
  __shared__ double s_bcast;
  const double *W = (it.w_buf == 0 ? w_in : w_buf) + it.w;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int i = tid; i < m * k; i += nt) A[i] = W[(i % m) + int64_t(i / m) * it.ld_w];
  __syncthreads();
  for (int j = 0; j < kp; ++j) {
    double part = 0.0;
    for (int i = j + 1 + tid; i < m; i += nt) part += A[i + j * m] * A[i + j * m];
    const double s2 = block_sum(part, red);
    if (tid == 0) {
      double t = 0.0;
      if (s2 != 0.0) {
        const double alpha = A[j + j * m];
        const double beta = -copysign(hypot(alpha, sqrt(s2)), alpha);
        t = (beta - alpha) / beta;
        s_bcast = 1.0 / (alpha - beta);
        A[j + j * m] = beta;
      }
      tau[j] = t;
    }
    __syncthreads();
    const double tj = tau[j];
    if (tj != 0.0) {
      const double scal = s_bcast;
      for (int i = j + 1 + tid; i < m; i += nt) A[i + j * m] *= scal;
      __syncthreads();
      // apply H_j to the remaining columns, one warp per column
      for (int c = j + 1 + wid; c < k; c += nw) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + j * m] * A[i + c * m];
        w = warp_sum(w) + A[j + c * m];
        const double tw = tj * w;
        if (lane == 0) A[j + c * m] -= tw;
        for (int i = j + 1 + lane; i < m; i += 32) A[i + c * m] -= tw * A[i + j * m];
      }
    }
    __syncthreads();
  }
  // Rr: upper trapezoid of A[:kp, :k]
  double *R = Rout + it.rr;
  for (int i = tid; i < kp * k; i += nt) {
    const int r = i % kp, c = i / kp;
    R[i] = (r <= c) ? A[r + c * m] : 0.0;
  }
  // Q = H_0 ... H_{kp-1} I, applied from the last reflector backwards
  for (int i = tid; i < m * m; i += nt) Q[i] = ((i % m) == (i / m)) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = kp - 1; j >= 0; --j) {
    const double tj = tau[j];
    if (tj != 0.0) {
      for (int c = j + wid; c < m; c += nw) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + j * m] * Q[i + c * m];
        w = warp_sum(w) + Q[j + c * m];
        const double tw = tj * w;
        if (lane == 0) Q[j + c * m] -= tw;
        for (int i = j + 1 + lane; i < m; i += 32) Q[i + c * m] -= tw * A[i + j * m];
      }
    }
    __syncthreads();
  }
  double *Qg = Qout + it.q;
  for (int i = tid; i < m * m; i += nt) Qg[i] = Q[i];
  __syncthreads();  // shared memory is reused by the next item
  }
}

// k_householder for m > kMaxBlock: the same reflectors and completion, with W
// (m x k) in shared memory and Q formed in place in its global output.  Each
// column of Q is updated by one warp per reflector; the CTA barrier between
// reflectors orders the global writes.
__global__ void __launch_bounds__(kThreads) k_householder_large(const QItem *__restrict__ items, int n_items,
                                                                const double *__restrict__ w_in,
                                                                const double *__restrict__ w_buf,
                                                                double *__restrict__ Qout, double *__restrict__ Rout) {
  // persistent: each CTA walks the work list with a stride of the grid
  for (int ib = blockIdx.x; ib < n_items; ib += gridDim.x) {
  const QItem it = items[ib];
  const int m = it.m, k = it.k, kp = min(m, k);
  extern __shared__ double sm[];
  double *A = sm;              // m x k, ld m
  double *tau = A + m * k;     // kp
  double *red = tau + kMaxRank + 1;
  __shared__ double s_bcast;
  const double *W = (it.w_buf == 0 ? w_in : w_buf) + it.w;
  double *Q = Qout + it.q;     // m x m, ld m
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int i = tid; i < m * k; i += nt) A[i] = W[(i % m) + int64_t(i / m) * it.ld_w];
  __syncthreads();
  for (int j = 0; j < kp; ++j) {
    double part = 0.0;
    for (int i = j + 1 + tid; i < m; i += nt) part += A[i + j * m] * A[i + j * m];
    const double s2 = block_sum(part, red);
    if (tid == 0) {
      double t = 0.0;
      if (s2 != 0.0) {
        const double alpha = A[j + j * m];
        const double beta = -copysign(hypot(alpha, sqrt(s2)), alpha);
        t = (beta - alpha) / beta;
        s_bcast = 1.0 / (alpha - beta);
        A[j + j * m] = beta;
      }
      tau[j] = t;
    }
    __syncthreads();
    const double tj = tau[j];
    if (tj != 0.0) {
      const double scal = s_bcast;
      for (int i = j + 1 + tid; i < m; i += nt) A[i + j * m] *= scal;
      __syncthreads();
      for (int c = j + 1 + wid; c < k; c += nw) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + j * m] * A[i + c * m];
        w = warp_sum(w) + A[j + c * m];
        const double tw = tj * w;
        __syncwarp();
        if (lane == 0) A[j + c * m] -= tw;
        for (int i = j + 1 + lane; i < m; i += 32) A[i + c * m] -= tw * A[i + j * m];
      }
    }
    __syncthreads();
  }
  double *R = Rout + it.rr;
  for (int i = tid; i < kp * k; i += nt) {
    const int r = i % kp, c = i / kp;
    R[i] = (r <= c) ? A[r + c * m] : 0.0;
  }
  for (int64_t i = tid; i < int64_t(m) * m; i += nt) Q[i] = ((i % m) == (i / m)) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = kp - 1; j >= 0; --j) {
    const double tj = tau[j];
    if (tj != 0.0) {
      for (int c = j + wid; c < m; c += nw) {
        double *qc = Q + int64_t(c) * m;
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + j * m] * qc[i];
        w = warp_sum(w) + qc[j];
        const double tw = tj * w;
        __syncwarp();
        if (lane == 0) qc[j] -= tw;
        for (int i = j + 1 + lane; i < m; i += 32) qc[i] -= tw * A[i + j * m];
      }
    }
    __syncthreads();
  }
  __syncthreads();  // shared memory is reused by the next item
  }
}

// rows [off_c, off_c + kp_c) of W_parent = Rr_c (kp_c x k_c) * T_c (k_c x k_p)
__global__ void __launch_bounds__(kThreads) k_stack_w(const WItem *__restrict__ items, int n_items, const double *__restrict__ Rr,
                                                      const double *__restrict__ Tr, double *__restrict__ W) {
  // persistent: each CTA walks the work list with a stride of the grid
  for (int ib = blockIdx.x; ib < n_items; ib += gridDim.x) {
  const WItem it = items[ib];
  const double *R = Rr + it.rr_c;
  const double *T = Tr + it.t_c;
  double *out = W + it.w_dst;
  for (int i = threadIdx.x; i < it.kp_c * it.k_p; i += blockDim.x) {
    const int r = i % it.kp_c, c = i / it.kp_c;
    double acc = 0.0;
    for (int q = 0; q < it.k_c; ++q) acc += R[r + q * it.kp_c] * T[q + c * it.k_c];
    out[r + int64_t(c) * it.ld_w] = acc;
  }
  __syncthreads();  // shared memory is reused by the next item
  }
}

// F = Rr_p (kp_p x k_p) * D (k_p x k_q) * Rrc_q^T (k_q x kp_q)
template <typename W>
__global__ void __launch_bounds__(kThreads) k_coupling(const CItem *__restrict__ items, int n_items, const double *__restrict__ Rr,
                                                       const double *__restrict__ Rrc, const double *__restrict__ Dc,
                                                       W *const *__restrict__ dst_base) {
  // persistent: each CTA walks the work list with a stride of the grid
  for (int ib = blockIdx.x; ib < n_items; ib += gridDim.x) {
  const CItem it = items[ib];
  extern __shared__ double sm[];
  const int kpp = it.kp_p, kpn = it.k_p, kqq = it.kp_q, kqn = it.k_q;
  double *sD = sm;                  // kpn x kqn
  double *sRq = sD + kpn * kqn;     // kqq x kqn
  double *sT = sRq + kqq * kqn;     // kpn x kqq
  double *sRp = sT + kpn * kqq;     // kpp x kpn
  const int tid = threadIdx.x, nt = blockDim.x;
  const double *D = Dc + it.dcoup;
  const double *Rq = Rrc + it.rr_q;
  const double *Rp = Rr + it.rr_p;
  for (int i = tid; i < kpn * kqn; i += nt) sD[i] = D[i];
  for (int i = tid; i < kqq * kqn; i += nt) sRq[i] = Rq[i];
  for (int i = tid; i < kpp * kpn; i += nt) sRp[i] = Rp[i];
  __syncthreads();
  for (int i = tid; i < kpn * kqq; i += nt) {
    const int r = i % kpn, c = i / kpn;
    double acc = 0.0;
    for (int q = 0; q < kqn; ++q) acc += sD[r + q * kpn] * sRq[c + q * kqq];
    sT[i] = acc;
  }
  __syncthreads();
  W *out = dst_base[it.dst_buf] + it.dst;
  for (int i = tid; i < kpp * kqq; i += nt) {
    const int r = i % kpp, c = i / kpp;
    double acc = 0.0;
    for (int q = 0; q < kpn; ++q) acc += sRp[r + q * kpp] * sT[q + c * kpn];
    out[r + int64_t(c) * it.ld] = W(acc);
  }
  __syncthreads();  // shared memory is reused by the next item
  }
}

// W is the arithmetic and storage type of the close blocks and cross-level
// panels being transformed: double, or float for the FP32 products of the
// mixed-precision path.  src_base[0] is the FP64 close-block input and
// src_base[1..3] level buffers of type W; Q is FP64 and rounded to W on load.
template <typename W>
__global__ void __launch_bounds__(kThreads) k_transform(const XItem *__restrict__ items, int n_items,
                                                        const void *const *__restrict__ src_base,
                                                        const double *__restrict__ Qrow, const double *__restrict__ Qcol,
                                                        W *const *__restrict__ dst_base) {
  // persistent: each CTA walks the work list with a stride of the grid
  for (int ib = blockIdx.x; ib < n_items; ib += gridDim.x) {
  const XItem it = items[ib];
  const int rows = it.rows, cols = it.cols;
  extern __shared__ __align__(16) unsigned char smraw_t[];
  W *X = reinterpret_cast<W *>(smraw_t);  // rows x cols, ld rows
  W *Qs = X + kMaxBlock * kMaxBlock;      // up to 64 x 64
  W *T = Qs + kMaxBlock * kMaxBlock;      // rows x cols
  const int tid = threadIdx.x, nt = blockDim.x;
  if (it.src_buf == SRC_NEAR) {
    const double *src = static_cast<const double *>(src_base[SRC_NEAR]) + it.src;
    for (int i = tid; i < rows * cols; i += nt) X[i] = W(src[(i % rows) + int64_t(i / rows) * it.ld_src]);
  } else {
    const W *src = static_cast<const W *>(src_base[it.src_buf]) + it.src;
    for (int i = tid; i < rows * cols; i += nt) X[i] = src[(i % rows) + int64_t(i / rows) * it.ld_src];
  }
  W *cur = X;
  if (it.qR >= 0) {
    const double *QR = ((it.qside & 2) ? Qcol : Qrow) + it.qR;  // cols x cols
    for (int i = tid; i < cols * cols; i += nt) Qs[i] = W(QR[i]);
    __syncthreads();
    for (int i = tid; i < rows * cols; i += nt) {
      const int r = i % rows, c = i / rows;
      const W *qc = Qs + c * cols;
      W acc = W(0);
      for (int q = 0; q < cols; ++q) acc += X[r + q * rows] * qc[q];
      T[i] = acc;
    }
    cur = T;
    __syncthreads();
  }
  if (it.qL >= 0) {
    const double *QL = ((it.qside & 1) ? Qcol : Qrow) + it.qL;  // rows x rows, stored transposed in smem
    for (int i = tid; i < rows * rows; i += nt) {
      const int r = i % rows, c = i / rows;
      Qs[c + r * rows] = W(QL[i]);
    }
    __syncthreads();
    W *out = (cur == X) ? T : X;
    for (int i = tid; i < rows * cols; i += nt) {
      const int r = i % rows, c = i / rows;
      const W *tc = cur + c * rows;
      W acc = W(0);
      for (int q = 0; q < rows; ++q) acc += Qs[r + q * rows] * tc[q];
      out[i] = acc;
    }
    cur = out;
  }
  __syncthreads();
  const int kr = it.kr, kc = it.kc;
#pragma unroll
  for (int qd = 0; qd < 4; ++qd) {
    if (it.dst[qd] < 0) continue;
    const int r0 = (qd & 2) ? kr : 0, r1 = (qd & 2) ? rows : kr;
    const int c0 = (qd & 1) ? kc : 0, c1 = (qd & 1) ? cols : kc;
    const int nr = r1 - r0, nc = c1 - c0;
    W *out = dst_base[it.dst_buf[qd]] + it.dst[qd];
    const int ld = it.ld[qd];
    for (int i = tid; i < nr * nc; i += nt) {
      const int r = i % nr, c = i / nr;
      out[r + int64_t(c) * ld] = cur[(r0 + r) + (c0 + c) * rows];
    }
  }
  __syncthreads();  // shared memory is reused by the next item
  }
}

// k_transform for blocks above kMaxBlock rows or columns: Y = QL^T X QR by
// output slabs of kSlab columns, register-tiled.  Per slab J:
//   stage 1  T_J = X QR[:, J]      (rows x kSlab, kept in shared memory)
//   stage 2  Y_J = QL^T T_J        (rows x kSlab)
// and each element of Y_J goes to its quadrant's destination.  Thread (tr,
// tc) of the 32 x 8 grid owns rows tr + 32 i (i < ceil(rows / 32) <= 12) and
// the four columns 4 tc .. 4 tc + 3 of the slab: 48 accumulators, so every
// operand value a thread loads from shared memory serves four (or twelve)
// multiply-adds.  The K dimension streams through shared memory in chunks of
// kKc: X (or QL^T) as kKc columns of all rows, QR (or T) as kKc rows of the
// slab.  Without QR (QL) the stage is a copy.  The FP32 form is held to 128
// registers (two CTAs per SM): with one CTA of 8 warps per SM nothing covers
// the latency of each chunk's global loads, and the FMA pipe idled (9 %).
constexpr int kSlab = 32;
constexpr int kKc = 8;
constexpr int kTrMax = kMaxLargeBlock / 32;  // row groups per thread

template <typename W>
__global__ void __launch_bounds__(kThreads, sizeof(W) == 4 ? 2 : 1)
    k_transform_large(const XItem *__restrict__ items, int n_items, const void *const *__restrict__ src_base,
                      const double *__restrict__ Qrow, const double *__restrict__ Qcol,
                      W *const *__restrict__ dst_base) {
  static_assert(kThreads == 256 && kSlab == 32, "thread grid of the tiles");
  // persistent: each CTA walks the work list with a stride of the grid
  for (int ib = blockIdx.x; ib < n_items; ib += gridDim.x) {
  const XItem it = items[ib];
  const int rows = it.rows, cols = it.cols;
  const int nti = (rows + 31) / 32;  // row groups in use
  extern __shared__ __align__(16) unsigned char smraw_l[];
  const int lda = rows + 1;                 // odd: the transposed stores of QL^T spread over the banks
  W *sT = reinterpret_cast<W *>(smraw_l);  // rows x kSlab, ld rows (the slab of T = X QR)
  W *sA = sT + size_t(rows) * kSlab;        // kKc columns of X or of QL^T, ld lda
  W *sB = sA + size_t(lda) * kKc;           // kKc x kSlab of QR (row-major)
  const int tid = threadIdx.x, tr = tid & 31, tc = tid >> 5;
  const bool near = it.src_buf == SRC_NEAR;
  const double *srcd = near ? static_cast<const double *>(src_base[SRC_NEAR]) + it.src : nullptr;
  const W *srcw = near ? nullptr : static_cast<const W *>(src_base[it.src_buf]) + it.src;
  const int64_t lds = it.ld_src;
  const double *QR = it.qR >= 0 ? ((it.qside & 2) ? Qcol : Qrow) + it.qR : nullptr;  // cols x cols
  const double *QL = it.qL >= 0 ? ((it.qside & 1) ? Qcol : Qrow) + it.qL : nullptr;  // rows x rows
  auto xval = [&](int r, int q) -> W { return near ? W(srcd[r + int64_t(q) * lds]) : srcw[r + int64_t(q) * lds]; };
  const int kr = it.kr, kc = it.kc;
  for (int c0 = 0; c0 < cols; c0 += kSlab) {
    const int cb = min(kSlab, cols - c0);
    // ---- stage 1: sT = X QR[:, c0 : c0 + cb] ----
    if (QR) {
      W acc[kTrMax][4];
#pragma unroll
      for (int i = 0; i < kTrMax; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = W(0);
      for (int q0 = 0; q0 < cols; q0 += kKc) {
        const int kn = min(kKc, cols - q0);
        __syncthreads();  // sA / sB free
        for (int e = tid; e < rows * kKc; e += kThreads) {
          const int r = e % rows, k = e / rows;  // down the columns of X (coalesced)
          sA[r + k * lda] = k < kn ? xval(r, q0 + k) : W(0);
        }
        for (int e = tid; e < kKc * kSlab; e += kThreads) {
          const int k = e % kKc, c = e / kKc;  // down the columns of QR
          sB[k * kSlab + c] = (k < kn && c < cb) ? W(QR[(q0 + k) + int64_t(c0 + c) * cols]) : W(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKc; ++k) {
          W b[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = sB[k * kSlab + 4 * tc + j];
#pragma unroll
          for (int i = 0; i < kTrMax; ++i) {
            if (i >= nti) break;
            const int r = tr + 32 * i;
            const W a = r < rows ? sA[r + k * lda] : W(0);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += a * b[j];
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kTrMax; ++i) {
        if (i >= nti) break;
        const int r = tr + 32 * i;
        if (r < rows)
#pragma unroll
          for (int j = 0; j < 4; ++j) sT[r + (4 * tc + j) * rows] = acc[i][j];
      }
    } else {
      __syncthreads();
      for (int e = tid; e < rows * kSlab; e += kThreads) {
        const int r = e % rows, c = e / rows;
        sT[e] = c < cb ? xval(r, c0 + c) : W(0);
      }
    }
    __syncthreads();
    // ---- stage 2: Y = QL^T sT, then the quadrant scatter ----
    W y[kTrMax][4];
    if (QL) {
#pragma unroll
      for (int i = 0; i < kTrMax; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) y[i][j] = W(0);
      for (int q0 = 0; q0 < rows; q0 += kKc) {
        const int kn = min(kKc, rows - q0);
        __syncthreads();  // sA free
        // sA[r + k lda] = QL^T[r][q0 + k] = QL[(q0 + k) + r rows]
        for (int e = tid; e < rows * kKc; e += kThreads) {
          const int k = e % kKc, r = e / kKc;  // down the columns of QL
          sA[r + k * lda] = k < kn ? W(QL[(q0 + k) + int64_t(r) * rows]) : W(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKc; ++k) {
          if (k >= kn) break;
          W b[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = sT[(q0 + k) + (4 * tc + j) * rows];
#pragma unroll
          for (int i = 0; i < kTrMax; ++i) {
            if (i >= nti) break;
            const int r = tr + 32 * i;
            const W a = r < rows ? sA[r + k * lda] : W(0);
#pragma unroll
            for (int j = 0; j < 4; ++j) y[i][j] += a * b[j];
          }
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < kTrMax; ++i) {
        if (i >= nti) break;
        const int r = tr + 32 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) y[i][j] = r < rows ? sT[r + (4 * tc + j) * rows] : W(0);
      }
    }
#pragma unroll
    for (int i = 0; i < kTrMax; ++i) {
      if (i >= nti) break;
      const int r = tr + 32 * i;
      if (r >= rows) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cc = c0 + 4 * tc + j;
        if (4 * tc + j >= cb) continue;
        const bool lo_r = r < kr, lo_c = cc < kc;
        // quadrant of (r, cc): 0 basis x basis, 1 basis x non-basis, 2 non-basis x basis, 3 non-basis x non-basis
        const int qd = (lo_r ? 0 : 2) + (lo_c ? 0 : 1);
        const int64_t doff = it.dst[qd];
        if (doff >= 0) {
          const int rr = lo_r ? r : r - kr, ccl = lo_c ? cc : cc - kc;
          dst_base[it.dst_buf[qd]][doff + rr + int64_t(ccl) * it.ld[qd]] = y[i][j];
        }
      }
    }
    __syncthreads();  // sT is rewritten by the next slab
  }
  __syncthreads();  // shared memory is reused by the next item
  }
}

}  // namespace

cudaError_t launch_householder(const QItem *items, int n, const double *w_in, const double *w_buf, double *Q,
                               double *Rr, int max_m, int max_k, cudaStream_t s, Prof *prof) {
  if (n == 0) return cudaSuccess;
  size_t smem = sizeof(double) * (size_t(max_m) * max_k + size_t(max_m) * max_m + kMaxRank + 1 + 64);
  if (cudaError_t ea = smem_attr((const void *)k_householder, int(smem)); ea != cudaSuccess) return ea;
  const size_t e0 = prof->begin();
  k_householder<<<persistent_grid((const void *)k_householder, kThreads, smem, n), kThreads, smem, s>>>(items, n, w_in, w_buf, Q, Rr);
  prof->end(P_HOUSEHOLDER, 1, e0, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_householder_large(const QItem *items, int n, const double *w_in, const double *w_buf, double *Q,
                                     double *Rr, int max_m, int max_k, cudaStream_t s, Prof *prof) {
  if (n == 0) return cudaSuccess;
  const size_t smem = sizeof(double) * (size_t(max_m) * max_k + kMaxRank + 1 + 64);
  if (cudaError_t ea = smem_attr((const void *)k_householder_large, int(smem)); ea != cudaSuccess) return ea;
  const size_t e0 = prof->begin();
  k_householder_large<<<persistent_grid((const void *)k_householder_large, kThreads, smem, n), kThreads, smem, s>>>(items, n, w_in, w_buf, Q, Rr);
  prof->end(P_HOUSEHOLDER, 1, e0, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_stack_w(const WItem *items, int n, const double *Rr, const double *T, double *W, cudaStream_t s,
                           Prof *prof) {
  if (n == 0) return cudaSuccess;
  const size_t e0 = prof->begin();
  k_stack_w<<<persistent_grid((const void *)k_stack_w, 64, 0, n), 64, 0, s>>>(items, n, Rr, T, W);
  prof->end(P_COUPLING, 1, e0, 0.0);
  return cudaGetLastError();
}

template <typename W>
cudaError_t launch_coupling(const CItem *items, int n, const double *Rr, const double *Rrc, const double *Dc,
                            W *const *dst_base, int max_k, cudaStream_t s, Prof *prof) {
  if (n == 0) return cudaSuccess;
  size_t smem = sizeof(double) * 4 * size_t(max_k) * max_k;
  if (cudaError_t ea = smem_attr((const void *)k_coupling<W>, int(smem)); ea != cudaSuccess) return ea;
  const size_t e0 = prof->begin();
  k_coupling<W><<<persistent_grid((const void *)k_coupling<W>, 128, smem, n), 128, smem, s>>>(items, n, Rr, Rrc, Dc, dst_base);
  prof->end(P_COUPLING, 1, e0, 0.0);
  return cudaGetLastError();
}

template <typename W>
cudaError_t launch_transform(const XItem *items, int n, const void *const *src_base, const double *Qrow,
                             const double *Qcol, W *const *dst_base, cudaStream_t s, Prof *prof, double flops) {
  if (n == 0) return cudaSuccess;
  size_t smem = sizeof(W) * 3 * size_t(kMaxBlock) * kMaxBlock;
  if (cudaError_t ea = smem_attr((const void *)k_transform<W>, int(smem)); ea != cudaSuccess) return ea;
  const size_t e0 = prof->begin();
  k_transform<W><<<persistent_grid((const void *)k_transform<W>, kThreads, smem, n), kThreads, smem, s>>>(items, n, src_base, Qrow, Qcol, dst_base);
  prof->end(P_TRANSFORM, 1, e0, flops);
  return cudaGetLastError();
}

template <typename W>
cudaError_t launch_transform_large(const XItem *items, int n, const void *const *src_base, const double *Qrow,
                                   const double *Qcol, W *const *dst_base, int max_rows, int max_cols, cudaStream_t s,
                                   Prof *prof, double flops) {
  if (n == 0) return cudaSuccess;
  const size_t smem = sizeof(W) * (size_t(max_rows) * kSlab + size_t(max_rows + 1) * kKc + size_t(kKc) * kSlab);
  (void)max_cols;
  if (cudaError_t ea = smem_attr((const void *)k_transform_large<W>, int(smem)); ea != cudaSuccess) return ea;
  const size_t e0 = prof->begin();
  k_transform_large<W><<<persistent_grid((const void *)k_transform_large<W>, kThreads, smem, n), kThreads, smem, s>>>(items, n, src_base, Qrow, Qcol, dst_base);
  prof->end(P_TRANSFORM, 1, e0, flops);
  return cudaGetLastError();
}

template cudaError_t launch_coupling<double>(const CItem *, int, const double *, const double *, const double *,
                                             double *const *, int, cudaStream_t, Prof *);
template cudaError_t launch_coupling<float>(const CItem *, int, const double *, const double *, const double *,
                                            float *const *, int, cudaStream_t, Prof *);
template cudaError_t launch_transform<double>(const XItem *, int, const void *const *, const double *, const double *,
                                              double *const *, cudaStream_t, Prof *, double);
template cudaError_t launch_transform<float>(const XItem *, int, const void *const *, const double *, const double *,
                                             float *const *, cudaStream_t, Prof *, double);

template cudaError_t launch_transform_large<double>(const XItem *, int, const void *const *, const double *,
                                                    const double *, double *const *, int, int, cudaStream_t, Prof *,
                                                    double);
template cudaError_t launch_transform_large<float>(const XItem *, int, const void *const *, const double *,
                                                   const double *, float *const *, int, int, cudaStream_t, Prof *,
                                                   double);

}  // namespace h2sp
