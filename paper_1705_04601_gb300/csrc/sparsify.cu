// Sparsification kernels (FP64): the per-level steps of §2.1-2.3 built from
// the H^2 parameters as in §4.2-4.3.
//
//   k_householder : Q_t = [Q^b | Q^perp] and Rr_t from W_t (orthogonal
//                   completion of the cluster basis, §4.2), one CTA per cluster.
//   k_stack_w     : W_p = [Rr_c T_c] stacked over the sons c (nested bases).
//   k_coupling    : Rr_p D_pq Rrc_q^T into the next level's close block (Eq. cl1).
//   k_transform   : Y = QL^T X QR on close blocks (Eq. cl0) and on the
//                   cross-level panels, split at the basis / non-basis
//                   boundary and scattered into S or the next level (§2.2).
//
// Every block here is at most 64 x 64, so each CTA stages its operands in
// shared memory; the level's work is one launch per kernel, one CTA per item.
#include <cstdint>

#include "internal.h"
#include "kernels.h"

namespace h2sp {
namespace {

constexpr int kThreads = 256;

template <typename W>
__device__ __forceinline__ W warp_sum(W v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the CTA; every thread receives the total
template <typename W>
__device__ W block_sum(W v, W *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  W t = W(0);
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// Householder QR of W (m x k) with LAPACK's conventions and the square
// completion Q = H_0 H_1 ... H_{k'-1} I_m.
// W is the working precision (double; float for the FP32 sparsification of
// the mixed-precision path); the leaf bases are FP64 input in either case.
template <typename W>
__global__ void __launch_bounds__(kThreads) k_householder(const QItem *__restrict__ items,
                                                          const double *__restrict__ w_in,
                                                          const W *__restrict__ w_buf,
                                                          W *__restrict__ Qout, W *__restrict__ Rout) {
  const QItem it = items[blockIdx.x];
  const int m = it.m, k = it.k, kp = min(m, k);
  extern __shared__ __align__(16) unsigned char smraw_h[];
  W *A = reinterpret_cast<W *>(smraw_h);  // m x k, ld m
  W *Q = A + m * k;                       // m x m, ld m
  W *tau = Q + m * m;                     // kp
  W *red = tau + kMaxRank + 1;
  __shared__ W s_bcast;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (it.w_buf == 0) {
    const double *src = w_in + it.w;
    for (int i = tid; i < m * k; i += nt) A[i] = W(src[(i % m) + int64_t(i / m) * it.ld_w]);
  } else {
    const W *src = w_buf + it.w;
    for (int i = tid; i < m * k; i += nt) A[i] = src[(i % m) + int64_t(i / m) * it.ld_w];
  }
  __syncthreads();
  for (int j = 0; j < kp; ++j) {
    W part = W(0);
    for (int i = j + 1 + tid; i < m; i += nt) part += A[i + j * m] * A[i + j * m];
    const W s2 = block_sum(part, red);
    if (tid == 0) {
      W t = W(0);
      if (s2 != W(0)) {
        const W alpha = A[j + j * m];
        const W beta = -copysign(hypot(alpha, sqrt(s2)), alpha);
        t = (beta - alpha) / beta;
        s_bcast = W(1) / (alpha - beta);
        A[j + j * m] = beta;
      }
      tau[j] = t;
    }
    __syncthreads();
    const W tj = tau[j];
    if (tj != W(0)) {
      const W scal = s_bcast;
      for (int i = j + 1 + tid; i < m; i += nt) A[i + j * m] *= scal;
      __syncthreads();
      // apply H_j to the remaining columns, one warp per column
      for (int c = j + 1 + wid; c < k; c += nw) {
        W w = W(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + j * m] * A[i + c * m];
        w = warp_sum(w) + A[j + c * m];
        const W tw = tj * w;
        if (lane == 0) A[j + c * m] -= tw;
        for (int i = j + 1 + lane; i < m; i += 32) A[i + c * m] -= tw * A[i + j * m];
      }
    }
    __syncthreads();
  }
  // Rr: upper trapezoid of A[:kp, :k]
  W *R = Rout + it.rr;
  for (int i = tid; i < kp * k; i += nt) {
    const int r = i % kp, c = i / kp;
    R[i] = (r <= c) ? A[r + c * m] : W(0);
  }
  // Q = H_0 ... H_{kp-1} I, applied from the last reflector backwards
  for (int i = tid; i < m * m; i += nt) Q[i] = ((i % m) == (i / m)) ? W(1) : W(0);
  __syncthreads();
  for (int j = kp - 1; j >= 0; --j) {
    const W tj = tau[j];
    if (tj != W(0)) {
      for (int c = j + wid; c < m; c += nw) {
        W w = W(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + j * m] * Q[i + c * m];
        w = warp_sum(w) + Q[j + c * m];
        const W tw = tj * w;
        if (lane == 0) Q[j + c * m] -= tw;
        for (int i = j + 1 + lane; i < m; i += 32) Q[i + c * m] -= tw * A[i + j * m];
      }
    }
    __syncthreads();
  }
  W *Qg = Qout + it.q;
  for (int i = tid; i < m * m; i += nt) Qg[i] = Q[i];
}

// rows [off_c, off_c + kp_c) of W_parent = Rr_c (kp_c x k_c) * T_c (k_c x k_p)
template <typename W>
__global__ void __launch_bounds__(kThreads) k_stack_w(const WItem *__restrict__ items, const W *__restrict__ Rr,
                                                      const double *__restrict__ Tr, W *__restrict__ Wout) {
  const WItem it = items[blockIdx.x];
  const W *R = Rr + it.rr_c;
  const double *T = Tr + it.t_c;
  W *out = Wout + it.w_dst;
  for (int i = threadIdx.x; i < it.kp_c * it.k_p; i += blockDim.x) {
    const int r = i % it.kp_c, c = i / it.kp_c;
    W acc = W(0);
    for (int q = 0; q < it.k_c; ++q) acc += R[r + q * it.kp_c] * W(T[q + c * it.k_c]);
    out[r + int64_t(c) * it.ld_w] = acc;
  }
}

// F = Rr_p (kp_p x k_p) * D (k_p x k_q) * Rrc_q^T (k_q x kp_q)
template <typename W>
__global__ void __launch_bounds__(kThreads) k_coupling(const CItem *__restrict__ items, const W *__restrict__ Rr,
                                                       const W *__restrict__ Rrc, const double *__restrict__ Dc,
                                                       W *const *__restrict__ dst_base) {
  const CItem it = items[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw_c[];
  const int kpp = it.kp_p, kpn = it.k_p, kqq = it.kp_q, kqn = it.k_q;
  W *sD = reinterpret_cast<W *>(smraw_c);  // kpn x kqn
  W *sRq = sD + kpn * kqn;                 // kqq x kqn
  W *sT = sRq + kqq * kqn;                 // kpn x kqq
  W *sRp = sT + kpn * kqq;                 // kpp x kpn
  const int tid = threadIdx.x, nt = blockDim.x;
  const double *D = Dc + it.dcoup;
  const W *Rq = Rrc + it.rr_q;
  const W *Rp = Rr + it.rr_p;
  for (int i = tid; i < kpn * kqn; i += nt) sD[i] = W(D[i]);
  for (int i = tid; i < kqq * kqn; i += nt) sRq[i] = Rq[i];
  for (int i = tid; i < kpp * kpn; i += nt) sRp[i] = Rp[i];
  __syncthreads();
  for (int i = tid; i < kpn * kqq; i += nt) {
    const int r = i % kpn, c = i / kpn;
    W acc = W(0);
    for (int q = 0; q < kqn; ++q) acc += sD[r + q * kpn] * sRq[c + q * kqq];
    sT[i] = acc;
  }
  __syncthreads();
  W *out = dst_base[it.dst_buf] + it.dst;
  for (int i = tid; i < kpp * kqq; i += nt) {
    const int r = i % kpp, c = i / kpp;
    W acc = W(0);
    for (int q = 0; q < kpn; ++q) acc += sRp[r + q * kpp] * sT[q + c * kpn];
    out[r + int64_t(c) * it.ld] = acc;
  }
}

// src_base[0] is the FP64 close-block input, src_base[1..3] working-precision
// level buffers; every destination is in the working precision.
template <typename W>
__global__ void __launch_bounds__(kThreads) k_transform(const XItem *__restrict__ items,
                                                        const void *const *__restrict__ src_base,
                                                        const W *__restrict__ Qrow, const W *__restrict__ Qcol,
                                                        W *const *__restrict__ dst_base) {
  const XItem it = items[blockIdx.x];
  const int rows = it.rows, cols = it.cols;
  extern __shared__ __align__(16) unsigned char smraw_t[];
  W *X = reinterpret_cast<W *>(smraw_t);  // rows x cols, ld rows
  W *Qs = X + kMaxBlock * kMaxBlock;      // up to 64 x 64
  W *T = Qs + kMaxBlock * kMaxBlock;      // rows x cols
  const int tid = threadIdx.x, nt = blockDim.x;
  if (it.src_buf == SRC_NEAR) {
    const double *src = static_cast<const double *>(src_base[0]) + it.src;
    for (int i = tid; i < rows * cols; i += nt) X[i] = W(src[(i % rows) + int64_t(i / rows) * it.ld_src]);
  } else {
    const W *src = static_cast<const W *>(src_base[it.src_buf]) + it.src;
    for (int i = tid; i < rows * cols; i += nt) X[i] = src[(i % rows) + int64_t(i / rows) * it.ld_src];
  }
  W *cur = X;
  if (it.qR >= 0) {
    const W *QR = ((it.qside & 2) ? Qcol : Qrow) + it.qR;  // cols x cols
    for (int i = tid; i < cols * cols; i += nt) Qs[i] = QR[i];
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
    const W *QL = ((it.qside & 1) ? Qcol : Qrow) + it.qL;  // rows x rows, stored transposed in smem
    for (int i = tid; i < rows * rows; i += nt) {
      const int r = i % rows, c = i / rows;
      Qs[c + r * rows] = QL[i];
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
}

}  // namespace

template <typename W>
cudaError_t launch_householder(const QItem *items, int n, const double *w_in, const W *w_buf, W *Q, W *Rr, int max_m,
                               int max_k, cudaStream_t s, Prof *prof) {
  if (n == 0) return cudaSuccess;
  size_t smem = sizeof(W) * (size_t(max_m) * max_k + size_t(max_m) * max_m + kMaxRank + 1 + 64);
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_householder<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_done = true;
  }
  const size_t e0 = prof->begin();
  k_householder<W><<<n, kThreads, smem, s>>>(items, w_in, w_buf, Q, Rr);
  prof->end(P_HOUSEHOLDER, 1, e0, 0.0);
  return cudaGetLastError();
}

template <typename W>
cudaError_t launch_stack_w(const WItem *items, int n, const W *Rr, const double *T, W *Wout, cudaStream_t s,
                           Prof *prof) {
  if (n == 0) return cudaSuccess;
  const size_t e0 = prof->begin();
  k_stack_w<W><<<n, 64, 0, s>>>(items, Rr, T, Wout);
  prof->end(P_COUPLING, 1, e0, 0.0);
  return cudaGetLastError();
}

template <typename W>
cudaError_t launch_coupling(const CItem *items, int n, const W *Rr, const W *Rrc, const double *Dc,
                            W *const *dst_base, int max_k, cudaStream_t s, Prof *prof) {
  if (n == 0) return cudaSuccess;
  size_t smem = sizeof(W) * 4 * size_t(max_k) * max_k;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_coupling<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_done = true;
  }
  const size_t e0 = prof->begin();
  k_coupling<W><<<n, 128, smem, s>>>(items, Rr, Rrc, Dc, dst_base);
  prof->end(P_COUPLING, 1, e0, 0.0);
  return cudaGetLastError();
}

template <typename W>
cudaError_t launch_transform(const XItem *items, int n, const void *const *src_base, const W *Qrow, const W *Qcol,
                             W *const *dst_base, cudaStream_t s, Prof *prof, double flops) {
  if (n == 0) return cudaSuccess;
  size_t smem = sizeof(W) * 3 * size_t(kMaxBlock) * kMaxBlock;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_transform<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    attr_done = true;
  }
  const size_t e0 = prof->begin();
  k_transform<W><<<n, kThreads, smem, s>>>(items, src_base, Qrow, Qcol, dst_base);
  prof->end(P_TRANSFORM, 1, e0, flops);
  return cudaGetLastError();
}

#define H2SP_SPARSIFY_INSTANTIATE(W)                                                                                  \
  template cudaError_t launch_householder<W>(const QItem *, int, const double *, const W *, W *, W *, int, int,      \
                                             cudaStream_t, Prof *);                                                  \
  template cudaError_t launch_stack_w<W>(const WItem *, int, const W *, const double *, W *, cudaStream_t, Prof *); \
  template cudaError_t launch_coupling<W>(const CItem *, int, const W *, const W *, const double *, W *const *, int, \
                                          cudaStream_t, Prof *);                                                     \
  template cudaError_t launch_transform<W>(const XItem *, int, const void *const *, const W *, const W *, W *const *, \
                                           cudaStream_t, Prof *, double);
H2SP_SPARSIFY_INSTANTIATE(double)
H2SP_SPARSIFY_INSTANTIATE(float)
#undef H2SP_SPARSIFY_INSTANTIATE

}  // namespace h2sp
