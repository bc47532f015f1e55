// Construction of the H^2 matrix of a kernel function on the GPU (the
// parameters of Definition 4.9 that the sparsification consumes): nested
// cluster bases by tensor Chebyshev interpolation on the cluster boxes, and
// the coupling and close blocks by kernel evaluation; then, optionally, a
// recompression of the bases to a tolerance:
//   1. orthogonalise bottom-up: the leaf basis R_t = Q_t Z_t (Householder QR);
//      above, W_t = [Z_c T_c]_c stacked over the children = Q_t Z_t, and the
//      rows of Q_t that belong to child c are its transfer in the
//      orthonormal basis, Tq_c;
//   2. the couplings in the orthonormal bases, Do_ts = Z_t D_ts Z_s^T;
//   3. top-down far-field weights: the Gram matrix of everything the basis
//      of t carries, M_t = sum_s Do_ts Do_ts^T + Tq_t M_parent Tq_t^T;
//   4. its eigenvectors (two-sided Jacobi) in decreasing order, the rank
//      R_t = #{ sigma_i > tol sigma_0 } with sigma_i = sqrt(lambda_i), and
//      B_t = the first R_t eigenvectors;
//   5. the recompressed parameters: leaf basis Q_t B_t, transfers
//      B_c^T Tq_c B_parent, couplings B_t^T Do_ts B_s.
// The weights are formed as Gram matrices, so singular values are resolved
// down to about 1e-8 of the largest: tolerances below 1e-7 are refused.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.h"

namespace h2sp {
namespace {

constexpr int kCMaxP = 64;  // Chebyshev points per cluster (p^dim)

struct CGeo {
  int dim, p, P, kernel;
  double diag;
};

// kernel value for x != y, r accumulated axis by axis without contraction
__device__ __forceinline__ double kernel_at(const CGeo &g, const double *x, const double *y) {
  double r2 = 0.0;
  for (int a = 0; a < g.dim; ++a) {
    const double d = __dsub_rn(x[a], y[a]);
    r2 = __dadd_rn(r2, __dmul_rn(d, d));
  }
  switch (g.kernel) {
    case 0: return -log(sqrt(r2));            // -log r
    case 1: return 1.0 / sqrt(r2);            // 1 / r
    case 2: {                                 // e^-r / r
      const double r = sqrt(r2);
      return exp(-r) / r;
    }
    default: return exp(-r2);                 // e^{-r^2}
  }
}

// the p Chebyshev points of [lo, hi]: c + h cos((2i + 1) pi / (2p))
__device__ __forceinline__ double cheb_node(double lo, double hi, int p, int i) {
  const double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
  return c + h * cos(((2.0 * i + 1.0) * 3.141592653589793) / (2.0 * p));
}

// node alpha = a_0 + p a_1 + p^2 a_2 of a box: coordinate a = cheb_node(axis a, a_a)
__device__ __forceinline__ void tensor_node(const CGeo &g, const double *lo, const double *hi, int alpha, double *x) {
  for (int a = 0; a < g.dim; ++a) {
    x[a] = cheb_node(lo[a], hi[a], g.p, alpha % g.p);
    alpha /= g.p;
  }
}

// 1D Lagrange polynomial a of the box's Chebyshev points at x
__device__ __forceinline__ double lagrange_1d(double lo, double hi, int p, int a, double x) {
  const double na = cheb_node(lo, hi, p, a);
  double v = 1.0;
  for (int b = 0; b < p; ++b)
    if (b != a) v *= (x - cheb_node(lo, hi, p, b)) / (na - cheb_node(lo, hi, p, b));
  return v;
}

// tensor Lagrange function beta of a box at x: L_{dim-1} * ( ... * (L_1 * L_0))
__device__ __forceinline__ double lagrange(const CGeo &g, const double *lo, const double *hi, int beta, const double *x) {
  double v = 1.0;
  for (int a = 0; a < g.dim; ++a) {
    const double la = lagrange_1d(lo[a], hi[a], g.p, beta % g.p, x[a]);
    v = a == 0 ? la : la * v;
    beta /= g.p;
  }
  return v;
}

// leaf bases: R_t[i, alpha] = L_alpha(x_{begin_t + i}), |t| x P column-major
__global__ void k_leaf_interp(CGeo g, int leaf0, int nleaf, const int64_t *__restrict__ begin,
                              const int64_t *__restrict__ size, const double *__restrict__ box_lo,
                              const double *__restrict__ box_hi, const double *__restrict__ pts,
                              const int64_t *__restrict__ off, double *__restrict__ out) {
  const int lf = blockIdx.x;
  if (lf >= nleaf) return;
  const int t = leaf0 + lf;
  const int64_t m = size[t], b0 = begin[t];
  const double *lo = box_lo + int64_t(t) * g.dim, *hi = box_hi + int64_t(t) * g.dim;
  double *R = out + off[lf];
  for (int64_t e = threadIdx.x; e < m * g.P; e += blockDim.x) {
    const int64_t i = e % m;
    const int alpha = int(e / m);
    R[e] = lagrange(g, lo, hi, alpha, pts + (b0 + i) * g.dim);
  }
}

// transfers: T_c[alpha, beta] = L^{parent}_beta(node_alpha of c), P x P
__global__ void k_transfer_interp(CGeo g, int c0, int nc, const int32_t *__restrict__ parent,
                                  const double *__restrict__ box_lo, const double *__restrict__ box_hi,
                                  double *__restrict__ out) {
  const int c = c0 + int(blockIdx.x);
  if (c >= c0 + nc) return;
  const int pa = parent[c];
  const double *lo = box_lo + int64_t(c) * g.dim, *hi = box_hi + int64_t(c) * g.dim;
  const double *plo = box_lo + int64_t(pa) * g.dim, *phi = box_hi + int64_t(pa) * g.dim;
  double *T = out + int64_t(c) * g.P * g.P;
  for (int e = threadIdx.x; e < g.P * g.P; e += blockDim.x) {
    const int alpha = e % g.P, beta = e / g.P;
    double x[3];
    tensor_node(g, lo, hi, alpha, x);
    T[e] = lagrange(g, plo, phi, beta, x);
  }
}

// couplings at the Chebyshev points: D_ts[alpha, beta] = a(node_alpha(t), node_beta(s)), P x P
__global__ void k_coupling_eval(CGeo g, int64_t nfar, const int32_t *__restrict__ far_row,
                                const int32_t *__restrict__ far_col, const double *__restrict__ box_lo,
                                const double *__restrict__ box_hi, double *__restrict__ out) {
  for (int64_t i = blockIdx.x; i < nfar; i += gridDim.x) {
    const int t = far_row[i], s = far_col[i];
    double *D = out + i * g.P * g.P;
    for (int e = threadIdx.x; e < g.P * g.P; e += blockDim.x) {
      const int alpha = e % g.P, beta = e / g.P;
      double x[3], y[3];
      tensor_node(g, box_lo + int64_t(t) * g.dim, box_hi + int64_t(t) * g.dim, alpha, x);
      tensor_node(g, box_lo + int64_t(s) * g.dim, box_hi + int64_t(s) * g.dim, beta, y);
      D[e] = kernel_at(g, x, y);
    }
  }
}

// close blocks: C_ts[i, j] = a(x_i, y_j), the diagonal of C_tt = diag
__global__ void k_near_eval(CGeo g, int64_t nnear, const int32_t *__restrict__ near_row,
                            const int32_t *__restrict__ near_col, const int64_t *__restrict__ begin,
                            const int64_t *__restrict__ size, const double *__restrict__ pts,
                            const int64_t *__restrict__ off, double *__restrict__ out) {
  for (int64_t z = blockIdx.x; z < nnear; z += gridDim.x) {
    const int t = near_row[z], s = near_col[z];
    const int64_t mt = size[t], ms = size[s], bt = begin[t], bs = begin[s];
    double *C = out + off[z];
    for (int64_t e = threadIdx.x; e < mt * ms; e += blockDim.x) {
      const int64_t i = e % mt, j = e / mt;
      C[e] = (t == s && i == j) ? g.diag : kernel_at(g, pts + (bt + i) * g.dim, pts + (bs + j) * g.dim);
    }
  }
}

// ---- batched small FP64 products C (m x n) = op(A) op(B), column-major ----
struct CGemm {
  int64_t a, b, c;
  int32_t m, n, k, lda, ldb, ldc;
  int32_t ta, tb;
};

__global__ void __launch_bounds__(256) k_gemm_batch(const CGemm *__restrict__ items, const double *__restrict__ A,
                                                    const double *__restrict__ B, double *__restrict__ C) {
  const CGemm it = items[blockIdx.x];
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  const int tid = threadIdx.x, tm = tid & 15, tn = tid >> 4;
  for (int m0 = 0; m0 < it.m; m0 += 64)
    for (int n0 = 0; n0 < it.n; n0 += 64) {
      double acc[4][4] = {};
      for (int k0 = 0; k0 < it.k; k0 += 16) {
        for (int e = tid; e < 1024; e += 256) {
          const int i = e & 63, kk = e >> 6, gi = m0 + i, gk = k0 + kk;
          As[kk][i] = (gi < it.m && gk < it.k)
                          ? (it.ta ? A[it.a + gk + int64_t(gi) * it.lda] : A[it.a + gi + int64_t(gk) * it.lda])
                          : 0.0;
        }
        for (int e = tid; e < 1024; e += 256) {
          const int kk = e & 15, j = e >> 4, gk = k0 + kk, gj = n0 + j;
          Bs[kk][j] = (gk < it.k && gj < it.n)
                          ? (it.tb ? B[it.b + gj + int64_t(gk) * it.ldb] : B[it.b + gk + int64_t(gj) * it.ldb])
                          : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          double av[4], bv[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) av[r] = As[kk][tm * 4 + r], bv[r] = Bs[kk][tn * 4 + r];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] += av[r] * bv[q];
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = m0 + tm * 4 + r, j = n0 + tn * 4 + q;
          if (i < it.m && j < it.n) C[it.c + i + int64_t(j) * it.ldc] = acc[r][q];
        }
    }
}

__device__ double block_sum_d(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < int(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// ---- Householder QR (LAPACK conventions) of A (m x k, ld m), in place in
// global memory: R (kr x k, kr = min(m, k)) and, when q >= 0, the reduced
// Q = H_0 ... H_{kr-1} [I; 0] (m x kr) ----
struct CQr {
  int64_t a, q, r;
  int32_t m, k;
};

__global__ void __launch_bounds__(256) k_qr_batch(const CQr *__restrict__ items, double *__restrict__ Abuf,
                                                  double *__restrict__ Qbuf, double *__restrict__ Rbuf) {
  const CQr it = items[blockIdx.x];
  const int m = it.m, k = it.k, kr = min(m, k);
  double *A = Abuf + it.a;
  __shared__ double tau[kCMaxP];
  __shared__ double red[8];
  __shared__ double s_scal;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < kr; ++j) {
    double part = 0.0;
    for (int i = j + 1 + tid; i < m; i += blockDim.x) part += A[i + int64_t(j) * m] * A[i + int64_t(j) * m];
    const double s2 = block_sum_d(part, red);
    if (tid == 0) {
      double t = 0.0;
      if (s2 != 0.0) {
        const double alpha = A[j + int64_t(j) * m];
        const double beta = -copysign(hypot(alpha, sqrt(s2)), alpha);
        t = (beta - alpha) / beta;
        s_scal = 1.0 / (alpha - beta);
        A[j + int64_t(j) * m] = beta;
      }
      tau[j] = t;
    }
    __syncthreads();
    const double tj = tau[j];
    if (tj != 0.0) {
      const double sc = s_scal;
      for (int i = j + 1 + tid; i < m; i += blockDim.x) A[i + int64_t(j) * m] *= sc;
      __syncthreads();
      for (int c = j + 1 + wid; c < k; c += nw) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + int64_t(j) * m] * A[i + int64_t(c) * m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w += A[j + int64_t(c) * m];
        const double tw = tj * w;
        if (lane == 0) A[j + int64_t(c) * m] -= tw;
        for (int i = j + 1 + lane; i < m; i += 32) A[i + int64_t(c) * m] -= tw * A[i + int64_t(j) * m];
      }
    }
    __syncthreads();
  }
  double *R = Rbuf + it.r;
  for (int e = tid; e < kr * k; e += blockDim.x) {
    const int r = e % kr, c = e / kr;
    R[e] = r <= c ? A[r + int64_t(c) * m] : 0.0;
  }
  if (it.q < 0) return;
  double *Q = Qbuf + it.q;
  for (int e = tid; e < m * kr; e += blockDim.x) Q[e] = (e % m) == (e / m) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = kr - 1; j >= 0; --j) {
    const double tj = tau[j];
    if (tj != 0.0) {
      for (int c = j + wid; c < kr; c += nw) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i + int64_t(j) * m] * Q[i + int64_t(c) * m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w += Q[j + int64_t(c) * m];
        const double tw = tj * w;
        if (lane == 0) Q[j + int64_t(c) * m] -= tw;
        for (int i = j + 1 + lane; i < m; i += 32) Q[i + int64_t(c) * m] -= tw * A[i + int64_t(j) * m];
      }
    }
    __syncthreads();
  }
}

// ---- far-field Gram of a cluster: M_t = sum over its far pairs of Do_ts Do_ts^T
// (one CTA per cluster; thread (tm, tn) owns a 4 x 4 block of M) ----
struct CGram {
  int64_t m_off;       // M_t (r x r)
  int64_t pair0, pair1;  // far pairs [pair0, pair1) of t
  int32_t r;
};

__global__ void __launch_bounds__(256) k_gram(const CGram *__restrict__ items, const int64_t *__restrict__ do_off,
                                              const int32_t *__restrict__ do_cols, const double *__restrict__ Do,
                                              double *__restrict__ M) {
  const CGram it = items[blockIdx.x];
  const int r = it.r;
  __shared__ double Ds[kCMaxP][kCMaxP + 1];  // Do_ts (r x c), [row][col]
  const int tid = threadIdx.x, tm = tid & 15, tn = tid >> 4;
  double acc[4][4] = {};
  for (int64_t z = it.pair0; z < it.pair1; ++z) {
    const int c = do_cols[z];
    const double *D = Do + do_off[z];
    for (int e = tid; e < r * c; e += 256) Ds[e % r][e / r] = D[e];
    __syncthreads();
    for (int q = 0; q < c; ++q) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = tm * 4 + i < r ? Ds[tm * 4 + i][q] : 0.0;
        bv[i] = tn * 4 + i < r ? Ds[tn * 4 + i][q] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
  double *Mt = M + it.m_off;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = tm * 4 + i, b = tn * 4 + j;
      if (a < r && b < r) Mt[a + b * r] = acc[i][j];
    }
}

// M_t += X (r x r) elementwise: the parent's share Tq_t M_p Tq_t^T
__global__ void k_add_items(const int64_t *__restrict__ dst, const int64_t *__restrict__ src,
                            const int32_t *__restrict__ len, double *__restrict__ M, const double *__restrict__ X) {
  const int i = blockIdx.x;
  for (int e = threadIdx.x; e < len[i]; e += blockDim.x) M[dst[i] + e] += X[src[i] + e];
}

// ---- symmetric eigenproblem of M_t (r x r) by cyclic two-sided Jacobi with
// the round-robin ordering (r/2 disjoint rotations per round, one warp each);
// eigenvectors sorted by decreasing eigenvalue into U (r x r), and the rank
// #{ lambda_i > tol^2 lambda_0 } (0 if lambda_0 <= 0) ----
struct CEig {
  int64_t m_off, u_off;
  int32_t r, cluster;
};

constexpr int kEigThreads = 1024;
constexpr int kEigSweeps = 40;

__global__ void __launch_bounds__(kEigThreads) k_eig_jacobi(const CEig *__restrict__ items, const double *__restrict__ M,
                                                            double *__restrict__ U, double tol2,
                                                            int32_t *__restrict__ rank) {
  const CEig it = items[blockIdx.x];
  const int r = it.r;
  extern __shared__ double sme[];
  double *A = sme;                         // r x r, column-major, ld r
  double *V = A + kCMaxP * kCMaxP;         // r x r
  __shared__ double cs[kCMaxP / 2][2];     // rotation of each pair
  __shared__ int pr[kCMaxP / 2][2];
  __shared__ int s_rot;
  __shared__ int order[kCMaxP];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < r * r; e += kEigThreads) {
    A[e] = M[it.m_off + e];
    V[e] = (e % r) == (e / r) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int n2 = r + (r & 1), npairs = n2 / 2;
  double fro = 0.0;
  for (int e = 0; e < r * r; ++e) fro += A[e] * A[e];  // every thread: the same sum
  const double eps = 1e-17 * sqrt(fro);
  for (int sweep = 0; sweep < kEigSweeps && r > 1; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < n2 - 1; ++round) {
      // pairs of this round: (0, p(0)), (p(i), p(n2 - 1 - i)) with p(j) = 1 + (j + round) mod (n2 - 1)
      if (tid < npairs) {
        // player 0 stays, players 1 .. n2 - 1 sit at q(j) = 1 + (j + round) mod (n2 - 1);
        // pairs (0, q(0)) and (q(i), q(n2 - 1 - i)), i = 1 .. n2/2 - 1
        const int i = tid;
        int a = i == 0 ? 0 : 1 + (i + round) % (n2 - 1);
        int b = 1 + ((i == 0 ? 0 : n2 - 1 - i) + round) % (n2 - 1);
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        double c = 1.0, s = 0.0;
        if (b < r) {
          const double apq = A[a + b * r];
          if (fabs(apq) > eps) {
            const double app = A[a + a * r], aqq = A[b + b * r];
            const double theta = (aqq - app) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            atomicAdd(&s_rot, 1);
          }
        }
        cs[i][0] = c;
        cs[i][1] = s;
        pr[i][0] = a;
        pr[i][1] = b;
      }
      __syncthreads();
      // A <- J^T A: rows a, b of every column (warp per pair, lanes over columns)
      for (int i = wid; i < npairs; i += kEigThreads / 32) {
        const int a = pr[i][0], b = pr[i][1];
        const double c = cs[i][0], s = cs[i][1];
        if (b >= r || s == 0.0) continue;
        for (int col = lane; col < r; col += 32) {
          const double x = A[a + col * r], y = A[b + col * r];
          A[a + col * r] = c * x - s * y;
          A[b + col * r] = s * x + c * y;
        }
      }
      __syncthreads();
      // A <- A J and V <- V J: columns a, b
      for (int i = wid; i < npairs; i += kEigThreads / 32) {
        const int a = pr[i][0], b = pr[i][1];
        const double c = cs[i][0], s = cs[i][1];
        if (b >= r || s == 0.0) continue;
        for (int row = lane; row < r; row += 32) {
          const double x = A[row + a * r], y = A[row + b * r];
          A[row + a * r] = c * x - s * y;
          A[row + b * r] = s * x + c * y;
          const double vx = V[row + a * r], vy = V[row + b * r];
          V[row + a * r] = c * vx - s * vy;
          V[row + b * r] = s * vx + c * vy;
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (rot == 0) break;
  }
  // decreasing eigenvalues (the diagonal), stable for ties
  if (tid == 0) {
    for (int i = 0; i < r; ++i) order[i] = i;
    for (int i = 1; i < r; ++i) {
      const int v = order[i];
      const double lv = A[v + v * r];
      int j = i - 1;
      while (j >= 0 && A[order[j] + order[j] * r] < lv) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = v;
    }
    int rk = 0;
    if (r > 0) {
      const double l0 = A[order[0] + order[0] * r];
      if (l0 > 0.0)
        for (int i = 0; i < r; ++i)
          if (A[order[i] + order[i] * r] > tol2 * l0) ++rk;
    }
    rank[it.cluster] = rk;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += kEigThreads) U[it.u_off + e] = V[(e % r) + order[e / r] * r];
}

}  // namespace
}  // namespace h2sp

using namespace h2sp;

struct h2sp_h2 {
  int64_t n = 0;
  int32_t D = 0, dim = 0;
  std::vector<int32_t> level_ptr, parent, rank, far_col, near_col;
  std::vector<int64_t> begin, size, far_ptr, near_ptr, leaf_basis_off, transfer_off, coupling_off, near_off;
  double *arr[4] = {nullptr, nullptr, nullptr, nullptr};  // leaf_basis, transfer, coupling, near_block (device)
  int64_t count[4] = {0, 0, 0, 0};
  int device = -1;
  ~h2sp_h2() {
    for (double *p : arr)
      if (p) cudaFree(p);
  }
};

namespace {

struct Fail2 {
  int st;
  std::string msg;
};

struct DevBufs {
  std::vector<void *> v;
  template <class T>
  T *get(size_t n) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Fail2{e == cudaErrorMemoryAllocation ? int(H2SP_ENOMEM) : int(H2SP_ECUDA), cudaGetErrorString(e)};
    }
    v.push_back(p);
    return static_cast<T *>(p);
  }
  template <class T>
  T *put(const std::vector<T> &h) {
    T *p = get<T>(h.size());
    if (!h.empty()) chk(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
  }
  static void chk(cudaError_t e) {
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Fail2{e == cudaErrorMemoryAllocation ? int(H2SP_ENOMEM) : int(H2SP_ECUDA), cudaGetErrorString(e)};
    }
  }
  ~DevBufs() {
    for (void *p : v) cudaFree(p);
  }
};

#define CREQ(c, msg)                          \
  do {                                        \
    if (!(c)) throw Fail2{H2SP_EINVAL, msg};  \
  } while (0)

inline void launch_gemms(const std::vector<CGemm> &items, const double *A, const double *B, double *C, DevBufs &db,
                         cudaStream_t s) {
  if (items.empty()) return;
  CGemm *d = db.put(items);
  k_gemm_batch<<<unsigned(items.size()), 256, 0, s>>>(d, A, B, C);
  DevBufs::chk(cudaGetLastError());
}

}  // namespace

extern "C" {

int h2sp_construct(const h2sp_construct_desc *c, h2sp_stream stream, h2sp_h2 **out) {
  if (!c || !out) return H2SP_EINVAL;
  *out = nullptr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto M = new (std::nothrow) h2sp_h2();
  if (!M) return H2SP_ENOMEM;
  try {
    // ---- validation of the tree and the lists (host) ----
    CREQ(c->n > 0 && (c->dim == 2 || c->dim == 3) && c->depth >= 0 && c->depth < 60, "n, dim or depth out of range");
    CREQ(c->order >= 1 && c->kernel >= 0 && c->kernel <= 3, "order or kernel out of range");
    int P = 1;
    for (int a = 0; a < c->dim; ++a) P *= c->order;
    CREQ(P <= kCMaxP, "order^dim above 64");
    CREQ(c->tol <= 0.0 || c->tol >= 1e-7, "recompression tolerance below 1e-7 (Gram weights)");
    CREQ(c->level_ptr && c->parent && c->begin && c->size && c->box_lo && c->box_hi && c->far_ptr && c->near_ptr &&
             c->points,
         "missing array");
    const int D = c->depth;
    const int32_t *lp = c->level_ptr;
    CREQ(lp[0] == 0 && lp[1] >= 1, "depth 0 must hold the root(s)");
    for (int d = 1; d <= D; ++d) CREQ(lp[d + 1] > lp[d], "empty depth");
    const int ncl = lp[D + 1], nleaf = lp[D + 1] - lp[D];
    for (int t = 0; t < lp[1]; ++t) CREQ(c->parent[t] == -1, "root parent must be -1");
    std::vector<int> dep(ncl);
    for (int d = 0; d <= D; ++d)
      for (int t = lp[d]; t < lp[d + 1]; ++t) dep[t] = d;
    std::vector<int> nkids(ncl, 0), kid0(ncl, -1);
    for (int t = lp[1]; t < ncl; ++t) {
      const int pa = c->parent[t];
      CREQ(pa >= 0 && pa < ncl && dep[pa] == dep[t] - 1, "parent not one depth up");
      if (t > lp[dep[t]]) CREQ(pa >= c->parent[t - 1], "children of a cluster must be consecutive");
      if (kid0[pa] < 0) kid0[pa] = t;
      nkids[pa]++;
    }
    for (int t = 0; t < lp[D]; ++t) CREQ(nkids[t] > 0, "non-leaf cluster without children");
    int64_t acc = 0;
    for (int t = lp[D]; t < ncl; ++t) {
      CREQ(c->size[t] > 0 && c->begin[t] == acc, "leaf ranges must be contiguous and non-empty");
      acc += c->size[t];
    }
    CREQ(acc == c->n, "leaf sizes must add up to n");
    for (int t = 0; t < ncl; ++t) CREQ(c->size[t] >= 0 && c->begin[t] >= 0 && c->begin[t] + c->size[t] <= c->n, "range");
    const int64_t nfar = c->far_ptr[ncl];
    CREQ(c->far_ptr[0] == 0 && nfar >= 0 && (nfar == 0 || c->far_col), "bad far_ptr");
    std::vector<int32_t> far_row(static_cast<size_t>(nfar));
    for (int t = 0; t < ncl; ++t) {
      CREQ(c->far_ptr[t + 1] >= c->far_ptr[t], "far_ptr not monotone");
      for (int64_t i = c->far_ptr[t]; i < c->far_ptr[t + 1]; ++i) {
        const int q = c->far_col[i];
        CREQ(q >= 0 && q < ncl && dep[q] == dep[t], "far pair across depths");
        far_row[size_t(i)] = t;
      }
    }
    const int64_t nnear = c->near_ptr[nleaf];
    CREQ(c->near_ptr[0] == 0 && nnear > 0 && c->near_col, "bad near_ptr");
    std::vector<int32_t> near_row(static_cast<size_t>(nnear));
    for (int lf = 0; lf < nleaf; ++lf) {
      CREQ(c->near_ptr[lf + 1] >= c->near_ptr[lf], "near_ptr not monotone");
      for (int64_t i = c->near_ptr[lf]; i < c->near_ptr[lf + 1]; ++i) {
        const int q = c->near_col[i];
        CREQ(q >= lp[D] && q < ncl, "close pair with a non-leaf");
        near_row[size_t(i)] = lp[D] + lf;
      }
    }
    cudaGetDevice(&M->device);
    M->n = c->n;
    M->D = D;
    M->dim = c->dim;
    M->level_ptr.assign(lp, lp + D + 2);
    M->parent.assign(c->parent, c->parent + ncl);
    M->begin.assign(c->begin, c->begin + ncl);
    M->size.assign(c->size, c->size + ncl);
    M->far_ptr.assign(c->far_ptr, c->far_ptr + ncl + 1);
    M->far_col.assign(c->far_col, c->far_col + nfar);
    M->near_ptr.assign(c->near_ptr, c->near_ptr + nleaf + 1);
    M->near_col.assign(c->near_col, c->near_col + nnear);
    // close blocks (final in either mode)
    M->near_off.resize(size_t(nnear));
    int64_t ne = 0;
    for (int64_t z = 0; z < nnear; ++z) {
      M->near_off[size_t(z)] = ne;
      ne += c->size[near_row[size_t(z)]] * c->size[c->near_col[z]];
    }
    DevBufs db;
    CGeo g{c->dim, c->order, P, c->kernel, c->diag};
    std::vector<double> blo(c->box_lo, c->box_lo + size_t(ncl) * c->dim), bhi(c->box_hi, c->box_hi + size_t(ncl) * c->dim);
    const double *d_lo = db.put(blo), *d_hi = db.put(bhi);
    const int64_t *d_begin = db.put(M->begin), *d_size = db.put(M->size);
    const int32_t *d_parent = db.put(M->parent);
    const int32_t *d_far_row = db.put(far_row), *d_far_col = db.put(M->far_col);
    const int32_t *d_near_row = db.put(near_row), *d_near_col = db.put(M->near_col);
    const int64_t *d_near_off = db.put(M->near_off);
    auto own = [&](int which, int64_t count) {
      void *p = nullptr;
      DevBufs::chk(cudaMalloc(&p, size_t(std::max<int64_t>(count, 1)) * sizeof(double)));
      M->arr[which] = static_cast<double *>(p);
      M->count[which] = count;
      return M->arr[which];
    };
    double *NB = own(3, ne);
    const unsigned grid_pairs = unsigned(std::max(1, 8 * device_sms()));
    k_near_eval<<<grid_pairs, 256, 0, s>>>(g, nnear, d_near_row, d_near_col, d_begin, d_size, c->points, d_near_off, NB);
    DevBufs::chk(cudaGetLastError());
    // raw interpolation parameters
    std::vector<int64_t> rl_off(static_cast<size_t>(nleaf));
    int64_t rl = 0;
    for (int lf = 0; lf < nleaf; ++lf) {
      rl_off[size_t(lf)] = rl;
      rl += c->size[lp[D] + lf] * P;
    }
    const bool recompress = c->tol > 0.0;
    double *RL = recompress ? db.get<double>(size_t(rl)) : own(0, rl);
    double *TR = db.get<double>(size_t(ncl) * P * P);  // T_c at c * P^2
    double *DR = recompress ? db.get<double>(size_t(nfar) * P * P) : own(2, nfar * P * P);
    k_leaf_interp<<<unsigned(std::max(nleaf, 1)), 128, 0, s>>>(g, lp[D], nleaf, d_begin, d_size, d_lo, d_hi, c->points,
                                                               db.put(rl_off), RL);
    if (ncl > lp[1]) k_transfer_interp<<<unsigned(ncl - lp[1]), 128, 0, s>>>(g, lp[1], ncl - lp[1], d_parent, d_lo, d_hi, TR);
    if (nfar) k_coupling_eval<<<grid_pairs, 256, 0, s>>>(g, nfar, d_far_row, d_far_col, d_lo, d_hi, DR);
    DevBufs::chk(cudaGetLastError());
    std::vector<int32_t> rank(static_cast<size_t>(ncl), P);
    if (!recompress) {
      M->leaf_basis_off = rl_off;
      M->transfer_off.assign(size_t(ncl), 0);
      int64_t to = 0;
      for (int t = lp[1]; t < ncl; ++t) M->transfer_off[size_t(t)] = to, to += int64_t(P) * P;
      double *T = own(1, to);
      if (to) DevBufs::chk(cudaMemcpyAsync(T, TR + size_t(lp[1]) * P * P, size_t(to) * sizeof(double),
                                           cudaMemcpyDeviceToDevice, s));
      M->coupling_off.resize(size_t(nfar));
      for (int64_t i = 0; i < nfar; ++i) M->coupling_off[size_t(i)] = i * P * P;
      M->rank = rank;
      DevBufs::chk(cudaStreamSynchronize(s));
      *out = M;
      return H2SP_OK;
    }
    // ---- 1. orthogonalise bottom-up ----
    std::vector<int> r(static_cast<size_t>(ncl), 0), rows(static_cast<size_t>(ncl), 0);
    for (int t = lp[D]; t < ncl; ++t) rows[size_t(t)] = int(c->size[t]), r[size_t(t)] = std::min(int(c->size[t]), P);
    for (int d = D - 1; d >= 0; --d)
      for (int t = lp[d]; t < lp[d + 1]; ++t) {
        int w = 0;
        for (int k = kid0[t]; k < kid0[t] + nkids[t]; ++k) w += r[size_t(k)];
        rows[size_t(t)] = w;
        r[size_t(t)] = std::min(w, P);
      }
    std::vector<int64_t> z_off(static_cast<size_t>(ncl)), q_off(static_cast<size_t>(ncl)), w_off(static_cast<size_t>(ncl), -1);
    int64_t zn = 0, qn = 0, wn = 0;
    for (int t = 0; t < ncl; ++t) {
      z_off[size_t(t)] = zn;
      zn += int64_t(r[size_t(t)]) * P;
      q_off[size_t(t)] = qn;
      qn += int64_t(rows[size_t(t)]) * r[size_t(t)];
      if (t < lp[D]) w_off[size_t(t)] = wn, wn += int64_t(rows[size_t(t)]) * P;
    }
    double *Z = db.get<double>(size_t(zn)), *Q = db.get<double>(size_t(qn)), *W = db.get<double>(size_t(wn));
    {
      std::vector<CQr> qi;
      for (int lf = 0; lf < nleaf; ++lf) {
        const int t = lp[D] + lf;
        qi.push_back(CQr{rl_off[size_t(lf)], q_off[size_t(t)], z_off[size_t(t)], rows[size_t(t)], P});
      }
      k_qr_batch<<<unsigned(qi.size()), 256, 0, s>>>(db.put(qi), RL, Q, Z);
      DevBufs::chk(cudaGetLastError());
    }
    for (int d = D - 1; d >= 0; --d) {
      std::vector<CGemm> gi;
      std::vector<CQr> qi;
      for (int t = lp[d]; t < lp[d + 1]; ++t) {
        int o = 0;
        for (int k = kid0[t]; k < kid0[t] + nkids[t]; ++k) {
          // W_t[o : o + r_k, :] = Z_k T_k
          if (r[size_t(k)] > 0)
            gi.push_back(CGemm{z_off[size_t(k)], int64_t(k) * P * P, w_off[size_t(t)] + o, r[size_t(k)], P, P,
                               r[size_t(k)], P, rows[size_t(t)], 0, 0});
          o += r[size_t(k)];
        }
        if (rows[size_t(t)] > 0) qi.push_back(CQr{w_off[size_t(t)], q_off[size_t(t)], z_off[size_t(t)], rows[size_t(t)], P});
      }
      launch_gemms(gi, Z, TR, W, db, s);
      if (!qi.empty()) {
        k_qr_batch<<<unsigned(qi.size()), 256, 0, s>>>(db.put(qi), W, Q, Z);
        DevBufs::chk(cudaGetLastError());
      }
    }
    // Tq_c: rows [o_c, o_c + r_c) of Q_parent (ld rows_parent)
    std::vector<int64_t> tq_off(static_cast<size_t>(ncl), -1);
    for (int t = 0; t < lp[D]; ++t) {
      int o = 0;
      for (int k = kid0[t]; k < kid0[t] + nkids[t]; ++k) {
        tq_off[size_t(k)] = q_off[size_t(t)] + o;
        o += r[size_t(k)];
      }
    }
    // ---- 2. Do_ts = Z_t D_ts Z_s^T ----
    std::vector<int64_t> do_off(static_cast<size_t>(nfar)), x_off(static_cast<size_t>(nfar));
    std::vector<int32_t> do_cols(static_cast<size_t>(nfar));
    int64_t don = 0, xn = 0;
    for (int64_t i = 0; i < nfar; ++i) {
      const int t = far_row[size_t(i)], q = c->far_col[i];
      do_off[size_t(i)] = don;
      don += int64_t(r[size_t(t)]) * r[size_t(q)];
      do_cols[size_t(i)] = r[size_t(q)];
      x_off[size_t(i)] = xn;
      xn += int64_t(P) * r[size_t(q)];
    }
    double *DO = db.get<double>(size_t(don));
    {
      double *X = db.get<double>(size_t(xn));
      std::vector<CGemm> g1, g2;
      for (int64_t i = 0; i < nfar; ++i) {
        const int t = far_row[size_t(i)], q = c->far_col[i];
        const int rt = r[size_t(t)], rq = r[size_t(q)];
        if (rt == 0 || rq == 0) continue;
        g1.push_back(CGemm{i * P * P, z_off[size_t(q)], x_off[size_t(i)], P, rq, P, P, rq, P, 0, 1});   // D Z_s^T
        g2.push_back(CGemm{z_off[size_t(t)], x_off[size_t(i)], do_off[size_t(i)], rt, rq, P, rt, P, rt, 0, 0});
      }
      launch_gemms(g1, DR, Z, X, db, s);
      launch_gemms(g2, Z, X, DO, db, s);
    }
    // ---- 3-4. weights and eigenvectors, top-down ----
    std::vector<int64_t> m_off(static_cast<size_t>(ncl));
    int64_t mn = 0;
    for (int t = 0; t < ncl; ++t) m_off[size_t(t)] = mn, mn += int64_t(r[size_t(t)]) * r[size_t(t)];
    double *Mg = db.get<double>(size_t(mn)), *U = db.get<double>(size_t(mn));
    int32_t *d_rank = db.get<int32_t>(size_t(ncl));
    DevBufs::chk(cudaMemsetAsync(d_rank, 0, sizeof(int32_t) * size_t(ncl), s));
    {
      std::vector<CGram> gr;
      for (int t = 0; t < ncl; ++t)
        if (r[size_t(t)] > 0) gr.push_back(CGram{m_off[size_t(t)], c->far_ptr[t], c->far_ptr[t + 1], r[size_t(t)]});
      if (!gr.empty()) {
        k_gram<<<unsigned(gr.size()), 256, 0, s>>>(db.put(gr), db.put(do_off), db.put(do_cols), DO, Mg);
        DevBufs::chk(cudaGetLastError());
      }
    }
    const size_t eig_smem = size_t(2) * kCMaxP * kCMaxP * sizeof(double);
    DevBufs::chk(smem_attr((const void *)k_eig_jacobi, int(eig_smem)));
    double *XP = db.get<double>(size_t(std::max<int64_t>(zn, 1)));  // parent-share scratch, r_t x P per cluster
    std::vector<int64_t> xp_off(static_cast<size_t>(ncl));
    {
      int64_t a = 0;
      for (int t = 0; t < ncl; ++t) {
        xp_off[size_t(t)] = a;
        a += int64_t(r[size_t(t)]) * P;
      }
    }
    double *XT = db.get<double>(size_t(std::max<int64_t>(zn, 1)));  // r_t x r_p scratch (<= r_t x P)
    for (int d = 0; d <= D; ++d) {
      if (d > 0) {
        // M_t += Tq_t (M_p Tq_t^T): X = M_p Tq_t^T (r_p x r_t), then Y = Tq_t X (r_t x r_t)
        std::vector<CGemm> g1, g2;
        std::vector<int64_t> ad, as;
        std::vector<int32_t> al;
        for (int t = lp[d]; t < lp[d + 1]; ++t) {
          const int pa = c->parent[t], rt = r[size_t(t)], rp = r[size_t(pa)];
          if (rt == 0 || rp == 0) continue;
          g1.push_back(CGemm{m_off[size_t(pa)], tq_off[size_t(t)], xp_off[size_t(t)], rp, rt, rp, rp,
                             rows[size_t(pa)], rp, 0, 1});
          g2.push_back(CGemm{tq_off[size_t(t)], xp_off[size_t(t)], z_off[size_t(t)], rt, rt, rp, rows[size_t(pa)], rp,
                             rt, 0, 0});
          ad.push_back(m_off[size_t(t)]);
          as.push_back(z_off[size_t(t)]);
          al.push_back(rt * rt);
        }
        launch_gemms(g1, Mg, Q, XP, db, s);
        launch_gemms(g2, Q, XP, XT, db, s);
        if (!ad.empty()) {
          k_add_items<<<unsigned(ad.size()), 256, 0, s>>>(db.put(ad), db.put(as), db.put(al), Mg, XT);
          DevBufs::chk(cudaGetLastError());
        }
      }
      std::vector<CEig> ei;
      for (int t = lp[d]; t < lp[d + 1]; ++t)
        if (r[size_t(t)] > 0) ei.push_back(CEig{m_off[size_t(t)], m_off[size_t(t)], r[size_t(t)], t});
      if (!ei.empty()) {
        k_eig_jacobi<<<unsigned(ei.size()), kEigThreads, eig_smem, s>>>(db.put(ei), Mg, U, c->tol * c->tol, d_rank);
        DevBufs::chk(cudaGetLastError());
      }
    }
    DevBufs::chk(cudaMemcpyAsync(rank.data(), d_rank, sizeof(int32_t) * size_t(ncl), cudaMemcpyDeviceToHost, s));
    DevBufs::chk(cudaStreamSynchronize(s));
    // ---- 5. recompressed parameters ----
    M->leaf_basis_off.resize(size_t(nleaf));
    int64_t lbn = 0;
    for (int lf = 0; lf < nleaf; ++lf) {
      M->leaf_basis_off[size_t(lf)] = lbn;
      lbn += c->size[lp[D] + lf] * rank[size_t(lp[D] + lf)];
    }
    M->transfer_off.assign(size_t(ncl), 0);
    int64_t tn = 0;
    for (int t = lp[1]; t < ncl; ++t) {
      M->transfer_off[size_t(t)] = tn;
      tn += int64_t(rank[size_t(t)]) * rank[size_t(c->parent[t])];
    }
    M->coupling_off.resize(size_t(nfar));
    int64_t cn = 0;
    for (int64_t i = 0; i < nfar; ++i) {
      M->coupling_off[size_t(i)] = cn;
      cn += int64_t(rank[size_t(far_row[size_t(i)])]) * rank[size_t(c->far_col[i])];
    }
    double *LB = own(0, lbn), *TT = own(1, tn), *CP = own(2, cn);
    {
      // leaf bases: Q_t (|t| x r_t) B_t (r_t x R_t)
      std::vector<CGemm> gl;
      for (int lf = 0; lf < nleaf; ++lf) {
        const int t = lp[D] + lf, R = rank[size_t(t)];
        if (R == 0) continue;
        gl.push_back(CGemm{q_off[size_t(t)], m_off[size_t(t)], M->leaf_basis_off[size_t(lf)], int(c->size[t]), R,
                           r[size_t(t)], int(c->size[t]), r[size_t(t)], int(c->size[t]), 0, 0});
      }
      launch_gemms(gl, Q, U, LB, db, s);
      // transfers: B_c^T (Tq_c B_p): X = Tq_c B_p (r_c x R_p) into XT
      std::vector<CGemm> g1, g2;
      std::vector<int64_t> xo(static_cast<size_t>(ncl), 0);
      int64_t xa = 0;
      for (int t = lp[1]; t < ncl; ++t) {
        const int pa = c->parent[t], Rc = rank[size_t(t)], Rp = rank[size_t(pa)];
        if (Rc == 0 || Rp == 0) continue;
        xo[size_t(t)] = xa;
        xa += int64_t(r[size_t(t)]) * Rp;
      }
      double *X2 = db.get<double>(size_t(std::max<int64_t>(xa, 1)));
      for (int t = lp[1]; t < ncl; ++t) {
        const int pa = c->parent[t], Rc = rank[size_t(t)], Rp = rank[size_t(pa)];
        if (Rc == 0 || Rp == 0) continue;
        g1.push_back(CGemm{tq_off[size_t(t)], m_off[size_t(pa)], xo[size_t(t)], r[size_t(t)], Rp, r[size_t(pa)],
                           rows[size_t(pa)], r[size_t(pa)], r[size_t(t)], 0, 0});
        g2.push_back(CGemm{m_off[size_t(t)], xo[size_t(t)], M->transfer_off[size_t(t)], Rc, Rp, r[size_t(t)],
                           r[size_t(t)], r[size_t(t)], Rc, 1, 0});
      }
      launch_gemms(g1, Q, U, X2, db, s);
      launch_gemms(g2, U, X2, TT, db, s);
    }
    {
      // couplings: B_t^T (Do_ts B_s)
      std::vector<int64_t> xo(static_cast<size_t>(nfar), 0);
      int64_t xa = 0;
      for (int64_t i = 0; i < nfar; ++i) {
        const int t = far_row[size_t(i)], q = c->far_col[i];
        if (rank[size_t(t)] == 0 || rank[size_t(q)] == 0) continue;
        xo[size_t(i)] = xa;
        xa += int64_t(r[size_t(t)]) * rank[size_t(q)];
      }
      double *X3 = db.get<double>(size_t(std::max<int64_t>(xa, 1)));
      std::vector<CGemm> g1, g2;
      for (int64_t i = 0; i < nfar; ++i) {
        const int t = far_row[size_t(i)], q = c->far_col[i];
        const int Rt = rank[size_t(t)], Rq = rank[size_t(q)];
        if (Rt == 0 || Rq == 0) continue;
        g1.push_back(CGemm{do_off[size_t(i)], m_off[size_t(q)], xo[size_t(i)], r[size_t(t)], Rq, r[size_t(q)],
                           r[size_t(t)], r[size_t(q)], r[size_t(t)], 0, 0});
        g2.push_back(CGemm{m_off[size_t(t)], xo[size_t(i)], M->coupling_off[size_t(i)], Rt, Rq, r[size_t(t)],
                           r[size_t(t)], r[size_t(t)], Rt, 1, 0});
      }
      launch_gemms(g1, DO, U, X3, db, s);
      launch_gemms(g2, U, X3, CP, db, s);
    }
    M->rank = rank;
    DevBufs::chk(cudaStreamSynchronize(s));
    *out = M;
    return H2SP_OK;
  } catch (const Fail2 &f) {
    set_last_error("h2sp_construct: " + f.msg);
    delete M;
    return f.st;
  } catch (const std::bad_alloc &) {
    delete M;
    return H2SP_ENOMEM;
  }
}

int h2sp_h2_describe(const h2sp_h2 *m, h2sp_h2_desc *d) {
  if (!m || !d) return H2SP_EINVAL;
  *d = h2sp_h2_desc{};
  d->n = m->n;
  d->depth = m->D;
  d->level_ptr = m->level_ptr.data();
  d->parent = m->parent.data();
  d->begin = m->begin.data();
  d->size = m->size.data();
  d->rank = m->rank.data();
  d->far_ptr = m->far_ptr.data();
  d->far_col = m->far_col.data();
  d->near_ptr = m->near_ptr.data();
  d->near_col = m->near_col.data();
  d->leaf_basis_off = m->leaf_basis_off.data();
  d->transfer_off = m->transfer_off.data();
  d->coupling_off = m->coupling_off.data();
  d->near_off = m->near_off.data();
  d->leaf_basis = m->arr[0];
  d->transfer = m->arr[1];
  d->coupling = m->arr[2];
  d->near_block = m->arr[3];
  return H2SP_OK;
}

int h2sp_h2_copy(const h2sp_h2 *m, int32_t which, double *dst, int64_t *count, h2sp_stream stream) {
  if (!m || which < 0 || which > 3) return H2SP_EINVAL;
  if (count) *count = m->count[which];
  if (!dst || m->count[which] == 0) return H2SP_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(dst, m->arr[which], size_t(m->count[which]) * sizeof(double), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    cudaGetLastError();
    return H2SP_ECUDA;
  }
  return H2SP_OK;
}

void h2sp_h2_destroy(h2sp_h2 *m) { delete m; }

}  // extern "C"
