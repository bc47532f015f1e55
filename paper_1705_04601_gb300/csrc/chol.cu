// Block Cholesky S = L L^T of a symmetric positive definite S.
//
// The sparse direct package the paper factors S with (§5.3-5.4) is a Cholesky
// code, and Proposition 2.1 makes S symmetric positive definite when A is
// (S = U^T A U with U orthogonal).  The supernodes, elimination order,
// boundaries and fronts are those of the block LU; a panel of NB columns
// needs no pivot search:
//   k_chol_diag : L11 = chol(F11) of the jb x jb diagonal tile, one CTA per
//                 front, a thread per tile row holding the row in registers,
//                 and the rows of L11^-1 into a per-front scratch tile;
//   k_chol_l21  : L21 = F21 L11^-T for every row below the tile, a thread per
//                 row: x_k = sum_{m <= k} a_m (L11^-1)_km, L11^-1 in shared memory;
// then the trailing update C -= L21 L21^T of the lower triangle only, with
// the B operand read from L21 itself (U12 = L21^T is never formed).  FP32
// fronts: 256-column outer blocks; inside a block, rank-64 tensor-core
// updates of the block's columns; at the block end one rank-256 tcgen05
// update of the lower 128 x 128 tiles from the packed L21, which serves as
// both operands.  FP64 fronts (and FP32 with CUDA-core updates): one
// lower-triangle update per panel.  The contribution blocks are
// extended-added by their lower triangles (the extend-add map is monotone).
//
// At the end every front is rewritten in the block LU's form -- unit lower
// L = L_chol D^-1 and U = D L_chol^T with D = diag(L_chol), no interchanges
// -- so the sweeps, the inverted diagonal blocks and the log-determinant of
// the LU path serve unchanged (u_jj = d_j^2 > 0).
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "kernels.h"

namespace h2sp {
namespace {

inline int cdiv_c(int64_t a, int64_t b) { return int((a + b - 1) / b); }

// Cholesky of the diagonal tile [j0, j0 + jb) of every front, and its inverse.
// The tile sits in shared memory; the loops stay compact (this kernel runs
// once per panel, so instruction fetch, not arithmetic, would bound a fully
// unrolled form).  kDiagThreads threads: four per row.
//   Cholesky, left-looking by columns: for column j, the four threads of row
//   r >= j each take a quarter of l_rj's dot product sum_{m<j} l_rm l_jm
//   (lanes of one warp, added by shuffles); l_jj = sqrt(a_jj - ...) and
//   l_rj = (a_rj - ...) / l_jj.  A pivot that is not positive and finite sets
//   bit 8 of *err (S is not positive definite in this precision) and is
//   replaced by 1 so that the factorization stays finite.  With `compensate`
//   (the BF16 block-end modes, whose factors serve as a preconditioner only)
//   it is replaced by a_jj as the tile holds it before this panel's sums
//   (diagonal compensation: the pivot of the updates received so far, which
//   an SPD S keeps positive), and counted in err[1] under bit 16.
//   Inverse, forward substitution by columns: the four threads of column c
//   (lanes of one warp) split y_r = -(sum_{c<=m<r} l_rm y_m) / l_rr, with
//   y_c = 1 / l_cc, row by row; it goes to inv[front][r * NB + c]
//   (row-major, zero above the diagonal and beyond jb).
constexpr int kDiagThreads = 256;
template <typename T, int NB>
__global__ void __launch_bounds__(kDiagThreads) k_chol_diag(const FrontDev *__restrict__ fr, int j0,
                                                            T *__restrict__ fronts, int32_t *__restrict__ piv,
                                                            int *__restrict__ err, T *__restrict__ inv,
                                                            int compensate) {
  static_assert(NB * 4 <= kDiagThreads, "four threads per row");
  const FrontDev F = fr[blockIdx.x];
  if (j0 >= F.s) return;  // uniform over the CTA
  const int jb = min(NB, F.s - j0);
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  constexpr int P = NB + 1;  // padded row length
  __shared__ T L[NB * P];    // row-major: L[r * P + c]
  __shared__ T Y[NB * P];    // L11^-1, row-major
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += kDiagThreads) {
    const int r = e % NB, c = e / NB;  // down the columns of the front
    L[r * P + c] = (r < jb && c <= r) ? A[(j0 + r) + int64_t(j0 + c) * ld] : T(0);
  }
  __syncthreads();
  const int r = tid >> 2, sub = tid & 3;  // row (or column, below) and quarter
  for (int j = 0; j < jb; ++j) {
    T part = T(0);
    if (r >= j && r < jb)
      for (int m = sub; m < j; m += 4) part += L[r * P + m] * L[j * P + m];
    part += __shfl_xor_sync(0xffffffffu, part, 1);
    part += __shfl_xor_sync(0xffffffffu, part, 2);
    if (sub == 0 && r == j) {
      const T a0 = L[j * P + j];
      T a = a0 - part;
      if (!(a > T(0)) || !isfinite(a)) {
        if (compensate && a0 > T(0) && isfinite(a0)) {
          atomicOr(err, 16);
          atomicAdd(err + 1, 1);
          a = a0;
        } else {
          atomicOr(err, 8);
          a = T(1);
        }
      }
      L[j * P + j] = sqrt(a);
    }
    __syncthreads();
    if (sub == 0 && r > j && r < jb) L[r * P + j] = (L[r * P + j] - part) / L[j * P + j];
    __syncthreads();
  }
  // inverse: the four lanes of column c = r walk the rows together
  const int c = r;
  for (int rr = 0; rr < NB; ++rr) {
    T part = T(0);
    if (c < jb && rr > c && rr < jb)
      for (int m = c + sub; m < rr; m += 4) part += L[rr * P + m] * Y[m * P + c];
    part += __shfl_xor_sync(0xffffffffu, part, 1);
    part += __shfl_xor_sync(0xffffffffu, part, 2);
    if (sub == 0 && c < NB) {  // (threads of columns c >= NB only join the shuffles)
      T y = T(0);
      if (c < jb && rr < jb) {
        if (rr == c) y = T(1) / L[rr * P + rr];
        else if (rr > c) y = -part / L[rr * P + rr];
      }
      Y[rr * P + c] = y;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += kDiagThreads) {
    const int rr = e % NB, cc = e / NB;
    if (rr < jb && cc <= rr) A[(j0 + rr) + int64_t(j0 + cc) * ld] = L[rr * P + cc];
  }
  T *Li = inv + int64_t(blockIdx.x) * NB * NB;
  for (int e = tid; e < NB * NB; e += kDiagThreads) Li[e] = Y[(e / NB) * P + e % NB];
  for (int j = tid; j < jb; j += kDiagThreads) piv[F.piv_off + j0 + j] = j0 + j;
}

// The same tile Cholesky and inverse as k_chol_diag, blocked by 8 columns
// so that the CTA synchronises 3 times per 8 columns instead of twice per
// column, with short dependent chains:
//   factorization, for each 8-column step c0 (right-looking):
//     (a) warp 0, lane i < 8 holding row c0 + i of the 8 x 8 diagonal block:
//         for j < 8, l_jj = sqrt(a_jj) (shuffled from lane j), l_ij = a_ij / l_jj,
//         then a_ik -= l_ij l_kj for j < k <= i (l_kj shuffled from lane k);
//     (b) a thread per row r below: x_j = (a_rj - sum_{m<j} x_m l_jm) / l_jj;
//     (c) the lower triangle below: a_rc -= sum_{m<8} l_rm l_cm (rank 8);
//   a pivot that is not positive is handled as in k_chol_diag (its "diagonal
//   as the panel found it" is the tile's entry before this kernel).
//   inverse Y = L^-1 by 8 x 8 blocks: each warp inverts one diagonal block
//   (lane c forms column c by forward substitution); then for d = 1, 2, ...
//   the blocks (i, j = i - d) at once: S = sum_{m = 8j}^{8i - 1} L[8i + r][m]
//   Y[m][8j + c], and Y_ij = -Y_ii S.
// Rows and columns beyond jb hold the identity, so they factor trivially and
// leave the result unchanged; only rows and columns below jb are written.
template <typename T, int NB>
__global__ void __launch_bounds__(kDiagThreads) k_chol_diag_blk(const FrontDev *__restrict__ fr, int j0,
                                                                T *__restrict__ fronts, int32_t *__restrict__ piv,
                                                                int *__restrict__ err, T *__restrict__ inv,
                                                                int compensate) {
  static_assert(NB % 8 == 0 && NB / 8 <= kDiagThreads / 32, "8-column blocks, a warp per diagonal block");
  const FrontDev F = fr[blockIdx.x];
  if (j0 >= F.s) return;  // uniform over the CTA
  const int jb = min(NB, F.s - j0);
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  constexpr int P = NB + 1;
  constexpr int NBK = NB / 8;
  __shared__ T L[NB * P];  // row-major
  __shared__ T Y[NB * P];
  __shared__ T S[(NBK - 1) * 64 + 1];
  __shared__ T d0[NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < NB * NB; e += kDiagThreads) {
    const int r = e % NB, c = e / NB;  // down the columns of the front
    T v = T(0);
    if (r < jb && c <= r) v = A[(j0 + r) + int64_t(j0 + c) * ld];
    else if (r == c) v = T(1);
    L[r * P + c] = v;
    Y[r * P + c] = T(0);
    if (r == c) d0[r] = v;
  }
  __syncthreads();
  for (int c0 = 0; c0 < NB; c0 += 8) {
    // (a) the 8 x 8 diagonal block
    if (warp == 0) {
      T rv[8];
      const bool own = lane < 8;
#pragma unroll
      for (int m = 0; m < 8; ++m) rv[m] = (own && m <= lane) ? L[(c0 + lane) * P + c0 + m] : T(0);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        T a = __shfl_sync(0xffffffffu, rv[j], j);
        if (!(a > T(0)) || !isfinite(a)) {
          const T a0 = d0[c0 + j];
          const bool comp = compensate && a0 > T(0) && isfinite(a0);
          if (lane == 0) {
            if (comp) {
              atomicOr(err, 16);
              atomicAdd(err + 1, 1);
            } else {
              atomicOr(err, 8);
            }
          }
          a = comp ? a0 : T(1);
        }
        const T djj = sqrt(a);
        if (lane == j) rv[j] = djj;
        if (lane > j) rv[j] = rv[j] / djj;
#pragma unroll
        for (int k = j + 1; k < 8; ++k) {
          const T lkj = __shfl_sync(0xffffffffu, rv[j], k);
          if (lane > j && k <= lane) rv[k] -= rv[j] * lkj;
        }
      }
      if (own)
#pragma unroll
        for (int m = 0; m < 8; ++m)
          if (m <= lane) L[(c0 + lane) * P + c0 + m] = rv[m];
    }
    __syncthreads();
    // (b) the rows below against the diagonal block
    const int nbelow = NB - c0 - 8;
    if (tid < nbelow) {
      const int r = c0 + 8 + tid;
      T x[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) x[m] = L[r * P + c0 + m];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        T v = x[j];
#pragma unroll
        for (int m = 0; m < j; ++m) v -= x[m] * L[(c0 + j) * P + c0 + m];
        x[j] = v / L[(c0 + j) * P + c0 + j];
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) L[r * P + c0 + m] = x[m];
    }
    __syncthreads();
    // (c) the rank-8 update of the lower triangle below
    if (nbelow > 0) {
      const int tr = tid >> 4, tc = tid & 15;
      for (int r = c0 + 8 + tr; r < NB; r += 16) {
        T xr[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) xr[m] = L[r * P + c0 + m];
        for (int c = c0 + 8 + tc; c <= r; c += 16) {
          T acc = L[r * P + c];
#pragma unroll
          for (int m = 0; m < 8; ++m) acc -= xr[m] * L[c * P + c0 + m];
          L[r * P + c] = acc;
        }
      }
    }
    __syncthreads();
  }
  // inverse: the diagonal blocks, a warp each (lane c: column c of the block)
  if (warp < NBK && lane < 8) {
    const int b = warp * 8, c = lane;
    T y[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      T v = T(0);
      if (r == c) {
        v = T(1) / L[(b + r) * P + b + r];
      } else if (r > c) {
#pragma unroll
        for (int m = 0; m < r; ++m)
          if (m >= c) v -= L[(b + r) * P + b + m] * y[m];
        v /= L[(b + r) * P + b + r];
      }
      y[r] = v;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) Y[(b + r) * P + b + c] = y[r];
  }
  __syncthreads();
  for (int d = 1; d < NBK; ++d) {
    const int nblk = NBK - d;
    for (int e = tid; e < nblk * 64; e += kDiagThreads) {
      const int j = e >> 6, i = j + d, r = (e >> 3) & 7, c = e & 7;
      T acc = T(0);
      for (int m = 8 * j; m < 8 * i; ++m) acc += L[(8 * i + r) * P + m] * Y[m * P + 8 * j + c];
      S[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < nblk * 64; e += kDiagThreads) {
      const int j = e >> 6, i = j + d, r = (e >> 3) & 7, c = e & 7;
      T acc = T(0);
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t <= r) acc += Y[(8 * i + r) * P + 8 * i + t] * S[(j << 6) + t * 8 + c];
      Y[(8 * i + r) * P + 8 * j + c] = -acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += kDiagThreads) {
    const int rr = e % NB, cc = e / NB;
    if (rr < jb && cc <= rr) A[(j0 + rr) + int64_t(j0 + cc) * ld] = L[rr * P + cc];
  }
  T *Li = inv + int64_t(blockIdx.x) * NB * NB;
  for (int e = tid; e < NB * NB; e += kDiagThreads) {
    const int rr = e / NB, cc = e % NB;
    Li[e] = (rr < jb && cc < jb) ? Y[rr * P + cc] : T(0);
  }
  for (int j = tid; j < jb; j += kDiagThreads) piv[F.piv_off + j0 + j] = j0 + j;
}

// Tile kernel of the panel: the blocked form unless H2SP_CHOL_DIAG=columns
inline bool chol_diag_blocked() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_CHOL_DIAG");
    v = (e && std::strcmp(e, "columns") == 0) ? 0 : 1;
  }
  return v == 1;
}

// L21 = F21 L11^-T for rows [j0 + jb, f) of the panel columns: a thread per
// row, the row a in registers, x_k = sum_{m <= k} a_m (L11^-1)_km with L11^-1
// from k_chol_diag's scratch tile.
constexpr int kL21Threads = 128;
template <typename T, int NB>
__global__ void __launch_bounds__(kL21Threads) k_chol_l21(const FrontDev *__restrict__ fr, int j0,
                                                         T *__restrict__ fronts, const T *__restrict__ inv) {
  const FrontDev F = fr[blockIdx.y];
  if (j0 >= F.s) return;
  const int jb = min(NB, F.s - j0);
  const int row0 = j0 + jb + int(blockIdx.x) * kL21Threads;
  if (row0 >= F.f) return;  // uniform over the CTA
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  // Li[k * P + m] = (L11^-1)_km: rows contiguous, padded to a 16-byte multiple
  constexpr int P = NB + 16 / int(sizeof(T));
  __shared__ __align__(16) T Li[NB * P];
  const T *src = inv + int64_t(blockIdx.y) * NB * NB;
  for (int e = threadIdx.x; e < NB * NB; e += kL21Threads) Li[(e / NB) * P + e % NB] = src[e];
  __syncthreads();
  const int row = row0 + int(threadIdx.x);
  if (row >= F.f) return;
  T a[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) a[k] = k < jb ? A[row + int64_t(j0 + k) * ld] : T(0);
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (k >= jb) break;
    T acc = T(0);
#pragma unroll
    for (int m = 0; m <= k; ++m) acc += a[m] * Li[k * P + m];
    A[row + int64_t(j0 + k) * ld] = acc;
  }
}

// Rewrite the factored columns [0, s) of every front from L_chol to the LU
// form.  32 x 32 tiles of the lower part (rows [0, f), columns [0, s)), a CTA
// per row tile looping over its column tiles.  diag = 0: the tiles strictly
// below the diagonal (every entry (r, c) has r > c): L[r][c] = l_rc / d_c and
// U[c][r] = d_c l_rc.  diag = 1 (after, since it rewrites the d_c the first
// pass reads): the diagonal tiles, the same for r > c and u_cc = d_c^2.
template <typename T>
__global__ void __launch_bounds__(256) k_chol_to_lu(const FrontDev *__restrict__ fr, T *__restrict__ fronts, int diag) {
  const FrontDev F = fr[blockIdx.y];
  const int bi = blockIdx.x;
  if (bi * 32 >= F.f) return;
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  __shared__ T t[32][33];
  __shared__ T d[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int nbj = (F.s + 31) / 32;
  const int bj_lo = diag ? bi : 0, bj_hi = diag ? min(bi + 1, nbj) : min(bi, nbj);
  for (int bj = bj_lo; bj < bj_hi; ++bj) {
    const int r0 = bi * 32, c0 = bj * 32;
    __syncthreads();
    for (int cc = ty; cc < 32; cc += 8) {
      const int r = r0 + tx, c = c0 + cc;
      t[tx][cc] = (r < F.f && c < F.s && r >= c) ? A[r + int64_t(c) * ld] : T(0);
    }
    if (threadIdx.x < 32) {
      const int c = c0 + threadIdx.x;
      d[threadIdx.x] = c < F.s ? A[c + int64_t(c) * ld] : T(1);
    }
    __syncthreads();
    // lower part, scaled by 1 / d_c (coalesced down the columns)
    for (int cc = ty; cc < 32; cc += 8) {
      const int r = r0 + tx, c = c0 + cc;
      if (r < F.f && c < F.s) {
        if (r > c) A[r + int64_t(c) * ld] = t[tx][cc] / d[cc];
        else if (r == c) A[r + int64_t(c) * ld] = d[cc] * d[cc];
      }
    }
    // upper part, U[c][r] = d_c l_rc (coalesced along c)
    for (int rr = ty; rr < 32; rr += 8) {
      const int c = c0 + tx, r = r0 + rr;
      if (r < F.f && c < F.s && r > c) A[c + int64_t(r) * ld] = d[tx] * t[rr][tx];
    }
  }
}

// FP64 (and CUDA-core FP32) panel width, the same as the block LU's
template <typename T>
constexpr int chol_nb() {
  return LuCfg<T>::NB;
}

}  // namespace

template <typename T>
cudaError_t launch_chol_level(const FrontDev *fr, const Front *host_fr, int nfront, int max_s, int max_f, T *fronts,
                              int32_t *piv, int *err, cudaStream_t s, const LuAsync *la, Prof *prof,
                              const uint8_t *maps, float *pack, T *inv, const CholSchedule *sched,
                              const uint8_t *maps64, int bf16) {
  constexpr int NB = chol_nb<T>();
  const CholSchedule sch = sched ? *sched : CholSchedule();
  const int nsm = device_sms();
  cudaError_t e = cudaSuccess;
  auto panel = [&](int j0, cudaStream_t st) -> cudaError_t {
    double fpanel = 0.0;
    if (prof->timing)
      for (int k = 0; k < nfront; ++k) {
        const Front &F = host_fr[k];
        if (j0 >= F.s) continue;
        const double jb = std::min(NB, F.s - j0), rows = F.f - j0 - jb;
        fpanel += jb * jb * jb / 3.0 + rows * jb * jb;  // tile Cholesky + triangular solve of the rows below
      }
    const size_t e0 = prof->begin(st);
    if (chol_diag_blocked())
      k_chol_diag_blk<T, NB><<<nfront, kDiagThreads, 0, st>>>(fr, j0, fronts, piv, err, inv, bf16 != 0 ? 1 : 0);
    else
      k_chol_diag<T, NB><<<nfront, kDiagThreads, 0, st>>>(fr, j0, fronts, piv, err, inv, bf16 != 0 ? 1 : 0);
    const int below = max_f - j0 - 1;
    if (below > 0)
      k_chol_l21<T, NB><<<dim3(unsigned(cdiv_c(below, kL21Threads)), unsigned(nfront)), kL21Threads, 0, st>>>(
          fr, j0, fronts, inv);
    prof->end(P_PANEL, below > 0 ? 2 : 1, e0, fpanel, st);
    return cudaGetLastError();
  };
  bool tc = false;
  if constexpr (std::is_same<T, float>::value) tc = use_tensor_core_gemm_host() && maps != nullptr && pack != nullptr;
  if (bf16 && !tc) return cudaErrorNotSupported;  // BF16 block ends need the tensor-core path
  if constexpr (std::is_same<T, float>::value) {
    if (tc) {
      // ---- FP32: outer blocks of KB columns, tensor-core updates ----
      constexpr int KB = kLuOuterBlock;
      static_assert(NB == 64 && KB % NB == 0, "panel and outer block");
      const bool ahead = sch.lookahead != 0 && la != nullptr && la->side != nullptr && la->rest != nullptr &&
                         la->next != nullptr && la->panel != nullptr && la->done != nullptr;
      int64_t pack_tiles = 0;
      for (int k = 0; k < nfront; ++k) pack_tiles += cdiv_c(host_fr[k].f, kTcTile);
      const int64_t pack_stride = pack_tiles * kPackTileFloats;
      float *apack[2] = {pack, pack + pack_stride};
      cudaStream_t ms = ahead ? la->side : s;
      cudaStream_t rs = ahead ? la->rest : s;
      cudaEvent_t done_ev[2] = {ahead ? la->panel : nullptr, ahead ? la->done : nullptr};
      if (ahead) {
        if ((e = cudaEventRecord(la->next, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(ms, la->next, 0)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(rs, la->next, 0)) != cudaSuccess) return e;
      }
      // the lower-triangle rank-jbo update of the trailing block, columns [lo, hi)
      auto block_end = [&](int J, int lo, int hi, int budget, float *ap, cudaStream_t st, int max_tiles) -> cudaError_t {
        double fg = 0.0;
        for (int k = 0; k < nfront; ++k) {
          const Front &F = host_fr[k];
          if (J >= F.s) continue;
          const int jbo = std::min(KB, F.s - J), nrest = F.f - J - jbo;
          const double c0 = std::min(nrest, lo), c1 = std::min(nrest, hi);
          if (c1 <= c0) continue;
          // algorithmic flops: 2 jbo per entry of the lower triangle in the columns
          const double lower = (c1 - c0) * (double(nrest) - 0.5 * (c0 + c1 - 1.0));
          fg += 2.0 * double(jbo) * lower;
        }
        if (fg <= 0.0) return cudaSuccess;
        const int tlo = lo / kTcTile, thi = hi >= (INT_MAX - kTcTile) ? INT_MAX : hi / kTcTile;
        const size_t e0 = prof->begin(st);
        cudaError_t ge =
            (sch.wide && bf16 == 0)
                ? launch_gemm_tc_wide(fr, J, KB, nfront, max_f, fronts, err, st, tlo, thi, budget, ap, ap, /*lower=*/1,
                                      max_tiles, maps64, sch.wide == 2 ? 1 : 0)
                : launch_gemm_tc_ws(fr, J, KB, nfront, max_f, fronts, err, st, tlo, thi, budget, maps, ap, ap,
                                    /*lower=*/1, max_tiles, maps64, bf16);
        prof->end(P_GEMM, 1, e0, fg, st);
        return ge;
      };
      const int nblk = cdiv_c(max_s, KB);
      if ((e = panel(0, ms)) != cudaSuccess) return e;
      for (int b = 0; b < nblk; ++b) {
        const int J = b * KB;
        for (int i = 0; i < KB / NB; ++i) {
          const int jp = J + i * NB;
          if (jp >= max_s) break;
          if (i > 0 && (e = panel(jp, ms)) != cudaSuccess) return e;
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
            if ((e = launch_gemm_tc_inner(fr, jp, KB, nfront, max_f, fronts, err, ms, nsm, /*sym=*/1)) != cudaSuccess)
              return e;
            prof->end(P_GEMM_INNER, 1, e0, fgemm, ms);
          }
        }
        const bool more = J + KB < max_s;
        float *ap = apack[b & 1];
        if ((e = bf16 ? launch_pack_bf16(fr, J, KB, nfront, max_f, fronts, ap, ms, bf16)
                      : launch_pack_a(fr, J, KB, nfront, max_f, fronts, ap, ms)) != cudaSuccess)
          return e;
        if (ahead) {
          // the rest of the block end on the low-priority stream; the next
          // block's columns stay on the panel stream
          if ((e = cudaEventRecord(la->next, ms)) != cudaSuccess) return e;
          if ((e = cudaStreamWaitEvent(rs, la->next, 0)) != cudaSuccess) return e;
          const int keep = sch.panel_sms >= 0 ? sch.panel_sms : nfront;
          if ((e = block_end(J, KB, INT_MAX, std::max(nsm - keep, nsm / 2), ap, rs, sch.tiles_per_cta)) != cudaSuccess)
            return e;
          if ((e = cudaEventRecord(done_ev[b & 1], rs)) != cudaSuccess) return e;
          if (b > 0 && (e = cudaStreamWaitEvent(ms, done_ev[(b - 1) & 1], 0)) != cudaSuccess) return e;
          if ((e = block_end(J, 0, KB, nsm, ap, ms, 0)) != cudaSuccess) return e;
        } else {
          if ((e = block_end(J, 0, INT_MAX, nsm, ap, s, 0)) != cudaSuccess) return e;
        }
        if (more && (e = panel(J + KB, ms)) != cudaSuccess) return e;
      }
      if (ahead) {
        if ((e = cudaStreamWaitEvent(ms, done_ev[(nblk - 1) & 1], 0)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(la->next, ms)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, la->next, 0)) != cudaSuccess) return e;
      }
      return cudaGetLastError();
    }
  }
  // ---- one lower-triangle update per panel on the CUDA cores ----
  for (int j0 = 0; j0 < max_s; j0 += NB) {
    if ((e = panel(j0, s)) != cudaSuccess) return e;
    double fgemm = 0.0;
    if (prof->timing)
      for (int k = 0; k < nfront; ++k) {
        const Front &F = host_fr[k];
        if (j0 >= F.s) continue;
        const double jb = std::min(NB, F.s - j0), nrest = F.f - j0 - jb;
        fgemm += nrest * (nrest + 1.0) * jb;  // 2 flop per entry of the lower triangle
      }
    const size_t e0 = prof->begin(s);
    if ((e = launch_gemm_update_sym<T>(fr, j0, nfront, max_f, fronts, s)) != cudaSuccess) return e;
    prof->end(P_GEMM, 1, e0, fgemm, s);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chol_to_lu(const FrontDev *fr, int nfront, int max_f, T *fronts, cudaStream_t s, Prof *prof,
                              double bytes) {
  if (nfront == 0) return cudaSuccess;
  const dim3 g(unsigned(cdiv_c(max_f, 32)), unsigned(nfront));
  const size_t e0 = prof->begin(s);
  k_chol_to_lu<T><<<g, 256, 0, s>>>(fr, fronts, 0);
  k_chol_to_lu<T><<<g, 256, 0, s>>>(fr, fronts, 1);
  prof->end(P_OTHER, 2, e0, bytes, s);
  return cudaGetLastError();
}

template cudaError_t launch_chol_level<double>(const FrontDev *, const Front *, int, int, int, double *, int32_t *,
                                               int *, cudaStream_t, const LuAsync *, Prof *, const uint8_t *, float *,
                                               double *, const CholSchedule *, const uint8_t *, int);
template cudaError_t launch_chol_level<float>(const FrontDev *, const Front *, int, int, int, float *, int32_t *,
                                              int *, cudaStream_t, const LuAsync *, Prof *, const uint8_t *, float *,
                                              float *, const CholSchedule *, const uint8_t *, int);
template cudaError_t launch_chol_to_lu<double>(const FrontDev *, int, int, double *, cudaStream_t, Prof *, double);
template cudaError_t launch_chol_to_lu<float>(const FrontDev *, int, int, float *, cudaStream_t, Prof *, double);

}  // namespace h2sp
