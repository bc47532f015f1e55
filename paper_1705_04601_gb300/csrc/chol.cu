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
#include <type_traits>

#include "kernels.h"

namespace h2sp {
namespace {

inline int cdiv_c(int64_t a, int64_t b) { return int((a + b - 1) / b); }

// Cholesky of the diagonal tile [j0, j0 + jb) of every front.  Thread r holds
// row r of the tile (its lower part) in registers.  Per column j: thread j
// takes the square root of its diagonal entry, every row below scales its
// entry j by it and publishes it, and updates its entries j+1 .. r.  A
// pivot that is not positive and finite sets bit 8 of *err (the matrix is
// not positive definite in this precision) and is replaced by 1 so that the
// factorization stays finite.  Then thread c forms column c of L11^-1 by
// forward substitution, y_r = -(sum_{c<=m<r} l_rm y_m) / l_rr with
// y_c = 1 / l_cc, each row's sum split over four partial sums, and writes it
// to inv[front][r * NB + c] (row-major, zero above the diagonal and beyond jb).
template <typename T, int NB>
__global__ void __launch_bounds__(NB) k_chol_diag(const FrontDev *__restrict__ fr, int j0, T *__restrict__ fronts,
                                                  int32_t *__restrict__ piv, int *__restrict__ err,
                                                  T *__restrict__ inv) {
  const FrontDev F = fr[blockIdx.x];
  if (j0 >= F.s) return;  // uniform over the CTA
  const int jb = min(NB, F.s - j0);
  T *A = fronts + F.off;
  const int64_t ld = F.ld;
  constexpr int P = NB + 1;       // padded row length of the tile in shared memory
  __shared__ T col[NB];           // the current column below the pivot, and the pivot itself
  __shared__ T Lr[NB * P];        // L11 row-major (row r at r * P), zero above the diagonal and beyond jb
  const int r = threadIdx.x;
  {
    T x[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) x[c] = (r < jb && c <= r) ? A[(j0 + r) + int64_t(j0 + c) * ld] : T(0);
    for (int j = 0; j < jb; ++j) {
      T xj = T(0);
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c == j) xj = x[c];
      if (r == j) {
        T a = xj;
        if (!(a > T(0)) || !isfinite(a)) {
          atomicOr(err, 8);
          a = T(1);
        }
        col[j] = sqrt(a);
      }
      __syncthreads();
      const T d = col[j];
      T l = T(0);
      if (r > j && r < jb) {
        l = xj / d;
        col[r] = l;
      }
      __syncthreads();
      if (r >= j && r < jb) {
        // entry j becomes final (l, or d on the diagonal); entries j+1 .. r take the update
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c == j) x[c] = (r == j) ? d : l;
          else if (c > j && c <= r) x[c] -= l * col[c];
        }
      }
      __syncthreads();  // col is rewritten by the next column
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) Lr[r * P + c] = (r < jb && c <= r) ? x[c] : T(0);
    if (r < jb) {
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c <= r) A[(j0 + r) + int64_t(j0 + c) * ld] = x[c];
      piv[F.piv_off + j0 + r] = j0 + r;
    }
  }
  __syncthreads();
  // column c = r of L11^-1
  const int c = r;
  T y[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) y[q] = T(0);
  if (c < jb) {
#pragma unroll
    for (int rr = 0; rr < NB; ++rr) {
      if (rr < c || rr >= jb) continue;
      if (rr == c) {
        y[rr] = T(1) / Lr[rr * P + rr];
        continue;
      }
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
      for (int m = 0; m < rr; m += 4) {
        if (m >= c) s0 += Lr[rr * P + m] * y[m];
        if (m + 1 < rr && m + 1 >= c) s1 += Lr[rr * P + m + 1] * y[m + 1];
        if (m + 2 < rr && m + 2 >= c) s2 += Lr[rr * P + m + 2] * y[m + 2];
        if (m + 3 < rr && m + 3 >= c) s3 += Lr[rr * P + m + 3] * y[m + 3];
      }
      y[rr] = -((s0 + s1) + (s2 + s3)) / Lr[rr * P + rr];
    }
  }
  T *Li = inv + int64_t(blockIdx.x) * NB * NB;
#pragma unroll
  for (int rr = 0; rr < NB; ++rr) Li[rr * NB + c] = y[rr];
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
                              const uint8_t *maps, float *pack, T *inv, const CholSchedule *sched) {
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
    k_chol_diag<T, NB><<<nfront, NB, 0, st>>>(fr, j0, fronts, piv, err, inv);
    const int below = max_f - j0 - 1;
    if (below > 0)
      k_chol_l21<T, NB><<<dim3(unsigned(cdiv_c(below, kL21Threads)), unsigned(nfront)), kL21Threads, 0, st>>>(
          fr, j0, fronts, inv);
    prof->end(P_PANEL, below > 0 ? 2 : 1, e0, fpanel, st);
    return cudaGetLastError();
  };
  bool tc = false;
  if constexpr (std::is_same<T, float>::value) tc = use_tensor_core_gemm_host() && maps != nullptr && pack != nullptr;
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
        cudaError_t ge = launch_gemm_tc_ws(fr, J, KB, nfront, max_f, fronts, err, st, tlo, thi, budget, maps, ap, ap,
                                           /*lower=*/1, max_tiles);
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
        if ((e = launch_pack_a(fr, J, KB, nfront, max_f, fronts, ap, ms)) != cudaSuccess) return e;
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
                                               double *, const CholSchedule *);
template cudaError_t launch_chol_level<float>(const FrontDev *, const Front *, int, int, int, float *, int32_t *,
                                              int *, cudaStream_t, const LuAsync *, Prof *, const uint8_t *, float *,
                                              float *, const CholSchedule *);
template cudaError_t launch_chol_to_lu<double>(const FrontDev *, int, int, double *, cudaStream_t, Prof *, double);
template cudaError_t launch_chol_to_lu<float>(const FrontDev *, int, int, float *, cudaStream_t, Prof *, double);

}  // namespace h2sp
