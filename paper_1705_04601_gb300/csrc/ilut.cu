// Threshold incomplete LU of S (the preconditioner of §5.5): the ILUt rule
// on the rows of S taken in the block LU's elimination order (supernodes in
// order, the rows of a node kept together), without pivoting:
//   for each row i:  w = A[i, :],  tau_i = tau ||A[i, :]||_2;
//   for k < i with w_k != 0, in increasing k:
//       w_k /= u_kk;  |w_k| < tau_i -> w_k = 0 (dropped), else w -= w_k U[k, :];
//   every w_j (j != i) with |w_j| < tau_i is dropped;  L[i, :i] = w[:i]
//   (unit diagonal),  U[i, i:] = w[i:].
// The fill of row i stays inside the structural pattern of the exact LU, so
// row i needs only rows of its own supernode before it and rows of the
// supernodes below it in the elimination tree: the supernodes of one
// elimination level are independent.  One CTA per supernode walks its rows
// in order, with the row in a dense work array (n values) and a bitmap of its
// columns (plus a summary bit per bitmap word in shared memory) to find the
// next column k; kept rows go to a shared pool (an atomic cursor), L part
// then U part, columns ascending.  The triangular solves walk the same
// levels (forward deepest first, backward from the top), one CTA per
// supernode, a row at a time.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.h"

namespace h2sp {
namespace {

constexpr int kIluThreads = 256;

__device__ __forceinline__ double cta_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < kIluThreads / 32; ++i) t += red[i];
  __syncthreads();
  return t;
}

__device__ __forceinline__ int64_t cta_scan(int64_t v, int64_t *red, int64_t *total) {
  // exclusive scan over the CTA
  __shared__ int64_t wsum[kIluThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t a = 0;
    for (int i = 0; i < kIluThreads / 32; ++i) {
      const int64_t t = wsum[i];
      red[i] = a;
      a += t;
    }
    red[kIluThreads / 32] = a;
  }
  __syncthreads();
  const int64_t before = red[w] + x - v;
  *total = red[kIluThreads / 32];
  __syncthreads();
  return before;
}

// A = S in elimination order, CSR: row e of A is row perm[e] of S.  One CTA
// per node v: its rows' entries, block by block in the order of the column
// nodes' first elimination row (ablk: the block row's blocks so sorted), each
// block a run of consecutive columns.
template <typename TS>
__global__ void __launch_bounds__(kIluThreads) k_ilu_gather(
    const int64_t *__restrict__ brow_ptr, const int32_t *__restrict__ bcol, const int64_t *__restrict__ val_off,
    const int64_t *__restrict__ node_off, const TS *__restrict__ vals, const int32_t *__restrict__ ablk,
    const int64_t *__restrict__ epos, const int64_t *__restrict__ a_ptr, int32_t *__restrict__ a_col,
    double *__restrict__ a_val) {
  const int v = blockIdx.x;
  const int64_t r0 = node_off[v], dv = node_off[v + 1] - r0;
  const int64_t z0 = brow_ptr[v], z1 = brow_ptr[v + 1];
  for (int64_t i = 0; i < dv; ++i) {
    const int64_t e = epos[r0 + i];
    int64_t at = a_ptr[e];
    for (int64_t q = z0; q < z1; ++q) {
      const int64_t z = ablk[q];
      const int w = bcol[z];
      const int64_t c0 = node_off[w], dw = node_off[w + 1] - c0;
      const int64_t ec = epos[c0];  // the node's columns are consecutive in elimination order
      const TS *B = vals + val_off[z];
      for (int64_t j = threadIdx.x; j < dw; j += kIluThreads) {
        a_col[at + j] = int32_t(ec + j);
        a_val[at + j] = double(B[i + j * dv]);
      }
      at += dw;
    }
  }
}

struct IluArgs {
  const int64_t *a_ptr;
  const int32_t *a_col;
  const double *a_val;
  const int64_t *sn_row;   // rows of supernode k: [sn_row[k], sn_row[k + 1])
  int64_t *row_off;        // pool offset of each row's entries
  int32_t *nl, *nu;        // kept L / U entries of each row (U starts with the diagonal)
  int32_t *pool_col;
  double *pool_val;
  unsigned long long *cursor;
  int64_t cap;
  double *w_all;           // per CTA: n values
  uint32_t *bits_all;      // per CTA: ceil(n / 32) words
  int64_t n, nwords;
  double tau;
  int *err;                // bit 1: zero pivot, bit 2: pool overflow
};

// one elimination level: supernodes [k0, k1), persistent CTAs
__global__ void __launch_bounds__(kIluThreads) k_ilut_level(IluArgs a, int k0, int k1) {
  extern __shared__ uint32_t summary[];  // a bit per bitmap word
  __shared__ double red[kIluThreads / 32];
  __shared__ int64_t sred[kIluThreads / 32 + 1];
  __shared__ int s_lo, s_hi;
  __shared__ int64_t s_k;
  __shared__ double s_wk;
  __shared__ int64_t s_off;
  double *w = a.w_all + int64_t(blockIdx.x) * a.n;
  uint32_t *bits = a.bits_all + int64_t(blockIdx.x) * a.nwords;
  const int nsum = int((a.nwords + 31) / 32);
  const int tid = threadIdx.x;
  for (int i = tid; i < nsum; i += kIluThreads) summary[i] = 0u;
  __syncthreads();
  for (int k = k0 + int(blockIdx.x); k < k1; k += gridDim.x) {
    for (int64_t i = a.sn_row[k]; i < a.sn_row[k + 1]; ++i) {
      // once the pool has overflowed, rows are not computed (the host retries
      // with a larger pool): their inputs may not have been stored
      if (tid == 0) s_lo = (*(volatile int *)a.err & 2) ? -2 : INT32_MAX, s_hi = -1;
      __syncthreads();
      if (s_lo == -2) {
        if (tid == 0) a.row_off[i] = 0, a.nl[i] = 0, a.nu[i] = 0;
        __syncthreads();
        continue;
      }
      // ---- load row i ----
      double nrm = 0.0;
      int lo = INT32_MAX, hi = -1;
      for (int64_t q = a.a_ptr[i] + tid; q < a.a_ptr[i + 1]; q += kIluThreads) {
        const int j = a.a_col[q];
        const double v = a.a_val[q];
        w[j] = v;
        nrm += v * v;
        atomicOr(&bits[j >> 5], 1u << (j & 31));
        atomicOr(&summary[j >> 10], 1u << ((j >> 5) & 31));
        lo = min(lo, j >> 5);
        hi = max(hi, j >> 5);
      }
      atomicMin(&s_lo, lo);
      atomicMax(&s_hi, hi);
      const double tau_i = a.tau * sqrt(cta_sum(nrm, red));
      // ---- eliminate with k < i in increasing order ----
      int64_t kcur = -1;
      while (true) {
        if (tid == 0) {
          // the smallest column j with kcur < j < i whose bit is set: the rest
          // of the first word, then the next words the summary marks
          int64_t nxt = -1;
          const int64_t start = kcur < 0 ? (int64_t(s_lo) << 5) : kcur + 1;
          if (start < i) {
            int64_t wd = start >> 5;
            const int64_t wlast = (i - 1) >> 5;
            uint32_t m = bits[wd] & (~0u << (start & 31));
            while (true) {
              if (m) {
                nxt = (wd << 5) + __ffs(m) - 1;
                break;
              }
              ++wd;
              while (wd <= wlast) {
                const uint32_t sb = summary[wd >> 5] >> (wd & 31);
                if (sb) {
                  wd += __ffs(sb) - 1;
                  break;
                }
                wd = ((wd >> 5) + 1) << 5;
              }
              if (wd > wlast) break;
              m = bits[wd];
            }
            if (nxt >= i) nxt = -1;
          }
          s_k = nxt;
          if (nxt >= 0) {
            const int64_t uo = a.row_off[nxt] + a.nl[nxt];  // U row of nxt: its diagonal first
            double wk = w[nxt] / a.pool_val[uo];
            if (fabs(wk) < tau_i) wk = 0.0;
            w[nxt] = wk;
            s_wk = wk;
          }
        }
        __syncthreads();
        const int64_t k = s_k;
        if (k < 0) break;
        const double wk = s_wk;
        if (wk != 0.0) {
          const int64_t uo = a.row_off[k] + a.nl[k];
          const int nuk = a.nu[k];
          for (int q = 1 + tid; q < nuk; q += kIluThreads) {
            const int j = a.pool_col[uo + q];
            w[j] -= wk * a.pool_val[uo + q];
            atomicOr(&bits[j >> 5], 1u << (j & 31));
            atomicOr(&summary[j >> 10], 1u << ((j >> 5) & 31));
            if ((j >> 5) > s_hi) atomicMax(&s_hi, j >> 5);
          }
        }
        kcur = k;
        __syncthreads();
      }
      // ---- keep, count, store ----
      const int wlo = s_lo, whi = s_hi;
      const int nw = whi - wlo + 1;
      const int per = (nw + kIluThreads - 1) / kIluThreads;
      const int w0 = wlo + min(nw, tid * per), w1 = wlo + min(nw, (tid + 1) * per);
      int64_t mine_l = 0, mine_u = 0;
      for (int wd = w0; wd < w1; ++wd) {
        uint32_t m = bits[wd];
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1u;
          const int64_t j = (int64_t(wd) << 5) + b;
          const double v = w[j];
          const bool keep = j == i ? true : (j < i ? v != 0.0 : fabs(v) >= tau_i);
          if (keep) {
            if (j < i) ++mine_l;
            else ++mine_u;
          }
        }
      }
      int64_t tot_l, tot_u;
      const int64_t pre_l = cta_scan(mine_l, sred, &tot_l);
      const int64_t pre_u = cta_scan(mine_u, sred, &tot_u);
      if (tid == 0) {
        const unsigned long long o = atomicAdd(a.cursor, (unsigned long long)(tot_l + tot_u));
        s_off = int64_t(o);
        if (int64_t(o) + tot_l + tot_u > a.cap) atomicOr(a.err, 2);
        a.row_off[i] = int64_t(o);
        a.nl[i] = int32_t(tot_l);
        a.nu[i] = int32_t(tot_u);
        if (w[i] == 0.0) atomicOr(a.err, 1);
      }
      __syncthreads();
      const int64_t off = s_off;
      const bool fits = off + tot_l + tot_u <= a.cap;
      int64_t pl = off + pre_l, pu = off + tot_l + pre_u;
      for (int wd = w0; wd < w1; ++wd) {
        uint32_t m = bits[wd];
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1u;
          const int64_t j = (int64_t(wd) << 5) + b;
          const double v = w[j];
          const bool keep = j == i ? true : (j < i ? v != 0.0 : fabs(v) >= tau_i);
          if (keep && fits) {
            const int64_t at = j < i ? pl++ : pu++;
            a.pool_col[at] = int32_t(j);
            a.pool_val[at] = v;
          }
          w[j] = 0.0;
        }
        bits[wd] = 0u;
      }
      __syncthreads();
      for (int sw = (wlo >> 5) + tid; sw <= (whi >> 5); sw += kIluThreads) summary[sw] = 0u;
      __syncthreads();
    }
  }
}

// forward: z_i = c_{perm[i]} - sum_{k < i} L_ik z_k (unit L), a row at a time
__global__ void __launch_bounds__(kIluThreads) k_ilut_fwd(IluArgs a, int k0, int k1, const int32_t *__restrict__ perm,
                                                          const double *__restrict__ c, double *__restrict__ z,
                                                          int nrhs) {
  __shared__ double red[kIluThreads / 32];
  for (int k = k0 + int(blockIdx.x); k < k1; k += gridDim.x)
    for (int64_t i = a.sn_row[k]; i < a.sn_row[k + 1]; ++i) {
      const int64_t o = a.row_off[i];
      const int nl = a.nl[i];
      for (int r = 0; r < nrhs; ++r) {
        double s = 0.0;
        for (int q = threadIdx.x; q < nl; q += kIluThreads) s += a.pool_val[o + q] * z[a.pool_col[o + q] + int64_t(r) * a.n];
        s = cta_sum(s, red);
        if (threadIdx.x == 0) z[i + int64_t(r) * a.n] = c[perm[i] + int64_t(r) * a.n] - s;
      }
      __syncthreads();
    }
}

// backward: z_i = (z_i - sum_{j > i} U_ij z_j) / U_ii, rows in reverse; y_{perm[i]} = z_i
__global__ void __launch_bounds__(kIluThreads) k_ilut_bwd(IluArgs a, int k0, int k1, const int32_t *__restrict__ perm,
                                                          double *__restrict__ z, double *__restrict__ y, int nrhs) {
  __shared__ double red[kIluThreads / 32];
  for (int k = k0 + int(blockIdx.x); k < k1; k += gridDim.x)
    for (int64_t i = a.sn_row[k + 1] - 1; i >= a.sn_row[k]; --i) {
      const int64_t o = a.row_off[i] + a.nl[i];
      const int nu = a.nu[i];
      for (int r = 0; r < nrhs; ++r) {
        double s = 0.0;
        for (int q = 1 + threadIdx.x; q < nu; q += kIluThreads)
          s += a.pool_val[o + q] * z[a.pool_col[o + q] + int64_t(r) * a.n];
        s = cta_sum(s, red);
        if (threadIdx.x == 0) {
          const double zi = (z[i + int64_t(r) * a.n] - s) / a.pool_val[o];
          z[i + int64_t(r) * a.n] = zi;
          y[perm[i] + int64_t(r) * a.n] = zi;
        }
      }
      __syncthreads();
    }
}

}  // namespace

// ---- host side ----

void IlutState::release() {
  for (void *p : bufs) cudaFree(p);
  bufs.clear();
  ready = false;
}

template <class T>
static T *ilu_alloc(IlutState &st, size_t n) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw IlutFail{e == cudaErrorMemoryAllocation ? int(H2SP_ENOMEM) : int(H2SP_ECUDA), cudaGetErrorString(e)};
  }
  st.bufs.push_back(p);
  return static_cast<T *>(p);
}

static void ilu_ck(cudaError_t e) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw IlutFail{e == cudaErrorMemoryAllocation ? int(H2SP_ENOMEM) : int(H2SP_ECUDA), cudaGetErrorString(e)};
  }
}

template <class T>
static T *ilu_put(IlutState &st, const std::vector<T> &v) {
  T *p = ilu_alloc<T>(st, v.size());
  if (!v.empty()) ilu_ck(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

void ilut_factor(IlutState &st, const Plan &p, const int64_t *brow_ptr, const int32_t *bcol, const int64_t *val_off,
                 const int64_t *node_off, const void *S, bool s_fp32, double tau, cudaStream_t s, Prof *prof) {
  st.release();
  const int64_t n = p.n;
  const int nn = int(p.node_size.size());
  const int nsn = int(p.sn_ptr.size()) - 1;
  // elimination order of the scalar rows: supernode by supernode, nodes in order, rows kept together
  std::vector<int32_t> perm(static_cast<size_t>(n));
  std::vector<int64_t> epos(static_cast<size_t>(n)), sn_row(static_cast<size_t>(nsn) + 1, 0);
  {
    int64_t e = 0;
    for (int k = 0; k < nsn; ++k) {
      sn_row[size_t(k)] = e;
      for (int q = p.sn_ptr[size_t(k)]; q < p.sn_ptr[size_t(k) + 1]; ++q) {
        const int v = p.order[size_t(q)];
        for (int64_t r = p.node_off[size_t(v)]; r < p.node_off[size_t(v) + 1]; ++r) {
          perm[size_t(e)] = int32_t(r);
          epos[size_t(r)] = e;
          ++e;
        }
      }
    }
    sn_row[size_t(nsn)] = e;
  }
  // rows of A: the block row's blocks sorted by the column node's first elimination row
  std::vector<int32_t> ablk(static_cast<size_t>(p.brow_ptr[size_t(nn)]));
  std::vector<int64_t> a_ptr(static_cast<size_t>(n) + 1, 0);
  for (int v = 0; v < nn; ++v) {
    const int64_t z0 = p.brow_ptr[size_t(v)], z1 = p.brow_ptr[size_t(v) + 1];
    int64_t len = 0;
    for (int64_t z = z0; z < z1; ++z) {
      ablk[size_t(z)] = int32_t(z);
      len += p.node_size[size_t(p.bcol[size_t(z)])];
    }
    std::sort(ablk.begin() + z0, ablk.begin() + z1, [&](int32_t x, int32_t y) {
      return epos[size_t(p.node_off[size_t(p.bcol[size_t(x)])])] < epos[size_t(p.node_off[size_t(p.bcol[size_t(y)])])];
    });
    for (int64_t r = p.node_off[size_t(v)]; r < p.node_off[size_t(v) + 1]; ++r) a_ptr[size_t(epos[size_t(r)]) + 1] = len;
  }
  for (int64_t e = 0; e < n; ++e) a_ptr[size_t(e) + 1] += a_ptr[size_t(e)];
  const int64_t nnz = a_ptr[size_t(n)];
  st.n = n;
  st.perm = ilu_put(st, perm);
  int64_t *d_epos = ilu_put(st, epos);
  int64_t *d_aptr = ilu_put(st, a_ptr);
  int32_t *d_ablk = ilu_put(st, ablk);
  int32_t *d_acol = ilu_alloc<int32_t>(st, size_t(nnz));
  double *d_aval = ilu_alloc<double>(st, size_t(nnz));
  {
    const size_t e0 = prof->begin();
    if (s_fp32)
      k_ilu_gather<float><<<unsigned(std::max(nn, 1)), kIluThreads, 0, s>>>(
          brow_ptr, bcol, val_off, node_off, static_cast<const float *>(S), d_ablk, d_epos, d_aptr, d_acol, d_aval);
    else
      k_ilu_gather<double><<<unsigned(std::max(nn, 1)), kIluThreads, 0, s>>>(
          brow_ptr, bcol, val_off, node_off, static_cast<const double *>(S), d_ablk, d_epos, d_aptr, d_acol, d_aval);
    ilu_ck(cudaGetLastError());
    prof->end(P_ASSEMBLE, 1, e0, double(nnz) * 20.0);
  }
  st.sn_row = ilu_put(st, sn_row);
  st.row_off = ilu_alloc<int64_t>(st, size_t(n));
  st.nl = ilu_alloc<int32_t>(st, size_t(n));
  st.nu = ilu_alloc<int32_t>(st, size_t(n));
  st.err = ilu_alloc<int>(st, 1);
  st.cursor = ilu_alloc<unsigned long long>(st, 1);
  st.levels.clear();
  for (size_t i = 0; i + 1 < p.front_level_ptr.size(); ++i)
    st.levels.push_back({p.front_level_ptr[i], p.front_level_ptr[i + 1]});
  int max_level = 1;
  for (auto &L : st.levels) max_level = std::max(max_level, L.second - L.first);
  const int grid = std::max(1, std::min(max_level, 2 * device_sms()));
  st.grid = grid;
  const int64_t nwords = (n + 31) / 32;
  double *d_w = ilu_alloc<double>(st, size_t(grid) * size_t(n));
  uint32_t *d_bits = ilu_alloc<uint32_t>(st, size_t(grid) * size_t(nwords));
  ilu_ck(cudaMemsetAsync(d_w, 0, sizeof(double) * size_t(grid) * size_t(n), s));
  ilu_ck(cudaMemsetAsync(d_bits, 0, sizeof(uint32_t) * size_t(grid) * size_t(nwords), s));
  const size_t smem = size_t((nwords + 31) / 32) * sizeof(uint32_t);
  if (smem > size_t(200) * 1024) throw IlutFail{H2SP_EUNSUPPORTED, "ILUt: n too large for the bitmap summary"};
  ilu_ck(smem_attr((const void *)k_ilut_level, int(std::max<size_t>(smem, 1))));
  // pool: grown on overflow
  int64_t cap = std::max<int64_t>(4 * nnz, 64 * n);
  for (int attempt = 0;; ++attempt) {
    st.pool_col = ilu_alloc<int32_t>(st, size_t(cap));
    st.pool_val = ilu_alloc<double>(st, size_t(cap));
    ilu_ck(cudaMemsetAsync(st.err, 0, sizeof(int), s));
    ilu_ck(cudaMemsetAsync(st.cursor, 0, sizeof(unsigned long long), s));
    IluArgs a{d_aptr, d_acol, d_aval, st.sn_row, st.row_off, st.nl, st.nu, st.pool_col, st.pool_val, st.cursor, cap,
              d_w, d_bits, n, nwords, tau, st.err};
    const size_t e0 = prof->begin();
    for (auto &L : st.levels) {
      const int g = std::min(grid, L.second - L.first);
      k_ilut_level<<<unsigned(g), kIluThreads, std::max<size_t>(smem, 4), s>>>(a, L.first, L.second);
    }
    ilu_ck(cudaGetLastError());
    prof->end(P_PANEL, int(st.levels.size()), e0, 0.0);
    int herr = 0;
    unsigned long long used = 0;
    ilu_ck(cudaMemcpyAsync(&herr, st.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ilu_ck(cudaMemcpyAsync(&used, st.cursor, sizeof(used), cudaMemcpyDeviceToHost, s));
    ilu_ck(cudaStreamSynchronize(s));
    if (herr & 1) throw IlutFail{H2SP_ESINGULAR, "ILUt: a zero pivot"};
    if (!(herr & 2)) {
      st.nnz = int64_t(used);
      break;
    }
    if (attempt >= 4) throw IlutFail{H2SP_ENOMEM, "ILUt: the factors outgrew the pool"};
    cap *= 4;
  }
  st.tau = tau;
  st.ready = true;
}

void ilut_solve(IlutState &st, double *y, int nrhs, double *z, cudaStream_t s, Prof *prof) {
  IluArgs a{nullptr, nullptr, nullptr, st.sn_row, st.row_off, st.nl, st.nu, st.pool_col, st.pool_val, st.cursor, 0,
            nullptr, nullptr, st.n, 0, st.tau, st.err};
  const size_t e0 = prof->begin();
  for (auto &L : st.levels) {
    const int g = std::min(st.grid, L.second - L.first);
    k_ilut_fwd<<<unsigned(g), kIluThreads, 0, s>>>(a, L.first, L.second, st.perm, y, z, nrhs);
  }
  for (int li = int(st.levels.size()) - 1; li >= 0; --li) {
    const auto &L = st.levels[size_t(li)];
    const int g = std::min(st.grid, L.second - L.first);
    k_ilut_bwd<<<unsigned(g), kIluThreads, 0, s>>>(a, L.first, L.second, st.perm, z, y, nrhs);
  }
  ilu_ck(cudaGetLastError());
  prof->end(P_SOLVE, int(2 * st.levels.size()), e0, double(st.nnz) * 12.0 * nrhs);
}

}  // namespace h2sp
