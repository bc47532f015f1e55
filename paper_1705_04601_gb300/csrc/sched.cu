// The level schedule of §2.2-2.3 on the device: integer kernels over the
// cluster tree that give, per cluster, the local block size m_t, the basis
// part k'_t = min(k_t, m_t) and the non-basis part d_t = m_t - k'_t (§2.2,
// the split of Q_t = [basis | non-basis]), the row offset of the basis part
// in the parent's block (the stacking of W_t, §4.2), the offset of X_l(t) in
// the level-l vector; the order of the S nodes (non-basis parts level by
// level, then the top clusters: the permutation of §2.3 that makes
// A = U S V^T with block-diagonal U, V); the close lists
// Near_{l+1} = sort-unique {(par a, par b) : (a, b) in Near_l or Far_l}
// (§2.3, the far pairs of level l fold into close blocks of level l+1); and
// the level maps of the applies U^T b / V y: for each cluster of a
// compressed level, where its basis part goes in the next level's vector
// and its non-basis part in S's.  Bit-exact integer work, run once per
// structure.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"

namespace h2sp {
namespace {

constexpr int kScanThreads = 1024;

// depth of cluster t: the d with lp[d] <= t < lp[d + 1]
__device__ __forceinline__ int depth_of(const int32_t *__restrict__ lp, int D, int t) {
  int lo = 0, hi = D;  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (lp[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// children of every cluster (consecutive by the descriptor's rule)
__global__ void k_children(const int32_t *__restrict__ parent, int first, int ncl, int32_t *__restrict__ cstart,
                           int32_t *__restrict__ ccnt) {
  const int c = first + int(blockIdx.x * blockDim.x + threadIdx.x);
  if (c >= ncl) return;
  const int pa = parent[c];
  atomicAdd(&ccnt[pa], 1);
  if (parent[c - 1] != pa) cstart[pa] = c;  // c - 1 >= 0: first >= 1
}

// l_stop = 1 + the highest level with an admissible pair
__global__ void k_lstop(const int32_t *__restrict__ lp, int D, const int64_t *__restrict__ far_ptr, int ncl,
                        int *__restrict__ lstop) {
  const int t = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (t >= ncl) return;
  if (far_ptr[t + 1] > far_ptr[t]) atomicMax(lstop, D - depth_of(lp, D, t) + 1);
}

// leaves: m_t = |t|
__global__ void k_leaf_sizes(const int64_t *__restrict__ size, int lo, int hi, int64_t *__restrict__ m) {
  const int t = lo + int(blockIdx.x * blockDim.x + threadIdx.x);
  if (t < hi) m[t] = size[t];
}

// level l < l_stop: one thread per parent (clusters [plo, phi) of level l + 1)
// splits each child's block (k'_c, d_c), stacks the basis parts in child
// order (off_c) and sets the parent's block size m_p = sum k'_c
__global__ void k_level_sizes(const int32_t *__restrict__ cstart, const int32_t *__restrict__ ccnt,
                              const int32_t *__restrict__ rank, int plo, int phi, int64_t *__restrict__ m,
                              int64_t *__restrict__ kp, int64_t *__restrict__ d, int64_t *__restrict__ off) {
  const int p = plo + int(blockIdx.x * blockDim.x + threadIdx.x);
  if (p >= phi) return;
  int64_t acc = 0;
  const int c0 = cstart[p], nc = ccnt[p];
  for (int c = c0; c < c0 + nc; ++c) {
    const int64_t mc = m[c];
    const int64_t k = min(int64_t(rank[c]), mc);
    kp[c] = k;
    d[c] = mc - k;
    off[c] = acc;
    acc += k;
  }
  m[p] = acc;
}

// level l_stop: nothing is compressed, d_t = m_t
__global__ void k_top_sizes(int lo, int hi, const int64_t *__restrict__ m, int64_t *__restrict__ kp,
                            int64_t *__restrict__ d) {
  const int t = lo + int(blockIdx.x * blockDim.x + threadIdx.x);
  if (t >= hi) return;
  kp[t] = 0;
  d[t] = m[t];
}

// exclusive scan of v over a 1024-thread CTA; returns the thread's prefix and
// leaves the CTA total in *total
__device__ int64_t block_scan(int64_t v, int64_t *total) {
  __shared__ int64_t warp_sum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < int(blockDim.x >> 5) ? warp_sum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sum[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int64_t before = (w > 0 ? warp_sum[w - 1] : 0) + x - v;
  *total = warp_sum[(blockDim.x >> 5) - 1];
  __syncthreads();  // warp_sum is reused by the next call
  return before;
}

// One CTA walks the levels l = 0 .. l_stop in order (clusters of level l are
// [lp[D - l], lp[D - l + 1])) and scans, with carries across chunks:
//   xoff_t        prefix of m within the level;
//   node_of_t     the S node of t (non-basis parts with d_t > 0, level-major);
//   node_off      first S row of each node (prefix of d), node_off[nn] = n;
//   q_off_t       offset of Q_t (m_t x m_t) in the Q buffer, levels < l_stop;
//   ap_idx_t      position of t among the level's clusters with m_t > 0 (the
//                 level map items), with the count per level in nap[l] and
//                 the first item of level l in ap_base[l] (levels < l_stop).
// node_of and q_off start at -1 (set by the caller).
__global__ void __launch_bounds__(kScanThreads) k_scan_levels(
    const int32_t *__restrict__ lp, int D, const int *__restrict__ lstop_p, const int64_t *__restrict__ m,
    const int64_t *__restrict__ d, int64_t *__restrict__ xoff, int32_t *__restrict__ node_of,
    int32_t *__restrict__ node_cluster, int32_t *__restrict__ node_level, int64_t *__restrict__ node_off,
    int64_t *__restrict__ q_off, int32_t *__restrict__ ap_idx, int32_t *__restrict__ nap, int32_t *__restrict__ ap_base,
    int32_t *__restrict__ nn_out) {
  const int lstop = *lstop_p;
  int64_t cn = 0, cno = 0, cq = 0;
  int32_t ab = 0;
  for (int l = 0; l <= lstop; ++l) {
    const int b = lp[D - l], e = lp[D - l + 1];
    int64_t cx = 0, ca = 0;
    for (int c0 = b; c0 < e; c0 += kScanThreads) {
      const int t = c0 + int(threadIdx.x);
      const bool ok = t < e;
      const int64_t mt = ok ? m[t] : 0, dt = ok ? d[t] : 0;
      const bool nf = ok && dt > 0, af = ok && mt > 0;
      int64_t tot;
      const int64_t ex = block_scan(mt, &tot);
      const int64_t xo = cx + ex;
      cx += tot;
      const int64_t en = block_scan(nf ? 1 : 0, &tot);
      const int64_t node = cn + en;
      cn += tot;
      const int64_t eno = block_scan(nf ? dt : 0, &tot);
      const int64_t no = cno + eno;
      cno += tot;
      const int64_t eq = block_scan(l < lstop ? mt * mt : 0, &tot);
      const int64_t qo = cq + eq;
      cq += tot;
      const int64_t ea = block_scan(af ? 1 : 0, &tot);
      const int64_t ai = ca + ea;
      ca += tot;
      if (ok) {
        xoff[t] = xo;
        if (nf) {
          node_of[t] = int32_t(node);
          node_cluster[node] = t;
          node_level[node] = l;
          node_off[node] = no;
        }
        if (l < lstop) q_off[t] = qo;
        ap_idx[t] = af ? int32_t(ai) : -1;
      }
    }
    if (threadIdx.x == 0) {
      nap[l] = int32_t(ca);
      ap_base[l] = ab;
    }
    if (l < lstop) ab += int32_t(ca);
  }
  if (threadIdx.x == 0) {
    node_off[cn] = cno;
    *nn_out = int32_t(cn);
  }
}

// The level maps: the apply item of each cluster of a compressed level
// (Q_t, where X_l(t) sits, where its non-basis rows go in S, where its basis
// rows go in X_{l+1}), and the copies of the top clusters into S.
__global__ void k_level_maps(const int32_t *__restrict__ lp, int D, const int *__restrict__ lstop_p, int ncl,
                             const int32_t *__restrict__ parent, const int64_t *__restrict__ begin,
                             const int64_t *__restrict__ m, const int64_t *__restrict__ kp,
                             const int64_t *__restrict__ d, const int64_t *__restrict__ off,
                             const int64_t *__restrict__ xoff, const int32_t *__restrict__ node_of,
                             const int64_t *__restrict__ node_off, const int64_t *__restrict__ q_off,
                             const int32_t *__restrict__ ap_idx, const int32_t *__restrict__ ap_base,
                             ApItem *__restrict__ ap, int64_t *__restrict__ top_src, int64_t *__restrict__ top_dst,
                             int32_t *__restrict__ top_len) {
  const int t = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (t >= ncl) return;
  const int lstop = *lstop_p;
  const int l = D - depth_of(lp, D, t);
  if (l > lstop || ap_idx[t] < 0) return;
  if (l < lstop) {
    ApItem a;
    a.q = q_off[t];
    a.m = int32_t(m[t]);
    a.kp = int32_t(kp[t]);
    a.xin = xoff[t];
    a.yout = d[t] > 0 ? node_off[node_of[t]] : -1;
    a.xout = kp[t] > 0 ? xoff[parent[t]] + off[t] : -1;
    ap[ap_base[l] + ap_idx[t]] = a;
  } else {
    const int i = ap_idx[t];
    top_src[i] = lstop == 0 ? begin[t] : xoff[t];
    top_dst[i] = node_off[node_of[t]];
    top_len[i] = int32_t(m[t]);
  }
}

// Near_{l+1}, row of parent P (one CTA per P at level l + 1): the parents of
// the columns of its children's rows of Near_l and Far_l, sorted and without
// repeats.  The candidates are marked in a bitmap over [lo, hi] (their
// range), one chunk of kBitWords words at a time; count mode writes the row
// length, fill mode the sorted columns (each thread owns a run of words and
// writes its set bits in order after a scan of the counts).
constexpr int kNearThreads = 256;
constexpr int kBitWords = 4096;  // 16 KB: 131,072 columns per chunk

__global__ void __launch_bounds__(kNearThreads) k_near_next(
    const int32_t *__restrict__ cstart, const int32_t *__restrict__ ccnt, const int32_t *__restrict__ parent,
    int plo, int near_row0, const int64_t *__restrict__ near_ptr, const int32_t *__restrict__ near_col,
    const int64_t *__restrict__ far_ptr, const int32_t *__restrict__ far_col, int64_t *__restrict__ cnt,
    const int64_t *__restrict__ out_ptr, int32_t *__restrict__ out_col) {
  const int P = plo + int(blockIdx.x);
  __shared__ uint32_t bits[kBitWords];
  __shared__ int s_lo, s_hi;
  __shared__ int64_t s_scan[kNearThreads];
  const int tid = threadIdx.x;
  if (tid == 0) s_lo = INT32_MAX, s_hi = -1;
  __syncthreads();
  const int c0 = cstart[P], nc = ccnt[P];
  // every candidate column (a parent), visited by `visit`
  auto for_each = [&](auto &&visit) {
    for (int c = c0; c < c0 + nc; ++c) {
      const int64_t r = int64_t(c) - near_row0;
      for (int64_t i = near_ptr[r] + tid; i < near_ptr[r + 1]; i += kNearThreads) visit(parent[near_col[i]]);
      for (int64_t i = far_ptr[c] + tid; i < far_ptr[c + 1]; i += kNearThreads) visit(parent[far_col[i]]);
    }
  };
  {
    int lo = INT32_MAX, hi = -1;
    for_each([&](int q) {
      lo = min(lo, q);
      hi = max(hi, q);
    });
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
  }
  __syncthreads();
  const int lo = s_lo, hi = s_hi;
  const bool fill = out_col != nullptr;
  int64_t pos = fill ? out_ptr[P - plo] : 0, total = 0;
  for (int64_t base = lo; base <= hi; base += int64_t(kBitWords) * 32) {
    const int nw = int(min(int64_t(kBitWords), (int64_t(hi) - base) / 32 + 1));
    for (int w = tid; w < nw; w += kNearThreads) bits[w] = 0u;
    __syncthreads();
    for_each([&](int q) {
      const int64_t x = q - base;
      if (x >= 0 && x < int64_t(nw) * 32) atomicOr(&bits[x >> 5], 1u << (x & 31));
    });
    __syncthreads();
    // thread tid owns words [w0, w1)
    const int per = (nw + kNearThreads - 1) / kNearThreads;
    const int w0 = min(nw, tid * per), w1 = min(nw, w0 + per);
    int64_t mine = 0;
    for (int w = w0; w < w1; ++w) mine += __popc(bits[w]);
    s_scan[tid] = mine;
    __syncthreads();
    // inclusive scan over the CTA (Hillis-Steele on shared memory)
    for (int o = 1; o < kNearThreads; o <<= 1) {
      const int64_t y = tid >= o ? s_scan[tid - o] : 0;
      __syncthreads();
      s_scan[tid] += y;
      __syncthreads();
    }
    const int64_t chunk_total = s_scan[kNearThreads - 1];
    if (fill) {
      int64_t at = pos + s_scan[tid] - mine;
      for (int w = w0; w < w1; ++w) {
        uint32_t b = bits[w];
        while (b) {
          const int bit = __ffs(b) - 1;
          b &= b - 1u;
          out_col[at++] = int32_t(base + int64_t(w) * 32 + bit);
        }
      }
    }
    pos += chunk_total;
    total += chunk_total;
    __syncthreads();  // bits and s_scan are reused by the next chunk
  }
  if (!fill && tid == 0) cnt[P - plo] = total;
}

// exclusive scan of n counts into ptr[0..n] (one CTA)
__global__ void __launch_bounds__(kScanThreads) k_scan_counts(const int64_t *__restrict__ cnt, int n,
                                                              int64_t *__restrict__ ptr) {
  int64_t carry = 0;
  for (int c0 = 0; c0 < n; c0 += kScanThreads) {
    const int i = c0 + int(threadIdx.x);
    int64_t tot;
    const int64_t ex = block_scan(i < n ? cnt[i] : 0, &tot);
    if (i < n) ptr[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) ptr[n] = carry;
}

struct Scratch {
  std::vector<void *> bufs;
  cudaError_t err = cudaSuccess;
  template <class T>
  T *get(size_t n) {
    void *p = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (err != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return static_cast<T *>(p);
  }
  template <class T>
  T *put(const std::vector<T> &v) {
    T *p = get<T>(v.size());
    if (p && !v.empty() && err == cudaSuccess) err = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return p;
  }
  void release() {
    for (void *p : bufs) cudaFree(p);
    bufs.clear();
  }
};

template <class T>
cudaError_t fetch(std::vector<T> &dst, const T *src, size_t n) {
  dst.resize(n);
  return n ? cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost) : cudaSuccess;
}

inline unsigned blocks_for(int64_t n, int per) { return unsigned(std::max<int64_t>(1, (n + per - 1) / per)); }

}  // namespace

int device_schedule(const Plan &p, A1Result *out, DeviceMaps *maps, std::string &err) {
  const int D = p.D, ncl = p.ncl, nleaf = p.nleaf;
  const int64_t nfar = p.far_ptr[ncl], nnear = p.near_ptr[nleaf];
  Scratch s;   // freed at the end
  Scratch kept;  // handed to `maps`
  auto fail = [&](cudaError_t e, const char *what) {
    err = std::string("device level schedule: ") + what + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    s.release();
    kept.release();
    return e == cudaErrorMemoryAllocation ? int(H2SP_ENOMEM) : int(H2SP_ECUDA);
  };
  const int32_t *lp = s.put(p.level_ptr);
  const int32_t *parent = s.put(p.parent);
  const int32_t *rank = s.put(p.rank);
  const int64_t *size = s.put(p.h_size);
  const int64_t *begin = s.put(p.h_begin);
  const int64_t *far_ptr = s.put(p.far_ptr);
  const int32_t *far_col = s.put(p.far_col);
  const int64_t *near_ptr0 = s.put(p.near_ptr);
  const int32_t *near_col0 = s.put(p.near_col);
  int32_t *cstart = s.get<int32_t>(ncl), *ccnt = s.get<int32_t>(ncl);
  int *lstop_d = s.get<int>(1);
  int64_t *m = s.get<int64_t>(ncl), *kp = s.get<int64_t>(ncl), *d = s.get<int64_t>(ncl), *off = s.get<int64_t>(ncl),
          *xoff = s.get<int64_t>(ncl), *q_off = s.get<int64_t>(ncl);
  int32_t *node_of = s.get<int32_t>(ncl), *node_cluster = s.get<int32_t>(ncl), *node_level = s.get<int32_t>(ncl);
  int64_t *node_off = kept.get<int64_t>(size_t(ncl) + 1);
  int32_t *ap_idx = s.get<int32_t>(ncl), *nap_d = s.get<int32_t>(D + 2), *ap_base_d = s.get<int32_t>(D + 2),
          *nn_d = s.get<int32_t>(1);
  ApItem *ap = kept.get<ApItem>(ncl);
  int64_t *top_src = kept.get<int64_t>(ncl), *top_dst = kept.get<int64_t>(ncl);
  int32_t *top_len = kept.get<int32_t>(ncl);
  if (s.err != cudaSuccess) return fail(s.err, "allocation");
  if (kept.err != cudaSuccess) return fail(kept.err, "allocation");
  cudaError_t e;
  if ((e = cudaMemset(ccnt, 0, sizeof(int32_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(cstart, 0xFF, sizeof(int32_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(lstop_d, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(m, 0, sizeof(int64_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(kp, 0, sizeof(int64_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(d, 0, sizeof(int64_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(off, 0, sizeof(int64_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(xoff, 0, sizeof(int64_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(q_off, 0xFF, sizeof(int64_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(node_of, 0xFF, sizeof(int32_t) * ncl)) != cudaSuccess ||
      (e = cudaMemset(ap_idx, 0xFF, sizeof(int32_t) * ncl)) != cudaSuccess)
    return fail(e, "memset");
  const int first = p.level_ptr[1];
  if (ncl > first) k_children<<<blocks_for(ncl - first, 256), 256>>>(parent, first, ncl, cstart, ccnt);
  k_lstop<<<blocks_for(ncl, 256), 256>>>(lp, D, far_ptr, ncl, lstop_d);
  int lstop = 0;
  if ((e = cudaMemcpy(&lstop, lstop_d, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e, "l_stop");
  auto lev_begin = [&](int l) { return p.level_ptr[D - l]; };
  auto lev_end = [&](int l) { return p.level_ptr[D - l + 1]; };
  k_leaf_sizes<<<blocks_for(nleaf, 256), 256>>>(size, lev_begin(0), lev_end(0), m);
  for (int l = 0; l < lstop; ++l)
    k_level_sizes<<<blocks_for(lev_end(l + 1) - lev_begin(l + 1), 128), 128>>>(cstart, ccnt, rank, lev_begin(l + 1),
                                                                              lev_end(l + 1), m, kp, d, off);
  k_top_sizes<<<blocks_for(lev_end(lstop) - lev_begin(lstop), 256), 256>>>(lev_begin(lstop), lev_end(lstop), m, kp, d);
  k_scan_levels<<<1, kScanThreads>>>(lp, D, lstop_d, m, d, xoff, node_of, node_cluster, node_level, node_off, q_off,
                                     ap_idx, nap_d, ap_base_d, nn_d);
  k_level_maps<<<blocks_for(ncl, 256), 256>>>(lp, D, lstop_d, ncl, parent, begin, m, kp, d, off, xoff, node_of,
                                               node_off, q_off, ap_idx, ap_base_d, ap, top_src, top_dst, top_len);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "launch");
  // Near_{l+1} for l = 0 .. l_stop - 1 (rows: the clusters of level l + 1)
  A1Result r;
  r.lstop = lstop;
  r.near_ptr.assign(lstop + 1, {});
  r.near_col.assign(lstop + 1, {});
  const int64_t *nptr = near_ptr0;
  const int32_t *ncol = near_col0;
  int row0 = lev_begin(0);
  (void)nnear;
  (void)nfar;
  for (int l = 0; l < lstop; ++l) {
    const int plo = lev_begin(l + 1), np = lev_end(l + 1) - plo;
    int64_t *cnt = s.get<int64_t>(np), *ptr = s.get<int64_t>(size_t(np) + 1);
    if (s.err != cudaSuccess) return fail(s.err, "allocation");
    k_near_next<<<unsigned(np), kNearThreads>>>(cstart, ccnt, parent, plo, row0, nptr, ncol, far_ptr, far_col, cnt,
                                                nullptr, nullptr);
    k_scan_counts<<<1, kScanThreads>>>(cnt, np, ptr);
    int64_t nnz = 0;
    if ((e = cudaMemcpy(&nnz, ptr + np, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return fail(e, "near list size");
    int32_t *col = s.get<int32_t>(size_t(nnz));
    if (s.err != cudaSuccess) return fail(s.err, "allocation");
    k_near_next<<<unsigned(np), kNearThreads>>>(cstart, ccnt, parent, plo, row0, nptr, ncol, far_ptr, far_col, cnt, ptr,
                                                col);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "launch");
    if ((e = fetch(r.near_ptr[l + 1], ptr, size_t(np) + 1)) != cudaSuccess ||
        (e = fetch(r.near_col[l + 1], col, size_t(nnz))) != cudaSuccess)
      return fail(e, "near list copy");
    nptr = ptr;
    ncol = col;
    row0 = plo;
  }
  int32_t nn = 0;
  std::vector<int32_t> nap, ap_base;
  if ((e = cudaMemcpy(&nn, nn_d, sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = fetch(nap, nap_d, size_t(lstop) + 1)) != cudaSuccess ||
      (e = fetch(ap_base, ap_base_d, size_t(lstop) + 1)) != cudaSuccess)
    return fail(e, "counts");
  r.nn = nn;
  if (out) {
    if ((e = fetch(r.m, m, ncl)) != cudaSuccess || (e = fetch(r.kp, kp, ncl)) != cudaSuccess ||
        (e = fetch(r.d, d, ncl)) != cudaSuccess || (e = fetch(r.off, off, ncl)) != cudaSuccess ||
        (e = fetch(r.xoff, xoff, ncl)) != cudaSuccess || (e = fetch(r.q_off, q_off, ncl)) != cudaSuccess ||
        (e = fetch(r.node_of, node_of, ncl)) != cudaSuccess ||
        (e = fetch(r.node_cluster, node_cluster, size_t(nn))) != cudaSuccess ||
        (e = fetch(r.node_level, node_level, size_t(nn))) != cudaSuccess ||
        (e = fetch(r.node_off, node_off, size_t(nn) + 1)) != cudaSuccess)
      return fail(e, "schedule copy");
    *out = std::move(r);
  }
  s.release();
  if (maps) {
    maps->allocs = kept.bufs;
    maps->ap = ap;
    maps->ap_base.assign(ap_base.begin(), ap_base.begin() + lstop);
    maps->nap.assign(nap.begin(), nap.begin() + lstop);
    maps->top_src = top_src;
    maps->top_dst = top_dst;
    maps->top_len = top_len;
    maps->ntop = nap[lstop];
    maps->node_off = node_off;
  } else {
    kept.release();
  }
  return H2SP_OK;
}

}  // namespace h2sp
