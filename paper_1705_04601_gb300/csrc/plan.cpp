// Host planning for h2sp: validation of the H^2 descriptor, the integer
// schedule of the level recursion (§2.2-2.3: basis / non-basis split, big
// blocks, close lists per level, cross-level panels), the block pattern of S
// (§3), the flat work items of the sparsification kernels, and the symbolic
// block LU of S (nested-dissection order along the cluster tree, supernodes,
// fronts).  No floating-point work happens here.
#include <algorithm>
#include <array>
#include <chrono>
#include <cstring>
#include <limits>
#include <utility>

#include "internal.h"

namespace h2sp {
namespace {

using u64 = uint64_t;
inline u64 key(int64_t a, int64_t b) { return (u64(uint32_t(a)) << 32) | u64(uint32_t(b)); }
inline int32_t kfirst(u64 k) { return int32_t(k >> 32); }
inline int32_t ksecond(u64 k) { return int32_t(k & 0xffffffffu); }

// Sorts (row << 32 | col) keys and drops repeats.  Large lists go through a
// counting sort on the row followed by a sort of each row's short column list,
// which is linear in the number of keys up to the per-row sorts.
void sort_unique(std::vector<u64> &v) {
  if (v.size() < 4096) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return;
  }
  uint32_t rmax = 0;
  for (u64 k : v) rmax = std::max(rmax, uint32_t(k >> 32));
  if (size_t(rmax) > 4 * v.size()) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return;
  }
  std::vector<int64_t> ptr(size_t(rmax) + 2, 0);
  for (u64 k : v) ptr[size_t(k >> 32) + 1]++;
  for (size_t r = 0; r + 1 < ptr.size(); ++r) ptr[r + 1] += ptr[r];
  std::vector<u64> tmp(v.size());
  {
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (u64 k : v) tmp[size_t(fill[size_t(k >> 32)]++)] = k;
  }
  size_t out = 0;
  for (size_t r = 0; r + 1 < ptr.size(); ++r) {
    auto b = tmp.begin() + ptr[r], e = tmp.begin() + ptr[r + 1];
    std::sort(b, e);
    for (auto it = b; it != e; ++it)
      if (out == 0 || v[out - 1] != *it) v[out++] = *it;
  }
  v.resize(out);
}

// index of k in a sorted vector, -1 if absent
int64_t find_sorted(const std::vector<u64> &v, u64 k) {
  auto it = std::lower_bound(v.begin(), v.end(), k);
  if (it == v.end() || *it != k) return -1;
  return int64_t(it - v.begin());
}

// Row index over a sorted vector of (row << 32 | col) keys: the keys of one
// row are [ptr[row], ptr[row + 1]), so a lookup searches a single row.
struct RowIndex {
  const std::vector<u64> *keys = nullptr;
  std::vector<int64_t> ptr;
  void build(const std::vector<u64> &k, int nrows) {
    keys = &k;
    ptr.assign(size_t(nrows) + 1, 0);
    for (u64 x : k) ptr[size_t(kfirst(x)) + 1]++;
    for (int r = 0; r < nrows; ++r) ptr[r + 1] += ptr[r];
  }
  int64_t find(int row, int col) const {
    if (row < 0 || size_t(row) + 1 >= ptr.size()) return -1;
    const u64 k = key(row, col);
    auto b = keys->begin() + ptr[row], e = keys->begin() + ptr[row + 1];
    auto it = std::lower_bound(b, e, k);
    return (it != e && *it == k) ? int64_t(it - keys->begin()) : -1;
  }
};

struct Fail {
  int code;
  std::string msg;
};

#define REQUIRE(cond, msg)                  \
  do {                                      \
    if (!(cond)) throw Fail{H2SP_EINVAL, msg}; \
  } while (0)

}  // namespace

int build_plan(const h2sp_h2_desc *d, Plan &p, std::string &err, bool need_numbers, const A1Source *a1) {
  try {
    REQUIRE(d != nullptr, "null descriptor");
    REQUIRE(d->n > 0 && d->n < (int64_t(1) << 31), "n out of range");
    REQUIRE(d->depth >= 0 && d->depth < 60, "depth out of range");
    REQUIRE(d->level_ptr && d->parent && d->begin && d->size && d->rank && d->far_ptr && d->near_ptr,
            "missing structure array");
    REQUIRE(d->leaf_basis_off && d->transfer_off && d->coupling_off && d->near_off, "missing offset array");
    if (need_numbers) {
      REQUIRE(d->leaf_basis && d->transfer && d->coupling && d->near_block, "missing numeric array");
      REQUIRE((d->col_leaf_basis == nullptr) == (d->col_transfer == nullptr), "column basis arrays must come together");
    }
    const bool sym = need_numbers ? d->col_leaf_basis == nullptr : d->col_leaf_basis_off == nullptr;
    REQUIRE(sym || (d->col_leaf_basis_off && d->col_transfer_off), "missing column offset arrays");
    const int D = d->depth;
    const int32_t *lp = d->level_ptr;
    REQUIRE(lp[0] == 0 && lp[1] >= 1, "depth 0 must hold the root(s)");
    for (int dd = 1; dd <= D; ++dd) REQUIRE(lp[dd + 1] > lp[dd], "empty depth");
    const int ncl = lp[D + 1];
    const int nleaf = lp[D + 1] - lp[D];
    p.n = d->n;
    p.D = D;
    p.ncl = ncl;
    p.nleaf = nleaf;
    p.sym = sym;
    p.level_ptr.assign(lp, lp + D + 2);
    p.parent.assign(d->parent, d->parent + ncl);
    p.rank.assign(d->rank, d->rank + ncl);
    p.h_begin.assign(d->begin, d->begin + ncl);
    p.h_size.assign(d->size, d->size + ncl);
    std::vector<int32_t> dep(ncl);
    for (int dd = 0; dd <= D; ++dd)
      for (int t = lp[dd]; t < lp[dd + 1]; ++t) dep[t] = dd;
    for (int c = 0; c < lp[1]; ++c) REQUIRE(p.parent[c] == -1, "root parent must be -1");
    std::vector<int32_t> nkids(ncl, 0);
    for (int c = lp[1]; c < ncl; ++c) {
      int pa = p.parent[c];
      REQUIRE(pa >= 0 && pa < ncl && dep[pa] == dep[c] - 1, "parent not one depth up");
      if (c > lp[dep[c]]) REQUIRE(pa >= p.parent[c - 1], "children of a cluster must be consecutive");
      nkids[pa]++;
    }
    for (int t = 0; t < lp[D]; ++t) REQUIRE(nkids[t] > 0, "non-leaf cluster without children");
    for (int t = 0; t < ncl; ++t) REQUIRE(p.rank[t] >= 0, "negative rank");
    // point ranges: leaves contiguous from 0, parents cover their children
    int64_t acc = 0;
    for (int t = lp[D]; t < lp[D + 1]; ++t) {
      REQUIRE(p.h_size[t] >= 0 && p.h_begin[t] == acc, "leaf ranges must be contiguous in tree order");
      acc += p.h_size[t];
    }
    REQUIRE(acc == d->n, "leaf sizes must add up to n");
    {
      std::vector<int64_t> sz(ncl, 0), bg(ncl, -1);
      for (int t = lp[D]; t < lp[D + 1]; ++t) sz[t] = p.h_size[t], bg[t] = p.h_begin[t];
      for (int c = ncl - 1; c >= lp[1]; --c) {
        int pa = p.parent[c];
        sz[pa] += sz[c];
        bg[pa] = bg[c];  // children visited downwards: ends at the first child
      }
      for (int t = 0; t < lp[D]; ++t)
        REQUIRE(sz[t] == p.h_size[t] && bg[t] == p.h_begin[t], "cluster range differs from its children");
    }
    // root of every cluster: depth 0 may hold several roots (independent systems)
    p.root.assign(ncl, 0);
    for (int c = 0; c < ncl; ++c) p.root[c] = c < lp[1] ? c : p.root[p.parent[c]];
    // lists
    p.far_ptr.assign(d->far_ptr, d->far_ptr + ncl + 1);
    const int64_t nfar = p.far_ptr[ncl];
    REQUIRE(p.far_ptr[0] == 0 && nfar >= 0, "bad far_ptr");
    if (nfar) REQUIRE(d->far_col != nullptr, "missing far_col");
    p.far_col.assign(d->far_col, d->far_col + nfar);
    for (int t = 0; t < ncl; ++t) {
      REQUIRE(p.far_ptr[t + 1] >= p.far_ptr[t], "far_ptr not monotone");
      for (int64_t i = p.far_ptr[t]; i < p.far_ptr[t + 1]; ++i) {
        int s = p.far_col[i];
        REQUIRE(s >= 0 && s < ncl && dep[s] == dep[t], "far pair across depths");
        if (i > p.far_ptr[t]) REQUIRE(s > p.far_col[i - 1], "far_col not ascending");
        REQUIRE(dep[t] > 0, "a root cannot be admissible");
        REQUIRE(p.root[s] == p.root[t], "admissible pair across independent systems");
      }
    }
    p.near_ptr.assign(d->near_ptr, d->near_ptr + nleaf + 1);
    const int64_t nnear = p.near_ptr[nleaf];
    REQUIRE(p.near_ptr[0] == 0 && nnear > 0 && d->near_col != nullptr, "bad near_ptr");
    p.near_col.assign(d->near_col, d->near_col + nnear);
    for (int lf = 0; lf < nleaf; ++lf) {
      REQUIRE(p.near_ptr[lf + 1] >= p.near_ptr[lf], "near_ptr not monotone");
      for (int64_t i = p.near_ptr[lf]; i < p.near_ptr[lf + 1]; ++i) {
        int s = p.near_col[i];
        REQUIRE(s >= lp[D] && s < lp[D + 1], "close pair with a non-leaf");
        if (i > p.near_ptr[lf]) REQUIRE(s > p.near_col[i - 1], "near_col not ascending");
        REQUIRE(p.root[s] == p.root[lp[D] + lf], "close pair across independent systems");
      }
    }
    p.leaf_basis_off.assign(d->leaf_basis_off, d->leaf_basis_off + nleaf);
    p.transfer_off.assign(d->transfer_off, d->transfer_off + ncl);
    p.coupling_off.assign(d->coupling_off, d->coupling_off + nfar);
    p.near_off.assign(d->near_off, d->near_off + nnear);
    if (!sym) {
      p.col_leaf_basis_off.assign(d->col_leaf_basis_off, d->col_leaf_basis_off + nleaf);
      p.col_transfer_off.assign(d->col_transfer_off, d->col_transfer_off + ncl);
    }
    for (int t = 0; t < ncl; ++t)
      if (p.rank[t] > kMaxRank) throw Fail{H2SP_EUNSUPPORTED, "cluster rank above 64"};

    // ---------------- level schedule (a1) ----------------
    p.level.resize(ncl);
    for (int t = 0; t < ncl; ++t) p.level[t] = D - dep[t];
    auto lev_begin = [&](int l) { return lp[D - l]; };
    auto lev_end = [&](int l) { return lp[D - l + 1]; };
    std::vector<std::vector<std::array<int64_t, 3>>> far(D + 1);
    for (int t = 0; t < ncl; ++t)
      for (int64_t i = p.far_ptr[t]; i < p.far_ptr[t + 1]; ++i) far[p.level[t]].push_back({t, p.far_col[i], i});
    int lstop = 0;
    for (int l = 0; l <= D; ++l)
      if (!far[l].empty()) lstop = l + 1;
    A1Result dev;
    if (a1) {
      const int st = (*a1)(p, dev, err);
      if (st != H2SP_OK) throw Fail{st, err};
      if (dev.lstop != lstop || int64_t(dev.m.size()) != ncl || int64_t(dev.near_ptr.size()) != lstop + 1)
        throw Fail{H2SP_EINVAL, "internal: device level schedule of another shape"};
    }
    p.lstop = lstop;
    std::vector<std::vector<u64>> near(lstop + 1);
    for (int lf = 0; lf < nleaf; ++lf)
      for (int64_t i = p.near_ptr[lf]; i < p.near_ptr[lf + 1]; ++i) near[0].push_back(key(lp[D] + lf, p.near_col[i]));
    // near[0] is sorted by construction (rows ascending, columns ascending)
    if (a1) {
      // the device's Near_l: CSR over the level's clusters, rows and columns ascending
      for (int l = 1; l <= lstop; ++l) {
        const auto &ptr = dev.near_ptr[l];
        const auto &col = dev.near_col[l];
        near[l].reserve(col.size());
        for (int r = 0; r + 1 < int(ptr.size()); ++r)
          for (int64_t i = ptr[r]; i < ptr[r + 1]; ++i) near[l].push_back(key(lev_begin(l) + r, col[i]));
      }
      p.m = std::move(dev.m);
      p.kp = std::move(dev.kp);
      p.d = std::move(dev.d);
      p.off = std::move(dev.off);
      p.xoff = std::move(dev.xoff);
    } else {
      for (int l = 0; l < lstop; ++l) {
        auto &nx = near[l + 1];
        nx.reserve(near[l].size() / 2 + far[l].size() / 4 + 1);
        for (u64 k : near[l]) nx.push_back(key(p.parent[kfirst(k)], p.parent[ksecond(k)]));
        for (auto &f : far[l]) nx.push_back(key(p.parent[f[0]], p.parent[f[1]]));
        sort_unique(nx);
      }
      // local sizes
      p.m.assign(ncl, 0);
      p.kp.assign(ncl, 0);
      p.d.assign(ncl, 0);
      p.off.assign(ncl, 0);
      p.xoff.assign(ncl, 0);
      for (int t = lev_begin(0); t < lev_end(0); ++t) p.m[t] = p.h_size[t];
      for (int l = 0; l <= lstop; ++l) {
        int64_t a = 0;
        for (int t = lev_begin(l); t < lev_end(l); ++t) {
          p.xoff[t] = a;
          a += p.m[t];
          if (l < lstop) {
            p.kp[t] = std::min<int64_t>(p.rank[t], p.m[t]);
            p.d[t] = p.m[t] - p.kp[t];
          } else {
            p.kp[t] = 0;
            p.d[t] = p.m[t];
          }
        }
        if (l < lstop)
          for (int t = lev_begin(l); t < lev_end(l); ++t) {
            int pa = p.parent[t];
            p.off[t] = p.m[pa];
            p.m[pa] += p.kp[t];
          }
      }
    }
    for (int l = 0; l < std::max(lstop, 1); ++l)
      for (int t = lev_begin(l); t < lev_end(l); ++t)
        if (p.m[t] > kMaxLargeBlock) throw Fail{H2SP_EUNSUPPORTED, "local block above 384 rows (leaf or level size)"};
    // S nodes: non-basis parts level by level, then the top clusters
    if (a1) {
      p.node_of = std::move(dev.node_of);
      p.node_level = std::move(dev.node_level);
      p.node_cluster = std::move(dev.node_cluster);
      p.node_off = std::move(dev.node_off);
      p.node_size.resize(p.node_cluster.size());
      for (size_t v = 0; v < p.node_cluster.size(); ++v) p.node_size[v] = p.d[p.node_cluster[v]];
    } else {
      p.node_of.assign(ncl, -1);
      for (int l = 0; l <= lstop; ++l)
        for (int t = lev_begin(l); t < lev_end(l); ++t)
          if (p.d[t] > 0) {
            p.node_of[t] = int32_t(p.node_size.size());
            p.node_level.push_back(l);
            p.node_cluster.push_back(t);
            p.node_size.push_back(p.d[t]);
          }
      const int nn0 = int(p.node_size.size());
      p.node_off.assign(nn0 + 1, 0);
      for (int v = 0; v < nn0; ++v) p.node_off[v + 1] = p.node_off[v] + p.node_size[v];
    }
    const int nn = int(p.node_size.size());
    REQUIRE(int64_t(p.node_off.size()) == nn + 1 && p.node_off[nn] == p.n, "internal: S nodes do not cover n");
    // Q / Rr storage for the compressed levels
    p.q_off.assign(ncl, -1);
    p.rr_off.assign(ncl, -1);
    for (int l = 0; l < lstop; ++l)
      for (int t = lev_begin(l); t < lev_end(l); ++t) {
        p.q_off[t] = p.q_elems;
        p.q_elems += p.m[t] * p.m[t];
        p.rr_off[t] = p.rr_elems;
        p.rr_elems += p.kp[t] * p.rank[t];
      }

    // ---------------- cross-level panels (a5) ----------------
    std::vector<std::vector<u64>> RP(lstop + 1), CP(lstop + 1);
    for (int l = 0; l < lstop; ++l) {
      auto &rn = RP[l + 1];
      auto &cn = CP[l + 1];
      for (u64 k : near[l]) {
        int a = kfirst(k), b = ksecond(k);
        if (p.d[a] > 0) rn.push_back(key(p.node_of[a], p.parent[b]));
        if (p.d[b] > 0) cn.push_back(key(p.parent[a], p.node_of[b]));
      }
      for (u64 k : RP[l]) rn.push_back(key(kfirst(k), p.parent[ksecond(k)]));
      for (u64 k : CP[l]) cn.push_back(key(p.parent[kfirst(k)], ksecond(k)));
      sort_unique(rn);
      sort_unique(cn);
    }

    // ---------------- block pattern of S (a6) ----------------
    std::vector<u64> sb;
    for (int l = 0; l < lstop; ++l) {
      for (u64 k : near[l]) {
        int a = kfirst(k), b = ksecond(k);
        if (p.d[a] > 0 && p.d[b] > 0) sb.push_back(key(p.node_of[a], p.node_of[b]));
      }
      if (l >= 1) {
        for (u64 k : RP[l])
          if (p.d[ksecond(k)] > 0) sb.push_back(key(kfirst(k), p.node_of[ksecond(k)]));
        for (u64 k : CP[l])
          if (p.d[kfirst(k)] > 0) sb.push_back(key(p.node_of[kfirst(k)], ksecond(k)));
      }
    }
    for (u64 k : near[lstop]) {
      int a = kfirst(k), b = ksecond(k);
      if (p.m[a] > 0 && p.m[b] > 0) sb.push_back(key(p.node_of[a], p.node_of[b]));
    }
    if (lstop >= 1) {
      for (u64 k : RP[lstop])
        if (p.node_of[ksecond(k)] >= 0) sb.push_back(key(kfirst(k), p.node_of[ksecond(k)]));
      for (u64 k : CP[lstop])
        if (p.node_of[kfirst(k)] >= 0) sb.push_back(key(p.node_of[kfirst(k)], ksecond(k)));
    }
    {
      size_t before = sb.size();
      sort_unique(sb);
      REQUIRE(before == sb.size(), "internal: duplicate S block");
    }
    const int64_t nnzb = int64_t(sb.size());
    p.brow_ptr.assign(nn + 1, 0);
    p.bcol.resize(nnzb);
    p.val_off.resize(nnzb);
    for (int64_t z = 0; z < nnzb; ++z) {
      int i = kfirst(sb[z]), j = ksecond(sb[z]);
      p.brow_ptr[i + 1]++;
      p.bcol[z] = j;
      p.val_off[z] = p.s_elems;
      p.s_elems += p.node_size[i] * p.node_size[j];
    }
    for (int v = 0; v < nn; ++v) p.brow_ptr[v + 1] += p.brow_ptr[v];
    RowIndex sb_idx;
    sb_idx.build(sb, nn);
    auto sblock = [&](int i, int j) -> int64_t {
      int64_t z = sb_idx.find(i, j);
      if (z < 0) throw Fail{H2SP_EINVAL, "internal: missing S block"};
      return p.val_off[z];
    };

    // ---------------- level buffers ----------------
    p.c_elems.assign(lstop + 1, 0);
    p.rp_elems.assign(lstop + 1, 0);
    p.cp_elems.assign(lstop + 1, 0);
    std::vector<std::vector<int64_t>> c_off(lstop + 1), rp_off(lstop + 1), cp_off(lstop + 1);
    for (int l = 1; l < lstop; ++l) {
      for (u64 k : near[l]) {
        c_off[l].push_back(p.c_elems[l]);
        p.c_elems[l] += p.m[kfirst(k)] * p.m[ksecond(k)];
      }
      for (u64 k : RP[l]) {
        rp_off[l].push_back(p.rp_elems[l]);
        p.rp_elems[l] += p.node_size[kfirst(k)] * p.m[ksecond(k)];
      }
      for (u64 k : CP[l]) {
        cp_off[l].push_back(p.cp_elems[l]);
        p.cp_elems[l] += p.m[kfirst(k)] * p.node_size[ksecond(k)];
      }
    }
    // row indexes of the next-level close blocks and panels
    std::vector<RowIndex> near_idx(lstop + 1), rp_idx(lstop + 1), cp_idx(lstop + 1);
    for (int l = 1; l < lstop; ++l) {
      near_idx[l].build(near[l], ncl);
      rp_idx[l].build(RP[l], nn);
      cp_idx[l].build(CP[l], ncl);
    }
    // destinations at level l+1 (a next-level buffer, or S itself at l_stop)
    struct Dst {
      int64_t off;
      int8_t buf;
    };
    auto dst_C = [&](int l1, int pa, int qa) -> Dst {
      if (l1 < lstop) {
        int64_t z = near_idx[l1].find(pa, qa);
        if (z < 0) throw Fail{H2SP_EINVAL, "internal: missing next-level close block"};
        return {c_off[l1][z], DST_C};
      }
      return {sblock(p.node_of[pa], p.node_of[qa]), DST_S};
    };
    auto dst_RP = [&](int l1, int v, int qa) -> Dst {
      if (l1 < lstop) {
        int64_t z = rp_idx[l1].find(v, qa);
        if (z < 0) throw Fail{H2SP_EINVAL, "internal: missing row panel"};
        return {rp_off[l1][z], DST_RP};
      }
      return {sblock(v, p.node_of[qa]), DST_S};
    };
    auto dst_CP = [&](int l1, int pa, int w) -> Dst {
      if (l1 < lstop) {
        int64_t z = cp_idx[l1].find(pa, w);
        if (z < 0) throw Fail{H2SP_EINVAL, "internal: missing column panel"};
        return {cp_off[l1][z], DST_CP};
      }
      return {sblock(p.node_of[pa], w), DST_S};
    };

    // ---------------- work items (a2-a5) ----------------
    const int nlw = std::max(lstop, 1);
    p.lw.assign(nlw, LevelWork());
    double flops = 0.0;
    std::vector<int64_t> near_index;  // position of each Near_0 pair in the input arrays
    near_index.resize(near[0].size());
    for (int64_t i = 0; i < int64_t(near[0].size()); ++i) near_index[i] = i;  // same order as the CSR
    if (lstop == 0) {
      auto &x = p.lw[0].x;
      for (int64_t z = 0; z < int64_t(near[0].size()); ++z) {
        int a = kfirst(near[0][z]), b = ksecond(near[0][z]);
        if (p.m[a] == 0 || p.m[b] == 0) continue;
        XItem it{};
        it.src = p.near_off[near_index[z]];
        it.src_buf = SRC_NEAR;
        it.ld_src = int32_t(p.m[a]);
        it.rows = int32_t(p.m[a]);
        it.cols = int32_t(p.m[b]);
        it.qL = it.qR = -1;
        it.kr = it.kc = 0;
        for (int q = 0; q < 3; ++q) it.dst[q] = -1;
        it.dst[3] = sblock(p.node_of[a], p.node_of[b]);
        it.dst_buf[3] = DST_S;
        it.ld[3] = int32_t(p.m[a]);
        x.push_back(it);
      }
    }
    for (int l = 0; l < lstop; ++l) {
      LevelWork &w = p.lw[l];
      w.x.reserve(near[l].size() + (l >= 1 ? RP[l].size() + CP[l].size() : 0));
      w.c.reserve(far[l].size());
      w.q.reserve(size_t(lev_end(l) - lev_begin(l)));
      if (!sym) w.qc.reserve(size_t(lev_end(l) - lev_begin(l)));
      // W for this level from the previous level's Rr (internal clusters)
      std::vector<int64_t> w_off(ncl, -1);
      if (l >= 1) {
        for (int t = lev_begin(l); t < lev_end(l); ++t) {
          w_off[t] = w.w_elems;
          w.w_elems += p.m[t] * p.rank[t];
        }
        for (int c = lev_begin(l - 1); c < lev_end(l - 1); ++c) {
          int pa = p.parent[c];
          if (p.kp[c] == 0 || p.rank[pa] == 0) continue;
          WItem wi{};
          wi.rr_c = p.rr_off[c];
          wi.t_c = p.transfer_off[c];
          wi.w_dst = w_off[pa] + p.off[c];
          wi.kp_c = int32_t(p.kp[c]);
          wi.k_c = p.rank[c];
          wi.k_p = p.rank[pa];
          wi.ld_w = int32_t(p.m[pa]);
          w.w.push_back(wi);
          if (!sym) {
            wi.t_c = p.col_transfer_off[c];
            w.wc.push_back(wi);
          }
          flops += 2.0 * wi.kp_c * wi.k_c * wi.k_p * (sym ? 1 : 2);
        }
        w.wc_elems = sym ? 0 : w.w_elems;
      }
      // Householder completions (a2)
      for (int t = lev_begin(l); t < lev_end(l); ++t) {
        if (p.m[t] == 0) continue;
        QItem qi{};
        qi.m = int32_t(p.m[t]);
        qi.k = p.rank[t];
        qi.q = p.q_off[t];
        qi.rr = p.rr_off[t];
        if (l == 0) {
          qi.w = p.leaf_basis_off[t - lp[D]];
          qi.w_buf = 0;
        } else {
          qi.w = w_off[t];
          qi.w_buf = 1;
        }
        qi.ld_w = qi.m;
        w.q.push_back(qi);
        if (!sym) {
          if (l == 0) qi.w = p.col_leaf_basis_off[t - lp[D]];
          w.qc.push_back(qi);
        }
        double mm = double(qi.m), kk = double(std::min(qi.m, qi.k));
        double f1 = 2.0 * kk * kk * (mm - kk / 3.0) + 4.0 * mm * mm * kk - 4.0 * mm * kk * kk + (4.0 / 3.0) * kk * kk * kk;
        flops += f1 * (sym ? 1 : 2);
        w.max_m = std::max(w.max_m, qi.m);
        w.max_k = std::max(w.max_k, qi.k);
      }
      // coupling projections F_ml (a3)
      for (auto &f : far[l]) {
        int a = int(f[0]), b = int(f[1]);
        if (p.kp[a] == 0 || p.kp[b] == 0) continue;
        int pa = p.parent[a], pb = p.parent[b];
        Dst ds = dst_C(l + 1, pa, pb);
        CItem ci{};
        ci.rr_p = p.rr_off[a];
        ci.rr_q = p.rr_off[b];
        ci.dcoup = p.coupling_off[f[2]];
        ci.dst = ds.off + p.off[a] + p.off[b] * p.m[pa];
        ci.dst_buf = ds.buf;
        ci.ld = int32_t(p.m[pa]);
        ci.kp_p = int32_t(p.kp[a]);
        ci.k_p = p.rank[a];
        ci.kp_q = int32_t(p.kp[b]);
        ci.k_q = p.rank[b];
        w.c.push_back(ci);
        flops += 2.0 * ci.k_p * ci.k_q * ci.kp_q + 2.0 * ci.kp_p * ci.k_p * ci.kp_q;
      }
      // close blocks (a4)
      for (int64_t z = 0; z < int64_t(near[l].size()); ++z) {
        int a = kfirst(near[l][z]), b = ksecond(near[l][z]);
        if (p.m[a] == 0 || p.m[b] == 0) continue;
        int pa = p.parent[a], pb = p.parent[b];
        XItem it{};
        if (l == 0) {
          it.src = p.near_off[near_index[z]];
          it.src_buf = SRC_NEAR;
        } else {
          it.src = c_off[l][z];
          it.src_buf = SRC_C;
        }
        it.ld_src = int32_t(p.m[a]);
        it.rows = int32_t(p.m[a]);
        it.cols = int32_t(p.m[b]);
        it.qL = p.q_off[a];
        it.qR = p.q_off[b];
        it.qside = sym ? 0 : 2;
        it.kr = int32_t(p.kp[a]);
        it.kc = int32_t(p.kp[b]);
        for (int q = 0; q < 4; ++q) it.dst[q] = -1;
        if (p.kp[a] > 0 && p.kp[b] > 0) {
          Dst ds = dst_C(l + 1, pa, pb);
          it.dst[0] = ds.off + p.off[a] + p.off[b] * p.m[pa];
          it.dst_buf[0] = ds.buf;
          it.ld[0] = int32_t(p.m[pa]);
        }
        if (p.kp[a] > 0 && p.d[b] > 0) {
          Dst ds = dst_CP(l + 1, pa, p.node_of[b]);
          it.dst[1] = ds.off + p.off[a];
          it.dst_buf[1] = ds.buf;
          it.ld[1] = int32_t(p.m[pa]);
        }
        if (p.d[a] > 0 && p.kp[b] > 0) {
          Dst ds = dst_RP(l + 1, p.node_of[a], pb);
          it.dst[2] = ds.off + p.off[b] * p.d[a];
          it.dst_buf[2] = ds.buf;
          it.ld[2] = int32_t(p.d[a]);
        }
        if (p.d[a] > 0 && p.d[b] > 0) {
          it.dst[3] = sblock(p.node_of[a], p.node_of[b]);
          it.dst_buf[3] = DST_S;
          it.ld[3] = int32_t(p.d[a]);
        }
        w.x.push_back(it);
        flops += 2.0 * double(it.rows) * it.cols * (it.rows + it.cols);
      }
      // cross-level panels (a5)
      if (l >= 1) {
        for (int64_t z = 0; z < int64_t(RP[l].size()); ++z) {
          int v = kfirst(RP[l][z]), q = ksecond(RP[l][z]);
          if (p.m[q] == 0) continue;
          XItem it{};
          it.src = rp_off[l][z];
          it.src_buf = SRC_RP;
          it.ld_src = int32_t(p.node_size[v]);
          it.rows = int32_t(p.node_size[v]);
          it.cols = int32_t(p.m[q]);
          it.qL = -1;
          it.qR = p.q_off[q];
          it.qside = sym ? 0 : 2;
          it.kr = 0;
          it.kc = int32_t(p.kp[q]);
          for (int k = 0; k < 4; ++k) it.dst[k] = -1;
          if (p.kp[q] > 0) {
            Dst ds = dst_RP(l + 1, v, p.parent[q]);
            it.dst[2] = ds.off + p.off[q] * p.node_size[v];
            it.dst_buf[2] = ds.buf;
            it.ld[2] = it.rows;
          }
          if (p.d[q] > 0) {
            it.dst[3] = sblock(v, p.node_of[q]);
            it.dst_buf[3] = DST_S;
            it.ld[3] = it.rows;
          }
          w.x.push_back(it);
          flops += 2.0 * double(it.rows) * it.cols * it.cols;
        }
        for (int64_t z = 0; z < int64_t(CP[l].size()); ++z) {
          int q = kfirst(CP[l][z]), wn = ksecond(CP[l][z]);
          if (p.m[q] == 0) continue;
          XItem it{};
          it.src = cp_off[l][z];
          it.src_buf = SRC_CP;
          it.ld_src = int32_t(p.m[q]);
          it.rows = int32_t(p.m[q]);
          it.cols = int32_t(p.node_size[wn]);
          it.qL = p.q_off[q];
          it.qR = -1;
          it.qside = 0;
          it.kr = int32_t(p.kp[q]);
          it.kc = 0;
          for (int k = 0; k < 4; ++k) it.dst[k] = -1;
          if (p.kp[q] > 0) {
            Dst ds = dst_CP(l + 1, p.parent[q], wn);
            it.dst[1] = ds.off + p.off[q];
            it.dst_buf[1] = ds.buf;
            it.ld[1] = int32_t(p.m[p.parent[q]]);
          }
          if (p.d[q] > 0) {
            it.dst[3] = sblock(p.node_of[q], wn);
            it.dst_buf[3] = DST_S;
            it.ld[3] = int32_t(p.d[q]);
          }
          w.x.push_back(it);
          flops += 2.0 * double(it.rows) * it.rows * it.cols;
        }
      }
    }
    p.sparsify_flops = flops;

    // ---------------- symbolic block LU (a7) ----------------
    auto lca = [&](int a, int b) {
      while (dep[a] > dep[b]) a = p.parent[a];
      while (dep[b] > dep[a]) b = p.parent[b];
      while (a != b) a = p.parent[a], b = p.parent[b];
      return a;
    };
    p.closure.assign(nn, 0);
    for (int v = 0; v < nn; ++v) {
      int l = p.node_level[v], t = p.node_cluster[v];
      if (l == lstop) {
        p.closure[v] = p.root[t];
        continue;
      }
      int c = t;
      auto lo = std::lower_bound(near[l].begin(), near[l].end(), key(t, 0));
      for (auto it = lo; it != near[l].end() && kfirst(*it) == t; ++it) {
        int e = ksecond(*it);
        if (e > t) c = lca(c, e);
      }
      p.closure[v] = c;
    }
    p.order.resize(nn);
    for (int v = 0; v < nn; ++v) p.order[v] = v;
    std::sort(p.order.begin(), p.order.end(), [&](int a, int b) {
      int ca = p.closure[a], cb = p.closure[b];
      if (dep[ca] != dep[cb]) return dep[ca] > dep[cb];
      if (ca != cb) return ca < cb;
      return a < b;
    });
    std::vector<int32_t> pos(nn);
    for (int i = 0; i < nn; ++i) pos[p.order[i]] = i;
    p.sn_ptr.assign(1, 0);
    for (int i = 1; i < nn; ++i)
      if (p.closure[p.order[i]] != p.closure[p.order[i - 1]]) p.sn_ptr.push_back(i);
    p.sn_ptr.push_back(nn);
    const int nsn = int(p.sn_ptr.size()) - 1;
    std::vector<int32_t> sn_of(nn);
    for (int k = 0; k < nsn; ++k)
      for (int i = p.sn_ptr[k]; i < p.sn_ptr[k + 1]; ++i) sn_of[p.order[i]] = k;
    // structurally symmetric adjacency of S
    std::vector<int64_t> adj_ptr(nn + 1, 0);
    for (int i = 0; i < nn; ++i)
      for (int64_t z = p.brow_ptr[i]; z < p.brow_ptr[i + 1]; ++z) {
        int j = p.bcol[z];
        if (i != j) adj_ptr[i + 1]++, adj_ptr[j + 1]++;
      }
    for (int i = 0; i < nn; ++i) adj_ptr[i + 1] += adj_ptr[i];
    std::vector<int32_t> adj(adj_ptr[nn]);
    {
      std::vector<int64_t> fill(adj_ptr.begin(), adj_ptr.end() - 1);
      for (int i = 0; i < nn; ++i)
        for (int64_t z = p.brow_ptr[i]; z < p.brow_ptr[i + 1]; ++z) {
          int j = p.bcol[z];
          if (i != j) adj[fill[i]++] = j, adj[fill[j]++] = i;
        }
    }
    std::vector<std::vector<int32_t>> bnd(nsn), kids(nsn);
    std::vector<int32_t> sn_parent(nsn, -1), mark(nn, -1);
    for (int k = 0; k < nsn; ++k) {
      const int end = p.sn_ptr[k + 1];
      std::vector<int32_t> &B = bnd[k];
      auto add = [&](int w) {
        if (pos[w] >= end && mark[w] != k) {
          mark[w] = k;
          B.push_back(w);
        }
      };
      for (int i = p.sn_ptr[k]; i < end; ++i) {
        int v = p.order[i];
        for (int64_t z = adj_ptr[v]; z < adj_ptr[v + 1]; ++z) add(adj[z]);
      }
      for (int c : kids[k])
        for (int w : bnd[c]) add(w);
      std::sort(B.begin(), B.end(), [&](int a, int b) { return pos[a] < pos[b]; });
      if (!B.empty()) {
        sn_parent[k] = sn_of[B[0]];
        kids[sn_parent[k]].push_back(k);
      }
    }
    p.bnd_ptr.assign(nsn + 1, 0);
    for (int k = 0; k < nsn; ++k) p.bnd_ptr[k + 1] = p.bnd_ptr[k] + int32_t(bnd[k].size());
    p.bnd.resize(p.bnd_ptr[nsn]);
    for (int k = 0; k < nsn; ++k) std::copy(bnd[k].begin(), bnd[k].end(), p.bnd.begin() + p.bnd_ptr[k]);
    // fronts
    p.fronts.resize(nsn);
    std::vector<int64_t> sn_local(nn, 0);  // scalar offset of a node inside its own supernode
    std::vector<std::vector<int64_t>> bpre(nsn);
    double fl = 0.0, flc = 0.0;
    for (int k = 0; k < nsn; ++k) {
      int64_t s = 0;
      for (int i = p.sn_ptr[k]; i < p.sn_ptr[k + 1]; ++i) {
        sn_local[p.order[i]] = s;
        s += p.node_size[p.order[i]];
      }
      int64_t b = 0;
      bpre[k].resize(bnd[k].size() + 1, 0);
      for (size_t i = 0; i < bnd[k].size(); ++i) {
        bpre[k][i] = b;
        b += p.node_size[bnd[k][i]];
      }
      bpre[k][bnd[k].size()] = b;
      if (s + b > (int64_t(1) << 30)) throw Fail{H2SP_EUNSUPPORTED, "front too large"};
      Front &F = p.fronts[k];
      F.s = int32_t(s);
      F.b = int32_t(b);
      F.f = int32_t(s + b);
      F.ld = int32_t((F.f + 3) / 4 * 4);
      F.parent = sn_parent[k];
      F.off = p.front_elems;
      F.piv_off = p.piv_elems;
      F.idx_off = int64_t(p.front_idx.size());
      F.map_off = 0;
      p.front_elems += int64_t(F.ld) * F.f;
      p.piv_elems += s;
      F.dinv_off = p.dinv_elems;
      p.dinv_elems += ((s + 63) / 64) * 2 * 64 * 64;
      p.max_front = std::max<int64_t>(p.max_front, F.f);
      for (int i = p.sn_ptr[k]; i < p.sn_ptr[k + 1]; ++i) {
        int v = p.order[i];
        for (int64_t r = 0; r < p.node_size[v]; ++r) p.front_idx.push_back(int32_t(p.node_off[v] + r));
      }
      for (int w : bnd[k])
        for (int64_t r = 0; r < p.node_size[w]; ++r) p.front_idx.push_back(int32_t(p.node_off[w] + r));
      double ds = double(s), db = double(b);
      fl += (2.0 / 3.0) * ds * ds * ds + 2.0 * ds * ds * db + 2.0 * ds * db * db;
      flc += ds * ds * ds / 3.0 + ds * ds * db + ds * db * db;
    }
    p.factor_flops = fl;
    p.chol_flops = flc;
    auto pos_in_front = [&](int k, int w) -> int64_t {
      if (sn_of[w] == k) return sn_local[w];
      const auto &B = bnd[k];
      auto it = std::lower_bound(B.begin(), B.end(), w, [&](int a, int b) { return pos[a] < pos[b]; });
      if (it == B.end() || *it != w) throw Fail{H2SP_EINVAL, "internal: node missing from front"};
      return p.fronts[k].s + bpre[k][it - B.begin()];
    };
    for (int k = 0; k < nsn; ++k) {
      int pk = sn_parent[k];
      p.fronts[k].map_off = int64_t(p.front_map.size());
      if (pk < 0) continue;
      for (int w : bnd[k]) {
        int64_t base = pos_in_front(pk, w);
        for (int64_t r = 0; r < p.node_size[w]; ++r) p.front_map.push_back(int32_t(base + r));
      }
    }
    // assembly of S blocks into fronts
    p.assemble.reserve(nnzb);
    for (int i = 0; i < nn; ++i)
      for (int64_t z = p.brow_ptr[i]; z < p.brow_ptr[i + 1]; ++z) {
        int j = p.bcol[z];
        int k = pos[i] < pos[j] ? sn_of[i] : sn_of[j];
        const Front &F = p.fronts[k];
        AItem a{};
        a.src = p.val_off[z];
        a.rows = int32_t(p.node_size[i]);
        a.cols = int32_t(p.node_size[j]);
        a.ld = F.ld;
        a.dst = F.off + pos_in_front(k, j) * F.ld + pos_in_front(k, i);
        p.assemble.push_back(a);
      }
    // elimination levels: consecutive supernodes of equal closure depth
    p.front_level_ptr.assign(1, 0);
    for (int k = 1; k < nsn; ++k)
      if (dep[p.closure[p.order[p.sn_ptr[k]]]] != dep[p.closure[p.order[p.sn_ptr[k - 1]]]])
        p.front_level_ptr.push_back(k);
    p.front_level_ptr.push_back(nsn);

    // ---------------- work lists: small items first, grouped by size ----------------
    // Items whose blocks fit kMaxBlock go to the shared-memory kernels, the
    // rest to the streaming ones: each level's list keeps the small items in
    // front, the row and column completions in step.  Inside each part the
    // items are grouped by (block size, rank), largest first, so that the
    // persistent kernels walking a list with the grid's stride see items of
    // like cost side by side and finish together.
    for (LevelWork &w : p.lw) {
      std::vector<size_t> qi(w.q.size());
      for (size_t i = 0; i < qi.size(); ++i) qi[i] = i;
      auto qsmall = std::stable_partition(qi.begin(), qi.end(), [&](size_t i) { return w.q[i].m <= kMaxBlock; });
      w.nq_small = int(qsmall - qi.begin());
      auto by_size_q = [&](size_t a, size_t b) {
        return w.q[a].m != w.q[b].m ? w.q[a].m > w.q[b].m : w.q[a].k > w.q[b].k;
      };
      std::stable_sort(qi.begin(), qsmall, by_size_q);
      std::stable_sort(qsmall, qi.end(), by_size_q);
      std::vector<QItem> q2, qc2;
      for (size_t i : qi) {
        q2.push_back(w.q[i]);
        if (!w.qc.empty()) qc2.push_back(w.qc[i]);
      }
      w.q.swap(q2);
      w.qc.swap(qc2);
      auto xsmall = std::stable_partition(w.x.begin(), w.x.end(), [](const XItem &it) {
        return it.rows <= kMaxBlock && it.cols <= kMaxBlock;
      });
      w.nx_small = int(xsmall - w.x.begin());
      auto by_size_x = [](const XItem &a, const XItem &b) {
        const int64_t ca = int64_t(a.rows) * a.cols, cb = int64_t(b.rows) * b.cols;
        return ca != cb ? ca > cb : a.rows > b.rows;
      };
      std::stable_sort(w.x.begin(), xsmall, by_size_x);
      std::stable_sort(xsmall, w.x.end(), by_size_x);
      std::stable_sort(w.c.begin(), w.c.end(), [](const CItem &a, const CItem &b) {
        const int64_t ca = int64_t(a.kp_p) * a.kp_q, cb = int64_t(b.kp_p) * b.kp_q;
        return ca != cb ? ca > cb : a.k_p > b.k_p;
      });
    }

    // ---------------- bounds audit of every work item ----------------
    // Each item's accessed range must lie inside the internal buffer it names;
    // a failure here is a planning bug and nothing is launched.
    {
      auto inside = [&](int64_t off, int64_t rows, int64_t cols, int64_t ld, int64_t size, const char *what) {
        if (rows <= 0 || cols <= 0) return;
        if (off < 0 || ld < rows || off + ld * (cols - 1) + rows > size)
          throw Fail{H2SP_EINVAL, std::string("internal: item out of bounds: ") + what};
      };
      for (int l = 0; l < int(p.lw.size()); ++l) {
        const LevelWork &w = p.lw[l];
        const int64_t cn = l + 1 < lstop ? p.c_elems[l + 1] : 0, rn = l + 1 < lstop ? p.rp_elems[l + 1] : 0,
                      pn = l + 1 < lstop ? p.cp_elems[l + 1] : 0;
        const int64_t dsz[4] = {p.s_elems, cn, rn, pn};
        const int64_t ssz[4] = {std::numeric_limits<int64_t>::max() / 4, l < lstop ? p.c_elems[l] : 0,
                                l < lstop ? p.rp_elems[l] : 0, l < lstop ? p.cp_elems[l] : 0};
        for (size_t i = 0; i < w.x.size(); ++i) {
          const XItem &it = w.x[i];
          const int cap = int(i) < w.nx_small ? kMaxBlock : kMaxLargeBlock;
          if (it.rows > cap || it.cols > cap || it.rows <= 0 || it.cols <= 0)
            throw Fail{H2SP_EINVAL, "internal: transform block size"};
          inside(it.src, it.rows, it.cols, it.ld_src, ssz[it.src_buf], "transform source");
          if (it.qL >= 0) inside(it.qL, it.rows, it.rows, it.rows, p.q_elems, "left Q");
          if (it.qR >= 0) inside(it.qR, it.cols, it.cols, it.cols, p.q_elems, "right Q");
          for (int qd = 0; qd < 4; ++qd) {
            if (it.dst[qd] < 0) continue;
            const int nr = (qd & 2) ? it.rows - it.kr : it.kr, nc = (qd & 1) ? it.cols - it.kc : it.kc;
            inside(it.dst[qd], nr, nc, it.ld[qd], dsz[it.dst_buf[qd]], "transform destination");
          }
        }
        for (const CItem &it : w.c) {
          inside(it.rr_p, it.kp_p, it.k_p, it.kp_p, p.rr_elems, "coupling Rr_p");
          inside(it.rr_q, it.kp_q, it.k_q, it.kp_q, p.rr_elems, "coupling Rr_q");
          inside(it.dst, it.kp_p, it.kp_q, it.ld, dsz[it.dst_buf], "coupling destination");
        }
        for (const WItem &it : w.w) {
          inside(it.rr_c, it.kp_c, it.k_c, it.kp_c, p.rr_elems, "stack Rr");
          inside(it.w_dst, it.kp_c, it.k_p, it.ld_w, w.w_elems, "stack W");
        }
        for (size_t i = 0; i < w.q.size(); ++i) {
          const QItem &it = w.q[i];
          const int cap = int(i) < w.nq_small ? kMaxBlock : kMaxLargeBlock;
          if (it.m > cap || it.k > kMaxRank) throw Fail{H2SP_EINVAL, "internal: Householder size"};
          inside(it.q, it.m, it.m, it.m, p.q_elems, "Q");
          inside(it.rr, std::min(it.m, it.k), it.k, std::min(it.m, it.k), p.rr_elems, "Rr");
          if (it.w_buf == 1) inside(it.w, it.m, it.k, it.ld_w, w.w_elems, "W");
        }
      }
      for (const AItem &a : p.assemble) {
        inside(a.src, a.rows, a.cols, a.rows, p.s_elems, "assembly source");
        inside(a.dst, a.rows, a.cols, a.ld, p.front_elems, "assembly destination");
      }
      for (size_t k = 0; k < p.fronts.size(); ++k) {
        const Front &F = p.fronts[k];
        inside(F.off, F.f, F.f, F.ld, p.front_elems, "front");
        if (F.piv_off + F.s > p.piv_elems || F.idx_off + F.f > int64_t(p.front_idx.size()))
          throw Fail{H2SP_EINVAL, "internal: front index arrays"};
        if (F.parent >= 0) {
          if (F.map_off + F.b > int64_t(p.front_map.size())) throw Fail{H2SP_EINVAL, "internal: front map"};
          const int pf = p.fronts[F.parent].f;
          for (int i = 0; i < F.b; ++i)
            if (p.front_map[F.map_off + i] < 0 || p.front_map[F.map_off + i] >= pf ||
                (i > 0 && p.front_map[F.map_off + i] <= p.front_map[F.map_off + i - 1]))
              // increasing: the lower triangle of a contribution block lands in the parent's
              throw Fail{H2SP_EINVAL, "internal: extend-add position"};
        }
        for (int i = 0; i < F.f; ++i)
          if (p.front_idx[F.idx_off + i] < 0 || p.front_idx[F.idx_off + i] >= p.n)
            throw Fail{H2SP_EINVAL, "internal: front global index"};
      }
      for (size_t i = 0; i + 1 < p.front_level_ptr.size(); ++i)
        if (p.front_level_ptr[i + 1] - p.front_level_ptr[i] > 65535)
          throw Fail{H2SP_EUNSUPPORTED, "more than 65535 fronts in one elimination level"};
    }

    // ---------------- H^2 matvec workspace ----------------
    p.xh_off.assign(ncl, 0);
    for (int t = 0; t < ncl; ++t) {
      p.xh_off[t] = p.xh_elems;
      p.xh_elems += p.rank[t];
    }
  } catch (const Fail &f) {
    err = f.msg;
    return f.code;
  } catch (const std::bad_alloc &) {
    err = "host allocation failed while planning";
    return H2SP_ENOMEM;
  }
  return H2SP_OK;
}

}  // namespace h2sp
