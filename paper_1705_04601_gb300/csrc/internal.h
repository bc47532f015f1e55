// Internal structures of the h2sp library: the host plan (integer structure
// of the level recursion of §2.3 and of the block LU of S) and the flat work
// items the kernels consume.  Everything here is host-built once per
// h2sp_sparsify call and uploaded as plain arrays.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/h2sp.h"

namespace h2sp {

// Largest local block (m_t) of the kernels that stage whole blocks in shared
// memory; items up to this size take them.
constexpr int kMaxBlock = 64;
// Largest local block (m_t) accepted at all: larger items (3D leaves of up to
// 128 points, upper-level blocks stacked from up to 8 sons) take the kernels
// that stream the block from global memory.
constexpr int kMaxLargeBlock = 384;
// Largest basis rank (columns of a Householder item).
constexpr int kMaxRank = 64;

// Buffers a transform item reads from / writes to.
enum SrcBuf : int8_t { SRC_NEAR = 0, SRC_C = 1, SRC_RP = 2, SRC_CP = 3 };
enum DstBuf : int8_t { DST_S = 0, DST_C = 1, DST_RP = 2, DST_CP = 3 };

// Y = (qL >= 0 ? QL^T : I) * X * (qR >= 0 ? QR : I), X is rows x cols,
// then Y is split at row kr and column kc into four quadrants:
//   0: [0,kr) x [0,kc)     basis rows,     basis cols      -> next-level close block
//   1: [0,kr) x [kc,cols)  basis rows,     non-basis cols  -> next-level column panel
//   2: [kr,rows) x [0,kc)  non-basis rows, basis cols      -> next-level row panel
//   3: [kr,rows) x [kc,..) non-basis rows, non-basis cols  -> final block of S
// Each quadrant goes to dst[i] (element offset in buffer dst_buf[i], column-
// major with leading dimension ld[i]); dst[i] < 0 skips it.
struct XItem {
  int64_t src;
  int64_t qL, qR;
  int64_t dst[4];
  int32_t ld_src, rows, cols, kr, kc;
  int32_t ld[4];
  int8_t src_buf;
  int8_t dst_buf[4];
  int8_t qside;  // bit 0: QL from the column-side Q buffer, bit 1: QR from the column-side buffer
  int8_t pad[2];
};

// Far pair (p, q) of level l: F = Rr_p D_pq Rrc_q^T (kp_p x kp_q) into a next-level block.
struct CItem {
  int64_t rr_p, rr_q, dcoup, dst;
  int32_t kp_p, k_p, kp_q, k_q, ld;
  int8_t dst_buf;
  int8_t pad[3];
};

// Child c of level l: rows [off_c, off_c + kp_c) of W_parent = Rr_c T_c.
struct WItem {
  int64_t rr_c, t_c, w_dst;
  int32_t kp_c, k_c, k_p, ld_w;
};

// Cluster t: Householder completion of W_t (m x k) -> Q_t (m x m), Rr_t (kp x k).
struct QItem {
  int64_t w, q, rr;
  int32_t m, k, ld_w;
  int8_t w_buf;  // 0: input leaf basis, 1: W buffer
  int8_t pad[3];
};

// Copy one block of S into its front (and convert to the factor precision).
struct AItem {
  int64_t src, dst;
  int32_t rows, cols, ld;
  int32_t pad;
};

struct Front {
  int64_t off;      // element offset of the f x f front (column-major, leading dimension ld)
  int64_t piv_off;  // offset into the pivot array (s entries)
  int64_t idx_off;  // offset into the global-index array (f entries)
  int64_t map_off;  // offset into the extend-add map (b entries)
  int64_t dinv_off; // offset of the inverted diagonal blocks (2 * 64 * 64 per 64 supernode columns)
  int32_t s, b, f;
  int32_t parent;   // parent front, -1 for a root
  int32_t ld;       // f rounded up to a multiple of 4: every column starts on a 16-byte boundary
};

struct LevelWork {
  // sparsification of level l (l < lstop)
  std::vector<QItem> q, qc;   // row side / column side completions
  std::vector<WItem> w, wc;   // stacking of the next level's W from this level's Rr
  std::vector<CItem> c;
  std::vector<XItem> x;
  int64_t w_elems = 0, wc_elems = 0;  // W buffer sizes for this level (built from level l-1)
  int max_m = 0, max_k = 0;
  // q / qc and x are ordered small items first (all sizes <= kMaxBlock), then
  // the large ones; these count the small ones
  int nq_small = 0, nx_small = 0;
};

struct Plan {
  int64_t n = 0;
  int D = 0, lstop = 0, ncl = 0, nleaf = 0;
  bool sym = true;
  // per cluster
  std::vector<int32_t> level, parent, rank, root;
  std::vector<int64_t> m, kp, d, off, xoff;
  std::vector<int64_t> q_off, rr_off;   // offsets in the Q / Rr buffers (-1 if none)
  // S nodes
  std::vector<int32_t> node_level, node_cluster, node_of;  // node_of[cluster] or -1
  std::vector<int64_t> node_size, node_off;
  // S pattern (VBR)
  std::vector<int64_t> brow_ptr, val_off;
  std::vector<int32_t> bcol;
  int64_t s_elems = 0;
  // level work and buffer sizes
  std::vector<LevelWork> lw;
  std::vector<int64_t> c_elems, rp_elems, cp_elems;  // per level (index l), 0 for l == 0 / l >= lstop
  int64_t q_elems = 0, rr_elems = 0;
  double sparsify_flops = 0.0;
  // symbolic factorization
  std::vector<int32_t> closure, order, sn_ptr, bnd_ptr, bnd;
  std::vector<Front> fronts;
  std::vector<int32_t> front_level_ptr;   // fronts grouped by elimination level
  std::vector<int32_t> front_idx;          // global scalar index of each front row
  std::vector<int32_t> front_map;          // position in the parent front of each boundary row
  std::vector<AItem> assemble;
  int64_t front_elems = 0, piv_elems = 0, max_front = 0, dinv_elems = 0;
  double factor_flops = 0.0;
  double chol_flops = 0.0;  // the block Cholesky's: sum over supernodes of s^3/3 + s^2 b + s b^2
  // H^2 matvec structure (Definition 4.9)
  std::vector<int64_t> h_begin, h_size;
  std::vector<int64_t> leaf_basis_off, transfer_off, coupling_off, near_off;
  std::vector<int64_t> col_leaf_basis_off, col_transfer_off;
  std::vector<int64_t> far_ptr, near_ptr;
  std::vector<int32_t> far_col, near_col;
  std::vector<int32_t> level_ptr;
  std::vector<int64_t> xh_off;  // offset of each cluster's coefficient vector (k_t) in the matvec workspace
  int64_t xh_elems = 0;
};

// Kernel classes of the per-launch profiler (h2sp_profile).
enum ProfClass : int {
  P_GEMM = 0,        // trailing update of the fronts
  P_PANEL = 1,       // panel factorization with pivoting
  P_TRSM = 2,        // row swaps + U12 triangular solve
  P_EXTEND = 3,      // extend-add into parent fronts
  P_ASSEMBLE = 4,    // S blocks into fronts
  P_TRANSFORM = 5,   // close blocks / panels Q^T X Q (sparsification)
  P_HOUSEHOLDER = 6, // basis completions
  P_COUPLING = 7,    // coupling projections and W stacking
  P_SOLVE = 8,       // triangular solves with the fronts
  P_MATVEC = 9,      // FP64 H^2 product
  P_APPLY = 10,      // U^T / V applies
  P_OTHER = 11,      // vector kernels, casts, permutations
  P_GEMM_INNER = 12, // FP32 blocked factorizations: in-block rank-64 updates and operand packing
  P_NCLASS = 13
};

// Counts every launch; when `timing` is on, brackets launches with CUDA events
// on the launching stream and accumulates their durations per class.
struct Prof {
  bool timing = false;
  cudaStream_t stream = nullptr;
  int64_t launches[P_NCLASS] = {};
  int64_t timed[P_NCLASS] = {};
  double ms[P_NCLASS] = {};
  double work[P_NCLASS] = {};
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  struct Rec {
    int cls;
    size_t e0, e1;
    double w;
  };
  std::vector<Rec> recs;
  // events go on `st` when given (work launched on a side stream), else on `stream`
  size_t begin(cudaStream_t st = nullptr) {
    if (!timing) return 0;
    return take(st);
  }
  void end(int cls, int nlaunch, size_t e0, double w, cudaStream_t st = nullptr) {
    launches[cls] += nlaunch;
    if (!timing) return;
    recs.push_back(Rec{cls, e0, take(st), w});
  }
  void count(int cls, int nlaunch) { launches[cls] += nlaunch; }
  size_t take(cudaStream_t st = nullptr) {
    if (used == ev.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
    }
    cudaEventRecord(ev[used], st ? st : stream);
    return used++;
  }
  void collect() {
    if (recs.empty()) {
      used = 0;
      return;
    }
    for (size_t i = 0; i < used; ++i) cudaEventSynchronize(ev[i]);  // events may sit on two streams
    for (const Rec &r : recs) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[r.e0], ev[r.e1]);
      ms[r.cls] += t;
      timed[r.cls] += 1;
      work[r.cls] += r.w;
    }
    recs.clear();
    used = 0;
  }
  void reset() {
    for (int i = 0; i < P_NCLASS; ++i) launches[i] = timed[i] = 0, ms[i] = work[i] = 0.0;
  }
  ~Prof() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// The level schedule of §2.2-2.3 as the device kernels give it (host copies):
// l_stop, per cluster m, k', d, off, xoff, q_off and its S node (-1: none),
// per node its cluster, level and first row (node_off[nn] = n), and Near_l
// for 1 <= l <= l_stop as CSR over the clusters of level l.
struct A1Result {
  int lstop = 0, nn = 0;
  std::vector<int64_t> m, kp, d, off, xoff, q_off, node_off;
  std::vector<int32_t> node_of, node_cluster, node_level;
  std::vector<std::vector<int64_t>> near_ptr;
  std::vector<std::vector<int32_t>> near_col;
};
// Called by build_plan once the descriptor is validated (the plan's copies of
// the structure arrays are set): fills the level schedule.  Returns an h2sp_status.
using A1Source = std::function<int(const Plan &, A1Result &, std::string &)>;

// Validate the descriptor and build the plan.  Returns an h2sp_status.  With
// `a1`, the level schedule comes from it; otherwise the host derives it.
int build_plan(const h2sp_h2_desc *d, Plan &p, std::string &err, bool need_numbers = true,
               const A1Source *a1 = nullptr);

}  // namespace h2sp
