// Launchers of the h2sp kernels (host side declarations).
#pragma once

#include <map>
#include <mutex>
#include <utility>

#include <cuda_runtime.h>

#include "internal.h"

namespace h2sp {

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device.  The attribute belongs to one device, so it is remembered per
// (kernel, device), under a lock shared by every host thread.
inline cudaError_t smem_attr(const void *fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int &have = done[{fn, dev}];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

// FMA rate of the current device in TFLOP/s (kind 0: FP64, 1: FP32), peak.cu.
cudaError_t measure_fma_peak(int kind, double *tflops, cudaStream_t s);

// Streaming multiprocessors of the current device (cached per device).
inline int device_sms() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
  cache[dev] = n;
  return n;
}

// Grid of a persistent launch over n work items: the CTAs of `fn` (threads,
// dynamic shared memory) that are resident at once on the current device
// (occupancy x SMs, cached per kernel, device and launch shape), at most n.
inline unsigned persistent_grid(const void *fn, int threads, size_t smem, int n) {
  static std::mutex mu;
  static std::map<std::pair<std::pair<const void *, int>, std::pair<int, size_t>>, int> cache;
  int dev = 0;
  if (n <= 0) return 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return unsigned(n);
  int per = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(std::make_pair(fn, dev), std::make_pair(threads, smem));
    auto it = cache.find(key);
    if (it != cache.end()) {
      per = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        per = 1;
      }
      per = per > 0 ? per : 1;
      cache[key] = per;
    }
  }
  const long long g = (long long)per * device_sms();
  return unsigned(g < n ? g : n);
}

// ---- sparsification (sparsify.cu).  Householder completions and stacked
// bases are FP64; the products that land in S (and in the level buffers that
// feed it) use W = double, or float for an FP32 S.
cudaError_t launch_householder(const QItem *items, int n, const double *w_in, const double *w_buf, double *Q,
                               double *Rr, int max_m, int max_k, cudaStream_t s, Prof *prof);
// the same for items with m > kMaxBlock (Q formed in its global output)
cudaError_t launch_householder_large(const QItem *items, int n, const double *w_in, const double *w_buf, double *Q,
                                     double *Rr, int max_m, int max_k, cudaStream_t s, Prof *prof);
cudaError_t launch_stack_w(const WItem *items, int n, const double *Rr, const double *T, double *W, cudaStream_t s,
                           Prof *prof);
template <typename W>
cudaError_t launch_coupling(const CItem *items, int n, const double *Rr, const double *Rrc, const double *Dc,
                            W *const *dst_base, int max_k, cudaStream_t s, Prof *prof);
// src_base[0] is the FP64 close-block array, src_base[1..3] level buffers of type W
template <typename W>
cudaError_t launch_transform(const XItem *items, int n, const void *const *src_base, const double *Qrow,
                             const double *Qcol, W *const *dst_base, cudaStream_t s, Prof *prof, double flops);
// the same for items with rows or cols above kMaxBlock (max_rows, max_cols: their largest sizes)
template <typename W>
cudaError_t launch_transform_large(const XItem *items, int n, const void *const *src_base, const double *Qrow,
                                   const double *Qcol, W *const *dst_base, int max_rows, int max_cols, cudaStream_t s,
                                   Prof *prof, double flops);

// ---- block LU of S (factor.cu), T = double or float ----
struct FrontDev {
  int64_t off, piv_off, idx_off, map_off, dinv_off;
  int32_t s, b, f, parent;
  int32_t ld;        // leading dimension of the front (f rounded up to a multiple of 4)
  int32_t pack_off;  // first 128-row tile of the front in its level's packed GEMM operands
};

// Packed operands of the blocked FP32 LU's block-end update: per 128-row
// (or 128-column) tile, kPackChunks chunks of 16 K values, each a TF32 hi
// array and a lo array of 128 x 16 in the tensor cores' shared-memory layout.
constexpr int kPackChunks = 16;
constexpr int64_t kPackTileFloats = int64_t(kPackChunks) * 2 * 128 * 16;

// Column block of the blocked triangular solves (and of the inverted diagonal blocks).
constexpr int kSolveBlock = 64;

// Panel width of the blocked LU per precision.
template <typename T>
struct LuCfg;
template <>
struct LuCfg<double> {
  static constexpr int NB = 32;
};
template <>
struct LuCfg<float> {
  static constexpr int NB = 64;
};

// Maximum number of rows a panel swaps (2 per column).
constexpr int kMaxSwapRows = 2 * 64;

// Outer block width of the blocked FP32 factorizations (four 64-column panels).
constexpr int kLuOuterBlock = 256;

// FP32 trailing updates on the tensor cores (H2SP_GEMM unset or not "simt").
bool use_tensor_core_gemm_host();

// S values of type TS (the sparsification's precision) into fronts of type T
template <typename TS, typename T>
cudaError_t launch_assemble(const AItem *items, int64_t n, const TS *S, T *fronts, cudaStream_t s, Prof *prof,
                            double bytes);
// Look-ahead resources of the block LU: a high-priority stream on which the
// next panel is factored and a low-priority one on which the rest of the
// trailing update runs meanwhile (both released by the same event, so the
// panel is dispatched first), and the events that order them.
struct LuAsync {
  cudaStream_t side = nullptr;  // high priority: the next panel
  cudaStream_t rest = nullptr;  // low priority: the rest of the trailing update
  cudaEvent_t next = nullptr, panel = nullptr, done = nullptr;
};
// Blocked LU with partial pivoting inside the supernode rows of every front of
// one level (all fronts in parallel).  With `la` (may be null) the panel of
// step k + 1 overlaps the trailing update of step k.
template <typename T>
cudaError_t launch_lu_level(const FrontDev *fr, const Front *host_fr, int nfront, int max_s, int max_f, T *fronts,
                            int32_t *piv, int32_t *swaps, int *err, cudaStream_t s, const LuAsync *la, Prof *prof,
                            const uint8_t *maps = nullptr, float *pack = nullptr, const uint8_t *maps64 = nullptr);
// lower: only the lower triangle of each contribution block (block Cholesky;
// the map is monotone, so it lands in the parent's lower triangle)
template <typename T>
cudaError_t launch_extend_add_impl(const FrontDev *fr_all, int lo, int nfront, int max_b, const int32_t *map,
                                   T *fronts, cudaStream_t s, Prof *prof, double elems, bool lower = false);
// Schedule of the blocked FP32 block Cholesky (h2sp_set_option; chosen by the
// package's autotuner): a cap on the 128-column tiles one CTA of the
// low-priority block-end update takes (0: whole-wave split), the SMs that
// update leaves free for the panel stream (-1: the level's front count), and
// the look-ahead (the next block's panels on their own stream).
struct CholSchedule {
  int tiles_per_cta = 0;
  int panel_sms = -1;
  int lookahead = 1;
  int wide = 2;  // TF32 block-end update: 2 = 128 x 256 tiles, C by TMA reduce-add, four operand stages
                 // (launch_gemm_tc_wide, reduce); 1 = 128 x 256 tiles, C loaded and stored; 0 = 128 x 128
};
// Block Cholesky of every front of one level (all fronts in parallel): no
// pivoting, lower-triangle updates, the B operand read from L21.  A pivot
// that is not positive sets bit 8 of *err.  FP32 with `maps` and `pack` uses
// the tensor cores in 256-column outer blocks (la as in launch_lu_level).
// inv: scratch of nfront x kCholInvElems elements (the panels' L11^-1).
constexpr int kCholInvElems = 64 * 64;
template <typename T>
cudaError_t launch_chol_level(const FrontDev *fr, const Front *host_fr, int nfront, int max_s, int max_f, T *fronts,
                              int32_t *piv, int *err, cudaStream_t s, const LuAsync *la, Prof *prof,
                              const uint8_t *maps, float *pack, T *inv, const CholSchedule *sched = nullptr,
                              const uint8_t *maps64 = nullptr, int bf16 = 0);
// Rewrite Cholesky-factored fronts in the LU form: unit L = L_chol D^-1, U = D L_chol^T.
template <typename T>
cudaError_t launch_chol_to_lu(const FrontDev *fr, int nfront, int max_f, T *fronts, cudaStream_t s, Prof *prof,
                              double bytes);
// One CUDA-core panel update of the lower triangle, the B operand read from L21.
template <typename T>
cudaError_t launch_gemm_update_sym(const FrontDev *fr, int j0, int nfront, int max_f, T *fronts, cudaStream_t s);
template <typename T>
cudaError_t launch_make_perm(const FrontDev *fr, int nfront, int max_s, const int32_t *piv, int32_t *perm,
                             cudaStream_t s, Prof *prof);
// Inverses of the kSolveBlock-square diagonal blocks of L11 and U11 of every front.
template <typename T>
cudaError_t launch_invert_diag(const FrontDev *fr, int nfront, int max_s, const T *fronts, T *dinv, cudaStream_t s,
                               Prof *prof);
// log|det| of the factored S per independent system (§5.3): per front, the sum
// of log|u_jj| over its pivot block and the parity of its interchanges and
// negative pivots (lsum, flips: one entry per front); then per system w the
// sums over its fronts sys_front[sys_ptr[w] .. sys_ptr[w+1]) into out[w] and
// sign[w] (+1 / -1).  Both sums in FP64, in a fixed order.
template <typename T>
cudaError_t launch_logdet(const FrontDev *fr, int nfront, const T *fronts, const int32_t *piv, const int32_t *sys_ptr,
                          const int32_t *sys_front, int nsys, double *lsum, int *flips, double *out, int32_t *sign,
                          cudaStream_t s, Prof *prof);
// Work lists of the flag-synchronised sweeps (one launch per level and
// direction): items (front, row block) of level li are items[fwd_off[li] ..
// fwd_off[li] + fwd_n[li]) in dependency order (a supernode item covers row
// blocks b and b+1 forward, b and b-1 backward), likewise for the backward
// sweep; one flag per supernode row block of every front (index
// dinv_off / (2 kSolveBlock^2) + block), published with the launch's epoch;
// two ticket counters per level, zero before each sweep; err |= 4 on a
// bounded-wait timeout.
struct ChainArgs {
  const int2 *items = nullptr;
  const int *fwd_off = nullptr, *fwd_n = nullptr, *bwd_off = nullptr, *bwd_n = nullptr;  // host arrays
  int *tickets = nullptr, *flags = nullptr, *err = nullptr;
  int epoch = 0;       // published by every solved block of the launch
  int wait_epoch = 0;  // awaited on the blocks a block depends on (= epoch, except in the wait test)
  uint32_t spin_cap = 1u << 22;  // polls of one wait before it gives up
};
// Forward sweep for one level (fronts [lo, lo+nfront) of fr): gathers P^T y into
// the fronts' work vectors, z = L11^-1 (.) block by block into zbuf, adds
// -L21 z into the boundary rows of y and stores z into the supernode rows.
template <typename T>
cudaError_t launch_solve_fwd_level_impl(const FrontDev *fr, int lo, int nfront, int max_s, int max_f, const T *fronts,
                                        const T *dinv, const int32_t *perm, const int32_t *idx, T *y, int64_t ldy,
                                        int nrhs, T *work, T *zbuf, const int64_t *work_off, cudaStream_t s,
                                        Prof *prof, double bytes, const ChainArgs *ca = nullptr, int li = 0);
// Backward sweep for one level: x_s = U11^-1 (z - U12 x_b), stored into y.
template <typename T>
cudaError_t launch_solve_bwd_level_impl(const FrontDev *fr, int lo, int nfront, int max_s, int max_f, const T *fronts,
                                        const T *dinv, const int32_t *idx, T *y, int64_t ldy, int nrhs, T *work,
                                        T *zbuf, const int64_t *work_off, cudaStream_t s, Prof *prof, double bytes,
                                        const ChainArgs *ca = nullptr, int li = 0);

// FP32 trailing update C -= L21 U12 of one panel step on the tensor cores
// (gemm_tc.cu), over the 128-column tiles [tile_lo, tile_hi) of the trailing
// block, sized for about sm_budget SMs.
// With `maps` (one TMA descriptor per front of the launch, make_front_tmaps),
// fronts with a full 64-column panel move their C tiles by TMA; any_full /
// any_partial say which kinds of front the step has.
constexpr int kTmapBytes = 128;
cudaError_t launch_gemm_tc(const FrontDev *fr, int j0, int nfront, int max_f, float *fronts, int *err,
                           cudaStream_t s, int tile_lo, int tile_hi, int sm_budget, const uint8_t *maps,
                           bool any_full, bool any_partial);
// Blocked FP32 LU (kb-column outer blocks of 64-column panels):
// inner step at panel j0: C -= L21 U12 on the columns left in the outer block
// only, [j0 + 64, min(J + kb, s)) with J = kb floor(j0 / kb); sym = 1 (block
// Cholesky): the B operand is L21^T, read from the panel columns;
cudaError_t launch_gemm_tc_inner(const FrontDev *fr, int j0, int kb, int nfront, int max_f, float *fronts, int *err,
                                 cudaStream_t s, int sm_budget, int sym = 0);
// block end at J = j0: C[t0:f, t0:f] -= L21 U12 with K = min(kb, s - j0)
// (t0 = j0 + K), over the 128-column tiles [tile_lo, tile_hi), from packed
// operands: k_pack_a writes L21 (the rows after the block, K = the block's
// columns) into apack, k_pack_b the U12 columns of tiles [ct_lo, ct_hi) of the
// trailing block into bpack; the warp-specialised GEMM streams both with bulk
// copies.  lower = 1 (block Cholesky, bpack = apack): only the tiles on and
// below the diagonal of the trailing block.
cudaError_t launch_pack_a(const FrontDev *fr, int j0, int kb, int nfront, int max_f, const float *fronts, float *apack,
                          cudaStream_t s);
cudaError_t launch_pack_b(const FrontDev *fr, int j0, int kb, int nfront, int max_f, const float *fronts, float *bpack,
                          int ct_lo, int ct_hi, cudaStream_t s);
cudaError_t launch_gemm_tc_ws(const FrontDev *fr, int j0, int kb, int nfront, int max_f, float *fronts, int *err,
                              cudaStream_t s, int tile_lo, int tile_hi, int sm_budget, const uint8_t *maps,
                              const float *apack, const float *bpack, int lower = 0, int max_tiles = 0,
                              const uint8_t *maps64 = nullptr, int bf16 = 0);
// The TF32 block-end update in 128 x 256 output tiles (pairs of packed
// column tiles of `bpack`; with `lower`, the block Cholesky's lower triangle
// with bpack = apack): k_gemm_tc_wide.
cudaError_t launch_gemm_tc_wide(const FrontDev *fr, int j0, int kb, int nfront, int max_f, float *fronts, int *err,
                                cudaStream_t s, int tile_lo, int tile_hi, int sm_budget, const float *apack,
                                const float *bpack, int lower, int max_tiles, const uint8_t *maps64, int reduce = 0);
// BF16 operands of the block-end update (block Cholesky): each 128-row tile of
// L21 scaled by a power of two and rounded to BF16 (mode 1), or split into a
// BF16 hi and lo part (mode 2); the exponent rides in the tile's slot of the
// pack buffer.  bf16 of launch_gemm_tc_ws takes the same mode.
cudaError_t launch_pack_bf16(const FrontDev *fr, int j0, int kb, int nfront, int max_f, const float *fronts,
                             float *pack, cudaStream_t s, int mode);
// one descriptor per front: 2D (rows, columns), boxes of 128 rows x box_cols columns
cudaError_t make_front_tmaps(const Front *fronts, int n, const float *base, uint8_t *maps_dev, int box_cols = 128);
constexpr int kTcTile = 128;

// ---- applies, H^2 product, vector kernels (apply.cu) ----
struct ApItem {
  int64_t q;      // Q offset (m x m)
  int64_t xin;    // offset of X_l(t) in the level-l vector (rows)
  int64_t yout;   // S-space row of the non-basis part, -1 if none
  int64_t xout;   // row in the level-(l+1) vector of the basis part, -1 if none
  int32_t m, kp;
};
// The level maps of the applies and the S node offsets built by the device
// level schedule (sched.cu): apply items of level l at ap + ap_base[l]
// (nap[l] of them), the top clusters' copies into S, node_off.  The buffers
// in `allocs` pass to the caller.
struct DeviceMaps {
  std::vector<void *> allocs;
  ApItem *ap = nullptr;
  std::vector<int32_t> ap_base, nap;
  int64_t *top_src = nullptr, *top_dst = nullptr;
  int32_t *top_len = nullptr;
  int ntop = 0;
  int64_t *node_off = nullptr;
};
// Runs the level schedule on the current device from the plan's (validated)
// structure arrays; host copies into *out, device level maps into *maps
// (either may be null).  Synchronous; returns an h2sp_status.
int device_schedule(const Plan &p, A1Result *out, DeviceMaps *maps, std::string &err);
// the message h2sp_last_cuda_error returns (this thread)
void set_last_error(const std::string &msg);

// ---- threshold incomplete LU of S (ilut.cu) ----
struct IlutFail {
  int st;
  std::string msg;
};
// The factors: rows in elimination order (row e is row perm[e] of S), each
// row's kept entries at pool offset row_off: nl L entries (columns below the
// row), then nu U entries starting with the diagonal, columns ascending.
struct IlutState {
  std::vector<void *> bufs;
  bool ready = false;
  int64_t n = 0, nnz = 0;
  double tau = 0.0;
  int32_t *perm = nullptr;
  int64_t *sn_row = nullptr, *row_off = nullptr;
  int32_t *nl = nullptr, *nu = nullptr;
  int32_t *pool_col = nullptr;
  double *pool_val = nullptr;
  unsigned long long *cursor = nullptr;
  int *err = nullptr;
  std::vector<std::pair<int, int>> levels;  // supernodes of each elimination level
  int grid = 1;
  void release();
  ~IlutState() { release(); }
};
// ILUt of the VBR S (values FP64, or FP32 when s_fp32) in the plan's
// elimination order; throws IlutFail.  Synchronous.
void ilut_factor(IlutState &st, const Plan &p, const int64_t *brow_ptr, const int32_t *bcol, const int64_t *val_off,
                 const int64_t *node_off, const void *S, bool s_fp32, double tau, cudaStream_t s, Prof *prof);
// y <- (L U)^-1 y in S order (ld n, nrhs columns); z: n x nrhs work
void ilut_solve(IlutState &st, double *y, int nrhs, double *z, cudaStream_t s, Prof *prof);

// out rows: non-basis -> S space (ys), basis -> next level (xn); op = Q^T.
// T = double (the API's applies) or float (inside the FP32 preconditioner).
// max_m: the level's largest block; above kMaxBlock the input slab is staged
// in dynamic shared memory.
template <typename T>
cudaError_t launch_apply_qt(const ApItem *items, int n, const T *Q, const T *x, int64_t ldx, T *ys, int64_t ldys, T *xn,
                            int64_t ldxn, int nrhs, cudaStream_t s, int max_m);
// reverse: X_l(t) = Q [xn part; ys part]
template <typename T>
cudaError_t launch_apply_q(const ApItem *items, int n, const T *Q, const T *xn, int64_t ldxn, const T *ys, int64_t ldys,
                           T *x, int64_t ldx, int nrhs, cudaStream_t s, int max_m);
// copy rows: dst[dst_row[i] + r] = src[src_row[i] + r] for r < len[i]
template <typename T>
cudaError_t launch_copy_rows(const int64_t *src_row, const int64_t *dst_row, const int32_t *len, int n, const T *src,
                             int64_t lds, T *dst, int64_t ldd, int nrhs, cudaStream_t s);
// y = S x (VBR; values of type TS, FP64 vectors and sums)
template <typename TS>
cudaError_t launch_spmv(const int64_t *brow_ptr, const int32_t *bcol, const int64_t *val_off, const int64_t *node_off,
                        int nnodes, const TS *vals, const double *x, int64_t ldx, double *y, int64_t ldy, int nrhs,
                        cudaStream_t s);

struct H2Dev {
  // device copies of the structure
  const int64_t *begin, *size;
  const int32_t *rank, *parent;
  const int64_t *leaf_basis_off, *transfer_off, *coupling_off, *near_off;
  const int64_t *col_leaf_basis_off, *col_transfer_off;
  const int64_t *far_ptr, *near_ptr;
  const int32_t *far_col, *near_col;
  const int64_t *xh_off;
  const double *leaf_basis, *transfer, *coupling, *near_block, *col_leaf_basis, *col_transfer;
  // launch order of the close-block and coupling CTAs: heaviest first, so that
  // the last wave is made of the lightest clusters
  const int32_t *leaf_order, *couple_order;
  int32_t leaf0;  // first leaf cluster
  // leaves with more than 64 points come last in leaf_order and take the
  // close-block kernel that loops over row groups
  int32_t nleaf_large;
  int32_t max_leaf;  // largest leaf (points); up to 128 admits the few-right-hand-side kernels
};
// y = A x with A of Definition 4.9 (upward pass, couplings, downward pass, close blocks);
// xh / yh: coefficient workspaces with leading dimension ldh (>= sum of ranks), 16 columns
cudaError_t launch_h2_matvec(const H2Dev &h, const int32_t *level_ptr_host, const int32_t *child_start,
                             const int32_t *child_cnt, int depth, const double *x, int64_t ldx, double *y,
                             int64_t ldy, int nrhs, double *xh, double *yh, int64_t ldh, cudaStream_t s);

// Size (doubles) of the static device workspace of h2sp_h2_matvec_static (16 MiB).
constexpr int64_t kStaticScratchElems = int64_t(1) << 21;
// Device address of that workspace on the current device (looked up once per device).
cudaError_t static_scratch_address(double **out);

// r = b - y; norms2[seg * nrhs + c] = ||r_c||^2 over the rows [seg_ptr[seg], seg_ptr[seg+1])
cudaError_t launch_residual(const double *b, int64_t ldb, const double *y, int64_t ldy, double *r, int64_t ldr,
                            const int64_t *seg_ptr, int nseg, int64_t n, int nrhs, double *norms2, cudaStream_t s);
cudaError_t launch_colnorm2(const double *x, int64_t ldx, const int64_t *seg_ptr, int nseg, int64_t n, int nrhs,
                            double *norms2, cudaStream_t s);
// GMRES helpers: out[i*nrhs + c] = <V_i[:,c], W[:,c]> for i < nv (V_i at V + i * vstride);
// W[:,c] += sum_i coef[i*nrhs + c] V_i[:,c]; X[:,c] *= sc[c]  (coefficients on the device)
cudaError_t launch_block_dots(const double *V, int64_t ldv, int64_t vstride, int nv, const double *W, int64_t ldw,
                              int64_t n, int nrhs, double *out, cudaStream_t s);
cudaError_t launch_block_axpy(const double *V, int64_t ldv, int64_t vstride, int nv, const double *coef, double *W,
                              int64_t ldw, int64_t n, int nrhs, cudaStream_t s);
cudaError_t launch_col_scale(double *X, int64_t ldx, const double *sc, int64_t n, int nrhs, cudaStream_t s);
// x += d
cudaError_t launch_axpy(const double *d, int64_t ldd, double *x, int64_t ldx, int64_t n, int nrhs, cudaStream_t s);
cudaError_t launch_cast_d2f(const double *a, int64_t lda, float *b, int64_t ldb, int64_t n, int nrhs, cudaStream_t s);
cudaError_t launch_cast_f2d(const float *a, int64_t lda, double *b, int64_t ldb, int64_t n, int nrhs, cudaStream_t s);

}  // namespace h2sp
