// The C ABI of h2sp (include/h2sp.h): handle management and the host-side
// orchestration of the kernels for h2sp_sparsify, h2sp_factor, h2sp_solve and
// h2sp_apply.  All device memory the handle owns comes from cudaMallocAsync on
// the call's stream; the numeric arrays of the H^2 descriptor are borrowed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "kernels.h"

using namespace h2sp;

namespace {

thread_local std::string g_cuda_err;

struct CudaFail {
  cudaError_t e;
};

// cudaMallocAsync that, when the device is out of memory, returns the memory
// the current device's pool keeps from freed buffers (the pool is set to
// keep it between calls) and tries once more.
cudaError_t malloc_async(void **p, size_t bytes, cudaStream_t s) {
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaErrorMemoryAllocation) return e;
  cudaGetLastError();
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
    cudaGetLastError();
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, s);
}

inline void ck(cudaError_t e) {
  if (e != cudaSuccess) {
    g_cuda_err = cudaGetErrorString(e);
    throw CudaFail{e};
  }
}

int status_of(cudaError_t e) { return e == cudaErrorMemoryAllocation ? H2SP_ENOMEM : H2SP_ECUDA; }

struct LevelDev {
  QItem *q = nullptr, *qc = nullptr;
  WItem *w = nullptr, *wc = nullptr;
  CItem *c = nullptr;
  XItem *x = nullptr;
  int nq = 0, nw = 0, nc = 0, nx = 0;
  int nq_small = 0, nx_small = 0;  // small items (blocks <= kMaxBlock) lead q / qc and x
  int max_m = 0;                   // largest block of the level (Householder and apply items)
  int max_xr = 0, max_xc = 0;      // largest rows / cols of the level's large transform items
  void **src_base = nullptr, **dst_base = nullptr;  // device arrays of 4 pointers
  double *W = nullptr, *Wc = nullptr;
  ApItem *ap = nullptr;  // applies of this level's Q blocks
  int nap = 0;
};

struct FrontLevel {
  int lo, hi, max_s, max_f, max_b;
  double b2 = 0.0;       // sum of b^2 (contribution elements) over the level's fronts
  double lu_elems = 0.0; // sum of s^2/2 + s*b (factor elements one sweep reads)
};

// Device copies of everything the numeric phases read that depends only on
// the structure (work items of every level, apply items, the VBR index of S,
// the H^2 index arrays, fronts, extend-add maps, assembly items, sweep work
// lists).  Built once per analysis, on the first numeric sparsification, and
// shared by every handle planned from it; freed with the last of them.
struct StructureDev {
  int device = -1;
  std::vector<void *> allocs;
  std::vector<LevelDev> lv;  // item arrays only
  std::vector<double> x_flops, x_flops_large;  // transform flops of each level's small / large items
  int max_rank = 1;
  int64_t max_pack_tiles = 0;  // largest sum over a level's fronts of ceil(f / 128)
  int64_t max_width = 0;
  int64_t *top_src = nullptr, *top_dst = nullptr;
  int32_t *top_len = nullptr;
  int ntop = 0;
  int64_t *brow_ptr = nullptr, *val_off = nullptr, *node_off = nullptr;
  int32_t *bcol = nullptr;
  H2Dev h2{};  // structure pointers only
  int32_t *child_start = nullptr, *child_cnt = nullptr;
  double near_bytes = 0.0, mv_flops_per_rhs = 0.0;
  int64_t *seg_ptr = nullptr;
  int nseg = 1;
  FrontDev *fr = nullptr;
  int32_t *fidx = nullptr, *fmap = nullptr;
  AItem *asm_items = nullptr;
  int max_s_all = 0;
  std::vector<FrontLevel> flev;
  int2 *chain_items = nullptr;
  std::vector<int> chain_fwd_off, chain_fwd_n, chain_bwd_off, chain_bwd_n;
  int nflags = 0;
  template <class T>
  T *upload(const std::vector<T> &v) {
    void *d = nullptr;
    ck(cudaMalloc(&d, std::max<size_t>(v.size(), 1) * sizeof(T)));
    allocs.push_back(d);
    if (!v.empty()) ck(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return static_cast<T *>(d);
  }
  ~StructureDev() {
    for (void *q : allocs) cudaFree(q);
  }
};

// the shared slot of one analysis
struct StructureCell {
  std::mutex m;
  std::shared_ptr<StructureDev> dev;
};

}  // namespace

struct h2sp_handle {
  std::shared_ptr<const Plan> plan_ptr;  // host analysis, shared with the handles planned from it
  std::shared_ptr<StructureCell> cell;   // its device copy (filled on first use), shared likewise
  std::shared_ptr<StructureDev> sdev;    // kept alive while this handle lives
  uint64_t structure_hash = 0;          // fingerprint of the descriptor's structure arrays
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  // borrowed H^2 numbers
  const double *leaf_basis = nullptr, *transfer = nullptr, *coupling = nullptr, *near_block = nullptr;
  const double *col_leaf_basis = nullptr, *col_transfer = nullptr;
  // sparsification: Q and R are FP64; S and the level buffers that feed it
  // hold doubles, or floats when sp_prec is H2SP_FP32
  int sp_prec = H2SP_FP64;
  double *Q = nullptr, *Qc = nullptr, *Rr = nullptr, *Rrc = nullptr;
  void *S = nullptr;
  std::vector<void *> Cbuf, RPbuf, CPbuf;
  std::vector<LevelDev> lv;
  // applies
  int64_t *top_src = nullptr, *top_dst = nullptr;
  int32_t *top_len = nullptr;
  int ntop = 0;
  int64_t max_width = 0;
  double *vecA = nullptr, *vecB = nullptr, *vecS = nullptr, *vecT = nullptr, *vecR = nullptr;
  int vec_rhs = 0;
  // S structure for products
  int64_t *brow_ptr = nullptr, *val_off = nullptr, *node_off = nullptr;
  int32_t *bcol = nullptr;
  // factor
  int prec = -1;
  void *fronts = nullptr;
  size_t fronts_esz = 0;  // element size the front buffer is sized for (4: FP32 fronts only, 8: either)
  FrontDev *fr = nullptr;
  int32_t *piv = nullptr, *perm = nullptr, *swaps = nullptr, *fidx = nullptr, *fmap = nullptr;
  AItem *asm_items = nullptr;
  int *err = nullptr;
  int compensated = 0;  // pivots the last factorization compensated (BF16 block-end modes)
  std::vector<FrontLevel> flev;
  int max_s_all = 0;
  int64_t *work_off = nullptr;
  void *work = nullptr, *zbuf = nullptr, *dinv = nullptr;
  float *yf = nullptr;
  // FP32 preconditioner: Q rounded to FP32, apply work vectors and the input
  float *Qf = nullptr, *Qcf = nullptr, *vecAf = nullptr, *vecBf = nullptr, *rf = nullptr;
  int vecf_rhs = 0;
  int work_rhs = 0;
  // H^2 product
  H2Dev h2{};
  int32_t *child_start = nullptr, *child_cnt = nullptr;
  double *xh = nullptr, *yh = nullptr;
  double *norms = nullptr;
  double *gmV = nullptr, *gmZ = nullptr, *gmW = nullptr, *gmC = nullptr;  // GMRES basis and workspace
  int gm_m = 0, gm_rhs = 0;
  int64_t *seg_ptr = nullptr;  // row ranges of the independent systems (roots)
  int nseg = 1;
  double plan_seconds = 0.0;
  bool device_ready = false;
  Prof prof;
  std::vector<double> x_flops, x_flops_large;  // algorithmic flops of each level's transform launches
  double near_bytes = 0.0;      // bytes of the close blocks (Definition 4.8)
  double mv_flops_per_rhs = 0.0;  // FP64 flops of one H^2 product per right-hand side

  template <class T>
  T *alloc(size_t n) {
    if (n == 0) n = 1;
    void *p = nullptr;
    ck(malloc_async(&p, n * sizeof(T), stream));
    allocs.push_back(p);
    return static_cast<T *>(p);
  }
  template <class T>
  T *upload(const std::vector<T> &v) {
    T *d = alloc<T>(v.size());
    if (!v.empty()) ck(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream));
    return d;
  }
  // free one buffer of `allocs` before the handle is released
  void free_one(void *p) {
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i] == p) {
        cudaFreeAsync(p, stream);
        allocs.erase(allocs.begin() + long(i));
        return;
      }
  }
  LuAsync la;  // look-ahead stream and events of the block LU (created on first use)
  uint8_t *tmaps = nullptr;  // TMA descriptors of the FP32 fronts (built on the first FP32 factorization)
  uint8_t *tmaps_buf = nullptr;     // their device storage
  uint8_t *tmaps64 = nullptr;       // the same fronts with 128 x 64 boxes (the block-end update's C halves)
  const void *tmaps_base = nullptr;  // the front buffer they were encoded for
  float *pack = nullptr;     // packed GEMM operands of the blocked FP32 LU (3 buffers of the largest level)
  int32_t last_prec = -1;    // h2sp_prec of the last h2sp_factor (h2sp_refactor repeats it)
  bool chol = false;         // the current factors come from the block Cholesky (stored in the LU form)
  bool ilut = false;         // the current factors are the threshold incomplete LU (ilu)
  IlutState ilu;
  double *ilu_z = nullptr;   // n x ilu_z_rhs work of the incomplete factors' solves
  int ilu_z_rhs = 0;
  double *chol_inv = nullptr;  // L11^-1 tiles of the block Cholesky's panels (one per front of a level)
  cudaGraphExec_t graph_exec = nullptr;  // sparsification + factorization, captured by h2sp_refactor
  cudaStream_t graph_stream = nullptr;    // the graph is captured and launched here (the caller's may be legacy)
  cudaEvent_t graph_in = nullptr, graph_out = nullptr;
  // h2sp_solve_captured: its graph and the arguments it was captured for
  cudaGraphExec_t solve_exec = nullptr;
  const double *cap_b = nullptr;
  double *cap_x = nullptr;
  int64_t cap_ldb = 0, cap_ldx = 0;
  int cap_nrhs = 0, cap_steps = -1, cap_prec = -1;
  double *cap_norms = nullptr;  // ||b||^2 and ||b - A x||^2 per (system, right-hand side)
  // flag-synchronised triangular sweeps
  int2 *chain_items = nullptr;
  std::vector<int> chain_fwd_off, chain_fwd_n, chain_bwd_off, chain_bwd_n;
  int *chain_tickets = nullptr, *chain_flags = nullptr, *serr = nullptr;
  int chain_epoch = 0;
  uint32_t chain_spin_cap = 1u << 22;  // H2SP_OPTION_WAIT_POLLS
  bool test_stale_epoch = false;       // H2SP_OPTION_TEST_STALE_EPOCH: the next solve's forward waits never end
  CholSchedule chol_sched;             // H2SP_OPTION_CHOL_*: schedule of the blocked FP32 block Cholesky
  // log-determinant: fronts of each independent system (CSR) and per-front / per-system sums
  int32_t *ld_sys_ptr = nullptr, *ld_sys_front = nullptr, *ld_sign = nullptr;
  int *ld_flips = nullptr;
  double *ld_lsum = nullptr, *ld_out = nullptr;
  void release() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
    if (solve_exec) cudaGraphExecDestroy(solve_exec);
    solve_exec = nullptr;
    if (graph_stream) cudaStreamSynchronize(graph_stream);
    if (graph_in) cudaEventDestroy(graph_in);
    if (graph_out) cudaEventDestroy(graph_out);
    if (graph_stream) cudaStreamDestroy(graph_stream);
    graph_stream = nullptr;
    graph_in = graph_out = nullptr;
    if (la.side) cudaStreamSynchronize(la.side);
    if (la.rest) cudaStreamSynchronize(la.rest);
    if (la.next) cudaEventDestroy(la.next);
    if (la.panel) cudaEventDestroy(la.panel);
    if (la.done) cudaEventDestroy(la.done);
    if (la.side) cudaStreamDestroy(la.side);
    if (la.rest) cudaStreamDestroy(la.rest);
    la = LuAsync();
    if (allocs.empty()) return;
    for (void *p : allocs) cudaFreeAsync(p, stream);
    allocs.clear();
    cudaStreamSynchronize(stream);
  }
};

namespace {

// FP32 trailing updates with a full panel move their C tiles by TMA;
// H2SP_GEMM_TMA=0 keeps them on thread loads and stores.
bool tma_enabled() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_GEMM_TMA");
    v = (e && std::strcmp(e, "0") == 0) ? 0 : 1;
  }
  return v == 1;
}

// The next panel is factored on a side stream while the trailing update runs;
// H2SP_LOOKAHEAD=0 keeps every step on the caller's stream.
bool lookahead_enabled() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_LOOKAHEAD");
    v = (e && std::strcmp(e, "0") == 0) ? 0 : 1;
  }
  return v == 1;
}

void init_pool_once() {
  // once per device: keep freed memory in that device's default pool
  static std::mutex mu;
  static bool done[128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  done[dev] = true;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed memory in the pool between calls of this process
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
}

// ---------------- vectors of the applies ----------------
void ensure_vectors(h2sp_handle *h, int nrhs) {
  if (h->vec_rhs >= nrhs) return;
  const int64_t n = (*h->plan_ptr).n;
  const int64_t w = std::max<int64_t>(h->max_width, n);
  h->vecA = h->alloc<double>(size_t(w) * nrhs);
  h->vecB = h->alloc<double>(size_t(w) * nrhs);
  h->vecS = h->alloc<double>(size_t(n) * nrhs);
  h->vecT = h->alloc<double>(size_t(n) * nrhs);
  h->vecR = h->alloc<double>(size_t(n) * nrhs);
  h->vec_rhs = nrhs;
}

// out (S space, ld n) = Q^T in (point space) with the blocks Qb of one side
template <typename T>
void apply_T_impl(h2sp_handle *h, const T *Qb, const T *in, int64_t ldin, T *out, int64_t ldout, int nrhs, T *bufA,
                  T *bufB) {
  const Plan &p = (*h->plan_ptr);
  cudaStream_t s = h->stream;
  const int chunks = (nrhs + 15) / 16;
  const size_t e0 = h->prof.begin();
  struct Done {
    h2sp_handle *h;
    size_t e0;
    int n;
    ~Done() { h->prof.end(P_APPLY, n, e0, 0.0); }
  } done{h, e0, 1 + p.lstop * chunks};
  if (p.lstop == 0) {
    ck(launch_copy_rows(h->top_src, h->top_dst, h->top_len, h->ntop, in, ldin, out, ldout, nrhs, s));
    return;
  }
  const int64_t ldw = std::max<int64_t>(h->max_width, p.n);
  const T *x = in;
  int64_t ldx = ldin;
  T *bufs[2] = {bufA, bufB};
  for (int l = 0; l < p.lstop; ++l) {
    T *xn = bufs[l & 1];
    ck(launch_apply_qt(h->lv[l].ap, h->lv[l].nap, Qb, x, ldx, out, ldout, xn, ldw, nrhs, s, h->lv[l].max_m));
    x = xn;
    ldx = ldw;
  }
  ck(launch_copy_rows(h->top_src, h->top_dst, h->top_len, h->ntop, x, ldx, out, ldout, nrhs, s));
}

// out (point space) = Q in (S space) with the blocks Qb of one side
template <typename T>
void apply_N_impl(h2sp_handle *h, const T *Qb, const T *in, int64_t ldin, T *out, int64_t ldout, int nrhs, T *bufA,
                  T *bufB) {
  const Plan &p = (*h->plan_ptr);
  cudaStream_t s = h->stream;
  const int chunks = (nrhs + 15) / 16;
  const size_t e0 = h->prof.begin();
  struct Done {
    h2sp_handle *h;
    size_t e0;
    int n;
    ~Done() { h->prof.end(P_APPLY, n, e0, 0.0); }
  } done{h, e0, 1 + p.lstop * chunks};
  if (p.lstop == 0) {
    ck(launch_copy_rows(h->top_dst, h->top_src, h->top_len, h->ntop, in, ldin, out, ldout, nrhs, s));
    return;
  }
  const int64_t ldw = std::max<int64_t>(h->max_width, p.n);
  T *bufs[2] = {bufA, bufB};
  T *xn = bufs[p.lstop & 1];
  ck(launch_copy_rows(h->top_dst, h->top_src, h->top_len, h->ntop, in, ldin, xn, ldw, nrhs, s));
  for (int l = p.lstop - 1; l >= 0; --l) {
    T *x = (l == 0) ? out : bufs[l & 1];
    const int64_t ldx = (l == 0) ? ldout : ldw;
    ck(launch_apply_q(h->lv[l].ap, h->lv[l].nap, Qb, xn, ldw, in, ldin, x, ldx, nrhs, s, h->lv[l].max_m));
    xn = x;
  }
}

// out (S space, ld n) = Qside^T in (point space)
void apply_T(h2sp_handle *h, bool col, const double *in, int64_t ldin, double *out, int64_t ldout, int nrhs) {
  apply_T_impl<double>(h, col ? h->Qc : h->Q, in, ldin, out, ldout, nrhs, h->vecA, h->vecB);
}

// out (point space) = Qside in (S space)
void apply_N(h2sp_handle *h, bool col, const double *in, int64_t ldin, double *out, int64_t ldout, int nrhs) {
  apply_N_impl<double>(h, col ? h->Qc : h->Q, in, ldin, out, ldout, nrhs, h->vecA, h->vecB);
}

void h2_matvec(h2sp_handle *h, const double *x, int64_t ldx, double *y, int64_t ldy, int nrhs) {
  const Plan &p = (*h->plan_ptr);
  const size_t e0 = h->prof.begin();
  ck(launch_h2_matvec(h->h2, p.level_ptr.data(), h->child_start, h->child_cnt, p.D, x, ldx, y, ldy, nrhs, h->xh,
                      h->yh, std::max<int64_t>(p.xh_elems, 1), h->stream));
  const int chunks = (nrhs + 15) / 16;
  // FP64 flops: the product is bound by the FP64 pipe
  h->prof.end(P_MATVEC, (3 + 2 * p.D) * chunks, e0, h->mv_flops_per_rhs * nrhs);
}

// per-front work vectors of the triangular solves, for 16 right-hand sides at a time
constexpr int kSolveRhs = 16;
void ensure_work(h2sp_handle *h, int nrhs) {
  if (h->work_off == nullptr) {
    const Plan &p = (*h->plan_ptr);
    std::vector<int64_t> off(p.fronts.size());
    int64_t acc = 0;
    for (size_t k = 0; k < p.fronts.size(); ++k) {
      off[k] = acc;
      acc += int64_t(p.fronts[k].f) * kSolveRhs;
    }
    h->work_off = h->upload(off);
    h->work = h->alloc<double>(size_t(std::max<int64_t>(acc, 1)));
    h->zbuf = h->alloc<double>(size_t(std::max<int64_t>(acc, 1)));
  }
  if (h->work_rhs < nrhs) {
    h->yf = h->alloc<float>(size_t((*h->plan_ptr).n) * nrhs);
    h->work_rhs = nrhs;
  }
}

// y (S space, type T, ld n) <- S^{-1} y with the current factors
// Triangular sweeps with one flag-synchronised launch per level and direction;
// H2SP_SOLVE=steps launches one kernel per kSolveBlock-column step instead.
bool chain_sweeps_enabled() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_SOLVE");
    v = (e && std::strcmp(e, "steps") == 0) ? 0 : 1;
  }
  return v == 1;
}

template <typename T>
void solve_S_T(h2sp_handle *h, T *y, int nrhs) {
  const Plan &p = (*h->plan_ptr);
  T *fronts = static_cast<T *>(h->fronts);
  T *work = static_cast<T *>(h->work);
  T *zbuf = static_cast<T *>(h->zbuf);
  const T *dinv = static_cast<const T *>(h->dinv);
  const bool chain = chain_sweeps_enabled();
  ChainArgs ca;
  ca.items = h->chain_items;
  ca.fwd_off = h->chain_fwd_off.data();
  ca.fwd_n = h->chain_fwd_n.data();
  ca.bwd_off = h->chain_bwd_off.data();
  ca.bwd_n = h->chain_bwd_n.data();
  ca.tickets = h->chain_tickets;
  ca.flags = h->chain_flags;
  ca.err = h->serr;
  ca.spin_cap = h->chain_spin_cap;
  // the wait test: the forward sweeps await an epoch that no block publishes
  const int stale = h->test_stale_epoch ? (1 << 29) : 0;
  h->test_stale_epoch = false;
  for (int r0 = 0; r0 < nrhs; r0 += kSolveRhs) {
    const int nr = std::min(kSolveRhs, nrhs - r0);
    T *yr = y + int64_t(r0) * p.n;
    if (chain) {
      ck(cudaMemsetAsync(h->chain_tickets, 0, sizeof(int) * 2 * h->flev.size(), h->stream));
      h->prof.count(P_OTHER, 1);
    }
    for (size_t li = 0; li < h->flev.size(); ++li) {
      const FrontLevel &L = h->flev[li];
      ca.epoch = ++h->chain_epoch;
      ca.wait_epoch = ca.epoch + stale;
      ck(launch_solve_fwd_level_impl<T>(h->fr, L.lo, L.hi - L.lo, L.max_s, L.max_f, fronts, dinv, h->perm, h->fidx,
                                        yr, p.n, nr, work, zbuf, h->work_off, h->stream, &h->prof,
                                        L.lu_elems * sizeof(T), chain ? &ca : nullptr, int(li)));
    }
    for (int i = int(h->flev.size()) - 1; i >= 0; --i) {
      const FrontLevel &L = h->flev[i];
      ca.epoch = ++h->chain_epoch;
      ca.wait_epoch = ca.epoch;
      ck(launch_solve_bwd_level_impl<T>(h->fr, L.lo, L.hi - L.lo, L.max_s, L.max_f, fronts, dinv, h->fidx, yr, p.n,
                                        nr, work, zbuf, h->work_off, h->stream, &h->prof, L.lu_elems * sizeof(T),
                                        chain ? &ca : nullptr, i));
    }
  }
}

// status of the sweeps since the last check (a bounded wait that ran out)
int sweep_status(h2sp_handle *h) {
  int e = 0;
  ck(cudaMemcpyAsync(&e, h->serr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  ck(cudaStreamSynchronize(h->stream));
  if (e != 0) {
    ck(cudaMemsetAsync(h->serr, 0, sizeof(int), h->stream));
    return H2SP_ETIMEOUT;
  }
  return H2SP_OK;
}

// in-place S^{-1} on an FP64 S-space vector (ld n)
void solve_S(h2sp_handle *h, double *y, int nrhs) {
  const int64_t n = (*h->plan_ptr).n;
  if (h->ilut) {
    // the incomplete factors: (L U)^{-1}
    if (h->ilu_z_rhs < nrhs) {
      h->ilu_z = h->alloc<double>(size_t(n) * size_t(nrhs));
      h->ilu_z_rhs = nrhs;
    }
    ilut_solve(h->ilu, y, nrhs, h->ilu_z, h->stream, &h->prof);
    return;
  }
  ensure_work(h, nrhs);
  if (h->prec == H2SP_FP64) {
    solve_S_T<double>(h, y, nrhs);
  } else {
    ck(launch_cast_d2f(y, n, h->yf, n, n, nrhs, h->stream));
    solve_S_T<float>(h, h->yf, nrhs);
    ck(launch_cast_f2d(h->yf, n, y, n, n, nrhs, h->stream));
    h->prof.count(P_OTHER, 2);
  }
}

// The FP32 factors are applied with FP32 U^T and V (Q rounded to FP32) and
// FP32 vectors; H2SP_PRECOND=fp64 keeps the FP64 applies around them.
bool fp32_applies_enabled() {
  static int v = -1;
  if (v < 0) {
    const char *e = std::getenv("H2SP_PRECOND");
    v = (e && std::strcmp(e, "fp64") == 0) ? 0 : 1;
  }
  return v == 1;
}

void ensure_vectors_f32(h2sp_handle *h, int nrhs) {
  const Plan &p = (*h->plan_ptr);
  if (h->Qf == nullptr) {
    const int64_t q = std::max<int64_t>(p.q_elems, 1);
    h->Qf = h->alloc<float>(size_t(q));
    ck(launch_cast_d2f(h->Q, q, h->Qf, q, q, 1, h->stream));
    if (p.sym) {
      h->Qcf = h->Qf;
    } else {
      h->Qcf = h->alloc<float>(size_t(q));
      ck(launch_cast_d2f(h->Qc, q, h->Qcf, q, q, 1, h->stream));
    }
  }
  if (h->vecf_rhs < nrhs) {
    const int64_t w = std::max<int64_t>(h->max_width, p.n);
    h->vecAf = h->alloc<float>(size_t(w) * nrhs);
    h->vecBf = h->alloc<float>(size_t(w) * nrhs);
    h->rf = h->alloc<float>(size_t(p.n) * nrhs);
    h->vecf_rhs = nrhs;
  }
}

// d = V S^{-1} U^T r   (the direct solve of Eq. sp0)
void precond(h2sp_handle *h, const double *r, int64_t ldr, double *d, int64_t ldd, int nrhs) {
  const int64_t n = (*h->plan_ptr).n;
  if (h->prec == H2SP_FP32 && fp32_applies_enabled()) {
    // all of M^{-1} in FP32: the FP64 residual around it decides convergence
    ensure_work(h, nrhs);
    ensure_vectors_f32(h, nrhs);
    ck(launch_cast_d2f(r, ldr, h->rf, n, n, nrhs, h->stream));
    apply_T_impl<float>(h, h->Qf, h->rf, n, h->yf, n, nrhs, h->vecAf, h->vecBf);
    solve_S_T<float>(h, h->yf, nrhs);
    apply_N_impl<float>(h, h->Qcf, h->yf, n, h->rf, n, nrhs, h->vecAf, h->vecBf);
    ck(launch_cast_f2d(h->rf, n, d, ldd, n, nrhs, h->stream));
    h->prof.count(P_OTHER, 2);
    return;
  }
  apply_T(h, false, r, ldr, h->vecS, n, nrhs);
  solve_S(h, h->vecS, nrhs);
  apply_N(h, true, h->vecS, n, d, ldd, nrhs);
}

// Restarted GMRES with right preconditioning M^{-1} = V S^{-1} U^T (§5.5), one
// Krylov process per right-hand side, all columns advanced together.  The
// basis is orthogonalised by classical Gram-Schmidt applied twice; the small
// Hessenberg least-squares problems (Givens rotations) are solved on the host.
// Convergence is judged on the Hessenberg estimate inside a cycle and on the
// true FP64 H^2 residual (per independent system and column) at its end.
int gmres(h2sp_handle *h, const h2sp_solve_opts *o, int nrhs, const double *b, int64_t ldb, double *x, int64_t ldx,
          h2sp_solve_info *info) {
  const Plan &p = (*h->plan_ptr);
  cudaStream_t s = h->stream;
  const int64_t n = p.n;
  const int m = std::max(1, std::min(o->restart > 0 ? o->restart : 20, 60));
  const int maxit = o->maxit > 0 ? o->maxit : 200;
  const int ns = h->nseg;
  if (h->gm_m < m || h->gm_rhs < nrhs) {
    h->gmV = h->alloc<double>(size_t(m + 1) * n * nrhs);
    h->gmZ = h->alloc<double>(size_t(m) * n * nrhs);
    h->gmW = h->alloc<double>(size_t(n) * nrhs);
    h->gmC = h->alloc<double>(size_t(m + 2) * nrhs);
    h->gm_m = m;
    h->gm_rhs = nrhs;
  }
  const int64_t vs = n * nrhs;  // stride between basis blocks (ld n)
  double *V = h->gmV, *Z = h->gmZ, *W = h->gmW, *C = h->gmC;
  std::vector<double> bn2(size_t(nrhs) * ns), rn2(size_t(nrhs) * ns), bnorm(nrhs), beta(nrhs);
  ck(launch_colnorm2(b, ldb, h->seg_ptr, ns, n, nrhs, h->norms, s));
  ck(cudaMemcpyAsync(bn2.data(), h->norms, sizeof(double) * nrhs * ns, cudaMemcpyDeviceToHost, s));
  ck(cudaStreamSynchronize(s));
  for (int c = 0; c < nrhs; ++c) {
    double t = 0.0;
    for (int q = 0; q < ns; ++q) t += bn2[size_t(q) * nrhs + c];
    bnorm[c] = std::sqrt(std::max(t, 1e-300));
  }
  for (int c = 0; c < nrhs; ++c) ck(cudaMemsetAsync(x + c * ldx, 0, sizeof(double) * n, s));
  int it = 0;
  double res = INFINITY;
  std::vector<double> H(size_t(m + 1) * m * nrhs), cs(size_t(m) * nrhs), sn(size_t(m) * nrhs), g(size_t(m + 1) * nrhs);
  std::vector<double> hcol(size_t(m + 2) * nrhs), coef(size_t(m + 1) * nrhs);
  auto Hat = [&](int i, int j, int c) -> double & { return H[(size_t(c) * (m + 1) + i) * m + j]; };
  for (;;) {
    // r = b - A x into V_0, true residual per system and column
    h2_matvec(h, x, ldx, W, n, nrhs);
    ck(launch_residual(b, ldb, W, n, V, n, h->seg_ptr, ns, n, nrhs, h->norms, s));
    ck(cudaMemcpyAsync(rn2.data(), h->norms, sizeof(double) * nrhs * ns, cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    res = 0.0;
    for (size_t q = 0; q < rn2.size(); ++q) res = std::max(res, std::sqrt(rn2[q] / std::max(bn2[q], 1e-300)));
    if (!(res > o->tol) || it >= maxit) break;
    std::vector<double> scale(nrhs);
    for (int c = 0; c < nrhs; ++c) {
      double t = 0.0;
      for (int q = 0; q < ns; ++q) t += rn2[size_t(q) * nrhs + c];
      beta[c] = std::sqrt(t);
      scale[c] = beta[c] > 0.0 ? 1.0 / beta[c] : 0.0;
    }
    ck(cudaMemcpyAsync(C, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    ck(launch_col_scale(V, n, C, n, nrhs, s));
    std::fill(g.begin(), g.end(), 0.0);
    for (int c = 0; c < nrhs; ++c) g[size_t(c) * (m + 1)] = beta[c];
    int j = 0;
    for (; j < m && it < maxit; ++j, ++it) {
      precond(h, V + j * vs, n, Z + j * vs, n, nrhs);
      h2_matvec(h, Z + j * vs, n, W, n, nrhs);
      // classical Gram-Schmidt, twice
      std::fill(hcol.begin(), hcol.end(), 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        ck(launch_block_dots(V, n, vs, j + 1, W, n, n, nrhs, C, s));
        ck(cudaMemcpyAsync(coef.data(), C, sizeof(double) * (j + 1) * nrhs, cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        for (size_t q = 0; q < size_t(j + 1) * nrhs; ++q) {
          hcol[q] += coef[q];
          coef[q] = -coef[q];
        }
        ck(cudaMemcpyAsync(C, coef.data(), sizeof(double) * (j + 1) * nrhs, cudaMemcpyHostToDevice, s));
        ck(launch_block_axpy(V, n, vs, j + 1, C, W, n, n, nrhs, s));
      }
      ck(launch_colnorm2(W, n, h->seg_ptr, ns, n, nrhs, h->norms, s));
      ck(cudaMemcpyAsync(rn2.data(), h->norms, sizeof(double) * nrhs * ns, cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));
      std::vector<double> inv(nrhs);
      double worst = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        double t = 0.0;
        for (int q = 0; q < ns; ++q) t += rn2[size_t(q) * nrhs + c];
        const double hn = std::sqrt(t);
        for (int i = 0; i <= j; ++i) Hat(i, j, c) = hcol[size_t(i) * nrhs + c];
        double hj1 = hn;
        inv[c] = hn > 0.0 ? 1.0 / hn : 0.0;
        // apply the previous rotations, then a new one
        for (int i = 0; i < j; ++i) {
          const double a0 = Hat(i, j, c), a1 = Hat(i + 1, j, c);
          Hat(i, j, c) = cs[size_t(c) * m + i] * a0 + sn[size_t(c) * m + i] * a1;
          Hat(i + 1, j, c) = -sn[size_t(c) * m + i] * a0 + cs[size_t(c) * m + i] * a1;
        }
        const double a0 = Hat(j, j, c);
        const double den = std::hypot(a0, hj1);
        const double cc = den > 0.0 ? a0 / den : 1.0, ss = den > 0.0 ? hj1 / den : 0.0;
        cs[size_t(c) * m + j] = cc;
        sn[size_t(c) * m + j] = ss;
        Hat(j, j, c) = den;
        double &gj = g[size_t(c) * (m + 1) + j];
        g[size_t(c) * (m + 1) + j + 1] = -ss * gj;
        gj = cc * gj;
        worst = std::max(worst, std::abs(g[size_t(c) * (m + 1) + j + 1]) / bnorm[c]);
      }
      ck(cudaMemcpyAsync(C, inv.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
      ck(cudaMemcpyAsync(V + (j + 1) * vs, W, sizeof(double) * vs, cudaMemcpyDeviceToDevice, s));
      ck(launch_col_scale(V + (j + 1) * vs, n, C, n, nrhs, s));
      // the global estimate is an upper bound on every system's share only up to
      // the ratio of norms; a margin keeps the true check the one that decides
      if (worst <= 0.25 * o->tol) {
        ++j;
        ++it;
        break;
      }
    }
    // x += Z y with y from the triangular systems
    std::vector<double> y(size_t(j) * nrhs, 0.0);
    for (int c = 0; c < nrhs; ++c)
      for (int i = j - 1; i >= 0; --i) {
        double t = g[size_t(c) * (m + 1) + i];
        for (int q = i + 1; q < j; ++q) t -= Hat(i, q, c) * y[size_t(q) * nrhs + c];
        y[size_t(i) * nrhs + c] = Hat(i, i, c) != 0.0 ? t / Hat(i, i, c) : 0.0;
      }
    if (j > 0) {
      ck(cudaMemcpyAsync(C, y.data(), sizeof(double) * j * nrhs, cudaMemcpyHostToDevice, s));
      ck(launch_block_axpy(Z, n, vs, j, C, x, ldx, n, nrhs, s));
    }
  }
  if (info) {
    info->iters = it;
    info->rel_residual = res;
    info->status = (res <= o->tol) ? H2SP_OK : H2SP_ENOCONV;
  }
  return res <= o->tol ? H2SP_OK : H2SP_ENOCONV;
}

}  // namespace

namespace {

// FNV-1a over the structure arrays of a descriptor whose sizes match plan p
// (the sizes come from the plan, which validated the descriptor it was built from)
uint64_t structure_hash(const h2sp_h2_desc *d, const Plan &p) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void *a, size_t bytes) {
    if (!a) {
      h = (h ^ 0xA5u) * 1099511628211ull;
      return;
    }
    const unsigned char *b = static_cast<const unsigned char *>(a);
    for (size_t i = 0; i < bytes; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  const size_t ncl = size_t(p.ncl), nleaf = size_t(p.nleaf);
  const size_t nfar = size_t(p.far_ptr[p.ncl]), nnear = size_t(p.near_ptr[p.nleaf]);
  mix(&d->n, sizeof(d->n));
  mix(d->level_ptr, sizeof(int32_t) * size_t(p.D + 2));
  mix(d->parent, sizeof(int32_t) * ncl);
  mix(d->begin, sizeof(int64_t) * ncl);
  mix(d->size, sizeof(int64_t) * ncl);
  mix(d->rank, sizeof(int32_t) * ncl);
  mix(d->far_ptr, sizeof(int64_t) * (ncl + 1));
  mix(d->far_col, sizeof(int32_t) * nfar);
  mix(d->near_ptr, sizeof(int64_t) * (nleaf + 1));
  mix(d->near_col, sizeof(int32_t) * nnear);
  mix(d->leaf_basis_off, sizeof(int64_t) * nleaf);
  mix(d->transfer_off, sizeof(int64_t) * ncl);
  mix(d->coupling_off, sizeof(int64_t) * nfar);
  mix(d->near_off, sizeof(int64_t) * nnear);
  if (!p.sym) {
    mix(d->col_leaf_basis_off, sizeof(int64_t) * nleaf);
    mix(d->col_transfer_off, sizeof(int64_t) * ncl);
  }
  return h;
}

// device copies of the structure (see StructureDev); synchronous uploads, once per analysis
std::shared_ptr<StructureDev> build_structure(const Plan &p) {
  auto sd = std::make_shared<StructureDev>();
  cudaGetDevice(&sd->device);
  const int L = p.lstop;
  for (int t = 0; t < p.ncl; ++t) sd->max_rank = std::max(sd->max_rank, p.rank[t]);
  // work items of every level
  const int nlw = int(p.lw.size());
  sd->lv.assign(std::max(nlw, 1), LevelDev());
  for (int l = 0; l < nlw; ++l) {
    const LevelWork &w = p.lw[l];
    LevelDev &d = sd->lv[l];
    d.q = sd->upload(w.q);
    d.nq = int(w.q.size());
    d.w = sd->upload(w.w);
    d.nw = int(w.w.size());
    d.c = sd->upload(w.c);
    d.nc = int(w.c.size());
    d.x = sd->upload(w.x);
    d.nx = int(w.x.size());
    d.nq_small = w.nq_small;
    d.nx_small = w.nx_small;
    d.max_m = w.max_m;
    double xf = 0.0, xfl = 0.0;
    for (size_t i = 0; i < w.x.size(); ++i) {
      const XItem &it = w.x[i];
      const double f =
          (it.qR >= 0 ? 2.0 * it.rows * it.cols * it.cols : 0.0) + (it.qL >= 0 ? 2.0 * it.rows * it.rows * it.cols : 0.0);
      if (int(i) < w.nx_small) {
        xf += f;
      } else {
        xfl += f;
        d.max_xr = std::max(d.max_xr, it.rows);
        d.max_xc = std::max(d.max_xc, it.cols);
      }
    }
    sd->x_flops.push_back(xf);
    sd->x_flops_large.push_back(xfl);
    if (!p.sym) {
      d.qc = sd->upload(w.qc);
      d.wc = sd->upload(w.wc);
    }
  }
  // apply items
  {
    int64_t width = 0;
    for (int l = 0; l <= L; ++l) {
      int64_t wl = 0;
      for (int t = p.level_ptr[p.D - l]; t < p.level_ptr[p.D - l + 1]; ++t) wl += p.m[t];
      width = std::max(width, wl);
    }
    sd->max_width = width;
    // the level maps come from the device level schedule, which must agree
    // with the plan (the host's, or the same device schedule's) to the integer
    DeviceMaps maps;
    A1Result a1;
    std::string err;
    const int st = device_schedule(p, &a1, &maps, err);
    for (void *q : maps.allocs) sd->allocs.push_back(q);
    if (st != H2SP_OK) {
      g_cuda_err = err;
      throw CudaFail{st == H2SP_ENOMEM ? cudaErrorMemoryAllocation : cudaErrorUnknown};
    }
    bool same = a1.lstop == L && a1.m == p.m && a1.kp == p.kp && a1.d == p.d && a1.off == p.off &&
                a1.xoff == p.xoff && a1.node_of == p.node_of && a1.node_off == p.node_off &&
                a1.node_cluster == p.node_cluster && a1.node_level == p.node_level && int(maps.nap.size()) == L;
    for (int l = 0; same && l < L; ++l) {
      // the apply items the plan implies, against the device's
      std::vector<ApItem> want, got(size_t(maps.nap[l]));
      for (int t = p.level_ptr[p.D - l]; t < p.level_ptr[p.D - l + 1]; ++t) {
        if (p.m[t] == 0) continue;
        ApItem a{};
        a.q = p.q_off[t];
        a.m = int32_t(p.m[t]);
        a.kp = int32_t(p.kp[t]);
        a.xin = p.xoff[t];
        a.yout = p.d[t] > 0 ? p.node_off[p.node_of[t]] : -1;
        a.xout = p.kp[t] > 0 ? p.xoff[p.parent[t]] + p.off[t] : -1;
        want.push_back(a);
      }
      same = want.size() == got.size();
      if (same && !got.empty())
        ck(cudaMemcpy(got.data(), maps.ap + maps.ap_base[l], got.size() * sizeof(ApItem), cudaMemcpyDeviceToHost));
      for (size_t i = 0; same && i < got.size(); ++i)
        same = got[i].q == want[i].q && got[i].m == want[i].m && got[i].kp == want[i].kp &&
               got[i].xin == want[i].xin && got[i].yout == want[i].yout && got[i].xout == want[i].xout;
      sd->lv[l].ap = maps.ap + maps.ap_base[l];
      sd->lv[l].nap = maps.nap[l];
    }
    if (same) {
      // the top clusters' copies
      std::vector<int64_t> ts, td;
      std::vector<int32_t> tl;
      for (int t = p.level_ptr[p.D - L]; t < p.level_ptr[p.D - L + 1]; ++t)
        if (p.m[t] > 0) {
          ts.push_back(L == 0 ? p.h_begin[t] : p.xoff[t]);
          td.push_back(p.node_off[p.node_of[t]]);
          tl.push_back(int32_t(p.m[t]));
        }
      same = int(ts.size()) == maps.ntop;
      if (same && !ts.empty()) {
        std::vector<int64_t> gs(ts.size()), gd(ts.size());
        std::vector<int32_t> gl(ts.size());
        ck(cudaMemcpy(gs.data(), maps.top_src, gs.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
        ck(cudaMemcpy(gd.data(), maps.top_dst, gd.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
        ck(cudaMemcpy(gl.data(), maps.top_len, gl.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        same = gs == ts && gd == td && gl == tl;
      }
    }
    if (!same) {
      g_cuda_err = "internal: the device level schedule differs from the plan";
      throw CudaFail{cudaErrorUnknown};
    }
    sd->top_src = maps.top_src;
    sd->top_dst = maps.top_dst;
    sd->top_len = maps.top_len;
    sd->ntop = maps.ntop;
    sd->node_off = maps.node_off;
  }
  // S structure, H^2 structure
  sd->brow_ptr = sd->upload(p.brow_ptr);
  sd->bcol = sd->upload(p.bcol);
  sd->val_off = sd->upload(p.val_off);
  {
    H2Dev &g = sd->h2;
    g.begin = sd->upload(p.h_begin);
    g.size = sd->upload(p.h_size);
    g.rank = sd->upload(p.rank);
    g.parent = sd->upload(p.parent);
    g.leaf_basis_off = sd->upload(p.leaf_basis_off);
    g.transfer_off = sd->upload(p.transfer_off);
    g.coupling_off = sd->upload(p.coupling_off);
    g.near_off = sd->upload(p.near_off);
    g.col_leaf_basis_off = p.sym ? nullptr : sd->upload(p.col_leaf_basis_off);
    g.col_transfer_off = p.sym ? nullptr : sd->upload(p.col_transfer_off);
    g.far_ptr = sd->upload(p.far_ptr);
    g.near_ptr = sd->upload(p.near_ptr);
    g.far_col = sd->upload(p.far_col);
    g.near_col = sd->upload(p.near_col);
    g.xh_off = sd->upload(p.xh_off);
    g.leaf0 = p.level_ptr[p.D];
    std::vector<int32_t> cs(p.ncl, 0), cc(p.ncl, 0);
    for (int c = p.ncl - 1; c >= p.level_ptr[1]; --c) {  // every non-root cluster
      cs[p.parent[c]] = c;
      cc[p.parent[c]]++;
    }
    sd->child_start = sd->upload(cs);
    sd->child_cnt = sd->upload(cc);
    // heaviest-first launch orders of the close-block and coupling kernels
    {
      std::vector<double> wl(p.nleaf, 0.0), wc(p.ncl, 0.0);
      for (int lf = 0; lf < p.nleaf; ++lf) {
        const int t = p.level_ptr[p.D] + lf;
        for (int64_t z = p.near_ptr[lf]; z < p.near_ptr[lf + 1]; ++z)
          wl[lf] += double(p.h_size[t]) * double(p.h_size[p.near_col[z]]);
      }
      for (int t = 0; t < p.ncl; ++t)
        for (int64_t z = p.far_ptr[t]; z < p.far_ptr[t + 1]; ++z) wc[t] += double(p.rank[t]) * p.rank[p.far_col[z]];
      std::vector<int32_t> ol(p.nleaf), oc(p.ncl);
      for (int i = 0; i < p.nleaf; ++i) ol[i] = i;
      for (int i = 0; i < p.ncl; ++i) oc[i] = i;
      std::stable_sort(ol.begin(), ol.end(), [&](int a, int b) { return wl[a] > wl[b]; });
      // leaves above 64 points last (their own launch)
      auto large = std::stable_partition(ol.begin(), ol.end(),
                                         [&](int lf) { return p.h_size[p.level_ptr[p.D] + lf] <= kMaxBlock; });
      g.nleaf_large = int32_t(ol.end() - large);
      g.max_leaf = 0;
      for (int lf = 0; lf < p.nleaf; ++lf)
        g.max_leaf = std::max<int32_t>(g.max_leaf, int32_t(p.h_size[p.level_ptr[p.D] + lf]));
      std::stable_sort(oc.begin(), oc.end(), [&](int a, int b) { return wc[a] > wc[b]; });
      g.leaf_order = sd->upload(ol);
      g.couple_order = sd->upload(oc);
    }
    // FP64 multiply-adds per right-hand side of one product: close blocks,
    // couplings, the leaf bases (up and down) and the transfers (up and down)
    double mv = 0.0;
    for (int lf = 0; lf < p.nleaf; ++lf) {
      const int t = p.level_ptr[p.D] + lf;
      for (int64_t z = p.near_ptr[lf]; z < p.near_ptr[lf + 1]; ++z) {
        const double e = double(p.h_size[t]) * double(p.h_size[p.near_col[z]]);
        sd->near_bytes += 8.0 * e;
        mv += e;
      }
      mv += 2.0 * double(p.h_size[t]) * p.rank[t];
    }
    for (int t = 0; t < p.ncl; ++t) {
      for (int64_t z = p.far_ptr[t]; z < p.far_ptr[t + 1]; ++z) mv += double(p.rank[t]) * p.rank[p.far_col[z]];
      if (t >= p.level_ptr[1]) mv += 2.0 * double(p.rank[t]) * p.rank[p.parent[t]];
    }
    sd->mv_flops_per_rhs = 2.0 * mv;
    std::vector<int64_t> sp(1, 0);
    for (int r = 0; r < p.level_ptr[1]; ++r) sp.push_back(p.h_begin[r] + p.h_size[r]);
    sd->nseg = int(sp.size()) - 1;
    sd->seg_ptr = sd->upload(sp);
  }
  // symbolic factorization
  {
    std::vector<FrontDev> fd(p.fronts.size());
    for (size_t k = 0; k < p.fronts.size(); ++k) {
      const Front &F = p.fronts[k];
      fd[k] = FrontDev{F.off, F.piv_off, F.idx_off, F.map_off, F.dinv_off, F.s, F.b, F.f, F.parent, F.ld, 0};
      sd->max_s_all = std::max(sd->max_s_all, F.s);
    }
    // 128-row tiles of the packed operands of the blocked FP32 LU, per level
    for (size_t i = 0; i + 1 < p.front_level_ptr.size(); ++i) {
      int64_t acc = 0;
      for (int k = p.front_level_ptr[i]; k < p.front_level_ptr[i + 1]; ++k) {
        fd[k].pack_off = int32_t(acc);
        acc += (p.fronts[k].f + 127) / 128;
      }
      sd->max_pack_tiles = std::max(sd->max_pack_tiles, acc);
    }
    sd->fr = sd->upload(fd);
    sd->fidx = sd->upload(p.front_idx);
    sd->fmap = sd->upload(p.front_map);
    sd->asm_items = sd->upload(p.assemble);
    for (size_t i = 0; i + 1 < p.front_level_ptr.size(); ++i) {
      FrontLevel fl{p.front_level_ptr[i], p.front_level_ptr[i + 1], 0, 0, 0};
      for (int k = fl.lo; k < fl.hi; ++k) {
        const Front &F = p.fronts[k];
        fl.max_s = std::max(fl.max_s, F.s);
        fl.max_f = std::max(fl.max_f, F.f);
        fl.max_b = std::max(fl.max_b, F.b);
        fl.b2 += double(F.b) * F.b;
        fl.lu_elems += 0.5 * double(F.s) * F.s + double(F.s) * F.b;
      }
      sd->flev.push_back(fl);
    }
    // row-block work lists of the sweeps, in dependency order per level
    std::vector<int2> items;
    for (const Front &F : p.fronts) sd->nflags += int((F.s + kSolveBlock - 1) / kSolveBlock);
    for (const FrontLevel &L : sd->flev) {
      int maxb = 0;
      for (int k = L.lo; k < L.hi; ++k) maxb = std::max<int>(maxb, (p.fronts[k].s + kSolveBlock - 1) / kSolveBlock);
      // supernode items are pairs of row blocks: (b, b+1) forward, (b, b-1) backward
      sd->chain_fwd_off.push_back(int(items.size()));
      for (int b = 0; b < maxb; b += 2)
        for (int k = L.lo; k < L.hi; ++k)
          if (b < (p.fronts[k].s + kSolveBlock - 1) / kSolveBlock) items.push_back(make_int2(k, b));
      // (the boundary rows take their L21 product after the forward sweep, in one rectangular product)
      sd->chain_fwd_n.push_back(int(items.size()) - sd->chain_fwd_off.back());
      sd->chain_bwd_off.push_back(int(items.size()));
      for (int d = 0; d < maxb; d += 2)
        for (int k = L.lo; k < L.hi; ++k) {
          const int nb = (p.fronts[k].s + kSolveBlock - 1) / kSolveBlock;
          if (d < nb) items.push_back(make_int2(k, nb - 1 - d));
        }
      sd->chain_bwd_n.push_back(int(items.size()) - sd->chain_bwd_off.back());
    }
    sd->chain_items = sd->upload(items);
  }
  return sd;
}

// per-level buffers of the sparsification (stacked bases) and the source /
// destination tables of its kernels
void sparsify_setup_levels(h2sp_handle *h, const Plan &p) {
  const int L = p.lstop;
  const int nlw = int(p.lw.size());
  for (int l = 0; l < nlw; ++l) {
    const LevelWork &w = p.lw[l];
    LevelDev &d = h->lv[l];
    if (l >= 1) {
      d.W = h->alloc<double>(size_t(w.w_elems));
      if (!p.sym) d.Wc = h->alloc<double>(size_t(w.wc_elems));
    }
    std::vector<void *> sb = {const_cast<double *>(h->near_block), l < L ? h->Cbuf[l] : nullptr,
                              l < L ? h->RPbuf[l] : nullptr, l < L ? h->CPbuf[l] : nullptr};
    std::vector<void *> db = {h->S, l + 1 < L ? h->Cbuf[l + 1] : nullptr, l + 1 < L ? h->RPbuf[l + 1] : nullptr,
                              l + 1 < L ? h->CPbuf[l + 1] : nullptr};
    d.src_base = h->upload(sb);
    d.dst_base = h->upload(db);
  }
}

// the level recursion of the sparsification (§2.1-2.3, §4.2-4.3), kernels
// only: FP64 Householder completions and couplings, products into S in
// precision W
template <typename W>
void sparsify_kernels(h2sp_handle *h, const Plan &p, const StructureDev &sd, cudaStream_t s) {
  const int L = p.lstop;
  const int nlw = int(p.lw.size());
  for (int l = 0; l < nlw; ++l) {
    const LevelWork &w = p.lw[l];
    LevelDev &d = h->lv[l];
    if (l < L) {
      if (l >= 1) {
        ck(launch_stack_w(d.w, d.nw, h->Rr, h->transfer, d.W, s, &h->prof));
        if (!p.sym) ck(launch_stack_w(d.wc, d.nw, h->Rrc, h->col_transfer, d.Wc, s, &h->prof));
      }
      // small items (m <= kMaxBlock) first, in shared memory; then the large ones
      const int ms = std::max(std::min(w.max_m, kMaxBlock), 1), mk = std::max(w.max_k, 1);
      const int nl = d.nq - d.nq_small;
      ck(launch_householder(d.q, d.nq_small, h->leaf_basis, d.W, h->Q, h->Rr, ms, mk, s, &h->prof));
      ck(launch_householder_large(d.q + d.nq_small, nl, h->leaf_basis, d.W, h->Q, h->Rr, w.max_m, mk, s, &h->prof));
      if (!p.sym) {
        ck(launch_householder(d.qc, d.nq_small, h->col_leaf_basis, d.Wc, h->Qc, h->Rrc, ms, mk, s, &h->prof));
        ck(launch_householder_large(d.qc + d.nq_small, nl, h->col_leaf_basis, d.Wc, h->Qc, h->Rrc, w.max_m, mk, s,
                                    &h->prof));
      }
      ck(launch_coupling<W>(d.c, d.nc, h->Rr, h->Rrc, h->coupling, reinterpret_cast<W *const *>(d.dst_base),
                            sd.max_rank, s, &h->prof));
    }
    ck(launch_transform<W>(d.x, d.nx_small, const_cast<const void *const *>(d.src_base), h->Q, h->Qc,
                           reinterpret_cast<W *const *>(d.dst_base), s, &h->prof,
                           l < int(h->x_flops.size()) ? h->x_flops[l] : 0.0));
    ck(launch_transform_large<W>(d.x + d.nx_small, d.nx - d.nx_small, const_cast<const void *const *>(d.src_base),
                                 h->Q, h->Qc, reinterpret_cast<W *const *>(d.dst_base), d.max_xr, d.max_xc, s,
                                 &h->prof, l < int(h->x_flops_large.size()) ? h->x_flops_large[l] : 0.0));
  }
}

// every launch of the numeric sparsification (no allocation, no host
// synchronisation): zero the accumulated buffers, then the level recursion
void sparsify_launch(h2sp_handle *h) {
  const Plan &p = (*h->plan_ptr);
  cudaStream_t s = h->stream;
  const size_t wsz = (h->sp_prec == H2SP_FP32) ? sizeof(float) : sizeof(double);
  ck(cudaMemsetAsync(h->S, 0, wsz * size_t(std::max<int64_t>(p.s_elems, 1)), s));
  for (int l = 1; l < p.lstop; ++l) {
    ck(cudaMemsetAsync(h->Cbuf[l], 0, wsz * size_t(std::max<int64_t>(p.c_elems[l], 1)), s));
    ck(cudaMemsetAsync(h->RPbuf[l], 0, wsz * size_t(std::max<int64_t>(p.rp_elems[l], 1)), s));
    ck(cudaMemsetAsync(h->CPbuf[l], 0, wsz * size_t(std::max<int64_t>(p.cp_elems[l], 1)), s));
  }
  if (h->sp_prec == H2SP_FP32)
    sparsify_kernels<float>(h, p, *h->sdev, s);
  else
    sparsify_kernels<double>(h, p, *h->sdev, s);
}

// numeric part of the sparsification: the handle's buffers and the kernels,
// on the (shared) device copy of the structure
int sparsify_numeric(h2sp_handle *h, const h2sp_h2_desc *desc, int32_t sp_prec, h2sp_stream stream,
                     h2sp_handle **out) {
  h->sp_prec = sp_prec;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->prof.stream = h->stream;
  h->leaf_basis = desc->leaf_basis;
  h->transfer = desc->transfer;
  h->coupling = desc->coupling;
  h->near_block = desc->near_block;
  h->col_leaf_basis = desc->col_leaf_basis;
  h->col_transfer = desc->col_transfer;
  const Plan &p = (*h->plan_ptr);
  cudaStream_t s = h->stream;
  try {
    init_pool_once();
    {
      int dev = 0;
      cudaGetDevice(&dev);
      std::lock_guard<std::mutex> lock(h->cell->m);
      if (!h->cell->dev || h->cell->dev->device != dev) h->cell->dev = build_structure(p);
      h->sdev = h->cell->dev;
    }
    const StructureDev &sd = *h->sdev;
    // ---- owned buffers ----
    const size_t wsz = (sp_prec == H2SP_FP32) ? sizeof(float) : sizeof(double);
    auto walloc = [&](int64_t n) -> void * { return h->alloc<char>(size_t(std::max<int64_t>(n, 1)) * wsz); };
    h->Q = h->alloc<double>(size_t(p.q_elems));
    h->Rr = h->alloc<double>(size_t(p.rr_elems));
    if (p.sym) {
      h->Qc = h->Q;
      h->Rrc = h->Rr;
    } else {
      h->Qc = h->alloc<double>(size_t(p.q_elems));
      h->Rrc = h->alloc<double>(size_t(p.rr_elems));
    }
    h->S = walloc(p.s_elems);
    const int L = p.lstop;
    h->Cbuf.assign(L + 1, nullptr);
    h->RPbuf.assign(L + 1, nullptr);
    h->CPbuf.assign(L + 1, nullptr);
    for (int l = 1; l < L; ++l) {
      h->Cbuf[l] = walloc(p.c_elems[l]);
      h->RPbuf[l] = walloc(p.rp_elems[l]);
      h->CPbuf[l] = walloc(p.cp_elems[l]);
    }
    // ---- per-level tables and the sparsification kernels, level by level ----
    h->lv = sd.lv;
    h->x_flops = sd.x_flops;
    h->x_flops_large = sd.x_flops_large;
    sparsify_setup_levels(h, p);
    sparsify_launch(h);
    // ---- structure views for the applies, products, factor and solves ----
    h->max_width = sd.max_width;
    h->top_src = sd.top_src;
    h->top_dst = sd.top_dst;
    h->top_len = sd.top_len;
    h->ntop = sd.ntop;
    h->brow_ptr = sd.brow_ptr;
    h->bcol = sd.bcol;
    h->val_off = sd.val_off;
    h->node_off = sd.node_off;
    h->h2 = sd.h2;
    h->h2.leaf_basis = h->leaf_basis;
    h->h2.transfer = h->transfer;
    h->h2.coupling = h->coupling;
    h->h2.near_block = h->near_block;
    h->h2.col_leaf_basis = h->col_leaf_basis;
    h->h2.col_transfer = h->col_transfer;
    h->child_start = sd.child_start;
    h->child_cnt = sd.child_cnt;
    h->near_bytes = sd.near_bytes;
    h->mv_flops_per_rhs = sd.mv_flops_per_rhs;
    h->xh = h->alloc<double>(size_t(std::max<int64_t>(p.xh_elems, 1)) * 16);
    h->yh = h->alloc<double>(size_t(std::max<int64_t>(p.xh_elems, 1)) * 16);
    h->nseg = sd.nseg;
    h->seg_ptr = sd.seg_ptr;
    h->norms = h->alloc<double>(size_t(h->nseg) * 64);
    h->fr = sd.fr;
    h->fidx = sd.fidx;
    h->fmap = sd.fmap;
    h->asm_items = sd.asm_items;
    h->max_s_all = sd.max_s_all;
    h->flev = sd.flev;
    h->chain_items = sd.chain_items;
    h->chain_fwd_off = sd.chain_fwd_off;
    h->chain_fwd_n = sd.chain_fwd_n;
    h->chain_bwd_off = sd.chain_bwd_off;
    h->chain_bwd_n = sd.chain_bwd_n;
    h->chain_flags = h->alloc<int>(size_t(std::max(sd.nflags, 1)));
    ck(cudaMemsetAsync(h->chain_flags, 0, sizeof(int) * size_t(std::max(sd.nflags, 1)), h->stream));
    h->chain_tickets = h->alloc<int>(2 * std::max<size_t>(h->flev.size(), 1));
    h->serr = h->alloc<int>(1);
    ck(cudaMemsetAsync(h->serr, 0, sizeof(int), h->stream));
    ck(cudaGetLastError());
  } catch (const CudaFail &f) {
    h->release();
    delete h;
    return status_of(f.e);
  } catch (const std::bad_alloc &) {
    h->release();
    delete h;
    return H2SP_ENOMEM;
  }
  h->device_ready = true;
  *out = h;
  return H2SP_OK;
}

// working precision of the sparsification selected by the options, -1 if they are malformed
int32_t sparsify_prec_of(const h2sp_opts *opts) {
  const int32_t f = opts ? opts->flags : 0;
  if (f & ~int32_t(H2SP_SPARSIFY_FP32)) return -1;
  return (f & H2SP_SPARSIFY_FP32) ? H2SP_FP32 : H2SP_FP64;
}

// device array of n values of S's precision -> n host doubles (synchronises)
void copy_out(h2sp_handle *h, double *dst, const void *src, int64_t n) {
  if (n <= 0) return;
  if (h->sp_prec == H2SP_FP32) {
    std::vector<float> tmp(static_cast<size_t>(n));
    ck(cudaMemcpyAsync(tmp.data(), src, sizeof(float) * size_t(n), cudaMemcpyDeviceToHost, h->stream));
    ck(cudaStreamSynchronize(h->stream));
    for (int64_t i = 0; i < n; ++i) dst[i] = double(tmp[size_t(i)]);
  } else {
    ck(cudaMemcpyAsync(dst, src, sizeof(double) * size_t(n), cudaMemcpyDeviceToHost, h->stream));
    ck(cudaStreamSynchronize(h->stream));
  }
}

// ---- factorization, in three parts: buffers (first call), launches, check ----
// `prec` is an h2sp_prec: bit 0 selects FP32 fronts, bit 1 the block Cholesky,
// bit 2 BF16 block-end updates, bit 3 their two-term (hi + lo) split.
inline bool prec_fp32(int32_t prec) { return (prec & 1) != 0; }
inline bool prec_chol(int32_t prec) { return (prec & 2) != 0; }
// the BF16 mode of the block-end updates: 0 none, 1 BF16, 2 BF16 hi + lo
inline int prec_bf16(int32_t prec) { return (prec & 4) ? ((prec & 8) ? 2 : 1) : 0; }
inline bool prec_valid(int32_t prec) {
  return (prec >= H2SP_FP64 && prec <= H2SP_FP32_CHOL) || prec == H2SP_BF16_CHOL || prec == H2SP_BF16X3_CHOL;
}

void factor_prepare(h2sp_handle *h, int32_t prec) {
  const Plan &p = (*h->plan_ptr);
  cudaStream_t s = h->stream;
  // the fronts are sized by the precision of the factorization: FP32 fronts
  // take half the memory of FP64 ones; a later FP64 factorization of the same
  // handle replaces the buffer by a wider one (which also holds FP32 fronts)
  const size_t esz = prec_fp32(prec) ? sizeof(float) : sizeof(double);
  if (h->fronts == nullptr || h->fronts_esz < esz) {
    if (h->fronts != nullptr) h->free_one(h->fronts);
    h->fronts = h->alloc<uint8_t>(size_t(std::max<int64_t>(p.front_elems, 1)) * esz);
    h->fronts_esz = esz;
  }
  if (h->piv == nullptr) {
    h->piv = h->alloc<int32_t>(size_t(std::max<int64_t>(p.piv_elems, 1)));
    h->perm = h->alloc<int32_t>(size_t(std::max<int64_t>(p.piv_elems, 1)));
    size_t maxn = 1;
    for (const FrontLevel &L : h->flev) maxn = std::max<size_t>(maxn, size_t(L.hi - L.lo));
    h->swaps = h->alloc<int32_t>(8 * maxn * (1 + 2 * kMaxSwapRows));  // two outer blocks of panels in flight
    h->err = h->alloc<int>(2);  // error bits, pivots compensated
    h->dinv = h->alloc<double>(size_t(std::max<int64_t>(p.dinv_elems, 1)));
  }
  if (prec_chol(prec) && h->chol_inv == nullptr) {
    // the L11^-1 tiles of one level's panels (one per front), sized for FP64
    size_t maxn = 1;
    for (const FrontLevel &L : h->flev) maxn = std::max<size_t>(maxn, size_t(L.hi - L.lo));
    h->chol_inv = h->alloc<double>(maxn * kCholInvElems);
  }
  if (h->la.side == nullptr && lookahead_enabled()) {
    int lo = 0, hi = 0;
    ck(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    ck(cudaStreamCreateWithPriority(&h->la.side, cudaStreamNonBlocking, hi));
    ck(cudaStreamCreateWithPriority(&h->la.rest, cudaStreamNonBlocking, lo));
    ck(cudaEventCreateWithFlags(&h->la.next, cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&h->la.panel, cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&h->la.done, cudaEventDisableTiming));
  }
  if (prec_fp32(prec) && tma_enabled() && !p.fronts.empty() && h->tmaps_base != h->fronts) {
    // (re-)encode the descriptors whenever the front buffer is new
    h->tmaps = nullptr;
    if (h->tmaps_buf == nullptr) h->tmaps_buf = h->alloc<uint8_t>(2 * p.fronts.size() * kTmapBytes);
    ck(cudaStreamSynchronize(s));  // the allocation is usable by the synchronous copy
    uint8_t *m64 = h->tmaps_buf + p.fronts.size() * kTmapBytes;
    if (make_front_tmaps(p.fronts.data(), int(p.fronts.size()), static_cast<float *>(h->fronts), h->tmaps_buf) ==
            cudaSuccess &&
        make_front_tmaps(p.fronts.data(), int(p.fronts.size()), static_cast<float *>(h->fronts), m64, 64) ==
            cudaSuccess) {
      h->tmaps = h->tmaps_buf;
      h->tmaps64 = m64;
      h->tmaps_base = h->fronts;
    }
    cudaGetLastError();
    if (h->tmaps != nullptr && h->pack == nullptr && h->sdev->max_pack_tiles > 0)
      h->pack = h->alloc<float>(size_t(3 * h->sdev->max_pack_tiles * kPackTileFloats));
  }
}

template <typename T>
void factor_launch_t(h2sp_handle *h, bool chol, int bf16) {
  const Plan &p = (*h->plan_ptr);
  cudaStream_t s = h->stream;
  const LuAsync *la = h->la.side ? &h->la : nullptr;
  ck(cudaMemsetAsync(h->fronts, 0, size_t(std::max<int64_t>(p.front_elems, 1)) * sizeof(T), s));
  ck(cudaMemsetAsync(h->err, 0, 2 * sizeof(int), s));
  const int64_t na = int64_t(p.assemble.size());
  const double abytes = double(p.s_elems) * double((h->sp_prec == H2SP_FP32 ? sizeof(float) : sizeof(double)) + sizeof(T));
  T *F = static_cast<T *>(h->fronts);
  if (h->sp_prec == H2SP_FP32)
    ck(launch_assemble<float, T>(h->asm_items, na, static_cast<const float *>(h->S), F, s, &h->prof, abytes));
  else
    ck(launch_assemble<double, T>(h->asm_items, na, static_cast<const double *>(h->S), F, s, &h->prof, abytes));
  const bool fp32 = std::is_same<T, float>::value;
  for (const FrontLevel &L : h->flev) {
    const uint8_t *maps = (fp32 && h->tmaps) ? h->tmaps + size_t(L.lo) * kTmapBytes : nullptr;
    const uint8_t *maps64 = (fp32 && h->tmaps64) ? h->tmaps64 + size_t(L.lo) * kTmapBytes : nullptr;
    if (chol) {
      ck(launch_chol_level<T>(h->fr + L.lo, p.fronts.data() + L.lo, L.hi - L.lo, L.max_s, L.max_f, F, h->piv, h->err,
                              s, la, &h->prof, maps, h->pack, reinterpret_cast<T *>(h->chol_inv), &h->chol_sched,
                              maps64, bf16));
    } else {
      ck(launch_lu_level<T>(h->fr + L.lo, p.fronts.data() + L.lo, L.hi - L.lo, L.max_s, L.max_f, F, h->piv, h->swaps,
                            h->err, s, la, &h->prof, maps, fp32 ? h->pack : nullptr, maps64));
    }
    ck(launch_extend_add_impl<T>(h->fr, L.lo, L.hi - L.lo, L.max_b, h->fmap, F, s, &h->prof, chol ? 0.5 * L.b2 : L.b2,
                                 chol));
  }
  const int nf = int(p.fronts.size());
  if (chol) {
    // the LU form: unit L and U = D L^T (read + written: sum of s(2f - s) entries)
    double el = 0.0;
    for (const Front &Fr : p.fronts) el += double(Fr.s) * (2.0 * Fr.f - Fr.s);
    ck(launch_chol_to_lu<T>(h->fr, nf, int(p.max_front), F, s, &h->prof, 1.5 * el * sizeof(T)));
  }
  ck(launch_make_perm<T>(h->fr, nf, h->max_s_all, h->piv, h->perm, s, &h->prof));
  ck(launch_invert_diag<T>(h->fr, nf, h->max_s_all, F, static_cast<T *>(h->dinv), s, &h->prof));
}

// every launch of the factorization (no allocation, no host synchronisation)
void factor_launch(h2sp_handle *h, int32_t prec) {
  if (prec_fp32(prec))
    factor_launch_t<float>(h, prec_chol(prec), prec_bf16(prec));
  else
    factor_launch_t<double>(h, prec_chol(prec), 0);
}

// the factorization's error word, after the stream has drained
int factor_finish(h2sp_handle *h, int32_t prec) {
  int herr2[2] = {0, 0};
  ck(cudaMemcpyAsync(herr2, h->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  ck(cudaStreamSynchronize(h->stream));
  const int herr = herr2[0] & ~16;
  h->compensated = (herr2[0] & 16) ? herr2[1] : 0;
  if (herr & 4) return H2SP_ETIMEOUT;
  if (herr & 8) {
    g_cuda_err = "h2sp_factor: a pivot of the block Cholesky is not positive: S is not positive definite "
                 "in this precision";
    return H2SP_ESINGULAR;
  }
  if (herr != 0) return H2SP_ESINGULAR;
  h->prec = prec_fp32(prec) ? H2SP_FP32 : H2SP_FP64;
  h->chol = prec_chol(prec);
  h->ilut = false;
  return H2SP_OK;
}

// the descriptor has the analysed structure: sizes first, then a fingerprint
// of every structure array; the numeric arrays are present as the analysis
// expects (with or without column bases)
bool same_structure(const h2sp_handle *an, const h2sp_h2_desc *desc) {
  const Plan &ap = *an->plan_ptr;
  if (desc->n != ap.n || desc->depth != ap.D || !desc->level_ptr || !desc->far_ptr || !desc->near_ptr) return false;
  for (int l = 0; l <= ap.D + 1; ++l)
    if (desc->level_ptr[l] != ap.level_ptr[l]) return false;
  if (desc->far_ptr[ap.ncl] != ap.far_ptr[ap.ncl] || desc->near_ptr[ap.nleaf] != ap.near_ptr[ap.nleaf]) return false;
  if (!desc->leaf_basis || !desc->transfer || !desc->coupling || !desc->near_block) return false;
  if ((desc->col_leaf_basis == nullptr) != ap.sym || (desc->col_transfer == nullptr) != ap.sym) return false;
  return structure_hash(desc, ap) == an->structure_hash;
}

// elements of each numeric array of a descriptor whose structure has been
// validated (the largest block end of each packed array)
struct NumericSizes {
  int64_t leaf = 0, transfer = 0, coupling = 0, near = 0, col_leaf = 0, col_transfer = 0;
};
NumericSizes numeric_sizes(const h2sp_h2_desc *d) {
  NumericSizes z;
  const int D = d->depth;
  const int l0 = d->level_ptr[D], ncl = d->level_ptr[D + 1];
  for (int t = l0; t < ncl; ++t) {
    const int64_t blk = d->size[t] * int64_t(d->rank[t]);
    if (blk > 0) z.leaf = std::max(z.leaf, d->leaf_basis_off[t - l0] + blk);
    if (blk > 0 && d->col_leaf_basis_off) z.col_leaf = std::max(z.col_leaf, d->col_leaf_basis_off[t - l0] + blk);
  }
  for (int c = 0; c < ncl; ++c) {
    if (d->parent[c] < 0) continue;
    const int64_t blk = int64_t(d->rank[c]) * d->rank[d->parent[c]];
    if (blk > 0) z.transfer = std::max(z.transfer, d->transfer_off[c] + blk);
    if (blk > 0 && d->col_transfer_off) z.col_transfer = std::max(z.col_transfer, d->col_transfer_off[c] + blk);
  }
  for (int t = 0; t < ncl; ++t)
    for (int64_t e = d->far_ptr[t]; e < d->far_ptr[t + 1]; ++e) {
      const int64_t blk = int64_t(d->rank[t]) * d->rank[d->far_col[e]];
      if (blk > 0) z.coupling = std::max(z.coupling, d->coupling_off[e] + blk);
    }
  for (int t = l0; t < ncl; ++t)
    for (int64_t e = d->near_ptr[t - l0]; e < d->near_ptr[t - l0 + 1]; ++e) {
      const int64_t blk = d->size[t] * d->size[d->near_col[e]];
      if (blk > 0) z.near = std::max(z.near, d->near_off[e] + blk);
    }
  return z;
}

}  // namespace

namespace h2sp {
void set_last_error(const std::string &msg) { g_cuda_err = msg; }
}  // namespace h2sp

extern "C" {

const char *h2sp_status_string(int32_t st) {
  switch (st) {
    case H2SP_OK: return "ok";
    case H2SP_EINVAL: return "invalid argument or descriptor";
    case H2SP_ENOMEM: return "out of device memory";
    case H2SP_ECUDA: return "CUDA error";
    case H2SP_ESINGULAR: return "singular pivot block";
    case H2SP_ESTATE: return "call out of order";
    case H2SP_ENOCONV: return "no convergence";
    case H2SP_ETIMEOUT: return "device wait timed out";
    case H2SP_EUNSUPPORTED: return "unsupported size";
    default: return "unknown status";
  }
}

const char *h2sp_last_cuda_error(void) { return g_cuda_err.c_str(); }

int h2sp_sparsify(const h2sp_h2_desc *desc, const h2sp_opts *opts, h2sp_stream stream, h2sp_handle **out) {
  if (!out) return H2SP_EINVAL;
  *out = nullptr;
  const int32_t sp_prec = sparsify_prec_of(opts);
  if (sp_prec < 0) return H2SP_EINVAL;
  h2sp_handle *h = new (std::nothrow) h2sp_handle();
  if (!h) return H2SP_ENOMEM;
  std::string err;
  auto t0 = std::chrono::steady_clock::now();
  auto plan = std::make_shared<Plan>();
  // the level schedule on the device, from the validated structure
  const A1Source dev_a1 = [](const Plan &p, A1Result &r, std::string &e) { return device_schedule(p, &r, nullptr, e); };
  int st = build_plan(desc, *plan, err, true, &dev_a1);
  h->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st != H2SP_OK) {
    g_cuda_err = err;
    delete h;
    return st;
  }
  h->plan_ptr = plan;
  h->cell = std::make_shared<StructureCell>();
  h->structure_hash = structure_hash(desc, *plan);
  return sparsify_numeric(h, desc, sp_prec, stream, out);
}

int h2sp_sparsify_analyzed(const h2sp_handle *an, const h2sp_h2_desc *desc, const h2sp_opts *opts,
                           h2sp_stream stream, h2sp_handle **out) {
  if (!out) return H2SP_EINVAL;
  *out = nullptr;
  const int32_t sp_prec = sparsify_prec_of(opts);
  if (sp_prec < 0) return H2SP_EINVAL;
  if (!an || !an->plan_ptr || !an->cell || !desc) return H2SP_EINVAL;
  if (!same_structure(an, desc)) return H2SP_EINVAL;
  h2sp_handle *h = new (std::nothrow) h2sp_handle();
  if (!h) return H2SP_ENOMEM;
  h->plan_ptr = an->plan_ptr;
  h->cell = an->cell;
  h->structure_hash = an->structure_hash;
  h->plan_seconds = 0.0;
  return sparsify_numeric(h, desc, sp_prec, stream, out);
}


int h2sp_analyze(const h2sp_h2_desc *desc, h2sp_handle **out) {
  if (!out) return H2SP_EINVAL;
  *out = nullptr;
  h2sp_handle *h = new (std::nothrow) h2sp_handle();
  if (!h) return H2SP_ENOMEM;
  std::string err;
  auto t0 = std::chrono::steady_clock::now();
  auto plan = std::make_shared<Plan>();
  int st = build_plan(desc, *plan, err, false);
  h->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st != H2SP_OK) {
    g_cuda_err = err;
    delete h;
    return st;
  }
  h->plan_ptr = plan;
  h->cell = std::make_shared<StructureCell>();
  h->structure_hash = structure_hash(desc, *plan);
  *out = h;
  return H2SP_OK;
}

int h2sp_factor(h2sp_handle *h, int32_t prec, h2sp_stream stream) {
  if (!h) return H2SP_EINVAL;
  if (!h->device_ready) return H2SP_ESTATE;
  if (!prec_valid(prec)) return H2SP_EINVAL;
  if (prec_bf16(prec) && (!tma_enabled() || !use_tensor_core_gemm_host())) {
    g_cuda_err = "h2sp_factor: the BF16 block-end updates need the tensor-core path";
    return H2SP_EUNSUPPORTED;
  }
  if (prec_chol(prec) && (h->col_leaf_basis != nullptr || h->col_transfer != nullptr)) {
    g_cuda_err = "h2sp_factor: the block Cholesky needs symmetric bases (V = U)";
    return H2SP_EINVAL;
  }
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->prof.stream = h->stream;
  try {
    if (h->graph_exec != nullptr && prec != h->last_prec) {
      // the captured refactorization is of the other precision
      ck(cudaGraphExecDestroy(h->graph_exec));
      h->graph_exec = nullptr;
    }
    factor_prepare(h, prec);
    h->prec = -1;
    factor_launch(h, prec);
    h->last_prec = prec;
    return factor_finish(h, prec);
  } catch (const CudaFail &f) {
    return status_of(f.e);
  }
}

int h2sp_factor_ilut(h2sp_handle *h, double tau, h2sp_stream stream) {
  if (!h || !(tau >= 0.0) || !std::isfinite(tau)) return H2SP_EINVAL;
  if (!h->device_ready) return H2SP_ESTATE;
  const Plan &p = (*h->plan_ptr);
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->prof.stream = h->stream;
  const StructureDev &sd = *h->sdev;
  h->prec = -1;
  h->ilut = false;
  try {
    ilut_factor(h->ilu, p, sd.brow_ptr, sd.bcol, sd.val_off, sd.node_off, h->S, h->sp_prec == H2SP_FP32, tau,
                h->stream, &h->prof);
  } catch (const IlutFail &f) {
    g_cuda_err = "h2sp_factor_ilut: " + f.msg;
    h->ilu.release();
    return f.st;
  }
  h->prec = H2SP_FP64;
  h->chol = false;
  h->ilut = true;
  return H2SP_OK;
}

int h2sp_export_ilut(h2sp_handle *h, int32_t *perm, int64_t *l_ptr, int32_t *l_col, double *l_val, int64_t *u_ptr,
                     int32_t *u_col, double *u_val, int64_t *nnz_l, int64_t *nnz_u) {
  if (!h) return H2SP_EINVAL;
  if (!h->ilut || !h->ilu.ready) return H2SP_ESTATE;
  IlutState &st = h->ilu;
  const int64_t n = st.n;
  std::vector<int64_t> off(static_cast<size_t>(n));
  std::vector<int32_t> nl(static_cast<size_t>(n)), nu(static_cast<size_t>(n)), pc(static_cast<size_t>(st.nnz));
  std::vector<double> pv(static_cast<size_t>(st.nnz));
  cudaError_t e = cudaMemcpy(off.data(), st.row_off, sizeof(int64_t) * size_t(n), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(nl.data(), st.nl, sizeof(int32_t) * size_t(n), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(nu.data(), st.nu, sizeof(int32_t) * size_t(n), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && st.nnz)
    e = cudaMemcpy(pc.data(), st.pool_col, sizeof(int32_t) * size_t(st.nnz), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && st.nnz)
    e = cudaMemcpy(pv.data(), st.pool_val, sizeof(double) * size_t(st.nnz), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && perm) e = cudaMemcpy(perm, st.perm, sizeof(int32_t) * size_t(n), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    g_cuda_err = cudaGetErrorString(e);
    cudaGetLastError();
    return H2SP_ECUDA;
  }
  int64_t tl = 0, tu = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t o = off[size_t(i)];
    if (l_ptr) l_ptr[i] = tl;
    if (u_ptr) u_ptr[i] = tu;
    for (int q = 0; q < nl[size_t(i)]; ++q, ++tl) {
      if (l_col) l_col[tl] = pc[size_t(o + q)];
      if (l_val) l_val[tl] = pv[size_t(o + q)];
    }
    for (int q = 0; q < nu[size_t(i)]; ++q, ++tu) {
      if (u_col) u_col[tu] = pc[size_t(o + nl[size_t(i)] + q)];
      if (u_val) u_val[tu] = pv[size_t(o + nl[size_t(i)] + q)];
    }
  }
  if (l_ptr) l_ptr[n] = tl;
  if (u_ptr) u_ptr[n] = tu;
  if (nnz_l) *nnz_l = tl;
  if (nnz_u) *nnz_u = tu;
  return H2SP_OK;
}

int h2sp_refactor(h2sp_handle *h, h2sp_stream stream) {
  if (!h) return H2SP_EINVAL;
  if (!h->device_ready || h->last_prec < 0 || h->ilut) return H2SP_ESTATE;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->prof.stream = h->stream;
  cudaStream_t s = h->stream;
  const int32_t prec = h->last_prec;
  bool capturing = false;
  try {
    if (h->graph_stream == nullptr) {
      ck(cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking));
      ck(cudaEventCreateWithFlags(&h->graph_in, cudaEventDisableTiming));
      ck(cudaEventCreateWithFlags(&h->graph_out, cudaEventDisableTiming));
    }
    cudaStream_t gs = h->graph_stream;
    if (h->graph_exec == nullptr) {
      // capture every launch of both phases, on every stream they use (the
      // handle's buffers exist since the first factorization); the capture
      // runs on the handle's own stream, since the caller's may be the legacy
      // default stream, which cannot be captured
      ck(cudaStreamSynchronize(s));
      const int timing = h->prof.timing;
      h->prof.timing = 0;
      h->stream = gs;
      ck(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
      capturing = true;
      sparsify_launch(h);
      factor_launch(h, prec);
      cudaGraph_t g = nullptr;
      capturing = false;
      const cudaError_t ee = cudaStreamEndCapture(gs, &g);
      h->stream = s;
      h->prof.timing = timing;
      ck(ee);
      const cudaError_t ie = cudaGraphInstantiate(&h->graph_exec, g, 0);
      cudaGraphDestroy(g);
      ck(ie);
    }
    h->prec = -1;
    ck(cudaEventRecord(h->graph_in, s));
    ck(cudaStreamWaitEvent(gs, h->graph_in, 0));
    ck(cudaGraphLaunch(h->graph_exec, gs));
    ck(cudaEventRecord(h->graph_out, gs));
    ck(cudaStreamWaitEvent(s, h->graph_out, 0));
    return factor_finish(h, prec);
  } catch (const CudaFail &f) {
    if (capturing) {
      cudaGraph_t g = nullptr;
      if (cudaStreamEndCapture(h->graph_stream, &g) == cudaSuccess && g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
    h->stream = s;
    return status_of(f.e);
  }
}

int h2sp_apply(h2sp_handle *h, int32_t op, int32_t nrhs, const double *in, int64_t ldin, double *out, int64_t ldout,
               h2sp_stream stream) {
  if (!h || !in || !out || nrhs <= 0) return H2SP_EINVAL;
  if (!h->device_ready) return H2SP_ESTATE;
  const Plan &p = (*h->plan_ptr);
  if (ldin < p.n || ldout < p.n) return H2SP_EINVAL;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->prof.stream = h->stream;
  try {
    ensure_vectors(h, nrhs);
    switch (op) {
      case H2SP_OP_UT: apply_T(h, false, in, ldin, out, ldout, nrhs); break;
      case H2SP_OP_VT: apply_T(h, true, in, ldin, out, ldout, nrhs); break;
      case H2SP_OP_U: apply_N(h, false, in, ldin, out, ldout, nrhs); break;
      case H2SP_OP_V: apply_N(h, true, in, ldin, out, ldout, nrhs); break;
      case H2SP_OP_S:
        if (h->sp_prec == H2SP_FP32)
          ck(launch_spmv(h->brow_ptr, h->bcol, h->val_off, h->node_off, int(p.node_size.size()),
                         static_cast<const float *>(h->S), in, ldin, out, ldout, nrhs, h->stream));
        else
          ck(launch_spmv(h->brow_ptr, h->bcol, h->val_off, h->node_off, int(p.node_size.size()),
                         static_cast<const double *>(h->S), in, ldin, out, ldout, nrhs, h->stream));
        break;
      case H2SP_OP_H2: h2_matvec(h, in, ldin, out, ldout, nrhs); break;
      case H2SP_OP_SINV:
        if (h->prec < 0) return H2SP_ESTATE;
        for (int r = 0; r < nrhs; ++r)
          ck(cudaMemcpyAsync(h->vecS + r * p.n, in + r * ldin, sizeof(double) * p.n, cudaMemcpyDeviceToDevice,
                             h->stream));
        solve_S(h, h->vecS, nrhs);
        for (int r = 0; r < nrhs; ++r)
          ck(cudaMemcpyAsync(out + r * ldout, h->vecS + r * p.n, sizeof(double) * p.n, cudaMemcpyDeviceToDevice,
                             h->stream));
        break;
      default: return H2SP_EINVAL;
    }
    ck(cudaGetLastError());
  } catch (const CudaFail &f) {
    return status_of(f.e);
  }
  return H2SP_OK;
}

int h2sp_solve(h2sp_handle *h, const h2sp_solve_opts *o, int32_t nrhs, const double *b, int64_t ldb, double *x,
               int64_t ldx, h2sp_solve_info *info, h2sp_stream stream) {
  if (!h || !o || !b || !x || nrhs <= 0 || nrhs > 64) return H2SP_EINVAL;
  if (!h->device_ready) return H2SP_ESTATE;
  const Plan &p = (*h->plan_ptr);
  if (ldb < p.n || ldx < p.n) return H2SP_EINVAL;
  if (o->mode != H2SP_DIRECT && o->mode != H2SP_IR && o->mode != H2SP_GMRES) return H2SP_EINVAL;
  if (h->prec < 0) return H2SP_ESTATE;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaStream_t s = h->stream;
  if (info) {
    info->iters = 0;
    info->rel_residual = -1.0;
    info->status = H2SP_OK;
  }
  try {
    ensure_vectors(h, nrhs);
    ensure_work(h, nrhs);
    if (o->mode == H2SP_DIRECT) {
      precond(h, b, ldb, x, ldx, nrhs);
      ck(cudaGetLastError());
      return sweep_status(h);
    }
    if (o->mode == H2SP_GMRES) {
      const int st = gmres(h, o, nrhs, b, ldb, x, ldx, info);
      const int ss = sweep_status(h);
      return ss != H2SP_OK ? ss : st;
    }
    // iterative refinement on the FP64 H^2 residual (§5.5)
    const int64_t n = p.n;
    const int ns = h->nseg;
    std::vector<double> bn2(size_t(nrhs) * ns), rn2(size_t(nrhs) * ns);
    ck(launch_colnorm2(b, ldb, h->seg_ptr, ns, n, nrhs, h->norms, s));
    h->prof.count(P_OTHER, 1);
    ck(cudaMemcpyAsync(bn2.data(), h->norms, sizeof(double) * nrhs * ns, cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    const int maxit = o->maxit > 0 ? o->maxit : 50;
    double res = INFINITY;
    int it = 0;
    precond(h, b, ldb, x, ldx, nrhs);  // x_0 = M^-1 b
    for (;;) {
      h2_matvec(h, x, ldx, h->vecT, n, nrhs);
      ck(launch_residual(b, ldb, h->vecT, n, h->vecR, n, h->seg_ptr, ns, n, nrhs, h->norms, s));
      h->prof.count(P_OTHER, 1);
      ck(cudaMemcpyAsync(rn2.data(), h->norms, sizeof(double) * nrhs * ns, cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));
      res = 0.0;  // worst system, worst column
      for (size_t q = 0; q < rn2.size(); ++q) res = std::max(res, std::sqrt(rn2[q] / std::max(bn2[q], 1e-300)));
      if (!(res > o->tol) || it >= maxit) break;
      precond(h, h->vecR, n, h->vecT, n, nrhs);
      ck(launch_axpy(h->vecT, n, x, ldx, n, nrhs, s));
      h->prof.count(P_OTHER, 1);
      ++it;
    }
    if (info) {
      info->iters = it;
      info->rel_residual = res;
      info->status = (res <= o->tol) ? H2SP_OK : H2SP_ENOCONV;
    }
    {
      const int ss = sweep_status(h);
      if (ss != H2SP_OK) return ss;
    }
    if (!(res <= o->tol)) return H2SP_ENOCONV;
  } catch (const CudaFail &f) {
    return status_of(f.e);
  }
  return H2SP_OK;
}

int h2sp_solve_host(const h2sp_handle *an, const h2sp_h2_desc *desc, const h2sp_opts *opts, int32_t prec,
                    const h2sp_solve_opts *sopts, int32_t nrhs, const double *b, int64_t ldb, double *x, int64_t ldx,
                    h2sp_solve_info *info, h2sp_stream stream) {
  if (!desc || !sopts || !b || !x || nrhs <= 0 || nrhs > 64) return H2SP_EINVAL;
  if (ldb < desc->n || ldx < desc->n) return H2SP_EINVAL;
  h2sp_handle *own = nullptr;
  if (an == nullptr) {
    // validates the structure and plans it
    const int st = h2sp_analyze(desc, &own);
    if (st != H2SP_OK) return st;
    an = own;
  } else if (!an->plan_ptr || !an->cell || !same_structure(an, desc)) {
    return H2SP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<void *> bufs;
  h2sp_handle *h = nullptr;
  int st = H2SP_OK;
  try {
    init_pool_once();
    const NumericSizes z = numeric_sizes(desc);
    auto up = [&](const double *src, int64_t n) -> const double * {
      if (src == nullptr) return nullptr;
      void *p = nullptr;
      ck(malloc_async(&p, size_t(std::max<int64_t>(n, 1)) * sizeof(double), s));
      bufs.push_back(p);
      if (n > 0) ck(cudaMemcpyAsync(p, src, size_t(n) * sizeof(double), cudaMemcpyHostToDevice, s));
      return static_cast<const double *>(p);
    };
    h2sp_h2_desc dd = *desc;
    dd.leaf_basis = up(desc->leaf_basis, z.leaf);
    dd.transfer = up(desc->transfer, z.transfer);
    dd.coupling = up(desc->coupling, z.coupling);
    dd.near_block = up(desc->near_block, z.near);
    dd.col_leaf_basis = up(desc->col_leaf_basis, z.col_leaf);
    dd.col_transfer = up(desc->col_transfer, z.col_transfer);
    const int64_t n = desc->n;
    void *db = nullptr, *dx = nullptr;
    ck(malloc_async(&db, size_t(std::max<int64_t>(n * nrhs, 1)) * sizeof(double), s));
    bufs.push_back(db);
    ck(malloc_async(&dx, size_t(std::max<int64_t>(n * nrhs, 1)) * sizeof(double), s));
    bufs.push_back(dx);
    if (n > 0)
      ck(cudaMemcpy2DAsync(db, size_t(n) * sizeof(double), b, size_t(ldb) * sizeof(double), size_t(n) * sizeof(double),
                           size_t(nrhs), cudaMemcpyHostToDevice, s));
    st = h2sp_sparsify_analyzed(an, &dd, opts, stream, &h);
    if (st == H2SP_OK) st = h2sp_factor(h, prec, stream);
    if (st == H2SP_OK) {
      st = h2sp_solve(h, sopts, nrhs, static_cast<const double *>(db), n, static_cast<double *>(dx), n, info, stream);
      if (st == H2SP_OK || st == H2SP_ENOCONV) {
        if (n > 0)
          ck(cudaMemcpy2DAsync(x, size_t(ldx) * sizeof(double), dx, size_t(n) * sizeof(double),
                               size_t(n) * sizeof(double), size_t(nrhs), cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
      }
    }
  } catch (const CudaFail &f) {
    st = status_of(f.e);
  }
  if (h) h2sp_destroy(h);
  for (void *p : bufs) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  if (own) h2sp_destroy(own);
  return st;
}

int h2sp_solve_captured(h2sp_handle *h, int32_t steps, double tol, int32_t nrhs, const double *b, int64_t ldb,
                        double *x, int64_t ldx, h2sp_solve_info *info, h2sp_stream stream) {
  if (!h || !b || !x || nrhs <= 0 || nrhs > 64 || steps < 0 || steps > 100) return H2SP_EINVAL;
  if (!h->device_ready) return H2SP_ESTATE;
  const Plan &p = (*h->plan_ptr);
  if (ldb < p.n || ldx < p.n) return H2SP_EINVAL;
  if (h->prec < 0 || h->ilut) return H2SP_ESTATE;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->prof.stream = h->stream;
  cudaStream_t s = h->stream;
  const int64_t n = p.n;
  const int ns = h->nseg;
  bool capturing = false;
  try {
    // every buffer the captured launches use exists before the capture
    ensure_vectors(h, nrhs);
    ensure_work(h, nrhs);
    if (h->prec == H2SP_FP32 && fp32_applies_enabled()) ensure_vectors_f32(h, nrhs);
    if (h->cap_norms == nullptr) h->cap_norms = h->alloc<double>(size_t(2) * ns * 64);
    if (h->graph_stream == nullptr) {
      ck(cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking));
      ck(cudaEventCreateWithFlags(&h->graph_in, cudaEventDisableTiming));
      ck(cudaEventCreateWithFlags(&h->graph_out, cudaEventDisableTiming));
    }
    const bool same = h->solve_exec && h->cap_b == b && h->cap_x == x && h->cap_ldb == ldb && h->cap_ldx == ldx &&
                      h->cap_nrhs == nrhs && h->cap_steps == steps && h->cap_prec == h->prec;
    if (!same && h->solve_exec) {
      ck(cudaGraphExecDestroy(h->solve_exec));
      h->solve_exec = nullptr;
    }
    cudaStream_t gs = h->graph_stream;
    if (h->solve_exec == nullptr) {
      ck(cudaStreamSynchronize(s));
      const int timing = h->prof.timing;
      h->prof.timing = 0;
      h->stream = gs;
      ck(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
      capturing = true;
      // the sweeps' flags start from zero in every replay, so the epochs
      // captured with the launches are new each time
      if (h->chain_flags) ck(cudaMemsetAsync(h->chain_flags, 0, sizeof(int) * size_t(h->sdev->nflags), gs));
      double *bn2 = h->cap_norms, *rn2 = h->cap_norms + size_t(ns) * 64;
      ck(launch_colnorm2(b, ldb, h->seg_ptr, ns, n, nrhs, bn2, gs));
      precond(h, b, ldb, x, ldx, nrhs);  // x_0 = M^-1 b
      for (int k = 0; k < steps; ++k) {
        h2_matvec(h, x, ldx, h->vecT, n, nrhs);
        ck(launch_residual(b, ldb, h->vecT, n, h->vecR, n, h->seg_ptr, ns, n, nrhs, rn2, gs));
        precond(h, h->vecR, n, h->vecT, n, nrhs);
        ck(launch_axpy(h->vecT, n, x, ldx, n, nrhs, gs));
      }
      h2_matvec(h, x, ldx, h->vecT, n, nrhs);
      ck(launch_residual(b, ldb, h->vecT, n, h->vecR, n, h->seg_ptr, ns, n, nrhs, rn2, gs));
      cudaGraph_t g = nullptr;
      capturing = false;
      const cudaError_t ee = cudaStreamEndCapture(gs, &g);
      h->stream = s;
      h->prof.timing = timing;
      ck(ee);
      const cudaError_t ie = cudaGraphInstantiate(&h->solve_exec, g, 0);
      cudaGraphDestroy(g);
      ck(ie);
      h->cap_b = b, h->cap_x = x, h->cap_ldb = ldb, h->cap_ldx = ldx;
      h->cap_nrhs = nrhs, h->cap_steps = steps, h->cap_prec = h->prec;
    }
    ck(cudaEventRecord(h->graph_in, s));
    ck(cudaStreamWaitEvent(gs, h->graph_in, 0));
    ck(cudaGraphLaunch(h->solve_exec, gs));
    ck(cudaEventRecord(h->graph_out, gs));
    ck(cudaStreamWaitEvent(s, h->graph_out, 0));
    std::vector<double> nb(size_t(ns) * nrhs), nr(size_t(ns) * nrhs);
    ck(cudaMemcpyAsync(nb.data(), h->cap_norms, sizeof(double) * nb.size(), cudaMemcpyDeviceToHost, s));
    ck(cudaMemcpyAsync(nr.data(), h->cap_norms + size_t(ns) * 64, sizeof(double) * nr.size(), cudaMemcpyDeviceToHost,
                       s));
    ck(cudaStreamSynchronize(s));
    double res = 0.0;  // worst system, worst column
    for (size_t q = 0; q < nr.size(); ++q) res = std::max(res, std::sqrt(nr[q] / std::max(nb[q], 1e-300)));
    const int ss = sweep_status(h);
    const int st = ss != H2SP_OK ? ss : (res <= tol ? H2SP_OK : H2SP_ENOCONV);
    if (info) {
      info->iters = steps;
      info->rel_residual = res;
      info->status = st;
    }
    return st;
  } catch (const CudaFail &f) {
    if (capturing) {
      cudaGraph_t g = nullptr;
      if (cudaStreamEndCapture(h->graph_stream, &g) == cudaSuccess && g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
    h->stream = s;
    return status_of(f.e);
  }
}

int h2sp_export_S(h2sp_handle *h, int64_t *node_size, int64_t *brow_ptr, int32_t *bcol_idx, int64_t *val_off,
                  double *vals, h2sp_stream stream) {
  if (!h) return H2SP_EINVAL;
  const Plan &p = (*h->plan_ptr);
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  if (node_size) std::copy(p.node_size.begin(), p.node_size.end(), node_size);
  if (brow_ptr) std::copy(p.brow_ptr.begin(), p.brow_ptr.end(), brow_ptr);
  if (bcol_idx) std::copy(p.bcol.begin(), p.bcol.end(), bcol_idx);
  if (val_off) std::copy(p.val_off.begin(), p.val_off.end(), val_off);
  if (!vals) return H2SP_OK;
  if (!h->device_ready) return H2SP_ESTATE;
  try {
    copy_out(h, vals, h->S, p.s_elems);
  } catch (const CudaFail &f) {
    return status_of(f.e);
  }
  return H2SP_OK;
}

int h2sp_logdet(h2sp_handle *h, double *logabsdet, int32_t *sign, h2sp_stream stream) {
  if (!h || !logabsdet) return H2SP_EINVAL;
  if (!h->device_ready || h->prec < 0 || h->ilut) return H2SP_ESTATE;
  const Plan &p = (*h->plan_ptr);
  const int nsys = p.level_ptr[1];
  const int nfront = int(p.fronts.size());
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->prof.stream = h->stream;
  try {
    if (h->ld_sys_ptr == nullptr) {
      // system of a front = root of its supernode's closure cluster
      std::vector<int32_t> ptr(static_cast<size_t>(nsys) + 1, 0), fronts(static_cast<size_t>(nfront));
      std::vector<int32_t> sys(static_cast<size_t>(nfront));
      for (int k = 0; k < nfront; ++k) {
        sys[size_t(k)] = p.root[p.closure[p.order[p.sn_ptr[k]]]];
        ptr[size_t(sys[size_t(k)]) + 1]++;
      }
      for (int w = 0; w < nsys; ++w) ptr[size_t(w) + 1] += ptr[size_t(w)];
      std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
      for (int k = 0; k < nfront; ++k) fronts[size_t(fill[size_t(sys[size_t(k)])]++)] = k;
      h->ld_sys_front = h->upload(fronts);
      h->ld_lsum = h->alloc<double>(size_t(nfront));
      h->ld_flips = h->alloc<int>(size_t(nfront));
      h->ld_out = h->alloc<double>(size_t(nsys));
      h->ld_sign = h->alloc<int32_t>(size_t(nsys));
      h->ld_sys_ptr = h->upload(ptr);  // last: marks the buffers above as ready
    }
    if (h->prec == H2SP_FP64)
      ck(launch_logdet<double>(h->fr, nfront, static_cast<const double *>(h->fronts), h->piv, h->ld_sys_ptr,
                               h->ld_sys_front, nsys, h->ld_lsum, h->ld_flips, h->ld_out, h->ld_sign, h->stream,
                               &h->prof));
    else
      ck(launch_logdet<float>(h->fr, nfront, static_cast<const float *>(h->fronts), h->piv, h->ld_sys_ptr,
                              h->ld_sys_front, nsys, h->ld_lsum, h->ld_flips, h->ld_out, h->ld_sign, h->stream,
                              &h->prof));
    std::vector<double> l(static_cast<size_t>(nsys));
    std::vector<int32_t> g(static_cast<size_t>(nsys));
    ck(cudaMemcpyAsync(l.data(), h->ld_out, sizeof(double) * size_t(nsys), cudaMemcpyDeviceToHost, h->stream));
    ck(cudaMemcpyAsync(g.data(), h->ld_sign, sizeof(int32_t) * size_t(nsys), cudaMemcpyDeviceToHost, h->stream));
    ck(cudaStreamSynchronize(h->stream));
    std::copy(l.begin(), l.end(), logabsdet);
    if (sign) std::copy(g.begin(), g.end(), sign);
  } catch (const CudaFail &f) {
    return status_of(f.e);
  }
  return H2SP_OK;
}

int h2sp_export_Q(h2sp_handle *h, int32_t cluster, int32_t col, int64_t *m, double *q, h2sp_stream stream) {
  if (!h || !m) return H2SP_EINVAL;
  const Plan &p = (*h->plan_ptr);
  if (cluster < 0 || cluster >= p.ncl) return H2SP_EINVAL;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  if (p.q_off[cluster] < 0) {
    *m = 0;
    return H2SP_OK;
  }
  *m = p.m[cluster];
  if (q && !h->device_ready) return H2SP_ESTATE;
  if (q) {
    try {
      ck(cudaMemcpyAsync(q, (col ? h->Qc : h->Q) + p.q_off[cluster], sizeof(double) * p.m[cluster] * p.m[cluster],
                         cudaMemcpyDeviceToHost, h->stream));
      ck(cudaStreamSynchronize(h->stream));
    } catch (const CudaFail &f) {
      return status_of(f.e);
    }
  }
  return H2SP_OK;
}

int h2sp_export_structure(h2sp_handle *h, int32_t *node_level, int32_t *node_cluster, int32_t *closure,
                          int32_t *order, int32_t *sn_ptr, int32_t *bnd_ptr, int32_t *bnd, int64_t *nbnd) {
  if (!h) return H2SP_EINVAL;
  const Plan &p = (*h->plan_ptr);
  if (node_level) std::copy(p.node_level.begin(), p.node_level.end(), node_level);
  if (node_cluster) std::copy(p.node_cluster.begin(), p.node_cluster.end(), node_cluster);
  if (closure) std::copy(p.closure.begin(), p.closure.end(), closure);
  if (order) std::copy(p.order.begin(), p.order.end(), order);
  if (sn_ptr) std::copy(p.sn_ptr.begin(), p.sn_ptr.end(), sn_ptr);
  if (bnd_ptr) std::copy(p.bnd_ptr.begin(), p.bnd_ptr.end(), bnd_ptr);
  if (bnd) std::copy(p.bnd.begin(), p.bnd.end(), bnd);
  if (nbnd) *nbnd = int64_t(p.bnd.size());
  return H2SP_OK;
}

int h2sp_export_schedule(h2sp_handle *h, int32_t *lstop, int64_t *m, int64_t *kp, int64_t *off, int64_t *xoff,
                         int64_t *node_off, int32_t *node_cluster) {
  if (!h || !h->plan_ptr) return H2SP_EINVAL;
  const Plan &p = (*h->plan_ptr);
  A1Result r;
  std::string err;
  const int st = device_schedule(p, &r, nullptr, err);
  if (st != H2SP_OK) {
    g_cuda_err = err;
    return st;
  }
  if (lstop) *lstop = r.lstop;
  if (m) std::copy(r.m.begin(), r.m.end(), m);
  if (kp) std::copy(r.kp.begin(), r.kp.end(), kp);
  if (off) std::copy(r.off.begin(), r.off.end(), off);
  if (xoff) std::copy(r.xoff.begin(), r.xoff.end(), xoff);
  if (node_off) std::copy(r.node_off.begin(), r.node_off.end(), node_off);
  if (node_cluster) std::copy(r.node_cluster.begin(), r.node_cluster.end(), node_cluster);
  return H2SP_OK;
}

int h2sp_export_near(h2sp_handle *h, int32_t level, int64_t *ptr, int32_t *col, int64_t *nnz) {
  if (!h || !h->plan_ptr) return H2SP_EINVAL;
  const Plan &p = (*h->plan_ptr);
  A1Result r;
  std::string err;
  const int st = device_schedule(p, &r, nullptr, err);
  if (st != H2SP_OK) {
    g_cuda_err = err;
    return st;
  }
  if (level < 1 || level > r.lstop) return H2SP_EINVAL;
  const auto &P = r.near_ptr[size_t(level)];
  const auto &C = r.near_col[size_t(level)];
  if (nnz) *nnz = int64_t(C.size());
  if (ptr) std::copy(P.begin(), P.end(), ptr);
  if (col) std::copy(C.begin(), C.end(), col);
  return H2SP_OK;
}

int h2sp_export_front(h2sp_handle *h, int32_t k, int64_t *f, int64_t *sz, double *vals, h2sp_stream stream) {
  if (!h) return H2SP_EINVAL;
  const Plan &p = (*h->plan_ptr);
  if (k < 0 || k >= int32_t(p.fronts.size())) return H2SP_EINVAL;
  const Front &F = p.fronts[size_t(k)];
  if (f) *f = F.f;
  if (sz) *sz = F.s;
  if (!vals) return H2SP_OK;
  if (!h->device_ready || h->prec < 0 || h->ilut) return H2SP_ESTATE;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  try {
    const size_t esz = h->prec == H2SP_FP32 ? sizeof(float) : sizeof(double);
    std::vector<unsigned char> tmp(size_t(F.f) * size_t(F.f) * esz);
    const unsigned char *src = static_cast<const unsigned char *>(h->fronts) + size_t(F.off) * esz;
    if (F.f > 0)
      ck(cudaMemcpy2DAsync(tmp.data(), size_t(F.f) * esz, src, size_t(F.ld) * esz, size_t(F.f) * esz, size_t(F.f),
                           cudaMemcpyDeviceToHost, h->stream));
    ck(cudaStreamSynchronize(h->stream));
    const size_t n = size_t(F.f) * size_t(F.f);
    if (esz == sizeof(float))
      for (size_t i = 0; i < n; ++i) vals[i] = double(reinterpret_cast<const float *>(tmp.data())[i]);
    else
      std::memcpy(vals, tmp.data(), n * sizeof(double));
  } catch (const CudaFail &e) {
    return status_of(e.e);
  }
  return H2SP_OK;
}

int h2sp_set_option(h2sp_handle *h, int32_t option, int64_t value) {
  if (!h) return H2SP_EINVAL;
  switch (option) {
    case H2SP_OPTION_WAIT_POLLS:
      if (value < 1 || value > (int64_t(1) << 31)) return H2SP_EINVAL;
      h->chain_spin_cap = uint32_t(value);
      return H2SP_OK;
    case H2SP_OPTION_TEST_STALE_EPOCH:
      h->test_stale_epoch = value != 0;
      return H2SP_OK;
    case H2SP_OPTION_CHOL_TILES_PER_CTA:
      if (value < 0 || value > (1 << 20)) return H2SP_EINVAL;
      h->chol_sched.tiles_per_cta = int(value);
      return H2SP_OK;
    case H2SP_OPTION_CHOL_PANEL_SMS:
      if (value < -1 || value > 4096) return H2SP_EINVAL;
      h->chol_sched.panel_sms = int(value);
      return H2SP_OK;
    case H2SP_OPTION_CHOL_LOOKAHEAD:
      h->chol_sched.lookahead = value != 0;
      return H2SP_OK;
    case H2SP_OPTION_CHOL_WIDE:
      if (value < 0 || value > 2) return H2SP_EINVAL;
      h->chol_sched.wide = int(value);
      return H2SP_OK;
    default:
      return H2SP_EINVAL;
  }
}

int h2sp_measure_peak(int32_t kind, double *tflops, h2sp_stream stream) {
  if (!tflops || (kind != 0 && kind != 1)) return H2SP_EINVAL;
  *tflops = 0.0;
  try {
    ck(measure_fma_peak(kind, tflops, reinterpret_cast<cudaStream_t>(stream)));
  } catch (const CudaFail &f) {
    return status_of(f.e);
  }
  return H2SP_OK;
}

int h2sp_query(const h2sp_handle *h, h2sp_stats *st) {
  if (!h || !st) return H2SP_EINVAL;
  const Plan &p = (*h->plan_ptr);
  std::memset(st, 0, sizeof(*st));
  st->n = p.n;
  st->depth = p.D;
  st->lstop = p.lstop;
  st->nnodes = int32_t(p.node_size.size());
  st->nnzb = int64_t(p.bcol.size());
  st->nnz = p.s_elems;
  st->nsupernodes = int32_t(p.fronts.size());
  st->nfront_levels = int32_t(h->flev.size());
  st->max_front = p.max_front;
  st->front_elems = p.front_elems;
  st->factor_flops = p.factor_flops;
  st->sparsify_flops = p.sparsify_flops;
  st->factor_prec = h->prec;
  st->factor_chol = h->prec >= 0 && h->chol ? 1 : 0;
  st->chol_flops = p.chol_flops;
  st->compensated_pivots = h->prec >= 0 ? h->compensated : 0;
  st->sparsify_prec = h->device_ready ? h->sp_prec : -1;
  st->plan_seconds = h->plan_seconds;
  st->nsys = p.level_ptr[1];
  return H2SP_OK;
}

int h2sp_h2_matvec_static(const h2sp_handle *h, int32_t nrhs, const double *x, int64_t ldx, double *y, int64_t ldy,
                          h2sp_stream stream) {
  if (!h || !x || !y || nrhs <= 0) return H2SP_EINVAL;
  if (!h->device_ready) return H2SP_ESTATE;
  const Plan &p = (*h->plan_ptr);
  if (ldx < p.n || ldy < p.n) return H2SP_EINVAL;
  const int64_t ldh = std::max<int64_t>(p.xh_elems, 1);
  const int64_t need = 2 * ldh * 16;  // x^ and y^, 16 right-hand sides per pass
  if (need > kStaticScratchElems) {
    g_cuda_err = "h2sp_h2_matvec_static: needs " + std::to_string(need) + " doubles of workspace, the static array has " +
                 std::to_string(kStaticScratchElems);
    return H2SP_EUNSUPPORTED;
  }
  // the structure pointers belong to the device the handle was built on; the
  // static array's address is looked up for the current device
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || !h->sdev || dev != h->sdev->device) {
    g_cuda_err = "h2sp_h2_matvec_static: the current device (" + std::to_string(dev) +
                 ") is not the device the handle was built on (" + std::to_string(h->sdev ? h->sdev->device : -1) + ")";
    return H2SP_EINVAL;
  }
  try {
    double *scratch = nullptr;
    ck(static_scratch_address(&scratch));
    ck(launch_h2_matvec(h->h2, p.level_ptr.data(), h->child_start, h->child_cnt, p.D, x, ldx, y, ldy, nrhs, scratch,
                        scratch + ldh * 16, ldh, reinterpret_cast<cudaStream_t>(stream)));
  } catch (const CudaFail &f) {
    return status_of(f.e);
  }
  return H2SP_OK;
}

int h2sp_profile(h2sp_handle *h, int32_t timing, int32_t reset, h2sp_kernel_times *out) {
  if (!h) return H2SP_EINVAL;
  if (h->device_ready) h->prof.collect();
  if (out) {
    std::memset(out, 0, sizeof(*out));
    for (int c = 0; c < P_NCLASS && c < 16; ++c) {
      out->launches[c] = h->prof.launches[c];
      out->timed[c] = h->prof.timed[c];
      out->ms[c] = h->prof.ms[c];
      out->work[c] = h->prof.work[c];
    }
  }
  if (reset) h->prof.reset();
  if (timing >= 0) h->prof.timing = timing != 0 && h->device_ready;
  return H2SP_OK;
}

void h2sp_destroy(h2sp_handle *h) {
  if (!h) return;
  h->release();
  delete h;
}

}  // extern "C"
