// hb_internal.cuh - handle layout and helpers shared by the library's
// translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <functional>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hb.h"

namespace hb {

// ------------------------------------------------------------- errors ----
struct Error {
  hb_status code;
  std::string msg;
};

#define HB_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      throw ::hb::Error{HB_ERR_CUDA, std::string(#call) + ": " +              \
                                         cudaGetErrorString(e_)};              \
    }                                                                          \
  } while (0)

#define HB_CHECK_LAUNCH() HB_CUDA(cudaGetLastError())

inline Error arg_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return Error{HB_ERR_ARG, buf};
}

// A named NVTX range for the scope (build stages, apply phases; no-ops
// unless a profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Every device allocation of the library goes through the registry
// (api.cu): it counts the live bytes, applies the optional cap of
// hb_device_alloc_cap (a cap that would be exceeded fails like a real
// out-of-memory, HB_ERR_OOM), and records the allocations made while a
// BuildAllocs scope is open on the calling thread.
void* registry_alloc(size_t bytes);   // throws Error (HB_ERR_OOM / HB_ERR_CUDA)
void registry_free(void* p);

// The allocations made by one hb_build: on failure free_all() releases
// those still live, so that a failed build leaves nothing behind.
class BuildAllocs {
 public:
  BuildAllocs();
  ~BuildAllocs();
  void free_all();
  BuildAllocs(const BuildAllocs&) = delete;
  BuildAllocs& operator=(const BuildAllocs&) = delete;
};

// Device allocation that reports HB_ERR_OOM.
template <class T>
T* dev_alloc(size_t count) {
  if (count == 0) count = 1;
  return static_cast<T*>(registry_alloc(count * sizeof(T)));
}

inline void dev_free(void* p) {
  if (p) registry_free(p);
}

template <class T>
T* upload(const std::vector<T>& v, cudaStream_t st = 0) {
  T* d = dev_alloc<T>(v.size());
  if (!v.empty()) {
    const cudaError_t e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      dev_free(d);
      throw Error{HB_ERR_CUDA, std::string("upload cudaMemcpyAsync: ") + cudaGetErrorString(e)};
    }
  }
  return d;
}

// ------------------------------------------------------ entry context ----
// Everything a kernel needs to evaluate K_ij (passed by value).
struct EntryParams {
  int nx, ny, nI;
  int NI;
  double omega;
  const double* LX;      // nx x nI   l_k(x_a)
  const double* LZ;      // ny x nI   l_k(z_b)
  const double* H;       // 3 x ny x NI x nI  (see entries.cu)
  const double2* self;   // Nv self terms K_ii
};

// ------------------------------------------------------ butterfly plan ----
// One step task: Y (r_out x R) (=|+=) sum_{t < nterm} op_t(F_t) X_t, with
// op(F) = F (F stored column-major r_out x r_in, ld = r_out) or, when
// conj_t, op(F) = F^H (F stored column-major r_in x r_out, ld = r_in).
// Vector buffers are row-major with the R right-hand sides contiguous:
// buffer 0 = x (tree-ordered input), 1 = y (tree-ordered output), 2 = xh
// (all butterfly intermediate vectors).
struct Task {
  long long y_off;
  long long f_off[2];
  long long x_off[2];
  int r_out;
  int r_in[2];
  unsigned char nterm, x_buf, y_buf, accumulate;
  unsigned char conj_t, kind, pad0, pad1;
};

// Native (MMA-fragment) layout of the mixed apply (bf_mma.cu).  A factor
// block op(F) (outputs x inputs) is stored as tiles of 8 outputs x 8 inputs
// (512 bytes); the n-tiles are cut into groups of ng (the last group may be
// smaller) and tiles are ordered [group][k-step][n-tile in group]; rows of a
// block part are padded to a multiple of 8 with zeros.  NatBlock says where
// a native block comes from: the column-major FP64 block at src_off
// (leading dimension ld), op = identity or conjugate transpose, outputs in
// one or two parts (r1, r2) and inputs in one or two parts (k1, k2), each
// part padded on its own.
struct NatBlock {
  long long src_off;
  long long tile0;       // first tile in the native arena
  int ld, conj;
  int r1, r2, k1, k2;
  int ng;                // n-tiles per group
  int pad;
};
// One term of a native task: ks k-steps of the block at f_tile, input row
// tiles x_tile .. x_tile + ks of buffer x_buf (0 = x, 1 = y, 2 = xh).
struct NatTerm {
  long long f_tile;
  long long x_tile;
  int ks;
  int x_buf;
};
// A task writes nt row tiles of buffer y_buf from y_tile on as the sum of
// its terms; depth d reads only what depths < d wrote.  tc_out: only the
// leaf outputs read what it writes (the tensor-core leaf kernel can take
// it in its operand layout).
struct NatTask {
  long long y_tile;
  int nt;
  int depth;
  int y_buf;
  int ng;                // n-tiles per group of its blocks
  bool tc_out = false;
  long long row_lo = 0, row_hi = 0;   // tree-position rows of its row node (a shard runs the tasks meeting its rows)
  // cone of the first butterfly levels (forward: blocks of one column group,
  // adjoint: one row group; closed under the dependencies of those levels):
  // cone id (-1: none) and the task's level within it
  long long cone = -1;
  int cone_level = 0;
  std::vector<NatTerm> terms;
};

// Tensor-core leaf outputs (leaf_tc.cu).  TcBlock: outputs o0 .. o0 + nout
// (<= 64) of op(F) (as NatBlock: column-major FP64 block at src_off, leading
// dimension ld, conjugate transpose when conj) with k inputs, converted to
// ceil(k / 8) 4 KB units from unit0 of the tc arena.  TcTerm: nkg units
// from unit0 times the input row tiles x_tile .. (x_buf 0 = the operand-layout
// copy of x, 2 = xh).  TcChainHost: one chain of up to 64 outputs from padded
// row tile y_tile on, written to u in natural order.
struct TcBlock {
  long long src_off;
  long long unit0;
  int ld, conj;
  int o0, nout, k;
  int pad;
};
struct TcTerm {
  long long unit0;
  long long x_tile;
  int nkg;
  int x_buf;
};
struct TcChainHost {
  long long y_tile;
  int nout;
  std::vector<TcTerm> terms;
};

// Factor index of one butterfly (what hb_save writes besides the arena):
// level-k block (i, j) = rank[k][i 2^(L-k) + j] x (its columns), stored
// column-major at f_off[k][.] of the FP64 arena; K^L block i at kl_off[i].
struct BflyIndex {
  int l, oi, si, L;
  std::vector<std::vector<int>> rank;
  std::vector<std::vector<long long>> f_off;
  std::vector<long long> kl_off;
};

// A sampled block that hb_build decomposed, kept on request
// (hb_record_id_blocks) so that a test can run the oracle's ID on exactly the
// same samples.
struct IdRecord {
  int level = 0;                       // butterfly level k of the block
  std::vector<long long> rows, cols;   // natural indices (proxy rows, column set)
  std::vector<double2> A;              // rows x cols, column-major, as sampled
  int rank = 0;
  std::vector<int> piv;                // full pivot order (positions in cols)
};

// Host-side batch of ragged entry blocks (entries.cu).
struct BlockMeta {
  long long row_off, m, col_off, n, out_off, seg_off, nseg, pad;
};
struct BlockBatchHost {
  std::vector<BlockMeta> meta;
  std::vector<long long> rows, cols, segs, items;
  std::vector<int> rdst;
};

}  // namespace hb

struct hb_ctx {
  // problem
  int nx = 0, ny = 0;
  long long Nv = 0;
  double x0 = 0, y0 = 0, h = 0, omega = 0;
  int nI = 0, NI = 0;
  hb_options opt{};
  std::string err;
  std::vector<double> nodes_x, nodes_y, n_cells;
  std::vector<double> tab[3];  // tau2, v0, v1 row-major NI x NI

  // device: interpolation and self terms
  double* d_nodes = nullptr;   // nodes_x then nodes_y
  double* d_tab = nullptr;     // 3 x NI x NI (forward), then 3 x NI x NI transposed
  double* d_LX = nullptr;
  double* d_LZ = nullptr;
  double* d_H[2] = {nullptr, nullptr};
  double* d_ncell = nullptr;
  double2* d_self = nullptr;

  // cluster tree
  int Lv = 0;
  std::vector<long long> perm;               // tree position -> natural index
  std::vector<long long> iperm;              // natural index -> tree position
  std::vector<std::vector<long long>> bounds;
  long long* d_perm = nullptr;

  // build results
  bool built = false;
  std::vector<hb::BflyIndex> bidx;   // factor index of every butterfly (HODBF order)
  std::vector<long long> leaf_off;   // dense leaf blocks in the FP64 arena
  hb_stats stats{};
  // FP64 factor arena (double2, column-major blocks)
  long long n_factor = 0;
  double2* d_f64 = nullptr;
  // native split-BF16 arenas of the mixed apply: [0] forward, [1] adjoint (512-byte tiles)
  uint4* d_nat[2] = {nullptr, nullptr};
  // operand-layout arenas of the tensor-core leaf outputs (4 KB units) and their plans
  uint4* d_tc[2] = {nullptr, nullptr};
  void* tc_plan[2] = {nullptr, nullptr};
  long long nat_tiles[2] = {0, 0};
  std::vector<long long> leaf_tile;   // first padded row tile of every leaf (+ total)
  long long nv_tiles = 0;             // row tiles of the padded tree-ordered vectors
  long long xh_tiles = 0;             // row tiles of the padded intermediate vectors
  long long* d_pperm = nullptr;       // padded row -> natural index (-1: padding)
  // apply plans: steps[0] forward, steps[1] adjoint; each step = task range
  std::vector<int> step_begin[2];
  std::vector<hb::Task> tasks_h[2];
  std::vector<std::pair<long long, long long>> task_rows[2];   // tree-position rows each task serves
  hb::Task* d_tasks[2] = {nullptr, nullptr};
  void* flow_plan[2] = {nullptr, nullptr};  // mixed apply plans (bf_mma.cu)
  int* h_err = nullptr;                    // mapped pinned error word of bounded device waits
  int* d_err = nullptr;
  bool wait_selftest = false;              // hb_set_wait_selftest
  long long xh_rows = 0;
  int max_rank = 0;

  // apply scratch (sized for cap_rhs right-hand sides)
  int cap_rhs = 0;
  void* d_x = nullptr;
  void* d_y = nullptr;
  void* d_xh = nullptr;
  // mixed apply scratch (native layout, up to 32 right-hand sides)
  uint4* d_mx = nullptr;
  uint4* d_mx_tc = nullptr;   // x again in the tensor-core operand layout
  uint4* d_mxh = nullptr;
  // readiness flags of the dataflow launch (x row tiles, then xh row tiles)
  // and its launch counter ([0] launches completed, [1] CTAs done)
  unsigned* d_flags = nullptr;
  unsigned* d_epoch = nullptr;
  // dense apply: per-split partial sums when source lines are split over CTAs
  double2* d_dense_part = nullptr;
  size_t dense_part_cap = 0;

  // curve inclusion (inclusion.cu): segments and the dense surface operators
  long long ns = 0;                // segments; 0: no curve set
  double2* d_seg = nullptr;        // ns centres (x, z)
  double* d_segw = nullptr;        // ns lengths
  double* d_segn = nullptr;        // ns values of n at the centres
  double2* d_cellpts = nullptr;    // N_v cell centres (x, z)
  double2* d_lu = nullptr;         // K^{s2s} LU-factored in place (ns x ns, column-major)
  int* d_piv = nullptr;            // its row interchanges
  double2* d_inv = nullptr;        // (K^{s2s})^{-1} from the LU factors, ns x ns column-major
  double2* d_kv2s = nullptr;       // K^{v2s}, ns x N_v column-major
  double2* d_ks2v = nullptr;       // K^{s2v}, N_v x ns column-major
  double2* d_cy = nullptr;         // surface vectors of an apply, 2 ns x cy_cap (Y, then P)
  int cy_cap = 0;
  void* curve_bf[2] = {nullptr, nullptr};   // hb_curve_compress: K^{v2s} (0), K^{s2v} (1) as butterflies

  // hb_record_id_blocks: blocks per butterfly level to keep, and the kept ones
  int id_rec_per_level = 0;
  std::vector<hb::IdRecord> id_recs;

  // shards (hb_apply_shard*): filtered FP64 step lists by (direction, rows)
  std::map<std::tuple<int, long long, long long>, void*> shard_cache;

  // timing
  bool timing = false;
  std::vector<std::string> tnames;
  std::vector<double> tms;
  std::vector<long long> tcount;
};

namespace hb {
hb::EntryParams entry_params(const hb_ctx* c, int transposed);
void setup_tables(hb_ctx* c);                 // entries.cu
void compute_self(hb_ctx* c);                 // entries.cu
// sweep.cu: the table builder (arguments as hb_sweep_tables / hb_sweep_taylor)
void sweep_tables(int M, double lo, double h, int w0, int w1, int roi0, int roi1, const double* n_mesh, int NI,
                  const double* px, const double* pz, int ns, const int* src, const double* taylor, int max_iter,
                  double tol, double* tau2, double* v0, double* v1, double* info);
void sweep_taylor_one(const double* s2, double* out);
void dense_apply(hb_ctx* c, const double2* s, double2* u, int nrhs, int adjoint, cudaStream_t st);
void eval_entries(hb_ctx* c, const long long* rows, int m, const long long* cols, int n,
                  double2* out, cudaStream_t st);
void add_block(BlockBatchHost& B, const hb_ctx* c, const long long* rows, long long m,
               const long long* cols, long long n, long long out_off);
void run_blocks(hb_ctx* c, BlockBatchHost& B, double2* d_out, cudaStream_t st);
void id_batch(int count, const int* d_m, const int* d_n, const long long* d_aoff, double2* d_A,
              double eps, int* d_rank, int* d_perm, const long long* d_soff, int max_n, cudaStream_t st);
void emit_v(int count, const int* d_m, const int* d_n, const long long* d_aoff, const double2* d_A,
            const int* d_rank, const int* d_perm, const long long* d_soff, const long long* d_voff,
            int ld_is_rank, double2* V64, float2* V32, cudaStream_t st);
void build(hb_ctx* c);
void plans_from_index(hb_ctx* c);                      // build.cu: hb_load
void save_file(const hb_ctx* c, const char* path);     // io.cu
hb_ctx* load_file(const char* path,
                  hb_ctx* (*create)(const hb_grid*, const hb_tables*, double, const hb_options*));
void id_batch_noalloc(int count, const int* m, const int* n, const long long* a_off, double2* A, double eps,
                      int* rank, int* skel, double2* V, cudaStream_t st);
void flow_plan_build(const std::vector<NatTask>& tasks, void** plan_out);
void flow_plan_free(void* plan);
int flow_plan_depths(const void* plan);
// R <= 32 right-hand sides: gather of s (scaled), every depth, the last
// depth writing u (natural order) itself; one launch per depth or one
// persistent dataflow launch (flags / epoch: its readiness words)
void flow_launch(void* plan, void* tc_plan, const void* F_tc, const uint4* F, const double2* s, double scale,
                 uint4* x, uint4* x_tc, uint4* xh, double2* u, const long long* pperm, long long Nv,
                 long long nv_tiles, int R, unsigned* flags, unsigned* epoch, int* err, long long budget_cycles,
                 bool selftest, int autotune_on, cudaStream_t st, const std::function<void(int, bool)>& timer);
void flow_shape(const void* plan, int MT, int* mode, int* item_bytes, int* stages, int* pub, int* slack,
                double* tuned_ms, int* candidates);
void nat_convert(const double2* F64, const std::vector<NatBlock>& blocks, uint4* out, cudaStream_t st);
void tc_convert(const double2* F64, const std::vector<TcBlock>& blocks, void* out, cudaStream_t st);
void* tc_plan_build(std::vector<TcChainHost>&& chains);
void tc_plan_free(void* plan);
void tc_leaf_launch(void* plan, int MT, const void* F, const uint4* x, const uint4* xh, double2* u,
                    const long long* pperm, long long Nv, int R, int* err, long long budget, cudaStream_t st);
void gather_native(const double2* s, const long long* pperm, uint4* x, uint4* x_tc, long long nv_tiles, long long Nv,
                   int R, int MT, double scale, cudaStream_t st, long long win_lo = 0,
                   long long win_hi = (1LL << 62));
void apply_bf(hb_ctx* c, const double2* s, double2* u, int nrhs, int adjoint, int precision,
              cudaStream_t st);
// shards of the apply (apply.cu): rank `rank` of `nranks` owns node `rank` of
// level log2(nranks) of the cluster tree
void shard_rows(const hb_ctx* c, int nranks, int rank, long long* lo, long long* hi);
void apply_bf_shard(hb_ctx* c, const double2* s, double2* u, int nrhs, int adjoint, int precision, int nranks,
                    int rank, cudaStream_t st);
void shard_cache_free(hb_ctx* c);
void flow_launch_shard(void* plan, const uint4* F, const double2* s, double scale, uint4* x, uint4* xh,
                       long long xh_tiles, double2* u, const long long* pperm, long long Nv, long long nv_tiles,
                       int R, long long row_lo, long long row_hi, long long pad_lo, long long pad_hi, bool adjoint,
                       int* err, long long budget, cudaStream_t st);
// inclusion.cu
void curve_set(hb_ctx* c, const double* centers, const double* lengths, const double* n_seg, long long ns);
// One column of a sampled curve-operator block: rows' points obs[obs0,
// obs0 + m) against the source point src, times w, into out[out_off ..].
struct GreenCol {
  long long obs0;
  long long out_off;
  double2 src;
  double w;
  int m;
  int pad;
};
void green_jobs(const hb_ctx* c, const double2* d_obs, const GreenCol* d_jobs, long long njobs, double2* d_out,
                cudaStream_t st);   // inclusion.cu
// curve_bf.cu: K^{v2s} and K^{s2v} of the curve as butterflies
void curve_compress(hb_ctx* c, int leaf_s);
void curve_bf_free(hb_ctx* c);
void curve_bf_info(const hb_ctx* c, int which, int* levels, int* max_rank, long long* entries);
void curve_bf_apply(hb_ctx* c, int which, const double2* x_nat, long long ldx, double scale, double2* y_nat,
                    long long ldy, int accumulate, int nrhs, cudaStream_t st);
void run_tasks_fp64(const Task* d_tasks, int n, const double2* F, double2* x, double2* y, double2* xh, int R,
                    cudaStream_t st);   // apply.cu
void curve_free(hb_ctx* c);
void curve_operators(hb_ctx* c, double2* k_s2s, double2* k_v2s, double2* k_s2v, cudaStream_t st);
void apply_inclusion(hb_ctx* c, const double2* s, double2* u, int nrhs, int v2v_dense, cudaStream_t st);
void tree_build(hb_ctx* c);
// K-D tree over curve segment centres (same split rule on real coordinates)
void segment_tree_build(const double* cx, const double* cz, long long ns, int leaf, std::vector<long long>& perm,
                        std::vector<std::vector<long long>>& bounds);
// Eq. proxyv2v between two point sets (rows and seed columns in real coordinates)
void point_proxy_rows(const double* rows_xz, long long t0, long long t1, const double* seeds_xz, int nseeds,
                      double chi, double radius, std::vector<long long>& out);
void proxy_rows(const hb_ctx* c, long long t0, long long t1, const long long* seeds, int nseeds,
                std::vector<long long>& out, std::vector<int>& stamp, int stamp_id);
}  // namespace hb
