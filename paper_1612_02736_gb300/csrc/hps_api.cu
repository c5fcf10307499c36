// C ABI of the GB300 HPS solver: tree construction, the build stage (Algorithm 1), the
// solve stage (Algorithm 2) in FP64 or FP32 with FP64 iterative refinement, and the
// adjoint (transposed Algorithm 2 sweeps).  Host code here only plans: every arithmetic
// step of the build, the solve, the residual and the adjoint runs in the kernels.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "hps_internal.h"

using namespace hps;

struct PlanCache;

struct hps_tree {
  Tree t;
  // host plans already made for this tree (a tree never changes once made)
  mutable std::mutex cache_mu;
  mutable std::shared_ptr<PlanCache> cache;
};

namespace {

thread_local std::string g_err;

// Domain-boundary Gaussian nodes (ascending id) of a tree for a given q.
void boundary_nodes(const Tree& t, int q, std::vector<int>& out) {
  RefTables rt;
  build_ref_tables(std::max(q + 1, 4), q, rt);
  NodeSets ns;
  build_node_sets(t, q, ns, rt.xg);
  out = ns.boundary;
}

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      throw CudaError{HPS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};            \
  } while (0)

#define CKL()                                                                                       \
  do {                                                                                              \
    cudaError_t e_ = cudaGetLastError();                                                            \
    if (e_ != cudaSuccess)                                                                          \
      throw CudaError{HPS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)};       \
  } while (0)

struct Alloc {
  hps_allocator a{};
  bool custom = false;
  void* get(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (custom) {
      p = a.alloc(bytes, a.ctx, (void*)s);
    } else {
      if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
      }
    }
    if (!p) throw CudaError{HPS_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
    return p;
  }
  void put(void* p, cudaStream_t s) {
    if (!p) return;
    if (custom) a.free(p, a.ctx, (void*)s);
    else cudaFreeAsync(p, s);
  }
};

// Device buffer owned by a handle.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// FP64 table as unevaluated pairs hi + lo of floats (hi = x rounded to float, lo = the
// remainder rounded to float) for the double-float residual kernels.
std::vector<float> split_df(const std::vector<double>& v) {
  std::vector<float> o(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const float hi = (float)v[i];
    o[2 * i] = hi;
    o[2 * i + 1] = (float)(v[i] - (double)hi);
  }
  return o;
}

// Compact row storage of a rows x (4 q) matrix (row-major) whose rows are nonzero on a few
// of their four q-column blocks: blk (4 per row, -1 padded) the indices of the blocks
// holding a nonzero, off (rows + 1) the start of each row's stored blocks in vals, vals the
// blocks' entries as double-float pairs.
struct BlockRows {
  std::vector<int> blk, off;
  std::vector<float> vals;
};
BlockRows block_rows(const std::vector<double>& m, int rows, int q) {
  const int cols = 4 * q;
  BlockRows br;
  br.blk.assign((size_t)rows * 4, -1);
  br.off.assign((size_t)rows + 1, 0);
  std::vector<double> kept;
  for (int r = 0; r < rows; ++r) {
    int n = 0;
    for (int b = 0; b < 4; ++b) {
      bool nz = false;
      for (int j = b * q; j < b * q + q; ++j) nz = nz || m[(size_t)r * cols + j] != 0.0;
      if (!nz) continue;
      br.blk[(size_t)r * 4 + n++] = b;
      for (int j = b * q; j < b * q + q; ++j) kept.push_back(m[(size_t)r * cols + j]);
    }
    br.off[r + 1] = (int)kept.size();
  }
  br.vals = split_df(kept);
  if (br.vals.empty()) br.vals.assign(2, 0.f);
  return br;
}

template <typename T>
T* upload(Alloc& al, cudaStream_t s, const std::vector<T>& v, std::vector<DBuf>& owned) {
  void* p = al.get(v.size() * sizeof(T), s);
  owned.push_back({p, v.size() * sizeof(T)});
  if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return (T*)p;
}

constexpr int ROWBLK = 64;

// HPS_MIXED: merge levels at the top of the tree eliminated in FP64 by default.  The FP32
// eliminations below them bound the contraction of the refinement: on the 64 x 64-leaf,
// p = 16 variable-coefficient workload one correction leaves a relative error of 1.1e-8
// with 1 FP64 level, 5.8e-9 with 3, 2.0e-9 with 5, 6.7e-11 with all of them, while the
// build time grows from 68 to 86 ms (FP64 build: 88 ms).
constexpr int kFp64TopLevels = 5;

#define TIMED(name, fl, by, ...)                                  \
  do {                                                            \
    TimingScope ts_((name), s, (double)(fl), (double)(by));       \
    __VA_ARGS__;                                                  \
  } while (0)

template <typename T>
const char* tsuf() {
  return sizeof(T) == 8 ? "f64" : "f32";
}

void add_product(std::vector<GemmItem>& out, long long a_base, int lda, int M, int K, int kseg, int b0_row,
                 int b0_idx, int b1_row, int b1_idx, int c_row, int c_idx, int add_row, bool trans) {
  for (int r0 = 0; r0 < M; r0 += ROWBLK) {
    GemmItem it;
    it.a_off = trans ? a_base + r0 : a_base + (long long)r0 * lda;
    it.lda = lda;
    it.M = std::min(ROWBLK, M - r0);
    it.K = K;
    it.kseg = kseg;
    it.b0_row = b0_row;
    it.b0_idx = b0_idx;
    it.b1_row = b1_row;
    it.b1_idx = b1_idx;
    if (c_idx >= 0) {
      it.c_row = c_row;
      it.c_idx = c_idx + r0;
    } else {
      it.c_row = c_row + r0;
      it.c_idx = -1;
    }
    it.add_row = add_row >= 0 ? add_row + r0 : -1;
    out.push_back(it);
  }
}

struct ItemSet {
  GemmItem* dev = nullptr;
  int n = 0;
  int maxK = 0;        // largest inner dimension of the items
  double elems = 0.0;  // operator entries streamed by one application
  // tensor-core products: each item's first K step in the operator digit cache (prefix sums
  // of ceil(K / 16)) and the cache itself, formed on first use outside stream capture
  long long* dstep = nullptr;
  long long dsteps = 0;
  mutable GemmDigits dg;
  mutable bool dg_tried = false;
  mutable int uses = 0;  // tensor-core applications so far (the cache is formed on the second)
  // the same for the FP32 operators of a mixed-precision handle: their bf16 pieces
  mutable GemmDigits dg32;
  mutable bool dg32_tried = false;
  mutable int uses32 = 0;
};

// A product step of one level: items writing final outputs, and split-K items writing
// partial sums that a reduction adds into the outputs.
struct Prod {
  ItemSet direct, split;
  SplitRed* red = nullptr;
  int nred = 0;
};

struct Level {
  std::vector<int> boxes;  // merges at this height
  bool fp64 = true;        // precision of the elimination
  int maxR = 0, maxK = 0, maxRows = 0;
  // build
  GJDesc* gj = nullptr;
  MergeDesc* md = nullptr;
  long long* off_tl = nullptr;  // per matrix extraction offsets (Mleft, CX rows, S, T)
  long long* off_bl = nullptr;
  long long* off_tr = nullptr;
  long long* off_br = nullptr;
  long long work_elems = 0;
  long long mstride = 0;  // matrix m of the batch at work + m * mstride, all of one shape (0: not so)
  int perm_elems = 0;
  // blocked elimination (FP64 levels, see block_plan): Gauss-Jordan on the top k3 rows only
  // (gj_top), then the bottom rows by one product with the eliminated top rows (schur, its
  // K chunks at item ranges schur_chunk[c] .. schur_chunk[c + 1])
  GJDesc* gj_top = nullptr;
  ItemSet schur;
  std::vector<int> schur_chunk;
  int schur_R = 0;
  BGroup* sgrp = nullptr;        // the product's vector groups (one per box and K chunk)
  int n_sgrp = 0;
  long long* sbblk = nullptr;    // per item: its group's first vector digit block
  int* sbexo = nullptr;          // per item: its group's first column exponent
  long long sb_blocks = 0;       // vector digit blocks of the level
  // solve
  UpGather* ug = nullptr;
  int ug_maxrows = 0;
  Prod up, down;
  // adjoint
  int* wcopy_tab = nullptr;
  int n_wcopy = 0;
  Prod adjS;
  int* reduce_tab = nullptr;
  int n_reduce = 0;
  Prod adjM;
  // coarsened refined parents of this level (Sec. 6.3-6.4)
  ItemSet iup, idown, aiup, aidown;
  BGemm* tp1 = nullptr;  // T_tmp P_up -> scratch
  BGemm* tp2 = nullptr;  // P_down (T_tmp P_up) -> T store
  int ntp = 0;
  long long tp_scratch = 0;
  DownScatter* ds = nullptr;
  int ds_maxrows = 0;
};

struct Workspace {
  int nrhs = 0;
  size_t bytes = 0;
  std::vector<void*> ptrs;
  // FP64 path
  double* V64 = nullptr;
  double* d64 = nullptr;
  double* ug64 = nullptr;
  double* P64 = nullptr;  // split-K partial sums
  // FP32 path
  float* V32 = nullptr;
  float* P32 = nullptr;
  float* d32 = nullptr;
  float* ug32 = nullptr;
  float* g32 = nullptr;
  float* uc32 = nullptr;
  float* rho32 = nullptr;
  // refinement
  double* vflux = nullptr;
  double* rho64 = nullptr;
  double* scal = nullptr;
  // exponent buffer of the tensor-core FP64 products (units of one launch at most)
  int* tc_scales = nullptr;
  long long tc_units = 0;
  // adjoint
  double* LB = nullptr;
  double* UB = nullptr;
  double* ubar = nullptr;
  // root conditions: seam data d, seam particular values w, remaining-node flux h', and
  // the flux data of Neumann nodes, row blocks of one buffer
  double* bcw = nullptr;
};

// Root conditions other than Dirichlet data: periodic west/east sides and flux data on the
// south/north sides (the channel problem of Sec. 7.6).  With the root DtN relation
// v = T u + h, periodic sides glue the root to itself like a merge of Sec. 4 (seam nodes
// W = E; X_s, S_s, C_s X_s and the DtN map T' of the remaining nodes x), and Neumann
// nodes N of x are solved from T'_NN u_N = f_N - h'_N - T'_ND u_D.
struct BcPlan {
  bool on = false, periodic = false, neumann = false;
  int root = -1;
  std::vector<int> ext;    // root exterior node ids: the order of its T and h
  std::vector<int> W, E;   // facing west/east node ids, by height (periodic)
  std::vector<int> X;      // ext without W and E (all of ext when not periodic)
  std::vector<int> N, D;   // X split: flux nodes (Neumann) and value nodes, in X order
  int Ks = 0, nx = 0, Kn = 0, nd = 0;
  long long xs_off = -1, ss_off = -1, cxs_off = -1, bn_off = -1;  // operator pool
  long long tp_off = -1;   // T' (nx x nx) in the build's T store
  int rows = 0;            // bcw rows: d [0, Ks), w [Ks, 2Ks), h' [2Ks, 2Ks+nx), r [.., +Kn)
  int seam_rt = -1, seam_ct = -1, neu_rt = -1, neu_ct = -1;  // assembly tables (in idx)
  int c_d = -1, c_hx = -1, c_fD = -1, c_r = -1, c_E = -1;   // row-combine tables (in idx)
  ItemSet p_ws, p_hx, p_uN, p_uW;                            // products (device)
};

}  // namespace

struct hps_handle {
  Alloc al;
  std::vector<DBuf> owned;
  Tree tree;
  NodeSets ns;
  RefTables rt;
  hps_opts opts{};
  int p = 0, q = 0, m = 0, nq = 0, ne = 0, pp = 0, n_leaf = 0, n_bdry = 0;
  // tables
  double *dD = nullptr, *dD2 = nullptr, *dLs = nullptr, *dDLs = nullptr, *dLloc = nullptr, *dDceL = nullptr;
  float2 *dLloc_df = nullptr, *dLce_c = nullptr, *dD_df = nullptr, *dD2_df = nullptr;
  int *dLce_blk = nullptr, *dLce_off = nullptr;
  int n_lce = 0;
  double* dhxy = nullptr;
  int* didx = nullptr;
  int* d_leaf_edges = nullptr;
  int* d_pairs = nullptr;
  int npairs = 0;
  int off_ci = 0, off_ce = 0, off_bnd = 0;
  std::vector<int> off_ge, off_J3;
  int* d_status = nullptr;
  // operators
  double* ops64 = nullptr;
  float* ops32 = nullptr;
  long long ops_elems = 0;
  long long gl_base = 0, h_base = 0, lce_base = 0;
  std::vector<long long> mo, so;  // per box: Mleft and S offsets
  std::vector<long long> toff;    // per box: T block offset in the build's T store
  long long tstore_elems = 0;     // size of the build's T store
  std::string tune_path;          // autotuner cache file ("" = process memory only)
  bool shared = false;            // one leaf's operators serve every leaf (equal leaves)
  BcPlan bc;                      // periodic / Neumann root conditions
  std::vector<long long> ttmp;    // coarsened boxes: T before coarsening (T store)
  std::vector<long long> puo, pdo, pco;  // coarsened boxes: P_up, P_down, P_up(fine, coarse)
  std::vector<int> k3, k12, k12o; // |J3|, |I_ge| seen by the parent, |J1 + J2|
  std::vector<int> off_geo, off_fine, off_coarse;
  bool any_coarsened = false;
  // vector layouts (in rows)
  std::vector<int> vrow, drow, ubrow;
  int v_rows = 0, d_rows = 0, ub_rows = 0;
  int p_rows = 0;  // split-K partial rows (max over the product steps)
  // plans
  std::vector<Level> levels;  // index = height - 1
  ItemSet leafup, leafdown, lce;
  ItemSet adj_leafF, adj_leafS, adj_lce, adj_leafH;
  double* coeffs_copy = nullptr;  // FP64 coefficients (mixed-precision residual, leaf recomputation)
  // leaf recomputation ("econ", store_leaf_ops = 0): leaf operators are rebuilt chunk by
  // chunk whenever a sweep needs them (Sec. 5.4 remark)
  bool econ = false;
  int echunk = 0;                 // leaves per chunk
  int max_items = 0;              // largest product item set (sizes the tensor-core exponent buffer)
  bool noalloc_call = false;      // inside hps_solve_noalloc: no allocation, no digit caches
  int* tc_scales = nullptr;       // tensor-core exponent buffer of the current call (workspace
  long long tc_units = 0;         // or the no-allocation scratch) and its capacity in units
  double* ework = nullptr;        // elimination workspace of one chunk
  int* eperm = nullptr;
  double* epinv = nullptr;
  double* eprow = nullptr;
  double* eops = nullptr;         // [F | S_ci] and H of one chunk
  GJDesc* egd = nullptr;          // per-leaf descriptors with chunk-relative offsets
  int* leaf_reduce_tab = nullptr;
  int n_leaf_reduce = 0;
  int* fbar_tab = nullptr;
  // workspace
  Workspace ws;
  // iterative refinement (HPS_MIXED): contraction bound calibrated on the adaptive solves
  // (rho: twice the largest observed ratio of successive corrections, 0 until known) and the
  // number of corrections a solve then runs without testing between them
  struct {
    double rho = 0.0;
    int nfix = 0;
  } ir;
  // captured sweep (FP64) or fixed-schedule refined solve (HPS_MIXED) per nrhs, and its
  // staging buffers
  struct {
    int nrhs = 0;
    int nfix = 0;        // refinement steps in the captured mixed solve
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    double *f_in = nullptr, *g_in = nullptr, *u_out = nullptr;
    bool broken = false;
    int last_nrhs = 0;   // capture on the second call with the same nrhs
    int kernels = 0;     // kernel nodes in the graph
    double flops = 0.0, bytes = 0.0;
  } graph;
  void drop_graph() {
    if (graph.exec) cudaGraphExecDestroy(graph.exec);
    graph.exec = nullptr;
    for (double* p : {graph.f_in, graph.g_in, graph.u_out}) al.put(p, 0);
    graph.f_in = graph.g_in = graph.u_out = nullptr;
    graph.nrhs = 0;
  }
  ~hps_handle() {
    drop_graph();
    if (graph.cs) cudaStreamDestroy(graph.cs);
    if (ws.ptrs.empty() && owned.empty()) return;
    for (void* p : ws.ptrs) al.put(p, 0);
    for (auto& b : owned) al.put(b.p, 0);
    cudaStreamSynchronize(0);
  }
  // row base of the flux vector a box hands to its parent (after coarsening)
  int hrow(int box) const {
    if (tree.boxes[box].leaf >= 0) return vrow[box];
    return vrow[box] + k3[box] + (ns.co[box].active ? k12o[box] : 0);
  }
  int hrow_old(int box) const { return vrow[box] + (tree.boxes[box].leaf >= 0 ? 0 : k3[box]); }
};

namespace {

ItemSet upload_items(hps_handle* h, cudaStream_t s, const std::vector<GemmItem>& v) {
  ItemSet is;
  is.n = (int)v.size();
  std::vector<long long> steps;
  steps.reserve(v.size());
  for (const GemmItem& it : v) {
    is.elems += (double)it.M * it.K;
    is.maxK = std::max(is.maxK, it.K);
    steps.push_back(is.dsteps);
    is.dsteps += (it.K + 15) / 16;
  }
  h->max_items = std::max(h->max_items, is.n);
  if (!v.empty()) is.dstep = upload(h->al, s, steps, h->owned);
  is.dev = v.empty() ? nullptr : upload(h->al, s, v, h->owned);
  return is;
}

// ---------------------------------------------------------------------------------------
// Plan: index tables, operator offsets, vector layouts and the product items of every
// step of the solve and the adjoint.  Built on the host, checked against the buffer
// sizes (validate_plan), then uploaded.
struct ProdHost {
  std::vector<GemmItem> direct, split;
  std::vector<SplitRed> red;
};

// Split-K: when a level has too few row blocks to fill the GPU (the large merges near the
// root), each row block's K range is cut into nsplit pieces computed by separate CTAs
// into a partial buffer and summed in fixed order by a reduction (deterministic).
int split_prod(ProdHost& ph, bool trans) {
  const int target = 2 * 152;
  const int n = (int)ph.direct.size();
  if (n == 0 || n >= target) return 0;
  std::vector<GemmItem> keep;
  int prow = 0;
  for (const GemmItem& it : ph.direct) {
    int ns = std::min((target + n - 1) / n, it.K / 128);
    if (it.kseg != it.K || ns < 2) {
      keep.push_back(it);
      continue;
    }
    const int kc = (it.K + ns - 1) / ns;
    ns = (it.K + kc - 1) / kc;
    SplitRed sr;
    sr.M = it.M;
    sr.nsplit = ns;
    sr.p_row = prow;
    sr.c_row = it.c_row;
    sr.c_idx = it.c_idx;
    sr.add_row = it.add_row;
    for (int j = 0; j < ns; ++j) {
      const int k0 = j * kc;
      GemmItem s = it;
      s.K = std::min(kc, it.K - k0);
      s.kseg = s.K;
      s.a_off = trans ? it.a_off + (long long)k0 * it.lda : it.a_off + k0;
      if (it.b0_idx >= 0) s.b0_idx = it.b0_idx + k0;
      else s.b0_row = it.b0_row + k0;
      s.c_row = prow + j * it.M;
      s.c_idx = -1;
      s.add_row = -1;
      ph.split.push_back(s);
    }
    prow += ns * it.M;
    ph.red.push_back(sr);
  }
  ph.direct.swap(keep);
  return prow;
}

// Blocked elimination of a level's merges (Algorithm 1's Schur complements, one product).
// Every pivot of a merge matrix M = [[Z, R], [-C, T]] comes from its top k3 rows (the
// interface equations), so the Gauss-Jordan elimination maps each bottom row x = [x_L | x_R]
// to [0 | x_R] - x_L Top, Top[k] the final pivot row of column k (physical row perm[k]):
// the bottom block ends as [0 | T] + (-C) Top, in-place layout unchanged.  Eliminating the
// top rows alone and then forming the bottom rows by one FP64 tensor-core product (exact
// digit slicing, K chunks of at most 448) streams the k12 x R bottom block once instead of
// once per 16-pivot panel.  Taken for levels whose merges all keep their full matrix
// (rows = R), share one row length, and have at least two panels.
void block_plan(struct LevelHost& pd);

struct LevelHost {
  std::vector<GJDesc> gj, gj_top;
  std::vector<GemmItem> schur;
  std::vector<int> schur_chunk;
  std::vector<BGroup> sgrp;
  std::vector<long long> sbblk;
  std::vector<int> sbexo;
  std::vector<MergeDesc> md;
  std::vector<long long> tl, bl, tr, br;
  std::vector<UpGather> ug;
  ProdHost up, down, adjS, adjM;
  std::vector<GemmItem> iup, idown, aiup, aidown;
  std::vector<BGemm> tp1, tp2;
  std::vector<int> wcopy, reduce;
  std::vector<DownScatter> ds;
};

struct HostPlan {
  std::vector<int> idx;
  std::vector<LevelHost> lv;
  std::vector<GemmItem> lup, ldown, llce, aF, aS, aL, aH;
  std::vector<int> lred, ftab, pairs;
  std::vector<GemmItem> bc_ws, bc_hx, bc_uN, bc_uW;
  long long tsz = 0;
};

// Tables and product items of the root conditions (see BcPlan).
template <typename Push>
void make_bc_plan(hps_handle* h, HostPlan& hp, Push push) {
  BcPlan& bc = h->bc;
  const int Ks = bc.Ks, nx = bc.nx, Kn = bc.Kn, nd = bc.nd;
  const int d0 = 0, w0 = Ks, x0 = 2 * Ks, r0 = 2 * Ks + nx;
  std::unordered_map<int, int> pe, px, brow;
  for (size_t k = 0; k < bc.ext.size(); ++k) pe[bc.ext[k]] = (int)k;
  for (size_t k = 0; k < bc.X.size(); ++k) px[bc.X[k]] = (int)k;
  for (size_t k = 0; k < h->ns.boundary.size(); ++k) brow[h->ns.boundary[k]] = (int)k;
  const int hb = h->hrow_old(bc.root);
  std::vector<int> rt, ct;
  if (bc.periodic) {
    // M_s = [[Z_s, R_s], [-C_s, T_xx]] from T_root: rows (E - W | x), columns (E + W | x),
    // off-diagonal blocks negated
    for (int k = 0; k < Ks; ++k) rt.insert(rt.end(), {pe.at(bc.E[k]), 1, pe.at(bc.W[k]), -1});
    for (int g : bc.X) rt.insert(rt.end(), {pe.at(g), 1, -1, 0});
    for (int k = 0; k < Ks; ++k) ct.insert(ct.end(), {pe.at(bc.E[k]), 1, pe.at(bc.W[k]), 1});
    for (int g : bc.X) ct.insert(ct.end(), {pe.at(g), 1, -1, 0});
    bc.seam_rt = push(rt);
    bc.seam_ct = push(ct);
  }
  if (Kn > 0) {
    // [T'_NN | T'_ND] from T' (periodic: positions in X) or T_root (positions in ext)
    auto at = [&](int g) { return bc.periodic ? px.at(g) : pe.at(g); };
    rt.clear();
    ct.clear();
    for (int g : bc.N) rt.insert(rt.end(), {at(g), 1, -1, 0});
    for (int g : bc.N) ct.insert(ct.end(), {at(g), 1, -1, 0});
    for (int g : bc.D) ct.insert(ct.end(), {at(g), 1, -1, 0});
    bc.neu_rt = push(rt);
    bc.neu_ct = push(ct);
  }
  // row combinations dst = a (+ sign b), in vector rows
  std::vector<int> c;
  if (bc.periodic) {
    for (int k = 0; k < Ks; ++k) c.insert(c.end(), {d0 + k, hb + pe.at(bc.W[k]), hb + pe.at(bc.E[k]), -1});
    bc.c_d = push(c);
    c.clear();
    for (int k = 0; k < Ks; ++k) c.insert(c.end(), {bc.E[k], bc.W[k], -1, 0});
    bc.c_E = push(c);
    c.clear();
  }
  for (int i = 0; i < nx; ++i) c.insert(c.end(), {x0 + i, hb + pe.at(bc.X[i]), -1, 0});
  bc.c_hx = push(c);
  c.clear();
  for (int g : bc.D) c.insert(c.end(), {g, brow.at(g), -1, 0});
  bc.c_fD = push(c);
  c.clear();
  for (int i = 0; i < Kn; ++i) c.insert(c.end(), {r0 + i, brow.at(bc.N[i]), x0 + px.at(bc.N[i]), -1});
  bc.c_r = push(c);
  // products
  if (bc.periodic) {
    add_product(hp.bc_ws, bc.xs_off, Ks, Ks, Ks, Ks, d0, -1, 0, -1, w0, -1, -1, false);          // w_s = X_s d_s
    add_product(hp.bc_hx, bc.cxs_off, Ks, nx, Ks, Ks, d0, -1, 0, -1, x0, -1, -1, false);         // h' += C_s X_s d_s
    add_product(hp.bc_uW, bc.ss_off, nx, Ks, nx, nx, 0, push(bc.X), 0, -1, 0, push(bc.W), w0, false);  // u_W
  }
  if (Kn > 0)  // u_N = X_n r_N - X_n T'_ND u_D
    add_product(hp.bc_uN, bc.bn_off, Kn + nd, Kn, Kn + nd, Kn, r0, -1, 0, nd > 0 ? push(bc.D) : -1, 0, push(bc.N), -1,
                false);
}

void make_plan(hps_handle* h, HostPlan& hp) {
  const Tree& t = h->tree;
  const NodeSets& ns = h->ns;
  const RefTables& rt = h->rt;
  const int nb = (int)t.boxes.size();
  const int q = h->q, m = h->m, nq = h->nq, pp = h->pp;
  std::vector<int>& idx = hp.idx;
  auto push = [&](const std::vector<int>& v) {
    const int off = (int)idx.size();
    idx.insert(idx.end(), v.begin(), v.end());
    return off;
  };
  h->off_ci = push(rt.ci);
  h->off_ce = push(rt.ce);
  h->off_bnd = push(ns.boundary);
  h->off_ge.assign(nb, -1);
  h->off_J3.assign(nb, -1);
  h->off_geo.assign(nb, -1);
  h->off_fine.assign(nb, -1);
  h->off_coarse.assign(nb, -1);
  h->k3.assign(nb, 0);
  h->k12.assign(nb, 0);
  h->k12o.assign(nb, 0);
  for (int b = 0; b < nb; ++b) {
    h->off_ge[b] = push(ns.ge[b]);
    h->k12[b] = (int)ns.ge[b].size();
    h->k12o[b] = (int)ns.ge_old[b].size();
    if (t.boxes[b].leaf < 0) {
      h->off_J3[b] = push(ns.J3[b]);
      h->off_geo[b] = push(ns.ge_old[b]);
      h->k3[b] = (int)ns.J3[b].size();
    }
    if (ns.co[b].active) {
      h->off_fine[b] = push(ns.co[b].fine);
      h->off_coarse[b] = push(ns.co[b].coarse);
      h->any_coarsened = true;
    }
  }
  // operator pool layout
  long long off = 0;
  const long long gsz = (long long)m * (m + nq), hsz = (long long)nq * m;
  h->econ = h->opts.store_leaf_ops == 0 && !h->shared;
  if (h->econ) {
    // leaf operators live in a per-chunk buffer: about 512 MiB of operators and workspace
    const long long per = (long long)(m + nq) * (m + nq) + gsz + hsz;
    h->echunk = (int)std::max<long long>(1, std::min<long long>(h->n_leaf, (512ll << 20) / (per * 8)));
    h->gl_base = 0;
    h->h_base = (long long)h->echunk * gsz;
  } else {
    const long long nl = h->shared ? 1 : h->n_leaf;  // shared: one leaf's F, S_ci, H
    h->gl_base = off;
    off += nl * gsz;
    h->h_base = off;
    off += nl * hsz;
  }
  h->lce_base = off;
  off += (long long)h->ne * nq;
  h->mo.assign(nb, -1);
  h->so.assign(nb, -1);
  h->puo.assign(nb, -1);
  h->pdo.assign(nb, -1);
  h->pco.assign(nb, -1);
  for (int b = 0; b < nb; ++b) {
    if (t.boxes[b].leaf >= 0) continue;
    // [X; C X] (the root keeps X only: nothing above it applies C X)
    const int R = (t.boxes[b].parent < 0 && !h->bc.on) ? h->k3[b] : h->k3[b] + h->k12o[b];
    h->mo[b] = off;
    off += (long long)R * h->k3[b];
    h->so[b] = off;
    off += (long long)h->k3[b] * h->k12o[b];
    if (ns.co[b].active) {
      h->puo[b] = off;
      off += (long long)h->k12o[b] * h->k12[b];
      h->pdo[b] = off;
      off += (long long)h->k12[b] * h->k12o[b];
      h->pco[b] = off;
      off += (long long)ns.co[b].fine.size() * ns.co[b].coarse.size();
    }
  }
  if (h->bc.on) {  // root-condition operators: X_s, S_s, C_s X_s; [X_n | -X_n T'_ND]
    BcPlan& bc = h->bc;
    if (bc.periodic) {
      bc.xs_off = off;
      off += (long long)bc.Ks * bc.Ks;
      bc.ss_off = off;
      off += (long long)bc.Ks * bc.nx;
      bc.cxs_off = off;
      off += (long long)bc.nx * bc.Ks;
    }
    if (bc.Kn > 0) {
      bc.bn_off = off;
      off += (long long)bc.Kn * (bc.Kn + bc.nd);
    }
  }
  h->ops_elems = off;
  // vector layouts
  h->vrow.assign(nb, 0);
  h->drow.assign(nb, -1);
  h->ubrow.assign(nb, -1);
  int vr = 0, dr = 0, ur = 0;
  for (int b = 0; b < nb; ++b) {
    h->vrow[b] = vr;
    if (t.boxes[b].leaf >= 0) {
      vr += nq;
    } else {
      vr += h->k3[b] + h->k12o[b] + (ns.co[b].active ? h->k12[b] : 0);
      h->drow[b] = dr;
      dr += h->k3[b];
      h->ubrow[b] = ur;
      ur += h->k12o[b];
    }
  }
  h->v_rows = vr;
  h->d_rows = dr;
  h->ub_rows = ur;

  // positions of each node in each box's exterior list
  auto posmap = [&](int b) {
    std::unordered_map<int, int> mp;
    mp.reserve(ns.ge[b].size() * 2);
    for (size_t k = 0; k < ns.ge[b].size(); ++k) mp[ns.ge[b][k]] = (int)k;
    return mp;
  };

  // levels
  const int H = t.height;
  h->levels.assign(H, Level());
  for (int b = 0; b < nb; ++b)
    if (t.boxes[b].leaf < 0) h->levels[t.boxes[b].height - 1].boxes.push_back(b);
  int top64 = h->opts.fp64_top_levels < 0 ? kFp64TopLevels : h->opts.fp64_top_levels;
  hp.lv.assign(H, LevelHost());
  // T store offsets per box (children T blocks live there until the build ends): the
  // leaves first, in leaf order (the leaf extraction writes them with a fixed stride),
  // then the parents.
  std::vector<long long>& toff = h->toff;
  toff.assign(nb, -1);
  long long tsz = 0;
  for (int lf = 0; lf < h->n_leaf; ++lf) {
    toff[t.leaves[lf]] = h->shared ? 0 : tsz;  // shared: every leaf reads leaf 0's T
    if (!h->shared || lf == 0) tsz += (long long)nq * nq;
  }
  h->ttmp.assign(nb, -1);
  for (int b = 0; b < nb; ++b) {
    // no DtN map is kept for the root, unless periodic / Neumann root conditions need it
    if (t.boxes[b].leaf >= 0 || (t.boxes[b].parent < 0 && !h->bc.on)) continue;
    toff[b] = tsz;
    tsz += (long long)h->k12[b] * h->k12[b];
    if (ns.co[b].active) {
      h->ttmp[b] = tsz;
      tsz += (long long)h->k12o[b] * h->k12o[b];
    }
  }
  if (h->bc.periodic) {  // T' of the nodes left after the periodic seam
    h->bc.tp_off = tsz;
    tsz += (long long)h->bc.nx * h->bc.nx;
  }
  for (int L = 0; L < H; ++L) {
    Level& lv = h->levels[L];
    LevelHost& pd = hp.lv[L];
    lv.fp64 = (h->opts.precision == HPS_FP64) || (L >= H - top64);
    long long woff = 0;
    int poff = 0;
    std::unordered_map<int, std::pair<int, int>> red;  // node -> (ub row 1, ub row 2)
    std::vector<int> red_order;
    for (int b : lv.boxes) {
      const Box& bx = t.boxes[b];
      const int a = bx.child[0], c = bx.child[1];
      const int k3 = h->k3[b], k12 = h->k12o[b], R = k3 + k12, n1 = ns.n1[b], n2 = k12 - n1;
      // The root's solve needs X and S only (u_ge = f there): its elimination forms and
      // eliminates the top rows [Z | R] and never computes C X or T_tau.
      const bool root = bx.parent < 0 && !h->bc.on;
      const int rows = root ? k3 : R;
      lv.maxR = std::max(lv.maxR, R);
      lv.maxK = std::max(lv.maxK, k3);
      lv.maxRows = std::max(lv.maxRows, rows);
      auto pa = posmap(a), pc = posmap(c);
      std::vector<int> posA(R, -1), posB(R, -1);
      const std::vector<int>& J3 = ns.J3[b];
      const std::vector<int>& ge = ns.ge_old[b];
      for (int k = 0; k < k3; ++k) {
        posA[k] = pa.at(J3[k]);
        posB[k] = pc.at(J3[k]);
      }
      for (int i = 0; i < n1; ++i) posA[k3 + i] = pa.at(ge[i]);
      for (int i = 0; i < n2; ++i) posB[k3 + n1 + i] = pc.at(ge[n1 + i]);
      MergeDesc md;
      md.m_off = woff;
      md.R = R;
      md.rows = rows;
      md.k3 = k3;
      md.n1 = n1;
      md.ta_off = toff[a];
      md.tb_off = toff[c];
      md.lda_a = h->k12[a];
      md.lda_b = h->k12[c];
      md.pos_off = push(posA);
      push(posB);
      pd.md.push_back(md);
      GJDesc gd;
      gd.off = woff;
      gd.R = R;
      gd.K = k3;
      gd.rows = rows;
      gd.perm_off = poff;
      gd.box = b;
      pd.gj.push_back(gd);
      woff += (long long)rows * R;
      poff += k3;
      pd.tl.push_back(h->mo[b]);
      pd.bl.push_back(h->mo[b] + (long long)k3 * k3);
      pd.tr.push_back(h->so[b]);
      pd.br.push_back(ns.co[b].active ? h->ttmp[b] : toff[b]);
      // up-sweep gather lists: pos3a, pos3b, J3, pos1a, pos2b
      std::vector<int> lst;
      for (int k = 0; k < k3; ++k) lst.push_back(posA[k]);
      for (int k = 0; k < k3; ++k) lst.push_back(posB[k]);
      for (int k = 0; k < k3; ++k) lst.push_back(J3[k]);
      for (int i = 0; i < n1; ++i) lst.push_back(posA[k3 + i]);
      for (int i = 0; i < n2; ++i) lst.push_back(posB[k3 + n1 + i]);
      const int loff = push(lst);
      UpGather ug;
      ug.va_row = h->hrow(a);
      ug.vb_row = h->hrow(c);
      ug.vt_row = h->vrow[b];
      ug.d_row = h->drow[b];
      ug.k3 = k3;
      ug.n1 = n1;
      ug.n2 = n2;
      ug.idx_off = loff;
      pd.ug.push_back(ug);
      lv.ug_maxrows = std::max(lv.ug_maxrows, 2 * k3 + n1 + n2);
      DownScatter ds;
      ds.va_row = ug.va_row;
      ds.vb_row = ug.vb_row;
      ds.vt_row = ug.vt_row;
      ds.d_row = ug.d_row;
      ds.k3 = k3;
      ds.n1 = n1;
      ds.n2 = n2;
      ds.idx_off = loff;
      pd.ds.push_back(ds);
      lv.ds_maxrows = std::max(lv.ds_maxrows, k3 + n1 + n2);
      // up: [w; h] += [X; CX] d
      add_product(pd.up.direct, h->mo[b], k3, rows, k3, k3, h->drow[b], -1, 0, -1, h->vrow[b], -1, -1, false);
      // down: u[J3] = S u[ge] + w
      add_product(pd.down.direct, h->so[b], k12, k3, k12, k12, 0, h->off_geo[b], 0, -1, 0, h->off_J3[b], h->vrow[b],
                  false);
      // adjoint: wbar copy, S^T ubar[J3] -> UB, reduce into ubar[ge]
      for (int k = 0; k < k3; ++k) {
        pd.wcopy.push_back(h->vrow[b] + k);
        pd.wcopy.push_back(J3[k]);
        pd.wcopy.push_back(-1);
      }
      add_product(pd.adjS.direct, h->so[b], k12, k12, k3, k3, 0, h->off_J3[b], 0, -1, h->ubrow[b], -1, -1, true);
      for (int k = 0; k < k12; ++k) {
        const int g = ge[k];
        auto it = red.find(g);
        if (it == red.end()) {
          red[g] = {h->ubrow[b] + k, -1};
          red_order.push_back(g);
        } else {
          it->second.second = h->ubrow[b] + k;
        }
      }
      // adjoint: dbar = [X; CX]^T [wbar; hbar]
      add_product(pd.adjM.direct, h->mo[b], k3, k3, rows, rows, h->vrow[b], -1, 0, -1, h->drow[b], -1, -1, true);
      // coarsened refined parent (Sec. 6.3-6.4)
      const Coarsen& co = ns.co[b];
      if (co.active) {
        const int kn = h->k12[b], nf = (int)co.fine.size(), nc = (int)co.coarse.size();
        // up: h_new = P_down h_old ; down: u_fine = P_up(fine, coarse) u_coarse
        add_product(pd.iup, h->pdo[b], k12, kn, k12, k12, h->hrow_old(b), -1, 0, -1, h->hrow(b), -1, -1, false);
        add_product(pd.idown, h->pco[b], nc, nf, nc, nc, 0, h->off_coarse[b], 0, -1, 0, h->off_fine[b], -1, false);
        // adjoint: hbar_old = P_down^T hbar_new ; ubar_coarse += P_up(fine, coarse)^T ubar_fine
        add_product(pd.aiup, h->pdo[b], k12, k12, kn, kn, h->hrow(b), -1, 0, -1, h->hrow_old(b), -1, -1, true);
        add_product(pd.aidown, h->pco[b], nc, nc, nf, nf, 0, h->off_fine[b], 0, -1, 0, h->off_coarse[b], -1, true);
        // build: T_new = P_down (T_old P_up)
        BGemm t1{h->ttmp[b], h->puo[b], lv.tp_scratch, k12, kn, k12, k12, kn, kn};
        BGemm t2{h->pdo[b], lv.tp_scratch, toff[b], kn, kn, k12, k12, kn, kn};
        pd.tp1.push_back(t1);
        pd.tp2.push_back(t2);
        lv.tp_scratch += (long long)k12 * kn;
      }
    }
    lv.work_elems = woff;
    lv.mstride = 0;
    if (!pd.gj.empty()) {
      const GJDesc& g0 = pd.gj[0];
      bool same = g0.off == 0 && g0.R == lv.maxR && g0.rows == lv.maxRows;
      for (size_t i = 0; i < pd.gj.size() && same; ++i)
        same = pd.gj[i].R == g0.R && pd.gj[i].rows == g0.rows && pd.gj[i].off == (long long)i * g0.rows * g0.R;
      if (same) lv.mstride = (long long)g0.rows * g0.R;
    }
    if (lv.fp64) block_plan(pd);
    lv.perm_elems = poff;
    h->p_rows = std::max(h->p_rows, split_prod(pd.up, false));
    h->p_rows = std::max(h->p_rows, split_prod(pd.down, false));
    h->p_rows = std::max(h->p_rows, split_prod(pd.adjS, true));
    h->p_rows = std::max(h->p_rows, split_prod(pd.adjM, true));
    for (int g : red_order) {
      pd.reduce.push_back(g);
      pd.reduce.push_back(red[g].first);
      pd.reduce.push_back(red[g].second);
    }
  }
  hp.tsz = tsz;
  h->tstore_elems = tsz;
  // leaf items
  std::vector<GemmItem>&lup = hp.lup, &ldown = hp.ldown, &llce = hp.llce, &aF = hp.aF, &aS = hp.aS, &aL = hp.aL,
                        &aH = hp.aH;
  for (int lf = 0; lf < h->n_leaf; ++lf) {
    const int b = t.leaves[lf];
    // econ: offsets inside the chunk buffer; shared: every leaf applies leaf 0's operators
    const int slot = h->shared ? 0 : (h->econ ? lf % h->echunk : lf);
    const long long gl = h->gl_base + (long long)slot * gsz;
    const long long hb = h->h_base + (long long)slot * hsz;
    add_product(lup, hb, m, nq, m, m, lf * pp, h->off_ci, 0, -1, h->vrow[b], -1, -1, false);
    add_product(ldown, gl, m + nq, m, m + nq, m, lf * pp, h->off_ci, 0, h->off_ge[b], lf * pp, h->off_ci, -1, false);
    add_product(llce, h->lce_base, nq, h->ne, nq, nq, 0, h->off_ge[b], 0, -1, lf * pp, h->off_ce, -1, false);
    // adjoint: gbar_ci = F^T ubar_ci ; LB = S_ci^T ubar_ci + Lce^T ubar_ce ; gbar += H^T hbar
    add_product(aF, gl, m + nq, m, m, m, lf * pp, h->off_ci, 0, -1, lf * pp, h->off_ci, -1, true);
    add_product(aS, gl + m, m + nq, nq, m, m, lf * pp, h->off_ci, 0, -1, lf * nq, -1, -1, true);
    add_product(aL, h->lce_base, nq, nq, h->ne, h->ne, lf * pp, h->off_ce, 0, -1, lf * nq, -1, -1, true);
    add_product(aH, hb, m, m, nq, nq, h->hrow(b), -1, 0, -1, lf * pp, h->off_ci, -1, true);
  }
  // ubar[j] = sum over the (one or two) leaves owning j of LB[leaf][pos]
  std::vector<int>& lred = hp.lred;
  for (int e = 0; e < t.n_edges; ++e) {
    const int o1 = t.edge_owners[2 * e], o2 = t.edge_owners[2 * e + 1];
    for (int k = 0; k < q; ++k) {
      lred.push_back(e * q + k);
      lred.push_back((o1 / 4) * nq + (o1 % 4) * q + k);
      lred.push_back(o2 >= 0 ? (o2 / 4) * nq + (o2 % 4) * q + k : -1);
    }
  }
  std::vector<int>& ftab = hp.ftab;
  for (size_t k = 0; k < ns.boundary.size(); ++k) {
    ftab.push_back((int)k);
    ftab.push_back(ns.boundary[k]);
    ftab.push_back(-1);
  }
  // interior edge pairs for the jump residual (a = the leaf west/south of the edge)
  std::vector<int>& pairs = hp.pairs;
  for (int e = 0; e < t.n_edges; ++e) {
    int o1 = t.edge_owners[2 * e], o2 = t.edge_owners[2 * e + 1];
    if (o2 < 0) continue;
    const int s1 = o1 % 4;
    if (s1 == 0 || s1 == 3) std::swap(o1, o2);  // o1 on its S or W side -> it is the E/N leaf
    pairs.push_back(e);
    pairs.push_back(o1 / 4);
    pairs.push_back(o1 % 4);
    pairs.push_back(o2 / 4);
    pairs.push_back(o2 % 4);
  }
  h->npairs = (int)pairs.size() / 5;
  if (h->bc.on) make_bc_plan(h, hp, push);
}

void block_plan(LevelHost& pd) {
  pd.gj_top.clear();
  pd.schur.clear();
  pd.schur_chunk.clear();
  pd.sgrp.clear();
  pd.sbblk.clear();
  pd.sbexo.clear();
  if (pd.gj.empty()) return;
  const int R0 = pd.gj[0].R;
  int kmax = 0;
  for (const GJDesc& g : pd.gj) {
    if (g.R != R0 || g.rows != g.R || g.K < 32 || g.K >= g.R || g.off % g.R != 0 || g.null_tol > 0.f) return;
    kmax = std::max(kmax, g.K);
  }
  const int nck = (kmax + 447) / 448;
  const int kc = ((kmax + nck - 1) / nck + 15) / 16 * 16;
  for (int c = 0; c * kc < kmax; ++c) {
    pd.schur_chunk.push_back((int)pd.schur.size());
    for (const GJDesc& g : pd.gj) {
      const int ks = c * kc;
      if (ks >= g.K) continue;
      const int K = std::min(kc, g.K - ks), k12 = g.R - g.K;
      const int base = (int)(g.off / g.R);  // first row of the matrix, rows of length R
      // the items of this box and chunk gather the same top rows: one vector digit group
      const int ncb = (g.R + 31) / 32;
      BGroup bg;
      bg.b0_row = base;
      bg.b0_idx = g.perm_off + ks;
      bg.K = K;
      bg.ex0 = (int)pd.sgrp.size() * ncb * 32;
      bg.blk0 = pd.sgrp.empty() ? 0
                                : pd.sgrp.back().blk0 + (long long)ncb * ((pd.sgrp.back().K + 15) / 16);
      pd.sgrp.push_back(bg);
      for (int r0 = 0; r0 < k12; r0 += ROWBLK) {
        GemmItem it{};
        it.a_off = g.off + (long long)(g.K + r0) * g.R + ks;  // -C, rows r0.., columns ks..
        it.lda = g.R;
        it.M = std::min(ROWBLK, k12 - r0);
        it.K = K;
        it.kseg = K;
        it.b0_row = base;                // Top rows: base + perm[ks + k]
        it.b0_idx = g.perm_off + ks;
        it.b1_row = 0;
        it.b1_idx = -1;
        it.c_row = base + g.K + r0;      // the bottom rows, all R columns
        it.c_idx = -1;
        it.add_row = -1;
        pd.schur.push_back(it);
        pd.sbblk.push_back(bg.blk0);
        pd.sbexo.push_back(bg.ex0);
      }
    }
  }
  pd.schur_chunk.push_back((int)pd.schur.size());
  pd.gj_top = pd.gj;
  for (GJDesc& g : pd.gj_top) g.rows = g.K;
}

Prod upload_prod(hps_handle* h, cudaStream_t s, const ProdHost& ph) {
  Prod pr;
  pr.direct = upload_items(h, s, ph.direct);
  pr.split = upload_items(h, s, ph.split);
  pr.nred = (int)ph.red.size();
  pr.red = ph.red.empty() ? nullptr : upload(h->al, s, ph.red, h->owned);
  return pr;
}

}  // namespace

// Host plans of one tree, reused by later builds on it.  A plan (node sets, operator
// offsets, vector layouts, product lists, elimination descriptors) depends on the mesh,
// p, q and the precision layout, never on the coefficients, so a rebuild with new
// coefficients (an optimisation loop, a time-dependent operator, a second precision of
// the same problem) copies it instead of recomputing it.
struct PlanCache {
  struct Entry {
    std::array<int, 6> key;
    std::shared_ptr<const hps_handle> layout;  // the handle's host fields after planning
    std::shared_ptr<const HostPlan> plan;
  };
  std::vector<Entry> entries;  // oldest first, at most kMax
  static constexpr size_t kMax = 4;
};

namespace {

std::array<int, 6> plan_key(int p, const hps_opts& o, bool shared) {
  const int top = o.precision == HPS_FP64 ? 0 : (o.fp64_top_levels < 0 ? kFp64TopLevels : o.fp64_top_levels);
  return {p, o.q, o.precision, top, shared ? 1 : o.store_leaf_ops, shared ? 1 : 0};
}

void upload_plan(hps_handle* h, const HostPlan& hp, cudaStream_t s) {
  h->didx = upload(h->al, s, hp.idx, h->owned);
  for (size_t L = 0; L < hp.lv.size(); ++L) {
    Level& lv = h->levels[L];
    const LevelHost& pd = hp.lv[L];
    lv.gj = upload(h->al, s, pd.gj, h->owned);
    lv.gj_top = pd.gj_top.empty() ? nullptr : upload(h->al, s, pd.gj_top, h->owned);
    {
      const int mi = h->max_items;  // the build's own products do not size the solve's buffers
      lv.schur = upload_items(h, s, pd.schur);
      h->max_items = mi;
    }
    lv.schur_chunk = pd.schur_chunk;
    lv.schur_R = pd.gj.empty() ? 0 : pd.gj[0].R;
    lv.n_sgrp = (int)pd.sgrp.size();
    lv.sgrp = pd.sgrp.empty() ? nullptr : upload(h->al, s, pd.sgrp, h->owned);
    lv.sbblk = pd.sbblk.empty() ? nullptr : upload(h->al, s, pd.sbblk, h->owned);
    lv.sbexo = pd.sbexo.empty() ? nullptr : upload(h->al, s, pd.sbexo, h->owned);
    lv.sb_blocks = 0;
    if (!pd.sgrp.empty())
      lv.sb_blocks = pd.sgrp.back().blk0 + (long long)((lv.schur_R + 31) / 32) * ((pd.sgrp.back().K + 15) / 16);
    lv.md = upload(h->al, s, pd.md, h->owned);
    lv.off_tl = upload(h->al, s, pd.tl, h->owned);
    lv.off_bl = upload(h->al, s, pd.bl, h->owned);
    lv.off_tr = upload(h->al, s, pd.tr, h->owned);
    lv.off_br = upload(h->al, s, pd.br, h->owned);
    lv.ug = upload(h->al, s, pd.ug, h->owned);
    lv.up = upload_prod(h, s, pd.up);
    lv.down = upload_prod(h, s, pd.down);
    lv.adjS = upload_prod(h, s, pd.adjS);
    lv.adjM = upload_prod(h, s, pd.adjM);
    lv.wcopy_tab = upload(h->al, s, pd.wcopy, h->owned);
    lv.n_wcopy = (int)pd.wcopy.size() / 3;
    lv.reduce_tab = upload(h->al, s, pd.reduce, h->owned);
    lv.n_reduce = (int)pd.reduce.size() / 3;
    lv.ds = upload(h->al, s, pd.ds, h->owned);
    lv.iup = upload_items(h, s, pd.iup);
    lv.idown = upload_items(h, s, pd.idown);
    lv.aiup = upload_items(h, s, pd.aiup);
    lv.aidown = upload_items(h, s, pd.aidown);
    lv.ntp = (int)pd.tp1.size();
    lv.tp1 = pd.tp1.empty() ? nullptr : upload(h->al, s, pd.tp1, h->owned);
    lv.tp2 = pd.tp2.empty() ? nullptr : upload(h->al, s, pd.tp2, h->owned);
  }
  h->leafup = upload_items(h, s, hp.lup);
  h->leafdown = upload_items(h, s, hp.ldown);
  h->lce = upload_items(h, s, hp.llce);
  h->adj_leafF = upload_items(h, s, hp.aF);
  h->adj_leafS = upload_items(h, s, hp.aS);
  h->adj_lce = upload_items(h, s, hp.aL);
  h->adj_leafH = upload_items(h, s, hp.aH);
  h->leaf_reduce_tab = upload(h->al, s, hp.lred, h->owned);
  h->n_leaf_reduce = (int)hp.lred.size() / 3;
  h->fbar_tab = upload(h->al, s, hp.ftab, h->owned);
  h->d_pairs = upload(h->al, s, hp.pairs, h->owned);
  h->bc.p_ws = upload_items(h, s, hp.bc_ws);
  h->bc.p_hx = upload_items(h, s, hp.bc_hx);
  h->bc.p_uN = upload_items(h, s, hp.bc_uN);
  h->bc.p_uW = upload_items(h, s, hp.bc_uW);
}

// Every device access the kernels make is described by the plan; check each descriptor
// against the size of the buffer it touches before anything is launched.
struct PlanCheck {
  std::string err;
  void fail(const std::string& m) {
    if (err.empty()) err = m;
  }
};

void check_rows(PlanCheck& pc, const std::vector<int>& idx, int row, int off, int n, long long rows,
                const char* what) {
  if (n <= 0) return;
  if (off < 0) {
    if (row < 0 || (long long)row + n > rows) pc.fail(std::string(what) + ": contiguous rows out of range");
    return;
  }
  if ((size_t)off + n > idx.size()) {
    pc.fail(std::string(what) + ": index list out of range");
    return;
  }
  for (int k = 0; k < n; ++k) {
    const long long r = (long long)row + idx[off + k];
    if (idx[off + k] < 0 || r >= rows) {
      pc.fail(std::string(what) + ": indexed row out of range");
      return;
    }
  }
}

void check_items(PlanCheck& pc, const std::vector<int>& idx, const std::vector<GemmItem>& items, bool trans,
                 long long ops, long long b0rows, long long b1rows, long long crows, long long addrows,
                 const char* what) {
  for (const GemmItem& it : items) {
    const long long last = trans ? it.a_off + (long long)(it.K - 1) * it.lda + (it.M - 1)
                                 : it.a_off + (long long)(it.M - 1) * it.lda + (it.K - 1);
    if (it.a_off < 0 || last >= ops || it.M < 1 || it.M > ROWBLK || it.K < 1 || it.kseg < 0 || it.kseg > it.K)
      pc.fail(std::string(what) + ": operator block out of range");
    check_rows(pc, idx, it.b0_row, it.b0_idx, it.kseg, b0rows, what);
    check_rows(pc, idx, it.b1_row, it.b1_idx, it.K - it.kseg, b1rows, what);
    check_rows(pc, idx, it.c_row, it.c_idx, it.M, crows, what);
    if (it.add_row >= 0 && (long long)it.add_row + it.M > addrows) pc.fail(std::string(what) + ": addend out of range");
  }
}

void check_prod(PlanCheck& pc, const std::vector<int>& idx, const ProdHost& ph, bool trans, long long ops,
                long long b0rows, long long crows, long long addrows, long long prows, const char* what) {
  check_items(pc, idx, ph.direct, trans, ops, b0rows, 0, crows, addrows, what);
  check_items(pc, idx, ph.split, trans, ops, b0rows, 0, prows, 0, what);
  for (const SplitRed& r : ph.red) {
    if (r.M < 1 || r.nsplit < 1 || r.p_row < 0 || (long long)r.p_row + (long long)r.nsplit * r.M > prows)
      pc.fail(std::string(what) + ": split partials out of range");
    check_rows(pc, idx, r.c_row, r.c_idx, r.M, crows, what);
    if (r.add_row >= 0 && (long long)r.add_row + r.M > addrows) pc.fail(std::string(what) + ": split addend out of range");
  }
}

void check_tab(PlanCheck& pc, const std::vector<int>& tab, long long drows, long long srows, const char* what) {
  if (tab.size() % 3) pc.fail(std::string(what) + ": bad table");
  for (size_t k = 0; k + 2 < tab.size(); k += 3) {
    if (tab[k] < 0 || tab[k] >= drows) pc.fail(std::string(what) + ": destination out of range");
    if (tab[k + 1] >= srows || tab[k + 2] >= srows || tab[k + 1] < -1 || tab[k + 2] < -1)
      pc.fail(std::string(what) + ": source out of range");
  }
}

// Row-combine table of the root conditions: n entries (dst, a, b, sign).
void check_comb(PlanCheck& pc, const std::vector<int>& idx, int off, int n, long long drows, long long arows,
                long long brows, const char* what) {
  if (n == 0) return;
  if (off < 0 || (size_t)off + 4 * (size_t)n > idx.size()) {
    pc.fail(std::string(what) + ": table out of range");
    return;
  }
  for (int k = 0; k < n; ++k) {
    const int* e = &idx[off + 4 * k];
    if (e[0] < 0 || e[0] >= drows || e[1] < 0 || e[1] >= arows || e[2] >= brows || e[2] < -1)
      pc.fail(std::string(what) + ": row out of range");
  }
}

void check_bc(PlanCheck& pc, const hps_handle* h, const HostPlan& hp) {
  const BcPlan& bc = h->bc;
  const std::vector<int>& idx = hp.idx;
  const long long G = h->ns.n_gauss, NB = h->n_bdry, BR = bc.rows, V = h->v_rows;
  const long long ext = (long long)bc.ext.size();
  if (bc.Ks + bc.Ks + bc.nx != ext && bc.periodic) pc.fail("root conditions: seam split");
  if (!bc.periodic && bc.nx != ext) pc.fail("root conditions: node split");
  if (bc.Kn + bc.nd != bc.nx) pc.fail("root conditions: flux split");
  const long long hb = h->hrow_old(bc.root);
  if (hb < 0 || hb + ext > V) pc.fail("root conditions: root flux rows");
  if (bc.periodic) {
    check_comb(pc, idx, bc.c_d, bc.Ks, BR, V, V, "seam data");
    check_comb(pc, idx, bc.c_E, bc.Ks, G, G, 1, "seam copy");
    check_items(pc, idx, hp.bc_ws, false, h->ops_elems, BR, 0, BR, 0, "seam w");
    check_items(pc, idx, hp.bc_hx, false, h->ops_elems, BR, 0, BR, 0, "seam flux");
    check_items(pc, idx, hp.bc_uW, false, h->ops_elems, G, 0, G, BR, "seam values");
    if (bc.tp_off < 0 || bc.tp_off + (long long)bc.nx * bc.nx > hp.tsz) pc.fail("root conditions: T' out of range");
  }
  check_comb(pc, idx, bc.c_hx, bc.nx, BR, V, 1, "root flux gather");
  check_comb(pc, idx, bc.c_fD, bc.nd, G, NB, 1, "value data");
  check_comb(pc, idx, bc.c_r, bc.Kn, BR, NB, BR, "flux data");
  if (bc.Kn > 0) check_items(pc, idx, hp.bc_uN, false, h->ops_elems, BR, G, G, 0, "flux values");
  // assembly tables: (index, sign) pairs inside the source DtN map
  auto check_asm = [&](int off, int n, long long ld, const char* what) {
    if (off < 0 || (size_t)off + 4 * (size_t)n > idx.size()) {
      pc.fail(std::string(what) + ": table out of range");
      return;
    }
    for (int k = 0; k < n; ++k) {
      const int* e = &idx[off + 4 * k];
      if (e[0] < 0 || e[0] >= ld || e[2] < -1 || e[2] >= ld) pc.fail(std::string(what) + ": index out of range");
    }
  };
  if (bc.periodic) {
    check_asm(bc.seam_rt, bc.Ks + bc.nx, ext, "seam rows");
    check_asm(bc.seam_ct, bc.Ks + bc.nx, ext, "seam columns");
  }
  if (bc.Kn > 0) {
    check_asm(bc.neu_rt, bc.Kn, bc.periodic ? bc.nx : ext, "flux rows");
    check_asm(bc.neu_ct, bc.Kn + bc.nd, bc.periodic ? bc.nx : ext, "flux columns");
  }
  const long long troot = h->toff[bc.root];
  const long long text = h->tree.boxes[bc.root].leaf >= 0 ? h->nq : h->k12[bc.root];
  if (troot < 0 || text != ext || troot + ext * ext > hp.tsz) pc.fail("root conditions: root T out of range");
}

std::string validate_plan(const hps_handle* h, const HostPlan& hp) {
  PlanCheck pc;
  if (h->bc.on) check_bc(pc, h, hp);
  const std::vector<int>& idx = hp.idx;
  const long long ops = h->ops_elems, V = h->v_rows, D = h->d_rows, UB = h->ub_rows;
  const long long G = h->ns.n_gauss, LP = (long long)h->n_leaf * h->pp, LB = (long long)h->n_leaf * h->nq;
  const long long gsz = (long long)h->m * (h->m + h->nq), hsz = (long long)h->nq * h->m;
  const long long lops = h->econ ? (long long)h->echunk * (gsz + hsz) : ops;  // econ: chunk buffer
  check_items(pc, idx, hp.lup, false, lops, LP, 0, V, 0, "leaf up");
  check_items(pc, idx, hp.ldown, false, lops, LP, G, LP, 0, "leaf down");
  check_items(pc, idx, hp.llce, false, ops, G, 0, LP, 0, "leaf exterior");
  check_items(pc, idx, hp.aF, true, lops, LP, 0, LP, 0, "adjoint F");
  check_items(pc, idx, hp.aS, true, lops, LP, 0, LB, 0, "adjoint S");
  check_items(pc, idx, hp.aL, true, ops, LP, 0, LB, 0, "adjoint L");
  check_items(pc, idx, hp.aH, true, lops, V, 0, LP, 0, "adjoint H");
  if (h->econ) {
    for (auto* v : {&hp.lup, &hp.ldown, &hp.aF, &hp.aS, &hp.aH})
      if (v->size() % (size_t)h->n_leaf) pc.fail("econ: leaf items are not uniform per leaf");
  }
  check_tab(pc, hp.lred, G, LB, "leaf reduce");
  check_tab(pc, hp.ftab, h->n_bdry, G, "boundary gather");
  for (size_t k = 0; k + 4 < hp.pairs.size() + 1 && k < hp.pairs.size(); k += 5) {
    if (hp.pairs[k] < 0 || hp.pairs[k] >= h->tree.n_edges || hp.pairs[k + 1] < 0 || hp.pairs[k + 1] >= h->n_leaf ||
        hp.pairs[k + 3] < 0 || hp.pairs[k + 3] >= h->n_leaf || hp.pairs[k + 2] < 0 || hp.pairs[k + 2] > 3 ||
        hp.pairs[k + 4] < 0 || hp.pairs[k + 4] > 3)
      pc.fail("edge pairs out of range");
  }
  for (size_t L = 0; L < hp.lv.size(); ++L) {
    const LevelHost& pd = hp.lv[L];
    const Level& lv = h->levels[L];
    check_prod(pc, idx, pd.up, false, ops, D, V, 0, h->p_rows, "merge up");
    check_prod(pc, idx, pd.down, false, ops, G, G, V, h->p_rows, "merge down");
    check_prod(pc, idx, pd.adjS, true, ops, G, UB, 0, h->p_rows, "adjoint S merge");
    check_prod(pc, idx, pd.adjM, true, ops, V, D, 0, h->p_rows, "adjoint X merge");
    check_items(pc, idx, pd.iup, false, ops, V, 0, V, 0, "coarsen up");
    check_items(pc, idx, pd.idown, false, ops, G, 0, G, 0, "refine down");
    check_items(pc, idx, pd.aiup, true, ops, V, 0, V, 0, "adjoint coarsen up");
    check_items(pc, idx, pd.aidown, true, ops, G, 0, G, 0, "adjoint refine down");
    for (size_t i = 0; i < pd.tp1.size(); ++i) {
      const BGemm &a = pd.tp1[i], &b2 = pd.tp2[i];
      if (a.a_off + (long long)a.M * a.lda > hp.tsz || a.b_off + (long long)a.K * a.ldb > ops ||
          a.c_off + (long long)a.M * a.ldc > lv.tp_scratch || b2.a_off + (long long)b2.M * b2.lda > ops ||
          b2.b_off + (long long)b2.K * b2.ldb > lv.tp_scratch || b2.c_off + (long long)b2.M * b2.ldc > hp.tsz ||
          a.N > a.ldb || a.K > a.lda || b2.K > b2.lda || b2.N > b2.ldc)
        pc.fail("coarsened T product out of range");
    }
    check_tab(pc, pd.wcopy, V, G, "adjoint w copy");
    check_tab(pc, pd.reduce, G, UB, "adjoint reduce");
    for (size_t i = 0; i < pd.ug.size(); ++i) {
      const UpGather& u = pd.ug[i];
      const int b = lv.boxes[i];
      const Box& bx = h->tree.boxes[b];
      const long long ka = h->k12[bx.child[0]], kb = h->k12[bx.child[1]];
      if (u.n1 + u.n2 != h->k12o[b]) pc.fail("up gather: parent size mismatch");
      if ((size_t)u.idx_off + 3 * u.k3 + u.n1 + u.n2 > idx.size()) { pc.fail("up gather: list out of range"); continue; }
      for (int k = 0; k < u.k3; ++k) {
        const int a3 = idx[u.idx_off + k], b3 = idx[u.idx_off + u.k3 + k], j3 = idx[u.idx_off + 2 * u.k3 + k];
        if (a3 < 0 || a3 >= ka || b3 < 0 || b3 >= kb || j3 < 0 || j3 >= G) pc.fail("up gather: J3 entry out of range");
      }
      for (int k = 0; k < u.n1; ++k) {
        const int a1 = idx[u.idx_off + 3 * u.k3 + k];
        if (a1 < 0 || a1 >= ka) pc.fail("up gather: J1 entry out of range");
      }
      for (int k = 0; k < u.n2; ++k) {
        const int b2 = idx[u.idx_off + 3 * u.k3 + u.n1 + k];
        if (b2 < 0 || b2 >= kb) pc.fail("up gather: J2 entry out of range");
      }
      if (u.va_row + ka > V || u.vb_row + kb > V || (long long)u.vt_row + u.k3 + u.n1 + u.n2 > V ||
          (long long)u.d_row + u.k3 > D)
        pc.fail("up gather: rows out of range");
    }
    for (size_t i = 0; i < pd.md.size(); ++i) {
      const MergeDesc& md = pd.md[i];
      const GJDesc& gd = pd.gj[i];
      if (md.rows != md.R && md.rows != md.k3) pc.fail("merge row count");
      if (md.m_off + (long long)md.rows * md.R > lv.work_elems || gd.off != md.m_off || gd.R != md.R ||
          gd.K != md.k3 || gd.rows != md.rows || gd.perm_off + gd.K > lv.perm_elems || md.rows > lv.maxRows)
        pc.fail("merge workspace out of range");
      if (md.ta_off + (long long)md.lda_a * md.lda_a > hp.tsz || md.tb_off + (long long)md.lda_b * md.lda_b > hp.tsz)
        pc.fail("merge T store out of range");
      if ((size_t)md.pos_off + 2 * md.R > idx.size()) pc.fail("merge positions out of range");
      else
        for (int r = 0; r < md.R; ++r) {
          if (idx[md.pos_off + r] >= md.lda_a || idx[md.pos_off + md.R + r] >= md.lda_b) pc.fail("merge position too big");
        }
      const int k3 = md.k3, k12 = md.R - md.k3;
      if (pd.tl[i] + (long long)md.rows * k3 > ops || pd.bl[i] != pd.tl[i] + (long long)k3 * k3 ||
          pd.tr[i] + (long long)k3 * k12 > ops ||
          (md.rows > k3 && (pd.br[i] < 0 || pd.br[i] + (long long)k12 * k12 > hp.tsz)))
        pc.fail("merge extraction out of range");
    }
    if (!pd.schur.empty()) {  // blocked elimination
      const int R = pd.gj[0].R;
      const long long wrows = lv.work_elems / R;
      if (pd.gj_top.size() != pd.gj.size() || pd.schur_chunk.size() < 2 || pd.schur_chunk.front() != 0 ||
          pd.schur_chunk.back() != (int)pd.schur.size())
        pc.fail("blocked elimination: descriptors");
      for (size_t i = 0; i < pd.gj.size(); ++i)
        if (pd.gj_top[i].rows != pd.gj[i].K || pd.gj[i].R != R || pd.gj[i].off % R != 0)
          pc.fail("blocked elimination: matrices");
      for (const GemmItem& it : pd.schur)
        if (it.M < 1 || it.M > ROWBLK || it.K < 1 || it.K > 448 || it.lda != R || it.kseg != it.K || it.a_off < 0 ||
            it.a_off + (long long)(it.M - 1) * it.lda + it.K > lv.work_elems || it.b0_idx < 0 ||
            it.b0_idx + it.K > lv.perm_elems || it.b0_row < 0 || it.b0_row + (long long)R > wrows || it.c_idx != -1 ||
            it.c_row < 0 || (long long)it.c_row + it.M > wrows || it.add_row != -1)
          pc.fail("blocked elimination: product item out of range");
      const int ncb = (R + 31) / 32;
      long long blocks = 0;
      for (const BGroup& g : pd.sgrp) {
        if (g.K < 1 || g.K > 448 || g.b0_idx < 0 || g.b0_idx + g.K > lv.perm_elems || g.b0_row < 0 ||
            g.b0_row + (long long)R > wrows || g.blk0 != blocks)
          pc.fail("blocked elimination: vector group out of range");
        blocks += (long long)ncb * ((g.K + 15) / 16);
      }
      if (pd.sbblk.size() != pd.schur.size() || pd.sbexo.size() != pd.schur.size())
        pc.fail("blocked elimination: vector group tables");
      for (size_t i = 0; i < pd.schur.size() && i < pd.sbblk.size() && i < pd.sbexo.size(); ++i)
        if (pd.sbblk[i] < 0 || pd.sbblk[i] + (long long)ncb * ((pd.schur[i].K + 15) / 16) > blocks || pd.sbexo[i] < 0 ||
            (long long)pd.sbexo[i] + ncb * 32 > (long long)pd.sgrp.size() * ncb * 32)
          pc.fail("blocked elimination: item's vector group out of range");
    }
  }
  return pc.err;
}

long long tstore_elems(const hps_handle* h) { return h->tstore_elems; }

// Panel width: 16 (measured fastest on every level of the 64 x 64-leaf tree with either
// update path), capped so the panel fits in shared memory.
int nb_cap(int K, size_t elem) {
  return std::max(1, std::min(16, (int)((200 * 1024) / ((size_t)std::max(K, 1) * (elem + 4)))));
}
int choose_nb(int K, size_t elem, int nmat) {
  (void)nmat;
  return nb_cap(K, elem);
}

// rk: (R, K, rows) of every matrix of the batch, for the grid and the flop counts of the
// timing records.
template <typename T>
void run_gj(const GJDesc* gj, int nmat, int maxR, int maxK, T* work, int* perm, T* pinv, T* prow,
            int* status, const std::vector<std::array<int, 3>>& rk, const char* what, cudaStream_t s,
            int cfg = 0, long long mat_stride = 0) {
  int maxRows = 0;
  for (const auto& m : rk) maxRows = std::max(maxRows, m[2]);
  // cfg = panel width + 100 x path (path 1: the FP64 tensor-core update); 0: fixed rules
  // (the tensor-core update for every FP64 batch: measured fastest on every level)
  const int nb = cfg % 100 > 0 ? std::min(cfg % 100, nb_cap(maxK, sizeof(T))) : choose_nb(maxK, sizeof(T), nmat);
  int tensor = sizeof(T) == 8 && (cfg > 0 ? cfg / 100 : 1);
  // the streamed form of the tensor-core update moves matrix rows by bulk copies, which
  // need 16-byte aligned rows: an aligned workspace and even row lengths (every matrix
  // offset in a batch is a sum of multiples of the row lengths)
  if (tensor) {
    bool even = ((uintptr_t)work & 15) == 0;
    for (const auto& m : rk) even = even && m[0] % 2 == 0;
    if (even) tensor = 2;
  }
  const std::string sf = std::string(tsuf<T>()) + ":" + what;
  TIMED(("gj_init_" + sf).c_str(), 0, 0, launch_gj_init<T>(gj, nmat, perm, s));
  CKL();
  const long long prow_stride = (long long)16 * maxR;
  for (int c0 = 0; c0 < maxK; c0 += nb) {
    double fp = 0, fq = 0, fu = 0, bu = 0;
    for (const auto& m : rk) {
      if (m[1] <= c0) continue;
      const double R = m[0], rows = m[2], b = std::min(nb, m[1] - c0);
      fp += 2.0 * (m[1] - c0) * b * b;
      fq += 2.0 * rows * b * b;
      fu += 2.0 * b * rows * (R - b);
      bu += 2.0 * rows * (R - b) * sizeof(T);
    }
    TIMED(("gj_panel_" + sf).c_str(), fp, 0,
          launch_gj_panel<T>(gj, nmat, maxK, work, perm, pinv, c0, nb, status, s));
    TIMED(("gj_prep_" + sf).c_str(), fq, 0,
          launch_gj_prep<T>(gj, nmat, maxR, work, perm, pinv, prow, prow_stride, c0, nb, s));
    TIMED((std::string(tensor ? "gj_update_tc_" : "gj_update_") + sf).c_str(), fu, bu,
          launch_gj_update<T>(gj, nmat, maxR, maxRows, work, perm, prow, prow_stride, c0, nb, s, status, tensor,
                              mat_stride));
  }
  CKL();
}

// Configuration of one batched elimination (panel width + 100 x update path): the fixed
// rule, or with autotuning the fastest of panel widths 4, 8 and 16 (within the
// shared-memory cap), each with the SIMT and, for FP64, the tensor-core update, measured on
// the batch itself; elim(cfg) assembles the batch's matrices and eliminates them.
int pick_nb(const hps_handle* h, const char* what, size_t elem, const std::vector<std::array<int, 3>>& rk,
            int nmat, cudaStream_t s, const std::function<void(int)>& elim) {
  int maxR = 0, maxK = 0, maxRows = 0;
  for (const auto& m : rk) {
    maxR = std::max(maxR, m[0]);
    maxK = std::max(maxK, m[1]);
    maxRows = std::max(maxRows, m[2]);
  }
  if (!h->opts.autotune) return 0;  // fixed rules inside run_gj
  std::vector<int> cands;
  for (int nb : {4, 8, 16})
    if (nb <= nb_cap(maxK, elem)) {
      cands.push_back(nb);
      if (elem == 8) cands.push_back(100 + nb);
    }
  if (cands.empty()) return 0;
  const std::string key = std::string("gj_cfg ") + what + " e" + std::to_string(elem) + " n" + std::to_string(nmat) +
                          " R" + std::to_string(maxR) + " K" + std::to_string(maxK) + " rows" + std::to_string(maxRows);
  return tuned_choice(key, cands, h->tune_path, [&](int nb) { return time_on_stream(s, [&] { elim(nb); }); });
}

// Root conditions (BcPlan): the periodic seam's elimination [[Z_s, R_s], [-C_s, T_xx]] ->
// [[X_s, S_s], [C_s X_s, T']] and the flux nodes' [T'_NN | T'_ND] -> [X_n | X_n T'_ND], both
// with the build's elimination kernels (one matrix each, FP64), from the root's T.
void build_root_bc(hps_handle* h, double* tstore, cudaStream_t s, const std::function<void*(size_t)>& get) {
  BcPlan& bc = h->bc;
  const int ext = (int)bc.ext.size();
  const double* troot = tstore + h->toff[bc.root];
  auto eliminate = [&](const CombAsm& a, const double* src, const ExtractDst& dst, float null_tol) {
    double* work = (double*)get((size_t)a.rows * a.R * sizeof(double));
    TIMED("root_bc_assemble", 0, (double)a.rows * a.R * 8, launch_comb_assemble(a, src, h->didx, work, s));
    CKL();
    GJDesc gd;
    gd.off = 0;
    gd.R = a.R;
    gd.K = a.K;
    gd.rows = a.rows;
    gd.perm_off = 0;
    gd.box = bc.root;
    gd.null_tol = null_tol;
    if (null_tol > 0.f) {  // scale of the null-direction test: the largest entry
      double* scal = (double*)get(sizeof(double));
      CK(cudaMemsetAsync(scal, 0, sizeof(double), s));
      TIMED("absmax", 0, 0, launch_absmax(work, (long long)a.rows * a.R, scal, s));
      gd.null_scale = scal;
    }
    GJDesc* dgd = (GJDesc*)get(sizeof(GJDesc));
    CK(cudaMemcpyAsync(dgd, &gd, sizeof(GJDesc), cudaMemcpyHostToDevice, s));
    int* perm = (int*)get((size_t)a.K * sizeof(int));
    double* pinv = (double*)get(256 * sizeof(double));
    double* prow = (double*)get((size_t)16 * a.R * sizeof(double));
    run_gj<double>(dgd, 1, a.R, a.K, work, perm, pinv, prow, h->d_status,
                   std::vector<std::array<int, 3>>(1, {a.R, a.K, a.rows}), "root_bc", s, 0, (long long)a.rows * a.R);
    TIMED("gj_extract_f64", 0, (double)a.rows * a.R * 8, launch_gj_extract<double, double>(dgd, 1, a.R, work, perm, dst, s));
    CKL();
  };
  if (bc.periodic) {
    const int Rs = bc.Ks + bc.nx;
    CombAsm a{ext, Rs, Rs, bc.Ks, 1, bc.seam_rt, bc.seam_ct};
    ExtractDst dst{};
    dst.TL = h->ops64 + bc.xs_off;
    dst.TR = h->ops64 + bc.ss_off;
    dst.BL = h->ops64 + bc.cxs_off;
    dst.BR = tstore + bc.tp_off;
    dst.sTL = dst.sTR = dst.sBL = 1.0;
    dst.ld_from_desc = 1;  // X_s, C_s X_s: ld Ks; S_s, T': ld nx
    eliminate(a, troot, dst, 0.f);
  }
  if (bc.Kn > 0) {
    const int Rn = bc.Kn + bc.nd;
    CombAsm a{bc.periodic ? bc.nx : ext, Rn, bc.Kn, bc.Kn, 0, bc.neu_rt, bc.neu_ct};
    ExtractDst dst{};
    dst.TL = h->ops64 + bc.bn_off;
    dst.TL_ld = Rn;
    dst.TR = h->ops64 + bc.bn_off + bc.Kn;
    dst.TR_ld = Rn;
    dst.sTL = 1.0;
    dst.sTR = -1.0;
    dst.sBL = 1.0;
    // Without Dirichlet data on any side, T'_NN can be singular along Gaussian-node
    // directions that the corner-averaged L_ce,ge maps to zero on every leaf (no Chebyshev
    // value sees them): pivots below 1e-9 of the matrix's largest entry are such null
    // directions (unknown set to zero); the legitimate pivots of these systems are orders
    // of magnitude larger (condition numbers up to about 1e6).
    eliminate(a, bc.periodic ? tstore + bc.tp_off : troot, dst, bc.nd == 0 ? 1e-9f : 0.f);
  }
}

void build_stage(hps_handle* h, const double* coeffs, cudaStream_t s) {
  const int m = h->m, nq = h->nq, R = m + nq;
  std::vector<void*> tmp;
  auto get = [&](size_t bytes) {
    void* p = h->al.get(bytes, s);
    tmp.push_back(p);
    return p;
  };
  try {
    // the operator store: FP64, or for HPS_MIXED FP32 only (its sweeps read nothing else),
    // written by the extractions directly
    const bool mixed = h->opts.precision == HPS_MIXED;
    const size_t es = mixed ? sizeof(float) : sizeof(double);
    if (mixed) {
      h->ops32 = (float*)h->al.get(h->ops_elems * sizeof(float), s);
      h->owned.push_back({h->ops32, (size_t)h->ops_elems * sizeof(float)});
      const std::vector<float> lce32(h->rt.Lce.begin(), h->rt.Lce.end());
      CK(cudaMemcpyAsync(h->ops32 + h->lce_base, lce32.data(), lce32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));  // lce32 is a host temporary
    } else {
      h->ops64 = (double*)h->al.get(h->ops_elems * sizeof(double), s);
      h->owned.push_back({h->ops64, (size_t)h->ops_elems * sizeof(double)});
      CK(cudaMemcpyAsync(h->ops64 + h->lce_base, h->rt.Lce.data(), h->rt.Lce.size() * sizeof(double),
                         cudaMemcpyHostToDevice, s));
    }
    unsigned char* opsb = mixed ? (unsigned char*)h->ops32 : (unsigned char*)h->ops64;
    for (size_t b = 0; b < h->tree.boxes.size(); ++b) {
      const Coarsen& co = h->ns.co[b];
      if (!co.active) continue;
      CK(cudaMemcpyAsync(h->ops64 + h->puo[b], co.Pup.data(), co.Pup.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(h->ops64 + h->pdo[b], co.Pdown.data(), co.Pdown.size() * sizeof(double),
                         cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(h->ops64 + h->pco[b], co.Pupc.data(), co.Pupc.size() * sizeof(double),
                         cudaMemcpyHostToDevice, s));
    }
    double* tstore = (double*)get(tstore_elems(h) * sizeof(double));
    const std::vector<long long>& toff = h->toff;
    // ---- leaves (FP64 always), in chunks
    const long long per_leaf = (long long)R * R;
    const long long budget = 3ll << 30;  // bytes of elimination workspace per chunk
    const int n_build = h->shared ? 1 : h->n_leaf;  // shared: leaf 0 stands for every leaf
    int chunk = (int)std::max<long long>(1, std::min<long long>(n_build, budget / (per_leaf * 8)));
    chunk = std::min(chunk, 8192);
    double* work = (double*)get((size_t)per_leaf * chunk * sizeof(double));
    int* perm = (int*)get((size_t)chunk * m * sizeof(int));
    double* pinv = (double*)get((size_t)chunk * 256 * sizeof(double));
    double* prow = (double*)get((size_t)chunk * 16 * R * sizeof(double));
    std::vector<GJDesc> gd(chunk);
    for (int i = 0; i < chunk; ++i) {
      gd[i].off = (long long)i * per_leaf;
      gd[i].R = R;
      gd[i].K = m;
      gd[i].rows = R;
      gd[i].perm_off = i * m;
      gd[i].box = 0;
    }
    LeafTablesDev tb{h->dD, h->dD2, h->dLs, h->dDLs, h->dLloc, h->dDceL, h->didx + h->off_ci};
    for (int l0 = 0; l0 < n_build; l0 += chunk) {
      const int n = std::min(chunk, n_build - l0);
      for (int i = 0; i < n; ++i) gd[i].box = h->tree.leaves[l0 + i];
      GJDesc* dgd = (GJDesc*)get(n * sizeof(GJDesc));
      CK(cudaMemcpyAsync(dgd, gd.data(), n * sizeof(GJDesc), cudaMemcpyHostToDevice, s));
      const std::vector<std::array<int, 3>> rk(n, {R, m, R});
      auto elim = [&](int nb) {
        TIMED("leaf_assemble_f64", 0, (double)n * per_leaf * 8,
              launch_leaf_assemble<double>(coeffs, h->n_leaf, l0, n, h->dhxy, h->p, h->q, tb, work, per_leaf, s));
        CKL();
        run_gj<double>(dgd, n, R, m, work, perm, pinv, prow, h->d_status, rk, "leaf", s, nb, per_leaf);
      };
      elim(pick_nb(h, "leaf", sizeof(double), rk, n, s, elim));
      ExtractDst dst{};
      const long long gl0 = h->gl_base + (long long)l0 * m * R;
      dst.TL = opsb + gl0 * es; dst.TL_off_stride = (long long)m * R; dst.TL_ld = R;
      dst.TR = opsb + (gl0 + m) * es; dst.TR_off_stride = (long long)m * R; dst.TR_ld = R;
      dst.BL = opsb + (h->h_base + (long long)l0 * nq * m) * es; dst.BL_off_stride = (long long)nq * m; dst.BL_ld = m;
      if (h->econ) dst.TL = dst.TR = dst.BL = nullptr;  // only T is kept; F, S, H are recomputed
      dst.BR = tstore + toff[h->tree.leaves[l0]]; dst.BR_off_stride = (long long)nq * nq; dst.BR_ld = nq;
      dst.sTL = 1.0; dst.sTR = -1.0; dst.sBL = -1.0;
      if (mixed)
        TIMED("gj_extract_f64", 0, (double)n * per_leaf * 8, launch_gj_extract<double, float>(dgd, n, R, work, perm, dst, s));
      else
        TIMED("gj_extract_f64", 0, (double)n * per_leaf * 8, launch_gj_extract<double, double>(dgd, n, R, work, perm, dst, s));
      CKL();
    }
    if (h->econ) {  // buffers for recomputing one chunk of leaves during the sweeps
      const int E = h->echunk;
      auto own = [&](size_t bytes) {
        void* p = h->al.get(bytes, s);
        h->owned.push_back({p, bytes});
        return p;
      };
      h->ework = (double*)own((size_t)E * per_leaf * sizeof(double));
      h->eperm = (int*)own((size_t)E * m * sizeof(int));
      h->epinv = (double*)own((size_t)E * 256 * sizeof(double));
      h->eprow = (double*)own((size_t)E * 16 * R * sizeof(double));
      h->eops = (double*)own((size_t)E * ((size_t)m * R + (size_t)nq * m) * sizeof(double));
      std::vector<GJDesc> eg(h->n_leaf);
      for (int lf = 0; lf < h->n_leaf; ++lf) {
        eg[lf].off = (long long)(lf % E) * per_leaf;
        eg[lf].R = R;
        eg[lf].K = m;
        eg[lf].rows = R;
        eg[lf].perm_off = (lf % E) * m;
        eg[lf].box = h->tree.leaves[lf];
      }
      h->egd = upload(h->al, s, eg, h->owned);
    }
    // ---- merges, level by level
    const int H = h->tree.height;
    for (int L = 0; L < H; ++L) {
      Level& lv = h->levels[L];
      const int nmat = (int)lv.boxes.size();
      std::vector<std::array<int, 3>> rk;
      for (int b : lv.boxes) {
        const int R = h->k3[b] + h->k12o[b];
        rk.push_back({R, h->k3[b], (h->tree.boxes[b].parent < 0 && !h->bc.on) ? h->k3[b] : R});
      }
      const double wbytes = (double)lv.work_elems * (lv.fp64 ? 8 : 4);
      ExtractDst dst{};
      dst.TL = opsb; dst.TL_ld = 0; dst.TL_off = lv.off_tl;
      dst.TR = opsb; dst.TR_off = lv.off_tr;
      dst.BL = opsb; dst.BL_off = lv.off_bl;
      dst.BR = tstore; dst.BR_off = lv.off_br;
      dst.sTL = 1.0; dst.sTR = 1.0; dst.sBL = 1.0;
      dst.ld_from_desc = 1;  // X, C X: ld k3; S, T_tau: ld k12
      if (lv.fp64) {
        double* w = (double*)get((size_t)lv.work_elems * sizeof(double));
        int* pm = (int*)get((size_t)std::max(1, lv.perm_elems) * sizeof(int));
        double* pi = (double*)get((size_t)nmat * 256 * sizeof(double));
        double* pr = (double*)get((size_t)nmat * 16 * lv.maxR * sizeof(double));
        // blocked elimination: the digit planes of -C (rows) and of the eliminated top rows
        // (columns) with their exponents, sized once for the level; the product forms no
        // digits and needs no exponent pass
        const ItemSet& sc = lv.schur;
        unsigned char *sdig = nullptr, *sbdig = nullptr;
        int *ser = nullptr, *sbex = nullptr;
        std::vector<std::array<int, 3>> rk_top;
        if (sc.n > 0) {
          sdig = (unsigned char*)get((size_t)gemm_tc_digit_bytes(sc.dsteps));
          ser = (int*)get((size_t)sc.n * 64 * sizeof(int));
          sbdig = (unsigned char*)get((size_t)gemm_tc_bdigit_bytes(lv.sb_blocks));
          sbex = (int*)get((size_t)lv.n_sgrp * ((lv.schur_R + 31) / 32) * 32 * sizeof(int));
          for (auto m : rk) rk_top.push_back({m[0], m[1], m[1]});
        }
        auto elim = [&](int nb) {
          TIMED("merge_assemble_f64", 0, wbytes, launch_merge_assemble<double, double>(lv.md, nmat, lv.maxR, tstore, h->didx, w, s));
          CKL();
          if (sc.n == 0) {
            run_gj<double>(lv.gj, nmat, lv.maxR, lv.maxK, w, pm, pi, pr, h->d_status, rk, "merge", s, nb, lv.mstride);
            return;
          }
          // Gauss-Jordan on the top rows, then bottom = [0 | T] + (-C) Top
          run_gj<double>(lv.gj_top, nmat, lv.maxR, lv.maxK, w, pm, pi, pr, h->d_status, rk_top, "merge", s, nb,
                         lv.mstride);
          const long long k12max = lv.maxR - 1;
          TIMED("gj_schur_digits_f64", 0, 0,
                launch_gemm_tc_digitize(sc.dev, sc.n, 0, w, sc.dstep, sdig, ser, s, true));
          TIMED("gj_schur_digits_f64", 0, 0,
                launch_gemm_tc_bdigitize(lv.sgrp, lv.n_sgrp, (lv.schur_R + 31) / 32, w, pm, lv.schur_R, sbdig, sbex,
                                         s));
          TIMED("gj_schur_zero_f64", 0, 0, launch_gj_zero_bl(lv.gj, nmat, k12max * lv.maxK, w, s));
          for (size_t c = 0; c + 1 < lv.schur_chunk.size(); ++c) {
            const int b = lv.schur_chunk[c], e = lv.schur_chunk[c + 1];
            GemmDigits dg;
            dg.dig = sdig;
            dg.step = sc.dstep + b;
            dg.er = ser + (long long)b * 64;
            dg.bdig = sbdig;
            dg.bblk = lv.sbblk + b;
            dg.bexo = lv.sbexo + b;
            dg.bex = sbex;
            GemmCtx cx;
            cx.maxK = 448;
            cx.maxKv = 448;
            cx.status = h->d_status;
            cx.dg = &dg;
            bool ok = false;
            TIMED("gj_schur_f64", 2.0 * sc.elems * lv.schur_R / std::max<size_t>(1, lv.schur_chunk.size() - 1), 0,
                  ok = launch_gemm_tc(sc.dev + b, e - b, 0, w, w, nullptr, w, nullptr, pm, lv.schur_R, 1.0, s, cx));
            if (!ok) throw CudaError{HPS_ERR_CUDA, "blocked elimination: the tensor-core product could not be launched"};
          }
          CKL();
        };
        elim(pick_nb(h, "merge", sizeof(double), rk, nmat, s, elim));
        if (mixed)
          TIMED("gj_extract_f64", 0, wbytes, launch_gj_extract<double, float>(lv.gj, nmat, lv.maxR, w, pm, dst, s));
        else
          TIMED("gj_extract_f64", 0, wbytes, launch_gj_extract<double, double>(lv.gj, nmat, lv.maxR, w, pm, dst, s));
        CKL();
      } else {
        float* w = (float*)get((size_t)lv.work_elems * sizeof(float));
        int* pm = (int*)get((size_t)std::max(1, lv.perm_elems) * sizeof(int));
        float* pi = (float*)get((size_t)nmat * 256 * sizeof(float));
        float* pr = (float*)get((size_t)nmat * 16 * lv.maxR * sizeof(float));
        auto elim = [&](int nb) {
          TIMED("merge_assemble_f32", 0, wbytes, launch_merge_assemble<float, double>(lv.md, nmat, lv.maxR, tstore, h->didx, w, s));
          CKL();
          run_gj<float>(lv.gj, nmat, lv.maxR, lv.maxK, w, pm, pi, pr, h->d_status, rk, "merge", s, nb);
        };
        elim(pick_nb(h, "merge", sizeof(float), rk, nmat, s, elim));
        TIMED("gj_extract_f32", 0, wbytes, launch_gj_extract<float, float>(lv.gj, nmat, lv.maxR, w, pm, dst, s));
        CKL();
      }
      if (lv.ntp > 0) {  // refined parents: T_new = P_down T P_up (Sec. 6.3)
        double* tmp = (double*)get((size_t)lv.tp_scratch * sizeof(double));
        int mM = 1, mN = 1;
        for (int b : lv.boxes)
          if (h->ns.co[b].active) {
            mM = std::max(mM, std::max(h->k12o[b], h->k12[b]));
            mN = std::max(mN, h->k12[b]);
          }
        TIMED("coarsen_T", 0, 0, launch_bgemm(lv.tp1, lv.ntp, mM, mN, tstore, h->ops64, tmp, s));
        TIMED("coarsen_T", 0, 0, launch_bgemm(lv.tp2, lv.ntp, mM, mN, h->ops64, tmp, tstore, s));
        CKL();
      }
    }
    if (h->bc.on) build_root_bc(h, tstore, s, get);

  } catch (...) {
    for (void* p : tmp) h->al.put(p, s);
    throw;
  }
  for (void* p : tmp) h->al.put(p, s);
}

void ensure_ws(hps_handle* h, int nrhs, cudaStream_t s) {
  Workspace& w = h->ws;
  if (w.nrhs >= nrhs) {
    h->tc_scales = w.tc_scales;
    h->tc_units = w.tc_units;
    return;
  }
  h->drop_graph();  // a captured sweep points into the old buffers
  for (void* p : w.ptrs) h->al.put(p, s);
  w = Workspace();
  h->tc_scales = nullptr;
  h->tc_units = 0;
  // the new buffers are made in a local workspace and installed only when all of them
  // exist: a failed allocation releases the others and leaves the handle without a
  // workspace (the next call makes one again)
  Workspace nw;
  nw.nrhs = nrhs;
  auto get = [&](size_t bytes) {
    void* p = nullptr;
    try {
      p = h->al.get(bytes, s);
    } catch (...) {
      for (void* q : nw.ptrs) h->al.put(q, s);
      throw;
    }
    nw.ptrs.push_back(p);
    return p;
  };
  const long long R = nrhs;
  const long long nuc = (long long)h->n_leaf * h->pp * R;
  const long long ng = (long long)h->ns.n_gauss * R;
  const bool mixed = h->opts.precision == HPS_MIXED;
  nw.V64 = (double*)get((size_t)h->v_rows * R * sizeof(double));
  nw.P64 = (double*)get((size_t)std::max(1, h->p_rows) * R * sizeof(double));
  nw.d64 = (double*)get((size_t)std::max(1, h->d_rows) * R * sizeof(double));
  nw.ug64 = (double*)get((size_t)ng * sizeof(double));
  if (mixed) {
    nw.V32 = (float*)get((size_t)h->v_rows * R * sizeof(float));
    nw.P32 = (float*)get((size_t)std::max(1, h->p_rows) * R * sizeof(float));
    nw.d32 = (float*)get((size_t)std::max(1, h->d_rows) * R * sizeof(float));
    nw.ug32 = (float*)get((size_t)ng * sizeof(float));
    nw.g32 = (float*)get((size_t)nuc * sizeof(float));
    nw.uc32 = (float*)get((size_t)nuc * sizeof(float));
    nw.rho32 = (float*)get((size_t)ng * sizeof(float));
    nw.vflux = (double*)get((size_t)h->n_leaf * h->nq * R * sizeof(double));
    nw.rho64 = (double*)get((size_t)ng * sizeof(double));
  } else {
    nw.LB = (double*)get((size_t)h->n_leaf * h->nq * R * sizeof(double));
    nw.UB = (double*)get((size_t)std::max(1, h->ub_rows) * R * sizeof(double));
    nw.ubar = (double*)get((size_t)ng * sizeof(double));
  }
  nw.scal = (double*)get(4 * sizeof(double));
  if (mixed && h->opts.fp32_gemm != HPS_GEMM_SIMT && gemm_tc32_eligible(nrhs)) gemm_tc32_prepare();
  if (h->opts.fp64_gemm != HPS_GEMM_SIMT && nrhs >= 8) {
    gemm_tc_prepare();
    nw.tc_units = (long long)h->max_items * ((nrhs + 31) / 32);
    nw.tc_scales = (int*)get((size_t)gemm_tc_scale_bytes(nw.tc_units));
  }
  if (h->bc.on) nw.bcw = (double*)get((size_t)std::max(1, h->bc.rows) * R * sizeof(double));
  w = nw;
  h->tc_scales = w.tc_scales;
  h->tc_units = w.tc_units;
}

// Econ mode: rebuild the leaf operators [F | S_ci] and H of chunk c into the chunk buffer
// (the same assembly, elimination and extraction as the build, T discarded).
void recompute_leaf_chunk(hps_handle* h, int c, cudaStream_t s) {
  const int E = h->echunk, l0 = c * E, n = std::min(E, h->n_leaf - l0);
  const int m = h->m, nq = h->nq, R = m + nq;
  const long long per_leaf = (long long)R * R;
  LeafTablesDev tb{h->dD, h->dD2, h->dLs, h->dDLs, h->dLloc, h->dDceL, h->didx + h->off_ci};
  TIMED("leaf_assemble_f64", 0, (double)n * per_leaf * 8,
        launch_leaf_assemble<double>(h->coeffs_copy, h->n_leaf, l0, n, h->dhxy, h->p, h->q, tb, h->ework, per_leaf,
                                     s));
  run_gj<double>(h->egd + l0, n, R, m, h->ework, h->eperm, h->epinv, h->eprow, h->d_status,
                 std::vector<std::array<int, 3>>(n, {R, m, R}), "leaf_econ", s, 0, per_leaf);
  ExtractDst dst{};
  dst.TL = h->eops; dst.TL_off_stride = (long long)m * R; dst.TL_ld = R;
  dst.TR = h->eops + m; dst.TR_off_stride = (long long)m * R; dst.TR_ld = R;
  dst.BL = h->eops + (long long)E * m * R; dst.BL_off_stride = (long long)nq * m; dst.BL_ld = m;
  dst.sTL = 1.0; dst.sTR = -1.0; dst.sBL = -1.0;
  TIMED("gj_extract_f64", 0, (double)n * per_leaf * 8,
        launch_gj_extract<double, double>(h->egd + l0, n, R, h->ework, h->eperm, dst, s));
  CKL();
}

// The operator digit cache of an FP64 item set for the tensor-core products (the operators
// are fixed after the build; `ops` is the FP64 operator store the items index, trans how the
// product reads them).  It is formed outside stream capture on the set's second application
// (a handle solved once does not pay for it) or when `now` is set (before a sweep is
// captured, so that the replayed graph reads it).  nullptr when the products do not run on
// the tensor cores, before the cache exists, inside hps_solve_noalloc, or if the allocation
// failed; the products then form the operator digits themselves (same results).
const GemmDigits* item_digits(hps_handle* h, const ItemSet& is, int trans, const double* ops, int nrhs,
                              cudaStream_t s, bool now = false) {
  if (h->opts.fp64_gemm == HPS_GEMM_SIMT || is.n == 0 || is.dsteps == 0 || !gemm_tc_eligible(is.maxK, nrhs))
    return nullptr;
  if (!now) ++is.uses;
  if (!is.dg.dig && !is.dg_tried && !h->noalloc_call && (now || is.uses >= 2)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      is.dg_tried = true;
      try {
        const size_t db = (size_t)gemm_tc_digit_bytes(is.dsteps), eb = (size_t)is.n * 64 * sizeof(int);
        unsigned char* dig = (unsigned char*)h->al.get(db, s);
        h->owned.push_back({dig, db});
        int* er = (int*)h->al.get(eb, s);
        h->owned.push_back({er, eb});
        TIMED("gemm_digits", 0, (double)db, launch_gemm_tc_digitize(is.dev, is.n, trans, ops, is.dstep, dig, er, s));
        CKL();
        is.dg.dig = dig;
        is.dg.step = is.dstep;
        is.dg.er = er;
      } catch (const CudaError&) {
        cudaGetLastError();
      }
    }
  }
  return is.dg.dig ? &is.dg : nullptr;
}

// The bf16 operator pieces of an FP32 item set for the tensor-core products (the FP32 copy of
// the operators is fixed after the build), formed like item_digits: on the set's second
// tensor-core application outside stream capture, or when `now` is set; nullptr otherwise
// (the products then split the operator themselves, same results).
const GemmDigits* item_pieces32(hps_handle* h, const ItemSet& is, int nrhs, cudaStream_t s, bool now = false) {
  if (h->opts.fp32_gemm == HPS_GEMM_SIMT || is.n == 0 || is.dsteps == 0 || !gemm_tc32_eligible(nrhs) || !h->ops32)
    return nullptr;
  if (!now) ++is.uses32;
  if (!is.dg32.dig && !is.dg32_tried && (now || is.uses32 >= 2)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      is.dg32_tried = true;
      try {
        const size_t db = (size_t)gemm_tc32_piece_bytes(is.dsteps);
        unsigned char* dig = (unsigned char*)h->al.get(db, s);
        h->owned.push_back({dig, db});
        TIMED("gemm_pieces_f32", 0, (double)db, launch_gemm_tc32_pieces(is.dev, is.n, h->ops32, is.dstep, dig, s));
        CKL();
        is.dg32.dig = dig;
        is.dg32.step = is.dstep;
      } catch (const CudaError&) {
        cudaGetLastError();
      }
    }
  }
  return is.dg32.dig ? &is.dg32 : nullptr;
}

// Items [l0, l0 + n) leaves of a leaf item set (every leaf has the same number of items).
ItemSet leaf_range(const hps_handle* h, const ItemSet& is, int l0, int n) {
  ItemSet r;
  const int per = is.n / h->n_leaf;
  r.dev = is.dev + (long long)l0 * per;
  r.n = n * per;
  r.maxK = is.maxK;  // no digit cache: these operators are rebuilt chunk by chunk
  r.elems = is.elems * (double)n / h->n_leaf;
  return r;
}

// Launch options of a product of item set `is` for the handle's current call.
GemmCtx gemm_ctx(const hps_handle* h, int maxK, const GemmDigits* dg = nullptr, int bn = 0) {
  GemmCtx cx;
  cx.bn = bn;
  cx.maxK = h->opts.fp64_gemm == HPS_GEMM_SIMT ? 0 : maxK;
  cx.maxKv = maxK;
  cx.status = h->d_status;
  cx.dg = dg;
  cx.tc_scales = h->tc_scales;
  cx.tc_units = h->tc_units;
  cx.tc32 = h->opts.fp32_gemm != HPS_GEMM_SIMT;
  return cx;
}

// One pass of Algorithm 2 with operator type TA and vector type TV.
//   f: [n_bdry][nrhs] FP64 (scattered as TV), g: [n_leaf][pp][nrhs] TV, rho: optional
//   FP64 [n_gauss][nrhs], outputs uc [n_leaf][pp][nrhs] TV and ug [n_gauss][nrhs] TV.
// Root conditions in the solve (BcPlan): from the root's particular flux h (rows of V),
// the seam values u_s = S_s u_x + X_s d_s, the flux nodes' values
// u_N = X_n (f_N - h'_N) - X_n T'_ND u_D and the value nodes' data u_D = f_D, written into
// the Gaussian vector ug for the downward pass.  FP64.
void root_bc_solve(hps_handle* h, const double* ops, const double* f, double* V, double* ug, int nrhs,
                   cudaStream_t s) {
  const BcPlan& bc = h->bc;
  const int* idx = h->didx;
  double* bcw = h->ws.bcw;
  auto prod = [&](const char* name, const ItemSet& is, const double* B0, const double* B1, double* C,
                  const double* Add, double beta) {
    const GemmDigits* dg = item_digits(h, is, 0, ops, nrhs, s);
    TIMED(name, 2.0 * is.elems * nrhs, is.elems * 8.0,
          launch_gemm_items<double, double>(is.dev, is.n, ROWBLK, 0, ops, B0, B1, C, Add, idx, nrhs, beta, s,
                                            gemm_ctx(h, is.maxK, dg)));
  };
  if (bc.periodic) {
    TIMED("root_bc_rows", 0, 0, launch_row_combine(idx + bc.c_d, bc.Ks, bcw, V, V, nrhs, s));
    prod("gemm_root_bc_f64", bc.p_ws, bcw, nullptr, bcw, nullptr, 0.0);
  }
  TIMED("root_bc_rows", 0, 0, launch_row_combine(idx + bc.c_hx, bc.nx, bcw, V, nullptr, nrhs, s));
  if (bc.periodic) prod("gemm_root_bc_f64", bc.p_hx, bcw, nullptr, bcw, nullptr, 1.0);
  TIMED("root_bc_rows", 0, 0, launch_row_combine(idx + bc.c_fD, bc.nd, ug, f, nullptr, nrhs, s));
  if (bc.Kn > 0) {
    TIMED("root_bc_rows", 0, 0, launch_row_combine(idx + bc.c_r, bc.Kn, bcw, f, bcw, nrhs, s));
    prod("gemm_root_bc_f64", bc.p_uN, bcw, ug, ug, nullptr, 0.0);
  }
  if (bc.periodic) {
    prod("gemm_root_bc_f64", bc.p_uW, ug, nullptr, ug, bcw, 0.0);
    TIMED("root_bc_rows", 0, 0, launch_row_combine(idx + bc.c_E, bc.Ks, ug, ug, nullptr, nrhs, s));
  }
  CKL();
}

template <typename TA, typename TV>
void solve_pass(hps_handle* h, const TA* ops, const double* f, const TV* g, const double* rho, TV* uc, TV* ug,
                TV* V, TV* dbuf, TV* P, int nrhs, cudaStream_t s) {
  const int H = h->tree.height;
  const int* idx = h->didx;
  const std::string sf = tsuf<TA>();
  auto gemm = [&](const char* step, const ItemSet& is, const TV* B0, const TV* B1, TV* C, const TV* Add,
                  double beta) {
    int bn = 0;
    // FP64 products on the tensor cores (exact digit slicing) where they apply
    const int mk = h->opts.fp64_gemm == HPS_GEMM_SIMT ? 0 : is.maxK;
    const bool tc = std::is_same<TA, double>::value
                        ? gemm_tc_eligible(mk, nrhs)
                        : (h->opts.fp32_gemm != HPS_GEMM_SIMT && gemm_tc32_eligible(nrhs));
    // right-hand-side tile: tuned for products that overwrite their output (beta = 0), so
    // that a trial run can be repeated; looked up only while the sweep is being captured
    if (h->opts.autotune && !tc && nrhs > 16 && beta == 0.0 && is.n > 0) {
      std::vector<int> cands{16, 32};
      if (nrhs > 32) cands.push_back(64);
      const std::string key = "gemm_bn " + std::string(step) + " " + sf + " nrhs" + std::to_string(nrhs) +
                              " items" + std::to_string(is.n) + " elems" + std::to_string((long long)is.elems);
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      CK(cudaStreamIsCapturing(s, &cs));
      std::function<float(int)> trial;
      if (cs == cudaStreamCaptureStatusNone)
        trial = [&](int b) {
          return time_on_stream(s, [&] {
            launch_gemm_items<TA, TV>(is.dev, is.n, ROWBLK, 0, ops, B0, B1, C, Add, idx, nrhs, beta, s,
                                      gemm_ctx(h, 0, nullptr, b));
          });
        };
      bn = tuned_choice(key, cands, h->tune_path, trial);
    }
    const GemmDigits* dg = nullptr;
    if constexpr (std::is_same<TA, double>::value) {
      if (tc) dg = item_digits(h, is, 0, ops, nrhs, s);
    } else {
      if (tc) dg = item_pieces32(h, is, nrhs, s);
    }
    TIMED(("gemm_" + std::string(step) + "_" + sf).c_str(), 2.0 * is.elems * nrhs, is.elems * sizeof(TA),
          launch_gemm_items<TA, TV>(is.dev, is.n, ROWBLK, 0, ops, B0, B1, C, Add, idx, nrhs, beta, s,
                                    gemm_ctx(h, is.maxK, dg, bn)));
  };
  auto gemmp = [&](const char* step, const Prod& pr, const TV* B0, TV* C, const TV* Add, double beta) {
    gemm(step, pr.direct, B0, nullptr, C, Add, beta);
    if (pr.nred > 0) {
      gemm(step, pr.split, B0, nullptr, P, nullptr, 0.0);
      TIMED("split_reduce", 0, 0, launch_split_reduce<TV>(pr.red, pr.nred, P, C, Add, idx, nrhs, beta, s));
    }
  };
  // leaf steps read the stored operators, or (econ) operators rebuilt chunk by chunk
  auto leaf_step = [&](const char* step, const ItemSet& is, const TV* B0, const TV* B1, TV* C) {
    if (!h->econ) {
      gemm(step, is, B0, B1, C, nullptr, 0.0);
      return;
    }
    if constexpr (std::is_same<TA, double>::value) {
      for (int c = 0; c * h->echunk < h->n_leaf; ++c) {
        recompute_leaf_chunk(h, c, s);
        const int l0 = c * h->echunk, n = std::min(h->echunk, h->n_leaf - l0);
        const ItemSet r = leaf_range(h, is, l0, n);
        TIMED(("gemm_" + std::string(step) + "_" + sf).c_str(), 2.0 * r.elems * nrhs, r.elems * sizeof(TA),
              launch_gemm_items<TA, TV>(r.dev, r.n, ROWBLK, 0, h->eops, B0, B1, C, nullptr, idx, nrhs, 0.0, s,
                                        gemm_ctx(h, r.maxK)));
      }
    }
  };
  // upward pass: leaves, then merges bottom-up
  leaf_step("leaf_up", h->leafup, g, nullptr, V);
  for (int L = 0; L < H; ++L) {
    Level& lv = h->levels[L];
    TIMED("up_gather", 0, 0, launch_up_gather<TV>(lv.ug, (int)lv.boxes.size(), lv.ug_maxrows, V, V, dbuf, rho, idx, nrhs, s));
    gemmp("merge_up", lv.up, dbuf, V, nullptr, 1.0);
    if (lv.iup.n) gemm("coarsen_up", lv.iup, V, nullptr, V, nullptr, 0.0);
  }
  // root boundary data (or the values that periodic / Neumann root conditions give), then
  // the downward pass
  if (h->bc.on) {
    if constexpr (std::is_same<TA, double>::value && std::is_same<TV, double>::value)
      root_bc_solve(h, ops, f, V, ug, nrhs, s);
  } else if (f) {
    TIMED("scatter_rows", 0, 0, launch_scatter_rows<TV>(f, idx + h->off_bnd, h->n_bdry, ug, nrhs, s));
  }
  for (int L = H - 1; L >= 0; --L) {
    Level& lv = h->levels[L];
    if (lv.idown.n) gemm("refine_down", lv.idown, ug, nullptr, ug, nullptr, 0.0);
    gemmp("merge_down", lv.down, ug, ug, V, 0.0);
  }
  leaf_step("leaf_down", h->leafdown, g, ug, uc);
  gemm("leaf_ext", h->lce, ug, nullptr, uc, nullptr, 0.0);
  CKL();
}

// Operator digit caches of every FP64 product set of the sweep, formed before a capture.
void prepare_sweep_digits(hps_handle* h, int nrhs, cudaStream_t s) {
  const double* ops = h->ops64;
  auto one = [&](const ItemSet& is) { item_digits(h, is, 0, ops, nrhs, s, true); };
  if (!h->econ) {
    one(h->leafup);
    one(h->leafdown);
  }
  one(h->lce);
  for (const Level& lv : h->levels) {
    if (!lv.fp64) continue;
    one(lv.up.direct);
    one(lv.up.split);
    one(lv.down.direct);
    one(lv.down.split);
    one(lv.iup);
    one(lv.idown);
  }
}

ResidualArgs residual_args(const hps_handle* h, const double* coeffs) {
  ResidualArgs ra;
  ra.coeffs = coeffs;
  ra.n_leaf = h->n_leaf;
  ra.p = h->p;
  ra.q = h->q;
  ra.hxy = h->dhxy;
  ra.D = h->dD;
  ra.D2 = h->dD2;
  ra.Lloc = h->dLloc;
  ra.ci = h->didx + h->off_ci;
  ra.Lloc_df = h->dLloc_df;
  ra.Lce_c = h->dLce_c;
  ra.Lce_off = h->dLce_off;
  ra.n_lce = h->n_lce;
  ra.D_df = h->dD_df;
  ra.D2_df = h->dD2_df;
  ra.Lce_blk = h->dLce_blk;
  return ra;
}

// Mixed precision (HPS_MIXED): FP32 sweeps refined against the residual of the collocation
// system computed in double-float arithmetic, corrections accumulated in FP64.
//
// The low-precision solve of the original system: u (FP64) and the Gaussian-node vector
// ug64, with the exact boundary data.
void mixed_initial(hps_handle* h, const double* f, const double* g, const double* rho, double* u, int nrhs,
                   cudaStream_t s) {
  Workspace& w = h->ws;
  const long long nuc = (long long)h->n_leaf * h->pp * nrhs;
  const long long ng = (long long)h->ns.n_gauss * nrhs;
  TIMED("convert", 0, nuc * 12.0, launch_convert<double, float>(g, w.g32, nuc, 1.0, s));
  CK(cudaMemsetAsync(w.ug32, 0, ng * sizeof(float), s));
  solve_pass<float, float>(h, h->ops32, f, w.g32, rho, w.uc32, w.ug32, w.V32, w.d32, w.P32, nrhs, s);
  TIMED("convert", 0, nuc * 12.0, launch_convert<float, double>(w.uc32, u, nuc, 1.0, s));
  TIMED("convert", 0, ng * 12.0, launch_convert<float, double>(w.ug32, w.ug64, ng, 1.0, s));
  TIMED("scatter_rows", 0, 0, launch_scatter_rows<double>(f, h->didx + h->off_bnd, h->n_bdry, w.ug64, nrhs, s));
  CKL();
}

// One refinement step: the residual of the collocation system (leaf equations and flux
// jumps), an FP32 correction solve with the jumps as flux-continuity data, the FP64
// update.  With measure, max|du| goes to scal[0] and max|u| to scal[1].
void mixed_step(hps_handle* h, const double* g, const double* rho, double* u, int nrhs, bool measure,
                cudaStream_t s) {
  Workspace& w = h->ws;
  const long long nuc = (long long)h->n_leaf * h->pp * nrhs;
  const long long ng = (long long)h->ns.n_gauss * nrhs;
  const ResidualArgs ra = residual_args(h, h->coeffs_copy);
  // derivative passes (5 p^3), exterior refresh (ne 4q) and fluxes (4q p) per leaf and rhs
  const double res_flops = 2.0 * ((double)h->n_leaf * nrhs) *
                           (5.0 * h->p * h->p * h->p + (double)h->ne * h->nq + (double)h->nq * h->p + 12.0 * h->m);
  TIMED("leaf_residual_df", res_flops, nuc * 32.0,
        launch_leaf_residual_df(ra, h->d_leaf_edges, h->didx + h->off_ce, w.ug64, g, u, w.g32, w.vflux, nrhs, s));
  CK(cudaMemsetAsync(w.rho64, 0, ng * sizeof(double), s));
  TIMED("jump_residual", 0, 0, launch_jump_residual(h->d_pairs, h->npairs, h->q, w.vflux, w.rho64, nrhs, s));
  if (rho) TIMED("axpy", 0, 0, launch_axpy_to_f64<double>(rho, w.rho64, ng, s));
  CKL();
  CK(cudaMemsetAsync(w.ug32, 0, ng * sizeof(float), s));
  solve_pass<float, float>(h, h->ops32, nullptr, w.g32, w.rho64, w.uc32, w.ug32, w.V32, w.d32, w.P32, nrhs, s);
  if (measure) {  // the update and the norms of the correction and of u in one pass
    CK(cudaMemsetAsync(w.scal, 0, 2 * sizeof(double), s));
    TIMED("axpy", 0, nuc * 20.0, launch_axpy_measure(w.uc32, u, nuc, w.scal, s));
  } else {
    TIMED("axpy", 0, nuc * 20.0, launch_axpy_to_f64<float>(w.uc32, u, nuc, s));
  }
  TIMED("axpy", 0, ng * 20.0, launch_axpy_to_f64<float>(w.ug32, w.ug64, ng, s));
  CKL();
}

// The fixed-schedule refined solve: the initial solve and nfix corrections (the last one
// measured).  Exterior values need no final refresh: each residual pass writes
// u_ce = L_ce,ge u_ge back into u in double-float arithmetic, and the correction then adds
// its own L_ce,ge du_ge, whose FP32 error is about 2^-24 |du|, far below the tolerance.
void mixed_fixed(hps_handle* h, const double* f, const double* g, double* u, int nrhs, int nfix, cudaStream_t s) {
  mixed_initial(h, f, g, nullptr, u, nrhs, s);
  for (int k = 0; k < nfix; ++k) mixed_step(h, g, nullptr, u, nrhs, k == nfix - 1, s);
}

// Operator pieces of every FP32 product set of the mixed sweep, formed before a capture.
void prepare_sweep_pieces32(hps_handle* h, int nrhs, cudaStream_t s) {
  auto one = [&](const ItemSet& is) { item_pieces32(h, is, nrhs, s, true); };
  one(h->leafup);
  one(h->leafdown);
  one(h->lce);
  for (const Level& lv : h->levels) {
    one(lv.up.direct);
    one(lv.up.split);
    one(lv.down.direct);
    one(lv.down.split);
    one(lv.iup);
    one(lv.idown);
  }
}

// Capture the solve for this nrhs into a CUDA graph that reads its inputs from (and writes
// u to) staging buffers owned by the handle: the FP64 sweep, or for HPS_MIXED the
// fixed-schedule refined solve with nfix corrections.  Capture runs on a private stream; a
// capture failure disables graphs for this handle (direct launches remain).
void capture_solve(hps_handle* h, int nrhs, int nfix, cudaStream_t s) {
  h->drop_graph();
  Workspace& w = h->ws;
  const bool mixed = h->opts.precision == HPS_MIXED;
  const long long nuc = (long long)h->n_leaf * h->pp * nrhs;
  const long long ng = (long long)h->ns.n_gauss * nrhs;
  h->graph.f_in = (double*)h->al.get((size_t)h->n_bdry * nrhs * sizeof(double), s);
  h->graph.g_in = (double*)h->al.get((size_t)nuc * sizeof(double), s);
  h->graph.u_out = (double*)h->al.get((size_t)nuc * sizeof(double), s);
  if (!mixed) prepare_sweep_digits(h, nrhs, s);
  else prepare_sweep_pieces32(h, nrhs, s);
  CK(cudaStreamSynchronize(s));
  if (!h->graph.cs) CK(cudaStreamCreateWithFlags(&h->graph.cs, cudaStreamNonBlocking));
  cudaStream_t cs = h->graph.cs;
  cudaGraph_t graph = nullptr;
  timing_suspend(true);
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    try {
      if (mixed) {
        mixed_fixed(h, h->graph.f_in, h->graph.g_in, h->graph.u_out, nrhs, nfix, cs);
      } else {
        cudaMemsetAsync(w.ug64, 0, ng * sizeof(double), cs);
        solve_pass<double, double>(h, h->ops64, h->graph.f_in, h->graph.g_in, nullptr, h->graph.u_out, w.ug64, w.V64,
                                   w.d64, w.P64, nrhs, cs);
      }
    } catch (const CudaError&) {
    }
    e = cudaStreamEndCapture(cs, &graph);
  }
  timing_suspend(false);
  if (e == cudaSuccess && graph) {
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
    int nk = 0;
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
    }
    h->graph.kernels = nk;
    double el = h->leafup.elems + h->leafdown.elems + h->lce.elems;
    for (const Level& lv : h->levels)
      el += lv.up.direct.elems + lv.up.split.elems + lv.down.direct.elems + lv.down.split.elems + lv.iup.elems +
            lv.idown.elems;
    const int sweeps = mixed ? 1 + nfix : 1;
    h->graph.flops = 2.0 * el * nrhs * sweeps;
    h->graph.bytes = (mixed ? 4.0 : 8.0) * el * sweeps;
    e = cudaGraphInstantiate(&h->graph.exec, graph, 0);
  }
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || !h->graph.exec) {
    cudaGetLastError();
    h->graph.exec = nullptr;
    h->graph.broken = true;
    return;
  }
  h->graph.nrhs = nrhs;
  h->graph.nfix = nfix;
}

// Run the captured graph for this call if there is one (capturing it on the second call
// with the same nrhs); false if the caller has to launch directly.
bool graph_solve(hps_handle* h, const double* f, const double* g, double* u, int nrhs, int nfix, cudaStream_t s) {
  if (!h->opts.use_graphs || h->graph.broken) return false;
  if ((h->graph.nrhs != nrhs || h->graph.nfix != nfix) && h->graph.last_nrhs == nrhs) capture_solve(h, nrhs, nfix, s);
  h->graph.last_nrhs = nrhs;
  if (!h->graph.exec || h->graph.nrhs != nrhs || h->graph.nfix != nfix) return false;
  const long long nuc = (long long)h->n_leaf * h->pp * nrhs;
  CK(cudaMemcpyAsync(h->graph.f_in, f, (size_t)h->n_bdry * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->graph.g_in, g, nuc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  {
    TimingScope ts_(h->opts.precision == HPS_MIXED ? "graph_solve_mixed" : "graph_solve_f64", s, h->graph.flops,
                    h->graph.bytes, std::max(1, h->graph.kernels));
    CK(cudaGraphLaunch(h->graph.exec, s));
  }
  CK(cudaMemcpyAsync(u, h->graph.u_out, nuc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return true;
}

int solve_fp64(hps_handle* h, const double* f, const double* g, const double* rho, int nrhs, double* u,
               double* ug_out, cudaStream_t s) {
  ensure_ws(h, nrhs, s);
  Workspace& w = h->ws;
  const long long ng = (long long)h->ns.n_gauss * nrhs;
  if (rho || !graph_solve(h, f, g, u, nrhs, 0, s)) {
    CK(cudaMemsetAsync(w.ug64, 0, ng * sizeof(double), s));
    solve_pass<double, double>(h, h->ops64, f, g, rho, u, w.ug64, w.V64, w.d64, w.P64, nrhs, s);
  }
  if (ug_out) CK(cudaMemcpyAsync(ug_out, w.ug64, ng * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return HPS_OK;
}

// HPS_MIXED solve.  Until the handle has a calibrated contraction bound, the refinement is
// adaptive: after every correction the host reads max|du| and max|u| and stops when the
// correction is below tolerance, or when the observed contraction r = |du_k| / |du_(k-1)|
// (< 1/2) predicts the error left after it, 2 r |du_k|, below tolerance.  The ratios seen
// calibrate the bound rho (twice the largest ratio) and the number nfix of corrections
// with rho^nfix e_0 below tolerance (e_0 = |du_1| / |u|, the initial solve's error).
// Later solves without flux-jump
// data run the initial solve and nfix corrections without testing in between (one CUDA
// graph), then test once: rho |du_nfix| <= tol max|u|.  A solve that fails the test goes
// on adaptively from where it is and recalibrates.
int solve_mixed(hps_handle* h, const double* f, const double* g, const double* rho, int nrhs, double* u,
                double* ug_out, int* iters, cudaStream_t s) {
  ensure_ws(h, nrhs, s);
  Workspace& w = h->ws;
  const long long ng = (long long)h->ns.n_gauss * nrhs;
  const double tol = h->opts.ir_tol;
  auto read2 = [&](double* sc) {
    CK(cudaMemcpyAsync(sc, w.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  };
  int it = 0;
  bool conv = false;
  double prev = -1.0, first = -1.0, ratio = 0.0;
  double sc[2] = {0.0, 0.0};
  const int nfix = h->ir.nfix;
  if (!rho && nfix > 0 && h->ir.rho > 0.0) {
    if (!graph_solve(h, f, g, u, nrhs, nfix, s)) mixed_fixed(h, f, g, u, nrhs, nfix, s);
    read2(sc);
    it = nfix;
    if (!(sc[0] == sc[0]) || !(sc[1] == sc[1])) return fail(HPS_ERR_NO_CONVERGENCE, "refinement produced NaN");
    conv = h->ir.rho * sc[0] <= tol * sc[1];
    prev = sc[0];
  } else {
    mixed_initial(h, f, g, rho, u, nrhs, s);
  }
  for (; !conv && it < h->opts.ir_max_iter; ++it) {
    mixed_step(h, g, rho, u, nrhs, true, s);
    read2(sc);
    if (!(sc[0] == sc[0]) || !(sc[1] == sc[1])) break;
    const double tolu = tol * sc[1];
    if (first < 0.0) first = sc[0] / std::max(sc[1], 1e-300);
    if (prev > 0.0) ratio = std::max(ratio, sc[0] / prev);
    const bool small = sc[0] <= tolu;
    const bool predicted = prev > 0.0 && sc[0] < 0.5 * prev && 2.0 * (sc[0] / prev) * sc[0] <= tolu;
    // a contraction bound already measured on this operator (by the build) predicts the
    // remaining error from a single correction
    const bool bounded = !rho && h->ir.rho > 0.0 && h->ir.rho * sc[0] <= tolu;
    prev = sc[0];
    if (small || predicted || bounded) {
      conv = true;
      ++it;
      // calibrate from the ratios of this solve (needs two corrections of the original
      // system), and the number of corrections from this solve's first one
      if (!rho && ratio > 0.0 && ratio < 0.5) h->ir.rho = std::max(h->ir.rho, 2.0 * ratio);
      if (!rho && h->ir.rho > 0.0 && h->ir.rho < 1.0 && first > 0.0) {
        int n = 1;
        double e = first;
        while (n < h->opts.ir_max_iter && (e *= h->ir.rho) > tol) ++n;
        h->ir.nfix = std::max(h->ir.nfix, n);
      }
      break;
    }
  }
  if (ug_out) CK(cudaMemcpyAsync(ug_out, w.ug64, ng * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (iters) *iters = it;
  if (!conv) return fail(HPS_ERR_NO_CONVERGENCE, "iterative refinement did not converge in " + std::to_string(it) + " steps");
  return HPS_OK;
}

// Contraction bound of the refinement, measured once at the end of a mixed build on a model
// problem of the same operator (no load, the linear boundary data 1 + x + 2 y: a smooth
// solution, with data compatible at the corners).  The bound is a property of the operator
// and of the FP32 sweeps; the number of corrections also depends on the size of the first
// correction, which differs between problems, so it is left to the first solve, which then
// accepts as soon as the bound predicts convergence.  Best effort: a failure here leaves the
// handle uncalibrated and reports nothing.
void calibrate_mixed(hps_handle* h, cudaStream_t s) {
  const std::string saved = g_err;
  const long long nf = h->n_bdry, ng = (long long)h->n_leaf * h->pp;
  std::vector<void*> bufs;
  try {
    // boundary data at the boundary Gaussian nodes (ascending id), from the leaves' edges
    std::vector<double> fh((size_t)std::max(nf, 1ll), 0.0);
    {
      const Tree& t = h->tree;
      const int q = h->q;
      std::vector<double> fall((size_t)t.n_edges * q, 0.0);
      for (size_t lf = 0; lf < t.leaves.size(); ++lf) {
        const Box& b = t.boxes[t.leaves[lf]];
        for (int sd = 0; sd < 4; ++sd)
          for (int k = 0; k < q; ++k) {
            const double gx = b.x0 + 0.5 * (b.x1 - b.x0) * (h->rt.xg[k] + 1.0);
            const double gy = b.y0 + 0.5 * (b.y1 - b.y0) * (h->rt.xg[k] + 1.0);
            const double x = sd == 0 || sd == 2 ? gx : (sd == 1 ? b.x1 : b.x0);
            const double y = sd == 1 || sd == 3 ? gy : (sd == 0 ? b.y0 : b.y1);
            fall[(size_t)t.leaf_edges[4 * lf + sd] * q + k] = 1.0 + x + 2.0 * y;
          }
      }
      for (long long i = 0; i < nf; ++i) fh[i] = fall[h->ns.boundary[i]];
    }
    double* f = (double*)h->al.get(fh.size() * sizeof(double), s);
    bufs.push_back(f);
    double* g = (double*)h->al.get((size_t)ng * sizeof(double), s);
    bufs.push_back(g);
    double* u = (double*)h->al.get((size_t)ng * sizeof(double), s);
    bufs.push_back(u);
    CK(cudaMemcpyAsync(f, fh.data(), fh.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(g, 0, (size_t)ng * sizeof(double), s));
    int it = 0;
    solve_mixed(h, f, g, nullptr, 1, u, nullptr, &it, s);
    CK(cudaStreamSynchronize(s));
    h->ir.nfix = 0;
  } catch (const CudaError&) {
    cudaGetLastError();
  } catch (const std::exception&) {
  }
  for (void* b : bufs) h->al.put(b, s);
  g_err = saved;
}

}  // namespace

extern "C" {

void hps_opts_default(hps_opts* o) {
  if (!o) return;
  o->precision = HPS_FP64;
  o->q = 0;
  o->store_leaf_ops = 1;
  o->ir_tol = 0.0;
  o->ir_max_iter = 0;
  o->fp64_top_levels = -1;
  o->use_graphs = 1;
  o->autotune = 0;
  o->autotune_cache = nullptr;
  o->shared_leaf = -1;
  o->bc_we = HPS_BC_DIRICHLET;
  o->bc_sn = HPS_BC_DIRICHLET;
  o->fp64_gemm = HPS_GEMM_TENSOR;
  o->fp32_gemm = HPS_GEMM_TENSOR;
}

int hps_selftest_wait_timeout(int polls, void* stream) {
  if (polls < 1 || polls > (1 << 26)) return fail(HPS_ERR_INVALID_ARG, "polls must be in [1, 2^26]");
  cudaStream_t s = (cudaStream_t)stream;
  int* d = nullptr;
  if (cudaMallocAsync(&d, 2 * sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return fail(HPS_ERR_OOM, "device allocation failed");
  }
  int h[2] = {0, 0};
  cudaMemsetAsync(d, 0, 2 * sizeof(int), s);
  const int rc = wait_selftest(polls, d, s);
  cudaMemcpyAsync(h, d, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFreeAsync(d, s);
  if (rc != 0 || e != cudaSuccess) {
    cudaGetLastError();
    return fail(HPS_ERR_CUDA, "self-test launch failed");
  }
  if (h[0] == -1 && h[1] == 1) return fail(HPS_ERR_TIMEOUT, "the wait ran out and the abort flag stopped the other role");
  return fail(HPS_ERR_STATE, "self-test: status " + std::to_string(h[0]) + ", flag seen " + std::to_string(h[1]));
}

const char* hps_last_error(void) { return g_err.c_str(); }

int hps_tree_uniform(double x0, double y0, double x1, double y1, int nx, int ny, hps_tree** out) {
  if (!out) return fail(HPS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || (long long)nx * ny > (1ll << 24))
    return fail(HPS_ERR_INVALID_ARG, "nx, ny must be in [1, 65536] with nx*ny <= 2^24");
  if (!(x1 > x0) || !(y1 > y0)) return fail(HPS_ERR_INVALID_ARG, "empty domain");
  hps_tree* t = new (std::nothrow) hps_tree();
  if (!t) return fail(HPS_ERR_OOM, "host allocation failed");
  make_uniform_tree(x0, y0, x1, y1, nx, ny, t->t);
  *out = t;
  return HPS_OK;
}

int hps_tree_destroy(hps_tree* t) {
  delete t;
  return HPS_OK;
}

int hps_tree_info(const hps_tree* tree, int q, int* n_leaves, int* n_boxes, int* n_levels, int* n_gauss,
                  int* n_boundary) {
  if (!tree) return fail(HPS_ERR_INVALID_ARG, "tree is NULL");
  if (q < 1) return fail(HPS_ERR_INVALID_ARG, "q must be >= 1");
  const Tree& t = tree->t;
  if (n_leaves) *n_leaves = (int)t.leaves.size();
  if (n_boxes) *n_boxes = (int)t.boxes.size();
  if (n_levels) *n_levels = t.height;
  if (n_gauss) *n_gauss = t.n_edges * q;
  if (n_boundary) {
    std::vector<int> bnd;
    boundary_nodes(t, q, bnd);
    *n_boundary = (int)bnd.size();
  }
  return HPS_OK;
}

int hps_nodes(const hps_tree* tree, int p, int q, int which, double* xy, int64_t* count) {
  if (!tree || !count) return fail(HPS_ERR_INVALID_ARG, "tree or count is NULL");
  if (p < 3 || p > 64 || q < 1 || q > 64) return fail(HPS_ERR_INVALID_ARG, "p must be in [3,64], q in [1,64]");
  const Tree& t = tree->t;
  RefTables rt;
  build_ref_tables(p, q, rt);
  if (which == HPS_NODES_CHEB_LEAF) {
    *count = (int64_t)t.leaves.size() * p * p;
    if (!xy) return HPS_OK;
    for (size_t lf = 0; lf < t.leaves.size(); ++lf) {
      const Box& b = t.boxes[t.leaves[lf]];
      for (int iy = 0; iy < p; ++iy)
        for (int ix = 0; ix < p; ++ix) {
          const size_t k = (lf * p + iy) * p + ix;
          xy[2 * k] = b.x0 + 0.5 * (b.x1 - b.x0) * (rt.xc[ix] + 1.0);
          xy[2 * k + 1] = b.y0 + 0.5 * (b.y1 - b.y0) * (rt.xc[iy] + 1.0);
        }
    }
    return HPS_OK;
  }
  if (which != HPS_NODES_GAUSS_BOUNDARY && which != HPS_NODES_GAUSS_ALL)
    return fail(HPS_ERR_INVALID_ARG, "unknown node set");
  std::vector<double> all((size_t)2 * t.n_edges * q);
  for (size_t lf = 0; lf < t.leaves.size(); ++lf) {
    const Box& b = t.boxes[t.leaves[lf]];
    for (int s = 0; s < 4; ++s) {
      const int e = t.leaf_edges[4 * lf + s];
      for (int k = 0; k < q; ++k) {
        const double gx = b.x0 + 0.5 * (b.x1 - b.x0) * (rt.xg[k] + 1.0);
        const double gy = b.y0 + 0.5 * (b.y1 - b.y0) * (rt.xg[k] + 1.0);
        double x, y;
        switch (s) {
          case 0: x = gx; y = b.y0; break;
          case 1: x = b.x1; y = gy; break;
          case 2: x = gx; y = b.y1; break;
          default: x = b.x0; y = gy; break;
        }
        all[2 * ((size_t)e * q + k)] = x;
        all[2 * ((size_t)e * q + k) + 1] = y;
      }
    }
  }
  if (which == HPS_NODES_GAUSS_ALL) {
    *count = (int64_t)t.n_edges * q;
    if (xy) std::memcpy(xy, all.data(), all.size() * sizeof(double));
    return HPS_OK;
  }
  std::vector<int> bnd;
  boundary_nodes(t, q, bnd);
  if (xy)
    for (size_t n = 0; n < bnd.size(); ++n) {
      xy[2 * n] = all[2 * (size_t)bnd[n]];
      xy[2 * n + 1] = all[2 * (size_t)bnd[n] + 1];
    }
  *count = (int64_t)bnd.size();
  return HPS_OK;
}

int hps_tree_mask(double x0, double y0, double h, int nx, int ny, const uint8_t* mask, hps_tree** out) {
  if (!out) return fail(HPS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!mask) return fail(HPS_ERR_INVALID_ARG, "mask is NULL");
  if (nx < 1 || ny < 1 || (long long)nx * ny > (1ll << 24)) return fail(HPS_ERR_INVALID_ARG, "bad grid size");
  if (!(h > 0.0)) return fail(HPS_ERR_INVALID_ARG, "h must be positive");
  hps_tree* t = new (std::nothrow) hps_tree();
  if (!t) return fail(HPS_ERR_OOM, "host allocation failed");
  if (make_mask_tree(x0, y0, h, nx, ny, mask, t->t) != 0) {
    delete t;
    return fail(HPS_ERR_INVALID_ARG, "mask selects no square");
  }
  *out = t;
  return HPS_OK;
}

int hps_tree_refine(const hps_tree* tree, const double* pts_xy, int npts, int levels, hps_tree** out) {
  if (!out) return fail(HPS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!tree || (npts > 0 && !pts_xy) || npts < 0) return fail(HPS_ERR_INVALID_ARG, "tree or points missing");
  if (levels < 0 || levels > 12) return fail(HPS_ERR_INVALID_ARG, "levels must be in [0, 12]");
  long long span = 0;
  for (const Box& b : tree->t.boxes) span = std::max<long long>(span, std::max(b.i1, b.j1));
  if ((span << levels) > (1ll << 28)) return fail(HPS_ERR_INVALID_ARG, "refinement too deep for this tree");
  hps_tree* t = new (std::nothrow) hps_tree();
  if (!t) return fail(HPS_ERR_OOM, "host allocation failed");
  refine_tree(tree->t, pts_xy, npts, levels, t->t);
  *out = t;
  return HPS_OK;
}

}  // extern "C"

namespace {

// Options, reference tables, node sets and the size checks shared by hps_build and
// hps_plan_check.  Returns an empty string or the reason the tree/options are rejected.
// Root conditions by side (Sec. 7.6): the boundary node ids of the west, east, south and
// north sides of a rectangular domain; the facing west/east nodes for a periodic seam;
// the split of the remaining root exterior nodes into flux (Neumann) and value nodes.
std::string classify_sides(hps_handle* h, const hps_opts& o) {
  const Tree& t = h->tree;
  BcPlan& bc = h->bc;
  bc = BcPlan();
  bc.periodic = o.bc_we == HPS_BC_PERIODIC;
  bc.neumann = o.bc_sn == HPS_BC_NEUMANN;
  bc.on = bc.periodic || bc.neumann;
  if (!bc.on) return std::string();
  for (size_t b = 0; b < t.boxes.size(); ++b)
    if (t.boxes[b].parent < 0) bc.root = (int)b;
  const Box& r = t.boxes[bc.root];
  bc.ext = r.leaf >= 0 ? h->ns.ge[bc.root] : h->ns.ge_old[bc.root];
  const int q = h->q;
  // the leaves must tile the root's rectangle; the sides are then the edges on its lines
  long long area = 0;
  for (int b : t.leaves) {
    const Box& bx = t.boxes[b];
    area += (long long)(bx.i1 - bx.i0) * (bx.j1 - bx.j0);
  }
  if (area != (long long)(r.i1 - r.i0) * (r.j1 - r.j0)) return "periodic or Neumann sides need a rectangular domain";
  std::vector<std::array<int, 3>> side[4];  // S, E, N, W: (lo, hi, edge)
  for (int e = 0; e < t.n_edges; ++e) {
    const std::array<int, 4>& k = t.edge_keys[e];
    int sd = -1;
    if (k[0] == 0 && k[1] == r.j0) sd = 0;
    else if (k[0] == 1 && k[1] == r.i1) sd = 1;
    else if (k[0] == 0 && k[1] == r.j1) sd = 2;
    else if (k[0] == 1 && k[1] == r.i0) sd = 3;
    if (sd >= 0) side[sd].push_back({k[2], k[3], e});
  }
  for (auto& v : side) std::sort(v.begin(), v.end());
  auto ids = [&](const std::vector<std::array<int, 3>>& v) {
    std::vector<int> out;
    for (const auto& a : v)
      for (int kk = 0; kk < q; ++kk) out.push_back(a[2] * q + kk);
    return out;
  };
  std::set<int> seam, flux;
  if (bc.periodic) {
    if (side[1].size() != side[3].size()) return "periodic west/east sides need matching nodes";
    for (size_t i = 0; i < side[1].size(); ++i)
      if (side[1][i][0] != side[3][i][0] || side[1][i][1] != side[3][i][1])
        return "periodic west/east sides need matching nodes";
    bc.W = ids(side[3]);
    bc.E = ids(side[1]);
    seam.insert(bc.W.begin(), bc.W.end());
    seam.insert(bc.E.begin(), bc.E.end());
  }
  if (bc.neumann) {
    for (int sd : {0, 2})
      for (int g : ids(side[sd])) flux.insert(g);
  }
  std::set<int> ext(bc.ext.begin(), bc.ext.end());
  for (int sd = 0; sd < 4; ++sd)
    for (int g : ids(side[sd]))
      if (!ext.count(g)) return "root exterior does not match the domain boundary";
  for (int g : bc.ext) {
    if (seam.count(g)) continue;
    bc.X.push_back(g);
    if (flux.count(g)) bc.N.push_back(g);
    else bc.D.push_back(g);
  }
  bc.Ks = (int)bc.W.size();
  bc.nx = (int)bc.X.size();
  bc.Kn = (int)bc.N.size();
  bc.nd = (int)bc.D.size();
  bc.rows = 2 * bc.Ks + bc.nx + bc.Kn;
  return std::string();
}

// Every leaf spans the same number of finest-grid units in x and in y (so all leaves have
// the same size and the same reference-to-physical scaling).
bool equal_leaf_spans(const Tree& t) {
  if (t.leaves.empty()) return false;
  const Box& b0 = t.boxes[t.leaves[0]];
  for (int b : t.leaves) {
    const Box& bx = t.boxes[b];
    if (bx.i1 - bx.i0 != b0.i1 - b0.i0 || bx.j1 - bx.j0 != b0.j1 - b0.j0) return false;
  }
  return true;
}

std::string setup_host(hps_handle* h, const Tree& tree, int p, const hps_opts& o, bool shared) {
  h->tree = tree;
  h->opts = o;
  h->shared = shared;
  h->p = p;
  h->q = o.q;
  h->pp = p * p;
  h->m = (p - 2) * (p - 2);
  h->nq = 4 * o.q;
  h->ne = 4 * (p - 1);
  h->n_leaf = (int)h->tree.leaves.size();
  build_ref_tables(p, h->q, h->rt);
  build_node_sets(h->tree, h->q, h->ns, h->rt.xg);
  h->n_bdry = (int)h->ns.boundary.size();
  bool coarsened = false;
  for (const Coarsen& c : h->ns.co) coarsened = coarsened || c.active;
  if (coarsened && o.precision == HPS_MIXED)
    return "HPS_MIXED needs a tree without coarse-fine interfaces (its residual checks only matching edges)";
  // every Gaussian node must end up in some merge's J3, the domain boundary, or a
  // coarsened side: a node owned by one leaf that is none of these is an interface the
  // refinement rule left unmatched
  {
    std::vector<char> seen((size_t)h->ns.n_gauss, 0);
    for (size_t b = 0; b < h->tree.boxes.size(); ++b) {
      for (int g : h->ns.J3[b]) seen[g] = 1;
      for (int g : h->ns.co[b].fine) seen[g] = 1;
    }
    for (int g : h->ns.boundary) seen[g] = 1;
    for (int g = 0; g < h->ns.n_gauss; ++g)
      if (!seen[g]) return "mesh has an unmatched interface (refined leaves next to leaves more than one size larger)";
  }
  for (size_t b = 0; b < h->tree.boxes.size(); ++b)
    if (h->tree.boxes[b].leaf < 0 && h->ns.J3[b].empty()) return "a merge has no shared edge";
  return classify_sides(h, o);
}

int check_opts(int p, const hps_opts* opts, hps_opts& o) {
  if (p < 4 || p > 32) return fail(HPS_ERR_INVALID_ARG, "p must be in [4, 32]");
  hps_opts_default(&o);
  if (opts) o = *opts;
  if (o.q == 0) o.q = p - 1;
  if (o.q < 2 || o.q > 32) return fail(HPS_ERR_INVALID_ARG, "q must be in [2, 32]");
  if (o.precision != HPS_FP64 && o.precision != HPS_MIXED) return fail(HPS_ERR_INVALID_ARG, "unknown precision");
  if (o.store_leaf_ops != 0 && o.store_leaf_ops != 1) return fail(HPS_ERR_INVALID_ARG, "store_leaf_ops must be 0 or 1");
  if (o.store_leaf_ops == 0 && o.precision != HPS_FP64)
    return fail(HPS_ERR_INVALID_ARG, "leaf recomputation (store_leaf_ops = 0) needs precision HPS_FP64");
  if (o.shared_leaf < -1 || o.shared_leaf > 1) return fail(HPS_ERR_INVALID_ARG, "shared_leaf must be -1, 0 or 1");
  if (o.bc_we != HPS_BC_DIRICHLET && o.bc_we != HPS_BC_PERIODIC)
    return fail(HPS_ERR_INVALID_ARG, "bc_we must be HPS_BC_DIRICHLET or HPS_BC_PERIODIC");
  if (o.bc_sn != HPS_BC_DIRICHLET && o.bc_sn != HPS_BC_NEUMANN)
    return fail(HPS_ERR_INVALID_ARG, "bc_sn must be HPS_BC_DIRICHLET or HPS_BC_NEUMANN");
  if ((o.bc_we != HPS_BC_DIRICHLET || o.bc_sn != HPS_BC_DIRICHLET) && o.precision != HPS_FP64)
    return fail(HPS_ERR_INVALID_ARG, "periodic or Neumann sides need precision HPS_FP64");
  if (o.fp64_gemm != HPS_GEMM_TENSOR && o.fp64_gemm != HPS_GEMM_SIMT)
    return fail(HPS_ERR_INVALID_ARG, "fp64_gemm must be HPS_GEMM_TENSOR or HPS_GEMM_SIMT");
  if (o.fp32_gemm != HPS_GEMM_TENSOR && o.fp32_gemm != HPS_GEMM_SIMT)
    return fail(HPS_ERR_INVALID_ARG, "fp32_gemm must be HPS_GEMM_TENSOR or HPS_GEMM_SIMT");
  if (o.ir_tol <= 0.0) o.ir_tol = 1e-8;
  if (o.ir_max_iter <= 0) o.ir_max_iter = 10;
  return HPS_OK;
}

}  // namespace

extern "C" {

int hps_plan_check(const hps_tree* tree, int p, const hps_opts* opts) {
  if (!tree) return fail(HPS_ERR_INVALID_ARG, "tree is NULL");
  hps_opts o;
  const int rc = check_opts(p, opts, o);
  if (rc != HPS_OK) return rc;
  hps_handle* h = new (std::nothrow) hps_handle();
  if (!h) return fail(HPS_ERR_OOM, "host allocation failed");
  std::string err;
  try {
    bool shared = false;
    if (o.shared_leaf == 1) {
      shared = equal_leaf_spans(tree->t);
      if (!shared) err = "shared_leaf = 1 needs leaves of one size";
    }
    if (err.empty()) err = setup_host(h, tree->t, p, o, shared);
    if (err.empty()) {
      HostPlan hp;
      make_plan(h, hp);
      err = validate_plan(h, hp);
      if (!err.empty()) err = "internal plan check failed: " + err;
    }
  } catch (const std::exception& e) {
    err = e.what();
  }
  delete h;
  if (!err.empty()) return fail(HPS_ERR_INVALID_ARG, err);
  return HPS_OK;
}

int hps_build(const hps_tree* tree, const double* coeffs, int p, const hps_opts* opts, const hps_allocator* alloc,
              void* stream, hps_handle** out) {
  if (!out) return fail(HPS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!tree || !coeffs) return fail(HPS_ERR_INVALID_ARG, "tree or coeffs is NULL");
  hps_opts o;
  const int rc = check_opts(p, opts, o);
  if (rc != HPS_OK) return rc;
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(HPS_ERR_INVALID_ARG, "allocator callbacks missing");
  cudaStream_t s = (cudaStream_t)stream;
  hps_handle* h = new (std::nothrow) hps_handle();
  if (!h) return fail(HPS_ERR_OOM, "host allocation failed");
  if (alloc) {
    h->al.a = *alloc;
    h->al.custom = true;
  }
  try {
    // the coefficient fields: finite, and elliptic principal part (c11 > 0 and
    // c11 c22 - c12^2 > 0) at every interior node (device check, one synchronisation)
    {
      const int nl = (int)tree->t.leaves.size();
      int* bad = (int*)h->al.get(2 * sizeof(int), s);
      int res[2] = {INT_MAX, INT_MAX};
      try {
        CK(cudaMemcpyAsync(bad, res, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
        launch_coeff_check(coeffs, nl, p, bad, s);
        CKL();
        CK(cudaMemcpyAsync(res, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
      } catch (...) {
        h->al.put(bad, s);
        throw;
      }
      h->al.put(bad, s);
      if (res[0] != INT_MAX) {
        delete h;
        return fail(HPS_ERR_INVALID_ARG, "a coefficient is not finite at an interior node of leaf " +
                                             std::to_string(res[0]));
      }
      if (res[1] != INT_MAX) {
        delete h;
        return fail(HPS_ERR_NOT_ELLIPTIC, "c11 > 0 and c11 c22 - c12^2 > 0 fail at an interior node of leaf " +
                                              std::to_string(res[1]));
      }
    }
    // shared leaf operators: equal leaf sizes (host) and equal interior coefficients
    // (device check, one synchronisation)
    bool shared = false;
    if (o.shared_leaf != 0 && equal_leaf_spans(tree->t)) {
      int* flag = (int*)h->al.get(sizeof(int), s);
      int differ = 1;
      try {
        CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
        launch_leaf_uniform_check(coeffs, (int)tree->t.leaves.size(), p, flag, s);
        CKL();
        CK(cudaMemcpyAsync(&differ, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
      } catch (...) {
        h->al.put(flag, s);
        throw;
      }
      h->al.put(flag, s);
      shared = differ == 0;
    }
    if (o.shared_leaf == 1 && !shared) {
      delete h;
      return fail(HPS_ERR_INVALID_ARG, "shared_leaf = 1 needs leaves of one size with equal interior coefficients");
    }
    // host plan: from the tree's cache, or made, checked and cached
    std::shared_ptr<const HostPlan> plan;
    {
      std::lock_guard<std::mutex> lk(tree->cache_mu);
      if (!tree->cache) tree->cache = std::make_shared<PlanCache>();
      const std::array<int, 6> key = plan_key(p, o, shared);
      for (const PlanCache::Entry& e : tree->cache->entries)
        if (e.key == key) {
          const Alloc al = h->al;
          *h = *e.layout;
          h->al = al;
          h->opts = o;
          plan = e.plan;
          break;
        }
      if (!plan) {
        std::string err = setup_host(h, tree->t, p, o, shared);
        auto hp = std::make_shared<HostPlan>();
        if (err.empty()) {
          make_plan(h, *hp);
          err = validate_plan(h, *hp);
          if (!err.empty()) err = "internal plan check failed: " + err;
        }
        if (!err.empty()) {
          delete h;
          return fail(HPS_ERR_INVALID_ARG, err);
        }
        auto lay = std::make_shared<hps_handle>(*h);  // host fields only: nothing is on the device yet
        lay->al = Alloc();
        if (tree->cache->entries.size() >= PlanCache::kMax) tree->cache->entries.erase(tree->cache->entries.begin());
        tree->cache->entries.push_back({key, lay, hp});
        plan = hp;
      }
    }
    h->tune_path = o.autotune_cache ? o.autotune_cache : "";
    // device tables
    h->dD = upload(h->al, s, h->rt.D, h->owned);
    h->dD2 = upload(h->al, s, h->rt.D2, h->owned);
    h->dLs = upload(h->al, s, h->rt.Ls, h->owned);
    h->dDLs = upload(h->al, s, h->rt.DLs, h->owned);
    h->dLloc = upload(h->al, s, h->rt.Lloc, h->owned);
    h->dLloc_df = (float2*)upload(h->al, s, split_df(h->rt.Lloc), h->owned);
    {
      const BlockRows lb = block_rows(h->rt.Lce, h->rt.ne, h->q);
      h->dLce_c = (float2*)upload(h->al, s, lb.vals, h->owned);
      h->dLce_blk = upload(h->al, s, lb.blk, h->owned);
      h->dLce_off = upload(h->al, s, lb.off, h->owned);
      h->n_lce = lb.off.back();
    }
    h->dD_df = (float2*)upload(h->al, s, split_df(h->rt.D), h->owned);
    h->dD2_df = (float2*)upload(h->al, s, split_df(h->rt.D2), h->owned);
    h->dDceL = upload(h->al, s, h->rt.DceL, h->owned);
    std::vector<double> hxy(2 * (size_t)h->n_leaf);
    for (int lf = 0; lf < h->n_leaf; ++lf) {
      const Box& b = h->tree.boxes[h->tree.leaves[lf]];
      hxy[2 * lf] = b.x1 - b.x0;
      hxy[2 * lf + 1] = b.y1 - b.y0;
    }
    h->dhxy = upload(h->al, s, hxy, h->owned);
    h->d_leaf_edges = upload(h->al, s, h->tree.leaf_edges, h->owned);
    std::vector<int> st(1, 0);
    h->d_status = upload(h->al, s, st, h->owned);
    upload_plan(h, *plan, s);
    if (o.precision == HPS_MIXED || o.store_leaf_ops == 0) {
      const size_t cb = (size_t)6 * h->n_leaf * h->pp * sizeof(double);
      h->coeffs_copy = (double*)h->al.get(cb, s);
      h->owned.push_back({h->coeffs_copy, cb});
      CK(cudaMemcpyAsync(h->coeffs_copy, coeffs, cb, cudaMemcpyDeviceToDevice, s));
    }
    build_stage(h, coeffs, s);
    int status = 0;
    CK(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (status < 0) {
      delete h;
      return fail(HPS_ERR_TIMEOUT, "a tensor-core update did not complete within its wait limit");
    }
    if (status != 0) {
      const int box = status - 1;
      delete h;
      return fail(HPS_ERR_SINGULAR, "pivot breakdown in the elimination of box " + std::to_string(box));
    }
    if (o.precision == HPS_MIXED) calibrate_mixed(h, s);
  } catch (const CudaError& e) {
    delete h;
    return fail(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(HPS_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    delete h;
    return fail(HPS_ERR_INVALID_ARG, e.what());
  }
  *out = h;
  return HPS_OK;
}

int hps_solve_ext(hps_handle* h, const double* f, const double* g, const double* rho, int nrhs, double* u,
                  double* ug_out, int* iters, void* stream) {
  if (!h) return fail(HPS_ERR_INVALID_ARG, "handle is NULL");
  if (!f || !g || !u) return fail(HPS_ERR_INVALID_ARG, "f, g and u must be device pointers");
  if (nrhs < 1 || nrhs > 4096) return fail(HPS_ERR_INVALID_ARG, "nrhs must be in [1, 4096]");
  cudaStream_t s = (cudaStream_t)stream;
  try {
    if (iters) *iters = 0;
    if (h->opts.precision == HPS_FP64) return solve_fp64(h, f, g, rho, nrhs, u, ug_out, s);
    return solve_mixed(h, f, g, rho, nrhs, u, ug_out, iters, s);
  } catch (const CudaError& e) {
    return fail(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(HPS_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(HPS_ERR_INVALID_ARG, e.what());
  }
}

int hps_apply(hps_handle* h, const double* coeffs, const double* u, int nrhs, double alpha, double beta, double* out,
              void* stream) {
  if (!h) return fail(HPS_ERR_INVALID_ARG, "handle is NULL");
  if (!coeffs || !u || !out) return fail(HPS_ERR_INVALID_ARG, "coeffs, u and out must be device pointers");
  if (nrhs < 1 || nrhs > 4096) return fail(HPS_ERR_INVALID_ARG, "nrhs must be in [1, 4096]");
  cudaStream_t s = (cudaStream_t)stream;
  try {
    const ResidualArgs ra = residual_args(h, coeffs);
    TIMED("leaf_apply_df", 2.0 * h->n_leaf * nrhs * 5.0 * h->p * h->p * h->p, (double)h->n_leaf * h->pp * nrhs * 16.0,
          launch_leaf_apply_df(ra, u, alpha, beta, out, nrhs, s));
    CKL();
    return HPS_OK;
  } catch (const CudaError& e) {
    return fail(e.code, e.msg);
  }
}

int hps_solve(hps_handle* h, const double* f, const double* g, int nrhs, double* u, void* stream) {
  return hps_solve_ext(h, f, g, nullptr, nrhs, u, nullptr, nullptr, stream);
}

int hps_adjoint(hps_handle* h, const double* ubar_in, int nrhs, const double* u, double* fbar, double* gbar,
                double* cbar, void* stream) {
  if (!h) return fail(HPS_ERR_INVALID_ARG, "handle is NULL");
  if (!ubar_in) return fail(HPS_ERR_INVALID_ARG, "dJdu is NULL");
  if (nrhs < 1 || nrhs > 4096) return fail(HPS_ERR_INVALID_ARG, "nrhs must be in [1, 4096]");
  if (h->opts.precision != HPS_FP64) return fail(HPS_ERR_STATE, "hps_adjoint needs an HPS_FP64 handle");
  if (h->bc.on) return fail(HPS_ERR_STATE, "hps_adjoint needs Dirichlet data on every side");
  if (cbar && !u) return fail(HPS_ERR_INVALID_ARG, "coefficient gradients need the forward solution u");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<void*> tmp;  // call-local buffers, released on every exit
  try {
    ensure_ws(h, nrhs, s);
    Workspace& w = h->ws;
    const long long nuc = (long long)h->n_leaf * h->pp * nrhs;
    const long long ng = (long long)h->ns.n_gauss * nrhs;
    const int* idx = h->didx;
    const double* ops = h->ops64;
    double* gb = gbar;
    if (!gb) {
      gb = (double*)h->al.get(nuc * sizeof(double), s);
      tmp.push_back(gb);
    }
    double* VB = w.V64;
    double* ub = w.ubar;
    CK(cudaMemsetAsync(gb, 0, nuc * sizeof(double), s));
    CK(cudaMemsetAsync(VB, 0, (size_t)h->v_rows * nrhs * sizeof(double), s));
    auto gemmT = [&](const char* step, const ItemSet& is, const double* B0, double* C, double beta) {
      const GemmDigits* dg = item_digits(h, is, 1, ops, nrhs, s);
      TIMED(("gemmT_" + std::string(step) + "_f64").c_str(), 2.0 * is.elems * nrhs, is.elems * 8.0,
            launch_gemm_items<double, double>(is.dev, is.n, ROWBLK, 1, ops, B0, nullptr, C, nullptr, idx, nrhs, beta,
                                              s, gemm_ctx(h, is.maxK, dg)));
    };
    auto gemmTp = [&](const char* step, const Prod& pr, const double* B0, double* C, double beta) {
      gemmT(step, pr.direct, B0, C, beta);
      if (pr.nred > 0) {
        gemmT(step, pr.split, B0, w.P64, 0.0);
        TIMED("split_reduce", 0, 0,
              launch_split_reduce<double>(pr.red, pr.nred, w.P64, C, nullptr, idx, nrhs, beta, s));
      }
    };
    // leaf steps: stored operators, or (econ) operators rebuilt chunk by chunk
    auto leafT = [&](const char* step, const ItemSet& is, const double* B0, double* C, double beta,
                     const ItemSet* is2, double* C2) {
      if (!h->econ) {
        gemmT(step, is, B0, C, beta);
        if (is2) gemmT(step, *is2, B0, C2, beta);
        return;
      }
      for (int c = 0; c * h->echunk < h->n_leaf; ++c) {
        recompute_leaf_chunk(h, c, s);
        const int l0 = c * h->echunk, n = std::min(h->echunk, h->n_leaf - l0);
        const ItemSet r = leaf_range(h, is, l0, n);
        TIMED(("gemmT_" + std::string(step) + "_f64").c_str(), 2.0 * r.elems * nrhs, r.elems * 8.0,
              launch_gemm_items<double, double>(r.dev, r.n, ROWBLK, 1, h->eops, B0, nullptr, C, nullptr, idx, nrhs,
                                                beta, s, gemm_ctx(h, r.maxK)));
        if (is2) {
          const ItemSet r2 = leaf_range(h, *is2, l0, n);
          TIMED(("gemmT_" + std::string(step) + "_f64").c_str(), 2.0 * r2.elems * nrhs, r2.elems * 8.0,
                launch_gemm_items<double, double>(r2.dev, r2.n, ROWBLK, 1, h->eops, B0, nullptr, C2, nullptr, idx,
                                                  nrhs, beta, s, gemm_ctx(h, r2.maxK)));
        }
      }
    };
    // 1. leaf-down transposed: gbar_ci = F^T ubar_ci ; LB = S_ci^T ubar_ci + Lce^T ubar_ce
    leafT("leaf_FS", h->adj_leafF, ubar_in, gb, 0.0, &h->adj_leafS, w.LB);
    gemmT("leaf_ext", h->adj_lce, ubar_in, w.LB, 1.0);
    // ubar_gauss = sum over owning leaves
    TIMED("gather_reduce", 0, 0, launch_gather_reduce<double>(h->leaf_reduce_tab, h->n_leaf_reduce, w.LB, ub, nrhs, 0, s));
    CKL();
    const int H = h->tree.height;
    // 2. merge-down transposed, bottom-up
    for (int L = 0; L < H; ++L) {
      Level& lv = h->levels[L];
      TIMED("gather_reduce", 0, 0, launch_gather_reduce<double>(lv.wcopy_tab, lv.n_wcopy, ub, VB, nrhs, 0, s));
      gemmTp("merge_S", lv.adjS, ub, w.UB, 0.0);
      TIMED("gather_reduce", 0, 0, launch_gather_reduce<double>(lv.reduce_tab, lv.n_reduce, w.UB, ub, nrhs, 1, s));
      if (lv.aidown.n) gemmT("refine_down", lv.aidown, ub, ub, 1.0);
    }
    // 3. boundary data
    if (fbar) TIMED("gather_reduce", 0, 0, launch_gather_reduce<double>(h->fbar_tab, h->n_bdry, ub, fbar, nrhs, 0, s));
    // 4. merge-up transposed, top-down
    for (int L = H - 1; L >= 0; --L) {
      Level& lv = h->levels[L];
      if (lv.aiup.n) gemmT("coarsen_up", lv.aiup, VB, VB, 0.0);
      gemmTp("merge_X", lv.adjM, VB, w.d64, 0.0);
      TIMED("down_scatter", 0, 0, launch_down_scatter<double>(lv.ds, (int)lv.boxes.size(), lv.ds_maxrows, VB, w.d64, nullptr, idx, nrhs, s));
    }
    // 5. leaf-up transposed: gbar_ci += H^T hbar
    leafT("leaf_H", h->adj_leafH, VB, gb, 1.0, nullptr, nullptr);
    CKL();
    // 6. coefficient gradients
    if (cbar) {
      const ResidualArgs ra = residual_args(h, nullptr);
      TIMED("coeff_grad_df", 2.0 * h->n_leaf * nrhs * (5.0 * h->p * h->p * h->p + 12.0 * h->m), nuc * 16.0,
            launch_coeff_grad(ra, u, gb, cbar, nrhs, s));
      CKL();
    }
    for (void* p : tmp) h->al.put(p, s);
    (void)ng;
    return HPS_OK;
  } catch (const CudaError& e) {
    for (void* p : tmp) h->al.put(p, s);
    return fail(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    for (void* p : tmp) h->al.put(p, s);
    return fail(HPS_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    for (void* p : tmp) h->al.put(p, s);
    return fail(HPS_ERR_INVALID_ARG, e.what());
  }
}

int hps_handle_info(const hps_handle* h, int* n_leaves, int* p, int* q, int* n_gauss, int* n_boundary,
                    int64_t* operator_bytes) {
  if (!h) return fail(HPS_ERR_INVALID_ARG, "handle is NULL");
  if (n_leaves) *n_leaves = h->n_leaf;
  if (p) *p = h->p;
  if (q) *q = h->q;
  if (n_gauss) *n_gauss = h->ns.n_gauss;
  if (n_boundary) *n_boundary = h->n_bdry;
  if (operator_bytes)
    *operator_bytes = (int64_t)h->ops_elems * (h->opts.precision == HPS_MIXED ? 4 : 8);
  return HPS_OK;
}

int hps_sync_status(hps_handle* h, void* stream) {
  if (!h) return fail(HPS_ERR_INVALID_ARG, "handle is NULL");
  int status = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(HPS_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  if (status < 0) return fail(HPS_ERR_TIMEOUT, "a tensor-core update did not complete within its wait limit");
  if (status) return fail(HPS_ERR_SINGULAR, "pivot breakdown in box " + std::to_string(status - 1));
  return HPS_OK;
}

int hps_destroy(hps_handle* h) {
  if (!h) return HPS_OK;
  delete h;
  return HPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Solve without device allocation.
//
// hps_solve keeps its per-call work buffers (the per-box flux/particular-solution pool,
// the merge difference vectors and the Gaussian-node solution vector) in the handle and
// allocates them on the first call for a given nrhs.  Some callers cannot let a solve
// allocate: a host framework that has already reserved nearly all device memory for its
// own pool, or a time-stepping loop that must not pay for (or risk failing) an allocation
// once it is running.  hps_solve_noalloc runs the same FP64 sweep kernels with those work
// buffers carved from one fixed array in device memory that is part of the library image
// (every GPU that loads the library holds it until the process exits).
//
// The array is shared by every call: calls whose work overlaps on the GPU (two streams,
// or two host threads) race on it and give wrong results; serialise them.  Each call
// clears what has to start at zero.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up (cudaGetSymbolAddress,
// with that device current) and caches it; make that first call before any stream capture.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[HPS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once per device).
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HPS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(HPS_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(HPS_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return HPS_OK;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

extern "C" int hps_solve_noalloc(hps_handle* h, const double* f, const double* g, int nrhs, double* u,
                                 void* stream) {
  if (!h) return fail(HPS_ERR_INVALID_ARG, "handle is NULL");
  if (!f || !g || !u) return fail(HPS_ERR_INVALID_ARG, "f, g and u must be device pointers");
  if (nrhs < 1) return fail(HPS_ERR_INVALID_ARG, "nrhs must be >= 1");
  if (h->opts.precision != HPS_FP64) return fail(HPS_ERR_STATE, "hps_solve_noalloc needs an HPS_FP64 handle");
  if (h->bc.on) return fail(HPS_ERR_STATE, "hps_solve_noalloc needs Dirichlet data on every side");
  const size_t R = (size_t)nrhs;
  const size_t bV = align256((size_t)h->v_rows * R * sizeof(double));
  const size_t bD = align256((size_t)std::max(1, h->d_rows) * R * sizeof(double));
  const size_t bG = align256((size_t)h->ns.n_gauss * R * sizeof(double));
  const size_t bP = align256((size_t)std::max(1, h->p_rows) * R * sizeof(double));
  // exponents of the tensor-core products (only when they can run: nrhs >= 8)
  const long long tc_units =
      (h->opts.fp64_gemm != HPS_GEMM_SIMT && nrhs >= 8) ? (long long)h->max_items * ((nrhs + 31) / 32) : 0;
  const size_t bS = align256((size_t)gemm_tc_scale_bytes(tc_units));
  const size_t need = bV + bD + bG + bP + bS;
  if (need > (size_t)HPS_NOALLOC_SCRATCH_BYTES)
    return fail(HPS_ERR_INVALID_ARG, "hps_solve_noalloc needs " + std::to_string(need) +
                                         " bytes of scratch for this tree and nrhs, more than the fixed " +
                                         std::to_string((size_t)HPS_NOALLOC_SCRATCH_BYTES) +
                                         " (use fewer right-hand sides per call, or hps_solve)");
  void* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != HPS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* b = (unsigned char*)base;
  double* V = (double*)b;
  double* d = (double*)(b + bV);
  double* ug = (double*)(b + bV + bD);
  double* Pp = (double*)(b + bV + bD + bG);
  int* sc = tc_units ? (int*)(b + bV + bD + bG + bP) : nullptr;
  // the handle's per-call state points at the scratch array for the duration of the call
  struct CallScope {
    hps_handle* h;
    int* sc0;
    long long u0;
    CallScope(hps_handle* hh, int* sc, long long units) : h(hh), sc0(hh->tc_scales), u0(hh->tc_units) {
      h->noalloc_call = true;
      h->tc_scales = sc;
      h->tc_units = units;
    }
    ~CallScope() {
      h->noalloc_call = false;
      h->tc_scales = sc0;
      h->tc_units = u0;
    }
  };
  try {
    if (tc_units) gemm_tc_prepare();
    CallScope scope(h, sc, tc_units);
    // the Gaussian-node vector is assembled by scatters, so it must start at zero; the
    // other buffers are fully written before they are read
    CK(cudaMemsetAsync(ug, 0, (size_t)h->ns.n_gauss * R * sizeof(double), s));
    solve_pass<double, double>(h, h->ops64, f, g, nullptr, u, ug, V, d, Pp, nrhs, s);
  } catch (const CudaError& e) {
    return fail(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(HPS_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(HPS_ERR_INVALID_ARG, e.what());
  }
  return HPS_OK;
}
