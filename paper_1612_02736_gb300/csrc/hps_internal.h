// Internal declarations of the GB300 HPS library: host tree, reference-element tables,
// per-level schedules and the kernel launchers.  Nothing here crosses the C ABI.
#pragma once

#include <array>
#include <cstdint>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hps.h"

namespace hps {

// ---------------------------------------------------------------------------------------
// Host tree (Sec. 2).  Boxes are numbered breadth-first from the root, so a parent has a
// smaller id than its children; the first child is the W (or S) half ("alpha").
struct Box {
  int i0 = 0, i1 = 0, j0 = 0, j1 = 0;  // span in finest-grid units
  double x0 = 0, y0 = 0, x1 = 0, y1 = 0;
  int leaf = -1;        // leaf index or -1
  int child[2] = {-1, -1};
  int parent = -1;
  int height = 0;       // 0 for leaves, 1 + max(child heights) for parents
  bool refined = false; // root of a 2 x 2 refinement of a former leaf (Sec. 6)
};

struct Tree {
  double ox = 0, oy = 0, ux = 1, uy = 1;  // origin and finest-grid unit
  std::vector<Box> boxes;
  std::vector<int> leaves;             // leaf index -> box id (ordered by lower-left corner)
  std::vector<int> leaf_edges;         // 4 per leaf (S, E, N, W): edge segment id
  int n_edges = 0;
  std::vector<int> edge_owners;        // 2 per edge: leaf*4+side of the owners, -1 if none
  std::vector<std::array<int, 4>> edge_keys;    // (orient 0=h/1=v, line, lo, hi)
  std::map<std::array<int, 4>, int> edge_of;    // key -> edge id
  int height = 0;
};

int make_uniform_tree(double x0, double y0, double x1, double y1, int nx, int ny, Tree& t);
int make_mask_tree(double x0, double y0, double h, int nx, int ny, const uint8_t* mask, Tree& t);
int refine_tree(const Tree& in, const double* pts, int npts, int levels, Tree& out);

// Coarsened sides of a refined parent (Sec. 6.3): dense interpolation operators.
struct Coarsen {
  bool active = false;
  std::vector<double> Pup;    // |ge_old| x |ge|  (fine <- coarse; identity on kept nodes)
  std::vector<double> Pdown;  // |ge| x |ge_old|  (coarse <- fine)
  std::vector<double> Pupc;   // |fine| x |coarse|: P_up rows of the fine nodes, coarse columns
  std::vector<int> fine;      // node ids replaced by the coarsening (in ge_old order)
  std::vector<int> coarse;    // coarse node ids (in ge order)
};

// Gaussian node bookkeeping for a given q: box exterior lists and merge index sets.
struct NodeSets {
  int q = 0;
  int n_gauss = 0;
  std::vector<std::vector<int>> ge;     // per box: exterior ids as seen by the parent (I_ge)
  std::vector<std::vector<int>> ge_old; // per parent: J1 ++ J2 (before coarsening)
  std::vector<std::vector<int>> J3;     // per parent: shared-edge node ids (alpha order)
  std::vector<int> n1;                  // per parent: |J1|
  std::vector<Coarsen> co;              // per box
  std::vector<int> boundary;            // domain-boundary node ids, ascending
};

void build_node_sets(const Tree& t, int q, NodeSets& ns, const std::vector<double>& xg);

// ---------------------------------------------------------------------------------------
// Reference-element tables for (p, q) on [-1, 1] (Sec. 3.1-3.4).
struct RefTables {
  int p = 0, q = 0, m = 0, ne = 0;     // m = (p-2)^2 interior, ne = 4(p-1) exterior
  std::vector<double> xc;              // p Chebyshev-Lobatto points, ascending
  std::vector<double> xg;              // q Gauss-Legendre points, ascending
  std::vector<double> D;               // p x p differentiation on xc
  std::vector<double> D2;              // p x p, D*D
  std::vector<double> Lg2c;            // p x q: Gauss data of one side -> its p Chebyshev points
  std::vector<double> Ls;              // p x q: Lg2c with corner rows halved (side block of L_ce,ge)
  std::vector<double> DLs;             // p x q: D * Ls (differentiation along a side, then Ls)
  std::vector<double> Lloc;            // q x p: Chebyshev -> Gauss on one side
  std::vector<double> DceL;            // 4q x 4q: D_ge,ce L_ce,ge on [-1,1]^2 (row s scaled later)
  std::vector<double> Lce;             // ne x 4q: L_ce,ge, rows = exterior nodes ascending
  std::vector<int> ci;                 // m interior node indices, ascending
  std::vector<int> ce;                 // ne exterior node indices, ascending
};

void build_ref_tables(int p, int q, RefTables& rt);

// ---------------------------------------------------------------------------------------
// Kernel-side parameter blocks.

// One matrix of a batched partial Gauss-Jordan elimination: an R x R row-major matrix at
// element offset off of the workspace, pivoting on its first K diagonal entries.
struct GJDesc {
  long long off;
  int R;
  int K;
  int rows;            // rows formed and eliminated: R, or K at the root, where only the
                       // top block rows [X | S] are wanted (row stride stays R)
  int perm_off;        // offset of its K-entry logical->physical row map
  int box;             // box id, for error reports
  float null_tol = 0.f;  // > 0: a pivot below null_tol x (*null_scale, the matrix's largest
                         // entry) is a null direction of a consistent singular system: its
                         // unknown is set to zero and its equation dropped, not reported
  const double* null_scale = nullptr;
};

// A gathered, batched matrix product item: rows [0, M) of a row block of operator A.
//   C[cidx[i]][r] = beta * C[cidx[i]][r] + sum_k A[i][k] * B(k)[r]  (+ Add[i][r])
// with B(k) = B0[b0idx[k]] for k < kseg and B1[b1idx[k - kseg]] otherwise.  Row indices
// are in units of vector rows (each row holds nrhs values).  An idx offset of -1 means
// the identity map.  trans = 1 applies A^T (A stored row-major K x M with leading
// dimension lda).
struct GemmItem {
  long long a_off;     // element offset of the block's first row (or column when trans)
  int lda;
  int M, K, kseg;
  int b0_row, b0_idx;
  int b1_row, b1_idx;
  int c_row, c_idx;
  int add_row;         // -1: no addend
};

// ---------------------------------------------------------------------------------------
// Launchers (defined in the .cu files).  All take the stream explicitly.

// Leaf matrices M = [[A_ci,ci, A_ci,ce L_ce,ge], [D_ge,ci, D_ge,ce L_ce,ge]] (size m+4q)
// for leaves [leaf0, leaf0 + nleaf) of coeffs [6][n_leaf_total][p*p].
struct LeafTablesDev {
  const double* D;      // p x p
  const double* D2;     // p x p
  const double* Ls;     // p x q
  const double* DLs;    // p x q: D Ls
  const double* Lloc;   // q x p
  const double* DceL;   // 4q x 4q
  const int* ci;        // m
};
// out[0] = smallest leaf index with a non-finite interior coefficient, out[1] = smallest leaf
// index whose principal part is not elliptic at an interior node (out preset by the caller).
void launch_coeff_check(const double* coeffs, int n_leaf, int p, int* out, cudaStream_t s);
// *flag = 1 when the interior coefficients of some leaf differ from leaf 0's.
void launch_leaf_uniform_check(const double* coeffs, int n_leaf, int p, int* flag, cudaStream_t s);
template <typename T>
void launch_leaf_assemble(const double* coeffs, long long n_leaf_total, int leaf0, int nleaf,
                          const double* hxy, int p, int q, const LeafTablesDev& tb, T* work,
                          long long mat_stride, cudaStream_t s);

template <typename T>
void launch_gj_init(const GJDesc* d, int nmat, int* perm, cudaStream_t s);
// Zeroes rows K .. R - 1, columns 0 .. K - 1 of each FP64 matrix (at most max_entries each).
void launch_gj_zero_bl(const GJDesc* d, int nmat, long long max_entries, double* work, cudaStream_t s);
template <typename T>
void launch_gj_panel(const GJDesc* d, int nmat, int maxK, T* work, int* perm, T* pinv, int c0,
                     int nb, int* status, cudaStream_t s);
template <typename T>
void launch_gj_prep(const GJDesc* d, int nmat, int maxR, T* work, const int* perm, const T* pinv,
                    T* prow, long long prow_stride, int c0, int nb, cudaStream_t s);
template <typename T>
// tensor (FP64 only): 1 the persistent tcgen05 kernel with exact digit slicing, 2 its
// streamed form (needs 16-byte aligned rows: even R and offsets, aligned work), 0 the FP64 /
// FP32 register-tiled SIMT kernel.  mat_stride > 0 states that every matrix has R = maxR,
// rows = maxRows and sits at work + m * mat_stride (the streamed form then copies tiles with
// a tensor map); 0 makes no such claim.
void launch_gj_update(const GJDesc* d, int nmat, int maxR, int maxRows, T* work, const int* perm, T* prow,
                      long long prow_stride, int c0, int nb, cudaStream_t s, int* status, int tensor,
                      long long mat_stride = 0);

// Extraction of a finished elimination: with sigma the logical->physical row map,
//   TL[i][j] = sTL * M[sigma(i)][sigma^-1(j)]   (i, j < K)
//   TR[i][c] = sTR * M[sigma(i)][K + c]
//   BL[r][j] = sBL * M[K + r][sigma^-1(j)]
//   BR[r][c] =       M[K + r][K + c]
// Destinations are per matrix: base + b * stride with the given leading dimensions.
struct ExtractDst {
  void* TL; long long TL_off_stride; int TL_ld;   // TL, TR, BL: element type given by the launcher
  void* TR; long long TR_off_stride; int TR_ld;
  void* BL; long long BL_off_stride; int BL_ld;
  void* BR; long long BR_off_stride; int BR_ld;   // FP64
  double sTL, sTR, sBL;  // +1 or -1
  const long long* TL_off;   // optional per-matrix offsets (override b * stride) or null
  const long long* TR_off;
  const long long* BL_off;
  const long long* BR_off;
  int ld_from_desc;          // 1: TL_ld = BL_ld = K and TR_ld = BR_ld = R - K per matrix
};
template <typename T, typename TO>
void launch_gj_extract(const GJDesc* d, int nmat, int maxR, const T* work, const int* perm,
                       const ExtractDst& dst, cudaStream_t s);

// Merge assembly (Sec. 4): M_tau = [[Z, R], [-C, blkdiag(T11a, T22b)]] with rows/columns
// ordered [J3 | J1 | J2], gathered from the children's T blocks.
struct MergeDesc {
  long long m_off;     // offset of M_tau in the workspace
  int R;               // k3 + k12
  int rows;            // rows to assemble (R, or k3 at the root)
  int k3, n1;          // |J3|, |J1| (|J2| = R - k3 - n1)
  long long ta_off, tb_off;  // children's T in the T store
  int lda_a, lda_b;    // children's T sizes
  int pos_off;         // offset of pos arrays: posA[R], posB[R] (position in child ge or -1)
};
template <typename T, typename TT>
void launch_merge_assemble(const MergeDesc* d, int nmat, int maxR, const TT* tstore,
                           const int* pos, T* work, cudaStream_t s);

// One root-condition matrix (rows x R, row-major) assembled from a DtN map src (ld):
// row r takes up to two (index, sign) pairs from idx[rt + 4r ..], column c from
// idx[ct + 4c ..]; flip negates the blocks off the K x K diagonal partition.
struct CombAsm {
  int ld, R, rows, K, flip, rt, ct;
};
void launch_comb_assemble(const CombAsm& a, const double* src, const int* idx, double* dst, cudaStream_t s);

// Small batched dense products C = A B (row-major, per-matrix offsets from three bases),
// used for the coarsened DtN maps T_new = P_down T P_up of refined parents.
struct BGemm {
  long long a_off, b_off, c_off;
  int M, N, K, lda, ldb, ldc;
};
void launch_bgemm(const BGemm* d, int n, int maxM, int maxN, const double* A, const double* B, double* C,
                  cudaStream_t s);

// The operator digit planes of an item set, formed once (launch_gemm_tc_digitize): item i's
// K steps at dig + step[i] * gemm_tc_digit_bytes(1), its 64 row exponents at er + 64 i.
// Optionally (FP64 products, with the operator digits) the vectors' digit planes too,
// formed once for groups of items that gather the same vector rows over the same K
// (launch_gemm_tc_bdigitize): for item i, column block nb (32 columns) and K step c at
// bdig + (bblk[i] + nb ceil(K / 16) + c) * gemm_tc_bdigit_bytes(1), the column exponents
// of column n at bex[bexo[i] + n]; the product kernel then forms no digits at all.
struct GemmDigits {
  const unsigned char* dig = nullptr;
  const long long* step = nullptr;
  const int* er = nullptr;
  const unsigned char* bdig = nullptr;
  const long long* bblk = nullptr;
  const int* bexo = nullptr;
  const int* bex = nullptr;
};
// A group of items sharing their gathered vectors: rows b0_row + idx[b0_idx + k],
// k < K (first segment only), its digit blocks from blk0 and exponents from ex0.
struct BGroup {
  int b0_row, b0_idx, K;
  int ex0;
  long long blk0;
};

// Options of one batched product launch.
//   bn        right-hand-side tile of the SIMT tiled product (16, 32 or 64; 0 = fixed rule)
//   maxK      > 0 states the largest inner dimension of the items: FP64 products with
//             maxK <= 448 and nrhs >= 8 then run on the tensor cores (launch_gemm_tc) when
//             the exponent buffer below is large enough, else on the SIMT kernels
//   status    receives -1 if a tensor-core wait times out
//   dg        optional operator digits of the items
//   tc_scales the tensor-core product's per-unit exponent buffer (gemm_tc_scale_bytes(units)
//             bytes, owned by the caller) and its capacity in units
//   tc32      FP32 non-transposed products with nrhs > 8 run on the tensor cores
struct GemmCtx {
  int bn = 0;
  int maxK = 0;
  int* status = nullptr;
  const GemmDigits* dg = nullptr;
  int* tc_scales = nullptr;
  long long tc_units = 0;
  bool tc32 = false;   // FP32 products may run on the tensor cores (launch_gemm_tc32)
  int maxKv = 0;       // largest inner dimension of the items, when known (0: unknown);
                       // small ones select the warp-per-item streaming product
};

template <typename TA, typename TV>
void launch_gemm_items(const GemmItem* items, int nitems, int maxM, int trans, const TA* A,
                       const TV* B0, const TV* B1, TV* C, const TV* Add, const int* idx,
                       int nrhs, double beta, cudaStream_t s, const GemmCtx& cx);

// FP64 gathered products on the tcgen05 tensor cores by exact digit slicing (k_gemm_tc.cu):
// items of at most 64 rows and K <= 448.  A launch needs units = items x ceil(nrhs / 32)
// entries of the exponent buffer cx.tc_scales; launch_gemm_tc returns false, launching
// nothing, when it is missing or too small.  With cx.dg the operator's digits are read from
// it instead of being formed (same results).  gemm_tc_prepare does the per-device set-up
// (call it outside stream capture; launches do it themselves otherwise).
bool gemm_tc_eligible(int maxK, int nrhs);
long long gemm_tc_scale_bytes(long long units);
void gemm_tc_prepare();
bool launch_gemm_tc(const GemmItem* items, int nitems, int trans, const double* A, const double* B0,
                    const double* B1, double* C, const double* Add, const int* idx, int nrhs, double beta,
                    cudaStream_t s, const GemmCtx& cx);
// FP32 gathered products on the tcgen05 tensor cores (k_gemm_tc32.cu): each entry split into
// three bf16 pieces, the six piece pairs of weight >= 2^-16 summed in FP32 accumulators
// (the accuracy of an FP32 product); items of at most 64 rows, non-transposed, nrhs > 8.
// Returns false, launching nothing, if the device set-up failed.
// With dg, the operator's bf16 pieces are read from it (launch_gemm_tc32_pieces, same
// results).
// Bounded-wait self-test kernel (out_dev: 2 ints, zeroed by the caller); 0 or -1 (launch error).
int wait_selftest(int polls, int* out_dev, cudaStream_t s);
bool gemm_tc32_eligible(int nrhs);
void gemm_tc32_prepare();
bool launch_gemm_tc32(const GemmItem* items, int nitems, const float* A, const float* B0, const float* B1, float* C,
                      const float* Add, const int* idx, int nrhs, double beta, int* status, cudaStream_t s,
                      const GemmDigits* dg);
// bytes of the bf16 operator pieces of `steps` K steps; fill adig for the items (astep: each
// item's first step)
long long gemm_tc32_piece_bytes(long long steps);
void launch_gemm_tc32_pieces(const GemmItem* items, int nitems, const float* A, const long long* astep,
                             unsigned char* adig, cudaStream_t s);
// bytes of the digit planes of `steps` K steps; fill adig / aer for the items (astep: each
// item's first step, prefix sums of ceil(K / 16))
long long gemm_tc_digit_bytes(long long steps);
long long gemm_tc_bdigit_bytes(long long blocks);
// The vectors' digit planes and column exponents of ngroups groups (ncb column blocks of 32
// each, nrhs columns of B0 with rows b0_row + idx[b0_idx + k]).
void launch_gemm_tc_bdigitize(const BGroup* groups, int ngroups, int ncb, const double* B0, const int* idx, int nrhs,
                              unsigned char* bdig, int* bex, cudaStream_t s);
void launch_gemm_tc_digitize(const GemmItem* items, int nitems, int trans, const double* A, const long long* astep,
                             unsigned char* adig, int* aer, cudaStream_t s, bool negate = false);

// Split-K partial products: rows [0, M) of one output block were computed in nsplit K
// ranges into the partial buffer P (rows p_row + j * M + i); the reduction writes
//   C[map(i)][r] = beta * C[map(i)][r] + sum_j P[p_row + j * M + i][r] (+ Add[add_row + i][r]).
struct SplitRed {
  int M, nsplit, p_row;
  int c_row, c_idx, add_row;
};
template <typename TV>
void launch_split_reduce(const SplitRed* d, int n, const TV* P, TV* C, const TV* Add, const int* idx,
                         int nrhs, double beta, cudaStream_t s);

// Up-sweep gather for a level of merges: d = h_b[pos3b] - h_a[pos3a] (+ rho[J3]) and
// prefill V_tau = [0 (k3 rows) ; h_a[pos1a] ; h_b[pos2b]].
struct UpGather {
  int va_row, vb_row;  // row base of child h within V (child V base + child k3)
  int vt_row;          // row base of V_tau
  int d_row;           // row base of d for this merge in the d buffer
  int k3, n1, n2;
  int idx_off;         // pos3a[k3], pos3b[k3], J3[k3], pos1a[n1], pos2b[n2]
};
template <typename TV>
void launch_up_gather(const UpGather* g, int n, int maxrows, const TV* V, TV* Vout, TV* dbuf,
                      const double* rho, const int* idx, int nrhs, cudaStream_t s);

// Scatter f into u at the boundary nodes and copy/convert vectors.
template <typename TV>
void launch_scatter_rows(const double* src, const int* idx, int n, TV* dst, int nrhs,
                         cudaStream_t s);
template <typename TI, typename TO>
void launch_convert(const TI* src, TO* dst, long long n, double scale, cudaStream_t s);
template <typename TI>
void launch_axpy_to_f64(const TI* x, double* y, long long n, cudaStream_t s);
// y += x (x FP32), and max |x| into out[0], max |y| (after the update) into out[1] (atomic
// maxima on the bit patterns of non-negative doubles; out preset to 0 by the caller).
void launch_axpy_measure(const float* x, double* y, long long n, double* out, cudaStream_t s);

// FP64 residual of the collocation system and leaf fluxes (mixed-precision refinement).
struct ResidualArgs {
  const double* coeffs; long long n_leaf; int p, q;
  const double* hxy;
  const double* D; const double* D2; const double* Lloc;
  const int* ci;
  // the same tables as unevaluated float pairs (hi, lo) for the double-float kernels
  const float2* Lloc_df;
  const float2* D_df; const float2* D2_df;
  // L_ce,ge by rows of exterior nodes k, only the edge blocks (q columns each) that hold the
  // row's nonzeros (the others are exactly zero): Lce_blk [ne][4] their indices (-1 padded),
  // Lce_off [ne + 1] the start of row k's stored blocks in Lce_c (double-float pairs)
  const float2* Lce_c;
  const int* Lce_blk;
  const int* Lce_off;
  int n_lce;  // entries of Lce_c
};
// Residual r = g - A u, leaf fluxes and u_ce = L_ce,ge u_ge, in double-float arithmetic.
void launch_leaf_residual_df(const ResidualArgs& a, const int* leaf_edges, const int* ce, const double* ug, const double* g, double* uc,
                             float* r_out, double* vflux, int nrhs, cudaStream_t s);  // r in FP32
// y = alpha u + beta A u at leaf interior nodes, 0 at exterior nodes, double-float.
void launch_leaf_apply_df(const ResidualArgs& a, const double* u, double alpha, double beta, double* out, int nrhs,
                          cudaStream_t s);
void launch_jump_residual(const int* pairs, int npairs, int q, const double* vflux,
                          double* rho_out, int nrhs, cudaStream_t s);
void launch_absmax(const double* x, long long n, double* out, cudaStream_t s);
void launch_fill(double* x, long long n, double v, cudaStream_t s);  // x[0..n) = v
void launch_absmax_f32(const float* x, long long n, double* out, cudaStream_t s);  // max |x| as a double
// Raises a kernel's dynamic shared-memory limit on the current device to at least `bytes`
// (set once per kernel, device and size, whatever the size; thread-safe).
void ensure_smem(const void* kernel, size_t bytes);
// SM count of the current device.
int device_sms();
// Row combinations dst[d] = A[a] (+ sign * B[b] if b >= 0), entries (d, a, b, sign) at tab,
// rows of nrhs values.
void launch_row_combine(const int* tab, int n, double* dst, const double* A, const double* B, int nrhs,
                        cudaStream_t s);

// Adjoint helpers.
void launch_coeff_grad(const ResidualArgs& a, const double* uc, const double* gbar,
                       double* grad, int nrhs, cudaStream_t s);
template <typename TV>
void launch_gather_reduce(const int* tab, int nnodes, const TV* src, TV* dst, int nrhs,
                          int accumulate, cudaStream_t s);
struct DownScatter {  // adjoint of the up gather: distribute hbar_tau and dbar to children
  int va_row, vb_row, vt_row, d_row, k3, n1, n2, idx_off;
};
template <typename TV>
void launch_down_scatter(const DownScatter* g, int n, int maxrows, TV* VB, const TV* dbar,
                         double* rhobar, const int* idx, int nrhs, cudaStream_t s);

// Error thrown inside the library and turned into a status code at the C boundary.
struct CudaError {
  int code;
  std::string msg;
};

// Tile autotuner: tuned_choice returns the stored choice for key, or runs trial_ms for
// every candidate (each returns the measured milliseconds of one run), keeps the fastest
// in process memory and appends it to the cache file at path (empty: none).  With an
// empty trial_ms it only looks up, and returns 0 for a shape not tuned yet.
// time_on_stream runs a callable between two CUDA events on s and synchronises.
int tuned_choice(const std::string& key, const std::vector<int>& cands, const std::string& path,
                 const std::function<float(int)>& trial_ms);
float time_on_stream(cudaStream_t s, const std::function<void()>& run);

// Optional launch timing (enabled with hps_timing_enable): records a pair of CUDA events
// around the launches made while the scope is alive.
bool timing_enabled();
void timing_suspend(bool on);  // no event records while a stream is being captured
class TimingScope {
 public:
  TimingScope(const char* name, cudaStream_t s, double flops = 0.0, double bytes = 0.0, int launches = 1);
  ~TimingScope();
  TimingScope(const TimingScope&) = delete;
  TimingScope& operator=(const TimingScope&) = delete;

 private:
  cudaStream_t stream_;
  double flops_, bytes_;
  int launches_ = 1;
  int cat_ = -1;
  void* e0_ = nullptr;
  void* e1_ = nullptr;
};

}  // namespace hps
