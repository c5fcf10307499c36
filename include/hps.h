/*
 * hps.h -- C ABI of the GB300 (sm_103a) hierarchical Poincare-Steklov direct solver for
 * variable-coefficient 2D elliptic problems with body loads.
 *
 * Problem (Sec. 1, Eqs. basic and defA):
 *     A u = g in Omega,  u = f on the boundary of Omega,
 *     A u = -c11 u_xx - 2 c12 u_xy - c22 u_yy + c1 u_x + c2 u_y + c u.
 * Omega is a rectangle split into a binary tree of boxes (Sec. 2).  Each leaf carries a
 * p x p Chebyshev-Lobatto grid (Sec. 3.1) and q Gauss-Legendre nodes per side (Sec. 2).
 *
 * Conventions shared by every call:
 *  - Leaves are numbered by their lower-left corner, y first, then x (j * nx + i on a
 *    uniform grid).  Leaf Chebyshev nodes are numbered iy * p + ix (x fastest),
 *    ascending coordinates.
 *  - Gaussian nodes get global ids edge segment by segment, visiting leaves in leaf order
 *    and their sides in the order S, E, N, W; the q ids of one segment ascend along it; a
 *    segment two leaves share exactly has one set of ids.  "Boundary order" lists the
 *    domain-boundary Gaussian nodes in ascending global id.
 *  - Fluxes are d/dx on vertical and d/dy on horizontal edges (Sec. 3.1).
 *  - Multi-RHS arrays put the right-hand-side index fastest: [row][rhs].
 *  - All floating-point inputs and outputs are FP64.  Device pointers are plain CUDA
 *    device addresses; "stream" is a cudaStream_t passed as void* (NULL = legacy stream).
 *  - Every call returns an hps_status.  Nothing aborts, traps or exits the process; the
 *    text of the last error of the calling thread is returned by hps_last_error().
 *  - Calls taking a stream are stream-ordered.  hps_solve and hps_adjoint return once
 *    their work is enqueued (the iterative refinement of HPS_MIXED synchronises the
 *    stream to test convergence: once per call once calibrated, once per refinement
 *    step before, see hps_solve).  Calls on one handle share its workspace and graphs:
 *    their work must not overlap on the GPU (one stream, or streams synchronised between
 *    the calls).  Errors found by device
 *    code (singular pivots) are reported by hps_build (which synchronises) and by
 *    hps_sync_status.
 */
#ifndef HPS_GB300_H
#define HPS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HPS_OK = 0,
  HPS_ERR_INVALID_ARG = 1,   /* bad pointer, size, tree or option                      */
  HPS_ERR_NOT_ELLIPTIC = 2,  /* c11 <= 0 or c11 c22 - c12^2 <= 0 at an interior node     */
  HPS_ERR_SINGULAR = 3,      /* a leaf or merge pivot fell below tiny * scale            */
  HPS_ERR_OOM = 4,           /* the allocator returned NULL                              */
  HPS_ERR_CUDA = 5,          /* a CUDA runtime call failed (message has the CUDA text)   */
  HPS_ERR_TIMEOUT = 6,       /* a bounded device wait (tensor-core product) ran out      */
  HPS_ERR_NO_CONVERGENCE = 7,/* iterative refinement hit ir_max_iter                     */
  HPS_ERR_STATE = 8          /* call not valid for this handle (e.g. precision)          */
} hps_status;

typedef enum { HPS_FP64 = 0, HPS_MIXED = 1 } hps_precision;

typedef enum {
  HPS_NODES_CHEB_LEAF = 0,      /* n_leaf * p * p points, leaf-major                     */
  HPS_NODES_GAUSS_BOUNDARY = 1, /* domain-boundary Gaussian nodes in boundary order      */
  HPS_NODES_GAUSS_ALL = 2       /* every Gaussian node, by global id                     */
} hps_node_set;

/* Arithmetic of the FP64 solve and adjoint products (hps_opts.fp64_gemm). */
typedef enum {
  HPS_GEMM_TENSOR = 0, /* tcgen05 tensor cores by exact digit slicing (9 base-128 digits per
                        * entry, scaled per operator row and per vector column, exact FP32
                        * digit sums, one rounding to FP64) where a product's inner
                        * dimension is at most 448 and nrhs >= 8; SIMT FP64 elsewhere      */
  HPS_GEMM_SIMT = 1    /* SIMT FP64 for every product                                     */
} hps_gemm;

/* Boundary condition kinds of a rectangular domain's sides (hps_opts.bc_we, bc_sn). */
typedef enum {
  HPS_BC_DIRICHLET = 0, /* u given (both pairs of sides)                                  */
  HPS_BC_PERIODIC = 1,  /* west/east only: u and its x-flux equal at facing nodes        */
  HPS_BC_NEUMANN = 2    /* south/north only: the y-flux du/dy given                       */
} hps_bc;

typedef struct hps_tree hps_tree;     /* opaque, host memory                              */
typedef struct hps_handle hps_handle; /* opaque, owns the device operator store          */

/* Device memory allocator.  alloc returns a device pointer or NULL; free releases it.
 * Both receive the stream the call runs on.  A NULL allocator means cudaMallocAsync /
 * cudaFreeAsync on that stream. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx, void* stream);
  void (*free)(void* ptr, void* ctx, void* stream);
  void* ctx;
} hps_allocator;

typedef struct {
  int precision;       /* HPS_FP64 or HPS_MIXED                                           */
  int q;               /* Gauss nodes per leaf side; 0 means p - 1 (Sec. 7)                */
  int store_leaf_ops;  /* 1: keep leaf F, S, H (Sec. 5.2); 0: keep only the coefficients and
                        * rebuild F, S, H chunk by chunk whenever a solve or adjoint needs
                        * them (the storage-efficient variant of the Sec. 5.4 remark;
                        * HPS_FP64 only)                                                    */
  double ir_tol;       /* HPS_MIXED: bound on the estimated remaining error relative to
                        * max|u| (see hps_solve); 0 means 1e-8                          */
  int ir_max_iter;     /* HPS_MIXED: refinement steps allowed; 0 means 10                  */
  int fp64_top_levels; /* HPS_MIXED: number of top merge levels eliminated in FP64 (their
                        * operators are stored in FP32 like the rest); -1 means 5         */
  int use_graphs;      /* HPS_FP64 solves without a flux-jump input: 1 (default) replays
                        * one captured CUDA graph of the whole sweep per nrhs (the inputs
                        * are copied into and the result out of staging buffers the
                        * handle owns); 0 launches the kernels one by one              */
  int autotune;        /* 1: the first time a launch shape is met, time each candidate tile
                        * configuration once (the elimination panel width of a batch of
                        * leaves or merges; the right-hand-side tile of a solve product) and
                        * keep the fastest for the rest of the process; 0 (default): fixed
                        * rules.  Candidates of one product give bit-identical results;
                        * panel widths change the rounding of the build within the stated
                        * tolerances.  Tuning runs synchronise the stream                 */
  const char* autotune_cache; /* with autotune: a text file of earlier choices, read once
                        * and appended to (one "key value" line per shape); NULL keeps the
                        * choices in process memory only.  The library copies the path    */
  int shared_leaf;     /* leaf operators shared by every leaf (the constant-coefficient remark
                        * of Sec. 7.1): -1 (default) shares them when every leaf has the same
                        * size and the same coefficient values at its interior nodes (checked
                        * on the device at build time, one synchronisation); 0 never; 1
                        * requires it (INVALID_ARG when the leaves differ).  Shared, one
                        * leaf is eliminated and stored, and store_leaf_ops is ignored     */
  int bc_we;           /* west/east sides: HPS_BC_DIRICHLET (default) or HPS_BC_PERIODIC   */
  int bc_sn;           /* south/north sides: HPS_BC_DIRICHLET (default) or HPS_BC_NEUMANN.
                        * Other than Dirichlet (the channel problem of Sec. 7.6): the
                        * domain must be a rectangle (hps_tree_uniform, refined or not, with
                        * matching west/east nodes when periodic); the root keeps its DtN
                        * map and the solve obtains the boundary values from it; HPS_FP64
                        * handles only; hps_adjoint and hps_solve_noalloc return STATE     */
  int fp64_gemm;       /* FP64 solve and adjoint products: HPS_GEMM_TENSOR (default) or
                        * HPS_GEMM_SIMT.  The two agree to FP64 rounding, not bit for bit   */
  int fp32_gemm;       /* FP32 sweep products of HPS_MIXED solves with more than 8 right-hand
                        * sides: HPS_GEMM_TENSOR (default: tcgen05 tensor cores, every entry
                        * split into three bf16 pieces, the six piece pairs of weight >= 2^-16
                        * summed in FP32) or HPS_GEMM_SIMT (FP32 FFMA).  Both are FP32-accurate
                        * products; the refined solution meets the same tolerance            */
} hps_opts;

/* Fills *opts with the defaults above (FP64, q = p - 1, store leaf operators, graphs on,
 * no autotuning, leaf operators shared when the leaves allow it). */
void hps_opts_default(hps_opts* opts);

/* Uniform tree of nx x ny equal leaves over [x0,x1] x [y0,y1] by recursive halving
 * (Sec. 2): a box is cut across its longer side in leaves, vertically on ties; the W
 * (or S) half is the first child.  *out receives a new tree (free with
 * hps_tree_destroy).  INVALID_ARG if nx, ny < 1, x1 <= x0, y1 <= y0 or out is NULL. */
int hps_tree_uniform(double x0, double y0, double x1, double y1, int nx, int ny, hps_tree** out);
int hps_tree_destroy(hps_tree* tree);

/* Union of squares (Sec. 1: domains that are unions of rectangles): the squares
 * [x0 + i h, x0 + (i+1) h] x [y0 + j h, y0 + (j+1) h] with mask[j * nx + i] != 0 are the
 * leaves.  The tree bisects the nx x ny grid as hps_tree_uniform does and skips empty
 * halves, so e.g. the L-shaped domain is glued from its squares by the top merges.
 * INVALID_ARG if the mask selects nothing. */
int hps_tree_mask(double x0, double y0, double h, int nx, int ny, const uint8_t* mask, hps_tree** out);

/* Local refinement (Sec. 6.1): returns a new tree in which, `levels` times over, every leaf
 * whose distance d to one of the npts points (pts_xy = x0, y0, x1, y1, ...) satisfies
 * d <= sqrt(2) l (leaf side 2 l) is split into 2 x 2 leaves (a vertical cut, then
 * horizontal cuts).  After such a refined parent is merged, each of its sides that faces a
 * leaf of its own size is re-expressed on that leaf's nodes with the interpolation
 * operators of Sec. 6.3 (P_up: fine <- coarse, one polynomial through the coarse Gauss
 * nodes; P_down: coarse <- fine, from the fine segment holding each coarse node, averaged
 * when a node sits on the junction of two segments).  The input tree is unchanged.
 * Refined trees support HPS_FP64 only; hps_build rejects meshes whose interfaces the rule
 * leaves unmatched. */
int hps_tree_refine(const hps_tree* tree, const double* pts_xy, int npts, int levels, hps_tree** out);

/* Counts: leaves, boxes, tree height (merge levels), and for a given q the number of
 * Gaussian nodes (all, and on the domain boundary). */
int hps_tree_info(const hps_tree* tree, int q, int* n_leaves, int* n_boxes, int* n_levels,
                  int* n_gauss, int* n_boundary);

/* Coordinates of a node set (host memory): xy_host receives 2 * count doubles
 * (x0, y0, x1, y1, ...).  If xy_host is NULL only *count is written. */
int hps_nodes(const hps_tree* tree, int p, int q, int which, double* xy_host, int64_t* count);

/* Host-only dry run of hps_build's planning for this tree, p and options: builds the
 * index tables and every kernel descriptor of the build, solve and adjoint, and checks
 * each against the size of the buffer it addresses.  Touches no GPU.  OK, or
 * INVALID_ARG with the failed check in the message (unsupported tree shapes included). */
int hps_plan_check(const hps_tree* tree, int p, const hps_opts* opts);

/* Build stage (Algorithm 1).  coeffs_dev: device FP64 [6][n_leaf][p*p] holding c11, c12,
 * c22, c1, c2, c at every leaf Chebyshev node (exterior values are unused).  The leaf
 * step forms A on each leaf, factors A_ci,ci and writes F, S, H, T (Sec. 3, Eqs.
 * alpine1-alpine4); each merge forms X, S, T from the children (Sec. 4).  p in [4, 32].
 * The library does not keep coeffs_dev.  opts and alloc may be NULL (defaults).  The
 * coefficients are checked first at every interior node: INVALID_ARG if one is not finite,
 * NOT_ELLIPTIC if c11 <= 0 or c11 c22 - c12^2 <= 0 (the leaf index is in the message).  The
 * call synchronises the stream before it returns and reports SINGULAR with the box id
 * in the message if a pivot broke down; an allocation failure gives OOM with everything
 * allocated so far released.  An HPS_MIXED build ends with one
 * refined solve of a model problem (no load, boundary data 1 + x + 2 y, one right-hand side)
 * that measures the contraction bound rho of the refinement (see hps_solve); a failure
 * there leaves the handle without it and is not reported.  *out receives the handle. */
int hps_build(const hps_tree* tree, const double* coeffs_dev, int p, const hps_opts* opts,
              const hps_allocator* alloc, void* stream, hps_handle** out);

/* Solve stage (Algorithm 2) for nrhs right-hand sides at once.
 *   f_dev : [n_boundary][nrhs]        Dirichlet data at the boundary Gaussian nodes; with
 *                                     HPS_BC_NEUMANN, du/dy at the south and north nodes;
 *                                     ignored at periodic west/east nodes
 *   g_dev : [n_leaf][p*p][nrhs]       body load at the leaf Chebyshev nodes (interior
 *                                     values used)
 *   u_dev : [n_leaf][p*p][nrhs]       output: the solution at every leaf Chebyshev node
 * FP64 handles run the sweeps in FP64.  HPS_MIXED handles run them in FP32 and refine
 * against the residual of the collocation system (leaf equations and flux jumps, in
 * double-float arithmetic) with FP64 accumulation.  Until a handle is calibrated the
 * refinement is adaptive, synchronising after every correction du: it stops when
 * max|du| <= ir_tol max|u|, when a contraction bound rho is known (measured by the build)
 * and rho max|du| <= ir_tol max|u|, or when the observed contraction of two successive
 * corrections (ratio r < 1/2) predicts the remaining error 2 r max|du| below ir_tol max|u|.
 * Those ratios raise rho to twice the largest ratio; with rho and the first correction
 * the solve calibrates the number n of corrections that bring the initial solve's error
 * below ir_tol; later calls without flux-jump
 * data run the initial solve and n corrections without a test in between (one CUDA graph
 * from the second such call with the same nrhs when use_graphs is set), synchronise once
 * and accept when rho max|du_n| <= ir_tol max|u|, else refine on adaptively.  NaN or
 * ir_max_iter steps without convergence give NO_CONVERGENCE. */
int hps_solve(hps_handle* h, const double* f_dev, const double* g_dev, int nrhs, double* u_dev,
              void* stream);

/* Operator application on the handle's leaves: out = alpha u + beta A u at every leaf's
 * interior Chebyshev nodes and 0 at its exterior nodes, with A the collocation of Eq.
 * basic (Sec. 3.2: tensor-product spectral derivatives) for the coefficient fields
 * coeffs_dev ([6][n_leaf][p*p], as hps_build takes them; they need not be the handle's).
 * u_dev, out_dev: [n_leaf][p*p][nrhs] device FP64 (u's exterior values are used as given,
 * e.g. a solution from hps_solve).  This is the explicit half of an implicit time step:
 * Crank-Nicolson (Sec. 7.6) solves (I/k - A/2) u_{n+1} = (I/k + A/2) u_n, whose right-hand
 * side is 2/k u_n - (I/k - A/2) u_n (alpha = 2/k, beta = -1 with the solved operator's
 * coefficients).  Computed in double-float arithmetic (about 48 significant bits),
 * asynchronous on stream. */
int hps_apply(hps_handle* h, const double* coeffs_dev, const double* u_dev, int nrhs, double alpha, double beta,
              double* out_dev, void* stream);

/* hps_solve with extras: rho_dev (may be NULL) is a right-hand side for the flux
 * continuity equations, [n_gauss][nrhs] by global id (entries off interior nodes are
 * ignored); ug_dev (may be NULL) receives the solution at every Gaussian node
 * [n_gauss][nrhs]; iters (may be NULL) receives the refinement steps taken. */
int hps_solve_ext(hps_handle* h, const double* f_dev, const double* g_dev, const double* rho_dev,
                  int nrhs, double* u_dev, double* ug_dev, int* iters, void* stream);

/* Solve without allocating device memory.  The paper has no counterpart: this serves
 * callers that cannot let a solve allocate -- a host framework that has already reserved
 * nearly all device memory for its own pool, or a time-stepping loop that must not pay
 * for (or risk failing) an allocation once it runs.  Same arguments and result as
 * hps_solve for an HPS_FP64 handle (STATE for other precisions); the handle itself still
 * comes from hps_build, which does allocate.  The per-call work buffers -- the box
 * flux/particular-solution pool, the merge difference vectors, the Gaussian-node
 * solution and the split-K partial sums, (box rows + merge rows + n_gauss + partial rows)
 * * nrhs doubles, and from 8 right-hand sides on the exponents of the tensor-core products
 * (96 ints per 64-row operator block and 32 right-hand sides) -- live in one fixed
 * array of HPS_NOALLOC_SCRATCH_BYTES in device memory that the library image carries and
 * every GPU that loads it keeps until the process exits; a call that would need more is
 * rejected with INVALID_ARG and a message giving the size.  All calls share that array:
 * calls whose work overlaps on the GPU (several streams or host threads) race on it and
 * must be serialised.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before any
 * stream capture. */
#define HPS_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int hps_solve_noalloc(hps_handle* h, const double* f_dev, const double* g_dev, int nrhs, double* u_dev,
                      void* stream);

/* Adjoint of the solve (transposed Algorithm 2 sweeps).  dJdu_dev: [n_leaf][p*p][nrhs],
 * the gradient of a functional with respect to the output of hps_solve.  Outputs (each
 * may be NULL): dJdf_dev [n_boundary][nrhs], dJdg_dev [n_leaf][p*p][nrhs] (zero at
 * exterior nodes), dJdcoeffs_dev [6][n_leaf][p*p] (summed over right-hand sides; needs
 * u_dev, the forward solution of hps_solve for the same nrhs).  Uses the FP64 operator
 * store, so the handle must be HPS_FP64 (STATE otherwise). */
int hps_adjoint(hps_handle* h, const double* dJdu_dev, int nrhs, const double* u_dev,
                double* dJdf_dev, double* dJdg_dev, double* dJdcoeffs_dev, void* stream);

/* Sizes held by a handle: leaves, p, q, Gaussian nodes, boundary nodes, operator bytes. */
int hps_handle_info(const hps_handle* h, int* n_leaves, int* p, int* q, int* n_gauss,
                    int* n_boundary, int64_t* operator_bytes);

/* Reads the device status word of the handle (synchronising the stream): OK or the
 * first device-detected error. */
int hps_sync_status(hps_handle* h, void* stream);

int hps_destroy(hps_handle* h);

/* Launch timing, process-wide.  While enabled, every kernel launch of the library is
 * bracketed by CUDA events on its stream and filed under a category name (kernel and
 * step) with the algorithmic flops and bytes of that launch.  hps_timing_count
 * synchronises on the recorded events and returns the number of categories;
 * hps_timing_get reads category i (name copied into name[0..name_len)).  Totals
 * accumulate until hps_timing_reset.  Disabled by default. */
int hps_timing_enable(int on);
int hps_timing_reset(void);
int hps_timing_count(int* n);
int hps_timing_get(int i, char* name, int name_len, int64_t* launches, double* ms, double* flops,
                   double* bytes);

/* Self-test of the bounded waits that every tensor-core kernel uses: one CTA waits on an
 * mbarrier that nothing arrives at, polling at most `polls` times (1 <= polls <= 2^26),
 * while a second warp waits on the CTA's abort flag; the first wait gives up, raises the
 * flag and sets the status word, the second sees the flag and returns.  Returns TIMEOUT
 * when both behaved so (the call synchronises the stream), INVALID_ARG for a bad polls,
 * CUDA for a launch error.  The device stays usable afterwards. */
int hps_selftest_wait_timeout(int polls, void* stream);

/* Message of the last failed call on this thread ("" if none).  Valid until the next
 * call on the same thread. */
const char* hps_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HPS_GB300_H */
