// Batched, blocked, partial Gauss-Jordan elimination (build stage, Algorithm 1).
//
// Every leaf and every merge of the build reduces to one dense elimination.  For a leaf
// the matrix is M = [[A_ci,ci, A_ci,ce L_ce,ge], [D_ge,ci, D_ge,ce L_ce,ge]] (Sec. 3); for
// a merge it is M = [[Z, R], [-C, blkdiag(T11a, T22b)]] with Z = T33a - T33b,
// R = [-T31a | T32b], C = [T13a ; T23b] (Sec. 4).  Eliminating the first K pivots in place
// (partial pivoting restricted to the first K rows) turns [[P, Q], [E, G]] into
// [[P^-1, P^-1 Q], [-E P^-1, G - E P^-1 Q]]: for a leaf that is [[F, -S_ci], [-H, T]]
// (Eqs. alpine1-alpine4) and for a merge [[X, S], [C X, T_tau]] (the merge formulas of
// Sec. 4).  One sweep gives every operator Algorithm 1 asks for.
//
// Row swaps are never executed: perm maps logical rows to physical rows, and the
// extraction kernel undoes the permutation (the inverse block picks up perm on its
// columns).  Each panel of nb pivots costs three launches over the whole batch:
//   gj_panel  : one CTA per matrix factors the nb-wide sub-panel (rows [c0, K)) with
//               partial pivoting, records the pivot rows and forms Pinv = M_PP^-1;
//   gj_prep   : writes the final panel columns (W_r = -M_rP Pinv, or Pinv on pivot rows)
//               and copies the pivot rows to a side buffer;
//   gj_update : rank-nb update of every other column, M_r += W_r Prow (pivot rows are
//               replaced by Pinv Prow).
// FP64 FFMA and DMMA run at about 1.2 TFLOP/s on GB300, so the FP64 update runs on the
// bf16 tensor cores by exact digit slicing (gj_update_tcs_kernel, gj_update_tcp_kernel
// below); the register-tiled SIMT kernel serves FP32 batches and remains a tuning
// candidate.
#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "hps_internal.h"

namespace hps {

namespace {

constexpr int NBMAX = 16;

template <typename T>
__device__ __forceinline__ T tabs(T v) { return v < T(0) ? -v : v; }

template <typename T> struct Eps;
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };
template <> struct Eps<float> { static constexpr float v = FLT_EPSILON; };

template <typename T>
__global__ void gj_init_kernel(const GJDesc* __restrict__ d, int* __restrict__ perm) {
  const GJDesc md = d[blockIdx.x];
  for (int i = threadIdx.x; i < md.K; i += blockDim.x) perm[md.perm_off + i] = i;
}

// Zeroes the bottom-left block (rows K .. R - 1, columns 0 .. K - 1) of every matrix: the
// blocked elimination then adds (-C) Top into it (matrix blockIdx.y).
__global__ void gj_zero_bl_kernel(const GJDesc* __restrict__ d, double* __restrict__ work) {
  const GJDesc md = d[blockIdx.y];
  const int K = md.K, R = md.R;
  const long long n = (long long)(R - K) * K;
  double* M = work + md.off + (long long)K * R;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / K;
    M[i * R + (e - i * K)] = 0.0;
  }
}

// Magnitude order of floating-point values as integers: the bit pattern of |v| read as an
// unsigned integer is monotone in |v| (finite values), so pivot searches run on the integer
// pipe instead of the scarce FP64 one.
template <typename T> struct KeyOf;
template <> struct KeyOf<double> {
  using type = unsigned long long;
  static __device__ __forceinline__ type key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  }
  static __device__ __forceinline__ double val(type k) { return __longlong_as_double((long long)k); }
};
template <> struct KeyOf<float> {
  using type = unsigned int;
  static __device__ __forceinline__ type key(float v) { return __float_as_uint(v) & 0x7FFFFFFFu; }
  static __device__ __forceinline__ float val(type k) { return __uint_as_float(k); }
};

// x rounded to FP32 with integer operations (significand rounded half up to 24 bits) for
// exponents inside FP32's normal range; others take the FP64-pipe conversion.
__device__ __forceinline__ float float_of(double x) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E < 897 || E > 1150) return __double2float_rn(x);
  const unsigned long long m = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned mh = (unsigned)((m + (1ull << 28)) >> 29);
  const unsigned sgn = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
  return __uint_as_float(sgn | (((unsigned)(E - 896) << 23) + mh - (1u << 23)));
}

// Panel of an FP64 elimination with the pivots chosen in FP32.  Partial pivoting only needs
// the magnitudes of the updated panel entries to pick its rows, so the LU of the panel that
// chooses them runs on the FP32 pipe (64 times GB300's FP64 pipe); the outputs the
// elimination uses exactly, the pivot block's inverse Pinv and the breakdown test, come from
// the chosen rows' FP64 values: the block (rows in pivot order) is factored without further
// pivoting in FP64 and inverted.  A pivot chosen in FP32 is within a relative 1e-6 or so of
// the FP64 choice's magnitude, so the growth of the elimination is that of partial pivoting.
// (Matrices with a null-direction tolerance keep the FP64 panel: FP32 cannot resolve it.)
__device__ __forceinline__ void gj_panel_f32_select(const GJDesc& md, double* __restrict__ M, int* __restrict__ pm,
                                                    double* __restrict__ pinv_out, int c0, int nb, int nrows,
                                                    int* __restrict__ status, unsigned char* smraw) {
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = bs >> 5;
  const int R = md.R, ldp = nb + 1;
  float* P = reinterpret_cast<float*>(smraw);
  int* pr = reinterpret_cast<int*>(P + (size_t)nrows * ldp);
  __shared__ unsigned int red_v[32];
  __shared__ int red_i[32];
  __shared__ double colscale[NBMAX];
  __shared__ double B[NBMAX][NBMAX + 1];
  for (int i = tid; i < nrows; i += bs) pr[i] = pm[i];
  __syncthreads();
  for (int e = tid; e < nrows * nb; e += bs) {
    const int i = e / nb, j = e - (e / nb) * nb;
    P[i * ldp + j] = float_of(M[(long long)pr[i] * R + c0 + j]);
  }
  __syncthreads();
  // column scales for the breakdown test (the largest |P_ij| of the column)
  for (int j = warp; j < nb; j += nwarp) {
    unsigned int mx = 0;
    for (int i = lane; i < nrows; i += 32) mx = max(mx, __float_as_uint(P[i * ldp + j]) & 0x7FFFFFFFu);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) colscale[j] = (double)__uint_as_float(mx);
  }
  // pivot of column j: the largest |P_ij|, i >= j, the first row among equals.  Each thread
  // scans the rows it eliminates (i = j + tid, j + tid + bs, ...), so the scan of column
  // j + 1 rides on the elimination of column j; two block barriers per column.
  unsigned int best = 0;
  int bi = nrows;
  for (int i = tid; i < nrows; i += bs) {
    const unsigned int v = __float_as_uint(P[i * ldp]) & 0x7FFFFFFFu;
    if (bi == nrows || v > best) { best = v; bi = i; }
  }
  for (int j = 0; j < nb; ++j) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned int ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (oi < nrows && (bi == nrows || ov > best || (ov == best && oi < bi))) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();  // every thread's eliminations of column j - 1 and its scan are in
    if (warp == 0) {
      best = lane < nwarp ? red_v[lane] : 0u;
      bi = lane < nwarp ? red_i[lane] : nrows;
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned int ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (oi < nrows && (bi == nrows || ov > best || (ov == best && oi < bi))) { best = ov; bi = oi; }
      }
      const int r = __shfl_sync(0xffffffffu, bi < nrows ? bi : j, 0);
      if (lane == 0) {
        const int t = pr[j]; pr[j] = pr[r]; pr[r] = t;
      }
      if (r != j && lane < nb) {
        const float t = P[j * ldp + lane]; P[j * ldp + lane] = P[r * ldp + lane]; P[r * ldp + lane] = t;
      }
    }
    __syncthreads();  // the pivot row is in place
    const float pv = P[j * ldp + j];
    const float inv = pv != 0.f ? 1.f / pv : 0.f;
    best = 0;
    bi = nrows;
    const bool next = j + 1 < nb;
    for (int i = j + 1 + tid; i < nrows; i += bs) {
      const float l = P[i * ldp + j] * inv;
      P[i * ldp + j] = l;
      for (int c = j + 1; c < nb; ++c) P[i * ldp + c] = fmaf(-l, P[j * ldp + c], P[i * ldp + c]);
      if (next) {
        const unsigned int v = __float_as_uint(P[i * ldp + j + 1]) & 0x7FFFFFFFu;
        if (bi == nrows || v > best) { best = v; bi = i; }
      }
    }
  }
  __syncthreads();
  // the pivot block in FP64 (rows in pivot order), inverted in place by Gauss-Jordan
  // elimination without further pivoting, one thread per entry; its pivots are those of the
  // block's LU, tested against 64 eps of their column's scale
  __shared__ double dinv;
  for (int e = tid; e < nb * nb; e += bs) {
    const int t = e / nb, c = e - (e / nb) * nb;
    B[t][c] = M[(long long)pr[t] * R + c0 + c];
  }
  __syncthreads();
  const int bi_ = tid / nb, bc_ = tid - (tid / nb) * nb;
  for (int k = 0; k < nb; ++k) {
    if (tid == 0) {
      const double pvk = B[k][k];
      if (!(fabs(pvk) > 64.0 * DBL_EPSILON * colscale[k]) && status) atomicCAS(status, 0, md.box + 1);
      dinv = pvk != 0.0 ? 1.0 / pvk : 0.0;
    }
    __syncthreads();
    double v = 0.0;
    if (tid < nb * nb) {
      const double di = dinv;
      if (bi_ == k) v = bc_ == k ? di : B[k][bc_] * di;
      else v = bc_ == k ? -B[bi_][k] * di : B[bi_][bc_] - B[bi_][k] * (B[k][bc_] * di);
    }
    __syncthreads();
    if (tid < nb * nb) B[bi_][bc_] = v;
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += bs) {
    const int k = e / nb, t = e - (e / nb) * nb;
    pinv_out[k * NBMAX + t] = B[k][t];
  }
  for (int i = tid; i < nrows; i += bs) pm[i] = pr[i];
}

template <typename T>
__global__ void __launch_bounds__(1024) gj_panel_kernel(const GJDesc* __restrict__ d,
                                                       T* __restrict__ work, int* __restrict__ perm,
                                                       T* __restrict__ pinv, int c0, int nb_req,
                                                       int* __restrict__ status) {
  using Key = typename KeyOf<T>::type;
  const GJDesc md = d[blockIdx.x];
  if (c0 >= md.K) return;
  const int nb = min(nb_req, md.K - c0);
  const int nrows = md.K - c0;
  const int tid = threadIdx.x, bs = blockDim.x;
  extern __shared__ __align__(16) unsigned char smraw[];
  if constexpr (std::is_same<T, double>::value) {
    if (!(md.null_tol > 0.f && md.null_scale)) {
      gj_panel_f32_select(md, work + md.off, perm + md.perm_off + c0, pinv + (long long)blockIdx.x * NBMAX * NBMAX,
                          c0, nb, nrows, status, smraw);
      return;
    }
  }
  // the panel, nrows x nb with row pitch nb + 1 (odd): a warp walking down a column hits
  // distinct banks
  const int ldp = nb + 1;
  T* P = reinterpret_cast<T*>(smraw);
  int* pr = reinterpret_cast<int*>(P + (size_t)nrows * ldp);  // nrows
  __shared__ Key red_v[32];
  __shared__ int red_i[32];
  __shared__ T colscale[NBMAX];
  __shared__ T piv_inv;
  __shared__ int piv_row, piv_null;
  T* M = work + md.off;
  const int R = md.R;
  int* pm = perm + md.perm_off + c0;
  for (int i = tid; i < nrows; i += bs) pr[i] = pm[i];
  __syncthreads();
  for (int e = tid; e < nrows * nb; e += bs) {
    const int i = e / nb, j = e - (e / nb) * nb;
    P[i * ldp + j] = M[(long long)pr[i] * R + c0 + j];
  }
  __syncthreads();
  // column scales for the breakdown test: one warp per column, lanes stride the rows
  const int lane = tid & 31, warp = tid >> 5, nwarp = bs >> 5;
  for (int j = warp; j < nb; j += nwarp) {
    Key mx = 0;
    for (int i = lane; i < nrows; i += 32) mx = max(mx, KeyOf<T>::key(P[i * ldp + j]));
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, (Key)__shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) colscale[j] = KeyOf<T>::val(mx);
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    // pivot: the largest |P_ij|, i >= j, the first row among equals
    Key best = 0;
    int bi = nrows;
    for (int i = j + tid; i < nrows; i += bs) {
      const Key v = KeyOf<T>::key(P[i * ldp + j]);
      if (bi == nrows || v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const Key ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (oi < nrows && (bi == nrows || ov > best || (ov == best && oi < bi))) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      Key kb = red_v[0];
      int ib = red_i[0];
      for (int w = 1; w < nwarp; ++w)
        if (red_i[w] < nrows && (ib == nrows || red_v[w] > kb || (red_v[w] == kb && red_i[w] < ib))) {
          kb = red_v[w];
          ib = red_i[w];
        }
      const T b = ib < nrows ? KeyOf<T>::val(kb) : T(-1);
      const T tiny = T(64) * Eps<T>::v * colscale[j];
      piv_null = md.null_tol > 0.f && md.null_scale && !(b > (T)(md.null_tol * *md.null_scale));
      if (!piv_null && !(b > tiny) && status) atomicCAS(status, 0, md.box + 1);
      if (ib >= nrows) ib = j;
      piv_row = ib;
      const int t = pr[j]; pr[j] = pr[ib]; pr[ib] = t;
    }
    __syncthreads();
    const int r = piv_row;
    if (r != j && tid < nb) {
      const T t = P[j * ldp + tid]; P[j * ldp + tid] = P[r * ldp + tid]; P[r * ldp + tid] = t;
    }
    __syncthreads();
    // one reciprocal for the block (null direction: zero pivot, so no multipliers and a
    // zero Pinv row)
    if (tid == 0) {
      if (piv_null) P[j * ldp + j] = T(0);
      const T pv = P[j * ldp + j];
      piv_inv = (pv != T(0)) ? T(1) / pv : T(0);
    }
    __syncthreads();
    const T inv = piv_inv;
    for (int i = j + 1 + tid; i < nrows; i += bs) {
      const T l = P[i * ldp + j] * inv;
      P[i * ldp + j] = l;
      for (int c = j + 1; c < nb; ++c) P[i * ldp + c] -= l * P[j * ldp + c];
    }
    __syncthreads();
  }
  // Pinv = (L U)^-1 of the leading nb x nb block, one column per thread.
  if (tid < nb) {
    T y[NBMAX];
    for (int k = 0; k < nb; ++k) {
      T s = (k == tid) ? T(1) : T(0);
      for (int l = 0; l < k; ++l) s -= P[k * ldp + l] * y[l];
      y[k] = s;
    }
    for (int k = nb - 1; k >= 0; --k) {
      T s = y[k];
      for (int l = k + 1; l < nb; ++l) s -= P[k * ldp + l] * y[l];
      const T pv = P[k * ldp + k];
      y[k] = (pv != T(0)) ? s / pv : T(0);
    }
    T* Pi = pinv + (long long)blockIdx.x * NBMAX * NBMAX;
    for (int k = 0; k < nb; ++k) Pi[k * NBMAX + tid] = y[k];
  }
  for (int i = tid; i < nrows; i += bs) pm[i] = pr[i];
}

template <typename T>
__global__ void __launch_bounds__(256) gj_prep_kernel(const GJDesc* __restrict__ d,
                                                      T* __restrict__ work, const int* __restrict__ perm,
                                                      const T* __restrict__ pinv, T* __restrict__ prow,
                                                      long long prow_stride, int c0, int nb_req) {
  const GJDesc md = d[blockIdx.y];
  if (c0 >= md.K) return;
  const int nb = min(nb_req, md.K - c0);
  const int R = md.R;
  __shared__ T Pi[NBMAX * NBMAX];
  __shared__ int pphys[NBMAX];
  const int tid = threadIdx.x;
  const T* Pg = pinv + (long long)blockIdx.y * NBMAX * NBMAX;
  for (int e = tid; e < NBMAX * NBMAX; e += blockDim.x) Pi[e] = Pg[e];
  if (tid < nb) pphys[tid] = perm[md.perm_off + c0 + tid];
  __syncthreads();
  T* M = work + md.off;
  // thread (row r, output column j): 16 rows per block, 16 threads per row; a row's 16
  // threads are in one warp, read the row's panel entries first, then write
  const int r = blockIdx.x * 16 + (tid >> 4), j = tid & 15;
  const bool act = r < md.rows && j < nb;
  T* Mr = M + (long long)(act ? r : 0) * R + c0;
  int tp = -1;
  T w = T(0);
  if (act) {
    for (int t = 0; t < nb; ++t)
      if (pphys[t] == r) tp = t;
    if (tp < 0) {
      T acc = T(0);
      for (int t = 0; t < nb; ++t) acc += Mr[t] * Pi[t * NBMAX + j];
      w = -acc;
    } else {
      w = Pi[tp * NBMAX + j];
    }
  }
  __syncwarp();
  if (act) Mr[j] = w;
  // copy the pivot rows (columns outside the panel) to the side buffer
  T* pb = prow + (long long)blockIdx.y * prow_stride;
  const long long total = (long long)nb * R;
  for (long long e = (long long)blockIdx.x * blockDim.x + tid; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / R);
    const int c = (int)(e - (long long)t * R);
    if (c < c0 || c >= c0 + nb) pb[(long long)t * R + c] = M[(long long)pphys[t] * R + c];
  }
}

constexpr int UBM = 64, UBN = 64;

template <typename T>
__global__ void __launch_bounds__(256) gj_update_kernel(const GJDesc* __restrict__ d,
                                                        T* __restrict__ work, const int* __restrict__ perm,
                                                        const T* __restrict__ prow, long long prow_stride,
                                                        int c0, int nb_req) {
  const GJDesc md = d[blockIdx.y];
  if (c0 >= md.K) return;
  const int nb = min(nb_req, md.K - c0);
  const int R = md.R, rows = md.rows;
  const int tiles = (R + UBN - 1) / UBN;  // column tiles
  const int tm = blockIdx.x / tiles, tn = blockIdx.x - (blockIdx.x / tiles) * tiles;
  if (tm * UBM >= rows) return;
  const int row0 = tm * UBM, col0 = tn * UBN;
  if (col0 >= c0 && col0 + UBN <= c0 + nb) return;  // tile entirely inside the panel
  __shared__ T Ws[UBM][NBMAX + 1];
  __shared__ T Ps[NBMAX][UBN];
  __shared__ int pphys[NBMAX];
  __shared__ unsigned char isp[UBM];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T* M = work + md.off;
  if (tid < nb) pphys[tid] = perm[md.perm_off + c0 + tid];
  __syncthreads();
  if (tid < UBM) {
    const int r = row0 + tid;
    unsigned char f = 0;
    for (int t = 0; t < nb; ++t)
      if (pphys[t] == r) f = 1;
    isp[tid] = f;
  }
  for (int e = tid; e < UBM * NBMAX; e += 256) {
    const int i = e / NBMAX, t = e - (e / NBMAX) * NBMAX;
    const int r = row0 + i;
    Ws[i][t] = (r < rows && t < nb) ? M[(long long)r * R + c0 + t] : T(0);
  }
  const T* pb = prow + (long long)blockIdx.y * prow_stride;
  for (int e = tid; e < NBMAX * UBN; e += 256) {
    const int t = e / UBN, j = e - (e / UBN) * UBN;
    const int c = col0 + j;
    Ps[t][j] = (t < nb && c < R) ? pb[(long long)t * R + c] : T(0);
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int t = 0; t < nb; ++t) {
    T a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = Ws[ty + 16 * i][t];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Ps[t][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int li = ty + 16 * i;
    const int r = row0 + li;
    if (r >= rows) continue;
    T* Mr = M + (long long)r * R;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c >= R || (c >= c0 && c < c0 + nb)) continue;
      const T old = isp[li] ? T(0) : Mr[c];
      Mr[c] = old + acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------------------
// FP64 rank-nb update on the tcgen05 tensor cores with exact digit slicing.
//
// GB300's FP64 pipe does 2 FMA per clock per SM, its bf16 tensor cores about 1000 times
// that.  The update M_r += W_r Prow is a product with inner dimension nb <= 16, so it is
// computed exactly in pieces: every row of W (over its nb entries) is scaled by a power
// of two 2^e_r (e_r the exponent of the row's largest entry) and written as 8 signed
// base-256 digits, W_rt = 2^e_r sum_s a_s 2^(1-8s), |a_s| <= 128, each digit an integer
// exactly representable in bf16; every column of Prow likewise with 2^f_c and digits b_t.
// Digit products are integers below 2^14 and a diagonal d = s + t sums at most 8 x 16 of
// them, so the FP32 accumulation of the tensor core is exact.  The digit pairs with
// s + t <= 9 accumulate diagonal d in its own TMEM columns, 8 tcgen05.mma per tile (one per
// W digit plane against the Prow planes side by side); the epilogue combines the diagonals
// exactly in integers and rounds once to FP64.  The neglected terms are below about 2^-64 x 16 x max|W_r| x
// max|P_c|: on the leaf and merge eliminations that normwise bound can exceed the
// elementwise FP64 bound 2^-53 sum_t |W_rt| |P_tc| by up to 1e5 (measured on leaf panels),
// which 7 digits (2^-56) did not absorb and 8 digits do.  The tensor work is small (the
// tensor pipe is about 8 % busy); the kernel is bound by the epilogue's exact integer
// recombination of the diagonals (ALU and issue about 67 % busy), ahead of the read and write
// of the updated matrix (HBM about 30 % busy).
//
// Tile: 128 rows x 32 columns (MMA M = 128, N = 32, K = 16); operands in shared memory in
// the canonical K-major no-swizzle layout (8-row x 16-byte core matrices, LBO 128 bytes
// along K, SBO 256 bytes between row groups).
constexpr int TCM = 128, TCN = 32, TCS = 8, TCKEEP = 9;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start, LBO, SBO (all >> 4), version 1,
// no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// byte offset of (row, k) in a K-major tile with 16 k per row
__device__ __forceinline__ int kmaj16(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Digits are formed with integer operations only (the FP64 pipe is the scarce unit):
// with E the biased exponent of x and Emax the largest of its row (or column), the
// fixed-point value X = x / 2^(Emax - 1022) * 2^63 is the 53-bit significand shifted by
// E - Emax + 10 (rounded when shifted right), |X| < 2^63; its balanced base-256 digits
// a_8 .. a_1 (each in [-128, 128]) satisfy x = 2^(Emax-1022) sum_s a_s 2^(1-8s).
__device__ __forceinline__ int biased_exp(long long bits) { return (int)((bits >> 52) & 0x7FF); }

__device__ __forceinline__ void write_digits(long long bits, int emax, unsigned char* base, int plane_bytes,
                                             int off) {
  const int E = biased_exp(bits);
  long long X = 0;
  if (E > 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = E - emax + 10;
    if (sh >= 0) X = m << sh;
    else if (sh > -60) X = (m + (1ll << (-sh - 1))) >> (-sh);
    if (bits < 0) X = -X;
  }
#pragma unroll
  for (int s = TCS - 1; s >= 0; --s) {
    int a;
    if (s > 0) {
      a = (int)((X + 128) & 255) - 128;
      X = (X - a) >> 8;
    } else {
      a = (int)X;
    }
    *reinterpret_cast<__nv_bfloat16*>(base + s * plane_bytes + off) = __float2bfloat16_rn((float)a);
  }
}

// ---------------------------------------------------------------------------------------
// Persistent, warp-specialised form of the tensor-core update.  One CTA per SM loops over
// the launch's tiles (tile t = blockIdx.x + k gridDim.x), and three roles work on three
// tiles at once:
//   warps 0-3  (producers): load the tile's W rows and pivot-row columns, write their
//              digit planes and scales into buffer k % 2;
//   warp 4     (one thread): issue the digit-pair products of tile k into TMEM buffer
//              k % 2 and commit them to an mbarrier;
//   warps 8-15 (epilogue): read TMEM (warp w reads lanes 32 (w % 4) ..., columns
//              16 ((w - 8) / 4) ...), recombine, update the matrix through a staging
//              buffer (coalesced).
// Handoffs use mbarriers per buffer: full (producers -> MMA), done (MMA -> epilogue),
// free (epilogue -> producers).  One elected thread per role waits, with an iteration
// limit, and broadcasts the result over the role's named barrier; a timeout stops every
// role (abort flag) and is reported as status -1.
constexpr int PT_THREADS = 512;
constexpr int PT_EPI = 256;  // epilogue threads: 2 per tile row, 16 columns each
constexpr int PT_PLANES = TCS * TCM * 16 * 2 + TCS * TCN * 16 * 2;  // 40 KB per buffer
constexpr long long PT_WAIT = 1ll << 26;

struct PtShared {
  unsigned char planes[2][PT_PLANES];
  double sW[TCM][17];            // producers: the W tile, loaded coalesced
  double stg[TCM][TCN + 1];      // epilogue: the products, stored coalesced
  int er[2][TCM];
  int cexp[2][TCN];
  unsigned char isp[2][TCM];
  unsigned long long full[2], done[2], freeb[2];
  unsigned int tmem_base;
  int abort_flag;
  int ok_prod, ok_epi;
  int pphys[16];
};

__device__ __forceinline__ void mb_init(unsigned long long* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mb_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// bounded wait for the phase with the given parity; false on timeout or abort
__device__ __forceinline__ bool mb_wait(unsigned long long* b, int parity, volatile int* abort_flag, int* status) {
  for (long long it = 0; it < PT_WAIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  if (status) atomicCAS(status, 0, -1);
  return false;
}
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__global__ void __launch_bounds__(PT_THREADS, 1) gj_update_tcp_kernel(
    const GJDesc* __restrict__ d, int nmat, int rtmax, int ctmax, double* __restrict__ work,
    const int* __restrict__ perm, const double* __restrict__ prow, long long prow_stride, int c0, int nb_req,
    int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char pt_raw[];
  PtShared& sh = *reinterpret_cast<PtShared*>(pt_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long tpm = (long long)rtmax * ctmax, total = (long long)nmat * tpm;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mb_init(&sh.full[b], TCM);
      mb_init(&sh.done[b], 1);
      mb_init(&sh.freeb[b], PT_EPI);
    }
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sh.tmem_base;
  volatile int* abort_flag = &sh.abort_flag;
  // tile decoding, identical in every role
  auto decode = [&](long long t, GJDesc& md, int& nb, int& row0, int& col0) -> bool {
    const int m = (int)(t / tpm);
    const int local = (int)(t - (long long)m * tpm);
    md = d[m];
    if (c0 >= md.K) return false;
    nb = min(nb_req, md.K - c0);
    row0 = (local / ctmax) * TCM;
    col0 = (local % ctmax) * TCN;
    if (row0 >= md.rows || col0 >= md.R) return false;
    if (col0 >= c0 && col0 + TCN <= c0 + nb) return false;
    return true;
  };
  if (warp < 4) {
    // ---------------- producers
    const int i = tid;  // row of the tile
    int k = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
      GJDesc md;
      int nb, row0, col0;
      if (!decode(t, md, nb, row0, col0)) continue;
      const int buf = k & 1;
      const int R = md.R, rows = md.rows;
      const double* M = work + md.off;
      long long pv[16];
      if (i < TCN) {
        const int c = col0 + i;
        const bool cvalid = c < R && !(c >= c0 && c < c0 + nb);
        const double* pb = prow + (long long)(t / tpm) * prow_stride;
#pragma unroll
        for (int q = 0; q < 16; ++q) pv[q] = (cvalid && q < nb) ? __double_as_longlong(pb[(long long)q * R + c]) : 0ll;
      }
      for (int e = i; e < TCM * 16; e += TCM) {
        const int r = e >> 4, q = e & 15, rr = row0 + r;
        sh.sW[r][q] = (rr < rows && q < nb) ? M[(long long)rr * R + c0 + q] : 0.0;
      }
      if (i < 16) sh.pphys[i] = i < nb ? perm[md.perm_off + c0 + i] : -1;
      // the loads above are in flight while waiting for buffer buf to be released
      if (k >= 2 && i == 0) sh.ok_prod = mb_wait(&sh.freeb[buf], ((k >> 1) - 1) & 1, abort_flag, status) ? 1 : 0;
      named_bar(1, TCM);
      if (k >= 2 && !sh.ok_prod) break;
      const int row = row0 + i;
      int er = 0;
      long long w[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        w[q] = __double_as_longlong(sh.sW[i][q]);
        er = max(er, biased_exp(w[q]));
      }
      bool isp = false;
#pragma unroll
      for (int q = 0; q < 16; ++q) isp |= (sh.pphys[q] == row);
      sh.er[buf][i] = er;
      sh.isp[buf][i] = (row < rows && isp) ? 1 : 0;
      unsigned char* A = sh.planes[buf];
      unsigned char* B = A + TCS * TCM * 32;
#pragma unroll
      for (int q = 0; q < 16; ++q) write_digits(w[q], er, A, TCM * 32, kmaj16(i, q));
      if (i < TCN) {
        int ec = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) ec = max(ec, biased_exp(pv[q]));
        sh.cexp[buf][i] = ec;
#pragma unroll
        for (int q = 0; q < 16; ++q) write_digits(pv[q], ec, B, TCN * 32, kmaj16(i, q));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mb_arrive(&sh.full[buf]);
      named_bar(1, TCM);  // sW is reused by the next tile
      ++k;
    }
  } else if (warp == 4) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TCM >> 4) << 24);  // N per product
      int k = 0;
      for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        GJDesc md;
        int nb, row0, col0;
        if (!decode(t, md, nb, row0, col0)) continue;
        const int buf = k & 1;
        if (!mb_wait(&sh.full[buf], (k >> 1) & 1, abort_flag, status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(sh.planes[buf]), b0 = a0 + TCS * TCM * 32;
        const uint32_t tb = tmem + (uint32_t)(buf * 256);
        // one product per A digit plane s against the B planes t = 1 .. 9 - s side by side
        // (contiguous in the K-major layout, N = 32 (9 - s)), written from TMEM column
        // 32 (s - 1): block t lands on diagonal s + t
        for (int sa = 1; sa < TCKEEP; ++sa) {
          const uint64_t ad = umma_desc(a0 + (sa - 1) * (TCM * 32), 128, 256);
          const uint64_t bd = umma_desc(b0, 128, 256);
          const uint32_t idn = idesc | ((uint32_t)((TCN * (TCKEEP - sa)) >> 3) << 17);
          const uint32_t acc = sa > 1 ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tb + (uint32_t)((sa - 1) * TCN)),
              "l"(ad), "l"(bd), "r"(idn), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&sh.done[buf])));
        ++k;
      }
    }
  } else if (warp >= 8) {
    // ---------------- epilogue: thread (half h, row e) takes columns 16 h .. 16 h + 15
    const int te = tid - 256, ew = warp & 3, h = (warp - 8) >> 2;
    const int e = ew * 32 + lane;  // row of the tile = TMEM lane
    int k = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
      GJDesc md;
      int nb, row0, col0;
      if (!decode(t, md, nb, row0, col0)) continue;
      const int buf = k & 1;
      // the old values of this thread's 16 entries do not depend on the products: load
      // them first, so that their latency overlaps the wait
      const int R = md.R, rows = md.rows, wq = te >> 5;
      double* M = work + md.off;
      const int c = col0 + lane;
      const bool cok = c < R && !(c >= c0 && c < c0 + nb);
      double cv[TCM / 8];
#pragma unroll
      for (int q = 0; q < TCM / 8; ++q) {
        const int rr = row0 + wq + 8 * q;
        cv[q] = (cok && rr < rows) ? M[(long long)rr * R + c] : 0.0;
      }
      if (te == 0) sh.ok_epi = mb_wait(&sh.done[buf], (k >> 1) & 1, abort_flag, status) ? 1 : 0;
      named_bar(2, PT_EPI);
      if (!sh.ok_epi) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int er = sh.er[buf][e];
      const int jb = 16 * h;
      // the 8 diagonals of 8 columns at a time: 8 TMEM loads in flight, one wait
      long long Ih[16], Il[16];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t v[TCKEEP - 1][8];
#pragma unroll
        for (int dg = 2; dg <= TCKEEP; ++dg) {
          const uint32_t addr =
              tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(buf * 256 + (dg - 2) * TCN + jb + 8 * half);
          uint32_t* vd = v[dg - 2];
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(vd[0]), "=r"(vd[1]), "=r"(vd[2]), "=r"(vd[3]), "=r"(vd[4]), "=r"(vd[5]), "=r"(vd[6]),
                         "=r"(vd[7])
                       : "r"(addr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          long long hsum = 0, lsum = 0;
#pragma unroll
          for (int dg = 2; dg <= TCKEEP; ++dg) {
            const long long a = (long long)__float2int_rz(__uint_as_float(v[dg - 2][j]));
            if (dg <= 5) hsum += a * (1ll << (8 * (5 - dg)));
            else lsum += a * (1ll << (8 * (9 - dg)));
          }
          Ih[8 * half + j] = hsum;
          Il[8 * half + j] = lsum;
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        double vv = 0.0;
        const __int128 I = (__int128)Ih[j] * ((__int128)1 << 32) + (__int128)Il[j];
        if (I != 0) {
          const unsigned __int128 mag = I < 0 ? (unsigned __int128)(-I) : (unsigned __int128)I;
          const unsigned long long hi = (unsigned long long)(mag >> 64), lo = (unsigned long long)mag;
          const int bl = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
          const int shf = bl > 62 ? bl - 62 : 0;
          const long long T = (long long)(I >> shf);
          const long long b = __double_as_longlong(__ll2double_rn(T));
          const int E = biased_exp(b) + shf + (er - 1022) + (sh.cexp[buf][jb + j] - 1022) - 70;
          vv = E > 0 ? __longlong_as_double((b & ~(0x7FFll << 52)) | ((long long)E << 52)) : 0.0;
        }
        sh.stg[e][jb + j] = vv;
      }
      __shared__ unsigned char isp_row[TCM];
      if (h == 0) isp_row[e] = sh.isp[buf][e];
      asm volatile("tcgen05.fence::before_thread_sync;");
      mb_arrive(&sh.freeb[buf]);  // TMEM and buffer metadata read: producers may refill
      named_bar(2, PT_EPI);
      // coalesced update: epilogue warp q = te / 32 takes rows q, q + 8, ...; lane = column
#pragma unroll
      for (int q = 0; q < TCM / 8; ++q) {
        const int r = wq + 8 * q, rr = row0 + r;
        if (cok && rr < rows) M[(long long)rr * R + c] = (isp_row[r] ? 0.0 : cv[q]) + sh.stg[r][lane];
      }
      named_bar(2, PT_EPI);  // stg and isp_row are reused by the next tile
      ++k;
    }
  }
  // warps 5-7 have no role
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 4) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------------------
// Streamed form of the tensor-core update, for batches whose matrices start on 16-byte
// boundaries and have an even row length.  The work unit is a block of 128 rows and a run
// of up to ct column tiles of one matrix: the digit planes of the block's W rows are
// formed once per unit and serve every tile of the run.  Matrix tiles reach shared memory
// three tiles ahead of the epilogue, so that no thread holds a matrix load in flight: for
// a batch of equal matrices at a fixed stride by two tensor-map (TMA) copies of 128 x 16
// entries each (128-byte swizzled rows), otherwise by 16-byte asynchronous copies.  The
// epilogue writes the updated entries straight back.
// Roles (24 warps):
//   warps 0-3   producers: per unit, the W rows -> A digit planes (buffer u % 2) and row
//               scales; per tile k, warp k % 4 forms the pivot-row column digits (B slot k % 4);
//   warp 4      one thread issues the digit-pair products of tile k into TMEM buffer k % 2;
//   warp 5      loader: tile k's rows into C buffer k % 3;
//   warps 8-23  epilogue (4 warps per TMEM lane quarter, 8 columns each): TMEM -> exact
//               recombination, rounded once to FP64 with integer operations -> + old value
//               from the C buffer -> matrix.
// Every handoff is an mbarrier; waits are bounded and a timeout stops every role (status -1).
constexpr int PS_THREADS = 768;
constexpr int PS_EPI = 512;
constexpr int PS_CP = 34;  // C buffer row pitch in doubles (16-byte copies): 272 bytes, 16-byte aligned rows
constexpr int PS_NC = 3;   // C buffers
constexpr int PS_NB = 4;   // B slots (one per producer warp)
constexpr int PS_NE = 8;   // column-scale slots (tile k uses k % 8)
constexpr int PS_NU = 4;   // row-scale slots (unit u uses u % 4)

struct PsShared {
  unsigned char A[2][TCS * TCM * 32];
  unsigned char B[PS_NB][TCS * TCN * 32];
  // C buffers, 1024-byte aligned; with tensor-map copies each holds two swizzled 128 x 16 halves
  double C[PS_NC][TCM][PS_CP];
  int er[PS_NU][TCM];
  int cexp[PS_NE][TCN];
  unsigned char isp[PS_NU][TCM];
  unsigned long long afull[2], afree[2], bfull[PS_NB], bfree[PS_NB], cfull[PS_NC], cfree[PS_NC];
  unsigned long long tfull[2], tfree[2], mdone;
  unsigned int tmem_base;
  int abort_flag;
};

struct PsGeom {
  int rtmax, ctmax, ct, ncc;
  long long upm, total;
};

// Unit u of the launch: matrix, row block and column-tile run [j0, j1).  False when the
// unit holds no tile to update (past the matrix, or inside the pivot columns only).
__device__ __forceinline__ bool ps_unit(const GJDesc* __restrict__ d, long long u, const PsGeom& g, int c0,
                                        int nb_req, GJDesc& md, int& nb, int& row0, int& j0, int& j1) {
  const long long m = u / g.upm;
  const int r = (int)(u - m * g.upm);
  const int rb = r / g.ncc, cc = r - rb * g.ncc;
  md = d[m];
  if (c0 >= md.K) return false;
  nb = min(nb_req, md.K - c0);
  row0 = rb * TCM;
  if (row0 >= md.rows) return false;
  j0 = cc * g.ct;
  j1 = min(j0 + g.ct, (md.R + TCN - 1) / TCN);
  for (int j = j0; j < j1; ++j)
    if (!(j * TCN >= c0 && j * TCN + TCN <= c0 + nb)) return true;
  return false;
}

__device__ __forceinline__ bool ps_tile(int j, int c0, int nb) { return !(j * TCN >= c0 && j * TCN + TCN <= c0 + nb); }

// the fixed-point form of x = bits against the row (or column) exponent emax, as in
// write_digits
__device__ __forceinline__ long long fixed_point(long long bits, int emax) {
  const int E = biased_exp(bits);
  long long X = 0;
  if (E > 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = E - emax + 10;
    if (sh >= 0) X = m << sh;
    else if (sh > -60) X = (m + (1ll << (-sh - 1))) >> (-sh);
    if (bits < 0) X = -X;
  }
  return X;
}

// bf16 bits of a small integer |a| <= 2^8, exactly: 1.5 2^23 + a is an FP32 number with
// unit spacing, so subtracting 1.5 2^23 leaves a exactly, and a value with at most 8
// significant bits keeps them all in the upper half of its FP32 encoding.
__device__ __forceinline__ uint32_t bf16_of_int(int a) {
  return __float_as_uint(__int_as_float(0x4B400000 + a) - 12582912.0f) >> 16;
}

// The 8 balanced base-256 digit planes of one K-major row of 16 values (a row of W, or a
// column of Prow), one 16-byte store per plane and half row.  With X = sum_(i<7) a_i 2^(8i)
// + a_top 2^56 and a_i in [-128, 127], Y = X + 128 sum_(i<7) 2^(8i) (modulo 2^64) holds
// a_i + 128 in its byte i, so each low digit is one bit-field extraction; a_top is
// floor(Y / 2^56) read as a signed value, or unsigned when X >= 0 carried Y past 2^63.
// The loop over planes stays rolled: the kernel's roles share each SM's instruction cache.
__device__ __forceinline__ void write_digit_row(const long long* w, int emax, unsigned char* base, int plane_bytes,
                                                int row) {
  constexpr unsigned long long kOff = 128ull * ((1ull << 56) - 1) / 255;  // 128 in bytes 0 .. 6
  unsigned char* p0 = base + kmaj16(row, 0);
#pragma unroll
  for (int hq = 0; hq < 2; ++hq) {
    unsigned long long Y[8];
    int top[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const long long X = fixed_point(w[8 * hq + q], emax);
      Y[q] = (unsigned long long)X + kOff;
      top[q] = X >= 0 ? (int)(Y[q] >> 56) : (int)((long long)Y[q] >> 56);
    }
    {
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) pk[q >> 1] = bf16_of_int(top[q]) | (bf16_of_int(top[q + 1]) << 16);
      *reinterpret_cast<uint4*>(p0 + 128 * hq) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
#pragma unroll 1
    for (int i = 0; i < TCS - 1; ++i) {  // digit i -> plane 7 - i
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        const int a0 = (int)((Y[q] >> (8 * i)) & 255ull) - 128, a1 = (int)((Y[q + 1] >> (8 * i)) & 255ull) - 128;
        pk[q >> 1] = bf16_of_int(a0) | (bf16_of_int(a1) << 16);
      }
      *reinterpret_cast<uint4*>(p0 + (TCS - 1 - i) * plane_bytes + 128 * hq) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  }
}

// FP32 accumulator holding an exact integer |v| <= 2^22 -> that integer plus 0x4B400000
// (same unit-spacing argument as bf16_of_int; the bias is removed in recombine)
__device__ __forceinline__ int biased_int_of_acc(uint32_t v) {
  return __float_as_int(__uint_as_float(v) + 12582912.0f);
}

// The product entry from its 8 diagonal sums S_2 .. S_9 (s[0] .. s[7], each biased by
// 0x4B400000 as biased_int_of_acc leaves it):
//   W_r Prow_c = 2^(er + ec - 2114) I,  I = sum_d S_d 2^(8 (9 - d)),
// with I assembled exactly (|I| < 2^80) and rounded once to FP64 with integer operations
// (the FP64 pipe is the scarce unit): to nearest, ties away from zero, so the error is at
// most half a unit in the last place.  Results below the normal range flush to zero.
__device__ __forceinline__ double recombine(const int* s, int er, int ec) {
  // pairs S_d 2^8 + S_(d+1) (|.| < 2^31), the biases removed modulo 2^32
  constexpr unsigned int kBias = 257u * 0x4B400000u;
  auto pair = [](int hi, int lo) { return (int)((unsigned int)hi * 256u + (unsigned int)lo - kBias); };
  const int p01 = pair(s[0], s[1]), p23 = pair(s[2], s[3]), p45 = pair(s[4], s[5]), p67 = pair(s[6], s[7]);
  const long long H = (long long)p01 * 65536 + p23;  // I = H 2^32 + L
  const long long L = (long long)p45 * 65536 + p67;
  const long long T = H + (L >> 32);  // I = T 2^32 + u, 0 <= u < 2^32
  const unsigned int u = (unsigned int)L;
  const bool neg = T < 0;
  // |I| = A 2^32 + B
  const unsigned long long A = neg ? (unsigned long long)(-T) - (u != 0u ? 1ull : 0ull) : (unsigned long long)T;
  const unsigned int B = neg ? 0u - u : u;
  // W: the leading 64 bits of |I| when A >= 2^32 (B's top bits are shifted in below), else
  // all of |I|; N: W normalised so that the leading bit is bit 63.  Bits shifted out lie
  // below the rounding position and cannot change a round-half-up decision.
  const bool big = (A >> 32) != 0;
  const unsigned long long W = big ? A : ((A << 32) | B);
  if (W == 0) return 0.0;
  const int z = __clzll((long long)W);  // 16 .. 31 when big
  unsigned long long N = W << z;
  if (big) N |= (unsigned long long)(B >> (32 - z));
  const int top = (big ? 95 : 63) - z;  // position of the leading bit in |I|
  const unsigned long long mant = (N >> 11) + ((N >> 10) & 1ull);  // 2^52 .. 2^53
  const int E = top + er + ec - 1091;
  if (E <= 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)neg << 63;
  if (E >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
  // the leading bit of mant lands in the exponent field: a rounding carry to 2^53 raises it
  return __longlong_as_double((long long)(sgn + ((unsigned long long)(E - 1) << 52) + mant));
}

// bounded wait that ignores the abort flag: used only to drain the role's own operations
// before the block exits
__device__ __forceinline__ bool mb_drain(unsigned long long* b, int parity) {
  for (long long it = 0; it < PT_WAIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void mb_expect_arrive(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// box (x .. x + 15, y .. y + 127) of matrix z into shared memory (128-byte swizzled rows)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// the barrier receives one arrival when this thread's earlier asynchronous copies have landed
__device__ __forceinline__ void cp_async_arrive(unsigned long long* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

template <bool TMA>
__global__ void __launch_bounds__(PS_THREADS, 1) gj_update_tcs_kernel(
    const GJDesc* __restrict__ d, PsGeom g, double* __restrict__ work, const int* __restrict__ perm,
    const double* __restrict__ prow, long long prow_stride, int c0, int nb_req, int* __restrict__ status,
    const __grid_constant__ CUtensorMap cmap) {
  extern __shared__ __align__(1024) unsigned char ps_raw[];
  PsShared& sh = *reinterpret_cast<PsShared*>(ps_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mb_init(&sh.afull[b], TCM);
      mb_init(&sh.afree[b], 1);
      mb_init(&sh.tfull[b], 1);
      mb_init(&sh.tfree[b], PS_EPI);
    }
    for (int b = 0; b < PS_NB; ++b) {
      mb_init(&sh.bfull[b], 32);
      mb_init(&sh.bfree[b], 1);
    }
    for (int b = 0; b < PS_NC; ++b) {
      mb_init(&sh.cfull[b], TMA ? 1 : 32);
      mb_init(&sh.cfree[b], PS_EPI);
    }
    mb_init(&sh.mdone, 1);
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sh.tmem_base;
  volatile int* abort_flag = &sh.abort_flag;

  if (warp < 4) {
    // ---------------- producers (no block-wide barrier: a warp that stops leaves the others free)
    const int i = tid;
    long long k = 0;
    int ua = 0;
    bool stop = false;
    for (long long u = blockIdx.x; u < g.total && !stop; u += gridDim.x) {
      GJDesc md;
      int nb, row0, j0, j1;
      if (!ps_unit(d, u, g, c0, nb_req, md, nb, row0, j0, j1)) continue;
      const int R = md.R, rows = md.rows;
      const double* Mw = work + md.off;
      // the unit's W rows; their loads are in flight during the wait for the A buffer
      const int row = row0 + i;
      const bool rowok = row < rows;
      long long w[16];
#pragma unroll
      for (int q = 0; q < 16; ++q)
        w[q] = (rowok && q < nb) ? __double_as_longlong(Mw[(long long)row * R + c0 + q]) : 0ll;
      bool isp = false;
#pragma unroll
      for (int q = 0; q < 16; ++q) isp |= (q < nb) && (perm[md.perm_off + c0 + q] == row);
      if (ua >= 2) {
        int ok = 1;
        if (lane == 0) ok = mb_wait(&sh.afree[ua & 1], ((ua >> 1) - 1) & 1, abort_flag, status) ? 1 : 0;
        if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      }
      int er = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q) er = max(er, biased_exp(w[q]));
      sh.er[ua & (PS_NU - 1)][i] = er;
      sh.isp[ua & (PS_NU - 1)][i] = (rowok && isp) ? 1 : 0;
      write_digit_row(w, er, sh.A[ua & 1], TCM * 32, i);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mb_arrive(&sh.afull[ua & 1]);
      const double* pb = prow + (long long)(u / g.upm) * prow_stride;
      for (int j = j0; j < j1; ++j) {
        if (!ps_tile(j, c0, nb)) continue;
        if ((int)(k & 3) == warp) {
          const int c = j * TCN + lane;
          const bool cvalid = c < R && !(c >= c0 && c < c0 + nb);
          long long pv[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) pv[q] = (cvalid && q < nb) ? __double_as_longlong(pb[(long long)q * R + c]) : 0ll;
          if (k >= PS_NB) {
            int ok = 1;
            if (lane == 0) ok = mb_wait(&sh.bfree[warp], ((k >> 2) - 1) & 1, abort_flag, status) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
              stop = true;
              break;
            }
          }
          int ec = 0;
#pragma unroll
          for (int q = 0; q < 16; ++q) ec = max(ec, biased_exp(pv[q]));
          sh.cexp[k & (PS_NE - 1)][lane] = ec;
          write_digit_row(pv, ec, sh.B[warp], TCN * 32, lane);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mb_arrive(&sh.bfull[warp]);
        }
        ++k;
      }
      ++ua;
    }
  } else if (warp == 4) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TCM >> 4) << 24);  // N per product
      long long k = 0;
      int ua = 0;
      bool stop = false;
      for (long long u = blockIdx.x; u < g.total && !stop; u += gridDim.x) {
        GJDesc md;
        int nb, row0, j0, j1;
        if (!ps_unit(d, u, g, c0, nb_req, md, nb, row0, j0, j1)) continue;
        if (!mb_wait(&sh.afull[ua & 1], (ua >> 1) & 1, abort_flag, status)) break;
        const uint32_t a0 = smem_u32(sh.A[ua & 1]);
        for (int j = j0; j < j1; ++j) {
          if (!ps_tile(j, c0, nb)) continue;
          const int tb = (int)(k & 1), bs = (int)(k & 3);
          if (!mb_wait(&sh.bfull[bs], (k >> 2) & 1, abort_flag, status) ||
              (k >= 2 && !mb_wait(&sh.tfree[tb], ((k >> 1) - 1) & 1, abort_flag, status))) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t b0 = smem_u32(sh.B[bs]);
          const uint32_t tcol = tmem + (uint32_t)(tb * 256);
          // one product per A digit plane s against the B planes t = 1 .. 9 - s side by side
          // (contiguous in the K-major layout, N = 32 (9 - s)), written from TMEM column
          // 32 (s - 1): block t lands on diagonal s + t
#pragma unroll 1
          for (int sa = 1; sa < TCKEEP; ++sa) {
            const uint64_t ad = umma_desc(a0 + (sa - 1) * (TCM * 32), 128, 256);
            const uint64_t bd = umma_desc(b0, 128, 256);
            const uint32_t idn = idesc | ((uint32_t)((TCN * (TCKEEP - sa)) >> 3) << 17);
            const uint32_t acc = sa > 1 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tcol + (uint32_t)((sa - 1) * TCN)),
                "l"(ad), "l"(bd), "r"(idn), "r"(acc));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&sh.tfull[tb])));
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&sh.bfree[bs])));
          ++k;
        }
        if (stop) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&sh.afree[ua & 1])));
        ++ua;
      }
      // every product issued has completed before the block frees TMEM
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&sh.mdone)));
      mb_drain(&sh.mdone, 0);
    }
  } else if (warp == 5) {
    // ---------------- loader: the tile rows into C buffer k % 3
    long long k = 0;
    int cb = 0;
    bool stop = false;
    for (long long u = blockIdx.x; u < g.total && !stop; u += gridDim.x) {
      GJDesc md;
      int nb, row0, j0, j1;
      if (!ps_unit(d, u, g, c0, nb_req, md, nb, row0, j0, j1)) continue;
      const double* Mw = work + md.off;
      const int R = md.R, nr = min(TCM, md.rows - row0), m = (int)(u / g.upm);
      for (int j = j0; j < j1; ++j) {
        if (!ps_tile(j, c0, nb)) continue;
        if (k >= PS_NC) {
          int ok = 1;
          if (lane == 0) ok = mb_wait(&sh.cfree[cb], (int)((k / PS_NC) - 1) & 1, abort_flag, status) ? 1 : 0;
          if (!__shfl_sync(0xffffffffu, ok, 0)) {
            stop = true;
            break;
          }
        }
        const int col0 = j * TCN;
        if (TMA) {
          // two 128 x 16 boxes; entries past the matrix arrive as zeros
          if (lane == 0) {
            const bool two = col0 + 16 < R;
            mb_expect_arrive(&sh.cfull[cb], (two ? 2u : 1u) * (TCM * 16 * 8));
            unsigned char* cbuf = reinterpret_cast<unsigned char*>(&sh.C[cb][0][0]);
            tma_load_3d(cbuf, &cmap, col0, row0, m, &sh.cfull[cb]);
            if (two) tma_load_3d(cbuf + TCM * 16 * 8, &cmap, col0 + 16, row0, m, &sh.cfull[cb]);
          }
        } else {
          const int cpr = min(TCN, R - col0) >> 1;  // 16-byte chunks per row (R is even)
          const int nch = nr * cpr;
          for (int c = lane; c < nch; c += 32) {
            const int r = c / cpr, q = c - r * cpr;
            cp_async16(&sh.C[cb][r][2 * q], Mw + (long long)(row0 + r) * R + col0 + 2 * q);
          }
          cp_async_arrive(&sh.cfull[cb]);
        }
        ++k;
        cb = cb == PS_NC - 1 ? 0 : cb + 1;
      }
    }
    // the copies issued have landed before the block exits
    if (TMA) {
      if (lane == 0)
        for (int b = 0; b < PS_NC; ++b) {
          const long long n = k > b ? (k - 1 - b) / PS_NC + 1 : 0;  // copies armed on buffer b
          if (n > 0) mb_drain(&sh.cfull[b], (int)((n - 1) & 1));
        }
    } else {
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
  } else if (warp >= 8) {
    // ---------------- epilogue: thread (row e, group cg) takes columns 8 cg .. 8 cg + 7
    const int ew = warp & 3, cg = (warp - 8) >> 2;
    const int e = ew * 32 + lane;  // row of the tile = TMEM lane
    long long k = 0;
    int ua = 0, cb = 0;
    bool stop = false;
    for (long long u = blockIdx.x; u < g.total && !stop; u += gridDim.x) {
      GJDesc md;
      int nb, row0, j0, j1;
      if (!ps_unit(d, u, g, c0, nb_req, md, nb, row0, j0, j1)) continue;
      const int R = md.R;
      const bool rowok = row0 + e < md.rows;
      double* grow = work + md.off + (long long)(rowok ? row0 + e : 0) * R;
      for (int j = j0; j < j1; ++j) {
        if (!ps_tile(j, c0, nb)) continue;
        const int tb = (int)(k & 1);
        // every warp waits for itself, so that the warps drift apart and one warp's TMEM
        // and shared-memory latency overlaps the others' arithmetic
        int ok = 1;
        if (lane == 0)
          ok = (mb_wait(&sh.tfull[tb], (int)(k >> 1) & 1, abort_flag, status) &&
                mb_wait(&sh.cfull[cb], (int)(k / PS_NC) & 1, abort_flag, status))
                   ? 1
                   : 0;
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // row scale and pivot flag of the unit (written before its first products)
        const int er = sh.er[ua & (PS_NU - 1)][e];
        const bool isp = sh.isp[ua & (PS_NU - 1)][e] != 0;
        const double* crow = &sh.C[cb][e][0];
        const unsigned char* cbyte = reinterpret_cast<const unsigned char*>(&sh.C[cb][0][0]);
        const int col0 = j * TCN;
#pragma unroll 1
        for (int bt = 0; bt < 2; ++bt) {
          const int jb = 8 * cg + 4 * bt;
          uint32_t v[TCKEEP - 1][4];
#pragma unroll
          for (int dg = 2; dg <= TCKEEP; ++dg) {
            const uint32_t addr =
                tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(tb * 256 + (dg - 2) * TCN + jb);
            uint32_t* vd = v[dg - 2];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(vd[0]), "=r"(vd[1]), "=r"(vd[2]), "=r"(vd[3])
                         : "r"(addr));
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          int ec[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) ec[q] = sh.cexp[k & (PS_NE - 1)][jb + q];
          double2 o0, o1;
          if (TMA) {
            // half jb / 16, row e: 16-byte chunk c of the row sits at chunk c ^ (e % 8)
            const unsigned char* rb = cbyte + (jb >> 4) * (TCM * 16 * 8) + e * 128;
            const int ch = (jb & 15) >> 1;
            o0 = *reinterpret_cast<const double2*>(rb + ((ch ^ (e & 7)) << 4));
            o1 = *reinterpret_cast<const double2*>(rb + (((ch + 1) ^ (e & 7)) << 4));
          } else {
            o0 = *reinterpret_cast<const double2*>(crow + jb);
            o1 = *reinterpret_cast<const double2*>(crow + jb + 2);
          }
          if (bt == 1) {
            // TMEM buffer, column scales and C buffer read: hand them back
            asm volatile("tcgen05.fence::before_thread_sync;");
            mb_arrive(&sh.tfree[tb]);
            mb_arrive(&sh.cfree[cb]);
          }
          const double ov[4] = {o0.x, o0.y, o1.x, o1.y};
          double nv[4];
          bool up[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int s[TCKEEP - 1];
#pragma unroll
            for (int dg = 0; dg < TCKEEP - 1; ++dg) s[dg] = biased_int_of_acc(v[dg][q]);
            const int col = col0 + jb + q;
            up[q] = rowok && col < R && !(col >= c0 && col < c0 + nb);
            nv[q] = (isp ? 0.0 : ov[q]) + recombine(s, er, ec[q]);
          }
#pragma unroll
          for (int q = 0; q < 4; q += 2) {
            double* dst = grow + col0 + jb + q;
            if (up[q] && up[q + 1]) {
              *reinterpret_cast<double2*>(dst) = make_double2(nv[q], nv[q + 1]);
            } else {
              if (up[q]) dst[0] = nv[q];
              if (up[q + 1]) dst[1] = nv[q + 1];
            }
          }
        }
        ++k;
        cb = cb == PS_NC - 1 ? 0 : cb + 1;
      }
      ++ua;
    }
  }
  // warps 6 and 7 have no role
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 4) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <typename T, typename TO>
__global__ void __launch_bounds__(256) gj_extract_kernel(const GJDesc* __restrict__ d,
                                                         const T* __restrict__ work,
                                                         const int* __restrict__ perm, ExtractDst dst) {
  const int b = blockIdx.y;
  const GJDesc md = d[b];
  const int R = md.R, K = md.K;
  extern __shared__ __align__(16) unsigned char smraw[];
  int* sig = reinterpret_cast<int*>(smraw);   // K
  int* isig = sig + K;                         // K
  for (int i = threadIdx.x; i < K; i += blockDim.x) sig[i] = perm[md.perm_off + i];
  __syncthreads();
  for (int i = threadIdx.x; i < K; i += blockDim.x) isig[sig[i]] = i;
  __syncthreads();
  const T* M = work + md.off;
  const long long total = (long long)md.rows * R;
  TO* TL = (TO*)dst.TL; TO* TR = (TO*)dst.TR; TO* BL = (TO*)dst.BL;
  double* BR = (double*)dst.BR;  // the T store of the parents' merges stays FP64
  const long long tlo = dst.TL_off ? dst.TL_off[b] : (long long)b * dst.TL_off_stride;
  const long long tro = dst.TR_off ? dst.TR_off[b] : (long long)b * dst.TR_off_stride;
  const long long blo = dst.BL_off ? dst.BL_off[b] : (long long)b * dst.BL_off_stride;
  const long long bro = dst.BR_off ? dst.BR_off[b] : (long long)b * dst.BR_off_stride;
  const int ldTL = dst.ld_from_desc ? K : dst.TL_ld, ldBL = dst.ld_from_desc ? K : dst.BL_ld;
  const int ldTR = dst.ld_from_desc ? R - K : dst.TR_ld, ldBR = dst.ld_from_desc ? R - K : dst.BR_ld;
  (void)total;
  // the blocks' scale factors are +1 or -1: applied as a sign flip on the integer pipe, and
  // FP32 outputs rounded with integer operations (GB300's FP64 pipe would otherwise carry a
  // multiply or a conversion per entry)
  const bool nTL = dst.sTL < 0.0, nTR = dst.sTR < 0.0, nBL = dst.sBL < 0.0;
  auto out = [](T x, bool neg) -> TO {
    double v = (double)x;
    if (neg) v = __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
    if constexpr (std::is_same<TO, float>::value) return std::is_same<T, float>::value ? (float)v : float_of(v);
    else return v;
  };
  // one warp per logical row, lanes along it (reads of a row stay within one physical row;
  // writes are contiguous)
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int lr = blockIdx.x * nw + (threadIdx.x >> 5); lr < md.rows; lr += gridDim.x * nw) {
    const int sr = lr < K ? sig[lr] : lr;
    const T* Mr = M + (long long)sr * R;
    if (lr < K) {
      if (TL)
        for (int lc = lane; lc < K; lc += 32) TL[tlo + (long long)lr * ldTL + lc] = out(Mr[isig[lc]], nTL);
      if (TR)
        for (int lc = K + lane; lc < R; lc += 32) TR[tro + (long long)lr * ldTR + (lc - K)] = out(Mr[lc], nTR);
    } else {
      if (BL)
        for (int lc = lane; lc < K; lc += 32)
          BL[blo + (long long)(lr - K) * ldBL + lc] = out(Mr[isig[lc]], nBL);
      if (BR)
        for (int lc = K + lane; lc < R; lc += 32) BR[bro + (long long)(lr - K) * ldBR + (lc - K)] = (double)Mr[lc];
    }
  }
}

}  // namespace

template <typename T>
void launch_gj_init(const GJDesc* d, int nmat, int* perm, cudaStream_t s) {
  gj_init_kernel<T><<<nmat, 256, 0, s>>>(d, perm);
}

void launch_gj_zero_bl(const GJDesc* d, int nmat, long long max_entries, double* work, cudaStream_t s) {
  if (nmat <= 0 || max_entries <= 0) return;
  const long long bx = std::min<long long>((max_entries + 255) / 256, 64);
  gj_zero_bl_kernel<<<dim3((unsigned)bx, (unsigned)nmat), 256, 0, s>>>(d, work);
}

template <typename T>
void launch_gj_panel(const GJDesc* d, int nmat, int maxK, T* work, int* perm, T* pinv, int c0,
                     int nb, int* status, cudaStream_t s) {
  const int nrows = maxK - c0;
  if (nrows <= 0) return;
  const size_t smem = (size_t)nrows * (nb + 1) * sizeof(T) + (size_t)nrows * sizeof(int) + 16;
  ensure_smem((const void*)gj_panel_kernel<T>, smem);
  // many matrices: 256 threads each, several CTAs per SM; few (the large merges near the
  // root): a thread per panel row, up to 1024, so that each pivot step is short
  const int threads = nmat >= 2 * 152 ? 256 : std::max(256, std::min(1024, (nrows + 31) / 32 * 32));
  gj_panel_kernel<T><<<nmat, threads, smem, s>>>(d, work, perm, pinv, c0, nb, status);
}

template <typename T>
void launch_gj_prep(const GJDesc* d, int nmat, int maxR, T* work, const int* perm, const T* pinv,
                    T* prow, long long prow_stride, int c0, int nb, cudaStream_t s) {
  dim3 grid((maxR + 15) / 16, nmat);  // 16 rows per block
  gj_prep_kernel<T><<<grid, 256, 0, s>>>(d, work, perm, pinv, prow, prow_stride, c0, nb);
}

// cuTensorMapEncodeTiled from the driver, or null
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static bool tried = false;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

template <typename T>
void launch_gj_update(const GJDesc* d, int nmat, int maxR, int maxRows, T* work, const int* perm, T* prow,
                      long long prow_stride, int c0, int nb, cudaStream_t s, int* status, int tensor,
                      long long mat_stride) {
  int nsm = 1;
  if (std::is_same<T, double>::value && tensor) {  // per device: SM count and shared-memory limits
    nsm = device_sms();
    ensure_smem((const void*)gj_update_tcp_kernel, sizeof(PtShared));
    ensure_smem((const void*)gj_update_tcs_kernel<true>, sizeof(PsShared));
    ensure_smem((const void*)gj_update_tcs_kernel<false>, sizeof(PsShared));
  }
  if (std::is_same<T, double>::value && tensor == 2) {
    // FP64, streamed tensor-core kernel (16-byte aligned rows): one CTA per SM over units
    // of 128 rows x ct column tiles, ct chosen to leave about 4 units per SM
    PsGeom g;
    g.rtmax = (maxRows + TCM - 1) / TCM;
    g.ctmax = (maxR + TCN - 1) / TCN;
    const long long tiles = (long long)nmat * g.rtmax * g.ctmax;
    g.ct = (int)std::min<long long>(g.ctmax, std::max<long long>(1, (tiles + 4ll * nsm - 1) / (4ll * nsm)));
    g.ncc = (g.ctmax + g.ct - 1) / g.ct;
    g.upm = (long long)g.rtmax * g.ncc;
    g.total = (long long)nmat * g.upm;
    const int grid = (int)std::min<long long>(nsm, g.total);
    // equal matrices (R = maxR, rows = maxRows) at a fixed stride: tensor-map tile copies
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    bool tma = false;
    if (mat_stride > 0) {
      if (auto enc = tensor_map_encoder()) {
        const cuuint64_t dims[3] = {(cuuint64_t)maxR, (cuuint64_t)maxRows, (cuuint64_t)nmat};
        const cuuint64_t strides[2] = {(cuuint64_t)maxR * 8, (cuuint64_t)mat_stride * 8};
        const cuuint32_t box[3] = {16, (cuuint32_t)TCM, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        tma = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)work, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
      }
    }
    if (tma)
      gj_update_tcs_kernel<true><<<grid, PS_THREADS, sizeof(PsShared), s>>>(d, g, (double*)work, perm,
                                                                           (const double*)prow, prow_stride, c0,
                                                                           nb, status, map);
    else
      gj_update_tcs_kernel<false><<<grid, PS_THREADS, sizeof(PsShared), s>>>(d, g, (double*)work, perm,
                                                                            (const double*)prow, prow_stride, c0,
                                                                            nb, status, map);
  } else if (std::is_same<T, double>::value && tensor) {
    // FP64: the persistent tensor-core kernel, one CTA per SM over ceil(rows / 128) x
    // ceil(R / 32) tiles of every matrix
    const int ctmax = (maxR + TCN - 1) / TCN, rtmax = (maxRows + TCM - 1) / TCM;
    const long long total = (long long)nmat * ctmax * rtmax;
    const int grid = (int)std::min<long long>(nsm, total);
    gj_update_tcp_kernel<<<grid, PT_THREADS, sizeof(PtShared), s>>>(d, nmat, rtmax, ctmax, (double*)work, perm,
                                                                    (const double*)prow, prow_stride, c0, nb, status);
  } else {
    // every matrix needs ceil(rows / UBM) x ceil(R / UBN) tiles, which this grid covers
    const int tiles = (maxR + UBN - 1) / UBN, rtiles = (maxRows + UBM - 1) / UBM;
    dim3 grid(rtiles * tiles, nmat);
    gj_update_kernel<T><<<grid, 256, 0, s>>>(d, work, perm, prow, prow_stride, c0, nb);
  }
}

template <typename T, typename TO>
void launch_gj_extract(const GJDesc* d, int nmat, int maxR, const T* work, const int* perm,
                       const ExtractDst& dst, cudaStream_t s) {
  int gx = (maxR + 7) / 8;  // one warp per row, 8 per block
  if (gx > 1024) gx = 1024;
  const size_t smem = (size_t)2 * maxR * sizeof(int);
  ensure_smem((const void*)gj_extract_kernel<T, TO>, smem);
  gj_extract_kernel<T, TO><<<dim3(gx, nmat), 256, smem, s>>>(d, work, perm, dst);
}

template void launch_gj_init<double>(const GJDesc*, int, int*, cudaStream_t);
template void launch_gj_init<float>(const GJDesc*, int, int*, cudaStream_t);
template void launch_gj_panel<double>(const GJDesc*, int, int, double*, int*, double*, int, int, int*, cudaStream_t);
template void launch_gj_panel<float>(const GJDesc*, int, int, float*, int*, float*, int, int, int*, cudaStream_t);
template void launch_gj_prep<double>(const GJDesc*, int, int, double*, const int*, const double*, double*, long long, int, int, cudaStream_t);
template void launch_gj_prep<float>(const GJDesc*, int, int, float*, const int*, const float*, float*, long long, int, int, cudaStream_t);
template void launch_gj_update<double>(const GJDesc*, int, int, int, double*, const int*, double*, long long, int, int, cudaStream_t, int*, int, long long);
template void launch_gj_update<float>(const GJDesc*, int, int, int, float*, const int*, float*, long long, int, int, cudaStream_t, int*, int, long long);
template void launch_gj_extract<double, double>(const GJDesc*, int, int, const double*, const int*, const ExtractDst&, cudaStream_t);
template void launch_gj_extract<float, double>(const GJDesc*, int, int, const float*, const int*, const ExtractDst&, cudaStream_t);
template void launch_gj_extract<double, float>(const GJDesc*, int, int, const double*, const int*, const ExtractDst&, cudaStream_t);
template void launch_gj_extract<float, float>(const GJDesc*, int, int, const float*, const int*, const ExtractDst&, cudaStream_t);

}  // namespace hps
