// Solve-stage kernels (Algorithm 2), the flux-jump residual used by mixed-precision
// iterative refinement, and the adjoint helpers.
//
// Every operator application of Algorithm 2 -- h = H g on leaves, [w; h] = [X; C X] d and
// u_gi = S u_ge + w on merges, u_c = [F | S_ci] [g_ci; u_ge] on leaves -- is a batched
// product of a stored dense operator with a block of gathered vectors (one column per
// right-hand side).  The stored operators are streamed exactly once per solve (Sec. 5.4).
// FP64 products with inner dimension up to 448 and at least 8 right-hand sides go to the
// tensor-core kernel (k_gemm_tc.cu); the SIMT kernels here take the rest (FP32 sweeps,
// few right-hand sides, long inner dimensions).  Vectors are [row][rhs] with the
// right-hand side fastest.
#include <cfloat>
#include <map>
#include <mutex>
#include <utility>
#include <type_traits>

#include "hps_internal.h"

namespace hps {

namespace {

template <typename T> struct AccOf { using type = T; };

__device__ __forceinline__ int map_row(const int* __restrict__ idx, int base_or_off, int row_base, int k) {
  // idx offset < 0: identity (row_base + k); else row_base + idx[off + k]
  return base_or_off < 0 ? row_base + k : row_base + idx[base_or_off + k];
}

constexpr int KC = 256;  // K chunk staged in shared memory (transposed GEMV path)
constexpr int ROWS_HINT = 64;  // rows of one split-K output block

// Warp-wide sums of V values per lane ("transposing" reduction: every shuffle step halves
// the values a lane carries while V > 1).  On return lane l holds, in v[0 .. n), n =
// max(1, V / 32), the sums of values j = base * n + t with base = l for V >= 32 and
// base = l >> (5 - log2 V) otherwise (the lanes sharing a base hold equal sums).  V is a
// power of two.  V - 1 + max(0, 5 - log2 V) shuffles instead of 5 V.
template <int V, typename T>
__device__ __forceinline__ void warp_transpose_sum(T (&v)[V], int lane) {
  int n = V;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (n > 1) {
      const bool up = (lane & o) != 0;
      const int hn = n / 2;
#pragma unroll
      for (int j = 0; j < V / 2; ++j) {
        if (j < hn) {
          const T send = up ? v[j] : v[j + hn];
          const T keep = up ? v[j + hn] : v[j];
          v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      n = hn;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
}

template <typename T> struct Vec16;
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };

template <typename T>
__device__ __forceinline__ T vget(const typename Vec16<T>::type& a, int j);
template <>
__device__ __forceinline__ double vget<double>(const double2& a, int j) { return j == 0 ? a.x : a.y; }
template <>
__device__ __forceinline__ float vget<float>(const float4& a, int j) {
  return j == 0 ? a.x : (j == 1 ? a.y : (j == 2 ? a.z : a.w));
}

// Streaming products for few right-hand sides (nrhs <= NR), non-transposed: the bytes of
// the stored operator dominate, so the kernel is built to stream them.  One CTA of 256
// threads per item (<= 64 rows).  The item's gathered vector block is staged in shared
// memory in chunks of KC entries ([k][NR], zero past nrhs); warp w owns rows w, w + 8, ...
// (at most 8) and accumulates all of them at once.  Those rows start 8 lda apart, so they
// share one offset modulo the 16-byte vector width: after a scalar head of fewer than VW
// entries the warp reads every row with 16-byte streaming loads (each operator entry is
// read once per solve), 8 rows in flight per lane, and each staged vector entry once for
// all 8 rows.  Lane sums are combined by a transposing warp reduction.
template <typename TA, typename TV, int NR>
__global__ void __launch_bounds__(256) gemv_items_kernel(const GemmItem* __restrict__ items,
                                                         const TA* __restrict__ A, const TV* __restrict__ B0,
                                                         const TV* __restrict__ B1, TV* __restrict__ C,
                                                         const TV* __restrict__ Add, const int* __restrict__ idx,
                                                         int nrhs, TV beta) {
  using VecT = typename Vec16<TA>::type;
  constexpr int VW = Vec16<TA>::n;
  constexpr int KC = 16384 / (NR * (int)sizeof(TV));  // 16 KB of staged vector entries
  constexpr int RW = 8;                                // rows per warp
  __shared__ __align__(16) TV xs[KC * NR];
  const GemmItem it = items[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nrow = it.M > warp ? (it.M - warp + 7) / 8 : 0;  // rows warp + 8 i < M
  const TA* Aw = A + it.a_off + (long long)warp * it.lda;
  const long long rs = 8ll * it.lda;                           // row step within the warp
  TV acc[RW * NR];
#pragma unroll
  for (int j = 0; j < RW * NR; ++j) acc[j] = TV(0);
  // FP64 products double-buffer the operator loads (the next 8 rows' vectors are in flight
  // while the current ones feed the FP64 pipe, which bounds these products)
  constexpr bool DB = sizeof(TA) == 8;
  for (int k0 = 0; k0 < it.K; k0 += KC) {
    const int kc = min(KC, it.K - k0);
    // head: entries before the first 16-byte boundary of this warp's rows
    const long long o0 = it.a_off + (long long)warp * it.lda + k0;
    const int h = min(kc, (int)((VW - (int)(o0 % VW)) % VW));
    const int nv = (kc - h) / VW;
    const int t0 = h + nv * VW;  // first tail entry
    const TA* Ak = Aw + k0;
    // FP64: the first vectors of this chunk are requested before the staging, so that the
    // two latencies overlap (FP32 keeps the registers for occupancy)
    VecT ap[DB ? RW : 1];
    if (DB && lane < nv) {
#pragma unroll
      for (int i = 0; i < RW; ++i)
        if (i < nrow) ap[i] = __ldcs(reinterpret_cast<const VecT*>(Ak + i * rs + h + lane * VW));
    }
    for (int e = tid; e < kc * NR; e += 256) {
      const int kk = e / NR, r = e % NR;
      const int k = k0 + kk;
      TV v = TV(0);
      if (r < nrhs) {
        if (k < it.kseg) v = B0[(long long)map_row(idx, it.b0_idx, it.b0_row, k) * nrhs + r];
        else v = B1[(long long)map_row(idx, it.b1_idx, it.b1_row, k - it.kseg) * nrhs + r];
      }
      xs[e] = v;
    }
    __syncthreads();
    if (nrow > 0) {
      // scalar entries: the head (lane l < h takes entry l) and the tail (lane l takes entry
      // t0 + l while it is below kc)
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        const int kk = pass == 0 ? (lane < h ? lane : -1) : (t0 + lane < kc ? t0 + lane : -1);
        if (kk < 0) continue;
        TV xv[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) xv[r] = xs[kk * NR + r];
#pragma unroll
        for (int i = 0; i < RW; ++i)
          if (i < nrow) {
            const TV av = (TV)Ak[i * rs + kk];
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[i * NR + r] += av * xv[r];
          }
      }
      // body: 16-byte vectors
      for (int v = lane; v < nv; v += 32) {
        const int kk = h + v * VW;
        VecT a[RW];
        VecT an[DB ? RW : 1];
        if constexpr (DB) {
#pragma unroll
          for (int i = 0; i < RW; ++i) a[i] = ap[i];
          if (v + 32 < nv) {
#pragma unroll
            for (int i = 0; i < RW; ++i)
              if (i < nrow) an[i] = __ldcs(reinterpret_cast<const VecT*>(Ak + i * rs + kk + 32 * VW));
          }
        } else {
#pragma unroll
          for (int i = 0; i < RW; ++i)
            if (i < nrow) a[i] = __ldcs(reinterpret_cast<const VecT*>(Ak + i * rs + kk));
        }
#pragma unroll
        for (int j = 0; j < VW; ++j) {
          TV xv[NR];
#pragma unroll
          for (int r = 0; r < NR; ++r) xv[r] = xs[(kk + j) * NR + r];
#pragma unroll
          for (int i = 0; i < RW; ++i)
            if (i < nrow) {
              const TV aij = (TV)vget<TA>(a[i], j);
#pragma unroll
              for (int r = 0; r < NR; ++r) acc[i * NR + r] += aij * xv[r];
            }
        }
        if constexpr (DB) {
#pragma unroll
          for (int i = 0; i < RW; ++i) ap[i] = an[i];
        }
      }
    }
    __syncthreads();
  }
  if (nrow == 0) return;
  constexpr int V = RW * NR;
  warp_transpose_sum<V>(acc, lane);
  constexpr int NV = V >= 32 ? V / 32 : 1;
  constexpr int SH = V >= 32 ? 0 : (V == 16 ? 1 : (V == 8 ? 2 : (V == 4 ? 3 : (V == 2 ? 4 : 5))));
  if ((lane & ((1 << SH) - 1)) != 0) return;
  const int base = lane >> SH;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const int j = base * NV + t;
    const int i = j / NR, r = j % NR;
    const int row = warp + 8 * i;
    if (row < it.M && r < nrhs) {
      TV v = acc[t];
      const long long cr = (long long)map_row(idx, it.c_idx, it.c_row, row) * nrhs + r;
      if (it.add_row >= 0) v += Add[(long long)(it.add_row + row) * nrhs + r];
      C[cr] = (beta != TV(0) ? beta * C[cr] : TV(0)) + v;
    }
  }
}

// Streaming products of small items (inner dimension K <= WKMAX, nrhs <= NR): one warp per
// item, 8 items per CTA, each warp staging its own vector block in shared memory, so that
// the thousands of small products near the leaves (merge levels, the exterior-value product)
// do not pay a CTA's set-up each.  K <= 64: lane l computes rows l and l + 32 (the row's
// entries are contiguous and stay in L1 across the k loop; the staged vector is read by all
// lanes at once).  64 < K <= WKMAX: the rows are taken 8 at a time with the lanes along K,
// as in gemv_items_kernel.
constexpr int WKMAX = 128;

template <typename TA, typename TV, int NR>
__global__ void __launch_bounds__(256) gemv_warp_items_kernel(const GemmItem* __restrict__ items, int nitems,
                                                              const TA* __restrict__ A, const TV* __restrict__ B0,
                                                              const TV* __restrict__ B1, TV* __restrict__ C,
                                                              const TV* __restrict__ Add, const int* __restrict__ idx,
                                                              int nrhs, TV beta) {
  __shared__ TV xs_all[8][WKMAX * NR];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int item = blockIdx.x * 8 + warp;
  if (item >= nitems) return;
  const GemmItem it = items[item];
  TV* xs = xs_all[warp];
  for (int e = lane; e < it.K * NR; e += 32) {
    const int k = e / NR, r = e % NR;
    TV v = TV(0);
    if (r < nrhs) {
      if (k < it.kseg) v = B0[(long long)map_row(idx, it.b0_idx, it.b0_row, k) * nrhs + r];
      else v = B1[(long long)map_row(idx, it.b1_idx, it.b1_row, k - it.kseg) * nrhs + r];
    }
    xs[e] = v;
  }
  __syncwarp();
  const TA* Ab = A + it.a_off;
  auto store = [&](int row, int r, TV v) {
    if (row < it.M && r < nrhs) {
      const long long cr = (long long)map_row(idx, it.c_idx, it.c_row, row) * nrhs + r;
      if (it.add_row >= 0) v += Add[(long long)(it.add_row + row) * nrhs + r];
      C[cr] = (beta != TV(0) ? beta * C[cr] : TV(0)) + v;
    }
  };
  if (it.K <= 64) {
    TV acc[2][NR];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[i][r] = TV(0);
    const int r0 = lane, r1 = lane + 32;
    const TA* a0 = Ab + (long long)min(r0, it.M - 1) * it.lda;
    const TA* a1 = Ab + (long long)min(r1, it.M - 1) * it.lda;
#pragma unroll 4
    for (int k = 0; k < it.K; ++k) {
      const TV v0 = (TV)a0[k], v1 = (TV)a1[k];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const TV xv = xs[k * NR + r];
        acc[0][r] += v0 * xv;
        acc[1][r] += v1 * xv;
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      store(r0, r, acc[0][r]);
      store(r1, r, acc[1][r]);
    }
    return;
  }
  // lanes along K (consecutive lanes read consecutive entries of a row), 8 rows at a time
  for (int g0 = 0; g0 < it.M; g0 += 8) {
    TV acc[8 * NR];
#pragma unroll
    for (int j = 0; j < 8 * NR; ++j) acc[j] = TV(0);
    for (int k = lane; k < it.K; k += 32) {
      TV xv[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) xv[r] = xs[k * NR + r];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (g0 + i < it.M) {
          const TV av = (TV)Ab[(long long)(g0 + i) * it.lda + k];
#pragma unroll
          for (int r = 0; r < NR; ++r) acc[i * NR + r] += av * xv[r];
        }
    }
    constexpr int V = 8 * NR;
    warp_transpose_sum<V>(acc, lane);
    constexpr int NV = V >= 32 ? V / 32 : 1;
    constexpr int SH = V >= 32 ? 0 : (V == 16 ? 1 : (V == 8 ? 2 : 3));
    if ((lane & ((1 << SH) - 1)) == 0) {
      const int base = lane >> SH;
#pragma unroll
      for (int t = 0; t < NV; ++t) {
        const int j = base * NV + t;
        store(g0 + j / NR, j % NR, acc[t]);
      }
    }
  }
}

// Transposed GEMV: output i is column i of the stored K x lda operator.  256 threads =
// 4 K-groups x 64 outputs.
template <typename TA, typename TV, int NR>
__global__ void __launch_bounds__(256) gemvT_items_kernel(const GemmItem* __restrict__ items,
                                                          const TA* __restrict__ A, const TV* __restrict__ B0,
                                                          const TV* __restrict__ B1, TV* __restrict__ C,
                                                          const TV* __restrict__ Add, const int* __restrict__ idx,
                                                          int nrhs, TV beta) {
  using Acc = TV;
  const GemmItem it = items[blockIdx.x];
  __shared__ Acc Bs[KC][NR];
  __shared__ Acc red[4][64][NR];
  const int tid = threadIdx.x, i = tid & 63, kg = tid >> 6;
  const TA* Ab = A + it.a_off;
  Acc acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = Acc(0);
  for (int k0 = 0; k0 < it.K; k0 += KC) {
    const int kc = min(KC, it.K - k0);
    for (int e = tid; e < kc * NR; e += 256) {
      const int kk = e / NR, r = e - (e / NR) * NR;
      const int k = k0 + kk;
      Acc v = Acc(0);
      if (r < nrhs) {
        if (k < it.kseg) v = B0[(long long)map_row(idx, it.b0_idx, it.b0_row, k) * nrhs + r];
        else v = B1[(long long)map_row(idx, it.b1_idx, it.b1_row, k - it.kseg) * nrhs + r];
      }
      Bs[kk][r] = v;
    }
    __syncthreads();
    if (i < it.M) {
      for (int kk = kg; kk < kc; kk += 4) {
        const Acc a = (Acc)Ab[(long long)(k0 + kk) * it.lda + i];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] += a * Bs[kk][r];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) red[kg][i][r] = acc[r];
  __syncthreads();
  if (kg == 0 && i < it.M) {
    for (int r = 0; r < NR && r < nrhs; ++r) {
      Acc v = red[0][i][r] + red[1][i][r] + red[2][i][r] + red[3][i][r];
      const long long cr = (long long)map_row(idx, it.c_idx, it.c_row, i) * nrhs + r;
      if (it.add_row >= 0) v += Add[(long long)(it.add_row + i) * nrhs + r];
      C[cr] = (beta != TV(0) ? beta * C[cr] : TV(0)) + v;
    }
  }
}

// Tiled product for nrhs > 4: 64 rows x BN right-hand sides per CTA, 16 x 16 threads,
// 4 x (BN/16) outputs per thread.
template <typename TA, typename TV, int BN, bool TRANS>
__global__ void __launch_bounds__(256) gemm_items_kernel(const GemmItem* __restrict__ items,
                                                         const TA* __restrict__ A, const TV* __restrict__ B0,
                                                         const TV* __restrict__ B1, TV* __restrict__ C,
                                                         const TV* __restrict__ Add, const int* __restrict__ idx,
                                                         int nrhs, TV beta) {
  using Acc = TV;
  constexpr int BM = 64, BK = 16, TN = BN / 16;
  const GemmItem it = items[blockIdx.x];
  const int n0 = blockIdx.y * BN;
  __shared__ Acc As[BK][BM + 1];
  __shared__ Acc Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const TA* Ab = A + it.a_off;
  Acc acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Acc(0);
  for (int k0 = 0; k0 < it.K; k0 += BK) {
    for (int e = tid; e < BK * BM; e += 256) {
      int kk, rr;
      if (TRANS) { kk = e / BM; rr = e - (e / BM) * BM; }
      else { rr = e / BK; kk = e - (e / BK) * BK; }
      const int k = k0 + kk;
      Acc v = Acc(0);
      if (k < it.K && rr < it.M)
        v = TRANS ? (Acc)Ab[(long long)k * it.lda + rr] : (Acc)Ab[(long long)rr * it.lda + k];
      As[kk][rr] = v;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int kk = e / BN, n = e - (e / BN) * BN;
      const int k = k0 + kk, r = n0 + n;
      Acc v = Acc(0);
      if (k < it.K && r < nrhs) {
        if (k < it.kseg) v = B0[(long long)map_row(idx, it.b0_idx, it.b0_row, k) * nrhs + r];
        else v = B1[(long long)map_row(idx, it.b1_idx, it.b1_row, k - it.kseg) * nrhs + r];
      }
      Bs[kk][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[4], b[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = ty + 16 * i;
    if (row >= it.M) continue;
    const long long crow = (long long)map_row(idx, it.c_idx, it.c_row, row) * nrhs;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int r = n0 + tx + 16 * j;
      if (r >= nrhs) continue;
      Acc v = acc[i][j];
      if (it.add_row >= 0) v += Add[(long long)(it.add_row + row) * nrhs + r];
      C[crow + r] = (beta != TV(0) ? beta * C[crow + r] : TV(0)) + v;
    }
  }
}

template <typename TV>
__global__ void up_gather_kernel(const UpGather* __restrict__ g, const TV* __restrict__ V, TV* __restrict__ Vout,
                                 TV* __restrict__ dbuf, const double* __restrict__ rho,
                                 const int* __restrict__ idx, int nrhs) {
  const UpGather u = g[blockIdx.y];
  const int* p3a = idx + u.idx_off;
  const int* p3b = p3a + u.k3;
  const int* j3 = p3b + u.k3;
  const int* p1a = j3 + u.k3;
  const int* p2b = p1a + u.n1;
  const int rows = u.k3 + u.k3 + u.n1 + u.n2;
  // row `row`, right-hand sides r = r0, r0 + step, ... below nrhs
  auto body = [&](int row, int r0, int step) {
    if (row < u.k3) {
      const TV* vb = V + (long long)(u.vb_row + p3b[row]) * nrhs;
      const TV* va = V + (long long)(u.va_row + p3a[row]) * nrhs;
      const double* rr = rho ? rho + (long long)j3[row] * nrhs : nullptr;
      TV* dst = dbuf + (long long)(u.d_row + row) * nrhs;
      for (int r = r0; r < nrhs; r += step) {
        TV v = vb[r] - va[r];
        if (rr) v += (TV)rr[r];
        dst[r] = v;
      }
    } else if (row < 2 * u.k3) {
      TV* dst = Vout + (long long)(u.vt_row + row - u.k3) * nrhs;
      for (int r = r0; r < nrhs; r += step) dst[r] = TV(0);
    } else {
      const bool a = row < 2 * u.k3 + u.n1;
      const int i = a ? row - 2 * u.k3 : row - 2 * u.k3 - u.n1;
      const TV* src = V + (long long)(a ? u.va_row + p1a[i] : u.vb_row + p2b[i]) * nrhs;
      TV* dst = Vout + (long long)(u.vt_row + u.k3 + (a ? 0 : u.n1) + i) * nrhs;
      for (int r = r0; r < nrhs; r += step) dst[r] = src[r];
    }
  };
  if (nrhs >= 32) {  // a warp per row, lanes along the right-hand sides
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int row = blockIdx.x * nw + (threadIdx.x >> 5); row < rows; row += gridDim.x * nw) body(row, lane, 32);
  } else {
    const int total = rows * nrhs;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
      const int row = e / nrhs;
      body(row, e - row * nrhs, nrhs);
    }
  }
}

template <typename TV>
__global__ void down_scatter_kernel(const DownScatter* __restrict__ g, TV* __restrict__ VB,
                                    const TV* __restrict__ dbar, double* __restrict__ rhobar,
                                    const int* __restrict__ idx, int nrhs) {
  const DownScatter u = g[blockIdx.y];
  const int* p3a = idx + u.idx_off;
  const int* p3b = p3a + u.k3;
  const int* j3 = p3b + u.k3;
  const int* p1a = j3 + u.k3;
  const int* p2b = p1a + u.n1;
  const int rows = u.k3 + u.n1 + u.n2;
  const long long total = (long long)rows * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(e / nrhs);
    const int r = (int)(e - (long long)row * nrhs);
    if (row < u.k3) {
      const TV v = dbar[(long long)(u.d_row + row) * nrhs + r];
      VB[(long long)(u.vb_row + p3b[row]) * nrhs + r] = v;
      VB[(long long)(u.va_row + p3a[row]) * nrhs + r] = -v;
      if (rhobar) rhobar[(long long)j3[row] * nrhs + r] = (double)v;
    } else if (row < u.k3 + u.n1) {
      const int i = row - u.k3;
      VB[(long long)(u.va_row + p1a[i]) * nrhs + r] = VB[(long long)(u.vt_row + u.k3 + i) * nrhs + r];
    } else {
      const int i = row - u.k3 - u.n1;
      VB[(long long)(u.vb_row + p2b[i]) * nrhs + r] = VB[(long long)(u.vt_row + u.k3 + u.n1 + i) * nrhs + r];
    }
  }
}

template <typename TV>
__global__ void scatter_rows_kernel(const double* __restrict__ src, const int* __restrict__ idx, int n,
                                    TV* __restrict__ dst, int nrhs) {
  const long long total = (long long)n * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / nrhs);
    const int r = (int)(e - (long long)k * nrhs);
    dst[(long long)idx[k] * nrhs + r] = (TV)src[e];
  }
}

template <typename TI, typename TO>
__global__ void convert_kernel(const TI* __restrict__ src, TO* __restrict__ dst, long long n, double scale) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = (TO)(scale * (double)src[e]);
}

template <typename TI>
__global__ void axpy_kernel(const TI* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] += (double)x[e];
}

// y += x with the maxima of |x| and of the updated |y| (one pass instead of three)
__global__ void axpy_measure_kernel(const float* __restrict__ x, double* __restrict__ y, long long n,
                                    unsigned long long* __restrict__ out) {
  double mx = 0.0, my = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float xv = x[e];
    const double yv = y[e] + (double)xv;
    y[e] = yv;
    mx = fmax(mx, fabs((double)xv));
    my = fmax(my, fabs(yv));
    if (xv != xv) mx = DBL_MAX;  // NaN propagates as "huge"
    if (yv != yv) my = DBL_MAX;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    my = fmax(my, __shfl_down_sync(0xffffffffu, my, o));
  }
  __shared__ double red[2][32];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = mx;
    red[1][threadIdx.x >> 5] = my;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mx = fmax(mx, red[0][w]);
      my = fmax(my, red[1][w]);
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(mx));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(my));
  }
}

template <typename T>
__global__ void absmax_kernel(const T* __restrict__ x, long long n, unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)x[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    m = fmax(m, red[0]);
    if (m != m) m = DBL_MAX;  // NaN propagates as "huge"
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
  }
}

// Rows: dst[tab[3k]] (+)= src[tab[3k+1]] (+ src[tab[3k+2]] if >= 0).
template <typename TV>
__global__ void gather_reduce_kernel(const int* __restrict__ tab, int n, const TV* __restrict__ src,
                                     TV* __restrict__ dst, int nrhs, int accumulate) {
  const long long total = (long long)n * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / nrhs);
    const int r = (int)(e - (long long)k * nrhs);
    const int d = tab[3 * k], s1 = tab[3 * k + 1], s2 = tab[3 * k + 2];
    TV v = s1 >= 0 ? src[(long long)s1 * nrhs + r] : TV(0);
    if (s2 >= 0) v += src[(long long)s2 * nrhs + r];
    TV* o = dst + (long long)d * nrhs + r;
    *o = accumulate ? *o + v : v;
  }
}

// rho[e q + k] = -(v_a - v_b) on each interior edge; pairs = (edge, leaf_a, side_a,
// leaf_b, side_b) with a the W/S leaf.
__global__ void jump_residual_kernel(const int* __restrict__ pairs, int npairs, int q,
                                     const double* __restrict__ vflux, double* __restrict__ rho, int nrhs) {
  const int nq = 4 * q;
  const long long total = (long long)npairs * q * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int pi = (int)(e / ((long long)q * nrhs));
    const int rem = (int)(e - (long long)pi * q * nrhs);
    const int k = rem / nrhs, r = rem - (rem / nrhs) * nrhs;
    const int* P = pairs + 5 * pi;
    const double va = vflux[((long long)P[1] * nq + P[2] * q + k) * nrhs + r];
    const double vb = vflux[((long long)P[3] * nq + P[4] * q + k) * nrhs + r];
    rho[((long long)P[0] * q + k) * nrhs + r] = -(va - vb);
  }
}

template <typename TV>
__global__ void split_reduce_kernel(const SplitRed* __restrict__ d, const TV* __restrict__ P, TV* __restrict__ C,
                                    const TV* __restrict__ Add, const int* __restrict__ idx, int nrhs, TV beta) {
  const SplitRed sr = d[blockIdx.y];
  // row i, right-hand sides r = r0, r0 + step, ... below nrhs
  auto body = [&](int i, int r0, int step) {
    const long long crow = (long long)map_row(idx, sr.c_idx, sr.c_row, i) * nrhs;
    for (int r = r0; r < nrhs; r += step) {
      TV v = TV(0);
      for (int j = 0; j < sr.nsplit; ++j) v += P[(long long)(sr.p_row + j * sr.M + i) * nrhs + r];
      if (sr.add_row >= 0) v += Add[(long long)(sr.add_row + i) * nrhs + r];
      C[crow + r] = (beta != TV(0) ? beta * C[crow + r] : TV(0)) + v;
    }
  };
  if (nrhs >= 32) {  // a warp per row, lanes along the right-hand sides
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = blockIdx.x * nw + (threadIdx.x >> 5); i < sr.M; i += gridDim.x * nw) body(i, lane, 32);
  } else {
    const int total = sr.M * nrhs;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
      const int i = e / nrhs;
      body(i, e - i * nrhs, nrhs);
    }
  }
}

__global__ void row_combine_kernel(const int* __restrict__ tab, int n, double* __restrict__ dst,
                                   const double* __restrict__ A, const double* __restrict__ B, int nrhs) {
  const long long total = (long long)n * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / nrhs), r = (int)(e - (e / nrhs) * nrhs);
    const int* t = tab + 4 * k;
    double v = A[(long long)t[1] * nrhs + r];
    if (t[2] >= 0) v += (double)t[3] * B[(long long)t[2] * nrhs + r];
    dst[(long long)t[0] * nrhs + r] = v;
  }
}

inline int grid_for(long long n, int bs = 256, int cap = 8192) {
  long long g = (n + bs - 1) / bs;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

template <typename TA, typename TV>
void launch_gemm_items(const GemmItem* items, int nitems, int maxM, int trans, const TA* A, const TV* B0,
                       const TV* B1, TV* C, const TV* Add, const int* idx, int nrhs, double beta,
                       cudaStream_t s, const GemmCtx& cx) {
  (void)maxM;
  if (nitems <= 0) return;
  if constexpr (std::is_same<TA, double>::value && std::is_same<TV, double>::value) {
    if (gemm_tc_eligible(cx.maxK, nrhs) && launch_gemm_tc(items, nitems, trans, A, B0, B1, C, Add, idx, nrhs, beta, s, cx))
      return;
  }
  if constexpr (std::is_same<TA, float>::value && std::is_same<TV, float>::value) {
    if (cx.tc32 && !trans && gemm_tc32_eligible(nrhs) &&
        launch_gemm_tc32(items, nitems, A, B0, B1, C, Add, idx, nrhs, beta, cx.status, s, cx.dg))
      return;
  }
  const int bn = cx.bn;
  const TV b = (TV)beta;
  if (trans && nrhs <= 4) {
    if (nrhs == 1) gemvT_items_kernel<TA, TV, 1><<<nitems, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    else if (nrhs == 2) gemvT_items_kernel<TA, TV, 2><<<nitems, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    else gemvT_items_kernel<TA, TV, 4><<<nitems, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    return;
  }
  // streaming products: up to 4 right-hand sides in FP64 (bound by the FP64 pipe beyond),
  // up to 8 in FP32
  // small items, and enough of them for 16 warps per SM: one warp per item
  if (!trans && nrhs <= (sizeof(TV) == 8 ? 4 : 8) && cx.maxKv > 0 && cx.maxKv <= WKMAX && nitems >= 16 * 152) {
    const int grid = (nitems + 7) / 8;
    if (nrhs == 1) gemv_warp_items_kernel<TA, TV, 1><<<grid, 256, 0, s>>>(items, nitems, A, B0, B1, C, Add, idx, nrhs, b);
    else if (nrhs == 2) gemv_warp_items_kernel<TA, TV, 2><<<grid, 256, 0, s>>>(items, nitems, A, B0, B1, C, Add, idx, nrhs, b);
    else if (nrhs <= 4) gemv_warp_items_kernel<TA, TV, 4><<<grid, 256, 0, s>>>(items, nitems, A, B0, B1, C, Add, idx, nrhs, b);
    else if constexpr (sizeof(TV) == 4)
      gemv_warp_items_kernel<TA, TV, 8><<<grid, 256, 0, s>>>(items, nitems, A, B0, B1, C, Add, idx, nrhs, b);
    return;
  }
  if (!trans && nrhs <= (sizeof(TV) == 8 ? 4 : 8)) {
    if (nrhs == 1) gemv_items_kernel<TA, TV, 1><<<nitems, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    else if (nrhs == 2) gemv_items_kernel<TA, TV, 2><<<nitems, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    else if (nrhs <= 4) gemv_items_kernel<TA, TV, 4><<<nitems, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    else if constexpr (sizeof(TV) == 4)
      gemv_items_kernel<TA, TV, 8><<<nitems, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    return;
  }
  // right-hand-side tile: the caller's (autotuned) choice, else 16 up to 16 rhs and 64 above;
  // every choice computes each output with the same k order (bit-identical results)
  const int BN = (bn == 16 || bn == 32 || bn == 64) ? bn : (nrhs <= 16 ? 16 : 64);
  dim3 grid(nitems, (nrhs + BN - 1) / BN);
  if (BN == 16) {
    if (trans) gemm_items_kernel<TA, TV, 16, true><<<grid, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    else gemm_items_kernel<TA, TV, 16, false><<<grid, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
  } else if (BN == 32) {
    if (trans) gemm_items_kernel<TA, TV, 32, true><<<grid, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    else gemm_items_kernel<TA, TV, 32, false><<<grid, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
  } else {
    if (trans) gemm_items_kernel<TA, TV, 64, true><<<grid, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
    else gemm_items_kernel<TA, TV, 64, false><<<grid, 256, 0, s>>>(items, A, B0, B1, C, Add, idx, nrhs, b);
  }
}

template <typename TV>
void launch_split_reduce(const SplitRed* d, int n, const TV* P, TV* C, const TV* Add, const int* idx, int nrhs,
                         double beta, cudaStream_t s) {
  if (n <= 0) return;
  dim3 grid(grid_for((long long)ROWS_HINT * nrhs, 256, 16), n);
  split_reduce_kernel<TV><<<grid, 256, 0, s>>>(d, P, C, Add, idx, nrhs, (TV)beta);
}

void launch_row_combine(const int* tab, int n, double* dst, const double* A, const double* B, int nrhs,
                        cudaStream_t s) {
  if (n <= 0) return;
  row_combine_kernel<<<grid_for((long long)n * nrhs), 256, 0, s>>>(tab, n, dst, A, B, nrhs);
}

template <typename TV>
void launch_up_gather(const UpGather* g, int n, int maxrows, const TV* V, TV* Vout, TV* dbuf,
                      const double* rho, const int* idx, int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  dim3 grid(grid_for((long long)maxrows * nrhs, 256, 64), n);
  up_gather_kernel<TV><<<grid, 256, 0, s>>>(g, V, Vout, dbuf, rho, idx, nrhs);
}

template <typename TV>
void launch_down_scatter(const DownScatter* g, int n, int maxrows, TV* VB, const TV* dbar, double* rhobar,
                         const int* idx, int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  dim3 grid(grid_for((long long)maxrows * nrhs, 256, 64), n);
  down_scatter_kernel<TV><<<grid, 256, 0, s>>>(g, VB, dbar, rhobar, idx, nrhs);
}

template <typename TV>
void launch_scatter_rows(const double* src, const int* idx, int n, TV* dst, int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  scatter_rows_kernel<TV><<<grid_for((long long)n * nrhs), 256, 0, s>>>(src, idx, n, dst, nrhs);
}

template <typename TI, typename TO>
void launch_convert(const TI* src, TO* dst, long long n, double scale, cudaStream_t s) {
  if (n <= 0) return;
  convert_kernel<TI, TO><<<grid_for(n), 256, 0, s>>>(src, dst, n, scale);
}

template <typename TI>
void launch_axpy_to_f64(const TI* x, double* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  axpy_kernel<TI><<<grid_for(n), 256, 0, s>>>(x, y, n);
}

__global__ void fill_kernel(double* __restrict__ x, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}
void ensure_smem(const void* kernel, size_t bytes) {
  // raised whatever the size: with its static shared memory a kernel can pass the default
  // 48 KB limit with less than 48 KB of dynamic shared memory
  if (bytes == 0) return;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = done[{kernel, dev}];
  if (bytes > cur) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cur = bytes;
  }
}

int device_sms() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm > 0 ? nsm : 1;
}

void launch_fill(double* x, long long n, double v, cudaStream_t s) {
  if (n <= 0) return;
  fill_kernel<<<grid_for(n, 256, 1024), 256, 0, s>>>(x, n, v);
}

void launch_axpy_measure(const float* x, double* y, long long n, double* out, cudaStream_t s) {
  if (n <= 0) return;
  axpy_measure_kernel<<<grid_for(n, 256, 1216), 256, 0, s>>>(x, y, n, reinterpret_cast<unsigned long long*>(out));
}
void launch_absmax(const double* x, long long n, double* out, cudaStream_t s) {
  absmax_kernel<double><<<grid_for(n, 256, 1024), 256, 0, s>>>(x, n, reinterpret_cast<unsigned long long*>(out));
}
void launch_absmax_f32(const float* x, long long n, double* out, cudaStream_t s) {
  absmax_kernel<float><<<grid_for(n, 256, 1024), 256, 0, s>>>(x, n, reinterpret_cast<unsigned long long*>(out));
}

template <typename TV>
void launch_gather_reduce(const int* tab, int nnodes, const TV* src, TV* dst, int nrhs, int accumulate,
                          cudaStream_t s) {
  if (nnodes <= 0) return;
  gather_reduce_kernel<TV><<<grid_for((long long)nnodes * nrhs), 256, 0, s>>>(tab, nnodes, src, dst, nrhs, accumulate);
}

void launch_jump_residual(const int* pairs, int npairs, int q, const double* vflux, double* rho_out, int nrhs,
                          cudaStream_t s) {
  if (npairs <= 0) return;
  jump_residual_kernel<<<grid_for((long long)npairs * q * nrhs), 256, 0, s>>>(pairs, npairs, q, vflux, rho_out, nrhs);
}

template void launch_gemm_items<double, double>(const GemmItem*, int, int, int, const double*, const double*,
                                                const double*, double*, const double*, const int*, int, double,
                                                cudaStream_t, const GemmCtx&);
template void launch_gemm_items<float, float>(const GemmItem*, int, int, int, const float*, const float*,
                                              const float*, float*, const float*, const int*, int, double,
                                              cudaStream_t, const GemmCtx&);
template void launch_split_reduce<double>(const SplitRed*, int, const double*, double*, const double*, const int*,
                                          int, double, cudaStream_t);
template void launch_split_reduce<float>(const SplitRed*, int, const float*, float*, const float*, const int*, int,
                                         double, cudaStream_t);
template void launch_up_gather<double>(const UpGather*, int, int, const double*, double*, double*, const double*,
                                       const int*, int, cudaStream_t);
template void launch_up_gather<float>(const UpGather*, int, int, const float*, float*, float*, const double*,
                                      const int*, int, cudaStream_t);
template void launch_down_scatter<double>(const DownScatter*, int, int, double*, const double*, double*,
                                          const int*, int, cudaStream_t);
template void launch_scatter_rows<double>(const double*, const int*, int, double*, int, cudaStream_t);
template void launch_scatter_rows<float>(const double*, const int*, int, float*, int, cudaStream_t);
template void launch_convert<double, float>(const double*, float*, long long, double, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, long long, double, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, long long, double, cudaStream_t);
template void launch_axpy_to_f64<float>(const float*, double*, long long, cudaStream_t);
template void launch_axpy_to_f64<double>(const double*, double*, long long, cudaStream_t);
template void launch_gather_reduce<double>(const int*, int, const double*, double*, int, int, cudaStream_t);

}  // namespace hps
