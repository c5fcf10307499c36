// FP64 batched gathered products on the tcgen05 tensor cores by exact digit slicing.
//
// The solve and the adjoint (Algorithm 2 and its transpose) apply stored dense operators
// to blocks of gathered vectors: C_rows = beta C_rows + A_item B_gathered (+ Add), one
// GemmItem per block of at most 64 operator rows.  In FP64 on GB300 these products are
// bound by the FP64 FFMA pipe.  Here every row of A (over the item's whole K) is scaled by
// the power of two 2^e_r of its largest entry and written as 9 signed base-128 digits,
// A_rk = 2^e_r sum_s a_s 2^(1-7s) with |a_s| <= 64, every column of B likewise with 2^f_n and
// digits b_t.  Digits are integers exactly representable in bf16; a digit product is at
// most 2^12 in magnitude, so a diagonal d = s + t of the digit-pair products summed over
// K <= 448 stays below 2^24 and the FP32 accumulation of the tensor core is exact.  The
// digit pairs with s + t <= 10 accumulate diagonal d in its own TMEM columns, 10 tcgen05.mma
// per K step of 16 (one per A digit plane against the B planes side by side); the epilogue
// combines the 9 diagonals exactly in integers and rounds once to FP64.  The pairs left out
// weigh below about K 2^-63 max|A_r| max|B_n|, and every digit of A and B is exact to 2^-62
// of its row (column) maximum: the product agrees with FP64 arithmetic to its normwise
// rounding level.
//
// Work unit: one item (<= 64 rows; MMA M = 128, rows 64..127 are padding that no epilogue
// reads) and 32 right-hand sides (MMA N = 32).  A first kernel writes every unit's 32 column
// exponents (and its 64 row exponents unless the operator's digits are cached: the
// operators are fixed after the build, so a product set can keep their digit planes, formed
// once by gemm_digits_kernel; a set of items that gathers the same vector rows, such as
// the Schur products of the blocked merge elimination, can likewise keep the vectors'
// digit planes, formed once by gemm_bdigits_kernel, and then needs no exponent pass and
// forms no digits at all).  The product kernel's roles (17 warps, one CTA per SM looping
// over the units):
//   warps 0, 1, 4, 5   epilogue: TMEM lanes 0..63 (warp w reads lane quarter w % 4), 16
//              right-hand sides per thread, copied from TMEM to padded shared-memory rows
//              (which frees TMEM for the next unit) and recombined from there, four at a
//              time; beta, Add, scatter;
//   the other warps but 16  producers (12 warps, spread over the four SM sub-partitions):
//              per K step of 16 the digit planes of A (64 x 16, or one bulk copy of the
//              cached planes) and B (32 x 16, or one bulk copy of cached planes), one task
//              of 4 consecutive k per thread, four stages deep;
//   warp 16    one thread issues the digit-pair products of each K step into TMEM.
// Handoffs are mbarriers with bounded waits; a timeout stops every role (status -1).
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda_bf16.h>

#include "hps_internal.h"

namespace hps {

namespace {

constexpr int GM = 128;     // MMA rows (item rows 0..63, the rest padding)
constexpr int GR = 64;      // item rows
constexpr int GN = 32;      // right-hand sides per unit
constexpr int GS = 9;       // digits per entry
constexpr int GD = 9;       // kept diagonals d = 2 .. 10
constexpr int GKMAX = 448;  // longest K with exact FP32 diagonal sums
constexpr int GST = 4;      // K-step stages
constexpr int G_THREADS = 544;  // 17 warps (5 on one SM sub-partition: at most 96 registers)
constexpr int G_PROD = 384;    // producer threads (12 warps, one task each)
constexpr int G_EPI = 128;     // epilogue threads (4 warps)
constexpr int G_MMA_WARP = 16;
constexpr long long G_WAIT = 1ll << 26;

// Stage of one K step.  The A planes hold the item's 64 rows (2048 bytes each); a product
// (M = 128) reads 128 rows from a plane's start, so its rows 64..127 are the next plane's
// (or the B planes') bytes: bf16 digits, accumulated into TMEM lanes 64..127, which no
// epilogue reads.  Rows are independent in the product, so lanes 0..63 stay exact.
constexpr int GAPL = GR * 32;          // bytes per A plane
constexpr int GASTEP = GS * GAPL;      // bytes of a K step's A planes (cached operators)
struct GStage {
  unsigned char A[GS][GAPL];     // K-major planes, 64 rows x 16 k
  unsigned char B[GS][GN * 32];  // 32 columns x 16 k
};

constexpr int GBSTEP = GS * GN * 32;  // bytes of a K step's B planes (cached vectors)
constexpr int GSC = GR + GN;  // exponents per unit: 64 rows, then 32 columns
constexpr int GTASK = (GR + GN) * 4;  // producer tasks per K step: 4 consecutive k of a row or column
constexpr int GPF = 2;                // K steps the entry copies run ahead of the digits
constexpr int GRAW = GPF + 1;         // raw entry slots

constexpr int GSTG = GR * 33;  // epilogue staging: one unit's diagonal sums, row pitch 33 words

struct GShared {
  GStage st[GST];
  double raw[GRAW][GTASK][4];  // the entries of a K step, per producer task
  uint32_t stg[GD][GSTG];      // the epilogue's copy of the unit's TMEM accumulators
  unsigned long long sfull[GST], sfree[GST], tfull, tfree, mdone;
  unsigned int tmem_base;
  int abort_flag;
};
static_assert(sizeof(GShared) + 1024 <= 232448, "shared memory of the product kernel");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// byte offset of (row, k) in a K-major plane with 16 k per row (8-row x 16-byte core
// matrices, LBO 128 bytes along K, SBO 256 bytes between row groups)
__device__ __forceinline__ int kmaj(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

__device__ __forceinline__ void mb_init(unsigned long long* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mb_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned long long* b, int parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity; false on timeout or abort
__device__ __forceinline__ bool mb_wait(unsigned long long* b, int parity, volatile int* abort_flag, int* status) {
  for (long long it = 0; it < G_WAIT; ++it) {
    if (mb_try(b, parity)) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  if (status) atomicCAS(status, 0, -1);
  return false;
}
// bounded wait that ignores the abort flag (drains the role's own operations at exit)
__device__ __forceinline__ void mb_drain(unsigned long long* b, int parity) {
  for (long long it = 0; it < G_WAIT; ++it)
    if (mb_try(b, parity)) return;
}
__device__ __forceinline__ void mb_expect_arrive(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// warp-uniform bounded wait: lane 0 waits, the result is broadcast
__device__ __forceinline__ bool warp_wait(unsigned long long* b, int parity, volatile int* abort_flag, int* status) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mb_wait(b, parity, abort_flag, status) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ int map_row(const int* __restrict__ idx, int base_or_off, int row_base, int k) {
  return base_or_off < 0 ? row_base + k : row_base + idx[base_or_off + k];
}

// bf16 bits of a small integer |a| <= 2^8 exactly: 1.5 2^23 + a is an FP32 number with unit
// spacing, and a value with at most 8 significant bits keeps them in the upper half.
__device__ __forceinline__ uint32_t bf16_of_int(int a) {
  return __float_as_uint(__int_as_float(0x4B400000 + a) - 12582912.0f) >> 16;
}

// Fixed-point form of x against the row (column) exponent emax: X = x 2^(62 - (emax - 1022))
// exactly (the 53-bit significand shifted, rounded when shifted right), |X| < 2^62.
__device__ __forceinline__ long long fixed62(double x, int emax) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long X = 0;
  if (E > 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = E - emax + 9;
    if (sh >= 0) X = m << sh;
    else if (sh > -60) X = (m + (1ll << (-sh - 1))) >> (-sh);
    if (bits < 0) X = -X;
  }
  return X;
}

// The 9 balanced base-128 digit planes of 4 consecutive k of one row (column): one 8-byte
// store per plane.  Plane s - 1 holds a_s (a_1 the most significant).  With
// X = sum_(i<8) a'_i 2^(7i) + a_top 2^56 and a'_i in [-64, 63], Y = X + 64 sum_(i<8) 2^(7i)
// has the base-128 digits a'_i + 64 in its low 56 bits and a_top in the bits above, so
// every digit is one bit-field extraction.
__device__ __forceinline__ void write_digits4(const double* v, int emax, unsigned char* plane0, int plane_bytes,
                                             int off) {
  constexpr long long kOff = 64ll * ((1ll << 56) - 1) / 127;  // 64 in each of the 8 low digits
  long long Y[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) Y[q] = fixed62(v[q], emax) + kOff;
  // the most significant digit (plane 0)
  {
    int a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = (int)(Y[q] >> 56);
    *reinterpret_cast<uint2*>(plane0 + off) = make_uint2(bf16_of_int(a[0]) | (bf16_of_int(a[1]) << 16),
                                                         bf16_of_int(a[2]) | (bf16_of_int(a[3]) << 16));
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {  // digit a'_i -> plane 8 - i
    int a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = (int)((unsigned long long)Y[q] >> (7 * i) & 127ull) - 64;
    *reinterpret_cast<uint2*>(plane0 + (GS - 1 - i) * plane_bytes + off) =
        make_uint2(bf16_of_int(a[0]) | (bf16_of_int(a[1]) << 16), bf16_of_int(a[2]) | (bf16_of_int(a[3]) << 16));
  }
}

// zero digits of 4 k of one row (a row past the item)
__device__ __forceinline__ void zero_digits4(unsigned char* plane0, int plane_bytes, int off) {
#pragma unroll
  for (int s = 0; s < GS; ++s) *reinterpret_cast<uint2*>(plane0 + s * plane_bytes + off) = make_uint2(0u, 0u);
}

// The product entry from its 9 diagonal sums S_2 .. S_10, each given as the FP32 bit
// pattern y_d of S_d + 1.5 2^23 (exact, |S_d| < 2^24):
//   sum_k A_rk B_kn = 2^(er + ec - 2112) I,  I = sum_d S_d 2^(7 (10 - d)),  |I| < 2^81,
// assembled exactly and rounded once to FP64 with integer operations: to nearest, ties
// away from zero.  Results below the normal range flush to zero.
__device__ __forceinline__ double recombine9(const uint32_t* v, int er, int ec) {
  long long y[GD];
#pragma unroll
  for (int d = 0; d < GD; ++d) y[d] = (long long)__float_as_int(__uint_as_float(v[d]) + 12582912.0f);
  constexpr long long K0 = 0x4B400000ll;
  // I = H 2^35 + L with the biases removed
  const long long H = (y[0] << 21) + (y[1] << 14) + (y[2] << 7) + y[3] - K0 * ((1ll << 21) + (1ll << 14) + (1ll << 7) + 1);
  const long long L = (y[4] << 28) + (y[5] << 21) + (y[6] << 14) + (y[7] << 7) + y[8] -
                      K0 * ((1ll << 28) + (1ll << 21) + (1ll << 14) + (1ll << 7) + 1);
  const long long T = (H << 3) + (L >> 32);  // I = T 2^32 + u, 0 <= u < 2^32
  const unsigned int u = (unsigned int)L;
  const bool neg = T < 0;
  const unsigned long long A = neg ? (unsigned long long)(-T) - (u != 0u ? 1ull : 0ull) : (unsigned long long)T;
  const unsigned int B = neg ? 0u - u : u;
  // W: the leading 64 bits of |I| when A >= 2^32 (B's top bits shifted in below), else all
  // of |I|; N: W normalised to a leading bit 63.  Bits shifted out lie below the rounding
  // position and cannot change a round-half-up decision.
  const bool big = (A >> 32) != 0;
  const unsigned long long W = big ? A : ((A << 32) | B);
  if (W == 0) return 0.0;
  const int z = __clzll((long long)W);  // 14 .. 31 when big
  unsigned long long N = W << z;
  if (big) N |= (unsigned long long)(B >> (32 - z));
  const int top = (big ? 95 : 63) - z;
  const unsigned long long mant = (N >> 11) + ((N >> 10) & 1ull);  // 2^52 .. 2^53
  const int E = top + er + ec - 1089;
  if (E <= 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)neg << 63;
  if (E >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sgn + ((unsigned long long)(E - 1) << 52) + mant));
}

// element k of column n (< nrhs) of the item's gathered B
__device__ __forceinline__ double b_at(const GemmItem& it, const double* __restrict__ B0, const double* __restrict__ B1,
                                       const int* __restrict__ idx, int k, int n, int nrhs) {
  return k < it.kseg ? B0[(long long)map_row(idx, it.b0_idx, it.b0_row, k) * nrhs + n]
                     : B1[(long long)map_row(idx, it.b1_idx, it.b1_row, k - it.kseg) * nrhs + n];
}

template <bool TRANS>
__device__ __forceinline__ double a_at(const GemmItem& it, const double* __restrict__ A, int r, int k) {
  return TRANS ? A[it.a_off + (long long)k * it.lda + r] : A[it.a_off + (long long)r * it.lda + k];
}

// Exponent (biased) of the largest entry of every row of A and every column of B, per
// unit: scales[u][0 .. 63] rows, scales[u][64 .. 95] columns (0 for rows or columns past
// the item).  256 threads: A rows 4 threads each (k phases), B columns 8 threads each.
template <bool TRANS>
__global__ void __launch_bounds__(256) gemm_scales_kernel(const GemmItem* __restrict__ items,
                                                          const double* __restrict__ A,
                                                          const double* __restrict__ B0,
                                                          const double* __restrict__ B1,
                                                          const int* __restrict__ idx, int nrhs,
                                                          int* __restrict__ scales, int rows) {
  const int nnb = (nrhs + GN - 1) / GN;
  const long long u = blockIdx.x;
  const GemmItem it = items[u / nnb];
  const int n0 = (int)(u % nnb) * GN;
  const int t = threadIdx.x;
  __shared__ int part[256 + 256];
  {
    // A: row r = t % 64 (trans: consecutive threads read consecutive addresses), or with
    // non-transposed storage row r = t / 4 with the 4 threads of a row on interleaved k
    int r, ph;
    if (TRANS) { r = t & 63; ph = t >> 6; }
    else { r = t >> 2; ph = t & 3; }
    int m = 0;
    if (rows && r < it.M) {
#pragma unroll 4
      for (int k = ph; k < it.K; k += 4) m = max(m, bexp(a_at<TRANS>(it, A, r, k)));
    }
    part[TRANS ? ph * 64 + r : r * 4 + ph] = m;
  }
  {
    // B: column n = t % 32, k phase t / 32
    const int nl = t & 31, ph = t >> 5, n = n0 + nl;
    int m = 0;
    if (n < nrhs) {
#pragma unroll 4
      for (int k = ph; k < it.K; k += 8) m = max(m, bexp(b_at(it, B0, B1, idx, k, n, nrhs)));
    }
    part[256 + ph * 32 + nl] = m;
  }
  __syncthreads();
  int* out = scales + u * GSC;
  if (t < GR) {
    int m = 0;
    for (int ph = 0; ph < 4; ++ph) m = max(m, TRANS ? part[ph * 64 + t] : part[t * 4 + ph]);
    out[t] = m;
  } else if (t < GR + GN) {
    const int nl = t - GR;
    int m = 0;
    for (int ph = 0; ph < 8; ++ph) m = max(m, part[256 + ph * 32 + nl]);
    out[t] = m;
  }
}

// The operator's digit planes of every K step of one item (one block per item), in the
// stage layout, at adig + astep[item] * GASTEP, and its 64 row exponents at aer[item * 64],
// of sgn A (sgn = +-1, exact).  Operators do not change between solves, so their digits are
// formed once.
template <bool TRANS>
__global__ void __launch_bounds__(256) gemm_digits_kernel(const GemmItem* __restrict__ items,
                                                          const double* __restrict__ A,
                                                          const long long* __restrict__ astep,
                                                          unsigned char* __restrict__ adig, int* __restrict__ aer,
                                                          double sgn) {
  const long long item = blockIdx.x;
  const GemmItem it = items[item];
  const int t = threadIdx.x;
  __shared__ int part[256];
  __shared__ int er[GR];
  {
    int r, ph;
    if (TRANS) { r = t & 63; ph = t >> 6; }
    else { r = t >> 2; ph = t & 3; }
    int m = 0;
    if (r < it.M) {
#pragma unroll 4
      for (int k = ph; k < it.K; k += 4) m = max(m, bexp(a_at<TRANS>(it, A, r, k)));
    }
    part[TRANS ? ph * 64 + r : r * 4 + ph] = m;
  }
  __syncthreads();
  if (t < GR) {
    int m = 0;
    for (int ph = 0; ph < 4; ++ph) m = max(m, TRANS ? part[ph * 64 + t] : part[t * 4 + ph]);
    er[t] = m;
    aer[item * GR + t] = m;
  }
  __syncthreads();
  unsigned char* dst = adig + astep[item] * GASTEP;
  const int nk = (it.K + 15) >> 4;
  const int row = t >> 2, kg = (t & 3) * 4;  // 64 rows x 4 groups of 4 k
  for (int c = 0; c < nk; ++c) {
    unsigned char* pl = dst + (long long)c * GASTEP;
    if (row >= it.M) {
      zero_digits4(pl, GAPL, kmaj(row, kg));
    } else {
      double v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = c * 16 + kg + q;
        v[q] = k < it.K ? sgn * a_at<TRANS>(it, A, row, k) : 0.0;
      }
      write_digits4(v, er[row], pl, GAPL, kmaj(row, kg));
    }
  }
}

// The vectors' digit planes of one group (blockIdx.y) and column block (blockIdx.x): the 32
// columns' exponents over the group's K rows, then every K step's planes in the stage
// layout, exactly as the product kernel's producers would form them.
__global__ void __launch_bounds__(256) gemm_bdigits_kernel(const BGroup* __restrict__ groups,
                                                           const double* __restrict__ B0,
                                                           const int* __restrict__ idx, int nrhs,
                                                           unsigned char* __restrict__ bdig, int* __restrict__ bex) {
  const BGroup g = groups[blockIdx.y];
  const int nb = blockIdx.x, t = threadIdx.x;
  __shared__ int part[256];
  __shared__ int ec[GN];
  {
    const int nl = t & 31, ph = t >> 5, n = nb * GN + nl;
    int m = 0;
    if (n < nrhs) {
#pragma unroll 4
      for (int k = ph; k < g.K; k += 8) m = max(m, bexp(B0[(long long)(g.b0_row + idx[g.b0_idx + k]) * nrhs + n]));
    }
    part[ph * 32 + nl] = m;
  }
  __syncthreads();
  if (t < GN) {
    int m = 0;
    for (int ph = 0; ph < 8; ++ph) m = max(m, part[ph * 32 + t]);
    ec[t] = m;
    bex[g.ex0 + nb * GN + t] = m;
  }
  __syncthreads();
  const int nk = (g.K + 15) >> 4;
  const int task = t & 127, col = task >> 2, kg = (task & 3) * 4, n = nb * GN + col;
  for (int c = t >> 7; c < nk; c += 2) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = c * 16 + kg + q;
      v[q] = (n < nrhs && k < g.K) ? B0[(long long)(g.b0_row + idx[g.b0_idx + k]) * nrhs + n] : 0.0;
    }
    write_digits4(v, ec[col], bdig + (g.blk0 + (long long)nb * nk + c) * GBSTEP, GN * 32, kmaj(col, kg));
  }
}

template <bool TRANS>
__global__ void __launch_bounds__(G_THREADS, 1) gemm_tc_kernel(const GemmItem* __restrict__ items, int nitems,
                                                                const double* __restrict__ A,
                                                                const double* __restrict__ B0,
                                                                const double* __restrict__ B1, double* __restrict__ C,
                                                                const double* __restrict__ Add,
                                                                const int* __restrict__ idx, int nrhs, double beta,
                                                                const int* __restrict__ scales,
                                                                const unsigned char* __restrict__ adig,
                                                                const long long* __restrict__ astep,
                                                                const int* __restrict__ aer,
                                                                const unsigned char* __restrict__ bdig,
                                                                const long long* __restrict__ bblk,
                                                                const int* __restrict__ bexo,
                                                                const int* __restrict__ bex,
                                                                int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char g_raw[];
  GShared& sh = *reinterpret_cast<GShared*>(g_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nnb = (nrhs + GN - 1) / GN;
  const long long total = (long long)nitems * nnb;
  // cached operator digits (adig): the producers form only the vectors' digits (threads
  // 256 .. 383) and one thread copies each K step's A planes
  const bool cached = adig != nullptr;
  const bool bcached = cached && bdig != nullptr;  // both operands' digits cached: copies only
  if (tid == 0) {
    for (int b = 0; b < GST; ++b) {
      mb_init(&sh.sfull[b], bcached ? 1 : (cached ? GN * 4 + 1 : G_PROD));
      mb_init(&sh.sfree[b], 1);
    }
    mb_init(&sh.tfull, 1);
    mb_init(&sh.tfree, G_EPI);
    mb_init(&sh.mdone, 1);
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == G_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sh.tmem_base;
  volatile int* abort_flag = &sh.abort_flag;
  const int q4 = warp & 3;

  if (warp == G_MMA_WARP) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      // kind::f16 with bf16 A and B, FP32 accumulators, M = 128; N is set per product
      const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GM >> 4) << 24);
      long long ks = 0;  // K steps issued so far (stage ks % GST)
      int nu = 0;
      bool stop = false;
      for (long long u = blockIdx.x; u < total && !stop; u += gridDim.x, ++nu) {
        const GemmItem it = items[u / nnb];
        const int nk = (it.K + 15) >> 4;
        if (nu >= 1 && !mb_wait(&sh.tfree, (nu - 1) & 1, abort_flag, status)) break;
        for (int c = 0; c < nk; ++c, ++ks) {
          const int st = (int)(ks % GST);
          if (!mb_wait(&sh.sfull[st], (int)((ks / GST) & 1), abort_flag, status)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = smem_u32(sh.st[st].A[0]), b0 = smem_u32(sh.st[st].B[0]);
          // one product per A digit plane s against the B planes t = 1 .. 10 - s side by side
          // (contiguous in the K-major layout: N = 32 (10 - s), at most 256 per instruction),
          // written from TMEM column 32 (s - 1): block t lands on diagonal s + t
#pragma unroll 1
          for (int sa = 1; sa <= GS; ++sa) {
            const int nt = GD + 1 - sa;
#pragma unroll 1
            for (int t0 = 1; t0 <= nt; t0 += 8) {
              const int cnt = min(8, nt - t0 + 1);
              const uint64_t ad = umma_desc(a0 + (sa - 1) * GAPL, 128, 256);
              const uint64_t bd = umma_desc(b0 + (t0 - 1) * (GN * 32), 128, 256);
              const uint32_t idesc = idesc0 | ((uint32_t)((GN * cnt) >> 3) << 17);
              const uint32_t acc = (c > 0 || sa > 1) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                      tmem + (uint32_t)((sa - 1 + t0 - 1) * GN)),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&sh.sfree[st])));
        }
        if (stop) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&sh.tfull)));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&sh.mdone)));
      mb_drain(&sh.mdone, 0);
    }
  } else if (!(warp < 8 && q4 < 2)) {
    // ---------------- producers: warps 2, 3, 6, 7, 8 .. 15 -> producer index 0 .. 11.
    // Thread pt owns task pt (4 consecutive k of one row of A or column of B) of every K
    // step; it copies the entries GPF steps ahead (asynchronously, into its own slot) and
    // turns them into digits when their step comes, so no thread waits on memory for the
    // step it is working on.
    const int pw = warp < 8 ? (warp >> 2) * 2 + (q4 - 2) : warp - 4;
    const int pt = pw * 32 + lane;
    const int ntask = pt + G_PROD < GTASK ? 2 : 1;  // 1 while G_PROD = GTASK
    if (cached && (bcached || pt < GR * 4)) {
      // the operator's digit planes (and with bcached the vectors') come from the caches:
      // thread 0 copies each K step's planes (bulk copies) and arms the stage's barrier
      // with their bytes
      if (pt == 0) {
        long long ks = 0;
        bool stop = false;
        for (long long u = blockIdx.x; u < total && !stop; u += gridDim.x) {
          const long long item = u / nnb;
          const int nk = (items[item].K + 15) >> 4;
          const unsigned char* src = adig + astep[item] * GASTEP;
          const unsigned char* bsrc = bcached ? bdig + (bblk[item] + (u % nnb) * nk) * GBSTEP : nullptr;
          for (int c = 0; c < nk; ++c, ++ks) {
            const int st = (int)(ks % GST);
            if (ks >= GST && !mb_wait(&sh.sfree[st], (int)((ks / GST) - 1) & 1, abort_flag, status)) {
              stop = true;
              break;
            }
            mb_expect_arrive(&sh.sfull[st], bcached ? GASTEP + GBSTEP : GASTEP);
            bulk_load(sh.st[st].A[0], src + (long long)c * GASTEP, GASTEP, &sh.sfull[st]);
            if (bcached) bulk_load(sh.st[st].B[0], bsrc + (long long)c * GBSTEP, GBSTEP, &sh.sfull[st]);
          }
        }
        // the copies issued have landed before the block exits
        for (int b = 0; b < GST; ++b) {
          const long long n = ks > b ? (ks - 1 - b) / GST + 1 : 0;  // copies armed on stage b
          if (n > 0) mb_drain(&sh.sfull[b], (int)((n - 1) & 1));
        }
      }
    } else {
    // step iterators over (unit, K step) in this block's order: cu/cc current, pu/pc copy
    long long cu = blockIdx.x, pu = blockIdx.x;
    int cc = 0, pc = 0;
    GemmItem cit, pit;
    if (cu < total) cit = pit = items[cu / nnb];
    auto advance = [&](long long& uu, int& c, GemmItem& it) {
      if (++c >= ((it.K + 15) >> 4)) {
        c = 0;
        uu += gridDim.x;
        if (uu < total) it = items[uu / nnb];
      }
    };
    auto issue = [&](long long uu, int c, const GemmItem& it, int slot) {
      if (uu < total) {
        const int n0 = (int)(uu % nnb) * GN, k0 = c * 16;
        for (int j = 0; j < ntask; ++j) {
          const int task = pt + j * G_PROD, line = task >> 2, kg = (task & 3) * 4;
          double* dst = sh.raw[slot][task];
          if (line < GR) {
            if (line >= it.M) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int k = k0 + kg + q;
              if (k < it.K) {
                if (TRANS) cp_async8(dst + q, A + it.a_off + (long long)k * it.lda + line);
                else cp_async8(dst + q, A + it.a_off + (long long)line * it.lda + k);
              } else {
                dst[q] = 0.0;
              }
            }
          } else {
            const int n = n0 + line - GR;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int k = k0 + kg + q;
              if (n < nrhs && k < it.K) {
                const double* src = k < it.kseg
                                        ? B0 + (long long)map_row(idx, it.b0_idx, it.b0_row, k) * nrhs + n
                                        : B1 + (long long)map_row(idx, it.b1_idx, it.b1_row, k - it.kseg) * nrhs + n;
                cp_async8(dst + q, src);
              } else {
                dst[q] = 0.0;
              }
            }
          }
        }
      }
      cp_commit();  // one group per step, empty past the end, so that the count stays aligned
    };
    for (int i = 0; i < GPF; ++i) {
      issue(pu, pc, pit, i % GRAW);
      if (pu < total) advance(pu, pc, pit);
    }
    long long ks = 0;
    while (cu < total) {
      cp_wait<GPF - 1>();  // this thread's entries of step ks have landed
      const int st = (int)(ks % GST), slot = (int)(ks % GRAW);
      if (ks >= GST && !warp_wait(&sh.sfree[st], (int)((ks / GST) - 1) & 1, abort_flag, status)) break;
      const int* sc = scales + cu * GSC;
      for (int j = 0; j < ntask; ++j) {
        const int task = pt + j * G_PROD, line = task >> 2, kg = (task & 3) * 4;
        const double* v = sh.raw[slot][task];
        if (line < GR) {
          if (line >= cit.M) zero_digits4(sh.st[st].A[0], GAPL, kmaj(line, kg));
          else write_digits4(v, sc[line], sh.st[st].A[0], GAPL, kmaj(line, kg));
        } else {
          write_digits4(v, sc[line], sh.st[st].B[0], GN * 32, kmaj(line - GR, kg));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mb_arrive(&sh.sfull[st]);
      // the copies of step ks + GPF (their index lookups may wait on memory) after this
      // step's digits are out, off the products' critical path
      issue(pu, pc, pit, (int)((ks + GPF) % GRAW));
      if (pu < total) advance(pu, pc, pit);
      advance(cu, cc, cit);
      ++ks;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // copies still in flight land before exit
    }
  } else {
    // ---------------- epilogue: warps 0, 1, 4, 5; row = 32 (w % 4) + lane, right-hand
    // sides 16 g .. 16 g + 15 with g = w / 4.  The unit's 9 diagonal sums are first copied
    // from TMEM to this thread's shared-memory row (pitch 33 words: the lanes' rows fall in
    // distinct banks), which frees TMEM for the next unit's products at once; the exact
    // recombination then runs from shared memory while those products are issued.
    const int row = q4 * 32 + lane, g = warp >> 2;
    int nu = 0;
    for (long long u = blockIdx.x; u < total; u += gridDim.x, ++nu) {
      const GemmItem it = items[u / nnb];
      const int n0 = (int)(u % nnb) * GN;
      const int* sc = scales ? scales + u * GSC : nullptr;  // none when both operands are cached
      const int er = cached ? aer[(u / nnb) * GR + row] : sc[row];
      if (!warp_wait(&sh.tfull, nu & 1, abort_flag, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
      for (int d = 0; d < GD; ++d) {
        const uint32_t addr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(d * GN + 16 * g);
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        uint32_t* dst = sh.stg[d] + row * 33 + 16 * g;
#pragma unroll
        for (int j = 0; j < 16; ++j) dst[j] = v[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      mb_arrive(&sh.tfree);  // TMEM read: the next unit's products may start
      if (row >= it.M) continue;
      const long long crow = (long long)map_row(idx, it.c_idx, it.c_row, row) * nrhs;
#pragma unroll 1
      for (int hh = 0; hh < 4; ++hh) {
        const int jb = 16 * g + 4 * hh;
        int ec[4];
        double cv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // the group's loads first: their latency overlaps the recombination
          const int n = n0 + jb + j;
          ec[j] = bcached ? bex[bexo[u / nnb] + n] : sc[GR + jb + j];
          cv[j] = (beta != 0.0 && n < nrhs) ? C[crow + n] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = n0 + jb + j;
          if (n >= nrhs) continue;
          uint32_t dj[GD];
#pragma unroll
          for (int d = 0; d < GD; ++d) dj[d] = sh.stg[d][row * 33 + jb + j];
          double r = recombine9(dj, er, ec[j]);
          if (it.add_row >= 0) r += Add[(long long)(it.add_row + row) * nrhs + n];
          C[crow + n] = (beta != 0.0 ? beta * cv[j] : 0.0) + r;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == G_MMA_WARP) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace

bool gemm_tc_eligible(int maxK, int nrhs) { return maxK > 0 && maxK <= GKMAX && nrhs >= 8; }

long long gemm_tc_scale_bytes(long long units) { return units * GSC * (long long)sizeof(int); }

// Per-device set-up, once per device (outside stream capture): the SM count and the
// kernels' dynamic shared-memory limit, which is a property of the device's context.
namespace {
constexpr int kTcMaxDev = 64;
std::mutex g_tc_mu;
int g_tc_nsm[kTcMaxDev] = {0};
}  // namespace

static int gemm_tc_nsm() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTcMaxDev) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (!g_tc_nsm[dev]) {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(gemm_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GShared));
    cudaFuncSetAttribute(gemm_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GShared));
    if (cudaGetLastError() != cudaSuccess) return 0;
    g_tc_nsm[dev] = nsm > 0 ? nsm : 1;
  }
  return g_tc_nsm[dev];
}

void gemm_tc_prepare() { (void)gemm_tc_nsm(); }

bool launch_gemm_tc(const GemmItem* items, int nitems, int trans, const double* A, const double* B0,
                    const double* B1, double* C, const double* Add, const int* idx, int nrhs, double beta,
                    cudaStream_t s, const GemmCtx& cx) {
  if (nitems <= 0) return true;
  const long long units = (long long)nitems * ((nrhs + GN - 1) / GN);
  const GemmDigits* dg = cx.dg;
  const unsigned char* adig = dg ? dg->dig : nullptr;
  const long long* astep = dg ? dg->step : nullptr;
  const int* aer = dg ? dg->er : nullptr;
  // both operands' digits cached (and not transposed): no exponent pass, no scales buffer
  const bool bc = adig && dg->bdig && dg->bblk && dg->bexo && dg->bex && !trans;
  if (!bc && (!cx.tc_scales || units > cx.tc_units)) return false;
  const int nsm = gemm_tc_nsm();
  if (!nsm) return false;
  const int grid = (int)std::min<long long>(nsm, units);
  const int rows = adig ? 0 : 1;
  int* scales = bc ? nullptr : cx.tc_scales;
  const unsigned char* bdig = bc ? dg->bdig : nullptr;
  const long long* bblk = bc ? dg->bblk : nullptr;
  const int* bexo = bc ? dg->bexo : nullptr;
  const int* bex = bc ? dg->bex : nullptr;
  if (trans) {
    gemm_scales_kernel<true><<<(unsigned)units, 256, 0, s>>>(items, A, B0, B1, idx, nrhs, scales, rows);
    gemm_tc_kernel<true><<<grid, G_THREADS, sizeof(GShared), s>>>(items, nitems, A, B0, B1, C, Add, idx, nrhs, beta,
                                                                  scales, adig, astep, aer, nullptr, nullptr,
                                                                  nullptr, nullptr, cx.status);
  } else {
    if (!bc) gemm_scales_kernel<false><<<(unsigned)units, 256, 0, s>>>(items, A, B0, B1, idx, nrhs, scales, rows);
    gemm_tc_kernel<false><<<grid, G_THREADS, sizeof(GShared), s>>>(items, nitems, A, B0, B1, C, Add, idx, nrhs, beta,
                                                                   scales, adig, astep, aer, bdig, bblk, bexo, bex,
                                                                   cx.status);
  }
  return true;
}

long long gemm_tc_digit_bytes(long long steps) { return steps * GASTEP; }

long long gemm_tc_bdigit_bytes(long long blocks) { return blocks * GBSTEP; }

void launch_gemm_tc_bdigitize(const BGroup* groups, int ngroups, int ncb, const double* B0, const int* idx, int nrhs,
                              unsigned char* bdig, int* bex, cudaStream_t s) {
  if (ngroups <= 0 || ncb <= 0) return;
  gemm_bdigits_kernel<<<dim3((unsigned)ncb, (unsigned)ngroups), 256, 0, s>>>(groups, B0, idx, nrhs, bdig, bex);
}

void launch_gemm_tc_digitize(const GemmItem* items, int nitems, int trans, const double* A, const long long* astep,
                             unsigned char* adig, int* aer, cudaStream_t s, bool negate) {
  if (nitems <= 0) return;
  const double sgn = negate ? -1.0 : 1.0;
  if (trans) gemm_digits_kernel<true><<<(unsigned)nitems, 256, 0, s>>>(items, A, astep, adig, aer, sgn);
  else gemm_digits_kernel<false><<<(unsigned)nitems, 256, 0, s>>>(items, A, astep, adig, aer, sgn);
}

}  // namespace hps
