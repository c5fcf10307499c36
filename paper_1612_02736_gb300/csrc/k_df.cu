// Residual of the collocation system in double-float arithmetic.
//
// Iterative refinement (mixed precision) needs r = g - A u and the leaf fluxes to about
// 1e-14 of |A| |u|, not to full FP64: the residual is handed to an FP32 correction solve.
// GB300 runs FP32 FFMA 64 times faster than FP64 FFMA, so every value here is an unevaluated
// sum hi + lo of two floats (about 48 significant bits) and every operation is built from
// error-free transformations: Knuth's TwoSum for additions and the FMA-based TwoProduct
// (the product a*b and its exact rounding error fma(a, b, -a*b)) for multiplications.
// All float operations use the _rn intrinsics so that the compiler cannot contract or
// reorder them.  Inputs and outputs stay FP64 in memory.
#include <mutex>

#include "hps_internal.h"

namespace hps {

namespace {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

// The same splitting and joining with integer operations (GB300's FP64 pipe, which also
// runs the FP64 <-> FP32 conversions, does 2 operations per clock per SM; the integer pipe
// 64): hi is the significand rounded to 24 bits (half up), lo the exact remainder scaled by
// a power of two, for exponents where both are normal floats; zero, tiny, huge and
// non-finite values take the FP64 form above.
__device__ __forceinline__ df df_from_i(double x) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E < 949 || E > 1150) return df_from(x);
  const unsigned long long m = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long mh = (m + (1ull << 28)) >> 29;           // 2^23 .. 2^24
  const int rem = (int)((long long)m - (long long)(mh << 29));      // |rem| <= 2^28
  const unsigned sgn = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
  const unsigned hb = sgn | (((unsigned)(E - 896) << 23) + (unsigned)mh - (1u << 23));
  const float lo = __int2float_rn(rem) * __int_as_float((E - 948) << 23);
  return {__uint_as_float(hb), __uint_as_float(__float_as_uint(lo) ^ sgn)};
}
__device__ __forceinline__ double df_to_i(float hi, float lo) {
  const unsigned hb = __float_as_uint(hi), lb = __float_as_uint(lo);
  const int eh = (int)((hb >> 23) & 0xFF), el = (int)((lb >> 23) & 0xFF);
  if (eh < 40 || eh > 250) return (double)hi + (double)lo;
  long long t = (long long)((hb & 0x7FFFFF) | 0x800000) << 29;     // hi = t 2^(eh - 179)
  if (el > 0) {                                                      // lo in the same units
    const long long ml = (long long)((lb & 0x7FFFFF) | 0x800000);
    const int sh = el - eh + 29;
    long long v = 0;
    if (sh >= 0) v = ml << min(sh, 30);
    else if (sh > -40) v = (ml + (1ll << (-sh - 1))) >> (-sh);
    t += ((lb ^ hb) >> 31) ? -v : v;
  }
  int e = eh + 896;                                                  // biased exponent for t in [2^52, 2^53)
  if (t >= (1ll << 53)) {
    t = (t + 1) >> 1;
    ++e;
  } else if (t < (1ll << 52)) {
    t <<= 1;
    --e;
  }
  const unsigned long long bits =
      ((unsigned long long)(hb >> 31) << 63) | ((unsigned long long)e << 52) | ((unsigned long long)t & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// |a| >= |b|: s + e == a + b exactly.
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  const df u = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
// TwoProduct with FMA, plus the cross terms of the low parts.
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_fma(df acc, df a, df b) { return df_add(acc, df_mul(a, b)); }
// Accumulating multiply-add for dot products (15 instead of 27 float operations): the
// product's hi part joins acc.hi through TwoSum, every low-order term (the product's
// rounding error, its cross terms and acc.lo) is summed in plain float, then the pair is
// renormalised.  Its error is about 2^-48 (|acc| + |a b|), the bound of a sum of
// products in FP64-like arithmetic relative to the magnitudes of the terms.
__device__ __forceinline__ df df_fma_acc(df acc, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = two_sum(acc.hi, p);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, e)));
}

// ---------------------------------------------------------------------------------------
// Two right-hand sides at once: a pair of floats in one 64-bit register, operated on by the
// packed FP32 instructions (add/sub/mul/fma .rn.f32x2: each lane of the pair is rounded as
// the scalar operation would be), so that one instruction carries two double-float streams.
using f2 = unsigned long long;  // low half: first right-hand side

__device__ __forceinline__ f2 f2_pack(float a, float b) {
  return ((f2)__float_as_uint(b) << 32) | (f2)__float_as_uint(a);
}
__device__ __forceinline__ float f2_lo(f2 v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f2_hi(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// A double-float per right-hand side of a pair.
struct df2 {
  f2 h, l;
};
// A double-float constant shared by both right-hand sides, with its negated high part.
struct dfc {
  f2 h, l, nh;
};
__device__ __forceinline__ dfc dfc_of(float hi, float lo) { return {f2_pack(hi, hi), f2_pack(lo, lo), f2_pack(-hi, -hi)}; }
// Shared-memory entries of a pair or of a broadcast constant are 16 bytes {h, l} read as two
// 64-bit halves in one 128-bit load, straight into the packed registers.
using q2 = ulonglong2;
__device__ __forceinline__ df2 df2_ld(const q2* p) {
  const q2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void df2_st(q2* p, df2 v) { *p = make_ulonglong2(v.h, v.l); }
__device__ __forceinline__ dfc dfc_ld(const q2* p) {
  const q2 v = *p;
  return {v.x, v.y, f2_mul(v.x, f2_pack(-1.f, -1.f))};
}

// acc += a b, the compensated dot product of Ogita, Rump and Oishi (Dot2): the product's
// rounding error (TwoProduct by FMA) and the cross terms of the low parts, and the rounding
// error of adding the product to acc.h (Knuth's TwoSum), are collected in acc.l without
// renormalising; 12 packed instructions per pair of products.  The result acc.h + acc.l
// carries an error of about 2^-24 of itself plus n^2 2^-48 of the sum of |a b| (n terms),
// the accuracy of the sum computed in twice the working precision.
__device__ __forceinline__ void dot2_acc(df2& acc, const dfc& a, const df2& b) {
  const f2 np = f2_mul(a.nh, b.h);  // -p, p = fl(a.h b.h)
  f2 e = f2_fma(a.h, b.h, np);      // a.h b.h - p, exactly
  e = f2_fma(a.h, b.l, e);
  e = f2_fma(a.l, b.h, e);
  const f2 s = f2_sub(acc.h, np);   // acc.h + p
  const f2 bb = f2_sub(s, acc.h);
  const f2 t = f2_sub(f2_sub(acc.h, f2_sub(s, bb)), f2_add(np, bb));  // (acc.h + p) - s, exactly
  acc.h = s;
  acc.l = f2_add(acc.l, f2_add(t, e));
}
// the pair renormalised so that |l| <= ulp(h) / 2 (TwoSum: after heavy cancellation the
// collected low part can exceed the high one)
__device__ __forceinline__ df2 df2_norm(df2 a) {
  const f2 s = f2_add(a.h, a.l);
  const f2 bb = f2_sub(s, a.h);
  return {s, f2_add(f2_sub(a.h, f2_sub(s, bb)), f2_sub(a.l, bb))};
}
// a b for a constant a (TwoProduct and cross terms, renormalised)
__device__ __forceinline__ df2 df2_mul(const dfc& a, const df2& b) {
  const f2 np = f2_mul(a.nh, b.h);
  f2 e = f2_fma(a.h, b.h, np);
  e = f2_fma(a.h, b.l, e);
  e = f2_fma(a.l, b.h, e);
  const f2 s = f2_sub(e, np);  // p + e
  return {s, f2_sub(e, f2_add(s, np))};
}
__device__ __forceinline__ double df2_to0(df2 v) { return df_to_i(f2_lo(v.h), f2_lo(v.l)); }
__device__ __forceinline__ double df2_to1(df2 v) { return df_to_i(f2_hi(v.h), f2_hi(v.l)); }

constexpr int RC = 4;  // right-hand sides per pass of the operator-application kernel

// Residual of the collocation system on one leaf per CTA (256 threads), 2 NP right-hand
// sides per pass as NP pairs: every thread owns one node (more than one when p > 16) and
// accumulates all its pairs at once, so each table entry read from shared memory serves 2 NP
// products.  Per pass: u_ce = L_ce,ge u_ge (Eq. alpine2p5, written back to u; only the edge
// blocks of L_ce,ge that hold a row's nonzeros are summed), the first derivatives at every
// node, then r = g - A u at the interior nodes and the leaf fluxes v = D_ge,c u (Sec. 3.4).
// The kernel is bound by the shared-memory / L1 data pipe, so rows of u, g and r move with
// four lanes per 32-byte row segment (one sector), r is collected in shared memory and
// stored coalesced, and with stage_l the small tables L_ce,ge and L_loc are read from
// shared copies.
template <int NP>
__global__ void __launch_bounds__(256, 3) leaf_residual_df_kernel(
    ResidualArgs a, const int* __restrict__ leaf_edges, const int* __restrict__ ce,
    const double* __restrict__ ug, const double* __restrict__ g, double* __restrict__ uc, float* __restrict__ r_out,
    double* __restrict__ vflux, int nrhs, int stage_l) {
  constexpr int NRC = 2 * NP;
  const int lf = blockIdx.x;
  const int p = a.p, q = a.q, pp = p * p, nq = 4 * q, ne = 4 * (p - 1);
  extern __shared__ __align__(16) unsigned char smraw[];
  // {hi, hi, lo, lo} of D[i][k] and D2[i][k] at k p + i: lanes that differ in i read
  // consecutive entries, lanes with equal i one entry (broadcast)
  q2* sDt = reinterpret_cast<q2*>(smraw);
  q2* sD2t = sDt + pp;
  // pair-major, node (ix, iy) of pair pr at pr PS + iy (p + 1) + ix (rows padded by one entry,
  // so that the two rows a warp spans fall on different banks), pairs {h0, h1, l0, l1}
  const int PS = pp + p;
  q2* us = sD2t + pp;
  q2* uxs = us + PS * NP;
  q2* uys = uxs + PS * NP;
  q2* gs = uys + PS * NP;
  q2* ugs = gs + PS * NP;                                  // NP x nq
  float* rs = reinterpret_cast<float*>(ugs + nq * NP);     // pp x NRC: r of the pass (FP32)
  df* cf = reinterpret_cast<df*>(rs + pp * NRC);           // 6 pp: -c11, -2 c12, -c22, c1, c2, c
  float2* sL = reinterpret_cast<float2*>(cf + 6 * pp);     // staged L_ce,ge blocks, then L_loc
  const int nlc = stage_l ? a.n_lce : 0;
  const float2* Lc = stage_l ? sL : a.Lce_c;
  const float2* Ll = stage_l ? sL + ((nlc + 1) & ~1) : a.Lloc_df;
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int e = tid; e < pp; e += bs) {
    const float2 d1 = __ldg(a.D_df + e), d2 = __ldg(a.D2_df + e);
    const int i = e / p, k = e - (e / p) * p;
    sDt[k * p + i] = make_ulonglong2(f2_pack(d1.x, d1.x), f2_pack(d1.y, d1.y));
    sD2t[k * p + i] = make_ulonglong2(f2_pack(d2.x, d2.x), f2_pack(d2.y, d2.y));
  }
  if (stage_l) {
    for (int e = tid; e < nlc; e += bs) sL[e] = __ldg(a.Lce_c + e);
    for (int e = tid; e < q * p; e += bs) sL[((nlc + 1) & ~1) + e] = __ldg(a.Lloc_df + e);
  }
  const long long st = a.n_leaf * pp;
  for (int e = tid; e < 6 * pp; e += bs) {
    const int k = e / pp, n = e - (e / pp) * pp;
    const double c = a.coeffs[k * st + (long long)lf * pp + n];
    cf[e] = df_from(k == 0 || k == 2 ? -c : (k == 1 ? -2.0 * c : c));
  }
  const double hx = a.hxy[2 * lf], hy = a.hxy[2 * lf + 1];
  const df sx1 = df_from(2.0 / hx), sy1 = df_from(2.0 / hy);
  const df sxx1 = df_mul(sx1, sx1), syy1 = df_mul(sy1, sy1);
  const dfc sx = dfc_of(sx1.hi, sx1.lo), sy = dfc_of(sy1.hi, sy1.lo);
  const dfc sxx = dfc_of(sxx1.hi, sxx1.lo), syy = dfc_of(syy1.hi, syy1.lo);
  const long long lbase = (long long)lf * pp * nrhs;
  // component rr of a pair-major entry: hi at rr & 1, lo at 2 + (rr & 1)
  auto put = [](q2* arr, int idx, int rr, double x) {
    float* f = reinterpret_cast<float*>(arr + idx);
    const df v = df_from_i(x);
    f[rr & 1] = v.hi;
    f[2 + (rr & 1)] = v.lo;
  };
  for (int r0 = 0; r0 < nrhs; r0 += NRC) {
    __syncthreads();
    // rows of u and g at this pass's right-hand sides, NRC consecutive lanes per row
    for (int e = tid; e < pp * NRC; e += bs) {
      const int n = e / NRC, rr = e - (e / NRC) * NRC;
      const bool ok = r0 + rr < nrhs;
      const long long at = lbase + (long long)n * nrhs + r0 + rr;
      const int pn = (rr >> 1) * PS + n + n / p;
      put(us, pn, rr, ok ? uc[at] : 0.0);
      put(gs, pn, rr, ok ? g[at] : 0.0);
    }
    for (int e = tid; e < nq * NRC; e += bs) {
      const int gq = e / NRC, rr = e - (e / NRC) * NRC;
      const int s = gq / q, k = gq - (gq / q) * q;
      const long long node = (long long)leaf_edges[4 * lf + s] * q + k;
      put(ugs, (rr >> 1) * nq + gq, rr, r0 + rr < nrhs ? ug[node * nrhs + r0 + rr] : 0.0);
    }
    __syncthreads();
    // exterior values u_ce = L_ce,ge u_ge, written back in FP64
    for (int e = tid; e < ne * NP; e += bs) {
      const int k = e / NP, pr = e - (e / NP) * NP;
      df2 v = {0ull, 0ull};
      const int4 blk = __ldg(reinterpret_cast<const int4*>(a.Lce_blk) + k);
      const float2* Lrow = Lc + __ldg(a.Lce_off + k);
#pragma unroll 1
      for (int b = 0; b < 4; ++b) {
        const int cb = b == 0 ? blk.x : b == 1 ? blk.y : b == 2 ? blk.z : blk.w;
        if (cb < 0) break;
        for (int j = 0; j < q; ++j) {
          const float2 l = Lrow[b * q + j];
          dot2_acc(v, dfc_of(l.x, l.y), df2_ld(ugs + pr * nq + cb * q + j));
        }
      }
      v = df2_norm(v);
      const int n = ce[k];
      df2_st(us + pr * PS + n + n / p, v);
      const int r = r0 + 2 * pr;
      if (r < nrhs) uc[lbase + (long long)n * nrhs + r] = df2_to0(v);
      if (r + 1 < nrhs) uc[lbase + (long long)n * nrhs + r + 1] = df2_to1(v);
    }
    __syncthreads();
    // first derivatives at every node, all pairs per thread
    for (int n = tid; n < pp; n += bs) {
      const int ix = n % p, iy = n / p;
      df2 vx[NP], vy[NP];
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) vx[pr] = vy[pr] = df2{0ull, 0ull};
      for (int k = 0; k < p; ++k) {
        const dfc dx = dfc_ld(sDt + k * p + ix), dy = dfc_ld(sDt + k * p + iy);
        const q2* ur = us + iy * (p + 1) + k;
        const q2* uc2 = us + k * (p + 1) + ix;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          dot2_acc(vx[pr], dx, df2_ld(ur + pr * PS));
          dot2_acc(vy[pr], dy, df2_ld(uc2 + pr * PS));
        }
      }
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) {
        df2_st(uxs + pr * PS + iy * (p + 1) + ix, df2_mul(sx, df2_norm(vx[pr])));
        df2_st(uys + pr * PS + iy * (p + 1) + ix, df2_mul(sy, df2_norm(vy[pr])));
      }
    }
    __syncthreads();
    // residual r = g - A u at the interior nodes, 0 at the exterior ones
    for (int n = tid; n < pp; n += bs) {
      const int ix = n % p, iy = n / p;
      const bool inner = ix > 0 && ix < p - 1 && iy > 0 && iy < p - 1;
      if (!inner) {
#pragma unroll
        for (int rr = 0; rr < NRC; ++rr) rs[n * NRC + rr] = 0.f;
        continue;
      }
      df2 xx[NP], yy[NP], xy[NP];
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) xx[pr] = yy[pr] = xy[pr] = df2{0ull, 0ull};
      for (int k = 0; k < p; ++k) {
        const dfc d2x = dfc_ld(sD2t + k * p + ix), d2y = dfc_ld(sD2t + k * p + iy), d1y = dfc_ld(sDt + k * p + iy);
        const q2* ur = us + iy * (p + 1) + k;
        const q2* uc2 = us + k * (p + 1) + ix;
        const q2* xc = uxs + k * (p + 1) + ix;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          dot2_acc(xx[pr], d2x, df2_ld(ur + pr * PS));
          dot2_acc(yy[pr], d2y, df2_ld(uc2 + pr * PS));
          dot2_acc(xy[pr], d1y, df2_ld(xc + pr * PS));
        }
      }
      dfc c6[6];
#pragma unroll
      for (int t = 0; t < 6; ++t) c6[t] = dfc_of(cf[t * pp + n].hi, cf[t * pp + n].lo);
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) {
        // A u = -c11 u_xx - 2 c12 u_xy - c22 u_yy + c1 u_x + c2 u_y + c u  (Sec. 3.2)
        df2 Au = {0ull, 0ull};
        dot2_acc(Au, c6[0], df2_mul(sxx, df2_norm(xx[pr])));
        dot2_acc(Au, c6[1], df2_mul(sy, df2_norm(xy[pr])));
        dot2_acc(Au, c6[2], df2_mul(syy, df2_norm(yy[pr])));
        const int pn = pr * PS + iy * (p + 1) + ix;
        dot2_acc(Au, c6[3], df2_ld(uxs + pn));
        dot2_acc(Au, c6[4], df2_ld(uys + pn));
        dot2_acc(Au, c6[5], df2_ld(us + pn));
        Au = df2_norm(Au);
        const df2 gg = df2_ld(gs + pn);
        // g - A u: TwoSum of the high parts plus the low parts
        const f2 sh = f2_sub(gg.h, Au.h);
        const f2 bb = f2_sub(sh, gg.h);
        const f2 t = f2_sub(f2_sub(gg.h, f2_sub(sh, bb)), f2_add(Au.h, bb));
        const df2 res = df2_norm({sh, f2_add(t, f2_sub(gg.l, Au.l))});
        // r rounded to FP32 (the high part of the renormalised pair): the correction solve's
        // right-hand side
        rs[n * NRC + 2 * pr] = f2_lo(res.h);
        rs[n * NRC + 2 * pr + 1] = f2_hi(res.h);
      }
    }
    // leaf fluxes v = D_ge,c u (Sec. 3.4), taken from the last threads first (the interior
    // nodes keep the first ones busy)
    for (int e = bs - 1 - tid; e < nq * NP; e += bs) {
      const int gq = e / NP, pr = e - (e / NP) * NP;
      const int s = gq / q, k = gq - (gq / q) * q;
      df2 v = {0ull, 0ull};
      for (int t = 0; t < p; ++t) {
        const q2* d;
        switch (s) {
          case 0: d = uys + pr * PS + t; break;
          case 1: d = uxs + pr * PS + t * (p + 1) + (p - 1); break;
          case 2: d = uys + pr * PS + (p - 1) * (p + 1) + t; break;
          default: d = uxs + pr * PS + t * (p + 1); break;
        }
        const float2 l = Ll[k * p + t];
        dot2_acc(v, dfc_of(l.x, l.y), df2_ld(d));
      }
      v = df2_norm(v);
      const long long row = ((long long)lf * nq + gq) * nrhs + r0 + 2 * pr;
      if (r0 + 2 * pr < nrhs) vflux[row] = df2_to0(v);
      if (r0 + 2 * pr + 1 < nrhs) vflux[row + 1] = df2_to1(v);
    }
    __syncthreads();
    for (int e = tid; e < pp * NRC; e += bs) {
      const int n = e / NRC, rr = e - (e / NRC) * NRC;
      if (r0 + rr < nrhs) r_out[lbase + (long long)n * nrhs + r0 + rr] = rs[e];
    }
  }
}

// Coefficient gradients (adjoint): grad_k[n] = sum_r gbar[n][r] t_k(u)[n][r] at interior
// nodes with t = (u_xx, 2 u_xy, u_yy, -u_x, -u_y, -u) (the operator of Sec. 3.2), 0 on the
// exterior; derivatives and sums in double-float.
__global__ void __launch_bounds__(256) coeff_grad_df_kernel(ResidualArgs a, const double* __restrict__ uc,
                                                            const double* __restrict__ gbar,
                                                            double* __restrict__ grad, int nrhs) {
  const int lf = blockIdx.x;
  const int p = a.p, pp = p * p;
  extern __shared__ __align__(16) unsigned char smraw[];
  df* sD = reinterpret_cast<df*>(smraw);
  df* sD2 = sD + pp;
  df* us = sD2 + pp;    // pp
  df* uxs = us + pp;    // pp
  df* acc = uxs + pp;   // 6 * pp
  df* sDt = acc + 6 * pp;  // transposed D, D2 (conflict-free reads across ix)
  df* sD2t = sDt + pp;
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int e = tid; e < pp; e += bs) {
    sD[e] = df_from(a.D[e]);
    sD2[e] = df_from(a.D2[e]);
    const int i = e / p, k = e - (e / p) * p;
    sDt[k * p + i] = sD[e];
    sD2t[k * p + i] = sD2[e];
  }
  for (int e = tid; e < 6 * pp; e += bs) acc[e] = {0.f, 0.f};
  const df sx = df_from(2.0 / a.hxy[2 * lf]), sy = df_from(2.0 / a.hxy[2 * lf + 1]);
  const df sxx = df_mul(sx, sx), syy = df_mul(sy, sy), two_sy = df_add(sy, sy);
  const long long lbase = (long long)lf * pp * nrhs;
  for (int r = 0; r < nrhs; ++r) {
    __syncthreads();
    for (int n = tid; n < pp; n += bs) us[n] = df_from(uc[lbase + (long long)n * nrhs + r]);
    __syncthreads();
    for (int n = tid; n < pp; n += bs) {
      const int ix = n % p, iy = n / p;
      df v = {0.f, 0.f};
      for (int k = 0; k < p; ++k) v = df_fma_acc(v, sDt[k * p + ix], us[iy * p + k]);
      uxs[n] = df_mul(sx, v);
    }
    __syncthreads();
    for (int n = tid; n < pp; n += bs) {
      const int ix = n % p, iy = n / p;
      if (!(ix > 0 && ix < p - 1 && iy > 0 && iy < p - 1)) continue;
      df uy = {0.f, 0.f}, uxx = {0.f, 0.f}, uyy = {0.f, 0.f}, uxy = {0.f, 0.f};
      for (int k = 0; k < p; ++k) {
        uy = df_fma_acc(uy, sD[iy * p + k], us[k * p + ix]);
        uxx = df_fma_acc(uxx, sD2t[k * p + ix], us[iy * p + k]);
        uyy = df_fma_acc(uyy, sD2[iy * p + k], us[k * p + ix]);
        uxy = df_fma_acc(uxy, sD[iy * p + k], uxs[k * p + ix]);
      }
      const df lam = df_from(gbar[lbase + (long long)n * nrhs + r]);
      acc[0 * pp + n] = df_fma_acc(acc[0 * pp + n], lam, df_mul(sxx, uxx));
      acc[1 * pp + n] = df_fma_acc(acc[1 * pp + n], lam, df_mul(two_sy, uxy));
      acc[2 * pp + n] = df_fma_acc(acc[2 * pp + n], lam, df_mul(syy, uyy));
      acc[3 * pp + n] = df_fma_acc(acc[3 * pp + n], df_neg(lam), uxs[n]);
      acc[4 * pp + n] = df_fma_acc(acc[4 * pp + n], df_neg(lam), df_mul(sy, uy));
      acc[5 * pp + n] = df_fma_acc(acc[5 * pp + n], df_neg(lam), us[n]);
    }
  }
  __syncthreads();
  for (int e = tid; e < 6 * pp; e += bs) {
    const int k = e / pp, n = e - (e / pp) * pp;
    grad[((long long)k * a.n_leaf + lf) * pp + n] = df_to(acc[e]);
  }
}

// y = alpha u + beta A u at interior nodes (0 on the exterior) with A the collocation
// operator of Sec. 3.2; u's exterior values are used as given.  Double-float arithmetic.
__global__ void __launch_bounds__(256) leaf_apply_df_kernel(ResidualArgs a, const double* __restrict__ u,
                                                            double alpha, double beta, double* __restrict__ out,
                                                            int nrhs) {
  const int lf = blockIdx.x;
  const int p = a.p, pp = p * p;
  extern __shared__ __align__(16) unsigned char smraw[];
  df* sD = reinterpret_cast<df*>(smraw);
  df* sD2 = sD + pp;
  df* sDt = sD2 + pp;
  df* sD2t = sDt + pp;
  df* cf = sD2t + pp;        // 6 * pp
  df* us = cf + 6 * pp;      // pp * RC
  df* uxs = us + pp * RC;    // pp * RC
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int e = tid; e < pp; e += bs) {
    sD[e] = df_from(a.D[e]);
    sD2[e] = df_from(a.D2[e]);
    const int i = e / p, k = e - (e / p) * p;
    sDt[k * p + i] = sD[e];
    sD2t[k * p + i] = sD2[e];
  }
  const long long st = a.n_leaf * pp;
  for (int e = tid; e < 6 * pp; e += bs) {
    const int k = e / pp, n = e - (e / pp) * pp;
    const double c = a.coeffs[k * st + (long long)lf * pp + n];
    cf[e] = df_from(k == 0 || k == 2 ? -c : (k == 1 ? -2.0 * c : c));
  }
  const df sx = df_from(2.0 / a.hxy[2 * lf]), sy = df_from(2.0 / a.hxy[2 * lf + 1]);
  const df sxx = df_mul(sx, sx), syy = df_mul(sy, sy);
  const df dal = df_from(alpha), dbe = df_from(beta);
  const long long lbase = (long long)lf * pp * nrhs;
  for (int r0 = 0; r0 < nrhs; r0 += RC) {
    const int rc = min(RC, nrhs - r0);
    __syncthreads();
    for (int e = tid; e < pp * RC; e += bs) {
      const int n = e / RC, rr = e - (e / RC) * RC;
      us[e] = df_from(rr < rc ? u[lbase + (long long)n * nrhs + r0 + rr] : 0.0);
    }
    __syncthreads();
    for (int e = tid; e < pp * RC; e += bs) {
      const int n = e / RC, rr = e - (e / RC) * RC;
      const int ix = n % p, iy = n / p;
      df v = {0.f, 0.f};
      for (int k = 0; k < p; ++k) v = df_fma_acc(v, sDt[k * p + ix], us[(iy * p + k) * RC + rr]);
      uxs[e] = df_mul(sx, v);
    }
    __syncthreads();
    for (int e = tid; e < pp * RC; e += bs) {
      const int n = e / RC, rr = e - (e / RC) * RC;
      if (rr >= rc) continue;
      const int ix = n % p, iy = n / p;
      double y = 0.0;
      if (ix > 0 && ix < p - 1 && iy > 0 && iy < p - 1) {
        df uy = {0.f, 0.f}, uxx = {0.f, 0.f}, uyy = {0.f, 0.f}, uxy = {0.f, 0.f};
        for (int k = 0; k < p; ++k) {
          uy = df_fma_acc(uy, sD[iy * p + k], us[(k * p + ix) * RC + rr]);
          uxx = df_fma_acc(uxx, sD2t[k * p + ix], us[(iy * p + k) * RC + rr]);
          uyy = df_fma_acc(uyy, sD2[iy * p + k], us[(k * p + ix) * RC + rr]);
          uxy = df_fma_acc(uxy, sD[iy * p + k], uxs[(k * p + ix) * RC + rr]);
        }
        // A u = -c11 u_xx - 2 c12 u_xy - c22 u_yy + c1 u_x + c2 u_y + c u  (Sec. 3.2)
        df Au = df_mul(cf[n], df_mul(uxx, sxx));
        Au = df_fma(Au, cf[pp + n], df_mul(uxy, sy));
        Au = df_fma(Au, cf[2 * pp + n], df_mul(uyy, syy));
        Au = df_fma(Au, cf[3 * pp + n], uxs[e]);
        Au = df_fma(Au, cf[4 * pp + n], df_mul(sy, uy));
        Au = df_fma(Au, cf[5 * pp + n], us[e]);
        y = df_to(df_add(df_mul(dal, us[e]), df_mul(dbe, Au)));
      }
      out[lbase + (long long)n * nrhs + r0 + rr] = y;
    }
  }
}

}  // namespace

void launch_leaf_apply_df(const ResidualArgs& a, const double* u, double alpha, double beta, double* out, int nrhs,
                          cudaStream_t s) {
  const int pp = a.p * a.p;
  const size_t smem = (size_t)(10 * pp + 2 * pp * RC) * sizeof(df);
  ensure_smem((const void*)leaf_apply_df_kernel, smem);
  leaf_apply_df_kernel<<<(unsigned)a.n_leaf, 256, smem, s>>>(a, u, alpha, beta, out, nrhs);
}

void launch_coeff_grad(const ResidualArgs& a, const double* uc, const double* gbar, double* grad, int nrhs,
                       cudaStream_t s) {
  const int pp = a.p * a.p;
  const size_t smem = (size_t)(12 * pp) * sizeof(df);
  ensure_smem((const void*)coeff_grad_df_kernel, smem);
  coeff_grad_df_kernel<<<(unsigned)a.n_leaf, 256, smem, s>>>(a, uc, gbar, grad, nrhs);
}

// Shared memory of the residual kernel: tables, pass buffers and coefficients, plus the
// staged L tables when stage_l.
static size_t residual_smem(const ResidualArgs& a, int np, int nlc, bool stage_l) {
  const size_t pp = (size_t)a.p * a.p, nq = 4 * (size_t)a.q;
  size_t b = (2 * pp + 4 * (pp + a.p) * np + nq * np) * sizeof(ulonglong2) + pp * 2 * np * sizeof(float) +
             6 * pp * sizeof(df);
  if (stage_l) b += (((size_t)nlc + 1) & ~(size_t)1) * sizeof(float2) + (size_t)a.q * a.p * sizeof(float2);
  return b;
}

template <int NP>
static void residual_launch(const ResidualArgs& a, const int* leaf_edges, const int* ce, const double* ug,
                            const double* g, double* uc, float* r_out, double* vflux, int nrhs, int nlc,
                            cudaStream_t s) {
  const size_t limit = 227 * 1024;
  const bool stage_l = residual_smem(a, NP, nlc, true) <= limit;
  const size_t smem = residual_smem(a, NP, nlc, stage_l);
  ensure_smem((const void*)leaf_residual_df_kernel<NP>, smem);
  leaf_residual_df_kernel<NP><<<(unsigned)a.n_leaf, 256, smem, s>>>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs,
                                                                    stage_l ? 1 : 0);
}

void launch_leaf_residual_df(const ResidualArgs& a, const int* leaf_edges, const int* ce,
                             const double* ug, const double* g, double* uc, float* r_out, double* vflux, int nrhs,
                             cudaStream_t s) {
  const int n_lce = a.n_lce;
  // two pairs per pass unless the buffers then exceed the shared memory of a CTA
  if (nrhs <= 2 || residual_smem(a, 2, n_lce, false) > 227 * 1024)
    residual_launch<1>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs, n_lce, s);
  else
    residual_launch<2>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs, n_lce, s);
}

}  // namespace hps
