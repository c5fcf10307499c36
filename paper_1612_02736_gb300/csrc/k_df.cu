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
// from a table entry {hi, hi, lo, lo}
__device__ __forceinline__ dfc dfc_of4(float4 v) {
  const f2 h = f2_pack(v.x, v.y);
  return {h, f2_pack(v.z, v.w), f2_mul(h, f2_pack(-1.f, -1.f))};
}
__device__ __forceinline__ df2 df2_of4(float4 v) { return {f2_pack(v.x, v.y), f2_pack(v.z, v.w)}; }
__device__ __forceinline__ float4 df2_to4(df2 v) { return make_float4(f2_lo(v.h), f2_hi(v.h), f2_lo(v.l), f2_hi(v.l)); }

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
// the pair's values of a row of FP64 data (two consecutive right-hand sides, the second
// zero when absent)
__device__ __forceinline__ df2 df2_from(double x0, double x1) {
  const df a = df_from(x0), b = df_from(x1);
  return {f2_pack(a.hi, b.hi), f2_pack(a.lo, b.lo)};
}
__device__ __forceinline__ double df2_to0(df2 v) { return (double)f2_lo(v.h) + (double)f2_lo(v.l); }
__device__ __forceinline__ double df2_to1(df2 v) { return (double)f2_hi(v.h) + (double)f2_hi(v.l); }

constexpr int RC = 4;  // right-hand sides per pass of the operator-application kernel

// Residual of the collocation system on one leaf per CTA (256 threads), 2 NP right-hand
// sides per pass as NP pairs: every thread owns one node (more than one when p > 16) and
// accumulates all its pairs at once, so each table entry read from shared memory serves 2 NP
// products.  Per pass: u_ce = L_ce,ge u_ge (Eq. alpine2p5, written back to u; only the edge
// blocks of L_ce,ge that hold a row's nonzeros are summed), the first derivatives at every
// node, then r = g - A u at the interior nodes and the leaf fluxes v = D_ge,c u (Sec. 3.4).
template <int NP>
__global__ void __launch_bounds__(256) leaf_residual_df_kernel(
    ResidualArgs a, const int* __restrict__ leaf_edges, const int* __restrict__ ce,
    const double* __restrict__ ug, const double* __restrict__ g, double* __restrict__ uc, double* __restrict__ r_out,
    double* __restrict__ vflux, int nrhs) {
  constexpr int NRC = 2 * NP;
  const int lf = blockIdx.x;
  const int p = a.p, q = a.q, pp = p * p, nq = 4 * q, ne = 4 * (p - 1);
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* sD = reinterpret_cast<float4*>(smraw);  // {hi, hi, lo, lo} of D[i][k] at i p + k
  float4* sD2 = sD + pp;
  float4* sDt = sD2 + pp;                          // transposed (D[i][k] at k p + i): lanes
  float4* sD2t = sDt + pp;                         // that differ in ix read consecutive entries
  // pair-major (pair pr of node n at pr pp + n): lanes that differ in ix read consecutive
  // 16-byte entries
  float4* us = sD2t + pp;                          // NP x pp pairs {h0, h1, l0, l1}
  float4* uxs = us + pp * NP;
  float4* uys = uxs + pp * NP;
  float4* ugs = uys + pp * NP;                     // NP x nq
  df* cf = reinterpret_cast<df*>(ugs + nq * NP);   // 6 pp: -c11, -2 c12, -c22, c1, c2, c of this leaf
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int e = tid; e < pp; e += bs) {
    const float2 d1 = __ldg(a.D_df + e), d2 = __ldg(a.D2_df + e);
    const int i = e / p, k = e - (e / p) * p;
    const float4 v1 = make_float4(d1.x, d1.x, d1.y, d1.y), v2 = make_float4(d2.x, d2.x, d2.y, d2.y);
    sD[e] = v1;
    sD2[e] = v2;
    sDt[k * p + i] = v1;
    sD2t[k * p + i] = v2;
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
  // the pair of FP64 values of row `row` at right-hand sides r, r + 1 (0 past nrhs)
  auto pair_of = [&](const double* base, long long row, int r) {
    const double x0 = r < nrhs ? base[row * nrhs + r] : 0.0;
    const double x1 = r + 1 < nrhs ? base[row * nrhs + r + 1] : 0.0;
    return df2_from(x0, x1);
  };
  auto store_pair = [&](double* base, long long row, int r, const df2& v) {
    if (r < nrhs) base[row * nrhs + r] = df2_to0(v);
    if (r + 1 < nrhs) base[row * nrhs + r + 1] = df2_to1(v);
  };
  for (int r0 = 0; r0 < nrhs; r0 += NRC) {
    __syncthreads();
    for (int e = tid; e < nq * NP; e += bs) {
      const int gq = e / NP, pr = e - (e / NP) * NP;
      const int s = gq / q, k = gq - (gq / q) * q;
      const int node = leaf_edges[4 * lf + s] * q + k;
      ugs[pr * nq + gq] = df2_to4(pair_of(ug, node, r0 + 2 * pr));
    }
    for (int e = tid; e < pp * NP; e += bs) {
      const int n = e / NP, pr = e - (e / NP) * NP;
      us[pr * pp + n] = df2_to4(pair_of(uc + lbase, n, r0 + 2 * pr));
    }
    __syncthreads();
    // exterior values u_ce = L_ce,ge u_ge, written back in FP64
    for (int e = tid; e < ne * NP; e += bs) {
      const int k = e / NP, pr = e - (e / NP) * NP;
      df2 v = {0ull, 0ull};
      const float2* Lrow = a.Lce_df + (long long)k * nq;
      const int4 blk = __ldg(reinterpret_cast<const int4*>(a.Lce_blk) + k);
      const int bl[4] = {blk.x, blk.y, blk.z, blk.w};
#pragma unroll 1
      for (int b = 0; b < 4; ++b) {
        if (bl[b] < 0) break;
        for (int gq = bl[b] * q; gq < bl[b] * q + q; ++gq) {
          const float2 l = __ldg(Lrow + gq);
          dot2_acc(v, dfc_of(l.x, l.y), df2_of4(ugs[pr * nq + gq]));
        }
      }
      v = df2_norm(v);
      const int n = ce[k];
      us[pr * pp + n] = df2_to4(v);
      store_pair(uc + lbase, n, r0 + 2 * pr, v);
    }
    __syncthreads();
    // first derivatives at every node, all pairs per thread
    for (int n = tid; n < pp; n += bs) {
      const int ix = n % p, iy = n / p;
      df2 vx[NP], vy[NP];
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) vx[pr] = vy[pr] = df2{0ull, 0ull};
      for (int k = 0; k < p; ++k) {
        const dfc dx = dfc_of4(sDt[k * p + ix]), dy = dfc_of4(sD[iy * p + k]);
        const float4* ur = us + iy * p + k;
        const float4* uc2 = us + k * p + ix;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          dot2_acc(vx[pr], dx, df2_of4(ur[pr * pp]));
          dot2_acc(vy[pr], dy, df2_of4(uc2[pr * pp]));
        }
      }
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) {
        uxs[pr * pp + n] = df2_to4(df2_mul(sx, df2_norm(vx[pr])));
        uys[pr * pp + n] = df2_to4(df2_mul(sy, df2_norm(vy[pr])));
      }
    }
    __syncthreads();
    // residual r = g - A u at the interior nodes, 0 at the exterior ones
    for (int n = tid; n < pp; n += bs) {
      const int ix = n % p, iy = n / p;
      const bool inner = ix > 0 && ix < p - 1 && iy > 0 && iy < p - 1;
      if (!inner) {
        for (int rr = 0; rr < NRC && r0 + rr < nrhs; ++rr) r_out[lbase + (long long)n * nrhs + r0 + rr] = 0.0;
        continue;
      }
      df2 xx[NP], yy[NP], xy[NP];
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) xx[pr] = yy[pr] = xy[pr] = df2{0ull, 0ull};
      for (int k = 0; k < p; ++k) {
        const dfc d2x = dfc_of4(sD2t[k * p + ix]), d2y = dfc_of4(sD2[iy * p + k]), d1y = dfc_of4(sD[iy * p + k]);
        const float4* ur = us + iy * p + k;
        const float4* uc2 = us + k * p + ix;
        const float4* xc = uxs + k * p + ix;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          dot2_acc(xx[pr], d2x, df2_of4(ur[pr * pp]));
          dot2_acc(yy[pr], d2y, df2_of4(uc2[pr * pp]));
          dot2_acc(xy[pr], d1y, df2_of4(xc[pr * pp]));
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
        dot2_acc(Au, c6[3], df2_of4(uxs[pr * pp + n]));
        dot2_acc(Au, c6[4], df2_of4(uys[pr * pp + n]));
        dot2_acc(Au, c6[5], df2_of4(us[pr * pp + n]));
        Au = df2_norm(Au);
        const df2 gg = pair_of(g + lbase, n, r0 + 2 * pr);
        // g - A u: TwoSum of the high parts plus the low parts
        const f2 sh = f2_sub(gg.h, Au.h);
        const f2 bb = f2_sub(sh, gg.h);
        const f2 t = f2_sub(f2_sub(gg.h, f2_sub(sh, bb)), f2_add(Au.h, bb));
        store_pair(r_out + lbase, n, r0 + 2 * pr, df2_norm({sh, f2_add(t, f2_sub(gg.l, Au.l))}));
      }
    }
    // leaf fluxes v = D_ge,c u (Sec. 3.4), taken from the last threads first (the interior
    // nodes keep the first ones busy)
    for (int e = bs - 1 - tid; e < nq * NP; e += bs) {
      const int gq = e / NP, pr = e - (e / NP) * NP;
      const int s = gq / q, k = gq - (gq / q) * q;
      df2 v = {0ull, 0ull};
      for (int t = 0; t < p; ++t) {
        float4 d;
        switch (s) {
          case 0: d = uys[pr * pp + 0 * p + t]; break;
          case 1: d = uxs[pr * pp + t * p + (p - 1)]; break;
          case 2: d = uys[pr * pp + (p - 1) * p + t]; break;
          default: d = uxs[pr * pp + t * p + 0]; break;
        }
        const float2 l = __ldg(a.Lloc_df + k * p + t);
        dot2_acc(v, dfc_of(l.x, l.y), df2_of4(d));
      }
      store_pair(vflux, (long long)lf * nq + gq, r0 + 2 * pr, df2_norm(v));
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
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaFuncSetAttribute(leaf_apply_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  leaf_apply_df_kernel<<<(unsigned)a.n_leaf, 256, smem, s>>>(a, u, alpha, beta, out, nrhs);
}

void launch_coeff_grad(const ResidualArgs& a, const double* uc, const double* gbar, double* grad, int nrhs,
                       cudaStream_t s) {
  const int pp = a.p * a.p;
  const size_t smem = (size_t)(12 * pp) * sizeof(df);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaFuncSetAttribute(coeff_grad_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
  coeff_grad_df_kernel<<<(unsigned)a.n_leaf, 256, smem, s>>>(a, uc, gbar, grad, nrhs);
}

template <int NP>
static void residual_launch(const ResidualArgs& a, const int* leaf_edges, const int* ce, const double* ug,
                            const double* g, double* uc, double* r_out, double* vflux, int nrhs, cudaStream_t s) {
  const int pp = a.p * a.p;
  const size_t smem = (size_t)(4 * pp + 3 * pp * NP + 4 * a.q * NP) * sizeof(float4) + (size_t)6 * pp * sizeof(df);
  if (smem > 48 * 1024) {
    // the limit is a property of the device's context: raised once per device (the first
    // launch is never inside a stream capture: a handle's first solve runs directly)
    static std::mutex mu;
    static size_t configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && smem > configured[dev]) {
      cudaFuncSetAttribute(leaf_residual_df_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      configured[dev] = smem;
    }
  }
  leaf_residual_df_kernel<NP><<<(unsigned)a.n_leaf, 256, smem, s>>>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs);
}

void launch_leaf_residual_df(const ResidualArgs& a, const int* leaf_edges, const int* ce,
                             const double* ug, const double* g, double* uc, double* r_out, double* vflux, int nrhs,
                             cudaStream_t s) {
  if (nrhs <= 2) residual_launch<1>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs, s);
  else residual_launch<2>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs, s);
}

}  // namespace hps
