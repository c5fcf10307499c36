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

constexpr int RC = 4;  // right-hand sides per pass of the operator-application kernel

// Residual of the collocation system on one leaf per CTA (256 threads), RC right-hand
// sides per pass: every thread owns one node (more than one when p > 16) and accumulates
// its RC values at once, so each table entry read from shared memory serves RC products.
// Per pass: u_ce = L_ce,ge u_ge (Eq. alpine2p5, written back to u), the first derivatives
// at every node, then r = g - A u at the interior nodes and the leaf fluxes
// v = D_ge,c u (Sec. 3.4).
template <int NRC>
__global__ void __launch_bounds__(256) leaf_residual_df_kernel(
    ResidualArgs a, const int* __restrict__ leaf_edges, const int* __restrict__ ce,
    const double* __restrict__ ug, const double* __restrict__ g, double* __restrict__ uc, double* __restrict__ r_out,
    double* __restrict__ vflux, int nrhs) {
  const int lf = blockIdx.x;
  const int p = a.p, q = a.q, pp = p * p, nq = 4 * q, ne = 4 * (p - 1);
  extern __shared__ __align__(16) unsigned char smraw[];
  df* sD = reinterpret_cast<df*>(smraw);
  df* sD2 = sD + pp;
  df* sDt = sD2 + pp;          // D and D2 transposed: lanes that differ in ix read
  df* sD2t = sDt + pp;         // consecutive words
  df* cf = sD2t + pp;          // 6 * pp: -c11, -2 c12, -c22, c1, c2, c of this leaf
  df* us = cf + 6 * pp;        // pp * NRC
  df* uxs = us + pp * NRC;     // pp * NRC
  df* uys = uxs + pp * NRC;    // pp * NRC
  df* ugs = uys + pp * NRC;    // nq * NRC
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int e = tid; e < pp; e += bs) {
    const float2 d1 = __ldg(a.D_df + e), d2 = __ldg(a.D2_df + e);
    const int i = e / p, k = e - (e / p) * p;
    sD[e] = df{d1.x, d1.y};
    sD2[e] = df{d2.x, d2.y};
    sDt[k * p + i] = df{d1.x, d1.y};
    sD2t[k * p + i] = df{d2.x, d2.y};
  }
  const long long st = a.n_leaf * pp;
  for (int e = tid; e < 6 * pp; e += bs) {
    const int k = e / pp, n = e - (e / pp) * pp;
    const double c = a.coeffs[k * st + (long long)lf * pp + n];
    cf[e] = df_from(k == 0 || k == 2 ? -c : (k == 1 ? -2.0 * c : c));
  }
  const double hx = a.hxy[2 * lf], hy = a.hxy[2 * lf + 1];
  const df sx = df_from(2.0 / hx), sy = df_from(2.0 / hy);
  const df sxx = df_mul(sx, sx), syy = df_mul(sy, sy);
  const long long lbase = (long long)lf * pp * nrhs;
  for (int r0 = 0; r0 < nrhs; r0 += NRC) {
    const int rc = min(NRC, nrhs - r0);
    __syncthreads();
    for (int e = tid; e < nq * NRC; e += bs) {
      const int gq = e / NRC, rr = e - (e / NRC) * NRC;
      const int s = gq / q, k = gq - (gq / q) * q;
      const int node = leaf_edges[4 * lf + s] * q + k;
      ugs[e] = df_from(rr < rc ? ug[(long long)node * nrhs + r0 + rr] : 0.0);
    }
    for (int e = tid; e < pp * NRC; e += bs) {
      const int n = e / NRC, rr = e - (e / NRC) * NRC;
      us[e] = df_from(rr < rc ? uc[lbase + (long long)n * nrhs + r0 + rr] : 0.0);
    }
    __syncthreads();
    // exterior values u_ce = L_ce,ge u_ge, written back in FP64
    for (int e = tid; e < ne * NRC; e += bs) {
      const int k = e / NRC, rr = e - (e / NRC) * NRC;
      df v = {0.f, 0.f};
      const float2* Lrow = a.Lce_df + (long long)k * nq;
      for (int gq = 0; gq < nq; ++gq) {
        const float2 l = __ldg(Lrow + gq);
        v = df_fma_acc(v, df{l.x, l.y}, ugs[gq * NRC + rr]);
      }
      const int n = ce[k];
      us[n * NRC + rr] = v;
      if (rr < rc) uc[lbase + (long long)n * nrhs + r0 + rr] = df_to(v);
    }
    __syncthreads();
    // first derivatives at every node, all NRC right-hand sides per thread
    for (int n = tid; n < pp; n += bs) {
      const int ix = n % p, iy = n / p;
      df vx[NRC], vy[NRC];
#pragma unroll
      for (int rr = 0; rr < NRC; ++rr) vx[rr] = vy[rr] = df{0.f, 0.f};
      for (int k = 0; k < p; ++k) {
        const df dx = sDt[k * p + ix], dy = sD[iy * p + k];
        const df* ur = us + (iy * p + k) * NRC;
        const df* uc2 = us + (k * p + ix) * NRC;
#pragma unroll
        for (int rr = 0; rr < NRC; ++rr) {
          vx[rr] = df_fma_acc(vx[rr], dx, ur[rr]);
          vy[rr] = df_fma_acc(vy[rr], dy, uc2[rr]);
        }
      }
#pragma unroll
      for (int rr = 0; rr < NRC; ++rr) {
        uxs[n * NRC + rr] = df_mul(sx, vx[rr]);
        uys[n * NRC + rr] = df_mul(sy, vy[rr]);
      }
    }
    __syncthreads();
    // residual r = g - A u at the interior nodes, 0 at the exterior ones
    for (int n = tid; n < pp; n += bs) {
      const int ix = n % p, iy = n / p;
      const bool inner = ix > 0 && ix < p - 1 && iy > 0 && iy < p - 1;
      if (!inner) {
        for (int rr = 0; rr < rc; ++rr) r_out[lbase + (long long)n * nrhs + r0 + rr] = 0.0;
        continue;
      }
      df xx[NRC], yy[NRC], xy[NRC];
#pragma unroll
      for (int rr = 0; rr < NRC; ++rr) xx[rr] = yy[rr] = xy[rr] = df{0.f, 0.f};
      for (int k = 0; k < p; ++k) {
        const df d2x = sD2t[k * p + ix], d2y = sD2[iy * p + k], d1y = sD[iy * p + k];
        const df* ur = us + (iy * p + k) * NRC;
        const df* uc2 = us + (k * p + ix) * NRC;
        const df* xc = uxs + (k * p + ix) * NRC;
#pragma unroll
        for (int rr = 0; rr < NRC; ++rr) {
          xx[rr] = df_fma_acc(xx[rr], d2x, ur[rr]);
          yy[rr] = df_fma_acc(yy[rr], d2y, uc2[rr]);
          xy[rr] = df_fma_acc(xy[rr], d1y, xc[rr]);
        }
      }
#pragma unroll
      for (int rr = 0; rr < NRC; ++rr) {
        if (rr >= rc) break;
        const int e = n * NRC + rr;
        // A u = -c11 u_xx - 2 c12 u_xy - c22 u_yy + c1 u_x + c2 u_y + c u  (Sec. 3.2)
        df Au = df_mul(cf[n], df_mul(xx[rr], sxx));
        Au = df_fma(Au, cf[pp + n], df_mul(xy[rr], sy));
        Au = df_fma(Au, cf[2 * pp + n], df_mul(yy[rr], syy));
        Au = df_fma(Au, cf[3 * pp + n], uxs[e]);
        Au = df_fma(Au, cf[4 * pp + n], uys[e]);
        Au = df_fma(Au, cf[5 * pp + n], us[e]);
        const df r = df_add(df_from(g[lbase + (long long)n * nrhs + r0 + rr]), df_neg(Au));
        r_out[lbase + (long long)n * nrhs + r0 + rr] = df_to(r);
      }
    }
    // leaf fluxes v = D_ge,c u (Sec. 3.4), taken from the last threads first (the interior
    // nodes keep the first ones busy)
    for (int e = bs - 1 - tid; e < nq * NRC; e += bs) {
      const int gq = e / NRC, rr = e - (e / NRC) * NRC;
      if (rr >= rc) continue;
      const int s = gq / q, k = gq - (gq / q) * q;
      df v = {0.f, 0.f};
      for (int t = 0; t < p; ++t) {
        df d;
        switch (s) {
          case 0: d = uys[(0 * p + t) * NRC + rr]; break;
          case 1: d = uxs[(t * p + (p - 1)) * NRC + rr]; break;
          case 2: d = uys[((p - 1) * p + t) * NRC + rr]; break;
          default: d = uxs[(t * p + 0) * NRC + rr]; break;
        }
        const float2 l = __ldg(a.Lloc_df + k * p + t);
        v = df_fma_acc(v, df{l.x, l.y}, d);
      }
      vflux[((long long)lf * nq + gq) * nrhs + r0 + rr] = df_to(v);
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

template <int NRC>
static void residual_launch(const ResidualArgs& a, const int* leaf_edges, const int* ce, const double* ug,
                            const double* g, double* uc, double* r_out, double* vflux, int nrhs, cudaStream_t s) {
  const int pp = a.p * a.p;
  const size_t smem = (size_t)(10 * pp + 3 * pp * NRC + 4 * a.q * NRC) * sizeof(df);
  if (smem > 48 * 1024) {
    // the limit is a property of the device's context: raised once per device (the first
    // launch is never inside a stream capture: a handle's first solve runs directly)
    static std::mutex mu;
    static size_t configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && smem > configured[dev]) {
      cudaFuncSetAttribute(leaf_residual_df_kernel<NRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      configured[dev] = smem;
    }
  }
  leaf_residual_df_kernel<NRC><<<(unsigned)a.n_leaf, 256, smem, s>>>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs);
}

void launch_leaf_residual_df(const ResidualArgs& a, const int* leaf_edges, const int* ce,
                             const double* ug, const double* g, double* uc, double* r_out, double* vflux, int nrhs,
                             cudaStream_t s) {
  if (nrhs == 1) residual_launch<1>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs, s);
  else if (nrhs == 2) residual_launch<2>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs, s);
  else residual_launch<4>(a, leaf_edges, ce, ug, g, uc, r_out, vflux, nrhs, s);
}

}  // namespace hps
