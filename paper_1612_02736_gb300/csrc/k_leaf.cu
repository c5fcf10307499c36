// Leaf assembly (Sec. 3.2-3.4, Algorithm 1 leaf branch): builds, per leaf, the matrix
//   M = [[A_ci,ci , A_ci,ce L_ce,ge],
//        [D_ge,ci , D_ge,ce L_ce,ge]]          (size m + 4q, rows/cols [interior | Gauss])
// whose partial Gauss-Jordan elimination on the first m pivots yields F, S, H and T.
//
// A = -C11 D1^2 - 2 C12 D1 D2 - C22 D2^2 + C1 D1 + C2 D2 + C is never formed: each entry
// follows from the 1D tables (D1 = I (x) Dx and D2 = Dy (x) I, x fastest) in O(1).
// A_ci,ce L_ce,ge uses the side structure of L_ce,ge: a Gauss node on side s only sees the
// p Chebyshev nodes of side s (corner rows carry weight one half, the corner average of
// Eq. alpine2p5), with the side block Ls.  For an interior row only two terms of A reach a
// side: the cross term -2 c12 Dx Dy (through every node of the side) and the 1D operator
// along the row's own line (through the one node on that line).  With the table
// DLs = D Ls the p-term sum collapses to two products, e.g. on the south side
//   sum_t A[i][(t,0)] Ls[t][a] = -2 c12 sx sy D[iy][0] DLs[ix][a]
//                                + (-c22 sy^2 D2[iy][0] + c2 sy D[iy][0]) Ls[ix][a].
// The bottom rows are reference-element constants scaled by 2/h of the side's
// derivative direction.
#include <algorithm>

#include "hps_internal.h"

namespace hps {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) leaf_assemble_kernel(
    const double* __restrict__ coeffs, long long n_leaf_total, int leaf0, const double* __restrict__ hxy,
    int p, int q, LeafTablesDev tb, T* __restrict__ work, long long mat_stride) {
  const int lf = leaf0 + blockIdx.x;
  const int pp = p * p;
  const int m = (p - 2) * (p - 2);
  const int nq = 4 * q;
  const int R = m + nq;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* cf = reinterpret_cast<double*>(smraw);  // 6 * pp
  double* sD = cf + 6 * pp;                        // pp
  double* sD2 = sD + pp;                           // pp
  double* sLs = sD2 + pp;                          // p * q
  double* sLl = sLs + p * q;                       // q * p
  double* sDL = sLl + q * p;                       // p * q
  double* wrow = sDL + p * q;                      // per warp: 4 p row factors (see below)
  int* sci = reinterpret_cast<int*>(wrow + (blockDim.x >> 5) * 4 * p);  // m
  int* sjx = sci + m;                              // m: x index of interior node sci[j]
  int* sjy = sjx + m;                              // m: y index
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int e = tid; e < 6 * pp; e += bs) {
    const int k = e / pp, n = e - (e / pp) * pp;
    cf[e] = coeffs[((long long)k * n_leaf_total + lf) * pp + n];
  }
  for (int e = tid; e < pp; e += bs) { sD[e] = tb.D[e]; sD2[e] = tb.D2[e]; }
  for (int e = tid; e < p * q; e += bs) { sLs[e] = tb.Ls[e]; sLl[e] = tb.Lloc[e]; sDL[e] = tb.DLs[e]; }
  for (int e = tid; e < m; e += bs) {
    const int n = tb.ci[e];
    sci[e] = n;
    sjx[e] = n % p;
    sjy[e] = n / p;
  }
  __syncthreads();
  const double sx = 2.0 / hxy[2 * lf], sy = 2.0 / hxy[2 * lf + 1];
  T* M = work + (long long)blockIdx.x * mat_stride;
  // one warp per row (the row's coefficients and factors once), lanes along the row
  const int lane = tid & 31, nwarp = bs >> 5;
  for (int row = tid >> 5; row < R; row += nwarp) {
    T* Mr = M + (long long)row * R;
    if (row < m) {
      const int ni = sci[row], ix = sjx[row], iy = sjy[row];
      const double c11 = cf[ni], c12 = cf[pp + ni], c22 = cf[2 * pp + ni];
      const double c1 = cf[3 * pp + ni], c2 = cf[4 * pp + ni], c0 = cf[5 * pp + ni];
      // A[ni][(jx, jy)] for the operator of Sec. 3.2:
      //   al Dx[ix][jx] Dy[iy][jy] + [iy = jy] (bx D2[ix][jx] + gx D[ix][jx])
      //   + [ix = jx] (by D2[iy][jy] + gy D[iy][jy]) + [ix = jx, iy = jy] c0
      // The row's factors are formed once by the warp (ax = al Dx[ix][.], dy = Dy[iy][.],
      // lx = the iy = jy line term, ly = the ix = jx line term), so that an entry is one FMA
      // with its line term picked by selects: FP64 instructions under lane-divergent branches
      // would cost the whole warp's FP64 pipe time.
      const double al = -2.0 * c12 * sx * sy;
      const double bx = -c11 * sx * sx, gx = c1 * sx, by = -c22 * sy * sy, gy = c2 * sy;
      const double* Dix = sD + ix * p;
      const double* Diy = sD + iy * p;
      const double* D2ix = sD2 + ix * p;
      const double* D2iy = sD2 + iy * p;
      double* ax = wrow + (tid >> 5) * 4 * p;
      double* dy = ax + p;
      double* lx = dy + p;
      double* ly = lx + p;
      __syncwarp();
      for (int j = lane; j < p; j += 32) {
        ax[j] = al * Dix[j];
        dy[j] = Diy[j];
        lx[j] = bx * D2ix[j] + gx * Dix[j];
        ly[j] = by * D2iy[j] + gy * Diy[j];
      }
      __syncwarp();
      const double diag = lx[ix] + ly[iy] + c0;
      for (int col = lane; col < m; col += 32) {
        const int jx = sjx[col], jy = sjy[col];
        const double line = (iy == jy) ? ((ix == jx) ? diag : lx[jx]) : ((ix == jx) ? ly[jy] : 0.0);
        Mr[col] = (T)fma(ax[jx], dy[jy], line);
      }
      // exterior columns: side s, Gaussian node a; per side the two factors of the row
      //   horizontal sides (jy = 0, p-1): al Dy[iy][jy] DL[ix][a] + ly[jy] Ls[ix][a]
      //   vertical sides (jx = p-1, 0):   al Dx[ix][jx] DL[iy][a] + lx[jx] Ls[iy][a]
      for (int g = lane; g < nq; g += 32) {
        const int sd = g / q, a = g - sd * q;
        const bool hz = sd == 0 || sd == 2;
        const int jl = (sd == 0 || sd == 3) ? 0 : p - 1;
        const double f1 = hz ? al * dy[jl] : ax[jl];
        const double f2 = hz ? ly[jl] : lx[jl];
        const int li = (hz ? ix : iy) * q + a;
        Mr[m + g] = (T)fma(f1, sDL[li], f2 * sLs[li]);
      }
    } else {
      const int g = row - m, s = g / q, a = g - (g / q) * q;
      const double sc = (s == 0 || s == 2) ? sy : sx;
      for (int col = lane; col < m; col += 32) {
        const int nx = sjx[col], ny = sjy[col];
        double r;
        switch (s) {
          case 0: r = sLl[a * p + nx] * sD[0 * p + ny]; break;
          case 1: r = sLl[a * p + ny] * sD[(p - 1) * p + nx]; break;
          case 2: r = sLl[a * p + nx] * sD[(p - 1) * p + ny]; break;
          default: r = sLl[a * p + ny] * sD[0 * p + nx]; break;
        }
        Mr[col] = (T)(sc * r);
      }
      for (int c = lane; c < nq; c += 32) Mr[m + c] = (T)(sc * tb.DceL[(long long)g * nq + c]);
    }
  }
}

// flag = 1 when some leaf's coefficient at an interior node differs from leaf 0's (the
// exterior values are never used by the method).
__global__ void leaf_uniform_kernel(const double* __restrict__ coeffs, long long n_leaf, int p,
                                    int* __restrict__ flag) {
  const int pp = p * p;
  const long long total = 6 * n_leaf * pp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / (n_leaf * pp);
    const int n = (int)(e % pp);
    const int ix = n % p, iy = n / p;
    if (ix == 0 || ix == p - 1 || iy == 0 || iy == p - 1) continue;
    if (coeffs[e] != coeffs[k * n_leaf * pp + n]) *flag = 1;
  }
}

// Validity of the coefficient fields at the interior nodes (the exterior values are never
// used): out[0] receives the smallest leaf index with a non-finite coefficient, out[1] the
// smallest leaf index where the principal part is not elliptic (c11 <= 0 or
// c11 c22 - c12^2 <= 0, Eq. defA); both stay as the caller set them otherwise.
__global__ void coeff_check_kernel(const double* __restrict__ coeffs, long long n_leaf, int p,
                                   int* __restrict__ out) {
  const int pp = p * p;
  const long long total = n_leaf * pp, st = n_leaf * pp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e % pp);
    const int ix = n % p, iy = n / p;
    if (ix == 0 || ix == p - 1 || iy == 0 || iy == p - 1) continue;
    const int lf = (int)(e / pp);
    double c[6];
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      c[k] = coeffs[k * st + e];
      finite = finite && isfinite(c[k]);
    }
    if (!finite) atomicMin(out, lf);
    else if (!(c[0] > 0.0) || !(c[0] * c[2] - c[1] * c[1] > 0.0)) atomicMin(out + 1, lf);
  }
}

}  // namespace

void launch_coeff_check(const double* coeffs, int n_leaf, int p, int* out, cudaStream_t s) {
  const long long total = (long long)n_leaf * p * p;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  coeff_check_kernel<<<grid, 256, 0, s>>>(coeffs, n_leaf, p, out);
}

void launch_leaf_uniform_check(const double* coeffs, int n_leaf, int p, int* flag, cudaStream_t s) {
  const long long total = 6ll * n_leaf * p * p;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  leaf_uniform_kernel<<<grid, 256, 0, s>>>(coeffs, n_leaf, p, flag);
}

template <typename T>
void launch_leaf_assemble(const double* coeffs, long long n_leaf_total, int leaf0, int nleaf,
                          const double* hxy, int p, int q, const LeafTablesDev& tb, T* work,
                          long long mat_stride, cudaStream_t s) {
  const int pp = p * p, m = (p - 2) * (p - 2);
  const size_t smem = (size_t)(6 * pp + 2 * pp + 3 * p * q + 8 * 4 * p) * sizeof(double) + (size_t)3 * m * sizeof(int) + 16;
  ensure_smem((const void*)leaf_assemble_kernel<T>, smem);
  leaf_assemble_kernel<T><<<nleaf, 256, smem, s>>>(coeffs, n_leaf_total, leaf0, hxy, p, q, tb, work,
                                                  mat_stride);
}

template void launch_leaf_assemble<double>(const double*, long long, int, int, const double*, int, int,
                                           const LeafTablesDev&, double*, long long, cudaStream_t);

}  // namespace hps
