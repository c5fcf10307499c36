// Merge assembly (Sec. 4, Algorithm 1 merge branch).  For a parent tau with children
// alpha and beta, rows and columns ordered [J3 | J1 | J2]:
//   M_tau = [[ T33a - T33b , -T31a , T32b ],
//            [ -T13a       ,  T11a , 0    ],
//            [ -T23b       ,  0    , T22b ]]
// Partial Gauss-Jordan on the first |J3| pivots then leaves X = (T33a - T33b)^-1,
// S = X [-T31a | T32b], C X and T_tau = blkdiag(T11a, T22b) + [T13a; T23b] S in place.
// posA / posB give each row's position in alpha's / beta's exterior list (or -1), so an
// entry is  sa * Ta[posA r][posA c] + sb * Tb[posB r][posB c]  with the signs above.
#include <algorithm>

#include "hps_internal.h"

namespace hps {

namespace {

template <typename T, typename TT>
__global__ void __launch_bounds__(256) merge_assemble_kernel(const MergeDesc* __restrict__ d,
                                                             const TT* __restrict__ tstore,
                                                             const int* __restrict__ pos,
                                                             T* __restrict__ work) {
  const MergeDesc md = d[blockIdx.y];
  const int R = md.R, k3 = md.k3;
  const int* pA = pos + md.pos_off;
  const int* pB = pA + R;
  const TT* Ta = tstore + md.ta_off;
  const TT* Tb = tstore + md.tb_off;
  T* M = work + md.m_off;
  // one warp per row, lanes along it.  The children's blocks enter with signs +1 or -1
  // (flipped on the integer pipe); only the pivot block Z = T33a - T33b adds two values,
  // and its entries fill whole warps, so no FP64 instruction sits under a divergent branch
  auto neg = [](double x) { return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull); };
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = blockIdx.x * nw + (threadIdx.x >> 5); r < md.rows; r += gridDim.x * nw) {
    const int ar = pA[r], br = pB[r];
    const bool rtop = r < k3;
    const TT* Tar = Ta + (long long)(ar >= 0 ? ar : 0) * md.lda_a;
    const TT* Tbr = Tb + (long long)(br >= 0 ? br : 0) * md.lda_b;
    T* Mr = M + (long long)r * R;
    for (int c = lane; c < R; c += 32) {
      const int ac = pA[c], bc = pB[c];
      const bool ctop = c < k3;
      const bool ha = ar >= 0 && ac >= 0, hb = br >= 0 && bc >= 0;
      double va = ha ? (double)Tar[ac] : 0.0, vb = hb ? (double)Tbr[bc] : 0.0;
      if (rtop != ctop) va = neg(va);  // sa = -1 off the diagonal blocks
      if (ctop) vb = neg(vb);          // sb = -1 in the first k3 columns
      double v;
      if (ha && hb) v = va + vb;
      else v = ha ? va : vb;
      Mr[c] = (T)v;
    }
  }
}

// Root-condition matrices (periodic seam, Neumann nodes): entry (r, c) is
// sum over (i, si) of row r and (j, sj) of column c of si sj src[i][j], with up to two
// terms each, negated in the off-diagonal blocks (r < K) != (c < K) when flip is set.
__global__ void __launch_bounds__(256) comb_assemble_kernel(CombAsm a, const double* __restrict__ src,
                                                            const int* __restrict__ idx,
                                                            double* __restrict__ dst) {
  const long long total = (long long)a.rows * a.R;
  const int* rt = idx + a.rt;
  const int* ct = idx + a.ct;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / a.R), c = (int)(e - (e / a.R) * a.R);
    double v = 0.0;
    for (int u = 0; u < 2; ++u) {
      const int i = rt[4 * r + 2 * u];
      if (i < 0) continue;
      const double si = (double)rt[4 * r + 2 * u + 1];
      for (int w = 0; w < 2; ++w) {
        const int j = ct[4 * c + 2 * w];
        if (j < 0) continue;
        v += si * (double)ct[4 * c + 2 * w + 1] * src[(long long)i * a.ld + j];
      }
    }
    if (a.flip && ((r < a.K) != (c < a.K))) v = -v;
    dst[e] = v;
  }
}

__global__ void __launch_bounds__(256) bgemm_kernel(const BGemm* __restrict__ d, const double* __restrict__ A,
                                                    const double* __restrict__ B, double* __restrict__ C) {
  const BGemm g = d[blockIdx.y];
  const int tilesN = (g.N + 15) / 16;
  const int ti = blockIdx.x / tilesN, tj = blockIdx.x - (blockIdx.x / tilesN) * tilesN;
  const int i = ti * 16 + (threadIdx.x >> 4), j = tj * 16 + (threadIdx.x & 15);
  if (ti * 16 >= g.M) return;
  __shared__ double As[16][17], Bs[16][17];
  double acc = 0.0;
  for (int k0 = 0; k0 < g.K; k0 += 16) {
    const int r = threadIdx.x >> 4, c = threadIdx.x & 15;
    const int ai = ti * 16 + r, ak = k0 + c, bk = k0 + r, bj = tj * 16 + c;
    As[r][c] = (ai < g.M && ak < g.K) ? A[g.a_off + (long long)ai * g.lda + ak] : 0.0;
    Bs[r][c] = (bk < g.K && bj < g.N) ? B[g.b_off + (long long)bk * g.ldb + bj] : 0.0;
    __syncthreads();
    for (int k = 0; k < 16; ++k) acc += As[threadIdx.x >> 4][k] * Bs[k][threadIdx.x & 15];
    __syncthreads();
  }
  if (i < g.M && j < g.N) C[g.c_off + (long long)i * g.ldc + j] = acc;
}

}  // namespace

void launch_bgemm(const BGemm* d, int n, int maxM, int maxN, const double* A, const double* B, double* C,
                  cudaStream_t s) {
  if (n <= 0) return;
  const int tiles = ((maxM + 15) / 16) * ((maxN + 15) / 16);
  bgemm_kernel<<<dim3(tiles, n), 256, 0, s>>>(d, A, B, C);
}

template <typename T, typename TT>
void launch_merge_assemble(const MergeDesc* d, int nmat, int maxR, const TT* tstore, const int* pos,
                           T* work, cudaStream_t s) {
  int gx = (maxR + 7) / 8;  // one warp per row, 8 per block
  if (gx > 2048) gx = 2048;
  merge_assemble_kernel<T, TT><<<dim3(gx, nmat), 256, 0, s>>>(d, tstore, pos, work);
}

void launch_comb_assemble(const CombAsm& a, const double* src, const int* idx, double* dst, cudaStream_t s) {
  const long long total = (long long)a.rows * a.R;
  const int grid = (int)std::min<long long>((total + 255) / 256, 4096);
  comb_assemble_kernel<<<grid, 256, 0, s>>>(a, src, idx, dst);
}

template void launch_merge_assemble<double, double>(const MergeDesc*, int, int, const double*, const int*,
                                                    double*, cudaStream_t);
template void launch_merge_assemble<float, double>(const MergeDesc*, int, int, const double*, const int*,
                                                   float*, cudaStream_t);

}  // namespace hps
