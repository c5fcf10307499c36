// FP32 batched gathered products on the tcgen05 tensor cores (the sweeps of the mixed-
// precision solve, Algorithm 2 with FP32 operators).
//
// Every FP32 entry x of the operator block and of the gathered vectors is split into three
// bf16 values, x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2) (each difference is
// exact in FP32), so that x1 + x2 + x3 carries the 24 significant bits of x.  A product
// a b is the sum of the pairs a_s b_t; the pairs with s + t <= 4 are kept, the others weigh
// below 2^-24 |a| |b|.  Per K step of 16 the three products A_s [B_1 .. B_(4-s)] (one
// tcgen05.mma each, N = 64 (4 - s), the B planes side by side) write block t of their
// result to TMEM block s + t - 2, and the epilogue adds the three blocks: FP32
// accumulation of exact bf16 x bf16 products, the accuracy of an FP32 product.
//
// Work unit: one item (<= 64 rows; MMA M = 128, rows 64..127 are padding that no epilogue
// reads) and 64 right-hand sides.  One CTA per SM loops over the units.  Roles (13 warps):
//   warps 0, 1, 4, 5   epilogue: TMEM lanes 0..63 (warp w reads lane quarter w % 4), 32
//                      right-hand sides each; adds the blocks, passes the 32 x 32 result
//                      through shared memory and stores whole rows (coalesced), with beta
//                      and Add;
//   warp 2             one thread issues the products of each K step;
//   warps 3, 6 .. 12   producers: warp w copies 8 operator rows and 8 vector columns of every
//                      K step (16-byte cp.async where aligned, GPF steps ahead, the gathered
//                      rows' indices read a step earlier) and splits them into the three bf16
//                      planes when the step comes; no exchange leaves the warp.
//   warp 13            with cached operator planes (formed once per product set by
//                      gemm_tc32_pieces_kernel), one thread copies each K step's planes with
//                      one bulk copy and the producers only split the vectors.
// Stages (GST) and the two TMEM accumulators are handed on with mbarriers; every wait is
// bounded and a timeout stops every role (status -1).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include <cuda_bf16.h>

#include "hps_internal.h"
#include "tc_common.cuh"

namespace hps {

namespace {

using namespace tc;

constexpr int T_GM = 128;           // MMA rows (item rows 0..63, the rest padding)
constexpr int T_GR = 64;            // item rows
constexpr int T_GN = 64;            // right-hand sides per unit
constexpr int T_PL = 3;             // bf16 pieces per entry
constexpr int T_GST = 4;            // K-step stages
constexpr int T_GPF = 4;            // K steps the entry copies run ahead
constexpr int T_GRAW = T_GPF + 1;   // raw entry slots
constexpr int T_THREADS = 448;      // 14 warps
constexpr int T_LOAD_WARP = 13;     // bulk copies of cached operator planes
constexpr int T_PROD = 256;         // producer threads (8 warps)
constexpr int T_EPI = 128;          // epilogue threads (4 warps)
constexpr int T_MMA_WARP = 2;
constexpr int T_APL = T_GR * 32;            // bytes per A plane (64 rows x 16 k x 2 B)
constexpr int T_BPL = T_GN * 32;            // bytes per B plane (64 columns x 16 k x 2 B)
constexpr int T_TBUF = 256;                 // TMEM columns between the two accumulators
constexpr int T_ASTEP = T_PL * T_APL;       // bytes of one K step's operator planes

// One K step.  A product (M = 128) reads 128 rows from an A plane's start: rows 64..127
// are the next plane's bytes (for the last plane, the first B plane's), bf16 values that
// land in TMEM lanes 64..127, which no epilogue reads.
struct TStage {
  unsigned char A[T_PL][T_APL];
  unsigned char B[T_PL][T_BPL];
};

// Entries of one K step as copied: the operator block row-major (64 rows x 16 k) and the
// vector block k-major (16 k x 64 right-hand sides), so that each producer thread moves one
// 16-byte piece of each.
struct TRaw {
  float A[T_GR][16];
  float B[16][T_GN];
};

struct TShared {
  TStage st[T_GST];
  TRaw raw[T_GRAW];
  float ct[4][32][33];  // epilogue: each warp's 32 x 32 result tile, for coalesced stores
  unsigned long long sfull[T_GST], sfree[T_GST], tfull[2], tfree[2], mdone;
  unsigned int tmem_base;
  int abort_flag;
};

// The three bf16 pieces of 4 consecutive k of one row (column), one 8-byte store per plane.
__device__ __forceinline__ void write_pieces4(const float* v, unsigned char* plane0, int plane_bytes, int off) {
  uint32_t w[T_PL][2];
#pragma unroll
  for (int q = 0; q < 4; q += 2) {
    uint32_t lo[T_PL], hi[T_PL];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float x = v[q + e];
#pragma unroll
      for (int s = 0; s < T_PL; ++s) {
        const __nv_bfloat16 b = __float2bfloat16_rn(x);
        x = x - __bfloat162float(b);  // exact: b is x rounded to 8 significant bits
        const uint32_t bits = (uint32_t)__bfloat16_as_ushort(b);
        if (e == 0) lo[s] = bits;
        else hi[s] = bits;
      }
    }
#pragma unroll
    for (int s = 0; s < T_PL; ++s) w[s][q / 2] = lo[s] | (hi[s] << 16);
  }
#pragma unroll
  for (int s = 0; s < T_PL; ++s)
    *reinterpret_cast<uint2*>(plane0 + s * plane_bytes + off) = make_uint2(w[s][0], w[s][1]);
}

__device__ __forceinline__ void zero_pieces4(unsigned char* plane0, int plane_bytes, int off) {
#pragma unroll
  for (int s = 0; s < T_PL; ++s) *reinterpret_cast<uint2*>(plane0 + s * plane_bytes + off) = make_uint2(0u, 0u);
}

__device__ __forceinline__ int map_row32(const int* __restrict__ idx, int base_or_off, int row_base, int k) {
  return base_or_off < 0 ? row_base + k : row_base + idx[base_or_off + k];
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}


__global__ void __launch_bounds__(T_THREADS, 1) gemm_tc32_kernel(const GemmItem* __restrict__ items, int nitems,
                                                                 const float* __restrict__ A,
                                                                 const float* __restrict__ B0,
                                                                 const float* __restrict__ B1, float* __restrict__ C,
                                                                 const float* __restrict__ Add,
                                                                 const int* __restrict__ idx, int nrhs, float beta,
                                                                 const unsigned char* __restrict__ adig,
                                                                 const long long* __restrict__ astep,
                                                                 int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char t_raw[];
  TShared& sh = *reinterpret_cast<TShared*>(t_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nnb = (nrhs + T_GN - 1) / T_GN;
  const long long total = (long long)nitems * nnb;
  // cached operator planes (adig): one thread of the loader warp copies each K step's planes
  // with one bulk copy, and the producers only split the vectors
  const bool cached = adig != nullptr;
  if (tid == 0) {
    for (int b = 0; b < T_GST; ++b) {
      mb_init(&sh.sfull[b], cached ? T_PROD + 1 : T_PROD);
      mb_init(&sh.sfree[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mb_init(&sh.tfull[b], 1);
      mb_init(&sh.tfree[b], T_EPI);
    }
    mb_init(&sh.mdone, 1);
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == T_MMA_WARP) {
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
  const bool epi = warp == 0 || warp == 1 || warp == 4 || warp == 5;

  if (warp == T_MMA_WARP) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      // kind::f16 with bf16 A and B, FP32 accumulators, M = 128; N set per product
      const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(T_GM >> 4) << 24);
      long long ks = 0;
      int nu = 0;
      bool stop = false;
      for (long long u = blockIdx.x; u < total && !stop; u += gridDim.x, ++nu) {
        const GemmItem it = items[u / nnb];
        const int nk = (it.K + 15) >> 4;
        const int tb = nu & 1;
        if (nu >= 2 && !mb_wait(&sh.tfree[tb], ((nu >> 1) - 1) & 1, abort_flag, status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int c = 0; c < nk; ++c, ++ks) {
          const int st = (int)(ks % T_GST);
          if (!mb_wait(&sh.sfull[st], (int)((ks / T_GST) & 1), abort_flag, status)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = smem_u32(sh.st[st].A[0]), b0 = smem_u32(sh.st[st].B[0]);
#pragma unroll 1
          for (int sa = 1; sa <= T_PL; ++sa) {
            const int nt = T_PL + 1 - sa;  // B pieces 1 .. 4 - sa
            const uint64_t ad = umma_desc(a0 + (sa - 1) * T_APL, 128, 256);
            const uint64_t bd = umma_desc(b0, 128, 256);
            const uint32_t idesc = idesc0 | ((uint32_t)((T_GN * nt) >> 3) << 17);
            const uint32_t acc = (c > 0 || sa > 1) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                    tmem + (uint32_t)(tb * T_TBUF + (sa - 1) * T_GN)),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&sh.sfree[st])));
        }
        if (stop) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&sh.tfull[tb])));
      }
      // every product issued has completed before the TMEM is released
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&sh.mdone)));
      mb_drain(&sh.mdone, 0);
    }
  } else if (warp == T_LOAD_WARP) {
    // ---------------- cached operator planes: lane 0 copies each K step's planes into its
    // stage once the stage is free, arming the stage's barrier with their bytes
    if (cached && lane == 0) {
      long long ks = 0;
      bool stop = false;
      for (long long u = blockIdx.x; u < total && !stop; u += gridDim.x) {
        const long long item = u / nnb;
        const int nk = (items[item].K + 15) >> 4;
        const unsigned char* src = adig + astep[item] * T_ASTEP;
        for (int c = 0; c < nk; ++c, ++ks) {
          const int st = (int)(ks % T_GST);
          if (ks >= T_GST && !mb_wait(&sh.sfree[st], (int)((ks / T_GST) - 1) & 1, abort_flag, status)) {
            stop = true;
            break;
          }
          mb_expect_arrive(&sh.sfull[st], T_ASTEP);
          bulk_load(sh.st[st].A[0], src + (long long)c * T_ASTEP, T_ASTEP, &sh.sfull[st]);
        }
      }
      // the copies issued have landed before the block exits
      for (int b = 0; b < T_GST; ++b) {
        const long long n = ks > b ? (ks - 1 - b) / T_GST + 1 : 0;  // copies armed on stage b
        if (n > 0) mb_drain(&sh.sfull[b], (int)((n - 1) & 1));
      }
    }
  } else if (!epi) {
    // ---------------- producers: warps 3, 6 .. 12 -> producer warp pw = 0 .. 7.  Warp pw owns
    // operator rows 8 pw .. 8 pw + 7 and vector columns 8 pw .. 8 pw + 7 of every K step: it
    // copies them GPF steps ahead (lane l: 4 consecutive k of row 8 pw + l / 4; 4 consecutive
    // right-hand sides 8 pw + 4 (l % 2) .. + 3 at k = l / 2) and, when the step comes, splits
    // them into the bf16 planes (lane l: 4 k of row 8 pw + l / 4 and of column 8 pw + l / 4),
    // so every exchange stays inside the warp.  The item of a step and the gathered vector row
    // of the lane's k are read one step before the step's copies are issued (the next unit's
    // item one unit ahead), so that no copy waits for an index load.
    const int pw = warp == 3 ? 0 : warp - 5;
    const int arow = 8 * pw + (lane >> 2), akq = (lane & 3) * 4;  // operator row: copy and split
    const int bk = lane >> 1, bnq = 8 * pw + (lane & 1) * 4;        // vector copy
    const int bcol = 8 * pw + (lane >> 2), bkg = (lane & 3) * 4;    // vector split
    const bool bvec = (nrhs & 3) == 0 && ((reinterpret_cast<uintptr_t>(B0) | reinterpret_cast<uintptr_t>(B1)) & 15) == 0;
    struct Cur {
      long long u;
      int c;
      GemmItem it, itn;  // the unit's item and the next unit's
    };
    auto start_cur = [&](Cur& x) {
      x.u = blockIdx.x;
      x.c = 0;
      if (x.u < total) x.it = items[x.u / nnb];
      if (x.u + gridDim.x < total) x.itn = items[(x.u + gridDim.x) / nnb];
    };
    auto step_cur = [&](Cur& x) {
      if (x.u >= total) return;
      if (++x.c >= ((x.it.K + 15) >> 4)) {
        x.c = 0;
        x.u += gridDim.x;
        x.it = x.itn;
        if (x.u + gridDim.x < total) x.itn = items[(x.u + gridDim.x) / nnb];
      }
    };
    // gathered vector row of this lane's k at the cursor's step: 2 row + (1 for B1), or -1
    auto brow_of = [&](const Cur& x) -> long long {
      if (x.u >= total) return -1;
      const int k = x.c * 16 + bk;
      if (k >= x.it.K) return -1;
      return k < x.it.kseg ? 2ll * map_row32(idx, x.it.b0_idx, x.it.b0_row, k)
                           : 2ll * map_row32(idx, x.it.b1_idx, x.it.b1_row, k - x.it.kseg) + 1;
    };
    auto issue = [&](const Cur& x, long long brow, int slot) {
      if (x.u < total) {
        TRaw& rw = sh.raw[slot];
        const GemmItem& it = x.it;
        const int n0 = (int)(x.u % nnb) * T_GN, k0 = x.c * 16;
        if (!cached && arow < it.M) {
          float* dst = &rw.A[arow][akq];
          const float* src = A + it.a_off + (long long)arow * it.lda + k0 + akq;
          if (k0 + akq + 3 < it.K && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            cp_async16(dst, src);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (k0 + akq + q < it.K) cp_async4(dst + q, src + q);
              else dst[q] = 0.f;
            }
          }
        }
        float* dst = &rw.B[bk][bnq];
        const int n = n0 + bnq;
        if (brow >= 0) {
          const float* src = ((brow & 1) ? B1 : B0) + (brow >> 1) * nrhs + n;
          if (bvec && n + 3 < nrhs) {
            cp_async16(dst, src);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (n + q < nrhs) cp_async4(dst + q, src + q);
              else dst[q] = 0.f;
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = 0.f;
        }
      }
      cp_commit();  // one group per step, empty past the end, so that the counts stay aligned
    };
    Cur cv, is, la;  // conversion (step ks), issue (ks + GPF), look-ahead (ks + GPF + 1)
    start_cur(cv);
    start_cur(is);
    long long brow = brow_of(is);
    for (int i = 0; i < T_GPF; ++i) {
      issue(is, brow, i % T_GRAW);
      step_cur(is);
      brow = brow_of(is);
    }
    la = is;
    step_cur(la);
    long long ks = 0;
    while (cv.u < total) {
      cp_wait<T_GPF - 1>();  // this lane's copies of step ks have landed
      __syncwarp();          // ... and every lane's of this warp
      const int st = (int)(ks % T_GST), slot = (int)(ks % T_GRAW);
      if (ks >= T_GST && !warp_wait(&sh.sfree[st], (int)((ks / T_GST) - 1) & 1, abort_flag, status)) break;
      const TRaw& rw = sh.raw[slot];
      if (!cached) {
        if (arow >= cv.it.M) zero_pieces4(sh.st[st].A[0], T_APL, kmaj(arow, akq));
        else write_pieces4(&rw.A[arow][akq], sh.st[st].A[0], T_APL, kmaj(arow, akq));
      }
      {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = rw.B[bkg + q][bcol];
        write_pieces4(v, sh.st[st].B[0], T_BPL, kmaj(bcol, bkg));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mb_arrive(&sh.sfull[st]);
      // step ks + GPF reuses the slot of step ks - 1, which this warp finished reading
      // before the warp barrier above
      const long long brow_la = brow_of(la);  // read a step ahead of its use
      issue(is, brow, (int)((ks + T_GPF) % T_GRAW));
      is = la;
      brow = brow_la;
      step_cur(la);
      step_cur(cv);
      ++ks;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // copies still in flight land before exit
  } else {
    // ---------------- epilogue: warps 0, 1, 4, 5; the warp owns rows 32 (w % 4) .. + 31
    // and right-hand sides 32 g .. 32 g + 31 (g = w / 4) of the unit.  Lane l reads its row's
    // 32 sums from TMEM (16 columns at a time, the three blocks added), the warp passes them
    // through its shared tile, and each of its 32 rows is then stored by the 32 lanes at
    // consecutive right-hand sides.
    const int g = warp >> 2, ew = (warp & 1) + 2 * g;  // tile of this warp
    float (*tile)[33] = sh.ct[ew];
    int nu = 0;
    for (long long u = blockIdx.x; u < total; u += gridDim.x, ++nu) {
      const GemmItem it = items[u / nnb];
      const int n0 = (int)(u % nnb) * T_GN;
      const int tb = nu & 1;
      if (!warp_wait(&sh.tfull[tb], (nu >> 1) & 1, abort_flag, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
      for (int hh = 0; hh < 2; ++hh) {
        const int jb = 32 * g + 16 * hh;
        float r[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0.f;
#pragma unroll
        for (int d = 0; d < T_PL; ++d) {
          uint32_t v[16];
          const uint32_t addr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(tb * T_TBUF + d * T_GN + jb);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(addr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int j = 0; j < 16; ++j) r[j] += __uint_as_float(v[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) tile[lane][16 * hh + j] = r[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      mb_arrive(&sh.tfree[tb]);  // accumulator read: the unit after next may write it
      __syncwarp();
      // the 32 rows' output addresses (one row index per lane, broadcast), the old values and
      // addends all requested before any store, so that the row loop does not wait on them
      // one by one
      const int n = n0 + 32 * g + lane;
      const int myrow = q4 * 32 + lane;
      const int mymap = myrow < it.M ? map_row32(idx, it.c_idx, it.c_row, myrow) : 0;
      const int nrow = min(32, it.M - q4 * 32);
      const bool col_ok = n < nrhs;
      float o[32];
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) o[rr] = tile[rr][lane];
      if (it.add_row >= 0) {
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
          if (rr < nrow && col_ok) o[rr] += Add[(long long)(it.add_row + q4 * 32 + rr) * nrhs + n];
      }
      if (beta != 0.f) {
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
          const int rmap = __shfl_sync(0xffffffffu, mymap, rr);
          if (rr < nrow && col_ok) o[rr] += beta * C[(long long)rmap * nrhs + n];
        }
      }
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) {
        const int rmap = __shfl_sync(0xffffffffu, mymap, rr);
        if (rr < nrow && col_ok) C[(long long)rmap * nrhs + n] = o[rr];
      }
      __syncwarp();  // the tile is rewritten for the next unit
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == T_MMA_WARP) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// The operator's bf16 pieces of every K step of one item (one block per item), in the stage
// layout, at adig + astep[item] * T_ASTEP; rows past the item are zero.  The operators do not
// change after the build, so a product set keeps these planes across solves.
__global__ void __launch_bounds__(256) gemm_tc32_pieces_kernel(const GemmItem* __restrict__ items,
                                                               const float* __restrict__ A,
                                                               const long long* __restrict__ astep,
                                                               unsigned char* __restrict__ adig) {
  const GemmItem it = items[blockIdx.x];
  const int t = threadIdx.x, row = t >> 2, kg = (t & 3) * 4;
  unsigned char* dst = adig + astep[blockIdx.x] * T_ASTEP;
  const int nk = (it.K + 15) >> 4;
  for (int c = 0; c < nk; ++c) {
    unsigned char* pl = dst + (long long)c * T_ASTEP;
    if (row >= it.M) {
      zero_pieces4(pl, T_APL, kmaj(row, kg));
      continue;
    }
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = c * 16 + kg + q;
      v[q] = k < it.K ? A[it.a_off + (long long)row * it.lda + k] : 0.f;
    }
    write_pieces4(v, pl, T_APL, kmaj(row, kg));
  }
}

}  // namespace

bool gemm_tc32_eligible(int nrhs) { return nrhs > 8; }

long long gemm_tc32_piece_bytes(long long steps) { return steps * T_ASTEP; }

void launch_gemm_tc32_pieces(const GemmItem* items, int nitems, const float* A, const long long* astep,
                             unsigned char* adig, cudaStream_t s) {
  if (nitems <= 0) return;
  gemm_tc32_pieces_kernel<<<(unsigned)nitems, 256, 0, s>>>(items, A, astep, adig);
}

namespace {
constexpr int kTc32MaxDev = 64;
std::mutex g_tc32_mu;
int g_tc32_nsm[kTc32MaxDev] = {0};

// SM count and the kernel's shared-memory limit of the current device, set once per device.
int tc32_nsm() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTc32MaxDev) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(g_tc32_mu);
  if (!g_tc32_nsm[dev]) {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(gemm_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TShared));
    if (cudaGetLastError() != cudaSuccess) return 0;
    g_tc32_nsm[dev] = nsm > 0 ? nsm : 1;
  }
  return g_tc32_nsm[dev];
}
}  // namespace

void gemm_tc32_prepare() { (void)tc32_nsm(); }

bool launch_gemm_tc32(const GemmItem* items, int nitems, const float* A, const float* B0, const float* B1, float* C,
                      const float* Add, const int* idx, int nrhs, double beta, int* status, cudaStream_t s,
                      const GemmDigits* dg) {
  if (nitems <= 0) return true;
  const int nsm = tc32_nsm();
  if (!nsm) return false;
  const long long units = (long long)nitems * ((nrhs + T_GN - 1) / T_GN);
  const int grid = (int)std::min<long long>(nsm, units);
  gemm_tc32_kernel<<<grid, T_THREADS, sizeof(TShared), s>>>(items, nitems, A, B0, B1, C, Add, idx, nrhs, (float)beta,
                                                            dg ? dg->dig : nullptr, dg ? dg->step : nullptr, status);
  return true;
}

}  // namespace hps
