// FP32 batched gathered products on the tcgen05 tensor cores (the sweeps of the mixed-
// precision solve, Algorithm 2 with FP32 operators).
//
// Every FP32 entry x of the operator block and of the gathered vectors is split into three
// bf16 values x1 = rna(x), x2 = rna(x - x1), x3 = x - x1 - x2 (rna: rounded to 8 significant
// bits, ties away from zero; each difference is exact in FP32 and x3 has at most 8
// significant bits), so that x1 + x2 + x3 = x.  A product a b is the sum of the pairs
// a_s b_t; the pairs with s + t <= 4 are kept, the others together weigh below 2^-23 |a| |b|.  Per
// K slice of 16 the three products A_s [B_1 .. B_(4-s)] (one tcgen05.mma each, N = 64 (4 - s),
// the B planes side by side) write block t of their result to TMEM block s + t - 2, and the
// epilogue adds the three blocks: FP32 accumulation of exact bf16 x bf16 products, the
// accuracy of an FP32 product.
//
// Work unit: one item (<= 64 rows; MMA M = 128, rows 64..127 are padding that no epilogue
// reads) and 64 right-hand sides.  One CTA per SM loops over the units; a stage carries 64
// k (four K slices).  Roles (14 warps):
//   warps 0, 1, 4, 5   epilogue: TMEM lanes 0..63 (warp w reads lane quarter w % 4), 32
//                      right-hand sides each; adds the blocks, passes the 32 x 32 result
//                      through shared memory and stores whole rows (coalesced), with beta
//                      and Add;
//   warp 2             one thread issues the products of each stage;
//   warps 3, 6 .. 10,  producers (two per SM sub-partition): producer warp w copies 8 operator
//   12, 13             rows and 8 vector columns of every stage (16-byte cp.async where
//                      aligned, GPF stages ahead, the gathered rows' indices read a stage
//                      earlier) and splits them into the bf16 planes when the stage comes; no
//                      exchange leaves the warp;
//   warp 11            with cached operator planes (formed once per product set by
//                      gemm_tc32_pieces_kernel), one thread copies each stage's planes with
//                      one bulk copy and the producers only split the vectors.
// Stages (GST) and the two TMEM accumulators are handed on with mbarriers; every wait is
// bounded and a timeout stops every role (status -1).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "hps_internal.h"
#include "tc_common.cuh"

namespace hps {

namespace {

using namespace tc;

constexpr int T_GM = 128;           // MMA rows (item rows 0..63, the rest padding)
constexpr int T_GR = 64;            // item rows
constexpr int T_GN = 64;            // right-hand sides per unit
constexpr int T_PL = 3;             // bf16 pieces per entry
constexpr int T_KS = 64;            // k per stage
constexpr int T_NSUB = T_KS / 16;   // K slices (MMA K steps) per stage
constexpr int T_THREADS = 448;      // 14 warps
constexpr int T_LOAD_WARP = 11;     // bulk copies of cached operator planes
constexpr int T_PROD = 256;         // producer threads (8 warps)
constexpr int T_EPI = 128;          // epilogue threads (4 warps)
constexpr int T_MMA_WARP = 2;
constexpr int T_SPL = 2048;                 // bytes of one piece of one K slice (64 rows x 16 k x 2 B)
constexpr int T_ASTEP = T_PL * T_SPL;       // bytes of one K slice's operator pieces
constexpr int T_TBUF = 256;                 // TMEM columns between the two accumulators

// One stage: per K slice j, the three pieces' planes side by side (K-major, 8 x 16-byte core
// matrices, kmaj layout).  The B pieces of a slice are adjacent, so that one product with
// N = 64 t reads the first t of them as one operand.  A product (M = 128) reads 128 rows from
// an A plane's start: rows 64..127 are the following bytes (the next plane, or for the last
// plane of the last slice the first B plane), bf16 values that land in TMEM lanes 64..127,
// which no epilogue reads.
struct TStage {
  unsigned char A[T_NSUB][T_PL][T_SPL];
  unsigned char B[T_NSUB][T_PL][T_SPL];
};

// Pipeline depth.  With cached operator pieces a stage's planes arrive by one bulk copy
// issued when the stage is freed, so the copy's HBM latency is hidden only by the stages
// ahead of it: three stages, and raw slots for the vectors alone, the vector copies three
// stages ahead.  Without the cache the raw slots also hold the operator entries and two
// stages fit.
template <bool CACHED>
struct TCfg {
  static constexpr int GST = CACHED ? 3 : 2;         // stages
  static constexpr int GPF = CACHED ? 3 : 2;         // stages the entry copies run ahead
  static constexpr int GRAW = GPF + 1;               // raw entry slots
  static constexpr int AROWS = CACHED ? 1 : T_GR;    // raw operator rows (none used when cached)
};

// Entries of one stage as copied: the operator block row-major (64 rows x 64 k, the 16-byte
// chunks of row r at chunk index c ^ 4 (r & 1)) and the vector block k-major (64 k x 64
// right-hand sides, the 16-byte chunks of row k at c ^ 2 ((k >> 2) & 3)), so that the
// producers' reads in the split hit distinct banks.
template <bool CACHED>
struct TRawT {
  float A[TCfg<CACHED>::AROWS][T_KS];
  float B[T_KS][T_GN];
};

template <bool CACHED>
struct TSharedT {
  TStage st[TCfg<CACHED>::GST];
  TRawT<CACHED> raw[TCfg<CACHED>::GRAW];
  float ct[4][32][33];  // epilogue: each warp's 32 x 32 result tile, for coalesced stores
  int2 meta[8][TCfg<CACHED>::GRAW];  // per producer warp and raw slot: item rows, K slices (0: none)
  unsigned long long sfull[TCfg<CACHED>::GST], sfree[TCfg<CACHED>::GST], tfull[2], tfree[2], mdone;
  unsigned int tmem_base;
  int abort_flag;
};

static_assert(sizeof(TSharedT<true>) <= 232448 && sizeof(TSharedT<false>) <= 232448,
              "a CTA's shared memory exceeds the 227 KB opt-in limit");

__device__ __forceinline__ int swz_a(int row, int chunk) { return chunk ^ ((row & 1) << 2); }
__device__ __forceinline__ int swz_b(int k, int chunk) { return chunk ^ (((k >> 2) & 3) << 1); }

// x rounded to 8 significant bits, ties away from zero, as an FP32 bit pattern whose low 16
// bits are garbage (the caller masks or takes the high half).
__device__ __forceinline__ uint32_t rna8(float x) { return __float_as_uint(x) + 0x8000u; }

// The three bf16 pieces of 4 consecutive k of one row (column), one 8-byte store per plane;
// the planes of a slice are `plane_bytes` apart.
__device__ __forceinline__ void write_pieces4(const float* v, unsigned char* plane0, int plane_bytes, int off) {
  uint32_t p[T_PL][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float x = v[e];
    const uint32_t h1 = rna8(x);
    const float r1 = x - __uint_as_float(h1 & 0xffff0000u);   // exact
    const uint32_t h2 = rna8(r1);
    const float r2 = r1 - __uint_as_float(h2 & 0xffff0000u);  // exact, 8 significant bits
    p[0][e] = h1;
    p[1][e] = h2;
    p[2][e] = __float_as_uint(r2);
  }
#pragma unroll
  for (int s = 0; s < T_PL; ++s) {
    const uint32_t lo = __byte_perm(p[s][0], p[s][1], 0x7632), hi = __byte_perm(p[s][2], p[s][3], 0x7632);
    *reinterpret_cast<uint2*>(plane0 + s * plane_bytes + off) = make_uint2(lo, hi);
  }
}

__device__ __forceinline__ void zero_pieces4(unsigned char* plane0, int plane_bytes, int off) {
#pragma unroll
  for (int s = 0; s < T_PL; ++s) *reinterpret_cast<uint2*>(plane0 + s * plane_bytes + off) = make_uint2(0u, 0u);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Position of a CTA in its sequence of units (item ii, column block nb), advanced by the
// grid size without division.
struct UnitCur {
  int ii, nb;
};
struct UnitStep {
  int nnb, dq, dr;  // column blocks per item; grid = dq nnb + dr
  __device__ UnitCur first() const { return {(int)blockIdx.x / nnb, (int)blockIdx.x % nnb}; }
  __device__ void next(UnitCur& u) const {
    u.ii += dq;
    u.nb += dr;
    if (u.nb >= nnb) {
      u.nb -= nnb;
      ++u.ii;
    }
  }
};

// Stages of a unit's item: ceil(K / 64); K slices of stage c: min(4, ceil((K - 64 c) / 16)).
__device__ __forceinline__ int item_stages(int K) { return (K + T_KS - 1) / T_KS; }
__device__ __forceinline__ int stage_slices(int K, int c) { return min(T_NSUB, (K - c * T_KS + 15) >> 4); }

template <bool CACHED>
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
  constexpr int T_GST = TCfg<CACHED>::GST, T_GPF = TCfg<CACHED>::GPF, T_GRAW = TCfg<CACHED>::GRAW;
  using TRaw = TRawT<CACHED>;
  TSharedT<CACHED>& sh = *reinterpret_cast<TSharedT<CACHED>*>(t_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  UnitStep us;
  us.nnb = (nrhs + T_GN - 1) / T_GN;
  us.dq = (int)gridDim.x / us.nnb;
  us.dr = (int)gridDim.x % us.nnb;
  // cached operator planes (adig): one thread of the loader warp copies each stage's planes
  // with one bulk copy, and the producers only split the vectors
  constexpr bool cached = CACHED;
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
      int ks = 0, nu = 0;
      bool stop = false;
      UnitCur u = us.first();
      int K = u.ii < nitems ? items[u.ii].K : 0;
      for (; u.ii < nitems && !stop; ++nu) {
        UnitCur un = u;
        us.next(un);
        const int Kn = un.ii < nitems ? items[un.ii].K : 0;  // read a unit ahead of its use
        const int tb = nu & 1;
        if (nu >= 2 && !mb_wait(&sh.tfree[tb], ((nu >> 1) - 1) & 1, abort_flag, status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int nk = item_stages(K);
        for (int c = 0; c < nk; ++c, ++ks) {
          const int st = ks % T_GST;
          if (!mb_wait(&sh.sfull[st], (ks / T_GST) & 1, abort_flag, status)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int nsub = stage_slices(K, c);
#pragma unroll 1
          for (int j = 0; j < nsub; ++j) {
            const uint64_t bd = umma_desc(smem_u32(sh.st[st].B[j][0]), 128, 256);
#pragma unroll
            for (int sa = 1; sa <= T_PL; ++sa) {
              const int nt = T_PL + 1 - sa;  // B pieces 1 .. 4 - sa
              const uint64_t ad = umma_desc(smem_u32(sh.st[st].A[j][sa - 1]), 128, 256);
              const uint32_t idesc = idesc0 | ((uint32_t)((T_GN * nt) >> 3) << 17);
              const uint32_t acc = (c > 0 || j > 0 || sa > 1) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                      tmem + (uint32_t)(tb * T_TBUF + (sa - 1) * T_GN)),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&sh.sfree[st])));
        }
        if (stop) break;
        // (an item with K = 0 issues no product: the epilogue does not read its accumulator)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&sh.tfull[tb])));
        u = un;
        K = Kn;
      }
      // every product issued has completed before the TMEM is released
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&sh.mdone)));
      mb_drain(&sh.mdone, 0);
    }
  } else if (warp == T_LOAD_WARP) {
    // ---------------- cached operator planes: lane 0 copies each stage's planes into the
    // stage once it is free, arming the stage's barrier with their bytes
    if (cached && lane == 0) {
      int ks = 0;
      bool stop = false;
      UnitCur u = us.first();
      int K = 0;
      long long a0 = 0;
      if (u.ii < nitems) {
        K = items[u.ii].K;
        a0 = astep[u.ii];
      }
      for (; u.ii < nitems && !stop;) {
        UnitCur un = u;
        us.next(un);
        int Kn = 0;
        long long an = 0;
        if (un.ii < nitems) {  // read a unit ahead of their use
          Kn = items[un.ii].K;
          an = astep[un.ii];
        }
        const unsigned char* src = adig + a0 * T_ASTEP;
        const int nk = item_stages(K);
        for (int c = 0; c < nk; ++c, ++ks) {
          const int st = ks % T_GST;
          if (ks >= T_GST && !mb_wait(&sh.sfree[st], ((ks / T_GST) - 1) & 1, abort_flag, status)) {
            stop = true;
            break;
          }
          const uint32_t bytes = (uint32_t)stage_slices(K, c) * T_ASTEP;
          mb_expect_arrive(&sh.sfull[st], bytes);
          bulk_load(sh.st[st].A[0][0], src + (long long)c * T_NSUB * T_ASTEP, bytes, &sh.sfull[st]);
        }
        u = un;
        K = Kn;
        a0 = an;
      }
      // the copies issued have landed before the block exits
      for (int b = 0; b < T_GST; ++b) {
        const int n = ks > b ? (ks - 1 - b) / T_GST + 1 : 0;  // copies armed on stage b
        if (n > 0) mb_drain(&sh.sfull[b], (n - 1) & 1);
      }
    }
  } else if (!epi) {
    // ---------------- producers: warps 3, 6 .. 10, 12, 13 -> producer warp pw = 0 .. 7.  Warp
    // pw owns operator rows 8 pw .. 8 pw + 7 and vector columns 8 pw .. 8 pw + 7 of every
    // stage.  Lane l copies, GPF stages ahead, 4 consecutive k (16 j + 4 (l % 4), j = 0..3) of
    // operator row 8 pw + l / 4, and 4 consecutive right-hand sides 8 pw + 4 (l % 2) .. + 3 at
    // stage k = l / 2 + 16 j; when the stage comes it splits its own operator entries and the
    // vector entries of column 8 pw + l / 4 at k = 16 j + 4 (l % 4) .. + 3 into the bf16 planes,
    // so every exchange stays inside the warp.  The gathered vector rows' indices of a stage
    // are read one stage before its copies are issued, the next unit's item one unit ahead,
    // so that no copy waits for an index load.
    const int pw = warp == 3 ? 0 : (warp <= 10 ? warp - 5 : warp - 6);
    const int arow = 8 * pw + (lane >> 2), aq = lane & 3;       // operator row, k quad
    const int bkl = lane >> 1, bch = 2 * pw + (lane & 1);        // vector copy: k, 16-byte chunk
    const int bcol = 8 * pw + (lane >> 2);                       // vector split: column
    const bool bvec = (nrhs & 3) == 0 && ((reinterpret_cast<uintptr_t>(B0) | reinterpret_cast<uintptr_t>(B1)) & 15) == 0;
    struct Cur {
      UnitCur u, un;   // this unit and the next
      int c;           // stage within the unit
      GemmItem it, itn;
    };
    auto load_item = [&](const UnitCur& x, GemmItem& it) {
      if (x.ii < nitems) it = items[x.ii];
      else it.K = 0;
    };
    // to the next unit with K > 0 (or past the end)
    auto next_unit = [&](Cur& x) {
      do {
        x.u = x.un;
        x.it = x.itn;
        us.next(x.un);
        load_item(x.un, x.itn);
      } while (x.u.ii < nitems && x.it.K == 0);
      x.c = 0;
    };
    auto start_cur = [&](Cur& x) {
      x.un = us.first();
      load_item(x.un, x.itn);
      next_unit(x);
    };
    auto advance = [&](Cur& x) {
      if (x.u.ii >= nitems) return;
      if (++x.c >= item_stages(x.it.K)) next_unit(x);
    };
    // raw index entries of the gathered vector rows of this lane's 4 k at the cursor's stage
    auto load_rows = [&](const Cur& x, int (&r)[T_NSUB]) {
#pragma unroll
      for (int j = 0; j < T_NSUB; ++j) {
        r[j] = 0;
        if (x.u.ii >= nitems) continue;
        const int k = x.c * T_KS + 16 * j + bkl;
        if (k >= x.it.K) continue;
        if (k < x.it.kseg) {
          if (x.it.b0_idx >= 0) r[j] = idx[x.it.b0_idx + k];
        } else if (x.it.b1_idx >= 0) {
          r[j] = idx[x.it.b1_idx + k - x.it.kseg];
        }
      }
    };
    auto issue = [&](const Cur& x, const int (&r)[T_NSUB], int slot) {
      const bool valid = x.u.ii < nitems;
      const int nsub = valid ? stage_slices(x.it.K, x.c) : 0;
      if (lane == 0) sh.meta[pw][slot] = make_int2(valid ? x.it.M : 0, nsub);
      if (valid) {
        TRaw& rw = sh.raw[slot];
        const GemmItem& it = x.it;
        const int k0 = x.c * T_KS;
        if constexpr (!CACHED) {
        if (arow < it.M) {
          const float* srow = A + it.a_off + (long long)arow * it.lda;
#pragma unroll
          for (int j = 0; j < T_NSUB; ++j) {
            if (j >= nsub) continue;
            const int k = k0 + 16 * j + 4 * aq;
            float* dst = &rw.A[arow][4 * swz_a(arow, 4 * j + aq)];
            const float* src = srow + k;
            if (k + 3 < it.K && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
              cp_async16(dst, src);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                if (k + q < it.K) cp_async4(dst + q, src + q);
                else dst[q] = 0.f;
              }
            }
          }
        }
        }
        const int n = x.u.nb * T_GN + 4 * bch;
#pragma unroll
        for (int j = 0; j < T_NSUB; ++j) {
          if (j >= nsub) continue;
          const int kl = 16 * j + bkl, k = k0 + kl;
          float* dst = &rw.B[kl][4 * swz_b(kl, bch)];
          if (k < it.K) {
            const bool s1 = k >= it.kseg;
            const int kk = s1 ? k - it.kseg : k;
            const int row = (s1 ? it.b1_row : it.b0_row) + ((s1 ? it.b1_idx : it.b0_idx) >= 0 ? r[j] : kk);
            const float* src = (s1 ? B1 : B0) + (long long)row * nrhs + n;
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
      }
      cp_commit();  // one group per stage, empty past the end, so that the counts stay aligned
    };
    Cur x;  // the stage whose copies are issued next
    int r[T_NSUB];
    start_cur(x);
    load_rows(x, r);
    for (int i = 0; i < T_GPF; ++i) {
      issue(x, r, i);
      advance(x);
      load_rows(x, r);
    }
    for (int ks = 0;; ++ks) {
      cp_wait<T_GPF - 1>();  // this lane's copies of stage ks have landed
      __syncwarp();          // ... and every lane's of this warp
      const int st = ks % T_GST, slot = ks % T_GRAW;
      const int2 mt = sh.meta[pw][slot];
      if (mt.y == 0) break;
      if (ks >= T_GST && !warp_wait(&sh.sfree[st], ((ks / T_GST) - 1) & 1, abort_flag, status)) break;
      const TRaw& rw = sh.raw[slot];
      TStage& sg = sh.st[st];
      // every slice's entries are read first (slices past the stage's last read stale but
      // in-bounds entries and store nothing), so that the slices' splits are independent
      // chains the compiler interleaves
      if constexpr (!CACHED) {
        const int off = kmaj(arow, 4 * aq);
        float va[T_NSUB][4];
#pragma unroll
        for (int j = 0; j < T_NSUB; ++j) {
          const float4 a4 = *reinterpret_cast<const float4*>(&rw.A[arow][4 * swz_a(arow, 4 * j + aq)]);
          va[j][0] = a4.x;
          va[j][1] = a4.y;
          va[j][2] = a4.z;
          va[j][3] = a4.w;
        }
#pragma unroll
        for (int j = 0; j < T_NSUB; ++j) {
          if (j < mt.y) {
            if (arow >= mt.x) zero_pieces4(sg.A[j][0], T_SPL, off);
            else write_pieces4(va[j], sg.A[j][0], T_SPL, off);
          }
        }
      }
      float vb[T_NSUB][4];
#pragma unroll
      for (int j = 0; j < T_NSUB; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int kl = 16 * j + 4 * aq + q;
          vb[j][q] = rw.B[kl][4 * swz_b(kl, bcol >> 2) + (bcol & 3)];
        }
#pragma unroll
      for (int j = 0; j < T_NSUB; ++j)
        if (j < mt.y) write_pieces4(vb[j], sg.B[j][0], T_SPL, kmaj(bcol, 4 * aq));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mb_arrive(&sh.sfull[st]);
      // stage ks + GPF reuses the slot of stage ks - 1, which this warp finished reading before
      // the warp barrier above
      issue(x, r, (ks + T_GPF) % T_GRAW);
      advance(x);
      load_rows(x, r);  // first used by the next stage's issue
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
    for (UnitCur u = us.first(); u.ii < nitems; us.next(u), ++nu) {
      const GemmItem it = items[u.ii];
      const int n0 = u.nb * T_GN;
      const int tb = nu & 1;
      if (!warp_wait(&sh.tfull[tb], (nu >> 1) & 1, abort_flag, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
      for (int hh = 0; hh < 2; ++hh) {
        const int jb = 32 * g + 16 * hh;
        float r[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0.f;
        if (it.K > 0) {  // (no product wrote the accumulator of an item with K = 0)
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
      const int mymap = myrow < it.M ? (it.c_idx < 0 ? it.c_row + myrow : it.c_row + idx[it.c_idx + myrow]) : 0;
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

// The operator's bf16 pieces of every K slice of one item (one block per item), in the stage
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
      zero_pieces4(pl, T_SPL, kmaj(row, kg));
      continue;
    }
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = c * 16 + kg + q;
      v[q] = k < it.K ? A[it.a_off + (long long)row * it.lda + k] : 0.f;
    }
    write_pieces4(v, pl, T_SPL, kmaj(row, kg));
  }
}

}  // namespace

namespace {
// Self-test of the bounded waits: warp 0 waits on a barrier nothing arrives at (polls at
// most `polls` times), warp 1 waits on a second such barrier with the full limit but gives
// up as soon as the abort flag is raised; out[0] = the status word, out[1] = 1 if warp 1
// returned through the flag.
__global__ void wait_selftest_kernel(long long polls, int* out) {
  __shared__ unsigned long long bar[2];
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mb_init(&bar[0], 1);
    mb_init(&bar[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0 && lane == 0) mb_wait_n(&bar[0], 0, polls, &abort_flag, out);
  if (warp == 1 && lane == 0) {
    const bool ok = mb_wait(&bar[1], 0, &abort_flag, nullptr);
    out[1] = (!ok && abort_flag) ? 1 : 0;
  }
  __syncthreads();
}
}  // namespace

int wait_selftest(int polls, int* out_dev, cudaStream_t s) {
  wait_selftest_kernel<<<1, 64, 0, s>>>((long long)polls, out_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

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
    cudaFuncSetAttribute(gemm_tc32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(TSharedT<true>));
    cudaFuncSetAttribute(gemm_tc32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(TSharedT<false>));
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
  if (dg && dg->dig)
    gemm_tc32_kernel<true><<<grid, T_THREADS, sizeof(TSharedT<true>), s>>>(items, nitems, A, B0, B1, C, Add, idx, nrhs,
                                                                           (float)beta, dg->dig, dg->step, status);
  else
    gemm_tc32_kernel<false><<<grid, T_THREADS, sizeof(TSharedT<false>), s>>>(items, nitems, A, B0, B1, C, Add, idx,
                                                                             nrhs, (float)beta, nullptr, nullptr, status);
  return true;
}

}  // namespace hps
