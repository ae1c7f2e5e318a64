// Complex-FP32 GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32) for sm_103a.
//
// C = beta*C + alpha*A*B with complex A (m x k), B (k x n), C (m x n), interleaved (re, im),
// row-major.  The complex product is computed in real ("4M", realified) form:
//   Cr (m x 2n) = Ar (m x 2k) * Br (2k x 2n),
// where Ar and Cr are the interleaved storage read as real matrices and each complex B[p][j]
// becomes the 2x2 real block [[re, im], [-im, re]] of Br.  FP32 accuracy comes from the 3xTF32
// split x = hi + lo (hi = x rounded to TF32): A*B ~ Ahi*Bhi + Ahi*Blo + Alo*Bhi, accumulated
// in FP32 in tensor memory.
//
// Operands are first packed (and split) into tiles already laid out in the UMMA K-major
// 128-byte-swizzled shared-memory format: A tiles of 128 rows x 32 floats (16 KB), B tiles of
// 256 rows x 32 floats (32 KB).  A CTA computes one 128 x 256 tile of Cr: one thread streams the
// tiles into shared memory with 1-D bulk copies (cp.async.bulk, completion on an mbarrier), one
// thread issues tcgen05.mma into a 256-column TMEM accumulator, and four warps read the
// accumulator back with tcgen05.ld for the epilogue.  Every mbarrier wait is bounded; on time-out
// the kernel records DS_WAIT_TIMEOUT and skips its output.  The kernel is persistent: one CTA per
// SM walks a static round-robin list of all output tiles of all batch items, with two TMEM
// accumulators so that draining tile i overlaps the MMAs of tile i+1.
#include "dense.cuh"
#include "tc_gemm.cuh"
#include "tc_tune.h"

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>

namespace rfdd {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_BK = 32;
constexpr int TC_STAGES = 2;
constexpr int A_TILE = TC_BM * TC_BK;  // floats
constexpr int B_TILE = TC_BN * TC_BK;  // floats
constexpr int STAGE_BYTES = (2 * A_TILE + 2 * B_TILE) * 4;  // 96 KB
constexpr int EPI_WARPS = 8;  // two per TMEM lane quarter, each drains half of the columns
constexpr int EPI_PITCH = 33;
constexpr int EPI_BYTES = EPI_WARPS * 32 * EPI_PITCH * 4;
constexpr int TC_THREADS = 64 + 32 * EPI_WARPS;  // producer warp, MMA warp, epilogue warps
constexpr int TC_SMEM = TC_STAGES * STAGE_BYTES + EPI_BYTES + 1024;
constexpr long long WAIT_LIMIT = 1ll << 24;

// Status word of the launches issued by the calling host thread (TcStatusScope): a kernel whose
// bounded wait ran out ORs DS_WAIT_TIMEOUT into it.  Each handle passes its own word, so a
// failure is reported by the solve that met it and by no other.
thread_local int *g_tc_status = nullptr;

TcStatusScope::TcStatusScope(int *w) : prev(g_tc_status) { g_tc_status = w; }
TcStatusScope::~TcStatusScope() { g_tc_status = prev; }

// Events recorded around the tensor-core kernel launches of the calling host thread (probes).
thread_local const cudaEvent_t *g_tc_events = nullptr;
TcKernelEvents::TcKernelEvents(const cudaEvent_t *ab) : prev(g_tc_events) { g_tc_events = ab; }
TcKernelEvents::~TcKernelEvents() { g_tc_events = prev; }

struct TcItem {
  const float *Ahi, *Alo, *Bhi, *Blo;
  float *C;
  long long ldc;  // real leading dimension of C
  int m, n2, nkt, mtc, ntc, tile0;  // tile0: first global tile index of this item
  long long amts;  // A tiles between consecutive 128-row tiles (0: nkt, a packed A of its own)
  int colmajor;    // 1: tiles walk down the columns (mt fastest), 0: along the rows (nt fastest)
};

// Position of tile `local` of an item.  Along the rows, the CTAs running at once share one row of
// A tiles and sweep all of B; down the columns they share one column of B tiles and sweep all of A.
// Down the columns is chosen when the item's packed A fits comfortably in L2 and B is wide, so that
// A stays cached while each B column is read once (tc_tile_order).
__device__ __forceinline__ void tile_pos(const TcItem &it, int local, int &mt, int &nt) {
  if (it.colmajor) {
    mt = local % it.mtc;
    nt = local / it.mtc;
  } else {
    mt = local / it.ntc;
    nt = local % it.ntc;
  }
}
constexpr int TC_MAXB = 64;
struct TcBatchP {
  TcItem it[TC_MAXB];
  int count, total_tiles;
  int *err;    // status word of the launch (DS_WAIT_TIMEOUT on a wait that ran out)
  int splits;  // 3: hi*hi + hi*lo + lo*hi (FP32 accuracy); 1: hi*hi only (plain TF32, peak probe)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// bounded wait; returns false on time-out or when another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 1023) == 1023 && *abort_flag) return false;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  const uint64_t g = (uint64_t)__cvta_generic_to_global(src);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(g), "r"(bytes), "r"(bar)
               : "memory");
}
// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused with 128B swizzle, K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define TC_LD32(taddr, v)                                                                                      \
  asm volatile(                                                                                                \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17," \
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                       \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),       \
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), \
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),            \
        "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),            \
        "=r"(v[30]), "=r"(v[31])                                                                              \
      : "r"(taddr))

__device__ __forceinline__ int find_item(const TcBatchP &b, int tile) {
  int lo = 0, hi = b.count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (b.it[mid].tile0 <= tile) lo = mid; else hi = mid;
  }
  return lo;
}

// Epilogue of one output tile by one warp: TMEM lanes 32q..32q+31 (rows mt*128 + 32q ..), column
// chunks of 32 accumulator columns [half*4, half*4 + 4), staged through shared memory so that C
// is read and written along its rows; C = alpha * acc + beta * C, rows and columns masked.
__device__ __forceinline__ void drain_tile(const TcItem &it, uint32_t tacc, int mt, int nt, int q, int half, int lane,
                                           float *stg, float alpha, float beta) {
  const int row0 = mt * TC_BM + q * 32;
  const int nrows = min(32, it.m - row0);
  float *__restrict__ Cb = it.C;
#pragma unroll 1
  for (int c = half * (TC_BN / 64); c < (half + 1) * (TC_BN / 64); ++c) {
    uint32_t v[32];
    TC_LD32(tacc + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 32), v);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) stg[lane * EPI_PITCH + j] = __uint_as_float(v[j]);
    __syncwarp();
    const int col = nt * TC_BN + c * 32 + lane;
    if (col < it.n2 && nrows > 0) {
      // all loads of C first (independent, in flight together), then the stores
      float cv[32];
#pragma unroll
      for (int r = 0; r < 32; ++r)
        cv[r] = (beta != 0.f && r < nrows) ? Cb[(long long)(row0 + r) * it.ldc + col] : 0.f;
#pragma unroll
      for (int r = 0; r < 32; ++r)
        if (r < nrows) Cb[(long long)(row0 + r) * it.ldc + col] = fmaf(alpha, stg[r * EPI_PITCH + lane], beta * cv[r]);
    }
    __syncwarp();
  }
}

// Persistent, warp-specialised: warp 0 streams operand tiles, warp 1 issues the MMAs into one of
// two TMEM accumulators (256 columns each), warps 2..5 drain the other accumulator to C.
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcBatchP b, float alpha,
                                                                float beta) {
  int *err = b.err;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float *epi = reinterpret_cast<float *>(base + TC_STAGES * STAGE_BYTES);
  __shared__ __align__(8) uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES], tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_s;
  __shared__ volatile int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&tfull_bar[a]), 1);
      mbar_init(smem_u32(&tempty_bar[a]), 32 * EPI_WARPS);
    }
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                 "r"(2 * TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_s;
  auto stage_addr = [&](int s, int which) -> uint32_t {  // which: 0 Ahi, 1 Alo, 2 Bhi, 3 Blo
    const uint32_t off = (uint32_t)s * STAGE_BYTES +
                         (which == 0 ? 0u : which == 1 ? A_TILE * 4u : which == 2 ? 2u * A_TILE * 4u
                                                                                  : 2u * A_TILE * 4u + B_TILE * 4u);
    return smem_u32(base + off);
  };
  if (warp == 0) {
    if (lane == 0) {  // producer
      long long g = 0;  // global k-tile counter (stage ring position)
      for (int tile = blockIdx.x; tile < b.total_tiles && !abort_s; tile += gridDim.x) {
        const TcItem &it = b.it[find_item(b, tile)];
        const int local = tile - it.tile0;
        int mt, nt;
        tile_pos(it, local, mt, nt);
        const long long ams = it.amts ? it.amts : it.nkt;
        const float *Ahi = it.Ahi + (long long)mt * ams * A_TILE, *Alo = it.Alo + (long long)mt * ams * A_TILE;
        const float *Bhi = it.Bhi + (long long)nt * it.nkt * B_TILE, *Blo = it.Blo + (long long)nt * it.nkt * B_TILE;
        for (int kt = 0; kt < it.nkt; ++kt, ++g) {
          const int s = (int)(g % TC_STAGES);
          const long long u = g / TC_STAGES;
          if (u >= 1 && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)((u - 1) & 1), &abort_s)) {
            atomicOr(err, DS_WAIT_TIMEOUT);
            abort_s = 1;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[s]);
          mbar_expect_tx(fb, b.splits > 1 ? STAGE_BYTES : (A_TILE + B_TILE) * 4);
          bulk_g2s(stage_addr(s, 0), Ahi + (long long)kt * A_TILE, A_TILE * 4, fb);
          bulk_g2s(stage_addr(s, 2), Bhi + (long long)kt * B_TILE, B_TILE * 4, fb);
          if (b.splits > 1) {
            bulk_g2s(stage_addr(s, 1), Alo + (long long)kt * A_TILE, A_TILE * 4, fb);
            bulk_g2s(stage_addr(s, 3), Blo + (long long)kt * B_TILE, B_TILE * 4, fb);
          }
        }
      }
      // drain: every issued copy must land before the CTA can exit
      for (long long q = (g > TC_STAGES ? g - TC_STAGES : 0); q < g; ++q)
        mbar_wait(smem_u32(&full_bar[q % TC_STAGES]), (uint32_t)((q / TC_STAGES) & 1), &abort_s);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                             ((uint32_t)(TC_BM >> 4) << 24);
      long long g = 0;
      int lt = 0;
      for (int tile = blockIdx.x; tile < b.total_tiles && !abort_s; tile += gridDim.x, ++lt) {
        const TcItem &it = b.it[find_item(b, tile)];
        const int acc = lt & 1;
        if (lt >= 2 && !mbar_wait(smem_u32(&tempty_bar[acc]), (uint32_t)(((lt >> 1) - 1) & 1), &abort_s)) {
          atomicOr(err, DS_WAIT_TIMEOUT);
          abort_s = 1;
          break;
        }
        fence_after();
        const uint32_t dacc = tmem + (uint32_t)(acc * TC_BN);
        bool ok = true;
        for (int kt = 0; kt < it.nkt; ++kt, ++g) {
          const int s = (int)(g % TC_STAGES);
          if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((g / TC_STAGES) & 1), &abort_s)) {
            atomicOr(err, DS_WAIT_TIMEOUT);
            abort_s = 1;
            ok = false;
            break;
          }
          fence_after();
          const uint32_t ah = stage_addr(s, 0), al = stage_addr(s, 1), bh = stage_addr(s, 2), bl = stage_addr(s, 3);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 8; ++kk) {
            const uint32_t o = kk * 32;  // 8 TF32 values = 32 bytes along K inside the swizzle row
            mma_tf32(dacc, sdesc(ah + o), sdesc(bh + o), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            if (b.splits > 1) {
              mma_tf32(dacc, sdesc(ah + o), sdesc(bl + o), idesc, 1u);
              mma_tf32(dacc, sdesc(al + o), sdesc(bh + o), idesc, 1u);
            }
          }
          mma_commit(smem_u32(&empty_bar[s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&tfull_bar[acc]));
      }
    }
  } else {
    // epilogue warps: warp w reads accumulator lanes 32*(w % 4) .. +31 (its TMEM sub-partition);
    // warps 2..5 take column chunks 0..3, warps 6..9 chunks 4..7
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    float *stg = epi + (warp - 2) * 32 * EPI_PITCH;
    int lt = 0;
    for (int tile = blockIdx.x; tile < b.total_tiles; tile += gridDim.x, ++lt) {
      const TcItem &it = b.it[find_item(b, tile)];
      const int local = tile - it.tile0;
      int mt, nt;
      tile_pos(it, local, mt, nt);
      const int acc = lt & 1;
      const bool ready = mbar_wait(smem_u32(&tfull_bar[acc]), (uint32_t)((lt >> 1) & 1), &abort_s);
      // the whole warp takes the same branch (tcgen05.ld below is a warp-collective)
      if (!__all_sync(0xffffffffu, ready && !abort_s)) {
        if (lane == 0) atomicOr(err, DS_WAIT_TIMEOUT);
        abort_s = 1;
        break;
      }
      fence_after();
      drain_tile(it, tmem + (uint32_t)(acc * TC_BN), mt, nt, q, half, lane, stg, alpha, beta);
      fence_before();
      mbar_arrive(smem_u32(&tempty_bar[acc]));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_BN) : "memory");
  }
}

// ---------------------------------------------------------------------------------------
// Two-CTA variant (cta_group::2): a cluster of two CTAs on two SMs computes a 256 x 256 tile of
// Cr with one MMA stream.  Each CTA holds its own 128 rows of A and its half (128 packed rows) of
// the B tile in shared memory; the MMAs, issued by the leader CTA (rank 0), read A and B from both
// CTAs and leave rows 0..127 of the accumulator in the leader's TMEM and rows 128..255 in the
// peer's.  Per 32-deep K tile an SM so takes in 64 KB instead of the 96 KB of the one-CTA kernel
// (whose 128 x 256 tile needs all of B), which is what limits that kernel (operand feed, not the
// tensor pipe).
//
// Synchronisation (all waits bounded; DS_WAIT_TIMEOUT into *err on time-out):
//  - each CTA's producer loads its halves into its own stage and completes its own full_bar;
//  - the peer's warp 1 forwards: it waits on its own full_bar and arrives on the leader's pfull_bar;
//  - the leader waits on full_bar and pfull_bar, issues the MMAs, and commits to empty_bar of both
//    CTAs (stage reusable) and, per tile, to tfull_bar of both CTAs (accumulator ready);
//  - every epilogue warp of both CTAs drains its TMEM lanes and arrives on the leader's tempty_bar.
// ---------------------------------------------------------------------------------------
constexpr int T2_STAGES = 3;
constexpr int T2_BHALF = (TC_BN / 2) * TC_BK;                       // floats of one CTA's B half
constexpr int T2_STAGE_BYTES = (2 * A_TILE + 2 * T2_BHALF) * 4;     // 64 KB
constexpr int T2_SMEM = T2_STAGES * T2_STAGE_BYTES + EPI_BYTES + 1024;

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// bounded wait with cluster-scope acquire (the barrier may be completed from the peer CTA)
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 1023) == 1023 && *abort_flag) return false;
  }
  return false;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mma2_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma2_commit_both(uint32_t bar) {
  const uint16_t mask = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

// pair tile `local` of an item -> (pair row mp, tile column nt); two CTAs take rows 2 mp, 2 mp + 1
__device__ __forceinline__ void pair_pos(const TcItem &it, int local, int &mp, int &nt) {
  const int mpc = (it.mtc + 1) >> 1;
  if (it.colmajor) {
    mp = local % mpc;
    nt = local / mpc;
  } else {
    mp = local / it.ntc;
    nt = local % it.ntc;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm2_kernel(const __grid_constant__ TcBatchP b, float alpha,
                                                                 float beta) {
  int *err = b.err;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float *epi = reinterpret_cast<float *>(base + T2_STAGES * T2_STAGE_BYTES);
  __shared__ __align__(8) uint64_t full_bar[T2_STAGES], pfull_bar[T2_STAGES], empty_bar[T2_STAGES], tfull_bar[2],
      tempty_bar[2];
  __shared__ uint32_t tmem_s;
  __shared__ volatile int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const int cl = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
  if (threadIdx.x == 0) {
    for (int s = 0; s < T2_STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&pfull_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&tfull_bar[a]), 1);
      mbar_init(smem_u32(&tempty_bar[a]), 2 * EPI_WARPS);  // one arrival per epilogue warp of each CTA
    }
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {  // both CTAs of the pair allocate together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                 "r"(2 * TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  cluster_sync_all();  // both CTAs' barriers initialised and TMEM allocated before any remote use
  fence_after();
  const uint32_t tmem = tmem_s;
  auto stage_addr = [&](int s, int which) -> uint32_t {  // which: 0 Ahi, 1 Alo, 2 Bhi half, 3 Blo half
    const uint32_t off = (uint32_t)s * T2_STAGE_BYTES +
                         (which == 0 ? 0u : which == 1 ? A_TILE * 4u : which == 2 ? 2u * A_TILE * 4u
                                                                                  : 2u * A_TILE * 4u + T2_BHALF * 4u);
    return smem_u32(base + off);
  };
  if (warp == 0) {
    if (lane == 0) {  // producer (both CTAs): this CTA's A rows and B half
      long long g = 0;
      for (int pt = cl; pt < b.total_tiles && !abort_s; pt += ncl) {
        const TcItem &it = b.it[find_item(b, pt)];
        int mp, nt;
        pair_pos(it, pt - it.tile0, mp, nt);
        const int mt = min(2 * mp + (int)rank, it.mtc - 1);  // a missing second row re-reads the last one
        const long long ams = it.amts ? it.amts : it.nkt;
        const float *Ahi = it.Ahi + (long long)mt * ams * A_TILE, *Alo = it.Alo + (long long)mt * ams * A_TILE;
        const long long boff = (long long)nt * it.nkt * B_TILE + (long long)rank * T2_BHALF;
        const float *Bhi = it.Bhi + boff, *Blo = it.Blo + boff;
        for (int kt = 0; kt < it.nkt; ++kt, ++g) {
          const int s = (int)(g % T2_STAGES);
          const long long u = g / T2_STAGES;
          if (u >= 1 && !mbar_wait_cl(smem_u32(&empty_bar[s]), (uint32_t)((u - 1) & 1), &abort_s)) {
            atomicOr(err, DS_WAIT_TIMEOUT);
            abort_s = 1;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[s]);
          mbar_expect_tx(fb, T2_STAGE_BYTES);
          bulk_g2s(stage_addr(s, 0), Ahi + (long long)kt * A_TILE, A_TILE * 4, fb);
          bulk_g2s(stage_addr(s, 1), Alo + (long long)kt * A_TILE, A_TILE * 4, fb);
          bulk_g2s(stage_addr(s, 2), Bhi + (long long)kt * B_TILE, T2_BHALF * 4, fb);
          bulk_g2s(stage_addr(s, 3), Blo + (long long)kt * B_TILE, T2_BHALF * 4, fb);
        }
      }
      // every issued copy lands, and every stage's last consumption is signalled here (the leader's
      // commits arrive on this CTA's empty barriers), before the CTA leaves
      for (long long q = (g > T2_STAGES ? g - T2_STAGES : 0); q < g; ++q) {
        mbar_wait_cl(smem_u32(&full_bar[q % T2_STAGES]), (uint32_t)((q / T2_STAGES) & 1), &abort_s);
        mbar_wait_cl(smem_u32(&empty_bar[q % T2_STAGES]), (uint32_t)((q / T2_STAGES) & 1), &abort_s);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 1) {  // peer: forward "my halves of stage s are in" to the leader
      long long g = 0;
      for (int pt = cl; pt < b.total_tiles && !abort_s; pt += ncl) {
        const TcItem &it = b.it[find_item(b, pt)];
        bool ok = true;
        for (int kt = 0; kt < it.nkt; ++kt, ++g) {
          const int s = (int)(g % T2_STAGES);
          if (!mbar_wait_cl(smem_u32(&full_bar[s]), (uint32_t)((g / T2_STAGES) & 1), &abort_s)) {
            atomicOr(err, DS_WAIT_TIMEOUT);
            abort_s = 1;
            ok = false;
            break;
          }
          mbar_arrive_cluster(map_to_rank(smem_u32(&pfull_bar[s]), 0));
        }
        if (!ok) break;
      }
    } else if (lane == 0 && rank == 0) {  // leader: MMA issuer for the pair
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                             ((uint32_t)((2 * TC_BM) >> 4) << 24);
      long long g = 0;
      int lt = 0;
      for (int pt = cl; pt < b.total_tiles && !abort_s; pt += ncl, ++lt) {
        const TcItem &it = b.it[find_item(b, pt)];
        const int acc = lt & 1;
        if (lt >= 2 && !mbar_wait_cl(smem_u32(&tempty_bar[acc]), (uint32_t)(((lt >> 1) - 1) & 1), &abort_s)) {
          atomicOr(err, DS_WAIT_TIMEOUT);
          abort_s = 1;
          break;
        }
        fence_after();
        const uint32_t dacc = tmem + (uint32_t)(acc * TC_BN);
        bool ok = true;
        for (int kt = 0; kt < it.nkt; ++kt, ++g) {
          const int s = (int)(g % T2_STAGES);
          const uint32_t par = (uint32_t)((g / T2_STAGES) & 1);
          if (!mbar_wait_cl(smem_u32(&full_bar[s]), par, &abort_s) ||
              !mbar_wait_cl(smem_u32(&pfull_bar[s]), par, &abort_s)) {
            atomicOr(err, DS_WAIT_TIMEOUT);
            abort_s = 1;
            ok = false;
            break;
          }
          fence_after();
          const uint32_t ah = stage_addr(s, 0), al = stage_addr(s, 1), bh = stage_addr(s, 2), bl = stage_addr(s, 3);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 8; ++kk) {
            const uint32_t o = kk * 32;
            mma2_tf32(dacc, sdesc(ah + o), sdesc(bh + o), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            mma2_tf32(dacc, sdesc(ah + o), sdesc(bl + o), idesc, 1u);
            mma2_tf32(dacc, sdesc(al + o), sdesc(bh + o), idesc, 1u);
          }
          mma2_commit_both(smem_u32(&empty_bar[s]));
        }
        if (!ok) break;
        mma2_commit_both(smem_u32(&tfull_bar[acc]));
      }
    }
  } else {
    // epilogue warps of both CTAs: this CTA's 128 accumulator rows of the pair tile
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    float *stg = epi + (warp - 2) * 32 * EPI_PITCH;
    const uint32_t tempty_leader0 = map_to_rank(smem_u32(&tempty_bar[0]), 0);
    const uint32_t tempty_leader1 = map_to_rank(smem_u32(&tempty_bar[1]), 0);
    int lt = 0;
    for (int pt = cl; pt < b.total_tiles; pt += ncl, ++lt) {
      const TcItem &it = b.it[find_item(b, pt)];
      int mp, nt;
      pair_pos(it, pt - it.tile0, mp, nt);
      const int mt = 2 * mp + (int)rank;  // rows beyond m (a missing second row) are masked
      const int acc = lt & 1;
      const bool ready = mbar_wait_cl(smem_u32(&tfull_bar[acc]), (uint32_t)((lt >> 1) & 1), &abort_s);
      if (!__all_sync(0xffffffffu, ready && !abort_s)) {
        if (lane == 0) atomicOr(err, DS_WAIT_TIMEOUT);
        abort_s = 1;
        break;
      }
      fence_after();
      drain_tile(it, tmem + (uint32_t)(acc * TC_BN), mt, nt, q, half, lane, stg, alpha, beta);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(acc ? tempty_leader1 : tempty_leader0);
    }
  }
  fence_before();
  cluster_sync_all();  // no CTA leaves while its peer may still signal it or read its shared memory
  fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_BN) : "memory");
  }
}

// ---------------------------------------------------------------------------------------
// Tensor-pipe throughput probe: one CTA per SM issues `iters` x 4 kind::tf32 MMAs of
// 128 x 256 x 8 from operand tiles that stay in shared memory (no loads), into one TMEM
// accumulator, then waits for their completion on an mbarrier (bounded; DS_WAIT_TIMEOUT into *err
// on time-out).  Measures the MMA issue rate alone, not the operand feed.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1) tf32_mma_probe_kernel(int iters, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_s;
  __shared__ volatile int abort_s;
  const int warp = threadIdx.x >> 5;
  // operand tiles: zeros (the rate does not depend on the values)
  for (int i = threadIdx.x; i < (A_TILE + B_TILE); i += blockDim.x) reinterpret_cast<float *>(base)[i] = 0.f;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&done_bar), 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                 "r"(TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_s;
  if (threadIdx.x == 0) {
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                           ((uint32_t)(TC_BM >> 4) << 24);
    const uint32_t a = smem_u32(base), b = smem_u32(base + A_TILE * 4);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk)
        mma_tf32(tmem, sdesc(a + kk * 32), sdesc(b + kk * 32), idesc, (it > 0 || kk > 0) ? 1u : 0u);
    }
    mma_commit(smem_u32(&done_bar));
    if (!mbar_wait(smem_u32(&done_bar), 0, &abort_s)) atomicOr(err, DS_WAIT_TIMEOUT);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
  }
}

double tc_mma_probe_tflops(cudaStream_t st, int *dev_status) {
  int dev = 0, nsm = 0;
  RFDD_CUDA(cudaGetDevice(&dev));
  RFDD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int smem = (A_TILE + B_TILE) * 4 + 1024;
  RFDD_CUDA(cudaFuncSetAttribute(tf32_mma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  cudaEvent_t e0, e1;
  RFDD_CUDA(cudaEventCreate(&e0));
  RFDD_CUDA(cudaEventCreate(&e1));
  const int iters = 4096;
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch is a warm-up
    RFDD_CUDA(cudaEventRecord(e0, st));
    tf32_mma_probe_kernel<<<nsm, 128, smem, st>>>(iters, dev_status);
    RFDD_CHECK_LAUNCH();
    RFDD_CUDA(cudaEventRecord(e1, st));
    RFDD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RFDD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double fl = 2.0 * TC_BM * TC_BN * 8.0 * (TC_BK / 8) * (double)iters * nsm;
    if (rep > 0 && ms > 0.f) best = std::max(best, fl / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// ---------------------------------------------------------------------------------------
// packing: split into TF32 hi/lo and write swizzled tiles
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  hi = __uint_as_float(r);
  lo = x - hi;
}

struct PackItem {
  const float *src;   // interleaved complex source (as floats)
  long long ld;       // complex leading dimension
  int m, n, k;        // A: m x k ; B: k x n (complex)
  float *hi, *lo;     // tile buffers
  int mtc, ntc, nkt;
};
struct PackBatchP {
  PackItem it[TC_MAXB];
};

// A tiles: [mt][kt] 128 rows x 32 floats; float4 chunk c of row r stored at chunk c ^ (r & 7)
__global__ void pack_a_kernel(PackBatchP pb) {
  const PackItem it = pb.it[blockIdx.y];
  const long long chunks = (long long)it.mtc * TC_BM * it.nkt * 8;
  const int k2 = 2 * it.k;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < chunks; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / (it.nkt * 8);
    const int q = (int)(e % (it.nkt * 8));
    const int kt = q >> 3, c = q & 7;
    const int mt = (int)(row / TC_BM), r = (int)(row % TC_BM);
    float h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int kr = kt * TC_BK + c * 4 + t;
      float x = 0.f;
      if (row < it.m && kr < k2) x = it.src[row * 2 * it.ld + kr];
      split_tf32(x, h[t], l[t]);
    }
    const long long off = ((long long)mt * it.nkt + kt) * A_TILE + r * TC_BK + ((c ^ (r & 7)) << 2);
    *reinterpret_cast<float4 *>(it.hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(it.lo + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// B tiles: Br^T rows n' = 2j + t (t: 0 real part column, 1 imaginary), K index k' = 2p + u:
//   Br^T[2j][2p] = re B[p][j], Br^T[2j][2p+1] = -im B[p][j], Br^T[2j+1][2p] = im, Br^T[2j+1][2p+1] = re
__global__ void pack_b_kernel(PackBatchP pb) {
  const PackItem it = pb.it[blockIdx.y];
  const long long chunks = (long long)it.ntc * TC_BN * it.nkt * 8;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < chunks; e += (long long)gridDim.x * blockDim.x) {
    const long long rowp = e / (it.nkt * 8);
    const int q = (int)(e % (it.nkt * 8));
    const int kt = q >> 3, c = q & 7;
    const int nt = (int)(rowp / TC_BN), r = (int)(rowp % TC_BN);
    const long long j = rowp >> 1;
    const int tt = (int)(rowp & 1);
    float h[4], l[4];
#pragma unroll
    for (int t2 = 0; t2 < 2; ++t2) {
      const int p = (kt * TC_BK + c * 4) / 2 + t2;
      float re = 0.f, im = 0.f;
      if (j < it.n && p < it.k) {
        const float *s = it.src + ((long long)p * it.ld + j) * 2;
        re = s[0];
        im = s[1];
      }
      const float x0 = tt == 0 ? re : im;    // coefficient of Re A
      const float x1 = tt == 0 ? -im : re;   // coefficient of Im A
      split_tf32(x0, h[2 * t2], l[2 * t2]);
      split_tf32(x1, h[2 * t2 + 1], l[2 * t2 + 1]);
    }
    const long long off = ((long long)nt * it.nkt + kt) * B_TILE + r * TC_BK + ((c ^ (r & 7)) << 2);
    *reinterpret_cast<float4 *>(it.hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(it.lo + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// The same B tiles, built through shared memory: a block stages a 16 (K) x 64 (N) complex slab
// of B with reads along B's rows (coalesced), then writes the 128 packed rows x 32 K-values it
// covers (half a tile) with coalesced 16-byte stores.  Threads of pack_b_kernel above read B down
// its columns instead (one 8-byte element per row of B per thread).
__global__ void __launch_bounds__(256) pack_b_t_kernel(PackBatchP pb) {
  const PackItem it = pb.it[blockIdx.y];
  const int jblocks = it.ntc * 2;  // 64 complex columns (128 packed rows) per block
  const int nblk = jblocks * it.nkt;
  __shared__ float2 sb[16][65];
  for (int bid = blockIdx.x; bid < nblk; bid += gridDim.x) {
    const int kt = bid % it.nkt, jb = bid / it.nkt;
    const long long j0 = (long long)jb * 64;
    const int p0 = kt * (TC_BK / 2);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = threadIdx.x + 256 * i;
      const int pl = idx >> 6, jl = idx & 63;
      const long long j = j0 + jl;
      const int pp = p0 + pl;
      float2 v = make_float2(0.f, 0.f);
      if (j < it.n && pp < it.k) v = *reinterpret_cast<const float2 *>(it.src + ((long long)pp * it.ld + j) * 2);
      sb[pl][jl] = v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int id = threadIdx.x + 256 * i;
      const int rl = id >> 3, c = id & 7;  // packed row within the half tile, 16-byte chunk
      const int jl = rl >> 1, tt = rl & 1;
      float h[4], l[4];
#pragma unroll
      for (int t2 = 0; t2 < 2; ++t2) {
        const float2 b = sb[2 * c + t2][jl];
        const float x0 = tt == 0 ? b.x : b.y;   // coefficient of Re A
        const float x1 = tt == 0 ? -b.y : b.x;  // coefficient of Im A
        split_tf32(x0, h[2 * t2], l[2 * t2]);
        split_tf32(x1, h[2 * t2 + 1], l[2 * t2 + 1]);
      }
      const long long rowp = 2 * j0 + rl;
      const int nt = (int)(rowp / TC_BN), r = (int)(rowp % TC_BN);
      const long long off = ((long long)nt * it.nkt + kt) * B_TILE + r * TC_BK + ((c ^ (r & 7)) << 2);
      *reinterpret_cast<float4 *>(it.hi + off) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4 *>(it.lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

// real B, same staging: a 32 (K) x 128 (N) slab, one packed tile half (128 rows x 32 K-values)
__global__ void __launch_bounds__(256) pack_b_real_t_kernel(PackBatchP pb) {
  const PackItem it = pb.it[blockIdx.y];
  const int jblocks = it.ntc * 2;  // 128 columns per block
  const int nblk = jblocks * it.nkt;
  __shared__ float sb[32][129];
  for (int bid = blockIdx.x; bid < nblk; bid += gridDim.x) {
    const int kt = bid % it.nkt, jb = bid / it.nkt;
    const long long j0 = (long long)jb * 128;
    const int p0 = kt * TC_BK;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int idx = threadIdx.x + 256 * i;
      const int pl = idx >> 7, jl = idx & 127;
      const long long j = j0 + jl;
      const int pp = p0 + pl;
      sb[pl][jl] = (j < it.n && pp < it.k) ? it.src[(long long)pp * it.ld + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int id = threadIdx.x + 256 * i;
      const int rl = id >> 3, c = id & 7;
      float h[4], l[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) split_tf32(sb[c * 4 + t][rl], h[t], l[t]);
      const long long row = j0 + rl;
      const int nt = (int)(row / TC_BN), r = (int)(row % TC_BN);
      const long long off = ((long long)nt * it.nkt + kt) * B_TILE + r * TC_BK + ((c ^ (r & 7)) << 2);
      *reinterpret_cast<float4 *>(it.hi + off) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4 *>(it.lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

// real operands: A (m x k, ld), B (k x n, ld) in FP32; the same tile formats with K' = k, N' = n
__global__ void pack_a_real_kernel(PackBatchP pb) {
  const PackItem it = pb.it[blockIdx.y];
  const long long chunks = (long long)it.mtc * TC_BM * it.nkt * 8;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < chunks; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / (it.nkt * 8);
    const int q = (int)(e % (it.nkt * 8));
    const int kt = q >> 3, c = q & 7;
    const int mt = (int)(row / TC_BM), r = (int)(row % TC_BM);
    float h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int kr = kt * TC_BK + c * 4 + t;
      const float x = (row < it.m && kr < it.k) ? it.src[row * it.ld + kr] : 0.f;
      split_tf32(x, h[t], l[t]);
    }
    const long long off = ((long long)mt * it.nkt + kt) * A_TILE + r * TC_BK + ((c ^ (r & 7)) << 2);
    *reinterpret_cast<float4 *>(it.hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(it.lo + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
}
__global__ void pack_b_real_kernel(PackBatchP pb) {
  const PackItem it = pb.it[blockIdx.y];
  const long long chunks = (long long)it.ntc * TC_BN * it.nkt * 8;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < chunks; e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / (it.nkt * 8);
    const int q = (int)(e % (it.nkt * 8));
    const int kt = q >> 3, c = q & 7;
    const int nt = (int)(j / TC_BN), r = (int)(j % TC_BN);
    float h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int p = kt * TC_BK + c * 4 + t;
      const float x = (j < it.n && p < it.k) ? it.src[(long long)p * it.ld + j] : 0.f;
      split_tf32(x, h[t], l[t]);
    }
    const long long off = ((long long)nt * it.nkt + kt) * B_TILE + r * TC_BK + ((c ^ (r & 7)) << 2);
    *reinterpret_cast<float4 *>(it.hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(it.lo + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// Per-device launch set-up of the tensor-core kernel: its dynamic shared-memory limit is raised
// once on every device it runs on, and the device's SM count sizes the persistent grid.
struct TcDevInfo {
  bool attr = false;
  int nsm = 0;
  int clusters2 = 0;  // two-CTA clusters of tc_gemm2_kernel that can be resident at once
};
static TcDevInfo tc_device_info() {
  static std::mutex mu;
  static std::vector<TcDevInfo> info;
  int dev = 0;
  RFDD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)info.size() <= dev) info.resize(dev + 1);
  TcDevInfo &d = info[dev];
  if (!d.attr) {
    RFDD_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    RFDD_CUDA(cudaFuncSetAttribute(tc_gemm2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, T2_SMEM));
    RFDD_CUDA(cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = T2_SMEM;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, (void *)tc_gemm2_kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      nc = 0;
    }
    d.clusters2 = nc;
    d.attr = true;
  }
  return d;
}
static int tc_device_setup() { return std::max(1, tc_device_info().nsm); }

// Kernel choice for a launch (g_tc_engine_override lets rfdd_cgemm force one for tests):
// the two-CTA kernel when it has work for every resident cluster and few of its pair tiles are
// half empty (an odd number of row tiles leaves the second CTA of the last pair without rows).
thread_local int g_tc_engine_override = 0;  // 0 automatic, 1 one-CTA kernel, 2 two-CTA kernel
TcEngineScope::TcEngineScope(int e) : prev(g_tc_engine_override) { g_tc_engine_override = e; }
TcEngineScope::~TcEngineScope() { g_tc_engine_override = prev; }

// The tile-shape autotuner (tc_tune.h) and the timings it is waiting for.  Launches it asks to
// measure are bracketed by events on their own stream; the events are polled without blocking at
// the next launch and when the table is read.
namespace {
struct TunePending {
  tune::Key key;
  int cand;
  double gflop;
  cudaEvent_t e0, e1;
};
std::mutex g_tune_mu;
tune::Tuner g_tuner;
std::vector<TunePending> g_tune_pending;

void tune_poll_locked() {
  for (size_t i = 0; i < g_tune_pending.size();) {
    TunePending &q = g_tune_pending[i];
    const cudaError_t r = cudaEventQuery(q.e1);
    if (r == cudaErrorNotReady) {
      ++i;
      continue;
    }
    float ms = 0.0f;
    if (r == cudaSuccess && cudaEventElapsedTime(&ms, q.e0, q.e1) == cudaSuccess && q.gflop > 0.0)
      g_tuner.record(q.key, q.cand, ms / q.gflop);
    else
      g_tuner.forget(q.key, q.cand);
    if (r != cudaSuccess) cudaGetLastError();
    cudaEventDestroy(q.e0);
    cudaEventDestroy(q.e1);
    g_tune_pending.erase(g_tune_pending.begin() + i);
  }
}
}  // namespace

int tc_autotune(int mode) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int prev = g_tuner.enabled ? 1 : 0;
  if (mode == 2) {
    tune_poll_locked();
    g_tuner.clear();
  } else {
    g_tuner.enabled = mode != 0;
  }
  return prev;
}

std::string tc_autotune_table() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_poll_locked();
  return g_tuner.dump();
}

// Tile walk of one item: down the columns when B spans at least 8 tile columns and the item's
// packed A (hi + lo) takes at most 48 MB of the 129 MB L2, else along the rows.
int tc_tile_order(int mtc, int ntc, int nkt) {
  const double a_bytes = (double)mtc * nkt * A_TILE * 8.0;
  return (ntc >= 8 && mtc >= 2 && a_bytes <= 48e6) ? 1 : 0;
}

template <bool CPLX, typename T>
static void tc_gemm_run(cudaStream_t st, const std::vector<GemmItem<T>> &items, double alpha, double beta,
                        const std::vector<TcPackedA> *pre = nullptr, int splits = 3) {
  constexpr int F = CPLX ? 2 : 1;  // real columns / K entries per element
  RFDD_REQUIRE(g_tc_status != nullptr, RFDD_ESTATE, "tensor-core GEMM launched without a status word");
  const int nsm = tc_device_setup();
  for (size_t s0 = 0; s0 < items.size(); s0 += TC_MAXB) {
    const int cnt = (int)std::min<size_t>(TC_MAXB, items.size() - s0);
    PackBatchP pa, pbb;
    TcBatchP tb;
    memset(&pa, 0, sizeof(pa));
    memset(&pbb, 0, sizeof(pbb));
    memset(&tb, 0, sizeof(tb));
    size_t total = 0;
    std::vector<size_t> offA(cnt), offB(cnt);
    int mtmax = 1, ntmax = 1;
    long long achunks = 1, bchunks = 1;
    double flops = 0.0, cbytes = 0.0;
    for (int i = 0; i < cnt; ++i) {
      const auto &g = items[s0 + i];
      const int mtc = ceil_div(g.m, TC_BM), ntc = ceil_div((int64_t)F * g.n, TC_BN), nkt = ceil_div((int64_t)F * g.k, TC_BK);
      const bool packed = pre && (*pre)[s0 + i].hi;
      offA[i] = total;
      if (!packed) total += (size_t)mtc * nkt * A_TILE * 2;
      offB[i] = total;
      total += (size_t)ntc * nkt * B_TILE * 2;
      mtmax = std::max(mtmax, mtc);
      ntmax = std::max(ntmax, ntc);
      achunks = std::max(achunks, (long long)mtc * TC_BM * nkt * 8);
      bchunks = std::max(bchunks, (long long)ntc * TC_BN * nkt * 8);
      flops += (CPLX ? 8.0 : 2.0) * g.m * (double)g.n * g.k;
      // compulsory DRAM bytes: C read (beta != 0) and written, packed hi/lo operands read once
      cbytes += (beta != 0.0 ? 2.0 : 1.0) * 4.0 * F * g.m * (double)g.n +
                8.0 * ((double)mtc * nkt * A_TILE + (double)ntc * nkt * B_TILE);
    }
    float *ws = nullptr;
    RFDD_CUDA(cudaMallocAsync((void **)&ws, total * sizeof(float), st));
    int tiles = 0;
    for (int i = 0; i < cnt; ++i) {
      const auto &g = items[s0 + i];
      const int mtc = ceil_div(g.m, TC_BM), ntc = ceil_div((int64_t)F * g.n, TC_BN), nkt = ceil_div((int64_t)F * g.k, TC_BK);
      const bool packed = pre && (*pre)[s0 + i].hi;
      const float *Ah = packed ? (*pre)[s0 + i].hi : ws + offA[i];
      const float *Al = packed ? (*pre)[s0 + i].lo : ws + offA[i] + (size_t)mtc * nkt * A_TILE;
      float *Bh = ws + offB[i], *Bl = Bh + (size_t)ntc * nkt * B_TILE;
      // a pre-packed A is not packed again (mtc = 0 gives its pack item no work)
      pa.it[i] = {reinterpret_cast<const float *>(g.A), g.lda, g.m, g.n, g.k, const_cast<float *>(Ah),
                  const_cast<float *>(Al), packed ? 0 : mtc, ntc, nkt};
      pbb.it[i] = {reinterpret_cast<const float *>(g.B), g.ldb, g.m, g.n, g.k, Bh, Bl, mtc, ntc, nkt};
      tb.it[i] = {Ah, Al, Bh, Bl, reinterpret_cast<float *>(g.C), (long long)F * g.ldc, g.m, F * g.n, nkt, mtc, ntc, tiles,
                  packed ? (long long)(*pre)[s0 + i].mt_stride : 0ll, tc_tile_order(mtc, ntc, nkt)};
      tiles += mtc * ntc;
    }
    tb.count = cnt;
    tb.total_tiles = tiles;
    tb.err = g_tc_status;
    tb.splits = splits;
    bool any_a = false;
    for (int i = 0; i < cnt; ++i) any_a |= pa.it[i].mtc > 0;
    const dim3 ga((unsigned)std::min<long long>(ceil_div(achunks, 256), 4096), cnt);
    long long bblocks = 1;  // staged half-tiles of the largest B
    for (int i = 0; i < cnt; ++i) bblocks = std::max(bblocks, (long long)pbb.it[i].ntc * 2 * pbb.it[i].nkt);
    const dim3 gbt((unsigned)std::min<long long>(bblocks, 8192), cnt);
    if (CPLX) {
      if (any_a) {
        pack_a_kernel<<<ga, 256, 0, st>>>(pa);
        RFDD_CHECK_LAUNCH();
      }
      pack_b_t_kernel<<<gbt, 256, 0, st>>>(pbb);
      RFDD_CHECK_LAUNCH();
    } else {
      pack_a_real_kernel<<<ga, 256, 0, st>>>(pa);
      RFDD_CHECK_LAUNCH();
      pack_b_real_t_kernel<<<gbt, 256, 0, st>>>(pbb);
      RFDD_CHECK_LAUNCH();
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (profiling_enabled()) {
      e0 = profile_event();
      e1 = profile_event();
      cudaEventRecord(e0, st);
    }
    // pair tiles of the two-CTA kernel
    long long pairs = 0, ghosts = 0;
    for (int i = 0; i < cnt; ++i) {
      pairs += (long long)((tb.it[i].mtc + 1) / 2) * tb.it[i].ntc;
      ghosts += (long long)(tb.it[i].mtc & 1) * tb.it[i].ntc;
    }
    const TcDevInfo dinfo = tc_device_info();
    // measured on 8192 x 8192 products: the two-CTA kernel gains from K = 256 (complex) on (4 %
    // there, 1.5 % at K = 1024) and loses at K = 128, where the epilogue, not the operand feed,
    // bounds both kernels
    int nkt_min = 1 << 30;
    for (int i = 0; i < cnt; ++i) nkt_min = std::min(nkt_min, tb.it[i].nkt);
    const bool two_ok = splits == 3 && dinfo.clusters2 > 0 && pairs >= dinfo.clusters2 && 8 * ghosts <= pairs;
    bool two = two_ok && (CPLX ? nkt_min >= 16 : nkt_min >= 8);
    // the autotuner decides where both kernels can run, outside stream capture
    tune::Key tkey;
    bool tmeasure = false;
    if (two_ok && g_tc_engine_override == 0) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      RFDD_CUDA(cudaStreamIsCapturing(st, &cs));
      RFDD_CUDA(cudaGetDevice(&tkey.device));
      tkey.cplx = CPLX ? 1 : 0;
      tkey.splits = splits;
      tkey.kbucket = tune::k_bucket(nkt_min);
      tkey.tbucket = tune::t_bucket(tiles, nsm);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_poll_locked();
      if (cs == cudaStreamCaptureStatusNone) {
        const tune::Choice ch = g_tuner.choose(tkey, two ? 1 : 0);
        two = ch.cand == 1;
        tmeasure = ch.measure;
      } else {
        const auto &t = g_tuner.table();
        const auto it = t.find(tkey);
        if (it != t.end() && it->second.winner >= 0) two = it->second.winner == 1;
      }
    }
    if (g_tc_engine_override == 1) two = false;
    if (g_tc_engine_override == 2) two = splits == 3 && dinfo.clusters2 > 0;
    cudaEvent_t te0 = nullptr, te1 = nullptr;
    if (tmeasure) {
      if (cudaEventCreate(&te0) != cudaSuccess || cudaEventCreate(&te1) != cudaSuccess) {
        cudaGetLastError();
        if (te0) cudaEventDestroy(te0);
        te0 = te1 = nullptr;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuner.forget(tkey, two ? 1 : 0);
      } else {
        RFDD_CUDA(cudaEventRecord(te0, st));
      }
    }
    if (g_tc_events) RFDD_CUDA(cudaEventRecord(g_tc_events[0], st));
    if (two) {
      TcBatchP t2 = tb;
      int p0 = 0;
      for (int i = 0; i < cnt; ++i) {
        t2.it[i].tile0 = p0;
        p0 += ((t2.it[i].mtc + 1) / 2) * t2.it[i].ntc;
      }
      t2.total_tiles = p0;
      const int ncl = std::max(1, std::min(p0, dinfo.clusters2));
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = 2;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.gridDim = dim3(2 * ncl, 1, 1);
      cfg.blockDim = dim3(TC_THREADS, 1, 1);
      cfg.dynamicSmemBytes = T2_SMEM;
      cfg.stream = st;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      RFDD_CUDA(cudaLaunchKernelEx(&cfg, tc_gemm2_kernel, t2, (float)alpha, (float)beta));
      RFDD_CHECK_LAUNCH();
    } else {
      const int grid = std::max(1, std::min(tiles, nsm));
      tc_gemm_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(tb, (float)alpha, (float)beta);
      RFDD_CHECK_LAUNCH();
    }
    if (g_tc_events) RFDD_CUDA(cudaEventRecord(g_tc_events[1], st));
    if (te1) {
      RFDD_CUDA(cudaEventRecord(te1, st));
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_pending.push_back({tkey, two ? 1 : 0, flops * 1e-9, te0, te1});
    }
    if (e0) {
      cudaEventRecord(e1, st);
      profile_push(e0, e1, flops, 1, cbytes);
    }
    RFDD_CUDA(cudaFreeAsync(ws, st));
  }
}


void tc_gemm_complex(cudaStream_t st, const std::vector<GemmItem<cx<float>>> &items, double alpha, double beta) {
  tc_gemm_run<true>(st, items, alpha, beta);
}

void tc_gemm_complex_pa(cudaStream_t st, const std::vector<GemmItem<cx<float>>> &items,
                        const std::vector<TcPackedA> &pa, double alpha, double beta) {
  RFDD_REQUIRE(pa.size() == items.size(), RFDD_EINVAL, "tc_gemm: one packed-A entry per item");
  std::vector<GemmItem<cx<float>>> live;
  std::vector<TcPackedA> lpa;
  for (size_t i = 0; i < items.size(); ++i)
    if (items[i].m > 0 && items[i].n > 0 && items[i].k > 0) {
      live.push_back(items[i]);
      lpa.push_back(pa[i]);
    }
  if (!live.empty()) tc_gemm_run<true>(st, live, alpha, beta, &lpa);
}

int64_t tc_packed_a_ktiles(int64_t k) { return ceil_div(2 * k, TC_BK); }
int64_t tc_packed_a_floats(int64_t m, int64_t k) { return (int64_t)ceil_div(m, TC_BM) * tc_packed_a_ktiles(k) * A_TILE; }

TcPackedA tc_packed_view(const float *hi, const float *lo, int64_t k_full, int64_t r0, int64_t c0) {
  RFDD_REQUIRE(r0 % TC_BM == 0 && (2 * c0) % TC_BK == 0, RFDD_EINVAL, "packed view must start on a tile");
  const int64_t kt = tc_packed_a_ktiles(k_full);
  const int64_t off = ((r0 / TC_BM) * kt + (2 * c0) / TC_BK) * A_TILE;
  return TcPackedA{hi + off, lo + off, kt};
}

void tc_pack_a_batched(cudaStream_t st, const std::vector<TcPackJob> &jobs) {
  for (size_t s0 = 0; s0 < jobs.size(); s0 += TC_MAXB) {
    const int cnt = (int)std::min<size_t>(TC_MAXB, jobs.size() - s0);
    PackBatchP pa;
    memset(&pa, 0, sizeof(pa));
    long long achunks = 1;
    for (int i = 0; i < cnt; ++i) {
      const TcPackJob &j = jobs[s0 + i];
      const int mtc = ceil_div(j.m, TC_BM), nkt = (int)tc_packed_a_ktiles(j.k);
      pa.it[i] = {reinterpret_cast<const float *>(j.A), j.lda, (int)j.m, 0, (int)j.k, j.hi, j.lo,
                  j.m > 0 && j.k > 0 ? mtc : 0, 0, nkt};
      achunks = std::max(achunks, (long long)mtc * TC_BM * nkt * 8);
    }
    pack_a_kernel<<<dim3((unsigned)std::min<long long>(ceil_div(achunks, 256), 4096), cnt), 256, 0, st>>>(pa);
    RFDD_CHECK_LAUNCH();
  }
}

void tc_gemm_real(cudaStream_t st, const std::vector<GemmItem<float>> &items, double alpha, double beta) {
  tc_gemm_run<false>(st, items, alpha, beta);
}

void tc_gemm_real_tf32(cudaStream_t st, const std::vector<GemmItem<float>> &items, double alpha, double beta) {
  tc_gemm_run<false>(st, items, alpha, beta, nullptr, 1);
}

// =========================================================================================
// Allocation-free variant of the tensor-core complex GEMM.
//
// Some callers cannot call cudaMalloc: code running inside a memory-capped process or allocator
// arena, real-time loops that must not touch the allocator, or host code that must not
// synchronise with other streams the way allocation can.  For them the packed operand tiles
// live in the file-scope array below instead of a per-call workspace.  The array's host-side
// name is only a stand-in: its device address is looked up with cudaGetSymbolAddress once per
// device (on that device's first call, with the device current) and passed to the kernels.
// =========================================================================================
constexpr int NOALLOC_MAX_M = 1024;   // complex rows of A and C
constexpr int NOALLOC_MAX_N = 1024;   // complex columns of B and C
constexpr int NOALLOC_MAX_K = 128;    // complex inner dimension
constexpr size_t NOALLOC_A_FLOATS =
    (size_t)((NOALLOC_MAX_M + TC_BM - 1) / TC_BM) * ((2 * NOALLOC_MAX_K + TC_BK - 1) / TC_BK) * A_TILE * 2;
constexpr size_t NOALLOC_B_FLOATS =
    (size_t)((2 * NOALLOC_MAX_N + TC_BN - 1) / TC_BN) * ((2 * NOALLOC_MAX_K + TC_BK - 1) / TC_BK) * B_TILE * 2;
constexpr size_t NOALLOC_FLOATS = NOALLOC_A_FLOATS + NOALLOC_B_FLOATS;  // 6 MiB of floats in total

static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];
// status word of the allocation-free launches (DS_WAIT_TIMEOUT), beside the scratch
static __device__ int g_noalloc_status;

struct NoallocAddr {
  float *scratch = nullptr;
  int *status = nullptr;
};
// Device addresses of the array and of its status word on the current device, looked up once per
// device with that device current (the host-side names are only stand-ins).
static NoallocAddr noalloc_addresses() {
  static std::mutex mu;
  static std::vector<NoallocAddr> addr;
  int dev = 0;
  RFDD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)addr.size() <= dev) addr.resize(dev + 1);
  if (!addr[dev].scratch) {
    void *p = nullptr, *q = nullptr;
    RFDD_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    RFDD_CUDA(cudaGetSymbolAddress(&q, g_noalloc_status));
    addr[dev].scratch = reinterpret_cast<float *>(p);
    addr[dev].status = reinterpret_cast<int *>(q);
  }
  return addr[dev];
}

int tc_gemm_complex_noalloc(cudaStream_t st, const cx<float> *A, int64_t lda, const cx<float> *B, int64_t ldb,
                            cx<float> *C, int64_t ldc, int m, int n, int k, double alpha, double beta) {
  RFDD_REQUIRE(m >= 1 && n >= 1 && k >= 1, RFDD_EINVAL, "cgemm_noalloc: sizes must be positive");
  RFDD_REQUIRE(m <= NOALLOC_MAX_M && n <= NOALLOC_MAX_N && k <= NOALLOC_MAX_K, RFDD_EINVAL,
               "cgemm_noalloc: m, n must be <= 1024 and k <= 128 (size of the static scratch)");
  const NoallocAddr na = noalloc_addresses();
  const int nsm = tc_device_setup();
  float *ws = na.scratch;
  const int mtc = ceil_div(m, TC_BM), ntc = ceil_div(2 * (int64_t)n, TC_BN), nkt = ceil_div(2 * (int64_t)k, TC_BK);
  float *Ah = ws, *Al = Ah + (size_t)mtc * nkt * A_TILE;
  float *Bh = ws + NOALLOC_A_FLOATS, *Bl = Bh + (size_t)ntc * nkt * B_TILE;
  PackBatchP pa, pbb;
  TcBatchP tb;
  memset(&pa, 0, sizeof(pa));
  memset(&pbb, 0, sizeof(pbb));
  memset(&tb, 0, sizeof(tb));
  pa.it[0] = {reinterpret_cast<const float *>(A), lda, m, n, k, Ah, Al, mtc, ntc, nkt};
  pbb.it[0] = {reinterpret_cast<const float *>(B), ldb, m, n, k, Bh, Bl, mtc, ntc, nkt};
  tb.it[0] = {Ah, Al, Bh, Bl, reinterpret_cast<float *>(C), 2ll * ldc, m, 2 * n, nkt, mtc, ntc, 0, 0ll,
              tc_tile_order(mtc, ntc, nkt)};
  tb.count = 1;
  tb.total_tiles = mtc * ntc;
  tb.err = na.status;
  tb.splits = 3;
  // the word keeps the last call's value: cleared on the caller's stream before this call's work
  RFDD_CUDA(cudaMemsetAsync(na.status, 0, sizeof(int), st));
  const long long achunks = (long long)mtc * TC_BM * nkt * 8;
  pack_a_kernel<<<dim3((unsigned)std::min<long long>(ceil_div(achunks, 256), 4096), 1), 256, 0, st>>>(pa);
  RFDD_CHECK_LAUNCH();
  // B staged through shared memory (rows of B read along their length): ntc * 2 half-tile column
  // blocks per K tile, every one inside the ntc x nkt tiles reserved for B above
  pack_b_t_kernel<<<dim3((unsigned)(ntc * 2 * nkt), 1), 256, 0, st>>>(pbb);
  RFDD_CHECK_LAUNCH();
  tc_gemm_kernel<<<std::max(1, std::min(tb.total_tiles, nsm)), TC_THREADS, TC_SMEM, st>>>(tb, (float)alpha,
                                                                                      (float)beta);
  RFDD_CHECK_LAUNCH();
  int status = 0;
  RFDD_CUDA(cudaMemcpyAsync(&status, na.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RFDD_CUDA(cudaStreamSynchronize(st));
  return status;
}

}  // namespace rfdd
