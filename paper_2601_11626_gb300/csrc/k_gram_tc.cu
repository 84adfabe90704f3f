// P = U^T A and G = A^T A for a batch of uneven candidates on the 5th-gen
// tensor cores (tcgen05), in one pass over each candidate.
//
// These are the two products the mixed merge evaluation needs: the Gram of
// the core, K^T K = [[S, diag(s) P], [P^T diag(s), A^T A]], is assembled from
// them (Lemma 1 with the residual folded into A^T A = P^T P + B^T B).
//
// Accuracy: every f32 operand x is split into bf16 parts x = hi + lo (+ a
// remainder below 2^-17 |x|); each 16-deep step issues three MMAs,
// hi*hi + hi*lo + lo*hi, accumulating in f32 in tensor memory, which keeps
// the products at f32-level accuracy (split-operand emulation, after Ootomo &
// Yokota 2022).
//
// Structure: persistent CTAs walk a list of 128 x 128 output tiles (tiles of
// one candidate are adjacent so its columns stay in L2 while they are
// reused).  Warp roles, connected by mbarrier rings:
//   warp 0      TMA: one 2-D tensor box (32 rows x 128 f32 columns, zero
//               outside the matrix) per operand into a 5-deep staging ring
//               (one cp.async.bulk per row when no tensor map is given)
//   warps 2-17  split staging f32 -> bf16 hi/lo into a 2-deep operand
//               ring, K-major with the 64-byte swizzle the UMMA
//               descriptors expect (one 8-deep chunk of one row per thread)
//   warp 1      one thread issues tcgen05.mma (M = 128, K = 16, N = the
//               tile's valid columns rounded up to 16) into a
//               double-buffered f32 accumulator in TMEM and commits
//   warps 18-21 tcgen05.ld the finished accumulator and store it
// Every mbarrier wait is bounded (2 s of device time); on expiry the CTA
// sets an abort flag, drains its own copies and MMAs, frees TMEM and
// reports kStatusWaitCap.
#include "tc_gram.cuh"

namespace csvd {
namespace {

// staging slot: f32 [32][128] for each operand
constexpr int kStA = 0;
constexpr int kStB = kStA + kTcBK * kTcBM * 4;
static_assert(kStB + kTcBK * kTcBN * 4 == kTcStageF, "staging layout");
// operand slot: bf16 [128][32] swizzled, hi and lo of each operand
constexpr int kAhi = 0;
constexpr int kAlo = kAhi + kTcBM * kTcBK * 2;
constexpr int kBhi = kAlo + kTcBM * kTcBK * 2;
constexpr int kBlo = kBhi + kTcBN * kTcBK * 2;
static_assert(kBlo + kTcBN * kTcBK * 2 == kTcStageB, "operand layout");
constexpr int kOpBase = kTcStagesF * kTcStageF;  // operand ring after the staging ring
constexpr uint64_t kWaitNs = 2000000000ull;

// kind::f16 instruction descriptor: f32 accumulate, bf16 A and B, both
// K-major, N = 128, M = 128.
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kTcBM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait.  Returns false when the 2 s budget is spent (and raises the
// abort flag) or, if honour_abort, when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag,
                                          bool honour_abort = true) {
  if (mbar_try(a, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t it = 1; it < 0x7fffffffu; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 63u) == 0) {
      if (honour_abort && *abort_flag) return false;
      if (gtimer() - t0 > kWaitNs) {
        *abort_flag = 1;
        return false;
      }
    }
  }
  *abort_flag = 1;
  return false;
}

// Warp-uniform wait: lane 0 polls, the verdict is broadcast.
__device__ __forceinline__ bool warp_wait(uint32_t a, uint32_t parity, volatile int* abort_flag) {
  bool ok = false;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(a, parity, abort_flag);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// One 2-D tensor box (32 rows x 128 f32 columns starting at column x, row y)
// into shared memory; out-of-range rows and columns arrive as zeros.
__device__ __forceinline__ void tma_box(uint32_t dst, const void* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of the 16-byte chunk (row, chunk) in a K-major 64B-swizzled
// tile of 32 bf16 per row.
__device__ __forceinline__ uint32_t sw64_off(int row, int chunk) {
  const int r8 = row & 7;
  return (uint32_t)((row >> 3) * 512 + r8 * 64 + ((chunk ^ (r8 >> 1)) & 3) * 16);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
  return lo | (hi << 16);
}

// Split 8 f32 values of one row/chunk into hi and lo bf16 chunks
// (x = hi + lo + a remainder below 2^-17 |x|), two values per conversion.
__device__ __forceinline__ void split_store(uint8_t* hi_base, uint8_t* lo_base, uint32_t off,
                                            const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * p], x[2 * p + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * p] - hf.x, x[2 * p + 1] - hf.y);
    h[p] = *reinterpret_cast<const uint32_t*>(&hb);
    l[p] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  *reinterpret_cast<uint4*>(hi_base + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo_base + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

struct TileInfo {
  const void* mapa;  // tensor maps (null: per-row bulk copies)
  const void* mapb;
  int xa, xb;        // first column of each operand inside its map
  const float* Xa;  // rows operand source (U or A), shifted to its first column
  int64_t lda;
  const float* Xb;  // columns operand source (A), shifted to its first column
  int64_t ldb;
  int validA, validB, m;
  bool diag;
  float* out;
  int64_t ldo;
};

__device__ __forceinline__ TileInfo tile_info(const TcItem* items, const TcTile& t) {
  const TcItem d = items[t.item];
  TileInfo ti;
  if (t.kind == 0) {
    ti.Xa = d.U + t.row0;
    ti.lda = d.ldu;
    ti.validA = min(kTcBM, d.rt - t.row0);
    ti.out = d.P + (int64_t)t.row0 * d.ldp + t.col0;
    ti.ldo = d.ldp;
  } else {
    ti.Xa = d.A + t.row0;
    ti.lda = d.lda;
    ti.validA = min(kTcBM, d.k - t.row0);
    ti.out = d.G + (int64_t)t.row0 * d.ldg + t.col0;
    ti.ldo = d.ldg;
  }
  ti.Xb = d.A + t.col0;
  ti.ldb = d.lda;
  ti.mapa = (t.kind == 0) ? d.mapU : d.mapA;
  ti.mapb = d.mapA;
  ti.xa = t.row0;
  ti.xb = t.col0;
  ti.validB = min(kTcBN, d.k - t.col0);
  ti.m = d.m;
  ti.diag = (t.kind == 1 && t.row0 == t.col0);
  return ti;
}

}  // namespace

__global__ void __launch_bounds__(kTcThreads, 1)
tc_gram_kernel(const TcItem* __restrict__ items, const TcTile* __restrict__ tiles, int n_tiles,
               int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOpBase + kTcStagesB * kTcStageB);
  // barrier slots
  const uint32_t b0 = smem_u32(bars);
  constexpr int F = kTcStagesF, B = kTcStagesB;
  auto full_st = [&](int s) { return b0 + 8u * s; };
  auto empty_st = [&](int s) { return b0 + 8u * (F + s); };
  auto full_bf = [&](int s) { return b0 + 8u * (2 * F + s); };
  auto empty_bf = [&](int s) { return b0 + 8u * (2 * F + B + s); };
  auto tmem_full = [&](int a) { return b0 + 8u * (2 * F + 2 * B + a); };
  auto tmem_empty = [&](int a) { return b0 + 8u * (2 * F + 2 * B + 2 + a); };
  const uint32_t final_bar = b0 + 8u * (2 * F + 2 * B + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * F + 2 * B + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStagesF; ++s) {
      mbar_init(full_st(s), 1);
      mbar_init(empty_st(s), kTcConvWarps);
    }
    for (int s = 0; s < kTcStagesB; ++s) {
      mbar_init(full_bf(s), kTcConvWarps);
      mbar_init(empty_bf(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tmem_full(a), 1);
      mbar_init(tmem_empty(a), 4);
    }
    mbar_init(final_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------- producer
    uint32_t it = 0;
    bool ok = true;
    for (int tt = blockIdx.x; ok && tt < n_tiles; tt += gridDim.x) {
      const TileInfo ti = tile_info(items, tiles[tt]);
      const uint32_t bytesA = 4u * (uint32_t)((ti.validA + 3) & ~3);
      const uint32_t bytesB = ti.diag ? 0u : 4u * (uint32_t)((ti.validB + 3) & ~3);
      const int nkb = (ti.m + kTcBK - 1) / kTcBK;
      const bool use_map = ti.mapa != nullptr && ti.mapb != nullptr;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int slot = it % kTcStagesF;
        const uint32_t ph = (it / kTcStagesF) & 1u;
        if (!warp_wait(empty_st(slot), ph ^ 1u, abort_flag)) { ok = false; break; }
        if (use_map) {
          // one tensor box per operand: full box bytes (zero-filled outside)
          if (lane == 0) {
            uint8_t* st = smem + slot * kTcStageF;
            const uint32_t box = (uint32_t)(kTcBK * kTcBM * 4);
            mbar_arrive_tx(full_st(slot), ti.diag ? box : 2u * box);
            tma_box(smem_u32(st + kStA), ti.mapa, ti.xa, kb * kTcBK, full_st(slot));
            if (!ti.diag) tma_box(smem_u32(st + kStB), ti.mapb, ti.xb, kb * kTcBK, full_st(slot));
          }
          __syncwarp();
          continue;
        }
        const int rows = min(kTcBK, ti.m - kb * kTcBK);
        if (lane == 0) mbar_arrive_tx(full_st(slot), (uint32_t)rows * (bytesA + bytesB));
        __syncwarp();
        if (lane < rows) {
          const int64_t l = (int64_t)kb * kTcBK + lane;
          uint8_t* st = smem + slot * kTcStageF;
          bulk_g2s(smem_u32(st + kStA + lane * (kTcBM * 4)), ti.Xa + l * ti.lda, bytesA,
                   full_st(slot));
          if (!ti.diag)
            bulk_g2s(smem_u32(st + kStB + lane * (kTcBN * 4)), ti.Xb + l * ti.ldb, bytesB,
                     full_st(slot));
        }
      }
    }
    // drain copies still in flight (all consumed on a normal exit)
    if (lane == 0) {
      const uint32_t n_last = it < (uint32_t)kTcStagesF ? it : (uint32_t)kTcStagesF;
      for (uint32_t j = it - n_last; j < it; ++j)
        mbar_wait(full_st(j % kTcStagesF), (j / kTcStagesF) & 1u, abort_flag, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t it = 0, tc = 0;
      bool ok = true;
      for (int tt = blockIdx.x; ok && tt < n_tiles; tt += gridDim.x, ++tc) {
        const TileInfo ti = tile_info(items, tiles[tt]);
        const int nkb = (ti.m + kTcBK - 1) / kTcBK;
        const uint32_t acc = tc & 1u, aph = (tc >> 1) & 1u;
        if (!mbar_wait(tmem_empty(acc), aph ^ 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t dt = tmem_base + acc * (uint32_t)kTcBN;
        // N = the valid columns rounded up to 16: columns past them are not stored
        const uint32_t idesc = idesc_n(min(kTcBN, (ti.validB + 15) & ~15));
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int slot = it % kTcStagesB;
          const uint32_t ph = (it / kTcStagesB) & 1u;
          if (!mbar_wait(full_bf(slot), ph, abort_flag)) { ok = false; break; }
          tc_fence_after();
          uint8_t* st = smem + kOpBase + slot * kTcStageB;
          const uint32_t ahi = smem_u32(st + kAhi), alo = smem_u32(st + kAlo);
          const uint32_t bhi = ti.diag ? ahi : smem_u32(st + kBhi);
          const uint32_t blo = ti.diag ? alo : smem_u32(st + kBlo);
#pragma unroll
          for (int s = 0; s < kTcBK / 16; ++s) {
            const uint32_t o = s * 32;  // 16 bf16 along K
            const uint64_t dah = sw64_desc(ahi + o), dal = sw64_desc(alo + o);
            const uint64_t dbh = sw64_desc(bhi + o), dbl = sw64_desc(blo + o);
            umma(dt, dah, dbh, idesc, (kb | s) != 0 ? 1u : 0u);
            umma(dt, dah, dbl, idesc, 1u);
            umma(dt, dal, dbh, idesc, 1u);
          }
          umma_commit(empty_bf(slot));
        }
        if (!ok) break;
        umma_commit(tmem_full(acc));
      }
      // all issued MMAs complete before TMEM is released
      umma_commit(final_bar);
      mbar_wait(final_bar, 0, abort_flag, false);
    }
    __syncwarp();
  } else if (warp < 2 + kTcConvWarps) {
    // ---------------------------------------------------- converters
    // Thread -> (row, 8-deep chunk).  Rows past an operand's valid extent
    // are not split: they only feed output rows / columns that are never
    // stored (each output element depends on one row of each operand).
    const int tc = threadIdx.x - 64;  // 0 .. 32 kTcConvWarps - 1
    const int row = tc & 127;
    const int c = tc >> 7;
    uint32_t it = 0;
    bool ok = true;
    for (int tt = blockIdx.x; ok && tt < n_tiles; tt += gridDim.x) {
      const TileInfo ti = tile_info(items, tiles[tt]);
      const int nkb = (ti.m + kTcBK - 1) / kTcBK;
      const bool masked = ti.mapa == nullptr || ti.mapb == nullptr;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int fs = it % kTcStagesF, bs = it % kTcStagesB;
        if (!warp_wait(full_st(fs), (it / kTcStagesF) & 1u, abort_flag)) { ok = false; break; }
        if (!warp_wait(empty_bf(bs), ((it / kTcStagesB) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        const uint8_t* st = smem + fs * kTcStageF;
        uint8_t* op = smem + kOpBase + bs * kTcStageB;
        const float* sa = reinterpret_cast<const float*>(st + kStA);
        const float* sb = reinterpret_cast<const float*>(st + kStB);
        const uint32_t off = sw64_off(row, c);
        const bool do_a = row < ti.validA, do_b = !ti.diag && row < ti.validB;
        float x[8];
        if (masked) {
          // per-row copies leave rows past m unwritten: zero the K tail
          const int lmax = ti.m - kb * kTcBK;
          if (do_a) {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = (c * 8 + e < lmax) ? sa[(c * 8 + e) * kTcBM + row] : 0.f;
            split_store(op + kAhi, op + kAlo, off, x);
          }
          if (do_b) {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = (c * 8 + e < lmax) ? sb[(c * 8 + e) * kTcBN + row] : 0.f;
            split_store(op + kBhi, op + kBlo, off, x);
          }
        } else {
          // tensor boxes arrive zero-filled outside the matrix
          if (do_a) {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = sa[(c * 8 + e) * kTcBM + row];
            split_store(op + kAhi, op + kAlo, off, x);
          }
          if (do_b) {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = sb[(c * 8 + e) * kTcBN + row];
            split_store(op + kBhi, op + kBlo, off, x);
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(full_bf(bs));
          mbar_arrive(empty_st(fs));
        }
      }
    }
  } else {
    // ------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    uint32_t tc = 0;
    for (int tt = blockIdx.x; tt < n_tiles; tt += gridDim.x, ++tc) {
      const TileInfo ti = tile_info(items, tiles[tt]);
      const uint32_t acc = tc & 1u, aph = (tc >> 1) & 1u;
      if (!warp_wait(tmem_full(acc), aph, abort_flag)) break;
      tc_fence_after();
      const int r = q * 32 + lane;
      const bool vec = (ti.ldo & 3) == 0 && (reinterpret_cast<uintptr_t>(ti.out) & 15) == 0;
#pragma unroll 1
      for (int cc = 0; cc < kTcBN / 32; ++cc) {
        const int nv = ti.validB - cc * 32;  // valid columns of this chunk (same in every lane)
        if (nv <= 0) break;
        float v[32];
        tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + acc * (uint32_t)kTcBN + cc * 32, v);
        if (r < ti.validA) {
          float* o = ti.out + (int64_t)r * ti.ldo + cc * 32;
          if (vec) {
#pragma unroll
            for (int e4 = 0; e4 < 8; ++e4) {
              const int e = 4 * e4;
              if (e + 3 < nv) {
                *reinterpret_cast<float4*>(o + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
              } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  if (e + u < nv) o[e + u] = v[e + u];
              }
            }
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (e < nv) o[e] = v[e];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_empty(acc));
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(256)
                 : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, kStatusWaitCap);
}

cudaError_t launch_tc_gram(const TcItem* d_items, const TcTile* d_tiles, int n_tiles, int n_ctas,
                           int* d_status, cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  // per device and cheap: set on every launch
  cudaError_t e = cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kTcSmemBytes);
  if (e != cudaSuccess) return e;
  if (n_ctas > n_tiles) n_ctas = n_tiles;
  prof_begin(s);
  tc_gram_kernel<<<n_ctas, kTcThreads, kTcSmemBytes, s>>>(d_items, d_tiles, n_tiles, d_status);
  prof_end("tc_gram", s);
  return cudaGetLastError();
}

}  // namespace csvd
