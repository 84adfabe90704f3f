// P = U^T A and G = A^T A for a batch of uneven candidates on the 5th-gen
// tensor cores (tcgen05), in one pass over each candidate, together with the
// exact column energies sum_i A_ic^2.
//
// These are the products the mixed merge evaluation needs: the Gram of the
// core, K^T K = [[S, diag(s) P], [P^T diag(s), A^T A]], is assembled from
// them (Lemma 1 with the residual folded into A^T A = P^T P + B^T B).
//
// Accuracy: every f32 operand x is split on the CUDA cores into three bf16
// parts, x = hi + mid + lo exactly (8 significant bits each, no underflow
// for the magnitudes met here); each 16-deep step issues six kind::f16 MMAs,
// hi*hi + hi*mid + mid*hi + hi*lo + lo*hi + mid*mid, accumulating in f32 in
// tensor memory.  The dropped mid*lo, lo*mid and lo*lo terms are below
// 2^-25 |x||y| per product (split-operand emulation after Ootomo & Yokota
// 2022, with three parts), so the products carry FP32-level accuracy and
// only the FP32 accumulation rounds.  The diagonal of A^T A is replaced by
// the exact column energies (compensated f32 sums, added in FP64).
//
// Layout: TMA lands each stage's 32 rows of both operands in a staging slot
// as boxes of 32 rows x 32 f32 columns with the 128-byte swizzle.  The split
// warps re-chunk them, without transposing, into the MN-major
// 128-byte-swizzled UMMA layout of bf16: per part and operand two atoms of
// 64 columns x 32 rows (4 KB each, rows 128 bytes apart, 16-byte chunks
// XOR-ed with the row), 8-row groups 1 KB apart along K.
//
// Structure: persistent CTAs walk a list of 128 x 128 output tiles (tiles of
// one candidate are adjacent so its columns stay in L2 while they are
// reused).  Warp roles, connected by mbarrier rings:
//   warp 0      TMA: up to four boxes per operand per stage into a 4-deep
//               staging ring
//   warps 2-9   split staging f32 into the bf16 parts of a 2-deep operand
//               ring; on diagonal tiles also the column sums of squares
//   warp 1      one thread issues tcgen05.mma (M = 128, K = 16, N = the
//               tile's valid columns rounded up to 16) into a fresh f32
//               accumulator per stage (kTcXBuf in TMEM, in turn) and commits
//   warps 10-17 add each stage's accumulator into the tile's running sum
//               (round to nearest, kept in TMEM) and store the last one;
//               the tensor cores' own accumulation truncates, so a long
//               chain of additions inside one accumulator would shrink every
//               sum by about half an ulp per addition
// Every mbarrier wait is bounded (2 s of device time); on expiry the CTA
// sets an abort flag, drains its own copies and MMAs, frees TMEM and
// reports kStatusWaitCap.
#include <mutex>

#include <cudaTypedefs.h>

#include "tc_gram.cuh"

namespace csvd {
namespace {

// staging slot: A boxes then B boxes (f32); operand slot: parts of A, then of B
constexpr int kStA = 0;
constexpr int kStB = (kTcBM / kTcBox) * kTcBoxBytes;
constexpr int kOpA = 0;                 // hi, mid, lo of A at kOpA + p * kTcPartBytes
constexpr int kOpB = 3 * kTcPartBytes;  // hi, mid, lo of B
constexpr int kOpBase = kTcStagesF * kTcStageF;  // operand ring after the staging ring
constexpr int kAtomBytes = kTcBK * 128;          // one 64-column bf16 atom of 32 rows
constexpr uint64_t kWaitNs = 2000000000ull;
// limit of the pipeline waits (kWaitNs; shortened only by the failure-path
// test hook); the drains after an abort always keep kWaitNs
__device__ unsigned long long d_wait_ns = kWaitNs;
// TMEM columns: two stage accumulators X and the running sum S of a tile
constexpr uint32_t kXCol0 = 0, kSCol0 = kTcXBuf * kTcBN, kTmemCols = 512;
// failure-path test hook: the MMA role first waits on a barrier nothing
// arrives at (so the bounded wait runs out); 0 in normal operation
__device__ int d_stall_test = 0;
static_assert(kTcConvWarps == 8, "four split warps per 64-column atom");

// kind::f16 instruction descriptor: f32 accumulate, bf16 A and B, both
// MN-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);
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
  const uint64_t limit = honour_abort ? (uint64_t)d_wait_ns : kWaitNs;
  for (uint32_t it = 1; it < 0x7fffffffu; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 63u) == 0) {
      if (honour_abort && *abort_flag) return false;
      if (gtimer() - t0 > limit) {
        *abort_flag = 1;
        return false;
      }
    }
  }
  *abort_flag = 1;
  return false;
}

// Warp-uniform wait: lane 0 polls, the result is broadcast.
__device__ __forceinline__ bool warp_wait(uint32_t a, uint32_t parity, volatile int* abort_flag) {
  bool ok = false;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(a, parity, abort_flag);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// One 2-D tensor box (32 rows x 32 f32 columns from column x, row y) into
// shared memory, 128-byte swizzled; out-of-range elements arrive as zeros.
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

// Shared-memory matrix descriptor of an MN-major bf16 operand with the
// 128-byte swizzle: atoms of 64 elements (MN) x 8 rows (K), 1 KB, aligned to
// 1 KB.  Leading byte offset = the stride between 64-column atoms (4 KB),
// stride byte offset = the stride between 8-row groups along K (1 KB).
// Descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t mn_sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(kAtomBytes >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
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

// tcgen05.ld of 32 columns without the wait (pair with tmem_wait_ld).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
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
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
}

// Split 8 f32 values into three bf16 parts (x = hi + mid + lo) and store
// each part as one 16-byte chunk.
__device__ __forceinline__ void split3_store(uint8_t* hi, uint8_t* mid, uint8_t* lo, uint32_t off,
                                             const float* x) {
  uint32_t h[4], md[4], l[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * p], x[2 * p + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const float r0 = x[2 * p] - hf.x, r1 = x[2 * p + 1] - hf.y;
    const __nv_bfloat162 mb = __floats2bfloat162_rn(r0, r1);
    const float2 mf = __bfloat1622float2(mb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
    h[p] = *reinterpret_cast<const uint32_t*>(&hb);
    md[p] = *reinterpret_cast<const uint32_t*>(&mb);
    l[p] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(mid + off) = make_uint4(md[0], md[1], md[2], md[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// s + c += x^2 without rounding loss: the square's rounding error by FMA,
// the sum's by a two-sum.
__device__ __forceinline__ void acc_sq(float& s, float& c, float x) {
  const float p = x * x;
  const float e = fmaf(x, x, -p);
  const float t = s + p;
  const float z = t - s;
  c += ((s - (t - z)) + (p - z)) + e;
  s = t;
}

struct TileInfo {
  const void* mapa;
  const void* mapb;
  int xa, xb;        // first column of each operand inside its map
  int validA, validB, m;
  int nbA, nbB;      // boxes loaded per operand
  bool diag;
  float* out;
  int64_t ldo;
  double* colE;      // column energies of the diagonal tile's columns (or null)
  int kcols;         // columns of A past col0 (bounds the energy writes)
};

__device__ __forceinline__ TileInfo tile_info(const TcItem* items, const TcTile& t) {
  const TcItem d = items[t.item];
  TileInfo ti;
  if (t.kind == 0) {
    ti.validA = min(kTcBM, d.rt - t.row0);
    ti.out = d.P + (int64_t)t.row0 * d.ldp + t.col0;
    ti.ldo = d.ldp;
    ti.mapa = d.mapU;
  } else {
    ti.validA = min(kTcBM, d.k - t.row0);
    ti.out = d.G + (int64_t)t.row0 * d.ldg + t.col0;
    ti.ldo = d.ldg;
    ti.mapa = d.mapA;
  }
  ti.mapb = d.mapA;
  ti.xa = t.row0;
  ti.xb = t.col0;
  ti.validB = min(kTcBN, d.k - t.col0);
  ti.m = d.m;
  ti.diag = (t.kind == 1 && t.row0 == t.col0);
  ti.nbA = (ti.validA + kTcBox - 1) / kTcBox;
  ti.nbB = ti.diag ? 0 : (ti.validB + kTcBox - 1) / kTcBox;
  ti.colE = (ti.diag && d.colE) ? d.colE + t.col0 : nullptr;
  ti.kcols = d.k - t.col0;
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
  constexpr int F = kTcStagesF, B = kTcStagesB;
  const uint32_t b0 = smem_u32(bars);
  auto full_st = [&](int s) { return b0 + 8u * s; };
  auto empty_st = [&](int s) { return b0 + 8u * (F + s); };
  // Operand slot s and stage accumulator s are used by the same stages
  // (B == X): ready(s) completes when the split warps have filled the slot
  // and the epilogue has drained the accumulator two stages back, so the MMA
  // thread waits once per stage; done(s) is the stage's single MMA commit,
  // which frees the slot and hands the accumulator to the epilogue.
  constexpr int X = kTcXBuf;
  static_assert(X == B, "one barrier pair per operand slot and accumulator");
  auto ready = [&](int s) { return b0 + 8u * (2 * F + s); };
  auto done = [&](int s) { return b0 + 8u * (2 * F + B + s); };
  const uint32_t final_bar = b0 + 8u * (2 * F + 2 * B + 2 * X);
  const uint32_t stall_bar = b0 + 8u * (2 * F + 2 * B + 2 * X + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * F + 2 * B + 2 * X + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < F; ++s) {
      mbar_init(full_st(s), 1);
      mbar_init(empty_st(s), kTcConvWarps);
    }
    for (int s = 0; s < B; ++s) {
      mbar_init(ready(s), kTcConvWarps + kTcEpiWarps);
      mbar_init(done(s), 1);
    }
    mbar_init(final_bar, 1);
    mbar_init(stall_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
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
      const int nkb = (ti.m + kTcBK - 1) / kTcBK;
      const uint32_t bytes = (uint32_t)(ti.nbA + ti.nbB) * (uint32_t)kTcBoxBytes;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int slot = it % F;
        const uint32_t ph = (it / F) & 1u;
        if (!warp_wait(empty_st(slot), ph ^ 1u, abort_flag)) { ok = false; break; }
        if (lane == 0) {
          uint8_t* st = smem + slot * kTcStageF;
          mbar_arrive_tx(full_st(slot), bytes);
          for (int j = 0; j < ti.nbA; ++j)
            tma_box(smem_u32(st + kStA + j * kTcBoxBytes), ti.mapa, ti.xa + j * kTcBox,
                    kb * kTcBK, full_st(slot));
          for (int j = 0; j < ti.nbB; ++j)
            tma_box(smem_u32(st + kStB + j * kTcBoxBytes), ti.mapb, ti.xb + j * kTcBox,
                    kb * kTcBK, full_st(slot));
        }
        __syncwarp();
      }
    }
    // drain copies still in flight (all consumed on a normal exit)
    if (lane == 0) {
      const uint32_t n_last = it < (uint32_t)F ? it : (uint32_t)F;
      for (uint32_t j = it - n_last; j < it; ++j)
        mbar_wait(full_st(j % F), (j / F) & 1u, abort_flag, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA
    // Every stage (32 rows) goes into a fresh accumulator X[it % 2]; the
    // epilogue adds the stages with round-to-nearest (the accumulator itself
    // truncates each addition).  Within a stage the ten small cross terms
    // come first and the two hi*hi products last, so the truncated additions
    // act on small partial sums.
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      if (d_stall_test) ok = mbar_wait(stall_bar, 0u, abort_flag);  // runs out: nothing arrives
      for (int tt = blockIdx.x; ok && tt < n_tiles; tt += gridDim.x) {
        const TileInfo ti = tile_info(items, tiles[tt]);
        const int nkb = (ti.m + kTcBK - 1) / kTcBK;
        // N = the valid columns rounded up to 16: columns past them are not stored
        const uint32_t idesc = idesc_n(min(kTcBN, (ti.validB + 15) & ~15));
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int slot = it % B;
          const uint32_t xb = it % X;
          if (!mbar_wait(ready(slot), (it / B) & 1u, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dt = tmem_base + kXCol0 + xb * (uint32_t)kTcBN;
          const uint32_t op = smem_u32(smem + kOpBase + slot * kTcStageB);
          const uint32_t a0 = op + kOpA, b0p = ti.diag ? a0 : op + kOpB;
          // the descriptors of a stage differ only in their start address
          // field: add the part and row-group offsets (in 16-byte units)
          constexpr uint64_t kPartD = kTcPartBytes >> 4, kRowsD = 2048 >> 4;
          const uint64_t da = mn_sw128_desc(a0), db = mn_sw128_desc(b0p);
          uint32_t accf = 0u;
#pragma unroll
          for (int s16 = 0; s16 < kTcBK / 16; ++s16) {
            // rows 16 s16 .. 16 s16 + 15 of each atom
            const uint64_t ah = da + s16 * kRowsD, am = ah + kPartD, al = ah + 2 * kPartD;
            const uint64_t bh = db + s16 * kRowsD, bm = bh + kPartD, bl = bh + 2 * kPartD;
            umma(dt, am, bm, idesc, accf);
            accf = 1u;
            umma(dt, al, bh, idesc, 1u);
            umma(dt, ah, bl, idesc, 1u);
            umma(dt, am, bh, idesc, 1u);
            umma(dt, ah, bm, idesc, 1u);
          }
#pragma unroll
          for (int s16 = 0; s16 < kTcBK / 16; ++s16)
            umma(dt, da + s16 * kRowsD, db + s16 * kRowsD, idesc, 1u);
          umma_commit(done(slot));
        }
      }
      // all issued MMAs complete before TMEM is released
      umma_commit(final_bar);
      mbar_wait(final_bar, 0, abort_flag, false);
    }
    __syncwarp();
  } else if (warp < 2 + kTcConvWarps) {
    // ---------------------------------------------------- converters
    // Warp w splits rows 8 (w % 4) .. + 7 of the 64-column atom w / 4 of each
    // operand.  Lane l writes bf16 chunk l % 8 (columns 64 (w / 4) + 8 (l % 8)
    // .. + 7) of rows 8 (w % 4) + 4 i + l / 8: a quarter warp writes one
    // whole 128-byte row (bank-conflict free) and reads the two f32 chunks
    // holding its eight columns, odd chunk first in the upper half of the
    // quarter so that its reads hit distinct banks.  Each thread keeps the
    // same eight columns, for the column energies.
    const int w = warp - 2;
    const int jb = w >> 2;                // bf16 atom (64 columns)
    const int cb = lane & 7;              // bf16 chunk in the row
    const int jf = 2 * jb + (cb >> 2);    // f32 box holding its columns
    const int lc0 = 2 * (cb & 3);         // first f32 chunk in that box
    const int swap = cb >> 2;
    const int rbase = 8 * (w & 3) + (lane >> 3);
    uint32_t it = 0;
    bool ok = true;
    for (int tt = blockIdx.x; ok && tt < n_tiles; tt += gridDim.x) {
      const TileInfo ti = tile_info(items, tiles[tt]);
      const int nkb = (ti.m + kTcBK - 1) / kTcBK;
      const bool do_a = 64 * jb < ti.validA, do_b = !ti.diag && 64 * jb < ti.validB;
      const bool energies = ti.colE != nullptr && do_a;
      float es[8], ec[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) es[e] = ec[e] = 0.f;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int fs = it % F, bs = it % B;
        if (!warp_wait(full_st(fs), (it / F) & 1u, abort_flag)) { ok = false; break; }
        if (!warp_wait(done(bs), ((it / B) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        const uint8_t* st = smem + fs * kTcStageF;
        uint8_t* op = smem + kOpBase + bs * kTcStageB;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int r = rbase + 4 * i;
          const uint32_t src = (uint32_t)(jf * kTcBoxBytes + r * 128);
          const uint32_t c0 = (uint32_t)(((lc0 + swap) ^ (r & 7)) << 4);
          const uint32_t c1 = (uint32_t)(((lc0 + 1 - swap) ^ (r & 7)) << 4);
          const uint32_t dst = (uint32_t)(jb * kAtomBytes + r * 128 + ((cb ^ (r & 7)) << 4));
          float x[8];
          if (do_a) {
            const float4 u = *reinterpret_cast<const float4*>(st + kStA + src + c0);
            const float4 v = *reinterpret_cast<const float4*>(st + kStA + src + c1);
            const float4 p0 = swap ? v : u, p1 = swap ? u : v;
            x[0] = p0.x; x[1] = p0.y; x[2] = p0.z; x[3] = p0.w;
            x[4] = p1.x; x[5] = p1.y; x[6] = p1.z; x[7] = p1.w;
            split3_store(op + kOpA, op + kOpA + kTcPartBytes, op + kOpA + 2 * kTcPartBytes, dst, x);
            if (energies) {
#pragma unroll
              for (int e = 0; e < 8; ++e) acc_sq(es[e], ec[e], x[e]);
            }
          }
          if (do_b) {
            const float4 u = *reinterpret_cast<const float4*>(st + kStB + src + c0);
            const float4 v = *reinterpret_cast<const float4*>(st + kStB + src + c1);
            const float4 p0 = swap ? v : u, p1 = swap ? u : v;
            x[0] = p0.x; x[1] = p0.y; x[2] = p0.z; x[3] = p0.w;
            x[4] = p1.x; x[5] = p1.y; x[6] = p1.z; x[7] = p1.w;
            split3_store(op + kOpB, op + kOpB + kTcPartBytes, op + kOpB + 2 * kTcPartBytes, dst, x);
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(ready(bs));
          mbar_arrive(empty_st(fs));
        }
      }
      if (energies && ok) {
        // sum over the warp's rows (lanes with the same chunk), one FP64 add
        // per column and warp
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          double v = (double)es[e] + (double)ec[e];
          v += __shfl_xor_sync(0xffffffffu, v, 8);
          v += __shfl_xor_sync(0xffffffffu, v, 16);
          const int col = 64 * jb + 8 * cb + e;
          if (lane < 8 && col < ti.kcols && col < kTcBN) atomicAdd(&ti.colE[col], v);
        }
      }
    }
  } else {
    // ------------------------------------------------------ epilogue
    // Per stage: S = X (first stage) or S += X, kept in TMEM columns
    // [kSCol0, kSCol0 + 128); at the tile's last stage S + X goes to global
    // memory instead.  Row r of the tile lives in TMEM lane r; two warps
    // share each lane quarter, 64 columns each, and load a chunk of X and of
    // S before waiting once.
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int half = (warp - 2 - kTcConvWarps) >> 2;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int r = q * 32 + lane;
    // both accumulators start empty: the first stage of each slot needs no drain
    if (lane == 0)
      for (int a = 0; a < X; ++a) mbar_arrive(ready(a));
    uint32_t it = 0;
    bool ok = true;
    for (int tt = blockIdx.x; ok && tt < n_tiles; tt += gridDim.x) {
      const TileInfo ti = tile_info(items, tiles[tt]);
      const int nkb = (ti.m + kTcBK - 1) / kTcBK;
      const bool vec = (ti.ldo & 3) == 0 && (reinterpret_cast<uintptr_t>(ti.out) & 15) == 0;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const uint32_t xb = it % X;
        if (!warp_wait(done(xb), (it / X) & 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const bool last = kb + 1 == nkb;
        bool stored = false;
#pragma unroll 1
        for (int c2 = 0; c2 < 2; ++c2) {
          const int cc = 2 * half + c2;
          const int nv = ti.validB - cc * 32;  // valid columns of this chunk (same in every lane)
          if (nv <= 0) break;
          uint32_t xv[32], sv[32];
          tmem_ld32_async(tmem_base + lane_off + kXCol0 + xb * (uint32_t)kTcBN + cc * 32, xv);
          if (kb > 0) tmem_ld32_async(tmem_base + lane_off + kSCol0 + cc * 32, sv);
          tmem_wait_ld();
          float v[32];
#pragma unroll
          for (int e = 0; e < 32; ++e)
            v[e] = __uint_as_float(xv[e]) + (kb > 0 ? __uint_as_float(sv[e]) : 0.f);
          if (!last) {
            tmem_st32(tmem_base + lane_off + kSCol0 + cc * 32, v);
            stored = true;
          } else if (r < ti.validA) {
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
        if (stored) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(ready(xb));  // counts toward stage it + X
      }
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, kStatusWaitCap);
}

// ------------------------------------------------------- TMA tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

cudaError_t tc_set_wait_ns(long long ns, int stall) {
  const unsigned long long v = ns < 0 ? kWaitNs : (unsigned long long)ns;
  cudaError_t e = cudaMemcpyToSymbol(d_wait_ns, &v, sizeof(v));
  const int st = stall > 0 ? 1 : 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(d_stall_test, &st, sizeof(int));
  return e;
}

bool tc_tensor_map(const void* ptr, int64_t cols, int64_t rows, int64_t ld, CUtensorMap* out) {
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) != 0 || (ld & 3) != 0 || cols < 1 || rows < 1)
    return false;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)kTcBox, (cuuint32_t)kTcBK};
  cuuint32_t es[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_tc_gram(const TcItem* d_items, const TcTile* d_tiles, int n_tiles, int n_ctas,
                           int* d_status, cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  static std::atomic<int> set_smem{0};
  if (cudaError_t e = ensure_smem(tc_gram_kernel, kTcSmemBytes, set_smem)) return e;
  if (n_ctas > n_tiles) n_ctas = n_tiles;
  prof_begin(s);
  tc_gram_kernel<<<n_ctas, kTcThreads, kTcSmemBytes, s>>>(d_items, d_tiles, n_tiles, d_status);
  prof_end("tc_gram", s);
  return cudaGetLastError();
}

}  // namespace csvd
