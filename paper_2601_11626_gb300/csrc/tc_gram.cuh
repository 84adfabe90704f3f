// Tensor-core Gram / projection kernel of the mixed merge evaluation.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace csvd {

// One candidate block A (m x k, f32, 16-byte aligned, ld % 4 == 0) and the
// basis U (m x rt, f32, 16-byte aligned, ldu % 4 == 0) of its state.
struct TcItem {
  const float* A;
  int64_t lda;
  const float* U;
  int64_t ldu;
  int m, k, rt, pad;
  float* P;      // rt x k, row-major ldp:  P = U^T A
  int64_t ldp;
  float* G;      // k x k, row-major ldg:   G = A^T A (tiles on and above the diagonal)
  int64_t ldg;   // P and G take 16-byte stores when ldp, ldg % 4 == 0 and 16-byte aligned
  double* colE;  // k column energies sum_i A_ic^2, accumulated (zeroed before the launch)
  const void* mapA;  // 2-D TMA tensor map of A (tc_tensor_map), device memory
  const void* mapU;  // tensor map of U (any valid map when rt == 0)
};

// A 128 x 128 output tile: kind 0 -> rows from U (P), kind 1 -> rows from A (G).
struct TcTile {
  int item, kind, row0, col0;
};

// Output tile 128 x 128.  A staging slot holds kTcBK rows of both operands
// as TMA boxes of kTcBK rows x kTcBox f32 columns (128 bytes, 128-byte
// swizzle), four boxes per 128-column panel; an operand slot holds the
// three bf16 parts of both operands in the MN-major 128-byte-swizzled UMMA
// layout (two 64-column atoms of kTcBK rows per part).
constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 32, kTcBox = 32;
// Ring depths: staging slots (F), operand slots (B) and stage accumulators
// in TMEM (X; the running sum takes one more 128-column buffer, X + 1 <= 4).
#ifndef CSVD_TC_STAGES_F
#define CSVD_TC_STAGES_F 4
#endif
#ifndef CSVD_TC_STAGES_B
#define CSVD_TC_STAGES_B 2
#endif
#ifndef CSVD_TC_XBUF
#define CSVD_TC_XBUF 2
#endif
constexpr int kTcStagesF = CSVD_TC_STAGES_F, kTcStagesB = CSVD_TC_STAGES_B;
constexpr int kTcXBuf = CSVD_TC_XBUF;
static_assert(kTcXBuf >= 2 && kTcXBuf <= 3, "two or three stage accumulators");
constexpr int kTcConvWarps = 8;  // warps splitting f32 into bf16 parts
constexpr int kTcEpiWarps = 8;   // two per TMEM lane quarter
constexpr int kTcThreads = (2 + kTcConvWarps + kTcEpiWarps) * 32;
constexpr int kTcBoxBytes = kTcBK * kTcBox * 4;                 // 4 KB
constexpr int kTcStageF = 2 * (kTcBM / kTcBox) * kTcBoxBytes;   // 32 KB: A and B, f32
constexpr int kTcPartBytes = kTcBK * kTcBM * 2;                 // 8 KB: one bf16 part
constexpr int kTcStageB = 6 * kTcPartBytes;                     // 48 KB: 3 parts x 2 operands
constexpr int kTcSmemBytes = kTcStagesF * kTcStageF + kTcStagesB * kTcStageB + 1024 + 256;
static_assert(kTcSmemBytes <= 227 * 1024, "one CTA per SM");

// Encodes the tensor map the kernel expects for a row-major f32 matrix
// (rows x cols, leading dimension ld floats): box kTcBK rows x kTcBox
// columns, 128-byte swizzle, zero fill outside the matrix.  False when the
// driver entry point is unavailable or rejects the matrix (alignment).
bool tc_tensor_map(const void* ptr, int64_t cols, int64_t rows, int64_t ld, CUtensorMap* out);

cudaError_t launch_tc_gram(const TcItem* d_items, const TcTile* d_tiles, int n_tiles,
                           int n_ctas, int* d_status, cudaStream_t s);

}  // namespace csvd
