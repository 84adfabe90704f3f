// Tensor-core Gram / projection kernel of the mixed merge evaluation.
#pragma once

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
  const void* mapA;  // optional 2-D TMA tensor map of A (box 32 rows x 128 cols), device memory
  const void* mapU;  // optional tensor map of U (same box); both or neither
};

// A 128 x 128 output tile: kind 0 -> rows from U (P), kind 1 -> rows from A (G).
struct TcTile {
  int item, kind, row0, col0;
};

// Two rings: f32 staging slots filled by TMA (deep, to cover the load
// latency) and split bf16 operand slots read by the MMAs.
constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 32;
constexpr int kTcStagesF = 5, kTcStagesB = 2;
constexpr int kTcConvWarps = 16;  // split warps: one 8-deep chunk of one row each
constexpr int kTcThreads = (2 + kTcConvWarps + 4) * 32;
constexpr int kTcStageF = 2 * kTcBK * kTcBM * 4;  // 32 KB: A and B rows, f32
constexpr int kTcStageB = 4 * kTcBM * kTcBK * 2;  // 32 KB: A hi/lo, B hi/lo, bf16
constexpr int kTcSmemBytes = kTcStagesF * kTcStageF + kTcStagesB * kTcStageB + 2048;

cudaError_t launch_tc_gram(const TcItem* d_items, const TcTile* d_tiles, int n_tiles,
                           int n_ctas, int* d_status, cudaStream_t s);

}  // namespace csvd
