// Batched FP32 SIMT GEMM over a flat tile list.
//
// Serves every small dense product of the plain path: the projection
// P = U^T A (Lemma 1, Y = Q_t^T A), the residual R = A - U P and its
// re-orthogonalisation, the Gram A^T A, the basis rotation
// U_new = U W_top + Q_res W_bot (Cor. 3) and the tail gradient
// 2 (I - U U^T) A.  Items of different shapes share one launch: the host
// lists only the 64x64 output tiles that exist, so uneven batches waste no
// CTAs.  Each CTA computes one tile with 256 threads (4x4 outputs each),
// staging 16-deep slices of both operands in shared memory.
#include "common.cuh"

namespace csvd {

__global__ void __launch_bounds__(kGemmThreads)
gemm_tiles_kernel(const GemmDesc* __restrict__ descs, const GemmTile* __restrict__ tiles) {
  __shared__ __align__(16) float As[kGemmBK][kGemmBM];
  __shared__ __align__(16) float Bs[kGemmBK][kGemmBN];
  const GemmTile t = tiles[blockIdx.x];
  const GemmDesc d = descs[t.desc];
  const int m0 = t.tm * kGemmBM, n0 = t.tn * kGemmBN;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;

  for (int k0 = 0; k0 < d.K; k0 += kGemmBK) {
    // op(A)[i][l] -> As[l][i]
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int i, l;
      if (d.tA) { l = (tid >> 6) + 4 * q; i = tid & 63; }
      else      { i = (tid >> 4) + 16 * q; l = tid & 15; }
      const int gi = m0 + i, gl = k0 + l;
      float v = 0.f;
      if (gi < d.M && gl < d.K) {
        const int64_t idx = d.tA ? (int64_t)gl * d.lda + gi : (int64_t)gi * d.lda + gl;
        v = load_elem(d.A, idx, d.a_bf16);
      }
      As[l][i] = v;
    }
    // op(B)[l][j] -> Bs[l][j]
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int l, j;
      if (d.tB) { j = (tid >> 4) + 16 * q; l = tid & 15; }
      else      { l = (tid >> 6) + 4 * q; j = tid & 63; }
      const int gj = n0 + j, gl = k0 + l;
      float v = 0.f;
      if (gj < d.N && gl < d.K) {
        const int64_t idx = d.tB ? (int64_t)gj * d.ldb + gl : (int64_t)gl * d.ldb + gj;
        v = load_elem(d.B, idx, d.b_bf16);
      }
      Bs[l][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < kGemmBK; ++l) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[l][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[l][tx * 4]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = m0 + ty * 4 + a;
    if (gi >= d.M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = n0 + tx * 4 + b;
      if (gj >= d.N) continue;
      float v = d.alpha * acc[a][b];
      if (d.beta != 0.f) {
        const int64_t ci = d.tCin ? (int64_t)gj * d.ldcin + gi : (int64_t)gi * d.ldcin + gj;
        v = fmaf(d.beta, d.Cin[ci], v);
      }
      const int64_t co = d.tC ? (int64_t)gj * d.ldc + gi : (int64_t)gi * d.ldc + gj;
      d.C[co] = v;
    }
  }
}

cudaError_t launch_gemm(const GemmDesc* d_desc, const GemmTile* d_tiles, int n_tiles,
                        cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  prof_begin(s);
  gemm_tiles_kernel<<<n_tiles, kGemmThreads, 0, s>>>(d_desc, d_tiles);
  prof_end("gemm_simt", s);
  return cudaGetLastError();
}

}  // namespace csvd
