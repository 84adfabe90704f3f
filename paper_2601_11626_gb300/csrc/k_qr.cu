// Thin QR of the residual R = Q_res B (Lemma 1) by Householder reflections,
// and the product Q_res W for the basis rotation (Cor. 3).
//
// One CTA per item.  R is held column-major (Rt, k x m) so that a column is
// contiguous: the reflector of column j is built from Rt[j][j:m] with a
// block reduction, then every warp applies it to its share of the trailing
// columns (dot product + axpy, coalesced along the column).  Only
// kp = min(k, m - r_t) reflectors are formed and no rank threshold is
// applied: zero columns give tau = 0, so R = Q_res B holds exactly even for
// rank-deficient residuals.
#include "common.cuh"

namespace csvd {

__global__ void __launch_bounds__(512)
householder_qr_kernel(const QRDesc* __restrict__ descs) {
  extern __shared__ __align__(16) float smem[];
  const QRDesc d = descs[blockIdx.x];
  float* v = smem;                 // m floats: current reflector
  float* red = smem + d.m;         // 33 floats
  __shared__ float s_tau, s_beta;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = blockDim.x >> 5;

  for (int j = 0; j < d.kp; ++j) {
    float* col = d.Rt + (int64_t)j * d.ldr;
    float part = 0.f;
    for (int i = j + 1 + tid; i < d.m; i += blockDim.x) part = fmaf(col[i], col[i], part);
    const float tail2 = block_sum(part, red);
    const float x0 = col[j];
    if (tid == 0) {
      if (tail2 == 0.f) {
        s_tau = 0.f;
        s_beta = x0;
      } else {
        const float nrm = sqrtf(fmaf(x0, x0, tail2));
        const float beta = x0 >= 0.f ? -nrm : nrm;
        s_tau = (beta - x0) / beta;
        s_beta = beta;
      }
    }
    __syncthreads();
    const float tau = s_tau, beta = s_beta;
    const float scale = tau != 0.f ? 1.f / (x0 - beta) : 0.f;
    if (tid == 0) v[j] = 1.f;
    for (int i = j + 1 + tid; i < d.m; i += blockDim.x) {
      const float vi = col[i] * scale;
      v[i] = vi;
      col[i] = vi;  // reflector stored below the diagonal
    }
    if (tid == 0) {
      col[j] = beta;
      d.tau[j] = tau;
    }
    __syncthreads();
    if (tau != 0.f) {
      for (int c = j + 1 + wid; c < d.k; c += nw) {
        float* cc = d.Rt + (int64_t)c * d.ldr;
        float w = 0.f;
        for (int i = j + lane; i < d.m; i += 32) w = fmaf(v[i], cc[i], w);
        w = warp_sum(w) * tau;
        for (int i = j + lane; i < d.m; i += 32) cc[i] = fmaf(-w, v[i], cc[i]);
      }
    }
    __syncthreads();
  }
  // upper-triangular factor B (kp x k)
  for (int e = tid; e < d.kp * d.k; e += blockDim.x) {
    const int i = e / d.k, c = e % d.k;
    d.B[(int64_t)i * d.ldb + c] = (c >= i) ? d.Rt[(int64_t)c * d.ldr + i] : 0.f;
  }
}

cudaError_t launch_householder_qr(const QRDesc* d_desc, int n_items, int max_m,
                                  cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const int smem = (max_m + 40) * (int)sizeof(float);
  static std::atomic<int> set_smem{0};
  if (cudaError_t e = ensure_smem(householder_qr_kernel, smem, set_smem)) return e;
  prof_begin(s);
  householder_qr_kernel<<<n_items, 512, smem, s>>>(d_desc);
  prof_end("householder_qr", s);
  return cudaGetLastError();
}

// Zt[j][:] = Q_res * W_bot[:, j] = H_0 H_1 ... H_{kp-1} [W_bot[:, j]; 0].
// One warp per (item, column j); blockIdx.y = item.
__global__ void __launch_bounds__(256)
apply_q_kernel(const ApplyQDesc* __restrict__ descs) {
  const ApplyQDesc d = descs[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= d.ncols) return;
  float* z = d.Zt + (int64_t)j * d.ldz;
  const float* w = d.Wt + (int64_t)j * d.ldw + d.woff;
  for (int i = lane; i < d.m; i += 32) z[i] = (i < d.kp) ? w[i] : 0.f;
  __syncwarp();
  for (int h = d.kp - 1; h >= 0; --h) {
    const float tau = d.tau[h];
    if (tau == 0.f) continue;
    const float* vh = d.Rt + (int64_t)h * d.ldr;
    float acc = 0.f;
    for (int i = h + lane; i < d.m; i += 32) acc = fmaf(i == h ? 1.f : vh[i], z[i], acc);
    acc = warp_sum(acc) * tau;
    for (int i = h + lane; i < d.m; i += 32) z[i] = fmaf(-acc, i == h ? 1.f : vh[i], z[i]);
    __syncwarp();
  }
}

cudaError_t launch_apply_q(const ApplyQDesc* d_desc, int n_items, int max_cols,
                           cudaStream_t s) {
  if (n_items <= 0 || max_cols <= 0) return cudaSuccess;
  dim3 grid((max_cols + 7) / 8, n_items);
  prof_begin(s);
  apply_q_kernel<<<grid, 256, 0, s>>>(d_desc);
  prof_end("apply_q", s);
  return cudaGetLastError();
}

}  // namespace csvd
