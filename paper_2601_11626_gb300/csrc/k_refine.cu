// FP64 re-solve of the mixed form's eigen core for merge evaluations whose
// tail is too small for FP32 eigenvalues to resolve.
//
// The FP32 core (core_tridiag) gives each top eigenvalue of the Gram
//     G = [[diag(s^2), diag(s) P], [P^T diag(s), A^T A]]          (Lemma 1)
// to a few units of FP32 rounding of ||G||, so the tail
//     E~^2 = discarded + tr(T) - sum_{j <= r_new} lambda_j               (Cor. 2)
// carries an absolute error of a few u ||M||^2.  When the estimate lies
// below kRefineFrac of the merged energy, that error can exceed 1e-4 of the
// tail, and the core epilogue marks the item.  This kernel then rebuilds G
// in FP64 from the same inputs (the FP32 products P and A^T A, the exact
// column energies on the diagonal), tridiagonalises it by Householder
// reflections in FP64 and takes the top eigenvalues by FP64 bisection; the
// FP32 results of the item are overwritten.  FP64 runs at 1/64 of the FP32
// rate on this GPU, so only the marked items pay for it.
//
// Persistent CTAs (one per workspace slot of n_max^2 doubles) take items from
// an atomic counter and skip the unmarked ones.  The symmetric matrix is
// kept as its lower triangle inside a full row-major n x n slot.
#include "common.cuh"

namespace csvd {
namespace {

constexpr int kThreads = 256;
constexpr int kBisect64 = 128;
__device__ int d_bisect64_cap = kBisect64;  // lowered only by the failure-path test hook

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum_d(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// Element (r, c), r >= c, of G in FP64.
__device__ __forceinline__ double gram64(const CoreDesc& d, int r, int c) {
  if (c < d.rt) {
    if (r < d.rt) return r == c ? (double)d.sigma[r] * (double)d.sigma[r] : 0.0;
    return (double)d.sigma[c] * (double)d.P[(int64_t)c * d.ldp + (r - d.rt)];
  }
  if (r == c && d.colE) return d.colE[r - d.rt];
  return (double)d.Gaa[(int64_t)(c - d.rt) * d.ldb + (r - d.rt)];
}

__device__ int sturm64(const double* dv, const double* e2, int n, double x, double pivmin) {
  double q = dv[0] - x;
  int cnt = q < 0.0;
  for (int i = 1; i < n; ++i) {
    if (fabs(q) < pivmin) q = -pivmin;
    q = (dv[i] - x) - e2[i - 1] / q;
    cnt += q < 0.0;
  }
  return cnt;
}

__global__ void __launch_bounds__(kThreads)
core_refine64_kernel(const CoreDesc* __restrict__ d0, int n0, const CoreDesc* __restrict__ d1,
                     int n1, const CoreDesc* __restrict__ d2, int n2, double* __restrict__ work,
                     int n_max, int* __restrict__ counter, int* __restrict__ status) {
  extern __shared__ __align__(16) double vsm[];
  double* v = vsm;             // n_max: reflector (rows s+1 ..)
  double* p = v + n_max;       // n_max: G v, then w
  double* dv = p + n_max;      // n_max: diagonal of T
  double* ev = dv + n_max;     // n_max: off-diagonal of T
  double* red = ev + n_max;    // 8 + 8
  __shared__ int s_item;
  const int tid = threadIdx.x;
  double* G = work + (int64_t)blockIdx.x * n_max * n_max;
  const int total = n0 + n1 + n2;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= total) break;
    const CoreDesc& d = item < n0 ? d0[item] : item < n0 + n1 ? d1[item - n0] : d2[item - n0 - n1];
    if (d.refine == nullptr || *d.refine == 0) continue;
    const int n = d.rt + d.k;
    if (n > n_max) {
      if (tid == 0) atomicOr(status, kStatusBadShape);
      continue;
    }
    // 1. lower triangle of G in FP64
    for (int64_t idx = tid; idx < (int64_t)n * n; idx += kThreads) {
      const int r = (int)(idx / n), c = (int)(idx % n);
      if (c <= r) G[idx] = gram64(d, r, c);
    }
    __syncthreads();
    // 2. Householder tridiagonalisation, G <- H G H on the trailing block
    for (int s = 0; s + 2 < n; ++s) {
      double part = 0.0;
      for (int i = s + 2 + tid; i < n; i += kThreads) {
        const double x = G[(int64_t)i * n + s];
        part = fma(x, x, part);
      }
      const double tail2 = block_sum_d(part, red);
      const double x0 = G[(int64_t)(s + 1) * n + s];
      if (tail2 == 0.0) {  // column already reduced
        if (tid == 0) { dv[s] = G[(int64_t)s * n + s]; ev[s] = x0; }
        __syncthreads();
        continue;
      }
      const double nrm = sqrt(fma(x0, x0, tail2));
      const double beta = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - beta;
      const double tau = 2.0 / fma(v0, v0, tail2);
      for (int i = s + 1 + tid; i < n; i += kThreads) v[i] = i == s + 1 ? v0 : G[(int64_t)i * n + s];
      if (tid == 0) { dv[s] = G[(int64_t)s * n + s]; ev[s] = beta; }
      __syncthreads();
      // p = tau G v over the trailing block (lower triangle: row part and column part)
      double pv = 0.0;
      for (int i = s + 1 + tid; i < n; i += kThreads) {
        const double* gi = G + (int64_t)i * n;
        double acc = 0.0;
        for (int j = s + 1; j <= i; ++j) acc = fma(gi[j], v[j], acc);
        for (int j = i + 1; j < n; ++j) acc = fma(G[(int64_t)j * n + i], v[j], acc);
        acc *= tau;
        p[i] = acc;
        pv = fma(acc, v[i], pv);
      }
      const double kk = 0.5 * tau * block_sum_d(pv, red);
      for (int i = s + 1 + tid; i < n; i += kThreads) p[i] = fma(-kk, v[i], p[i]);  // w
      __syncthreads();
      // G -= v w^T + w v^T (lower triangle of the trailing block)
      const int nt = n - s - 1;
      for (int64_t idx = tid; idx < (int64_t)nt * nt; idx += kThreads) {
        const int i = s + 1 + (int)(idx / nt), j = s + 1 + (int)(idx % nt);
        if (j <= i) {
          double* g = G + (int64_t)i * n + j;
          *g = fma(-v[i], p[j], fma(-p[i], v[j], *g));
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (n >= 2) {
        dv[n - 2] = G[(int64_t)(n - 2) * n + n - 2];
        ev[n - 2] = G[(int64_t)(n - 1) * n + n - 2];
        dv[n - 1] = G[(int64_t)(n - 1) * n + n - 1];
      } else {
        dv[0] = G[0];
      }
      ev[n - 1] = 0.0;
    }
    __syncthreads();
    // 3. Gershgorin interval and trace; squared off-diagonals into v
    double lo = 1e300, hi = -1e300, tr = 0.0, emax = 0.0;
    for (int i = tid; i < n; i += kThreads) {
      const double el = i > 0 ? fabs(ev[i - 1]) : 0.0, er = i + 1 < n ? fabs(ev[i]) : 0.0;
      lo = fmin(lo, dv[i] - el - er);
      hi = fmax(hi, dv[i] + el + er);
      tr += dv[i];
      emax = fmax(emax, er * er);
      v[i] = (i + 1 < n) ? ev[i] * ev[i] : 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    __shared__ double s_lo[kThreads / 32], s_hi[kThreads / 32], s_em[kThreads / 32];
    if ((tid & 31) == 0) { s_lo[tid >> 5] = lo; s_hi[tid >> 5] = hi; s_em[tid >> 5] = emax; }
    const double trace = block_sum_d(tr, red);
    double glo = s_lo[0], ghi = s_hi[0], gem = s_em[0];
    for (int w = 1; w < kThreads / 32; ++w) {
      glo = fmin(glo, s_lo[w]);
      ghi = fmax(ghi, s_hi[w]);
      gem = fmax(gem, s_em[w]);
    }
    // 4. bisection for the top r_new eigenvalues (one thread each)
    const double gnorm = fmax(fabs(glo), fabs(ghi));
    const double pivmin = 1e-290 * fmax(1.0, gem);
    const double atol = 1e-15 * gnorm + 1e-300;
    int capped = 0;
    double top = 0.0;
    for (int q = tid; q < d.r_new; q += kThreads) {
      double a = glo, b = ghi;
      int it = 0;
      const int cap = d_bisect64_cap;
      for (; it < cap; ++it) {
        if (!(b - a > fmax(atol, 4e-16 * fmax(fabs(a), fabs(b))))) break;
        const double x = 0.5 * (a + b);
        if (!(x > a && x < b)) break;
        if (sturm64(dv, v, n, x, pivmin) > n - 1 - q) b = x;
        else a = x;
      }
      if (it == cap) capped = 1;
      const double lam = 0.5 * (a + b);
      p[q] = lam;
      top += lam;
    }
    if (capped) atomicOr(status, kStatusBisectCap);
    top = block_sum_d(top, red);
    // 5. epilogue: overwrite the FP32 results
    for (int q = tid; q < d.r_new; q += kThreads) d.sigma_out[q] = (float)sqrt(fmax(p[q], 0.0));
    if (tid == 0) {
      double ea = 0.0;
      if (d.energy_add) ea = d.energy_add[0];
      else
        for (int c = 0; c < d.k; ++c) ea += d.colE[c];
      const double energy_new = d.scal[0] + ea;
      double tail = d.scal[1] + (trace - top);
      if (tail < 0.0) tail = 0.0;
      double paper = energy_new - top;
      if (paper < 0.0) paper = 0.0;
      d.tail_out[0] = tail;
      if (d.tail_paper_out) d.tail_paper_out[0] = paper;
      if (d.energy_out) d.energy_out[0] = energy_new;
      if (d.accept_out) d.accept_out[0] = (tail <= d.eps * d.eps * energy_new) ? 1 : 0;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t refine64_set_bisect_cap(int cap) {
  if (cap < 0) cap = kBisect64;
  return cudaMemcpyToSymbol(d_bisect64_cap, &cap, sizeof(int));
}

size_t refine64_smem_bytes(int n_max) { return sizeof(double) * (4 * (size_t)n_max + 16); }

cudaError_t launch_core_refine64(const CoreDesc* d0, int n0, const CoreDesc* d1, int n1,
                                 const CoreDesc* d2, int n2, double* work, int slots, int n_max,
                                 int* d_counter, int* d_status, cudaStream_t s) {
  if (n0 + n1 + n2 <= 0 || slots <= 0) return cudaSuccess;
  const size_t smem = refine64_smem_bytes(n_max);
  static std::atomic<int> set_smem{0};
  if (cudaError_t e = ensure_smem(core_refine64_kernel, (int)smem, set_smem)) return e;
  prof_begin(s);
  core_refine64_kernel<<<slots, kThreads, smem, s>>>(d0, n0, d1, n1, d2, n2, work, n_max,
                                                     d_counter, d_status);
  prof_end("core_refine64", s);
  return cudaGetLastError();
}

}  // namespace csvd
