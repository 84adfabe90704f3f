// The small core of a merge evaluation, its truncation and the tail
// estimate (Lemma 1, Cor. 3 and Cor. 2), plus the block-energy reduction.
//
// Two core solvers, one CTA per item:
//  * core_jacobi_kernel (plain form): one-sided (Hestenes) Jacobi on the
//    columns of K = [[diag(s), P], [0, B]] (n_r = r_t + kp rows, n_c = r_t + k
//    columns).  Disjoint column pairs of a round-robin schedule are rotated
//    by separate warps; column norms at convergence are the singular values
//    and the normalised columns the left singular vectors.
//    (The mixed form's eigenvalue core is in k_tridiag.cu.)
// The epilogue gives sigma~ = top r_new values, the tail as accumulated
// discarded energy (equal to sum ||A||^2 - sum sigma~^2 in exact arithmetic,
// without its cancellation) and the merge certificate
// tail <= eps^2 ||M_{C u j}||^2 (Alg. 3 step 3(e)).
// The core lives in shared memory when it fits, else in a global workspace.
#include "common.cuh"

namespace csvd {

constexpr int kJacobiMaxSweeps = 40;
__device__ int d_jacobi_cap = kJacobiMaxSweeps;  // lowered only by the failure-path test hook

// ------------------------------------------------------------- energy
__global__ void __launch_bounds__(256)
energy_kernel(const EnergyDesc* __restrict__ descs) {
  __shared__ double red[8];
  const EnergyDesc d = descs[blockIdx.y];
  float s = 0.f, comp = 0.f;  // Kahan-compensated FP32 partial
  // rows strided over the CTAs of this item, columns over the threads
  for (int i = blockIdx.x; i < d.m; i += gridDim.x) {
    for (int c = threadIdx.x; c < d.k; c += blockDim.x) {
      const float a = load_elem(d.A, (int64_t)i * d.ld + c, d.bf16);
      const float y = fmaf(a, a, -comp);
      const float t = s + y;
      comp = (t - s) - y;
      s = t;
    }
  }
  double v = warp_sum_d((double)s - (double)comp);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(d.out, t);
  }
}

cudaError_t jacobi_set_cap(int cap) {
  if (cap < 0) cap = kJacobiMaxSweeps;
  return cudaMemcpyToSymbol(d_jacobi_cap, &cap, sizeof(int));
}

cudaError_t launch_energy(const EnergyDesc* d_desc, int n_items, int max_chunks,
                          cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  dim3 grid(max_chunks < 1 ? 1 : max_chunks, n_items);
  prof_begin(s);
  energy_kernel<<<grid, 256, 0, s>>>(d_desc);
  prof_end("block_energy", s);
  return cudaGetLastError();
}

// Column energies for blocks the tensor-core Gram does not read: a CTA
// takes 32 columns and a slice of the rows (one coalesced 128-byte row
// segment per warp step); squares are summed exactly (FMA for the rounding
// error of the square, two-sum for the addition) and each warp adds its
// FP64 totals into the column's slot.
constexpr int kColRows = 256;  // rows per CTA
__global__ void __launch_bounds__(256)
col_energy_kernel(const EnergyDesc* __restrict__ descs) {
  const EnergyDesc d = descs[blockIdx.z];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int r0 = blockIdx.y * kColRows;
  if (blockIdx.x * 32 >= d.k || r0 >= d.m) return;
  float s = 0.f, comp = 0.f;
  const int r1 = min(d.m, r0 + kColRows);
  if (c < d.k) {
    for (int i = r0 + (threadIdx.x >> 5); i < r1; i += 8) {
      const float x = load_elem(d.A, (int64_t)i * d.ld + c, d.bf16);
      const float p = x * x;
      const float e = fmaf(x, x, -p);
      const float t = s + p;
      const float z = t - s;
      comp += ((s - (t - z)) + (p - z)) + e;
      s = t;
    }
    atomicAdd(d.out + c, (double)s + (double)comp);
  }
}

cudaError_t launch_col_energy(const EnergyDesc* d_desc, int n_items, int max_k, int max_m,
                              cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  dim3 grid((max_k + 31) / 32, (max_m + kColRows - 1) / kColRows, n_items);
  prof_begin(s);
  col_energy_kernel<<<grid, 256, 0, s>>>(d_desc);
  prof_end("col_energy", s);
  return cudaGetLastError();
}

// Residual energies without materialising the residual: for every block
// sum_ij (A - U P)_ij^2 with P = U^T A given (r x k, ld k).  A CTA of 256
// threads takes a 64 x 64 tile of one block (each thread a 4 x 4 patch),
// accumulates U P over r in chunks of 32 staged in shared memory, and sums
// the squares of A - U P exactly (FMA error of the square, two-sum), one
// FP64 atomic per thread group.
__global__ void __launch_bounds__(256)
resid_energy_kernel(const ResidDesc* __restrict__ descs, int r) {
  const ResidDesc d = descs[blockIdx.z];
  const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
  if (row0 >= d.m || col0 >= d.k) return;
  __shared__ float su[64][33];  // U rows x r chunk
  __shared__ float sp[32][64];  // r chunk x P columns
  const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;  // 16 x 16 threads, 4 x 4 each
  float acc[4][4] = {};
  for (int c0 = 0; c0 < r; c0 += 32) {
    for (int e = tid; e < 64 * 32; e += 256) {
      const int i = e >> 5, j = e & 31;
      const int gi = row0 + i, gj = c0 + j;
      su[i][j] = (gi < d.m && gj < r) ? d.U[(int64_t)gi * d.ldu + gj] : 0.f;
    }
    for (int e = tid; e < 32 * 64; e += 256) {
      const int i = e >> 6, j = e & 63;
      const int gi = c0 + i, gj = col0 + j;
      sp[i][j] = (gi < r && gj < d.k) ? d.P[(int64_t)gi * d.ldp + gj] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < 32; ++l) {
      float ua[4], pb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) ua[a] = su[tr * 4 + a][l];
#pragma unroll
      for (int b = 0; b < 4; ++b) pb[b] = sp[l][tc * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(ua[a], pb[b], acc[a][b]);
    }
    __syncthreads();
  }
  float s = 0.f, comp = 0.f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = row0 + tr * 4 + a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = col0 + tc * 4 + b;
      if (gi < d.m && gj < d.k) {
        const float x = d.A[(int64_t)gi * d.lda + gj] - acc[a][b];
        const float p = x * x;
        const float e = fmaf(x, x, -p);
        const float t = s + p;
        const float z = t - s;
        comp += ((s - (t - z)) + (p - z)) + e;
        s = t;
      }
    }
  }
  double v = warp_sum_d((double)s + (double)comp);
  if ((tid & 31) == 0) atomicAdd(d.out, v);
}

cudaError_t launch_resid_energy(const ResidDesc* d_desc, int n_items, int max_m, int max_k, int r,
                                cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  dim3 grid((max_k + 63) / 64, (max_m + 63) / 64, n_items);
  prof_begin(s);
  resid_energy_kernel<<<grid, 256, 0, s>>>(d_desc, r);
  prof_end("resid_energy", s);
  return cudaGetLastError();
}

// ------------------------------------------------------ shared epilogue
// vals[0..nv) non-increasing; writes sigma~, tails and the accept flag.
// Called by warp 0 only; vals_are_sq says whether vals hold sigma^2.
__device__ void core_epilogue(const CoreDesc& d, const float* vals, int nv, bool vals_are_sq) {
  const int lane = threadIdx.x & 31;
  double top = 0.0, disc = 0.0;
  for (int q = lane; q < nv; q += 32) {
    const double x = vals[q];
    const double sq = vals_are_sq ? x : x * x;
    if (q < d.r_new) top += sq; else disc += sq;
    if (q < d.r_new)
      d.sigma_out[q] = vals_are_sq ? sqrtf(fmaxf(vals[q], 0.f)) : vals[q];
  }
  top = warp_sum_d(top);
  disc = warp_sum_d(disc);
  if (lane == 0) {
    const double energy_new = d.scal[0] + d.energy_add[0];
    double tail = d.scal[1] + disc;
    if (tail < 0.0) tail = 0.0;
    double paper = energy_new - top;
    if (paper < 0.0) paper = 0.0;
    d.tail_out[0] = tail;
    if (d.tail_paper_out) d.tail_paper_out[0] = paper;
    if (d.energy_out) d.energy_out[0] = energy_new;
    if (d.accept_out) d.accept_out[0] = (tail <= d.eps * d.eps * energy_new) ? 1 : 0;
  }
}

// --------------------------------------------------------- Jacobi core
__device__ __forceinline__ void rr_pair(int t, int p, int n, int& a, int& b) {
  // t, p < n - 1: one conditional wrap each instead of a division
  if (p == 0) { a = n - 1; b = t; }
  else {
    a = t + p;
    if (a >= n - 1) a -= n - 1;
    b = t - p;
    if (b < 0) b += n - 1;
  }
}

__global__ void __launch_bounds__(1024)
core_jacobi_kernel(const CoreDesc* __restrict__ descs, int* __restrict__ status) {
  extern __shared__ __align__(16) float smem[];
  const CoreDesc d = descs[blockIdx.x];
  const int nr = d.rt + d.kp, nc = d.rt + d.k;
  const int ncp = nc + (nc & 1);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  float* norms = smem;                                  // ncp
  int* order = reinterpret_cast<int*>(smem + ncp);      // ncp
  float* svals = smem + 2 * ncp;                        // ncp
  __shared__ int s_rot;
  const int scratch = ((3 * ncp + 3) / 4) * 4;
  float* K = d.in_smem ? smem + scratch : d.work;
  const int64_t ldk = d.in_smem ? nr : d.ldwork;

  // assemble K column-major
  for (int64_t e = tid; e < (int64_t)ncp * nr; e += blockDim.x) {
    const int c = (int)(e / nr), i = (int)(e % nr);
    float v = 0.f;
    if (c < d.rt) v = (i == c) ? d.sigma[c] : 0.f;
    else if (c < nc) {
      const int cc = c - d.rt;
      if (i < d.rt) {
        v = d.P[(int64_t)i * d.ldp + cc];
        if (d.P2) v += d.P2[(int64_t)i * d.ldp + cc];
      } else {
        v = d.B[(int64_t)(i - d.rt) * d.ldb + cc];
      }
    }
    K[(int64_t)c * ldk + i] = v;
  }
  __syncthreads();

  const float tol = 4.f * 5.9604645e-8f * sqrtf((float)(nr > 1 ? nr : 1));
  bool converged = (ncp < 2);
  const int cap = d_jacobi_cap;
  for (int sweep = 0; sweep < cap && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int t = 0; t < ncp - 1; ++t) {
      for (int p = wid; p < ncp / 2; p += nw) {
        int a, b;
        rr_pair(t, p, ncp, a, b);
        if (a >= nc || b >= nc) continue;
        float* x = K + (int64_t)a * ldk;
        float* y = K + (int64_t)b * ldk;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int i = lane; i < nr; i += 32) {
          const float xi = x[i], yi = y[i];
          al = fmaf(xi, xi, al);
          be = fmaf(yi, yi, be);
          ga = fmaf(xi, yi, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        const float scale = sqrtf(al) * sqrtf(be);
        if (!(scale > 1e-36f) || !(fabsf(ga) > tol * scale)) continue;
        const float zeta = (be - al) / (2.f * ga);
        float tt;
        if (fabsf(zeta) > 1e7f) tt = 0.5f / zeta;
        else tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
        const float cs = __frsqrt_rn(fmaf(tt, tt, 1.f));  // correctly rounded: c^2 + s^2 = 1 to rounding
        const float sn = cs * tt;
        for (int i = lane; i < nr; i += 32) {
          const float xi = x[i], yi = y[i];
          x[i] = cs * xi - sn * yi;
          y[i] = fmaf(sn, xi, cs * yi);
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    converged = (s_rot == 0);
    __syncthreads();
  }
  if (!converged && tid == 0) atomicOr(status, kStatusJacobiCap);

  // column norms = singular values, sorted non-increasing (ties: index)
  for (int c = wid; c < nc; c += nw) {
    const float* x = K + (int64_t)c * ldk;
    float s = 0.f;
    for (int i = lane; i < nr; i += 32) s = fmaf(x[i], x[i], s);
    s = warp_sum(s);
    if (lane == 0) norms[c] = sqrtf(s);
  }
  __syncthreads();
  for (int c = tid; c < nc; c += blockDim.x) {
    const float v = norms[c];
    int rank = 0;
    for (int e = 0; e < nc; ++e) {
      const float u = norms[e];
      rank += (u > v) || (u == v && e < c);
    }
    order[rank] = c;
  }
  __syncthreads();
  for (int q = tid; q < nc; q += blockDim.x) svals[q] = norms[order[q]];
  __syncthreads();
  if (wid == 0) core_epilogue(d, svals, nc, false);
  if (d.Wt) {
    for (int64_t e = tid; e < (int64_t)d.r_new * nr; e += blockDim.x) {
      const int j = (int)(e / nr), i = (int)(e % nr);
      const float s = svals[j];
      const float v = K[(int64_t)order[j] * ldk + i];
      d.Wt[(int64_t)j * d.ldw + i] = s > 0.f ? v / s : 0.f;
    }
  }
}

int jacobi_scratch_floats(int nc) {
  const int ncp = nc + (nc & 1);
  return ((3 * ncp + 3) / 4) * 4;
}

cudaError_t launch_core_jacobi(const CoreDesc* d_desc, int n_items, int smem_bytes,
                               int* d_status, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  static std::atomic<int> set_smem{0};
  if (cudaError_t e = ensure_smem(core_jacobi_kernel, smem_bytes, set_smem)) return e;
  prof_begin(s);
  core_jacobi_kernel<<<n_items, 1024, smem_bytes, s>>>(d_desc, d_status);
  prof_end("core_jacobi", s);
  return cudaGetLastError();
}

// ------------------------------------------------ basis re-orthonormalisation
// D = U^T U - I (r x r) with f32 inputs and FP64 products and sums; one
// warp per entry of the upper triangle, mirrored.  Used for one
// Newton-Schulz step U <- U - U D / 2 after a basis commit, which removes
// the orthogonality drift that Jacobi's convergence threshold leaves.
__global__ void __launch_bounds__(256)
gram_dev_kernel(const float* __restrict__ U, int64_t ldu, int m, int r, float* __restrict__ D) {
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= r * r) return;
  const int i = e / r, j = e % r;
  if (j < i) return;
  double acc = 0.0;
  for (int l = lane; l < m; l += 32)
    acc += (double)U[(int64_t)l * ldu + i] * (double)U[(int64_t)l * ldu + j];
  acc = warp_sum_d(acc);
  if (lane == 0) {
    const float v = (float)(acc - (i == j ? 1.0 : 0.0));
    D[(int64_t)i * r + j] = v;
    D[(int64_t)j * r + i] = v;
  }
}

cudaError_t launch_gram_dev(const float* U, int64_t ldu, int m, int r, float* D, cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  const int warps = r * r;
  prof_begin(s);
  gram_dev_kernel<<<(warps + 7) / 8, 256, 0, s>>>(U, ldu, m, r, D);
  prof_end("gram_dev", s);
  return cudaGetLastError();
}

// ------------------------------------------------------ small helpers
__global__ void state_commit_kernel(const float* sigma_new, int r_new, float* sigma,
                                    const double* energy_new, const double* tail_new,
                                    double* scal) {
  for (int i = threadIdx.x; i < r_new; i += blockDim.x) sigma[i] = sigma_new[i];
  if (threadIdx.x == 0) {
    scal[0] = energy_new[0];
    scal[1] = tail_new[0];
  }
}

cudaError_t launch_state_commit(const float* sigma_new, int r_new, float* sigma,
                                const double* energy_new, const double* tail_new,
                                double* scal, cudaStream_t s) {
  prof_begin(s);
  state_commit_kernel<<<1, 256, 0, s>>>(sigma_new, r_new, sigma, energy_new, tail_new, scal);
  prof_end("state_commit", s);
  return cudaGetLastError();
}

__global__ void add_inplace_kernel(float* dst, const float* src, int rows, int cols,
                                   int64_t ld_dst, int64_t ld_src) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    dst[i * ld_dst + j] += src[i * ld_src + j];
  }
}

cudaError_t launch_add_inplace(float* dst, const float* src, int rows, int cols,
                               int64_t ld_dst, int64_t ld_src, cudaStream_t s) {
  const int64_t total = (int64_t)rows * cols;
  if (total <= 0) return cudaSuccess;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  prof_begin(s);
  add_inplace_kernel<<<blocks, 256, 0, s>>>(dst, src, rows, cols, ld_dst, ld_src);
  prof_end("add_inplace", s);
  return cudaGetLastError();
}

// Column scaling of an m x r row-major factor: out[i][j] = U[i][j] * s[j]
// (U~ = U diag(s)), or with `inverse` U[i][j] / s[j] (0 where s[j] == 0).
__global__ void scale_cols_kernel(const float* __restrict__ U, int64_t ldu, int m, int r,
                                  const float* __restrict__ s, int inverse,
                                  float* __restrict__ out, int64_t ld_out) {
  const int64_t total = (int64_t)m * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    const float sj = s[j], u = U[(int64_t)i * ldu + j];
    out[(int64_t)i * ld_out + j] = inverse ? (sj > 0.f ? u / sj : 0.f) : u * sj;
  }
}

cudaError_t launch_scale_cols(const float* U, int64_t ldu, int m, int r, const float* s,
                              int inverse, float* out, int64_t ld_out, cudaStream_t st) {
  const int64_t total = (int64_t)m * r;
  if (total <= 0) return cudaSuccess;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  prof_begin(st);
  scale_cols_kernel<<<blocks, 256, 0, st>>>(U, ldu, m, r, s, inverse, out, ld_out);
  prof_end("scale_cols", st);
  return cudaGetLastError();
}

}  // namespace csvd
