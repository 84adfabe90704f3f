// Eigenvalue core of the mixed merge evaluation.
//
// For an item with state (s_1..s_rt) and block A (k columns) the Gram of the
// core K = [[diag(s), P], [0, B]] is
//     G = K^T K = [[diag(s^2), diag(s) P], [P^T diag(s), A^T A]]   (n = rt + k),
// whose nonzero eigenvalues are those of K K^T = S_{t+1} (Lemma 1), i.e. the
// squared singular values of the core.  Only the top r_new of them are
// needed: sigma~_j = sqrt(lambda_j) (Cor. 3), and the tail follows from the
// trace, sum_{j > r_new} lambda_j = tr(G) - sum_{j <= r_new} lambda_j.
//
// One CTA per item:
//  1. G is assembled in packed lower-triangular, column-major storage.  It
//     lives in shared memory when n(n+1)/2 floats fit; otherwise in a global
//     workspace until the trailing matrix fits, then it migrates on-chip.
//  2. Householder tridiagonalisation, G <- H G H with H = I - tau v v^T.  The
//     rank-2 update of step j is applied lazily, fused with the symmetric
//     matrix-vector product of step j+1 in one pass over 32 x 32 tiles of the
//     trailing triangle (one load, one store, four FMAs per element); tile
//     column sums use a 31-shuffle transpose reduction.
//  3. Multisection bisection on Sturm counts of the tridiagonal matrix for
//     the top r_new eigenvalues (g threads per eigenvalue, each iteration
//     shrinks the interval (g + 1)-fold).
//  4. FP64 epilogue: sigma~, tail = discarded_state + tr(T) - sum top, the
//     subtraction form sum ||A||^2 - sum sigma~^2, and the accept flag.
#include "common.cuh"

namespace csvd {
namespace {

constexpr int kTriThreads = 512;
constexpr int kTriWarps = kTriThreads / 32;
constexpr int kBisectMax = 64;

__device__ __forceinline__ int64_t col_off(int l, int N) {
  return (int64_t)l * N - ((int64_t)l * (l - 1)) / 2;
}

// Packed lower matrix view: holds global rows/cols >= g0, N = n - g0.
struct Packed {
  float* p;
  int g0, N;
  __device__ __forceinline__ float* at(int i, int l) const {  // global indices, i >= l >= g0
    const int li = i - g0, ll = l - g0;
    return p + col_off(ll, N) + (li - ll);
  }
};

__device__ __forceinline__ int sturm_count(const float* dv, const float* e2, int n, float x,
                                           float pivmin) {
  float q = dv[0] - x;
  int cnt = q < 0.f;
  for (int i = 1; i < n; ++i) {
    if (fabsf(q) < pivmin) q = -pivmin;
    q = (dv[i] - x) - e2[i - 1] / q;
    cnt += q < 0.f;
  }
  return cnt;
}

}  // namespace

// Largest trailing size kept in shared memory for a given dynamic size.
__host__ __device__ int tridiag_smem_cap(int smem_bytes, int n_max) {
  const int scratch = 6 * n_max + 96;
  long avail = (long)smem_bytes / 4 - scratch;
  if (avail <= 0) return 0;
  int t = (int)((sqrt(8.0 * (double)avail + 1.0) - 1.0) / 2.0);
  while ((long)t * (t + 1) / 2 > avail) --t;
  return t;
}

__global__ void __launch_bounds__(kTriThreads)
core_tridiag_kernel(const CoreDesc* __restrict__ descs, int smem_bytes, int n_max,
                    int* __restrict__ status) {
  extern __shared__ __align__(16) float smem[];
  const CoreDesc d = descs[blockIdx.x];
  const int n = d.rt + d.k;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* dv = smem;              // n_max: diagonal of T
  float* ev = dv + n_max;        // n_max: off-diagonal e[j] couples j, j+1
  float* vcur = ev + n_max;      // n_max: reflector of the current step
  float* wcur = vcur + n_max;    // n_max: p then w of the current step
  float* vprev = wcur + n_max;   // n_max: reflector of the previous step
  float* wprev = vprev + n_max;  // n_max
  float* red = wprev + n_max;    // 96
  float* Ms = red + 96;          // packed on-chip matrix
  const int cap = tridiag_smem_cap(smem_bytes, n_max);
  __shared__ float s_tau2, s_v0;
  __shared__ double s_trace;

  Packed M;
  const bool start_smem = n <= cap;
  M.p = start_smem ? Ms : d.work;
  M.g0 = 0;
  M.N = n;

  // 1. assemble the Gram core (packed lower, column-major)
  for (int l = wid; l < n; l += kTriWarps) {
    for (int i = l + lane; i < n; i += 32) {
      float v;
      if (l < d.rt) {
        if (i < d.rt) v = (i == l) ? d.sigma[i] * d.sigma[i] : 0.f;
        else v = d.sigma[l] * d.P[(int64_t)l * d.ldp + (i - d.rt)];
      } else {
        v = d.Gaa[(int64_t)(l - d.rt) * d.ldb + (i - d.rt)];  // upper part of A^T A
      }
      *M.at(i, l) = v;
    }
  }
  __syncthreads();

  // 2. tridiagonalisation with a lazily applied rank-2 update
  bool have_prev = false;
  for (int j = 0; j + 2 < n; ++j) {
    const int t = n - j - 1;  // trailing size of this step
    if (M.p != Ms && n - j <= cap) {
      // migrate rows/cols >= j on-chip
      Packed S{Ms, j, n - j};
      for (int l = j + wid; l < n; l += kTriWarps)
        for (int i = l + lane; i < n; i += 32) *S.at(i, l) = *M.at(i, l);
      __syncthreads();
      M = S;
    }
    // (a) bring column j up to date with the pending update of step j-1
    if (have_prev) {
      const float vp0 = vprev[0], wp0 = wprev[0];
      for (int i = j + tid; i < n; i += kTriThreads) {
        float* g = M.at(i, j);
        *g = fmaf(-vprev[i - j], wp0, fmaf(-wprev[i - j], vp0, *g));
      }
    }
    __syncthreads();
    // reflector from x = G[j+1:, j]
    float part = 0.f;
    for (int i = j + 2 + tid; i < n; i += kTriThreads) {
      const float x = *M.at(i, j);
      part = fmaf(x, x, part);
    }
    const float tail2 = block_sum(part, red);
    if (tid == 0) {
      const float x0 = *M.at(j + 1, j);
      dv[j] = *M.at(j, j);
      if (tail2 == 0.f) {
        ev[j] = x0;
        s_tau2 = 0.f;
        s_v0 = 0.f;
      } else {
        const float nrm = sqrtf(fmaf(x0, x0, tail2));
        const float beta = x0 >= 0.f ? -nrm : nrm;
        const float v0 = x0 - beta;
        ev[j] = beta;
        s_v0 = v0;
        s_tau2 = 2.f / fmaf(v0, v0, tail2);
      }
    }
    __syncthreads();
    const float tau2 = s_tau2;
    for (int r = tid; r < t; r += kTriThreads) {
      vcur[r] = (tau2 == 0.f) ? 0.f : (r == 0 ? s_v0 : *M.at(j + 1 + r, j));
      wcur[r] = 0.f;
    }
    __syncthreads();
    // (b) fused pass over the trailing triangle (rows/cols >= j+1, local r, c):
    //     G -= vprev wprev^T + wprev vprev^T (pending), then p += G v
    {
      const int T = (t + 31) >> 5;
      int idx = 0;
      for (int b = 0; b < T; ++b) {
        for (int a = b; a < T; ++a, ++idx) {
          if ((idx % kTriWarps) != wid) continue;
          const int r = 32 * a + lane;
          const bool rv = r < t;
          const float vr = rv ? vcur[r] : 0.f;
          const float vpr = (rv && have_prev) ? vprev[r + 1] : 0.f;
          const float wpr = (rv && have_prev) ? wprev[r + 1] : 0.f;
          float rowacc = 0.f;
          float cp[32];
#pragma unroll
          for (int cc = 0; cc < 32; ++cc) {
            const int c = 32 * b + cc;
            float val = 0.f;
            const bool ok = rv && c < t && c <= r;
            if (ok) {
              float* g = M.at(j + 1 + r, j + 1 + c);
              val = *g;
              if (have_prev) {
                val = fmaf(-vpr, wprev[c + 1], fmaf(-wpr, vprev[c + 1], val));
                *g = val;
              }
            }
            const float vc = (c < t) ? vcur[c] : 0.f;
            rowacc = fmaf(val, vc, rowacc);
            cp[cc] = (ok && r > c) ? val * vr : 0.f;
          }
          // transpose reduction: lane L ends with the sum of cp[L] over lanes
#pragma unroll
          for (int sh = 16; sh >= 1; sh >>= 1) {
#pragma unroll
            for (int i = 0; i < sh; ++i) {
              const bool up = (lane & sh) != 0;
              const float send = up ? cp[i] : cp[i + sh];
              const float keep = up ? cp[i + sh] : cp[i];
              cp[i] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
            }
          }
          if (rv) atomicAdd(&wcur[r], rowacc);
          const int c = 32 * b + lane;
          if (c < t) atomicAdd(&wcur[c], cp[0]);
        }
      }
    }
    __syncthreads();
    // w = tau2 p - (tau2^2 / 2)(p^T v) v
    float pp = 0.f;
    for (int r = tid; r < t; r += kTriThreads) pp = fmaf(wcur[r], vcur[r], pp);
    const float kk = 0.5f * tau2 * tau2 * block_sum(pp, red);
    for (int r = tid; r < t; r += kTriThreads) wcur[r] = fmaf(tau2, wcur[r], -kk * vcur[r]);
    __syncthreads();
    // the current step becomes the pending update
    float* tv = vprev; vprev = vcur; vcur = tv;
    float* tw = wprev; wprev = wcur; wcur = tw;
    have_prev = true;
  }
  // last 2 x 2 (or 1 x 1) block, with the pending update applied
  if (tid == 0) {
    if (n >= 2) {
      const int j = n - 2;
      float a = *M.at(j, j), b = *M.at(j + 1, j), c = *M.at(j + 1, j + 1);
      if (have_prev) {  // pending step n-3: its local index 0 is row n-2, 1 is row n-1
        a = fmaf(-2.f * vprev[0], wprev[0], a);
        b = fmaf(-vprev[1], wprev[0], fmaf(-wprev[1], vprev[0], b));
        c = fmaf(-2.f * vprev[1], wprev[1], c);
      }
      dv[j] = a;
      ev[j] = b;
      dv[j + 1] = c;
    } else {
      dv[0] = *M.at(0, 0);
    }
    ev[n - 1] = 0.f;
  }
  __syncthreads();

  // 3. Gershgorin interval, trace, squared off-diagonals
  float lo = 3.0e38f, hi = -3.0e38f, emax = 0.f;
  double tr = 0.0;
  for (int i = tid; i < n; i += kTriThreads) {
    const float el = i > 0 ? fabsf(ev[i - 1]) : 0.f;
    const float er = i + 1 < n ? fabsf(ev[i]) : 0.f;
    lo = fminf(lo, dv[i] - el - er);
    hi = fmaxf(hi, dv[i] + el + er);
    emax = fmaxf(emax, er * er);
    tr += (double)dv[i];
  }
  __shared__ float s_lo[kTriWarps], s_hi[kTriWarps], s_em[kTriWarps];
  __shared__ double s_tr[kTriWarps];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
  }
  if (lane == 0) { s_lo[wid] = lo; s_hi[wid] = hi; s_em[wid] = emax; s_tr[wid] = tr; }
  __syncthreads();
  float glo = s_lo[0], ghi = s_hi[0], gem = s_em[0];
  double gtr = s_tr[0];
  for (int w = 1; w < kTriWarps; ++w) {
    glo = fminf(glo, s_lo[w]);
    ghi = fmaxf(ghi, s_hi[w]);
    gem = fmaxf(gem, s_em[w]);
    gtr += s_tr[w];
  }
  float* e2 = vcur;  // reuse
  float* lam = wcur;
  for (int i = tid; i < n; i += kTriThreads) e2[i] = (i + 1 < n) ? ev[i] * ev[i] : 0.f;
  if (tid == 0) s_trace = gtr;
  __syncthreads();

  // 4. multisection bisection for the top r_new eigenvalues
  const float gnorm = fmaxf(fabsf(glo), fabsf(ghi));
  const float pivmin = 1.0e-30f * fmaxf(1.f, gem);
  const float atol = 2.4e-7f * gnorm + 1e-30f;
  const int rq = d.r_new;
  int g = 1;
  while (g < 16 && g * 2 * rq <= kTriThreads) g *= 2;
  const int ngroups = kTriThreads / g;
  const int grp = tid / g, sub = tid % g;
  int capped = 0;
  for (int q0 = 0; q0 < rq; q0 += ngroups) {  // uniform trip count across the block
    const int q = q0 + grp;
    const bool active = q < rq;
    const int target = n - 1 - q;  // ascending index of the q-th largest
    float a = glo, b = ghi;
    bool stuck = false;
    const unsigned shift = (unsigned)((lane / g) * g);
    const unsigned gmask = (g == 32) ? 0xffffffffu : (((1u << g) - 1u) << shift);
    int it = 0;
    for (; it < kBisectMax; ++it) {
      // every lane of the warp runs the same number of iterations
      const bool done = !active || stuck || !((b - a) > atol);
      if (__all_sync(0xffffffffu, done)) break;
      const float step = (b - a) / (float)(g + 1);
      const float x = a + step * (float)(sub + 1);
      bool above = false;
      if (!done) above = (x > a && x < b) ? (sturm_count(dv, e2, n, x, pivmin) > target) : (x >= b);
      const unsigned bal = (__ballot_sync(0xffffffffu, above) & gmask) >> shift;
      if (!done) {
        // the first point whose count exceeds target bounds the eigenvalue from above
        const int s = bal ? __ffs(bal) - 1 : g;
        const float na = (s == 0) ? a : a + step * (float)s;
        const float nb = (s == g) ? b : a + step * (float)(s + 1);
        if (!(nb < b || na > a)) stuck = true;  // representable limit reached
        a = na;
        b = nb;
      }
    }
    if (active && it == kBisectMax) capped = 1;
    if (active && sub == 0) lam[q] = 0.5f * (a + b);
  }
  if (capped) atomicOr(status, kStatusBisectCap);
  __syncthreads();

  // 5. FP64 epilogue (warp 0)
  if (wid == 0) {
    double top = 0.0;
    for (int q = lane; q < rq; q += 32) {
      const double x = lam[q];
      top += x;
      d.sigma_out[q] = sqrtf(fmaxf(lam[q], 0.f));
    }
    top = warp_sum_d(top);
    if (lane == 0) {
      const double energy_new = d.scal[0] + d.energy_add[0];
      double tail = d.scal[1] + (s_trace - top);
      if (tail < 0.0) tail = 0.0;
      double paper = energy_new - top;
      if (paper < 0.0) paper = 0.0;
      d.tail_out[0] = tail;
      if (d.tail_paper_out) d.tail_paper_out[0] = paper;
      if (d.energy_out) d.energy_out[0] = energy_new;
      if (d.accept_out) d.accept_out[0] = (tail <= d.eps * d.eps * energy_new) ? 1 : 0;
    }
  }
}

int tridiag_work_floats(int n, int cap) {
  return n <= cap ? 0 : (int)((int64_t)n * (n + 1) / 2);
}

cudaError_t launch_core_tridiag(const CoreDesc* d_desc, int n_items, int smem_bytes, int n_max,
                                int* d_status, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  if (smem_bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(core_tridiag_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
  }
  prof_begin(s);
  core_tridiag_kernel<<<n_items, kTriThreads, smem_bytes, s>>>(d_desc, smem_bytes, n_max,
                                                               d_status);
  prof_end("core_tridiag", s);
  return cudaGetLastError();
}

}  // namespace csvd
