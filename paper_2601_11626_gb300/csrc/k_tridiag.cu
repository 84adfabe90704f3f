// Eigenvalue core of the mixed merge evaluation.
//
// For an item with state (s_1..s_rt) and block A (k columns) the Gram of the
// core K = [[diag(s), P], [0, B]] is
//     G = K^T K = [[diag(s^2), diag(s) P], [P^T diag(s), A^T A]]   (n = rt + k),
// whose nonzero eigenvalues are those of K K^T = S_{t+1} (Lemma 1), i.e. the
// squared singular values of the core.  Only the top r_new of them are
// needed: sigma~_j = sqrt(lambda_j) (Cor. 3), and the tail follows from the
// trace, sum_{j > r_new} lambda_j = tr(T) - sum_{j <= r_new} lambda_j.
//
// One CTA per item:
//  1. G is assembled as 32 x 32 tiles of its lower tile triangle, each tile
//     contiguous (4 KB, column-major inside); diagonal tiles hold both
//     halves.  The tiles live in shared memory when they fit; otherwise in a
//     global workspace until the trailing tiles fit, then they move on-chip.
//  2. Householder tridiagonalisation, G <- H G H, H = I - tau v v^T.  The
//     rank-2 update of step j is applied lazily, fused with the symmetric
//     matrix-vector product of step j+1 in one pass over the trailing tiles
//     (one load, one store, four FMAs per element).  All vectors are indexed
//     by global row and vanish outside the trailing range, so boundary tiles
//     need no masks.  Column sums of off-diagonal tiles accumulate across a
//     tile column and are reduced once per column (31-shuffle transpose).
//  3. Multisection bisection on Sturm counts of the tridiagonal matrix for
//     the top r_new eigenvalues (g threads per eigenvalue, the interval
//     shrinks (g + 1)-fold per iteration).
//  4. FP64 epilogue: sigma~, tail = discarded_state + tr(T) - sum top, the
//     subtraction form sum ||A||^2 - sum sigma~^2, and the accept flag; the
//     block energy ||A||^2 is the trace of A^T A unless given.
#include "common.cuh"

namespace csvd {
namespace {

constexpr int kTriThreads = 512;
constexpr int kTriWarps = kTriThreads / 32;
constexpr int kBisectMax = 64;
constexpr int kTile = 32;
constexpr int kTileFloats = kTile * kTile;

// Lower tile triangle of a T x T tile grid whose first tile row/column is a0.
struct Tiles {
  float* p;
  int a0, T;  // tile rows held: global tile rows a0 .. a0+T-1
  __device__ __forceinline__ float* tile(int a, int b) const {  // global tile indices, a >= b >= a0
    const int aa = a - a0, bb = b - a0;
    return p + ((int64_t)bb * T - ((int64_t)bb * (bb - 1)) / 2 + (aa - bb)) * kTileFloats;
  }
  __device__ __forceinline__ float* at(int r, int c) const {  // global indices, any order
    if (r < c) { const int t = r; r = c; c = t; }
    return tile(r >> 5, c >> 5) + (c & 31) * kTile + (r & 31);
  }
};

__device__ __forceinline__ int sturm_count(const float* dv, const float* e2, int n, float x,
                                           float pivmin) {
  float q = dv[0] - x;
  int cnt = q < 0.f;
  for (int i = 1; i < n; ++i) {
    if (fabsf(q) < pivmin) q = -pivmin;
    q = (dv[i] - x) - __fdividef(e2[i - 1], q);
    cnt += q < 0.f;
  }
  return cnt;
}

__host__ __device__ __forceinline__ int tiles_in(int T) { return T * (T + 1) / 2; }

// Tile index t of a T-row lower tile triangle (column-major order) -> (a, b)
// relative to its origin.
__device__ __forceinline__ void tile_rc(int t, int T, int& a, int& b) {
  b = 0;
  while (t >= T - b) { t -= T - b; ++b; }
  a = b + t;
}

}  // namespace

// Tile rows kept in shared memory for a given dynamic size and n_max.
__host__ __device__ int tridiag_smem_cap(int smem_bytes, int n_max) {
  const int npad = (n_max + kTile - 1) / kTile * kTile;
  const long scratch = 6L * npad + 128;
  const long avail = (long)smem_bytes / 4 - scratch;
  int T = 0;
  while ((long)tiles_in(T + 1) * kTileFloats <= avail) ++T;
  return T;
}

__global__ void __launch_bounds__(kTriThreads)
core_tridiag_kernel(const CoreDesc* __restrict__ descs, int smem_bytes, int n_max,
                    int* __restrict__ status) {
  extern __shared__ __align__(16) float smem[];
  const CoreDesc d = descs[blockIdx.x];
  const int n = d.rt + d.k;
  const int T = (n + kTile - 1) / kTile;
  const int npad = (n_max + kTile - 1) / kTile * kTile;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* dv = smem;             // npad: diagonal of T
  float* ev = dv + npad;        // npad: off-diagonal e[j] couples j, j+1
  float* vcur = ev + npad;      // npad: reflector of this step (global rows)
  float* pcur = vcur + npad;    // npad: p, then w of this step
  float* vprev = pcur + npad;   // npad: pending reflector
  float* wprev = vprev + npad;  // npad: pending w
  float* red = wprev + npad;    // 128
  float* tiles_smem = red + 128;
  const int capT = tridiag_smem_cap(smem_bytes, n_max);
  __shared__ float s_tau2, s_v0;
  __shared__ double s_trace;

  Tiles M;
  M.a0 = 0;
  M.T = T;
  M.p = (T <= capT) ? tiles_smem : d.work;

  // 1. assemble (both halves of diagonal tiles; zero padding beyond n)
  for (int t = wid; t < tiles_in(T); t += kTriWarps) {
    int a, b;
    tile_rc(t, T, a, b);
    float* tp = M.tile(a, b);
    const int r = a * kTile + lane;
    for (int cc = 0; cc < kTile; ++cc) {
      const int c = b * kTile + cc;
      float v = 0.f;
      if (r < n && c < n) {
        const int i = max(r, c), l = min(r, c);
        if (l < d.rt) {
          if (i < d.rt) v = (i == l) ? d.sigma[i] * d.sigma[i] : 0.f;
          else v = d.sigma[l] * d.P[(int64_t)l * d.ldp + (i - d.rt)];
        } else {
          v = d.Gaa[(int64_t)(l - d.rt) * d.ldb + (i - d.rt)];  // upper part of A^T A
        }
      }
      tp[cc * kTile + lane] = v;
    }
  }
  for (int i = tid; i < npad; i += kTriThreads) {
    vprev[i] = 0.f;
    wprev[i] = 0.f;
  }
  // ||A||_F^2 = tr(A^T A) from the Gram's diagonal when no energy is given
  __shared__ double s_energy_add;
  if (d.energy_add == nullptr) {
    double e = 0.0;
    for (int i = tid; i < d.k; i += kTriThreads) e += (double)d.Gaa[(int64_t)i * d.ldb + i];
    e = warp_sum_d(e);
    if (lane == 0) reinterpret_cast<double*>(red)[wid] = e;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kTriWarps; ++w) t += reinterpret_cast<double*>(red)[w];
      s_energy_add = t;
    }
  }
  __syncthreads();

  // 2. tridiagonalisation with a lazily applied rank-2 update
  for (int j = 0; j + 2 < n; ++j) {
    const int b0 = (j + 1) >> 5;  // first tile row/col holding trailing elements
    if (M.p != tiles_smem && (j & 31) == 0 && T - (j >> 5) <= capT) {
      // move tile rows >= j/32 on-chip
      Tiles S{tiles_smem, j >> 5, T - (j >> 5)};
      for (int t = wid; t < tiles_in(S.T); t += kTriWarps) {
        int a, b;
        tile_rc(t, S.T, a, b);
        const float* src = M.tile(S.a0 + a, S.a0 + b);
        float* dst = S.tile(S.a0 + a, S.a0 + b);
        for (int e = lane; e < kTileFloats; e += 32) dst[e] = src[e];
      }
      __syncthreads();
      M = S;
    }
    // (a) bring column j up to date with the pending update (support [j, n))
    {
      const float vpj = vprev[j], wpj = wprev[j];
      for (int i = j + tid; i < n; i += kTriThreads) {
        float* g = M.at(i, j);
        *g = fmaf(-vprev[i], wpj, fmaf(-wprev[i], vpj, *g));
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
    for (int i = tid; i < npad; i += kTriThreads) {
      float v = 0.f;
      if (tau2 != 0.f && i > j && i < n) v = (i == j + 1) ? s_v0 : *M.at(i, j);
      vcur[i] = v;
      pcur[i] = 0.f;
    }
    __syncthreads();
    // (b) fused pass over the trailing tiles: G -= vp wp^T + wp vp^T, p += G v
    {
      const int Tt = T - b0;  // trailing tile rows
      const int nt = tiles_in(Tt);
      const int lo = (int)((int64_t)nt * wid / kTriWarps);
      const int hi = (int)((int64_t)nt * (wid + 1) / kTriWarps);
      if (lo < hi) {
        int a, b;
        tile_rc(lo, Tt, a, b);
        float cp[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) cp[q] = 0.f;
        for (int t = lo; t < hi; ++t) {
          const int ga = b0 + a, gb = b0 + b;
          float* tp = M.tile(ga, gb);
          const int r = ga * kTile + lane;
          const float vr = vcur[r], vpr = vprev[r], wpr = wprev[r];
          const float4* vc4 = reinterpret_cast<const float4*>(vcur + gb * kTile);
          const float4* vp4 = reinterpret_cast<const float4*>(vprev + gb * kTile);
          const float4* wp4 = reinterpret_cast<const float4*>(wprev + gb * kTile);
          const float colw = (a == b) ? 0.f : vr;  // diagonal tiles: row sums cover both halves
          float rowacc = 0.f;
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            const float4 vc = vc4[q4], vp = vp4[q4], wp = wp4[q4];
            const float vcs[4] = {vc.x, vc.y, vc.z, vc.w};
            const float vps[4] = {vp.x, vp.y, vp.z, vp.w};
            const float wps[4] = {wp.x, wp.y, wp.z, wp.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int cc = q4 * 4 + u;
              float* g = tp + cc * kTile + lane;
              float val = *g;
              val = fmaf(-vpr, wps[u], fmaf(-wpr, vps[u], val));
              *g = val;
              rowacc = fmaf(val, vcs[u], rowacc);
              cp[cc] = fmaf(val, colw, cp[cc]);
            }
          }
          atomicAdd(&pcur[r], rowacc);
          ++a;
          const bool col_end = (a == Tt) || (t + 1 == hi);
          if (col_end) {
            // lane L ends with the sum over lanes of cp[L]
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
            atomicAdd(&pcur[gb * kTile + lane], cp[0]);
#pragma unroll
            for (int q = 0; q < 32; ++q) cp[q] = 0.f;
            if (a == Tt) { ++b; a = b; }
          }
        }
      }
    }
    __syncthreads();
    // w = tau2 p - (tau2^2 / 2)(p^T v) v, kept only on the trailing range
    float pp = 0.f;
    for (int i = j + 1 + tid; i < n; i += kTriThreads) pp = fmaf(pcur[i], vcur[i], pp);
    const float kk = 0.5f * tau2 * tau2 * block_sum(pp, red);
    for (int i = tid; i < npad; i += kTriThreads)
      pcur[i] = (i > j && i < n) ? fmaf(tau2, pcur[i], -kk * vcur[i]) : 0.f;
    __syncthreads();
    // the current step becomes the pending update
    float* tv = vprev; vprev = vcur; vcur = tv;
    float* tw = wprev; wprev = pcur; pcur = tw;
  }
  // last 2 x 2 (or 1 x 1) block, with the pending update (support [n-2, n))
  if (tid == 0) {
    if (n >= 2) {
      const int j = n - 2;
      float a = *M.at(j, j), b = *M.at(j + 1, j), c = *M.at(j + 1, j + 1);
      a = fmaf(-2.f * vprev[j], wprev[j], a);
      b = fmaf(-vprev[j + 1], wprev[j], fmaf(-wprev[j + 1], vprev[j], b));
      c = fmaf(-2.f * vprev[j + 1], wprev[j + 1], c);
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
  float* lam = pcur;
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
      top += (double)lam[q];
      d.sigma_out[q] = sqrtf(fmaxf(lam[q], 0.f));
    }
    top = warp_sum_d(top);
    if (lane == 0) {
      const double energy_new = d.scal[0] + (d.energy_add ? d.energy_add[0] : s_energy_add);
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

int64_t tridiag_work_floats(int n) {
  const int T = (n + kTile - 1) / kTile;
  return (int64_t)tiles_in(T) * kTileFloats;
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
