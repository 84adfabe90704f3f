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
//  1. G is assembled as 32 x 32 tiles of its lower tile triangle (diagonal
//     tiles hold both halves), listed column by column.  The tiles consumed
//     last live in shared memory; when they do not all fit, the next ones go
//     to tensor memory (up to 64 tiles, one tile per warp-wide 32x32b load),
//     and only what still does not fit -- the leading tile columns of the
//     largest cores -- stays in a global workspace.  Nothing migrates: a
//     tile column leaves the trailing matrix before any tile could move.
//  2. Householder tridiagonalisation, G <- H G H, H = I - tau v v^T, with two
//     block barriers per step:
//       serial phase (warp 0): finish w of the previous step from p, apply
//         the pending rank-2 update to column s (kept as a vector), build
//         the reflector of column s;
//       main pass (all warps): one sweep over the trailing tiles applies the
//         pending update and accumulates p = G v and p^T v; it also copies
//         out column s + 1 for the next serial phase.
//     Vectors are indexed by global row and vanish outside the trailing
//     range, so boundary tiles need no masks.  Column sums of off-diagonal
//     tiles accumulate across a tile column and are reduced once per column.
//  3. Multisection bisection on Sturm counts of the tridiagonal matrix for
//     the top r_new eigenvalues (g threads per eigenvalue, the interval
//     shrinks (g + 1)-fold per iteration).
//  4. FP64 epilogue: sigma~, tail = discarded_state + tr(T) - sum top, the
//     subtraction form sum ||A||^2 - sum sigma~^2, and the accept flag; the
//     block energy ||A||^2 is the trace of A^T A unless given.
#include "common.cuh"
#include "tmem.cuh"

namespace csvd {
namespace {

constexpr int kTriThreads = 512;
constexpr int kTriWarps = kTriThreads / 32;
constexpr int kBisectMax = 64;
constexpr int kTile = 32;
constexpr int kTileFloats = kTile * kTile;
constexpr int kTmemTiles = 64;            // 4 lane quarters x 16 tiles of 32 columns
constexpr int kTmemCols = 512;
constexpr int kTmemMinSmem = 120 * 1024;  // at most one CTA per SM from this size on
constexpr int kVecs = 7;                  // dv, ev, v (2), p/w (2), column

__host__ __device__ __forceinline__ int tiles_in(int T) { return T * (T + 1) / 2; }
// First list position of tile column b in a T-row lower tile triangle.
__host__ __device__ __forceinline__ int col_start(int b, int T) { return b * T - b * (b - 1) / 2; }

// Placement of the tile list of one core: positions [0, Lg) in the global
// workspace (tile columns 0 .. g-1), [Lg, Lg + Ntm) in TMEM (tile t = L - Lg
// at lane quarter t % 4, column 32 (t / 4)), [Ls, T(T+1)/2) in shared memory.
struct TileLayout {
  int T, Lg, Ntm, Ls;
};

__host__ __device__ int smem_tile_cap(int smem_bytes, int n_max) {
  const int npad = (n_max + kTile - 1) / kTile * kTile;
  const long avail = (long)smem_bytes / 4 - (long)kVecs * npad - 128;
  return avail > 0 ? (int)(avail / kTileFloats) : 0;
}

__host__ __device__ TileLayout tile_layout(int n, int smem_bytes, int n_max) {
  TileLayout L;
  L.T = (n + kTile - 1) / kTile;
  const int cs = smem_tile_cap(smem_bytes, n_max);
  const int cap = cs + (smem_bytes >= kTmemMinSmem ? kTmemTiles : 0);
  int g = 0;
  while (g < L.T && tiles_in(L.T - g) > cap) ++g;
  L.Lg = col_start(g, L.T);
  const int on = tiles_in(L.T - g);
  L.Ntm = on > cs ? on - cs : 0;
  L.Ls = L.Lg + L.Ntm;
  return L;
}

__device__ __forceinline__ void tile_of(int L, int T, int& a, int& b) {
  b = 0;
  int st = 0;
  while (st + T - b <= L) {
    st += T - b;
    ++b;
  }
  a = b + (L - st);
}

__device__ __forceinline__ void tile_next(int& a, int& b, int T) {
  if (++a == T) {
    ++b;
    a = b;
  }
}

// Element (r, c) of G (zero outside n x n).
__device__ __forceinline__ float core_gram(const CoreDesc& d, int n, int r, int c) {
  if (r >= n || c >= n) return 0.f;
  const int i = max(r, c), l = min(r, c);
  if (l < d.rt) {
    if (i < d.rt) return (i == l) ? d.sigma[i] * d.sigma[i] : 0.f;
    return d.sigma[l] * d.P[(int64_t)l * d.ldp + (i - d.rt)];
  }
  return d.Gaa[(int64_t)(l - d.rt) * d.ldb + (i - d.rt)];  // upper part of A^T A
}

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

// Vectors of one main pass.
struct Step {
  const float* vcur;   // v of this step
  const float* vprev;  // pending update: v and w of the previous step
  const float* wprev;
  float* pcur;         // p = G v accumulator
  float* colv;         // receives column s + 1
  int b0, ccn;         // tile column and in-tile column of s + 1
};

// Lane L ends with the sum over lanes of cp[L]; added to p[32 b + L].
__device__ __forceinline__ void flush_cols(float (&cp)[32], int b, int lane, const Step& st,
                                           float& pv) {
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
  const int c = b * kTile + lane;
  atomicAdd(&st.pcur[c], cp[0]);
  pv = fmaf(cp[0], st.vcur[c], pv);
#pragma unroll
  for (int q = 0; q < 32; ++q) cp[q] = 0.f;
}

// The per-element work of a tile whose row `lane` holds val[0..31]:
// G -= vp wp^T + wp vp^T, then row sums into rowacc and column sums into cp.
__device__ __forceinline__ void tile_update(float (&val)[32], float (&cp)[32], float& rowacc,
                                            int a, int b, int lane, const Step& st) {
  const int r = a * kTile + lane;
  const float vr = st.vcur[r], vpr = st.vprev[r], wpr = st.wprev[r];
  const float colw = (a == b) ? 0.f : vr;  // diagonal tiles: row sums cover both halves
  const float4* vc4 = reinterpret_cast<const float4*>(st.vcur + b * kTile);
  const float4* vp4 = reinterpret_cast<const float4*>(st.vprev + b * kTile);
  const float4* wp4 = reinterpret_cast<const float4*>(st.wprev + b * kTile);
#pragma unroll
  for (int q4 = 0; q4 < 8; ++q4) {
    const float4 vc = vc4[q4], vp = vp4[q4], wp = wp4[q4];
    const float vcs[4] = {vc.x, vc.y, vc.z, vc.w};
    const float vps[4] = {vp.x, vp.y, vp.z, vp.w};
    const float wps[4] = {wp.x, wp.y, wp.z, wp.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cc = q4 * 4 + u;
      const float x = fmaf(-vpr, wps[u], fmaf(-wpr, vps[u], val[cc]));
      val[cc] = x;
      rowacc = fmaf(x, vcs[u], rowacc);
      cp[cc] = fmaf(x, colw, cp[cc]);
    }
  }
}

// Tiles at list positions [La, Lb), stored at base + (L - Lbase) tiles
// (shared or global memory).
__device__ __forceinline__ void mem_tiles(float* base, int Lbase, int La, int Lb, int T, int lane,
                                          const Step& st, float& pv) {
  if (La >= Lb) return;
  int a, b;
  tile_of(La, T, a, b);
  float cp[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) cp[q] = 0.f;
  for (int L = La; L < Lb; ++L) {
    float* tp = base + (int64_t)(L - Lbase) * kTileFloats;
    const int r = a * kTile + lane;
    // The same ordering as the TMEM path: load the row, update, store.  The
    // 32 loads are independent, so they are all in flight together.
    float val[32];
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) val[cc] = tp[cc * kTile + lane];
    float rowacc = 0.f;
    tile_update(val, cp, rowacc, a, b, lane, st);
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) tp[cc * kTile + lane] = val[cc];
    if (b == st.b0) {
      float x = 0.f;
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) x = (cc == st.ccn) ? val[cc] : x;
      st.colv[r] = x;
    }
    atomicAdd(&st.pcur[r], rowacc);
    pv = fmaf(rowacc, st.vcur[r], pv);
    const int bb = b;
    tile_next(a, b, T);
    if (b != bb || L + 1 == Lb) flush_cols(cp, bb, lane, st, pv);
  }
}

// The warp's TMEM tiles: positions Lg + t, t = tfirst + 4 j, j in [ja, jb).
__device__ __forceinline__ void tmem_tiles(uint32_t tq, int Lg, int tfirst, int ja, int jb, int T,
                                           int lane, const Step& st, float& pv) {
  if (ja >= jb) return;
  int t = tfirst + 4 * ja;
  int a, b;
  tile_of(Lg + t, T, a, b);
  float cp[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) cp[q] = 0.f;
  for (int j = ja; j < jb; ++j, t += 4) {
    const uint32_t taddr = tq + (uint32_t)(t >> 2) * 32u;
    float val[32];
    tmem_load_tile(taddr, val);
    float rowacc = 0.f;
    tile_update(val, cp, rowacc, a, b, lane, st);
    tmem_store_tile(taddr, val);
    const int r = a * kTile + lane;
    if (b == st.b0) {
      float x = 0.f;
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) x = (cc == st.ccn) ? val[cc] : x;
      st.colv[r] = x;
    }
    atomicAdd(&st.pcur[r], rowacc);
    pv = fmaf(rowacc, st.vcur[r], pv);
    const int bb = b;
#pragma unroll
    for (int u = 0; u < 4; ++u) tile_next(a, b, T);
    if (b != bb || j + 1 == jb) flush_cols(cp, bb, lane, st, pv);
  }
}

}  // namespace

__global__ void __launch_bounds__(kTriThreads)
core_tridiag_kernel(const CoreDesc* __restrict__ descs, int smem_bytes, int n_max,
                    int* __restrict__ status) {
  extern __shared__ __align__(16) float smem[];
  const CoreDesc d = descs[blockIdx.x];
  const int n = d.rt + d.k;
  const int npad = (n_max + kTile - 1) / kTile * kTile;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* dv = smem;          // npad: diagonal of T
  float* ev = dv + npad;     // npad: off-diagonal e[j] couples j, j+1
  float* vb0 = ev + npad;    // npad x 2: v of even / odd steps
  float* vb1 = vb0 + npad;
  float* pb0 = vb1 + npad;   // npad x 2: p of a step, turned into its w in place
  float* pb1 = pb0 + npad;
  float* colv = pb1 + npad;  // npad: the current column (rows >= s)
  float* red = colv + npad;  // 128
  float* tsm = red + 128;    // shared-memory tiles
  const TileLayout Lay = tile_layout(n, smem_bytes, n_max);
  const int T = Lay.T, Nt = tiles_in(T);
  __shared__ uint32_t s_tmem;
  __shared__ float s_pv[2];
  __shared__ double s_trace, s_energy_add;

  if (n < 1 || n > n_max || Lay.Ls > Nt - 1 || Lay.Ntm > kTmemTiles ||
      (Lay.Lg > 0 && d.work == nullptr)) {
    if (tid == 0) atomicOr(status, kStatusBadShape);
    return;
  }
  const bool use_tmem = Lay.Ntm > 0;
  if (use_tmem && wid == 0) tmem_alloc(&s_tmem, kTmemCols);

  // 1. assemble global and shared-memory tiles, the first column, zero vectors
  for (int v = wid; v < Lay.Lg + (Nt - Lay.Ls); v += kTriWarps) {
    const bool glob = v < Lay.Lg;
    const int L = glob ? v : Lay.Ls + (v - Lay.Lg);
    float* tp = glob ? d.work + (int64_t)L * kTileFloats : tsm + (int64_t)(L - Lay.Ls) * kTileFloats;
    int a, b;
    tile_of(L, T, a, b);
    const int r = a * kTile + lane;
    for (int cc = 0; cc < kTile; ++cc) tp[cc * kTile + lane] = core_gram(d, n, r, b * kTile + cc);
  }
  for (int i = tid; i < npad; i += kTriThreads) {
    vb0[i] = 0.f;
    vb1[i] = 0.f;
    pb0[i] = 0.f;
    pb1[i] = 0.f;
    colv[i] = core_gram(d, n, i, 0);
  }
  // ||A||_F^2 = tr(A^T A) from the Gram's diagonal when no energy is given
  if (d.energy_add == nullptr) {
    double e = 0.0;
    for (int i = tid; i < d.k; i += kTriThreads) e += (double)d.Gaa[(int64_t)i * d.ldb + i];
    e = warp_sum_d(e);
    if (lane == 0) reinterpret_cast<double*>(red)[wid] = e;
  }
  if (tid == 0) {
    s_pv[0] = 0.f;
    s_pv[1] = 0.f;
  }
  __syncthreads();
  if (tid == 0 && d.energy_add == nullptr) {
    double t = 0.0;
    for (int w = 0; w < kTriWarps; ++w) t += reinterpret_cast<double*>(red)[w];
    s_energy_add = t;
  }
  uint32_t tq = 0;  // TMEM address of this warp's lane quarter
  if (use_tmem) {
    tmem_fence_after();
    const int q = wid & 3;
    tq = s_tmem + ((uint32_t)(q * 32) << 16);
    for (int t = q + 4 * (wid >> 2); t < Lay.Ntm; t += 16) {
      int a, b;
      tile_of(Lay.Lg + t, T, a, b);
      const int r = a * kTile + lane;
      float val[32];
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) val[cc] = core_gram(d, n, r, b * kTile + cc);
      tmem_store_tile(tq + (uint32_t)(t >> 2) * 32u, val);
    }
    tmem_wait_st();
    tmem_fence_before();
  }
  __syncthreads();

  // 2. tridiagonalisation
  float tau_prev = 0.f;  // warp 0: tau of the pending reflector
  for (int s = 0;; ++s) {
    float* vcur = (s & 1) ? vb1 : vb0;
    float* vprev = (s & 1) ? vb0 : vb1;
    float* pcur = (s & 1) ? pb1 : pb0;
    float* wprev = (s & 1) ? pb0 : pb1;
    const bool last = s + 2 >= n;
    const int b0 = (s + 1) >> 5;
    if (wid == 0) {
      // w of the previous step (in place of its p), the pending update on
      // column s, and the reflector of column s
      const float kk = (s >= 1) ? 0.5f * tau_prev * tau_prev * s_pv[(s + 1) & 1] : 0.f;
      const float vs = vprev[s];
      const float ws = (s >= 1) ? fmaf(tau_prev, wprev[s], -kk * vs) : 0.f;
      __syncwarp();
      const int ilo = min(s, b0 * kTile);  // rows the main pass of this step touches start here
      float part = 0.f;
      for (int i = ilo + lane; i < n; i += 32) {
        const float vp = vprev[i];
        float w = 0.f;
        if (s >= 1 && i >= s) w = fmaf(tau_prev, wprev[i], -kk * vp);
        wprev[i] = w;
        if (i >= s) {
          const float c = fmaf(-vp, ws, fmaf(-w, vs, colv[i]));
          colv[i] = c;
          if (i >= s + 2) part = fmaf(c, c, part);
        }
      }
      part = warp_sum(part);
      __syncwarp();
      if (last) {
        if (lane == 0) {
          if (n >= 2) {
            const int j = n - 1;
            const float* tl = tsm + (int64_t)(Nt - 1 - Lay.Ls) * kTileFloats;
            const float gjj = tl[(j & 31) * kTile + (j & 31)];
            dv[j - 1] = colv[j - 1];
            ev[j - 1] = colv[j];
            dv[j] = fmaf(-2.f * vprev[j], wprev[j], gjj);
          } else {
            dv[0] = colv[0];
          }
          ev[n - 1] = 0.f;
        }
      } else {
        const float x0 = colv[s + 1];
        float beta = x0, tau = 0.f, v0 = 0.f;
        if (part != 0.f) {
          const float nrm = sqrtf(fmaf(x0, x0, part));
          beta = x0 >= 0.f ? -nrm : nrm;
          v0 = x0 - beta;
          tau = 2.f / fmaf(v0, v0, part);
        }
        if (lane == 0) {
          dv[s] = colv[s];
          ev[s] = beta;
          s_pv[s & 1] = 0.f;
        }
        for (int i = ilo + lane; i < npad; i += 32) {
          float v = 0.f;
          if (tau != 0.f && i > s && i < n) v = (i == s + 1) ? v0 : colv[i];
          vcur[i] = v;
          pcur[i] = 0.f;
        }
        tau_prev = tau;
      }
    }
    if (last) break;
    __syncthreads();
    if (use_tmem) tmem_fence_after();

    // main pass over the trailing tiles (tile columns >= b0)
    {
      const Step st{vcur, vprev, wprev, pcur, colv, b0, (s + 1) & 31};
      const int L0 = col_start(b0, T);
      const int ng = max(0, Lay.Lg - L0);  // trailing tiles in global memory
      const int Ls0 = max(L0, Lay.Ls);
      const int nf = ng + (Nt - Ls0);      // ... plus those in shared memory
      const int t0 = max(0, L0 - Lay.Lg);  // first trailing TMEM tile
      int nq0 = 0, nq1 = 0, nq2 = 0, nq3 = 0;
      if (use_tmem) {
        const int f0 = t0 + ((0 - t0) & 3), f1 = t0 + ((1 - t0) & 3);
        const int f2 = t0 + ((2 - t0) & 3), f3 = t0 + ((3 - t0) & 3);
        nq0 = Lay.Ntm > f0 ? (Lay.Ntm - f0 + 3) >> 2 : 0;
        nq1 = Lay.Ntm > f1 ? (Lay.Ntm - f1 + 3) >> 2 : 0;
        nq2 = Lay.Ntm > f2 ? (Lay.Ntm - f2 + 3) >> 2 : 0;
        nq3 = Lay.Ntm > f3 ? (Lay.Ntm - f3 + 3) >> 2 : 0;
      }
      const int ntm = nq0 + nq1 + nq2 + nq3;
      const int q = wid & 3, qi = wid >> 2;
      auto quarter = [&](int u) {
        const int qq = u & 3;
        return qq == 0 ? nq0 : qq == 1 ? nq1 : qq == 2 ? nq2 : nq3;
      };
      auto tm_count = [&](int u) {
        const int nn = quarter(u), ui = u >> 2;
        return (ui + 1) * nn / 4 - ui * nn / 4;
      };
      int f_lo, f_hi;
      if (ntm == 0) {
        f_lo = nf * wid / kTriWarps;
        f_hi = nf * (wid + 1) / kTriWarps;
      } else {
        // water-filling: free tiles top every warp up to the same level
        int lam = (nf + ntm + kTriWarps - 1) / kTriWarps;
        for (;;) {
          int sum = 0;
          for (int u = 0; u < kTriWarps; ++u) sum += max(0, lam - tm_count(u));
          if (sum >= nf) break;
          ++lam;
        }
        int st0 = 0;
        for (int u = 0; u < wid; ++u) st0 += max(0, lam - tm_count(u));
        f_lo = min(st0, nf);
        f_hi = min(nf, st0 + max(0, lam - tm_count(wid)));
      }
      float pv = 0.f;
      // free tiles: virtual positions [0, ng) global, [ng, nf) shared
      mem_tiles(d.work, 0, L0 + f_lo, L0 + min(f_hi, ng), T, lane, st, pv);
      mem_tiles(tsm, Lay.Ls, Ls0 + max(f_lo - ng, 0), Ls0 + max(f_hi - ng, 0), T, lane, st, pv);
      if (ntm > 0) {
        const int nn = quarter(q);
        const int tfirst = t0 + ((q - t0) & 3);
        tmem_tiles(tq, Lay.Lg, tfirst, qi * nn / 4, (qi + 1) * nn / 4, T, lane, st, pv);
        tmem_wait_st();
      }
      pv = warp_sum(pv);
      if (lane == 0) atomicAdd(&s_pv[s & 1], pv);
    }
    if (use_tmem) tmem_fence_before();
    __syncthreads();
  }
  __syncthreads();
  if (use_tmem && wid == 0) {
    tmem_fence_after();
    tmem_dealloc(s_tmem, kTmemCols);
  }

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
  float* e2 = vb0;  // reuse
  float* lam = pb0;
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

int tridiag_smem_bytes(int n_max, bool large) {
  if (large) return kTriLargeSmemBytes;
  const int npad = (n_max + kTile - 1) / kTile * kTile;
  const int T = npad / kTile;
  return (kVecs * npad + 128 + tiles_in(T) * kTileFloats) * 4;
}

int64_t tridiag_work_floats(int n, int smem_bytes, int n_max) {
  return (int64_t)tile_layout(n, smem_bytes, n_max).Lg * kTileFloats;
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
