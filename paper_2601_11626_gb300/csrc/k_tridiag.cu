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
// One CTA per item, in three launch classes by core size: 4 warps (four
// CTAs per SM) for n <= 192, 8 warps (two per SM) for n <= 320, 16 warps
// (one per SM) above.  Each CTA owns its SM share of tensor memory (TMEM).
// Tiles are processed 16 columns at a time.
//  1. G is assembled as 32 x 32 tiles of its lower tile triangle (diagonal
//     tiles hold both halves), listed column by column.  The tiles consumed
//     last -- revisited by the most steps -- live in TMEM (one tile per
//     warp-wide 32x32b load or store); the ones before them in shared memory;
//     only what still does not fit, the leading tile columns of the largest
//     cores, stays in a global workspace.  Nothing migrates: a tile column
//     leaves the trailing matrix before any tile could move.
//  2. Householder tridiagonalisation, G <- H G H, H = I - tau v v^T, with two
//     block barriers per step:
//       phase A (one row per thread): w of the previous step from its p, the
//         pending rank-2 update on column s (kept as a vector), v below
//         s + 1, a zeroed p, and partial sums of ||x||^2;
//       phase B: every thread forms the reflector scalars itself, then all
//         warps sweep the trailing tiles once: apply the pending update,
//         accumulate p = G v and p^T v, and copy out column s + 1.
//     Vectors are indexed by global row and vanish outside the trailing
//     range, so boundary tiles need no masks.  Column sums of off-diagonal
//     tiles accumulate across a tile column and are reduced once per column.
//     A warp reaches only its TMEM lane quarter, so TMEM tiles are dealt to
//     quarters in pairs, round-robin; shared-memory tiles top the warps up
//     to equal counts; global tiles are shared evenly.  The shares are set
//     once per tile column.  Tile updates use packed f32x2 FMAs.
//  3. Multisection bisection on Sturm counts of the tridiagonal matrix for
//     the top r_new eigenvalues (g threads per eigenvalue, the interval
//     shrinks (g + 1)-fold per iteration).
//  4. FP64 epilogue: sigma~, tail = discarded_state + tr(T) - sum top, the
//     subtraction form sum ||A||^2 - sum sigma~^2, and the accept flag; the
//     block energy ||A||^2 is the trace of A^T A unless given.
#include <atomic>
#include <cstdio>
#include <string>

#include "common.cuh"
#include "tmem.cuh"

namespace csvd {
namespace {

constexpr int kBisectMax = 64;
// iteration cap of the bisection (kBisectMax; lowered only by the failure-path test hook)
__device__ int d_bisect_cap = kBisectMax;
constexpr int kTile = 32;
constexpr int kTileFloats = kTile * kTile;
constexpr int kVecs = 9;  // dv, ev, v (2), p (2), w, column (2)
constexpr int kRed = 128;

struct ClassCfg {
  int warps, max_n;
};
constexpr ClassCfg kClass[3] = {{4, 192}, {8, 320}, {16, 1 << 30}};
// CTAs per SM of each class (16 warps per SM at 128 registers a thread) and
// the TMEM columns each CTA allocates (a power of two, the class's SM share).
constexpr int kPerSm[3] = {4, 2, 1};
constexpr int kTmemColsOf[3] = {128, 256, 512};

__host__ __device__ __forceinline__ int tiles_in(int T) { return T * (T + 1) / 2; }
// First list position of tile column b in a T-row lower tile triangle.
__host__ __device__ __forceinline__ int col_start(int b, int T) { return b * T - b * (b - 1) / 2; }

// Placement of the tile list of one core: positions [0, Lg) in the global
// workspace (tile columns 0 .. g-1), [Lg, Lt) in shared memory (slot L - Lg),
// [Lt, T(T+1)/2) in TMEM (tile t = L - Lt at the lane quarter and slot
// given by tm_tile / tm_slot below, 32 columns per slot).
struct TileLayout {
  int T, Lg, Lt, Ntm;
};

__host__ __device__ int smem_tile_cap(int smem_bytes, int n_max) {
  const int npad = (n_max + kTile - 1) / kTile * kTile;
  const long avail = (long)smem_bytes / 4 - (long)kVecs * npad - kRed;
  return avail > 0 ? (int)(avail / kTileFloats) : 0;
}

__host__ __device__ TileLayout tile_layout(int n, int tmem_cols, int smem_bytes, int n_max) {
  TileLayout L;
  L.T = (n + kTile - 1) / kTile;
  const int nt = tiles_in(L.T);
  const int ct = tmem_cols / 8;  // TMEM tiles: 4 lane quarters x (columns / 32)
  const int cap = ct + smem_tile_cap(smem_bytes, n_max);
  int g = 0;
  while (g < L.T && tiles_in(L.T - g) > cap) ++g;
  L.Lg = col_start(g, L.T);
  L.Ntm = min(nt - L.Lg, ct);
  L.Lt = nt - L.Ntm;
  return L;
}

// List position L -> tile (a, b) (rows a >= b).
__host__ __device__ __forceinline__ void tile_of(int L, int T, int& a, int& b) {
  const float q = (float)(2 * T + 1);
  int bb = (int)((q - sqrtf(fmaxf(q * q - 8.f * (float)L, 0.f))) * 0.5f);
  bb = max(0, min(bb, T - 1));
  while (bb > 0 && col_start(bb, T) > L) --bb;
  while (bb + 1 < T && col_start(bb + 1, T) <= L) ++bb;
  b = bb;
  a = bb + (L - col_start(bb, T));
}

__host__ __device__ __forceinline__ void tile_next(int& a, int& b, int T) {
  if (++a == T) {
    ++b;
    a = b;
  }
}

// Move k >= 0 positions forward in the column-major tile list.
__host__ __device__ __forceinline__ void tile_skip(int& a, int& b, int T, int k) {
  a += k;
  while (a >= T && b + 1 < T) {  // column b has rows b .. T-1
    a -= T - (b + 1);
    ++b;
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
  if (i == l && d.colE) return (float)d.colE[l - d.rt];    // exact column energy
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

// Vectors of one main pass.  Every warp writes v_s[s+1] (= v0, the same
// value) into the shared vector itself before it reads it.
struct Step {
  const float* vcur;   // v of this step
  const float* vprev;  // pending update: v and w of the previous step
  const float* wprev;
  float* pcur;         // p = G v accumulator
  float* cnext;        // receives column s + 1
  float* glast;        // receives G(n-1, n-1)
  int b0, ccn, s1;     // tile column and in-tile column of s + 1; s + 1
  int last_r;          // n - 1
  float v0;
};

// Column-sum accumulators: cp[i] holds columns 2i and 2i + 1 of a tile column.
#define CP(k) ((k) & 1 ? cp[(k) >> 1].y : cp[(k) >> 1].x)

// Lane L ends with the sum over lanes of column L's accumulator; added to
// p[32 b + L].
__device__ __forceinline__ void flush_cols(float2 (&cp)[16], int b, int lane, const Step& st,
                                           float& pv) {
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) {
#pragma unroll
    for (int i = 0; i < sh; ++i) {
      const bool up = (lane & sh) != 0;
      const float send = up ? CP(i) : CP(i + sh);
      const float keep = up ? CP(i + sh) : CP(i);
      CP(i) = keep + __shfl_xor_sync(0xffffffffu, send, sh);
    }
  }
  const int c = b * kTile + lane;
  atomicAdd(&st.pcur[c], cp[0].x);
  pv = fmaf(cp[0].x, st.vcur[c], pv);
#pragma unroll
  for (int q = 0; q < 16; ++q) cp[q] = make_float2(0.f, 0.f);
}
#undef CP

// Where row `lane` of a tile lives, moved 16 columns at a time.  Shared-memory
// tiles are row-major with 16-byte chunks XOR-swizzled by row (element
// (i, j) at 32 i + 4 ((j / 4) ^ (i % 8)) + j % 4), so a row moves with
// conflict-free 128-bit accesses; global tiles are column-major (element
// (i, j) at 32 j + i), one coalesced access per column; TMEM tiles hold row
// i in lane i of the warp's quarter.
struct SmemTile {
  float* tp;
  __device__ __forceinline__ void load16(int lane, int k16, float2 (&v)[8]) const {
    const float4* rp = reinterpret_cast<const float4*>(tp + lane * kTile);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 x = rp[(4 * k16 + c) ^ (lane & 7)];
      v[2 * c] = make_float2(x.x, x.y);
      v[2 * c + 1] = make_float2(x.z, x.w);
    }
  }
  __device__ __forceinline__ void store16(int lane, int k16, const float2 (&v)[8]) const {
    float4* rp = reinterpret_cast<float4*>(tp + lane * kTile);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      rp[(4 * k16 + c) ^ (lane & 7)] = make_float4(v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y);
  }
};
struct GlobTile {
  float* tp;
  __device__ __forceinline__ void load16(int lane, int k16, float2 (&v)[8]) const {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      v[j] = make_float2(tp[(16 * k16 + 2 * j) * kTile + lane], tp[(16 * k16 + 2 * j + 1) * kTile + lane]);
  }
  __device__ __forceinline__ void store16(int lane, int k16, const float2 (&v)[8]) const {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      tp[(16 * k16 + 2 * j) * kTile + lane] = v[j].x;
      tp[(16 * k16 + 2 * j + 1) * kTile + lane] = v[j].y;
    }
  }
};
struct TmemTile {
  uint32_t taddr;
  __device__ __forceinline__ void load16(int, int k16, float2 (&v)[8]) const {
    uint32_t r[16];
    tmem_load16(taddr + 16u * k16, r);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
  }
  __device__ __forceinline__ void store16(int, int k16, const float2 (&v)[8]) const {
    uint32_t r[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) { r[2 * j] = __float_as_uint(v[j].x); r[2 * j + 1] = __float_as_uint(v[j].y); }
    tmem_store16(taddr + 16u * k16, r);
  }
};

// Columns 16 k16 .. 16 k16 + 15 of the K tiles into registers (a TMEM pair:
// both loads before one wait).
template <int K, class Tile>
__device__ __forceinline__ void load_group(const Tile (&tl)[K], int lane, int k16, float2 (&v)[K][8]) {
#pragma unroll
  for (int t = 0; t < K; ++t) tl[t].load16(lane, k16, v[t]);
}
template <>
__device__ __forceinline__ void load_group<2, TmemTile>(const TmemTile (&tl)[2], int, int k16,
                                                        float2 (&v)[2][8]) {
  uint32_t r[16], q[16];
  tmem_load16x2(tl[0].taddr + 16u * k16, tl[1].taddr + 16u * k16, r, q);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v[0][j] = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
    v[1][j] = make_float2(__uint_as_float(q[2 * j]), __uint_as_float(q[2 * j + 1]));
  }
}

// K tiles of one tile column b (rows a, a + 1, ...), 16 columns at a time:
// G -= vp wp^T + wp vp^T, row sums (two partial chains per tile, added to
// p[row]) and column sums (kept in cp across the tiles of the column),
// column s + 1 and G(n-1, n-1) copied out.  Pairs of columns go through
// packed f32x2 FMAs; the column vectors are loaded once for the K tiles.
template <int K, class Tile>
__device__ __forceinline__ void process_tiles(const Tile (&tl)[K], int a, int b, int lane,
                                              const Step& st, float2 (&cp)[16], float& pv) {
  float vr[K], cx[K], gx[K];
  float2 nvp[K], nwp[K], colw[K], ra[K];
  bool last_tile[K];  // the diagonal tile holding G(n-1, n-1): same in every lane
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const int r = (a + t) * kTile + lane;
    vr[t] = st.vcur[r];
    const float p = -st.vprev[r], w = -st.wprev[r];
    nvp[t] = make_float2(p, p);
    nwp[t] = make_float2(w, w);
    const float cw = (a + t == b) ? 0.f : vr[t];  // diagonal tiles: row sums cover both halves
    colw[t] = make_float2(cw, cw);
    ra[t] = make_float2(0.f, 0.f);
    cx[t] = gx[t] = 0.f;
    last_tile[t] = a + t == b && b == (st.last_r >> 5);
  }
  const float4* vc4 = reinterpret_cast<const float4*>(st.vcur + b * kTile);
  const float4* vp4 = reinterpret_cast<const float4*>(st.vprev + b * kTile);
  const float4* wp4 = reinterpret_cast<const float4*>(st.wprev + b * kTile);
  const bool col_next = b == st.b0;  // this tile column holds column s + 1
#pragma unroll
  for (int k16 = 0; k16 < 2; ++k16) {
    float2 v[K][8];
    load_group<K>(tl, lane, k16, v);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int q4 = 4 * k16 + h;
      const float4 vc = vc4[q4], vp = vp4[q4], wp = wp4[q4];
      const float2 vc0 = make_float2(vc.x, vc.y), vc1 = make_float2(vc.z, vc.w);
      const float2 vp0 = make_float2(vp.x, vp.y), vp1 = make_float2(vp.z, vp.w);
      const float2 wp0 = make_float2(wp.x, wp.y), wp1 = make_float2(wp.z, wp.w);
#pragma unroll
      for (int t = 0; t < K; ++t) {
        float2 x0 = v[t][2 * h], x1 = v[t][2 * h + 1];
        x0 = __ffma2_rn(nwp[t], vp0, x0);
        x1 = __ffma2_rn(nwp[t], vp1, x1);
        x0 = __ffma2_rn(nvp[t], wp0, x0);
        x1 = __ffma2_rn(nvp[t], wp1, x1);
        v[t][2 * h] = x0;
        v[t][2 * h + 1] = x1;
        ra[t] = __ffma2_rn(x0, vc0, ra[t]);
        ra[t] = __ffma2_rn(x1, vc1, ra[t]);
        cp[2 * q4] = __ffma2_rn(x0, colw[t], cp[2 * q4]);
        cp[2 * q4 + 1] = __ffma2_rn(x1, colw[t], cp[2 * q4 + 1]);
      }
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
      tl[t].store16(lane, k16, v[t]);
      if (col_next) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          cx[t] = (16 * k16 + j == st.ccn) ? ((j & 1) ? v[t][j >> 1].y : v[t][j >> 1].x) : cx[t];
      }
      if (last_tile[t]) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          gx[t] = (16 * k16 + j == (st.last_r & 31)) ? ((j & 1) ? v[t][j >> 1].y : v[t][j >> 1].x)
                                                    : gx[t];
      }
    }
  }
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const int r = (a + t) * kTile + lane;
    if (col_next) st.cnext[r] = cx[t];
    if (last_tile[t] && r == st.last_r) *st.glast = gx[t];
    const float rowacc = ra[t].x + ra[t].y;
    atomicAdd(&st.pcur[r], rowacc);
    pv = fmaf(rowacc, vr[t], pv);
  }
}

// Tiles at list positions [La, Lb), stored at base + (L - Lbase) tiles;
// two at a time while they share a tile column.
template <class Tile>
__device__ __forceinline__ void mem_tiles(float* base, int Lbase, int La, int Lb, int a, int b,
                                          int T, int lane, const Step& st, float& pv) {
  if (La >= Lb) return;
  float2 cp[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) cp[q] = make_float2(0.f, 0.f);
  for (int L = La; L < Lb;) {
    int used;
    if (L + 1 < Lb && a + 1 < T) {
      const Tile tl[2] = {Tile{base + (int64_t)(L - Lbase) * kTileFloats},
                          Tile{base + (int64_t)(L + 1 - Lbase) * kTileFloats}};
      process_tiles<2>(tl, a, b, lane, st, cp, pv);
      used = 2;
    } else {
      const Tile tl[1] = {Tile{base + (int64_t)(L - Lbase) * kTileFloats}};
      process_tiles<1>(tl, a, b, lane, st, cp, pv);
      used = 1;
    }
    L += used;
    const int bb = b;
    tile_skip(a, b, T, used);
    if (b != bb || L >= Lb) flush_cols(cp, bb, lane, st, pv);
  }
}

// TMEM tiles go to lane quarters in pairs: tile t sits in quarter
// (t / 2) % 4 at slot 2 (t / 8) + t % 2.  Index j of quarter q's tiles:
__host__ __device__ __forceinline__ int tm_tile(int q, int j) { return 8 * (j >> 1) + 2 * q + (j & 1); }
// number of quarter-q tiles below position t
__host__ __device__ __forceinline__ int tm_count(int q, int t) {
  return 2 * (t >> 3) + min(max(t - 8 * (t >> 3) - 2 * q, 0), 2);
}
__host__ __device__ __forceinline__ uint32_t tm_slot(int t) {
  return (uint32_t)(((t >> 3) << 1) | (t & 1));
}

// The warp's TMEM tiles: quarter q's tiles j in [ja, jb), at positions Lt + t.
__device__ __forceinline__ void tmem_tiles(uint32_t tq, int q, int ja, int jb, int a, int b,
                                           int T, int lane, const Step& st, float& pv) {
  if (ja >= jb) return;
  int t = tm_tile(q, ja);
  float2 cp[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) cp[i] = make_float2(0.f, 0.f);
  for (int j = ja; j < jb;) {
    int adv;  // list positions to the quarter's next unprocessed tile
    if ((j & 1) == 0 && j + 1 < jb && a + 1 < T) {
      // tiles t and t + 1: one pair, consecutive rows of one tile column
      const TmemTile tl[2] = {TmemTile{tq + tm_slot(t) * 32u}, TmemTile{tq + tm_slot(t + 1) * 32u}};
      process_tiles<2>(tl, a, b, lane, st, cp, pv);
      j += 2;
      adv = 8;
    } else {
      const TmemTile tl[1] = {TmemTile{tq + tm_slot(t) * 32u}};
      process_tiles<1>(tl, a, b, lane, st, cp, pv);
      adv = (j & 1) ? 7 : 1;
      j += 1;
    }
    const int bb = b;
    tile_skip(a, b, T, adv);
    t += adv;
    if (b != bb || j >= jb) flush_cols(cp, bb, lane, st, pv);
  }
}

// Assemble tile (a, b) of G into its place, 16 columns at a time.
template <class Tile>
__device__ __forceinline__ void assemble_tile(const Tile& tl, const CoreDesc& d, int n, int a,
                                              int b, int lane) {
  const int r = a * kTile + lane;
#pragma unroll
  for (int k16 = 0; k16 < 2; ++k16) {
    float2 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      v[j] = make_float2(core_gram(d, n, r, b * kTile + 16 * k16 + 2 * j),
                         core_gram(d, n, r, b * kTile + 16 * k16 + 2 * j + 1));
    tl.store16(lane, k16, v);
  }
}

template <int kCls>
__global__ void __launch_bounds__(kClass[kCls].warps * 32, kPerSm[kCls])
core_tridiag_kernel(const CoreDesc* __restrict__ descs, int smem_bytes, int n_max,
                    int* __restrict__ status) {
  constexpr int kWarps = kClass[kCls].warps;
  constexpr int kThreads = kWarps * 32;
  constexpr uint32_t kTmemCols = kTmemColsOf[kCls];
  extern __shared__ __align__(16) float smem[];
  const CoreDesc d = descs[blockIdx.x];
  const int n = d.rt + d.k;
  const int npad = (n_max + kTile - 1) / kTile * kTile;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* dv = smem;            // npad: diagonal of T
  float* ev = dv + npad;       // npad: off-diagonal e[j] couples j, j+1
  float* vb0 = ev + npad;      // v of even / odd steps
  float* vb1 = ev + 2 * npad;
  float* pb0 = ev + 3 * npad;  // p of even / odd steps
  float* pb1 = ev + 4 * npad;
  float* wv = ev + 5 * npad;   // w of the pending update
  float* cb0 = ev + 6 * npad;  // column s (rows >= s) / column s + 1
  float* cb1 = ev + 7 * npad;
  float* red = ev + 8 * npad;  // kRed: per-warp partial sums
  float* tsm = red + kRed;     // shared-memory tiles
  const TileLayout Lay = tile_layout(n, kTmemCols, smem_bytes, n_max);
  const int T = Lay.T;
  __shared__ uint32_t s_tmem;
  __shared__ float s_glast;
  __shared__ double s_trace, s_energy_add;

  if (n < 1 || n > n_max || Lay.Lt - Lay.Lg > smem_tile_cap(smem_bytes, n_max) ||
      (Lay.Lg > 0 && d.work == nullptr)) {
    if (tid == 0) atomicOr(status, kStatusBadShape);
    return;
  }
  const bool use_tmem = Lay.Ntm > 0;
  if (use_tmem && wid == 0) tmem_alloc(&s_tmem, kTmemCols);

  // 1. assemble global and shared-memory tiles, the first column, zero vectors
  for (int L = wid; L < Lay.Lt; L += kWarps) {
    int a, b;
    tile_of(L, T, a, b);
    if (L < Lay.Lg) assemble_tile(GlobTile{d.work + (int64_t)L * kTileFloats}, d, n, a, b, lane);
    else assemble_tile(SmemTile{tsm + (int64_t)(L - Lay.Lg) * kTileFloats}, d, n, a, b, lane);
  }
  for (int i = tid; i < npad; i += kThreads) {
    vb0[i] = 0.f;
    vb1[i] = 0.f;
    pb0[i] = 0.f;
    pb1[i] = 0.f;
    wv[i] = 0.f;
    cb0[i] = core_gram(d, n, i, 0);
    cb1[i] = 0.f;
  }
  // ||A||_F^2 = the sum of the column energies (else the Gram's diagonal)
  // when no energy is given
  if (d.energy_add == nullptr) {
    double e = 0.0;
    for (int i = tid; i < d.k; i += kThreads)
      e += d.colE ? d.colE[i] : (double)d.Gaa[(int64_t)i * d.ldb + i];
    e = warp_sum_d(e);
    if (lane == 0) reinterpret_cast<double*>(red)[wid] = e;
  }
  if (tid == 0) s_glast = core_gram(d, n, n - 1, n - 1);
  __syncthreads();
  if (tid == 0 && d.energy_add == nullptr) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += reinterpret_cast<double*>(red)[w];
    s_energy_add = t;
  }
  uint32_t tq = 0;  // TMEM address of this warp's lane quarter
  if (use_tmem) {
    tmem_fence_after();
    const int q = wid & 3;
    tq = s_tmem + ((uint32_t)(q * 32) << 16);
    for (int j = wid >> 2;; j += kWarps / 4) {
      const int t = tm_tile(q, j);
      if (t >= Lay.Ntm) break;
      int a, b;
      tile_of(Lay.Lt + t, T, a, b);
      assemble_tile(TmemTile{tq + tm_slot(t) * 32u}, d, n, a, b, lane);
    }
    tmem_wait_st();
    tmem_fence_before();
  }
  __syncthreads();
  float* pvred = red + 64;  // per-warp p^T v partials of the last main pass
  if (tid < kWarps) pvred[tid] = 0.f;
  __syncthreads();

  // 2. tridiagonalisation (see the file comment for the two phases)
  float tau_prev = 0.f;  // tau of the pending reflector (same in every thread)
  int as_glo = 0, as_ghi = 0, as_slo = 0, as_shi = 0, as_ja = 0, as_jb = 0;  // the warp's share
  int ga = 0, gb = 0, sa = 0, sb = 0, ta = 0, tb = 0;  // and the first tile of each part
  const int Nt = tiles_in(T);
  for (int s = 0;; ++s) {
    const bool odd = (s & 1) != 0;
    float* vcur = odd ? vb1 : vb0;
    const float* vprev = odd ? vb0 : vb1;
    float* pcur = odd ? pb1 : pb0;
    const float* pprev = odd ? pb0 : pb1;
    float* ccur = odd ? cb1 : cb0;
    float* cnext = odd ? cb0 : cb1;
    const bool last = s + 2 >= n;
    const int b0 = (s + 1) >> 5;
    {
      const float pvs = warp_sum(lane < kWarps ? pvred[lane] : 0.f);
      const float kk = (s >= 1) ? 0.5f * tau_prev * tau_prev * pvs : 0.f;
      const float vs = vprev[s];
      const float ws = (s >= 1) ? fmaf(tau_prev, pprev[s], -kk * vs) : 0.f;
      const int ilo = min(s, b0 * kTile);  // rows the main pass of this step touches start here
      float part = 0.f;
      for (int i = ilo + tid; i < npad; i += kThreads) {
        const float vp = vprev[i];
        float w = 0.f;
        if (s >= 1 && i >= s) w = fmaf(tau_prev, pprev[i], -kk * vp);
        wv[i] = w;
        float c = 0.f;
        if (i >= s && i < n) {
          c = fmaf(-vp, ws, fmaf(-w, vs, ccur[i]));
          ccur[i] = c;
          if (i >= s + 2) part = fmaf(c, c, part);
        }
        vcur[i] = (i >= s + 2 && i < n) ? c : 0.f;
        pcur[i] = 0.f;
      }
      part = warp_sum(part);
      if (lane == 0) red[wid] = part;
    }
    __syncthreads();
    const float tail2 = warp_sum(lane < kWarps ? red[lane] : 0.f);  // the same in every lane
    if (last) {
      if (tid == 0) {
        if (n >= 2) {
          const int j = n - 1;
          dv[j - 1] = ccur[j - 1];
          ev[j - 1] = ccur[j];
          dv[j] = fmaf(-2.f * vprev[j], wv[j], s_glast);
        } else {
          dv[0] = ccur[0];
        }
        ev[n - 1] = 0.f;
      }
      break;
    }
    const float x0 = ccur[s + 1];
    float beta = x0, tau = 0.f, v0 = 0.f;
    if (tail2 != 0.f) {
      const float nrm = sqrtf(fmaf(x0, x0, tail2));
      beta = x0 >= 0.f ? -nrm : nrm;
      v0 = x0 - beta;
      tau = 2.f / fmaf(v0, v0, tail2);
    }
    if (tid == 0) {
      dv[s] = ccur[s];
      ev[s] = beta;
    }
    if (lane == 0) vcur[s + 1] = v0;  // every warp writes the same value
    __syncwarp();
    tau_prev = tau;
    if (use_tmem) tmem_fence_after();

    // main pass over the trailing tiles (tile columns >= b0); the warp's
    // share changes only when b0 does
    if (s == 0 || ((s + 1) & 31) == 0) {
      const int L0 = col_start(b0, T);
      const int ng = max(0, Lay.Lg - L0);  // trailing tiles in global memory
      const int Ls0 = max(L0, Lay.Lg);
      const int ns = max(0, Lay.Lt - Ls0);  // ... in shared memory
      const int t0 = max(L0, Lay.Lt) - Lay.Lt;  // first trailing TMEM tile
      // TMEM tiles of quarter q, split evenly among its warps
      constexpr int kPerQ = kWarps / 4;
      const int q = wid & 3, qi = wid >> 2;
      const int j0 = tm_count(q, t0), nq = tm_count(q, Lay.Ntm) - j0;
      as_ja = j0 + qi * nq / kPerQ;
      as_jb = j0 + (qi + 1) * nq / kPerQ;
      int s_lo, s_hi;
      if (Lay.Ntm - t0 <= 0) {
        s_lo = ns * wid / kWarps;
        s_hi = ns * (wid + 1) / kWarps;
      } else {
        // shared-memory tiles top every warp up to the same level
        int cu = 0;
        if (lane < kWarps) {
          const int lq = lane & 3, lqi = lane >> 2;
          const int lj0 = tm_count(lq, t0), ln = tm_count(lq, Lay.Ntm) - lj0;
          cu = (lqi + 1) * ln / kPerQ - lqi * ln / kPerQ;
        }
        const int ntm = Lay.Ntm - t0;
        int lam = (ns + ntm + kWarps - 1) / kWarps;
        for (;;) {
          const int dd = (lane < kWarps) ? max(0, lam - cu) : 0;
          if ((int)__reduce_add_sync(0xffffffffu, (unsigned)dd) >= ns) break;
          ++lam;
        }
        const int dmine = (lane < kWarps) ? max(0, lam - cu) : 0;
        const int before =
            (int)__reduce_add_sync(0xffffffffu, (unsigned)(lane < wid ? dmine : 0));
        const int mine = __shfl_sync(0xffffffffu, dmine, wid);
        s_lo = min(before, ns);
        s_hi = min(ns, before + mine);
      }
      as_slo = Ls0 + s_lo;
      as_shi = Ls0 + s_hi;
      // global tiles: an even share each; half the warps take them first
      as_glo = L0 + ng * wid / kWarps;
      as_ghi = L0 + ng * (wid + 1) / kWarps;
      // first tile of each share (unchanged until b0 moves)
      tile_of(min(as_glo, Nt - 1), T, ga, gb);
      tile_of(min(as_slo, Nt - 1), T, sa, sb);
      tile_of(min(Lay.Lt + tm_tile(q, as_ja), Nt - 1), T, ta, tb);
    }
    {
      const Step st{vcur, vprev, wv, pcur, cnext, &s_glast, b0, (s + 1) & 31, s + 1, n - 1, v0};
      const int g_lo = as_glo, g_hi = as_ghi;
      float pv = 0.f;
      if ((wid & 1) == 0) mem_tiles<GlobTile>(d.work, 0, g_lo, g_hi, ga, gb, T, lane, st, pv);
      mem_tiles<SmemTile>(tsm, Lay.Lg, as_slo, as_shi, sa, sb, T, lane, st, pv);
      if (use_tmem) {
        tmem_tiles(tq, wid & 3, as_ja, as_jb, ta, tb, T, lane, st, pv);
        tmem_wait_st();
      }
      if ((wid & 1) != 0) mem_tiles<GlobTile>(d.work, 0, g_lo, g_hi, ga, gb, T, lane, st, pv);
      pv = warp_sum(pv);
      if (lane == 0) pvred[wid] = pv;
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
  for (int i = tid; i < n; i += kThreads) {
    const float el = i > 0 ? fabsf(ev[i - 1]) : 0.f;
    const float er = i + 1 < n ? fabsf(ev[i]) : 0.f;
    lo = fminf(lo, dv[i] - el - er);
    hi = fmaxf(hi, dv[i] + el + er);
    emax = fmaxf(emax, er * er);
    tr += (double)dv[i];
  }
  __shared__ float s_lo[kWarps], s_hi[kWarps], s_em[kWarps];
  __shared__ double s_tr[kWarps];
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
  for (int w = 1; w < kWarps; ++w) {
    glo = fminf(glo, s_lo[w]);
    ghi = fmaxf(ghi, s_hi[w]);
    gem = fmaxf(gem, s_em[w]);
    gtr += s_tr[w];
  }
  float* e2 = vb0;  // reuse
  float* lam = pb0;
  for (int i = tid; i < n; i += kThreads) e2[i] = (i + 1 < n) ? ev[i] * ev[i] : 0.f;
  if (tid == 0) s_trace = gtr;
  __syncthreads();

  // 4. multisection bisection for the top r_new eigenvalues
  const float gnorm = fmaxf(fabsf(glo), fabsf(ghi));
  const float pivmin = 1.0e-30f * fmaxf(1.f, gem);
  // each eigenvalue to a few units in its own last place (the top-r sum
  // then carries no bisection error beyond the Sturm counts' own), with an
  // absolute floor far below the FP32 accuracy of the reduction
  const float atol = 1e-12f * gnorm + 1e-30f;
  const int rq = d.r_new;
  int g = 1;
  while (g < 16 && g * 2 * rq <= kThreads) g *= 2;
  const int ngroups = kThreads / g;
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
    const int cap = d_bisect_cap;
    for (; it < cap; ++it) {
      // every lane of the warp runs the same number of iterations
      const bool done = !active || stuck || !((b - a) > fmaxf(atol, 2.4e-7f * fmaxf(fabsf(a), fabsf(b))));
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
    if (active && it == cap) capped = 1;
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
      if (d.refine) {
        const bool mark = d.refine_near
                              ? fabs(tail - d.eps * d.eps * energy_new) <= kDecisionBand * energy_new
                              : tail < kRefineFrac * energy_new;
        d.refine[0] = mark ? 1 : 0;
      }
    }
  }
}

}  // namespace

cudaError_t tridiag_set_bisect_cap(int cap) {
  if (cap < 0) cap = kBisectMax;
  return cudaMemcpyToSymbol(d_bisect_cap, &cap, sizeof(int));
}

// Launch-class edges: cores of size n <= edge0 take class 0, n <= edge1
// class 1, larger ones class 2 (defaults kClass[0..1].max_n; set by the
// autotuner within [kEdgeMin, kEdgeMax[c]]).
static std::atomic<int> g_edge0{kClass[0].max_n}, g_edge1{kClass[1].max_n};

bool tridiag_set_edges(int e0, int e1) {
  if (e0 < 0 && e1 < 0) {
    g_edge0 = kClass[0].max_n;
    g_edge1 = kClass[1].max_n;
    return true;
  }
  if (e0 < kEdgeMin || e0 > kEdgeMax[0] || e1 <= e0 || e1 > kEdgeMax[1]) return false;
  g_edge0 = e0;
  g_edge1 = e1;
  return true;
}

void tridiag_get_edges(int* e0, int* e1) {
  *e0 = g_edge0;
  *e1 = g_edge1;
}

int tridiag_class(int n) {
  if (n <= g_edge0) return 0;
  if (n <= g_edge1) return 1;
  return 2;
}

int tridiag_smem_bytes(int cls, int n_max) {
  if (cls == 2) return kTriLargeSmemBytes;
  // at most the class's SM share of shared memory, less when the cores are small
  const int share = (cls == 0) ? 56 * 1024 : 112 * 1024;
  const int npad = (n_max + kTile - 1) / kTile * kTile;
  const int T = npad / kTile;
  const int need_tiles = max(0, tiles_in(T) - kTmemColsOf[cls] / 8);
  const int need = (kVecs * npad + kRed + need_tiles * kTileFloats) * 4;
  return min(need, share);
}

int64_t tridiag_work_floats(int cls, int n, int n_max) {
  return (int64_t)tile_layout(n, kTmemColsOf[cls], tridiag_smem_bytes(cls, n_max), n_max).Lg *
         kTileFloats;
}

template <int kCls>
static cudaError_t launch_class(const CoreDesc* d_desc, int n_items, int smem_bytes, int n_max,
                                int* d_status, cudaStream_t s) {
  static std::atomic<int> set_smem{0};
  if (cudaError_t e = ensure_smem(core_tridiag_kernel<kCls>, smem_bytes, set_smem)) return e;
  prof_begin(s);
  core_tridiag_kernel<kCls><<<n_items, kClass[kCls].warps * 32, smem_bytes, s>>>(
      d_desc, smem_bytes, n_max, d_status);
  prof_end(kCls == 0 ? "core_tridiag.small" : kCls == 1 ? "core_tridiag.medium"
                                                        : "core_tridiag.large", s);
  return cudaGetLastError();
}

// Host-side checks of the launch planning (no GPU): the tile placement of
// every class and core size partitions the tile list within the TMEM and
// shared-memory capacities, the list walk agrees with its closed forms, and
// the dynamic shared memory of every launch fits a CTA.  Returns an empty
// string or the first failure.
std::string tridiag_selftest() {
  char buf[256];
  int e0, e1;
  tridiag_get_edges(&e0, &e1);
  for (int n = 1; n <= 1024; ++n) {
    const int cls = tridiag_class(n);
    if ((n <= e0) != (cls == 0) || (n > e0 && n <= e1) != (cls == 1))
      return "launch class of n = " + std::to_string(n);
  }
  // every core size a class can receive under any tunable edges
  for (int n = 1; n <= 1536; ++n) for (int cls = 0; cls < 3; ++cls) {
    const int class_max = cls == 0 ? kEdgeMax[0] : cls == 1 ? kEdgeMax[1] : 1536;
    const int class_min = cls == 0 ? 1 : kEdgeMin + 1;
    if (n < class_min || n > class_max) continue;
    for (int n_max = n; n_max <= class_max; n_max += (cls == 2 ? 5 : 1)) {
      const int smem = tridiag_smem_bytes(cls, n_max);
      if (smem <= 0 || smem > 227 * 1024) {
        snprintf(buf, sizeof buf, "shared memory %d B for class %d, n_max %d", smem, cls, n_max);
        return buf;
      }
      const TileLayout L = tile_layout(n, kTmemColsOf[cls], smem, n_max);
      const int nt = tiles_in(L.T);
      // shared memory holds kVecs padded vectors, the reduction buffer and
      // the shared tiles; TMEM holds 128 lanes x its columns f32 cells
      const int64_t npad = (n_max + kTile - 1) / kTile * kTile;
      const int64_t smem_need =
          4 * ((int64_t)kVecs * npad + kRed + (int64_t)(L.Lt - L.Lg) * kTileFloats);
      const bool ok = L.T == (n + kTile - 1) / kTile && 0 <= L.Lg && L.Lg <= L.Lt &&
                      L.Lt <= nt && L.Ntm == nt - L.Lt &&
                      (int64_t)L.Ntm * kTileFloats <= 128LL * kTmemColsOf[cls] &&
                      smem_need <= smem &&
                      tridiag_work_floats(cls, n, n_max) == (int64_t)L.Lg * kTileFloats;
      bool col_boundary = false;
      for (int g = 0; g <= L.T; ++g) col_boundary |= col_start(g, L.T) == L.Lg;
      if (!ok || !col_boundary) {
        snprintf(buf, sizeof buf, "tile layout n = %d, class %d, n_max %d: T %d Lg %d Lt %d Ntm %d",
                 n, cls, n_max, L.T, L.Lg, L.Lt, L.Ntm);
        return buf;
      }
    }
  }
  // TMEM tile placement: every tile of [0, Ntm) in exactly one lane quarter,
  // at a slot of that quarter below its capacity, indices consistent both ways
  for (int cls = 0; cls < 3; ++cls) {
    const int slots = kTmemColsOf[cls] / 32;
    for (int ntm = 0; ntm <= 4 * slots; ++ntm) {
      int total = 0;
      for (int q = 0; q < 4; ++q) {
        const int cnt = tm_count(q, ntm);
        total += cnt;
        unsigned used = 0;
        for (int j = 0; j < cnt; ++j) {
          const int t = tm_tile(q, j);
          const uint32_t sl = tm_slot(t);
          if (t < 0 || t >= ntm || ((t >> 1) & 3) != q || tm_count(q, t) != j ||
              sl >= (uint32_t)slots || ((used >> sl) & 1u)) {
            snprintf(buf, sizeof buf, "TMEM placement class %d, %d tiles, quarter %d, index %d",
                     cls, ntm, q, j);
            return buf;
          }
          used |= 1u << sl;
        }
      }
      if (total != ntm) {
        snprintf(buf, sizeof buf, "TMEM placement class %d covers %d of %d tiles", cls, total, ntm);
        return buf;
      }
    }
  }
  for (int T = 1; T <= 48; ++T) {
    const int nt = tiles_in(T);
    int a = 0, b = 0;
    for (int L = 0; L < nt; ++L) {
      int a2, b2;
      tile_of(L, T, a2, b2);
      if (a2 != a || b2 != b || a < b || a >= T || col_start(b, T) + (a - b) != L) {
        snprintf(buf, sizeof buf, "tile list walk T = %d at %d", T, L);
        return buf;
      }
      for (int k = 0; L + k < nt; k += 1 + k / 3) {
        int a3 = a, b3 = b, a4, b4;
        tile_skip(a3, b3, T, k);
        tile_of(L + k, T, a4, b4);
        if (a3 != a4 || b3 != b4) {
          snprintf(buf, sizeof buf, "tile skip T = %d from %d by %d", T, L, k);
          return buf;
        }
      }
      tile_next(a, b, T);
    }
  }
  return "";
}

cudaError_t launch_core_tridiag(int cls, const CoreDesc* d_desc, int n_items, int n_max,
                                int* d_status, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const int smem = tridiag_smem_bytes(cls, n_max);
  if (cls == 0) return launch_class<0>(d_desc, n_items, smem, n_max, d_status, s);
  if (cls == 1) return launch_class<1>(d_desc, n_items, smem, n_max, d_status, s);
  return launch_class<2>(d_desc, n_items, smem, n_max, d_status, s);
}

}  // namespace csvd
