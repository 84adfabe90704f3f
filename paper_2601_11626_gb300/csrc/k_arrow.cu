// One-column merge evaluations (k = 1) in the mixed form.
//
// With a single new column a, the Gram of the core (Lemma 1) is an arrowhead
//     G = [[diag(d), z], [z^T, alpha]],  d_j = s_j^2, z_j = s_j p_j,
//     p = U^T a, alpha = ||a||^2   (n = r_t + 1),
// whose eigenvalues are the squared singular values of the merge.  For x off
// the poles d_j, G - xI has as many negative eigenvalues as diag(d) - xI
// plus the sign of its Schur complement, so
//     #{lambda < x} = #{j : d_j < x} + [f(x) < 0],
//     f(x) = alpha - x - sum_j z_j^2 / (d_j - x)   (the secular function),
// an exact O(r_t) count.  The top r_new eigenvalues give sigma~_j =
// sqrt(lambda_j) (Cor. 3); when the merge truncates (r_new = r_t), the one
// discarded eigenvalue is found the same way and is the step's tail, each
// root to a few units in its own last place.
//
// diag(d) is the leading principal block of G, so (Cauchy interlacing) with
// s non-increasing the q-th largest eigenvalue lies in [d_q, d_{q-1}] (ends
// closed by the Gershgorin interval).  Inside that bracket no pole lies
// between x and the root, the count is (r_t - q) + [f(x) < 0], and f is
// decreasing; each evaluation narrows the bracket by the sign of f and
// proposes the next point from a rational model fitted to f and f' at x:
//   interior brackets: one pole (the end nearer the bracket's centre),
//     f ~ A + B / (pole - y)                       -> y = pole + B / A;
//   end brackets (no pole beyond the top / below the bottom eigenvalue):
//     f ~ C - y - E / (pole - y), linear term kept -> a quadratic in y.
// A proposal outside the bracket is replaced by the midpoint; once proposals
// have run kArrowModelIters times the rest is plain bisection, so every
// eigenvalue ends within 16 + 24 evaluations.  States whose sigma is not
// sorted fall back to multisection bisection on the full count over the
// Gershgorin interval.
//
// One 128-thread CTA per group of up to kArrowGroup candidates of the same
// state.  The group's columns are staged in shared memory 512 rows at a time
// (all loads of a pass in flight together), so every row of U read from L2
// serves the whole group; with 16-byte rows of U a lane reads 4 columns at
// once.  ||a||^2 is accumulated per thread as a compensated FP32 pair.  Two
// entry kernels fill the group's view (a descriptor per candidate, or
// candidates as the rows of one matrix with outputs indexed by row) and
// share the body.
#include "common.cuh"

namespace csvd {
namespace {

constexpr int kArrowThreads = 128;
constexpr int kArrowWarps = kArrowThreads / 32;
constexpr int kArrowBisectMax = 64;
__device__ int d_arrow_cap = kArrowBisectMax;  // lowered only by the failure-path test hook
constexpr int kArrowModelIters = 16;
constexpr int kArrowStage = 512;  // rows of the group's columns staged per pass
constexpr int kArrowPerThread = kArrowStage / kArrowThreads;
static_assert(kArrowGroup == 4, "rows of the group are staged as float4");
static_assert(kArrowGroup <= kArrowWarps, "one warp per candidate in the per-item steps");

__device__ __forceinline__ int arrow_count(const float* d, const float* z2, int rt, float alpha,
                                           float x, float pivmin) {
  int c = 0;
  float s = alpha - x;
  for (int j = 0; j < rt; ++j) {
    float q = d[j] - x;
    c += q < 0.f;
    if (fabsf(q) < pivmin) q = q < 0.f ? -pivmin : pivmin;
    s -= __fdividef(z2[j], q);
  }
  return c + (s < 0.f);
}

// s + c += v^2 with the square split exactly (v^2 = p + e) and the sum
// compensated (Knuth's two-sum): a double-float accumulator in FP32 pipes.
__device__ __forceinline__ void arrow_acc_sq(float& s, float& c, float v) {
  const float p = v * v;
  const float e = fmaf(v, v, -p);
  const float t = s + p;
  const float bp = t - s;
  c += ((s - (t - bp)) + (p - bp)) + e;
  s = t;
}

// (s, c) += (s2, c2) for double-float pairs (two-sum of the heads).
__device__ __forceinline__ void arrow_ff_add(float& s, float& c, float s2, float c2) {
  const float t = s + s2;
  const float bp = t - s;
  c += c2 + ((s - (t - bp)) + (s2 - bp));
  s = t;
}

// Warp sum of double-float pairs; every lane gets the total.
__device__ __forceinline__ void arrow_ff_warp_sum(float& s, float& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    arrow_ff_add(s, c, s2, c2);
  }
}

// Root t of t^2 - h t - E = 0 (E >= 0): the non-negative one if `positive`,
// else the non-positive one, each in a form free of cancellation.
__device__ __forceinline__ float arrow_quad_root(float h, float E, bool positive) {
  const float sq = sqrtf(fmaf(h, h, 4.f * E));
  if (positive) return h >= 0.f ? 0.5f * (h + sq) : __fdividef(2.f * E, sq - h);
  return h <= 0.f ? 0.5f * (h - sq) : __fdividef(-2.f * E, sq + h);
}

// What one CTA evaluates: a state and up to kArrowGroup candidates of it.
struct ArrowGroupView {
  const float* U;
  const float* sigma;
  const double* scal;
  int64_t ldu, m;
  int rt, rq, cnt;
  double eps;
  const float* a[kArrowGroup];
  int64_t lda[kArrowGroup];
  float* sigma_out[kArrowGroup];
  double* tail_out[kArrowGroup];
  double* paper_out[kArrowGroup];   // may be null
  double* energy_out[kArrowGroup];  // may be null
  uint8_t* accept_out[kArrowGroup]; // may be null
};

__device__ __forceinline__ void arrow_group(const ArrowGroupView& V, int* __restrict__ status) {
  const int cnt = V.cnt;
  const int rt = V.rt, n = rt + 1, rq = V.rq;
  const int64_t m = V.m, ldu = V.ldu;
  const float* __restrict__ U = V.U;
  const float* __restrict__ sigma = V.sigma;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  __shared__ float4 s_a[kArrowStage];
  __shared__ float s_part[kArrowWarps][kArrowGroup][32];
  __shared__ float s_d[kArrowMaxRt];
  __shared__ float s_z2[kArrowGroup][kArrowMaxRt];
  __shared__ float2 s_dz[kArrowGroup][kArrowMaxRt];  // {d_j, z_j^2}
  __shared__ float s_lam[kArrowGroup][kArrowMaxRt + 1];
  __shared__ float s_lo[kArrowGroup], s_hi[kArrowGroup];
  __shared__ float2 s_red[kArrowWarps][kArrowGroup];
  __shared__ double s_alpha[kArrowGroup];

  const float* ap[kArrowGroup];
  int64_t lda[kArrowGroup];
#pragma unroll
  for (int g = 0; g < kArrowGroup; ++g) {
    ap[g] = g < cnt ? V.a[g] : nullptr;
    lda[g] = g < cnt ? V.lda[g] : 0;
  }

  // 1. p = U^T a for every candidate and ||a||^2 (double-float pairs).  The
  //    r_t columns of U are cut into 32-wide slabs, one per warp; warps left
  //    over split the rows of each staged chunk between them.
  const int nslab = (rt + 31) / 32;
  const int nrg = nslab > 0 ? kArrowWarps / nslab : 1;
  const int slab = nslab > 0 ? wid % nslab : 0, rg = nslab > 0 ? wid / nslab : wid;
  const int col = slab * 32 + lane;
  const bool pj_on = nslab > 0 && rg < nrg && col < rt;
  // 16-byte rows of U: a lane reads 4 columns at once (lane % 8 picks the
  // column quad of the slab, lane / 8 the row within a block of 4 rows;
  // blocks of 4 rows go round-robin to the row groups) and keeps 4 x 4
  // sums; otherwise a lane reads one column and keeps acc[g][0]
  const bool vec = (ldu & 3) == 0 && (reinterpret_cast<uintptr_t>(U) & 15) == 0;
  const int quad = lane & 7, rsub = lane >> 3;
  const bool quad_on = nslab > 0 && rg < nrg && slab * 32 + 4 * quad < rt;
  float acc[kArrowGroup][4] = {};
  float es[kArrowGroup] = {}, ec[kArrowGroup] = {};
  for (int64_t i0 = 0; i0 < m; i0 += kArrowStage) {
    const int len = (int)(m - i0 < kArrowStage ? m - i0 : kArrowStage);
    // every load of the pass is issued before any is used
    float v[kArrowPerThread][kArrowGroup];
#pragma unroll
    for (int k = 0; k < kArrowPerThread; ++k) {
      const int ii = tid + k * kArrowThreads;
#pragma unroll
      for (int g = 0; g < kArrowGroup; ++g)
        v[k][g] = (g < cnt && ii < len) ? ap[g][(i0 + ii) * lda[g]] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kArrowPerThread; ++k) {
      s_a[tid + k * kArrowThreads] = make_float4(v[k][0], v[k][1], v[k][2], v[k][3]);
#pragma unroll
      for (int g = 0; g < kArrowGroup; ++g) arrow_acc_sq(es[g], ec[g], v[k][g]);
    }
    __syncthreads();
    if (vec) {
      if (quad_on) {
        const float* u = U + i0 * ldu + slab * 32 + 4 * quad;
#pragma unroll 4
        for (int ii = 4 * rg + rsub; ii < len; ii += 4 * nrg) {
          const float4 uu = __ldg(reinterpret_cast<const float4*>(u + (int64_t)ii * ldu));
          const float4 x = s_a[ii];
          const float xs[kArrowGroup] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int g = 0; g < kArrowGroup; ++g) {
            acc[g][0] = fmaf(uu.x, xs[g], acc[g][0]);
            acc[g][1] = fmaf(uu.y, xs[g], acc[g][1]);
            acc[g][2] = fmaf(uu.z, xs[g], acc[g][2]);
            acc[g][3] = fmaf(uu.w, xs[g], acc[g][3]);
          }
        }
      }
    } else if (pj_on) {
      const float* u = U + i0 * ldu + col;
#pragma unroll 16
      for (int ii = rg; ii < len; ii += nrg) {
        const float uu = __ldg(u + (int64_t)ii * ldu);
        const float4 x = s_a[ii];
        acc[0][0] = fmaf(uu, x.x, acc[0][0]);
        acc[1][0] = fmaf(uu, x.y, acc[1][0]);
        acc[2][0] = fmaf(uu, x.z, acc[2][0]);
        acc[3][0] = fmaf(uu, x.w, acc[3][0]);
      }
    }
    __syncthreads();
  }
  if (vec) {  // sum the 4 row lanes of each column quad
#pragma unroll
    for (int g = 0; g < kArrowGroup; ++g)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[g][c] += __shfl_xor_sync(0xffffffffu, acc[g][c], 8);
        acc[g][c] += __shfl_xor_sync(0xffffffffu, acc[g][c], 16);
      }
  }
#pragma unroll
  for (int g = 0; g < kArrowGroup; ++g) {
    if (!vec) {
      s_part[wid][g][lane] = acc[g][0];
    } else if (rsub == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) s_part[wid][g][4 * quad + c] = acc[g][c];
    }
    arrow_ff_warp_sum(es[g], ec[g]);
    if (lane == 0) s_red[wid][g] = make_float2(es[g], ec[g]);
  }
  __syncthreads();
  if (tid < kArrowGroup) {
    double t = 0.0;
    for (int w = 0; w < kArrowWarps; ++w) t += (double)s_red[w][tid].x + (double)s_red[w][tid].y;
    s_alpha[tid] = t;
  }
  bool sorted_ok = true;
  if (tid < rt) {
    const int sl = tid / 32, ln = tid % 32;
    const float sj = sigma[tid];
    s_d[tid] = sj * sj;
    if (tid + 1 < rt) sorted_ok = sj >= sigma[tid + 1];
#pragma unroll
    for (int g = 0; g < kArrowGroup; ++g) {
      float p = 0.f;
      for (int r2 = 0; r2 < nrg; ++r2) p += s_part[r2 * nslab + sl][g][ln];
      const float zj = sj * p;
      s_z2[g][tid] = zj * zj;
      s_dz[g][tid] = make_float2(sj * sj, zj * zj);
    }
  }
  const bool sorted = __syncthreads_and(sorted_ok);

  // 2. Gershgorin interval of each arrowhead (warp g <-> candidate g)
  if (wid < cnt) {
    const float alpha = (float)s_alpha[wid];
    float lo = alpha, hi = alpha, zsum = 0.f;
    for (int j = lane; j < rt; j += 32) {
      const float zj = sqrtf(s_z2[wid][j]);
      lo = fminf(lo, s_d[j] - zj);
      hi = fmaxf(hi, s_d[j] + zj);
      zsum += zj;
    }
    zsum = warp_sum(zsum);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      s_lo[wid] = fminf(lo, alpha - zsum);
      s_hi[wid] = fmaxf(hi, alpha + zsum);
    }
  }
  __syncthreads();

  // 3. one task per (candidate, eigenvalue): the top rq and, when the merge
  //    truncates, the discarded one (n - rq <= 1 for one column)
  const int nroot = n;
  const int ntask = cnt * nroot;
  int capped = 0;
  if (sorted) {
    // bracketed rational-model iteration, one thread per task
    for (int t0 = 0; t0 < ntask; t0 += kArrowThreads) {  // uniform trip count
      const int t = t0 + tid;
      const bool active = t < ntask;
      const int item = active ? t / nroot : 0, q = active ? t % nroot : 0;
      const float glo = s_lo[item], ghi = s_hi[item];
      const float gnorm = fmaxf(fabsf(glo), fabsf(ghi));
      const float pivmin = 1.0e-30f * fmaxf(1.f, gnorm);
      // each root to a few units in its own last place (the discarded one
      // is the tail itself), with an absolute floor far below FP32 accuracy
      const float afloor = 1e-12f * gnorm + 1e-30f;
      const float alpha = (float)s_alpha[item];
      const float2* dz = s_dz[item];
      const bool has_l = q < rt, has_r = q > 0;
      const float dl = has_l ? s_d[q] : 0.f, dr = has_r ? s_d[q - 1] : 0.f;
      float a = has_l ? fmaxf(glo, dl) : glo, b = has_r ? fminf(ghi, dr) : ghi;
      if (a > b) a = b;
      float x = 0.5f * (a + b), lam = x;
      float atol = fmaxf(afloor, 2.4e-7f * fmaxf(fabsf(a), fabsf(b)));
      bool done = !active || !((b - a) > atol);
      bool probed = false;
      int it = 0;
      const int cap = d_arrow_cap;
      for (; it < cap; ++it) {
        if (__all_sync(0xffffffffu, done)) break;
        if (done) continue;
        float f = alpha - x, D = 0.f;
        for (int j = 0; j < rt; ++j) {
          const float2 e = dz[j];
          const float qq = copysignf(fmaxf(fabsf(e.x - x), pivmin), e.x - x);
          const float inv = __fdividef(1.f, qq);
          const float tt = e.y * inv;
          f -= tt;
          D = fmaf(tt, inv, D);
        }
        if (f < 0.f) b = x; else a = x;  // x above the root iff f(x) < 0
        atol = fmaxf(afloor, 2.4e-7f * fmaxf(fabsf(a), fabsf(b)));
        if (!((b - a) > atol)) {
          done = true;
          lam = x;
          continue;
        }
        float delta = 0.f;
        bool have = false;
        if (it < kArrowModelIters && (has_l || has_r)) {
          if (has_l && has_r) {
            const float mid = 0.5f * (a + b);
            const float pole = (mid - dl < dr - mid) ? dl : dr;
            const float fp = -1.f - D;
            const float dx = pole - x;
            const float A = fmaf(-fp, dx, f), B = fp * dx * dx;
            if (A != 0.f) {
              delta = dx + __fdividef(B, A);
              have = true;
            }
          } else {
            const float pole = has_l ? dl : dr;
            const float dx = pole - x;
            const float E = D * dx * dx;
            const float C = f + x + __fdividef(E, dx);
            delta = dx + arrow_quad_root(C - pole, E, has_l);
            have = true;
          }
        }
        if (have && fabsf(delta) <= 0.5f * atol) {
          done = true;
          lam = x + delta;
          continue;
        }
        float y = x + delta;
        if (have && !probed && y <= a) {
          y = a + fminf(0.5f * (b - a), 0.5f * atol);
          probed = true;
        } else if (have && !probed && y >= b) {
          y = b - fminf(0.5f * (b - a), 0.5f * atol);
          probed = true;
        }
        if (!have || !(y > a && y < b)) y = 0.5f * (a + b);
        x = y;
      }
      if (active && !done) {  // ran out of iterations (cap) without converging
        capped = 1;
        lam = 0.5f * (a + b);
      }
      if (active) s_lam[item][q] = lam;
    }
  } else {
    // multisection bisection on the full count, g threads per task
    int g = 1;
    while (g < 16 && g * 2 * ntask <= kArrowThreads) g *= 2;
    const int ngroups = kArrowThreads / g;
    const int grp = tid / g, sub = tid % g;
    const unsigned shift = (unsigned)((lane / g) * g);
    const unsigned gmask = ((1u << g) - 1u) << shift;
    for (int t0 = 0; t0 < ntask; t0 += ngroups) {  // uniform trip count across the block
      const int t = t0 + grp;
      const bool active = t < ntask;
      const int item = active ? t / nroot : 0, q = active ? t % nroot : 0;
      const int target = n - 1 - q;  // ascending index of the q-th largest
      const float glo = s_lo[item], ghi = s_hi[item];
      const float gnorm = fmaxf(fabsf(glo), fabsf(ghi));
      const float pivmin = 1.0e-30f * fmaxf(1.f, gnorm);
      const float afloor = 1e-12f * gnorm + 1e-30f;
      const float alpha = (float)s_alpha[item];
      const float* z2 = s_z2[item];
      float a = glo, b = ghi;
      bool stuck = false;
      int it = 0;
      const int cap = d_arrow_cap;
      for (; it < cap; ++it) {
        const float atol = fmaxf(afloor, 2.4e-7f * fmaxf(fabsf(a), fabsf(b)));
        const bool done = !active || stuck || !((b - a) > atol);
        if (__all_sync(0xffffffffu, done)) break;
        const float step = (b - a) / (float)(g + 1);
        const float x = a + step * (float)(sub + 1);
        bool above = false;
        if (!done)
          above = (x > a && x < b) ? (arrow_count(s_d, z2, rt, alpha, x, pivmin) > target)
                                   : (x >= b);
        const unsigned bal = (__ballot_sync(0xffffffffu, above) & gmask) >> shift;
        if (!done) {
          const int s = bal ? __ffs(bal) - 1 : g;
          const float na = (s == 0) ? a : a + step * (float)s;
          const float nb = (s == g) ? b : a + step * (float)(s + 1);
          if (!(nb < b || na > a)) stuck = true;
          a = na;
          b = nb;
        }
      }
      if (active && it == cap) capped = 1;
      if (active && sub == 0) s_lam[item][q] = 0.5f * (a + b);
    }
  }
  if (capped) atomicOr(status, kStatusBisectCap);
  __syncthreads();

  // 4. FP64 epilogue (warp g <-> candidate g): sigma~, the tail as the
  //    discarded eigenvalue itself (no difference of sums as large as
  //    ||M||^2), energy, accept flag
  if (wid < cnt) {
    const double alpha_d = s_alpha[wid];
    float* sig_out = V.sigma_out[wid];
    float ts = 0.f, tc = 0.f;  // double-float sum of the top
    for (int q = lane; q < rq; q += 32) {
      arrow_ff_add(ts, tc, s_lam[wid][q], 0.f);
      sig_out[q] = sqrtf(fmaxf(s_lam[wid][q], 0.f));
    }
    arrow_ff_warp_sum(ts, tc);
    if (lane == 0) {
      const double top = (double)ts + (double)tc;
      double disc = 0.0;
      for (int q = rq; q < nroot; ++q) disc += (double)fmaxf(s_lam[wid][q], 0.f);
      const double energy_new = V.scal[0] + alpha_d;
      double tail = V.scal[1] + disc;
      if (tail < 0.0) tail = 0.0;
      double paper = energy_new - top;
      if (paper < 0.0) paper = 0.0;
      V.tail_out[wid][0] = tail;
      if (V.paper_out[wid]) V.paper_out[wid][0] = paper;
      if (V.energy_out[wid]) V.energy_out[wid][0] = energy_new;
      if (V.accept_out[wid]) V.accept_out[wid][0] = (tail <= V.eps * V.eps * energy_new) ? 1 : 0;
    }
  }
}

}  // namespace

cudaError_t arrow_set_cap(int cap) {
  if (cap < 0) cap = kArrowBisectMax;
  return cudaMemcpyToSymbol(d_arrow_cap, &cap, sizeof(int));
}

// A descriptor per candidate; group = {first descriptor, count}.
__global__ void __launch_bounds__(kArrowThreads, 7)
core_arrow_kernel(const ArrowDesc* __restrict__ descs, const int2* __restrict__ groups,
                  int* __restrict__ status) {
  __shared__ ArrowGroupView V;
  const int2 gr = groups[blockIdx.x];
  const int t = threadIdx.x;
  if (t == 0) {
    const ArrowDesc& d = descs[gr.x];
    V.U = d.U;
    V.sigma = d.sigma;
    V.scal = d.scal;
    V.ldu = d.ldu;
    V.m = d.m;
    V.rt = d.rt;
    V.rq = d.r_new;
    V.cnt = gr.y;
    V.eps = d.eps;
  }
  if (t < kArrowGroup) {
    const bool on = t < gr.y;
    const ArrowDesc* d = on ? descs + gr.x + t : nullptr;
    V.a[t] = on ? d->a : nullptr;
    V.lda[t] = on ? d->lda : 0;
    V.sigma_out[t] = on ? d->sigma_out : nullptr;
    V.tail_out[t] = on ? d->tail_out : nullptr;
    V.paper_out[t] = on ? d->tail_paper_out : nullptr;
    V.energy_out[t] = on ? d->energy_out : nullptr;
    V.accept_out[t] = on ? d->accept_out : nullptr;
  }
  __syncthreads();
  arrow_group(V, status);
}

// Candidates as rows of Xt; group = {first row, count, state, unused}.
__global__ void __launch_bounds__(kArrowThreads, 7)
core_arrow_columns_kernel(const ArrowState* __restrict__ states, const int4* __restrict__ groups,
                          const float* __restrict__ Xt, int64_t ldx, float* sigma_out,
                          int64_t ld_sigma, double* tail_out, double* paper_out,
                          uint8_t* accept_out, double eps, int* __restrict__ status) {
  __shared__ ArrowGroupView V;
  const int4 gr = groups[blockIdx.x];
  const int t = threadIdx.x;
  if (t == 0) {
    const ArrowState& st = states[gr.z];
    V.U = st.U;
    V.sigma = st.sigma;
    V.scal = st.scal;
    V.ldu = st.ldu;
    V.m = st.m;
    V.rt = st.rt;
    V.rq = st.r_new;
    V.cnt = gr.y;
    V.eps = eps;
  }
  if (t < kArrowGroup) {
    const bool on = t < gr.y;
    const int64_t j = (int64_t)gr.x + t;
    V.a[t] = on ? Xt + j * ldx : nullptr;
    V.lda[t] = 1;
    V.sigma_out[t] = on ? sigma_out + j * ld_sigma : nullptr;
    V.tail_out[t] = on ? tail_out + j : nullptr;
    V.paper_out[t] = on && paper_out ? paper_out + j : nullptr;
    V.energy_out[t] = nullptr;
    V.accept_out[t] = on && accept_out ? accept_out + j : nullptr;
  }
  __syncthreads();
  arrow_group(V, status);
}

cudaError_t launch_core_arrow(const ArrowDesc* d_desc, const int2* d_groups, int n_groups,
                              int* d_status, cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  prof_begin(s);
  core_arrow_kernel<<<n_groups, kArrowThreads, 0, s>>>(d_desc, d_groups, d_status);
  prof_end("core_arrow", s);
  return cudaGetLastError();
}

cudaError_t launch_core_arrow_columns(const ArrowState* d_states, const int4* d_groups,
                                      int n_groups, const float* Xt, int64_t ldx,
                                      float* sigma_out, int64_t ld_sigma, double* tail_out,
                                      double* tail_paper_out, uint8_t* accept_out, double eps,
                                      int* d_status, cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  prof_begin(s);
  core_arrow_columns_kernel<<<n_groups, kArrowThreads, 0, s>>>(
      d_states, d_groups, Xt, ldx, sigma_out, ld_sigma, tail_out, tail_paper_out, accept_out, eps,
      d_status);
  prof_end("core_arrow", s);
  return cudaGetLastError();
}

}  // namespace csvd
