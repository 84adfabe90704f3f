// Shared descriptors, helpers and launcher declarations of the csvd library.
// Every kernel works on batches of independent items described by small
// structs uploaded once per call; one call may mix items of different widths
// and ranks (the uneven batches of batched merge scoring).
#pragma once

#include <atomic>
#include <string>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace csvd {

// Device status bits (OR-ed into a per-call status word).
enum : int {
  kStatusJacobiCap = 1,      // one-sided Jacobi hit its sweep cap
  kStatusBisectCap = 2,      // bisection hit its iteration cap
  kStatusWaitCap = 4,        // a bounded wait on an mbarrier gave up
  kStatusBadShape = 8,       // a kernel met sizes outside its limits
};

// ---------------------------------------------------------------- GEMM
// C = alpha * op(A) op(B) + beta * op(Cin), row-major storage.  op(A) is
// M x K: tA = 0 -> A[i*lda + l], tA = 1 -> A[l*lda + i].  op(B) is K x N:
// tB = 0 -> B[l*ldb + j], tB = 1 -> B[j*ldb + l].  tC / tCin select C[i*ldc+j]
// or C[j*ldc+i].  beta == 0 never reads Cin.  Inputs are f32 unless
// a_bf16 / b_bf16 mark the A or B operand as bf16.
struct GemmDesc {
  const void* A;
  const void* B;
  const float* Cin;
  float* C;
  int64_t lda, ldb, ldcin, ldc;
  int M, N, K;
  int tA, tB, tCin, tC;
  int a_bf16, b_bf16;
  float alpha, beta;
};
struct GemmTile {
  int desc, tm, tn, pad;
};
constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16, kGemmThreads = 256;

// ------------------------------------------------------- Householder QR
// Column-major residual Rt (k x m row-major: column c of R is Rt + c*ldr),
// factorised in place for its first kp columns; B (kp x k, row-major ldb)
// receives the upper-triangular factor, tau the reflector scales.
struct QRDesc {
  float* Rt;
  int64_t ldr;
  float* tau;
  float* B;
  int64_t ldb;
  int m, k, kp, pad;
};

// Q_res W_bot for the basis rotation: Zt (ncols x m, ld m) row j = column j.
struct ApplyQDesc {
  const float* Rt;     // reflectors (as left by the QR kernel)
  int64_t ldr;
  const float* tau;
  const float* Wt;     // ncols x ldw, row j holds the left vector j (core rows)
  int64_t ldw;
  int woff;            // offset of the Q_res rows inside a Wt row (= r_t)
  float* Zt;
  int64_t ldz;
  int m, kp, ncols, pad;
};

// ------------------------------------------------ core of a merge evaluation
// Shared by the Jacobi (plain) and tridiagonal (mixed) core kernels.
struct CoreDesc {
  const float* P;        // r_t x k, row-major ldp (projection)
  const float* P2;       // optional re-orthogonalisation correction, same layout
  int64_t ldp;
  const float* B;        // plain: kp x k upper-triangular R factor (ldb)
  const float* Gaa;      // mixed: k x k Gram A^T A (upper triangle valid, ldb)
  int64_t ldb;
  const double* colE;    // mixed: k column energies sum_i A_ic^2 (the diagonal of A^T A)
  const float* sigma;    // r_t retained singular values of the state
  const double* scal;    // state scalars {energy, discarded}
  const double* energy_add;  // ||A||_F^2 of this block
  float* work;           // n_rows x n_cols workspace when the core is not in smem
  int64_t ldwork;
  float* sigma_out;      // r_new values
  float* Wt;             // optional: r_new x n_rows left vectors (row j = vector j)
  int64_t ldw;
  double* tail_out;      // accumulated-discard form
  double* tail_paper_out;// sum ||A||^2 - sum sigma~^2 (may be null)
  double* energy_out;    // ||M||^2 after the append (may be null)
  uint8_t* accept_out;   // may be null
  uint8_t* refine;       // mixed: set to 1 when the tail needs the FP64 re-solve (may be null)
  double eps;
  int rt, k, kp, r_new;  // r_new = min(r, rt + kp)
  int in_smem;
  int refine_near;       // mark only tails within kDecisionBand of the accept threshold
};

// ----------------------------------------------------- one-column merges
// Mixed-form evaluation of a one-column candidate a (m values, stride lda)
// against a state (U: m x rt, ldu; sigma; scal = {energy, discarded}).
// Candidates of one state are launched in groups of up to kArrowGroup
// (int2 {first descriptor, count} per CTA) so that U is read once per group.
constexpr int kArrowMaxRt = 128;
constexpr int kArrowGroup = 4;
struct ArrowDesc {
  const float* a;
  int64_t lda;
  const float* U;
  int64_t ldu;
  int64_t m;
  int rt, r_new;
  const float* sigma;
  const double* scal;
  float* sigma_out;
  double* tail_out;
  double* tail_paper_out;  // may be null
  double* energy_out;      // may be null
  uint8_t* accept_out;     // may be null
  double eps;
};
// One state as the one-column path reads it.
struct ArrowState {
  const float* U;
  int64_t ldu;
  int64_t m;
  int rt, r_new;
  const float* sigma;
  const double* scal;
};

// ------------------------------------------------------------ energy
struct EnergyDesc {
  const void* A;
  int64_t ld;
  int m, k, bf16, pad;
  double* out;
};

// Residual energy of one block: out += ||A - U P||_F^2 (A m x k f32, lda;
// U m x r, ldu; P r x k, ldp).
struct ResidDesc {
  const float* A;
  int64_t lda;
  const float* U;
  int64_t ldu;
  const float* P;
  int64_t ldp;
  int m, k;
  double* out;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; `red` holds >= 33 floats of shared memory.  All threads
// receive the result.  Contains two __syncthreads.
__device__ __forceinline__ float block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    float x = lane < nw ? red[lane] : 0.f;
    x = warp_sum(x);
    if (lane == 0) red[32] = x;
  }
  __syncthreads();
  float r = red[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ float load_elem(const void* p, int64_t idx, int bf16) {
  if (bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[idx]);
  return reinterpret_cast<const float*>(p)[idx];
}

// Raises a kernel's dynamic shared-memory limit when a launch needs more than
// any earlier one (one device per process), so that repeated launches make
// no attribute call -- a launch-only path can then be captured into a CUDA
// graph after one launch outside the capture.
template <class Kernel>
cudaError_t ensure_smem(Kernel* kernel, int bytes, std::atomic<int>& set_bytes) {
  if (bytes <= 48 * 1024 || bytes <= set_bytes.load(std::memory_order_relaxed)) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  int cur = set_bytes.load(std::memory_order_relaxed);
  while (bytes > cur && !set_bytes.compare_exchange_weak(cur, bytes)) {
  }
  return cudaSuccess;
}

// ------------------------------------------------------- launch tracing
// Every kernel launch is bracketed by prof_begin / prof_end: the launch is
// counted, and while tracing is on a pair of CUDA events is recorded on the
// launch stream so per-kernel device time can be read back.
void prof_begin(cudaStream_t s);
void prof_end(const char* name, cudaStream_t s);

// ------------------------------------------------------------- launchers
// Each returns the cudaError_t of its launch.
cudaError_t launch_gemm(const GemmDesc* d_desc, const GemmTile* d_tiles, int n_tiles,
                        cudaStream_t s);
cudaError_t launch_householder_qr(const QRDesc* d_desc, int n_items, int max_m,
                                  cudaStream_t s);
cudaError_t launch_apply_q(const ApplyQDesc* d_desc, int n_items, int max_cols,
                           cudaStream_t s);
cudaError_t launch_energy(const EnergyDesc* d_desc, int n_items, int max_chunks,
                          cudaStream_t s);
cudaError_t launch_resid_energy(const ResidDesc* d_desc, int n_items, int max_m, int max_k, int r,
                                cudaStream_t s);
// Column energies: out[c] += sum_i A_ic^2 for every column of every item
// (EnergyDesc.out points at k doubles, zeroed before the launch).
cudaError_t launch_col_energy(const EnergyDesc* d_desc, int n_items, int max_k, int max_m,
                              cudaStream_t s);
int jacobi_scratch_floats(int nc);
// Eigen core launch classes by core size n (0: n <= 192, 1: n <= 320,
// 2: larger), the dynamic shared memory of a class launch whose largest
// core is n_max, and the global workspace (floats) a core of size n needs in
// that launch (nonzero only for the largest cores).
constexpr int kTriLargeSmemBytes = 227 * 1024 - 1024;
int tridiag_class(int n);
// Tunable launch-class edges (autotuner): edge0 in [kEdgeMin, kEdgeMax[0]],
// edge0 < edge1 <= kEdgeMax[1]; (-1, -1) restores the defaults.  False for
// values out of range (nothing changes).
constexpr int kEdgeMin = 64;
constexpr int kEdgeMax[2] = {288, 480};
bool tridiag_set_edges(int e0, int e1);
void tridiag_get_edges(int* e0, int* e1);
int tridiag_smem_bytes(int cls, int n_max);
int64_t tridiag_work_floats(int cls, int n, int n_max);
cudaError_t launch_core_jacobi(const CoreDesc* d_desc, int n_items, int smem_bytes,
                               int* d_status, cudaStream_t s);
cudaError_t launch_core_tridiag(int cls, const CoreDesc* d_desc, int n_items, int n_max,
                                int* d_status, cudaStream_t s);
std::string tridiag_selftest();
// Failure-path test hook: per-device iteration caps of the solvers and the
// limit of the tensor-core kernel's pipeline waits (negative: the default).
cudaError_t tridiag_set_bisect_cap(int cap);
cudaError_t refine64_set_bisect_cap(int cap);
cudaError_t arrow_set_cap(int cap);
cudaError_t jacobi_set_cap(int cap);
cudaError_t tc_set_wait_ns(long long ns, int stall);
// The mixed core marks an item for the FP64 re-solve when its estimated tail
// lies below this fraction of the merged energy.
constexpr double kRefineFrac = 2e-3;
// Callers that use only the accept decision (the clustering scan) re-solve
// only the items whose FP32 tail lies within this fraction of the merged
// energy from eps^2 times it: far above the FP32 core's error (a few u of
// the energy), so every other decision is already exact.
constexpr double kDecisionBand = 1e-5;
// FP64 re-solve of the marked items of up to three core arrays: `slots`
// persistent CTAs, each with n_max^2 doubles of `work`; *d_counter must be 0.
size_t refine64_smem_bytes(int n_max);
cudaError_t launch_core_refine64(const CoreDesc* d0, int n0, const CoreDesc* d1, int n1,
                                 const CoreDesc* d2, int n2, double* work, int slots, int n_max,
                                 int* d_counter, int* d_status, cudaStream_t s);
cudaError_t launch_core_arrow(const ArrowDesc* d_desc, const int2* d_groups, int n_groups,
                              int* d_status, cudaStream_t s);
// Candidates as rows of one matrix: group g = {first row, count, state, 0};
// row j of Xt (ldx floats apart) is candidate j, whose outputs sit at index
// j of the output arrays (sigma rows ld_sigma apart; paper, accept may be null).
cudaError_t launch_core_arrow_columns(const ArrowState* d_states, const int4* d_groups,
                                      int n_groups, const float* Xt, int64_t ldx,
                                      float* sigma_out, int64_t ld_sigma, double* tail_out,
                                      double* tail_paper_out, uint8_t* accept_out, double eps,
                                      int* d_status, cudaStream_t s);
cudaError_t launch_gram_dev(const float* U, int64_t ldu, int m, int r, float* D, cudaStream_t s);
cudaError_t launch_state_commit(const float* sigma_new, int r_new, float* sigma,
                                const double* energy_new, const double* tail_new,
                                double* scal, cudaStream_t s);
cudaError_t launch_add_inplace(float* dst, const float* src, int rows, int cols,
                               int64_t ld_dst, int64_t ld_src, cudaStream_t s);
cudaError_t launch_scale_cols(const float* U, int64_t ldu, int m, int r, const float* s,
                              int inverse, float* out, int64_t ld_out, cudaStream_t st);

}  // namespace csvd
