// csvd_score_one_noalloc: one mixed-form merge evaluation that allocates no
// memory.  Some callers cannot allocate device memory at the point where
// they score a merge: a process whose device memory is entirely reserved by
// another allocator (a framework's caching allocator that owns the GPU), or
// a latency-critical loop that must not pay cudaMalloc / cudaFree (which can
// synchronise the device).  This entry point runs the same kernels as
// csvd_score with CSVD_MIXED, with every intermediate (column energies, P = U^T A,
// A^T A, the eigen core's global workspace, the kernel descriptors) placed
// in one file-scope device array of fixed size that every GPU loading the
// library holds until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "csvd.h"
#include "common.cuh"
#include "internal.h"
#include "tc_gram.cuh"

using namespace csvd;

namespace {

constexpr size_t kScratchBytes = size_t(4) << 20;  // 4 MiB per GPU
constexpr int kMaxK = 512;
constexpr int kMaxRt = 128;
constexpr int kMaxTiles = 4 + 10;  // P tiles (rt <= 128, k <= 512) + upper G tiles

struct Descs {
  CUtensorMap mapA;  // 64-byte aligned: first
  CUtensorMap mapU;
  CoreDesc core;
  TcItem item;
  TcTile tiles[kMaxTiles];
};

// Scratch layout (byte offsets, 256-byte aligned).
constexpr size_t kOffColE = 0;  // k column energies (FP64)
constexpr size_t kOffDescs = size_t(kMaxK) * 8;
constexpr size_t kOffP = kOffDescs + 4096;
constexpr size_t kOffG = kOffP + size_t(kMaxRt) * kMaxK * 4;
constexpr size_t kOffWork = kOffG + size_t(kMaxK) * kMaxK * 4;
static_assert(sizeof(Descs) <= kOffP - kOffDescs, "descriptor region");
static_assert(kOffDescs % 64 == 0, "tensor maps need 64-byte alignment");

__global__ void write_descs_kernel(Descs d, Descs* dst) {
  if (threadIdx.x == 0) *dst = d;
}

std::mutex g_mu;
void* g_ptr[64] = {};

}  // namespace

// Scratch shared by every call on a device; contents persist between calls.
static __device__ __align__(256) unsigned char csvd_noalloc_scratch[kScratchBytes];

extern "C" csvd_status csvd_score_one_noalloc(csvd_state st, const csvd_block* A, double eps,
                                              float* sigma_out, double* tail_sq_out,
                                              double* tail_paper_out, uint8_t* accept_out) {
  if (!st || !A || !A->ptr || !sigma_out || !tail_sq_out)
    return set_error(CSVD_ERR_ARG, "NULL argument");
  if (A->dtype != CSVD_F32 || A->k < 1 || A->ld < A->k)
    return set_error(CSVD_ERR_ARG, "needs an f32 block with k >= 1 and ld >= k");
  if ((reinterpret_cast<uintptr_t>(A->ptr) & 15) != 0 || (A->ld & 3) != 0)
    return set_error(CSVD_ERR_ARG, "needs 16-byte aligned rows (ptr % 16 == 0, ld % 4 == 0)");
  const int k = (int)A->k;
  const int rt = st->rt;
  const int64_t m = st->m;
  if (k > kMaxK || rt > kMaxRt)
    return set_error(CSVD_ERR_SHAPE, "scratch limit: needs k <= 512 and rank <= 128");
  if (rt > 0 && (st->r & 3) != 0)
    return set_error(CSVD_ERR_SHAPE, "needs a state rank cap r divisible by 4");
  const float* U = st->U[st->cur];
  if (rt > 0 && (reinterpret_cast<uintptr_t>(U) & 15) != 0)
    return set_error(CSVD_ERR_SHAPE, "needs a 16-byte aligned state basis");
  const int n = rt + k;
  const int cls = tridiag_class(n);
  const int64_t work_floats = tridiag_work_floats(cls, n, n);
  if ((size_t)kOffWork + (size_t)work_floats * 4 > kScratchBytes)
    return set_error(CSVD_ERR_SHAPE, "scratch limit exceeded");
  // tensor maps of A and U (host-side encoding, no allocation)
  Descs h;
  std::memset(&h, 0, sizeof(h));
  if (!tc_tensor_map(A->ptr, k, m, A->ld, &h.mapA))
    return set_error(CSVD_ERR_SHAPE, "block cannot be described by a TMA tensor map");
  if (rt > 0 && !tc_tensor_map(U, rt, m, st->r, &h.mapU))
    return set_error(CSVD_ERR_SHAPE, "state basis cannot be described by a TMA tensor map");

  // set-up: the device address of the scratch array on the current device
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess || dev < 0 || dev >= 64)
    return set_error(CSVD_ERR_CUDA, "cudaGetDevice failed");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
      void* p = nullptr;
      e0 = cudaGetSymbolAddress(&p, csvd_noalloc_scratch);
      if (e0 != cudaSuccess || !p)
        return set_error(CSVD_ERR_CUDA, "cudaGetSymbolAddress failed");
      g_ptr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_ptr[dev]);
  }
  cudaStream_t s = st->stream;
  double* colE = reinterpret_cast<double*>(base + kOffColE);
  Descs* ddesc = reinterpret_cast<Descs*>(base + kOffDescs);
  float* P = reinterpret_cast<float*>(base + kOffP);
  float* G = reinterpret_cast<float*>(base + kOffG);
  float* work = reinterpret_cast<float*>(base + kOffWork);

  const int kld = (k + 3) & ~3;  // 16-byte rows for the Gram kernel's stores
  h.item = TcItem{reinterpret_cast<const float*>(A->ptr), A->ld, U, st->r, (int)m, k, rt, 0,
                  P, kld, G, kld, colE, &ddesc->mapA, rt > 0 ? &ddesc->mapU : &ddesc->mapA};
  int nt = 0;
  for (int r0 = 0; r0 < rt; r0 += kTcBM)
    for (int c0 = 0; c0 < k; c0 += kTcBN) h.tiles[nt++] = TcTile{0, 0, r0, c0};
  for (int r0 = 0; r0 < k; r0 += kTcBM)
    for (int c0 = r0; c0 < k; c0 += kTcBN) h.tiles[nt++] = TcTile{0, 1, r0, c0};
  CoreDesc& c = h.core;
  c.P = rt > 0 ? P : nullptr;
  c.ldp = kld;
  c.Gaa = G;
  c.colE = colE;
  c.ldb = kld;
  c.sigma = st->sigma;
  c.scal = st->scal;
  c.energy_add = nullptr;  // the sum of the column energies
  c.work = work_floats > 0 ? work : nullptr;
  c.ldwork = n;
  c.sigma_out = sigma_out;
  c.tail_out = tail_sq_out;
  c.tail_paper_out = tail_paper_out;
  c.accept_out = accept_out;
  c.eps = eps;
  c.rt = rt;
  c.k = k;
  c.kp = (int)std::min<int64_t>(k, m - rt);
  c.r_new = std::min(st->r, rt + c.kp);

  // column energies start at zero; descriptors are written by a kernel (no
  // host staging)
  cudaError_t e = cudaMemsetAsync(colE, 0, sizeof(double) * (size_t)k, s);
  if (e == cudaSuccess) {
    write_descs_kernel<<<1, 32, 0, s>>>(h, ddesc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_tc_gram(&ddesc->item, ddesc->tiles, nt, device_sm_count(), st->status, s);
  if (e == cudaSuccess) e = launch_core_tridiag(cls, &ddesc->core, 1, n, st->status, s);
  if (e != cudaSuccess)
    return set_error(CSVD_ERR_CUDA, cudaGetErrorString(e));
  return CSVD_OK;
}
