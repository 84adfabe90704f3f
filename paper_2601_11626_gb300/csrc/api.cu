// Host side of the csvd C ABI: state objects, workspace, batched pipelines
// for the merge evaluation (plain and mixed forms), the basis commit, the
// bounds, the clustering drivers of Algorithms 1-3 and the tail gradient.
//
// Every pipeline is a fixed sequence of batched launches; the host only
// builds descriptor tables (uploaded once per call through a pinned staging
// ring) and, in the clustering drivers, takes the greedy decisions between
// launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <unordered_map>

#include "csvd.h"
#include "common.cuh"
#include "internal.h"
#include "tc_gram.cuh"

using namespace csvd;

// =================================================================== errors
static thread_local std::string g_err = "";

static csvd_status fail(csvd_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

namespace csvd {
csvd_status set_error(csvd_status st, const char* msg) { return fail(st, msg); }
}  // namespace csvd

#define CUDA_TRY(expr)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? CSVD_ERR_OOM : CSVD_ERR_CUDA,      \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                \
  } while (0)

#define CSVD_TRY(expr)                    \
  do {                                    \
    csvd_status s_ = (expr);              \
    if (s_ != CSVD_OK) return s_;         \
  } while (0)

// ================================================================ tracing
namespace csvd {
static std::atomic<long long> g_launch_count{0};
static std::atomic<bool> g_prof_on{false};
struct ProfEv {
  const char* name;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::vector<ProfEv> g_prof;
static thread_local cudaEvent_t t_prof_begin = nullptr;

void prof_begin(cudaStream_t s) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  if (cudaEventCreate(&t_prof_begin) != cudaSuccess) { t_prof_begin = nullptr; return; }
  cudaEventRecord(t_prof_begin, s);
}

void prof_end(const char* name, cudaStream_t s) {
  g_launch_count.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof_on.load(std::memory_order_relaxed) || !t_prof_begin) return;
  cudaEvent_t b = nullptr;
  if (cudaEventCreate(&b) != cudaSuccess) return;
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back(ProfEv{name, t_prof_begin, b});
  t_prof_begin = nullptr;
}
}  // namespace csvd

// =============================================================== allocation
static csvd_alloc_fn g_alloc = nullptr;
static csvd_free_fn g_free = nullptr;
static void* g_actx = nullptr;
static std::once_flag g_pool_once;

static void* dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 256;
  if (g_alloc) return g_alloc(bytes, (void*)s, g_actx);
  std::call_once(g_pool_once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
    }
  });
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) return nullptr;
  return p;
}

static void dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  if (g_free) g_free(p, (void*)s, g_actx);
  else cudaFreeAsync(p, s);
}

// Byte layout of one workspace allocation (256-byte aligned pieces).
struct Layout {
  size_t size = 0;
  size_t add(size_t bytes) {
    size_t off = (size + 255) & ~size_t(255);
    size = off + bytes;
    return off;
  }
};

struct Workspace {
  char* base = nullptr;
  cudaStream_t s = nullptr;
  ~Workspace() { dev_free(base, s); }
  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(base + off); }
};

// The stream work of a prepared batched evaluation (csvd_score_plan): memsets
// and kernel launches on device buffers the plan owns, replayed by
// csvd_plan_launch without any allocation, host copy or synchronisation.
using StreamOp = std::function<cudaError_t(cudaStream_t)>;
struct LaunchPlan {
  std::vector<StreamOp> ops;
  std::vector<void*> bufs;   // device buffers the ops use (freed with the plan)
  cudaStream_t s = nullptr;  // stream the plan was built on
  int* status = nullptr;     // its device status word (in bufs)
};

// Runs the stream work now, or appends it to a plan.
static csvd_status run_or_keep(std::vector<StreamOp>& ops, cudaStream_t s, LaunchPlan* plan) {
  if (plan) {
    for (auto& op : ops) plan->ops.push_back(std::move(op));
    return CSVD_OK;
  }
  for (auto& op : ops) CUDA_TRY(op(s));
  return CSVD_OK;
}

// Pinned host staging ring for descriptor uploads.
struct StagingRing {
  struct Slot {
    void* host = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool used = false;
  };
  static constexpr int kSlots = 16;
  std::mutex mu;
  Slot slots[kSlots];
  int next = 0;
};
static StagingRing g_ring;

static cudaError_t upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  std::lock_guard<std::mutex> lk(g_ring.mu);
  StagingRing::Slot& sl = g_ring.slots[g_ring.next];
  g_ring.next = (g_ring.next + 1) % StagingRing::kSlots;
  cudaError_t e;
  if (sl.used) {
    e = cudaEventSynchronize(sl.ev);
    if (e != cudaSuccess) return e;
  }
  if (sl.cap < bytes) {
    if (sl.host) cudaFreeHost(sl.host);
    sl.host = nullptr;
    size_t cap = std::max<size_t>(bytes + bytes / 2, 1 << 16);
    e = cudaHostAlloc(&sl.host, cap, cudaHostAllocPortable);
    if (e != cudaSuccess) { sl.cap = 0; return e; }
    sl.cap = cap;
  }
  if (!sl.ev) {
    e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  std::memcpy(sl.host, src, bytes);
  e = cudaMemcpyAsync(dst, sl.host, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(sl.ev, s);
  sl.used = true;
  return e;
}

// Host-side packing of descriptor tables into one upload.
struct Pack {
  std::vector<char> buf;
  template <class T>
  size_t add(const std::vector<T>& v) {
    size_t off = (buf.size() + 255) & ~size_t(255);
    buf.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

// ============================================================ GEMM batches
struct GemmBatch {
  std::vector<GemmDesc> descs;
  std::vector<GemmTile> tiles;
  size_t off_d = 0, off_t = 0;
  void add(const GemmDesc& d, bool upper_only = false) {
    if (d.M <= 0 || d.N <= 0) return;
    const int id = (int)descs.size();
    descs.push_back(d);
    const int tm = (d.M + kGemmBM - 1) / kGemmBM, tn = (d.N + kGemmBN - 1) / kGemmBN;
    for (int a = 0; a < tm; ++a)
      for (int b = 0; b < tn; ++b)
        if (!upper_only || a <= b) tiles.push_back(GemmTile{id, a, b, 0});
  }
  void pack(Pack& p) {
    off_d = p.add(descs);
    off_t = p.add(tiles);
  }
  cudaError_t launch(char* dbase, cudaStream_t s) const {
    if (tiles.empty()) return cudaSuccess;
    return launch_gemm(reinterpret_cast<const GemmDesc*>(dbase + off_d),
                       reinterpret_cast<const GemmTile*>(dbase + off_t), (int)tiles.size(), s);
  }
  // the launch as a stream operation (captures offsets and counts only)
  StreamOp op(char* dbase) const {
    const size_t d = off_d, t = off_t;
    const int nt = (int)tiles.size();
    return [=](cudaStream_t st) {
      if (nt == 0) return cudaSuccess;
      return launch_gemm(reinterpret_cast<const GemmDesc*>(dbase + d),
                         reinterpret_cast<const GemmTile*>(dbase + t), nt, st);
    };
  }
};

static GemmDesc gemm(const void* A, int64_t lda, int tA, const void* B, int64_t ldb, int tB,
                     float* C, int64_t ldc, int tC, int M, int N, int K, float alpha = 1.f,
                     const float* Cin = nullptr, int64_t ldcin = 0, int tCin = 0,
                     float beta = 0.f, int a_bf16 = 0, int b_bf16 = 0) {
  GemmDesc d;
  d.A = A; d.B = B; d.Cin = Cin; d.C = C;
  d.lda = lda; d.ldb = ldb; d.ldcin = ldcin; d.ldc = ldc;
  d.M = M; d.N = N; d.K = K;
  d.tA = tA; d.tB = tB; d.tCin = tCin; d.tC = tC;
  d.a_bf16 = a_bf16; d.b_bf16 = b_bf16;
  d.alpha = alpha; d.beta = beta;
  return d;
}

// ================================================================== state
// Read-only view of a state for the batched pipelines.
struct StateView {
  const float* U;
  int64_t ldu;
  int rt, r;
  const float* sigma;
  const double* scal;
};

static StateView view_of(const csvd_state_s* s) {
  return StateView{s->U[s->cur], s->r, s->rt, s->r, s->sigma, s->scal};
}

static csvd_status check_block(const csvd_block* b, int64_t m) {
  if (!b || !b->ptr) return fail(CSVD_ERR_ARG, "block pointer is NULL");
  if (b->k < 1 || b->ld < b->k) return fail(CSVD_ERR_ARG, "block needs k >= 1 and ld >= k");
  if (b->dtype != CSVD_F32 && b->dtype != CSVD_BF16) return fail(CSVD_ERR_ARG, "bad dtype");
  if (b->k > (int64_t)1 << 20) return fail(CSVD_ERR_SHAPE, "block too wide");
  (void)m;
  return CSVD_OK;
}

static csvd_status take_status(int* d_status, cudaStream_t s) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (h) {
    CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), s));
    if (h & kStatusJacobiCap) return fail(CSVD_ERR_NOT_CONVERGED, "Jacobi core hit its sweep cap");
    if (h & kStatusBisectCap) return fail(CSVD_ERR_NOT_CONVERGED, "bisection hit its iteration cap");
    if (h & kStatusWaitCap) return fail(CSVD_ERR_TIMEOUT, "a bounded device wait gave up");
    return fail(CSVD_ERR_SHAPE, "device kernel reported bad sizes");
  }
  return CSVD_OK;
}

// Largest core kept in shared memory (bytes of dynamic shared memory).
static constexpr int kCoreSmemBudget = 200 * 1024;
// FP64 re-solve of the mixed core: at most this many persistent CTAs, and at
// most this many bytes of slots per call (at least one slot)
static constexpr int kRefineSlots = 64;
static constexpr size_t kRefineBytes = size_t(192) << 20;

static int num_sms();
namespace csvd {
int device_sm_count() { return num_sms(); }
csvd_status set_error(csvd_status st, const char* msg);
}  // namespace csvd

// SM count of the current device (cached per device).
static int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// The Gram of the mixed form runs on the tensor cores unless CSVD_GRAM=simt.
static bool gram_on_tensor_cores() {
  static const bool on = [] {
    const char* e = std::getenv("CSVD_GRAM");
    return !(e && std::strcmp(e, "simt") == 0);
  }();
  return on;
}

// ------------------------------------------------------- TMA tensor maps
// 2-D maps of the candidate blocks and state bases read by the tensor-core
// Gram (tc_tensor_map: box 32 rows x 32 f32 columns, 128-byte swizzle, zero
// fill), cached by (address, shape).
struct MapKey {
  uintptr_t ptr;
  int64_t cols, rows, ld;
  bool operator==(const MapKey& o) const {
    return ptr == o.ptr && cols == o.cols && rows == o.rows && ld == o.ld;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    size_t h = std::hash<uintptr_t>()(k.ptr);
    h ^= std::hash<int64_t>()(k.cols) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h ^= std::hash<int64_t>()(k.rows) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h ^= std::hash<int64_t>()(k.ld) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
  }
};
static std::mutex g_map_mu;
static std::unordered_map<MapKey, CUtensorMap, MapKeyHash> g_maps;

// Tensor map of a row-major f32 matrix (rows x cols, leading dimension ld);
// false when it cannot be encoded (the item then takes the SIMT Gram).
static bool tensor_map(const void* ptr, int64_t cols, int64_t rows, int64_t ld, CUtensorMap* out) {
  const MapKey key{reinterpret_cast<uintptr_t>(ptr), cols, rows, ld};
  std::lock_guard<std::mutex> lk(g_map_mu);
  auto it = g_maps.find(key);
  if (it != g_maps.end()) {
    *out = it->second;
    return true;
  }
  CUtensorMap m;
  if (!tc_tensor_map(ptr, cols, rows, ld, &m)) return false;
  if (g_maps.size() > (1u << 20)) g_maps.clear();
  g_maps.emplace(key, m);
  *out = m;
  return true;
}

// ===================================================== the batched pipeline
// One merge evaluation per item: (state view, block).  Produces sigma~,
// tails, energies and accept flags into caller arrays (device).  When
// `want_W` is set (plain form only) the left vectors Wt and the QR
// workspace stay alive in `keep` for a basis commit.
struct Item {
  StateView st;
  const csvd_block* blk;
  int r;        // target rank
  int64_t m;
  // outputs (device)
  float* sigma_out;
  double* tail_out;
  double* tail_paper_out;
  double* energy_out;
  uint8_t* accept_out;
};

struct CommitKeep {  // workspace kept for the commit of a single plain item
  float* Rt = nullptr;
  float* tau = nullptr;
  float* Wt = nullptr;
  int kp = 0, nr = 0, r_new = 0;
};

// Mixed-form evaluations of one-column candidates: the Gram of the core is
// an arrowhead, solved by bisection on its exact O(r_t) inertia count.
static bool arrow_eligible(const Item& it) {
  return it.blk->k == 1 && it.blk->dtype == CSVD_F32 && it.st.rt <= kArrowMaxRt;
}

static_assert(sizeof(ArrowDesc) % alignof(int2) == 0, "group table follows the descriptors");

static bool same_arrow_state(const Item& x, const Item& y) {
  return x.st.U == y.st.U && x.st.ldu == y.st.ldu && x.st.rt == y.st.rt && x.r == y.r &&
         x.m == y.m && x.st.sigma == y.st.sigma && x.st.scal == y.st.scal;
}

// One-column items in launch order (candidates of one state side by side)
// and their CTA groups {first position in that order, count <= kArrowGroup},
// each group one state.
static void arrow_item_groups(const std::vector<Item>& items, std::vector<int>& order,
                              std::vector<int2>& groups) {
  const int n = (int)items.size();
  order.resize(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return reinterpret_cast<uintptr_t>(items[x].st.U) < reinterpret_cast<uintptr_t>(items[y].st.U);
  });
  groups.clear();
  for (int i = 0; i < n; ++i) {
    if (groups.empty() || groups.back().y == kArrowGroup ||
        !same_arrow_state(items[order[i]], items[order[groups.back().x]]))
      groups.push_back(make_int2(i, 0));
    ++groups.back().y;
  }
}

static csvd_status run_arrow_items(const std::vector<Item>& items, double eps, cudaStream_t s,
                                   int* d_status, LaunchPlan* plan = nullptr) {
  const int n = (int)items.size();
  if (n == 0) return CSVD_OK;
  std::vector<int> order;
  std::vector<int2> groups;
  arrow_item_groups(items, order, groups);
  std::vector<ArrowDesc> ad(n);
  for (int i = 0; i < n; ++i) {
    const Item& it = items[order[i]];
    ArrowDesc& d = ad[i];
    d.a = reinterpret_cast<const float*>(it.blk->ptr);
    d.lda = it.blk->ld;
    d.U = it.st.U;
    d.ldu = it.st.ldu;
    d.m = it.m;
    d.rt = it.st.rt;
    d.r_new = std::min<int64_t>(it.r, it.st.rt + std::min<int64_t>(1, it.m - it.st.rt));
    d.sigma = it.st.sigma;
    d.scal = it.st.scal;
    d.sigma_out = it.sigma_out;
    d.tail_out = it.tail_out;
    d.tail_paper_out = it.tail_paper_out;
    d.energy_out = it.energy_out;
    d.accept_out = it.accept_out;
    d.eps = eps;
  }
  const size_t desc_bytes = sizeof(ArrowDesc) * n, group_bytes = sizeof(int2) * groups.size();
  std::vector<char> host(desc_bytes + group_bytes);
  std::memcpy(host.data(), ad.data(), desc_bytes);
  std::memcpy(host.data() + desc_bytes, groups.data(), group_bytes);
  Workspace w;
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(host.size(), s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  CUDA_TRY(upload(w.base, host.data(), host.size(), s));
  std::vector<StreamOp> ops;
  {
    ArrowDesc* dd = w.at<ArrowDesc>(0);
    int2* dg = w.at<int2>(desc_bytes);
    const int ng = (int)groups.size();
    ops.push_back([=](cudaStream_t st) { return launch_core_arrow(dd, dg, ng, d_status, st); });
  }
  CSVD_TRY(run_or_keep(ops, s, plan));
  if (plan) {
    plan->bufs.push_back(w.base);  // the plan owns the descriptors now
    w.base = nullptr;
  }
  return CSVD_OK;
}

static csvd_status run_items_general(const std::vector<Item>& items, double eps, int precision,
                                     cudaStream_t s, int* d_status, Workspace& ws,
                                     CommitKeep* keep, bool want_W, LaunchPlan* plan = nullptr);

// Set while a caller scores candidates only for their accept decisions (the
// clustering scan): the mixed core then re-solves in FP64 only the items
// near the threshold (kDecisionBand) instead of every small tail.
static thread_local bool t_decision_only = false;
struct DecisionOnly {
  DecisionOnly() { t_decision_only = true; }
  ~DecisionOnly() { t_decision_only = false; }
};

// With a plan, the stream work is kept in it (and the buffers it uses move
// into it) instead of running.
static csvd_status run_items(const std::vector<Item>& items, double eps, int precision,
                             cudaStream_t s, int* d_status, Workspace& ws, CommitKeep* keep,
                             bool want_W, LaunchPlan* plan = nullptr) {
  if (precision != CSVD_PLAIN_FP32 && !want_W) {
    std::vector<Item> arrow, rest;
    for (const Item& it : items) (arrow_eligible(it) ? arrow : rest).push_back(it);
    if (!arrow.empty()) {
      CSVD_TRY(run_arrow_items(arrow, eps, s, d_status, plan));
      return rest.empty() ? CSVD_OK : run_items_general(rest, eps, precision, s, d_status, ws, keep,
                                                        want_W, plan);
    }
  }
  return run_items_general(items, eps, precision, s, d_status, ws, keep, want_W, plan);
}

static csvd_status run_items_general(const std::vector<Item>& items, double eps, int precision,
                                     cudaStream_t s, int* d_status, Workspace& ws,
                                     CommitKeep* keep, bool want_W, LaunchPlan* plan) {
  const int n = (int)items.size();
  if (n == 0) return CSVD_OK;
  Layout L;
  struct Off { size_t energy, colE, P, P2, Rt, tau, B, G, work, Wt; int64_t ldwork; int kp, nr, nc, r_new, cls; bool smem; };
  std::vector<Off> off(n);
  // the Gram route (tensor-core products for CSVD_MIXED, FP32 SIMT products
  // for CSVD_GRAM_FP32); the plain route also serves basis commits
  const bool mixed = (precision != CSVD_PLAIN_FP32) && !want_W;
  const bool tensor = mixed && precision == CSVD_MIXED && gram_on_tensor_cores();
  const size_t energies = L.add(sizeof(double) * (size_t)n);  // one array, zeroed at once
  // mixed: the column energies of every block, one array zeroed at once
  size_t colE_total = 0;
  if (mixed)
    for (int i = 0; i < n; ++i) colE_total += (size_t)items[i].blk->k;
  const size_t colE_base = mixed ? L.add(sizeof(double) * colE_total) : 0;
  for (int i = 0; i < n; ++i) {
    const Item& it = items[i];
    const int64_t m = it.m;
    const int k = (int)it.blk->k, rt = it.st.rt;
    Off& o = off[i];
    o.kp = (int)std::min<int64_t>(k, m - rt);
    o.nr = rt + o.kp;
    o.nc = rt + k;
    o.r_new = std::min(it.r, o.nr);
    o.energy = energies + sizeof(double) * (size_t)i;
    o.colE = 0;
    if (mixed) {
      size_t before = 0;
      for (int j = 0; j < i; ++j) before += (size_t)items[j].blk->k;
      o.colE = colE_base + sizeof(double) * before;
    }
    // mixed form: P and A^T A rows padded to 4 floats (16-byte stores)
    const int kld = mixed ? (k + 3) & ~3 : k;
    o.P = rt > 0 ? L.add(sizeof(float) * (size_t)rt * kld) : 0;
    if (mixed) {
      o.G = L.add(sizeof(float) * (size_t)k * kld);
      o.ldwork = rt + k;
      o.smem = false;
      o.work = 0;
      o.cls = 0;
    } else {
      o.P2 = rt > 0 ? L.add(sizeof(float) * (size_t)rt * k) : 0;
      o.Rt = L.add(sizeof(float) * (size_t)k * m);
      o.tau = L.add(sizeof(float) * (size_t)std::max(o.kp, 1));
      o.B = L.add(sizeof(float) * (size_t)std::max(o.kp, 1) * k);
      const int ncp = o.nc + (o.nc & 1);
      const int need = (jacobi_scratch_floats(o.nc) + ncp * o.nr) * 4;
      o.smem = need <= kCoreSmemBudget;
      o.ldwork = o.nr;
      o.work = o.smem ? 0 : L.add(sizeof(float) * (size_t)ncp * o.nr);
      o.Wt = want_W ? L.add(sizeof(float) * (size_t)std::max(o.r_new, 1) * o.nr) : 0;
    }
  }
  // mixed form: eigen-core launch classes by core size; the leading tile
  // columns of the largest cores get a global workspace
  int tri_nmax[3] = {1, 1, 1};
  // mixed form: per-item FP64 re-solve marks, the persistent re-solve's item
  // counter and its workspace slots (n_max^2 doubles each)
  size_t refine_flags = 0, refine_ctr = 0, refine_work = 0;
  int refine_slots = 0, refine_nmax = 1;
  if (mixed) {
    for (int i = 0; i < n; ++i)
      refine_nmax = std::max(refine_nmax, items[i].st.rt + (int)items[i].blk->k);
    const size_t slot_bytes = sizeof(double) * (size_t)refine_nmax * refine_nmax;
    refine_slots = (int)std::min<size_t>({(size_t)n, (size_t)kRefineSlots,
                                          std::max<size_t>(1, kRefineBytes / slot_bytes)});
    refine_flags = L.add((size_t)n);
    refine_ctr = L.add(sizeof(int));
    refine_work = L.add(slot_bytes * (size_t)refine_slots);
  }
  if (mixed) {
    for (int i = 0; i < n; ++i) {
      const int nn = items[i].st.rt + (int)items[i].blk->k;
      off[i].cls = tridiag_class(nn);
      tri_nmax[off[i].cls] = std::max(tri_nmax[off[i].cls], nn);
    }
    for (int i = 0; i < n; ++i) {
      const int nn = items[i].st.rt + (int)items[i].blk->k;
      const int64_t wf = tridiag_work_floats(off[i].cls, nn, tri_nmax[off[i].cls]);
      if (wf > 0) off[i].work = L.add(sizeof(float) * (size_t)wf);
    }
  }
  // tensor-core Gram: eligible items (f32, 16-byte aligned rows)
  std::vector<char> tc_ok(n, 0);
  if (tensor) {
    for (int i = 0; i < n; ++i) {
      const Item& it = items[i];
      const bool a_ok = it.blk->dtype == CSVD_F32 && (reinterpret_cast<uintptr_t>(it.blk->ptr) & 15) == 0 &&
                        (it.blk->ld & 3) == 0;
      const bool u_ok = it.st.rt == 0 || ((reinterpret_cast<uintptr_t>(it.st.U) & 15) == 0 && (it.st.ldu & 3) == 0);
      tc_ok[i] = a_ok && u_ok;
    }
  }
  // upper bound for the descriptor region: computed after building with a dummy base
  // -> build twice: sizes do not depend on the base pointer.
  // tensor maps of the tensor-core items: candidates, then distinct bases
  std::vector<CUtensorMap> maps;
  std::vector<int> mapA_idx(n, -1), mapU_idx(n, -1);
  {
    std::vector<std::pair<const float*, int>> seenU;
    for (int i = 0; i < n; ++i) {
      if (!tc_ok[i]) continue;
      const Item& it = items[i];
      tc_ok[i] = 0;  // set again once both maps exist
      CUtensorMap ma;
      if (!tensor_map(it.blk->ptr, it.blk->k, it.m, it.blk->ld, &ma)) continue;
      int iu = -1;
      if (it.st.rt > 0) {
        for (auto& pr : seenU)
          if (pr.first == it.st.U) iu = pr.second;
        if (iu < 0) {
          CUtensorMap mu;
          if (!tensor_map(it.st.U, it.st.rt, it.m, it.st.ldu, &mu)) continue;
          iu = (int)maps.size();
          maps.push_back(mu);
          seenU.push_back({it.st.U, iu});
        }
      }
      mapA_idx[i] = (int)maps.size();
      maps.push_back(ma);
      mapU_idx[i] = iu;
      tc_ok[i] = 1;
    }
  }
  char* pk_base = nullptr;  // device address of the descriptor region (maps first)
  auto build = [&](char* base, Pack& pk, GemmBatch& gP, GemmBatch& gR, GemmBatch& gP2,
                   GemmBatch& gRu, GemmBatch& gG, std::vector<EnergyDesc>& ed,
                   std::vector<EnergyDesc>& ced, std::vector<QRDesc>& qd, std::vector<CoreDesc>& cd_s,
                   std::vector<CoreDesc>& cd_g, std::vector<CoreDesc>& cd_m, std::vector<TcItem>& tci,
                   std::vector<TcTile>& tct) {
    pk.add(maps);
    int max_m = 1;
    for (int i = 0; i < n; ++i) {
      const Item& it = items[i];
      const Off& o = off[i];
      const int64_t m = it.m;
      const int k = (int)it.blk->k, rt = it.st.rt;
      const int bf = it.blk->dtype == CSVD_BF16;
      max_m = std::max<int>(max_m, (int)m);
      double* energy = reinterpret_cast<double*>(base + o.energy);
      float* P = rt > 0 ? reinterpret_cast<float*>(base + o.P) : nullptr;
      EnergyDesc e{it.blk->ptr, it.blk->ld, (int)m, k, bf, 0, energy};
      ed.push_back(e);
      const int kld = mixed ? (k + 3) & ~3 : k;
      if (rt > 0 && !mixed)
        gP.add(gemm(it.st.U, it.st.ldu, 1, it.blk->ptr, it.blk->ld, 0, P, kld, 0, rt, k, (int)m,
                    1.f, nullptr, 0, 0, 0.f, 0, bf));
      CoreDesc c;
      std::memset(&c, 0, sizeof(c));
      c.P = P;
      c.P2 = nullptr;
      c.ldp = kld;
      c.sigma = it.st.sigma;
      c.scal = it.st.scal;
      // mixed form: the eigen core takes ||A||^2 as the sum of the column energies
      c.energy_add = mixed ? nullptr : energy;
      c.sigma_out = it.sigma_out;
      c.tail_out = it.tail_out;
      c.tail_paper_out = it.tail_paper_out;
      c.energy_out = it.energy_out;
      c.accept_out = it.accept_out;
      c.eps = eps;
      c.rt = rt;
      c.k = k;
      c.kp = o.kp;
      c.r_new = o.r_new;
      c.in_smem = o.smem ? 1 : 0;
      c.refine_near = t_decision_only ? 1 : 0;
      c.work = o.smem ? nullptr : reinterpret_cast<float*>(base + o.work);
      c.ldwork = o.ldwork;
      if (mixed) {
        float* G = reinterpret_cast<float*>(base + o.G);
        double* colE = reinterpret_cast<double*>(base + o.colE);
        if (tc_ok[i]) {
          const int id = (int)tci.size();
          TcItem ti{reinterpret_cast<const float*>(it.blk->ptr), it.blk->ld, it.st.U,
                    it.st.ldu, (int)m, k, rt, 0, P, kld, G, kld, colE, nullptr, nullptr};
          // maps are the first array of the descriptor region
          ti.mapA = pk_base + (size_t)mapA_idx[i] * sizeof(CUtensorMap);
          ti.mapU = rt > 0 ? pk_base + (size_t)mapU_idx[i] * sizeof(CUtensorMap) : ti.mapA;
          tci.push_back(ti);
          for (int r0 = 0; r0 < rt; r0 += kTcBM)
            for (int c0 = 0; c0 < k; c0 += kTcBN) tct.push_back(TcTile{id, 0, r0, c0});
          for (int r0 = 0; r0 < k; r0 += kTcBM)
            for (int c0 = r0; c0 < k; c0 += kTcBN) tct.push_back(TcTile{id, 1, r0, c0});
        } else {
          if (rt > 0)
            gP.add(gemm(it.st.U, it.st.ldu, 1, it.blk->ptr, it.blk->ld, 0, P, kld, 0, rt, k, (int)m,
                        1.f, nullptr, 0, 0, 0.f, 0, bf));
          gG.add(gemm(it.blk->ptr, it.blk->ld, 1, it.blk->ptr, it.blk->ld, 0, G, kld, 0, k, k,
                      (int)m, 1.f, nullptr, 0, 0, 0.f, bf, bf), true);
          ced.push_back(EnergyDesc{it.blk->ptr, it.blk->ld, (int)m, k, bf, 0, colE});
        }
        c.Gaa = G;
        c.colE = colE;
        c.ldb = kld;
        c.refine = reinterpret_cast<uint8_t*>(base + refine_flags) + i;
        c.work = o.work ? reinterpret_cast<float*>(base + o.work) : nullptr;
      } else {
        if (bf) return false;
        float* P2 = rt > 0 ? reinterpret_cast<float*>(base + o.P2) : nullptr;
        float* Rt = reinterpret_cast<float*>(base + o.Rt);
        // R^T = (A - U P)^T  (K = 0 when rt == 0: a transpose copy)
        gR.add(gemm(it.st.U, it.st.ldu, 0, P, k, 0, Rt, m, 1, (int)m, k, rt, -1.f,
                    reinterpret_cast<const float*>(it.blk->ptr), it.blk->ld, 0, 1.f));
        if (rt > 0) {
          gP2.add(gemm(it.st.U, it.st.ldu, 1, Rt, m, 1, P2, k, 0, rt, k, (int)m));
          gRu.add(gemm(it.st.U, it.st.ldu, 0, P2, k, 0, Rt, m, 1, (int)m, k, rt, -1.f, Rt, m,
                       1, 1.f));
        }
        QRDesc q{Rt, m, reinterpret_cast<float*>(base + o.tau), reinterpret_cast<float*>(base + o.B),
                 k, (int)m, k, o.kp, 0};
        if (o.kp > 0) qd.push_back(q);
        c.P2 = P2;
        c.B = reinterpret_cast<float*>(base + o.B);
        c.ldb = k;
        if (want_W) {
          c.Wt = reinterpret_cast<float*>(base + o.Wt);
          c.ldw = o.nr;
        }
      }
      if (mixed) (o.cls == 0 ? cd_s : o.cls == 1 ? cd_m : cd_g).push_back(c);
      else (o.smem ? cd_s : cd_g).push_back(c);
    }
    gP.pack(pk); gR.pack(pk); gP2.pack(pk); gRu.pack(pk); gG.pack(pk);
    (void)max_m;
    return true;
  };
  // the core of an item lands in cd_s (small / on-chip class) or cd_g
  // pass 1: sizes of the descriptor region
  size_t desc_bytes = 0;
  {
    Pack pk;
    GemmBatch a, b, c, d, e;
    std::vector<EnergyDesc> ed, ce; std::vector<QRDesc> qd; std::vector<CoreDesc> cs, cg, cm;
    std::vector<TcItem> ti; std::vector<TcTile> tt;
    char* fake = reinterpret_cast<char*>(uintptr_t(1) << 20);
    if (!build(fake, pk, a, b, c, d, e, ed, ce, qd, cs, cg, cm, ti, tt))
      return fail(CSVD_ERR_UNIMPLEMENTED, "bf16 blocks need the mixed form");
    pk.add(ed); pk.add(ce); pk.add(qd); pk.add(cs); pk.add(cg); pk.add(cm); pk.add(ti); pk.add(tt);
    desc_bytes = pk.buf.size();
  }
  const size_t off_desc = L.add(desc_bytes);
  ws.s = s;
  ws.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!ws.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  pk_base = ws.base + off_desc;
  Pack pk;
  GemmBatch gP, gR, gP2, gRu, gG;
  std::vector<EnergyDesc> ed, ced; std::vector<QRDesc> qd; std::vector<CoreDesc> cd_s, cd_g, cd_m;
  std::vector<TcItem> tci; std::vector<TcTile> tct;
  build(ws.base, pk, gP, gR, gP2, gRu, gG, ed, ced, qd, cd_s, cd_g, cd_m, tci, tct);
  if (mixed) {
    // one CTA per core, dispatched in descriptor order: the largest cores
    // (cost ~ n^3) first, so the end of each launch is not one big core
    auto larger = [](const CoreDesc& a, const CoreDesc& b) { return a.rt + a.k > b.rt + b.k; };
    for (auto* v : {&cd_s, &cd_m, &cd_g}) std::stable_sort(v->begin(), v->end(), larger);
  }
  const size_t o_ed = pk.add(ed), o_ce = pk.add(ced), o_qd = pk.add(qd), o_cs = pk.add(cd_s),
               o_cg = pk.add(cd_g);
  const size_t o_cm = pk.add(cd_m);
  const size_t o_ti = pk.add(tci), o_tt = pk.add(tct);
  char* dbase = ws.base + off_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), s));
  // from here on stream work only (memsets and launches on the workspace):
  // run now, or kept as a plan's operations
  std::vector<StreamOp> ops;
  char* wb = ws.base;
  // block energies start at zero (the mixed form sums its column energies)
  if (!mixed)
    ops.push_back([=](cudaStream_t st) {
      return cudaMemsetAsync(wb + energies, 0, sizeof(double) * (size_t)n, st);
    });
  if (mixed)
    ops.push_back([=](cudaStream_t st) {
      cudaError_t e = cudaMemsetAsync(wb + colE_base, 0, sizeof(double) * colE_total, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(wb + refine_flags, 0, (size_t)n, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(wb + refine_ctr, 0, sizeof(int), st);
      return e;
    });
  int max_chunks = 1;
  int max_m = 1;
  for (int i = 0; i < n; ++i) {
    const int64_t tot = items[i].m * items[i].blk->k;
    max_chunks = std::max<int>(max_chunks, (int)std::min<int64_t>(64, (tot + 8191) / 8192));
    max_m = std::max<int>(max_m, (int)items[i].m);
  }
  if (!mixed)
    ops.push_back([=](cudaStream_t st) {
      return launch_energy(reinterpret_cast<EnergyDesc*>(dbase + o_ed), n, max_chunks, st);
    });
  ops.push_back(gP.op(dbase));
  if (mixed) {
    int max_k = 1;
    for (const EnergyDesc& e : ced) max_k = std::max(max_k, e.k);
    const int n_ce = (int)ced.size(), n_tt = (int)tct.size(), n_sms = num_sms();
    const int n_g = (int)cd_g.size(), n_m = (int)cd_m.size(), n_s = (int)cd_s.size();
    const int nx0 = tri_nmax[0], nx1 = tri_nmax[1], nx2 = tri_nmax[2];
    ops.push_back([=](cudaStream_t st) {
      return launch_col_energy(reinterpret_cast<EnergyDesc*>(dbase + o_ce), n_ce, max_k, max_m, st);
    });
    ops.push_back([=](cudaStream_t st) {
      return launch_tc_gram(reinterpret_cast<TcItem*>(dbase + o_ti),
                            reinterpret_cast<TcTile*>(dbase + o_tt), n_tt, n_sms, d_status, st);
    });
    ops.push_back(gG.op(dbase));
    ops.push_back([=](cudaStream_t st) {
      cudaError_t e = launch_core_tridiag(2, reinterpret_cast<CoreDesc*>(dbase + o_cg), n_g, nx2,
                                          d_status, st);
      if (e == cudaSuccess)
        e = launch_core_tridiag(1, reinterpret_cast<CoreDesc*>(dbase + o_cm), n_m, nx1, d_status, st);
      if (e == cudaSuccess)
        e = launch_core_tridiag(0, reinterpret_cast<CoreDesc*>(dbase + o_cs), n_s, nx0, d_status, st);
      if (e == cudaSuccess)
        e = launch_core_refine64(reinterpret_cast<CoreDesc*>(dbase + o_cg), n_g,
                                 reinterpret_cast<CoreDesc*>(dbase + o_cm), n_m,
                                 reinterpret_cast<CoreDesc*>(dbase + o_cs), n_s,
                                 reinterpret_cast<double*>(wb + refine_work), refine_slots,
                                 refine_nmax, reinterpret_cast<int*>(wb + refine_ctr), d_status, st);
      return e;
    });
  } else {
    ops.push_back(gR.op(dbase));
    ops.push_back(gP2.op(dbase));
    ops.push_back(gRu.op(dbase));
    const int n_qd = (int)qd.size();
    ops.push_back([=](cudaStream_t st) {
      return launch_householder_qr(reinterpret_cast<QRDesc*>(dbase + o_qd), n_qd, max_m, st);
    });
    int sm = 0;
    for (auto& c : cd_s) {
      const int nc = c.rt + c.k, nr = c.rt + c.kp;
      sm = std::max(sm, (jacobi_scratch_floats(nc) + (nc + (nc & 1)) * nr) * 4);
    }
    int gm = 0;
    for (auto& c : cd_g) gm = std::max(gm, jacobi_scratch_floats(c.rt + c.k) * 4);
    const int n_s = (int)cd_s.size(), n_g = (int)cd_g.size();
    ops.push_back([=](cudaStream_t st) {
      cudaError_t e = launch_core_jacobi(reinterpret_cast<CoreDesc*>(dbase + o_cs), n_s, sm, d_status, st);
      if (e == cudaSuccess)
        e = launch_core_jacobi(reinterpret_cast<CoreDesc*>(dbase + o_cg), n_g, gm, d_status, st);
      return e;
    });
  }
  CSVD_TRY(run_or_keep(ops, s, plan));
  if (plan) {
    plan->bufs.push_back(ws.base);  // the plan owns the workspace now
    ws.base = nullptr;
    return CSVD_OK;
  }
  if (keep && n == 1 && !mixed) {
    keep->Rt = ws.at<float>(off[0].Rt);
    keep->tau = ws.at<float>(off[0].tau);
    keep->Wt = want_W ? ws.at<float>(off[0].Wt) : nullptr;
    keep->kp = off[0].kp;
    keep->nr = off[0].nr;
    keep->r_new = off[0].r_new;
  }
  return CSVD_OK;
}

// One Newton-Schulz step U <- U - U (U^T U - I) / 2 on the state's basis
// (U^T U accumulated in FP64): keeps U orthonormal to FP32 rounding across
// many appends.  The Gram form of the merge evaluation relies on it, since
// [U diag(s), A]^T [U diag(s), A] equals its Gram core only when U^T U = I.
static csvd_status reorthonormalize(csvd_state_s* st) {
  if (st->rt == 0) return CSVD_OK;
  cudaStream_t s = st->stream;
  const int r = st->rt;
  float* U = st->U[st->cur];
  float* Un = st->U[1 - st->cur];
  // descriptor sizes do not depend on the workspace address: size first
  auto make = [&](float* D) {
    GemmBatch g;
    g.add(gemm(U, st->r, 0, D, r, 0, Un, st->r, 0, (int)st->m, r, r, -0.5f, U, st->r, 0, 1.f));
    return g;
  };
  Pack probe;
  make(nullptr).pack(probe);
  Layout L;
  const size_t o_D = L.add(sizeof(float) * (size_t)r * r);
  const size_t o_desc = L.add(probe.buf.size());
  Workspace w;
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  float* D = w.at<float>(o_D);
  CUDA_TRY(launch_gram_dev(U, st->r, (int)st->m, r, D, s));
  GemmBatch g = make(D);
  Pack pk;
  g.pack(pk);
  CUDA_TRY(upload(w.base + o_desc, pk.buf.data(), pk.buf.size(), s));
  CUDA_TRY(g.launch(w.base + o_desc, s));
  st->cur = 1 - st->cur;
  return CSVD_OK;
}

// Tentative append of one block and commit of the rotated basis (Cor. 3):
// U_new = U W_top + Q_res W_bot.
static csvd_status append_commit(csvd_state_s* st, const csvd_block* A) {
  cudaStream_t s = st->stream;
  const int k = (int)A->k;
  const int kp = (int)std::min<int64_t>(k, st->m - st->rt);
  const int r_new = std::min(st->r, st->rt + kp);
  // small outputs of the evaluation
  Layout L;
  const size_t o_sig = L.add(sizeof(float) * std::max(r_new, 1));
  const size_t o_tail = L.add(sizeof(double) * 3);
  const size_t o_Zt = L.add(sizeof(float) * (size_t)std::max(r_new, 1) * st->m);
  const size_t tiles = (size_t)((st->m + kGemmBM - 1) / kGemmBM) * ((r_new + kGemmBN - 1) / kGemmBN);
  const size_t desc_cap = 1024 + sizeof(ApplyQDesc) + sizeof(GemmDesc) + tiles * sizeof(GemmTile);
  const size_t o_desc = L.add(desc_cap);
  Workspace w2;
  w2.s = s;
  w2.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w2.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  float* sig_new = w2.at<float>(o_sig);
  double* tails = w2.at<double>(o_tail);
  Item it{view_of(st), A, st->r, st->m, sig_new, tails + 1, nullptr, tails + 0, nullptr};
  Workspace ws;
  CommitKeep keep;
  CSVD_TRY(run_items({it}, 0.0, CSVD_PLAIN_FP32, s, st->status, ws, &keep, true));
  float* Zt = w2.at<float>(o_Zt);
  Pack pk;
  std::vector<ApplyQDesc> ad;
  if (kp > 0 && r_new > 0) {
    ad.push_back(ApplyQDesc{keep.Rt, st->m, keep.tau, keep.Wt, keep.nr, st->rt, Zt, st->m,
                            (int)st->m, kp, r_new, 0});
  } else {
    CUDA_TRY(cudaMemsetAsync(Zt, 0, sizeof(float) * (size_t)std::max(r_new, 1) * st->m, s));
  }
  GemmBatch gU;
  float* Unew = st->U[1 - st->cur];
  gU.add(gemm(st->U[st->cur], st->r, 0, keep.Wt, keep.nr, 1, Unew, st->r, 0, (int)st->m, r_new,
              st->rt, 1.f, Zt, st->m, 1, 1.f));
  const size_t o_ad = pk.add(ad);
  gU.pack(pk);
  if (pk.buf.size() > desc_cap) return fail(CSVD_ERR_ARG, "internal: descriptor region too small");
  char* dbase = w2.base + o_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), s));
  if (!ad.empty())
    CUDA_TRY(launch_apply_q(reinterpret_cast<ApplyQDesc*>(dbase + o_ad), 1, r_new, s));
  CUDA_TRY(gU.launch(dbase, s));
  CUDA_TRY(launch_state_commit(sig_new, r_new, st->sigma, tails + 0, tails + 1, st->scal, s));
  st->cur = 1 - st->cur;
  st->rt = r_new;
  st->nblocks += 1;
  return reorthonormalize(st);
}

// ================================================================ C ABI
extern "C" {

const char* csvd_last_error(void) { return g_err.c_str(); }
const char* csvd_version(void) { return "csvd 0.1 (sm_103a)"; }

csvd_status csvd_tune_set(int32_t edge_small, int32_t edge_medium) {
  if (!tridiag_set_edges(edge_small, edge_medium))
    return fail(CSVD_ERR_ARG, "launch-class edges out of range");
  return CSVD_OK;
}

csvd_status csvd_tune_get(int32_t* edge_small, int32_t* edge_medium) {
  if (!edge_small || !edge_medium) return fail(CSVD_ERR_ARG, "NULL argument");
  int a, b;
  tridiag_get_edges(&a, &b);
  *edge_small = a;
  *edge_medium = b;
  return CSVD_OK;
}

csvd_status csvd_debug_limits(int32_t jacobi_sweeps, int32_t solver_iters, int64_t wait_ns,
                              int32_t stall_gram) {
  cudaError_t e = jacobi_set_cap(jacobi_sweeps);
  if (e == cudaSuccess) e = tridiag_set_bisect_cap(solver_iters);
  if (e == cudaSuccess) e = refine64_set_bisect_cap(solver_iters);
  if (e == cudaSuccess) e = arrow_set_cap(solver_iters);
  if (e == cudaSuccess) e = tc_set_wait_ns(wait_ns, stall_gram);
  if (e != cudaSuccess) return fail(CSVD_ERR_CUDA, cudaGetErrorString(e));
  return CSVD_OK;
}

csvd_status csvd_set_allocator(csvd_alloc_fn alloc, csvd_free_fn free_, void* ctx) {
  if ((alloc == nullptr) != (free_ == nullptr))
    return fail(CSVD_ERR_ARG, "allocator and free must both be set or both be NULL");
  g_alloc = alloc;
  g_free = free_;
  g_actx = ctx;
  return CSVD_OK;
}

csvd_status csvd_incr_init(csvd_state* out, int64_t m, int32_t r, int32_t precision,
                           void* cuda_stream) {
  if (!out) return fail(CSVD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (m < 1 || m > 65536 || r < 1 || r > 1024 || r > m)
    return fail(CSVD_ERR_ARG, "need 1 <= r <= min(m, 1024), m <= 65536");
  if (precision != CSVD_PLAIN_FP32 && precision != CSVD_MIXED && precision != CSVD_GRAM_FP32)
    return fail(CSVD_ERR_ARG, "bad precision");
  csvd_state_s* st = new csvd_state_s();
  st->m = m;
  st->r = r;
  st->prec = precision;
  st->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&st->U[b], sizeof(float) * m * r);
  if (e == cudaSuccess) e = cudaMalloc(&st->sigma, sizeof(float) * r);
  if (e == cudaSuccess) e = cudaMalloc(&st->scal, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&st->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(st->scal, 0, sizeof(double) * 4, st->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->status, 0, sizeof(int), st->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->sigma, 0, sizeof(float) * r, st->stream);
  if (e != cudaSuccess) {
    csvd_incr_free(st);
    return fail(e == cudaErrorMemoryAllocation ? CSVD_ERR_OOM : CSVD_ERR_CUDA,
                std::string("state allocation: ") + cudaGetErrorString(e));
  }
  *out = st;
  return CSVD_OK;
}

csvd_status csvd_incr_free(csvd_state st) {
  if (!st) return CSVD_OK;
  if (st->stream || st->U[0]) cudaStreamSynchronize(st->stream);
  cudaFree(st->U[0]);
  cudaFree(st->U[1]);
  cudaFree(st->sigma);
  cudaFree(st->scal);
  cudaFree(st->status);
  delete st;
  return CSVD_OK;
}

csvd_status csvd_incr_append(csvd_state st, const csvd_block* A) {
  if (!st) return fail(CSVD_ERR_ARG, "state is NULL");
  CSVD_TRY(check_block(A, st->m));
  if (A->dtype != CSVD_F32) return fail(CSVD_ERR_UNIMPLEMENTED, "append takes f32 blocks");
  return append_commit(st, A);
}

csvd_status csvd_incr_load(csvd_state st, const float* U_dev, int64_t ldu, int32_t rt,
                           const float* sigma_host, double energy, double discarded) {
  if (!st) return fail(CSVD_ERR_ARG, "state is NULL");
  if (rt < 0 || rt > st->r || (rt > 0 && (!U_dev || !sigma_host || ldu < rt)))
    return fail(CSVD_ERR_ARG, "need 0 <= rt <= r, U and sigma for rt > 0, ldu >= rt");
  if (!(energy >= 0.0) || !(discarded >= 0.0)) return fail(CSVD_ERR_ARG, "negative energy");
  if (rt > 0) {
    CUDA_TRY(cudaMemcpy2DAsync(st->U[st->cur], sizeof(float) * st->r, U_dev, sizeof(float) * ldu,
                               sizeof(float) * rt, st->m, cudaMemcpyDeviceToDevice, st->stream));
    CUDA_TRY(cudaMemcpyAsync(st->sigma, sigma_host, sizeof(float) * rt, cudaMemcpyHostToDevice,
                             st->stream));
  }
  const double sc[2] = {energy, discarded};
  CUDA_TRY(cudaMemcpyAsync(st->scal, sc, sizeof(sc), cudaMemcpyHostToDevice, st->stream));
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  st->rt = rt;
  st->nblocks = rt > 0 ? 1 : 0;
  return CSVD_OK;
}

csvd_status csvd_incr_sigma(csvd_state st, float* sigma_host, int32_t* r_eff) {
  if (!st) return fail(CSVD_ERR_ARG, "state is NULL");
  if (r_eff) *r_eff = st->rt;
  if (sigma_host && st->rt > 0)
    CUDA_TRY(cudaMemcpyAsync(sigma_host, st->sigma, sizeof(float) * st->rt,
                             cudaMemcpyDeviceToHost, st->stream));
  return take_status(st->status, st->stream);
}

csvd_status csvd_incr_basis(csvd_state st, float* U_dev, int64_t ldu) {
  if (!st || !U_dev) return fail(CSVD_ERR_ARG, "NULL argument");
  if (st->rt == 0) return CSVD_OK;
  if (ldu < st->rt) return fail(CSVD_ERR_ARG, "ldu < r_eff");
  CUDA_TRY(cudaMemcpy2DAsync(U_dev, sizeof(float) * ldu, st->U[st->cur], sizeof(float) * st->r,
                             sizeof(float) * st->rt, st->m, cudaMemcpyDeviceToDevice, st->stream));
  return CSVD_OK;
}

csvd_status csvd_tail_error(csvd_state st, double* tail_sq, double* tail_rel,
                            double* tail_sq_paper, double* energy) {
  if (!st) return fail(CSVD_ERR_ARG, "state is NULL");
  double h[2] = {0, 0};
  std::vector<float> sg(std::max(st->rt, 1));
  CUDA_TRY(cudaMemcpyAsync(h, st->scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, st->stream));
  if (st->rt > 0)
    CUDA_TRY(cudaMemcpyAsync(sg.data(), st->sigma, sizeof(float) * st->rt,
                             cudaMemcpyDeviceToHost, st->stream));
  CSVD_TRY(take_status(st->status, st->stream));
  if (tail_sq) *tail_sq = h[1];
  if (tail_rel) *tail_rel = h[0] > 0 ? std::sqrt(h[1] / h[0]) : 0.0;
  if (tail_sq_paper) {
    double top = 0.0;
    for (int i = 0; i < st->rt; ++i) top += (double)sg[i] * (double)sg[i];
    *tail_sq_paper = std::max(0.0, h[0] - top);
  }
  if (energy) *energy = h[0];
  return CSVD_OK;
}

}  // extern "C"

// Items of a batched evaluation (csvd_score's arguments, checked).
static csvd_status score_items(const csvd_state* states, int32_t n_states,
                               const int32_t* cand_state, const csvd_block* cands, int32_t n,
                               int32_t precision, float* sigma_out, int64_t ld_sigma,
                               double* tail_sq_out, double* tail_paper_out, uint8_t* accept_out,
                               std::vector<Item>& items) {
  if (!states || n_states < 1 || !cands || n < 0 || !sigma_out || !tail_sq_out)
    return fail(CSVD_ERR_ARG, "NULL argument");
  if (precision != CSVD_PLAIN_FP32 && precision != CSVD_MIXED && precision != CSVD_GRAM_FP32)
    return fail(CSVD_ERR_ARG, "bad precision");
  if (!states[0]) return fail(CSVD_ERR_ARG, "state 0 is NULL");
  const int64_t m = states[0]->m;
  items.resize(n);
  for (int i = 0; i < n; ++i) {
    const int si = cand_state ? cand_state[i] : 0;
    if (si < 0 || si >= n_states || !states[si]) return fail(CSVD_ERR_ARG, "bad cand_state");
    if (states[si]->m != m) return fail(CSVD_ERR_SHAPE, "states differ in m");
    CSVD_TRY(check_block(&cands[i], m));
    if (ld_sigma < states[si]->r) return fail(CSVD_ERR_ARG, "ld_sigma < r");
    items[i] = Item{view_of(states[si]), &cands[i], states[si]->r, m, sigma_out + (int64_t)i * ld_sigma,
                    tail_sq_out + i, tail_paper_out ? tail_paper_out + i : nullptr, nullptr,
                    accept_out ? accept_out + i : nullptr};
  }
  return CSVD_OK;
}

struct csvd_plan_s {
  LaunchPlan lp;
};

static void plan_release(csvd_plan_s* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  for (void* b : p->lp.bufs) dev_free(b, p->lp.s);
  cudaStreamSynchronize(p->lp.s);
  delete p;
}

extern "C" {

csvd_status csvd_score(const csvd_state* states, int32_t n_states, const int32_t* cand_state,
                       const csvd_block* cands, int32_t n, double eps, int32_t precision,
                       float* sigma_out, int64_t ld_sigma, double* tail_sq_out,
                       double* tail_paper_out, uint8_t* accept_out) {
  std::vector<Item> items;
  CSVD_TRY(score_items(states, n_states, cand_state, cands, n, precision, sigma_out, ld_sigma,
                       tail_sq_out, tail_paper_out, accept_out, items));
  if (n == 0) return CSVD_OK;
  Workspace ws;
  return run_items(items, eps, precision, states[0]->stream, states[0]->status, ws, nullptr, false);
}

csvd_status csvd_score_plan(const csvd_state* states, int32_t n_states, const int32_t* cand_state,
                            const csvd_block* cands, int32_t n, double eps, int32_t precision,
                            float* sigma_out, int64_t ld_sigma, double* tail_sq_out,
                            double* tail_paper_out, uint8_t* accept_out, csvd_plan* out) {
  if (!out) return fail(CSVD_ERR_ARG, "NULL argument");
  *out = nullptr;
  std::vector<Item> items;
  CSVD_TRY(score_items(states, n_states, cand_state, cands, n, precision, sigma_out, ld_sigma,
                       tail_sq_out, tail_paper_out, accept_out, items));
  cudaStream_t s = states[0]->stream;
  auto* p = new csvd_plan_s;
  p->lp.s = s;
  p->lp.status = static_cast<int*>(dev_alloc(sizeof(int), s));
  if (!p->lp.status) {
    delete p;
    return fail(CSVD_ERR_OOM, "plan status allocation failed");
  }
  p->lp.bufs.push_back(p->lp.status);
  csvd_status st = CSVD_OK;
  if (cudaMemsetAsync(p->lp.status, 0, sizeof(int), s) != cudaSuccess)
    st = fail(CSVD_ERR_CUDA, "plan status memset failed");
  if (st == CSVD_OK && n > 0) {
    Workspace ws;
    st = run_items(items, eps, precision, s, p->lp.status, ws, nullptr, false, &p->lp);
  }
  if (st == CSVD_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = fail(CSVD_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  if (st != CSVD_OK) {
    plan_release(p);
    return st;
  }
  *out = p;
  return CSVD_OK;
}

csvd_status csvd_plan_launch(csvd_plan p, void* cuda_stream) {
  if (!p) return fail(CSVD_ERR_ARG, "plan is NULL");
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : p->lp.s;
  for (auto& op : p->lp.ops) CUDA_TRY(op(s));
  return CSVD_OK;
}

csvd_status csvd_plan_status(csvd_plan p, void* cuda_stream) {
  if (!p) return fail(CSVD_ERR_ARG, "plan is NULL");
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : p->lp.s;
  return take_status(p->lp.status, s);
}

csvd_status csvd_plan_free(csvd_plan p) {
  if (!p) return fail(CSVD_ERR_ARG, "plan is NULL");
  plan_release(p);
  return CSVD_OK;
}

}  // extern "C"

// Rows of csvd_score_columns in CTA groups {first row, count, state, 0}: runs
// of adjacent rows of one state, at most kArrowGroup each; rows whose state
// cannot take the one-column core go to `rest` in order.
static csvd_status arrow_row_groups(const int32_t* cand_state, int n, int n_states,
                                    const std::vector<char>& arrow_ok, std::vector<int4>& groups,
                                    std::vector<int>& rest) {
  groups.clear();
  rest.clear();
  for (int j = 0; j < n; ++j) {
    const int si = cand_state ? cand_state[j] : 0;
    if (si < 0 || si >= n_states) return fail(CSVD_ERR_ARG, "bad cand_state");
    if (!arrow_ok[si]) {
      rest.push_back(j);
      continue;
    }
    if (groups.empty() || groups.back().z != si || groups.back().y == kArrowGroup ||
        groups.back().x + groups.back().y != j)
      groups.push_back(make_int4(j, 0, si, 0));
    ++groups.back().y;
  }
  return CSVD_OK;
}

extern "C" {

csvd_status csvd_score_columns(const csvd_state* states, int32_t n_states,
                               const int32_t* cand_state, const float* Xt, int64_t ldx, int32_t n,
                               double eps, float* sigma_out, int64_t ld_sigma, double* tail_sq_out,
                               double* tail_paper_out, uint8_t* accept_out) {
  if (!states || n_states < 1 || n < 0 || (n > 0 && (!Xt || !sigma_out || !tail_sq_out)))
    return fail(CSVD_ERR_ARG, "NULL argument");
  if (n == 0) return CSVD_OK;
  const int64_t m = states[0]->m;
  if (ldx < m) return fail(CSVD_ERR_ARG, "ldx < m");
  cudaStream_t s = states[0]->stream;
  std::vector<ArrowState> tab(n_states);
  std::vector<char> arrow_ok(n_states, 0);
  for (int i = 0; i < n_states; ++i) {
    if (!states[i]) return fail(CSVD_ERR_ARG, "NULL state");
    if (states[i]->m != m) return fail(CSVD_ERR_SHAPE, "states differ in m");
    const StateView v = view_of(states[i]);
    tab[i] = ArrowState{v.U, v.ldu, m, v.rt,
                        (int)std::min<int64_t>(v.r, v.rt + std::min<int64_t>(1, m - v.rt)),
                        v.sigma, v.scal};
    arrow_ok[i] = v.rt <= kArrowMaxRt;
  }
  // runs of adjacent rows of one state, up to kArrowGroup per CTA; rows of
  // states past the one-column core's limit take the general path
  std::vector<int4> groups;
  std::vector<int> rest_rows;
  CSVD_TRY(arrow_row_groups(cand_state, n, n_states, arrow_ok, groups, rest_rows));
  for (int j = 0; j < n; ++j)
    if (ld_sigma < states[cand_state ? cand_state[j] : 0]->r)
      return fail(CSVD_ERR_ARG, "ld_sigma < r");
  std::vector<csvd_block> rest_blocks;
  for (int j : rest_rows) rest_blocks.push_back(csvd_block{Xt + (int64_t)j * ldx, 1, 1, CSVD_F32, 0});
  if (!groups.empty()) {
    const size_t tab_bytes = sizeof(ArrowState) * n_states, grp_bytes = sizeof(int4) * groups.size();
    const size_t grp_off = (tab_bytes + 15) & ~size_t(15);
    std::vector<char> host(grp_off + grp_bytes, 0);
    std::memcpy(host.data(), tab.data(), tab_bytes);
    std::memcpy(host.data() + grp_off, groups.data(), grp_bytes);
    Workspace w;
    w.s = s;
    w.base = static_cast<char*>(dev_alloc(host.size(), s));
    if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
    CUDA_TRY(upload(w.base, host.data(), host.size(), s));
    CUDA_TRY(launch_core_arrow_columns(w.at<ArrowState>(0), w.at<int4>(grp_off),
                                       (int)groups.size(), Xt, ldx, sigma_out, ld_sigma,
                                       tail_sq_out, tail_paper_out, accept_out, eps,
                                       states[0]->status, s));
  }
  if (!rest_rows.empty()) {
    std::vector<Item> items(rest_rows.size());
    for (size_t i = 0; i < rest_rows.size(); ++i) {
      const int j = rest_rows[i];
      const int si = cand_state ? cand_state[j] : 0;
      items[i] = Item{view_of(states[si]), &rest_blocks[i], states[si]->r, m,
                      sigma_out + (int64_t)j * ld_sigma, tail_sq_out + j,
                      tail_paper_out ? tail_paper_out + j : nullptr, nullptr,
                      accept_out ? accept_out + j : nullptr};
    }
    Workspace ws;
    CSVD_TRY(run_items_general(items, eps, CSVD_MIXED, s, states[0]->status, ws, nullptr, false));
  }
  return CSVD_OK;
}

// ------------------------------------------------ streaming assignment
}  // extern "C"

struct csvd_stream_s {
  int64_t m = 0;
  int r = 0;
  double eps = 0.0;
  int prec = 0;
  cudaStream_t s = nullptr;
  std::vector<csvd_state> clusters;
  std::vector<int32_t> sizes;  // blocks per cluster
};

extern "C" {

csvd_status csvd_stream_init(csvd_stream* out, int64_t m, int32_t r, double eps,
                             int32_t precision, void* cuda_stream) {
  if (!out) return fail(CSVD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (m < 1 || m > 65536 || r < 1 || r > 1024 || r > m)
    return fail(CSVD_ERR_ARG, "need 1 <= r <= min(m, 1024), m <= 65536");
  if (!(eps >= 0.0)) return fail(CSVD_ERR_ARG, "need eps >= 0");
  if (precision != CSVD_PLAIN_FP32 && precision != CSVD_MIXED && precision != CSVD_GRAM_FP32)
    return fail(CSVD_ERR_ARG, "bad precision");
  csvd_stream_s* h = new csvd_stream_s();
  h->m = m;
  h->r = r;
  h->eps = eps;
  h->prec = precision;
  h->s = static_cast<cudaStream_t>(cuda_stream);
  *out = h;
  return CSVD_OK;
}

csvd_status csvd_stream_push(csvd_stream h, const csvd_block* block, int32_t* label_out,
                             double* tail_sq_out, double* energy_out) {
  if (!h || !block) return fail(CSVD_ERR_ARG, "NULL argument");
  CSVD_TRY(check_block(block, h->m));
  const int C = (int)h->clusters.size();
  int best = -1;
  if (C > 0) {
    // one batched evaluation of the block against every open cluster
    Layout L;
    const size_t o_sig = L.add(sizeof(float) * (size_t)C * h->r);
    const size_t o_t = L.add(sizeof(double) * C);
    const size_t o_e = L.add(sizeof(double) * C);
    Workspace w;
    w.s = h->s;
    w.base = static_cast<char*>(dev_alloc(L.size, h->s));
    if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
    std::vector<Item> items(C);
    for (int c = 0; c < C; ++c)
      items[c] = Item{view_of(h->clusters[c]), block, h->r, h->m,
                      w.at<float>(o_sig) + (size_t)c * h->r, w.at<double>(o_t) + c, nullptr,
                      w.at<double>(o_e) + c, nullptr};
    int* d_status = h->clusters[0]->status;
    {
      Workspace ws;
      CSVD_TRY(run_items(items, h->eps, h->prec, h->s, d_status, ws, nullptr, false));
    }
    std::vector<double> tail(C), energy(C);
    CUDA_TRY(cudaMemcpyAsync(tail.data(), w.base + o_t, sizeof(double) * C, cudaMemcpyDeviceToHost,
                             h->s));
    CUDA_TRY(cudaMemcpyAsync(energy.data(), w.base + o_e, sizeof(double) * C,
                             cudaMemcpyDeviceToHost, h->s));
    CSVD_TRY(take_status(d_status, h->s));
    // best fit: the smallest estimated relative error among the clusters
    // that accept (ties to the lowest index)
    const double e2 = h->eps * h->eps;
    double best_rel = 0.0;
    for (int c = 0; c < C; ++c) {
      if (!(tail[c] <= e2 * energy[c])) continue;
      const double rel = energy[c] > 0.0 ? tail[c] / energy[c] : 0.0;
      if (best < 0 || rel < best_rel) {
        best = c;
        best_rel = rel;
      }
    }
  }
  if (best < 0) {
    csvd_state st = nullptr;
    CSVD_TRY(csvd_incr_init(&st, h->m, h->r, h->prec, h->s));
    const csvd_status rc = append_commit(st, block);
    if (rc != CSVD_OK) {
      csvd_incr_free(st);
      return rc;
    }
    h->clusters.push_back(st);
    h->sizes.push_back(1);
    best = C;
  } else {
    CSVD_TRY(append_commit(h->clusters[best], block));
    h->sizes[best] += 1;
  }
  if (label_out) *label_out = best;
  if (tail_sq_out || energy_out) {
    double t = 0.0, en = 0.0;
    CSVD_TRY(csvd_tail_error(h->clusters[best], &t, nullptr, nullptr, &en));
    if (tail_sq_out) *tail_sq_out = t;
    if (energy_out) *energy_out = en;
  }
  return CSVD_OK;
}

csvd_status csvd_stream_count(csvd_stream h, int32_t* n_clusters) {
  if (!h || !n_clusters) return fail(CSVD_ERR_ARG, "NULL argument");
  *n_clusters = (int32_t)h->clusters.size();
  return CSVD_OK;
}

csvd_status csvd_stream_cluster(csvd_stream h, int32_t c, csvd_state* state_out,
                                int32_t* n_blocks_out) {
  if (!h) return fail(CSVD_ERR_ARG, "NULL argument");
  if (c < 0 || c >= (int32_t)h->clusters.size()) return fail(CSVD_ERR_ARG, "no such cluster");
  if (state_out) *state_out = h->clusters[c];
  if (n_blocks_out) *n_blocks_out = h->sizes[c];
  return CSVD_OK;
}

csvd_status csvd_selftest(char* msg, int64_t cap) {
  std::string err = tridiag_selftest();
  if (err.empty()) {
    // candidate grouping of csvd_score_columns on pseudo-random patterns
    uint64_t x = 0x9E3779B97F4A7C15ull;
    auto next = [&x](int mod) {
      x ^= x << 13;
      x ^= x >> 7;
      x ^= x << 17;
      return (int)(x % (uint64_t)mod);
    };
    for (int trial = 0; trial < 500 && err.empty(); ++trial) {
      const int n = 1 + next(200), n_states = 1 + next(6);
      std::vector<char> ok(n_states);
      for (auto& o : ok) o = next(4) != 0;
      std::vector<int32_t> cs(n);
      for (int j = 0; j < n; ++j) cs[j] = (j > 0 && next(3) != 0) ? cs[j - 1] : next(n_states);
      std::vector<int4> groups;
      std::vector<int> rest;
      if (arrow_row_groups(cs.data(), n, n_states, ok, groups, rest) != CSVD_OK) {
        err = "row grouping rejected a valid pattern";
        break;
      }
      std::vector<int> seen(n, 0);
      for (const int4& g : groups) {
        if (g.y < 1 || g.y > kArrowGroup || !ok[g.z]) err = "row group size or state";
        for (int t = 0; t < g.y && err.empty(); ++t) {
          if (g.x + t >= n || cs[g.x + t] != g.z) err = "row group not one state";
          else ++seen[g.x + t];
        }
      }
      for (int j : rest) {
        if (ok[cs[j]]) err = "row sent to the general path needlessly";
        ++seen[j];
      }
      for (int j = 0; j < n && err.empty(); ++j)
        if (seen[j] != 1) err = "row not covered exactly once";
    }
    // CTA groups of one-column items handed to csvd_score: fake states
    // (pointers compared, never dereferenced), some sharing U but not r
    for (int trial = 0; trial < 500 && err.empty(); ++trial) {
      // states 3t, 3t+1, 3t+2 share U and r_t; 3t+1 differs from 3t only in
      // r, 3t+2 only in sigma and the energy scalars
      const int n = 1 + next(150), n_states = 1 + next(9);
      std::vector<Item> items(n);
      std::vector<int> sid(n);
      for (int i = 0; i < n; ++i) {
        const int si = sid[i] = next(n_states), t = si / 3, u = si % 3;
        Item& it = items[i];
        it.st.U = reinterpret_cast<const float*>(uintptr_t(0x10000) * (uintptr_t)(1 + t));
        it.st.ldu = 32;
        it.st.rt = 8 + t;
        it.st.r = it.r = 16 + (u == 1 ? 1 : 0);
        it.st.sigma = reinterpret_cast<const float*>(uintptr_t(0x900000) + 64 * (uintptr_t)(3 * t + (u == 2 ? 2 : 0)));
        it.st.scal = reinterpret_cast<const double*>(uintptr_t(0xA00000) + 64 * (uintptr_t)(3 * t + (u == 2 ? 2 : 0)));
        it.m = 64;
      }
      std::vector<int> order;
      std::vector<int2> groups;
      arrow_item_groups(items, order, groups);
      std::vector<int> seen(n, 0), pos_seen(n, 0);
      for (int i : order) ++seen[i];
      int next_pos = 0;
      for (const int2& g : groups) {
        if (g.x != next_pos || g.y < 1 || g.y > kArrowGroup || g.x + g.y > n) {
          err = "item groups not a partition of the order";
          break;
        }
        for (int t = 0; t < g.y; ++t)
          if (sid[order[g.x + t]] != sid[order[g.x]]) err = "item group mixes states";
        next_pos += g.y;
      }
      if (err.empty() && next_pos != n) err = "item groups do not cover the order";
      for (int i = 0; i < n && err.empty(); ++i)
        if (seen[i] != 1) err = "item order not a permutation";
    }
  }
  if (msg && cap > 0) {
    std::strncpy(msg, err.empty() ? "ok" : err.c_str(), (size_t)cap - 1);
    msg[cap - 1] = 0;
  }
  return err.empty() ? CSVD_OK : fail(CSVD_ERR_SHAPE, err.c_str());
}

csvd_status csvd_stream_free(csvd_stream h) {
  if (!h) return CSVD_OK;
  csvd_status rc = CSVD_OK;
  for (csvd_state st : h->clusters) {
    const csvd_status r2 = csvd_incr_free(st);
    if (rc == CSVD_OK) rc = r2;
  }
  delete h;
  return rc;
}

}  // extern "C"

// ====================================================== internal helpers
// Empty-state view (r_t = 0) used for per-block spectra.
static StateView empty_view(const double* zero_scal) {
  return StateView{nullptr, 1, 0, 0, nullptr, zero_scal};
}

// Per-block top-r energies, energies and spectra via empty-state evaluations.
static csvd_status block_spectra(const csvd_block* blocks, const std::vector<int>& idx, int64_t m,
                                 int r, int precision, cudaStream_t s, int* d_status,
                                 std::vector<double>& energy, std::vector<double>& top,
                                 std::vector<std::vector<float>>* spectra) {
  const int n = (int)idx.size();
  energy.assign(n, 0.0);
  top.assign(n, 0.0);
  if (spectra) spectra->assign(n, {});
  if (n == 0) return CSVD_OK;
  Layout L;
  const size_t o_z = L.add(sizeof(double) * 4);
  const size_t o_sig = L.add(sizeof(float) * (size_t)n * r);
  const size_t o_t = L.add(sizeof(double) * n);
  const size_t o_e = L.add(sizeof(double) * n);
  Workspace w;
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  CUDA_TRY(cudaMemsetAsync(w.base + o_z, 0, sizeof(double) * 4, s));
  std::vector<Item> items(n);
  for (int i = 0; i < n; ++i)
    items[i] = Item{empty_view(w.at<double>(o_z)), &blocks[idx[i]], r, m, w.at<float>(o_sig) + (size_t)i * r,
                    w.at<double>(o_t) + i, nullptr, w.at<double>(o_e) + i, nullptr};
  Workspace ws;
  CSVD_TRY(run_items(items, 0.0, precision, s, d_status, ws, nullptr, false));
  std::vector<double> tl(n);
  std::vector<float> sg((size_t)n * r);
  CUDA_TRY(cudaMemcpyAsync(tl.data(), w.base + o_t, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(energy.data(), w.base + o_e, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (spectra)
    CUDA_TRY(cudaMemcpyAsync(sg.data(), w.base + o_sig, sizeof(float) * n * r, cudaMemcpyDeviceToHost, s));
  CSVD_TRY(take_status(d_status, s));
  for (int i = 0; i < n; ++i) {
    top[i] = std::max(0.0, energy[i] - tl[i]);
    if (spectra) {
      const int rn = (int)std::min<int64_t>({(int64_t)r, blocks[idx[i]].k, m});
      (*spectra)[i].assign(sg.begin() + (size_t)i * r, sg.begin() + (size_t)i * r + rn);
    }
  }
  return CSVD_OK;
}

// ||A_j||_F^2 for the listed blocks (host result).
static csvd_status block_energies(const csvd_block* blocks, const std::vector<int>& idx, int64_t m,
                                  cudaStream_t s, std::vector<double>& out) {
  const int n = (int)idx.size();
  out.assign(n, 0.0);
  if (n == 0) return CSVD_OK;
  std::vector<EnergyDesc> ed(n);
  Layout L;
  const size_t o_e = L.add(sizeof(double) * n);
  const size_t o_d = L.add(sizeof(EnergyDesc) * n);
  Workspace w;
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  int chunks = 1;
  for (int i = 0; i < n; ++i) {
    const csvd_block& b = blocks[idx[i]];
    ed[i] = EnergyDesc{b.ptr, b.ld, (int)m, (int)b.k, b.dtype == CSVD_BF16, 0, w.at<double>(o_e) + i};
    chunks = std::max<int>(chunks, (int)std::min<int64_t>(64, (m * b.k + 8191) / 8192));
  }
  CUDA_TRY(cudaMemsetAsync(w.base + o_e, 0, sizeof(double) * n, s));
  CUDA_TRY(upload(w.base + o_d, ed.data(), sizeof(EnergyDesc) * n, s));
  CUDA_TRY(launch_energy(w.at<EnergyDesc>(o_d), n, chunks, s));
  CUDA_TRY(cudaMemcpyAsync(out.data(), w.base + o_e, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return CSVD_OK;
}

// Full-span residual state of Alg. 2 / Cor. 1: basis Qf (m x rho, row-major ld m).
struct SpanState {
  int64_t m = 0;
  int rho = 0;
  float* Qf = nullptr;        // m x m capacity, ld = m (from the installed allocator)
  cudaStream_t s = nullptr;   // stream of Qf's allocation
  double energy = 0.0;
  double proj = 0.0;          // sum_i ||Q_{i-1}^T A_i||^2 over the accepted blocks
  std::vector<double> mu;     // residual singular values (multiset)
  bool alloc(int64_t m_, cudaStream_t st) {
    m = m_;
    s = st;
    Qf = static_cast<float*>(dev_alloc(sizeof(float) * (size_t)m * m, s));
    return Qf != nullptr;
  }
  ~SpanState() { dev_free(Qf, s); }
};

// R_j = (I - Qf Qf^T) A_j (one re-orthogonalisation pass) for several blocks,
// written row-major into `R` (each m x k_j, ld k_j, consecutive).
static csvd_status span_residuals(const SpanState& sp, const csvd_block* blocks,
                                  const std::vector<int>& idx, cudaStream_t s, Workspace& w,
                                  std::vector<csvd_block>& out, std::vector<double>& proj) {
  const int n = (int)idx.size();
  Layout L;
  std::vector<size_t> oR(n), oP(n), oP2(n);
  for (int i = 0; i < n; ++i) {
    const int k = (int)blocks[idx[i]].k;
    oR[i] = L.add(sizeof(float) * (size_t)sp.m * k);
    oP[i] = L.add(sizeof(float) * (size_t)std::max(sp.rho, 1) * k);
    oP2[i] = L.add(sizeof(float) * (size_t)std::max(sp.rho, 1) * k);
  }
  const size_t o_pe = L.add(sizeof(double) * n);
  GemmBatch g1, g2, g3, g4;
  std::vector<EnergyDesc> ed;
  auto fill = [&](char* base) {
    g1 = GemmBatch(); g2 = GemmBatch(); g3 = GemmBatch(); g4 = GemmBatch();
    ed.clear();
    for (int i = 0; i < n; ++i) {
      const csvd_block& b = blocks[idx[i]];
      const int k = (int)b.k;
      float* R = reinterpret_cast<float*>(base + oR[i]);
      float* P = reinterpret_cast<float*>(base + oP[i]);
      float* P2 = reinterpret_cast<float*>(base + oP2[i]);
      if (sp.rho > 0) g1.add(gemm(sp.Qf, sp.m, 1, b.ptr, b.ld, 0, P, k, 0, sp.rho, k, (int)sp.m));
      g2.add(gemm(sp.Qf, sp.m, 0, P, k, 0, R, k, 0, (int)sp.m, k, sp.rho, -1.f,
                  reinterpret_cast<const float*>(b.ptr), b.ld, 0, 1.f));
      if (sp.rho > 0) {
        g3.add(gemm(sp.Qf, sp.m, 1, R, k, 0, P2, k, 0, sp.rho, k, (int)sp.m));
        g4.add(gemm(sp.Qf, sp.m, 0, P2, k, 0, R, k, 0, (int)sp.m, k, sp.rho, -1.f, R, k, 0, 1.f));
        ed.push_back(EnergyDesc{P, k, sp.rho, k, 0, 0, reinterpret_cast<double*>(base + o_pe) + i});
      }
    }
  };
  fill(reinterpret_cast<char*>(uintptr_t(1) << 20));
  Pack probe;
  g1.pack(probe); g2.pack(probe); g3.pack(probe); g4.pack(probe);
  probe.add(ed);
  const size_t o_desc = L.add(probe.buf.size());
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  fill(w.base);
  Pack pk;
  g1.pack(pk); g2.pack(pk); g3.pack(pk); g4.pack(pk);
  const size_t o_ed = pk.add(ed);
  char* dbase = w.base + o_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), s));
  CUDA_TRY(cudaMemsetAsync(w.base + o_pe, 0, sizeof(double) * n, s));
  CUDA_TRY(g1.launch(dbase, s));
  CUDA_TRY(g2.launch(dbase, s));
  CUDA_TRY(g3.launch(dbase, s));
  CUDA_TRY(g4.launch(dbase, s));
  if (!ed.empty()) CUDA_TRY(launch_energy(reinterpret_cast<EnergyDesc*>(dbase + o_ed), (int)ed.size(), 8, s));
  proj.assign(n, 0.0);
  CUDA_TRY(cudaMemcpyAsync(proj.data(), w.base + o_pe, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  out.resize(n);
  for (int i = 0; i < n; ++i)
    out[i] = csvd_block{w.base + oR[i], blocks[idx[i]].k, blocks[idx[i]].k, CSVD_F32, 0};
  return CSVD_OK;
}

// Extend Qf by the left singular vectors of R whose singular values exceed
// tol (rank-revealing step of Thm. 2's full-span basis).
static csvd_status span_extend(SpanState& sp, const csvd_block& R, const std::vector<float>& sv,
                               double tol, cudaStream_t s) {
  int q = 0;
  while (q < (int)sv.size() && (double)sv[q] > tol && sp.rho + q < sp.m) ++q;
  if (q == 0) return CSVD_OK;
  csvd_state tmp = nullptr;
  const int rk = (int)std::min<int64_t>(R.k, sp.m);
  CSVD_TRY(csvd_incr_init(&tmp, sp.m, rk, CSVD_PLAIN_FP32, s));
  csvd_status st = append_commit(tmp, &R);
  if (st == CSVD_OK) {
    q = std::min(q, tmp->rt);
    cudaError_t e = cudaMemcpy2DAsync(sp.Qf + sp.rho, sizeof(float) * sp.m, tmp->U[tmp->cur],
                                      sizeof(float) * tmp->r, sizeof(float) * q, sp.m,
                                      cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = fail(CSVD_ERR_CUDA, cudaGetErrorString(e));
    sp.rho += q;
  }
  csvd_incr_free(tmp);
  return st;
}

// sum of mu^2 beyond the r largest: with the projection energies this gives
// Cor. 1's bound  S - sum_{j<=r} mu_j^2 = sum_i ||Q_{i-1}^T A_i||^2 +
// sum_{j>r} mu_j^2  (since ||A_i||^2 = ||Q^T A_i||^2 + ||R_i||^2 and
// sum_j mu_j^2 = sum_i ||R_i||^2), a sum of non-negative terms free of the
// subtraction's cancellation.
static double rest_sum_sq(std::vector<double> v, int r) {
  std::sort(v.begin(), v.end(), std::greater<double>());
  double t = 0.0;
  for (int i = r; i < (int)v.size(); ++i) t += v[i] * v[i];
  return t;
}

extern "C" csvd_status csvd_bounds(const csvd_block* blocks, int32_t n, int64_t m, int32_t r,
                                   void* cuda_stream, double* weyl_sq, double* residual_sq,
                                   double* plugin_sq, double* energy) {
  if (!blocks || n < 1 || m < 1 || r < 1 || r > m) return fail(CSVD_ERR_ARG, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < n; ++i) {
    CSVD_TRY(check_block(&blocks[i], m));
    if (blocks[i].dtype != CSVD_F32) return fail(CSVD_ERR_UNIMPLEMENTED, "bounds take f32 blocks");
  }
  Workspace ws_status;
  ws_status.s = s;
  ws_status.base = static_cast<char*>(dev_alloc(sizeof(int), s));
  if (!ws_status.base) return fail(CSVD_ERR_OOM, "status allocation failed");
  int* d_status = ws_status.at<int>(0);
  CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), s));
  std::vector<int> all(n);
  std::iota(all.begin(), all.end(), 0);
  std::vector<double> en, top;
  csvd_status st = block_spectra(blocks, all, m, r, CSVD_PLAIN_FP32, s, d_status, en, top, nullptr);
  double S = 0.0;
  int jstar = 0;
  for (int i = 0; i < n; ++i) {
    S += en[i];
    if (top[i] > top[jstar]) jstar = i;
  }
  if (st == CSVD_OK && energy) *energy = S;
  if (st == CSVD_OK && weyl_sq) {
    // Thm. 1: S - top_r(A_j*) = sum_{i != j*} ||A_i||^2 + sum_{l>r} sigma_l^2(A_j*)
    double others = 0.0;
    for (int i = 0; i < n; ++i)
      if (i != jstar) others += en[i];
    *weyl_sq = others + std::max(0.0, en[jstar] - top[jstar]);
  }
  if (st == CSVD_OK && residual_sq) {
    SpanState sp;
    if (!sp.alloc(m, s)) st = fail(CSVD_ERR_OOM, "span basis allocation failed");
    double Ssofar = 0.0;
    for (int i = 0; i < n && st == CSVD_OK; ++i) {
      Workspace w;
      std::vector<csvd_block> R;
      std::vector<double> pe;
      st = span_residuals(sp, blocks, {i}, s, w, R, pe);
      if (st != CSVD_OK) break;
      sp.proj += pe[0];
      std::vector<double> e1, t1;
      std::vector<std::vector<float>> sv;
      const int rk = (int)std::min<int64_t>(blocks[i].k, m);
      st = block_spectra(R.data(), {0}, m, rk, CSVD_PLAIN_FP32, s, d_status, e1, t1, &sv);
      if (st != CSVD_OK) break;
      for (float x : sv[0]) sp.mu.push_back(x);
      Ssofar += en[i];
      st = span_extend(sp, R[0], sv[0], 1e-6 * std::sqrt(Ssofar), s);
    }
    if (st == CSVD_OK) *residual_sq = sp.proj + rest_sum_sq(sp.mu, r);
  }
  if (st == CSVD_OK && plugin_sq) {
    csvd_state inc = nullptr;
    st = csvd_incr_init(&inc, m, r, CSVD_PLAIN_FP32, s);
    for (int i = 0; i < n && st == CSVD_OK; ++i) st = csvd_incr_append(inc, &blocks[i]);
    if (st == CSVD_OK) st = csvd_tail_error(inc, plugin_sq, nullptr, nullptr, nullptr);
    csvd_incr_free(inc);
  }
  cudaStreamSynchronize(s);
  return st;
}

// ================================================================ clustering
namespace {

struct Driver {
  const csvd_block* blocks;
  int n;
  int64_t m;
  int r;
  double eps;
  int precision;
  cudaStream_t s;
  int* d_status;
  std::vector<double> norms;   // ||A_j||^2
  std::vector<int> widths;
};

// Score candidates `cand` against an incremental state; returns E~^2 and
// the post-merge energies (host).
csvd_status score_state(Driver& D, csvd_state st, const std::vector<int>& cand,
                        std::vector<double>& tail, std::vector<double>& energy) {
  const int n = (int)cand.size();
  tail.assign(n, 0.0);
  energy.assign(n, 0.0);
  if (n == 0) return CSVD_OK;
  Layout L;
  const size_t o_sig = L.add(sizeof(float) * (size_t)n * st->r);
  const size_t o_t = L.add(sizeof(double) * n);
  const size_t o_e = L.add(sizeof(double) * n);
  Workspace w;
  w.s = D.s;
  w.base = static_cast<char*>(dev_alloc(L.size, D.s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  std::vector<Item> items(n);
  for (int i = 0; i < n; ++i)
    items[i] = Item{view_of(st), &D.blocks[cand[i]], st->r, D.m, w.at<float>(o_sig) + (size_t)i * st->r,
                    w.at<double>(o_t) + i, nullptr, w.at<double>(o_e) + i, nullptr};
  {
    Workspace ws;
    DecisionOnly only_decisions;  // first_accept reads nothing but tail <= eps^2 energy
    CSVD_TRY(run_items(items, D.eps, D.precision, D.s, D.d_status, ws, nullptr, false));
  }
  CUDA_TRY(cudaMemcpyAsync(tail.data(), w.base + o_t, sizeof(double) * n, cudaMemcpyDeviceToHost, D.s));
  CUDA_TRY(cudaMemcpyAsync(energy.data(), w.base + o_e, sizeof(double) * n, cudaMemcpyDeviceToHost, D.s));
  return take_status(D.d_status, D.s);
}

// Residual norms ||(I - U U^T) A_j||^2 against an incremental state's basis.
csvd_status residual_norms_state(Driver& D, csvd_state st, const std::vector<int>& cand,
                                 std::vector<double>& out) {
  const int n = (int)cand.size();
  out.assign(n, 0.0);
  if (n == 0) return CSVD_OK;
  Layout L;
  std::vector<size_t> oR(n), oP(n), oP2(n);
  for (int i = 0; i < n; ++i) {
    const int k = (int)D.blocks[cand[i]].k;
    oR[i] = L.add(sizeof(float) * (size_t)D.m * k);
    oP[i] = L.add(sizeof(float) * (size_t)std::max(st->rt, 1) * k);
    oP2[i] = L.add(sizeof(float) * (size_t)std::max(st->rt, 1) * k);
  }
  const size_t o_en = L.add(sizeof(double) * n);
  GemmBatch g1, g2, g3, g4;
  std::vector<EnergyDesc> ed;
  const float* U = st->U[st->cur];
  const int64_t ldu = st->r;
  auto fill = [&](char* base) {
    g1 = GemmBatch(); g2 = GemmBatch(); g3 = GemmBatch(); g4 = GemmBatch();
    ed.clear();
    for (int i = 0; i < n; ++i) {
      const csvd_block& b = D.blocks[cand[i]];
      const int k = (int)b.k;
      float* R = reinterpret_cast<float*>(base + oR[i]);
      float* P = reinterpret_cast<float*>(base + oP[i]);
      float* P2 = reinterpret_cast<float*>(base + oP2[i]);
      if (st->rt > 0) g1.add(gemm(U, ldu, 1, b.ptr, b.ld, 0, P, k, 0, st->rt, k, (int)D.m));
      g2.add(gemm(U, ldu, 0, P, k, 0, R, k, 0, (int)D.m, k, st->rt, -1.f,
                  reinterpret_cast<const float*>(b.ptr), b.ld, 0, 1.f));
      if (st->rt > 0) {
        g3.add(gemm(U, ldu, 1, R, k, 0, P2, k, 0, st->rt, k, (int)D.m));
        g4.add(gemm(U, ldu, 0, P2, k, 0, R, k, 0, (int)D.m, k, st->rt, -1.f, R, k, 0, 1.f));
      }
      ed.push_back(EnergyDesc{R, k, (int)D.m, k, 0, 0, reinterpret_cast<double*>(base + o_en) + i});
    }
  };
  fill(reinterpret_cast<char*>(uintptr_t(1) << 20));
  Pack probe;
  g1.pack(probe); g2.pack(probe); g3.pack(probe); g4.pack(probe);
  probe.add(ed);
  const size_t o_desc = L.add(probe.buf.size());
  Workspace w;
  w.s = D.s;
  w.base = static_cast<char*>(dev_alloc(L.size, D.s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  fill(w.base);
  Pack pk;
  g1.pack(pk); g2.pack(pk); g3.pack(pk); g4.pack(pk);
  const size_t o_ed = pk.add(ed);
  char* dbase = w.base + o_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), D.s));
  CUDA_TRY(cudaMemsetAsync(w.base + o_en, 0, sizeof(double) * n, D.s));
  CUDA_TRY(g1.launch(dbase, D.s));
  CUDA_TRY(g2.launch(dbase, D.s));
  CUDA_TRY(g3.launch(dbase, D.s));
  CUDA_TRY(g4.launch(dbase, D.s));
  CUDA_TRY(launch_energy(reinterpret_cast<EnergyDesc*>(dbase + o_ed), n, 16, D.s));
  CUDA_TRY(cudaMemcpyAsync(out.data(), w.base + o_en, sizeof(double) * n, cudaMemcpyDeviceToHost, D.s));
  CUDA_TRY(cudaStreamSynchronize(D.s));
  return CSVD_OK;
}

std::vector<int> sorted_by(const std::vector<int>& ids, const std::vector<double>& key) {
  std::vector<int> o(ids.size());
  std::iota(o.begin(), o.end(), 0);
  std::stable_sort(o.begin(), o.end(), [&](int a, int b) {
    if (key[a] != key[b]) return key[a] < key[b];
    return ids[a] < ids[b];
  });
  std::vector<int> out(ids.size());
  for (size_t i = 0; i < o.size(); ++i) out[i] = ids[o[i]];
  return out;
}

// Alg. 3: approximate incremental clustering.
// First candidate of `order` (from `pos` on) whose merge with the state is
// accepted, or order.size().  The scan is the sequential one of Alg. 3 (the
// first candidate in order that passes joins); candidates are scored in
// chunks of doubling size from `pos`, so an early accept does not pay for
// scoring the whole remainder.  A candidate's score does not depend on the
// batch it is scored in, so the decision equals that of scoring all at once.
static csvd_status first_accept(Driver& D, csvd_state st, const std::vector<int>& order,
                                size_t pos, size_t& hit) {
  constexpr size_t kFirstChunk = 256;
  const double e2 = D.eps * D.eps;
  hit = order.size();
  size_t chunk = kFirstChunk;
  while (pos < order.size()) {
    const size_t end = std::min(order.size(), pos + chunk);
    std::vector<int> cand(order.begin() + pos, order.begin() + end);
    std::vector<double> tail, energy;
    CSVD_TRY(score_state(D, st, cand, tail, energy));
    for (size_t i = 0; i < cand.size(); ++i)
      if (tail[i] <= e2 * energy[i]) {
        hit = pos + i;
        return CSVD_OK;
      }
    pos = end;
    chunk *= 2;
  }
  return CSVD_OK;
}

csvd_status cluster_approx(Driver& D, int sort_mode, std::vector<std::vector<int>>& clusters,
                           std::vector<double>& est) {
  std::vector<int> remaining(D.n);
  std::iota(remaining.begin(), remaining.end(), 0);
  std::stable_sort(remaining.begin(), remaining.end(), [&](int a, int b) {
    if (D.norms[a] != D.norms[b]) return D.norms[a] > D.norms[b];
    return a < b;
  });
  while (!remaining.empty()) {
    const int anchor = remaining.front();
    remaining.erase(remaining.begin());
    csvd_state st = nullptr;
    CSVD_TRY(csvd_incr_init(&st, D.m, D.r, D.precision, D.s));
    std::vector<int> members{anchor};
    csvd_status rc = append_commit(st, &D.blocks[anchor]);
    while (rc == CSVD_OK && !remaining.empty()) {
      if (sort_mode == CSVD_SORT_FROBENIUS) {
        // one scan in ascending norm; the first accept commits, the scan
        // goes on after it with the grown state
        std::vector<double> key(remaining.size());
        for (size_t i = 0; i < remaining.size(); ++i) key[i] = D.norms[remaining[i]];
        std::vector<int> order = sorted_by(remaining, key);
        bool any = false;
        size_t pos = 0;
        while (pos < order.size() && rc == CSVD_OK) {
          size_t hit = order.size();
          rc = first_accept(D, st, order, pos, hit);
          if (rc != CSVD_OK || hit == order.size()) break;
          rc = append_commit(st, &D.blocks[order[hit]]);
          members.push_back(order[hit]);
          remaining.erase(std::find(remaining.begin(), remaining.end(), order[hit]));
          any = true;
          pos = hit + 1;
        }
        if (!any) break;
      } else {
        std::vector<double> res;
        rc = residual_norms_state(D, st, remaining, res);
        if (rc != CSVD_OK) break;
        std::vector<int> order = sorted_by(remaining, res);
        size_t hit = order.size();
        rc = first_accept(D, st, order, 0, hit);
        if (rc != CSVD_OK || hit == order.size()) break;
        rc = append_commit(st, &D.blocks[order[hit]]);
        members.push_back(order[hit]);
        remaining.erase(std::find(remaining.begin(), remaining.end(), order[hit]));
      }
    }
    double tail = 0.0;
    if (rc == CSVD_OK) rc = csvd_tail_error(st, &tail, nullptr, nullptr, nullptr);
    csvd_incr_free(st);
    if (rc != CSVD_OK) return rc;
    clusters.push_back(members);
    est.push_back(tail);
  }
  return CSVD_OK;
}

// Alg. 2: residual clustering with a full-span basis.  The certificate of
// candidate j is Cor. 1 evaluated cancellation-free:
//   bound^2 = proj + ||Q^T A_j||^2 + sum_{beyond top r} (mu u sigma(R_j))^2.
// Candidate offers follow the scan semantics shared with the oracle:
// frobenius -- ascending norm, one pass accepting greedily (the span grows
// after each accept), passes repeat until one accepts nothing; residual --
// after every accept the residual norms are recomputed and the smallest
// candidate whose certificate holds joins.
csvd_status residual_bounds(Driver& D, SpanState& sp, const std::vector<int>& cand, Workspace& w,
                            std::vector<csvd_block>& R, std::vector<std::vector<float>>& sv,
                            std::vector<double>& bound, std::vector<double>& energy,
                            std::vector<double>& rnorm, std::vector<double>& pe) {
  CSVD_TRY(span_residuals(sp, D.blocks, cand, D.s, w, R, pe));
  std::vector<int> ridx(cand.size());
  std::iota(ridx.begin(), ridx.end(), 0);
  int rmax = 1;
  for (auto& b : R) rmax = std::max<int>(rmax, (int)std::min<int64_t>(b.k, D.m));
  std::vector<double> top;
  CSVD_TRY(block_spectra(R.data(), ridx, D.m, rmax, CSVD_PLAIN_FP32, D.s, D.d_status, rnorm, top, &sv));
  bound.assign(cand.size(), 0.0);
  energy.assign(cand.size(), 0.0);
  for (size_t i = 0; i < cand.size(); ++i) {
    std::vector<double> mu = sp.mu;
    for (float x : sv[i]) mu.push_back(x);
    energy[i] = sp.energy + D.norms[cand[i]];
    bound[i] = sp.proj + pe[i] + rest_sum_sq(mu, D.r);
  }
  return CSVD_OK;
}

csvd_status cluster_residual(Driver& D, int sort_mode, std::vector<std::vector<int>>& clusters,
                             std::vector<double>& est) {
  std::vector<int> remaining(D.n);
  std::iota(remaining.begin(), remaining.end(), 0);
  std::stable_sort(remaining.begin(), remaining.end(), [&](int a, int b) {
    if (D.norms[a] != D.norms[b]) return D.norms[a] > D.norms[b];
    return a < b;
  });
  const double e2 = D.eps * D.eps;
  while (!remaining.empty()) {
    const int anchor = remaining.front();
    remaining.erase(remaining.begin());
    SpanState sp;
    if (!sp.alloc(D.m, D.s)) return fail(CSVD_ERR_OOM, "span basis allocation failed");
    std::vector<int> members{anchor};
    {
      std::vector<double> e1, t1;
      std::vector<std::vector<float>> sv;
      const int rk = (int)std::min<int64_t>(D.blocks[anchor].k, D.m);
      CSVD_TRY(block_spectra(D.blocks, {anchor}, D.m, rk, CSVD_PLAIN_FP32, D.s, D.d_status, e1, t1, &sv));
      for (float x : sv[0]) sp.mu.push_back(x);
      sp.energy = D.norms[anchor];
      CSVD_TRY(span_extend(sp, D.blocks[anchor], sv[0], 1e-6 * std::sqrt(sp.energy), D.s));
    }
    auto accept = [&](int j, const csvd_block& R, const std::vector<float>& sv, double energy,
                      double pe) -> csvd_status {
      for (float x : sv) sp.mu.push_back(x);
      sp.proj += pe;
      sp.energy = energy;
      CSVD_TRY(span_extend(sp, R, sv, 1e-6 * std::sqrt(sp.energy), D.s));
      members.push_back(j);
      remaining.erase(std::find(remaining.begin(), remaining.end(), j));
      return CSVD_OK;
    };
    if (sort_mode == CSVD_SORT_FROBENIUS) {
      while (!remaining.empty()) {
        std::vector<double> key(remaining.size());
        for (size_t i = 0; i < remaining.size(); ++i) key[i] = D.norms[remaining[i]];
        const std::vector<int> order = sorted_by(remaining, key);
        bool any = false;
        size_t pos = 0;
        while (pos < order.size()) {
          std::vector<int> cand(order.begin() + pos, order.end());
          Workspace w;
          std::vector<csvd_block> R;
          std::vector<std::vector<float>> sv;
          std::vector<double> bound, energy, rn, pe;
          CSVD_TRY(residual_bounds(D, sp, cand, w, R, sv, bound, energy, rn, pe));
          size_t hit = cand.size();
          for (size_t i = 0; i < cand.size(); ++i)
            if (bound[i] <= e2 * energy[i]) { hit = i; break; }
          if (hit == cand.size()) break;
          CSVD_TRY(accept(cand[hit], R[hit], sv[hit], energy[hit], pe[hit]));
          any = true;
          pos += hit + 1;
        }
        if (!any) break;
      }
    } else {
      while (!remaining.empty()) {
        Workspace w;
        std::vector<csvd_block> R;
        std::vector<std::vector<float>> sv;
        std::vector<double> bound, energy, rn, pe;
        CSVD_TRY(residual_bounds(D, sp, remaining, w, R, sv, bound, energy, rn, pe));
        std::vector<int> pos(remaining.size());
        std::iota(pos.begin(), pos.end(), 0);
        std::stable_sort(pos.begin(), pos.end(), [&](int a, int b) {
          if (rn[a] != rn[b]) return rn[a] < rn[b];
          return remaining[a] < remaining[b];
        });
        int hit = -1;
        for (int p : pos)
          if (bound[p] <= e2 * energy[p]) { hit = p; break; }
        if (hit < 0) break;
        CSVD_TRY(accept(remaining[hit], R[hit], sv[hit], energy[hit], pe[hit]));
      }
    }
    clusters.push_back(members);
    est.push_back(sp.proj + rest_sum_sq(sp.mu, D.r));
  }
  return CSVD_OK;
}

// Alg. 1: max-norm (Weyl) clustering with a head of width <= r.  Bounds are
// sums of non-negative terms: with a head, S - S_head = the energy of the
// non-head members; without, S - top_r(A_j*) = sum_{i != j*} ||A_i||^2 +
// (tail of A_j*), j* the member with the largest top-r energy.
csvd_status cluster_weyl(Driver& D, std::vector<std::vector<int>>& clusters,
                         std::vector<double>& est) {
  std::vector<int> all(D.n);
  std::iota(all.begin(), all.end(), 0);
  std::vector<double> en, top;
  CSVD_TRY(block_spectra(D.blocks, all, D.m, D.r, D.precision, D.s, D.d_status, en, top, nullptr));
  std::vector<double> tail(D.n);
  for (int i = 0; i < D.n; ++i) tail[i] = std::max(0.0, en[i] - top[i]);
  std::vector<int> desc = all;
  std::stable_sort(desc.begin(), desc.end(), [&](int a, int b) {
    if (D.norms[a] != D.norms[b]) return D.norms[a] > D.norms[b];
    return a < b;
  });
  std::vector<int> remaining = desc;
  const double e2 = D.eps * D.eps;
  while (!remaining.empty()) {
    const int anchor = remaining.front();
    remaining.erase(remaining.begin());
    std::vector<int> members{anchor};
    bool head = false;
    double S = D.norms[anchor];
    double nonhead = 0.0;      // head case: energy outside the head
    int jstar = anchor;        // no-head case: member with the largest top-r energy
    double others = 0.0;       // no-head case: energy of the members other than jstar
    if (D.widths[anchor] <= D.r) {
      head = true;
      int width = D.widths[anchor];
      while (!remaining.empty() && width + D.widths[remaining.front()] <= D.r) {
        const int j = remaining.front();
        remaining.erase(remaining.begin());
        members.push_back(j);
        width += D.widths[j];
        S += D.norms[j];
      }
    }
    auto bound_with = [&](int j, int& js, double& oth) {
      if (head) return nonhead + D.norms[j];
      if (top[j] > top[jstar]) { js = j; oth = others + D.norms[jstar]; }
      else { js = jstar; oth = others + D.norms[j]; }
      return oth + tail[js];
    };
    while (true) {
      std::vector<double> key(remaining.size());
      for (size_t i = 0; i < remaining.size(); ++i) key[i] = D.norms[remaining[i]];
      std::vector<int> order = sorted_by(remaining, key);
      bool any = false;
      for (int j : order) {
        int js = jstar;
        double oth = others;
        const double b = bound_with(j, js, oth);
        const double S2 = S + D.norms[j];
        if (b <= e2 * S2) {
          S = S2;
          if (head) nonhead += D.norms[j];
          else { jstar = js; others = oth; }
          members.push_back(j);
          remaining.erase(std::find(remaining.begin(), remaining.end(), j));
          any = true;
        }
      }
      if (!any || remaining.empty()) break;
    }
    clusters.push_back(members);
    est.push_back(head ? nonhead : others + tail[jstar]);
  }
  return CSVD_OK;
}

}  // namespace

extern "C" csvd_status csvd_cluster(const csvd_block* blocks, int32_t n, int64_t m, int32_t r,
                                    double eps, int32_t algo, int32_t sort_mode, int32_t precision,
                                    void* cuda_stream, int32_t* labels_out,
                                    double* cluster_est_sq_out, double* energy_out,
                                    double* compression_ratio_out) {
  if (!blocks || n < 1 || m < 1 || r < 1 || r > m || !labels_out || !(eps >= 0.0))
    return fail(CSVD_ERR_ARG, "bad arguments");
  if (algo != CSVD_ALG_WEYL && algo != CSVD_ALG_RESIDUAL && algo != CSVD_ALG_APPROX)
    return fail(CSVD_ERR_ARG, "bad algo");
  if (sort_mode != CSVD_SORT_FROBENIUS && sort_mode != CSVD_SORT_RESIDUAL)
    return fail(CSVD_ERR_ARG, "bad sort mode");
  if (precision != CSVD_PLAIN_FP32 && precision != CSVD_MIXED && precision != CSVD_GRAM_FP32)
    return fail(CSVD_ERR_ARG, "bad precision");
  for (int i = 0; i < n; ++i) {
    CSVD_TRY(check_block(&blocks[i], m));
    if (blocks[i].dtype != CSVD_F32) return fail(CSVD_ERR_UNIMPLEMENTED, "clustering takes f32 blocks");
  }
  Driver D;
  D.blocks = blocks;
  D.n = n;
  D.m = m;
  D.r = r;
  D.eps = eps;
  D.precision = precision;
  D.s = static_cast<cudaStream_t>(cuda_stream);
  Workspace ws_status;
  ws_status.s = D.s;
  ws_status.base = static_cast<char*>(dev_alloc(sizeof(int), D.s));
  if (!ws_status.base) return fail(CSVD_ERR_OOM, "status allocation failed");
  D.d_status = ws_status.at<int>(0);
  CUDA_TRY(cudaMemsetAsync(D.d_status, 0, sizeof(int), D.s));
  std::vector<int> all(n);
  std::iota(all.begin(), all.end(), 0);
  D.widths.resize(n);
  for (int i = 0; i < n; ++i) D.widths[i] = (int)blocks[i].k;
  // block energies
  csvd_status rc;
  rc = block_energies(blocks, all, m, D.s, D.norms);
  std::vector<std::vector<int>> clusters;
  std::vector<double> est;
  if (rc == CSVD_OK) {
    if (algo == CSVD_ALG_APPROX) rc = cluster_approx(D, sort_mode, clusters, est);
    else if (algo == CSVD_ALG_RESIDUAL) rc = cluster_residual(D, sort_mode, clusters, est);
    else rc = cluster_weyl(D, clusters, est);
  }
  cudaStreamSynchronize(D.s);
  if (rc != CSVD_OK) return rc;
  int64_t raw = 0, stored = 0;
  for (size_t c = 0; c < clusters.size(); ++c) {
    int64_t nc = 0;
    double en = 0.0;
    for (int j : clusters[c]) {
      labels_out[j] = (int32_t)c;
      nc += D.widths[j];
      en += D.norms[j];
    }
    if (cluster_est_sq_out) cluster_est_sq_out[c] = est[c];
    if (energy_out) energy_out[c] = en;
    const int64_t reff = std::min<int64_t>({(int64_t)r, nc, m});
    raw += m * nc;
    stored += std::min<int64_t>(m * nc, reff * (m + nc));
  }
  for (size_t c = clusters.size(); c < (size_t)n; ++c) {
    if (cluster_est_sq_out) cluster_est_sq_out[c] = 0.0;
    if (energy_out) energy_out[c] = 0.0;
  }
  if (compression_ratio_out) *compression_ratio_out = (double)raw / (double)stored;
  return CSVD_OK;
}

extern "C" csvd_status csvd_tail_grad(const float* U, int64_t ldu, int64_t m, int32_t r,
                                      const csvd_block* blocks, const csvd_block* grads,
                                      int32_t n, double g, void* cuda_stream) {
  if (!U || !blocks || !grads || n < 0 || m < 1 || r < 0 || ldu < r)
    return fail(CSVD_ERR_ARG, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < n; ++i) {
    CSVD_TRY(check_block(&blocks[i], m));
    CSVD_TRY(check_block(&grads[i], m));
    if (blocks[i].dtype != CSVD_F32 || grads[i].dtype != CSVD_F32 || grads[i].k != blocks[i].k)
      return fail(CSVD_ERR_ARG, "gradients take f32 blocks of the same width");
  }
  if (n == 0) return CSVD_OK;
  Layout L;
  std::vector<size_t> oP(n);
  for (int i = 0; i < n; ++i) oP[i] = L.add(sizeof(float) * (size_t)std::max(r, 1) * blocks[i].k);
  GemmBatch g1, g2;
  auto fill = [&](char* base) {
    g1 = GemmBatch(); g2 = GemmBatch();
    for (int i = 0; i < n; ++i) {
      const int k = (int)blocks[i].k;
      float* P = reinterpret_cast<float*>(base + oP[i]);
      if (r > 0) g1.add(gemm(U, ldu, 1, blocks[i].ptr, blocks[i].ld, 0, P, k, 0, r, k, (int)m));
      g2.add(gemm(U, ldu, 0, P, k, 0, const_cast<float*>(reinterpret_cast<const float*>(grads[i].ptr)),
                  grads[i].ld, 0, (int)m, k, r, (float)(-2.0 * g),
                  reinterpret_cast<const float*>(blocks[i].ptr), blocks[i].ld, 0, (float)(2.0 * g)));
    }
  };
  fill(reinterpret_cast<char*>(uintptr_t(1) << 20));
  Pack probe;
  g1.pack(probe); g2.pack(probe);
  const size_t o_desc = L.add(probe.buf.size());
  Workspace w;
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  fill(w.base);
  Pack pk;
  g1.pack(pk); g2.pack(pk);
  char* dbase = w.base + o_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), s));
  CUDA_TRY(g1.launch(dbase, s));
  CUDA_TRY(g2.launch(dbase, s));
  return CSVD_OK;
}

// Final decomposition of a cluster (Section 2): V_i = A_i^T U diag(s)^-1 and
// the explicit residuals A_i - U U^T A_i with their energies.
extern "C" csvd_status csvd_reconstruct(const float* U, int64_t ldu, const float* s, int64_t m,
                                        int32_t r, const csvd_block* blocks, int32_t n,
                                        float* Ut_out, int64_t ldut, float* const* V_out,
                                        int64_t ldv, void* cuda_stream, double* resid_sq,
                                        double* energy) {
  if (!U || !s || !blocks || n < 0 || m < 1 || r < 1 || ldu < r || !resid_sq || !energy)
    return fail(CSVD_ERR_ARG, "bad arguments");
  if (V_out && ldv < r) return fail(CSVD_ERR_ARG, "ldv < r");
  if (Ut_out && ldut < r) return fail(CSVD_ERR_ARG, "ldut < r");
  for (int i = 0; i < n; ++i) {
    CSVD_TRY(check_block(&blocks[i], m));
    if (blocks[i].dtype != CSVD_F32) return fail(CSVD_ERR_ARG, "decomposition takes f32 blocks");
    if (V_out && !V_out[i]) return fail(CSVD_ERR_ARG, "NULL V_out entry");
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (Ut_out) CUDA_TRY(launch_scale_cols(U, ldu, (int)m, r, s, 0, Ut_out, ldut, st));
  if (n == 0) return CSVD_OK;
  // workspace: U diag(s)^-1, and per block P = U^T A (r x k) and R = A - U P (m x k)
  Layout L;
  const size_t oUs = L.add(sizeof(float) * (size_t)m * r);
  std::vector<size_t> oP(n), oR(n);
  for (int i = 0; i < n; ++i) {
    oP[i] = L.add(sizeof(float) * (size_t)r * blocks[i].k);
    oR[i] = L.add(sizeof(float) * (size_t)m * blocks[i].k);
  }
  GemmBatch gP, gR, gV;
  auto fill = [&](char* base) {
    gP = GemmBatch(); gR = GemmBatch(); gV = GemmBatch();
    const float* Us = reinterpret_cast<const float*>(base + oUs);
    for (int i = 0; i < n; ++i) {
      const int k = (int)blocks[i].k;
      float* P = reinterpret_cast<float*>(base + oP[i]);
      float* R = reinterpret_cast<float*>(base + oR[i]);
      gP.add(gemm(U, ldu, 1, blocks[i].ptr, blocks[i].ld, 0, P, k, 0, r, k, (int)m));
      gR.add(gemm(U, ldu, 0, P, k, 0, R, k, 0, (int)m, k, r, -1.f,
                  reinterpret_cast<const float*>(blocks[i].ptr), blocks[i].ld, 0, 1.f));
      // V_i = (Us^T A_i)^T, written transposed (k x r)
      if (V_out) gV.add(gemm(Us, r, 1, blocks[i].ptr, blocks[i].ld, 0, V_out[i], ldv, 1, r, k, (int)m));
    }
  };
  fill(reinterpret_cast<char*>(uintptr_t(1) << 20));
  Pack probe;
  gP.pack(probe); gR.pack(probe); gV.pack(probe);
  const size_t o_desc = L.add(probe.buf.size());
  Workspace w;
  w.s = st;
  w.base = static_cast<char*>(dev_alloc(L.size, st));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  fill(w.base);
  Pack pk;
  gP.pack(pk); gR.pack(pk); gV.pack(pk);
  char* dbase = w.base + o_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), st));
  if (V_out) CUDA_TRY(launch_scale_cols(U, ldu, (int)m, r, s, 1, w.at<float>(oUs), r, st));
  CUDA_TRY(gP.launch(dbase, st));
  CUDA_TRY(gR.launch(dbase, st));
  if (V_out) CUDA_TRY(gV.launch(dbase, st));
  // energies of the residuals and of the blocks
  std::vector<csvd_block> rb(n);
  for (int i = 0; i < n; ++i) rb[i] = csvd_block{w.base + oR[i], blocks[i].k, blocks[i].k, CSVD_F32, 0};
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::vector<double> er, ea;
  CSVD_TRY(block_energies(rb.data(), idx, m, st, er));
  CSVD_TRY(block_energies(blocks, idx, m, st, ea));
  for (int i = 0; i < n; ++i) {
    resid_sq[i] = er[i];
    energy[i] = ea[i];
  }
  return CSVD_OK;
}

// Eckart-Young tail energy of a basis: per block ||(I - U U^T) A_j||_F^2,
// P = U^T A_j by the batched GEMM, then the residual's squares summed tile
// by tile without storing it.
extern "C" csvd_status csvd_tail_energy(const float* U, int64_t ldu, int64_t m, int32_t r,
                                        const csvd_block* blocks, int32_t n, void* cuda_stream,
                                        double* resid_sq) {
  if (!U || !blocks || !resid_sq || n < 0 || m < 1 || r < 1 || ldu < r)
    return fail(CSVD_ERR_ARG, "bad arguments");
  for (int i = 0; i < n; ++i) {
    CSVD_TRY(check_block(&blocks[i], m));
    if (blocks[i].dtype != CSVD_F32) return fail(CSVD_ERR_UNIMPLEMENTED, "f32 blocks only");
  }
  if (n == 0) return CSVD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Layout L;
  const size_t o_out = L.add(sizeof(double) * (size_t)n);
  std::vector<size_t> oP(n);
  for (int i = 0; i < n; ++i) oP[i] = L.add(sizeof(float) * (size_t)r * blocks[i].k);
  GemmBatch gP;
  std::vector<ResidDesc> rd;
  int max_k = 1;
  auto fill = [&](char* base) {
    gP = GemmBatch();
    rd.clear();
    for (int i = 0; i < n; ++i) {
      const int k = (int)blocks[i].k;
      max_k = std::max(max_k, k);
      float* P = reinterpret_cast<float*>(base + oP[i]);
      gP.add(gemm(U, ldu, 1, blocks[i].ptr, blocks[i].ld, 0, P, k, 0, r, k, (int)m));
      rd.push_back(ResidDesc{reinterpret_cast<const float*>(blocks[i].ptr), blocks[i].ld, U, ldu, P,
                             k, (int)m, k, reinterpret_cast<double*>(base + o_out) + i});
    }
  };
  fill(reinterpret_cast<char*>(uintptr_t(1) << 20));
  Pack probe;
  gP.pack(probe);
  probe.add(rd);
  const size_t o_desc = L.add(probe.buf.size());
  Workspace w;
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  fill(w.base);
  Pack pk;
  gP.pack(pk);
  const size_t o_rd = pk.add(rd);
  char* dbase = w.base + o_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), s));
  CUDA_TRY(cudaMemsetAsync(w.base + o_out, 0, sizeof(double) * (size_t)n, s));
  CUDA_TRY(gP.launch(dbase, s));
  CUDA_TRY(launch_resid_energy(reinterpret_cast<ResidDesc*>(dbase + o_rd), n, (int)m, max_k, r, s));
  CUDA_TRY(cudaMemcpyAsync(resid_sq, w.base + o_out, sizeof(double) * (size_t)n,
                           cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return CSVD_OK;
}

// Top-r left basis of a block collection: the incremental estimator at a
// working rank, then `refine` sweeps of subspace iteration (Y = M M^T U,
// orthonormalised as the left singular vectors of Y by a rank-r append).
extern "C" csvd_status csvd_top_basis(const csvd_block* blocks, int32_t n, int64_t m, int32_t r,
                                      int32_t working_rank, int32_t refine, void* cuda_stream,
                                      float* U_out, int64_t ldu, int32_t* r_eff) {
  if (!blocks || n < 1 || m < 1 || r < 1 || !U_out || ldu < r || refine < 0)
    return fail(CSVD_ERR_ARG, "bad arguments");
  if (working_rank < r) working_rank = r;
  working_rank = (int32_t)std::min<int64_t>(working_rank, m);
  if (r > working_rank) return fail(CSVD_ERR_ARG, "r > min(m, working rank)");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  csvd_state st = nullptr;
  CSVD_TRY(csvd_incr_init(&st, m, working_rank, CSVD_PLAIN_FP32, cuda_stream));
  csvd_status rc = CSVD_OK;
  for (int i = 0; i < n && rc == CSVD_OK; ++i) rc = csvd_incr_append(st, &blocks[i]);
  int32_t rk = 0;
  if (rc == CSVD_OK) rc = csvd_incr_sigma(st, nullptr, &rk);
  const int rr = std::min<int>(r, rk);
  if (r_eff) *r_eff = rr;
  if (rc == CSVD_OK && rr > 0)
    rc = cudaMemcpy2DAsync(U_out, sizeof(float) * ldu, st->U[st->cur], sizeof(float) * st->r,
                           sizeof(float) * rr, m, cudaMemcpyDeviceToDevice, s) == cudaSuccess
             ? CSVD_OK
             : fail(CSVD_ERR_CUDA, "basis copy failed");
  csvd_incr_free(st);
  if (rc != CSVD_OK || rr == 0) return rc;
  // subspace iteration: Y = M M^T U, U <- left singular vectors of Y
  float* Y = static_cast<float*>(dev_alloc(sizeof(float) * (size_t)m * rr, s));
  if (!Y) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  for (int it = 0; it < refine && rc == CSVD_OK; ++it) {
    rc = csvd_gram_apply(U_out, ldu, m, rr, blocks, n, Y, rr, cuda_stream);
    csvd_state q = nullptr;
    if (rc == CSVD_OK) rc = csvd_incr_init(&q, m, rr, CSVD_PLAIN_FP32, cuda_stream);
    if (rc == CSVD_OK) {
      const csvd_block yb{Y, rr, rr, CSVD_F32, 0};
      rc = csvd_incr_append(q, &yb);
      int32_t qk = 0;
      if (rc == CSVD_OK) rc = csvd_incr_sigma(q, nullptr, &qk);
      if (rc == CSVD_OK && qk == rr)
        rc = cudaMemcpy2DAsync(U_out, sizeof(float) * ldu, q->U[q->cur], sizeof(float) * q->r,
                               sizeof(float) * rr, m, cudaMemcpyDeviceToDevice, s) == cudaSuccess
                 ? CSVD_OK
                 : fail(CSVD_ERR_CUDA, "basis copy failed");
    }
    if (q) csvd_incr_free(q);
  }
  dev_free(Y, s);
  return rc;
}

// Randomized range-finder tail estimate: Y = sum_i A_i Omega_i, q power
// iterations Y <- M M^T Q (Q the left singular basis of Y), U_r the top-r
// left singular vectors of Y, and the explicit residual energy of U_r.
extern "C" csvd_status csvd_randomized_tail(const csvd_block* blocks, const float* const* omegas,
                                            int32_t n, int64_t m, int32_t r, int32_t l,
                                            int32_t power_iters, void* cuda_stream,
                                            double* tail_sq, float* U_out, int64_t ldu) {
  if (!blocks || !omegas || !tail_sq || n < 1 || m < 1 || r < 1 || l < r || l > m ||
      power_iters < 0 || (U_out && ldu < r))
    return fail(CSVD_ERR_ARG, "bad arguments");
  for (int i = 0; i < n; ++i) {
    CSVD_TRY(check_block(&blocks[i], m));
    if (blocks[i].dtype != CSVD_F32) return fail(CSVD_ERR_UNIMPLEMENTED, "f32 blocks only");
    if (!omegas[i]) return fail(CSVD_ERR_ARG, "NULL test matrix");
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // 1. Y = sum_i A_i Omega_i (one GEMM per block, accumulating)
  Layout L;
  const size_t oY = L.add(sizeof(float) * (size_t)m * l);
  const size_t oQ = L.add(sizeof(float) * (size_t)m * l);
  const size_t oU = L.add(sizeof(float) * (size_t)m * r);
  std::vector<GemmBatch> gY(n);
  auto fill = [&](char* base) {
    float* Y = reinterpret_cast<float*>(base + oY);
    for (int i = 0; i < n; ++i) {
      gY[i] = GemmBatch();
      gY[i].add(gemm(blocks[i].ptr, blocks[i].ld, 0, omegas[i], l, 0, Y, l, 0, (int)m, l,
                     (int)blocks[i].k, 1.f, i == 0 ? nullptr : Y, l, 0, i == 0 ? 0.f : 1.f));
    }
  };
  fill(reinterpret_cast<char*>(uintptr_t(1) << 20));
  Pack probe;
  for (auto& g : gY) g.pack(probe);
  const size_t o_desc = L.add(probe.buf.size());
  Workspace w;
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  fill(w.base);
  Pack pk;
  for (auto& g : gY) g.pack(pk);
  char* dbase = w.base + o_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), s));
  for (auto& g : gY) CUDA_TRY(g.launch(dbase, s));
  float* Y = w.at<float>(oY);
  float* Q = w.at<float>(oQ);
  float* U = w.at<float>(oU);
  const csvd_block yb{Y, l, l, CSVD_F32, 0};
  int32_t rk = 0;
  // 2. power iterations: Q = left singular basis of Y, Y = M M^T Q
  for (int it = 0; it < power_iters; ++it) {
    CSVD_TRY(csvd_top_basis(&yb, 1, m, l, l, 0, cuda_stream, Q, l, &rk));
    if (rk < l) CUDA_TRY(cudaMemset2DAsync(Q + rk, sizeof(float) * l, 0, sizeof(float) * (l - rk),
                                           m, s));
    CSVD_TRY(csvd_gram_apply(Q, l, m, l, blocks, n, Y, l, cuda_stream));
  }
  // 3. U_r: the top r left singular vectors of Y
  CSVD_TRY(csvd_top_basis(&yb, 1, m, r, l, 0, cuda_stream, U, r, &rk));
  if (rk < r) CUDA_TRY(cudaMemset2DAsync(U + rk, sizeof(float) * r, 0, sizeof(float) * (r - rk), m, s));
  // 4. the explicit residual energy of U_r
  std::vector<double> res(n);
  CSVD_TRY(csvd_tail_energy(U, r, m, r, blocks, n, cuda_stream, res.data()));
  double t = 0.0;
  for (double x : res) t += x;
  *tail_sq = t;
  if (U_out)
    CUDA_TRY(cudaMemcpy2DAsync(U_out, sizeof(float) * ldu, U, sizeof(float) * r, sizeof(float) * r,
                               m, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return CSVD_OK;
}

extern "C" csvd_status csvd_block_energy(const csvd_block* blocks, int32_t n, int64_t m,
                                         void* cuda_stream, double* energy_host) {
  if (!blocks || n < 0 || m < 1 || !energy_host) return fail(CSVD_ERR_ARG, "bad arguments");
  for (int i = 0; i < n; ++i) CSVD_TRY(check_block(&blocks[i], m));
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::vector<double> out;
  CSVD_TRY(block_energies(blocks, idx, m, static_cast<cudaStream_t>(cuda_stream), out));
  for (int i = 0; i < n; ++i) energy_host[i] = out[i];
  return CSVD_OK;
}

extern "C" int64_t csvd_launch_count(void) { return (int64_t)g_launch_count.load(); }

extern "C" csvd_status csvd_profile(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& e : g_prof) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  g_prof.clear();
  g_prof_on.store(enable != 0);
  return CSVD_OK;
}

extern "C" csvd_status csvd_profile_report(char* buf, int64_t len) {
  if (!buf || len < 1) return fail(CSVD_ERR_ARG, "bad buffer");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  struct Acc { std::string name; long long n = 0; double ms = 0.0; };
  std::vector<Acc> acc;
  for (auto& e : g_prof) {
    cudaError_t err = cudaEventSynchronize(e.b);
    if (err != cudaSuccess) return fail(CSVD_ERR_CUDA, cudaGetErrorString(err));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e.a, e.b);
    auto it = std::find_if(acc.begin(), acc.end(), [&](const Acc& a) { return a.name == e.name; });
    if (it == acc.end()) { acc.push_back(Acc{e.name, 0, 0.0}); it = acc.end() - 1; }
    it->n += 1;
    it->ms += ms;
  }
  std::string out;
  for (auto& a : acc) out += a.name + " " + std::to_string(a.n) + " " + std::to_string(a.ms) + "\n";
  std::snprintf(buf, (size_t)len, "%s", out.c_str());
  return CSVD_OK;
}

extern "C" csvd_status csvd_gram_apply(const float* U, int64_t ldu, int64_t m, int32_t r,
                                       const csvd_block* blocks, int32_t n, float* Y, int64_t ldy,
                                       void* cuda_stream) {
  if (!U || !blocks || !Y || n < 1 || m < 1 || r < 1 || ldu < r || ldy < r)
    return fail(CSVD_ERR_ARG, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < n; ++i) {
    CSVD_TRY(check_block(&blocks[i], m));
    if (blocks[i].dtype != CSVD_F32) return fail(CSVD_ERR_UNIMPLEMENTED, "f32 blocks only");
  }
  Layout L;
  std::vector<size_t> oT(n);
  for (int i = 0; i < n; ++i) oT[i] = L.add(sizeof(float) * (size_t)blocks[i].k * r);
  std::vector<GemmBatch> gY(n);
  GemmBatch gT;
  auto fill = [&](char* base) {
    gT = GemmBatch();
    for (int i = 0; i < n; ++i) {
      gY[i] = GemmBatch();
      const int k = (int)blocks[i].k;
      float* T = reinterpret_cast<float*>(base + oT[i]);
      // T_j = A_j^T U (k x r)
      gT.add(gemm(blocks[i].ptr, blocks[i].ld, 1, U, ldu, 0, T, r, 0, k, r, (int)m));
      // Y (+)= A_j T_j
      gY[i].add(gemm(blocks[i].ptr, blocks[i].ld, 0, T, r, 0, Y, ldy, 0, (int)m, r, k, 1.f,
                     i == 0 ? nullptr : Y, ldy, 0, i == 0 ? 0.f : 1.f));
    }
  };
  fill(reinterpret_cast<char*>(uintptr_t(1) << 20));
  Pack probe;
  gT.pack(probe);
  for (auto& g : gY) g.pack(probe);
  const size_t o_desc = L.add(probe.buf.size());
  Workspace w;
  w.s = s;
  w.base = static_cast<char*>(dev_alloc(L.size, s));
  if (!w.base) return fail(CSVD_ERR_OOM, "workspace allocation failed");
  fill(w.base);
  Pack pk;
  gT.pack(pk);
  for (auto& g : gY) g.pack(pk);
  char* dbase = w.base + o_desc;
  CUDA_TRY(upload(dbase, pk.buf.data(), pk.buf.size(), s));
  CUDA_TRY(gT.launch(dbase, s));
  for (auto& g : gY) CUDA_TRY(g.launch(dbase, s));
  return CSVD_OK;
}
