// C ABI (include/fc.h): forest lifetime, device store, and the time-stepping
// scheduler (Alg. 1 fills, global and multirate level substeps, regrid).
#include <algorithm>
#include <atomic>
#include <functional>
#include <mutex>
#include <unordered_map>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fc_internal.hpp"

using namespace fc;

namespace {

thread_local std::string g_err;

fc_status fail(fc_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

fc_status cuda_fail(cudaError_t e, const char* where) {
  return fail(FC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define FC_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Device memory of a forest comes from the stream-ordered allocator: a
// regrid allocates the new layout's store and frees the old one without
// synchronising the device, and the pool keeps freed blocks for the next
// regrid.  Allocations and frees are ordered on the calling thread's current
// allocation stream (the API call's stream while a regrid runs).
thread_local cudaStream_t g_alloc_stream = 0;

struct AllocStream {
  explicit AllocStream(cudaStream_t s) : prev_(g_alloc_stream) { g_alloc_stream = s; }
  ~AllocStream() { g_alloc_stream = prev_; }

 private:
  cudaStream_t prev_;
};

// keep freed blocks in the device's default pool (per process)
void keep_pool_memory() {
  static thread_local int done_for = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev == done_for) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done_for = dev;
}

// Pluggable device allocator (fc_set_allocator): when set, every device
// allocation of the library goes through the caller's functions instead of
// the stream-ordered pool, with the same stream the pool would have used.
// The sizes of hooked blocks are kept so the free callback receives them.
struct AllocHook {
  fc_alloc_fn alloc = nullptr;
  fc_free_fn release = nullptr;
  void* user = nullptr;
};
AllocHook g_hook;
std::mutex g_hook_mu;
std::unordered_map<void*, size_t> g_hook_sizes;
std::atomic<int> g_live_forests{0};

cudaError_t dmalloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  if (g_hook.alloc) {
    void* q = g_hook.alloc(bytes, static_cast<void*>(g_alloc_stream), g_hook.user);
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) & 255) {  // the kernels' bulk copies and vector reads
      g_hook.release(q, bytes, static_cast<void*>(g_alloc_stream), g_hook.user);
      return cudaErrorMemoryAllocation;
    }
    std::lock_guard<std::mutex> lock(g_hook_mu);
    g_hook_sizes[q] = bytes;
    *p = q;
    return cudaSuccess;
  }
  return cudaMallocAsync(p, bytes, g_alloc_stream);
}

template <typename T>
cudaError_t dmalloc(T** p, size_t n) {
  void* v = nullptr;
  const cudaError_t e = dmalloc_bytes(&v, (n ? n : 1) * sizeof(T));
  *p = static_cast<T*>(v);
  return e;
}

void dfree_bytes(void* p) {
  if (!p) return;
  if (g_hook.release) {
    size_t bytes = 0;
    {
      std::lock_guard<std::mutex> lock(g_hook_mu);
      auto it = g_hook_sizes.find(p);
      if (it != g_hook_sizes.end()) {
        bytes = it->second;
        g_hook_sizes.erase(it);
      }
    }
    g_hook.release(p, bytes, static_cast<void*>(g_alloc_stream), g_hook.user);
    return;
  }
  cudaFreeAsync(p, g_alloc_stream);
}

template <typename T>
void dfree(T*& p) {
  dfree_bytes((void*)p);
  p = nullptr;
}

}  // namespace

struct fc_forest {
  HostForest host;
  // the tables of the layout before the current one, whose memory the next
  // regrid's build writes its rows into
  std::vector<NbrEntry, UninitAlloc<NbrEntry>> spare_nbr;
  std::vector<PatchMeta, UninitAlloc<PatchMeta>> spare_meta;
  size_t esize = 8;
  // one allocation (store) holds the two state buffers, the
  // time-interpolation tiles qT, the refluxing fluxes and the device staging
  // for host copies, in that order
  void* store = nullptr;
  void* buf[2] = {nullptr, nullptr};
  void* qT = nullptr;
  void* stage = nullptr;  // device staging for host copies
  // refluxing (desc.reflux): per patch, two substep slots of the final fluxes
  // through its four faces (field precision), and the slot each level's
  // latest update wrote
  void* bflux = nullptr;
  int bslot[kMaxLevel + 1] = {};
  // the layout's small tables and per-patch scratch share one allocation
  // (d_tables, filled by one copy): d_meta, d_lists, d_api_to_dev, d_fstart,
  // d_patch_sums, d_mass and d_delta point into it
  void* d_tables = nullptr;
  PatchMeta* d_meta = nullptr;
  NbrEntry* d_nbr = nullptr;
  int* d_lists = nullptr;  // all work lists, concatenated
  size_t off_all = 0, off_coarse_all = 0, off_a[kMaxLevel + 1] = {0}, off_b[kMaxLevel + 1] = {0},
         off_t[kMaxLevel + 1] = {0};
  bool fuse = true;  // multirate substeps: update kernel gathers its own ghosts
  int* d_api_to_dev = nullptr;
  int* d_fstart = nullptr;
  double* d_patch_sums = nullptr;
  double* d_mass = nullptr;
  double* d_delta = nullptr;
  RemapEntry* d_remap = nullptr;
  int* d_err = nullptr;  // device error word (bit kErrTimeout)
  int cur[kMaxLevel + 1] = {0};
  bool has_old[kMaxLevel + 1] = {false};
  double t_start[kMaxLevel + 1] = {0};
  double dt_last[kMaxLevel + 1] = {0};
  // per-phase CUDA-event timers: every timed launch is bracketed by a pair
  struct TimerPair {
    cudaEvent_t a = nullptr, b = nullptr;
    double bytes = 0.0;
    int phase = 0;
  };
  struct PhaseTotal {
    double ms = 0.0, bytes = 0.0;
    int64_t launches = 0;
  };
  bool timing = false;
  std::vector<TimerPair> pending;  // recorded by direct launches, not yet read
  std::vector<TimerPair> spare;    // event pairs free for reuse
  PhaseTotal ph[4];
  std::vector<TimerPair>* capture_pairs = nullptr;  // non-null while capturing a graph

  // captured coarse multirate steps (CUDA graphs), valid for one layout
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    double dt = 0.0;
    int cur_before[kMaxLevel + 1] = {0};
    int cur_after[kMaxLevel + 1] = {0};
    bool timing = false;
    bool replayed = false;  // replayed since its timers were last read
    uint64_t kernels = 0;   // kernel nodes (counted per replay)
    std::vector<TimerPair> pairs;
  };
  bool use_graphs = true;
  // untimed executable graphs of a previous layout: a new capture of the same
  // shape updates one in place instead of instantiating a new one
  std::vector<cudaGraphExec_t> stale;
  // while a coarse step is captured: each level's point before and after
  // its latest update (ev_pre, ev_post; pre_ok, post_ok once recorded in the
  // step), and its stream's end (ev_fill)
  bool dag = false;
  cudaEvent_t ev_pre[kMaxLevel + 1] = {}, ev_post[kMaxLevel + 1] = {}, ev_fill[kMaxLevel + 1] = {};
  bool pre_ok[kMaxLevel + 1] = {}, post_ok[kMaxLevel + 1] = {};
  // a captured coarse step with fused fills runs each level on its own
  // stream (lev_stream[L], forked from ev_start), each update waiting only
  // for what it reads: the coarser level's state (before its latest update
  // at alpha = 0, after it otherwise) and the finer level's state at the
  // same time (after its latest update); the critical path is then the
  // finest level's chain of substeps, not all of them
  bool dag_levels = false;
  cudaStream_t lev_stream[kMaxLevel + 1] = {};
  bool lev_forked[kMaxLevel + 1] = {};
  cudaEvent_t ev_start = nullptr;
  std::vector<cudaEvent_t> ev_rev;  // the adjoint's reversed substeps (one per substep)
  // the adjoint's replay of a coarse step: times relative to the step start
  // (on the device), and where each substep keeps the update's ghost-filled
  // input tiles and the time-interpolated coarse tiles it read
  bool rel_time = false;
  void* keep_tiles = nullptr;
  void* keep_qT = nullptr;
  // autotuned patch-update configuration per launch size (bucket = log2 of
  // the patches in one launch): variant and warps per CTA
  struct Tune {
    bool tuned = false;
    int variant = ADV_STAGED, warps = 4;
    int fused = 1;  // substep fills the level's ghosts inside the update kernel
    float us = 0.f;
  };
  Tune tune[32];
  int forced_variant = -1, forced_warps = 4;
  int walk_ctas = 0;                    // cap on the walk grid (0: residency)
  uint32_t wait_polls = kWaitLimit;     // polls of the update kernels' bounded waits
  double vel_scale = 1.0;                 // multiplies every edge speed
  double* d_metric = nullptr;             // cubed sphere: FP64 metric blocks per patch
  double* d_corner = nullptr;             // deformational flow: grid corners per patch
  void* lam[2] = {nullptr, nullptr};      // adjoint tiles (patch-store layout), lazily allocated
  void* madj[3] = {nullptr, nullptr, nullptr};  // multirate adjoint: current, previous, qT tiles
  void* mio = nullptr;                    // multirate adjoint: lam in field layout (graph input)
  double* d_ds = nullptr;                 // multirate adjoint: the step's dscale (graph output)
  void* msnap = nullptr;                  // multirate adjoint: the start state, then the filled
  size_t msnap_bytes = 0;                 // tiles of every substep
  // an adjoint coarse step (mode 0: replay and reverse), a recorded
  // forward coarse step (1: fc_step_multirate_record into tape `slot`) or
  // the reverse of a recorded one (2: fc_adjoint_step_multirate_taped)
  struct AdjGraph {
    cudaGraphExec_t exec = nullptr;
    double dt = 0.0;
    int cur[kMaxLevel + 1] = {0};
    int cur_after[kMaxLevel + 1] = {0};  // mode 1: the buffer parities it leaves
    int mode = 0, slot = -1;
    uint64_t kernels = 0;
  };
  // tapes of recorded forward coarse steps: per slot the kept tiles of every
  // substep (the pool layout of the adjoint step without its start state),
  // the step's length and the buffer parities it started from
  struct Tape {
    void* pool = nullptr;
    size_t bytes = 0;
    bool valid = false;
    double dt = 0.0;
    int cur0[kMaxLevel + 1] = {0};  // the buffer parities the step started from
  };
  std::vector<Tape> tapes;
  std::vector<AdjGraph> adj_graphs;       // captured adjoint coarse steps, valid for one layout
  cudaStream_t cap_stream = nullptr;
  double* d_t0 = nullptr;  // start time of the replayed coarse step
  std::vector<Graph> graphs;
  // a partition's exchange lists on the device: for each level (kMaxLevel + 1:
  // all levels, level-major) and rank, the send then the receive list
  int* d_halo = nullptr;
  std::vector<size_t> halo_off;  // [((l * nranks + r) * 2 + dir)] offset; count at + 1
  // refluxing on the cubed sphere: the host pairing per device patch, face
  // and face cell (kind, patch across, its face, j0, j1), and the levels
  // that have any pair
  int* d_pairs = nullptr;
  bool pair_level[kMaxLevel + 1] = {};
};

namespace {

fc_forest::TimerPair take_pair(fc_forest* F) {
  if (!F->spare.empty()) {
    fc_forest::TimerPair p = F->spare.back();
    F->spare.pop_back();
    return p;
  }
  fc_forest::TimerPair p;
  if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) {
    p.a = p.b = nullptr;
  }
  return p;
}

// Brackets one launch with a pair of events when the forest's timers are on.
// While a graph is being captured the pair belongs to that graph.
class Timed {
 public:
  Timed(fc_forest* F, int phase, cudaStream_t s, double bytes) : s_(s) {
    if (!F->timing) return;
    fc_forest::TimerPair p = take_pair(F);
    if (!p.a) return;
    p.bytes = bytes;
    p.phase = phase;
    list_ = F->capture_pairs ? F->capture_pairs : &F->pending;
    list_->push_back(p);
    idx_ = list_->size() - 1;
    // inside a capture only an external record becomes an event-record node
    flags_ = F->capture_pairs ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaEventRecordWithFlags(p.a, s_, flags_);
  }
  ~Timed() {
    if (list_) cudaEventRecordWithFlags((*list_)[idx_].b, s_, flags_);
  }

 private:
  cudaStream_t s_;
  unsigned flags_ = cudaEventRecordDefault;
  std::vector<fc_forest::TimerPair>* list_ = nullptr;
  size_t idx_ = 0;
};

// add one timed launch to its phase's totals (waits for its end event)
cudaError_t account_pair(fc_forest* F, const fc_forest::TimerPair& p) {
  cudaError_t e = cudaEventSynchronize(p.b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
  if (e != cudaSuccess) return e;
  fc_forest::PhaseTotal& T = F->ph[p.phase];
  T.ms += t;
  T.bytes += p.bytes;
  T.launches += 1;
  return cudaSuccess;
}

// a replayed graph's event pairs hold only its latest replay: they are read
// before the graph is replayed again or destroyed
cudaError_t account_graph(fc_forest* F, fc_forest::Graph& g) {
  if (!g.replayed) return cudaSuccess;
  g.replayed = false;
  for (const auto& p : g.pairs) {
    cudaError_t e = account_pair(F, p);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void destroy_graphs(fc_forest* F) {
  for (auto& g : F->graphs) {
    account_graph(F, g);
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& p : g.pairs) F->spare.push_back(p);
  }
  F->graphs.clear();
  for (auto& g : F->adj_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  F->adj_graphs.clear();
  for (auto& x : F->stale) cudaGraphExecDestroy(x);
  F->stale.clear();
  for (auto& t : F->tapes) t.valid = false;  // recorded with the graphs' launches
}

// after a regrid: the captured steps are stale; untimed ones are kept for
// an in-place update by the next capture
void retire_graphs(fc_forest* F) {
  std::vector<cudaGraphExec_t> keep;
  for (auto& g : F->graphs)
    if (!g.timing && g.pairs.empty() && g.exec) {
      keep.push_back(g.exec);
      g.exec = nullptr;
    }
  destroy_graphs(F);
  F->stale = std::move(keep);
}

void destroy_timers(fc_forest* F) {
  destroy_graphs(F);
  for (auto* v : {&F->pending, &F->spare})
    for (auto& p : *v) {
      if (p.a) cudaEventDestroy(p.a);
      if (p.b) cudaEventDestroy(p.b);
    }
  F->pending.clear();
  F->spare.clear();
}

void free_tables(fc_forest* F) {
  dfree(F->d_tables);
  F->d_nbr = nullptr;
  F->d_meta = nullptr;
  F->d_lists = nullptr;
  F->d_api_to_dev = nullptr;
  F->d_fstart = nullptr;
  F->d_patch_sums = nullptr;
  F->d_mass = nullptr;
  F->d_delta = nullptr;
}

void free_device(fc_forest* F) {
  dfree(F->store);
  F->buf[0] = F->buf[1] = F->qT = F->stage = F->bflux = nullptr;
  free_tables(F);
  dfree(F->d_remap);
  dfree(F->d_err);
  dfree(F->d_t0);
  dfree(F->lam[0]);
  dfree(F->lam[1]);
  for (auto& b : F->madj) dfree(b);
  dfree(F->mio);
  dfree(F->d_ds);
  dfree(F->msnap);
  F->msnap_bytes = 0;
  for (auto& t : F->tapes) dfree(t.pool);
  F->tapes.clear();
  dfree(F->d_metric);
  dfree(F->d_corner);
  dfree(F->d_halo);
  dfree(F->d_pairs);
}

// cubed sphere: (re)compute the metric blocks of the current layout for the
// rotation vector times the velocity scale (synchronous); after a regrid the
// kept patches copy theirs from the old layout (rm, old: device).  The
// deformational flow keeps every patch's grid corners instead of fixed edge
// fluxes (its fluxes are refreshed per substep): all patches are computed.
fc_status update_metrics(fc_forest* F, const RemapEntry* rm = nullptr,
                         const double* old = nullptr) {
  const HostForest& H = F->host;
  if (H.desc.domain != FC_DOMAIN_SPHERE) return FC_OK;
  const int n = H.npatch();
  const int S = H.desc.mx + 2 * kMbc;
  const bool deform = H.desc.vel_kind == FC_VEL_DEFORM;
  dfree(F->d_metric);
  dfree(F->d_corner);
  if (dmalloc(&F->d_metric, (size_t)n * metric_stride(S)) != cudaSuccess)
    return fail(FC_ERR_OOM, "metric allocation failed");
  if (deform && dmalloc(&F->d_corner, (size_t)n * 3 * (S + 1) * (S + 1)) != cudaSuccess)
    return fail(FC_ERR_OOM, "corner allocation failed");
  double w[3] = {F->vel_scale * H.desc.vel[0], F->vel_scale * H.desc.vel[1],
                 F->vel_scale * H.desc.vel[2]};
  if (deform) {
    w[0] = w[1] = w[2] = 0.0;
    rm = nullptr;
    old = nullptr;
  }
  FC_CUDA(launch_sphere_metrics(F->d_meta, n, H.desc.mx, w, F->d_metric, rm, old, F->d_corner,
                                g_alloc_stream));
  return FC_OK;
}

// the deformational flow: the edge fluxes of level L's patches for the
// substep t -> t + dt (a: its update's arguments, whose time they share)
fc_status deform_fluxes(fc_forest* F, int p0, int p1, const AdvArgs& a, cudaStream_t s) {
  const fc_forest_desc& d = F->host.desc;
  if (d.vel_kind != FC_VEL_DEFORM || p1 <= p0) return FC_OK;
  const double kc = d.vel[0] * F->vel_scale, rot = 2.0 * M_PI / d.vel[2] * F->vel_scale;
  FC_CUDA(launch_deform_fluxes(p0, p1, d.mx, F->d_corner, F->d_metric, kc, d.vel[1], rot,
                               a.t_half, a.t0_dev, a.t_off, s));
  return FC_OK;
}

// upload tables (and allocate a store) for the current host layout; the
// sphere's metrics too unless the caller builds them (regrid)
fc_status upload(fc_forest* F, bool alloc_store, bool metrics = true) {
  const HostForest& H = F->host;
  const int n = H.npatch();
  const size_t S = (size_t)H.desc.mx + 2 * kMbc;
  const size_t cells = (size_t)n * S * S;
  if (alloc_store) {
    // buf[0], buf[1], qT, bflux zeroed (one memset), then stage; each part
    // 16-byte aligned
    dfree(F->store);
    F->buf[0] = F->buf[1] = F->qT = F->stage = F->bflux = nullptr;
    const size_t tb = (std::max<size_t>(cells, 1) * F->esize + 15) & ~(size_t)15;
    const size_t fb =
        H.desc.reflux ? ((size_t)std::max(n, 1) * 2 * 4 * H.desc.mx * F->esize + 15) & ~(size_t)15
                      : 0;
    if (dmalloc_bytes(&F->store, 4 * tb + fb) != cudaSuccess)
      return fail(FC_ERR_OOM, "device store allocation failed");
    char* base = static_cast<char*>(F->store);
    F->buf[0] = base;
    F->buf[1] = base + tb;
    F->qT = base + 2 * tb;
    F->bflux = fb ? base + 3 * tb : nullptr;
    F->stage = base + 3 * tb + fb;
    FC_CUDA(cudaMemsetAsync(F->store, 0, 3 * tb + fb, g_alloc_stream));
  }
  free_tables(F);
  // every work list, concatenated
  std::vector<int> lists;
  F->off_all = lists.size();
  lists.insert(lists.end(), H.list_all.begin(), H.list_all.end());
  F->off_coarse_all = lists.size();
  lists.insert(lists.end(), H.list_coarse_all.begin(), H.list_coarse_all.end());
  for (int l = 0; l <= kMaxLevel; ++l) {
    F->off_a[l] = lists.size();
    lists.insert(lists.end(), H.list_a[l].begin(), H.list_a[l].end());
    F->off_b[l] = lists.size();
    lists.insert(lists.end(), H.list_b[l].begin(), H.list_b[l].end());
    F->off_t[l] = lists.size();
    lists.insert(lists.end(), H.list_t[l].begin(), H.list_t[l].end());
  }
  // one block: the uploaded tables, the neighbour table, then the
  // device-written scratch (each part 16-byte aligned)
  const int nf = H.desc.nforests;
  size_t off = 0;
  const auto part = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 15) & ~(size_t)15;
    return at;
  };
  const size_t o_meta = part(sizeof(PatchMeta) * n), o_lists = part(sizeof(int) * lists.size()),
               o_api = part(sizeof(int) * n), o_fstart = part(sizeof(int) * (nf + 1));
  const size_t uploaded = off;
  const size_t o_nbr = part(sizeof(NbrEntry) * n * 8);  // its own copy, from the host table
  const size_t o_sums = part(sizeof(double) * n), o_mass = part(sizeof(double) * nf),
               o_delta = part(sizeof(double) * n);
  std::vector<char> host(uploaded, 0);
  std::memcpy(host.data() + o_meta, H.meta.data(), sizeof(PatchMeta) * n);
  if (!lists.empty()) std::memcpy(host.data() + o_lists, lists.data(), sizeof(int) * lists.size());
  std::memcpy(host.data() + o_api, H.dev_of.data(), sizeof(int) * n);
  std::memcpy(host.data() + o_fstart, H.forest_start.data(), sizeof(int) * (nf + 1));
  FC_CUDA(dmalloc_bytes(&F->d_tables, off));
  char* base = static_cast<char*>(F->d_tables);
  F->d_meta = reinterpret_cast<PatchMeta*>(base + o_meta);
  F->d_lists = reinterpret_cast<int*>(base + o_lists);
  F->d_api_to_dev = reinterpret_cast<int*>(base + o_api);
  F->d_fstart = reinterpret_cast<int*>(base + o_fstart);
  F->d_patch_sums = reinterpret_cast<double*>(base + o_sums);
  F->d_mass = reinterpret_cast<double*>(base + o_mass);
  F->d_delta = reinterpret_cast<double*>(base + o_delta);
  F->d_nbr = reinterpret_cast<NbrEntry*>(base + o_nbr);
  // (host sources are pageable: each copy has taken its data when it returns)
  FC_CUDA(cudaMemcpyAsync(F->d_tables, host.data(), uploaded, cudaMemcpyHostToDevice,
                          g_alloc_stream));
  FC_CUDA(cudaMemcpyAsync(F->d_nbr, H.nbr.data(), sizeof(NbrEntry) * n * 8,
                          cudaMemcpyHostToDevice, g_alloc_stream));
  // the coarse neighbours' ghost sources, on the device (the host goes on)
  FC_CUDA(launch_coarse_sources(F->d_nbr, F->d_meta, n, H.desc.mx,
                                H.desc.domain == FC_DOMAIN_WALLS ? 1 : 0, g_alloc_stream));
  if (!F->d_err) {
    FC_CUDA(dmalloc(&F->d_err, 1));
    FC_CUDA(cudaMemsetAsync(F->d_err, 0, sizeof(int), g_alloc_stream));
  }
  if (!F->d_t0) {
    FC_CUDA(dmalloc(&F->d_t0, 1));
    FC_CUDA(cudaMemsetAsync(F->d_t0, 0, sizeof(double), g_alloc_stream));
  }
  // refluxing on the cubed sphere: the pairing of coarse faces with finer
  // ones and of the cube edges' two sides, in device order
  dfree(F->d_pairs);
  for (bool& b : F->pair_level) b = false;
  if (H.desc.reflux && H.desc.domain == FC_DOMAIN_SPHERE) {
    const size_t row = (size_t)4 * H.desc.mx * 5;
    std::vector<int> field((size_t)n * row), tab((size_t)n * row);
    const std::string err = H.reflux_pairs(field.data());
    if (!err.empty()) return fail(FC_ERR_STATE, err);
    for (int k = 0; k < n; ++k) {
      const int* src = field.data() + (size_t)k * row;
      int* dst = tab.data() + (size_t)H.dev_of[k] * row;
      for (size_t r = 0; r < row; r += 5) {
        dst[r] = src[r];
        dst[r + 1] = src[r] ? H.dev_of[src[r + 1]] : -1;
        dst[r + 2] = src[r + 2];
        dst[r + 3] = src[r + 3];
        dst[r + 4] = src[r + 4];
        if (src[r]) F->pair_level[H.leaves[k].l] = true;
      }
    }
    FC_CUDA(dmalloc(&F->d_pairs, tab.size()));
    FC_CUDA(cudaMemcpyAsync(F->d_pairs, tab.data(), sizeof(int) * tab.size(),
                            cudaMemcpyHostToDevice, g_alloc_stream));
    // (pageable source: the copy has taken the data when it returns)
  }
  return metrics ? update_metrics(F) : FC_OK;
}

template <typename real>
DevForest<real> dev(const fc_forest* F) {
  DevForest<real> D{};
  const HostForest& H = F->host;
  D.mx = H.desc.mx;
  D.S = H.desc.mx + 2 * kMbc;
  D.npatch = H.npatch();
  D.napi = H.napi();
  D.domain = H.desc.domain;
  D.meta = F->d_meta;
  D.nbr = F->d_nbr;
  D.metric = F->d_metric;
  D.buf[0] = static_cast<real*>(F->buf[0]);
  D.buf[1] = static_cast<real*>(F->buf[1]);
  D.qT = static_cast<real*>(F->qT);
  for (int l = 0; l <= kMaxLevel; ++l) D.cur[l] = F->cur[l];
  D.vel_kind = H.desc.vel_kind;
  for (int k = 0; k < 4; ++k) D.vel[k] = H.desc.vel[k];
  if (D.vel_kind == FC_VEL_CONST) {  // the velocity scale multiplies every edge speed
    D.vel[0] *= F->vel_scale;
    D.vel[1] *= F->vel_scale;
  }
  D.order = H.desc.order;
  D.limiter = H.desc.limiter;
  D.transverse = H.desc.transverse;
  return D;
}

// per-launch scalars of the patch update for level L, step t -> t + dt; while
// a graph is captured, t is relative to the replayed step's start time
void choose_variant(const fc_forest* F, int n, AdvArgs* a);

AdvArgs adv_args(const fc_forest* F, int L, double t, double dt, int n) {
  const fc_forest_desc& d = F->host.desc;
  AdvArgs a{};
  a.h = std::ldexp(1.0, -L) / d.mx;
  a.nu = dt / a.h;
  a.dt = dt;
  a.period = d.vel[0];
  a.sfac = d.vel_kind == FC_VEL_SWIRL ? F->vel_scale * std::sin(M_PI * a.h) / (M_PI * a.h) : 0.0;
  a.t_half = t + 0.5 * dt;
  a.t_off = t + 0.5 * dt;
  a.t0_dev = (F->capture_pairs || F->rel_time) ? F->d_t0 : nullptr;
  a.variant = ADV_STAGED;
  a.warps = 4;
  a.ctas = F->walk_ctas;
  a.wait_limit = F->wait_polls;
  a.gather = 0;
  a.tlevel = -1;
  a.alpha = 0.0;
  a.bflux = F->bflux;
  a.bslot = 0;
  choose_variant(F, n, &a);
  return a;
}

int size_bucket(int n) {
  int b = 0;
  while ((2 << b) <= n && b < 31) ++b;
  return b;
}

// the patch-update configuration for a launch of n patches: the autotuned
// choice when this size was tuned, else walk for launches that fill the GPU
// (planar grids) and band for the others
void choose_variant(const fc_forest* F, int n, AdvArgs* a) {
  const fc_forest::Tune& t = F->tune[size_bucket(n)];
  if (F->forced_variant >= 0) {
    a->variant = F->forced_variant;
    a->warps = F->forced_warps;
  } else if (t.tuned) {
    a->variant = t.variant;
    a->warps = t.warps;
  } else if (n >= 1024 && !F->d_metric && F->host.desc.domain != FC_DOMAIN_SPHERE) {
    a->variant = ADV_WALK;  // (it has no capacity form)
    a->warps = F->esize == 4 ? 4 : 2;
  } else {
    a->variant = ADV_BAND;
    a->warps = 8;
  }
  // only the staged and band updates record the face fluxes
  if (F->bflux && a->variant != ADV_STAGED && a->variant != ADV_BAND) {
    a->variant = ADV_STAGED;
    a->warps = 4;
  }
}

// device error word -> status (and clear it)
fc_status check_device_error(fc_forest* F, cudaStream_t s) {
  int v = 0;
  FC_CUDA(cudaMemcpyAsync(&v, F->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FC_CUDA(cudaStreamSynchronize(s));
  if (v == 0) return FC_OK;
  FC_CUDA(cudaMemsetAsync(F->d_err, 0, sizeof(int), s));
  if (v & kErrTimeout) return fail(FC_ERR_TIMEOUT, "a bounded device wait gave up");
  return fail(FC_ERR_CUDA, "device error word set");
}

// algorithmic bytes of filling one patch's ghost ring (source read + write)
double ghost_bytes(const fc_forest* F) {
  const int mx = F->host.desc.mx;
  return 2.0 * (4.0 * (mx + 4) + 4.0 * mx) * (double)F->esize;
}

// algorithmic bytes of advancing n patches: read (mx+4)^2, write mx^2 each
double advance_bytes(const fc_forest* F, int n) {
  const double mx = F->host.desc.mx;
  // read the patch with its ghosts, write the interior; a mapped grid also
  // reads its FP64 metric block
  const double metric = F->d_metric ? 8.0 * metric_stride(F->host.desc.mx + 2 * kMbc) : 0.0;
  return (double)n * (((mx + 4) * (mx + 4) + mx * mx) * (double)F->esize + metric);
}

template <typename real>
fc_status fill_all_t(fc_forest* F, cudaStream_t s) {
  DevForest<real> D = dev<real>(F);
  const HostForest& H = F->host;
  const double gb = ghost_bytes(F);
  FillArgs A{F->d_lists + F->off_all, (int)H.list_all.size(), -1, 0.0};
  {
    Timed tm(F, 1, s, gb * A.ntargets);
    FC_CUDA(launch_fill_coarse(D, A, s));
  }
  FillArgs B{F->d_lists + F->off_coarse_all, (int)H.list_coarse_all.size(), -1, 0.0};
  {
    Timed tm(F, 1, s, gb * B.ntargets);
    FC_CUDA(launch_fill_fine(D, B, s));
  }
  return FC_OK;
}

fc_status fill_all(fc_forest* F, cudaStream_t s) {
  return F->esize == 4 ? fill_all_t<float>(F, s) : fill_all_t<double>(F, s);
}

// the adjoint's replay: copy the time-interpolated tiles of level L-1 (what
// level L's interpolation reads) to where the adjoint will read them
cudaError_t keep_coarse_tiles(fc_forest* F, int L, cudaStream_t s) {
  const HostForest& H = F->host;
  if (!F->keep_qT || L <= H.desc.lmin) return cudaSuccess;
  const size_t tile = (size_t)(H.desc.mx + 2 * kMbc) * (H.desc.mx + 2 * kMbc) * F->esize;
  const int a = H.lev_start[L - 1], b = H.lev_start[L];
  if (b <= a) return cudaSuccess;
  return cudaMemcpyAsync(F->keep_qT, static_cast<char*>(F->qT) + (size_t)a * tile,
                         (size_t)(b - a) * tile, cudaMemcpyDeviceToDevice, s);
}

// the level streams and events of captured steps (created outside a capture)
fc_status ensure_streams(fc_forest* F) {
  if (F->ev_start) return FC_OK;
  for (int l = 0; l <= kMaxLevel; ++l)
    for (cudaEvent_t* ev : {&F->ev_pre[l], &F->ev_post[l], &F->ev_fill[l]})
      FC_CUDA(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  for (int l = 0; l <= kMaxLevel; ++l)
    FC_CUDA(cudaStreamCreateWithFlags(&F->lev_stream[l], cudaStreamNonBlocking));
  FC_CUDA(cudaEventCreateWithFlags(&F->ev_start, cudaEventDisableTiming));  // last: "created"
  return FC_OK;
}

template <typename real>
fc_status advance_level_t(fc_forest* F, int L, double t, double dt, cudaStream_t s) {
  const HostForest& H = F->host;
  // updated: the level's patches (a partition: its owned ones); held: any
  // patch of the level here, mirrors included, whose state buffer turns over
  const int p0 = H.lev_start[L], p1 = H.upd_end(L);
  const bool held = H.lev_start[L + 1] > p0;
  int tlevel = -1;
  double alpha = 0.0;
  if (L > H.desc.lmin && F->has_old[L - 1] && F->dt_last[L - 1] > 0.0) {
    tlevel = L - 1;
    alpha = (t - F->t_start[L - 1]) / F->dt_last[L - 1];
    alpha = std::min(1.0, std::max(0.0, alpha));
  }
  DevForest<real> D = dev<real>(F);
  if (p1 > p0) {
    const double gb = ghost_bytes(F);
    AdvArgs a = adv_args(F, L, t, dt, p1 - p0);
    const fc_forest::Tune& tn = F->tune[size_bucket(p1 - p0)];
    const bool fused = F->fuse && (F->forced_variant >= 0 || !tn.tuned || tn.fused);
    // per-level streams of a captured step (see fc_forest::dag_levels)
    const bool lev = F->dag_levels;
    if (lev) {
      s = F->lev_stream[L];
      if (!F->lev_forked[L]) {
        FC_CUDA(cudaStreamWaitEvent(s, F->ev_start, 0));
        F->lev_forked[L] = true;
      }
      // the coarser level's state this substep reads: from before its
      // latest update (alpha = 0) or after it
      if (tlevel >= 0) {
        if (alpha == 0.0) {
          if (F->pre_ok[L - 1]) FC_CUDA(cudaStreamWaitEvent(s, F->ev_pre[L - 1], 0));
        } else if (F->post_ok[L - 1]) {
          FC_CUDA(cudaStreamWaitEvent(s, F->ev_post[L - 1], 0));
        }
      }
      // separate fills also read the finer level now
      if (!fused && L < H.desc.lmax && F->post_ok[L + 1])
        FC_CUDA(cudaStreamWaitEvent(s, F->ev_post[L + 1], 0));
    }
    if (fused) {
      // coarse neighbours first (their interiors time-interpolated into qT,
      // their coarse ghost regions filled); the update kernel then fills
      // each level-L patch's ghost ring in shared memory itself
      FillArgs A{F->d_lists + F->off_t[L], (int)H.list_t[L].size(), tlevel, alpha};
      // the staged and band updates compute the time-interpolated coarse
      // cells they read themselves, so no fill launch sits before them on
      // the level's chain (at alpha = 0 from the coarser level's older
      // state, which its running update does not write); in the adjoint's
      // replay they also store those cells in the kept time-interpolated
      // tiles, all the reverse reads of them.  The walk keeps the fill: with
      // one warp per patch, computing those cells in the update measured
      // slower on the ensemble (5.5e10 vs 7.4e10 cell-updates/s)
      const bool direct = tlevel >= 0 && (a.variant == ADV_STAGED || a.variant == ADV_BAND);
      if (direct) A.ntargets = 0;
      a.direct = direct ? 1 : 0;
      if (direct && F->keep_qT) {
        a.keep_t = F->keep_qT;
        a.keep_t_p0 = H.lev_start[L - 1];
      }
      // (inside a captured step this runs on the level's own stream, after
      // the waits above: see fc_forest::dag_levels)
      {
        Timed tm(F, 1, s, gb * A.ntargets);
        FC_CUDA(launch_fill_coarse(D, A, s));
      }
      if (!direct) FC_CUDA(keep_coarse_tiles(F, L, s));
      a.gather = 1;
      a.tlevel = tlevel;
      a.alpha = alpha;
    } else {
      FillArgs A{F->d_lists + F->off_a[L], (int)H.list_a[L].size(), tlevel, alpha};
      {
        Timed tm(F, 1, s, gb * A.ntargets);
        FC_CUDA(launch_fill_coarse(D, A, s));
      }
      FillArgs B{F->d_lists + F->off_b[L], (int)H.list_b[L].size(), tlevel, alpha};
      {
        Timed tm(F, 1, s, gb * B.ntargets);
        FC_CUDA(launch_fill_fine(D, B, s));
      }
      FC_CUDA(keep_coarse_tiles(F, L, s));
    }
    a.keep = F->keep_tiles;
    a.keep_p0 = p0;
    a.bslot = alpha != 0.0 ? 1 : 0;  // the second substep of a pair
    F->bslot[L] = a.bslot;
    // the update reads the finer level at this time: after its latest update
    if (lev && fused && L < H.desc.lmax && F->post_ok[L + 1])
      FC_CUDA(cudaStreamWaitEvent(s, F->ev_post[L + 1], 0));
    if (F->dag) {
      FC_CUDA(cudaEventRecord(F->ev_pre[L], s));
      F->pre_ok[L] = true;
    }
    {
      const fc_status fs = deform_fluxes(F, p0, p1, a, s);
      if (fs != FC_OK) return fs;
    }
    {
      Timed tm(F, 0, s, advance_bytes(F, p1 - p0));
      FC_CUDA(launch_advance(D, p0, p1, a, F->d_err, s));
    }
    if (F->dag) {
      FC_CUDA(cudaEventRecord(F->ev_post[L], s));
      F->post_ok[L] = true;
    }
  }
  if (held) F->cur[L] ^= 1;
  F->has_old[L] = true;
  F->t_start[L] = t;
  F->dt_last[L] = dt;
  return FC_OK;
}

fc_status advance_level(fc_forest* F, int L, double t, double dt, cudaStream_t s) {
  return F->esize == 4 ? advance_level_t<float>(F, L, t, dt, s)
                       : advance_level_t<double>(F, L, t, dt, s);
}

// refluxing of level L after one of its updates of length dt: with nfs
// finer substeps of weight w (see fc_step_multirate); on the cubed sphere
// from the host pairing, whose fluxes are volume fluxes (the weight is the
// time ratio alone, 2 w) and which also exchanges the cube edges' fluxes
bool reflux_due(const fc_forest* F, int L) {
  const HostForest& H = F->host;
  if (!F->bflux || H.lev_start[L + 1] <= H.lev_start[L]) return false;
  if (F->d_pairs) return F->pair_level[L];
  return L < H.desc.lmax && H.lev_start[L + 2] > H.lev_start[L + 1];
}

fc_status reflux_level(fc_forest* F, int L, double dt, int nfs, double w, cudaStream_t s) {
  const HostForest& H = F->host;
  const int p0 = H.lev_start[L], p1 = H.lev_start[L + 1];
  if (!reflux_due(F, L)) return FC_OK;
  Timed tm(F, 3, s, 0.0);
  cudaError_t e;
  if (F->d_pairs) {
    e = F->esize == 4
            ? launch_reflux_pairs(dev<float>(F), p0, p1, static_cast<const float*>(F->bflux),
                                  F->d_pairs, F->bslot[L], nfs, 2.0 * w, dt, s)
            : launch_reflux_pairs(dev<double>(F), p0, p1, static_cast<const double*>(F->bflux),
                                  F->d_pairs, F->bslot[L], nfs, 2.0 * w, dt, s);
  } else {
    const double nu = dt / (std::ldexp(1.0, -L) / H.desc.mx);
    e = F->esize == 4 ? launch_reflux(dev<float>(F), p0, p1, static_cast<const float*>(F->bflux),
                                      F->bslot[L], nfs, w, nu, s)
                      : launch_reflux(dev<double>(F), p0, p1,
                                      static_cast<const double*>(F->bflux), F->bslot[L], nfs, w,
                                      nu, s);
  }
  return e == cudaSuccess ? FC_OK : cuda_fail(e, "reflux");
}

fc_status multirate(fc_forest* F, int L, double t, double dt, cudaStream_t s) {
  fc_status st = advance_level(F, L, t, dt, s);
  if (st != FC_OK) return st;
  const int lmax = F->host.desc.lmax;
  if (L < lmax) {
    if ((st = multirate(F, L + 1, t, 0.5 * dt, s)) != FC_OK) return st;
    if ((st = multirate(F, L + 1, t + 0.5 * dt, 0.5 * dt, s)) != FC_OK) return st;
  }
  if (reflux_due(F, L)) {
    // after both finer substeps (their fluxes written, their reads of this
    // level's states done); on a captured step's level stream, and the
    // level's post-update event moves past the correction (what the coarser
    // level and this level's next substep read)
    if (F->dag_levels) {
      s = F->lev_stream[L];
      if (L < lmax && F->post_ok[L + 1]) FC_CUDA(cudaStreamWaitEvent(s, F->ev_post[L + 1], 0));
    }
    if ((st = reflux_level(F, L, dt, 2, 0.25, s)) != FC_OK) return st;
    if (F->dag) {
      FC_CUDA(cudaEventRecord(F->ev_post[L], s));
      F->post_ok[L] = true;
    }
  }
  return FC_OK;
}

void reset_times(fc_forest* F) {
  for (int l = 0; l <= kMaxLevel; ++l) {
    F->has_old[l] = false;
    F->t_start[l] = 0.0;
    F->dt_last[l] = 0.0;
  }
}

fc_status check_desc(const fc_forest_desc* d) {
  if (!d) return fail(FC_ERR_INVALID_ARG, "null descriptor");
  if (d->mx != 8 && d->mx != 16 && d->mx != 32)
    return fail(FC_ERR_INVALID_ARG, "mx must be 8, 16 or 32");
  if (d->mbc != kMbc) return fail(FC_ERR_INVALID_ARG, "only mbc = 2 is built");
  if (4 * d->mbc > d->mx) return fail(FC_ERR_PRECONDITION, "Proposition 1 needs mbc <= mx/4");
  if (d->lmin < 0 || d->lmax > 16 || d->lmin > d->lmax)
    return fail(FC_ERR_INVALID_ARG, "level range must satisfy 0 <= lmin <= lmax <= 16");
  if (d->nforests < 1 || d->nforests > 65535) return fail(FC_ERR_INVALID_ARG, "bad nforests");
  if (d->dtype != FC_F32 && d->dtype != FC_F64) return fail(FC_ERR_INVALID_ARG, "bad dtype");
  if (d->domain != FC_DOMAIN_WALLS && d->domain != FC_DOMAIN_PERIODIC &&
      d->domain != FC_DOMAIN_SPHERE && d->domain != FC_DOMAIN_BRICK)
    return fail(FC_ERR_INVALID_ARG, "bad domain");
  if (d->domain == FC_DOMAIN_BRICK &&
      (d->brick_nx < 1 || d->brick_ny < 1 || d->brick_nx * d->brick_ny > 256))
    return fail(FC_ERR_INVALID_ARG, "a brick needs 1..256 blocks (brick_nx, brick_ny >= 1)");
  if (d->vel_kind != FC_VEL_CONST && d->vel_kind != FC_VEL_SWIRL &&
      d->vel_kind != FC_VEL_ROTATION && d->vel_kind != FC_VEL_DEFORM)
    return fail(FC_ERR_INVALID_ARG, "bad velocity kind");
  if ((d->domain == FC_DOMAIN_SPHERE) !=
      (d->vel_kind == FC_VEL_ROTATION || d->vel_kind == FC_VEL_DEFORM))
    return fail(FC_ERR_INVALID_ARG,
                "the cubed sphere takes the solid-body rotation or the deformational flow, and "
                "only they");
  if (d->vel_kind == FC_VEL_DEFORM && !(d->vel[1] != 0.0 && d->vel[2] != 0.0))
    return fail(FC_ERR_INVALID_ARG, "the deformational flow needs nonzero T and T_f");
  if (d->vel_kind == FC_VEL_SWIRL && !(d->vel[0] != 0.0))
    return fail(FC_ERR_INVALID_ARG, "swirl period must be nonzero");
  if (d->order < 1 || d->order > 2 || d->limiter < 0 || d->limiter > 1 || d->transverse < 0 ||
      d->transverse > 2)
    return fail(FC_ERR_INVALID_ARG, "bad scheme options");
  if (d->indicator < 0 || d->indicator > 1 || d->smooth < 0 || d->smooth > 1)
    return fail(FC_ERR_INVALID_ARG, "bad regrid policy");
  if (d->reflux < 0 || d->reflux > 1) return fail(FC_ERR_INVALID_ARG, "reflux must be 0 or 1");
  return FC_OK;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

const char* fc_last_error(void) { return g_err.c_str(); }

uint64_t fc_launch_count(int reset) {
  uint64_t v = launch_counter();
  if (reset) launch_counter() = 0;
  return v;
}

fc_status fc_set_allocator(fc_alloc_fn alloc, fc_free_fn release, void* user) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(FC_ERR_INVALID_ARG, "fc_set_allocator: give both functions or neither");
  if (g_live_forests.load() != 0)
    return fail(FC_ERR_STATE, "fc_set_allocator: forests are alive (destroy them first)");
  g_hook = AllocHook{alloc, release, user};
  return FC_OK;
}

fc_status fc_forest_info(const fc_forest* F, fc_info* out) {
  if (!F || !out) return fail(FC_ERR_INVALID_ARG, "null argument");
  const HostForest& H = F->host;
  std::memset(out, 0, sizeof *out);
  out->nleaves = H.napi();
  out->nforests = H.desc.nforests;
  out->mx = H.desc.mx;
  out->mbc = H.desc.mbc;
  out->lmin = H.desc.lmin;
  out->lmax = H.desc.lmax;
  out->dtype = H.desc.dtype;
  out->domain = H.desc.domain;
  for (int l = 0; l <= kMaxLevel && l < FC_INFO_LEVELS; ++l)  // (a partition: its own leaves)
    out->leaves_per_level[l] = H.upd_end(l) - H.lev_start[l];
  const size_t S = (size_t)H.desc.mx + 2 * kMbc;
  const size_t n = (size_t)std::max(H.npatch(), 1);
  const size_t store = n * S * S * F->esize;
  size_t bytes = 4 * store;  // two state buffers, the time-interpolated tiles, the stage
  if (F->bflux) bytes += n * 2 * 4 * H.desc.mx * F->esize;
  bytes += sizeof(NbrEntry) * n * 8 + sizeof(PatchMeta) * n + 3 * sizeof(double) * n;
  if (F->d_metric) bytes += sizeof(double) * n * metric_stride((int)S);
  if (F->d_corner) bytes += sizeof(double) * n * 3 * (S + 1) * (S + 1);
  for (void* b : F->lam) bytes += b ? store : 0;
  for (void* b : F->madj) bytes += b ? store : 0;
  if (F->mio) bytes += n * H.desc.mx * H.desc.mx * F->esize;
  bytes += F->msnap_bytes;
  for (const auto& t : F->tapes) bytes += t.bytes;
  out->device_bytes = (int64_t)bytes;
  out->graphs = (int)(F->graphs.size() + F->adj_graphs.size());
  int tuned = 0;
  for (const auto& t : F->tune) tuned += t.tuned ? 1 : 0;
  out->tuned_buckets = tuned;
  if (F->d_nbr && H.npatch() > 0) {  // the ghost sources the device wrote
    std::vector<NbrEntry> rows((size_t)H.npatch() * 8);
    FC_CUDA(cudaDeviceSynchronize());
    FC_CUDA(cudaMemcpy(rows.data(), F->d_nbr, sizeof(NbrEntry) * rows.size(),
                       cudaMemcpyDeviceToHost));
    for (const NbrEntry& e : rows)
      if (e.kind == NB_COARSE) {
        ++out->coarse_entries;
        out->coarse_unlisted += (e.code[0] & kSrcComplete) ? 0 : 1;
      }
  }
  return FC_OK;
}

fc_status fc_forest_create(const fc_forest_desc* desc, int nleaves, const int* leaves,
                           fc_forest** out) {
  if (!out) return fail(FC_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  fc_status st = check_desc(desc);
  if (st != FC_OK) return st;
  if (nleaves < 1 || !leaves) return fail(FC_ERR_INVALID_ARG, "empty leaf list");
  fc_forest* F = new (std::nothrow) fc_forest();
  if (!F) return fail(FC_ERR_OOM, "host allocation failed");
  F->host.desc = *desc;
  F->esize = desc->dtype == FC_F32 ? 4 : 8;
  F->host.leaves.resize(nleaves);
  for (int k = 0; k < nleaves; ++k)
    F->host.leaves[k] = Leaf{leaves[5 * k], leaves[5 * k + 1], leaves[5 * k + 2],
                             leaves[5 * k + 3], leaves[5 * k + 4]};
  std::string err = F->host.build();
  if (!err.empty()) {
    delete F;
    return fail(FC_ERR_PRECONDITION, err);
  }
  keep_pool_memory();
  st = upload(F, true);  // on the legacy default stream
  if (st == FC_OK && cudaStreamSynchronize(0) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "create");
  if (st != FC_OK) {
    free_device(F);
    cudaStreamSynchronize(0);
    delete F;
    return st;
  }
  *out = F;
  g_live_forests.fetch_add(1);
  return FC_OK;
}

fc_status fc_forest_destroy(fc_forest* F) {
  if (!F) return FC_OK;
  g_live_forests.fetch_sub(1);
  cudaDeviceSynchronize();
  destroy_timers(F);
  if (F->cap_stream) cudaStreamDestroy(F->cap_stream);
  if (F->ev_start) {
    for (int l = 0; l <= kMaxLevel; ++l)
      for (cudaEvent_t ev : {F->ev_pre[l], F->ev_post[l], F->ev_fill[l]})
        if (ev) cudaEventDestroy(ev);
    if (F->ev_start) cudaEventDestroy(F->ev_start);
    for (cudaEvent_t ev : F->ev_rev)
      if (ev) cudaEventDestroy(ev);
    for (cudaStream_t ls : F->lev_stream)
      if (ls) cudaStreamDestroy(ls);
  }
  free_device(F);
  cudaStreamSynchronize(0);
  delete F;
  return FC_OK;
}

fc_status fc_timers_enable(fc_forest* F, int enable) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  F->timing = enable != 0;
  return FC_OK;
}

fc_status fc_timers_read(fc_forest* F, int phase, double* ms, int64_t* launches, double* bytes,
                         int reset) {
  if (!F || phase < 0 || phase > 3) return fail(FC_ERR_INVALID_ARG, "bad phase");
  for (const auto& p : F->pending) {
    FC_CUDA(account_pair(F, p));
    F->spare.push_back(p);
  }
  F->pending.clear();
  for (auto& g : F->graphs) FC_CUDA(account_graph(F, g));
  fc_forest::PhaseTotal& T = F->ph[phase];
  if (ms) *ms = T.ms;
  if (launches) *launches = T.launches;
  if (bytes) *bytes = T.bytes;
  if (reset) T = fc_forest::PhaseTotal{};
  return FC_OK;
}

fc_status fc_mass_noalloc(const void* q, const double* capacity, int dtype, int mx, int nleaves,
                          const int* level, const int* forest_start, int nforests, double* out,
                          void* stream) {
  if (!q || !level || !forest_start || !out)
    return fail(FC_ERR_INVALID_ARG, "fc_mass_noalloc: null pointer");
  if (dtype != FC_F32 && dtype != FC_F64)
    return fail(FC_ERR_INVALID_ARG, "fc_mass_noalloc: dtype must be FC_F32 or FC_F64");
  if (mx < 1 || nleaves < 1 || nforests < 1)
    return fail(FC_ERR_INVALID_ARG, "fc_mass_noalloc: mx, nleaves and nforests must be >= 1");
  if (nleaves > FC_NOALLOC_MAX_LEAVES)
    return fail(FC_ERR_INVALID_ARG, "fc_mass_noalloc: nleaves " + std::to_string(nleaves) +
                                        " exceeds FC_NOALLOC_MAX_LEAVES (" +
                                        std::to_string(FC_NOALLOC_MAX_LEAVES) + ")");
  cudaError_t e = noalloc_mass(q, capacity, dtype, mx, nleaves, level, forest_start, nforests,
                               out, as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "fc_mass_noalloc");
  return FC_OK;
}

fc_status fc_forest_get_capacity(const fc_forest* F, double* out, int on_device, void* stream) {
  if (!F || !out) return fail(FC_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = as_stream(stream);
  const size_t n = (size_t)F->host.napi() * F->host.desc.mx * F->host.desc.mx;
  double* dst = out;
  if (!on_device && F->esize < sizeof(double)) {
    // the staging buffer holds a float field: stage through a temporary
    AllocStream alloc_on(s);
    if (dmalloc(&dst, n) != cudaSuccess) return fail(FC_ERR_OOM, "staging allocation failed");
  } else if (!on_device) {
    dst = static_cast<double*>(F->stage);
  }
  const cudaError_t e =
      F->esize == 4 ? launch_pack_capacity(dev<float>(F), F->d_api_to_dev, dst, s)
                    : launch_pack_capacity(dev<double>(F), F->d_api_to_dev, dst, s);
  if (e != cudaSuccess) return cuda_fail(e, "pack capacity");
  if (!on_device) {
    FC_CUDA(cudaMemcpyAsync(out, dst, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (dst != F->stage) {
      AllocStream alloc_on(s);
      dfree(dst);
    }
    FC_CUDA(cudaStreamSynchronize(s));
    return check_device_error(const_cast<fc_forest*>(F), s);
  }
  return FC_OK;
}

fc_status fc_set_advance_variant(fc_forest* F, int variant, int warps) {
  const bool warps_ok = warps == 2 || warps == 4 || warps == 8 || (warps == 16 && variant == ADV_BAND);
  if (!F || variant < -1 || variant > ADV_BAND || !warps_ok)
    return fail(FC_ERR_INVALID_ARG,
                "variant must be -1, 0, 1, 2 or 3 and warps 2, 4 or 8 (16 with variant 3)");
  F->forced_variant = variant;
  F->forced_warps = warps;
  destroy_graphs(F);
  return FC_OK;
}

fc_status fc_set_limits(fc_forest* F, int walk_ctas, int64_t wait_polls) {
  if (!F || walk_ctas < 0 || wait_polls > (int64_t)UINT32_MAX)
    return fail(FC_ERR_INVALID_ARG, "walk_ctas must be >= 0 and wait_polls < 2^32");
  F->walk_ctas = walk_ctas;
  F->wait_polls = wait_polls < 0 ? kWaitLimit : (uint32_t)wait_polls;
  destroy_graphs(F);  // captured launches carry the old values
  return FC_OK;
}

fc_status fc_autotune(fc_forest* F, int* report, void* stream) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  cudaStream_t s = as_stream(stream);
  const HostForest& H = F->host;
  const struct {
    int variant, warps;
  // (band with 16 warps is left out: timed a level at a time it can win,
  // but beside the other levels' branches of a captured step it measured
  // slower than with 8)
  } cand[] = {{ADV_STAGED, 4}, {ADV_BAND, 4}, {ADV_BAND, 8},  {ADV_WALK, 2},
              {ADV_WALK, 4},   {ADV_WALK, 8}, {ADV_WALK1, 4}, {ADV_WALK1, 8}};
  constexpr int ncand = sizeof(cand) / sizeof(cand[0]);
  cudaEvent_t e0, e1;
  FC_CUDA(cudaEventCreate(&e0));
  FC_CUDA(cudaEventCreate(&e1));
  if (!F->cap_stream) FC_CUDA(cudaStreamCreateWithFlags(&F->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = F->cap_stream;
  int dev_id = 0, nsm = 0;
  FC_CUDA(cudaGetDevice(&dev_id));
  FC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_id));
  DevForest<float> Df = dev<float>(F);
  DevForest<double> Dd = dev<double>(F);
  fc_status st = FC_OK;
  for (int L = H.desc.lmin; L <= H.desc.lmax && st == FC_OK; ++L) {
    const int p0 = H.lev_start[L], p1 = H.upd_end(L);
    if (p1 <= p0) continue;
    fc_forest::Tune& t = F->tune[size_bucket(p1 - p0)];
    if (t.tuned) continue;
    AdvArgs a = adv_args(F, L, 0.0, 0.5 * std::ldexp(1.0, -L) / H.desc.mx, p1 - p0);
    float best = 1e30f;
    // every candidate is timed as a whole substep: its fills plus the update
    for (int c2 = 0; c2 < 2 * ncand; ++c2) {
      const auto& c = cand[c2 % ncand];
      const int fused = c2 / ncand;
      if (fused && !F->fuse) continue;
      const bool walk = c.variant == ADV_WALK || c.variant == ADV_WALK1;
      // no capacity form in walk
      if (walk && (F->d_metric || H.desc.domain == FC_DOMAIN_SPHERE)) continue;
      if (walk && F->bflux) continue;  // (it would run staged)
      // below two patches per SM the walk's warps mostly idle: staged has
      // measured about twice as fast there (graph-replayed substeps)
      if (walk && p1 - p0 < 2 * nsm) continue;
      // a band of one row recomputes three rows of x-edges
      if (c.variant == ADV_BAND && H.desc.mx * H.desc.mx < 64 * c.warps) continue;
      a.variant = c.variant;
      a.warps = c.warps;
      a.gather = fused;
      a.tlevel = -1;
      auto run = [&]() {
        cudaError_t e;
        if (fused) {
          FillArgs A{F->d_lists + F->off_t[L], (int)H.list_t[L].size(), -1, 0.0};
          e = F->esize == 4 ? launch_fill_coarse(Df, A, s) : launch_fill_coarse(Dd, A, s);
        } else {
          FillArgs A{F->d_lists + F->off_a[L], (int)H.list_a[L].size(), -1, 0.0};
          FillArgs B{F->d_lists + F->off_b[L], (int)H.list_b[L].size(), -1, 0.0};
          e = F->esize == 4 ? launch_fill_coarse(Df, A, s) : launch_fill_coarse(Dd, A, s);
          if (e == cudaSuccess)
            e = F->esize == 4 ? launch_fill_fine(Df, B, s) : launch_fill_fine(Dd, B, s);
        }
        if (e != cudaSuccess) return e;
        return F->esize == 4 ? launch_advance(Df, p0, p1, a, F->d_err, s)
                             : launch_advance(Dd, p0, p1, a, F->d_err, s);
      };
      // timed as in a captured step: kRep substeps in one graph, so the
      // launches' host cost (which dominates direct launches of small
      // levels) stays out of the comparison
      constexpr int kRep = 8;
      cudaError_t e = run();  // warm-up (module load, attributes)
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        std::swap(s, cs);  // run() launches on s
        for (int k = 0; k < kRep && e == cudaSuccess; ++k) e = run();
        std::swap(s, cs);
        const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = ee;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);  // warm
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "autotune");
        break;
      }
      const float us = 1e3f * ms / (2.f * kRep);
      if (us < best) {
        best = us;
        t.variant = c.variant;
        t.warps = c.warps;
        t.fused = fused;
        t.us = us;
      }
    }
    t.tuned = st == FC_OK;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FC_OK) return st;
  // the candidates overwrote the previous-state buffers
  reset_times(F);
  destroy_graphs(F);
  if (report)
    for (int b = 0; b < 32; ++b) {
      report[4 * b] = F->tune[b].tuned ? F->tune[b].variant : -1;
      report[4 * b + 1] = F->tune[b].warps;
      report[4 * b + 2] = F->tune[b].fused;
      report[4 * b + 3] = (int)(1e3f * F->tune[b].us);
    }
  return check_device_error(F, s);
}

fc_status fc_set_velocity_scale(fc_forest* F, double scale) {
  if (!F || !(scale == scale)) return fail(FC_ERR_INVALID_ARG, "bad velocity scale");
  if (scale == F->vel_scale) return FC_OK;  // the captured steps and tapes stay valid
  F->vel_scale = scale;
  destroy_graphs(F);
  FC_CUDA(cudaDeviceSynchronize());  // no launch may still read the old metrics
  fc_status st = update_metrics(F);   // sphere: the edge fluxes carry the scale
  if (st == FC_OK) FC_CUDA(cudaStreamSynchronize(0));
  return st;
}

}  // extern "C"

template <typename real>
static fc_status adjoint_step_t(fc_forest* F, double t, double dt, void* lam, double* dscale,
                                cudaStream_t s) {
  AllocStream alloc_on(s);
  const HostForest& H = F->host;
  const size_t S = (size_t)H.desc.mx + 2 * kMbc;
  const size_t cells = std::max<size_t>((size_t)H.npatch() * S * S, 1);
  for (int b = 0; b < 2; ++b)
    if (!F->lam[b] && dmalloc_bytes(&F->lam[b], cells * sizeof(real)) != cudaSuccess)
      return fail(FC_ERR_OOM, "adjoint buffer allocation failed");
  // the caller's adjoint (field layout) into the interior of lam[0]
  DevForest<real> L = dev<real>(F);
  L.buf[0] = L.buf[1] = static_cast<real*>(F->lam[0]);
  for (int l = 0; l <= kMaxLevel; ++l) L.cur[l] = 0;
  FC_CUDA(launch_unpack(L, F->d_api_to_dev, static_cast<const real*>(lam), s));
  // the forward ghost fill of the current state: the forward tiles
  fc_status st = fill_all(F, s);
  if (st != FC_OK) return st;
  AdjArgs g{};
  g.t = t;
  g.dt = dt;
  g.period = H.desc.vel[0];
  g.scale = F->vel_scale;
  g.dscale_factor = F->vel_scale != 0.0 ? 1.0 / F->vel_scale : 0.0;
  g.lev_start = H.lev_start;
  g.coarse_list = F->d_lists + F->off_coarse_all;
  g.ncoarse = (int)H.list_coarse_all.size();
  {
    Timed tm(F, 3, s, 0.0);
    FC_CUDA(launch_adjoint_step(dev<real>(F), g, static_cast<const real*>(F->lam[0]),
                                static_cast<real*>(F->lam[1]), dscale, s));
  }
  L.buf[0] = L.buf[1] = static_cast<real*>(F->lam[1]);
  FC_CUDA(launch_pack(L, F->d_api_to_dev, static_cast<real*>(lam), 0, s));
  return FC_OK;
}

// Adjoint of one coarse multirate step (the coarse-first recursion of
// fc_step_multirate).  The forward step is replayed once, keeping after each
// substep's fill the level's ghost-filled tiles and the time-interpolated
// coarse tiles (qT) it read; the substeps are then reversed, each on its kept
// tiles.  The whole sequence is captured once per (layout, dt, buffer
// parity) as a CUDA graph and replayed; the step's start time, lam and
// dscale pass through device buffers of the forest.  The forest is left at
// the step's start state.
//
// mode 1 captures the replay alone, as a recorded forward step: it keeps the
// same tiles in tape `slot` (no start state saved) and leaves the forest at
// the step's end state; mode 2 captures the reverse alone, from that tape.
template <typename real>
static fc_status capture_adjoint_multirate(fc_forest* F, double dtc, cudaStream_t cs,
                                           fc_forest::AdjGraph* out, int mode = 0,
                                           int slot = -1) {
  const HostForest& H = F->host;
  const int lmin = H.desc.lmin, lmax = H.desc.lmax;
  const size_t S2 = (size_t)(H.desc.mx + 2 * kMbc) * (H.desc.mx + 2 * kMbc);
  const size_t tile = S2 * sizeof(real);
  const size_t cells = std::max<size_t>((size_t)H.npatch() * S2, 1);
  struct Sub {
    int L, j;             // level and its substep index in the step
    double t, dt, alpha;  // t relative to the step's start
    size_t offq, offt;    // byte offsets of the kept level-L tiles and qT tiles
    int cur[kMaxLevel + 1];
  };
  std::vector<Sub> subs;
  int nsub[kMaxLevel + 2] = {0};
  std::function<void(int, double, double, double)> rec = [&](int L, double t, double dt,
                                                               double alpha) {
    subs.push_back(Sub{L, nsub[L]++, t, dt, alpha, 0, 0, {0}});
    if (L < lmax) {
      rec(L + 1, t, 0.5 * dt, 0.0);
      rec(L + 1, t + 0.5 * dt, 0.5 * dt, 0.5);
    }
  };
  rec(lmin, 0.0, dtc, 0.0);
  // sub index of level L's substep j
  auto sub_of = [&](int L, int j) -> int {
    if (L < lmin || L > lmax || j < 0 || j >= nsub[L]) return -1;
    for (size_t k = 0; k < subs.size(); ++k)
      if (subs[k].L == L && subs[k].j == j) return (int)k;
    return -1;
  };
  if (F->ev_rev.size() < subs.size()) {
    const size_t have = F->ev_rev.size();
    F->ev_rev.resize(subs.size(), nullptr);
    for (size_t k = have; k < subs.size(); ++k)
      FC_CUDA(cudaEventCreateWithFlags(&F->ev_rev[k], cudaEventDisableTiming));
  }
  const size_t store = cells * sizeof(real);
  size_t need = mode == 0 ? 2 * store : 0;  // the start state: both stores
  for (auto& u : subs) {
    u.offq = need;
    need += (size_t)(H.lev_start[u.L + 1] - H.lev_start[u.L]) * tile;
    u.offt = need;
    if (u.L > lmin) need += (size_t)(H.lev_start[u.L] - H.lev_start[u.L - 1]) * tile;
  }
  for (auto& b : F->madj)
    if (!b && dmalloc_bytes(&b, cells * sizeof(real)) != cudaSuccess)
      return fail(FC_ERR_OOM, "adjoint buffer allocation failed");
  if (!F->mio && dmalloc_bytes(&F->mio, std::max<size_t>((size_t)H.npatch() * H.desc.mx *
                                                              H.desc.mx, 1) * sizeof(real)) !=
                     cudaSuccess)
    return fail(FC_ERR_OOM, "adjoint buffer allocation failed");
  if (!F->d_ds) FC_CUDA(dmalloc(&F->d_ds, 1));
  fc_forest::Tape* tape = mode != 0 ? &F->tapes[slot] : nullptr;
  if (mode == 0 && need > F->msnap_bytes) {
    dfree(F->msnap);
    F->msnap_bytes = 0;
    if (dmalloc_bytes(&F->msnap, need) != cudaSuccess)
      return fail(FC_ERR_OOM, "adjoint state allocation failed");
    F->msnap_bytes = need;
  }
  if (mode == 1 && need > tape->bytes) {
    dfree(tape->pool);
    tape->bytes = 0;
    if (dmalloc_bytes(&tape->pool, need) != cudaSuccess)
      return fail(FC_ERR_OOM, "tape allocation failed");
    tape->bytes = need;
  }
  if (mode == 2 && need > tape->bytes)
    return fail(FC_ERR_STATE, "the tape does not hold this layout's step");
  char* pool = static_cast<char*>(mode == 0 ? F->msnap : tape->pool);
  real* LQ = static_cast<real*>(F->madj[0]);
  real* LO = static_cast<real*>(F->madj[1]);
  real* LT = static_cast<real*>(F->madj[2]);
  int cur0[kMaxLevel + 1];
  std::copy(F->cur, F->cur + kMaxLevel + 1, cur0);
  {
    const fc_status sst = ensure_streams(F);
    if (sst != FC_OK) return sst;
  }
  const bool timing = F->timing;
  F->timing = false;  // no timer events inside the adjoint's graph
  fc_status replay_st = FC_OK;
  const uint64_t launches_before = launch_counter();
  FC_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  auto body = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* dst, const void* src, size_t n) {
      if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, cs);
    };
    if (mode == 0) {
      cp(pool, F->buf[0], store);
      cp(pool + store, F->buf[1], store);
    }
    if (mode == 2) {  // the parities the recorded step saw: each held level turns over
      int c[kMaxLevel + 1];
      std::copy(F->cur, F->cur + kMaxLevel + 1, c);
      for (auto& u : subs) {
        std::copy(c, c + kMaxLevel + 1, u.cur);
        if (H.lev_start[u.L + 1] > H.lev_start[u.L]) c[u.L] ^= 1;
      }
    }
    if (mode != 2) {
      // forward replay through the forward's own level substeps (fused gather,
      // fills forked where their inputs are final), keeping what the reverse
      // reads: each update's ghost-filled input tiles and the coarse tiles
      reset_times(F);
      F->dag = true;
      F->dag_levels = F->fuse;  // each level on its own stream, as in a captured step
      F->rel_time = true;
      for (int l = 0; l <= kMaxLevel; ++l) {
        F->pre_ok[l] = F->post_ok[l] = false;
        F->lev_forked[l] = false;
      }
      if (e == cudaSuccess) e = cudaEventRecord(F->ev_start, cs);
      for (auto& u : subs) {
        std::copy(F->cur, F->cur + kMaxLevel + 1, u.cur);
        F->keep_tiles = pool + u.offq;
        F->keep_qT = u.L > lmin ? pool + u.offt : nullptr;
        if (e == cudaSuccess && replay_st == FC_OK) replay_st = advance_level(F, u.L, u.t, u.dt, cs);
      }
      for (int l = 0; l <= kMaxLevel; ++l)  // the level streams rejoin before the reverse sweep
        if (F->lev_forked[l]) {
          if (e == cudaSuccess) e = cudaEventRecord(F->ev_fill[l], F->lev_stream[l]);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, F->ev_fill[l], 0);
          F->lev_forked[l] = false;
        }
      F->dag = false;
      F->dag_levels = false;
      F->rel_time = false;
      F->keep_tiles = F->keep_qT = nullptr;
    }
    if (mode == 1) return e;  // a recorded forward step: the state advanced
    if (e == cudaSuccess) e = cudaMemsetAsync(LQ, 0, cells * sizeof(real), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(LO, 0, cells * sizeof(real), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(LT, 0, cells * sizeof(real), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(F->d_ds, 0, sizeof(double), cs);
    DevForest<real> Lv = dev<real>(F);
    Lv.buf[0] = LQ;
    Lv.buf[1] = LO;
    for (int l = 0; l <= kMaxLevel; ++l) Lv.cur[l] = 0;
    if (e == cudaSuccess)
      e = launch_unpack(Lv, F->d_api_to_dev, static_cast<const real*>(F->mio), cs);
    // Reverse sweep.  Each level's adjoint of its latest state accumulates in
    // buf[par[L]] (LQ or LO), the next older one in the other buffer.  Each
    // level runs on its own stream; the reverse of level L's substep j waits
    // for the reverses of the substeps that read what it wrote: the finer
    // level's substeps 2j + 1 and 2j + 2 (they read level L's new state), and
    // for odd j the coarser level's substep (j + 1) / 2 (its ghosts averaged
    // level L's new state).  These are the forward's waits reversed, so the
    // critical path is again the finest level's chain.
    real* bufs[2] = {LQ, LO};
    int par[kMaxLevel + 2] = {0};
    std::vector<char> done(subs.size(), 0);
    bool forked[kMaxLevel + 1] = {};
    if (e == cudaSuccess) e = cudaEventRecord(F->ev_start, cs);
    for (size_t k = subs.size(); k-- > 0 && e == cudaSuccess;) {
      const Sub& u = subs[k];
      const int p0 = H.lev_start[u.L], p1 = H.lev_start[u.L + 1];
      if (p1 <= p0) continue;
      cudaStream_t ls = F->lev_stream[u.L];
      if (!forked[u.L]) {
        e = cudaStreamWaitEvent(ls, F->ev_start, 0);
        forked[u.L] = true;
      }
      const int deps[3] = {sub_of(u.L + 1, 2 * u.j + 1), sub_of(u.L + 1, 2 * u.j + 2),
                           (u.j & 1) ? sub_of(u.L - 1, (u.j + 1) / 2) : -1};
      for (int d : deps)
        if (d >= 0 && done[d] && e == cudaSuccess) e = cudaStreamWaitEvent(ls, F->ev_rev[d], 0);
      std::copy(u.cur, u.cur + kMaxLevel + 1, F->cur);
      const int tl = u.L > lmin ? u.L - 1 : -1;
      AdjSubArgs g{};
      g.tiles = pool + u.offq;  // read where they were kept: no copies back
      g.tiles_p0 = p0;
      g.coarse = tl >= 0 ? pool + u.offt : nullptr;
      g.coarse_p0 = tl >= 0 ? H.lev_start[tl] : 0;
      g.L = u.L;
      g.p0 = p0;
      g.p1 = p1;
      g.t = u.t;
      g.dt = u.dt;
      g.t0_dev = F->d_t0;
      g.period = H.desc.vel[0];
      g.scale = F->vel_scale;
      g.dscale_factor = F->vel_scale != 0.0 ? 1.0 / F->vel_scale : 0.0;
      g.tlevel = tl;
      g.alpha = u.alpha;
      g.list_a = F->d_lists + F->off_a[u.L];
      g.na = (int)H.list_a[u.L].size();
      g.list_b = F->d_lists + F->off_b[u.L];
      g.nb = (int)H.list_b[u.L].size();
      g.list_t = F->d_lists + F->off_t[u.L];
      g.nt = (int)H.list_t[u.L].size();
      AdjAcc<real> c{};
      c.lam_in = bufs[par[u.L]];
      c.lam_out = bufs[par[u.L] ^ 1];
      c.lam_fine = bufs[par[u.L + 1]];
      c.lam_new = tl >= 0 ? bufs[par[tl]] : nullptr;
      c.lam_old = tl >= 0 ? bufs[par[tl] ^ 1] : nullptr;
      c.lamT = LT;
      if (e == cudaSuccess) e = launch_adjoint_substep(dev<real>(F), g, c, F->d_ds, ls);
      if (e == cudaSuccess) e = cudaEventRecord(F->ev_rev[k], ls);
      done[k] = 1;
      par[u.L] ^= 1;
    }
    for (int l = 0; l <= kMaxLevel && e == cudaSuccess; ++l)  // rejoin before the result is read
      if (forked[l]) {
        e = cudaEventRecord(F->ev_fill[l], F->lev_stream[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, F->ev_fill[l], 0);
      }
    // each level's adjoint of the step's start state is in buf[par[l]]
    for (int l = 0; l <= kMaxLevel; ++l) Lv.cur[l] = par[l];
    if (e == cudaSuccess) e = launch_pack(Lv, F->d_api_to_dev, static_cast<real*>(F->mio), 0, cs);
    if (mode == 0) {
      cp(F->buf[0], pool, store);
      cp(F->buf[1], pool + store, store);
    }
    return e;
  };
  const cudaError_t eb = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
  out->kernels = launch_counter() - launches_before;  // counted when replayed
  launch_counter() = launches_before;
  std::copy(F->cur, F->cur + kMaxLevel + 1, out->cur_after);
  std::copy(cur0, cur0 + kMaxLevel + 1, F->cur);
  F->timing = timing;
  reset_times(F);
  if (replay_st != FC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return replay_st;
  }
  if (eb != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(eb != cudaSuccess ? eb : ee, "adjoint capture");
  }
  const cudaError_t ei = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate");
  out->dt = dtc;
  out->mode = mode;
  out->slot = slot;
  std::copy(cur0, cur0 + kMaxLevel + 1, out->cur);
  return FC_OK;
}

template <typename real>
static fc_status adjoint_multirate_t(fc_forest* F, double t0, double dtc, void* lam,
                                     double* dscale, cudaStream_t s) {
  AllocStream alloc_on(s);  // buffers first allocated here are ordered before the replay on s
  fc_forest::AdjGraph* g = nullptr;
  for (auto& c : F->adj_graphs)
    if (c.mode == 0 && c.dt == dtc && std::equal(c.cur, c.cur + kMaxLevel + 1, F->cur)) g = &c;
  if (!g) {
    if (!F->cap_stream)
      FC_CUDA(cudaStreamCreateWithFlags(&F->cap_stream, cudaStreamNonBlocking));
    fc_forest::AdjGraph ng;
    fc_status st = capture_adjoint_multirate<real>(F, dtc, F->cap_stream, &ng, 0, -1);
    if (st != FC_OK) return st;
    F->adj_graphs.push_back(ng);
    g = &F->adj_graphs.back();
  }
  const size_t nbytes = (size_t)F->host.npatch() * F->host.desc.mx * F->host.desc.mx * sizeof(real);
  FC_CUDA(cudaMemcpyAsync(F->mio, lam, nbytes, cudaMemcpyDeviceToDevice, s));
  FC_CUDA(launch_set_time(F->d_t0, t0, s));
  FC_CUDA(cudaGraphLaunch(g->exec, s));
  launch_counter() += g->kernels;
  FC_CUDA(cudaMemcpyAsync(lam, F->mio, nbytes, cudaMemcpyDeviceToDevice, s));
  FC_CUDA(launch_add_double(dscale, F->d_ds, s));
  reset_times(F);  // the state is the step's start state again
  return FC_OK;
}

// the graph of `mode` (1: record, 2: reverse) for tape `slot` at this step
// length and buffer parity, captured on first use
template <typename real>
static fc_status tape_graph(fc_forest* F, double dtc, int mode, int slot,
                            fc_forest::AdjGraph** out) {
  fc_forest::AdjGraph* g = nullptr;
  for (auto& c : F->adj_graphs)
    if (c.mode == mode && c.slot == slot && c.dt == dtc &&
        std::equal(c.cur, c.cur + kMaxLevel + 1, F->cur))
      g = &c;
  if (!g) {
    if (!F->cap_stream)
      FC_CUDA(cudaStreamCreateWithFlags(&F->cap_stream, cudaStreamNonBlocking));
    fc_forest::AdjGraph ng;
    const fc_status st = capture_adjoint_multirate<real>(F, dtc, F->cap_stream, &ng, mode, slot);
    if (st != FC_OK) return st;
    F->adj_graphs.push_back(ng);
    g = &F->adj_graphs.back();
  }
  *out = g;
  return FC_OK;
}

// a coarse multirate step that also keeps, in tape `slot`, what the reverse
// of the step reads
template <typename real>
static fc_status record_multirate_t(fc_forest* F, double t0, double dtc, int slot,
                                    cudaStream_t s) {
  AllocStream alloc_on(s);  // the tape's memory is ordered before the step on s
  if ((int)F->tapes.size() <= slot) F->tapes.resize(slot + 1);
  fc_forest::Tape& tp = F->tapes[slot];
  tp.valid = false;
  fc_forest::AdjGraph* g = nullptr;
  const fc_status st = tape_graph<real>(F, dtc, 1, slot, &g);
  if (st != FC_OK) return st;
  std::copy(F->cur, F->cur + kMaxLevel + 1, tp.cur0);
  FC_CUDA(launch_set_time(F->d_t0, t0, s));
  FC_CUDA(cudaGraphLaunch(g->exec, s));
  launch_counter() += g->kernels;
  std::copy(g->cur_after, g->cur_after + kMaxLevel + 1, F->cur);
  const int lmin = F->host.desc.lmin, lmax = F->host.desc.lmax;
  for (int L = lmin; L <= lmax; ++L) {  // as a coarse step leaves them
    const double dtl = std::ldexp(dtc, -(L - lmin));
    F->has_old[L] = true;
    F->dt_last[L] = dtl;
    F->t_start[L] = t0 + dtc - dtl;
  }
  tp.valid = true;
  tp.dt = dtc;
  return FC_OK;
}

// the adjoint of the step recorded in tape `slot` (its reverse alone)
template <typename real>
static fc_status adjoint_taped_t(fc_forest* F, double t0, double dtc, int slot, void* lam,
                                 double* dscale, cudaStream_t s) {
  AllocStream alloc_on(s);
  if (slot >= (int)F->tapes.size() || !F->tapes[slot].valid || F->tapes[slot].dt != dtc)
    return fail(FC_ERR_STATE,
                "no step of this length recorded in the slot since the layout or the "
                "captured steps last changed");
  int cur_now[kMaxLevel + 1];
  std::copy(F->cur, F->cur + kMaxLevel + 1, cur_now);
  std::copy(F->tapes[slot].cur0, F->tapes[slot].cur0 + kMaxLevel + 1, F->cur);
  fc_forest::AdjGraph* g = nullptr;
  const fc_status st = tape_graph<real>(F, dtc, 2, slot, &g);
  std::copy(cur_now, cur_now + kMaxLevel + 1, F->cur);
  if (st != FC_OK) return st;
  const size_t nbytes = (size_t)F->host.npatch() * F->host.desc.mx * F->host.desc.mx * sizeof(real);
  FC_CUDA(cudaMemcpyAsync(F->mio, lam, nbytes, cudaMemcpyDeviceToDevice, s));
  FC_CUDA(launch_set_time(F->d_t0, t0, s));
  FC_CUDA(cudaGraphLaunch(g->exec, s));
  launch_counter() += g->kernels;
  FC_CUDA(cudaMemcpyAsync(lam, F->mio, nbytes, cudaMemcpyDeviceToDevice, s));
  FC_CUDA(launch_add_double(dscale, F->d_ds, s));
  return FC_OK;
}

// Adjoint of one level substep (fc_adjoint_advance): the forward fill of the
// substep is redone (separate kernels: ghost rings in the store, the coarse
// neighbours' time-interpolated tiles in qT), then the substep's transposes
// run on four accumulators in tile layout: the current states' adjoint (the
// level's entries read and cleared, the finer level's and the coarser
// level's newer-state shares added), the level's state before the substep,
// the older states' adjoint and the qT tiles' adjoint.
template <typename real>
static fc_status adjoint_advance_t(fc_forest* F, int L, double t, double dt, void* lam,
                                   void* lam_old, double* dscale, cudaStream_t s) {
  AllocStream alloc_on(s);
  const HostForest& H = F->host;
  const size_t S = (size_t)H.desc.mx + 2 * kMbc;
  const size_t cells = std::max<size_t>((size_t)H.npatch() * S * S, 1);
  int tlevel = -1;
  double alpha = 0.0;
  if (L > H.desc.lmin && F->has_old[L - 1] && F->dt_last[L - 1] > 0.0) {
    tlevel = L - 1;
    alpha = (t - F->t_start[L - 1]) / F->dt_last[L - 1];
    alpha = std::min(1.0, std::max(0.0, alpha));
  }
  if (tlevel >= 0 && !lam_old)
    return fail(FC_ERR_INVALID_ARG,
                "fc_adjoint_advance: level-1 is time-interpolated; lam_old is needed");
  for (auto& b : F->madj)
    if (!b && dmalloc_bytes(&b, cells * sizeof(real)) != cudaSuccess)
      return fail(FC_ERR_OOM, "adjoint buffer allocation failed");
  if (!F->lam[0] && dmalloc_bytes(&F->lam[0], cells * sizeof(real)) != cudaSuccess)
    return fail(FC_ERR_OOM, "adjoint buffer allocation failed");
  real* LQ = static_cast<real*>(F->madj[0]);
  real* LB = static_cast<real*>(F->madj[1]);
  real* LT = static_cast<real*>(F->madj[2]);
  real* LO = static_cast<real*>(F->lam[0]);
  DevForest<real> D = dev<real>(F);
  const int p0 = H.lev_start[L], p1 = H.lev_start[L + 1];
  // the substep's forward fill, as fc_advance_level does it with separate fills
  FillArgs A{F->d_lists + F->off_a[L], (int)H.list_a[L].size(), tlevel, alpha, 1};
  FillArgs B{F->d_lists + F->off_b[L], (int)H.list_b[L].size(), tlevel, alpha};
  if (p1 > p0) {
    FC_CUDA(launch_fill_coarse(D, A, s));
    FC_CUDA(launch_fill_fine(D, B, s));
  }
  for (real* b : {LQ, LB, LT, LO}) FC_CUDA(cudaMemsetAsync(b, 0, cells * sizeof(real), s));
  DevForest<real> Lv = dev<real>(F);
  for (int l = 0; l <= kMaxLevel; ++l) Lv.cur[l] = 0;
  Lv.buf[0] = Lv.buf[1] = LQ;
  FC_CUDA(launch_unpack(Lv, F->d_api_to_dev, static_cast<const real*>(lam), s));
  if (lam_old) {
    Lv.buf[0] = Lv.buf[1] = LO;
    FC_CUDA(launch_unpack(Lv, F->d_api_to_dev, static_cast<const real*>(lam_old), s));
  }
  if (p1 > p0) {
    AdjSubArgs g{};
    g.L = L;
    g.p0 = p0;
    g.p1 = p1;
    g.t = t;
    g.dt = dt;
    g.t0_dev = nullptr;
    g.period = H.desc.vel[0];
    g.scale = F->vel_scale;
    g.dscale_factor = F->vel_scale != 0.0 ? 1.0 / F->vel_scale : 0.0;
    g.tlevel = tlevel;
    g.alpha = alpha;
    g.list_a = F->d_lists + F->off_a[L];
    g.na = (int)H.list_a[L].size();
    g.list_b = F->d_lists + F->off_b[L];
    g.nb = (int)H.list_b[L].size();
    g.list_t = F->d_lists + F->off_t[L];
    g.nt = (int)H.list_t[L].size();
    AdjAcc<real> c{};
    c.lam_in = LQ;     // level L's entries: the new state's adjoint, read then cleared
    c.lam_out = LB;    // level L before the substep
    c.lam_fine = LQ;   // level L + 1, read at its current state
    c.lam_new = LQ;    // level L - 1, the newer state of the interpolation
    c.lam_old = LO;    // level L - 1, the older state
    c.lamT = LT;
    Timed tm(F, 3, s, 0.0);
    FC_CUDA(launch_adjoint_substep(D, g, c, dscale, s));
  }
  FC_CUDA(launch_add_store(LQ, LB, cells, s));
  Lv.buf[0] = Lv.buf[1] = LQ;
  FC_CUDA(launch_pack(Lv, F->d_api_to_dev, static_cast<real*>(lam), 0, s));
  if (lam_old) {
    Lv.buf[0] = Lv.buf[1] = LO;
    FC_CUDA(launch_pack(Lv, F->d_api_to_dev, static_cast<real*>(lam_old), 0, s));
  }
  return FC_OK;
}

extern "C" {

fc_status fc_adjoint_advance(fc_forest* F, int level, double t, double dt, void* lam,
                             void* lam_old, double* dscale, void* stream) {
  if (!F || !lam || !dscale) return fail(FC_ERR_INVALID_ARG, "null argument");
  if (F->host.partial) return fail(FC_ERR_STATE, "the adjoint is built for whole forests");
  if (level < F->host.desc.lmin || level > F->host.desc.lmax)
    return fail(FC_ERR_INVALID_ARG, "level outside [lmin, lmax]");
  if (!(dt > 0.0)) return fail(FC_ERR_INVALID_ARG, "dt must be positive");
  if (F->host.desc.domain == FC_DOMAIN_SPHERE)
    return fail(FC_ERR_INVALID_ARG, "the adjoint is built for the square domains");
  if (F->host.desc.reflux)
    return fail(FC_ERR_PRECONDITION, "the adjoint is built without refluxing");
  cudaStream_t s = as_stream(stream);
  return F->esize == 4 ? adjoint_advance_t<float>(F, level, t, dt, lam, lam_old, dscale, s)
                       : adjoint_advance_t<double>(F, level, t, dt, lam, lam_old, dscale, s);
}

fc_status fc_adjoint_step_multirate(fc_forest* F, double t, double dt_coarse, void* lam,
                                    double* dscale, void* stream) {
  if (!F || !lam || !dscale) return fail(FC_ERR_INVALID_ARG, "null argument");
  if (F->host.partial) return fail(FC_ERR_STATE, "the adjoint is built for whole forests");
  if (!(dt_coarse > 0.0)) return fail(FC_ERR_INVALID_ARG, "dt must be positive");
  if (F->host.desc.domain == FC_DOMAIN_SPHERE)
    return fail(FC_ERR_INVALID_ARG, "the adjoint is built for the square domains");
  if (F->host.desc.reflux)
    return fail(FC_ERR_PRECONDITION, "the adjoint is built without refluxing");
  cudaStream_t s = as_stream(stream);
  fc_status st = F->esize == 4 ? adjoint_multirate_t<float>(F, t, dt_coarse, lam, dscale, s)
                               : adjoint_multirate_t<double>(F, t, dt_coarse, lam, dscale, s);
  if (st != FC_OK) return st;
  return check_device_error(F, s);
}

// the checks the multirate adjoint's entry points share
static fc_status adjoint_preconditions(const fc_forest* F, double dt) {
  if (F->host.partial) return fail(FC_ERR_STATE, "the adjoint is built for whole forests");
  if (!(dt > 0.0)) return fail(FC_ERR_INVALID_ARG, "dt must be positive");
  if (F->host.desc.domain == FC_DOMAIN_SPHERE)
    return fail(FC_ERR_INVALID_ARG, "the adjoint is built for the square domains");
  if (F->host.desc.reflux)
    return fail(FC_ERR_PRECONDITION, "the adjoint is built without refluxing");
  return FC_OK;
}

fc_status fc_step_multirate_record(fc_forest* F, double t, double dt_coarse, int slot,
                                   void* stream) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  if (slot < 0 || slot >= FC_MAX_TAPE_SLOTS)
    return fail(FC_ERR_INVALID_ARG, "tape slot out of range");
  const fc_status pre = adjoint_preconditions(F, dt_coarse);
  if (pre != FC_OK) return pre;
  cudaStream_t s = as_stream(stream);
  return F->esize == 4 ? record_multirate_t<float>(F, t, dt_coarse, slot, s)
                       : record_multirate_t<double>(F, t, dt_coarse, slot, s);
}

fc_status fc_adjoint_step_multirate_taped(fc_forest* F, double t, double dt_coarse, int slot,
                                          void* lam, double* dscale, void* stream) {
  if (!F || !lam || !dscale) return fail(FC_ERR_INVALID_ARG, "null argument");
  if (slot < 0 || slot >= FC_MAX_TAPE_SLOTS)
    return fail(FC_ERR_INVALID_ARG, "tape slot out of range");
  const fc_status pre = adjoint_preconditions(F, dt_coarse);
  if (pre != FC_OK) return pre;
  cudaStream_t s = as_stream(stream);
  const fc_status st =
      F->esize == 4 ? adjoint_taped_t<float>(F, t, dt_coarse, slot, lam, dscale, s)
                    : adjoint_taped_t<double>(F, t, dt_coarse, slot, lam, dscale, s);
  if (st != FC_OK) return st;
  return check_device_error(F, s);
}

fc_status fc_tape_release(fc_forest* F) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  for (auto it = F->adj_graphs.begin(); it != F->adj_graphs.end();)
    if (it->mode != 0) {
      if (it->exec) cudaGraphExecDestroy(it->exec);
      it = F->adj_graphs.erase(it);
    } else {
      ++it;
    }
  for (auto& t : F->tapes) dfree(t.pool);
  F->tapes.clear();
  return FC_OK;
}

fc_status fc_adjoint_step_global(fc_forest* F, double t, double dt, void* lam, double* dscale,
                                 void* stream) {
  if (!F || !lam || !dscale) return fail(FC_ERR_INVALID_ARG, "null argument");
  if (F->host.partial) return fail(FC_ERR_STATE, "the adjoint is built for whole forests");
  if (!(dt > 0.0)) return fail(FC_ERR_INVALID_ARG, "dt must be positive");
  if (F->host.desc.domain == FC_DOMAIN_SPHERE)
    return fail(FC_ERR_INVALID_ARG, "the adjoint is built for the square domains");
  if (F->host.desc.reflux)
    return fail(FC_ERR_PRECONDITION, "the adjoint is built without refluxing");
  cudaStream_t s = as_stream(stream);
  return F->esize == 4 ? adjoint_step_t<float>(F, t, dt, lam, dscale, s)
                       : adjoint_step_t<double>(F, t, dt, lam, dscale, s);
}

fc_status fc_set_fused_fill(fc_forest* F, int enable) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  F->fuse = enable != 0;
  destroy_graphs(F);
  return FC_OK;
}

fc_status fc_set_graphs(fc_forest* F, int enable) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  F->use_graphs = enable != 0;
  if (!F->use_graphs) destroy_graphs(F);
  return FC_OK;
}

fc_status fc_forest_num_leaves(const fc_forest* F, int* n) {
  if (!F || !n) return fail(FC_ERR_INVALID_ARG, "null argument");
  *n = F->host.napi();
  return FC_OK;
}

fc_status fc_forest_leaves(const fc_forest* F, int* out) {
  if (!F || !out) return fail(FC_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < F->host.napi(); ++k) {
    const Leaf& a = F->host.leaves[k];
    out[5 * k] = a.f;
    out[5 * k + 1] = a.b;
    out[5 * k + 2] = a.l;
    out[5 * k + 3] = a.x;
    out[5 * k + 4] = a.y;
  }
  return FC_OK;
}

fc_status fc_forest_set_q(fc_forest* F, const void* q, int on_device, void* stream) {
  if (!F || !q) return fail(FC_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = as_stream(stream);
  const size_t bytes = (size_t)F->host.napi() * F->host.desc.mx * F->host.desc.mx * F->esize;
  const void* src = q;
  if (!on_device) {
    FC_CUDA(cudaMemcpyAsync(F->stage, q, bytes, cudaMemcpyHostToDevice, s));
    src = F->stage;
  }
  cudaError_t e = F->esize == 4
                      ? launch_unpack(dev<float>(F), F->d_api_to_dev, (const float*)src, s)
                      : launch_unpack(dev<double>(F), F->d_api_to_dev, (const double*)src, s);
  if (e != cudaSuccess) return cuda_fail(e, "unpack");
  if (!on_device) FC_CUDA(cudaStreamSynchronize(s));
  reset_times(F);
  return FC_OK;
}

static fc_status get_q_impl(const fc_forest* F, void* q, int on_device, void* stream, int full) {
  if (!F || !q) return fail(FC_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = as_stream(stream);
  const size_t per = full ? (size_t)(F->host.desc.mx + 4) * (F->host.desc.mx + 4)
                          : (size_t)F->host.desc.mx * F->host.desc.mx;
  const size_t bytes = (size_t)F->host.napi() * per * F->esize;
  void* dst = on_device ? q : F->stage;
  cudaError_t e = F->esize == 4
                      ? launch_pack(dev<float>(F), F->d_api_to_dev, (float*)dst, full, s)
                      : launch_pack(dev<double>(F), F->d_api_to_dev, (double*)dst, full, s);
  if (e != cudaSuccess) return cuda_fail(e, "pack");
  if (!on_device) {
    FC_CUDA(cudaMemcpyAsync(q, F->stage, bytes, cudaMemcpyDeviceToHost, s));
    FC_CUDA(cudaStreamSynchronize(s));
    return check_device_error(const_cast<fc_forest*>(F), s);
  }
  return FC_OK;
}

fc_status fc_forest_get_q(const fc_forest* F, void* q, int on_device, void* stream) {
  return get_q_impl(F, q, on_device, stream, 0);
}

fc_status fc_forest_poison(fc_forest* F, double value, void* stream) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  cudaStream_t s = as_stream(stream);
  const cudaError_t e = F->esize == 4 ? launch_poison(dev<float>(F), value, s)
                                      : launch_poison(dev<double>(F), value, s);
  return e == cudaSuccess ? FC_OK : cuda_fail(e, "poison");
}

fc_status fc_forest_get_q_full(const fc_forest* F, void* q, int on_device, void* stream) {
  return get_q_impl(F, q, on_device, stream, 1);
}

fc_status fc_fill_ghosts(fc_forest* F, void* stream) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  return fill_all(F, as_stream(stream));
}

fc_status fc_advance_level(fc_forest* F, int level, double t, double dt, void* stream) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  if (level < F->host.desc.lmin || level > F->host.desc.lmax)
    return fail(FC_ERR_INVALID_ARG, "level outside [lmin, lmax]");
  if (!(dt > 0.0)) return fail(FC_ERR_INVALID_ARG, "dt must be positive");
  return advance_level(F, level, t, dt, as_stream(stream));
}

fc_status fc_step_global(fc_forest* F, double t, double dt, void* stream) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  if (!(dt > 0.0)) return fail(FC_ERR_INVALID_ARG, "dt must be positive");
  cudaStream_t s = as_stream(stream);
  fc_status st = fill_all(F, s);
  if (st != FC_OK) return st;
  const HostForest& H = F->host;
  // one launch per level (per-level h and dt/h); all read the pre-step state
  DevForest<float> Df = dev<float>(F);
  DevForest<double> Dd = dev<double>(F);
  for (int L = H.desc.lmin; L <= H.desc.lmax; ++L) {
    const int p0 = H.lev_start[L], p1 = H.upd_end(L);  // (a partition: its owned patches)
    if (p1 <= p0) continue;
    const AdvArgs a = adv_args(F, L, t, dt, p1 - p0);
    if ((st = deform_fluxes(F, p0, p1, a, s)) != FC_OK) return st;
    Timed tm(F, 0, s, advance_bytes(F, p1 - p0));
    cudaError_t e = F->esize == 4 ? launch_advance(Df, p0, p1, a, F->d_err, s)
                                  : launch_advance(Dd, p0, p1, a, F->d_err, s);
    if (e != cudaSuccess) return cuda_fail(e, "advance");
  }
  for (int l = 0; l <= kMaxLevel; ++l) F->cur[l] ^= 1;
  // refluxing: every level took one step of dt, one fine step per face
  for (int L = H.desc.lmin; L <= H.desc.lmax && F->bflux; ++L) {
    F->bslot[L] = 0;
    if ((st = reflux_level(F, L, dt, 1, 0.5, s)) != FC_OK) return st;
  }
  reset_times(F);
  return FC_OK;
}

fc_status fc_step_multirate(fc_forest* F, double t, double dt_coarse, void* stream) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  if (F->host.partial)
    return fail(FC_ERR_STATE, "a partitioned forest steps level by level (fc_advance_level), "
                              "with a halo exchange after each substep");
  if (!(dt_coarse > 0.0)) return fail(FC_ERR_INVALID_ARG, "dt must be positive");
  cudaStream_t s = as_stream(stream);
  const int lmin = F->host.desc.lmin, lmax = F->host.desc.lmax;
  if (!F->use_graphs) return multirate(F, lmin, t, dt_coarse, s);
  // A coarse step is replayed from a CUDA graph captured for this layout, dt
  // and starting buffer parity; the step's start time is written to device
  // memory first (one single-thread kernel), the captured kernels read it.
  fc_forest::Graph* g = nullptr;
  for (auto& c : F->graphs)
    if (c.dt == dt_coarse && c.timing == F->timing &&
        std::equal(c.cur_before, c.cur_before + kMaxLevel + 1, F->cur))
      g = &c;
  if (!g) {
    if (!F->cap_stream)
      FC_CUDA(cudaStreamCreateWithFlags(&F->cap_stream, cudaStreamNonBlocking));
    fc_forest::Graph ng;
    ng.dt = dt_coarse;
    ng.timing = F->timing;
    std::copy(F->cur, F->cur + kMaxLevel + 1, ng.cur_before);
    // capture with relative times; the host bookkeeping done while capturing
    // is what one replay does to the state
    {
      const fc_status sst = ensure_streams(F);
      if (sst != FC_OK) return sst;
    }
    F->capture_pairs = &ng.pairs;
    F->dag = true;
    // with the per-launch timers on, the levels run one after another on one
    // stream, so each timed launch has the GPU to itself (its event pair
    // measures that kernel, not the levels sharing the SMs with it)
    F->dag_levels = F->fuse && !F->timing;
    for (int l = 0; l <= kMaxLevel; ++l) {
      F->pre_ok[l] = F->post_ok[l] = false;
      F->lev_forked[l] = false;
    }
    const uint64_t launches_before = launch_counter();
    FC_CUDA(cudaStreamBeginCapture(F->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t ej = cudaEventRecord(F->ev_start, F->cap_stream);
    fc_status st = ej == cudaSuccess ? multirate(F, lmin, 0.0, dt_coarse, F->cap_stream)
                                     : cuda_fail(ej, "cudaEventRecord");
    // join every level stream back into the step's stream
    for (int l = 0; l <= kMaxLevel && st == FC_OK; ++l)
      if (F->lev_forked[l]) {
        ej = cudaEventRecord(F->ev_fill[l], F->lev_stream[l]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(F->cap_stream, F->ev_fill[l], 0);
        if (ej != cudaSuccess) st = cuda_fail(ej, "level join");
      }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(F->cap_stream, &graph);
    F->capture_pairs = nullptr;
    F->dag = false;
    F->dag_levels = false;
    for (int l = 0; l <= kMaxLevel; ++l) F->lev_forked[l] = false;
    ng.kernels = launch_counter() - launches_before;  // counted when replayed
    launch_counter() = launches_before;
    std::copy(F->cur, F->cur + kMaxLevel + 1, ng.cur_after);
    std::copy(ng.cur_before, ng.cur_before + kMaxLevel + 1, F->cur);
    if (st != FC_OK) {
      if (graph) cudaGraphDestroy(graph);
      for (auto& p : ng.pairs) F->spare.push_back(p);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    if (!ng.timing)  // same shape as a stale step: update its parameters in place
      while (!ng.exec && !F->stale.empty()) {
        cudaGraphExec_t x = F->stale.back();
        F->stale.pop_back();
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(x, graph, &info) == cudaSuccess) {
          ng.exec = x;
        } else {
          cudaGetLastError();  // clear the failed update's status
          cudaGraphExecDestroy(x);
        }
      }
    if (!ng.exec) e = cudaGraphInstantiate(&ng.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    F->graphs.push_back(std::move(ng));
    g = &F->graphs.back();
  }
  FC_CUDA(account_graph(F, *g));  // its pairs are about to be re-recorded
  FC_CUDA(launch_set_time(F->d_t0, t, s));
  FC_CUDA(cudaGraphLaunch(g->exec, s));
  launch_counter() += g->kernels;
  g->replayed = F->timing;
  std::copy(g->cur_after, g->cur_after + kMaxLevel + 1, F->cur);
  // per-level step bookkeeping after the replay (as the recursion leaves it)
  for (int L = lmin; L <= lmax; ++L) {
    const double dtl = std::ldexp(dt_coarse, -(L - lmin));
    F->has_old[L] = true;
    F->dt_last[L] = dtl;
    F->t_start[L] = t + dt_coarse - dtl;
  }
  return FC_OK;
}

fc_status fc_tag(fc_forest* F, double* delta_host, void* stream) {
  if (!F || !delta_host) return fail(FC_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = as_stream(stream);
  const int kind = F->host.desc.indicator;
  {  // Alg. 1 first: central differences read the first ghost layer, and a
     // regrid's new children interpolate from their parent's cells with its
     // ghosts (the update kernels keep ghosts in shared memory only)
    const fc_status st = fill_all(F, s);
    if (st != FC_OK) return st;
  }
  const int n = F->host.npatch();
  cudaError_t e;
  {
    Timed tm(F, 2, s, (double)n * F->host.desc.mx * F->host.desc.mx * F->esize);
    e = F->esize == 4 ? launch_tag(dev<float>(F), kind, F->d_delta, s)
                      : launch_tag(dev<double>(F), kind, F->d_delta, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "tag");
  std::vector<double> dd(n);
  FC_CUDA(cudaMemcpyAsync(dd.data(), F->d_delta, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  FC_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < F->host.napi(); ++k) delta_host[k] = dd[F->host.dev_of[k]];
  return FC_OK;
}

fc_status fc_tag_regrid(fc_forest* F, double tau_refine, double tau_coarsen,
                        const int* lmax_per_forest, int* changed, void* stream) {
  if (!F) return fail(FC_ERR_INVALID_ARG, "null forest");
  if (F->host.partial)
    return fail(FC_ERR_STATE, "a partitioned forest keeps its layout (no regrid)");
  cudaStream_t s = as_stream(stream);
  host_pool_arm();  // the host workers wake while the tag waits on the device
  const int n = F->host.npatch();
  std::vector<double> delta(n);
  fc_status st = fc_tag(F, delta.data(), stream);
  if (st != FC_OK) return st;
  std::vector<int> lmax_f;
  if (lmax_per_forest) lmax_f.assign(lmax_per_forest, lmax_per_forest + F->host.desc.nforests);
  std::vector<Leaf> nl;
  std::string err = regrid_layout(F->host, delta, tau_refine, tau_coarsen, lmax_f, &nl);
  if (!err.empty()) return fail(FC_ERR_STATE, err);
  // unchanged layout?
  bool same = (int)nl.size() == n;
  for (int k = 0; same && k < n; ++k) {
    const Leaf& a = nl[k];
    const Leaf& b = F->host.leaves[k];
    same = a.f == b.f && a.b == b.b && a.l == b.l && a.x == b.x && a.y == b.y;
  }
  if (same) {
    if (changed) *changed = 0;
    return FC_OK;
  }
  AllocStream alloc_on(s);  // the new layout's memory and the old one's release, ordered on s
  fc_forest* G = new (std::nothrow) fc_forest();
  if (!G) return fail(FC_ERR_OOM, "host allocation failed");
  G->host.desc = F->host.desc;
  G->esize = F->esize;
  G->vel_scale = F->vel_scale;  // the sphere's metrics carry it
  G->host.leaves = nl;
  // the new layout's build carries over the rows of the old one that it
  // keeps (the old tables are read, not reused; the memory of the tables
  // before them is)
  G->host.nbr.swap(F->spare_nbr);
  G->host.meta.swap(F->spare_meta);
  // the forest's error word and step-time word carry over to the new layout
  // (G borrows them until it takes F's place)
  G->d_err = F->d_err;
  G->d_t0 = F->d_t0;
  const auto abandon = [&](fc_status why) {  // G's own memory goes, F stays as it was
    G->d_err = nullptr;
    G->d_t0 = nullptr;
    free_device(G);
    delete G;
    return why;
  };
  err = G->host.build(&F->host);
  if (!err.empty())
    return abandon(fail(FC_ERR_STATE, "regrid produced an invalid layout: " + err));
  st = upload(G, true, false);
  if (st != FC_OK) return abandon(st);
  // remap list in G's device order
  const HostForest& O = F->host;
  const HostForest& N = G->host;
  std::vector<RemapEntry> rm(N.npatch());
  // each entry reads the two layouts' tables only: host threads take ranges
  // of large layouts (below some thousands of patches one thread measured
  // faster: the tables would have to move between cores)
  std::vector<char> orphan(16, 0);
  parallel_chunks(N.npatch(), 8192, [&](int pb, int pe, int tid) {
    for (int p = pb; p < pe; ++p) {
      const Leaf& a = N.leaves[N.api_of[p]];
      RemapEntry e{RM_COPY, {-1, -1, -1, -1}, 0, 0};
      int o = O.find(a.f, a.b, a.l, a.x, a.y);
      if (o >= 0) {
        e.src[0] = O.dev_of[o];
      } else {
        int par = a.l > 0 ? O.find(a.f, a.b, a.l - 1, a.x >> 1, a.y >> 1) : -1;
        if (par >= 0) {
          e.kind = RM_INTERP;
          e.src[0] = O.dev_of[par];
          e.cx = a.x & 1;
          e.cy = a.y & 1;
        } else {
          e.kind = RM_AVERAGE;
          for (int c = 0; c < 4; ++c) {
            int ch = O.find(a.f, a.b, a.l + 1, 2 * a.x + (c & 1), 2 * a.y + (c >> 1));
            if (ch < 0) {
              orphan[tid] = 1;
              break;
            }
            e.src[c] = O.dev_of[ch];
          }
        }
      }
      rm[p] = e;
    }
  });
  for (char o : orphan)
    if (o) return abandon(fail(FC_ERR_STATE, "regrid: new leaf has neither an old parent nor children"));
  int kept = 0;
  for (const RemapEntry& e : rm) kept += e.kind == RM_COPY;
  const int created = N.npatch() - kept;
  dfree(G->d_remap);
  if (dmalloc(&G->d_remap, rm.size()) != cudaSuccess)
    return abandon(fail(FC_ERR_OOM, "remap list allocation failed"));
  cudaError_t e = cudaMemcpyAsync(G->d_remap, rm.data(), sizeof(RemapEntry) * rm.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return abandon(cuda_fail(e, "remap list copy"));
  if (F->d_metric) {  // the new layout's metrics: kept patches copy theirs
    st = update_metrics(G, G->d_remap, F->d_metric);
    if (st != FC_OK) return abandon(st);
  }
  {
    Timed tm(F, 2, s, 2.0 * (double)N.npatch() * N.desc.mx * N.desc.mx * F->esize);
    e = F->esize == 4 ? launch_remap(dev<float>(F), dev<float>(G), G->d_remap, s)
                      : launch_remap(dev<double>(F), dev<double>(G), G->d_remap, s);
  }
  if (e != cudaSuccess) return abandon(cuda_fail(e, "remap"));
  // swap contents: F takes G's layout and store; captured steps are stale
  retire_graphs(F);
  F->d_err = nullptr;  // (G holds them)
  F->d_t0 = nullptr;
  free_device(F);
  F->spare_nbr.swap(F->host.nbr);  // the next regrid's build writes here
  F->spare_meta.swap(F->host.meta);
  F->host = std::move(G->host);
  F->store = G->store;
  std::memcpy(F->buf, G->buf, sizeof F->buf);
  F->qT = G->qT;
  F->stage = G->stage;
  F->bflux = G->bflux;
  F->d_tables = G->d_tables;
  F->d_meta = G->d_meta;
  F->d_nbr = G->d_nbr;
  F->d_lists = G->d_lists;
  F->off_all = G->off_all;
  F->off_coarse_all = G->off_coarse_all;
  std::memcpy(F->off_a, G->off_a, sizeof F->off_a);
  std::memcpy(F->off_b, G->off_b, sizeof F->off_b);
  std::memcpy(F->off_t, G->off_t, sizeof F->off_t);
  F->d_api_to_dev = G->d_api_to_dev;
  F->d_fstart = G->d_fstart;
  F->d_patch_sums = G->d_patch_sums;
  F->d_mass = G->d_mass;
  F->d_delta = G->d_delta;
  F->d_remap = G->d_remap;
  F->d_err = G->d_err;
  F->d_t0 = G->d_t0;
  F->d_metric = G->d_metric;
  F->d_corner = G->d_corner;
  F->d_pairs = G->d_pairs;
  std::memcpy(F->pair_level, G->pair_level, sizeof F->pair_level);
  for (int l = 0; l <= kMaxLevel; ++l) F->cur[l] = 0;
  reset_times(F);
  delete G;  // its device pointers now belong to F
  if (changed) *changed = created + (n - kept);
  FC_CUDA(cudaStreamSynchronize(s));  // the new layout is ready for any stream
  return FC_OK;
}

static fc_status host_layout(const fc_forest_desc* desc, int nleaves, const int* leaves,
                             HostForest* H) {
  fc_status st = check_desc(desc);
  if (st != FC_OK) return st;
  if (nleaves < 1 || !leaves) return fail(FC_ERR_INVALID_ARG, "empty leaf list");
  H->desc = *desc;
  H->leaves.resize(nleaves);
  for (int k = 0; k < nleaves; ++k)
    H->leaves[k] = Leaf{leaves[5 * k], leaves[5 * k + 1], leaves[5 * k + 2], leaves[5 * k + 3],
                        leaves[5 * k + 4]};
  std::string err = H->build();
  if (!err.empty()) return fail(FC_ERR_PRECONDITION, err);
  return FC_OK;
}

fc_status fc_layout_check(const fc_forest_desc* desc, int nleaves, const int* leaves) {
  HostForest H;
  return host_layout(desc, nleaves, leaves, &H);
}

fc_status fc_layout_neighbours(const fc_forest_desc* desc, int nleaves, const int* leaves,
                               int* out) {
  if (!out) return fail(FC_ERR_INVALID_ARG, "null output");
  HostForest H;
  fc_status st = host_layout(desc, nleaves, leaves, &H);
  if (st != FC_OK) return st;
  for (int k = 0; k < nleaves; ++k) {
    const int p = H.dev_of[k];
    for (int d = 0; d < 8; ++d) {
      const NbrEntry& e = H.nbr[(size_t)p * 8 + d];
      int* o = out + ((size_t)k * 8 + d) * 6;
      o[0] = e.kind;
      o[1] = e.n0 >= 0 ? H.api_of[e.n0] : -1;
      o[2] = e.n1 >= 0 ? H.api_of[e.n1] : -1;
      o[3] = e.a;
      o[4] = e.fx;
      o[5] = e.fy;
    }
  }
  return FC_OK;
}

fc_status fc_layout_reflux(const fc_forest_desc* desc, int nleaves, const int* leaves, int* out) {
  if (!out) return fail(FC_ERR_INVALID_ARG, "null output");
  HostForest H;
  fc_status st = host_layout(desc, nleaves, leaves, &H);
  if (st != FC_OK) return st;
  const std::string err = H.reflux_pairs(out);
  return err.empty() ? FC_OK : fail(FC_ERR_STATE, err);
}

// field index of each of the caller's leaves (H built from them)
static std::vector<int> caller_to_field(const HostForest& H, int nleaves, const int* leaves) {
  std::vector<int> k_of(nleaves);
  for (int i = 0; i < nleaves; ++i)
    k_of[i] = H.find(leaves[5 * i], leaves[5 * i + 1], leaves[5 * i + 2], leaves[5 * i + 3],
                     leaves[5 * i + 4]);
  return k_of;
}

// the caller's per-leaf ranks in field order, checked
static fc_status part_in_field_order(const HostForest& H, int nleaves, const int* leaves,
                                     const int* part, std::vector<int>* out, int* nranks) {
  const std::vector<int> k_of = caller_to_field(H, nleaves, leaves);
  out->assign(nleaves, -1);
  *nranks = 0;
  for (int i = 0; i < nleaves; ++i) {
    if (part[i] < 0) return fail(FC_ERR_INVALID_ARG, "partition: negative rank");
    (*out)[k_of[i]] = part[i];
    *nranks = std::max(*nranks, part[i] + 1);
  }
  return FC_OK;
}

fc_status fc_layout_partition(const fc_forest_desc* desc, int nleaves, const int* leaves,
                              int nranks, int* part_out) {
  if (!part_out || nranks < 1) return fail(FC_ERR_INVALID_ARG, "bad output or rank count");
  HostForest H;
  fc_status st = host_layout(desc, nleaves, leaves, &H);
  if (st != FC_OK) return st;
  const std::vector<int> part = partition_ranges(H, nranks);
  const std::vector<int> k_of = caller_to_field(H, nleaves, leaves);
  for (int i = 0; i < nleaves; ++i) part_out[i] = part[k_of[i]];
  return FC_OK;
}

fc_status fc_layout_halo(const fc_forest_desc* desc, int nleaves, const int* leaves,
                         const int* part, int rank, int* nmirror, int* mirror_out) {
  if (!part || !nmirror || !mirror_out) return fail(FC_ERR_INVALID_ARG, "null argument");
  HostForest H;
  fc_status st = host_layout(desc, nleaves, leaves, &H);
  if (st != FC_OK) return st;
  std::vector<int> pf;
  int nranks = 0;
  if ((st = part_in_field_order(H, nleaves, leaves, part, &pf, &nranks)) != FC_OK) return st;
  if (rank < 0 || rank >= nranks) return fail(FC_ERR_INVALID_ARG, "rank outside the partition");
  const std::vector<int> m = partition_mirrors(H, pf, rank);
  // field index -> the caller's index
  const std::vector<int> k_of = caller_to_field(H, nleaves, leaves);
  std::vector<int> caller_of(nleaves);
  for (int i = 0; i < nleaves; ++i) caller_of[k_of[i]] = i;
  *nmirror = (int)m.size();
  for (size_t j = 0; j < m.size(); ++j) mirror_out[j] = caller_of[m[j]];
  return FC_OK;
}

fc_status fc_forest_create_part(const fc_forest_desc* desc, int nleaves, const int* leaves,
                                const int* part, int rank, fc_forest** out) {
  if (!out || !part) return fail(FC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (desc && desc->reflux)
    return fail(FC_ERR_INVALID_ARG, "a partitioned forest is built without refluxing");
  HostForest G;
  fc_status st = host_layout(desc, nleaves, leaves, &G);
  if (st != FC_OK) return st;
  std::vector<int> pf;
  int nranks = 0;
  if ((st = part_in_field_order(G, nleaves, leaves, part, &pf, &nranks)) != FC_OK) return st;
  fc_forest* F = new (std::nothrow) fc_forest();
  if (!F) return fail(FC_ERR_OOM, "host allocation failed");
  F->esize = desc->dtype == FC_F32 ? 4 : 8;
  const std::string err = build_partition(G, pf, rank, &F->host);
  if (!err.empty()) {
    delete F;
    return fail(FC_ERR_INVALID_ARG, err);
  }
  keep_pool_memory();
  const HostForest& H = F->host;
  st = upload(F, true);
  // the exchange lists, one block: per (level or all, rank) the send list,
  // then the receive list
  std::vector<int> lists;
  F->halo_off.assign((size_t)(kMaxLevel + 2) * nranks * 2 + 1, 0);
  for (int l = 0; l <= kMaxLevel + 1; ++l)
    for (int r = 0; r < nranks; ++r)
      for (int dir = 0; dir < 2; ++dir) {
        F->halo_off[((size_t)l * nranks + r) * 2 + dir] = lists.size();
        for (int lv = (l <= kMaxLevel ? l : 0); lv <= (l <= kMaxLevel ? l : kMaxLevel); ++lv) {
          const std::vector<int>& v = dir == 0 ? H.send[lv][r] : H.recv[lv][r];
          lists.insert(lists.end(), v.begin(), v.end());
        }
      }
  F->halo_off.back() = lists.size();
  if (st == FC_OK && dmalloc(&F->d_halo, lists.size()) != cudaSuccess)
    st = fail(FC_ERR_OOM, "exchange list allocation failed");
  if (st == FC_OK && !lists.empty() &&
      cudaMemcpyAsync(F->d_halo, lists.data(), sizeof(int) * lists.size(),
                      cudaMemcpyHostToDevice, g_alloc_stream) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "exchange lists");
  if (st == FC_OK && cudaStreamSynchronize(0) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "create");
  if (st != FC_OK) {
    free_device(F);
    cudaStreamSynchronize(0);
    delete F;
    return st;
  }
  *out = F;
  g_live_forests.fetch_add(1);
  return FC_OK;
}

// one exchange list of a partition: (device pointer, count)
static fc_status halo_list(const fc_forest* F, int peer, int level, int dir, const int** p,
                           int* n) {
  const HostForest& H = F->host;
  if (!H.partial) return fail(FC_ERR_STATE, "not a partitioned forest");
  if (peer < 0 || peer >= H.nranks || peer == H.rank)
    return fail(FC_ERR_INVALID_ARG, "peer must be another rank of the partition");
  if (level != -1 && (level < 0 || level > kMaxLevel))
    return fail(FC_ERR_INVALID_ARG, "level must be -1 (all) or a level");
  const int l = level < 0 ? kMaxLevel + 1 : level;
  const size_t at = ((size_t)l * H.nranks + peer) * 2 + dir;
  *p = F->d_halo + F->halo_off[at];
  *n = (int)(F->halo_off[at + 1] - F->halo_off[at]);
  return FC_OK;
}

fc_status fc_halo_count(const fc_forest* F, int peer, int level, int* nsend, int* nrecv) {
  if (!F || !nsend || !nrecv) return fail(FC_ERR_INVALID_ARG, "null argument");
  const int* p;
  fc_status st = halo_list(F, peer, level, 0, &p, nsend);
  if (st == FC_OK) st = halo_list(F, peer, level, 1, &p, nrecv);
  return st;
}

static fc_status halo_move(const fc_forest* F, int peer, int level, void* buf, int pack,
                           void* stream) {
  if (!F || !buf) return fail(FC_ERR_INVALID_ARG, "null argument");
  const int* list;
  int n = 0;
  fc_status st = halo_list(F, peer, level, pack ? 0 : 1, &list, &n);
  if (st != FC_OK) return st;
  cudaStream_t s = as_stream(stream);
  const cudaError_t e =
      F->esize == 4 ? launch_halo(dev<float>(F), list, n, static_cast<float*>(buf), pack, s)
                    : launch_halo(dev<double>(F), list, n, static_cast<double*>(buf), pack, s);
  return e == cudaSuccess ? FC_OK : cuda_fail(e, "halo exchange");
}

fc_status fc_halo_pack(const fc_forest* F, int peer, int level, void* dst, void* stream) {
  return halo_move(F, peer, level, dst, 1, stream);
}

fc_status fc_halo_unpack(fc_forest* F, int peer, int level, const void* src, void* stream) {
  return halo_move(F, peer, level, const_cast<void*>(src), 0, stream);
}

fc_status fc_layout_regrid(const fc_forest_desc* desc, int nleaves, const int* leaves,
                           const double* delta, double tau_refine, double tau_coarsen,
                           const int* lmax_per_forest, int cap, int* out_leaves, int* nout) {
  if (!delta || !out_leaves || !nout) return fail(FC_ERR_INVALID_ARG, "null argument");
  HostForest H;
  fc_status st = host_layout(desc, nleaves, leaves, &H);
  if (st != FC_OK) return st;
  // delta arrives in the caller's leaf order; H sorted its leaves
  std::vector<double> d(nleaves);
  for (int k = 0; k < nleaves; ++k) {
    const int* a = leaves + 5 * k;
    d[H.find(a[0], a[1], a[2], a[3], a[4])] = delta[k];
  }
  std::vector<int> lmax_f;
  if (lmax_per_forest) lmax_f.assign(lmax_per_forest, lmax_per_forest + desc->nforests);
  std::vector<Leaf> nl;
  std::string err = regrid_layout(H, d, tau_refine, tau_coarsen, lmax_f, &nl);
  if (!err.empty()) return fail(FC_ERR_STATE, err);
  *nout = (int)nl.size();
  if ((int)nl.size() > cap) return fail(FC_ERR_INVALID_ARG, "output capacity too small");
  for (size_t k = 0; k < nl.size(); ++k) {
    int* o = out_leaves + 5 * k;
    o[0] = nl[k].f;
    o[1] = nl[k].b;
    o[2] = nl[k].l;
    o[3] = nl[k].x;
    o[4] = nl[k].y;
  }
  return FC_OK;
}

fc_status fc_forest_mass(const fc_forest* F, double* out, void* stream) {
  if (!F || !out) return fail(FC_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = as_stream(stream);
  const int nf = F->host.desc.nforests;
  cudaError_t e =
      F->esize == 4
          ? launch_mass(dev<float>(F), F->d_api_to_dev, F->d_fstart, nf, F->d_patch_sums,
                        F->d_mass, s)
          : launch_mass(dev<double>(F), F->d_api_to_dev, F->d_fstart, nf, F->d_patch_sums,
                        F->d_mass, s);
  if (e != cudaSuccess) return cuda_fail(e, "mass");
  FC_CUDA(cudaMemcpyAsync(out, F->d_mass, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
  FC_CUDA(cudaStreamSynchronize(s));
  return check_device_error(const_cast<fc_forest*>(F), s);
}

}  // extern "C"
