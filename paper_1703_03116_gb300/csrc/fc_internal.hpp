// Internal declarations shared by the host forest, the scheduler and the
// CUDA kernels.  Nothing here crosses the C ABI (include/fc.h).
#pragma once

#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <unordered_map>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "fc.h"

namespace fc {

constexpr int kMaxLevel = 20;
constexpr int kMbc = 2;  // ghost layers built into the kernels

// Neighbour relation of one face or corner region of a patch (Sec. 2.2):
// same-size neighbour (copy), finer neighbour(s) (average), coarser neighbour
// (interpolate), outside the physical domain (boundary condition), or the
// corner region beyond a cube vertex of the cubed sphere, where only three
// blocks meet and no block holds the diagonal cells (Sec. 2.4).
// NB_ABSENT marks, in one rank's part of a partitioned layout, a region of a
// mirror patch whose neighbour that rank does not hold: no kernel reads it.
enum NbrKind : int {
  NB_EXTERIOR = 0,
  NB_SAME = 1,
  NB_FINE = 2,
  NB_COARSE = 3,
  NB_CORNER3 = 4,
  NB_ABSENT = 5
};

// Region order: faces -x, +x, -y, +y, then corners (-,-), (+,-), (-,+), (+,+).
constexpr int kDirX[8] = {-1, 1, 0, 0, -1, 1, -1, 1};
constexpr int kDirY[8] = {0, 0, -1, 1, -1, -1, 1, 1};

// Index transform of Eq. (transform): I' = A I + F maps the owner's level-l
// global cell index I into the neighbour block's level-l global index I'.
// A is a signed permutation: bit 0 swaps the axes, bits 1 and 2 negate the
// first and second output component.
inline void apply_code_host(int a, int x, int y, int* u, int* v) {
  *u = (a & 1) ? y : x;
  *v = (a & 1) ? x : y;
  if (a & 2) *u = -*u;
  if (a & 4) *v = -*v;
}

struct NbrEntry {
  int kind;
  int n0, n1;  // device patch indices; n1 only for a face with two fine patches
  int a;       // orientation code of A
  int fx, fy;  // F
  // the neighbours' level and quadrant coordinates, copied here so a
  // kernel gathering ghosts reads one table instead of two dependent ones
  int lev, x0, y0, x1, y1, pad;
  // A coarser neighbour c (NB_COARSE): where the coarse-neighbour fill
  // takes the ghosts of c that the interpolation of this region reads, so a
  // kernel computing them needs no read of c's entries (written on the
  // device after each upload, launch_coarse_sources; -1 and 0 on the host).
  // The ghosts of c next to the owner are averages of the owner's own cells;
  // up to two others, each (src[k], code[k]): code bits 0-5 and 6-11 the ghost's
  // indices in c plus one, 12-17 and 18-23 the source cell (the first of a
  // 2 x 2 block) in patch src[k], 24-25 the rule (1 copy, 2 average of the
  // block, 3 keep the time-interpolated tile's value); bit 28 of code[0]:
  // every ghost of c read is the owner's or one of these two (else, or when
  // code[0] is 0, the kernel reads c's entries).
  int src[2], code[2];
};
constexpr int kSrcComplete = 1 << 28;

// Allocator whose construct without arguments leaves trivially constructible
// elements uninitialised: host tables that are written in full (by host
// threads, which then also take the first-touch page faults in parallel)
// skip a serial zero fill.
template <class T>
struct UninitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};

// Host worker threads for the layout builds (leaf maps, neighbour rows,
// remap lists).  host_pool_run(n, chunks, fn) runs fn(begin, end, slot) over
// [0, n) split into `chunks` contiguous pieces, each taken by whichever
// thread claims it first; slot (0 the caller, 1..15 a worker) names the
// thread, which may run several pieces.  The caller claims pieces too, so a
// call completes even if no worker joins (a worker that has claimed a piece
// finishes it; nothing waits on a worker that has not).  host_pool_arm()
// wakes a few workers ahead of parallel work: they poll for pieces for about
// a millisecond before they sleep again (a regrid arms them before its tag
// waits on the device, so they are awake when its tables are built).  One
// call at a time per process: a concurrent call runs on its caller alone.
// In a child process forked after the workers started, every call runs on
// the caller.
void host_pool_arm();
void host_pool_run(int n, int chunks, const std::function<void(int, int, int)>& fn);

// Run fn(begin, end, slot) over [0, n) on host threads in pieces of at least
// min_per_piece items (on the calling thread alone when n is small).
template <class Fn>
inline void parallel_chunks(int n, int min_per_piece, Fn fn) {
  const int pieces = n / std::max(1, min_per_piece);
  if (pieces <= 1) {
    fn(0, n, 0);
    return;
  }
  host_pool_run(n, std::min(pieces, 64), std::function<void(int, int, int)>(fn));
}

struct PatchMeta {
  int level, x, y, block, forest, flags;  // flags bit 0: has a coarser neighbour
};

struct Leaf {
  int f, b, l, x, y;
};

// forest (16 bits), block (8), level (5), x (17), y (18): levels up to 16
// (x, y < 2^16) and up to 256 blocks
inline uint64_t leaf_key(int f, int b, int l, int x, int y) {
  return ((uint64_t)(uint32_t)f << 48) | ((uint64_t)(uint32_t)b << 40) |
         ((uint64_t)(uint32_t)l << 35) | ((uint64_t)(uint32_t)x << 18) | (uint64_t)(uint32_t)y;
}
inline Leaf leaf_of_key(uint64_t k) {
  return Leaf{(int)(k >> 48), (int)((k >> 40) & 0xFF), (int)((k >> 35) & 31),
              (int)((k >> 18) & 0x1FFFF), (int)(k & 0x3FFFF)};
}

// blocks of one forest: 6 cube faces, a brick's unit blocks, or one square
inline int num_blocks(const fc_forest_desc& d) {
  return d.domain == FC_DOMAIN_SPHERE ? 6
         : d.domain == FC_DOMAIN_BRICK ? d.brick_nx * d.brick_ny
                                       : 1;
}

// Leaf key -> int map with open addressing and linear probing (host tables
// of up to millions of leaves; no allocation per entry).  Keys with the top
// 16 bits all set never occur (forest < 65535) and mark empty / erased slots.
// The probe of a key starts inside a window of slots that belongs to its
// forest (the forest index picks the window, a hash of the key the slot in
// it), so the lookups around one forest's leaves stay within a few
// cache-resident kilobytes; probing itself runs on over the whole table.
class KeyMap {
 public:
  // n_expected keys from nforests consecutive forests
  void clear(size_t n_expected = 0, size_t nforests = 1) {
    size_t cap = 16;
    while (cap < 2 * n_expected + 2) cap <<= 1;
    slots_.assign(cap, Slot{kEmpty, 0});
    forests_ = nforests < 1 ? 1 : nforests;
    win_ = cap;
    while (win_ > 16 && win_ * forests_ > cap) win_ >>= 1;
    used_ = live_ = 0;
  }
  // false if the key is present already
  bool insert(uint64_t k, int v) {
    if (slots_.empty() || 2 * (used_ + 1) > slots_.size()) grow();
    const size_t mask = slots_.size() - 1;
    size_t i = start(k), tomb = SIZE_MAX;
    for (;; i = (i + 1) & mask) {
      if (slots_[i].k == k) return false;
      if (slots_[i].k == kErased && tomb == SIZE_MAX) tomb = i;
      if (slots_[i].k == kEmpty) break;
    }
    if (tomb != SIZE_MAX) {
      i = tomb;
    } else {
      ++used_;
    }
    slots_[i] = Slot{k, v};
    ++live_;
    return true;
  }
  // Insert from several threads at once into a map just cleared for at
  // least as many keys (no growth, no erased slots); false if the key is
  // present.  The map is read only after the threads have joined, and the
  // count is then set by set_size.
  bool insert_concurrent(uint64_t k, int v) {
    const size_t mask = slots_.size() - 1;
    for (size_t i = start(k);; i = (i + 1) & mask) {
      uint64_t seen = kEmpty;
      if (__atomic_compare_exchange_n(&slots_[i].k, &seen, k, false, __ATOMIC_RELAXED,
                                      __ATOMIC_RELAXED)) {
        slots_[i].v = v;
        return true;
      }
      if (seen == k) return false;
    }
  }
  void set_size(size_t n) { used_ = live_ = n; }
  int find(uint64_t k) const {  // -1 if absent
    if (slots_.empty()) return -1;
    const size_t mask = slots_.size() - 1;
    for (size_t i = start(k);; i = (i + 1) & mask) {
      if (slots_[i].k == k) return slots_[i].v;
      if (slots_[i].k == kEmpty) return -1;
    }
  }
  bool erase(uint64_t k) {
    if (slots_.empty()) return false;
    const size_t mask = slots_.size() - 1;
    for (size_t i = start(k);; i = (i + 1) & mask) {
      if (slots_[i].k == k) {
        slots_[i].k = kErased;
        --live_;
        return true;
      }
      if (slots_[i].k == kEmpty) return false;
    }
  }
  size_t size() const { return live_; }
  template <class Fn>
  void for_each(Fn fn) const {
    for (const Slot& e : slots_)
      if (e.k != kEmpty && e.k != kErased) fn(e.k, e.v);
  }

 private:
  struct Slot {
    uint64_t k;
    int v;
  };
  static constexpr uint64_t kEmpty = ~0ull, kErased = ~0ull - 1;
  static uint64_t mix(uint64_t k) {  // a 64-bit finaliser (xor-shift-multiply)
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
  }
  size_t start(uint64_t k) const {
    return ((k >> 48) * win_ + (mix(k) & (win_ - 1))) & (slots_.size() - 1);
  }
  void grow() {
    std::vector<Slot> old;
    old.swap(slots_);
    clear(live_ + 16, forests_);
    for (const Slot& e : old)
      if (e.k != kEmpty && e.k != kErased) insert(e.k, e.v);
  }
  std::vector<Slot> slots_;
  size_t forests_ = 1, win_ = 16;
  size_t used_ = 0, live_ = 0;
};

// Remap entry for regridding (Sec. 3.1).
enum RemapKind : int { RM_COPY = 0, RM_INTERP = 1, RM_AVERAGE = 2 };
struct RemapEntry {
  int kind;
  int src[4];  // old device patches: COPY/INTERP use src[0]; AVERAGE uses 4 children
  int cx, cy;  // INTERP: position of the new child inside the old parent
};

// Host-side forest: leaves, lookup, neighbour tables, level work lists.
struct HostForest {
  fc_forest_desc desc{};
  std::vector<Leaf> leaves;              // field order (forest, block, Morton)
  KeyMap idx;                            // key -> index in `leaves`
  std::vector<int> dev_of;               // leaves index -> device patch index
  std::vector<int> api_of;               // device patch index -> leaves index
  std::vector<PatchMeta, UninitAlloc<PatchMeta>> meta;  // device order
  std::vector<NbrEntry, UninitAlloc<NbrEntry>> nbr;     // device order, 8 per patch
  int lev_start[kMaxLevel + 2] = {0};    // device patches of level l: [lev_start[l], lev_start[l+1])
  std::vector<int> list_all, list_coarse_all;
  // multirate substep of level l: list_t = coarse neighbours (level l-1) of
  // level-l patches, filled through the time-interpolation buffer; list_a =
  // list_t plus the level-l patches; list_b = level-l patches with a coarser
  // neighbour
  std::vector<int> list_a[kMaxLevel + 1], list_b[kMaxLevel + 1], list_t[kMaxLevel + 1];
  std::vector<int> forest_start;         // leaves of forest f: [forest_start[f], forest_start[f+1])
  std::vector<char> feeds_finer;         // device order: coarser neighbour of a patch one level finer

  // One rank's part of a partitioned layout (Sec. 3, partitioning): `leaves`
  // holds the owned leaves (field order) followed by the mirrors -- leaves of
  // other ranks whose interiors the owned leaves' ghost fills read -- and the
  // device order puts each level's owned patches first: level l's owned
  // patches are [lev_start[l], own_end[l]).  The field layout of get/set
  // covers the owned leaves only.
  bool partial = false;
  int nowned = 0;
  int own_end[kMaxLevel + 1] = {0};
  // halo exchange with each other rank, per level: local device indices of
  // the owned patches that rank mirrors (send) and of this rank's mirrors
  // that rank owns (recv), both in the global field order
  std::vector<std::vector<int>> send[kMaxLevel + 1], recv[kMaxLevel + 1];
  int nranks = 1, rank = 0;
  // leaves in the field layout of get/set (all, or the owned ones)
  int napi() const { return partial ? nowned : (int)leaves.size(); }
  // end of level l's patches that an update advances
  int upd_end(int l) const { return partial ? own_end[l] : lev_start[l + 1]; }

  // Build everything from `leaves`; returns an empty string or an error.
  // prev (optional): the layout this one replaces (a regrid), built and
  // unchanged since; the rows of leaves it held whose neighbours it held too
  // are its rows with the patch indices renumbered (the same rows a full
  // build computes: a row depends only on the leaves it names).
  std::string build(const HostForest* prev = nullptr);
  // rows of `nbr` and `meta` for the leaves [kb, ke) (field order); marks
  // feeds_finer
  std::string neighbour_rows(int kb, int ke);
  std::string work_lists();
  // Refluxing's pairing, from the neighbour table and its index transforms:
  // per leaf (field order), face (-x, +x, -y, +y) and face cell k, 5 ints
  // (kind, leaf across (field index), its face on the shared edge, j0, j1):
  // kind 1 finer across (j0, j1: its cells beside the lower and upper half
  // of cell k along this leaf's face), 2 same level across a cube edge with
  // this leaf on the block of higher index (j0: its cell), 0 none (-1
  // elsewhere).  Returns an empty string or an error.
  std::string reflux_pairs(int* out) const;
  // dense leaf lookup (when `dense`): owner[own_off[f] + (b << 2 lo) +
  // (Y << lo) + X] is the leaf covering cell (X, Y) of block b at level
  // lo = own_lo[f], forest f's finest occupied level
  bool dense = false;
  std::vector<int, UninitAlloc<int>> owner;
  std::vector<size_t> own_off;
  std::vector<int> own_lo;
  // the leaf (b, l, x, y) of forest f, or -1 (in-range f, b expected)
  int find(int f, int b, int l, int x, int y) const {
    if (dense) {
      const int lo = own_lo[f];
      if (l > lo || l < 0 || x < 0 || y < 0 || x >= (1 << l) || y >= (1 << l)) return -1;
      const int s = lo - l;
      const int k = owner[own_off[f] + ((size_t)b << (2 * lo)) + ((size_t)(y << s) << lo) +
                          (x << s)];
      return leaves[k].l == l ? k : -1;
    }
    return idx.find(leaf_key(f, b, l, x, y));
  }
  // the leaf covering quadrant (b, l, x, y) of forest f if it is at level l
  // or l - 1, else -1 (the quadrant is subdivided, or lies in a leaf two or
  // more levels coarser); quadrant in range and l <= own_lo[f] expected
  int holder(int f, int b, int l, int x, int y) const {
    if (dense) {
      const int lo = own_lo[f], s = lo - l;
      const int k = owner[own_off[f] + ((size_t)b << (2 * lo)) + ((size_t)(y << s) << lo) +
                          (x << s)];
      const int lk = leaves[k].l;
      return lk == l || lk == l - 1 ? k : -1;
    }
    const int k = idx.find(leaf_key(f, b, l, x, y));
    return k >= 0 || l == 0 ? k : idx.find(leaf_key(f, b, l - 1, x >> 1, y >> 1));
  }
  int npatch() const { return (int)leaves.size(); }
};

// The mirrors of `rank` in a built layout G under the partition `part` (per
// leaf of G, field order): the leaves of other ranks whose interiors the
// ghost fills of rank's leaves read -- their face and corner neighbours and,
// for a coarser neighbour, its same-size and finer neighbours (whose copies
// and averages the interpolation reads, Prop. 1) -- as field indices of G in
// field order.
std::vector<int> partition_mirrors(const HostForest& G, const std::vector<int>& part, int rank);
// Contiguous ranges of G's field order weighted by level work (2^(l - lmin)
// updates per coarse step), one per rank: part[k] for each leaf of G.
std::vector<int> partition_ranges(const HostForest& G, int nranks);
// rank's part of G (H: empty): its owned leaves and mirrors, the neighbour
// rows of G restricted to them, the work lists restricted to what the owned
// leaves' updates and fills need, and the exchange lists with every rank.
std::string build_partition(const HostForest& G, const std::vector<int>& part, int rank,
                            HostForest* H);

// Regrid: new leaf list and remap list (in the new field order).
std::string regrid_layout(const HostForest& F, const std::vector<double>& delta, double tau_r,
                          double tau_c, const std::vector<int>& lmax_f,
                          std::vector<Leaf>* out_leaves);
void sort_leaves(std::vector<Leaf>* v);

// ---------------------------------------------------------------- device side

// Cubed-sphere metric block of one patch, FP64 over the extended index range
// (cells -2..mx+1): capacity kappa[S*S] (spherical cell area), then the
// volume flux of the velocity field through every x-edge, phix[S*(S+1)]
// (edge i-1/2 of row j at j*(S+1) + i, shifted by 2), then through every
// y-edge, phiy[(S+1)*S] (edge j-1/2 of column i at j*S + i, shifted by 2).
__host__ __device__ constexpr int metric_stride(int S) { return S * S + 2 * S * (S + 1); }

// Cubed sphere (FC_DOMAIN_SPHERE): block b is the face of the cube [-1,1]^3
// with outward normal n; its block coordinates (x, y) in [0,1]^2 sit at
// n + (2x - 1) ex + (2y - 1) ey.  Axes are signed codes: +-1, +-2, +-3 for
// +-X, +-Y, +-Z.  (The block numbering is part of the C ABI.)
__host__ __device__ inline void cube_face(int b, int* n, int* ex, int* ey) {
  switch (b) {
    case 0: *n = 3; *ex = 1; *ey = 2; break;     // +Z
    case 1: *n = -3; *ex = 1; *ey = -2; break;   // -Z
    case 2: *n = 1; *ex = 2; *ey = 3; break;     // +X
    case 3: *n = -1; *ex = -2; *ey = 3; break;   // -X
    case 4: *n = 2; *ex = -1; *ey = 3; break;    // +Y
    default: *n = -2; *ex = 1; *ey = 3; break;   // -Y
  }
}

template <typename real>
struct DevForest {
  int mx, S, npatch, domain;
  int napi;  // leaves in the field layout (get/set, mass): npatch, or the owned ones
  const double* metric;  // cubed sphere: metric_stride(S) doubles per patch; else null
  const PatchMeta* meta;
  const NbrEntry* nbr;
  real* buf[2];
  real* qT;
  int cur[kMaxLevel + 1];
  int vel_kind;
  double vel[4];
  int order, limiter, transverse;
};

struct FillArgs {
  const int* targets;
  int ntargets;
  int tlevel;    // level read/written through the time-interpolated buffer, -1 none
  double alpha;  // time-interpolation weight of the newer state
  // targets on tlevel: 0 time-interpolates only the interior cells within
  // two of the patch's edge (all that a finer neighbour's interpolation
  // stencil, or its transpose, reads: the coarse cell beside the shared
  // edge and its neighbours), 1 the whole interior
  int full_interior;
};

// Per-launch scalars of the patch update for one level: cell width h,
// Courant ratio dt/h, and the swirl coefficient cos(pi t / T) * sfac with
// sfac = sin(pi h) / (pi h) (0 for a constant velocity).  The velocity time t
// is t_half, or *t0_dev + t_off when t0_dev is set (graph replay: the coarse
// step's start time lives in device memory, the offset is baked in).
struct AdvArgs {
  double h, nu, sfac, period, t_half, t_off;
  double dt;  // time step (capacity form: dt / kappa per cell)
  const double* t0_dev;
  int variant;  // AdvVariant
  int warps;    // walk and band variants: warps per CTA
  int ctas;     // walk variant: cap on the CTAs in the grid (0: the SMs' residency)
  // polls of a kernel's bounded wait for its tile copy before it gives up
  // (FC_ERR_TIMEOUT); the copies in flight are then still awaited with the
  // default limit before the CTA leaves
  uint32_t wait_limit;
  // gather != 0: the kernel fills each patch's ghost ring itself (Alg. 1 in
  // shared memory) before the update; coarser neighbours on `tlevel` are
  // read through the time-interpolation buffer
  int gather, tlevel;
  double alpha;
  // set: each patch's ghost-filled input tile is also written to
  // keep + (p - keep_p0) tiles (the adjoint's replay of the forward)
  void* keep;
  int keep_p0;
  // direct != 0 (staged update, gather on): coarse neighbours on tlevel are
  // not read from a filled time-interpolated tile; the update computes the
  // cells its interpolation reads as that fill would (no fill launch before
  // it on the critical path)
  int direct;
  // direct with keep_t set (the adjoint's replay): the coarse cells the
  // interpolation computes are also stored in the kept time-interpolated
  // tiles, keep_t + (patch - keep_t_p0) tiles, as the fill would leave them
  void* keep_t;
  int keep_t_p0;
  // refluxing: each patch's final fluxes through its faces go to
  // bflux + ((p * 2 + bslot) * 4 + face) * mx (faces -x, +x, -y, +y; null: off)
  void* bflux;
  int bslot;
};

// Patch-update kernel variants (chosen per level launch by the autotuner):
// staged -- one CTA per patch, every thread on every phase (low latency);
// walk   -- lanes own patch columns and walk the rows, one warp per patch
//           (fewest instructions per cell; the throughput choice), tiles
//           double-buffered per warp;
// walk1  -- the walk with one tile buffer per warp (twice the warps per SM);
// band   -- one CTA per patch whose warps each walk a band of rows as the
//           walk does (low latency at few instructions per cell).
enum AdvVariant : int { ADV_STAGED = 0, ADV_WALK = 1, ADV_WALK1 = 2, ADV_BAND = 3 };

template <typename real>
cudaError_t launch_advance_walk(const DevForest<real>& D, int p0, int p1, const AdvArgs& a,
                                int* err, cudaStream_t s);
template <typename real>
cudaError_t launch_advance_band(const DevForest<real>& D, int p0, int p1, const AdvArgs& a,
                                int* err, cudaStream_t s);

cudaError_t launch_set_time(double* t0_dev, double t0, cudaStream_t s);
// *dst += *src (one thread; device doubles)
cudaError_t launch_add_double(double* dst, const double* src, cudaStream_t s);

// Adjoint of one global step (t -> t + dt): per-level update transposes, then
// the transpose of Alg. 1 (interpolation, boundary condition, copy/average).
struct AdjArgs {
  double t, dt, period, scale, dscale_factor;  // dscale += factor * sum_e dL/ds_e s_e
  const int* lev_start;                        // host, device-order level ranges
  const int* coarse_list;                      // device: patches with a coarser neighbour
  int ncoarse;
};
template <typename real>
cudaError_t launch_adjoint_step(const DevForest<real>& D, const AdjArgs& g, const real* lam_in,
                                real* lam_out, double* dscale, cudaStream_t s);

// Adjoint of one multirate substep of level L over (t, t + dt), on the
// forward state before it (ghosts of the substep's fill in place, qT
// filled), adding into the accumulators of AdjAcc.  tlevel = L - 1 with
// weight alpha, or -1 on the coarsest level.
struct AdjSubArgs {
  int L, p0, p1;  // level and its device range
  double t, dt, period, scale, dscale_factor;
  const double* t0_dev;  // set: t is relative to the time stored there (graph replay)
  int tlevel;
  double alpha;
  const int* list_a;  // device: list_t then level L's patches (the substep's fill targets)
  int na;
  const int* list_b;  // device: level-L patches with a coarser neighbour
  int nb;
  const int* list_t;  // device: level L-1 patches read through qT
  int nt;
  // the forward's kept tiles: level L's ghost-filled tiles (patch p at
  // tiles + (p - tiles_p0) tiles) and the time-interpolated coarse tiles
  // (coarse + (c - coarse_p0) tiles); null: read the store and qT
  const void* tiles;
  int tiles_p0;
  const void* coarse;
  int coarse_p0;
};
// The adjoint's accumulators for one substep of level L (patch-store tile
// layout): each level's adjoint of one state lives in one of two buffers and
// receives every contribution by atomic adds, starting from zero.
template <typename real>
struct AdjAcc {
  real* lam_in;    // level L, the state after the substep: read, then cleared
  real* lam_out;   // level L, the state before it
  real* lam_fine;  // level L+1, its state at the substep's start
  real* lam_old;   // level L-1, the older and newer states of the time
  real* lam_new;   //   interpolation
  real* lamT;      // the qT tiles' adjoint (zero on entry and on return)
};
template <typename real>
cudaError_t launch_adjoint_substep(const DevForest<real>& D, const AdjSubArgs& g,
                                   const AdjAcc<real>& c, double* dscale, cudaStream_t s);

// device error word bits
constexpr int kErrTimeout = 1;
// polls of a bounded device wait before it gives up (default)
constexpr uint32_t kWaitLimit = 1u << 22;

template <typename real>
cudaError_t launch_fill_coarse(const DevForest<real>& D, const FillArgs& A, cudaStream_t s);
template <typename real>
cudaError_t launch_fill_fine(const DevForest<real>& D, const FillArgs& A, cudaStream_t s);
template <typename real>
cudaError_t launch_advance(const DevForest<real>& D, int p0, int p1, const AdvArgs& a, int* err,
                           cudaStream_t s);
template <typename real>
cudaError_t launch_tag(const DevForest<real>& D, int kind, double* delta, cudaStream_t s);
// refluxing of the level-L patches p0..p1 (all on one level, cell width h,
// their latest update of length dt wrote flux slot cslot; the finer
// neighbours' fluxes of nfs slots are averaged with weight w)
template <typename real>
cudaError_t launch_reflux(const DevForest<real>& D, int p0, int p1, const real* bflux, int cslot,
                          int nfs, double w, double nu, cudaStream_t s);
// refluxing on the cubed sphere from the host pairing (pairs: per device
// patch, face and face cell 5 ints: kind, patch across, its face, j0, j1)
template <typename real>
cudaError_t launch_reflux_pairs(const DevForest<real>& D, int p0, int p1, const real* bflux,
                                const int* pairs, int cslot, int nfs, double w, double dt,
                                cudaStream_t s);
template <typename real>
cudaError_t launch_mass(const DevForest<real>& D, const int* api_to_dev, const int* fstart,
                        int nforests, double* patch_sums, double* out, cudaStream_t s);
template <typename real>
cudaError_t launch_pack(const DevForest<real>& D, const int* api_to_dev, real* out, int full,
                        cudaStream_t s);
template <typename real>
cudaError_t launch_unpack(const DevForest<real>& D, const int* api_to_dev, const real* in,
                          cudaStream_t s);
template <typename real>
cudaError_t launch_remap(const DevForest<real>& Old, const DevForest<real>& New,
                         const RemapEntry* rm, cudaStream_t s);
template <typename real>
cudaError_t launch_poison(const DevForest<real>& D, double value, cudaStream_t s);

uint64_t& launch_counter();

// The coarse neighbours' ghost sources (NbrEntry::src, code) of a layout's
// neighbour table in device memory (n patches, mx, walls: the square
// domain with walls), in place.
cudaError_t launch_coarse_sources(NbrEntry* nbr, const PatchMeta* meta, int n, int mx, int walls,
                                  cudaStream_t s);

// Cubed-sphere metric blocks of patches [0, npatch) for the solid-body
// rotation omega (already scaled): equiangular gnomonic mapping of each
// face, capacities from two spherical triangles per cell, edge fluxes from
// the stream function -omega . X (Sec. 5.3 mapped grids).  With a remap list
// (rm, device, one entry per patch), RM_COPY patches copy their block from
// old_metric (same omega) instead.
// With corner_out set, every patch's grid corners (three planes of
// (mx+5)^2 unit-sphere components) are also written there.
cudaError_t launch_sphere_metrics(const PatchMeta* meta, int npatch, int mx, const double* omega,
                                  double* metric, const RemapEntry* rm, const double* old_metric,
                                  double* corner_out, cudaStream_t s);

// The deformational flow (FC_VEL_DEFORM): the edge volume fluxes of the
// metric blocks of patches [p0, p1) for time t (t0_dev ? *t0_dev + t_off :
// t_half) from their kept corners; coefficients already scaled:
// kc = k * scale, rot = 2 pi / T_f * scale.
cudaError_t launch_deform_fluxes(int p0, int p1, int mx, const double* corner, double* metric,
                                 double kc, double T, double rot, double t_half,
                                 const double* t0_dev, double t_off, cudaStream_t s);

// fc_mass_noalloc's kernels (scratch in a file-scope device array)
cudaError_t noalloc_mass(const void* q, const double* capacity, int dtype, int mx, int nleaves,
                         const int* level, const int* fstart, int nforests, double* out,
                         cudaStream_t s);
// a partition's halo exchange: pack (pack != 0) the interiors of the listed
// patches into buf, or unpack buf into them
template <typename real>
cudaError_t launch_halo(const DevForest<real>& D, const int* list, int n, real* buf, int pack,
                        cudaStream_t s);
// dst += src over n values (adjoint accumulators)
template <typename real>
cudaError_t launch_add_store(real* dst, const real* src, size_t n, cudaStream_t s);
// interior cell capacities in field order (h^2, or kappa on the cubed sphere)
template <typename real>
cudaError_t launch_pack_capacity(const DevForest<real>& D, const int* api_to_dev, double* out,
                                 cudaStream_t s);

}  // namespace fc
