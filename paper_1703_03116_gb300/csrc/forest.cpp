// Host-side forest of quadtrees: leaf lookup, face/corner neighbour tables
// with index transforms, level work lists, and the regrid layout (refine,
// 2:1 balance, coarsen).
//
// Sec. 2 (quadtree layout): a level-l quadrant of a unit block has edge 2^-l;
// only leaves hold patches; leaves are enumerated in Morton order; any two
// leaves sharing a face or corner differ by at most one level.
// Sec. 2.2/2.4: each face or corner region of a patch is filled from one
// same-size neighbour, two (face) or one (corner) finer neighbours, or one
// coarser neighbour; Eq. (transform) I_n = A I_c + F maps indices between
// the two patches.
// Sec. 3.1: tagged grids are refined, quiet families of four siblings are
// coarsened, and 2:1 balancing may add refinement.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <mutex>
#include <thread>

#include "fc_internal.hpp"

namespace fc {

// ------------------------------------------------------------------ host pool

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// The workers and the one open job.  A job is open while `gen` is odd; its
// fields are written before it opens and read by a worker only after it
// has announced itself in `active` and seen the job still open, and the
// caller closes the job and waits for `active` to drain before it returns,
// so no worker touches a job's function after its call has returned.
struct HostPool {
  static constexpr int kSpinners = 3;     // workers that arm() keeps polling
  static constexpr int64_t kPollNs = 1000000;  // how long they poll
  int workers = 0;
  pid_t pid = 0;
  std::mutex sleep_mu, run_mu;
  std::condition_variable wake_spin, wake_all;  // the polling workers; every worker
  std::atomic<uint64_t> gen{0};
  std::atomic<int> next{0}, done{0}, active{0};
  std::atomic<int64_t> poll_until{0};
  int n = 0, chunks = 0;
  const std::function<void(int, int, int)>* fn = nullptr;

  bool open() const { return gen.load() & 1; }

  // claim and run pieces of the open job g; returns when none is left
  void take(uint64_t g, int slot);

  void worker(int slot) {
    const bool spinner = slot <= kSpinners;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(sleep_mu);
        if (spinner)
          wake_spin.wait(lk, [&] { return open() || now_ns() < poll_until.load(); });
        else
          wake_all.wait(lk, [&] { return open(); });
      }
      do {
        const uint64_t g = gen.load();
        if (g & 1)
          take(g, slot);
        else
          std::this_thread::yield();
      } while (spinner ? now_ns() < poll_until.load() : open());
    }
  }

  void start() {
    pid = getpid();
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    workers = std::min(15, hw - 1);
    // the workers live as long as the process (the pool is never freed, so
    // a worker never outlives what it reads)
    for (int w = 1; w <= workers; ++w) std::thread([this, w] { worker(w); }).detach();
  }

  void extend_poll() {
    poll_until.store(now_ns() + kPollNs);
    { std::lock_guard<std::mutex> lk(sleep_mu); }
    wake_spin.notify_all();
  }
};

// set while this thread runs a piece: a nested call runs on its caller
thread_local bool t_in_piece = false;

void HostPool::take(uint64_t g, int slot) {
  active.fetch_add(1);
  if (gen.load() == g) {
    t_in_piece = true;
    for (int c = next.fetch_add(1); c < chunks; c = next.fetch_add(1)) {
      (*fn)((int)((long)n * c / chunks), (int)((long)n * (c + 1) / chunks), slot);
      done.fetch_add(1);
    }
    t_in_piece = false;
  }
  active.fetch_sub(1);
}

HostPool* host_pool() {
  static HostPool* p = [] {
    HostPool* q = new HostPool();
    q->start();
    return q;
  }();
  return p;
}

}  // namespace

void host_pool_arm() {
  HostPool* P = host_pool();
  if (P->workers > 0 && P->pid == getpid()) P->extend_poll();
}

void host_pool_run(int n, int chunks, const std::function<void(int, int, int)>& fn) {
  HostPool* P = host_pool();
  std::unique_lock<std::mutex> one(P->run_mu, std::defer_lock);
  if (!t_in_piece) (void)one.try_lock();
  if (!one.owns_lock() || P->workers == 0 || P->pid != getpid() || chunks <= 1) {
    for (int c = 0; c < std::max(1, chunks); ++c)
      fn((int)((long)n * c / std::max(1, chunks)), (int)((long)n * (c + 1) / std::max(1, chunks)),
         0);
    return;
  }
  P->n = n;
  P->chunks = chunks;
  P->fn = &fn;
  P->next.store(0);
  P->done.store(0);
  {
    std::lock_guard<std::mutex> lk(P->sleep_mu);
    P->gen.fetch_add(1);  // open
  }
  P->wake_spin.notify_all();
  P->wake_all.notify_all();
  P->poll_until.store(std::max(P->poll_until.load(), now_ns() + HostPool::kPollNs));
  const uint64_t g = P->gen.load();
  P->take(g, 0);
  while (P->done.load() < chunks) std::this_thread::yield();
  P->gen.fetch_add(1);  // close
  while (P->active.load() > 0) std::this_thread::yield();
  P->fn = nullptr;
}

static uint64_t spread_bits(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

static uint64_t morton_key(const Leaf& a) {
  const int sh = kMaxLevel - a.l;
  return spread_bits((uint32_t)a.x << sh) | (spread_bits((uint32_t)a.y << sh) << 1);
}

void sort_leaves(std::vector<Leaf>* v) {
  // order (forest, block, Morton key, level)
  struct K {
    uint64_t fb, m;
    int l;
    Leaf a;
  };
  const auto key = [](const Leaf& a) {
    return K{((uint64_t)(uint32_t)a.f << 8) | (uint32_t)a.b, morton_key(a), a.l, a};
  };
  const auto less = [](const K& a, const K& b) {
    if (a.fb != b.fb) return a.fb < b.fb;
    if (a.m != b.m) return a.m < b.m;
    return a.l < b.l;
  };
  // a regrid's output is in order already: check that without a copy
  bool sorted = true;
  if (!v->empty()) {
    K prev = key((*v)[0]);
    for (size_t i = 1; sorted && i < v->size(); ++i) {
      const K cur = key((*v)[i]);
      sorted = !less(cur, prev);
      prev = cur;
    }
  }
  if (sorted) return;
  std::vector<K> ks(v->size());  // keys computed once
  for (size_t i = 0; i < v->size(); ++i) ks[i] = key((*v)[i]);
  std::sort(ks.begin(), ks.end(), less);
  for (size_t i = 0; i < v->size(); ++i) (*v)[i] = ks[i].a;
}

static int nblocks(const fc_forest_desc& d) { return num_blocks(d); }

namespace {

// ------------------------------------------------------------ cubed sphere
//
// Folding across a cube edge in index space (Sec. 2.4).  At resolution M
// cells per block side, cell I has the doubled cube coordinate
// U = 2I + 1 - M in (-M, M); M times the cell centre on the face plane is
// M n + U ex + V ey.  A cell beyond the +ex side (U > M) overshoots by
// O = U - M; it is carried over the edge onto the face whose normal is ex,
// at depth O below the edge: M ex + V ey + (M - O) n.  Its doubled
// coordinates there are the components along that face's axes.

int axis_comp(int code, int k) {  // component k of the signed axis `code`
  return (code == k + 1) ? 1 : (code == -(k + 1)) ? -1 : 0;
}

int face_with_normal(int code) {
  for (int c = 0; c < 6; ++c) {
    int n, ex, ey;
    cube_face(c, &n, &ex, &ey);
    if (n == code) return c;
  }
  return -1;
}

// Map cell (I, J) of face b across its side `side` (0: -x, 1: +x, 2: -y,
// 3: +y) at resolution M, without checking that (I, J) lies beyond it; the
// map is affine in (I, J).
void fold_side(int b, int side, long M, long I, long J, int* c, long* Ic, long* Jc) {
  int n, ex, ey;
  cube_face(b, &n, &ex, &ey);
  const long U = 2 * I + 1 - M, V = 2 * J + 1 - M;
  long P[3];
  for (int k = 0; k < 3; ++k) {
    const long en = axis_comp(n, k), e1 = axis_comp(ex, k), e2 = axis_comp(ey, k);
    if (side < 2) {
      const long s = side == 0 ? -1 : 1;  // crossing direction s ex
      const long O = s * U - M;
      P[k] = M * s * e1 + V * e2 + (M - O) * en;
    } else {
      const long s = side == 2 ? -1 : 1;
      const long O = s * V - M;
      P[k] = M * s * e2 + U * e1 + (M - O) * en;
    }
  }
  const int dir = side < 2 ? (side == 0 ? -ex : ex) : (side == 2 ? -ey : ey);
  *c = face_with_normal(dir);
  int cn, cex, cey;
  cube_face(*c, &cn, &cex, &cey);
  long Uc = 0, Vc = 0;
  for (int k = 0; k < 3; ++k) {
    Uc += P[k] * axis_comp(cex, k);
    Vc += P[k] * axis_comp(cey, k);
  }
  *Ic = (Uc + M - 1) / 2;
  *Jc = (Vc + M - 1) / 2;
}

// the transform I' = A I + F of side `side` of face b at resolution M
void side_transform(int b, int side, long M, int* a, int* fx, int* fy) {
  const long I0 = side == 0 ? -1 : (side == 1 ? M : 0);
  const long J0 = side == 2 ? -1 : (side == 3 ? M : 0);
  int c;
  long x0, y0, x1, y1, x2, y2;
  fold_side(b, side, M, I0, J0, &c, &x0, &y0);
  fold_side(b, side, M, I0 + 1, J0, &c, &x1, &y1);
  fold_side(b, side, M, I0, J0 + 1, &c, &x2, &y2);
  const long a11 = x1 - x0, a21 = y1 - y0, a12 = x2 - x0, a22 = y2 - y0;
  int code;
  if (a11 == 0)  // axes swapped: u = +-J, v = +-I
    code = 1 | (a12 < 0 ? 2 : 0) | (a21 < 0 ? 4 : 0);
  else
    code = (a11 < 0 ? 2 : 0) | (a22 < 0 ? 4 : 0);
  int u, v;
  apply_code_host(code, (int)I0, (int)J0, &u, &v);
  *a = code;
  *fx = (int)(x0 - u);
  *fy = (int)(y0 - v);
}

// Where does quadrant (b, l, x, y) of a forest lie once moved across the
// block boundary?  For the square domains the neighbour lies in the same
// block (periodic) or outside the domain (walls); on the cubed sphere it is
// folded across the cube edge.  Returns false for the exterior and beyond a
// cube vertex (then corner3 is set).  (a, fx, fy): the transform of level-l
// cell indices into the new block's frame.
struct Moved {
  int b, x, y, a, fx, fy;
  bool corner3;
};

bool move_quadrant(const fc_forest_desc& d, int b, int l, int x, int y, int mx, Moved* m) {
  const int N = 1 << l;
  m->b = b;
  m->x = x;
  m->y = y;
  m->a = 0;
  m->fx = 0;
  m->fy = 0;
  m->corner3 = false;
  if (x >= 0 && x < N && y >= 0 && y < N) return true;
  if (d.domain == FC_DOMAIN_WALLS) return false;
  if (d.domain == FC_DOMAIN_PERIODIC || d.domain == FC_DOMAIN_BRICK) {
    // the periodic square wraps onto itself; a brick's block continues into
    // the next block of its row or column (periodic at the brick's faces),
    // in the identity orientation with the same level-l cell offsets
    int dx = 0, dy = 0;
    if (x < 0) { m->x = x + N; m->fx = N * mx; dx = -1; }
    if (x >= N) { m->x = x - N; m->fx = -N * mx; dx = 1; }
    if (y < 0) { m->y = y + N; m->fy = N * mx; dy = -1; }
    if (y >= N) { m->y = y - N; m->fy = -N * mx; dy = 1; }
    if (d.domain == FC_DOMAIN_BRICK) {
      const int nx = d.brick_nx, ny = d.brick_ny;
      const int bx = b % nx, by = b / nx;
      m->b = ((by + dy + ny) % ny) * nx + (bx + dx + nx) % nx;
    }
    return true;
  }
  // cubed sphere: one coordinate out -> fold across that cube edge; both out
  // -> beyond a cube vertex
  const bool ox = x < 0 || x >= N, oy = y < 0 || y >= N;
  if (ox && oy) {
    m->corner3 = true;
    return false;
  }
  const int side = ox ? (x < 0 ? 0 : 1) : (y < 0 ? 2 : 3);
  long X, Y;
  fold_side(b, side, N, x, y, &m->b, &X, &Y);
  m->x = (int)X;
  m->y = (int)Y;
  side_transform(b, side, (long)N * mx, &m->a, &m->fx, &m->fy);
  return true;
}

}  // namespace

std::string HostForest::build(const HostForest* prev) {
  const fc_forest_desc& d = desc;
  const int nb = nblocks(d);
  sort_leaves(&leaves);
  const int n = (int)leaves.size();
  for (const Leaf& a : leaves)
    if (a.f < 0 || a.f >= d.nforests || a.b < 0 || a.b >= nb || a.l < d.lmin || a.l > d.lmax ||
        a.x < 0 || a.y < 0 || a.x >= (1 << a.l) || a.y >= (1 << a.l))
      return "leaf out of range";
  forest_start.assign(d.nforests + 1, 0);
  for (const Leaf& a : leaves) forest_start[a.f + 1]++;
  for (int f = 0; f < d.nforests; ++f) forest_start[f + 1] += forest_start[f];

  // Leaf lookup.  Where it is small, a dense map from every cell of each
  // block's finest occupied level to the leaf covering it (filling it also
  // checks that the leaves tile every block exactly); else the key map.
  own_lo.assign(d.nforests, 0);
  for (const Leaf& a : leaves) own_lo[a.f] = std::max(own_lo[a.f], a.l);
  own_off.assign(d.nforests + 1, 0);
  for (int f = 0; f < d.nforests; ++f)
    own_off[f + 1] = own_off[f] + ((size_t)nb << (2 * own_lo[f]));
  dense = own_off[d.nforests] <= std::max<size_t>((size_t)1 << 22, 64 * (size_t)n);
  if (dense) {
    owner.resize(own_off[d.nforests]);
    // forests are independent: host threads take ranges of forests
    std::vector<int> bad(16, 0);  // 1 overlap, 2 a cell without a leaf
    const int per = std::max(1, 16384 / std::max(1, n / std::max(1, d.nforests)));
    parallel_chunks(d.nforests, per, [&](int fb, int fe, int tid) {
      for (int f = fb; f < fe && !bad[tid]; ++f) {
        const int lo = own_lo[f];
        int* own = owner.data() + own_off[f];
        std::fill(own, owner.data() + own_off[f + 1], -1);
        for (int k = forest_start[f]; k < forest_start[f + 1] && !bad[tid]; ++k) {
          const Leaf& a = leaves[k];
          const int s = lo - a.l, w = 1 << s;
          int* o = own + ((size_t)a.b << (2 * lo)) + ((size_t)(a.y << s) << lo) + (a.x << s);
          for (int j = 0; j < w; ++j, o += (size_t)1 << lo)
            for (int i = 0; i < w; ++i) {
              if (o[i] >= 0) bad[tid] = 1;
              o[i] = k;
            }
        }
        for (const int* o = own; !bad[tid] && o < owner.data() + own_off[f + 1]; ++o)
          if (*o < 0) bad[tid] = 2;
      }
    });
    for (int e : bad) {
      if (e == 1) return "overlapping leaves";
      if (e == 2) return "leaves do not tile every block";
    }
  } else {
    owner.clear();
    // the key map, filled by host threads (leaves of a thread: a few
    // forests, whose probe windows are their own)
    idx.clear(leaves.size(), d.nforests);
    std::vector<char> dup(16, 0);
    parallel_chunks(n, 16384, [&](int kb, int ke, int tid) {
      for (int k = kb; k < ke; ++k) {
        const Leaf& a = leaves[k];
        if (!idx.insert_concurrent(leaf_key(a.f, a.b, a.l, a.x, a.y), k)) dup[tid] = 1;
      }
    });
    idx.set_size(leaves.size());
    for (char c : dup)
      if (c) return "duplicate leaf";
    // exact tiling: areas of each block sum to one and no leaf has a leaf
    // ancestor (the ancestor lookups read the finished key map: host threads)
    std::vector<char> overlap(16, 0);
    parallel_chunks(n, 16384, [&](int kb, int ke, int tid) {
      for (int k = kb; k < ke && !overlap[tid]; ++k) {
        const Leaf& a = leaves[k];
        for (int l = a.l - 1; l >= d.lmin; --l)
          if (find(a.f, a.b, l, a.x >> (a.l - l), a.y >> (a.l - l)) >= 0) {
            overlap[tid] = 1;
            break;
          }
      }
    });
    for (char o : overlap)
      if (o) return "overlapping leaves";
    std::vector<double> area((size_t)d.nforests * nb, 0.0);
    for (const Leaf& a : leaves) area[(size_t)a.f * nb + a.b] += std::ldexp(1.0, -2 * a.l);
    for (double s : area)
      if (s != 1.0) return "leaves do not tile every block";
  }

  // device order: (level, field order), a counting sort by level
  for (int l = 0; l <= kMaxLevel + 1; ++l) lev_start[l] = 0;
  for (const Leaf& a : leaves) lev_start[a.l + 1]++;
  for (int l = 1; l <= kMaxLevel + 1; ++l) lev_start[l] += lev_start[l - 1];
  api_of.resize(n);
  dev_of.resize(n);
  {
    int next[kMaxLevel + 1];
    for (int l = 0; l <= kMaxLevel; ++l) next[l] = lev_start[l];
    for (int k = 0; k < n; ++k) {
      const int p = next[leaves[k].l]++;
      api_of[p] = k;
      dev_of[k] = p;
    }
  }

  // every row is written below (no zero fill)
  meta.resize(n);
  nbr.resize((size_t)n * 8);
  feeds_finer.assign(n, 0);
  // rows carried over from the replaced layout: prev's device index -> ours
  const bool incr = prev && prev != this && !prev->partial && !partial &&
                    prev->desc.nforests == d.nforests && prev->desc.mx == d.mx &&
                    prev->nbr.size() == (size_t)prev->npatch() * 8 &&
                    prev->meta.size() == (size_t)prev->npatch();
  std::vector<int> prev_k, dev_map;
  if (incr) {
    prev_k.resize(n);
    dev_map.assign(prev->npatch(), -1);
    for (int k = 0; k < n; ++k) {
      const Leaf& a = leaves[k];
      const int o = prev->find(a.f, a.b, a.l, a.x, a.y);
      prev_k[k] = o;
      if (o >= 0) dev_map[prev->dev_of[o]] = dev_of[k];
    }
  }
  // a carried row: every patch it names still a leaf; false leaves the row
  // to be computed
  const auto carry = [&](int k) {
    const int o = prev_k[k];
    if (o < 0) return false;
    const int op = prev->dev_of[o], p = dev_of[k];
    NbrEntry row[8];
    for (int dir = 0; dir < 8; ++dir) {
      NbrEntry e = prev->nbr[(size_t)op * 8 + dir];
      for (int* id : {&e.n0, &e.n1})
        if (*id >= 0 && (*id = dev_map[*id]) < 0) return false;
      row[dir] = e;
    }
    for (int dir = 0; dir < 8; ++dir) {
      nbr[(size_t)p * 8 + dir] = row[dir];
      if (row[dir].kind == NB_COARSE)  // (several threads may store the same byte)
        __atomic_store_n(&feeds_finer[row[dir].n0], (char)1, __ATOMIC_RELAXED);
    }
    meta[p] = prev->meta[op];
    return true;
  };
  // the rows are independent (each reads the leaf tables only): host threads
  // take contiguous ranges of leaves in field order, so one thread's lookups
  // stay within a few forests
  std::vector<std::string> row_err(16);
  parallel_chunks(n, 64, [&](int kb, int ke, int tid) {
    for (int k = kb; k < ke; ++k) {
      if (incr && carry(k)) continue;
      const std::string e = neighbour_rows(k, k + 1);
      if (!e.empty()) row_err[tid] = e;
    }
  });
  for (const auto& e : row_err)
    if (!e.empty()) return e;
  // work lists
  return work_lists();
}

std::string HostForest::neighbour_rows(int kb, int ke) {
  const fc_forest_desc& d = desc;
  const int mx = d.mx;
  for (int k = kb; k < ke; ++k) {
    const int p = dev_of[k];
    const Leaf& a = leaves[k];
    meta[p] = PatchMeta{a.l, a.x, a.y, a.b, a.f, 0};
    for (int dir = 0; dir < 8; ++dir) {
      NbrEntry e{NB_EXTERIOR, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, {-1, -1}, {0, 0}};
      int k0 = -1, k1 = -1;  // the neighbours' leaf indices
      Moved m;
      if (move_quadrant(d, a.b, a.l, a.x + kDirX[dir], a.y + kDirY[dir], mx, &m)) {
        e.a = m.a;
        e.fx = m.fx;
        e.fy = m.fy;
        const int h = holder(a.f, m.b, a.l, m.x, m.y);
        if (h >= 0 && leaves[h].l == a.l) {
          e.kind = NB_SAME;
          k0 = h;
        } else {
          const int c = h;  // a coarser leaf, one level up
          if (c >= 0) {
            e.kind = NB_COARSE;
            k0 = c;
            meta[p].flags |= 1;
            // several threads may mark the same patch: all store the same byte
            __atomic_store_n(&feeds_finer[dev_of[c]], (char)1, __ATOMIC_RELAXED);
          } else {
            // finer: the children of the same-size quadrant that touch this
            // patch, on its side facing back along the direction of travel
            // (expressed in the neighbour block's frame)
            int ox, oy;
            apply_code_host(m.a, kDirX[dir], kDirY[dir], &ox, &oy);
            int cx[2], cy[2], nc;
            if (ox != 0 && oy != 0) {
              nc = 1;
              cx[0] = 2 * m.x + (ox < 0 ? 1 : 0);
              cy[0] = 2 * m.y + (oy < 0 ? 1 : 0);
            } else if (ox != 0) {
              nc = 2;
              cx[0] = cx[1] = 2 * m.x + (ox < 0 ? 1 : 0);
              cy[0] = 2 * m.y;
              cy[1] = 2 * m.y + 1;
            } else {
              nc = 2;
              cy[0] = cy[1] = 2 * m.y + (oy < 0 ? 1 : 0);
              cx[0] = 2 * m.x;
              cx[1] = 2 * m.x + 1;
            }
            int ids[2] = {-1, -1};
            for (int q = 0; q < nc; ++q) {
              ids[q] = (a.l < d.lmax) ? find(a.f, m.b, a.l + 1, cx[q], cy[q]) : -1;
              if (ids[q] < 0) {
                char buf[160];
                std::snprintf(buf, sizeof buf,
                              "leaf (f=%d b=%d l=%d x=%d y=%d): region %d has no neighbour within "
                              "one level (layout not 2:1 balanced)",
                              a.f, a.b, a.l, a.x, a.y, dir);
                return buf;
              }
            }
            e.kind = NB_FINE;
            k0 = ids[0];
            k1 = nc == 2 ? ids[1] : -1;
          }
        }
      } else if (m.corner3) {
        e.kind = NB_CORNER3;
      }
      if (k0 >= 0) {
        const Leaf& n0 = leaves[k0];
        e.n0 = dev_of[k0];
        e.lev = n0.l;
        e.x0 = n0.x;
        e.y0 = n0.y;
      }
      if (k1 >= 0) {
        const Leaf& n1 = leaves[k1];
        e.n1 = dev_of[k1];
        e.x1 = n1.x;
        e.y1 = n1.y;
      }
      nbr[(size_t)p * 8 + dir] = e;
    }
  }
  return "";
}

// the face whose outward normal is (nx, ny): 0 -x, 1 +x, 2 -y, 3 +y
static int face_of_normal(int nx, int ny) {
  return nx < 0 ? 0 : nx > 0 ? 1 : ny < 0 ? 2 : 3;
}

std::string HostForest::reflux_pairs(int* out) const {
  const int mx = desc.mx;
  const bool sphere = desc.domain == FC_DOMAIN_SPHERE;
  for (int k = 0; k < npatch(); ++k) {
    const Leaf& a = leaves[k];
    const int p = dev_of[k];
    const int X0 = a.x * mx, Y0 = a.y * mx;
    for (int dir = 0; dir < 4; ++dir) {
      const NbrEntry& e = nbr[(size_t)p * 8 + dir];
      // the neighbour's outward normal on the shared edge: back along the
      // direction of travel, in its block's frame
      int dx, dy;
      apply_code_host(e.a, kDirX[dir], kDirY[dir], &dx, &dy);
      const int g = face_of_normal(-dx, -dy);
      for (int c = 0; c < mx; ++c) {
        int* o = out + (((size_t)k * 4 + dir) * mx + c) * 5;
        o[0] = 0;
        o[1] = o[2] = o[3] = o[4] = -1;
        // the level-l ghost cell across the face beside cell c
        const int Ix = dir == 0 ? X0 - 1 : dir == 1 ? X0 + mx : X0 + c;
        const int Iy = dir == 2 ? Y0 - 1 : dir == 3 ? Y0 + mx : Y0 + c;
        int u, v;
        apply_code_host(e.a, Ix, Iy, &u, &v);
        u += e.fx;
        v += e.fy;
        if (e.kind == NB_FINE) {
          int j[2], leaf = -1;
          for (int half = 0; half < 2; ++half) {
            // the fine cell of the ghost cell beside this leaf, at the lower
            // or upper half of cell c along the face, in this leaf's frame
            const int ox = dir == 0 ? 1 : dir == 1 ? 0 : half;
            const int oy = dir == 2 ? 1 : dir == 3 ? 0 : half;
            int du, dv;
            apply_code_host(e.a, ox, oy, &du, &dv);
            const int fx = 2 * u + ((e.a & 2) ? 1 + du : du);
            const int fy = 2 * v + ((e.a & 4) ? 1 + dv : dv);
            int n = -1, lx = 0, ly = 0;
            if (fx / mx == e.x0 && fy / mx == e.y0 && fx >= 0 && fy >= 0) {
              n = e.n0;
              lx = fx - e.x0 * mx;
              ly = fy - e.y0 * mx;
            } else if (e.n1 >= 0 && fx >= 0 && fy >= 0 && fx / mx == e.x1 && fy / mx == e.y1) {
              n = e.n1;
              lx = fx - e.x1 * mx;
              ly = fy - e.y1 * mx;
            }
            if (n < 0 || (leaf >= 0 && n != leaf)) return "reflux pairing: fine cell outside the face's leaves";
            leaf = n;
            j[half] = g < 2 ? ly : lx;
          }
          o[0] = 1;
          o[1] = api_of[leaf];
          o[2] = g;
          o[3] = j[0];
          o[4] = j[1];
        } else if (e.kind == NB_SAME && sphere && leaves[api_of[e.n0]].b < a.b) {
          const int lx = u - e.x0 * mx, ly = v - e.y0 * mx;
          if (lx < 0 || lx >= mx || ly < 0 || ly >= mx)
            return "reflux pairing: ghost cell outside the same-size leaf";
          o[0] = 2;
          o[1] = api_of[e.n0];
          o[2] = g;
          o[3] = g < 2 ? ly : lx;
        }
      }
    }
  }
  return "";
}

std::string HostForest::work_lists() {
  const int n = npatch();
  list_all.resize(n);
  list_coarse_all.clear();
  // feeds_finer[p]: p is the coarser neighbour of a patch one level finer
  // (2:1 balance: a coarse neighbour is always exactly one level coarser)
  const std::vector<char>& inT = feeds_finer;
  for (int p = 0; p < n; ++p) {
    list_all[p] = p;
    if (meta[p].flags & 1) list_coarse_all.push_back(p);
  }
  for (int l = 0; l <= kMaxLevel; ++l) {
    list_a[l].clear();
    list_b[l].clear();
    list_t[l].clear();
    if (l > 0)
      for (int p = lev_start[l - 1]; p < lev_start[l]; ++p)
        if (inT[p]) {
          list_a[l].push_back(p);
          list_t[l].push_back(p);
        }
    for (int p = lev_start[l]; p < lev_start[l + 1]; ++p) {
      list_a[l].push_back(p);
      if (meta[p].flags & 1) list_b[l].push_back(p);
    }
  }
  return "";
}

// ------------------------------------------------------------------ regrid

namespace {

// The leaf set of a regrid in progress.  Where it is small, a dense map from
// every cell of each forest's finest level in play to the level of the leaf
// covering it (a byte a cell; the set is a tiling throughout, so a leaf is
// present when its anchor cell carries its level, and every erase is
// followed by adds over the same cells); else a key map.
struct LeafSet {
  const fc_forest_desc* d;
  bool dense = false;
  int f0 = 0;
  std::vector<int> lo;      // finest level in play, per forest from f0
  std::vector<size_t> off;  // start of each forest's cells
  std::vector<int8_t> lev;
  KeyMap m;  // leaf key -> 1
  size_t anchor(int f, int b, int l, int x, int y) const {
    const int L = lo[f - f0], s = L - l;
    return off[f - f0] + ((size_t)b << (2 * L)) + ((size_t)(y << s) << L) + (x << s);
  }
  bool has(int f, int b, int l, int x, int y) const {
    if (dense) return l <= lo[f - f0] && lev[anchor(f, b, l, x, y)] == l;
    return m.find(leaf_key(f, b, l, x, y)) >= 0;
  }
  void add(const Leaf& a) {
    if (!dense) {
      m.insert(leaf_key(a.f, a.b, a.l, a.x, a.y), 1);
      return;
    }
    const int L = lo[a.f - f0], w = 1 << (L - a.l);
    int8_t* row = lev.data() + anchor(a.f, a.b, a.l, a.x, a.y);
    for (int j = 0; j < w; ++j, row += (size_t)1 << L) std::fill(row, row + w, (int8_t)a.l);
  }
  void erase(const Leaf& a) {
    if (!dense) m.erase(leaf_key(a.f, a.b, a.l, a.x, a.y));
  }
  // level of the leaf containing quadrant (b, l, x, y) if that leaf is at
  // level <= l, else -1 (the quadrant is subdivided)
  int holder_level(int f, int b, int l, int x, int y, Leaf* out) const {
    if (dense) {
      const int L = lo[f - f0];
      const int cl = l < L ? l : L;
      const int k = lev[anchor(f, b, cl, x >> (l - cl), y >> (l - cl))];
      if (k > l) return -1;
      if (out) *out = Leaf{f, b, k, x >> (l - k), y >> (l - k)};
      return k;
    }
    for (int k = l; k >= d->lmin; --k) {
      const int xs = x >> (l - k), ys = y >> (l - k);
      if (m.find(leaf_key(f, b, k, xs, ys)) >= 0) {
        if (out) *out = Leaf{f, b, k, xs, ys};
        return k;
      }
    }
    return -1;
  }
};

void refine_into(LeafSet* s, const Leaf& a) {
  s->erase(a);
  for (int c = 0; c < 4; ++c) s->add(Leaf{a.f, a.b, a.l + 1, 2 * a.x + (c & 1), 2 * a.y + (c >> 1)});
}

// 2:1 balance by refinement: any leaf that holds a quadrant adjacent to a
// leaf two or more levels finer is refined, until no such leaf remains.  The
// layout before the new refinements was balanced, so only leaves next to new
// leaves can violate it: a worklist seeded with the new leaves ripples the
// refinement outwards.  Every leaf refined here is refined in any balanced
// refinement, so the result is the (unique) coarsest balanced one.
void balance(LeafSet* s, int mx, std::vector<Leaf> work) {
  while (!work.empty()) {
    const Leaf c = work.back();
    work.pop_back();
    if (c.l < s->d->lmin + 2 || !s->has(c.f, c.b, c.l, c.x, c.y)) continue;
    for (int dir = 0; dir < 8; ++dir) {
      Moved m;
      if (!move_quadrant(*s->d, c.b, c.l, c.x + kDirX[dir], c.y + kDirY[dir], mx, &m)) continue;
      Leaf h;
      int hl = s->holder_level(c.f, m.b, c.l, m.x, m.y, &h);
      if (hl >= 0 && hl <= c.l - 2) {
        refine_into(s, h);
        for (int k = 0; k < 4; ++k)
          work.push_back(Leaf{h.f, h.b, h.l + 1, 2 * h.x + (k & 1), 2 * h.y + (k >> 1)});
        work.push_back(c);  // look again: the new holder may still be too coarse
        break;
      }
    }
  }
}

// Would the parent P of a family stay balanced?  Every quadrant two levels
// finer than P that touches P must lie inside a leaf at most one level finer.
bool parent_balanced(const LeafSet& s, const Leaf& P, int mx) {
  const int l2 = P.l + 2;
  const int x0 = 4 * P.x, y0 = 4 * P.y;
  for (int k = -1; k <= 4; ++k)
    for (int side = 0; side < 4; ++side) {
      int zx, zy;
      if (side == 0) { zx = x0 - 1; zy = y0 + k; }
      else if (side == 1) { zx = x0 + 4; zy = y0 + k; }
      else if (side == 2) { zx = x0 + k; zy = y0 - 1; }
      else { zx = x0 + k; zy = y0 + 4; }
      Moved m;
      if (!move_quadrant(*s.d, P.b, l2, zx, zy, mx, &m)) continue;
      if (s.holder_level(P.f, m.b, l2 - 1, m.x >> 1, m.y >> 1, nullptr) < 0) return false;
    }
  return true;
}

// append the leaves of s that cover quadrant a, in field order (a is a
// leaf of the previous layout)
void emit_region(const LeafSet& s, const Leaf& a, int lmin, std::vector<Leaf>* out) {
  if (s.has(a.f, a.b, a.l, a.x, a.y)) {
    out->push_back(a);
    return;
  }
  if (a.l > lmin && s.has(a.f, a.b, a.l - 1, a.x >> 1, a.y >> 1)) {
    if (!(a.x & 1) && !(a.y & 1)) out->push_back(Leaf{a.f, a.b, a.l - 1, a.x >> 1, a.y >> 1});
    return;
  }
  for (int c = 0; c < 4; ++c)
    emit_region(s, Leaf{a.f, a.b, a.l + 1, 2 * a.x + (c & 1), 2 * a.y + (c >> 1)}, lmin, out);
}

}  // namespace

namespace {

// the new layout of the leaves [k0, k1) of F (whole forests: balance and
// coarsening never cross a forest)
void regrid_range(const HostForest& F, const std::vector<double>& delta, double tau_r,
                  double tau_c, const std::vector<int>& lmax_f, int k0, int k1,
                  std::vector<Leaf>* out) {
  const fc_forest_desc& d = F.desc;
  const int n = F.npatch();
  std::vector<char> refine(n, 0);
  for (int k = k0; k < k1; ++k) {
    const Leaf& a = F.leaves[k];
    int lm = lmax_f.empty() ? d.lmax : std::min(lmax_f[a.f], d.lmax);
    refine[k] = (delta[k] > tau_r) && (a.l < lm);
  }
  // Sec. 3.3 smooth grading: each leaf's target level (one finer if tagged
  // to refine, one coarser if below tau_c, else its own) is raised to the
  // largest target among the leaves it touches (the neighbour table's
  // entries); a leaf refines when its graded target is finer, and a family
  // coarsens only when all four graded targets are coarser
  std::vector<int> target;
  if (d.smooth) {
    std::vector<int> t0(n, 0);
    for (int k = k0; k < k1; ++k) {
      const int l = F.leaves[k].l;
      t0[k] = refine[k] ? l + 1 : (delta[k] < tau_c && l > d.lmin) ? l - 1 : l;
    }
    target.assign(n, 0);
    for (int k = k0; k < k1; ++k) {
      int t = t0[k];
      const int p = F.dev_of[k];
      for (int dir = 0; dir < 8; ++dir) {
        const NbrEntry& e = F.nbr[(size_t)p * 8 + dir];
        if (e.kind != NB_SAME && e.kind != NB_COARSE && e.kind != NB_FINE) continue;
        for (const int id : {e.n0, e.n1})
          if (id >= 0) t = std::max(t, t0[F.api_of[id]]);
      }
      target[k] = t;
      const Leaf& a = F.leaves[k];
      const int lm = lmax_f.empty() ? d.lmax : std::min(lmax_f[a.f], d.lmax);
      refine[k] = t > a.l && a.l < lm;
    }
  }
  std::vector<Leaf> parents;
  for (int k = k0; k < k1; ++k) {
    const Leaf& a = F.leaves[k];
    if (a.l <= d.lmin || (a.x & 1) || (a.y & 1)) continue;
    bool ok = true;
    for (int c = 0; c < 4 && ok; ++c) {
      int s = F.find(a.f, a.b, a.l, a.x + (c & 1), a.y + (c >> 1));
      if (s < 0 || refine[s]) ok = false;
      else if (d.smooth ? !(target[s] < a.l) : !(delta[s] < tau_c)) ok = false;
    }
    if (ok) parents.push_back(Leaf{a.f, a.b, a.l - 1, a.x / 2, a.y / 2});
  }
  LeafSet s;
  s.d = &d;
  {
    const int nb = num_blocks(d);
    const int fa = k1 > k0 ? F.leaves[k0].f : 0, fb = k1 > k0 ? F.leaves[k1 - 1].f + 1 : 0;
    s.f0 = fa;
    s.lo.assign(fb - fa, 0);
    for (int f = fa; f < fb; ++f)
      s.lo[f - fa] = lmax_f.empty() ? d.lmax : std::min(lmax_f[f], d.lmax);
    for (int k = k0; k < k1; ++k)
      s.lo[F.leaves[k].f - fa] = std::max(s.lo[F.leaves[k].f - fa], F.leaves[k].l);
    s.off.assign(fb - fa + 1, 0);
    for (int f = fa; f < fb; ++f)
      s.off[f - fa + 1] = s.off[f - fa] + ((size_t)nb << (2 * s.lo[f - fa]));
    s.dense = s.off[fb - fa] <= ((size_t)1 << 22);
    if (s.dense)
      s.lev.assign(s.off[fb - fa], (int8_t)-1);
    else
      s.m.clear((size_t)(k1 - k0) * 2, fb - fa > 0 ? fb - fa : 1);
  }
  for (int k = k0; k < k1; ++k)
    if (!refine[k]) s.add(F.leaves[k]);
  std::vector<Leaf> fresh;
  for (int k = k0; k < k1; ++k)
    if (refine[k]) {
      const Leaf& a = F.leaves[k];
      for (int c = 0; c < 4; ++c) {
        const Leaf ch{a.f, a.b, a.l + 1, 2 * a.x + (c & 1), 2 * a.y + (c >> 1)};
        s.add(ch);
        fresh.push_back(ch);
      }
    }
  const size_t fresh_count = fresh.size();
  balance(&s, d.mx, std::move(fresh));
  std::vector<Leaf> accepted;
  for (const Leaf& P : parents) {
    bool all = true;
    for (int c = 0; c < 4 && all; ++c)
      all = s.has(P.f, P.b, P.l + 1, 2 * P.x + (c & 1), 2 * P.y + (c >> 1));
    if (all && parent_balanced(s, P, d.mx)) accepted.push_back(P);
  }
  for (const Leaf& P : accepted) {
    for (int c = 0; c < 4; ++c)
      s.erase(Leaf{P.f, P.b, P.l + 1, 2 * P.x + (c & 1), 2 * P.y + (c >> 1)});
    s.add(P);
  }
  // the new leaves in field order, without a sort: each old leaf's region
  // now holds the old leaf itself, or new leaves below it (refinement and
  // balance), or lies in a new parent (a coarsened family, emitted in place
  // of the family's first child, where its key sorts)
  out->clear();
  out->reserve((size_t)(k1 - k0) + 3 * fresh_count);
  for (int k = k0; k < k1; ++k) emit_region(s, F.leaves[k], d.lmin, out);
}

}  // namespace

std::string regrid_layout(const HostForest& F, const std::vector<double>& delta, double tau_r,
                          double tau_c, const std::vector<int>& lmax_f,
                          std::vector<Leaf>* out) {
  // forests are independent: host threads take contiguous ranges of forests
  const int nf = F.desc.nforests;
  const int n = F.npatch();
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::max(1, std::min({hw, 16, nf, n / 8192}));
  std::vector<std::vector<Leaf>> parts(nt);
  parallel_chunks(nt, 1, [&](int tb, int te, int) {
    for (int t = tb; t < te; ++t) {
      const int f0 = (int)((long)nf * t / nt), f1 = (int)((long)nf * (t + 1) / nt);
      regrid_range(F, delta, tau_r, tau_c, lmax_f, F.forest_start[f0], F.forest_start[f1],
                   &parts[t]);
    }
  });
  out->clear();
  for (auto& pt : parts) out->insert(out->end(), pt.begin(), pt.end());
  return "";
}

}  // namespace fc

namespace fc {

// ------------------------------------------------------------------ partition
//
// Sec. 3 (partitioning): the leaves, in their Morton (field) order, are split
// into contiguous ranges of equal work, a level-l leaf weighing 2^(l - lmin)
// (its updates per coarse step).  Each rank holds its own leaves plus the
// mirrors its ghost fills read; one exchange per level substep refreshes the
// mirrors from their owners (Sec. 3, parallel ghost filling).

std::vector<int> partition_ranges(const HostForest& G, int nranks) {
  const int n = G.npatch(), lmin = G.desc.lmin;
  std::vector<double> cum(n + 1, 0.0);
  for (int k = 0; k < n; ++k) cum[k + 1] = cum[k] + std::ldexp(1.0, G.leaves[k].l - lmin);
  const double W = cum[n];
  std::vector<int> part(n);
  for (int k = 0; k < n; ++k) {
    // the rank whose share of the work holds this leaf's midpoint
    const double mid = 0.5 * (cum[k] + cum[k + 1]);
    int r = (int)(mid * nranks / W);
    part[k] = std::min(std::max(r, 0), nranks - 1);
  }
  return part;
}

std::vector<int> partition_mirrors(const HostForest& G, const std::vector<int>& part, int rank) {
  const int n = G.npatch();
  std::vector<char> need(n, 0);
  auto mark = [&](int dev) {
    if (dev < 0) return;
    const int k = G.api_of[dev];
    if (part[k] != rank) need[k] = 1;
  };
  for (int k = 0; k < n; ++k) {
    if (part[k] != rank) continue;
    const int p = G.dev_of[k];
    for (int dir = 0; dir < 8; ++dir) {
      const NbrEntry& e = G.nbr[(size_t)p * 8 + dir];
      mark(e.n0);
      mark(e.n1);
      if (e.kind != NB_COARSE) continue;
      // the coarse neighbour's ghosts that the interpolation reads come from
      // its same-size and finer neighbours (copies and averages)
      for (int d2 = 0; d2 < 8; ++d2) {
        const NbrEntry& c = G.nbr[(size_t)e.n0 * 8 + d2];
        if (c.kind == NB_SAME || c.kind == NB_FINE) {
          mark(c.n0);
          mark(c.n1);
        }
      }
    }
  }
  std::vector<int> out;
  for (int k = 0; k < n; ++k)
    if (need[k]) out.push_back(k);
  return out;
}

std::string build_partition(const HostForest& G, const std::vector<int>& part, int rank,
                            HostForest* H) {
  const int n = G.npatch();
  int nranks = 0;
  for (int r : part) nranks = std::max(nranks, r + 1);
  if (rank < 0 || rank >= nranks) return "rank outside the partition";
  std::vector<std::vector<int>> mirrors(nranks);
  for (int r = 0; r < nranks; ++r) mirrors[r] = partition_mirrors(G, part, r);
  // local leaves: owned (field order), then mirrors (field order)
  std::vector<int> local;  // G field index of each local leaf
  for (int k = 0; k < n; ++k)
    if (part[k] == rank) local.push_back(k);
  const int nowned = (int)local.size();
  if (nowned == 0) return "rank owns no leaf";
  for (int k : mirrors[rank]) local.push_back(k);
  const int nl = (int)local.size();
  std::vector<int> loc_of(n, -1);  // G field index -> local field index
  for (int i = 0; i < nl; ++i) loc_of[local[i]] = i;

  H->desc = G.desc;
  H->partial = true;
  H->nowned = nowned;
  H->nranks = nranks;
  H->rank = rank;
  H->dense = false;
  H->leaves.resize(nl);
  for (int i = 0; i < nl; ++i) H->leaves[i] = G.leaves[local[i]];
  H->idx.clear(nl, G.desc.nforests);
  for (int i = 0; i < nl; ++i) {
    const Leaf& a = H->leaves[i];
    H->idx.insert(leaf_key(a.f, a.b, a.l, a.x, a.y), i);
  }
  // the field layout covers the owned leaves
  H->forest_start.assign(G.desc.nforests + 1, 0);
  for (int i = 0; i < nowned; ++i) H->forest_start[H->leaves[i].f + 1]++;
  for (int f = 0; f < G.desc.nforests; ++f) H->forest_start[f + 1] += H->forest_start[f];
  // device order: by level, each level's owned patches first
  for (int l = 0; l <= kMaxLevel + 1; ++l) H->lev_start[l] = 0;
  for (const Leaf& a : H->leaves) H->lev_start[a.l + 1]++;
  for (int l = 1; l <= kMaxLevel + 1; ++l) H->lev_start[l] += H->lev_start[l - 1];
  H->api_of.assign(nl, 0);
  H->dev_of.assign(nl, 0);
  {
    int next[kMaxLevel + 1];
    for (int l = 0; l <= kMaxLevel; ++l) next[l] = H->lev_start[l];
    for (int pass = 0; pass < 2; ++pass)
      for (int i = pass ? nowned : 0; i < (pass ? nl : nowned); ++i) {
        const int p = next[H->leaves[i].l]++;
        H->api_of[p] = i;
        H->dev_of[i] = p;
      }
    // owned patches were placed first: level l's end of them
    for (int l = 0; l <= kMaxLevel; ++l) H->own_end[l] = H->lev_start[l];
    for (int i = 0; i < nowned; ++i) H->own_end[H->leaves[i].l]++;
  }
  // rows of G restricted to the local leaves; a neighbour not held here
  // makes the region NB_ABSENT (only mirrors have such regions)
  H->meta.resize(nl);
  H->nbr.resize((size_t)nl * 8);
  H->feeds_finer.assign(nl, 0);
  auto to_local_dev = [&](int gdev) -> int {
    if (gdev < 0) return -1;
    const int i = loc_of[G.api_of[gdev]];
    return i < 0 ? -1 : H->dev_of[i];
  };
  for (int i = 0; i < nl; ++i) {
    const int gp = G.dev_of[local[i]], p = H->dev_of[i];
    H->meta[p] = G.meta[gp];
    for (int dir = 0; dir < 8; ++dir) {
      NbrEntry e = G.nbr[(size_t)gp * 8 + dir];
      const bool two = e.n1 >= 0;
      const int a0 = to_local_dev(e.n0), a1 = to_local_dev(e.n1);
      if ((e.n0 >= 0 && a0 < 0) || (two && a1 < 0)) {
        if (i < nowned) return "partition: an owned leaf's neighbour is not held";
        e.kind = NB_ABSENT;
        e.n0 = e.n1 = -1;
      } else {
        e.n0 = a0;
        e.n1 = a1;
      }

      H->nbr[(size_t)p * 8 + dir] = e;
      if (i < nowned && e.kind == NB_COARSE) H->feeds_finer[e.n0] = 1;
    }
  }
  // work lists of what the owned leaves' updates and fills touch
  H->list_all.clear();
  H->list_coarse_all.clear();
  for (int p = 0; p < nl; ++p) {
    const bool own = H->api_of[p] < nowned;
    if (own || H->feeds_finer[p]) H->list_all.push_back(p);
    if (own && (H->meta[p].flags & 1)) H->list_coarse_all.push_back(p);
  }
  for (int l = 0; l <= kMaxLevel; ++l) {
    H->list_a[l].clear();
    H->list_b[l].clear();
    H->list_t[l].clear();
    if (l > 0)
      for (int p = H->lev_start[l - 1]; p < H->lev_start[l]; ++p)
        if (H->feeds_finer[p]) {
          H->list_a[l].push_back(p);
          H->list_t[l].push_back(p);
        }
    for (int p = H->lev_start[l]; p < H->own_end[l]; ++p) {
      H->list_a[l].push_back(p);
      if (H->meta[p].flags & 1) H->list_b[l].push_back(p);
    }
  }
  // exchange lists with every other rank, per level, in G's field order
  for (int l = 0; l <= kMaxLevel; ++l) {
    H->send[l].assign(nranks, {});
    H->recv[l].assign(nranks, {});
  }
  for (int r = 0; r < nranks; ++r) {
    if (r == rank) continue;
    for (int k : mirrors[r])
      if (part[k] == rank) H->send[G.leaves[k].l][r].push_back(H->dev_of[loc_of[k]]);
    for (int k : mirrors[rank])
      if (part[k] == r) H->recv[G.leaves[k].l][r].push_back(H->dev_of[loc_of[k]]);
  }
  return "";
}

}  // namespace fc
