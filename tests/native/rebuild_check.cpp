// Host check: a layout built from the one it replaces (the regrid's
// incremental build, rows of kept leaves carried over with their patch
// indices renumbered) equals the same layout built from scratch, table for
// table, over sequences of random regrids on every domain kind.
#include <cstdio>
#include <cstring>
#include <random>

#include "fc_internal.hpp"

using namespace fc;

static bool same(const HostForest& A, const HostForest& B) {
  if (A.npatch() != B.npatch()) return false;
  if (std::memcmp(A.nbr.data(), B.nbr.data(), sizeof(NbrEntry) * A.nbr.size())) return false;
  if (std::memcmp(A.meta.data(), B.meta.data(), sizeof(PatchMeta) * A.meta.size())) return false;
  if (A.feeds_finer != B.feeds_finer || A.dev_of != B.dev_of) return false;
  for (int l = 0; l <= kMaxLevel; ++l)
    if (A.list_a[l] != B.list_a[l] || A.list_b[l] != B.list_b[l] || A.list_t[l] != B.list_t[l])
      return false;
  return A.list_all == B.list_all && A.list_coarse_all == B.list_coarse_all;
}

int main() {
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> U(0, 1);
  int ok = 0, bad = 0, carried = 0;
  for (int dom : {FC_DOMAIN_WALLS, FC_DOMAIN_PERIODIC, FC_DOMAIN_SPHERE, FC_DOMAIN_BRICK})
    for (int mx : {8, 32})
      for (int nf : {1, 2}) {
        fc_forest_desc d{};
        d.domain = dom;
        d.mx = mx;
        d.mbc = 2;
        d.lmin = 1;
        d.lmax = 5;
        d.nforests = nf;
        if (dom == FC_DOMAIN_BRICK) {
          d.brick_nx = 2;
          d.brick_ny = 2;
        }
        const int nb = dom == FC_DOMAIN_SPHERE ? 6 : dom == FC_DOMAIN_BRICK ? 4 : 1;
        HostForest H;
        H.desc = d;
        for (int f = 0; f < nf; ++f)
          for (int b = 0; b < nb; ++b)
            for (int y = 0; y < 2; ++y)
              for (int x = 0; x < 2; ++x) H.leaves.push_back(Leaf{f, b, 1, x, y});
        if (!H.build().empty()) return 2;
        for (int it = 0; it < 16; ++it) {
          std::vector<double> delta(H.npatch());
          const double pr = it < 6 ? 0.4 : 0.05;  // grow, then small changes
          for (auto& x : delta) x = U(rng) < pr ? 1.0 : (U(rng) < 0.3 ? 0.0 : 0.5);
          std::vector<Leaf> nl;
          regrid_layout(H, delta, 0.9, 0.1, std::vector<int>(), &nl);
          HostForest A, B;
          A.desc = B.desc = d;
          A.leaves = B.leaves = nl;
          if (!A.build().empty() || !B.build(&H).empty()) return 3;
          if (same(A, B))
            ++ok;
          else
            ++bad;
          carried += A.npatch();
          H = std::move(B);
        }
      }
  std::printf("rebuilds %d equal, %d different\n", ok, bad);
  return bad ? 1 : 0;
}
