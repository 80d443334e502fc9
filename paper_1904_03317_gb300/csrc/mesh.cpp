// Forest of a Cartesian brick: isotropic refinement and 2:1 closure (host).
//
// A cell is (level l, integer coordinates c on the level-l lattice of
// n0[d] * 2^l cells per direction); its children are (l+1, 2c + b),
// b in {0,1}^dim (Sec. 2.2).  The closure keeps leaves whose closures touch
// within one level of each other (Sec. 3.5; one-irregular meshes, Sec. 1):
// every refined cell of level l >= 1 must have all its lattice neighbours of
// level l inside the domain.  It is restored in one sweep from the finest
// level down; a missing neighbour is created by refining its parent, which
// is first made to exist the same way.  Every refinement made is forced, so
// the result is the minimal balanced refinement.
#include <algorithm>
#include <numeric>

#include "gmg_internal.h"

namespace gmg {

void Forest::init(const gmg_coarse_mesh& cm) {
  dim = cm.dim;
  for (int d = 0; d < 3; ++d) {
    n0[d] = d < dim ? cm.n0[d] : 1;
    lo[d] = cm.lo[d];
    hi[d] = cm.hi[d];
  }
  cells.assign(1, HashMap64());
  cells[0].reserve((size_t)n0[0] * n0[1] * n0[2]);
  for (int z = 0; z < n0[2]; ++z)
    for (int y = 0; y < n0[1]; ++y)
      for (int x = 0; x < n0[0]; ++x) cells[0].insert(pack3(x, y, z), 0);
  rebuild_leaves();
}

bool Forest::inside(int level, const int64_t* c) const {
  for (int d = 0; d < 3; ++d) {
    int64_t ext = d < dim ? ((int64_t)n0[d] << level) : 1;
    if (c[d] < 0 || c[d] >= ext) return false;
  }
  return true;
}

bool Forest::exists(int level, const int64_t* c) const {
  if (level >= (int)cells.size() || !inside(level, c)) return false;
  return cells[level].find(pack3(c[0], c[1], c[2])) != nullptr;
}

bool Forest::refined(int level, const int64_t* c) const {
  if (level >= (int)cells.size() || !inside(level, c)) return false;
  const int32_t* v = cells[level].find(pack3(c[0], c[1], c[2]));
  return v && *v;
}

void Forest::refine_cell(int level, const int64_t* c) {
  int32_t* v = cells[level].find(pack3(c[0], c[1], c[2]));
  if (!v || *v) return;
  *v = 1;
  if (level + 1 == (int)cells.size()) cells.emplace_back();
  HashMap64& next = cells[level + 1];
  int nb = 1 << dim;
  for (int b = 0; b < nb; ++b) {
    int64_t ch[3] = {2 * c[0] + (b & 1), dim > 1 ? 2 * c[1] + ((b >> 1) & 1) : 0,
                     dim > 2 ? 2 * c[2] + ((b >> 2) & 1) : 0};
    next.insert(pack3(ch[0], ch[1], ch[2]), 0);
  }
}

void Forest::ensure_exists(int level, const int64_t* c) {
  if (exists(level, c)) return;
  int64_t p[3] = {c[0] >> 1, dim > 1 ? c[1] >> 1 : 0, dim > 2 ? c[2] >> 1 : 0};
  ensure_exists(level - 1, p);
  refine_cell(level - 1, p);
}

void Forest::close() {
  const int r2 = dim > 2 ? 1 : 0, r1 = dim > 1 ? 1 : 0;
  for (int l = (int)cells.size() - 1; l >= 1; --l) {
    std::vector<uint64_t> ref;
    cells[l].for_each([&](uint64_t k, int32_t v) {
      if (v) ref.push_back(k);
    });
    std::sort(ref.begin(), ref.end());
    for (uint64_t k : ref) {
      int64_t c[3];
      unpack3(k, c);
      for (int oz = -r2; oz <= r2; ++oz)
        for (int oy = -r1; oy <= r1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            int64_t n[3] = {c[0] + ox, c[1] + oy, c[2] + oz};
            if (inside(l, n) && !exists(l, n)) ensure_exists(l, n);
          }
    }
  }
}

static inline uint64_t spread_bits(uint64_t v, int dim) {
  // interleave: bit i of v goes to bit dim*i
  uint64_t out = 0;
  for (int i = 0; i < 21; ++i) out |= ((v >> i) & 1ull) << (dim * i);
  return out;
}

void Forest::rebuild_leaves() {
  int L = (int)cells.size() - 1;
  struct Item {
    uint64_t tree, morton;
    int32_t level;
    int64_t c[3];
  };
  std::vector<Item> items;
  for (int l = 0; l <= L; ++l) {
    cells[l].for_each([&](uint64_t k, int32_t v) {
      if (v) return;
      Item it;
      it.level = l;
      unpack3(k, it.c);
      int64_t t[3], loc[3];
      for (int d = 0; d < 3; ++d) {
        t[d] = it.c[d] >> l;
        loc[d] = (it.c[d] - (t[d] << l)) << (L - l);
      }
      it.tree = (uint64_t)(t[0] + (int64_t)n0[0] * (t[1] + (int64_t)n0[1] * t[2]));
      it.morton = spread_bits(loc[0], dim);
      if (dim > 1) it.morton |= spread_bits(loc[1], dim) << 1;
      if (dim > 2) it.morton |= spread_bits(loc[2], dim) << 2;
      items.push_back(it);
    });
  }
  std::sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
    return a.tree != b.tree ? a.tree < b.tree : a.morton < b.morton;
  });
  leaf_level.resize(items.size());
  leaf_coords.resize(3 * items.size());
  for (size_t i = 0; i < items.size(); ++i) {
    leaf_level[i] = items[i].level;
    for (int d = 0; d < 3; ++d) leaf_coords[3 * i + d] = items[i].c[d];
  }
}

}  // namespace gmg
