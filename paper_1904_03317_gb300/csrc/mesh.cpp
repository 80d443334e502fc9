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
#include <omp.h>

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
  const size_t nc = (size_t)n0[0] * n0[1] * n0[2];
  present.clear();
  if (cm.present) present.assign(cm.present, cm.present + nc);
  cells.assign(1, HashMap64());
  cells[0].reserve(nc);
  for (int64_t z = 0; z < n0[2]; ++z)
    for (int64_t y = 0; y < n0[1]; ++y)
      for (int64_t x = 0; x < n0[0]; ++x) {
        const int64_t c[3] = {x, y, z};
        if (coarse_present(c)) cells[0].insert(pack3(x, y, z), 0);
      }
  rebuild_leaves();
}

// A lattice cell of level l lies in the domain if it is inside the brick and
// its coarse ancestor is present.
bool Forest::inside(int level, const int64_t* c) const {
  int64_t cc[3];
  for (int d = 0; d < 3; ++d) {
    int64_t ext = d < dim ? ((int64_t)n0[d] << level) : 1;
    if (c[d] < 0 || c[d] >= ext) return false;
    cc[d] = d < dim ? c[d] >> level : 0;
  }
  return coarse_present(cc);
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

int Forest::state(int level, const int64_t* c) const {
  if (level >= (int)cells.size() || !inside(level, c)) return -1;
  const int32_t* v = cells[level].find(pack3(c[0], c[1], c[2]));
  return v ? (*v ? 1 : 0) : -1;
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

// Keys of the cells of one level whose value satisfies `pick`, collected
// over the hash table's slots in parallel (in slot order).
template <class P>
static std::vector<uint64_t> collect_keys(const HashMap64& m, P pick) {
  const int nt = omp_get_max_threads();
  std::vector<std::vector<uint64_t>> part(nt);
  const size_t n = m.keys.size();
#pragma omp parallel num_threads(nt)
  {
    const int t = omp_get_thread_num();
    const size_t b = n * t / nt, e = n * (t + 1) / nt;
    for (size_t i = b; i < e; ++i)
      if (m.keys[i] != HashMap64::kEmpty && pick(m.vals[i])) part[t].push_back(m.keys[i]);
  }
  std::vector<uint64_t> out;
  for (auto& v : part) out.insert(out.end(), v.begin(), v.end());
  return out;
}

void Forest::close() {
  const int r2 = dim > 2 ? 1 : 0, r1 = dim > 1 ? 1 : 0;
  for (int l = (int)cells.size() - 1; l >= 1; --l) {
    // lattice neighbours of refined cells that do not exist yet (found in
    // parallel on the unchanged level), then created one by one; a created
    // cell is a leaf, so the level's refined set is final when the scan runs
    const std::vector<uint64_t> ref = collect_keys(cells[l], [](int32_t v) { return v != 0; });
    const int nt = omp_get_max_threads();
    std::vector<std::vector<uint64_t>> miss(nt);
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t i = 0; i < (int64_t)ref.size(); ++i) {
      int64_t c[3];
      unpack3(ref[i], c);
      for (int oz = -r2; oz <= r2; ++oz)
        for (int oy = -r1; oy <= r1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            int64_t n[3] = {c[0] + ox, c[1] + oy, c[2] + oz};
            if (inside(l, n) && !exists(l, n)) miss[omp_get_thread_num()].push_back(pack3(n[0], n[1], n[2]));
          }
    }
    std::vector<uint64_t> all;
    for (auto& v : miss) all.insert(all.end(), v.begin(), v.end());
    parallel_sort_u64(all);
    all.erase(std::unique(all.begin(), all.end()), all.end());
    for (uint64_t k : all) {
      int64_t n[3];
      unpack3(k, n);
      ensure_exists(l, n);
    }
  }
}

// bit i of v to bit 3i (v < 2^21) and back; bit i to bit 2i (v < 2^32) and back
static inline uint64_t part1by2(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}
static inline uint64_t compact1by2(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return x;
}
static inline uint64_t part1by1(uint64_t x) {
  x &= 0xffffffffull;
  x = (x | x << 16) & 0x0000ffff0000ffffull;
  x = (x | x << 8) & 0x00ff00ff00ff00ffull;
  x = (x | x << 4) & 0x0f0f0f0f0f0f0f0full;
  x = (x | x << 2) & 0x3333333333333333ull;
  x = (x | x << 1) & 0x5555555555555555ull;
  return x;
}
static inline uint64_t compact1by1(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x ^ (x >> 1)) & 0x3333333333333333ull;
  x = (x ^ (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
  x = (x ^ (x >> 4)) & 0x00ff00ff00ff00ffull;
  x = (x ^ (x >> 8)) & 0x0000ffff0000ffffull;
  x = (x ^ (x >> 16)) & 0x00000000ffffffffull;
  return x;
}

static inline uint64_t spread_bits(uint64_t v, int dim) {
  // interleave: bit i of v goes to bit dim*i
  uint64_t out = 0;
  for (int i = 0; i < 21; ++i) out |= ((v >> i) & 1ull) << (dim * i);
  return out;
}

void Forest::rebuild_leaves() {
  int L = (int)cells.size() - 1;
  // Canonical order: coarse cell (tree) index, then Morton (z-order) index
  // of the lower corner on the finest lattice.  When tree, Morton index and
  // level fit in one 64-bit key, the leaves are radix-sorted by it in
  // parallel; the key of a leaf is unique, since leaves do not overlap.
  {
    const uint64_t ntree = (uint64_t)n0[0] * n0[1] * n0[2];
    int tb = 1;
    while ((1ull << tb) < ntree) ++tb;
    const int mb = dim * L;
    if (dim >= 2 && tb + mb + 5 <= 64) {
      std::vector<uint64_t> keys;
      for (int l = 0; l <= L; ++l) {
        std::vector<uint64_t> lk = collect_keys(cells[l], [](int32_t v) { return v == 0; });
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)lk.size(); ++i) {
          int64_t c[3], t[3];
          unpack3(lk[i], c);
          uint64_t m = 0;
          for (int d = 0; d < dim; ++d) {
            t[d] = c[d] >> l;
            const uint64_t loc = (uint64_t)((c[d] - (t[d] << l)) << (L - l));
            m |= (dim == 3 ? part1by2(loc) : part1by1(loc)) << d;
          }
          const uint64_t tree = (uint64_t)(t[0] + (int64_t)n0[0] * ((dim > 1 ? t[1] : 0) +
                                                                     (int64_t)n0[1] * (dim > 2 ? t[2] : 0)));
          lk[i] = (((tree << mb) | m) << 5) | (uint64_t)l;
        }
        keys.insert(keys.end(), lk.begin(), lk.end());
      }
      parallel_sort_u64(keys);
      const int64_t n = (int64_t)keys.size();
      leaf_level.resize(n);
      leaf_coords.resize(3 * n);
      const uint64_t mmask = mb >= 64 ? ~0ull : ((1ull << mb) - 1);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        const int l = (int)(keys[i] & 31);
        const uint64_t m = (keys[i] >> 5) & mmask, tree = (keys[i] >> 5) >> mb;
        const int64_t t[3] = {(int64_t)(tree % (uint64_t)n0[0]), (int64_t)((tree / (uint64_t)n0[0]) % (uint64_t)n0[1]),
                              (int64_t)(tree / ((uint64_t)n0[0] * n0[1]))};
        leaf_level[i] = l;
        for (int d = 0; d < 3; ++d) {
          int64_t c = 0;
          if (d < dim) {
            const uint64_t loc = dim == 3 ? compact1by2(m >> d) : compact1by1(m >> d);
            c = (t[d] << l) + (int64_t)(loc >> (L - l));
          }
          leaf_coords[3 * i + d] = c;
        }
      }
      return;
    }
  }
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
