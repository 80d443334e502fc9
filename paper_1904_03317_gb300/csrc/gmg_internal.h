// Internal structures of the GB300 multigrid library (host side).
#pragma once

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gmg.h"

namespace gmg {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
struct Error {
  gmg_status status;
  std::string msg;
};

// ------------------------------------------------------------- hash map
// Open-addressing map from 64-bit keys to 32-bit values (keys != ~0).
struct HashMap64 {
  std::vector<uint64_t> keys;
  std::vector<int32_t> vals;
  uint64_t mask = 0;
  size_t count = 0;
  static constexpr uint64_t kEmpty = ~0ull;

  HashMap64() { rehash(16); }
  static uint64_t mix(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
  }
  void rehash(size_t cap) {
    size_t n = 16;
    while (n < cap) n <<= 1;
    std::vector<uint64_t> ok = std::move(keys);
    std::vector<int32_t> ov = std::move(vals);
    keys.assign(n, kEmpty);
    vals.assign(n, 0);
    mask = n - 1;
    count = 0;
    for (size_t i = 0; i < ok.size(); ++i)
      if (ok[i] != kEmpty) insert(ok[i], ov[i]);
  }
  void reserve(size_t n) {
    if (2 * n > keys.size()) rehash(2 * n);
  }
  const int32_t* find(uint64_t k) const {
    uint64_t i = mix(k) & mask;
    while (true) {
      if (keys[i] == k) return &vals[i];
      if (keys[i] == kEmpty) return nullptr;
      i = (i + 1) & mask;
    }
  }
  int32_t* find(uint64_t k) {
    return const_cast<int32_t*>(static_cast<const HashMap64*>(this)->find(k));
  }
  // inserts if absent; returns pointer to the value and whether it was new
  std::pair<int32_t*, bool> insert(uint64_t k, int32_t v) {
    if (2 * (count + 1) > keys.size()) rehash(2 * keys.size());
    uint64_t i = mix(k) & mask;
    while (true) {
      if (keys[i] == k) return {&vals[i], false};
      if (keys[i] == kEmpty) {
        keys[i] = k;
        vals[i] = v;
        ++count;
        return {&vals[i], true};
      }
      i = (i + 1) & mask;
    }
  }
  template <class F>
  void for_each(F&& f) const {
    for (size_t i = 0; i < keys.size(); ++i)
      if (keys[i] != kEmpty) f(keys[i], vals[i]);
  }
};

// Radix sort of 64-bit keys (OpenMP), ascending.
void parallel_sort_u64(std::vector<uint64_t>& v);

// Cell lattice coordinates packed into 64 bits (21 bits each).
inline uint64_t pack3(int64_t x, int64_t y, int64_t z) {
  return (uint64_t)x | ((uint64_t)y << 21) | ((uint64_t)z << 42);
}
inline void unpack3(uint64_t k, int64_t* c) {
  c[0] = (int64_t)(k & 0x1FFFFF);
  c[1] = (int64_t)((k >> 21) & 0x1FFFFF);
  c[2] = (int64_t)(k >> 42);
}

// ------------------------------------------------------------------ forest
struct Forest {
  int dim = 3;
  int n0[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  // one byte per coarse cell (x fastest), nonzero if it belongs to the
  // domain; empty: the whole brick
  std::vector<uint8_t> present;
  bool coarse_present(const int64_t* cc) const {
    return present.empty() || present[cc[0] + (int64_t)n0[0] * (cc[1] + (int64_t)n0[1] * cc[2])] != 0;
  }
  // per level: packed coords -> 1 if refined (has children), 0 if leaf
  std::vector<HashMap64> cells;
  // leaf list in canonical order, rebuilt after each refinement
  std::vector<int32_t> leaf_level;
  std::vector<int64_t> leaf_coords;  // 3 per leaf

  void init(const gmg_coarse_mesh& cm);
  bool inside(int level, const int64_t* c) const;
  bool exists(int level, const int64_t* c) const;
  bool refined(int level, const int64_t* c) const;
  // one lookup: -1 if the cell does not exist (or lies outside), 0 for a
  // leaf, 1 for a refined cell
  int state(int level, const int64_t* c) const;
  void refine_cell(int level, const int64_t* c);
  void ensure_exists(int level, const int64_t* c);
  void close();
  void rebuild_leaves();
  int num_levels() const { return (int)cells.size(); }
};

// --------------------------------------------------------- level (host)
// Level l >= 1 is stored by sibling groups: the 2^d children of one refined
// cell of level l-1.  Group g owns the (2k)^d nodes of its (2k+1)^d node
// block with local index < 2k in every direction; the nodes with local
// index 2k belong to the +1 neighbour group's block.  Blocks of neighbour
// positions that are not refined but inside the domain ("ghost" blocks)
// store refinement-edge nodes.
struct LevelHost {
  int level = 0;
  int64_t n_groups = 0, n_ghosts = 0;
  std::vector<int32_t> nbr;         // n_groups x 3^d slots of neighbour blocks (-1 outside)
  std::vector<uint64_t> state;      // n_groups: 2 bits per 3^d offset + child bits
  std::vector<double> coeff;        // n_groups: a of the group's cells
  std::vector<uint64_t> smask;      // n_groups: bit i set if stored node i is an S node
  std::vector<double> lcoef;        // n_groups x 2^d: a of the groups at offsets {-1,0}^d (0 if not refined)
  // groups whose refined lower neighbours all share the group's coefficient
  // (one merged tensor product suffices), and the rest
  std::vector<int32_t> list_uniform, list_jump;
  // 2x2x2 bricks of uniform groups sharing one coefficient (3D): per brick the
  // 4^3 block indices of positions -1..2 around it (own groups at 0..1).  The
  // first n_bricks_full are full (eight member groups); the rest are partial
  // bricks, smoothed only, whose members are marked in brick_members (bit
  // bx + 2 by + 4 bz).  list_uniform then holds only the uniform groups
  // outside bricks.
  std::vector<int32_t> bricks;
  int64_t n_bricks_full = 0;
  std::vector<uint8_t> brick_members;  // per partial brick
  // groups outside full bricks (all groups when there are none), increasing
  std::vector<int32_t> list_rest;

  // prolongation write masks over the group's (2k+1)^d nodes (2 x 64 bits):
  // add = stored S nodes (u += P uc), set = I nodes this group writes
  std::vector<uint64_t> pmask;      // n_groups x 4: add[0], add[1], set[0], set[1]
  std::vector<int32_t> parent;      // n_groups: parent's group at l-1 (or coarse cell at l=1)
  std::vector<int64_t> block_pos;   // (n_groups + n_ghosts) x 3: parent-lattice position
  std::vector<int8_t> slot_class;   // 0 unused, 1 S, 2 I, 3 D
  std::vector<int64_t> slot_key;    // node key per slot (-1 unused)
  uint64_t n_cells = 0, n_leaves = 0, n_S = 0, n_I = 0, n_S_jump = 0;
};

enum : int { kStateRefined = 0, kStateGhost = 1, kStateOutside = 2 };

struct ActiveHost {
  int64_t n_unknowns = 0;
  std::vector<int64_t> unknown_keys;
  std::vector<int32_t> home_level;
  std::vector<int64_t> home_slot;   // slot within the home level
  std::vector<uint32_t> home_global;  // slot in the concatenated level vector
  // leaf cells
  int64_t n_cells = 0;
  std::vector<int32_t> cell_nodes;  // n_cells x (k+1)^d: >=0 unknown, -1 Dirichlet, <=-2 hanging
  std::vector<double> cell_coeff;
  std::vector<uint8_t> cell_level;
  std::vector<int32_t> cell_coords;  // 3 per cell (for rhs quadrature)
  // hanging constraints (CSR over hanging rows)
  std::vector<int64_t> hang_key;
  std::vector<int32_t> hang_ptr;
  std::vector<int32_t> hang_col;
  std::vector<double> hang_w;
  std::vector<int64_t> hang_master_key;  // for export (Dirichlet masters dropped)
  // the same constraints by master: unknown hm_node[i] is a master of the
  // hanging rows hm_hang[hm_ptr[i] .. hm_ptr[i+1]) with weights hm_w
  std::vector<int32_t> hm_node, hm_ptr, hm_hang;
  std::vector<double> hm_w;
  int64_t n_leaf_nodes = 0;
  // leaf sibling groups: refined parents whose 2^d children are all leaves;
  // node table over the group's (2k+1)^d nodes, same encoding as cell_nodes
  int64_t n_groups = 0;
  std::vector<int32_t> grp_nodes;
  std::vector<double> grp_coeff;
  std::vector<uint8_t> grp_level;
  // leaf patches: cells whose 4^d grandchildren are all leaves, node table
  // over the patch's (4k+1)^d nodes; their cells are in no group
  int64_t n_patches = 0;
  std::vector<int32_t> pat_nodes;
  std::vector<double> pat_coeff;
  std::vector<uint8_t> pat_level;
  std::vector<int32_t> loose_cells;  // leaf cells in neither a patch nor a full group
  // the same cells as contiguous (k+1)^d node tables, coefficients and levels
  std::vector<int32_t> loose_nodes;
  std::vector<double> loose_coeff;
  std::vector<uint8_t> loose_level;
};

struct DeviceState;  // defined in the CUDA translation units

struct Hier {
  gmg_ctx* ctx = nullptr;
  int dim = 3, k = 2;
  int L = 0;  // finest level
  int n0[3] = {1, 1, 1};
  double lo[3], hi[3];
  gmg_params params;
  std::vector<double> fixed_lambda;
  std::vector<double> coarse_coeff;
  std::vector<LevelHost> levels;  // index 0: coarse lattice (only slot tables)
  std::vector<int64_t> level_offset;  // start of each level in the concatenated vectors
  int64_t total_slots = 0;
  ActiveHost active;
  // coarse level: lattice (k n0 + 1)^d; interior nodes are the unknowns of A_0
  int64_t coarse_lattice[3] = {1, 1, 1};
  int64_t n_coarse = 0;
  std::vector<int32_t> coarse_slots;   // level-0 slot of each coarse unknown (in slot order)
  std::vector<double> coarse_inverse;  // n_coarse^2, row-major: A_0^-1, or the Chebyshev coarse operator
  // unpreconditioned CG coarse solver: A_0 in CSR
  std::vector<int32_t> coarse_ptr, coarse_col;
  std::vector<double> coarse_val;
  int coarse_degree = 0;
  double coarse_range[2] = {0, 0};
  bool coarse_too_large = false;
  double setup_phase_s[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // the chosen coarse solver does not take this many unknowns
  std::vector<double> lambda;          // per level
  double setup_host_s = 0, setup_device_s = 0;
  DeviceState* dev = nullptr;
  // device address of the library's static smoothing scratch array, looked up
  // in this hierarchy's context when it is built (noalloc.cu)
  void* noalloc_scratch = nullptr;
};

struct Ctx {
  int device = -1;
  void* stream = nullptr;
};

// host builder (hierarchy.cpp)
void build_host_hierarchy(Hier& h, const Forest& f);
// 1-D reference matrices of degree k on [0, 1] (mass, stiffness) and the
// embedding of the parent's basis into the two children's nodes.
void reference_1d(int k, std::vector<double>& M, std::vector<double>& K, std::vector<double>& E);
// dense SPD inverse via Cholesky (returns false if not SPD)
bool spd_inverse(std::vector<double>& A, int64_t n);
// Chebyshev-Jacobi coarse operator of Sec. 4.1 (dense, row-major): the linear
// map g -> u of the iteration from zero; sets degree and range
void chebyshev_coarse_operator(const std::vector<double>& A, int64_t n, double tol, std::vector<double>& C,
                               int& degree, double range[2]);
double tridiag_max_eig(const std::vector<double>& diag, const std::vector<double>& off);

// device side (device.cu)
gmg_status device_setup(Hier& h);
void device_free(Hier& h);
gmg_status device_apply(Hier& h, const double* x, double* y);
gmg_status device_vcycle(Hier& h, const double* r, double* z);
gmg_status device_solve(Hier& h, const double* b, double* x, double tol, int max_iter,
                        int fixed_iterations, gmg_stats* st);
gmg_status device_rhs(Hier& h, int kind, uint64_t seed, double* b);
gmg_status device_solve_async(Hier& h, const double* b, double* x, double tol, int max_iter);
gmg_status device_solve_poll(Hier& h, int wait, int* ready, gmg_stats* st, gmg_status* status);
gmg_status device_solve_batch(Hier* const* hs, const double* const* b, double* const* x, int n, double tol,
                              int max_iter, int n_streams, gmg_stats* st, gmg_status* status);
gmg_status device_level_apply(Hier& h, int level, const void* x, void* y);
gmg_status device_level_residual_restrict(Hier& h, int level, const void* u, const void* g,
                                          void* gc);
gmg_status device_level_prolongate(Hier& h, int level, const void* uc, void* u, void* u2);
gmg_status device_level_smooth(Hier& h, int level, const void* g, void* u, void* tmp,
                               int from_zero);
gmg_status device_level_inv_diag(Hier& h, int level, void* out);
gmg_status device_coarse_solve(Hier& h, const void* g0, void* u0);
// looks up the static scratch array of gmg_level_smooth_noalloc in the current
// context (loading the module that holds it) and keeps its address in h
gmg_status noalloc_prepare(Hier& h);
uint64_t device_bytes(const Hier& h);
void profile_reset(Hier& h, bool timing);
void profile_read(Hier& h, gmg_kernel_stats* out);

}  // namespace gmg

struct gmg_ctx {
  gmg::Ctx c;
};
struct gmg_mesh {
  gmg::Forest f;
};
struct gmg_hier {
  gmg::Hier h;
};
