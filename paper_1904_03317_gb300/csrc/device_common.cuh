// Device-side declarations shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gmg_internal.h"

namespace gmg {

#define GMG_CUDA_TRY(expr)                                                         \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error(std::string("CUDA error: ") + cudaGetErrorString(e_) + " at " +    \
                __FILE__ + ":" + std::to_string(__LINE__));                        \
      return GMG_ECUDA;                                                            \
    }                                                                              \
  } while (0)

// Kernels launched by this thread: every launch site counts itself, and the
// launch accounting attributes the launches made inside one accounting scope
// to that scope's kind.
extern thread_local uint64_t g_kernel_launches;
#define GMG_COUNT_LAUNCH() (++::gmg::g_kernel_launches)

// Per-level device data (level l >= 1 is stored by sibling groups).
struct LevelDev {
  int64_t n_groups = 0;
  int64_t n_slots = 0;
  int64_t offset = 0;           // in the concatenated level vectors
  // the V-cycle zeroes the level's smoother vectors before each down-sweep:
  // level 0 and levels with refinement-edge (I) nodes or ghost blocks
  bool zero_each_cycle = true;
  int32_t* nbr = nullptr;       // n_groups x 3^d
  uint64_t* state = nullptr;    // n_groups
  double* coeff = nullptr;      // n_groups
  int32_t* parent = nullptr;    // n_groups
  uint64_t* smask = nullptr;    // n_groups
  double* lcoef64 = nullptr;    // n_groups x 2^d
  float* lcoef32 = nullptr;     // n_groups x 2^d
  float* coeff32 = nullptr;     // n_groups
  int32_t* list_uniform = nullptr;
  int32_t* list_jump = nullptr;
  uint64_t* pmask = nullptr;    // n_groups x 4
  int32_t* bricks = nullptr;    // n_bricks_all x 64: full bricks, then partial ones
  int64_t n_bricks = 0;         // full bricks
  int64_t n_bricks_all = 0;
  uint8_t* brick_members = nullptr;  // per partial brick: member positions
  // per brick (full and partial): x = member bits 0..7 | kBrickAllS, y = the
  // bits of the bricks' FP32 coefficient
  uint2* brick_info = nullptr;
  // per full brick (levels >= 2): the level l-1 neighbour row of the parent
  // group of its eight groups, so that the transfer kernels need not chase
  // parent -> neighbour table
  int32_t* brick_cnb = nullptr;
  int32_t* group_cnb = nullptr;  // the same per group (levels >= 2)
  bool iso = false;             // cubic cells: one scale factor for all directions
  int32_t* list_rest = nullptr; // groups outside full bricks
  int64_t n_rest = 0;
  // deterministic mode: full bricks ordered by colour (offsets into them),
  // and every group of the level in a list ordered by colour (offsets); one
  // colour's bricks or groups share no coarse node
  std::vector<int64_t> brick_off, group_off;
  int32_t* list_color = nullptr;
  int64_t n_uniform = 0, n_jump = 0;
  double scale[3] = {0, 0, 0};  // K-term factor per direction: prod_{j!=i} h_j / h_i
  // Chebyshev parameters (host)
  double lambda = 0, theta = 0, delta = 0, sigma = 0;
  // accounting: S and I nodes, FP operations of one smoothing launch
  double n_S = 0, n_I = 0, n_S_jump = 0, cheb_flops = 0;
};

// Arguments of the level kernels, passed by value.
struct LevelArgs {
  int64_t n_groups;
  const int32_t* nbr;
  const uint64_t* state;
  const double* coeff;
  const float* coeff32;
  const uint64_t* smask;
  const double* lcoef64;
  const float* lcoef32;
  const int32_t* parent;
  const int32_t* list_uniform;
  const int32_t* list_jump;
  const uint64_t* pmask;
  const int32_t* bricks;
  int64_t n_bricks;           // full bricks (smoothing, residual, prolongation)
  int64_t n_bricks_all;       // with the partial bricks (smoothing only)
  const uint8_t* brick_members;
  const uint2* brick_info;    // per brick: member bits | kBrickAllS, coefficient bits
  const int32_t* brick_cnb;   // per full brick: parent group's 27 level l-1 neighbours (l >= 2)
  const int32_t* group_cnb;   // per group: its parent group's level l-1 neighbours (l >= 2)
  bool iso;                   // s_x = s_y = s_z (cubic cells)
  const int32_t* list_rest;
  int64_t n_rest;
  bool no_ghosts;             // the level has no refinement-edge (ghost) blocks
  // deterministic mode (host-side launch data): restriction launches one
  // colour at a time and adds without atomics
  bool deterministic;
  const int64_t* brick_off;   // n_brick_colors + 1 offsets into the full bricks
  int n_brick_colors;
  const int32_t* list_color;  // all groups, ordered by colour
  const int64_t* group_off;   // n_group_colors + 1 offsets into list_color
  int n_group_colors;
  int64_t n_uniform, n_jump;
  const int32_t* nbr_coarse;  // level l-1 neighbour table (l >= 2)
  int64_t coarse_lat[3];      // coarse lattice extents (l == 1)
  double scale[3];
  float scale32[3];
  int level;
};

// Launch accounting (gmg_profile_*).
struct Profile {
  uint64_t launches[GMG_NUM_KERNEL_KINDS] = {};
  double ms[GMG_NUM_KERNEL_KINDS] = {};
  double bytes[GMG_NUM_KERNEL_KINDS] = {};
  double flops[GMG_NUM_KERNEL_KINDS] = {};
  bool timing = false;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
};

// Launch counts of a captured graph section, added to Profile per execution.
struct Tally {
  uint64_t launches[GMG_NUM_KERNEL_KINDS] = {};
  double bytes[GMG_NUM_KERNEL_KINDS] = {};
  double flops[GMG_NUM_KERNEL_KINDS] = {};
};

// Scalars and loop control of the graph-mode CG, in device memory.
struct GraphCtl {
  double bb;      // b.b
  double rz_old;  // r_{i-1}.z_{i-1} (1 before the first iteration, where p = 0)
  double rz;      // r_i.z_i
  double pAp;     // p_i.A p_i
  double rr;      // r_{i+1}.r_{i+1}
  double tol;     // relative tolerance
  int it;         // completed iterations
  int limit;      // iteration limit
  int fixed;      // > 0: run exactly this many iterations
  int status;     // GraphStatus
};
enum GraphStatus { GS_RUNNING = 0, GS_DONE = 1, GS_NOTCONV = 2, GS_NAN = 3, GS_BREAKDOWN = 4 };

struct DeviceState {
  cudaStream_t stream = nullptr;
  Profile prof;
  int prec = GMG_PREC_FP32;
  size_t bytes = 0;
  std::vector<LevelDev> lv;
  // concatenated level vectors in the V-cycle precision
  void* uA = nullptr;
  void* uB = nullptr;
  void* g = nullptr;
  void* dinv = nullptr;
  // coarse level
  int32_t* coarse_slot = nullptr;  // level-0 slot of each coarse unknown
  double* coarse_inv = nullptr;  // n_coarse^2
  int64_t coarse_nnz = 0;         // CG coarse solver: A_0 in CSR
  int32_t* coarse_ptr = nullptr;
  int32_t* coarse_col = nullptr;
  double* coarse_val = nullptr;
  int64_t n_coarse = 0;
  int64_t coarse_lat[3] = {1, 1, 1};
  // active (leaf) mesh
  int64_t n_unknowns = 0, n_cells = 0;
  int32_t* cell_nodes = nullptr;
  double* cell_coeff = nullptr;
  uint8_t* cell_level = nullptr;
  int32_t* cell_coords = nullptr;
  int32_t* loose = nullptr;
  int64_t n_loose = 0, n_grp = 0;
  int32_t* grp_nodes = nullptr;
  double* grp_coeff = nullptr;
  uint8_t* grp_level = nullptr;
  int32_t* loose_nodes = nullptr;
  double* loose_coeff = nullptr;
  uint8_t* loose_level = nullptr;
  int64_t n_pat = 0;
  int32_t* pat_nodes = nullptr;
  double* pat_coeff = nullptr;
  uint8_t* pat_level = nullptr;
  int32_t* hang_ptr = nullptr;
  int32_t* hang_col = nullptr;
  // constraint weights as 1-byte codes into a table of the distinct values
  // (a handful for Q1 and Q2 on 2:1 meshes)
  uint8_t* hang_wc = nullptr;
  double* hw_table = nullptr;
  int n_hw = 0;
  int64_t n_hang = 0, n_masters = 0;
  double* xh = nullptr;
  double* yh = nullptr;
  int32_t* hm_node = nullptr;
  int32_t* hm_ptr = nullptr;
  int32_t* hm_hang = nullptr;
  uint8_t* hm_wc = nullptr;
  uint32_t* home = nullptr;
  // The device numbers the unknowns in the order of their home slots, so that
  // the copies between active and level vectors and the leaf operator's
  // gathers touch memory in order; perm[j] is the canonical index of internal
  // unknown j.  Every table on the device (home, leaf node tables, hanging
  // constraints) uses the internal numbering; the entry points convert the
  // caller's canonical vectors on the way in and out.
  int32_t* perm = nullptr;
  // deterministic mode: colour offsets of the patch, group and single-cell
  // tables (each ordered by colour)
  std::vector<int64_t> pat_off, grp_off, loose_off;
  double level_scale[GMG_MAX_LEVELS][3];  // leaf-cell operator factors per level
  double cell_h[GMG_MAX_LEVELS][3];       // cell sizes per level
  // CG work vectors
  double* r = nullptr;
  double* p = nullptr;
  double* Ap = nullptr;
  // reductions
  double* partials = nullptr;     // kMaxReduceBlocks
  unsigned* counter = nullptr;
  double* scal = nullptr;         // device scalars (see ScalarSlot)
  double* scal_host = nullptr;    // pinned mirror
  int max_scal = 0;
  double active_flops = 0, active_bytes = 0;  // per leaf-operator launch
  // graph-mode CG, built by the first graph-mode solve
  Tally* cap = nullptr;            // non-null while a graph section is captured
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t cg_graph = nullptr;
  cudaGraphExec_t cg_exec = nullptr;
  Tally cg_pre, cg_body;           // launches before the loop and per loop pass
  double* x_iter = nullptr;        // iterate of the graph-mode CG
  GraphCtl* ctl = nullptr;
  GraphCtl* ctl_host = nullptr;    // pinned mirror
  cudaEvent_t done = nullptr;      // end of the pending asynchronous solve
  bool async_pending = false;
  double async_tol = 0.0;
};

constexpr int kMaxReduceBlocks = 4096;
// brick_info flag: every stored node of every member group is an S node
constexpr unsigned kBrickAllS = 1u << 8;

// ------------------------------------------------------------ launchers
// Level kernels (kernels_level.cu).  T = float or double; all pointers are
// level-local (already offset to the level's first slot) unless noted.
template <typename T>
cudaError_t launch_level_cheb(int dim, int k, const LevelArgs& a, const T* x, const T* xprev,
                              const T* g, const T* dinv, T* out, T c1, T c2, bool apply_only,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_level_residual_restrict(int dim, int k, const LevelArgs& a, const T* u,
                                           const T* g, T* gc, cudaStream_t s);
template <typename T>
cudaError_t launch_level_prolongate(int dim, int k, const LevelArgs& a, const T* uc, T* u, T* u2,
                                    cudaStream_t s);
cudaError_t launch_level_diag(int dim, int k, const LevelArgs& a, double* diag_inv,
                              cudaStream_t s);

// Active mesh and vector kernels (kernels_active.cu).
struct ActiveArgs {
  int64_t n_cells;
  const int32_t* cell_list;  // optional: process only these cells (n_list of them)
  int64_t n_list;
  int64_t n_groups;          // full leaf sibling groups
  const int32_t* grp_nodes;
  const double* grp_coeff;
  const uint8_t* grp_level;
  const int32_t* loose_nodes;  // the cell_list cells as contiguous tables
  const double* loose_coeff;
  const uint8_t* loose_level;
  int64_t n_patches;         // leaf patches (4^d cells)
  const int32_t* pat_nodes;
  const double* pat_coeff;
  const uint8_t* pat_level;
  const int32_t* cell_nodes;
  const double* cell_coeff;
  const uint8_t* cell_level;
  const int32_t* hang_ptr;
  const int32_t* hang_col;
  const uint8_t* hang_wc;    // weight of each entry: hw_table[code]
  const double* hw_table;    // n_hw distinct constraint weights
  int n_hw;
  int64_t n_hang;
  double* xh;                // hanging-node values of the operand
  double* yh;                // contributions to hanging nodes
  int64_t n_masters;         // unknowns that are masters of hanging nodes
  const int32_t* hm_node;    // their unknown indices
  const int32_t* hm_ptr;     // n_masters + 1
  const int32_t* hm_hang;    // hanging node of each entry
  const uint8_t* hm_wc;      // its weight's code
  // deterministic mode: shared nodes are added to without atomics, one
  // colour of patches, groups and single cells per launch (offsets into the
  // colour-ordered tables; host-side launch data)
  bool deterministic;
  const int64_t* pat_off;
  int n_pat_colors;
  const int64_t* grp_off;
  int n_grp_colors;
  const int64_t* loose_off;
  int n_loose_colors;
  // per-level factors of the hierarchy (kernel parameters, so hierarchies
  // that live side by side never share them)
  double scale[GMG_MAX_LEVELS][3];  // s_i = prod_{j != i} h_j / h_i
  double h[GMG_MAX_LEVELS][3];      // cell sizes
  double lo[3];                     // brick origin
};
cudaError_t launch_active_apply(int dim, int k, const ActiveArgs& a, const double* x, double* y,
                                double* partials, unsigned* counter, double* energy_out,
                                cudaStream_t s);
// b = C^T int f phi_i with f = d pi^2 prod sin(pi x_i), or f = 1 if `one`
cudaError_t launch_rhs_sine(int dim, int k, const ActiveArgs& a, const int32_t* cell_coords,
                            double* b, bool one, cudaStream_t s);
// b_i = U[-1, 1) from SplitMix64 keyed by (seed, canonical index i)
cudaError_t launch_rhs_random(int64_t n, uint64_t seed, double* b, cudaStream_t s);
template <typename T>
cudaError_t launch_copy_to_mg(int64_t n, const double* r, const uint32_t* home, T* g,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_copy_from_mg(int64_t n, const T* u, const uint32_t* home, const double* r,
                                double* z, double* partials, unsigned* counter, double* rz_out,
                                cudaStream_t s);
// Coarse solves on the coarse unknowns, which sit at the level-0 slots
// `slot` (the interior nodes of the coarse lattice, or those of the present
// coarse cells' union).
template <typename T>
cudaError_t launch_coarse_solve(int64_t n_coarse, const int32_t* slot, const double* inv, const T* g0, T* u0,
                                cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_cg(int64_t nc, const int32_t* slot, const int32_t* ptr, const int32_t* col,
                             const double* val, int64_t nnz, double tol, const T* g0, T* u0, cudaStream_t s);
template <typename T>
cudaError_t launch_scale_vec(int64_t n, const T* dinv, const T* g, T c, T* out, cudaStream_t s);
cudaError_t launch_dot(int64_t n, const double* a, const double* b, double* partials,
                       unsigned* counter, double* out, cudaStream_t s);
// Canonical <-> internal unknown order: dst[j] = src[perm[j]] (gather) or
// dst[perm[j]] = src[j] (scatter).
cudaError_t launch_perm(int64_t n, const int32_t* perm, const double* src, double* dst, bool scatter,
                        cudaStream_t s);
// The outer CG's streaming passes, fused with the active <-> level copies
// (z_i = u[home_i] is never stored): r = b with b.b and the first level
// right-hand sides; r.z; p = z + (rz_new / rz_old) p with Ap = 0; and x += a
// p, r -= a Ap with r.r and the next level right-hand sides (a = rz / pAp).
template <typename T>
cudaError_t launch_cg_start(int64_t n, const double* b, const uint32_t* home, double* r, T* g, double* partials,
                            unsigned* counter, double* bb_out, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_rz(int64_t n, const T* u, const uint32_t* home, const double* r, double* partials,
                         unsigned* counter, double* rz_out, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_p(int64_t n, const T* u, const uint32_t* home, double* p, double* Ap, const double* rz_new,
                        const double* rz_old, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_xr(int64_t n, double* x, double* r, const double* p, const double* Ap, const uint32_t* home,
                         T* g, const double* rz, const double* pAp, double* partials, unsigned* counter,
                         double* rr_out, cudaStream_t s);
// Loop control of the graph-mode CG: `init` starts the loop when b.b > 0,
// `check` counts an iteration, applies the stopping rules and sets the loop
// condition.
cudaError_t launch_cg_graph_init(GraphCtl* c, cudaGraphConditionalHandle loop, cudaStream_t s);
cudaError_t launch_cg_graph_check(GraphCtl* c, cudaGraphConditionalHandle loop, cudaStream_t s);
cudaError_t launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s);
cudaError_t launch_mul(int64_t n, const double* a, const double* b, double* out, cudaStream_t s);
cudaError_t launch_xpay(int64_t n, const double* x, double beta, double* y, cudaStream_t s);
cudaError_t launch_convert_d2f(int64_t n, const double* in, float* out, cudaStream_t s);

}  // namespace gmg
