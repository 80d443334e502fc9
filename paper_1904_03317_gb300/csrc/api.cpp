// C ABI (include/gmg.h): argument checking, error reporting, ownership.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "gmg_internal.h"

namespace gmg {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace gmg

using namespace gmg;

#define GMG_GUARD_BEGIN try {
#define GMG_GUARD_END                              \
  }                                                \
  catch (const std::bad_alloc&) {                  \
    set_error("host allocation failed");           \
    return GMG_ENOMEM;                             \
  }                                                \
  catch (const std::exception& e) {                \
    set_error(e.what());                           \
    return GMG_EINVAL;                             \
  }                                                \
  catch (...) {                                    \
    set_error("unknown exception");                \
    return GMG_EINVAL;                             \
  }

#define CHECK_ARG(cond, msg)   \
  do {                         \
    if (!(cond)) {             \
      set_error(msg);          \
      return GMG_EINVAL;       \
    }                          \
  } while (0)

static gmg_status bind_device(const Hier& h) {
  if (!h.ctx || h.ctx->c.device < 0 || !h.dev) {
    set_error("this call needs a hierarchy built on a device context");
    return GMG_EINVAL;
  }
  cudaError_t e = cudaSetDevice(h.ctx->c.device);
  if (e != cudaSuccess) {
    set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return GMG_ECUDA;
  }
  return GMG_OK;
}

extern "C" {

const char* gmg_last_error(void) { return g_last_error.c_str(); }

gmg_status gmg_build_info(int* has_sm103a, int* version) {
  CHECK_ARG(has_sm103a && version, "null argument");
#if defined(GMG_BUILT_FOR_SM103A)
  *has_sm103a = 1;
#else
  *has_sm103a = 0;
#endif
  *version = 2;
  return GMG_OK;
}

gmg_status gmg_create(int device, void* cuda_stream, gmg_ctx** out) {
  CHECK_ARG(out, "out is null");
  *out = nullptr;
  GMG_GUARD_BEGIN
  if (device >= 0) {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device >= n) {
      set_error(std::string("no CUDA device ") + std::to_string(device) + ": " +
                (e != cudaSuccess ? cudaGetErrorString(e) : "index out of range"));
      return GMG_ECUDA;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) {
      set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
      return GMG_ECUDA;
    }
  } else if (device != -1) {
    set_error("device must be >= 0 or -1 (host-only)");
    return GMG_EINVAL;
  }
  gmg_ctx* c = new gmg_ctx();
  c->c.device = device;
  c->c.stream = cuda_stream;
  *out = c;
  return GMG_OK;
  GMG_GUARD_END
}

void gmg_destroy(gmg_ctx* ctx) { delete ctx; }

gmg_status gmg_mesh_create(const gmg_coarse_mesh* cm, gmg_mesh** out) {
  CHECK_ARG(cm && out, "null argument");
  *out = nullptr;
  CHECK_ARG(cm->dim == 2 || cm->dim == 3, "dim must be 2 or 3");
  for (int d = 0; d < cm->dim; ++d) {
    CHECK_ARG(cm->n0[d] >= 1 && cm->n0[d] <= 1024, "n0 out of range [1, 1024]");
    CHECK_ARG(std::isfinite(cm->lo[d]) && std::isfinite(cm->hi[d]) && cm->hi[d] > cm->lo[d],
              "need finite lo < hi");
  }
  if (cm->present) {
    const int64_t nc = (int64_t)cm->n0[0] * cm->n0[1] * (cm->dim == 3 ? cm->n0[2] : 1);
    bool any = false;
    for (int64_t i = 0; i < nc && !any; ++i) any = cm->present[i] != 0;
    CHECK_ARG(any, "at least one coarse cell must be present");
  }
  GMG_GUARD_BEGIN
  gmg_mesh* m = new gmg_mesh();
  m->f.init(*cm);
  *out = m;
  return GMG_OK;
  GMG_GUARD_END
}

void gmg_mesh_destroy(gmg_mesh* mesh) { delete mesh; }

gmg_status gmg_mesh_num_leaves(const gmg_mesh* mesh, uint64_t* n) {
  CHECK_ARG(mesh && n, "null argument");
  *n = mesh->f.leaf_level.size();
  return GMG_OK;
}

gmg_status gmg_mesh_num_levels(const gmg_mesh* mesh, int* n) {
  CHECK_ARG(mesh && n, "null argument");
  *n = mesh->f.num_levels();
  return GMG_OK;
}

gmg_status gmg_mesh_leaves(const gmg_mesh* mesh, int32_t* level, int32_t* coords) {
  CHECK_ARG(mesh && level && coords, "null argument");
  const Forest& f = mesh->f;
  for (size_t i = 0; i < f.leaf_level.size(); ++i) {
    level[i] = f.leaf_level[i];
    for (int d = 0; d < 3; ++d) coords[3 * i + d] = (int32_t)f.leaf_coords[3 * i + d];
  }
  return GMG_OK;
}

gmg_status gmg_mesh_partition_model(const gmg_mesh* mesh, int64_t n_parts, gmg_partition_model* out) {
  CHECK_ARG(mesh && out, "null argument");
  CHECK_ARG(n_parts >= 1 && n_parts < ((int64_t)1 << 31), "n_parts out of range");
  GMG_GUARD_BEGIN
  const Forest& f = mesh->f;
  const int L = f.num_levels();
  CHECK_ARG(L <= GMG_MAX_LEVELS, "too many levels");
  const int64_t nleaf = (int64_t)f.leaf_level.size();
  // owner of every cell, finest level first (first-child rule)
  std::vector<std::unordered_map<uint64_t, int64_t>> own(L);
  for (int64_t i = 0; i < nleaf; ++i) {
    const int64_t* c = &f.leaf_coords[3 * i];
    own[f.leaf_level[i]][pack3(c[0], c[1], c[2])] = (int64_t)((__int128)i * n_parts / nleaf);
  }
  std::memset(out, 0, sizeof(*out));
  out->n_levels = L;
  std::unordered_map<int64_t, int64_t> counts;
  for (int l = L - 1; l >= 0; --l) {
    f.cells[l].for_each([&](uint64_t k, int32_t refined) {
      if (!refined) return;
      int64_t c[3];
      unpack3(k, c);
      const int64_t first[3] = {2 * c[0], f.dim > 1 ? 2 * c[1] : 0, f.dim > 2 ? 2 * c[2] : 0};
      own[l][k] = own[l + 1].at(pack3(first[0], first[1], first[2]));
    });
    counts.clear();
    int64_t nl = 0, wl = 0;
    for (const auto& kv : own[l]) {
      wl = std::max(wl, ++counts[kv.second]);
      ++nl;
    }
    out->n_cells[l] = (double)nl;
    out->w_level[l] = (double)wl;
  }
  double tot = 0.0;
  for (int l = 0; l < L; ++l) {
    tot += out->n_cells[l];
    out->w_sync += std::ceil(out->n_cells[l] / (double)n_parts);
    out->w += out->w_level[l];
  }
  out->w_opt = tot / (double)n_parts;
  out->efficiency = out->w > 0 ? out->w_opt / out->w : 0.0;
  return GMG_OK;
  GMG_GUARD_END
}

gmg_status gmg_mesh_refine(gmg_mesh* mesh, const uint8_t* flags, uint64_t n_flags) {
  CHECK_ARG(mesh, "null mesh");
  Forest& f = mesh->f;
  CHECK_ARG(n_flags == f.leaf_level.size(), "n_flags must equal the number of leaves");
  CHECK_ARG(flags || n_flags == 0, "null flags");
  GMG_GUARD_BEGIN
  for (uint64_t i = 0; i < n_flags; ++i) {
    if (!flags[i]) continue;
    if (f.leaf_level[i] + 1 > 20) {
      set_error("refinement beyond level 20");
      return GMG_EINVAL;
    }
  }
  {
    // room for the children first: one rehash per level instead of a doubling cascade
    std::vector<uint64_t> per_level(f.cells.size() + 1, 0);
    for (uint64_t i = 0; i < n_flags; ++i)
      if (flags[i]) per_level[(size_t)f.leaf_level[i] + 1] += (uint64_t)1 << f.dim;
    for (size_t l = 1; l < per_level.size(); ++l) {
      if (!per_level[l]) continue;
      if (l == f.cells.size()) f.cells.emplace_back();
      f.cells[l].reserve(f.cells[l].count + per_level[l]);
    }
  }
  for (uint64_t i = 0; i < n_flags; ++i) {
    if (!flags[i]) continue;
    int64_t c[3] = {f.leaf_coords[3 * i], f.leaf_coords[3 * i + 1], f.leaf_coords[3 * i + 2]};
    f.refine_cell(f.leaf_level[i], c);
  }
  f.close();
  f.rebuild_leaves();
  return GMG_OK;
  GMG_GUARD_END
}

void gmg_params_default(gmg_params* p) {
  if (!p) return;
  p->cheb_degree = 5;
  p->eig_lo = 0.08;
  p->eig_hi = 1.2;
  p->eig_iters = 10;
  p->vcycle_prec = GMG_PREC_FP32;
  p->fixed_lambda = nullptr;
  p->smoother = GMG_SMOOTHER_CHEBYSHEV;
  p->coarse_solver = GMG_COARSE_CHOLESKY;
  p->coarse_tol = 1e-3;
  p->solve_graph = 1;
  p->deterministic = 0;
  p->brick_min_members = 0;
}

gmg_status gmg_hier_build(gmg_ctx* ctx, const gmg_mesh* mesh, int degree, const double* coarse_coeff,
                          const gmg_params* p, gmg_hier** out) {
  CHECK_ARG(ctx && mesh && out, "null argument");
  *out = nullptr;
  CHECK_ARG(degree == 1 || degree == 2, "degree must be 1 or 2");
  gmg_params prm;
  gmg_params_default(&prm);
  if (p) prm = *p;
  CHECK_ARG(prm.cheb_degree >= 1 && prm.cheb_degree <= 64, "cheb_degree out of range [1, 64]");
  CHECK_ARG(prm.eig_iters >= 1 && prm.eig_iters <= 1000, "eig_iters out of range");
  CHECK_ARG(prm.eig_lo > 0 && prm.eig_hi > prm.eig_lo, "need 0 < eig_lo < eig_hi");
  CHECK_ARG(prm.vcycle_prec == GMG_PREC_FP32 || prm.vcycle_prec == GMG_PREC_FP64, "bad vcycle_prec");
  CHECK_ARG(prm.smoother == GMG_SMOOTHER_CHEBYSHEV || prm.smoother == GMG_SMOOTHER_JACOBI, "bad smoother");
  CHECK_ARG(prm.coarse_solver == GMG_COARSE_CHOLESKY || prm.coarse_solver == GMG_COARSE_CHEBYSHEV ||
                prm.coarse_solver == GMG_COARSE_CG,
            "bad coarse_solver");
  CHECK_ARG(prm.coarse_tol > 0.0 && prm.coarse_tol < 1.0, "coarse_tol must be in (0, 1)");
  CHECK_ARG(prm.deterministic == 0 || prm.deterministic == 1, "deterministic must be 0 or 1");
  CHECK_ARG(prm.brick_min_members == 0 || (prm.brick_min_members >= 2 && prm.brick_min_members <= 8),
            "brick_min_members must be 0 or in [2, 8]");
  if (prm.brick_min_members == 0) prm.brick_min_members = 4;
  const Forest& f = mesh->f;
  CHECK_ARG(f.num_levels() <= GMG_MAX_LEVELS, "too many levels");
  GMG_GUARD_BEGIN
  gmg_hier* hh = new gmg_hier();
  Hier& h = hh->h;
  h.ctx = ctx;
  h.k = degree;
  h.params = prm;
  int64_t ncoarse = (int64_t)f.n0[0] * f.n0[1] * f.n0[2];
  h.coarse_coeff.assign(ncoarse, 1.0);
  if (coarse_coeff) {
    for (int64_t i = 0; i < ncoarse; ++i) {
      if (!(coarse_coeff[i] > 0.0) || !std::isfinite(coarse_coeff[i])) {
        delete hh;
        set_error("coefficients must be finite and > 0");
        return GMG_EINVAL;
      }
      h.coarse_coeff[i] = coarse_coeff[i];
    }
  }
  if (prm.fixed_lambda) {
    h.fixed_lambda.assign(prm.fixed_lambda, prm.fixed_lambda + f.num_levels());
    for (int l = 1; l < f.num_levels(); ++l)
      if (!(h.fixed_lambda[l] > 0.0)) {
        delete hh;
        set_error("fixed_lambda must be > 0 on levels >= 1");
        return GMG_EINVAL;
      }
    h.params.fixed_lambda = nullptr;
  }
  try {
    build_host_hierarchy(h, f);
  } catch (...) {
    delete hh;
    throw;
  }
  if (h.coarse_too_large) {
    delete hh;
    set_error("coarse level too large for the chosen coarse solver (Cholesky: 25600, Chebyshev: 2048, "
              "CG: 4096 unknowns)");
    return GMG_EUNSUPPORTED;
  }
  if (ctx->c.device >= 0) {
    cudaError_t e = cudaSetDevice(ctx->c.device);
    if (e != cudaSuccess) {
      delete hh;
      set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
      return GMG_ECUDA;
    }
    gmg_status st = device_setup(h);
    if (st == GMG_OK) st = noalloc_prepare(h);
    if (st != GMG_OK) {
      device_free(h);
      delete hh;
      return st;
    }
  }
  *out = hh;
  return GMG_OK;
  GMG_GUARD_END
}

void gmg_hier_destroy(gmg_hier* h) {
  if (!h) return;
  if (h->h.dev) {
    if (h->h.ctx && h->h.ctx->c.device >= 0) cudaSetDevice(h->h.ctx->c.device);
    device_free(h->h);
  }
  delete h;
}

gmg_status gmg_build_hierarchy(gmg_ctx* ctx, const gmg_coarse_mesh* cm, int n_rounds, gmg_refine_fn refine,
                               void* user, int degree, const double* coarse_coeff, const gmg_params* p,
                               gmg_hier** out) {
  CHECK_ARG(ctx && cm && out, "null argument");
  *out = nullptr;
  CHECK_ARG(n_rounds >= 0, "n_rounds must be >= 0");
  CHECK_ARG(refine || n_rounds == 0, "refine callback is null");
  gmg_mesh* m = nullptr;
  gmg_status st = gmg_mesh_create(cm, &m);
  if (st != GMG_OK) return st;
  std::unique_ptr<gmg_mesh, void (*)(gmg_mesh*)> hold(m, gmg_mesh_destroy);  // released on every path
  GMG_GUARD_BEGIN
  std::vector<int32_t> level, coords;
  std::vector<uint8_t> flags;
  for (int r = 0; r < n_rounds && st == GMG_OK; ++r) {
    const uint64_t n = m->f.leaf_level.size();
    level.resize(n);
    coords.resize(3 * n);
    st = gmg_mesh_leaves(m, level.data(), coords.data());
    if (st != GMG_OK) break;
    flags.assign(n, 0);
    if (refine(user, r, n, level.data(), coords.data(), flags.data()) != 0) {
      set_error("refinement callback stopped the build in round " + std::to_string(r));
      st = GMG_EINVAL;
      break;
    }
    st = gmg_mesh_refine(m, flags.data(), n);
  }
  if (st == GMG_OK) st = gmg_hier_build(ctx, m, degree, coarse_coeff, p, out);
  return st;
  GMG_GUARD_END
}

gmg_status gmg_hier_info(const gmg_hier* hh, gmg_info* info) {
  CHECK_ARG(hh && info, "null argument");
  const Hier& h = hh->h;
  std::memset(info, 0, sizeof(*info));
  info->dim = h.dim;
  info->degree = h.k;
  info->n_levels = h.L + 1;
  info->vcycle_prec = h.params.vcycle_prec;
  info->n_unknowns = h.active.n_unknowns;
  info->n_leaves = h.active.n_cells;
  info->n_hanging = h.active.hang_key.size();
  info->n_leaf_nodes = h.active.n_leaf_nodes;
  for (int l = 0; l <= h.L && l < GMG_MAX_LEVELS; ++l) {
    const LevelHost& L = h.levels[l];
    info->cells[l] = L.n_cells;
    info->leaves[l] = L.n_leaves;
    info->groups[l] = L.n_groups;
    info->ghosts[l] = L.n_ghosts;
    info->slots[l] = h.level_offset[l + 1] - h.level_offset[l];
    info->n_S[l] = L.n_S;
    info->n_I[l] = L.n_I;
    info->bricks[l] = L.n_bricks_full;
    info->bricks_partial[l] = L.bricks.size() / 64 - L.n_bricks_full;
    info->groups_jump[l] = L.list_jump.size();
    info->lambda_max[l] = l < (int)h.lambda.size() ? h.lambda[l] : 0.0;
  }
  for (int32_t lv : h.active.home_level) info->n_home[lv]++;
  info->device_bytes = device_bytes(h);
  info->setup_host_s = h.setup_host_s;
  info->setup_device_s = h.setup_device_s;
  info->leaf_patches = (uint64_t)h.active.n_patches;
  info->leaf_groups = (uint64_t)h.active.n_groups;
  info->leaf_single_cells = h.active.loose_cells.size();
  info->coarse_degree = h.coarse_degree;
  info->coarse_range[0] = h.coarse_range[0];
  info->coarse_range[1] = h.coarse_range[1];
  for (int i = 0; i < 8; ++i) info->setup_phase_s[i] = h.setup_phase_s[i];
  return GMG_OK;
}

gmg_status gmg_hier_export(const gmg_hier* hh, int what, int level, void* buf, uint64_t* count) {
  CHECK_ARG(hh && count, "null argument");
  const Hier& h = hh->h;
  const ActiveHost& A = h.active;
  uint64_t n = 0;
  size_t esz = 0;
  switch (what) {
    case GMG_EXPORT_UNKNOWN_KEYS: n = A.unknown_keys.size(); esz = 8; break;
    case GMG_EXPORT_HOME_LEVEL: n = A.home_level.size(); esz = 4; break;
    case GMG_EXPORT_HANGING: n = A.hang_col.size(); esz = 24; break;
    case GMG_EXPORT_HOME_SLOT: n = A.home_slot.size(); esz = 8; break;
    case GMG_EXPORT_LEVEL_KEYS:
    case GMG_EXPORT_LEVEL_CLASS:
      CHECK_ARG(level >= 0 && level <= h.L, "level out of range");
      n = h.levels[level].slot_key.size();
      esz = what == GMG_EXPORT_LEVEL_KEYS ? 8 : 1;
      break;
    default: set_error("unknown export item"); return GMG_EINVAL;
  }
  if (!buf) {
    *count = n;
    return GMG_OK;
  }
  CHECK_ARG(*count >= n, "buffer too small");
  unsigned char* out = (unsigned char*)buf;
  switch (what) {
    case GMG_EXPORT_UNKNOWN_KEYS: std::memcpy(out, A.unknown_keys.data(), n * esz); break;
    case GMG_EXPORT_HOME_LEVEL: std::memcpy(out, A.home_level.data(), n * esz); break;
    case GMG_EXPORT_HOME_SLOT: std::memcpy(out, A.home_slot.data(), n * esz); break;
    case GMG_EXPORT_LEVEL_KEYS: std::memcpy(out, h.levels[level].slot_key.data(), n * esz); break;
    case GMG_EXPORT_LEVEL_CLASS: std::memcpy(out, h.levels[level].slot_class.data(), n * esz); break;
    case GMG_EXPORT_HANGING: {
      size_t rec = 0;
      for (size_t r = 0; r + 1 < A.hang_ptr.size(); ++r)
        for (int32_t m = A.hang_ptr[r]; m < A.hang_ptr[r + 1]; ++m, ++rec) {
          int64_t hk = A.hang_key[r], mk = A.hang_master_key[m];
          double w = A.hang_w[m];
          std::memcpy(out + 24 * rec, &hk, 8);
          std::memcpy(out + 24 * rec + 8, &mk, 8);
          std::memcpy(out + 24 * rec + 16, &w, 8);
        }
      break;
    }
  }
  *count = n;
  return GMG_OK;
}

gmg_status gmg_assemble_rhs(gmg_hier* hh, int kind, uint64_t seed, double* d_b) {
  CHECK_ARG(hh && d_b, "null argument");
  CHECK_ARG(kind == GMG_RHS_SINE || kind == GMG_RHS_ONE || kind == GMG_RHS_RANDOM, "unknown right-hand side kind");
  GMG_GUARD_BEGIN
  gmg_status st = bind_device(hh->h);
  if (st != GMG_OK) return st;
  return device_rhs(hh->h, kind, seed, d_b);
  GMG_GUARD_END
}

gmg_status gmg_apply(gmg_hier* hh, const double* d_x, double* d_y) {
  CHECK_ARG(hh && d_x && d_y, "null argument");
  CHECK_ARG((const void*)d_x != (const void*)d_y, "x and y must not overlap");
  GMG_GUARD_BEGIN
  gmg_status st = bind_device(hh->h);
  if (st != GMG_OK) return st;
  return device_apply(hh->h, d_x, d_y);
  GMG_GUARD_END
}

gmg_status gmg_vcycle(gmg_hier* hh, const double* d_r, double* d_z) {
  CHECK_ARG(hh && d_r && d_z, "null argument");
  CHECK_ARG((const void*)d_r != (const void*)d_z, "r and z must not overlap");
  GMG_GUARD_BEGIN
  gmg_status st = bind_device(hh->h);
  if (st != GMG_OK) return st;
  return device_vcycle(hh->h, d_r, d_z);
  GMG_GUARD_END
}

gmg_status gmg_solve(gmg_hier* hh, const double* d_b, double* d_x, double tol, int max_iter,
                     int fixed_iterations, gmg_stats* stats) {
  CHECK_ARG(hh && d_b && d_x, "null argument");
  CHECK_ARG((const void*)d_b != (const void*)d_x, "b and x must not overlap");
  CHECK_ARG(fixed_iterations > 0 || (tol > 0 && std::isfinite(tol)), "tol must be finite and > 0");
  CHECK_ARG(max_iter >= 1 && max_iter <= 100000, "max_iter out of range [1, 100000]");
  CHECK_ARG(fixed_iterations >= 0 && fixed_iterations <= 100000, "fixed_iterations out of range");
  GMG_GUARD_BEGIN
  gmg_status st = bind_device(hh->h);
  if (st != GMG_OK) return st;
  return device_solve(hh->h, d_b, d_x, tol, max_iter, fixed_iterations, stats);
  GMG_GUARD_END
}

gmg_status gmg_solve_async(gmg_hier* hh, const double* d_b, double* d_x, double tol, int max_iter) {
  CHECK_ARG(hh && d_b && d_x, "null argument");
  CHECK_ARG((const void*)d_b != (const void*)d_x, "b and x must not overlap");
  CHECK_ARG(tol > 0 && std::isfinite(tol), "tol must be finite and > 0");
  CHECK_ARG(max_iter >= 1 && max_iter <= 100000, "max_iter out of range [1, 100000]");
  Hier& h = hh->h;
  CHECK_ARG(h.ctx && h.ctx->c.device >= 0 && h.dev, "needs a hierarchy built on a device");
  CHECK_ARG(h.params.solve_graph, "asynchronous solves need solve_graph = 1");
  GMG_GUARD_BEGIN
  gmg_status st = bind_device(h);
  if (st != GMG_OK) return st;
  return device_solve_async(h, d_b, d_x, tol, max_iter);
  GMG_GUARD_END
}

gmg_status gmg_solve_poll(gmg_hier* hh, int wait, int* ready, gmg_stats* stats, gmg_status* status) {
  CHECK_ARG(hh && ready && status, "null argument");
  Hier& h = hh->h;
  CHECK_ARG(h.ctx && h.ctx->c.device >= 0 && h.dev, "needs a hierarchy built on a device");
  GMG_GUARD_BEGIN
  gmg_status st = bind_device(h);
  if (st != GMG_OK) return st;
  return device_solve_poll(h, wait, ready, stats, status);
  GMG_GUARD_END
}

gmg_status gmg_solve_batch(gmg_hier* const* hs, const double* const* d_b, double* const* d_x, int n, double tol,
                           int max_iter, int n_streams, gmg_stats* stats, gmg_status* status) {
  CHECK_ARG(hs && d_b && d_x && status, "null argument");
  CHECK_ARG(n >= 1 && n <= (1 << 20), "n out of range [1, 2^20]");
  CHECK_ARG(n_streams >= 1 && n_streams <= 128, "n_streams out of range [1, 128]");
  CHECK_ARG(tol > 0 && std::isfinite(tol), "tol must be finite and > 0");
  CHECK_ARG(max_iter >= 1 && max_iter <= 100000, "max_iter out of range [1, 100000]");
  GMG_GUARD_BEGIN
  std::vector<Hier*> h(n);
  for (int i = 0; i < n; ++i) {
    CHECK_ARG(hs[i] && d_b[i] && d_x[i], "null hierarchy or vector");
    CHECK_ARG((const void*)d_b[i] != (const void*)d_x[i], "b and x must not overlap");
    h[i] = &hs[i]->h;
    CHECK_ARG(h[i]->ctx && h[i]->ctx->c.device >= 0 && h[i]->dev, "needs hierarchies built on a device");
    CHECK_ARG(h[i]->ctx->c.device == h[0]->ctx->c.device, "all hierarchies must live on one device");
    CHECK_ARG(h[i]->params.solve_graph, "batched solves need solve_graph = 1");
    for (int j = 0; j < i; ++j) CHECK_ARG(h[j] != h[i], "a hierarchy appears twice in the batch");
    status[i] = GMG_OK;
  }
  gmg_status st = bind_device(*h[0]);
  if (st != GMG_OK) return st;
  return device_solve_batch(h.data(), d_b, d_x, n, tol, max_iter, n_streams, stats, status);
  GMG_GUARD_END
}

static gmg_status check_level(const gmg_hier* hh, int level, int lo) {
  if (!hh) {
    set_error("null hierarchy");
    return GMG_EINVAL;
  }
  if (level < lo || level > hh->h.L) {
    set_error("level out of range");
    return GMG_EINVAL;
  }
  return bind_device(hh->h);
}

gmg_status gmg_level_apply(gmg_hier* hh, int level, const void* d_x, void* d_y) {
  gmg_status st = check_level(hh, level, 1);
  if (st != GMG_OK) return st;
  CHECK_ARG(d_x && d_y && d_x != d_y, "bad vectors");
  return device_level_apply(hh->h, level, d_x, d_y);
}

gmg_status gmg_level_residual_restrict(gmg_hier* hh, int level, const void* d_u, const void* d_g, void* d_gc) {
  gmg_status st = check_level(hh, level, 1);
  if (st != GMG_OK) return st;
  CHECK_ARG(d_u && d_g && d_gc, "bad vectors");
  return device_level_residual_restrict(hh->h, level, d_u, d_g, d_gc);
}

gmg_status gmg_level_prolongate(gmg_hier* hh, int level, const void* d_uc, void* d_u, void* d_u2) {
  gmg_status st = check_level(hh, level, 1);
  if (st != GMG_OK) return st;
  CHECK_ARG(d_uc && d_u && d_u2, "bad vectors");
  return device_level_prolongate(hh->h, level, d_uc, d_u, d_u2);
}

gmg_status gmg_level_smooth(gmg_hier* hh, int level, const void* d_g, void* d_u, void* d_tmp, int from_zero) {
  gmg_status st = check_level(hh, level, 1);
  if (st != GMG_OK) return st;
  CHECK_ARG(d_g && d_u && d_tmp && d_u != d_tmp && d_g != d_u && d_g != d_tmp, "bad vectors");
  return device_level_smooth(hh->h, level, d_g, d_u, d_tmp, from_zero);
}

gmg_status gmg_level_inv_diag(gmg_hier* hh, int level, void* d_out) {
  gmg_status st = check_level(hh, level, 1);
  if (st != GMG_OK) return st;
  CHECK_ARG(d_out, "bad vector");
  return device_level_inv_diag(hh->h, level, d_out);
}

gmg_status gmg_coarse_solve(gmg_hier* hh, const void* d_g0, void* d_u0) {
  gmg_status st = check_level(hh, 0, 0);
  if (st != GMG_OK) return st;
  CHECK_ARG(d_g0 && d_u0 && d_g0 != d_u0, "bad vectors");
  return device_coarse_solve(hh->h, d_g0, d_u0);
}

gmg_status gmg_profile_reset(gmg_hier* hh, int enable_timing) {
  CHECK_ARG(hh, "null hierarchy");
  gmg_status st = bind_device(hh->h);
  if (st != GMG_OK) return st;
  profile_reset(hh->h, enable_timing != 0);
  return GMG_OK;
}

gmg_status gmg_profile_read(gmg_hier* hh, gmg_kernel_stats* out) {
  CHECK_ARG(hh && out, "null argument");
  gmg_status st = bind_device(hh->h);
  if (st != GMG_OK) return st;
  profile_read(hh->h, out);
  return GMG_OK;
}

}  // extern "C"
