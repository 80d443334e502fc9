// Device setup and drivers: V-cycle (Algorithm 2, local smoothing of
// Sec. 2.3), Chebyshev-Jacobi smoothing and eigenvalue estimate (Sec. 4.1),
// and the outer preconditioned CG.
#include <algorithm>
#include <cstring>
#include <chrono>
#include <cmath>
#include <mutex>
#include <numeric>

#include "device_common.cuh"

namespace gmg {

thread_local uint64_t g_kernel_launches = 0;

namespace {

template <typename T>
gmg_status dev_alloc(DeviceState* d, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return GMG_OK;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? GMG_ENOMEM : GMG_ECUDA;
  }
  d->bytes += n * sizeof(T);
  return GMG_OK;
}

template <typename T>
gmg_status upload(DeviceState* d, T** p, const std::vector<T>& v) {
  gmg_status st = dev_alloc(d, p, v.size());
  if (st != GMG_OK) return st;
  if (!v.empty()) GMG_CUDA_TRY(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return GMG_OK;
}

#define GMG_TRY(expr)                  \
  do {                                 \
    gmg_status s_ = (expr);            \
    if (s_ != GMG_OK) return s_;       \
  } while (0)

int ipow_h(int b, int e) {
  int r = 1;
  while (e--) r *= b;
  return r;
}

}  // namespace

// ------------------------------------------------------ launch accounting
static cudaEvent_t take_event(Profile& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void drain(DeviceState* d) {
  Profile& p = d->prof;
  if (p.pending.empty()) return;
  cudaStreamSynchronize(d->stream);
  for (auto& q : p.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) p.ms[q.kind] += ms;
    p.pool.push_back(q.a);
    p.pool.push_back(q.b);
  }
  p.pending.clear();
}

// Accounts the kernels launched in its scope (one step of the path) to
// `kind`, with the step's algorithmic bytes and flops; with timing on,
// brackets the step with events.
struct Track {
  DeviceState* d;
  int kind;
  uint64_t first;
  uint64_t* launches;
  cudaEvent_t a = nullptr;
  Track(DeviceState* dd, int k, double bytes, double flops) : d(dd), kind(k), first(g_kernel_launches) {
    if (d->cap) {  // captured into a graph: counted per execution of the graph
      launches = &d->cap->launches[k];
      d->cap->bytes[k] += bytes;
      d->cap->flops[k] += flops;
      return;
    }
    Profile& p = d->prof;
    launches = &p.launches[k];
    p.bytes[k] += bytes;
    p.flops[k] += flops;
    if (p.timing) {
      if (p.pending.size() > 30000) drain(d);
      a = take_event(p);
      cudaEventRecord(a, d->stream);
    }
  }
  ~Track() {
    *launches += g_kernel_launches - first;
    if (!a) return;
    cudaEvent_t b = take_event(d->prof);
    cudaEventRecord(b, d->stream);
    d->prof.pending.push_back({kind, a, b});
  }
};

void profile_reset(Hier& h, bool timing) {
  DeviceState* d = h.dev;
  drain(d);
  Profile& p = d->prof;
  for (int k = 0; k < GMG_NUM_KERNEL_KINDS; ++k) p.launches[k] = 0, p.ms[k] = p.bytes[k] = p.flops[k] = 0.0;
  p.timing = timing;
}

void profile_read(Hier& h, gmg_kernel_stats* out) {
  DeviceState* d = h.dev;
  drain(d);
  cudaStreamSynchronize(d->stream);
  for (int k = 0; k < GMG_NUM_KERNEL_KINDS; ++k) {
    out->launches[k] = d->prof.launches[k];
    out->ms[k] = d->prof.ms[k];
    out->bytes[k] = d->prof.bytes[k];
    out->flops[k] = d->prof.flops[k];
  }
}

// floating-point operations of one sibling group in the smoothing kernel
// (nonzeros of the extended 1-D matrices per sum-factorisation stage)
static double cheb_group_flops(int dim, int k) {
  std::vector<double> M, K, E;
  reference_1d(k, M, K, E);
  const int NH = 3 * k + 1, NE = 2 * k + 1, n1 = k + 1;
  auto nnz = [&](const std::vector<double>& B) {
    int c = 0;
    for (int e = 0; e < NE; ++e)
      for (int col = 0; col < NH; ++col) {
        int p = col - k;
        double v = 0;
        if (e < 2 * k) {
          for (int cell = 0; cell < 2; ++cell) {
            int lo = k * cell;
            if (e >= lo && e <= lo + k && p >= lo && p <= lo + k) v += std::fabs(B[(e - lo) * n1 + (p - lo)]);
          }
        } else if (p >= -k && p <= 0) {
          v = std::fabs(B[k * n1 + p + k]);
        }
        c += v != 0.0;
      }
    return c;
  };
  double nm = nnz(M), nk = nnz(K);
  double fma = dim == 3 ? NH * NH * (nm + nk) + NH * NE * (2 * nm + nk) + NE * NE * (nm + nk + NH)
                        : NH * (nm + nk) + NE * (nm + nk);
  return 2.0 * fma + 4.0 * std::pow(2 * k, dim);
}

static double ipow_d(int b, int e) {
  double r = 1;
  while (e--) r *= b;
  return r;
}

static LevelArgs level_args(const Hier& h, int l) {
  const LevelDev& L = h.dev->lv[l];
  LevelArgs a;
  a.n_groups = L.n_groups;
  a.nbr = L.nbr;
  a.state = L.state;
  a.coeff = L.coeff;
  a.coeff32 = L.coeff32;
  a.smask = L.smask;
  a.lcoef64 = L.lcoef64;
  a.lcoef32 = L.lcoef32;
  a.parent = L.parent;
  a.list_uniform = L.list_uniform;
  a.pmask = L.pmask;
  a.bricks = L.bricks;
  a.n_bricks = L.n_bricks;
  a.n_bricks_all = L.n_bricks_all;
  a.brick_members = L.brick_members;
  a.brick_info = L.brick_info;
  a.brick_cnb = L.brick_cnb;
  a.group_cnb = L.group_cnb;
  a.iso = L.iso;
  a.list_rest = L.list_rest;
  a.n_rest = L.n_rest;
  a.no_ghosts = L.n_slots == L.n_groups * (int64_t)ipow_h(2 * h.k, h.dim);
  a.list_jump = L.list_jump;
  a.n_uniform = L.n_uniform;
  a.n_jump = L.n_jump;
  a.nbr_coarse = l >= 2 ? h.dev->lv[l - 1].nbr : nullptr;
  a.deterministic = h.params.deterministic != 0;
  a.brick_off = L.brick_off.empty() ? nullptr : L.brick_off.data();
  a.n_brick_colors = L.brick_off.empty() ? 0 : (int)L.brick_off.size() - 1;
  a.list_color = L.list_color;
  a.group_off = L.group_off.empty() ? nullptr : L.group_off.data();
  a.n_group_colors = L.group_off.empty() ? 0 : (int)L.group_off.size() - 1;
  for (int d = 0; d < 3; ++d) {
    a.coarse_lat[d] = h.coarse_lattice[d];
    a.scale[d] = L.scale[d];
    a.scale32[d] = (float)L.scale[d];
  }
  a.level = l;
  return a;
}

static ActiveArgs active_args(const Hier& h) {
  ActiveArgs a;
  a.n_cells = h.dev->n_cells;
  a.cell_list = h.dev->loose;
  a.n_list = h.dev->n_loose;
  a.n_groups = h.dev->n_grp;
  a.grp_nodes = h.dev->grp_nodes;
  a.grp_coeff = h.dev->grp_coeff;
  a.grp_level = h.dev->grp_level;
  a.loose_nodes = h.dev->loose_nodes;
  a.loose_coeff = h.dev->loose_coeff;
  a.loose_level = h.dev->loose_level;
  a.n_patches = h.dev->n_pat;
  a.pat_nodes = h.dev->pat_nodes;
  a.pat_coeff = h.dev->pat_coeff;
  a.pat_level = h.dev->pat_level;
  a.cell_nodes = h.dev->cell_nodes;
  a.cell_coeff = h.dev->cell_coeff;
  a.cell_level = h.dev->cell_level;
  a.hang_ptr = h.dev->hang_ptr;
  a.hang_col = h.dev->hang_col;
  a.hang_wc = h.dev->hang_wc;
  a.hw_table = h.dev->hw_table;
  a.n_hw = h.dev->n_hw;
  a.n_hang = h.dev->n_hang;
  a.xh = h.dev->xh;
  a.yh = h.dev->yh;
  a.n_masters = h.dev->n_masters;
  a.hm_node = h.dev->hm_node;
  a.hm_ptr = h.dev->hm_ptr;
  a.hm_hang = h.dev->hm_hang;
  a.hm_wc = h.dev->hm_wc;
  const DeviceState* d = h.dev;
  a.deterministic = h.params.deterministic != 0;
  a.pat_off = d->pat_off.empty() ? nullptr : d->pat_off.data();
  a.n_pat_colors = d->pat_off.empty() ? 0 : (int)d->pat_off.size() - 1;
  a.grp_off = d->grp_off.empty() ? nullptr : d->grp_off.data();
  a.n_grp_colors = d->grp_off.empty() ? 0 : (int)d->grp_off.size() - 1;
  a.loose_off = d->loose_off.empty() ? nullptr : d->loose_off.data();
  a.n_loose_colors = d->loose_off.empty() ? 0 : (int)d->loose_off.size() - 1;
  for (int l = 0; l < GMG_MAX_LEVELS; ++l)
    for (int d = 0; d < 3; ++d) {
      a.scale[l][d] = h.dev->level_scale[l][d];
      a.h[l][d] = h.dev->cell_h[l][d];
    }
  for (int d = 0; d < 3; ++d) a.lo[d] = h.lo[d];
  return a;
}

// K-term factors s_i = prod_{j != i} h_j / h_i of a level's cells
static void level_scales(const Hier& h, int l, double* s, double* hh) {
  for (int d = 0; d < 3; ++d) hh[d] = d < h.dim ? (h.hi[d] - h.lo[d]) / ((double)h.n0[d] * (double)(1ll << l)) : 1.0;
  for (int i = 0; i < 3; ++i) {
    if (i >= h.dim) {
      s[i] = 0.0;
      continue;
    }
    double v = 1.0 / hh[i];
    for (int j = 0; j < h.dim; ++j)
      if (j != i) v *= hh[j];
    s[i] = v;
  }
}

void device_free(Hier& h) {
  DeviceState* d = h.dev;
  if (!d) return;
  for (auto& L : d->lv) {
    cudaFree(L.nbr);
    cudaFree(L.state);
    cudaFree(L.coeff);
    cudaFree(L.parent);
    cudaFree(L.smask);
    cudaFree(L.lcoef64);
    cudaFree(L.lcoef32);
    cudaFree(L.coeff32);
    cudaFree(L.list_uniform);
    cudaFree(L.pmask);
    cudaFree(L.bricks);
    cudaFree(L.brick_members);
    cudaFree(L.brick_info);
    cudaFree(L.brick_cnb);
    cudaFree(L.group_cnb);
    cudaFree(L.list_jump);
    cudaFree(L.list_rest);
    cudaFree(L.list_color);
  }
  void* ptrs[] = {d->uA, d->uB, d->g, d->dinv, d->coarse_slot, d->coarse_inv, d->coarse_ptr, d->coarse_col, d->coarse_val, d->cell_nodes, d->cell_coeff, d->cell_level,
                  d->cell_coords, d->hang_ptr, d->hang_col, d->hang_wc, d->hw_table, d->home, d->perm, d->r, d->p, d->Ap,
                  d->partials, d->counter, d->scal, d->loose, d->grp_nodes, d->grp_coeff, d->grp_level,
                  d->pat_nodes, d->pat_coeff, d->pat_level, d->loose_nodes, d->loose_coeff, d->loose_level,
                  d->xh, d->yh, d->hm_node, d->hm_ptr,
                  d->hm_hang, d->hm_wc};
  for (void* p : ptrs) cudaFree(p);
  if (d->scal_host) cudaFreeHost(d->scal_host);
  if (d->cg_exec) cudaGraphExecDestroy(d->cg_exec);
  if (d->cg_graph) cudaGraphDestroy(d->cg_graph);
  cudaFree(d->x_iter);
  cudaFree(d->ctl);
  if (d->ctl_host) cudaFreeHost(d->ctl_host);
  if (d->cap_stream) cudaStreamDestroy(d->cap_stream);
  if (d->done) cudaEventDestroy(d->done);
  for (auto& q : d->prof.pending) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  for (cudaEvent_t e : d->prof.pool) cudaEventDestroy(e);
  delete d;
  h.dev = nullptr;
}

uint64_t device_bytes(const Hier& h) { return h.dev ? h.dev->bytes : 0; }

static gmg_status ensure_scalars(DeviceState* d, int n) {
  if (n <= d->max_scal) return GMG_OK;
  cudaFree(d->scal);
  if (d->scal_host) cudaFreeHost(d->scal_host);
  d->scal = nullptr;
  d->scal_host = nullptr;
  int cap = std::max(n, 4096);
  GMG_CUDA_TRY(cudaMalloc(&d->scal, sizeof(double) * cap));
  GMG_CUDA_TRY(cudaMallocHost(&d->scal_host, sizeof(double) * cap));
  GMG_CUDA_TRY(cudaMemset(d->scal, 0, sizeof(double) * cap));
  d->max_scal = cap;
  return GMG_OK;
}

static double host_dot(DeviceState* d, int64_t n, const double* a, const double* b) {
  launch_dot(n, a, b, d->partials, d->counter, d->scal, d->stream);
  cudaMemcpyAsync(d->scal_host, d->scal, sizeof(double), cudaMemcpyDeviceToHost, d->stream);
  cudaStreamSynchronize(d->stream);
  return d->scal_host[0];
}

// lambda_max of D^{-1} A_l^S: PCG from y0 = 0 on A^S y = b0 with Jacobi
// preconditioning; Lanczos tridiagonal from the CG coefficients (Sec. 4.1).
static gmg_status estimate_lambda(Hier& h, int l, double* r, double* z, double* p, double* Ap,
                                  const double* dinv64, double* out) {
  DeviceState* d = h.dev;
  const LevelDev& L = d->lv[l];
  const LevelHost& LH = h.levels[l];
  const int64_t n = L.n_slots;
  cudaStream_t s = d->stream;
  // start vector on S slots: -5.5 + (rank mod 12), rank in canonical key order
  std::vector<int64_t> sidx;
  for (int64_t i = 0; i < n; ++i)
    if (LH.slot_class[i] == 1) sidx.push_back(i);
  std::sort(sidx.begin(), sidx.end(), [&](int64_t a, int64_t b) { return LH.slot_key[a] < LH.slot_key[b]; });
  std::vector<double> b0(n, 0.0);
  for (size_t i = 0; i < sidx.size(); ++i) b0[sidx[i]] = -5.5 + (double)(i % 12);
  GMG_CUDA_TRY(cudaMemcpyAsync(r, b0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  GMG_CUDA_TRY(cudaMemsetAsync(Ap, 0, n * sizeof(double), s));
  launch_mul(n, dinv64, r, z, s);
  GMG_CUDA_TRY(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double rz = host_dot(d, n, r, z);
  const double rz0 = rz;
  const int iters = (int)std::min<int64_t>(h.params.eig_iters, (int64_t)sidx.size());
  std::vector<double> alpha, beta;
  LevelArgs a = level_args(h, l);
  for (int j = 0; j < iters; ++j) {
    GMG_CUDA_TRY(launch_level_cheb<double>(h.dim, h.k, a, p, nullptr, nullptr, nullptr, Ap, 0.0, 0.0, true, s));
    double pAp = host_dot(d, n, p, Ap);
    double al = rz / pAp;
    alpha.push_back(al);
    launch_axpy(n, -al, Ap, r, s);
    launch_mul(n, dinv64, r, z, s);
    double rz_new = host_dot(d, n, r, z);
    if (j == iters - 1 || rz_new <= 1e-24 * rz0) break;
    double be = rz_new / rz;
    beta.push_back(be);
    launch_xpay(n, z, be, p, s);
    rz = rz_new;
  }
  GMG_CUDA_TRY(cudaGetLastError());
  size_t m = alpha.size();
  std::vector<double> diag(m), off(m > 0 ? m - 1 : 0);
  for (size_t j = 0; j < m; ++j) {
    diag[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j + 1 < m) off[j] = std::sqrt(beta[j]) / alpha[j];
  }
  *out = tridiag_max_eig(diag, off);
  return GMG_OK;
}

gmg_status device_setup(Hier& h) {
  auto t0 = std::chrono::steady_clock::now();
  DeviceState* d = new DeviceState();
  h.dev = d;
  d->stream = (cudaStream_t)h.ctx->c.stream;
  d->prec = h.params.vcycle_prec;
  const int L = h.L, dim = h.dim, k = h.k;
  const int NOWN = ipow_h(2 * k, dim);
  d->lv.resize(L + 1);
  for (int l = 0; l <= L; ++l) {
    LevelDev& D = d->lv[l];
    const LevelHost& H = h.levels[l];
    D.offset = h.level_offset[l];
    D.n_slots = (int64_t)H.slot_class.size();
    double hh[3];
    level_scales(h, l, D.scale, hh);
    D.n_S = (double)H.n_S;
    D.n_I = (double)H.n_I;
    D.n_S_jump = (double)H.n_S_jump;
    D.zero_each_cycle = l == 0 || H.n_I > 0 || H.n_ghosts > 0;
    if (l == 0) continue;
    D.cheb_flops = (double)H.n_groups * cheb_group_flops(dim, k);
    D.n_groups = H.n_groups;
    GMG_TRY(upload(d, &D.nbr, H.nbr));
    GMG_TRY(upload(d, &D.state, H.state));
    GMG_TRY(upload(d, &D.coeff, H.coeff));
    GMG_TRY(upload(d, &D.parent, H.parent));
    GMG_TRY(upload(d, &D.smask, H.smask));
    GMG_TRY(upload(d, &D.lcoef64, H.lcoef));
    GMG_TRY(upload(d, &D.lcoef32, std::vector<float>(H.lcoef.begin(), H.lcoef.end())));
    GMG_TRY(upload(d, &D.coeff32, std::vector<float>(H.coeff.begin(), H.coeff.end())));
    GMG_TRY(upload(d, &D.list_uniform, H.list_uniform));
    GMG_TRY(upload(d, &D.pmask, H.pmask));
    std::vector<int32_t> bricks = H.bricks;
    D.n_bricks = H.n_bricks_full;
    D.n_bricks_all = (int64_t)bricks.size() / 64;
    if (h.params.deterministic) {
      // restriction colours.  A full brick adds into the nodes of the eight
      // parent cells p + {0,1}^d (p even, its first group's position), a
      // group into those of its parent cell c: two bricks whose (p / 2) have
      // the same parities, or two groups whose c have, are at least two
      // parent groups (cells) apart and share no coarse node.
      auto parity = [&](const int64_t* q, int shift) {
        int c = 0;
        for (int dd = 0; dd < dim; ++dd) c |= (int)((q[dd] >> shift) & 1) << dd;
        return c;
      };
      const int nc = 1 << dim;
      std::vector<std::vector<int64_t>> by(nc);
      for (int64_t br = 0; br < D.n_bricks; ++br) {
        const int32_t g0 = H.bricks[(size_t)br * 64 + 21];  // own group (0, 0, 0) at table position (1, 1, 1)
        by[parity(&H.block_pos[3 * (size_t)g0], 1)].push_back(br);
      }
      D.brick_off.assign(1, 0);
      int64_t at = 0;
      for (int c = 0; c < nc; ++c) {
        for (int64_t br : by[c]) {
          std::copy(H.bricks.begin() + br * 64, H.bricks.begin() + br * 64 + 64, bricks.begin() + at * 64);
          ++at;
        }
        D.brick_off.push_back(at);
      }
      std::vector<std::vector<int32_t>> gby(nc);
      for (int64_t g = 0; g < H.n_groups; ++g) gby[parity(&H.block_pos[3 * (size_t)g], 0)].push_back((int32_t)g);
      std::vector<int32_t> list;
      D.group_off.assign(1, 0);
      for (int c = 0; c < nc; ++c) {
        list.insert(list.end(), gby[c].begin(), gby[c].end());
        D.group_off.push_back((int64_t)list.size());
      }
      GMG_TRY(upload(d, &D.list_color, list));
    }
    GMG_TRY(upload(d, &D.bricks, bricks));
    GMG_TRY(upload(d, &D.brick_members, H.brick_members));
    if (l >= 2) {
      // each group's parent group (level l-1) and its 3^d neighbours
      const int nnb = ipow_h(3, dim);
      const std::vector<int32_t>& cn = h.levels[l - 1].nbr;
      std::vector<int32_t> rows((size_t)H.n_groups * nnb, -1);
      for (int64_t g = 0; g < H.n_groups; ++g) {
        const int64_t p = H.parent[g];
        if (p >= 0) std::copy(cn.begin() + p * nnb, cn.begin() + (p + 1) * nnb, rows.begin() + g * nnb);
      }
      GMG_TRY(upload(d, &D.group_cnb, rows));
    }
    if (dim == 3 && l >= 2 && D.n_bricks > 0) {
      // the parent group (level l-1) of a full brick's groups and its 27 neighbours
      const std::vector<int32_t>& cn = h.levels[l - 1].nbr;
      std::vector<int32_t> cnb((size_t)D.n_bricks * 27);
      for (int64_t br = 0; br < D.n_bricks; ++br) {
        const int32_t g0 = bricks[(size_t)br * 64 + 21];  // own group (0, 0, 0)
        const int64_t p = H.parent[g0];
        std::copy(cn.begin() + p * 27, cn.begin() + p * 27 + 27, cnb.begin() + br * 27);
      }
      GMG_TRY(upload(d, &D.brick_cnb, cnb));
    }
    {
      // per-brick flags and coefficient, read once per brick by the brick
      // smoother instead of per node
      const uint64_t full = NOWN >= 64 ? ~0ull : ((1ull << NOWN) - 1);
      std::vector<uint2> info((size_t)D.n_bricks_all);
      for (int64_t br = 0; br < D.n_bricks_all; ++br) {
        const unsigned members = br < D.n_bricks ? 0xFFu : (unsigned)H.brick_members[br - D.n_bricks];
        bool all_s = true;
        int32_t m0 = -1;
        for (int b = 0; b < 8; ++b) {
          if (!((members >> b) & 1u)) continue;
          const int32_t gid = bricks[(size_t)br * 64 + ((b & 1) + 1) + 4 * ((((b >> 1) & 1) + 1) + 4 * ((b >> 2) + 1))];
          if (m0 < 0) m0 = gid;
          if ((H.smask[gid] & full) != full) all_s = false;
        }
        const float c = m0 >= 0 ? (float)H.coeff[m0] : 0.f;
        unsigned cb;
        std::memcpy(&cb, &c, 4);
        info[br] = make_uint2(members | (all_s ? kBrickAllS : 0u), cb);
      }
      GMG_TRY(upload(d, &D.brick_info, info));
    }
    D.iso = dim == 3 && D.scale[0] == D.scale[1] && D.scale[1] == D.scale[2];
    GMG_TRY(upload(d, &D.list_rest, H.list_rest));
    D.n_rest = (int64_t)H.list_rest.size();
    GMG_TRY(upload(d, &D.list_jump, H.list_jump));
    D.n_uniform = (int64_t)H.list_uniform.size();
    D.n_jump = (int64_t)H.list_jump.size();
    if (D.n_slots != (H.n_groups + H.n_ghosts) * NOWN) {
      set_error("level slot count mismatch");
      return GMG_EINVAL;
    }
  }
  for (int dd = 0; dd < 3; ++dd) d->coarse_lat[dd] = h.coarse_lattice[dd];
  d->n_coarse = h.n_coarse;
  GMG_TRY(upload(d, &d->coarse_slot, h.coarse_slots));
  GMG_TRY(upload(d, &d->coarse_inv, h.coarse_inverse));
  GMG_TRY(upload(d, &d->coarse_ptr, h.coarse_ptr));
  GMG_TRY(upload(d, &d->coarse_col, h.coarse_col));
  d->coarse_nnz = (int64_t)h.coarse_col.size();
  GMG_TRY(upload(d, &d->coarse_val, h.coarse_val));
  // level vectors
  const size_t esz = d->prec == GMG_PREC_FP32 ? sizeof(float) : sizeof(double);
  const int64_t ns = h.total_slots;
  {
    unsigned char* p;
    GMG_TRY(dev_alloc(d, &p, ns * esz)); d->uA = p;
    GMG_TRY(dev_alloc(d, &p, ns * esz)); d->uB = p;
    GMG_TRY(dev_alloc(d, &p, ns * esz)); d->g = p;
    GMG_TRY(dev_alloc(d, &p, ns * esz)); d->dinv = p;
    // Dirichlet slots of the smoother vectors are never written: zero once
    GMG_CUDA_TRY(cudaMemsetAsync(d->uA, 0, ns * esz, d->stream));
    GMG_CUDA_TRY(cudaMemsetAsync(d->uB, 0, ns * esz, d->stream));
  }
  // active mesh, unknowns renumbered by home slot (every unknown has one
  // home slot, so this is a permutation); tables keep their encoding (-1
  // Dirichlet, <= -2 hanging row) and only unknown indices change
  const ActiveHost& A = h.active;
  d->n_unknowns = A.n_unknowns;
  d->n_cells = A.n_cells;
  std::vector<int32_t> perm, inv;
  {
    const int64_t nu = A.n_unknowns;
    std::vector<int32_t> at_slot((size_t)h.total_slots, -1);
    for (int64_t u = 0; u < nu; ++u) at_slot[A.home_global[u]] = (int32_t)u;
    perm.reserve((size_t)nu);
    for (int64_t sl = 0; sl < h.total_slots; ++sl)
      if (at_slot[sl] >= 0) perm.push_back(at_slot[sl]);
    if ((int64_t)perm.size() != nu) {
      set_error("internal: home slots are not one per unknown");
      return GMG_EINVAL;
    }
    inv.assign((size_t)nu, 0);
    for (int64_t j = 0; j < nu; ++j) inv[perm[j]] = (int32_t)j;
  }
  // hanging rows in the order of their number of masters (stable), so that
  // the threads of a warp in the constraint kernels take rows of one length
  const int64_t nh = (int64_t)A.hang_key.size();
  std::vector<int32_t> hold((size_t)nh), hnew((size_t)nh);
  std::iota(hold.begin(), hold.end(), 0);
  std::stable_sort(hold.begin(), hold.end(), [&](int32_t x, int32_t y) {
    return A.hang_ptr[x + 1] - A.hang_ptr[x] < A.hang_ptr[y + 1] - A.hang_ptr[y];
  });
  for (int64_t k = 0; k < nh; ++k) hnew[hold[k]] = (int32_t)k;
  auto renumbered = [&](const std::vector<int32_t>& v) {
    std::vector<int32_t> out(v.size());
    const int64_t m = (int64_t)v.size();
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) out[i] = v[i] >= 0 ? inv[v[i]] : (v[i] <= -2 ? -2 - hnew[-2 - v[i]] : v[i]);
    return out;
  };
  // deterministic mode: colour the patches, the groups and the single cells
  // (each kind on its own, greedily in table order) so that elements of one
  // colour share no node (unknown or hanging), and order each kind's tables
  // by colour.  A launch per colour then adds to shared nodes without
  // atomics, in a fixed order.
  auto colour_order = [&](const std::vector<int32_t>& nodes, int nn, int64_t n, std::vector<int64_t>& off,
                          std::vector<int64_t>& order) -> bool {
    const int64_t nu = A.n_unknowns, nh = (int64_t)A.hang_key.size();
    std::vector<uint64_t> used((size_t)(nu + nh), 0);
    std::vector<int> col((size_t)n, 0);
    int ncol = 0;
    for (int64_t e = 0; e < n; ++e) {
      uint64_t busy = 0;
      for (int j = 0; j < nn; ++j) {
        const int32_t id = nodes[(size_t)e * nn + j];
        if (id >= 0) busy |= used[id];
        else if (id <= -2) busy |= used[nu + (-2 - id)];
      }
      if (~busy == 0) return false;  // more than 64 colours
      const int c = __builtin_ctzll(~busy);
      col[e] = c;
      ncol = std::max(ncol, c + 1);
      for (int j = 0; j < nn; ++j) {
        const int32_t id = nodes[(size_t)e * nn + j];
        if (id >= 0) used[id] |= 1ull << c;
        else if (id <= -2) used[nu + (-2 - id)] |= 1ull << c;
      }
    }
    off.assign(ncol + 1, 0);
    for (int64_t e = 0; e < n; ++e) ++off[col[e] + 1];
    for (int c = 0; c < ncol; ++c) off[c + 1] += off[c];
    std::vector<int64_t> at(off.begin(), off.end() - 1);
    order.assign((size_t)n, 0);
    for (int64_t e = 0; e < n; ++e) order[at[col[e]]++] = e;
    return true;
  };
  auto reorder = [](const auto& v, const std::vector<int64_t>& order, int per) {
    std::decay_t<decltype(v)> out(v.size());
    for (size_t i = 0; i < order.size(); ++i)
      std::copy(v.begin() + order[i] * per, v.begin() + order[i] * per + per, out.begin() + i * per);
    return out;
  };
  const int NN4 = ipow_h(4 * k + 1, dim), NN2 = ipow_h(2 * k + 1, dim), NC1 = ipow_h(k + 1, dim);
  std::vector<int32_t> pat_nodes = A.pat_nodes, grp_nodes = A.grp_nodes, loose_nodes = A.loose_nodes,
                       loose_cells = A.loose_cells;
  std::vector<double> pat_coeff = A.pat_coeff, grp_coeff = A.grp_coeff, loose_coeff = A.loose_coeff;
  std::vector<uint8_t> pat_level = A.pat_level, grp_level = A.grp_level, loose_level = A.loose_level;
  d->pat_off.clear();
  d->grp_off.clear();
  d->loose_off.clear();
  if (h.params.deterministic) {
    std::vector<int64_t> order;
    bool ok = colour_order(A.pat_nodes, NN4, A.n_patches, d->pat_off, order);
    if (ok) {
      pat_nodes = reorder(A.pat_nodes, order, NN4);
      pat_coeff = reorder(A.pat_coeff, order, 1);
      pat_level = reorder(A.pat_level, order, 1);
    }
    ok = ok && colour_order(A.grp_nodes, NN2, A.n_groups, d->grp_off, order);
    if (ok) {
      grp_nodes = reorder(A.grp_nodes, order, NN2);
      grp_coeff = reorder(A.grp_coeff, order, 1);
      grp_level = reorder(A.grp_level, order, 1);
    }
    ok = ok && colour_order(A.loose_nodes, NC1, (int64_t)A.loose_cells.size(), d->loose_off, order);
    if (ok) {
      loose_nodes = reorder(A.loose_nodes, order, NC1);
      loose_coeff = reorder(A.loose_coeff, order, 1);
      loose_level = reorder(A.loose_level, order, 1);
      loose_cells = reorder(A.loose_cells, order, 1);
    }
    if (!ok) {
      set_error("deterministic mode: the leaf elements need more than 64 colours");
      return GMG_EUNSUPPORTED;
    }
  }
  std::vector<uint32_t> home_int((size_t)A.n_unknowns);
  for (int64_t j = 0; j < A.n_unknowns; ++j) home_int[j] = A.home_global[perm[j]];
  GMG_TRY(upload(d, &d->perm, perm));
  GMG_TRY(upload(d, &d->cell_nodes, renumbered(A.cell_nodes)));
  GMG_TRY(upload(d, &d->cell_coeff, A.cell_coeff));
  GMG_TRY(upload(d, &d->cell_level, A.cell_level));
  GMG_TRY(upload(d, &d->cell_coords, A.cell_coords));
  // constraint rows in the new hanging order; master rows (C^T) ordered by
  // their number of entries (stable)
  std::vector<int32_t> hptr(1, 0), hcol, mptr(1, 0), mnode, mhang;
  std::vector<double> hw, mw;
  hcol.reserve(A.hang_col.size());
  hw.reserve(A.hang_w.size());
  for (int64_t k = 0; k < nh; ++k) {
    const int32_t h0 = hold[k];
    for (int32_t m = A.hang_ptr[h0]; m < A.hang_ptr[h0 + 1]; ++m) {
      hcol.push_back(inv[A.hang_col[m]]);
      hw.push_back(A.hang_w[m]);
    }
    hptr.push_back((int32_t)hcol.size());
  }
  {
    const int64_t nm = (int64_t)A.hm_node.size();
    std::vector<int32_t> mold((size_t)nm);
    std::iota(mold.begin(), mold.end(), 0);
    std::stable_sort(mold.begin(), mold.end(), [&](int32_t x, int32_t y) {
      return A.hm_ptr[x + 1] - A.hm_ptr[x] < A.hm_ptr[y + 1] - A.hm_ptr[y];
    });
    mhang.reserve(A.hm_hang.size());
    mw.reserve(A.hm_w.size());
    for (int64_t k = 0; k < nm; ++k) {
      const int32_t i0 = mold[k];
      mnode.push_back(inv[A.hm_node[i0]]);
      for (int32_t j = A.hm_ptr[i0]; j < A.hm_ptr[i0 + 1]; ++j) {
        mhang.push_back(hnew[A.hm_hang[j]]);
        mw.push_back(A.hm_w[j]);
      }
      mptr.push_back((int32_t)mhang.size());
    }
  }
  GMG_TRY(upload(d, &d->hang_ptr, hptr));
  GMG_TRY(upload(d, &d->hang_col, hcol));
  {
    // distinct weights (bit-exact) and a code per entry
    std::vector<double> table;
    std::vector<uint8_t> wc(hw.size()), mc(mw.size());
    auto code = [&](double w, uint8_t& out) {
      for (size_t i = 0; i < table.size(); ++i)
        if (std::memcmp(&table[i], &w, sizeof(double)) == 0) {
          out = (uint8_t)i;
          return true;
        }
      if (table.size() == 256) return false;
      table.push_back(w);
      out = (uint8_t)(table.size() - 1);
      return true;
    };
    for (size_t m = 0; m < hw.size(); ++m)
      if (!code(hw[m], wc[m])) {
        set_error("more than 256 distinct hanging-node weights");
        return GMG_EUNSUPPORTED;
      }
    for (size_t m = 0; m < mw.size(); ++m)
      if (!code(mw[m], mc[m])) {
        set_error("more than 256 distinct hanging-node weights");
        return GMG_EUNSUPPORTED;
      }
    d->n_hw = (int)table.size();
    GMG_TRY(upload(d, &d->hw_table, table));
    GMG_TRY(upload(d, &d->hang_wc, wc));
    GMG_TRY(upload(d, &d->hm_wc, mc));
  }
  d->n_hang = (int64_t)A.hang_key.size();
  d->n_masters = (int64_t)A.hm_node.size();
  GMG_TRY(dev_alloc(d, &d->xh, (size_t)d->n_hang));
  GMG_TRY(dev_alloc(d, &d->yh, (size_t)d->n_hang));
  GMG_TRY(upload(d, &d->hm_node, mnode));
  GMG_TRY(upload(d, &d->hm_ptr, mptr));
  GMG_TRY(upload(d, &d->hm_hang, mhang));
  GMG_TRY(upload(d, &d->home, home_int));
  GMG_TRY(upload(d, &d->loose, loose_cells));
  GMG_TRY(upload(d, &d->grp_nodes, renumbered(grp_nodes)));
  GMG_TRY(upload(d, &d->grp_coeff, grp_coeff));
  GMG_TRY(upload(d, &d->grp_level, grp_level));
  GMG_TRY(upload(d, &d->loose_nodes, renumbered(loose_nodes)));
  GMG_TRY(upload(d, &d->loose_coeff, loose_coeff));
  GMG_TRY(upload(d, &d->loose_level, loose_level));
  GMG_TRY(upload(d, &d->pat_nodes, renumbered(pat_nodes)));
  GMG_TRY(upload(d, &d->pat_coeff, pat_coeff));
  GMG_TRY(upload(d, &d->pat_level, pat_level));
  d->n_loose = (int64_t)A.loose_cells.size();
  d->n_grp = A.n_groups;
  d->n_pat = A.n_patches;
  for (int l = 0; l < GMG_MAX_LEVELS; ++l) level_scales(h, l, d->level_scale[l], d->cell_h[l]);
  {
    // floating-point operations (FMA = 2) of one leaf-operator application
    const int n1 = k + 1;
    const double nc = ipow_d(n1, dim);
    double s0[3], h0[3];
    level_scales(h, 0, s0, h0);
    const bool iso = s0[0] == s0[1] && (dim == 2 || s0[1] == s0[2]);
    // a group of P^d cells: 1-D passes over (Pk+1)^(d-1) lines with the
    // P n1^2 - (P - 1) nonzeros of the assembled 1-D matrices
    auto group_flops = [&](int P) {
      const double ng = P * k + 1.0, ngn = std::pow(ng, dim), lines = std::pow(ng, dim - 1);
      const double nnz = P * n1 * n1 - (P - 1.0);
      if (dim == 3)  // isotropic: no per-direction scaling (one multiply per node)
        return lines * 2.0 * (2 * nnz + 3 * nnz + 2 * nnz) + ngn * (iso ? 2.0 + 1.0 : 2.0 * 3 + 2.0);
      return lines * 2.0 * (2 * nnz + 2 * nnz) + ngn * (2.0 * 2 + 2.0);
    };
    const double cell_flops = dim == 3 ? nc * (2.0 * (2 * n1 + 3 * n1 + 1 + 2 * n1 + 1 + 1) + 2.0)
                                       : nc * (2.0 * (2 * n1 + 2 * n1 + 1 + 1) + 2.0);
    const double ngn2 = ipow_d(2 * k + 1, dim), ngn4 = ipow_d(4 * k + 1, dim);
    const double nl = (double)A.loose_cells.size(), ng2 = (double)A.n_groups, ng4 = (double)A.n_patches;
    // hanging nodes: x_h = C_h x before, y += C_h^T y_h after (one FMA per entry each)
    const double nnzc = (double)A.hang_col.size();
    d->active_flops = cell_flops * nl + group_flops(2) * ng2 + group_flops(4) * ng4 + 4.0 * nnzc;
    d->active_bytes = 4.0 * (nc * nl + ngn2 * ng2 + ngn4 * ng4) + 9.0 * (nl + ng2 + ng4) +
                      24.0 * (double)A.n_unknowns + 2.0 * 5.0 * nnzc + 32.0 * (double)A.hang_key.size() +
                      16.0 * (double)A.hm_node.size();
  }
  GMG_TRY(dev_alloc(d, &d->r, A.n_unknowns));
  GMG_TRY(dev_alloc(d, &d->p, A.n_unknowns));
  GMG_TRY(dev_alloc(d, &d->Ap, A.n_unknowns));
  GMG_TRY(dev_alloc(d, &d->x_iter, A.n_unknowns));
  GMG_TRY(dev_alloc(d, &d->partials, kMaxReduceBlocks));
  GMG_TRY(dev_alloc(d, &d->counter, 1));
  GMG_CUDA_TRY(cudaMemset(d->counter, 0, sizeof(unsigned)));
  GMG_TRY(ensure_scalars(d, 4096));
  cudaStream_t s = d->stream;
  // inverse diagonals (FP64), eigenvalue estimates on each level l >= 1
  double* dinv64 = nullptr;
  if (d->prec == GMG_PREC_FP64) {
    dinv64 = (double*)d->dinv;
  } else {
    GMG_CUDA_TRY(cudaMalloc(&dinv64, ns * sizeof(double)));
  }
  GMG_CUDA_TRY(cudaMemsetAsync(dinv64, 0, ns * sizeof(double), s));
  for (int l = 1; l <= L; ++l)
    GMG_CUDA_TRY(launch_level_diag(dim, k, level_args(h, l), dinv64 + d->lv[l].offset, s));
  h.lambda.assign(L + 1, 0.0);
  int64_t max_slots = 0;
  for (int l = 1; l <= L; ++l) max_slots = std::max(max_slots, d->lv[l].n_slots);
  gmg_status st = GMG_OK;
  if (max_slots > 0) {
    double *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr;
    bool need = h.fixed_lambda.empty();
    if (need) {
      GMG_CUDA_TRY(cudaMalloc(&r, max_slots * sizeof(double)));
      GMG_CUDA_TRY(cudaMalloc(&z, max_slots * sizeof(double)));
      GMG_CUDA_TRY(cudaMalloc(&p, max_slots * sizeof(double)));
      GMG_CUDA_TRY(cudaMalloc(&Ap, max_slots * sizeof(double)));
    }
    for (int l = 1; l <= L && st == GMG_OK; ++l) {
      if (need) st = estimate_lambda(h, l, r, z, p, Ap, dinv64 + d->lv[l].offset, &h.lambda[l]);
      else h.lambda[l] = h.fixed_lambda[l];
    }
    cudaFree(r);
    cudaFree(z);
    cudaFree(p);
    cudaFree(Ap);
  }
  if (st != GMG_OK) return st;
  if (d->prec == GMG_PREC_FP32) {
    GMG_CUDA_TRY(launch_convert_d2f(ns, dinv64, (float*)d->dinv, s));
    GMG_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(dinv64);
  }
  for (int l = 1; l <= L; ++l) {
    LevelDev& D = d->lv[l];
    D.lambda = h.lambda[l];
    double a = h.params.eig_lo * D.lambda, b = h.params.eig_hi * D.lambda;
    D.theta = 0.5 * (a + b);
    D.delta = 0.5 * (b - a);
    D.sigma = D.theta / D.delta;
  }
  GMG_CUDA_TRY(cudaStreamSynchronize(s));
  h.setup_device_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return GMG_OK;
}

// ------------------------------------------------------------ coarse solve
// u_0 = A_0^{-1} g_0 by the dense inverse (or the dense Chebyshev operator),
// or by the unpreconditioned CG kernel; level-0 lattice slots in and out.
template <typename T>
static cudaError_t coarse(const Hier& h, const T* g0, T* u0, cudaStream_t s) {
  const DeviceState* d = h.dev;
  if (h.params.coarse_solver == GMG_COARSE_CG)
    return launch_coarse_cg<T>(d->n_coarse, d->coarse_slot, d->coarse_ptr, d->coarse_col, d->coarse_val,
                               d->coarse_nnz, h.params.coarse_tol, g0, u0, s);
  return launch_coarse_solve<T>(d->n_coarse, d->coarse_slot, d->coarse_inv, g0, u0, s);
}

// ------------------------------------------------------------- smoothing
// m Chebyshev updates on level l: x_{j+1} = x_j + rho_j rho_{j-1} (x_j - x_{j-1})
// + (2 rho_j / delta) D^{-1} (g - A x_j), x_1 = x_0 + D^{-1}(g - A x_0) / theta
// (Saad, Alg. 12.1, written as a three-term recurrence).  `cur` holds x_0;
// from_zero: x_0 = 0 and `other` must be zero on I slots (its S slots are
// written before they are read; x_prev = 0 is not read).  Returns the
// buffer that holds the result.
template <typename T>
static cudaError_t smooth(const Hier& h, int l, const T* g, const T* dinv, T* cur, T* other, bool from_zero,
                          T** result) {
  const LevelDev& D = h.dev->lv[l];
  cudaStream_t s = h.dev->stream;
  LevelArgs a = level_args(h, l);
  const int m = h.params.cheb_degree;
  double rho = 1.0 / D.sigma;
  cudaError_t e;
  // x (S and I), x_prev, g and the new x on S nodes; D^-1 is read only by
  // groups at coefficient jumps (the others recompute it)
  const double cheb_bytes = sizeof(T) * (4.0 * D.n_S + D.n_S_jump + D.n_I);
  // undamped Jacobi (Sec. 4.3): every step x <- x + D^{-1} (g - A x)
  const bool jacobi = h.params.smoother == GMG_SMOOTHER_JACOBI;
  const double first = jacobi ? 1.0 : 1.0 / D.theta;
  if (from_zero) {
    // x_1 = c D^{-1} g on the groups' own slots; ghost slots (I nodes) stay 0
    const int64_t owned = D.n_groups * ipow_h(2 * h.k, h.dim);
    Track t(h.dev, GMG_K_SMOOTH_FIRST, 3.0 * sizeof(T) * owned, 2.0 * owned);
    e = launch_scale_vec<T>(owned, dinv, g, (T)first, cur, s);
  } else {
    Track t(h.dev, GMG_K_CHEB, cheb_bytes, D.cheb_flops);
    e = launch_level_cheb<T>(h.dim, h.k, a, cur, nullptr, g, dinv, other, (T)0, (T)first, false, s);
    std::swap(cur, other);
  }
  if (e != cudaSuccess) return e;
  for (int j = 1; j < m; ++j) {
    double rho_new = 1.0 / (2.0 * D.sigma - rho);
    T c1 = jacobi ? (T)0 : (T)(rho_new * rho), c2 = jacobi ? (T)1 : (T)(2.0 * rho_new / D.delta);
    // from zero, x_prev = x_0 = 0 on S: passed as null instead of read
    const T* xprev = from_zero && j == 1 ? nullptr : other;
    Track t(h.dev, GMG_K_CHEB, xprev ? cheb_bytes : cheb_bytes - sizeof(T) * D.n_S, D.cheb_flops);
    e = launch_level_cheb<T>(h.dim, h.k, a, cur, xprev, g, dinv, other, c1, c2, false, s);
    if (e != cudaSuccess) return e;
    std::swap(cur, other);
    rho = rho_new;
  }
  *result = cur;
  return cudaSuccess;
}

// The V-cycle on the level vectors, Algorithm 2 in the local-smoothing form
// of Sec. 2.3: the level right-hand sides g are in place (the active
// residual at each unknown's home slot, zero elsewhere); the result ends in
// u_B, each unknown's value at its home slot.
template <typename T>
static gmg_status vcycle_levels(Hier& h) {
  DeviceState* d = h.dev;
  cudaStream_t s = d->stream;
  const int L = h.L;
  T* uA = (T*)d->uA;
  T* uB = (T*)d->uB;
  T* g = (T*)d->g;
  const T* dinv = (const T*)d->dinv;
  // u_A, u_B: the down-sweep needs zeros on I and ghost slots (the up-sweep's
  // prolongation sets them).  S slots need none: the first smoothing update
  // writes every stored slot of u_A and the second takes no x_prev, and
  // Dirichlet slots stay zero from setup.  So only levels with I nodes or
  // ghost blocks (and level 0) are cleared, in runs of consecutive levels.
  for (int l = 0; l <= L;) {
    if (!d->lv[l].zero_each_cycle) {
      ++l;
      continue;
    }
    int e = l;
    while (e + 1 <= L && d->lv[e + 1].zero_each_cycle) ++e;
    const int64_t a = d->lv[l].offset, b = d->lv[e].offset + d->lv[e].n_slots;
    GMG_CUDA_TRY(cudaMemsetAsync(uA + a, 0, (size_t)(b - a) * sizeof(T), s));
    GMG_CUDA_TRY(cudaMemsetAsync(uB + a, 0, (size_t)(b - a) * sizeof(T), s));
    l = e + 1;
  }
  const double kd = ipow_d(h.k, h.dim);
  // down-sweep: pre-smoothing on V^S from zero, residual on S u I, restriction
  for (int l = L; l >= 1; --l) {
    const LevelDev& D = d->lv[l];
    T* res = nullptr;
    GMG_CUDA_TRY(smooth<T>(h, l, g + D.offset, dinv + D.offset, uA + D.offset, uB + D.offset, true, &res));
    Track t(d, GMG_K_RESTRICT, sizeof(T) * (2.0 * (D.n_S + D.n_I) + 2.0 * kd * D.n_groups), 0.0);
    GMG_CUDA_TRY(launch_level_residual_restrict<T>(h.dim, h.k, level_args(h, l), res, g + D.offset,
                                                   g + d->lv[l - 1].offset, s));
  }
  // The smoother alternates buffers so that every level's final result (after
  // m pre- and m post-smoothing updates) ends in uB; the coarse solution goes
  // there too.
  {
    const double nc = (double)d->n_coarse;
    Track t(d, GMG_K_COARSE, 8.0 * nc * nc + 2.0 * sizeof(T) * nc, 2.0 * nc * nc);
    GMG_CUDA_TRY(coarse<T>(h, g, uB, s));
  }
  for (int l = 1; l <= L; ++l) {
    const LevelDev& D = d->lv[l];
    const int m = h.params.cheb_degree;
    T* pre = (m % 2 == 1) ? uA + D.offset : uB + D.offset;
    T* oth = (m % 2 == 1) ? uB + D.offset : uA + D.offset;
    {
      Track t(d, GMG_K_PROLONG, sizeof(T) * (kd * D.n_groups + 2.0 * D.n_S + 2.0 * D.n_I), 0.0);
      GMG_CUDA_TRY(launch_level_prolongate<T>(h.dim, h.k, level_args(h, l), uB + d->lv[l - 1].offset, pre, oth, s));
    }
    T* res = nullptr;
    GMG_CUDA_TRY(smooth<T>(h, l, g + D.offset, dinv + D.offset, pre, oth, false, &res));
    if (res != uB + D.offset) {
      set_error("internal: V-cycle result not in the final buffer");
      return GMG_EINVAL;
    }
  }
  return GMG_OK;
}

// z = B r (one V-cycle, gmg_vcycle); rz_out (device) receives r.z.
template <typename T>
static gmg_status vcycle_impl(Hier& h, const double* r, double* z, double* rz_out) {
  DeviceState* d = h.dev;
  cudaStream_t s = d->stream;
  GMG_CUDA_TRY(cudaMemsetAsync(d->g, 0, (size_t)h.total_slots * sizeof(T), s));
  {
    Track t(d, GMG_K_COPY_TO, (12.0 + sizeof(T)) * d->n_unknowns, 0.0);
    GMG_CUDA_TRY(launch_copy_to_mg<T>(d->n_unknowns, r, d->home, (T*)d->g, s));
  }
  GMG_TRY(vcycle_levels<T>(h));
  Track t(d, GMG_K_COPY_FROM, (20.0 + sizeof(T)) * d->n_unknowns, 2.0 * d->n_unknowns);
  GMG_CUDA_TRY(launch_copy_from_mg<T>(d->n_unknowns, (const T*)d->uB, d->home, r, z, d->partials, d->counter,
                                      rz_out, s));
  return GMG_OK;
}

static gmg_status vcycle_any(Hier& h, const double* r, double* z, double* rz_out) {
  if (h.dev->prec == GMG_PREC_FP32) return vcycle_impl<float>(h, r, z, rz_out);
  return vcycle_impl<double>(h, r, z, rz_out);
}

// A caller's canonical vector into the internal order (dst[j] = src[perm[j]])
// and an internal one back out.
static gmg_status to_internal(DeviceState* d, const double* src, double* dst, cudaStream_t s) {
  Track t(d, GMG_K_OTHER, 20.0 * d->n_unknowns, 0.0);
  GMG_CUDA_TRY(launch_perm(d->n_unknowns, d->perm, src, dst, false, s));
  return GMG_OK;
}
static gmg_status to_canonical(DeviceState* d, const double* src, double* dst, cudaStream_t s) {
  Track t(d, GMG_K_OTHER, 20.0 * d->n_unknowns, 0.0);
  GMG_CUDA_TRY(launch_perm(d->n_unknowns, d->perm, src, dst, true, s));
  return GMG_OK;
}

// ---------------------------------------------- CG passes around the V-cycle
// One preconditioned CG iteration in the order both solve modes use
// (Sec. 4.1: CG preconditioned by one V-cycle), with z = B r read from the
// level solutions and never stored:
//   V-cycle on g (filled by the previous pass), rz = r.z,
//   p = z + (rz / rz_old) p with Ap = 0, Ap = A p with pAp = p.Ap,
//   x += (rz / pAp) p, r -= (rz / pAp) Ap with rr = r.r and g = r at the home slots.
// With p = 0 and rz_old = 1 before the first iteration this is the textbook
// PCG recurrence.

// r = b (b may be r), bb = b.b, g = b at the home slots and 0 elsewhere
template <typename T>
static gmg_status cg_start_t(Hier& h, const double* b, double* bb) {
  DeviceState* d = h.dev;
  const int64_t n = d->n_unknowns;
  GMG_CUDA_TRY(cudaMemsetAsync(d->g, 0, (size_t)h.total_slots * sizeof(T), d->stream));
  Track t(d, GMG_K_COPY_TO, (20.0 + sizeof(T)) * n, 2.0 * n);
  GMG_CUDA_TRY(launch_cg_start<T>(n, b, d->home, d->r, (T*)d->g, d->partials, d->counter, bb, d->stream));
  return GMG_OK;
}

template <typename T>
static gmg_status cg_iteration_t(Hier& h, double* x, double* rz, const double* rz_old, double* pAp, double* rr) {
  DeviceState* d = h.dev;
  cudaStream_t s = d->stream;
  const int64_t n = d->n_unknowns;
  const T* u = (const T*)d->uB;
  GMG_TRY(vcycle_levels<T>(h));
  {
    Track t(d, GMG_K_COPY_FROM, (12.0 + sizeof(T)) * n, 2.0 * n);
    GMG_CUDA_TRY(launch_cg_rz<T>(n, u, d->home, d->r, d->partials, d->counter, rz, s));
  }
  {
    Track t(d, GMG_K_CG_P, (28.0 + sizeof(T)) * n, 2.0 * n);
    GMG_CUDA_TRY(launch_cg_p<T>(n, u, d->home, d->p, d->Ap, rz, rz_old, s));
  }
  {
    Track t(d, GMG_K_ACTIVE, d->active_bytes, d->active_flops);
    GMG_CUDA_TRY(launch_active_apply(h.dim, h.k, active_args(h), d->p, d->Ap, d->partials, d->counter, pAp, s));
  }
  GMG_CUDA_TRY(cudaMemsetAsync(d->g, 0, (size_t)h.total_slots * sizeof(T), s));
  Track t(d, GMG_K_CG_XR, (52.0 + sizeof(T)) * n, 6.0 * n);
  GMG_CUDA_TRY(launch_cg_xr<T>(n, x, d->r, d->p, d->Ap, d->home, (T*)d->g, rz, pAp, d->partials, d->counter, rr, s));
  return GMG_OK;
}

static gmg_status cg_start(Hier& h, const double* b, double* bb) {
  return h.dev->prec == GMG_PREC_FP32 ? cg_start_t<float>(h, b, bb) : cg_start_t<double>(h, b, bb);
}
static gmg_status cg_iteration(Hier& h, double* x, double* rz, const double* rz_old, double* pAp, double* rr) {
  return h.dev->prec == GMG_PREC_FP32 ? cg_iteration_t<float>(h, x, rz, rz_old, pAp, rr)
                                      : cg_iteration_t<double>(h, x, rz, rz_old, pAp, rr);
}

gmg_status device_vcycle(Hier& h, const double* r, double* z) {
  DeviceState* d = h.dev;
  GMG_TRY(ensure_scalars(d, 8));
  GMG_TRY(to_internal(d, r, d->r, d->stream));
  GMG_TRY(vcycle_any(h, d->r, d->p, d->scal + 1));
  return to_canonical(d, d->p, z, d->stream);
}

gmg_status device_apply(Hier& h, const double* x, double* y) {
  DeviceState* d = h.dev;
  GMG_TRY(to_internal(d, x, d->p, d->stream));
  GMG_CUDA_TRY(cudaMemsetAsync(d->Ap, 0, sizeof(double) * d->n_unknowns, d->stream));
  {
    Track t(d, GMG_K_ACTIVE, d->active_bytes, d->active_flops);
    GMG_CUDA_TRY(launch_active_apply(h.dim, h.k, active_args(h), d->p, d->Ap, d->partials, d->counter, nullptr,
                                     d->stream));
  }
  return to_canonical(d, d->Ap, y, d->stream);
}

gmg_status device_rhs(Hier& h, int kind, uint64_t seed, double* b) {
  DeviceState* d = h.dev;
  if (kind == GMG_RHS_RANDOM) {  // a function of the canonical index: written in place
    GMG_CUDA_TRY(launch_rhs_random(d->n_unknowns, seed, b, d->stream));
    return GMG_OK;
  }
  if (kind != GMG_RHS_SINE && kind != GMG_RHS_ONE) {
    set_error("gmg_assemble_rhs: unknown kind");
    return GMG_EINVAL;
  }
  GMG_CUDA_TRY(cudaMemsetAsync(d->r, 0, sizeof(double) * d->n_unknowns, d->stream));
  GMG_CUDA_TRY(launch_rhs_sine(h.dim, h.k, active_args(h), d->cell_coords, d->r, kind == GMG_RHS_ONE, d->stream));
  return to_canonical(d, d->r, b, d->stream);
}

// Preconditioned CG (x0 = 0), stream mode: the host reads the scalars of
// every iteration and decides whether to go on.  Scalars live on the device:
// slot 0 = b.b, slot 1 = 1 (r.z before the first iteration), slots 2+3i ..
// 4+3i = (r_i.z_i, p_i.A p_i, r_{i+1}.r_{i+1}) of iteration i.
static gmg_status solve_stream(Hier& h, const double* b, double* x, double tol, int max_iter, int fixed_iterations,
                               gmg_stats* st) {
  DeviceState* d = h.dev;
  cudaStream_t s = d->stream;
  const int64_t n = d->n_unknowns;
  const int limit = fixed_iterations > 0 ? fixed_iterations : max_iter;
  GMG_TRY(ensure_scalars(d, 3 * limit + 8));
  double* S = d->scal;
  double* H = d->scal_host;
  double* xi = d->x_iter;  // the iterate in the internal order
  GMG_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  GMG_CUDA_TRY(cudaMemsetAsync(xi, 0, sizeof(double) * n, s));
  GMG_CUDA_TRY(cudaMemsetAsync(d->p, 0, sizeof(double) * n, s));
  H[1] = 1.0;
  GMG_CUDA_TRY(cudaMemcpyAsync(S + 1, H + 1, sizeof(double), cudaMemcpyHostToDevice, s));
  GMG_TRY(to_internal(d, b, d->r, s));
  GMG_TRY(cg_start(h, d->r, S));
  GMG_CUDA_TRY(cudaMemcpyAsync(H, S, sizeof(double), cudaMemcpyDeviceToHost, s));
  GMG_CUDA_TRY(cudaStreamSynchronize(s));
  const double bb = H[0];
  gmg_stats stats;
  stats.iterations = 0;
  stats.converged = 0;
  stats.rel_residual = bb > 0 ? 1.0 : 0.0;
  stats.norm_b = std::sqrt(bb);
  if (!(bb > 0.0)) {
    stats.converged = 1;
    if (st) *st = stats;
    if (std::isnan(bb)) {
      set_error("right-hand side contains NaN");
      return GMG_ENAN;
    }
    return GMG_OK;
  }
  gmg_status result = GMG_ENOTCONV;
  for (int it = 0; it < limit; ++it) {
    double* base = S + 2 + 3 * it;
    const double* rz_old = it == 0 ? S + 1 : base - 3;
    GMG_TRY(cg_iteration(h, xi, base, rz_old, base + 1, base + 2));
    GMG_CUDA_TRY(cudaMemcpyAsync(H + 2 + 3 * it, base, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GMG_CUDA_TRY(cudaStreamSynchronize(s));
    const double rz = H[2 + 3 * it], pAp = H[3 + 3 * it], rr = H[4 + 3 * it];
    stats.iterations = it + 1;
    stats.rel_residual = std::sqrt(rr / bb);
    if (std::isnan(rz) || std::isnan(pAp) || std::isnan(rr) || std::isinf(rr)) {
      set_error("NaN/Inf in a CG scalar");
      result = GMG_ENAN;
      break;
    }
    if (!(pAp > 0.0)) {
      set_error("CG breakdown: p.Ap <= 0");
      result = GMG_EBREAKDOWN;
      break;
    }
    if (fixed_iterations > 0) {
      if (it + 1 == fixed_iterations) {
        stats.converged = stats.rel_residual <= tol;
        result = GMG_OK;
        break;
      }
    } else if (stats.rel_residual <= tol) {
      stats.converged = 1;
      result = GMG_OK;
      break;
    }
  }
  GMG_TRY(to_canonical(d, xi, x, s));
  GMG_CUDA_TRY(cudaStreamSynchronize(s));
  if (result == GMG_ENOTCONV) set_error("CG did not converge within max_iter");
  if (st) *st = stats;
  return result;
}

// ------------------------------------------------------ graph-mode CG
// The iteration of solve_stream (cg_iteration) as the body of a conditional
// WHILE node whose condition a check kernel sets after each pass, with the
// stream mode's stopping rules: a solve is one graph launch and one host
// synchronisation, and performs exactly the stream-mode operations.

// Ends a capture that failed and passes its status on.
static gmg_status abandon_capture(cudaStream_t s, gmg_status st) {
  cudaGraph_t g = nullptr;
  cudaStreamEndCapture(s, &g);
  cudaGetLastError();
  return st;
}

static gmg_status capture_prelude(Hier& h, cudaGraph_t g, cudaGraphConditionalHandle* loop, cudaGraph_t* body) {
  DeviceState* d = h.dev;
  cudaStream_t s = d->stream;
  const int64_t n = d->n_unknowns;
  GMG_CUDA_TRY(cudaMemsetAsync(d->x_iter, 0, sizeof(double) * n, s));
  GMG_CUDA_TRY(cudaMemsetAsync(d->p, 0, sizeof(double) * n, s));
  GMG_TRY(cg_start(h, d->r, &d->ctl->bb));  // b was copied into r before the launch
  GMG_CUDA_TRY(cudaGraphConditionalHandleCreate(loop, g, 0, cudaGraphCondAssignDefault));
  {
    Track t(d, GMG_K_OTHER, 0.0, 0.0);
    GMG_CUDA_TRY(launch_cg_graph_init(d->ctl, *loop, s));
  }
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  GMG_CUDA_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = *loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  GMG_CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
  *body = cp.conditional.phGraph_out[0];
  GMG_CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return GMG_OK;
}

static gmg_status capture_body(Hier& h, cudaGraphConditionalHandle loop) {
  DeviceState* d = h.dev;
  cudaStream_t s = d->stream;
  GraphCtl* c = d->ctl;
  GMG_TRY(cg_iteration(h, d->x_iter, &c->rz, &c->rz_old, &c->pAp, &c->rr));
  Track t(d, GMG_K_OTHER, 0.0, 0.0);
  GMG_CUDA_TRY(launch_cg_graph_check(c, loop, s));
  return GMG_OK;
}

static gmg_status build_solve_graph(Hier& h) {
  DeviceState* d = h.dev;
  if (!d->ctl) GMG_TRY(dev_alloc(d, &d->ctl, 1));
  if (!d->ctl_host) GMG_CUDA_TRY(cudaMallocHost(&d->ctl_host, sizeof(GraphCtl)));
  // capture on a private stream: the context's stream may be the legacy
  // default stream, which cannot be captured
  if (!d->cap_stream) GMG_CUDA_TRY(cudaStreamCreateWithFlags(&d->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  GMG_CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaStream_t user = d->stream;
  d->stream = d->cap_stream;
  d->cg_pre = Tally();
  d->cg_body = Tally();
  cudaGraphConditionalHandle loop = 0;
  cudaGraph_t body = nullptr;
  gmg_status st = GMG_OK;
  cudaError_t e = cudaStreamBeginCaptureToGraph(d->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    set_error(std::string("graph capture: ") + cudaGetErrorString(e));
    st = GMG_ECUDA;
  }
  if (st == GMG_OK) {
    d->cap = &d->cg_pre;
    st = capture_prelude(h, g, &loop, &body);
    if (st != GMG_OK) {
      st = abandon_capture(d->stream, st);
    } else {
      cudaGraph_t out = nullptr;
      e = cudaStreamEndCapture(d->stream, &out);
      if (e != cudaSuccess) {
        set_error(std::string("graph capture: ") + cudaGetErrorString(e));
        st = GMG_ECUDA;
      }
    }
  }
  if (st == GMG_OK) {
    e = cudaStreamBeginCaptureToGraph(d->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      set_error(std::string("graph capture: ") + cudaGetErrorString(e));
      st = GMG_ECUDA;
    } else {
      d->cap = &d->cg_body;
      st = capture_body(h, loop);
      if (st != GMG_OK) {
        st = abandon_capture(d->stream, st);
      } else {
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(d->stream, &out);
        if (e != cudaSuccess) {
          set_error(std::string("graph capture: ") + cudaGetErrorString(e));
          st = GMG_ECUDA;
        }
      }
    }
  }
  d->cap = nullptr;
  d->stream = user;
  cudaGraphExec_t ex = nullptr;
  if (st == GMG_OK) {
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
      set_error(std::string("graph instantiation: ") + cudaGetErrorString(e));
      st = GMG_ECUDA;
    }
  }
  if (st != GMG_OK) {
    cudaGraphDestroy(g);
    return st;
  }
  d->cg_graph = g;
  d->cg_exec = ex;
  return GMG_OK;
}

static void add_tally(Profile& p, const Tally& t, uint64_t times) {
  for (int k = 0; k < GMG_NUM_KERNEL_KINDS; ++k) {
    p.launches[k] += t.launches[k] * times;
    p.bytes[k] += t.bytes[k] * (double)times;
    p.flops[k] += t.flops[k] * (double)times;
  }
}

// Enqueue one graph-mode solve on stream s (no synchronisation); the status
// and scalars land in the pinned control mirror.
static gmg_status enqueue_graph_solve(Hier& h, const double* b, double* x, double tol, int max_iter,
                                      int fixed_iterations, cudaStream_t s) {
  DeviceState* d = h.dev;
  if (!d->cg_exec) GMG_TRY(build_solve_graph(h));
  GraphCtl* c = d->ctl_host;
  *c = GraphCtl();
  c->tol = tol;
  c->limit = fixed_iterations > 0 ? fixed_iterations : max_iter;
  c->fixed = fixed_iterations > 0 ? fixed_iterations : 0;
  c->status = GS_RUNNING;
  GMG_TRY(to_internal(d, b, d->r, s));
  GMG_CUDA_TRY(cudaMemcpyAsync(d->ctl, c, sizeof(GraphCtl), cudaMemcpyHostToDevice, s));
  GMG_CUDA_TRY(cudaGraphLaunch(d->cg_exec, s));
  GMG_TRY(to_canonical(d, d->x_iter, x, s));
  GMG_CUDA_TRY(cudaMemcpyAsync(c, d->ctl, sizeof(GraphCtl), cudaMemcpyDeviceToHost, s));
  return GMG_OK;
}

// After the stream has been synchronised: statistics and status of the solve.
static gmg_status finish_graph_solve(Hier& h, double tol, gmg_stats* st) {
  DeviceState* d = h.dev;
  const GraphCtl* c = d->ctl_host;
  add_tally(d->prof, d->cg_pre, 1);
  add_tally(d->prof, d->cg_body, (uint64_t)std::max(c->it, 0));
  gmg_stats stats;
  stats.iterations = c->it;
  stats.norm_b = std::sqrt(c->bb);
  stats.rel_residual = c->it > 0 ? std::sqrt(c->rr / c->bb) : (c->bb > 0 ? 1.0 : 0.0);
  stats.converged = c->status == GS_DONE && (c->it == 0 || stats.rel_residual <= tol);
  if (st) *st = stats;
  switch (c->status) {
    case GS_DONE:
      return GMG_OK;
    case GS_NOTCONV:
      set_error("CG did not converge within max_iter");
      return GMG_ENOTCONV;
    case GS_NAN:
      set_error(c->it == 0 ? "right-hand side contains NaN" : "NaN/Inf in a CG scalar");
      return GMG_ENAN;
    case GS_BREAKDOWN:
      set_error("CG breakdown: p.Ap <= 0");
      return GMG_EBREAKDOWN;
    default:
      set_error("internal: graph-mode CG ended without a status");
      return GMG_ECUDA;
  }
}

static gmg_status solve_graph(Hier& h, const double* b, double* x, double tol, int max_iter, int fixed_iterations,
                              gmg_stats* st) {
  cudaStream_t s = h.dev->stream;
  GMG_TRY(enqueue_graph_solve(h, b, x, tol, max_iter, fixed_iterations, s));
  GMG_CUDA_TRY(cudaStreamSynchronize(s));
  return finish_graph_solve(h, tol, st);
}

// Asynchronous graph-mode solve on the context stream: enqueue, then poll.
gmg_status device_solve_async(Hier& h, const double* b, double* x, double tol, int max_iter) {
  DeviceState* d = h.dev;
  if (d->prof.timing) {
    set_error("asynchronous solves run without per-launch timing");
    return GMG_EINVAL;
  }
  if (!d->done) GMG_CUDA_TRY(cudaEventCreateWithFlags(&d->done, cudaEventDisableTiming));
  GMG_TRY(enqueue_graph_solve(h, b, x, tol, max_iter, 0, d->stream));
  GMG_CUDA_TRY(cudaEventRecord(d->done, d->stream));
  d->async_tol = tol;
  d->async_pending = true;
  return GMG_OK;
}

gmg_status device_solve_poll(Hier& h, int wait, int* ready, gmg_stats* st, gmg_status* status) {
  DeviceState* d = h.dev;
  if (!d->async_pending) {
    set_error("no asynchronous solve pending");
    return GMG_EINVAL;
  }
  cudaError_t e = wait ? cudaEventSynchronize(d->done) : cudaEventQuery(d->done);
  if (e == cudaErrorNotReady) {
    *ready = 0;
    return GMG_OK;
  }
  GMG_CUDA_TRY(e);
  *ready = 1;
  d->async_pending = false;
  *status = finish_graph_solve(h, d->async_tol, st);
  return GMG_OK;
}

// Independent solves at once: the problems' solve graphs go round-robin onto
// a pool of streams, so small problems share the GPU; one wait at the end.
// Each problem starts after the work already queued on its own stream.
gmg_status device_solve_batch(Hier* const* hs, const double* const* b, double* const* x, int n, double tol,
                              int max_iter, int n_streams, gmg_stats* st, gmg_status* status) {
  static std::mutex pool_mutex;
  static std::vector<cudaStream_t> pool;
  static std::vector<cudaEvent_t> ready;
  std::lock_guard<std::mutex> lock(pool_mutex);
  while ((int)pool.size() < n_streams) {
    cudaStream_t s = nullptr;
    GMG_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    pool.push_back(s);
  }
  while ((int)ready.size() < n) {
    cudaEvent_t e = nullptr;
    GMG_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ready.push_back(e);
  }
  for (int i = 0; i < n; ++i)
    if (hs[i]->dev->prof.timing) {
      set_error("batched solves run without per-launch timing (gmg_profile_reset with timing off)");
      return GMG_EINVAL;
    }
  // graphs are captured (and their buffers allocated) before any launch
  for (int i = 0; i < n; ++i)
    if (!hs[i]->dev->cg_exec) GMG_TRY(build_solve_graph(*hs[i]));
  gmg_status first_error = GMG_OK;
  std::vector<char> launched(n, 0);
  for (int i = 0; i < n; ++i) {
    cudaStream_t s = pool[i % n_streams];
    GMG_CUDA_TRY(cudaEventRecord(ready[i], hs[i]->dev->stream));
    GMG_CUDA_TRY(cudaStreamWaitEvent(s, ready[i], 0));
    gmg_status e = enqueue_graph_solve(*hs[i], b[i], x[i], tol, max_iter, 0, s);
    if (e != GMG_OK) {
      status[i] = e;
      if (first_error == GMG_OK) first_error = e;
      continue;
    }
    launched[i] = 1;
  }
  for (int k = 0; k < n_streams && k < n; ++k) GMG_CUDA_TRY(cudaStreamSynchronize(pool[k]));
  for (int i = 0; i < n; ++i)
    if (launched[i]) status[i] = finish_graph_solve(*hs[i], tol, st ? st + i : nullptr);
  return first_error;
}

// Graph mode unless it is switched off or per-kernel timing is on (the
// events that time single launches exist only in stream mode).
gmg_status device_solve(Hier& h, const double* b, double* x, double tol, int max_iter, int fixed_iterations,
                        gmg_stats* st) {
  if (h.params.solve_graph && !h.dev->prof.timing) return solve_graph(h, b, x, tol, max_iter, fixed_iterations, st);
  return solve_stream(h, b, x, tol, max_iter, fixed_iterations, st);
}

// ------------------------------------------------- level operations (tests)
template <typename T>
static gmg_status level_apply_t(Hier& h, int l, const void* x, void* y) {
  GMG_CUDA_TRY(launch_level_cheb<T>(h.dim, h.k, level_args(h, l), (const T*)x, nullptr, nullptr, nullptr, (T*)y,
                                    (T)0, (T)0, true, h.dev->stream));
  return GMG_OK;
}
gmg_status device_level_apply(Hier& h, int l, const void* x, void* y) {
  return h.dev->prec == GMG_PREC_FP32 ? level_apply_t<float>(h, l, x, y) : level_apply_t<double>(h, l, x, y);
}

gmg_status device_level_residual_restrict(Hier& h, int l, const void* u, const void* g, void* gc) {
  cudaError_t e = h.dev->prec == GMG_PREC_FP32
                      ? launch_level_residual_restrict<float>(h.dim, h.k, level_args(h, l), (const float*)u,
                                                              (const float*)g, (float*)gc, h.dev->stream)
                      : launch_level_residual_restrict<double>(h.dim, h.k, level_args(h, l), (const double*)u,
                                                               (const double*)g, (double*)gc, h.dev->stream);
  GMG_CUDA_TRY(e);
  return GMG_OK;
}

gmg_status device_level_prolongate(Hier& h, int l, const void* uc, void* u, void* u2) {
  cudaError_t e = h.dev->prec == GMG_PREC_FP32
                      ? launch_level_prolongate<float>(h.dim, h.k, level_args(h, l), (const float*)uc, (float*)u,
                                                       (float*)u2, h.dev->stream)
                      : launch_level_prolongate<double>(h.dim, h.k, level_args(h, l), (const double*)uc, (double*)u,
                                                        (double*)u2, h.dev->stream);
  GMG_CUDA_TRY(e);
  return GMG_OK;
}

template <typename T>
static gmg_status level_smooth_t(Hier& h, int l, const void* g, void* u, void* tmp, int from_zero) {
  DeviceState* d = h.dev;
  const LevelDev& D = d->lv[l];
  const T* dinv = (const T*)d->dinv + D.offset;
  T* res = nullptr;
  if (from_zero) GMG_CUDA_TRY(cudaMemsetAsync(tmp, 0, D.n_slots * sizeof(T), d->stream));
  else GMG_CUDA_TRY(cudaMemcpyAsync(tmp, u, D.n_slots * sizeof(T), cudaMemcpyDeviceToDevice, d->stream));
  GMG_CUDA_TRY(smooth<T>(h, l, (const T*)g, dinv, (T*)u, (T*)tmp, from_zero != 0, &res));
  if (res != (T*)u)
    GMG_CUDA_TRY(cudaMemcpyAsync(u, res, D.n_slots * sizeof(T), cudaMemcpyDeviceToDevice, d->stream));
  return GMG_OK;
}
gmg_status device_level_smooth(Hier& h, int l, const void* g, void* u, void* tmp, int from_zero) {
  return h.dev->prec == GMG_PREC_FP32 ? level_smooth_t<float>(h, l, g, u, tmp, from_zero)
                                      : level_smooth_t<double>(h, l, g, u, tmp, from_zero);
}

gmg_status device_level_inv_diag(Hier& h, int l, void* out) {
  DeviceState* d = h.dev;
  const LevelDev& D = d->lv[l];
  size_t esz = d->prec == GMG_PREC_FP32 ? sizeof(float) : sizeof(double);
  GMG_CUDA_TRY(cudaMemcpyAsync(out, (const unsigned char*)d->dinv + D.offset * esz, D.n_slots * esz,
                               cudaMemcpyDeviceToDevice, d->stream));
  return GMG_OK;
}

gmg_status device_coarse_solve(Hier& h, const void* g0, void* u0) {
  DeviceState* d = h.dev;
  cudaError_t e = d->prec == GMG_PREC_FP32 ? coarse<float>(h, (const float*)g0, (float*)u0, d->stream)
                                           : coarse<double>(h, (const double*)g0, (double*)u0, d->stream);
  GMG_CUDA_TRY(e);
  return GMG_OK;
}

}  // namespace gmg
