// Host construction of the multigrid hierarchy (setup; Sec. 2.3 and Sec. 1).
//
// Level l >= 1 consists of all cells of level l (leaves or not).  They come
// in sibling groups -- the 2^d children of a refined cell of level l-1 --
// and each group is stored as one block of (2k)^d nodes (see LevelHost).
// A node of level l is
//   D  if it lies on the boundary of the brick (value fixed to 0),
//   I  if some level-l lattice cell inside the brick whose closure contains
//      it does not exist (refinement edge, Sec. 2.3, Fig. 1),
//   S  otherwise (strictly inside the level-l cells).
// Because the level-l lattice cells touching a node are children of the
// refined level-(l-1) positions touching it, the class follows from the
// states of the 3^d parent positions around a group.
//
// The leaf mesh: its nodes are the nodes of the leaf cells; a node lying in
// the closure of a coarser leaf without being one of its nodes is hanging
// and takes the value of that leaf's interpolant (Sec. 1).  Unknowns are the
// leaf nodes that are neither hanging nor on the boundary, in key order.
// Each unknown is copied to one level only, its home level: the coarsest
// level of the leaves that contain it, where it is an S node.
#include <omp.h>

#include <algorithm>
#include <chrono>
#include <memory>
#include <cmath>
#include <numeric>
#include <stdexcept>
#include <unordered_set>

#include "gmg_internal.h"

namespace gmg {

// ------------------------------------------------------------- 1-D tables
static void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  // Gauss-Legendre on [0, 1] for n = 1..3 (exact to degree 2n-1)
  x.clear();
  w.clear();
  if (n == 1) {
    x = {0.5};
    w = {1.0};
  } else if (n == 2) {
    double a = 0.5 / std::sqrt(3.0);
    x = {0.5 - a, 0.5 + a};
    w = {0.5, 0.5};
  } else if (n == 3) {
    double a = 0.5 * std::sqrt(0.6);
    x = {0.5 - a, 0.5, 0.5 + a};
    w = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  } else {
    throw std::runtime_error("gauss_rule: unsupported n");
  }
}

static double lagrange(int k, int j, double t) {
  double v = 1.0;
  for (int m = 0; m <= k; ++m)
    if (m != j) v *= (t - (double)m / k) / ((double)(j - m) / k);
  return v;
}

static double lagrange_d(int k, int j, double t) {
  double s = 0.0;
  for (int i = 0; i <= k; ++i) {
    if (i == j) continue;
    double v = 1.0 / ((double)(j - i) / k);
    for (int m = 0; m <= k; ++m)
      if (m != j && m != i) v *= (t - (double)m / k) / ((double)(j - m) / k);
    s += v;
  }
  return s;
}

void reference_1d(int k, std::vector<double>& M, std::vector<double>& K, std::vector<double>& E) {
  int n = k + 1;
  std::vector<double> xq, wq;
  gauss_rule(n, xq, wq);
  M.assign(n * n, 0.0);
  K.assign(n * n, 0.0);
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        M[i * n + j] += wq[q] * lagrange(k, i, xq[q]) * lagrange(k, j, xq[q]);
        K[i * n + j] += wq[q] * lagrange_d(k, i, xq[q]) * lagrange_d(k, j, xq[q]);
      }
  // parent basis at the 2k+1 child nodes of the parent interval
  E.assign((2 * k + 1) * n, 0.0);
  for (int r = 0; r <= 2 * k; ++r)
    for (int j = 0; j < n; ++j) {
      double v = lagrange(k, j, (double)r / (2 * k));
      E[r * n + j] = std::fabs(v) < 1e-15 ? 0.0 : v;
    }
}

bool spd_inverse(std::vector<double>& A, int64_t n) {
  // Cholesky A = L L^T in place (lower), then A^{-1} = L^-T L^-1.
  std::vector<double> Lm(A);
  for (int64_t j = 0; j < n; ++j) {
    double s = Lm[j * n + j];
    for (int64_t p = 0; p < j; ++p) s -= Lm[j * n + p] * Lm[j * n + p];
    if (!(s > 0.0)) return false;
    double d = std::sqrt(s);
    Lm[j * n + j] = d;
#pragma omp parallel for if (n > 256)
    for (int64_t i = j + 1; i < n; ++i) {
      double t = Lm[i * n + j];
      for (int64_t p = 0; p < j; ++p) t -= Lm[i * n + p] * Lm[j * n + p];
      Lm[i * n + j] = t / d;
    }
  }
  // invert L (lower triangular) column by column
  std::vector<double> Li(n * n, 0.0);
#pragma omp parallel for if (n > 256)
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = c; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int64_t p = c; p < i; ++p) t -= Lm[i * n + p] * Li[p * n + c];
      Li[i * n + c] = t / Lm[i * n + i];
    }
  }
  // A^{-1} = Li^T Li
#pragma omp parallel for if (n > 256)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double t = 0.0;
      for (int64_t p = std::max(i, j); p < n; ++p) t += Li[p * n + i] * Li[p * n + j];
      A[i * n + j] = t;
    }
  return true;
}

// smallest (largest = false) or largest eigenvalue of the symmetric
// tridiagonal (diag a, off-diagonal b) by Sturm-sequence bisection on a
// Gershgorin interval
static double tridiag_extreme_eig(const std::vector<double>& a, const std::vector<double>& b, bool largest);

double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  return tridiag_extreme_eig(a, b, true);
}

static double tridiag_extreme_eig(const std::vector<double>& a, const std::vector<double>& b, bool largest) {
  size_t m = a.size();
  if (m == 0) return 0.0;
  double lo = a[0], hi = a[0];
  for (size_t i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // number of eigenvalues < x
    int cnt = 0;
    double d = 1.0;
    for (size_t i = 0; i < m; ++i) {
      double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      d = a[i] - x - (i > 0 ? bb / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++cnt;
    }
    return cnt;
  };
  const int want = largest ? (int)m : 1;  // eigenvalues below the answer's upper bracket
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= want) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

void chebyshev_coarse_operator(const std::vector<double>& A, int64_t n, double tol, std::vector<double>& C,
                               int& degree, double range[2]) {
  std::vector<double> dinv(n);
  for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / A[i * n + i];
  auto matvec = [&](const std::vector<double>& x, std::vector<double>& y) {
    for (int64_t i = 0; i < n; ++i) {
      double t = 0.0;
      for (int64_t j = 0; j < n; ++j) t += A[i * n + j] * x[j];
      y[i] = t;
    }
  };
  // Jacobi-PCG on A y = b0 (the start pattern of the eigenvalue estimate) to
  // the relative unpreconditioned residual tol; Lanczos tridiagonal
  std::vector<double> r(n), z(n), p(n), Ap(n);
  double nb = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    r[i] = -5.5 + (double)(i % 12);
    nb += r[i] * r[i];
  }
  nb = std::sqrt(nb);
  for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i], p[i] = z[i];
  double rz = 0.0;
  for (int64_t i = 0; i < n; ++i) rz += r[i] * z[i];
  std::vector<double> alphas, betas;
  for (int64_t j = 0; j < n; ++j) {
    matvec(p, Ap);
    double pAp = 0.0;
    for (int64_t i = 0; i < n; ++i) pAp += p[i] * Ap[i];
    const double alpha = rz / pAp;
    alphas.push_back(alpha);
    double rr = 0.0;
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * Ap[i], rr += r[i] * r[i];
    if (std::sqrt(rr) <= tol * nb || j == n - 1) break;
    double rz_new = 0.0;
    for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i], rz_new += r[i] * z[i];
    const double beta = rz_new / rz;
    betas.push_back(beta);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
  }
  const size_t m = alphas.size();
  std::vector<double> ta(m), tb(m > 0 ? m - 1 : 0);
  for (size_t j = 0; j < m; ++j) {
    ta[j] = 1.0 / alphas[j] + (j > 0 ? betas[j - 1] / alphas[j - 1] : 0.0);
    if (j + 1 < m) tb[j] = std::sqrt(betas[j]) / alphas[j];
  }
  const double lmin = tridiag_extreme_eig(ta, tb, false), lmax = tridiag_extreme_eig(ta, tb, true);
  const double a = lmin, b = 1.2 * lmax;
  range[0] = a;
  range[1] = b;
  const double kappa = b / a, q = (std::sqrt(kappa) + 1.0) / (std::sqrt(kappa) - 1.0);
  degree = (int)std::ceil(std::log(2.0 / tol) / std::log(q));
  if (degree < 1) degree = 1;
  // the iteration from zero (Saad, Alg. 12.1, as the smoother) applied to
  // every unit vector at once: X = sum of updates, R = I - A X
  const double theta = 0.5 * (a + b), delta = 0.5 * (b - a), sigma = theta / delta;
  std::vector<double> X((size_t)n * n, 0.0), R((size_t)n * n, 0.0), D((size_t)n * n), AD((size_t)n * n);
  for (int64_t i = 0; i < n; ++i) R[i * n + i] = 1.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) D[i * n + j] = dinv[i] * R[i * n + j] / theta;
  double rho = 1.0 / sigma;
  for (int step = 0; step < degree; ++step) {
    for (size_t e = 0; e < X.size(); ++e) X[e] += D[e];
    if (step == degree - 1) break;
#pragma omp parallel for if (n > 128)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double t = 0.0;
        for (int64_t k2 = 0; k2 < n; ++k2) t += A[i * n + k2] * D[k2 * n + j];
        AD[i * n + j] = t;
      }
    for (size_t e = 0; e < R.size(); ++e) R[e] -= AD[e];
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j)
        D[i * n + j] = rho_new * rho * D[i * n + j] + (2.0 * rho_new / delta) * (dinv[i] * R[i * n + j]);
    rho = rho_new;
  }
  C.swap(X);
}

// ---------------------------------------------------------------- helpers
static inline int ipow(int b, int e) {
  int r = 1;
  while (e--) r *= b;
  return r;
}

// LSD radix sort of n keys in place, 16-bit digits, skipping digits above
// the largest key; `scratch` holds n keys (contents ignored)
static void radix_sort_u64(uint64_t* v, uint64_t* scratch, size_t n) {
  if (n == 0) return;
  uint64_t mx = 0;
#pragma omp parallel for reduction(max : mx)
  for (size_t i = 0; i < n; ++i) mx = std::max(mx, v[i]);
  int bits = 0;
  while (bits < 64 && (mx >> bits)) bits += 16;
  const int nt = omp_get_max_threads();
  std::vector<size_t> hist((size_t)nt * 65536);
  uint64_t* src = v;
  uint64_t* dst = scratch;
  for (int shift = 0; shift < bits; shift += 16) {
    std::fill(hist.begin(), hist.end(), 0);
#pragma omp parallel num_threads(nt)
    {
      int t = omp_get_thread_num();
      size_t b = n * t / nt, e = n * (t + 1) / nt;
      size_t* h = &hist[(size_t)t * 65536];
      for (size_t i = b; i < e; ++i) ++h[(src[i] >> shift) & 0xFFFF];
    }
    size_t sum = 0;
    for (int d = 0; d < 65536; ++d)
      for (int t = 0; t < nt; ++t) {
        size_t c = hist[(size_t)t * 65536 + d];
        hist[(size_t)t * 65536 + d] = sum;
        sum += c;
      }
#pragma omp parallel num_threads(nt)
    {
      int t = omp_get_thread_num();
      size_t b = n * t / nt, e = n * (t + 1) / nt;
      size_t* h = &hist[(size_t)t * 65536];
      for (size_t i = b; i < e; ++i) dst[h[(src[i] >> shift) & 0xFFFF]++] = src[i];
    }
    std::swap(src, dst);
  }
  if (src != v) {
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < n; ++i) v[i] = src[i];
  }
}

// a buffer of n keys that is not zero-filled (every element is written before it is read)
static std::unique_ptr<uint64_t[]> raw_keys(size_t n) { return std::unique_ptr<uint64_t[]>(new uint64_t[n]); }

void parallel_sort_u64(std::vector<uint64_t>& v) {
  std::unique_ptr<uint64_t[]> tmp = raw_keys(v.size());
  radix_sort_u64(v.data(), tmp.get(), v.size());
}

static inline int64_t lower_index(const std::vector<uint64_t>& keys, uint64_t k) {
  auto it = std::lower_bound(keys.begin(), keys.end(), k);
  if (it == keys.end() || *it != k) return -1;
  return it - keys.begin();
}

// Lookup in the sorted node-key array through row offsets: keys are
// (z << 42) | (y << 21) | x, so all keys of one lattice row (z, y) are
// contiguous; a search touches only that row.
struct RowIndex {
  const std::vector<uint64_t>* keys = nullptr;
  int64_t ny = 1;
  std::vector<int64_t> start;  // (nz * ny + 1) row offsets
  void build(const std::vector<uint64_t>& k, int64_t nz, int64_t ny_) {
    keys = &k;
    ny = ny_;
    const int64_t nr = nz * ny;
    start.assign((size_t)(nr + 1), 0);
    // the keys are sorted: row r starts at the first key >= (z << 42) | (y << 21)
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nr; ++r) {
      const uint64_t first = ((uint64_t)(r / ny) << 42) | ((uint64_t)(r % ny) << 21);
      start[(size_t)r] = std::lower_bound(k.begin(), k.end(), first) - k.begin();
    }
    start[(size_t)nr] = (int64_t)k.size();
  }
  int64_t row(uint64_t v) const { return (int64_t)(v >> 42) * ny + (int64_t)((v >> 21) & ((1u << 21) - 1)); }
  int64_t find(uint64_t v) const {
    const int64_t r = row(v);
    if (r < 0 || r + 1 >= (int64_t)start.size()) return -1;
    auto b = keys->begin() + start[(size_t)r], e = keys->begin() + start[(size_t)r + 1];
    auto it = std::lower_bound(b, e, v);
    if (it == e || *it != v) return -1;
    return it - keys->begin();
  }
};

// ------------------------------------------------------------------ build
void build_host_hierarchy(Hier& h, const Forest& f) {
  auto t0 = std::chrono::steady_clock::now();
  // wall time of the build phases (gmg_info.setup_phase_s)
  auto last = t0;
  auto phase_mark = [&](int ph) {
    const auto now = std::chrono::steady_clock::now();
    if (ph > 0) h.setup_phase_s[ph - 1] = std::chrono::duration<double>(now - last).count();
    last = now;
  };
  phase_mark(0);
  const int dim = f.dim, k = h.k;
  h.dim = dim;
  for (int d = 0; d < 3; ++d) {
    h.n0[d] = f.n0[d];
    h.lo[d] = f.lo[d];
    h.hi[d] = d < dim ? f.hi[d] : f.lo[d] + 1.0;
  }
  const int L = f.num_levels() - 1;
  h.L = L;
  if (L > 20) throw std::runtime_error("more than 20 levels");
  const int NO = 2 * k;                  // owned nodes per direction of a block
  const int NOWN = ipow(NO, dim);        // nodes per block
  const int NNB = ipow(3, dim);          // neighbour offsets incl. centre
  const int NLOC = ipow(k + 1, dim);     // nodes per cell
  std::vector<double> M1, K1, E1;
  reference_1d(k, M1, K1, E1);

  auto coarse_coeff_of = [&](int level, const int64_t* c) {
    int64_t cc[3];
    for (int d = 0; d < 3; ++d) cc[d] = d < dim ? c[d] >> level : 0;
    return h.coarse_coeff[cc[0] + (int64_t)h.n0[0] * (cc[1] + (int64_t)h.n0[1] * cc[2])];
  };
  auto node_key = [&](int level, const int64_t* q) -> int64_t {
    int s = L - level;
    return (int64_t)pack3(q[0] << s, dim > 1 ? q[1] << s : 0, dim > 2 ? q[2] << s : 0);
  };
  int64_t node_ext[3];  // largest finest-lattice node coordinate per direction
  for (int d = 0; d < 3; ++d) node_ext[d] = d < dim ? (int64_t)h.n0[d] * k << L : 0;
  // a node is on the boundary of the domain (the union of the present coarse
  // cells) if some coarse cell whose closure contains it is outside the brick
  // or absent
  const int64_t s0 = (int64_t)k << L;  // node-lattice units per coarse cell
  auto key_is_boundary = [&](uint64_t key) {
    int64_t q[3];
    unpack3(key, q);
    int64_t cand[3][2];
    int nc[3];
    for (int d = 0; d < 3; ++d) {
      if (d >= dim) {
        cand[d][0] = 0;
        nc[d] = 1;
        continue;
      }
      const int64_t up = q[d] / s0;
      cand[d][0] = up;
      nc[d] = 1;
      if (q[d] % s0 == 0) {
        cand[d][1] = up - 1;
        nc[d] = 2;
      }
    }
    for (int a = 0; a < nc[0]; ++a)
      for (int b = 0; b < nc[1]; ++b)
        for (int c = 0; c < nc[2]; ++c) {
          const int64_t cc[3] = {cand[0][a], cand[1][b], cand[2][c]};
          for (int d = 0; d < dim; ++d)
            if (cc[d] < 0 || cc[d] >= h.n0[d]) return true;
          if (!f.coarse_present(cc)) return true;
        }
    return false;
  };
  (void)node_ext;

  h.levels.assign(L + 1, LevelHost());
  h.level_offset.assign(L + 2, 0);

  // ---------------------------------------------------- level 0: lattice
  {
    LevelHost& lv = h.levels[0];
    lv.level = 0;
    int64_t n = 1;
    for (int d = 0; d < 3; ++d) {
      h.coarse_lattice[d] = d < dim ? (int64_t)k * h.n0[d] + 1 : 1;
      n *= h.coarse_lattice[d];
    }
    lv.slot_class.assign(n, 0);
    lv.slot_key.assign(n, -1);
    h.n_coarse = 0;
    for (int64_t z = 0; z < h.coarse_lattice[2]; ++z)
      for (int64_t y = 0; y < h.coarse_lattice[1]; ++y)
        for (int64_t x = 0; x < h.coarse_lattice[0]; ++x) {
          int64_t s = x + h.coarse_lattice[0] * (y + h.coarse_lattice[1] * z);
          int64_t q[3] = {x, y, z};
          lv.slot_key[s] = node_key(0, q);
          bool bd = key_is_boundary((uint64_t)lv.slot_key[s]);
          lv.slot_class[s] = bd ? 3 : 1;
          if (!bd) ++h.n_coarse;
        }
    lv.n_cells = (uint64_t)f.cells[0].count;
    lv.n_S = h.n_coarse;
  }
  auto pad64 = [](int64_t v) { return (v + 63) / 64 * 64; };  // level starts 256-byte aligned
  h.level_offset[1] = pad64((int64_t)h.levels[0].slot_class.size());

  phase_mark(0);
  // ------------------------------------------------ levels l >= 1: blocks
  std::vector<HashMap64> block_map(L + 1);  // parent position (level l-1) -> block index
  for (int l = 1; l <= L; ++l) {
    LevelHost& lv = h.levels[l];
    lv.level = l;
    // groups = refined cells of level l-1, in canonical (tree, Morton) order
    struct G {
      uint64_t tree, morton;
      int64_t c[3];
    };
    std::vector<G> gs;
    int Lp = l - 1;
    f.cells[Lp].for_each([&](uint64_t key, int32_t v) {
      if (!v) return;
      G g;
      unpack3(key, g.c);
      int64_t t[3], loc[3];
      for (int d = 0; d < 3; ++d) {
        t[d] = g.c[d] >> Lp;
        loc[d] = g.c[d] - (t[d] << Lp);
      }
      g.tree = (uint64_t)(t[0] + (int64_t)h.n0[0] * (t[1] + (int64_t)h.n0[1] * t[2]));
      uint64_t m = 0;
      for (int i = 0; i < 21; ++i)
        for (int d = 0; d < dim; ++d) m |= (((uint64_t)loc[d] >> i) & 1ull) << (dim * i + d);
      g.morton = m;
      gs.push_back(g);
    });
    std::sort(gs.begin(), gs.end(), [](const G& a, const G& b) {
      return a.tree != b.tree ? a.tree < b.tree : a.morton < b.morton;
    });
    lv.n_groups = (int64_t)gs.size();
    HashMap64& bm = block_map[l];
    bm.reserve(gs.size() * 2);
    lv.block_pos.resize(3 * gs.size());
    for (size_t i = 0; i < gs.size(); ++i) {
      bm.insert(pack3(gs[i].c[0], gs[i].c[1], gs[i].c[2]), (int32_t)i);
      for (int d = 0; d < 3; ++d) lv.block_pos[3 * i + d] = gs[i].c[d];
    }
    lv.nbr.assign((size_t)lv.n_groups * NNB, -1);
    lv.state.assign(lv.n_groups, 0);
    lv.coeff.resize(lv.n_groups);
    lv.parent.resize(lv.n_groups);
    // neighbour states and the blocks of refined neighbours (lookups only, in
    // parallel); ghost blocks are then numbered in (group, offset) order
    constexpr int32_t kGhostPending = -3;
    bool bad_parent = false;
#pragma omp parallel for schedule(static) reduction(|| : bad_parent)
    for (int64_t g = 0; g < lv.n_groups; ++g) {
      const int64_t* p = gs[g].c;
      uint64_t st = 0;
      for (int nb = 0; nb < NNB; ++nb) {
        int o[3] = {nb % 3 - 1, dim > 1 ? (nb / 3) % 3 - 1 : 0, dim > 2 ? nb / 9 - 1 : 0};
        int64_t q[3] = {p[0] + o[0], p[1] + o[1], p[2] + o[2]};
        int s;
        int32_t slot;
        const int fs = f.state(Lp, q);
        if (!f.inside(Lp, q)) {
          s = kStateOutside;
          slot = -1;
        } else if (fs == 1) {
          s = kStateRefined;
          slot = *bm.find(pack3(q[0], q[1], q[2]));
        } else {
          s = kStateGhost;
          slot = kGhostPending;
        }
        lv.nbr[(size_t)g * NNB + nb] = slot;
        st |= (uint64_t)s << (2 * nb);
      }
      // child position of the parent cell inside its own sibling group
      uint64_t cb = (p[0] & 1) | (dim > 1 ? (p[1] & 1) << 1 : 0) | (dim > 2 ? (p[2] & 1) << 2 : 0);
      st |= cb << 60;
      lv.state[g] = st;
      lv.coeff[g] = coarse_coeff_of(Lp, p);
      if (l == 1) {
        lv.parent[g] = (int32_t)(p[0] + (int64_t)h.n0[0] * (p[1] + (int64_t)h.n0[1] * p[2]));
      } else {
        const int32_t* pp = block_map[l - 1].find(pack3(p[0] >> 1, dim > 1 ? p[1] >> 1 : 0,
                                                        dim > 2 ? p[2] >> 1 : 0));
        if (!pp || *pp >= h.levels[l - 1].n_groups) bad_parent = true;
        else lv.parent[g] = *pp;
      }
    }
    if (bad_parent) throw std::runtime_error("parent of a refined cell is not a sibling group");
    int64_t next_ghost = lv.n_groups;
    for (int64_t g = 0; g < lv.n_groups; ++g) {
      const int64_t* p = gs[g].c;
      for (int nb = 0; nb < NNB; ++nb) {
        if (lv.nbr[(size_t)g * NNB + nb] != kGhostPending) continue;
        int o[3] = {nb % 3 - 1, dim > 1 ? (nb / 3) % 3 - 1 : 0, dim > 2 ? nb / 9 - 1 : 0};
        int64_t q[3] = {p[0] + o[0], p[1] + o[1], p[2] + o[2]};
        auto ins = bm.insert(pack3(q[0], q[1], q[2]), (int32_t)next_ghost);
        if (ins.second) {
          ++next_ghost;
          for (int d = 0; d < 3; ++d) lv.block_pos.push_back(q[d]);
        }
        lv.nbr[(size_t)g * NNB + nb] = *ins.first;
      }
    }
    lv.n_ghosts = next_ghost - lv.n_groups;
    int64_t nslots = (lv.n_groups + lv.n_ghosts) * NOWN;
    h.level_offset[l + 1] = pad64(h.level_offset[l] + nslots);
    // slot classes and keys, from every real group's (2k+1)^d node block
    lv.slot_class.assign(nslots, 0);
    lv.slot_key.assign(nslots, -1);
    const int NG = 2 * k + 1;
    const int NGRP = ipow(NG, dim);
    bool bad = false;
    // pass 0 writes every node's class and key; pass 1 re-derives them from
    // every group that touches the node and checks that all groups agree
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(static) reduction(|| : bad)
    for (int64_t g = 0; g < lv.n_groups; ++g) {
      const int64_t* p = gs[g].c;
      uint64_t st = lv.state[g];
      for (int n = 0; n < NGRP; ++n) {
        int loc[3] = {n % NG, dim > 1 ? (n / NG) % NG : 0, dim > 2 ? n / (NG * NG) : 0};
        // touching parent positions and the block that stores the node
        int lo_o[3], hi_o[3], own[3], ol[3];
        for (int d = 0; d < 3; ++d) {
          if (d >= dim) {
            lo_o[d] = hi_o[d] = 0; own[d] = 0; ol[d] = 0;
            continue;
          }
          lo_o[d] = loc[d] == 0 ? -1 : 0;
          hi_o[d] = loc[d] == 2 * k ? 1 : 0;
          own[d] = loc[d] == 2 * k ? 1 : 0;
          ol[d] = loc[d] == 2 * k ? 0 : loc[d];
        }
        bool outside = false, ghost = false;
        for (int oz = lo_o[2]; oz <= hi_o[2]; ++oz)
          for (int oy = lo_o[1]; oy <= hi_o[1]; ++oy)
            for (int ox = lo_o[0]; ox <= hi_o[0]; ++ox) {
              int nb = (ox + 1) + 3 * (oy + 1) + (dim > 2 ? 9 * (oz + 1) : 0);
              int s = (int)((st >> (2 * nb)) & 3);
              if (s == kStateOutside) outside = true;
              if (s == kStateGhost) ghost = true;
            }
        int cls = outside ? 3 : (ghost ? 2 : 1);
        int nbo = (own[0] + 1) + 3 * (own[1] + 1) + (dim > 2 ? 9 * (own[2] + 1) : 0);
        int32_t blk = lv.nbr[(size_t)g * NNB + nbo];
        if (blk < 0) continue;  // stored outside the domain: Dirichlet, no slot
        int64_t slot = (int64_t)blk * NOWN + ol[0] + NO * (ol[1] + NO * ol[2]);
        int64_t q[3] = {2 * k * p[0] + loc[0], dim > 1 ? 2 * k * p[1] + loc[1] : 0,
                        dim > 2 ? 2 * k * p[2] + loc[2] : 0};
        int64_t key = node_key(l, q);
        if (pass == 0) {
          lv.slot_class[slot] = (int8_t)cls;
          lv.slot_key[slot] = key;
        } else if (lv.slot_class[slot] != cls || lv.slot_key[slot] != key) {
          bad = true;
        }
      }
    }
    }
    if (bad) throw std::runtime_error("inconsistent node classes between sibling groups");
    // prolongation masks: each stored S node is updated by its own group; an I
    // node is written by its own group, or -- when its block is a ghost -- by
    // every group that touches it (the same value)
    lv.pmask.assign((size_t)lv.n_groups * 4, 0);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < lv.n_groups; ++g) {
      for (int n = 0; n < NGRP; ++n) {
        int loc[3] = {n % NG, dim > 1 ? (n / NG) % NG : 0, dim > 2 ? n / (NG * NG) : 0};
        int own[3] = {0, 0, 0}, ol[3] = {0, 0, 0};
        bool in_own = true;
        for (int d = 0; d < dim; ++d) {
          own[d] = loc[d] == 2 * k ? 1 : 0;
          ol[d] = loc[d] == 2 * k ? 0 : loc[d];
          if (own[d]) in_own = false;
        }
        int nbo = (own[0] + 1) + 3 * (own[1] + 1) + (dim > 2 ? 9 * (own[2] + 1) : 0);
        int32_t blk = lv.nbr[(size_t)g * NNB + nbo];
        if (blk < 0) continue;
        int8_t cls = lv.slot_class[(int64_t)blk * NOWN + ol[0] + NO * (ol[1] + NO * ol[2])];
        uint64_t bit = 1ull << (n & 63);
        if (cls == 1 && in_own) lv.pmask[(size_t)g * 4 + (n >> 6)] |= bit;
        if (cls == 2 && (in_own || blk >= lv.n_groups)) lv.pmask[(size_t)g * 4 + 2 + (n >> 6)] |= bit;
      }
    }
    // per-group S mask of the stored nodes and coefficients of the lower neighbours
    lv.smask.assign(lv.n_groups, 0);
    lv.lcoef.assign((size_t)lv.n_groups << dim, 0.0);
    for (int64_t g = 0; g < lv.n_groups; ++g) {
      uint64_t m = 0;
      for (int i = 0; i < NOWN; ++i)
        if (lv.slot_class[g * NOWN + i] == 1) m |= 1ull << i;
      lv.smask[g] = m;
      for (int b = 0; b < (1 << dim); ++b) {
        int o[3] = {-(b & 1), dim > 1 ? -((b >> 1) & 1) : 0, dim > 2 ? -((b >> 2) & 1) : 0};
        int nb = (o[0] + 1) + 3 * (o[1] + 1) + (dim > 2 ? 9 * (o[2] + 1) : 0);
        if (((lv.state[g] >> (2 * nb)) & 3) == kStateRefined)
          lv.lcoef[((size_t)g << dim) + b] = lv.coeff[lv.nbr[(size_t)g * NNB + nb]];
      }
      bool uniform = true;
      for (int b = 1; b < (1 << dim); ++b) {
        double c = lv.lcoef[((size_t)g << dim) + b];
        if (c != 0.0 && c != lv.coeff[g]) uniform = false;
      }
      (uniform ? lv.list_uniform : lv.list_jump).push_back((int32_t)g);
      if (!uniform) lv.n_S_jump += (uint64_t)__builtin_popcountll(m);
    }
    // bricks: 8 uniform groups at positions p + {0,1}^3 with p even, one coefficient
    if (dim == 3) {
      std::vector<char> is_uniform(lv.n_groups, 0), taken(lv.n_groups, 0);
      for (int32_t g : lv.list_uniform) is_uniform[g] = 1;
      auto slot_at = [&](int64_t x, int64_t y, int64_t z) -> int32_t {
        int64_t q[3] = {x, y, z};
        if (!f.inside(Lp, q)) return -1;
        const int32_t* b = bm.find(pack3(x, y, z));
        return b ? *b : -2;
      };
      for (int64_t g = 0; g < lv.n_groups; ++g) {
        const int64_t* p = gs[g].c;
        if ((p[0] | p[1] | p[2]) & 1) continue;
        bool ok = true;
        int32_t own[8];
        for (int b = 0; b < 8 && ok; ++b) {
          int32_t s = slot_at(p[0] + (b & 1), p[1] + ((b >> 1) & 1), p[2] + ((b >> 2) & 1));
          if (s < 0 || s >= lv.n_groups || !is_uniform[s] || lv.coeff[s] != lv.coeff[g]) ok = false;
          else own[b] = s;
        }
        if (!ok) continue;
        std::vector<int32_t> tab(64);
        for (int z = 0; z < 4 && ok; ++z)
          for (int y = 0; y < 4 && ok; ++y)
            for (int x = 0; x < 4 && ok; ++x) {
              int32_t s = slot_at(p[0] + x - 1, p[1] + y - 1, p[2] + z - 1);
              if (s == -2) ok = false;  // a position without a block cannot occur next to a group
              tab[x + 4 * (y + 4 * z)] = s;
            }
        if (!ok) continue;
        lv.bricks.insert(lv.bricks.end(), tab.begin(), tab.end());
        for (int b = 0; b < 8; ++b) taken[own[b]] = 1;
      }
      lv.n_bricks_full = (int64_t)lv.bricks.size() / 64;
      // groups outside full bricks go to the per-group residual and
      // prolongation kernels
      for (int32_t g : lv.list_uniform)
        if (!taken[g]) lv.list_rest.push_back(g);
      // partial bricks (smoothing only): a brick position holding at least
      // kMinMembers uniform groups of one coefficient outside full bricks.
      // The other positions keep whatever block is there (another group or a
      // ghost block) and are read as halo only; a position without a block
      // reads zeros: the stencil of an S node of a member covers only cells
      // of this level, whose nodes all lie in blocks.
      const int kMinMembers = h.params.brick_min_members > 0 ? h.params.brick_min_members : 4;
      std::unordered_set<uint64_t> seen;
      for (int32_t g0 : lv.list_uniform) {
        if (taken[g0]) continue;
        const int64_t* c = gs[g0].c;
        const int64_t p[3] = {c[0] & ~int64_t(1), c[1] & ~int64_t(1), c[2] & ~int64_t(1)};
        if (!seen.insert(pack3(p[0], p[1], p[2])).second) continue;
        int32_t own[8];
        unsigned members = 0;
        for (int b = 0; b < 8; ++b) {
          own[b] = slot_at(p[0] + (b & 1), p[1] + ((b >> 1) & 1), p[2] + ((b >> 2) & 1));
          const int32_t s = own[b];
          if (s >= 0 && s < lv.n_groups && is_uniform[s] && !taken[s] && lv.coeff[s] == lv.coeff[g0])
            members |= 1u << b;
        }
        if (__builtin_popcount(members) < kMinMembers) continue;
        std::vector<int32_t> tab(64);
        for (int z = 0; z < 4; ++z)
          for (int y = 0; y < 4; ++y)
            for (int x = 0; x < 4; ++x) {
              const int32_t s = slot_at(p[0] + x - 1, p[1] + y - 1, p[2] + z - 1);
              tab[x + 4 * (y + 4 * z)] = s < 0 ? -1 : s;
            }
        lv.bricks.insert(lv.bricks.end(), tab.begin(), tab.end());
        lv.brick_members.push_back((uint8_t)members);
        for (int b = 0; b < 8; ++b)
          if ((members >> b) & 1) taken[own[b]] = 1;
      }
      std::vector<int32_t> rest;
      for (int32_t g : lv.list_uniform)
        if (!taken[g]) rest.push_back(g);
      lv.list_uniform.swap(rest);
    } else {
      lv.list_rest = lv.list_uniform;
    }
    lv.list_rest.insert(lv.list_rest.end(), lv.list_jump.begin(), lv.list_jump.end());
    std::sort(lv.list_rest.begin(), lv.list_rest.end());
    for (int64_t s = 0; s < nslots; ++s) {
      if (lv.slot_class[s] == 1) ++lv.n_S;
      if (lv.slot_class[s] == 2) ++lv.n_I;
    }
    lv.n_cells = (uint64_t)lv.n_groups << dim;
  }
  h.total_slots = h.level_offset[L + 1];
  if (h.total_slots >= (int64_t)1 << 32) throw std::runtime_error("level vectors exceed 2^32 slots");

  phase_mark(1);
  // --------------------------------------------------------- leaf mesh
  ActiveHost& A = h.active;
  const int64_t nleaf = (int64_t)f.leaf_level.size();
  A.n_cells = nleaf;
  for (int l = 0; l <= L; ++l) h.levels[l].n_leaves = 0;
  for (int64_t i = 0; i < nleaf; ++i) h.levels[f.leaf_level[i]].n_leaves++;
  // every leaf cell's nodes as dense lattice indices (z ny + y) nx + x on the
  // finest node lattice: the order of the node keys, with fewer radix passes
  const uint64_t lnx = (uint64_t)node_ext[0] + 1, lny = (uint64_t)node_ext[1] + 1;
  const size_t nk = (size_t)nleaf * NLOC;
  std::unique_ptr<uint64_t[]> ckeys = raw_keys(nk);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nleaf; ++i) {
    const int s = L - f.leaf_level[i];
    for (int j = 0; j < NLOC; ++j) {
      const int loc[3] = {j % (k + 1), dim > 1 ? (j / (k + 1)) % (k + 1) : 0, dim > 2 ? j / ((k + 1) * (k + 1)) : 0};
      uint64_t q[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) q[d] = (uint64_t)(f.leaf_coords[3 * i + d] * k + loc[d]) << s;
      ckeys[(size_t)i * NLOC + j] = (q[2] * lny + q[1]) * lnx + q[0];
    }
  }
  // distinct nodes in key order, then back to node keys
  std::vector<uint64_t> nodes;
  {
    std::unique_ptr<uint64_t[]> srt = raw_keys(nk), tmp = raw_keys(nk);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)nk; ++i) srt[i] = ckeys[i];
    radix_sort_u64(srt.get(), tmp.get(), nk);
    tmp.reset();
    const size_t nu0 = (size_t)(std::unique(srt.get(), srt.get() + nk) - srt.get());
    nodes.resize(nu0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)nu0; ++i) {
      const uint64_t t = srt[i] / lnx;
      nodes[i] = pack3((int64_t)(srt[i] % lnx), (int64_t)(t % lny), (int64_t)(t / lny));
    }
  }
  const int64_t nn = (int64_t)nodes.size();
  A.n_leaf_nodes = nn;
  std::vector<int32_t> node_of(nk);
  RowIndex node_index;
  node_index.build(nodes, dim > 2 ? node_ext[2] + 1 : 1, dim > 1 ? node_ext[1] + 1 : 1);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)nk; ++i) {
    const uint64_t t = ckeys[i] / lnx;
    node_of[i] = (int32_t)node_index.find(pack3((int64_t)(ckeys[i] % lnx), (int64_t)(t % lny), (int64_t)(t / lny)));
  }
  ckeys.reset();
  // coarsest leaf level having each node
  std::vector<int8_t> lmin(nn, 127);
  {
    std::vector<std::vector<int64_t>> by_level(L + 1);
    for (int64_t i = 0; i < nleaf; ++i) by_level[f.leaf_level[i]].push_back(i);
    for (int l = L; l >= 0; --l) {
      const auto& cl = by_level[l];
#pragma omp parallel for schedule(static)
      for (int64_t t = 0; t < (int64_t)cl.size(); ++t)
        for (int j = 0; j < NLOC; ++j) lmin[node_of[(size_t)cl[t] * NLOC + j]] = (int8_t)l;
    }
  }
  phase_mark(2);
  // classify: 0 unknown, 1 Dirichlet, 2 hanging
  std::vector<int8_t> ncls(nn, 0);
  std::vector<int32_t> hang_of(nn, -1);
  struct HRow {
    int64_t node;
    int n;
    int64_t mkey[9];
    double w[9];
  };
  std::vector<std::vector<HRow>> hrows_t(omp_get_max_threads());
  bool chain_or_bad = false;
#pragma omp parallel for schedule(dynamic, 4096) reduction(|| : chain_or_bad)
  for (int64_t i = 0; i < nn; ++i) {
    if (key_is_boundary(nodes[i])) {
      ncls[i] = 1;
      continue;
    }
    int lm = lmin[i];
    if (lm == 0) continue;
    int lc = lm - 1;
    int64_t kq[3];
    unpack3(nodes[i], kq);
    int64_t q[3];  // node-lattice coordinates at level lm
    for (int d = 0; d < 3; ++d) q[d] = d < dim ? kq[d] >> (L - lm) : 0;
    // candidate level-lc cells containing the node
    int64_t cand[3][2];
    int nc[3];
    for (int d = 0; d < 3; ++d) {
      if (d >= dim) {
        cand[d][0] = 0;
        nc[d] = 1;
        continue;
      }
      int64_t c = q[d] / (2 * k);
      if (q[d] % (2 * k) == 0) {
        cand[d][0] = c - 1;
        cand[d][1] = c;
        nc[d] = 2;
      } else {
        cand[d][0] = c;
        nc[d] = 1;
      }
    }
    for (int a = 0; a < nc[0]; ++a)
      for (int b = 0; b < nc[1]; ++b)
        for (int c2 = 0; c2 < nc[2]; ++c2) {
          int64_t cc[3] = {cand[0][a], cand[1][b], cand[2][c2]};
          if (f.state(lc, cc) != 0) continue;  // not a leaf of level lc
          if (ncls[i] == 2) continue;
          // a coarser leaf contains the node, which is not one of its nodes
          HRow row;
          row.node = i;
          row.n = 0;
          int r[3];
          for (int d = 0; d < 3; ++d) r[d] = d < dim ? (int)(q[d] - 2 * k * cc[d]) : 0;
          for (int j = 0; j < NLOC; ++j) {
            int jl[3] = {j % (k + 1), dim > 1 ? (j / (k + 1)) % (k + 1) : 0,
                         dim > 2 ? j / ((k + 1) * (k + 1)) : 0};
            double w = 1.0;
            for (int d = 0; d < dim; ++d) w *= E1[r[d] * (k + 1) + jl[d]];
            if (w == 0.0) continue;
            int64_t mq[3];
            for (int d = 0; d < 3; ++d) mq[d] = d < dim ? cc[d] * k + jl[d] : 0;
            if (row.n >= 9) {
              chain_or_bad = true;
              break;
            }
            row.mkey[row.n] = node_key(lc, mq);
            row.w[row.n] = w;
            ++row.n;
          }
          ncls[i] = 2;
          hrows_t[omp_get_thread_num()].push_back(row);
        }
  }
  if (chain_or_bad) throw std::runtime_error("hanging node with too many masters");
  // rows in node order: a row's place is the number of hanging nodes before it
  std::vector<int32_t> hrank(nn + 1, 0);
  for (int64_t i = 0; i < nn; ++i) hrank[i + 1] = hrank[i] + (ncls[i] == 2 ? 1 : 0);
  std::vector<HRow> hrows((size_t)hrank[nn]);
  {
    std::vector<size_t> base(hrows_t.size() + 1, 0);
    for (size_t t = 0; t < hrows_t.size(); ++t) base[t + 1] = base[t] + hrows_t[t].size();
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < (int64_t)hrows_t.size(); ++t)
      for (const HRow& r : hrows_t[t]) hrows[(size_t)hrank[r.node]] = r;
    std::vector<std::vector<HRow>>().swap(hrows_t);
  }
  // unknown numbering: unknowns in node (key) order, by a prefix sum over
  // contiguous pieces of the node range
  std::vector<int64_t> unk_of(nn, -1);
  int64_t nu = 0;
  {
    const int nt = omp_get_max_threads();
    std::vector<int64_t> cnt(nt + 1, 0);
#pragma omp parallel num_threads(nt)
    {
      const int t = omp_get_thread_num();
      const int64_t b = nn * t / nt, e = nn * (t + 1) / nt;
      int64_t c = 0;
      for (int64_t i = b; i < e; ++i) c += ncls[i] == 0;
      cnt[t + 1] = c;
    }
    for (int t = 0; t < nt; ++t) cnt[t + 1] += cnt[t];
    nu = cnt[nt];
    A.n_unknowns = nu;
    A.unknown_keys.resize(nu);
    A.home_level.resize(nu);
#pragma omp parallel num_threads(nt)
    {
      const int t = omp_get_thread_num();
      const int64_t b = nn * t / nt, e = nn * (t + 1) / nt;
      int64_t u = cnt[t];
      for (int64_t i = b; i < e; ++i)
        if (ncls[i] == 0) {
          unk_of[i] = u;
          A.unknown_keys[u] = (int64_t)nodes[i];
          A.home_level[u] = lmin[i];
          ++u;
        }
    }
  }
  phase_mark(3);
  // hanging rows
  A.hang_key.resize(hrows.size());
  A.hang_ptr.assign(hrows.size() + 1, 0);
  A.hang_col.clear();
  A.hang_w.clear();
  A.hang_master_key.clear();
  {
    // masters of every row resolved in parallel (Dirichlet masters dropped),
    // then laid out by a prefix sum over the rows
    const int64_t nh = (int64_t)hrows.size();
    std::vector<int32_t> mnode((size_t)nh * 9, -1);
    std::vector<int32_t> nkeep(nh + 1, 0);
    bool not_leaf = false, chain = false;
#pragma omp parallel for schedule(static) reduction(|| : not_leaf, chain)
    for (int64_t r = 0; r < nh; ++r) {
      hang_of[hrows[r].node] = (int32_t)r;
      A.hang_key[r] = (int64_t)nodes[hrows[r].node];
      int keep = 0;
      for (int m = 0; m < hrows[r].n; ++m) {
        const int64_t mi = node_index.find((uint64_t)hrows[r].mkey[m]);
        if (mi < 0) {
          not_leaf = true;
          continue;
        }
        if (ncls[mi] == 2) chain = true;
        if (ncls[mi] != 0) continue;  // Dirichlet master carries 0
        mnode[(size_t)r * 9 + m] = (int32_t)mi;
        ++keep;
      }
      nkeep[r + 1] = keep;
    }
    if (not_leaf) throw std::runtime_error("master node of a hanging node is not a leaf node");
    if (chain) throw std::runtime_error("constraint chain");
    for (int64_t r = 0; r < nh; ++r) A.hang_ptr[r + 1] = A.hang_ptr[r] + nkeep[r + 1];
    const size_t nnz = (size_t)A.hang_ptr[nh];
    A.hang_col.resize(nnz);
    A.hang_w.resize(nnz);
    A.hang_master_key.resize(nnz);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nh; ++r) {
      int32_t at = A.hang_ptr[r];
      for (int m = 0; m < hrows[r].n; ++m) {
        const int32_t mi = mnode[(size_t)r * 9 + m];
        if (mi < 0) continue;
        A.hang_col[at] = (int32_t)unk_of[mi];
        A.hang_w[at] = hrows[r].w[m];
        A.hang_master_key[at] = hrows[r].mkey[m];
        ++at;
      }
    }
  }
  {
    // transposed constraints, masters in increasing unknown order
    const size_t nnz = A.hang_col.size();
    std::vector<int32_t> cnt(nu + 1, 0);
    for (int32_t c : A.hang_col) cnt[c + 1]++;
    for (int64_t u = 0; u < nu; ++u) cnt[u + 1] += cnt[u];
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    A.hm_hang.assign(nnz, 0);
    A.hm_w.assign(nnz, 0.0);
    for (size_t r = 0; r + 1 < A.hang_ptr.size(); ++r)
      for (int32_t m = A.hang_ptr[r]; m < A.hang_ptr[r + 1]; ++m) {
        const int32_t at = fill[A.hang_col[m]]++;
        A.hm_hang[at] = (int32_t)r;
        A.hm_w[at] = A.hang_w[m];
      }
    A.hm_node.clear();
    A.hm_ptr.assign(1, 0);
    for (int64_t u = 0; u < nu; ++u)
      if (cnt[u + 1] > cnt[u]) {
        A.hm_node.push_back((int32_t)u);
        A.hm_ptr.push_back(cnt[u + 1]);
      }
  }
  phase_mark(4);
  // per leaf cell tables
  A.cell_nodes.resize((size_t)nleaf * NLOC);
  A.cell_coeff.resize(nleaf);
  A.cell_level.resize(nleaf);
  A.cell_coords.resize(3 * nleaf);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nleaf; ++i) {
    int64_t c[3] = {f.leaf_coords[3 * i], f.leaf_coords[3 * i + 1], f.leaf_coords[3 * i + 2]};
    A.cell_coeff[i] = coarse_coeff_of(f.leaf_level[i], c);
    A.cell_level[i] = (uint8_t)f.leaf_level[i];
    for (int d = 0; d < 3; ++d) A.cell_coords[3 * i + d] = (int32_t)c[d];
    for (int j = 0; j < NLOC; ++j) {
      int32_t n = node_of[(size_t)i * NLOC + j];
      int32_t v;
      if (ncls[n] == 0) v = (int32_t)unk_of[n];
      else if (ncls[n] == 1) v = -1;
      else v = -2 - hang_of[n];
      A.cell_nodes[(size_t)i * NLOC + j] = v;
    }
  }
  phase_mark(5);
  // leaf patches and full leaf sibling groups: in canonical (Morton) order
  // the 2^d children of a parent (and the 4^d grandchildren of a grandparent)
  // are consecutive, the first one with the low coordinate bits 0
  {
    const int nch = 1 << dim, NG = 2 * k + 1;
    const int NGN = ipow(NG, dim);
    const int npc = nch * nch, NP = 4 * k + 1;
    const int NPN = ipow(NP, dim);
    A.grp_nodes.clear();
    A.grp_coeff.clear();
    A.grp_level.clear();
    A.pat_nodes.clear();
    A.pat_coeff.clear();
    A.pat_level.clear();
    A.loose_cells.clear();
    // whether a patch or a full group starts at leaf i (independent per i)
    std::vector<uint8_t> starts((size_t)nleaf, 0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nleaf; ++i) {
      const int lvl = f.leaf_level[i];
      bool patch = lvl > 1 && i + npc <= nleaf;
      for (int d = 0; d < dim && patch; ++d)
        if (f.leaf_coords[3 * i + d] & 3) patch = false;
      for (int b = 1; b < npc && patch; ++b) {
        if (f.leaf_level[i + b] != lvl) patch = false;
        const int hi = b >> dim, lo = b & (nch - 1);
        for (int d = 0; d < dim && patch; ++d)
          if (f.leaf_coords[3 * (i + b) + d] != f.leaf_coords[3 * i + d] + 2 * ((hi >> d) & 1) + ((lo >> d) & 1))
            patch = false;
      }
      bool full = lvl > 0 && i + nch <= nleaf;
      for (int d = 0; d < dim && full; ++d)
        if (f.leaf_coords[3 * i + d] & 1) full = false;
      for (int b = 1; b < nch && full; ++b) {
        if (f.leaf_level[i + b] != lvl) full = false;
        for (int d = 0; d < dim && full; ++d)
          if (f.leaf_coords[3 * (i + b) + d] != f.leaf_coords[3 * i + d] + ((b >> d) & 1)) full = false;
      }
      starts[i] = (uint8_t)((patch ? 2 : 0) | (full ? 1 : 0));
    }
    // greedy walk in canonical order: a patch where one starts, else a full
    // group, else a single cell
    std::vector<int64_t> pat_at, grp_at;
    for (int64_t i = 0; i < nleaf;) {
      if (starts[i] & 2) {
        pat_at.push_back(i);
        i += npc;
      } else if (starts[i] & 1) {
        grp_at.push_back(i);
        i += nch;
      } else {
        A.loose_cells.push_back((int32_t)i);
        ++i;
      }
    }
    std::vector<uint8_t>().swap(starts);
    const int64_t np = (int64_t)pat_at.size(), ngr = (int64_t)grp_at.size();
    A.pat_nodes.resize((size_t)np * NPN);
    A.pat_coeff.resize(np);
    A.pat_level.resize(np);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; ++p) {
      const int64_t i = pat_at[p];
      const size_t base = (size_t)p * NPN;
      for (int b = 0; b < npc; ++b) {
        const int hi = b >> dim, lo = b & (nch - 1);
        int pc[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) pc[d] = 2 * ((hi >> d) & 1) + ((lo >> d) & 1);
        for (int j = 0; j < NLOC; ++j) {
          const int lx = j % (k + 1), ly = dim > 1 ? (j / (k + 1)) % (k + 1) : 0,
                    lz = dim > 2 ? j / ((k + 1) * (k + 1)) : 0;
          const int gx = pc[0] * k + lx, gy = pc[1] * k + ly, gz = pc[2] * k + lz;
          A.pat_nodes[base + gx + NP * (gy + NP * gz)] = A.cell_nodes[(size_t)(i + b) * NLOC + j];
        }
      }
      A.pat_coeff[p] = A.cell_coeff[i];
      A.pat_level[p] = (uint8_t)f.leaf_level[i];
    }
    A.grp_nodes.resize((size_t)ngr * NGN);
    A.grp_coeff.resize(ngr);
    A.grp_level.resize(ngr);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < ngr; ++q) {
      const int64_t i = grp_at[q];
      const size_t base = (size_t)q * NGN;
      for (int b = 0; b < nch; ++b) {
        const int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
        for (int j = 0; j < NLOC; ++j) {
          const int lx = j % (k + 1), ly = dim > 1 ? (j / (k + 1)) % (k + 1) : 0,
                    lz = dim > 2 ? j / ((k + 1) * (k + 1)) : 0;
          const int gx = bx * k + lx, gy = by * k + ly, gz = bz * k + lz;
          A.grp_nodes[base + gx + NG * (gy + NG * gz)] = A.cell_nodes[(size_t)(i + b) * NLOC + j];
        }
      }
      A.grp_coeff[q] = A.cell_coeff[i];
      A.grp_level[q] = (uint8_t)f.leaf_level[i];
    }
    A.n_groups = (int64_t)A.grp_coeff.size();
    A.n_patches = (int64_t)A.pat_coeff.size();
    const size_t nl = A.loose_cells.size();
    A.loose_nodes.resize(nl * NLOC);
    A.loose_coeff.resize(nl);
    A.loose_level.resize(nl);
    for (size_t c = 0; c < nl; ++c) {
      const int64_t cell = A.loose_cells[c];
      std::copy(A.cell_nodes.begin() + cell * NLOC, A.cell_nodes.begin() + (cell + 1) * NLOC,
                A.loose_nodes.begin() + c * NLOC);
      A.loose_coeff[c] = A.cell_coeff[cell];
      A.loose_level[c] = A.cell_level[cell];
    }
  }
  phase_mark(6);
  // home slots
  A.home_slot.resize(nu);
  A.home_global.resize(nu);
  bool bad_home = false;
#pragma omp parallel for schedule(static)
  for (int64_t u = 0; u < nu; ++u) {
    int lm = A.home_level[u];
    int64_t kq[3];
    unpack3((uint64_t)A.unknown_keys[u], kq);
    int64_t q[3];
    for (int d = 0; d < 3; ++d) q[d] = d < dim ? kq[d] >> (L - lm) : 0;
    int64_t slot;
    if (lm == 0) {
      slot = q[0] + h.coarse_lattice[0] * (q[1] + h.coarse_lattice[1] * q[2]);
    } else {
      int64_t gp[3], ol[3];
      for (int d = 0; d < 3; ++d) {
        gp[d] = d < dim ? q[d] / (2 * k) : 0;
        ol[d] = d < dim ? q[d] % (2 * k) : 0;
      }
      const int32_t* b = block_map[lm].find(pack3(gp[0], gp[1], gp[2]));
      if (!b || *b >= h.levels[lm].n_groups) {
        bad_home = true;
        continue;
      }
      slot = (int64_t)(*b) * NOWN + ol[0] + NO * (ol[1] + NO * ol[2]);
    }
    if (h.levels[lm].slot_class[slot] != 1 || h.levels[lm].slot_key[slot] != A.unknown_keys[u])
      bad_home = true;
    A.home_slot[u] = slot;
    A.home_global[u] = (uint32_t)(h.level_offset[lm] + slot);
  }
  if (bad_home) throw std::runtime_error("an unknown is not an S node of its home level");

  phase_mark(7);
  // ------------------------------------------------- coarse matrix A_0
  {
    const int n1 = k + 1;
    double hc[3];
    for (int d = 0; d < 3; ++d) hc[d] = d < dim ? (h.hi[d] - h.lo[d]) / h.n0[d] : 1.0;
    // element matrix: sum_i (prod_{j != i} h_j / h_i) K in direction i, M elsewhere
    std::vector<double> Ae((size_t)NLOC * NLOC, 0.0);
    for (int a = 0; a < NLOC; ++a)
      for (int b = 0; b < NLOC; ++b) {
        int ia[3] = {a % n1, (a / n1) % n1, a / (n1 * n1)};
        int ib[3] = {b % n1, (b / n1) % n1, b / (n1 * n1)};
        double s = 0.0;
        for (int dir = 0; dir < dim; ++dir) {
          double t = 1.0;
          for (int e = 0; e < dim; ++e) {
            if (e == dir) t *= K1[ia[e] * n1 + ib[e]] / hc[e];
            else t *= M1[ia[e] * n1 + ib[e]] * hc[e];
          }
          s += t;
        }
        Ae[(size_t)a * NLOC + b] = s;
      }
    std::vector<int64_t> interior_index(h.levels[0].slot_class.size(), -1);
    int64_t ni = 0;
    h.coarse_slots.clear();
    for (size_t s = 0; s < interior_index.size(); ++s)
      if (h.levels[0].slot_class[s] == 1) {
        interior_index[s] = ni++;
        h.coarse_slots.push_back((int32_t)s);
      }
    std::vector<double> A0((size_t)ni * ni, 0.0);
    for (int64_t cz = 0; cz < h.n0[2]; ++cz)
      for (int64_t cy = 0; cy < h.n0[1]; ++cy)
        for (int64_t cx = 0; cx < h.n0[0]; ++cx) {
          int64_t cc[3] = {cx, cy, cz};
          if (!f.coarse_present(cc)) continue;
          double a = coarse_coeff_of(0, cc);
          int64_t id[64];
          for (int j = 0; j < NLOC; ++j) {
            int jl[3] = {j % n1, dim > 1 ? (j / n1) % n1 : 0, dim > 2 ? j / (n1 * n1) : 0};
            int64_t q[3] = {cx * k + jl[0], dim > 1 ? cy * k + jl[1] : 0, dim > 2 ? cz * k + jl[2] : 0};
            id[j] = interior_index[q[0] + h.coarse_lattice[0] * (q[1] + h.coarse_lattice[1] * q[2])];
          }
          for (int a1 = 0; a1 < NLOC; ++a1)
            for (int b1 = 0; b1 < NLOC; ++b1)
              if (id[a1] >= 0 && id[b1] >= 0) A0[id[a1] * ni + id[b1]] += a * Ae[(size_t)a1 * NLOC + b1];
        }
    h.coarse_degree = 0;
    h.coarse_range[0] = h.coarse_range[1] = 0.0;
    h.coarse_ptr.clear();
    h.coarse_col.clear();
    h.coarse_val.clear();
    h.coarse_inverse.clear();
    const int64_t limit = h.params.coarse_solver == GMG_COARSE_CG ? 4096
                          : h.params.coarse_solver == GMG_COARSE_CHEBYSHEV ? 2048 : 25600;
    h.coarse_too_large = ni > limit;
    if (h.coarse_too_large) {
      // nothing to build; gmg_hier_build reports GMG_EUNSUPPORTED
    } else if (h.params.coarse_solver == GMG_COARSE_CG) {
      h.coarse_ptr.assign(1, 0);
      for (int64_t i = 0; i < ni; ++i) {
        for (int64_t j = 0; j < ni; ++j)
          if (A0[i * ni + j] != 0.0) {
            h.coarse_col.push_back((int32_t)j);
            h.coarse_val.push_back(A0[i * ni + j]);
          }
        h.coarse_ptr.push_back((int32_t)h.coarse_col.size());
      }
    } else if (h.params.coarse_solver == GMG_COARSE_CHEBYSHEV) {
      if (ni > 0) chebyshev_coarse_operator(A0, ni, h.params.coarse_tol, h.coarse_inverse, h.coarse_degree,
                                            h.coarse_range);
    } else {
      if (ni > 0 && !spd_inverse(A0, ni)) throw std::runtime_error("coarse matrix is not SPD");
      h.coarse_inverse.swap(A0);
    }
  }
  phase_mark(8);
  h.setup_host_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace gmg
