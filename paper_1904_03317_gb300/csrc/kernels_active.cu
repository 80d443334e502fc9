// Leaf-mesh (active) operator, right-hand side, CG vector kernels, copy
// maps between active and level vectors, and the coarse solve.
//
// Active operator (outer CG, FP64): y = C^T A_leaf C x.  Each leaf cell
// gathers its (K+1)^d node values -- an unknown's value, 0 on the boundary,
// or for a hanging node the interpolant of the coarser neighbour leaf (the
// constraint row C, Sec. 1) -- applies the cell's Kronecker-sum Laplacian by
// sum factorisation, and scatters the result back through C^T with FP64
// atomics.  x^T A x is accumulated from the cells' local energies
// x_K^T A_K x_K, which needs no second pass over y.
//
// Reductions are deterministic: each block writes its partial sum, and the
// last block to finish (atomic ticket) sums the partials in index order.
#include <algorithm>

#include "device_common.cuh"
#include "int_split.cuh"

namespace gmg {

template <int K>
__host__ __device__ constexpr double amass1(int i, int j) {
  if constexpr (K == 1) {
    return i == j ? 1.0 / 3.0 : 1.0 / 6.0;
  } else {
    return (i == 1 && j == 1) ? 16.0 / 30.0
           : (i == 1 || j == 1) ? 2.0 / 30.0
           : (i == j) ? 4.0 / 30.0 : -1.0 / 30.0;
  }
}

template <int K>
__host__ __device__ constexpr double astiff1(int i, int j) {
  if constexpr (K == 1) {
    return i == j ? 1.0 : -1.0;
  } else {
    return (i == 1 && j == 1) ? 16.0 / 3.0
           : (i == 1 || j == 1) ? -8.0 / 3.0
           : (i == j) ? 7.0 / 3.0 : 1.0 / 3.0;
  }
}

template <int I, int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    sfor<I + 1, N>(f);
  }
}

// ------------------------------------------------------------ reductions
// Block sum in a fixed order; result valid in thread 0.
template <int BS>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < BS / 32; ++i) s += sh[i];
  }
  __syncthreads();
  return s;
}

// Write this block's partial; the last block sums all partials in order into *out.
template <int BS>
__device__ __forceinline__ void finish_reduction(double block_total, double* partials, unsigned* counter,
                                                 double* out, bool accumulate = false) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = block_total;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double sh[BS / 32];
  double v = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += BS) v += ((volatile double*)partials)[i];
  double s = block_sum<BS>(v, sh);
  if (threadIdx.x == 0) {
    *out = accumulate ? *out + s : s;
    *counter = 0;
  }
}

static inline unsigned reduce_grid(int64_t n, int bs) {
  int64_t b = (n + bs - 1) / bs;
  if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// ------------------------------------------------------- active operator
template <int DIM, int K>
struct ActGeo {
  static constexpr int N1 = K + 1;
  static constexpr int NC = DIM == 3 ? N1 * N1 * N1 : N1 * N1;  // nodes per cell
  static constexpr int CPB = NC == 4 ? 64 : 32;  // cells per block: CPB * NC is a multiple of 32
  static constexpr int BS = CPB * NC;
  static constexpr int MAX_GRID = 152 * 12;       // bounded grid-stride (reduction partials)
};

// Value of a cell node: an unknown, 0 at a Dirichlet node, or the value of a
// hanging node, which hang_gather_kernel has formed beforehand.
__device__ __forceinline__ double gather_node(int32_t id, const double* __restrict__ x,
                                              const double* __restrict__ xh) {
  if (id >= 0) return x[id];
  if (id == -1) return 0.0;
  return xh[-2 - id];
}

// Adds a cell contribution to node `id`; contributions to a hanging node are
// summed per hanging node and passed on to its masters by hang_scatter_kernel.
// In deterministic mode the launch holds one colour of elements, which share
// no node, so a plain addition is race-free and the colours fix the order.
__device__ __forceinline__ void scatter_node(int32_t id, double v, double* __restrict__ y, double* __restrict__ yh,
                                             bool det = false) {
  if (det) {
    if (id >= 0)
      y[id] += v;
    else if (id <= -2)
      yh[-2 - id] += v;
    return;
  }
  if (id >= 0)
    atomicAdd(y + id, v);
  else if (id <= -2)
    atomicAdd(yh + (-2 - id), v);
}

// Hanging-node values x_h = sum_m w_hm x_m (the rows of C), and zeroed
// accumulators for their contributions.
__global__ void __launch_bounds__(256) hang_gather_kernel(int64_t nh, const int32_t* __restrict__ hp,
                                                          const int32_t* __restrict__ hc,
                                                          const uint8_t* __restrict__ hwc,
                                                          const double* __restrict__ table, int n_table,
                                                          const double* __restrict__ x, double* __restrict__ xh,
                                                          double* __restrict__ yh) {
  __shared__ double w[256];
  for (int i = threadIdx.x; i < n_table; i += blockDim.x) w[i] = table[i];
  __syncthreads();
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int m = hp[h]; m < hp[h + 1]; ++m) v += w[hwc[m]] * x[hc[m]];
    xh[h] = v;
    yh[h] = 0.0;
  }
}

// y_m += sum_h w_hm y_h for every master unknown m (C^T applied to the
// hanging-node sums); one thread per master, so no atomics.
__global__ void __launch_bounds__(256) hang_scatter_kernel(int64_t nm, const int32_t* __restrict__ node,
                                                           const int32_t* __restrict__ mp,
                                                           const int32_t* __restrict__ mh,
                                                           const uint8_t* __restrict__ mwc,
                                                           const double* __restrict__ table, int n_table,
                                                           const double* __restrict__ yh, double* __restrict__ y) {
  __shared__ double w[256];
  for (int i = threadIdx.x; i < n_table; i += blockDim.x) w[i] = table[i];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = mp[i]; j < mp[i + 1]; ++j) s += w[mwc[j]] * yh[mh[j]];
    y[node[i]] += s;
  }
}

template <int DIM, int K>
__global__ void __launch_bounds__(ActGeo<DIM, K>::BS, ActGeo<DIM, K>::BS <= 512 ? 4 : 1)
active_apply_kernel(ActiveArgs a, const double* __restrict__ x, double* __restrict__ y,
                    double* partials, unsigned* counter, double* energy_out, bool accumulate) {
  using G = ActGeo<DIM, K>;
  constexpr int N1 = G::N1, NC = G::NC;
  __shared__ double X[G::CPB][NC];
  __shared__ double T1M[G::CPB][NC], T1K[G::CPB][NC];
  __shared__ double T2C[G::CPB][NC], T2D[G::CPB][NC];
  __shared__ double red[G::BS / 32];
  const int cl = threadIdx.x / NC;      // cell within block
  const int n = threadIdx.x % NC;       // node within cell
  const int ix = n % N1, iy = (n / N1) % N1, iz = DIM == 3 ? n / (N1 * N1) : 0;
  const int64_t ncell = a.cell_list ? a.n_list : a.n_cells;
  const int64_t nbatch = (ncell + G::CPB - 1) / G::CPB;
  double e = 0.0;
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int64_t ci = batch * G::CPB + cl;
    const bool active = ci < ncell;
    const int64_t cell = active ? (a.cell_list ? (int64_t)a.cell_list[ci] : ci) : 0;
    int32_t id = -1;
    double coef = 0.0;
    int lvl = 0;
    if (active) {
      id = a.cell_nodes[cell * NC + n];
      coef = a.cell_coeff[cell];
      lvl = a.cell_level[cell];
    }
    X[cl][n] = active ? gather_node(id, x, a.xh) : 0.0;
    __syncthreads();
    // Kronecker sum  sx Kx My Mz + sy Mx Ky Mz + sz Mx My Kz  as
    //   A = Mx X, B = Kx X;  C = My A, D = sx My B + sy Ky A;  out = a (Mz D + sz Kz C)
    double out;
    if constexpr (DIM == 3) {
      double A = 0, B = 0;
      sfor<0, N1>([&](auto c) {
        const double v = X[cl][c + N1 * (iy + N1 * iz)];
        A += amass1<K>(ix, c) * v;
        B += astiff1<K>(ix, c) * v;
      });
      T1M[cl][n] = A;
      T1K[cl][n] = B;
      __syncthreads();
      double C = 0, t1 = 0, t2 = 0;
      sfor<0, N1>([&](auto c) {
        const int j = ix + N1 * (c + N1 * iz);
        const double va = T1M[cl][j], vb = T1K[cl][j];
        C += amass1<K>(iy, c) * va;
        t1 += amass1<K>(iy, c) * vb;
        t2 += astiff1<K>(iy, c) * va;
      });
      T2C[cl][n] = C;
      T2D[cl][n] = a.scale[lvl][0] * t1 + a.scale[lvl][1] * t2;
      __syncthreads();
      double t3 = 0, t4 = 0;
      sfor<0, N1>([&](auto c) {
        const int j = ix + N1 * (iy + N1 * c);
        t3 += amass1<K>(iz, c) * T2D[cl][j];
        t4 += astiff1<K>(iz, c) * T2C[cl][j];
      });
      out = coef * (t3 + a.scale[lvl][2] * t4);
    } else {
      double A = 0, B = 0;
      sfor<0, N1>([&](auto c) {
        const double v = X[cl][c + N1 * iy];
        A += amass1<K>(ix, c) * v;
        B += astiff1<K>(ix, c) * v;
      });
      T1M[cl][n] = A;
      T1K[cl][n] = B;
      __syncthreads();
      double t1 = 0, t2 = 0;
      sfor<0, N1>([&](auto c) {
        const int j = ix + N1 * c;
        t1 += amass1<K>(iy, c) * T1K[cl][j];
        t2 += astiff1<K>(iy, c) * T1M[cl][j];
      });
      out = coef * (a.scale[lvl][0] * t1 + a.scale[lvl][1] * t2);
    }
    if (active) {
      e += X[cl][n] * out;
      scatter_node(id, out, y, a.yh, a.deterministic);
    }
    __syncthreads();  // X / T arrays are reused by the next batch
  }
  if (energy_out) {
    double s = block_sum<G::BS>(e, red);
    finish_reduction<G::BS>(s, partials, counter, energy_out, accumulate);
  }
}

// ------------------------------- active operator, leaf groups and leaf patches
// A group (P = 2) is a refined cell whose 2^d children are all leaves, a patch
// (P = 4) a cell whose 4^d grandchildren are.  All P^d cells share one
// coefficient, so the operator of the group is the Kronecker sum of
// (PK+1) x (PK+1) assembled 1-D matrices and nodes shared between its cells
// are computed once.  Q groups per block, one thread per line of a group's
// (PK+1)^d node lattice.
template <int K, int P, bool STIFF>
__host__ __device__ constexpr double agrp(int a, int b) {
  double v = 0.0;
  for (int cell = 0; cell < P; ++cell) {
    int lo = K * cell;
    if (a >= lo && a <= lo + K && b >= lo && b <= lo + K)
      v += STIFF ? astiff1<K>(a - lo, b - lo) : amass1<K>(a - lo, b - lo);
  }
  return v;
}

template <int DIM, int K, int P>
struct AGrp {
  static constexpr int NG = P * K + 1;
  static constexpr int NN = DIM == 3 ? NG * NG * NG : NG * NG;
  static constexpr int LINES = DIM == 3 ? NG * NG : NG;
  // groups per block: as many lines as fit 128 threads (two Q2 3D patches,
  // 162 lines in 192 threads: measured faster than one or three)
  static constexpr int TARGET = (DIM == 3 && P == 4 && K == 2) ? 162 : 128;
  static constexpr int Q = TARGET / LINES > 0 ? TARGET / LINES : 1;
  static constexpr int BS = (Q * LINES + 31) / 32 * 32;
  static constexpr int MAX_GRID = 152 * 16;
  // resident blocks per SM the register budget is sized for
  static constexpr int MIN_BLOCKS = BS >= 256 ? 3 : (BS >= 192 ? 4 : 8);
  // dynamic shared memory: X, A (later C) and B (later D) per group
  static constexpr size_t SMEM = sizeof(double) * (3 * Q * NN + 4 * Q + BS / 32);
};

template <int DIM, int K, int P, bool ISO>
__global__ void __launch_bounds__(AGrp<DIM, K, P>::BS, AGrp<DIM, K, P>::MIN_BLOCKS)
active_group_kernel(ActiveArgs a, int64_t n_grp, const int32_t* __restrict__ grp_nodes,
                    const double* __restrict__ grp_coeff, const uint8_t* __restrict__ grp_level,
                    const double* __restrict__ x, double* __restrict__ y, double* partials, unsigned* counter,
                    double* energy_out, bool accumulate) {
  using G = AGrp<DIM, K, P>;
  constexpr int NG = G::NG, NN = G::NN, Q = G::Q;
  extern __shared__ double smem_g[];
  double (*X)[NN] = reinterpret_cast<double (*)[NN]>(smem_g);
  double (*A)[NN] = reinterpret_cast<double (*)[NN]>(smem_g + Q * NN);
  double (*B)[NN] = reinterpret_cast<double (*)[NN]>(smem_g + 2 * Q * NN);
  double* coef = smem_g + 3 * Q * NN;
  double (*sc)[3] = reinterpret_cast<double (*)[3]>(coef + Q);
  double* red = coef + 4 * Q;
  const int tid = threadIdx.x;
  const int64_t nbatch = (n_grp + Q - 1) / Q;
  double e = 0.0;
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    for (int idx = tid; idx < Q * NN; idx += G::BS) {
      const int q = idx / NN, n = idx % NN;
      const int64_t grp = batch * Q + q;
      X[q][n] = grp < n_grp ? gather_node(grp_nodes[grp * NN + n], x, a.xh) : 0.0;
    }
    if (tid < Q) {
      const int64_t grp = batch * Q + tid;
      const bool ok = grp < n_grp;
      const int lvl = ok ? grp_level[grp] : 0;
      coef[tid] = ok ? grp_coeff[grp] : 0.0;
      sc[tid][0] = a.scale[lvl][0];
      sc[tid][1] = a.scale[lvl][1];
      sc[tid][2] = a.scale[lvl][2];
    }
    __syncthreads();
    const int q = tid / G::LINES, line = tid % G::LINES;
    const bool act = tid < Q * G::LINES;
    // x direction: rows are contiguous
    if (act) {
      double v[NG];
      sfor<0, NG>([&](auto c) { v[c] = X[q][c + NG * line]; });
      sfor<0, NG>([&](auto r) {
        double am = 0, bk = 0;
        sfor<0, NG>([&](auto c) {
          constexpr double m = agrp<K, P, false>(r, c), kk = agrp<K, P, true>(r, c);
          if constexpr (m != 0.0) am += m * v[c];
          if constexpr (kk != 0.0) bk += kk * v[c];
        });
        A[q][r + NG * line] = am;
        B[q][r + NG * line] = bk;
      });
    }
    __syncthreads();
    if constexpr (DIM == 3) {
      // cubic cells (s_x = s_y = s_z = s): D = My B + Ky A and out = a s (Mz D + Kz C)
      // need no per-direction scaling
      constexpr bool iso = ISO;
      // y direction: line = (ix, iz); a thread reads its whole line before it
      // overwrites it, so C and D take the places of A and B
      if (act) {
        const int ix = line % NG, iz = line / NG;
        double va[NG], vb[NG];
        sfor<0, NG>([&](auto c) {
          va[c] = A[q][ix + NG * (c + NG * iz)];
          vb[c] = B[q][ix + NG * (c + NG * iz)];
        });
        const double sx = sc[q][0], sy = sc[q][1];
        sfor<0, NG>([&](auto r) {
          double cc = 0, t1 = 0, t2 = 0;
          sfor<0, NG>([&](auto c) {
            constexpr double m = agrp<K, P, false>(r, c), kk = agrp<K, P, true>(r, c);
            if constexpr (m != 0.0) {
              cc += m * va[c];
              t1 += m * vb[c];
            }
            if constexpr (kk != 0.0) {
              if constexpr (iso) t1 += kk * va[c];
              else t2 += kk * va[c];
            }
          });
          A[q][ix + NG * (r + NG * iz)] = cc;
          B[q][ix + NG * (r + NG * iz)] = iso ? t1 : sx * t1 + sy * t2;
        });
      }
      __syncthreads();
      // z direction: line = (ix, iy), then scatter
      if (act) {
        const int64_t grp = batch * Q + q;
        const int ix = line % NG, iy = line / NG;
        double vc[NG], vd[NG];
        sfor<0, NG>([&](auto c) {
          vc[c] = A[q][ix + NG * (iy + NG * c)];
          vd[c] = B[q][ix + NG * (iy + NG * c)];
        });
        const double cf = coef[q], sz = sc[q][2];
        const double cfs = cf * sz;
        if (grp < n_grp) {
          sfor<0, NG>([&](auto r) {
            double t3 = 0, t4 = 0;
            sfor<0, NG>([&](auto c) {
              constexpr double m = agrp<K, P, false>(r, c), kk = agrp<K, P, true>(r, c);
              if constexpr (m != 0.0) t3 += m * vd[c];
              if constexpr (kk != 0.0) {
                if constexpr (iso) t3 += kk * vc[c];
                else t4 += kk * vc[c];
              }
            });
            const double out = iso ? cfs * t3 : cf * (t3 + sz * t4);
            const int n = ix + NG * (iy + NG * r);
            e += X[q][n] * out;
            const int32_t id = grp_nodes[grp * NN + n];
            const bool interior = ix > 0 && ix < NG - 1 && iy > 0 && iy < NG - 1 && r > 0 && r < NG - 1;
            if (interior && id >= 0)
              y[id] = out;  // interior nodes belong to this group's cells only
            else
              scatter_node(id, out, y, a.yh, a.deterministic);
          });
        }
      }
    } else {
      if (act) {
        const int64_t grp = batch * Q + q;
        const int ix = line;
        double va[NG], vb[NG];
        sfor<0, NG>([&](auto c) {
          va[c] = A[q][ix + NG * c];
          vb[c] = B[q][ix + NG * c];
        });
        const double cf = coef[q], sx = sc[q][0], sy = sc[q][1];
        if (grp < n_grp) {
          sfor<0, NG>([&](auto r) {
            double t1 = 0, t2 = 0;
            sfor<0, NG>([&](auto c) {
              constexpr double m = agrp<K, P, false>(r, c), kk = agrp<K, P, true>(r, c);
              if constexpr (m != 0.0) t1 += m * vb[c];
              if constexpr (kk != 0.0) t2 += kk * va[c];
            });
            const double out = cf * (sx * t1 + sy * t2);
            const int n = ix + NG * r;
            e += X[q][n] * out;
            const int32_t id = grp_nodes[grp * NN + n];
            const bool interior = ix > 0 && ix < NG - 1 && r > 0 && r < NG - 1;
            if (interior && id >= 0)
              y[id] = out;
            else
              scatter_node(id, out, y, a.yh, a.deterministic);
          });
        }
      }
    }
    __syncthreads();  // the next batch overwrites the shared arrays
  }
  if (energy_out) {
    double s = block_sum<G::BS>(e, red);
    finish_reduction<G::BS>(s, partials, counter, energy_out, accumulate);
  }
}

// ------------------------ active operator, exact split-integer evaluation
// (the scheme and its error bound: int_split.cuh)
// integer 1-D matrix of P cells assembled along a row of a patch
template <int K, int P, bool STIFF>
__host__ __device__ constexpr int igrp(int a, int b) {
  int v = 0;
  for (int cell = 0; cell < P; ++cell) {
    int lo = K * cell;
    if (a >= lo && a <= lo + K && b >= lo && b <= lo + K) v += ielem1<K, STIFF>(a - lo, b - lo);
  }
  return v;
}

// the integer matrices are the FP64 ones times their denominators
template <int K>
constexpr bool int_elems_match() {
  for (int i = 0; i <= K; ++i)
    for (int j = 0; j <= K; ++j) {
      const double dm = amass1<K>(i, j) * IntElem<K>::DM - ielem1<K, false>(i, j);
      const double dk = astiff1<K>(i, j) * IntElem<K>::DK - ielem1<K, true>(i, j);
      if (dm > 1e-12 || dm < -1e-12 || dk > 1e-12 || dk < -1e-12) return false;
    }
  return true;
}
static_assert(int_elems_match<1>() && int_elems_match<2>(), "integer element matrices");

// largest sum of |entries| of a row of the assembled integer matrices
template <int K, int P, bool STIFF>
constexpr long long igrp_rowsum() {
  long long best = 0;
  for (int r = 0; r <= P * K; ++r) {
    long long t = 0;
    for (int c = 0; c <= P * K; ++c) t += igrp<K, P, STIFF>(r, c) < 0 ? -igrp<K, P, STIFF>(r, c) : igrp<K, P, STIFF>(r, c);
    best = t > best ? t : best;
  }
  return best;
}

// bound on |integer Kronecker sum| per unit input
template <int DIM, int K, int P>
constexpr long long ikron_bound() {
  constexpr long long m = igrp_rowsum<K, P, false>(), k = igrp_rowsum<K, P, true>();
  return DIM == 3 ? 3 * m * m * k : 2 * m * k;
}

template <int DIM, int K, int P>
constexpr bool int_recombination_fits(int k) {
  return int_recombination_fits_bound(ikron_bound<DIM, K, P>(), k);
}
template <int DIM, int K, int P>
constexpr int int_recombination_bits() {
  return int_recombination_bits_bound(ikron_bound<DIM, K, P>());
}

template <int DIM, int K, int P>
struct AGrpI {
  using G = AGrp<DIM, K, P>;
  static constexpr int NN = G::NN, Q = G::Q, BS = G::BS;
  // X (FP64) and, per component (P1, P2, r), the in-place array and the
  // second stage-1 output, 4 bytes each
  static constexpr size_t SMEM = sizeof(double) * ((size_t)Q * NN + 2 * Q + BS / 32) + 4 * (6 * (size_t)Q * NN + Q);
  // blocks per SM the registers are sized for: 64 registers let eight
  // blocks of five P = 2 groups share an SM (measured 6 % faster than six)
  static constexpr int MIN_BLOCKS = BS >= 256 ? 3 : (BS >= 192 ? 4 : (P == 2 ? 8 : 6));
};

template <int DIM, int K, int P>
__global__ void __launch_bounds__(AGrp<DIM, K, P>::BS, AGrpI<DIM, K, P>::MIN_BLOCKS)
active_group_int_kernel(ActiveArgs a, int64_t n_grp, const int32_t* __restrict__ grp_nodes,
                        const double* __restrict__ grp_coeff, const uint8_t* __restrict__ grp_level,
                        const double* __restrict__ x, double* __restrict__ y, double* partials, unsigned* counter,
                        double* energy_out, bool accumulate) {
  using G = AGrp<DIM, K, P>;
  constexpr int NG = G::NG, NN = G::NN, Q = G::Q, BS = G::BS;
  static_assert(ikron_bound<DIM, K, P>() * 32768LL < 2147483648LL, "integer Kronecker sum exceeds int32");
  constexpr int KR = int_recombination_bits<DIM, K, P>();
  static_assert(KR >= 5 && int_recombination_fits<DIM, K, P>(KR), "integer recombination exceeds 2^51");
  extern __shared__ double smem_g[];
  double (*X)[NN] = reinterpret_cast<double (*)[NN]>(smem_g);
  double* scl = smem_g + Q * NN;       // per group: q 2^-15 a s / (DM^(d-1) DK)
  double* red = scl + 2 * Q;
  int (*A1)[NN] = reinterpret_cast<int (*)[NN]>(red + BS / 32);
  int (*B1)[NN] = A1 + Q;
  int (*A2)[NN] = B1 + Q;
  int (*B2)[NN] = A2 + Q;
  float (*A3)[NN] = reinterpret_cast<float (*)[NN]>(B2 + Q);
  float (*B3)[NN] = A3 + Q;
  int* emax = reinterpret_cast<int*>(B3 + Q);
  constexpr double DEN = DIM == 3 ? (double)IntElem<K>::DM * IntElem<K>::DM * IntElem<K>::DK
                                  : (double)IntElem<K>::DM * IntElem<K>::DK;
  const int tid = threadIdx.x;
  const int64_t nbatch = (n_grp + Q - 1) / Q;
  double e = 0.0;
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    if (tid < Q) emax[tid] = 1;
    __syncthreads();
    {
      // all node indices first, then all values: PER loads in flight per thread
      constexpr int PER = (Q * NN + BS - 1) / BS;
      int32_t ids[PER];
      double vals[PER];
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int idx = tid + k * BS;
        const int64_t grp = batch * Q + idx / NN;
        ids[k] = (idx < Q * NN && grp < n_grp) ? grp_nodes[grp * NN + idx % NN] : -1;
      }
#pragma unroll
      for (int k = 0; k < PER; ++k) vals[k] = gather_node(ids[k], x, a.xh);
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int idx = tid + k * BS;
        const int qq = idx < Q * NN ? idx / NN : Q;  // lanes past the end form their own set
        if (idx < Q * NN) X[qq][idx % NN] = vals[k];
        // largest exponent per group: one shared atomic per group present in the warp
        const int ex = (int)((__double_as_longlong(vals[k]) >> 52) & 0x7FF);
        const unsigned same = __match_any_sync(0xffffffffu, qq);
        const int mx = __reduce_max_sync(same, ex);
        if (qq < Q && (threadIdx.x & 31) == __ffs(same) - 1) atomicMax(&emax[qq], mx);
      }
    }
    __syncthreads();
    if (tid < Q) {
      const int64_t grp = batch * Q + tid;
      const bool ok = grp < n_grp;
      const int lvl = ok ? grp_level[grp] : 0;
      const double cs = ok ? grp_coeff[grp] * a.scale[lvl][0] / DEN : 0.0;
      // q 2^-15 2^-KR = 2^(emax - 1023 - 14 - 15 - KR); a NaN or Inf input makes the group's output NaN
      const int eo = emax[tid] - 1023 - 29 - KR;
      scl[tid] = emax[tid] == 0x7FF ? __longlong_as_double(0x7FF8000000000000LL)
                                     : cs * ldexp(1.0, eo);
    }
    for (int idx = tid; idx < Q * NN; idx += BS) {
      const int q = idx / NN, n = idx % NN;
      int p1, p2;
      float r;
      split_exact(X[q][n], emax[q] == 0x7FF ? 1010 : emax[q] - 1037, p1, p2, r);
      A1[q][n] = p1;
      A2[q][n] = p2;
      A3[q][n] = r;
    }
    __syncthreads();
    const int q = tid / G::LINES, line = tid % G::LINES;
    const bool act = tid < Q * G::LINES;
    // x direction, in place: A <- M~ v, B <- K~ v
    auto xstage = [&](auto* Av, auto* Bv) {
      using T = typename std::remove_reference<decltype(Av[0])>::type;
      T v[NG];
      sfor<0, NG>([&](auto c) { v[c] = Av[c + NG * line]; });
      sfor<0, NG>([&](auto r) {
        T am = 0, bk = 0;
        sfor<0, NG>([&](auto c) {
          constexpr int m = igrp<K, P, false>(r, c), kk = igrp<K, P, true>(r, c);
          if constexpr (m != 0) am += (T)m * v[c];
          if constexpr (kk != 0) bk += (T)kk * v[c];
        });
        Av[r + NG * line] = am;
        Bv[r + NG * line] = bk;
      });
    };
    if (act) {
      xstage(A1[q], B1[q]);
      xstage(A2[q], B2[q]);
      xstage(A3[q], B3[q]);
    }
    __syncthreads();
    if constexpr (DIM == 3) {
      // y direction, in place: C = M~ A, D = M~ B + K~ A
      auto ystage = [&](auto* Av, auto* Bv) {
        using T = typename std::remove_reference<decltype(Av[0])>::type;
        const int ix = line % NG, iz = line / NG;
        T va[NG], vb[NG];
        sfor<0, NG>([&](auto c) {
          va[c] = Av[ix + NG * (c + NG * iz)];
          vb[c] = Bv[ix + NG * (c + NG * iz)];
        });
        sfor<0, NG>([&](auto r) {
          T cc = 0, dd = 0;
          sfor<0, NG>([&](auto c) {
            constexpr int m = igrp<K, P, false>(r, c), kk = igrp<K, P, true>(r, c);
            if constexpr (m != 0) {
              cc += (T)m * va[c];
              dd += (T)m * vb[c];
            }
            if constexpr (kk != 0) dd += (T)kk * va[c];
          });
          Av[ix + NG * (r + NG * iz)] = cc;
          Bv[ix + NG * (r + NG * iz)] = dd;
        });
      };
      if (act) {
        ystage(A1[q], B1[q]);
        ystage(A2[q], B2[q]);
        ystage(A3[q], B3[q]);
      }
      __syncthreads();
    }
    // last direction: out = M~ D + K~ C (3D) or M~ B + K~ A (2D), recombined in FP64
    if (act) {
      const int64_t grp = batch * Q + q;
      if (grp < n_grp) {
        const int ix = line % NG, iy = DIM == 3 ? line / NG : 0;
        auto at = [&](int c) { return DIM == 3 ? ix + NG * (iy + NG * c) : ix + NG * c; };
        int c1[NG], d1[NG], c2[NG], d2[NG];
        float c3[NG], d3[NG];
        sfor<0, NG>([&](auto c) {
          c1[c] = A1[q][at(c)];
          d1[c] = B1[q][at(c)];
          c2[c] = A2[q][at(c)];
          d2[c] = B2[q][at(c)];
          c3[c] = A3[q][at(c)];
          d3[c] = B3[q][at(c)];
        });
        const double sc = scl[q];
        sfor<0, NG>([&](auto r) {
          int o1 = 0, o2 = 0;
          float o3 = 0.f;
          sfor<0, NG>([&](auto c) {
            constexpr int m = igrp<K, P, false>(r, c), kk = igrp<K, P, true>(r, c);
            if constexpr (m != 0) {
              o1 += m * d1[c];
              o2 += m * d2[c];
              o3 += (float)m * d3[c];
            }
            if constexpr (kk != 0) {
              o1 += kk * c1[c];
              o2 += kk * c2[c];
              o3 += (float)kk * c3[c];
            }
          });
          const double t = i64_to_double(((long long)o1 << (15 + KR)) + ((long long)o2 << KR) +
                                         (long long)f32_fixed_rint<KR>(o3));
          const double out = t * sc;
          const int n = DIM == 3 ? ix + NG * (iy + NG * r) : ix + NG * r;
          e += X[q][n] * out;
          const int32_t id = grp_nodes[grp * NN + n];
          const bool interior = ix > 0 && ix < NG - 1 && r > 0 && r < NG - 1 &&
                                (DIM == 2 || (iy > 0 && iy < NG - 1));
          if (interior && id >= 0)
            y[id] = out;
          else
            scatter_node(id, out, y, a.yh, a.deterministic);
        });
      }
    }
    __syncthreads();  // the next batch overwrites the shared arrays
  }
  if (energy_out) {
    double s = block_sum<BS>(e, red);
    finish_reduction<BS>(s, partials, counter, energy_out, accumulate);
  }
}

template <int DIM, int K, int P>
static void group_launch(const ActiveArgs& a, int64_t n, const int32_t* nodes, const double* coeff,
                         const uint8_t* level, const double* x, double* y, double* partials, unsigned* counter,
                         double* energy, bool accumulate, cudaStream_t s) {
  using G = AGrp<DIM, K, P>;
  static_assert(G::MAX_GRID <= kMaxReduceBlocks, "reduction partials");
  using GI = AGrpI<DIM, K, P>;
  static const bool init = [] {
    cudaFuncSetAttribute(active_group_int_kernel<DIM, K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)GI::SMEM);
    cudaFuncSetAttribute(active_group_kernel<DIM, K, P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)G::SMEM);
    return true;
  }();
  (void)init;
  int64_t blocks = (n + G::Q - 1) / G::Q;
  if (blocks > G::MAX_GRID) blocks = G::MAX_GRID;
  // cubic cells on every level (the ratios of the sides are those of the coarse
  // cells): one integer Kronecker sum; otherwise the FP64 kernel with
  // per-direction factors
  const bool iso = a.scale[0][0] == a.scale[0][1] && (DIM == 2 || a.scale[0][1] == a.scale[0][2]);
  if (iso)
    active_group_int_kernel<DIM, K, P><<<(unsigned)blocks, G::BS, GI::SMEM, s>>>(
        a, n, nodes, coeff, level, x, y, partials, counter, energy, accumulate);
  else
    active_group_kernel<DIM, K, P, false><<<(unsigned)blocks, G::BS, G::SMEM, s>>>(
        a, n, nodes, coeff, level, x, y, partials, counter, energy, accumulate);
  GMG_COUNT_LAUNCH();
}

template <int DIM, int K>
static cudaError_t active_dispatch(const ActiveArgs& a, const double* x, double* y, double* partials,
                                   unsigned* counter, double* energy, cudaStream_t s) {
  bool wrote = false;
  if (a.n_hang > 0) {
    const int64_t b = (a.n_hang + 255) / 256;
    hang_gather_kernel<<<(unsigned)(b > 152 * 32 ? 152 * 32 : b), 256, 0, s>>>(a.n_hang, a.hang_ptr, a.hang_col,
                                                                                a.hang_wc, a.hw_table, a.n_hw, x,
                                                                                a.xh, a.yh);
    GMG_COUNT_LAUNCH();
  }
  // one launch per kind, or in deterministic mode one per colour of the kind
  // (colour-ordered tables, offsets off[0..n])
  auto ranges = [&](int64_t n, const int64_t* off, int ncol, auto&& launch) {
    if (n == 0) return;
    if (!a.deterministic || !off) {
      launch((int64_t)0, n);
      return;
    }
    for (int c = 0; c < ncol; ++c)
      if (off[c + 1] > off[c]) launch(off[c], off[c + 1] - off[c]);
  };
  constexpr int NN4 = AGrp<DIM, K, 4>::NN, NN2 = AGrp<DIM, K, 2>::NN, NN1 = AGrp<DIM, K, 1>::NN;
  ranges(a.n_patches, a.pat_off, a.n_pat_colors, [&](int64_t b, int64_t n) {
    group_launch<DIM, K, 4>(a, n, a.pat_nodes + b * NN4, a.pat_coeff + b, a.pat_level + b, x, y, partials, counter,
                            energy, wrote, s);
    wrote = true;
  });
  ranges(a.n_groups, a.grp_off, a.n_grp_colors, [&](int64_t b, int64_t n) {
    group_launch<DIM, K, 2>(a, n, a.grp_nodes + b * NN2, a.grp_coeff + b, a.grp_level + b, x, y, partials, counter,
                            energy, wrote, s);
    wrote = true;
  });
  const int64_t ncell = a.cell_list ? a.n_list : a.n_cells;
  const bool iso = a.scale[0][0] == a.scale[0][1] && (DIM == 2 || a.scale[0][1] == a.scale[0][2]);
  if (ncell > 0 && iso && a.cell_list) {
    // single cells of cubic shape: the split-integer kernel with one cell per group
    ranges(a.n_list, a.loose_off, a.n_loose_colors, [&](int64_t b, int64_t n) {
      group_launch<DIM, K, 1>(a, n, a.loose_nodes + b * NN1, a.loose_coeff + b, a.loose_level + b, x, y, partials,
                              counter, energy, wrote, s);
      wrote = true;
    });
  } else if (ncell > 0) {
    using G = ActGeo<DIM, K>;
    static_assert(G::MAX_GRID <= kMaxReduceBlocks, "reduction partials");
    auto cells = [&](const ActiveArgs& aa, int64_t n) {
      int64_t blocks = (n + G::CPB - 1) / G::CPB;
      if (blocks > G::MAX_GRID) blocks = G::MAX_GRID;
      active_apply_kernel<DIM, K><<<(unsigned)blocks, G::BS, 0, s>>>(aa, x, y, partials, counter, energy, wrote);
      GMG_COUNT_LAUNCH();
      wrote = true;
    };
    if (a.cell_list) {
      ranges(a.n_list, a.loose_off, a.n_loose_colors, [&](int64_t b, int64_t n) {
        ActiveArgs aa = a;
        aa.cell_list = a.cell_list + b;
        aa.n_list = n;
        cells(aa, n);
      });
    } else {
      cells(a, ncell);
    }
  }
  if (a.n_masters > 0) {
    const int64_t b = (a.n_masters + 255) / 256;
    hang_scatter_kernel<<<(unsigned)(b > 152 * 32 ? 152 * 32 : b), 256, 0, s>>>(a.n_masters, a.hm_node, a.hm_ptr,
                                                                                 a.hm_hang, a.hm_wc, a.hw_table,
                                                                                 a.n_hw, a.yh, y);
    GMG_COUNT_LAUNCH();
  }
  if (!wrote && energy) cudaMemsetAsync(energy, 0, sizeof(double), s);
  return cudaGetLastError();
}

cudaError_t launch_active_apply(int dim, int k, const ActiveArgs& a, const double* x, double* y,
                                double* partials, unsigned* counter, double* energy_out,
                                cudaStream_t s) {
  if (dim == 3 && k == 2) return active_dispatch<3, 2>(a, x, y, partials, counter, energy_out, s);
  if (dim == 3 && k == 1) return active_dispatch<3, 1>(a, x, y, partials, counter, energy_out, s);
  if (dim == 2 && k == 2) return active_dispatch<2, 2>(a, x, y, partials, counter, energy_out, s);
  if (dim == 2 && k == 1) return active_dispatch<2, 1>(a, x, y, partials, counter, energy_out, s);
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------ right-hand side
// b_i += int_K f phi_i with f = d pi^2 prod sin(pi x_i), (K+1)^d Gauss points.
template <int K>
__device__ __forceinline__ void gauss_point(int q, double& x, double& w) {
  if constexpr (K == 1) {
    const double a = 0.28867513459481288225;  // 1 / (2 sqrt 3)
    x = q == 0 ? 0.5 - a : 0.5 + a;
    w = 0.5;
  } else {
    const double a = 0.38729833462074168852;  // sqrt(3/5) / 2
    x = q == 0 ? 0.5 - a : (q == 1 ? 0.5 : 0.5 + a);
    w = q == 1 ? 8.0 / 18.0 : 5.0 / 18.0;
  }
}

template <int K>
__device__ __forceinline__ double lagr(int j, double t) {
  double v = 1.0;
  for (int m = 0; m <= K; ++m)
    if (m != j) v *= (t - (double)m / K) / ((double)(j - m) / K);
  return v;
}

template <int DIM, int K>
__global__ void rhs_sine_kernel(ActiveArgs a, const int32_t* __restrict__ coords, double* __restrict__ b,
                                bool one) {
  using G = ActGeo<DIM, K>;
  constexpr int N1 = G::N1, NC = G::NC;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cell = t / NC;
  const int n = (int)(t % NC);
  if (cell >= a.n_cells) return;
  const int lvl = a.cell_level[cell];
  const int i[3] = {n % N1, (n / N1) % N1, DIM == 3 ? n / (N1 * N1) : 0};
  double h[3], lo[3];
  for (int d = 0; d < 3; ++d) {
    h[d] = a.h[lvl][d];
    lo[d] = a.lo[d] + coords[3 * cell + d] * h[d];
  }
  const double PI = 3.14159265358979323846;
  double acc = 0.0;
  for (int qz = 0; qz < (DIM == 3 ? N1 : 1); ++qz)
    for (int qy = 0; qy < N1; ++qy)
      for (int qx = 0; qx < N1; ++qx) {
        double px, wx, py, wy, pz = 0.5, wz = 1.0;
        gauss_point<K>(qx, px, wx);
        gauss_point<K>(qy, py, wy);
        if (DIM == 3) gauss_point<K>(qz, pz, wz);
        double f = 1.0;
        if (!one) {
          f = DIM * PI * PI * sin(PI * (lo[0] + h[0] * px)) * sin(PI * (lo[1] + h[1] * py));
          if (DIM == 3) f *= sin(PI * (lo[2] + h[2] * pz));
        }
        double phi = lagr<K>(i[0], px) * lagr<K>(i[1], py) * (DIM == 3 ? lagr<K>(i[2], pz) : 1.0);
        acc += wx * wy * wz * f * phi;
      }
  acc *= h[0] * h[1] * (DIM == 3 ? h[2] : 1.0);
  int32_t id = a.cell_nodes[cell * NC + n];
  if (id >= 0) {
    atomicAdd(b + id, acc);
  } else if (id <= -2) {
    int hh = -2 - id;
    for (int m = a.hang_ptr[hh]; m < a.hang_ptr[hh + 1]; ++m)
      atomicAdd(b + a.hang_col[m], a.hw_table[a.hang_wc[m]] * acc);
  }
}

cudaError_t launch_rhs_sine(int dim, int k, const ActiveArgs& a, const int32_t* coords, double* b, bool one,
                            cudaStream_t s) {
  int nc = (dim == 3 ? (k + 1) * (k + 1) * (k + 1) : (k + 1) * (k + 1));
  int64_t n = a.n_cells * nc;
  if (n == 0) return cudaSuccess;
  unsigned grid = (unsigned)((n + 255) / 256);
  if (dim == 3 && k == 2) rhs_sine_kernel<3, 2><<<grid, 256, 0, s>>>(a, coords, b, one);
  else if (dim == 3 && k == 1) rhs_sine_kernel<3, 1><<<grid, 256, 0, s>>>(a, coords, b, one);
  else if (dim == 2 && k == 2) rhs_sine_kernel<2, 2><<<grid, 256, 0, s>>>(a, coords, b, one);
  else if (dim == 2 && k == 1) rhs_sine_kernel<2, 1><<<grid, 256, 0, s>>>(a, coords, b, one);
  else return cudaErrorInvalidValue;
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

// Seeded uniform right-hand side: the SplitMix64 output function (Steele,
// Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
// applied to seed xor (i * 0xD1B54A32D192ED03) for canonical index i; its
// top 53 bits give u in [0, 1), and b_i = 2 u - 1.
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) rhs_random_kernel(int64_t n, uint64_t seed, double* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t bits = splitmix64_out(seed ^ ((uint64_t)i * 0xD1B54A32D192ED03ull)) >> 11;
    const double u = (double)bits * (1.0 / 9007199254740992.0);
    b[i] = __dsub_rn(__dmul_rn(2.0, u), 1.0);
  }
}

cudaError_t launch_rhs_random(int64_t n, uint64_t seed, double* b, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  rhs_random_kernel<<<(unsigned)(g > 152 * 64 ? 152 * 64 : g), 256, 0, s>>>(n, seed, b);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ------------------------------------------------------------ copy maps
template <typename T>
__global__ void copy_to_mg_kernel(int64_t n, const double* __restrict__ r, const uint32_t* __restrict__ home,
                                  T* __restrict__ g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    g[home[i]] = (T)r[i];
}

template <typename T>
cudaError_t launch_copy_to_mg(int64_t n, const double* r, const uint32_t* home, T* g, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  copy_to_mg_kernel<T><<<(unsigned)(b > 152 * 64 ? 152 * 64 : b), 256, 0, s>>>(n, r, home, g);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) copy_from_mg_kernel(int64_t n, const T* __restrict__ u,
                                                           const uint32_t* __restrict__ home,
                                                           const double* __restrict__ r, double* __restrict__ z,
                                                           double* partials, unsigned* counter, double* rz_out) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)u[home[i]];
    z[i] = v;
    acc += r[i] * v;
  }
  double s = block_sum<256>(acc, sh);
  finish_reduction<256>(s, partials, counter, rz_out);
}

template <typename T>
cudaError_t launch_copy_from_mg(int64_t n, const T* u, const uint32_t* home, const double* r, double* z,
                                double* partials, unsigned* counter, double* rz_out, cudaStream_t s) {
  copy_from_mg_kernel<T><<<reduce_grid(n, 256), 256, 0, s>>>(n, u, home, r, z, partials, counter, rz_out);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ------------------------------------------------------------ coarse solve
// u0 = A0^{-1} g0 over the interior nodes of the coarse lattice (dense FP64 inverse).
template <typename T>
__global__ void coarse_solve_kernel(int64_t nc, const int32_t* __restrict__ slot, const double* __restrict__ inv,
                                    const T* __restrict__ g0, T* __restrict__ u0) {
  extern __shared__ double gs[];
  auto slot_of = [&](int64_t i) { return slot[i]; };
  for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) gs[i] = (double)g0[slot_of(i)];
  __syncthreads();
  // one warp per row: coalesced reads of the row, fixed-order reduction
  const int lane = threadIdx.x % 32;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= nc) return;
  const double* a = inv + row * nc;
  double acc = 0.0;
  for (int64_t j = lane; j < nc; j += 32) acc += a[j] * gs[j];
#pragma unroll
  for (int o = 16; o > 0; o /= 2) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) u0[slot_of(row)] = (T)acc;
}

template <typename T>
cudaError_t launch_coarse_solve(int64_t nc, const int32_t* slot, const double* inv, const T* g0, T* u0,
                                cudaStream_t s) {
  if (nc == 0) return cudaSuccess;
  size_t sm = (size_t)nc * sizeof(double);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  // set once, thread-safe (function-local static)
  static const bool init = [&] {
    cudaFuncSetAttribute(coarse_solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)init;
  unsigned grid = (unsigned)((nc + 7) / 8);  // 8 rows (warps) per block
  coarse_solve_kernel<T><<<grid, 256, sm, s>>>(nc, slot, inv, g0, u0);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

// Unpreconditioned CG coarse solver (Sec. 4.3): one block iterates from zero
// until ||r|| <= tol ||g|| or nc steps.  The vectors live in shared memory,
// and so does A_0 in CSR when it fits (`smem_matrix`); p.Ap is formed in the
// matrix-vector pass and r.r in the update pass, each reduced once per
// iteration in a fixed order (every thread sums the warp partials in warp
// order), with the two partial buffers used alternately so that one barrier
// per reduction suffices.
template <typename T>
__device__ __forceinline__ T coarse_block_sum(T v, T* red, int nwarps) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < nwarps; ++i) s += red[i];
  return s;
}

// The iteration runs in the level vectors' precision T: an FP32 V-cycle
// solves its coarse problem in FP32 (A_0 rounded to FP32 when it is staged),
// which on GB300 runs on the FP32 pipe instead of the FP64 pipe that issues
// two operations per clock per SM; an FP64 V-cycle solves it in FP64.
template <typename T>
__global__ void __launch_bounds__(1024) coarse_cg_kernel(int64_t nc, const int32_t* __restrict__ slot,
                                                         const int32_t* __restrict__ gptr,
                                                         const int32_t* __restrict__ gcol,
                                                         const double* __restrict__ gval, int64_t nnz,
                                                         bool smem_matrix, double tol, const T* __restrict__ g0,
                                                         T* __restrict__ u0) {
  extern __shared__ __align__(16) unsigned char cg_raw[];
  T* x = reinterpret_cast<T*>(cg_raw);
  T* r = x + nc;
  T* p = r + nc;
  T* Ap = p + nc;
  __shared__ T red[2][32];
  const int nwarps = (int)(blockDim.x >> 5);
  const int32_t* ptr = gptr;
  const int32_t* col = gcol;
  T* sval = Ap + nc;
  if (smem_matrix) {
    int32_t* scol = reinterpret_cast<int32_t*>(sval + nnz);
    int32_t* sptr = scol + nnz;
    for (int64_t m = threadIdx.x; m < nnz; m += blockDim.x) {
      sval[m] = (T)gval[m];
      scol[m] = gcol[m];
    }
    for (int64_t i = threadIdx.x; i <= nc; i += blockDim.x) sptr[i] = gptr[i];
    ptr = sptr;
    col = scol;
  }
  T part = 0;
  for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) {
    const T gi = g0[slot[i]];
    x[i] = 0;
    r[i] = gi;
    p[i] = gi;
    part += gi * gi;
  }
  int buf = 0;
  T rr = coarse_block_sum<T>(part, red[buf], nwarps);  // its barrier also publishes p
  const T stop = (T)(tol * tol) * rr;
  for (int64_t it = 0; it < nc && rr > stop; ++it) {
    part = 0;
    for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) {
      T t = 0;
      if (smem_matrix)
        for (int32_t m = ptr[i]; m < ptr[i + 1]; ++m) t += sval[m] * p[col[m]];
      else
        for (int32_t m = ptr[i]; m < ptr[i + 1]; ++m) t += (T)gval[m] * p[col[m]];
      Ap[i] = t;
      part += p[i] * t;
    }
    buf ^= 1;
    const T pAp = coarse_block_sum<T>(part, red[buf], nwarps);
    if (!(pAp > 0)) break;
    const T alpha = rr / pAp;
    part = 0;
    for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) {  // rows of this thread only
      x[i] += alpha * p[i];
      const T ri = r[i] - alpha * Ap[i];
      r[i] = ri;
      part += ri * ri;
    }
    buf ^= 1;
    const T rr_new = coarse_block_sum<T>(part, red[buf], nwarps);
    const T beta = rr_new / rr;
    rr = rr_new;
    if (!(rr > stop)) break;
    for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) p[i] = r[i] + beta * p[i];
    __syncthreads();  // p is read by every thread in the next product
  }
  for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) u0[slot[i]] = x[i];
}

template <typename T>
cudaError_t launch_coarse_cg(int64_t nc, const int32_t* slot, const int32_t* ptr, const int32_t* col,
                             const double* val, int64_t nnz, double tol, const T* g0, T* u0, cudaStream_t s) {
  if (nc == 0) return cudaSuccess;
  constexpr size_t kMax = 200 * 1024;
  const size_t vec = 4 * (size_t)nc * sizeof(T);
  if (vec > kMax) return cudaErrorInvalidValue;
  const size_t mat = (size_t)nnz * (sizeof(T) + sizeof(int32_t)) + (size_t)(nc + 1) * sizeof(int32_t);
  const bool smem_matrix = vec + mat <= kMax;
  const size_t sm = smem_matrix ? vec + mat : vec;
  // set once, thread-safe (function-local static)
  static const bool init = [&] {
    cudaFuncSetAttribute(coarse_cg_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMax);
    return true;
  }();
  (void)init;
  const unsigned threads = (unsigned)std::min<int64_t>(1024, (nc + 31) / 32 * 32);
  coarse_cg_kernel<T><<<1, threads, sm, s>>>(nc, slot, ptr, col, val, nnz, smem_matrix, tol, g0, u0);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}
template cudaError_t launch_coarse_cg<float>(int64_t, const int32_t*, const int32_t*, const int32_t*,
                                             const double*, int64_t, double, const float*, float*, cudaStream_t);
template cudaError_t launch_coarse_cg<double>(int64_t, const int32_t*, const int32_t*, const int32_t*,
                                              const double*, int64_t, double, const double*, double*, cudaStream_t);

// --------------------------------------------------------- vector kernels
template <typename T>
__global__ void scale_vec_kernel(int64_t n, const T* __restrict__ dinv, const T* __restrict__ g, T c,
                                 T* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = c * dinv[i] * g[i];
}

template <typename T>
cudaError_t launch_scale_vec(int64_t n, const T* dinv, const T* g, T c, T* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  scale_vec_kernel<T><<<(unsigned)(b > 152 * 64 ? 152 * 64 : b), 256, 0, s>>>(n, dinv, g, c, out);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) dot_kernel(int64_t n, const double* __restrict__ a,
                                                  const double* __restrict__ b, double* partials,
                                                  unsigned* counter, double* out) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  double s = block_sum<256>(acc, sh);
  finish_reduction<256>(s, partials, counter, out);
}

cudaError_t launch_dot(int64_t n, const double* a, const double* b, double* partials, unsigned* counter,
                       double* out, cudaStream_t s) {
  dot_kernel<<<reduce_grid(n, 256), 256, 0, s>>>(n, a, b, partials, counter, out);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

// --------------------------------------------- internal unknown numbering
// The device numbers the unknowns by their home slots (see device_setup); the
// caller's vectors are in canonical order.  dst[j] = src[perm[j]] brings a
// canonical vector in, dst[perm[j]] = src[j] takes an internal one out.
__global__ void __launch_bounds__(256) perm_gather_kernel(int64_t n, const int32_t* __restrict__ perm,
                                                          const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = src[perm[j]];
}
__global__ void __launch_bounds__(256) perm_scatter_kernel(int64_t n, const int32_t* __restrict__ perm,
                                                           const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    dst[perm[j]] = src[j];
}
cudaError_t launch_perm(int64_t n, const int32_t* perm, const double* src, double* dst, bool scatter,
                        cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  const unsigned grid = (unsigned)(b > 152 * 64 ? 152 * 64 : b);
  if (scatter) perm_scatter_kernel<<<grid, 256, 0, s>>>(n, perm, src, dst);
  else perm_gather_kernel<<<grid, 256, 0, s>>>(n, perm, src, dst);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ------------------------------------------- CG passes fused with the copies
// The outer CG of the solve keeps no z = B r vector: its entries are the
// level solutions at the unknowns' home slots, z_i = u[home_i], read where
// they are needed, and the level right-hand sides of the next V-cycle are
// written by the pass that updates r.

// The passes below are grid-stride loops unrolled four times: each thread
// first issues the independent loads of four entries (one grid stride apart,
// so every group of loads is coalesced), then the dependent gathers and
// stores, which keeps enough loads in flight to stream at HBM speed.
constexpr int kUnroll = 4;

// r = b, b.b, and g[home_i] = b_i (the first V-cycle's right-hand sides; g
// must be zero elsewhere; b may be r itself)
template <typename T>
__global__ void __launch_bounds__(256) cg_start_kernel(int64_t n, const double* b,
                                                       const uint32_t* __restrict__ home, double* r,
                                                       T* __restrict__ g, double* partials, unsigned* counter,
                                                       double* bb_out) {
  __shared__ double sh[8];
  double acc = 0.0;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUnroll - 1) * st < n; i += kUnroll * st) {
    double v[kUnroll];
    uint32_t hm[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      v[k] = b[i + k * st];
      hm[k] = home[i + k * st];
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      r[i + k * st] = v[k];
      g[hm[k]] = (T)v[k];
      acc += v[k] * v[k];
    }
  }
  for (; i < n; i += st) {
    const double v = b[i];
    r[i] = v;
    g[home[i]] = (T)v;
    acc += v * v;
  }
  double s = block_sum<256>(acc, sh);
  finish_reduction<256>(s, partials, counter, bb_out);
}

// r.z with z_i = u[home_i]
template <typename T>
__global__ void __launch_bounds__(256) cg_rz_kernel(int64_t n, const T* __restrict__ u,
                                                    const uint32_t* __restrict__ home, const double* __restrict__ r,
                                                    double* partials, unsigned* counter, double* rz_out) {
  __shared__ double sh[8];
  double acc = 0.0;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUnroll - 1) * st < n; i += kUnroll * st) {
    double rv[kUnroll];
    uint32_t hm[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      rv[k] = r[i + k * st];
      hm[k] = home[i + k * st];
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) acc += rv[k] * (double)u[hm[k]];
  }
  for (; i < n; i += st) acc += r[i] * (double)u[home[i]];
  double s = block_sum<256>(acc, sh);
  finish_reduction<256>(s, partials, counter, rz_out);
}

// p = z + beta p with z_i = u[home_i], beta = rz_new / rz_old, and Ap = 0
// (the leaf operator accumulates into it)
template <typename T>
__global__ void __launch_bounds__(256) cg_p_kernel(int64_t n, const T* __restrict__ u,
                                                   const uint32_t* __restrict__ home, double* __restrict__ p,
                                                   double* __restrict__ Ap, const double* rz_new,
                                                   const double* rz_old) {
  const double beta = *rz_new / *rz_old;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUnroll - 1) * st < n; i += kUnroll * st) {
    double pv[kUnroll];
    uint32_t hm[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      pv[k] = p[i + k * st];
      hm[k] = home[i + k * st];
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      p[i + k * st] = (double)u[hm[k]] + beta * pv[k];
      Ap[i + k * st] = 0.0;
    }
  }
  for (; i < n; i += st) {
    p[i] = (double)u[home[i]] + beta * p[i];
    Ap[i] = 0.0;
  }
}

// x += alpha p, r -= alpha Ap, r.r, and g[home_i] = r_i for the next V-cycle
// (alpha = rz / pAp read on the device; g must be zero elsewhere)
template <typename T>
__global__ void __launch_bounds__(256) cg_xr_kernel(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                    const double* __restrict__ p, const double* __restrict__ Ap,
                                                    const uint32_t* __restrict__ home, T* __restrict__ g,
                                                    const double* rz, const double* pAp, double* partials,
                                                    unsigned* counter, double* rr_out) {
  __shared__ double sh[8];
  const double alpha = *rz / *pAp;
  double acc = 0.0;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kUnroll - 1) * st < n; i += kUnroll * st) {
    double xv[kUnroll], rv[kUnroll], pv[kUnroll], av[kUnroll];
    uint32_t hm[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int64_t j = i + k * st;
      xv[k] = x[j];
      rv[k] = r[j];
      pv[k] = p[j];
      av[k] = Ap[j];
      hm[k] = home[j];
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int64_t j = i + k * st;
      x[j] = xv[k] + alpha * pv[k];
      const double ri = rv[k] - alpha * av[k];
      r[j] = ri;
      g[hm[k]] = (T)ri;
      acc += ri * ri;
    }
  }
  for (; i < n; i += st) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * Ap[i];
    r[i] = ri;
    g[home[i]] = (T)ri;
    acc += ri * ri;
  }
  double s = block_sum<256>(acc, sh);
  finish_reduction<256>(s, partials, counter, rr_out);
}

template <typename T>
cudaError_t launch_cg_start(int64_t n, const double* b, const uint32_t* home, double* r, T* g, double* partials,
                            unsigned* counter, double* bb_out, cudaStream_t s) {
  cg_start_kernel<T><<<reduce_grid(n, 256), 256, 0, s>>>(n, b, home, r, g, partials, counter, bb_out);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_rz(int64_t n, const T* u, const uint32_t* home, const double* r, double* partials,
                         unsigned* counter, double* rz_out, cudaStream_t s) {
  cg_rz_kernel<T><<<reduce_grid(n, 256), 256, 0, s>>>(n, u, home, r, partials, counter, rz_out);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_p(int64_t n, const T* u, const uint32_t* home, double* p, double* Ap, const double* rz_new,
                        const double* rz_old, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  cg_p_kernel<T><<<(unsigned)(b > 152 * 64 ? 152 * 64 : b), 256, 0, s>>>(n, u, home, p, Ap, rz_new, rz_old);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_xr(int64_t n, double* x, double* r, const double* p, const double* Ap, const uint32_t* home,
                         T* g, const double* rz, const double* pAp, double* partials, unsigned* counter,
                         double* rr_out, cudaStream_t s) {
  cg_xr_kernel<T><<<reduce_grid(n, 256), 256, 0, s>>>(n, x, r, p, Ap, home, g, rz, pAp, partials, counter, rr_out);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}
#define GMG_CG_INST(T)                                                                                          \
  template cudaError_t launch_cg_start<T>(int64_t, const double*, const uint32_t*, double*, T*, double*,        \
                                          unsigned*, double*, cudaStream_t);                                     \
  template cudaError_t launch_cg_rz<T>(int64_t, const T*, const uint32_t*, const double*, double*, unsigned*,   \
                                       double*, cudaStream_t);                                                   \
  template cudaError_t launch_cg_p<T>(int64_t, const T*, const uint32_t*, double*, double*, const double*,      \
                                      const double*, cudaStream_t);                                              \
  template cudaError_t launch_cg_xr<T>(int64_t, double*, double*, const double*, const double*, const uint32_t*, \
                                       T*, const double*, const double*, double*, unsigned*, double*, cudaStream_t);
GMG_CG_INST(float)
GMG_CG_INST(double)
#undef GMG_CG_INST

// ---------------------------------------------------- graph-mode CG control
// Single-thread kernels; the stopping rules are those of the stream-mode loop
// (NaN/Inf scalar, p.Ap <= 0, fixed count, ||r|| <= tol ||b||, limit).
__global__ void cg_graph_init_kernel(GraphCtl* c, cudaGraphConditionalHandle loop) {
  const double bb = c->bb;
  c->rz_old = 1.0;
  const bool go = bb > 0.0;
  if (!go) c->status = isnan(bb) ? GS_NAN : GS_DONE;
  cudaGraphSetConditional(loop, go ? 1u : 0u);
}

__global__ void cg_graph_check_kernel(GraphCtl* c, cudaGraphConditionalHandle loop) {
  const int it = c->it + 1;
  c->it = it;
  const double rz = c->rz, pAp = c->pAp, rr = c->rr;
  int status = GS_RUNNING;
  if (isnan(rz) || isnan(pAp) || isnan(rr) || isinf(rr))
    status = GS_NAN;
  else if (!(pAp > 0.0))
    status = GS_BREAKDOWN;
  else if (c->fixed > 0) {
    if (it == c->fixed) status = GS_DONE;
  } else if (sqrt(rr / c->bb) <= c->tol)
    status = GS_DONE;
  if (status == GS_RUNNING && it >= c->limit) status = GS_NOTCONV;
  c->status = status;
  c->rz_old = rz;
  cudaGraphSetConditional(loop, status == GS_RUNNING ? 1u : 0u);
}

cudaError_t launch_cg_graph_init(GraphCtl* c, cudaGraphConditionalHandle loop, cudaStream_t s) {
  cg_graph_init_kernel<<<1, 1, 0, s>>>(c, loop);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t launch_cg_graph_check(GraphCtl* c, cudaGraphConditionalHandle loop, cudaStream_t s) {
  cg_graph_check_kernel<<<1, 1, 0, s>>>(c, loop);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

__global__ void axpy_kernel(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
__global__ void mul_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}
__global__ void xpay_kernel(int64_t n, const double* __restrict__ x, double beta, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] + beta * y[i];
}
__global__ void d2f_kernel(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

static inline unsigned vgrid(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}
cudaError_t launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  axpy_kernel<<<vgrid(n), 256, 0, s>>>(n, a, x, y);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t launch_mul(int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
  mul_kernel<<<vgrid(n), 256, 0, s>>>(n, a, b, out);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t launch_xpay(int64_t n, const double* x, double beta, double* y, cudaStream_t s) {
  xpay_kernel<<<vgrid(n), 256, 0, s>>>(n, x, beta, y);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t launch_convert_d2f(int64_t n, const double* in, float* out, cudaStream_t s) {
  d2f_kernel<<<vgrid(n), 256, 0, s>>>(n, in, out);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

template cudaError_t launch_copy_to_mg<float>(int64_t, const double*, const uint32_t*, float*, cudaStream_t);
template cudaError_t launch_copy_to_mg<double>(int64_t, const double*, const uint32_t*, double*, cudaStream_t);
template cudaError_t launch_copy_from_mg<float>(int64_t, const float*, const uint32_t*, const double*, double*,
                                                double*, unsigned*, double*, cudaStream_t);
template cudaError_t launch_copy_from_mg<double>(int64_t, const double*, const uint32_t*, const double*, double*,
                                                 double*, unsigned*, double*, cudaStream_t);
template cudaError_t launch_coarse_solve<float>(int64_t, const int32_t*, const double*, const float*, float*,
                                                cudaStream_t);
template cudaError_t launch_coarse_solve<double>(int64_t, const int32_t*, const double*, const double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_scale_vec<float>(int64_t, const float*, const float*, float, float*, cudaStream_t);
template cudaError_t launch_scale_vec<double>(int64_t, const double*, const double*, double, double*,
                                              cudaStream_t);

}  // namespace gmg
