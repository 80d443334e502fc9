// Level kernels of the local-smoothing V-cycle (Sec. 2.3, Algorithm 2).
//
// Storage: level l >= 1 is a list of sibling groups (the 2^d children of a
// refined level-(l-1) cell).  A group's node block is the (2K+1)^d lattice
// of its cells' nodes; the group stores the (2K)^d nodes with local index
// < 2K, and nodes with local index 2K live in the +1 neighbour's block.
// nbr[g][o] (o in {-1,0,1}^d) is the block of the neighbour at offset o
// (a real group, a ghost block holding refinement-edge nodes, or -1 outside
// the brick); state[g] holds 2 bits per offset (refined / not refined
// inside / outside) and, in bits 60..62, the parent's position inside its
// own sibling group.
//
// The level operator on Cartesian cells is the Kronecker sum
//   A_cell = a_cell * sum_i s_i (K (x) M (x) M  with K in direction i),
// s_i = prod_{j != i} h_j / h_i, K and M the 1-D stiffness and mass
// matrices of Q_K on [0,1], evaluated by sum factorisation (Sec. 3.2).
//
// Smoothing / apply kernel: one pass per group that reads the (3K+1)^d halo
// [-K, 2K]^d around the group (cells of the group and of the 7 lower
// neighbours touch the group's stored nodes) and writes the group's stored
// nodes -- no atomics.  Rows of the 1-D matrices are "extended": rows
// 0..2K-1 hold the group's own two cells, row 2K the lower neighbour's cell
// at node 0; the extended result is combined with the coefficient of the
// group each row combination belongs to, so coefficient jumps between
// groups are exact.
//
// Residual + restriction kernel: per group, t = w g - A_G u on the group's
// (2K+1)^d nodes (A_G = the group's own cells, w = 1 / number of refined
// groups sharing the node), then R = P^T restricted to the parent cell's
// (K+1)^d nodes and accumulated atomically.  Summed over groups this is
// R (g - A u) exactly, without forming t.
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "int_split.cuh"

namespace gmg {

// ------------------------------------------------- 1-D closed-form tables
template <int K>
__host__ __device__ constexpr double mass1(int i, int j) {
  if constexpr (K == 1) {
    return i == j ? 1.0 / 3.0 : 1.0 / 6.0;
  } else {
    // (1/30) [[4, 2, -1], [2, 16, 2], [-1, 2, 4]]
    return (i == 1 && j == 1) ? 16.0 / 30.0
           : (i == 1 || j == 1) ? 2.0 / 30.0
           : (i == j) ? 4.0 / 30.0 : -1.0 / 30.0;
  }
}

template <int K>
__host__ __device__ constexpr double stiff1(int i, int j) {
  if constexpr (K == 1) {
    return i == j ? 1.0 : -1.0;
  } else {
    // (1/3) [[7, -8, 1], [-8, 16, -8], [1, -8, 7]]
    return (i == 1 && j == 1) ? 16.0 / 3.0
           : (i == 1 || j == 1) ? -8.0 / 3.0
           : (i == j) ? 7.0 / 3.0 : 1.0 / 3.0;
  }
}

template <int K, bool STIFF>
__host__ __device__ constexpr double elem1(int i, int j) {
  return STIFF ? stiff1<K>(i, j) : mass1<K>(i, j);
}

// parent basis function j evaluated at child node r (r = 0..2K) of the parent interval
template <int K>
__host__ __device__ constexpr double embed1(int r, int j) {
  if constexpr (K == 1) {
    return r == 1 ? 0.5 : ((r == 0) == (j == 0) ? 1.0 : 0.0);
  } else {
    if (r == 0) return j == 0 ? 1.0 : 0.0;
    if (r == 2) return j == 1 ? 1.0 : 0.0;
    if (r == 4) return j == 2 ? 1.0 : 0.0;
    if (r == 1) return j == 0 ? 0.375 : (j == 1 ? 0.75 : -0.125);
    return j == 0 ? -0.125 : (j == 1 ? 0.75 : 0.375);  // r == 3
  }
}

// extended halo matrix: rows e in [0, 2K], halo columns c in [0, 3K] (position c - K)
template <int K, bool STIFF>
__host__ __device__ constexpr double bext(int e, int c) {
  int p = c - K;
  double v = 0.0;
  if (e < 2 * K) {
    for (int cell = 0; cell < 2; ++cell) {
      int lo = K * cell;
      if (e >= lo && e <= lo + K && p >= lo && p <= lo + K) v += elem1<K, STIFF>(e - lo, p - lo);
    }
  } else if (p >= -K && p <= 0) {
    v = elem1<K, STIFF>(K, p + K);
  }
  return v;
}

// group-local matrix over the group's two cells, (2K+1) x (2K+1)
template <int K, bool STIFF>
__host__ __device__ constexpr double bgrp(int a, int b) {
  double v = 0.0;
  for (int cell = 0; cell < 2; ++cell) {
    int lo = K * cell;
    if (a >= lo && a <= lo + K && b >= lo && b <= lo + K) v += elem1<K, STIFF>(a - lo, b - lo);
  }
  return v;
}

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// The last stage of the sum factorisations gives a thread the output rows
// r = part + R o (o = 0, 1, ...), r < N.  `part` is uniform over a warp, so
// one branch per part selects fully unrolled bodies in which r and o are
// compile-time constants: f(o, r).
template <int N, int R, class F>
__device__ __forceinline__ void own_rows(int part, F&& f) {
  static_for<0, R>([&](auto p) {
    if (part == p) {
      static_for<0, (N - p + R - 1) / R>([&](auto o) { f(o, std::integral_constant<int, p + R * o>{}); });
    }
  });
}

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

template <int DIM, int K>
struct Geo {
  static constexpr int NH = 3 * K + 1;   // halo nodes per direction
  static constexpr int NE = 2 * K + 1;   // extended rows per direction
  static constexpr int NO = 2 * K;       // stored nodes per direction of a block
  static constexpr int NG = 2 * K + 1;   // group nodes per direction
  static constexpr int N1 = K + 1;       // cell nodes per direction
  static constexpr int NOWN = ipow_c(NO, DIM);
  static constexpr int NHALO = ipow_c(NH, DIM);
  static constexpr int NGRP = ipow_c(NG, DIM);
  static constexpr int NCELL = ipow_c(N1, DIM);
  static constexpr int NNB = ipow_c(3, DIM);
  static constexpr int TEAM = NOWN;      // threads per group
  static constexpr int GPB = TEAM >= 256 ? 1 : 256 / TEAM;  // groups per block
};

// index of neighbour offset (ox, oy, oz) in a group's 3^DIM neighbour table
template <int DIM>
__device__ __forceinline__ int nbi(int ox, int oy, int oz) {
  return DIM == 3 ? (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1) : (ox + 1) + 3 * (oy + 1);
}

__device__ __forceinline__ int state_of(uint64_t st, int nb) { return (int)((st >> (2 * nb)) & 3); }

// class of a node from its touching-offset ranges: 1 S, 2 I, 3 D
template <int DIM>
__device__ __forceinline__ int node_class(uint64_t st, const int* lo_o, const int* hi_o) {
  bool outside = false, ghost = false;
  for (int oz = (DIM > 2 ? lo_o[2] : 0); oz <= (DIM > 2 ? hi_o[2] : 0); ++oz)
    for (int oy = lo_o[1]; oy <= hi_o[1]; ++oy)
      for (int ox = lo_o[0]; ox <= hi_o[0]; ++ox) {
        int s = state_of(st, nbi<DIM>(ox, oy, oz));
        outside |= (s == kStateOutside);
        ghost |= (s == kStateGhost);
      }
  return outside ? 3 : (ghost ? 2 : 1);
}

// ------------------------------------------------------ smoothing kernel
template <typename T, int DIM, int K>
struct ChebSmem {
  using G = Geo<DIM, K>;
  static constexpr int X = G::NHALO;
  static constexpr int T1 = (DIM == 3 ? G::NH * G::NH : G::NH) * G::NE;  // per array
  static constexpr int T2 = DIM == 3 ? G::NH * G::NE * G::NE : 0;         // per array
  static constexpr int Y = ipow_c(G::NE, DIM);
  static constexpr int PER_GROUP = X + 2 * T1 + 3 * T2 + Y + (1 << DIM);
  static constexpr size_t HEADER = ((size_t)G::GPB * (8 + 4 * G::NNB) + 15) / 16 * 16;
  static constexpr size_t bytes() { return HEADER + (size_t)G::GPB * PER_GROUP * sizeof(T); }
};

// Sum-factorised extended operator: X (halo, NH^DIM) -> Y (NE^DIM, unscaled by coefficients).
template <typename T, int DIM, int K>
__device__ __forceinline__ void ext_operator(const T* X, T* T1M, T* T1K, T* T2MM, T* T2MK, T* T2KM,
                                             T* Y, int lane, const T* scale) {
  using G = Geo<DIM, K>;
  constexpr int NH = G::NH, NE = G::NE;
  const T sx = scale[0], sy = scale[1], sz = scale[2];
  if constexpr (DIM == 3) {
    // stage x: lines (z, y)
    for (int line = lane; line < NH * NH; line += G::TEAM) {
      const T* in = X + line * NH;
      T v[NH];
      static_for<0, NH>([&](auto c) { v[c] = in[c]; });
      static_for<0, NE>([&](auto e) {
        T m = 0, kk = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bext<K, false>(e, c);
          constexpr double bk = bext<K, true>(e, c);
          if constexpr (bm != 0.0) m += (T)bm * v[c];
          if constexpr (bk != 0.0) kk += (T)bk * v[c];
        });
        T1M[line * NE + e] = m;
        T1K[line * NE + e] = kk;
      });
    }
    __syncthreads();
    // stage y: lines (z, ex); T1 layout [z][y][ex]
    for (int line = lane; line < NH * NE; line += G::TEAM) {
      int z = line / NE, ex = line % NE;
      T vm[NH], vk[NH];
      static_for<0, NH>([&](auto y) {
        vm[y] = T1M[(z * NH + y) * NE + ex];
        vk[y] = T1K[(z * NH + y) * NE + ex];
      });
      static_for<0, NE>([&](auto e) {
        T mm = 0, mk = 0, km = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bext<K, false>(e, c);
          constexpr double bk = bext<K, true>(e, c);
          if constexpr (bm != 0.0) {
            mm += (T)bm * vm[c];
            km += (T)bm * vk[c];
          }
          if constexpr (bk != 0.0) mk += (T)bk * vm[c];
        });
        int o = (z * NE + e) * NE + ex;  // [z][ey][ex]
        T2MM[o] = mm;
        T2MK[o] = mk;
        T2KM[o] = km;
      });
    }
    __syncthreads();
    // stage z: lines (ey, ex); T2 layout [z][ey][ex]
    for (int line = lane; line < NE * NE; line += G::TEAM) {
      T a[NH], b[NH];
      static_for<0, NH>([&](auto z) {
        a[z] = T2MM[z * NE * NE + line];
        b[z] = sy * T2MK[z * NE * NE + line] + sx * T2KM[z * NE * NE + line];
      });
      static_for<0, NE>([&](auto e) {
        T acc = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bext<K, false>(e, c);
          constexpr double bk = bext<K, true>(e, c);
          if constexpr (bk != 0.0) acc += (T)bk * sz * a[c];
          if constexpr (bm != 0.0) acc += (T)bm * b[c];
        });
        Y[e * NE * NE + line] = acc;
      });
    }
    __syncthreads();
  } else {
    // DIM == 2: stage x over lines y, then stage y
    for (int line = lane; line < NH; line += G::TEAM) {
      const T* in = X + line * NH;
      T v[NH];
      static_for<0, NH>([&](auto c) { v[c] = in[c]; });
      static_for<0, NE>([&](auto e) {
        T m = 0, kk = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bext<K, false>(e, c);
          constexpr double bk = bext<K, true>(e, c);
          if constexpr (bm != 0.0) m += (T)bm * v[c];
          if constexpr (bk != 0.0) kk += (T)bk * v[c];
        });
        T1M[line * NE + e] = m;
        T1K[line * NE + e] = kk;
      });
    }
    __syncthreads();
    for (int line = lane; line < NE; line += G::TEAM) {
      T vm[NH], vk[NH];
      static_for<0, NH>([&](auto y) {
        vm[y] = T1M[y * NE + line];
        vk[y] = T1K[y * NE + line];
      });
      static_for<0, NE>([&](auto e) {
        T acc = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bext<K, false>(e, c);
          constexpr double bk = bext<K, true>(e, c);
          if constexpr (bk != 0.0) acc += (T)bk * sy * vm[c];
          if constexpr (bm != 0.0) acc += (T)bm * sx * vk[c];
        });
        Y[e * NE + line] = acc;
      });
    }
    __syncthreads();
  }
}

// Scale factors and coefficients in the kernel's precision (no FP64 work in
// the FP32 kernels: FP64 throughput is a small fraction of FP32 on this GPU).
template <typename T>
__device__ __forceinline__ T level_scale(const LevelArgs& a, int d) {
  if constexpr (std::is_same<T, float>::value) return a.scale32[d];
  else return a.scale[d];
}
template <typename T>
__device__ __forceinline__ const T* lower_coefs(const LevelArgs& a) {
  if constexpr (std::is_same<T, float>::value) return a.lcoef32;
  else return a.lcoef64;
}
template <typename T>
__device__ __forceinline__ T group_coef(const LevelArgs& a, int64_t g) {
  if constexpr (std::is_same<T, float>::value) return a.coeff32[g];
  else return a.coeff[g];
}

// Load the (3K+1)^d halo of a group into X, one neighbour block at a time.
// Along each direction the halo [-K, 2K] is three segments: positions
// -K..-1 (stored nodes K..2K-1 of the -1 neighbour), 0..2K-1 (own block) and
// 2K (node 0 of the +1 neighbour); the sub-box of every neighbour block has
// compile-time extents, so decoding an element index is shifts and masks.
template <int K>
struct Seg {
  __device__ static constexpr int len(int o) { return o < 0 ? K : (o == 0 ? 2 * K : 1); }
  __device__ static constexpr int src(int o) { return o < 0 ? K : 0; }       // first stored index read
  __device__ static constexpr int dst(int o) { return o < 0 ? 0 : (o == 0 ? K : 3 * K); }  // halo index
};

template <typename T, int DIM, int K>
__device__ __forceinline__ void load_halo(const T* __restrict__ x, const int32_t* nb, T* X, int lane) {
  using G = Geo<DIM, K>;
  constexpr int NH = G::NH, NO = G::NO;
  static_for<0, G::NNB>([&](auto ni) {
    constexpr int ox = ni % 3 - 1;
    constexpr int oy = DIM > 1 ? (ni / 3) % 3 - 1 : 0;
    constexpr int oz = DIM > 2 ? ni / 9 - 1 : 0;
    constexpr int LX = Seg<K>::len(ox), LY = DIM > 1 ? Seg<K>::len(oy) : 1, LZ = DIM > 2 ? Seg<K>::len(oz) : 1;
    constexpr int COUNT = LX * LY * LZ;
    const int32_t blk = nb[ni];
    const T* src = x + (int64_t)(blk < 0 ? 0 : blk) * G::NOWN;
    for (int e = lane; e < COUNT; e += G::TEAM) {
      const int a = e % LX, b = (e / LX) % LY, c = e / (LX * LY);
      const int s = (Seg<K>::src(ox) + a) + NO * ((DIM > 1 ? Seg<K>::src(oy) + b : 0) +
                                                   NO * (DIM > 2 ? Seg<K>::src(oz) + c : 0));
      const int h = (Seg<K>::dst(ox) + a) + NH * ((DIM > 1 ? Seg<K>::dst(oy) + b : 0) +
                                                   NH * (DIM > 2 ? Seg<K>::dst(oz) + c : 0));
      X[h] = blk < 0 ? T(0) : src[s];
    }
  });
}

// mode: 0 = apply (out[S] = A x), 1 = Chebyshev step
//   out[S] = x + c1 (x - xprev) + c2 dinv (g - A x)
template <typename T, int DIM, int K, int MODE>
__global__ void __launch_bounds__(Geo<DIM, K>::GPB * Geo<DIM, K>::TEAM)
level_cheb_kernel(LevelArgs a, const T* __restrict__ x, const T* xprev,
                  const T* __restrict__ gvec, const T* __restrict__ dinv, T* out, T c1, T c2) {
  using G = Geo<DIM, K>;
  using S = ChebSmem<T, DIM, K>;
  constexpr int NO = G::NO, NE = G::NE, ND = 1 << DIM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / G::TEAM;
  const int lane = threadIdx.x % G::TEAM;
  const int64_t t = (int64_t)blockIdx.x * G::GPB + team;
  const bool active = t < a.n_jump;
  const int64_t g = active ? a.list_jump[t] : 0;
  uint64_t* masks = reinterpret_cast<uint64_t*>(smem_raw);
  int32_t* nbs = reinterpret_cast<int32_t*>(masks + G::GPB) + team * G::NNB;
  T* base = reinterpret_cast<T*>(smem_raw + S::HEADER) + (size_t)team * S::PER_GROUP;
  T* X = base;
  T* T1M = X + S::X;
  T* T1K = T1M + S::T1;
  T* T2MM = T1K + S::T1;
  T* T2MK = T2MM + S::T2;
  T* T2KM = T2MK + S::T2;
  T* Y = T2KM + S::T2;
  T* coefs = Y + S::Y;
  if (active) {
    for (int i = lane; i < G::NNB; i += G::TEAM) nbs[i] = a.nbr[g * G::NNB + i];
    if (lane < ND) coefs[lane] = lower_coefs<T>(a)[g * ND + lane];
    if (lane == 0) masks[team] = a.smask[g];
  }
  __syncthreads();
  if (active) load_halo<T, DIM, K>(x, nbs, X, lane);
  __syncthreads();
  const T sc[3] = {level_scale<T>(a, 0), level_scale<T>(a, 1), level_scale<T>(a, 2)};
  ext_operator<T, DIM, K>(X, T1M, T1K, T2MM, T2MK, T2KM, Y, active ? lane : G::TEAM, sc);
  if (!active || !((masks[team] >> lane) & 1ull)) return;  // only S nodes are written
  // combine extended rows: rows 2K stand for the lower neighbour's cell at node 0
  const int i0 = lane % NO, i1 = DIM > 1 ? (lane / NO) % NO : 0, i2 = DIM > 2 ? lane / (NO * NO) : 0;
  T y = 0;
  const int nbx = i0 == 0 ? 2 : 1, nby = (DIM > 1 && i1 == 0) ? 2 : 1, nbz = (DIM > 2 && i2 == 0) ? 2 : 1;
  for (int bz = 0; bz < nbz; ++bz)
    for (int by = 0; by < nby; ++by)
      for (int bx = 0; bx < nbx; ++bx) {
        const int ex = bx ? 2 * K : i0, ey = by ? 2 * K : i1, ez = bz ? 2 * K : i2;
        const int yi = DIM == 3 ? (ez * NE + ey) * NE + ex : ey * NE + ex;
        y += coefs[bx | (by << 1) | (bz << 2)] * Y[yi];
      }
  const int64_t slot = g * G::NOWN + lane;
  if constexpr (MODE == 0) {
    out[slot] = y;
  } else {
    const int hx = (i0 + K) + G::NH * ((DIM > 1 ? i1 + K : 0) + G::NH * (DIM > 2 ? i2 + K : 0));
    const T xv = X[hx];
    const T xp = xprev ? xprev[slot] : T(0);
    out[slot] = xv + c1 * (xv - xp) + c2 * dinv[slot] * (gvec[slot] - y);
  }
}

// ------------------------------------------- smoothing kernel, uniform groups
// Groups whose refined lower neighbours all share the group's coefficient:
// the lower neighbour's cell at node 0 merges into row 0 of the 1-D matrices,
// and one tensor product with (2K) x (3K+1) matrices gives the operator on
// the stored nodes.  (Rows of nodes next to a missing neighbour pick up terms
// of cells that do not exist, but those nodes are I or Dirichlet nodes and
// are never written.)  A team of TW threads (within one warp) handles one
// group, synchronising with __syncwarp only:
//   stage 1: each thread loads one halo row along x (three vector loads: the
//            -1, own and +1 blocks) and contracts it in registers;
//   stage 2: y-contraction on shared memory;
//   stage 3: z-contraction fused with the Chebyshev update of its nodes.
template <int K, bool STIFF>
__host__ __device__ constexpr double bmerged(int r, int c) {
  return bext<K, STIFF>(r, c) + (r == 0 ? bext<K, STIFF>(2 * K, c) : 0.0);
}

template <int DIM, int K>
struct Fast {
  static constexpr int NH = 3 * K + 1, NO = 2 * K;
  static constexpr int NOWN = ipow_c(NO, DIM), NNB = ipow_c(3, DIM);
  static constexpr int L1 = DIM == 3 ? NH * NH : NH;  // stage-1 lines
  static constexpr int TW = DIM == 3 ? (K == 2 ? 32 : 16) : (K == 2 ? 8 : 4);
  static constexpr int TPB = 256 / TW;               // teams per block
};

template <typename T, int DIM, int K>
struct FastSmem {
  using F = Fast<DIM, K>;
  static constexpr int T1 = F::L1 * F::NO;
  static constexpr int T2 = DIM == 3 ? F::NH * F::NO * F::NO : 0;
  static constexpr int PER = 2 * T1 + 3 * T2 + F::NOWN;
  static constexpr size_t HEADER = ((size_t)F::TPB * (8 + sizeof(T) + 4 * F::NNB) + 15) / 16 * 16;
  static constexpr size_t bytes() { return HEADER + (size_t)F::TPB * PER * sizeof(T); }
};

// N consecutive values from an address aligned to N * sizeof(T) (N = 1, 2, 4)
template <typename T, int N>
__device__ __forceinline__ void load_run(const T* __restrict__ p, T* v) {
  if constexpr (N == 4 && sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (N == 2 && sizeof(T) == 4) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else if constexpr (N == 4 && sizeof(T) == 8) {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
  } else if constexpr (N == 2 && sizeof(T) == 8) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}

// halo index h in [0, 3K] -> neighbour offset and stored index in that block
template <int K>
__device__ __forceinline__ void halo_seg(int h, int& o, int& l) {
  o = h < K ? -1 : (h < 3 * K ? 0 : 1);
  l = h < K ? h + K : (h < 3 * K ? h - K : 0);
}

// store N consecutive values to shared memory (vector stores where aligned)
template <typename T, int N>
__device__ __forceinline__ void store_run(T* p, const T* v) {
  if constexpr (N == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (N == 2 && sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (N == 4 && sizeof(T) == 8) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  } else if constexpr (N == 2 && sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v[i];
  }
}

// diagonal entry of the merged 1-D matrix at stored node i
template <int K, bool STIFF>
__device__ __forceinline__ double merged_diag(int i) {
  double v = 0.0;
  static_for<0, 2 * K>([&](auto r) {
    if (i == r) v = bmerged<K, STIFF>(r, K + r);
  });
  return v;
}

// One single group (list entry t of list_uniform; none if t >= n_uniform)
// smoothed by one team of TW threads: its mask and coefficient slots, its
// 3^d neighbour table and its S::PER values of shared memory.
template <typename T, int DIM, int K, int MODE>
__device__ __forceinline__ void fast_group_step(const LevelArgs& a, int64_t t, int lane, uint64_t* mask_slot,
                                                T* coef_slot, int32_t* nb, T* T1M, const T* __restrict__ x,
                                                const T* xprev, const T* __restrict__ gvec, T* out, T c1, T c2) {
  using F = Fast<DIM, K>;
  using S = FastSmem<T, DIM, K>;
  constexpr int NH = F::NH, NO = F::NO, TW = F::TW;
  // last stage: L3 lines of NO outputs, R threads per line
  constexpr int L3 = DIM == 3 ? NO * NO : NO;
  constexpr int R = TW / L3 > 0 ? TW / L3 : 1;
  constexpr int OPT = (NO + R - 1) / R;  // outputs per thread
  const bool active = t < a.n_uniform;
  const int64_t g = active ? a.list_uniform[t] : 0;
  T* T1K = T1M + S::T1;
  T* T2MM = T1K + S::T1;
  T* T2MK = T2MM + S::T2;
  T* T2KM = T2MK + S::T2;
  T* Xown = T2KM + S::T2;
  // this thread's output nodes: line `ol`, outputs k = part + R * o
  const int ol = lane % L3, part = lane / L3;
  const bool has_out = lane < L3 * R;
  // prefetch the update's operands; they are used only after the contractions
  T pre_xp[OPT], pre_g[OPT];
  if constexpr (MODE == 1) {
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
      const int kk = part + R * o;
      pre_xp[o] = T(0);
      pre_g[o] = T(0);
      if (active && has_out && kk < NO) {
        const int64_t slot = g * F::NOWN + ol + L3 * kk;
        pre_g[o] = gvec[slot];
        if (xprev) pre_xp[o] = xprev[slot];
      }
    }
  }
  if (active) {
    for (int i = lane; i < F::NNB; i += TW) nb[i] = a.nbr[g * F::NNB + i];
    if (lane == 0) {
      *mask_slot = a.smask[g];
      *coef_slot = group_coef<T>(a, g);
    }
  }
  __syncwarp();
  // stage 1: halo rows along x, contracted with the merged 1-D matrices
  if (active) {
    for (int line = lane; line < F::L1; line += TW) {
      int oy = 0, ly = 0, oz = 0, lz = 0;
      halo_seg<K>(DIM == 3 ? line % NH : line, oy, ly);
      if constexpr (DIM == 3) halo_seg<K>(line / NH, oz, lz);
      const int row = NO * (ly + NO * lz);
      T v[NH];
      const int32_t b0 = nb[nbi<DIM>(-1, oy, oz)], b1 = nb[nbi<DIM>(0, oy, oz)], b2 = nb[nbi<DIM>(1, oy, oz)];
      if (b0 >= 0) load_run<T, K>(x + (int64_t)b0 * F::NOWN + row + K, v);
      else for (int i = 0; i < K; ++i) v[i] = T(0);
      if (b1 >= 0) load_run<T, 2 * K>(x + (int64_t)b1 * F::NOWN + row, v + K);
      else for (int i = 0; i < 2 * K; ++i) v[K + i] = T(0);
      v[3 * K] = b2 >= 0 ? x[(int64_t)b2 * F::NOWN + row] : T(0);
      if (oy == 0 && oz == 0) store_run<T, NO>(Xown + row, v + K);
      T m[NO], k[NO];
      static_for<0, NO>([&](auto r) {
        T sm = 0, sk = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bmerged<K, false>(r, c);
          constexpr double bk = bmerged<K, true>(r, c);
          if constexpr (bm != 0.0) sm += (T)bm * v[c];
          if constexpr (bk != 0.0) sk += (T)bk * v[c];
        });
        m[r] = sm;
        k[r] = sk;
      });
      store_run<T, NO>(T1M + line * NO, m);
      store_run<T, NO>(T1K + line * NO, k);
    }
  }
  __syncwarp();
  const T sx = level_scale<T>(a, 0), sy = level_scale<T>(a, 1), sz = level_scale<T>(a, 2);
  const uint64_t smask = *mask_slot;
  const T coef = *coef_slot;
  // Chebyshev update of stored node `node`.  D^{-1} of an S node of a uniform
  // group is the inverse of coef * sum_d s_d prod_e (diagonal of the merged
  // 1-D matrices); that diagonal depends on an index only through its parity,
  // and all outputs of this thread share one parity pattern (R is even or the
  // thread has one output), so one reciprocal serves them.
  T c2d = T(0);
  if constexpr (MODE == 1) {
    const T md0 = (T)bmerged<K, false>(0, K), kd0 = (T)bmerged<K, true>(0, K);
    const T md1 = (T)bmerged<K, false>(1, K + 1), kd1 = (T)bmerged<K, true>(1, K + 1);
    const int p0 = (DIM == 3 ? ol % NO : ol) & 1, p1 = (DIM == 3 ? ol / NO : part) & 1, p2 = part & 1;
    const T mdx = p0 ? md1 : md0, kdx = p0 ? kd1 : kd0;
    const T mdy = p1 ? md1 : md0, kdy = p1 ? kd1 : kd0;
    T diag;
    if constexpr (DIM == 3) {
      const T mdz = p2 ? md1 : md0, kdz = p2 ? kd1 : kd0;
      diag = coef * (sx * kdx * mdy * mdz + sy * mdx * kdy * mdz + sz * mdx * mdy * kdz);
    } else {
      diag = coef * (sx * kdx * mdy + sy * mdx * kdy);
    }
    c2d = c2 / diag;
  }
  static_assert(R % 2 == 0 || OPT == 1, "outputs of a thread must share one parity pattern");
  auto update = [&](int node, T y, int o) {
    if (!((smask >> node) & 1ull)) return;
    const int64_t slot = g * F::NOWN + node;
    y *= coef;
    if constexpr (MODE == 0) {
      out[slot] = y;
    } else {
      const T xv = Xown[node];
      out[slot] = xv + c1 * (xv - pre_xp[o]) + c2d * (pre_g[o] - y);
    }
  };
  if constexpr (DIM == 3) {
    // stage 2: y direction; T1 layout [z][y][i] -> T2 layout [z][j][i]
    if (active) {
      for (int line = lane; line < NH * NO; line += TW) {
        const int z = line / NO, i = line % NO;
        T vm[NH], vk[NH];
        static_for<0, NH>([&](auto y) {
          vm[y] = T1M[(z * NH + y) * NO + i];
          vk[y] = T1K[(z * NH + y) * NO + i];
        });
        static_for<0, NO>([&](auto j) {
          T mm = 0, mk = 0, km = 0;
          static_for<0, NH>([&](auto c) {
            constexpr double bm = bmerged<K, false>(j, c);
            constexpr double bk = bmerged<K, true>(j, c);
            if constexpr (bm != 0.0) {
              mm += (T)bm * vm[c];
              km += (T)bm * vk[c];
            }
            if constexpr (bk != 0.0) mk += (T)bk * vm[c];
          });
          const int o = (z * NO + j) * NO + i;
          T2MM[o] = mm;
          T2MK[o] = mk;
          T2KM[o] = km;
        });
      }
    }
    __syncwarp();
    // stage 3: z direction for this thread's outputs, then the update
    if (active && has_out) {
      T p[NH], q[NH];
      static_for<0, NH>([&](auto z) {
        p[z] = sz * T2MM[z * L3 + ol];
        q[z] = sy * T2MK[z * L3 + ol] + sx * T2KM[z * L3 + ol];
      });
#pragma unroll
      for (int o = 0; o < OPT; ++o) {
        const int kk = part + R * o;
        if (kk >= NO) break;
        T y = 0;
        static_for<0, NO>([&](auto r) {
          if (kk == r) {
            static_for<0, NH>([&](auto c) {
              constexpr double bm = bmerged<K, false>(r, c);
              constexpr double bk = bmerged<K, true>(r, c);
              if constexpr (bk != 0.0) y += (T)bk * p[c];
              if constexpr (bm != 0.0) y += (T)bm * q[c];
            });
          }
        });
        update(ol + L3 * kk, y, o);
      }
    }
  } else {
    if (active && has_out) {
      T vm[NH], vk[NH];
      static_for<0, NH>([&](auto y) {
        vm[y] = sy * T1M[y * NO + ol];
        vk[y] = sx * T1K[y * NO + ol];
      });
#pragma unroll
      for (int o = 0; o < OPT; ++o) {
        const int kk = part + R * o;
        if (kk >= NO) break;
        T y = 0;
        static_for<0, NO>([&](auto r) {
          if (kk == r) {
            static_for<0, NH>([&](auto c) {
              constexpr double bm = bmerged<K, false>(r, c);
              constexpr double bk = bmerged<K, true>(r, c);
              if constexpr (bk != 0.0) y += (T)bk * vm[c];
              if constexpr (bm != 0.0) y += (T)bm * vk[c];
            });
          }
        });
        update(ol + L3 * kk, y, o);
      }
    }
  }
}

template <typename T, int DIM, int K, int MODE>
__global__ void __launch_bounds__(256)
level_cheb_fast_kernel(LevelArgs a, const T* __restrict__ x, const T* xprev, const T* __restrict__ gvec, T* out,
                       T c1, T c2) {
  using F = Fast<DIM, K>;
  using S = FastSmem<T, DIM, K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / F::TW, lane = threadIdx.x % F::TW;
  uint64_t* masks = reinterpret_cast<uint64_t*>(smem_raw);
  T* coefs = reinterpret_cast<T*>(masks + F::TPB);
  int32_t* nb = reinterpret_cast<int32_t*>(coefs + F::TPB) + team * F::NNB;
  T* base = reinterpret_cast<T*>(smem_raw + S::HEADER) + (size_t)team * S::PER;
  fast_group_step<T, DIM, K, MODE>(a, (int64_t)blockIdx.x * F::TPB + team, lane, masks + team, coefs + team, nb,
                                   base, x, xprev, gvec, out, c1, c2);
}


// ------------------------------- smoothing kernel, groups at coefficient jumps
// The extended operator of level_cheb_kernel (rows 0..2K-1 for the group's
// own cells, row 2K for the lower neighbour's cell, combined per neighbour
// coefficient) with the memory pattern of level_cheb_fast_kernel: one warp
// per group, halo rows by vector loads, warp-level synchronisation only.
template <typename T, int K>
struct JumpSmem {
  using F = Fast<3, K>;
  static constexpr int NE = 2 * K + 1;
  static constexpr int T1 = F::L1 * NE;
  static constexpr int T2 = F::NH * NE * NE;
  static constexpr int Y = NE * NE * NE;
  static constexpr int PER = 2 * T1 + 3 * T2 + Y + F::NOWN + 8;
  static constexpr size_t HEADER = ((size_t)F::TPB * (8 + 4 * F::NNB) + 15) / 16 * 16;
  static constexpr size_t bytes() { return HEADER + (size_t)F::TPB * PER * sizeof(T); }
};

template <typename T, int K, int MODE>
__global__ void __launch_bounds__(256)
level_cheb_jump_kernel(LevelArgs a, const T* __restrict__ x, const T* xprev, const T* __restrict__ gvec,
                       const T* __restrict__ dinv, T* out, T c1, T c2) {
  using F = Fast<3, K>;
  using S = JumpSmem<T, K>;
  constexpr int NH = F::NH, NO = F::NO, TW = F::TW, NE = S::NE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / TW;
  const int lane = threadIdx.x % TW;
  const int64_t t = (int64_t)blockIdx.x * F::TPB + team;
  const bool active = t < a.n_jump;
  const int64_t g = active ? a.list_jump[t] : 0;
  uint64_t* masks = reinterpret_cast<uint64_t*>(smem_raw);
  int32_t* nb = reinterpret_cast<int32_t*>(masks + F::TPB) + team * F::NNB;
  T* T1M = reinterpret_cast<T*>(smem_raw + S::HEADER) + (size_t)team * S::PER;
  T* T1K = T1M + S::T1;
  T* T2MM = T1K + S::T1;
  T* T2MK = T2MM + S::T2;
  T* T2KM = T2MK + S::T2;
  T* Y = T2KM + S::T2;
  T* Xown = Y + S::Y;
  T* coefs = Xown + F::NOWN;
  if (active) {
    for (int i = lane; i < F::NNB; i += TW) nb[i] = a.nbr[g * F::NNB + i];
    if (lane < 8) coefs[lane] = lower_coefs<T>(a)[g * 8 + lane];
    if (lane == 0) masks[team] = a.smask[g];
  }
  __syncwarp();
  const T sx = level_scale<T>(a, 0), sy = level_scale<T>(a, 1), sz = level_scale<T>(a, 2);
  if (active) {
    // stage 1: halo rows along x -> extended mass and stiffness rows
    for (int line = lane; line < F::L1; line += TW) {
      int oy = 0, ly = 0, oz = 0, lz = 0;
      halo_seg<K>(line % NH, oy, ly);
      halo_seg<K>(line / NH, oz, lz);
      const int row = NO * (ly + NO * lz);
      T v[NH];
      const int32_t b0 = nb[nbi<3>(-1, oy, oz)], b1 = nb[nbi<3>(0, oy, oz)], b2 = nb[nbi<3>(1, oy, oz)];
      if (b0 >= 0) load_run<T, K>(x + (int64_t)b0 * F::NOWN + row + K, v);
      else for (int i = 0; i < K; ++i) v[i] = T(0);
      if (b1 >= 0) load_run<T, 2 * K>(x + (int64_t)b1 * F::NOWN + row, v + K);
      else for (int i = 0; i < 2 * K; ++i) v[K + i] = T(0);
      v[3 * K] = b2 >= 0 ? x[(int64_t)b2 * F::NOWN + row] : T(0);
      if (oy == 0 && oz == 0) store_run<T, NO>(Xown + row, v + K);
      static_for<0, NE>([&](auto e) {
        T m = 0, kk = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bext<K, false>(e, c);
          constexpr double bk = bext<K, true>(e, c);
          if constexpr (bm != 0.0) m += (T)bm * v[c];
          if constexpr (bk != 0.0) kk += (T)bk * v[c];
        });
        T1M[line * NE + e] = m;
        T1K[line * NE + e] = kk;
      });
    }
  }
  __syncwarp();
  if (active) {
    // stage 2: y direction, lines (z, ex); T1 layout [z][y][ex]
    for (int line = lane; line < NH * NE; line += TW) {
      const int z = line / NE, ex = line % NE;
      T vm[NH], vk[NH];
      static_for<0, NH>([&](auto y) {
        vm[y] = T1M[(z * NH + y) * NE + ex];
        vk[y] = T1K[(z * NH + y) * NE + ex];
      });
      static_for<0, NE>([&](auto e) {
        T mm = 0, mk = 0, km = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bext<K, false>(e, c);
          constexpr double bk = bext<K, true>(e, c);
          if constexpr (bm != 0.0) {
            mm += (T)bm * vm[c];
            km += (T)bm * vk[c];
          }
          if constexpr (bk != 0.0) mk += (T)bk * vm[c];
        });
        const int o = (z * NE + e) * NE + ex;
        T2MM[o] = mm;
        T2MK[o] = mk;
        T2KM[o] = km;
      });
    }
  }
  __syncwarp();
  if (active) {
    // stage 3: z direction, lines (ey, ex)
    for (int line = lane; line < NE * NE; line += TW) {
      T p[NH], q[NH];
      static_for<0, NH>([&](auto z) {
        p[z] = sz * T2MM[z * NE * NE + line];
        q[z] = sy * T2MK[z * NE * NE + line] + sx * T2KM[z * NE * NE + line];
      });
      static_for<0, NE>([&](auto e) {
        T acc = 0;
        static_for<0, NH>([&](auto c) {
          constexpr double bm = bext<K, false>(e, c);
          constexpr double bk = bext<K, true>(e, c);
          if constexpr (bk != 0.0) acc += (T)bk * p[c];
          if constexpr (bm != 0.0) acc += (T)bm * q[c];
        });
        Y[e * NE * NE + line] = acc;
      });
    }
  }
  __syncwarp();
  if (!active) return;
  const uint64_t smask = masks[team];
  // combine the extended rows: row 2K stands for the lower neighbour's cell
  for (int n = lane; n < F::NOWN; n += TW) {
    if (!((smask >> n) & 1ull)) continue;
    const int i0 = n % NO, i1 = (n / NO) % NO, i2 = n / (NO * NO);
    T y = 0;
    const int nbx = i0 == 0 ? 2 : 1, nby = i1 == 0 ? 2 : 1, nbz = i2 == 0 ? 2 : 1;
    for (int bz = 0; bz < nbz; ++bz)
      for (int by = 0; by < nby; ++by)
        for (int bx = 0; bx < nbx; ++bx) {
          const int ex = bx ? 2 * K : i0, ey = by ? 2 * K : i1, ez = bz ? 2 * K : i2;
          y += coefs[bx | (by << 1) | (bz << 2)] * Y[(ez * NE + ey) * NE + ex];
        }
    const int64_t slot = g * F::NOWN + n;
    if constexpr (MODE == 0) {
      out[slot] = y;
    } else {
      const T xv = Xown[n];
      const T xp = xprev ? xprev[slot] : T(0);
      out[slot] = xv + c1 * (xv - xp) + c2 * dinv[slot] * (gvec[slot] - y);
    }
  }
}

// --------------------------------------------- smoothing kernel, 2x2x2 bricks
// Eight uniform sibling groups at positions p + {0,1}^3 (one coefficient)
// form a brick of (4K)^3 stored nodes whose halo is (5K+1)^3: the halo rows
// per stored node drop by about 2x against single groups.  A 128-thread
// team handles one brick with the same three contractions; the rows of the
// 1-D matrices cover the brick's four cells per direction plus the lower
// neighbour's cell.
template <int K, bool STIFF>
__host__ __device__ constexpr double bbrick(int r, int c) {
  const int p = c - K;
  double v = 0.0;
  for (int cell = -1; cell < 4; ++cell) {
    const int lo = K * cell;
    if (r >= lo && r <= lo + K && p >= lo && p <= lo + K) v += elem1<K, STIFF>(r - lo, p - lo);
  }
  return v;
}

template <int K>
struct BrickG {
  static constexpr int NO = 2 * K, OB = 4 * K, HB = 5 * K + 1;
  static constexpr int NOWN = NO * NO * NO;
  static constexpr int TB = K == 2 ? 128 : 64;  // threads per brick (= block)
  static constexpr int L3 = OB * OB;            // last-stage lines
  static constexpr int R = TB / L3 > 0 ? TB / L3 : 1;
  static constexpr int OPT = (OB + R - 1) / R;
};

template <typename T, int K>
struct BrickSmem {
  using B = BrickG<K>;
  static constexpr int T1 = B::HB * B::HB * B::OB;
  static constexpr int ZS = B::OB * B::OB + (B::OB == 8 ? 8 : 4);  // padded z stride of the stage-2 arrays
  static constexpr int T2 = B::HB * ZS;
  static constexpr int XO = B::OB * B::OB * B::OB;
  static constexpr size_t bytes() { return (size_t)(2 * T1 + 3 * T2 + XO) * sizeof(T) + 64 * 4 + 8 * 8 + 16; }
};

// halo index h in [0, 5K] -> group index (-1..2) along the direction and stored index
template <int K>
__device__ __forceinline__ void brick_seg(int h, int& gidx, int& l) {
  const int p = h - K;
  gidx = p < 0 ? -1 : (p < 2 * K ? 0 : (p < 4 * K ? 1 : 2));
  l = p - 2 * K * gidx;
}

// Member positions (bit bx + 2 by + 4 bz) of brick br: all eight for a full
// brick, those of the table for a partial one (smoothing launches only).
__device__ __forceinline__ unsigned brick_members(const LevelArgs& a, int64_t br) {
  return br < a.n_bricks ? 0xFFu : (unsigned)a.brick_members[br - a.n_bricks];
}

template <typename T, int K, int MODE>
__global__ void __launch_bounds__(BrickG<K>::TB)
level_cheb_brick_kernel(LevelArgs a, const T* __restrict__ x, const T* xprev, const T* __restrict__ gvec, T* out,
                        T c1, T c2) {
  using B = BrickG<K>;
  using S = BrickSmem<T, K>;
  constexpr int NO = B::NO, OB = B::OB, HB = B::HB, TB = B::TB, L3 = B::L3, R = B::R, OPT = B::OPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* T1M = reinterpret_cast<T*>(smem_raw);
  T* T1K = T1M + S::T1;
  T* T2MM = T1K + S::T1;
  T* T2MK = T2MM + S::T2;
  T* T2KM = T2MK + S::T2;
  T* Xown = T2KM + S::T2;
  int32_t* tab = reinterpret_cast<int32_t*>(Xown + S::XO);
  uint64_t* smask = reinterpret_cast<uint64_t*>(tab + 64);
  const int tid = threadIdx.x;
  const int64_t br = blockIdx.x;
  if (tid < 64) tab[tid] = a.bricks[br * 64 + tid];
  __syncthreads();
  // own groups sit at table positions (1..2)^3
  auto own_group = [&](int bx, int by, int bz) { return tab[(bx + 1) + 4 * ((by + 1) + 4 * (bz + 1))]; };
  const unsigned members = brick_members(a, br);
  if (tid < 8) smask[tid] = ((members >> tid) & 1u) ? a.smask[own_group(tid & 1, (tid >> 1) & 1, tid >> 2)] : 0ull;
  const int m0 = __ffs(members) - 1;  // a member: the coefficient is common to all
  const T coef = group_coef<T>(a, own_group(m0 & 1, (m0 >> 1) & 1, m0 >> 2));
  // this thread's outputs: line ol = (i, j), k = part + R * o
  const int ol = tid % L3, part = tid / L3;
  const bool has_out = tid < L3 * R;
  const int oi = ol % OB, oj = ol / OB;
  T pre_xp[OPT], pre_g[OPT];
  int64_t slots[OPT];
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    const int kk = part + R * o;
    slots[o] = -1;
    pre_xp[o] = pre_g[o] = T(0);
    if (has_out && kk < OB && ((members >> ((oi / NO) + 2 * ((oj / NO) + 2 * (kk / NO)))) & 1u)) {
      const int32_t gid = own_group(oi / NO, oj / NO, kk / NO);
      slots[o] = (int64_t)gid * B::NOWN + (oi % NO) + NO * ((oj % NO) + NO * (kk % NO));
      if constexpr (MODE == 1) {
        pre_g[o] = gvec[slots[o]];
        if (xprev) pre_xp[o] = xprev[slots[o]];
      }
    }
  }
  // stage 1: halo rows along x (four segments: groups -1, 0, 1, 2)
  for (int line = tid; line < HB * HB; line += TB) {
    int gy, ly, gz, lz;
    brick_seg<K>(line % HB, gy, ly);
    brick_seg<K>(line / HB, gz, lz);
    const int row = NO * (ly + NO * lz);
    const int tb = 4 * ((gy + 1) + 4 * (gz + 1));
    T v[HB];
    const int32_t b0 = tab[tb + 0], b1 = tab[tb + 1], b2 = tab[tb + 2], b3 = tab[tb + 3];
    if (b0 >= 0) load_run<T, K>(x + (int64_t)b0 * B::NOWN + row + K, v);
    else for (int i = 0; i < K; ++i) v[i] = T(0);
    if (b1 >= 0) load_run<T, 2 * K>(x + (int64_t)b1 * B::NOWN + row, v + K);
    else for (int i = 0; i < 2 * K; ++i) v[K + i] = T(0);
    if (b2 >= 0) load_run<T, 2 * K>(x + (int64_t)b2 * B::NOWN + row, v + 3 * K);
    else for (int i = 0; i < 2 * K; ++i) v[3 * K + i] = T(0);
    v[5 * K] = b3 >= 0 ? x[(int64_t)b3 * B::NOWN + row] : T(0);
    if (gy >= 0 && gy <= 1 && gz >= 0 && gz <= 1) {
      const int by = gy * NO + ly, bz = gz * NO + lz;
      store_run<T, OB>(Xown + OB * (by + OB * bz), v + K);
    }
    T m[OB], k[OB];
    static_for<0, OB>([&](auto r) {
      T sm = 0, sk = 0;
      static_for<0, HB>([&](auto c) {
        constexpr double bm = bbrick<K, false>(r, c);
        constexpr double bk = bbrick<K, true>(r, c);
        if constexpr (bm != 0.0) sm += (T)bm * v[c];
        if constexpr (bk != 0.0) sk += (T)bk * v[c];
      });
      m[r] = sm;
      k[r] = sk;
    });
    store_run<T, 4>(T1M + line * OB, m);
    store_run<T, 4>(T1K + line * OB, k);
    if constexpr (OB == 8) {
      store_run<T, 4>(T1M + line * OB + 4, m + 4);
      store_run<T, 4>(T1K + line * OB + 4, k + 4);
    }
  }
  __syncthreads();
  // stage 2: y direction, lines (z, i)
  for (int line = tid; line < HB * OB; line += TB) {
    const int z = line / OB, i = line % OB;
    T vm[HB], vk[HB];
    static_for<0, HB>([&](auto y) {
      vm[y] = T1M[(z * HB + y) * OB + i];
      vk[y] = T1K[(z * HB + y) * OB + i];
    });
    static_for<0, OB>([&](auto j) {
      T mm = 0, mk = 0, km = 0;
      static_for<0, HB>([&](auto c) {
        constexpr double bm = bbrick<K, false>(j, c);
        constexpr double bk = bbrick<K, true>(j, c);
        if constexpr (bm != 0.0) {
          mm += (T)bm * vm[c];
          km += (T)bm * vk[c];
        }
        if constexpr (bk != 0.0) mk += (T)bk * vm[c];
      });
      const int o = z * S::ZS + j * OB + i;
      T2MM[o] = mm;
      T2MK[o] = mk;
      T2KM[o] = km;
    });
  }
  __syncthreads();
  // stage 3: z direction and the update
  if (!has_out) return;
  const T sx = level_scale<T>(a, 0), sy = level_scale<T>(a, 1), sz = level_scale<T>(a, 2);
  T p[HB], q[HB];
  static_for<0, HB>([&](auto z) {
    p[z] = sz * T2MM[z * S::ZS + ol];
    q[z] = sy * T2MK[z * S::ZS + ol] + sx * T2KM[z * S::ZS + ol];
  });
  // The diagonal of the merged brick matrices depends on the index only
  // through its parity (vertex or interior node of a cell), and all outputs
  // of this thread share one parity pattern, so one reciprocal serves them.
  T c2d = T(0);
  if constexpr (MODE == 1) {
    const T md0 = (T)bbrick<K, false>(0, K), kd0 = (T)bbrick<K, true>(0, K);
    const T md1 = (T)bbrick<K, false>(1, K + 1), kd1 = (T)bbrick<K, true>(1, K + 1);
    const T mdx = (oi & 1) ? md1 : md0, kdx = (oi & 1) ? kd1 : kd0;
    const T mdy = (oj & 1) ? md1 : md0, kdy = (oj & 1) ? kd1 : kd0;
    const T mdz = (part & 1) ? md1 : md0, kdz = (part & 1) ? kd1 : kd0;
    c2d = c2 / (coef * (sx * kdx * mdy * mdz + sy * mdx * kdy * mdz + sz * mdx * mdy * kdz));
  }
  static_assert(R % 2 == 0 || OPT == 1, "outputs of a thread must share the parity of k");
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    const int kk = part + R * o;
    if (kk >= OB) break;
    T y = 0;
    static_for<0, OB>([&](auto r) {
      if (kk == r) {
        static_for<0, HB>([&](auto c) {
          constexpr double bm = bbrick<K, false>(r, c);
          constexpr double bk = bbrick<K, true>(r, c);
          if constexpr (bk != 0.0) y += (T)bk * p[c];
          if constexpr (bm != 0.0) y += (T)bm * q[c];
        });
      }
    });
    const int gsel = (oi / NO) + 2 * ((oj / NO) + 2 * (kk / NO));
    const int node = (oi % NO) + NO * ((oj % NO) + NO * (kk % NO));
    if (!((smask[gsel] >> node) & 1ull)) continue;
    y *= coef;
    if constexpr (MODE == 0) {
      out[slots[o]] = y;
    } else {
      const T xv = Xown[oi + OB * (oj + OB * kk)];
      out[slots[o]] = xv + c1 * (xv - pre_xp[o]) + c2d * (pre_g[o] - y);
    }
  }
}

// FP32 brick kernel with packed two-wide FMAs (fma.rn.f32x2): stage 1 forms
// the mass and stiffness rows of a halo line as one pair, stage 2 pairs the
// two stage-1 results and stores the two stage-3 operands (p, q) as a pair,
// stage 3 contracts (bk, bm) against (p, q).  Per component the arithmetic is
// that of the scalar kernel; the shared arrays hold float2 and are padded so
// that consecutive z planes fall on opposite halves of the banks.
template <int K>
struct Brick2S {
  using B = BrickG<K>;
  static constexpr int S1 = B::OB + 1;                          // stage-1 row stride (float2)
  static constexpr int PZ1 = ((B::HB * S1 + 7) / 16) * 16 + 8;  // stage-1 z-plane stride, = 8 (mod 16)
  static constexpr int T1 = B::HB * PZ1;
  static constexpr int ZS = B::OB * B::OB + 8;                  // stage-2 z-plane stride, = 8 (mod 16)
  static constexpr int T2 = B::HB * ZS;
  static constexpr int XO = B::OB * B::OB * B::OB;
  static constexpr size_t bytes() { return (size_t)(T1 + T2) * sizeof(float2) + XO * sizeof(float) + 64 * 4 + 8 * 8 + 16; }
  // threads per brick (64 was measured slower: fewer warps to hide latency)
  static constexpr int TB = 128;
  static constexpr int R = TB / B::L3 > 0 ? TB / B::L3 : 1;
  static constexpr int OPT = (B::OB + R - 1) / R;
};

template <int K>
__host__ __device__ constexpr double ebrick(int f, int c) {
  const int cell = f / (2 * K) > 1 ? 1 : f / (2 * K);
  const int r = f - 2 * K * cell, j = c - K * cell;
  return (j >= 0 && j <= K) ? embed1<K>(r, j) : 0.0;
}

// MODE 2 (residual + restriction, levels >= 2 without refinement-edge nodes):
// r = g - A x on the brick's own nodes, then g_{l-1} += R r with R = P^T on
// the parent group's (2K+1)^3 coarse nodes; `out` is g_{l-1}.  Coarse nodes
// inside the parent group receive only this brick's fine nodes; those on its
// faces are shared with neighbouring bricks (atomics).
template <int K, int MODE>
__global__ void __launch_bounds__(Brick2S<K>::TB)
level_cheb_brick_f2_kernel(LevelArgs a, const float* __restrict__ x, const float* xprev,
                           const float* __restrict__ gvec, float* out, float c1, float c2) {
  using B = BrickG<K>;
  using S = Brick2S<K>;
  constexpr int NO = B::NO, OB = B::OB, HB = B::HB, TB = S::TB, L3 = B::L3, R = S::R, OPT = S::OPT;
  static_assert(TB >= 64, "the brick table is loaded by 64 threads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* T1 = reinterpret_cast<float2*>(smem_raw);
  float2* T2 = T1 + S::T1;
  float* Xown = reinterpret_cast<float*>(T2 + S::T2);
  int32_t* tab = reinterpret_cast<int32_t*>(Xown + S::XO);
  uint64_t* smask = reinterpret_cast<uint64_t*>(tab + 64);
  const int tid = threadIdx.x;
  const int64_t br = blockIdx.x;
  if (tid < 64) tab[tid] = a.bricks[br * 64 + tid];
  // mode 2: the parent group's coarse neighbour row, needed only at the end
  int32_t cnb_pre = 0;
  if constexpr (MODE == 2) {
    if (tid < 27) cnb_pre = a.brick_cnb[br * 27 + tid];
  }
  __syncthreads();
  auto own_group = [&](int bx, int by, int bz) { return tab[(bx + 1) + 4 * ((by + 1) + 4 * (bz + 1))]; };
  const unsigned members = MODE == 2 ? 0xFFu : brick_members(a, br);
  if (tid < 8) smask[tid] = ((members >> tid) & 1u) ? a.smask[own_group(tid & 1, (tid >> 1) & 1, tid >> 2)] : 0ull;
  const int m0 = __ffs(members) - 1;  // a member: the coefficient is common to all
  const float coef = a.coeff32[own_group(m0 & 1, (m0 >> 1) & 1, m0 >> 2)];
  const int ol = tid % L3, part = tid / L3;
  const bool has_out = tid < L3 * R;
  const int oi = ol % OB, oj = ol / OB;
  float pre_xp[OPT], pre_g[OPT];
  int64_t slots[OPT];
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    const int kk = part + R * o;
    slots[o] = -1;
    pre_xp[o] = pre_g[o] = 0.f;
    if (has_out && kk < OB && ((members >> ((oi / NO) + 2 * ((oj / NO) + 2 * (kk / NO)))) & 1u)) {
      const int32_t gid = own_group(oi / NO, oj / NO, kk / NO);
      slots[o] = (int64_t)gid * B::NOWN + (oi % NO) + NO * ((oj % NO) + NO * (kk % NO));
      if constexpr (MODE >= 1) pre_g[o] = gvec[slots[o]];
      if constexpr (MODE == 1) {
        if (xprev) pre_xp[o] = xprev[slots[o]];
      }
    }
  }
  // stage 1: halo rows along x -> (mass, stiffness) pairs
  for (int line = tid; line < HB * HB; line += TB) {
    const int hy = line % HB, hz = line / HB;
    int gy, ly, gz, lz;
    brick_seg<K>(hy, gy, ly);
    brick_seg<K>(hz, gz, lz);
    const int row = NO * (ly + NO * lz);
    const int tb = 4 * ((gy + 1) + 4 * (gz + 1));
    float v[HB];
    const int32_t b0 = tab[tb + 0], b1 = tab[tb + 1], b2 = tab[tb + 2], b3 = tab[tb + 3];
    if (b0 >= 0) load_run<float, K>(x + (int64_t)b0 * B::NOWN + row + K, v);
    else for (int i = 0; i < K; ++i) v[i] = 0.f;
    if (b1 >= 0) load_run<float, 2 * K>(x + (int64_t)b1 * B::NOWN + row, v + K);
    else for (int i = 0; i < 2 * K; ++i) v[K + i] = 0.f;
    if (b2 >= 0) load_run<float, 2 * K>(x + (int64_t)b2 * B::NOWN + row, v + 3 * K);
    else for (int i = 0; i < 2 * K; ++i) v[3 * K + i] = 0.f;
    v[5 * K] = b3 >= 0 ? x[(int64_t)b3 * B::NOWN + row] : 0.f;
    if (gy >= 0 && gy <= 1 && gz >= 0 && gz <= 1) {
      const int by = gy * NO + ly, bz = gz * NO + lz;
      store_run<float, OB>(Xown + OB * (by + OB * bz), v + K);
    }
    float2 vv[HB];
    static_for<0, HB>([&](auto c) { vv[c] = make_float2(v[c], v[c]); });
    float2* dst = T1 + hz * S::PZ1 + hy * S::S1;
    static_for<0, OB>([&](auto r) {
      float2 acc = make_float2(0.f, 0.f);
      static_for<0, HB>([&](auto c) {
        constexpr double bm = bbrick<K, false>(r, c);
        constexpr double bk = bbrick<K, true>(r, c);
        if constexpr (bm != 0.0 || bk != 0.0) acc = __ffma2_rn(make_float2((float)bm, (float)bk), vv[c], acc);
      });
      dst[r] = acc;
    });
  }
  __syncthreads();
  const float sx = a.scale32[0], sy = a.scale32[1], sz = a.scale32[2];
  // stage 2: y direction, lines (z, i); stores p = sz MM and q = sy MK + sx KM
  for (int line = tid; line < HB * OB; line += TB) {
    const int z = line / OB, i = line % OB;
    float2 w[HB];
    static_for<0, HB>([&](auto y) { w[y] = T1[z * S::PZ1 + y * S::S1 + i]; });
    static_for<0, OB>([&](auto j) {
      float2 mmkm = make_float2(0.f, 0.f);
      float mk = 0.f;
      static_for<0, HB>([&](auto c) {
        constexpr double bm = bbrick<K, false>(j, c);
        constexpr double bk = bbrick<K, true>(j, c);
        if constexpr (bm != 0.0) mmkm = __ffma2_rn(make_float2((float)bm, (float)bm), w[c], mmkm);
        if constexpr (bk != 0.0) mk += (float)bk * w[c].x;
      });
      T2[z * S::ZS + j * OB + i] = make_float2(sz * mmkm.x, sy * mk + sx * mmkm.y);
    });
  }
  __syncthreads();
  // stage 3: z direction and the update
  if constexpr (MODE == 2) {
    // residual on the own nodes into shared memory (T1 is free now)
    float* Rs = reinterpret_cast<float*>(T1);
    if (has_out) {
      float2 pq[HB];
      static_for<0, HB>([&](auto z) { pq[z] = T2[z * S::ZS + ol]; });
      own_rows<OB, R>(part, [&](auto o, auto r) {
        float2 acc = make_float2(0.f, 0.f);
        static_for<0, HB>([&](auto c) {
          constexpr double bm = bbrick<K, false>(r, c);
          constexpr double bk = bbrick<K, true>(r, c);
          if constexpr (bm != 0.0 || bk != 0.0) acc = __ffma2_rn(make_float2((float)bk, (float)bm), pq[c], acc);
        });
        Rs[oi + OB * (oj + OB * (int)r)] = pre_g[o] - coef * (acc.x + acc.y);
      });
    }
    __syncthreads();
    constexpr int NC = 2 * K + 1;  // coarse nodes per direction of the parent group
    float* Q1 = Rs + OB * OB * OB;  // [fz][fy][cx]
    float* Q2 = Q1 + OB * OB * NC;  // [fz][cy][cx]
    int32_t* cnb = reinterpret_cast<int32_t*>(Q2 + OB * NC * NC);
    if (tid < 27) cnb[tid] = cnb_pre;
    for (int line = tid; line < OB * OB; line += TB) {  // x: (fy, fz)
      float v[OB];
      static_for<0, OB>([&](auto f) { v[f] = Rs[f + OB * line]; });
      static_for<0, NC>([&](auto c) {
        float t = 0.f;
        static_for<0, OB>([&](auto f) {
          constexpr double e = ebrick<K>(f, c);
          if constexpr (e != 0.0) t += (float)e * v[f];
        });
        Q1[line * NC + c] = t;
      });
    }
    __syncthreads();
    for (int line = tid; line < OB * NC; line += TB) {  // y: (fz, cx)
      const int fz = line / NC, cx = line % NC;
      float v[OB];
      static_for<0, OB>([&](auto f) { v[f] = Q1[(fz * OB + f) * NC + cx]; });
      static_for<0, NC>([&](auto c) {
        float t = 0.f;
        static_for<0, OB>([&](auto f) {
          constexpr double e = ebrick<K>(f, c);
          if constexpr (e != 0.0) t += (float)e * v[f];
        });
        Q2[(fz * NC + c) * NC + cx] = t;
      });
    }
    __syncthreads();
    for (int line = tid; line < NC * NC; line += TB) {  // z: (cx, cy), then add into g_{l-1}
      const int cx = line % NC, cy = line / NC;
      float v[OB];
      static_for<0, OB>([&](auto f) { v[f] = Q2[(f * NC + cy) * NC + cx]; });
      static_for<0, NC>([&](auto cz) {
        float t = 0.f;
        static_for<0, OB>([&](auto f) {
          constexpr double e = ebrick<K>(f, cz);
          if constexpr (e != 0.0) t += (float)e * v[f];
        });
        const int ox = cx == 2 * K, oy = cy == 2 * K, oz = (int)cz == 2 * K;
        const int32_t blk = cnb[(ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1))];
        if (blk >= 0) {
          float* dst = out + (int64_t)blk * NO * NO * NO + (cx - 2 * K * ox) +
                       NO * ((cy - 2 * K * oy) + NO * ((int)cz - 2 * K * oz));
          const bool inner = cx > 0 && cx < 2 * K && cy > 0 && cy < 2 * K && (int)cz > 0 && (int)cz < 2 * K;
          if (inner || a.deterministic) *dst += t;  // deterministic: this launch's bricks share no node
          else atomicAdd(dst, t);
        }
      });
    }
    return;
  }
  if (!has_out) return;
  float2 pq[HB];
  static_for<0, HB>([&](auto z) { pq[z] = T2[z * S::ZS + ol]; });
  // the diagonal depends on the node only through index parities: one
  // reciprocal per parity of k
  float c2d[2] = {0.f, 0.f};
  if constexpr (MODE == 1) {
    const float md0 = (float)bbrick<K, false>(0, K), kd0 = (float)bbrick<K, true>(0, K);
    const float md1 = (float)bbrick<K, false>(1, K + 1), kd1 = (float)bbrick<K, true>(1, K + 1);
    const float mdx = (oi & 1) ? md1 : md0, kdx = (oi & 1) ? kd1 : kd0;
    const float mdy = (oj & 1) ? md1 : md0, kdy = (oj & 1) ? kd1 : kd0;
#pragma unroll
    for (int pz = 0; pz < 2; ++pz) {
      if (R % 2 == 0 && pz != (part & 1)) continue;
      const float mdz = pz ? md1 : md0, kdz = pz ? kd1 : kd0;
      c2d[pz] = c2 / (coef * (sx * kdx * mdy * mdz + sy * mdx * kdy * mdz + sz * mdx * mdy * kdz));
    }
  }
  const int gsel_xy = (oi / NO) + 2 * (oj / NO), node_xy = (oi % NO) + NO * (oj % NO);
  own_rows<OB, R>(part, [&](auto o, auto r) {
    float2 acc = make_float2(0.f, 0.f);
    static_for<0, HB>([&](auto c) {
      constexpr double bm = bbrick<K, false>(r, c);
      constexpr double bk = bbrick<K, true>(r, c);
      if constexpr (bm != 0.0 || bk != 0.0) acc = __ffma2_rn(make_float2((float)bk, (float)bm), pq[c], acc);
    });
    float y = acc.x + acc.y;
    constexpr int gz = r / NO, nz = r % NO;
    const int node = node_xy + NO * NO * nz;
    if (!((smask[gsel_xy + 4 * gz] >> node) & 1ull)) return;
    y *= coef;
    if constexpr (MODE == 0) {
      out[slots[o]] = y;
    } else {
      const float xv = Xown[oi + OB * (oj + OB * (int)r)];
      out[slots[o]] = xv + c1 * (xv - pre_xp[o]) + c2d[r & 1] * (pre_g[o] - y);
    }
  });
}

// ------------------- FP64 brick smoother, exact split-integer evaluation
// For cubic cells (s_x = s_y = s_z = s) the merged brick matrices are the
// integer matrices ibrick over the element denominators, so the operator of
// a brick is a s / (DM^2 DK) times an integer Kronecker sum, evaluated as
// the leaf operator's integer kernels do (int_split.cuh): each thread loads
// one halo line in FP64, the block takes the brick's largest exponent, the
// thread splits its line exactly into P1, P2 (int32) and r (FP32) in
// registers, the three contractions run per component, and the results are
// recombined in integers and converted to FP64 exactly (integer operations
// only).  The Chebyshev update stays in FP64: four operations per node, with
// its diagonal factors and scale formed once per brick.  This takes the FP64
// smoother's contractions off the FP64 pipe, a small fraction of this GPU's
// int32/FP32 throughput.  Layout, halo and outputs are those of level_cheb_brick_kernel;
// MODE 2 is the residual + restriction pass of level_cheb_brick_f2_kernel
// (full bricks, levels >= 2 without refinement-edge nodes), with the
// restriction in FP64.
template <int K, bool STIFF>
__host__ __device__ constexpr int ibrick(int r, int c) {
  const int p = c - K;
  int v = 0;
  for (int cell = -1; cell < 4; ++cell) {
    const int lo = K * cell;
    if (r >= lo && r <= lo + K && p >= lo && p <= lo + K) v += ielem1<K, STIFF>(r - lo, p - lo);
  }
  return v;
}

// the integer brick matrices are the FP64 ones times the element denominators
template <int K>
constexpr bool ibrick_matches() {
  for (int r = 0; r < 4 * K; ++r)
    for (int c = 0; c <= 5 * K; ++c) {
      const double dm = bbrick<K, false>(r, c) * IntElem<K>::DM - ibrick<K, false>(r, c);
      const double dk = bbrick<K, true>(r, c) * IntElem<K>::DK - ibrick<K, true>(r, c);
      if (dm > 1e-12 || dm < -1e-12 || dk > 1e-12 || dk < -1e-12) return false;
    }
  return true;
}
static_assert(ibrick_matches<1>() && ibrick_matches<2>(), "integer brick matrices");

// largest sum of |entries| over the rows of an integer brick matrix
template <int K, bool STIFF>
constexpr long long ibrick_rowsum() {
  long long best = 0;
  for (int r = 0; r < 4 * K; ++r) {
    long long t = 0;
    for (int c = 0; c <= 5 * K; ++c) t += ibrick<K, STIFF>(r, c) < 0 ? -ibrick<K, STIFF>(r, c) : ibrick<K, STIFF>(r, c);
    best = t > best ? t : best;
  }
  return best;
}

template <int K>
struct BrickI {
  using B = BrickG<K>;
  static constexpr int HB = B::HB, OB = B::OB;
  static constexpr int T1 = HB * HB * OB;     // stage-1 outputs per matrix and component
  static constexpr int ZS = OB * OB + (OB == 8 ? 8 : 4);  // padded z stride of the stage-2 arrays
  static constexpr int T2 = HB * ZS;
  // bound of the integer Kronecker sum per unit input (38,400 for Q2)
  static constexpr long long BOUND =
      3 * ibrick_rowsum<K, false>() * ibrick_rowsum<K, false>() * ibrick_rowsum<K, true>();
  static constexpr int KR = int_recombination_bits_bound(BOUND);
  // region 1: the stage-1 outputs (M, K) of the three components; region 2:
  // the stage-2 outputs (MM and MK + KM: the scales are equal) of the three
  // components.  The halo never goes to shared memory: each thread loads,
  // splits and contracts one halo line in registers.
  static constexpr size_t R1 = (size_t)6 * T1 * 4;
  static constexpr size_t R2 = ((size_t)6 * T2 * 4 + 15) / 16 * 16;
  // after the arrays: brick table, S masks, largest exponent (16 bytes), the
  // Chebyshev factor c2 / diagonal per parity class of (i, j, k) and the
  // brick's scale a s / (DM^2 DK)
  static constexpr size_t bytes() { return R1 + R2 + 64 * 4 + 8 * 8 + 16 + 9 * 8; }
  static_assert(R1 % 16 == 0 && (4 * T2 * 4) % 16 == 0, "16-byte aligned arrays");
  static_assert(HB * HB <= B::TB, "one halo line per thread");
  // blocks per SM the registers are sized for (shared memory admits five Q2 blocks)
  static constexpr int MIN_BLOCKS = K == 2 ? 5 : 8;
};

// four 4-byte values to 16-byte aligned shared memory
template <typename T>
__device__ __forceinline__ void st4(T* p, const T* v) {
  if constexpr (std::is_same<T, int>::value) *reinterpret_cast<int4*>(p) = make_int4(v[0], v[1], v[2], v[3]);
  else *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

template <int K, int MODE>
__global__ void __launch_bounds__(BrickG<K>::TB, BrickI<K>::MIN_BLOCKS)
level_cheb_brick_int_kernel(LevelArgs a, const double* __restrict__ x, const double* xprev,
                            const double* __restrict__ gvec, double* out, double c1, double c2) {
  using B = BrickG<K>;
  using S = BrickI<K>;
  constexpr int NO = B::NO, OB = B::OB, HB = B::HB, TB = B::TB, L3 = B::L3, R = B::R, OPT = B::OPT;
  constexpr int T1 = S::T1, T2 = S::T2, ZS = S::ZS, KR = S::KR;
  static_assert(S::BOUND * 32768LL < 2147483648LL, "integer Kronecker sum exceeds int32");
  static_assert(KR >= 5 && int_recombination_fits_bound(S::BOUND, KR), "integer recombination exceeds 2^51");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* T1i = reinterpret_cast<int*>(smem_raw);          // P1 (M, K), P2 (M, K)
  float* T1f = reinterpret_cast<float*>(T1i + 4 * T1);  // r (M, K)
  unsigned char* r2 = smem_raw + S::R1;
  int* T2i = reinterpret_cast<int*>(r2);                // P1 (MM, MK + KM), P2 (MM, MK + KM)
  float* T2f = reinterpret_cast<float*>(T2i + 4 * T2);  // r (MM, MK + KM)
  int32_t* tab = reinterpret_cast<int32_t*>(r2 + S::R2);
  uint64_t* smask = reinterpret_cast<uint64_t*>(tab + 64);
  int* emax = reinterpret_cast<int*>(smask + 8);
  double* c2cls = reinterpret_cast<double*>(smask + 10);
  double* sbase = c2cls + 8;
  const int tid = threadIdx.x;
  const int64_t br = blockIdx.x;
  if (tid < 64) tab[tid] = a.bricks[br * 64 + tid];
  if (tid == 0) *emax = 1;
  // mode 2: the parent group's coarse neighbour row, needed only at the end
  int32_t cnb_pre = 0;
  if constexpr (MODE == 2) {
    if (tid < 27) cnb_pre = a.brick_cnb[br * 27 + tid];
  }
  __syncthreads();
  auto own_group = [&](int bx, int by, int bz) { return tab[(bx + 1) + 4 * ((by + 1) + 4 * (bz + 1))]; };
  const unsigned members = MODE == 2 ? 0xFFu : brick_members(a, br);
  if (tid < 8) smask[tid] = ((members >> tid) & 1u) ? a.smask[own_group(tid & 1, (tid >> 1) & 1, tid >> 2)] : 0ull;
  const int m0 = __ffs(members) - 1;  // a member: the coefficient is common to all
  constexpr double DEN = (double)IntElem<K>::DM * IntElem<K>::DM * IntElem<K>::DK;
  if (tid < 9) {
    // per brick, not per thread: the divisions would load the FP64 pipe.  The
    // diagonal of the merged brick matrices depends on a node only through
    // the parities of (i, j, k): class tid = px + 2 py + 4 pz.
    const double coef = a.coeff[own_group(m0 & 1, (m0 >> 1) & 1, m0 >> 2)];
    const double s = a.scale[0];
    if (tid == 8) {
      *sbase = coef * s / DEN;
    } else if constexpr (MODE == 1) {
      const double md0 = bbrick<K, false>(0, K), kd0 = bbrick<K, true>(0, K);
      const double md1 = bbrick<K, false>(1, K + 1), kd1 = bbrick<K, true>(1, K + 1);
      const double mdx = (tid & 1) ? md1 : md0, kdx = (tid & 1) ? kd1 : kd0;
      const double mdy = (tid & 2) ? md1 : md0, kdy = (tid & 2) ? kd1 : kd0;
      const double mdz = (tid & 4) ? md1 : md0, kdz = (tid & 4) ? kd1 : kd0;
      c2cls[tid] = c2 / (coef * (s * kdx * mdy * mdz + s * mdx * kdy * mdz + s * mdx * mdy * kdz));
    }
  }
  // this thread's outputs: line ol = (i, j), k = part + R * o
  const int ol = tid % L3, part = tid / L3;
  const bool has_out = tid < L3 * R;
  const int oi = ol % OB, oj = ol / OB;
  double pre_xp[OPT], pre_g[OPT], xv[OPT];
  int64_t slots[OPT];
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    const int kk = part + R * o;
    slots[o] = -1;
    pre_xp[o] = pre_g[o] = xv[o] = 0.0;
    if (has_out && kk < OB && ((members >> ((oi / NO) + 2 * ((oj / NO) + 2 * (kk / NO)))) & 1u)) {
      const int32_t gid = own_group(oi / NO, oj / NO, kk / NO);
      slots[o] = (int64_t)gid * B::NOWN + (oi % NO) + NO * ((oj % NO) + NO * (kk % NO));
      if constexpr (MODE >= 1) pre_g[o] = gvec[slots[o]];
      if constexpr (MODE == 1) {
        xv[o] = x[slots[o]];
        if (xprev) pre_xp[o] = xprev[slots[o]];
      }
    }
  }
  // this thread's halo line in FP64 (four segments: groups -1, 0, 1, 2) and
  // the brick's largest biased exponent
  const int line = tid;
  const bool has_line = line < HB * HB;
  double v[HB];
  int ex = 0;
  if (has_line) {
    int gy, ly, gz, lz;
    brick_seg<K>(line % HB, gy, ly);
    brick_seg<K>(line / HB, gz, lz);
    const int row = NO * (ly + NO * lz);
    const int tb = 4 * ((gy + 1) + 4 * (gz + 1));
    const int32_t b0 = tab[tb + 0], b1 = tab[tb + 1], b2 = tab[tb + 2], b3 = tab[tb + 3];
    if (b0 >= 0) load_run<double, K>(x + (int64_t)b0 * B::NOWN + row + K, v);
    else for (int i = 0; i < K; ++i) v[i] = 0.0;
    if (b1 >= 0) load_run<double, 2 * K>(x + (int64_t)b1 * B::NOWN + row, v + K);
    else for (int i = 0; i < 2 * K; ++i) v[K + i] = 0.0;
    if (b2 >= 0) load_run<double, 2 * K>(x + (int64_t)b2 * B::NOWN + row, v + 3 * K);
    else for (int i = 0; i < 2 * K; ++i) v[3 * K + i] = 0.0;
    v[5 * K] = b3 >= 0 ? x[(int64_t)b3 * B::NOWN + row] : 0.0;
    static_for<0, HB>([&](auto c) {
      const int e = (int)((__double_as_longlong(v[c]) >> 52) & 0x7FF);
      ex = e > ex ? e : ex;
    });
  }
  ex = __reduce_max_sync(0xffffffffu, ex);
  if ((tid & 31) == 0) atomicMax(emax, ex);
  __syncthreads();
  // exact split against q = 2^(emax - 1037): |x| < 2^15 q; a NaN or Inf in
  // the halo makes the brick's outputs NaN
  const int em = *emax;
  // stage 1: the line's split parts, x direction (M and K rows), per component
  if (has_line) {
    const int eq = em == 0x7FF ? 1010 : em - 1037;
    auto xrows = [&](const auto* v, auto* oM, auto* oK) {
      using T = std::remove_const_t<std::remove_reference_t<decltype(v[0])>>;
      T m[OB], k[OB];
      static_for<0, OB>([&](auto r) {
        T sm = 0, sk = 0;
        static_for<0, HB>([&](auto c) {
          constexpr int bm = ibrick<K, false>(r, c), bk = ibrick<K, true>(r, c);
          if constexpr (bm != 0) sm += (T)bm * v[c];
          if constexpr (bk != 0) sk += (T)bk * v[c];
        });
        m[r] = sm;
        k[r] = sk;
      });
      static_for<0, OB / 4>([&](auto h) {
        st4<T>(oM + line * OB + 4 * h, m + 4 * h);
        st4<T>(oK + line * OB + 4 * h, k + 4 * h);
      });
    };
    int v1[HB], v2[HB];
    float v3[HB];
    static_for<0, HB>([&](auto c) { split_exact(v[c], eq, v1[c], v2[c], v3[c]); });
    xrows(v1, T1i, T1i + T1);
    xrows(v2, T1i + 2 * T1, T1i + 3 * T1);
    xrows(v3, T1f, T1f + T1);
  }
  __syncthreads();
  // stage 2: y direction, lines (z, i), per component
  for (int l2 = tid; l2 < HB * OB; l2 += TB) {
    const int z = l2 / OB, i = l2 % OB;
    auto yrows = [&](const auto* iM, const auto* iK, auto* oMM, auto* oQ) {
      using T = std::remove_const_t<std::remove_reference_t<decltype(iM[0])>>;
      T vm[HB], vk[HB];
      static_for<0, HB>([&](auto y) {
        vm[y] = iM[(z * HB + y) * OB + i];
        vk[y] = iK[(z * HB + y) * OB + i];
      });
      static_for<0, OB>([&](auto j) {
        T mm = 0, mk = 0, km = 0;
        static_for<0, HB>([&](auto c) {
          constexpr int bm = ibrick<K, false>(j, c), bk = ibrick<K, true>(j, c);
          if constexpr (bm != 0) {
            mm += (T)bm * vm[c];
            km += (T)bm * vk[c];
          }
          if constexpr (bk != 0) mk += (T)bk * vm[c];
        });
        const int o = z * ZS + j * OB + i;
        oMM[o] = mm;
        oQ[o] = mk + km;
      });
    };
    yrows(T1i, T1i + T1, T2i, T2i + T2);
    yrows(T1i + 2 * T1, T1i + 3 * T1, T2i + 2 * T2, T2i + 3 * T2);
    yrows(T1f, T1f + T1, T2f, T2f + T2);
  }
  __syncthreads();
  // stage 3: z direction per component, then the recombination and the update
  int o1[OPT], o2[OPT];
  float o3[OPT];
  auto zrows = [&](const auto* iMM, const auto* iQ, auto* acc) {
    using T = std::remove_const_t<std::remove_reference_t<decltype(iMM[0])>>;
    T p[HB], q[HB];
    static_for<0, HB>([&](auto z) {
      p[z] = iMM[z * ZS + ol];
      q[z] = iQ[z * ZS + ol];
    });
    own_rows<OB, R>(part, [&](auto o, auto r) {
      T y = 0;
      static_for<0, HB>([&](auto c) {
        constexpr int bm = ibrick<K, false>(r, c), bk = ibrick<K, true>(r, c);
        if constexpr (bk != 0) y += (T)bk * p[c];
        if constexpr (bm != 0) y += (T)bm * q[c];
      });
      acc[o] = y;
    });
  };
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    o1[o] = o2[o] = 0;
    o3[o] = 0.f;
  }
  if (has_out) {
    zrows(T2i, T2i + T2, o1);
    zrows(T2i + 2 * T2, T2i + 3 * T2, o2);
    zrows(T2f, T2f + T2, o3);
  }
  // q 2^-15 2^-KR = 2^(emax - 1023) 2^-(29 + KR); the recombined integer T
  // converts to FP64 exactly with integer operations
  constexpr double LOW = 1.0 / (double)(1LL << (29 + KR));
  const double sc = em == 0x7FF ? __longlong_as_double(0x7FF8000000000000LL)
                                : *sbase * LOW * pow2_normal(em - 1023);
  auto tsum = [&](int o) {
    return i64_to_double_alu(((long long)o1[o] << (15 + KR)) + ((long long)o2[o] << KR) +
                             (long long)f32_fixed_rint<KR>(o3[o]));
  };
  auto result = [&](int o) { return sc * tsum(o); };
  if constexpr (MODE == 2) {
    // residual on the own nodes (region 1 is free after stage 2), then
    // g_{l-1} += R r over the parent group's coarse nodes, in FP64
    double* Rs = reinterpret_cast<double*>(smem_raw);
    if (has_out) {
#pragma unroll
      for (int o = 0; o < OPT; ++o) {
        const int kk = part + R * o;
        if (kk < OB) Rs[oi + OB * (oj + OB * kk)] = pre_g[o] - result(o);
      }
    }
    __syncthreads();
    constexpr int NC = 2 * K + 1;     // coarse nodes per direction of the parent group
    double* Q1 = Rs + OB * OB * OB;   // [fz][fy][cx]
    double* Q2 = Q1 + OB * OB * NC;   // [fz][cy][cx]
    int32_t* cnb = reinterpret_cast<int32_t*>(Q2 + OB * NC * NC);
    static_assert((OB * OB * OB + OB * OB * NC + OB * NC * NC) * 8 + 27 * 4 <= S::R1, "restriction fits region 1");
    if (tid < 27) cnb[tid] = cnb_pre;
    for (int line = tid; line < OB * OB; line += TB) {  // x: (fy, fz)
      double v[OB];
      static_for<0, OB>([&](auto f) { v[f] = Rs[f + OB * line]; });
      static_for<0, NC>([&](auto c) {
        double t = 0.0;
        static_for<0, OB>([&](auto f) {
          constexpr double e = ebrick<K>(f, c);
          if constexpr (e != 0.0) t += e * v[f];
        });
        Q1[line * NC + c] = t;
      });
    }
    __syncthreads();
    for (int line = tid; line < OB * NC; line += TB) {  // y: (fz, cx)
      const int fz = line / NC, cx = line % NC;
      double v[OB];
      static_for<0, OB>([&](auto f) { v[f] = Q1[(fz * OB + f) * NC + cx]; });
      static_for<0, NC>([&](auto c) {
        double t = 0.0;
        static_for<0, OB>([&](auto f) {
          constexpr double e = ebrick<K>(f, c);
          if constexpr (e != 0.0) t += e * v[f];
        });
        Q2[(fz * NC + c) * NC + cx] = t;
      });
    }
    __syncthreads();
    for (int line = tid; line < NC * NC; line += TB) {  // z: (cx, cy), then add into g_{l-1}
      const int cx = line % NC, cy = line / NC;
      double v[OB];
      static_for<0, OB>([&](auto f) { v[f] = Q2[(f * NC + cy) * NC + cx]; });
      static_for<0, NC>([&](auto cz) {
        double t = 0.0;
        static_for<0, OB>([&](auto f) {
          constexpr double e = ebrick<K>(f, cz);
          if constexpr (e != 0.0) t += e * v[f];
        });
        const int ox = cx == 2 * K, oy = cy == 2 * K, oz = (int)cz == 2 * K;
        const int32_t blk = cnb[(ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1))];
        if (blk >= 0) {
          double* dst = out + (int64_t)blk * NO * NO * NO + (cx - 2 * K * ox) +
                        NO * ((cy - 2 * K * oy) + NO * ((int)cz - 2 * K * oz));
          const bool inner = cx > 0 && cx < 2 * K && cy > 0 && cy < 2 * K && (int)cz > 0 && (int)cz < 2 * K;
          if (inner || a.deterministic) *dst += t;  // deterministic: this launch's bricks share no node
          else atomicAdd(dst, t);
        }
      });
    }
    return;
  }
  if (!has_out) return;
  // out = x + c1 (x - x_prev) + c2d g - (c2d sc) T: four FP64 operations per node
  double c2d = 0.0, c2s = 0.0;
  if constexpr (MODE == 1) {
    c2d = c2cls[(oi & 1) + 2 * (oj & 1) + 4 * (part & 1)];
    c2s = c2d * sc;
  }
  static_assert(R % 2 == 0 || OPT == 1, "outputs of a thread must share the parity of k");
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    const int kk = part + R * o;
    if (kk >= OB) break;
    const int gsel = (oi / NO) + 2 * ((oj / NO) + 2 * (kk / NO));
    const int node = (oi % NO) + NO * ((oj % NO) + NO * (kk % NO));
    if (!((smask[gsel] >> node) & 1ull)) continue;
    if constexpr (MODE == 0) {
      out[slots[o]] = result(o);
    } else {
      out[slots[o]] = fma(-c2s, tsum(o), fma(c2d, pre_g[o], fma(c1, xv[o] - pre_xp[o], xv[o])));
    }
  }
}

// FP64 single groups on cubic cells, split-integer contractions: the single-
// group smoother of level_cheb_fast_kernel (one team of TW threads per group,
// the (3K+1)^3 halo, the merged 1-D matrices) with the split-integer scheme of
// level_cheb_brick_int_kernel.  A team takes its group's largest exponent by
// a team-wide max, splits its halo lines in registers and contracts P1, P2
// (int32) and r (FP32); the update is the brick kernel's four FP64
// operations per node.
template <int K, bool STIFF>
__host__ __device__ constexpr int imerged(int r, int c) {
  // integer counterpart of bmerged: rows 0..2K-1, halo columns 0..3K
  const int p = c - K;
  int v = 0;
  for (int cell = 0; cell < 2; ++cell) {
    const int lo = K * cell;
    if (r >= lo && r <= lo + K && p >= lo && p <= lo + K) v += ielem1<K, STIFF>(r - lo, p - lo);
  }
  if (r == 0 && p >= -K && p <= 0) v += ielem1<K, STIFF>(K, p + K);  // the lower neighbour's cell
  return v;
}

template <int K>
constexpr bool imerged_matches() {
  for (int r = 0; r < 2 * K; ++r)
    for (int c = 0; c <= 3 * K; ++c) {
      const double dm = bmerged<K, false>(r, c) * IntElem<K>::DM - imerged<K, false>(r, c);
      const double dk = bmerged<K, true>(r, c) * IntElem<K>::DK - imerged<K, true>(r, c);
      if (dm > 1e-12 || dm < -1e-12 || dk > 1e-12 || dk < -1e-12) return false;
    }
  return true;
}
static_assert(imerged_matches<1>() && imerged_matches<2>(), "integer merged matrices");

template <int K, bool STIFF>
constexpr long long imerged_rowsum() {
  long long best = 0;
  for (int r = 0; r < 2 * K; ++r) {
    long long t = 0;
    for (int c = 0; c <= 3 * K; ++c) t += imerged<K, STIFF>(r, c) < 0 ? -imerged<K, STIFF>(r, c) : imerged<K, STIFF>(r, c);
    best = t > best ? t : best;
  }
  return best;
}

template <int K>
struct SingleI {
  using F = Fast<3, K>;
  static constexpr int NH = F::NH, NO = F::NO, TW = F::TW, TPB = F::TPB;
  static constexpr int L1 = NH * NH;              // stage-1 lines
  static constexpr int LPT = (L1 + TW - 1) / TW;  // stage-1 lines per thread
  static constexpr int T1 = L1 * NO;              // per matrix and component
  static constexpr int T2 = NH * NO * NO;         // per array and component
  static constexpr long long BOUND =
      3 * imerged_rowsum<K, false>() * imerged_rowsum<K, false>() * imerged_rowsum<K, true>();
  static constexpr int KR = int_recombination_bits_bound(BOUND);
  // per team: c2 / diagonal per parity class and the scale (9 doubles), the
  // stage-1 outputs (M, K) and the stage-2 outputs (MM, MK + KM) of the three
  // components
  // (the arrays start 80 bytes into the team's slice, 16-byte aligned)
  static constexpr size_t PER = ((size_t)80 + (size_t)(6 * T1 + 6 * T2) * 4 + 15) / 16 * 16;
  static constexpr size_t bytes() { return (size_t)TPB * PER; }
};

template <int K, int MODE>
__global__ void __launch_bounds__(256, 3)
level_cheb_single_int_kernel(LevelArgs a, const double* __restrict__ x, const double* xprev,
                             const double* __restrict__ gvec, double* out, double c1, double c2) {
  using F = Fast<3, K>;
  using S = SingleI<K>;
  constexpr int NH = S::NH, NO = S::NO, TW = S::TW, L1 = S::L1, LPT = S::LPT, T1 = S::T1, T2 = S::T2;
  constexpr int KR = S::KR;
  constexpr int L3 = NO * NO;
  constexpr int R = TW / L3 > 0 ? TW / L3 : 1;
  constexpr int OPT = (NO + R - 1) / R;
  static_assert(S::BOUND * 32768LL < 2147483648LL, "integer Kronecker sum exceeds int32");
  static_assert(KR >= 5 && int_recombination_fits_bound(S::BOUND, KR), "integer recombination exceeds 2^51");
  static_assert(R % 2 == 0 || OPT == 1, "outputs of a thread must share one parity pattern");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / TW, lane = threadIdx.x % TW;
  const unsigned tmask = TW == 32 ? 0xffffffffu : (((1u << TW) - 1u) << ((threadIdx.x % 32) / TW * TW));
  unsigned char* base = smem_raw + (size_t)team * S::PER;
  double* c2cls = reinterpret_cast<double*>(base);
  double* sbase = c2cls + 8;
  int* T1i = reinterpret_cast<int*>(base + 80);         // P1 (M, K), P2 (M, K)
  float* T1f = reinterpret_cast<float*>(T1i + 4 * T1);  // r (M, K)
  int* T2i = reinterpret_cast<int*>(T1f + 2 * T1);      // P1 (MM, MK + KM), P2 (MM, MK + KM)
  float* T2f = reinterpret_cast<float*>(T2i + 4 * T2);  // r (MM, MK + KM)
  const int64_t t = (int64_t)blockIdx.x * S::TPB + team;
  const bool active = t < a.n_uniform;
  const int64_t g = active ? a.list_uniform[t] : 0;
  const uint64_t smask = active ? a.smask[g] : 0ull;
  constexpr double DEN = (double)IntElem<K>::DM * IntElem<K>::DM * IntElem<K>::DK;
  if (active && lane < 9) {
    const double coef = a.coeff[g];
    const double s = a.scale[0];
    if (lane == 8) {
      *sbase = coef * s / DEN;
    } else if constexpr (MODE == 1) {
      const double md0 = bmerged<K, false>(0, K), kd0 = bmerged<K, true>(0, K);
      const double md1 = bmerged<K, false>(1, K + 1), kd1 = bmerged<K, true>(1, K + 1);
      const double mdx = (lane & 1) ? md1 : md0, kdx = (lane & 1) ? kd1 : kd0;
      const double mdy = (lane & 2) ? md1 : md0, kdy = (lane & 2) ? kd1 : kd0;
      const double mdz = (lane & 4) ? md1 : md0, kdz = (lane & 4) ? kd1 : kd0;
      c2cls[lane] = c2 / (coef * (s * kdx * mdy * mdz + s * mdx * kdy * mdz + s * mdx * mdy * kdz));
    }
  }
  // this thread's outputs: line ol = (i, j), k = part + R * o
  const int ol = lane % L3, part = lane / L3;
  const bool has_out = lane < L3 * R;
  double pre_xp[OPT], pre_g[OPT], xv[OPT];
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    const int kk = part + R * o;
    pre_xp[o] = pre_g[o] = xv[o] = 0.0;
    if constexpr (MODE == 1) {
      if (active && has_out && kk < NO) {
        const int64_t slot = g * F::NOWN + ol + L3 * kk;
        pre_g[o] = gvec[slot];
        xv[o] = x[slot];
        if (xprev) pre_xp[o] = xprev[slot];
      }
    }
  }
  // the halo lines of this thread in FP64 (three segments: neighbours -1, 0, +1)
  double v[LPT][NH];
  int ex = 0;
#pragma unroll
  for (int q = 0; q < LPT; ++q) {
    const int line = lane + q * TW;
#pragma unroll
    for (int c = 0; c < NH; ++c) v[q][c] = 0.0;
    if (active && line < L1) {
      int oy, ly, oz, lz;
      halo_seg<K>(line % NH, oy, ly);
      halo_seg<K>(line / NH, oz, lz);
      const int row = NO * (ly + NO * lz);
      const int32_t* nb = a.nbr + g * F::NNB;
      const int32_t b0 = nb[nbi<3>(-1, oy, oz)], b1 = nb[nbi<3>(0, oy, oz)], b2 = nb[nbi<3>(1, oy, oz)];
      if (b0 >= 0) load_run<double, K>(x + (int64_t)b0 * F::NOWN + row + K, v[q]);
      if (b1 >= 0) load_run<double, 2 * K>(x + (int64_t)b1 * F::NOWN + row, v[q] + K);
      if (b2 >= 0) v[q][3 * K] = x[(int64_t)b2 * F::NOWN + row];
#pragma unroll
      for (int c = 0; c < NH; ++c) {
        const int e = (int)((__double_as_longlong(v[q][c]) >> 52) & 0x7FF);
        ex = e > ex ? e : ex;
      }
    }
  }
  // the group's largest biased exponent (1 for an all-zero halo)
  const int em = max(1, (int)__reduce_max_sync(tmask, (unsigned)ex));
  const int eq = em == 0x7FF ? 1010 : em - 1037;
  // stage 1: x direction per halo line, per component
#pragma unroll
  for (int q = 0; q < LPT; ++q) {
    const int line = lane + q * TW;
    if (!active || line >= L1) continue;
    auto xrows = [&](const auto* w, auto* oM, auto* oK) {
      using T = std::remove_const_t<std::remove_reference_t<decltype(w[0])>>;
      T m[NO], k[NO];
      static_for<0, NO>([&](auto r) {
        T sm = 0, sk = 0;
        static_for<0, NH>([&](auto c) {
          constexpr int bm = imerged<K, false>(r, c), bk = imerged<K, true>(r, c);
          if constexpr (bm != 0) sm += (T)bm * w[c];
          if constexpr (bk != 0) sk += (T)bk * w[c];
        });
        m[r] = sm;
        k[r] = sk;
      });
      static_for<0, NO / 2>([&](auto h) {
        oM[line * NO + 2 * h] = m[2 * h];
        oM[line * NO + 2 * h + 1] = m[2 * h + 1];
        oK[line * NO + 2 * h] = k[2 * h];
        oK[line * NO + 2 * h + 1] = k[2 * h + 1];
      });
    };
    int w1[NH], w2[NH];
    float w3[NH];
    static_for<0, NH>([&](auto c) { split_exact(v[q][c], eq, w1[c], w2[c], w3[c]); });
    xrows(w1, T1i, T1i + T1);
    xrows(w2, T1i + 2 * T1, T1i + 3 * T1);
    xrows(w3, T1f, T1f + T1);
  }
  __syncwarp(tmask);
  // stage 2: y direction; T1 layout [z][y][i] -> T2 layout [z][j][i]
  if (active) {
    for (int l2 = lane; l2 < NH * NO; l2 += TW) {
      const int z = l2 / NO, i = l2 % NO;
      auto yrows = [&](const auto* iM, const auto* iK, auto* oMM, auto* oQ) {
        using T = std::remove_const_t<std::remove_reference_t<decltype(iM[0])>>;
        T vm[NH], vk[NH];
        static_for<0, NH>([&](auto y) {
          vm[y] = iM[(z * NH + y) * NO + i];
          vk[y] = iK[(z * NH + y) * NO + i];
        });
        static_for<0, NO>([&](auto j) {
          T mm = 0, mk = 0, km = 0;
          static_for<0, NH>([&](auto c) {
            constexpr int bm = imerged<K, false>(j, c), bk = imerged<K, true>(j, c);
            if constexpr (bm != 0) {
              mm += (T)bm * vm[c];
              km += (T)bm * vk[c];
            }
            if constexpr (bk != 0) mk += (T)bk * vm[c];
          });
          const int o = (z * NO + j) * NO + i;
          oMM[o] = mm;
          oQ[o] = mk + km;
        });
      };
      yrows(T1i, T1i + T1, T2i, T2i + T2);
      yrows(T1i + 2 * T1, T1i + 3 * T1, T2i + 2 * T2, T2i + 3 * T2);
      yrows(T1f, T1f + T1, T2f, T2f + T2);
    }
  }
  __syncwarp(tmask);
  if (!active || !has_out) return;
  // stage 3: z direction per component, the recombination and the update
  int o1[OPT], o2[OPT];
  float o3[OPT];
  auto zrows = [&](const auto* iMM, const auto* iQ, auto* acc) {
    using T = std::remove_const_t<std::remove_reference_t<decltype(iMM[0])>>;
    T p[NH], q[NH];
    static_for<0, NH>([&](auto z) {
      p[z] = iMM[z * L3 + ol];
      q[z] = iQ[z * L3 + ol];
    });
    own_rows<NO, R>(part, [&](auto o, auto r) {
      T y = 0;
      static_for<0, NH>([&](auto c) {
        constexpr int bm = imerged<K, false>(r, c), bk = imerged<K, true>(r, c);
        if constexpr (bk != 0) y += (T)bk * p[c];
        if constexpr (bm != 0) y += (T)bm * q[c];
      });
      acc[o] = y;
    });
  };
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    o1[o] = o2[o] = 0;
    o3[o] = 0.f;
  }
  zrows(T2i, T2i + T2, o1);
  zrows(T2i + 2 * T2, T2i + 3 * T2, o2);
  zrows(T2f, T2f + T2, o3);
  constexpr double LOW = 1.0 / (double)(1LL << (29 + KR));
  const double sc = em == 0x7FF ? __longlong_as_double(0x7FF8000000000000LL)
                                : *sbase * LOW * pow2_normal(em - 1023);
  double c2d = 0.0, c2s = 0.0;
  if constexpr (MODE == 1) {
    c2d = c2cls[(ol % NO & 1) + 2 * (ol / NO & 1) + 4 * (part & 1)];
    c2s = c2d * sc;
  }
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    const int kk = part + R * o;
    if (kk >= NO) break;
    const int node = ol + L3 * kk;
    if (!((smask >> node) & 1ull)) continue;
    const double ts = i64_to_double_alu(((long long)o1[o] << (15 + KR)) + ((long long)o2[o] << KR) +
                                        (long long)f32_fixed_rint<KR>(o3[o]));
    const int64_t slot = g * F::NOWN + node;
    if constexpr (MODE == 0) {
      out[slot] = sc * ts;
    } else {
      out[slot] = fma(-c2s, ts, fma(c2d, pre_g[o], fma(c1, xv[o] - pre_xp[o], xv[o])));
    }
  }
}

// ------------------------------------- Q2 brick smoother, persistent blocks
// The FP32 Q2 brick smoother (apply and Chebyshev step) with the same three
// packed contractions as level_cheb_brick_f2_kernel, arranged so that the
// work per stored node is mostly the contractions themselves:
//   * each block loops over bricks (grid = resident blocks), so every
//     thread's halo-line geometry, output columns and diagonal factors are
//     computed once per launch, not once per brick;
//   * slots are 32-bit (level vectors stay below 2^32 slots);
//   * the members, an "every member node is an S node" flag and the
//     coefficient come from one 8-byte record per brick, so interior bricks
//     skip the S-mask tests;
//   * with cubic cells (s_x = s_y = s_z = s) the scale factor joins the
//     coefficient and the contractions carry no scale multiplications;
//   * in the last stage a thread takes four consecutive z rows of its
//     column (two vertex and two interior rows, so both halves of the block
//     do the same work), all in one group of the brick: one base slot and
//     compile-time offsets.
// The Chebyshev step is out = x + c1 (x - x_prev) + (c2 / d) (g / (a s) - y)
// with A x = a s y and D = a s d, d the node's diagonal of the unscaled
// Kronecker sum (it depends on index parities only).
// Shared arrays (float2 units for T1, T2): stage-1 result of halo line
// (hy, hz), output row r at T1[hz PZ1 + 9 hy + 2 r]; stage-2 result at
// T2[z ZS + 8 j + i]; the brick's own x values at Xown[64 z + 8 y + (x ^ 4
// ((y >> 2) & 1))].  8-byte accesses are served per half-warp; with these
// strides the 16 lanes of a half-warp meet 16 distinct bank pairs in the
// stage-1 stores and the stage-2 loads (no bank conflicts), and the swizzle
// spreads the own-value rows of eight consecutive lines over distinct banks.
struct BrickQ2 {
  static constexpr int K = 2, NO = 4, OB = 8, HB = 11, NOWN = 64, TB = 128;
  static constexpr int HY1 = 9;    // stage-1 halo-line stride (float2)
  static constexpr int R1 = 2;     // stage-1 output-row stride (float2)
  static constexpr int PZ1 = 115;  // stage-1 z-plane stride (float2)
  static constexpr int ZS = 72;    // stage-2 z-plane stride (float2), 8 mod 16
  // array sizes in bytes, each rounded up to 16 so that every array starts
  // 16-byte aligned (the own values and the table are read and written as
  // 16-byte vectors)
  static constexpr size_t T1B = ((size_t)HB * PZ1 * 8 + 15) / 16 * 16;
  static constexpr size_t T2B = ((size_t)HB * ZS * 8 + 15) / 16 * 16;
  static constexpr size_t XOB = (size_t)OB * OB * OB * 4;
  static constexpr size_t bytes() { return T1B + T2B + XOB + 64 * 4; }
  // single groups after the bricks, one per warp: per warp a mask, a
  // coefficient, a neighbour table and the single-group kernel's arrays,
  // over the same shared memory
  static constexpr int WARPS = TB / 32;
  static constexpr size_t SG_HEAD = ((size_t)WARPS * (8 + 4 + 4 * 27) + 15) / 16 * 16;
  static constexpr size_t SG_PER = (size_t)FastSmem<float, 3, 2>::PER * 4;
  static_assert(SG_HEAD + WARPS * SG_PER <= T1B + T2B + XOB + 64 * 4, "single groups fit the brick layout");
};

// Persistent blocks over the work items [0, n_bricks_all + n_single_chunks):
// first the bricks, then chunks of four single groups (list_uniform), one
// group per warp with the single-group kernel's code, so that the groups
// outside bricks need no launch of their own and fill the tail of the brick
// phase.
template <int MODE, bool ISO>
__global__ void __launch_bounds__(BrickQ2::TB, 9)
level_cheb_brick_q2_kernel(LevelArgs a, int64_t n_single_chunks, const float* __restrict__ x,
                           const float* __restrict__ xprev, const float* __restrict__ gvec,
                           float* __restrict__ out, float c1, float c2) {
  using B = BrickQ2;
  constexpr int K = B::K, NO = B::NO, OB = B::OB, HB = B::HB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* T1 = reinterpret_cast<float2*>(smem_raw);
  float2* T2 = reinterpret_cast<float2*>(smem_raw + B::T1B);
  float* Xown = reinterpret_cast<float*>(smem_raw + B::T1B + B::T2B);
  int32_t* tab = reinterpret_cast<int32_t*>(smem_raw + B::T1B + B::T2B + B::XOB);
  static_assert(B::T1B % 16 == 0 && B::T2B % 16 == 0 && B::XOB % 16 == 0, "16-byte aligned arrays");
  const int tid = threadIdx.x;

  // ---- per-thread constants of the launch
  // stage 1: halo line (hy, hz), one per thread below HB * HB
  const bool st1 = tid < HB * HB;
  const int hy = tid % HB, hz = tid / HB;
  int gy, ly, gz, lz;
  brick_seg<K>(hy, gy, ly);
  brick_seg<K>(hz, gz, lz);
  const uint32_t row = NO * (ly + NO * lz);
  const int tb = 4 * ((gy + 1) + 4 * (gz + 1));
  const bool own_line = gy >= 0 && gy <= 1 && gz >= 0 && gz <= 1;
  const int by1 = gy * NO + ly;
  float* xo_dst = Xown + OB * (by1 + OB * (gz * NO + lz));
  const int xo_swz = 4 * ((by1 >> 2) & 1);  // own x halves swap places on rows 4..7
  float2* t1_dst = T1 + hz * B::PZ1 + B::HY1 * hy;
  // stage 2: line (z, i)
  const bool st2 = tid < HB * OB;
  const int z2 = tid / OB, i2 = tid % OB;
  // stage 3: column (oi, oj), rows 4 part .. 4 part + 3 of the brick, i.e.
  // z planes 0..3 of the groups at brick position (oi / 4, oj / 4, part)
  const int ol = tid % (OB * OB), part = tid / (OB * OB);
  const int oi = ol % OB, oj = ol / OB;
  const int gsel = (oi / NO) + 2 * (oj / NO) + 4 * part;
  const int own_tab = (oi / NO + 1) + 4 * ((oj / NO + 1) + 4 * (part + 1));
  const uint32_t node_xy = (oi % NO) + NO * (oj % NO);
  const float sx = a.scale32[0], sy = a.scale32[1], sz = a.scale32[2];
  const float s_iso = ISO ? sx : 1.f;
  // c2 / d for the two z parities of the rows (x and y parities are fixed)
  float c2od[2] = {0.f, 0.f};
  if constexpr (MODE == 1) {
    const float md0 = (float)bbrick<K, false>(0, K), kd0 = (float)bbrick<K, true>(0, K);
    const float md1 = (float)bbrick<K, false>(1, K + 1), kd1 = (float)bbrick<K, true>(1, K + 1);
    const float mdx = (oi & 1) ? md1 : md0, kdx = (oi & 1) ? kd1 : kd0;
    const float mdy = (oj & 1) ? md1 : md0, kdy = (oj & 1) ? kd1 : kd0;
#pragma unroll
    for (int pz = 0; pz < 2; ++pz) {
      const float mdz = pz ? md1 : md0, kdz = pz ? kd1 : kd0;
      const float d = ISO ? (kdx * mdy * mdz + mdx * kdy * mdz + mdx * mdy * kdz)
                          : (sx * kdx * mdy * mdz + sy * mdx * kdy * mdz + sz * mdx * mdy * kdz);
      c2od[pz] = c2 / d;
    }
  }

  const int64_t n_items = a.n_bricks_all + n_single_chunks;
  for (int64_t br = blockIdx.x; br < n_items; br += gridDim.x) {
    if (br >= a.n_bricks_all) {
      // a chunk of single groups; the barrier ends every warp's use of the
      // brick arrays that this layout overlays
      __syncthreads();
      const int warp = tid / 32, lane = tid % 32;
      uint64_t* masks = reinterpret_cast<uint64_t*>(smem_raw);
      float* coefs = reinterpret_cast<float*>(masks + B::WARPS);
      int32_t* nb = reinterpret_cast<int32_t*>(coefs + B::WARPS) + warp * 27;
      float* mine = reinterpret_cast<float*>(smem_raw + B::SG_HEAD + warp * B::SG_PER);
      fast_group_step<float, 3, K, MODE>(a, (br - a.n_bricks_all) * B::WARPS + warp, lane, masks + warp,
                                         coefs + warp, nb, mine, x, xprev, gvec, out, c1, c2);
      continue;
    }
    if (tid < 64) tab[tid] = a.bricks[br * 64 + tid];
    const uint2 info = a.brick_info[br];
    __syncthreads();
    const float ce = __uint_as_float(info.y) * s_iso;  // a s (ISO) or a
    const bool member = (info.x >> gsel) & 1u;
    // this thread's four outputs: slots base + 16 nz, nz = 0..3
    const uint32_t base = (uint32_t)tab[own_tab] * B::NOWN + node_xy;
    float pg[4] = {0.f, 0.f, 0.f, 0.f}, pxp[4] = {0.f, 0.f, 0.f, 0.f};
    if constexpr (MODE == 1) {
      if (member) {
#pragma unroll
        for (int nz = 0; nz < 4; ++nz) pg[nz] = gvec[base + 16 * nz];
        if (xprev) {
#pragma unroll
          for (int nz = 0; nz < 4; ++nz) pxp[nz] = xprev[base + 16 * nz];
        }
      }
    }
    // stage 1: halo rows along x -> (mass, stiffness) pairs
    if (st1) {
      const int4 b = *reinterpret_cast<const int4*>(tab + tb);
      float v[HB];
      if (b.x >= 0) load_run<float, K>(x + ((uint32_t)b.x * B::NOWN + row + K), v);
      else v[0] = v[1] = 0.f;
      if (b.y >= 0) load_run<float, 2 * K>(x + ((uint32_t)b.y * B::NOWN + row), v + K);
      else v[2] = v[3] = v[4] = v[5] = 0.f;
      if (b.z >= 0) load_run<float, 2 * K>(x + ((uint32_t)b.z * B::NOWN + row), v + 3 * K);
      else v[6] = v[7] = v[8] = v[9] = 0.f;
      v[5 * K] = b.w >= 0 ? x[(uint32_t)b.w * B::NOWN + row] : 0.f;
      if (own_line) {
        *reinterpret_cast<float4*>(xo_dst + xo_swz) = make_float4(v[2], v[3], v[4], v[5]);
        *reinterpret_cast<float4*>(xo_dst + (4 ^ xo_swz)) = make_float4(v[6], v[7], v[8], v[9]);
      }
      float2 vv[HB];
      static_for<0, HB>([&](auto c) { vv[c] = make_float2(v[c], v[c]); });
      static_for<0, OB>([&](auto r) {
        float2 acc = make_float2(0.f, 0.f);
        static_for<0, HB>([&](auto c) {
          constexpr double bm = bbrick<K, false>(r, c);
          constexpr double bk = bbrick<K, true>(r, c);
          if constexpr (bm != 0.0 || bk != 0.0) acc = __ffma2_rn(make_float2((float)bm, (float)bk), vv[c], acc);
        });
        t1_dst[B::R1 * r] = acc;
      });
    }
    __syncthreads();
    // stage 2: y direction; stores (P, Q) = (sz MM, sy MK + sx KM), or
    // (MM, MK + KM) for cubic cells
    if (st2) {
      float2 w[HB];
      static_for<0, HB>([&](auto yy) { w[yy] = T1[z2 * B::PZ1 + B::HY1 * yy + B::R1 * i2]; });
      static_for<0, OB>([&](auto j) {
        float2 acc = make_float2(0.f, 0.f);  // (MM, KM)
        float mk = 0.f;
        static_for<0, HB>([&](auto c) {
          constexpr double bm = bbrick<K, false>(j, c);
          constexpr double bk = bbrick<K, true>(j, c);
          if constexpr (bm != 0.0) acc = __ffma2_rn(make_float2((float)bm, (float)bm), w[c], acc);
          if constexpr (bk != 0.0) mk = fmaf((float)bk, w[c].x, mk);
        });
        T2[z2 * B::ZS + j * OB + i2] = ISO ? make_float2(acc.x, mk + acc.y)
                                           : make_float2(sz * acc.x, sy * mk + sx * acc.y);
      });
    }
    __syncthreads();
    // stage 3: z direction for rows 4 part .. 4 part + 3, then the update
    if (member) {
      uint32_t wmask = 0xFu;  // outputs that are S nodes
      if (!(info.x & kBrickAllS)) {
        const uint64_t m = a.smask[base / B::NOWN] >> node_xy;
        wmask = (uint32_t)(m & 1u) | (uint32_t)((m >> 15) & 2u) | (uint32_t)((m >> 30) & 4u) |
                (uint32_t)((m >> 45) & 8u);
      }
      const float inv_ce = MODE == 1 ? __frcp_rn(ce) : 0.f;
      auto rows = [&](auto P) {
        constexpr int R0 = decltype(P)::value * 4;
        float2 pq[HB];
        static_for<0, HB>([&](auto c) { pq[c] = T2[c * B::ZS + ol]; });
        static_for<0, 4>([&](auto nz) {
          constexpr int r = R0 + nz;
          float2 acc = make_float2(0.f, 0.f);
          static_for<0, HB>([&](auto c) {
            constexpr double bm = bbrick<K, false>(r, c);
            constexpr double bk = bbrick<K, true>(r, c);
            if constexpr (bm != 0.0 || bk != 0.0) acc = __ffma2_rn(make_float2((float)bk, (float)bm), pq[c], acc);
          });
          const float y = acc.x + acc.y;
          if (!((wmask >> nz) & 1u)) return;
          if constexpr (MODE == 0) {
            out[base + 16 * nz] = ce * y;
          } else {
            const float xv = Xown[(oi ^ (4 * ((oj >> 2) & 1))) + OB * (oj + OB * r)];
            out[base + 16 * nz] = fmaf(c2od[nz & 1], fmaf(pg[nz], inv_ce, -y), fmaf(c1, xv - pxp[nz], xv));
          }
        });
      };
      if (part == 0) rows(std::integral_constant<int, 0>{});
      else rows(std::integral_constant<int, 1>{});
    }
  }
}

// Slot (in the level l-1 vector) of node jd of the parent cell of group g
// at level l: level 1 parents are coarse cells on the (K n0 + 1)^d lattice;
// otherwise the parent is child cb of its own group, whose node block and
// +1 neighbours hold the parent's nodes at local index cb*K + jd.
template <int DIM, int K>
__device__ __forceinline__ int64_t parent_node_slot(const LevelArgs& a, int64_t parent, uint64_t st,
                                                    const int* jd) {
  using G = Geo<DIM, K>;
  if (a.level == 1) {
    const int64_t n0x = (a.coarse_lat[0] - 1) / K, n0y = (a.coarse_lat[1] - 1) / K;
    const int64_t c[3] = {parent % n0x, DIM > 1 ? (parent / n0x) % n0y : 0, DIM > 2 ? parent / (n0x * n0y) : 0};
    int64_t q[3];
    for (int d = 0; d < 3; ++d) q[d] = d < DIM ? K * c[d] + jd[d] : 0;
    return q[0] + a.coarse_lat[0] * (q[1] + a.coarse_lat[1] * q[2]);
  }
  const int cb[3] = {(int)((st >> 60) & 1), (int)((st >> 61) & 1), (int)((st >> 62) & 1)};
  int ni = 0, loc = 0, mul3 = 1, mulo = 1;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int pl = cb[d] * K + jd[d];
    const int o = pl == 2 * K ? 1 : 0;
    ni += (o + 1) * mul3;
    loc += (pl - 2 * K * o) * mulo;
    mul3 *= 3;
    mulo *= G::NO;
  }
  const int32_t blk = a.nbr_coarse[parent * G::NNB + ni];
  if (blk < 0) return -1;
  return (int64_t)blk * G::NOWN + loc;
}

// parent_node_slot with the parent group's level l-1 neighbour row already
// at hand (`cnb`, levels l >= 2)
template <int DIM, int K>
__device__ __forceinline__ int64_t parent_node_slot_row(uint64_t st, const int* jd, const int32_t* cnb) {
  using G = Geo<DIM, K>;
  int ni = 0, loc = 0, mul3 = 1, mulo = 1;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int pl = (int)((st >> (60 + d)) & 1) * K + jd[d];
    const int o = pl == 2 * K ? 1 : 0;
    ni += (o + 1) * mul3;
    loc += (pl - 2 * K * o) * mulo;
    mul3 *= 3;
    mulo *= G::NO;
  }
  const int32_t blk = cnb[ni];
  if (blk < 0) return -1;
  return (int64_t)blk * G::NOWN + loc;
}

// ------------------------------------------------- residual + restriction
// Per group: g_{l-1} += R (w g) - a R A_G u on the parent cell's (K+1)^d nodes.
// R A_G is again a Kronecker sum, of the (K+1) x (2K+1) products E^T K and
// E^T M, so the restricted residual is one sum factorisation of u (and of
// w g with E^T).  w = 1 / (number of groups sharing the node) is only needed
// where g can be nonzero -- on S nodes, which every touching group refines --
// so it is 2^-(number of directions in which the node is on the group's
// boundary), a separable factor of E^T.  Dirichlet fine nodes interpolate
// from Dirichlet coarse nodes only, so their garbage lands on coarse slots
// that are never read.  u^I = 0 and g^I = 0 here (down-sweep).
template <int K, int WHICH>  // WHICH: 0 = E^T M, 1 = E^T K, 2 = E^T diag(w)
__host__ __device__ constexpr double rmat(int j, int a) {
  if (WHICH == 2) return embed1<K>(a, j) * ((a == 0 || a == 2 * K) ? 0.5 : 1.0);
  double v = 0.0;
  for (int r = 0; r <= 2 * K; ++r) v += embed1<K>(r, j) * bgrp<K, WHICH == 1>(r, a);
  return v;
}

template <typename T, int DIM, int K>
struct RestrictSmem {
  using F = Fast<DIM, K>;
  static constexpr int NG = 2 * K + 1, N1 = K + 1;
  static constexpr int LX = DIM == 3 ? NG * NG : NG;      // stage-x lines
  static constexpr int SX = LX * N1;                       // per array
  static constexpr int SY = DIM == 3 ? NG * N1 * N1 : 0;   // per array
  static constexpr int PER = 3 * SX + 4 * SY;
  // per team: state, coefficient, neighbour table, parent's coarse row
  static constexpr size_t HEADER = ((size_t)F::TPB * (8 + sizeof(T) + 8 * F::NNB) + 15) / 16 * 16;
  static constexpr size_t bytes() { return HEADER + (size_t)F::TPB * PER * sizeof(T); }
};

template <typename T, int DIM, int K>
__global__ void __launch_bounds__(256)
level_residual_restrict_kernel(LevelArgs a, const T* __restrict__ u, const T* __restrict__ gvec,
                               T* __restrict__ gc, const int32_t* __restrict__ list, int64_t n_list) {
  using F = Fast<DIM, K>;
  using S = RestrictSmem<T, DIM, K>;
  constexpr int NG = S::NG, N1 = S::N1, NO = F::NO, TW = F::TW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / TW;
  const int lane = threadIdx.x % TW;
  const int64_t gi = (int64_t)blockIdx.x * F::TPB + team;
  const bool active = gi < n_list;
  const int64_t g = active ? (list ? (int64_t)list[gi] : gi) : 0;
  uint64_t* states = reinterpret_cast<uint64_t*>(smem_raw);
  T* coefs = reinterpret_cast<T*>(states + F::TPB);
  int32_t* nb = reinterpret_cast<int32_t*>(coefs + F::TPB) + team * F::NNB;
  int32_t* crow = reinterpret_cast<int32_t*>(coefs + F::TPB) + (F::TPB + team) * F::NNB;
  const bool rows = a.group_cnb != nullptr;  // levels >= 2: the coarse row comes with the header
  T* XM = reinterpret_cast<T*>(smem_raw + S::HEADER) + (size_t)team * S::PER;
  T* XK = XM + S::SX;
  T* XG = XK + S::SX;
  T* YMM = XG + S::SX;
  T* YMK = YMM + S::SY;
  T* YKM = YMK + S::SY;
  T* YG = YKM + S::SY;
  if (active) {
    for (int i = lane; i < F::NNB; i += TW) nb[i] = a.nbr[g * F::NNB + i];
    if (rows)
      for (int i = lane; i < F::NNB; i += TW) crow[i] = a.group_cnb[g * F::NNB + i];
    if (lane == 0) {
      states[team] = a.state[g];
      coefs[team] = group_coef<T>(a, g);
    }
  }
  __syncwarp();
  // stage x: rows (y, z) of the group's node lattice; u and g from the own
  // block (2K values) and the +x neighbour (1 value)
  if (active) {
    for (int line = lane; line < S::LX; line += TW) {
      const int y = DIM > 1 ? line % NG : 0, z = DIM > 2 ? line / NG : 0;
      const int oy = y == 2 * K ? 1 : 0, oz = z == 2 * K ? 1 : 0;
      const int row = NO * ((oy ? 0 : y) + NO * (oz ? 0 : z));
      T uv[NG], gv[NG];
      const int32_t b1 = nb[nbi<DIM>(0, oy, oz)], b2 = nb[nbi<DIM>(1, oy, oz)];
      if (b1 >= 0) {
        load_run<T, 2 * K>(u + (int64_t)b1 * F::NOWN + row, uv);
        load_run<T, 2 * K>(gvec + (int64_t)b1 * F::NOWN + row, gv);
      } else {
        for (int i = 0; i < 2 * K; ++i) uv[i] = gv[i] = T(0);
      }
      uv[2 * K] = b2 >= 0 ? u[(int64_t)b2 * F::NOWN + row] : T(0);
      gv[2 * K] = b2 >= 0 ? gvec[(int64_t)b2 * F::NOWN + row] : T(0);
      static_for<0, N1>([&](auto j) {
        T m = 0, kk = 0, w = 0;
        static_for<0, NG>([&](auto c) {
          constexpr double em = rmat<K, 0>(j, c), ek = rmat<K, 1>(j, c), ew = rmat<K, 2>(j, c);
          if constexpr (em != 0.0) m += (T)em * uv[c];
          if constexpr (ek != 0.0) kk += (T)ek * uv[c];
          if constexpr (ew != 0.0) w += (T)ew * gv[c];
        });
        XM[line * N1 + j] = m;
        XK[line * N1 + j] = kk;
        XG[line * N1 + j] = w;
      });
    }
  }
  __syncwarp();
  const T sx = level_scale<T>(a, 0), sy = level_scale<T>(a, 1), sz = level_scale<T>(a, 2);
  const T coef = coefs[team];
  const uint64_t st = states[team];
  const int64_t parent = active && !rows ? a.parent[g] : 0;
  if constexpr (DIM == 3) {
    // stage y: lines (z, jx); X layout [z][y][jx] -> Y layout [z][jy][jx]
    if (active) {
      for (int line = lane; line < NG * N1; line += TW) {
        const int z = line / N1, jx = line % N1;
        T vm[NG], vk[NG], vg[NG];
        static_for<0, NG>([&](auto y) {
          vm[y] = XM[(z * NG + y) * N1 + jx];
          vk[y] = XK[(z * NG + y) * N1 + jx];
          vg[y] = XG[(z * NG + y) * N1 + jx];
        });
        static_for<0, N1>([&](auto j) {
          T mm = 0, mk = 0, km = 0, gg = 0;
          static_for<0, NG>([&](auto c) {
            constexpr double em = rmat<K, 0>(j, c), ek = rmat<K, 1>(j, c), ew = rmat<K, 2>(j, c);
            if constexpr (em != 0.0) {
              mm += (T)em * vm[c];
              km += (T)em * vk[c];
            }
            if constexpr (ek != 0.0) mk += (T)ek * vm[c];
            if constexpr (ew != 0.0) gg += (T)ew * vg[c];
          });
          const int o = (z * N1 + j) * N1 + jx;
          YMM[o] = mm;
          YMK[o] = mk;
          YKM[o] = km;
          YG[o] = gg;
        });
      }
    }
    __syncwarp();
    // stage z: lines (jy, jx), scatter into the parent's nodes
    if (active) {
      for (int line = lane; line < N1 * N1; line += TW) {
        T pm[NG], pq[NG], pg[NG];
        static_for<0, NG>([&](auto z) {
          pm[z] = sz * YMM[z * N1 * N1 + line];
          pq[z] = sy * YMK[z * N1 * N1 + line] + sx * YKM[z * N1 * N1 + line];
          pg[z] = YG[z * N1 * N1 + line];
        });
        static_for<0, N1>([&](auto j) {
          T op = 0, rg = 0;
          static_for<0, NG>([&](auto c) {
            constexpr double em = rmat<K, 0>(j, c), ek = rmat<K, 1>(j, c), ew = rmat<K, 2>(j, c);
            if constexpr (ek != 0.0) op += (T)ek * pm[c];
            if constexpr (em != 0.0) op += (T)em * pq[c];
            if constexpr (ew != 0.0) rg += (T)ew * pg[c];
          });
          const int jd[3] = {line % N1, line / N1, j};
          const int64_t slot = rows ? parent_node_slot_row<DIM, K>(st, jd, crow) : parent_node_slot<DIM, K>(a, parent, st, jd);
          if (slot >= 0) {
            if (a.deterministic) gc[slot] += rg - coef * op;  // one colour: parent cells share no node
            else atomicAdd(gc + slot, rg - coef * op);
          }
        });
      }
    }
  } else {
    if (active) {
      for (int jx = lane; jx < N1; jx += TW) {
        T vm[NG], vk[NG], vg[NG];
        static_for<0, NG>([&](auto y) {
          vm[y] = sy * XM[y * N1 + jx];
          vk[y] = sx * XK[y * N1 + jx];
          vg[y] = XG[y * N1 + jx];
        });
        static_for<0, N1>([&](auto j) {
          T op = 0, rg = 0;
          static_for<0, NG>([&](auto c) {
            constexpr double em = rmat<K, 0>(j, c), ek = rmat<K, 1>(j, c), ew = rmat<K, 2>(j, c);
            if constexpr (ek != 0.0) op += (T)ek * vm[c];
            if constexpr (em != 0.0) op += (T)em * vk[c];
            if constexpr (ew != 0.0) rg += (T)ew * vg[c];
          });
          const int jd[3] = {jx, j, 0};
          const int64_t slot = rows ? parent_node_slot_row<DIM, K>(st, jd, crow) : parent_node_slot<DIM, K>(a, parent, st, jd);
          if (slot >= 0) {
            if (a.deterministic) gc[slot] += rg - coef * op;  // one colour: parent cells share no node
            else atomicAdd(gc + slot, rg - coef * op);
          }
        });
      }
    }
  }
}

// ------------------------------------------------------------ prolongation
// Per group: the parent's (K+1)^d values interpolated to the group's
// (2K+1)^d nodes with E in each direction; stored S nodes get u += P uc, I
// nodes u = u2 = P uc (masks prepared on the host).
template <typename T, int DIM, int K>
struct ProlongSmem {
  using F = Fast<DIM, K>;
  static constexpr int NG = 2 * K + 1, N1 = K + 1;
  static constexpr int NC = ipow_c(N1, DIM);
  static constexpr int PX = (DIM == 3 ? N1 * N1 : N1) * NG;
  static constexpr int PY = DIM == 3 ? N1 * NG * NG : 0;
  static constexpr int PER = NC + PX + PY;
  // per team: state, add[2], set[2], neighbour table, parent's coarse row
  static constexpr size_t HEADER = ((size_t)F::TPB * (8 * 5 + 8 * F::NNB) + 15) / 16 * 16;
  static constexpr size_t bytes() { return HEADER + (size_t)F::TPB * PER * sizeof(T); }
};

template <typename T, int DIM, int K>
__global__ void __launch_bounds__(256)
level_prolongate_kernel(LevelArgs a, const T* __restrict__ uc, T* __restrict__ u, T* __restrict__ u2,
                        const int32_t* __restrict__ list, int64_t n_list) {
  using F = Fast<DIM, K>;
  using S = ProlongSmem<T, DIM, K>;
  constexpr int NG = S::NG, N1 = S::N1, NO = F::NO, TW = F::TW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int team = threadIdx.x / TW;
  const int lane = threadIdx.x % TW;
  const int64_t gi = (int64_t)blockIdx.x * F::TPB + team;
  const bool active = gi < n_list;
  const int64_t g = active ? (list ? (int64_t)list[gi] : gi) : 0;
  uint64_t* hdr = reinterpret_cast<uint64_t*>(smem_raw) + team * 5;  // state, add[2], set[2]
  int32_t* nb = reinterpret_cast<int32_t*>(reinterpret_cast<uint64_t*>(smem_raw) + F::TPB * 5) + team * F::NNB;
  int32_t* crow = reinterpret_cast<int32_t*>(reinterpret_cast<uint64_t*>(smem_raw) + F::TPB * 5) +
                  (F::TPB + team) * F::NNB;
  T* C = reinterpret_cast<T*>(smem_raw + S::HEADER) + (size_t)team * S::PER;
  T* PXa = C + S::NC;
  T* PYa = PXa + S::PX;
  const bool rows = a.group_cnb != nullptr;  // levels >= 2: the coarse row comes with the header
  if (active) {
    for (int i = lane; i < F::NNB; i += TW) nb[i] = a.nbr[g * F::NNB + i];
    if (rows)
      for (int i = lane; i < F::NNB; i += TW) crow[i] = a.group_cnb[g * F::NNB + i];
    if (lane == 0) hdr[0] = a.state[g];
    if (lane < 4) hdr[1 + lane] = a.pmask[g * 4 + lane];
  }
  // 3D: u at the own-block nodes of this lane's z line (the line it writes
  // below), loaded with the coarse values so that the update does not wait;
  // every fine node has one writer
  constexpr bool PRE = DIM == 3 && NG * NG <= TW;
  T u_pre[NG];
  if constexpr (PRE) {
    const int px = lane % NG, py = lane / NG;
#pragma unroll
    for (int r = 0; r < NG; ++r)
      u_pre[r] = (active && lane < NG * NG && px < NO && py < NO && r < NO) ? u[g * F::NOWN + px + NO * (py + NO * r)]
                                                                              : T(0);
  }
  __syncwarp();
  if (active) {
    const int64_t parent = rows ? 0 : a.parent[g];
    const uint64_t st = hdr[0];
    for (int n = lane; n < S::NC; n += TW) {
      const int jd[3] = {n % N1, DIM > 1 ? (n / N1) % N1 : 0, DIM > 2 ? n / (N1 * N1) : 0};
      const int64_t s = rows ? parent_node_slot_row<DIM, K>(st, jd, crow) : parent_node_slot<DIM, K>(a, parent, st, jd);
      C[n] = s >= 0 ? uc[s] : T(0);
    }
  }
  __syncwarp();
  auto write = [&](int n, T v, T pre) {  // pre: u at n, loaded early (PRE)
    const uint64_t add = hdr[1 + (n >> 6)], set = hdr[3 + (n >> 6)];
    const uint64_t bit = 1ull << (n & 63);
    const int x = n % NG, y = DIM > 1 ? (n / NG) % NG : 0, z = DIM > 2 ? n / (NG * NG) : 0;
    if (add & bit) {
      if constexpr (PRE) u[g * F::NOWN + x + NO * (y + NO * z)] = pre + v;
      else u[g * F::NOWN + x + NO * (y + NO * z)] += v;
    } else if (set & bit) {
      const int ox = x == 2 * K, oy = y == 2 * K, oz = z == 2 * K;
      const int32_t blk = nb[nbi<DIM>(ox, oy, oz)];
      const int64_t s = (int64_t)blk * F::NOWN + (ox ? 0 : x) + NO * ((oy ? 0 : y) + NO * (oz ? 0 : z));
      u[s] = v;
      u2[s] = v;
    }
  };
  if constexpr (DIM == 3) {
    // x: lines (jy, jz)
    if (active) {
      for (int line = lane; line < N1 * N1; line += TW) {
        T c[N1];
        static_for<0, N1>([&](auto j) { c[j] = C[line * N1 + j]; });
        static_for<0, NG>([&](auto r) {
          T v = 0;
          static_for<0, N1>([&](auto j) {
            constexpr double e = embed1<K>(r, j);
            if constexpr (e != 0.0) v += (T)e * c[j];
          });
          PXa[line * NG + r] = v;
        });
      }
    }
    __syncwarp();
    // y: lines (jz, x); PX layout [jz][jy][x] -> PY layout [jz][y][x]
    if (active) {
      for (int line = lane; line < N1 * NG; line += TW) {
        const int jz = line / NG, x = line % NG;
        T c[N1];
        static_for<0, N1>([&](auto j) { c[j] = PXa[(jz * N1 + j) * NG + x]; });
        static_for<0, NG>([&](auto r) {
          T v = 0;
          static_for<0, N1>([&](auto j) {
            constexpr double e = embed1<K>(r, j);
            if constexpr (e != 0.0) v += (T)e * c[j];
          });
          PYa[(jz * NG + r) * NG + x] = v;
        });
      }
    }
    __syncwarp();
    // z: lines (y, x), write
    if (active) {
      for (int line = lane; line < NG * NG; line += TW) {
        T c[N1];
        static_for<0, N1>([&](auto j) { c[j] = PYa[j * NG * NG + line]; });
        static_for<0, NG>([&](auto r) {
          T v = 0;
          static_for<0, N1>([&](auto j) {
            constexpr double e = embed1<K>(r, j);
            if constexpr (e != 0.0) v += (T)e * c[j];
          });
          write(line + NG * NG * r, v, PRE ? u_pre[r] : T(0));
        });
      }
    }
  } else {
    if (active) {
      for (int line = lane; line < N1; line += TW) {
        T c[N1];
        static_for<0, N1>([&](auto j) { c[j] = C[line * N1 + j]; });
        static_for<0, NG>([&](auto r) {
          T v = 0;
          static_for<0, N1>([&](auto j) {
            constexpr double e = embed1<K>(r, j);
            if constexpr (e != 0.0) v += (T)e * c[j];
          });
          PXa[line * NG + r] = v;
        });
      }
    }
    __syncwarp();
    if (active) {
      for (int x = lane; x < NG; x += TW) {
        T c[N1];
        static_for<0, N1>([&](auto j) { c[j] = PXa[j * NG + x]; });
        static_for<0, NG>([&](auto r) {
          T v = 0;
          static_for<0, N1>([&](auto j) {
            constexpr double e = embed1<K>(r, j);
            if constexpr (e != 0.0) v += (T)e * c[j];
          });
          write(x + NG * r, v, T(0));
        });
      }
    }
  }
}

// ------------------------------------------------------------ diagonal
template <int DIM, int K>
__global__ void __launch_bounds__(256) level_diag_kernel(LevelArgs a, double* __restrict__ dinv) {
  using G = Geo<DIM, K>;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = idx / G::NOWN;
  const int lane = (int)(idx % G::NOWN);
  if (g >= a.n_groups) return;
  const uint64_t st = a.state[g];
  constexpr int NO = G::NO;
  int i[3] = {lane % NO, DIM > 1 ? (lane / NO) % NO : 0, DIM > 2 ? lane / (NO * NO) : 0};
  int lo_o[3] = {i[0] == 0 ? -1 : 0, DIM > 1 && i[1] == 0 ? -1 : 0, DIM > 2 && i[2] == 0 ? -1 : 0};
  int hi_o[3] = {0, 0, 0};
  const int64_t slot = g * G::NOWN + lane;
  if (node_class<DIM>(st, lo_o, hi_o) != 1) {
    dinv[slot] = 0.0;
    return;
  }
  double diag = 0.0;
  for (int bz = 0; bz < (lo_o[2] ? 2 : 1); ++bz)
    for (int by = 0; by < (lo_o[1] ? 2 : 1); ++by)
      for (int bx = 0; bx < (lo_o[0] ? 2 : 1); ++bx) {
        int ni = nbi<DIM>(-bx, -by, -bz);
        if (state_of(st, ni) != kStateRefined) continue;
        double c = a.coeff[a.nbr[g * G::NNB + ni]];
        int e[3] = {bx ? 2 * K : i[0], by ? 2 * K : i[1], bz ? 2 * K : i[2]};
        double md[3], kd[3];
        for (int d = 0; d < 3; ++d) {
          md[d] = bext<K, false>(e[d], K + i[d]);
          kd[d] = bext<K, true>(e[d], K + i[d]);
        }
        double s = 0.0;
        for (int dir = 0; dir < DIM; ++dir) {
          double t = a.scale[dir];
          for (int d = 0; d < DIM; ++d) t *= (d == dir) ? kd[d] : md[d];
          s += t;
        }
        diag += c * s;
      }
  dinv[slot] = 1.0 / diag;
}

// ----------------------------------------------------------- launchers
// Grid of a persistent kernel: the blocks that are resident at once on the
// current device (looked up once per kernel and device), at most `work`.
template <typename KERN>
static unsigned persistent_grid(KERN kern, int threads, size_t smem, int64_t work) {
  struct Entry {
    const void* fn;
    int device;
    unsigned blocks;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  unsigned blocks = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
      if (e.fn == (const void*)kern && e.device == dev) blocks = e.blocks;
    if (!blocks) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int per_sm = 0, sms = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      blocks = (unsigned)std::max(1, per_sm * sms);
      cache.push_back({(const void*)kern, dev, blocks});
    }
  }
  return (unsigned)std::min<int64_t>(work, blocks);
}

template <typename T, int DIM, int K, int MODE>
static cudaError_t cheb_launch(const LevelArgs& a, const T* x, const T* xprev, const T* g, const T* dinv,
                               T* out, T c1, T c2, cudaStream_t s) {
  bool singles_done = false;
  if constexpr (DIM == 3) {
    if (a.n_bricks_all > 0) {  // full and partial bricks
      if constexpr (std::is_same<T, float>::value && K == 2) {
        // the single groups of the level run in the same launch, after the bricks
        const int64_t chunks = (a.n_uniform + BrickQ2::WARPS - 1) / BrickQ2::WARPS;
        singles_done = true;
        auto kern = a.iso ? level_cheb_brick_q2_kernel<MODE, true> : level_cheb_brick_q2_kernel<MODE, false>;
        const unsigned grid = persistent_grid(kern, BrickQ2::TB, BrickQ2::bytes(), a.n_bricks_all + chunks);
        kern<<<grid, BrickQ2::TB, BrickQ2::bytes(), s>>>(a, chunks, x, xprev, g, out, c1, c2);
        GMG_COUNT_LAUNCH();
      } else if constexpr (std::is_same<T, float>::value) {
        const size_t sm = Brick2S<K>::bytes();
        // set once, thread-safe (function-local static)
        static const bool init = [&] {
          cudaFuncSetAttribute(level_cheb_brick_f2_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sm);
          return true;
        }();
        (void)init;
        level_cheb_brick_f2_kernel<K, MODE><<<(unsigned)a.n_bricks_all, Brick2S<K>::TB, sm, s>>>(a, x, xprev, g,
                                                                                                 out, c1, c2);
        GMG_COUNT_LAUNCH();
      } else if (a.iso) {
        // FP64 on cubic cells: the split-integer brick kernel
        const size_t sm = BrickI<K>::bytes();
        static const bool init = [&] {
          cudaFuncSetAttribute(level_cheb_brick_int_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sm);
          return true;
        }();
        (void)init;
        level_cheb_brick_int_kernel<K, MODE><<<(unsigned)a.n_bricks_all, BrickG<K>::TB, sm, s>>>(a, x, xprev, g,
                                                                                                 out, c1, c2);
        GMG_COUNT_LAUNCH();
      } else {
        const size_t sm = BrickSmem<T, K>::bytes();
        // set once, thread-safe (function-local static)
        static const bool init = [&] {
          cudaFuncSetAttribute(level_cheb_brick_kernel<T, K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sm);
          return true;
        }();
        (void)init;
        level_cheb_brick_kernel<T, K, MODE><<<(unsigned)a.n_bricks_all, BrickG<K>::TB, sm, s>>>(a, x, xprev, g, out,
                                                                                               c1, c2);
        GMG_COUNT_LAUNCH();
      }
    }
  }
  if constexpr (DIM == 3 && std::is_same<T, double>::value) {
    if (a.n_uniform > 0 && !singles_done && a.iso) {
      // FP64 single groups on cubic cells: the split-integer team kernel
      using SI = SingleI<K>;
      static const bool init = [&] {
        cudaFuncSetAttribute(level_cheb_single_int_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SI::bytes());
        return true;
      }();
      (void)init;
      level_cheb_single_int_kernel<K, MODE><<<(unsigned)((a.n_uniform + SI::TPB - 1) / SI::TPB), 256, SI::bytes(),
                                              s>>>(a, x, xprev, g, out, c1, c2);
      GMG_COUNT_LAUNCH();
      singles_done = true;
    }
  }
  if (a.n_uniform > 0 && !singles_done) {
    using F = Fast<DIM, K>;
    const size_t sm = FastSmem<T, DIM, K>::bytes();
    // set once, thread-safe (function-local static)
    static const bool init = [&] {
      cudaFuncSetAttribute(level_cheb_fast_kernel<T, DIM, K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      return true;
    }();
    (void)init;
    dim3 grid((unsigned)((a.n_uniform + F::TPB - 1) / F::TPB));
    level_cheb_fast_kernel<T, DIM, K, MODE><<<grid, 256, sm, s>>>(a, x, xprev, g, out, c1, c2);
    GMG_COUNT_LAUNCH();
  }
  if constexpr (DIM == 3) {
    if (a.n_jump > 0) {
      using F = Fast<3, K>;
      const size_t sm = JumpSmem<T, K>::bytes();
      static const bool initj = [&] {
        cudaFuncSetAttribute(level_cheb_jump_kernel<T, K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        return true;
      }();
      (void)initj;
      dim3 grid((unsigned)((a.n_jump + F::TPB - 1) / F::TPB));
      level_cheb_jump_kernel<T, K, MODE><<<grid, 256, sm, s>>>(a, x, xprev, g, dinv, out, c1, c2);
      GMG_COUNT_LAUNCH();
    }
    return cudaGetLastError();
  }
  if (a.n_jump > 0) {
    using G = Geo<DIM, K>;
    const size_t sm = ChebSmem<T, DIM, K>::bytes() + 16;
    // set once, thread-safe (function-local static)
    static const bool init = [&] {
      cudaFuncSetAttribute(level_cheb_kernel<T, DIM, K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      return true;
    }();
    (void)init;
    dim3 grid((unsigned)((a.n_jump + G::GPB - 1) / G::GPB));
    level_cheb_kernel<T, DIM, K, MODE><<<grid, G::GPB * G::TEAM, sm, s>>>(a, x, xprev, g, dinv, out, c1, c2);
    GMG_COUNT_LAUNCH();
  }
  return cudaGetLastError();
}

template <typename T, int DIM, int K>
static cudaError_t cheb_dispatch(const LevelArgs& a, const T* x, const T* xprev, const T* g,
                                 const T* dinv, T* out, T c1, T c2, bool apply_only,
                                 cudaStream_t s) {
  if (a.n_groups == 0) return cudaSuccess;
  return apply_only ? cheb_launch<T, DIM, K, 0>(a, x, xprev, g, dinv, out, c1, c2, s)
                    : cheb_launch<T, DIM, K, 1>(a, x, xprev, g, dinv, out, c1, c2, s);
}

template <typename T>
cudaError_t launch_level_cheb(int dim, int k, const LevelArgs& a, const T* x, const T* xprev,
                              const T* g, const T* dinv, T* out, T c1, T c2, bool apply_only,
                              cudaStream_t s) {
  if (dim == 3 && k == 2) return cheb_dispatch<T, 3, 2>(a, x, xprev, g, dinv, out, c1, c2, apply_only, s);
  if (dim == 3 && k == 1) return cheb_dispatch<T, 3, 1>(a, x, xprev, g, dinv, out, c1, c2, apply_only, s);
  if (dim == 2 && k == 2) return cheb_dispatch<T, 2, 2>(a, x, xprev, g, dinv, out, c1, c2, apply_only, s);
  if (dim == 2 && k == 1) return cheb_dispatch<T, 2, 1>(a, x, xprev, g, dinv, out, c1, c2, apply_only, s);
  return cudaErrorInvalidValue;
}

template <typename T, int DIM, int K>
static cudaError_t res_dispatch(const LevelArgs& a, const T* u, const T* g, T* gc, cudaStream_t s) {
  using F = Fast<DIM, K>;
  if (a.n_groups == 0) return cudaSuccess;
  // FP32 (FP64: cubic cells), above level 1, every group of the level in a
  // brick and no refinement-edge nodes: one brick pass for residual and
  // restriction.  (The brick pass assigns each fine node's whole residual to
  // the brick owning it, the per-group kernel splits g between the groups
  // touching a node and takes each group's own cells' A u: the two do not mix
  // on one level.)
  const bool bricks = DIM == 3 && (std::is_same<T, float>::value || a.iso) && a.level >= 2 && a.n_bricks > 0 &&
                      a.n_rest == 0 && a.no_ghosts;
  // deterministic mode: one launch per colour of bricks (groups), which share
  // no coarse node, in a fixed colour order
  const bool det = a.deterministic && a.n_brick_colors > 0;
  if constexpr (DIM == 3 && std::is_same<T, float>::value) {
    if (bricks) {
      const size_t smb = Brick2S<K>::bytes();
      static const bool initb = [&] {
        cudaFuncSetAttribute(level_cheb_brick_f2_kernel<K, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
        return true;
      }();
      (void)initb;
      for (int c = 0; c < (det ? a.n_brick_colors : 1); ++c) {
        LevelArgs ac = a;
        int64_t nb = a.n_bricks;
        if (det) {
          ac.bricks = a.bricks + a.brick_off[c] * 64;
          ac.brick_cnb = a.brick_cnb + a.brick_off[c] * 27;
          nb = a.brick_off[c + 1] - a.brick_off[c];
        }
        if (nb == 0) continue;
        level_cheb_brick_f2_kernel<K, 2><<<(unsigned)nb, Brick2S<K>::TB, smb, s>>>(ac, u, nullptr, g, gc, 0.f, 0.f);
        GMG_COUNT_LAUNCH();
      }
    }
  } else if constexpr (DIM == 3) {
    if (bricks) {  // FP64 on cubic cells: the split-integer brick kernel
      const size_t smb = BrickI<K>::bytes();
      static const bool initb = [&] {
        cudaFuncSetAttribute(level_cheb_brick_int_kernel<K, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
        return true;
      }();
      (void)initb;
      for (int c = 0; c < (det ? a.n_brick_colors : 1); ++c) {
        LevelArgs ac = a;
        int64_t nb = a.n_bricks;
        if (det) {
          ac.bricks = a.bricks + a.brick_off[c] * 64;
          ac.brick_cnb = a.brick_cnb + a.brick_off[c] * 27;
          nb = a.brick_off[c + 1] - a.brick_off[c];
        }
        if (nb == 0) continue;
        level_cheb_brick_int_kernel<K, 2><<<(unsigned)nb, BrickG<K>::TB, smb, s>>>(ac, u, nullptr, g, gc, 0.0, 0.0);
        GMG_COUNT_LAUNCH();
      }
    }
  }
  const int32_t* list = bricks ? a.list_rest : nullptr;
  const int64_t n = bricks ? a.n_rest : a.n_groups;
  if (n == 0) return cudaGetLastError();
  const size_t sm = RestrictSmem<T, DIM, K>::bytes();
  // set once, thread-safe (function-local static)
  static const bool init = [&] {
    cudaFuncSetAttribute(level_residual_restrict_kernel<T, DIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return true;
  }();
  (void)init;
  if (a.deterministic && a.n_group_colors > 0 && !bricks) {
    for (int c = 0; c < a.n_group_colors; ++c) {
      const int64_t nc = a.group_off[c + 1] - a.group_off[c];
      if (nc == 0) continue;
      level_residual_restrict_kernel<T, DIM, K><<<(unsigned)((nc + F::TPB - 1) / F::TPB), 256, sm, s>>>(
          a, u, g, gc, a.list_color + a.group_off[c], nc);
      GMG_COUNT_LAUNCH();
    }
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((n + F::TPB - 1) / F::TPB));
  level_residual_restrict_kernel<T, DIM, K><<<grid, 256, sm, s>>>(a, u, g, gc, list, n);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_level_residual_restrict(int dim, int k, const LevelArgs& a, const T* u,
                                           const T* g, T* gc, cudaStream_t s) {
  if (dim == 3 && k == 2) return res_dispatch<T, 3, 2>(a, u, g, gc, s);
  if (dim == 3 && k == 1) return res_dispatch<T, 3, 1>(a, u, g, gc, s);
  if (dim == 2 && k == 2) return res_dispatch<T, 2, 2>(a, u, g, gc, s);
  if (dim == 2 && k == 1) return res_dispatch<T, 2, 1>(a, u, g, gc, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------- prolongation, 2x2x2 bricks
// The eight groups of a brick at level l >= 2 are the children of the eight
// cells of one sibling group at level l-1, so the brick's (4K+1)^3 fine nodes
// are the tensor-product embedding of that group's (2K+1)^3 coarse nodes:
// three 1-D passes shared by the eight groups.  Each fine node is written by
// the brick group whose lattice holds it with the smallest offset, with that
// group's add / set masks, exactly as the per-group kernel would.

template <typename T, int K>
struct ProBrick {
  static constexpr int NO = 2 * K, NC = 2 * K + 1, NF = 4 * K + 1, NG = 2 * K + 1;
  static constexpr int NOWN = NO * NO * NO;
  static constexpr int TB = 128;
  static constexpr int C = NC * NC * NC, PX = NC * NC * NF, PY = NC * NF * NF;
  static constexpr size_t HEAD = 1024;  // masks (256 B), brick table (256 B), coarse neighbours (108 B)
  static constexpr size_t bytes() { return HEAD + (size_t)(C + PX + PY) * sizeof(T); }
};

template <typename T, int K>
__global__ void __launch_bounds__(ProBrick<T, K>::TB)
level_prolongate_brick_kernel(LevelArgs a, const T* __restrict__ uc, T* __restrict__ u, T* __restrict__ u2) {
  using P = ProBrick<T, K>;
  constexpr int NO = P::NO, NC = P::NC, NF = P::NF, NG = P::NG, TB = P::TB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* masks = reinterpret_cast<uint64_t*>(smem_raw);     // 8 groups x (add0, add1, set0, set1)
  int32_t* tab = reinterpret_cast<int32_t*>(masks + 32);
  int32_t* cnb = tab + 64;                                       // 27 neighbours of the coarse group
  T* C = reinterpret_cast<T*>(smem_raw + P::HEAD);
  T* PXa = C + P::C;
  T* PYa = PXa + P::PX;
  const int tid = threadIdx.x;
  const int64_t br = blockIdx.x;
  if (tid < 64) tab[tid] = a.bricks[br * 64 + tid];
  if (tid < 27) cnb[tid] = a.brick_cnb[br * 27 + tid];
  __syncthreads();
  auto own = [&](int gx, int gy, int gz) { return tab[(gx + 1) + 4 * ((gy + 1) + 4 * (gz + 1))]; };
  if (tid < 32) masks[tid] = a.pmask[(int64_t)own((tid >> 2) & 1, (tid >> 3) & 1, (tid >> 4) & 1) * 4 + (tid & 3)];
  // u at the nodes of this thread's z line that lie in a group's own block
  // (the only nodes the update adds to), loaded now so that the update does
  // not wait for them; every fine node has one writer, so the values are
  // current
  static_assert(NF * NF <= TB, "one z line per thread: the prefetched line is the written one");
  T u_pre[NF];
  {
    const int line = tid < NF * NF ? tid : 0;
    const int fx = line % NF, fy = line / NF;
    const int gx = fx / NO > 1 ? 1 : fx / NO, gy = fy / NO > 1 ? 1 : fy / NO;
    const int lx = fx - NO * gx, ly = fy - NO * gy;
    static_for<0, NF>([&](auto r) {
      constexpr int gz = r / NO > 1 ? 1 : r / NO, lz = r - NO * gz;
      u_pre[r] = (tid < NF * NF && lx < NO && ly < NO && lz < NO)
                     ? u[(int64_t)own(gx, gy, gz) * P::NOWN + lx + NO * (ly + NO * lz)]
                     : T(0);
    });
  }
  __syncthreads();
  // coarse nodes of the parent group (its +1 faces from the neighbours)
  for (int i = tid; i < P::C; i += TB) {
    const int cx = i % NC, cy = (i / NC) % NC, cz = i / (NC * NC);
    const int ox = cx == 2 * K, oy = cy == 2 * K, oz = cz == 2 * K;
    const int32_t blk = cnb[(ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1))];
    C[i] = blk >= 0 ? uc[(int64_t)blk * NO * NO * NO + (cx - 2 * K * ox) + NO * ((cy - 2 * K * oy) + NO * (cz - 2 * K * oz))]
                    : T(0);
  }
  __syncthreads();
  // x: lines (cy, cz)
  for (int line = tid; line < NC * NC; line += TB) {
    T c[NC];
    static_for<0, NC>([&](auto j) { c[j] = C[line * NC + j]; });
    static_for<0, NF>([&](auto r) {
      T v = 0;
      static_for<0, NC>([&](auto j) {
        constexpr double e = ebrick<K>(r, j);
        if constexpr (e != 0.0) v += (T)e * c[j];
      });
      PXa[line * NF + r] = v;
    });
  }
  __syncthreads();
  // y: lines (cz, fx); PX [cz][cy][fx] -> PY [cz][fy][fx]
  for (int line = tid; line < NC * NF; line += TB) {
    const int cz = line / NF, fx = line % NF;
    T c[NC];
    static_for<0, NC>([&](auto j) { c[j] = PXa[(cz * NC + j) * NF + fx]; });
    static_for<0, NF>([&](auto r) {
      T v = 0;
      static_for<0, NC>([&](auto j) {
        constexpr double e = ebrick<K>(r, j);
        if constexpr (e != 0.0) v += (T)e * c[j];
      });
      PYa[(cz * NF + r) * NF + fx] = v;
    });
  }
  __syncthreads();
  // z: lines (fx, fy), then write
  for (int line = tid; line < NF * NF; line += TB) {
    const int fx = line % NF, fy = line / NF;
    T c[NC];
    static_for<0, NC>([&](auto j) { c[j] = PYa[(j * NF + fy) * NF + fx]; });
    const int bx = fx / NO, by = fy / NO;                 // storage block offsets 0..2
    const int gx = bx > 1 ? 1 : bx, gy = by > 1 ? 1 : by;  // writing group
    const int lx = fx - NO * gx, ly = fy - NO * gy;        // its lattice position 0..2K
    static_for<0, NF>([&](auto r) {
      T v = 0;
      static_for<0, NC>([&](auto j) {
        constexpr double e = ebrick<K>(r, j);
        if constexpr (e != 0.0) v += (T)e * c[j];
      });
      constexpr int bz = r / NO, gz = bz > 1 ? 1 : bz, lz = r - NO * gz;
      const int gsel = gx + 2 * (gy + 2 * gz);
      const int n = lx + NG * (ly + NG * lz);
      const uint64_t bit = 1ull << (n & 63);
      if (masks[gsel * 4 + (n >> 6)] & bit) {
        u[(int64_t)own(gx, gy, gz) * P::NOWN + lx + NO * (ly + NO * lz)] = u_pre[r] + v;
      } else if (masks[gsel * 4 + 2 + (n >> 6)] & bit) {
        const int32_t blk = tab[(bx + 1) + 4 * ((by + 1) + 4 * (bz + 1))];
        const int64_t s = (int64_t)blk * P::NOWN + (fx - NO * bx) + NO * ((fy - NO * by) + NO * (r - NO * bz));
        u[s] = v;
        u2[s] = v;
      }
    });
  }
}

template <typename T, int DIM, int K>
static cudaError_t pro_dispatch(const LevelArgs& a, const T* uc, T* u, T* u2, cudaStream_t s) {
  using F = Fast<DIM, K>;
  if (a.n_groups == 0) return cudaSuccess;
  // bricks above level 1 (whose parents form one coarse group) take the brick
  // kernel, the other groups the per-group kernel
  const bool bricks = DIM == 3 && a.level >= 2 && a.n_bricks > 0;
  if constexpr (DIM == 3) {
    if (bricks) {
      const size_t sm = ProBrick<T, K>::bytes();
      // set once, thread-safe (function-local static)
      static const bool init = [&] {
        cudaFuncSetAttribute(level_prolongate_brick_kernel<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
        return true;
      }();
      (void)init;
      level_prolongate_brick_kernel<T, K><<<(unsigned)a.n_bricks, ProBrick<T, K>::TB, sm, s>>>(a, uc, u, u2);
      GMG_COUNT_LAUNCH();
    }
  }
  const int32_t* list = bricks ? a.list_rest : nullptr;
  const int64_t n = bricks ? a.n_rest : a.n_groups;
  if (n == 0) return cudaGetLastError();
  const size_t sm = ProlongSmem<T, DIM, K>::bytes();
  // set once, thread-safe (function-local static)
  static const bool init = [&] {
    cudaFuncSetAttribute(level_prolongate_kernel<T, DIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return true;
  }();
  (void)init;
  dim3 grid((unsigned)((n + F::TPB - 1) / F::TPB));
  level_prolongate_kernel<T, DIM, K><<<grid, 256, sm, s>>>(a, uc, u, u2, list, n);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_level_prolongate(int dim, int k, const LevelArgs& a, const T* uc, T* u, T* u2,
                                    cudaStream_t s) {
  if (dim == 3 && k == 2) return pro_dispatch<T, 3, 2>(a, uc, u, u2, s);
  if (dim == 3 && k == 1) return pro_dispatch<T, 3, 1>(a, uc, u, u2, s);
  if (dim == 2 && k == 2) return pro_dispatch<T, 2, 2>(a, uc, u, u2, s);
  if (dim == 2 && k == 1) return pro_dispatch<T, 2, 1>(a, uc, u, u2, s);
  return cudaErrorInvalidValue;
}

template <int DIM, int K>
static cudaError_t diag_dispatch(const LevelArgs& a, double* d, cudaStream_t s) {
  using G = Geo<DIM, K>;
  int64_t n = a.n_groups * G::NOWN;
  if (n == 0) return cudaSuccess;
  level_diag_kernel<DIM, K><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, d);
  GMG_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t launch_level_diag(int dim, int k, const LevelArgs& a, double* d, cudaStream_t s) {
  if (dim == 3 && k == 2) return diag_dispatch<3, 2>(a, d, s);
  if (dim == 3 && k == 1) return diag_dispatch<3, 1>(a, d, s);
  if (dim == 2 && k == 2) return diag_dispatch<2, 2>(a, d, s);
  if (dim == 2 && k == 1) return diag_dispatch<2, 1>(a, d, s);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_level_cheb<float>(int, int, const LevelArgs&, const float*, const float*,
                                              const float*, const float*, float*, float, float, bool,
                                              cudaStream_t);
template cudaError_t launch_level_cheb<double>(int, int, const LevelArgs&, const double*, const double*,
                                               const double*, const double*, double*, double, double,
                                               bool, cudaStream_t);
template cudaError_t launch_level_residual_restrict<float>(int, int, const LevelArgs&, const float*,
                                                           const float*, float*, cudaStream_t);
template cudaError_t launch_level_residual_restrict<double>(int, int, const LevelArgs&, const double*,
                                                            const double*, double*, cudaStream_t);
template cudaError_t launch_level_prolongate<float>(int, int, const LevelArgs&, const float*, float*,
                                                    float*, cudaStream_t);
template cudaError_t launch_level_prolongate<double>(int, int, const LevelArgs&, const double*,
                                                     double*, double*, cudaStream_t);

}  // namespace gmg
