// Hot-path kernels: the matrix-free element-by-element operator (Sec. 4.6
// "Matrix-Free EBE Formulation": K u = sum_e A_e^T K_e A_e u_e), applied node by node, the
// damped block-Jacobi / Chebyshev smoother (Sec. 4.6 "Parallel Smoothing" update form
// u <- u + omega D^-1 r, all nodes at once), the trilinear transfers (App. E.2, restriction
// written as a gather so every sum has a fixed order), the coarsest solve (Alg. 1), the
// element-energy reduction for C^H (App. F.1/F.2) and the vector kernels of the solver.
//
// Node-centric operator. For node n with octant mask m(n),
//     (K u)_n = sum_{d in {-1,0,1}^3} S_n(d) u_{n+d},
//     S_n(d) = sum_{a in {0,1}^3, a+d in {0,1}^3} [element n-a active] K(n-a)[a, a+d],
// i.e. the node's rows of every active incident element (a = local index of n in element
// n - a). At level 0 every element carries the same K_e, which is passed in the kernel's
// parameter (constant) bank, so the D x D blocks S_n(d) are formed in registers from the
// mask bits and K_e operands; coarser levels read each incident element's Galerkin matrix.
// One 64-thread block owns one 4^3 brick and stages the brick plus a one-node halo
// (6^3 nodes x C values) in shared memory; every output sum runs in a fixed order.
#include <cstring>
#include <type_traits>

#include "stencil.cuh"

namespace gmt {

// ------------------------------------------------------------------ packed FP32 pairs
// Blackwell f32x2 arithmetic: one instruction on two FP32 values held in a 64-bit register
// pair, each lane rounded exactly as the scalar instruction. The stencils pair the load
// cases m = (2k, 2k + 1), which sit next to each other in the 16-byte tile groups.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2_t r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {  // a * b + c
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// ------------------------------------------------------------------ parameters
template <typename A, int D, int M>
struct FineC {
  A Ke[64 * D * D];         // (8D) x (8D)
  A Fe[8 * D * M];          // K_e x0, (8D) x M
  A Sf[27 * D * D];         // S_n(d) of a node whose 8 incident elements are all active
  f2_t Sf2[27 * D * D];     // FP32: Sf entries duplicated into packed pairs
};

template <typename TS, typename A, int D, int M>
struct StArgs {
  const int* nbr;
  const uint8_t* mask;
  const int* kidx;
  const A* kmat;
  const A* dinv;
  const TS* u;
  const TS* f;
  const TS* dprev;
  const TS* aux;
  TS* out;
  TS* dout;
  double* part;
  A omega, c1, c2;
  int colour;
  FineC<A, D, M> fc;
};

template <typename T> struct ArithOf { using type = float; };
template <> struct ArithOf<double> { using type = double; };

// ------------------------------------------------------------------ block reduction helper
// 64-thread block: reduce K <= 32 values per thread into out[K] (fixed order). Each warp
// reduces all K values at once by a transposing butterfly: with the values padded to
// P = 2^p >= K, the step at lane offset o halves the values a lane holds (it keeps one half
// and adds its partner's copy of that half, received for the other), so after p steps each
// lane holds one column summed over P lanes; plain xor steps finish the sum over the warp.
// That is P - 1 + (5 - p) shuffles instead of 5 K. Lanes and warps add in the values' own
// type T (FP32 kernels keep FP64 off the per-element path, where B300's FP64 rate is 1/64
// of FP32); the two warp sums are combined in FP64.
template <int K, typename T>
__device__ __forceinline__ void block_partial_64(T (&v)[K], double* __restrict__ out) {
  static_assert(K >= 1 && K <= 32, "at most 32 values per thread");
  constexpr int P = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
  constexpr int LP = P == 1 ? 0 : P == 2 ? 1 : P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : 5;
  __shared__ double red[2][P];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x[P];
#pragma unroll
  for (int i = 0; i < P; ++i) x[i] = i < K ? v[i] : T(0);
  int col = 0;
#pragma unroll
  for (int s = 0; s < LP; ++s) {
    const int h = P >> (s + 1), o = 16 >> s;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? x[i] : x[i + h];
      const T keep = up ? x[i + h] : x[i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    if (up) col += h;
  }
#pragma unroll
  for (int o = 16 >> LP; o > 0; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
  if ((lane & ((32 >> LP) - 1)) == 0) red[w][col] = (double)x[0];
  __syncthreads();
  if (threadIdx.x < K) out[threadIdx.x] = red[0][threadIdx.x] + red[1][threadIdx.x];
}

// symmetric-positive D x D inverse (D = 1 or 3)
template <typename A, int D>
__device__ __forceinline__ void inv_block(const A (&Bk)[D * D], A (&I)[D * D]) {
  if constexpr (D == 1) {
    I[0] = A(1) / Bk[0];
  } else {
    A c00 = Bk[4] * Bk[8] - Bk[5] * Bk[7], c01 = Bk[5] * Bk[6] - Bk[3] * Bk[8],
      c02 = Bk[3] * Bk[7] - Bk[4] * Bk[6];
    A id = A(1) / (Bk[0] * c00 + Bk[1] * c01 + Bk[2] * c02);
    I[0] = c00 * id;
    I[1] = (Bk[2] * Bk[7] - Bk[1] * Bk[8]) * id;
    I[2] = (Bk[1] * Bk[5] - Bk[2] * Bk[4]) * id;
    I[3] = c01 * id;
    I[4] = (Bk[0] * Bk[8] - Bk[2] * Bk[6]) * id;
    I[5] = (Bk[2] * Bk[3] - Bk[0] * Bk[5]) * id;
    I[6] = c02 * id;
    I[7] = (Bk[1] * Bk[6] - Bk[0] * Bk[7]) * id;
    I[8] = (Bk[0] * Bk[4] - Bk[1] * Bk[3]) * id;
  }
}

// level-0 diagonal block D_n = sum_{a in mask} K_e[a, a]
template <typename A, int D, int M>
__device__ __forceinline__ void fine_diag_inv(const FineC<A, D, M>& fc, unsigned mk,
                                              A (&I)[D * D]) {
  A Bk[D * D];
#pragma unroll
  for (int q = 0; q < D * D; ++q) Bk[q] = A(0);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const A bit = ((mk >> a) & 1u) ? A(1) : A(0);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) Bk[i * D + j] += bit * fc.Ke[(a * D + i) * (8 * D) + a * D + j];
  }
  inv_block<A, D>(Bk, I);
}

// ------------------------------------------------------------------ tile staging
// Thread t of a 64-thread block owns brick node (lx, ly, lz) = (t & 3, t >> 4, (t >> 2) & 3):
// the 8 lanes of a quarter-warp then cover (lx, lz) in 4 x 2, whose 16-byte tile entries
// fall in distinct shared-memory banks.
__device__ __forceinline__ int own_local(int t) { return (t & 3) + 4 * (t >> 4) + 16 * ((t >> 2) & 3); }
__device__ __forceinline__ int own_q0(int t) {
  return ((t & 3) + 1) + 6 * ((t >> 4) + 1) + 36 * (((t >> 2) & 3) + 1);
}

// 16-byte shared-memory vector of the arithmetic type
template <typename A> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

// node-stencil layout of the coarse levels: 27 * DD coefficients per node in 16-byte groups
template <typename A>
__host__ __device__ constexpr int node_stencil_groups(int DD) {
  return (27 * DD + Vec16<A>::n - 1) / Vec16<A>::n;
}
__host__ __device__ __forceinline__ int64_t node_stencil_index(int64_t slot, int c, int groups,
                                                             int W) {
  return (slot >> 6) * ((int64_t)groups * 64 * W) + (int64_t)(c / W) * (64 * W) +
         (slot & 63) * W + c % W;
}

template <typename A>
__device__ __forceinline__ void vec_put(typename Vec16<A>::type& w, int k, A x) {
  if constexpr (Vec16<A>::n == 4) {
    if (k == 0) w.x = x; else if (k == 1) w.y = x; else if (k == 2) w.z = x; else w.w = x;
  } else {
    if (k == 0) w.x = x; else w.y = x;
  }
}
template <typename A>
__device__ __forceinline__ A vec_get(const typename Vec16<A>::type& w, int k) {
  if constexpr (Vec16<A>::n == 4) {
    return k == 0 ? w.x : (k == 1 ? w.y : (k == 2 ? w.z : w.w));
  } else {
    return k == 0 ? w.x : w.y;
  }
}

// Stage the brick (own node of every thread, kept in registers) plus its one-node halo
// (152 of the 216 tile positions, gathered from the 26 neighbour bricks) in shared memory
// as tile[g][q] = 16-byte groups of values; index arithmetic once per tile position.
template <typename TS, typename A, int C>
__device__ __forceinline__ void stage_tile(const TS* __restrict__ u, int64_t b, int t,
                                           const int* nb, typename Vec16<A>::type* tile,
                                           A (&self)[C]) {
  using V = typename Vec16<A>::type;
  constexpr int NV = Vec16<A>::n, G = (C + NV - 1) / NV;
  const int q0 = own_q0(t);
  const TS* own = u + b * (64 * C) + own_local(t);
#pragma unroll
  for (int v = 0; v < C; ++v) self[v] = load_as<A>(own + v * 64);
#pragma unroll
  for (int g = 0; g < G; ++g) {
    V w;
#pragma unroll
    for (int k = 0; k < NV; ++k) vec_put<A>(w, k, g * NV + k < C ? self[g * NV + k] : A(0));
    tile[g * 216 + q0] = w;
  }
  for (int q = t; q < 216; q += 64) {
    const int tx = q % 6, ty = (q / 6) % 6, tz = q / 36;
    if (tx >= 1 && tx <= 4 && ty >= 1 && ty <= 4 && tz >= 1 && tz <= 4) continue;
    const int bx = tx == 0 ? 0 : (tx == 5 ? 2 : 1);
    const int by = ty == 0 ? 0 : (ty == 5 ? 2 : 1);
    const int bz = tz == 0 ? 0 : (tz == 5 ? 2 : 1);
    const int nbi = nb[bz * 9 + by * 3 + bx];
    A vals[C];
    if (nbi >= 0) {
      const TS* src = u + (int64_t)nbi * (64 * C) + ((tx + 3) & 3) + 4 * ((ty + 3) & 3) +
                      16 * ((tz + 3) & 3);
#pragma unroll
      for (int v = 0; v < C; ++v) vals[v] = load_as<A>(src + v * 64);
    } else {
#pragma unroll
      for (int v = 0; v < C; ++v) vals[v] = A(0);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      V w;
#pragma unroll
      for (int k = 0; k < NV; ++k) vec_put<A>(w, k, g * NV + k < C ? vals[g * NV + k] : A(0));
      tile[g * 216 + q] = w;
    }
  }
}

// ------------------------------------------------------------------ the stencil kernel
// KIND 0: level 0, S_n(d) formed from the octant mask and K_e (parameter bank); warps whose
//         32 nodes all have full masks use the precomputed full stencil instead.
// KIND 1: coarse levels, S_n(d) read from the per-node assembled stencil, stored
//         brick-major as [brick][27 * D * D][64] so each coefficient load is coalesced.
// ST_APPLY uses the difference form sum_{d != 0} S_n(d) (u_{n+d} - u_n) (rows of K sum to
// zero): the differences of a smooth Krylov direction are small, which keeps the FP32
// product accurate (about 20x closer to the FP64 product than the direct form on V-cycle
// output). It annihilates translations exactly, so the mixed-precision solver keeps its
// residual and preconditioned directions free of translations (see solver.cu).
// SUMS (smoother modes): also write per-block partials [2M + C]: f . out per case, aux . out
// per case (0 without aux) and out per value over active nodes (the V-cycle's last sweep:
// r.z, (K p).z and the mean of z for the Krylov step, without another pass over vectors).
template <typename TS, typename A, int D, int M, int KIND, int MODE, bool SUMS = false>
__global__ void __launch_bounds__(64)
    k_stencil(const __grid_constant__ StArgs<TS, A, D, M> p) {
  using V = typename Vec16<A>::type;
  constexpr int C = D * M, R = 8 * D, DD = D * D;
  constexpr int NV = Vec16<A>::n, G = (C + NV - 1) / NV;
  constexpr bool DIFF = MODE == ST_APPLY;
  __shared__ V tile[G * 216];
  __shared__ int nb[27];
  const int t = threadIdx.x;
  const int64_t b = blockIdx.x;
  if (t < 27) nb[t] = p.nbr[b * 27 + t];
  __syncthreads();
  // level-0 smoother sweeps and residuals: the right-hand side of this thread's node is
  // loaded before the staging so that its latency overlaps the stencil instead of
  // following it (measured: the level-0 sweep 20 % faster; coarse levels, with more
  // registers in use, are left as they are)
  constexpr bool PREF = KIND == 0 && (MODE == ST_JACOBI || MODE == ST_CHEB || MODE == ST_RESID);
  A fpre[PREF ? C : 1];
  if constexpr (PREF) {
    if (p.f != nullptr) {
      const TS* fo = p.f + b * (64 * C) + own_local(t);
#pragma unroll
      for (int v = 0; v < C; ++v) fpre[v] = load_as<A>(fo + v * 64);
    }
  }
  A self[C];
  stage_tile<TS, A, C>(p.u, b, t, nb, tile, self);
  __syncthreads();
  const int q0 = own_q0(t);
  const int loc = own_local(t);
  const int64_t slot = b * 64 + loc;
  const unsigned mk = p.mask[slot];
  // warp vote taken by every lane (before any divergence): all 32 nodes have full masks
  const bool warp_full = __all_sync(0xffffffffu, mk == 0xffu);
  A acc[C];
#pragma unroll
  for (int v = 0; v < C; ++v) acc[v] = A(0);
  // FP32 with an even number of cases: accumulate in packed pairs of cases
  constexpr bool PK = sizeof(A) == 4 && M % 2 == 0;
  constexpr int H = M / 2, CP = PK ? C / 2 : 1;
  f2_t acc2[CP], self2[CP];
  if constexpr (PK) {
#pragma unroll
    for (int k = 0; k < CP; ++k) {
      acc2[k] = 0ull;
      self2[k] = f2_pack((float)self[2 * k], (float)self[2 * k + 1]);
    }
  }
  // neighbour d's contribution with S given as packed duplicated pairs
  auto contribute2 = [&](int d, const f2_t (&S2)[DD]) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    const int q = q0 + dx + 6 * dy + 36 * dz;
    const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(tile);
    f2_t u2[CP];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const ulonglong2 w = t2[g * 216 + q];
      if (2 * g < CP) u2[2 * g] = w.x;
      if (2 * g + 1 < CP) u2[2 * g + 1] = w.y;
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
#pragma unroll
      for (int h2 = 0; h2 < H; ++h2) {
        f2_t x = u2[j * H + h2];
        if constexpr (DIFF) x = f2_sub(x, self2[j * H + h2]);
#pragma unroll
        for (int i = 0; i < D; ++i) acc2[i * H + h2] = f2_fma(S2[i * D + j], x, acc2[i * H + h2]);
      }
    }
  };
  auto contribute_s = [&](int d, const A (&S)[DD]) {
    f2_t S2[DD];
#pragma unroll
    for (int k = 0; k < DD; ++k) S2[k] = f2_pack((float)S[k], (float)S[k]);
    contribute2(d, S2);
  };
  // neighbour d's contribution with the D x D block S
  auto contribute = [&](int d, const A (&S)[DD]) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    const int q = q0 + dx + 6 * dy + 36 * dz;
    A uv[G * NV];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const V w = tile[g * 216 + q];
#pragma unroll
      for (int k = 0; k < NV; ++k) uv[g * NV + k] = vec_get<A>(w, k);
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        A x = uv[j * M + m];
        if constexpr (DIFF) x -= self[j * M + m];
#pragma unroll
        for (int i = 0; i < D; ++i) acc[i * M + m] += S[i * D + j] * x;
      }
    }
  };
  if (mk) {
    if constexpr (KIND == 0) {
      if (warp_full) {
#pragma unroll
        for (int d = 0; d < 27; ++d) {
          if (DIFF && d == 13) continue;
          if constexpr (PK) {
            f2_t S2[DD];
#pragma unroll
            for (int k = 0; k < DD; ++k) S2[k] = p.fc.Sf2[d * DD + k];
            if (d == 13) {  // own node: no shared-memory round trip
#pragma unroll
              for (int j = 0; j < D; ++j)
#pragma unroll
                for (int h2 = 0; h2 < H; ++h2)
#pragma unroll
                  for (int i = 0; i < D; ++i)
                    acc2[i * H + h2] = f2_fma(S2[i * D + j], self2[j * H + h2], acc2[i * H + h2]);
            } else {
              contribute2(d, S2);
            }
          } else {
            A S[DD];
#pragma unroll
            for (int k = 0; k < DD; ++k) S[k] = p.fc.Sf[d * DD + k];
            if (d == 13) {  // own node: no shared-memory round trip
#pragma unroll
              for (int j = 0; j < D; ++j)
#pragma unroll
                for (int m = 0; m < M; ++m)
#pragma unroll
                  for (int i = 0; i < D; ++i) acc[i * M + m] += S[i * D + j] * self[j * M + m];
            } else {
              contribute(d, S);
            }
          }
        }
      } else {
        A bf[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) bf[a] = ((mk >> a) & 1u) ? A(1) : A(0);
#pragma unroll
        for (int d = 0; d < 27; ++d) {
          if (DIFF && d == 13) continue;
          const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
          A S[DD];
#pragma unroll
          for (int k = 0; k < DD; ++k) S[k] = A(0);
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            const int ex = (a & 1) + dx, ey = ((a >> 1) & 1) + dy, ez = (a >> 2) + dz;
            if (ex < 0 || ex > 1 || ey < 0 || ey > 1 || ez < 0 || ez > 1) continue;
            const int bb = ex + 2 * ey + 4 * ez;
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
              for (int j = 0; j < D; ++j)
                S[i * D + j] += bf[a] * p.fc.Ke[(a * D + i) * R + bb * D + j];
          }
          if constexpr (PK) contribute_s(d, S);
          else contribute(d, S);
        }
      }
    } else {
      // coefficient c = d * DD + k of this node sits in 16-byte group c / W (see
      // node_stencil_index); each group is loaded once, when its first coefficient is needed
      constexpr int W = Vec16<A>::n, NGW = node_stencil_groups<A>(DD) * W;
      const A* sten = p.kmat + b * (NGW * 64) + loc * W;
      V cur;
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        A S[DD];
#pragma unroll
        for (int k = 0; k < DD; ++k) {
          const int c = d * DD + k;
          if (c % W == 0) cur = *reinterpret_cast<const V*>(sten + (c / W) * (64 * W));
          S[k] = vec_get<A>(cur, c % W);
        }
        if (DIFF && d == 13) continue;
        if constexpr (PK) contribute_s(d, S);
        else contribute(d, S);
      }
    }
  }
  if constexpr (PK) {
#pragma unroll
    for (int k = 0; k < CP; ++k) {
      float lo, hi;
      f2_unpack(acc2[k], lo, hi);
      acc[2 * k] = (A)lo;
      acc[2 * k + 1] = (A)hi;
    }
  }
  const int64_t base = b * (64 * C) + loc;
  if constexpr (MODE == ST_APPLY) {
    A dots[M];
#pragma unroll
    for (int m = 0; m < M; ++m) dots[m] = A(0);
#pragma unroll
    for (int v = 0; v < C; ++v) {
      p.out[base + v * 64] = store_as<TS>(mk ? acc[v] : A(0));
      if (mk) dots[v % M] += self[v] * acc[v];
    }
    if (p.part) block_partial_64<M, A>(dots, p.part + b * M);
  } else if constexpr (MODE == ST_RESID) {
    A nrm[M];
#pragma unroll
    for (int m = 0; m < M; ++m) nrm[m] = A(0);
#pragma unroll
    for (int v = 0; v < C; ++v) {
      A fv;
      if constexpr (KIND == 0) {
        if (p.f != nullptr) {
          fv = fpre[v];
        } else {  // level-0 load from the mask: f_n = sum_{a in mask} (K_e x0)[a]
          fv = A(0);
          const int i = v / M, m = v % M;
#pragma unroll
          for (int a = 0; a < 8; ++a)
            fv += (((mk >> a) & 1u) ? A(1) : A(0)) * p.fc.Fe[(a * D + i) * M + m];
        }
      } else {
        fv = load_as<A>(p.f + base + v * 64);
      }
      const A r = mk ? fv - acc[v] : A(0);
      p.out[base + v * 64] = store_as<TS>(r);
      nrm[v % M] += r * r;
    }
    if (p.part) block_partial_64<M, A>(nrm, p.part + b * M);
  } else {
    A Iv[DD];
    if (mk) {
      if constexpr (KIND == 0) {
        fine_diag_inv<A, D, M>(p.fc, mk, Iv);
      } else {
#pragma unroll
        for (int k = 0; k < DD; ++k) Iv[k] = p.dinv[slot * DD + k];
      }
    }
    // colour of this node: the parity of its coordinates (bricks start at multiples of 4)
    const int lx = t & 3, ly = t >> 4, lz = (t >> 2) & 3;
    const bool upd = p.colour < 0 || p.colour == (lx & 1) + 2 * (ly & 1) + 4 * (lz & 1);
    A sums[SUMS ? 2 * M + C : 1];
    if constexpr (SUMS) {
#pragma unroll
      for (int k = 0; k < 2 * M + C; ++k) sums[k] = A(0);
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
      A fv[D], r[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        if constexpr (PREF) fv[i] = fpre[i * M + m];
        else fv[i] = load_as<A>(p.f + base + (i * M + m) * 64);
        r[i] = fv[i] - acc[i * M + m];
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        A z = A(0);
#pragma unroll
        for (int j = 0; j < D; ++j) z += Iv[i * D + j] * r[j];
        const int v = i * M + m;
        A o;
        if constexpr (MODE == ST_JACOBI) {
          o = mk ? (upd ? self[v] + p.omega * z : self[v]) : A(0);
        } else {
          const A dn = (p.c1 != A(0) ? p.c1 * load_as<A>(p.dprev + base + v * 64) : A(0)) + p.c2 * z;
          o = mk ? self[v] + dn : A(0);
          if (p.dout) p.dout[base + v * 64] = store_as<TS>(mk ? dn : A(0));
        }
        const TS os = store_as<TS>(o);
        p.out[base + v * 64] = os;
        if constexpr (SUMS) {
          const A ov = load_as<A>(&os);   // the stored value
          sums[m] += mk ? fv[i] * ov : A(0);
          if (p.aux) sums[M + m] += mk ? load_as<A>(p.aux + base + v * 64) * ov : A(0);
          sums[2 * M + v] += ov;
        }
      }
    }
    if constexpr (SUMS) block_partial_64<2 * M + C, A>(sums, p.part + b * (2 * M + C));
  }
}

// per-node assembled stencil of a coarse level: S_n(d) = sum over active elements e = n - a
// with a + d in {0,1}^3 of K(e)[a, a + d], written as [brick][group][64][W]: coefficient
// c = d * D * D + k of a node in 16-byte group c / W (W = 4 floats or 2 doubles), so that a
// thread reads its node's coefficients with one 16-byte load per group and a warp's loads
// are contiguous
// T = float: the FP32 stencils summed from the FP32 element copies (the stencils are FP32
// anyway; FP64 sums would cost 1/64 of the FP32 rate on B300); T = double: FP64 throughout.
// coef (nullable, per slot of the element's origin): element matrices scaled by s_e (level 0
// with densities, where every element shares K_e)
template <typename T, int D>
__global__ void k_node_stencil(int n, int nbx, const int* __restrict__ bxyz,
                               const int* __restrict__ bmap, bool dense, int64_t nslots,
                               const uint8_t* __restrict__ mask, const int* __restrict__ kidx,
                               const T* __restrict__ K, const T* __restrict__ coef,
                               T* __restrict__ S) {
  constexpr int R = 8 * D, MM = R * R, DD = D * D, W = Vec16<T>::n;
  constexpr int G = node_stencil_groups<T>(DD);
  const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslots) return;
  const unsigned mk = mask[sl];
  int x = 0, y = 0, z = 0;
  if (mk) slot_coords(sl, n, dense, bxyz, x, y, z);
  const T* Ka[8];   // element matrix of each incident element (nullptr when inactive)
  T sa[8];          // its scale
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    Ka[a] = nullptr;
    sa[a] = T(1);
    if ((mk >> a) & 1u) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
      const int64_t es = site_slot((x - ax + n) % n, (y - ay + n) % n, (z - az + n) % n, n, nbx,
                                   bmap, dense);
      Ka[a] = K + (int64_t)kidx[es] * MM;
      if (coef) sa[a] = coef[es];
    }
  }
#pragma unroll 1
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    T Sd[DD];
#pragma unroll
    for (int k = 0; k < DD; ++k) Sd[k] = T(0);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
      const int ex = ax + dx, ey = ay + dy, ez = az + dz;
      if (!Ka[a] || ex < 0 || ex > 1 || ey < 0 || ey > 1 || ez < 0 || ez > 1) continue;
      const int bb = ex + 2 * ey + 4 * ez;
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) Sd[i * D + j] += sa[a] * Ka[a][(a * D + i) * R + bb * D + j];
    }
#pragma unroll
    for (int k = 0; k < DD; ++k) S[node_stencil_index(sl, d * DD + k, G, W)] = Sd[k];
  }
}

void build_node_stencils(gmt_hierarchy* h, int level, bool fp64) {
  Level& lv = h->lv[level];
  if (fp64 ? lv.S64 != nullptr : lv.S32 != nullptr) return;
  TraceScope ts(&h->tracer, h->stream, TR_OPS, 0.0);
  const int D = h->mat.D;
  const unsigned g = grid_for(lv.nslots, 128);
  cudaStream_t s = h->stream;
  // level 0 (densities only): every element carries s_e K_e
  const bool fine = level == 0;
  const int* kidx = op_kidx(lv);
  if (fp64) {
    const size_t cnt = (size_t)lv.nslots * node_stencil_groups<double>(D * D) * 2;
    lv.S64 = h->op.alloc<double>(cnt);
    GMT_CUDA(cudaMemsetAsync(lv.S64, 0, cnt * sizeof(double), s));
    const double* K = fine ? h->Ke64 : lv.K64;
    const double* cf = fine ? h->coef64 : nullptr;
    if (D == 3)
      k_node_stencil<double, 3><<<g, 128, 0, s>>>(lv.n, lv.nbx, lv.brick_xyz, lv.brick_map,
                                                  lv.dense, lv.nslots, lv.mask, kidx, K, cf,
                                                  lv.S64);
    else
      k_node_stencil<double, 1><<<g, 128, 0, s>>>(lv.n, lv.nbx, lv.brick_xyz, lv.brick_map,
                                                  lv.dense, lv.nslots, lv.mask, kidx, K, cf,
                                                  lv.S64);
  } else {
    const size_t cnt = (size_t)lv.nslots * node_stencil_groups<float>(D * D) * 4;
    lv.S32 = h->op.alloc<float>(cnt);
    GMT_CUDA(cudaMemsetAsync(lv.S32, 0, cnt * sizeof(float), s));
    const float* K = fine ? h->Ke32 : lv.K32;
    const float* cf = fine ? h->coef32 : nullptr;
    if (D == 3)
      k_node_stencil<float, 3><<<g, 128, 0, s>>>(lv.n, lv.nbx, lv.brick_xyz, lv.brick_map,
                                                 lv.dense, lv.nslots, lv.mask, kidx, K, cf,
                                                 lv.S32);
    else
      k_node_stencil<float, 1><<<g, 128, 0, s>>>(lv.n, lv.nbx, lv.brick_xyz, lv.brick_map,
                                                 lv.dense, lv.nslots, lv.mask, kidx, K, cf,
                                                 lv.S32);
  }
  GMT_LAUNCH_CHECK();
}

// first smoothing step from a zero initial guess: out = scale * D^-1 f
template <typename TS, typename A, int D, int M, int KIND>
__global__ void k_diag(const __grid_constant__ StArgs<TS, A, D, M> p, int64_t nslots) {
  constexpr int C = D * M;
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nslots) return;
  const unsigned mk = p.mask[slot];
  A Iv[D * D];
  if (mk) {
    if constexpr (KIND == 0) {
      fine_diag_inv<A, D, M>(p.fc, mk, Iv);
    } else {
#pragma unroll
      for (int k = 0; k < D * D; ++k) Iv[k] = p.dinv[slot * D * D + k];
    }
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    A f[D];
#pragma unroll
    for (int i = 0; i < D; ++i) f[i] = load_as<A>(p.f + vaddr(slot, i * M + m, C));
#pragma unroll
    for (int i = 0; i < D; ++i) {
      A z = A(0);
#pragma unroll
      for (int j = 0; j < D; ++j) z += Iv[i * D + j] * f[j];
      const A o = mk ? p.omega * z : A(0);
      p.out[vaddr(slot, i * M + m, C)] = store_as<TS>(o);
      if (p.dout) p.dout[vaddr(slot, i * M + m, C)] = store_as<TS>(o);
    }
  }
}

// ------------------------------------------------------------------ float-float residual
template <int D, int M>
struct FFArgs {
  const int* nbr;
  const uint8_t* mask;
  const float* hi;
  const float* lo;
  float* out;
  double* part;
  const float* kmat;   // STORED: per-node stencils [brick][group][64][4]
  const float* f;      // STORED: the level-0 load (slot layout)
  FineC<float, D, M> fc;
};

// r = f - K u at level 0 with u = hi + lo, in difference form
//   (K u)_n = sum_{d != 0} S_n(d) (u_{n+d} - u_n)     (rows of K sum to zero),
// each difference formed as (hi_{n+d} - hi_n) + (lo_{n+d} - lo_n) in FP32: the differences
// of a smooth field are O(1) while u itself grows with N, so FP32 arithmetic on them keeps
// the residual accurate to ~1e-7 of the load without FP64 instructions.
// ZERO: u = 0 (a zero start), r = f without staging or the stencil.
// STORED (element densities): S_n(d) read from the stored per-node stencils and f from the
// stored load, instead of both formed from the octant mask.
template <int D, int M, bool ZERO, bool STORED = false>
__global__ void __launch_bounds__(64) k_resid_ff(const __grid_constant__ FFArgs<D, M> p) {
  using V = float4;
  constexpr int C = D * M, R = 8 * D, G = (C + 3) / 4;
  __shared__ V th[ZERO ? 1 : G * 216];
  __shared__ V tl[ZERO ? 1 : G * 216];
  __shared__ int nb[27];
  const int t = threadIdx.x;
  const int64_t b = blockIdx.x;
  float sh[C], sl[C];
  if constexpr (!ZERO) {
    if (t < 27) nb[t] = p.nbr[b * 27 + t];
    __syncthreads();
    stage_tile<float, float, C>(p.hi, b, t, nb, th, sh);
    stage_tile<float, float, C>(p.lo, b, t, nb, tl, sl);
    __syncthreads();
  }
  const int q0 = own_q0(t), loc = own_local(t);
  const int64_t slot = b * 64 + loc;
  const unsigned mk = p.mask[slot];
  const bool warp_full = !STORED && __all_sync(0xffffffffu, mk == 0xffu);  // every lane votes
  float acc[C];
#pragma unroll
  for (int v = 0; v < C; ++v) acc[v] = 0.f;
  constexpr bool PK = M % 2 == 0;   // packed pairs of cases (f32x2)
  constexpr int H = M / 2, CP = PK ? C / 2 : 1;
  f2_t acc2[CP], sh2[CP], sl2[CP];
  if constexpr (PK && !ZERO) {
#pragma unroll
    for (int k = 0; k < CP; ++k) {
      acc2[k] = 0ull;
      sh2[k] = f2_pack(sh[2 * k], sh[2 * k + 1]);
      sl2[k] = f2_pack(sl[2 * k], sl[2 * k + 1]);
    }
  }
  if (!ZERO && mk) {
    float bf[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) bf[a] = ((mk >> a) & 1u) ? 1.f : 0.f;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      if (d == 13) continue;  // d = 0 carries no difference
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      float S[D * D];
      f2_t S2[D * D];
      if constexpr (STORED) {
        constexpr int NG = node_stencil_groups<float>(D * D) * 4;
        const float* sten = p.kmat + b * (NG * 64) + loc * 4;
#pragma unroll
        for (int k = 0; k < D * D; ++k) {
          const int c = d * D * D + k;
          S[k] = sten[(c / 4) * 256 + c % 4];
        }
        if constexpr (PK) {
#pragma unroll
          for (int k = 0; k < D * D; ++k) S2[k] = f2_pack(S[k], S[k]);
        }
      } else if (warp_full) {
#pragma unroll
        for (int k = 0; k < D * D; ++k) {
          if constexpr (PK) S2[k] = p.fc.Sf2[d * D * D + k];
          else S[k] = p.fc.Sf[d * D * D + k];
        }
      } else {
#pragma unroll
        for (int k = 0; k < D * D; ++k) S[k] = 0.f;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int ex = (a & 1) + dx, ey = ((a >> 1) & 1) + dy, ez = (a >> 2) + dz;
          if (ex < 0 || ex > 1 || ey < 0 || ey > 1 || ez < 0 || ez > 1) continue;
          const int bb = ex + 2 * ey + 4 * ez;
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j)
              S[i * D + j] += bf[a] * p.fc.Ke[(a * D + i) * R + bb * D + j];
        }
        if constexpr (PK) {
#pragma unroll
          for (int k = 0; k < D * D; ++k) S2[k] = f2_pack(S[k], S[k]);
        }
      }
      const int q = q0 + dx + 6 * dy + 36 * dz;
      if constexpr (PK) {
        const ulonglong2* th2 = reinterpret_cast<const ulonglong2*>(th);
        const ulonglong2* tl2 = reinterpret_cast<const ulonglong2*>(tl);
        f2_t du2[CP];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const ulonglong2 wh = th2[g * 216 + q], wl = tl2[g * 216 + q];
          if (2 * g < CP) du2[2 * g] = f2_add(f2_sub(wh.x, sh2[2 * g]), f2_sub(wl.x, sl2[2 * g]));
          if (2 * g + 1 < CP)
            du2[2 * g + 1] = f2_add(f2_sub(wh.y, sh2[2 * g + 1]), f2_sub(wl.y, sl2[2 * g + 1]));
        }
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
          for (int h2 = 0; h2 < H; ++h2)
#pragma unroll
            for (int i = 0; i < D; ++i)
              acc2[i * H + h2] = f2_fma(S2[i * D + j], du2[j * H + h2], acc2[i * H + h2]);
      } else {
        float uh[G * 4], ul[G * 4];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const V wh = th[g * 216 + q], wl = tl[g * 216 + q];
          uh[4 * g] = wh.x; uh[4 * g + 1] = wh.y; uh[4 * g + 2] = wh.z; uh[4 * g + 3] = wh.w;
          ul[4 * g] = wl.x; ul[4 * g + 1] = wl.y; ul[4 * g + 2] = wl.z; ul[4 * g + 3] = wl.w;
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const int v = j * M + m;
            const float du = (uh[v] - sh[v]) + (ul[v] - sl[v]);
#pragma unroll
            for (int i = 0; i < D; ++i) acc[i * M + m] += S[i * D + j] * du;
          }
        }
      }
    }
  }
  if constexpr (PK && !ZERO) {
#pragma unroll
    for (int k = 0; k < CP; ++k) f2_unpack(acc2[k], acc[2 * k], acc[2 * k + 1]);
  }
  float nrm[M];
#pragma unroll
  for (int m = 0; m < M; ++m) nrm[m] = 0.f;
  const int64_t base = b * (64 * C) + loc;
#pragma unroll
  for (int v = 0; v < C; ++v) {
    const int i = v / M, m = v % M;
    float fv = 0.f;
    if constexpr (STORED) {
      fv = p.f[base + v * 64];
    } else {
#pragma unroll
      for (int a = 0; a < 8; ++a)
        fv += (((mk >> a) & 1u) ? 1.f : 0.f) * p.fc.Fe[(a * D + i) * M + m];
    }
    const float r = mk ? fv - acc[v] : 0.f;
    p.out[base + v * 64] = r;
    nrm[m] += r * r;
  }
  if (p.part) block_partial_64<M, float>(nrm, p.part + b * M);
}

// ------------------------------------------------------------------ transfers
struct LvView {
  int n, nbx;
  bool dense;
  int64_t nslots;
  const int* bmap;
  const int* bxyz;
  const uint8_t* mask;
};

static LvView view(const Level& l) {
  return LvView{l.n, l.nbx, l.dense, l.nslots, l.brick_map, l.brick_xyz, l.mask};
}

// f_c(j) = sum_{d in {-1,0,1}^3} prod_k (1 - |d_k|/2) r_f(2j + d): the transpose of the
// trilinear prolongation of App. E.2, gathered per coarse node
template <typename TS, typename A, int C>
__global__ void k_restrict(const TS* __restrict__ rf, TS* __restrict__ fc, LvView f, LvView c) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= c.nslots) return;
  A acc[C];
#pragma unroll
  for (int v = 0; v < C; ++v) acc[v] = A(0);
  if (c.mask[s]) {
    int X, Y, Z;
    slot_coords(s, c.n, c.dense, c.bxyz, X, Y, Z);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const A w = (dx ? A(0.5) : A(1)) * (dy ? A(0.5) : A(1)) * (dz ? A(0.5) : A(1));
      const int fx = (2 * X + dx + f.n) % f.n, fy = (2 * Y + dy + f.n) % f.n,
                fz = (2 * Z + dz + f.n) % f.n;
      const int64_t fs = site_slot(fx, fy, fz, f.n, f.nbx, f.bmap, false);
      if (fs < 0) continue;
#pragma unroll
      for (int v = 0; v < C; ++v) acc[v] += w * load_as<A>(rf + vaddr(fs, v, C));
    }
  }
#pragma unroll
  for (int v = 0; v < C; ++v) fc[vaddr(s, v, C)] = store_as<TS>(acc[v]);
}

// u_f(i) += sum_k W_ik u_c(I_ik) (App. E.2 weighted gather)
template <typename TS, typename A, int C>
__global__ void k_prolong(const TS* __restrict__ uc, TS* __restrict__ uf, LvView f, LvView c) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= f.nslots || !f.mask[s]) return;
  int x, y, z;
  slot_coords(s, f.n, false, f.bxyz, x, y, z);
  const int xs[3] = {x, y, z};
  int j0[3], j1[3];
  int cnt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    j0[k] = xs[k] >> 1;
    cnt[k] = (xs[k] & 1) ? 2 : 1;
    j1[k] = (j0[k] + 1) % c.n;
  }
  A acc[C];
#pragma unroll
  for (int v = 0; v < C; ++v) acc[v] = A(0);
  for (int cz = 0; cz < cnt[2]; ++cz)
    for (int cy = 0; cy < cnt[1]; ++cy)
      for (int cx = 0; cx < cnt[0]; ++cx) {
        const A w = (cnt[0] == 2 ? A(0.5) : A(1)) * (cnt[1] == 2 ? A(0.5) : A(1)) *
                    (cnt[2] == 2 ? A(0.5) : A(1));
        const int64_t cs = site_slot(cx ? j1[0] : j0[0], cy ? j1[1] : j0[1], cz ? j1[2] : j0[2],
                                     c.n, c.nbx, c.bmap, c.dense);
        if (cs < 0) continue;  // cannot happen: nonzero weights land on active coarse nodes
#pragma unroll
        for (int v = 0; v < C; ++v) acc[v] += w * load_as<A>(uc + vaddr(cs, v, C));
      }
#pragma unroll
  for (int v = 0; v < C; ++v) {
    const int64_t a = vaddr(s, v, C);
    uf[a] = store_as<TS>(load_as<A>(uf + a) + acc[v]);
  }
}

// Bricked levels: the same sums, staged through shared memory. One block per coarse brick
// stages the 9^3 fine sites its 64 nodes gather from (coalesced within fine bricks), then
// each thread forms its node's sum over d in the order of k_restrict (bitwise equal).
template <typename A>
constexpr int vec_groups(int C) { return (C + Vec16<A>::n - 1) / Vec16<A>::n; }

template <typename TS, typename A, int C>
__global__ void __launch_bounds__(256) k_restrict_tile(const TS* __restrict__ rf,
                                                       TS* __restrict__ fc, LvView f, LvView c) {
  using V = typename Vec16<A>::type;
  constexpr int NV = Vec16<A>::n, G = (C + NV - 1) / NV;
  extern __shared__ __align__(16) unsigned char tr_smem[];
  V* tile = reinterpret_cast<V*>(tr_smem);   // [G][729]
  const int64_t b = blockIdx.x;
  const int t = threadIdx.x;
  const int ox = 8 * c.bxyz[3 * b] - 1, oy = 8 * c.bxyz[3 * b + 1] - 1,
            oz = 8 * c.bxyz[3 * b + 2] - 1;
  // 256 threads stage the 729 sites (about 3 each, all loads of a site in flight together)
  for (int q = t; q < 729; q += 256) {
    const int rx = q % 9, ry = (q / 9) % 9, rz = q / 81;
    const int fx = (ox + rx + f.n) % f.n, fy = (oy + ry + f.n) % f.n, fz = (oz + rz + f.n) % f.n;
    const int64_t fs = site_slot(fx, fy, fz, f.n, f.nbx, f.bmap, false);
    A vals[G * NV];
#pragma unroll
    for (int v = 0; v < G * NV; ++v) vals[v] = A(0);
    if (fs >= 0) {
      const TS* src = rf + vaddr(fs, 0, C);
#pragma unroll
      for (int v = 0; v < C; ++v) vals[v] = load_as<A>(src + v * 64);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      V w;
#pragma unroll
      for (int k = 0; k < NV; ++k) vec_put<A>(w, k, vals[g * NV + k]);
      tile[g * 729 + q] = w;
    }
  }
  __syncthreads();
  // thread (node, part): coarse node t & 63 of the brick, value groups g = part, part + 4
  const int node = t & 63, part = t >> 6;
  const int lx = node & 3, ly = (node >> 2) & 3, lz = node >> 4;
  const bool act = c.mask[b * 64 + node] != 0;
  const int qc = (2 * lx + 1) + 9 * (2 * ly + 1) + 81 * (2 * lz + 1);
  TS* dst = fc + vaddr(b * 64 + node, 0, C);
  for (int g = part; g < G; g += 4) {
    A acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = A(0);
    if (act) {
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const A w = (dx ? A(0.5) : A(1)) * (dy ? A(0.5) : A(1)) * (dz ? A(0.5) : A(1));
        const V x = tile[g * 729 + qc + dx + 9 * dy + 81 * dz];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += w * vec_get<A>(x, k);
      }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (g * NV + k < C) dst[(g * NV + k) * 64] = store_as<TS>(acc[k]);
  }
}

// One block per fine brick: the 3^3 coarse sites its nodes interpolate from are staged in
// shared memory; each node adds its weighted terms in the order of k_prolong.
template <typename TS, typename A, int C>
__global__ void __launch_bounds__(64) k_prolong_tile(const TS* __restrict__ uc,
                                                     TS* __restrict__ uf, LvView f, LvView c) {
  __shared__ A cv[C][27];
  const int64_t b = blockIdx.x;
  const int t = threadIdx.x;
  const int bx = f.bxyz[3 * b], by = f.bxyz[3 * b + 1], bz = f.bxyz[3 * b + 2];
  for (int k = t; k < 27 * C; k += 64) {
    const int pos = k / C, v = k % C;
    const int px = pos % 3, py = (pos / 3) % 3, pz = pos / 9;
    const int64_t cs = site_slot((2 * bx + px) % c.n, (2 * by + py) % c.n, (2 * bz + pz) % c.n,
                                 c.n, c.nbx, c.bmap, false);
    cv[v][pos] = cs >= 0 ? load_as<A>(uc + vaddr(cs, v, C)) : A(0);
  }
  __syncthreads();
  const int64_t s = b * 64 + t;
  if (!f.mask[s]) return;
  const int lx = t & 3, ly = (t >> 2) & 3, lz = t >> 4;
  const int cnt[3] = {(lx & 1) ? 2 : 1, (ly & 1) ? 2 : 1, (lz & 1) ? 2 : 1};
  const int j0[3] = {lx >> 1, ly >> 1, lz >> 1};
  const A w = (cnt[0] == 2 ? A(0.5) : A(1)) * (cnt[1] == 2 ? A(0.5) : A(1)) *
              (cnt[2] == 2 ? A(0.5) : A(1));
  A acc[C];
#pragma unroll
  for (int v = 0; v < C; ++v) acc[v] = A(0);
  for (int cz = 0; cz < cnt[2]; ++cz)
    for (int cy = 0; cy < cnt[1]; ++cy)
      for (int cx = 0; cx < cnt[0]; ++cx) {
        const int pos = (j0[0] + cx) + 3 * (j0[1] + cy) + 9 * (j0[2] + cz);
#pragma unroll
        for (int v = 0; v < C; ++v) acc[v] += w * cv[v][pos];
      }
  TS* dst = uf + vaddr(s, 0, C);
#pragma unroll
  for (int v = 0; v < C; ++v) dst[v * 64] = store_as<TS>(load_as<A>(dst + v * 64) + acc[v]);
}

// ------------------------------------------------------------------ coarsest solve
template <typename TS, int D, int M>
__global__ void k_coarse_gather(const TS* __restrict__ f, const int* __restrict__ canon_slot,
                                int64_t nn, double* __restrict__ bvec, float* __restrict__ b32) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nn * D * M) return;
  const int64_t i = g / (D * M);
  const int v = (int)(g % (D * M));
  const auto x = load_as<typename ArithOf<TS>::type>(f + vaddr(canon_slot[i], v, D * M));
  bvec[g] = (double)x;
  if (b32) b32[g] = (float)x;
}

// FP32 product with the FP32 generalized inverse: u[r][m] = sum_k X[r][k] b[k][m]
// (+ add[r][m]); one warp per row, lanes over k in a fixed stride, fixed shuffle tree
template <int M>
__global__ void __launch_bounds__(256) k_coarse_gemv32(const float* __restrict__ X,
                                                       const float* __restrict__ b32,
                                                       int64_t mrows,
                                                       const double* __restrict__ add,
                                                       double* __restrict__ uvec) {
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= mrows) return;   // whole warp
  float acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = 0.f;
  const float* xr = X + r * mrows;
#pragma unroll 4
  for (int64_t k = lane; k < mrows; k += 32) {
    const float a = xr[k];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += a * b32[k * M + m];
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    float x = acc[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    acc[m] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) uvec[r * M + m] = (add ? add[r * M + m] : 0.0) + (double)acc[m];
  }
}

// u[r][m] = sum_k X[r][k] b[k][m] (+ u0[r][m]); one block per row r, fixed-order tree per
// row. With `A` given: res[r][m] = b[r][m] - sum_k A[r][k] u[k][m] instead (a residual).
template <typename TX, int M>
__global__ void k_coarse_gemv(const TX* __restrict__ X, const double* __restrict__ bvec,
                              int64_t mrows, const double* __restrict__ add,
                              double* __restrict__ uvec) {
  const int64_t r = blockIdx.x;
  double acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = 0.0;
  for (int64_t k = threadIdx.x; k < mrows; k += blockDim.x) {
    const double a = (double)X[r * mrows + k];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += a * bvec[k * M + m];
  }
  __shared__ double sh[M][128];
#pragma unroll
  for (int m = 0; m < M; ++m) sh[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
#pragma unroll
      for (int m = 0; m < M; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x < M) {
    const double v = sh[threadIdx.x][0];
    uvec[r * M + threadIdx.x] = add ? add[r * M + threadIdx.x] + v : v;
  }
}

// res = b - A u (FP64), same row-block structure
template <int M>
__global__ void k_coarse_resid(const double* __restrict__ A, const double* __restrict__ uvec,
                               const double* __restrict__ bvec, int64_t mrows,
                               double* __restrict__ res, float* __restrict__ res32) {
  const int64_t r = blockIdx.x;
  double acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = 0.0;
  for (int64_t k = threadIdx.x; k < mrows; k += blockDim.x) {
    const double a = A[r * mrows + k];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += a * uvec[k * M + m];
  }
  __shared__ double sh[M][128];
#pragma unroll
  for (int m = 0; m < M; ++m) sh[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
#pragma unroll
      for (int m = 0; m < M; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x < M) {
    const double v = bvec[r * M + threadIdx.x] - sh[threadIdx.x][0];
    res[r * M + threadIdx.x] = v;
    if (res32) res32[r * M + threadIdx.x] = (float)v;
  }
}

template <typename TS, int D, int M>
__global__ void k_coarse_scatter(const double* __restrict__ uvec, const int* __restrict__ canon_slot,
                                 int64_t nn, TS* __restrict__ u) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nn * D * M) return;
  const int64_t i = g / (D * M);
  const int v = (int)(g % (D * M));
  u[vaddr(canon_slot[i], v, D * M)] = store_as<TS>((typename ArithOf<TS>::type)uvec[g]);
}

// ------------------------------------------------------------------ element energies
template <typename A, int D, int M>
struct EnArgs {
  const int* nbr;
  const uint8_t* mask;
  const void* hi;   // A-typed field, or float hi part (ff)
  const float* lo;  // ff low part or nullptr
  double* part;
  A Ke[64 * D * D];       // FP64 path: K_e; ff path: K_e rounded to FP32 (hi part)
  A Kl[64 * D * D];       // ff path: K_e - hi (lo part)
  A X0[8 * D * M];        // FP64 path: x0
  A Fh[8 * D * M];        // ff path: f_e = K_e x0, hi and lo parts
  A Fl[8 * D * M];
  f2_t Ke2[32 * D * D];   // ff path: rows (2 rp, 2 rp + 1) of Ke / Kl packed per column
  f2_t Kl2[32 * D * D];
  // per-element output (sensitivities): out[e][I][J] = scale * (E_IJ of element e), with e
  // the canonical element index of the slot (slot_elem) and C0 added back on the ff path
  double* per;
  const int* slot_elem;
  double scale;
  double C0[M * M];
  // element densities (nullable): the block sums weight element e by coef[slot] = s_e; the
  // per-element output is multiplied by simp_p rho[slot]^(simp_p - 1) (App. F.3)
  const double* coef;
  const double* rho;
  double simp_p;
};

// Per active element e (origin slot n) and load cases I <= J, the energy
// (x0^I - u_e^I)^T K_e (x0^J - u_e^J). The element displacement enters through
// d = u_e - u_n (a translation, which K_e annihilates, removed so that FP32 sees O(1)
// values). FP64 path: w = x0 - d, E_IJ = w^I . K_e w^J. Float-float path, expanded so that
// no FP32 rounding is common to every element:
//     E_IJ - C0_IJ = d^I . K_e d^J - f^I . d^J - d^I . f^J,      f = K_e x0,
// with K_e and f split into FP32 hi + lo parts; C0_IJ (exact) is added once per element in
// FP64 on the host side (n_e C0).
// One thread per element: its d (or w) for every case goes to a thread-private column of
// shared memory, then each case J forms z = K_e d^J once and dots it with d^I for I <= J.
// The per-pair sums live in shared memory (runtime J, no local-memory arrays); they reuse
// the space of the staged tiles once d is formed.
template <typename A, int D, int M, bool FF>
constexpr size_t energy_smem_bytes() {
  constexpr int C = D * M, NV = Vec16<A>::n, G = (C + NV - 1) / NV;
  return (size_t)(FF ? 2 : 1) * G * 216 * 16 + (size_t)8 * D * M * 64 * sizeof(A);
}

// PER: write each element's energies (times p.scale) instead of the block sums.
template <typename A, int D, int M, bool FF, bool PER = false>
__global__ void __launch_bounds__(64) k_energy(const __grid_constant__ EnArgs<A, D, M> p) {
  using V = typename Vec16<A>::type;
  constexpr int C = D * M, R = 8 * D, K = M * (M + 1) / 2;
  constexpr int NV = Vec16<A>::n, G = (C + NV - 1) / NV;
  static_assert((size_t)K * 64 * 8 <= (size_t)(FF ? 2 : 1) * G * 216 * 16,
                "pair sums must fit in the tile space");
  extern __shared__ __align__(16) unsigned char en_smem[];
  V* th = reinterpret_cast<V*>(en_smem);
  V* tl = th + G * 216;                                              // FF only
  A* ws = reinterpret_cast<A*>(en_smem + (size_t)(FF ? 2 : 1) * G * 216 * 16);  // [R*M][64]
  // per-pair energies [K][64] after phase 1 (FP32 on the float-float path: per-element
  // rounding, not common to the elements, is summed away in FP64 across blocks)
  using ES = typename std::conditional<FF, float, double>::type;
  ES* es = reinterpret_cast<ES*>(en_smem);
  __shared__ int nb[27];
  const int t = threadIdx.x;
  const int64_t b = blockIdx.x;
  if (t < 27) nb[t] = p.nbr[b * 27 + t];
  __syncthreads();
  {
    A own[C];
    stage_tile<A, A, C>((const A*)p.hi, b, t, nb, th, own);
    if constexpr (FF) stage_tile<float, A, C>(p.lo, b, t, nb, tl, own);
  }
  __syncthreads();
  const int q0 = own_q0(t), loc = own_local(t);
  const bool act = (p.mask[b * 64 + loc] & 1u) != 0;  // element with origin at this node
  // phase 1: d (FF) or w = x0 - d (FP64) of this element, every dof r and case m
  if (act) {
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) {
      const int q = q0 + (bb & 1) + 6 * ((bb >> 1) & 1) + 36 * (bb >> 2);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const V a = th[g * 216 + q], a0 = th[g * 216 + q0];
        V l = a, l0 = a0;
        if constexpr (FF) {
          l = tl[g * 216 + q];
          l0 = tl[g * 216 + q0];
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const int v = g * NV + k;
          if (v < C) {
            const int r = (v / M) + D * bb, m = v % M;
            A du = vec_get<A>(a, k) - vec_get<A>(a0, k);
            if constexpr (FF) {
              du += vec_get<A>(l, k) - vec_get<A>(l0, k);
              ws[(r * M + m) * 64 + t] = du;
            } else {
              ws[(r * M + m) * 64 + t] = p.X0[r * M + m] - du;
            }
          }
        }
      }
    }
  }
  __syncthreads();  // tiles dead: es takes their space
  if (act) {
    // phase 2 (FF): the load terms f^I . d^J + f^J . d^I, kept as the pair's start value
    if constexpr (FF) {
      A phi[M][M];
#pragma unroll
      for (int J = 0; J < M; ++J) {
        A d[R];
#pragma unroll
        for (int r = 0; r < R; ++r) d[r] = ws[(r * M + J) * 64 + t];
#pragma unroll
        for (int I = 0; I < M; ++I) {
          A sh = A(0), sl = A(0);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            sh += p.Fh[r * M + I] * d[r];
            sl += p.Fl[r * M + I] * d[r];
          }
          phi[I][J] = sh + sl;
        }
      }
#pragma unroll
      for (int I = 0; I < M; ++I)
#pragma unroll
        for (int J = I; J < M; ++J)
          es[(I * M - I * (I - 1) / 2 + (J - I)) * 64 + t] = phi[I][J] + phi[J][I];
    }
    // phase 3: z = K_e d^J (hi + lo in FF), pair sums d^I . z for I <= J
#pragma unroll 1
    for (int J = 0; J < M; ++J) {
      A w[R], z[R];
#pragma unroll
      for (int r = 0; r < R; ++r) w[r] = ws[(r * M + J) * 64 + t];
      if constexpr (FF) {
        // two rows per f32x2 instruction, the same operations in the same order per row
        f2_t w2[R];
#pragma unroll
        for (int c = 0; c < R; ++c) w2[c] = f2_pack(w[c], w[c]);
#pragma unroll
        for (int rp = 0; rp < R / 2; ++rp) {
          f2_t sh2 = 0ull, sl2 = 0ull;
#pragma unroll
          for (int c = 0; c < R; ++c) {
            sh2 = f2_fma(p.Ke2[rp * R + c], w2[c], sh2);
            sl2 = f2_fma(p.Kl2[rp * R + c], w2[c], sl2);
          }
          f2_unpack(f2_add(sh2, sl2), z[2 * rp], z[2 * rp + 1]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          A sacc = A(0);
#pragma unroll
          for (int c = 0; c < R; ++c) sacc += p.Ke[r * R + c] * w[c];
          z[r] = sacc;
        }
      }
#pragma unroll
      for (int I = 0; I < M; ++I) {
        if (I <= J) {
          A sacc = A(0);
#pragma unroll
          for (int r = 0; r < R; ++r) sacc += ws[(r * M + I) * 64 + t] * z[r];
          ES* ep = es + (I * M - I * (I - 1) / 2 + (J - I)) * 64 + t;
          if constexpr (FF) *ep = sacc - *ep;
          else *ep = sacc;
        }
      }
    }
  }
  if constexpr (PER) {
    if (!act) return;
    const int64_t el = p.slot_elem[b * 64 + loc];
    const double fac = p.rho ? p.simp_p * pow(p.rho[b * 64 + loc], p.simp_p - 1.0) : 1.0;
#pragma unroll
    for (int I = 0; I < M; ++I)
#pragma unroll
      for (int J = I; J < M; ++J) {
        double v = (double)es[(I * M - I * (I - 1) / 2 + (J - I)) * 64 + t];
        if constexpr (FF) v += p.C0[I * M + J];
        v *= p.scale * fac;
        p.per[(el * M + I) * M + J] = v;
        p.per[(el * M + J) * M + I] = v;
      }
  } else {
    ES e[K];
    const ES w = (act && p.coef) ? (ES)p.coef[b * 64 + loc] : ES(1);
#pragma unroll
    for (int k = 0; k < K; ++k) e[k] = act ? w * es[k * 64 + t] : ES(0);
    block_partial_64<K, ES>(e, p.part + b * K);
  }
}

// deterministic reduction of [nblk][K] partials. Column k is split over gridDim.y blocks;
// each reduces its row range (Neumaier-compensated per thread over a fixed stride, then a
// fixed-order tree), writes (sum, compensation) to scratch, and the block that arrives last
// (atomic ticket) combines the gridDim.y pairs in index order and runs the epilogue. The
// result does not depend on which block arrives last; no block waits for another.
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  const double tt = s + x;
  c += fabs(s) >= fabs(x) ? (s - tt) + x : (x - tt) + s;
  s = tt;
}

// Several column groups of the same partials in one launch: blockIdx.x runs over the
// groups' columns in order; each group has its own first column, output and epilogue.
struct RedGroups {
  int n = 0;
  int col0[3] = {0, 0, 0}, ncols[3] = {0, 0, 0};
  double* out[3] = {nullptr, nullptr, nullptr};
  RedEpi epi[3];
};

__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ part, int64_t nblk,
                                                int ld, const __grid_constant__ RedGroups grp,
                                                double* __restrict__ scratch,
                                                unsigned* __restrict__ ticket) {
  __shared__ double ss[256], sc[256];
  __shared__ bool last;
  const int kg = blockIdx.x, sp = blockIdx.y, S = gridDim.y;   // kg: column among all groups
  int gi = 0, k = kg;
  while (gi + 1 < grp.n && k >= grp.ncols[gi]) k -= grp.ncols[gi++];
  const int col = grp.col0[gi] + k;                               // column of the partials
  double* __restrict__ out = grp.out[gi];
  const RedEpi& epi = grp.epi[gi];
  const int64_t chunk = (nblk + S - 1) / S;
  const int64_t lo = (int64_t)sp * chunk;
  const int64_t hi = lo + chunk < nblk ? lo + chunk : nblk;
  double s = 0.0, c = 0.0;
  for (int64_t i0 = lo + threadIdx.x; i0 < hi; i0 += 256 * 4) {
    double x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t i = i0 + (int64_t)j * 256;
      x[j] = i < hi ? part[i * ld + col] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) neumaier(s, c, x[j]);
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double a = ss[threadIdx.x], ca = sc[threadIdx.x] + sc[threadIdx.x + o];
      neumaier(a, ca, ss[threadIdx.x + o]);
      ss[threadIdx.x] = a;
      sc[threadIdx.x] = ca;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (S == 1) {
      last = true;
    } else {
      scratch[((int64_t)kg * S + sp) * 2] = ss[0];
      scratch[((int64_t)kg * S + sp) * 2 + 1] = sc[0];
      __threadfence();
      last = atomicAdd(&ticket[kg], 1u) == (unsigned)(S - 1);
    }
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  double v;
  if (S == 1) {
    v = ss[0] + sc[0];
  } else {
    __threadfence();
    double a = 0.0, ca = 0.0;
    for (int j = 0; j < S; ++j) {
      ca += __ldcg(&scratch[((int64_t)kg * S + j) * 2 + 1]);
      neumaier(a, ca, __ldcg(&scratch[((int64_t)kg * S + j) * 2]));
    }
    v = a + ca;
    ticket[kg] = 0u;  // ready for the next launch on this stream
  }
  out[k] = v;
  const bool act = epi.active == nullptr || epi.active[k] != 0;
  if (epi.mode == 1) {
    epi.ratio[k] = (act && v != 0.0) ? epi.other[k] / v : 0.0;
  } else if (epi.mode == 2) {
    epi.ratio[k] = (act && epi.other[k] != 0.0) ? v / epi.other[k] : 0.0;
  } else if (epi.mode == 3) {
    epi.out32[k] = (float)(v * epi.scale);
  } else if (epi.mode == 4) {
    const double x = v * epi.scale;
    const float hf = (float)x;
    epi.out32[k] = hf;
    epi.out32[epi.count + k] = (float)(x - (double)hf);
  } else if (epi.mode == 5) {
    epi.ratio[k] = 1.0 / sqrt(fmax(v, 1e-300));
  } else if (epi.mode == 6) {
    epi.ratio[k] = (act && epi.other[k] != 0.0) ? -epi.other2[k] * v / epi.other[k] : 0.0;
  }
}

// ------------------------------------------------------------------ vector kernels
template <typename TS>
__global__ void k_vzero(TS* __restrict__ x, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = store_as<TS>((typename ArithOf<TS>::type)0);
}

template <typename TS>
__global__ void k_vcopy(const TS* __restrict__ a, TS* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

template <typename TS>
__global__ void k_vadd(const TS* __restrict__ y, TS* __restrict__ x, int64_t n) {
  using A = typename ArithOf<TS>::type;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = store_as<TS>(load_as<A>(x + i) + load_as<A>(y + i));
}

// block of 64 slots (one brick) per block
template <typename TS, int M, int C>
__global__ void __launch_bounds__(64) k_vdot(const TS* __restrict__ x, const TS* __restrict__ y,
                                             double* __restrict__ part) {
  using A = typename ArithOf<TS>::type;
  const int64_t base = (int64_t)blockIdx.x * 64 * C + threadIdx.x;
  A d[M];
#pragma unroll
  for (int m = 0; m < M; ++m) d[m] = A(0);
#pragma unroll
  for (int v = 0; v < C; ++v) d[v % M] += load_as<A>(x + base + v * 64) * load_as<A>(y + base + v * 64);
  block_partial_64<M, A>(d, part + (int64_t)blockIdx.x * M);
}

// per-case step ratio from the device (0 for inactive cases), staged once per block
template <typename A, int M>
__device__ __forceinline__ void block_ratios(const double* ratio, const int* active, A* out) {
  if (threadIdx.x < M) {
    const int m = threadIdx.x;
    out[m] = (active == nullptr || active[m]) ? (A)ratio[m] : A(0);
  }
  __syncthreads();
}

// SUMS: partials [M + C]: ||r||^2 per case, then the sums of r per value (r is zero at
// inactive slots)
template <typename TS, int M, int C, bool SUMS>
__global__ void __launch_bounds__(64)
    k_cg_update(const double* __restrict__ ratio, const int* __restrict__ active,
                TS* __restrict__ x, const TS* __restrict__ pp, TS* __restrict__ r,
                const TS* __restrict__ q, double* __restrict__ part) {
  using A = typename ArithOf<TS>::type;
  constexpr int K = SUMS ? M + C : M;
  __shared__ A alpha[M];
  block_ratios<A, M>(ratio, active, alpha);
  const int64_t base = (int64_t)blockIdx.x * 64 * C + threadIdx.x;
  A nr[K];
#pragma unroll
  for (int k = 0; k < K; ++k) nr[k] = A(0);
#pragma unroll
  for (int v = 0; v < C; ++v) {
    const A al = alpha[v % M];
    const int64_t a = base + v * 64;
    x[a] = store_as<TS>(load_as<A>(x + a) + al * load_as<A>(pp + a));
    const TS rs = store_as<TS>(load_as<A>(r + a) - al * load_as<A>(q + a));
    r[a] = rs;
    const A rn = load_as<A>(&rs);
    nr[v % M] += rn * rn;
    if constexpr (SUMS) nr[M + v] += rn;
  }
  block_partial_64<K, A>(nr, part + (int64_t)blockIdx.x * K);
}

// one block per brick: p = (z - zmean) + beta p, the mean removed at active slots only
template <typename TS, int M, int C>
__global__ void __launch_bounds__(64) k_cg_dir(const double* __restrict__ ratio,
                                               const TS* __restrict__ z, TS* __restrict__ pp,
                                               const float* __restrict__ zmean,
                                               const uint8_t* __restrict__ mask) {
  using A = typename ArithOf<TS>::type;
  __shared__ A beta[M];
  block_ratios<A, M>(ratio, nullptr, beta);
  const int64_t b = blockIdx.x;
  const int t = threadIdx.x;
  const bool sub = zmean != nullptr && mask[b * 64 + t] != 0;
  const int64_t base = b * 64 * C + t;
#pragma unroll
  for (int v = 0; v < C; ++v) {
    const int64_t a = base + v * 64;
    A zv = load_as<A>(z + a);
    if (sub) zv -= (A)zmean[v];
    pp[a] = store_as<TS>(zv + beta[v % M] * load_as<A>(pp + a));
  }
}

// float-float accumulate (hi, lo) += d with Knuth's TwoSum and a fast renormalisation
__global__ void k_ff_add(const float* __restrict__ d, float* __restrict__ hi,
                         float* __restrict__ lo, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = hi[i], b = d[i];
  const float s = a + b;
  const float bb = s - a;
  const float err = (a - (s - bb)) + (b - bb);
  const float l = lo[i] + err;
  const float h2 = s + l;
  hi[i] = h2;
  lo[i] = l - (h2 - s);
}

// float-float minus a mean given as float pairs, one block per brick, active slots only
template <int C>
__global__ void __launch_bounds__(64) k_ff_sub_mean(const float* __restrict__ mean,
                                                    const uint8_t* __restrict__ mask,
                                                    float* __restrict__ hi,
                                                    float* __restrict__ lo) {
  const int64_t b = blockIdx.x;
  const int t = threadIdx.x;
  if (!mask[b * 64 + t]) return;
  const int64_t base = b * 64 * C + t;
#pragma unroll
  for (int v = 0; v < C; ++v) {
    const int64_t i = base + v * 64;
    const float a = hi[i], bm = -mean[v];
    const float s = a + bm;
    const float bb = s - a;
    const float err = (a - (s - bb)) + (bm - bb);
    const float l = lo[i] - mean[C + v] + err;
    const float h2 = s + l;
    hi[i] = h2;
    lo[i] = l - (h2 - s);
  }
}

// per-block sums of hi + lo per value over active slots: lanes and warps reduce float-float
// pairs (TwoSum), the two warp sums are combined in FP64
template <int C>
__global__ void __launch_bounds__(64) k_sum_ff(const float* __restrict__ hi,
                                               const float* __restrict__ lo,
                                               const uint8_t* __restrict__ mask,
                                               double* __restrict__ part) {
  __shared__ double red[2][C];
  const int64_t b = blockIdx.x;
  const int t = threadIdx.x;
  const bool act = mask[b * 64 + t] != 0;
  const int64_t base = b * 64 * C + t;
#pragma unroll
  for (int v = 0; v < C; ++v) {
    float sh = act ? hi[base + v * 64] : 0.f;
    float sl = act ? lo[base + v * 64] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_down_sync(0xffffffffu, sh, o);
      const float ol = __shfl_down_sync(0xffffffffu, sl, o);
      const float s = sh + oh;
      const float bb = s - sh;
      const float err = (sh - (s - bb)) + (oh - bb);
      const float l = sl + ol + err;
      sh = s + l;
      sl = l - (sh - s);
    }
    if ((t & 31) == 0) red[t >> 5][v] = (double)sh + (double)sl;
  }
  __syncthreads();
  if (t < C) part[b * C + t] = red[0][t] + red[1][t];
}

template <typename TS, int C>
__global__ void __launch_bounds__(64) k_sum_values(const TS* __restrict__ x,
                                                   const float* __restrict__ lo,
                                                   const uint8_t* __restrict__ mask,
                                                   double* __restrict__ part) {
  using A = typename ArithOf<TS>::type;
  const int64_t base = (int64_t)blockIdx.x * 64 * C + threadIdx.x;
  const bool act = mask[(int64_t)blockIdx.x * 64 + threadIdx.x] != 0;
  double s[C];
#pragma unroll
  for (int v = 0; v < C; ++v) {
    double val = act ? (double)load_as<A>(x + base + v * 64) : 0.0;
    if (lo && act) val += (double)lo[base + v * 64];
    s[v] = val;
  }
  block_partial_64<C, double>(s, part + (int64_t)blockIdx.x * C);
}

// x -= sums[v] / n over active slots (FP32 field; sums on the device)
// per-block sums of each value over active slots, FP32 per lane and warp (projections)
template <int C>
__global__ void __launch_bounds__(64) k_sum_values32(const float* __restrict__ x,
                                                     const uint8_t* __restrict__ mask,
                                                     double* __restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * 64 * C + threadIdx.x;
  const bool act = mask[(int64_t)blockIdx.x * 64 + threadIdx.x] != 0;
  float s[C];
#pragma unroll
  for (int v = 0; v < C; ++v) s[v] = act ? x[base + v * 64] : 0.f;
  block_partial_64<C, float>(s, part + (int64_t)blockIdx.x * C);
}

template <int C>
__global__ void __launch_bounds__(64) k_sub_mean32(const float* __restrict__ mean,
                                                   const uint8_t* __restrict__ mask,
                                                   float* __restrict__ x) {
  const int64_t b = blockIdx.x;
  const int t = threadIdx.x;
  if (!mask[b * 64 + t]) return;
  float* xb = x + b * 64 * C + t;
#pragma unroll
  for (int v = 0; v < C; ++v) xb[v * 64] -= mean[v];
}

template <int C>
__global__ void k_sub_mean64(const double* __restrict__ mean, const uint8_t* __restrict__ mask,
                             double* __restrict__ x, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t slot = ((i >> 6) / C) * 64 + (i & 63);
  if (!mask[slot]) return;
  x[i] -= mean[(i >> 6) % C];
}

template <typename TS, int M, int C>
__global__ void k_scale_cases(const double* __restrict__ s, TS* __restrict__ x, int64_t n) {
  using A = typename ArithOf<TS>::type;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int v = (int)((i >> 6) % C);
  x[i] = store_as<TS>(load_as<A>(x + i) * (A)s[v % M]);
}

template <typename TS>
__global__ void k_canon_to_slots(const double* __restrict__ src, const int* __restrict__ canon_slot,
                                 int64_t nn, int C, TS* __restrict__ dst) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nn * C) return;
  const int64_t i = g / C;
  const int v = (int)(g % C);
  dst[vaddr(canon_slot[i], v, C)] = store_as<TS>((typename ArithOf<TS>::type)src[g]);
}

template <typename TS>
__global__ void k_slots_to_canon(const TS* __restrict__ src, const int* __restrict__ canon_slot,
                                 int64_t nn, int C, double* __restrict__ dst) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nn * C) return;
  const int64_t i = g / C;
  const int v = (int)(g % C);
  dst[g] = (double)load_as<typename ArithOf<TS>::type>(src + vaddr(canon_slot[i], v, C));
}

__global__ void k_canon_to_ff(const double* __restrict__ src, const int* __restrict__ canon_slot,
                              int64_t nn, int C, float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nn * C) return;
  const int64_t i = g / C;
  const int v = (int)(g % C);
  const double x = src[g];
  const float h = (float)x;
  const int64_t a = vaddr(canon_slot[i], v, C);
  hi[a] = h;
  lo[a] = (float)(x - (double)h);
}

__global__ void k_ff_to_canon(const float* __restrict__ hi, const float* __restrict__ lo,
                              const int* __restrict__ canon_slot, int64_t nn, int C,
                              double* __restrict__ dst) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nn * C) return;
  const int64_t i = g / C;
  const int v = (int)(g % C);
  const int64_t a = vaddr(canon_slot[i], v, C);
  dst[g] = (double)hi[a] + (double)lo[a];
}

__global__ void k_ff_to_f64(const float* __restrict__ hi, const float* __restrict__ lo,
                            double* __restrict__ dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)hi[i] + (double)lo[i];
}

__global__ void k_f64_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

// ------------------------------------------------------------------ host launchers
template <typename A, int D, int M>
static void fill_fine(const Material& mt, FineC<A, D, M>& fc) {
  for (int i = 0; i < 64 * D * D; ++i) fc.Ke[i] = (A)mt.Ke[i];
  for (int i = 0; i < 8 * D * M; ++i) fc.Fe[i] = (A)mt.Fe[i];
  const int R = 8 * D;
  for (int d = 0; d < 27; ++d) {
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    for (int k = 0; k < D * D; ++k) {
      double acc = 0.0;
      for (int a = 0; a < 8; ++a) {
        const int ex = (a & 1) + dx, ey = ((a >> 1) & 1) + dy, ez = (a >> 2) + dz;
        if (ex < 0 || ex > 1 || ey < 0 || ey > 1 || ez < 0 || ez > 1) continue;
        const int bb = ex + 2 * ey + 4 * ez;
        acc += mt.Ke[(a * D + k / D) * R + bb * D + k % D];
      }
      fc.Sf[d * D * D + k] = (A)acc;
      const float sf = (float)acc;
      uint32_t bits;
      std::memcpy(&bits, &sf, 4);
      fc.Sf2[d * D * D + k] = ((f2_t)bits << 32) | (f2_t)bits;
    }
  }
}

template <typename TS, typename A, int D, int M>
static void stencil_t(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& va) {
  const Level& lv = h->lv[level];
  StArgs<TS, A, D, M> p;
  std::memset(&p, 0, sizeof(p));
  p.nbr = lv.brick_nbr;
  p.mask = lv.mask;
  p.kidx = lv.kidx;
  // level 0 forms its stencil from the octant masks and K_e (KIND 0), unless element
  // densities are set: then it reads stored per-node stencils like a coarse level (KIND 1)
  const bool fine = level == 0 && !h->dens;
  if (!fine) build_node_stencils(h, level, sizeof(A) == 8);
  if constexpr (sizeof(A) == 8) {
    p.kmat = (const A*)lv.S64;
    p.dinv = (const A*)lv.dinv64;
  } else {
    p.kmat = (const A*)lv.S32;
    p.dinv = (const A*)lv.dinv32;
  }
  p.u = (const TS*)va.u;
  p.f = (const TS*)va.f;
  p.dprev = (const TS*)va.dprev;
  p.aux = (const TS*)va.aux;
  p.out = (TS*)va.out;
  p.dout = (TS*)va.dout;
  p.part = va.part;
  p.omega = (A)va.omega;
  p.c1 = (A)va.c1;
  p.c2 = (A)va.c2;
  p.colour = va.colour;
  if (fine) fill_fine<A, D, M>(h->mat, p.fc);
  if (level == 0 && h->dens && p.f == nullptr)   // the stored level-0 load
    p.f = sizeof(TS) == 8 ? (const TS*)h->f0_64 : (const TS*)h->f0_32;
  const unsigned g = (unsigned)lv.nb;
  cudaStream_t s = h->stream;
  int nvec = 2, cat = level == 1 ? TR_COARSE_ST : TR_COARSE_ST2;
  if (mode == ST_RESID) nvec = va.f ? 3 : 2;
  if (mode == ST_JACOBI) nvec = 3 + (va.aux != nullptr);   // the last sweep also reads K p
  if (mode == ST_CHEB) nvec = 3 + (va.c1 != 0.0) + (va.dout != nullptr);
  if (level == 0) {
    cat = mode == ST_APPLY ? TR_APPLY0 : (mode == ST_RESID ? (va.f ? TR_RESID0 : TR_OUTER) : TR_SMOOTH0);
  }
  TraceScope ts(&h->tracer, s, cat, (double)lv.n_nodes * nvec * D * M * sizeof(TS));
#define GMT_ST(KIND, MODE) k_stencil<TS, A, D, M, KIND, MODE><<<g, 64, 0, s>>>(p)
  // smoother modes at level 0: fused r.z and sums of z
  const bool sums = level == 0 && va.part != nullptr;
  switch (mode) {
    case ST_APPLY: if (fine) GMT_ST(0, ST_APPLY); else GMT_ST(1, ST_APPLY); break;
    case ST_RESID: if (fine) GMT_ST(0, ST_RESID); else GMT_ST(1, ST_RESID); break;
    case ST_JACOBI:
      if (sums && fine) k_stencil<TS, A, D, M, 0, ST_JACOBI, true><<<g, 64, 0, s>>>(p);
      else if (sums) k_stencil<TS, A, D, M, 1, ST_JACOBI, true><<<g, 64, 0, s>>>(p);
      else if (fine) GMT_ST(0, ST_JACOBI);
      else GMT_ST(1, ST_JACOBI);
      break;
    case ST_CHEB:
      if (sums && fine) k_stencil<TS, A, D, M, 0, ST_CHEB, true><<<g, 64, 0, s>>>(p);
      else if (sums) k_stencil<TS, A, D, M, 1, ST_CHEB, true><<<g, 64, 0, s>>>(p);
      else if (fine) GMT_ST(0, ST_CHEB);
      else GMT_ST(1, ST_CHEB);
      break;
  }
#undef GMT_ST
  GMT_LAUNCH_CHECK();
}

#define GMT_DISPATCH_PREC(prec, FN, ...)                                  \
  do {                                                                    \
    if (h->mat.D == 3) {                                                  \
      if (prec == P64) FN<double, double, 3, 6>(__VA_ARGS__);             \
      else if (prec == P32) FN<float, float, 3, 6>(__VA_ARGS__);          \
      else FN<__nv_bfloat16, float, 3, 6>(__VA_ARGS__);                   \
    } else {                                                              \
      if (prec == P64) FN<double, double, 1, 3>(__VA_ARGS__);             \
      else if (prec == P32) FN<float, float, 1, 3>(__VA_ARGS__);          \
      else FN<__nv_bfloat16, float, 1, 3>(__VA_ARGS__);                   \
    }                                                                     \
  } while (0)

void launch_stencil(gmt_hierarchy* h, int level, Prec prec, StencilMode mode, const VecArgs& a) {
  GMT_DISPATCH_PREC(prec, stencil_t, h, level, mode, a);
}

template <typename TS, typename A, int D, int M>
static void diag_t(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double scale) {
  const Level& lv = h->lv[level];
  StArgs<TS, A, D, M> p;
  std::memset(&p, 0, sizeof(p));
  p.mask = lv.mask;
  p.dinv = sizeof(A) == 8 ? (const A*)lv.dinv64 : (const A*)lv.dinv32;
  p.f = (const TS*)f;
  p.out = (TS*)out;
  p.dout = (TS*)dout;
  p.omega = (A)scale;
  const unsigned g = grid_for(lv.nslots, 128);
  TraceScope ts(&h->tracer, h->stream,
                level == 0 ? TR_DIAG0 : (level == 1 ? TR_COARSE_ST : TR_COARSE_ST2),
                (double)lv.n_nodes * (dout ? 3 : 2) * D * M * sizeof(TS));
  if (level == 0 && !h->dens) {
    fill_fine<A, D, M>(h->mat, p.fc);
    k_diag<TS, A, D, M, 0><<<g, 128, 0, h->stream>>>(p, lv.nslots);
  } else {
    k_diag<TS, A, D, M, 1><<<g, 128, 0, h->stream>>>(p, lv.nslots);
  }
  GMT_LAUNCH_CHECK();
}

void launch_diag(gmt_hierarchy* h, int level, Prec prec, const void* f, void* out, void* dout,
                 double scale) {
  GMT_DISPATCH_PREC(prec, diag_t, h, level, f, out, dout, scale);
}

template <int D, int M>
static void resid_ff_t(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part) {
  const Level& lv = h->lv[0];
  FFArgs<D, M> p;
  std::memset(&p, 0, sizeof(p));
  p.nbr = lv.brick_nbr;
  p.mask = lv.mask;
  p.hi = hi;
  p.lo = lo;
  p.out = r;
  p.part = part;
  fill_fine<float, D, M>(h->mat, p.fc);
  if (h->dens) {
    build_node_stencils(h, 0, false);
    p.kmat = lv.S32;
    p.f = h->f0_32;
  }
  TraceScope ts(&h->tracer, h->stream, TR_OUTER, (double)lv.n_nodes * 3 * D * M * sizeof(float));
  const unsigned g = (unsigned)lv.nb;
  if (h->dens) {
    if (hi == nullptr) k_resid_ff<D, M, true, true><<<g, 64, 0, h->stream>>>(p);
    else k_resid_ff<D, M, false, true><<<g, 64, 0, h->stream>>>(p);
  } else {
    if (hi == nullptr) k_resid_ff<D, M, true><<<g, 64, 0, h->stream>>>(p);
    else k_resid_ff<D, M, false><<<g, 64, 0, h->stream>>>(p);
  }
  GMT_LAUNCH_CHECK();
}

void launch_resid_ff(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part) {
  if (h->mat.D == 3) resid_ff_t<3, 6>(h, hi, lo, r, part);
  else resid_ff_t<1, 3>(h, hi, lo, r, part);
}

template <typename TS, typename A, int D, int M>
static void restrict_t(gmt_hierarchy* h, int level, const void* rf, void* fc) {
  const Level& c = h->lv[level + 1];
  TraceScope ts(&h->tracer, h->stream, TR_RESTRICT,
                (double)(h->lv[level].n_nodes + c.n_nodes) * D * M * sizeof(TS));
  const Level& f = h->lv[level];
  if (!f.dense && !c.dense) {
    constexpr int C = D * M;
    constexpr size_t smem = (size_t)vec_groups<A>(C) * 729 * 16;
    ensure_smem_attr((const void*)k_restrict_tile<TS, A, C>, (int)smem);
    k_restrict_tile<TS, A, C><<<(unsigned)c.nb, 256, smem, h->stream>>>((const TS*)rf, (TS*)fc,
                                                                       view(f), view(c));
  } else {
    k_restrict<TS, A, D * M><<<grid_for(c.nslots, 64), 64, 0, h->stream>>>(
        (const TS*)rf, (TS*)fc, view(f), view(c));
  }
  GMT_LAUNCH_CHECK();
}
void launch_restrict(gmt_hierarchy* h, int level, Prec prec, const void* rf, void* fc) {
  GMT_DISPATCH_PREC(prec, restrict_t, h, level, rf, fc);
}

template <typename TS, typename A, int D, int M>
static void prolong_t(gmt_hierarchy* h, int level, const void* uc, void* uf) {
  const Level& f = h->lv[level];
  TraceScope ts(&h->tracer, h->stream, TR_PROLONG,
                (double)(2 * f.n_nodes + h->lv[level + 1].n_nodes) * D * M * sizeof(TS));
  const Level& c = h->lv[level + 1];
  if (!f.dense && !c.dense) {
    k_prolong_tile<TS, A, D * M><<<(unsigned)f.nb, 64, 0, h->stream>>>((const TS*)uc, (TS*)uf,
                                                                       view(f), view(c));
  } else {
    k_prolong<TS, A, D * M><<<grid_for(f.nslots, 64), 64, 0, h->stream>>>(
        (const TS*)uc, (TS*)uf, view(f), view(c));
  }
  GMT_LAUNCH_CHECK();
}
void launch_prolong(gmt_hierarchy* h, int level, Prec prec, const void* uc, void* uf) {
  GMT_DISPATCH_PREC(prec, prolong_t, h, level, uc, uf);
}

template <typename TS, typename A, int D, int M>
static void coarse_t(gmt_hierarchy* h, const void* f, void* u) {
  const Level& c = h->lv[h->L - 1];
  const int64_t cnt = c.n_nodes * D * M;
  const unsigned rows = (unsigned)h->m;
  if constexpr (sizeof(TS) == 8) build_coarse_inverse64(h);
  TraceScope ts(&h->tracer, h->stream, TR_CSOLVE, (double)h->m * h->m * 8.0);
  constexpr bool f64 = sizeof(TS) == 8;
  k_coarse_gather<TS, D, M><<<grid_for(cnt, 256), 256, 0, h->stream>>>(
      (const TS*)f, c.canon_slot, c.n_nodes, h->cb, f64 ? nullptr : h->cb32);
  GMT_LAUNCH_CHECK();
  if constexpr (f64) {
    // all-FP64 path: exact inverse
    k_coarse_gemv<double, M><<<rows, 128, 0, h->stream>>>(h->Ainv, h->cb, h->m, nullptr, h->cu);
    GMT_LAUNCH_CHECK();
  } else {
    // u = X f (FP32), then one refinement u += X (f - A u) with the residual in FP64
    const unsigned g8 = (unsigned)((h->m + 7) / 8);
    k_coarse_gemv32<M><<<g8, 256, 0, h->stream>>>(h->X32, h->cb32, h->m, nullptr, h->cu);
    GMT_LAUNCH_CHECK();
    k_coarse_resid<M><<<rows, 128, 0, h->stream>>>(h->A64, h->cu, h->cb, h->m, h->cr, h->cb32);
    GMT_LAUNCH_CHECK();
    k_coarse_gemv32<M><<<g8, 256, 0, h->stream>>>(h->X32, h->cb32, h->m, h->cu, h->cu);
    GMT_LAUNCH_CHECK();
  }
  vec_zero(h, h->L - 1, sizeof(TS) == 8 ? P64 : (sizeof(TS) == 4 ? P32 : PBF), u);
  k_coarse_scatter<TS, D, M><<<grid_for(cnt, 256), 256, 0, h->stream>>>(h->cu, c.canon_slot,
                                                                        c.n_nodes, (TS*)u);
  GMT_LAUNCH_CHECK();
}
void launch_coarse_solve(gmt_hierarchy* h, Prec prec, const void* f, void* u) {
  GMT_DISPATCH_PREC(prec, coarse_t, h, f, u);
}

template <typename A, int D, int M, bool FF>
static void energy_t(gmt_hierarchy* h, const void* hi, const float* lo, double* part,
                     double* per = nullptr, double scale = 0.0) {
  const Level& lv = h->lv[0];
  EnArgs<A, D, M> p;
  std::memset(&p, 0, sizeof(p));
  p.nbr = lv.brick_nbr;
  p.mask = lv.mask;
  p.hi = hi;
  p.lo = lo;
  p.part = part;
  for (int i = 0; i < 64 * D * D; ++i) {
    p.Ke[i] = (A)h->mat.Ke[i];
    p.Kl[i] = (A)(h->mat.Ke[i] - (double)p.Ke[i]);
  }
  if constexpr (FF) {
    const int R = 8 * D;
    auto bits = [](float x) {
      uint32_t u;
      std::memcpy(&u, &x, 4);
      return (f2_t)u;
    };
    for (int rp = 0; rp < R / 2; ++rp)
      for (int c = 0; c < R; ++c) {
        p.Ke2[rp * R + c] = bits((float)p.Ke[2 * rp * R + c]) |
                            (bits((float)p.Ke[(2 * rp + 1) * R + c]) << 32);
        p.Kl2[rp * R + c] = bits((float)p.Kl[2 * rp * R + c]) |
                            (bits((float)p.Kl[(2 * rp + 1) * R + c]) << 32);
      }
  }
  for (int i = 0; i < 8 * D * M; ++i) {
    p.X0[i] = (A)h->mat.X0[i];
    p.Fh[i] = (A)h->mat.Fe[i];
    p.Fl[i] = (A)(h->mat.Fe[i] - (double)p.Fh[i]);
  }
  constexpr size_t smem = energy_smem_bytes<A, D, M, FF>();
  TraceScope ts(&h->tracer, h->stream, TR_ENERGY, (double)lv.n_nodes * D * M * 8.0);
  if (h->dens) {
    p.coef = h->coef64;
    p.rho = h->rho64;
    p.simp_p = h->simp_p;
  }
  if (per) {
    p.per = per;
    p.slot_elem = level0_slot_elem(h);
    p.scale = scale;
    for (int i = 0; i < M * M; ++i) p.C0[i] = h->mat.C0[i];
    ensure_smem_attr((const void*)k_energy<A, D, M, FF, true>, (int)smem);
    k_energy<A, D, M, FF, true><<<(unsigned)lv.nb, 64, smem, h->stream>>>(p);
  } else {
    ensure_smem_attr((const void*)k_energy<A, D, M, FF>, (int)smem);
    k_energy<A, D, M, FF><<<(unsigned)lv.nb, 64, smem, h->stream>>>(p);
  }
  GMT_LAUNCH_CHECK();
}

// canonical element index of each level-0 slot whose element (origin at the slot) is
// active, -1 elsewhere; built on first use from the element -> slot map
__global__ void k_slot_elem(const int* __restrict__ elem_slot, int64_t ne, int* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne) out[elem_slot[e]] = (int)e;
}

const int* level0_slot_elem(gmt_hierarchy* h) {
  Level& l0 = h->lv[0];
  if (!l0.slot_elem) {
    l0.slot_elem = h->geo.alloc<int>(l0.nslots);
    GMT_CUDA(cudaMemsetAsync(l0.slot_elem, 0xff, l0.nslots * sizeof(int), h->stream));
    k_slot_elem<<<grid_for(l0.n_elems, 256), 256, 0, h->stream>>>(l0.elem_slot, l0.n_elems,
                                                                  l0.slot_elem);
    GMT_LAUNCH_CHECK();
  }
  return l0.slot_elem;
}

void launch_energy_per(gmt_hierarchy* h, Prec prec, const void* u_hi, const float* u_lo,
                       double* per, double scale) {
  const bool d3 = h->mat.D == 3;
  if (prec == P64) {
    if (d3) energy_t<double, 3, 6, false>(h, u_hi, nullptr, nullptr, per, scale);
    else energy_t<double, 1, 3, false>(h, u_hi, nullptr, nullptr, per, scale);
  } else {
    if (d3) energy_t<float, 3, 6, true>(h, u_hi, u_lo, nullptr, per, scale);
    else energy_t<float, 1, 3, true>(h, u_hi, u_lo, nullptr, per, scale);
  }
}

void launch_energy(gmt_hierarchy* h, Prec prec, const void* u_hi, const float* u_lo,
                   double* part) {
  const bool d3 = h->mat.D == 3;
  if (prec == P64) {
    if (d3) energy_t<double, 3, 6, false>(h, u_hi, nullptr, part);
    else energy_t<double, 1, 3, false>(h, u_hi, nullptr, part);
  } else {
    if (d3) energy_t<float, 3, 6, true>(h, u_hi, u_lo, part);
    else energy_t<float, 1, 3, true>(h, u_hi, u_lo, part);
  }
}

static void reduce_groups(gmt_hierarchy* h, const double* part, int64_t nblk, int ld,
                          const RedGroups& g) {
  int K = 0;
  for (int i = 0; i < g.n; ++i) K += g.ncols[i];
  GMT_REQUIRE(g.n >= 1 && g.n <= 3 && K >= 1 && K <= kRedMaxCols, GMT_ERR_ARG,
              "reduction over %d columns", K);
  if (h->red_scratch == nullptr) {
    h->red_scratch = h->geo.alloc<double>(kRedMaxCols * kRedSplit * 2);
    h->red_ticket = h->geo.alloc<unsigned>(kRedMaxCols);
    GMT_CUDA(cudaMemsetAsync(h->red_ticket, 0, kRedMaxCols * sizeof(unsigned), h->stream));
  }
  // about 2048 rows per block, at most kRedSplit blocks per column
  const int S = (int)std::min<int64_t>(kRedSplit, std::max<int64_t>(1, (nblk + 2047) / 2048));
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)nblk * K * 8.0);
  k_reduce<<<dim3(K, S), 256, 0, h->stream>>>(part, nblk, ld, g, h->red_scratch,
                                             h->red_ticket);
  GMT_LAUNCH_CHECK();
}

void launch_reduce(gmt_hierarchy* h, const double* part, int64_t nblk, int K, double* out,
                   RedEpi epi, int ld) {
  RedGroups g;
  g.n = 1;
  g.ncols[0] = K;
  g.out[0] = out;
  g.epi[0] = epi;
  reduce_groups(h, part, nblk, ld <= 0 ? K : ld, g);
}

void launch_reduce_multi(gmt_hierarchy* h, const double* part, int64_t nblk, int ld, int n,
                         const int* col0, const int* ncols, double* const* out,
                         const RedEpi* epi) {
  RedGroups g;
  g.n = n;
  for (int i = 0; i < n && i < 3; ++i) {
    g.col0[i] = col0[i];
    g.ncols[i] = ncols[i];
    g.out[i] = out[i];
    g.epi[i] = epi[i];
  }
  reduce_groups(h, part, nblk, ld, g);
}

static int64_t nvals(gmt_hierarchy* h, int level) { return h->lv[level].nslots * h->mat.C; }

void vec_zero(gmt_hierarchy* h, int level, Prec prec, void* x) {
  const int64_t n = nvals(h, level);
  if (prec == P64) k_vzero<double><<<grid_for(n, 256), 256, 0, h->stream>>>((double*)x, n);
  else if (prec == P32) k_vzero<float><<<grid_for(n, 256), 256, 0, h->stream>>>((float*)x, n);
  else k_vzero<__nv_bfloat16><<<grid_for(n, 256), 256, 0, h->stream>>>((__nv_bfloat16*)x, n);
  GMT_LAUNCH_CHECK();
}

void vec_copy(gmt_hierarchy* h, int level, Prec prec, const void* a, void* b) {
  GMT_CUDA(cudaMemcpyAsync(b, a, nvals(h, level) * prec_bytes(prec), cudaMemcpyDeviceToDevice,
                           h->stream));
}

void vec_add(gmt_hierarchy* h, int level, Prec prec, const void* y, void* x) {
  const int64_t n = nvals(h, level);
  if (prec == P64) k_vadd<double><<<grid_for(n, 256), 256, 0, h->stream>>>((const double*)y, (double*)x, n);
  else if (prec == P32) k_vadd<float><<<grid_for(n, 256), 256, 0, h->stream>>>((const float*)y, (float*)x, n);
  else k_vadd<__nv_bfloat16><<<grid_for(n, 256), 256, 0, h->stream>>>((const __nv_bfloat16*)y, (__nv_bfloat16*)x, n);
  GMT_LAUNCH_CHECK();
}


template <typename TS, int M, int C>
static void vdot_dispatch(const void* x, const void* y, double* part, unsigned g, cudaStream_t s) {
  k_vdot<TS, M, C><<<g, 64, 0, s>>>((const TS*)x, (const TS*)y, part);
}

void vec_dot(gmt_hierarchy* h, int level, Prec prec, const void* x, const void* y, double* part) {
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)h->lv[level].n_nodes * h->mat.C * 2 * prec_bytes(prec));
  const unsigned g = (unsigned)h->lv[level].nb;
  if (h->mat.D == 3) {
    if (prec == P64) vdot_dispatch<double, 6, 18>(x, y, part, g, h->stream);
    else if (prec == P32) vdot_dispatch<float, 6, 18>(x, y, part, g, h->stream);
    else vdot_dispatch<__nv_bfloat16, 6, 18>(x, y, part, g, h->stream);
  } else {
    if (prec == P64) vdot_dispatch<double, 3, 3>(x, y, part, g, h->stream);
    else if (prec == P32) vdot_dispatch<float, 3, 3>(x, y, part, g, h->stream);
    else vdot_dispatch<__nv_bfloat16, 3, 3>(x, y, part, g, h->stream);
  }
  GMT_LAUNCH_CHECK();
}

template <typename TS, int M, int C>
static void cgu(const double* alpha, const int* act, void* x, const void* p, void* r,
                const void* q, double* part, bool sums, unsigned g, cudaStream_t s) {
  if (sums)
    k_cg_update<TS, M, C, true><<<g, 64, 0, s>>>(alpha, act, (TS*)x, (const TS*)p, (TS*)r,
                                                 (const TS*)q, part);
  else
    k_cg_update<TS, M, C, false><<<g, 64, 0, s>>>(alpha, act, (TS*)x, (const TS*)p, (TS*)r,
                                                  (const TS*)q, part);
}

void vec_cg_update(gmt_hierarchy* h, Prec prec, const double* alpha, const int* active,
                   void* x, const void* p, void* r, const void* q, double* part, bool sums) {
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)h->lv[0].n_nodes * h->mat.C * 6 * prec_bytes(prec));
  const unsigned g = (unsigned)h->lv[0].nb;
  if (h->mat.D == 3) {
    if (prec == P64) cgu<double, 6, 18>(alpha, active, x, p, r, q, part, sums, g, h->stream);
    else cgu<float, 6, 18>(alpha, active, x, p, r, q, part, sums, g, h->stream);
  } else {
    if (prec == P64) cgu<double, 3, 3>(alpha, active, x, p, r, q, part, sums, g, h->stream);
    else cgu<float, 3, 3>(alpha, active, x, p, r, q, part, sums, g, h->stream);
  }
  GMT_LAUNCH_CHECK();
}

template <typename TS, int M, int C>
static void cgd(const double* beta, const void* z, void* p, const float* zmean,
                const uint8_t* mask, unsigned g, cudaStream_t s) {
  k_cg_dir<TS, M, C><<<g, 64, 0, s>>>(beta, (const TS*)z, (TS*)p, zmean, mask);
}

void vec_cg_dir(gmt_hierarchy* h, Prec prec, const double* beta, const void* z, void* p,
                const float* zmean) {
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)h->lv[0].n_nodes * h->mat.C * 3 * prec_bytes(prec));
  const unsigned g = (unsigned)h->lv[0].nb;
  const uint8_t* mk = h->lv[0].mask;
  if (h->mat.D == 3) {
    if (prec == P64) cgd<double, 6, 18>(beta, z, p, nullptr, mk, g, h->stream);
    else cgd<float, 6, 18>(beta, z, p, zmean, mk, g, h->stream);
  } else {
    if (prec == P64) cgd<double, 3, 3>(beta, z, p, nullptr, mk, g, h->stream);
    else cgd<float, 3, 3>(beta, z, p, zmean, mk, g, h->stream);
  }
  GMT_LAUNCH_CHECK();
}

void vec_ff_add(gmt_hierarchy* h, const float* d, float* hi, float* lo) {
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)h->lv[0].n_nodes * h->mat.C * 5 * prec_bytes(P32));
  const int64_t n = nvals(h, 0);
  k_ff_add<<<grid_for(n, 256), 256, 0, h->stream>>>(d, hi, lo, n);
  GMT_LAUNCH_CHECK();
}

void vec_ff_sub_mean(gmt_hierarchy* h, const float* mean, float* hi, float* lo) {
  const unsigned g = (unsigned)h->lv[0].nb;
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)h->lv[0].n_nodes * h->mat.C * 16.0);
  if (h->mat.C == 18) k_ff_sub_mean<18><<<g, 64, 0, h->stream>>>(mean, h->lv[0].mask, hi, lo);
  else k_ff_sub_mean<3><<<g, 64, 0, h->stream>>>(mean, h->lv[0].mask, hi, lo);
  GMT_LAUNCH_CHECK();
}

void vec_sum_ff(gmt_hierarchy* h, const float* hi, const float* lo, double* part) {
  const unsigned g = (unsigned)h->lv[0].nb;
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)h->lv[0].n_nodes * h->mat.C * 8.0);
  if (h->mat.C == 18) k_sum_ff<18><<<g, 64, 0, h->stream>>>(hi, lo, h->lv[0].mask, part);
  else k_sum_ff<3><<<g, 64, 0, h->stream>>>(hi, lo, h->lv[0].mask, part);
  GMT_LAUNCH_CHECK();
}

void vec_sum_values(gmt_hierarchy* h, int level, Prec prec, const void* x, const float* lo,
                    double* part) {
  const unsigned g = (unsigned)h->lv[level].nb;
  const uint8_t* mk = h->lv[level].mask;
  if (h->mat.C == 18) {
    if (prec == P64) k_sum_values<double, 18><<<g, 64, 0, h->stream>>>((const double*)x, lo, mk, part);
    else k_sum_values<float, 18><<<g, 64, 0, h->stream>>>((const float*)x, lo, mk, part);
  } else {
    if (prec == P64) k_sum_values<double, 3><<<g, 64, 0, h->stream>>>((const double*)x, lo, mk, part);
    else k_sum_values<float, 3><<<g, 64, 0, h->stream>>>((const float*)x, lo, mk, part);
  }
  GMT_LAUNCH_CHECK();
}

void vec_sum_values32(gmt_hierarchy* h, const float* x, double* part) {
  const unsigned g = (unsigned)h->lv[0].nb;
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)h->lv[0].n_nodes * h->mat.C * 4.0);
  if (h->mat.C == 18) k_sum_values32<18><<<g, 64, 0, h->stream>>>(x, h->lv[0].mask, part);
  else k_sum_values32<3><<<g, 64, 0, h->stream>>>(x, h->lv[0].mask, part);
  GMT_LAUNCH_CHECK();
}

void vec_sub_mean32(gmt_hierarchy* h, const float* mean, float* x) {
  const unsigned g = (unsigned)h->lv[0].nb;
  TraceScope ts(&h->tracer, h->stream, TR_VEC, (double)h->lv[0].n_nodes * h->mat.C * 8.0);
  if (h->mat.C == 18) k_sub_mean32<18><<<g, 64, 0, h->stream>>>(mean, h->lv[0].mask, x);
  else k_sub_mean32<3><<<g, 64, 0, h->stream>>>(mean, h->lv[0].mask, x);
  GMT_LAUNCH_CHECK();
}

void vec_sub_mean64(gmt_hierarchy* h, int level, const double* mean, double* x) {
  const int64_t n = nvals(h, level);
  if (h->mat.C == 18) k_sub_mean64<18><<<grid_for(n, 256), 256, 0, h->stream>>>(mean, h->lv[level].mask, x, n);
  else k_sub_mean64<3><<<grid_for(n, 256), 256, 0, h->stream>>>(mean, h->lv[level].mask, x, n);
  GMT_LAUNCH_CHECK();
}

void vec_scale_cases(gmt_hierarchy* h, int level, Prec prec, const double* s, void* x) {
  const int64_t n = nvals(h, level);
  const unsigned g = grid_for(n, 256);
  cudaStream_t st = h->stream;
  if (h->mat.D == 3) {
    if (prec == P64) k_scale_cases<double, 6, 18><<<g, 256, 0, st>>>(s, (double*)x, n);
    else if (prec == P32) k_scale_cases<float, 6, 18><<<g, 256, 0, st>>>(s, (float*)x, n);
    else k_scale_cases<__nv_bfloat16, 6, 18><<<g, 256, 0, st>>>(s, (__nv_bfloat16*)x, n);
  } else {
    if (prec == P64) k_scale_cases<double, 3, 3><<<g, 256, 0, st>>>(s, (double*)x, n);
    else if (prec == P32) k_scale_cases<float, 3, 3><<<g, 256, 0, st>>>(s, (float*)x, n);
    else k_scale_cases<__nv_bfloat16, 3, 3><<<g, 256, 0, st>>>(s, (__nv_bfloat16*)x, n);
  }
  GMT_LAUNCH_CHECK();
}

void canon_to_slots(gmt_hierarchy* h, int level, Prec prec, const double* src, void* dst) {
  const Level& lv = h->lv[level];
  const int C = h->mat.C;
  const int64_t cnt = lv.n_nodes * C;
  vec_zero(h, level, prec, dst);
  if (prec == P64) k_canon_to_slots<double><<<grid_for(cnt, 256), 256, 0, h->stream>>>(src, lv.canon_slot, lv.n_nodes, C, (double*)dst);
  else if (prec == P32) k_canon_to_slots<float><<<grid_for(cnt, 256), 256, 0, h->stream>>>(src, lv.canon_slot, lv.n_nodes, C, (float*)dst);
  else k_canon_to_slots<__nv_bfloat16><<<grid_for(cnt, 256), 256, 0, h->stream>>>(src, lv.canon_slot, lv.n_nodes, C, (__nv_bfloat16*)dst);
  GMT_LAUNCH_CHECK();
}

void slots_to_canon(gmt_hierarchy* h, int level, Prec prec, const void* src, double* dst) {
  const Level& lv = h->lv[level];
  const int C = h->mat.C;
  const int64_t cnt = lv.n_nodes * C;
  if (prec == P64) k_slots_to_canon<double><<<grid_for(cnt, 256), 256, 0, h->stream>>>((const double*)src, lv.canon_slot, lv.n_nodes, C, dst);
  else if (prec == P32) k_slots_to_canon<float><<<grid_for(cnt, 256), 256, 0, h->stream>>>((const float*)src, lv.canon_slot, lv.n_nodes, C, dst);
  else k_slots_to_canon<__nv_bfloat16><<<grid_for(cnt, 256), 256, 0, h->stream>>>((const __nv_bfloat16*)src, lv.canon_slot, lv.n_nodes, C, dst);
  GMT_LAUNCH_CHECK();
}

void canon_to_ff(gmt_hierarchy* h, const double* src, float* hi, float* lo) {
  const Level& lv = h->lv[0];
  const int C = h->mat.C;
  vec_zero(h, 0, P32, hi);
  vec_zero(h, 0, P32, lo);
  k_canon_to_ff<<<grid_for(lv.n_nodes * C, 256), 256, 0, h->stream>>>(src, lv.canon_slot, lv.n_nodes, C, hi, lo);
  GMT_LAUNCH_CHECK();
}

void ff_to_canon(gmt_hierarchy* h, const float* hi, const float* lo, double* dst) {
  const Level& lv = h->lv[0];
  const int C = h->mat.C;
  k_ff_to_canon<<<grid_for(lv.n_nodes * C, 256), 256, 0, h->stream>>>(hi, lo, lv.canon_slot, lv.n_nodes, C, dst);
  GMT_LAUNCH_CHECK();
}

void ff_to_f64(gmt_hierarchy* h, const float* hi, const float* lo, double* dst) {
  const int64_t n = nvals(h, 0);
  k_ff_to_f64<<<grid_for(n, 256), 256, 0, h->stream>>>(hi, lo, dst, n);
  GMT_LAUNCH_CHECK();
}

void f64_to_f32(gmt_hierarchy* h, const double* src, float* dst) {
  const int64_t n = nvals(h, 0);
  k_f64_to_f32<<<grid_for(n, 256), 256, 0, h->stream>>>(src, dst, n);
  GMT_LAUNCH_CHECK();
}

}  // namespace gmt
