// Device helpers shared by the stencil, transfer, energy and vector kernels: packed FP32
// pairs, kernel parameter blocks, the 64-thread block reduction, D x D inverses, and the
// brick tile staging (4^3 brick plus a one-node halo in shared memory).
#pragma once

#include <cuda_fp16.h>

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
  A kscale;        // KIND 2: the scale of the FP16 stencils
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
// of FP32); the two warp sums are combined in FP64. NW: the block's warps (2 for 64 threads;
// a larger block calls it with every thread, and the warp sums are added in warp order).
template <int K, typename T, int NW = 2>
__device__ __forceinline__ void block_partial_64(T (&v)[K], double* __restrict__ out) {
  static_assert(K >= 1 && K <= 32, "at most 32 values per thread");
  constexpr int P = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
  constexpr int LP = P == 1 ? 0 : P == 2 ? 1 : P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : 5;
  __shared__ double red[NW][P];
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
  if (threadIdx.x < K) {
    double acc = red[0][threadIdx.x] + red[1][threadIdx.x];
#pragma unroll
    for (int i = 2; i < NW; ++i) acc += red[i][threadIdx.x];
    out[threadIdx.x] = acc;
  }
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
// the FP16 copy: 8 coefficients per 16-byte group, same brick-major layout
__host__ __device__ constexpr int node_stencil_groups16(int DD) { return (27 * DD + 7) / 8; }

// coefficient j (0..7) of a 16-byte group of FP16 values
__device__ __forceinline__ float half_of(const uint4& g, int j) {
  const uint32_t w = j < 2 ? g.x : (j < 4 ? g.y : (j < 6 ? g.z : g.w));
  const unsigned short b = (unsigned short)((j & 1) ? (w >> 16) : (w & 0xffffu));
  return __half2float(__ushort_as_half(b));
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

// FineC for a material: K_e, K_e x0 and the full-mask stencil (also as packed pairs)
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

}  // namespace gmt
