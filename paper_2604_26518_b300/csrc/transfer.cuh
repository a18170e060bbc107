// Transfers (App. E.2 trilinear prolongation and its transpose, written as gathers) and the
// coarsest solve's gather / FP32 product / scatter, as device functions of one node, brick,
// value or row: launched per level by stencil.cu and over many lattices at once by batch.cu.
#pragma once

#include "stencil_dev.cuh"

namespace gmt {

struct LvView {
  int n, nbx;
  bool dense;
  int64_t nslots;
  const int* bmap;
  const int* bxyz;
  const uint8_t* mask;
};

inline LvView view(const Level& l) {
  return LvView{l.n, l.nbx, l.dense, l.nslots, l.brick_map, l.brick_xyz, l.mask};
}

// f_c(j) = sum_{d in {-1,0,1}^3} prod_k (1 - |d_k|/2) r_f(2j + d): the transpose of the
// trilinear prolongation of App. E.2, gathered per coarse node
template <typename TS, typename A, int C>
__device__ __forceinline__ void restrict_node(const TS* __restrict__ rf, TS* __restrict__ fc,
                                              const LvView& f, const LvView& c, int64_t s) {
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
__device__ __forceinline__ void prolong_node(const TS* __restrict__ uc, TS* __restrict__ uf,
                                             const LvView& f, const LvView& c, int64_t s) {
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

// (a 256-thread block; tile: G x 729 16-byte groups of dynamic shared memory)
template <typename TS, typename A, int C>
__device__ __forceinline__ void restrict_brick(const TS* __restrict__ rf, TS* __restrict__ fc,
                                               const LvView& f, const LvView& c, int64_t b,
                                               typename Vec16<A>::type* tile) {
  using V = typename Vec16<A>::type;
  constexpr int NV = Vec16<A>::n, G = (C + NV - 1) / NV;
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
// (a 64-thread block)
template <typename TS, typename A, int C>
__device__ __forceinline__ void prolong_brick(const TS* __restrict__ uc, TS* __restrict__ uf,
                                              const LvView& f, const LvView& c, int64_t b) {
  __shared__ A cv[C][27];
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
__device__ __forceinline__ void coarse_gather_at(const TS* __restrict__ f,
                                                 const int* __restrict__ canon_slot, int64_t nn,
                                                 double* __restrict__ bvec,
                                                 float* __restrict__ b32, int64_t g) {
  if (g >= nn * D * M) return;
  const int64_t i = g / (D * M);
  const int v = (int)(g % (D * M));
  const auto x = load_as<typename ArithOf<TS>::type>(f + vaddr(canon_slot[i], v, D * M));
  bvec[g] = (double)x;
  if (b32) b32[g] = (float)x;
}

// FP32 product with the FP32 generalized inverse: u[r][m] = sum_k X[r][k] b[k][m]
// (+ add[r][m]); one warp per row, lanes over k in a fixed stride, fixed shuffle tree
// (one warp per row r)
template <int M>
__device__ __forceinline__ void coarse_gemv32_row(const float* __restrict__ X,
                                                  const float* __restrict__ b32, int64_t mrows,
                                                  const double* __restrict__ add,
                                                  double* __restrict__ uvec, int64_t r) {
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

template <typename TS, int D, int M>
__device__ __forceinline__ void coarse_scatter_at(const double* __restrict__ uvec,
                                                  const int* __restrict__ canon_slot, int64_t nn,
                                                  TS* __restrict__ u, int64_t g) {
  if (g >= nn * D * M) return;
  const int64_t i = g / (D * M);
  const int v = (int)(g % (D * M));
  u[vaddr(canon_slot[i], v, D * M)] = store_as<TS>((typename ArithOf<TS>::type)uvec[g]);
}


}  // namespace gmt
