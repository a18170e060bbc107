// Per-node stencils of stored operators (coarse levels; level 0 with element densities) and
// the dispatch of the operator kernels (stencil_op.cuh) to their per-physics instances.
#include <algorithm>
#include <cmath>

#include "stencil_op.cuh"

namespace gmt {

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

// FP16 copy of the FP32 node stencils of one level, divided by `scale`
__global__ void k_stencil_to_half(const float* __restrict__ S32, int64_t nslots, int DD,
                                  float inv_scale, __half* __restrict__ S16) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = 27 * DD;
  if (i >= nslots * n) return;
  const int64_t slot = i / n;
  const int c = (int)(i % n);
  const float v = S32[node_stencil_index(slot, c, node_stencil_groups<float>(DD), 4)];
  S16[node_stencil_index(slot, c, node_stencil_groups16(DD), 8)] = __float2half_rn(v * inv_scale);
}

void build_node_stencils16(gmt_hierarchy* h, int level) {
  Level& lv = h->lv[level];
  if (lv.S16 != nullptr) return;
  build_node_stencils(h, level, false);
  TraceScope ts(&h->tracer, h->stream, TR_OPS, 0.0);
  const int D = h->mat.D, DD = D * D;
  // every stored coefficient is a sum of at most 8 incident elements' blocks, and a
  // Galerkin level's element matrices are about twice the next finer level's: dividing by
  // 2^level max|K_e| keeps the FP16 values below ~8 (the FP16 range ends at 65504)
  double kmax = 0.0;
  for (int i = 0; i < 64 * DD; ++i) kmax = std::max(kmax, std::fabs(h->mat.Ke[i]));
  const double scale = kmax * std::ldexp(1.0, level);
  lv.s16_scale = (float)scale;
  const size_t cnt = (size_t)lv.nslots * node_stencil_groups16(DD) * 8;
  lv.S16 = h->op.alloc<uint16_t>(cnt);
  GMT_CUDA(cudaMemsetAsync(lv.S16, 0, cnt * sizeof(uint16_t), h->stream));
  const int64_t n = lv.nslots * 27 * DD;
  k_stencil_to_half<<<grid_for(n, 256), 256, 0, h->stream>>>(lv.S32, lv.nslots, DD,
                                                             (float)(1.0 / scale),
                                                             (__half*)lv.S16);
  GMT_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ dispatch
// The V-cycle stores its vectors in FP64, FP32 or BF16 (FP32 arithmetic for the last two).
void launch_stencil(gmt_hierarchy* h, int level, Prec prec, StencilMode mode, const VecArgs& a) {
  if (h->mat.D == 3) {
    if (prec == P64) stencil_el64(h, level, mode, a);
    else if (prec == PBF) stencil_elbf(h, level, mode, a);
    else stencil_el32(h, level, mode, a);
  } else {
    if (prec == P64) stencil_heat64(h, level, mode, a);
    else if (prec == PBF) stencil_heatbf(h, level, mode, a);
    else stencil_heat32(h, level, mode, a);
  }
}

void launch_diag(gmt_hierarchy* h, int level, Prec prec, const void* f, void* out, void* dout,
                 double scale) {
  if (h->mat.D == 3) {
    if (prec == P64) diag_el64(h, level, f, out, dout, scale);
    else if (prec == PBF) diag_elbf(h, level, f, out, dout, scale);
    else diag_el32(h, level, f, out, dout, scale);
  } else {
    if (prec == P64) diag_heat64(h, level, f, out, dout, scale);
    else if (prec == PBF) diag_heatbf(h, level, f, out, dout, scale);
    else diag_heat32(h, level, f, out, dout, scale);
  }
}

void launch_resid_ff(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part) {
  if (h->mat.D == 3) resid_ff_el(h, hi, lo, r, part);
  else resid_ff_heat(h, hi, lo, r, part);
}

}  // namespace gmt
