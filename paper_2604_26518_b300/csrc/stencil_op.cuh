// Operator kernels of the hot path and their host launch templates, instantiated per
// physics and precision in stencil_el32.cu, stencil_el64.cu and stencil_heat.cu (separate
// translation units so that they compile in parallel): the matrix-free element-by-element
// operator (Sec. 4.6 "Matrix-Free EBE Formulation": K u = sum_e A_e^T K_e A_e u_e), applied
// node by node, the damped block-Jacobi / Chebyshev smoother (Sec. 4.6 "Parallel Smoothing"
// update form u <- u + omega D^-1 r, all nodes at once), the first smoothing step from zero
// and the float-float outer residual.
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
#pragma once

#include "stencil_dev.cuh"

namespace gmt {

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
// The per-brick work of the stencil kernels, after the tile of brick b (own nodes plus a
// one-node halo, 16-byte groups of values) is in shared memory: this thread's node gets
// acc = sum_d S_n(d) u_{n+d} and the mode's epilogue. self: the node's own values; fpre
// (FPRE): its right-hand side, already loaded.
// P: StArgs, or any parameter view with the same members (the batched launches of
// batch.cu pass one lattice's pointers with the shared material's FineC).
template <typename TS, typename A, int D, int M, int KIND, int MODE, bool SUMS, bool FPRE,
          class P>
__device__ __forceinline__ void stencil_brick(const P& p, int64_t b,
                                              const typename Vec16<A>::type* __restrict__ tile,
                                              const A (&fpre)[FPRE ? D * M : 1],
                                              const A (&self)[D * M]) {
  using V = typename Vec16<A>::type;
  constexpr int C = D * M, R = 8 * D, DD = D * D;
  constexpr int NV = Vec16<A>::n, G = (C + NV - 1) / NV;
  constexpr bool DIFF = MODE == ST_APPLY;
  constexpr bool PREF = FPRE;
  const int t = threadIdx.x;
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
    } else if constexpr (KIND == 2) {
      // FP16 copy (8 coefficients per 16-byte group), scaled by kscale after the sum
      constexpr int NG = node_stencil_groups16(DD);
      const uint4* sten = reinterpret_cast<const uint4*>(p.kmat) + b * (NG * 64) + loc;
      uint4 cur;
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        A S[DD];
#pragma unroll
        for (int k = 0; k < DD; ++k) {
          const int c = d * DD + k;
          if (c % 8 == 0) cur = sten[(c / 8) * 64];
          S[k] = (A)half_of(cur, c % 8);
        }
        if (DIFF && d == 13) continue;
        if constexpr (PK) contribute_s(d, S);
        else contribute(d, S);
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
  if constexpr (KIND == 2) {
    // a rounded product, never contracted into the epilogue's subtraction: every kernel
    // that shares this function rounds the same way (the batched sweeps are bitwise equal)
#pragma unroll
    for (int v = 0; v < C; ++v) acc[v] = __fmul_rn(acc[v], p.kscale);
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
      A fv = A(0);
      if (p.f != nullptr) {
        if constexpr (FPRE) fv = fpre[v];
        else fv = load_as<A>(p.f + base + v * 64);
      } else if constexpr (KIND == 0) {
        // level-0 load from the mask: f_n = sum_{a in mask} (K_e x0)[a]
        const int i = v / M, m = v % M;
#pragma unroll
        for (int a = 0; a < 8; ++a)
          fv += (((mk >> a) & 1u) ? A(1) : A(0)) * p.fc.Fe[(a * D + i) * M + m];
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

template <typename TS, typename A, int D, int M, int KIND, int MODE, bool SUMS = false>
__global__ void __launch_bounds__(64)
    k_stencil(const __grid_constant__ StArgs<TS, A, D, M> p) {
  using V = typename Vec16<A>::type;
  constexpr int C = D * M, NV = Vec16<A>::n, G = (C + NV - 1) / NV;
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
  stencil_brick<TS, A, D, M, KIND, MODE, SUMS, PREF>(p, b, tile, fpre, self);
}

// first smoothing step from a zero initial guess: out = scale * D^-1 f, at one slot
template <typename TS, typename A, int D, int M, int KIND, class P>
__device__ __forceinline__ void diag_slot(const P& p, int64_t slot) {
  constexpr int C = D * M;
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

template <typename TS, typename A, int D, int M, int KIND>
__global__ void k_diag(const __grid_constant__ StArgs<TS, A, D, M> p, int64_t nslots) {
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot < nslots) diag_slot<TS, A, D, M, KIND>(p, slot);
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

// ------------------------------------------------------------------ host launchers

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
  // levels >= 1 of the FP32 V-cycle with coarse_fp16: the FP16 stencil copy (KIND 2)
  const bool half = sizeof(A) == 4 && level > 0 && h->opts.coarse_fp16 != 0;
  if (!fine) build_node_stencils(h, level, sizeof(A) == 8);
  if (half) build_node_stencils16(h, level);
  if constexpr (sizeof(A) == 8) {
    p.kmat = (const A*)lv.S64;
    p.dinv = (const A*)lv.dinv64;
  } else {
    p.kmat = half ? (const A*)lv.S16 : (const A*)lv.S32;
    p.dinv = (const A*)lv.dinv32;
    p.kscale = (A)lv.s16_scale;
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
  // KIND 2 exists for FP32 only (the FP64 instances keep KIND 1 there: never launched)
  constexpr int K2 = sizeof(A) == 4 ? 2 : 1;
  switch (mode) {
    case ST_APPLY:
      if (fine) GMT_ST(0, ST_APPLY); else if (half) GMT_ST(K2, ST_APPLY); else GMT_ST(1, ST_APPLY);
      break;
    case ST_RESID:
      if (fine) GMT_ST(0, ST_RESID); else if (half) GMT_ST(K2, ST_RESID); else GMT_ST(1, ST_RESID);
      break;
    case ST_JACOBI:
      if (sums && fine) k_stencil<TS, A, D, M, 0, ST_JACOBI, true><<<g, 64, 0, s>>>(p);
      else if (sums) k_stencil<TS, A, D, M, 1, ST_JACOBI, true><<<g, 64, 0, s>>>(p);
      else if (fine) GMT_ST(0, ST_JACOBI);
      else if (half) GMT_ST(K2, ST_JACOBI);
      else GMT_ST(1, ST_JACOBI);
      break;
    case ST_CHEB:
      if (sums && fine) k_stencil<TS, A, D, M, 0, ST_CHEB, true><<<g, 64, 0, s>>>(p);
      else if (sums) k_stencil<TS, A, D, M, 1, ST_CHEB, true><<<g, 64, 0, s>>>(p);
      else if (fine) GMT_ST(0, ST_CHEB);
      else if (half) GMT_ST(K2, ST_CHEB);
      else GMT_ST(1, ST_CHEB);
      break;
  }
#undef GMT_ST
  GMT_LAUNCH_CHECK();
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

// per physics / precision instances (stencil_el32.cu, stencil_el64.cu, stencil_heat.cu,
// stencil_bf16.cu)
void stencil_el32(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a);
void stencil_elbf(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a);
void stencil_heatbf(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a);
void diag_elbf(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s);
void diag_heatbf(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s);
void stencil_el64(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a);
void stencil_heat32(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a);
void stencil_heat64(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a);
void diag_el32(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s);
void diag_el64(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s);
void diag_heat32(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s);
void diag_heat64(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s);
void resid_ff_el(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part);
void resid_ff_heat(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part);

}  // namespace gmt
