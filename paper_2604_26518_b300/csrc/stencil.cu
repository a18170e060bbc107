// Transfers (App. E.2 trilinear prolongation and its transpose, written as gathers), the
// coarsest-level solve (Alg. 1), the element-energy reduction for C^H (App. F.1/F.2), the
// deterministic column reductions and the vector kernels of the solver. The operator and
// smoother kernels are in stencil_op.cu.
#include "stencil_dev.cuh"
#include "transfer.cuh"

namespace gmt {

// ------------------------------------------------------------------ transfer kernels
template <typename TS, typename A, int C>
__global__ void k_restrict(const TS* __restrict__ rf, TS* __restrict__ fc, LvView f, LvView c) {
  restrict_node<TS, A, C>(rf, fc, f, c, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename TS, typename A, int C>
__global__ void k_prolong(const TS* __restrict__ uc, TS* __restrict__ uf, LvView f, LvView c) {
  prolong_node<TS, A, C>(uc, uf, f, c, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename TS, typename A, int C>
__global__ void __launch_bounds__(256) k_restrict_tile(const TS* __restrict__ rf,
                                                       TS* __restrict__ fc, LvView f, LvView c) {
  extern __shared__ __align__(16) unsigned char tr_smem[];
  restrict_brick<TS, A, C>(rf, fc, f, c, blockIdx.x,
                           reinterpret_cast<typename Vec16<A>::type*>(tr_smem));
}

template <typename TS, typename A, int C>
__global__ void __launch_bounds__(64) k_prolong_tile(const TS* __restrict__ uc,
                                                     TS* __restrict__ uf, LvView f, LvView c) {
  prolong_brick<TS, A, C>(uc, uf, f, c, blockIdx.x);
}

// ------------------------------------------------------------------ coarsest solve
template <typename TS, int D, int M>
__global__ void k_coarse_gather(const TS* __restrict__ f, const int* __restrict__ canon_slot,
                                int64_t nn, double* __restrict__ bvec, float* __restrict__ b32) {
  coarse_gather_at<TS, D, M>(f, canon_slot, nn, bvec, b32,
                             (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <int M>
__global__ void __launch_bounds__(256) k_coarse_gemv32(const float* __restrict__ X,
                                                       const float* __restrict__ b32,
                                                       int64_t mrows,
                                                       const double* __restrict__ add,
                                                       double* __restrict__ uvec) {
  coarse_gemv32_row<M>(X, b32, mrows, add, uvec, (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5));
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

template <typename TS, int D, int M>
__global__ void k_coarse_scatter(const double* __restrict__ uvec, const int* __restrict__ canon_slot,
                                 int64_t nn, TS* __restrict__ u) {
  coarse_scatter_at<TS, D, M>(uvec, canon_slot, nn, u,
                              (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
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
// A 128-thread block takes the 64 elements whose origins are the nodes of one brick, two
// threads per element (halves h = 0, 1 of the block). The element's d (or w) for every case
// goes to a column of shared memory (the two halves form the corners 0-3 and 4-7; on the
// float-float path the hi tile is staged and differenced first, then the lo tile in the
// same space). Each case J then forms z = K_e d^J once, in the half that owns J, and dots
// it with d^I for I <= J. The per-pair sums (and the load terms f^I . d^J) live in shared
// memory, reusing the tile space once d is formed. Every value is computed by one thread
// with the same operations in the same order whatever the split. Three resident blocks per
// SM (at most 168 registers; left alone the compiler takes 187 and fits two): 826 -> 638 us
// on a 651 k-node 128^3 cell.
// shared memory: a first region holding the tile, later the pair sums and load terms, then
// the element columns [R*M][64]
template <typename A, int D, int M, bool FF>
constexpr size_t energy_region0_bytes() {
  constexpr int C = D * M, NV = Vec16<A>::n, G = (C + NV - 1) / NV, K = M * (M + 1) / 2;
  constexpr size_t tile = (size_t)G * 216 * 16;
  constexpr size_t sums = (size_t)K * 64 * (FF ? sizeof(float) : sizeof(double)) +
                          (FF ? (size_t)M * M * 64 * sizeof(A) : 0);
  return (tile > sums ? tile : sums + 15) / 16 * 16;
}
template <typename A, int D, int M, bool FF>
constexpr size_t energy_smem_bytes() {
  return energy_region0_bytes<A, D, M, FF>() + (size_t)8 * D * M * 64 * sizeof(A);
}

// the half of the block that forms z = K_e d^J for case J (K_e products balanced 3 : 3, the
// dot products 10 : 11 for six cases)
template <int M>
__device__ __forceinline__ int energy_owner(int J) {
  if constexpr (M == 6) return (J == 0 || J == 2 || J == 5) ? 0 : 1;
  else return J == M - 1 ? 0 : 1;
}

// PER: write each element's energies (times p.scale) instead of the block sums.
template <typename A, int D, int M, bool FF, bool PER = false>
__global__ void __launch_bounds__(128, 3) k_energy(const __grid_constant__ EnArgs<A, D, M> p) {
  using V = typename Vec16<A>::type;
  constexpr int C = D * M, R = 8 * D, K = M * (M + 1) / 2;
  constexpr int NV = Vec16<A>::n, G = (C + NV - 1) / NV;
  // per-pair energies [K][64] (FP32 on the float-float path: per-element rounding, not
  // common to the elements, is summed away in FP64 across blocks), then the load terms
  // phi[I][J] = f^I . d^J [M * M][64], in the tile's region
  using ES = typename std::conditional<FF, float, double>::type;
  extern __shared__ __align__(16) unsigned char en_smem[];
  V* tile = reinterpret_cast<V*>(en_smem);
  A* ws = reinterpret_cast<A*>(en_smem + energy_region0_bytes<A, D, M, FF>());   // [R*M][64]
  ES* es = reinterpret_cast<ES*>(en_smem);
  A* ph = reinterpret_cast<A*>(en_smem + (size_t)K * 64 * sizeof(ES));
  __shared__ int nb[27];
  const int t = threadIdx.x, el = t & 63, half = t >> 6;
  const int64_t b = blockIdx.x;
  if (t < 27) nb[t] = p.nbr[b * 27 + t];
  __syncthreads();
  if (t < 64) {
    A own[C];
    stage_tile<A, A, C>((const A*)p.hi, b, t, nb, tile, own);
  }
  __syncthreads();
  const int q0 = own_q0(el), loc = own_local(el);
  const bool act = (p.mask[b * 64 + loc] & 1u) != 0;  // element with origin at this node
  // phase 1: d (FF: hi part, then lo part added) or w = x0 - d (FP64), corners 4 h .. 4 h + 3
  auto differences = [&](bool lo) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int bb = 4 * half + c;
      const int q = q0 + (bb & 1) + 6 * ((bb >> 1) & 1) + 36 * (bb >> 2);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const V a = tile[g * 216 + q], a0 = tile[g * 216 + q0];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const int v = g * NV + k;
          if (v < C) {
            const int r = (v / M) + D * bb, m = v % M;
            const A du = vec_get<A>(a, k) - vec_get<A>(a0, k);
            A* wp = ws + (r * M + m) * 64 + el;
            if constexpr (FF) *wp = lo ? *wp + du : du;
            else *wp = p.X0[r * M + m] - du;
          }
        }
      }
    }
  };
  if (act) differences(false);
  if constexpr (FF) {
    __syncthreads();   // the hi tile is dead: stage lo in its place
    if (t < 64) {
      A own[C];
      stage_tile<float, A, C>(p.lo, b, t, nb, tile, own);
    }
    __syncthreads();
    if (act) differences(true);
  }
  __syncthreads();  // tiles dead: es (and ph) take their space
  // phase 2 (FF): the load terms, phi[I][J] = (f_hi + f_lo)^I . d^J for the I of this half,
  // then the pair start values phi[I][J] + phi[J][I]
  if constexpr (FF) {
    if (act) {
#pragma unroll 1
      for (int J = 0; J < M; ++J) {
        A d[R];
#pragma unroll
        for (int r = 0; r < R; ++r) d[r] = ws[(r * M + J) * 64 + el];
#pragma unroll
        for (int I = half; I < M; I += 2) {
          A sh = A(0), sl = A(0);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            sh += p.Fh[r * M + I] * d[r];
            sl += p.Fl[r * M + I] * d[r];
          }
          ph[(I * M + J) * 64 + el] = sh + sl;
        }
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int I = 0; I < M; ++I)
#pragma unroll
        for (int J = I; J < M; ++J)
          if (energy_owner<M>(J) == half)
            es[(I * M - I * (I - 1) / 2 + (J - I)) * 64 + el] =
                ph[(I * M + J) * 64 + el] + ph[(J * M + I) * 64 + el];
    }
    // each pair's start value is read back below by the thread that wrote it
  }
  // phase 3: z = K_e d^J (hi + lo in FF), pair sums d^I . z for I <= J, J owned by this half
  if (act) {
#pragma unroll 1
    for (int J = 0; J < M; ++J) {
      if (energy_owner<M>(J) != half) continue;
      A w[R], z[R];
#pragma unroll
      for (int r = 0; r < R; ++r) w[r] = ws[(r * M + J) * 64 + el];
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
          for (int r = 0; r < R; ++r) sacc += ws[(r * M + I) * 64 + el] * z[r];
          ES* ep = es + (I * M - I * (I - 1) / 2 + (J - I)) * 64 + el;
          if constexpr (FF) *ep = sacc - *ep;
          else *ep = sacc;
        }
      }
    }
  }
  __syncthreads();
  if constexpr (PER) {
    if (!act || half) return;
    const int64_t e = p.slot_elem[b * 64 + loc];
    const double fac = p.rho ? p.simp_p * pow(p.rho[b * 64 + loc], p.simp_p - 1.0) : 1.0;
#pragma unroll
    for (int I = 0; I < M; ++I)
#pragma unroll
      for (int J = I; J < M; ++J) {
        double v = (double)es[(I * M - I * (I - 1) / 2 + (J - I)) * 64 + el];
        if constexpr (FF) v += p.C0[I * M + J];
        v *= p.scale * fac;
        p.per[(e * M + I) * M + J] = v;
        p.per[(e * M + J) * M + I] = v;
      }
  } else {
    // the first two warps hold the 64 elements; the other two add zeros
    ES e[K];
    const bool mine = act && half == 0;
    const ES w = (mine && p.coef) ? (ES)p.coef[b * 64 + loc] : ES(1);
#pragma unroll
    for (int k = 0; k < K; ++k) e[k] = mine ? w * es[k * 64 + el] : ES(0);
    block_partial_64<K, ES, 4>(e, p.part + b * K);
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

__global__ void k_f32_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                              int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ src, float* __restrict__ dst,
                              int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __bfloat162float(src[i]);
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
    // u = X f with the FP32 generalized inverse. Its error (~eps32 cond(K_L)) is far below
    // what one V-cycle leaves; a refinement against the FP64 matrix changed no cycle count
    // on the bench or batch cells and cost 3 % of the throughput, so there is none.
    const unsigned g8 = (unsigned)((h->m + 7) / 8);
    k_coarse_gemv32<M><<<g8, 256, 0, h->stream>>>(h->X32, h->cb32, h->m, nullptr, h->cu);
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
    k_energy<A, D, M, FF, true><<<(unsigned)lv.nb, 128, smem, h->stream>>>(p);
  } else {
    ensure_smem_attr((const void*)k_energy<A, D, M, FF>, (int)smem);
    k_energy<A, D, M, FF><<<(unsigned)lv.nb, 128, smem, h->stream>>>(p);
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

void f32_to_bf16(gmt_hierarchy* h, const float* src, void* dst) {
  const int64_t n = nvals(h, 0);
  k_f32_to_bf16<<<grid_for(n, 256), 256, 0, h->stream>>>(src, (__nv_bfloat16*)dst, n);
  GMT_LAUNCH_CHECK();
}

void bf16_to_f32(gmt_hierarchy* h, const void* src, float* dst) {
  const int64_t n = nvals(h, 0);
  k_bf16_to_f32<<<grid_for(n, 256), 256, 0, h->stream>>>((const __nv_bfloat16*)src, dst, n);
  GMT_LAUNCH_CHECK();
}

}  // namespace gmt
