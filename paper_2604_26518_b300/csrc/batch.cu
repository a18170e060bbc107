// Batched V-cycle phases: one launch per phase over the bricks (or slots, or rows) of many
// lattices at once. Every block finds its lattice from the prefix sums of the per-lattice
// block counts and then does exactly the work, in the same order, that the single-lattice
// kernel does for that brick, so a batched V-cycle is bitwise the per-lattice one. The
// small coarse levels of one lattice fill a fraction of one wave; a batch of them fills the
// GPU, and the launch count of a V-cycle no longer grows with the number of lattices.
// Per-lattice pointers travel in the kernel parameters (at most kBatchMax lattices).
// FP32 vectors (the mixed-precision V-cycle), damped-Jacobi smoothing.
#include <memory>

#include "stencil_op.cuh"
#include "transfer.cuh"

namespace gmt {

namespace {

// block b of a batched launch belongs to lattice l with start[l] <= b < start[l + 1]
__device__ __forceinline__ int lattice_of(const int64_t* start, int n, int64_t b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// one lattice's view for stencil_brick / diag_slot (the material's FineC is shared)
template <typename TS, typename A, int D, int M>
struct LatView {
  const uint8_t* mask;
  const A* kmat;
  const A* dinv;
  const TS* f;
  const TS* dprev;
  const TS* aux;
  TS* out;
  TS* dout;
  double* part;
  A omega, c1, c2;
  int colour;
  A kscale;
  const FineC<A, D, M>& fc;
};

template <typename TS, typename A>
struct StPtrs {
  const int* nbr;
  const uint8_t* mask;
  const A* kmat;
  const A* dinv;
  const TS* u;
  const TS* f;
  TS* out;
  int64_t nslots;
  double* part;    // SUMS: the sweep's per-brick partials (see stencil_brick)
  const TS* aux;   // SUMS: the vector dotted with the result per case (or nullptr)
  A kscale;        // KIND 2: the scale of the FP16 stencils
};

template <typename TS, typename A, int D, int M>
struct MultiSt {
  FineC<A, D, M> fc;
  A omega;
  int n;
  int64_t start[kBatchMax + 1];
  StPtrs<TS, A> lp[kBatchMax];
};

// the stencil sweep (Jacobi or residual) of brick b of lattice l, as k_stencil does it;
// SUMS: a Jacobi sweep that also writes the fused Krylov partials
template <typename TS, typename A, int D, int M, int KIND, int MODE, bool SUMS = false>
__global__ void __launch_bounds__(64) k_stencil_multi(const __grid_constant__ MultiSt<TS, A, D, M> mp) {
  using V = typename Vec16<A>::type;
  constexpr int C = D * M, NV = Vec16<A>::n, G = (C + NV - 1) / NV;
  __shared__ V tile[G * 216];
  __shared__ int nb[27];
  const int t = threadIdx.x;
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const int64_t b = (int64_t)blockIdx.x - mp.start[l];
  const StPtrs<TS, A>& lp = mp.lp[l];
  if (t < 27) nb[t] = lp.nbr[b * 27 + t];
  __syncthreads();
  constexpr bool PREF = KIND == 0 && (MODE == ST_JACOBI || MODE == ST_RESID);
  A fpre[PREF ? C : 1];
  if constexpr (PREF) {
    const TS* fo = lp.f + b * (64 * C) + own_local(t);
#pragma unroll
    for (int v = 0; v < C; ++v) fpre[v] = load_as<A>(fo + v * 64);
  }
  A self[C];
  stage_tile<TS, A, C>(lp.u, b, t, nb, tile, self);
  __syncthreads();
  const LatView<TS, A, D, M> v{lp.mask, lp.kmat, lp.dinv, lp.f, nullptr, lp.aux, lp.out,
                               nullptr, lp.part, mp.omega, A(0), A(0), -1, lp.kscale, mp.fc};
  stencil_brick<TS, A, D, M, KIND, MODE, SUMS, PREF>(v, b, tile, fpre, self);
}

// first smoothing step from zero, slots of lattice l in blocks of 128
template <typename TS, typename A, int D, int M, int KIND>
__global__ void k_diag_multi(const __grid_constant__ MultiSt<TS, A, D, M> mp) {
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const StPtrs<TS, A>& lp = mp.lp[l];
  const int64_t slot = ((int64_t)blockIdx.x - mp.start[l]) * 128 + threadIdx.x;
  if (slot >= lp.nslots) return;
  const LatView<TS, A, D, M> v{lp.mask, lp.kmat, lp.dinv, lp.f, nullptr, nullptr, lp.out,
                               nullptr, nullptr, mp.omega, A(0), A(0), -1, lp.kscale, mp.fc};
  diag_slot<TS, A, D, M, KIND>(v, slot);
}

template <typename TS>
struct TrPtrs {
  LvView f, c;
  const TS* in;
  TS* out;
};
template <typename TS>
struct MultiTr {
  int n;
  int64_t start[kBatchMax + 1];
  TrPtrs<TS> lp[kBatchMax];
};

template <typename TS, typename A, int C>
__global__ void __launch_bounds__(256) k_restrict_tile_multi(const __grid_constant__ MultiTr<TS> mp) {
  extern __shared__ __align__(16) unsigned char btr_smem[];
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const TrPtrs<TS>& lp = mp.lp[l];
  restrict_brick<TS, A, C>(lp.in, lp.out, lp.f, lp.c, (int64_t)blockIdx.x - mp.start[l],
                           reinterpret_cast<typename Vec16<A>::type*>(btr_smem));
}

template <typename TS, typename A, int C>
__global__ void k_restrict_node_multi(const __grid_constant__ MultiTr<TS> mp) {
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const TrPtrs<TS>& lp = mp.lp[l];
  restrict_node<TS, A, C>(lp.in, lp.out, lp.f, lp.c,
                          ((int64_t)blockIdx.x - mp.start[l]) * 64 + threadIdx.x);
}

template <typename TS, typename A, int C>
__global__ void __launch_bounds__(64) k_prolong_tile_multi(const __grid_constant__ MultiTr<TS> mp) {
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const TrPtrs<TS>& lp = mp.lp[l];
  prolong_brick<TS, A, C>(lp.in, lp.out, lp.f, lp.c, (int64_t)blockIdx.x - mp.start[l]);
}

template <typename TS, typename A, int C>
__global__ void k_prolong_node_multi(const __grid_constant__ MultiTr<TS> mp) {
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const TrPtrs<TS>& lp = mp.lp[l];
  prolong_node<TS, A, C>(lp.in, lp.out, lp.f, lp.c,
                         ((int64_t)blockIdx.x - mp.start[l]) * 64 + threadIdx.x);
}

struct CsPtrs {
  const float* f;          // coarsest right-hand side (slot layout)
  float* u;                // coarsest solution (slot layout)
  const int* canon_slot;
  int64_t nn;              // coarsest nodes
  int64_t nvals;           // slots x values (zeroing)
  const float* X;          // FP32 generalized inverse, m x m
  int64_t m;
  double* cb;
  float* cb32;
  double* cu;
};
struct MultiCs {
  int n;
  int64_t start[kBatchMax + 1];
  CsPtrs lp[kBatchMax];
};

template <int D, int M>
__global__ void k_coarse_gather_multi(const __grid_constant__ MultiCs mp) {
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const CsPtrs& lp = mp.lp[l];
  coarse_gather_at<float, D, M>(lp.f, lp.canon_slot, lp.nn, lp.cb, lp.cb32,
                                ((int64_t)blockIdx.x - mp.start[l]) * 256 + threadIdx.x);
}

template <int M>
__global__ void __launch_bounds__(256) k_coarse_gemv32_multi(const __grid_constant__ MultiCs mp) {
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const CsPtrs& lp = mp.lp[l];
  coarse_gemv32_row<M>(lp.X, lp.cb32, lp.m, nullptr, lp.cu,
                       ((int64_t)blockIdx.x - mp.start[l]) * 8 + (threadIdx.x >> 5));
}

template <int D, int M>
__global__ void k_coarse_scatter_multi(const __grid_constant__ MultiCs mp) {
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const CsPtrs& lp = mp.lp[l];
  coarse_scatter_at<float, D, M>(lp.cu, lp.canon_slot, lp.nn, lp.u,
                                 ((int64_t)blockIdx.x - mp.start[l]) * 256 + threadIdx.x);
}

__global__ void k_zero_multi(const __grid_constant__ MultiCs mp) {
  const int l = lattice_of(mp.start, mp.n, blockIdx.x);
  const CsPtrs& lp = mp.lp[l];
  const int64_t i = ((int64_t)blockIdx.x - mp.start[l]) * 256 + threadIdx.x;
  if (i < lp.nvals) lp.u[i] = 0.f;
}

}  // namespace

// ------------------------------------------------------------------ host launchers
static unsigned nblocks(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// one launch over the lattices `sel` of hs (diag: the first smoothing step from zero)
template <int D, int M>
static void stencil_multi_t(gmt_hierarchy* const* hs, const std::vector<int>& sel,
                            cudaStream_t s, int level, StencilMode mode, const void* const* u,
                            const void* const* f, void* const* out, double* const* part,
                            const void* const* aux, double omega, bool diag) {
  using TS = float;
  using A = float;
  if (sel.empty()) return;
  auto mp = std::make_unique<MultiSt<TS, A, D, M>>();
  std::memset(mp.get(), 0, sizeof(*mp));
  fill_fine<A, D, M>(hs[0]->mat, mp->fc);
  mp->omega = (A)omega;
  mp->n = (int)sel.size();
  const bool fine = level == 0;
  const bool half = !fine && hs[0]->opts.coarse_fp16 != 0;   // KIND 2 (as stencil_t)
  const bool sums = part != nullptr && part[sel[0]] != nullptr;
  int64_t tot = 0;
  for (int k = 0; k < mp->n; ++k) {
    const int i = sel[k];
    Level& lv = hs[i]->lv[level];
    GMT_REQUIRE(fine || (half ? lv.S16 != nullptr : lv.S32 != nullptr), GMT_ERR_STATE,
                "batched sweep: level %d stencils of lattice %d are not built", level, i);
    mp->start[k] = tot;
    tot += diag ? (int64_t)nblocks(lv.nslots, 128) : lv.nb;
    mp->lp[k] = StPtrs<TS, A>{lv.brick_nbr, lv.mask,
                              half ? (const A*)lv.S16 : (const A*)lv.S32, (const A*)lv.dinv32,
                              (const TS*)u[i], (const TS*)f[i], (TS*)out[i], lv.nslots,
                              sums ? part[i] : nullptr,
                              sums && aux ? (const TS*)aux[i] : nullptr, (A)lv.s16_scale};
  }
  mp->start[mp->n] = tot;
  if (tot == 0) return;
  const unsigned g = (unsigned)tot;
  if (diag) {
    if (fine) k_diag_multi<TS, A, D, M, 0><<<g, 128, 0, s>>>(*mp);
    else k_diag_multi<TS, A, D, M, 1><<<g, 128, 0, s>>>(*mp);
  } else if (mode == ST_JACOBI && sums) {
    k_stencil_multi<TS, A, D, M, 0, ST_JACOBI, true><<<g, 64, 0, s>>>(*mp);
  } else if (mode == ST_JACOBI) {
    if (fine) k_stencil_multi<TS, A, D, M, 0, ST_JACOBI><<<g, 64, 0, s>>>(*mp);
    else if (half) k_stencil_multi<TS, A, D, M, 2, ST_JACOBI><<<g, 64, 0, s>>>(*mp);
    else k_stencil_multi<TS, A, D, M, 1, ST_JACOBI><<<g, 64, 0, s>>>(*mp);
  } else {
    if (fine) k_stencil_multi<TS, A, D, M, 0, ST_RESID><<<g, 64, 0, s>>>(*mp);
    else if (half) k_stencil_multi<TS, A, D, M, 2, ST_RESID><<<g, 64, 0, s>>>(*mp);
    else k_stencil_multi<TS, A, D, M, 1, ST_RESID><<<g, 64, 0, s>>>(*mp);
  }
  GMT_LAUNCH_CHECK();
}

static void check_batch(gmt_hierarchy* const* hs, int n) {
  GMT_REQUIRE(n >= 1 && n <= kBatchMax, GMT_ERR_ARG, "batch of %d lattices (1..%d)", n, kBatchMax);
  for (int i = 1; i < n; ++i)
    GMT_REQUIRE(hs[i]->mat.D == hs[0]->mat.D, GMT_ERR_ARG, "batched launch mixes physics");
}

template <int D, int M>
static void stencil_split_t(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                            StencilMode mode, const void* const* u, const void* const* f,
                            void* const* out, double* const* part, const void* const* aux,
                            double omega, bool diag) {
  // lattices with and without the fused partials go to separate launches
  std::vector<int> with, without;
  for (int i = 0; i < n; ++i) (part && part[i] ? with : without).push_back(i);
  stencil_multi_t<D, M>(hs, without, s, level, mode, u, f, out, nullptr, nullptr, omega, diag);
  stencil_multi_t<D, M>(hs, with, s, level, mode, u, f, out, part, aux, omega, diag);
}

void prepare_batched_levels(gmt_hierarchy* h) {
  for (int l = 1; l + 1 < h->L; ++l) {
    build_node_stencils(h, l, false);
    if (h->opts.coarse_fp16) build_node_stencils16(h, l);
  }
}

void batch_stencil(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                   StencilMode mode, const void* const* u, const void* const* f,
                   void* const* out, double* const* part, const void* const* aux) {
  check_batch(hs, n);
  GMT_REQUIRE(mode == ST_JACOBI || mode == ST_RESID, GMT_ERR_ARG, "batched stencil mode");
  GMT_REQUIRE(part == nullptr || (level == 0 && mode == ST_JACOBI), GMT_ERR_ARG,
              "fused partials belong to a level-0 smoothing sweep");
  const double om = hs[0]->opts.omega;
  if (hs[0]->mat.D == 3) stencil_split_t<3, 6>(hs, n, s, level, mode, u, f, out, part, aux, om, false);
  else stencil_split_t<1, 3>(hs, n, s, level, mode, u, f, out, part, aux, om, false);
}

void batch_diag(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                const void* const* f, void* const* out, double scale) {
  check_batch(hs, n);
  if (hs[0]->mat.D == 3)
    stencil_split_t<3, 6>(hs, n, s, level, ST_JACOBI, f, f, out, nullptr, nullptr, scale, true);
  else
    stencil_split_t<1, 3>(hs, n, s, level, ST_JACOBI, f, f, out, nullptr, nullptr, scale, true);
}

template <int C>
static void transfer_multi_t(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                             const void* const* in, void* const* out, bool restrict_) {
  using TS = float;
  using A = float;
  // two launches at most: lattices whose two levels are both bricked (tiled form) and the
  // others (a dense coarsest level: per-node form)
  for (int tiled = 1; tiled >= 0; --tiled) {
    auto mp = std::make_unique<MultiTr<TS>>();
    std::memset(mp.get(), 0, sizeof(*mp));
    int k = 0;
    int64_t tot = 0;
    for (int i = 0; i < n; ++i) {
      const Level& fl = hs[i]->lv[level];
      const Level& cl = hs[i]->lv[level + 1];
      const bool t = !fl.dense && !cl.dense;
      if (t != (tiled == 1)) continue;
      mp->start[k] = tot;
      if (restrict_) tot += tiled ? cl.nb : (int64_t)nblocks(cl.nslots, 64);
      else tot += tiled ? fl.nb : (int64_t)nblocks(fl.nslots, 64);
      mp->lp[k] = TrPtrs<TS>{view(fl), view(cl), (const TS*)in[i], (TS*)out[i]};
      ++k;
    }
    if (k == 0 || tot == 0) continue;
    mp->n = k;
    mp->start[k] = tot;
    const unsigned g = (unsigned)tot;
    if (restrict_) {
      if (tiled) {
        constexpr size_t smem = (size_t)vec_groups<A>(C) * 729 * 16;
        ensure_smem_attr((const void*)k_restrict_tile_multi<TS, A, C>, (int)smem);
        k_restrict_tile_multi<TS, A, C><<<g, 256, smem, s>>>(*mp);
      } else {
        k_restrict_node_multi<TS, A, C><<<g, 64, 0, s>>>(*mp);
      }
    } else {
      if (tiled) k_prolong_tile_multi<TS, A, C><<<g, 64, 0, s>>>(*mp);
      else k_prolong_node_multi<TS, A, C><<<g, 64, 0, s>>>(*mp);
    }
    GMT_LAUNCH_CHECK();
  }
}

void batch_restrict(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                    const void* const* rf, void* const* fc) {
  check_batch(hs, n);
  if (hs[0]->mat.D == 3) transfer_multi_t<18>(hs, n, s, level, rf, fc, true);
  else transfer_multi_t<3>(hs, n, s, level, rf, fc, true);
}

void batch_prolong(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                   const void* const* uc, void* const* uf) {
  check_batch(hs, n);
  if (hs[0]->mat.D == 3) transfer_multi_t<18>(hs, n, s, level, uc, uf, false);
  else transfer_multi_t<3>(hs, n, s, level, uc, uf, false);
}

template <typename Kern, typename Count>
static void launch_cs(MultiCs& mp, int n, Kern kern, Count count, int per, cudaStream_t s) {
  int64_t tot = 0;
  for (int i = 0; i < n; ++i) {
    mp.start[i] = tot;
    tot += nblocks(count(mp.lp[i]), per);
  }
  mp.start[n] = tot;
  if (tot == 0) return;
  kern<<<(unsigned)tot, 256, 0, s>>>(mp);
  GMT_LAUNCH_CHECK();
}

template <int D, int M>
static void coarse_multi_t(gmt_hierarchy* const* hs, int n, cudaStream_t s, const void* const* f,
                           void* const* u) {
  constexpr int C = D * M;
  auto mp = std::make_unique<MultiCs>();
  std::memset(mp.get(), 0, sizeof(*mp));
  mp->n = n;
  for (int i = 0; i < n; ++i) {
    gmt_hierarchy* h = hs[i];
    const Level& c = h->lv[h->L - 1];
    mp->lp[i] = CsPtrs{(const float*)f[i], (float*)u[i], c.canon_slot, c.n_nodes, c.nslots * C,
                       h->X32, h->m, h->cb, h->cb32, h->cu};
  }
  launch_cs(*mp, n, k_coarse_gather_multi<D, M>, [](const CsPtrs& p) { return p.nn * C; }, 256, s);
  launch_cs(*mp, n, k_coarse_gemv32_multi<M>, [](const CsPtrs& p) { return p.m; }, 8, s);
  launch_cs(*mp, n, k_zero_multi, [](const CsPtrs& p) { return p.nvals; }, 256, s);
  launch_cs(*mp, n, k_coarse_scatter_multi<D, M>, [](const CsPtrs& p) { return p.nn * C; }, 256, s);
}

void batch_coarse_solve(gmt_hierarchy* const* hs, int n, cudaStream_t s, const void* const* f,
                        void* const* u) {
  check_batch(hs, n);
  if (hs[0]->mat.D == 3) coarse_multi_t<3, 6>(hs, n, s, f, u);
  else coarse_multi_t<1, 3>(hs, n, s, f, u);
}

void batch_zero(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level, void* const* x) {
  check_batch(hs, n);
  auto mp = std::make_unique<MultiCs>();
  std::memset(mp.get(), 0, sizeof(*mp));
  mp->n = n;
  for (int i = 0; i < n; ++i) {
    mp->lp[i].u = (float*)x[i];
    mp->lp[i].nvals = hs[i]->lv[level].nslots * hs[i]->mat.C;
  }
  launch_cs(*mp, n, k_zero_multi, [](const CsPtrs& p) { return p.nvals; }, 256, s);
}

}  // namespace gmt
