// Kernel launch interface of the hot path (stencil.cu), used by solver.cu and api.cu.
#pragma once

#include "common.cuh"

namespace gmt {

enum StencilMode { ST_APPLY = 0, ST_RESID = 1, ST_JACOBI = 2, ST_CHEB = 3 };

// Precision of a launch: storage type of the vectors and arithmetic type.
enum Prec { P64 = 0, P32 = 1, PBF = 2 };

struct VecArgs {
  const void* u = nullptr;     // input field (tile-loaded with halo)
  const void* f = nullptr;     // right-hand side (nullptr at level 0 RESID: load from masks)
  const void* dprev = nullptr; // Chebyshev previous direction
  void* out = nullptr;
  void* dout = nullptr;
  double* part = nullptr;      // per-block partial sums [blocks][M] (APPLY, RESID); level-0
                               // smoother: [blocks][2M + C] of f . out, aux . out (0 when
                               // aux is null) and the sums of out
  const void* aux = nullptr;   // level-0 smoother with part: second vector dotted with out
  double omega = 0, c1 = 0, c2 = 0;
  int colour = -1;             // ST_JACOBI: update only nodes of this parity colour
                               // (x & 1) + 2 (y & 1) + 4 (z & 1), copy the others; -1 = all
};

// per-node assembled stencils of a coarse level (FP32 or FP64 copy; built once)
void build_node_stencils(gmt_hierarchy* h, int level, bool fp64);
// y/r/u' on one level (bricked levels only)
void launch_stencil(gmt_hierarchy* h, int level, Prec prec, StencilMode mode, const VecArgs& a);
// first smoothing step from a zero guess: out = scale * D^-1 f (and dout = out if non-null)
void launch_diag(gmt_hierarchy* h, int level, Prec prec, const void* f, void* out, void* dout,
                 double scale);
// float-float level-0 residual r = f - K (hi + lo) in difference form, FP32 arithmetic;
// hi == nullptr means u = 0 (r = f)
void launch_resid_ff(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part);
// restriction level -> level+1, prolongation+correction level+1 -> level
void launch_restrict(gmt_hierarchy* h, int level, Prec prec, const void* rf, void* fc);
void launch_prolong(gmt_hierarchy* h, int level, Prec prec, const void* uc, void* uf);
// coarsest solve on slot-layout vectors of the coarsest level
void launch_coarse_solve(gmt_hierarchy* h, Prec prec, const void* f, void* u);
// per-element energies of level 0 -> block partials [blocks][M(M+1)/2]; ff: u = (hi, lo)
void launch_energy(gmt_hierarchy* h, Prec prec, const void* u_hi, const float* u_lo,
                   double* part);
// per-element energies times scale into per[n_elems][M][M] (canonical element order)
void launch_energy_per(gmt_hierarchy* h, Prec prec, const void* u_hi, const float* u_lo,
                       double* per, double scale);
// level-0 slot -> canonical element index (-1 where no element has its origin)
const int* level0_slot_elem(gmt_hierarchy* h);

// deterministic fixed-order reduction of [nblk][K] partials into out[K] (device);
// compensated (Neumaier) per thread
// column reductions: at most kRedMaxCols columns, each split over at most kRedSplit blocks
constexpr int kRedMaxCols = 32;
constexpr int kRedSplit = 16;
// Epilogue of a column reduction (thread 0 of the column's block), so that per-case step
// ratios and per-value means are formed once on the device instead of in every block of
// the vector kernel that consumes them.
struct RedEpi {
  int mode = 0;                  // 0: none; 1: ratio = other / out; 2: ratio = out / other;
                                 // 3: out32 = (float)(out * scale);
                                 // 4: out * scale split into floats: out32[k] (hi) and
                                 //    out32[count + k] (lo);
                                 // 5: ratio = 1 / sqrt(max(out, 1e-300));
                                 // 6: ratio = -other2[k] * out / other[k] (flexible CG beta)
  const double* other = nullptr;
  const double* other2 = nullptr;
  const int* active = nullptr;   // modes 1, 2, 6: ratio 0 for inactive cases (may be null)
  double* ratio = nullptr;
  float* out32 = nullptr;
  double scale = 0.0;
  int count = 0;
};
// columns k < K of rows part[i * ld + k] (ld = K when <= 0)
void launch_reduce(gmt_hierarchy* h, const double* part, int64_t nblk, int K, double* out,
                   RedEpi epi = RedEpi(), int ld = 0);
// n <= 3 column groups of the same [nblk][ld] partials in one launch: group i reduces
// columns col0[i] .. col0[i] + ncols[i] - 1 into out[i] with epilogue epi[i]
void launch_reduce_multi(gmt_hierarchy* h, const double* part, int64_t nblk, int ld, int n,
                         const int* col0, const int* ncols, double* const* out,
                         const RedEpi* epi);

// vector kernels on slot layouts (level `level`, C values per slot)
void vec_zero(gmt_hierarchy* h, int level, Prec prec, void* x);
void vec_copy(gmt_hierarchy* h, int level, Prec prec, const void* src, void* dst);
// part[b][m] = sum x.y over case m (same precision)
void vec_dot(gmt_hierarchy* h, int level, Prec prec, const void* x, const void* y, double* part);
// CG: x += alpha p; r -= alpha q; part = ||r||^2 per case; alpha per case from the device
// (RedEpi mode 1), 0 where active[m] == 0. sums: part rows are [M + C], the sums of the new
// r per value following the norms.
void vec_cg_update(gmt_hierarchy* h, Prec prec, const double* alpha, const int* active,
                   void* x, const void* p, void* r, const void* q, double* part,
                   bool sums = false);
// CG: p = z + beta p with beta per case from the device (RedEpi mode 2); with zmean (device
// means of z per value over active nodes) the mean of z is removed on the fly:
// p = (z - zmean) + beta p
void vec_cg_dir(gmt_hierarchy* h, Prec prec, const double* beta, const void* z, void* p,
                const float* zmean = nullptr);
// per-block FP32 sums of each value of a level-0 FP32 field over active slots
void vec_sum_values32(gmt_hierarchy* h, const float* x, double* part);
// x += y (same precision)
void vec_add(gmt_hierarchy* h, int level, Prec prec, const void* y, void* x);
// float-float: (hi, lo) += d
void vec_ff_add(gmt_hierarchy* h, const float* d, float* hi, float* lo);
// float-float: (hi, lo) -= mean[v] (double means, device)
// (hi, lo) -= mean over active slots, mean as float pairs on the device: hi parts
// mean[0..C), lo parts mean[C..2C) (RedEpi mode 4)
void vec_ff_sub_mean(gmt_hierarchy* h, const float* mean, float* hi, float* lo);
// per-block float-float sums of each value of the level-0 field hi + lo over active slots
void vec_sum_ff(gmt_hierarchy* h, const float* hi, const float* lo, double* part);
// per-block sums of each value over active slots: part[b][C]; ff adds hi + lo
void vec_sum_values(gmt_hierarchy* h, int level, Prec prec, const void* x, const float* lo,
                    double* part);
// x -= mean[v] over active slots (level-0 FP32 field; means on the device, RedEpi mode 3)
void vec_sub_mean32(gmt_hierarchy* h, const float* mean, float* x);
// x -= mean[v] (FP64 field)
void vec_sub_mean64(gmt_hierarchy* h, int level, const double* mean, double* x);
// scale case m of x by s[m] (device doubles)
void vec_scale_cases(gmt_hierarchy* h, int level, Prec prec, const double* s, void* x);

// canonical FP64 <-> slot layouts
void canon_to_slots(gmt_hierarchy* h, int level, Prec prec, const double* src, void* dst);
void slots_to_canon(gmt_hierarchy* h, int level, Prec prec, const void* src, double* dst);
void canon_to_ff(gmt_hierarchy* h, const double* src, float* hi, float* lo);
void ff_to_canon(gmt_hierarchy* h, const float* hi, const float* lo, double* dst);
void ff_to_f64(gmt_hierarchy* h, const float* hi, const float* lo, double* dst);
// level-0 slot field FP64 -> FP32, FP32 -> BF16 (round to nearest even), BF16 -> FP32
void f64_to_f32(gmt_hierarchy* h, const double* src, float* dst);
void f32_to_bf16(gmt_hierarchy* h, const float* src, void* dst);
void bf16_to_f32(gmt_hierarchy* h, const void* src, float* dst);

inline int64_t blocks_of(const Level& lv) { return lv.nb; }

// ---- batched V-cycle phases (batch.cu): one launch on stream s over level `level` of n <=
// kBatchMax lattices (FP32 vectors; the same physics and material prepared on each; levels
// 1..L-2 prepared by prepare_batched_levels). Per-lattice arguments are arrays of n
// pointers, as for the single-lattice launchers. Callers pass only lattices that have the
// operation at that level (a sweep or transfer below their coarsest level).
constexpr int kBatchMax = GMT_BATCH_MAX;
// builds the stored FP32 stencils of levels 1..L-2 that the batched sweeps read
void prepare_batched_levels(gmt_hierarchy* h);
// the FP16 copy of level `level`'s FP32 node stencils (coarse_fp16), built once
void build_node_stencils16(gmt_hierarchy* h, int level);
// damped-Jacobi sweep (mode ST_JACOBI: out = u + omega D^-1 (f - K u)) or residual
// (ST_RESID: out = f - K u). part (level-0 Jacobi only, nullable, entries nullable): the
// lattices with part[i] set also write the fused Krylov partials of the last sweep of a
// V-cycle, dotted with aux[i] (k_stencil's SUMS form).
void batch_stencil(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                   StencilMode mode, const void* const* u, const void* const* f,
                   void* const* out, double* const* part = nullptr,
                   const void* const* aux = nullptr);
// first smoothing step from zero: out = scale D^-1 f
void batch_diag(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                const void* const* f, void* const* out, double scale);
void batch_restrict(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                    const void* const* rf, void* const* fc);
void batch_prolong(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level,
                   const void* const* uc, void* const* uf);
// the coarsest solve of each lattice (its own coarsest level)
void batch_coarse_solve(gmt_hierarchy* const* hs, int n, cudaStream_t s, const void* const* f,
                        void* const* u);
// x[i] = 0 over level `level` of lattice i
void batch_zero(gmt_hierarchy* const* hs, int n, cudaStream_t s, int level, void* const* x);
inline size_t prec_bytes(Prec p) { return p == P64 ? 8 : (p == P32 ? 4 : 2); }

}  // namespace gmt
