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
  double* part = nullptr;      // per-block partial sums [blocks][M]
  double omega = 0, c1 = 0, c2 = 0;
};

// per-node assembled stencils of a coarse level (FP32 or FP64 copy; built once)
void build_node_stencils(gmt_hierarchy* h, int level, bool fp64);
// y/r/u' on one level (bricked levels only)
void launch_stencil(gmt_hierarchy* h, int level, Prec prec, StencilMode mode, const VecArgs& a);
// first smoothing step from a zero guess: out = scale * D^-1 f (and dout = out if non-null)
void launch_diag(gmt_hierarchy* h, int level, Prec prec, const void* f, void* out, void* dout,
                 double scale);
// float-float level-0 residual r = f - K (hi + lo) in difference form, FP32 arithmetic
void launch_resid_ff(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part);
// restriction level -> level+1, prolongation+correction level+1 -> level
void launch_restrict(gmt_hierarchy* h, int level, Prec prec, const void* rf, void* fc);
void launch_prolong(gmt_hierarchy* h, int level, Prec prec, const void* uc, void* uf);
// coarsest solve on slot-layout vectors of the coarsest level
void launch_coarse_solve(gmt_hierarchy* h, Prec prec, const void* f, void* u);
// per-element energies of level 0 -> block partials [blocks][M(M+1)/2]; ff: u = (hi, lo)
void launch_energy(gmt_hierarchy* h, Prec prec, const void* u_hi, const float* u_lo,
                   double* part);

// deterministic fixed-order reduction of [nblk][K] partials into out[K] (device);
// compensated (Neumaier) per thread
void launch_reduce(gmt_hierarchy* h, const double* part, int64_t nblk, int K, double* out);

// vector kernels on slot layouts (level `level`, C values per slot)
void vec_zero(gmt_hierarchy* h, int level, Prec prec, void* x);
void vec_copy(gmt_hierarchy* h, int level, Prec prec, const void* src, void* dst);
// part[b][m] = sum x.y over case m (same precision)
void vec_dot(gmt_hierarchy* h, int level, Prec prec, const void* x, const void* y, double* part);
// CG: alpha_m = num[m] / den[m]; x += alpha p; r -= alpha q; part = ||r||^2 per case
void vec_cg_update(gmt_hierarchy* h, Prec prec, const double* num, const double* den,
                   const int* active, void* x, const void* p, void* r, const void* q,
                   double* part);
// CG: beta_m = num[m] / den[m]; p = z + beta p; with zsum (device sums of z per value over
// active nodes) the mean of z is removed on the fly: p = (z - zsum / n) + beta p
void vec_cg_dir(gmt_hierarchy* h, Prec prec, const double* num, const double* den,
                const int* active, const void* z, void* p, const double* zsum = nullptr);
// per-block FP32 sums of each value of a level-0 FP32 field over active slots
void vec_sum_values32(gmt_hierarchy* h, const float* x, double* part);
// x += y (same precision)
void vec_add(gmt_hierarchy* h, int level, Prec prec, const void* y, void* x);
// float-float: (hi, lo) += d
void vec_ff_add(gmt_hierarchy* h, const float* d, float* hi, float* lo);
// float-float: (hi, lo) -= mean[v] (double means, device)
void vec_ff_sub_mean(gmt_hierarchy* h, const double* mean, float* hi, float* lo);
// per-block sums of each value over active slots: part[b][C]; ff adds hi + lo
void vec_sum_values(gmt_hierarchy* h, int level, Prec prec, const void* x, const float* lo,
                    double* part);
// x -= sums[v] / n_active (level-0 FP32 field; sums on the device)
void vec_sub_mean32(gmt_hierarchy* h, const double* sums, float* x);
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
// level-0 slot field FP64 -> FP32
void f64_to_f32(gmt_hierarchy* h, const double* src, float* dst);

inline int64_t blocks_of(const Level& lv) { return lv.nb; }
inline size_t prec_bytes(Prec p) { return p == P64 ? 8 : (p == P32 ? 4 : 2); }

}  // namespace gmt
