// extern "C" boundary of libgmt.so (declarations and contracts in include/gmt.h).
// Every entry point validates its arguments, converts internal failures into a
// gmt_status, and never lets an exception or a CUDA error escape.
#include <chrono>
#include <functional>
#include <string>
#include <vector>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace gmt {
gmt_status solve(gmt_hierarchy* h, double tol, const double* u0, double* u_out, gmt_info* info);
void homogenize(gmt_hierarchy* h, const double* u, double* CH);
void sensitivities(gmt_hierarchy* h, const double* u, double simp_p, double* out);
void residual_of(gmt_hierarchy* h, int precision, const double* u, double* out);
void estimate_lmax(gmt_hierarchy* h);
void step_apply(gmt_hierarchy* h, int level, int precision, const double* u, double* y);
void step_smooth(gmt_hierarchy* h, int level, int precision, const double* f, double* u,
                 int sweeps, bool zero);
void step_restrict(gmt_hierarchy* h, int level, int precision, const double* rf, double* fc);
void step_prolong(gmt_hierarchy* h, int level, int precision, const double* uc, double* uf);
void step_coarse(gmt_hierarchy* h, const double* f, double* u);
void step_vcycle(gmt_hierarchy* h, int precision, const double* f, double* u, bool zero);
void step_vcycle_inject(gmt_hierarchy* h, int precision, const double* f, double* u, bool zero,
                        const double* const* e);
void step_vcycle_batch(gmt_hierarchy* const* hs, int n, const double* const* f,
                       double* const* u, bool zero);
void run_batched(gmt_hierarchy* const* hs, int n, const std::function<void(int)>& body);
void leave_batch_group();
void prepare_batched_levels(gmt_hierarchy* h);
bool batch_thread();
void build_node_stencils(gmt_hierarchy* h, int level, bool fp64);
void build_node_stencils16(gmt_hierarchy* h, int level);
void export_nodes(gmt_hierarchy* h, int l, int32_t* xyz, uint8_t* m);
void export_elems(gmt_hierarchy* h, int l, int32_t* xyz, uint8_t* c);
void export_stencil(gmt_hierarchy* h, int l, int32_t* idx, double* w);
int64_t launch_count();
}  // namespace gmt

using gmt::Fail;

#define GMT_API_BEGIN \
  gmt::ApiGuard gmt_api_guard; \
  gmt::set_error("%s", ""); \
  try {
#define GMT_API_END                                           \
  }                                                           \
  catch (const Fail& f) {                                     \
    return f.status;                                          \
  }                                                           \
  catch (...) {                                               \
    gmt::set_error("unexpected host exception");              \
    return GMT_ERR_ARG;                                       \
  }

static bool opts_valid(const gmt_options& o) {
  return o.levels >= 0 && o.coarsest_max >= 4 && o.smoother >= 0 && o.smoother <= 2 &&
         o.cycle >= 0 && o.cycle <= 2 && o.nu_coarse >= 0 &&
         o.nu_pre >= 0 && o.nu_post >= 0 && o.nu_pre + o.nu_post > 0 && o.omega > 0 &&
         o.cheb_ratio > 1 && o.cheb_upper >= 1 && o.precision >= 0 && o.precision <= 2 &&
         o.inner_tol > 0 && o.inner_tol < 1 && o.max_inner > 0 && o.max_outer >= 0 &&
         (o.coarse_fp16 == 0 || o.coarse_fp16 == 1) && o.warm_sweeps >= 0 &&
         o.warm_sweeps <= 16;
}

static void ensure_device(gmt_hierarchy* h) { GMT_CUDA(cudaSetDevice(h->device)); }

static void ensure_material(gmt_hierarchy* h, gmt_physics ph, double E, double nu, double k,
                            double* setup_ms) {
  GMT_REQUIRE(ph == GMT_ELASTIC || ph == GMT_HEAT, GMT_ERR_ARG, "unknown physics %d", (int)ph);
  if (ph == GMT_ELASTIC)
    GMT_REQUIRE(E > 0 && nu > -1.0 && nu < 0.5 && std::isfinite(E), GMT_ERR_ARG,
                "elastic material needs E > 0 and -1 < nu < 0.5");
  else
    GMT_REQUIRE(k > 0 && std::isfinite(k), GMT_ERR_ARG, "heat conduction needs k > 0");
  const gmt::Material& m = h->mat;
  const bool same = h->prepared && m.physics == (int)ph &&
                    (ph == GMT_ELASTIC ? (m.E == E && m.nu == nu) : m.k == k);
  if (same) {
    if (setup_ms) *setup_ms = 0.0;
    return;
  }
  auto t0 = std::chrono::steady_clock::now();
  gmt::free_workspace(h);
  h->have_solution = false;
  gmt::prepare_material(h, (int)ph, E, nu, k);
  if (h->opts.smoother == GMT_SMOOTH_CHEBYSHEV && h->L > 1) gmt::estimate_lmax(h);
  if (setup_ms)
    *setup_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

static void check_level(const gmt_hierarchy* h, int level) {
  GMT_REQUIRE(h && level >= 0 && level < h->L, GMT_ERR_ARG, "level %d out of range", level);
}

extern "C" {

void gmt_default_options(gmt_options* o) {
  if (!o) return;
  o->levels = 0;
  o->coarsest_max = 8;
  o->smoother = GMT_SMOOTH_JACOBI;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->omega = 0.6;
  o->cheb_ratio = 30.0;
  o->cheb_upper = 1.1;
  o->precision = GMT_PREC_FP32;
  o->krylov = 1;
  o->inner_tol = 0.03;
  o->max_inner = 40;
  o->max_outer = 40;
  o->cycle = GMT_CYCLE_V;
  o->fp64_fallback = 1;
  o->nu_coarse = 2;
  o->graphs = 1;
  o->coarse_fp16 = 0;
  o->warm_sweeps = 0;
}

const char* gmt_status_string(gmt_status s) {
  switch (s) {
    case GMT_OK: return "ok";
    case GMT_ERR_ARG: return "invalid argument";
    case GMT_ERR_RES: return "unsupported resolution / level count";
    case GMT_ERR_EMPTY: return "cell has no solid voxel";
    case GMT_ERR_OOM: return "device out of memory";
    case GMT_ERR_CUDA: return "CUDA error";
    case GMT_NOT_CONVERGED: return "not converged";
    case GMT_DIVERGED: return "diverged";
    case GMT_ERR_STATE: return "operation needs a prepared material or a solution";
  }
  return "unknown status";
}

const char* gmt_last_error(void) { return gmt::last_error(); }

gmt_status gmt_build_hierarchy(const uint8_t* voxels, int res, int voxels_on_device,
                               const gmt_options* opts, void* stream, gmt_hierarchy** out) {
  GMT_API_BEGIN
  GMT_REQUIRE(voxels && out, GMT_ERR_ARG, "null voxels or output pointer");
  *out = nullptr;
  gmt_options o;
  gmt_default_options(&o);
  if (opts) o = *opts;
  GMT_REQUIRE(opts_valid(o), GMT_ERR_ARG, "invalid options");
  GMT_REQUIRE(res >= 4 && res % 4 == 0 && res <= 2048, GMT_ERR_RES,
              "resolution %d must be a multiple of 4 in [4, 2048]", res);
  int L = o.levels > 0 ? o.levels : gmt::choose_levels(res, o.coarsest_max);
  GMT_REQUIRE(L >= 1 && res % (1 << (L - 1)) == 0, GMT_ERR_RES,
              "resolution %d not divisible by 2^(L-1) with L = %d", res, L);
  for (int l = 0; l + 1 < L; ++l)
    GMT_REQUIRE((res >> l) % 4 == 0, GMT_ERR_RES, "non-coarsest level %d side %d not a multiple of 4",
                l, res >> l);
  GMT_REQUIRE((res >> (L - 1)) >= 4, GMT_ERR_RES, "coarsest level must be at least 4 per side");
  GMT_REQUIRE(((int64_t)(res >> (L - 1)) * (res >> (L - 1)) * (res >> (L - 1))) <= 4096,
              GMT_ERR_RES, "coarsest level too large for the dense solve (use more levels)");
  gmt_hierarchy* h = new gmt_hierarchy();
  try {
    GMT_CUDA(cudaGetDevice(&h->device));
    h->stream = (cudaStream_t)stream;
    h->geo.bind(h->stream);
    h->op.bind(h->stream);
    h->work.bind(h->stream);
    h->dn.bind(h->stream);
    h->opts = o;
    h->N = res;
    h->L = L;
    gmt::build_hierarchy(h, voxels, voxels_on_device != 0);
  } catch (...) {
    gmt::free_workspace(h);
    delete h;
    throw;
  }
  *out = h;
  return GMT_OK;
  GMT_API_END
}

void gmt_free_hierarchy(gmt_hierarchy* h) {
  if (!h) return;
  gmt::ApiGuard guard;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  h->tracer.destroy();
  gmt::free_workspace(h);
  delete h;
}

gmt_status gmt_set_stream(gmt_hierarchy* h, void* stream) {
  GMT_API_BEGIN
  GMT_REQUIRE(h, GMT_ERR_ARG, "null hierarchy");
  // work queued on the previous stream finishes before the new stream may reuse buffers
  if (h->stream != (cudaStream_t)stream) GMT_CUDA(cudaStreamSynchronize(h->stream));
  h->stream = (cudaStream_t)stream;
  h->geo.bind(h->stream);
  h->op.bind(h->stream);
  h->work.bind(h->stream);
  h->dn.bind(h->stream);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_set_options(gmt_hierarchy* h, const gmt_options* opts) {
  GMT_API_BEGIN
  GMT_REQUIRE(h && opts && opts_valid(*opts), GMT_ERR_ARG, "invalid options");
  gmt_options o = *opts;
  o.levels = h->opts.levels;
  o.coarsest_max = h->opts.coarsest_max;
  const bool cheb_new = o.smoother == GMT_SMOOTH_CHEBYSHEV && h->opts.smoother != o.smoother;
  h->opts = o;
  if (cheb_new && h->prepared && h->L > 1) {
    ensure_device(h);
    gmt::estimate_lmax(h);
  }
  return GMT_OK;
  GMT_API_END
}

int gmt_num_levels(const gmt_hierarchy* h) { return h ? h->L : 0; }
int gmt_level_res(const gmt_hierarchy* h, int level) {
  return (h && level >= 0 && level < h->L) ? h->lv[level].n : 0;
}
int64_t gmt_num_nodes(const gmt_hierarchy* h, int level) {
  return (h && level >= 0 && level < h->L) ? h->lv[level].n_nodes : -1;
}
int64_t gmt_num_elements(const gmt_hierarchy* h, int level) {
  return (h && level >= 0 && level < h->L) ? h->lv[level].n_elems : -1;
}
int64_t gmt_num_bricks(const gmt_hierarchy* h, int level) {
  return (h && level >= 0 && level < h->L) ? (h->lv[level].dense ? 0 : h->lv[level].nb) : -1;
}
int64_t gmt_device_bytes(const gmt_hierarchy* h) {
  return h ? (int64_t)(h->geo.bytes + h->op.bytes + h->work.bytes) : 0;
}

gmt_status gmt_node_coords(const gmt_hierarchy* h, int level, int32_t* xyz_out, uint8_t* mask_out) {
  GMT_API_BEGIN
  check_level(h, level);
  GMT_REQUIRE(xyz_out, GMT_ERR_ARG, "null output");
  gmt_hierarchy* hh = const_cast<gmt_hierarchy*>(h);
  ensure_device(hh);
  gmt::export_nodes(hh, level, xyz_out, mask_out);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_element_coords(const gmt_hierarchy* h, int level, int32_t* xyz_out,
                              uint8_t* child_mask_out) {
  GMT_API_BEGIN
  check_level(h, level);
  GMT_REQUIRE(xyz_out, GMT_ERR_ARG, "null output");
  gmt_hierarchy* hh = const_cast<gmt_hierarchy*>(h);
  ensure_device(hh);
  gmt::export_elems(hh, level, xyz_out, child_mask_out);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_transfer_stencil(const gmt_hierarchy* h, int level, int32_t* idx_out, double* w_out) {
  GMT_API_BEGIN
  GMT_REQUIRE(h && level >= 0 && level + 1 < h->L, GMT_ERR_ARG, "no level below %d", level);
  GMT_REQUIRE(idx_out && w_out, GMT_ERR_ARG, "null output");
  gmt_hierarchy* hh = const_cast<gmt_hierarchy*>(h);
  ensure_device(hh);
  gmt::export_stencil(hh, level, idx_out, w_out);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_prepare(gmt_hierarchy* h, gmt_physics physics, double E, double nu, double k) {
  GMT_API_BEGIN
  GMT_REQUIRE(h, GMT_ERR_ARG, "null hierarchy");
  ensure_device(h);
  ensure_material(h, physics, E, nu, k, nullptr);
  return GMT_OK;
  GMT_API_END
}

static void need_prepared(gmt_hierarchy* h) {
  GMT_REQUIRE(h, GMT_ERR_ARG, "null hierarchy");
  GMT_REQUIRE(h->prepared, GMT_ERR_STATE, "gmt_prepare has not run");
}

gmt_status gmt_apply(gmt_hierarchy* h, int level, int precision, const double* u, double* y) {
  GMT_API_BEGIN
  need_prepared(h);
  check_level(h, level);
  GMT_REQUIRE(u && y, GMT_ERR_ARG, "null field");
  GMT_REQUIRE(precision == GMT_PREC_FP64 || precision == GMT_PREC_FP32, GMT_ERR_ARG, "precision");
  GMT_REQUIRE(!h->lv[level].dense, GMT_ERR_ARG,
              "level %d is the dense coarsest level (side not a multiple of 4)", level);
  ensure_device(h);
  gmt::step_apply(h, level, precision, u, y);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_smooth(gmt_hierarchy* h, int level, int precision, const double* f, double* u,
                      int sweeps, int zero_init) {
  GMT_API_BEGIN
  need_prepared(h);
  check_level(h, level);
  GMT_REQUIRE(f && u && sweeps >= 0, GMT_ERR_ARG, "bad arguments");
  GMT_REQUIRE(precision == GMT_PREC_FP64 || precision == GMT_PREC_FP32, GMT_ERR_ARG, "precision");
  GMT_REQUIRE(!h->lv[level].dense, GMT_ERR_ARG, "level %d is the dense coarsest level", level);
  GMT_REQUIRE(!(h->opts.smoother == GMT_SMOOTH_CHEBYSHEV && level == h->L - 1), GMT_ERR_ARG,
              "no Chebyshev bounds on the coarsest level");
  ensure_device(h);
  gmt::step_smooth(h, level, precision, f, u, sweeps, zero_init != 0);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_restrict(gmt_hierarchy* h, int level, int precision, const double* r_fine,
                        double* f_coarse) {
  GMT_API_BEGIN
  need_prepared(h);
  GMT_REQUIRE(level >= 0 && level + 1 < h->L, GMT_ERR_ARG, "no level below %d", level);
  GMT_REQUIRE(r_fine && f_coarse, GMT_ERR_ARG, "null field");
  GMT_REQUIRE(precision == GMT_PREC_FP64 || precision == GMT_PREC_FP32, GMT_ERR_ARG, "precision");
  ensure_device(h);
  gmt::step_restrict(h, level, precision, r_fine, f_coarse);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_prolong(gmt_hierarchy* h, int level, int precision, const double* u_coarse,
                       double* u_fine) {
  GMT_API_BEGIN
  need_prepared(h);
  GMT_REQUIRE(level >= 0 && level + 1 < h->L, GMT_ERR_ARG, "no level below %d", level);
  GMT_REQUIRE(u_coarse && u_fine, GMT_ERR_ARG, "null field");
  GMT_REQUIRE(precision == GMT_PREC_FP64 || precision == GMT_PREC_FP32, GMT_ERR_ARG, "precision");
  ensure_device(h);
  gmt::step_prolong(h, level, precision, u_coarse, u_fine);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_coarse_solve(gmt_hierarchy* h, const double* f, double* u) {
  GMT_API_BEGIN
  need_prepared(h);
  GMT_REQUIRE(f && u, GMT_ERR_ARG, "null field");
  ensure_device(h);
  gmt::step_coarse(h, f, u);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_vcycle(gmt_hierarchy* h, int precision, const double* f, double* u, int zero_init) {
  GMT_API_BEGIN
  need_prepared(h);
  GMT_REQUIRE(f && u, GMT_ERR_ARG, "null field");
  GMT_REQUIRE(precision == GMT_PREC_FP64 || precision == GMT_PREC_FP32, GMT_ERR_ARG, "precision");
  ensure_device(h);
  gmt::step_vcycle(h, precision, f, u, zero_init != 0);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_vcycle_inject(gmt_hierarchy* h, int precision, const double* f, double* u,
                             int zero_init, const double* const* e, int n_e) {
  GMT_API_BEGIN
  need_prepared(h);
  GMT_REQUIRE(f && u && e, GMT_ERR_ARG, "null argument");
  GMT_REQUIRE(precision == GMT_PREC_FP64 || precision == GMT_PREC_FP32, GMT_ERR_ARG, "precision");
  GMT_REQUIRE(n_e == h->L, GMT_ERR_ARG, "n_e = %d, the hierarchy has %d levels", n_e, h->L);
  GMT_REQUIRE(h->opts.cycle == GMT_CYCLE_V, GMT_ERR_ARG,
              "corrections are injected into V-cycles only (the options select a W- or F-cycle)");
  ensure_device(h);
  gmt::step_vcycle_inject(h, precision, f, u, zero_init != 0, e);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_vcycle_batch(gmt_hierarchy* const* hs, int n, const double* const* f,
                            double* const* u, int zero_init) {
  GMT_API_BEGIN
  GMT_REQUIRE(hs && f && u, GMT_ERR_ARG, "null array");
  GMT_REQUIRE(n >= 1 && n <= GMT_BATCH_MAX, GMT_ERR_ARG, "batch of %d hierarchies (1..%d)", n,
              GMT_BATCH_MAX);
  for (int i = 0; i < n; ++i) {
    need_prepared(hs[i]);
    GMT_REQUIRE(f[i] && u[i], GMT_ERR_ARG, "null field of hierarchy %d", i);
    for (int j = 0; j < i; ++j)
      GMT_REQUIRE(hs[j] != hs[i], GMT_ERR_ARG, "hierarchy %d appears twice", i);
  }
  const gmt_hierarchy* a = hs[0];
  for (int i = 0; i < n; ++i) {
    const gmt_hierarchy* h = hs[i];
    const gmt_options& o = h->opts;
    GMT_REQUIRE(o.smoother == GMT_SMOOTH_JACOBI && o.cycle == GMT_CYCLE_V, GMT_ERR_ARG,
                "batched V-cycle: damped-Jacobi smoother and V-cycle only (hierarchy %d)", i);
    GMT_REQUIRE(!h->dens, GMT_ERR_ARG, "batched V-cycle: hierarchy %d has element densities", i);
    GMT_REQUIRE(h->device == a->device && h->stream == a->stream, GMT_ERR_ARG,
                "batched V-cycle: hierarchy %d is on another device or stream", i);
    GMT_REQUIRE(o.omega == a->opts.omega && o.nu_pre == a->opts.nu_pre &&
                    o.nu_post == a->opts.nu_post && o.nu_coarse == a->opts.nu_coarse &&
                    o.coarse_fp16 == a->opts.coarse_fp16,
                GMT_ERR_ARG, "batched V-cycle: hierarchy %d has other smoothing options", i);
    GMT_REQUIRE(h->mat.physics == a->mat.physics && h->mat.E == a->mat.E &&
                    h->mat.nu == a->mat.nu && h->mat.k == a->mat.k,
                GMT_ERR_ARG, "batched V-cycle: hierarchy %d has another material", i);
  }
  ensure_device(hs[0]);
  gmt::step_vcycle_batch(hs, n, f, u, zero_init != 0);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_lambda_max(gmt_hierarchy* h, int level, double* out) {
  GMT_API_BEGIN
  need_prepared(h);
  GMT_REQUIRE(out && level >= 0 && level + 1 < h->L, GMT_ERR_ARG, "bad level");
  ensure_device(h);
  if (h->lv[level].lmax == 0.0) gmt::estimate_lmax(h);
  *out = h->lv[level].lmax;
  return GMT_OK;
  GMT_API_END
}

// gmt_solve's work (throws Fail): the solve at the hierarchy's precision and, when the
// mixed-precision iteration diverges, the plain FP64 solve. Inside gmt_solve_batch the
// lattice leaves the batch's shared V-cycles when its mixed-precision iteration ends.
static gmt_status solve_one(gmt_hierarchy* h, gmt_physics physics, double E, double nu,
                            double k, double tol, const double* u0, double* u_out,
                            gmt_info* info) {
  ensure_device(h);
  double setup = 0.0;
  ensure_material(h, physics, E, nu, k, &setup);
  if (gmt::batch_thread()) gmt::prepare_batched_levels(h);
  gmt_info first;
  gmt_status st = gmt::solve(h, tol, u0, u_out, info ? info : &first);
  gmt::leave_batch_group();
  if (info) info->fp64_fallback = 0;
  if (st == GMT_DIVERGED && h->opts.precision != GMT_PREC_FP64 && h->opts.fp64_fallback) {
    // the mixed-precision iteration failed on this cell: solve again in plain FP64
    const gmt_info f = info ? *info : first;
    const int keep = h->opts.precision;
    h->opts.precision = GMT_PREC_FP64;
    try {
      st = gmt::solve(h, tol, u0, u_out, info);
    } catch (...) {
      h->opts.precision = keep;
      throw;
    }
    h->opts.precision = keep;
    if (info) {
      info->inner_total += f.inner_total;
      info->outer += f.outer;
      info->t_solve_ms += f.t_solve_ms;
      info->fp64_fallback = 1;
    }
  }
  if (info) info->t_setup_ms = setup;
  return st;
}

gmt_status gmt_solve(gmt_hierarchy* h, gmt_physics physics, double E, double nu, double k,
                     double tol, const double* u0, double* u_out, gmt_info* info) {
  GMT_API_BEGIN
  GMT_REQUIRE(h, GMT_ERR_ARG, "null hierarchy");
  GMT_REQUIRE(tol > 0 && tol < 1, GMT_ERR_ARG, "tol must be in (0, 1)");
  return solve_one(h, physics, E, nu, k, tol, u0, u_out, info);
  GMT_API_END
}

gmt_status gmt_solve_batch(gmt_hierarchy* const* hs, int n, gmt_physics physics, double E,
                           double nu, double k, double tol, const double* const* u0,
                           double* const* u_out, gmt_info* info, gmt_status* status) {
  GMT_API_BEGIN
  GMT_REQUIRE(hs, GMT_ERR_ARG, "null hierarchy array");
  GMT_REQUIRE(n >= 1 && n <= GMT_BATCH_MAX, GMT_ERR_ARG, "batch of %d hierarchies (1..%d)", n,
              GMT_BATCH_MAX);
  GMT_REQUIRE(tol > 0 && tol < 1, GMT_ERR_ARG, "tol must be in (0, 1)");
  for (int i = 0; i < n; ++i) {
    GMT_REQUIRE(hs[i], GMT_ERR_ARG, "null hierarchy %d", i);
    for (int j = 0; j < i; ++j)
      GMT_REQUIRE(hs[j] != hs[i], GMT_ERR_ARG, "hierarchy %d appears twice", i);
  }
  const gmt_hierarchy* a = hs[0];
  for (int i = 0; i < n; ++i) {
    const gmt_hierarchy* h = hs[i];
    const gmt_options& o = h->opts;
    GMT_REQUIRE(o.precision == GMT_PREC_FP32, GMT_ERR_ARG,
                "batched solve: mixed precision only (hierarchy %d)", i);
    GMT_REQUIRE(o.smoother == GMT_SMOOTH_JACOBI && o.cycle == GMT_CYCLE_V, GMT_ERR_ARG,
                "batched solve: damped-Jacobi smoother and V-cycle only (hierarchy %d)", i);
    GMT_REQUIRE(!h->dens, GMT_ERR_ARG, "batched solve: hierarchy %d has element densities", i);
    GMT_REQUIRE(h->device == a->device, GMT_ERR_ARG,
                "batched solve: hierarchy %d is on another device", i);
    GMT_REQUIRE(o.omega == a->opts.omega && o.nu_pre == a->opts.nu_pre &&
                    o.nu_post == a->opts.nu_post && o.nu_coarse == a->opts.nu_coarse &&
                    o.coarse_fp16 == a->opts.coarse_fp16,
                GMT_ERR_ARG, "batched solve: hierarchy %d has other smoothing options", i);
  }
  std::vector<gmt_status> st(n, GMT_OK);
  std::vector<std::string> msg(n);
  gmt::run_batched(hs, n, [&](int i) {
    try {
      st[i] = solve_one(hs[i], physics, E, nu, k, tol, u0 ? u0[i] : nullptr,
                        u_out ? u_out[i] : nullptr, info ? &info[i] : nullptr);
    } catch (const Fail& f) {
      gmt::leave_batch_group();
      st[i] = f.status;
      msg[i] = gmt::last_error();
    } catch (...) {
      gmt::leave_batch_group();
      st[i] = GMT_ERR_ARG;
      msg[i] = "unexpected host exception";
    }
  });
  gmt_status worst = GMT_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = st[i];
    if (worst == GMT_OK && st[i] != GMT_OK) {
      worst = st[i];
      if (!msg[i].empty()) gmt::set_error("lattice %d: %s", i, msg[i].c_str());
    }
  }
  return worst;
  GMT_API_END
}

// the finer true-residual replacement threshold gmt_autotune tries last
constexpr double kAutotuneInnerTol = 0.003;

gmt_status gmt_autotune(gmt_hierarchy* h, gmt_physics physics, double E, double nu, double k,
                        double tol, gmt_options* best, double* times_ms) {
  GMT_API_BEGIN
  GMT_REQUIRE(h, GMT_ERR_ARG, "null hierarchy");
  GMT_REQUIRE(tol > 0 && tol < 1, GMT_ERR_ARG, "tol must be in (0, 1)");
  ensure_device(h);
  ensure_material(h, physics, E, nu, k, nullptr);
  const gmt_options base = h->opts;
  const bool mixed = base.precision != GMT_PREC_FP64;
  // build what the candidates create lazily, so that no candidate's time includes it
  for (int l = 1; l + 1 < h->L; ++l) {
    gmt::build_node_stencils(h, l, !mixed);
    if (mixed) gmt::build_node_stencils16(h, l);
  }
  struct Cand {
    int nu, nc, fp16;
    double itol;
  };
  std::vector<Cand> cands;
  for (int nu_ = 1; nu_ <= 2; ++nu_)
    for (int nc = 1; nc <= 3; ++nc)
      for (int f = 0; f <= 1; ++f) cands.push_back(Cand{nu_, nc, f, base.inner_tol});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GMT_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) cudaEventDestroy(e0);
  GMT_CUDA(ce);
  double best_ms = INFINITY;
  int best_i = -1;
  try {
    // one untimed solve: the workspace of this precision is allocated on first use
    (void)solve_one(h, physics, E, nu, k, tol, nullptr, nullptr, nullptr);
    auto timed = [&](const Cand& c) -> double {
      gmt_options o = base;
      o.nu_pre = o.nu_post = c.nu;
      o.nu_coarse = c.nc;
      o.coarse_fp16 = c.fp16;
      o.inner_tol = c.itol;
      h->opts = o;
      gmt_info info;
      GMT_CUDA(cudaEventRecord(e0, h->stream));
      const gmt_status st = solve_one(h, physics, E, nu, k, tol, nullptr, nullptr, &info);
      GMT_CUDA(cudaEventRecord(e1, h->stream));
      GMT_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      GMT_CUDA(cudaEventElapsedTime(&t, e0, e1));
      return st == GMT_OK ? (double)t : INFINITY;
    };
    for (size_t i = 0; i < cands.size(); ++i) {
      const double ms = (mixed || cands[i].fp16 == 0) ? timed(cands[i]) : INFINITY;
      if (times_ms) times_ms[i] = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best_i = (int)i;
      }
    }
    // the last candidate: the fastest schedule with the finer replacement threshold (fewer
    // true-residual replacements pay on cells that converge in a few cycles, and cost
    // cycles on slow ones, so it is measured, not assumed); mixed precision only
    double ms = INFINITY;
    if (best_i >= 0 && mixed && base.inner_tol > kAutotuneInnerTol) {
      Cand c = cands[best_i];
      c.itol = kAutotuneInnerTol;
      cands.push_back(c);
      ms = timed(c);
      if (ms < best_ms) {
        best_ms = ms;
        best_i = (int)cands.size() - 1;
      }
    }
    if (times_ms) times_ms[GMT_AUTOTUNE_CANDIDATES - 1] = ms;
  } catch (...) {
    h->opts = base;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->opts = base;
  GMT_REQUIRE(best_i >= 0, GMT_NOT_CONVERGED, "autotune: no candidate reached tol %g", tol);
  h->opts.nu_pre = h->opts.nu_post = cands[best_i].nu;
  h->opts.nu_coarse = cands[best_i].nc;
  h->opts.coarse_fp16 = cands[best_i].fp16;
  h->opts.inner_tol = cands[best_i].itol;
  if (best) *best = h->opts;
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_homogenize(gmt_hierarchy* h, gmt_physics physics, double E, double nu, double k,
                          const double* u, double* CH_out) {
  GMT_API_BEGIN
  GMT_REQUIRE(h && CH_out, GMT_ERR_ARG, "null argument");
  ensure_device(h);
  const bool stored = u == nullptr;
  if (stored) GMT_REQUIRE(h->have_solution, GMT_ERR_STATE, "no stored solution");
  ensure_material(h, physics, E, nu, k, nullptr);
  if (stored) GMT_REQUIRE(h->have_solution, GMT_ERR_STATE, "stored solution belongs to another material");
  gmt::homogenize(h, u, CH_out);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_set_densities(gmt_hierarchy* h, const double* rho, int rho_on_device,
                             double rho_min, double simp_p) {
  GMT_API_BEGIN
  GMT_REQUIRE(h, GMT_ERR_ARG, "null hierarchy");
  if (rho)
    GMT_REQUIRE(std::isfinite(rho_min) && rho_min >= 0.0 && std::isfinite(simp_p) && simp_p > 0.0,
                GMT_ERR_ARG, "densities need rho_min >= 0 and simp_p > 0");
  ensure_device(h);
  gmt::set_densities(h, rho, rho_on_device != 0, rho_min, simp_p);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_sensitivities(gmt_hierarchy* h, gmt_physics physics, double E, double nu,
                             double k, double simp_p, const double* u, double* dCH_out) {
  GMT_API_BEGIN
  GMT_REQUIRE(h && dCH_out, GMT_ERR_ARG, "null argument");
  GMT_REQUIRE(std::isfinite(simp_p) && simp_p > 0.0, GMT_ERR_ARG, "simp_p must be > 0");
  GMT_REQUIRE(!h->dens || simp_p == h->simp_p, GMT_ERR_ARG,
              "simp_p %g differs from the p %g given with the densities", simp_p, h->simp_p);
  ensure_device(h);
  const bool stored = u == nullptr;
  if (stored) GMT_REQUIRE(h->have_solution, GMT_ERR_STATE, "no stored solution");
  ensure_material(h, physics, E, nu, k, nullptr);
  if (stored) GMT_REQUIRE(h->have_solution, GMT_ERR_STATE, "stored solution belongs to another material");
  gmt::sensitivities(h, u, simp_p, dCH_out);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_residual(gmt_hierarchy* h, int precision, const double* u, double* out) {
  GMT_API_BEGIN
  need_prepared(h);
  GMT_REQUIRE(u && out, GMT_ERR_ARG, "null argument");
  GMT_REQUIRE(precision == GMT_PREC_FP64 || precision == GMT_PREC_FP32, GMT_ERR_ARG, "precision");
  ensure_device(h);
  gmt::residual_of(h, precision, u, out);
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_trace_enable(gmt_hierarchy* h, int on) {
  GMT_API_BEGIN
  GMT_REQUIRE(h, GMT_ERR_ARG, "null hierarchy");
  ensure_device(h);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
  h->tracer.reset();
  h->tracer.on = on != 0;
  h->tracer.brackets_only = on == 2;
  return GMT_OK;
  GMT_API_END
}

gmt_status gmt_trace_query(gmt_hierarchy* h, int category, int64_t* launches, double* ms,
                           double* bytes) {
  GMT_API_BEGIN
  GMT_REQUIRE(h && category >= 0 && category < gmt::TR_NCAT, GMT_ERR_ARG, "bad category");
  ensure_device(h);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
  h->tracer.flush();
  if (launches) *launches = h->tracer.launches[category];
  if (ms) *ms = h->tracer.ms[category];
  if (bytes) *bytes = h->tracer.bytes[category];
  return GMT_OK;
  GMT_API_END
}

const char* gmt_trace_name(int c) {
  static const char* names[gmt::TR_NCAT] = {
      "smooth_l0", "resid_l0", "apply_l0", "outer_resid", "diag_l0", "stencil_l1",
      "restrict", "prolong", "coarse_solve", "energy", "vector", "setup_hierarchy",
      "setup_operators", "setup_coarse_inverse", "stencil_l2up", "vcycle"};
  return (c >= 0 && c < gmt::TR_NCAT) ? names[c] : "";
}

int64_t gmt_launch_count(void) { return gmt::launch_count(); }

void gmt_release_cached_memory(void) { gmt::pool_trim(); }

int64_t gmt_cached_bytes(void) { return (int64_t)gmt::pool_cached_bytes(); }

}  // extern "C"
