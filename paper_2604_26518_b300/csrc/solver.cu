// Solver orchestration: the V-cycle of Alg. 1 (smoother, residual, restriction, recursion,
// coarsest solve, prolongation, smoother), used either as the preconditioner of a
// conjugate-gradient loop or as a stationary iteration (the paper's GMG loop, Sec. 5
// baselines), with the solution kept in FP64 (precision FP64) or as a float-float pair
// refined by reliable residual replacement (precision FP32; see solve()). The Krylov step
// uses the flexible (Polak-Ribiere) beta; a mixed solve that diverges is reported as such
// and gmt_solve repeats it in FP64.
// Tolerances below 2e-6 evaluate the mixed-precision true residual in native FP64.
// Stopping rule (Sec. 5 metric r, reading: the maximum over load cases must meet tol).
// Gauge (Sec. 3.1 zero-mean constraint): the mean over active nodes of every component
// and case is removed from the final field. Load cases whose assembled load cancels
// (||f_m|| <= 1e-12 of its gross element-load norm) have u_m = 0 and r_m = 0.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>

#include "stencil.cuh"

namespace gmt {

// deterministic pseudo-random fill (power iteration start vector)
__global__ void k_hash_fill(float* __restrict__ x, const uint8_t* __restrict__ mask, int C,
                            int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t slot = ((i >> 6) / C) * 64 + (i & 63);
  uint32_t hsh = (uint32_t)(i * 2654435761ull) ^ 0x9e3779b9u;
  hsh ^= hsh >> 16;
  hsh *= 0x7feb352du;
  hsh ^= hsh >> 15;
  hsh *= 0x846ca68bu;
  hsh ^= hsh >> 16;
  x[i] = mask[slot] ? ((float)(hsh & 0xffffff) / 16777216.0f - 0.5f) : 0.0f;
}

// histogram of the octant masks of the active level-0 slots (integer atomics: exact)
__global__ void k_mask_hist(const uint8_t* __restrict__ mask, int64_t n,
                            unsigned long long* __restrict__ hist) {
  __shared__ unsigned int sh[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned m = mask[i];
    if (m) atomicAdd(&sh[m], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// ||f_m||^2 of the level-0 load, f_n = sum_{a in mask} (K_e x0)[a]: the load of a node
// depends on its octant mask alone, so the norm is the mask histogram times per-mask norms
// (FP64 on the host, masks in increasing order)
static void dens_load_norms2(gmt_hierarchy* h, double* fn2);
static void load_norms2(gmt_hierarchy* h, double* fn2) {
  if (h->dens) {
    dens_load_norms2(h, fn2);
    return;
  }
  if (!h->have_hist) {
    const Level& l0 = h->lv[0];
    Arena tmp(h->stream);
    unsigned long long* d = tmp.alloc<unsigned long long>(256);
    GMT_CUDA(cudaMemsetAsync(d, 0, 256 * sizeof(unsigned long long), h->stream));
    const unsigned g = std::min<unsigned>(grid_for(l0.nslots, 256), 148u * 8u);
    k_mask_hist<<<g, 256, 0, h->stream>>>(l0.mask, l0.nslots, d);
    GMT_LAUNCH_CHECK();
    unsigned long long hh[256];
    GMT_CUDA(cudaMemcpyAsync(hh, d, sizeof(hh), cudaMemcpyDeviceToHost, h->stream));
    GMT_CUDA(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 256; ++k) h->mask_hist[k] = (long long)hh[k];
    h->have_hist = true;
  }
  const Material& mt = h->mat;
  const int D = mt.D, M = mt.M;
  for (int m = 0; m < M; ++m) fn2[m] = 0.0;
  for (int k = 1; k < 256; ++k) {
    if (h->mask_hist[k] == 0) continue;
    for (int i = 0; i < D; ++i)
      for (int m = 0; m < M; ++m) {
        double f = 0.0;
        for (int a = 0; a < 8; ++a)
          if ((k >> a) & 1) f += mt.Fe[(a * D + i) * M + m];
        fn2[m] += (double)h->mask_hist[k] * f * f;
      }
  }
}

struct Workspace {
  Prec prec = P32;       // inner storage precision
  Prec arith = P32;      // CG vector precision (P64 for the FP64 solve, else P32)
  std::vector<void*> ua, ub, f, r, dc;  // per level: ping-pong u, rhs, residual, Chebyshev d
  void *x = nullptr, *rr = nullptr, *p = nullptr, *q = nullptr, *cvt = nullptr;
  float *hi = nullptr, *lo = nullptr, *rout = nullptr;
  double* u64 = nullptr;
  double* f64 = nullptr;
  double* part = nullptr;
  int64_t part_rows = 0;
  double* red = nullptr;     // reduction slots, 12 x 32 doubles
  int* active = nullptr;     // per case flags (device)
  double* ones = nullptr;    // per case 1.0 (device)
  // the solve's two V-cycle forms (plain; with the fused Krylov partials), replayed from CUDA
  // graphs once captured: graph, result buffer, kernels in it, the options it was captured
  // with, and how often the form has run directly
  struct Captured {
    cudaGraphExec_t exec = nullptr;
    void* out = nullptr;
    int64_t kernels = 0;
    gmt_options opts;
    int direct = 0;
  } vg[2];
  // levels l >= 1 whose coarse unknown starts from the field already in ua[l] instead of
  // zero on the way down (bit l; set only for the duration of one step_vcycle_inject)
  unsigned inject = 0;
  ~Workspace() {
    for (Captured& c : vg) retire_graph(c.exec);   // destroyed once no other call is in flight
  }
};

void free_workspace(gmt_hierarchy* h) {
  h->work.release();
  delete h->ws;
  h->ws = nullptr;
  h->ws_for_prec = -1;
}

static Workspace* workspace(gmt_hierarchy* h, Prec prec) {
  if (h->ws && h->ws_for_prec == (int64_t)prec) return h->ws;
  // a stored solution outlives the switch to another precision's workspace: it waits as a
  // canonical FP64 field (exact for a float-float pair) and moves into the new workspace's
  // form below; the block goes back to the pool once the stream has finished with it
  struct Keep {
    double* p = nullptr;
    cudaStream_t s = nullptr;
    ~Keep() {
      if (p) {
        cudaStreamSynchronize(s);
        pool_free(p);
      }
    }
  } keep;
  keep.s = h->stream;
  if (h->ws && h->have_solution) {
    keep.p = (double*)pool_alloc((size_t)h->lv[0].n_nodes * h->mat.C * sizeof(double));
    if (h->ws->prec == P64) slots_to_canon(h, 0, P64, h->ws->u64, keep.p);
    else ff_to_canon(h, h->ws->hi, h->ws->lo, keep.p);
  }
  free_workspace(h);   // waits for the hierarchy's stream
  // built aside and published only when complete: a failed allocation leaves no
  // half-built workspace behind for a later call to use
  Workspace* w = new Workspace();
  try {
    w->prec = prec;
    w->arith = prec == P64 ? P64 : P32;
    const int C = h->mat.C;
    const size_t sb = prec_bytes(prec), ab = prec_bytes(w->arith);
    for (int l = 0; l < h->L; ++l) {
      const int64_t nv = h->lv[l].nslots * C;
      w->ua.push_back(h->work.raw(nv * sb));
      w->ub.push_back(h->work.raw(nv * sb));
      w->f.push_back(h->work.raw(nv * sb));
      w->r.push_back(h->work.raw(nv * sb));
      w->dc.push_back(h->work.raw(nv * sb));
    }
    const int64_t n0 = h->lv[0].nslots * C;
    w->x = h->work.raw(n0 * ab);
    w->rr = h->work.raw(n0 * ab);
    w->p = h->work.raw(n0 * ab);
    w->q = h->work.raw(n0 * ab);
    w->cvt = h->work.raw(n0 * ab);
    w->hi = h->work.alloc<float>(n0);
    w->lo = h->work.alloc<float>(n0);
    w->rout = h->work.alloc<float>(n0);
    w->u64 = h->work.alloc<double>(n0);
    w->f64 = h->work.alloc<double>(n0);
    int64_t rows = 1;
    for (int l = 0; l < h->L; ++l) rows = std::max<int64_t>(rows, h->lv[l].nb);
    w->part_rows = rows;
    w->part = h->work.alloc<double>(rows * 32);
    w->red = h->work.alloc<double>(12 * 32);
    w->active = h->work.alloc<int>(8);
    w->ones = h->work.alloc<double>(8);
    double ones[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    GMT_CUDA(cudaMemcpyAsync(w->ones, ones, sizeof(ones), cudaMemcpyHostToDevice, h->stream));
    if (keep.p) {
      if (prec == P64) canon_to_slots(h, 0, P64, keep.p, w->u64);
      else canon_to_ff(h, keep.p, w->hi, w->lo);
    }
    GMT_CUDA(cudaStreamSynchronize(h->stream));
  } catch (...) {
    h->work.release();
    delete w;
    h->have_solution = false;   // it lived in the workspace just freed
    throw;
  }
  h->ws = w;
  h->ws_for_prec = prec;
  return w;
}

// reduce the [nb][K] partials of `level` into red slot `slot` (device)
static double* reduce_to(gmt_hierarchy* h, Workspace* w, int level, int K, int slot) {
  double* out = w->red + slot * 32;
  launch_reduce(h, w->part, h->lv[level].nb, K, out);
  return out;
}

static void fetch(gmt_hierarchy* h, const double* dev, double* host, int n);

// element densities: ||f_m||^2 of the stored level-0 load vector, by a device reduction
static void dens_load_norms2(gmt_hierarchy* h, double* fn2) {
  Workspace* w = h->ws;
  vec_dot(h, 0, P64, h->f0_64, h->f0_64, w->part);
  fetch(h, reduce_to(h, w, 0, h->mat.M, 1), fn2, h->mat.M);
}

static void fetch(gmt_hierarchy* h, const double* dev, double* host, int n) {
  GMT_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

// ------------------------------------------------------------------ smoother / V-cycle
// smooth `sweeps` times on level l from *u (or zero); the result pointer is returned in *u
// (it alternates between the level's two buffers). part (level 0, zero == false): the last
// sweep also writes [blocks][M + C] partials of f . u and the sums of u (fused).
static void smooth(gmt_hierarchy* h, Workspace* w, int l, const void* f, void** u, void** other,
                   int sweeps, bool zero, double* part = nullptr, const void* aux = nullptr) {
  const gmt_options& o = h->opts;
  const Prec pr = w->prec;
  if (sweeps <= 0) {
    if (zero) vec_zero(h, l, pr, *u);
    return;
  }
  if (o.smoother == GMT_SMOOTH_GS8) {
    // 8-colour Gauss-Seidel: per sweep the colours in turn, each a damped block-Jacobi step
    // on the nodes of that colour with the values the previous colours left
    if (zero) vec_zero(h, l, pr, *u);
    for (int s = 0; s < sweeps; ++s)
      for (int c = 0; c < 8; ++c) {
        VecArgs a;
        a.u = *u;
        a.f = f;
        a.out = *other;
        a.omega = o.omega;
        a.colour = c;
        if (s + 1 == sweeps && c == 7) {
          a.part = part;
          a.aux = aux;
        }
        launch_stencil(h, l, pr, ST_JACOBI, a);
        std::swap(*u, *other);
      }
    return;
  }
  if (o.smoother == GMT_SMOOTH_JACOBI) {
    int s0 = 0;
    if (zero) {
      launch_diag(h, l, pr, f, *u, nullptr, o.omega);
      s0 = 1;
    }
    for (int s = s0; s < sweeps; ++s) {
      VecArgs a;
      a.u = *u;
      a.f = f;
      a.out = *other;
      a.omega = o.omega;
      if (s + 1 == sweeps) {
        a.part = part;
        a.aux = aux;
      }
      launch_stencil(h, l, pr, ST_JACOBI, a);
      std::swap(*u, *other);
    }
    return;
  }
  // Chebyshev polynomial of degree `sweeps` on D^-1 K over [lmax/ratio, upper*lmax]
  const double lmax = h->lv[l].lmax;
  const double bnd = o.cheb_upper * lmax, a0 = lmax / o.cheb_ratio;
  const double theta = 0.5 * (bnd + a0), delta = 0.5 * (bnd - a0), sigma = theta / delta;
  double rho = 1.0 / sigma;
  void* d = w->dc[l];
  int s0 = 0;
  if (zero) {
    launch_diag(h, l, pr, f, *u, d, 1.0 / theta);  // d0 = D^-1 f / theta, u1 = d0
    s0 = 1;
  } else {
    VecArgs a;  // d0 = D^-1 (f - K u) / theta, u1 = u + d0
    a.u = *u;
    a.f = f;
    a.dprev = d;
    a.out = *other;
    a.dout = d;
    a.c1 = 0.0;
    a.c2 = 1.0 / theta;
    if (sweeps == 1) {
      a.part = part;
      a.aux = aux;
    }
    launch_stencil(h, l, pr, ST_CHEB, a);
    std::swap(*u, *other);
    s0 = 1;
  }
  for (int s = s0; s < sweeps; ++s) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    VecArgs a;
    a.u = *u;
    a.f = f;
    a.dprev = d;
    a.out = *other;
    a.dout = (s + 1 < sweeps) ? d : nullptr;
    a.c1 = rho_new * rho;
    a.c2 = 2.0 * rho_new / delta;
    if (s + 1 == sweeps) {
      a.part = part;
      a.aux = aux;
    }
    launch_stencil(h, l, pr, ST_CHEB, a);
    std::swap(*u, *other);
    rho = rho_new;
  }
}

// One V-cycle on level l for K_l u = f (u zero on entry when zero == true). Returns the
// buffer that holds the result: one of the level's two ping-pong buffers (level 0: ua/ub).
// part (level 0, nu_post >= 1): the last post-smoothing sweep writes [blocks][M + C]
// partials of f . u and the sums of u (see smooth()).
// cycle: GMT_CYCLE_V, _W or _F (the coarse problem of level l gets one V-cycle, two
// W-cycles, or an F-cycle followed by a V-cycle; the coarsest level is solved once).
static void* vcycle(gmt_hierarchy* h, Workspace* w, int l, const void* f, void* u_init, bool zero,
                    double* part = nullptr, int cycle = -1, const void* aux = nullptr) {
  const Prec pr = w->prec;
  if (cycle < 0) cycle = h->opts.cycle;
  if (l == h->L - 1) {
    launch_coarse_solve(h, pr, f, w->ua[l]);
    return w->ua[l];
  }
  void* u = zero ? w->ua[l] : u_init;
  void* other = (u == w->ua[l]) ? w->ub[l] : w->ua[l];
  const gmt_options& o = h->opts;
  const int nu1 = (l > 0 && o.nu_coarse > 0) ? o.nu_coarse : o.nu_pre;
  const int nu2 = (l > 0 && o.nu_coarse > 0) ? o.nu_coarse : o.nu_post;
  smooth(h, w, l, f, &u, &other, nu1, zero);
  VecArgs a;
  a.u = u;
  a.f = f;
  a.out = w->r[l];
  launch_stencil(h, l, pr, ST_RESID, a);
  launch_restrict(h, l, pr, w->r[l], w->f[l + 1]);
  // Alg. 2: the coarse unknown starts from an injected correction where one is given
  void* uc = ((w->inject >> (l + 1)) & 1u)
                 ? vcycle(h, w, l + 1, w->f[l + 1], w->ua[l + 1], false, nullptr, cycle)
                 : vcycle(h, w, l + 1, w->f[l + 1], nullptr, true, nullptr, cycle);
  if (l + 2 < h->L && cycle != GMT_CYCLE_V)
    uc = vcycle(h, w, l + 1, w->f[l + 1], uc, false, nullptr,
                cycle == GMT_CYCLE_W ? GMT_CYCLE_W : GMT_CYCLE_V);
  launch_prolong(h, l, pr, uc, u);
  smooth(h, w, l, f, &u, &other, nu2, false, part, aux);
  return u;
}

// One level-0 V-cycle of the solve on w->rr (form 0: plain; form 1: the last sweep also
// writes the Krylov partials of w->part against w->q). The launch sequence of a form is the
// same every time (fixed buffers, sizes and scalars), so once the form has run directly
// kDirectBeforeCapture times (the first run builds what the levels create lazily) it is
// captured into a CUDA graph and replayed with one launch, which removes the per-kernel
// launch cost of the small coarse levels. Not while tracing (the tracer times every
// launch), with graphs switched off, on the legacy default stream, when the caller's stream
// is itself being captured, or while another library call is in flight in another host
// thread (then the form runs directly; see GraphLock).
// A form is captured after this many direct runs: capture and instantiation cost about as
// much as a few V-cycles, so solves of a handful of cycles (and a hierarchy is rebuilt per
// cell) never capture, and long solves replay.
constexpr int kDirectBeforeCapture = 16;

static void* group_vcycle(gmt_hierarchy* h, Workspace* w, int form);
bool in_batch_group(const Workspace* w);
bool batch_thread();

static void* run_vcycle(gmt_hierarchy* h, Workspace* w, int form) {
  if (in_batch_group(w)) return group_vcycle(h, w, form);   // gmt_solve_batch
  double* part = form ? w->part : nullptr;
  const void* aux = form ? w->q : nullptr;
  Workspace::Captured& c = w->vg[form];
  // the cycle on the FP32 residual rr; the BF16 V-cycle rounds rr to BF16 on entry and
  // returns its result widened to FP32 in cvt (form 0 only: the fused partials need the
  // FP32 vectors inside the last sweep)
  auto body = [&]() -> void* {
    if (w->prec != PBF) return vcycle(h, w, 0, w->rr, nullptr, true, part, -1, aux);
    f32_to_bf16(h, (const float*)w->rr, w->f[0]);
    void* res = vcycle(h, w, 0, w->f[0], nullptr, true, nullptr, -1, nullptr);
    bf16_to_f32(h, res, (float*)w->cvt);
    return w->cvt;
  };
  auto direct = [&]() {
    TraceScope tv(&h->tracer, h->stream, TR_VCYCLE, 0.0);
    return body();
  };
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool can = h->opts.graphs != 0 && !h->tracer.on && h->stream != nullptr && !batch_thread() &&
                   cudaStreamIsCapturing(h->stream, &cap) == cudaSuccess &&
                   cap == cudaStreamCaptureStatusNone;
  if (!can) {
    if (c.exec) {
      retire_graph(c.exec);
      c.exec = nullptr;
      c.direct = 0;
    }
    return direct();
  }
  if (!c.exec && c.direct < kDirectBeforeCapture) {
    ++c.direct;
    return direct();
  }
  // graph operations only while no other library call is in flight (see GraphLock)
  GraphLock gl;
  if (!gl.alone) {
    gl.release();
    return direct();
  }
  if (c.exec && std::memcmp(&c.opts, &h->opts, sizeof(gmt_options)) != 0) {
    cudaGraphExecDestroy(c.exec);
    c.exec = nullptr;
    c.direct = 0;
  }
  if (c.exec) {
    GMT_CUDA(cudaGraphLaunch(c.exec, h->stream));
    count_launch(c.kernels);
    return c.out;
  }
  if (c.direct < kDirectBeforeCapture) {
    gl.release();
    ++c.direct;
    return direct();
  }
  const int64_t k0 = thread_launch_count();
  cudaGraph_t g = nullptr;
  GMT_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  void* out = nullptr;
  try {
    out = body();
  } catch (...) {
    cudaStreamEndCapture(h->stream, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  GMT_CUDA(cudaStreamEndCapture(h->stream, &g));
  cudaError_t e = cudaGraphInstantiate(&c.exec, g, 0);
  cudaGraphDestroy(g);
  GMT_CUDA(e);
  c.out = out;
  c.kernels = thread_launch_count() - k0;
  c.opts = h->opts;
  GMT_CUDA(cudaGraphLaunch(c.exec, h->stream));
  return out;
}

// ------------------------------------------------------------------ Chebyshev bounds
void estimate_lmax(gmt_hierarchy* h) {
  Workspace* w = workspace(h, P32);
  const int C = h->mat.C, M = h->mat.M;
  for (int l = 0; l + 1 < h->L; ++l) {
    const int64_t n = h->lv[l].nslots * C;
    float* x = (float*)w->ua[l];
    float* y = (float*)w->ub[l];
    k_hash_fill<<<grid_for(n, 256), 256, 0, h->stream>>>(x, h->lv[l].mask, C, n);
    GMT_LAUNCH_CHECK();
    // 20 power iterations on D^-1 K, each case normalised on the device (the scale
    // 1 / ||y|| comes from the reduction's epilogue); only the last iteration is read back
    constexpr int kIters = 20;
    double hy[8], hx[8];
    for (int it = 0; it < kIters; ++it) {
      VecArgs a;
      a.u = x;
      a.out = y;
      launch_stencil(h, l, P32, ST_APPLY, a);
      launch_diag(h, l, P32, y, y, nullptr, 1.0);   // y = D^-1 K x (pointwise, in place)
      vec_dot(h, l, P32, y, y, w->part);
      RedEpi e;
      e.mode = 5;
      e.ratio = w->red + 3 * 32;
      launch_reduce(h, w->part, h->lv[l].nb, M, w->red, e);
      if (it + 1 == kIters) {
        vec_dot(h, l, P32, x, x, w->part);
        launch_reduce(h, w->part, h->lv[l].nb, M, w->red + 2 * 32);
        fetch(h, w->red, hy, M);
        fetch(h, w->red + 2 * 32, hx, M);
        break;
      }
      vec_scale_cases(h, l, P32, w->red + 3 * 32, y);
      std::swap(x, y);
    }
    double lam = 0.0;
    for (int m = 0; m < M; ++m) lam = std::max(lam, std::sqrt(hy[m] / std::max(hx[m], 1e-300)));
    h->lv[l].lmax = lam;
  }
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

// ------------------------------------------------------------------ solve
static Prec prec_of(int p) { return p == GMT_PREC_FP64 ? P64 : (p == GMT_PREC_BF16 ? PBF : P32); }

// Preconditioned iteration on K u = f with the V-cycle as preconditioner.
//   krylov = 1: conjugate gradients; krylov = 0: stationary V-cycle iteration u += V(f - K u).
// FP64: all vectors FP64; the recursively updated residual is trusted until it reaches
//   tol / 2, then the true residual decides.
// FP32 (mixed precision with reliable updates): the iteration vectors are FP32 and the
//   correction accumulates in an FP32 vector x; whenever the iterated residual has dropped
//   by `inner_tol` relative to the last true residual (or looks converged), x is added to
//   the float-float solution (hi, lo), the true residual f - K u is recomputed with the
//   float-float difference-form kernel and replaces the iterated one. The Krylov recurrence
//   (p, r.z) continues across these replacements instead of restarting, so the iteration
//   count stays that of FP64 CG while every vector operation runs in FP32.
// warm_sweeps damped-Jacobi sweeps on level 0 applied to the given initial field (the
// solution buffers of the solve: u64, or hi with lo cleared) against the level-0 load
static void smooth_start(gmt_hierarchy* h, Workspace* w, bool mixed) {
  const gmt_options& o = h->opts;
  const Prec pr = mixed ? P32 : P64;
  // FP32 sweeps: on a BF16 workspace the level-0 buffers hold BF16, so the load and the
  // ping-pong partner go to the FP32 scratch cvt and x (x is cleared before the iteration)
  const bool bf = w->prec == PBF;
  void* f = bf ? w->cvt : w->f[0];
  if (mixed) {
    launch_resid_ff(h, nullptr, nullptr, (float*)f, nullptr);   // the load (zero start)
  } else {
    vec_zero(h, 0, P64, w->ub[0]);
    VecArgs r;   // f - K 0 with the load formed by the kernel
    r.u = w->ub[0];
    r.out = f;
    launch_stencil(h, 0, P64, ST_RESID, r);
  }
  void* cur = mixed ? (void*)w->hi : (void*)w->u64;
  void* oth = bf ? w->x : w->ua[0];
  for (int k = 0; k < o.warm_sweeps; ++k) {
    VecArgs a;
    a.u = cur;
    a.f = f;
    a.out = oth;
    a.omega = o.omega;
    launch_stencil(h, 0, pr, ST_JACOBI, a);
    std::swap(cur, oth);
  }
  void* sol = mixed ? (void*)w->hi : (void*)w->u64;
  if (cur != sol) vec_copy(h, 0, pr, cur, sol);
  if (mixed) vec_zero(h, 0, P32, w->lo);
}

gmt_status solve(gmt_hierarchy* h, double tol, const double* u0, double* u_out, gmt_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  const gmt_options& o = h->opts;
  const Prec pr = prec_of(o.precision);
  if (o.smoother == GMT_SMOOTH_CHEBYSHEV && h->L > 1 && h->lv[0].lmax == 0.0) estimate_lmax(h);
  Workspace* w = workspace(h, pr);
  const int M = h->mat.M, C = h->mat.C;
  const Material& mt = h->mat;
  const bool mixed = pr != P64;
  const bool krylov = o.krylov != 0;
  // ||f_m|| and the load-cancellation rule
  double fn[8];
  load_norms2(h, fn);
  int act[8] = {0}, live[8] = {0};   // live: the case has a load; act: still iterating
  for (int m = 0; m < M; ++m) {
    fn[m] = std::sqrt(fn[m]);
    live[m] = act[m] = fn[m] > 1e-12 * mt.gross[m];
  }
  // the float-float residual is accurate to ~1e-7 of ||f||; tighter tolerances use FP64
  const bool ff_outer = mixed && tol >= 2e-6;
  double rel[8] = {0};
  // true residual of the current solution into w->rr (arith precision), norms into rel[]
  bool zero_guess = u0 == nullptr;   // the first residual of a zero start is the load
  auto true_residual = [&]() -> double {
    double rn[8];
    if (ff_outer && zero_guess) {
      launch_resid_ff(h, nullptr, nullptr, (float*)w->rr, w->part);
      zero_guess = false;
    } else if (!mixed) {
      VecArgs a;
      a.u = w->u64;
      a.out = w->rr;
      a.part = w->part;
      launch_stencil(h, 0, P64, ST_RESID, a);
    } else if (ff_outer) {
      launch_resid_ff(h, w->hi, w->lo, (float*)w->rr, w->part);
    } else {
      ff_to_f64(h, w->hi, w->lo, w->u64);
      VecArgs a;
      a.u = w->u64;
      a.out = w->f64;
      a.part = w->part;
      launch_stencil(h, 0, P64, ST_RESID, a);
      f64_to_f32(h, w->f64, (float*)w->rr);
    }
    fetch(h, reduce_to(h, w, 0, M, 0), rn, M);
    double mx = 0.0;
    for (int m = 0; m < M; ++m) {
      rel[m] = live[m] ? std::sqrt(rn[m]) / fn[m] : 0.0;
      if (live[m]) mx = std::max(mx, rel[m]);
    }
    return mx;
  };
  if (!mixed) {
    if (u0) canon_to_slots(h, 0, P64, u0, w->u64);
    else vec_zero(h, 0, P64, w->u64);
  } else {
    if (u0) canon_to_ff(h, u0, w->hi, w->lo);
    else {
      vec_zero(h, 0, P32, w->hi);
      vec_zero(h, 0, P32, w->lo);
    }
  }
  if (u0 && o.warm_sweeps > 0) smooth_start(h, w, mixed);
  const Prec ar = w->arith;
  // Mixed precision: the difference-form FP32 operator annihilates translations exactly,
  // while FP32 rounding leaves the iterated residual, and the V-cycle output, with small
  // translation components that no step can reduce; left alone they grow through the
  // recurrence and corrupt r.z versus p.Kp. Both vectors are therefore projected onto the
  // zero-mean (per component and case) subspace, where the periodic problem lives.
  double* vsums = w->red + 7 * 32 + 8;          // device sums per value (C <= 18)
  double* alpha = w->red + 8 * 32;              // device step ratios per case
  double* beta = w->red + 9 * 32;
  float* vmean = (float*)(w->red + 10 * 32);    // device means per value (FP32)
  auto sum_values = [&](const void* vec) {
    double* part = w->part + h->lv[0].nb * M;    // rows beyond the per-case partials
    vec_sum_values32(h, (const float*)vec, part);
    RedEpi e;
    e.mode = 3;
    e.out32 = vmean;
    e.scale = 1.0 / (double)h->lv[0].n_nodes;
    launch_reduce(h, part, h->lv[0].nb, h->mat.C, vsums, e);
  };
  auto project = [&](void* vec) {
    if (!mixed) return;
    sum_values(vec);
    vec_sub_mean32(h, vmean, (float*)vec);
  };
  int cycles = 0, updates = 0, restarts = 0, trips = 0;
  static const bool verbose = std::getenv("GMT_VERBOSE") != nullptr;
  gmt_status st = GMT_NOT_CONVERGED;
  double mx = true_residual();
  const double first = mx;
  double ref[8];   // true residual norms at the last replacement
  for (int m = 0; m < M; ++m) ref[m] = rel[m];
  auto push_active = [&]() {
    GMT_CUDA(cudaMemcpyAsync(w->active, act, sizeof(act), cudaMemcpyHostToDevice, h->stream));
  };
  auto deactivate_converged = [&]() {
    for (int m = 0; m < M; ++m)
      if (act[m] && rel[m] <= tol) act[m] = 0;
  };
  const int max_cycles = o.max_inner * std::max(1, o.max_outer);
  if (mx <= tol) {
    st = GMT_OK;
  } else {
    for (int m = 0; m < M; ++m) act[m] = live[m] && rel[m] > tol;
    push_active();
    vec_zero(h, 0, ar, w->x);
    double* rz = w->red + 4 * 32;
    double* pq = w->red + 5 * 32;
    double* rz_new = w->red + 6 * 32;
    project(w->rr);
    void* z = run_vcycle(h, w, 0);
    project(z);
    ++cycles;
    if (krylov) {
      vec_copy(h, 0, ar, z, w->p);
      vec_dot(h, 0, ar, w->rr, z, w->part);
      launch_reduce(h, w->part, h->lv[0].nb, M, rz);
    }
    for (;;) {
      if (!krylov) project(z);
      VecArgs a;
      a.u = krylov ? w->p : z;
      a.out = w->q;
      a.part = krylov ? w->part : nullptr;
      launch_stencil(h, 0, ar, ST_APPLY, a);  // q = K p (and p.q)
      if (krylov) {
        RedEpi e;
        e.mode = 1;   // alpha = rz / pq
        e.other = rz;
        e.active = w->active;
        e.ratio = alpha;
        launch_reduce(h, w->part, h->lv[0].nb, M, pq, e);
        vec_cg_update(h, ar, alpha, w->active, w->x, w->p, w->rr, w->q, w->part, mixed);
      } else {
        vec_cg_update(h, ar, w->ones, w->active, w->x, z, w->rr, w->q, w->part, mixed);
      }
      double* rn_dev = w->red;
      if (mixed) {
        // ||r||^2 and the sums of r from the update's partials (one launch), then r loses
        // its mean
        RedEpi em;
        em.mode = 3;
        em.out32 = vmean;
        em.scale = 1.0 / (double)h->lv[0].n_nodes;
        const int col0[2] = {0, M}, ncols[2] = {M, C};
        double* outs[2] = {rn_dev, vsums};
        const RedEpi epis[2] = {RedEpi(), em};
        launch_reduce_multi(h, w->part, h->lv[0].nb, M + C, 2, col0, ncols, outs, epis);
        vec_sub_mean32(h, vmean, (float*)w->rr);
      } else {
        rn_dev = reduce_to(h, w, 0, M, 0);
      }
      double rn[8];
      fetch(h, rn_dev, rn, M);
      if (verbose) {
        std::fprintf(stderr, "gmt: cycle %d iterated r/|f|:", cycles);
        for (int m = 0; m < M; ++m) std::fprintf(stderr, " %.3e", std::sqrt(rn[m]) / fn[m]);
        std::fprintf(stderr, "\n");
      }
      bool replace = false, nan = false, grew = false;
      double rit[8] = {0};   // iterated residuals of this cycle
      for (int m = 0; m < M; ++m) {
        if (!act[m]) continue;
        const double r = std::sqrt(rn[m]) / fn[m];
        rit[m] = r;
        if (std::isnan(r)) nan = true;
        if (r <= 0.5 * tol || (mixed && r <= o.inner_tol * ref[m])) replace = true;
        // growth guard: an iterated residual 10x above the last true one means the
        // recurrence has lost its conjugacy in the inner precision
        if (krylov && r > 10.0 * ref[m]) grew = true;
      }
      if (grew) replace = true;
      const bool last = cycles >= max_cycles;
      bool restart = false;
      if (replace || nan || last) {
        // fold the correction into the solution and take the true residual
        if (mixed) vec_ff_add(h, (const float*)w->x, w->hi, w->lo);
        else vec_add(h, 0, P64, w->x, w->u64);
        vec_zero(h, 0, ar, w->x);
        mx = true_residual();
        ++updates;
        if (verbose) {
          std::fprintf(stderr, "gmt: update %d true r/|f|:", updates);
          for (int m = 0; m < M; ++m) std::fprintf(stderr, " %.3e", rel[m]);
          std::fprintf(stderr, "\n");
        }
        if (mx <= tol) {
          st = GMT_OK;
          break;
        }
        project(w->rr);
        if (std::isnan(mx) || mx > 1e4 * std::max(first, 1e-300)) {
          st = GMT_DIVERGED;
          break;
        }
        if (last) break;
        // a second growth-guard trip in the inner precision: the FP32 V-cycle is too far from
        // symmetric for CG on this cell (near-singular modes that FP32 cannot resolve); stop
        // and let the caller fall back to the FP64 solve
        if (grew && ++trips >= 2 && mixed) {
          st = GMT_DIVERGED;
          break;
        }
        // restart the Krylov recurrence from the true residual when the replacement gained
        // less than 10 % (stagnation), when the iterated residual had grown (growth guard),
        // or when the true residual is more than 2x the iterated one (the recurrence no
        // longer tracks the residual it claims)
        if (grew) restart = true;
        for (int m = 0; m < M; ++m) {
          if (!act[m]) continue;
          if (rel[m] > 0.9 * ref[m]) restart = true;
          if (rit[m] > 0.0 && rel[m] > 2.0 * rit[m]) restart = true;
        }
        for (int m = 0; m < M; ++m) ref[m] = rel[m];
        deactivate_converged();
        push_active();
      }
      // the last post-smoothing sweep writes the partials of r.z, q.z (q = K p of the last
      // direction) and of the sums of z
      const bool fused = krylov && h->L > 1 && o.nu_post >= 1 && w->prec != PBF;
      z = run_vcycle(h, w, fused ? 1 : 0);
      ++cycles;
      if (krylov) {
        // rr is mean-free, so r.z needs no correction for the mean of z; the mean of z is
        // removed while forming the new direction.
        // Flexible CG (Polak-Ribiere): beta = z_new.(r_new - r_old) / (z_old.r_old)
        //   = -alpha (z_new.q) / (z_old.r_old), since r_new - r_old = -alpha q. With a fixed
        // symmetric preconditioner this is the Fletcher-Reeves beta of plain PCG; it stays
        // robust when FP32 rounding makes the V-cycle slightly non-symmetric.
        RedEpi eb;
        eb.mode = 6;   // beta = -alpha (q.z) / rz
        eb.other = rz;
        eb.other2 = alpha;
        eb.active = w->active;
        eb.ratio = beta;
        RedEpi em;
        em.mode = 3;   // per-value means of z
        em.out32 = vmean;
        em.scale = 1.0 / (double)h->lv[0].n_nodes;
        if (fused) {
          // one launch: r.z, q.z (beta) and the sums of z (means) from the fused partials
          const int col0[3] = {0, M, 2 * M}, ncols[3] = {M, M, C};
          double* outs[3] = {rz_new, w->red + 10 * 32 + 16, vsums};
          const RedEpi epis[3] = {RedEpi(), eb, em};
          launch_reduce_multi(h, w->part, h->lv[0].nb, 2 * M + C, mixed ? 3 : 2, col0, ncols,
                              outs, epis);
        } else {
          double* zq = w->part + (int64_t)h->lv[0].nb * M;   // partials of q.z
          if (mixed) sum_values(z);
          vec_dot(h, 0, ar, w->q, z, zq);
          vec_dot(h, 0, ar, w->rr, z, w->part);
          launch_reduce(h, w->part, h->lv[0].nb, M, rz_new);
          launch_reduce(h, zq, h->lv[0].nb, M, w->red + 10 * 32 + 16, eb);
        }
        if (restart) {
          if (mixed) vec_sub_mean32(h, vmean, (float*)z);
          vec_copy(h, 0, ar, z, w->p);
          ++restarts;
        } else {
          vec_cg_dir(h, ar, beta, z, w->p, mixed ? vmean : nullptr);
        }
        GMT_CUDA(cudaMemcpyAsync(rz, rz_new, M * sizeof(double), cudaMemcpyDeviceToDevice,
                                 h->stream));
      }
    }
  }
  // gauge: remove the mean of every component and case over active nodes
  {
    const int C = mt.C;
    if (!mixed) {
      vec_sum_values(h, 0, P64, w->u64, nullptr, w->part);
      double* sums = reduce_to(h, w, 0, C, 1);
      double hs[18];
      fetch(h, sums, hs, C);
      for (int v = 0; v < C; ++v) hs[v] /= (double)h->lv[0].n_nodes;
      GMT_CUDA(cudaMemcpyAsync(w->red + 2 * 32, hs, C * sizeof(double), cudaMemcpyHostToDevice,
                               h->stream));
      vec_sub_mean64(h, 0, w->red + 2 * 32, w->u64);
    } else {
      // float-float sums and means formed on the device (no host round trip)
      vec_sum_ff(h, w->hi, w->lo, w->part);
      RedEpi e;
      e.mode = 4;
      e.out32 = (float*)(w->red + 11 * 32);
      e.scale = 1.0 / (double)h->lv[0].n_nodes;
      e.count = C;
      launch_reduce(h, w->part, h->lv[0].nb, C, w->red + 32, e);
      vec_ff_sub_mean(h, (const float*)(w->red + 11 * 32), w->hi, w->lo);
    }
  }
  if (u_out) {
    if (!mixed) slots_to_canon(h, 0, P64, w->u64, u_out);
    else ff_to_canon(h, w->hi, w->lo, u_out);
  }
  GMT_CUDA(cudaStreamSynchronize(h->stream));
  h->have_solution = true;
  if (info) {
    info->outer = updates;
    info->inner_total = cycles;
    info->cases = M;
    for (int m = 0; m < 6; ++m) info->rel_residual[m] = m < M ? rel[m] : 0.0;
    info->t_solve_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return st;
}

// A caller's canonical field in the workspace's form, in scratch buffers (the stored
// solution stays): FP64 slots on an FP64 workspace, else a float-float pair in the
// conversion scratch (cvt and rout hold n0 floats there)
static void external_field(gmt_hierarchy* h, Workspace* w, const double* u, const void** u64,
                           const float** hi, const float** lo) {
  if (w->prec == P64) {
    canon_to_slots(h, 0, P64, u, w->f64);
    *u64 = w->f64;
  } else {
    float* shi = (float*)w->cvt;
    canon_to_ff(h, u, shi, w->rout);
    *hi = shi;
    *lo = w->rout;
  }
}

// C^H from the stored solution (u == nullptr) or a canonical field
void homogenize(gmt_hierarchy* h, const double* u, double* CH) {
  const Material& mt = h->mat;
  const int M = mt.M, K = M * (M + 1) / 2;
  Workspace* w = h->ws;
  Prec pr = w ? w->prec : P32;
  if (!w) w = workspace(h, P32);
  const void* u64 = w->u64;
  const float *hi = w->hi, *lo = w->lo;
  if (u) external_field(h, w, u, &u64, &hi, &lo);
  if (pr == P64) launch_energy(h, P64, u64, nullptr, w->part);
  else launch_energy(h, P32, hi, lo, w->part);
  double e[21];
  fetch(h, reduce_to(h, w, 0, K, 0), e, K);
  const double vol = (double)h->N * h->N * h->N;
  // ff path: + sum_e s_e C0 (s_e = 1 without densities)
  const double ne = pr == P64 ? 0.0 : (h->dens ? h->coef_sum : (double)h->lv[0].n_elems);
  for (int I = 0; I < M; ++I)
    for (int J = I; J < M; ++J) {
      const double v = (e[I * M - I * (I - 1) / 2 + (J - I)] + ne * mt.C0[I * M + J]) / vol;
      CH[I * M + J] = v;
      CH[J * M + I] = v;
    }
}

// dC^H_IJ / d rho_e of the SIMP model C_e = (rho_min + rho_e^p) C0 at the solid elements
// (rho_e = 1): p / |Omega| (x0^I - u_e^I)^T K0 (x0^J - u_e^J) (App. F.3), per element
void sensitivities(gmt_hierarchy* h, const double* u, double simp_p, double* out) {
  Workspace* w = h->ws;
  Prec pr = w ? w->prec : P32;
  if (!w) w = workspace(h, P32);
  const void* u64 = w->u64;
  const float *hi = w->hi, *lo = w->lo;
  if (u) external_field(h, w, u, &u64, &hi, &lo);
  // with densities the factor p rho_e^(p-1) is applied per element by the kernel
  const double vol = (double)h->N * h->N * h->N;
  const double scale = h->dens ? 1.0 / vol : simp_p / vol;
  if (pr == P64) launch_energy_per(h, P64, u64, nullptr, out, scale);
  else launch_energy_per(h, P32, hi, lo, out, scale);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

// relative residuals of a canonical field
void residual_of(gmt_hierarchy* h, int precision, const double* u, double* out) {
  const Material& mt = h->mat;
  const int M = mt.M;
  Workspace* w = workspace(h, h->ws ? (Prec)h->ws_for_prec : P32);
  double fn[8], rn[8];
  load_norms2(h, fn);
  if (precision == GMT_PREC_FP64) {
    // scratch for the FP64 copy: u64 holds the stored solution on an FP64 workspace, where
    // the correction x has n0 doubles; on the others u64 is scratch
    void* ucp = w->prec == P64 ? w->x : w->u64;
    canon_to_slots(h, 0, P64, u, ucp);
    VecArgs a;
    a.u = ucp;
    a.out = w->f64;
    a.part = w->part;
    launch_stencil(h, 0, P64, ST_RESID, a);
  } else {
    float* hi = (float*)w->cvt;  // scratch of >= n0 floats
    float* lo = w->rout;
    canon_to_ff(h, u, hi, lo);
    launch_resid_ff(h, hi, lo, (float*)w->q, w->part);
  }
  fetch(h, reduce_to(h, w, 0, M, 0), rn, M);
  for (int m = 0; m < M; ++m) {
    const double f = std::sqrt(fn[m]);
    out[m] = f > 1e-12 * mt.gross[m] ? std::sqrt(rn[m]) / f : std::sqrt(rn[m]);
  }
}

// ------------------------------------------------------------------ per-step entry points
void step_apply(gmt_hierarchy* h, int level, int precision, const double* u, double* y) {
  const Prec pr = precision == GMT_PREC_FP64 ? P64 : P32;
  Workspace* w = workspace(h, pr);
  canon_to_slots(h, level, pr, u, w->ua[level]);
  VecArgs a;
  a.u = w->ua[level];
  a.out = w->ub[level];
  launch_stencil(h, level, pr, ST_APPLY, a);
  slots_to_canon(h, level, pr, w->ub[level], y);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

void step_smooth(gmt_hierarchy* h, int level, int precision, const double* f, double* u,
                 int sweeps, bool zero) {
  const Prec pr = precision == GMT_PREC_FP64 ? P64 : P32;
  if (h->opts.smoother == GMT_SMOOTH_CHEBYSHEV && h->lv[level].lmax == 0.0) estimate_lmax(h);
  Workspace* w = workspace(h, pr);
  canon_to_slots(h, level, pr, f, w->f[level]);
  void* cur = w->ua[level];
  void* oth = w->ub[level];
  if (!zero) canon_to_slots(h, level, pr, u, cur);
  smooth(h, w, level, w->f[level], &cur, &oth, sweeps, zero);
  slots_to_canon(h, level, pr, cur, u);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

void step_restrict(gmt_hierarchy* h, int level, int precision, const double* rf, double* fc) {
  const Prec pr = precision == GMT_PREC_FP64 ? P64 : P32;
  Workspace* w = workspace(h, pr);
  canon_to_slots(h, level, pr, rf, w->r[level]);
  launch_restrict(h, level, pr, w->r[level], w->f[level + 1]);
  slots_to_canon(h, level + 1, pr, w->f[level + 1], fc);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

void step_prolong(gmt_hierarchy* h, int level, int precision, const double* uc, double* uf) {
  const Prec pr = precision == GMT_PREC_FP64 ? P64 : P32;
  Workspace* w = workspace(h, pr);
  canon_to_slots(h, level + 1, pr, uc, w->ua[level + 1]);
  canon_to_slots(h, level, pr, uf, w->ub[level]);
  launch_prolong(h, level, pr, w->ua[level + 1], w->ub[level]);
  slots_to_canon(h, level, pr, w->ub[level], uf);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

void step_coarse(gmt_hierarchy* h, const double* f, double* u) {
  Workspace* w = workspace(h, P64);
  const int lc = h->L - 1;
  canon_to_slots(h, lc, P64, f, w->f[lc]);
  launch_coarse_solve(h, P64, w->f[lc], w->ua[lc]);
  slots_to_canon(h, lc, P64, w->ua[lc], u);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

void step_vcycle(gmt_hierarchy* h, int precision, const double* f, double* u, bool zero) {
  const Prec pr = precision == GMT_PREC_FP64 ? P64 : P32;
  if (h->opts.smoother == GMT_SMOOTH_CHEBYSHEV && h->L > 1 && h->lv[0].lmax == 0.0) estimate_lmax(h);
  Workspace* w = workspace(h, pr);
  canon_to_slots(h, 0, pr, f, w->f[0]);
  void* init = nullptr;
  if (!zero) {
    canon_to_slots(h, 0, pr, u, w->ua[0]);
    init = w->ua[0];
  }
  void* res = vcycle(h, w, 0, w->f[0], init, zero);
  slots_to_canon(h, 0, pr, res, u);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

// One V-cycle in which the coarse unknown of each level l with e[l] != nullptr
// (1 <= l < L - 1) starts from that canonical field instead of zero (Alg. 2's injected
// corrections); the coarsest level is solved exactly, so its entry is not read
void step_vcycle_inject(gmt_hierarchy* h, int precision, const double* f, double* u, bool zero,
                        const double* const* e) {
  const Prec pr = precision == GMT_PREC_FP64 ? P64 : P32;
  if (h->opts.smoother == GMT_SMOOTH_CHEBYSHEV && h->L > 1 && h->lv[0].lmax == 0.0) estimate_lmax(h);
  Workspace* w = workspace(h, pr);
  canon_to_slots(h, 0, pr, f, w->f[0]);
  void* init = nullptr;
  if (!zero) {
    canon_to_slots(h, 0, pr, u, w->ua[0]);
    init = w->ua[0];
  }
  unsigned mask = 0;
  for (int l = 1; l + 1 < h->L; ++l)
    if (e[l]) {
      canon_to_slots(h, l, pr, e[l], w->ua[l]);
      mask |= 1u << l;
    }
  w->inject = mask;
  void* res = nullptr;
  try {
    res = vcycle(h, w, 0, w->f[0], init, zero);
  } catch (...) {
    w->inject = 0;
    throw;
  }
  w->inject = 0;
  slots_to_canon(h, 0, pr, res, u);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

// ------------------------------------------------------------------ batched V-cycle
// The FP32 damped-Jacobi V-cycle of vcycle() on several hierarchies at once: each phase
// (first sweep from zero, sweep, residual, restriction, coarsest solve, prolongation) is
// one launch over the bricks of all of them (batch.cu), in the order the single-lattice
// cycle runs them, so every lattice's result is bitwise its own V-cycle's. Lattices may
// have different level counts: at level l those whose coarsest level is l take their
// coarsest solve, the others the smoothing part of the cycle.
using PtrVec = std::vector<void*>;

struct BMember {
  gmt_hierarchy* h;
  Workspace* w;
};

static void bsmooth(std::vector<gmt_hierarchy*>& hs, cudaStream_t s, int l, const PtrVec& f,
                    PtrVec& u, PtrVec& o, int sweeps, bool zero,
                    const std::vector<double*>* part, const PtrVec* aux) {
  const int n = (int)hs.size();
  if (sweeps <= 0) {
    if (zero) batch_zero(hs.data(), n, s, l, u.data());
    return;
  }
  int s0 = 0;
  if (zero) {
    batch_diag(hs.data(), n, s, l, f.data(), u.data(), hs[0]->opts.omega);
    s0 = 1;
  }
  for (int k = s0; k < sweeps; ++k) {
    const bool last = k + 1 == sweeps;
    batch_stencil(hs.data(), n, s, l, ST_JACOBI, u.data(), f.data(), o.data(),
                  last && part ? part->data() : nullptr, last && aux ? aux->data() : nullptr);
    std::swap(u, o);
  }
}

// m[i] at level l (l <= its coarsest level) for K_l u = f[i], from init[i] (or zero);
// part/aux (level 0): the last post-smoothing sweep also writes the fused Krylov partials
static PtrVec bvcycle(const std::vector<BMember>& m, int l, const PtrVec& f, const PtrVec* init,
                      const std::vector<double*>* part, const PtrVec* aux, cudaStream_t s) {
  const int n = (int)m.size();
  PtrVec u(n, nullptr);
  std::vector<gmt_hierarchy*> hc;
  PtrVec fc, uc;
  std::vector<int> sm;
  for (int i = 0; i < n; ++i) {
    if (m[i].h->L - 1 == l) {
      hc.push_back(m[i].h);
      fc.push_back(f[i]);
      uc.push_back(m[i].w->ua[l]);
      u[i] = m[i].w->ua[l];
    } else {
      sm.push_back(i);
    }
  }
  if (!hc.empty()) batch_coarse_solve(hc.data(), (int)hc.size(), s, fc.data(), uc.data());
  if (sm.empty()) return u;
  const int k = (int)sm.size();
  std::vector<BMember> mm;
  std::vector<gmt_hierarchy*> hs;
  PtrVec fs(k), us(k), os(k), r(k), fn(k), ax(k, nullptr);
  std::vector<double*> pt(k, nullptr);
  for (int j = 0; j < k; ++j) {
    const int i = sm[j];
    Workspace* w = m[i].w;
    mm.push_back(m[i]);
    hs.push_back(m[i].h);
    fs[j] = f[i];
    us[j] = init ? (*init)[i] : w->ua[l];
    os[j] = us[j] == w->ua[l] ? w->ub[l] : w->ua[l];
    r[j] = w->r[l];
    fn[j] = w->f[l + 1];
    if (part) {
      pt[j] = (*part)[i];
      ax[j] = (*aux)[i];
    }
  }
  const gmt_options& op = hs[0]->opts;
  const int nu1 = (l > 0 && op.nu_coarse > 0) ? op.nu_coarse : op.nu_pre;
  const int nu2 = (l > 0 && op.nu_coarse > 0) ? op.nu_coarse : op.nu_post;
  bsmooth(hs, s, l, fs, us, os, nu1, init == nullptr, nullptr, nullptr);
  batch_stencil(hs.data(), k, s, l, ST_RESID, us.data(), fs.data(), r.data());
  batch_restrict(hs.data(), k, s, l, r.data(), fn.data());
  const PtrVec ucn = bvcycle(mm, l + 1, fn, nullptr, nullptr, nullptr, s);
  batch_prolong(hs.data(), k, s, l, ucn.data(), us.data());
  bsmooth(hs, s, l, fs, us, os, nu2, false, part ? &pt : nullptr, part ? &ax : nullptr);
  for (int j = 0; j < k; ++j) u[sm[j]] = us[j];
  return u;
}

void step_vcycle_batch(gmt_hierarchy* const* hs, int n, const double* const* f,
                       double* const* u, bool zero) {
  std::vector<BMember> m(n);
  PtrVec fs(n), init(n);
  for (int i = 0; i < n; ++i) {
    m[i] = BMember{hs[i], workspace(hs[i], P32)};
    prepare_batched_levels(hs[i]);
    canon_to_slots(hs[i], 0, P32, f[i], m[i].w->f[0]);
    fs[i] = m[i].w->f[0];
    if (!zero) {
      canon_to_slots(hs[i], 0, P32, u[i], m[i].w->ua[0]);
      init[i] = m[i].w->ua[0];
    }
  }
  const PtrVec res = bvcycle(m, 0, fs, zero ? nullptr : &init, nullptr, nullptr, hs[0]->stream);
  for (int i = 0; i < n; ++i) slots_to_canon(hs[i], 0, P32, res[i], u[i]);
  GMT_CUDA(cudaStreamSynchronize(hs[0]->stream));
}

// ------------------------------------------------------------------ batched solves
// Lattices solved together (gmt_solve_batch): one host thread per lattice runs the
// single-lattice solve on the lattice's own stream; its mixed-precision V-cycles meet here.
// Once every lattice still in its mixed-precision iteration has asked for a V-cycle, the
// last to arrive launches one batched V-cycle for all of them on the group's stream
// (ordered after each lattice's work by an event, and each lattice's stream after it by
// another). Every lattice's arithmetic is that of its own solve, so its results are
// bitwise gmt_solve's; the small coarse levels of all lattices share each launch.
// The wait for the other lattices is a host wait with a time limit.
constexpr int kRendezvousLimitS = 900;

struct BatchGroup {
  struct Req {
    gmt_hierarchy* h;
    Workspace* w;
    int form;
    void* out = nullptr;
    bool done = false;
    gmt_status st = GMT_OK;
    std::string err;
  };
  std::mutex mu;
  std::condition_variable cv;
  int members = 0;               // lattices still in their mixed-precision iteration
  std::vector<Req*> pending;
  cudaStream_t stream = nullptr;
  cudaEvent_t finished = nullptr;   // recorded after each batched V-cycle
  std::vector<cudaEvent_t> ready;   // per lattice: its work before the V-cycle

  // with mu held: one batched V-cycle for every pending request (each form its own)
  void launch_locked() {
    std::vector<Req*> batch;
    batch.swap(pending);
    gmt_status st = GMT_OK;
    std::string err;
    try {
      for (int form = 0; form < 2; ++form) {
        std::vector<BMember> m;
        std::vector<Req*> rs;
        PtrVec f, ax;
        std::vector<double*> part;
        for (Req* r : batch) {
          if (r->form != form) continue;
          m.push_back(BMember{r->h, r->w});
          rs.push_back(r);
          f.push_back(r->w->rr);
          part.push_back(form ? r->w->part : nullptr);
          ax.push_back(form ? r->w->q : nullptr);
        }
        if (m.empty()) continue;
        const PtrVec out = bvcycle(m, 0, f, nullptr, form ? &part : nullptr,
                                   form ? &ax : nullptr, stream);
        for (size_t k = 0; k < rs.size(); ++k) rs[k]->out = out[k];
      }
      GMT_CUDA(cudaEventRecord(finished, stream));
    } catch (const Fail& e) {
      st = e.status;
      err = last_error();
    } catch (...) {
      st = GMT_ERR_ARG;
      err = "unexpected host exception in a batched V-cycle";
    }
    for (Req* r : batch) {
      r->st = st;
      r->err = err;
      r->done = true;
    }
    cv.notify_all();
  }

  void* vcycle(gmt_hierarchy* h, Workspace* w, int form, cudaEvent_t ev) {
    GMT_CUDA(cudaEventRecord(ev, h->stream));
    Req r{h, w, form};
    std::unique_lock<std::mutex> lk(mu);
    GMT_CUDA(cudaStreamWaitEvent(stream, ev, 0));
    pending.push_back(&r);
    if ((int)pending.size() == members) launch_locked();
    const auto t0 = std::chrono::steady_clock::now();
    while (!r.done) {
      cv.wait_for(lk, std::chrono::seconds(1));
      if (!r.done && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(kRendezvousLimitS)) {
        // (a leader completes every request it takes under the lock, so an undone request
        // is still pending here)
        const auto it = std::find(pending.begin(), pending.end(), &r);
        if (it != pending.end()) pending.erase(it);
        GMT_REQUIRE(false, GMT_ERR_STATE,
                    "batched solve: waited %d s for the other lattices' V-cycles",
                    kRendezvousLimitS);
      }
    }
    lk.unlock();
    GMT_REQUIRE(r.st == GMT_OK, r.st, "%s", r.err.c_str());
    GMT_CUDA(cudaStreamWaitEvent(h->stream, finished, 0));
    return r.out;
  }

  void leave() {
    std::lock_guard<std::mutex> lk(mu);
    --members;
    if (members > 0 && (int)pending.size() == members) launch_locked();
  }
};

namespace {
thread_local BatchGroup* t_group = nullptr;    // the group of this solve thread
thread_local cudaEvent_t t_ready = nullptr;    // its event before each V-cycle
thread_local bool t_batch_thread = false;      // a solve thread of gmt_solve_batch
}  // namespace

void leave_batch_group() {
  if (t_group) {
    BatchGroup* g = t_group;
    t_group = nullptr;
    g->leave();
  }
}

static void* group_vcycle(gmt_hierarchy* h, Workspace* w, int form) {
  return t_group->vcycle(h, w, form, t_ready);
}

bool in_batch_group(const Workspace* w) { return t_group != nullptr && w->prec == P32; }
bool batch_thread() { return t_batch_thread; }

void run_batched(gmt_hierarchy* const* hs, int n, const std::function<void(int)>& body) {
  BatchGroup g;
  g.members = n;
  GMT_CUDA(cudaSetDevice(hs[0]->device));
  GMT_CUDA(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
  cudaError_t ce = cudaEventCreateWithFlags(&g.finished, cudaEventDisableTiming);
  g.ready.assign(n, nullptr);
  for (int i = 0; i < n && ce == cudaSuccess; ++i)
    ce = cudaEventCreateWithFlags(&g.ready[i], cudaEventDisableTiming);
  auto cleanup = [&]() {
    for (cudaEvent_t e : g.ready)
      if (e) cudaEventDestroy(e);
    if (g.finished) cudaEventDestroy(g.finished);
    cudaStreamSynchronize(g.stream);
    cudaStreamDestroy(g.stream);
  };
  if (ce != cudaSuccess) {
    cleanup();
    GMT_CUDA(ce);
  }
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i]() {
      t_group = &g;
      t_ready = g.ready[i];
      t_batch_thread = true;
      body(i);               // catches its own failures and calls leave_batch_group()
      leave_batch_group();   // (a no-op when body has left)
      t_batch_thread = false;
    });
  for (std::thread& t : th) t.join();
  cleanup();
}

}  // namespace gmt
