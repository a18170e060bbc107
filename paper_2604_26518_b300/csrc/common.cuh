// Internal definitions shared by the library's translation units.
//
// Data layout (all non-coarsest levels): the N_l^3 node sites are cut into 4x4x4 bricks;
// only bricks that hold at least one active node are stored. A "slot" is
// brick * 64 + (x & 3) + 4 (y & 3) + 16 (z & 3). A field with C values per node
// (C = D * M: components x load cases) is stored brick-major, value-major inside the
// brick: value v of slot s lives at (s >> 6) * 64 * C + v * 64 + (s & 63), so a warp
// reading one value of 32 consecutive slots touches 128 contiguous bytes. Inactive nodes
// inside stored bricks hold 0. The coarsest level uses the same formula on a dense
// N_L^3 slot range (slot = x + N y + N^2 z), padded to a multiple of 64.
// Value index v = component * M + case, matching the canonical [node][comp][case] order.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "gmt.h"

namespace gmt {

// ------------------------------------------------------------------ error handling
void set_error(const char* fmt, ...);
const char* last_error();

struct Fail {
  gmt_status status;
};

#define GMT_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      ::gmt::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                       __LINE__);                                                         \
      throw ::gmt::Fail{e_ == cudaErrorMemoryAllocation ? GMT_ERR_OOM : GMT_ERR_CUDA};   \
    }                                                                                     \
  } while (0)

// every kernel launch site ends with GMT_LAUNCH_CHECK(), which also counts the launch
void count_launch(int64_t n = 1);
int64_t thread_launch_count();   // launches counted by the calling host thread

// CUDA-graph operations (capture, instantiation, replay, destruction) never overlap a
// kernel launch of another host thread through this library: concurrent solves on separate
// streams, with one thread capturing or replaying a V-cycle graph while others launched,
// crashed inside the driver's kernel launch (a null dereference in cuLaunchKernel).
// Every entry point holds an ApiGuard: it counts the calls in flight and, on entry, waits
// for a graph operation that holds the graph lock. A GraphLock takes that lock; its
// `alone` says that no other library call is in flight, and only then may the holder run
// graph operations. Graph executables released while other calls are in flight are
// retired and destroyed at the next moment the library is alone.
struct ApiGuard {
  explicit ApiGuard(bool may_drain = true);   // false: never destroys retired graphs
  ~ApiGuard();
  bool drain;
  ApiGuard(const ApiGuard&) = delete;
  ApiGuard& operator=(const ApiGuard&) = delete;
};
struct GraphLock {
  GraphLock();
  ~GraphLock();
  void release();   // unlock early (idempotent)
  bool alone = false;
  bool held = false;
  GraphLock(const GraphLock&) = delete;
  GraphLock& operator=(const GraphLock&) = delete;
};
void retire_graph(cudaGraphExec_t e);
#define GMT_LAUNCH_CHECK()              \
  do {                                  \
    ::gmt::count_launch();              \
    GMT_CUDA(cudaGetLastError());       \
  } while (0)

#define GMT_REQUIRE(cond, st, ...)        \
  do {                                    \
    if (!(cond)) {                        \
      ::gmt::set_error(__VA_ARGS__);      \
      throw ::gmt::Fail{st};              \
    }                                     \
  } while (0)

// ------------------------------------------------------------------ layout helpers
__host__ __device__ __forceinline__ int64_t vaddr(int64_t slot, int v, int C) {
  return (slot >> 6) * (int64_t)(64 * C) + (int64_t)v * 64 + (slot & 63);
}

// slot of node site (x, y, z) of a level: dense levels index the site directly, bricked
// levels go through the brick map (-1 when the brick is not stored)
__device__ __forceinline__ int64_t site_slot(int x, int y, int z, int n, int nbx,
                                             const int* bmap, bool dense) {
  if (dense) return x + (int64_t)n * (y + (int64_t)n * z);
  int b = bmap[(x >> 2) + (int64_t)nbx * ((y >> 2) + (int64_t)nbx * (z >> 2))];
  if (b < 0) return -1;
  return (int64_t)b * 64 + (x & 3) + 4 * (y & 3) + 16 * (z & 3);
}

__device__ __forceinline__ void slot_coords(int64_t s, int n, bool dense, const int* bxyz,
                                            int& x, int& y, int& z) {
  if (dense) {
    x = (int)(s % n);
    y = (int)((s / n) % n);
    z = (int)(s / ((int64_t)n * n));
  } else {
    int64_t b = s >> 6;
    int l = (int)(s & 63);
    x = 4 * bxyz[3 * b] + (l & 3);
    y = 4 * bxyz[3 * b + 1] + ((l >> 2) & 3);
    z = 4 * bxyz[3 * b + 2] + (l >> 4);
  }
}

static inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T> __device__ __forceinline__ float to_f(T x);
template <> __device__ __forceinline__ float to_f<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

template <typename A, typename T> __device__ __forceinline__ A load_as(const T* p) {
  return (A)(*p);
}
template <> __device__ __forceinline__ float load_as<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <typename T, typename A> __device__ __forceinline__ T store_as(A x) { return (T)x; }
template <> __device__ __forceinline__ __nv_bfloat16 store_as<__nv_bfloat16, float>(float x) {
  return __float2bfloat16_rn(x);
}

// ------------------------------------------------------------------ device arena
// Every device allocation of a hierarchy goes through one Arena, which owns it until the
// hierarchy is freed (or the material-dependent part is rebuilt).
// process-wide caching device allocator (hierarchy.cu)
void* pool_alloc(size_t n);
void pool_free(void* p);
void pool_trim();
size_t pool_cached_bytes();

// Blocks from the caching pool, returned on release() after the work that may still use
// them has finished: the arena's stream when it has one (so that hierarchies on other
// streams keep running), else the whole device.
struct Arena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  bool has_stream = false;
  Arena() = default;
  explicit Arena(cudaStream_t s) : stream(s), has_stream(true) {}
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  void bind(cudaStream_t s) {
    stream = s;
    has_stream = true;
  }
  void* raw(size_t n);
  template <typename T> T* alloc(size_t count) { return (T*)raw(count * sizeof(T)); }
  void release();
  ~Arena() { release(); }
};

// dynamic shared memory above the 48 KB default for a kernel on the current device (set
// once per kernel and device; thread-safe)
void ensure_smem_attr(const void* kernel, int bytes);

// ------------------------------------------------------------------ hierarchy
struct Level {
  int n = 0;             // N_l
  int nbx = 0;           // n / 4 for bricked levels
  bool dense = false;    // coarsest level stored as a dense slot range
  int64_t nb = 0;        // stored bricks (dense: nslots / 64)
  int64_t nslots = 0;    // nb * 64
  int64_t n_nodes = 0, n_elems = 0;
  // geometry (device)
  uint8_t* eflag = nullptr;     // dense n^3 element flags (1 = active)
  uint8_t* child = nullptr;     // dense n^3 child masks (levels >= 1)
  int* brick_map = nullptr;     // nbx^3 -> brick or -1 (bricked)
  int* brick_xyz = nullptr;     // nb x 3 (bricked)
  int* brick_nbr = nullptr;     // nb x 27, index (dz+1)*9 + (dy+1)*3 + (dx+1) (bricked)
  uint8_t* mask = nullptr;      // nslots octant masks (0 = inactive node)
  int* slot_canon = nullptr;    // nslots -> canonical node or -1
  int* canon_slot = nullptr;    // n_nodes -> slot
  int* kidx = nullptr;          // nslots -> element-matrix index of the element with origin
                                // at this slot (level 1: child mask; >= 2: element id), -1
  int* elem_slot = nullptr;     // n_elems -> slot of the element's origin (canonical order)
  int* slot_elem = nullptr;     // level 0, lazy: slot -> canonical element or -1
  int* kidx_el = nullptr;       // level 1 with element densities: slot -> element id (the
                                // level's matrices are then stored per element, not per mask)
  // material-dependent operator data (device)
  double* K64 = nullptr;        // level 1: [256][MM] table; level >= 2: [n_elems][MM]
  float* K32 = nullptr;
  double* S64 = nullptr;        // levels >= 1: per-node stencils [brick][27 D D][64] (lazy)
  float* S32 = nullptr;
  uint16_t* S16 = nullptr;      // levels >= 1 with coarse_fp16: FP16 copy of S32 / s16_scale
  float s16_scale = 0.f;        //   [brick][27 D D / 8 groups][64][8] (lazy)
  double* dinv64 = nullptr;     // levels >= 1: nslots x D*D block-diagonal inverses
  float* dinv32 = nullptr;
  double lmax = 0.0;            // Chebyshev: estimate of lambda_max(D^-1 K)
};

struct Material {
  int physics = -1;
  double E = 0, nu = 0, k = 0;
  int D = 0, M = 0, C = 0, MM = 0;   // dofs/node, cases, values/node, (8D)^2
  double Ke[576];                    // element matrix, (8D) x (8D) row-major
  double Fe[144];                    // K_e x0, (8D) x M
  double X0[144];                    // x0, (8D) x M
  double C0[36];                     // x0^T K_e x0 (base tensor)
  double gross[6];                   // sqrt(n_e * ||K_e x0_m||^2) per case
};

struct Workspace;  // solver buffers (solver.cu)

// Per-hierarchy event tracing of kernel launches (see gmt_trace_* in gmt.h)
enum TraceCat {
  TR_SMOOTH0 = 0, TR_RESID0 = 1, TR_APPLY0 = 2, TR_OUTER = 3, TR_DIAG0 = 4, TR_COARSE_ST = 5,
  TR_RESTRICT = 6, TR_PROLONG = 7, TR_CSOLVE = 8, TR_ENERGY = 9, TR_VEC = 10, TR_SETUP = 11,
  TR_OPS = 12, TR_CINV = 13, TR_COARSE_ST2 = 14,
  TR_VCYCLE = 15,   // a whole V-cycle (one event pair around the level-0 cycle)
  TR_NCAT = 16
};
struct Tracer {
  bool on = false;
  bool brackets_only = false;   // record only TR_VCYCLE (no per-launch events inside it)
  struct Rec {
    int cat;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> recs;
  int64_t launches[TR_NCAT] = {0};
  double ms[TR_NCAT] = {0};
  double bytes[TR_NCAT] = {0};
  cudaEvent_t get();
  void flush();      // harvest completed records (synchronize first)
  void reset();
  void destroy();
};

// RAII scope recording an event pair around the launches it encloses
struct TraceScope {
  Tracer* t;
  cudaStream_t s;
  int cat;
  double bytes;
  cudaEvent_t a = nullptr;
  TraceScope(Tracer* tr, cudaStream_t st, int c, double b);
  ~TraceScope();
};

}  // namespace gmt

struct gmt_hierarchy {
  int device = 0;
  cudaStream_t stream = nullptr;
  gmt_options opts;
  int N = 0, L = 0;
  std::vector<gmt::Level> lv;
  gmt::Arena geo;         // geometry allocations
  gmt::Arena op;          // material-dependent allocations
  gmt::Arena work;        // solver work buffers
  gmt::Material mat;
  bool prepared = false;
  double* Ke64 = nullptr;  // device copies of the level-0 element matrix
  float* Ke32 = nullptr;
  // coarsest level, m = n_nodes(L-1) * D: regularized dense matrix (FP64), its FP32
  // generalized inverse, and the exact FP64 inverse (built on first FP64 use)
  int64_t m = 0;
  double* A64 = nullptr;
  float* X32 = nullptr;
  double* Ainv = nullptr;
  double* cscal = nullptr;  // device [rho, FP32 pivot tolerance, FP64 pivot tolerance]
  double* cb = nullptr;   // m x M gather buffer
  double* cu = nullptr;   // m x M result buffer
  float* cb32 = nullptr;  // m x M FP32 copy of the right-hand side / refinement residual
  gmt::Workspace* ws = nullptr;
  gmt::Tracer tracer;
  bool have_solution = false;
  int64_t ws_for_prec = -1;
  // histogram of the level-0 octant masks over active nodes (the load f_n depends on the
  // mask alone); filled on first use
  long long mask_hist[256] = {};
  bool have_hist = false;
  // split-column reductions: per-block (sum, compensation) pairs and arrival tickets
  double* red_scratch = nullptr;
  unsigned* red_ticket = nullptr;
  // element densities of the SIMP interpolation (gmt_set_densities): C_e = s_e C0 with
  // s_e = rho_min + rho_e^p. Per level-0 slot (the element whose origin is the slot; 0 where
  // there is none): s_e in FP64 and FP32 and rho_e. With densities the level-0 operator is
  // stored per node (like the coarse levels) and the level-0 load is kept as a vector.
  bool dens = false;
  gmt::Arena dn;
  double* coef64 = nullptr;
  float* coef32 = nullptr;
  double* rho64 = nullptr;
  double rho_min = 0.0, simp_p = 0.0;
  double coef_sum = 0.0, coef_sum2 = 0.0;   // sum of s_e and of s_e^2 over the elements
  double* f0_64 = nullptr;   // level-0 load f = sum_e s_e A_e^T K_e x0 (slot layout; op arena)
  float* f0_32 = nullptr;
};

namespace gmt {
// element-matrix index of the slots of a level as the operator kernels read it
inline const int* op_kidx(const Level& l) { return l.kidx_el ? l.kidx_el : l.kidx; }
// hierarchy.cu
void build_hierarchy(gmt_hierarchy* h, const uint8_t* vox, bool on_device);
int choose_levels(int n, int coarsest_max);
// operators.cu
void prepare_material(gmt_hierarchy* h, int physics, double E, double nu, double k);
void set_densities(gmt_hierarchy* h, const double* rho, bool on_device, double rho_min,
                   double p);
void build_coarse_inverse64(gmt_hierarchy* h);
// solver.cu
void free_workspace(gmt_hierarchy* h);
}  // namespace gmt
