// Sparse periodic hierarchy on the device (Sec. 4.1 "Domain Discretization" and
// "Solver-Aligned Hierarchy Construction"; App. E.1 periodic wrap).
//
//   level 0 elements  = solid voxels
//   node octant mask  = bit o set when element (p - o) mod N_l is active
//   active nodes      = sites with a nonzero mask (vertex union, eq. gmgcoarsenode)
//   coarse element X  = active when any child 2X + c is active (conservative rule)
//
// Everything is computed by kernels on dense N_l^3 flag grids, then compacted into 4^3
// bricks with exclusive scans. Counts are read back once per level to size allocations.
#include <atomic>
#include <map>
#include <set>
#include <mutex>
#include <unordered_map>
#include <cstdarg>
#include <cstring>

#include "common.cuh"

namespace gmt {

// ------------------------------------------------------------------ errors and arena
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* last_error() { return g_err; }

// ------------------------------------------------------------------ caching allocator
// Process-wide pool of device blocks keyed by (device, size bucket). cudaMalloc and
// cudaFree synchronise the device and cost tens to hundreds of microseconds each; a solve
// per cell would otherwise pay dozens of them. Buckets: powers of two up to 1 MB, then
// multiples of 1 MB. Released blocks return to the pool; gmt_release_cached_memory() (or
// a failed cudaMalloc) hands the cached blocks back to the driver.
namespace {
struct Pool {
  std::mutex mu;
  std::map<std::pair<int, size_t>, std::vector<void*>> free_blocks;
  std::unordered_map<void*, std::pair<int, size_t>> owner;
  size_t cached = 0;
};
Pool& pool() {
  static Pool* p = new Pool();   // never destroyed: blocks may outlive static destructors
  return *p;
}
size_t bucket(size_t n) {
  if (n <= 256) return 256;
  if (n <= (1u << 20)) {
    size_t b = 256;
    while (b < n) b <<= 1;
    return b;
  }
  return (n + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
}
void trim_locked(Pool& P) {
  for (auto& kv : P.free_blocks)
    for (void* q : kv.second) {
      cudaFree(q);
      P.owner.erase(q);
    }
  P.free_blocks.clear();
  P.cached = 0;
}
}  // namespace

void* pool_alloc(size_t n) {
  int dev = 0;
  GMT_CUDA(cudaGetDevice(&dev));
  const size_t sz = bucket(n);
  Pool& P = pool();
  std::lock_guard<std::mutex> lock(P.mu);
  auto it = P.free_blocks.find({dev, sz});
  if (it != P.free_blocks.end() && !it->second.empty()) {
    void* q = it->second.back();
    it->second.pop_back();
    P.cached -= sz;
    return q;
  }
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sz);
  if (e != cudaSuccess) {  // give the cache back to the driver and retry once
    cudaGetLastError();
    trim_locked(P);
    e = cudaMalloc(&q, sz);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu bytes) failed: %s", sz, cudaGetErrorString(e));
    throw Fail{GMT_ERR_OOM};
  }
  P.owner[q] = {dev, sz};
  return q;
}

void pool_free(void* q) {
  if (!q) return;
  Pool& P = pool();
  std::lock_guard<std::mutex> lock(P.mu);
  auto it = P.owner.find(q);
  if (it == P.owner.end()) return;
  P.free_blocks[it->second].push_back(q);
  P.cached += it->second.second;
}

void pool_trim() {
  Pool& P = pool();
  std::lock_guard<std::mutex> lock(P.mu);
  trim_locked(P);
}

size_t pool_cached_bytes() {
  Pool& P = pool();
  std::lock_guard<std::mutex> lock(P.mu);
  return P.cached;
}

void* Arena::raw(size_t n) {
  void* p = pool_alloc(n);
  ptrs.push_back(p);
  bytes += bucket(n);
  return p;
}

void Arena::release() {
  // like cudaFree, wait for device work that may still use the blocks before they can be
  // handed to another allocation
  if (!ptrs.empty()) {
    if (has_stream) cudaStreamSynchronize(stream);
    else cudaDeviceSynchronize();
  }
  for (void* p : ptrs) pool_free(p);
  ptrs.clear();
  bytes = 0;
}

void ensure_smem_attr(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  GMT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kernel, dev})) return;
  GMT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({kernel, dev});
}

// ------------------------------------------------------------------ graph lock
namespace {
std::atomic<int> g_inflight{0};
std::mutex g_graph_mu;
// graph executables waiting for a moment without other calls in flight (under g_graph_mu;
// never destroyed: they may outlive static destructors)
std::vector<cudaGraphExec_t>* g_retired = new std::vector<cudaGraphExec_t>();
void drain_retired_locked() {
  for (cudaGraphExec_t e : *g_retired) cudaGraphExecDestroy(e);
  g_retired->clear();
}
}  // namespace

ApiGuard::ApiGuard(bool may_drain) : drain(may_drain) {
  g_inflight.fetch_add(1);
  std::lock_guard<std::mutex> lock(g_graph_mu);   // wait for a graph operation in progress
}

ApiGuard::~ApiGuard() {
  if (g_inflight.fetch_sub(1) == 1 && drain) {   // the last call in flight: destroy retired graphs
    std::lock_guard<std::mutex> lock(g_graph_mu);
    if (g_inflight.load() == 0 && !g_retired->empty()) drain_retired_locked();
  }
}

GraphLock::GraphLock() {
  g_graph_mu.lock();
  held = true;
  // a call that entered after this point waits in its ApiGuard until release(); one that
  // entered before is counted here
  alone = g_inflight.load() == 1;
  if (alone && !g_retired->empty()) drain_retired_locked();
}

void GraphLock::release() {
  if (held) g_graph_mu.unlock();
  held = false;
  alone = false;
}

GraphLock::~GraphLock() { release(); }

void retire_graph(cudaGraphExec_t e) {
  if (!e) return;
  std::lock_guard<std::mutex> lock(g_graph_mu);
  g_retired->push_back(e);
}

// ------------------------------------------------------------------ launch counting, tracing
static std::atomic<int64_t> g_launches{0};
static thread_local int64_t t_launches = 0;   // this host thread's launches
void count_launch(int64_t n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
int64_t launch_count() { return g_launches.load(); }
int64_t thread_launch_count() { return t_launches; }

cudaEvent_t Tracer::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  GMT_CUDA(cudaEventCreate(&e));
  return e;
}

void Tracer::flush() {
  for (Rec& r : recs) {
    float t = 0.f;
    GMT_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    launches[r.cat] += 1;
    ms[r.cat] += t;
    bytes[r.cat] += r.bytes;
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  recs.clear();
}

void Tracer::reset() {
  for (Rec& r : recs) {
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  recs.clear();
  for (int c = 0; c < TR_NCAT; ++c) {
    launches[c] = 0;
    ms[c] = 0;
    bytes[c] = 0;
  }
}

void Tracer::destroy() {
  reset();
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
  pool.clear();
}

TraceScope::TraceScope(Tracer* tr, cudaStream_t st, int c, double b)
    : t(tr), s(st), cat(c), bytes(b) {
  if (t && t->on && (!t->brackets_only || c == TR_VCYCLE)) {
    a = t->get();
    GMT_CUDA(cudaEventRecord(a, s));
  }
}

TraceScope::~TraceScope() {
  if (a) {
    cudaEvent_t b = t->get();
    cudaEventRecord(b, s);
    t->recs.push_back(Tracer::Rec{cat, bytes, a, b});
  }
}

// ------------------------------------------------------------------ exclusive scan
// Three phases: per-block scan of 4096 int32 values, recursive scan of the block totals,
// offset add. Deterministic (integer).
constexpr int SCAN_T = 1024, SCAN_V = 4, SCAN_TILE = SCAN_T * SCAN_V;

__global__ void __launch_bounds__(SCAN_T) k_scan_tile(const int* __restrict__ in,
                                                      int* __restrict__ out,
                                                      int* __restrict__ sums, int64_t n) {
  __shared__ int warp_tot[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_V;
  int v[SCAN_V];
  int run = 0;
#pragma unroll
  for (int i = 0; i < SCAN_V; ++i) {
    int x = (base + i < n) ? in[base + i] : 0;
    v[i] = run;
    run += x;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int t = warp_tot[lane];
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == 31) sums[blockIdx.x] = ti;
  }
  __syncthreads();
  int off = warp_tot[w] + incl - run;
#pragma unroll
  for (int i = 0; i < SCAN_V; ++i)
    if (base + i < n) out[base + i] = v[i] + off;
}

__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ offs, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / SCAN_TILE];
}

static void scan_rec(const int* in, int* out, int64_t n, Arena& tmp, cudaStream_t s) {
  int64_t nblk = (n + SCAN_TILE - 1) / SCAN_TILE;
  int* sums = tmp.alloc<int>(nblk);
  k_scan_tile<<<(unsigned)nblk, SCAN_T, 0, s>>>(in, out, sums, n);
  GMT_LAUNCH_CHECK();
  if (nblk > 1) {
    int* offs = tmp.alloc<int>(nblk);
    scan_rec(sums, offs, nblk, tmp, s);
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, offs, n);
    GMT_LAUNCH_CHECK();
  }
}

// Exclusive scan of n flags; returns the total (synchronizes the stream).
static int64_t exclusive_scan(const int* in, int* out, int64_t n, Arena& tmp, cudaStream_t s) {
  scan_rec(in, out, n, tmp, s);
  int last_in = 0, last_out = 0;
  GMT_CUDA(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMT_CUDA(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMT_CUDA(cudaStreamSynchronize(s));
  return (int64_t)last_in + last_out;
}

// ------------------------------------------------------------------ kernels

__global__ void k_vox_to_flags(const uint8_t* __restrict__ vox, uint8_t* __restrict__ ef,
                               int64_t n3) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) ef[i] = vox[i] ? 1 : 0;
}

// coarse element X active iff any child 2X + c is; child bit c = child c active
__global__ void k_coarsen(const uint8_t* __restrict__ ef, int nf, uint8_t* __restrict__ ec,
                          uint8_t* __restrict__ child) {
  int nc = nf >> 1;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nc * nc * nc) return;
  int x = (int)(i % nc), y = (int)((i / nc) % nc), z = (int)(i / ((int64_t)nc * nc));
  unsigned m = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int fx = 2 * x + (c & 1), fy = 2 * y + ((c >> 1) & 1), fz = 2 * z + ((c >> 2) & 1);
    if (ef[fx + (int64_t)nf * (fy + (int64_t)nf * fz)]) m |= 1u << c;
  }
  child[i] = (uint8_t)m;
  ec[i] = m ? 1 : 0;
}

// octant mask of every node site: bit o <- element (p - o) mod n
__global__ void k_node_masks(const uint8_t* __restrict__ ef, int n, uint8_t* __restrict__ nm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n * n) return;
  int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((int64_t)n * n));
  unsigned m = 0;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    int ex = x - (o & 1), ey = y - ((o >> 1) & 1), ez = z - ((o >> 2) & 1);
    ex += ex < 0 ? n : 0;
    ey += ey < 0 ? n : 0;
    ez += ez < 0 ? n : 0;
    if (ef[ex + (int64_t)n * (ey + (int64_t)n * ez)]) m |= 1u << o;
  }
  nm[i] = (uint8_t)m;
}

__global__ void k_brick_flags(const uint8_t* __restrict__ nm, int n, int nbx,
                              int* __restrict__ flags) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= (int64_t)nbx * nbx * nbx) return;
  int bx = (int)(b % nbx), by = (int)((b / nbx) % nbx), bz = (int)(b / ((int64_t)nbx * nbx));
  int any = 0;
  for (int l = 0; l < 64 && !any; ++l) {
    int x = 4 * bx + (l & 3), y = 4 * by + ((l >> 2) & 3), z = 4 * bz + (l >> 4);
    any = nm[x + (int64_t)n * (y + (int64_t)n * z)] != 0;
  }
  flags[b] = any;
}

__global__ void k_brick_compact(const int* __restrict__ flags, const int* __restrict__ pre,
                                int nbx, int* __restrict__ bmap, int* __restrict__ bxyz) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= (int64_t)nbx * nbx * nbx) return;
  if (flags[b]) {
    int k = pre[b];
    bmap[b] = k;
    bxyz[3 * k + 0] = (int)(b % nbx);
    bxyz[3 * k + 1] = (int)((b / nbx) % nbx);
    bxyz[3 * k + 2] = (int)(b / ((int64_t)nbx * nbx));
  } else {
    bmap[b] = -1;
  }
}

__global__ void k_brick_nbr(const int* __restrict__ bxyz, const int* __restrict__ bmap,
                            int nbx, int64_t nb, int* __restrict__ nbr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * 27) return;
  int64_t k = i / 27;
  int d = (int)(i % 27);
  int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
  int x = (bxyz[3 * k] + dx + nbx) % nbx;
  int y = (bxyz[3 * k + 1] + dy + nbx) % nbx;
  int z = (bxyz[3 * k + 2] + dz + nbx) % nbx;
  nbr[i] = bmap[x + (int64_t)nbx * (y + (int64_t)nbx * z)];
}


// per node site: write mask into its slot; flag active nodes / elements for numbering
__global__ void k_site_pass(const uint8_t* __restrict__ nm, const uint8_t* __restrict__ ef,
                            int n, int nbx, const int* __restrict__ bmap, bool dense,
                            uint8_t* __restrict__ mask, int* __restrict__ nflag,
                            int* __restrict__ eflag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n * n) return;
  int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((int64_t)n * n));
  uint8_t m = nm[i];
  nflag[i] = m != 0;
  eflag[i] = ef[i] != 0;
  if (m) {
    int64_t s = site_slot(x, y, z, n, nbx, bmap, dense);
    mask[s] = m;
  }
}

__global__ void k_numbering(const uint8_t* __restrict__ nm, const uint8_t* __restrict__ ef,
                            const uint8_t* __restrict__ child, const int* __restrict__ npre,
                            const int* __restrict__ epre, int n, int nbx,
                            const int* __restrict__ bmap, bool dense, int level,
                            int* __restrict__ slot_canon, int* __restrict__ canon_slot,
                            int* __restrict__ kidx, int* __restrict__ elem_slot) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n * n) return;
  if (!nm[i]) return;
  int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((int64_t)n * n));
  int64_t s = site_slot(x, y, z, n, nbx, bmap, dense);
  int c = npre[i];
  slot_canon[s] = c;
  canon_slot[c] = (int)s;
  if (ef[i]) {
    int e = epre[i];
    elem_slot[e] = (int)s;
    kidx[s] = level == 0 ? 0 : (level == 1 ? (int)child[i] : e);
  }
}

template <typename T>
__global__ void k_fill(T* __restrict__ p, T v, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

template <typename T>
static void fill(T* p, T v, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<T><<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
  GMT_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ host driver
int choose_levels(int n, int coarsest_max) {
  int L = 1;
  while ((n >> (L - 1)) > coarsest_max && n % (1 << (L + 1)) == 0) ++L;
  return L;
}

void build_hierarchy(gmt_hierarchy* h, const uint8_t* vox, bool on_device) {
  cudaStream_t s = h->stream;
  TraceScope ts(&h->tracer, s, TR_SETUP, 0.0);
  const int N = h->N;
  const int64_t n3 = (int64_t)N * N * N;
  Arena tmp(s);
  uint8_t* dvox = nullptr;
  if (on_device) {
    dvox = const_cast<uint8_t*>(vox);
  } else {
    dvox = tmp.alloc<uint8_t>(n3);
    GMT_CUDA(cudaMemcpyAsync(dvox, vox, n3, cudaMemcpyHostToDevice, s));
  }
  h->lv.assign(h->L, Level());
  int* flags = tmp.alloc<int>(n3);
  int* pre = tmp.alloc<int>(n3);
  int* eflg = tmp.alloc<int>(n3);
  int* epre = tmp.alloc<int>(n3);
  uint8_t* nm = tmp.alloc<uint8_t>(n3);
  for (int l = 0; l < h->L; ++l) {
    Level& lv = h->lv[l];
    const int n = N >> l;
    const int64_t s3 = (int64_t)n * n * n;
    lv.n = n;
    lv.eflag = h->geo.alloc<uint8_t>(s3);
    if (l == 0) {
      k_vox_to_flags<<<grid_for(s3, 256), 256, 0, s>>>(dvox, lv.eflag, s3);
      GMT_LAUNCH_CHECK();
    } else {
      lv.child = h->geo.alloc<uint8_t>(s3);
      k_coarsen<<<grid_for(s3, 256), 256, 0, s>>>(h->lv[l - 1].eflag, 2 * n, lv.eflag, lv.child);
      GMT_LAUNCH_CHECK();
    }
    k_node_masks<<<grid_for(s3, 256), 256, 0, s>>>(lv.eflag, n, nm);
    GMT_LAUNCH_CHECK();
    lv.dense = (n % 4) != 0;
    if (!lv.dense) {
      lv.nbx = n / 4;
      const int64_t nb3 = (int64_t)lv.nbx * lv.nbx * lv.nbx;
      k_brick_flags<<<grid_for(nb3, 128), 128, 0, s>>>(nm, n, lv.nbx, flags);
      GMT_LAUNCH_CHECK();
      lv.nb = exclusive_scan(flags, pre, nb3, tmp, s);
      GMT_REQUIRE(lv.nb > 0, GMT_ERR_EMPTY, "cell has no active element");
      lv.brick_map = h->geo.alloc<int>(nb3);
      lv.brick_xyz = h->geo.alloc<int>(lv.nb * 3);
      lv.brick_nbr = h->geo.alloc<int>(lv.nb * 27);
      k_brick_compact<<<grid_for(nb3, 256), 256, 0, s>>>(flags, pre, lv.nbx, lv.brick_map,
                                                         lv.brick_xyz);
      GMT_LAUNCH_CHECK();
      k_brick_nbr<<<grid_for(lv.nb * 27, 256), 256, 0, s>>>(lv.brick_xyz, lv.brick_map, lv.nbx,
                                                            lv.nb, lv.brick_nbr);
      GMT_LAUNCH_CHECK();
      lv.nslots = lv.nb * 64;
    } else {
      lv.nslots = (s3 + 63) / 64 * 64;
      lv.nb = lv.nslots / 64;
    }
    lv.mask = h->geo.alloc<uint8_t>(lv.nslots);
    lv.slot_canon = h->geo.alloc<int>(lv.nslots);
    lv.kidx = h->geo.alloc<int>(lv.nslots);
    GMT_CUDA(cudaMemsetAsync(lv.mask, 0, lv.nslots, s));
    fill<int>(lv.slot_canon, -1, lv.nslots, s);
    fill<int>(lv.kidx, -1, lv.nslots, s);
    k_site_pass<<<grid_for(s3, 256), 256, 0, s>>>(nm, lv.eflag, n, lv.nbx, lv.brick_map, lv.dense,
                                                  lv.mask, flags, eflg);
    GMT_LAUNCH_CHECK();
    lv.n_nodes = exclusive_scan(flags, pre, s3, tmp, s);
    lv.n_elems = exclusive_scan(eflg, epre, s3, tmp, s);
    GMT_REQUIRE(lv.n_elems > 0, GMT_ERR_EMPTY, "cell has no active element");
    lv.canon_slot = h->geo.alloc<int>(lv.n_nodes);
    lv.elem_slot = h->geo.alloc<int>(lv.n_elems);
    k_numbering<<<grid_for(s3, 256), 256, 0, s>>>(nm, lv.eflag, lv.child, pre, epre, n, lv.nbx,
                                                  lv.brick_map, lv.dense, l, lv.slot_canon,
                                                  lv.canon_slot, lv.kidx, lv.elem_slot);
    GMT_LAUNCH_CHECK();
  }
  GMT_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ exports

__global__ void k_export_nodes(const int* __restrict__ canon_slot, const uint8_t* __restrict__ mask,
                               const int* __restrict__ bxyz, int n, bool dense, int64_t cnt,
                               int32_t* __restrict__ xyz, uint8_t* __restrict__ mout) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  int64_t s = canon_slot[i];
  int x, y, z;
  slot_coords(s, n, dense, bxyz, x, y, z);
  xyz[3 * i] = x;
  xyz[3 * i + 1] = y;
  xyz[3 * i + 2] = z;
  if (mout) mout[i] = mask[s];
}

__global__ void k_export_elems(const int* __restrict__ elem_slot, const int* __restrict__ bxyz,
                               const uint8_t* __restrict__ child, int n, bool dense, int64_t cnt,
                               int32_t* __restrict__ xyz, uint8_t* __restrict__ cout) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  int64_t s = elem_slot[i];
  int x, y, z;
  slot_coords(s, n, dense, bxyz, x, y, z);
  xyz[3 * i] = x;
  xyz[3 * i + 1] = y;
  xyz[3 * i + 2] = z;
  if (cout) cout[i] = child ? child[x + (int64_t)n * (y + (int64_t)n * z)] : 0;
}

// App. E.1/E.2 stencil tuples of every canonical node of the fine level
__global__ void k_export_stencil(const int* __restrict__ canon_slot, const int* __restrict__ fbxyz,
                                 int nf, const int* __restrict__ cbmap, int nc, int cnbx,
                                 bool cdense, const int* __restrict__ cslot_canon, int64_t cnt,
                                 int32_t* __restrict__ idx, double* __restrict__ w) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  int x, y, z;
  slot_coords(canon_slot[i], nf, false, fbxyz, x, y, z);
  for (int k = 0; k < 8; ++k) {
    int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
    int f[3] = {x, y, z};
    double wt = 1.0;
    int c[3];
    for (int d = 0; d < 3; ++d) {
      double xi = 0.5 * (f[d] & 1);
      wt *= 1.0 - fabs(xi - o[d]);
      c[d] = ((f[d] >> 1) + o[d]) % nc;
    }
    if (wt == 0.0) {
      idx[8 * i + k] = -1;
      w[8 * i + k] = 0.0;
    } else {
      int64_t cs = site_slot(c[0], c[1], c[2], nc, cnbx, cbmap, cdense);
      idx[8 * i + k] = cs < 0 ? -2 : cslot_canon[cs];
      w[8 * i + k] = wt;
    }
  }
}

void export_nodes(gmt_hierarchy* h, int l, int32_t* xyz, uint8_t* m) {
  const Level& lv = h->lv[l];
  k_export_nodes<<<grid_for(lv.n_nodes, 256), 256, 0, h->stream>>>(
      lv.canon_slot, lv.mask, lv.brick_xyz, lv.n, lv.dense, lv.n_nodes, xyz, m);
  GMT_LAUNCH_CHECK();
}

void export_elems(gmt_hierarchy* h, int l, int32_t* xyz, uint8_t* c) {
  const Level& lv = h->lv[l];
  k_export_elems<<<grid_for(lv.n_elems, 256), 256, 0, h->stream>>>(
      lv.elem_slot, lv.brick_xyz, lv.child, lv.n, lv.dense, lv.n_elems, xyz, c);
  GMT_LAUNCH_CHECK();
}

void export_stencil(gmt_hierarchy* h, int l, int32_t* idx, double* w) {
  const Level& f = h->lv[l];
  const Level& c = h->lv[l + 1];
  k_export_stencil<<<grid_for(f.n_nodes, 128), 128, 0, h->stream>>>(
      f.canon_slot, f.brick_xyz, f.n, c.brick_map, c.n, c.nbx, c.dense, c.slot_canon, f.n_nodes,
      idx, w);
  GMT_LAUNCH_CHECK();
}

}  // namespace gmt
