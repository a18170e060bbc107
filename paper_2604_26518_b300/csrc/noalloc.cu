// Allocation-free homogenization: gmt_homogenize_dense_noalloc (declared in gmt.h).
//
// Some callers cannot call cudaMalloc: an application whose memory manager already owns
// the device memory and forbids side allocations, a fixed-budget embedded or sandboxed
// process, or a latency-bound loop that cannot afford the implicit device synchronisation
// of an allocation. For them this entry point evaluates the energy average of the
// homogenized tensor for a nodal field the caller already has, without building a
// hierarchy and without allocating: inputs and the output are the caller's buffers, and
// the only working memory is the file-scope array below, which every GPU that loads the
// library holds until the process exits.
//
// Scratch layout (doubles): [0, 1024) element matrix, loads, affine modes and base tensor
// of the requested material; [1024, 1024 + 2048 * 21) one row of C^H partial sums per
// block of the fixed 2048-block grid. Every call overwrites all of it before reading it,
// so nothing needs clearing, but two calls that overlap on the GPU (different streams, or
// different host threads) share the array and race: serialise them.
#include <mutex>

#include "common.cuh"

namespace gmt {
void launch_element_matrices(cudaStream_t s, int physics, double E, double nu, double kappa,
                             double* out);
}

namespace {

constexpr int kNoallocBlocks = 2048;       // fixed grid of the energy kernel
constexpr int kNoallocK = 21;              // unique entries of a symmetric 6 x 6 tensor
constexpr int kNoallocElem = 1024;         // element-data region
constexpr int kNoallocMaxRes = 512;        // largest accepted cell side N
constexpr size_t kNoallocDoubles = kNoallocElem + (size_t)kNoallocBlocks * kNoallocK;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
double* g_noalloc_addr[kMaxDevices] = {nullptr};

// Per active voxel e: (x0^I - u_e^I)^T K_e (x0^J - u_e^J) for I <= J in FP64, with the
// element field taken relative to its first node (a translation, annihilated by K_e).
// Grid-stride over the N^3 voxels; each block writes its partial row (all blocks write).
// One warp per block; each thread's element field and partial sums live in shared memory
// (indexed at run time there), so the kernel needs no per-thread stack.
constexpr int kEnergyThreads = 32;

template <int D, int M>
__global__ void __launch_bounds__(kEnergyThreads) k_energy_dense(const uint8_t* __restrict__ vox,
                                                                 int n,
                                                                 const double* __restrict__ u,
                                                                 double* __restrict__ scratch) {
  constexpr int C = D * M, R = 8 * D, K = M * (M + 1) / 2;
  constexpr int WS = R * M + 1;               // padded row of one thread's element field
  __shared__ double w[kEnergyThreads * WS];   // w[t][r * M + m]
  __shared__ double e[kEnergyThreads * K];
  const double* Ke = scratch;                 // (8D)^2
  const double* X0 = scratch + R * R + R * M; // after Ke and Fe
  const int t = threadIdx.x;
  double* wt = w + t * WS;
  double* et = e + t * K;
  for (int k = 0; k < K; ++k) et[k] = 0.0;
  const int64_t n3 = (int64_t)n * n * n;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + t; s < n3;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (!vox[s]) continue;
    const int x = (int)(s % n), y = (int)((s / n) % n), z = (int)(s / ((int64_t)n * n));
    const double* u0 = u + s * C;
    for (int a = 0; a < 8; ++a) {
      const int ax = (x + (a & 1)) % n, ay = (y + ((a >> 1) & 1)) % n, az = (z + (a >> 2)) % n;
      const double* ua = u + ((int64_t)ax + (int64_t)n * (ay + (int64_t)n * az)) * C;
      for (int i = 0; i < D; ++i)
        for (int m = 0; m < M; ++m)
          wt[(a * D + i) * M + m] = X0[(a * D + i) * M + m] - (ua[i * M + m] - u0[i * M + m]);
    }
    for (int J = 0; J < M; ++J) {
      for (int r = 0; r < R; ++r) {
        double zr = 0.0;
        for (int c = 0; c < R; ++c) zr += Ke[r * R + c] * wt[c * M + J];
        for (int I = 0; I <= J; ++I) et[I * M - I * (I - 1) / 2 + (J - I)] += wt[r * M + I] * zr;
      }
    }
  }
  __syncwarp();
  if (t < K) {
    double v = 0.0;
    for (int q = 0; q < kEnergyThreads; ++q) v += e[q * K + t];   // fixed order
    scratch[kNoallocElem + (int64_t)blockIdx.x * K + t] = v;
  }
}

// block (I, J): fixed-order, compensated sum over the block partials, scaled by 1/N^3
template <int M>
__global__ void __launch_bounds__(256) k_energy_finish(const double* __restrict__ scratch,
                                                       int n, double* __restrict__ CH) {
  constexpr int K = M * (M + 1) / 2;
  const int I = blockIdx.x / M, J = blockIdx.x % M;
  const int lo = I < J ? I : J, hi = I < J ? J : I;
  const int k = lo * M - lo * (lo - 1) / 2 + (hi - lo);
  __shared__ double ss[256], sc[256];
  double s = 0.0, c = 0.0;
  for (int b = threadIdx.x; b < kNoallocBlocks; b += 256) {
    const double x = scratch[kNoallocElem + (int64_t)b * K + k];
    const double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = ss[threadIdx.x], x = ss[threadIdx.x + o];
      const double t = a + x;
      sc[threadIdx.x] += sc[threadIdx.x + o] + (fabs(a) >= fabs(x) ? (a - t) + x : (x - t) + a);
      ss[threadIdx.x] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) CH[I * M + J] = (ss[0] + sc[0]) / ((double)n * n * n);
}

}  // namespace

extern "C" gmt_status gmt_homogenize_dense_noalloc(const uint8_t* voxels, int res,
                                                   gmt_physics physics, double E, double nu,
                                                   double k, const double* u_dense, double* CH,
                                                   void* stream) {
  gmt::ApiGuard guard(false);   // a lock and a counter; frees and allocates nothing
  gmt::set_error("%s", "");
  if (!voxels || !u_dense || !CH) {
    gmt::set_error("gmt_homogenize_dense_noalloc: null pointer");
    return GMT_ERR_ARG;
  }
  if (res < 1 || res > kNoallocMaxRes) {
    gmt::set_error("gmt_homogenize_dense_noalloc: res %d outside [1, %d]", res, kNoallocMaxRes);
    return GMT_ERR_ARG;
  }
  if (physics == GMT_ELASTIC) {
    if (!(E > 0 && nu > -1.0 && nu < 0.5)) {
      gmt::set_error("gmt_homogenize_dense_noalloc: elastic material needs E > 0, -1 < nu < 0.5");
      return GMT_ERR_ARG;
    }
  } else if (physics == GMT_HEAT) {
    if (!(k > 0)) {
      gmt::set_error("gmt_homogenize_dense_noalloc: heat conduction needs k > 0");
      return GMT_ERR_ARG;
    }
  } else {
    gmt::set_error("gmt_homogenize_dense_noalloc: unknown physics %d", (int)physics);
    return GMT_ERR_ARG;
  }
  int dev = 0;
  cudaError_t rc = cudaGetDevice(&dev);
  if (rc != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    gmt::set_error("gmt_homogenize_dense_noalloc: no usable current device (%s)",
                   cudaGetErrorString(rc));
    return GMT_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the static array
    // (its host-side name is only a stand-in and must not be passed to a kernel)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (rc != cudaSuccess) {
        gmt::set_error("gmt_homogenize_dense_noalloc: cudaGetSymbolAddress failed: %s",
                       cudaGetErrorString(rc));
        return GMT_ERR_CUDA;
      }
      g_noalloc_addr[dev] = (double*)p;
    }
    scratch = g_noalloc_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  try {
    gmt::launch_element_matrices(s, (int)physics, E, nu, k, scratch);
  } catch (const gmt::Fail& f) {
    return f.status;
  }
  if (physics == GMT_ELASTIC) {
    k_energy_dense<3, 6><<<kNoallocBlocks, kEnergyThreads, 0, s>>>(voxels, res, u_dense, scratch);
    k_energy_finish<6><<<36, 256, 0, s>>>(scratch, res, CH);
  } else {
    k_energy_dense<1, 3><<<kNoallocBlocks, kEnergyThreads, 0, s>>>(voxels, res, u_dense, scratch);
    k_energy_finish<3><<<9, 256, 0, s>>>(scratch, res, CH);
  }
  gmt::count_launch(2);
  rc = cudaGetLastError();
  if (rc != cudaSuccess) {
    gmt::set_error("gmt_homogenize_dense_noalloc: launch failed: %s", cudaGetErrorString(rc));
    return GMT_ERR_CUDA;
  }
  return GMT_OK;
}
