// Learned initializer: a sparse 3D convolutional U-Net over the node hierarchy that
// predicts the fine-level cell-problem field from the geometry (Sec. 4.2-4.3 describe the
// paper's learned initial guess; its transformer is replaced here by a convolutional
// U-Net). The prediction enters the solver as its warm start u0 (Alg. 2: the network's
// field followed by V-cycles, with the plain V-cycles continuing until the tolerance is met).
//
// Network (all activations are [node][channel] FP32 over the canonical active-node list of
// a hierarchy level; every convolution has 27 taps, tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)):
//   same-level conv:  z[n] = b + sum_t W[t]^T x[nbr(n, d_t)]            (periodic wrap)
//   down (l -> l+1):  z[q] = b + sum_t W[t]^T x[fine node at 2q + d_t]
//   up   (l+1 -> l):  z[p] = b + sum_t W[t]^T x[coarse node q with p = 2q + d_t]
// (down and up use the parent/child relation of the trilinear transfer of App. E.2), a
// missing neighbour contributes zero, y = relu(z + skip). Layers, widths (w0, w1, w2):
//   0 same@0 8->w0   1 same@0 w0->w0   2 down 0->1 w0->w1   3 same@1 w1->w1
//   4 down 1->2 w1->w2   5 same@2   6 same@2   7 up 2->1 w2->w1 (+ skip from 3)
//   8 same@1   9 up 1->0 w1->w0 (+ skip from 1)   10 same@0   11 same@0 w0->cout (linear)
// Input: the node's 8-bit octant mask as 8 channels of 0/1. Output: cout = D*M channels,
// the field in canonical [node][D][M] order divided by `scale`.
// Parameters: per layer W [27][cin][cout] then b [cout], layers in order, FP32.
// Training: against a solved field u, either the mean squared error of y - u/scale or the
// relative energy norm of the error, (e^T K e) / (u^T K u) with e = scale*y - u summed over
// the load cases (the norm the conjugate-gradient solve minimises, K the level-0 operator of
// Sec. 4.6 applied matrix-free in FP32); AdamW (decoupled weight decay).
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include <cuda_fp16.h>

#include "common.cuh"

namespace gmt {
bool tc_supported(int cin, int cout);                                        // gconv_tc.cu
int64_t tc_image_halves(int cin, int cout);
void tc_build_image(cudaStream_t s, const float* W, int cin, int cout, __half* img);
void launch_gconv_tc(cudaStream_t s, const __half* x, int cin, const int* tab, const __half* img,
                     const float* bias, const __half* add, int relu, float* out32,
                     __half* out16, int cout, int64_t n_out, const int* omap);
void tc_to_half(cudaStream_t s, const float* x, int64_t n, __half* y);
int tc_take_status(cudaStream_t s);
void export_nodes(gmt_hierarchy* h, int l, int32_t* xyz, uint8_t* m);       // hierarchy.cu
void step_apply(gmt_hierarchy* h, int level, int precision, const double* u, double* y);  // solver.cu
}

namespace {

constexpr int NLAYERS = 12;
constexpr int NACT = 13;  // activation 0 is the input, activation i+1 the output of layer i
constexpr int IN_CH = 8;
enum { SAME = 0, DOWN = 1, UP = 2 };

struct LayerDef {
  int kind, lvl_out, in, skip, cin, cout, relu;
};

// layer list for widths w[3] and output channels co
void layer_defs(const int* w, int co, LayerDef* L) {
  const LayerDef d[NLAYERS] = {
      {SAME, 0, 0, -1, IN_CH, w[0], 1}, {SAME, 0, 1, -1, w[0], w[0], 1},
      {DOWN, 1, 2, -1, w[0], w[1], 1},  {SAME, 1, 3, -1, w[1], w[1], 1},
      {DOWN, 2, 4, -1, w[1], w[2], 1},  {SAME, 2, 5, -1, w[2], w[2], 1},
      {SAME, 2, 6, -1, w[2], w[2], 1},  {UP, 1, 7, 4, w[2], w[1], 1},
      {SAME, 1, 8, -1, w[1], w[1], 1},  {UP, 0, 9, 2, w[1], w[0], 1},
      {SAME, 0, 10, -1, w[0], w[0], 1}, {SAME, 0, 11, -1, w[0], co, 0}};
  for (int i = 0; i < NLAYERS; ++i) L[i] = d[i];
}

int act_level(const LayerDef* L, int a) { return a == 0 ? 0 : L[a - 1].lvl_out; }
int act_ch(const LayerDef* L, int a) { return a == 0 ? IN_CH : L[a - 1].cout; }

int64_t param_count(const LayerDef* L) {
  int64_t p = 0;
  for (int i = 0; i < NLAYERS; ++i) p += 27LL * L[i].cin * L[i].cout + L[i].cout;
  return p;
}

constexpr int WG_CHUNK = 1024;  // nodes per weight-gradient partial

// ------------------------------------------------------------------ tables
__device__ __forceinline__ int wrap(int a, int n) { return ((a % n) + n) % n; }

__device__ __forceinline__ int site_canon(int x, int y, int z, const gmt::Level& L) {
  int64_t s = gmt::site_slot(x, y, z, L.n, L.nbx, L.brick_map, L.dense);
  return s < 0 ? -1 : L.slot_canon[s];
}

__global__ void k_same_table(const int32_t* __restrict__ xyz, int64_t n, gmt::Level L,
                             int* __restrict__ tab) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  for (int t = 0; t < 27; ++t) {
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    tab[i * 27 + t] = site_canon(wrap(x + dx, L.n), wrap(y + dy, L.n), wrap(z + dz, L.n), L);
  }
}

// coarse node q (level l+1) -> fine node at 2q + d_t (level l)
__global__ void k_down_table(const int32_t* __restrict__ xyzc, int64_t nc, gmt::Level F,
                             int* __restrict__ tab) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int x = 2 * xyzc[3 * i], y = 2 * xyzc[3 * i + 1], z = 2 * xyzc[3 * i + 2];
  for (int t = 0; t < 27; ++t) {
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    tab[i * 27 + t] = site_canon(wrap(x + dx, F.n), wrap(y + dy, F.n), wrap(z + dz, F.n), F);
  }
}

// fine node p (level l) -> coarse node q (level l+1) with p = 2q + d_t, or -1
__global__ void k_up_table(const int32_t* __restrict__ xyzf, int64_t nf, int nfine, gmt::Level C,
                           int* __restrict__ tab) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const int x = xyzf[3 * i], y = xyzf[3 * i + 1], z = xyzf[3 * i + 2];
  for (int t = 0; t < 27; ++t) {
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    const int a = wrap(x - dx, nfine), b = wrap(y - dy, nfine), c = wrap(z - dz, nfine);
    tab[i * 27 + t] = ((a | b | c) & 1) ? -1 : site_canon(a >> 1, b >> 1, c >> 1, C);
  }
}

__global__ void k_features(const int* __restrict__ canon_slot, const uint8_t* __restrict__ mask,
                           int64_t n, float* __restrict__ x0) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned m = mask[canon_slot[i]];
#pragma unroll
  for (int o = 0; o < 8; ++o) x0[i * 8 + o] = (float)((m >> o) & 1u);
}

// Rows of an up table grouped by the parity class (x&1) + 2(y&1) + 4(z&1) of the fine node:
// a fine node of class c has a coarse parent under tap t only when every axis with d = 0 is
// even and every axis with d = +-1 is odd, so a block of one class visits 1 to 8 taps.
// Row order within a class is arbitrary (atomic slots): every output row is computed on its
// own, with the same sum order whatever its position.
__global__ void k_class_count(const int32_t* __restrict__ xyz, int64_t n, int* __restrict__ cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  atomicAdd(&cnt[(xyz[3 * i] & 1) + 2 * (xyz[3 * i + 1] & 1) + 4 * (xyz[3 * i + 2] & 1)], 1);
}

__global__ void k_class_offsets(int* __restrict__ cnt) {   // cnt[0..8) -> cursors cnt[8..16)
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int off = 0;
    for (int c = 0; c < 8; ++c) {
      cnt[8 + c] = off;
      off += cnt[c];
    }
  }
}

__global__ void k_class_fill(const int32_t* __restrict__ xyz, const int* __restrict__ tab, int64_t n,
                             int* __restrict__ cursor, int* __restrict__ perm,
                             int* __restrict__ tab_perm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (xyz[3 * i] & 1) + 2 * (xyz[3 * i + 1] & 1) + 4 * (xyz[3 * i + 2] & 1);
  const int pos = atomicAdd(&cursor[c], 1);
  perm[pos] = (int)i;
  for (int t = 0; t < 27; ++t) tab_perm[(int64_t)pos * 27 + t] = tab[i * 27 + t];
}

// ------------------------------------------------------------------ gather convolution
// out[n][co] (=, or += with accum) act(b[co] + add[n][co] + sum_t sum_ci w(t,ci,co) x[s][ci]),
// s = tab[n][flip ? 26 - t : t] (skipped when < 0); w(t,ci,co) = W[t][ci][co], or
// W[t][co][ci] with wtrans (the backward-data form of a layer whose forward weights are
// [27][cout'][cin']). With omap, row r of the table computes output node omap[r] (the up
// layers' rows grouped by parity class, so that a block meets few taps).
// Block: GC_NODES nodes x 32 output channels, 256 threads as 8 channel
// quads x 32 node groups, each thread a 4 x 4 register tile: per staged input channel 4
// shared loads (rows of the gathered inputs) and one 16-byte load (4 weights) feed 16 FMAs.
constexpr int GC_NODES = 128;
// dynamic shared memory: weights [2][32][32], gathered rows [2][GC_NODES][GC_LD], tap flags
// [27] and the active-tap list [28] (the block's tap table rows are read from global memory,
// where they stay in L1, to keep four blocks per SM). Row stride
// 36 floats keeps 16-byte copies aligned; thread row r = j * 32 + ty makes the 4 rows a warp
// reads at once fall in distinct banks.
constexpr int GC_LD = 36;
constexpr int GC_SW = 2 * 32 * 32 * 4;
constexpr int GC_SX = 2 * GC_NODES * GC_LD * 4;
constexpr int GC_SMEM = GC_SW + GC_SX + 27 * 4 + 28 * 4;

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Two-stage pipeline over (active tap, 32-channel input chunk): while one stage's gathered
// rows and weights are multiplied out of shared memory, the next stage's are copied in with
// cp.async (zero-filled where a neighbour is missing or a channel is out of range).
__global__ void __launch_bounds__(256) k_gconv(const float* __restrict__ x, int cin,
                                               const int* __restrict__ tab, int flip,
                                               const float* __restrict__ W, int wtrans,
                                               const float* __restrict__ bias,
                                               const float* __restrict__ add, int relu, int accum,
                                               float* __restrict__ out, int cout, int64_t n_out,
                                               const int* __restrict__ omap) {
  extern __shared__ __align__(16) unsigned char gc_smem[];
  float (*sW)[32][32] = reinterpret_cast<float (*)[32][32]>(gc_smem);
  float (*sX)[GC_NODES][GC_LD] = reinterpret_cast<float (*)[GC_NODES][GC_LD]>(gc_smem + GC_SW);
  int* sAny = reinterpret_cast<int*>(gc_smem + GC_SW + GC_SX);
  int* sTaps = sAny + 27;   // [0]: count, then the active weight taps in order
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 8 + tx;   // blockDim (8, 32)
  const int64_t n0 = (int64_t)blockIdx.x * GC_NODES;
  const int co0 = blockIdx.y * 32;
  const int64_t rows = min((int64_t)GC_NODES, n_out - n0);
  const int* bTab = tab + n0 * 27;   // this block's rows of the table
  if (tid < 27) sAny[tid] = 0;
  __syncthreads();
  for (int e = tid; e < rows * 27; e += 256)
    if (bTab[e] >= 0) sAny[e % 27] = 1;
  __syncthreads();
  if (tid == 0) {
    int k = 0;
    for (int t = 0; t < 27; ++t)
      if (sAny[flip ? 26 - t : t]) sTaps[1 + k++] = t;
    sTaps[0] = k;
  }
  __syncthreads();
  const int nch = (cin + 31) / 32;
  const int S = sTaps[0] * nch;

  auto issue = [&](int k, int buf) {
    const int t = sTaps[1 + k / nch];
    const int tt = flip ? 26 - t : t;
    const int ci0 = (k % nch) * 32;
    if ((cin & 3) == 0) {   // rows of whole 16-byte quads (x is 16-byte aligned)
      for (int e = tid; e < GC_NODES * 8; e += 256) {
        const int r = e >> 3, q = (e & 7) * 4;
        const int src = r < rows ? __ldg(bTab + r * 27 + tt) : -1;
        const bool ok = src >= 0 && ci0 + q < cin;
        cp_async16(&sX[buf][r][q],
                   ok ? (const void*)(x + (int64_t)src * cin + ci0 + q) : (const void*)x, ok);
      }
    } else {
      for (int e = tid; e < GC_NODES * 32; e += 256) {
        const int r = e >> 5, c = e & 31;
        const int src = r < rows ? __ldg(bTab + r * 27 + tt) : -1;
        const bool ok = src >= 0 && ci0 + c < cin;
        cp_async4(&sX[buf][r][c],
                  ok ? (const void*)(x + (int64_t)src * cin + ci0 + c) : (const void*)x, ok);
      }
    }
    for (int e = tid; e < 32 * 32; e += 256) {
      const int r = e >> 5, c = e & 31;   // r: input channel, c: output channel
      const int ci = ci0 + r, co = co0 + c;
      const bool ok = ci < cin && co < cout;
      const float* src = ok ? (wtrans ? W + ((int64_t)t * cout + co) * cin + ci
                                      : W + ((int64_t)t * cin + ci) * cout + co)
                            : W;
      cp_async4(&sW[buf][r][c], src, ok);
    }
    cp_async_commit();
  };

  float acc[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = 0.f;
  if (S > 0) issue(0, 0);
  for (int k = 0; k < S; ++k) {
    const int buf = k & 1;
    if (k + 1 < S) {
      issue(k + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int lim = min(32, cin - (k % nch) * 32);
    for (int kk = 0; kk < lim; ++kk) {
      const float4 w = *reinterpret_cast<const float4*>(&sW[buf][kk][tx * 4]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float xv = sX[buf][j * 32 + ty][kk];
        acc[j][0] = fmaf(xv, w.x, acc[j][0]);
        acc[j][1] = fmaf(xv, w.y, acc[j][1]);
        acc[j][2] = fmaf(xv, w.z, acc[j][2]);
        acc[j][3] = fmaf(xv, w.w, acc[j][3]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t row = n0 + j * 32 + ty;
    if (row >= n_out) break;
    const int64_t node = omap ? (int64_t)omap[row] : row;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int co = co0 + tx * 4 + c;
      if (co >= cout) break;
      const int64_t o = node * cout + co;
      float v = acc[j][c] + (bias ? bias[co] : 0.f) + (add ? add[o] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      out[o] = accum ? out[o] + v : v;
    }
  }
}

// Weight-gradient partials of the forward gather conv: for chunk c of WG_CHUNK output
// nodes, part[c][t][ci][co] = sum_n x[tab[n][t]][ci] dz[n][co] and bpart[c][co] = sum_n
// dz[n][co]. Grid (27, chunks, ci tiles x co tiles), block 32 x 8, each thread 4 ci x 1 co.
__global__ void __launch_bounds__(256) k_wgrad(const float* __restrict__ x, int cin,
                                               const int* __restrict__ tab,
                                               const float* __restrict__ dz, int cout, int64_t n,
                                               float* __restrict__ part, float* __restrict__ bpart) {
  __shared__ float sX[64][33];
  __shared__ float sD[64][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int t = blockIdx.x;
  const int64_t c = blockIdx.y;
  const int tiles_co = (cout + 31) / 32;
  const int ci0 = (blockIdx.z / tiles_co) * 32, co0 = (blockIdx.z % tiles_co) * 32;
  const int64_t beg = c * WG_CHUNK, end = min(n, beg + WG_CHUNK);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float bacc = 0.f;
  for (int64_t j0 = beg; j0 < end; j0 += 64) {
    for (int r = ty; r < 64; r += 8) {
      const int64_t node = j0 + r;
      float xv = 0.f, dv = 0.f;
      if (node < end) {
        const int s = tab[node * 27 + t];
        if (s >= 0 && ci0 + tx < cin) xv = x[(int64_t)s * cin + ci0 + tx];
        if (co0 + tx < cout) dv = dz[node * cout + co0 + tx];
      }
      sX[r][tx] = xv;
      sD[r][tx] = dv;
    }
    __syncthreads();
    for (int r = 0; r < 64; ++r) {
      const float d = sD[r][tx];
      bacc += d;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] = fmaf(sX[r][ty * 4 + k], d, acc[k]);
    }
    __syncthreads();
  }
  const int co = co0 + tx;
  if (co >= cout) return;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int ci = ci0 + ty * 4 + k;
    if (ci < cin) part[((c * 27 + t) * cin + ci) * cout + co] = acc[k];
  }
  if (t == 0 && ci0 == 0 && ty == 0) bpart[c * cout + co] = bacc;
}

// gW[i] = sum_c part[c][i], gb[co] = sum_c bpart[c][co] (fixed order)
__global__ void k_wgrad_reduce(const float* __restrict__ part, const float* __restrict__ bpart,
                               int64_t chunks, int64_t nw, int cout, float* __restrict__ gW,
                               float* __restrict__ gb) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nw) {
    float s = 0.f;
    for (int64_t c = 0; c < chunks; ++c) s += part[c * nw + i];
    gW[i] = s;
  } else if (i < nw + cout) {
    const int co = (int)(i - nw);
    float s = 0.f;
    for (int64_t c = 0; c < chunks; ++c) s += bpart[c * cout + co];
    gb[co] = s;
  }
}

__global__ void k_relu_grad(const float* __restrict__ dy, const float* __restrict__ y, int64_t n,
                            float* __restrict__ dz) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dz[i] = y[i] > 0.f ? dy[i] : 0.f;
}

__global__ void k_add_into(float* __restrict__ g, const float* __restrict__ d, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) g[i] += d[i];
}

// Mean squared error over n values: loss partial per block (double) and the gradient
// g = 2 (pred - u / scale) / n.
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ pred,
                                             const double* __restrict__ u, double inv_scale,
                                             int64_t n, float* __restrict__ g,
                                             double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  const double inv_n = 1.0 / (double)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double e = (double)pred[i] - u[i] * inv_scale;
    s += e * e;
    if (g) g[i] = (float)(2.0 * e * inv_n);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0] * inv_n;
}

__global__ void k_sum_blocks(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];
    *out = s;
  }
}

// per-block partial sums of a . b (double)
__global__ void __launch_bounds__(256) k_dot(const double* __restrict__ a,
                                             const double* __restrict__ b, int64_t n,
                                             double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_err_field(const float* __restrict__ y, const double* __restrict__ u, double scale,
                            int64_t n, double* __restrict__ e) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) e[i] = scale * (double)y[i] - u[i];
}

// energy loss: loss = num / den, gradient g = 2 scale (K e) / den
__global__ void k_energy_grad(const double* __restrict__ ke, const double* __restrict__ numden,
                              double scale, int64_t n, float* __restrict__ g,
                              double* __restrict__ loss) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double den = numden[1];
  if (i < n) g[i] = (float)(2.0 * scale * ke[i] / den);
  if (i == 0) *loss = numden[0] / den;
}

__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                        float wd, float bc1, float bc2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float step = (mi / bc1) / (sqrtf(vi / bc2) + eps);
  p[i] = p[i] - lr * (step + wd * p[i]);
}

__global__ void k_to_field(const float* __restrict__ y, int64_t n, double scale,
                           double* __restrict__ u) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) u[i] = scale * (double)y[i];
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct gmt_unet {
  int device = 0;
  int w[3] = {0, 0, 0};
  int cout = 0;
  LayerDef L[NLAYERS];
  int64_t P = 0;
  int64_t woff[NLAYERS], boff[NLAYERS];
  float* p = nullptr;     // parameters
  float* g = nullptr;     // gradient
  float* m = nullptr;     // AdamW moments
  float* v = nullptr;
  int64_t steps = 0;
  // inference on the tensor cores (gmt_unet_set_tensor_cores): FP16 weight images per layer
  int tc = 0;
  __half* img = nullptr;
  int64_t img_off[NLAYERS];
};

struct gmt_netgraph {
  int device = 0;
  cudaStream_t stream = nullptr;
  int N = 0;
  int64_t n[3] = {0, 0, 0};
  int* same[3] = {nullptr, nullptr, nullptr};
  int* down[2] = {nullptr, nullptr};
  int* up[2] = {nullptr, nullptr};
  int* up_perm[2] = {nullptr, nullptr};   // up tables with rows grouped by parity class
  int* up_rows[2] = {nullptr, nullptr};   // row -> fine node of up_perm
  float* x0 = nullptr;
  gmt::Arena geo;
  // buffers for one network shape
  gmt::Arena buf;
  int key[4] = {0, 0, 0, 0};
  float* a[NACT] = {};
  float* g[NACT] = {};
  __half* h[NACT] = {};   // tensor-core inference: FP16 copies of the activations 0..NACT-2
  float* dz = nullptr;
  float* part = nullptr;
  float* bpart = nullptr;
  double* lpart = nullptr;
  double* loss = nullptr;
  double* e64 = nullptr;     // energy loss: error field and K times it, [n_0][cout]
  double* ke64 = nullptr;
  double* numden = nullptr;  // [e.Ke, u.Ku]
};

namespace {

constexpr int LOSS_BLOCKS = 296;

void ensure_buffers(gmt_netgraph* G, const gmt_unet* net) {
  if (G->key[0] == net->w[0] && G->key[1] == net->w[1] && G->key[2] == net->w[2] &&
      G->key[3] == net->cout)
    return;
  G->buf.release();
  G->buf.bind(G->stream);
  for (int a = 0; a < NACT; ++a) G->h[a] = nullptr;
  int64_t maxe = 0, maxpart = 0, maxb = 0;
  for (int a = 1; a < NACT; ++a) {
    const int64_t e = G->n[act_level(net->L, a)] * act_ch(net->L, a);
    G->a[a] = G->buf.alloc<float>(e);
    G->g[a] = G->buf.alloc<float>(e);
    maxe = std::max(maxe, e);
  }
  G->a[0] = G->x0;
  G->g[0] = nullptr;
  for (int i = 0; i < NLAYERS; ++i) {
    const LayerDef& d = net->L[i];
    const int64_t chunks = (G->n[d.lvl_out] + WG_CHUNK - 1) / WG_CHUNK;
    maxpart = std::max(maxpart, chunks * 27 * d.cin * d.cout);
    maxb = std::max(maxb, chunks * d.cout);
  }
  G->dz = G->buf.alloc<float>(maxe);
  G->part = G->buf.alloc<float>(maxpart);
  G->bpart = G->buf.alloc<float>(maxb);
  G->lpart = G->buf.alloc<double>(LOSS_BLOCKS);
  G->loss = G->buf.alloc<double>(1);
  G->e64 = G->buf.alloc<double>(G->n[0] * net->cout);
  G->ke64 = G->buf.alloc<double>(G->n[0] * net->cout);
  G->numden = G->buf.alloc<double>(2);
  G->key[0] = net->w[0];
  G->key[1] = net->w[1];
  G->key[2] = net->w[2];
  G->key[3] = net->cout;
}

// the table a layer gathers its input through, and the one its backward-data pass uses
const int* fwd_table(const gmt_netgraph* G, const LayerDef& d) {
  if (d.kind == SAME) return G->same[d.lvl_out];
  if (d.kind == DOWN) return G->down[d.lvl_out - 1];
  return G->up[d.lvl_out];
}
const int* bwd_table(const gmt_netgraph* G, const LayerDef& d) {
  if (d.kind == SAME) return G->same[d.lvl_out];
  if (d.kind == DOWN) return G->up[d.lvl_out - 1];
  return G->down[d.lvl_out];
}

void launch_gconv(cudaStream_t s, const float* x, int cin, const int* tab, int flip,
                  const float* W, int wtrans, const float* b, const float* add, int relu,
                  int accum, float* out, int cout, int64_t n_out, const int* omap = nullptr) {
  if (n_out <= 0) return;
  dim3 grid((unsigned)((n_out + GC_NODES - 1) / GC_NODES), (unsigned)((cout + 31) / 32));
  gmt::ensure_smem_attr((const void*)k_gconv, GC_SMEM);
  k_gconv<<<grid, dim3(8, 32), GC_SMEM, s>>>(x, cin, tab, flip, W, wtrans, b, add, relu, accum,
                                             out, cout, n_out, omap);
  GMT_LAUNCH_CHECK();
}

// tc: the layers run as tensor-core convolutions (FP16 operands, FP32 accumulation) from
// FP16 images of the current weights; training keeps the FP32 kernels (tc = false)
void forward(gmt_unet* net, gmt_netgraph* G, bool tc = false) {
  ensure_buffers(G, net);
  if (tc && net->img == nullptr) {
    int64_t off = 0;
    for (int i = 0; i < NLAYERS; ++i) {
      net->img_off[i] = off;
      off += gmt::tc_image_halves(net->L[i].cin, net->L[i].cout);
    }
    GMT_CUDA(cudaMalloc(&net->img, sizeof(__half) * (size_t)off));
  }
  bool all_tc = tc;
  for (int i = 0; i < NLAYERS; ++i) all_tc = all_tc && gmt::tc_supported(net->L[i].cin, net->L[i].cout);
  if (all_tc) {
    // every layer on the tensor cores: the activations stay in FP16 between layers (the
    // gathers move half the bytes); the last layer writes FP32
    if (G->h[0] == nullptr)
      for (int a = 0; a + 1 < NACT; ++a)
        G->h[a] = G->buf.alloc<__half>(G->n[act_level(net->L, a)] * act_ch(net->L, a));
    gmt::tc_to_half(G->stream, G->a[0], G->n[0] * IN_CH, G->h[0]);
  }
  for (int i = 0; i < NLAYERS; ++i) {
    const LayerDef& d = net->L[i];
    const bool up = d.kind == UP;
    const int* tab = up ? G->up_perm[d.lvl_out] : fwd_table(G, d);
    const int* omap = up ? G->up_rows[d.lvl_out] : nullptr;
    const float* add = d.skip >= 0 ? G->a[d.skip] : nullptr;
    if (all_tc) {
      gmt::tc_build_image(G->stream, net->p + net->woff[i], d.cin, d.cout,
                          net->img + net->img_off[i]);
      const bool last = i + 1 == NLAYERS;
      gmt::launch_gconv_tc(G->stream, G->h[d.in], d.cin, tab, net->img + net->img_off[i],
                           net->p + net->boff[i], d.skip >= 0 ? G->h[d.skip] : nullptr, d.relu,
                           last ? G->a[i + 1] : nullptr, last ? nullptr : G->h[i + 1], d.cout,
                           G->n[d.lvl_out], omap);
    } else {
      launch_gconv(G->stream, G->a[d.in], d.cin, tab, 0, net->p + net->woff[i], 0,
                   net->p + net->boff[i], add, d.relu, 0, G->a[i + 1], d.cout, G->n[d.lvl_out],
                   omap);
    }
  }
}

void dot_into(cudaStream_t s, const double* a, const double* b, int64_t n, double* part,
              double* out) {
  k_dot<<<LOSS_BLOCKS, 256, 0, s>>>(a, b, n, part);
  GMT_LAUNCH_CHECK();
  k_sum_blocks<<<1, 32, 0, s>>>(part, LOSS_BLOCKS, out);
  GMT_LAUNCH_CHECK();
}

// loss and gradient into net->g (forward must have run); h: the prepared hierarchy of the
// graph for the energy loss
void backward(gmt_unet* net, gmt_netgraph* G, gmt_hierarchy* h, int loss_kind, const double* u,
              double scale) {
  cudaStream_t s = G->stream;
  const int64_t n_out = G->n[0] * net->cout;
  for (int a = 1; a < NACT; ++a)
    GMT_CUDA(cudaMemsetAsync(G->g[a], 0,
                             sizeof(float) * G->n[act_level(net->L, a)] * act_ch(net->L, a), s));
  if (loss_kind == GMT_UNET_LOSS_MSE) {
    k_mse<<<LOSS_BLOCKS, 256, 0, s>>>(G->a[NACT - 1], u, 1.0 / scale, n_out, G->g[NACT - 1],
                                      G->lpart);
    GMT_LAUNCH_CHECK();
    k_sum_blocks<<<1, 32, 0, s>>>(G->lpart, LOSS_BLOCKS, G->loss);
    GMT_LAUNCH_CHECK();
  } else {
    gmt::step_apply(h, 0, GMT_PREC_FP32, u, G->ke64);
    dot_into(s, u, G->ke64, n_out, G->lpart, G->numden + 1);
    k_err_field<<<blocks(n_out), 256, 0, s>>>(G->a[NACT - 1], u, scale, n_out, G->e64);
    GMT_LAUNCH_CHECK();
    gmt::step_apply(h, 0, GMT_PREC_FP32, G->e64, G->ke64);
    dot_into(s, G->e64, G->ke64, n_out, G->lpart, G->numden);
    k_energy_grad<<<blocks(n_out), 256, 0, s>>>(G->ke64, G->numden, scale, n_out,
                                                G->g[NACT - 1], G->loss);
    GMT_LAUNCH_CHECK();
  }
  for (int i = NLAYERS - 1; i >= 0; --i) {
    const LayerDef& d = net->L[i];
    const int64_t no = G->n[d.lvl_out];
    const int64_t e = no * d.cout;
    const float* dz = G->g[i + 1];
    if (d.relu) {
      k_relu_grad<<<blocks(e), 256, 0, s>>>(G->g[i + 1], G->a[i + 1], e, G->dz);
      GMT_LAUNCH_CHECK();
      dz = G->dz;
    }
    if (d.skip >= 0) {
      k_add_into<<<blocks(e), 256, 0, s>>>(G->g[d.skip], dz, e);
      GMT_LAUNCH_CHECK();
    }
    const int64_t chunks = (no + WG_CHUNK - 1) / WG_CHUNK;
    if (chunks > 0) {
      const int tiles = ((d.cin + 31) / 32) * ((d.cout + 31) / 32);
      k_wgrad<<<dim3(27, (unsigned)chunks, tiles), dim3(32, 8), 0, s>>>(
          G->a[d.in], d.cin, fwd_table(G, d), dz, d.cout, no, G->part, G->bpart);
      GMT_LAUNCH_CHECK();
      const int64_t nw = 27LL * d.cin * d.cout;
      k_wgrad_reduce<<<blocks(nw + d.cout), 256, 0, s>>>(G->part, G->bpart, chunks, nw, d.cout,
                                                          net->g + net->woff[i],
                                                          net->g + net->boff[i]);
      GMT_LAUNCH_CHECK();
    } else {
      GMT_CUDA(cudaMemsetAsync(net->g + net->woff[i], 0,
                               sizeof(float) * (27LL * d.cin * d.cout + d.cout), s));
    }
    if (d.in > 0)
      launch_gconv(s, dz, d.cout, bwd_table(G, d), d.kind == SAME, net->p + net->woff[i], 1,
                   nullptr, nullptr, 0, 1, G->g[d.in], d.cin, G->n[act_level(net->L, d.in)]);
  }
}

void check_pair(const gmt_unet* net, const gmt_netgraph* G) {
  GMT_REQUIRE(net && G, GMT_ERR_ARG, "null network or graph");
  GMT_REQUIRE(net->device == G->device, GMT_ERR_ARG, "network and graph on different devices");
  GMT_CUDA(cudaSetDevice(G->device));
}

void check_loss(const gmt_unet* net, const gmt_netgraph* G, const gmt_hierarchy* h, int kind) {
  GMT_REQUIRE(kind == GMT_UNET_LOSS_MSE || kind == GMT_UNET_LOSS_ENERGY, GMT_ERR_ARG,
              "unknown loss %d", kind);
  if (kind == GMT_UNET_LOSS_MSE) return;
  GMT_REQUIRE(h, GMT_ERR_ARG, "the energy loss needs the graph's hierarchy");
  GMT_REQUIRE(h->prepared, GMT_ERR_STATE, "the energy loss needs a prepared material");
  GMT_REQUIRE(h->N == G->N && h->lv[0].n_nodes == G->n[0] && h->stream == G->stream,
              GMT_ERR_ARG, "hierarchy does not match the graph (size or stream)");
  GMT_REQUIRE(h->mat.C == net->cout, GMT_ERR_ARG,
              "network outputs %d channels, the prepared material has %d values per node",
              net->cout, h->mat.C);
  GMT_REQUIRE(!h->lv[0].dense, GMT_ERR_ARG, "level 0 is dense");
}

}  // namespace

#define UNET_BEGIN \
  gmt::ApiGuard gmt_api_guard; \
  gmt::set_error("%s", ""); \
  try {
#define UNET_END                                   \
  }                                                \
  catch (const gmt::Fail& f) {                     \
    return f.status;                               \
  }                                                \
  catch (...) {                                    \
    gmt::set_error("unexpected host exception");   \
    return GMT_ERR_ARG;                            \
  }

extern "C" {

int64_t gmt_unet_param_count(int out_channels, const int* widths) {
  if (!widths || out_channels <= 0 || widths[0] <= 0 || widths[1] <= 0 || widths[2] <= 0) return -1;
  LayerDef L[NLAYERS];
  layer_defs(widths, out_channels, L);
  return param_count(L);
}

gmt_status gmt_unet_layers(int out_channels, const int* widths, int32_t* layers_out) {
  UNET_BEGIN
  GMT_REQUIRE(gmt_unet_param_count(out_channels, widths) > 0 && layers_out, GMT_ERR_ARG,
              "bad network shape");
  LayerDef L[NLAYERS];
  layer_defs(widths, out_channels, L);
  for (int i = 0; i < NLAYERS; ++i) {
    int32_t* r = layers_out + 6 * i;
    r[0] = L[i].kind;
    r[1] = L[i].lvl_out;
    r[2] = L[i].in;
    r[3] = L[i].skip;
    r[4] = L[i].cin;
    r[5] = L[i].cout;
  }
  return GMT_OK;
  UNET_END
}

gmt_status gmt_unet_create(int out_channels, const int* widths, const float* params,
                           gmt_unet** out) {
  UNET_BEGIN
  GMT_REQUIRE(out && params, GMT_ERR_ARG, "null argument");
  GMT_REQUIRE(gmt_unet_param_count(out_channels, widths) > 0, GMT_ERR_ARG, "bad network shape");
  *out = nullptr;
  std::unique_ptr<gmt_unet> net(new gmt_unet());
  GMT_CUDA(cudaGetDevice(&net->device));
  for (int i = 0; i < 3; ++i) net->w[i] = widths[i];
  net->cout = out_channels;
  layer_defs(widths, out_channels, net->L);
  int64_t off = 0;
  for (int i = 0; i < NLAYERS; ++i) {
    net->woff[i] = off;
    off += 27LL * net->L[i].cin * net->L[i].cout;
    net->boff[i] = off;
    off += net->L[i].cout;
  }
  net->P = off;
  const size_t bytes = sizeof(float) * (size_t)off;
  struct Guard {
    gmt_unet* n;
    ~Guard() {
      if (n) {
        cudaFree(n->p);
        cudaFree(n->g);
        cudaFree(n->m);
        cudaFree(n->v);
      }
    }
  } guard{net.get()};
  GMT_CUDA(cudaMalloc(&net->p, bytes));
  GMT_CUDA(cudaMalloc(&net->g, bytes));
  GMT_CUDA(cudaMalloc(&net->m, bytes));
  GMT_CUDA(cudaMalloc(&net->v, bytes));
  GMT_CUDA(cudaMemcpy(net->p, params, bytes, cudaMemcpyDefault));
  GMT_CUDA(cudaMemset(net->g, 0, bytes));
  GMT_CUDA(cudaMemset(net->m, 0, bytes));
  GMT_CUDA(cudaMemset(net->v, 0, bytes));
  guard.n = nullptr;
  *out = net.release();
  return GMT_OK;
  UNET_END
}

void gmt_unet_free(gmt_unet* net) {
  if (!net) return;
  cudaSetDevice(net->device);
  cudaDeviceSynchronize();
  cudaFree(net->p);
  cudaFree(net->g);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->img);
  delete net;
}

gmt_status gmt_unet_set_tensor_cores(gmt_unet* net, int on) {
  UNET_BEGIN
  GMT_REQUIRE(net, GMT_ERR_ARG, "null network");
  net->tc = on != 0;
  return GMT_OK;
  UNET_END
}

int64_t gmt_unet_num_params(const gmt_unet* net) { return net ? net->P : -1; }

gmt_status gmt_unet_get_params(const gmt_unet* net, float* dst) {
  UNET_BEGIN
  GMT_REQUIRE(net && dst, GMT_ERR_ARG, "null argument");
  GMT_CUDA(cudaSetDevice(net->device));
  GMT_CUDA(cudaDeviceSynchronize());
  GMT_CUDA(cudaMemcpy(dst, net->p, sizeof(float) * net->P, cudaMemcpyDefault));
  return GMT_OK;
  UNET_END
}

gmt_status gmt_unet_set_params(gmt_unet* net, const float* src) {
  UNET_BEGIN
  GMT_REQUIRE(net && src, GMT_ERR_ARG, "null argument");
  GMT_CUDA(cudaSetDevice(net->device));
  GMT_CUDA(cudaDeviceSynchronize());
  GMT_CUDA(cudaMemcpy(net->p, src, sizeof(float) * net->P, cudaMemcpyDefault));
  GMT_CUDA(cudaMemset(net->m, 0, sizeof(float) * net->P));
  GMT_CUDA(cudaMemset(net->v, 0, sizeof(float) * net->P));
  net->steps = 0;
  return GMT_OK;
  UNET_END
}

gmt_status gmt_netgraph_build(gmt_hierarchy* h, gmt_netgraph** out) {
  UNET_BEGIN
  GMT_REQUIRE(h && out, GMT_ERR_ARG, "null argument");
  GMT_REQUIRE(h->L >= 3, GMT_ERR_RES, "the network needs a hierarchy of at least 3 levels (has %d)",
              h->L);
  *out = nullptr;
  GMT_CUDA(cudaSetDevice(h->device));
  std::unique_ptr<gmt_netgraph> G(new gmt_netgraph());
  G->device = h->device;
  G->stream = h->stream;
  G->geo.bind(h->stream);
  G->N = h->N;
  cudaStream_t s = h->stream;
  int32_t* xyz[3];
  for (int l = 0; l < 3; ++l) {
    G->n[l] = h->lv[l].n_nodes;
    xyz[l] = G->geo.alloc<int32_t>(3 * std::max<int64_t>(G->n[l], 1));
    gmt::export_nodes(h, l, xyz[l], nullptr);
    G->same[l] = G->geo.alloc<int>(27 * std::max<int64_t>(G->n[l], 1));
    k_same_table<<<blocks(G->n[l]), 256, 0, s>>>(xyz[l], G->n[l], h->lv[l], G->same[l]);
    GMT_LAUNCH_CHECK();
  }
  for (int l = 0; l < 2; ++l) {
    G->down[l] = G->geo.alloc<int>(27 * std::max<int64_t>(G->n[l + 1], 1));
    k_down_table<<<blocks(G->n[l + 1]), 256, 0, s>>>(xyz[l + 1], G->n[l + 1], h->lv[l],
                                                     G->down[l]);
    GMT_LAUNCH_CHECK();
    G->up[l] = G->geo.alloc<int>(27 * std::max<int64_t>(G->n[l], 1));
    k_up_table<<<blocks(G->n[l]), 256, 0, s>>>(xyz[l], G->n[l], h->lv[l].n, h->lv[l + 1], G->up[l]);
    GMT_LAUNCH_CHECK();
    G->up_perm[l] = G->geo.alloc<int>(27 * std::max<int64_t>(G->n[l], 1));
    G->up_rows[l] = G->geo.alloc<int>(std::max<int64_t>(G->n[l], 1));
    int* cnt = G->geo.alloc<int>(16);
    GMT_CUDA(cudaMemsetAsync(cnt, 0, 16 * sizeof(int), s));
    k_class_count<<<blocks(G->n[l]), 256, 0, s>>>(xyz[l], G->n[l], cnt);
    GMT_LAUNCH_CHECK();
    k_class_offsets<<<1, 32, 0, s>>>(cnt);
    GMT_LAUNCH_CHECK();
    k_class_fill<<<blocks(G->n[l]), 256, 0, s>>>(xyz[l], G->up[l], G->n[l], cnt + 8, G->up_rows[l],
                                                 G->up_perm[l]);
    GMT_LAUNCH_CHECK();
  }
  G->x0 = G->geo.alloc<float>(8 * std::max<int64_t>(G->n[0], 1));
  k_features<<<blocks(G->n[0]), 256, 0, s>>>(h->lv[0].canon_slot, h->lv[0].mask, G->n[0], G->x0);
  GMT_LAUNCH_CHECK();
  GMT_CUDA(cudaStreamSynchronize(s));
  *out = G.release();
  return GMT_OK;
  UNET_END
}

void gmt_netgraph_free(gmt_netgraph* G) {
  if (!G) return;
  cudaSetDevice(G->device);
  delete G;  // the arenas wait for the graph's stream before returning their blocks
}

int64_t gmt_netgraph_nodes(const gmt_netgraph* G, int level) {
  return (G && level >= 0 && level < 3) ? G->n[level] : -1;
}

gmt_status gmt_netgraph_tables(const gmt_netgraph* G, int level, int32_t* same_out,
                               int32_t* down_out, int32_t* up_out) {
  UNET_BEGIN
  GMT_REQUIRE(G && level >= 0 && level < 3, GMT_ERR_ARG, "bad graph level");
  GMT_CUDA(cudaSetDevice(G->device));
  GMT_CUDA(cudaStreamSynchronize(G->stream));
  if (same_out)
    GMT_CUDA(cudaMemcpy(same_out, G->same[level], sizeof(int) * 27 * G->n[level], cudaMemcpyDefault));
  if (down_out && level < 2)
    GMT_CUDA(cudaMemcpy(down_out, G->down[level], sizeof(int) * 27 * G->n[level + 1],
                        cudaMemcpyDefault));
  if (up_out && level < 2)
    GMT_CUDA(cudaMemcpy(up_out, G->up[level], sizeof(int) * 27 * G->n[level], cudaMemcpyDefault));
  return GMT_OK;
  UNET_END
}

gmt_status gmt_unet_forward(gmt_unet* net, gmt_netgraph* G, double scale, double* u_out) {
  UNET_BEGIN
  check_pair(net, G);
  GMT_REQUIRE(u_out && scale > 0 && std::isfinite(scale), GMT_ERR_ARG, "bad output or scale");
  forward(net, G, net->tc != 0);
  const int64_t e = G->n[0] * net->cout;
  k_to_field<<<blocks(e), 256, 0, G->stream>>>(G->a[NACT - 1], e, scale, u_out);
  GMT_LAUNCH_CHECK();
  GMT_CUDA(cudaStreamSynchronize(G->stream));
  if (net->tc)
    GMT_REQUIRE(gmt::tc_take_status(G->stream) == 0, GMT_ERR_CUDA,
                "tensor-core convolution: a bounded wait for the MMAs ran out");
  return GMT_OK;
  UNET_END
}

gmt_status gmt_unet_gradient(gmt_unet* net, gmt_netgraph* G, gmt_hierarchy* h, int loss_kind,
                             const double* u_target, double scale, float* grad_out,
                             double* loss_out) {
  UNET_BEGIN
  check_pair(net, G);
  check_loss(net, G, h, loss_kind);
  GMT_REQUIRE(u_target && scale > 0 && std::isfinite(scale), GMT_ERR_ARG, "bad target or scale");
  forward(net, G);
  backward(net, G, h, loss_kind, u_target, scale);
  if (grad_out)
    GMT_CUDA(cudaMemcpyAsync(grad_out, net->g, sizeof(float) * net->P, cudaMemcpyDefault,
                             G->stream));
  if (loss_out)
    GMT_CUDA(cudaMemcpyAsync(loss_out, G->loss, sizeof(double), cudaMemcpyDefault, G->stream));
  GMT_CUDA(cudaStreamSynchronize(G->stream));
  return GMT_OK;
  UNET_END
}

gmt_status gmt_unet_train_step(gmt_unet* net, gmt_netgraph* G, gmt_hierarchy* h, int loss_kind,
                               const double* u_target, double scale, const gmt_adamw* hp,
                               double* loss_out) {
  UNET_BEGIN
  check_pair(net, G);
  check_loss(net, G, h, loss_kind);
  GMT_REQUIRE(u_target && hp && scale > 0 && std::isfinite(scale), GMT_ERR_ARG,
              "bad target, scale or hyper-parameters");
  GMT_REQUIRE(hp->lr > 0 && hp->beta1 >= 0 && hp->beta1 < 1 && hp->beta2 >= 0 && hp->beta2 < 1 &&
                  hp->eps > 0 && hp->weight_decay >= 0,
              GMT_ERR_ARG, "bad AdamW hyper-parameters");
  forward(net, G);
  backward(net, G, h, loss_kind, u_target, scale);
  net->steps += 1;
  const float bc1 = (float)(1.0 - std::pow((double)hp->beta1, (double)net->steps));
  const float bc2 = (float)(1.0 - std::pow((double)hp->beta2, (double)net->steps));
  k_adamw<<<blocks(net->P), 256, 0, G->stream>>>(net->p, net->g, net->m, net->v, net->P,
                                                 (float)hp->lr, (float)hp->beta1,
                                                 (float)hp->beta2, (float)hp->eps,
                                                 (float)hp->weight_decay, bc1, bc2);
  GMT_LAUNCH_CHECK();
  if (loss_out) {
    GMT_CUDA(cudaMemcpyAsync(loss_out, G->loss, sizeof(double), cudaMemcpyDefault, G->stream));
    GMT_CUDA(cudaStreamSynchronize(G->stream));
  }
  return GMT_OK;
  UNET_END
}

}  // extern "C"
