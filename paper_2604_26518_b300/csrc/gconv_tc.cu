// Tensor-core (tcgen05) forward gather convolution of the learned initializer; the layout,
// pipeline and descriptors are described in gconv_tc.cuh.
#include "common.cuh"
#include "gconv_tc.cuh"

namespace gmt {

namespace {

__device__ int g_tc_status = 0;   // 0, or 1 once a bounded wait ran out

// about one second at the B300's 2.03 GHz SM clock
constexpr long long kTcWaitBudget = 2000000000LL;

// FP16 weight image of one layer: stage (t, c) is the B tile of input channels c*32..c*32+31
// of tap t, W[t][ci][co] at byte tc_offset_b(co, ci - 32 c, npad) of npad * 64 bytes (zero
// where ci >= cin or co >= cout)
__global__ void k_tc_image(const float* __restrict__ W, int cin, int cout, int nch, int npad,
                           __half* __restrict__ img) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int per = npad * TC_KC;   // FP16 values per stage
  if (i >= 27LL * nch * per) return;
  const int64_t stage = i / per;
  const int b = (int)(i % per) * 2;   // byte within the tile
  const int t = (int)(stage / nch), c = (int)(stage % nch);
  const int kk = b / (npad * 32), rem = b % (npad * 32);
  const int g = rem / 256, kc = (rem % 256) / 128, r = (rem % 128) / 16, e = (rem % 16) / 2;
  const int co = g * 8 + r, ci = c * TC_KC + kk * 16 + kc * 8 + e;
  const float w = (co < cout && ci < cin) ? W[((int64_t)t * cin + ci) * cout + co] : 0.f;
  img[i] = __float2half_rn(w);
}

__global__ void k_to_half(const float* __restrict__ x, int64_t n, __half* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2half_rn(x[i]);
}

// shared memory: A tiles [2][8 KB], B tiles [2][npad * 64 bytes], the CTA's table rows
// [27][128], mbarriers, TMEM slot, tap flags and list
__host__ __device__ constexpr int tc_off_src(int npad) { return 2 * TC_TILE + 2 * npad * 64; }
__host__ __device__ constexpr int tc_off_bar(int npad) { return tc_off_src(npad) + 27 * TC_ROWS * 4; }
__host__ __device__ constexpr int tc_smem_used(int npad) { return tc_off_bar(npad) + 32 + 55 * 4; }
// dynamic shared memory per CTA, chosen so that the CTAs an SM can hold never ask for more
// than its 512 TMEM columns: N = 128 (128 columns) -> 47 KB, at most 4 CTAs (each CTA also
// holds 1 KB of reserved shared memory); N <= 64 -> what the tiles need, at most 38 KB (the
// registers allow 6 CTAs: 6 x 64 columns fit)
constexpr int TC_SMEM_MAX = 47 * 1024;
__host__ __device__ constexpr int tc_smem_bytes(int npad) {
  return npad > 64 ? TC_SMEM_MAX : (tc_smem_used(npad) + 1023) / 1024 * 1024;
}
static_assert(tc_smem_used(128) <= TC_SMEM_MAX && 5 * (TC_SMEM_MAX + 1024) > 228 * 1024,
              "at most four 128-column CTAs per SM");
static_assert(8 * 64 <= 512, "any number of 64-column CTAs the registers allow fits");
constexpr int TC_BQ = TC_TILE / 16 / TC_ROWS;   // 16-byte B chunks per thread at npad = 128

// x: FP16 input activations [rows of the input level][cin]; out32 / out16: the output
// activations in FP32 (the last layer) or FP16 (one of them is null); add: FP16 skip input
__global__ void __launch_bounds__(128) k_gconv_tc(const __half* __restrict__ x, int cin,
                                                  const int* __restrict__ tab,
                                                  const __half* __restrict__ img,
                                                  const float* __restrict__ bias,
                                                  const __half* __restrict__ add, int relu,
                                                  float* __restrict__ out32,
                                                  __half* __restrict__ out16, int cout,
                                                  int npad, int64_t n_out,
                                                  const int* __restrict__ omap) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  const int btile = npad * 64;                    // bytes of one B tile
  unsigned char* sA = tc_smem;
  unsigned char* sB = tc_smem + 2 * TC_TILE;
  int* sSrc = reinterpret_cast<int*>(tc_smem + tc_off_src(npad));           // [27][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(tc_smem + tc_off_bar(npad)); // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + tc_off_bar(npad) + 16);
  int* sAny = reinterpret_cast<int*>(tc_smem + tc_off_bar(npad) + 32);      // [27]
  int* sTaps = sAny + 27;                                                 // [28]
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t n0 = (int64_t)blockIdx.x * TC_ROWS;
  const int64_t rows = min((int64_t)TC_ROWS, n_out - n0);
  const int64_t row = n0 + tid;
  const uint32_t ncols = (uint32_t)tc_cols(npad);
  if (warp == 0) tc_alloc(smem_u32(tslot), ncols);
  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 27) sAny[tid] = 0;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // this row's neighbours under every tap (kept in shared memory), and the taps that any
  // of the CTA's rows uses
  {
    int v[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) v[t] = tid < rows ? __ldg(tab + row * 27 + t) : -1;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      sSrc[t * TC_ROWS + tid] = v[t];
      if (v[t] >= 0) sAny[t] = 1;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int k = 0;
    for (int t = 0; t < 27; ++t)
      if (sAny[t]) sTaps[1 + k++] = t;
    sTaps[0] = k;
  }
  __syncthreads();
  const int nch = (cin + TC_KC - 1) / TC_KC;
  const int S = sTaps[0] * nch;
  const int nq = npad * 4;   // 16-byte chunks of a B tile
  const uint32_t idesc = tc_idesc(TC_ROWS, npad);
  // stage k's operands, loaded into registers one stage ahead
  uint4 an[TC_KC / 8];
  uint4 bn[TC_BQ];
  auto prefetch = [&](int k) {
    const int t = sTaps[1 + k / nch];
    const int ci0 = (k % nch) * TC_KC;
    const int src = sSrc[t * TC_ROWS + tid];
#pragma unroll
    for (int q = 0; q < TC_KC / 8; ++q) {
      const int ch = ci0 + 8 * q;
      an[q] = (src >= 0 && ch < cin)
                  ? __ldg(reinterpret_cast<const uint4*>(x + (int64_t)src * cin + ch))
                  : make_uint4(0u, 0u, 0u, 0u);
    }
    const uint4* bsrc =
        reinterpret_cast<const uint4*>(img + ((int64_t)t * nch + k % nch) * (npad * TC_KC));
#pragma unroll
    for (int j = 0; j < TC_BQ; ++j) {
      const int i = tid + j * TC_ROWS;
      bn[j] = i < nq ? __ldg(bsrc + i) : make_uint4(0u, 0u, 0u, 0u);
    }
  };
  if (S > 0) prefetch(0);
  bool failed = false;
  int issued = 0;
  for (int k = 0; k < S; ++k) {
    const int buf = k & 1;
    uint4 ac[TC_KC / 8];
    uint4 bc[TC_BQ];
#pragma unroll
    for (int q = 0; q < TC_KC / 8; ++q) ac[q] = an[q];
#pragma unroll
    for (int j = 0; j < TC_BQ; ++j) bc[j] = bn[j];
    if (k + 1 < S) prefetch(k + 1);   // in flight while this stage is written and issued
    bool bad = false;
    if (k >= 2) bad = !mbar_wait(smem_u32(&bars[buf]), ((k - 2) >> 1) & 1, kTcWaitBudget);
    if (__syncthreads_or(bad)) {
      failed = true;
      break;
    }
    unsigned char* a = sA + buf * TC_TILE;
#pragma unroll
    for (int q = 0; q < TC_KC / 8; ++q) *reinterpret_cast<uint4*>(a + tc_offset(tid, 8 * q)) = ac[q];
    uint4* bdst = reinterpret_cast<uint4*>(sB + buf * btile);
#pragma unroll
    for (int j = 0; j < TC_BQ; ++j) {
      const int i = tid + j * TC_ROWS;
      if (i < nq) bdst[i] = bc[j];
    }
    tc_fence_proxy_async();   // the generic-proxy stores become visible to the tensor core
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(a), b0 = smem_u32(sB + buf * btile);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
        tc_mma(tmem, tc_smem_desc(a0 + kk * 4096, 128, 256),
               tc_smem_desc(b0 + kk * npad * 32, 128, 256), idesc, (k > 0 || kk > 0) ? 1u : 0u);
      tc_commit(smem_u32(&bars[buf]));
    }
    issued = k + 1;
  }
  if (!failed && S > 0) {
    const bool bad = !mbar_wait(smem_u32(&bars[(S - 1) & 1]), ((S - 1) >> 1) & 1, kTcWaitBudget);
    if (__syncthreads_or(bad)) failed = true;
  }
  if (failed) {
    if (tid == 0) atomicCAS(&g_tc_status, 0, 1);
    // MMAs may still be in flight: wait (bounded again) for the last committed stage
    if (issued > 0)
      (void)mbar_wait(smem_u32(&bars[(issued - 1) & 1]), ((issued - 1) >> 1) & 1, kTcWaitBudget);
    __syncthreads();
  }
  tc_fence_after();
  if (!failed) {
    const int64_t node = (tid < rows) ? (omap ? (int64_t)omap[row] : row) : 0;
    for (int c0 = 0; c0 < npad; c0 += 16) {
      float v[16];
      if (S > 0) {
        tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (tid < rows) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int co = c0 + i;
          if (co < cout) {
            const int64_t o = node * cout + co;
            float r = v[i] + (bias ? bias[co] : 0.f) + (add ? __half2float(add[o]) : 0.f);
            if (relu) r = fmaxf(r, 0.f);
            if (out32) out32[o] = r;
            else out16[o] = __float2half_rn(r);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, ncols);
}

}  // namespace

bool tc_supported(int cin, int cout) { return cin > 0 && cin % 8 == 0 && cout > 0 && cout <= 128; }

int64_t tc_image_halves(int cin, int cout) {
  return 27LL * ((cin + TC_KC - 1) / TC_KC) * tc_npad(cout) * TC_KC;
}

void tc_build_image(cudaStream_t s, const float* W, int cin, int cout, __half* img) {
  const int nch = (cin + TC_KC - 1) / TC_KC;
  const int64_t n = tc_image_halves(cin, cout);
  k_tc_image<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(W, cin, cout, nch, tc_npad(cout), img);
  GMT_LAUNCH_CHECK();
}

void tc_to_half(cudaStream_t s, const float* x, int64_t n, __half* y) {
  if (n <= 0) return;
  k_to_half<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, y);
  GMT_LAUNCH_CHECK();
}

void launch_gconv_tc(cudaStream_t s, const __half* x, int cin, const int* tab, const __half* img,
                     const float* bias, const __half* add, int relu, float* out32,
                     __half* out16, int cout, int64_t n_out, const int* omap) {
  GMT_REQUIRE((out32 == nullptr) != (out16 == nullptr), GMT_ERR_ARG,
              "tensor-core convolution: exactly one output");
  GMT_REQUIRE(tc_supported(cin, cout), GMT_ERR_ARG, "tensor-core convolution: %d -> %d channels",
              cin, cout);
  if (n_out <= 0) return;
  ensure_smem_attr((const void*)k_gconv_tc, TC_SMEM_MAX);
  const int npad = tc_npad(cout);
  const unsigned grid = (unsigned)((n_out + TC_ROWS - 1) / TC_ROWS);
  k_gconv_tc<<<grid, TC_ROWS, tc_smem_bytes(npad), s>>>(x, cin, tab, img, bias, add, relu, out32,
                                                        out16, cout, npad, n_out, omap);
  GMT_LAUNCH_CHECK();
}

int tc_take_status(cudaStream_t s) {
  int st = 0;
  GMT_CUDA(cudaMemcpyFromSymbolAsync(&st, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  GMT_CUDA(cudaStreamSynchronize(s));
  if (st) {
    const int zero = 0;
    GMT_CUDA(cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    GMT_CUDA(cudaStreamSynchronize(s));
  }
  return st;
}

}  // namespace gmt
