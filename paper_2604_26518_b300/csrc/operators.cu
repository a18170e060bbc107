// Material-dependent operators, all built by kernels:
//   * the hex8 element matrix K_e, the affine modes x0, the element load K_e x0 and the
//     base tensor x0^T K_e x0 (App. F.1 / F.2; 2x2x2 Gauss-Legendre, exact here);
//   * element-local Galerkin coarse matrices (Sec. 4.6 "Operator Consistency via Galerkin
//     Projection": K_c = R_loc K_patch P_loc, written as the sum over the 8 children of
//     P_c^T K_child P_c with the trilinear weights of App. E.1). Level 1 depends only on the
//     8-bit child mask, so it is a 256-entry table; levels >= 2 are stored per element;
//   * D x D block-diagonal inverses of the coarse operators (smoother, Sec. 4.6);
//   * the coarsest level's dense matrix K_L + rho J (J couples equal components of all
//     nodes, rho = mean diagonal / number of coarse nodes) kept in FP64, and its
//     generalized inverse by blocked in-place Gauss-Jordan with semidefinite pivot
//     dropping: in FP32 for the mixed-precision solves, and in FP64 (built on first use)
//     for the all-FP64 path. For right-hand sides orthogonal to translations this returns
//     the zero-mean solution (the gauge of Sec. 3.1); Alg. 1's inexact coarsest GS is
//     replaced by this exact solve.
#include <algorithm>
#include <mutex>
#include <optional>
#include <set>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace gmt {

void build_node_stencils(gmt_hierarchy* h, int level, bool fp64);

// ------------------------------------------------------------------ element matrices
__device__ double gauss_x(int q) { return q ? 0.5 + 0.5 / sqrt(3.0) : 0.5 - 0.5 / sqrt(3.0); }

__device__ double shape_grad(int a, int d, const double xi[3]) {
  double v = ((a >> d) & 1) ? 1.0 : -1.0;
  for (int e = 0; e < 3; ++e)
    if (e != d) v *= ((a >> e) & 1) ? xi[e] : 1.0 - xi[e];
  return v;
}

// Voigt (xx, yy, zz, yz, xz, xy) engineering strain of dof col = 3a + i
__device__ double strain_B(int row, int col, const double xi[3]) {
  int a = col / 3, i = col % 3;
  double g[3] = {shape_grad(a, 0, xi), shape_grad(a, 1, xi), shape_grad(a, 2, xi)};
  switch (row) {
    case 0: return i == 0 ? g[0] : 0.0;
    case 1: return i == 1 ? g[1] : 0.0;
    case 2: return i == 2 ? g[2] : 0.0;
    case 3: return i == 1 ? g[2] : (i == 2 ? g[1] : 0.0);
    case 4: return i == 0 ? g[2] : (i == 2 ? g[0] : 0.0);
    default: return i == 0 ? g[1] : (i == 1 ? g[0] : 0.0);
  }
}

// out: Ke[(8D)^2], Fe[8D*M], X0[8D*M], C0[M*M]
__global__ void k_element(int physics, double E, double nu, double kappa, double* out) {
  const int D = physics == GMT_ELASTIC ? 3 : 1, M = physics == GMT_ELASTIC ? 6 : 3;
  const int R = 8 * D, MM = R * R;
  __shared__ double sK[576], sX[144], sF[144];
  const int t = threadIdx.x;
  if (t < MM) {
    int r = t / R, c = t % R;
    double acc = 0.0;
    if (physics == GMT_ELASTIC) {
      double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E / (2.0 * (1.0 + nu));
      for (int q = 0; q < 8; ++q) {
        double xi[3] = {gauss_x(q & 1), gauss_x((q >> 1) & 1), gauss_x((q >> 2) & 1)};
        double br[6], bc[6];
        for (int i = 0; i < 6; ++i) {
          br[i] = strain_B(i, r, xi);
          bc[i] = strain_B(i, c, xi);
        }
        double s = 0.0;
        for (int i = 0; i < 6; ++i) {
          double ci = 0.0;  // (C0 bc)_i
          if (i < 3) {
            for (int j = 0; j < 3; ++j) ci += (i == j ? lam + 2.0 * mu : lam) * bc[j];
          } else {
            ci = mu * bc[i];
          }
          s += br[i] * ci;
        }
        acc += 0.125 * s;
      }
    } else {
      for (int q = 0; q < 8; ++q) {
        double xi[3] = {gauss_x(q & 1), gauss_x((q >> 1) & 1), gauss_x((q >> 2) & 1)};
        double s = 0.0;
        for (int d = 0; d < 3; ++d) s += shape_grad(r, d, xi) * shape_grad(c, d, xi);
        acc += 0.125 * kappa * s;
      }
    }
    sK[t] = acc;
    out[t] = acc;
  }
  if (t < R * M) {
    int r = t / M, m = t % M;
    double v;
    if (physics == GMT_ELASTIC) {
      int a = r / 3, i = r % 3;
      double x[3] = {(double)(a & 1), (double)((a >> 1) & 1), (double)((a >> 2) & 1)};
      // symmetric strain tensor of Voigt mode m (engineering shear -> 1/2 entries)
      double Em[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      if (m < 3) {
        Em[m][m] = 1.0;
      } else {
        int p = m == 3 ? 1 : 0, q = m == 5 ? 1 : 2;
        Em[p][q] = Em[q][p] = 0.5;
      }
      v = Em[i][0] * x[0] + Em[i][1] * x[1] + Em[i][2] * x[2];
    } else {
      v = (double)((r >> m) & 1);
    }
    sX[t] = v;
  }
  __syncthreads();
  if (t < R * M) {
    int r = t / M, m = t % M;
    double s = 0.0;
    for (int c = 0; c < R; ++c) s += sK[r * R + c] * sX[c * M + m];
    sF[t] = s;
    out[MM + t] = s;
    out[MM + R * M + t] = sX[t];
  }
  __syncthreads();
  if (t < M * M) {
    int I = t / M, J = t % M;
    double s = 0.0;
    for (int r = 0; r < R; ++r) s += sX[r * M + I] * sF[r * M + J];
    out[MM + 2 * R * M + t] = s;
  }
}

// launch wrapper for other translation units: element data of one material into `out`
// (layout as k_element)
void launch_element_matrices(cudaStream_t s, int physics, double E, double nu, double kappa,
                             double* out) {
  k_element<<<1, 576, 0, s>>>(physics, E, nu, kappa, out);
  GMT_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ Galerkin
// weight of coarse-local vertex b at child c's local vertex a (App. E.1 trilinear weights)
__device__ __forceinline__ double wchild(int c, int a, int b) {
  double w = 1.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double pos = 0.5 * (((c >> d) & 1) + ((a >> d) & 1));
    w *= 1.0 - fabs(pos - (double)((b >> d) & 1));
  }
  return w;
}

// Q[c][y] = P_c^T K[y] P_c for the gridDim.y input matrices K[y] (block (c, y), one thread
// per entry)
__global__ void k_child_products(const double* __restrict__ Kin, int D, double* __restrict__ Q) {
  const int R = 8 * D, MM = R * R;
  const int c = blockIdx.x, y = blockIdx.y, t = threadIdx.x;
  const double* Ke = Kin + (int64_t)y * MM;
  if (t >= MM) return;
  int r = t / R, s = t % R;
  int b = r / D, i = r % D, bb = s / D, j = s % D;
  double acc = 0.0;
  for (int a = 0; a < 8; ++a) {
    double wa = wchild(c, a, b);
    if (wa == 0.0) continue;
    for (int aa = 0; aa < 8; ++aa) {
      double wb = wchild(c, aa, bb);
      if (wb == 0.0) continue;
      acc += wa * wb * Ke[(a * D + i) * R + aa * D + j];
    }
  }
  Q[((int64_t)c * gridDim.y + y) * MM + t] = acc;
}

// mask tables: T[y][mask] = sum_{c in mask} Q[y][c] for gridDim.y groups of 8 matrices
// (level 1: one group, Q[c] = P_c^T K_e P_c; level 2: group c holds P_c^T Q[c'] P_c)
__global__ void k_mask_table(const double* __restrict__ Q, int MM, double* __restrict__ T64,
                             float* __restrict__ T32) {
  const int m = blockIdx.x;
  const int64_t y = blockIdx.y;
  const double* Qy = Q + y * 8 * MM;
  for (int t = threadIdx.x; t < MM; t += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < 8; ++c)
      if ((m >> c) & 1) acc += Qy[(int64_t)c * MM + t];
    T64[(y * 256 + m) * MM + t] = acc;
    if (T32) T32[(y * 256 + m) * MM + t] = (float)acc;
  }
}

// level 2: K(E) = sum over active children c of T2[c][mask(c)], where mask(c) is the
// level-1 child's own child mask (its index into the level-1 table) and
// T2[c][m] = sum_{c' in m} P_c^T Q[c'] P_c = P_c^T K1[m] P_c (Galerkin products are linear)
__global__ void k_galerkin_l2(int D, int nc, const int* __restrict__ elem_slot,
                              const int* __restrict__ cbxyz, bool cdense,
                              const uint8_t* __restrict__ cchild, int nf, int fnbx,
                              const int* __restrict__ fbmap, bool fdense,
                              const int* __restrict__ fkidx, const double* __restrict__ T2,
                              double* __restrict__ K64, float* __restrict__ K32) {
  const int MM = 64 * D * D;
  const int64_t e = blockIdx.x;
  const int t = threadIdx.x;
  __shared__ int sidx[8];
  int X, Y, Z;
  slot_coords(elem_slot[e], nc, cdense, cbxyz, X, Y, Z);
  const unsigned cm = cchild[X + (int64_t)nc * (Y + (int64_t)nc * Z)];
  if (t < 8) {
    int id = -1;
    if ((cm >> t) & 1) {
      const int fx = 2 * X + (t & 1), fy = 2 * Y + ((t >> 1) & 1), fz = 2 * Z + ((t >> 2) & 1);
      id = t * 256 + fkidx[site_slot(fx, fy, fz, nf, fnbx, fbmap, fdense)];
    }
    sidx[t] = id;
  }
  __syncthreads();
  if (t >= MM) return;
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (sidx[c] >= 0) acc += T2[(int64_t)sidx[c] * MM + t];
  K64[e * MM + t] = acc;
  K32[e * MM + t] = (float)acc;
}

// Nonzero trilinear weights per (child c, coarse-local vertex b): the child-local vertices
// a with W[c][a][b] != 0 and the weights (exact binary fractions). 1, 2, 4 or 8 per (c, b).
struct ChildWeights {
  unsigned char cnt[8][8];
  unsigned char a[8][8][8];
  double w[8][8][8];
};
__constant__ ChildWeights c_cw;

static ChildWeights make_child_weights() {
  ChildWeights cw;
  std::memset(&cw, 0, sizeof(cw));
  for (int c = 0; c < 8; ++c)
    for (int b = 0; b < 8; ++b)
      for (int a = 0; a < 8; ++a) {
        double w = 1.0;
        for (int d = 0; d < 3; ++d) {
          const double pos = 0.5 * (((c >> d) & 1) + ((a >> d) & 1));
          w *= 1.0 - std::fabs(pos - (double)((b >> d) & 1));
        }
        if (w != 0.0) {
          const int k = cw.cnt[c][b]++;
          cw.a[c][b][k] = (unsigned char)a;
          cw.w[c][b][k] = w;
        }
      }
  return cw;
}

// the weight table is the same for every hierarchy: uploaded once per device, before any
// kernel that reads it (a synchronous copy, so no stream of another hierarchy sees it change)
static void upload_child_weights() {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  GMT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(dev)) return;
  const ChildWeights cw = make_child_weights();
  GMT_CUDA(cudaMemcpyToSymbol(c_cw, &cw, sizeof(cw)));
  done.insert(dev);
}

// levels >= 2: K(E) = sum over active children c of P_c^T K(child) P_c, using only the
// nonzero weights: T[(a i), (b' j)] = sum_{a'} K[(a i)(a' j)] W[c][a'][b'], then
// K(E)[(b i), (b' j)] += sum_a W[c][a][b] T[(a i), (b' j)]
__global__ void k_galerkin_elem(int D, int nc, const int* __restrict__ elem_slot,
                                const int* __restrict__ cbxyz, bool cdense,
                                const uint8_t* __restrict__ cchild, int nf, int fnbx,
                                const int* __restrict__ fbmap, bool fdense,
                                const int* __restrict__ fkidx, const double* __restrict__ Kf,
                                double* __restrict__ K64, float* __restrict__ K32) {
  const int R = 8 * D, MM = R * R;
  __shared__ double sK[576], sT[576];
  const int64_t e = blockIdx.x;
  const int t = threadIdx.x;
  int X, Y, Z;
  slot_coords(elem_slot[e], nc, cdense, cbxyz, X, Y, Z);
  const unsigned cm = cchild[X + (int64_t)nc * (Y + (int64_t)nc * Z)];
  const int r = t / R, s = t % R;
  const int rb = r / D, ri = r % D, sb = s / D, sj = s % D;
  double acc = 0.0;
  for (int c = 0; c < 8; ++c) {
    if (!((cm >> c) & 1)) continue;  // uniform across the block
    const int fx = 2 * X + (c & 1), fy = 2 * Y + ((c >> 1) & 1), fz = 2 * Z + ((c >> 2) & 1);
    const int64_t fs = site_slot(fx, fy, fz, nf, fnbx, fbmap, fdense);
    const double* Kc = Kf + (int64_t)fkidx[fs] * MM;
    __syncthreads();
    if (t < MM) sK[t] = Kc[t];
    __syncthreads();
    if (t < MM) {
      double v = 0.0;
      const int n = c_cw.cnt[c][sb];
      for (int k = 0; k < n; ++k) v += sK[r * R + c_cw.a[c][sb][k] * D + sj] * c_cw.w[c][sb][k];
      sT[t] = v;
    }
    __syncthreads();
    if (t < MM) {
      const int n = c_cw.cnt[c][rb];
      for (int k = 0; k < n; ++k) acc += c_cw.w[c][rb][k] * sT[(c_cw.a[c][rb][k] * D + ri) * R + s];
    }
  }
  if (t < MM) {
    K64[e * MM + t] = acc;
    K32[e * MM + t] = (float)acc;
  }
}

// ------------------------------------------------------------------ element densities
// s_e = rho_min + rho_e^p (SIMP, App. F.3) at the level-0 slot of each element's origin
__global__ void k_set_density(int64_t ne, const int* __restrict__ elem_slot,
                              const double* __restrict__ rho, double rho_min, double p,
                              double* __restrict__ c64, float* __restrict__ c32,
                              double* __restrict__ r64) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int64_t s = elem_slot[e];
  const double r = rho[e];
  const double c = rho_min + pow(r, p);
  c64[s] = c;
  c32[s] = (float)c;
  r64[s] = r;
}

// level 1 with densities: element matrices indexed by element id at the element's origin
__global__ void k_kidx_el(int64_t ne, const int* __restrict__ elem_slot, int* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne) out[elem_slot[e]] = (int)e;
}

// level 1 with densities: K(E) = sum over active children c of s_c P_c^T K_e P_c, with
// Q[c] = P_c^T K_e P_c and s_c the coefficient of the level-0 element at child position c
// (the Galerkin product is linear in the child matrices)
__global__ void k_galerkin_l1_coef(int D, int nc, const int* __restrict__ elem_slot,
                                   const int* __restrict__ cbxyz, bool cdense,
                                   const uint8_t* __restrict__ cchild, int nf, int fnbx,
                                   const int* __restrict__ fbmap, bool fdense,
                                   const double* __restrict__ fcoef, const double* __restrict__ Q,
                                   double* __restrict__ K64, float* __restrict__ K32) {
  const int MM = 64 * D * D;
  const int64_t e = blockIdx.x;
  const int t = threadIdx.x;
  __shared__ double sc[8];
  int X, Y, Z;
  slot_coords(elem_slot[e], nc, cdense, cbxyz, X, Y, Z);
  const unsigned cm = cchild[X + (int64_t)nc * (Y + (int64_t)nc * Z)];
  if (t < 8) {
    double v = 0.0;
    if ((cm >> t) & 1) {
      const int fx = 2 * X + (t & 1), fy = 2 * Y + ((t >> 1) & 1), fz = 2 * Z + ((t >> 2) & 1);
      v = fcoef[site_slot(fx, fy, fz, nf, fnbx, fbmap, fdense)];
    }
    sc[t] = v;
  }
  __syncthreads();
  if (t >= MM) return;
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (sc[c] != 0.0) acc += sc[c] * Q[(int64_t)c * MM + t];
  K64[e * MM + t] = acc;
  K32[e * MM + t] = (float)acc;
}

// level-0 load with densities: f_n = sum over active incident elements e = n - a of
// s_e (K_e x0)[a], written in the slot layout in FP64 and FP32
template <int D, int M>
__global__ void k_fine_load(int n, int nbx, const int* __restrict__ bxyz,
                            const int* __restrict__ bmap, bool dense, int64_t nslots,
                            const uint8_t* __restrict__ mask, const double* __restrict__ coef,
                            const double* __restrict__ Fe, double* __restrict__ f64,
                            float* __restrict__ f32) {
  constexpr int C = D * M;
  const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslots) return;
  const unsigned mk = mask[sl];
  double f[C];
#pragma unroll
  for (int v = 0; v < C; ++v) f[v] = 0.0;
  if (mk) {
    int x, y, z;
    slot_coords(sl, n, dense, bxyz, x, y, z);
    for (int a = 0; a < 8; ++a) {
      if (!((mk >> a) & 1u)) continue;
      const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
      const double sc =
          coef[site_slot((x - ax + n) % n, (y - ay + n) % n, (z - az + n) % n, n, nbx, bmap, dense)];
#pragma unroll
      for (int v = 0; v < C; ++v) f[v] += sc * Fe[(a * D + v / M) * M + v % M];
    }
  }
#pragma unroll
  for (int v = 0; v < C; ++v) {
    f64[vaddr(sl, v, C)] = f[v];
    f32[vaddr(sl, v, C)] = (float)f[v];
  }
}

// D x D block-diagonal inverse of a stored operator at every active slot; coef (nullable,
// per slot of the element's origin) scales each element matrix (level 0 with densities)
__global__ void k_diag_inv(int D, int n, int nbx, const int* __restrict__ bxyz,
                           const int* __restrict__ bmap, bool dense, int64_t nslots,
                           const uint8_t* __restrict__ mask, const int* __restrict__ kidx,
                           const double* __restrict__ K, const double* __restrict__ coef,
                           double* __restrict__ d64, float* __restrict__ d32) {
  const int R = 8 * D, MM = R * R;
  int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslots) return;
  unsigned m = mask[sl];
  double A[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (m && (dense ? sl < (int64_t)n * n * n : true)) {
    int x, y, z;
    slot_coords(sl, n, dense, bxyz, x, y, z);
    for (int a = 0; a < 8; ++a) {
      if (!((m >> a) & 1)) continue;
      int ex = (x - (a & 1) + n) % n, ey = (y - ((a >> 1) & 1) + n) % n,
          ez = (z - ((a >> 2) & 1) + n) % n;
      int64_t es = site_slot(ex, ey, ez, n, nbx, bmap, dense);
      const double* Kc = K + (int64_t)kidx[es] * MM;
      const double sc = coef ? coef[es] : 1.0;
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) A[i * D + j] += sc * Kc[(a * D + i) * R + a * D + j];
    }
  }
  double Inv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (m) {
    if (D == 1) {
      Inv[0] = 1.0 / A[0];
    } else {
      double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8],
             c02 = A[3] * A[7] - A[4] * A[6];
      double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
      double id = 1.0 / det;
      Inv[0] = c00 * id;
      Inv[1] = (A[2] * A[7] - A[1] * A[8]) * id;
      Inv[2] = (A[1] * A[5] - A[2] * A[4]) * id;
      Inv[3] = c01 * id;
      Inv[4] = (A[0] * A[8] - A[2] * A[6]) * id;
      Inv[5] = (A[2] * A[3] - A[0] * A[5]) * id;
      Inv[6] = c02 * id;
      Inv[7] = (A[1] * A[6] - A[0] * A[7]) * id;
      Inv[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    }
  }
  for (int q = 0; q < D * D; ++q) {
    d64[sl * D * D + q] = Inv[q];
    d32[sl * D * D + q] = (float)Inv[q];
  }
}

// ------------------------------------------------------------------ coarsest dense solve
// thread per (canonical node i, neighbour offset d): the D x D block K(i, i + d)
__global__ void k_coarse_assemble(int D, int level, int n, int nbx, const int* __restrict__ bxyz,
                                  const int* __restrict__ bmap, bool dense,
                                  const uint8_t* __restrict__ eflag,
                                  const int* __restrict__ canon_slot,
                                  const int* __restrict__ slot_canon,
                                  const int* __restrict__ kidx, const double* __restrict__ K,
                                  const double* __restrict__ Ke, const double* __restrict__ coef,
                                  int64_t nn, int64_t m, double* __restrict__ A) {
  const int R = 8 * D, MM = R * R;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nn * 27) return;
  int64_t i = g / 27;
  int d = (int)(g % 27);
  int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
  int x, y, z;
  slot_coords(canon_slot[i], n, dense, bxyz, x, y, z);
  double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  bool any = false;
  for (int a = 0; a < 8; ++a) {
    int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
    int bx = ax + dx, by = ay + dy, bz = az + dz;
    if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
    int b = bx + 2 * by + 4 * bz;
    int ex = (x - ax + n) % n, ey = (y - ay + n) % n, ez = (z - az + n) % n;
    if (!eflag[ex + (int64_t)n * (ey + (int64_t)n * ez)]) continue;
    const double* Kc;
    double sc = 1.0;
    if (level == 0) {
      Kc = Ke;
      if (coef) sc = coef[site_slot(ex, ey, ez, n, nbx, bmap, dense)];
    } else {
      int64_t es = site_slot(ex, ey, ez, n, nbx, bmap, dense);
      Kc = K + (int64_t)kidx[es] * MM;
    }
    for (int p = 0; p < D; ++p)
      for (int q = 0; q < D; ++q) S[p * D + q] += sc * Kc[(a * D + p) * R + b * D + q];
    any = true;
  }
  if (!any) return;
  int jx = (x + dx + n) % n, jy = (y + dy + n) % n, jz = (z + dz + n) % n;
  int64_t js = site_slot(jx, jy, jz, n, nbx, bmap, dense);
  int64_t j = slot_canon[js];
  for (int p = 0; p < D; ++p)
    for (int q = 0; q < D; ++q) A[(i * D + p) * m + j * D + q] = S[p * D + q];
}

__global__ void k_diag_sum(const double* __restrict__ A, int64_t m, double* __restrict__ out) {
  __shared__ double sh[1024];
  double s = 0.0, mx = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    s += A[i * m + i];
    mx = fmax(mx, A[i * m + i]);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
  __syncthreads();
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[1] = sh[0];
}

// rho J adds rho * n to the eigenvalue of each translation; rho = mean diagonal / n puts it
// at the mean diagonal, inside the spectrum of K_L, so the regularized matrix is as well
// conditioned as K_L on the complement of the translations (for right-hand sides orthogonal
// to translations the solution does not depend on rho > 0). Pivot tolerances are relative
// to the largest diagonal entry of the regularized matrix. All on the device: no host
// round trip.
__global__ void k_coarse_scalars(const double* __restrict__ ds, int64_t m, int64_t n_nodes,
                                 double* __restrict__ out) {
  const double rho = ds[0] / (double)m / (double)n_nodes;
  const double dmax = ds[1] + rho * (double)n_nodes;
  out[0] = rho;
  out[1] = 1e-6 * dmax;
  out[2] = 1e-12 * dmax;
}

__global__ void k_add_rho(double* __restrict__ A, int64_t m, int D, const double* __restrict__ sc) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m * m) return;
  int64_t r = g / m, c = g % m;
  if (r % D == c % D) A[g] += sc[0];
}

// Blocked in-place Gauss-Jordan inversion with 32-wide pivot panels. For the panel
// rows/columns P and the rest Q of the current matrix:
//   A_PP <- A_PP^+ (small GJ in shared memory, null pivots dropped: semidefinite case)
//   A_PQ <- A_PP^+ A_PQ,   A_QP <- -A_QP A_PP^+,   A_QQ <- A_QQ - A_QP A_PP^+ A_PQ
// After all panels the matrix holds the (generalized) inverse.
constexpr int GJB = 32;

// one block of GJB x GJB threads inverts the bb x bb diagonal panel block (pivots <= tol
// dropped), thread (i, j) owning entry (i, j). Step k reads the pivot row and column from a
// double buffer that the owners of row / column k filled while updating in step k - 1, so
// each step needs a single block barrier.
template <typename T>
__global__ void __launch_bounds__(GJB * GJB) k_gj_panel(const T* __restrict__ A, int64_t m,
                                                       int64_t k0, int bb,
                                                       const double* __restrict__ tolp,
                                                       T* __restrict__ inv) {
  __shared__ T rowk[2][GJB], colk[2][GJB];
  const int t = threadIdx.x, i = t / GJB, j = t % GJB;
  const bool in = i < bb && j < bb;
  const T tol = (T)*tolp;
  T v = in ? A[(k0 + i) * m + k0 + j] : T(0);
  if (i == 0) rowk[0][j] = v;
  if (j == 0) colk[0][i] = v;
  for (int k = 0; k < bb; ++k) {
    const int buf = k & 1;
    __syncthreads();
    const T p = rowk[buf][k];
    const bool ok = p > tol;
    const T ip = ok ? T(1) / p : T(0);
    const T rk = rowk[buf][j], ck = colk[buf][i];
    if (in) {
      if (!ok) v = (i == k || j == k) ? T(0) : v;
      else if (i == k) v = (j == k) ? ip : rk * ip;
      else if (j == k) v = -ck * ip;
      else v = v - ck * (rk * ip);
    }
    if (i == k + 1) rowk[buf ^ 1][j] = v;
    if (j == k + 1) colk[buf ^ 1][i] = v;
  }
  if (in) inv[i * GJB + j] = v;
}

// T = A_PP^+ A_P* (rows of the panel, all columns) and O = A_*P (copy of the panel columns);
// one thread per (panel row c, column j)
template <typename T>
__global__ void k_gj_rows(const T* __restrict__ A, int64_t m, int64_t k0, int bb,
                          const T* __restrict__ inv, T* __restrict__ Tp, T* __restrict__ O) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)GJB * m) return;
  const int c = (int)(g / m);
  const int64_t j = g % m;
  if (c < bb) {
    T acc = T(0);
    for (int r = 0; r < bb; ++r) acc += inv[c * GJB + r] * A[(k0 + r) * m + j];
    Tp[c * m + j] = acc;
    O[j * GJB + c] = A[j * m + k0 + c];
  }
}

// the rank-bb update of everything: 64 x 64 tiles per 256-thread block, each thread a
// 4 x 4 register tile (8 shared-memory loads per 16 multiply-adds per panel column)
template <typename T>
__global__ void __launch_bounds__(256) k_gj_update(T* __restrict__ A, int64_t m, int64_t k0,
                                                   int bb, const T* __restrict__ inv,
                                                   const T* __restrict__ Tp,
                                                   const T* __restrict__ O) {
  __shared__ T sO[GJB][64 + 1];   // O^T of this tile's rows: sO[r][a] = O[i0 + a][r]
  __shared__ T sT[GJB][64 + 1];   // T of this tile's columns: sT[r][b] = T[r][j0 + b]
  __shared__ T sI[GJB][GJB + 1];  // the panel inverse
  const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
  const int t = threadIdx.x;
  for (int q = t; q < 64 * GJB; q += 256) {
    const int a = q / GJB, r = q % GJB;
    sO[r][a] = (i0 + a < m && r < bb) ? O[(i0 + a) * GJB + r] : T(0);
    const int rr = q / 64, c = q % 64;
    sT[rr][c] = (rr < bb && j0 + c < m) ? Tp[rr * m + j0 + c] : T(0);
  }
  for (int q = t; q < GJB * GJB; q += 256) sI[q / GJB][q % GJB] = inv[q];
  __syncthreads();
  const int tx = t & 15, ty = t >> 4;   // 16 x 16 threads, rows ty + 16 k, columns tx + 16 l
  T acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[k][l] = T(0);
#pragma unroll 8
  for (int r = 0; r < GJB; ++r) {
    T o[4], tv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = sO[r][ty + 16 * k];
#pragma unroll
    for (int l = 0; l < 4; ++l) tv[l] = sT[r][tx + 16 * l];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) acc[k][l] += o[k] * tv[l];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int a = ty + 16 * k;
    const int64_t i = i0 + a;
    if (i >= m) continue;
    const bool ip = i >= k0 && i < k0 + bb;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int c = tx + 16 * l;
      const int64_t j = j0 + c;
      if (j >= m) continue;
      const bool jp = j >= k0 && j < k0 + bb;
      T v;
      if (ip && jp) {
        v = sI[i - k0][j - k0];
      } else if (ip) {
        v = sT[i - k0][c];
      } else if (jp) {
        T s2 = T(0);
        for (int r = 0; r < bb; ++r) s2 += sO[r][a] * sI[r][j - k0];
        v = -s2;
      } else {
        v = A[i * m + j] - acc[k][l];
      }
      A[i * m + j] = v;
    }
  }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// in-place blocked Gauss-Jordan of an m x m matrix (generalized inverse, pivots <= tol dropped)
template <typename T>
static void gauss_jordan(gmt_hierarchy* h, T* A, int64_t m, const double* tol, Arena& tmp) {
  cudaStream_t s = h->stream;
  T* inv = tmp.alloc<T>(GJB * GJB);
  T* Tp = tmp.alloc<T>(GJB * m);
  T* O = tmp.alloc<T>(GJB * m);
  const dim3 ug((unsigned)((m + 63) / 64), (unsigned)((m + 63) / 64));
  for (int64_t k0 = 0; k0 < m; k0 += GJB) {
    const int bb = (int)std::min<int64_t>(GJB, m - k0);
    k_gj_panel<T><<<1, GJB * GJB, 0, s>>>(A, m, k0, bb, tol, inv);
    GMT_LAUNCH_CHECK();
    k_gj_rows<T><<<grid_for(GJB * m, 256), 256, 0, s>>>(A, m, k0, bb, inv, Tp, O);
    GMT_LAUNCH_CHECK();
    k_gj_update<T><<<ug, 256, 0, s>>>(A, m, k0, bb, inv, Tp, O);
    GMT_LAUNCH_CHECK();
  }
}

// exact FP64 generalized inverse of the regularized coarsest matrix (FP64 solve path; lazy)
void build_coarse_inverse64(gmt_hierarchy* h) {
  if (h->Ainv) return;
  const int64_t m = h->m;
  h->Ainv = h->op.alloc<double>(m * m);
  GMT_CUDA(cudaMemcpyAsync(h->Ainv, h->A64, m * m * sizeof(double), cudaMemcpyDeviceToDevice,
                           h->stream));
  Arena tmp(h->stream);
  gauss_jordan<double>(h, h->Ainv, m, h->cscal + 2, tmp);
  GMT_CUDA(cudaStreamSynchronize(h->stream));
}

// ------------------------------------------------------------------ host driver
void prepare_material(gmt_hierarchy* h, int physics, double E, double nu, double kappa) {
  cudaStream_t s = h->stream;
  std::optional<TraceScope> ts_ops;
  ts_ops.emplace(&h->tracer, s, TR_OPS, 0.0);
  h->op.release();
  h->A64 = nullptr;
  h->X32 = nullptr;
  h->Ainv = nullptr;
  h->cscal = nullptr;
  for (Level& l : h->lv) {
    l.K64 = l.S64 = l.dinv64 = nullptr;
    l.K32 = l.S32 = l.dinv32 = nullptr;
    l.S16 = nullptr;
    l.kidx_el = nullptr;
    l.lmax = 0.0;
  }
  h->f0_64 = nullptr;
  h->f0_32 = nullptr;
  h->prepared = false;
  Material& mt = h->mat;
  mt = Material();
  mt.physics = physics;
  mt.E = E;
  mt.nu = nu;
  mt.k = kappa;
  mt.D = physics == GMT_ELASTIC ? 3 : 1;
  mt.M = physics == GMT_ELASTIC ? 6 : 3;
  mt.C = mt.D * mt.M;
  const int D = mt.D, M = mt.M, R = 8 * D, MM = R * R;
  mt.MM = MM;
  Arena tmp(s);
  // element matrices
  double* eout = tmp.alloc<double>(MM + 2 * R * M + M * M);
  k_element<<<1, 576, 0, s>>>(physics, E, nu, kappa, eout);
  GMT_LAUNCH_CHECK();
  std::vector<double> host(MM + 2 * R * M + M * M);
  GMT_CUDA(cudaMemcpyAsync(host.data(), eout, host.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  GMT_CUDA(cudaStreamSynchronize(s));
  std::memcpy(mt.Ke, host.data(), MM * sizeof(double));
  std::memcpy(mt.Fe, host.data() + MM, R * M * sizeof(double));
  std::memcpy(mt.X0, host.data() + MM + R * M, R * M * sizeof(double));
  std::memcpy(mt.C0, host.data() + MM + 2 * R * M, M * M * sizeof(double));
  // gross load norm sqrt(sum_e ||s_e K_e x0||^2) per case (s_e = 1 without densities)
  const double ss2 = h->dens ? h->coef_sum2 : (double)h->lv[0].n_elems;
  for (int m = 0; m < M; ++m) {
    double s2 = 0.0;
    for (int r = 0; r < R; ++r) s2 += mt.Fe[r * M + m] * mt.Fe[r * M + m];
    mt.gross[m] = std::sqrt(ss2 * s2);
  }
  h->Ke64 = h->op.alloc<double>(MM);
  h->Ke32 = h->op.alloc<float>(MM);
  GMT_CUDA(cudaMemcpyAsync(h->Ke64, eout, MM * sizeof(double), cudaMemcpyDeviceToDevice, s));
  {
    std::vector<float> k32(MM);
    for (int i = 0; i < MM; ++i) k32[i] = (float)mt.Ke[i];
    GMT_CUDA(cudaMemcpyAsync(h->Ke32, k32.data(), MM * sizeof(float), cudaMemcpyHostToDevice, s));
    GMT_CUDA(cudaStreamSynchronize(s));
  }
  // Galerkin coarse operators
  upload_child_weights();
  double* Q = nullptr;
  if (h->L >= 2) {
    Q = tmp.alloc<double>(8 * MM);
    k_child_products<<<dim3(8, 1), MM, 0, s>>>(h->Ke64, D, Q);
    GMT_LAUNCH_CHECK();
    Level& l1 = h->lv[1];
    if (h->dens) {
      // per element: the child coefficients weight the 8 child products
      l1.K64 = h->op.alloc<double>(l1.n_elems * (size_t)MM);
      l1.K32 = h->op.alloc<float>(l1.n_elems * (size_t)MM);
      l1.kidx_el = h->op.alloc<int>(l1.nslots);
      GMT_CUDA(cudaMemsetAsync(l1.kidx_el, 0xff, l1.nslots * sizeof(int), s));
      k_kidx_el<<<grid_for(l1.n_elems, 256), 256, 0, s>>>(l1.n_elems, l1.elem_slot, l1.kidx_el);
      GMT_LAUNCH_CHECK();
      const Level& l0 = h->lv[0];
      k_galerkin_l1_coef<<<(unsigned)l1.n_elems, MM, 0, s>>>(
          D, l1.n, l1.elem_slot, l1.brick_xyz, l1.dense, l1.child, l0.n, l0.nbx, l0.brick_map,
          l0.dense, h->coef64, Q, l1.K64, l1.K32);
    } else {
      l1.K64 = h->op.alloc<double>(256 * (size_t)MM);
      l1.K32 = h->op.alloc<float>(256 * (size_t)MM);
      k_mask_table<<<dim3(256, 1), 256, 0, s>>>(Q, MM, l1.K64, l1.K32);
    }
    GMT_LAUNCH_CHECK();
  }
  for (int l = 2; l < h->L; ++l) {
    Level& c = h->lv[l];
    Level& f = h->lv[l - 1];
    c.K64 = h->op.alloc<double>(c.n_elems * (size_t)MM);
    c.K32 = h->op.alloc<float>(c.n_elems * (size_t)MM);
    if (l == 2 && !h->dens) {
      // 8 x 8 products P_c^T Q[c'] P_c, then the 8 x 256 table T2[c][m]
      double* Q2 = tmp.alloc<double>(64 * (size_t)MM);
      k_child_products<<<dim3(8, 8), MM, 0, s>>>(Q, D, Q2);
      GMT_LAUNCH_CHECK();
      double* T2 = tmp.alloc<double>(8 * 256 * (size_t)MM);
      k_mask_table<<<dim3(256, 8), 256, 0, s>>>(Q2, MM, T2, nullptr);
      GMT_LAUNCH_CHECK();
      k_galerkin_l2<<<(unsigned)c.n_elems, MM, 0, s>>>(D, c.n, c.elem_slot, c.brick_xyz, c.dense,
                                                       c.child, f.n, f.nbx, f.brick_map, f.dense,
                                                       f.kidx, T2, c.K64, c.K32);
    } else {
      k_galerkin_elem<<<(unsigned)c.n_elems, MM, 0, s>>>(D, c.n, c.elem_slot, c.brick_xyz,
                                                         c.dense, c.child, f.n, f.nbx,
                                                         f.brick_map, f.dense, op_kidx(f), f.K64,
                                                         c.K64, c.K32);
    }
    GMT_LAUNCH_CHECK();
  }
  if (h->dens) {
    // level 0 with densities: block-diagonal inverses, the load vector and (unless level 0
    // is the coarsest) the per-node stencils, like a coarse level
    Level& l0 = h->lv[0];
    l0.dinv64 = h->op.alloc<double>(l0.nslots * D * D);
    l0.dinv32 = h->op.alloc<float>(l0.nslots * D * D);
    k_diag_inv<<<grid_for(l0.nslots, 128), 128, 0, s>>>(D, l0.n, l0.nbx, l0.brick_xyz,
                                                        l0.brick_map, l0.dense, l0.nslots, l0.mask,
                                                        l0.kidx, h->Ke64, h->coef64, l0.dinv64,
                                                        l0.dinv32);
    GMT_LAUNCH_CHECK();
    double* Fe = tmp.alloc<double>(R * M);
    GMT_CUDA(cudaMemcpyAsync(Fe, mt.Fe, R * M * sizeof(double), cudaMemcpyHostToDevice, s));
    h->f0_64 = h->op.alloc<double>(l0.nslots * mt.C);
    h->f0_32 = h->op.alloc<float>(l0.nslots * mt.C);
    if (D == 3)
      k_fine_load<3, 6><<<grid_for(l0.nslots, 128), 128, 0, s>>>(
          l0.n, l0.nbx, l0.brick_xyz, l0.brick_map, l0.dense, l0.nslots, l0.mask, h->coef64, Fe,
          h->f0_64, h->f0_32);
    else
      k_fine_load<1, 3><<<grid_for(l0.nslots, 128), 128, 0, s>>>(
          l0.n, l0.nbx, l0.brick_xyz, l0.brick_map, l0.dense, l0.nslots, l0.mask, h->coef64, Fe,
          h->f0_64, h->f0_32);
    GMT_LAUNCH_CHECK();
    GMT_CUDA(cudaStreamSynchronize(s));   // Fe (tmp) is read by the kernel above
    if (h->L > 1) build_node_stencils(h, 0, false);
  }
  for (int l = 1; l < h->L; ++l) {
    Level& c = h->lv[l];
    c.dinv64 = h->op.alloc<double>(c.nslots * D * D);
    c.dinv32 = h->op.alloc<float>(c.nslots * D * D);
    k_diag_inv<<<grid_for(c.nslots, 128), 128, 0, s>>>(D, c.n, c.nbx, c.brick_xyz, c.brick_map,
                                                       c.dense, c.nslots, c.mask, op_kidx(c),
                                                       c.K64, nullptr, c.dinv64, c.dinv32);
    GMT_LAUNCH_CHECK();
  }
  for (int l = 1; l + 1 < h->L; ++l) build_node_stencils(h, l, false);
  // coarsest generalized inverse
  ts_ops.reset();
  TraceScope ts_cinv(&h->tracer, s, TR_CINV, 0.0);
  {
    const int lc = h->L - 1;
    Level& c = h->lv[lc];
    const int64_t m = c.n_nodes * D;
    h->m = m;
    h->A64 = h->op.alloc<double>(m * m);
    h->cb = h->op.alloc<double>(m * M);
    h->cu = h->op.alloc<double>(m * M);
    h->cb32 = h->op.alloc<float>(m * M);
    GMT_CUDA(cudaMemsetAsync(h->A64, 0, m * m * sizeof(double), s));
    k_coarse_assemble<<<grid_for(c.n_nodes * 27, 128), 128, 0, s>>>(
        D, lc, c.n, c.nbx, c.brick_xyz, c.brick_map, c.dense, c.eflag, c.canon_slot, c.slot_canon,
        op_kidx(c), c.K64, h->Ke64, lc == 0 && h->dens ? h->coef64 : nullptr, c.n_nodes, m,
        h->A64);
    GMT_LAUNCH_CHECK();
    double* ds = tmp.alloc<double>(2);
    k_diag_sum<<<1, 1024, 0, s>>>(h->A64, m, ds);
    GMT_LAUNCH_CHECK();
    h->cscal = h->op.alloc<double>(3);
    k_coarse_scalars<<<1, 1, 0, s>>>(ds, m, c.n_nodes, h->cscal);
    GMT_LAUNCH_CHECK();
    k_add_rho<<<grid_for(m * m, 256), 256, 0, s>>>(h->A64, m, D, h->cscal);
    GMT_LAUNCH_CHECK();
    // FP32 generalized inverse for the mixed-precision solves
    h->X32 = h->op.alloc<float>(m * m);
    k_to_f32<<<grid_for(m * m, 256), 256, 0, s>>>(h->A64, h->X32, m * m);
    GMT_LAUNCH_CHECK();
    gauss_jordan<float>(h, h->X32, m, h->cscal + 1, tmp);
  }
  GMT_CUDA(cudaStreamSynchronize(s));
  h->prepared = true;
}

// Element densities (App. F.3 SIMP): s_e = rho_min + rho_e^p per level-0 element, stored at
// the slot of the element's origin; rho == nullptr returns to the binary design. The
// operators are rebuilt on the next gmt_prepare / gmt_solve.
void set_densities(gmt_hierarchy* h, const double* rho, bool on_device, double rho_min,
                   double p) {
  cudaStream_t s = h->stream;
  free_workspace(h);
  h->have_solution = false;
  h->prepared = false;
  h->dn.release();
  h->coef64 = nullptr;
  h->coef32 = nullptr;
  h->rho64 = nullptr;
  h->dens = false;
  if (!rho) return;
  const Level& l0 = h->lv[0];
  const int64_t ne = l0.n_elems;
  std::vector<double> hr((size_t)ne);
  GMT_CUDA(cudaMemcpyAsync(hr.data(), rho, ne * sizeof(double),
                           on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
  GMT_CUDA(cudaStreamSynchronize(s));
  double cs = 0.0, cs2 = 0.0;
  for (int64_t e = 0; e < ne; ++e) {
    const double r = hr[(size_t)e];
    GMT_REQUIRE(r >= 0.0 && r <= 1.0, GMT_ERR_ARG, "density of element %lld is %g, not in [0, 1]",
                (long long)e, r);
    const double c = rho_min + std::pow(r, p);
    GMT_REQUIRE(c > 0.0, GMT_ERR_ARG,
                "element %lld has a zero coefficient (rho_min = 0 and rho = 0)", (long long)e);
    cs += c;
    cs2 += c * c;
  }
  h->coef64 = h->dn.alloc<double>(l0.nslots);
  h->coef32 = h->dn.alloc<float>(l0.nslots);
  h->rho64 = h->dn.alloc<double>(l0.nslots);
  GMT_CUDA(cudaMemsetAsync(h->coef64, 0, l0.nslots * sizeof(double), s));
  GMT_CUDA(cudaMemsetAsync(h->coef32, 0, l0.nslots * sizeof(float), s));
  GMT_CUDA(cudaMemsetAsync(h->rho64, 0, l0.nslots * sizeof(double), s));
  double* rd = h->dn.alloc<double>(ne);
  GMT_CUDA(cudaMemcpyAsync(rd, hr.data(), ne * sizeof(double), cudaMemcpyHostToDevice, s));
  k_set_density<<<grid_for(ne, 256), 256, 0, s>>>(ne, l0.elem_slot, rd, rho_min, p, h->coef64,
                                                  h->coef32, h->rho64);
  GMT_LAUNCH_CHECK();
  GMT_CUDA(cudaStreamSynchronize(s));
  h->rho_min = rho_min;
  h->simp_p = p;
  h->coef_sum = cs;
  h->coef_sum2 = cs2;
  h->dens = true;
}

}  // namespace gmt
