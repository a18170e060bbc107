// Operator kernels with BF16 vectors and FP32 arithmetic (the BF16 V-cycle), for
// elasticity (3 dofs, 6 load cases) and heat conduction (1 dof, 3 load cases).
#include "stencil_op.cuh"

namespace gmt {

void stencil_elbf(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a) {
  stencil_t<__nv_bfloat16, float, 3, 6>(h, level, mode, a);
}
void stencil_heatbf(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a) {
  stencil_t<__nv_bfloat16, float, 1, 3>(h, level, mode, a);
}
void diag_elbf(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s) {
  diag_t<__nv_bfloat16, float, 3, 6>(h, level, f, out, dout, s);
}
void diag_heatbf(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s) {
  diag_t<__nv_bfloat16, float, 1, 3>(h, level, f, out, dout, s);
}

}  // namespace gmt
