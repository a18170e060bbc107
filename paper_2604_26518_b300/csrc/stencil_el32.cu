// Operator kernels for elasticity (3 dofs, 6 load cases) with FP32 vectors.
#include "stencil_op.cuh"

namespace gmt {

void stencil_el32(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a) {
  stencil_t<float, float, 3, 6>(h, level, mode, a);
}
void diag_el32(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s) {
  diag_t<float, float, 3, 6>(h, level, f, out, dout, s);
}
void resid_ff_el(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part) {
  resid_ff_t<3, 6>(h, hi, lo, r, part);
}

}  // namespace gmt
