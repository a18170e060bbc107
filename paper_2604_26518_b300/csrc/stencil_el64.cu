// Operator kernels for elasticity (3 dofs, 6 load cases) with FP64 vectors.
#include "stencil_op.cuh"

namespace gmt {

void stencil_el64(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a) {
  stencil_t<double, double, 3, 6>(h, level, mode, a);
}
void diag_el64(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s) {
  diag_t<double, double, 3, 6>(h, level, f, out, dout, s);
}

}  // namespace gmt
