// Operator kernels for heat conduction (1 dof, 3 load cases) with FP32 and FP64 vectors.
#include "stencil_op.cuh"

namespace gmt {

void stencil_heat32(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a) {
  stencil_t<float, float, 1, 3>(h, level, mode, a);
}
void stencil_heat64(gmt_hierarchy* h, int level, StencilMode mode, const VecArgs& a) {
  stencil_t<double, double, 1, 3>(h, level, mode, a);
}
void diag_heat32(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s) {
  diag_t<float, float, 1, 3>(h, level, f, out, dout, s);
}
void diag_heat64(gmt_hierarchy* h, int level, const void* f, void* out, void* dout, double s) {
  diag_t<double, double, 1, 3>(h, level, f, out, dout, s);
}
void resid_ff_heat(gmt_hierarchy* h, const float* hi, const float* lo, float* r, double* part) {
  resid_ff_t<1, 3>(h, hi, lo, r, part);
}

}  // namespace gmt
