// FP32-inner instances of the inner-step kernels: inner SpMV, Arnoldi update and fused step (FP32 values, basis and
// arithmetic).
#include "inner_step.cuh"

namespace sfg {

void inner_spmv_f32(const Plan& p, int i) { inner_spmv_t<float, float, float>(p, i, p.val32); }
bool inner_step_f32(const Plan& p, int i, bool last) { return inner_step_t<float, float, float>(p, i, p.val32, last); }
void inner_axpy_f32(const Plan& p, int i, bool last) { inner_axpy_t<float, float>(p, i, last); }

}  // namespace sfg
