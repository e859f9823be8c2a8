// BF16-basis instances of the inner-step kernels: inner SpMV, Arnoldi update and fused step (FP32 values and
// arithmetic, the basis stored as BF16).
#include "inner_step.cuh"

namespace sfg {

void inner_spmv_bf16(const Plan& p, int i) { inner_spmv_t<float, __nv_bfloat16, float>(p, i, p.val32); }
bool inner_step_bf16(const Plan& p, int i, bool last) {
    return inner_step_t<float, __nv_bfloat16, float>(p, i, p.val32, last);
}
void inner_axpy_bf16(const Plan& p, int i, bool last) { inner_axpy_t<__nv_bfloat16, float>(p, i, last); }

}  // namespace sfg
