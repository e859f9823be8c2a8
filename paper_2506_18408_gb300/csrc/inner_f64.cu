// FP64 instances of the inner-step kernels: inner SpMV (SELL-32 copy for one thread per row), Arnoldi update and
// fused step.
#include "inner_step.cuh"

namespace sfg {

void inner_spmv_f64(const Plan& p, int i) { inner_spmv_t<double, double, double>(p, i, p.val); }
bool inner_step_f64(const Plan& p, int i, bool last) { return inner_step_t<double, double, double>(p, i, p.val, last); }
void inner_axpy_f64(const Plan& p, int i, bool last) { inner_axpy_t<double, double>(p, i, last); }

}  // namespace sfg
