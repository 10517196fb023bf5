// FP32 instantiations of the sample kernel (FP32 integrand, compensated
// FP32 per-thread sums, FP64 per-segment records), for n_total <= 4 at
// several register budgets (CTAs per SM); eval_f32_n6.cu has n_total 5, 6.
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<float, 4, 3>(EvalParams);
template __global__ void eval_kernel<float, 4, 4>(EvalParams);
template __global__ void eval_kernel<float, 4, 5>(EvalParams);

// Variants for n_total <= 4, in autotuner order; the first is the default.
int eval_variants_f32_n4(void** fn, int* mb) {
    fn[0] = reinterpret_cast<void*>(&eval_kernel<float, 4, 5>); mb[0] = 5;
    fn[1] = reinterpret_cast<void*>(&eval_kernel<float, 4, 4>); mb[1] = 4;
    fn[2] = reinterpret_cast<void*>(&eval_kernel<float, 4, 3>); mb[2] = 3;
    return 3;
}
}  // namespace best
