// FP32 instantiations of the sample kernel (FP32 integrand, compensated
// FP32 per-thread sums, FP64 per-segment records) for n_total <= 4, one
// sample per lane per step, 256 threads, at several register budgets (CTAs
// per SM); eval_f32_b.cu has the other launch shapes, eval_f32_n6.cu and
// eval_f32_n6_b.cu n_total 5, 6.
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<float, 4, 3>(EvalParams);
template __global__ void eval_kernel<float, 4, 4>(EvalParams);
template __global__ void eval_kernel<float, 4, 5>(EvalParams);

int eval_variants_f32_n4_b(SampleVariant* v);

// Variants for n_total <= 4, in autotuner order; the first is the default.
int eval_variants_f32_n4(SampleVariant* v) {
    v[0] = {reinterpret_cast<void*>(&eval_kernel<float, 4, 5>), 5, 256, 1};
    v[1] = {reinterpret_cast<void*>(&eval_kernel<float, 4, 4>), 4, 256, 1};
    v[2] = {reinterpret_cast<void*>(&eval_kernel<float, 4, 3>), 3, 256, 1};
    return 3 + eval_variants_f32_n4_b(v + 3);
}
}  // namespace best
