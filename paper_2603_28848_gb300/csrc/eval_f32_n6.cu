// FP32 instantiations of the sample kernel for n_total 5 and 6 with two
// samples per lane per step (packed FP32x2 arithmetic), 256 threads, at
// several register budgets (CTAs per SM); eval_f32_n6_b.cu has one sample per
// lane per step.
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<float, 5, 2, false, 256, 2>(EvalParams);
template __global__ void eval_kernel<float, 5, 3, false, 256, 2>(EvalParams);
template __global__ void eval_kernel<float, 6, 2, false, 256, 2>(EvalParams);
template __global__ void eval_kernel<float, 6, 3, false, 256, 2>(EvalParams);

int eval_variants_f32_n6_b(int nmax, SampleVariant* v);

int eval_variants_f32_n6(int nmax, SampleVariant* v) {
    if (nmax == 5) {
        v[0] = {reinterpret_cast<void*>(&eval_kernel<float, 5, 3, false, 256, 2>), 3, 256, 2};
        v[1] = {reinterpret_cast<void*>(&eval_kernel<float, 5, 2, false, 256, 2>), 2, 256, 2};
    } else {
        v[0] = {reinterpret_cast<void*>(&eval_kernel<float, 6, 3, false, 256, 2>), 3, 256, 2};
        v[1] = {reinterpret_cast<void*>(&eval_kernel<float, 6, 2, false, 256, 2>), 2, 256, 2};
    }
    return 2 + eval_variants_f32_n6_b(nmax, v + 2);
}
}  // namespace best
