// FP32 instantiations of the sample kernel for n_total <= 4 with the other
// launch shapes the autotuner tries: two samples per lane per step (packed
// FP32x2 arithmetic) and CTAs of 128 and 512 threads.
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<float, 4, 4, false, 256, 2>(EvalParams);
template __global__ void eval_kernel<float, 4, 10, false, 128, 1>(EvalParams);
template __global__ void eval_kernel<float, 4, 2, false, 512, 1>(EvalParams);

int eval_variants_f32_n4_b(SampleVariant* v) {
    v[0] = {reinterpret_cast<void*>(&eval_kernel<float, 4, 4, false, 256, 2>), 4, 256, 2};
    v[1] = {reinterpret_cast<void*>(&eval_kernel<float, 4, 10, false, 128, 1>), 10, 128, 1};
    v[2] = {reinterpret_cast<void*>(&eval_kernel<float, 4, 2, false, 512, 1>), 2, 512, 1};
    return 3;
}
}  // namespace best
