// FP32 instantiations of the sample kernel for n_total 5 and 6 with one
// sample per lane per step, and with 128-thread CTAs.
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<float, 5, 3, false, 256, 1>(EvalParams);
template __global__ void eval_kernel<float, 6, 3, false, 256, 1>(EvalParams);
template __global__ void eval_kernel<float, 6, 6, false, 128, 2>(EvalParams);

int eval_variants_f32_n6_b(int nmax, SampleVariant* v) {
    if (nmax == 5) {
        v[0] = {reinterpret_cast<void*>(&eval_kernel<float, 5, 3, false, 256, 1>), 3, 256, 1};
        return 1;
    }
    v[0] = {reinterpret_cast<void*>(&eval_kernel<float, 6, 3, false, 256, 1>), 3, 256, 1};
    v[1] = {reinterpret_cast<void*>(&eval_kernel<float, 6, 6, false, 128, 2>), 6, 128, 2};
    return 2;
}
}  // namespace best
