// Instantiations of the sample kernel that also run stratified (VEGAS+)
// tasks and s-dependent matrix elements; used by contexts with at least one
// such process.
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<float, 4, 4, true>(EvalParams);
template __global__ void eval_kernel<float, 4, 3, true>(EvalParams);
template __global__ void eval_kernel<float, 6, 2, true>(EvalParams);
template __global__ void eval_kernel<double, 4, 1, true>(EvalParams);
template __global__ void eval_kernel<double, 6, 1, true>(EvalParams);

int eval_variants_strat(bool f32, int nmax, SampleVariant* v) {
    if (!f32) {
        v[0] = {nmax <= 4 ? reinterpret_cast<void*>(&eval_kernel<double, 4, 1, true>)
                          : reinterpret_cast<void*>(&eval_kernel<double, 6, 1, true>), 1, 256, 1};
        return 1;
    }
    if (nmax <= 4) {
        v[0] = {reinterpret_cast<void*>(&eval_kernel<float, 4, 4, true>), 4, 256, 1};
        v[1] = {reinterpret_cast<void*>(&eval_kernel<float, 4, 3, true>), 3, 256, 1};
        return 2;
    }
    v[0] = {reinterpret_cast<void*>(&eval_kernel<float, 6, 2, true>), 2, 256, 1};
    return 1;
}
}  // namespace best
