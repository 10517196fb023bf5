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

int eval_variants_strat(bool f32, int nmax, void** fn, int* mb) {
    if (!f32) {
        fn[0] = nmax <= 4 ? reinterpret_cast<void*>(&eval_kernel<double, 4, 1, true>)
                          : reinterpret_cast<void*>(&eval_kernel<double, 6, 1, true>);
        mb[0] = 1;
        return 1;
    }
    if (nmax <= 4) {
        fn[0] = reinterpret_cast<void*>(&eval_kernel<float, 4, 4, true>); mb[0] = 4;
        fn[1] = reinterpret_cast<void*>(&eval_kernel<float, 4, 3, true>); mb[1] = 3;
        return 2;
    }
    fn[0] = reinterpret_cast<void*>(&eval_kernel<float, 6, 2, true>); mb[0] = 2;
    return 1;
}
}  // namespace best
