// FP32 instantiations of the sample kernel for n_total 5 and 6 at several
// register budgets (CTAs per SM).
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<float, 5, 2>(EvalParams);
template __global__ void eval_kernel<float, 5, 3>(EvalParams);
template __global__ void eval_kernel<float, 6, 2>(EvalParams);
template __global__ void eval_kernel<float, 6, 3>(EvalParams);

int eval_variants_f32_n6(int nmax, void** fn, int* mb) {
    if (nmax == 5) {
        fn[0] = reinterpret_cast<void*>(&eval_kernel<float, 5, 2>); mb[0] = 2;
        fn[1] = reinterpret_cast<void*>(&eval_kernel<float, 5, 3>); mb[1] = 3;
    } else {
        fn[0] = reinterpret_cast<void*>(&eval_kernel<float, 6, 2>); mb[0] = 2;
        fn[1] = reinterpret_cast<void*>(&eval_kernel<float, 6, 3>); mb[1] = 3;
    }
    return 2;
}
}  // namespace best
