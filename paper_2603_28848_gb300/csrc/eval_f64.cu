// FP64 instantiations of the sample kernel (the parity path).
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<double, 4, 1>(EvalParams);
template __global__ void eval_kernel<double, 5, 1>(EvalParams);
template __global__ void eval_kernel<double, 6, 1>(EvalParams);

int eval_variants_f64(int nmax, void** fn, int* mb) {
    switch (nmax) {
        case 3: case 4: fn[0] = reinterpret_cast<void*>(&eval_kernel<double, 4, 1>); break;
        case 5: fn[0] = reinterpret_cast<void*>(&eval_kernel<double, 5, 1>); break;
        default: fn[0] = reinterpret_cast<void*>(&eval_kernel<double, 6, 1>); break;
    }
    mb[0] = 1;
    return 1;
}
}  // namespace best
