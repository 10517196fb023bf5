// FP64 instantiations of the sample kernel (the parity path).
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<double, 4, 1>(EvalParams);
template __global__ void eval_kernel<double, 5, 1>(EvalParams);
template __global__ void eval_kernel<double, 6, 1>(EvalParams);

int eval_variants_f64(int nmax, SampleVariant* v) {
    void* fn;
    switch (nmax) {
        case 3: case 4: fn = reinterpret_cast<void*>(&eval_kernel<double, 4, 1>); break;
        case 5: fn = reinterpret_cast<void*>(&eval_kernel<double, 5, 1>); break;
        default: fn = reinterpret_cast<void*>(&eval_kernel<double, 6, 1>); break;
    }
    v[0] = {fn, 1, 256, 1};
    return 1;
}
}  // namespace best
