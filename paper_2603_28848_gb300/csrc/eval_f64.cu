// FP64 instantiations of the sample kernel (the parity path).
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<double, 4>(EvalParams);
template __global__ void eval_kernel<double, 5>(EvalParams);
template __global__ void eval_kernel<double, 6>(EvalParams);

void* eval_kernel_ptr_f64(int nmax) {
    switch (nmax) {
        case 3: case 4: return reinterpret_cast<void*>(&eval_kernel<double, 4>);
        case 5: return reinterpret_cast<void*>(&eval_kernel<double, 5>);
        default: return reinterpret_cast<void*>(&eval_kernel<double, 6>);
    }
}
}  // namespace best
