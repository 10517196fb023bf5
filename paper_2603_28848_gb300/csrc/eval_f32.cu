// FP32 instantiations of the sample kernel (FP32 integrand, compensated
// FP32 per-thread sums, FP64 per-segment records).
#include "eval_impl.cuh"

namespace best {
template __global__ void eval_kernel<float, 4>(EvalParams);
template __global__ void eval_kernel<float, 5>(EvalParams);
template __global__ void eval_kernel<float, 6>(EvalParams);

void* eval_kernel_ptr_f32(int nmax) {
    switch (nmax) {
        case 3: case 4: return reinterpret_cast<void*>(&eval_kernel<float, 4>);
        case 5: return reinterpret_cast<void*>(&eval_kernel<float, 5>);
        default: return reinterpret_cast<void*>(&eval_kernel<float, 6>);
    }
}
}  // namespace best
