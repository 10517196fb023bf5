// Instantiations of the adjoint / tangent sample kernel with an s-dependent
// matrix element; used by contexts with such a process.
#include "vjp_impl.cuh"

namespace best {

template <bool JVP>
static void* me_ptr(bool f32, int nmax) {
    if (f32) return nmax <= 4 ? reinterpret_cast<void*>(&vjp_kernel<float, 4, JVP, true>)
                              : reinterpret_cast<void*>(&vjp_kernel<float, 6, JVP, true>);
    return nmax <= 4 ? reinterpret_cast<void*>(&vjp_kernel<double, 4, JVP, true>)
                     : reinterpret_cast<void*>(&vjp_kernel<double, 6, JVP, true>);
}

void* vjp_me_kernel_ptr(bool f32, int nmax, bool jvp) { return jvp ? me_ptr<true>(f32, nmax) : me_ptr<false>(f32, nmax); }

}  // namespace best
