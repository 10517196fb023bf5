// Sample-kernel variants per precision and leg count (for the autotuner).
#include "internal.cuh"

namespace best {
int eval_variants_f32_n4(void** fn, int* mb);
int eval_variants_f32_n6(int nmax, void** fn, int* mb);
int eval_variants_f64(int nmax, void** fn, int* mb);
int eval_variants_strat(bool f32, int nmax, void** fn, int* mb);

int eval_variants(bool f32, int nmax, void** fn, int* mb, bool strat) {
    if (strat) return eval_variants_strat(f32, nmax, fn, mb);
    if (!f32) return eval_variants_f64(nmax, fn, mb);
    if (nmax <= 4) return eval_variants_f32_n4(fn, mb);
    return eval_variants_f32_n6(nmax, fn, mb);
}

void* eval_kernel_ptr_f32(int nmax) {
    void* fn[4];
    int mb[4];
    eval_variants(true, nmax, fn, mb, false);
    return fn[0];
}

void* eval_kernel_ptr_f64(int nmax) {
    void* fn[4];
    int mb[4];
    eval_variants(false, nmax, fn, mb, false);
    return fn[0];
}
}  // namespace best
