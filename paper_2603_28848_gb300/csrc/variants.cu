// Sample-kernel variants per precision and leg count (for the autotuner).
#include "internal.cuh"

namespace best {
int eval_variants_f32_n4(SampleVariant* v);
int eval_variants_f32_n6(int nmax, SampleVariant* v);
int eval_variants_f64(int nmax, SampleVariant* v);
int eval_variants_strat(bool f32, int nmax, SampleVariant* v);

int eval_variants(bool f32, int nmax, SampleVariant* v, bool strat) {
    if (strat) return eval_variants_strat(f32, nmax, v);
    if (!f32) return eval_variants_f64(nmax, v);
    if (nmax <= 4) return eval_variants_f32_n4(v);
    return eval_variants_f32_n6(nmax, v);
}

// The default (first) variant of each precision: 256 threads per CTA.
void* eval_kernel_ptr_f32(int nmax) {
    SampleVariant v[kMaxVariants];
    eval_variants(true, nmax, v, false);
    return v[0].fn;
}

void* eval_kernel_ptr_f64(int nmax) {
    SampleVariant v[kMaxVariants];
    eval_variants(false, nmax, v, false);
    return v[0].fn;
}
}  // namespace best
