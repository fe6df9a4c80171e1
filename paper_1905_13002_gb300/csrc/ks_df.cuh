// ks_df.cuh -- double-float arithmetic: a value carried as an unevaluated sum
// hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2), about 44 significant
// bits, with FP32's exponent range.
//
// Used for the few short dependent chains that want more than FP32 (the
// k = 1 filtering element: the prior's prediction and update), because a
// dependent FP64 operation on this part costs far more cycles than the
// handful of FP32 operations below.
//
// Methods (written from the published algorithms):
//   two_sum        Knuth's error-free addition (TAOCP vol. 2, 4.2.2);
//   quick_two_sum  Dekker's Fast2Sum (|a| >= |b|), Dekker 1971;
//   two_prod       the error-free product through a fused multiply-add;
//   add / mul      double-length addition and multiplication as in Dekker
//                  1971 and the double-double library of Hida, Li and
//                  Bailey (2001), with the error terms of both halves kept;
//   sqrt           Karp and Markstein's (1997) single Newton correction of an
//                  FP32 reciprocal square root;
//   recip          one Newton-Raphson correction of an FP32 reciprocal.
#pragma once

#include <cuda_runtime.h>

#ifndef KS_DEV
#define KS_DEV __device__ __forceinline__
#endif

namespace ks {

struct df {
    float hi, lo;
};

KS_DEV df df_make(float x) { return df{x, 0.f}; }

KS_DEV df df_make(double x) {
    const float h = __double2float_rn(x);
    return df{h, __double2float_rn(x - (double)h)};
}

KS_DEV float df_float(df a) { return a.hi + a.lo; }

KS_DEV df quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return df{s, b - (s - a)};
}

KS_DEV df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return df{s, (a - (s - bb)) + (b - bb)};
}

KS_DEV df two_prod(float a, float b) {
    const float p = a * b;
    return df{p, fmaf(a, b, -p)};
}

KS_DEV df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

KS_DEV df df_neg(df a) { return df{-a.hi, -a.lo}; }

KS_DEV df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

KS_DEV df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}

// c + a b
KS_DEV df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

// 1 / a for a != 0: x = 1/a.hi, then x + x (1 - a x).
KS_DEV df df_recip(df a) {
    const float x = 1.0f / a.hi;
    const df r = df_sub(df_make(1.0f), df_mul(a, df_make(x)));
    return df_add(df_make(x), df_mul(r, df_make(x)));
}

// sqrt(a) for a > 0 (0 otherwise): with x ~ 1/sqrt(a.hi) and s = a.hi x,
// sqrt(a) ~ s + (a - s^2) x / 2.
KS_DEV df df_sqrt(df a) {
    if (!(a.hi > 0.f)) return df{0.f, 0.f};
    const float x = rsqrtf(a.hi);
    const float s = a.hi * x;
    const df e = df_sub(a, two_prod(s, s));
    return df_add(df_make(s), df_make(e.hi * (0.5f * x)));
}

}  // namespace ks
