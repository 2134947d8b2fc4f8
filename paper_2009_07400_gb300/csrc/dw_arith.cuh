// Double-word arithmetic for the MD_DW kernels (k_force_dw.cu): a value is
// the unevaluated sum h + l of two FP32 numbers.  Written from the published
// error-free transformations:
//   two_sum      s + e = a + b exactly (Knuth, TAOCP vol. 2, Sec. 4.2.2);
//   fast_two_sum the same for |a| >= |b| in three operations (Dekker 1971);
//   two_prod     p + e = a b exactly, e = fma(a, b, -p);
//   dw_mul       product of double words: the exact product of the high
//                parts plus the two cross terms (the low x low term is below
//                2^-46 of the product), as in the double-word multiplication
//                of Joldes, Muller and Popescu (ACM TOMS 2017);
//   dw_add       exact sum of the high parts plus the low parts.
// Every operation rounds to nearest and nothing may be contracted or
// reassociated: device code uses the _rn intrinsics; the host build of these
// functions (the CPU test of their error bounds) needs IEEE binary32
// arithmetic with floating-point contraction off.
#pragma once

#include <cmath>

namespace mdk {
namespace dwa {

__host__ __device__ __forceinline__ float add_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ __forceinline__ float sub_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ __forceinline__ float mul_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ __forceinline__ float fma_rn(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

struct dw {
    float h, l;
};

__host__ __device__ __forceinline__ dw two_sum(float a, float b)
{
    const float s = add_rn(a, b);
    const float bv = sub_rn(s, a);
    const float av = sub_rn(s, bv);
    return {s, add_rn(sub_rn(a, av), sub_rn(b, bv))};
}

__host__ __device__ __forceinline__ dw fast_two_sum(float a, float b)
{
    const float s = add_rn(a, b);
    return {s, sub_rn(b, sub_rn(s, a))};
}

__host__ __device__ __forceinline__ dw two_prod(float a, float b)
{
    const float p = mul_rn(a, b);
    return {p, fma_rn(a, b, -p)};
}

__host__ __device__ __forceinline__ dw dw_mul(dw x, dw y)
{
    dw p = two_prod(x.h, y.h);
    p.l = fma_rn(x.h, y.l, fma_rn(x.l, y.h, p.l));
    return p;
}

__host__ __device__ __forceinline__ dw dw_add(dw x, dw y)
{
    dw s = two_sum(x.h, y.h);
    s.l = add_rn(s.l, add_rn(x.l, y.l));
    return s;
}

// (h + l)^2 for an exact high part h and a small low part l:
// h^2 exactly, plus (2h + l) l
__host__ __device__ __forceinline__ dw dw_sq_of(float h, float l)
{
    dw p = two_prod(h, h);
    p.l = fma_rn(fma_rn(2.f, h, l), l, p.l);
    return p;
}

// 1/a for a double word a (not necessarily normalised) from af = fl(a.h +
// a.l) and a seed y0 ~ 1/af: one FP32 Newton step y (2 - af y) (to about an
// ulp), then one step in double word, y (1 + e) with e = 1 - a y.
__host__ __device__ __forceinline__ dw dw_recip(dw a, float af, float y0)
{
    const float y = fma_rn(y0, fma_rn(-af, y0, 1.f), y0);
    const float e = fma_rn(-a.l, y, fma_rn(-a.h, y, 1.f));
    return {y, mul_rn(y, e)};
}

// 1/sqrt(a) from af = fl(a.h + a.l) and a seed y0 ~ 1/sqrt(af): one FP32
// Newton step y (3 - af y^2) / 2, then one in double word, y (1 + e / 2)
// with e = 1 - a y^2 (y^2 exact by two_prod).
__host__ __device__ __forceinline__ dw dw_rsqrt(dw a, float af, float y0)
{
    const float y = mul_rn(y0, fma_rn(-0.5f * mul_rn(af, y0), y0, 1.5f));
    const dw p = dw_mul(a, two_prod(y, y));
    const float e = sub_rn(sub_rn(1.f, p.h), p.l);
    return {y, mul_rn(y, 0.5f * e)};
}

}  // namespace dwa
}  // namespace mdk
