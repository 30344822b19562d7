// Double-FP32 ("double-float") arithmetic for the FP32 pipe.
//
// A value is the unevaluated sum h + l of two FP32 numbers.  The operations
// are built from error-free transformations:
//   * TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2, Theorem B): s = fl(a + b) and
//     e = (a - (s - v)) + (b - v), v = s - a, satisfy s + e = a + b exactly;
//   * TwoProduct with a fused multiply-add: p = fl(a b) and
//     e = fma(a, b, -p) satisfy p + e = a b exactly (the FMA form of Dekker's
//     1971 product);
// and are kept unnormalised: the low word is not folded back below half an
// ulp of the high word after every step.  Each add rounds only the sum of the
// low words, each product only its cross terms, so a chain of k operations
// on values of magnitude M carries an absolute error of about k 2^-47 M --
// about 2^6 times the unit roundoff of FP64 instead of 2^29 for FP32.
//
// Conversions from FP64 split the 53-bit significand with integer
// operations and one FP32 subtraction (no FP64 or conversion instruction):
// h is the value truncated to 24 significant bits, l the remaining 29 bits
// rounded to 23 (relative error 2^-47 of the value).  Magnitudes below
// 2^-103 keep only h; below 2^-126 both words are zero.
//
// Every arithmetic step uses an explicit rounding intrinsic so that the
// compiler can neither contract nor reassociate it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace topo {

struct dfl {
    float h, l;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h_, float l_) : h(h_), l(l_) {}
    __host__ __device__ explicit dfl(double x);   // split, see df_from_double
};

__host__ __device__ __forceinline__ uint64_t dbl_bits(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}
__host__ __device__ __forceinline__ float flt_from_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}

// x = h + l + O(2^-47 |x|), see the header comment
__host__ __device__ __forceinline__ dfl df_from_double(double x) {
    const uint64_t b = dbl_bits(x);
    const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
    const int e = (int)((bh >> 20) & 0x7FFu);   // biased FP64 exponent
    const uint32_t sign = bh & 0x80000000u;
    dfl r(0.0f, 0.0f);
    if (e >= 897 && e <= 1150) {                // |x| in [2^-126, 2^128)
        r.h = flt_from_bits(sign | ((uint32_t)(e - 896) << 23) | ((bh & 0xFFFFFu) << 3) | (bl >> 29));
        // remainder m 2^(e - 1075) (same sign) as k 2^(e - 1069), k = m / 64
        // rounded (k <= 2^23): with B = 2^(e - 1046) the FP32 number
        // A = B + k 2^(e - 1069) is B's bit pattern plus k, and A - B is exact
        const uint32_t k = ((bl & 0x1FFFFFFFu) + 32u) >> 6;
        const uint32_t bB = sign | ((uint32_t)(e - 919) << 23);
        r.l = (e >= 920) ? flt_from_bits(bB + k) - flt_from_bits(bB) : 0.0f;
    } else if (e < 897) {                       // below the FP32 normal range
        r.h = 0.0f;
        r.l = 0.0f;
    } else {   // beyond the FP32 range: Inf of the sign, or NaN (integer operations only)
        const bool nan = e == 0x7FF && (((bh & 0xFFFFFu) | bl) != 0u);
        r.h = flt_from_bits(sign | 0x7F800000u | (nan ? 0x400000u : 0u));
        r.l = 0.0f;
    }
    return r;
}

__host__ __device__ __forceinline__ dfl::dfl(double x) : dfl(df_from_double(x)) {}

__host__ __device__ __forceinline__ double df_to_double(dfl a) { return (double)a.h + (double)a.l; }

#ifdef __CUDACC__
__device__ __forceinline__ float df_to_float(dfl a) { return __fadd_rn(a.h, a.l); }

// a + b: TwoSum of the high words, low words added with the rounding error
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
#ifdef TOPO_DF_PAIRED
    const float2 st = __fadd2_rn(make_float2(a.h, a.l), make_float2(b.h, b.l));   // s = a.h + b.h, t = a.l + b.l
    const float s = st.x, t = st.y;
#else
    const float s = __fadd_rn(a.h, b.h), t = __fadd_rn(a.l, b.l);
#endif
    const float v = __fsub_rn(s, a.h);
    const float p = __fsub_rn(s, v), q = __fsub_rn(b.h, v);
    const float e = __fadd_rn(__fsub_rn(a.h, p), q);
    return dfl{s, __fadd_rn(e, t)};
}
__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.h, -a.l}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
// a b: TwoProduct of the high words plus the cross terms (l_a l_b dropped)
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return dfl{p, e};
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) { return df_add(a, b); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return df_sub(a, b); }
__device__ __forceinline__ dfl operator-(dfl a) { return df_neg(a); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) { return df_mul(a, b); }
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) {
    a = df_add(a, b);
    return a;
}
#endif

}  // namespace topo
