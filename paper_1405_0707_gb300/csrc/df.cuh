// df.cuh -- double-float (FP32 pair) helpers shared by the mixed-precision kernels.
#pragma once

namespace expm {

// v = hi + lo with hi = v truncated to 24 significant bits (exact as a float) and lo the
// remainder rounded to a float (relative error 2^-48 of v), built from the bit pattern with
// integer and FP32 operations only.  Values below 2^-74 in magnitude keep hi = (float)v.
__device__ __forceinline__ void split_df(double v, float& hi, float& lo) {
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 949 || e > 1150) {          // outside the range where the split is exact
        hi = (float)v;
        lo = 0.f;
        return;
    }
    hi = (float)__longlong_as_double(b & ~((1LL << 29) - 1));
    const float mag = (float)(int)(b & ((1LL << 29) - 1)) * __int_as_float((e - 1075 + 127) << 23);
    lo = (b < 0) ? -mag : mag;
}

// v rounded to a float (nearest, ties away from zero) with integer operations only: on GB300
// a double -> float conversion issues to the FP64 pipe (a small fraction of the FP32 rate,
// with a variable latency that stalls the dependent FP32 chain), so the bulk row kernels
// build the float from the bit pattern.  Magnitudes below 2^-126 flush to a signed zero;
// overflow gives inf and a NaN stays a NaN.  No branch reaches a hardware conversion.
__device__ __forceinline__ float f32_rn_i(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned f = ((unsigned)(e - 896) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu);
    unsigned r = sgn | (f + ((unsigned)(b >> 28) & 1u));                 // 897 <= e <= 1150
    if (e < 897) r = sgn;
    if (e > 1150) r = sgn | ((e == 2047 && (b & 0xFFFFFFFFFFFFFull)) ? 0x7FC00000u : 0x7F800000u);
    return __uint_as_float(r);
}

// The split of split_df with integer operations only: hi is v's sign, exponent and top 23
// stored mantissa bits; lo is the remaining 29-bit integer k rounded once to a float (an FMA
// of its top 23 bits times 2^6 plus its low 6 bits, each an exact float by the 2^23 trick)
// and scaled by 2^(e - 1075).  Equal to split_df's result for 2^-74 <= |v| < 2^127; outside,
// hi = f32_rn_i(v) and lo = 0.
__device__ __forceinline__ void split_df_i(double v, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned k = (unsigned)b & 0x1FFFFFFFu;
    const float top = __uint_as_float(0x4B000000u | (k >> 6)) - 8388608.f;
    const float low = __uint_as_float(0x4B000000u | (k & 63u)) - 8388608.f;
    const float mag = fmaf(top, 64.f, low) * __uint_as_float((unsigned)(e - 948) << 23);
    const bool in = e >= 949 && e <= 1150;
    hi = in ? __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu)) : f32_rn_i(v);
    lo = in ? __uint_as_float(__float_as_uint(mag) | sgn) : 0.f;
}

// s + x into the pair (s, c): TwoSum for the large parts, the rounding error into c
__device__ __forceinline__ void df_add(float& s, float& c, float x) {
    const float t = s + x;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (x - bp);
    s = t;
    c += err;
}

// exact float -> double from the bit pattern with integer operations only (a hardware
// float -> double conversion also issues to the FP64 pipe): normal floats, zeros, subnormals
// (normalised with a leading-zero count), inf and NaN.
__device__ __forceinline__ double f64_of_f32_i(float x) {
    const unsigned u = __float_as_uint(x), ex = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    const unsigned long long sg = (unsigned long long)(u >> 31) << 63;
    unsigned long long b = sg | ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)m << 29);
    if (ex == 0xFFu) b = sg | (0x7FFull << 52) | ((unsigned long long)m << 29);
    if (ex == 0u) {
        const int lead = 31 - __clz((int)(m | 1u));          // position of m's leading one
        const unsigned long long frac = ((unsigned long long)m << (52 - lead)) & 0xFFFFFFFFFFFFFull;
        b = m ? (sg | ((unsigned long long)(lead + 874) << 52) | frac) : sg;
    }
    return __longlong_as_double((long long)b);
}

// one double-float multiply-add: (sh, sl) += (vh + vl)(h1 + h2)
__device__ __forceinline__ void df_fma(float& sh, float& sl, float vh, float vl, float h1, float h2) {
    const float pr = vh * h1;
    float t = fmaf(vh, h1, -pr);
    t = fmaf(vl, h1, t);
    t = fmaf(vh, h2, t);
    df_add(sh, sl, pr);
    sl += t;
}

}  // namespace expm
