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

// s + x into the pair (s, c): TwoSum for the large parts, the rounding error into c
__device__ __forceinline__ void df_add(float& s, float& c, float x) {
    const float t = s + x;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (x - bp);
    s = t;
    c += err;
}

}  // namespace expm
