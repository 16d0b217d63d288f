// FP64 building blocks of the cell-integral tables (Section 2 closed forms).
#pragma once

#include <math.h>

// asinh(a) - asinh(b) for a >= b >= 0 given d = a - b computed without rounding loss:
//   asinh(a) - asinh(b) = asinh((a - b)(a + b) / (a sqrt(1 + b^2) + b sqrt(1 + a^2)))
static __device__ __forceinline__ double asinh_diff(double a, double b, double d)
{
    return asinh(d * (a + b) / (a * sqrt(1.0 + b * b) + b * sqrt(1.0 + a * a)));
}

// asinh(t2 / s) - asinh(t1 / s), t2 - t1 = 1, s > 0.
static __device__ __forceinline__ double asinh_span(double t1, double t2, double s)
{
    if (t1 >= 0.0) return asinh_diff(t2 / s, t1 / s, 1.0 / s);
    if (t2 <= 0.0) return asinh_diff(-t1 / s, -t2 / s, 1.0 / s);
    return asinh(t2 / s) + asinh(-t1 / s);
}
