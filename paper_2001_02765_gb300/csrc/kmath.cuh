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

// Potential integrals of the unit cell centred at (cx, cy), target at the origin:
// P^0 = integral of 1/r, P^x = integral of (xbar - cx)/r, P^y likewise, from the
// antiderivatives u ln(v + r) + v ln(u + r) (of 1/r) and (v r + u^2 ln(v + r))/2
// (of u/r), double-differenced over the corners u = cx -+ 1/2, v = cy -+ 1/2.
// Each logarithm carries a factor vanishing where it is singular, so the
// integrals are finite everywhere (the target's own cell included): those terms
// are 0 there. ln(v + r) differences along an edge are asinh differences.
static __device__ __forceinline__ void unit_cell_potentials(double cx, double cy, double out3[3])
{
    const double u1 = cx - 0.5, u2 = cx + 0.5, v1 = cy - 0.5, v2 = cy + 0.5;
    const double dv1 = u1 != 0.0 ? asinh_span(v1, v2, fabs(u1)) : 0.0;
    const double dv2 = u2 != 0.0 ? asinh_span(v1, v2, fabs(u2)) : 0.0;
    const double du1 = v1 != 0.0 ? asinh_span(u1, u2, fabs(v1)) : 0.0;
    const double du2 = v2 != 0.0 ? asinh_span(u1, u2, fabs(v2)) : 0.0;
    const double p0 = u2 * dv2 - u1 * dv1 + v2 * du2 - v1 * du1;
    const double r22 = sqrt(u2 * u2 + v2 * v2), r12 = sqrt(u1 * u1 + v2 * v2);
    const double r21 = sqrt(u2 * u2 + v1 * v1), r11 = sqrt(u1 * u1 + v1 * v1);
    const double ru2 = (u2 + u1) / (r22 + r12), ru1 = (u2 + u1) / (r21 + r11);  // r(u2,v) - r(u1,v)
    const double rv2 = (v2 + v1) / (r22 + r21), rv1 = (v2 + v1) / (r12 + r11);  // r(u,v2) - r(u,v1)
    out3[0] = p0;
    out3[1] = 0.5 * (v2 * ru2 - v1 * ru1 + u2 * u2 * dv2 - u1 * u1 * dv1) - cx * p0;
    out3[2] = 0.5 * (u2 * rv2 - u1 * rv1 + v2 * v2 * du2 - v1 * v1 * du1) - cy * p0;
}
