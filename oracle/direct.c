/*
 * Plain FP64 direct summation of the thin-disk in-plane force (oracle).
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product path. Shares no code with
 * the CUDA library.
 *
 * For every target (tx[t], ty[t]) and every source cell [xl,xr]x[yd,yu] with
 * surface density sigma0 + deltax (xbar - xc) + deltay (ybar - yc) (the order-1
 * Taylor reconstruction of Section 2, Eq. eqnGamma), add
 *     G [sigma0 K^{x,0} + deltax K^{x,x} + deltay K^{x,y}]   to fx[t]
 *     G [sigma0 K^{y,0} + deltax K^{y,x} + deltay K^{y,y}]   to fy[t]
 * with the closed-form cell integrals of Section 2 at z = 0:
 *     K^{x,0} = -dd ln(v + r),  K^{x,x} = (x - xc) K^{x,0} + dd[v ln(u + r)],
 *     K^{x,y} = (y - yc) K^{x,0} - dd r,  and the y-family with u <-> v,
 * where u = xbar - x, v = ybar - y, r = sqrt(u^2 + v^2) and dd is the double
 * difference over the four cell corners. Where u == 0 the paper's coincident-line
 * form sgn(v) ln|v| replaces ln(v + r) (and sgn(u) ln|u| replaces ln(u + r)
 * where v == 0). For v < 0, ln(v + r) is evaluated as 2 ln|u| - ln(r - v),
 * the same number without the cancellation.
 *
 * A target on a source corner or strictly inside a source edge span is a
 * log-divergent integral; such a pair sets *status = 1 and contributes 0.
 */
#include <math.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ln(s + sqrt(t^2 + s^2)) with sgn(s) ln|s| on the line t == 0. */
static double ln_s_plus_r(double t, double s, int *bad)
{
    if (t == 0.0) {
        if (s == 0.0) { *bad = 1; return 0.0; }
        return s > 0.0 ? log(s) : -log(-s);
    }
    double r = sqrt(t * t + s * s);
    if (s >= 0.0) return log(s + r);
    return 2.0 * log(fabs(t)) - log(r - s);
}

typedef struct { double x0, xx, xy, y0, yx, yy; } kern6;

static kern6 cell_kernels(double x, double y, double xl, double xr, double yd, double yu, int *bad)
{
    double us[2] = { xl - x, xr - x };
    double vs[2] = { yd - y, yu - y };
    kern6 k = { 0, 0, 0, 0, 0, 0 };
    if (((us[0] == 0.0) || (us[1] == 0.0)) && vs[0] < 0.0 && vs[1] > 0.0) { *bad = 1; return k; }
    if (((vs[0] == 0.0) || (vs[1] == 0.0)) && us[0] < 0.0 && us[1] > 0.0) { *bad = 1; return k; }
    double ddl_v = 0.0, ddl_u = 0.0, dd_vlu = 0.0, dd_ulv = 0.0, dd_r = 0.0;
    for (int a = 0; a < 2; ++a) {
        for (int b = 0; b < 2; ++b) {
            /* corner sign of the double difference: + at (u2,v2) and (u1,v1) */
            double sgn = (a == b) ? 1.0 : -1.0;
            double u = us[a], v = vs[b];
            double lv = ln_s_plus_r(u, v, bad);   /* ln(v + r) */
            double lu = ln_s_plus_r(v, u, bad);   /* ln(u + r) */
            ddl_v += sgn * lv;
            ddl_u += sgn * lu;
            dd_vlu += sgn * (v == 0.0 ? 0.0 : v * lu);
            dd_ulv += sgn * (u == 0.0 ? 0.0 : u * lv);
            dd_r += sgn * sqrt(u * u + v * v);
        }
    }
    double xc = 0.5 * (xl + xr), yc = 0.5 * (yd + yu);
    k.x0 = -ddl_v;
    k.y0 = -ddl_u;
    k.xx = (x - xc) * k.x0 + dd_vlu;
    k.xy = (y - yc) * k.x0 - dd_r;
    k.yx = (x - xc) * k.y0 - dd_r;
    k.yy = (y - yc) * k.y0 + dd_ulv;
    return k;
}

/* Returns 0 on success, 1 if any pair was log-divergent (those pairs add 0). */
int oracle_direct_force(long ns, const double *xl, const double *xr, const double *yd, const double *yu,
                        const double *s0, const double *sx, const double *sy,
                        long nt, const double *tx, const double *ty, double G,
                        double *fx, double *fy, int nthreads)
{
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(| : status)
    for (long t = 0; t < nt; ++t) {
        double ax = 0.0, ay = 0.0;
        int bad = 0;
        for (long i = 0; i < ns; ++i) {
            int pair_bad = 0;
            kern6 k = cell_kernels(tx[t], ty[t], xl[i], xr[i], yd[i], yu[i], &pair_bad);
            if (pair_bad) { bad = 1; continue; }
            double a = s0[i], bx = sx ? sx[i] : 0.0, by = sy ? sy[i] : 0.0;
            ax += a * k.x0 + bx * k.xx + by * k.xy;
            ay += a * k.y0 + bx * k.yx + by * k.yy;
        }
        fx[t] = G * ax;
        fy[t] = G * ay;
        status |= bad;
    }
    return status;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Off the plane (targets at height z != 0; Section 2, the antiderivatives with
 * the arctan terms): with r = sqrt(u^2 + v^2 + z^2),
 *   K^{x,0} = -dd ln(v + r),  K^{x,x} = (x - xc) K^{x,0} + dd[v ln(u + r) - |z| atan(u v / (|z| r))],
 *   K^{x,y} = (y - yc) K^{x,0} - dd r, the y-family with u <-> v, and
 *   K^{z,0} = -dd atan(u v / (z r)),  K^{z,x} = (x - xc) K^{z,0} - z K^{x,0},
 *   K^{z,y} = (y - yc) K^{z,0} - z K^{y,0};
 * F = G sum_i [sigma0_i K^{.,0} + deltax_i K^{.,x} + deltay_i K^{.,y}] for . = x, y, z.
 */
static double ln_s_plus_rz(double t, double s, double z)
{
    double r = sqrt(t * t + s * s + z * z);
    if (s >= 0.0) return log(s + r);
    return log(t * t + z * z) - log(r - s);
}

int oracle_direct_force3(long ns, const double *xl, const double *xr, const double *yd, const double *yu,
                         const double *s0, const double *sx, const double *sy,
                         long nt, const double *tx, const double *ty, double z, double G,
                         double *fx, double *fy, double *fz, int nthreads)
{
    if (z == 0.0) return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const double az = fabs(z);
#pragma omp parallel for schedule(dynamic, 16)
    for (long t = 0; t < nt; ++t) {
        double ax = 0.0, ay = 0.0, azs = 0.0;
        for (long i = 0; i < ns; ++i) {
            double us[2] = { xl[i] - tx[t], xr[i] - tx[t] };
            double vs[2] = { yd[i] - ty[t], yu[i] - ty[t] };
            double ddlv = 0, ddlu = 0, ddvlu = 0, ddulv = 0, ddr = 0, ddat = 0;
            for (int a = 0; a < 2; ++a) {
                for (int b = 0; b < 2; ++b) {
                    double sgn = (a == b) ? 1.0 : -1.0;
                    double u = us[a], v = vs[b];
                    double r = sqrt(u * u + v * v + z * z);
                    double lv = ln_s_plus_rz(u, v, z);   /* ln(v + r) */
                    double lu = ln_s_plus_rz(v, u, z);   /* ln(u + r) */
                    ddlv += sgn * lv;
                    ddlu += sgn * lu;
                    ddvlu += sgn * v * lu;
                    ddulv += sgn * u * lv;
                    ddr += sgn * r;
                    ddat += sgn * atan(u * v / (az * r));
                }
            }
            double xc = 0.5 * (xl[i] + xr[i]), yc = 0.5 * (yd[i] + yu[i]);
            double kx0 = -ddlv, ky0 = -ddlu, kz0 = (z > 0 ? -1.0 : 1.0) * ddat;
            double kxx = (tx[t] - xc) * kx0 + ddvlu - az * ddat;
            double kxy = (ty[t] - yc) * kx0 - ddr;
            double kyx = (tx[t] - xc) * ky0 - ddr;
            double kyy = (ty[t] - yc) * ky0 + ddulv - az * ddat;
            double kzx = (tx[t] - xc) * kz0 - z * kx0;
            double kzy = (ty[t] - yc) * kz0 - z * ky0;
            double a0 = s0[i], bx = sx ? sx[i] : 0.0, by = sy ? sy[i] : 0.0;
            ax += a0 * kx0 + bx * kxx + by * kxy;
            ay += a0 * ky0 + bx * kyx + by * kyy;
            azs += a0 * kz0 + bx * kzx + by * kzy;
        }
        fx[t] = G * ax;
        fy[t] = G * ay;
        fz[t] = G * azs;
    }
    return 0;
}

/*
 * Mid-plane potential (Section 2, the singular kernel integral with K = 1/r):
 *   Phi(t) = -G sum_i [sigma0_i P0 + deltax_i Px + deltay_i Py],
 *   P0 = dd[u ln(v + r) + v ln(u + r)],
 *   Px = dd[(v r + u^2 ln(v + r)) / 2] + (x - xc) P0,   Py = dd[(u r + v^2 ln(u + r)) / 2] + (y - yc) P0,
 * every logarithm multiplied by a factor that vanishes where it is singular (0 there).
 */
static double lvr(double u, double v)   /* ln(v + sqrt(u^2 + v^2)), u != 0 */
{
    double r = sqrt(u * u + v * v);
    if (v >= 0.0) return log(v + r);
    return 2.0 * log(fabs(u)) - log(r - v);
}

int oracle_direct_potential(long ns, const double *xl, const double *xr, const double *yd, const double *yu,
                            const double *s0, const double *sx, const double *sy,
                            long nt, const double *tx, const double *ty, double G, double *phi, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (long t = 0; t < nt; ++t) {
        double acc = 0.0;
        for (long i = 0; i < ns; ++i) {
            double us[2] = { xl[i] - tx[t], xr[i] - tx[t] };
            double vs[2] = { yd[i] - ty[t], yu[i] - ty[t] };
            double p0 = 0.0, pu = 0.0, pv = 0.0;
            for (int a = 0; a < 2; ++a) {
                for (int b = 0; b < 2; ++b) {
                    double sgn = (a == b) ? 1.0 : -1.0;
                    double u = us[a], v = vs[b], r = sqrt(u * u + v * v);
                    double lv = u != 0.0 ? lvr(u, v) : 0.0;   /* ln(v + r), used with factor u */
                    double lu = v != 0.0 ? lvr(v, u) : 0.0;   /* ln(u + r), used with factor v */
                    p0 += sgn * (u * lv + v * lu);
                    pu += sgn * 0.5 * (v * r + u * u * lv);
                    pv += sgn * 0.5 * (u * r + v * v * lu);
                }
            }
            double xc = 0.5 * (xl[i] + xr[i]), yc = 0.5 * (yd[i] + yu[i]);
            double px = pu + (tx[t] - xc) * p0, py = pv + (ty[t] - yc) * p0;
            acc += s0[i] * p0 + (sx ? sx[i] * px : 0.0) + (sy ? sy[i] * py : 0.0);
        }
        phi[t] = -G * acc;
    }
    return 0;
}
