// Kernel tables and kernel spectra (FP64, one-off per plan).
//
// For a uniform patch of square cells the cell integrals of Section 2 depend
// only on the integer offset (m, n) = (source - target) / h:
//   K^{x,0}(m,n) = -dd ln(v + r)                      (scale-free)
//   K^{x,x}(m,n) = -m h K^{x,0} + dd[v ln(u + r)]     (proportional to h)
//   K^{x,y}(m,n) = -n h K^{x,0} - dd r
//   K^{y,.}(m,n) = K^{x,.}(n,m) with x and y exchanged
// over the cell u in [(m-1/2)h, (m+1/2)h], v in [(n-1/2)h, (n+1/2)h].
//
// The tables are evaluated in FP64 from algebraically identical forms that
// avoid cancellation at large offsets: ln(v + r) - ln|u| = asinh(v/|u|), whose
// u-independent part cancels in the double difference, and first differences
//   asinh(a) - asinh(b) = asinh((a - b)(a + b) / (a sqrt(1 + b^2) + b sqrt(1 + a^2)))   (a >= b >= 0)
//   r(u2, v) - r(u1, v) = (u2 - u1)(u2 + u1) / (r(u2, v) + r(u1, v))
// so that only the outer difference cancels. Parities (K^{x,0} odd in m and
// even in n, K^{x,x} even-even, K^{x,y} odd-odd) are imposed exactly.
//
// Spectra: the correlation F[t] = sum_s q[s] K[s - t] is a convolution with
// Kr[e] = K[-e]; Kr is placed on the padded Px x Py grid (index e mod P, zero
// outside |m| <= nx-1, |n| <= ny-1) and transformed with the shared-memory FFT.
// By parity the transforms of the x0 and y0 tables are imaginary and the other
// four real, so pairs are packed into one complex transform and the planes
//   a = Im Kr^x0, b = Re Kr^xx, c = Re Kr^xy, d = Im Kr^y0, e = Re Kr^yy, f = Re Kr^yx
// are stored for kx in [0, Px/2], ky in [0, Py/2] (the rest follows by parity),
// scaled by G / (Px Py) and by h for the order-1 planes.
#include "common.cuh"
#include "fft.cuh"
#include "kmath.cuh"

#include <math.h>

// unit-cell tables for m, n >= 0 (parity applied by the caller)
struct k3 {
    double x0, xx, xy;
};

__device__ k3 unit_kernels_pos(int m, int n)
{
    k3 k;
    const double u1 = m - 0.5, u2 = m + 0.5, v1 = n - 0.5, v2 = n + 0.5;
    // K^{x,0} = -dd asinh(v/|u|) = Dv(u1) - Dv(u2), Dv(u) = asinh(v2/u) - asinh(v1/u)
    if (m == 0) {
        k.x0 = 0.0;
    } else {
        k.x0 = asinh_span(v1, v2, u1) - asinh_span(v1, v2, u2);
    }
    // dd[v asinh(u/|v|)] = v2 Du(v2) - v1 Du(v1), Du(v) = asinh(u2/|v|) - asinh(u1/|v|)
    const double psi = v2 * asinh_span(u1, u2, fabs(v2)) - v1 * asinh_span(u1, u2, fabs(v1));
    k.xx = -(double)m * k.x0 + psi;
    // dd r = Dr(v2) - Dr(v1), Dr(v) = r(u2,v) - r(u1,v) = (u2 + u1) / (r(u2,v) + r(u1,v))
    if (m == 0 || n == 0) {
        k.xy = 0.0;
    } else {
        const double r22 = sqrt(u2 * u2 + v2 * v2), r12 = sqrt(u1 * u1 + v2 * v2);
        const double r21 = sqrt(u2 * u2 + v1 * v1), r11 = sqrt(u1 * u1 + v1 * v1);
        const double ddr = (u2 + u1) / (r22 + r12) - (u2 + u1) / (r21 + r11);
        k.xy = -(double)n * k.x0 - ddr;
    }
    return k;
}

// All six unit-h kernels at offset (m, n).
__device__ void unit_kernels(int m, int n, double *out6)
{
    const int am = m < 0 ? -m : m, an = n < 0 ? -n : n;
    const double sm = m < 0 ? -1.0 : 1.0, sn = n < 0 ? -1.0 : 1.0;
    k3 a = unit_kernels_pos(am, an);   // x-family at (|m|, |n|)
    k3 b = unit_kernels_pos(an, am);   // x-family at (|n|, |m|) -> y-family at (m, n)
    out6[0] = sm * a.x0;               // K^{x,0}: odd in m, even in n
    out6[1] = a.xx;                    // K^{x,x}: even-even
    out6[2] = sm * sn * a.xy;          // K^{x,y}: odd-odd
    out6[3] = sn * b.x0;               // K^{y,0}(m,n) = K^{x,0}(n,m)
    out6[4] = sm * sn * b.xy;          // K^{y,x}(m,n) = K^{x,y}(n,m)
    out6[5] = b.xx;                    // K^{y,y}(m,n) = K^{x,x}(n,m)
}

// ---- off the plane: unit-h kernels at height zeta = z / h != 0 ----
//   K^{x,0} = -dd asinh(v / rho_u),  rho_u = sqrt(u^2 + zeta^2)
//   K^{x,x} = -m K^{x,0} + dd[v asinh(u / rho_v)] - |zeta| dd atan(u v / (|zeta| r))
//   K^{x,y} = -n K^{x,0} - dd r,  r = sqrt(u^2 + v^2 + zeta^2)
//   K^{z,0} = -sgn(zeta) dd atan(u v / (|zeta| r)),  K^{z,x} = -m K^{z,0} - zeta K^{x,0}
// (the u-only and v-only parts of ln(v + r) and v ln(u + r) cancel in the double
// differences, as in the plane).
struct k5 {
    double x0, xx, xy, z0, zx;
};

__device__ k5 unit_kernels_pos_z(int m, int n, double zeta)
{
    const double u1 = m - 0.5, u2 = m + 0.5, v1 = n - 0.5, v2 = n + 0.5;
    const double z2 = zeta * zeta, az = fabs(zeta);
    k5 k;
    k.x0 = m == 0 ? 0.0 : asinh_span(v1, v2, sqrt(u1 * u1 + z2)) - asinh_span(v1, v2, sqrt(u2 * u2 + z2));
    const double r22 = sqrt(u2 * u2 + v2 * v2 + z2), r12 = sqrt(u1 * u1 + v2 * v2 + z2);
    const double r21 = sqrt(u2 * u2 + v1 * v1 + z2), r11 = sqrt(u1 * u1 + v1 * v1 + z2);
    const double solid = atan(u2 * v2 / (az * r22)) - atan(u1 * v2 / (az * r12)) - atan(u2 * v1 / (az * r21)) +
                         atan(u1 * v1 / (az * r11));
    const double psi = v2 * asinh_span(u1, u2, sqrt(v2 * v2 + z2)) - v1 * asinh_span(u1, u2, sqrt(v1 * v1 + z2));
    k.xx = -(double)m * k.x0 + psi - az * solid;
    if (m == 0 || n == 0) {
        k.xy = 0.0;
    } else {
        const double ddr = (u2 + u1) / (r22 + r12) - (u2 + u1) / (r21 + r11);
        k.xy = -(double)n * k.x0 - ddr;
    }
    k.z0 = (zeta > 0.0 ? -1.0 : 1.0) * solid;
    k.zx = -(double)m * k.z0 - zeta * k.x0;
    return k;
}

// All nine unit-h kernels at offset (m, n), height zeta:
// x0 xx xy y0 yx yy z0 zx zy.
__device__ void unit_kernels_z(int m, int n, double zeta, double *out9)
{
    const int am = m < 0 ? -m : m, an = n < 0 ? -n : n;
    const double sm = m < 0 ? -1.0 : 1.0, sn = n < 0 ? -1.0 : 1.0;
    k5 a = unit_kernels_pos_z(am, an, zeta);
    k5 b = unit_kernels_pos_z(an, am, zeta);
    out9[0] = sm * a.x0;
    out9[1] = a.xx;
    out9[2] = sm * sn * a.xy;
    out9[3] = sn * b.x0;
    out9[4] = sm * sn * b.xy;
    out9[5] = b.xx;
    out9[6] = a.z0;          // even in m and n
    out9[7] = sm * a.zx;     // odd in m, even in n
    out9[8] = sn * b.zx;     // even in m, odd in n
}

// ---- the mid-plane potential (Section 2, K = 1/r): integrals over the unit cell
// [m-1/2, m+1/2] x [n-1/2, n+1/2] (target at the origin) of 1/r, (xbar - xc)/r and
// (ybar - yc)/r. From the antiderivatives u ln(v + r) + v ln(u + r), (v r + u^2 ln(v + r))/2
// and (u r + v^2 ln(u + r))/2, with the u-only (v-only) logarithm cancelled inside each
// difference as for the force:
//   P0 = u2 Dv(u2) - u1 Dv(u1) + v2 Du(v2) - v1 Du(v1)
//   Px = [v2 Ru(v2) - v1 Ru(v1) + u2^2 Dv(u2) - u1^2 Dv(u1)] / 2 - m P0
//   Py = [u2 Rv(u2) - u1 Rv(u1) + v2^2 Du(v2) - v1^2 Du(v1)] / 2 - n P0
// Dv(u) = asinh(v2/|u|) - asinh(v1/|u|), Du(v) likewise, Ru(v) = r(u2, v) - r(u1, v),
// Rv(u) = r(u, v2) - r(u, v1); terms whose prefactor is 0 are 0 (their limits), so every
// offset, the own cell included, is finite. P0 scales with h, Px and Py with h^2.
// (the closed forms themselves: unit_cell_potentials in kmath.cuh, at real offsets)
__device__ void unit_potentials(int m, int n, double *out3) { unit_cell_potentials((double)m, (double)n, out3); }

// Wrapped correlation tables of the potential packed as z0 = Pr^x + i Pr^y (both
// transforms imaginary by parity), z1 = Pr^0 (transform real), each [py][px].
__global__ void k_tables_wrapped_pot(double2 *z, int nx, int ny, int px, int py)
{
    const int64_t plane = (int64_t)px * py;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % px), b = (int)(e / px);
        const int ex = a < px / 2 ? a : a - px;
        const int ey = b < py / 2 ? b : b - py;
        const int m = -ex, n = -ey;  // Pr[e] = P[-e]
        double p3[3] = {0, 0, 0};
        if (m <= nx - 1 && m >= -(nx - 1) && n <= ny - 1 && n >= -(ny - 1)) unit_potentials(m, n, p3);
        z[e] = make_double2(p3[1], p3[2]);
        z[plane + e] = make_double2(p3[0], 0.0);
    }
}

// Quarter planes p = Re P^0, a = Im P^x, b = Im P^y (the potential's spectra),
// [kx][ky] with row stride sg_spec_stride(py), scaled by -G/(px py) times h (p) or h^2.
template <typename T>
__global__ void k_extract_pot(const double2 *z, T *planes, int px, int py, double scale0, double scale1)
{
    const int qx = px / 2 + 1, qy = py / 2 + 1, qs = sg_spec_stride(py);
    const int64_t plane = (int64_t)px * py, qplane = (int64_t)qx * qs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < qplane; e += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e / qs), ky = (int)(e % qs);
        if (ky >= qy) {
            for (int c = 0; c < 3; ++c) planes[c * qplane + e] = (T)0;
            continue;
        }
        const int64_t src = (int64_t)ky * px + kx;
        const double2 z0 = z[src], z1 = z[plane + src];
        // z0 = i a + i (i b) = -b + i a
        planes[0 * qplane + e] = (T)(scale0 * z1.x);
        planes[1 * qplane + e] = (T)(scale1 * z0.y);
        planes[2 * qplane + e] = (T)(-scale1 * z0.x);
    }
}

// Unwrapped table of one kernel, physical units, [(2ny-1)][(2nx-1)].
__global__ void k_table_unwrapped(double *out, int nx, int ny, double h, double zeta, int which)
{
    const int w = 2 * nx - 1, hgt = 2 * ny - 1;
    const int64_t total = (int64_t)w * hgt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(e % w), row = (int)(e / w);
        double k9[9];
        if (zeta == 0.0) unit_kernels(col - (nx - 1), row - (ny - 1), k9);
        else unit_kernels_z(col - (nx - 1), row - (ny - 1), zeta, k9);
        const double scale = (which == 0 || which == 3 || which == 6) ? 1.0 : h;
        out[e] = scale * k9[which];
    }
}

// Wrapped correlation kernels packed in pairs: z0 = Kr^x0 + i Kr^y0,
// z1 = Kr^xx + i Kr^xy, z2 = Kr^yy + i Kr^yx, each [py][px].
__global__ void k_tables_wrapped(double2 *z, int nx, int ny, int px, int py)
{
    const int64_t plane = (int64_t)px * py;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % px), b = (int)(e / px);
        const int ex = a < px / 2 ? a : a - px;
        const int ey = b < py / 2 ? b : b - py;
        const int m = -ex, n = -ey;  // Kr[e] = K[-e]
        double k6[6] = {0, 0, 0, 0, 0, 0};
        if (m <= nx - 1 && m >= -(nx - 1) && n <= ny - 1 && n >= -(ny - 1)) unit_kernels(m, n, k6);
        z[e] = make_double2(k6[0], k6[3]);
        z[plane + e] = make_double2(k6[1], k6[2]);
        z[2 * plane + e] = make_double2(k6[5], k6[4]);
    }
}

// Off the plane: five packed planes, z0..z2 as above and
// z3 = Kr^zx + i Kr^zy, z4 = Kr^z0.
__global__ void k_tables_wrapped_z(double2 *z, int nx, int ny, int px, int py, double zeta)
{
    const int64_t plane = (int64_t)px * py;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % px), b = (int)(e / px);
        const int ex = a < px / 2 ? a : a - px;
        const int ey = b < py / 2 ? b : b - py;
        const int m = -ex, n = -ey;  // Kr[e] = K[-e]
        double k9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (m <= nx - 1 && m >= -(nx - 1) && n <= ny - 1 && n >= -(ny - 1)) unit_kernels_z(m, n, zeta, k9);
        z[e] = make_double2(k9[0], k9[3]);
        z[plane + e] = make_double2(k9[1], k9[2]);
        z[2 * plane + e] = make_double2(k9[5], k9[4]);
        z[3 * plane + e] = make_double2(k9[7], k9[8]);
        z[4 * plane + e] = make_double2(k9[6], 0.0);
    }
}

// In-place complex FFT along rows (stride 1) or columns (stride = row length)
// of `count` sequences of length L, one sequence per CTA, FP64.
template <int L>
__global__ void __launch_bounds__(L / 8 >= 64 ? L / 8 : 64) k_fft_lines(double2 *data, int64_t seq_stride, int64_t elem_stride,
                                                                          const double2 *__restrict__ tw)
{
    constexpr int THREADS = L / 8 >= 64 ? L / 8 : 64;
    extern __shared__ double2 buf[];
    double2 *base = data + blockIdx.x * seq_stride;
    for (int k = threadIdx.x; k < L; k += THREADS) buf[spad<double2>(k)] = base[k * elem_stride];
    __syncthreads();
    fft_batch<double2, L, 1, THREADS, false>(buf, tw);
    for (int k = threadIdx.x; k < L; k += THREADS) base[k * elem_stride] = buf[spad<double2>(k)];
}

template <typename T>
__global__ void k_extract_spectra(const double2 *z, T *planes, int px, int py, double scale0, double scale1, int nplanes)
{
    const int qx = px / 2 + 1, qy = py / 2 + 1, qs = sg_spec_stride(py);
    const int64_t plane = (int64_t)px * py, qplane = (int64_t)qx * qs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < qplane; e += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e / qs), ky = (int)(e % qs);  // planes are [kx][ky], row stride qs
        if (ky >= qy) {
            for (int c = 0; c < nplanes; ++c) planes[c * qplane + e] = (T)0;
            continue;
        }
        const int64_t src = (int64_t)ky * px + kx;          // z is [ky][kx]
        const double2 z0 = z[src], z1 = z[plane + src], z2 = z[2 * plane + src];
        // z0 = Kx0^ + i Ky0^ = i a + i (i d) = -d + i a
        planes[0 * qplane + e] = (T)(scale0 * z0.y);   // a
        planes[3 * qplane + e] = (T)(-scale0 * z0.x);  // d
        // z1 = Kxx^ + i Kxy^ = b + i c ; z2 = Kyy^ + i Kyx^ = e + i f
        planes[1 * qplane + e] = (T)(scale1 * z1.x);   // b
        planes[2 * qplane + e] = (T)(scale1 * z1.y);   // c
        planes[4 * qplane + e] = (T)(scale1 * z2.x);   // e
        planes[5 * qplane + e] = (T)(scale1 * z2.y);   // f
        if (nplanes == 9) {
            // z3 = Kzx^ + i Kzy^ = i hh + i (i kk) = -kk + i hh ; z4 = Kz0^ = g
            const double2 z3 = z[3 * plane + src], z4 = z[4 * plane + src];
            planes[6 * qplane + e] = (T)(scale0 * z4.x);   // g
            planes[7 * qplane + e] = (T)(scale1 * z3.y);   // hh
            planes[8 * qplane + e] = (T)(-scale1 * z3.x);  // kk
        }
    }
}

// Compact stage table of a length-L transform: for each stage of span NS > 1
// and radix R, entries W_{NS R}^k = exp(-2 pi i k / (NS R)), k < NS.
__global__ void k_twiddles(double2 *tw64, float2 *tw32, int L)
{
    for (int ns = 8, off = 0; ns < L; off += ns, ns *= 8) {
        const int span = L / ns >= 8 ? 8 * ns : L;  // NS R
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += gridDim.x * blockDim.x) {
            double s, c;
            sincospi(-2.0 * (double)k / (double)span, &s, &c);
            tw64[off + k] = make_double2(c, s);
            tw32[off + k] = make_float2((float)c, (float)s);
        }
    }
}

sg_status sg_fft_lines_fp64(double2 *data, int L, int count, int64_t seq_stride, int64_t elem_stride,
                           const double2 *tw)
{
    switch (L) {
#define SG_CASE(LL)                                                                                           \
    case LL:                                                                                                  \
        SG_CUDA_TRY(cudaFuncSetAttribute(k_fft_lines<LL>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                         (int)(spad_size<double2>(LL) * sizeof(double2))));                   \
        k_fft_lines<LL><<<count, (LL / 8 >= 64 ? LL / 8 : 64), spad_size<double2>(LL) * sizeof(double2)>>>(   \
            data, seq_stride, elem_stride, tw);                                                               \
        break;
        SG_CASE(64) SG_CASE(128) SG_CASE(256) SG_CASE(512) SG_CASE(1024) SG_CASE(2048) SG_CASE(4096) SG_CASE(8192)
#undef SG_CASE
    default:
        return SG_EINVAL;
    }
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

// Compact twiddle tables (see fft.cuh): FP64 for every power of two in
// [SG_MIN_PAD, max_pad], then FP32 copies of each (read by FP32 plans).
sg_status sg_twiddles_build(sg_plan *plan)
{
    int64_t off = 0;
    for (int L = SG_MIN_PAD; L <= plan->max_pad; L <<= 1) {
        plan->tw64_off[sg_ilog2(L)] = off;
        off += ((int64_t)stage_table_size(L) * sizeof(double2) + 255) / 256 * 256;
    }
    for (int L = SG_MIN_PAD; L <= plan->max_pad; L <<= 1) {
        plan->tw32_off[sg_ilog2(L)] = off;
        off += ((int64_t)stage_table_size(L) * sizeof(float2) + 255) / 256 * 256;
    }
    SG_CUDA_TRY(cudaMalloc(&plan->twiddles, (size_t)off));
    plan->device_bytes += off;
    for (int L = SG_MIN_PAD; L <= plan->max_pad; L <<= 1) {
        double2 *t64 = (double2 *)((char *)plan->twiddles + plan->tw64_off[sg_ilog2(L)]);
        float2 *t32 = (float2 *)((char *)plan->twiddles + plan->tw32_off[sg_ilog2(L)]);
        k_twiddles<<<(L / 8 + 255) / 256, 256>>>(t64, t32, L);
        SG_CUDA_TRY(cudaGetLastError());
    }
    return SG_OK;
}

sg_status sg_tables_build(sg_plan *plan)
{
    // one temporary of the largest padded patch, three complex planes
    int64_t maxplane = 0;
    for (int p = 0; p < plan->npatches; ++p) {
        const sg_patch_dev &d = plan->pp[p].d;
        int64_t pl = (int64_t)d.px * d.py;
        if (plan->pp[p].spectra && pl > maxplane) maxplane = pl;
    }
    if (maxplane == 0) return SG_OK;
    const bool offplane = plan->geom.z != 0.0;
    const int npacked = offplane ? 5 : 3;
    double2 *z = nullptr;
    SG_CUDA_TRY(cudaMalloc(&z, (size_t)(npacked * maxplane * sizeof(double2))));
    sg_status st = SG_OK;
    for (int p = 0; p < plan->npatches && st == SG_OK; ++p) {
        sg_patch_plan &pp = plan->pp[p];
        if (!pp.spectra) continue;  // level convolutions keep no per-patch spectra
        const int px = pp.d.px, py = pp.d.py;
        const int64_t plane = (int64_t)px * py;
        if (offplane) k_tables_wrapped_z<<<1024, 256>>>(z, pp.d.nx, pp.d.ny, px, py, plan->geom.z / pp.d.h);
        else k_tables_wrapped<<<1024, 256>>>(z, pp.d.nx, pp.d.ny, px, py);
        if (cudaGetLastError() != cudaSuccess) { st = SG_ECUDA; break; }
        const double2 *twx = (const double2 *)((const char *)plan->twiddles + plan->tw64_off[sg_ilog2(px)]);
        const double2 *twy = (const double2 *)((const char *)plan->twiddles + plan->tw64_off[sg_ilog2(py)]);
        for (int q = 0; q < npacked && st == SG_OK; ++q) {
            double2 *zq = z + q * plane;
            st = sg_fft_lines_fp64(zq, px, py, px, 1, twx);       // rows
            if (st == SG_OK) st = sg_fft_lines_fp64(zq, py, px, 1, px, twy);   // columns
        }
        if (st != SG_OK) break;
        const double scale0 = plan->geom.G / ((double)px * (double)py);
        const double scale1 = scale0 * pp.d.h;
        const int nplanes = offplane ? 9 : 6;
        if (plan->prec == SG_FP64)
            k_extract_spectra<double><<<1024, 256>>>(z, (double *)pp.spectra, px, py, scale0, scale1, nplanes);
        else
            k_extract_spectra<float><<<1024, 256>>>(z, (float *)pp.spectra, px, py, scale0, scale1, nplanes);
        if (cudaGetLastError() != cudaSuccess) st = SG_ECUDA;
    }
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(z);
    if (st != SG_OK) return st;
    if (e != cudaSuccess) {
        sg_set_last_cuda_error(e, "sg_tables_build");
        return SG_ECUDA;
    }
    return SG_OK;
}

// Central-slope factors of a patch (see fftconv.cuh), in the plan precision:
//   ce1[kx] = e^{+2 pi i kx / Px} / 2h,  ce2[kx] = e^{-2 pi i nx kx / Px} / 2h
// for kx in [0, Px/2], and the same along y for ky in [0, Py) (re1, re2).
// Layout: pairs (e1, e2) per kx, then pairs (e1, e2) per ky, each entry
// complex (re, im): 4 T per index, so that a pair is one aligned 16-byte load
// in FP32 (the y pairs start at 4 qx T). The sine factor sin(2 pi k / P) / h of
// the spectral difference is twice the imaginary part of e1 (a power-of-two
// scaling of the same rounded value, so the kernels form it exactly).
template <typename T>
__global__ void k_phase(T *out, int nx, int ny, int px, int py, double h)
{
    const int qx = px / 2 + 1;
    T *ce1 = out, *ce2 = out + 2;
    T *re1 = out + 4 * qx, *re2 = re1 + 2;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < qx + py; k += gridDim.x * blockDim.x) {
        const bool col = k < qx;
        const int kk = col ? k : k - qx;
        const int P = col ? px : py, n = col ? nx : ny;
        double s1, c1, s2, c2;
        sincospi(2.0 * (double)kk / (double)P, &s1, &c1);
        // e^{-2 pi i n k / P}: reduce n k mod P first so the argument stays small
        sincospi(-2.0 * (double)(((long long)n * kk) % P) / (double)P, &s2, &c2);
        T *e1 = col ? ce1 : re1, *e2 = col ? ce2 : re2;
        e1[4 * kk] = (T)(c1 / (2.0 * h));
        e1[4 * kk + 1] = (T)(s1 / (2.0 * h));
        e2[4 * kk] = (T)(c2 / (2.0 * h));
        e2[4 * kk + 1] = (T)(s2 / (2.0 * h));
    }
}

sg_status sg_phase_build(sg_plan *plan)
{
    for (int p = 0; p < plan->npatches; ++p) {
        sg_patch_plan &pp = plan->pp[p];
        if (!pp.phase) continue;
        const sg_patch_dev &d = pp.d;
        const int n = d.px / 2 + 1 + d.py;
        if (plan->prec == SG_FP64)
            k_phase<double><<<(n + 255) / 256, 256>>>((double *)pp.phase, d.nx, d.ny, d.px, d.py, d.h);
        else
            k_phase<float><<<(n + 255) / 256, 256>>>((float *)pp.phase, d.nx, d.ny, d.px, d.py, d.h);
        SG_CUDA_TRY(cudaGetLastError());
    }
    return SG_OK;
}

sg_status sg_tables_copy(const sg_plan *plan, int patch, int which, double *host_out, size_t n)
{
    const int maxw = plan && plan->geom.z != 0.0 ? 8 : 5;
    if (!plan || !host_out || patch < 0 || patch >= plan->npatches || which < 0 || which > maxw) {
        sg_set_last_error_message("sg_kernel_tables: no such patch or table (0..5, and 6..8 for z != 0)");
        return SG_EINVAL;
    }
    const sg_patch_dev &d = plan->pp[patch].d;
    const size_t need = (size_t)(2 * d.nx - 1) * (size_t)(2 * d.ny - 1);
    if (n < need) return SG_EINVAL;
    double *tmp = nullptr;
    SG_CUDA_TRY(cudaMalloc(&tmp, need * sizeof(double)));
    k_table_unwrapped<<<1024, 256>>>(tmp, d.nx, d.ny, d.h, plan->geom.z / d.h, which);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(host_out, tmp, need * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        sg_set_last_cuda_error(e, "sg_kernel_tables");
        return SG_ECUDA;
    }
    return SG_OK;
}

// Potential spectra of patch p, built once (synchronous).
static sg_status potential_spectra_patch(sg_plan *plan, int p)
{
    sg_patch_plan &pp = plan->pp[p];
    if (pp.pspectra) return SG_OK;
    const int px = pp.d.px, py = pp.d.py;
    const size_t es = plan->prec == SG_FP64 ? 8 : 4;
    const size_t bytes = 3 * (size_t)(px / 2 + 1) * sg_spec_stride(py) * es;
    const int64_t plane = (int64_t)px * py;
    double2 *z = nullptr;
    SG_CUDA_TRY(cudaMalloc(&z, (size_t)(2 * plane * sizeof(double2))));
    void *spec = nullptr;
    cudaError_t e = cudaMalloc(&spec, bytes);
    if (e != cudaSuccess) {
        cudaFree(z);
        cudaGetLastError();
        sg_set_last_cuda_error(e, "cudaMalloc");
        return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
    }
    k_tables_wrapped_pot<<<1024, 256>>>(z, pp.d.nx, pp.d.ny, px, py);
    sg_status st = cudaGetLastError() == cudaSuccess ? SG_OK : SG_ECUDA;
    const double2 *twx = (const double2 *)((const char *)plan->twiddles + plan->tw64_off[sg_ilog2(px)]);
    const double2 *twy = (const double2 *)((const char *)plan->twiddles + plan->tw64_off[sg_ilog2(py)]);
    for (int q = 0; q < 2 && st == SG_OK; ++q) {
        st = sg_fft_lines_fp64(z + q * plane, px, py, px, 1, twx);
        if (st == SG_OK) st = sg_fft_lines_fp64(z + q * plane, py, px, 1, px, twy);
    }
    const double scale0 = -plan->geom.G / ((double)px * (double)py) * pp.d.h;
    const double scale1 = scale0 * pp.d.h;
    if (st == SG_OK) {
        if (plan->prec == SG_FP64) k_extract_pot<double><<<1024, 256>>>(z, (double *)spec, px, py, scale0, scale1);
        else k_extract_pot<float><<<1024, 256>>>(z, (float *)spec, px, py, scale0, scale1);
        if (cudaGetLastError() != cudaSuccess) st = SG_ECUDA;
    }
    e = cudaDeviceSynchronize();
    cudaFree(z);
    if (st == SG_OK && e != cudaSuccess) {
        sg_set_last_cuda_error(e, "sg_potential");
        st = SG_ECUDA;
    }
    if (st != SG_OK) {
        cudaFree(spec);
        return st;
    }
    pp.pspectra = spec;
    plan->device_bytes += (int64_t)bytes;
    return SG_OK;
}

// Potential spectra of every patch (each patch's own convolution).
sg_status sg_potential_spectra_build(sg_plan *plan)
{
    for (int p = 0; p < plan->npatches; ++p) SG_TRY(potential_spectra_patch(plan, p));
    return SG_OK;
}
