// Level convolutions: the whole AMR sum of Eq. eqnXforce2 (over the composite
// sources S_l of every level, see amr.cu) as FFT convolutions on the lattice of
// the finest cells, replacing the per-patch convolutions and the cross-patch
// direct sum.
//
// Let h_f be the finest cell width, lmax the finest level, and s = lmax - m the
// width exponent of level m (its cells are 2^s finest cells wide). A cell of
// level m with global index (i, j) is sampled at finest-lattice index
//   I = i 2^s + phi_s,  phi_s = 2^(s-1) for s >= 1, 0 for s = 0,
// whose centre lies half a finest cell up and right of the coarse cell's centre
// when s >= 1 (a coarse centre is a corner of the finest lattice). For a source
// on level m and a target on level l the offset of the source centre from the
// target centre is then (I_s - I_t) - d with d = f(s_m) - f(s_l), f(s) = 1/2 for
// s >= 1 and 0 for s = 0: one translation-invariant kernel per ordered level
// pair, evaluated at fractional offsets -e - d for lattice offsets e = I_t - I_s,
// for a source cell 2^s finest cells wide. The force on level l is the sum over
// source levels m of the convolutions of S_m's three fields with the six
// kernels, read at the level-l sample points.
//
// Pipeline per solve (after the composite sources): for every level, the row
// transforms of its sampled rows and the column transforms to full spectra; for
// every target level, a column kernel that sums sources x kernel spectra over
// all source levels and fields and inverse-transforms Fx, Fy at the target's
// sampled rows; then the inverse row transforms, written to the level's cells.
// Kernel spectra (six planes per distinct (s, d), FP64-built) depend only on
// the lattice, not on the density.
//
// Compact source spectra: a level of width exponent s has samples only every
// 2^s finest cells, so the transform of its sampled field repeats with period
// P / 2^c along an axis for any c <= s. Its row and column transforms run at
// length Pc = P / 2^c (c = s, or less where Pc would fall below 64 points),
// on compact positions p = I / 2^c. When c = s >= 1 these are half-integers
// (I = 2^s i + 2^(s-1)): the samples sit at integer positions q = p - 1/2 and
// the half shift is the factor psi(k) = exp(-i pi k / Pc). The full spectrum
// is then
//   F(kx, ky) = Ghat(kx mod Pcx, ky mod Pcy) psi_x(kx) psi_y(ky),
//   psi(k + r Pc) = (-1)^r psi(k)  (psi = 1 without the half shift),
// and the column pass stores Ghat psi over kx in [0, Pcx/2], ky in [0, Pcy).
// The column kernel reads the other half of the compact kx range from the
// Hermitian partner, Ghat(kx, ky) = conj Ghat(Pcx - kx, -ky mod Pcy), whose
// stored phase differs by a sign on every half-shifted axis (but not at
// ky = 0 on the y axis). This cuts the source spectra of a level by 4^c.
//
// Tables: the closed forms of Section 2 at a real-valued centre offset (cx, cy)
// in units of the cell width,
//   K^{x,0} = D(u1) - D(u2),  D(u) = asinh(v2/|u|) - asinh(v1/|u|), or on the line
//             u = 0 the coincident-line form sgn(v2) ln|v2| - sgn(v1) ln|v1|
//   K^{x,x} = -cx K^{x,0} + v2 G(v2) - v1 G(v1),  G(v) = asinh(u2/|v|) - asinh(u1/|v|)
//   K^{x,y} = -cy K^{x,0} - [R(v2) - R(v1)],  R(v) = (u2 + u1) / (r(u2, v) + r(u1, v))
// with u1,2 = cx -+ 1/2, v1,2 = cy -+ 1/2 (target at the origin); the y-family
// by exchanging x and y. Offsets where the integral diverges (the target on a
// source corner or strictly inside an edge span) get zero: for a leaf target
// and a source cell that carries density they cannot occur, since the cells of
// finer levels lie inside refined cells and a leaf's centre is inside the leaf.
#include "common.cuh"
#include "fft.cuh"
#include "kmath.cuh"

#include <math.h>
#include <string.h>

#include <new>
#include <vector>

namespace {

// --------------------------------------------------------------- tables --

__device__ __forceinline__ bool line_diff(double t1, double t2, double &out)
{
    // sgn(t2) ln|t2| - sgn(t1) ln|t1|; diverges when the span [t1, t2] holds 0
    if (t1 == 0.0 || t2 == 0.0 || (t1 < 0.0 && t2 > 0.0)) return false;
    out = (t2 > 0.0 ? log(t2) : -log(-t2)) - (t1 > 0.0 ? log(t1) : -log(-t1));
    return true;
}

// x-family of the unit cell centred at (cx, cy), target at the origin.
__device__ bool unit_x_family(double cx, double cy, double &x0, double &xx, double &xy)
{
    const double u1 = cx - 0.5, u2 = cx + 0.5, v1 = cy - 0.5, v2 = cy + 0.5;
    double d1, d2;
    if (u1 != 0.0) d1 = asinh_span(v1, v2, fabs(u1));
    else if (!line_diff(v1, v2, d1)) return false;
    if (u2 != 0.0) d2 = asinh_span(v1, v2, fabs(u2));
    else if (!line_diff(v1, v2, d2)) return false;
    x0 = d1 - d2;
    const double g2 = v2 != 0.0 ? v2 * asinh_span(u1, u2, fabs(v2)) : 0.0;
    const double g1 = v1 != 0.0 ? v1 * asinh_span(u1, u2, fabs(v1)) : 0.0;
    xx = -cx * x0 + (g2 - g1);
    const double r22 = sqrt(u2 * u2 + v2 * v2), r12 = sqrt(u1 * u1 + v2 * v2);
    const double r21 = sqrt(u2 * u2 + v1 * v1), r11 = sqrt(u1 * u1 + v1 * v1);
    const double ddr = (u2 + u1) / (r22 + r12) - (u2 + u1) / (r21 + r11);
    xy = -cy * x0 - ddr;
    return true;
}

// Packed wrapped tables of one kernel key: z0 = Kr^x0 + i Kr^y0, z1 = Kr^xx + i Kr^xy,
// z2 = Kr^yy + i Kr^yx, each [py][px], for a source cell w = 2^s finest cells wide
// and sample shift d = d2 / 2: Kr[e] = K(centre offset -e - d). The stored period
// is symmetric about e = -d, so that the compressed spectra below are exact.
__global__ void k_lv_tables(double2 *z, int px, int py, int s, int d2)
{
    const int64_t plane = (int64_t)px * py;
    const double w = (double)(1 << s), d = 0.5 * d2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % px), b = (int)(e / px);
        // wrap representatives symmetric about -d (offsets |e| = P/2 are never used):
        // [-P/2, P/2) for d >= 0, (-P/2, P/2] for d < 0, and zero at e = -P/2 for d = 0
        const int ex = d2 < 0 ? (a <= px / 2 ? a : a - px) : (a < px / 2 ? a : a - px);
        const int ey = d2 < 0 ? (b <= py / 2 ? b : b - py) : (b < py / 2 ? b : b - py);
        const double cx = (-ex - d) / w, cy = (-ey - d) / w;
        double x0 = 0, xx = 0, xy = 0, y0 = 0, yy = 0, yx = 0;
        if ((d2 == 0 && (ex == -px / 2 || ey == -py / 2)) || !unit_x_family(cx, cy, x0, xx, xy) ||
            !unit_x_family(cy, cx, y0, yy, yx)) {
            x0 = xx = xy = y0 = yy = yx = 0.0;
        }
        z[e] = make_double2(x0, y0);
        z[plane + e] = make_double2(w * xx, w * xy);
        z[2 * plane + e] = make_double2(w * yy, w * yx);
    }
}

// Kernel spectra are stored compressed. A table Kr(e) = K(-e - d) of parities
// (sx, sy) (+1 even, -1 odd in that coordinate of the source offset) is
// symmetric about e = -d along each axis, so its transform G satisfies
//   H(k) = G(k) exp(-i pi d2 (kx/Px + ky/Py)),  d2 = 2d in {-1, 0, 1},
//   H(kx, ky) = sx H(-kx, ky) = sy H(kx, -ky),  H real if sx sy = +1, imaginary if -1,
// and H is determined by kx, ky in [0, P/2]: G(kx, ky) = ph_x(kx) ph_y(ky) H(kx, ky) for
// ky <= Py/2 and sy ph_x(kx) ph_y(ky - Py) H(kx, Py - ky) above, ph(k) = exp(i pi d2 k / P).
// Planes x0 xx xy y0 yx yy have (sx, sy) = (-,+) (+,+) (-,-) (+,-) (-,-) (+,+); the
// imaginary ones (x0, y0) store Im H, the others Re H, [kx][ky] for kx in [0, px/2],
// ky in [0, py/2] (rows padded to sg_spec_stride(py) entries, 16-byte aligned for bulk
// copies), scaled by 1 / (px py) and by G (x0, y0) or G h_f (the order-1 planes).
__host__ __device__ constexpr bool lv_plane_imag(int p) { return p == 0 || p == 3; }

// Unpack the transforms of the packed pairs (A + i B: A^(k) = (Z(k) + conj Z(-k)) / 2,
// B^(k) = (Z(k) - conj Z(-k)) / 2i), remove the half-cell phase and keep the real
// or imaginary part of every plane.
template <typename T>
__global__ void k_lv_extract(const double2 *z, T *out, int px, int py, int d2, double sc0, double sc1)
{
    const int qx = px / 2 + 1, qy = py / 2 + 1, qs = sg_spec_stride(py);
    const int64_t plane = (int64_t)px * py, qplane = (int64_t)qx * qs;
    const double inv = 1.0 / ((double)px * (double)py);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < qplane; e += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e / qs), ky = (int)(e % qs);
        if (ky >= qy) {  // row padding
            for (int q = 0; q < 6; ++q) out[q * qplane + e] = (T)0;
            continue;
        }
        const int64_t ip = (int64_t)ky * px + kx;
        const int64_t im = (int64_t)((py - ky) % py) * px + (px - kx) % px;
        double sn, cs;  // exp(-i pi d2 (kx/px + ky/py))
        sincospi(-(double)d2 * ((double)kx / px + (double)ky / py), &sn, &cs);
        // destination planes of the A and B halves of each packed pair
        const int pa[3] = {0, 1, 5}, pb[3] = {3, 2, 4};
        for (int q = 0; q < 3; ++q) {
            const double2 zp = z[q * plane + ip], zm = z[q * plane + im];
            const double ar = 0.5 * (zp.x + zm.x), ai = 0.5 * (zp.y - zm.y);
            const double br = 0.5 * (zp.y + zm.y), bi = -0.5 * (zp.x - zm.x);
            // H = G (cs + i sn)
            const double har = ar * cs - ai * sn, hai = ar * sn + ai * cs;
            const double hbr = br * cs - bi * sn, hbi = br * sn + bi * cs;
            // order-0 planes (x0, y0) scaled by G, order-1 planes by G h_f
            const double sa = inv * (lv_plane_imag(pa[q]) ? sc0 : sc1), sb = inv * (lv_plane_imag(pb[q]) ? sc0 : sc1);
            out[pa[q] * qplane + e] = (T)(sa * (lv_plane_imag(pa[q]) ? hai : har));
            out[pb[q] * qplane + e] = (T)(sb * (lv_plane_imag(pb[q]) ? hbi : hbr));
        }
    }
}

// Potential tables of one key (Section 2 with K = 1/r): for a source cell w = 2^s
// finest cells wide at centre offset c (finest units), P^0 = w p0(c/w) and
// P^x, P^y = w^2 px(c/w), w^2 py(c/w) with the unit-cell integrals of
// unit_cell_potentials (finite everywhere). Packed z0 = Kr^px + i Kr^py,
// z1 = Kr^p0, Kr[e] = P(-e - d), stored period symmetric about -d as for the force.
__global__ void k_lv_tables_pot(double2 *z, int px, int py, int s, int d2)
{
    const int64_t plane = (int64_t)px * py;
    const double w = (double)(1 << s), d = 0.5 * d2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % px), b = (int)(e / px);
        const int ex = d2 < 0 ? (a <= px / 2 ? a : a - px) : (a < px / 2 ? a : a - px);
        const int ey = d2 < 0 ? (b <= py / 2 ? b : b - py) : (b < py / 2 ? b : b - py);
        double p3[3] = {0.0, 0.0, 0.0};
        if (!(d2 == 0 && (ex == -px / 2 || ey == -py / 2))) unit_cell_potentials((-ex - d) / w, (-ey - d) / w, p3);
        z[e] = make_double2(w * w * p3[1], w * w * p3[2]);
        z[plane + e] = make_double2(w * p3[0], 0.0);
    }
}

// Compressed potential spectra: planes p0 (Re H, even-even), px (Im H, odd in x)
// and py (Im H, odd in y), [kx][ky] for kx in [0, px/2], ky in [0, py/2] (rows padded
// to sg_spec_stride(py)), scaled by 1 / (px py) and by sc0 (p0) or sc1 (px, py).
template <typename T>
__global__ void k_lv_extract_pot(const double2 *z, T *out, int px, int py, int d2, double sc0, double sc1)
{
    const int qx = px / 2 + 1, qy = py / 2 + 1, qs = sg_spec_stride(py);
    const int64_t plane = (int64_t)px * py, qplane = (int64_t)qx * qs;
    const double inv = 1.0 / ((double)px * (double)py);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < qplane; e += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e / qs), ky = (int)(e % qs);
        if (ky >= qy) {  // row padding
            out[e] = out[qplane + e] = out[2 * qplane + e] = (T)0;
            continue;
        }
        const int64_t ip = (int64_t)ky * px + kx;
        const int64_t im = (int64_t)((py - ky) % py) * px + (px - kx) % px;
        double sn, cs;  // exp(-i pi d2 (kx/px + ky/py))
        sincospi(-(double)d2 * ((double)kx / px + (double)ky / py), &sn, &cs);
        const double2 zp = z[ip], zm = z[im], z1 = z[plane + ip];
        const double ar = 0.5 * (zp.x + zm.x), ai = 0.5 * (zp.y - zm.y);   // transform of Kr^px
        const double br = 0.5 * (zp.y + zm.y), bi = -0.5 * (zp.x - zm.x);  // of Kr^py
        out[e] = (T)(inv * sc0 * (z1.x * cs - z1.y * sn));
        out[qplane + e] = (T)(inv * sc1 * (ar * sn + ai * cs));
        out[2 * qplane + e] = (T)(inv * sc1 * (br * sn + bi * cs));
    }
}

// Phase factors exp(i pi k / P) for k in [-P/2, P/2] (index k + P/2), per axis;
// and the half-shift factors exp(-i pi j / P) for j in [0, P], per axis.
template <typename T>
__global__ void k_lv_phase(cplx_t<T> *out, int px, int py)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < px + py + 2; e += gridDim.x * blockDim.x) {
        const bool xa = e < px + 1;
        const int P = xa ? px : py, k = (xa ? e : e - (px + 1)) - P / 2;
        double sn, cs;
        sincospi((double)k / P, &sn, &cs);
        out[e] = cmake<cplx_t<T>>((T)cs, (T)sn);
    }
}

template <typename T>
__global__ void k_lv_cphase(cplx_t<T> *out, int px, int py)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < px + py + 2; e += gridDim.x * blockDim.x) {
        const bool xa = e < px + 1;
        const int P = xa ? px : py, j = xa ? e : e - (px + 1);
        double sn, cs;
        sincospi(-(double)j / P, &sn, &cs);
        out[e] = cmake<cplx_t<T>>((T)cs, (T)sn);
    }
}

// ----------------------------------------------------------- solve kernels --

template <typename T>
struct lv_rows_src {
    const T *S;         // composite source planes (sigma0, deltax, deltay), plane stride `plane`
    int64_t plane;
    const int *map;
    int nx, ny;
    int p0, st;         // image column i sits at compact position p0 + i 2^st
};

template <typename T>
__device__ __forceinline__ T lv_sample(const lv_rows_src<T> &a, int f, int j, int I)
{
    if (j >= a.ny) return (T)0;
    const int rel = I - a.p0;
    if (rel < 0 || (rel & ((1 << a.st) - 1))) return (T)0;
    const int i = rel >> a.st;
    if (i >= a.nx) return (T)0;
    const int c = a.map[(int64_t)j * a.nx + i];
    return c < 0 ? (T)0 : a.S[f * a.plane + c];
}

// Launch shapes of the transform passes: the row passes run NB = 4096 / PX
// sequences (two rows each) of length PX per CTA of 512 threads; the forward
// column pass NB = 4096 / PY columns per CTA of 512 threads (one radix-8
// butterfly per thread and stage up to 4096 points).
__host__ __device__ constexpr int lv_log2(int v) { return v <= 1 ? 0 : 1 + lv_log2(v >> 1); }
// Coarse target levels are folded onto their compact lengths before the inverse
// transforms only from 4096-point transforms up: below, the transforms are a
// small part of those passes and the folded ones measured no faster (their
// stages are latency-bound, and the extra lengths enlarge the kernels).
__host__ __device__ constexpr bool lv_fold_targets(int p) { return p >= 4096; }
__host__ __device__ constexpr int lv_nb(int px) { return px >= 4096 ? 1 : 4096 / px; }
__host__ __device__ constexpr int lv_cnb(int py) { return py >= 4096 ? 1 : 4096 / py; }
constexpr int LV_ROW_THREADS = 512, LV_CFWD_THREADS = 512;
// loads per thread issued before their shared-memory stores in the staging loops
constexpr int LV_LOAD_UNROLL = 4;

// All levels in one launch: blockIdx.x runs over the levels' CTA ranges
// [cta0[m], cta0[m+1]); each level dispatches to the transform of its length.
__device__ __forceinline__ int lv_level_of(const int *cta0, int nlev)
{
    int m = 0;
    while (m + 1 < nlev && (int)blockIdx.x >= cta0[m + 1]) ++m;
    return m;
}

// Row transforms (length PX = the level's compact Pcx) of a level's sampled
// rows (three fields, blockIdx.y), two real rows per complex sequence;
// out[(f qx + kx) ny + j], qx = PX/2 + 1.
template <typename T, int PX>
__device__ __forceinline__ void lv_row_fwd_body(const lv_rows_src<T> &a, cplx_t<T> *__restrict__ out,
                                                const cplx_t<T> *__restrict__ tw, int blk, cplx_t<T> *buf)
{
    using C = cplx_t<T>;
    constexpr int NB = lv_nb(PX), THREADS = LV_ROW_THREADS;
    constexpr int RB = 2 * NB;
    constexpr int QX = PX / 2 + 1;
    const int f = blockIdx.y;
    const int j0 = blk * RB;
    // LV_LOAD_UNROLL samples per thread in flight before their stores
    constexpr int NE = NB * (PX / 2);
    for (int e0 = threadIdx.x; e0 < NE; e0 += LV_LOAD_UNROLL * THREADS) {
        T va[LV_LOAD_UNROLL], vb[LV_LOAD_UNROLL];
#pragma unroll
        for (int u = 0; u < LV_LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS, q = e / (PX / 2), I = e % (PX / 2), ja = j0 + 2 * q;
            va[u] = e < NE ? lv_sample(a, f, ja, I) : (T)0;
            vb[u] = e < NE ? lv_sample(a, f, ja + 1, I) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < LV_LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS;
            if (e < NE) buf[spad<C>((e / (PX / 2)) * PX + e % (PX / 2))] = cmake<C>(va[u], vb[u]);
        }
    }
    __syncthreads();
    fft_batch<C, PX, NB, THREADS, false, true>(buf, tw);
    const T half = (T)0.5;
    for (int e = threadIdx.x; e < QX * RB; e += THREADS) {
        const int kx = e / RB, r = e % RB;
        const int j = j0 + r;
        if (j >= a.ny) continue;
        const int q = r >> 1;
        const C zz = buf[spad<C>(q * PX + kx)];
        const C w = buf[spad<C>(q * PX + ((PX - kx) & (PX - 1)))];
        C o;
        if ((r & 1) == 0) o = cmake<C>(half * (zz.x + w.x), half * (zz.y - w.y));
        else o = cmake<C>(half * (zz.y + w.y), half * (w.x - zz.x));
        out[((int64_t)f * QX + kx) * a.ny + j] = o;
    }
}

template <typename T>
struct lv_row_fwd_args {
    int nlev;
    int cta0[SG_MAX_LEVELS + 1];
    lv_rows_src<T> a[SG_MAX_LEVELS];
    cplx_t<T> *out[SG_MAX_LEVELS];
    const cplx_t<T> *tw[SG_MAX_LEVELS];
    int lp[SG_MAX_LEVELS];  // log2 of the level's compact row length
};

#define SG_LV_BODY_SWITCH(LP, LMAX, BODY)                                                 \
    switch (LP) {                                                                      \
    case 6: { constexpr int PP = 64; BODY; break; }                                    \
    case 7: { constexpr int PP = 128; BODY; break; }                                   \
    case 8: { constexpr int PP = 256; BODY; break; }                                   \
    case 9: { constexpr int PP = 512; BODY; break; }                                   \
    case 10: { constexpr int PP = 1024; BODY; break; }                                 \
    case 11: { constexpr int PP = 2048; BODY; break; }                                 \
    case 12: { constexpr int PP = 4096; BODY; break; }                                 \
    case 13: if constexpr (LMAX >= 8192) { constexpr int PP = 8192; BODY; } break;     \
    default: break;                                                                    \
    }

template <typename T, int LMAX>
__global__ void __launch_bounds__(LV_ROW_THREADS) k_lv_row_fwd(lv_row_fwd_args<T> A)
{
    sg_dep_trigger();
    sg_dep_wait();  // the composite sources
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int m = lv_level_of(A.cta0, A.nlev);
    const int blk = blockIdx.x - A.cta0[m];
    SG_LV_BODY_SWITCH(A.lp[m], LMAX, (lv_row_fwd_body<T, PP>(A.a[m], A.out[m], A.tw[m], blk, buf)));
}

struct lv_col_src {
    int ny, p0, st;     // image row j sits at compact position p0 + j 2^st
    int qx;             // compact half-spectrum width Pcx/2 + 1
    int cx, cy;         // compression exponents (half-shift table index shifts)
    int hx, hy;         // samples half-shifted on that axis (c = s >= 1)
};

// Column transforms (length PY = the level's compact Pcy) to compact spectra
// times the half-shift factors psi_x(kx) psi_y(ky), NB = lv_cnb(PY) columns
// per CTA; spec[(f qx + kx) PY + ky].
template <typename T, int PY>
__device__ __forceinline__ void lv_col_fwd_body(const cplx_t<T> *__restrict__ in, cplx_t<T> *__restrict__ spec,
                                                const lv_col_src &a, const cplx_t<T> *__restrict__ tw,
                                                const cplx_t<T> *__restrict__ cphx, const cplx_t<T> *__restrict__ cphy,
                                                int blk, cplx_t<T> *buf)
{
    using C = cplx_t<T>;
    constexpr int NB = lv_cnb(PY), THREADS = LV_CFWD_THREADS;
    const int f = blockIdx.y, kx0 = blk * NB;
    for (int e = threadIdx.x; e < NB * (PY / 2); e += THREADS)
        buf[spad<C>((e / (PY / 2)) * PY + e % (PY / 2))] = cmake<C>((T)0, (T)0);
    __syncthreads();
    const int ne = NB * a.ny;
    for (int e0 = threadIdx.x; e0 < ne; e0 += LV_LOAD_UNROLL * THREADS) {
        C v[LV_LOAD_UNROLL];
#pragma unroll
        for (int u = 0; u < LV_LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS, q = e / a.ny, j = e % a.ny, kx = kx0 + q;
            v[u] = (e < ne && kx < a.qx) ? in[((int64_t)f * a.qx + kx) * a.ny + j] : cmake<C>((T)0, (T)0);
        }
#pragma unroll
        for (int u = 0; u < LV_LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS, q = e / a.ny, j = e % a.ny, kx = kx0 + q;
            if (e < ne && kx < a.qx) buf[spad<C>(q * PY + a.p0 + (j << a.st))] = v[u];
        }
    }
    __syncthreads();
    fft_batch<C, PY, NB, THREADS, false, true>(buf, tw);
    for (int e = threadIdx.x; e < NB * PY; e += THREADS) {
        const int q = e / PY, k = e % PY, kx = kx0 + q;
        if (kx >= a.qx) continue;
        C v = buf[spad<C>(e)];
        if (a.hy) v = cmul(v, cphy[k << a.cy]);
        if (a.hx) v = cmul(v, cphx[kx << a.cx]);
        spec[((int64_t)f * a.qx + kx) * PY + k] = v;
    }
}

template <typename T>
struct lv_col_fwd_args {
    int nlev;
    int cta0[SG_MAX_LEVELS + 1];
    lv_col_src a[SG_MAX_LEVELS];
    const cplx_t<T> *in[SG_MAX_LEVELS];
    cplx_t<T> *spec[SG_MAX_LEVELS];
    const cplx_t<T> *tw[SG_MAX_LEVELS];
    int lp[SG_MAX_LEVELS];  // log2 of the level's compact column length
    const cplx_t<T> *cphx, *cphy;
};

// (resident CTAs per SM asked of the register allocator: FP32 three at up to
// 4096 points, two at 8192; FP64 two)
template <typename T, int LMAX>
__global__ void __launch_bounds__(LV_CFWD_THREADS, sizeof(T) == 4 ? (LMAX <= 4096 ? 3 : 2) : (LMAX <= 4096 ? 2 : 1))
    k_lv_col_fwd(lv_col_fwd_args<T> A)
{
    sg_dep_trigger();
    sg_dep_wait();  // the row transforms
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int m = lv_level_of(A.cta0, A.nlev);
    const int blk = blockIdx.x - A.cta0[m];
    SG_LV_BODY_SWITCH(A.lp[m], LMAX,
                      (lv_col_fwd_body<T, PP>(A.in[m], A.spec[m], A.a[m], A.tw[m], A.cphx, A.cphy, blk, buf)));
}

struct lv_mac_args {
    int nsrc;
    int64_t spec_off[SG_MAX_LEVELS];    // complex-element offset of each source level's compact spectra
    int lpx[SG_MAX_LEVELS];             // log2 of its compact lengths Pcx, Pcy
    int lpy[SG_MAX_LEVELS];
    int hx[SG_MAX_LEVELS];              // its samples half-shifted along x, y
    int hy[SG_MAX_LEVELS];
    int key[SG_MAX_LEVELS][SG_MAX_LEVELS];  // kernel of source level m for target level l, [m][l]
    int d2[SG_MAX_LEVELS][SG_MAX_LEVELS];   // its 2 x sample shift
    // target level l: its ny sampled rows sit at compact positions p0 + j 2^st of
    // its compact column length 2^lm (lm < log2 PY: the bins are folded onto it,
    // with the half-sample shift when fh), inverse twiddles tw[l]
    int ny[SG_MAX_LEVELS];
    int p0[SG_MAX_LEVELS];
    int st[SG_MAX_LEVELS];
    int lm[SG_MAX_LEVELS];
    int fh[SG_MAX_LEVELS];
    const void *tw[SG_MAX_LEVELS];
    int64_t inv_off[SG_MAX_LEVELS];     // complex-element offset of its inverse-column outputs
    int qx;
};

// Transform length switch for the compact target lengths 64 .. LMAX (only the
// lengths up to LMAX are instantiated).
#define SG_LV_LEN_SWITCH(LP, LMAX, BODY)                                                   \
    switch (LP) {                                                                        \
    case 6: if constexpr (64 <= LMAX) { constexpr int PP = 64; BODY; } break;            \
    case 7: if constexpr (128 <= LMAX) { constexpr int PP = 128; BODY; } break;          \
    case 8: if constexpr (256 <= LMAX) { constexpr int PP = 256; BODY; } break;          \
    case 9: if constexpr (512 <= LMAX) { constexpr int PP = 512; BODY; } break;          \
    case 10: if constexpr (1024 <= LMAX) { constexpr int PP = 1024; BODY; } break;       \
    case 11: if constexpr (2048 <= LMAX) { constexpr int PP = 2048; BODY; } break;       \
    case 12: if constexpr (4096 <= LMAX) { constexpr int PP = 4096; BODY; } break;       \
    case 13: if constexpr (8192 <= LMAX) { constexpr int PP = 8192; BODY; } break;       \
    default: break;                                                                      \
    }

// Sampling a length-L inverse transform every 2^c points from position r
// (c >= 1, L = M 2^c) equals the length-M inverse transform of the folded
// spectrum Z(k) = sum_q X(k + q M) exp(2 pi i (k + q M) r / L), k < M. Here r is 0,
// or half a compact sample (r = 2^(c-1), half): Z(k) = conj(psi(k)) sum_q (-1)^q
// X(k + q M), psi(k) = exp(-i pi k / M) = cph[k 2^c].
template <typename C, int L>
__device__ __forceinline__ C lv_fold_bin(const C *buf, int k, int lm, bool half, const C *__restrict__ cph)
{
    const int M = 1 << lm, nq = L >> lm;
    C acc = buf[spad<C>(k)];
    for (int q = 1; q < nq; ++q) {
        const C u = buf[spad<C>(k + q * M)];
        acc = (half && (q & 1)) ? csub(acc, u) : cadd(acc, u);
    }
    return half ? cmulc(acc, cph[k << (lv_log2(L) - lm)]) : acc;
}

// NSEQ sequences of length L back to back in buf become NSEQ folded sequences of
// length M back to back (staged through registers: the outputs overlap inputs
// of other threads).
template <typename C, int L, int NSEQ, int THREADS>
__device__ __forceinline__ void lv_fold_spectrum(C *buf, int lm, bool half, const C *__restrict__ cph)
{
    constexpr int IT = (NSEQ * (L / 2) + THREADS - 1) / THREADS;  // M <= L/2
    const int M = 1 << lm;
    C v[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int e = threadIdx.x + i * THREADS;
        if (e < NSEQ * M) v[i] = lv_fold_bin<C, L>(buf + spad<C>((e >> lm) * L), e & (M - 1), lm, half, cph);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int e = threadIdx.x + i * THREADS;
        if (e < NSEQ * M) buf[spad<C>(e)] = v[i];
    }
    __syncthreads();
}

// The compact source column of column kx for source level m: kx mod Pcx, or its
// Hermitian partner (fold), with the sign of the x half-shift.
struct lv_src_col {
    int lpy, pcy;
    bool fold, hy, xneg;
    int col;        // compact column index
    int64_t splane; // field plane stride of the source's compact spectra
};

__device__ __forceinline__ lv_src_col lv_source_column(const lv_mac_args &a, int m, int kx)
{
    lv_src_col c;
    const int lpx = a.lpx[m], pcx = 1 << lpx;
    c.lpy = a.lpy[m];
    c.pcy = 1 << c.lpy;
    const int kxr = kx & (pcx - 1);
    c.fold = kxr > (pcx >> 1);
    c.col = c.fold ? pcx - kxr : kxr;
    c.splane = (int64_t)((pcx >> 1) + 1) * c.pcy;
    c.hy = a.hy[m] != 0;
    // sign of the x half-shift: (-1)^(kx div Pcx), times -1 on the folded half
    c.xneg = a.hx[m] && ((((kx >> lpx) & 1) != 0) != c.fold);
    return c;
}

// Row of bin ky in the compact column, and the sign of the half-shifts there.
__device__ __forceinline__ void lv_source_row(const lv_src_col &c, int ky, int &row, bool &neg)
{
    const int kyr = ky & (c.pcy - 1);
    row = c.fold ? ((c.pcy - kyr) & (c.pcy - 1)) : kyr;
    neg = c.xneg != (c.hy && ((((ky >> c.lpy) & 1) != 0) != (c.fold && kyr != 0)));
}

// One bin of one source: the three fields X0..X2 (conjugated on the folded
// half) times the kernel planes g (x family, or the potential's p0 px py) and h
// (y family), sg = -1 on the upper half for the planes odd in ky, half-cell
// phase p when d2 != 0, added into ax (and ay) with the half-shift sign.
template <typename T, int NOUT>
__device__ __forceinline__ void lv_mac_bin(cplx_t<T> X0, cplx_t<T> X1, cplx_t<T> X2, bool fold, T g0, T g1, T g2,
                                           T h0, T h1, T h2, T sg, cplx_t<T> p, int d2, bool neg, cplx_t<T> &ax,
                                           cplx_t<T> &ay)
{
    using C = cplx_t<T>;
    if (fold) {
        X0.y = -X0.y;
        X1.y = -X1.y;
        X2.y = -X2.y;
    }
    if constexpr (NOUT == 2) {
        // planes (prescaled by G, G h_f): x0 imaginary, xx real, xy real; y0 imaginary,
        // yx real, yy real. The parts odd in ky (xy; y0, yx) change sign on the upper half.
        const T o2 = sg * g2, o0 = sg * h0, o1 = sg * h1;
        C hx = cmake<C>(g1 * X1.x - g0 * X0.y + o2 * X2.x, g1 * X1.y + g0 * X0.x + o2 * X2.y);
        C hy = cmake<C>(h2 * X2.x - o0 * X0.y + o1 * X1.x, h2 * X2.y + o0 * X0.x + o1 * X1.y);
        if (d2 != 0) {
            if (d2 < 0) p.y = -p.y;
            hx = cmul(hx, p);
            hy = cmul(hy, p);
        }
        const T sn = neg ? (T)-1 : (T)1;
        ax = cmake<C>(ax.x + sn * hx.x, ax.y + sn * hx.y);
        ay = cmake<C>(ay.x + sn * hy.x, ay.y + sn * hy.y);
    } else {
        // potential planes: p0 real, px imaginary, py imaginary and odd in ky
        const T o2 = sg * g2;
        C hp = cmake<C>(g0 * X0.x - g1 * X1.y - o2 * X2.y, g0 * X0.y + g1 * X1.x + o2 * X2.x);
        if (d2 != 0) {
            if (d2 < 0) p.y = -p.y;
            hp = cmul(hp, p);
        }
        const T sn = neg ? (T)-1 : (T)1;
        ax = cmake<C>(ax.x + sn * hp.x, ax.y + sn * hp.y);
    }
}

// Inverse transforms (length L) of the NOUT outputs, held PY apart in shared
// memory. One at a time, and with the length switch outside the loop: a batch of
// both, or a switch inside the loop, makes the register allocation of the
// whole kernel (its per-bin loads) grow by a quarter or more.
template <typename C, int PY, int L, int NOUT, int THREADS>
__device__ __forceinline__ void lv_inv_columns(C *bx, const C *__restrict__ tw)
{
#pragma unroll 1
    for (int o = 0; o < NOUT; ++o) fft_batch<C, L, 1, THREADS, true, false, true>(bx + spad<C>(o * PY), tw);
}

// One (column kx, target level l) per CTA, kx = blockIdx.x / nsrc and
// l = blockIdx.x % nsrc, so that the CTAs of all target levels of a column run
// side by side and read its source spectra (and shared kernel planes) from L2:
// Fx^, Fy^ = sum over source levels and fields of source spectrum (unfolded
// from the compact one) x kernel spectrum (decompressed, see k_lv_extract),
// formed element by element straight into two shared buffers; from 4096-point
// columns up, for a coarse target level, folded in place onto its compact column
// length (lv_fold_bin); inverse column transforms of that length; the target
// level's sampled rows to out[(o qx + kx) ny + j] (out at the level's
// inverse-column offset). NOUT = 1: the potential, one output from 3 kernel
// planes per key (p0 real, px and py imaginary; py odd in ky).
template <typename T, int PY, int THREADS, int MINB, int NOUT>
__global__ void __launch_bounds__(THREADS, MINB) k_lv_col_mac_inv(lv_mac_args a, const cplx_t<T> *__restrict__ spec,
                                                            const T *__restrict__ kspec,
                                                            const cplx_t<T> *__restrict__ phx,
                                                            const cplx_t<T> *__restrict__ phy,
                                                            cplx_t<T> *__restrict__ out,
                                                            const cplx_t<T> *__restrict__ cph)
{
    sg_dep_trigger();
    sg_dep_wait();  // the source spectra
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *bx = reinterpret_cast<C *>(smem_raw);
    C *by = bx + spad<C>(PY);
    constexpr int QS = ((PY / 2 + 1) + 3) & ~3;  // kernel plane row stride (sg_spec_stride)
    const int kx = blockIdx.x / a.nsrc, l = blockIdx.x % a.nsrc;
    const int64_t kqplane = (int64_t)a.qx * QS;
    constexpr int NPL = NOUT == 2 ? 6 : 3;  // kernel planes per key
    // Bins in mirror pairs: slot j in [0, PY/2) holds bins j and PY - j, which read
    // the same kernel values (kq = j); slot 0 holds bins 0 and PY/2 (kq = 0 and PY/2).
    // V slots per thread at a time, so that their loads are in flight together.
    constexpr int NSLOT = PY / 2;
    // (FP32 2048-point force columns: one slot pair, 56 registers, four CTAs per
    // SM measured 2 % faster than two pairs at three CTAs; two pairs elsewhere,
    // measured faster than one at 4096 and 8192 points)
    constexpr int VMAX = sizeof(T) == 8 ? 1 : (NOUT == 2 && PY == 2048 ? 1 : 2);
    constexpr int V = NSLOT / THREADS >= VMAX ? VMAX : 1;
    const C phk = phx[kx + (a.qx - 1)];
    for (int j0 = threadIdx.x; j0 < NSLOT; j0 += V * THREADS) {
        int ky[V][2];
        C ph[V][2], ax[V][2], ay[V][2];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = j0 + v * THREADS;
            ky[v][0] = j;
            ky[v][1] = j == 0 ? PY / 2 : PY - j;
            // half-cell phase exp(i pi (kx / Px + ky / Py)) at the signed frequencies j and -j (PY/2 for slot 0)
            ph[v][0] = cmul(phk, phy[j + PY / 2]);
            ph[v][1] = cmul(phk, phy[(j == 0 ? PY / 2 : -j) + PY / 2]);
#pragma unroll
            for (int b = 0; b < 2; ++b) ax[v][b] = ay[v][b] = cmake<C>((T)0, (T)0);
        }
        for (int m = 0; m < a.nsrc; ++m) {
            const lv_src_col sc = lv_source_column(a, m, kx);
            const int64_t splane = sc.splane;
            const C *sm = spec + a.spec_off[m] + (int64_t)sc.col * sc.pcy;
            const T *km = kspec + (int64_t)a.key[m][l] * NPL * kqplane + (int64_t)kx * QS;
            int row[V][2];
            bool neg[V][2];
#pragma unroll
            for (int v = 0; v < V; ++v) {
#pragma unroll
                for (int b = 0; b < 2; ++b) lv_source_row(sc, ky[v][b], row[v][b], neg[v][b]);
            }
            C X[3][V][2];
            T gx[3][V][2], gy[3][V][2];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int j = j0 + v * THREADS;
                    X[f][v][0] = sm[f * splane + row[v][0]];
                    X[f][v][1] = sm[f * splane + row[v][1]];
                    gx[f][v][0] = gx[f][v][1] = km[f * kqplane + j];
                    if constexpr (NOUT == 2) gy[f][v][0] = gy[f][v][1] = km[(3 + f) * kqplane + j];
                }
            }
            if (j0 == 0) {  // slot 0: bin PY/2 has kernel values of its own
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    gx[f][0][1] = km[f * kqplane + PY / 2];
                    if constexpr (NOUT == 2) gy[f][0][1] = km[(3 + f) * kqplane + PY / 2];
                }
            }
            const int d2 = a.d2[m][l];
#pragma unroll
            for (int v = 0; v < V; ++v) {
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const T sg = (b == 0 || ky[v][1] == PY / 2) ? (T)1 : (T)-1;
                    if constexpr (NOUT == 2)
                        lv_mac_bin<T, 2>(X[0][v][b], X[1][v][b], X[2][v][b], sc.fold, gx[0][v][b], gx[1][v][b],
                                         gx[2][v][b], gy[0][v][b], gy[1][v][b], gy[2][v][b], sg, ph[v][b], d2,
                                         neg[v][b], ax[v][b], ay[v][b]);
                    else
                        lv_mac_bin<T, 1>(X[0][v][b], X[1][v][b], X[2][v][b], sc.fold, gx[0][v][b], gx[1][v][b],
                                         gx[2][v][b], (T)0, (T)0, (T)0, sg, ph[v][b], d2, neg[v][b], ax[v][b],
                                         ay[v][b]);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                bx[spad<C>(ky[v][b])] = ax[v][b];
                if constexpr (NOUT == 2) by[spad<C>(ky[v][b])] = ay[v][b];
            }
        }
    }
    __syncthreads();
    const int lm = a.lm[l];
    if constexpr (lv_fold_targets(PY)) {
        // a coarse target level is sampled every 2^c rows: fold onto its compact
        // length, in place (bin k < M of an output is written only by the thread
        // that reads it)
        if (lm < lv_log2(PY)) {
            for (int e = threadIdx.x; e < (NOUT << lm); e += THREADS) {
                C *seq = bx + spad<C>((e >> lm) * PY);
                const int k = e & ((1 << lm) - 1);
                seq[spad<C>(k)] = lv_fold_bin<C, PY>(seq, k, lm, a.fh[l] != 0, cph);
            }
            __syncthreads();
        }
        SG_LV_LEN_SWITCH(lm, PY, (lv_inv_columns<C, PY, PP, NOUT, THREADS>(bx, (const C *)a.tw[l])));
    }
    const int ny = a.ny[l], p0 = a.p0[l], st = a.st[l];
    for (int o = 0; o < NOUT; ++o) {
        C *seq = bx + spad<C>(o * PY);
        if constexpr (!lv_fold_targets(PY)) fft_batch<C, PY, 1, THREADS, true, false, true>(seq, (const C *)a.tw[l]);
        C *dst = out + a.inv_off[l] + ((int64_t)o * a.qx + kx) * ny;
        for (int j = threadIdx.x; j < ny; j += THREADS) dst[j] = seq[spad<C>(p0 + (j << st))];
    }
}

struct lv_out_dst {
    const int *map;
    int nx, ny;
    int p0, st;  // image column i sits at compact position p0 + i 2^st
    int lm, fh;  // log2 of the compact row length; samples half-shifted along x
};

template <typename T>
struct lv_row_inv_args {
    int nlev;
    int cta0[SG_MAX_LEVELS + 1];
    lv_out_dst a[SG_MAX_LEVELS];
    const cplx_t<T> *in[SG_MAX_LEVELS];
    const cplx_t<T> *tw[SG_MAX_LEVELS];  // inverse twiddles of the compact row length
    const cplx_t<T> *cph;               // psi_x table (finest length)
};

// Inverse row transforms of every target level's rows (blockIdx.y = Fx, Fy),
// all levels in one launch: the full rows are unpacked from the half spectra,
// folded onto the level's compact row length (lv_fold_spectrum) when its cells
// are wider than a finest cell, transformed, and the samples at compact columns
// p0 + i 2^st go to the level's cells through the map.
template <typename T, int PX>
__global__ void __launch_bounds__(LV_ROW_THREADS) k_lv_row_inv(lv_row_inv_args<T> A, T *__restrict__ fx,
                                                              T *__restrict__ fy)
{
    sg_dep_trigger();
    sg_dep_wait();  // the target columns
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    constexpr int NB = lv_nb(PX), THREADS = LV_ROW_THREADS;
    constexpr int RB = 2 * NB;
    constexpr int QX = PX / 2 + 1;
    const int lvl = lv_level_of(A.cta0, A.nlev);
    const lv_out_dst &a = A.a[lvl];
    const int o = blockIdx.y;
    const int j0 = (blockIdx.x - A.cta0[lvl]) * RB;
    const int ny = a.ny;
    const C *w = A.in[lvl] + (int64_t)o * QX * ny;
    T *out = o == 0 ? fx : fy;
    constexpr int NE = NB * QX;
    for (int e0 = threadIdx.x; e0 < NE; e0 += LV_LOAD_UNROLL * THREADS) {
        C xv[LV_LOAD_UNROLL], yv[LV_LOAD_UNROLL];
#pragma unroll
        for (int u = 0; u < LV_LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS, q = e % NB, k = e / NB, ja = j0 + 2 * q;
            xv[u] = (e < NE && ja < ny) ? w[(int64_t)k * ny + ja] : cmake<C>((T)0, (T)0);
            yv[u] = (e < NE && ja + 1 < ny) ? w[(int64_t)k * ny + ja + 1] : cmake<C>((T)0, (T)0);
        }
#pragma unroll
        for (int u = 0; u < LV_LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS, q = e % NB, k = e / NB;
            if (e >= NE) continue;
            C x = xv[u], y = yv[u];
            if (k == 0 || k == PX / 2) {
                x.y = (T)0;
                y.y = (T)0;
            }
            buf[spad<C>(q * PX + k)] = cmake<C>(x.x - y.y, x.y + y.x);
            if (k > 0 && k < PX / 2) buf[spad<C>(q * PX + PX - k)] = cmake<C>(x.x + y.y, y.x - x.y);
        }
    }
    __syncthreads();
    const int lm = a.lm;
    if constexpr (lv_fold_targets(PX)) {
        if (lm < lv_log2(PX)) lv_fold_spectrum<C, PX, NB, THREADS>(buf, lm, a.fh != 0, A.cph);
        SG_LV_LEN_SWITCH(lm, PX, (fft_batch<C, PP, NB, THREADS, true, false, true>(buf, A.tw[lvl])));
    } else {
        fft_batch<C, PX, NB, THREADS, true, false, true>(buf, A.tw[lvl]);
    }
    for (int e = threadIdx.x; e < NB * a.nx; e += THREADS) {
        const int q = e / a.nx, i = e % a.nx;
        const int ja = j0 + 2 * q;
        const C zz = buf[spad<C>((q << lm) + a.p0 + (i << a.st))];
        if (ja < ny) {
            const int c = a.map[(int64_t)ja * a.nx + i];
            if (c >= 0) out[c] = zz.x;
        }
        if (ja + 1 < ny) {
            const int c = a.map[(int64_t)(ja + 1) * a.nx + i];
            if (c >= 0) out[c] = zz.y;
        }
    }
}

// ----------------------------------------------------------- launchers --

constexpr int lv_col_threads(int py) { return py / 8 < 64 ? 64 : (py / 8 > 512 ? 512 : py / 8); }
// Column-MAC CTAs: the two shared spectra of a column grow to 2 x 8192 x 8 bytes
// (FP32) or 2 x 4096 x 16 (FP64), which leaves one CTA per SM; the FP32 one gets
// 1024 threads (at most 64 registers each) so that more loads are in flight, the
// FP64 one 512 (its allocation spills at 64).
template <typename T>
constexpr int lv_mac_threads(int py)
{
    return sizeof(T) == 8 ? (py >= 4096 ? 512 : lv_col_threads(py)) : (py >= 8192 ? 1024 : lv_col_threads(py));
}
// FP32 2048-point columns with two outputs: four CTAs of 256 threads per SM (at
// most 64 registers; one slot pair per thread)
template <typename T>
constexpr int lv_mac_minb(int py, int nout)
{
    return sizeof(T) == 4 && py == 4096               ? 2
           : sizeof(T) == 4 && py == 2048 && nout == 2 ? 4
                                                        : (lv_mac_threads<T>(py) >= 1024 ? 1 : 0);
}

template <typename K>
sg_status smem_attr(K kern, size_t bytes)
{
    if (bytes > 48 * 1024) SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return SG_OK;
}

template <typename T>
sg_status launch_row_fwd(const lv_row_fwd_args<T> &A, int ncta, int lmax, cudaStream_t st)
{
    const size_t sm = spad_size<cplx_t<T>>(lv_nb(lmax) * lmax) * sizeof(cplx_t<T>);
    auto kern = lmax > 4096 ? k_lv_row_fwd<T, 8192> : k_lv_row_fwd<T, 4096>;
    SG_TRY(smem_attr(kern, sm));
    SG_CUDA_TRY(sg_launch_dep(kern, dim3(ncta, 3), dim3(LV_ROW_THREADS), sm, st, A));
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T>
sg_status launch_col_fwd(const lv_col_fwd_args<T> &A, int ncta, int lmax, cudaStream_t st)
{
    const size_t sm = spad_size<cplx_t<T>>(lv_cnb(lmax) * lmax) * sizeof(cplx_t<T>);
    auto kern = lmax > 4096 ? k_lv_col_fwd<T, 8192> : k_lv_col_fwd<T, 4096>;
    SG_TRY(smem_attr(kern, sm));
    SG_CUDA_TRY(sg_launch_dep(kern, dim3(ncta, 3), dim3(LV_CFWD_THREADS), sm, st, A));
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PY, int NOUT>
sg_status launch_col_mac_inv(const lv_mac_args &a, const cplx_t<T> *spec, const T *kspec, const cplx_t<T> *phx,
                             const cplx_t<T> *phy, cplx_t<T> *out, const cplx_t<T> *cph, cudaStream_t st)
{
    constexpr int TH = lv_mac_threads<T>(PY);
    const size_t sm = spad_size<cplx_t<T>>(NOUT * PY) * sizeof(cplx_t<T>);
    auto kern = k_lv_col_mac_inv<T, PY, TH, lv_mac_minb<T>(PY, NOUT), NOUT>;
    SG_TRY(smem_attr(kern, sm));
    SG_CUDA_TRY(sg_launch_dep(kern, dim3(a.qx * a.nsrc), dim3(TH), sm, st, a, spec, kspec, phx, phy, out, cph));
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PX>
sg_status launch_row_inv(const lv_row_inv_args<T> &A, int ncta, int nout, T *fx, T *fy, cudaStream_t st)
{
    const size_t sm = spad_size<cplx_t<T>>(lv_nb(PX) * PX) * sizeof(cplx_t<T>);
    auto kern = k_lv_row_inv<T, PX>;
    SG_TRY(smem_attr(kern, sm));
    SG_CUDA_TRY(sg_launch_dep(kern, dim3(ncta, nout), dim3(LV_ROW_THREADS), sm, st, A, fx, fy));
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

#define SG_LV_SWITCH(P, CALL)                  \
    switch (P) {                               \
    case 64: { constexpr int PP = 64; CALL; break; }     \
    case 128: { constexpr int PP = 128; CALL; break; }   \
    case 256: { constexpr int PP = 256; CALL; break; }   \
    case 512: { constexpr int PP = 512; CALL; break; }   \
    case 1024: { constexpr int PP = 1024; CALL; break; } \
    case 2048: { constexpr int PP = 2048; CALL; break; } \
    case 4096: { constexpr int PP = 4096; CALL; break; } \
    case 8192: { constexpr int PP = 8192; CALL; break; } \
    default: return SG_EINVAL;                 \
    }

// One solve on the composite sources in ws->sfield: the force (Fx, Fy into
// out0, out1) or, with pot, the potential (into out0) from the potential spectra.
template <typename T>
sg_status lv_solve_t(sg_plan *plan, const sg_workspace *ws, void *out0, void *out1, bool pot, cudaStream_t st)
{
    using C = cplx_t<T>;
    const sg_lv &lv = *plan->lv;
    const int qx = lv.px / 2 + 1;
    const int64_t *twoff = sizeof(T) == 8 ? plan->tw64_off : plan->tw32_off;
    auto twid = [&](int L) { return (const C *)((const char *)plan->twiddles + twoff[sg_ilog2(L)]); };
    const C *cphx = (const C *)lv.cphase, *cphy = cphx + lv.px + 1;
    C *wf = (C *)ws->work_fwd;
    C *wi = (C *)ws->work_inv;
    C *spec = wf + lv.fwd_elems;
    sg_timing_begin(ws, SG_STAGE_ROW_FWD, st);
    {
        // row transforms of every level's sampled rows, at the level's compact length
        lv_row_fwd_args<T> A;
        memset(&A, 0, sizeof(A));
        A.nlev = lv.nlev;
        int ncta = 0;
        for (int m = 0; m < lv.nlev; ++m) {
            const sg_lv_level &L = lv.lev[m];
            const int pcx = lv.px >> L.cx;
            A.cta0[m] = ncta;
            A.a[m] = {(const T *)ws->sfield, plan->ncells, L.map, L.nx, L.ny, L.i0 >> L.cx, L.s - L.cx};
            A.out[m] = wf + L.fwd_off;
            A.tw[m] = twid(pcx);
            A.lp[m] = sg_ilog2(pcx);
            ncta += (L.ny + 2 * lv_nb(pcx) - 1) / (2 * lv_nb(pcx));
        }
        A.cta0[lv.nlev] = ncta;
        SG_TRY(launch_row_fwd<T>(A, ncta, lv.px, st));
    }
    sg_timing_end(ws, SG_STAGE_ROW_FWD, st);
    sg_timing_begin(ws, SG_STAGE_COL_CONV, st);
    {
        // column transforms to compact source spectra
        lv_col_fwd_args<T> A;
        memset(&A, 0, sizeof(A));
        A.nlev = lv.nlev;
        A.cphx = cphx;
        A.cphy = cphy;
        int ncta = 0;
        for (int m = 0; m < lv.nlev; ++m) {
            const sg_lv_level &L = lv.lev[m];
            const int pcx = lv.px >> L.cx, pcy = lv.py >> L.cy;
            A.cta0[m] = ncta;
            A.a[m] = {L.ny, L.j0 >> L.cy, L.s - L.cy, pcx / 2 + 1, L.cx, L.cy,
                      L.cx == L.s && L.s >= 1, L.cy == L.s && L.s >= 1};
            A.in[m] = wf + L.fwd_off;
            A.spec[m] = spec + L.spec_off;
            A.tw[m] = twid(pcy);
            A.lp[m] = sg_ilog2(pcy);
            ncta += (pcx / 2 + 1 + lv_cnb(pcy) - 1) / lv_cnb(pcy);
        }
        A.cta0[lv.nlev] = ncta;
        SG_TRY(launch_col_fwd<T>(A, ncta, lv.py, st));
    }
    {
        // one launch for all target levels
        lv_mac_args a;
        memset(&a, 0, sizeof(a));
        a.nsrc = lv.nlev;
        for (int m = 0; m < lv.nlev; ++m) {
            const sg_lv_level &M = lv.lev[m];
            a.spec_off[m] = M.spec_off;
            a.lpx[m] = sg_ilog2(lv.px >> M.cx);
            a.lpy[m] = sg_ilog2(lv.py >> M.cy);
            a.hx[m] = M.cx == M.s && M.s >= 1;
            a.hy[m] = M.cy == M.s && M.s >= 1;
            for (int l = 0; l < lv.nlev; ++l) {
                a.key[m][l] = lv.key[m][l];
                a.d2[m][l] = lv.key_d2[lv.key[m][l]];
            }
            const int fy = lv_fold_targets(lv.py) ? M.cy : 0;  // target fold exponent
            a.ny[m] = M.ny;
            a.p0[m] = M.j0 >> fy;
            a.st[m] = M.s - fy;
            a.lm[m] = sg_ilog2(lv.py >> fy);
            a.fh[m] = fy == M.s && M.s >= 1;
            a.tw[m] = twid(lv.py >> fy);
            a.inv_off[m] = M.inv_off;
        }
        a.qx = qx;
        const C *phx = (const C *)lv.phase, *phy = phx + lv.px + 1;
        if (pot) {
            SG_LV_SWITCH(lv.py, SG_TRY((launch_col_mac_inv<T, PP, 1>(a, spec, (const T *)lv.pspectra, phx, phy, wi, cphy,
                                                                      st))));
        } else {
            SG_LV_SWITCH(lv.py, SG_TRY((launch_col_mac_inv<T, PP, 2>(a, spec, (const T *)lv.spectra, phx, phy, wi, cphy,
                                                                      st))));
        }
    }
    sg_timing_end(ws, SG_STAGE_COL_CONV, st);
    sg_timing_begin(ws, SG_STAGE_ROW_INV, st);
    {
        lv_row_inv_args<T> A;
        memset(&A, 0, sizeof(A));
        A.nlev = lv.nlev;
        int ncta = 0;
        for (int l = 0; l < lv.nlev; ++l) {
            const sg_lv_level &L = lv.lev[l];
            A.cta0[l] = ncta;
            const int fx = lv_fold_targets(lv.px) ? L.cx : 0;
            A.a[l] = {L.map, L.nx, L.ny, L.i0 >> fx, L.s - fx, sg_ilog2(lv.px >> fx), fx == L.s && L.s >= 1};
            A.in[l] = wi + L.inv_off;
            A.tw[l] = twid(lv.px >> fx);
            ncta += (L.ny + 2 * lv_nb(lv.px) - 1) / (2 * lv_nb(lv.px));
        }
        A.cta0[lv.nlev] = ncta;
        A.cph = cphx;
        SG_LV_SWITCH(lv.px, SG_TRY((launch_row_inv<T, PP>(A, ncta, pot ? 1 : 2, (T *)out0, (T *)out1, st))));
    }
    sg_timing_end(ws, SG_STAGE_ROW_INV, st);
    return SG_OK;
}

}  // namespace

void sg_lv_free(sg_plan *plan)
{
    if (!plan || !plan->lv) return;
    for (int m = 0; m < plan->lv->nlev; ++m) cudaFree(plan->lv->lev[m].map);
    cudaFree(plan->lv->spectra);
    cudaFree(plan->lv->phase);
    cudaFree(plan->lv->cphase);
    cudaFree(plan->lv->pspectra);
    delete plan->lv;
    plan->lv = nullptr;
}

sg_status sg_lv_setup(sg_plan *plan, const sg_lv_setup_args *a)
{
    sg_lv *lv = new (std::nothrow) sg_lv();
    if (!lv) return SG_ENOMEM;
    memset(lv, 0, sizeof(*lv));
    plan->lv = lv;
    lv->nlev = a->nlev;
    lv->px = a->px;
    lv->py = a->py;
    lv->hf = a->hf;
    const int qx = a->px / 2 + 1;
    const size_t cs = plan->prec == SG_FP64 ? sizeof(double2) : sizeof(float2);
    int64_t fwd = 0, spec = 0, inv = 0;
    for (int m = 0; m < a->nlev; ++m) {
        sg_lv_level &L = lv->lev[m];
        L.s = a->s[m];
        L.nx = a->nx[m];
        L.ny = a->ny[m];
        L.i0 = a->i0[m];
        L.j0 = a->j0[m];
        L.cx = sg_lv_cexp(L.s, a->px);
        L.cy = sg_lv_cexp(L.s, a->py);
        L.fwd_off = fwd;
        L.spec_off = spec;
        L.inv_off = inv;
        // every compact sample position lies in the first half of its transform
        // (the level's image is inside the finest extent, at most P/2 wide)
        if ((L.i0 >> L.cx) + ((int64_t)(L.nx - 1) << (L.s - L.cx)) >= (a->px >> L.cx) / 2 ||
            (L.j0 >> L.cy) + ((int64_t)(L.ny - 1) << (L.s - L.cy)) >= (a->py >> L.cy) / 2) {
            sg_set_last_error_message("level convolutions: a level image lies outside the padded lattice");
            return SG_EINVAL;
        }
        const int64_t qxc = (a->px >> L.cx) / 2 + 1;
        fwd += 3LL * qxc * L.ny;
        spec += 3LL * qxc * (a->py >> L.cy);
        inv += 2LL * qx * L.ny;
        SG_TRY(sg_plan_upload(plan, (void **)&L.map, a->map[m], (size_t)L.nx * L.ny * sizeof(int)));
    }
    lv->fwd_elems = fwd;
    lv->spec_elems = spec;
    lv->inv_elems = inv;
    // kernel keys: (width exponent of the source, 2 x sample shift)
    auto phi2 = [](int s) { return s >= 1 ? 1 : 0; };
    for (int m = 0; m < a->nlev; ++m) {
        for (int l = 0; l < a->nlev; ++l) {
            const int s = a->s[m], d2 = phi2(a->s[m]) - phi2(a->s[l]);
            int k = 0;
            while (k < lv->nkeys && !(lv->key_s[k] == s && lv->key_d2[k] == d2)) ++k;
            if (k == lv->nkeys) {
                lv->key_s[k] = s;
                lv->key_d2[k] = d2;
                ++lv->nkeys;
            }
            lv->key[m][l] = k;
        }
    }
    const size_t rs = cs / 2;  // real element
    const int64_t qplane = (int64_t)qx * sg_spec_stride(a->py);
    cudaError_t e = cudaMalloc(&lv->spectra, (size_t)lv->nkeys * 6 * qplane * rs);
    if (e == cudaSuccess) e = cudaMalloc(&lv->phase, (size_t)(a->px + a->py + 2) * cs);
    if (e == cudaSuccess) e = cudaMalloc(&lv->cphase, (size_t)(a->px + a->py + 2) * cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sg_set_last_cuda_error(e, "cudaMalloc");
        return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
    }
    plan->device_bytes += (int64_t)lv->nkeys * 6 * qplane * (int64_t)rs + 2 * (int64_t)(a->px + a->py + 2) * (int64_t)cs;
    if (plan->prec == SG_FP64) {
        k_lv_phase<double><<<16, 256>>>((double2 *)lv->phase, a->px, a->py);
        k_lv_cphase<double><<<16, 256>>>((double2 *)lv->cphase, a->px, a->py);
    } else {
        k_lv_phase<float><<<16, 256>>>((float2 *)lv->phase, a->px, a->py);
        k_lv_cphase<float><<<16, 256>>>((float2 *)lv->cphase, a->px, a->py);
    }
    // tables: FP64 wrapped, FP64 2-D transforms, unpacked and cast
    const int64_t plane = (int64_t)a->px * a->py;
    double2 *z = nullptr;
    e = cudaMalloc(&z, (size_t)(3 * plane * sizeof(double2)));
    if (e != cudaSuccess) {
        cudaGetLastError();
        sg_set_last_cuda_error(e, "cudaMalloc");
        return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
    }
    const double2 *twx = (const double2 *)((const char *)plan->twiddles + plan->tw64_off[sg_ilog2(a->px)]);
    const double2 *twy = (const double2 *)((const char *)plan->twiddles + plan->tw64_off[sg_ilog2(a->py)]);
    sg_status st = SG_OK;
    for (int k = 0; k < lv->nkeys && st == SG_OK; ++k) {
        k_lv_tables<<<2048, 256>>>(z, a->px, a->py, lv->key_s[k], lv->key_d2[k]);
        if (cudaGetLastError() != cudaSuccess) st = SG_ECUDA;
        for (int q = 0; q < 3 && st == SG_OK; ++q) {
            double2 *zq = z + q * plane;
            st = sg_fft_lines_fp64(zq, a->px, a->py, a->px, 1, twx);
            if (st == SG_OK) st = sg_fft_lines_fp64(zq, a->py, a->px, 1, a->px, twy);
        }
        if (st != SG_OK) break;
        char *dst = (char *)lv->spectra + (size_t)k * 6 * qplane * rs;
        const double G = plan->geom.G, Gh = plan->geom.G * a->hf;
        if (plan->prec == SG_FP64)
            k_lv_extract<double><<<2048, 256>>>(z, (double *)dst, a->px, a->py, lv->key_d2[k], G, Gh);
        else k_lv_extract<float><<<2048, 256>>>(z, (float *)dst, a->px, a->py, lv->key_d2[k], G, Gh);
        if (cudaGetLastError() != cudaSuccess) st = SG_ECUDA;
    }
    e = cudaDeviceSynchronize();
    cudaFree(z);
    if (st == SG_OK && e != cudaSuccess) {
        sg_set_last_cuda_error(e, "level-convolution tables");
        st = SG_ECUDA;
    }
    plan->ws_fwd_bytes = (lv->fwd_elems + lv->spec_elems) * (int64_t)cs;
    plan->ws_inv_bytes = lv->inv_elems * (int64_t)cs;
    return st;
}

sg_status sg_lv_potential_spectra_build(sg_plan *plan)
{
    sg_lv *lv = plan->lv;
    if (!lv) return SG_EINVAL;
    if (lv->pspectra) return SG_OK;
    const int px = lv->px, py = lv->py;
    const size_t rs = plan->prec == SG_FP64 ? sizeof(double) : sizeof(float);
    const int64_t qplane = (int64_t)(px / 2 + 1) * sg_spec_stride(py), plane = (int64_t)px * py;
    void *spec = nullptr;
    double2 *z = nullptr;
    cudaError_t e = cudaMalloc(&spec, (size_t)lv->nkeys * 3 * qplane * rs);
    if (e == cudaSuccess) e = cudaMalloc(&z, (size_t)(2 * plane * sizeof(double2)));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(spec);
        cudaFree(z);
        sg_set_last_cuda_error(e, "cudaMalloc");
        return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
    }
    const double2 *twx = (const double2 *)((const char *)plan->twiddles + plan->tw64_off[sg_ilog2(px)]);
    const double2 *twy = (const double2 *)((const char *)plan->twiddles + plan->tw64_off[sg_ilog2(py)]);
    // Phi = -G sum [sigma0 P^0 + deltax P^x + deltay P^y]: P^0 in units of h_f, P^x, P^y of h_f^2
    const double sc0 = -plan->geom.G * lv->hf, sc1 = -plan->geom.G * lv->hf * lv->hf;
    sg_status st = SG_OK;
    for (int k = 0; k < lv->nkeys && st == SG_OK; ++k) {
        k_lv_tables_pot<<<2048, 256>>>(z, px, py, lv->key_s[k], lv->key_d2[k]);
        if (cudaGetLastError() != cudaSuccess) st = SG_ECUDA;
        for (int q = 0; q < 2 && st == SG_OK; ++q) {
            double2 *zq = z + q * plane;
            st = sg_fft_lines_fp64(zq, px, py, px, 1, twx);
            if (st == SG_OK) st = sg_fft_lines_fp64(zq, py, px, 1, px, twy);
        }
        if (st != SG_OK) break;
        char *dst = (char *)spec + (size_t)k * 3 * qplane * rs;
        if (plan->prec == SG_FP64)
            k_lv_extract_pot<double><<<2048, 256>>>(z, (double *)dst, px, py, lv->key_d2[k], sc0, sc1);
        else k_lv_extract_pot<float><<<2048, 256>>>(z, (float *)dst, px, py, lv->key_d2[k], sc0, sc1);
        if (cudaGetLastError() != cudaSuccess) st = SG_ECUDA;
    }
    e = cudaDeviceSynchronize();
    cudaFree(z);
    if (st == SG_OK && e != cudaSuccess) {
        sg_set_last_cuda_error(e, "level-convolution potential tables");
        st = SG_ECUDA;
    }
    if (st != SG_OK) {
        cudaFree(spec);
        return st;
    }
    lv->pspectra = spec;
    plan->device_bytes += (int64_t)lv->nkeys * 3 * qplane * (int64_t)rs;
    return SG_OK;
}

sg_status sg_lv_potential(sg_plan *plan, const sg_workspace *ws, void *phi, cudaStream_t st)
{
    if (plan->prec == SG_FP64) return lv_solve_t<double>(plan, ws, phi, nullptr, true, st);
    return lv_solve_t<float>(plan, ws, phi, nullptr, true, st);
}

sg_status sg_lv_solve(sg_plan *plan, const sg_workspace *ws, void *fx, void *fy, cudaStream_t st)
{
    if (plan->prec == SG_FP64) return lv_solve_t<double>(plan, ws, fx, fy, false, st);
    return lv_solve_t<float>(plan, ws, fx, fy, false, st);
}
