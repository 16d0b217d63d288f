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
// ky in [0, py/2], scaled by 1 / (px py).
__host__ __device__ constexpr bool lv_plane_imag(int p) { return p == 0 || p == 3; }
__host__ __device__ constexpr int lv_plane_sy(int p) { return (p == 2 || p == 3 || p == 4) ? -1 : 1; }

// Unpack the transforms of the packed pairs (A + i B: A^(k) = (Z(k) + conj Z(-k)) / 2,
// B^(k) = (Z(k) - conj Z(-k)) / 2i), remove the half-cell phase and keep the real
// or imaginary part of every plane.
template <typename T>
__global__ void k_lv_extract(const double2 *z, T *out, int px, int py, int d2)
{
    const int qx = px / 2 + 1, qy = py / 2 + 1;
    const int64_t plane = (int64_t)px * py, qplane = (int64_t)qx * qy;
    const double sc = 1.0 / ((double)px * (double)py);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < qplane; e += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e / qy), ky = (int)(e % qy);
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
            out[pa[q] * qplane + e] = (T)(sc * (lv_plane_imag(pa[q]) ? hai : har));
            out[pb[q] * qplane + e] = (T)(sc * (lv_plane_imag(pb[q]) ? hbi : hbr));
        }
    }
}

// Phase factors exp(i pi k / P) for k in [-P/2, P/2] (index k + P/2), per axis.
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

// ----------------------------------------------------------- solve kernels --

template <typename T>
struct lv_rows_src {
    const T *S;         // composite source planes (sigma0, deltax, deltay), plane stride `plane`
    int64_t plane;
    const int *map;
    int nx, ny, i0, s;
};

template <typename T>
__device__ __forceinline__ T lv_sample(const lv_rows_src<T> &a, int f, int j, int I)
{
    if (j >= a.ny) return (T)0;
    const int rel = I - a.i0;
    if (rel < 0 || (rel & ((1 << a.s) - 1))) return (T)0;
    const int i = rel >> a.s;
    if (i >= a.nx) return (T)0;
    const int c = a.map[(int64_t)j * a.nx + i];
    return c < 0 ? (T)0 : a.S[f * a.plane + c];
}

// Row transforms of a level's sampled rows (three fields, blockIdx.y), two real
// rows per complex sequence; out[(f qx + kx) ny + j].
template <typename T, int PX, int NB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_lv_row_fwd(lv_rows_src<T> a, cplx_t<T> *__restrict__ out,
                                                        const cplx_t<T> *__restrict__ tw)
{
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    constexpr int RB = 2 * NB;
    constexpr int QX = PX / 2 + 1;
    const int f = blockIdx.y;
    const int j0 = blockIdx.x * RB;
    for (int e = threadIdx.x; e < NB * (PX / 2); e += THREADS) {
        const int q = e / (PX / 2), I = e % (PX / 2);
        const int ja = j0 + 2 * q;
        buf[spad<C>(q * PX + I)] = cmake<C>(lv_sample(a, f, ja, I), lv_sample(a, f, ja + 1, I));
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

// Column transforms to full spectra: the level's ny rows sit at finest rows
// j0 + j 2^s; spec[(f qx + kx) PY + ky].
template <typename T, int PY, int THREADS>
__global__ void __launch_bounds__(THREADS) k_lv_col_fwd(const cplx_t<T> *__restrict__ in, cplx_t<T> *__restrict__ spec,
                                                        int ny, int j0, int s, int qx, const cplx_t<T> *__restrict__ tw)
{
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int kx = blockIdx.x, f = blockIdx.y;
    for (int e = threadIdx.x; e < PY / 2; e += THREADS) buf[spad<C>(e)] = cmake<C>((T)0, (T)0);
    __syncthreads();
    const C *col = in + ((int64_t)f * qx + kx) * ny;
    for (int j = threadIdx.x; j < ny; j += THREADS) buf[spad<C>(j0 + (j << s))] = col[j];
    __syncthreads();
    fft_batch<C, PY, 1, THREADS, false, true>(buf, tw);
    C *o = spec + ((int64_t)f * qx + kx) * PY;
    for (int k = threadIdx.x; k < PY; k += THREADS) o[k] = buf[spad<C>(k)];
}

struct lv_mac_args {
    int nsrc;
    int64_t spec_off[SG_MAX_LEVELS];    // complex-element offset of each source level's spectra
    int key[SG_MAX_LEVELS];             // kernel of each source level for this target level
    int d2[SG_MAX_LEVELS];              // its 2 x sample shift
    int ny, j0, t;                      // target level: sampled rows j0 + j 2^t, j < ny
    int qx;
    double sc0, sc1;                    // G, and G h_f for the order-1 planes
};

// One column kx per CTA: Fx^, Fy^ = sum over source levels and fields of
// source spectrum x kernel spectrum (decompressed, see k_lv_extract), formed
// element by element straight into two shared buffers; inverse column
// transforms; the target level's sampled rows to out[(o qx + kx) ny + j].
template <typename T, int PY, int THREADS>
__global__ void __launch_bounds__(THREADS) k_lv_col_mac_inv(lv_mac_args a, const cplx_t<T> *__restrict__ spec,
                                                            const T *__restrict__ kspec,
                                                            const cplx_t<T> *__restrict__ phx,
                                                            const cplx_t<T> *__restrict__ phy,
                                                            cplx_t<T> *__restrict__ out,
                                                            const cplx_t<T> *__restrict__ tw)
{
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *bx = reinterpret_cast<C *>(smem_raw);
    C *by = bx + spad_size<C>(PY);
    constexpr int QY = PY / 2 + 1;
    const int kx = blockIdx.x;
    const int64_t sqplane = (int64_t)a.qx * PY, kqplane = (int64_t)a.qx * QY;
    // U bins per thread at a time, so that their loads are in flight together
    constexpr int UMAX = sizeof(T) == 8 ? 2 : 4;
    constexpr int U = PY / THREADS >= UMAX ? UMAX : PY / THREADS;
    for (int k0 = threadIdx.x; k0 < PY; k0 += U * THREADS) {
        int kq[U];
        bool lower[U];
        C pyk[U], ax[U], ay[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int ky = k0 + u * THREADS;
            lower[u] = ky <= PY / 2;
            kq[u] = lower[u] ? ky : PY - ky;
            pyk[u] = phy[(lower[u] ? ky : ky - PY) + PY / 2];
            ax[u] = ay[u] = cmake<C>((T)0, (T)0);
        }
        for (int m = 0; m < a.nsrc; ++m) {
            const C *sm = spec + a.spec_off[m] + (int64_t)kx * PY + k0;
            const T *km = kspec + (int64_t)a.key[m] * 6 * kqplane + (int64_t)kx * QY;
            C X[3][U];
            T gx[3][U], gy[3][U];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    X[f][u] = sm[f * sqplane + u * THREADS];
                    gx[f][u] = km[f * kqplane + kq[u]];
                    gy[f][u] = km[(3 + f) * kqplane + kq[u]];
                }
            }
            const int d2 = a.d2[m];
            const C phk = phx[kx + (a.qx - 1)];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                C hx = cmake<C>((T)0, (T)0), hy = cmake<C>((T)0, (T)0);
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const T sc = (T)(f == 0 ? a.sc0 : a.sc1);
                    T g1 = sc * gx[f][u], g2 = sc * gy[f][u];
                    if (!lower[u]) {
                        g1 *= (T)lv_plane_sy(f);
                        g2 *= (T)lv_plane_sy(3 + f);
                    }
                    const C Xv = X[f][u];
                    // real planes multiply by g, imaginary planes by i g
                    if (lv_plane_imag(f)) hx = cadd(hx, cmake<C>(-g1 * Xv.y, g1 * Xv.x));
                    else hx = cadd(hx, cmake<C>(g1 * Xv.x, g1 * Xv.y));
                    if (lv_plane_imag(3 + f)) hy = cadd(hy, cmake<C>(-g2 * Xv.y, g2 * Xv.x));
                    else hy = cadd(hy, cmake<C>(g2 * Xv.x, g2 * Xv.y));
                }
                if (d2 != 0) {
                    // half-cell phase exp(i pi d2 (kx / Px + ky / Py))
                    C ph = cmul(phk, pyk[u]);
                    if (d2 < 0) ph.y = -ph.y;
                    hx = cmul(hx, ph);
                    hy = cmul(hy, ph);
                }
                ax[u] = cadd(ax[u], hx);
                ay[u] = cadd(ay[u], hy);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            bx[spad<C>(k0 + u * THREADS)] = ax[u];
            by[spad<C>(k0 + u * THREADS)] = ay[u];
        }
    }
    __syncthreads();
    for (int o = 0; o < 2; ++o) {
        C *buf = o == 0 ? bx : by;
        fft_batch<C, PY, 1, THREADS, true, false, true>(buf, tw);
        C *dst = out + ((int64_t)o * a.qx + kx) * a.ny;
        for (int j = threadIdx.x; j < a.ny; j += THREADS) dst[j] = buf[spad<C>(a.j0 + (j << a.t))];
    }
}

struct lv_out_dst {
    const int *map;
    int nx, ny, i0, t;
};

// Inverse row transforms of a target level's rows (blockIdx.y = Fx, Fy); the
// samples at columns i0 + i 2^t go to the level's cells through the map.
template <typename T, int PX, int NB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_lv_row_inv(const cplx_t<T> *__restrict__ in, lv_out_dst a,
                                                        T *__restrict__ fx, T *__restrict__ fy,
                                                        const cplx_t<T> *__restrict__ tw)
{
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    constexpr int RB = 2 * NB;
    constexpr int QX = PX / 2 + 1;
    const int o = blockIdx.y;
    const int j0 = blockIdx.x * RB;
    const int ny = a.ny;
    const C *w = in + (int64_t)o * QX * ny;
    T *out = o == 0 ? fx : fy;
    for (int e = threadIdx.x; e < NB * QX; e += THREADS) {
        const int q = e % NB, k = e / NB;
        const int ja = j0 + 2 * q;
        C x = ja < ny ? w[(int64_t)k * ny + ja] : cmake<C>((T)0, (T)0);
        C y = ja + 1 < ny ? w[(int64_t)k * ny + ja + 1] : cmake<C>((T)0, (T)0);
        if (k == 0 || k == PX / 2) {
            x.y = (T)0;
            y.y = (T)0;
        }
        buf[spad<C>(q * PX + k)] = cmake<C>(x.x - y.y, x.y + y.x);
        if (k > 0 && k < PX / 2) buf[spad<C>(q * PX + PX - k)] = cmake<C>(x.x + y.y, y.x - x.y);
    }
    __syncthreads();
    fft_batch<C, PX, NB, THREADS, true, false, true>(buf, tw);
    for (int e = threadIdx.x; e < NB * a.nx; e += THREADS) {
        const int q = e / a.nx, i = e % a.nx;
        const int ja = j0 + 2 * q;
        const C zz = buf[spad<C>(q * PX + a.i0 + (i << a.t))];
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

constexpr int lv_nb(int px) { return px >= 4096 ? 1 : 4096 / px; }
constexpr int lv_row_threads(int px) { return lv_nb(px) * px / 8 > 512 ? 512 : lv_nb(px) * px / 8; }
constexpr int lv_col_threads(int py) { return py / 8 < 64 ? 64 : (py / 8 > 512 ? 512 : py / 8); }

template <typename K>
sg_status smem_attr(K kern, size_t bytes)
{
    if (bytes > 48 * 1024) SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return SG_OK;
}

template <typename T, int PX>
sg_status launch_row_fwd(const lv_rows_src<T> &a, cplx_t<T> *out, const cplx_t<T> *tw, cudaStream_t st)
{
    constexpr int NB = lv_nb(PX), TH = lv_row_threads(PX);
    const size_t sm = spad_size<cplx_t<T>>(NB * PX) * sizeof(cplx_t<T>);
    auto kern = k_lv_row_fwd<T, PX, NB, TH>;
    SG_TRY(smem_attr(kern, sm));
    dim3 grid((a.ny + 2 * NB - 1) / (2 * NB), 3);
    kern<<<grid, TH, sm, st>>>(a, out, tw);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PY>
sg_status launch_col_fwd(const cplx_t<T> *in, cplx_t<T> *spec, int ny, int j0, int s, int qx, const cplx_t<T> *tw,
                         cudaStream_t st)
{
    constexpr int TH = lv_col_threads(PY);
    const size_t sm = spad_size<cplx_t<T>>(PY) * sizeof(cplx_t<T>);
    auto kern = k_lv_col_fwd<T, PY, TH>;
    SG_TRY(smem_attr(kern, sm));
    kern<<<dim3(qx, 3), TH, sm, st>>>(in, spec, ny, j0, s, qx, tw);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PY>
sg_status launch_col_mac_inv(const lv_mac_args &a, const cplx_t<T> *spec, const T *kspec, const cplx_t<T> *phx,
                             const cplx_t<T> *phy, cplx_t<T> *out, const cplx_t<T> *tw, cudaStream_t st)
{
    constexpr int TH = lv_col_threads(PY);
    const size_t sm = 2 * spad_size<cplx_t<T>>(PY) * sizeof(cplx_t<T>);
    auto kern = k_lv_col_mac_inv<T, PY, TH>;
    SG_TRY(smem_attr(kern, sm));
    kern<<<a.qx, TH, sm, st>>>(a, spec, kspec, phx, phy, out, tw);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PX>
sg_status launch_row_inv(const cplx_t<T> *in, const lv_out_dst &a, T *fx, T *fy, const cplx_t<T> *tw, cudaStream_t st)
{
    constexpr int NB = lv_nb(PX), TH = lv_row_threads(PX);
    const size_t sm = spad_size<cplx_t<T>>(NB * PX) * sizeof(cplx_t<T>);
    auto kern = k_lv_row_inv<T, PX, NB, TH>;
    SG_TRY(smem_attr(kern, sm));
    dim3 grid((a.ny + 2 * NB - 1) / (2 * NB), 2);
    kern<<<grid, TH, sm, st>>>(in, a, fx, fy, tw);
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

template <typename T>
sg_status lv_solve_t(sg_plan *plan, const sg_workspace *ws, void *fx, void *fy, cudaStream_t st)
{
    using C = cplx_t<T>;
    const sg_lv &lv = *plan->lv;
    const int qx = lv.px / 2 + 1;
    const int64_t *twoff = sizeof(T) == 8 ? plan->tw64_off : plan->tw32_off;
    const C *twx = (const C *)((const char *)plan->twiddles + twoff[sg_ilog2(lv.px)]);
    const C *twy = (const C *)((const char *)plan->twiddles + twoff[sg_ilog2(lv.py)]);
    C *wf = (C *)ws->work_fwd;
    C *wi = (C *)ws->work_inv;
    C *spec = wf + lv.fwd_elems;
    const T *S = (const T *)ws->sfield;
    sg_timing_begin(ws, SG_STAGE_ROW_FWD, st);
    for (int m = 0; m < lv.nlev; ++m) {
        const sg_lv_level &L = lv.lev[m];
        lv_rows_src<T> a = {S, plan->ncells, L.map, L.nx, L.ny, L.i0, L.s};
        SG_LV_SWITCH(lv.px, SG_TRY((launch_row_fwd<T, PP>(a, wf + L.fwd_off, twx, st))));
    }
    sg_timing_end(ws, SG_STAGE_ROW_FWD, st);
    sg_timing_begin(ws, SG_STAGE_COL_CONV, st);
    for (int m = 0; m < lv.nlev; ++m) {
        const sg_lv_level &L = lv.lev[m];
        SG_LV_SWITCH(lv.py, SG_TRY((launch_col_fwd<T, PP>(wf + L.fwd_off, spec + L.spec_off, L.ny, L.j0, L.s, qx, twy, st))));
    }
    for (int l = 0; l < lv.nlev; ++l) {
        const sg_lv_level &L = lv.lev[l];
        lv_mac_args a;
        memset(&a, 0, sizeof(a));
        a.nsrc = lv.nlev;
        for (int m = 0; m < lv.nlev; ++m) {
            a.spec_off[m] = lv.lev[m].spec_off;
            a.key[m] = lv.key[m][l];
            a.d2[m] = lv.key_d2[lv.key[m][l]];
        }
        a.ny = L.ny;
        a.j0 = L.j0;
        a.t = L.s;
        a.qx = qx;
        a.sc0 = plan->geom.G;
        a.sc1 = plan->geom.G * lv.hf;
        const C *phx = (const C *)lv.phase, *phy = phx + lv.px + 1;
        SG_LV_SWITCH(lv.py, SG_TRY((launch_col_mac_inv<T, PP>(a, spec, (const T *)lv.spectra, phx, phy, wi + L.inv_off,
                                                               twy, st))));
    }
    sg_timing_end(ws, SG_STAGE_COL_CONV, st);
    sg_timing_begin(ws, SG_STAGE_ROW_INV, st);
    for (int l = 0; l < lv.nlev; ++l) {
        const sg_lv_level &L = lv.lev[l];
        lv_out_dst a = {L.map, L.nx, L.ny, L.i0, L.s};
        SG_LV_SWITCH(lv.px, SG_TRY((launch_row_inv<T, PP>(wi + L.inv_off, a, (T *)fx, (T *)fy, twx, st))));
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
        L.fwd_off = fwd;
        L.spec_off = spec;
        L.inv_off = inv;
        fwd += 3LL * qx * L.ny;
        spec += 3LL * qx * a->py;
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
    const int64_t qplane = (int64_t)qx * (a->py / 2 + 1);
    cudaError_t e = cudaMalloc(&lv->spectra, (size_t)lv->nkeys * 6 * qplane * rs);
    if (e == cudaSuccess) e = cudaMalloc(&lv->phase, (size_t)(a->px + a->py + 2) * cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sg_set_last_cuda_error(e, "cudaMalloc");
        return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
    }
    plan->device_bytes += (int64_t)lv->nkeys * 6 * qplane * (int64_t)rs + (int64_t)(a->px + a->py + 2) * (int64_t)cs;
    if (plan->prec == SG_FP64) k_lv_phase<double><<<16, 256>>>((double2 *)lv->phase, a->px, a->py);
    else k_lv_phase<float><<<16, 256>>>((float2 *)lv->phase, a->px, a->py);
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
        if (plan->prec == SG_FP64) k_lv_extract<double><<<2048, 256>>>(z, (double *)dst, a->px, a->py, lv->key_d2[k]);
        else k_lv_extract<float><<<2048, 256>>>(z, (float *)dst, a->px, a->py, lv->key_d2[k]);
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

sg_status sg_lv_solve(sg_plan *plan, const sg_workspace *ws, void *fx, void *fy, cudaStream_t st)
{
    if (plan->prec == SG_FP64) return lv_solve_t<double>(plan, ws, fx, fy, st);
    return lv_solve_t<float>(plan, ws, fx, fy, st);
}
