// Kernels of the uniform-patch force as a zero-padded 2-D FFT convolution (introduction and
// conclusion of Tseng, Shang & Yen; the uniform-grid route of Yen et al. 2012).
//
// For a patch of nx x ny cells padded to Px x Py (powers of two, P >= 2n - 1):
//   1. k_row_fwd : per row j < ny, the three input fields (sigma0, deltax,
//                  deltay; the slopes either read or formed by central
//                  differences on the fly, covered cells masked to zero) are
//                  real-to-complex transformed along x, two rows per complex
//                  FFT, and the Px/2+1 bins are written transposed:
//                  work_fwd[f][kx][j].
//   2. k_col_conv: per bin column kx, each field's column (ny values, zero
//                  padded to Py) is transformed along y, multiplied with the
//                  kernel spectra and accumulated into Fx^, Fy^ in registers:
//                    Fx^ = sigma^ (i a) + deltax^ b + deltay^ (s c)
//                    Fy^ = sigma^ (i s d) + deltay^ e + deltax^ (s f)
//                  (s = -1 for ky > Py/2: those planes are odd in ky); both are
//                  transformed back along y and the first ny rows written:
//                  work_inv[o][kx][j].
//   3. k_row_inv : per row j < ny, the two half spectra are inverse transformed
//                  along x (two rows per complex FFT) and the first nx values
//                  written to Fx, Fy. The spectra already carry G / (Px Py).
// Every transform is the shared-memory Stockham FFT of fft.cuh.
//
// Central slopes. When deltax, deltay are central differences of sigma with
// zero outside the patch, their transforms follow from sigma's exactly: along
// x the stencil (s[i+1] - s[i-1]) / 2h applied to the zero-padded row has the
// transform i sin(2 pi k / P) / h times sigma's, except that it also puts
// s[0] / 2h at i = -1 and -s[nx-1] / 2h at i = nx, outside the patch, whose
// transforms are removed again:
//   deltax^(kx, ky) = i sin(2 pi kx/Px)/h S - e^{+2 pi i kx/Px}/2h C0(ky) + e^{-2 pi i nx kx/Px}/2h C1(ky)
//   deltay^(kx, ky) = i sin(2 pi ky/Py)/h S - e^{+2 pi i ky/Py}/2h R0(kx) + e^{-2 pi i ny ky/Py}/2h R1(kx)
// with S = sigma^(kx, ky), C0 / C1 the y-transforms of sigma's first / last
// column (k_edge_cols), R0 / R1 the x-transforms of its first / last row (the
// column pass reads them from its own input). So only sigma is transformed:
// one row field and one forward column transform instead of three.
//
// The kernels and their launch-shape variants are split over translation
// units by stage (fftconv_rows.cu, fftconv_cols.cu, fftconv_central.cu); the
// solve (fftconv.cu) calls them through the dispatchers declared below with
// the launch shapes of the tuning table (tune.cu).
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "tma.cuh"

namespace sgk {

template <typename T>
struct field_src {
    const T *sigma, *dx, *dy;
    int nx, ny;
    T inv2h;
    int mode;          // sg_slope_mode
};

template <typename T>
__device__ __forceinline__ T sigma_at(const field_src<T> &s, int j, int i)
{
    if (i < 0 || i >= s.nx || j < 0 || j >= s.ny) return (T)0;
    return s.sigma[(int64_t)j * s.nx + i];
}

template <typename T>
__device__ __forceinline__ T field_value(const field_src<T> &s, int f, int j, int i)
{
    if (j >= s.ny || i >= s.nx) return (T)0;
    const int64_t o = (int64_t)j * s.nx + i;
    if (f == 0) return s.sigma[o];
    if (s.mode == SG_SLOPES_CALLER) return f == 1 ? s.dx[o] : s.dy[o];
    // central differences, zero beyond the patch edge
    if (f == 1) return (sigma_at(s, j, i + 1) - sigma_at(s, j, i - 1)) * s.inv2h;
    return (sigma_at(s, j + 1, i) - sigma_at(s, j - 1, i)) * s.inv2h;
}

// Per-solve arguments of the passes. A kernel instantiated with BATCH = true
// runs one member of a batch per blockIdx.z, its arguments read from a device
// array (members of one padded length share the launch; CTAs beyond a member's
// own row count return at once); with BATCH = false it runs the solve passed by
// value.
template <typename T>
struct row_fwd_args {
    field_src<T> src;
    cplx_t<T> *work;
};
template <typename T>
struct col_args {
    const cplx_t<T> *wf;
    cplx_t<T> *wi;
    const T *spec;
    const cplx_t<T> *edge;   // central slopes: sigma's edge-column transforms
    const T *phase;          // central slopes: spectral factors
    int ny;
    int tries;               // attempts of the bounded wait for the spectra (the plan's wait limit)
};
template <typename T>
struct row_inv_args {
    const cplx_t<T> *wi;
    T *fx, *fy, *fz;
    int nx, ny;
};
template <typename T>
struct edge_args {
    const T *sigma;
    int nx, ny;
    cplx_t<T> *edge;
};

// Global-to-shared staging loops issue LOAD_UNROLL loads per thread before
// their shared-memory stores, so that these loads are in flight together.
constexpr int LOAD_UNROLL = 4;

template <bool BATCH, typename A>
__device__ __forceinline__ A pass_args(const A &one, const A *__restrict__ many)
{
    if constexpr (BATCH) return many[blockIdx.z];
    return one;
}

// ---------------------------------------------------------------- kernels --

// Every pass is a device body run by one CTA on one tile of its work (row
// group bx, field or output f, column group bx), called by the pass's kernel
// with blockIdx and by the persistent batch kernel (batch_run.inl) with the
// coordinates of a work item; both run the same arithmetic (the central column
// pass's kernel holds its own copy of that arithmetic; see there). With CO (the
// persistent kernel) buffers that an earlier pass wrote are read with coherent
// loads (__ldcg for data read once, __ldca for tables every CTA reads) rather
// than through the non-coherent read-only path, since that pass ran in the same
// launch (they are read only after its items completed, by SMs that had not
// read them); the pass kernels keep plain loads of the spectra and the
// read-only path for tables (CO = false; an __ldg of the spectra measured
// slower in the column pass).
template <bool CO, typename X>
__device__ __forceinline__ X ld_plain(const X *p)
{
    if constexpr (CO) return __ldcg(p);
    return *p;
}
template <bool CO, typename X>
__device__ __forceinline__ X ld_table(const X *p)
{
    if constexpr (CO) return __ldca(p);
    return __ldg(p);
}
// Two adjacent FP32 complex values (16-byte aligned) in one load, through the
// same path as ld_plain; FP64 (not used there): two loads.
template <bool CO, typename C>
__device__ __forceinline__ void ld_pair_plain(const C *p, C &a, C &b)
{
    if constexpr (sizeof(C) == 8) {
        const float4 q = ld_plain<CO>(reinterpret_cast<const float4 *>(p));
        a = make_float2(q.x, q.y);
        b = make_float2(q.z, q.w);
    } else {
        a = ld_plain<CO>(p);
        b = ld_plain<CO>(p + 1);
    }
}
// The pair (a, b) at index k of an array of interleaved complex pairs: one
// 16-byte load in FP32 (the array 16-byte aligned), two in FP64.
template <bool CO, typename C>
__device__ __forceinline__ void ld_pair(const C *p, int k, C &a, C &b)
{
    if constexpr (sizeof(C) == 8) {
        const float4 q = ld_table<CO>(reinterpret_cast<const float4 *>(p) + k);
        a = make_float2(q.x, q.y);
        b = make_float2(q.z, q.w);
    } else {
        a = ld_table<CO>(p + 2 * k);
        b = ld_table<CO>(p + 2 * k + 1);
    }
}
template <typename T, int PX, int NB, int THREADS, bool WAIT_AT_END = false>
__device__ __forceinline__ void row_fwd_body(const row_fwd_args<T> &args, int bx, int f,
                                             const cplx_t<T> *__restrict__ tw)
{
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    constexpr int RB = 2 * NB;
    constexpr int QX = PX / 2 + 1;
    const field_src<T> &src = args.src;
    cplx_t<T> *__restrict__ work = args.work;
    const int j0 = bx * RB;
    const int ny = src.ny;
    if (j0 >= ny) return;
    // WAIT_AT_END: launched after the edge-column transform, which waited for the
    // previous solve before letting this kernel start, so the scratch is free
    // now; the wait at the end makes this kernel's completion imply the edge
    // transform's (CTA 0 always reaches it)
    if constexpr (!WAIT_AT_END) sg_dep_wait();

    // two rows per complex sequence: z = row(2s) + i row(2s+1); positions >= PX/2 are zero
    constexpr int NE = NB * (PX / 2);
    for (int e0 = threadIdx.x; e0 < NE; e0 += LOAD_UNROLL * THREADS) {
        T a[LOAD_UNROLL], b[LOAD_UNROLL];
#pragma unroll
        for (int u = 0; u < LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS;
            a[u] = b[u] = (T)0;
            if (e < NE) {
                const int s = e / (PX / 2), i = e % (PX / 2);
                const int ja = j0 + 2 * s;
                a[u] = field_value(src, f, ja, i);
                b[u] = field_value(src, f, ja + 1, i);
            }
        }
#pragma unroll
        for (int u = 0; u < LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS;
            if (e < NE) buf[spad<C>((e / (PX / 2)) * PX + e % (PX / 2))] = cmake<C>(a[u], b[u]);
        }
    }
    __syncthreads();
    fft_batch<C, PX, NB, THREADS, false, true>(buf, tw);

    // unpack: A[k] = (Z[k] + conj Z[-k]) / 2, B[k] = (Z[k] - conj Z[-k]) / 2i
    const T half = (T)0.5;
    for (int e = threadIdx.x; e < QX * RB; e += THREADS) {
        const int kx = e / RB, r = e % RB;
        const int j = j0 + r;
        if (j >= ny) continue;
        const int s = r >> 1;
        const C z = buf[spad<C>(s * PX + kx)];
        const C w = buf[spad<C>(s * PX + ((PX - kx) & (PX - 1)))];
        C out;
        if ((r & 1) == 0) out = cmake<C>(half * (z.x + w.x), half * (z.y - w.y));
        else out = cmake<C>(half * (z.y + w.y), half * (w.x - z.x));
        work[((int64_t)f * QX + kx) * ny + j] = out;
    }
    if constexpr (WAIT_AT_END) sg_dep_wait();
}

template <typename T, int PX, int NB, int THREADS, bool BATCH = false, bool WAIT_AT_END = false>
__global__ void __launch_bounds__(THREADS) k_row_fwd(row_fwd_args<T> one, const row_fwd_args<T> *__restrict__ many,
                                                     const cplx_t<T> *__restrict__ tw)
{
    sg_dep_trigger();
    const row_fwd_args<T> args = pass_args<BATCH>(one, many);
    row_fwd_body<T, PX, NB, THREADS, WAIT_AT_END>(args, blockIdx.x, blockIdx.y, tw);
}

// Shared-memory layout of the column kernels: the padded FFT buffer, then the
// kernel spectra of the CTA's columns, [planes][CB][sg_spec_stride(PY)] of T,
// which one thread fetches with one 1-D bulk copy (TMA) per plane at kernel
// start so that they arrive while the forward transform runs.
// Column kernels keep each column in registers between transform stages and
// exchange through col_nbuf shared buffers (fft_regs in fft.cuh): two (one
// barrier per exchange), except FP64 columns of 4096 points, whose two buffers
// and six spectrum planes would exceed a CTA's 227 KB: one buffer there (a
// barrier before each transform's first exchange).
template <typename T, int PY>
__host__ __device__ constexpr int col_nbuf() { return sizeof(T) == 8 && PY >= 4096 ? 1 : 2; }
// The central-slope pass kernel on FP32 2048-point columns, one column per CTA,
// runs four CTAs per SM instead of three (1025 columns in 1.7 waves instead of
// 2.25): 64 registers (one spilled) and one exchange buffer, so that four CTAs'
// buffers and spectrum planes (41 KB each) fit in an SM's shared memory.
// Measured 28.3 -> 27.2 us per pass at 2048 x 2048; the caller-slope pass
// spills 100 bytes at 64 registers and keeps three.
template <typename T, int PY, int CB>
__host__ __device__ constexpr bool col_central_four() { return sizeof(T) == 4 && PY == 2048 && CB == 1; }
template <typename T, int PY, int CB>
__host__ __device__ constexpr int col_central_nbuf() { return col_central_four<T, PY, CB>() ? 1 : col_nbuf<T, PY>(); }
template <typename T, int PY, int CB, int NB = col_nbuf<T, PY>()>
__host__ __device__ constexpr int col_buf_bytes() { return NB * ((spad_size<cplx_t<T>>(CB * PY) * (int)sizeof(cplx_t<T>) + 15) & ~15); }
template <typename T, int PY, int CB, int NPL = 6, int NB = col_nbuf<T, PY>()>
__host__ __device__ constexpr int col_smem_bytes() { return col_buf_bytes<T, PY, CB, NB>() + CB * NPL * ((PY / 2 + 1 + 3) & ~3) * (int)sizeof(T); }

template <typename T, int PY, int CB, int NPL = 6, bool CO = false>
__device__ __forceinline__ void fetch_spectra(T *ssp, const T *__restrict__ spec, int kx0, int qx, uint64_t *bar)
{
    constexpr int QS = (PY / 2 + 1 + 3) & ~3;
    const int ncol = qx - kx0 < CB ? qx - kx0 : CB;
    const int64_t qplane = (int64_t)qx * QS;
    if constexpr (CO) fence_proxy_async_smem();  // shared memory an earlier body in the same CTA used
    mbar_arrive_expect_tx(bar, (uint32_t)(ncol * NPL * QS * sizeof(T)));
    // the CTA's columns are consecutive rows of every plane: one copy per plane
    for (int p = 0; p < NPL; ++p)
        bulk_copy_g2s(ssp + p * CB * QS, spec + p * qplane + (int64_t)kx0 * QS, ncol * QS * sizeof(T), bar);
}

// Bounded wait for the spectra (`tries` attempts); on timeout records the
// error, waits for the copies in flight (bounded, full limit) and tells the CTA
// to return (uniformly).
__device__ __forceinline__ bool spectra_ready(uint64_t *bar, int *err, int tries)
{
    const bool ok = mbar_wait_bounded(bar, 0, tries);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            mbar_wait_bounded(bar, 0, SG_MBAR_MAX_TRIES);
        }
        __syncthreads();
        return false;
    }
    return true;
}

// resident CTAs per SM asked of the register allocator (spill-free choices at
// the default shapes, scaled by the CTA size for the other candidates). FP32
// 2048-point columns: the two exchange buffers and six spectrum planes take
// 59.5 KB of shared memory, so three CTAs fit per SM: 80 registers each (the
// central-slope pass kernel's four-CTA form, above, overrides this).
template <typename T, int PY, int NOUT>
constexpr int col_min_blocks_def()
{
    return sizeof(T) == 4 ? (PY == 2048 ? (NOUT == 3 ? 2 : 3) : (PY == 4096 ? 1 : 2)) : 1;
}
template <typename T, int PY, int THREADS, int NOUT = 2>
constexpr int col_min_blocks()
{
    constexpr int def_threads = (PY >= 2048 ? 1 : 2048 / PY) * PY / 8;
    constexpr int d = col_min_blocks_def<T, PY, NOUT>();
    return d * def_threads / THREADS >= 1 ? d * def_threads / THREADS : 1;
}

template <typename T, int PY, int CB, int THREADS, int NOUT, bool CO = false>
__device__ __forceinline__ void col_body(const col_args<T> &args, int bx, int qx, int nf,
                                         const cplx_t<T> *__restrict__ tw, int *err)
{
    using C = cplx_t<T>;
    const cplx_t<T> *__restrict__ work_fwd = args.wf;
    cplx_t<T> *__restrict__ work_inv = args.wi;
    const T *__restrict__ spec = args.spec;
    const int ny = args.ny;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *bufs = reinterpret_cast<C *>(smem_raw);
    T *ssp = reinterpret_cast<T *>(smem_raw + col_buf_bytes<T, PY, CB>());
    __shared__ uint64_t bar;
    static_assert(CB * PY / THREADS == 8, "eight elements per thread");
    constexpr int QS = (PY / 2 + 1 + 3) & ~3;
    constexpr int STEP = PY / 8;
    const int kx0 = bx * CB;
    // this thread's column and the rows it holds: jt + m PY/8, m = 0..7
    const int c = threadIdx.x / STEP, jt = threadIdx.x % STEP;
    const int kx = kx0 + c;
    constexpr int NPL = NOUT == 3 ? 9 : (NOUT == 1 ? 3 : 6);
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) fetch_spectra<T, PY, CB, NPL, CO>(ssp, spec, kx0, qx, &bar);
    sg_dep_wait();  // the row pass's output (the kernel spectra are the plan's own)

    C accx[8], accy[8], accz[NOUT == 3 ? 8 : 1];
#pragma unroll
    for (int q = 0; q < 8; ++q) accx[q] = accy[q] = cmake<C>((T)0, (T)0);
#pragma unroll
    for (int q = 0; q < (NOUT == 3 ? 8 : 1); ++q) accz[q] = cmake<C>((T)0, (T)0);

    int par = 0;
    for (int f = 0; f < nf; ++f) {
        // the lower half of the column straight into registers (the upper half is zero)
        C v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int j = jt + m * STEP;
            v[m] = (m < 4 && j < ny && kx < qx) ? ld_plain<CO>(&work_fwd[((int64_t)f * qx + kx) * ny + j])
                                                : cmake<C>((T)0, (T)0);
        }
        if (col_nbuf<T, PY>() == 1 && f > 0) __syncthreads();
        fft_regs<C, PY, CB, THREADS, col_nbuf<T, PY>(), false>(v, bufs, par, tw);
        if (f == 0) {
            if (!spectra_ready(&bar, err, args.tries)) return;
            if (CO && threadIdx.x == 0) mbar_inval(&bar);  // every thread has passed its wait; the body runs again
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int ky = jt + q * STEP;
            if (kx >= qx) continue;
            const bool lower = ky <= PY / 2;
            const int kq = lower ? ky : PY - ky;
            const T sg = lower ? (T)1 : (T)-1;
            const T *sp = ssp + c * QS + kq;  // plane p at sp[p * CB * QS]
            const C X = v[q];
            // explicitly rounded (see mul_rn): the result must not depend on the launch shape
            if constexpr (NOUT == 1) {
                // potential planes: p (real, even-even), a (i a: odd in kx), b (i b: odd in ky)
                if (f == 0) {
                    const T pp = sp[0];
                    accx[q] = cmake<C>(mul_rn(pp, X.x), mul_rn(pp, X.y));
                } else {
                    const T g = f == 1 ? sp[1 * CB * QS] : sg * sp[2 * CB * QS];
                    accx[q] = cmake<C>(fma(-g, X.y, accx[q].x), fma(g, X.x, accx[q].y));
                }
                continue;
            }
            if (f == 0) {
                const T a = sp[0 * CB * QS];
                const T d = sg * sp[3 * CB * QS];
                accx[q] = cmake<C>(-mul_rn(a, X.y), mul_rn(a, X.x));
                accy[q] = cmake<C>(-mul_rn(d, X.y), mul_rn(d, X.x));
                if constexpr (NOUT == 3) {
                    const T g = sp[6 * CB * QS];  // real: sigma^ g
                    accz[q] = cmake<C>(mul_rn(g, X.x), mul_rn(g, X.y));
                }
            } else if (f == 1) {
                const T b = sp[1 * CB * QS];
                const T ff = sg * sp[5 * CB * QS];
                accx[q] = cmake<C>(fma(b, X.x, accx[q].x), fma(b, X.y, accx[q].y));
                accy[q] = cmake<C>(fma(ff, X.x, accy[q].x), fma(ff, X.y, accy[q].y));
                if constexpr (NOUT == 3) {
                    const T hh = sp[7 * CB * QS];  // imaginary: deltax^ (i hh)
                    accz[q] = cmake<C>(fma(-hh, X.y, accz[q].x), fma(hh, X.x, accz[q].y));
                }
            } else {
                const T cc = sg * sp[2 * CB * QS];
                const T ee = sp[4 * CB * QS];
                accx[q] = cmake<C>(fma(cc, X.x, accx[q].x), fma(cc, X.y, accx[q].y));
                accy[q] = cmake<C>(fma(ee, X.x, accy[q].x), fma(ee, X.y, accy[q].y));
                if constexpr (NOUT == 3) {
                    const T kk = sg * sp[8 * CB * QS];  // imaginary, odd in ky: deltay^ (i s kk)
                    accz[q] = cmake<C>(fma(-kk, X.y, accz[q].x), fma(kk, X.x, accz[q].y));
                }
            }
        }
    }

    // inverse transforms: the accumulators are already in the transform's input pattern
#pragma unroll 1
    for (int o = 0; o < NOUT; ++o) {
        C v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = o == 0 ? accx[q] : accy[q];
            if constexpr (NOUT == 3) {
                if (o == 2) v[q] = accz[q];
            }
        }
        if (col_nbuf<T, PY>() == 1) __syncthreads();
        fft_regs<C, PY, CB, THREADS, col_nbuf<T, PY>(), true>(v, bufs, par, tw);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = jt + m * STEP;
            if (j < ny && kx < qx) work_inv[((int64_t)o * qx + kx) * ny + j] = v[m];
        }
    }
}

template <typename T, int PY, int CB, int THREADS, int NOUT, bool BATCH = false>
__global__ void __launch_bounds__(THREADS, (col_min_blocks<T, PY, THREADS, NOUT>())) k_col_conv(col_args<T> one, const col_args<T> *__restrict__ many,
                                                      int qx, int nf, const cplx_t<T> *__restrict__ tw, int *err)
{
    sg_dep_trigger();
    const col_args<T> args = pass_args<BATCH>(one, many);
    col_body<T, PY, CB, THREADS, NOUT>(args, blockIdx.x, qx, nf, tw, err);
}

template <typename T, int PX, int NB, int THREADS, bool CO = false>
__device__ __forceinline__ void row_inv_body(const row_inv_args<T> &args, int bx, int o,
                                             const cplx_t<T> *__restrict__ tw)
{
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    constexpr int RB = 2 * NB;
    constexpr int QX = PX / 2 + 1;
    const cplx_t<T> *__restrict__ work_inv = args.wi;
    T *fx = args.fx, *fy = args.fy, *fz = args.fz;
    const int nx = args.nx, ny = args.ny;
    const int j0 = bx * RB;
    if (j0 >= ny) return;
    sg_dep_wait();
    const C *w = work_inv + (int64_t)o * QX * ny;
    T *out = o == 0 ? fx : (o == 1 ? fy : fz);

    // Z[k] = A[k] + i B[k] over the full length, from the half spectra of rows 2s, 2s+1.
    // In FP32 with an even row count the two rows' values of a column are one
    // aligned 16-byte pair (ja is even): one load instead of two.
    constexpr int NE = NB * QX;
    const bool pairs = sizeof(C) == 8 && (ny & 1) == 0;
    for (int e0 = threadIdx.x; e0 < NE; e0 += LOAD_UNROLL * THREADS) {
        C av[LOAD_UNROLL], bv[LOAD_UNROLL];
#pragma unroll
        for (int u = 0; u < LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS, s = e % NB, k = e / NB, ja = j0 + 2 * s;
            if (pairs) {
                av[u] = bv[u] = cmake<C>((T)0, (T)0);
                if (e < NE && ja < ny) ld_pair_plain<CO>(&w[(int64_t)k * ny + ja], av[u], bv[u]);
            } else {
                av[u] = (e < NE && ja < ny) ? ld_plain<CO>(&w[(int64_t)k * ny + ja]) : cmake<C>((T)0, (T)0);
                bv[u] = (e < NE && ja + 1 < ny) ? ld_plain<CO>(&w[(int64_t)k * ny + ja + 1]) : cmake<C>((T)0, (T)0);
            }
        }
#pragma unroll
        for (int u = 0; u < LOAD_UNROLL; ++u) {
            const int e = e0 + u * THREADS, s = e % NB, k = e / NB;
            if (e >= NE) continue;
            C a = av[u], b = bv[u];
            if (k == 0 || k == PX / 2) {
                a.y = (T)0;
                b.y = (T)0;
            }
            buf[spad<C>(s * PX + k)] = cmake<C>(a.x - b.y, a.y + b.x);
            if (k > 0 && k < PX / 2) buf[spad<C>(s * PX + PX - k)] = cmake<C>(a.x + b.y, b.x - a.y);  // conj(a) + i conj(b)
        }
    }
    __syncthreads();
    fft_batch<C, PX, NB, THREADS, true, false, true>(buf, tw);
    for (int e = threadIdx.x; e < NB * PX; e += THREADS) {
        const int s = e / PX, i = e % PX;
        if (i >= nx) continue;
        const int ja = j0 + 2 * s;
        const C z = buf[spad<C>(e)];
        if (ja < ny) out[(int64_t)ja * nx + i] = z.x;
        if (ja + 1 < ny) out[(int64_t)(ja + 1) * nx + i] = z.y;
    }
}

template <typename T, int PX, int NB, int THREADS, bool BATCH = false>
__global__ void __launch_bounds__(THREADS) k_row_inv(row_inv_args<T> one, const row_inv_args<T> *__restrict__ many,
                                                     const cplx_t<T> *__restrict__ tw)
{
    sg_dep_trigger();
    const row_inv_args<T> args = pass_args<BATCH>(one, many);
    row_inv_body<T, PX, NB, THREADS>(args, blockIdx.x, blockIdx.y, tw);
}

// y-transforms of sigma's first and last columns, packed as z = c0 + i c1:
// edge[2k] = C0(k), edge[2k + 1] = C1(k), k < PY (pairs: one load per bin).
template <typename T, int PY, int THREADS>
__device__ __forceinline__ void edge_body(const edge_args<T> &args, const cplx_t<T> *__restrict__ tw)
{
    using C = cplx_t<T>;
    const T *__restrict__ sigma = args.sigma;
    const int nx = args.nx, ny = args.ny;
    cplx_t<T> *__restrict__ edge = args.edge;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    for (int j = threadIdx.x; j < PY / 2; j += THREADS) {  // positions >= PY/2 are zero
        const T a = j < ny ? sigma[(int64_t)j * nx] : (T)0;
        const T b = j < ny ? sigma[(int64_t)j * nx + nx - 1] : (T)0;
        buf[spad<C>(j)] = cmake<C>(a, b);
    }
    __syncthreads();
    fft_batch<C, PY, 1, THREADS, false, true>(buf, tw);
    const T half = (T)0.5;
    for (int k = threadIdx.x; k < PY; k += THREADS) {
        const C z = buf[spad<C>(k)];
        const C w = buf[spad<C>((PY - k) & (PY - 1))];
        edge[2 * k] = cmake<C>(half * (z.x + w.x), half * (z.y - w.y));
        edge[2 * k + 1] = cmake<C>(half * (z.y + w.y), half * (w.x - z.x));
    }
}

template <typename T, int PY, int THREADS, bool BATCH = false>
__global__ void __launch_bounds__(THREADS) k_edge_cols(edge_args<T> one, const edge_args<T> *__restrict__ many,
                                                       const cplx_t<T> *__restrict__ tw)
{
    // the first kernel of a central-slope solve: it waits for the previous
    // kernel of the stream (its scratch is the solve's scratch), then lets the
    // row pass start beside it (k_row_fwd with WAIT_AT_END), whose completion
    // then implies this kernel's for the column pass after them
    sg_dep_wait();
    sg_dep_trigger();
    const edge_args<T> args = pass_args<BATCH>(one, many);
    edge_body<T, PY, THREADS>(args, tw);
}

// Column pass for central slopes: one forward transform (sigma), the slope
// spectra formed per bin (see the header comment), two inverse transforms.
template <typename T, int PY, int CB, int THREADS, bool CO = false>
__device__ __forceinline__ void col_central_body(const col_args<T> &args, int bx, int qx,
                                                 const cplx_t<T> *__restrict__ tw, int *err)
{
    using C = cplx_t<T>;
    const cplx_t<T> *__restrict__ work_fwd = args.wf;
    cplx_t<T> *__restrict__ work_inv = args.wi;
    const T *__restrict__ spec = args.spec;
    const cplx_t<T> *__restrict__ edge = args.edge;
    const T *__restrict__ phase = args.phase;
    const int ny = args.ny;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *bufs = reinterpret_cast<C *>(smem_raw);
    T *ssp = reinterpret_cast<T *>(smem_raw + col_buf_bytes<T, PY, CB>());
    __shared__ uint64_t bar;
    __shared__ C rows[CB][2];  // R0, R1 of each column
    static_assert(CB * PY / THREADS == 8, "eight elements per thread");
    constexpr int QS = (PY / 2 + 1 + 3) & ~3;
    constexpr int STEP = PY / 8;
    const int kx0 = bx * CB;
    const int c = threadIdx.x / STEP, jt = threadIdx.x % STEP;
    const int kx = kx0 + c;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) fetch_spectra<T, PY, CB, 6, CO>(ssp, spec, kx0, qx, &bar);
    sg_dep_wait();  // the row pass's output (the kernel spectra are the plan's own)
    const C *cpair = reinterpret_cast<const C *>(phase), *rpair = cpair + 2 * qx;  // (e1, e2) per kx, per ky

    // the lower half of the column straight into registers (the upper half is zero)
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int j = jt + m * STEP;
        v[m] = (m < 4 && j < ny && kx < qx) ? ld_plain<CO>(&work_fwd[(int64_t)kx * ny + j]) : cmake<C>((T)0, (T)0);
    }
    // the column's first and last rows (read after the transform's barriers)
    if (jt == 0) rows[c][0] = v[0];
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (jt + m * STEP == ny - 1) rows[c][1] = v[m];
    int par = 0;
    fft_regs<C, PY, CB, THREADS, col_nbuf<T, PY>(), false>(v, bufs, par, tw);
    if (!spectra_ready(&bar, err, args.tries)) return;
    if (CO && threadIdx.x == 0) mbar_inval(&bar);  // every thread has passed its wait; the body runs again

    C accx[8], accy[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int ky = jt + q * STEP;
        accx[q] = accy[q] = cmake<C>((T)0, (T)0);
        if (kx >= qx) continue;
        const bool lower = ky <= PY / 2;
        const int kq = lower ? ky : PY - ky;
        const T sg = lower ? (T)1 : (T)-1;
        const T *sp = ssp + c * QS + kq;  // plane p at sp[p * CB * QS]
        const C S = v[q];
        // slope spectra
        C e1, e2, f1, f2;
        ld_pair<false>(cpair, kx, e1, e2);
        ld_pair<false>(rpair, ky, f1, f2);
        const T cs = (T)2 * e1.y, rs = (T)2 * f1.y;  // sin(2 pi k / P) / h, exactly
        C c0, c1;
        ld_pair<CO>(edge, ky, c0, c1);
        // every operation explicitly rounded (see mul_rn): the result must not depend on the launch shape
        const C p2 = cmul_rn(e2, c1), p1 = cmul_rn(e1, c0);
        const C q2 = cmul_rn(f2, rows[c][1]), q1 = cmul_rn(f1, rows[c][0]);
        const C X = cmake<C>(add_rn(add_rn(-mul_rn(cs, S.y), p2.x), -p1.x), add_rn(add_rn(mul_rn(cs, S.x), p2.y), -p1.y));
        const C Y = cmake<C>(add_rn(add_rn(-mul_rn(rs, S.y), q2.x), -q1.x), add_rn(add_rn(mul_rn(rs, S.x), q2.y), -q1.y));
        const T a = sp[0 * CB * QS];
        const T b = sp[1 * CB * QS];
        const T cc = sg * sp[2 * CB * QS];
        const T d = sg * sp[3 * CB * QS];
        const T ee = sp[4 * CB * QS];
        const T ff = sg * sp[5 * CB * QS];
        accx[q] = cmake<C>(fma(cc, Y.x, fma(b, X.x, -mul_rn(a, S.y))), fma(cc, Y.y, fma(b, X.y, mul_rn(a, S.x))));
        accy[q] = cmake<C>(fma(ff, X.x, fma(ee, Y.x, -mul_rn(d, S.y))), fma(ff, X.y, fma(ee, Y.y, mul_rn(d, S.x))));
    }

    // inverse transforms: the products are already in the transform's input pattern
    if (col_nbuf<T, PY>() == 1) __syncthreads();
    fft_regs<C, PY, CB, THREADS, col_nbuf<T, PY>(), true>(accx, bufs, par, tw);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int j = jt + m * STEP;
        if (j < ny && kx < qx) work_inv[(int64_t)kx * ny + j] = accx[m];
    }
    if (col_nbuf<T, PY>() == 1) __syncthreads();
    fft_regs<C, PY, CB, THREADS, col_nbuf<T, PY>(), true>(accy, bufs, par, tw);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int j = jt + m * STEP;
        if (j < ny && kx < qx) work_inv[((int64_t)qx + kx) * ny + j] = accy[m];
    }
}


// The pass kernel for one solve or a batch of launches keeps its own copy of
// col_central_body's arithmetic, operation for operation: compiled through the
// inlined body it ran 19% slower (32.8 against 27.6 us at 2048 x 2048, FP32;
// same registers, more time waiting on global loads). The batch tests check that
// the persistent kernel (which runs the body) and this kernel agree bit for bit.
template <typename T, int PY, int CB, int THREADS, bool BATCH = false>
__global__ void __launch_bounds__(THREADS, (col_central_four<T, PY, CB>() ? 4 : col_min_blocks<T, PY, THREADS>())) k_col_conv_central(
    col_args<T> one, const col_args<T> *__restrict__ many, int qx, const cplx_t<T> *__restrict__ tw, int *err)
{
    using C = cplx_t<T>;
    sg_dep_trigger();
    const col_args<T> args = pass_args<BATCH>(one, many);
    const cplx_t<T> *__restrict__ work_fwd = args.wf;
    cplx_t<T> *__restrict__ work_inv = args.wi;
    const T *__restrict__ spec = args.spec;
    const cplx_t<T> *__restrict__ edge = args.edge;
    const T *__restrict__ phase = args.phase;
    const int ny = args.ny;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *bufs = reinterpret_cast<C *>(smem_raw);
    T *ssp = reinterpret_cast<T *>(smem_raw + col_buf_bytes<T, PY, CB, col_central_nbuf<T, PY, CB>()>());
    __shared__ uint64_t bar;
    __shared__ C rows[CB][2];  // R0, R1 of each column
    static_assert(CB * PY / THREADS == 8, "eight elements per thread");
    constexpr int QS = (PY / 2 + 1 + 3) & ~3;
    constexpr int STEP = PY / 8;
    const int kx0 = blockIdx.x * CB;
    const int c = threadIdx.x / STEP, jt = threadIdx.x % STEP;
    const int kx = kx0 + c;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) fetch_spectra<T, PY, CB>(ssp, spec, kx0, qx, &bar);
    sg_dep_wait();  // the row pass's output (the kernel spectra are the plan's own)
    const C *cpair = reinterpret_cast<const C *>(phase), *rpair = cpair + 2 * qx;  // (e1, e2) per kx, per ky

    // the lower half of the column straight into registers (the upper half is zero)
    C v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int j = jt + m * STEP;
        v[m] = (m < 4 && j < ny && kx < qx) ? work_fwd[(int64_t)kx * ny + j] : cmake<C>((T)0, (T)0);
    }
    // the column's first and last rows (read after the transform's barriers)
    if (jt == 0) rows[c][0] = v[0];
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (jt + m * STEP == ny - 1) rows[c][1] = v[m];
    int par = 0;
    fft_regs<C, PY, CB, THREADS, col_central_nbuf<T, PY, CB>(), false>(v, bufs, par, tw);
    if (!spectra_ready(&bar, err, args.tries)) return;

    C accx[8], accy[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int ky = jt + q * STEP;
        accx[q] = accy[q] = cmake<C>((T)0, (T)0);
        if (kx >= qx) continue;
        const bool lower = ky <= PY / 2;
        const int kq = lower ? ky : PY - ky;
        const T sg = lower ? (T)1 : (T)-1;
        const T *sp = ssp + c * QS + kq;  // plane p at sp[p * CB * QS]
        const C S = v[q];
        // slope spectra
        C e1, e2, f1, f2;
        ld_pair<false>(cpair, kx, e1, e2);
        ld_pair<false>(rpair, ky, f1, f2);
        const T cs = (T)2 * e1.y, rs = (T)2 * f1.y;  // sin(2 pi k / P) / h, exactly
        C c0, c1;
        ld_pair<false>(edge, ky, c0, c1);
        // every operation explicitly rounded (see mul_rn): the result must not depend on the launch shape
        const C p2 = cmul_rn(e2, c1), p1 = cmul_rn(e1, c0);
        const C q2 = cmul_rn(f2, rows[c][1]), q1 = cmul_rn(f1, rows[c][0]);
        const C X = cmake<C>(add_rn(add_rn(-mul_rn(cs, S.y), p2.x), -p1.x), add_rn(add_rn(mul_rn(cs, S.x), p2.y), -p1.y));
        const C Y = cmake<C>(add_rn(add_rn(-mul_rn(rs, S.y), q2.x), -q1.x), add_rn(add_rn(mul_rn(rs, S.x), q2.y), -q1.y));
        const T a = sp[0 * CB * QS];
        const T b = sp[1 * CB * QS];
        const T cc = sg * sp[2 * CB * QS];
        const T d = sg * sp[3 * CB * QS];
        const T ee = sp[4 * CB * QS];
        const T ff = sg * sp[5 * CB * QS];
        accx[q] = cmake<C>(fma(cc, Y.x, fma(b, X.x, -mul_rn(a, S.y))), fma(cc, Y.y, fma(b, X.y, mul_rn(a, S.x))));
        accy[q] = cmake<C>(fma(ff, X.x, fma(ee, Y.x, -mul_rn(d, S.y))), fma(ff, X.y, fma(ee, Y.y, mul_rn(d, S.x))));
    }

    // inverse transforms: the products are already in the transform's input pattern
    if (col_central_nbuf<T, PY, CB>() == 1) __syncthreads();
    fft_regs<C, PY, CB, THREADS, col_central_nbuf<T, PY, CB>(), true>(accx, bufs, par, tw);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int j = jt + m * STEP;
        if (j < ny && kx < qx) work_inv[(int64_t)kx * ny + j] = accx[m];
    }
    if (col_central_nbuf<T, PY, CB>() == 1) __syncthreads();
    fft_regs<C, PY, CB, THREADS, col_central_nbuf<T, PY, CB>(), true>(accy, bufs, par, tw);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int j = jt + m * STEP;
        if (j < ny && kx < qx) work_inv[((int64_t)qx + kx) * ny + j] = accy[m];
    }
}

// ------------------------------------------------------------ launch shapes --

// Default shapes (measured): row sequences (two rows each) per CTA of the
// forward and inverse row passes, columns per CTA of the column passes.
__host__ __device__ constexpr int row_nb_default(int px) { return px >= 4096 ? 2 : (4096 / px < 2 ? 2 : 4096 / px); }
__host__ __device__ constexpr int row_nb_inv_default(int px) { return px >= 4096 ? 2 : (px == 2048 ? 4 : 4096 / px); }
__host__ __device__ constexpr int col_cb_default(int py) { return py >= 2048 ? 1 : 2048 / py; }
// Row-pass CTAs of 512 threads: a 1024² solve has only 256 row CTAs per pass,
// and 512 threads (instead of 256) double the warps per SM; measured 2-3 %
// faster per solve (potential, off-plane, central slopes), no spills.
constexpr int ROW_THREADS = 512;

// Candidate shapes: half, the default, and twice the default, where feasible
// (shared memory within 200 KB, 32..512 threads per CTA: 1024 would cap registers at 64).
__host__ __device__ constexpr int shape_candidate(int def, int k) { return k == 0 ? def / 2 : (k == 1 ? def : 2 * def); }
template <typename T>
__host__ __device__ constexpr bool row_feasible_t(int px, int nb)
{
    return nb >= 1 && nb <= 64 && (int64_t)spad_size<cplx_t<T>>(nb * px) * (int64_t)sizeof(cplx_t<T>) <= 200 * 1024;
}
template <typename T, int PY, int CB, int NPL>
__host__ __device__ constexpr bool col_feasible_t()
{
    return CB >= 1 && CB * PY / 8 >= 32 && CB * PY / 8 <= 512 && col_smem_bytes<T, PY, CB, NPL>() <= 200 * 1024;
}

// Dispatchers (explicitly instantiated for float and double in their units).
// A batch (one launch for `nmem` members of one padded length): `many` is a
// device array of the members' arguments and `maxny` their largest row count;
// the by-value arguments are then unused. nmem == 0: the one solve `one`.
struct batch_shape {
    int nmem;   // members (0: a single solve)
    int maxny;  // largest member row count
};
template <typename T>
sg_status rows_fwd(int px, int nb, const row_fwd_args<T> &one, int nf, const cplx_t<T> *tw, cudaStream_t st,
                   const row_fwd_args<T> *many = nullptr, batch_shape bs = {0, 0}, bool after_edge = false);
// The column and inverse-row passes are launched as dependent launches
// (sg_launch_dep) on the pass before them in the stream; dep = false launches a
// column pass normally (when its stream waits on an event just before it).
template <typename T>
sg_status rows_inv(int px, int nb, const row_inv_args<T> &one, int nout, const cplx_t<T> *tw, cudaStream_t st,
                   const row_inv_args<T> *many = nullptr, batch_shape bs = {0, 0});
template <typename T>
sg_status cols(int py, int cb, int nout, const col_args<T> &one, int qx, int nf, const cplx_t<T> *tw, int *err,
               cudaStream_t st, const col_args<T> *many = nullptr, batch_shape bs = {0, 0}, bool dep = true);
template <typename T>
sg_status cols_central(int py, int cb, const col_args<T> &one, int qx, const cplx_t<T> *tw, int *err, cudaStream_t st,
                       const col_args<T> *many = nullptr, batch_shape bs = {0, 0}, bool dep = true);
template <typename T>
sg_status edge_cols(int py, const edge_args<T> &one, const cplx_t<T> *tw, cudaStream_t st,
                    const edge_args<T> *many = nullptr, batch_shape bs = {0, 0});

// The arguments of every pass of one patch's solve (fftconv.cu), shared by the
// single solve and by batches (batch.cu). pot_spec != NULL: the potential (one
// output, three spectrum planes) with the forward scratch wf_pot, slopes formed
// in the row pass.
template <typename T>
struct uniform_passes {
    row_fwd_args<T> rf;
    edge_args<T> ed;
    col_args<T> col;
    row_inv_args<T> ri;
    int nf_rows;    // fields the row pass transforms
    int nf_cols;    // fields of the generic column pass
    int nout;       // outputs
    bool central;   // central slopes formed in the spectrum (edge columns, central column pass)
    int px, py, qx;
    const cplx_t<T> *twx, *twy;
    int shx[SG_TUNE_KNOBS], shy[SG_TUNE_KNOBS];  // launch shapes of the x and y lengths (tuning table)
};

template <typename T>
inline uniform_passes<T> uniform_setup(const sg_plan *plan, const sg_workspace *ws, int p, const void *sigma,
                                       const void *dx, const void *dy, void *fx, void *fy, void *fz,
                                       const T *pot_spec = nullptr, void *wf_pot = nullptr)
{
    using C = cplx_t<T>;
    uniform_passes<T> u;
    const sg_patch_plan &pp = plan->pp[p];
    const sg_patch_dev &d = pp.d;
    const int64_t off = d.cell_off;
    field_src<T> &src = u.rf.src;
    src.sigma = (const T *)sigma + off;
    src.dx = dx ? (const T *)dx + off : nullptr;
    src.dy = dy ? (const T *)dy + off : nullptr;
    src.nx = d.nx;
    src.ny = d.ny;
    src.inv2h = (T)(0.5 / d.h);
    src.mode = plan->geom.slope_mode;
    if (plan->composite) {
        // AMR or masks: the composite source fields (three planes, zero where no cell exists)
        const T *S = (const T *)ws->sfield;
        src.sigma = S + off;
        src.dx = S + plan->ncells + off;
        src.dy = S + 2 * plan->ncells + off;
        src.mode = SG_SLOPES_CALLER;
    }
    const int nf = src.mode == SG_SLOPES_NONE ? 1 : 3;
    u.px = d.px;
    u.py = d.py;
    u.qx = d.px / 2 + 1;
    C *wf = pot_spec ? (C *)wf_pot : (C *)ws->work_fwd;
    C *wi = (C *)ws->work_inv;
    const int64_t *twoff = sizeof(T) == 8 ? plan->tw64_off : plan->tw32_off;
    u.twx = (const C *)((const char *)plan->twiddles + twoff[sg_ilog2(d.px)]);
    u.twy = (const C *)((const char *)plan->twiddles + twoff[sg_ilog2(d.py)]);
    u.central = src.mode == SG_SLOPES_CENTRAL && pp.phase && !pot_spec;
    u.nf_rows = u.central ? 1 : nf;
    u.nf_cols = nf;
    u.nout = pot_spec ? 1 : (fz ? 3 : 2);
    u.rf.work = wf;
    // after sigma's row transforms (central slopes), at an even element: 16-byte pairs
    C *edge = wf + (((int64_t)u.qx * d.ny + 1) & ~(int64_t)1);
    u.ed = {src.sigma, d.nx, d.ny, edge};
    u.col = {wf, wi, pot_spec ? pot_spec : (const T *)pp.spectra, edge, (const T *)pp.phase, d.ny, plan->wait_tries};
    u.ri = {wi, (T *)fx + off, pot_spec ? nullptr : (T *)fy + off, fz ? (T *)fz + off : nullptr, d.nx, d.ny};
    sg_tune_shape(plan->prec, d.px, u.shx);
    sg_tune_shape(plan->prec, d.py, u.shy);
    return u;
}

#define SG_PAD_SWITCH(P, CALL)                 \
    switch (P) {                               \
    case 64: { constexpr int PP = 64; CALL; } break;     \
    case 128: { constexpr int PP = 128; CALL; } break;   \
    case 256: { constexpr int PP = 256; CALL; } break;   \
    case 512: { constexpr int PP = 512; CALL; } break;   \
    case 1024: { constexpr int PP = 1024; CALL; } break; \
    case 2048: { constexpr int PP = 2048; CALL; } break; \
    case 4096: { constexpr int PP = 4096; CALL; } break; \
    default: return SG_EINVAL;                 \
    }

}  // namespace sgk

