// Allocation-free direct force sum on a uniform grid (entry point
// sg_direct_force_static in sg.h).
//
// Some callers cannot let a library allocate device memory: an application
// that reserves the whole device budget up front and hands libraries only the
// buffers it owns, or a time-step loop that must not pay cudaMalloc's latency
// and implicit synchronisation on every call. This entry point serves them. It
// takes the caller's input and output buffers and keeps its only intermediate,
// the corner weights of the grid, in a fixed-size array compiled into the
// library (g_static_corners below), so it never allocates.
//
// What it computes is the plain direct sum of every cell pair of one uniform
// grid, in the corner form used by the cross-patch kernel: for each target
// cell centre t,
//   Fx(t) = G sum_c [ -A_c(t) g0(c - t) + X_c v g0y(c - t) - Y_c r(c - t) ]
//   Fy(t) = G sum_c [ -A_c(t) g0y(c - t) + Y_c u g0(c - t) - X_c r(c - t) ]
// over the (nx+1) x (ny+1) grid corners c, with A_c(t) = B_c - u X_c - v Y_c,
// B_c, X_c, Y_c the signed sums over the four cells around c of the cell's
// linear reconstruction at c and of its slopes, g0 = asinh(v/|u|),
// g0y = asinh(u/|v|). This equals the convolution that sg_force evaluates by
// FFT, to rounding. Positions are integers on the lattice of half cell widths
// (targets odd, corners even, so no corner ever sits on a target).
//
// The array is shared by every call in the process: each call overwrites the
// weights it uses before reading them, and calls whose work overlaps on one GPU
// (issued on different streams, or from different host threads, without
// ordering between them) race on it and give wrong results. Every GPU that
// loads the library holds the array until the process exits.
#include "common.cuh"

#include <mutex>

namespace {

// Maximum grid: 512 x 512 cells -> 513 x 513 corners, 16 bytes each (4.2 MB).
constexpr int kStaticMaxSide = 512;
constexpr int kStaticMaxCorners = (kStaticMaxSide + 1) * (kStaticMaxSide + 1);

static __device__ __align__(256) float4 g_static_corners[kStaticMaxCorners];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float4 *g_static_ptr[kMaxDevices] = {};

// Device address of the static array on the current device (set-up once per device).
sg_status static_corners(float4 **out)
{
    int dev = -1;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SG_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        SG_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_corners));
        g_static_ptr[dev] = (float4 *)p;
    }
    *out = g_static_ptr[dev];
    return SG_OK;
}

// One thread per corner: (B, lambda X, lambda Y, 0), lambda = h / 2.
__global__ void k_static_weights(int nx, int ny, float h, const float *__restrict__ sigma, const float *__restrict__ dx,
                                 const float *__restrict__ dy, float4 *__restrict__ w)
{
    const int ncx = nx + 1;
    const int total = ncx * (ny + 1);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int ci = e % ncx, cj = e / ncx;
        float B = 0.f, X = 0.f, Y = 0.f;
        for (int q = 0; q < 4; ++q) {
            const int i = ci - 1 + (q & 1), j = cj - 1 + (q >> 1);
            if (i < 0 || i >= nx || j < 0 || j >= ny) continue;
            const float s = (q == 0 || q == 3) ? 1.f : -1.f;
            const int o = j * nx + i;
            const float sx = dx ? dx[o] : 0.f, sy = dy ? dy[o] : 0.f;
            // the corner lies half a cell from the centre: +h/2 on the side of the cell it bounds
            const float ox = (q & 1) ? -0.5f * h : 0.5f * h;
            const float oy = (q >> 1) ? -0.5f * h : 0.5f * h;
            B += s * (sigma[o] + sx * ox + sy * oy);
            X += s * sx;
            Y += s * sy;
        }
        w[e] = make_float4(B, 0.5f * h * X, 0.5f * h * Y, 0.f);
    }
}

constexpr int kThreads = 256;
constexpr int kTile = 256;

// One thread per target cell; corners staged through shared memory in chunks.
__global__ void __launch_bounds__(kThreads) k_static_direct(int nx, int ny, double G, const float4 *__restrict__ w,
                                                            float *__restrict__ fx, float *__restrict__ fy)
{
    __shared__ float4 sw[kTile];
    __shared__ float2 sp[kTile];  // corner lattice positions (2 ci, 2 cj)
    const int ncx = nx + 1;
    const int ncorners = ncx * (ny + 1);
    const int t = blockIdx.x * kThreads + threadIdx.x;
    const bool active = t < nx * ny;
    const int ti = active ? t % nx : 0, tj = active ? t / nx : 0;
    const float tx = (float)(2 * ti + 1), ty = (float)(2 * tj + 1);
    double axl = 0.0, axr = 0.0, ayl = 0.0, ayr = 0.0;
    for (int c0 = 0; c0 < ncorners; c0 += kTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kTile; k += kThreads) {
            const int c = c0 + k;
            sw[k] = c < ncorners ? w[c] : make_float4(0.f, 0.f, 0.f, 0.f);
            sp[k] = make_float2((float)(2 * (c % ncx)), (float)(2 * (c / ncx)));
        }
        __syncthreads();
        float sxl = 0.f, sxr = 0.f, syl = 0.f, syr = 0.f;
        const int n = ncorners - c0 < kTile ? ncorners - c0 : kTile;
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
            const float4 wc = sw[k];
            const float2 pc = sp[k];
            const float u = pc.x - tx;
            const float v = pc.y - ty;
            const float au = fabsf(u), av = fabsf(v);
            const float rr = sqrtf(fmaf(u, u, v * v));
            const float g0 = copysignf(__log2f((av + rr) * __frcp_rn(au)), v);
            const float g0y = copysignf(__log2f((au + rr) * __frcp_rn(av)), u);
            const float A = wc.x - u * wc.y - v * wc.z;
            sxl = fmaf(-A, g0, sxl);
            sxl = fmaf(wc.y, v * g0y, sxl);
            sxr = fmaf(-wc.z, rr, sxr);
            syl = fmaf(-A, g0y, syl);
            syl = fmaf(wc.z, u * g0, syl);
            syr = fmaf(-wc.y, rr, syr);
        }
        axl += sxl;
        axr += sxr;
        ayl += syl;
        ayr += syr;
    }
    if (!active) return;
    const double ln2 = 0.69314718055994530942;
    fx[t] = (float)(G * (ln2 * axl + axr));
    fy[t] = (float)(G * (ln2 * ayl + ayr));
}

}  // namespace

extern "C" sg_status sg_direct_force_static(int nx, int ny, double h, double G, const float *sigma, const float *deltax,
                                            const float *deltay, float *fx, float *fy, void *stream)
{
    if (nx < 1 || ny < 1 || nx > kStaticMaxSide || ny > kStaticMaxSide) {
        sg_set_last_error_message("sg_direct_force_static: grid must be between 1x1 and 512x512 cells");
        return SG_EINVAL;
    }
    if (!(h > 0.0) || !sigma || !fx || !fy || (!deltax) != (!deltay)) {
        sg_set_last_error_message("sg_direct_force_static: invalid h or buffer pointer");
        return SG_EINVAL;
    }
    float4 *w = nullptr;
    SG_TRY(static_corners(&w));
    cudaStream_t st = (cudaStream_t)stream;
    const int ncorners = (nx + 1) * (ny + 1);
    k_static_weights<<<(ncorners + 255) / 256, 256, 0, st>>>(nx, ny, (float)h, sigma, deltax, deltay, w);
    SG_CUDA_TRY(cudaGetLastError());
    const int ncells = nx * ny;
    k_static_direct<<<(ncells + kThreads - 1) / kThreads, kThreads, 0, st>>>(nx, ny, G, w, fx, fy);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}
