// Cross-patch direct sum of an AMR hierarchy (Section 2, Eq. eqnXforce2 with
// the order-1 reconstruction of Eq. eqnGamma). The sources are the composite
// fields S_p of every patch (see amr.cu); each leaf target receives the sum
// over the cells of every patch other than its own, whose contribution comes
// from the FFT convolution of its own patch.
//
// Corner form. Every cell integral is a double difference over the cell's four
// corners, dd_i f = sum_c s_ic f(c - t) with s = +1 at the lower-left and
// upper-right corners and -1 at the other two. Writing the reconstruction of
// source i evaluated at the target, l_i(t) = sigma0_i + deltax_i (x_t - xc_i)
// + deltay_i (y_t - yc_i), the closed forms of Section 2 give
//   Fx(t) = G sum_c [ -A_c(t) g0(c - t) + X_c v g0y(c - t) - Y_c r(c - t) ]
//   Fy(t) = G sum_c [ -A_c(t) g0y(c - t) + Y_c u g0(c - t) - X_c r(c - t) ]
// with A_c(t) = sum_i s_ic l_i(t), X_c = sum_i s_ic deltax_i, Y_c = sum_i s_ic deltay_i,
//   g0(u, v) = asinh(v/|u|) = ln(v + r) - ln|u|,   g0y(u, v) = asinh(u/|v|),
// since the terms that depend on u alone (ln|u|) or v alone cancel in each
// cell's double difference. On u = 0 the coincident-line form of Section 2,
// sgn(v) ln|v|, is the same as g0 with ln|u| replaced by ln 2 (likewise for
// g0y on v = 0), which is what the kernel evaluates. A_c(t) is linear in the
// target position: A_c(t) = B_c + (x_t - x_T) X_c + (y_t - y_T) Y_c with B_c
// built relative to the tile origin (x_T, y_T) so that its terms stay local.
//
// All positions are integers on the lattice of half the finest cell width
// (lambda), so u and v are exact; X and Y are stored premultiplied by lambda.
// Pairs are summed in tiles of 16 x 16 corners staged in shared memory: FP32
// per tile, then added to FP64 accumulators across tiles (compensation of the
// long sum). FP64 plans run the same loop in FP64.
#include "common.cuh"

#include <math.h>

namespace {

// One thread per (tile, corner): signed sums of the (up to) four cells of the
// patch around the corner, from the composite source fields.
template <typename T>
__global__ void k_corner_weights(const sg_tile_desc *__restrict__ tiles, int ntiles, const sg_patch_dev *__restrict__ pd,
                                 const T *__restrict__ sigma, const T *__restrict__ dx, const T *__restrict__ dy,
                                 double lambda, T *__restrict__ wout)
{
    const int64_t total = (int64_t)ntiles * SG_TILE_N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e / SG_TILE_N), k = (int)(e % SG_TILE_N);
        const sg_tile_desc td = tiles[t];
        const sg_patch_dev p = pd[td.patch];
        const int ci = td.ci0 + k % SG_TILE_X, cj = td.cj0 + k / SG_TILE_X;
        double B = 0.0, X = 0.0, Y = 0.0;
        if (ci <= p.nx && cj <= p.ny) {
            // tile origin relative to cell centres, in lattice units
            for (int q = 0; q < 4; ++q) {
                const int i = ci - 1 + (q & 1), j = cj - 1 + (q >> 1);
                if (i < 0 || i >= p.nx || j < 0 || j >= p.ny) continue;
                const double s = (q == 0 || q == 3) ? 1.0 : -1.0;
                const int64_t o = p.cell_off + (int64_t)j * p.nx + i;
                const double s0 = (double)sigma[o];
                const double sx = dx ? (double)dx[o] : 0.0;
                const double sy = dy ? (double)dy[o] : 0.0;
                // cell centre (lattice) = patch origin + (2i + 1) step / 2
                const double cx = p.ox + (2 * i + 1) * (p.step / 2);
                const double cy = p.oy + (2 * j + 1) * (p.step / 2);
                B += s * (s0 + sx * (td.ox - cx) * lambda + sy * (td.oy - cy) * lambda);
                X += s * sx;
                Y += s * sy;
            }
        }
        wout[e * 4 + 0] = (T)B;
        wout[e * 4 + 1] = (T)(X * lambda);
        wout[e * 4 + 2] = (T)(Y * lambda);
        wout[e * 4 + 3] = (T)0;
    }
}

struct acc4 {
    double xl, xr, yl, yr;
};

// FP32 pair loop over one tile. g0 and g0y are evaluated as one base-2
// logarithm of an O(1) ratio, log2((|v| + r) / |u|) and log2((|u| + r) / |v|)
// (1/|u| and 1/|v| correctly rounded once per column and row; 1/2 on u = 0
// or v = 0, which gives the coincident-line form), instead of a difference of
// two logarithms of size ln(distance): the rounding of the result then scales
// with the ratio, not with the distance. ln 2 is applied at the end.
__device__ __forceinline__ void tile_pairs_f32(const float4 *__restrict__ w, float du0, float dv0, float st, float dxT,
                                               float dyT, acc4 &acc)
{
    float iu[SG_TILE_X];
#pragma unroll
    for (int c = 0; c < SG_TILE_X; ++c) {
        const float u = fmaf((float)c, st, du0);
        iu[c] = u == 0.0f ? 0.5f : __frcp_rn(fabsf(u));
    }
    float sxl = 0.f, sxr = 0.f, syl = 0.f, syr = 0.f;
#pragma unroll 1
    for (int r = 0; r < SG_TILE_Y; ++r) {
        const float v = fmaf((float)r, st, dv0);
        // + 1e-30 keeps q > 0 where a zero-weight padding corner sits on a target
        const float av = fabsf(v), v2 = fmaf(v, v, 1e-30f);
        const float iv = v == 0.0f ? 0.5f : __frcp_rn(av);
#pragma unroll
        for (int c = 0; c < SG_TILE_X; ++c) {
            const float4 wc = w[r * SG_TILE_X + c];
            const float u = fmaf((float)c, st, du0);
            const float q = fmaf(u, u, v2);
            const float rr = q * rsqrtf(q);
            const float g0 = copysignf(__log2f((av + rr) * iu[c]), v);
            const float g0y = copysignf(__log2f((fabsf(u) + rr) * iv), u);
            const float A = fmaf(dxT, wc.y, fmaf(dyT, wc.z, wc.x));
            sxl = fmaf(-A, g0, sxl);
            sxl = fmaf(wc.y, v * g0y, sxl);
            sxr = fmaf(-wc.z, rr, sxr);
            syl = fmaf(-A, g0y, syl);
            syl = fmaf(wc.z, u * g0, syl);
            syr = fmaf(-wc.y, rr, syr);
        }
    }
    acc.xl += sxl;
    acc.xr += sxr;
    acc.yl += syl;
    acc.yr += syr;
}

// FP64 pair loop over one tile (natural logarithms).
__device__ __forceinline__ void tile_pairs_f64(const sg_dvec4 *__restrict__ w, double du0, double dv0, double st,
                                               double dxT, double dyT, acc4 &acc)
{
    double Lu[SG_TILE_X];
#pragma unroll
    for (int c = 0; c < SG_TILE_X; ++c) {
        const double u = fma((double)c, st, du0);
        Lu[c] = u == 0.0 ? 0.69314718055994530942 : log(fabs(u));
    }
    double sxl = 0, sxr = 0, syl = 0, syr = 0;
#pragma unroll 1
    for (int r = 0; r < SG_TILE_Y; ++r) {
        const double v = fma((double)r, st, dv0);
        const double av = fabs(v), v2 = v * v;
        const double Lv = v == 0.0 ? 0.69314718055994530942 : log(av);
#pragma unroll 4
        for (int c = 0; c < SG_TILE_X; ++c) {
            const sg_dvec4 wc = w[r * SG_TILE_X + c];
            const double u = fma((double)c, st, du0);
            const double rr = sqrt(fma(u, u, v2));
            const double la = log(av + rr);
            const double lb = log(fabs(u) + rr);
            const double g0 = v == 0.0 ? 0.0 : copysign(la - Lu[c], v);
            const double g0y = u == 0.0 ? 0.0 : copysign(lb - Lv, u);
            const double A = fma(dxT, wc.y, fma(dyT, wc.z, wc.x));
            sxl = fma(-A, g0, sxl);
            sxl = fma(wc.y, v * g0y, sxl);
            sxr = fma(-wc.z, rr, sxr);
            syl = fma(-A, g0y, syl);
            syl = fma(wc.z, u * g0, syl);
            syr = fma(-wc.y, rr, syr);
        }
    }
    acc.xl += sxl;
    acc.xr += sxr;
    acc.yl += syl;
    acc.yr += syr;
}

template <typename T>
struct vec4_of;
template <>
struct vec4_of<float> { using type = float4; };
template <>
struct vec4_of<double> { using type = sg_dvec4; };

// grid (nblocks, nsplit); block SG_DIRECT_THREADS; one leaf target per thread.
template <typename T>
__global__ void __launch_bounds__(SG_DIRECT_THREADS) k_cross_direct(
    const sg_target_block *__restrict__ blocks, const int4 *__restrict__ targets, const sg_tile_desc *__restrict__ tiles,
    int ntiles, const T *__restrict__ wts, int nsplit, double G, T *__restrict__ fx, T *__restrict__ fy,
    double *__restrict__ partial, int ntargets)
{
    using V = typename vec4_of<T>::type;
    __shared__ V sw[SG_TILE_N];
    const sg_target_block blk = blocks[blockIdx.x];
    const int split = blockIdx.y;
    const int t0 = (int)((int64_t)ntiles * split / nsplit);
    const int t1 = (int)((int64_t)ntiles * (split + 1) / nsplit);
    const bool active = threadIdx.x < blk.count;
    int4 tg = make_int4(0, 0, -1, -1);
    if (active) tg = targets[blk.first + threadIdx.x];
    acc4 acc = {0.0, 0.0, 0.0, 0.0};
    const V *wv = reinterpret_cast<const V *>(wts);
    for (int t = t0; t < t1; ++t) {
        const sg_tile_desc td = tiles[t];
        if (td.patch == blk.patch) continue;  // same-patch pairs come from the FFT
        __syncthreads();
        for (int k = threadIdx.x; k < SG_TILE_N; k += SG_DIRECT_THREADS) sw[k] = wv[(int64_t)t * SG_TILE_N + k];
        __syncthreads();
        const T du0 = (T)(td.ox - tg.x), dv0 = (T)(td.oy - tg.y);
        const T dxT = (T)(tg.x - td.ox), dyT = (T)(tg.y - td.oy);
        if (sizeof(T) == 4)
            tile_pairs_f32(reinterpret_cast<const float4 *>(sw), (float)du0, (float)dv0, (float)td.step, (float)dxT,
                           (float)dyT, acc);
        else
            tile_pairs_f64(reinterpret_cast<const sg_dvec4 *>(sw), (double)du0, (double)dv0, (double)td.step,
                           (double)dxT, (double)dyT, acc);
    }
    if (!active) return;
    const double lnk = sizeof(T) == 4 ? 0.69314718055994530942 : 1.0;
    const double Fx = G * (lnk * acc.xl + acc.xr);
    const double Fy = G * (lnk * acc.yl + acc.yr);
    const int ti = blk.first + threadIdx.x;
    if (nsplit == 1) {
        fx[tg.z] = (T)((double)fx[tg.z] + Fx);
        fy[tg.z] = (T)((double)fy[tg.z] + Fy);
    } else {
        partial[((int64_t)split * ntargets + ti) * 2 + 0] = Fx;
        partial[((int64_t)split * ntargets + ti) * 2 + 1] = Fy;
    }
}

// Fixed-order sum of the per-split partials into the outputs.
template <typename T>
__global__ void k_cross_reduce(const int4 *__restrict__ targets, int ntargets, int nsplit,
                               const double *__restrict__ partial, T *__restrict__ fx, T *__restrict__ fy)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntargets; t += gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        for (int s = 0; s < nsplit; ++s) {
            sx += partial[((int64_t)s * ntargets + t) * 2 + 0];
            sy += partial[((int64_t)s * ntargets + t) * 2 + 1];
        }
        const int o = targets[t].z;
        fx[o] = (T)((double)fx[o] + sx);
        fy[o] = (T)((double)fy[o] + sy);
    }
}

template <typename T>
sg_status cross_solve_t(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                        void *fx, void *fy, cudaStream_t st)
{
    if (plan->ntiles == 0 || plan->ntargets == 0) return SG_OK;
    T *w = (T *)ws->tile_w;
    const int64_t nw = (int64_t)plan->ntiles * SG_TILE_N;
    int grid_w = (int)((nw + 255) / 256);
    if (grid_w > 65535) grid_w = 65535;
    sg_timing_begin(ws, SG_STAGE_WEIGHTS, st);
    k_corner_weights<T><<<grid_w, 256, 0, st>>>(plan->tiles, plan->ntiles, plan->patch_dev, (const T *)sigma,
                                                 (const T *)dx, (const T *)dy, plan->lattice_unit, w);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_WEIGHTS, st);
    sg_timing_begin(ws, SG_STAGE_DIRECT, st);
    dim3 grid(plan->nblocks, plan->nsplit);
    k_cross_direct<T><<<grid, SG_DIRECT_THREADS, 0, st>>>(plan->blocks, plan->targets, plan->tiles, plan->ntiles, w,
                                                          plan->nsplit, plan->geom.G, (T *)fx, (T *)fy,
                                                          ws->partial, plan->ntargets);
    SG_CUDA_TRY(cudaGetLastError());
    if (plan->nsplit > 1) {
        k_cross_reduce<T><<<(plan->ntargets + 255) / 256, 256, 0, st>>>(plan->targets, plan->ntargets, plan->nsplit,
                                                                         ws->partial, (T *)fx, (T *)fy);
        SG_CUDA_TRY(cudaGetLastError());
    }
    sg_timing_end(ws, SG_STAGE_DIRECT, st);
    return SG_OK;
}

}  // namespace

sg_status sg_cross_solve(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                         void *fx, void *fy, cudaStream_t st)
{
    if (plan->prec == SG_FP64) return cross_solve_t<double>(plan, ws, sigma, dx, dy, fx, fy, st);
    return cross_solve_t<float>(plan, ws, sigma, dx, dy, fx, fy, st);
}
