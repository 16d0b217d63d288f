// Cross-patch direct sum of an AMR hierarchy (Section 2, Eq. eqnXforce2 with
// the order-1 reconstruction of Eq. eqnGamma). The sources are the composite
// fields S_p of every patch (see amr.cu); each leaf target receives the sum
// over the cells of every patch other than its own, whose contribution comes
// from the FFT convolution of its own patch.
//
// Two evaluations of the same sum.
//
// FP64 plans: corner form. Every cell integral is a double difference over the
// cell's four corners, dd_i f = sum_c s_ic f(c - t) with s = +1 at the
// lower-left and upper-right corners and -1 at the other two. Writing the
// reconstruction of source i evaluated at the target, l_i(t) = sigma0_i +
// deltax_i (x_t - xc_i) + deltay_i (y_t - yc_i), the closed forms of Section 2 give
//   Fx(t) = G sum_c [ -A_c(t) g0(c - t) + X_c v g0y(c - t) - Y_c r(c - t) ]
//   Fy(t) = G sum_c [ -A_c(t) g0y(c - t) + Y_c u g0(c - t) - X_c r(c - t) ]
// with A_c(t) = sum_i s_ic l_i(t), X_c = sum_i s_ic deltax_i, Y_c = sum_i s_ic deltay_i,
//   g0(u, v) = asinh(v/|u|) = ln(v + r) - ln|u|,   g0y(u, v) = asinh(u/|v|),
// since the terms that depend on u alone (ln|u|) or v alone cancel in each
// cell's double difference. On u = 0 the coincident-line form of Section 2,
// sgn(v) ln|v|, is the same as g0 with ln|u| replaced by ln 2 (likewise for
// g0y on v = 0). A_c(t) = B_c + (x_t - x_T) X_c + (y_t - y_T) Y_c with B_c
// built relative to the tile origin (x_T, y_T). Pairs are summed in tiles of
// 16 x 16 corners staged in shared memory, per tile and across tiles in FP64.
//
// FP32 plans: near field in FP64, far field by the expansion of each cell's
// integrals about its centre. The corner form is unsuited to FP32: a corner's
// term is O(sigma) times an O(1) logarithm while a distant cell's integral is
// O(sigma H^2 / rho^2), so rounding of every corner term, not the integrals,
// sets the error (it grows like the square root of the number of corners).
//  * Far cells (centre at least SG_NEAR_R cell widths from the target along
//    some axis). With a, b = (centre - target) / H, rho^2 = a^2 + b^2, and the
//    complex derivatives d = (d_a - i d_b) / 2, d~ = (d_a + i d_b) / 2, the
//    integral of sigma0 + deltax xi + deltay eta times (1/rho) over the cell is
//    an operator series in d, d~ applied to 1/rho (the moments of the square),
//    and d^k d~^l (1/rho) = (-1)^(k+l) C_k C_l rho^-1 w^k conj(w)^l with
//    w = 1/(a + i b), C_k = (2k - 1)!! / 2^k. The force is minus the gradient,
//    Fx - i Fy = -2 d(...), which gives, per unit G, with s = 1/rho^2,
//    m = sigma0, D = (deltax + i deltay) H:
//      Q = rho^-1 { m [w (1 + s/8 + 7 s^2/256) - 21 w^5/512 - 7 s conj(w)^3/1536]
//                 - D w^2/8 - conj(D) s/24
//                 + 7 conj(D) w^4/384 + D s (conj(w)^2 - 7 w^2)/384 - 7 conj(D) s^2/640 }
//    (terms through H^6; through H^4: m w (1 + s/8) - D w^2/8 - conj(D) s/24).
//    Relative to 1/rho^2, per unit sigma0 or unit slope times H, the
//    truncation is at most 1.3e-7 (sigma0) and 1.02e-6 (slopes) from 6 cell
//    widths on (through H^6), 3e-8 and 7.6e-7 from 32 on (through H^4), all
//    far under the 1e-5 the FP32 path is held to;
//    every term is a small positive-scale product, so FP32 rounding stays
//    relative to the cell's own contribution.
//  * Near cells (both |a|, |b| < SG_NEAR_R): the closed forms in FP64, as the
//    corner form over the corners of the box of near cells with weights from
//    the box's cells only.
// The far field is one persistent launch: each CTA takes (target block,
// source-tile range) items from a counter, streams the tiles' cell
// coefficients into a ring of shared-memory buffers by 1-D bulk copies (TMA)
// completed on mbarriers, and sums per tile in FP32, across tiles in FP64. The
// near field is one warp per target: lanes take the corners of the box, the
// warp reduces with shuffles. A last launch adds the far partials, the near
// field and the patch's own FFT result in a fixed order.
//
// The mid-plane potential (sg_potential on hierarchies of this path) is the
// same sum with the kernel 1/r: its corner form, far-field moments and
// kernels follow the force's (see the potential section below).
#include "common.cuh"
#include "tma.cuh"

#include <math.h>

namespace {

// ================================================================= FP64 ====

// One thread per (tile, corner): signed sums of the (up to) four cells of the
// patch around the corner, from the composite source fields.
template <typename T>
__global__ void k_corner_weights(const sg_tile_desc *__restrict__ tiles, int ntiles, const sg_patch_dev *__restrict__ pd,
                                 const T *__restrict__ sigma, const T *__restrict__ dx,
                                 const T *__restrict__ dy, double lambda, double *__restrict__ wout)
{
    const int64_t total = (int64_t)ntiles * SG_TILE_N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e / SG_TILE_N), k = (int)(e % SG_TILE_N);
        const sg_tile_desc td = tiles[t];
        const sg_patch_dev p = pd[td.patch];
        const int ci = td.ci0 + k % SG_TILE_X, cj = td.cj0 + k / SG_TILE_X;
        double B = 0.0, X = 0.0, Y = 0.0;
        if (ci <= p.nx && cj <= p.ny) {
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
        wout[e * 4 + 0] = B;
        wout[e * 4 + 1] = X * lambda;
        wout[e * 4 + 2] = Y * lambda;
        wout[e * 4 + 3] = 0.0;
    }
}

struct acc4 {
    double xl, xr, yl, yr;
};

// FP64 pair loop over one corner tile (natural logarithms).
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

// grid (nblocks, nsplit); block SG_DIRECT_THREADS; one leaf target per thread.
__global__ void __launch_bounds__(SG_DIRECT_THREADS) k_cross_direct(
    const sg_target_block *__restrict__ blocks, const int4 *__restrict__ targets, const sg_tile_desc *__restrict__ tiles,
    int ntiles, const double *__restrict__ wts, int nsplit, double G, double *__restrict__ fx, double *__restrict__ fy,
    double *__restrict__ partial, int ntargets)
{
    __shared__ sg_dvec4 sw[SG_TILE_N];
    const sg_target_block blk = blocks[blockIdx.x];
    const int split = blockIdx.y;
    const int t0 = (int)((int64_t)ntiles * split / nsplit);
    const int t1 = (int)((int64_t)ntiles * (split + 1) / nsplit);
    const bool active = threadIdx.x < blk.count;
    int4 tg = make_int4(0, 0, -1, -1);
    if (active) tg = targets[blk.first + threadIdx.x];
    acc4 acc = {0.0, 0.0, 0.0, 0.0};
    const sg_dvec4 *wv = reinterpret_cast<const sg_dvec4 *>(wts);
    for (int t = t0; t < t1; ++t) {
        const sg_tile_desc td = tiles[t];
        if (td.patch == blk.patch) continue;  // same-patch pairs come from the FFT
        __syncthreads();
        for (int k = threadIdx.x; k < SG_TILE_N; k += SG_DIRECT_THREADS) sw[k] = wv[(int64_t)t * SG_TILE_N + k];
        __syncthreads();
        tile_pairs_f64(sw, (double)(td.ox - tg.x), (double)(td.oy - tg.y), (double)td.step, (double)(tg.x - td.ox),
                       (double)(tg.y - td.oy), acc);
    }
    if (!active) return;
    const double Fx = G * (acc.xl + acc.xr);
    const double Fy = G * (acc.yl + acc.yr);
    const int ti = blk.first + threadIdx.x;
    if (nsplit == 1) {
        fx[tg.z] += Fx;
        fy[tg.z] += Fy;
    } else {
        partial[((int64_t)split * ntargets + ti) * 2 + 0] = Fx;
        partial[((int64_t)split * ntargets + ti) * 2 + 1] = Fy;
    }
}

// Fixed-order sum of the per-split partials into the outputs.
__global__ void k_cross_reduce(const int4 *__restrict__ targets, int ntargets, int nsplit,
                               const double *__restrict__ partial, double *__restrict__ fx, double *__restrict__ fy)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntargets; t += gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        for (int s = 0; s < nsplit; ++s) {
            sx += partial[((int64_t)s * ntargets + t) * 2 + 0];
            sy += partial[((int64_t)s * ntargets + t) * 2 + 1];
        }
        const int o = targets[t].z;
        fx[o] += sx;
        fy[o] += sy;
    }
}

sg_status cross_solve_f64(sg_plan *plan, const sg_workspace *ws, const double *sigma, const double *dx,
                          const double *dy, double *fx, double *fy, cudaStream_t st)
{
    double *w = (double *)ws->tile_w;
    const int64_t nw = (int64_t)plan->ntiles * SG_TILE_N;
    int grid_w = (int)((nw + 255) / 256);
    if (grid_w > 65535) grid_w = 65535;
    sg_timing_begin(ws, SG_STAGE_WEIGHTS, st);
    k_corner_weights<double><<<grid_w, 256, 0, st>>>(plan->tiles, plan->ntiles, plan->patch_dev, sigma, dx, dy,
                                             plan->lattice_unit, w);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_WEIGHTS, st);
    sg_timing_begin(ws, SG_STAGE_DIRECT, st);
    dim3 grid(plan->nblocks, plan->nsplit);
    k_cross_direct<<<grid, SG_DIRECT_THREADS, 0, st>>>(plan->blocks, plan->targets, plan->tiles, plan->ntiles, w,
                                                       plan->nsplit, plan->geom.G, fx, fy, ws->partial,
                                                       plan->ntargets);
    SG_CUDA_TRY(cudaGetLastError());
    if (plan->nsplit > 1) {
        k_cross_reduce<<<(plan->ntargets + 255) / 256, 256, 0, st>>>(plan->targets, plan->ntargets, plan->nsplit,
                                                                      ws->partial, fx, fy);
        SG_CUDA_TRY(cudaGetLastError());
    }
    sg_timing_end(ws, SG_STAGE_DIRECT, st);
    return SG_OK;
}

// ================================================================= FP32 ====

constexpr int FAR_STAGES = 4;
constexpr uint32_t TILE_BYTES = SG_TILE_N * sizeof(float4);

// Cell coefficients of every tile, (sigma0, deltax H / 8, deltay H / 8, 0) of
// the composite source (zero outside the patch); also resets the far-field
// launch's work counter.
__global__ void k_cell_coefs(const sg_tile_desc *__restrict__ tiles, int ntiles, const sg_patch_dev *__restrict__ pd,
                             const float *__restrict__ sigma, const float *__restrict__ dx,
                             const float *__restrict__ dy, double lambda, float4 *__restrict__ wout,
                             int *__restrict__ counter)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
    const int64_t total = (int64_t)ntiles * SG_TILE_N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e / SG_TILE_N), k = (int)(e % SG_TILE_N);
        const sg_tile_desc td = tiles[t];
        const sg_patch_dev &p = pd[td.patch];
        const int nx = p.nx, ny = p.ny;
        const int i = td.ci0 + k % SG_TILE_X, j = td.cj0 + k / SG_TILE_X;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < nx && j < ny) {
            const int64_t o = p.cell_off + (int64_t)j * nx + i;
            const double h8 = p.step * lambda * 0.125;
            c.x = sigma[o];
            c.y = (float)((double)dx[o] * h8);
            c.z = (float)((double)dy[o] * h8);
        }
        wout[e] = c;
    }
}

// Contribution Q = (Fx - i Fy) / G of one cell (see the file comment),
// accumulated into (qr, qi). (a, b): centre minus target in cell widths, b2 =
// b^2, tb = 2 b; c = (m, d_x, d_y) with d = D / 8. Through H^4, in real form
// with s = 1/rho^2, ir3 = rho^-3, ir5 = rho^-5, c2 = a^2 - b^2, ab2 = 2 a b:
//   Re Q = m (1 + s/8) ir3 a - d_x (ir5 c2 + ir3/3) - d_y ir5 ab2
//   Im Q = -m (1 + s/8) ir3 b + d_y (ir3/3 - ir5 c2) + d_x ir5 ab2
// (m w (1 + s/8) - d w^2 - conj(d) s / 3, times 1/rho); the H^6 terms are added
// in complex form.
template <int ORDER>
__device__ __forceinline__ void cell_far(float a, float b, float b2, float tb, const float4 c, float &qr, float &qi)
{
    const float r2 = fmaf(a, a, b2);
    const float c2 = fmaf(a, a, -b2);
    const float ab2 = a * tb;
    const float ir = rsqrtf(r2);
    const float s = ir * ir;
    const float ir3 = ir * s, ir5 = ir3 * s;
    const float poly = ORDER >= 6 ? fmaf(s, fmaf(s, 7.f / 256.f, 0.125f), 1.f) : fmaf(s, 0.125f, 1.f);
    const float g = c.x * poly * ir3;
    const float u3 = ir3 * (1.f / 3.f);
    const float e1 = fmaf(ir5, c2, u3), e2 = fmaf(-ir5, c2, u3), f = ir5 * ab2;
    qr = fmaf(g, a, qr);
    qr = fmaf(-c.y, e1, qr);
    qr = fmaf(-c.z, f, qr);
    qi = fmaf(-g, b, qi);
    qi = fmaf(c.z, e2, qi);
    qi = fmaf(c.y, f, qi);
    if (ORDER >= 6) {
        // w = (a - i b) s, w^2 = (c2 - i ab2) s^2
        const float wr = a * s, wi = -b * s;
        const float ss = s * s;
        const float w2r = c2 * ss, w2i = -ab2 * ss;
        const float w3r = fmaf(w2r, wr, -w2i * wi), w3i = fmaf(w2r, wi, w2i * wr);
        const float w4r = fmaf(w2r, w2r, -w2i * w2i), w4i = 2.f * w2r * w2i;
        const float w5r = fmaf(w4r, wr, -w4i * wi), w5i = fmaf(w4r, wi, w4i * wr);
        // - m (21/512) w^5 - m s (7/1536) conj(w^3)
        const float m1 = c.x * (21.f / 512.f), m2 = c.x * s * (7.f / 1536.f);
        float pr = -m1 * w5r, pi = -m1 * w5i;
        pr = fmaf(-m2, w3r, pr);
        pi = fmaf(m2, w3i, pi);
        // + 7 conj(D) w^4 / 384 = (7/48) conj(d) w^4
        const float e7 = 7.f / 48.f;
        pr = fmaf(e7, fmaf(c.y, w4r, c.z * w4i), pr);
        pi = fmaf(e7, fmaf(c.y, w4i, -c.z * w4r), pi);
        // + D s (conj(w^2) - 7 w^2) / 384 = (s/48) d (-6 w2r - 8 i w2i)
        const float ur = s * (-6.f / 48.f) * w2r, ui = s * (-8.f / 48.f) * w2i;
        pr = fmaf(c.y, ur, pr);
        pr = fmaf(-c.z, ui, pr);
        pi = fmaf(c.y, ui, pi);
        pi = fmaf(c.z, ur, pi);
        // - 7 conj(D) s^2 / 640 = -(7/80) conj(d) s^2
        const float s2 = ss * (7.f / 80.f);
        pr = fmaf(-c.y, s2, pr);
        pi = fmaf(c.z, s2, pi);
        qr = fmaf(ir, pr, qr);
        qi = fmaf(ir, pi, qi);
    }
}

// All cells of one staged tile against one target: (a0, b0) = offsets of cell
// (0, 0) in cell widths; MASK drops near cells (summed by the FP64 near field).
template <int ORDER, bool MASK>
__device__ __forceinline__ void tile_far(const float4 *__restrict__ w, float a0, float b0, double &ar, double &ai)
{
    float qr = 0.f, qi = 0.f;
#pragma unroll 1
    for (int r = 0; r < SG_TILE_Y; ++r) {
        const float b = b0 + (float)r;
        const float b2 = b * b, tb = 2.f * b;
        const bool bnear = fabsf(b) < (float)SG_NEAR_R;
#pragma unroll
        for (int c = 0; c < SG_TILE_X; ++c) {
            const float a = a0 + (float)c;
            if (MASK) {
                float pr = qr, pi = qi;
                cell_far<ORDER>(a, b, b2, tb, w[r * SG_TILE_X + c], pr, pi);
                const bool nearc = bnear && fabsf(a) < (float)SG_NEAR_R;
                qr = nearc ? qr : pr;
                qi = nearc ? qi : pi;
            } else {
                cell_far<ORDER>(a, b, b2, tb, w[r * SG_TILE_X + c], qr, qi);
            }
        }
    }
    ar += qr;
    ai += qi;
}

// Persistent far-field sum. Work item = (target block, split of the tile list);
// CTAs take items from words[1] (reset by k_cell_coefs). Thread 0 streams the
// item's tiles (the split minus the block's own patch) into FAR_STAGES shared
// buffers by bulk copies; every thread (one target each) waits on the buffer's
// mbarrier, sums the tile, and after a block barrier thread 0 refills the
// buffer with the tile FAR_STAGES ahead. Each tile is summed through H^4 when
// every one of its cell centres is at least SG_FAR_R4 cell widths from the
// block's targets along some axis, else through H^6, with the near cells
// dropped when some centre is within SG_NEAR_R (exact integer tests on the
// lattice). Waits are bounded: if one runs out, the CTA records words[0] = 1,
// waits (bounded) for its copies in flight and returns.
__global__ void __launch_bounds__(SG_DIRECT_THREADS) k_cross_far(
    const sg_target_block *__restrict__ blocks, int nblocks, const int4 *__restrict__ targets,
    const sg_tile_desc *__restrict__ tiles, const sg_patch_dev *__restrict__ pd, int ntiles,
    const float4 *__restrict__ coefs, int nsplit, double G, double *__restrict__ partial, int ntargets,
    int *__restrict__ words, int tries)
{
    __shared__ __align__(128) float4 buf[FAR_STAGES][SG_TILE_N];
    __shared__ uint64_t full[FAR_STAGES];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    if (tid == 0)
        for (int s = 0; s < FAR_STAGES; ++s) mbar_init(&full[s], 1);
    __syncthreads();
    uint32_t used = 0;    // tiles consumed by this CTA (the same in every thread)
    uint32_t issued = 0;  // tiles whose copy thread 0 has issued
    const int nitems = nblocks * nsplit;
    bool failed = false;
    while (!failed) {
        if (tid == 0) s_item = atomicAdd(&words[1], 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        const int bi = item / nsplit, split = item - bi * nsplit;
        const sg_target_block blk = blocks[bi];
        const int t0 = (int)((int64_t)ntiles * split / nsplit), t1 = (int)((int64_t)ntiles * (split + 1) / nsplit);
        const int own0 = pd[blk.patch].tile_first, own1 = own0 + pd[blk.patch].tile_count;
        const int n1 = max(0, min(t1, own0) - t0), s2 = max(t0, own1);
        const int n = n1 + max(0, t1 - s2);
        const bool active = tid < blk.count;
        const int4 tg = targets[blk.first + (active ? tid : 0)];
        if (tid == 0) {
            for (int k = 0; k < n && k < FAR_STAGES; ++k, ++issued) {
                const int stg = issued % FAR_STAGES;
                const int t = k < n1 ? t0 + k : s2 + (k - n1);
                mbar_arrive_expect_tx(&full[stg], TILE_BYTES);
                bulk_copy_g2s(buf[stg], coefs + (int64_t)t * SG_TILE_N, TILE_BYTES, &full[stg]);
            }
        }
        double ar = 0.0, ai = 0.0;
        for (int k = 0; k < n; ++k, ++used) {
            const int stg = used % FAR_STAGES;
            const int t = k < n1 ? t0 + k : s2 + (k - n1);
            const bool ok = mbar_wait_bounded(&full[stg], (used / FAR_STAGES) & 1, tries);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            const sg_tile_desc td = tiles[t];
            // Chebyshev gap between the block's targets and the tile's cell centres (lattice units)
            const int cx0 = td.ox + td.step / 2, cx1 = cx0 + (SG_TILE_X - 1) * td.step;
            const int cy0 = td.oy + td.step / 2, cy1 = cy0 + (SG_TILE_Y - 1) * td.step;
            const int gx = max(0, max(cx0 - blk.tx1, blk.tx0 - cx1));
            const int gy = max(0, max(cy0 - blk.ty1, blk.ty0 - cy1));
            const int gap = max(gx, gy);
            const float inv = 1.0f / (float)td.step;  // a power of two: exact
            const float a0 = (float)(td.ox - tg.x) * inv + 0.5f, b0 = (float)(td.oy - tg.y) * inv + 0.5f;
            if (gap >= SG_FAR_R4 * td.step)
                tile_far<4, false>(buf[stg], a0, b0, ar, ai);
            else if (gap >= SG_NEAR_R * td.step)
                tile_far<6, false>(buf[stg], a0, b0, ar, ai);
            else
                tile_far<6, true>(buf[stg], a0, b0, ar, ai);
            __syncthreads();  // every thread is done with buf[stg]
            if (tid == 0 && k + FAR_STAGES < n) {
                const int kk = k + FAR_STAGES;
                const int tn = kk < n1 ? t0 + kk : s2 + (kk - n1);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect_tx(&full[stg], TILE_BYTES);
                bulk_copy_g2s(buf[stg], coefs + (int64_t)tn * SG_TILE_N, TILE_BYTES, &full[stg]);
                ++issued;
            }
        }
        if (failed) break;
        if (active) {
            const int64_t o = ((int64_t)split * ntargets + blk.first + tid) * 2;
            partial[o + 0] = G * ar;
            partial[o + 1] = -G * ai;
        }
    }
    if (failed && tid == 0) {
        atomicExch(&words[0], 1);
        for (uint32_t g = used; g < issued; ++g) mbar_wait_bounded(&full[g % FAR_STAGES], (g / FAR_STAGES) & 1, SG_MBAR_MAX_TRIES);
    }
}

__device__ __forceinline__ int floor_div(int64_t a, int64_t b)
{
    return (int)(a >= 0 ? a / b : -((-a + b - 1) / b));
}

// Near field in FP64: one warp per target; for every other patch, the box of
// cells whose centres lie within SG_NEAR_R cell widths of the target along
// both axes (the cells k_cross_far drops, at most 2 SG_NEAR_R per axis),
// summed in the corner form over the box's corners with weights from the
// box's cells only. The warp first stores the box's cell values l_i(t),
// deltax_i, deltay_i in shared memory with a zero border and the logarithms of
// |u| and |v| of the corner columns and rows in lanes; then lanes take
// corners (two logarithms each) and the warp reduces with shuffles.
constexpr int NEAR_WARPS = 8;
constexpr int NEAR_SLOTS = (2 * SG_NEAR_R + 2) * (2 * SG_NEAR_R + 2);

__global__ void __launch_bounds__(NEAR_WARPS * 32) k_cross_near(const int4 *__restrict__ targets, int ntargets,
                                                               const sg_patch_dev *__restrict__ pd, int npatches,
                                                               const float *__restrict__ sigma,
                                                               const float *__restrict__ dx,
                                                               const float *__restrict__ dy, double lambda, double G,
                                                               double *__restrict__ near_out)
{
    __shared__ double cellv[NEAR_WARPS][3][NEAR_SLOTS];
    const int lane = threadIdx.x & 31;
    double *cl = cellv[threadIdx.x >> 5][0], *cx = cellv[threadIdx.x >> 5][1], *cy = cellv[threadIdx.x >> 5][2];
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    const double LN2 = 0.69314718055994530942;
    for (int t = warp; t < ntargets; t += nwarps) {
        const int4 tg = targets[t];
        double fx = 0.0, fy = 0.0;
        for (int q = 0; q < npatches; ++q) {
            if (q == tg.w) continue;
            const sg_patch_dev &p = pd[q];
            const int64_t L = p.step, RL = (int64_t)SG_NEAR_R * L;
            // cells i with |ox + i L + L/2 - x_t| < R L, j likewise
            const int64_t ex = (int64_t)tg.x - p.ox - L / 2, ey = (int64_t)tg.y - p.oy - L / 2;
            const int i0 = max(0, floor_div(ex - RL, L) + 1), j0 = max(0, floor_div(ey - RL, L) + 1);
            const int i1 = min(p.nx - 1, -floor_div(-(ex + RL), L) - 1);
            const int j1 = min(p.ny - 1, -floor_div(-(ey + RL), L) - 1);
            if (i0 > i1 || j0 > j1) continue;
            const int nbx = i1 - i0 + 1, nby = j1 - j0 + 1, W = nbx + 2;
            __syncwarp();  // the previous box's values have been read
            for (int k = lane; k < W * (nby + 2); k += 32) {
                const int bi = k % W - 1, bj = k / W - 1;
                double l = 0.0, X = 0.0, Y = 0.0;
                if (bi >= 0 && bi < nbx && bj >= 0 && bj < nby) {
                    const int i = i0 + bi, j = j0 + bj;
                    const int64_t o = p.cell_off + (int64_t)j * p.nx + i;
                    X = dx[o];
                    Y = dy[o];
                    // target minus cell centre, physical units
                    const double ux = ((double)tg.x - ((double)p.ox + (i + 0.5) * (double)L)) * lambda;
                    const double uy = ((double)tg.y - ((double)p.oy + (j + 0.5) * (double)L)) * lambda;
                    l = fma(X, ux, fma(Y, uy, (double)sigma[o]));
                }
                cl[k] = l;
                cx[k] = X;
                cy[k] = Y;
            }
            // corner column ci (lane ci <= nbx) and row cj: u, v relative to the target
            const double uc = ((double)p.ox + (double)(i0 + lane) * L - tg.x) * lambda;
            const double vc = ((double)p.oy + (double)(j0 + lane) * L - tg.y) * lambda;
            const double lnu = lane <= nbx ? (uc == 0.0 ? LN2 : log(fabs(uc))) : 0.0;
            const double lnv = lane <= nby ? (vc == 0.0 ? LN2 : log(fabs(vc))) : 0.0;
            __syncwarp();
            const int nci = nbx + 1, ncorner = nci * (nby + 1);
            for (int base = 0; base < ncorner; base += 32) {
                const int k = base + lane;
                const bool valid = k < ncorner;
                const int kk = valid ? k : 0;
                const int ci = kk % nci, cj = kk / nci;
                const double Lu = __shfl_sync(0xffffffffu, lnu, ci);
                const double Lv = __shfl_sync(0xffffffffu, lnv, cj);
                if (!valid) continue;
                // cells around corner (ci, cj) of the box: lower-left and upper-right count +1
                const int s00 = cj * W + ci, s10 = s00 + 1, s01 = s00 + W, s11 = s01 + 1;
                const double A = (cl[s00] - cl[s10]) - (cl[s01] - cl[s11]);
                const double X = (cx[s00] - cx[s10]) - (cx[s01] - cx[s11]);
                const double Y = (cy[s00] - cy[s10]) - (cy[s01] - cy[s11]);
                const double u = ((double)p.ox + (double)(i0 + ci) * L - tg.x) * lambda;
                const double v = ((double)p.oy + (double)(j0 + cj) * L - tg.y) * lambda;
                const double au = fabs(u), av = fabs(v);
                const double r = sqrt(fma(u, u, v * v));
                // sgn(v) (ln(|v| + r) - ln|u|), ln|u| -> ln 2 on u = 0 (the coincident-line form
                // sgn(v) ln|v|, which may be negative: the sign multiplies, it is not copied)
                const double t0 = log(av + r) - Lu;
                const double t1 = log(au + r) - Lv;
                const double g0 = v == 0.0 ? 0.0 : (v > 0.0 ? t0 : -t0);
                const double g0y = u == 0.0 ? 0.0 : (u > 0.0 ? t1 : -t1);
                fx += fma(X * v, g0y, fma(-A, g0, -Y * r));
                fy += fma(Y * u, g0, fma(-A, g0y, -X * r));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, off);
            fy += __shfl_xor_sync(0xffffffffu, fy, off);
        }
        if (lane == 0) {
            near_out[(int64_t)t * 2 + 0] = G * fx;
            near_out[(int64_t)t * 2 + 1] = G * fy;
        }
    }
}

// Fixed-order sum: the patch's own FFT result, the far partials of every split,
// then the near field.
__global__ void k_cross_combine(const int4 *__restrict__ targets, int ntargets, int nsplit,
                                const double *__restrict__ partial, float *__restrict__ fx, float *__restrict__ fy)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntargets; t += gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        for (int s = 0; s <= nsplit; ++s) {
            sx += partial[((int64_t)s * ntargets + t) * 2 + 0];
            sy += partial[((int64_t)s * ntargets + t) * 2 + 1];
        }
        const int o = targets[t].z;
        fx[o] = (float)((double)fx[o] + sx);
        fy[o] = (float)((double)fy[o] + sy);
    }
}

sg_status cross_solve_f32(sg_plan *plan, const sg_workspace *ws, const float *sigma, const float *dx,
                          const float *dy, float *fx, float *fy, cudaStream_t st)
{
    float4 *w = (float4 *)ws->tile_w;
    const int64_t nw = (int64_t)plan->ntiles * SG_TILE_N;
    int grid_w = (int)((nw + 255) / 256);
    if (grid_w > 65535) grid_w = 65535;
    sg_timing_begin(ws, SG_STAGE_WEIGHTS, st);
    k_cell_coefs<<<grid_w, 256, 0, st>>>(plan->tiles, plan->ntiles, plan->patch_dev, sigma, dx, dy,
                                         plan->lattice_unit, w, ws->err + 1);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_WEIGHTS, st);
    sg_timing_begin(ws, SG_STAGE_DIRECT, st);
    k_cross_far<<<plan->far_grid, SG_DIRECT_THREADS, 0, st>>>(plan->blocks, plan->nblocks, plan->targets, plan->tiles,
                                                              plan->patch_dev, plan->ntiles, w, plan->nsplit,
                                                              plan->geom.G, ws->partial, plan->ntargets, ws->err,
                                                              plan->wait_tries);
    SG_CUDA_TRY(cudaGetLastError());
    double *near = ws->partial + (int64_t)plan->nsplit * plan->ntargets * 2;
    const int64_t nblk = ((int64_t)plan->ntargets + NEAR_WARPS - 1) / NEAR_WARPS;
    const int grid_n = (int)(nblk < (1 << 20) ? nblk : (1 << 20));
    k_cross_near<<<grid_n, NEAR_WARPS * 32, 0, st>>>(plan->targets, plan->ntargets, plan->patch_dev, plan->npatches, sigma, dx, dy,
                                         plan->lattice_unit, plan->geom.G, near);
    SG_CUDA_TRY(cudaGetLastError());
    k_cross_combine<<<(plan->ntargets + 255) / 256, 256, 0, st>>>(plan->targets, plan->ntargets, plan->nsplit,
                                                                   ws->partial, fx, fy);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_DIRECT, st);
    return SG_OK;
}

// ============================================================ potential ====
//
// The same cross-patch sum for the mid-plane potential Phi = -G sum_i of the
// cell integrals of (sigma0_i + deltax_i (xbar - xc_i) + deltay_i (ybar - yc_i)) / r.
// With l_i(t) as above, xbar - xc_i = u + (x_t - xc_i), so the cell integral is
// l_i(t) P0 + deltax_i U + deltay_i V with P0, U, V the integrals of 1/r, u/r,
// v/r, and Section 2's antiderivatives give the corner form
//   Phi(t) = -G sum_c [ A_c(t) F0(c - t) + X_c Fu(c - t) + Y_c Fv(c - t) ],
//   F0 = u g0 + v g0y,  Fu = (v r + u^2 g0) / 2,  Fv = (u r + v^2 g0y) / 2
// (u ln(v + r) + v ln(u + r) and (v r + u^2 ln(v + r)) / 2 with the terms of one
// variable alone dropped, which cancel in each cell's double difference; every
// term vanishes where its factor u or v does, so the potential needs no
// coincident-line form). Far cells in FP32 plans: the cell average of 1/rho
// over the unit square by its moments (f = 1/rho, p = 1/rho, centre minus
// target (a, b) in cell widths, Laplacian of p = p^3, bilaplacian = 9 p^5):
//   I0 = p + p^3/24 + p^5 (-7/1920 + (7/96) a^2 b^2 p^4)
//   Ix = -a p^3/12 + (7/240) a p^5 - a p^7 (a^2/32 + 5 b^2/96)   (Iy: a <-> b)
// and Phi_cell = -G H (m I0 + deltax H Ix + deltay H Iy). Truncation relative
// to the cell's p is below 1e-7 from SG_NEAR_R cell widths on; from SG_FAR_R4
// on the p^5 and p^7 terms (below 2e-7 relative) are dropped.

// One cell's far potential per unit (-G H): c = (m, deltax H / 8, deltay H / 8).
template <int ORDER>
__device__ __forceinline__ float cell_far_pot(float a, float b, float b2, const float4 c)
{
    const float r2 = fmaf(a, a, b2);
    const float p = rsqrtf(r2);
    const float s = p * p;
    const float p3 = p * s;
    // m-moments and slope moments (8 d = deltax H)
    float i0 = fmaf(p3, 1.f / 24.f, p);
    float kx = p3 * (-8.f / 12.f), ky = kx;
    if (ORDER >= 6) {
        const float p5 = p3 * s, p7 = p5 * s;
        const float ab = a * b;
        i0 = fmaf(p5, fmaf(ab * ab * s * s, 7.f / 96.f, -7.f / 1920.f), i0);
        kx = fmaf(p5, 8.f * 7.f / 240.f, kx);
        ky = kx;
        kx = fmaf(-8.f * p7, fmaf(a, a * (1.f / 32.f), b2 * (5.f / 96.f)), kx);
        ky = fmaf(-8.f * p7, fmaf(b2, 1.f / 32.f, a * a * (5.f / 96.f)), ky);
    }
    return fmaf(c.x, i0, fmaf(c.y * a, kx, c.z * b * ky));
}

template <int ORDER, bool MASK>
__device__ __forceinline__ float tile_far_pot(const float4 *__restrict__ w, float a0, float b0)
{
    float q = 0.f;
#pragma unroll 1
    for (int r = 0; r < SG_TILE_Y; ++r) {
        const float b = b0 + (float)r;
        const float b2 = b * b;
        const bool bnear = fabsf(b) < (float)SG_NEAR_R;
#pragma unroll
        for (int c = 0; c < SG_TILE_X; ++c) {
            const float a = a0 + (float)c;
            const float v = cell_far_pot<ORDER>(a, b, b2, w[r * SG_TILE_X + c]);
            if (MASK) q += (bnear && fabsf(a) < (float)SG_NEAR_R) ? 0.f : v;
            else q += v;
        }
    }
    return q;
}

// The potential's persistent far-field launch: k_cross_far's work items,
// staging and bounded waits; one output per target (partial[.. * 2]).
__global__ void __launch_bounds__(SG_DIRECT_THREADS) k_cross_far_pot(
    const sg_target_block *__restrict__ blocks, int nblocks, const int4 *__restrict__ targets,
    const sg_tile_desc *__restrict__ tiles, const sg_patch_dev *__restrict__ pd, int ntiles,
    const float4 *__restrict__ coefs, int nsplit, double G, double lambda, double *__restrict__ partial,
    int ntargets, int *__restrict__ words, int tries)
{
    __shared__ __align__(128) float4 buf[FAR_STAGES][SG_TILE_N];
    __shared__ uint64_t full[FAR_STAGES];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    if (tid == 0)
        for (int s = 0; s < FAR_STAGES; ++s) mbar_init(&full[s], 1);
    __syncthreads();
    uint32_t used = 0, issued = 0;
    const int nitems = nblocks * nsplit;
    bool failed = false;
    while (!failed) {
        if (tid == 0) s_item = atomicAdd(&words[1], 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        const int bi = item / nsplit, split = item - bi * nsplit;
        const sg_target_block blk = blocks[bi];
        const int t0 = (int)((int64_t)ntiles * split / nsplit), t1 = (int)((int64_t)ntiles * (split + 1) / nsplit);
        const int own0 = pd[blk.patch].tile_first, own1 = own0 + pd[blk.patch].tile_count;
        const int n1 = max(0, min(t1, own0) - t0), s2 = max(t0, own1);
        const int n = n1 + max(0, t1 - s2);
        const bool active = tid < blk.count;
        const int4 tg = targets[blk.first + (active ? tid : 0)];
        if (tid == 0) {
            for (int k = 0; k < n && k < FAR_STAGES; ++k, ++issued) {
                const int stg = issued % FAR_STAGES;
                const int t = k < n1 ? t0 + k : s2 + (k - n1);
                mbar_arrive_expect_tx(&full[stg], TILE_BYTES);
                bulk_copy_g2s(buf[stg], coefs + (int64_t)t * SG_TILE_N, TILE_BYTES, &full[stg]);
            }
        }
        double acc = 0.0;
        for (int k = 0; k < n; ++k, ++used) {
            const int stg = used % FAR_STAGES;
            const int t = k < n1 ? t0 + k : s2 + (k - n1);
            const bool ok = mbar_wait_bounded(&full[stg], (used / FAR_STAGES) & 1, tries);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            const sg_tile_desc td = tiles[t];
            const int cx0 = td.ox + td.step / 2, cx1 = cx0 + (SG_TILE_X - 1) * td.step;
            const int cy0 = td.oy + td.step / 2, cy1 = cy0 + (SG_TILE_Y - 1) * td.step;
            const int gx = max(0, max(cx0 - blk.tx1, blk.tx0 - cx1));
            const int gy = max(0, max(cy0 - blk.ty1, blk.ty0 - cy1));
            const int gap = max(gx, gy);
            const float inv = 1.0f / (float)td.step;
            const float a0 = (float)(td.ox - tg.x) * inv + 0.5f, b0 = (float)(td.oy - tg.y) * inv + 0.5f;
            float q;
            if (gap >= SG_FAR_R4 * td.step) q = tile_far_pot<4, false>(buf[stg], a0, b0);
            else if (gap >= SG_NEAR_R * td.step) q = tile_far_pot<6, false>(buf[stg], a0, b0);
            else q = tile_far_pot<6, true>(buf[stg], a0, b0);
            acc = fma((double)td.step * lambda, (double)q, acc);  // times the tile's cell width H
            __syncthreads();
            if (tid == 0 && k + FAR_STAGES < n) {
                const int kk = k + FAR_STAGES;
                const int tn = kk < n1 ? t0 + kk : s2 + (kk - n1);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect_tx(&full[stg], TILE_BYTES);
                bulk_copy_g2s(buf[stg], coefs + (int64_t)tn * SG_TILE_N, TILE_BYTES, &full[stg]);
                ++issued;
            }
        }
        if (failed) break;
        if (active) partial[((int64_t)split * ntargets + blk.first + tid) * 2] = -G * acc;
    }
    if (failed && tid == 0) {
        atomicExch(&words[0], 1);
        for (uint32_t g = used; g < issued; ++g) mbar_wait_bounded(&full[g % FAR_STAGES], (g / FAR_STAGES) & 1, SG_MBAR_MAX_TRIES);
    }
}

// The corner functions of the potential at (u, v) = corner - target, r = |(u, v)|,
// from the logarithms ln(|v| + r) - ln|u| and ln(|u| + r) - ln|v| (t0, t1);
// accumulates A F0 + X Fu + Y Fv.
__device__ __forceinline__ double corner_pot(double u, double v, double r, double t0, double t1, double A, double X,
                                             double Y)
{
    const double g0 = (v == 0.0 || u == 0.0) ? 0.0 : (v > 0.0 ? t0 : -t0);   // multiplied by u, u^2
    const double g0y = (u == 0.0 || v == 0.0) ? 0.0 : (u > 0.0 ? t1 : -t1);  // multiplied by v, v^2
    const double ug = u * g0, vg = v * g0y;
    const double F0 = ug + vg;
    const double Fu = 0.5 * fma(v, r, u * ug);
    const double Fv = 0.5 * fma(u, r, v * vg);
    return fma(A, F0, fma(X, Fu, Y * Fv));
}

// FP64 corner form of the potential (k_cross_direct's layout; one output).
__global__ void __launch_bounds__(SG_DIRECT_THREADS) k_cross_direct_pot(
    const sg_target_block *__restrict__ blocks, const int4 *__restrict__ targets, const sg_tile_desc *__restrict__ tiles,
    int ntiles, const double *__restrict__ wts, int nsplit, double G, double lambda, double *__restrict__ phi,
    double *__restrict__ partial, int ntargets)
{
    __shared__ sg_dvec4 sw[SG_TILE_N];
    const sg_target_block blk = blocks[blockIdx.x];
    const int split = blockIdx.y;
    const int t0 = (int)((int64_t)ntiles * split / nsplit);
    const int t1 = (int)((int64_t)ntiles * (split + 1) / nsplit);
    const bool active = threadIdx.x < blk.count;
    int4 tg = make_int4(0, 0, -1, -1);
    if (active) tg = targets[blk.first + threadIdx.x];
    double acc = 0.0;
    const sg_dvec4 *wv = reinterpret_cast<const sg_dvec4 *>(wts);
    for (int t = t0; t < t1; ++t) {
        const sg_tile_desc td = tiles[t];
        if (td.patch == blk.patch) continue;  // same-patch pairs come from the FFT
        __syncthreads();
        for (int k = threadIdx.x; k < SG_TILE_N; k += SG_DIRECT_THREADS) sw[k] = wv[(int64_t)t * SG_TILE_N + k];
        __syncthreads();
        const double du0 = (double)(td.ox - tg.x), dv0 = (double)(td.oy - tg.y), st = (double)td.step;
        const double dxT = (double)(tg.x - td.ox), dyT = (double)(tg.y - td.oy);
        double Lu[SG_TILE_X];
#pragma unroll
        for (int c = 0; c < SG_TILE_X; ++c) {
            const double u = fma((double)c, st, du0);
            Lu[c] = u == 0.0 ? 0.0 : log(fabs(u));
        }
        double sum = 0.0;
#pragma unroll 1
        for (int r = 0; r < SG_TILE_Y; ++r) {
            const double v = fma((double)r, st, dv0);
            const double av = fabs(v), v2 = v * v;
            const double Lv = v == 0.0 ? 0.0 : log(av);
#pragma unroll 4
            for (int c = 0; c < SG_TILE_X; ++c) {
                const sg_dvec4 wc = sw[r * SG_TILE_X + c];
                const double u = fma((double)c, st, du0);
                const double rr = sqrt(fma(u, u, v2));
                const double A = fma(dxT, wc.y, fma(dyT, wc.z, wc.x));
                sum += corner_pot(u, v, rr, log(av + rr) - Lu[c], log(fabs(u) + rr) - Lv, A, wc.y, wc.z);
            }
        }
        acc += sum;
    }
    if (!active) return;
    // corner offsets are in lattice units: F0 is a length and Fu, Fv are lengths
    // squared, against weights X, Y that carry one lattice unit already, so one
    // factor lambda makes every term physical
    const double P = -G * lambda * acc;
    const int ti = blk.first + threadIdx.x;
    if (nsplit == 1) phi[tg.z] += P;
    else partial[(int64_t)split * ntargets + ti] = P;
}

__global__ void k_cross_reduce_pot(const int4 *__restrict__ targets, int ntargets, int nsplit,
                                   const double *__restrict__ partial, double *__restrict__ phi)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntargets; t += gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int s = 0; s < nsplit; ++s) sum += partial[(int64_t)s * ntargets + t];
        phi[targets[t].z] += sum;
    }
}

// Near field of the potential in FP64 (k_cross_near's boxes, staging and warp
// reduction; one output).
__global__ void __launch_bounds__(NEAR_WARPS * 32) k_cross_near_pot(const int4 *__restrict__ targets, int ntargets,
                                                                   const sg_patch_dev *__restrict__ pd, int npatches,
                                                                   const float *__restrict__ sigma,
                                                                   const float *__restrict__ dx,
                                                                   const float *__restrict__ dy, double lambda,
                                                                   double G, double *__restrict__ near_out)
{
    __shared__ double cellv[NEAR_WARPS][3][NEAR_SLOTS];
    const int lane = threadIdx.x & 31;
    double *cl = cellv[threadIdx.x >> 5][0], *cx = cellv[threadIdx.x >> 5][1], *cy = cellv[threadIdx.x >> 5][2];
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    for (int t = warp; t < ntargets; t += nwarps) {
        const int4 tg = targets[t];
        double ph = 0.0;
        for (int q = 0; q < npatches; ++q) {
            if (q == tg.w) continue;
            const sg_patch_dev &p = pd[q];
            const int64_t L = p.step, RL = (int64_t)SG_NEAR_R * L;
            const int64_t ex = (int64_t)tg.x - p.ox - L / 2, ey = (int64_t)tg.y - p.oy - L / 2;
            const int i0 = max(0, floor_div(ex - RL, L) + 1), j0 = max(0, floor_div(ey - RL, L) + 1);
            const int i1 = min(p.nx - 1, -floor_div(-(ex + RL), L) - 1);
            const int j1 = min(p.ny - 1, -floor_div(-(ey + RL), L) - 1);
            if (i0 > i1 || j0 > j1) continue;
            const int nbx = i1 - i0 + 1, nby = j1 - j0 + 1, W = nbx + 2;
            __syncwarp();  // the previous box's values have been read
            for (int k = lane; k < W * (nby + 2); k += 32) {
                const int bi = k % W - 1, bj = k / W - 1;
                double l = 0.0, X = 0.0, Y = 0.0;
                if (bi >= 0 && bi < nbx && bj >= 0 && bj < nby) {
                    const int i = i0 + bi, j = j0 + bj;
                    const int64_t o = p.cell_off + (int64_t)j * p.nx + i;
                    X = dx[o];
                    Y = dy[o];
                    const double ux = ((double)tg.x - ((double)p.ox + (i + 0.5) * (double)L)) * lambda;
                    const double uy = ((double)tg.y - ((double)p.oy + (j + 0.5) * (double)L)) * lambda;
                    l = fma(X, ux, fma(Y, uy, (double)sigma[o]));
                }
                cl[k] = l;
                cx[k] = X;
                cy[k] = Y;
            }
            const double uc = ((double)p.ox + (double)(i0 + lane) * L - tg.x) * lambda;
            const double vc = ((double)p.oy + (double)(j0 + lane) * L - tg.y) * lambda;
            const double lnu = lane <= nbx ? (uc == 0.0 ? 0.0 : log(fabs(uc))) : 0.0;
            const double lnv = lane <= nby ? (vc == 0.0 ? 0.0 : log(fabs(vc))) : 0.0;
            __syncwarp();
            const int nci = nbx + 1, ncorner = nci * (nby + 1);
            for (int base = 0; base < ncorner; base += 32) {
                const int k = base + lane;
                const bool valid = k < ncorner;
                const int kk = valid ? k : 0;
                const int ci = kk % nci, cj = kk / nci;
                const double Lu = __shfl_sync(0xffffffffu, lnu, ci);
                const double Lv = __shfl_sync(0xffffffffu, lnv, cj);
                if (!valid) continue;
                const int s00 = cj * W + ci, s10 = s00 + 1, s01 = s00 + W, s11 = s01 + 1;
                const double A = (cl[s00] - cl[s10]) - (cl[s01] - cl[s11]);
                const double X = (cx[s00] - cx[s10]) - (cx[s01] - cx[s11]);
                const double Y = (cy[s00] - cy[s10]) - (cy[s01] - cy[s11]);
                const double u = ((double)p.ox + (double)(i0 + ci) * L - tg.x) * lambda;
                const double v = ((double)p.oy + (double)(j0 + cj) * L - tg.y) * lambda;
                const double r = sqrt(fma(u, u, v * v));
                ph += corner_pot(u, v, r, log(fabs(v) + r) - Lu, log(fabs(u) + r) - Lv, A, X, Y);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ph += __shfl_xor_sync(0xffffffffu, ph, off);
        if (lane == 0) near_out[(int64_t)t * 2] = -G * ph;
    }
}

// Fixed-order sum into the potential: the patch's own FFT result, the far
// partials of every split, then the near field.
__global__ void k_cross_combine_pot(const int4 *__restrict__ targets, int ntargets, int nsplit,
                                    const double *__restrict__ partial, float *__restrict__ phi)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntargets; t += gridDim.x * blockDim.x) {
        double sum = 0.0;
        for (int s = 0; s <= nsplit; ++s) sum += partial[((int64_t)s * ntargets + t) * 2];
        const int o = targets[t].z;
        phi[o] = (float)((double)phi[o] + sum);
    }
}

sg_status cross_potential_f64(sg_plan *plan, const sg_workspace *ws, const double *sigma, const double *dx,
                              const double *dy, double *phi, cudaStream_t st)
{
    double *w = (double *)ws->tile_w;
    const int64_t nw = (int64_t)plan->ntiles * SG_TILE_N;
    int grid_w = (int)((nw + 255) / 256);
    if (grid_w > 65535) grid_w = 65535;
    sg_timing_begin(ws, SG_STAGE_WEIGHTS, st);
    k_corner_weights<double><<<grid_w, 256, 0, st>>>(plan->tiles, plan->ntiles, plan->patch_dev, sigma, dx, dy,
                                             plan->lattice_unit, w);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_WEIGHTS, st);
    sg_timing_begin(ws, SG_STAGE_DIRECT, st);
    dim3 grid(plan->nblocks, plan->nsplit);
    k_cross_direct_pot<<<grid, SG_DIRECT_THREADS, 0, st>>>(plan->blocks, plan->targets, plan->tiles, plan->ntiles, w,
                                                           plan->nsplit, plan->geom.G, plan->lattice_unit, phi,
                                                           ws->partial, plan->ntargets);
    SG_CUDA_TRY(cudaGetLastError());
    if (plan->nsplit > 1) {
        k_cross_reduce_pot<<<(plan->ntargets + 255) / 256, 256, 0, st>>>(plan->targets, plan->ntargets,
                                                                          plan->nsplit, ws->partial, phi);
        SG_CUDA_TRY(cudaGetLastError());
    }
    sg_timing_end(ws, SG_STAGE_DIRECT, st);
    return SG_OK;
}

sg_status cross_potential_f32(sg_plan *plan, const sg_workspace *ws, const float *sigma, const float *dx,
                              const float *dy, float *phi, cudaStream_t st)
{
    float4 *w = (float4 *)ws->tile_w;
    const int64_t nw = (int64_t)plan->ntiles * SG_TILE_N;
    int grid_w = (int)((nw + 255) / 256);
    if (grid_w > 65535) grid_w = 65535;
    sg_timing_begin(ws, SG_STAGE_WEIGHTS, st);
    k_cell_coefs<<<grid_w, 256, 0, st>>>(plan->tiles, plan->ntiles, plan->patch_dev, sigma, dx, dy,
                                         plan->lattice_unit, w, ws->err + 1);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_WEIGHTS, st);
    sg_timing_begin(ws, SG_STAGE_DIRECT, st);
    k_cross_far_pot<<<plan->far_grid, SG_DIRECT_THREADS, 0, st>>>(plan->blocks, plan->nblocks, plan->targets,
                                                                  plan->tiles, plan->patch_dev, plan->ntiles, w,
                                                                  plan->nsplit, plan->geom.G, plan->lattice_unit,
                                                                  ws->partial, plan->ntargets, ws->err,
                                                                  plan->wait_tries);
    SG_CUDA_TRY(cudaGetLastError());
    double *near = ws->partial + (int64_t)plan->nsplit * plan->ntargets * 2;
    const int64_t nblk = ((int64_t)plan->ntargets + NEAR_WARPS - 1) / NEAR_WARPS;
    const int grid_n = (int)(nblk < (1 << 20) ? nblk : (1 << 20));
    k_cross_near_pot<<<grid_n, NEAR_WARPS * 32, 0, st>>>(plan->targets, plan->ntargets, plan->patch_dev,
                                                         plan->npatches, sigma, dx, dy, plan->lattice_unit,
                                                         plan->geom.G, near);
    SG_CUDA_TRY(cudaGetLastError());
    k_cross_combine_pot<<<(plan->ntargets + 255) / 256, 256, 0, st>>>(plan->targets, plan->ntargets, plan->nsplit,
                                                                       ws->partial, phi);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_DIRECT, st);
    return SG_OK;
}

// ============================================================ off plane ====
//
// Targets at height z != 0 above the plane of the sources (Section 2's kernels
// with R = sqrt(u^2 + v^2 + z^2)): FP64 plans sum every pair in the corner form
// with the off-plane antiderivatives; FP32 plans use it for the near cells and
// Gauss-Legendre quadrature of the cell integrals for the far cells (below).
// With the corner weights A_c(t), X_c, Y_c as in the plane,
//   Fx(t) = G sum_c [ -A_c G0 + X_c (v G0y - |z| T) - Y_c R ]
//   Fy(t) = G sum_c [ -A_c G0y + Y_c (u G0 - |z| T) - X_c R ]
//   Fz(t) = G sum_c [ -sgn(z) A_c T + z (X_c G0 + Y_c G0y) ]
// G0 = asinh(v / rho_u), rho_u = sqrt(u^2 + z^2), G0y = asinh(u / rho_v),
// T = atan(u v / (|z| R)): the x-family kernels K^{x,0} = -dd G0,
// K^{x,x} = -m K^{x,0} + dd[v G0y] - |z| dd T, K^{x,y} = -n K^{x,0} - dd R, and
// K^{z,0} = -sgn(z) dd T, K^{z,x} = -m K^{z,0} - z K^{x,0} (y-family by
// symmetry), the -m, -n terms folded into A_c(t). R >= |z| > 0: no coincident
// lines. asinh(v / rho) = sgn(v) (ln(|v| + R) - ln rho), rho per corner column
// (row) of the tile.

// grid (nblocks, nsplit); one leaf target per thread; partial[(split, target)][3].
__global__ void __launch_bounds__(SG_DIRECT_THREADS) k_cross_direct_z(
    const sg_target_block *__restrict__ blocks, const int4 *__restrict__ targets, const sg_tile_desc *__restrict__ tiles,
    int ntiles, const double *__restrict__ wts, int nsplit, double G, double zl, double *__restrict__ partial,
    int ntargets)
{
    __shared__ sg_dvec4 sw[SG_TILE_N];
    const sg_target_block blk = blocks[blockIdx.x];
    const int split = blockIdx.y;
    const int t0 = (int)((int64_t)ntiles * split / nsplit);
    const int t1 = (int)((int64_t)ntiles * (split + 1) / nsplit);
    const bool active = threadIdx.x < blk.count;
    int4 tg = make_int4(0, 0, -1, -1);
    if (active) tg = targets[blk.first + threadIdx.x];
    const double az = fabs(zl), z2 = zl * zl, sz = zl > 0.0 ? 1.0 : -1.0;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    const sg_dvec4 *wv = reinterpret_cast<const sg_dvec4 *>(wts);
    for (int t = t0; t < t1; ++t) {
        const sg_tile_desc td = tiles[t];
        if (td.patch == blk.patch) continue;  // same-patch pairs come from the FFT
        __syncthreads();
        for (int k = threadIdx.x; k < SG_TILE_N; k += SG_DIRECT_THREADS) sw[k] = wv[(int64_t)t * SG_TILE_N + k];
        __syncthreads();
        const double du0 = (double)(td.ox - tg.x), dv0 = (double)(td.oy - tg.y), st = (double)td.step;
        const double dxT = (double)(tg.x - td.ox), dyT = (double)(tg.y - td.oy);
        double Lu[SG_TILE_X];
#pragma unroll
        for (int c = 0; c < SG_TILE_X; ++c) {
            const double u = fma((double)c, st, du0);
            Lu[c] = 0.5 * log(fma(u, u, z2));  // ln rho_u
        }
        double sx = 0.0, sy = 0.0, sz3 = 0.0;
#pragma unroll 1
        for (int r = 0; r < SG_TILE_Y; ++r) {
            const double v = fma((double)r, st, dv0);
            const double av = fabs(v), v2z = fma(v, v, z2);
            const double Lv = 0.5 * log(v2z);  // ln rho_v
#pragma unroll 2
            for (int c = 0; c < SG_TILE_X; ++c) {
                const sg_dvec4 wc = sw[r * SG_TILE_X + c];
                const double u = fma((double)c, st, du0);
                const double R = sqrt(fma(u, u, v2z));
                const double ta = log(av + R) - Lu[c];
                const double tb = log(fabs(u) + R) - Lv;
                const double g0 = v > 0.0 ? ta : (v < 0.0 ? -ta : 0.0);
                const double g0y = u > 0.0 ? tb : (u < 0.0 ? -tb : 0.0);
                const double T = atan(u * v / (az * R));
                const double A = fma(dxT, wc.y, fma(dyT, wc.z, wc.x));
                sx += fma(-A, g0, fma(wc.y, fma(v, g0y, -az * T), -wc.z * R));
                sy += fma(-A, g0y, fma(wc.z, fma(u, g0, -az * T), -wc.y * R));
                sz3 += fma(-sz * A, T, zl * fma(wc.y, g0, wc.z * g0y));
            }
        }
        fx += sx;
        fy += sy;
        fz += sz3;
    }
    if (!active) return;
    double *o = partial + ((int64_t)split * ntargets + blk.first + threadIdx.x) * 3;
    o[0] = G * fx;
    o[1] = G * fy;
    o[2] = G * fz;
}

// Fixed-order sum of the splits, added into the outputs.
template <typename T>
__global__ void k_cross_reduce_z(const int4 *__restrict__ targets, int ntargets, int nsplit,
                                 const double *__restrict__ partial, T *__restrict__ fx, T *__restrict__ fy,
                                 T *__restrict__ fz)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntargets; t += gridDim.x * blockDim.x) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int s = 0; s < nsplit; ++s) {
            const double *q = partial + ((int64_t)s * ntargets + t) * 3;
            a += q[0];
            b += q[1];
            c += q[2];
        }
        const int o = targets[t].z;
        fx[o] = (T)((double)fx[o] + a);
        fy[o] = (T)((double)fy[o] + b);
        if (fz) fz[o] = (T)((double)fz[o] + c);  // sg_force on such a plan returns Fx, Fy only
    }
}

// FP32 plans off the plane: near cells (k_cross_far's near box) in the FP64
// corner form above, far cells by tensor Gauss-Legendre quadrature of the cell
// integrals of (m + deltax H xi + deltay H eta) (a + xi, b + eta, -zeta) / R^3
// over the unit cell (a, b = centre minus target, zeta = z, in cell widths):
// 3 x 3 nodes from SG_NEAR_R cell widths on (relative error below 3e-7 there,
// from the sixth derivative of the kernel), 2 x 2 from SG_FAR_R4 on (below 1e-6),
// in FP32 per tile and FP64 across tiles like the in-plane far field.
template <int NG>
__device__ __forceinline__ void cell_far_z(float a, float b, float zeta2, float4 c, float &qx, float &qy, float &qz)
{
    // nodes on [-1/2, 1/2] and weights summing to 1
    constexpr float X3 = 0.387298334620742f, W3a = 5.f / 18.f, W3b = 8.f / 18.f;
    constexpr float X2 = 0.288675134594813f;
    float sx = 0.f, sy = 0.f, s0 = 0.f;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const float xi = NG == 3 ? (i == 0 ? -X3 : (i == 1 ? 0.f : X3)) : (i == 0 ? -X2 : X2);
        const float wi = NG == 3 ? (i == 1 ? W3b : W3a) : 0.5f;
        const float da = a + xi;
        const float da2z = fmaf(da, da, zeta2);
#pragma unroll
        for (int j = 0; j < NG; ++j) {
            const float eta = NG == 3 ? (j == 0 ? -X3 : (j == 1 ? 0.f : X3)) : (j == 0 ? -X2 : X2);
            const float wj = NG == 3 ? (j == 1 ? W3b : W3a) : 0.5f;
            const float db = b + eta;
            const float ir = rsqrtf(fmaf(db, db, da2z));
            // density at the node (c.y, c.z = deltax H / 8, deltay H / 8) times weight / R^3
            const float w = wi * wj * fmaf(8.f * c.y, xi, fmaf(8.f * c.z, eta, c.x)) * (ir * ir * ir);
            sx = fmaf(w, da, sx);
            sy = fmaf(w, db, sy);
            s0 += w;
        }
    }
    qx += sx;
    qy += sy;
    qz += s0;  // times -zeta by the caller
}

template <int NG, bool MASK>
__device__ __forceinline__ void tile_far_z(const float4 *__restrict__ w, float a0, float b0, float zeta, double &ax,
                                           double &ay, double &az)
{
    float qx = 0.f, qy = 0.f, qz = 0.f;
    const float zeta2 = zeta * zeta;
#pragma unroll 1
    for (int r = 0; r < SG_TILE_Y; ++r) {
        const float b = b0 + (float)r;
        const bool bnear = fabsf(b) < (float)SG_NEAR_R;
#pragma unroll 2
        for (int c = 0; c < SG_TILE_X; ++c) {
            const float a = a0 + (float)c;
            if (MASK && bnear && fabsf(a) < (float)SG_NEAR_R) continue;
            cell_far_z<NG>(a, b, zeta2, w[r * SG_TILE_X + c], qx, qy, qz);
        }
    }
    ax += qx;
    ay += qy;
    az += (double)(-zeta) * (double)qz;
}

// Persistent far field off the plane (k_cross_far's items, staging, waits);
// partial[(split, target)][3].
__global__ void __launch_bounds__(SG_DIRECT_THREADS) k_cross_far_z(
    const sg_target_block *__restrict__ blocks, int nblocks, const int4 *__restrict__ targets,
    const sg_tile_desc *__restrict__ tiles, const sg_patch_dev *__restrict__ pd, int ntiles,
    const float4 *__restrict__ coefs, int nsplit, double G, double zl, double *__restrict__ partial, int ntargets,
    int *__restrict__ words, int tries)
{
    __shared__ __align__(128) float4 buf[FAR_STAGES][SG_TILE_N];
    __shared__ uint64_t full[FAR_STAGES];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    if (tid == 0)
        for (int s = 0; s < FAR_STAGES; ++s) mbar_init(&full[s], 1);
    __syncthreads();
    uint32_t used = 0, issued = 0;
    const int nitems = nblocks * nsplit;
    bool failed = false;
    while (!failed) {
        if (tid == 0) s_item = atomicAdd(&words[1], 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        const int bi = item / nsplit, split = item - bi * nsplit;
        const sg_target_block blk = blocks[bi];
        const int t0 = (int)((int64_t)ntiles * split / nsplit), t1 = (int)((int64_t)ntiles * (split + 1) / nsplit);
        const int own0 = pd[blk.patch].tile_first, own1 = own0 + pd[blk.patch].tile_count;
        const int n1 = max(0, min(t1, own0) - t0), s2 = max(t0, own1);
        const int n = n1 + max(0, t1 - s2);
        const bool active = tid < blk.count;
        const int4 tg = targets[blk.first + (active ? tid : 0)];
        if (tid == 0) {
            for (int k = 0; k < n && k < FAR_STAGES; ++k, ++issued) {
                const int stg = issued % FAR_STAGES;
                const int t = k < n1 ? t0 + k : s2 + (k - n1);
                mbar_arrive_expect_tx(&full[stg], TILE_BYTES);
                bulk_copy_g2s(buf[stg], coefs + (int64_t)t * SG_TILE_N, TILE_BYTES, &full[stg]);
            }
        }
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int k = 0; k < n; ++k, ++used) {
            const int stg = used % FAR_STAGES;
            const int t = k < n1 ? t0 + k : s2 + (k - n1);
            const bool ok = mbar_wait_bounded(&full[stg], (used / FAR_STAGES) & 1, tries);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            const sg_tile_desc td = tiles[t];
            const int cx0 = td.ox + td.step / 2, cx1 = cx0 + (SG_TILE_X - 1) * td.step;
            const int cy0 = td.oy + td.step / 2, cy1 = cy0 + (SG_TILE_Y - 1) * td.step;
            const int gx = max(0, max(cx0 - blk.tx1, blk.tx0 - cx1));
            const int gy = max(0, max(cy0 - blk.ty1, blk.ty0 - cy1));
            const int gap = max(gx, gy);
            const float inv = 1.0f / (float)td.step;
            const float a0 = (float)(td.ox - tg.x) * inv + 0.5f, b0 = (float)(td.oy - tg.y) * inv + 0.5f;
            const float zeta = (float)(zl / (double)td.step);  // the height in the tile's cell widths
            if (gap >= SG_FAR_R4 * td.step) tile_far_z<2, false>(buf[stg], a0, b0, zeta, ax, ay, az);
            else if (gap >= SG_NEAR_R * td.step) tile_far_z<3, false>(buf[stg], a0, b0, zeta, ax, ay, az);
            else tile_far_z<3, true>(buf[stg], a0, b0, zeta, ax, ay, az);
            __syncthreads();
            if (tid == 0 && k + FAR_STAGES < n) {
                const int kk = k + FAR_STAGES;
                const int tn = kk < n1 ? t0 + kk : s2 + (kk - n1);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect_tx(&full[stg], TILE_BYTES);
                bulk_copy_g2s(buf[stg], coefs + (int64_t)tn * SG_TILE_N, TILE_BYTES, &full[stg]);
                ++issued;
            }
        }
        if (failed) break;
        if (active) {
            double *o = partial + ((int64_t)split * ntargets + blk.first + tid) * 3;
            o[0] = G * ax;
            o[1] = G * ay;
            o[2] = G * az;
        }
    }
    if (failed && tid == 0) {
        atomicExch(&words[0], 1);
        for (uint32_t g = used; g < issued; ++g) mbar_wait_bounded(&full[g % FAR_STAGES], (g / FAR_STAGES) & 1, SG_MBAR_MAX_TRIES);
    }
}

// Near cells off the plane in FP64: k_cross_near's boxes and warp reduction
// with the off-plane corner form; writes slice nsplit of partial[.][3].
__global__ void __launch_bounds__(NEAR_WARPS * 32) k_cross_near_z(const int4 *__restrict__ targets, int ntargets,
                                                                 const sg_patch_dev *__restrict__ pd, int npatches,
                                                                 const float *__restrict__ sigma,
                                                                 const float *__restrict__ dx,
                                                                 const float *__restrict__ dy, double lambda,
                                                                 double G, double z, double *__restrict__ near_out)
{
    __shared__ double cellv[NEAR_WARPS][3][NEAR_SLOTS];
    const int lane = threadIdx.x & 31;
    double *cl = cellv[threadIdx.x >> 5][0], *cx = cellv[threadIdx.x >> 5][1], *cy = cellv[threadIdx.x >> 5][2];
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    const double az = fabs(z), z2 = z * z, sz = z > 0.0 ? 1.0 : -1.0;
    for (int t = warp; t < ntargets; t += nwarps) {
        const int4 tg = targets[t];
        double fx = 0.0, fy = 0.0, fzs = 0.0;
        for (int q = 0; q < npatches; ++q) {
            if (q == tg.w) continue;
            const sg_patch_dev &p = pd[q];
            const int64_t L = p.step, RL = (int64_t)SG_NEAR_R * L;
            const int64_t ex = (int64_t)tg.x - p.ox - L / 2, ey = (int64_t)tg.y - p.oy - L / 2;
            const int i0 = max(0, floor_div(ex - RL, L) + 1), j0 = max(0, floor_div(ey - RL, L) + 1);
            const int i1 = min(p.nx - 1, -floor_div(-(ex + RL), L) - 1);
            const int j1 = min(p.ny - 1, -floor_div(-(ey + RL), L) - 1);
            if (i0 > i1 || j0 > j1) continue;
            const int nbx = i1 - i0 + 1, nby = j1 - j0 + 1, W = nbx + 2;
            __syncwarp();  // the previous box's values have been read
            for (int k = lane; k < W * (nby + 2); k += 32) {
                const int bi = k % W - 1, bj = k / W - 1;
                double l = 0.0, X = 0.0, Y = 0.0;
                if (bi >= 0 && bi < nbx && bj >= 0 && bj < nby) {
                    const int i = i0 + bi, j = j0 + bj;
                    const int64_t o = p.cell_off + (int64_t)j * p.nx + i;
                    X = dx[o];
                    Y = dy[o];
                    const double ux = ((double)tg.x - ((double)p.ox + (i + 0.5) * (double)L)) * lambda;
                    const double uy = ((double)tg.y - ((double)p.oy + (j + 0.5) * (double)L)) * lambda;
                    l = fma(X, ux, fma(Y, uy, (double)sigma[o]));
                }
                cl[k] = l;
                cx[k] = X;
                cy[k] = Y;
            }
            // ln rho_u of corner column ci and ln rho_v of corner row cj in lanes
            const double uc = ((double)p.ox + (double)(i0 + lane) * L - tg.x) * lambda;
            const double vc = ((double)p.oy + (double)(j0 + lane) * L - tg.y) * lambda;
            const double lnu = lane <= nbx ? 0.5 * log(fma(uc, uc, z2)) : 0.0;
            const double lnv = lane <= nby ? 0.5 * log(fma(vc, vc, z2)) : 0.0;
            __syncwarp();
            const int nci = nbx + 1, ncorner = nci * (nby + 1);
            for (int base = 0; base < ncorner; base += 32) {
                const int k = base + lane;
                const bool valid = k < ncorner;
                const int kk = valid ? k : 0;
                const int ci = kk % nci, cj = kk / nci;
                const double Lu = __shfl_sync(0xffffffffu, lnu, ci);
                const double Lv = __shfl_sync(0xffffffffu, lnv, cj);
                if (!valid) continue;
                const int s00 = cj * W + ci, s10 = s00 + 1, s01 = s00 + W, s11 = s01 + 1;
                const double A = (cl[s00] - cl[s10]) - (cl[s01] - cl[s11]);
                const double X = (cx[s00] - cx[s10]) - (cx[s01] - cx[s11]);
                const double Y = (cy[s00] - cy[s10]) - (cy[s01] - cy[s11]);
                const double u = ((double)p.ox + (double)(i0 + ci) * L - tg.x) * lambda;
                const double v = ((double)p.oy + (double)(j0 + cj) * L - tg.y) * lambda;
                const double R = sqrt(fma(u, u, fma(v, v, z2)));
                const double ta = log(fabs(v) + R) - Lu, tb = log(fabs(u) + R) - Lv;
                const double g0 = v > 0.0 ? ta : (v < 0.0 ? -ta : 0.0);
                const double g0y = u > 0.0 ? tb : (u < 0.0 ? -tb : 0.0);
                const double T = atan(u * v / (az * R));
                fx += fma(-A, g0, fma(X, fma(v, g0y, -az * T), -Y * R));
                fy += fma(-A, g0y, fma(Y, fma(u, g0, -az * T), -X * R));
                fzs += fma(-sz * A, T, z * fma(X, g0, Y * g0y));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, off);
            fy += __shfl_xor_sync(0xffffffffu, fy, off);
            fzs += __shfl_xor_sync(0xffffffffu, fzs, off);
        }
        if (lane == 0) {
            near_out[(int64_t)t * 3 + 0] = G * fx;
            near_out[(int64_t)t * 3 + 1] = G * fy;
            near_out[(int64_t)t * 3 + 2] = G * fzs;
        }
    }
}

sg_status cross_solve_z_f32(sg_plan *plan, const sg_workspace *ws, const float *sigma, const float *dx,
                            const float *dy, float *fx, float *fy, float *fz, cudaStream_t st)
{
    float4 *w = (float4 *)ws->tile_w;
    const int64_t nw = (int64_t)plan->ntiles * SG_TILE_N;
    int grid_w = (int)((nw + 255) / 256);
    if (grid_w > 65535) grid_w = 65535;
    sg_timing_begin(ws, SG_STAGE_WEIGHTS, st);
    k_cell_coefs<<<grid_w, 256, 0, st>>>(plan->tiles, plan->ntiles, plan->patch_dev, sigma, dx, dy,
                                         plan->lattice_unit, w, ws->err + 1);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_WEIGHTS, st);
    sg_timing_begin(ws, SG_STAGE_DIRECT, st);
    k_cross_far_z<<<plan->far_grid, SG_DIRECT_THREADS, 0, st>>>(plan->blocks, plan->nblocks, plan->targets, plan->tiles,
                                                                plan->patch_dev, plan->ntiles, w, plan->nsplit,
                                                                plan->geom.G, plan->geom.z / plan->lattice_unit,
                                                                ws->partial, plan->ntargets, ws->err,
                                                                plan->wait_tries);
    SG_CUDA_TRY(cudaGetLastError());
    double *near = ws->partial + (int64_t)plan->nsplit * plan->ntargets * 3;
    const int64_t nblk = ((int64_t)plan->ntargets + NEAR_WARPS - 1) / NEAR_WARPS;
    const int grid_n = (int)(nblk < (1 << 20) ? nblk : (1 << 20));
    k_cross_near_z<<<grid_n, NEAR_WARPS * 32, 0, st>>>(plan->targets, plan->ntargets, plan->patch_dev,
                                                       plan->npatches, sigma, dx, dy, plan->lattice_unit,
                                                       plan->geom.G, plan->geom.z, near);
    SG_CUDA_TRY(cudaGetLastError());
    // the splits and the near slice, in a fixed order
    k_cross_reduce_z<float><<<(plan->ntargets + 255) / 256, 256, 0, st>>>(plan->targets, plan->ntargets,
                                                                           plan->nsplit + 1, ws->partial, fx, fy, fz);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_DIRECT, st);
    return SG_OK;
}

template <typename T>
sg_status cross_solve_z(sg_plan *plan, const sg_workspace *ws, const T *sigma, const T *dx, const T *dy, T *fx,
                        T *fy, T *fz, cudaStream_t st)
{
    double *w = (double *)ws->tile_w;
    const int64_t nw = (int64_t)plan->ntiles * SG_TILE_N;
    int grid_w = (int)((nw + 255) / 256);
    if (grid_w > 65535) grid_w = 65535;
    sg_timing_begin(ws, SG_STAGE_WEIGHTS, st);
    k_corner_weights<T><<<grid_w, 256, 0, st>>>(plan->tiles, plan->ntiles, plan->patch_dev, sigma, dx, dy,
                                                plan->lattice_unit, w);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_WEIGHTS, st);
    sg_timing_begin(ws, SG_STAGE_DIRECT, st);
    dim3 grid(plan->nblocks, plan->nsplit);
    k_cross_direct_z<<<grid, SG_DIRECT_THREADS, 0, st>>>(plan->blocks, plan->targets, plan->tiles, plan->ntiles, w,
                                                         plan->nsplit, plan->geom.G, plan->geom.z / plan->lattice_unit,
                                                         ws->partial, plan->ntargets);
    SG_CUDA_TRY(cudaGetLastError());
    k_cross_reduce_z<T><<<(plan->ntargets + 255) / 256, 256, 0, st>>>(plan->targets, plan->ntargets, plan->nsplit,
                                                                       ws->partial, fx, fy, fz);
    SG_CUDA_TRY(cudaGetLastError());
    sg_timing_end(ws, SG_STAGE_DIRECT, st);
    return SG_OK;
}

}  // namespace

sg_status sg_cross_far_grid(sg_plan *plan, int nsm)
{
    int per_sm = 0;
    if (plan->geom.z != 0.0)
        SG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cross_far_z, SG_DIRECT_THREADS, 0));
    else
        SG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cross_far, SG_DIRECT_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    const int64_t items = (int64_t)plan->nblocks * plan->nsplit;
    int64_t g = (int64_t)nsm * per_sm;
    if (g > items) g = items;
    plan->far_grid = (int)(g < 1 ? 1 : g);
    return SG_OK;
}

sg_status sg_cross_solve(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                         void *fx, void *fy, void *fz, cudaStream_t st)
{
    if (plan->ntiles == 0 || plan->ntargets == 0) return SG_OK;
    if (plan->geom.z != 0.0) {
        if (plan->prec == SG_FP64)
            return cross_solve_z<double>(plan, ws, (const double *)sigma, (const double *)dx, (const double *)dy,
                                         (double *)fx, (double *)fy, (double *)fz, st);
        return cross_solve_z_f32(plan, ws, (const float *)sigma, (const float *)dx, (const float *)dy, (float *)fx,
                                 (float *)fy, (float *)fz, st);
    }
    if (plan->prec == SG_FP64)
        return cross_solve_f64(plan, ws, (const double *)sigma, (const double *)dx, (const double *)dy, (double *)fx,
                               (double *)fy, st);
    return cross_solve_f32(plan, ws, (const float *)sigma, (const float *)dx, (const float *)dy, (float *)fx,
                           (float *)fy, st);
}

sg_status sg_cross_potential(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                             void *phi, cudaStream_t st)
{
    if (plan->ntiles == 0 || plan->ntargets == 0) return SG_OK;
    if (plan->prec == SG_FP64)
        return cross_potential_f64(plan, ws, (const double *)sigma, (const double *)dx, (const double *)dy,
                                   (double *)phi, st);
    return cross_potential_f32(plan, ws, (const float *)sigma, (const float *)dx, (const float *)dy, (float *)phi,
                               st);
}
