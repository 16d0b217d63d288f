// Composite sources of an AMR hierarchy.
//
// The force of Eq. eqnXforce2 sums the piecewise-linear density of the leaf
// cells. The same function is the telescoping sum over patches of
//   S_0 = f_0                                  on level-0 patches,
//   S_l = f_l - P(f_{l-1})                     on a patch of level l >= 1,
// where f_l is the level-l data with every covered cell filled by the
// restriction of its four children, and P(f_{l-1}) is the parent's linear
// function evaluated on the children (exact: a linear function restricted to a
// child cell is linear, same slopes, value at the child centre). At any point
// the sum telescopes to the leaf density there, so summing the closed-form
// integrals over the S_l of every patch gives the leaf sum exactly. The gain is
// numerical: S_l (l >= 1) is the difference between two representations of the
// same density and is small, and f_0 has no hole, so no corner weight along a
// patch boundary is of the size of the density itself.
//
// Restriction (any choice cancels in the sum): sigma0 = mean(sigma0_k) over the
// four children, and
//   with caller slopes:  deltax = mean(deltax_k), deltay = mean(deltay_k);
//   order 0:             the least-squares linear fit over the parent of width H,
//                        deltax = (3 / (4 H)) (sum_right sigma0_k - sum_left sigma0_k),
//                        deltay likewise with top and bottom.
// For smooth data both give the gradient to O(H^2), so the defects S_l are
// O(H^2). With slopes supplied the children's mean slope stays of the size of
// the data's slopes even for rough data, where a least-squares slope grows like
// (jump in sigma) / H and the large slope terms of consecutive levels, which
// cancel in the sum, would cost digits in the corner-form sum.
#include "common.cuh"

namespace {

// Fill the cells of patch p: leaves copy the input, covered cells restrict
// their children's filled values (already written: patches run finest first),
// cells that do not exist get zero.
template <typename T>
__global__ void k_fill(sg_patch_dev p, const int *__restrict__ code, const sg_patch_dev *__restrict__ pd,
                       const T *__restrict__ sigma, const T *__restrict__ dx, const T *__restrict__ dy,
                       T *__restrict__ s)
{
    const bool slopes = dx != nullptr;
    const int64_t n = (int64_t)p.nx * p.ny;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % p.nx), j = (int)(e / p.nx);
        const int64_t o = p.cell_off + e;
        const int c = code[o];
        double s0 = 0.0, sx = 0.0, sy = 0.0;
        if (c == SG_CELL_LEAF) {
            s0 = (double)sigma[o];
            sx = dx ? (double)dx[o] : 0.0;
            sy = dy ? (double)dy[o] : 0.0;
        } else if (c >= 0) {
            const sg_patch_dev q = pd[c];
            const int ci = 2 * (i - q.pi0), cj = 2 * (j - q.pj0);
            double sum = 0, right = 0, top = 0, gx = 0, gy = 0;
            for (int b = 0; b < 2; ++b) {
                for (int a = 0; a < 2; ++a) {
                    const int64_t oc = q.cell_off + (int64_t)(cj + b) * q.nx + (ci + a);
                    const double v = (double)s[oc];
                    sum += v;
                    right += a ? v : -v;
                    top += b ? v : -v;
                    gx += (double)s[oc + q.ncells_plane];
                    gy += (double)s[oc + 2 * q.ncells_plane];
                }
            }
            s0 = 0.25 * sum;
            sx = slopes ? 0.25 * gx : 0.75 / p.h * right;
            sy = slopes ? 0.25 * gy : 0.75 / p.h * top;
        }
        s[o] = (T)s0;
        s[o + p.ncells_plane] = (T)sx;
        s[o + 2 * p.ncells_plane] = (T)sy;
    }
}

// Replace the filled values of patch q (level >= 1) by q - P(parent), in place.
template <typename T>
__global__ void k_defect(sg_patch_dev q, sg_patch_dev p, const int *__restrict__ code, T *__restrict__ s)
{
    const int64_t n = (int64_t)q.nx * q.ny;
    const int64_t P = q.ncells_plane;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % q.nx), j = (int)(e / q.nx);
        const int64_t o = q.cell_off + e;
        if (code[o] == SG_CELL_ABSENT) continue;
        const int64_t op = p.cell_off + (int64_t)(q.pj0 + j / 2) * p.nx + (q.pi0 + i / 2);
        const double ox = ((i & 1) - 0.5) * q.h, oy = ((j & 1) - 0.5) * q.h;
        const double px = (double)s[op + P], py = (double)s[op + 2 * P];
        const double pv = (double)s[op] + px * ox + py * oy;
        s[o] = (T)((double)s[o] - pv);
        s[o + P] = (T)((double)s[o + P] - px);
        s[o + 2 * P] = (T)((double)s[o + 2 * P] - py);
    }
}

template <typename T>
sg_status prepare_t(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                    cudaStream_t st)
{
    T *s = (T *)ws->sfield;
    const bool slopes = plan->geom.slope_mode == SG_SLOPES_CALLER;
    for (int k = plan->npatches - 1; k >= 0; --k) {
        const sg_patch_dev &d = plan->pp[k].d;
        const int64_t n = (int64_t)d.nx * d.ny;
        int grid = (int)((n + 255) / 256);
        if (grid > 4096) grid = 4096;
        k_fill<T><<<grid, 256, 0, st>>>(d, plan->cell_code, plan->patch_dev, (const T *)sigma,
                                        slopes ? (const T *)dx : nullptr, slopes ? (const T *)dy : nullptr, s);
        SG_CUDA_TRY(cudaGetLastError());
    }
    for (int k = plan->npatches - 1; k >= 0; --k) {
        const sg_patch_dev &d = plan->pp[k].d;
        if (d.parent < 0) continue;
        const int64_t n = (int64_t)d.nx * d.ny;
        int grid = (int)((n + 255) / 256);
        if (grid > 4096) grid = 4096;
        k_defect<T><<<grid, 256, 0, st>>>(d, plan->pp[d.parent].d, plan->cell_code, s);
        SG_CUDA_TRY(cudaGetLastError());
    }
    return SG_OK;
}

}  // namespace

sg_status sg_amr_prepare(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                         cudaStream_t st)
{
    sg_timing_begin(ws, SG_STAGE_COMPOSITE, st);
    sg_status r = plan->prec == SG_FP64 ? prepare_t<double>(plan, ws, sigma, dx, dy, st)
                                        : prepare_t<float>(plan, ws, sigma, dx, dy, st);
    sg_timing_end(ws, SG_STAGE_COMPOSITE, st);
    return r;
}
