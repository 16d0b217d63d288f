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
//
// Launches: one per refined level below the finest (finest first) for the
// filled values of its covered cells, then one for every S_l: a refined level's
// defect needs only its own 2x2 sibling blocks (the parent's filled value is
// their restriction), so all levels are finalised together.
#include "common.cuh"

namespace {

// Filled value of a cell that is the child of a covered cell, or of a cell being
// finalised: its input on a leaf, zero where it does not exist, and the filled
// value computed by an earlier launch (planes F) where it is covered itself.
// Arithmetic here runs in the plan precision T (FP64 throughput is a small
// fraction of FP32 on this GPU, and every value is stored in T anyway).
template <typename T>
__device__ __forceinline__ void cell_value(const int *__restrict__ code, const T *__restrict__ sigma,
                                           const T *__restrict__ dx, const T *__restrict__ dy,
                                           const T *__restrict__ F, int64_t P, int64_t o, T v[3])
{
    const int c = code[o];
    if (c == SG_CELL_LEAF) {
        v[0] = sigma[o];
        v[1] = dx ? dx[o] : (T)0;
        v[2] = dy ? dy[o] : (T)0;
    } else if (c == SG_CELL_ABSENT) {
        v[0] = v[1] = v[2] = (T)0;
    } else {
        v[0] = F[o];
        v[1] = F[o + P];
        v[2] = F[o + 2 * P];
    }
}

// Restriction of the four cells (ci..ci+1, cj..cj+1) of patch q to their parent
// of width hp.
template <typename T>
__device__ __forceinline__ void restrict4(const int *__restrict__ code, const T *__restrict__ sigma,
                                          const T *__restrict__ dx, const T *__restrict__ dy,
                                          const T *__restrict__ F, const sg_patch_dev &q, int ci, int cj, double hp,
                                          T v[4][3], T out[3])
{
    const bool slopes = dx != nullptr;
    T sum = 0, right = 0, top = 0, gx = 0, gy = 0;
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 2; ++a) {
            T *w = v[2 * b + a];
            cell_value(code, sigma, dx, dy, F, q.ncells_plane, q.cell_off + (int64_t)(cj + b) * q.nx + (ci + a), w);
            sum += w[0];
            right += a ? w[0] : -w[0];
            top += b ? w[0] : -w[0];
            gx += w[1];
            gy += w[2];
        }
    }
    const T c = (T)0.75 / (T)hp;
    out[0] = (T)0.25 * sum;
    out[1] = slopes ? (T)0.25 * gx : c * right;
    out[2] = slopes ? (T)0.25 * gy : c * top;
}

// The patch table (sorted order, prefix sums, descriptors) of plans with few
// patches is copied into shared memory at kernel start, so that the lookups of
// every work item (binary search, patch, child patch) do not wait on global loads.
constexpr int COMP_SMEM_PATCHES = 128;

struct patch_table {
    const sg_patch_dev *pd;
    const int *order;
    const int64_t *pre;
};

__device__ __forceinline__ patch_table stage_patch_table(const sg_patch_dev *__restrict__ pd,
                                                         const int *__restrict__ order,
                                                         const int64_t *__restrict__ pre, int n)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (n > COMP_SMEM_PATCHES) return {pd, order, pre};
    sg_patch_dev *spd = reinterpret_cast<sg_patch_dev *>(smem_raw);
    int64_t *spre = reinterpret_cast<int64_t *>(spd + n);
    int *sorder = reinterpret_cast<int *>(spre + n + 1);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        spd[k] = pd[k];
        sorder[k] = order[k];
    }
    for (int k = threadIdx.x; k <= n; k += blockDim.x) spre[k] = pre[k];
    __syncthreads();
    return {spd, sorder, spre};
}

inline size_t patch_table_bytes(int n)
{
    return n > COMP_SMEM_PATCHES ? 0 : (size_t)n * sizeof(sg_patch_dev) + (size_t)(n + 1) * 8 + (size_t)n * 4;
}

// Patch k and item r of the patches order[t0 .. t1) with item prefix sums pre[]
__device__ __forceinline__ int find_item(const int64_t *__restrict__ pre, int t0, int t1, int64_t e)
{
    int lo = t0, hi = t1 - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Filled values F of the covered cells of one refined level (patches order[t0 .. t1),
// cells prefix cpre): the restriction of their children (finer levels done earlier).
template <typename T>
__global__ void k_fill_covered(const sg_patch_dev *__restrict__ gpd, const int *__restrict__ code,
                               const int *__restrict__ gorder, const int64_t *__restrict__ gcpre, int npatches, int t0,
                               int t1, const T *__restrict__ sigma, const T *__restrict__ dx, const T *__restrict__ dy,
                               T *__restrict__ F)
{
    sg_dep_trigger();
    sg_dep_wait();  // the covered cells of the level above
    const patch_table tab = stage_patch_table(gpd, gorder, gcpre, npatches);
    const sg_patch_dev *pd = tab.pd;
    const int *order = tab.order;
    const int64_t *cpre = tab.pre;
    const int64_t base = cpre[t0], n = cpre[t1] - base;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = find_item(cpre, t0, t1, base + e);
        const sg_patch_dev p = pd[order[t]];
        const int64_t r = base + e - cpre[t];
        const int i = (int)(r % p.nx), j = (int)(r / p.nx);
        const int64_t o = p.cell_off + r;
        const int c = code[o];
        if (c < 0) continue;
        const sg_patch_dev q = pd[c];
        T v[4][3], f[3];
        restrict4(code, sigma, dx, dy, F, q, 2 * (i - q.pi0), 2 * (j - q.pj0), p.h, v, f);
        const int64_t P = p.ncells_plane;
        F[o] = f[0];
        F[o + P] = f[1];
        F[o + 2 * P] = f[2];
    }
}

// The composite sources of every patch (items of the patches order[0 .. n),
// prefix fpre): a level-0 cell gets its filled value; a 2x2 block of siblings on
// a refined level gets filled value - P(parent), where the parent's filled value
// is the restriction of these four cells (the value the parent's own restriction
// produced).
template <typename T>
__global__ void k_composite(const sg_patch_dev *__restrict__ gpd, const int *__restrict__ code,
                            const int *__restrict__ gorder, const int64_t *__restrict__ gfpre, int n,
                            const T *__restrict__ sigma, const T *__restrict__ dx, const T *__restrict__ dy,
                            const T *__restrict__ F, T *__restrict__ s)
{
    sg_dep_trigger();
    sg_dep_wait();  // the filled values of the covered cells
    const patch_table tab = stage_patch_table(gpd, gorder, gfpre, n);
    const sg_patch_dev *pd = tab.pd;
    const int *order = tab.order;
    const int64_t *fpre = tab.pre;
    const int64_t nitems = fpre[n];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nitems; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = find_item(fpre, 0, n, e);
        const sg_patch_dev p = pd[order[t]];
        const int64_t P = p.ncells_plane;
        const int64_t r = e - fpre[t];
        T v[4][3], f[3];
        if (p.parent < 0) {
            const int64_t o = p.cell_off + r;
            const int c = code[o];
            if (c >= 0) {
                const sg_patch_dev q = pd[c];
                const int i = (int)(r % p.nx), j = (int)(r / p.nx);
                restrict4(code, sigma, dx, dy, F, q, 2 * (i - q.pi0), 2 * (j - q.pj0), p.h, v, f);
            } else {
                cell_value(code, sigma, dx, dy, F, P, o, f);
            }
            s[o] = f[0];
            s[o + P] = f[1];
            s[o + 2 * P] = f[2];
            continue;
        }
        const int bw = p.nx / 2;
        const int bi = (int)(r % bw), bj = (int)(r / bw);
        const int64_t o00 = p.cell_off + (int64_t)(2 * bj) * p.nx + 2 * bi;
        if (code[o00] == SG_CELL_ABSENT) {  // blocks are wholly absent or present
            for (int q = 0; q < 4; ++q) {
                const int64_t o = o00 + (int64_t)(q >> 1) * p.nx + (q & 1);
                s[o] = s[o + P] = s[o + 2 * P] = (T)0;
            }
            continue;
        }
        restrict4(code, sigma, dx, dy, F, p, 2 * bi, 2 * bj, pd[p.parent].h, v, f);
        for (int q = 0; q < 4; ++q) {
            const int a = q & 1, b = q >> 1;
            const int64_t o = o00 + (int64_t)b * p.nx + a;
            const T ox = ((T)a - (T)0.5) * (T)p.h, oy = ((T)b - (T)0.5) * (T)p.h;
            const T pv = f[0] + f[1] * ox + f[2] * oy;
            s[o] = v[q][0] - pv;
            s[o + P] = v[q][1] - f[1];
            s[o + 2 * P] = v[q][2] - f[2];
        }
    }
}

int grid_for(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// Neighbour-leaf slopes of the leaves among the cells c0 .. c1 (one level; the
// coarser levels' slopes are in D already). Per axis, deltax = (v_R - v_L) /
// (x_R - x_L) from what lies across the two sides (links nb, see sg_plan):
// a leaf of the level (its sigma0 at its centre), a refined cell (the mean of
// the two children touching the side: their sigma0, or their filled value F
// when refined themselves, at their centres), a coarser leaf (its linear
// reconstruction sigma0 + delta_perp (t_perp - c_perp) at its centre line), or
// nothing (0 at one cell width). Exact for a linear density. FP64 arithmetic.
template <typename T>
__global__ void k_amr_slopes(const int2 *__restrict__ nb, const int2 *__restrict__ pos, const int *__restrict__ code,
                             const T *__restrict__ sigma, const T *__restrict__ F, T *__restrict__ D, int64_t P,
                             int64_t c0, int64_t c1, int step, double lambda)
{
    for (int64_t c = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < c1; c += (int64_t)gridDim.x * blockDim.x) {
        if (code[c] != SG_CELL_LEAF) {
            D[c] = D[c + P] = (T)0;
            continue;
        }
        const int2 tp = pos[c];
        double out[2];
#pragma unroll
        for (int axis = 0; axis < 2; ++axis) {
            double v[2], x[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int side = axis == 0 ? 2 * k : 2 * k + 1;  // left, down, right, up
                const int2 d = nb[c * 4 + side];
                const double t_ax = axis == 0 ? tp.x : tp.y;
                if (d.y >= 0) {
                    const double va = code[d.x] == SG_CELL_LEAF ? (double)sigma[d.x] : (double)F[d.x];
                    const double vb = code[d.y] == SG_CELL_LEAF ? (double)sigma[d.y] : (double)F[d.y];
                    const int2 pa = pos[d.x], pb = pos[d.y];
                    v[k] = 0.5 * (va + vb);
                    x[k] = axis == 0 ? 0.5 * ((double)pa.x + pb.x) : 0.5 * ((double)pa.y + pb.y);
                } else if (d.y == -1) {
                    const int2 pa = pos[d.x];
                    v[k] = sigma[d.x];
                    x[k] = axis == 0 ? pa.x : pa.y;
                } else if (d.y == -2) {
                    const int2 pa = pos[d.x];
                    // the coarser leaf's slope across the axis: deltay for the x axis, deltax for y
                    const double perp = axis == 0 ? (double)D[d.x + P] * ((double)tp.y - pa.y)
                                                  : (double)D[d.x] * ((double)tp.x - pa.x);
                    v[k] = (double)sigma[d.x] + perp * lambda;
                    x[k] = axis == 0 ? pa.x : pa.y;
                } else {
                    v[k] = 0.0;
                    x[k] = t_ax + (k ? step : -step);
                }
            }
            out[axis] = (v[1] - v[0]) / ((x[1] - x[0]) * lambda);
        }
        D[c] = (T)out[0];
        D[c + P] = (T)out[1];
    }
}

template <typename T>
sg_status prepare_t(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                    cudaStream_t st, bool fill_only = false)
{
    T *s = (T *)ws->sfield;
    T *F = s + 3 * plan->ncells;  // filled values of covered cells
    const bool slopes = dx != nullptr && dy != nullptr;
    const T *sx = slopes ? (const T *)dx : nullptr, *sy = slopes ? (const T *)dy : nullptr;
    const int lmax = plan->comp_depth - 1;
    // covered cells of the refined levels, finest first (level lmax has none)
    for (int l = lmax - 1; l >= 1; --l) {
        const int t0 = plan->comp_lev_first[l], t1 = plan->comp_lev_first[l + 1];
        const int64_t n = plan->comp_cells_host[t1] - plan->comp_cells_host[t0];
        if (n <= 0) continue;
        // the finest fill reads the caller's fields: an ordinary launch; the next ones depend on it
        auto kf = k_fill_covered<T>;
        if (l == lmax - 1)
            kf<<<grid_for(n), 256, patch_table_bytes(plan->npatches), st>>>(
                plan->patch_dev, plan->cell_code, plan->comp_order, plan->comp_cells, plan->npatches, t0, t1,
                (const T *)sigma, sx, sy, F);
        else
            SG_CUDA_TRY(sg_launch_dep(kf, dim3(grid_for(n)), dim3(256), patch_table_bytes(plan->npatches), st,
                                      plan->patch_dev, plan->cell_code, plan->comp_order, plan->comp_cells,
                                      plan->npatches, t0, t1, (const T *)sigma, sx, sy, F));
        SG_CUDA_TRY(cudaGetLastError());
    }
    if (fill_only) return SG_OK;
    auto kc = k_composite<T>;
    if (lmax >= 2)  // after the fills of the covered cells
        SG_CUDA_TRY(sg_launch_dep(kc, dim3(grid_for(plan->comp_items)), dim3(256), patch_table_bytes(plan->npatches),
                                  st, plan->patch_dev, plan->cell_code, plan->comp_order, plan->comp_item_off,
                                  plan->npatches, (const T *)sigma, sx, sy, (const T *)F, s));
    else
        kc<<<grid_for(plan->comp_items), 256, patch_table_bytes(plan->npatches), st>>>(
            plan->patch_dev, plan->cell_code, plan->comp_order, plan->comp_item_off, plan->npatches, (const T *)sigma,
            sx, sy, F, s);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

}  // namespace

// Slopes of a hierarchy with SG_SLOPES_CENTRAL into the workspace planes D
// (after the composite's filled values F of the covered cells), one launch per
// level from the coarsest (a leaf's slope reads only coarser leaves' slopes).
template <typename T>
sg_status slopes_t(sg_plan *plan, const sg_workspace *ws, const void *sigma, cudaStream_t st)
{
    T *s = (T *)ws->sfield;
    const int64_t P = plan->ncells;
    const T *F = s + 3 * P;
    T *D = s + 6 * P;
    for (int l = 0; l < plan->comp_depth; ++l) {
        const int64_t c0 = plan->lev_cells[l], c1 = plan->lev_cells[l + 1];
        if (c1 <= c0) continue;
        k_amr_slopes<T><<<grid_for(c1 - c0), 256, 0, st>>>(plan->slope_nb, plan->cell_pos, plan->cell_code,
                                                          (const T *)sigma, F, D, P, c0, c1, plan->lev_step[l],
                                                          plan->lattice_unit);
        SG_CUDA_TRY(cudaGetLastError());
    }
    return SG_OK;
}

sg_status sg_composite_prepare(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx,
                               const void *dy, cudaStream_t st)
{
    if (!plan->amr_central) return sg_amr_prepare(plan, ws, sigma, dx, dy, st);
    sg_timing_begin(ws, SG_STAGE_COMPOSITE, st);
    const size_t es = plan->prec == SG_FP64 ? 8 : 4;
    const char *D = (const char *)ws->sfield + 6 * (size_t)plan->ncells * es;
    sg_status r = plan->prec == SG_FP64 ? prepare_t<double>(plan, ws, sigma, nullptr, nullptr, st, true)
                                        : prepare_t<float>(plan, ws, sigma, nullptr, nullptr, st, true);
    if (r == SG_OK)
        r = plan->prec == SG_FP64 ? slopes_t<double>(plan, ws, sigma, st) : slopes_t<float>(plan, ws, sigma, st);
    if (r == SG_OK)
        r = plan->prec == SG_FP64 ? prepare_t<double>(plan, ws, sigma, D, D + (size_t)plan->ncells * es, st)
                                  : prepare_t<float>(plan, ws, sigma, D, D + (size_t)plan->ncells * es, st);
    sg_timing_end(ws, SG_STAGE_COMPOSITE, st);
    return r;
}

sg_status sg_amr_prepare(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                         cudaStream_t st)
{
    sg_timing_begin(ws, SG_STAGE_COMPOSITE, st);
    sg_status r = plan->prec == SG_FP64 ? prepare_t<double>(plan, ws, sigma, dx, dy, st)
                                        : prepare_t<float>(plan, ws, sigma, dx, dy, st);
    sg_timing_end(ws, SG_STAGE_COMPOSITE, st);
    return r;
}
