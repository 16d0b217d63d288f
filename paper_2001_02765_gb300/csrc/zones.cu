// Zone-by-zone (quadtree) hierarchies: Berger-Oliger refinement as in Fig. 1
// and Table 10 (each refined zone split into four children), of which the ILR
// and VLR hierarchies of Section 4 are instances. The force acts on, and is
// summed over, the leaf zones (Eq. eqnXforce2).
//
// A zone list is laid out as masked patches so that the patch machinery (FFT
// convolution inside a patch, corner-form direct sum across patches, composite
// sources) applies unchanged:
//   level 0   the bounding box of the level-0 zones, cut into at most 2048-wide
//             pieces;
//   level l   for every patch of level l - 1, the bounding box of the level-l
//             zones whose parents lie in it (aligned to whole parent zones),
//             cut the same way;
// each piece shrunk to the zones it holds (whole parent zones) and dropped if
// empty. A cell of a patch exists where a zone was listed. Solves take and
// return zone-ordered arrays: a gather into the patch layout, the solve, a
// scatter of the leaf forces back.
#include "common.cuh"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <unordered_map>
#include <vector>

namespace {

sg_status zfail(const char *msg)
{
    sg_set_last_error_message(msg);
    return SG_EINVAL;
}

inline uint64_t zkey(int level, int64_t ix, int64_t iy)
{
    return ((uint64_t)level << 58) | ((uint64_t)iy << 29) | (uint64_t)ix;
}

// Checks the rules of sg_zones and builds the (level, ix, iy) -> index map.
sg_status zones_index(const sg_zones *z, std::unordered_map<uint64_t, int64_t> &idx, int &lmax)
{
    if (!z) return zfail("zone list is NULL");
    if (z->nzones < 1 || !z->level || !z->ix || !z->iy) return zfail("zone list is empty");
    if (z->nx0 < 1 || z->ny0 < 1) return zfail("level-0 grid size must be >= 1");
    if (!(z->h0 > 0.0) || !isfinite(z->h0) || !isfinite(z->x0) || !isfinite(z->y0))
        return zfail("level-0 origin or zone width invalid");
    char msg[160];
    lmax = 0;
    idx.clear();
    idx.reserve((size_t)z->nzones * 2);
    for (int64_t k = 0; k < z->nzones; ++k) {
        const int l = z->level[k];
        if (l < 0 || l >= SG_MAX_LEVELS) {
            snprintf(msg, sizeof(msg), "zone %lld: level %d out of range [0, %d)", (long long)k, l, SG_MAX_LEVELS);
            return zfail(msg);
        }
        const int64_t nx = (int64_t)z->nx0 << l, ny = (int64_t)z->ny0 << l;
        if (nx > (1LL << 22) || ny > (1LL << 22)) {
            snprintf(msg, sizeof(msg), "zone %lld: level %d spans more than 2^22 zones per axis", (long long)k, l);
            return zfail(msg);
        }
        if (z->ix[k] < 0 || z->ix[k] >= nx || z->iy[k] < 0 || z->iy[k] >= ny) {
            snprintf(msg, sizeof(msg), "zone %lld: (%d, %d) outside the level-%d grid", (long long)k, z->ix[k],
                     z->iy[k], l);
            return zfail(msg);
        }
        if (!idx.emplace(zkey(l, z->ix[k], z->iy[k]), k).second) {
            snprintf(msg, sizeof(msg), "zone %lld: (level %d, %d, %d) listed twice", (long long)k, l, z->ix[k],
                     z->iy[k]);
            return zfail(msg);
        }
        if (l > lmax) lmax = l;
    }
    for (int64_t k = 0; k < z->nzones; ++k) {
        const int l = z->level[k];
        if (l == 0) continue;
        const int64_t i = z->ix[k], j = z->iy[k];
        if (!idx.count(zkey(l - 1, i >> 1, j >> 1))) {
            snprintf(msg, sizeof(msg), "zone %lld: parent (level %d, %lld, %lld) not listed", (long long)k, l - 1,
                     (long long)(i >> 1), (long long)(j >> 1));
            return zfail(msg);
        }
        for (int q = 0; q < 4; ++q) {
            if (!idx.count(zkey(l, (i & ~1LL) + (q & 1), (j & ~1LL) + (q >> 1)))) {
                snprintf(msg, sizeof(msg), "zone %lld: a sibling of (level %d, %lld, %lld) is not listed", (long long)k,
                         l, (long long)i, (long long)j);
                return zfail(msg);
            }
        }
    }
    return SG_OK;
}

struct box {
    int64_t x0, y0, x1, y1;  // half-open, in zones of the box's level
};

// Cut [a0, a1) (even ends when `even`) into n nearly equal pieces of whole parent zones.
std::vector<int64_t> cuts(int64_t a0, int64_t a1, bool even)
{
    const int64_t unit = even ? 2 : 1;
    const int64_t m = (a1 - a0) / unit;
    const int64_t n = (a1 - a0 + SG_MAX_PATCH_SIDE - 1) / SG_MAX_PATCH_SIDE;
    std::vector<int64_t> c(n + 1);
    for (int64_t p = 0; p <= n; ++p) c[p] = a0 + unit * (m * p / n);
    return c;
}

struct layout {
    std::vector<sg_patch> patches;
    std::vector<std::vector<uint8_t>> masks;
    std::vector<int64_t> slot;  // per zone, cell index in the patch layout
};

// Masked-patch layout of a validated zone list.
sg_status zones_layout(const sg_zones *z, int lmax, layout &out)
{
    const int64_t n = z->nzones;
    std::vector<int> zpatch(n, -1);
    std::vector<std::vector<int64_t>> by_level(lmax + 1);
    for (int64_t k = 0; k < n; ++k) by_level[z->level[k]].push_back(k);
    std::vector<box> boxes;  // per patch
    for (int l = 0; l <= lmax; ++l) {
        const double h = z->h0 / (double)(1LL << l);
        // group the level's zones by the patch of their parent (one group on level 0)
        std::unordered_map<int, std::vector<int64_t>> groups;
        std::vector<int> order;
        for (int64_t k : by_level[l]) {
            int g = 0;
            if (l > 0) {
                // the parent is the zone at level l-1 containing (ix/2, iy/2); its patch is known
                g = -1;
                const int64_t pi = z->ix[k] >> 1, pj = z->iy[k] >> 1;
                // find among the level-(l-1) patches the one whose box holds the parent
                for (size_t q = 0; q < boxes.size(); ++q) {
                    const sg_patch &pp = out.patches[q];
                    const box &b = boxes[q];
                    if (pp.level == l - 1 && pi >= b.x0 && pi < b.x1 && pj >= b.y0 && pj < b.y1) {
                        g = (int)q;
                        break;
                    }
                }
                if (g < 0) return zfail("internal: a zone's parent lies in no patch");
            }
            auto it = groups.find(g);
            if (it == groups.end()) {
                order.push_back(g);
                groups[g].push_back(k);
            } else {
                it->second.push_back(k);
            }
        }
        std::sort(order.begin(), order.end());
        for (int g : order) {
            const std::vector<int64_t> &zs = groups[g];
            box bb = {INT64_MAX, INT64_MAX, INT64_MIN, INT64_MIN};
            for (int64_t k : zs) {
                bb.x0 = std::min<int64_t>(bb.x0, z->ix[k]);
                bb.y0 = std::min<int64_t>(bb.y0, z->iy[k]);
                bb.x1 = std::max<int64_t>(bb.x1, z->ix[k] + 1);
                bb.y1 = std::max<int64_t>(bb.y1, z->iy[k] + 1);
            }
            const bool even = l > 0;  // whole parent zones (siblings are complete, so the box is even already)
            const std::vector<int64_t> cx = cuts(bb.x0, bb.x1, even), cy = cuts(bb.y0, bb.y1, even);
            const int npx = (int)cx.size() - 1, npy = (int)cy.size() - 1;
            // assign zones to pieces, then shrink every piece to its zones
            std::vector<std::vector<int64_t>> piece((size_t)npx * npy);
            for (int64_t k : zs) {
                const int a = (int)(std::upper_bound(cx.begin(), cx.end(), (int64_t)z->ix[k]) - cx.begin()) - 1;
                const int b = (int)(std::upper_bound(cy.begin(), cy.end(), (int64_t)z->iy[k]) - cy.begin()) - 1;
                piece[(size_t)b * npx + a].push_back(k);
            }
            for (const std::vector<int64_t> &pz : piece) {
                if (pz.empty()) continue;
                box t = {INT64_MAX, INT64_MAX, INT64_MIN, INT64_MIN};
                for (int64_t k : pz) {
                    t.x0 = std::min<int64_t>(t.x0, z->ix[k]);
                    t.y0 = std::min<int64_t>(t.y0, z->iy[k]);
                    t.x1 = std::max<int64_t>(t.x1, z->ix[k] + 1);
                    t.y1 = std::max<int64_t>(t.y1, z->iy[k] + 1);
                }
                const int pidx = (int)out.patches.size();
                sg_patch p;
                p.level = l;
                p.nx = (int)(t.x1 - t.x0);
                p.ny = (int)(t.y1 - t.y0);
                p.x0 = z->x0 + (double)t.x0 * h;
                p.y0 = z->y0 + (double)t.y0 * h;
                p.h = h;
                out.patches.push_back(p);
                boxes.push_back(t);
                std::vector<uint8_t> m((size_t)p.nx * p.ny, 0);
                for (int64_t k : pz) {
                    m[(size_t)(z->iy[k] - t.y0) * p.nx + (z->ix[k] - t.x0)] = 1;
                    zpatch[k] = pidx;
                }
                out.masks.push_back(std::move(m));
            }
        }
    }
    // cell offsets in patch order, then every zone's slot
    std::vector<int64_t> off(out.patches.size() + 1, 0);
    for (size_t q = 0; q < out.patches.size(); ++q)
        off[q + 1] = off[q] + (int64_t)out.patches[q].nx * out.patches[q].ny;
    out.slot.assign(n, 0);
    for (int64_t k = 0; k < n; ++k) {
        const int q = zpatch[k];
        out.slot[k] = off[q] + (z->iy[k] - boxes[q].y0) * out.patches[q].nx + (z->ix[k] - boxes[q].x0);
    }
    return SG_OK;
}

template <typename T>
__global__ void k_zone_gather(const int64_t *__restrict__ slot, int64_t n, const T *__restrict__ s, const T *__restrict__ dx,
                              const T *__restrict__ dy, T *__restrict__ buf, int64_t ncells)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = slot[k];
        buf[o] = s[k];
        if (dx) {
            buf[ncells + o] = dx[k];
            buf[2 * ncells + o] = dy[k];
        }
    }
}

template <typename T>
__global__ void k_zone_scatter(const int64_t *__restrict__ slot, const int *__restrict__ code, int64_t n,
                               const T *__restrict__ fxp, const T *__restrict__ fyp, T *__restrict__ fx,
                               T *__restrict__ fy)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = slot[k];
        const bool leaf = code[o] == SG_CELL_LEAF;
        fx[k] = leaf ? fxp[o] : (T)0;
        fy[k] = leaf ? fyp[o] : (T)0;
    }
}

template <typename T>
__global__ void k_zone_scatter1(const int64_t *__restrict__ slot, const int *__restrict__ code, int64_t n,
                                const T *__restrict__ vp, T *__restrict__ v)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = slot[k];
        v[k] = code[o] == SG_CELL_LEAF ? vp[o] : (T)0;
    }
}

// The potential of a zone plan: zone-ordered inputs gathered into the patch
// layout, sg_potential, the leaf values scattered back (zeros at non-leaves).
template <typename T>
sg_status potential_zones_t(sg_plan *plan, const void *sigma, const void *dx, const void *dy, void *phi,
                            cudaStream_t st)
{
    const int64_t nc = plan->ncells;
    T *buf = (T *)plan->ws->zone_buf;
    const bool caller = plan->geom.slope_mode == SG_SLOPES_CALLER;
    int grid = (int)((plan->nzones + 255) / 256);
    if (grid > 8192) grid = 8192;
    k_zone_gather<T><<<grid, 256, 0, st>>>(plan->zone_slot, plan->nzones, (const T *)sigma,
                                           caller ? (const T *)dx : nullptr, caller ? (const T *)dy : nullptr, buf, nc);
    SG_CUDA_TRY(cudaGetLastError());
    SG_TRY(sg_potential(plan, buf, caller ? buf + nc : nullptr, caller ? buf + 2 * nc : nullptr, buf + 3 * nc, st));
    k_zone_scatter1<T><<<grid, 256, 0, st>>>(plan->zone_slot, plan->cell_code, plan->nzones, buf + 3 * nc, (T *)phi);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T>
sg_status force_zones_t(sg_plan *plan, const void *sigma, const void *dx, const void *dy, void *fx, void *fy,
                        cudaStream_t st)
{
    const int64_t nc = plan->ncells;
    T *buf = (T *)plan->ws->zone_buf;
    const bool caller = plan->geom.slope_mode == SG_SLOPES_CALLER;
    int grid = (int)((plan->nzones + 255) / 256);
    if (grid > 8192) grid = 8192;
    k_zone_gather<T><<<grid, 256, 0, st>>>(plan->zone_slot, plan->nzones, (const T *)sigma,
                                           caller ? (const T *)dx : nullptr, caller ? (const T *)dy : nullptr, buf, nc);
    SG_CUDA_TRY(cudaGetLastError());
    SG_TRY(sg_force_ws(plan, plan->ws, buf, buf + nc, buf + 2 * nc, buf + 3 * nc, buf + 4 * nc, st));
    k_zone_scatter<T><<<grid, 256, 0, st>>>(plan->zone_slot, plan->cell_code, plan->nzones, buf + 3 * nc,
                                            buf + 4 * nc, (T *)fx, (T *)fy);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

}  // namespace

extern "C" {

sg_status sg_plan_create_zones(const sg_zones *zones, double G, int slope_mode, int cross_mode, sg_precision prec,
                               size_t hbm_budget, sg_plan **out)
{
    if (!out || (prec != SG_FP64 && prec != SG_FP32)) return zfail("invalid precision or output pointer");
    if (slope_mode < SG_SLOPES_NONE || slope_mode > SG_SLOPES_CALLER) return zfail("unknown slope mode");
    std::unordered_map<uint64_t, int64_t> idx;
    int lmax = 0;
    SG_TRY(zones_index(zones, idx, lmax));
    idx.clear();
    layout lay;
    SG_TRY(zones_layout(zones, lmax, lay));
    std::vector<const uint8_t *> mp(lay.masks.size());
    for (size_t q = 0; q < lay.masks.size(); ++q) mp[q] = lay.masks[q].data();
    sg_geom g;
    memset(&g, 0, sizeof(g));
    g.npatches = (int)lay.patches.size();
    g.patches = lay.patches.data();
    g.G = G;
    g.slope_mode = slope_mode;
    g.z = 0.0;
    g.masks = mp.data();
    g.cross_mode = cross_mode;
    sg_plan *plan = nullptr;
    SG_TRY(sg_plan_build(&g, prec, hbm_budget, &plan));
    plan->nzones = zones->nzones;
    plan->launches += 2;  // gather and scatter
    const size_t es = prec == SG_FP64 ? 8 : 4;
    plan->ws_zone_bytes = 5 * plan->ncells * (int64_t)es;
    plan->scratch_bytes += plan->ws_zone_bytes;
    sg_status st = sg_plan_upload(plan, (void **)&plan->zone_slot, lay.slot.data(), lay.slot.size() * sizeof(int64_t));
    if (st == SG_OK && hbm_budget && (size_t)plan->device_bytes > hbm_budget) {
        sg_set_last_error_message("plan exceeds the device-memory budget");
        st = SG_EBUDGET;
    }
    if (st != SG_OK) {
        sg_plan_release(plan);
        return st;
    }
    *out = plan;
    return SG_OK;
}

// Checks shared by the zone entry points, and the plan's workspace with its
// zone buffer (allocated at the first call).
static sg_status zones_call_setup(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay,
                                  const void *out0, const void *out1)
{
    if (!plan || plan->nzones <= 0) return zfail("not a zone plan");
    if (!sigma || !out0) return zfail("null field pointer");
    const bool caller = plan->geom.slope_mode == SG_SLOPES_CALLER;
    if (caller && (!deltax || !deltay)) return zfail("caller slopes requested but deltax/deltay is NULL");
    const size_t es = plan->prec == SG_FP64 ? 8 : 4;
    const void *ptrs[5] = {sigma, out0, out1, caller ? deltax : nullptr, caller ? deltay : nullptr};
    for (const void *p : ptrs)
        if (p && (uintptr_t)p % es) return zfail("misaligned field pointer");
    int dev = -1;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != plan->device) return zfail("the plan's device is not current");
    if (!plan->ws) {
        sg_workspace *ws = new (std::nothrow) sg_workspace();
        if (!ws) return SG_ENOMEM;
        sg_status a = sg_workspace_alloc(plan, ws, 0, false);
        if (a != SG_OK) {
            delete ws;
            return a;
        }
        plan->ws = ws;
        plan->device_bytes += sg_workspace_bytes(plan);
    }
    if (!plan->ws->zone_buf) {
        cudaError_t e = cudaMalloc(&plan->ws->zone_buf, (size_t)plan->ws_zone_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            plan->ws->zone_buf = nullptr;
            sg_set_last_cuda_error(e, "cudaMalloc");
            return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
        }
        plan->device_bytes += plan->ws_zone_bytes;
    }
    return SG_OK;
}

sg_status sg_force_zones(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx,
                         void *fy, void *stream)
{
    if (!fx || !fy) return zfail("null field pointer");
    SG_TRY(zones_call_setup(plan, sigma, deltax, deltay, fx, fy));
    sg_timing_reset(plan->timing);
    plan->ws->timing = plan->timing;
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->prec == SG_FP64) return force_zones_t<double>(plan, sigma, deltax, deltay, fx, fy, st);
    return force_zones_t<float>(plan, sigma, deltax, deltay, fx, fy, st);
}

sg_status sg_potential_zones(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *phi,
                             void *stream)
{
    if (!phi) return zfail("null field pointer");
    SG_TRY(zones_call_setup(plan, sigma, deltax, deltay, phi, nullptr));
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->prec == SG_FP64) return potential_zones_t<double>(plan, sigma, deltax, deltay, phi, st);
    return potential_zones_t<float>(plan, sigma, deltax, deltay, phi, st);
}

sg_status sg_plan_zone_slots(const sg_plan *plan, int64_t *host_out, int64_t n)
{
    if (!plan || plan->nzones <= 0 || !host_out || n < plan->nzones) return zfail("not a zone plan, or n too small");
    SG_CUDA_TRY(cudaMemcpy(host_out, plan->zone_slot, (size_t)plan->nzones * sizeof(int64_t), cudaMemcpyDeviceToHost));
    return SG_OK;
}

sg_status sg_zones_from_records(int64_t n, int ncols, const double *rec, int nx0, int ny0, double x0, double y0,
                                double h0, int32_t *level, int32_t *ix, int32_t *iy)
{
    if (n < 1 || ncols < 6 || !rec || !level || !ix || !iy) return zfail("invalid record arguments");
    if (nx0 < 1 || ny0 < 1 || !(h0 > 0.0) || !isfinite(h0) || !isfinite(x0) || !isfinite(y0))
        return zfail("invalid level-0 grid");
    char msg[160];
    std::vector<uint8_t> named(n, 0);
    for (int64_t r = 0; r < n; ++r) {
        const double *c = rec + r * ncols;
        if (c[0] != (double)(r + 1)) {
            snprintf(msg, sizeof(msg), "record %lld: ID %g, expected %lld", (long long)(r + 1), c[0], (long long)(r + 1));
            return zfail(msg);
        }
        const double L = c[3];
        if (!(L >= 1.0 && L <= SG_MAX_LEVELS) || L != floor(L)) {
            snprintf(msg, sizeof(msg), "record %lld: level L = %g invalid", (long long)(r + 1), L);
            return zfail(msg);
        }
        const int l = (int)L - 1;
        const double h = h0 / (double)(1LL << l);
        const double fx = (c[1] - x0) / h - 0.5, fy = (c[2] - y0) / h - 0.5;
        const double rx = nearbyint(fx), ry = nearbyint(fy);
        if (!(fabs(fx - rx) <= 0.25 && fabs(fy - ry) <= 0.25) || rx < 0 || ry < 0 ||
            rx >= (double)((int64_t)nx0 << l) || ry >= (double)((int64_t)ny0 << l)) {
            snprintf(msg, sizeof(msg), "record %lld: centre (%g, %g) is not a level-%d zone centre", (long long)(r + 1),
                     c[1], c[2], (int)L);
            return zfail(msg);
        }
        level[r] = l;
        ix[r] = (int32_t)rx;
        iy[r] = (int32_t)ry;
    }
    for (int64_t r = 0; r < n; ++r) {
        const double *c = rec + r * ncols;
        const double P = c[4];
        if (level[r] == 0) {
            if (P != 0.0) {
                snprintf(msg, sizeof(msg), "record %lld: a level-1 zone names parent %g", (long long)(r + 1), P);
                return zfail(msg);
            }
            continue;
        }
        if (!(P >= 1.0 && P <= (double)n) || P != floor(P)) {
            snprintf(msg, sizeof(msg), "record %lld: parent %g invalid", (long long)(r + 1), P);
            return zfail(msg);
        }
        const int64_t p = (int64_t)P - 1;
        if (level[p] != level[r] - 1 || ix[p] != (ix[r] >> 1) || iy[p] != (iy[r] >> 1)) {
            snprintf(msg, sizeof(msg), "record %lld: parent %lld does not contain it", (long long)(r + 1),
                     (long long)(p + 1));
            return zfail(msg);
        }
        named[p] = 1;
    }
    for (int64_t r = 0; r < n; ++r) {
        const double EL = rec[r * ncols + 5];
        if ((EL != 0.0 && EL != 1.0) || (EL == 1.0) == (named[r] != 0)) {
            snprintf(msg, sizeof(msg), "record %lld: leaf flag %g contradicts the parent links", (long long)(r + 1), EL);
            return zfail(msg);
        }
    }
    sg_zones z = {nx0, ny0, x0, y0, h0, n, level, ix, iy};
    std::unordered_map<uint64_t, int64_t> idx;
    int lmax = 0;
    return zones_index(&z, idx, lmax);
}

sg_status sg_zones_links(const sg_zones *zones, int64_t *parent, uint8_t *leaf, int64_t *neighbours)
{
    std::unordered_map<uint64_t, int64_t> idx;
    int lmax = 0;
    SG_TRY(zones_index(zones, idx, lmax));
    const int64_t n = zones->nzones;
    if (leaf)
        for (int64_t k = 0; k < n; ++k) leaf[k] = 1;
    for (int64_t k = 0; k < n; ++k) {
        const int l = zones->level[k];
        const int64_t i = zones->ix[k], j = zones->iy[k];
        int64_t p = -1;
        if (l > 0) {
            p = idx.at(zkey(l - 1, i >> 1, j >> 1));
            if (leaf) leaf[p] = 0;
        }
        if (parent) parent[k] = p + 1;
        if (!neighbours) continue;
        // sides: left, down, right, up; the point just across the side's midpoint,
        // in units of half a level-l zone: (2i + 1 + 2 dx, 2j + 1 + 2 dy) - (dx, dy)
        const int dxs[4] = {-1, 0, 1, 0}, dys[4] = {0, -1, 0, 1};
        for (int s = 0; s < 4; ++s) {
            const int64_t qi = i + dxs[s], qj = j + dys[s];
            int64_t found = 0;
            if (qi >= 0 && qj >= 0 && qi < ((int64_t)zones->nx0 << l) && qj < ((int64_t)zones->ny0 << l)) {
                for (int m = l; m >= 0 && !found; --m) {
                    auto it = idx.find(zkey(m, qi >> (l - m), qj >> (l - m)));
                    if (it != idx.end()) found = it->second + 1;
                }
            }
            neighbours[4 * k + s] = found;
        }
    }
    return SG_OK;
}

}  // extern "C"
