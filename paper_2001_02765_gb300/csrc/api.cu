// Host side of the C ABI: geometry analysis, plan construction, entry points.
#include "common.cuh"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <unordered_map>
#include <vector>

// ------------------------------------------------------------------ errors --

static thread_local char g_last_error[256] = "";

void sg_set_last_cuda_error(cudaError_t e, const char *what)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

void sg_set_last_error_message(const char *msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

static void set_error(const char *msg) { sg_set_last_error_message(msg); }

// ------------------------------------------------------------------ timing --

struct sg_timing {
    std::vector<cudaEvent_t> pool;      // created on demand, reused
    std::vector<int> stage;             // stage of each recorded (begin, end) pair
    int used = 0;                       // events used by the last solve
    int open = -1;                      // index of the pending begin event
};

static cudaEvent_t timing_event(sg_timing *t)
{
    if (t->used == (int)t->pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        t->pool.push_back(e);
    }
    return t->pool[t->used++];
}

void sg_timing_reset(sg_timing *t)
{
    if (!t) return;
    t->used = 0;
    t->stage.clear();
    t->open = -1;
}

void sg_timing_begin(const sg_workspace *ws, int stage, cudaStream_t st)
{
    sg_timing *t = ws->timing;
    if (!t) return;
    cudaEvent_t e = timing_event(t);
    if (!e) return;
    cudaEventRecord(e, st);
    t->open = t->used - 1;
    t->stage.push_back(stage);
}

void sg_timing_end(const sg_workspace *ws, int stage, cudaStream_t st)
{
    sg_timing *t = ws->timing;
    if (!t || t->open < 0) return;
    cudaEvent_t e = timing_event(t);
    if (!e) return;
    cudaEventRecord(e, st);
    t->open = -1;
    (void)stage;
}

// --------------------------------------------------------- geometry analysis --

namespace {

struct geom_info {
    int n = 0;
    int lmax = 0;
    double h0 = 0, X0 = 0, Y0 = 0, lambda = 0;
    std::vector<int> parent, ox, oy, step;
    std::vector<std::vector<int>> code;       // per patch [ny][nx]: SG_CELL_ABSENT, SG_CELL_LEAF or child patch
    bool masked = false;                      // some patch has a mask
    std::vector<int64_t> nleaf, cell_off;
    int64_t ncells = 0, nleaves = 0, cross_pairs = 0;
};

bool near_int(double x, long long *out)
{
    const double r = nearbyint(x);
    if (fabs(x - r) > 1e-9 * (fabs(x) > 1.0 ? fabs(x) : 1.0)) return false;
    if (out) *out = (long long)r;
    return true;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

sg_status fail(const char *msg)
{
    set_error(msg);
    return SG_EINVAL;
}

sg_status analyse(const sg_geom *g, geom_info &gi)
{
    if (!g) return fail("geometry is NULL");
    if (g->npatches < 1 || !g->patches) return fail("geometry has no patches");
    if (!isfinite(g->G)) return fail("G is not finite");
    if (!isfinite(g->z)) return fail("z is not finite");
    if (g->slope_mode < SG_SLOPES_NONE || g->slope_mode > SG_SLOPES_CALLER) return fail("unknown slope mode");
    if (g->cross_mode < SG_CROSS_AUTO || g->cross_mode > SG_CROSS_LEVELS) return fail("unknown cross mode");
    const int n = g->npatches;
    const sg_patch *P = g->patches;
    gi.n = n;
    if (g->masks)
        for (int k = 0; k < n; ++k) gi.masked = gi.masked || g->masks[k] != nullptr;
    if (P[0].level != 0) return fail("the first patch must be on level 0");
    for (int k = 0; k < n; ++k) {
        if (P[k].nx < 1 || P[k].ny < 1 || P[k].nx > SG_MAX_PATCH_SIDE || P[k].ny > SG_MAX_PATCH_SIDE)
            return fail("patch size out of range [1, 2048]");
        if (!finite_pos(P[k].h) || !isfinite(P[k].x0) || !isfinite(P[k].y0)) return fail("patch origin or h invalid");
        if (P[k].level < 0 || P[k].level >= SG_MAX_LEVELS) return fail("patch level out of range");
        if (k > 0 && P[k].level < P[k - 1].level) return fail("patches are not sorted by level");
        if (P[k].level > gi.lmax) gi.lmax = P[k].level;
    }
    gi.h0 = P[0].h;
    gi.X0 = P[0].x0;
    gi.Y0 = P[0].y0;
    for (int k = 0; k < n; ++k) {
        const double want = gi.h0 / (double)(1 << P[k].level);
        if (fabs(P[k].h - want) > 1e-12 * want) return fail("cell width must halve per level");
        if (P[k].level == 0) {
            if (P[k].x0 < gi.X0) gi.X0 = P[k].x0;
            if (P[k].y0 < gi.Y0) gi.Y0 = P[k].y0;
        }
    }
    gi.lambda = gi.h0 / (double)(1LL << (gi.lmax + 1));
    gi.parent.assign(n, -1);
    gi.ox.assign(n, 0);
    gi.oy.assign(n, 0);
    gi.step.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        long long ix, iy;
        if (!near_int((P[k].x0 - gi.X0) / gi.lambda, &ix) || !near_int((P[k].y0 - gi.Y0) / gi.lambda, &iy))
            return fail("patch origin is off the lattice");
        const long long st = 1LL << (gi.lmax - P[k].level + 1);
        if (ix + (long long)P[k].nx * st > (1LL << 23) || iy + (long long)P[k].ny * st > (1LL << 23))
            return fail("hierarchy spans more than 2^23 finest half-cells");
        gi.ox[k] = (int)ix;
        gi.oy[k] = (int)iy;
        gi.step[k] = (int)st;
    }
    // alignment, nesting and overlap, on the lattice
    for (int k = 0; k < n; ++k) {
        const int L = P[k].level;
        const long long x0 = gi.ox[k], y0 = gi.oy[k];
        const long long x1 = x0 + (long long)P[k].nx * gi.step[k], y1 = y0 + (long long)P[k].ny * gi.step[k];
        if (L == 0) {
            if (x0 % gi.step[k] || y0 % gi.step[k]) return fail("level-0 patches are not on one lattice");
        } else {
            if (P[k].nx % 2 || P[k].ny % 2) return fail("refined patches need even cell counts");
            int par = -1;
            for (int q = 0; q < n; ++q) {
                if (P[q].level != L - 1) continue;
                const long long px0 = gi.ox[q], py0 = gi.oy[q];
                const long long px1 = px0 + (long long)P[q].nx * gi.step[q], py1 = py0 + (long long)P[q].ny * gi.step[q];
                if (x0 >= px0 && x1 <= px1 && y0 >= py0 && y1 <= py1) {
                    par = q;
                    break;
                }
            }
            if (par < 0) return fail("a refined patch does not lie inside one patch of the level below");
            if ((x0 - gi.ox[par]) % gi.step[par] || (y0 - gi.oy[par]) % gi.step[par])
                return fail("a refined patch does not start on its parent's cell lattice");
            gi.parent[k] = par;
        }
        for (int q = 0; q < k; ++q) {
            if (P[q].level != L) continue;
            const long long qx0 = gi.ox[q], qy0 = gi.oy[q];
            const long long qx1 = qx0 + (long long)P[q].nx * gi.step[q], qy1 = qy0 + (long long)P[q].ny * gi.step[q];
            if (x0 < qx1 && qx0 < x1 && y0 < qy1 && qy0 < y1) return fail("patches of one level overlap");
        }
    }
    // cell codes: absent, leaf, or covered by a child patch
    gi.code.assign(n, {});
    gi.nleaf.assign(n, 0);
    gi.cell_off.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        const uint8_t *m = g->masks ? g->masks[k] : nullptr;
        const size_t nc = (size_t)P[k].nx * P[k].ny;
        gi.code[k].assign(nc, SG_CELL_LEAF);
        if (m)
            for (size_t c = 0; c < nc; ++c)
                if (!m[c]) gi.code[k][c] = SG_CELL_ABSENT;
    }
    char msg[160];
    for (int k = 0; k < n; ++k) {
        const int par = gi.parent[k];
        if (par < 0) continue;
        const int pi0 = (gi.ox[k] - gi.ox[par]) / gi.step[par], pj0 = (gi.oy[k] - gi.oy[par]) / gi.step[par];
        const int nx = P[k].nx, pnx = P[par].nx;
        for (int bj = 0; bj < P[k].ny / 2; ++bj) {
            for (int bi = 0; bi < nx / 2; ++bi) {
                int present = 0;
                for (int q = 0; q < 4; ++q)
                    present += gi.code[k][(size_t)(2 * bj + (q >> 1)) * nx + 2 * bi + (q & 1)] != SG_CELL_ABSENT;
                if (present == 0) continue;
                if (present != 4) {
                    snprintf(msg, sizeof(msg), "patch %d: cells (%d..%d, %d..%d) are not a whole 2x2 block", k,
                             2 * bi, 2 * bi + 1, 2 * bj, 2 * bj + 1);
                    return fail(msg);
                }
                int &pc = gi.code[par][(size_t)(pj0 + bj) * pnx + pi0 + bi];
                if (pc == SG_CELL_ABSENT) {
                    snprintf(msg, sizeof(msg), "patch %d: cells over an absent parent cell (%d, %d) of patch %d", k,
                             pi0 + bi, pj0 + bj, par);
                    return fail(msg);
                }
                pc = k;
            }
        }
    }
    gi.ncells = 0;
    gi.nleaves = 0;
    for (int k = 0; k < n; ++k) {
        gi.cell_off[k] = gi.ncells;
        gi.ncells += (int64_t)P[k].nx * P[k].ny;
        int64_t leaves = 0;
        for (int c : gi.code[k]) leaves += c == SG_CELL_LEAF;
        gi.nleaf[k] = leaves;
        gi.nleaves += leaves;
    }
    if (gi.nleaves == 0) return fail("the geometry has no leaf cell");
    gi.cross_pairs = 0;
    for (int k = 0; k < n; ++k) gi.cross_pairs += gi.nleaf[k] * (gi.nleaves - gi.nleaf[k]);
    return SG_OK;
}

size_t elem_size(sg_precision prec) { return prec == SG_FP64 ? 8 : 4; }

// Source tiles of every patch (the composite sources cover whole patches):
// 16 x 16 corners for the FP64 corner-form sum, 16 x 16 cells for the FP32
// near/far sum. With masks, tiles that touch no existing cell carry zero
// weights and are left out.
void build_tiles(const sg_geom *g, const geom_info &gi, bool cell_tiles, std::vector<sg_tile_desc> &tiles,
                 std::vector<int> &first, std::vector<int> &count)
{
    first.assign(gi.n, 0);
    count.assign(gi.n, 0);
    std::vector<int64_t> sat;  // summed-area table of existing cells, (ny + 1) x (nx + 1)
    const int extra = cell_tiles ? 0 : 1;  // a patch has nx + 1 corners per row, nx cells
    for (int k = 0; k < gi.n; ++k) {
        const sg_patch &p = g->patches[k];
        const bool masked = g->masks && g->masks[k];
        if (masked) {
            sat.assign((size_t)(p.nx + 1) * (p.ny + 1), 0);
            for (int j = 0; j < p.ny; ++j)
                for (int i = 0; i < p.nx; ++i)
                    sat[(size_t)(j + 1) * (p.nx + 1) + i + 1] =
                        (gi.code[k][(size_t)j * p.nx + i] != SG_CELL_ABSENT) + sat[(size_t)j * (p.nx + 1) + i + 1] +
                        sat[(size_t)(j + 1) * (p.nx + 1) + i] - sat[(size_t)j * (p.nx + 1) + i];
        }
        first[k] = (int)tiles.size();
        const int ntx = (p.nx + extra + SG_TILE_X - 1) / SG_TILE_X, nty = (p.ny + extra + SG_TILE_Y - 1) / SG_TILE_Y;
        for (int b = 0; b < nty; ++b) {
            for (int a = 0; a < ntx; ++a) {
                const int ci0 = a * SG_TILE_X, cj0 = b * SG_TILE_Y;
                if (masked) {
                    // cells of the tile (cell tiles: i in [ci0, ci0 + TILE_X - 1]) or around
                    // its corners (corner tiles: i in [ci0 - 1, ci0 + TILE_X - 1]); same in j
                    const int i0 = ci0 - extra > 0 ? ci0 - extra : 0, j0 = cj0 - extra > 0 ? cj0 - extra : 0;
                    const int i1 = ci0 + SG_TILE_X < p.nx ? ci0 + SG_TILE_X : p.nx;
                    const int j1 = cj0 + SG_TILE_Y < p.ny ? cj0 + SG_TILE_Y : p.ny;
                    const int64_t w = p.nx + 1;
                    const int64_t cnt = sat[(size_t)j1 * w + i1] - sat[(size_t)j0 * w + i1] - sat[(size_t)j1 * w + i0] +
                                        sat[(size_t)j0 * w + i0];
                    if (cnt == 0) continue;
                }
                sg_tile_desc t;
                memset(&t, 0, sizeof(t));
                t.patch = k;
                t.ci0 = ci0;
                t.cj0 = cj0;
                t.step = gi.step[k];
                t.ox = gi.ox[k] + ci0 * gi.step[k];
                t.oy = gi.oy[k] + cj0 * gi.step[k];
                tiles.push_back(t);
            }
        }
        count[k] = (int)tiles.size() - first[k];
    }
}

// Leaf targets of the direct sum and their blocks: per patch, the leaves of
// every 16 x 16-cell square, row-major inside the square (a block is compact,
// so the distance from a source tile to all of its targets is bounded from below).
void build_targets(const sg_geom *g, const geom_info &gi, std::vector<int4> &tg, std::vector<sg_target_block> &blocks)
{
    tg.clear();
    blocks.clear();
    tg.reserve((size_t)gi.nleaves);
    for (int k = 0; k < gi.n; ++k) {
        const sg_patch &p = g->patches[k];
        for (int bj = 0; bj < p.ny; bj += 16) {
            for (int bi = 0; bi < p.nx; bi += 16) {
                sg_target_block b;
                memset(&b, 0, sizeof(b));
                b.patch = k;
                b.first = (int)tg.size();
                b.tx0 = b.ty0 = INT32_MAX;
                b.tx1 = b.ty1 = INT32_MIN;
                for (int j = bj; j < std::min(bj + 16, p.ny); ++j) {
                    for (int i = bi; i < std::min(bi + 16, p.nx); ++i) {
                        if (gi.code[k][(size_t)j * p.nx + i] != SG_CELL_LEAF) continue;
                        int4 t;
                        t.x = gi.ox[k] + (2 * i + 1) * (gi.step[k] / 2);
                        t.y = gi.oy[k] + (2 * j + 1) * (gi.step[k] / 2);
                        t.z = (int)(gi.cell_off[k] + (int64_t)j * p.nx + i);
                        t.w = k;
                        tg.push_back(t);
                        b.tx0 = std::min(b.tx0, t.x);
                        b.tx1 = std::max(b.tx1, t.x);
                        b.ty0 = std::min(b.ty0, t.y);
                        b.ty1 = std::max(b.ty1, t.y);
                        b.count++;
                    }
                }
                if (b.count > 0) blocks.push_back(b);
            }
        }
    }
}

// Links of the neighbour-leaf slope rule (amr.cu): per cell and side (left,
// down, right, up) what lies across the side's midpoint (see sg_plan), found
// through per-level maps of the cells' level-grid coordinates; and the lattice
// coordinates of every cell centre.
int64_t floor_div64(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

void build_slope_links(const sg_geom *g, const geom_info &gi, std::vector<int2> &nb, std::vector<int2> &pos)
{
    const int nlev = gi.lmax + 1;
    std::vector<std::unordered_map<uint64_t, int64_t>> map(nlev);
    auto key = [](int64_t x, int64_t y) { return ((uint64_t)(uint32_t)x << 32) | (uint32_t)y; };
    for (int k = 0; k < gi.n; ++k) {
        const sg_patch &p = g->patches[k];
        const int64_t gx0 = gi.ox[k] / gi.step[k], gy0 = gi.oy[k] / gi.step[k];
        auto &m = map[p.level];
        m.reserve(m.size() + (size_t)p.nx * p.ny);
        for (int j = 0; j < p.ny; ++j)
            for (int i = 0; i < p.nx; ++i)
                if (gi.code[k][(size_t)j * p.nx + i] != SG_CELL_ABSENT)
                    m[key(gx0 + i, gy0 + j)] = gi.cell_off[k] + (int64_t)j * p.nx + i;
    }
    auto find = [&](int l, int64_t x, int64_t y) -> int64_t {
        if (x < 0 || y < 0) return -1;
        auto it = map[l].find(key(x, y));
        return it == map[l].end() ? -1 : it->second;
    };
    std::vector<int> code_of((size_t)gi.ncells);
    for (int k = 0; k < gi.n; ++k)
        std::copy(gi.code[k].begin(), gi.code[k].end(), code_of.begin() + gi.cell_off[k]);
    nb.assign((size_t)gi.ncells * 4, make_int2(-1, -3));
    pos.assign((size_t)gi.ncells, make_int2(0, 0));
    const int sdx[4] = {-1, 0, 1, 0}, sdy[4] = {0, -1, 0, 1};
    for (int k = 0; k < gi.n; ++k) {
        const sg_patch &p = g->patches[k];
        const int l = p.level;
        const int64_t gx0 = gi.ox[k] / gi.step[k], gy0 = gi.oy[k] / gi.step[k];
        for (int j = 0; j < p.ny; ++j) {
            for (int i = 0; i < p.nx; ++i) {
                const int64_t c = gi.cell_off[k] + (int64_t)j * p.nx + i;
                pos[c] = make_int2(gi.ox[k] + (2 * i + 1) * (gi.step[k] / 2), gi.oy[k] + (2 * j + 1) * (gi.step[k] / 2));
                if (code_of[c] != SG_CELL_LEAF) continue;
                const int64_t gx = gx0 + i, gy = gy0 + j;
                for (int s = 0; s < 4; ++s) {
                    const int dx = sdx[s], dy = sdy[s];
                    int2 d = make_int2(-1, -3);
                    const int64_t n = find(l, gx + dx, gy + dy);
                    if (n >= 0 && code_of[n] == SG_CELL_LEAF) {
                        d = make_int2((int)n, -1);
                    } else if (n >= 0 && code_of[n] >= 0 && l + 1 < nlev) {
                        // the two children of the refined neighbour that touch the side
                        const int64_t nx2 = 2 * (gx + dx), ny2 = 2 * (gy + dy);
                        int64_t a, b;
                        if (dx != 0) {
                            const int64_t cx = nx2 + (dx > 0 ? 0 : 1);
                            a = find(l + 1, cx, ny2);
                            b = find(l + 1, cx, ny2 + 1);
                        } else {
                            const int64_t cy = ny2 + (dy > 0 ? 0 : 1);
                            a = find(l + 1, nx2, cy);
                            b = find(l + 1, nx2 + 1, cy);
                        }
                        if (a >= 0 && b >= 0) d = make_int2((int)a, (int)b);
                    } else {
                        // the coarser leaf containing the point just across the side's midpoint
                        // (quarters of a level-l cell: 4 g + 2 + 3 d)
                        const int64_t qx = 4 * gx + 2 + 3 * dx, qy = 4 * gy + 2 + 3 * dy;
                        for (int m = l - 1; m >= 0; --m) {
                            const int64_t w = 4LL << (l - m);
                            const int64_t c2 = find(m, floor_div64(qx, w), floor_div64(qy, w));
                            if (c2 >= 0 && code_of[c2] == SG_CELL_LEAF) {
                                d = make_int2((int)c2, -2);
                                break;
                            }
                        }
                    }
                    nb[(size_t)c * 4 + s] = d;
                }
            }
        }
    }
}

// Level-convolution parameters (lvconv.cu) of a composite hierarchy, or false
// when it does not qualify: z == 0, not central slopes, at least two levels,
// and a finest-lattice extent whose padded length fits the transforms.
// bytes: device memory the level convolutions add (maps, kernel spectra, scratch).
bool lv_params(const sg_geom *g, const geom_info &gi, sg_precision prec, sg_lv_setup_args &a,
               std::vector<std::vector<int>> &maps, int64_t &bytes)
{
    if (gi.lmax < 1 || g->z != 0.0) return false;
    const sg_patch *P = g->patches;
    int64_t wx = 0, wy = 0;  // level-0 extent in finest cells (lattice units are half finest cells)
    for (int k = 0; k < gi.n; ++k) {
        if (P[k].level != 0) continue;
        wx = std::max<int64_t>(wx, ((int64_t)gi.ox[k] + (int64_t)P[k].nx * gi.step[k]) / 2);
        wy = std::max<int64_t>(wy, ((int64_t)gi.oy[k] + (int64_t)P[k].ny * gi.step[k]) / 2);
    }
    auto pad = [](int64_t w) {
        int64_t p = SG_MIN_PAD;
        while (p < 2 * w - 1) p <<= 1;
        return p;
    };
    const int64_t px = pad(wx), py = pad(wy);
    const int64_t maxp = prec == SG_FP64 ? SG_MAX_PAD : SG_LV_MAX_PAD;
    if (px > maxp || py > maxp) return false;
    memset(&a, 0, sizeof(a));
    a.nlev = gi.lmax + 1;
    a.px = (int)px;
    a.py = (int)py;
    a.hf = gi.h0 / (double)(1 << gi.lmax);
    maps.assign(a.nlev, {});
    const int64_t qx = px / 2 + 1;
    const int64_t cs = prec == SG_FP64 ? 16 : 8;
    int64_t work = 0, mapbytes = 0;
    for (int m = 0; m < a.nlev; ++m) {
        const int sx = gi.lmax - m;
        int64_t gx0 = INT64_MAX, gy0 = INT64_MAX, gx1 = INT64_MIN, gy1 = INT64_MIN;
        for (int k = 0; k < gi.n; ++k) {
            if (P[k].level != m) continue;
            const int64_t gx = gi.ox[k] / gi.step[k], gy = gi.oy[k] / gi.step[k];
            gx0 = std::min(gx0, gx);
            gy0 = std::min(gy0, gy);
            gx1 = std::max(gx1, gx + P[k].nx);
            gy1 = std::max(gy1, gy + P[k].ny);
        }
        if (gx0 == INT64_MAX) return false;
        a.s[m] = sx;
        a.nx[m] = (int)(gx1 - gx0);
        a.ny[m] = (int)(gy1 - gy0);
        const int64_t half = sx >= 1 ? (1LL << (sx - 1)) : 0;
        a.i0[m] = (int)((gx0 << sx) + half);
        a.j0[m] = (int)((gy0 << sx) + half);
        std::vector<int> &mp = maps[m];
        mp.assign((size_t)a.nx[m] * a.ny[m], -1);
        for (int k = 0; k < gi.n; ++k) {
            if (P[k].level != m) continue;
            const int64_t bx = gi.ox[k] / gi.step[k] - gx0, by = gi.oy[k] / gi.step[k] - gy0;
            for (int j = 0; j < P[k].ny; ++j)
                for (int i = 0; i < P[k].nx; ++i)
                    if (gi.code[k][(size_t)j * P[k].nx + i] != SG_CELL_ABSENT)
                        mp[(size_t)(by + j) * a.nx[m] + bx + i] = (int)(gi.cell_off[k] + (int64_t)j * P[k].nx + i);
        }
        a.map[m] = mp.data();
        mapbytes += (int64_t)mp.size() * 4;
        // compact row transforms and source spectra, full-width inverse columns
        const int64_t qxc = (px >> sg_lv_cexp(sx, (int)px)) / 2 + 1, pcy = py >> sg_lv_cexp(sx, (int)py);
        work += (3 * qxc * a.ny[m] + 3 * qxc * pcy + 2 * qx * a.ny[m]) * cs;
    }
    int nkeys = 0;
    int ks[3 * SG_MAX_LEVELS], kd[3 * SG_MAX_LEVELS];
    for (int m = 0; m < a.nlev; ++m) {
        for (int l = 0; l < a.nlev; ++l) {
            const int d2 = (a.s[m] >= 1) - (a.s[l] >= 1);
            int k = 0;
            while (k < nkeys && !(ks[k] == a.s[m] && kd[k] == d2)) ++k;
            if (k == nkeys) {
                ks[k] = a.s[m];
                kd[k] = d2;
                ++nkeys;
            }
        }
    }
    bytes = mapbytes + (int64_t)nkeys * 6 * qx * sg_spec_stride((int)py) * (cs / 2) + 2 * (px + py + 2) * cs + work;
    return true;
}

// Source-tile ranges per target block. FP64 plans: enough (block, range) CTAs
// for two per SM. FP32 plans: work items of the persistent far-field launch,
// about 32 per SM so that dynamic scheduling evens out their unequal costs.
int choose_nsplit(int nblocks, int ntiles, int nsm, sg_precision prec)
{
    if (nblocks <= 0) return 1;
    const int want = prec == SG_FP64 ? 2 * nsm : 32 * nsm;
    int s = (want + nblocks - 1) / nblocks;
    const int cap = ntiles / 4 > 1 ? ntiles / 4 : 1;
    if (s > cap) s = cap;
    if (s < 1) s = 1;
    return s;
}

struct sizes {
    int64_t spectra = 0, twiddles = 0, work = 0, direct = 0, geometry = 0;
    int max_pad = SG_MIN_PAD;
    int64_t total() const { return spectra + twiddles + work + direct + geometry; }
};

sizes plan_sizes(const sg_geom *g, const geom_info &gi, sg_precision prec, int ntiles, int nblocks, int nsplit,
                 int64_t lv_bytes = -1)
{
    sizes s;
    const size_t es = elem_size(prec);
    int64_t work = 0;
    for (int k = 0; k < gi.n; ++k) {
        const int px = sg_pad_length(g->patches[k].nx), py = sg_pad_length(g->patches[k].ny);
        if (px > s.max_pad) s.max_pad = px;
        if (py > s.max_pad) s.max_pad = py;
        if (lv_bytes < 0) s.spectra += (g->z != 0.0 ? 9LL : 6LL) * (px / 2 + 1) * sg_spec_stride(py) * (int64_t)es;
        const int64_t w = 5LL * (px / 2 + 1) * g->patches[k].ny * (int64_t)(2 * es);
        if (w > work) work = w;
    }
    s.work = lv_bytes < 0 ? work : lv_bytes;
    for (int L = SG_MIN_PAD; L <= s.max_pad; L <<= 1) s.twiddles += (int64_t)L * (16 + 8);
    if (gi.n > 1 || gi.masked) s.direct = 3 * gi.ncells * (int64_t)es + gi.ncells * (int64_t)sizeof(int);
    if ((gi.n > 1 || gi.masked) && g->slope_mode == SG_SLOPES_CENTRAL) s.direct += 40 * gi.ncells;  // links, centres
    if (gi.n > 1 && lv_bytes < 0) {
        // off the plane: three partial components per split (and the near field in FP32 plans)
        const bool off = g->z != 0.0;
        const int64_t slices = off ? ((int64_t)nsplit + (prec == SG_FP32 ? 1 : 0)) * 3 / 2 + 1
                                   : (prec == SG_FP64 ? (nsplit > 1 ? nsplit : 0) : nsplit + 1);
        s.direct += (int64_t)ntiles * ((int64_t)sizeof(sg_tile_desc) + SG_TILE_N * 4 * (int64_t)es) +
                    gi.nleaves * (int64_t)sizeof(int4) + (int64_t)nblocks * (int64_t)sizeof(sg_target_block) +
                    slices * gi.nleaves * 16;
    }
    s.geometry = (int64_t)gi.n * (int64_t)sizeof(sg_patch_dev) + 16 * (int64_t)gi.n;
    return s;
}

int count_blocks(const sg_geom *g, const geom_info &gi)
{
    if (gi.n <= 1) return 0;
    int64_t b = 0;
    for (int k = 0; k < gi.n; ++k) {
        const sg_patch &p = g->patches[k];
        for (int bj = 0; bj < p.ny; bj += 16)
            for (int bi = 0; bi < p.nx; bi += 16) {
                bool any = false;
                for (int j = bj; j < std::min(bj + 16, p.ny) && !any; ++j)
                    for (int i = bi; i < std::min(bi + 16, p.nx) && !any; ++i)
                        any = gi.code[k][(size_t)j * p.nx + i] == SG_CELL_LEAF;
                b += any;
            }
    }
    return (int)b;
}

template <typename X>
sg_status dev_alloc(sg_plan *plan, X **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) return SG_OK;
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sg_set_last_cuda_error(e, "cudaMalloc");
        return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
    }
    plan->device_bytes += (int64_t)bytes;
    return SG_OK;
}

void plan_free(sg_plan *plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    if (plan->timing) {
        for (cudaEvent_t e : plan->timing->pool) cudaEventDestroy(e);
        delete plan->timing;
    }
    if (plan->pp) {
        for (int k = 0; k < plan->npatches; ++k) {
            cudaFree(plan->pp[k].spectra);
            cudaFree(plan->pp[k].phase);
            cudaFree(plan->pp[k].pspectra);
        }
        cudaFree(plan->pot_fwd);
    }
    sg_lv_free(plan);
    cudaFree(plan->twiddles);
    cudaFree(plan->cell_code);
    cudaFree(plan->comp_item_off);
    cudaFree(plan->comp_order);
    cudaFree(plan->comp_cells);
    delete[] plan->comp_cells_host;
    cudaFree(plan->zone_slot);
    cudaFree(plan->slope_nb);
    cudaFree(plan->cell_pos);
    if (plan->ws) {
        sg_workspace_free(plan->ws, 0, false);
        delete plan->ws;
    }
    cudaFree(plan->tiles);
    cudaFree(plan->targets);
    cudaFree(plan->blocks);
    cudaFree(plan->patch_dev);
    cudaFree(plan->stage_in);
    cudaFree(plan->stage_out);
    cudaFreeHost(plan->err_host);
    delete[] plan->pp;
    delete[] plan->patches_host;
    delete plan;
}

sg_status plan_build(const sg_geom *g, sg_precision prec, size_t budget, sg_plan **out)
{
    geom_info gi;
    SG_TRY(analyse(g, gi));
    // level convolutions, or per-patch convolutions plus the cross-patch direct sum
    sg_lv_setup_args lva;
    std::vector<std::vector<int>> lvmaps;
    int64_t lv_bytes = -1;
    bool use_lv = false;
    if ((gi.n > 1 || gi.masked) && g->cross_mode != SG_CROSS_DIRECT && gi.lmax >= 1) {
        use_lv = lv_params(g, gi, prec, lva, lvmaps, lv_bytes);
        if (!use_lv) lv_bytes = -1;
        if (!use_lv && g->cross_mode == SG_CROSS_LEVELS)
            return fail("level convolutions need z == 0 and a finest-lattice extent of at most "
                        "4096 cells per axis (2048 for FP64 plans)");
    }
    std::vector<sg_tile_desc> tiles;
    std::vector<int> tfirst, tcount;
    // corner tiles for the corner form (FP64 plans), cell tiles for the FP32 far field
    const bool corner_form = prec == SG_FP64;
    if (gi.n > 1 && !use_lv) build_tiles(g, gi, !corner_form, tiles, tfirst, tcount);
    int dev = 0, nsm = 152;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    SG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int nblocks = use_lv ? 0 : count_blocks(g, gi);
    const int nsplit = choose_nsplit(nblocks, (int)tiles.size(), nsm, corner_form ? SG_FP64 : prec);
    const sizes sz = plan_sizes(g, gi, prec, (int)tiles.size(), nblocks, nsplit, lv_bytes);
    if (budget && (size_t)sz.total() > budget) {
        set_error("plan exceeds the device-memory budget");
        return SG_EBUDGET;
    }

    sg_plan *plan = new (std::nothrow) sg_plan();
    if (!plan) return SG_ENOMEM;
    memset(plan, 0, sizeof(*plan));
    plan->device = dev;
    plan->prec = prec;
    plan->geom = *g;
    plan->npatches = gi.n;
    plan->patches_host = new (std::nothrow) sg_patch[gi.n];
    plan->pp = new (std::nothrow) sg_patch_plan[gi.n];
    if (!plan->patches_host || !plan->pp) {
        plan_free(plan);
        return SG_ENOMEM;
    }
    memcpy(plan->patches_host, g->patches, sizeof(sg_patch) * gi.n);
    plan->geom.patches = plan->patches_host;
    plan->ncells = gi.ncells;
    plan->nleaves = gi.nleaves;
    plan->cross_pairs = gi.cross_pairs;
    plan->max_pad = use_lv ? std::max(sz.max_pad, std::max(lva.px, lva.py)) : sz.max_pad;
    plan->lattice_unit = gi.lambda;
    plan->lattice_x0 = gi.X0;
    plan->lattice_y0 = gi.Y0;
    plan->nsplit = nsplit;
    plan->wait_tries = SG_MBAR_MAX_TRIES;

    plan->geom.masks = nullptr;  // the cell codes below carry them
    plan->composite = gi.n > 1 || gi.masked;
    plan->cross_mode = use_lv ? SG_CROSS_LEVELS : (gi.n > 1 ? SG_CROSS_DIRECT : 0);
    if (use_lv) plan->cross_pairs = 0;

    sg_status st = SG_OK;
    const size_t es = elem_size(prec);
    std::vector<sg_patch_dev> pdev(gi.n);
    for (int k = 0; k < gi.n && st == SG_OK; ++k) {
        sg_patch_plan &pp = plan->pp[k];
        memset(&pp, 0, sizeof(pp));
        pp.geom = g->patches[k];
        sg_patch_dev &d = pp.d;
        d.nx = g->patches[k].nx;
        d.ny = g->patches[k].ny;
        d.px = sg_pad_length(d.nx);
        d.py = sg_pad_length(d.ny);
        d.cell_off = gi.cell_off[k];
        d.h = g->patches[k].h;
        d.ox = gi.ox[k];
        d.oy = gi.oy[k];
        d.step = gi.step[k];
        d.parent = gi.parent[k];
        d.pi0 = d.parent >= 0 ? (gi.ox[k] - gi.ox[d.parent]) / gi.step[d.parent] : 0;
        d.pj0 = d.parent >= 0 ? (gi.oy[k] - gi.oy[d.parent]) / gi.step[d.parent] : 0;
        d.ncells_plane = gi.ncells;
        if (!tfirst.empty()) {
            pp.tile_first = d.tile_first = tfirst[k];
            pp.tile_count = d.tile_count = tcount[k];
        }
        pdev[k] = d;
        const int nplanes = g->z != 0.0 ? 9 : 6;
        if (!use_lv) st = dev_alloc(plan, &pp.spectra, nplanes * (size_t)(d.px / 2 + 1) * sg_spec_stride(d.py) * es);
        if (st == SG_OK && g->slope_mode == SG_SLOPES_CENTRAL && g->z == 0.0 && !(gi.n > 1 || gi.masked))
            st = dev_alloc(plan, &pp.phase, (4 * (size_t)(d.px / 2 + 1) + 4 * (size_t)d.py) * es);
    }
    if (plan->composite) {
        plan->ws_sfield_bytes = 6 * gi.ncells * (int64_t)es;  // composite sources S, filled values F
        std::vector<int> codes;
        codes.reserve((size_t)gi.ncells);
        for (int k = 0; k < gi.n; ++k) codes.insert(codes.end(), gi.code[k].begin(), gi.code[k].end());
        if (st == SG_OK) st = sg_plan_upload(plan, (void **)&plan->cell_code, codes.data(), codes.size() * sizeof(int));
        // patches sorted by level; prefix sums of their cells and of the final launch's items
        std::vector<int> order;
        for (int l = 0; l <= gi.lmax; ++l) {
            plan->comp_lev_first[l] = (int)order.size();
            for (int k = 0; k < gi.n; ++k)
                if (g->patches[k].level == l) order.push_back(k);
        }
        plan->comp_lev_first[gi.lmax + 1] = (int)order.size();
        std::vector<int64_t> cells((size_t)gi.n + 1, 0), items((size_t)gi.n + 1, 0);
        for (int t = 0; t < gi.n; ++t) {
            const sg_patch &q = g->patches[order[t]];
            cells[t + 1] = cells[t] + (int64_t)q.nx * q.ny;
            items[t + 1] = items[t] + (q.level == 0 ? (int64_t)q.nx * q.ny : (int64_t)(q.nx / 2) * (q.ny / 2));
        }
        plan->comp_items = items[gi.n];
        plan->comp_depth = gi.lmax + 1;
        plan->comp_cells_host = new (std::nothrow) int64_t[gi.n + 1];
        if (!plan->comp_cells_host) st = SG_ENOMEM;
        else std::copy(cells.begin(), cells.end(), plan->comp_cells_host);
        if (st == SG_OK) st = sg_plan_upload(plan, (void **)&plan->comp_order, order.data(), order.size() * sizeof(int));
        if (st == SG_OK) st = sg_plan_upload(plan, (void **)&plan->comp_cells, cells.data(), cells.size() * sizeof(int64_t));
        if (st == SG_OK)
            st = sg_plan_upload(plan, (void **)&plan->comp_item_off, items.data(), items.size() * sizeof(int64_t));
        if (st == SG_OK && g->slope_mode == SG_SLOPES_CENTRAL) {
            // neighbour-leaf slopes: links across every side, cell centres, level ranges,
            // and two more workspace planes for the slopes
            std::vector<int2> nb, pos;
            build_slope_links(g, gi, nb, pos);
            plan->amr_central = true;
            plan->ws_sfield_bytes = 8 * gi.ncells * (int64_t)es;
            st = sg_plan_upload(plan, (void **)&plan->slope_nb, nb.data(), nb.size() * sizeof(int2));
            if (st == SG_OK) st = sg_plan_upload(plan, (void **)&plan->cell_pos, pos.data(), pos.size() * sizeof(int2));
            for (int l = 0; l <= SG_MAX_LEVELS; ++l) plan->lev_cells[l] = gi.ncells;
            for (int k = gi.n - 1; k >= 0; --k) {
                plan->lev_cells[g->patches[k].level] = gi.cell_off[k];
                plan->lev_step[g->patches[k].level] = gi.step[k];
            }
            for (int l = SG_MAX_LEVELS - 1; l >= 0; --l)
                if (plan->lev_cells[l] > plan->lev_cells[l + 1]) plan->lev_cells[l] = plan->lev_cells[l + 1];
        }
    }
    if (st == SG_OK) st = dev_alloc(plan, &plan->patch_dev, gi.n * sizeof(sg_patch_dev));
    if (st == SG_OK)
        st = cudaMemcpy(plan->patch_dev, pdev.data(), gi.n * sizeof(sg_patch_dev), cudaMemcpyHostToDevice) == cudaSuccess
                 ? SG_OK : SG_ECUDA;
    // transform scratch, sized for the largest patch
    int64_t wf = 0, wi = 0;
    for (int k = 0; k < gi.n; ++k) {
        const int64_t q = (int64_t)(pdev[k].px / 2 + 1) * pdev[k].ny * (int64_t)(2 * es);
        // central slopes of a single unmasked patch (in the plane) transform sigma only, plus the
        // two edge columns (2 x py complex); hierarchies transform three composite fields
        const bool central = g->slope_mode == SG_SLOPES_CENTRAL && g->z == 0.0 && !(gi.n > 1 || gi.masked);
        const int64_t f = central ? q + (2LL * pdev[k].py + 1) * (int64_t)(2 * es) : 3 * q;  // edge pairs, even start
        const int nout = g->z != 0.0 ? 3 : 2;
        if (f > wf) wf = f;
        if (nout * q > wi) wi = nout * q;
    }
    plan->ws_fwd_bytes = wf;
    plan->ws_inv_bytes = wi;
    // cross-patch direct sum
    if (st == SG_OK && gi.n > 1 && !tiles.empty()) {
        plan->ntiles = (int)tiles.size();
        st = dev_alloc(plan, &plan->tiles, tiles.size() * sizeof(sg_tile_desc));
        if (st == SG_OK)
            st = cudaMemcpy(plan->tiles, tiles.data(), tiles.size() * sizeof(sg_tile_desc), cudaMemcpyHostToDevice) ==
                         cudaSuccess ? SG_OK : SG_ECUDA;
        const size_t nw = (size_t)plan->ntiles * SG_TILE_N;
        // FP64 corner weights (FP64 plans), FP32 cell coefficients (FP32 plans)
        const bool wide = prec == SG_FP64;
        plan->ws_tile_bytes = (int64_t)nw * (wide ? (int64_t)sizeof(sg_dvec4) : (int64_t)sizeof(float4));
        // targets: every leaf, in blocks of the leaves of 16 x 16 cells
        std::vector<int4> tg;
        std::vector<sg_target_block> blocks;
        build_targets(g, gi, tg, blocks);
        plan->ntargets = (int)tg.size();
        plan->nblocks = (int)blocks.size();
        if (st == SG_OK) st = dev_alloc(plan, &plan->targets, tg.size() * sizeof(int4));
        if (st == SG_OK)
            st = cudaMemcpy(plan->targets, tg.data(), tg.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess
                     ? SG_OK : SG_ECUDA;
        if (st == SG_OK) st = dev_alloc(plan, &plan->blocks, blocks.size() * sizeof(sg_target_block));
        if (st == SG_OK)
            st = cudaMemcpy(plan->blocks, blocks.data(), blocks.size() * sizeof(sg_target_block),
                            cudaMemcpyHostToDevice) == cudaSuccess ? SG_OK : SG_ECUDA;
        const int64_t slices = prec == SG_FP64 ? (nsplit > 1 ? nsplit : 0) : nsplit + 1;
        plan->ws_partial_bytes = slices * (int64_t)tg.size() * 2 * (int64_t)sizeof(double);
        if (g->z != 0.0)  // off the plane: three components per split (FP32: and one slice for the near field)
            plan->ws_partial_bytes =
                ((int64_t)nsplit + (prec == SG_FP32 ? 1 : 0)) * (int64_t)tg.size() * 3 * (int64_t)sizeof(double);
        if (st == SG_OK && prec == SG_FP32) st = sg_cross_far_grid(plan, nsm);
    }
    if (st == SG_OK) st = sg_twiddles_build(plan);
    if (st == SG_OK) st = sg_phase_build(plan);
    if (st == SG_OK) st = sg_tables_build(plan);
    if (st == SG_OK && use_lv) st = sg_lv_setup(plan, &lva);  // sets the transform scratch sizes
    plan->scratch_bytes = sg_workspace_bytes(plan);  // the plan's own workspace is allocated at its first sg_force
    {
        const bool central = g->slope_mode == SG_SLOPES_CENTRAL && g->z == 0.0 && !(gi.n > 1 || gi.masked);
        // level convolutions: one launch each for the row, column, column-MAC and inverse-row passes
        int n = use_lv ? 4 : gi.n * (central ? 4 : 3);
        if (plan->composite) {
            n += gi.lmax > 0 ? gi.lmax : 1;  // composite sources: covered cells of levels 1 .. lmax-1, then all S_l
            if (plan->amr_central) n += (gi.lmax > 1 ? gi.lmax - 1 : 0) + gi.lmax + 1;  // fills, then slopes per level
            // direct sum: corner weights, pair sum (+ split reduction) in FP64; cell coefficients,
            // far field, near field and the combination in FP32
            if (plan->ntiles > 0) n += prec == SG_FP64 ? 2 + (nsplit > 1) : 4;
        }
        plan->launches = n;
    }
    if (st == SG_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            sg_set_last_cuda_error(e, "sg_plan_create");
            st = SG_ECUDA;
        }
    }
    if (st != SG_OK) {
        plan_free(plan);
        return st;
    }
    *out = plan;
    return SG_OK;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

sg_status sg_plan_upload(sg_plan *plan, void **dst, const void *src, size_t n)
{
    SG_TRY(dev_alloc(plan, dst, n));
    if (n) SG_CUDA_TRY(cudaMemcpy(*dst, src, n, cudaMemcpyHostToDevice));
    return SG_OK;
}

sg_status sg_plan_build(const sg_geom *geom, sg_precision prec, size_t budget, sg_plan **out)
{
    return plan_build(geom, prec, budget, out);
}

void sg_plan_release(sg_plan *plan) { plan_free(plan); }

// ------------------------------------------------------------- workspaces --

int64_t sg_workspace_bytes(const sg_plan *plan)
{
    return plan->ws_fwd_bytes + plan->ws_inv_bytes + plan->ws_sfield_bytes + plan->ws_tile_bytes +
           plan->ws_partial_bytes;
}

static sg_status ws_alloc_one(void **p, int64_t bytes, cudaStream_t st, bool async)
{
    *p = nullptr;
    if (bytes <= 0) return SG_OK;
    cudaError_t e = async ? cudaMallocAsync(p, (size_t)bytes, st) : cudaMalloc(p, (size_t)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        sg_set_last_cuda_error(e, async ? "cudaMallocAsync" : "cudaMalloc");
        return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
    }
    return SG_OK;
}

void sg_workspace_free(sg_workspace *ws, cudaStream_t st, bool async)
{
    void *bufs[7] = {ws->work_fwd, ws->work_inv, ws->sfield, ws->tile_w, ws->partial, ws->err, ws->zone_buf};
    for (void *b : bufs) {
        if (!b) continue;
        if (async) cudaFreeAsync(b, st);
        else cudaFree(b);
    }
    ws->work_fwd = ws->work_inv = ws->sfield = ws->tile_w = ws->zone_buf = nullptr;
    ws->partial = nullptr;
    ws->err = nullptr;
}

sg_status sg_workspace_alloc(const sg_plan *plan, sg_workspace *ws, cudaStream_t st, bool async)
{
    memset(ws, 0, sizeof(*ws));
    sg_status r = ws_alloc_one(&ws->work_fwd, plan->ws_fwd_bytes, st, async);
    if (r == SG_OK) r = ws_alloc_one(&ws->work_inv, plan->ws_inv_bytes, st, async);
    if (r == SG_OK) r = ws_alloc_one(&ws->sfield, plan->ws_sfield_bytes, st, async);
    if (r == SG_OK) r = ws_alloc_one(&ws->tile_w, plan->ws_tile_bytes, st, async);
    if (r == SG_OK) r = ws_alloc_one((void **)&ws->partial, plan->ws_partial_bytes, st, async);
    if (r == SG_OK) r = ws_alloc_one((void **)&ws->err, 16, st, async);
    if (r == SG_OK) {
        cudaError_t e = async ? cudaMemsetAsync(ws->err, 0, 16, st) : cudaMemset(ws->err, 0, 16);
        if (e != cudaSuccess) r = SG_ECUDA;
    }
    if (r != SG_OK) sg_workspace_free(ws, st, async);
    return r;
}

sg_status sg_force_ws(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *deltax, const void *deltay,
                      void *fx, void *fy, cudaStream_t st, void *fz)
{
    const bool caller = plan->geom.slope_mode == SG_SLOPES_CALLER;
    const void *dx = caller ? deltax : nullptr, *dy = caller ? deltay : nullptr;
    if (!plan->composite) return sg_uniform_solve(plan, ws, 0, sigma, dx, dy, fx, fy, fz, st);
    // AMR or masks: composite sources, then level convolutions, or same-patch FFT
    // convolutions plus the cross-patch direct sum
    SG_TRY(sg_composite_prepare(plan, ws, sigma, dx, dy, st));
    if (plan->lv) return sg_lv_solve(plan, ws, fx, fy, st);
    const size_t es = elem_size(plan->prec);
    const char *S = (const char *)ws->sfield;
    const size_t plane = (size_t)plan->ncells * es;
    for (int k = 0; k < plan->npatches; ++k)
        SG_TRY(sg_uniform_solve(plan, ws, k, S, S + plane, S + 2 * plane, fx, fy, fz, st));
    return sg_cross_solve(plan, ws, S, S + plane, S + 2 * plane, fx, fy, fz, st);
}

// Reads and clears the device error word of the plan's workspace (synchronises).
static sg_status check_device_error(sg_plan *plan)
{
    if (!plan->ws || !plan->ws->err) return SG_OK;
    int e = 0;
    SG_CUDA_TRY(cudaMemcpy(&e, plan->ws->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        SG_CUDA_TRY(cudaMemset(plan->ws->err, 0, sizeof(int)));
        sg_set_last_error_message("a bounded wait for a bulk copy ran out in a kernel");
        return SG_ETIMEOUT;
    }
    return SG_OK;
}

template <typename T>
__global__ void k_fz_plane(const T *__restrict__ sigma, T *__restrict__ fz, int64_t n, double c)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        fz[i] = (T)(c * (double)sigma[i]);
}

// The plan's own workspace, allocated at its first solve.
static sg_status ensure_ws(sg_plan *plan)
{
    if (plan->ws) return SG_OK;
    sg_workspace *ws = new (std::nothrow) sg_workspace();
    if (!ws) return SG_ENOMEM;
    sg_status a = sg_workspace_alloc(plan, ws, 0, false);
    if (a != SG_OK) {
        delete ws;
        return a;
    }
    plan->ws = ws;
    plan->device_bytes += sg_workspace_bytes(plan);
    return SG_OK;
}

// Validation, the plan's own workspace (allocated at the first call), timers, solve.
static sg_status force_common(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx,
                              void *fy, void *fz, void *stream)
{
    if (!plan || !sigma || !fx || !fy) return fail("null plan or field pointer");
    const bool caller = plan->geom.slope_mode == SG_SLOPES_CALLER;
    if (caller && (!deltax || !deltay)) return fail("caller slopes requested but deltax/deltay is NULL");
    const size_t es = elem_size(plan->prec);
    if (!aligned(sigma, es) || !aligned(fx, es) || !aligned(fy, es) || (fz && !aligned(fz, es)) ||
        (caller && (!aligned(deltax, es) || !aligned(deltay, es))))
        return fail("misaligned field pointer");
    int dev = -1;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != plan->device) return fail("the plan's device is not current");
    SG_TRY(ensure_ws(plan));
    sg_timing_reset(plan->timing);
    plan->ws->timing = plan->timing;
    return sg_force_ws(plan, plan->ws, sigma, deltax, deltay, fx, fy, (cudaStream_t)stream, fz);
}

// --------------------------------------------------------------- the C ABI --

extern "C" {

sg_status sg_geom_validate(const sg_geom *geom)
{
    geom_info gi;
    return analyse(geom, gi);
}

sg_status sg_plan_bytes(const sg_geom *geom, sg_precision prec, int64_t *bytes)
{
    if (!bytes || (prec != SG_FP64 && prec != SG_FP32)) return SG_EINVAL;
    geom_info gi;
    SG_TRY(analyse(geom, gi));
    sg_lv_setup_args lva;
    std::vector<std::vector<int>> lvmaps;
    int64_t lv_bytes = -1;
    if ((gi.n > 1 || gi.masked) && geom->cross_mode != SG_CROSS_DIRECT && gi.lmax >= 1 &&
        !lv_params(geom, gi, prec, lva, lvmaps, lv_bytes))
        lv_bytes = -1;
    std::vector<sg_tile_desc> tiles;
    std::vector<int> tf, tc;
    const bool corner_form = prec == SG_FP64;
    if (gi.n > 1 && lv_bytes < 0) build_tiles(geom, gi, !corner_form, tiles, tf, tc);
    const int nblocks = lv_bytes < 0 ? count_blocks(geom, gi) : 0;
    const int nsplit = choose_nsplit(nblocks, (int)tiles.size(), 152, corner_form ? SG_FP64 : prec);
    *bytes = plan_sizes(geom, gi, prec, (int)tiles.size(), nblocks, nsplit, lv_bytes).total();
    return SG_OK;
}

sg_status sg_plan_create(const sg_geom *geom, sg_precision prec, size_t hbm_budget, sg_plan **out)
{
    if (!out || (prec != SG_FP64 && prec != SG_FP32)) return fail("invalid precision or output pointer");
    return plan_build(geom, prec, hbm_budget, out);
}

sg_status sg_plan_destroy(sg_plan *plan)
{
    plan_free(plan);
    return SG_OK;
}

sg_status sg_plan_get_info(const sg_plan *plan, sg_plan_info *out)
{
    if (!plan || !out) return SG_EINVAL;
    out->npatches = plan->npatches;
    out->ncells = plan->ncells;
    out->nleaves = plan->nleaves;
    out->cross_pairs = plan->cross_pairs;
    out->device_bytes = plan->device_bytes;
    out->scratch_bytes = plan->scratch_bytes;
    out->max_pad = plan->max_pad;
    out->nzones = plan->nzones;
    out->launches = plan->launches;
    out->cross_mode = plan->cross_mode;
    return SG_OK;
}

sg_status sg_kernel_tables(const sg_plan *plan, int patch, int which, double *host_out, size_t n)
{
    return sg_tables_copy(plan, patch, which, host_out, n);
}

sg_status sg_force(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx, void *fy,
                   void *stream)
{
    return force_common(plan, sigma, deltax, deltay, fx, fy, nullptr, stream);
}

sg_status sg_force3(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx, void *fy,
                    void *fz, void *stream)
{
    if (!plan || !fz) return fail("null plan or fz pointer");
    if (plan->geom.z != 0.0) return force_common(plan, sigma, deltax, deltay, fx, fy, fz, stream);
    SG_TRY(force_common(plan, sigma, deltax, deltay, fx, fy, nullptr, stream));
    // in the plane: Fz from above is -2 pi G sigma0 of the target's own cell
    const int64_t n = plan->ncells;
    const double c = -2.0 * 3.14159265358979323846 * plan->geom.G;
    const int grid = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
    if (plan->prec == SG_FP64)
        k_fz_plane<double><<<grid, 256, 0, (cudaStream_t)stream>>>((const double *)sigma, (double *)fz, n, c);
    else
        k_fz_plane<float><<<grid, 256, 0, (cudaStream_t)stream>>>((const float *)sigma, (float *)fz, n, c);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

sg_status sg_potential(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *phi,
                       void *stream)
{
    if (!plan || !sigma || !phi) return fail("null plan or field pointer");
    if (plan->geom.z != 0.0) return fail("sg_potential takes plans in the plane (z = 0)");
    const bool caller = plan->geom.slope_mode == SG_SLOPES_CALLER;
    if (caller && (!deltax || !deltay)) return fail("caller slopes requested but deltax/deltay is NULL");
    const size_t es = elem_size(plan->prec);
    if (!aligned(sigma, es) || !aligned(phi, es) || (caller && (!aligned(deltax, es) || !aligned(deltay, es))))
        return fail("misaligned field pointer");
    int dev = -1;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != plan->device) return fail("the plan's device is not current");
    if (plan->lv) {
        // hierarchy: composite sources, then the level convolutions with the potential kernels
        SG_TRY(sg_lv_potential_spectra_build(plan));
        SG_TRY(ensure_ws(plan));
        sg_timing_reset(plan->timing);
        plan->ws->timing = plan->timing;
        SG_TRY(sg_composite_prepare(plan, plan->ws, sigma, caller ? deltax : nullptr, caller ? deltay : nullptr,
                                    (cudaStream_t)stream));
        return sg_lv_potential(plan, plan->ws, phi, (cudaStream_t)stream);
    }
    if (plan->composite) {
        // hierarchy on the direct path: composite sources, each patch's own
        // convolution with its potential spectra, then the cross-patch sum
        SG_TRY(sg_potential_spectra_build(plan));
        SG_TRY(ensure_ws(plan));
        sg_timing_reset(plan->timing);
        plan->ws->timing = plan->timing;
        cudaStream_t st = (cudaStream_t)stream;
        SG_TRY(sg_composite_prepare(plan, plan->ws, sigma, caller ? deltax : nullptr, caller ? deltay : nullptr, st));
        const char *S = (const char *)plan->ws->sfield;
        const size_t plane = (size_t)plan->ncells * es;
        for (int k = 0; k < plan->npatches; ++k)
            SG_TRY(sg_uniform_potential(plan, plan->ws, k, plan->ws->work_fwd, S, S + plane, S + 2 * plane, phi, st));
        return sg_cross_potential(plan, plan->ws, S, S + plane, S + 2 * plane, phi, st);
    }
    SG_TRY(sg_potential_spectra_build(plan));
    SG_TRY(ensure_ws(plan));
    const sg_patch_dev &d = plan->pp[0].d;
    const int64_t need = 3LL * (d.px / 2 + 1) * d.ny * (int64_t)(2 * es);
    void *wf = plan->ws->work_fwd;
    if (plan->ws_fwd_bytes < need) {
        if (!plan->pot_fwd) {
            SG_TRY(dev_alloc(plan, &plan->pot_fwd, (size_t)need));
            plan->pot_fwd_bytes = need;
        }
        wf = plan->pot_fwd;
    }
    sg_timing_reset(plan->timing);
    plan->ws->timing = plan->timing;
    return sg_uniform_potential(plan, plan->ws, 0, wf, sigma, caller ? deltax : nullptr, caller ? deltay : nullptr, phi,
                                (cudaStream_t)stream);
}

// The device address of a page-locked host buffer, or NULL for other memory.
static const void *mapped_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The host-buffer solve enqueued on `stream`. mapped_io: pinned buffers of a
// single in-plane patch are read and written in place by the transform passes
// (the transfers overlap the solve's own passes: the lower latency of one
// solve); otherwise every transfer is a copy-engine copy into or out of the
// plan's staging buffers, leaving the SMs to the other solves in flight (the
// higher throughput when solves on several streams overlap).
static sg_status host_enqueue(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx,
                              void *fy, void *stream, bool mapped_io)
{
    if (!plan || !sigma || !fx || !fy) return fail("null plan or field pointer");
    const bool caller = plan->geom.slope_mode == SG_SLOPES_CALLER;
    if (caller && (!deltax || !deltay)) return fail("caller slopes requested but deltax/deltay is NULL");
    int dev = -1;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != plan->device) return fail("the plan's device is not current");
    cudaStream_t st = (cudaStream_t)stream;
    // Pinned output buffers are mapped into the device address space: for a
    // single in-plane patch the inverse row pass writes Fx, Fy there in place
    // (streaming writes over the CPU-GPU link) instead of a copy after the solve.
    void *hfx = nullptr, *hfy = nullptr;
    if (mapped_io && !plan->composite && plan->geom.z == 0.0) {
        hfx = (void *)mapped_host(fx);
        hfy = (void *)mapped_host(fy);
        if (!hfx || !hfy) hfx = hfy = nullptr;
    }
    const size_t bytes = (size_t)plan->ncells * elem_size(plan->prec);
    if (!plan->stage_in) {
        SG_TRY(dev_alloc(plan, &plan->stage_in, 3 * bytes));
        sg_status s = dev_alloc(plan, &plan->stage_out, 2 * bytes);
        if (s != SG_OK) {
            cudaFree(plan->stage_in);
            plan->stage_in = nullptr;
            plan->device_bytes -= (int64_t)(3 * bytes);
            return s;
        }
        plan->stage_bytes = bytes;
    }
    char *in = (char *)plan->stage_in, *out = (char *)plan->stage_out;
    // Likewise pinned inputs of a single in-plane patch are read in place by the
    // forward row pass (and the edge-column transform), so the transfer overlaps
    // the transform instead of preceding it.
    const void *ms = hfx ? mapped_host(sigma) : nullptr;
    const void *mdx = ms && caller ? mapped_host(deltax) : nullptr;
    const void *mdy = ms && caller ? mapped_host(deltay) : nullptr;
    const bool in_place = ms && (!caller || (mdx && mdy));
    if (!in_place) {
        SG_CUDA_TRY(cudaMemcpyAsync(in, sigma, bytes, cudaMemcpyHostToDevice, st));
        if (caller) {
            SG_CUDA_TRY(cudaMemcpyAsync(in + bytes, deltax, bytes, cudaMemcpyHostToDevice, st));
            SG_CUDA_TRY(cudaMemcpyAsync(in + 2 * bytes, deltay, bytes, cudaMemcpyHostToDevice, st));
        }
    }
    if (in_place) {
        SG_TRY(sg_force(plan, ms, mdx, mdy, hfx, hfy, stream));
    } else if (hfx) {
        SG_TRY(sg_force(plan, in, caller ? in + bytes : nullptr, caller ? in + 2 * bytes : nullptr, hfx, hfy, stream));
    } else {
        SG_TRY(sg_force(plan, in, caller ? in + bytes : nullptr, caller ? in + 2 * bytes : nullptr, out, out + bytes,
                        stream));
        SG_CUDA_TRY(cudaMemcpyAsync(fx, out, bytes, cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaMemcpyAsync(fy, out + bytes, bytes, cudaMemcpyDeviceToHost, st));
    }
    // the error word follows the solve on the stream, so that the wait reads it
    // without another round trip to the device
    if (!plan->ws || !plan->ws->err) return SG_OK;
    if (!plan->err_host) SG_CUDA_TRY(cudaHostAlloc((void **)&plan->err_host, sizeof(int), cudaHostAllocDefault));
    SG_CUDA_TRY(cudaMemcpyAsync(plan->err_host, plan->ws->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    return SG_OK;
}

sg_status sg_force_host_async(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx,
                              void *fy, void *stream)
{
    return host_enqueue(plan, sigma, deltax, deltay, fx, fy, stream, false);
}

sg_status sg_plan_wait(sg_plan *plan, void *stream)
{
    if (!plan) return fail("null plan");
    SG_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (plan->err_host && *(volatile int *)plan->err_host) {
        *(volatile int *)plan->err_host = 0;
        SG_CUDA_TRY(cudaMemset(plan->ws->err, 0, sizeof(int)));
        sg_set_last_error_message("a bounded wait for a bulk copy ran out in a kernel");
        return SG_ETIMEOUT;
    }
    return SG_OK;
}

sg_status sg_force_host(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx, void *fy,
                        void *stream)
{
    SG_TRY(host_enqueue(plan, sigma, deltax, deltay, fx, fy, stream, true));
    return sg_plan_wait(plan, stream);
}

sg_status sg_plan_set_wait_limit(sg_plan *plan, int tries)
{
    if (!plan || tries < -1) return fail("null plan or wait limit below -1");
    plan->wait_tries = tries == -1 ? SG_MBAR_MAX_TRIES : tries;
    return SG_OK;
}

sg_status sg_plan_check_error(sg_plan *plan)
{
    if (!plan) return fail("null plan");
    SG_CUDA_TRY(cudaDeviceSynchronize());
    return check_device_error(plan);
}

sg_status sg_plan_set_timing(sg_plan *plan, int enable)
{
    if (!plan) return SG_EINVAL;
    if (enable && !plan->timing) {
        plan->timing = new (std::nothrow) sg_timing();
        if (!plan->timing) return SG_ENOMEM;
    } else if (!enable && plan->timing) {
        cudaDeviceSynchronize();
        for (cudaEvent_t e : plan->timing->pool) cudaEventDestroy(e);
        delete plan->timing;
        plan->timing = nullptr;
    }
    return SG_OK;
}

sg_status sg_plan_get_timing(sg_plan *plan, double *ms, int n)
{
    if (!plan || !ms || n < SG_NSTAGES) return SG_EINVAL;
    for (int i = 0; i < SG_NSTAGES; ++i) ms[i] = 0.0;
    sg_timing *t = plan->timing;
    if (!t) return SG_EINVAL;
    for (size_t k = 0; k < t->stage.size(); ++k) {
        const int b = 2 * (int)k, e = b + 1;
        if (e >= t->used) break;
        SG_CUDA_TRY(cudaEventSynchronize(t->pool[e]));
        float v = 0.f;
        SG_CUDA_TRY(cudaEventElapsedTime(&v, t->pool[b], t->pool[e]));
        ms[t->stage[k]] += v;
    }
    return check_device_error(plan);
}

const char *sg_strerror(sg_status s)
{
    switch (s) {
    case SG_OK: return "ok";
    case SG_EINVAL: return "invalid argument";
    case SG_ENOMEM: return "out of memory";
    case SG_EBUDGET: return "device-memory budget exceeded";
    case SG_ECUDA: return "CUDA error";
    case SG_ETIMEOUT: return "timed out";
    case SG_EBUSY: return "busy";
    case SG_ECANCELLED: return "cancelled";
    case SG_ENOTFOUND: return "not found";
    }
    return "unknown status";
}

const char *sg_last_error(void) { return g_last_error; }

int sg_version(void) { return 100; }

}  // extern "C"
