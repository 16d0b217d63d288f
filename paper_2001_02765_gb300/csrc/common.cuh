// Common definitions of the thin-disk self-gravity library (device and host).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "sg.h"
#include "tma.cuh"

#define SG_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t sg_e_ = (expr);                        \
        if (sg_e_ != cudaSuccess) {                        \
            sg_set_last_cuda_error(sg_e_, #expr);          \
            return SG_ECUDA;                               \
        }                                                  \
    } while (0)

#define SG_TRY(expr)                                       \
    do {                                                   \
        sg_status sg_s_ = (expr);                          \
        if (sg_s_ != SG_OK) return sg_s_;                  \
    } while (0)

void sg_set_last_cuda_error(cudaError_t e, const char *what);
void sg_set_last_error_message(const char *msg);

// Programmatic dependent launch. A kernel launched by sg_launch_dep may be
// scheduled before the previous kernel of its stream has finished, once every
// CTA of that kernel has executed sg_dep_trigger (or exited); it calls
// sg_dep_wait before it reads anything that kernel wrote. Both are no-ops for
// kernels launched without the attribute.
__device__ __forceinline__ void sg_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void sg_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t sg_launch_dep(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------ complex math --

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx_of<T>::type;

template <typename C> __host__ __device__ __forceinline__ C cmake(decltype(C::x) re, decltype(C::x) im)
{
    C c;
    c.x = re;
    c.y = im;
    return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b)
{
    return cmake<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }

// Explicitly rounded product and sum: the optimiser may fuse a plain multiply
// and add into an FMA, and may decide differently in different instantiations
// of one kernel; these pin the rounding of expressions whose results must not
// depend on the launch shape.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
// p q with one FMA per component: (fma(p.x, q.x, -(p.y q.y)), fma(p.x, q.y, p.y q.x))
template <typename C> __device__ __forceinline__ C cmul_rn(C a, C b)
{
    return cmake<C>(fma(a.x, b.x, -mul_rn(a.y, b.y)), fma(a.x, b.y, mul_rn(a.y, b.x)));
}

// 32-byte aligned FP64 4-vector (corner weights of FP64 plans)
struct __align__(32) sg_dvec4 {
    double x, y, z, w;
};

// ------------------------------------------------------------- plan layout --

// Largest padded FFT length handled by the transform kernels.
#define SG_MAX_PAD 4096
// Largest padded length of the level convolutions (FP32; FP64 stops at SG_MAX_PAD).
#define SG_LV_MAX_PAD 8192
#define SG_MIN_PAD 64
#define SG_MAX_PATCH_SIDE 2048
#define SG_MAX_LEVELS 12

// Source tiles of the cross-patch direct sum: TILE_X x TILE_Y corners (FP64
// plans, corner form) or cells (FP32 plans, near/far split).
#define SG_TILE_X 16
#define SG_TILE_Y 16
#define SG_TILE_N (SG_TILE_X * SG_TILE_Y)
// Leaf targets per CTA of the direct sum (a block covers 16 x 16 cells of one patch).
#define SG_DIRECT_THREADS 256
// FP32 direct sum: a source cell whose centre lies less than SG_NEAR_R of its
// own widths from the target along both axes is summed exactly in FP64 (near
// field); every other cell by the expansion of its integrals about its centre,
// through H^6 for tiles closer than SG_FAR_R4 cell widths to a block, through
// H^4 beyond.
#define SG_NEAR_R 6
#define SG_FAR_R4 32

struct sg_tile_desc {
    int patch;          // source patch
    int ox, oy;         // lattice coordinates of corner (0, 0) of the tile (corner tiles) or of
                        // the lower-left corner of its cell (0, 0) (cell tiles)
    int step;           // corner spacing (cell width) in lattice units
    int ci0, cj0;       // first corner (cell) index (i, j) of the tile in its patch
    int pad0, pad1;
};

struct sg_target_block {
    int patch;          // patch of every target in the block
    int first;          // first index into the target arrays
    int count;          // targets in the block (<= SG_DIRECT_THREADS)
    int pad;
    int tx0, ty0;       // lattice bounding box of the block's target positions
    int tx1, ty1;
};

struct sg_patch_dev {
    int nx, ny;
    int px, py;         // padded FFT lengths
    int64_t cell_off;   // offset of the patch in the field arrays
    double h;
    int ox, oy;         // lattice coordinates of the patch's lower-left corner
    int step;           // cell width in lattice units
    int parent;         // parent patch (-1 on level 0)
    int pi0, pj0;       // offset of this patch in its parent's cells
    int64_t ncells_plane;  // plane stride of the 3-field composite source arrays (= total cells)
    int tile_first, tile_count;  // the patch's source tiles in the direct-sum tile list
};

// Level convolutions (lvconv.cu): every level's composite source sampled on the
// finest lattice (cells of level m are 2^s finest cells wide, s = lmax - m; the
// sample of a cell of a coarser level sits half a finest cell up and right of
// its centre), one FFT convolution per ordered pair of levels.
struct sg_lv_level {
    int s;              // cells of this level are 2^s finest cells wide
    int nx, ny;         // level image: bounding box of the level's patches, in cells
    int i0, j0;         // finest-lattice index of the sample point of image cell (0, 0)
    int cx, cy;         // compression exponents: source transforms of length px >> cx, py >> cy
    int *map;           // device [ny][nx]: index of the cell in the field arrays, or -1
    int64_t fwd_off;    // complex-element offset of the level's row transforms (3 fields)
    int64_t spec_off;   // of its compact source spectra (3 fields)
    int64_t inv_off;    // of its inverse-column outputs (Fx, Fy)
};


struct sg_lv {
    int nlev;
    int px, py;                              // padded lengths of the finest lattice
    double hf;                               // finest cell width
    sg_lv_level lev[SG_MAX_LEVELS];
    int nkeys;
    int key[SG_MAX_LEVELS][SG_MAX_LEVELS];   // kernel of source level m, target level l
    int key_s[3 * SG_MAX_LEVELS];            // per kernel: source width exponent s
    int key_d2[3 * SG_MAX_LEVELS];           // per kernel: 2 x sample shift (-1, 0, 1)
    void *spectra;                           // [nkeys][6][px/2+1][sg_spec_stride(py)] T (compressed, see lvconv.cu)
    void *phase;                             // exp(i pi k / P), k in [-P/2, P/2], x then y, complex T
    void *cphase;                            // exp(-i pi j / P), j in [0, P], x then y, complex T
    void *pspectra;                          // potential: [nkeys][3][px/2+1][sg_spec_stride(py)] T, built at the first call
    int64_t fwd_elems, spec_elems, inv_elems;
};

struct sg_patch_plan {
    sg_patch geom;
    sg_patch_dev d;
    // device buffers owned by the plan
    void *spectra;      // 6 planes [(px/2+1) x sg_spec_stride(py)] of T (quarter spectra, scaled)
    void *phase;        // central-slope spectral factors (see fftconv.cu), NULL unless SG_SLOPES_CENTRAL
    void *pspectra;     // potential planes p, a, b [(px/2+1) x sg_spec_stride(py)] of T, built at the first sg_potential
    // tile range of this patch in the tile list
    int tile_first, tile_count;
};

struct sg_plan {
    int device;
    sg_precision prec;
    sg_geom geom;
    int npatches;
    sg_patch *patches_host;
    sg_patch_plan *pp;
    int64_t ncells;
    int64_t nleaves;
    int64_t cross_pairs;
    int64_t device_bytes;
    int64_t scratch_bytes;
    int max_pad;
    double lattice_unit;            // lambda: half of the finest cell width
    double lattice_x0, lattice_y0;  // physical position of lattice coordinate 0

    // twiddle tables exp(-2 pi i k / L), k < L, for each power of two L in
    // [SG_MIN_PAD, max_pad]: FP64 copies then FP32 copies, back to back
    void *twiddles;
    int64_t tw64_off[16];           // byte offsets, indexed by log2 L
    int64_t tw32_off[16];

    // per cell (device, ncells): SG_CELL_ABSENT, SG_CELL_LEAF, or the index of the
    // child patch that covers the cell
    int *cell_code;
    // composite sources (AMR prepare + per-patch FFT on them): several patches or masks
    bool composite;
    // composite-source launches (amr.cu), over the patches sorted by level
    // (comp_order; level l is comp_lev_first[l] .. comp_lev_first[l+1]): prefix
    // sums of their cells (comp_cells, device, and a host copy) and of the final
    // launch's items (comp_item_off: cells on level 0, 2x2 blocks above)
    int *comp_order;
    int64_t *comp_cells;
    int64_t *comp_cells_host;
    int64_t *comp_item_off;
    int64_t comp_items;
    int comp_lev_first[SG_MAX_LEVELS + 1];
    int comp_depth;                 // levels of the hierarchy (lmax + 1)

    // slopes of hierarchies with SG_SLOPES_CENTRAL (the neighbour-leaf rule, amr.cu):
    // per cell and side (left, down, right, up) what lies across it, {a, b}: b >= 0 the
    // two children a, b of a refined cell of the same level that touch the side; b = -1
    // the leaf a of the same level; b = -2 the coarser leaf a; b = -3 nothing (outside)
    bool amr_central;
    int2 *slope_nb;                 // device, 4 x ncells
    int2 *cell_pos;                 // device, ncells: lattice coordinates of the cell centres
    int64_t lev_cells[SG_MAX_LEVELS + 1];  // cells of level l: [lev_cells[l], lev_cells[l+1]) (patches sorted by level)
    int lev_step[SG_MAX_LEVELS];    // cell width of level l in lattice units

    // zone plans (sg_plan_create_zones): zone k sits at cell zone_slot[k] (device)
    int64_t nzones;
    int64_t *zone_slot;
    int64_t ws_zone_bytes;          // per-call zone-order staging, 5 x ncells of T
    int launches;                   // kernels one solve enqueues
    int cross_mode;                 // SG_CROSS_DIRECT, SG_CROSS_LEVELS, or 0 (single unmasked patch)
    void *pot_fwd;                  // forward scratch of sg_potential (three fields), when work_fwd is smaller
    int64_t pot_fwd_bytes;
    sg_lv *lv;                      // level-convolution plan (SG_CROSS_LEVELS), else NULL

    // per-call scratch sizes (bytes) and the plan's own workspace (used by sg_force)
    int64_t ws_fwd_bytes, ws_inv_bytes, ws_sfield_bytes, ws_tile_bytes, ws_partial_bytes;
    struct sg_workspace *ws;

    // cross-patch direct sum
    int ntiles;
    sg_tile_desc *tiles;            // device
    int nsplit;                     // source-tile ranges per target block
    int far_grid;                   // CTAs of the persistent far-field launch (FP32 plans)
    int wait_tries;                 // attempts of the kernels' bounded waits (SG_MBAR_MAX_TRIES by default)
    int ntargets;
    int4 *targets;                  // device: (lattice x, lattice y, output index, patch)
    int nblocks;
    sg_target_block *blocks;        // device
    sg_patch_dev *patch_dev;        // device copy of every patch's sg_patch_dev

    // host staging for sg_force_host
    void *stage_in, *stage_out;
    size_t stage_bytes;
    int *err_host;                  // pinned: the workspace's error word, copied after each host-buffer solve

    // per-stage device timers of the last sg_force (NULL when timing is off)
    struct sg_timing *timing;
};

// Per-call scratch of a solve. A plan owns one (sg_force); the request server
// gives every in-flight request its own, so requests on one plan can overlap.
struct sg_workspace {
    void *work_fwd;         // uniform-transform scratch: 3 x (px/2+1) x ny complex (largest patch)
    void *work_inv;         // 2 x (px/2+1) x ny complex
    void *sfield;           // AMR composite source fields, 3 x ncells of T
    void *tile_w;           // AMR corner weights (FP64 plans) or cell coefficients (FP32 plans),
                            // ntiles x SG_TILE_N x 4 of T
    double *partial;        // AMR direct-sum partial sums: nsplit x ntargets x 2 (FP64 plans, nsplit > 1);
                            // (nsplit + 1) x ntargets x 2, the last slice the near field (FP32 plans)
    void *zone_buf;         // zone plans: inputs (3 planes) and outputs (2 planes) in patch layout
    int *err;               // device words: err[0] nonzero after a bounded wait in a kernel ran out;
                            // err[1] the work-item counter of the persistent far-field launch
    struct sg_timing *timing;  // stage timers, or NULL
};

// Cell codes of sg_plan::cell_code.
#define SG_CELL_ABSENT (-2)
#define SG_CELL_LEAF (-1)

// Build a plan for a validated geometry (api.cu); zone plans add their map afterwards.
sg_status sg_plan_build(const sg_geom *geom, sg_precision prec, size_t budget, sg_plan **out);
void sg_plan_release(sg_plan *plan);
// Copy n bytes to a new device buffer owned by the plan (counted in device_bytes).
sg_status sg_plan_upload(sg_plan *plan, void **dst, const void *src, size_t n);

// Allocate / free a workspace for a plan. async: stream-ordered allocation on st.
sg_status sg_workspace_alloc(const sg_plan *plan, sg_workspace *ws, cudaStream_t st, bool async);
void sg_workspace_free(sg_workspace *ws, cudaStream_t st, bool async);
int64_t sg_workspace_bytes(const sg_plan *plan);
// One solve on an explicit workspace (sg_force uses the plan's own).
sg_status sg_force_ws(sg_plan *plan, const sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                      void *fx, void *fy, cudaStream_t st, void *fz = nullptr);

// Stages timed by sg_plan_get_timing.
enum { SG_STAGE_ROW_FWD = 0, SG_STAGE_COL_CONV = 1, SG_STAGE_ROW_INV = 2, SG_STAGE_WEIGHTS = 3,
       SG_STAGE_DIRECT = 4, SG_STAGE_COMPOSITE = 5, SG_NSTAGES = 6 };

// Record the start / end of a stage on a stream (no-op when timing is off).
void sg_timing_begin(const struct sg_workspace *ws, int stage, cudaStream_t st);
void sg_timing_end(const struct sg_workspace *ws, int stage, cudaStream_t st);
void sg_timing_reset(struct sg_timing *t);

// ---------------------------------------------------------- host functions --

struct sg_workspace;
struct sg_timing;

sg_status sg_tables_build(sg_plan *plan);     // tables + spectra of every patch
sg_status sg_tables_copy(const sg_plan *plan, int patch, int which, double *host_out, size_t n);
sg_status sg_twiddles_build(sg_plan *plan);
sg_status sg_phase_build(sg_plan *plan);     // central-slope factors of every patch
sg_status sg_uniform_solve(sg_plan *plan, const struct sg_workspace *ws, int patch, const void *sigma, const void *dx,
                           const void *dy, void *fx, void *fy, void *fz, cudaStream_t st);
sg_status sg_uniform_potential(sg_plan *plan, const struct sg_workspace *ws, int patch, void *wf, const void *sigma,
                               const void *dx, const void *dy, void *phi, cudaStream_t st);
sg_status sg_potential_spectra_build(sg_plan *plan);   // synchronous, every patch
// Launch shapes of the uniform-patch passes for a padded length (tune.cu):
// shape[0] row sequences per CTA (forward), [1] (inverse), [2] columns per CTA
// of the column pass, [3] of the central-slope column pass.
#define SG_TUNE_KNOBS 4
void sg_tune_shape(sg_precision prec, int pad, int *shape);
sg_status sg_cross_solve(sg_plan *plan, const struct sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                         void *fx, void *fy, void *fz, cudaStream_t st);  // fz: z != 0 plans only
// Grid of the persistent far-field launch of an FP32 plan (sets plan->far_grid).
sg_status sg_cross_far_grid(sg_plan *plan, int nsm);
// the potential's cross-patch sum, added into phi (the patches' own convolutions already there)
sg_status sg_cross_potential(sg_plan *plan, const struct sg_workspace *ws, const void *sigma, const void *dx,
                             const void *dy, void *phi, cudaStream_t st);
sg_status sg_amr_prepare(sg_plan *plan, const struct sg_workspace *ws, const void *sigma, const void *dx, const void *dy,
                         cudaStream_t st);
// Composite sources of a solve (amr.cu): with caller slopes or none as given; for
// SG_SLOPES_CENTRAL hierarchies the neighbour-leaf slopes first (workspace planes).
sg_status sg_composite_prepare(sg_plan *plan, const struct sg_workspace *ws, const void *sigma, const void *dx,
                               const void *dy, cudaStream_t st);
sg_status sg_fft_lines_fp64(double2 *data, int L, int count, int64_t seq_stride, int64_t elem_stride,
                           const double2 *tw);
// Level convolutions: host setup (level images, maps, kernel spectra) and the solve.
struct sg_lv_setup_args {
    int nlev, px, py;
    double hf;
    int s[SG_MAX_LEVELS], nx[SG_MAX_LEVELS], ny[SG_MAX_LEVELS], i0[SG_MAX_LEVELS], j0[SG_MAX_LEVELS];
    const int *map[SG_MAX_LEVELS];          // host [ny][nx] cell index or -1
};
sg_status sg_lv_setup(sg_plan *plan, const sg_lv_setup_args *a);
void sg_lv_free(sg_plan *plan);
sg_status sg_lv_solve(sg_plan *plan, const struct sg_workspace *ws, void *fx, void *fy, cudaStream_t st);
// The mid-plane potential of a level-convolution plan (composite sources already
// in the workspace); its spectra are built by the first call (synchronously).
sg_status sg_lv_potential_spectra_build(sg_plan *plan);
sg_status sg_lv_potential(sg_plan *plan, const struct sg_workspace *ws, void *phi, cudaStream_t st);

static inline int sg_ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Compression exponent of a level of width exponent s on an axis of padded
// length p: its samples lie every 2^s finest cells, so its spectrum repeats
// with period p / 2^s; transforms stay at 64 points or more.
static inline int sg_lv_cexp(int s, int p)
{
    const int c = sg_ilog2(p) - 6;
    return s < c ? s : c;
}

// Row stride of the spectra planes: (Py/2 + 1) rounded up to 4 entries so that
// every row starts on a 16-byte boundary (bulk copies need it).
static inline __host__ __device__ int sg_spec_stride(int py) { return ((py / 2 + 1) + 3) & ~3; }

static inline int sg_pad_length(int n)
{
    int p = SG_MIN_PAD;
    while (p < 2 * n - 1) p <<= 1;
    return p;
}
