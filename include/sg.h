/*
 * sg.h -- C ABI of the thin-disk self-gravity library (GB300, sm_103a).
 *
 * The library computes the in-plane gravitational force (Fx, Fy) at the centre
 * of every leaf cell of an infinitesimally thin disk whose surface density is
 * piecewise linear on rectangular cells (Tseng, Shang & Yen, Section 2):
 *
 *   sigma_i(x, y) = sigma0_i + deltax_i (x - xc_i) + deltay_i (y - yc_i)   (Eq. eqnGamma)
 *   Fx(t) = G sum_i [sigma0_i K^{x,0}_i(t) + deltax_i K^{x,x}_i(t) + deltay_i K^{x,y}_i(t)]
 *   Fy(t) = G sum_i [sigma0_i K^{y,0}_i(t) + deltax_i K^{y,x}_i(t) + deltay_i K^{y,y}_i(t)]
 *
 * with the closed-form cell integrals of (xbar - x)/r^3 and (ybar - y)/r^3 listed
 * in Section 2 (z = 0), including the coincident-line form for targets on a
 * source edge line. The force is attractive (points towards mass).
 *
 * Grids are sets of patches: uniform blocks of square cells. A single patch is
 * a uniform grid; several patches on refinement levels 0, 1, 2, ... (ratio 2,
 * Section 3 and Fig. 1) form an AMR hierarchy whose leaves are the cells not
 * covered by a patch of the next level. Pairs of cells in the same patch are
 * summed as a zero-padded FFT convolution; pairs in different patches either
 * by level convolutions (every level on the finest lattice, fractional-offset
 * kernel tables) or by a direct sum (the corner form in FP64; in FP32 plans
 * FP64 near cells and a cell-centred expansion of far cells). All give the sum
 * above to rounding.
 *
 * Conventions
 *  - Every entry point returns an sg_status; no exception or signal crosses
 *    the ABI. sg_strerror() names a status.
 *  - Field arrays (sigma, deltax, deltay, Fx, Fy) are per-patch dense arrays,
 *    row-major [y][x] (cell (j, i) of a patch has centre
 *    (x0 + (i + 1/2) h, y0 + (j + 1/2) h)), concatenated in patch order;
 *    element type double for SG_FP64 plans and float for SG_FP32 plans.
 *    Values at covered (non-leaf) cells are ignored on input and unspecified
 *    on output.
 *  - The caller owns every field buffer. A plan owns its device memory
 *    (kernel spectra, geometry tables, scratch) until sg_plan_destroy.
 *  - A plan is bound to the CUDA device that was current at sg_plan_create and
 *    must be used with that device current. A plan is not thread-safe: calls on
 *    one plan must not overlap (they share the plan's scratch).
 *  - Streams are passed as opaque pointers (a cudaStream_t; NULL is the legacy
 *    default stream). Work is enqueued and the call returns without waiting.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SG_OK = 0,
    SG_EINVAL = 1,      /* invalid argument or geometry */
    SG_ENOMEM = 2,      /* a device or host allocation failed */
    SG_EBUDGET = 3,     /* the plan would exceed the caller's device-memory budget */
    SG_ECUDA = 4,       /* a CUDA runtime call failed */
    SG_ETIMEOUT = 5,    /* a bounded wait ran out */
    SG_EBUSY = 6,       /* the request is still running */
    SG_ECANCELLED = 7,  /* the request was cancelled */
    SG_ENOTFOUND = 8    /* unknown ticket */
} sg_status;

typedef enum {
    SG_FP64 = 0,        /* FP64 fields, FP64 transforms and sums */
    SG_FP32 = 1         /* FP32 fields and transforms with FP64-built kernel spectra;
                           compensated (FP64) accumulation across direct-sum tiles */
} sg_precision;

typedef enum {
    SG_SLOPES_NONE = 0,     /* order-0: deltax = deltay = 0 (first-order accurate) */
    SG_SLOPES_CENTRAL = 1,  /* deltax, deltay by central differences on the patch,
                               neighbours outside the patch counting as zero
                               (single-patch geometries only) */
    SG_SLOPES_CALLER = 2    /* deltax, deltay supplied by the caller */
} sg_slope_mode;

typedef struct {
    int level;          /* refinement level, 0 = coarsest */
    int nx, ny;         /* cells along x and y, each >= 1 */
    double x0, y0;      /* lower-left corner of the patch */
    double h;           /* cell width (square cells) */
} sg_patch;

typedef struct {
    int npatches;               /* >= 1 */
    const sg_patch *patches;    /* sorted by level; level-0 patches first */
    double G;                   /* gravitational constant */
    int slope_mode;             /* an sg_slope_mode */
    double z;                   /* height of the targets above the disk plane; 0 = in the plane.
                                   z != 0 (off-plane forces, Section 2 with the arctan terms;
                                   sg_force3): one patch, or a hierarchy on the direct-sum path
                                   (level convolutions are for z == 0) */
    const uint8_t *const *masks; /* NULL, or one entry per patch: NULL (every cell of the patch
                                   exists) or nx*ny bytes, row-major, nonzero where the cell
                                   exists. Cells that do not exist carry no density and get no
                                   force (quadtree hierarchies, where a refined region is not a
                                   rectangle). Rules: on a refined patch existing cells come in
                                   whole 2 x 2 blocks over an existing parent cell; a parent
                                   cell with children is not a leaf. With SG_SLOPES_CENTRAL the
                                   neighbour-leaf rule applies (absent cells count as outside).
                                   Read during sg_plan_create only. */
    int cross_mode;             /* an sg_cross_mode: how pairs of cells in different patches
                                   (and, with level convolutions, all pairs) are summed */
} sg_geom;

typedef enum {
    SG_CROSS_AUTO = 0,          /* level convolutions when the hierarchy fits, else direct */
    SG_CROSS_DIRECT = 1,        /* per-patch FFT convolutions + the direct sum across patches (corner
                                   form in FP64 plans; FP64 near cells and a far-field expansion,
                                   or quadrature off the plane, in FP32 plans) */
    SG_CROSS_LEVELS = 2         /* level convolutions (SG_EINVAL if the hierarchy does not fit):
                                   every level's composite source on the finest lattice, every
                                   ordered pair of levels one zero-padded FFT convolution with
                                   fractional-offset kernel tables; needs a finest-lattice
                                   extent of at most 4096 cells per axis (2048 in FP64 plans)
                                   and z == 0 */
} sg_cross_mode;

typedef struct {
    int npatches;
    int64_t ncells;             /* total cells over all patches (field array length) */
    int64_t nleaves;            /* leaf cells (targets) */
    int64_t cross_pairs;        /* leaf-target x leaf-source pairs summed directly */
    int64_t device_bytes;       /* device memory held by the plan now */
    int64_t scratch_bytes;      /* per-call scratch (workspace) of one solve */
    int max_pad;                /* largest padded FFT length */
    int64_t nzones;             /* zones of a plan made by sg_plan_create_zones, else 0 */
    int launches;               /* kernels one sg_force (sg_force_zones for zone plans) enqueues */
    int cross_mode;             /* the path chosen: SG_CROSS_DIRECT or SG_CROSS_LEVELS (0 for a
                                   single unmasked patch, whose only pairs are same-patch pairs) */
} sg_plan_info;

typedef struct sg_plan sg_plan;

/*
 * Check a geometry without touching a GPU. Rules: every patch has nx, ny >= 1
 * and h > 0; level-0 patches share one lattice of cell width h0 and do not
 * overlap; a patch of level l+1 has h = h_l / 2, lies inside one level-l patch,
 * starts on that patch's cell lattice and covers whole parent cells (even nx,
 * ny); patches of one level do not overlap; at most 12 levels; the lattice of
 * the finest level's half-cells spans at most 2^23 units per axis; a single
 * patch has at most 2048 cells per side. slope_mode SG_SLOPES_CENTRAL needs a
 * single patch. Masks, where given, follow the rules stated at sg_geom.masks.
 * Returns SG_OK or SG_EINVAL.
 */
sg_status sg_geom_validate(const sg_geom *geom);

/*
 * Create a plan: validate the geometry, allocate the plan's device memory,
 * generate the FP64 kernel tables of every patch (Section 2 closed forms),
 * transform them into kernel spectra, and build the cross-patch target and
 * corner-tile lists. Device work runs on the legacy default stream and is
 * complete when the call returns. The plan's own per-call scratch
 * (sg_plan_info.scratch_bytes) is allocated at its first sg_force; the request
 * server gives each request its own instead.
 *   geom        geometry (host memory, read during the call only)
 *   prec        SG_FP64 or SG_FP32
 *   hbm_budget  maximum device bytes the plan may hold (0 = no limit);
 *               SG_EBUDGET if exceeded
 *   out         receives the plan handle (unchanged on error)
 * Errors: SG_EINVAL (geometry, precision, null pointer), SG_EBUDGET,
 * SG_ENOMEM, SG_ECUDA.
 */
sg_status sg_plan_create(const sg_geom *geom, sg_precision prec, size_t hbm_budget, sg_plan **out);

/* Release a plan and its device memory (synchronises the device first). NULL is a no-op. */
sg_status sg_plan_destroy(sg_plan *plan);

/* Sizes and counts of a plan (host memory). */
sg_status sg_plan_get_info(const sg_plan *plan, sg_plan_info *out);

/*
 * Host-only estimate of the device bytes sg_plan_create would hold for this
 * geometry and precision (written to *bytes). SG_EINVAL for an invalid geometry.
 */
sg_status sg_plan_bytes(const sg_geom *geom, sg_precision prec, int64_t *bytes);

/*
 * Copy one FP64 kernel table of patch `patch` to host memory, regenerated on
 * the device: which = 0..5 selects K^{x,0}, K^{x,x}, K^{x,y}, K^{y,0},
 * K^{y,x}, K^{y,y} (Section 2); for plans with z != 0 also 6..8 = K^{z,0},
 * K^{z,x}, K^{z,y}. Entry [n + ny - 1][m + nx - 1] (row-major,
 * (2 nx - 1) x (2 ny - 1) doubles) holds the integral over a source cell whose
 * centre is offset by (m h, n h) from the target centre, in physical units
 * (K^{.,0} dimensionless, the others proportional to h).
 *   host_out  caller-owned host buffer of n doubles; n must be >= (2nx-1)(2ny-1)
 * Synchronous. Errors: SG_EINVAL, SG_ECUDA.
 */
sg_status sg_kernel_tables(const sg_plan *plan, int patch, int which, double *host_out, size_t n);

/*
 * Enqueue one force solve on `stream` (plans with z == 0; use sg_force3 for z != 0).
 *   sigma       device pointer, ncells elements (sigma0 per cell)
 *   deltax/y    device pointers, ncells elements each; read only for
 *               SG_SLOPES_CALLER, otherwise may be NULL
 *   fx, fy      device pointers, ncells elements each, written at leaf cells
 * Pointers must be aligned to their element size. Input and output buffers must
 * not overlap. The call returns once the work is enqueued; the caller
 * synchronises the stream before reading fx, fy.
 * Errors: SG_EINVAL (null plan or pointer, wrong device current), SG_ECUDA.
 */
sg_status sg_force(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay,
                   void *fx, void *fy, void *stream);

/*
 * Fx, Fy and Fz (enqueued on `stream`, buffers as for sg_force plus fz).
 * For a plan with z != 0 the targets are the points (xc, yc, z) above the leaf
 * cell centres and all three components come from the off-plane cell
 * integrals (Section 2): K^{z,0} = integral of (zbar - z)/r^3 = -dd atan(uv/(z r)),
 * K^{z,x} = (x - xc) K^{z,0} - z K^{x,0}, K^{z,y} = (y - yc) K^{z,0} - z K^{y,0};
 * a hierarchy (or masked patch) takes each patch's own convolution with its
 * height-z tables plus the cross-patch sum: the corner form of the off-plane
 * antiderivatives in FP64 (every pair in FP64 plans; the near cells in FP32
 * plans, whose far cells take Gauss-Legendre quadrature of the cell integrals).
 * For a z = 0 plan Fx, Fy are those of sg_force and Fz is the limit from
 * above the plane, -2 pi G sigma0 of the target's own cell (the other cells'
 * normal forces vanish in the plane). Errors: as sg_force.
 */
sg_status sg_force3(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx, void *fy,
                    void *fz, void *stream);

/*
 * Mid-plane potential (Section 2: Phi(x, y, 0) = -G times the integral of
 * K(xbar - x, ybar - y, 0) sigma with K = 1/r, the singular kernel integral
 * whose gradient gives the force) at every cell centre of a plan in the plane
 * (z == 0): one unmasked patch, with the plan's slope mode (central slopes are
 * formed in the row transform here), or a hierarchy (patches, masks) on either
 * path of its plan (level convolutions, or each patch's own convolution plus
 * the cross-patch direct sum: the corner form in FP64 plans, FP64 near cells
 * and a moment expansion of far cells in FP32 plans), summed over the leaf
 * cells as for sg_force (the output at covered cells is unspecified):
 *   Phi(t) = -G sum_i [sigma0_i P^0_i(t) + deltax_i P^x_i(t) + deltay_i P^y_i(t)],
 *   P^0, P^x, P^y = integrals over cell i of 1/r, (xbar - xc_i)/r, (ybar - yc_i)/r,
 * from the antiderivatives u ln(v + r) + v ln(u + r) and (v r + u^2 ln(v + r))/2
 * (finite everywhere, the own cell included). The first call on a plan builds
 * its three FP64-built potential spectra synchronously (legacy default
 * stream); later calls only enqueue on `stream`.
 *   sigma, deltax, deltay  as for sg_force;  phi  device pointer, ncells elements
 * Errors: SG_EINVAL (off the plane, null or misaligned pointer, missing caller
 * slopes), SG_ENOMEM, SG_ECUDA.
 */
sg_status sg_potential(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *phi,
                       void *stream);

/*
 * The same solve with HOST buffers, waiting for `stream` before it returns:
 * the inputs are copied to the plan's device staging buffers and sg_force runs
 * on `stream`. Fx, Fy are copied back, or, for a single in-plane patch whose
 * Fx, Fy buffers are page-locked (pinned, so mapped into the device address
 * space), written in place by the inverse row pass over the CPU-GPU link; when
 * its input buffers are pinned too, the forward row pass reads them in place
 * (no staging copy). Host buffers may be pageable or pinned.
 * Errors: as sg_force, plus SG_ENOMEM if the staging buffers cannot be allocated.
 */
sg_status sg_force_host(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay,
                        void *fx, void *fy, void *stream);

/*
 * A host-buffer solve in two halves (not in the paper: a host-side interface).
 * sg_force_host_async enqueues on `stream` the copies of the inputs into the
 * plan's device staging buffers, the solve, the copies of Fx, Fy back (all
 * transfers on the copy engines, even for pinned buffers, so that the SMs stay
 * free for other solves) and a copy of the workspace's error word into a
 * pinned word of the plan, and returns without waiting; the host buffers must
 * stay valid and untouched until sg_plan_wait(plan, stream) returns, which
 * waits for `stream` and then reports that error word (SG_ETIMEOUT if a
 * kernel's bounded wait ran out, clearing it; else SG_OK). Solves on two plans
 * (each with its own workspace and staging) and two streams overlap one
 * solve's transfers over the CPU-GPU link with the other's transforms. For
 * pinned buffers the copies are asynchronous; pageable ones are copied
 * synchronously. sg_force_host (in-place transfers for a single in-plane patch,
 * the lower latency of one solve) also reads the error word this way.
 * Errors: as sg_force_host (sg_force_host_async); SG_EINVAL for a null plan,
 * SG_ECUDA, SG_ETIMEOUT (sg_plan_wait).
 */
sg_status sg_force_host_async(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay,
                              void *fx, void *fy, void *stream);
sg_status sg_plan_wait(sg_plan *plan, void *stream);

/*
 * Bounded waits (not in the paper). Kernels that wait for bulk copies into
 * shared memory (the column passes' kernel spectra, the FP32 direct sum's
 * source tiles) give up after a number of attempts, record the failure in the
 * workspace's device error word, wait for their copies in flight (with the
 * default limit) and return early; the solve's outputs are then invalid.
 *
 * sg_plan_set_wait_limit sets the attempts of the solves of `plan` enqueued
 * from then on (a batch keeps the limit in force when it was created): tries
 * >= 0 attempts (0 gives up at once: a test of the error path), -1 the
 * default (far above any real copy time). Host only. Errors: SG_EINVAL.
 *
 * sg_plan_check_error waits for all work on the device, then reads and clears
 * the error word of the plan's own workspace (the one sg_force uses):
 * SG_ETIMEOUT if a wait ran out since the last check, else SG_OK. The host
 * entry points (sg_force_host) check it themselves; requests of a server
 * report it as their result (sg_poll / sg_wait: SG_ETIMEOUT).
 */
sg_status sg_plan_set_wait_limit(sg_plan *plan, int tries);
sg_status sg_plan_check_error(sg_plan *plan);

/*
 * Per-stage device timers (tracing). With timing enabled, every sg_force on the
 * plan records CUDA events around each kernel on the call's stream;
 * sg_plan_get_timing waits for the last call's events and writes the summed
 * milliseconds of its stages to ms[0..5]: 0 row transforms (forward), 1 column
 * transforms with the spectral multiply, 2 row transforms (inverse), 3 corner
 * weights, 4 cross-patch direct sum, 5 composite AMR sources. n must be >= 6.
 * Timing adds two event records per stage; it is off by default.
 */
sg_status sg_plan_set_timing(sg_plan *plan, int enable);
sg_status sg_plan_get_timing(sg_plan *plan, double *ms, int n);

/*
 * Allocation-free direct force sum on one uniform grid, FP32. The paper has no
 * counterpart for this entry point: it computes the same sum as sg_force on a
 * single nx x ny patch with caller slopes (or order 0 when deltax and deltay
 * are both NULL), by direct summation over the grid corners, for callers that
 * cannot let a library allocate device memory (an application that owns the
 * whole device budget and passes libraries only its own buffers, or a
 * time-step loop that must not pay cudaMalloc's latency and implicit
 * synchronisation). No plan is needed and nothing is allocated: the one
 * intermediate (the corner weights, 16 bytes per corner) lives in a fixed
 * array compiled into the library, sized for at most 512 x 512 cells
 * (513^2 corners, 4.2 MB), which every GPU that loads the library holds until
 * the process exits.
 *   nx, ny      cells, 1..512 each (SG_EINVAL beyond, with sg_last_error set)
 *   h, G        cell width (> 0) and gravitational constant
 *   sigma, deltax, deltay, fx, fy
 *               caller-owned device arrays of nx*ny floats, row-major [y][x];
 *               deltax and deltay both NULL or both non-NULL
 *   stream      cudaStream_t (NULL = legacy default stream); the call enqueues
 *               two kernels and returns
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. Every call shares the array and overwrites what it uses, so calls
 * whose work overlaps on the GPU race and give wrong results; serialise them
 * (one stream, or events between streams). Cost O((nx ny)^2).
 */
sg_status sg_direct_force_static(int nx, int ny, double h, double G, const float *sigma, const float *deltax,
                                 const float *deltay, float *fx, float *fy, void *stream);

/* ------------------------------------------------------------------------
 * Zone-by-zone hierarchies (Section 2 and Fig. 1: Berger-Oliger refinement,
 * each refined zone split into four children; the ILR and VLR hierarchies of
 * Section 4 are of this kind). A hierarchy is the list of its zones: level l
 * (0 = the coarsest grid of nx0 x ny0 zones of width h0 with lower-left corner
 * (x0, y0); the paper's L is l + 1) and the zone's column ix and row iy on the
 * level-l grid, zone (l, ix, iy) spanning [x0 + ix h_l, x0 + (ix + 1) h_l] x
 * [y0 + iy h_l, y0 + (iy + 1) h_l] with h_l = h0 / 2^l. A zone is a leaf when
 * none of its children is listed; the force acts on and is summed over the
 * leaf zones (Eq. eqnXforce2).
 *
 * Rules: 0 <= level < 12, 0 <= ix < nx0 2^level, 0 <= iy < ny0 2^level; no
 * zone is listed twice; every zone of level >= 1 has its parent
 * (level - 1, ix / 2, iy / 2) and its three siblings listed; nx0, ny0 >= 1,
 * h0 > 0, the finest level spans at most 2^22 zones per axis.
 *
 * The library lays the zones out as masked patches (one or more per level,
 * each at most 2048 zones per side and inside one patch of the level below)
 * and solves them with the same FFT convolutions and cross-patch direct sum
 * as a patch hierarchy.
 * ------------------------------------------------------------------------ */
typedef struct {
    int nx0, ny0;               /* level-0 grid, zones per axis */
    double x0, y0;              /* lower-left corner of the level-0 grid */
    double h0;                  /* level-0 zone width */
    int64_t nzones;             /* zones listed, >= 1 */
    const int32_t *level;       /* [nzones] host arrays */
    const int32_t *ix;
    const int32_t *iy;
} sg_zones;

/*
 * Create a plan for a zone list (host memory, read during the call only).
 * G, slope_mode (SG_SLOPES_NONE or SG_SLOPES_CALLER), cross_mode (an
 * sg_cross_mode), prec and hbm_budget as for sg_plan_create. Errors: SG_EINVAL (rules above, with sg_last_error
 * naming the first offending zone), SG_EBUDGET, SG_ENOMEM, SG_ECUDA.
 */
sg_status sg_plan_create_zones(const sg_zones *zones, double G, int slope_mode, int cross_mode, sg_precision prec,
                               size_t hbm_budget, sg_plan **out);

/*
 * Enqueue one solve of a zone plan on `stream`. sigma, deltax, deltay, fx, fy
 * are device arrays of nzones elements in the order of the zone list (double
 * for SG_FP64, float for SG_FP32); deltax, deltay are read for
 * SG_SLOPES_CALLER only. Values at non-leaf zones are ignored on input; fx, fy
 * receive the force at every leaf zone and 0 at non-leaf zones.
 * Errors: SG_EINVAL (not a zone plan, null or misaligned pointer), SG_ECUDA.
 */
sg_status sg_force_zones(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *fx,
                         void *fy, void *stream);

/*
 * The mid-plane potential of a zone plan (sg_potential's sum, Section 2's
 * K = 1/r integral over the leaf cells) on zone-ordered arrays: sigma, deltax,
 * deltay as for sg_force_zones; phi (nzones elements) receives the potential
 * at every leaf zone and 0 at non-leaf zones, on either path of the plan. The
 * first call builds the potential spectra synchronously. Errors: SG_EINVAL (not
 * a zone plan, null or misaligned pointer, missing caller slopes), SG_ENOMEM,
 * SG_ECUDA.
 */
sg_status sg_potential_zones(sg_plan *plan, const void *sigma, const void *deltax, const void *deltay, void *phi,
                             void *stream);

/*
 * Index of every zone in the plan's patch layout (the field arrays of
 * sg_force): host_out[k] for zone k, n >= nzones. Synchronous.
 */
sg_status sg_plan_zone_slots(const sg_plan *plan, int64_t *host_out, int64_t n);

/*
 * Read zone records of the paper's Table 10 form (Appendix A): one row of
 * ncols >= 6 doubles per zone, row-major, columns ID, x_c, y_c, L, P, EL
 * (further columns, the neighbours LN, DN, RN, UN, are not read). IDs are
 * 1..n in row order; L >= 1 is the paper's level (level = L - 1); P is the
 * parent's ID (0 on L = 1); EL = 1 marks a leaf. The centre must lie within a
 * quarter zone width of a zone centre of its level on the grid (nx0, ny0, x0,
 * y0, h0) (printed centres are rounded). Writes level, ix, iy (caller arrays
 * of n int32) after checking that every parent is the zone containing its
 * child one level up and that EL is 1 exactly for the zones nobody names as
 * parent. Host only. Errors: SG_EINVAL (sg_last_error names the record).
 */
sg_status sg_zones_from_records(int64_t n, int ncols, const double *records, int nx0, int ny0, double x0,
                                double y0, double h0, int32_t *level, int32_t *ix, int32_t *iy);

/*
 * Links of a valid zone list (host only), the remaining columns of the record
 * form: parent[k] = 1-based index of zone k's parent (0 on level 0); leaf[k] =
 * 1 for leaf zones; neighbours[4k + s] for sides s = left, down, right, up =
 * 1-based index of the zone across that side: the zone of the same level if
 * listed, else the listed coarser zone containing the point just across the
 * side's midpoint; 0 at the domain boundary. Any output may be NULL.
 * Errors: SG_EINVAL.
 */
sg_status sg_zones_links(const sg_zones *zones, int64_t *parent, uint8_t *leaf, int64_t *neighbours);

/* ------------------------------------------------------------------------
 * Launch-shape tuning (not in the paper). The uniform-patch passes come in
 * three compiled launch shapes per padded length: half, the measured default
 * and twice the default number of row sequences (forward and inverse row
 * passes) or columns (column passes) per CTA, where shared memory and CTA size
 * allow. A process-wide table, initially the defaults, selects one per
 * (precision, padded length); results are bit-identical under every shape
 * (only the grouping of sequences into CTAs changes). Solves read the table
 * when they enqueue (a graph captures the shapes in force at capture).
 *   shape[4]: 0 forward row pass, 1 inverse row pass, 2 column pass,
 *             3 central-slope column pass; 0 in sg_tune_set = the default.
 * ------------------------------------------------------------------------ */

/* Shapes in force for `precision` (SG_FP64 / SG_FP32) and padded length `pad`
 * (64 ... 4096, a power of two). Host only. Errors: SG_EINVAL. */
sg_status sg_tune_get(int precision, int pad, int *shape);

/* Select shapes (each 0 or one of the compiled candidates; SG_EINVAL names the
 * first other value). Host only. */
sg_status sg_tune_set(int precision, int pad, const int *shape);

/* Time every candidate of every pass on a square patch of each padded length
 * min_pad ... max_pad (powers of two; caller slopes for the row and column
 * passes, central slopes for the central column pass), median of `reps`
 * solves after one warm-up, one pass at a time in order, and keep the fastest.
 * best_ms (NULL or one entry per length) receives the median solve time with
 * the chosen shapes. Synchronous on the current device; allocates temporary
 * plans and buffers. Errors: SG_EINVAL, SG_ENOMEM, SG_ECUDA. */
sg_status sg_autotune(int precision, int min_pad, int max_pad, int reps, double *best_ms);

/* Tune the cross-patch direct sum of one plan (hierarchies on the direct
 * path; a no-op returning *best_ms = 0 for other plans): the source-tile
 * ranges per target block (the plan's value, a half or a quarter of it) and,
 * for FP32 plans, the CTAs of the persistent far-field launch (1, 2, 3, 4, 6
 * or 8 per SM), each timed as the median of `reps` solves on zero fields with
 * the plan's own workspace; the fastest pair stays in the plan. The split only
 * regroups the FP64 partial sums of the far field (results agree to FP64
 * rounding; the far-field grid changes nothing). Synchronous; call with no
 * solve of the plan in flight and before capturing the plan into a batch.
 * sg_plan_direct_shape reads the pair. best_ms may be NULL. Errors: SG_EINVAL,
 * SG_ENOMEM, SG_ECUDA. */
sg_status sg_plan_autotune(sg_plan *plan, int reps, double *best_ms);
sg_status sg_plan_direct_shape(const sg_plan *plan, int *nsplit, int *far_grid);

/* ------------------------------------------------------------------------
 * Batches (not in the paper): n independent solves bound to their plans and
 * caller-owned device buffers at creation and captured once into a CUDA graph,
 * so the whole batch costs one graph launch. Members that are single in-plane
 * patches run in one of two layouts:
 *   SG_BATCH_PERSISTENT  those with padded lengths up to 2048 (any mix of
 *     lengths and slope modes) in ONE persistent kernel per precision: every
 *     pass of every such member is a work item taken from a counter, column
 *     items waiting (bounded) for their member's row items and inverse row
 *     items for its column items;
 *   SG_BATCH_GROUPED  members of one precision, padded lengths and slope
 *     handling form a group; each pass of a group is one launch of that pass's
 *     kernel over all its members; groups run as concurrent graph branches.
 * SG_BATCH_AUTO (sg_batch_create) captures both and keeps the one that replays
 * faster (a median of three replays each, run on the bound buffers during
 * creation: their outputs are written then). Other members (hierarchies,
 * off-plane plans, 4096-point transforms, a group of one) run as graph
 * branches beside them, each on its own workspace. The buffers stay bound:
 * refill them and launch again. Results are bit-for-bit those of sg_force on
 * the same inputs, in either layout.
 * ------------------------------------------------------------------------ */
typedef struct sg_batch sg_batch;

typedef enum { SG_BATCH_AUTO = 0, SG_BATCH_PERSISTENT = 1, SG_BATCH_GROUPED = 2 } sg_batch_mode;

/* plans, sigma, fx, fy: arrays of n entries; deltax, deltay: arrays of n
 * entries (entries used for SG_SLOPES_CALLER plans) or NULL. The buffers are
 * device memory, or page-locked host memory (mapped into the device address
 * space: read and written in place by the kernels). Capture runs on internal
 * streams; with SG_BATCH_AUTO the candidate layouts are replayed during
 * creation (synchronously), otherwise nothing executes until sg_batch_launch.
 * sg_batch_create is sg_batch_create_mode with SG_BATCH_AUTO. Errors:
 * SG_EINVAL (also an unknown mode), SG_ENOMEM, SG_ECUDA. */
sg_status sg_batch_create(int n, sg_plan *const *plans, const void *const *sigma, const void *const *deltax,
                          const void *const *deltay, void *const *fx, void *const *fy, sg_batch **out);
sg_status sg_batch_create_mode(int n, sg_plan *const *plans, const void *const *sigma, const void *const *deltax,
                               const void *const *deltay, void *const *fx, void *const *fy, int mode,
                               sg_batch **out);

/* Enqueue the whole batch on `stream` (one graph launch). */
sg_status sg_batch_launch(sg_batch *batch, void *stream);

/* Release the batch's graph and workspaces (synchronises the device). NULL is a no-op. */
sg_status sg_batch_destroy(sg_batch *batch);

/* Wait for all work on the device, then read and clear the device error words
 * of the batch's workspaces: SG_ETIMEOUT if a bounded wait ran out in one of
 * its kernels since the last check (see sg_plan_set_wait_limit), else SG_OK. */
sg_status sg_batch_check_error(sg_batch *batch);

/* Kernel launches one sg_batch_launch replays (1 for a persistent batch of
 * single patches of one precision). Errors: SG_EINVAL (NULL batch or out). */
sg_status sg_batch_launches(const sg_batch *batch, int *out);

/* The layout the batch runs (SG_BATCH_PERSISTENT or SG_BATCH_GROUPED) and, for
 * SG_BATCH_AUTO, the median replay times of both candidates in milliseconds
 * (0 otherwise); ms_persistent, ms_grouped may be NULL. Errors: SG_EINVAL. */
sg_status sg_batch_layout(const sg_batch *batch, int *mode, double *ms_persistent, double *ms_grouped);

/* ------------------------------------------------------------------------
 * Request server (continuous batching on one GPU; not in the paper).
 *
 * sg_submit queues a solve (a plan plus caller-owned device buffers, as for
 * sg_force) and returns at once. A worker thread admits queued requests in
 * arrival order while one of max_inflight slots is free and the per-request
 * workspace (sg_plan_info.scratch_bytes) fits in what remains of hbm_budget
 * (0 = no limit); each admitted request gets its own workspace from the
 * server's stream-ordered memory pool and runs on its slot's stream, so
 * requests arriving while others run start as slots and memory free up and
 * overlap on the device. When the head of the queue is a single in-plane
 * patch, queued requests with the same padded lengths, precision and slope
 * handling that fit the budget join it (up to the group limit, 16 by default):
 * they run on its slot, each with its own workspace, and each pass of the
 * convolution is one launch over all of them (the batches' grouped launches).
 * Plans stay resident and may be shared by many requests; a result is
 * bit-for-bit the same alone, grouped and in any mix. Completion
 * is observed on the host (a stream host function); nothing waits on the GPU.
 * The caller keeps the plan and the buffers alive until the request finished,
 * and must not destroy a plan with requests in flight. The server is
 * thread-safe. Latency = completion time of the request's GPU work minus its
 * submission time (host steady clock).
 * ------------------------------------------------------------------------ */
typedef struct sg_server sg_server;

typedef struct {
    uint64_t submitted, completed, failed, cancelled, rejected;
    int64_t queued, running;        /* right now */
    int64_t bytes_in_use, peak_bytes;
    int64_t latency_count;          /* completed requests the latencies cover */
    double latency_p50_ms, latency_p99_ms, latency_mean_ms;
    uint64_t groups_started;        /* grouped admissions so far */
    uint64_t grouped_requests;      /* requests run in them */
} sg_server_stats;

/* Create a server on the current device. max_inflight: 1..256 concurrent
 * requests (one stream each). Errors: SG_EINVAL, SG_ENOMEM, SG_ECUDA. */
sg_status sg_server_create(size_t hbm_budget, int max_inflight, sg_server **out);

/* Cancel queued requests, wait for running ones, release everything. NULL is a no-op. */
sg_status sg_server_destroy(sg_server *server);

/* Most requests admitted together as one group (1..16; 1 admits every request
 * alone). Applies to admissions from then on. Errors: SG_EINVAL. */
sg_status sg_server_set_group_limit(sg_server *server, int max_members);

/* Queue one solve; *ticket identifies it. SG_EBUDGET (rejected) if its workspace
 * alone exceeds the budget; SG_EINVAL for null pointers, missing caller slopes or
 * a plan of another device. */
sg_status sg_submit(sg_server *server, sg_plan *plan, const void *sigma, const void *deltax, const void *deltay,
                    void *fx, void *fy, uint64_t *ticket);

/* Non-blocking. SG_EBUSY while queued or running; SG_OK once finished, with
 * *result the solve's status (SG_ECANCELLED if cancelled) and *latency_ms its
 * latency; the ticket is then retired (SG_ENOTFOUND afterwards, or for an
 * unknown ticket). result and latency_ms may be NULL. */
sg_status sg_poll(sg_server *server, uint64_t ticket, sg_status *result, double *latency_ms);

/* As sg_poll but waits up to timeout_ms; SG_ETIMEOUT if the request has not
 * finished by then (it keeps running and can be waited for again). */
sg_status sg_wait(sg_server *server, uint64_t ticket, double timeout_ms, sg_status *result, double *latency_ms);

/* Cancel a request that has not started (SG_OK); SG_EBUSY if it is running. */
sg_status sg_cancel(sg_server *server, uint64_t ticket);

/* Counters and latency percentiles over the requests completed so far (the
 * latency samples are cleared afterwards when reset_latencies != 0). */
sg_status sg_server_get_stats(sg_server *server, sg_server_stats *out, int reset_latencies);

/* ------------------------------------------------------------------------
 * Pipe calibration (not in the paper): the arithmetic peaks the roofline
 * fractions of the direct sum and the transforms divide by, measured on the
 * current device (every SM, 8 CTAs x 256 threads each, independent chains per
 * thread, best of five timed launches after a warm-up).
 * ------------------------------------------------------------------------ */
typedef enum {
    SG_PEAK_FP64_FMA = 0,   /* FP64 fused multiply-add, flop/s (2 per FMA) */
    SG_PEAK_FP32_FMA = 1,   /* FP32 fused multiply-add, flop/s (2 per FMA) */
    SG_PEAK_FP32_LG2 = 2    /* FP32 base-2 logarithm (special-function unit), results/s */
} sg_peak_kind;

/* Measure one peak (synchronous on the current device; allocates and frees a
 * small output buffer). Errors: SG_EINVAL (kind, NULL out), SG_ECUDA. */
sg_status sg_alu_peak(int kind, double *ops_per_s);

/* Static, human-readable name of a status. */
const char *sg_strerror(sg_status status);

/* Message of the last error reported on the calling thread ("" if none). */
const char *sg_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int sg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
