// Persistent batch kernel: every pass of every member of a batch in one launch.
//
// The members are single in-plane patches of one precision with padded
// lengths up to 2048 (any mix of lengths and slope handling). Their passes are
// cut into work items: forward row groups (per field), the edge-column
// transform (central slopes), column groups, inverse row groups (per output),
// each the tile one CTA of the pass's own kernel would take, run by the same
// device body (fftconv.cuh) on 256 threads: NB = 2048 / Px row sequences per
// row item, CB = 2048 / Py columns per column item (eight elements per thread).
// The item list holds every member's forward items, then every member's column
// items, then every member's inverse items. CTAs take items from a counter; a
// column item first waits until its member's forward items (and edge item)
// are done, an inverse item until its member's column items are: per-member
// completion counters, released by the finishing CTA (barrier, fence, atomic
// add) and acquired by the waiting CTA's thread 0. A CTA only ever waits for
// items taken earlier, by CTAs that are running, so the waits end; they are
// bounded all the same (on running out: the error word, and the item is
// skipped). Results are those of the pass kernels bit for bit (same bodies,
// same arithmetic; only the grouping of sequences into CTAs differs).
#pragma once
#include "fftconv.cuh"

namespace sgk {

enum { BI_ROWF = 0, BI_EDGE = 1, BI_COL = 2, BI_ROWI = 3 };

struct batch_item {
    short kind;  // BI_*
    short nt;    // tiles: row or column groups bx .. bx + nt - 1, one after another
    int member;
    int bx;      // first row group or column group
    int f;       // field (forward rows) or output (inverse rows)
};

template <typename T>
struct batch_member {
    row_fwd_args<T> rf;
    edge_args<T> ed;
    col_args<T> col;
    row_inv_args<T> ri;
    const cplx_t<T> *twx, *twy;
    int px, py, qx;
    int nf_cols;     // fields of the generic column pass
    int central;     // central slopes formed in the spectrum
    int need_fwd;    // forward items (and the edge item) the column items wait for
    int need_col;    // column items the inverse items wait for
};

constexpr int BATCH_THREADS = 256;
// CTAs per SM the FP32 kernel is compiled for (registers: 65536 / (256 x this))
constexpr int BATCH_MIN_BLOCKS_F32 = 3;
// tiles (row or column groups) per work item: fewer items, so less of the
// per-item cost (taking an item, checking and signalling completion)
constexpr int BATCH_TILES = 4;
constexpr int BATCH_MAX_PAD = 2048;
__host__ __device__ constexpr int batch_nb(int px) { return BATCH_MAX_PAD / px; }
__host__ __device__ constexpr int batch_cb(int py) { return BATCH_MAX_PAD / py; }

// Enqueue the persistent kernel (and the reset of its counters) on `st`
// (batch_run_f32.cu / batch_run_f64.cu). items, members, ctl: device arrays.
template <typename T>
sg_status batch_run_launch(const batch_item *items, int nitems, const batch_member<T> *members, int nmem, int *ctl,
                           int *err, int tries, int smem, int nsm, cudaStream_t st);
// Dynamic shared memory of the kernel for a member of padded lengths px, py (-1 if unsupported).
int batch_run_smem(bool fp64, int px, int py);

}  // namespace sgk
