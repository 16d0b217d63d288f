// The persistent batch kernel (see batch_run.cuh), included by
// batch_run_f32.cu and batch_run_f64.cu.
#pragma once
#include "batch_run.cuh"

namespace sgk {

// dynamic shared memory of one item of each kind at padded length p
template <typename T>
__host__ __device__ constexpr int batch_row_smem(int) { return spad_size<cplx_t<T>>(BATCH_MAX_PAD) * (int)sizeof(cplx_t<T>); }
template <typename T>
__host__ __device__ constexpr int batch_edge_smem(int p) { return spad_size<cplx_t<T>>(p) * (int)sizeof(cplx_t<T>); }

template <typename T, int PY>
constexpr int batch_col_smem_t() { return col_smem_bytes<T, PY, batch_cb(PY), 6>(); }

template <typename T>
inline int batch_smem(int px, int py)
{
    int c = 0;
    switch (py) {
    case 64: c = batch_col_smem_t<T, 64>(); break;
    case 128: c = batch_col_smem_t<T, 128>(); break;
    case 256: c = batch_col_smem_t<T, 256>(); break;
    case 512: c = batch_col_smem_t<T, 512>(); break;
    case 1024: c = batch_col_smem_t<T, 1024>(); break;
    case 2048: c = batch_col_smem_t<T, 2048>(); break;
    default: return -1;
    }
    const int r = batch_row_smem<T>(px), e = batch_edge_smem<T>(py);
    return c > r ? (c > e ? c : e) : (r > e ? r : e);
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Each body is called through a function of its own (not inlined), so that
// every body keeps the register allocation it has in its pass kernel instead
// of sharing one with every other body and length of the batch.
template <typename T, int P>
__device__ __noinline__ void batch_rowf(const row_fwd_args<T> &a, int bx, int f, const cplx_t<T> *tw)
{
    row_fwd_body<T, P, batch_nb(P), BATCH_THREADS>(a, bx, f, tw);
}
template <typename T, int P>
__device__ __noinline__ void batch_edge(const edge_args<T> &a, const cplx_t<T> *tw)
{
    edge_body<T, P, BATCH_THREADS>(a, tw);
}
template <typename T, int P>
__device__ __noinline__ void batch_colc(const col_args<T> &a, int bx, int qx, const cplx_t<T> *tw, int *err)
{
    col_central_body<T, P, batch_cb(P), BATCH_THREADS, true>(a, bx, qx, tw, err);
}
template <typename T, int P>
__device__ __noinline__ void batch_col(const col_args<T> &a, int bx, int qx, int nf, const cplx_t<T> *tw, int *err)
{
    col_body<T, P, batch_cb(P), BATCH_THREADS, 2, true>(a, bx, qx, nf, tw, err);
}
template <typename T, int P>
__device__ __noinline__ void batch_rowi(const row_inv_args<T> &a, int bx, int o, const cplx_t<T> *tw)
{
    row_inv_body<T, P, batch_nb(P), BATCH_THREADS, true>(a, bx, o, tw);
}

template <typename T, int P>
__device__ __forceinline__ void batch_item_len(const batch_item &it, const batch_member<T> &m, int *err)
{
    for (int t = 0; t < it.nt; ++t) {
        if (t > 0) __syncthreads();  // the previous tile's use of shared memory is over
        const int bx = it.bx + t;
        switch (it.kind) {
        case BI_ROWF: batch_rowf<T, P>(m.rf, bx, it.f, m.twx); break;
        case BI_EDGE: batch_edge<T, P>(m.ed, m.twy); break;
        case BI_COL:
            if (m.central) batch_colc<T, P>(m.col, bx, m.qx, m.twy, err);
            else batch_col<T, P>(m.col, bx, m.qx, m.nf_cols, m.twy, err);
            break;
        default: batch_rowi<T, P>(m.ri, bx, it.f, m.twx); break;
        }
    }
}

template <typename T>
__device__ __forceinline__ void batch_run_item(const batch_item &it, const batch_member<T> &m, int *err)
{
    // row items run at the x length, column and edge items at the y length
    const int p = (it.kind == BI_ROWF || it.kind == BI_ROWI) ? m.px : m.py;
    switch (p) {
    case 64: batch_item_len<T, 64>(it, m, err); break;
    case 128: batch_item_len<T, 128>(it, m, err); break;
    case 256: batch_item_len<T, 256>(it, m, err); break;
    case 512: batch_item_len<T, 512>(it, m, err); break;
    case 1024: batch_item_len<T, 1024>(it, m, err); break;
    default: batch_item_len<T, 2048>(it, m, err); break;
    }
}

// ctl: [0] the item counter, [1 .. nmem] forward items done per member,
// [1 + nmem .. 2 nmem] column items done per member (all zero at launch).
// Thread 0 takes the CTA's next item while the current one runs (its atomic's
// round trip then overlaps the work); a CTA holding an item it has not started
// never blocks another, since that item's index exceeds the one it works on,
// so the lowest unfinished item always runs.
template <typename T>
__global__ void __launch_bounds__(BATCH_THREADS, sizeof(T) == 4 ? BATCH_MIN_BLOCKS_F32 : 1) k_batch_run(
    const batch_item *__restrict__ items, int nitems, const batch_member<T> *__restrict__ members, int nmem,
    int *__restrict__ ctl, int *err, int tries)
{
    __shared__ int s_item;
    int next = 0;
    if (threadIdx.x == 0) next = atomicAdd(&ctl[0], 1);
    for (;;) {
        __syncthreads();  // the previous item's use of shared memory is over
        if (threadIdx.x == 0) s_item = next;
        __syncthreads();
        const int i = s_item;
        if (i >= nitems) break;
        if (threadIdx.x == 0) next = atomicAdd(&ctl[0], 1);
        const batch_item it = items[i];
        const batch_member<T> &m = members[it.member];
        bool ok = true;
        if (it.kind == BI_COL || it.kind == BI_ROWI) {
            if (threadIdx.x == 0) {
                const int *cnt = it.kind == BI_COL ? &ctl[1 + it.member] : &ctl[1 + nmem + it.member];
                const int need = it.kind == BI_COL ? m.need_fwd : m.need_col;
                for (int k = 0; ld_acquire_gpu(cnt) < need; ++k) {
                    if (k >= tries) {
                        ok = false;
                        atomicExch(err, 1);
                        break;
                    }
                    __nanosleep(256);
                }
            }
            ok = !__syncthreads_or(!ok);
        }
        if (ok) batch_run_item<T>(it, m, err);
        __syncthreads();
        if (threadIdx.x == 0 && it.kind != BI_ROWI) {
            __threadfence();
            atomicAdd(it.kind == BI_COL ? &ctl[1 + nmem + it.member] : &ctl[1 + it.member], 1);
        }
    }
}

template <typename T>
sg_status batch_run_launch(const batch_item *items, int nitems, const batch_member<T> *members, int nmem, int *ctl,
                           int *err, int tries, int smem, int nsm, cudaStream_t st)
{
    auto kern = k_batch_run<T>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    SG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BATCH_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    int grid = nsm * per_sm;
    if (grid > nitems) grid = nitems;
    SG_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(int) * (1 + 2 * (size_t)nmem), st));
    kern<<<grid, BATCH_THREADS, smem, st>>>(items, nitems, members, nmem, ctl, err, tries);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

}  // namespace sgk
