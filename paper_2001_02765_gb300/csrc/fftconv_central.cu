// Column pass of the central-slope convolution (slope spectra formed from
// sigma's, see fftconv.cuh) with its launch-shape variants, and the edge-column
// transforms it needs, for one solve or a batch of solves of one padded length.
#include "fftconv.cuh"

namespace sgk {
namespace {

template <typename T, int PY, int CB, bool BATCH>
sg_status launch_cols_central(const col_args<T> &one, const col_args<T> *many, batch_shape bs, int qx,
                              const cplx_t<T> *tw, int *err, cudaStream_t st, bool dep)
{
    constexpr int THREADS = CB * PY / 8;
    const size_t smem = (size_t)col_smem_bytes<T, PY, CB, 6, col_central_nbuf<T, PY, CB>()>();
    auto kern = k_col_conv_central<T, PY, CB, THREADS, BATCH>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((qx + CB - 1) / CB, 1, BATCH ? bs.nmem : 1);
    if (dep) SG_CUDA_TRY(sg_launch_dep(kern, grid, dim3(THREADS), smem, st, one, many, qx, tw, err));
    else kern<<<grid, THREADS, smem, st>>>(one, many, qx, tw, err);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PY, int CB>
sg_status launch_cols_central_any(const col_args<T> &one, const col_args<T> *many, batch_shape bs, int qx,
                                  const cplx_t<T> *tw, int *err, cudaStream_t st, bool dep)
{
    if (many) return launch_cols_central<T, PY, CB, true>(one, many, bs, qx, tw, err, st, dep);
    return launch_cols_central<T, PY, CB, false>(one, many, bs, qx, tw, err, st, dep);
}

template <typename T, int PY>
sg_status cols_central_py(int cb, const col_args<T> &one, const col_args<T> *many, batch_shape bs, int qx,
                          const cplx_t<T> *tw, int *err, cudaStream_t st, bool dep)
{
    constexpr int D = col_cb_default(PY);
    constexpr int A = shape_candidate(D, 0), C = shape_candidate(D, 2);
    if (cb == D) return launch_cols_central_any<T, PY, D>(one, many, bs, qx, tw, err, st, dep);
    if constexpr (col_feasible_t<T, PY, A, 6>()) {
        if (cb == A) return launch_cols_central_any<T, PY, A>(one, many, bs, qx, tw, err, st, dep);
    }
    if constexpr (col_feasible_t<T, PY, C, 6>()) {
        if (cb == C) return launch_cols_central_any<T, PY, C>(one, many, bs, qx, tw, err, st, dep);
    }
    return SG_EINVAL;
}

template <typename T, int PY>
sg_status launch_edge_cols(const edge_args<T> &one, const edge_args<T> *many, batch_shape bs, const cplx_t<T> *tw,
                           cudaStream_t st)
{
    constexpr int THREADS = PY / 8 >= 64 ? PY / 8 : 64;
    const size_t smem = (size_t)spad_size<cplx_t<T>>(PY) * sizeof(cplx_t<T>);
    // a dependent launch after the row pass (see k_edge_cols)
    if (many) {
        auto kern = k_edge_cols<T, PY, THREADS, true>;
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SG_CUDA_TRY(sg_launch_dep(kern, dim3(1, 1, bs.nmem), dim3(THREADS), smem, st, one, many, tw));
    } else {
        auto kern = k_edge_cols<T, PY, THREADS, false>;
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SG_CUDA_TRY(sg_launch_dep(kern, dim3(1), dim3(THREADS), smem, st, one, many, tw));
    }
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

}  // namespace

template <typename T>
sg_status cols_central(int py, int cb, const col_args<T> &one, int qx, const cplx_t<T> *tw, int *err, cudaStream_t st,
                       const col_args<T> *many, batch_shape bs, bool dep)
{
    SG_PAD_SWITCH(py, return (cols_central_py<T, PP>(cb, one, many, bs, qx, tw, err, st, dep)));
    return SG_EINVAL;
}

template <typename T>
sg_status edge_cols(int py, const edge_args<T> &one, const cplx_t<T> *tw, cudaStream_t st, const edge_args<T> *many,
                    batch_shape bs)
{
    SG_PAD_SWITCH(py, return (launch_edge_cols<T, PP>(one, many, bs, tw, st)));
    return SG_EINVAL;
}

template sg_status cols_central<float>(int, int, const col_args<float> &, int, const float2 *, int *, cudaStream_t,
                                       const col_args<float> *, batch_shape, bool);
template sg_status cols_central<double>(int, int, const col_args<double> &, int, const double2 *, int *, cudaStream_t,
                                        const col_args<double> *, batch_shape, bool);
template sg_status edge_cols<float>(int, const edge_args<float> &, const float2 *, cudaStream_t,
                                    const edge_args<float> *, batch_shape);
template sg_status edge_cols<double>(int, const edge_args<double> &, const double2 *, cudaStream_t,
                                     const edge_args<double> *, batch_shape);

}  // namespace sgk
