// Column pass of the central-slope convolution (slope spectra formed from
// sigma's, see fftconv.cuh) with its launch-shape variants, and the edge-column
// transforms it needs.
#include "fftconv.cuh"

namespace sgk {
namespace {

template <typename T, int PY, int CB>
sg_status launch_cols_central(const cplx_t<T> *wf, cplx_t<T> *wi, const T *spec, const cplx_t<T> *edge, const T *phase,
                              int ny, int qx, const cplx_t<T> *tw, int *err, cudaStream_t st)
{
    constexpr int THREADS = CB * PY / 8;
    const size_t smem = (size_t)col_smem_bytes<T, PY, CB>();
    auto kern = k_col_conv_central<T, PY, CB, THREADS>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((qx + CB - 1) / CB);
    kern<<<grid, THREADS, smem, st>>>(wf, wi, spec, edge, phase, ny, qx, tw, err);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PY>
sg_status cols_central_py(int cb, const cplx_t<T> *wf, cplx_t<T> *wi, const T *spec, const cplx_t<T> *edge,
                          const T *phase, int ny, int qx, const cplx_t<T> *tw, int *err, cudaStream_t st)
{
    constexpr int D = col_cb_default(PY);
    constexpr int A = shape_candidate(D, 0), C = shape_candidate(D, 2);
    if (cb == D) return launch_cols_central<T, PY, D>(wf, wi, spec, edge, phase, ny, qx, tw, err, st);
    if constexpr (col_feasible_t<T, PY, A, 6>()) {
        if (cb == A) return launch_cols_central<T, PY, A>(wf, wi, spec, edge, phase, ny, qx, tw, err, st);
    }
    if constexpr (col_feasible_t<T, PY, C, 6>()) {
        if (cb == C) return launch_cols_central<T, PY, C>(wf, wi, spec, edge, phase, ny, qx, tw, err, st);
    }
    return SG_EINVAL;
}

template <typename T, int PY>
sg_status launch_edge_cols(const T *sigma, int nx, int ny, cplx_t<T> *edge, const cplx_t<T> *tw, cudaStream_t st)
{
    constexpr int THREADS = PY / 8 >= 64 ? PY / 8 : 64;
    const size_t smem = (size_t)spad_size<cplx_t<T>>(PY) * sizeof(cplx_t<T>);
    auto kern = k_edge_cols<T, PY, THREADS>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<1, THREADS, smem, st>>>(sigma, nx, ny, edge, tw);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

}  // namespace

template <typename T>
sg_status cols_central(int py, int cb, const cplx_t<T> *wf, cplx_t<T> *wi, const T *spec, const cplx_t<T> *edge,
                       const T *phase, int ny, int qx, const cplx_t<T> *tw, int *err, cudaStream_t st)
{
    SG_PAD_SWITCH(py, return (cols_central_py<T, PP>(cb, wf, wi, spec, edge, phase, ny, qx, tw, err, st)));
    return SG_EINVAL;
}

template <typename T>
sg_status edge_cols(int py, const T *sigma, int nx, int ny, cplx_t<T> *edge, const cplx_t<T> *tw, cudaStream_t st)
{
    SG_PAD_SWITCH(py, return (launch_edge_cols<T, PP>(sigma, nx, ny, edge, tw, st)));
    return SG_EINVAL;
}

template sg_status cols_central<float>(int, int, const float2 *, float2 *, const float *, const float2 *, const float *,
                                       int, int, const float2 *, int *, cudaStream_t);
template sg_status cols_central<double>(int, int, const double2 *, double2 *, const double *, const double2 *,
                                        const double *, int, int, const double2 *, int *, cudaStream_t);
template sg_status edge_cols<float>(int, const float *, int, int, float2 *, const float2 *, cudaStream_t);
template sg_status edge_cols<double>(int, const double *, int, int, double2 *, const double2 *, cudaStream_t);

}  // namespace sgk
