// Inverse row pass of the uniform-patch convolution (C2R with the crop) and
// its launch-shape variants.
#include "fftconv.cuh"

namespace sgk {
namespace {

template <typename T, int PX, int NB>
sg_status launch_rows_inv(const cplx_t<T> *work, T *fx, T *fy, T *fz, int nx, int ny, const cplx_t<T> *tw,
                          cudaStream_t st)
{
    const size_t smem = (size_t)spad_size<cplx_t<T>>(NB * PX) * sizeof(cplx_t<T>);
    auto kern = k_row_inv<T, PX, NB, ROW_THREADS>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((ny + 2 * NB - 1) / (2 * NB), fz ? 3 : (fy ? 2 : 1));
    kern<<<grid, ROW_THREADS, smem, st>>>(work, fx, fy, fz, nx, ny, tw);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PX>
sg_status rows_inv_px(int nb, const cplx_t<T> *work, T *fx, T *fy, T *fz, int nx, int ny, const cplx_t<T> *tw,
                      cudaStream_t st)
{
    constexpr int D = row_nb_inv_default(PX);
    constexpr int A = shape_candidate(D, 0), C = shape_candidate(D, 2);
    if (nb == D) return launch_rows_inv<T, PX, D>(work, fx, fy, fz, nx, ny, tw, st);
    if constexpr (row_feasible_t<T>(PX, A)) {
        if (nb == A) return launch_rows_inv<T, PX, A>(work, fx, fy, fz, nx, ny, tw, st);
    }
    if constexpr (row_feasible_t<T>(PX, C)) {
        if (nb == C) return launch_rows_inv<T, PX, C>(work, fx, fy, fz, nx, ny, tw, st);
    }
    return SG_EINVAL;
}

}  // namespace

template <typename T>
sg_status rows_inv(int px, int nb, const cplx_t<T> *work, T *fx, T *fy, T *fz, int nx, int ny, const cplx_t<T> *tw,
                   cudaStream_t st)
{
    SG_PAD_SWITCH(px, return (rows_inv_px<T, PP>(nb, work, fx, fy, fz, nx, ny, tw, st)));
    return SG_EINVAL;
}

template sg_status rows_inv<float>(int, int, const float2 *, float *, float *, float *, int, int, const float2 *,
                                   cudaStream_t);
template sg_status rows_inv<double>(int, int, const double2 *, double *, double *, double *, int, int, const double2 *,
                                    cudaStream_t);

}  // namespace sgk
