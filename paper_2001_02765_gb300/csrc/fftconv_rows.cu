// Forward row pass of the uniform-patch convolution (R2C with the fields
// formed) and its launch-shape variants.
#include "fftconv.cuh"

namespace sgk {
namespace {

template <typename T, int PX, int NB>
sg_status launch_rows_fwd(const field_src<T> &src, cplx_t<T> *work, int nf, const cplx_t<T> *tw, cudaStream_t st)
{
    const size_t smem = (size_t)spad_size<cplx_t<T>>(NB * PX) * sizeof(cplx_t<T>);
    auto kern = k_row_fwd<T, PX, NB, ROW_THREADS>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((src.ny + 2 * NB - 1) / (2 * NB), nf);
    kern<<<grid, ROW_THREADS, smem, st>>>(src, work, tw);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PX>
sg_status rows_fwd_px(int nb, const field_src<T> &src, cplx_t<T> *work, int nf, const cplx_t<T> *tw, cudaStream_t st)
{
    constexpr int D = row_nb_default(PX);
    constexpr int A = shape_candidate(D, 0), C = shape_candidate(D, 2);
    if (nb == D) return launch_rows_fwd<T, PX, D>(src, work, nf, tw, st);
    if constexpr (row_feasible_t<T>(PX, A)) {
        if (nb == A) return launch_rows_fwd<T, PX, A>(src, work, nf, tw, st);
    }
    if constexpr (row_feasible_t<T>(PX, C)) {
        if (nb == C) return launch_rows_fwd<T, PX, C>(src, work, nf, tw, st);
    }
    return SG_EINVAL;
}

}  // namespace

template <typename T>
sg_status rows_fwd(int px, int nb, const field_src<T> &src, cplx_t<T> *work, int nf, const cplx_t<T> *tw,
                   cudaStream_t st)
{
    SG_PAD_SWITCH(px, return (rows_fwd_px<T, PP>(nb, src, work, nf, tw, st)));
    return SG_EINVAL;
}

template sg_status rows_fwd<float>(int, int, const field_src<float> &, float2 *, int, const float2 *, cudaStream_t);
template sg_status rows_fwd<double>(int, int, const field_src<double> &, double2 *, int, const double2 *, cudaStream_t);

}  // namespace sgk
