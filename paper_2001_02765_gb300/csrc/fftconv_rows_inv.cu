// Inverse row pass of the uniform-patch convolution (C2R with the crop) and
// its launch-shape variants, for one solve or a batch of solves of one padded
// length.
#include "fftconv.cuh"

namespace sgk {
namespace {

template <typename T, int PX, int NB, bool BATCH>
sg_status launch_rows_inv(const row_inv_args<T> &one, const row_inv_args<T> *many, batch_shape bs, int nout,
                          const cplx_t<T> *tw, cudaStream_t st)
{
    const size_t smem = (size_t)spad_size<cplx_t<T>>(NB * PX) * sizeof(cplx_t<T>);
    auto kern = k_row_inv<T, PX, NB, ROW_THREADS, BATCH>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int ny = BATCH ? bs.maxny : one.ny;
    dim3 grid((ny + 2 * NB - 1) / (2 * NB), nout, BATCH ? bs.nmem : 1);
    SG_CUDA_TRY(sg_launch_dep(kern, grid, dim3(ROW_THREADS), smem, st, one, many, tw));
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PX, int NB>
sg_status launch_rows_inv_any(const row_inv_args<T> &one, const row_inv_args<T> *many, batch_shape bs, int nout,
                              const cplx_t<T> *tw, cudaStream_t st)
{
    if (many) return launch_rows_inv<T, PX, NB, true>(one, many, bs, nout, tw, st);
    return launch_rows_inv<T, PX, NB, false>(one, many, bs, nout, tw, st);
}

template <typename T, int PX>
sg_status rows_inv_px(int nb, const row_inv_args<T> &one, const row_inv_args<T> *many, batch_shape bs, int nout,
                      const cplx_t<T> *tw, cudaStream_t st)
{
    constexpr int D = row_nb_inv_default(PX);
    constexpr int A = shape_candidate(D, 0), C = shape_candidate(D, 2);
    if (nb == D) return launch_rows_inv_any<T, PX, D>(one, many, bs, nout, tw, st);
    if constexpr (row_feasible_t<T>(PX, A)) {
        if (nb == A) return launch_rows_inv_any<T, PX, A>(one, many, bs, nout, tw, st);
    }
    if constexpr (row_feasible_t<T>(PX, C)) {
        if (nb == C) return launch_rows_inv_any<T, PX, C>(one, many, bs, nout, tw, st);
    }
    return SG_EINVAL;
}

}  // namespace

template <typename T>
sg_status rows_inv(int px, int nb, const row_inv_args<T> &one, int nout, const cplx_t<T> *tw, cudaStream_t st,
                   const row_inv_args<T> *many, batch_shape bs)
{
    SG_PAD_SWITCH(px, return (rows_inv_px<T, PP>(nb, one, many, bs, nout, tw, st)));
    return SG_EINVAL;
}

template sg_status rows_inv<float>(int, int, const row_inv_args<float> &, int, const float2 *, cudaStream_t,
                                   const row_inv_args<float> *, batch_shape);
template sg_status rows_inv<double>(int, int, const row_inv_args<double> &, int, const double2 *, cudaStream_t,
                                    const row_inv_args<double> *, batch_shape);

}  // namespace sgk
