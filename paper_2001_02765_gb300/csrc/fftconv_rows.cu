// Forward row pass of the uniform-patch convolution (R2C with the fields
// formed) and its launch-shape variants, for one solve or a batch of solves of
// one padded length.
#include "fftconv.cuh"

namespace sgk {
namespace {

// after_edge: launched right after the edge-column transform of a central-slope
// solve, as a dependent launch that runs beside it and waits for it at its end
// (k_row_fwd with WAIT_AT_END); otherwise the first kernel of the solve.
template <typename T, int PX, int NB, bool BATCH, bool AFTER_EDGE>
sg_status launch_rows_fwd(const row_fwd_args<T> &one, const row_fwd_args<T> *many, batch_shape bs, int nf,
                          const cplx_t<T> *tw, cudaStream_t st)
{
    const size_t smem = (size_t)spad_size<cplx_t<T>>(NB * PX) * sizeof(cplx_t<T>);
    auto kern = k_row_fwd<T, PX, NB, ROW_THREADS, BATCH, AFTER_EDGE>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int ny = BATCH ? bs.maxny : one.src.ny;
    dim3 grid((ny + 2 * NB - 1) / (2 * NB), nf, BATCH ? bs.nmem : 1);
    if (AFTER_EDGE) SG_CUDA_TRY(sg_launch_dep(kern, grid, dim3(ROW_THREADS), smem, st, one, many, tw));
    else kern<<<grid, ROW_THREADS, smem, st>>>(one, many, tw);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PX, int NB>
sg_status launch_rows_fwd_any(const row_fwd_args<T> &one, const row_fwd_args<T> *many, batch_shape bs, int nf,
                              const cplx_t<T> *tw, cudaStream_t st, bool after_edge)
{
    if (after_edge) {
        if (many) return launch_rows_fwd<T, PX, NB, true, true>(one, many, bs, nf, tw, st);
        return launch_rows_fwd<T, PX, NB, false, true>(one, many, bs, nf, tw, st);
    }
    if (many) return launch_rows_fwd<T, PX, NB, true, false>(one, many, bs, nf, tw, st);
    return launch_rows_fwd<T, PX, NB, false, false>(one, many, bs, nf, tw, st);
}

template <typename T, int PX>
sg_status rows_fwd_px(int nb, const row_fwd_args<T> &one, const row_fwd_args<T> *many, batch_shape bs, int nf,
                      const cplx_t<T> *tw, cudaStream_t st, bool after_edge)
{
    constexpr int D = row_nb_default(PX);
    constexpr int A = shape_candidate(D, 0), C = shape_candidate(D, 2);
    if (nb == D) return launch_rows_fwd_any<T, PX, D>(one, many, bs, nf, tw, st, after_edge);
    if constexpr (row_feasible_t<T>(PX, A)) {
        if (nb == A) return launch_rows_fwd_any<T, PX, A>(one, many, bs, nf, tw, st, after_edge);
    }
    if constexpr (row_feasible_t<T>(PX, C)) {
        if (nb == C) return launch_rows_fwd_any<T, PX, C>(one, many, bs, nf, tw, st, after_edge);
    }
    return SG_EINVAL;
}

}  // namespace

template <typename T>
sg_status rows_fwd(int px, int nb, const row_fwd_args<T> &one, int nf, const cplx_t<T> *tw, cudaStream_t st,
                   const row_fwd_args<T> *many, batch_shape bs, bool after_edge)
{
    SG_PAD_SWITCH(px, return (rows_fwd_px<T, PP>(nb, one, many, bs, nf, tw, st, after_edge)));
    return SG_EINVAL;
}

template sg_status rows_fwd<float>(int, int, const row_fwd_args<float> &, int, const float2 *, cudaStream_t,
                                   const row_fwd_args<float> *, batch_shape, bool);
template sg_status rows_fwd<double>(int, int, const row_fwd_args<double> &, int, const double2 *, cudaStream_t,
                                    const row_fwd_args<double> *, batch_shape, bool);

}  // namespace sgk
