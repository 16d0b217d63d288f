// Column pass of the uniform-patch convolution (forward column FFT, spectral
// multiply with the kernel spectra, inverse column FFT) for one, two or three
// outputs, and its launch-shape variants. Included by fftconv_cols_f32.cu and
// fftconv_cols_f64.cu, which instantiate it for one precision each.
#pragma once
#include "fftconv.cuh"

namespace sgk {
namespace {

template <typename T, int PY, int CB, int NOUT, bool BATCH>
sg_status launch_cols(const col_args<T> &one, const col_args<T> *many, batch_shape bs, int qx, int nf,
                      const cplx_t<T> *tw, int *err, cudaStream_t st, bool dep)
{
    constexpr int THREADS = CB * PY / 8;
    const size_t smem = (size_t)col_smem_bytes<T, PY, CB, NOUT == 3 ? 9 : (NOUT == 1 ? 3 : 6)>();
    auto kern = k_col_conv<T, PY, CB, THREADS, NOUT, BATCH>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((qx + CB - 1) / CB, 1, BATCH ? bs.nmem : 1);
    if (dep) SG_CUDA_TRY(sg_launch_dep(kern, grid, dim3(THREADS), smem, st, one, many, qx, nf, tw, err));
    else kern<<<grid, THREADS, smem, st>>>(one, many, qx, nf, tw, err);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

// batches are built for the force (two outputs) only
template <typename T, int PY, int CB, int NOUT>
sg_status launch_cols_any(const col_args<T> &one, const col_args<T> *many, batch_shape bs, int qx, int nf,
                          const cplx_t<T> *tw, int *err, cudaStream_t st, bool dep)
{
    if constexpr (NOUT == 2) {
        if (many) return launch_cols<T, PY, CB, NOUT, true>(one, many, bs, qx, nf, tw, err, st, dep);
    }
    if (many) return SG_EINVAL;
    return launch_cols<T, PY, CB, NOUT, false>(one, many, bs, qx, nf, tw, err, st, dep);
}

template <typename T, int PY, int NOUT>
sg_status cols_py(int cb, const col_args<T> &one, const col_args<T> *many, batch_shape bs, int qx, int nf,
                  const cplx_t<T> *tw, int *err, cudaStream_t st, bool dep)
{
    constexpr int NPL = NOUT == 3 ? 9 : (NOUT == 1 ? 3 : 6);
    constexpr int D = col_cb_default(PY);
    constexpr int A = shape_candidate(D, 0), C = shape_candidate(D, 2);
    if (cb == D) return launch_cols_any<T, PY, D, NOUT>(one, many, bs, qx, nf, tw, err, st, dep);
    if constexpr (col_feasible_t<T, PY, A, NPL>()) {
        if (cb == A) return launch_cols_any<T, PY, A, NOUT>(one, many, bs, qx, nf, tw, err, st, dep);
    }
    if constexpr (col_feasible_t<T, PY, C, NPL>()) {
        if (cb == C) return launch_cols_any<T, PY, C, NOUT>(one, many, bs, qx, nf, tw, err, st, dep);
    }
    return SG_EINVAL;
}

}  // namespace

template <typename T>
sg_status cols(int py, int cb, int nout, const col_args<T> &one, int qx, int nf, const cplx_t<T> *tw, int *err,
               cudaStream_t st, const col_args<T> *many, batch_shape bs, bool dep)
{
    if (nout == 1) {
        SG_PAD_SWITCH(py, return (cols_py<T, PP, 1>(cb, one, many, bs, qx, nf, tw, err, st, dep)));
    } else if (nout == 2) {
        SG_PAD_SWITCH(py, return (cols_py<T, PP, 2>(cb, one, many, bs, qx, nf, tw, err, st, dep)));
    } else if (nout == 3) {
        SG_PAD_SWITCH(py, return (cols_py<T, PP, 3>(cb, one, many, bs, qx, nf, tw, err, st, dep)));
    }
    return SG_EINVAL;
}

}  // namespace sgk
