// Column pass of the uniform-patch convolution (forward column FFT, spectral
// multiply with the kernel spectra, inverse column FFT) for one, two or three
// outputs, and its launch-shape variants. Included by fftconv_cols_f32.cu and
// fftconv_cols_f64.cu, which instantiate it for one precision each.
#pragma once
#include "fftconv.cuh"

namespace sgk {
namespace {

template <typename T, int PY, int CB, int NOUT>
sg_status launch_cols(const cplx_t<T> *wf, cplx_t<T> *wi, const T *spec, int ny, int qx, int nf, const cplx_t<T> *tw,
                      int *err, cudaStream_t st)
{
    constexpr int THREADS = CB * PY / 8;
    const size_t smem = (size_t)col_smem_bytes<T, PY, CB, NOUT == 3 ? 9 : (NOUT == 1 ? 3 : 6)>();
    auto kern = k_col_conv<T, PY, CB, THREADS, NOUT>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((qx + CB - 1) / CB);
    kern<<<grid, THREADS, smem, st>>>(wf, wi, spec, ny, qx, nf, tw, err);
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
}

template <typename T, int PY, int NOUT>
sg_status cols_py(int cb, const cplx_t<T> *wf, cplx_t<T> *wi, const T *spec, int ny, int qx, int nf,
                  const cplx_t<T> *tw, int *err, cudaStream_t st)
{
    constexpr int NPL = NOUT == 3 ? 9 : (NOUT == 1 ? 3 : 6);
    constexpr int D = col_cb_default(PY);
    constexpr int A = shape_candidate(D, 0), C = shape_candidate(D, 2);
    if (cb == D) return launch_cols<T, PY, D, NOUT>(wf, wi, spec, ny, qx, nf, tw, err, st);
    if constexpr (col_feasible_t<T, PY, A, NPL>()) {
        if (cb == A) return launch_cols<T, PY, A, NOUT>(wf, wi, spec, ny, qx, nf, tw, err, st);
    }
    if constexpr (col_feasible_t<T, PY, C, NPL>()) {
        if (cb == C) return launch_cols<T, PY, C, NOUT>(wf, wi, spec, ny, qx, nf, tw, err, st);
    }
    return SG_EINVAL;
}

}  // namespace

template <typename T>
sg_status cols(int py, int cb, int nout, const cplx_t<T> *wf, cplx_t<T> *wi, const T *spec, int ny, int qx, int nf,
               const cplx_t<T> *tw, int *err, cudaStream_t st)
{
    if (nout == 1) {
        SG_PAD_SWITCH(py, return (cols_py<T, PP, 1>(cb, wf, wi, spec, ny, qx, nf, tw, err, st)));
    } else if (nout == 2) {
        SG_PAD_SWITCH(py, return (cols_py<T, PP, 2>(cb, wf, wi, spec, ny, qx, nf, tw, err, st)));
    } else if (nout == 3) {
        SG_PAD_SWITCH(py, return (cols_py<T, PP, 3>(cb, wf, wi, spec, ny, qx, nf, tw, err, st)));
    }
    return SG_EINVAL;
}


}  // namespace sgk
