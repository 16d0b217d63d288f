// Column pass, FP32 instantiation (see fftconv_cols.inl).
#include "fftconv_cols.inl"

namespace sgk {
template sg_status cols<float>(int, int, int, const col_args<float> &, int, int, const float2 *, int *, cudaStream_t,
                               const col_args<float> *, batch_shape, bool);
}  // namespace sgk
