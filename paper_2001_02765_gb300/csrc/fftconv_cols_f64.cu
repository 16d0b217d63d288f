// Column pass, FP64 instantiation (see fftconv_cols.inl).
#include "fftconv_cols.inl"

namespace sgk {
template sg_status cols<double>(int, int, int, const col_args<double> &, int, int, const double2 *, int *,
                                cudaStream_t, const col_args<double> *, batch_shape, bool);
}  // namespace sgk
