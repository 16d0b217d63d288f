// Persistent batch kernel, FP64 instantiation (see batch_run.cuh).
#include "batch_run.inl"

namespace sgk {

template sg_status batch_run_launch<double>(const batch_item *, int, const batch_member<double> *, int, int *, int *, int, int,
                                        int, cudaStream_t);

}  // namespace sgk
