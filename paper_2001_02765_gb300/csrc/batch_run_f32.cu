// Persistent batch kernel, FP32 instantiation (see batch_run.cuh).
#include "batch_run.inl"

namespace sgk {

template sg_status batch_run_launch<float>(const batch_item *, int, const batch_member<float> *, int, int *, int *, int, int,
                                        int, cudaStream_t);

int batch_run_smem(bool fp64, int px, int py)
{
    if (px > BATCH_MAX_PAD || py > BATCH_MAX_PAD) return -1;
    return fp64 ? batch_smem<double>(px, py) : batch_smem<float>(px, py);
}

}  // namespace sgk
