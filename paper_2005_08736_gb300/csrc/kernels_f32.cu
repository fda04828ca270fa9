// FP32 instantiation of the step kernels (deviation storage, FP64 reductions).
#include "enqueue.cuh"

namespace hgks {
HGKS_INSTANTIATE(float)
}  // namespace hgks
