// FP64 instantiation of the step kernels.
#include "enqueue.cuh"

namespace hgks {
HGKS_INSTANTIATE(double)
}  // namespace hgks
