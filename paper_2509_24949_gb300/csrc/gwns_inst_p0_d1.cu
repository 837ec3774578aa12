// FP64 likelihood and slice-update kernels for 1 detector.
#include "gwns_slice.cuh"

namespace gwns {
GWNS_INSTANTIATE(0, 1)
}  // namespace gwns
