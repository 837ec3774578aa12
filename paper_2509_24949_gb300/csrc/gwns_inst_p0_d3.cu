// FP64 likelihood and slice-update kernels for 3 detectors.
#include "gwns_slice.cuh"

namespace gwns {
GWNS_INSTANTIATE(0, 3)
}  // namespace gwns
