// FP64 likelihood and slice-update kernels for 2 detectors.
#include "gwns_slice.cuh"

namespace gwns {
GWNS_INSTANTIATE(0, 2)
}  // namespace gwns
