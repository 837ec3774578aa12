// mixed-precision likelihood and slice-update kernels for 2 detectors.
#include "gwns_slice.cuh"

namespace gwns {
GWNS_INSTANTIATE(1, 2)
}  // namespace gwns
