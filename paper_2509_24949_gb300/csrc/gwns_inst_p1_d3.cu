// mixed-precision likelihood and slice-update kernels for 3 detectors.
#include "gwns_slice.cuh"

namespace gwns {
GWNS_INSTANTIATE(1, 3)
}  // namespace gwns
