// mixed-precision likelihood and slice-update kernels for 4 detectors.
#include "gwns_slice.cuh"

namespace gwns {
GWNS_INSTANTIATE(1, 4)
}  // namespace gwns
