// mixed-precision likelihood and slice-update kernels for 1 detector.
#include "gwns_slice.cuh"

namespace gwns {
GWNS_INSTANTIATE(1, 1)
}  // namespace gwns
