// Reachability kernels for 32-bit buckets, rows of 1 to 4 16-byte chunks (W <= 16).
#include "reach_kernels.cuh"

namespace vss {

bool reach_kernels_w32_lo(int nv, int L, ReachKernels* out) {
  switch (nv) {
    case 1: *out = kernels_w32<1>(L); return true;
    case 2: *out = kernels_w32<2>(L); return true;
    case 3: *out = kernels_w32<3>(L); return true;
    case 4: *out = kernels_w32<4>(L); return true;
    default: return false;
  }
}

}  // namespace vss
