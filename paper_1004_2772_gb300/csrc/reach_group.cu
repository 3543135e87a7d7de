// Reachability kernels with cooperative probing (groups of 2, 4 or 8 lanes
// per successor, 32-bit buckets), every row width.
#include "reach_kernels.cuh"

namespace vss {

bool reach_kernels_group(int nv, int G, ReachKernels* out) {
  if (G != 2 && G != 4 && G != 8) return false;
  switch (nv) {
    case 1: *out = kernels_group<1>(G); return true;
    case 2: *out = kernels_group<2>(G); return true;
    case 3: *out = kernels_group<3>(G); return true;
    case 4: *out = kernels_group<4>(G); return true;
    case 5: *out = kernels_group<5>(G); return true;
    case 6: *out = kernels_group<6>(G); return true;
    case 7: *out = kernels_group<7>(G); return true;
    case 8: *out = kernels_group<8>(G); return true;
    default: return false;
  }
}

}  // namespace vss
