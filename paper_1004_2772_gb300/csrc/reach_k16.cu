// Reachability kernels for 16-bit buckets, every row width.
#include "reach_kernels.cuh"

namespace vss {

bool reach_kernels_w16(int nv, int L, ReachKernels* out) {
  switch (nv) {
    case 1: *out = kernels_w16<1>(L); return true;
    case 2: *out = kernels_w16<2>(L); return true;
    case 3: *out = kernels_w16<3>(L); return true;
    case 4: *out = kernels_w16<4>(L); return true;
    case 5: *out = kernels_w16<5>(L); return true;
    case 6: *out = kernels_w16<6>(L); return true;
    case 7: *out = kernels_w16<7>(L); return true;
    case 8: *out = kernels_w16<8>(L); return true;
    default: return false;
  }
}

}  // namespace vss
