// Reachability kernels for 32-bit buckets, rows of 5 to 8 16-byte chunks (16 < W <= 32).
#include "reach_kernels.cuh"

namespace vss {

bool reach_kernels_w32_hi(int nv, int L, ReachKernels* out) {
  switch (nv) {
    case 5: *out = kernels_w32<5>(L); return true;
    case 6: *out = kernels_w32<6>(L); return true;
    case 7: *out = kernels_w32<7>(L); return true;
    case 8: *out = kernels_w32<8>(L); return true;
    default: return false;
  }
}

}  // namespace vss
