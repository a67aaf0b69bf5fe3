// k_plane instantiated for the radix sets of the grid sizes the plane path
// serves (2,3,5-smooth n up to 160, odd or even; bit r set: radix r used by the
// fewest-pass factorisation of n), double plans.
#include "plane.cuh"

namespace ofdft {

template <>
PlaneKernel<double> plane_kernel<double>(unsigned mask) {
  switch (mask) {
    case 0x100u: return k_plane<double, 0x100u>;
    case 0x204u: return k_plane<double, 0x204u>;
    case 0x240u: return k_plane<double, 0x240u>;
    case 0x400u: return k_plane<double, 0x400u>;
    case 0x404u: return k_plane<double, 0x404u>;
    case 0x408u: return k_plane<double, 0x408u>;
    case 0x410u: return k_plane<double, 0x410u>;
    case 0x420u: return k_plane<double, 0x420u>;
    case 0x428u: return k_plane<double, 0x428u>;
    case 0x600u: return k_plane<double, 0x600u>;
    case 0x1000u: return k_plane<double, 0x1000u>;
    case 0x1004u: return k_plane<double, 0x1004u>;
    case 0x1008u: return k_plane<double, 0x1008u>;
    case 0x1020u: return k_plane<double, 0x1020u>;
    case 0x1040u: return k_plane<double, 0x1040u>;
    case 0x1200u: return k_plane<double, 0x1200u>;
    case 0x1400u: return k_plane<double, 0x1400u>;
    case 0x10000u: return k_plane<double, 0x10000u>;
    case 0x10004u: return k_plane<double, 0x10004u>;
    case 0x10008u: return k_plane<double, 0x10008u>;
    case 0x10010u: return k_plane<double, 0x10010u>;
    case 0x10020u: return k_plane<double, 0x10020u>;
    case 0x10040u: return k_plane<double, 0x10040u>;
    case 0x10100u: return k_plane<double, 0x10100u>;
    case 0x10200u: return k_plane<double, 0x10200u>;
    case 0x10400u: return k_plane<double, 0x10400u>;
    case 0x20u: return k_plane<double, 0x20u>;
    case 0x28u: return k_plane<double, 0x28u>;
    case 0x200u: return k_plane<double, 0x200u>;
    case 0x208u: return k_plane<double, 0x208u>;
    case 0x220u: return k_plane<double, 0x220u>;
    case 0x228u: return k_plane<double, 0x228u>;
    default: return k_plane<double, kAllRadices>;
  }
}

}  // namespace ofdft
