// k_plane_prec2 (the one-field preconditioning pass on two-block clusters)
// instantiated for the radix sets of the even 2,3,5-smooth grids up to 160
// (bit r set: radix r used by the fewest-pass factorisation of n), double
// plans; any other set gets the kernel with every radix.
#include "plane.cuh"

namespace ofdft {

template <>
PlaneKernel<double> plane_prec2_kernel<double>(unsigned mask) {
  switch (mask) {
    case 0x100u: return k_plane_prec2<double, 0x100u>;
    case 0x204u: return k_plane_prec2<double, 0x204u>;
    case 0x240u: return k_plane_prec2<double, 0x240u>;
    case 0x400u: return k_plane_prec2<double, 0x400u>;
    case 0x404u: return k_plane_prec2<double, 0x404u>;
    case 0x408u: return k_plane_prec2<double, 0x408u>;
    case 0x410u: return k_plane_prec2<double, 0x410u>;
    case 0x420u: return k_plane_prec2<double, 0x420u>;
    case 0x428u: return k_plane_prec2<double, 0x428u>;
    case 0x600u: return k_plane_prec2<double, 0x600u>;
    case 0x1000u: return k_plane_prec2<double, 0x1000u>;
    case 0x1004u: return k_plane_prec2<double, 0x1004u>;
    case 0x1008u: return k_plane_prec2<double, 0x1008u>;
    case 0x1020u: return k_plane_prec2<double, 0x1020u>;
    case 0x1040u: return k_plane_prec2<double, 0x1040u>;
    case 0x1200u: return k_plane_prec2<double, 0x1200u>;
    case 0x1400u: return k_plane_prec2<double, 0x1400u>;
    case 0x10000u: return k_plane_prec2<double, 0x10000u>;
    case 0x10004u: return k_plane_prec2<double, 0x10004u>;
    case 0x10008u: return k_plane_prec2<double, 0x10008u>;
    case 0x10010u: return k_plane_prec2<double, 0x10010u>;
    case 0x10020u: return k_plane_prec2<double, 0x10020u>;
    case 0x10040u: return k_plane_prec2<double, 0x10040u>;
    case 0x10100u: return k_plane_prec2<double, 0x10100u>;
    case 0x10200u: return k_plane_prec2<double, 0x10200u>;
    case 0x10400u: return k_plane_prec2<double, 0x10400u>;
    default: return k_plane_prec2<double, kAllRadices>;
  }
}

}  // namespace ofdft
