// FP64 instantiation of the sweep kernels and their launchers.
#include "mhd_launch_impl.cuh"

namespace mhd {
MHD_INSTANTIATE_LAUNCH(double)
}  // namespace mhd
