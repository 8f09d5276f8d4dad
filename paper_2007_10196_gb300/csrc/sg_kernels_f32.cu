// FP32 instantiation of the kernels (WENO arithmetic in float; reductions and the
// combination sum stay FP64).
#include "sg_launch_impl.cuh"

namespace sg {

template struct Launch<float>;

}  // namespace sg
