// Single-precision instantiation of the transport-step kernels.
#include "ts_launch.cuh"

namespace ts {
template struct Launch<float, float>;
}  // namespace ts
