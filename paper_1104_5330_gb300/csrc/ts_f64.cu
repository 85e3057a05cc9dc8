// Double-precision instantiation of the transport-step kernels.
#include "ts_launch.cuh"

namespace ts {
template struct Launch<double, double>;
}  // namespace ts
