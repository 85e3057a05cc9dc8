// Single-precision instantiation of the transport-step kernels and the
// tensor-core (split-TF32) radial pass.
#include "ts_launch.cuh"
#include "ts_tc.cuh"

namespace ts {

template struct Launch<float, float>;

cudaError_t launch_radial_tc(const Problem& p, const Tables<float>& t, const float* U,
                             const float* K, float sgn, bool tau, int mode, float* F, float* Acc,
                             float* Uout, float* out, double dt, cudaStream_t s) {
  static bool init = false;
  const TcShape sh = tc_shape(p.d.Nr);
  if (!init) {
    const cudaError_t ea = allow_smem(k_radial_tc);
    if (ea != cudaSuccess) return ea;
    init = true;
  }
  const Dims& d = p.d;
  const int S = d.NT * d.NP;
  const long long nct = (long long)d.G * d.Nt * d.Np * ((S + 127) / 128);
  k_radial_tc<<<grid1(nct), 128, sh.bytes, s>>>(p, t, t.TcBhi, t.TcBlo, U, K, sgn, tau ? 1 : 0,
                                                mode, F, Acc, Uout, out, (float)dt);
  return cudaGetLastError();
}

}  // namespace ts
