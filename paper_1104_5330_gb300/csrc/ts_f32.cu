// Single-precision instantiation of the transport-step kernels and the
// tensor-core (split-TF32 and split-BF16) radial passes.
#include "ts_launch.cuh"
#include "ts_tc.cuh"

namespace ts {

template struct Launch<float, float>;

template <int KIND>
static cudaError_t radial_tc(const Problem& p, const void* Bterms, const Tables<float>& t,
                             const float* U, const float* K, float sgn, bool tau, int mode,
                             float* F, float* Acc, float* Uout, float* out, double dt,
                             cudaStream_t s) {
  static const cudaError_t e = allow_smem(k_radial_tc<KIND>);  // once per kernel
  if (e != cudaSuccess) return e;
  const TcShape sh = tc_shape<KIND>(p.d.Nr);
  const Dims& d = p.d;
  const int S = d.NT * d.NP;
  const long long nct = (long long)d.G * d.Nt * d.Np * ((S + 127) / 128);
  k_radial_tc<KIND><<<grid1(nct), 128, sh.bytes, s>>>(p, t, Bterms, U, K, sgn, tau ? 1 : 0, mode,
                                                      F, Acc, Uout, out, (float)dt);
  return cudaGetLastError();
}

cudaError_t launch_radial_tc(const Problem& p, const Tables<float>& t, const float* U,
                             const float* K, float sgn, bool tau, int mode, float* F, float* Acc,
                             float* Uout, float* out, double dt, cudaStream_t s) {
  if (p.tc == TC_BF16X3)
    return radial_tc<TC_BF16X3>(p, p.tcb16, t, U, K, sgn, tau, mode, F, Acc, Uout, out, dt, s);
  // TF32 terms: TcBlo follows TcBhi in the table block (both multiples of 128 floats)
  return radial_tc<TC_TF32X3>(p, t.TcBhi, t, U, K, sgn, tau, mode, F, Acc, Uout, out, dt, s);
}

}  // namespace ts
