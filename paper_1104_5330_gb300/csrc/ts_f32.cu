// Single-precision instantiation of the transport-step kernels, the
// tensor-core (split-TF32 and split-BF16) radial passes and the fused
// angular + radial pass.
#include "ts_fused.cuh"
#include "ts_launch.cuh"
#include "ts_tc.cuh"
#include "ts_tc_angular.cuh"

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
  k_radial_tc<KIND><<<grid1(nct), kTcThreads, sh.bytes, s>>>(p, t, Bterms, U, K, sgn, tau ? 1 : 0, mode,
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


cudaError_t launch_angular_tc(const Problem& p, const Tables<float>& t, const float* U, float* K,
                              float sgn, bool collision, cudaStream_t s) {
  static const cudaError_t e = allow_smem(k_angular_tc);  // once
  if (e != cudaSuccess) return e;
  const long long ntiles = (p.d.nblk + TcAng::BPT - 1) / TcAng::BPT;
  static int per_sm = 0, nsm = 0;
  if (!per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_angular_tc, 128, TcAng::bytes) !=
            cudaSuccess || per_sm < 1)
      per_sm = 1;
    if (nsm < 1) nsm = 1;
  }
  const int ctas = (int)std::min<long long>(ntiles, (long long)per_sm * nsm);
  k_angular_tc<<<ctas, 128, TcAng::bytes, s>>>(p, t, p.tcang, U, K, sgn, collision ? 1 : 0,
                                               ntiles);
  return cudaGetLastError();
}

bool fused_plan(const Dims& d, int n64, int* nb, int* nbuf) {
  // one chunk of all N_r blocks and two staging buffers if they fit; else one
  // buffer; else chunks of the angular phase small enough to fit
  const size_t cap = kSmemMax - 1024;
  for (int buf = 2; buf >= 1; --buf)
    for (int chunks = 1; chunks <= 4; ++chunks) {
      const int n = (d.Nr + chunks - 1) / chunks;
      if (fused_shape<float>(d, n64, n, buf).bytes <= cap) {
        *nb = n;
        *nbuf = buf;
        return true;
      }
    }
  return false;
}

template <int R, int A, int KF>
static cudaError_t fused_form(const Problem& p, const Tables<float>& t, const double* Dr64,
                              const float* U, const float* Kp, float sgn, int col, int tau,
                              int mode, float* F, float* Acc, float* Uout, float* out, float dt,
                              cudaStream_t s) {
  static const cudaError_t e = allow_smem(k_fused<R, A, KF, float, float>);  // once per kernel
  if (e != cudaSuccess) return e;
  const Dims& d = p.d;
  const FusedShape fs = fused_shape<float>(d, p.n_fp64_rows, p.tp.fnb, p.tp.fnbuf);
  const long long ntiles = (long long)d.G * d.Nt * d.Np;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const int ctas = (int)std::min<long long>(ntiles, nsm);
  k_fused<R, A, KF, float, float><<<ctas, kFusedThreads, fs.bytes, s>>>(
      p, t, Dr64, U, Kp, sgn, col, tau, mode, F, Acc, Uout, out, dt, p.tp.fnb, p.tp.fnbuf,
      ntiles);
  return cudaGetLastError();
}

template <int R, int A>
static cudaError_t fused_kf(const Problem& p, const Tables<float>& t, const double* Dr64,
                            const float* U, const float* Kp, float sgn, bool collision, int tau,
                            int mode, float* F, float* Acc, float* Uout, float* out, float dt,
                            cudaStream_t s) {
  const int col = collision ? 1 : 0;
  switch (kernel_form(p, col)) {
    case KF_QUADRATIC:
      return fused_form<R, A, KF_QUADRATIC>(p, t, Dr64, U, Kp, sgn, col, tau, mode, F, Acc, Uout,
                                            out, dt, s);
    case KF_LINEAR:
      return fused_form<R, A, KF_LINEAR>(p, t, Dr64, U, Kp, sgn, col, tau, mode, F, Acc, Uout,
                                         out, dt, s);
    default:
      return fused_form<R, A, KF_ISO>(p, t, Dr64, U, Kp, sgn, col, tau, mode, F, Acc, Uout, out,
                                      dt, s);
  }
}

cudaError_t launch_fused(const Problem& p, const Tables<float>& t, const double* Dr64,
                         const float* U, const float* Kp, float sgn, bool collision, bool tau,
                         int mode, float* F, float* Acc, float* Uout, float* out, double dt,
                         cudaStream_t s) {
  const Dims& d = p.d;
  const int ta = tau ? 1 : 0;
  // compiled line lengths for the 33 x 16^4 workload grids, the run-time form otherwise
  if (d.Nr == 33 && d.NT == 16 && d.NP == 16)
    return fused_kf<33, 16>(p, t, Dr64, U, Kp, sgn, collision, ta, mode, F, Acc, Uout, out,
                            (float)dt, s);
  return fused_kf<0, 0>(p, t, Dr64, U, Kp, sgn, collision, ta, mode, F, Acc, Uout, out,
                        (float)dt, s);
}

}  // namespace ts
