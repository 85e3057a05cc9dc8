// Radial pass of the hybrid grid (Sect. 5.3): first-order one-sided differences
// in r on uniform nodes, upstream of each direction, in place of the Chebyshev
// derivative; the angular passes are the spectral ones.
//
// One thread per r-line (a column (k, m) of the angular blocks at fixed
// (g, theta_j, phi_l)): consecutive threads take consecutive columns, so every
// row access of a warp is one coalesced segment. The thread walks its line from
// the inflow end (i = 0 when cos(Theta_k) > 0, i = N_r - 1 otherwise), keeping the
// upstream value in a register:
//   K_i += sgn cos(Theta_k) (U_i - U_upstream) / dr   (forward: (U_upstream - U_i)/dr),
// the inflow node (no upstream point) gets no radial term, and with held inflow
// data its rate is zero. Then the stage update of the selected mode, as in the
// spectral radial pass. Every line is read before it is written at the same
// index, so the AB2 update may write F while U is F.
#include "ts_internal.h"

namespace ts {

namespace {

template <typename T, typename C>
__device__ __forceinline__ void fd_store(int mode, long long gi, C kv, T* F, T* Acc, T* Uout,
                                         T* out, C dt) {
  switch (mode) {
    case RAD_RHS:
      out[gi] = (T)kv;
      break;
    case RAD_STAGE0:
      Acc[gi] = (T)kv;
      Uout[gi] = (T)((C)F[gi] + (C)0.5 * dt * kv);
      break;
    case RAD_STAGE1:
      Acc[gi] = (T)((C)Acc[gi] + (C)2 * kv);
      Uout[gi] = (T)((C)F[gi] + (C)0.5 * dt * kv);
      break;
    case RAD_STAGE2:
      Acc[gi] = (T)((C)Acc[gi] + (C)2 * kv);
      Uout[gi] = (T)((C)F[gi] + dt * kv);
      break;
    case RAD_STAGE3:
      F[gi] = (T)((C)F[gi] + dt / (C)6 * ((C)Acc[gi] + kv));
      break;
    case RAD_AB2:
      F[gi] = (T)((C)F[gi] + dt * ((C)1.5 * kv - (C)0.5 * (C)Acc[gi]));
      Acc[gi] = (T)kv;
      break;
    default:  // RAD_AB2_START
      F[gi] = (T)((C)F[gi] + dt * kv);
      Acc[gi] = (T)kv;
      break;
  }
}

template <typename T, typename C>
__global__ void __launch_bounds__(256)
k_radial_fd(Problem p, const C* __restrict__ cosT, const T* U, const T* Kin, C sgn, C inv_dr,
            int hold, int mode, T* F, T* Acc, T* Uout, T* out, C dt) {
  const Dims d = p.d;
  const long long S = (long long)d.NT * d.NP;
  const long long nlines = d.total / d.Nr;
  for (long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x; line < nlines;
       line += (long long)gridDim.x * blockDim.x) {
    const long long col = line % S, blk = line / S;   // blk = (g, j, l)
    const long long g = blk / ((long long)d.Nt * d.Np), jl = blk % ((long long)d.Nt * d.Np);
    const long long base = g * d.S_g + jl * d.S_l + col;
    const int k = (int)(col / d.NP);
    const C a = cosT[k];
    const bool up = a > (C)0;   // inflow at r = R1, walk outwards
    const int N = d.Nr - 1;
    const C ca = sgn * a * inv_dr;
    C prev = 0;
#pragma unroll 4
    for (int s = 0; s <= N; ++s) {
      const int i = up ? s : N - s;
      const long long gi = base + (long long)i * d.S_i;
      const C u = (C)U[gi];
      C kv = (C)Kin[gi];
      if (s > 0) kv += up ? ca * (u - prev) : ca * (prev - u);
      else if (hold) kv = 0;
      prev = u;
      fd_store<T, C>(mode, gi, kv, F, Acc, Uout, out, dt);
    }
  }
}

}  // namespace

template <typename T, typename C>
cudaError_t launch_radial_fd(const Problem& p, const Tables<C>& t, const T* U, const T* K, C sgn,
                             bool hold, int mode, T* F, T* Acc, T* Uout, T* out, double dt,
                             double dr, cudaStream_t s) {
  const long long nlines = p.d.total / p.d.Nr;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long want = (nlines + 255) / 256;
  const int ctas = (int)std::min<long long>(want, (long long)nsm * 8);
  k_radial_fd<T, C><<<ctas, 256, 0, s>>>(p, t.cosT, U, K, sgn, (C)(1.0 / dr), hold ? 1 : 0, mode,
                                         F, Acc, Uout, out, (C)dt);
  return cudaGetLastError();
}

template cudaError_t launch_radial_fd<double, double>(const Problem&, const Tables<double>&,
                                                      const double*, const double*, double, bool,
                                                      int, double*, double*, double*, double*,
                                                      double, double, cudaStream_t);
template cudaError_t launch_radial_fd<float, float>(const Problem&, const Tables<float>&,
                                                    const float*, const float*, float, bool, int,
                                                    float*, float*, float*, float*, double, double,
                                                    cudaStream_t);

}  // namespace ts
