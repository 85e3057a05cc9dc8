// The outgoing radial flux through r = R2 (Eq. Flux, App. A) and its adjoint
// seed, the objective of the differentiation workload:
//   J_R2[g] = R2^2 sum_{j,l} w_th[j] (2 pi/N_phi) sum_{k,m} Fejer_k cos(Th_k) (2 pi/N_Phi)
//             F[g][N_r-1][j][l][k][m]
// (Fejer's first rule in cos theta and cos Theta, trapezoid in phi and Phi: the
// quadrature of ts_moments, restricted to the r = R2 slab).
//  * k_outgoing_flux: one warp per angular block of the slab; the per-block
//    sums go to the grid's partJ buffer and k_flux_reduce adds them per group
//    in a fixed order (deterministic).
//  * k_flux_seed: dJ/dF for a cotangent gJ[g] -- gJ[g] times the weight at
//    r = R2, zero at every other radial node.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "ts_internal.h"

namespace {

constexpr int kFluxThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kFluxThreads)
k_outgoing_flux(ts::Dims d, const double* __restrict__ qdir, const double* __restrict__ cosT,
                const double* __restrict__ wth, const T* __restrict__ F, double* part, double R2) {
  const int S = d.NT * d.NP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nJ = (long long)d.Nt * d.Np;
  const long long q = blockIdx.x * (long long)(blockDim.x >> 5) + warp;   // (g, j, l)
  if (q >= d.G * nJ) return;
  const int g = (int)(q / nJ);
  const long long pos = q - g * nJ;
  const int j = (int)(pos / d.Np);
  const T* blk = F + (long long)g * d.S_g + (long long)(d.Nr - 1) * d.S_i + pos * S;
  double sr = 0.0;
  for (int x = lane; x < S; x += 32) {
    const int k = x / d.NP;
    sr = fma(qdir[k] * cosT[k], (double)blk[x], sr);
  }
  for (int o = 16; o; o >>= 1) sr += __shfl_xor_sync(0xffffffffu, sr, o);
  if (lane == 0) part[q] = R2 * R2 * wth[j] * (2.0 * M_PI / d.Np) * 4.0 * M_PI * sr;
}

__global__ void k_flux_reduce(ts::Dims d, const double* part, double* J) {
  __shared__ double red[kFluxThreads];
  const int g = blockIdx.x;
  const long long nJ = (long long)d.Nt * d.Np;
  double a = 0.0;
  for (long long x = threadIdx.x; x < nJ; x += blockDim.x) a += part[g * nJ + x];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) J[g] = red[0];
}

template <typename T>
__global__ void __launch_bounds__(kFluxThreads)
k_flux_seed(ts::Dims d, const double* __restrict__ qdir, const double* __restrict__ cosT,
            const double* __restrict__ wth, const double* __restrict__ gJ, T* lam, double R2) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < d.total; x += stride) {
    const long long g = x / d.S_g, rem = x - g * d.S_g;
    const int i = (int)(rem / d.S_i);
    double v = 0.0;
    if (i == d.Nr - 1) {
      const long long a = rem - (long long)i * d.S_i;          // (j, l, k, m)
      const int j = (int)(a / d.S_j);
      const int k = (int)((a % d.S_l) / d.NP);
      v = gJ[g] * R2 * R2 * wth[j] * (2.0 * M_PI / d.Np) * 4.0 * M_PI * qdir[k] * cosT[k];
    }
    lam[x] = (T)v;
  }
}

}  // namespace

extern "C" {

ts_status ts_outgoing_flux(ts_grid* g, const void* F, double* J_R2, void* stream) {
  if (!g) return ts::fail_status(TS_ERR_ARG, "grid is NULL");
  if (!F || !J_R2) return ts::fail_status(TS_ERR_ARG, "ts_outgoing_flux: NULL argument");
  if (g->desc.form != TS_FORM_ADVECTIVE)
    return ts::fail_status(TS_ERR_UNSUPPORTED, "ts_outgoing_flux: advective form only");
  if (!ts::aligned16(F)) return ts::fail_status(TS_ERR_ARG, "ts_outgoing_flux: F is not 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ts::Dims& d = g->d;
  const long long nq = (long long)d.G * d.Nt * d.Np;
  const int wpb = kFluxThreads / 32;
  const unsigned blocks = (unsigned)((nq + wpb - 1) / wpb);
  double* part = g->partJ;   // [G][2][Nt*Np]: the first G*Nt*Np slots serve here
  if (g->es == 8)
    k_outgoing_flux<double><<<blocks, kFluxThreads, 0, st>>>(d, g->t64.qdir, g->t64.cosT, g->wth,
                                                             (const double*)F, part, g->desc.R2);
  else
    k_outgoing_flux<float><<<blocks, kFluxThreads, 0, st>>>(d, g->t64.qdir, g->t64.cosT, g->wth,
                                                            (const float*)F, part, g->desc.R2);
  k_flux_reduce<<<d.G, kFluxThreads, 0, st>>>(d, part, J_R2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TS_OK : ts::cuda_status(e, "ts_outgoing_flux");
}

ts_status ts_outgoing_flux_adjoint(ts_grid* g, const double* gJ, void* lambda, void* stream) {
  if (!g) return ts::fail_status(TS_ERR_ARG, "grid is NULL");
  if (!gJ || !lambda) return ts::fail_status(TS_ERR_ARG, "ts_outgoing_flux_adjoint: NULL argument");
  if (g->desc.form != TS_FORM_ADVECTIVE)
    return ts::fail_status(TS_ERR_UNSUPPORTED, "ts_outgoing_flux_adjoint: advective form only");
  if (!ts::aligned16(lambda))
    return ts::fail_status(TS_ERR_ARG, "ts_outgoing_flux_adjoint: lambda is not 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ts::Dims& d = g->d;
  const long long blocks = std::min<long long>((d.total + kFluxThreads - 1) / kFluxThreads, 152LL * 16);
  if (g->es == 8)
    k_flux_seed<double><<<(unsigned)blocks, kFluxThreads, 0, st>>>(d, g->t64.qdir, g->t64.cosT,
                                                                   g->wth, gJ, (double*)lambda,
                                                                   g->desc.R2);
  else
    k_flux_seed<float><<<(unsigned)blocks, kFluxThreads, 0, st>>>(d, g->t64.qdir, g->t64.cosT,
                                                                  g->wth, gJ, (float*)lambda,
                                                                  g->desc.R2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TS_OK : ts::cuda_status(e, "ts_outgoing_flux_adjoint");
}

}  // extern "C"
