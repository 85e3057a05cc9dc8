// Radial pass of the three-zone radial grid of App. B: first-order upwind
// differences on uniform nodes in the two edge zones, Chebyshev-Gauss-Lobatto
// differentiation in the central zone; neighbouring zones share their interface
// node. The rate at an interface is the upstream zone's, and the central zone
// takes that rate at its inflow interface by the Tau method; since the
// non-radial parts of the rate are equal at the node, the Tau correction is a
// correction of the radial derivative alone:
//   d(i) = dB(i) + c T_N(x_i),   c = (dFD(b) - dB(b)) / T_N(x_b)   (central zone),
// b its inflow interface (the first central node for cos(Theta) > 0, the last
// one otherwise), dB the Chebyshev derivative on the central nodes, dFD the
// upstream zone's one-sided difference at b. The outer inflow node of each
// direction holds its data (zero rate with held inflow data), as on the hybrid
// grid of Sect. 5.3.
//
// One CTA per (g, theta_j, phi_l) and W consecutive (Theta, Phi) columns: the
// tile's lines are staged in shared memory with the central-zone matrix, one
// thread per column forms c, then every (row, column) gets its derivative, the
// radial term, the hold, and the stage update (every row is staged before any is
// written, so the pass may overwrite the array it differentiates).
#include <algorithm>

#include "ts_internal.h"

namespace ts {

namespace {

template <typename T, typename C>
__device__ __forceinline__ void zoned_store(int mode, long long gi, C kv, T* F, T* Acc, T* Uout,
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
k_radial_zoned(Problem p, const C* __restrict__ cosT, const C* __restrict__ DB,
               const C* __restrict__ tNB, int nA, int nB, C inv_h, const T* U, const T* Kin, C sgn,
               int hold, int mode, T* F, T* Acc, T* Uout, T* out, C dt, int W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nr = d.Nr, N = Nr - 1, S = d.NT * d.NP;
  const int iB0 = nA - 1, iB1 = nA - 1 + nB - 1;
  C* sD = reinterpret_cast<C*>(smem_raw);        // [nB][nB], [out][in]
  C* sU = sD + nB * nB;                           // [Nr][W]
  C* sc = sU + Nr * W;                            // [W] interface corrections
  const int nch = (S + W - 1) / W;
  long long q = blockIdx.x;
  const int chunk = (int)(q % nch);
  q /= nch;   // (g, j, l)
  const long long g = q / ((long long)d.Nt * d.Np), jl = q % ((long long)d.Nt * d.Np);
  const int c0 = chunk * W, Wc = min(W, S - c0);
  const long long base = g * d.S_g + jl * d.S_l + c0;
  for (int x = threadIdx.x; x < nB * nB; x += blockDim.x) sD[x] = DB[x];
  for (int x = threadIdx.x; x < Nr * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    sU[i * W + w] = (C)U[base + (long long)i * d.S_i + w];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < Wc; w += blockDim.x) {
    const int k = (c0 + w) / d.NP;
    const bool outward = cosT[k] > (C)0;
    const int b = outward ? 0 : nB - 1;
    C dB = 0;
    for (int j = 0; j < nB; ++j) dB = fma(sD[b * nB + j], sU[(iB0 + j) * W + w], dB);
    const C dfd = outward ? (sU[iB0 * W + w] - sU[(iB0 - 1) * W + w]) * inv_h
                          : (sU[(iB1 + 1) * W + w] - sU[iB1 * W + w]) * inv_h;
    sc[w] = (dfd - dB) / tNB[b];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < Nr * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    const int k = (c0 + w) / d.NP;
    const C a = cosT[k];
    const bool outward = a > (C)0;
    const long long gi = base + (long long)i * d.S_i + w;
    C kv = (C)Kin[gi];
    const bool inflow = outward ? i == 0 : i == N;
    if (inflow) {
      if (hold) kv = 0;
    } else {
      C dr;
      const bool central = outward ? (i > iB0 && i <= iB1) : (i >= iB0 && i < iB1);
      if (central) {
        const int ib = i - iB0;
        C s = 0;
        for (int j = 0; j < nB; ++j) s = fma(sD[ib * nB + j], sU[(iB0 + j) * W + w], s);
        dr = s + sc[w] * tNB[ib];
      } else if (outward) {
        dr = (sU[i * W + w] - sU[(i - 1) * W + w]) * inv_h;
      } else {
        dr = (sU[(i + 1) * W + w] - sU[i * W + w]) * inv_h;
      }
      kv += sgn * a * dr;
    }
    zoned_store<T, C>(mode, gi, kv, F, Acc, Uout, out, dt);
  }
}

}  // namespace

template <typename T, typename C>
cudaError_t launch_radial_zoned(const Problem& p, const Tables<C>& t, const C* DB, const C* tNB,
                                int nA, int nB, double h, const T* U, const T* K, C sgn, bool hold,
                                int mode, T* F, T* Acc, T* Uout, T* out, double dt, cudaStream_t s) {
  const int W = 32;
  const int S = p.d.NT * p.d.NP;
  const size_t smem = (size_t)(nB * nB + p.d.Nr * W + W) * sizeof(C);
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(k_radial_zoned<T, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    init = true;
  }
  const long long nct = (long long)p.d.G * p.d.Nt * p.d.Np * ((S + W - 1) / W);
  k_radial_zoned<T, C><<<(unsigned)nct, 256, smem, s>>>(p, t.cosT, DB, tNB, nA, nB, (C)(1.0 / h), U,
                                                        K, sgn, hold ? 1 : 0, mode, F, Acc, Uout,
                                                        out, (C)dt, W);
  return cudaGetLastError();
}

template cudaError_t launch_radial_zoned<double, double>(const Problem&, const Tables<double>&,
                                                         const double*, const double*, int, int,
                                                         double, const double*, const double*,
                                                         double, bool, int, double*, double*,
                                                         double*, double*, double, cudaStream_t);
template cudaError_t launch_radial_zoned<float, float>(const Problem&, const Tables<float>&,
                                                       const float*, const float*, int, int,
                                                       double, const float*, const float*, float,
                                                       bool, int, float*, float*, float*, float*,
                                                       double, cudaStream_t);

}  // namespace ts
