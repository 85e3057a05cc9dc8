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
// The central derivative is taken in even/odd form: the Gauss-Lobatto matrix D
// (M + 1 nodes) is centro-antisymmetric, D[M-i][M-j] = -D[i][j], so with
// e_j = u_j + u_{M-j}, o_j = u_j - u_{M-j} (j < H = (M+1)/2 rounded down) and
// Ep = (D[i][j] + D[i][M-j])/2, Op = (D[i][j] - D[i][M-j])/2 (i, j < H),
//   dB(i) = A + B + Dm[i] u_mid,  dB(M-i) = -A + B - Dm[i] u_mid,
//   A = sum_j Ep[i][j] e_j,  B = sum_j Op[i][j] o_j,  Dm[i] = D[i][M/2],
// and, for an odd number of central nodes, dB(M/2) = sum_j D[M/2][j] o_j: half
// the multiply-adds of the dense rows.
//
// One CTA per (g, theta_j, phi_l) and W consecutive (Theta, Phi) columns: the
// tile's lines are staged in shared memory with the central zone's even/odd
// parts; one thread per column forms c from the row pair (0, M); then the
// central row pairs and the edge-zone rows are finished, each row by the zone
// its direction takes it from (every row is staged before any is written, so
// the pass may overwrite the array it differentiates). The folded matrices are
// read through the L1 cache: the threads of a warp share a row pair.
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

// Folded central-zone tables (layout of ZonedTables on the host side):
// [Ep H*H | Op H*H | Dm H | Mr H | tN nB], row-major [i][j].
template <typename C>
struct ZTab {
  const C *Ep, *Op, *Dm, *Mr, *tN;
};

template <typename C>
__device__ __forceinline__ ZTab<C> ztab(const C* z, int nB) {
  const int H = nB / 2;
  ZTab<C> t;
  t.Ep = z;
  t.Op = z + H * H;
  t.Dm = t.Op + H * H;
  t.Mr = t.Dm + H;
  t.tN = t.Mr + H;
  return t;
}

// The central derivative at the row pair (p, M-p) of column w.
template <typename C>
__device__ __forceinline__ void zoned_pair(const ZTab<C>& z, int H, bool oddB, int p,
                                           const C* sE, const C* sO, const C* sMid, int W, int w,
                                           C& lo, C& hi) {
  C a = 0, b = 0;
  for (int j = 0; j < H; ++j) {
    a = fma(__ldg(z.Ep + p * H + j), sE[j * W + w], a);
    b = fma(__ldg(z.Op + p * H + j), sO[j * W + w], b);
  }
  const C m = oddB ? __ldg(z.Dm + p) * sMid[w] : (C)0;
  lo = a + b + m;
  hi = -a + b - m;
}

template <typename T, typename C>
__global__ void __launch_bounds__(256)
k_radial_zoned(Problem p, const C* __restrict__ cosT, const C* __restrict__ ZT, int nA, int nB,
               C inv_h, const T* U, const T* Kin, C sgn, int hold, int mode, T* F, T* Acc,
               T* Uout, T* out, C dt, int W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nr = d.Nr, N = Nr - 1, S = d.NT * d.NP;
  const int iB0 = nA - 1, iB1 = nA - 1 + nB - 1, M = nB - 1, H = nB / 2;
  const bool oddB = nB & 1;
  const ZTab<C> z = ztab<C>(ZT, nB);
  C* sU = reinterpret_cast<C*>(smem_raw);   // [Nr][W]
  C* sE = sU + Nr * W;                      // [H][W] central even parts
  C* sO = sE + H * W;                       // [H][W] central odd parts
  C* sMid = sO + H * W;                     // [W] central middle node (odd nB)
  C* sc = sMid + W;                         // [W] interface corrections
  const int nch = (S + W - 1) / W;
  long long q = blockIdx.x;
  const int chunk = (int)(q % nch);
  q /= nch;   // (g, j, l)
  const long long g = q / ((long long)d.Nt * d.Np), jl = q % ((long long)d.Nt * d.Np);
  const int c0 = chunk * W, Wc = min(W, S - c0);
  const long long base = g * d.S_g + jl * d.S_l + c0;
  for (int x = threadIdx.x; x < Nr * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    sU[i * W + w] = (C)U[base + (long long)i * d.S_i + w];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < H * Wc; x += blockDim.x) {
    const int j = x / Wc, w = x - j * Wc;
    const C a = sU[(iB0 + j) * W + w], b = sU[(iB0 + M - j) * W + w];
    sE[j * W + w] = a + b;
    sO[j * W + w] = a - b;
  }
  if (oddB)
    for (int w = threadIdx.x; w < Wc; w += blockDim.x) sMid[w] = sU[(iB0 + H) * W + w];
  __syncthreads();
  // interface correction of each column from the pair (0, M)
  for (int w = threadIdx.x; w < Wc; w += blockDim.x) {
    const bool outward = cosT[(c0 + w) / d.NP] > (C)0;
    C d0, dM;
    zoned_pair<C>(z, H, oddB, 0, sE, sO, sMid, W, w, d0, dM);
    const C dfd = outward ? (sU[iB0 * W + w] - sU[(iB0 - 1) * W + w]) * inv_h
                          : (sU[(iB1 + 1) * W + w] - sU[iB1 * W + w]) * inv_h;
    sc[w] = outward ? (dfd - d0) / __ldg(z.tN) : (dfd - dM) / __ldg(z.tN + M);
  }
  __syncthreads();
  // central rows: pairs (iB0 + p, iB0 + M - p) and the middle row; a row is
  // finished here when its direction takes it from the central zone
  const int np = H + (oddB ? 1 : 0);
  for (int x = threadIdx.x; x < np * Wc; x += blockDim.x) {
    const int pr = x / Wc, w = x - pr * Wc;
    const C a = cosT[(c0 + w) / d.NP];
    const bool outward = a > (C)0;
    C dlo, dhi;
    int ilo, ihi;
    if (pr < H) {
      zoned_pair<C>(z, H, oddB, pr, sE, sO, sMid, W, w, dlo, dhi);
      ilo = iB0 + pr;
      ihi = iB0 + M - pr;
    } else {   // the middle row
      C s = 0;
      for (int j = 0; j < H; ++j) s = fma(__ldg(z.Mr + j), sO[j * W + w], s);
      dlo = dhi = s;
      ilo = ihi = iB0 + H;
    }
    for (int side = 0; side < (ilo == ihi ? 1 : 2); ++side) {
      const int i = side ? ihi : ilo;
      const bool central = outward ? (i > iB0 && i <= iB1) : (i >= iB0 && i < iB1);
      if (!central) continue;
      const C dr = (side ? dhi : dlo) + sc[w] * __ldg(z.tN + (i - iB0));
      const long long gi = base + (long long)i * d.S_i + w;
      zoned_store<T, C>(mode, gi, (C)Kin[gi] + sgn * a * dr, F, Acc, Uout, out, dt);
    }
  }
  // edge-zone rows [0, iB0] and [iB1, N]: upwind differences, or the held outer
  // inflow node; a row is finished here when its direction does not take it from
  // the central zone
  const int ne = 2 * nA;
  for (int x = threadIdx.x; x < ne * Wc; x += blockDim.x) {
    const int r = x / Wc, w = x - r * Wc;
    const int i = r < nA ? r : iB1 + (r - nA);
    const C a = cosT[(c0 + w) / d.NP];
    const bool outward = a > (C)0;
    const bool central = outward ? (i > iB0 && i <= iB1) : (i >= iB0 && i < iB1);
    if (central) continue;
    const long long gi = base + (long long)i * d.S_i + w;
    C kv = (C)Kin[gi];
    const bool inflow = outward ? i == 0 : i == N;
    if (inflow) {
      if (hold) kv = 0;
    } else {
      const C dr = outward ? (sU[i * W + w] - sU[(i - 1) * W + w]) * inv_h
                           : (sU[(i + 1) * W + w] - sU[i * W + w]) * inv_h;
      kv += sgn * a * dr;
    }
    zoned_store<T, C>(mode, gi, kv, F, Acc, Uout, out, dt);
  }
}

}  // namespace

template <typename T, typename C>
cudaError_t launch_radial_zoned(const Problem& p, const Tables<C>& t, const C* ZT, int nA, int nB,
                                double h, const T* U, const T* K, C sgn, bool hold, int mode,
                                T* F, T* Acc, T* Uout, T* out, double dt, cudaStream_t s) {
  const int W = 32;
  const int S = p.d.NT * p.d.NP, H = nB / 2;
  const size_t smem = (size_t)((p.d.Nr + 2 * H + 2) * W) * sizeof(C);
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(k_radial_zoned<T, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    init = true;
  }
  const long long nct = (long long)p.d.G * p.d.Nt * p.d.Np * ((S + W - 1) / W);
  k_radial_zoned<T, C><<<(unsigned)nct, 256, smem, s>>>(p, t.cosT, ZT, nA, nB, (C)(1.0 / h), U,
                                                        K, sgn, hold ? 1 : 0, mode, F, Acc, Uout,
                                                        out, (C)dt, W);
  return cudaGetLastError();
}

template cudaError_t launch_radial_zoned<double, double>(const Problem&, const Tables<double>&,
                                                         const double*, int, int, double,
                                                         const double*, const double*, double,
                                                         bool, int, double*, double*, double*,
                                                         double*, double, cudaStream_t);
template cudaError_t launch_radial_zoned<float, float>(const Problem&, const Tables<float>&,
                                                       const float*, int, int, double,
                                                       const float*, const float*, float, bool,
                                                       int, float*, float*, float*, float*,
                                                       double, cudaStream_t);

}  // namespace ts
