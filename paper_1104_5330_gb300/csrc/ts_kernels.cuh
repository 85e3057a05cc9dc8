// Kernels of one RK4 stage of the 6-D transport step and of its adjoint.
//
// A stage derivative K = Tau(-L_sph U + CT(U)) (Eqs. Liouvsph, Transpfpsph,
// Transp) is built in three passes over the field, each staging the lines it
// contracts in shared memory:
//   1. angular pass, one angular block (fixed g,i,j,l: all Theta, Phi) per
//      tile: d_Theta (double-Fourier-sphere pair: Theta_k and the partner at
//      Phi + pi), d_Phi, the scattering mean J (Fejer x trapezoid, warp
//      reduction), the collision term, and the Theta/Phi terms of L_sph;
//   2. plane pass, one (theta, phi) plane at fixed (g,i,Theta) and a set of
//      Phi columns closed under Phi -> Phi + pi: d_theta (partner at
//      (phi + pi, Phi + pi)) and d_phi, the theta/phi terms of L_sph;
//   3. radial pass, full r-lines: d_r (Chebyshev-Gauss-Lobatto matrix), the
//      r term, the Tau inflow rows (Sect. 5.1), and the RK4 stage update.
// Derivative matrices are applied as dense contractions; their transposes
// give the adjoint passes.
#pragma once

#include "ts_internal.h"

namespace ts {

constexpr int kThreads = 256;

template <typename C>
__device__ __forceinline__ C fmac(C a, C b, C c) { return fma(a, b, c); }

__device__ __forceinline__ void decode_block(const Dims& d, long long blk, int& g, int& i, int& j,
                                             int& l) {
  l = (int)(blk % d.Np);
  long long q = blk / d.Np;
  j = (int)(q % d.Nt);
  q /= d.Nt;
  i = (int)(q % d.Nr);
  g = (int)(q / d.Nr);
}

// ----------------------------------------------------------------------------
// Pass 1 (forward): angular blocks. A CTA owns `nb` consecutive blocks, which
// are contiguous in memory (block b = elements [b*S, (b+1)*S), S = NT*NP).
// K = sgn * (a_Th dTh U + a_Ph dPh U)
//     + [eta - (kappa+kappa_s) U + kappa_s (J + b omega.H + c omega.M~.omega)]
// a_Th = -sin(Th)/r, a_Ph = -sin(Th) sin(Ph) cot(th)/r; b, c: the kernel's mu and
// mu^2 - 1/3 coefficients (p.scb, p.scc, NULL = 0), H and M~ = M - J I/3 the
// first and traceless second angular moments, taken in the local frame:
// omega = cos(Th) e_r + sin(Th) cos(Ph) e_th + sin(Th) sin(Ph) e_ph.
template <typename T, typename C>
__device__ __forceinline__ void angular_tile(const Problem& p, const Tables<C>& t,
                                             const T* __restrict__ U, T* __restrict__ K, C sgn,
                                             int collision, int nb, long long tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP, hP = NP / 2;
  C* sA = reinterpret_cast<C*>(smem_raw);  // AThT [k'][k]
  C* sB = sA + NT * NT;                    // BThT [k'][k]
  C* sD = sB + NT * NT;                    // DPhT [m'][m]
  C* su = sD + NP * NP;                    // tile [bb][k][m]
  C* sJ = su + nb * S;   // [kAngMoments][nb]: J, H_r, H_th, H_ph, M_rr, M_thth, M_phph, M_thph, M_rth, M_rph
  const long long b0 = tile * nb;
  const int kf = kernel_form(p, collision);
  const bool aniso = kf >= KF_LINEAR, quad = kf >= KF_QUADRATIC;
  const int nbb = (int)min((long long)nb, d.nblk - b0);
  for (int x = threadIdx.x; x < NT * NT; x += blockDim.x) {
    sA[x] = t.AThT[x];
    sB[x] = t.BThT[x];
  }
  for (int x = threadIdx.x; x < NP * NP; x += blockDim.x) sD[x] = t.DPhT[x];
  const T* src = U + b0 * S;
  for (int x = threadIdx.x; x < nbb * S; x += blockDim.x) su[x] = (C)src[x];
  __syncthreads();
  if (collision) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bb = warp; bb < nbb; bb += blockDim.x >> 5) {
      C mo[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // J, H (3), M (6)
      for (int x = lane; x < S; x += 32) {
        const int k = x / NP, m = x - k * NP;
        const C u = su[bb * S + x];
        mo[0] = fmac(t.qdir[k], u, mo[0]);
        if (aniso) {
          const C qu = t.qdir[k] * u, qs = t.sinT[k] * qu, ct = t.cosT[k];
          const C cp = t.cosP[m], sp = t.sinP[m];
          mo[1] = fmac(ct, qu, mo[1]);
          mo[2] = fmac(cp, qs, mo[2]);
          mo[3] = fmac(sp, qs, mo[3]);
          if (quad) {
            const C qss = t.sinT[k] * qs;
            mo[4] = fmac(ct * ct, qu, mo[4]);
            mo[5] = fmac(cp * cp, qss, mo[5]);
            mo[6] = fmac(sp * sp, qss, mo[6]);
            mo[7] = fmac(cp * sp, qss, mo[7]);
            mo[8] = fmac(ct * cp, qs, mo[8]);
            mo[9] = fmac(ct * sp, qs, mo[9]);
          }
        }
      }
      const int na = quad ? 10 : aniso ? 4 : 1;   // uniform over the block
#pragma unroll
      for (int a = 0; a < 10; ++a)   // constant indices keep mo in registers
        if (a < na)
          for (int o = 16; o; o >>= 1) mo[a] += __shfl_xor_sync(0xffffffffu, mo[a], o);
      if (lane == 0) {
#pragma unroll
        for (int a = 0; a < 10; ++a)
          if (a < na) sJ[a * nb + bb] = mo[a];
      }
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < nbb * S; x += blockDim.x) {
    const int bb = x / S, r = x - bb * S, k = r / NP, m = r - k * NP;
    const int mh = (m + hP) % NP;
    const C* ub = su + bb * S;
    C dT = 0, dP = 0;
    for (int kk = 0; kk < NT; ++kk) {
      dT = fmac(sA[kk * NT + k], ub[kk * NP + m], dT);
      dT = fmac(sB[kk * NT + k], ub[kk * NP + mh], dT);
    }
    for (int mm = 0; mm < NP; ++mm) dP = fmac(sD[mm * NP + m], ub[k * NP + mm], dP);
    const long long blk = b0 + bb;
    int g, i, j, l;
    decode_block(d, blk, g, i, j, l);
    const C aT = -t.sinT[k] * t.inv_r[i];
    const C aP = aT * t.sinP[m] * t.cot_th[j];
    C v = sgn * (aT * dT + aP * dP);
    if (collision) {
      const C u = ub[r];
      const C kap = (C)p.kap[blk], eta = (C)p.eta[blk], ks = (C)p.kaps[blk];
      v += eta - (kap + ks) * u + ks * sJ[bb];
      const C ct = t.cosT[k], st = t.sinT[k], cp = t.cosP[m], sp = t.sinP[m];
      if (aniso && p.scb) {
        const C kb = (C)(p.kaps[blk] * p.scb[blk]);
        v += kb * (ct * sJ[nb + bb] + st * (cp * sJ[2 * nb + bb] + sp * sJ[3 * nb + bb]));
      }
      if (quad) {
        const C kc = (C)(p.kaps[blk] * p.scc[blk]), j3 = sJ[bb] * ((C)1 / (C)3);
        const C* M = sJ + 4 * nb + bb;
        v += kc * (ct * ct * (M[0] - j3) +
                   st * st * (cp * cp * (M[nb] - j3) + sp * sp * (M[2 * nb] - j3) +
                              (C)2 * cp * sp * M[3 * nb]) +
                   (C)2 * ct * st * (cp * M[4 * nb] + sp * M[5 * nb]));
      }
    }
    K[blk * S + r] = (T)v;
  }
}

// ----------------------------------------------------------------------------
// Pass 2 (forward): (theta, phi) planes. A CTA owns (g, i, k) and the Phi
// columns m0..m0+c-1 and m0+NP/2..m0+NP/2+c-1; tile [j][l][w], w < 2c.
// K += sgn * (a_th dth U + a_ph dph U), a_th = sin(Th)cos(Ph)/r,
// a_ph = sin(Th) sin(Ph)/(r sin(th)).
__device__ __forceinline__ int plane_m(int w, int c, int m0, int hP) {
  return w < c ? m0 + w : m0 + hP + (w - c);
}

template <typename T, typename C>
__device__ __forceinline__ void plane_tile(const Problem& p, const Tables<C>& t,
                                           const T* __restrict__ U, T* __restrict__ K, C sgn,
                                           int c, long long tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nt = d.Nt, Np = d.Np, NP = d.NP, hP = NP / 2, hp = Np / 2, W = 2 * c;
  C* sA = reinterpret_cast<C*>(smem_raw);  // AthT [j'][j]
  C* sB = sA + Nt * Nt;                    // BthT
  C* sD = sB + Nt * Nt;                    // DphT [l'][l]
  C* su = sD + Np * Np;                    // [j][l][w]
  const int nchunk = hP / c;
  long long q = tile;
  const int chunk = (int)(q % nchunk);
  q /= nchunk;
  const int k = (int)(q % d.NT);
  q /= d.NT;
  const int i = (int)(q % d.Nr);
  const int g = (int)(q / d.Nr);
  const int m0 = chunk * c;
  const long long base = (long long)g * d.S_g + (long long)i * d.S_i + (long long)k * NP;
  for (int x = threadIdx.x; x < Nt * Nt; x += blockDim.x) {
    sA[x] = t.AthT[x];
    sB[x] = t.BthT[x];
  }
  for (int x = threadIdx.x; x < Np * Np; x += blockDim.x) sD[x] = t.DphT[x];
  const int n = Nt * Np * W;
  for (int x = threadIdx.x; x < n; x += blockDim.x) {
    const int w = x % W, jl = x / W, l = jl % Np, j = jl / Np;
    su[x] = (C)U[base + (long long)j * d.S_j + (long long)l * d.S_l + plane_m(w, c, m0, hP)];
  }
  __syncthreads();
  const C sTk = t.sinT[k], ir = t.inv_r[i];
  for (int x = threadIdx.x; x < n; x += blockDim.x) {
    const int w = x % W, jl = x / W, l = jl % Np, j = jl / Np;
    const int lh = (l + hp) % Np, wh = w < c ? w + c : w - c;
    C dth = 0, dph = 0;
    for (int jj = 0; jj < Nt; ++jj) {
      dth = fmac(sA[jj * Nt + j], su[(jj * Np + l) * W + w], dth);
      dth = fmac(sB[jj * Nt + j], su[(jj * Np + lh) * W + wh], dth);
    }
    for (int ll = 0; ll < Np; ++ll) dph = fmac(sD[ll * Np + l], su[(j * Np + ll) * W + w], dph);
    const int m = plane_m(w, c, m0, hP);
    const C ath = sTk * t.cosP[m] * ir;
    const C aph = sTk * t.sinP[m] * ir * t.inv_sinth[j];
    const long long idx = base + (long long)j * d.S_j + (long long)l * d.S_l + m;
    K[idx] = (T)((p.plane_store ? (C)0 : (C)K[idx]) + sgn * (ath * dth + aph * dph));
  }
}

// ----------------------------------------------------------------------------
// Pass 3 (forward): r-lines. A CTA owns (g, j, l) and W consecutive columns
// col = k*NP + m of the angular block, all Nr radial nodes: tile [i][w].
// K += sgn * cos(Th) d_r U, then the Tau rows, then the stage update.
// Tau (Sect. 5.1): K_i += (gdot - K_b) T_N(x_b) T_N(x_i), gdot = 0 for static
// inflow data, b = 0 if cos(Th) > 0 else Nr-1; T_N(x_i) = (-1)^(N-i). This is
// the nodal form of replacing the top Chebyshev coefficient of K.
template <typename T, typename C>
__device__ __forceinline__ void radial_tile(const Problem& p, const Tables<C>& t,
                                            const double* __restrict__ Dr64, const T* U,
                                            const T* Kin, C sgn, int tau, int mode, T* F,
                                            T* Acc, T* Uout, T* out, C dt, int W,
                                            long long tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nr = d.Nr, NP = d.NP, S = d.NT * d.NP;
  C* sDr = reinterpret_cast<C*>(smem_raw);  // Dr [i][i']
  C* su = sDr + Nr * Nr;                    // [i][w]
  C* sk = su + Nr * W;                      // [i][w]
  const int nchunk = (S + W - 1) / W;
  long long q = tile;
  const int chunk = (int)(q % nchunk);
  q /= nchunk;
  const int l = (int)(q % d.Np);
  q /= d.Np;
  const int j = (int)(q % d.Nt);
  const int g = (int)(q / d.Nt);
  const int c0 = chunk * W;
  const int Wc = min(W, S - c0);
  const long long base =
      (long long)g * d.S_g + (long long)j * d.S_j + (long long)l * d.S_l + c0;
  for (int x = threadIdx.x; x < Nr * Nr; x += blockDim.x) sDr[x] = t.Dr[x];
  for (int x = threadIdx.x; x < Nr * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    const long long gi = base + (long long)i * d.S_i + w;
    su[i * W + w] = (C)U[gi];
    sk[i * W + w] = (C)Kin[gi];
  }
  __syncthreads();
  const int nlo = p.n_fp64_rows, nhi = Nr - p.n_fp64_rows;
  for (int x = threadIdx.x; x < Nr * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    const int k = (c0 + w) / NP;
    C dr;
    if (i < nlo || i >= nhi) {  // rows with the largest entries: accumulate in double
      double a = 0;
      for (int ii = 0; ii < Nr; ++ii) a = fma(Dr64[i * Nr + ii], (double)su[ii * W + w], a);
      dr = (C)a;
    } else {
      C a = 0;
      for (int ii = 0; ii < Nr; ++ii) a = fmac(sDr[i * Nr + ii], su[ii * W + w], a);
      dr = a;
    }
    sk[i * W + w] += sgn * t.cosT[k] * dr;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < Nr * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    const int k = (c0 + w) / NP;
    C kv = sk[i * W + w];
    if (tau) {
      const int b = t.cosT[k] > (C)0 ? 0 : Nr - 1;
      kv -= sk[b * W + w] * t.tsign[b] * t.tsign[i];
    }
    const long long gi = base + (long long)i * d.S_i + w;
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
      case RAD_AB2:   // in place: the tile's F lines were staged before the barrier
        F[gi] = (T)((C)F[gi] + dt * ((C)1.5 * kv - (C)0.5 * (C)Acc[gi]));
        Acc[gi] = (T)kv;
        break;
      default:        // RAD_AB2_START
        F[gi] = (T)((C)F[gi] + dt * kv);
        Acc[gi] = (T)kv;
        break;
    }
  }
}

// ----------------------------------------------------------------------------
// Adjoint pass 3^T: r-lines. Kbar = scale * X. lt = Tau^T Kbar:
// lt_i = Kbar_i - [i == b] T_N(x_b) sum_i' T_N(x_i') Kbar_i'. Then the radial
// part of the stage adjoint: Ubar = -cos(Th) D_r^T lt, with D_r^T (also
// centro-antisymmetric) applied to the even/odd parts of lt: one thread per
// output pair (i, N-i) and column, half the multiply-adds of the dense product.
template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_radial_T(Problem p, Tables<C> t, const T* __restrict__ X, C scale, int tau,
           T* __restrict__ lt, T* __restrict__ Ubar, int W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nr = d.Nr, N = Nr - 1, hh = Nr / 2, NP = d.NP, S = d.NT * d.NP;
  C* sE = reinterpret_cast<C*>(smem_raw);  // EpTa [i'][i]
  C* sO = sE + hh * hh;                    // OpTa [i'][i]
  C* sMc = sO + hh * hh;
  C* sMr = sMc + hh;
  C* sk = sMr + hh;                        // Kbar, then lt  [i][w]
  C* sEv = sk + Nr * W;                    // lt_i' + lt_{N-i'}
  C* sOd = sEv + hh * W;                   // lt_i' - lt_{N-i'}
  const int nchunk = (S + W - 1) / W;
  long long q = blockIdx.x;
  const int chunk = (int)(q % nchunk);
  q /= nchunk;
  const int l = (int)(q % d.Np);
  q /= d.Np;
  const int j = (int)(q % d.Nt);
  const int g = (int)(q / d.Nt);
  const int c0 = chunk * W;
  const int Wc = min(W, S - c0);
  const long long base =
      (long long)g * d.S_g + (long long)j * d.S_j + (long long)l * d.S_l + c0;
  for (int x = threadIdx.x; x < hh * hh; x += blockDim.x) {
    sE[x] = t.EpTa[x];
    sO[x] = t.OpTa[x];
  }
  for (int x = threadIdx.x; x < hh; x += blockDim.x) {
    sMc[x] = t.DrMca[x];
    sMr[x] = t.DrMra[x];
  }
  for (int x = threadIdx.x; x < Nr * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    sk[i * W + w] = scale * (C)X[base + (long long)i * d.S_i + w];
  }
  __syncthreads();
  if (tau) {
    for (int w = threadIdx.x; w < Wc; w += blockDim.x) {
      const int b = t.cosT[(c0 + w) / NP] > (C)0 ? 0 : N;
      C s = 0;
      for (int ii = 0; ii < Nr; ++ii) s = fmac(t.tsign[ii], sk[ii * W + w], s);
      sk[b * W + w] -= t.tsign[b] * s;
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < Nr * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    const C v = sk[i * W + w];
    lt[base + (long long)i * d.S_i + w] = (T)v;
    if (i < hh) {
      const C u = sk[(N - i) * W + w];
      sEv[i * W + w] = v + u;
      sOd[i * W + w] = v - u;
    }
  }
  __syncthreads();
  const bool odd = Nr & 1;
  const int npair = hh + (odd ? 1 : 0);
  for (int x = threadIdx.x; x < npair * Wc; x += blockDim.x) {
    const int i = x / Wc, w = x - i * Wc;
    const C ck = -t.cosT[(c0 + w) / NP];
    if (i < hh) {
      C ae = 0, ao = 0;
      for (int ip = 0; ip < hh; ++ip) {
        ae = fmac(sE[ip * hh + i], sEv[ip * W + w], ae);
        ao = fmac(sO[ip * hh + i], sOd[ip * W + w], ao);
      }
      if (odd) ae = fmac((C)2 * sMc[i], sk[(N / 2) * W + w], ae);
      Ubar[base + (long long)i * d.S_i + w] = (T)(ck * (C)0.5 * (ao + ae));
      Ubar[base + (long long)(N - i) * d.S_i + w] = (T)(ck * (C)0.5 * (ao - ae));
    } else {  // middle node
      C am = 0;
      for (int ip = 0; ip < hh; ++ip) am = fmac(sMr[ip], sOd[ip * W + w], am);
      Ubar[base + (long long)(N / 2) * d.S_i + w] = (T)(ck * am);
    }
  }
}

// Adjoint pass 2^T: Ubar -= D_th^T (a_th lt) + D_ph^T (a_ph lt).
// (D_th^T mu)(j', l, m) = sum_j Ath[j][j'] mu(j,l,m) + Bth[j][j'] mu(j, l+Np/2, m+NP/2):
// the output and its DFS partner (j', l+Np/2, m+NP/2) come from the sum and
// difference of mu with its partner through (A+B)/2 and (A-B)/2 -- one thread
// per output pair.
template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_plane_T(Problem p, Tables<C> t, const T* __restrict__ lt, T* __restrict__ Ubar, int c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nt = d.Nt, Np = d.Np, NP = d.NP, hP = NP / 2, hp = Np / 2, W = 2 * c;
  C* sP = reinterpret_cast<C*>(smem_raw);  // PthA [j][j']
  C* sQ = sP + Nt * Nt;
  C* sD = sQ + Nt * Nt;                    // Dph [l][l']
  C* sS = sD + Np * Np;                    // a_th lt + partner   [j][l < Np/2][w]
  C* sDf = sS + Nt * hp * W;               // a_th lt - partner
  C* s2 = sDf + Nt * hp * W;               // a_ph * lt            [j][l][w]
  const int nchunk = hP / c;
  long long q = blockIdx.x;
  const int chunk = (int)(q % nchunk);
  q /= nchunk;
  const int k = (int)(q % d.NT);
  q /= d.NT;
  const int i = (int)(q % d.Nr);
  const int g = (int)(q / d.Nr);
  const int m0 = chunk * c;
  const long long base = (long long)g * d.S_g + (long long)i * d.S_i + (long long)k * NP;
  for (int x = threadIdx.x; x < Nt * Nt; x += blockDim.x) {
    sP[x] = t.PthA[x];
    sQ[x] = t.QthA[x];
  }
  for (int x = threadIdx.x; x < Np * Np; x += blockDim.x) sD[x] = t.Dph[x];
  const C sTk = t.sinT[k] * t.inv_r[i];
  const int n2 = Nt * hp * W;
  for (int x = threadIdx.x; x < n2; x += blockDim.x) {   // (j, l < Np/2, w) and its partner
    const int w = x % W, jl = x / W, l = jl % hp, j = jl / hp;
    const int wh = w < c ? w + c : w - c;
    const int m = plane_m(w, c, m0, hP), mh = plane_m(wh, c, m0, hP);
    const C v1 = (C)lt[base + (long long)j * d.S_j + (long long)l * d.S_l + m];
    const C v2 = (C)lt[base + (long long)j * d.S_j + (long long)(l + hp) * d.S_l + mh];
    const C a1 = sTk * t.cosP[m] * v1, a2 = sTk * t.cosP[mh] * v2;
    sS[x] = a1 + a2;
    sDf[x] = a1 - a2;
    const C isn = t.inv_sinth[j];
    s2[(j * Np + l) * W + w] = sTk * t.sinP[m] * isn * v1;
    s2[(j * Np + l + hp) * W + wh] = sTk * t.sinP[mh] * isn * v2;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < n2; x += blockDim.x) {   // output pair (j, l, w), (j, l+hp, wh)
    const int w = x % W, jl = x / W, l = jl % hp, j = jl / hp;
    const int wh = w < c ? w + c : w - c;
    C ps = 0, qd = 0;
    for (int jj = 0; jj < Nt; ++jj) {
      const int o = (jj * hp + l) * W + w;
      ps = fmac(sP[jj * Nt + j], sS[o], ps);
      qd = fmac(sQ[jj * Nt + j], sDf[o], qd);
    }
    C f1 = 0, f2 = 0;
    for (int ll = 0; ll < Np; ++ll) {
      f1 = fmac(sD[ll * Np + l], s2[(j * Np + ll) * W + w], f1);
      f2 = fmac(sD[ll * Np + l + hp], s2[(j * Np + ll) * W + wh], f2);
    }
    const long long i1 =
        base + (long long)j * d.S_j + (long long)l * d.S_l + plane_m(w, c, m0, hP);
    const long long i2 =
        base + (long long)j * d.S_j + (long long)(l + hp) * d.S_l + plane_m(wh, c, m0, hP);
    Ubar[i1] = (T)((C)Ubar[i1] - (ps + qd) - f1);
    Ubar[i2] = (T)((C)Ubar[i2] - (ps - qd) - f2);
  }
}

// Adjoint pass 2^T with the theta folding (even N_theta): D_th^T through the
// two DFS pairs that the columns w and w^ = w +- c form at (l, l + Np/2), and
// over j -> Nt-1-j (P^T, Q^T centro-antisymmetric) through the theta-even/odd
// parts of the pair sums and differences; D_ph^T (circulant) on the phi pair
// halves at each column. One thread per (j < Nt/2, l < Np/2, w < c): the 8
// outputs at rows j, Nt-1-j x phi l, l + Np/2 x columns w, w^.
template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_plane_T_fold(Problem p, Tables<C> t, const T* __restrict__ lt, T* __restrict__ Ubar, int c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nt = d.Nt, Np = d.Np, NP = d.NP, hP = NP / 2, hp = Np / 2, ht = Nt / 2, W = 2 * c;
  const int FQ = ht * hp * W;               // one folded theta-sum array [jj][l][w]
  const int HQ = Nt * hp * W;               // one phi-half array [j][l'][w]
  C* sPe = reinterpret_cast<C*>(smem_raw);  // folded P^T, Q^T [jj][j] (Nt/2 x Nt/2 each)
  C* sPo = sPe + ht * ht;
  C* sQe = sPo + ht * ht;
  C* sQo = sQe + ht * ht;
  C* sMs = sQo + ht * ht;                   // D_ph^T on pair halves [l'][l]
  C* sMd = sMs + hp * hp;
  C* sF = sMd + hp * hp;                    // [ES | OS | ED | OD] of a_th lt
  C* sH = sF + 4 * FQ;                      // [sigma | delta] of a_ph lt
  const int nchunk = hP / c;
  long long q = blockIdx.x;
  const int chunk = (int)(q % nchunk);
  q /= nchunk;
  const int k = (int)(q % d.NT);
  q /= d.NT;
  const int i = (int)(q % d.Nr);
  const int g = (int)(q / d.Nr);
  const int m0 = chunk * c;
  const long long base = (long long)g * d.S_g + (long long)i * d.S_i + (long long)k * NP;
  for (int x = threadIdx.x; x < ht * ht; x += blockDim.x) {
    sPe[x] = t.PethA[x];
    sPo[x] = t.PothA[x];
    sQe[x] = t.QethA[x];
    sQo[x] = t.QothA[x];
  }
  for (int x = threadIdx.x; x < hp * hp; x += blockDim.x) {
    sMs[x] = t.MsphA[x];
    sMd[x] = t.MdphA[x];
  }
  const C sTk = t.sinT[k] * t.inv_r[i];
  const int nq = ht * hp * c;
  for (int x = threadIdx.x; x < nq; x += blockDim.x) {   // (jj, l, w < c) and partners
    const int w = x % c, jl = x / c, l = jl % hp, jj = jl / hp;
    const int wh = w + c;
    const int mA = plane_m(w, c, m0, hP), mB = plane_m(wh, c, m0, hP);
    const C cA = sTk * t.cosP[mA], cB = sTk * t.cosP[mB];
    C sAv[2], dAv[2], sBv[2], dBv[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int j = side ? Nt - 1 - jj : jj;
      const long long r0 = base + (long long)j * d.S_j + (long long)l * d.S_l;
      const long long r1 = r0 + (long long)hp * d.S_l;
      const C u0A = (C)lt[r0 + mA], u0B = (C)lt[r0 + mB];   // (l, w), (l, w^)
      const C u1A = (C)lt[r1 + mA], u1B = (C)lt[r1 + mB];   // (l+hp, w), (l+hp, w^)
      sAv[side] = cA * u0A + cB * u1B;   // DFS pair (l, w) ~ (l+hp, w^)
      dAv[side] = cA * u0A - cB * u1B;
      sBv[side] = cB * u0B + cA * u1A;   // DFS pair (l, w^) ~ (l+hp, w)
      dBv[side] = cB * u0B - cA * u1A;
      const C isn = t.inv_sinth[j];
      const C pA = sTk * t.sinP[mA] * isn, pB = sTk * t.sinP[mB] * isn;
      C* h = sH + (j * hp + l) * W;
      h[w] = pA * (u0A + u1A);          // phi pair halves at column w
      h[HQ + w] = pA * (u0A - u1A);
      h[wh] = pB * (u0B + u1B);         // and at column w^
      h[HQ + wh] = pB * (u0B - u1B);
    }
    C* f = sF + (jj * hp + l) * W;
    f[w] = sAv[0] + sAv[1];
    f[FQ + w] = sAv[0] - sAv[1];
    f[2 * FQ + w] = dAv[0] + dAv[1];
    f[3 * FQ + w] = dAv[0] - dAv[1];
    f[wh] = sBv[0] + sBv[1];
    f[FQ + wh] = sBv[0] - sBv[1];
    f[2 * FQ + wh] = dBv[0] + dBv[1];
    f[3 * FQ + wh] = dBv[0] - dBv[1];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nq; x += blockDim.x) {
    const int w = x % c, jl = x / c, l = jl % hp, j0 = jl / hp;
    const int wh = w + c;
    C th[2][4];   // [column w / w^][aE, aO, bE, bO]
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) th[a][b] = 0;
    for (int jj = 0; jj < ht; ++jj) {
      const C* f = sF + (jj * hp + l) * W;
      const int o = jj * ht + j0;
      const C pe = sPe[o], po = sPo[o], qe = sQe[o], qo = sQo[o];
      th[0][0] = fmac(pe, f[w], th[0][0]);
      th[0][1] = fmac(po, f[FQ + w], th[0][1]);
      th[0][2] = fmac(qe, f[2 * FQ + w], th[0][2]);
      th[0][3] = fmac(qo, f[3 * FQ + w], th[0][3]);
      th[1][0] = fmac(pe, f[wh], th[1][0]);
      th[1][1] = fmac(po, f[FQ + wh], th[1][1]);
      th[1][2] = fmac(qe, f[2 * FQ + wh], th[1][2]);
      th[1][3] = fmac(qo, f[3 * FQ + wh], th[1][3]);
    }
    C ph[2][2][2];   // [row j0 / mirror][column w / w^][sigma, delta sums]
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) ph[a][b][0] = ph[a][b][1] = 0;
    for (int ll = 0; ll < hp; ++ll) {
      const C ms = sMs[ll * hp + l], md = sMd[ll * hp + l];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int j = side ? Nt - 1 - j0 : j0;
        const C* h = sH + (j * hp + ll) * W;
        ph[side][0][0] = fmac(ms, h[w], ph[side][0][0]);
        ph[side][0][1] = fmac(md, h[HQ + w], ph[side][0][1]);
        ph[side][1][0] = fmac(ms, h[wh], ph[side][1][0]);
        ph[side][1][1] = fmac(md, h[HQ + wh], ph[side][1][1]);
      }
    }
    const int mA = plane_m(w, c, m0, hP), mB = plane_m(wh, c, m0, hP);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int j = side ? Nt - 1 - j0 : j0;
      const C sg = side ? (C)-1 : (C)1;
      const C psA = (C)0.5 * (th[0][1] + sg * th[0][0]), qdA = (C)0.5 * (th[0][3] + sg * th[0][2]);
      const C psB = (C)0.5 * (th[1][1] + sg * th[1][0]), qdB = (C)0.5 * (th[1][3] + sg * th[1][2]);
      const C fwA = (C)0.5 * (ph[side][0][0] + ph[side][0][1]);   // phi at (l, w)
      const C fwB = (C)0.5 * (ph[side][0][0] - ph[side][0][1]);   // phi at (l+hp, w)
      const C fhA = (C)0.5 * (ph[side][1][0] + ph[side][1][1]);   // phi at (l, w^)
      const C fhB = (C)0.5 * (ph[side][1][0] - ph[side][1][1]);   // phi at (l+hp, w^)
      const long long r0 = base + (long long)j * d.S_j + (long long)l * d.S_l;
      const long long r1 = r0 + (long long)hp * d.S_l;
      Ubar[r0 + mA] = (T)((C)Ubar[r0 + mA] - (psA + qdA) - fwA);   // (l, w)
      Ubar[r1 + mB] = (T)((C)Ubar[r1 + mB] - (psA - qdA) - fhB);   // (l+hp, w^)
      Ubar[r0 + mB] = (T)((C)Ubar[r0 + mB] - (psB + qdB) - fhA);   // (l, w^)
      Ubar[r1 + mA] = (T)((C)Ubar[r1 + mA] - (psB - qdB) - fwB);   // (l+hp, w)
    }
  }
}

// Adjoint pass 1^T: angular blocks.
//   Ubar_s = Ubar - D_Th^T(a_Th lt) - D_Ph^T(a_Ph lt) - (kappa+kappa_s) lt + kappa_s q_k sum lt
//            + q_k omega.G + q_k (omega.G2.omega - g0/3)   (anisotropic kernels)
//   G = kappa_s b sum_block omega lt, G2 = kappa_s c sum_block omega omega lt,
//   g0 = kappa_s c sum_block lt
//   gk -= sum_block lt*Us,  ge += sum_block lt
//   lam_out = lam_in + Ubar_s;   Kbar_out = wl*lam + wu*Ubar_s (if Kbar_out)
// The transposed derivatives are folded as in the forward pass: D_Th^T on the
// DFS pair (k, m), (k, m+NP/2) through the pair sum and difference, and over
// k -> NT-1-k (P^T and Q^T are centro-antisymmetric) through their Theta-even/
// odd parts; D_Ph^T (circulant) on the pair halves. One thread per 2 x 2 output
// quadruple (k, NT-1-k) x (m, m+NP/2).
template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_angular_T(Problem p, Tables<C> t, const T* __restrict__ lt, const T* __restrict__ Ubar,
            const T* __restrict__ Us, double* gk, double* ge, const T* lam, const T* lam_in,
            T* lam_out, T* Kbar_out, C wl, C wu, int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP, hP = NP / 2, hT = NT / 2;
  const int Q4 = hT * hP, hS = NT * hP;
  C* sPe = reinterpret_cast<C*>(smem_raw);  // folded P^T, Q^T [kk][k] (NT/2 x NT/2 each)
  C* sPo = sPe + hT * hT;
  C* sQe = sPo + hT * hT;
  C* sQo = sQe + hT * hT;
  C* sMs = sQo + hT * hT;                   // D_Ph^T on pair halves [p'][p] (NP/2 x NP/2)
  C* sMd = sMs + hP * hP;
  C* s1 = sMd + hP * hP;                    // a_Th lt folded: [bb][ES | OS | ED | OD][kk][p]
  C* s2 = s1 + nb * S;                      // a_Ph lt pair halves: [bb][sigma | delta][k][p]
  C* sSum = s2 + nb * S;   // [kAngMoments][nb] kappa_s sum lt, G (3), G2 (6: rr thth phph thph rth rph), g0
  const long long b0 = (long long)blockIdx.x * nb;
  const int kf = kernel_form(p, 1);
  const bool aniso = kf >= KF_LINEAR, quad = kf >= KF_QUADRATIC;
  const int nbb = (int)min((long long)nb, d.nblk - b0);
  for (int x = threadIdx.x; x < hT * hT; x += blockDim.x) {
    sPe[x] = t.PeThA[x];
    sPo[x] = t.PoThA[x];
    sQe[x] = t.QeThA[x];
    sQo[x] = t.QoThA[x];
  }
  for (int x = threadIdx.x; x < hP * hP; x += blockDim.x) {
    sMs[x] = t.MsPhA[x];
    sMd[x] = t.MdPhA[x];
  }
  for (int x = threadIdx.x; x < nbb * Q4; x += blockDim.x) {   // (bb, kk < NT/2, p < NP/2)
    const int bb = x / Q4, r = x - bb * Q4, kk = r / hP, m = r - kk * hP, km = NT - 1 - kk;
    int g, i, j, l;
    decode_block(d, b0 + bb, g, i, j, l);
    const C ir = t.inv_r[i], ct = t.cot_th[j];
    const long long gb = (b0 + bb) * S;
    C sv[2], dv[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int k = side ? km : kk;
      const C v1 = (C)lt[gb + k * NP + m], v2 = (C)lt[gb + k * NP + m + hP];
      const C aT = -t.sinT[k] * ir;
      sv[side] = aT * (v1 + v2);
      dv[side] = aT * (v1 - v2);
      const C n1 = aT * ct * t.sinP[m] * v1, n2 = aT * ct * t.sinP[m + hP] * v2;
      s2[bb * S + k * hP + m] = n1 + n2;
      s2[bb * S + hS + k * hP + m] = n1 - n2;
    }
    C* f = s1 + bb * S + kk * hP + m;
    f[0] = sv[0] + sv[1];
    f[Q4] = sv[0] - sv[1];
    f[2 * Q4] = dv[0] + dv[1];
    f[3 * Q4] = dv[0] - dv[1];
  }
  __syncthreads();
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bb = warp; bb < nbb; bb += blockDim.x >> 5) {
      double sl = 0, slu = 0, g[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // G (3), G2 (6)
      for (int x = lane; x < S; x += 32) {
        const double v = (double)lt[(b0 + bb) * S + x];
        sl += v;
        slu = fma(v, (double)Us[(b0 + bb) * S + x], slu);
        if (aniso) {
          const int k = x / NP, m = x - k * NP;
          const double ct = (double)t.cosT[k], st = (double)t.sinT[k];
          const double cp = (double)t.cosP[m], sp = (double)t.sinP[m], vs = st * v;
          g[0] = fma(ct, v, g[0]);
          g[1] = fma(cp, vs, g[1]);
          g[2] = fma(sp, vs, g[2]);
          if (quad) {
            const double vss = st * vs;
            g[3] = fma(ct * ct, v, g[3]);
            g[4] = fma(cp * cp, vss, g[4]);
            g[5] = fma(sp * sp, vss, g[5]);
            g[6] = fma(cp * sp, vss, g[6]);
            g[7] = fma(ct * cp, vs, g[7]);
            g[8] = fma(ct * sp, vs, g[8]);
          }
        }
      }
      const int ng = quad ? 9 : aniso ? 3 : 0;   // uniform over the block
      for (int o = 16; o; o >>= 1) {
        sl += __shfl_xor_sync(0xffffffffu, sl, o);
        slu += __shfl_xor_sync(0xffffffffu, slu, o);
#pragma unroll
        for (int a = 0; a < 9; ++a)   // constant indices keep g in registers
          if (a < ng) g[a] += __shfl_xor_sync(0xffffffffu, g[a], o);
      }
      if (lane == 0) {
        const long long blk = b0 + bb;
        sSum[bb] = (C)(p.kaps[blk] * sl);
        if (aniso) {
          const double kb = p.scb ? p.kaps[blk] * p.scb[blk] : 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a) sSum[(1 + a) * nb + bb] = (C)(kb * g[a]);
        }
        if (quad) {
          const double kc = p.kaps[blk] * p.scc[blk];
#pragma unroll
          for (int a = 3; a < 9; ++a) sSum[(1 + a) * nb + bb] = (C)(kc * g[a]);
          sSum[10 * nb + bb] = (C)(kc * sl);
        }
        ge[blk] += sl;
        gk[blk] -= slu;
      }
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nbb * Q4; x += blockDim.x) {   // quadruple (k, NT-1-k) x (m, m+hP)
    const int bb = x / Q4, r = x - bb * Q4, k = r / hP, m = r - k * hP, km = NT - 1 - k;
    const C* f = s1 + bb * S;
    C aE = 0, aO = 0, bE = 0, bO = 0;
    for (int kk = 0; kk < hT; ++kk) {
      const int o = kk * hP + m, w = kk * hT + k;
      aE = fmac(sPe[w], f[o], aE);
      aO = fmac(sPo[w], f[Q4 + o], aO);
      bE = fmac(sQe[w], f[2 * Q4 + o], bE);
      bO = fmac(sQo[w], f[3 * Q4 + o], bO);
    }
    const C* g2 = s2 + bb * S;
    C fs[2] = {0, 0}, fd[2] = {0, 0};
    for (int pp = 0; pp < hP; ++pp) {
      const C ms = sMs[pp * hP + m], md = sMd[pp * hP + m];
      fs[0] = fmac(ms, g2[k * hP + pp], fs[0]);
      fd[0] = fmac(md, g2[hS + k * hP + pp], fd[0]);
      fs[1] = fmac(ms, g2[km * hP + pp], fs[1]);
      fd[1] = fmac(md, g2[hS + km * hP + pp], fd[1]);
    }
    const long long blk = b0 + bb;
    const C kap = (C)p.kap[blk], ks = (C)p.kaps[blk];
    // omega.G at (k, m) and (k, m + NP/2): cos(Th) G_r +- sin(Th) gc; omega.G2.omega:
    // cos^2(Th) G2_rr + sin^2(Th) gq +- 2 cos(Th) sin(Th) gr2
    const C cpm = t.cosP[m], spm = t.sinP[m];
    const C gc = aniso ? cpm * sSum[2 * nb + bb] + spm * sSum[3 * nb + bb] : (C)0;
    C gq = 0, gr2 = 0;
    if (quad) {
      gq = cpm * cpm * sSum[5 * nb + bb] + spm * spm * sSum[6 * nb + bb] +
           (C)2 * cpm * spm * sSum[7 * nb + bb];
      gr2 = (C)2 * (cpm * sSum[8 * nb + bb] + spm * sSum[9 * nb + bb]);
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int kr = side ? km : k;
      const C sg = side ? (C)-1 : (C)1;
      const C ps = (C)0.5 * (aO + sg * aE), qd = (C)0.5 * (bO + sg * bE);
      const C f1 = (C)0.5 * (fs[side] + fd[side]), f2 = (C)0.5 * (fs[side] - fd[side]);
      const long long gi = blk * S + kr * NP + m;
      C qs = t.qdir[kr] * sSum[bb], qa = 0;
      if (aniso) {
        const C ct = t.cosT[kr], st = t.sinT[kr];
        qs += t.qdir[kr] * ct * sSum[nb + bb];
        qa = t.qdir[kr] * st * gc;
        if (quad) {
          qs += t.qdir[kr] * (ct * ct * sSum[4 * nb + bb] + st * st * gq -
                              sSum[10 * nb + bb] * ((C)1 / (C)3));
          qa += t.qdir[kr] * ct * st * gr2;
        }
      }
      const C ub1 = (C)Ubar[gi] - (ps + qd) - f1 - (kap + ks) * (C)lt[gi] + qs + qa;
      const C ub2 = (C)Ubar[gi + hP] - (ps - qd) - f2 - (kap + ks) * (C)lt[gi + hP] + qs - qa;
      lam_out[gi] = (T)((C)lam_in[gi] + ub1);
      lam_out[gi + hP] = (T)((C)lam_in[gi + hP] + ub2);
      if (Kbar_out) {
        Kbar_out[gi] = (T)(wl * (C)lam[gi] + wu * ub1);
        Kbar_out[gi + hP] = (T)(wl * (C)lam[gi + hP] + wu * ub2);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Split scheme: backward-Euler collision step in closed form per angular block,
//   J+ = (J* + dt eta)/(1 + dt kappa),  F+ = (F* + dt (eta + kappa_s J+))/(1 + dt (kappa+kappa_s)),
// with an anisotropic kernel also H+ = H*/(1 + dt (kappa + kappa_s) - dt kappa_s b/3),
// M~+ = M~*/(1 + dt (kappa + kappa_s) - dt kappa_s 2c/15) and
// F+ += dt kappa_s (b omega.H+ + c omega.M~+.omega) / (1 + dt (kappa+kappa_s)): the
// quadrature integrates the products of up to four components of omega exactly
// (NTheta, NPhi >= 3 for b, >= 6 for c), so (1/4pi) sum q omega_i omega_j = delta_ij/3
// and M~ of omega.A.omega is 2A/15 for traceless A, and the odd moments of even
// functions vanish by symmetry. Then F = inflow data at the inflow nodes (if the
// grid has Tau rows).
template <typename T, typename C>
__device__ __forceinline__ void implicit_collision_tile(const Problem& p, const Tables<C>& t,
                                                        T* F, double dt, int nb,
                                                        long long tile) {
  // Computed in double for every storage type: the stiff collision update
  // (dt kappa up to 1e2) is kept in FP64 on the GPU.
  const Dims d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP, hT = NT / 2;
  const long long b0 = tile * nb;
  const int nbb = (int)min((long long)nb, d.nblk - b0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int kf = kernel_form(p, 1);
  const bool aniso = kf >= KF_LINEAR, quad = kf >= KF_QUADRATIC;
  for (int bb = warp; bb < nbb; bb += nw) {
    const long long blk = b0 + bb;
    double acc = 0, mo[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // H (3), M (6: rr thth phph thph rth rph)
    for (int x = lane; x < S; x += 32) {
      const int k = x / NP, m = x - k * NP;
      const double u = (double)F[blk * S + x];
      acc = fma((double)t.qdir[k], u, acc);
      if (aniso) {
        const double ct = (double)t.cosT[k], cp = (double)t.cosP[m], sp = (double)t.sinP[m];
        const double qu = (double)t.qdir[k] * u, qs = (double)t.sinT[k] * qu;
        mo[0] = fma(ct, qu, mo[0]);
        mo[1] = fma(cp, qs, mo[1]);
        mo[2] = fma(sp, qs, mo[2]);
        if (quad) {
          const double qss = (double)t.sinT[k] * qs;
          mo[3] = fma(ct * ct, qu, mo[3]);
          mo[4] = fma(cp * cp, qss, mo[4]);
          mo[5] = fma(sp * sp, qss, mo[5]);
          mo[6] = fma(cp * sp, qss, mo[6]);
          mo[7] = fma(ct * cp, qs, mo[7]);
          mo[8] = fma(ct * sp, qs, mo[8]);
        }
      }
    }
    const int nm = quad ? 9 : aniso ? 3 : 0;   // uniform over the block
    for (int o = 16; o; o >>= 1) {
      acc += __shfl_xor_sync(0xffffffffu, acc, o);
#pragma unroll
      for (int a = 0; a < 9; ++a)   // constant indices keep mo in registers
        if (a < nm) mo[a] += __shfl_xor_sync(0xffffffffu, mo[a], o);
    }
    const double kap = p.kap[blk], eta = p.eta[blk], ks = p.kaps[blk];
    const double Jp = (acc + dt * eta) / (1.0 + dt * kap);
    const double num = dt * (eta + ks * Jp), den = 1.0 + dt * (kap + ks);
    double kbr = 0, kbt = 0, kbp = 0;   // dt kappa_s b H+
    double q6[6] = {0, 0, 0, 0, 0, 0};  // dt kappa_s c M~+ (rr thth phph, 2 thph, 2 rth, 2 rph)
    if (aniso && p.scb) {
      const double kb = ks * p.scb[blk], f = dt * kb / (den - dt * kb / 3.0);
      kbr = f * mo[0];
      kbt = f * mo[1];
      kbp = f * mo[2];
    }
    if (quad) {
      const double kc = ks * p.scc[blk], f = dt * kc / (den - dt * kc * (2.0 / 15.0));
      const double j3 = acc / 3.0;
      q6[0] = f * (mo[3] - j3);
      q6[1] = f * (mo[4] - j3);
      q6[2] = f * (mo[5] - j3);
      q6[3] = 2.0 * f * mo[6];
      q6[4] = 2.0 * f * mo[7];
      q6[5] = 2.0 * f * mo[8];
    }
    int g, i, j, l;
    decode_block(d, blk, g, i, j, l);
    const T* g1 = reinterpret_cast<const T*>(p.gR1);
    const T* g2 = reinterpret_cast<const T*>(p.gR2);
    for (int x = lane; x < S; x += 32) {
      const int k = x / NP, m = x - k * NP;
      double v = (double)F[blk * S + x] + num;
      if (aniso) {
        const double ct = (double)t.cosT[k], st = (double)t.sinT[k];
        const double cp = (double)t.cosP[m], sp = (double)t.sinP[m];
        v += ct * kbr + st * (cp * kbt + sp * kbp);
        if (quad)
          v += ct * ct * q6[0] + st * st * (cp * cp * q6[1] + sp * sp * q6[2] + cp * sp * q6[3]) +
               ct * st * (cp * q6[4] + sp * q6[5]);
      }
      v /= den;
      if (p.bc == TS_BC_TAU_INFLOW) {
        const long long pos = (((long long)g * d.Nt + j) * d.Np + l) * hT;
        if (i == 0 && k < hT) v = g1 ? (double)g1[(pos + k) * NP + m] : 0.0;
        if (i == d.Nr - 1 && k >= hT) v = g2 ? (double)g2[(pos + k - hT) * NP + m] : 0.0;
      }
      F[blk * S + x] = (T)v;
    }
  }
}

template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_implicit_collision(Problem p, Tables<C> t, T* F, double dt, int nb) {
  implicit_collision_tile<T, C>(p, t, F, dt, nb, blockIdx.x);
}

// F = inflow data at the inflow nodes.
template <typename T>
__global__ void k_apply_inflow(Problem p, T* F) {
  const Dims d = p.d;
  const int hT = d.NT / 2;
  const long long n = (long long)d.G * d.Nt * d.Np * d.NT * d.NP;  // one value per (g,j,l,k,m)
  const T* g1 = reinterpret_cast<const T*>(p.gR1);
  const T* g2 = reinterpret_cast<const T*>(p.gR2);
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n;
       x += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(x % d.NP);
    long long q = x / d.NP;
    const int k = (int)(q % d.NT);
    q /= d.NT;
    const int l = (int)(q % d.Np);
    q /= d.Np;
    const int j = (int)(q % d.Nt);
    const int g = (int)(q / d.Nt);
    const long long pos = (((long long)g * d.Nt + j) * d.Np + l) * hT;
    const long long off = (long long)j * d.S_j + (long long)l * d.S_l + (long long)k * d.NP + m;
    if (k < hT)
      F[(long long)g * d.S_g + off] = g1 ? g1[(pos + k) * d.NP + m] : (T)0;
    else
      F[(long long)g * d.S_g + (long long)(d.Nr - 1) * d.S_i + off] =
          g2 ? g2[(pos + k - hT) * d.NP + m] : (T)0;
  }
}

// ----------------------------------------------------------------------------
// Filter, one axis per launch (off the hot loop): out = M along `axis`,
// with the DFS partner term for theta (axis 1) and Theta (axis 3).
// M1T, M2T are [in][out].
template <typename T, typename C>
__global__ void k_filter_axis(Problem p, const C* __restrict__ M1T, const C* __restrict__ M2T,
                              int axis, const T* __restrict__ in, T* __restrict__ out) {
  const Dims d = p.d;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < d.total;
       x += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(x % d.NP);
    long long q = x / d.NP;
    const int k = (int)(q % d.NT);
    q /= d.NT;
    const int l = (int)(q % d.Np);
    q /= d.Np;
    const int j = (int)(q % d.Nt);
    q /= d.Nt;
    const int i = (int)(q % d.Nr);
    const int g = (int)(q / d.Nr);
    const long long g0 = (long long)g * d.S_g;
    C a = 0;
    if (axis == 0) {
      const long long b = g0 + (long long)j * d.S_j + (long long)l * d.S_l + k * d.NP + m;
      for (int n = 0; n < d.Nr; ++n) a = fmac(M1T[n * d.Nr + i], (C)in[b + n * d.S_i], a);
    } else if (axis == 1) {
      const int lh = (l + d.Np / 2) % d.Np, mh = (m + d.NP / 2) % d.NP;
      const long long b = g0 + (long long)i * d.S_i + (long long)l * d.S_l + k * d.NP + m;
      const long long bh = g0 + (long long)i * d.S_i + (long long)lh * d.S_l + k * d.NP + mh;
      for (int n = 0; n < d.Nt; ++n) {
        a = fmac(M1T[n * d.Nt + j], (C)in[b + n * d.S_j], a);
        a = fmac(M2T[n * d.Nt + j], (C)in[bh + n * d.S_j], a);
      }
    } else if (axis == 2) {
      const long long b = g0 + (long long)i * d.S_i + (long long)j * d.S_j + k * d.NP + m;
      for (int n = 0; n < d.Np; ++n) a = fmac(M1T[n * d.Np + l], (C)in[b + n * d.S_l], a);
    } else if (axis == 3) {
      const int mh = (m + d.NP / 2) % d.NP;
      const long long b = x - (long long)k * d.NP - m;
      for (int n = 0; n < d.NT; ++n) {
        a = fmac(M1T[n * d.NT + k], (C)in[b + n * d.NP + m], a);
        a = fmac(M2T[n * d.NT + k], (C)in[b + n * d.NP + mh], a);
      }
    } else {
      const long long b = x - m;
      for (int n = 0; n < d.NP; ++n) a = fmac(M1T[n * d.NP + m], (C)in[b + n], a);
    }
    out[x] = (T)a;
  }
}

// ----------------------------------------------------------------------------
// Moments (App. A, App. C). One warp per angular block (double arithmetic):
// S0 = sum q_k F, Sr = sum q_k cos(Th) F, St = sum q_k sin(Th)cos(Ph) F,
// Sp = sum q_k sin(Th) sin(Ph) F with q_k = Fejer_k (2pi/NP)/(4pi). F0 = S0 and
// F1 is (Sr, St, Sp) rotated from the local (rhat, thetahat, phihat) frame to
// Cartesian axes (Eqs. omegax-omegaz). Per-block contributions to N and to the
// fluxes go to partN/partJ and are summed per group by k_moments_reduce in a
// fixed order (deterministic).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_moments(Problem p, Tables<double> t, const double* __restrict__ wr,
          const double* __restrict__ wth, const T* __restrict__ F, double* F0, double* F1,
          double* partN, double* partJ, double R1, double R2) {
  const Dims d = p.d;
  const int NP = d.NP, S = d.NT * NP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long blk = blockIdx.x * (long long)(blockDim.x >> 5) + warp;
  if (blk >= d.nblk) return;
  double s0 = 0, sr = 0, st = 0, sp = 0;
  for (int x = lane; x < S; x += 32) {
    const int k = x / NP, m = x - k * NP;
    const double v = t.qdir[k] * (double)F[blk * S + x];
    s0 += v;
    sr = fma(v, t.cosT[k], sr);
    st = fma(v, t.sinT[k] * t.cosP[m], st);
    sp = fma(v, t.sinT[k] * t.sinP[m], sp);
  }
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    st += __shfl_xor_sync(0xffffffffu, st, o);
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
  }
  if (lane != 0) return;
  int g, i, j, l;
  decode_block(d, blk, g, i, j, l);
  const double sth = t.sin_th[j], cth = t.cos_th[j], sph = t.sin_ph[l], cph = t.cos_ph[l];
  if (F0) F0[blk] = s0;
  if (F1) {
    F1[blk] = sr * sth * cph + st * cth * cph - sp * sph;
    F1[d.nblk + blk] = sr * sth * sph + st * cth * sph + sp * cph;
    F1[2 * d.nblk + blk] = sr * cth - st * sth;
  }
  const double area = wth[j] * (2.0 * M_PI / d.Np) * 4.0 * M_PI;  // position-angle weight x 4 pi
  partN[blk] = wr[i] * area * s0;
  const long long pos = (long long)j * d.Np + l;
  if (i == 0) partJ[((long long)g * 2 + 0) * d.Nt * d.Np + pos] = R1 * R1 * area * sr;
  if (i == d.Nr - 1) partJ[((long long)g * 2 + 1) * d.Nt * d.Np + pos] = R2 * R2 * area * sr;
}

static __global__ void k_moments_reduce(Dims d, const double* partN, const double* partJ, double* N,
                                 double* JR1, double* JR2) {
  __shared__ double red[3][kThreads];
  const int g = blockIdx.x;
  const long long nN = (long long)d.Nr * d.Nt * d.Np, nJ = (long long)d.Nt * d.Np;
  double a = 0, b = 0, c = 0;
  for (long long x = threadIdx.x; x < nN; x += blockDim.x) a += partN[g * nN + x];
  for (long long x = threadIdx.x; x < nJ; x += blockDim.x) {
    b += partJ[(g * 2 + 0) * nJ + x];
    c += partJ[(g * 2 + 1) * nJ + x];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < 3; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (N) N[g] = red[0][0];
    if (JR1) JR1[g] = red[1][0];
    if (JR2) JR2[g] = red[2][0];
  }
}

}  // namespace ts
