// Register-blocked forms of the three forward passes.
//
// Each pass is a batch of small matrix products (the per-axis derivative
// matrices against the staged lines). Here every thread owns an RB x 4 block of
// outputs, so one shared-memory load feeds several multiply-adds, and the
// derivative matrices are used in even/odd form:
//  * DFS axes (theta with partner (phi+pi, Phi+pi); Theta with partner Phi+pi):
//    the outputs at a node and at its partner come from P (F + F') and
//    Q (F - F') with P = (A+B)/2, Q = (A-B)/2 -- half the multiply-adds;
//  * r: the Gauss-Lobatto differentiation matrix is centro-antisymmetric, so
//    the outputs at i and N-i come from E = u_i' + u_{N-i'} and
//    O = u_i' - u_{N-i'} against half-size matrices -- half the multiply-adds.
// Requirements (checked on the host): NT, Nt multiples of RB, NP a multiple
// of 8, plane columns per half (c) a multiple of 4, Nr/2 a multiple of RB.
// Results equal the generic passes up to rounding.
#pragma once

#include "ts_kernels.cuh"

namespace ts {

template <typename C>
__device__ __forceinline__ void ld4(const C* p, C (&v)[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename C>
__device__ __forceinline__ void st4(C* p, const C (&v)[4]);
template <>
__device__ __forceinline__ void st4<float>(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
template <typename C, int RB>
__device__ __forceinline__ void ldr(const C* p, C (&v)[RB]) {
#pragma unroll
  for (int r = 0; r < RB; ++r) v[r] = p[r];
}

// RB for the angular pass (rows of Theta per thread); kRBPlane, kRBRad in ts_internal.h.
template <typename C> struct RBAng { static constexpr int v = sizeof(C) == 4 ? 4 : 2; };

// ----------------------------------------------------------------------------
// Angular pass. Thread: RB Theta rows k0.. x 4 column pairs (m, m + NP/2) of one block.
template <typename T, typename C>
__device__ __forceinline__ void angular_tile_rb(const Problem& p, const Tables<C>& t,
                                                const T* __restrict__ U, T* __restrict__ K,
                                                C sgn, int collision, int nb, long long tile) {
  constexpr int RB = RBAng<C>::v, CB = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP, hP = NP / 2;
  C* sP = reinterpret_cast<C*>(smem_raw);  // PThT [k'][k]
  C* sQ = sP + NT * NT;                    // QThT [k'][k]
  C* sD = sQ + NT * NT;                    // DPhT [m'][m]
  C* su = sD + NP * NP;                    // [bb][k][m]
  C* sc = su + nb * S;                     // J, kappa, eta, kappa_s per block
  const long long b0 = tile * nb;
  const int nbb = (int)min((long long)nb, d.nblk - b0);
  for (int x = threadIdx.x; x < NT * NT; x += blockDim.x) {
    sP[x] = t.PThT[x];
    sQ[x] = t.QThT[x];
  }
  for (int x = threadIdx.x; x < NP * NP; x += blockDim.x) sD[x] = t.DPhT[x];
  const T* src = U + b0 * S;
  for (int x = 4 * threadIdx.x; x < nbb * S; x += 4 * blockDim.x) {
    T v[4];
    ld4<T>(src + x, v);
    C w[4] = {(C)v[0], (C)v[1], (C)v[2], (C)v[3]};
    st4<C>(su + x, w);
  }
  for (int x = threadIdx.x; x < nbb; x += blockDim.x) {  // one conversion per block
    sc[nb + x] = (C)p.kap[b0 + x];
    sc[2 * nb + x] = (C)p.eta[b0 + x];
    sc[3 * nb + x] = (C)p.kaps[b0 + x];
  }
  __syncthreads();
  if (collision) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bb = warp; bb < nbb; bb += blockDim.x >> 5) {
      C acc = 0;
      for (int x = lane; x < S; x += 32) acc = fmac(t.qdir[x / NP], su[bb * S + x], acc);
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) sc[bb] = acc;
    }
    __syncthreads();
  }
  const int KR = NT / RB, PC = hP / CB;
  const int units = nbb * KR * PC;
  for (int unit = threadIdx.x; unit < units; unit += blockDim.x) {
    const int pc = unit % PC, rest = unit / PC, kr = rest % KR, bb = rest / KR;
    const int p0 = pc * CB, k0 = kr * RB;
    const C* ub = su + bb * S;
    C ps[RB][CB], qd[RB][CB], da[RB][CB], db[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < CB; ++c) ps[r][c] = qd[r][c] = da[r][c] = db[r][c] = 0;
    for (int kk = 0; kk < NT; ++kk) {
      C a[CB], b[CB], P[RB], Q[RB];
      ld4<C>(ub + kk * NP + p0, a);
      ld4<C>(ub + kk * NP + p0 + hP, b);
      ldr<C, RB>(sP + kk * NT + k0, P);
      ldr<C, RB>(sQ + kk * NT + k0, Q);
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const C sv = a[c] + b[c], dv = a[c] - b[c];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          ps[r][c] = fmac(P[r], sv, ps[r][c]);
          qd[r][c] = fmac(Q[r], dv, qd[r][c]);
        }
      }
    }
    for (int mm = 0; mm < NP; ++mm) {
      C A4[CB], B4[CB];
      ld4<C>(sD + mm * NP + p0, A4);
      ld4<C>(sD + mm * NP + p0 + hP, B4);
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const C uv = ub[(k0 + r) * NP + mm];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          da[r][c] = fmac(A4[c], uv, da[r][c]);
          db[r][c] = fmac(B4[c], uv, db[r][c]);
        }
      }
    }
    const long long blk = b0 + bb;
    int g, i, j, l;
    decode_block(d, blk, g, i, j, l);
    const C ir = t.inv_r[i], ct = t.cot_th[j];
    const C J = sc[bb], kap = sc[nb + bb], eta = sc[2 * nb + bb], ks = sc[3 * nb + bb];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int k = k0 + r;
      const C aT = -t.sinT[k] * ir;
      C v1[CB], v2[CB], u1[CB], u2[CB];
      ld4<C>(ub + k * NP + p0, u1);
      ld4<C>(ub + k * NP + p0 + hP, u2);
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const int m = p0 + c;
        v1[c] = sgn * aT * (ps[r][c] + qd[r][c] + t.sinP[m] * ct * da[r][c]);
        v2[c] = sgn * aT * (ps[r][c] - qd[r][c] + t.sinP[m + hP] * ct * db[r][c]);
        if (collision) {
          v1[c] += eta - (kap + ks) * u1[c] + ks * J;
          v2[c] += eta - (kap + ks) * u2[c] + ks * J;
        }
      }
      T* out = K + blk * S + k * NP + p0;
      T o1[CB] = {(T)v1[0], (T)v1[1], (T)v1[2], (T)v1[3]};
      T o2[CB] = {(T)v2[0], (T)v2[1], (T)v2[2], (T)v2[3]};
      st4<T>(out, o1);
      st4<T>(out + hP, o2);
    }
  }
}

// ----------------------------------------------------------------------------
// Plane pass. Thread: RB theta rows j0.. x 4 columns w0.. at phi l < Np/2, and the
// partner outputs (l + Np/2, w0^..) of the same E/O pair.
template <typename T, typename C>
__device__ __forceinline__ void plane_tile_rb(const Problem& p, const Tables<C>& t,
                                              const T* __restrict__ U, T* __restrict__ K, C sgn,
                                              int c, long long tile) {
  constexpr int RB = kRBPlane, CB = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nt = d.Nt, Np = d.Np, NP = d.NP, hP = NP / 2, hp = Np / 2, W = 2 * c;
  C* sP = reinterpret_cast<C*>(smem_raw);  // PthT [j'][j]
  C* sQ = sP + Nt * Nt;
  C* sD = sQ + Nt * Nt;                    // DphT [l'][l]
  C* su = sD + Np * Np + ((Np * Np) & 3 ? 4 - ((Np * Np) & 3) : 0);  // [j][l][w], 16B aligned
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
    sP[x] = t.PthT[x];
    sQ[x] = t.QthT[x];
  }
  for (int x = threadIdx.x; x < Np * Np; x += blockDim.x) sD[x] = t.DphT[x];
  const int nq = Nt * Np * (W / 4);
  for (int x = threadIdx.x; x < nq; x += blockDim.x) {
    const int w4 = (x % (W / 4)) * 4, jl = x / (W / 4), l = jl % Np, j = jl / Np;
    T v[4];
    ld4<T>(U + base + (long long)j * d.S_j + (long long)l * d.S_l + plane_m(w4, c, m0, hP), v);
    C w[4] = {(C)v[0], (C)v[1], (C)v[2], (C)v[3]};
    st4<C>(su + jl * W + w4, w);
  }
  __syncthreads();
  const C sTk = t.sinT[k], ir = t.inv_r[i];
  const int JR = Nt / RB, WQ = W / CB;
  const int units = JR * hp * WQ;
  for (int unit = threadIdx.x; unit < units; unit += blockDim.x) {
    const int wq = unit % WQ, rest = unit / WQ, l = rest % hp, jr = rest / hp;
    const int w0 = wq * CB, j0 = jr * RB;
    const int w0h = w0 < c ? w0 + c : w0 - c, lh = l + hp;
    C ps[RB][CB], qd[RB][CB], da[RB][CB], db[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) ps[r][cc] = qd[r][cc] = da[r][cc] = db[r][cc] = 0;
    for (int jj = 0; jj < Nt; ++jj) {
      C a[CB], b[CB], P[RB], Q[RB];
      ld4<C>(su + (jj * Np + l) * W + w0, a);
      ld4<C>(su + (jj * Np + lh) * W + w0h, b);
      ldr<C, RB>(sP + jj * Nt + j0, P);
      ldr<C, RB>(sQ + jj * Nt + j0, Q);
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
        const C sv = a[cc] + b[cc], dv = a[cc] - b[cc];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          ps[r][cc] = fmac(P[r], sv, ps[r][cc]);
          qd[r][cc] = fmac(Q[r], dv, qd[r][cc]);
        }
      }
    }
    for (int ll = 0; ll < Np; ++ll) {
      const C Dl = sD[ll * Np + l], Dh = sD[ll * Np + lh];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        C a[CB], b[CB];
        ld4<C>(su + ((j0 + r) * Np + ll) * W + w0, a);
        ld4<C>(su + ((j0 + r) * Np + ll) * W + w0h, b);
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) {
          da[r][cc] = fmac(Dl, a[cc], da[r][cc]);
          db[r][cc] = fmac(Dh, b[cc], db[r][cc]);
        }
      }
    }
    const int mA = plane_m(w0, c, m0, hP), mB = plane_m(w0h, c, m0, hP);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int j = j0 + r;
      const C isn = t.inv_sinth[j];
      T* pa = K + base + (long long)j * d.S_j + (long long)l * d.S_l + mA;
      T* pb = K + base + (long long)j * d.S_j + (long long)lh * d.S_l + mB;
      T ka[CB], kb[CB];
      ld4<T>(pa, ka);
      ld4<T>(pb, kb);
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
        const C athA = sTk * t.cosP[mA + cc] * ir, aphA = sTk * t.sinP[mA + cc] * ir * isn;
        const C athB = sTk * t.cosP[mB + cc] * ir, aphB = sTk * t.sinP[mB + cc] * ir * isn;
        ka[cc] = (T)((C)ka[cc] + sgn * (athA * (ps[r][cc] + qd[r][cc]) + aphA * da[r][cc]));
        kb[cc] = (T)((C)kb[cc] + sgn * (athB * (ps[r][cc] - qd[r][cc]) + aphB * db[r][cc]));
      }
      st4<T>(pa, ka);
      st4<T>(pb, kb);
    }
  }
}

// ----------------------------------------------------------------------------
// Radial pass. Thread: RB output pairs (i, N-i) x 4 columns; the middle node
// (odd Nr) by separate units; rows 0..n64-1 and N-n64+1..N (n64 = p.n_fp64_rows)
// in double from the full matrix. Then the Tau rows and the stage update.
template <typename T, typename C>
__device__ __forceinline__ void radial_tile_rb(const Problem& p, const Tables<C>& t,
                                               const double* __restrict__ Dr64, const T* U,
                                               const T* Kin, C sgn, int tau, int mode, T* F,
                                               T* Acc, T* Uout, T* out, C dt, int W,
                                               long long tile) {
  constexpr int RB = kRBRad, CB = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nr = d.Nr, N = Nr - 1, hh = Nr / 2, NP = d.NP, S = d.NT * d.NP;
  const int hh4 = (hh * hh + 3) & ~3, h4 = (hh + 3) & ~3;
  C* sE = reinterpret_cast<C*>(smem_raw);  // EpT [i'][i]
  C* sO = sE + hh4;                        // OpT [i'][i]
  C* sMc = sO + hh4;                       // D[i][M]
  C* sMr = sMc + h4;                       // D[M][i']
  C* su = sMr + h4;                        // [i][w]
  C* sk = su + Nr * W;                     // [i][w]
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
  for (int x = threadIdx.x; x < hh * hh; x += blockDim.x) {
    sE[x] = t.EpT[x];
    sO[x] = t.OpT[x];
  }
  for (int x = threadIdx.x; x < hh; x += blockDim.x) {
    sMc[x] = t.DrMc[x];
    sMr[x] = t.DrMr[x];
  }
  const int W4 = Wc / 4;
  for (int x = threadIdx.x; x < Nr * W4; x += blockDim.x) {
    const int ii = x / W4, w = (x - ii * W4) * 4;
    const long long gi = base + (long long)ii * d.S_i + w;
    T a[4], b[4];
    ld4<T>(U + gi, a);
    ld4<T>(Kin + gi, b);
    C ca[4] = {(C)a[0], (C)a[1], (C)a[2], (C)a[3]};
    C cb[4] = {(C)b[0], (C)b[1], (C)b[2], (C)b[3]};
    st4<C>(su + ii * W + w, ca);
    st4<C>(sk + ii * W + w, cb);
  }
  __syncthreads();
  const int n64 = p.n_fp64_rows;
  const int IR = hh / RB;
  const int units = IR * W4 + ((Nr & 1) ? W4 : 0) + 2 * n64 * W4;
  for (int unit = threadIdx.x; unit < units; unit += blockDim.x) {
    if (unit < IR * W4) {
      const int wq = unit % W4, ir = unit / W4;
      const int w0 = wq * CB, i0 = ir * RB;
      C ae[RB][CB], ao[RB][CB];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) ae[r][cc] = ao[r][cc] = 0;
      for (int ii = 0; ii < hh; ++ii) {
        C a[CB], b[CB], E[RB], O[RB];
        ld4<C>(su + ii * W + w0, a);
        ld4<C>(su + (N - ii) * W + w0, b);
        ldr<C, RB>(sE + ii * hh + i0, E);
        ldr<C, RB>(sO + ii * hh + i0, O);
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) {
          const C ev = a[cc] + b[cc], ov = a[cc] - b[cc];
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            ae[r][cc] = fmac(E[r], ev, ae[r][cc]);
            ao[r][cc] = fmac(O[r], ov, ao[r][cc]);
          }
        }
      }
      if (Nr & 1) {
        C um[CB];
        ld4<C>(su + (N / 2) * W + w0, um);
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int cc = 0; cc < CB; ++cc) ae[r][cc] = fmac((C)2 * sMc[i0 + r], um[cc], ae[r][cc]);
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = i0 + r;
        if (i < n64) continue;  // those rows are done in double below
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) {
          const C ck = sgn * t.cosT[(c0 + w0 + cc) / NP] * (C)0.5;
          sk[i * W + w0 + cc] += ck * (ao[r][cc] + ae[r][cc]);
          sk[(N - i) * W + w0 + cc] += ck * (ao[r][cc] - ae[r][cc]);
        }
      }
    } else if (unit < IR * W4 + ((Nr & 1) ? W4 : 0)) {
      const int w0 = (unit - IR * W4) * CB;
      C am[CB] = {0, 0, 0, 0};
      for (int ii = 0; ii < hh; ++ii) {
        C a[CB], b[CB];
        ld4<C>(su + ii * W + w0, a);
        ld4<C>(su + (N - ii) * W + w0, b);
        const C mr = sMr[ii];
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) am[cc] = fmac(mr, a[cc] - b[cc], am[cc]);
      }
#pragma unroll
      for (int cc = 0; cc < CB; ++cc)
        sk[(N / 2) * W + w0 + cc] += sgn * t.cosT[(c0 + w0 + cc) / NP] * am[cc];
    } else {
      // rows nearest the ends, accumulated in double from the full matrix
      const int v = unit - IR * W4 - ((Nr & 1) ? W4 : 0);
      const int w0 = (v % W4) * CB, rr = v / W4;
      const int i = rr < n64 ? rr : N - (rr - n64);
      double a[CB] = {0, 0, 0, 0};
      for (int ii = 0; ii < Nr; ++ii) {
        const double dv = Dr64[i * Nr + ii];
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) a[cc] = fma(dv, (double)su[ii * W + w0 + cc], a[cc]);
      }
#pragma unroll
      for (int cc = 0; cc < CB; ++cc)
        sk[i * W + w0 + cc] += sgn * t.cosT[(c0 + w0 + cc) / NP] * (C)a[cc];
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < Nr * W4; x += blockDim.x) {
    const int i = x / W4, w = (x - i * W4) * 4;
    const long long gi = base + (long long)i * d.S_i + w;
    C kv[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      kv[cc] = sk[i * W + w + cc];
      if (tau) {
        const int k = (c0 + w + cc) / NP;
        const int b = t.cosT[k] > (C)0 ? 0 : Nr - 1;
        kv[cc] -= sk[b * W + w + cc] * t.tsign[b] * t.tsign[i];
      }
    }
    T o[4];
    if (mode == RAD_RHS) {
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) o[cc] = (T)kv[cc];
      st4<T>(out + gi, o);
    } else if (mode == RAD_STAGE3) {
      T f[4], ac[4];
      ld4<T>(F + gi, f);
      ld4<T>(Acc + gi, ac);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) o[cc] = (T)((C)f[cc] + dt / (C)6 * ((C)ac[cc] + kv[cc]));
      st4<T>(F + gi, o);
    } else {
      T f[4], ac[4];
      ld4<T>(F + gi, f);
      const C cu = mode == RAD_STAGE2 ? dt : (C)0.5 * dt;
      if (mode != RAD_STAGE0) ld4<T>(Acc + gi, ac);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        o[cc] = (T)((C)f[cc] + cu * kv[cc]);
        ac[cc] = mode == RAD_STAGE0 ? (T)kv[cc] : (T)((C)ac[cc] + (C)2 * kv[cc]);
      }
      st4<T>(Acc + gi, ac);
      st4<T>(Uout + gi, o);
    }
  }
}

// ----------------------------------------------------------------------------
// Pass dispatch (register-blocked form where the grid allows it) and the
// single-problem kernels: one tile per CTA.
template <typename T, typename C>
__device__ __forceinline__ void angular_tile_any(const Problem& p, const Tables<C>& t,
                                                 const T* U, T* K, C sgn, int collision, int nb,
                                                 long long tile) {
  if (p.tp.rb & 1) angular_tile_rb<T, C>(p, t, U, K, sgn, collision, nb, tile);
  else angular_tile<T, C>(p, t, U, K, sgn, collision, nb, tile);
}

template <typename T, typename C>
__device__ __forceinline__ void plane_tile_any(const Problem& p, const Tables<C>& t, const T* U,
                                               T* K, C sgn, int c, long long tile) {
  if (p.tp.rb & 2) plane_tile_rb<T, C>(p, t, U, K, sgn, c, tile);
  else plane_tile<T, C>(p, t, U, K, sgn, c, tile);
}

template <typename T, typename C>
__device__ __forceinline__ void radial_tile_any(const Problem& p, const Tables<C>& t,
                                                const double* Dr64, const T* U, const T* Kin,
                                                C sgn, int tau, int mode, T* F, T* Acc, T* Uout,
                                                T* out, C dt, int W, long long tile) {
  if (p.tp.rb & 4)
    radial_tile_rb<T, C>(p, t, Dr64, U, Kin, sgn, tau, mode, F, Acc, Uout, out, dt, W, tile);
  else
    radial_tile<T, C>(p, t, Dr64, U, Kin, sgn, tau, mode, F, Acc, Uout, out, dt, W, tile);
}

template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_angular(Problem p, Tables<C> t, const T* __restrict__ U, T* __restrict__ K, C sgn,
          int collision, int nb) {
  angular_tile_any<T, C>(p, t, U, K, sgn, collision, nb, blockIdx.x);
}

template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_plane(Problem p, Tables<C> t, const T* __restrict__ U, T* __restrict__ K, C sgn, int c) {
  plane_tile_any<T, C>(p, t, U, K, sgn, c, blockIdx.x);
}

template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_radial(Problem p, Tables<C> t, const double* __restrict__ Dr64, const T* U, const T* Kin,
         C sgn, int tau, int mode, T* F, T* Acc, T* Uout, T* out, C dt, int W) {
  radial_tile_any<T, C>(p, t, Dr64, U, Kin, sgn, tau, mode, F, Acc, Uout, out, dt, W,
                        blockIdx.x);
}

}  // namespace ts
