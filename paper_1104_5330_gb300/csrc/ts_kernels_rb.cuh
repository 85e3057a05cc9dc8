// Register-blocked forms of the three forward passes, and their persistent,
// double-buffered launches.
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
// The sums and differences are formed once per tile in shared memory.
//
// Every pass is split into a staging step (the tile's input lines into shared
// memory) and a compute step. The single-tile form stages synchronously (used
// by the batched kernels); the persistent kernels k_*_pp keep the derivative
// matrices in shared memory for all their tiles and stage tile t + gridDim.x
// with asynchronous 16-byte copies (cp.async) into a second buffer while tile
// t is computed.
//
// Requirements (checked on the host): NT, Nt multiples of RB, NP a multiple
// of 8, plane columns per half (c) a multiple of 4, Nr/2 a multiple of RB.
// Results equal the generic passes up to rounding.
#pragma once

#include <stdint.h>

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

// Four consecutive elements global -> shared: plain (convert T -> C) or as
// asynchronous 16-byte copies (T == C), completed by cp.async.wait_group.
template <bool ASYNC, typename T, typename C>
__device__ __forceinline__ void copy4(C* dst, const T* src) {
  if constexpr (ASYNC) {
    static_assert(sizeof(T) == sizeof(C), "async staging copies raw elements");
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
#pragma unroll
    for (int h = 0; h < (int)sizeof(T) * 4 / 16; ++h)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                   :: "r"(d + 16 * h), "l"(reinterpret_cast<const char*>(src) + 16 * h)
                   : "memory");
  } else {
    T v[4];
    ld4<T>(src, v);
    C w[4] = {(C)v[0], (C)v[1], (C)v[2], (C)v[3]};
    st4<C>(dst, w);
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// RB for the angular pass (rows of Theta per thread); kRBPlane, kRBRad in ts_internal.h.
template <typename C> struct RBAng { static constexpr int v = sizeof(C) == 4 ? 4 : 2; };

// ============================================================================
// Angular pass. Thread: RB Theta rows k0.. x 4 column pairs (m, m + NP/2) of one block.
// Shared layout: [PThT | QThT | DPhT | tile buffer(s) nb*S | sums/diffs nb*S | 4 nb]
template <typename C>
__device__ __forceinline__ void angular_rb_mats(const Tables<C>& t, const Dims& d, C* sP, C* sQ,
                                                C* sD) {
  const int NT = d.NT, NP = d.NP;
  for (int x = threadIdx.x; x < NT * NT; x += blockDim.x) {
    sP[x] = t.PThT[x];
    sQ[x] = t.QThT[x];
  }
  for (int x = threadIdx.x; x < NP * NP; x += blockDim.x) sD[x] = t.DPhT[x];
}

template <bool ASYNC, typename T, typename C>
__device__ __forceinline__ void angular_rb_load(const Dims& d, const T* U, int nb, long long tile,
                                                C* su) {
  const int S = d.NT * d.NP;
  const long long b0 = tile * nb;
  const int nbb = (int)min((long long)nb, d.nblk - b0);
  const T* src = U + b0 * S;
  for (int x = 4 * threadIdx.x; x < nbb * S; x += 4 * blockDim.x) copy4<ASYNC, T, C>(su + x, src + x);
}

// Compute one staged tile. Entry: su complete and visible to all threads; sSD
// and sc free. Exit: all outputs written (sSD/sc may still be read until the
// caller's next barrier).
template <typename T, typename C>
__device__ __forceinline__ void angular_rb_body(const Problem& p, const Tables<C>& t,
                                                const C* su, C* sSD, C* sc, const C* sP,
                                                const C* sQ, const C* sD, T* __restrict__ K,
                                                C sgn, int collision, int nb, long long tile) {
  constexpr int RB = RBAng<C>::v, CB = 4;
  const Dims& d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP, hP = NP / 2;
  const long long b0 = tile * nb;
  const int nbb = (int)min((long long)nb, d.nblk - b0);
  for (int x = threadIdx.x; x < nbb; x += blockDim.x) {  // one conversion per block
    sc[nb + x] = (C)p.kap[b0 + x];
    sc[2 * nb + x] = (C)p.eta[b0 + x];
    sc[3 * nb + x] = (C)p.kaps[b0 + x];
  }
  // F + F(partner) and F - F(partner) once per pair (the partner of Phi_m is Phi_{m+NP/2})
  for (int x = threadIdx.x; x < nbb * NT * (hP / 4); x += blockDim.x) {
    const int p4 = (x % (hP / 4)) * 4, rest = x / (hP / 4), kk = rest % NT, bb = rest / NT;
    C a[4], b[4], s[4], df[4];
    ld4<C>(su + bb * S + kk * NP + p4, a);
    ld4<C>(su + bb * S + kk * NP + p4 + hP, b);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      s[c] = a[c] + b[c];
      df[c] = a[c] - b[c];
    }
    st4<C>(sSD + bb * S + kk * hP + p4, s);
    st4<C>(sSD + bb * S + NT * hP + kk * hP + p4, df);
  }
  if (collision) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bb = warp; bb < nbb; bb += blockDim.x >> 5) {
      C acc = 0;
      for (int x = lane; x < S; x += 32) acc = fmac(t.qdir[x / NP], su[bb * S + x], acc);
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) sc[bb] = acc;
    }
  }
  __syncthreads();
  const int KR = NT / RB, PC = hP / CB;
  const int units = nbb * KR * PC;
  for (int unit = threadIdx.x; unit < units; unit += blockDim.x) {
    const int pc = unit % PC, rest = unit / PC, kr = rest % KR, bb = rest / KR;
    const int p0 = pc * CB, k0 = kr * RB;
    const C* ub = su + bb * S;
    const C* us = sSD + bb * S;
    const C* ud = us + NT * hP;
    C ps[RB][CB], qd[RB][CB], da[RB][CB], db[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < CB; ++c) ps[r][c] = qd[r][c] = da[r][c] = db[r][c] = 0;
    for (int kk = 0; kk < NT; ++kk) {
      C sv[CB], dv[CB], P[RB], Q[RB];
      ld4<C>(us + kk * hP + p0, sv);
      ld4<C>(ud + kk * hP + p0, dv);
      ldr<C, RB>(sP + kk * NT + k0, P);
      ldr<C, RB>(sQ + kk * NT + k0, Q);
#pragma unroll
      for (int c = 0; c < CB; ++c) {
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          ps[r][c] = fmac(P[r], sv[c], ps[r][c]);
          qd[r][c] = fmac(Q[r], dv[c], qd[r][c]);
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

template <typename T, typename C>
__device__ __forceinline__ void angular_tile_rb(const Problem& p, const Tables<C>& t,
                                                const T* __restrict__ U, T* __restrict__ K,
                                                C sgn, int collision, int nb, long long tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP;
  C* sP = reinterpret_cast<C*>(smem_raw);
  C* sQ = sP + NT * NT;
  C* sD = sQ + NT * NT;
  C* su = sD + NP * NP;
  C* sSD = su + nb * S;
  C* sc = sSD + nb * S;
  angular_rb_mats<C>(t, d, sP, sQ, sD);
  angular_rb_load<false, T, C>(d, U, nb, tile, su);
  __syncthreads();
  angular_rb_body<T, C>(p, t, su, sSD, sc, sP, sQ, sD, K, sgn, collision, nb, tile);
}

template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_angular_pp(Problem p, Tables<C> t, const T* __restrict__ U, T* __restrict__ K, C sgn,
             int collision, int nb, long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP;
  C* sP = reinterpret_cast<C*>(smem_raw);
  C* sQ = sP + NT * NT;
  C* sD = sQ + NT * NT;
  C* sbuf[2] = {sD + NP * NP, sD + NP * NP + nb * S};
  C* sSD = sbuf[1] + nb * S;
  C* sc = sSD + nb * S;
  angular_rb_mats<C>(t, d, sP, sQ, sD);
  long long tile = blockIdx.x;
  if (tile < ntiles) angular_rb_load<true, T, C>(d, U, nb, tile, sbuf[0]);
  cp_async_commit();
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const long long next = tile + gridDim.x;
    if (next < ntiles) angular_rb_load<true, T, C>(d, U, nb, next, sbuf[(it + 1) & 1]);
    cp_async_commit();
    cp_async_wait1();  // this tile's copies (every group but the newest) have landed
    __syncthreads();
    angular_rb_body<T, C>(p, t, sbuf[it & 1], sSD, sc, sP, sQ, sD, K, sgn, collision, nb, tile);
    __syncthreads();   // buffer and scratch free before they are refilled
  }
  cp_async_wait0();
}

// ============================================================================
// Plane pass. Thread: RB theta rows j0.. x 4 columns w0.. at phi l < Np/2, and the
// partner outputs (l + Np/2, w0^..) of the same E/O pair.
// Shared layout: [PthT | QthT | DphT | tile buffer(s) Nt*Np*W | sums, diffs Nt*Np*W]
__device__ __forceinline__ void plane_tile_coords(const Dims& d, int c, long long tile, int& k,
                                                  int& i, int& g, int& m0) {
  const int nchunk = d.NP / 2 / c;
  long long q = tile;
  const int chunk = (int)(q % nchunk);
  q /= nchunk;
  k = (int)(q % d.NT);
  q /= d.NT;
  i = (int)(q % d.Nr);
  g = (int)(q / d.Nr);
  m0 = chunk * c;
}

template <typename C>
__device__ __forceinline__ void plane_rb_mats(const Tables<C>& t, const Dims& d, C* sP, C* sQ,
                                              C* sD) {
  const int Nt = d.Nt, Np = d.Np;
  for (int x = threadIdx.x; x < Nt * Nt; x += blockDim.x) {
    sP[x] = t.PthT[x];
    sQ[x] = t.QthT[x];
  }
  for (int x = threadIdx.x; x < Np * Np; x += blockDim.x) sD[x] = t.DphT[x];
}

template <bool ASYNC, typename T, typename C>
__device__ __forceinline__ void plane_rb_load(const Dims& d, const T* U, int c, long long tile,
                                              C* su) {
  int k, i, g, m0;
  plane_tile_coords(d, c, tile, k, i, g, m0);
  const int Np = d.Np, hP = d.NP / 2, W = 2 * c;
  const long long base = (long long)g * d.S_g + (long long)i * d.S_i + (long long)k * d.NP;
  const int nq = d.Nt * Np * (W / 4);
  for (int x = threadIdx.x; x < nq; x += blockDim.x) {
    const int w4 = (x % (W / 4)) * 4, jl = x / (W / 4), l = jl % Np, j = jl / Np;
    copy4<ASYNC, T, C>(su + jl * W + w4,
                       U + base + (long long)j * d.S_j + (long long)l * d.S_l + plane_m(w4, c, m0, hP));
  }
}

template <typename T, typename C>
__device__ __forceinline__ void plane_rb_body(const Problem& p, const Tables<C>& t, const C* su,
                                              C* sSm, const C* sP, const C* sQ, const C* sD,
                                              T* __restrict__ K, C sgn, int c, long long tile) {
  constexpr int RB = kRBPlane, CB = 4;
  const Dims& d = p.d;
  const int Nt = d.Nt, Np = d.Np, hP = d.NP / 2, hp = Np / 2, W = 2 * c;
  C* sDf = sSm + Nt * hp * W;
  int k, i, g, m0;
  plane_tile_coords(d, c, tile, k, i, g, m0);
  const long long base = (long long)g * d.S_g + (long long)i * d.S_i + (long long)k * d.NP;
  // sums and differences with the partner (phi + pi, Phi + pi) once per pair
  for (int x = threadIdx.x; x < Nt * hp * (W / 4); x += blockDim.x) {
    const int w4 = (x % (W / 4)) * 4, jl = x / (W / 4), l = jl % hp, jj = jl / hp;
    const int w4h = w4 < c ? w4 + c : w4 - c;
    C a[4], b[4], s[4], df[4];
    ld4<C>(su + (jj * Np + l) * W + w4, a);
    ld4<C>(su + (jj * Np + l + hp) * W + w4h, b);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      s[cc] = a[cc] + b[cc];
      df[cc] = a[cc] - b[cc];
    }
    st4<C>(sSm + jl * W + w4, s);
    st4<C>(sDf + jl * W + w4, df);
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
      C sv[CB], dv[CB], P[RB], Q[RB];
      ld4<C>(sSm + (jj * hp + l) * W + w0, sv);
      ld4<C>(sDf + (jj * hp + l) * W + w0, dv);
      ldr<C, RB>(sP + jj * Nt + j0, P);
      ldr<C, RB>(sQ + jj * Nt + j0, Q);
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          ps[r][cc] = fmac(P[r], sv[cc], ps[r][cc]);
          qd[r][cc] = fmac(Q[r], dv[cc], qd[r][cc]);
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

template <typename T, typename C>
__device__ __forceinline__ void plane_tile_rb(const Problem& p, const Tables<C>& t,
                                              const T* __restrict__ U, T* __restrict__ K, C sgn,
                                              int c, long long tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int Nt = d.Nt, Np = d.Np, W = 2 * c;
  C* sP = reinterpret_cast<C*>(smem_raw);  // PthT [j'][j]
  C* sQ = sP + Nt * Nt;
  C* sD = sQ + Nt * Nt;                    // DphT [l'][l]
  C* su = sD + Np * Np;                    // [j][l][w] (Np even: 16-byte aligned)
  C* sSm = su + Nt * Np * W;
  plane_rb_mats<C>(t, d, sP, sQ, sD);
  plane_rb_load<false, T, C>(d, U, c, tile, su);
  __syncthreads();
  plane_rb_body<T, C>(p, t, su, sSm, sP, sQ, sD, K, sgn, c, tile);
}

template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_plane_pp(Problem p, Tables<C> t, const T* __restrict__ U, T* __restrict__ K, C sgn, int c,
           long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int Nt = d.Nt, Np = d.Np, W = 2 * c, TS = Nt * Np * W;
  C* sP = reinterpret_cast<C*>(smem_raw);
  C* sQ = sP + Nt * Nt;
  C* sD = sQ + Nt * Nt;
  C* sbuf[2] = {sD + Np * Np, sD + Np * Np + TS};
  C* sSm = sbuf[1] + TS;
  plane_rb_mats<C>(t, d, sP, sQ, sD);
  long long tile = blockIdx.x;
  if (tile < ntiles) plane_rb_load<true, T, C>(d, U, c, tile, sbuf[0]);
  cp_async_commit();
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const long long next = tile + gridDim.x;
    if (next < ntiles) plane_rb_load<true, T, C>(d, U, c, next, sbuf[(it + 1) & 1]);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    plane_rb_body<T, C>(p, t, sbuf[it & 1], sSm, sP, sQ, sD, K, sgn, c, tile);
    __syncthreads();
  }
  cp_async_wait0();
}

// ============================================================================
// Radial pass. Thread: RB output pairs (i, N-i) x 4 columns; the middle node
// (odd Nr) by separate units; rows 0..n64-1 and N-n64+1..N (n64 = p.n_fp64_rows)
// in double from the full matrix. Then the Tau rows and the stage update.
// Shared layout: [EpT | OpT | DrMc | DrMr | (u, K) buffer(s) 2 Nr W | E, O 2 hh W]
__device__ __forceinline__ void radial_tile_coords(const Dims& d, int W, long long tile,
                                                   long long& base, int& c0, int& Wc) {
  const int S = d.NT * d.NP;
  const int nchunk = (S + W - 1) / W;
  long long q = tile;
  const int chunk = (int)(q % nchunk);
  q /= nchunk;
  const int l = (int)(q % d.Np);
  q /= d.Np;
  const int j = (int)(q % d.Nt);
  const int g = (int)(q / d.Nt);
  c0 = chunk * W;
  Wc = min(W, S - c0);
  base = (long long)g * d.S_g + (long long)j * d.S_j + (long long)l * d.S_l + c0;
}

template <typename C>
__device__ __forceinline__ void radial_rb_mats(const Tables<C>& t, int Nr, C* sE, C* sO, C* sMc,
                                               C* sMr) {
  const int hh = Nr / 2;
  for (int x = threadIdx.x; x < hh * hh; x += blockDim.x) {
    sE[x] = t.EpT[x];
    sO[x] = t.OpT[x];
  }
  for (int x = threadIdx.x; x < hh; x += blockDim.x) {
    sMc[x] = t.DrMc[x];
    sMr[x] = t.DrMr[x];
  }
}

template <bool ASYNC, typename T, typename C>
__device__ __forceinline__ void radial_rb_load(const Dims& d, const T* U, const T* Kin, int W,
                                               long long tile, C* su, C* sk) {
  long long base;
  int c0, Wc;
  radial_tile_coords(d, W, tile, base, c0, Wc);
  const int W4 = Wc / 4;
  for (int x = threadIdx.x; x < d.Nr * W4; x += blockDim.x) {
    const int ii = x / W4, w = (x - ii * W4) * 4;
    const long long gi = base + (long long)ii * d.S_i + w;
    copy4<ASYNC, T, C>(su + ii * W + w, U + gi);
    copy4<ASYNC, T, C>(sk + ii * W + w, Kin + gi);
  }
}

template <typename T, typename C>
__device__ __forceinline__ void radial_rb_body(const Problem& p, const Tables<C>& t,
                                               const double* __restrict__ Dr64, const C* su,
                                               C* sk, C* sEv, const C* sE, const C* sO,
                                               const C* sMc, const C* sMr, C sgn, int tau,
                                               int mode, T* F, T* Acc, T* Uout, T* out, C dt,
                                               int W, long long tile) {
  constexpr int RB = kRBRad, CB = 4;
  const Dims& d = p.d;
  const int Nr = d.Nr, N = Nr - 1, hh = Nr / 2, NP = d.NP;
  C* sOd = sEv + hh * W;
  long long base;
  int c0, Wc;
  radial_tile_coords(d, W, tile, base, c0, Wc);
  const int W4 = Wc / 4;
  for (int x = threadIdx.x; x < hh * W4; x += blockDim.x) {   // even/odd parts once per pair
    const int ii = x / W4, w = (x - ii * W4) * 4;
    C a[4], b[4], e[4], o[4];
    ld4<C>(su + ii * W + w, a);
    ld4<C>(su + (N - ii) * W + w, b);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      e[cc] = a[cc] + b[cc];
      o[cc] = a[cc] - b[cc];
    }
    st4<C>(sEv + ii * W + w, e);
    st4<C>(sOd + ii * W + w, o);
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
        C ev[CB], ov[CB], E[RB], O[RB];
        ld4<C>(sEv + ii * W + w0, ev);
        ld4<C>(sOd + ii * W + w0, ov);
        ldr<C, RB>(sE + ii * hh + i0, E);
        ldr<C, RB>(sO + ii * hh + i0, O);
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) {
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            ae[r][cc] = fmac(E[r], ev[cc], ae[r][cc]);
            ao[r][cc] = fmac(O[r], ov[cc], ao[r][cc]);
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
        C ov[CB];
        ld4<C>(sOd + ii * W + w0, ov);
        const C mr = sMr[ii];
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) am[cc] = fmac(mr, ov[cc], am[cc]);
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

template <typename T, typename C>
__device__ __forceinline__ void radial_tile_rb(const Problem& p, const Tables<C>& t,
                                               const double* __restrict__ Dr64, const T* U,
                                               const T* Kin, C sgn, int tau, int mode, T* F,
                                               T* Acc, T* Uout, T* out, C dt, int W,
                                               long long tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nr = p.d.Nr, hh = Nr / 2;
  const int hh4 = (hh * hh + 3) & ~3, h4 = (hh + 3) & ~3;
  C* sE = reinterpret_cast<C*>(smem_raw);
  C* sO = sE + hh4;
  C* sMc = sO + hh4;
  C* sMr = sMc + h4;
  C* su = sMr + h4;
  C* sk = su + Nr * W;
  C* sEv = sk + Nr * W;
  radial_rb_mats<C>(t, Nr, sE, sO, sMc, sMr);
  radial_rb_load<false, T, C>(p.d, U, Kin, W, tile, su, sk);
  __syncthreads();
  radial_rb_body<T, C>(p, t, Dr64, su, sk, sEv, sE, sO, sMc, sMr, sgn, tau, mode, F, Acc, Uout,
                       out, dt, W, tile);
}

template <typename T, typename C>
__global__ void __launch_bounds__(kThreads)
k_radial_pp(Problem p, Tables<C> t, const double* __restrict__ Dr64, const T* U, const T* Kin,
            C sgn, int tau, int mode, T* F, T* Acc, T* Uout, T* out, C dt, int W,
            long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nr = p.d.Nr, hh = Nr / 2;
  const int hh4 = (hh * hh + 3) & ~3, h4 = (hh + 3) & ~3;
  C* sE = reinterpret_cast<C*>(smem_raw);
  C* sO = sE + hh4;
  C* sMc = sO + hh4;
  C* sMr = sMc + h4;
  C* sbuf[2] = {sMr + h4, sMr + h4 + 2 * Nr * W};   // each: u [Nr][W] then K [Nr][W]
  C* sEv = sbuf[1] + 2 * Nr * W;
  radial_rb_mats<C>(t, Nr, sE, sO, sMc, sMr);
  long long tile = blockIdx.x;
  if (tile < ntiles) radial_rb_load<true, T, C>(p.d, U, Kin, W, tile, sbuf[0], sbuf[0] + Nr * W);
  cp_async_commit();
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const long long next = tile + gridDim.x;
    C* nb_ = sbuf[(it + 1) & 1];
    if (next < ntiles) radial_rb_load<true, T, C>(p.d, U, Kin, W, next, nb_, nb_ + Nr * W);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    C* cb = sbuf[it & 1];
    radial_rb_body<T, C>(p, t, Dr64, cb, cb + Nr * W, sEv, sE, sO, sMc, sMr, sgn, tau, mode, F,
                         Acc, Uout, out, dt, W, tile);
    __syncthreads();
  }
  cp_async_wait0();
}

// ----------------------------------------------------------------------------
// Pass dispatch (register-blocked form where the grid allows it) and the
// single-problem one-tile-per-CTA kernels (generic form, or rb without a
// persistent launch).
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
