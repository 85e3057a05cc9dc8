// Register-blocked forms of the three forward passes, and their persistent
// launches.
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
// memory), a preparation step (sums/differences, transposed copy) and a
// compute step. The single-tile form stages synchronously (used by the batched
// kernels); the persistent kernels k_*_pp keep the derivative matrices in
// shared memory for all their tiles and stage the next tile with asynchronous
// 16-byte copies (cp.async) while the current one is computed.
//
// The line lengths are template parameters (0 = read from the grid at run
// time): with them fixed, the contraction loops unroll completely and the
// index arithmetic folds into immediate offsets.
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

// RB consecutive elements from an address aligned to RB elements (vector loads
// where RB elements make 8 or 16 bytes).
template <typename C, int RB>
__device__ __forceinline__ void ldv(const C* p, C (&v)[RB]) {
  if constexpr (sizeof(C) == 4 && RB == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if constexpr (sizeof(C) == 4 && RB == 2) {
    const float2 a = *reinterpret_cast<const float2*>(p);
    v[0] = a.x; v[1] = a.y;
  } else if constexpr (sizeof(C) == 8 && RB == 2) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    v[0] = a.x; v[1] = a.y;
  } else {
#pragma unroll
    for (int r = 0; r < RB; ++r) v[r] = p[r];
  }
}

// Compile-time line length if given, else the run-time one.
template <int CT>
__device__ __forceinline__ int ctsz(int rt) { return CT ? CT : rt; }

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
// Ask for the 16 bytes at p to be brought into L2 (no register, no wait).
template <typename T>
__device__ __forceinline__ void prefetch_l2(const T* p) {
  asm volatile("prefetch.global.L2 [%0];" :: "l"(p));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// RB per pass (rows per thread): 4 in float, 2 in double for the angular and
// radial passes (rb_ang / rb_rad in ts_internal.h), kRBPlane for the plane pass.
template <typename C> struct RBAng { static constexpr int v = rb_ang((int)sizeof(C)); };
template <typename C> struct RBRad { static constexpr int v = rb_rad((int)sizeof(C)); };

// Row pitch of the transposed angular block (16 bytes of padding: the
// transposing stores of a warp then cover all banks once).
template <typename C>
__host__ __device__ constexpr int ang_utp(int NT) { return NT + 16 / (int)sizeof(C); }
// Per-block strides of the angular sums/differences and transposed copy: 8
// elements of padding put the blocks that one 16-byte load phase touches on
// distinct banks.
__host__ __device__ constexpr int ang_ss(int NT, int NP) { return NT * NP + 8; }
template <typename C>
__host__ __device__ constexpr int ang_us(int NT, int NP) { return NP * ang_utp<C>(NT) + 8; }

// Line lengths with compiled-in forms of the single-problem kernels (0: the
// run-time form, which the batched kernel always uses). The two forms perform
// the same operations; results agree to rounding, not bit for bit.
// Square direction blocks (16, 24, 32) return N; the 24 x 16 blocks of the hybrid-grid
// shell workload return 2416.
__host__ __device__ inline int ang_spec(const Dims& d) {
  if (d.NT == 24 && d.NP == 16) return 2416;
  if (d.NT != d.NP) return 0;
  return (d.NT == 16 || d.NT == 24 || d.NT == 32) ? d.NT : 0;
}
__host__ __device__ inline int plane_spec(const Dims& d, int c) {
  const bool sq = d.Nt == d.Np && d.Np == d.NT && d.NT == d.NP && 2 * c == d.NP;
  return (sq && (d.NP == 8 || d.NP == 16 || d.NP == 24 || d.NP == 32)) ? d.NP : 0;
}
__host__ __device__ inline int rad_spec(const Dims& d) {
  return (d.Nr == 17 || d.Nr == 33 || d.Nr == 65) ? d.Nr : 0;
}

// ============================================================================
// Angular pass. Thread: RB Theta rows k0.. and their mirror rows NT-1-k0-.. x 4
// column pairs (m, m + NP/2) of one block. Both contractions work on the pair
// halves s = F(m) + F(m+NP/2), d = F(m) - F(m+NP/2):
//  * Theta through P, Q (DFS partner). P and Q are centro-antisymmetric (the
//    Theta nodes are symmetric about pi/2 and the derivative is odd), so rows k
//    and NT-1-k come from the Theta-even/odd parts e = h(k') + h(NT-1-k'),
//    o = h(k') - h(NT-1-k') of each half h (k' < NT/2) through the folded
//    matrices Pe, Po, Qe, Qo: a quarter of the dense multiply-adds;
//  * Phi through Ms, Md (the circulant Fourier derivative on the halves): half.
// Shared layout: [PeT | PoT | QeT | QoT (NT/2 x NT/2 each) | MsPhT | MdPhT |
//                 tile nb*S | folded halves nb*(S+8) | transposed halves
//                 nb*(NP*UTP+8) | kAngScalars nb per-block scalars]
// The angular blocks of one tile: block bb (< nbb) of the tile is the global
// block b0 + bb * bs (consecutive blocks in the angular pass; the N_r blocks of
// one (g, theta, phi) position, stride N_theta N_phi, in the fused pass).
struct AngBlocks {
  long long b0, bs;
  int nbb;
};
__device__ __forceinline__ AngBlocks ang_blocks(const Dims& d, int nb, long long tile) {
  AngBlocks a;
  a.b0 = tile * nb;
  a.bs = 1;
  a.nbb = (int)min((long long)nb, d.nblk - a.b0);
  return a;
}

template <typename C>
__device__ __forceinline__ void angular_rb_mats(const Tables<C>& t, const Dims& d, C* sP, C* sQ,
                                                C* sD) {
  const int hT = d.NT / 2, hP = d.NP / 2;
  for (int x = threadIdx.x; x < hT * hT; x += blockDim.x) {
    sP[x] = t.PeThT[x];
    sP[hT * hT + x] = t.PoThT[x];
    sQ[x] = t.QeThT[x];
    sQ[hT * hT + x] = t.QoThT[x];
  }
  for (int x = threadIdx.x; x < hP * hP; x += blockDim.x) {
    sD[x] = t.MsPhT[x];
    sD[hP * hP + x] = t.MdPhT[x];
  }
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

// Preparation of a staged tile: coefficients, J (and, with an anisotropic
// kernel, kappa_s b, kappa_s c and the first and second moments H, M), the
// folded halves
// [se | so | de | do] ([k' < NT/2][p < NP/2] each) for the Theta contraction and
// the pointwise terms, and the transposed halves uT[p][k] = s, uT[NP/2 + p][k] =
// d for the Phi contraction. Entry: su complete and visible. Exit (after the
// caller's barrier): su is no longer read.
template <int NT_, int NP_, int KF, typename T, typename C>
__device__ __forceinline__ void angular_rb_prep(const Problem& p, const Tables<C>& t,
                                                const C* su, C* sSD, C* uT, C* sc, int collision,
                                                int nb, AngBlocks ab) {
  const Dims& d = p.d;
  const int NT = ctsz<NT_>(d.NT), NP = ctsz<NP_>(d.NP), S = NT * NP, hP = NP / 2, hT = NT / 2;
  const int UTP = ang_utp<C>(NT), H4 = hP / 4, SS = ang_ss(NT, NP), US = ang_us<C>(NT, NP);
  const int Q4 = hT * hP;   // one folded half
  const int nbb = ab.nbb;
  const bool aniso = KF >= KF_LINEAR && collision;
  const bool quad = KF >= KF_QUADRATIC && collision;
  for (int x = threadIdx.x; x < nbb; x += blockDim.x) {  // once per block
    const long long bx = ab.b0 + x * ab.bs;
    sc[nb + x] = (C)p.kap[bx];
    sc[2 * nb + x] = (C)p.eta[bx];
    sc[3 * nb + x] = (C)p.kaps[bx];
    if (aniso) sc[6 * nb + x] = p.scb ? (C)(p.kaps[bx] * p.scb[bx]) : (C)0;
    if (quad) sc[10 * nb + x] = (C)(p.kaps[bx] * p.scc[bx]);
    int g, i, j, l;
    decode_block(d, bx, g, i, j, l);
    sc[4 * nb + x] = t.inv_r[i];
    sc[5 * nb + x] = t.cot_th[j];
  }
  // When the threads of one block form an aligned power-of-two group of at
  // most a warp, J comes out of this loop by a segmented warp reduction;
  // otherwise from a separate pass over the block.
  const int tpb = hT * H4;
  const bool warp_J = tpb <= 32 && (tpb & (tpb - 1)) == 0;
  // With the warp reduction the trip count is rounded up to whole warps
  // (blockDim.x is a multiple of 32), so every lane of a warp takes part in
  // every shuffle; lanes past the tile contribute zero and store nothing.
  const int nx = nbb * tpb, nxw = warp_J ? (nx + 31) / 32 * 32 : nx;
  // lanes run over k fastest: the transposing stores of a warp hit distinct banks
  for (int x = threadIdx.x; x < nxw; x += blockDim.x) {
    const bool act = x < nx;
    const int kk = x % hT, rest = x / hT, p4 = (rest % H4) * 4, bb = rest / H4;
    const int km = NT - 1 - kk;
    C a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0}, a2[4] = {0, 0, 0, 0}, b2[4] = {0, 0, 0, 0};
    if (act) {
      ld4<C>(su + bb * S + kk * NP + p4, a);
      ld4<C>(su + bb * S + kk * NP + p4 + hP, b);
      ld4<C>(su + bb * S + km * NP + p4, a2);
      ld4<C>(su + bb * S + km * NP + p4 + hP, b2);
    }
    C s[4], df[4], s2[4], d2[4], e1[4], o1[4], e2[4], o2[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      s[c] = a[c] + b[c];
      df[c] = a[c] - b[c];
      s2[c] = a2[c] + b2[c];
      d2[c] = a2[c] - b2[c];
      e1[c] = s[c] + s2[c];
      o1[c] = s[c] - s2[c];
      e2[c] = df[c] + d2[c];
      o2[c] = df[c] - d2[c];
    }
    if (act) {
      C* q = sSD + bb * SS + kk * hP + p4;
      st4<C>(q, e1);
      st4<C>(q + Q4, o1);
      st4<C>(q + 2 * Q4, e2);
      st4<C>(q + 3 * Q4, o2);
      C* ut = uT + bb * US;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        ut[(p4 + c) * UTP + kk] = s[c];
        ut[(p4 + c) * UTP + km] = s2[c];
        ut[(p4 + hP + c) * UTP + kk] = df[c];
        ut[(p4 + hP + c) * UTP + km] = d2[c];
      }
    }
    if (collision && warp_J) {   // warp-uniform: the trip count covers whole warps
      C acc = act ? t.qdir[kk] * ((s[0] + s[1]) + (s[2] + s[3])) +
                        t.qdir[km] * ((s2[0] + s2[1]) + (s2[2] + s2[3]))
                  : (C)0;
      for (int o = tpb >> 1; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (act && (x % tpb) == 0) sc[bb] = acc;
      if (aniso) {
        // First moment in the local frame from the pair halves: cos(Theta) is odd
        // under k -> NT-1-k, cos(Phi) and sin(Phi) under m -> m + NP/2, so
        // H_r takes the Theta-odd part of the sums, H_theta and H_phi the
        // Theta-even part of the differences.
        C hr = 0, ht = 0, hp = 0;
        if (act) {
          C a1 = 0, a2 = 0;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            a1 = fmac(t.cosP[p4 + c], e2[c], a1);
            a2 = fmac(t.sinP[p4 + c], e2[c], a2);
          }
          const C qs = t.qdir[kk] * t.sinT[kk];
          hr = t.qdir[kk] * t.cosT[kk] * ((o1[0] + o1[1]) + (o1[2] + o1[3]));
          ht = qs * a1;
          hp = qs * a2;
        }
        for (int o = tpb >> 1; o; o >>= 1) {
          hr += __shfl_xor_sync(0xffffffffu, hr, o);
          ht += __shfl_xor_sync(0xffffffffu, ht, o);
          hp += __shfl_xor_sync(0xffffffffu, hp, o);
        }
        if (act && (x % tpb) == 0) {
          sc[7 * nb + bb] = hr;
          sc[8 * nb + bb] = ht;
          sc[9 * nb + bb] = hp;
        }
      }
      if (quad) {
        // second moment: cos^2(Th), sin^2(Th) are even under k -> NT-1-k and
        // cos(Th) sin(Th) odd; cos^2(Ph), sin^2(Ph), cos(Ph) sin(Ph) are even under
        // m -> m + NP/2 and cos(Ph), sin(Ph) odd. So M_rr, M_thth, M_phph, M_thph
        // take the Theta-even part of the sums, M_rth, M_rph the Theta-odd part of
        // the differences.
        C m6[6] = {0, 0, 0, 0, 0, 0};
        if (act) {
          C se = 0, sc2 = 0, ss2 = 0, scs = 0, tc = 0, tsn = 0;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const C cp = t.cosP[p4 + c], sp = t.sinP[p4 + c];
            se += e1[c];
            sc2 = fmac(cp * cp, e1[c], sc2);
            ss2 = fmac(sp * sp, e1[c], ss2);
            scs = fmac(cp * sp, e1[c], scs);
            tc = fmac(cp, o2[c], tc);
            tsn = fmac(sp, o2[c], tsn);
          }
          const C q = t.qdir[kk], ct = t.cosT[kk], st = t.sinT[kk];
          const C qss = q * st * st, qcs = q * ct * st;
          m6[0] = q * ct * ct * se;
          m6[1] = qss * sc2;
          m6[2] = qss * ss2;
          m6[3] = qss * scs;
          m6[4] = qcs * tc;
          m6[5] = qcs * tsn;
        }
#pragma unroll
        for (int a = 0; a < 6; ++a)
          for (int o = tpb >> 1; o; o >>= 1) m6[a] += __shfl_xor_sync(0xffffffffu, m6[a], o);
        if (act && (x % tpb) == 0) {
#pragma unroll
          for (int a = 0; a < 6; ++a) sc[(11 + a) * nb + bb] = m6[a];
        }
      }
    }
  }
  if (collision && !warp_J) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bb = warp; bb < nbb; bb += blockDim.x >> 5) {
      C acc = 0, hr = 0, ht = 0, hp = 0, m6[6] = {0, 0, 0, 0, 0, 0};
      for (int x = lane; x < S; x += 32) {
        const int k = x / NP, m = x - k * NP;
        const C u = su[bb * S + x];
        acc = fmac(t.qdir[k], u, acc);
        if (aniso) {
          const C qu = t.qdir[k] * u, qs = t.sinT[k] * qu;
          hr = fmac(t.cosT[k], qu, hr);
          ht = fmac(t.cosP[m], qs, ht);
          hp = fmac(t.sinP[m], qs, hp);
          if (quad) {
            const C ct = t.cosT[k], cp = t.cosP[m], sp = t.sinP[m], qss = t.sinT[k] * qs;
            m6[0] = fmac(ct * ct, qu, m6[0]);
            m6[1] = fmac(cp * cp, qss, m6[1]);
            m6[2] = fmac(sp * sp, qss, m6[2]);
            m6[3] = fmac(cp * sp, qss, m6[3]);
            m6[4] = fmac(ct * cp, qs, m6[4]);
            m6[5] = fmac(ct * sp, qs, m6[5]);
          }
        }
      }
      for (int o = 16; o; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (aniso) {
          hr += __shfl_xor_sync(0xffffffffu, hr, o);
          ht += __shfl_xor_sync(0xffffffffu, ht, o);
          hp += __shfl_xor_sync(0xffffffffu, hp, o);
        }
        if (quad) {
#pragma unroll
          for (int a = 0; a < 6; ++a) m6[a] += __shfl_xor_sync(0xffffffffu, m6[a], o);
        }
      }
      if (lane == 0) {
        sc[bb] = acc;
        if (aniso) {
          sc[7 * nb + bb] = hr;
          sc[8 * nb + bb] = ht;
          sc[9 * nb + bb] = hp;
        }
        if (quad) {
#pragma unroll
          for (int a = 0; a < 6; ++a) sc[(11 + a) * nb + bb] = m6[a];
        }
      }
    }
  }
}

// Compute a prepared tile and write K. Reads sSD, uT, sc and the matrices.
// KF: add the kernel's mu (and mu^2) terms (separate instantiations keep the
// register allocation of the isotropic form unchanged).
// Kt: the output of the tile's block 0 (block bb at Kt + bb S, global memory or
// a shared-memory tile).
template <int NT_, int NP_, int KF, typename T, typename C>
__device__ __forceinline__ void angular_rb_compute(const Problem& p, const Tables<C>& t,
                                                   const C* sSD, const C* uT, const C* sc,
                                                   const C* sP, const C* sQ, const C* sD,
                                                   T* __restrict__ Kt, C sgn, int collision,
                                                   int nb, AngBlocks ab) {
  constexpr int RB = RBAng<C>::v, CB = 4;
  const Dims& d = p.d;
  const int NT = ctsz<NT_>(d.NT), NP = ctsz<NP_>(d.NP), S = NT * NP, hP = NP / 2, hT = NT / 2;
  const int UTP = ang_utp<C>(NT), SS = ang_ss(NT, NP), US = ang_us<C>(NT, NP);
  const int Q4 = hT * hP;
  const int nbb = ab.nbb;
  const int KR = hT / RB, PC = hP / CB;
  constexpr bool aniso = KF >= KF_LINEAR;
  constexpr bool quad = KF >= KF_QUADRATIC;
  // unit = (pc, 4 blocks, kr, block group): a 16-byte load phase spans 4 blocks
  const int units = ((nbb + 3) / 4) * 4 * KR * PC;
  const C* sPe = sP;
  const C* sPo = sP + hT * hT;
  const C* sQe = sQ;
  const C* sQo = sQ + hT * hT;
  const C* sMs = sD;
  const C* sMd = sD + hP * hP;
  for (int unit = threadIdx.x; unit < units; unit += blockDim.x) {
    const int pc = unit % PC, r1 = unit / PC, b4 = r1 % 4, r2 = r1 / 4, kr = r2 % KR;
    const int bb = (r2 / KR) * 4 + b4;
    if (bb >= nbb) continue;
    const int p0 = pc * CB, k0 = kr * RB, k1 = NT - RB - k0;   // mirror rows k1.. (reversed)
    const C* qb = sSD + bb * SS;
    const C* ut = uT + bb * US;
    C aE[RB][CB], aO[RB][CB], bE[RB][CB], bO[RB][CB];
    C fs[RB][CB], fd[RB][CB], gs[RB][CB], gd[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < CB; ++c)
        aE[r][c] = aO[r][c] = bE[r][c] = bO[r][c] = fs[r][c] = fd[r][c] = gs[r][c] =
            gd[r][c] = 0;
#pragma unroll
    for (int kk = 0; kk < hT; ++kk) {
      C ev[CB], ov[CB], ew[CB], ow[CB], Pe[RB], Po[RB], Qe[RB], Qo[RB];
      const C* qk = qb + kk * hP + p0;
      ld4<C>(qk, ev);
      ld4<C>(qk + Q4, ov);
      ld4<C>(qk + 2 * Q4, ew);
      ld4<C>(qk + 3 * Q4, ow);
      ldv<C, RB>(sPe + kk * hT + k0, Pe);
      ldv<C, RB>(sPo + kk * hT + k0, Po);
      ldv<C, RB>(sQe + kk * hT + k0, Qe);
      ldv<C, RB>(sQo + kk * hT + k0, Qo);
#pragma unroll
      for (int c = 0; c < CB; ++c) {
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          aE[r][c] = fmac(Pe[r], ev[c], aE[r][c]);
          aO[r][c] = fmac(Po[r], ov[c], aO[r][c]);
          bE[r][c] = fmac(Qe[r], ew[c], bE[r][c]);
          bO[r][c] = fmac(Qo[r], ow[c], bO[r][c]);
        }
      }
    }
#pragma unroll
    for (int pp = 0; pp < hP; ++pp) {
      C A4[CB], B4[CB], sv[RB], dv[RB], sw[RB], dw[RB];
      ld4<C>(sMs + pp * hP + p0, A4);
      ld4<C>(sMd + pp * hP + p0, B4);
      ldv<C, RB>(ut + pp * UTP + k0, sv);
      ldv<C, RB>(ut + (hP + pp) * UTP + k0, dv);
      ldv<C, RB>(ut + pp * UTP + k1, sw);
      ldv<C, RB>(ut + (hP + pp) * UTP + k1, dw);
#pragma unroll
      for (int r = 0; r < RB; ++r) {
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          fs[r][c] = fmac(A4[c], sv[r], fs[r][c]);
          fd[r][c] = fmac(B4[c], dv[r], fd[r][c]);
          gs[r][c] = fmac(A4[c], sw[r], gs[r][c]);
          gd[r][c] = fmac(B4[c], dw[r], gd[r][c]);
        }
      }
    }
    const C ir = sc[4 * nb + bb], ct = sc[5 * nb + bb];
    const C J = sc[bb], kap = sc[nb + bb], eta = sc[2 * nb + bb], ks = sc[3 * nb + bb];
    const C src = eta + ks * J, kks = kap + ks;
    C s1[CB], s2[CB];   // a_Phi / a_Theta at m and m + NP/2, with the 1/2 of the halves
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      s1[c] = (C)0.5 * t.sinP[p0 + c] * ct;
      s2[c] = (C)0.5 * t.sinP[p0 + c + hP] * ct;
    }
    // row k = k0 + r (side 0) and its mirror NT-1-k = k1 + RB-1-r (side 1)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int k = side ? NT - 1 - k0 - r : k0 + r;
        const int rm = side ? RB - 1 - r : r;   // index of row k in the mirror loads
        const C sg = side ? (C)-1 : (C)1;
        const C aT = sgn * -t.sinT[k] * ir;
        C ps[CB], qd[CB], fa[CB], fb[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          // the folded tables carry the 1/2 of the Theta folding
          ps[c] = aO[r][c] + sg * aE[r][c];
          qd[c] = bO[r][c] + sg * bE[r][c];
          fa[c] = side ? gs[rm][c] : fs[r][c];
          fb[c] = side ? gd[rm][c] : fd[r][c];
        }
        C sv[CB], dv[CB];   // 2 F-halves at (k, m) from the folded halves: e + sg o
        if (collision) {
          C e1[CB], o1[CB], e2[CB], o2[CB];
          const int kk = k0 + r;
          ld4<C>(qb + kk * hP + p0, e1);
          ld4<C>(qb + Q4 + kk * hP + p0, o1);
          ld4<C>(qb + 2 * Q4 + kk * hP + p0, e2);
          ld4<C>(qb + 3 * Q4 + kk * hP + p0, o2);
#pragma unroll
          for (int c = 0; c < CB; ++c) {
            sv[c] = e1[c] + sg * o1[c];
            dv[c] = e2[c] + sg * o2[c];
          }
        }
        const C kq = (C)0.25 * kks;   // F(k, m) = (sv + dv) / 4, F(k, m + NP/2) = (sv - dv) / 4
        T o1v[CB], o2v[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          C v1 = aT * (ps[c] + qd[c] + s1[c] * (fa[c] + fb[c]));
          C v2 = aT * (ps[c] - qd[c] + s2[c] * (fa[c] - fb[c]));
          if (collision) {
            v1 += src - kq * (sv[c] + dv[c]);
            v2 += src - kq * (sv[c] - dv[c]);
          }
          o1v[c] = (T)v1;
          o2v[c] = (T)v2;
        }
        T* out = Kt + (long long)bb * S + k * NP + p0;
        st4<T>(out, o1v);
        st4<T>(out + hP, o2v);
      }
    }
    if (aniso) {
      // The kernel's mu (and mu^2) terms, added in a second sweep over this
      // unit's outputs once its accumulators are dead (volatile reloads of the
      // values this thread has just stored keep them out of registers):
      //   kappa_s b omega.H = cos(Th) hr + sin(Th) hc,
      //   kappa_s c omega.M~.omega = cos^2(Th) mrr + sin^2(Th) qmc + cos(Th) sin(Th) rmc,
      // M~ = M - J I/3; at m + NP/2 the terms odd in (cos Ph, sin Ph) change sign.
      C hr, hc[CB], mrr = 0, qmc[CB], rmc[CB];
      {
        const C kb = sc[6 * nb + bb], ht = kb * sc[8 * nb + bb], hp = kb * sc[9 * nb + bb];
        hr = kb * sc[7 * nb + bb];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          hc[c] = t.cosP[p0 + c] * ht + t.sinP[p0 + c] * hp;
          qmc[c] = rmc[c] = 0;
        }
      }
      if (quad) {
        const C kc = sc[10 * nb + bb], j3 = J * ((C)1 / (C)3);
        mrr = kc * (sc[11 * nb + bb] - j3);
        const C mtt = kc * (sc[12 * nb + bb] - j3), mpp = kc * (sc[13 * nb + bb] - j3);
        const C mtp = (C)2 * kc * sc[14 * nb + bb];
        const C mrt = (C)2 * kc * sc[15 * nb + bb], mrp = (C)2 * kc * sc[16 * nb + bb];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          const C cp = t.cosP[p0 + c], sp = t.sinP[p0 + c];
          qmc[c] = cp * cp * mtt + sp * sp * mpp + cp * sp * mtp;
          rmc[c] = cp * mrt + sp * mrp;
        }
      }
#pragma unroll
      for (int side = 0; side < 2; ++side) {
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const int k = side ? NT - 1 - k0 - r : k0 + r;
          const C ct = t.cosT[k], st = t.sinT[k];
          T* out = Kt + (long long)bb * S + k * NP + p0;
          volatile T* vout = out;
          T o1v[CB], o2v[CB];
#pragma unroll
          for (int c = 0; c < CB; ++c) {
            C ev = ct * hr, od = st * hc[c];
            if (quad) {
              ev += ct * ct * mrr + st * st * qmc[c];
              od += ct * st * rmc[c];
            }
            o1v[c] = (T)((C)vout[c] + (ev + od));
            o2v[c] = (T)((C)vout[hP + c] + (ev - od));
          }
          st4<T>(out, o1v);
          st4<T>(out + hP, o2v);
        }
      }
    }
  }
}

template <int NT_, int NP_, int KF, typename T, typename C>
__device__ __forceinline__ void angular_tile_rb_form(const Problem& p, const Tables<C>& t,
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
  C* uT = sSD + nb * ang_ss(NT, NP);
  C* sc = uT + nb * ang_us<C>(NT, NP);
  angular_rb_mats<C>(t, d, sP, sQ, sD);
  angular_rb_load<false, T, C>(d, U, nb, tile, su);
  __syncthreads();
  const AngBlocks ab = ang_blocks(d, nb, tile);
  angular_rb_prep<NT_, NP_, KF, T, C>(p, t, su, sSD, uT, sc, collision, nb, ab);
  __syncthreads();
  angular_rb_compute<NT_, NP_, KF, T, C>(p, t, sSD, uT, sc, sP, sQ, sD, K + ab.b0 * S, sgn,
                                         collision, nb, ab);
}

template <int NT_, int NP_, typename T, typename C>
__device__ __forceinline__ void angular_tile_rb(const Problem& p, const Tables<C>& t,
                                                const T* __restrict__ U, T* __restrict__ K,
                                                C sgn, int collision, int nb, long long tile) {
  switch (kernel_form(p, collision)) {
    case KF_QUADRATIC:
      angular_tile_rb_form<NT_, NP_, KF_QUADRATIC, T, C>(p, t, U, K, sgn, collision, nb, tile);
      break;
    case KF_LINEAR:
      angular_tile_rb_form<NT_, NP_, KF_LINEAR, T, C>(p, t, U, K, sgn, collision, nb, tile);
      break;
    default:
      angular_tile_rb_form<NT_, NP_, KF_ISO, T, C>(p, t, U, K, sgn, collision, nb, tile);
  }
}

// Persistent: the next tile is copied into the staging buffer as soon as the
// current one has been prepared, and lands while the current one is computed.
// KF: the kernel form (launched by the grid's scattering kernel when the pass
// includes the collision term); separate kernels, so that the isotropic form
// keeps its own register allocation.
template <typename T, typename C, int NT_, int NP_, int KF>
__global__ void __launch_bounds__(kThreads, 2)
k_angular_pp(Problem p, Tables<C> t, const T* __restrict__ U, T* __restrict__ K, C sgn,
             int collision, int nb, long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int NT = ctsz<NT_>(d.NT), NP = ctsz<NP_>(d.NP), S = NT * NP;
  C* sP = reinterpret_cast<C*>(smem_raw);
  C* sQ = sP + NT * NT;
  C* sD = sQ + NT * NT;
  C* su = sD + NP * NP;
  C* sSD = su + nb * S;
  C* uT = sSD + nb * ang_ss(NT, NP);
  C* sc = uT + nb * ang_us<C>(NT, NP);
  angular_rb_mats<C>(t, d, sP, sQ, sD);
  long long tile = blockIdx.x;
  if (tile < ntiles) angular_rb_load<true, T, C>(d, U, nb, tile, su);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    cp_async_wait0();
    __syncthreads();   // this tile staged; the previous tile's compute is done
    const AngBlocks ab = ang_blocks(d, nb, tile);
    angular_rb_prep<NT_, NP_, KF, T, C>(p, t, su, sSD, uT, sc, collision, nb, ab);
    __syncthreads();   // staging buffer free
    const long long next = tile + gridDim.x;
    if (next < ntiles) angular_rb_load<true, T, C>(d, U, nb, next, su);
    cp_async_commit();
    angular_rb_compute<NT_, NP_, KF, T, C>(p, t, sSD, uT, sc, sP, sQ, sD, K + ab.b0 * S, sgn,
                                           collision, nb, ab);
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

// N_ > 0: square grid (N_ nodes on every angular axis) with c = N_/2, i.e. a
// tile holds whole Phi rows; 0: sizes and c from the grid at run time.
template <int N_, typename T, typename C>
__device__ __forceinline__ void plane_rb_body(const Problem& p, const Tables<C>& t, const C* su,
                                              C* sSm, const C* sP, const C* sQ, const C* sD,
                                              T* __restrict__ K, C sgn, int c_rt, long long tile) {
  constexpr int RB = kRBPlane, CB = 4;
  const Dims& d = p.d;
  const int Nt = ctsz<N_>(d.Nt), Np = ctsz<N_>(d.Np), hP = ctsz<N_>(d.NP) / 2, hp = Np / 2;
  const int c = N_ ? N_ / 2 : c_rt, W = 2 * c;
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
  const C sTk = t.sinT[k] * t.inv_r[i];
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
#pragma unroll
    for (int jj = 0; jj < Nt; ++jj) {
      C sv[CB], dv[CB], P[RB], Q[RB];
      ld4<C>(sSm + (jj * hp + l) * W + w0, sv);
      ld4<C>(sDf + (jj * hp + l) * W + w0, dv);
      ldv<C, RB>(sP + jj * Nt + j0, P);
      ldv<C, RB>(sQ + jj * Nt + j0, Q);
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          ps[r][cc] = fmac(P[r], sv[cc], ps[r][cc]);
          qd[r][cc] = fmac(Q[r], dv[cc], qd[r][cc]);
        }
      }
    }
#pragma unroll
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
    C cA[CB], sA[CB], cB[CB], sB[CB];
#pragma unroll
    for (int cc = 0; cc < CB; ++cc) {
      cA[cc] = sgn * sTk * t.cosP[mA + cc];
      sA[cc] = sgn * sTk * t.sinP[mA + cc];
      cB[cc] = sgn * sTk * t.cosP[mB + cc];
      sB[cc] = sgn * sTk * t.sinP[mB + cc];
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int j = j0 + r;
      const C isn = t.inv_sinth[j];
      T* pa = K + base + (long long)j * d.S_j + (long long)l * d.S_l + mA;
      T* pb = K + base + (long long)j * d.S_j + (long long)lh * d.S_l + mB;
      T ka[CB] = {0, 0, 0, 0}, kb[CB] = {0, 0, 0, 0};
      if (!p.plane_store) {
        ld4<T>(pa, ka);
        ld4<T>(pb, kb);
      }
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
        ka[cc] = (T)((C)ka[cc] + cA[cc] * (ps[r][cc] + qd[r][cc]) + sA[cc] * isn * da[r][cc]);
        kb[cc] = (T)((C)kb[cc] + cB[cc] * (ps[r][cc] - qd[r][cc]) + sB[cc] * isn * db[r][cc]);
      }
      st4<T>(pa, ka);
      st4<T>(pb, kb);
    }
  }
}

template <int N_, typename T, typename C>
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
  plane_rb_body<N_, T, C>(p, t, su, sSm, sP, sQ, sD, K, sgn, c, tile);
}

template <typename T, typename C, int N_>
__global__ void __launch_bounds__(kThreads, 2)
k_plane_pp(Problem p, Tables<C> t, const T* __restrict__ U, T* __restrict__ K, C sgn, int c,
           long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int Nt = ctsz<N_>(d.Nt), Np = ctsz<N_>(d.Np), W = 2 * c, TS = Nt * Np * W;
  C* sP = reinterpret_cast<C*>(smem_raw);
  C* sQ = sP + Nt * Nt;
  C* sD = sQ + Nt * Nt;
  C* buf0 = sD + Np * Np;
  C* sSm = buf0 + 2 * TS;
  plane_rb_mats<C>(t, d, sP, sQ, sD);
  long long tile = blockIdx.x;
  if (tile < ntiles) plane_rb_load<true, T, C>(d, U, c, tile, buf0);
  cp_async_commit();
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const long long next = tile + gridDim.x;
    C* cur = buf0 + (it & 1) * TS;
    C* nxt = buf0 + ((it + 1) & 1) * TS;
    if (next < ntiles) plane_rb_load<true, T, C>(d, U, c, next, nxt);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    plane_rb_body<N_, T, C>(p, t, cur, sSm, sP, sQ, sD, K, sgn, c, tile);
    __syncthreads();
  }
  cp_async_wait0();
}

// ----------------------------------------------------------------------------
// Plane pass on a square grid (N nodes on every angular axis), whole Phi rows
// per tile: a tile is (g, i) and KT consecutive Theta values, i.e. columns
// w = kl*N + m (KT*N of them, contiguous in memory for every (theta, phi)).
// Thread: one theta row j < N/2 and its mirror N-1-j x one phi pair (l, l+N/2)
// x CB columns m0.. and the CB partner columns m0 + N/2.. of one Theta value
// (CB = 4 in float, 2 in double). Folding:
//  * theta through the DFS pairs it owns -- (l, m) with (l+N/2, m+N/2) and
//    (l, m+N/2) with (l+N/2, m) -- and, since P and Q are centro-antisymmetric,
//    through the theta-even/odd parts of the pair sums and differences
//    (folded matrices Pe, Po, Qe, Qo): a quarter of the dense multiply-adds;
//  * phi on the phi pair halves sigma = u(l) + u(l+N/2), delta = u(l) -
//    u(l+N/2) through Ms, Md: half.
// The staged tile is turned into sigma (rows l < N/2) and delta (rows
// l + N/2) in place once the theta sums are formed. The folded sums use a row
// pitch of KT*N + 32 bytes so that the lanes of a load phase hit distinct banks.
// Shared layout: [PeT, PoT | QeT, QoT | MsphT, MdphT | 2 tiles N*N*KT*N |
//                 folded theta sums se, so, de, do: 4 x (N/2)*(N/2)*(KT*N+pad)]
template <int N, int KT, typename C>
struct PlaneSq {
  static constexpr int W = KT * N, hp = N / 2, SP = W + 32 / (int)sizeof(C);
  static constexpr int TS = N * N * W, CB = sizeof(C) == 4 ? 4 : 2, HC = hp / CB;
  static constexpr int QS = hp * hp * SP;   // one folded sum array [j' < N/2][l < N/2][w]
  static constexpr int units = hp * hp * KT * HC;
};

template <int N, int KT, typename C>
size_t smem_plane_sq() {
  using S = PlaneSq<N, KT, C>;
  return (size_t)(3 * N * N + 2 * S::TS + 4 * S::QS) * sizeof(C);
}

template <typename C, int NV>
__device__ __forceinline__ void stv(C* p, const C (&v)[NV]) {
  if constexpr (NV == 4) {
    st4<C>(p, v);
  } else if constexpr (sizeof(C) == 8 && NV == 2) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else if constexpr (sizeof(C) == 4 && NV == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int r = 0; r < NV; ++r) p[r] = v[r];
  }
}

template <typename C>
__device__ __forceinline__ void plane_sq_mats(const Tables<C>& t, const Dims& d, C* sP, C* sQ,
                                              C* sD) {
  const int ht = d.Nt / 2, hp = d.Np / 2;
  for (int x = threadIdx.x; x < ht * ht; x += blockDim.x) {
    sP[x] = t.PethT[x];
    sP[ht * ht + x] = t.PothT[x];
    sQ[x] = t.QethT[x];
    sQ[ht * ht + x] = t.QothT[x];
  }
  for (int x = threadIdx.x; x < hp * hp; x += blockDim.x) {
    sD[x] = t.MsphT[x];
    sD[hp * hp + x] = t.MdphT[x];
  }
}

template <int N, int KT, typename T, typename C>
__device__ __forceinline__ void plane_sq_load(const Dims& d, const T* U, long long tile, C* su) {
  using S = PlaneSq<N, KT, C>;
  const long long q = tile / (N / KT);
  const int k0 = (int)(tile - q * (N / KT)) * KT;
  const long long base = q * d.S_i + (long long)k0 * N;   // q = g*Nr + i
  for (int x = threadIdx.x; x < N * N * (S::W / 4); x += blockDim.x) {
    const int w4 = (x % (S::W / 4)) * 4, jl = x / (S::W / 4);
    copy4<true, T, C>(su + jl * S::W + w4, U + base + (long long)jl * d.S_l + w4);
  }
}

template <int N, int KT, typename T, typename C>
__device__ __forceinline__ void plane_sq_body(const Problem& p, const Tables<C>& t, C* su,
                                              C* sF, const C* sP, const C* sQ, const C* sD,
                                              T* __restrict__ K, C sgn, long long tile) {
  using S = PlaneSq<N, KT, C>;
  constexpr int CB = S::CB, W = S::W, hp = S::hp, SP = S::SP, HC = S::HC, QS = S::QS;
  const Dims& d = p.d;
  const long long q = tile / (N / KT);
  const int k0 = (int)(tile - q * (N / KT)) * KT;
  const int i = (int)(q % d.Nr);
  const long long base = q * d.S_i + (long long)k0 * N;
  // Per (theta row j < N/2 with its mirror, phi pair, CB columns m.. and
  // m + N/2..): the DFS sums/differences of both rows folded over the theta
  // mirror into sF, then the phi pair halves written over the eight staged
  // row segments this thread read.
  for (int x = threadIdx.x; x < S::units; x += blockDim.x) {
    const int mq = x % HC, r1 = x / HC, kl = r1 % KT, r2 = r1 / KT, l = r2 % hp, jj = r2 / hp;
    const int wA = kl * N + mq * CB, wB = wA + hp;
    C a0[2][CB], a1[2][CB], b0[2][CB], b1[2][CB];   // [row jj / mirror][cols]
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int j = side ? N - 1 - jj : jj;
      ldv<C, CB>(su + (j * N + l) * W + wA, a0[side]);
      ldv<C, CB>(su + (j * N + l) * W + wB, a1[side]);
      ldv<C, CB>(su + (j * N + l + hp) * W + wA, b0[side]);
      ldv<C, CB>(su + (j * N + l + hp) * W + wB, b1[side]);
    }
    C se[2][CB], so[2][CB], de[2][CB], dO[2][CB];   // [column A / B]
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      // DFS pairs (l, m)~(l+N/2, m+N/2) at column A and (l, m+N/2)~(l+N/2, m) at B
      const C sA0 = a0[0][c] + b1[0][c], dA0 = a0[0][c] - b1[0][c];
      const C sA1 = a0[1][c] + b1[1][c], dA1 = a0[1][c] - b1[1][c];
      const C sB0 = a1[0][c] + b0[0][c], dB0 = a1[0][c] - b0[0][c];
      const C sB1 = a1[1][c] + b0[1][c], dB1 = a1[1][c] - b0[1][c];
      se[0][c] = sA0 + sA1;
      so[0][c] = sA0 - sA1;
      de[0][c] = dA0 + dA1;
      dO[0][c] = dA0 - dA1;
      se[1][c] = sB0 + sB1;
      so[1][c] = sB0 - sB1;
      de[1][c] = dB0 + dB1;
      dO[1][c] = dB0 - dB1;
    }
    C* f = sF + (jj * hp + l) * SP;
    stv<C, CB>(f + wA, se[0]);
    stv<C, CB>(f + QS + wA, so[0]);
    stv<C, CB>(f + 2 * QS + wA, de[0]);
    stv<C, CB>(f + 3 * QS + wA, dO[0]);
    stv<C, CB>(f + wB, se[1]);
    stv<C, CB>(f + QS + wB, so[1]);
    stv<C, CB>(f + 2 * QS + wB, de[1]);
    stv<C, CB>(f + 3 * QS + wB, dO[1]);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int j = side ? N - 1 - jj : jj;
      C sg0[CB], dl0[CB], sg1[CB], dl1[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        sg0[c] = a0[side][c] + b0[side][c];   // phi pair halves at column A
        dl0[c] = a0[side][c] - b0[side][c];
        sg1[c] = a1[side][c] + b1[side][c];   // and at column B
        dl1[c] = a1[side][c] - b1[side][c];
      }
      stv<C, CB>(su + (j * N + l) * W + wA, sg0);
      stv<C, CB>(su + (j * N + l + hp) * W + wA, dl0);
      stv<C, CB>(su + (j * N + l) * W + wB, sg1);
      stv<C, CB>(su + (j * N + l + hp) * W + wB, dl1);
    }
  }
  __syncthreads();
  const C ir = t.inv_r[i];
  const C* sPe = sP;
  const C* sPo = sP + hp * hp;
  const C* sQe = sQ;
  const C* sQo = sQ + hp * hp;
  for (int unit = threadIdx.x; unit < S::units; unit += blockDim.x) {
    const int mq = unit % HC, r1 = unit / HC, kl = r1 % KT, r2 = r1 / KT;
    const int l = r2 % hp, j0 = r2 / hp, j1 = N - 1 - j0;
    const int m0 = mq * CB;
    const int wA = kl * N + m0, wB = wA + hp;      // columns m0.. and m0 + N/2..
    // theta: [column A / B][even / odd of P / Q]
    C aEA[CB], aOA[CB], bEA[CB], bOA[CB], aEB[CB], aOB[CB], bEB[CB], bOB[CB];
    // phi: [row j0 / mirror j1][column A / B]
    C fs[2][2][CB], fd[2][2][CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      aEA[c] = aOA[c] = bEA[c] = bOA[c] = aEB[c] = aOB[c] = bEB[c] = bOB[c] = 0;
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int ab = 0; ab < 2; ++ab) fs[s2][ab][c] = fd[s2][ab][c] = 0;
    }
#pragma unroll
    for (int jj = 0; jj < hp; ++jj) {
      const C* f = sF + (jj * hp + l) * SP;
      C v[8][CB];
      ldv<C, CB>(f + wA, v[0]);
      ldv<C, CB>(f + QS + wA, v[1]);
      ldv<C, CB>(f + 2 * QS + wA, v[2]);
      ldv<C, CB>(f + 3 * QS + wA, v[3]);
      ldv<C, CB>(f + wB, v[4]);
      ldv<C, CB>(f + QS + wB, v[5]);
      ldv<C, CB>(f + 2 * QS + wB, v[6]);
      ldv<C, CB>(f + 3 * QS + wB, v[7]);
      const C Pe = sPe[jj * hp + j0], Po = sPo[jj * hp + j0];
      const C Qe = sQe[jj * hp + j0], Qo = sQo[jj * hp + j0];
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        aEA[c] = fmac(Pe, v[0][c], aEA[c]);
        aOA[c] = fmac(Po, v[1][c], aOA[c]);
        bEA[c] = fmac(Qe, v[2][c], bEA[c]);
        bOA[c] = fmac(Qo, v[3][c], bOA[c]);
        aEB[c] = fmac(Pe, v[4][c], aEB[c]);
        aOB[c] = fmac(Po, v[5][c], aOB[c]);
        bEB[c] = fmac(Qe, v[6][c], bEB[c]);
        bOB[c] = fmac(Qo, v[7][c], bOB[c]);
      }
    }
#pragma unroll
    for (int ll = 0; ll < hp; ++ll) {
      const C Ms = sD[ll * hp + l], Md = sD[hp * hp + ll * hp + l];
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        const int j = s2 ? j1 : j0;
        C sa[CB], da_[CB], sb[CB], db_[CB];
        ldv<C, CB>(su + (j * N + ll) * W + wA, sa);
        ldv<C, CB>(su + (j * N + ll + hp) * W + wA, da_);
        ldv<C, CB>(su + (j * N + ll) * W + wB, sb);
        ldv<C, CB>(su + (j * N + ll + hp) * W + wB, db_);
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          fs[s2][0][c] = fmac(Ms, sa[c], fs[s2][0][c]);
          fd[s2][0][c] = fmac(Md, da_[c], fd[s2][0][c]);
          fs[s2][1][c] = fmac(Ms, sb[c], fs[s2][1][c]);
          fd[s2][1][c] = fmac(Md, db_[c], fd[s2][1][c]);
        }
      }
    }
    const C sTk = sgn * t.sinT[k0 + kl] * ir;
    C cA[CB], sA[CB], cB[CB], sB[CB];   // a_phi carries the 1/2 of the phi pair halves
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      cA[c] = (C)0.5 * sTk * t.cosP[m0 + c];   // and a_theta the 1/2 of the theta folding
      sA[c] = (C)0.5 * sTk * t.sinP[m0 + c];
      cB[c] = (C)0.5 * sTk * t.cosP[m0 + hp + c];
      sB[c] = (C)0.5 * sTk * t.sinP[m0 + hp + c];
    }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int j = s2 ? j1 : j0;
      const C sg = s2 ? (C)-1 : (C)1;
      const C isn = t.inv_sinth[j];
      T* p0 = K + base + (long long)j * d.S_j + (long long)l * d.S_l + kl * N + m0;
      T* p1 = p0 + (long long)hp * d.S_l;      // phi partner row l + N/2
      T k0a[CB], k0b[CB], k1a[CB], k1b[CB];
      if (p.plane_store) {
#pragma unroll
        for (int c = 0; c < CB; ++c) k0a[c] = k0b[c] = k1a[c] = k1b[c] = (T)0;
      } else {
        ldv<T, CB>(p0, k0a);
        ldv<T, CB>(p0 + hp, k0b);
        ldv<T, CB>(p1, k1a);
        ldv<T, CB>(p1 + hp, k1b);
      }
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const C psA = aOA[c] + sg * aEA[c], qdA = bOA[c] + sg * bEA[c];   // x 2
        const C psB = aOB[c] + sg * aEB[c], qdB = bOB[c] + sg * bEB[c];
        const C fA = fs[s2][0][c], gA = fd[s2][0][c], fB = fs[s2][1][c], gB = fd[s2][1][c];
        k0a[c] = (T)((C)k0a[c] + cA[c] * (psA + qdA) + sA[c] * isn * (fA + gA));
        k0b[c] = (T)((C)k0b[c] + cB[c] * (psB + qdB) + sB[c] * isn * (fB + gB));
        k1a[c] = (T)((C)k1a[c] + cA[c] * (psB - qdB) + sA[c] * isn * (fA - gA));
        k1b[c] = (T)((C)k1b[c] + cB[c] * (psA - qdA) + sB[c] * isn * (fB - gB));
      }
      stv<T, CB>(p0, k0a);
      stv<T, CB>(p0 + hp, k0b);
      stv<T, CB>(p1, k1a);
      stv<T, CB>(p1 + hp, k1b);
    }
  }
}

template <typename T, typename C, int N, int KT>
__global__ void __launch_bounds__(kThreads, 2)
k_plane_sq(Problem p, Tables<C> t, const T* __restrict__ U, T* __restrict__ K, C sgn,
           long long ntiles) {
  using S = PlaneSq<N, KT, C>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  C* sP = reinterpret_cast<C*>(smem_raw);
  C* sQ = sP + N * N;
  C* sD = sQ + N * N;
  C* buf0 = sD + N * N;
  C* sF = buf0 + 2 * S::TS;
  plane_sq_mats<C>(t, d, sP, sQ, sD);
  long long tile = blockIdx.x;
  if (tile < ntiles) plane_sq_load<N, KT, T, C>(d, U, tile, buf0);
  cp_async_commit();
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const long long next = tile + gridDim.x;
    C* cur = buf0 + (it & 1) * S::TS;
    C* nxt = buf0 + ((it + 1) & 1) * S::TS;
    if (next < ntiles) plane_sq_load<N, KT, T, C>(d, U, next, nxt);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    plane_sq_body<N, KT, T, C>(p, t, cur, sF, sP, sQ, sD, K, sgn, tile);
    __syncthreads();
  }
  cp_async_wait0();
}

// ============================================================================
// Radial pass. Thread: RB output pairs (i, N-i) x 4 columns of one tile of W
// (Theta, Phi) columns at fixed (g, theta, phi). The even/odd parts of U are
// formed straight from global memory into shared memory; each thread then
// contracts them, adds the result to its rows of K (read from global memory),
// publishes rows 0 and N (the Tau rows read them), and after one barrier
// applies the Tau rows and the RK4 stage update to its own rows. The middle
// node (odd Nr) is handled by the threads of the rows nearest to it; rows
// 0..n64-1 and N-n64+1..N (n64 = p.n_fp64_rows) are accumulated in double from
// the full matrix.
// Shared layout: [EpT | OpT | DrMc | DrMr | E hh*W | O hh*W | middle W |
//                 K rows 0, N 2W | double rows 4W]
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

// Stage update of one row segment (4 columns at gi) with the finished K values kv.
template <typename T, typename C>
__device__ __forceinline__ void radial_store(int mode, long long gi, const C (&kv)[4], T* F,
                                             T* Acc, T* Uout, T* out, C dt) {
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
  } else if (mode >= RAD_AB2) {
    // in place: every read of this tile's F lines happened before the tile's barrier
    T f[4], ac[4];
    ld4<T>(F + gi, f);
    if (mode == RAD_AB2) ld4<T>(Acc + gi, ac);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const C inc = mode == RAD_AB2 ? (C)1.5 * kv[cc] - (C)0.5 * (C)ac[cc] : kv[cc];
      o[cc] = (T)((C)f[cc] + dt * inc);
      ac[cc] = (T)kv[cc];
    }
    st4<T>(Acc + gi, ac);
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

template <int Nr_, typename T, typename C>
__device__ __forceinline__ void radial_rb_body(const Problem& p, const Tables<C>& t,
                                               const double* __restrict__ Dr64,
                                               const T* __restrict__ U,
                                               const T* __restrict__ Kin, C* sEv, const C* sE,
                                               const C* sO, const C* sMc, const C* sMr, C sgn,
                                               int tau, int mode, T* F, T* Acc, T* Uout, T* out,
                                               C dt, int W, long long tile) {
  constexpr int RB = RBRad<C>::v, CB = 4;
  const Dims& d = p.d;
  const int Nr = ctsz<Nr_>(d.Nr), N = Nr - 1, hh = Nr / 2, NP = d.NP;
  const bool odd = Nr & 1;
  const long long Si = d.S_i;
  C* sOd = sEv + hh * W;
  C* sMid = sOd + hh * W;
  C* sBnd = sMid + W;
  C* sR = sBnd + 2 * W;
  long long base;
  int c0, Wc;
  radial_tile_coords(d, W, tile, base, c0, Wc);
  const int W4 = Wc / 4;
  const int n64 = p.n_fp64_rows;
  const T* Ub = U + base;
  {
    // even/odd parts once per pair; UL row pairs per trip, all their loads
    // issued before the first store
    constexpr int UL = sizeof(T) == 4 ? 4 : 2;
    const int n = hh * W4;
    for (int x0 = threadIdx.x; x0 < n; x0 += UL * (int)blockDim.x) {
      T a[UL][4], b[UL][4];
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        const int x = x0 + u * (int)blockDim.x;
        if (x < n) {
          const int ii = x / W4, w = (x - ii * W4) * 4;
          ld4<T>(Ub + ii * Si + w, a[u]);
          ld4<T>(Ub + (N - ii) * Si + w, b[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        const int x = x0 + u * (int)blockDim.x;
        if (x < n) {
          const int ii = x / W4, w = (x - ii * W4) * 4;
          C e[4], o[4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            e[cc] = (C)a[u][cc] + (C)b[u][cc];
            o[cc] = (C)a[u][cc] - (C)b[u][cc];
          }
          st4<C>(sEv + ii * W + w, e);
          st4<C>(sOd + ii * W + w, o);
        }
      }
    }
  }
  if (odd) {
    for (int x = threadIdx.x; x < W4; x += blockDim.x) {
      T a[4];
      ld4<T>(Ub + (N / 2) * Si + 4 * x, a);
      C m[4] = {(C)a[0], (C)a[1], (C)a[2], (C)a[3]};
      st4<C>(sMid + 4 * x, m);
    }
  }
  // rows nearest the ends in double: the row pairs (i, N-i), i < n64, from the
  // even / odd parts of the line, folded like the float rows (half the
  // multiply-adds of two dense rows): row i = (Op O + Ep E)/2 + D[i][M] u_M,
  // row N-i = (Op O - Ep E)/2 - D[i][M] u_M. One thread per column forms each
  // even / odd value once, in double (the sum and difference of two floats are
  // exact there), and feeds it to every pair: two conversions, two additions and
  // 2 n64 multiply-adds per line point pair.
  if (n64 > 0) {
    // tpc threads per column (adjacent lanes), each over every tpc-th point pair,
    // summed by shuffles: long lines keep every thread of the tile busy
    constexpr int M64 = 2;   // at most two pairs (TS_FP32_R64)
    int tpc = 1;
    while (tpc < 8 && 2 * tpc * Wc <= (int)blockDim.x) tpc *= 2;
    for (int v0 = 0; v0 < Wc * tpc; v0 += blockDim.x) {   // uniform trip count
      const int v = v0 + (int)threadIdx.x;
      const bool act = v < Wc * tpc;
      const int w = act ? v / tpc : 0, part = v % tpc;
      double ae[M64] = {0, 0}, ao[M64] = {0, 0};
      // point pairs ii = part, part + stride, ... of column w
      auto sum = [&](int first, int stride) {
#pragma unroll 4
        for (int ii = first; ii < hh; ii += stride) {
          const double a = widen_f32((float)Ub[ii * Si + w]);
          const double b = widen_f32((float)Ub[(N - ii) * Si + w]);
          const double e = a + b, o = a - b;
#pragma unroll
          for (int q = 0; q < M64; ++q) {
            if (q < n64) {
              ae[q] = fma(p.ep64[ii * hh + q], e, ae[q]);
              ao[q] = fma(p.op64[ii * hh + q], o, ao[q]);
            }
          }
        }
      };
      if (act) {
        if (tpc == 1) sum(0, 1);   // the whole line (a compile-time trip count)
        else sum(part, tpc);
      }
      for (int o = tpc >> 1; o; o >>= 1) {   // the tpc lanes of a column (whole warps take part)
#pragma unroll
        for (int q = 0; q < M64; ++q) {
          ae[q] += __shfl_xor_sync(0xffffffffu, ae[q], o);
          ao[q] += __shfl_xor_sync(0xffffffffu, ao[q], o);
        }
      }
      if (act && part == 0) {
        const double um = odd ? widen_f32((float)Ub[(N / 2) * Si + w]) : 0.0;
#pragma unroll
        for (int q = 0; q < M64; ++q) {
          if (q < n64) {
            const double mid = odd ? p.mc64[q] * um : 0.0;
            sR[q * W + w] = (C)(0.5 * (ao[q] + ae[q]) + mid);
            sR[(n64 + q) * W + w] = (C)(0.5 * (ao[q] - ae[q]) - mid);
          }
        }
      }
    }
  }
  __syncthreads();
  const int IR = hh / RB, units = IR * W4;
  const int rounds = (units + (int)blockDim.x - 1) / (int)blockDim.x;
  for (int rd = 0; rd < rounds; ++rd) {   // uniform trip count: every thread meets the barrier
    const int unit = rd * (int)blockDim.x + (int)threadIdx.x;
    const bool act = unit < units;
    const int wq = act ? unit % W4 : 0, ir = act ? unit / W4 : 0;
    const int w0 = wq * CB, i0 = ir * RB;
    const bool mid = odd && ir == IR - 1;
    C klo[RB][CB], khi[RB][CB], kmid[CB];
    C cT = 0, ckf = 0;
    if (act) {
      // this thread's K rows, and the F / Acc rows of its stage update, are
      // requested before the contraction so that their latency overlaps it
      T k1[RB][CB], k2[RB][CB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const long long g1 = base + (i0 + r) * Si + w0, g2 = base + (N - i0 - r) * Si + w0;
        ld4<T>(Kin + g1, k1[r]);
        ld4<T>(Kin + g2, k2[r]);
        if (mode != RAD_RHS) {
          prefetch_l2(F + g1);
          prefetch_l2(F + g2);
          if (mode != RAD_STAGE0 && mode != RAD_AB2_START) {
            prefetch_l2(Acc + g1);
            prefetch_l2(Acc + g2);
          }
        }
      }
      C ae[RB][CB], ao[RB][CB];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) ae[r][cc] = ao[r][cc] = 0;
#pragma unroll 8
      for (int ii = 0; ii < hh; ++ii) {
        C ev[CB], ov[CB], E[RB], O[RB];
        ld4<C>(sEv + ii * W + w0, ev);
        ld4<C>(sOd + ii * W + w0, ov);
        ldv<C, RB>(sE + ii * hh + i0, E);
        ldv<C, RB>(sO + ii * hh + i0, O);
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) {
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            ae[r][cc] = fmac(E[r], ev[cc], ae[r][cc]);
            ao[r][cc] = fmac(O[r], ov[cc], ao[r][cc]);
          }
        }
      }
      cT = t.cosT[(c0 + w0) / NP];   // 4 | w0, 8 | NP: the 4 columns share one Theta row
      ckf = sgn * cT;
      if (odd) {
        C um[CB];
        ld4<C>(sMid + w0, um);
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int cc = 0; cc < CB; ++cc) ae[r][cc] = fmac((C)2 * sMc[i0 + r], um[cc], ae[r][cc]);
      }
      if (mid) {
        C am[CB] = {0, 0, 0, 0};
#pragma unroll
        for (int ii = 0; ii < hh; ++ii) {
          C ov[CB];
          ld4<C>(sOd + ii * W + w0, ov);
          const C mr = sMr[ii];
#pragma unroll
          for (int cc = 0; cc < CB; ++cc) am[cc] = fmac(mr, ov[cc], am[cc]);
        }
        T km[CB];
        ld4<T>(Kin + base + (N / 2) * Si + w0, km);
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) kmid[cc] = (C)km[cc] + ckf * am[cc];
      }
      const C ck = ckf * (C)0.5;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = i0 + r;
        if (i < n64) {
#pragma unroll
          for (int cc = 0; cc < CB; ++cc) {
            klo[r][cc] = (C)k1[r][cc] + ckf * sR[i * W + w0 + cc];
            khi[r][cc] = (C)k2[r][cc] + ckf * sR[(n64 + i) * W + w0 + cc];
          }
        } else {
#pragma unroll
          for (int cc = 0; cc < CB; ++cc) {
            klo[r][cc] = (C)k1[r][cc] + ck * (ao[r][cc] + ae[r][cc]);
            khi[r][cc] = (C)k2[r][cc] + ck * (ao[r][cc] - ae[r][cc]);
          }
        }
      }
      if (i0 == 0) {   // rows 0 and N of these columns: the Tau rows read them
        st4<C>(sBnd + w0, klo[0]);
        st4<C>(sBnd + W + w0, khi[0]);
      }
    }
    __syncthreads();
    if (act) {
      C kb[CB];
      const int b = cT > (C)0 ? 0 : N;   // inflow node: cos(Theta) > 0 at R1
      if (tau) ld4<C>(sBnd + (b ? W : 0) + w0, kb);
      const C tb = t.tsign[b];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = i0 + r;
        if (tau) {
          const C s1 = tb * t.tsign[i], s2 = tb * t.tsign[N - i];
#pragma unroll
          for (int cc = 0; cc < CB; ++cc) {
            klo[r][cc] -= kb[cc] * s1;
            khi[r][cc] -= kb[cc] * s2;
          }
        }
        radial_store<T, C>(mode, base + i * Si + w0, klo[r], F, Acc, Uout, out, dt);
        radial_store<T, C>(mode, base + (N - i) * Si + w0, khi[r], F, Acc, Uout, out, dt);
      }
      if (mid) {
        if (tau) {
          const C s = tb * t.tsign[N / 2];
#pragma unroll
          for (int cc = 0; cc < CB; ++cc) kmid[cc] -= kb[cc] * s;
        }
        radial_store<T, C>(mode, base + (N / 2) * Si + w0, kmid, F, Acc, Uout, out, dt);
      }
    }
  }
}

template <int Nr_, typename T, typename C>
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
  C* sEv = sMr + h4;
  radial_rb_mats<C>(t, Nr, sE, sO, sMc, sMr);
  radial_rb_body<Nr_, T, C>(p, t, Dr64, U, Kin, sEv, sE, sO, sMc, sMr, sgn, tau, mode, F, Acc,
                            Uout, out, dt, W, tile);
}

// One tile per CTA with the radial line length fixed at compile time.
// Four CTAs per SM in float (64 registers: a few bytes of spills, more warps to
// hide the latency of the line loads), two in double.
template <typename T, typename C, int Nr_>
__global__ void __launch_bounds__(kThreads, sizeof(C) == 4 ? 4 : 2)
k_radial_eo(Problem p, Tables<C> t, const double* __restrict__ Dr64, const T* U, const T* Kin,
            C sgn, int tau, int mode, T* F, T* Acc, T* Uout, T* out, C dt, int W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nr = ctsz<Nr_>(p.d.Nr), hh = Nr / 2;
  const int hh4 = (hh * hh + 3) & ~3, h4 = (hh + 3) & ~3;
  C* sE = reinterpret_cast<C*>(smem_raw);
  C* sO = sE + hh4;
  C* sMc = sO + hh4;
  C* sMr = sMc + h4;
  C* sEv = sMr + h4;
  radial_rb_mats<C>(t, Nr, sE, sO, sMc, sMr);
  radial_rb_body<Nr_, T, C>(p, t, Dr64, U, Kin, sEv, sE, sO, sMc, sMr, sgn, tau, mode, F, Acc,
                            Uout, out, dt, W, blockIdx.x);
}

// ----------------------------------------------------------------------------
// Pass dispatch (register-blocked form where the grid allows it) and the
// single-problem one-tile-per-CTA kernels (generic form, or rb without a
// persistent launch).
template <typename T, typename C>
__device__ __forceinline__ void angular_tile_any(const Problem& p, const Tables<C>& t,
                                                 const T* U, T* K, C sgn, int collision, int nb,
                                                 long long tile) {
  if (p.tp.rb & 1) angular_tile_rb<0, 0, T, C>(p, t, U, K, sgn, collision, nb, tile);
  else angular_tile<T, C>(p, t, U, K, sgn, collision, nb, tile);
}

template <typename T, typename C>
__device__ __forceinline__ void plane_tile_any(const Problem& p, const Tables<C>& t, const T* U,
                                               T* K, C sgn, int c, long long tile) {
  if (p.tp.rb & 2) plane_tile_rb<0, T, C>(p, t, U, K, sgn, c, tile);
  else plane_tile<T, C>(p, t, U, K, sgn, c, tile);
}

template <typename T, typename C>
__device__ __forceinline__ void radial_tile_any(const Problem& p, const Tables<C>& t,
                                                const double* Dr64, const T* U, const T* Kin,
                                                C sgn, int tau, int mode, T* F, T* Acc, T* Uout,
                                                T* out, C dt, int W, long long tile) {
  if (p.tp.rb & 4)
    radial_tile_rb<0, T, C>(p, t, Dr64, U, Kin, sgn, tau, mode, F, Acc, Uout, out, dt, W, tile);
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
