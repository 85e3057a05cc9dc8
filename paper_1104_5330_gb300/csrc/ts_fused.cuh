// Fused angular + radial pass of one stage derivative (float grids).
//
// One RK4 or AB2 stage needs every axis of U: the plane pass supplies the
// theta and phi terms (written, not accumulated, into K), and this pass does
// the rest for one (g, theta_j, phi_l) position at a time -- all N_r radial
// nodes and every direction (Theta, Phi), a tile of N_r contiguous angular
// blocks at stride S_i:
//   1. the tile of U is staged in shared memory (16-byte cp.async; with two
//      staging buffers the next tile's copy runs under the current tile);
//   2. angular phase, per angular block (fixed r): the Theta and Phi
//      derivatives on the DFS pair halves (the folded forms of the angular
//      pass), J (and H, M for anisotropic kernels) and the collision term,
//      written to a shared-memory K tile;
//   3. the radial rows in double (TS_FP32_R64) from the staged values, then the
//      staged U is replaced in place by its radial even/odd parts
//      E_i = u_i + u_{N-i}, O_i = u_i - u_{N-i};
//   4. radial phase, per thread RB row pairs (i, N-i) x 4 columns: the radial
//      derivative from E and O through the folded D_r halves, plus the angular
//      K tile and the plane terms read from global memory; the Tau rows (the K
//      values at rows 0 and N go through shared memory); the stage update.
// Per point this moves U once (read), the plane terms once (read), and the
// stage update's fields (F, Acc read; U or F, Acc written) -- against the
// three-pass form it saves one read of U and one read and one write of K.
//
// Requirements (host-checked): the register-blocked angular and radial forms
// apply (rb_mask 1 and 4), and the tile fits shared memory (fused_shape).
#pragma once

#include "ts_kernels_rb.cuh"

namespace ts {

constexpr int kFusedThreads = 512;

struct FusedShape {
  int nb;      // angular blocks per chunk of the angular phase
  int nbuf;    // U staging buffers (2: double-buffered)
  size_t amat, rmat, su, sK, sSD, uT, sc, sR, bytes;   // offsets in elements of C
};

// Shared-memory layout of the fused pass (elements of the compute type):
//   [angular matrices | radial matrices | U tile x nbuf | K tile | folded halves
//    nb*SS | transposed halves nb*US | per-block scalars | double-precision rows]
template <typename C>
__host__ __device__ inline FusedShape fused_shape(const Dims& d, int n64, int nb, int nbuf) {
  FusedShape f;
  const size_t S = (size_t)d.NT * d.NP, tile = (size_t)d.Nr * S;
  const int hh = d.Nr / 2;
  f.nb = nb;
  f.nbuf = nbuf;
  f.amat = 0;
  f.rmat = f.amat + 2 * (size_t)d.NT * d.NT + (size_t)d.NP * d.NP;
  f.su = f.rmat + 2 * (size_t)((hh * hh + 3) & ~3) + 2 * (size_t)((hh + 3) & ~3);
  f.sK = f.su + nbuf * tile;
  f.sSD = f.sK + tile;
  f.uT = f.sSD + (size_t)nb * ang_ss(d.NT, d.NP);
  f.sc = f.uT + (size_t)nb * ang_us<C>(d.NT, d.NP);
  f.sR = f.sc + (size_t)((kAngScalars * nb + 3) & ~3);
  f.bytes = (f.sR + 2 * (size_t)n64 * S + 2 * S) * sizeof(C);   // + rows 0 and N of K
  return f;
}

template <int Nr_, int NA_, int KF, typename T, typename C>
__global__ void __launch_bounds__(kFusedThreads, 1)
k_fused(Problem p, Tables<C> t, const double* __restrict__ Dr64, const T* __restrict__ U,
        const T* __restrict__ Kp, C sgn,
        int collision, int tau, int mode, T* F, T* Acc, T* Uout, T* out, C dt, int nb, int nbuf,
        long long ntiles) {
  constexpr int RB = RBRad<C>::v, CB = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const Dims& d = p.d;
  const int Nr = ctsz<Nr_>(d.Nr), N = Nr - 1, hh = Nr / 2;
  const int NT = ctsz<NA_>(d.NT), NP = ctsz<NA_>(d.NP), S = NT * NP;
  const bool odd = Nr & 1;
  const long long Si = d.S_i, nJ = (long long)d.Nt * d.Np;
  const int n64 = p.n_fp64_rows;
  const FusedShape fs = fused_shape<C>(d, n64, nb, nbuf);
  C* sP = sm + fs.amat;
  C* sQ = sP + NT * NT;
  C* sD = sQ + NT * NT;
  const int hh4 = (hh * hh + 3) & ~3, h4 = (hh + 3) & ~3;
  C* sE = sm + fs.rmat;
  C* sO = sE + hh4;
  C* sMc = sO + hh4;
  C* sMr = sMc + h4;
  C* sK = sm + fs.sK;
  C* sSD = sm + fs.sSD;
  C* uT = sm + fs.uT;
  C* sc = sm + fs.sc;
  C* sR = sm + fs.sR;
  C* sBnd = sR + 2 * n64 * S;
  angular_rb_mats<C>(t, d, sP, sQ, sD);
  radial_rb_mats<C>(t, Nr, sE, sO, sMc, sMr);

  auto tile_base = [&](long long tl) {   // offset of (g, i = 0, j, l, 0, 0)
    const int l = (int)(tl % d.Np);
    const long long q = tl / d.Np;
    const int j = (int)(q % d.Nt);
    const int g = (int)(q / d.Nt);
    return (long long)g * d.S_g + (long long)j * d.S_j + (long long)l * d.S_l;
  };
  auto stage = [&](long long tl, C* dst) {   // the N_r blocks of a tile, 16-byte copies
    const T* src = U + tile_base(tl);
    for (int x = 4 * (int)threadIdx.x; x < Nr * S; x += 4 * (int)blockDim.x) {
      const int i = x / S, w = x - i * S;
      copy4<true, T, C>(dst + x, src + (long long)i * Si + w);
    }
  };

  long long tile = blockIdx.x;
  int cur = 0;
  if (tile < ntiles) stage(tile, sm + fs.su);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    C* su = sm + fs.su + (size_t)cur * Nr * S;
    cp_async_wait0();
    __syncthreads();   // this tile staged; every phase of the previous tile done
    const long long next = tile + gridDim.x;
    if (nbuf == 2 && next < ntiles) stage(next, sm + fs.su + (size_t)(cur ^ 1) * Nr * S);
    cp_async_commit();
    const long long base = tile_base(tile);
    const int l = (int)(tile % d.Np);
    const int g = (int)(tile / nJ), j = (int)((tile / d.Np) % d.Nt);
    const long long blk0 = ((long long)g * Nr * d.Nt + j) * d.Np + l;   // block (g, 0, j, l)

    // 2. angular phase, nb blocks (radial nodes) at a time
    for (int c0 = 0; c0 < Nr; c0 += nb) {
      AngBlocks ab;
      ab.b0 = blk0 + (long long)c0 * nJ;
      ab.bs = nJ;
      ab.nbb = min(nb, Nr - c0);
      angular_rb_prep<NA_, NA_, KF, T, C>(p, t, su + (size_t)c0 * S, sSD, uT, sc, collision, nb,
                                         ab);
      __syncthreads();
      angular_rb_compute<NA_, NA_, KF, C, C>(p, t, sSD, uT, sc, sP, sQ, sD, sK + (size_t)c0 * S,
                                             sgn, collision, nb, ab);
      __syncthreads();
    }

    // 3. double-precision end rows (pairs (i, N-i), i < n64) from the staged
    // values, folded like the float rows; then E/O in place
    const int W4 = S / 4;
    for (int v = threadIdx.x; v < n64 * W4; v += blockDim.x) {
      const int w0 = (v % W4) * 4, i = v / W4;
      double ae[4] = {0, 0, 0, 0}, ao[4] = {0, 0, 0, 0};
      for (int ii = 0; ii < hh; ++ii) {
        C a[4], b[4];
        ld4<C>(su + (size_t)ii * S + w0, a);
        ld4<C>(su + (size_t)(N - ii) * S + w0, b);
        // the folded D_r in double: D[i][ii] + D[i][N-ii] and D[i][ii] - D[i][N-ii]
        const double Ep = p.ep64[ii * hh + i], Op = p.op64[ii * hh + i];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          ae[cc] = fma(Ep, (double)a[cc] + (double)b[cc], ae[cc]);
          ao[cc] = fma(Op, (double)a[cc] - (double)b[cc], ao[cc]);
        }
      }
      C m4[4] = {0, 0, 0, 0};
      if (odd) ld4<C>(su + (size_t)(N / 2) * S + w0, m4);
      const double dm = odd ? p.mc64[i] : 0.0;
      C lo[4], hi[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        // row i = (Op O + Ep E)/2 + D[i][M] u_M; row N-i = (Op O - Ep E)/2 - D[i][M] u_M
        const double mid = dm * (double)m4[cc];
        lo[cc] = (C)(0.5 * (ao[cc] + ae[cc]) + mid);
        hi[cc] = (C)(0.5 * (ao[cc] - ae[cc]) - mid);
      }
      st4<C>(sR + (size_t)i * S + w0, lo);
      st4<C>(sR + (size_t)(n64 + i) * S + w0, hi);
    }
    __syncthreads();
    for (int x = 4 * (int)threadIdx.x; x < hh * S; x += 4 * (int)blockDim.x) {
      const int ii = x / S, w = x - ii * S;
      C a[4], b[4], e[4], o[4];
      ld4<C>(su + (size_t)ii * S + w, a);
      ld4<C>(su + (size_t)(N - ii) * S + w, b);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        e[cc] = a[cc] + b[cc];
        o[cc] = a[cc] - b[cc];
      }
      st4<C>(su + (size_t)ii * S + w, e);
      st4<C>(su + (size_t)(N - ii) * S + w, o);
    }
    __syncthreads();

    // 4. radial phase
    const int IR = hh / RB, units = IR * W4;
    const int rounds = (units + (int)blockDim.x - 1) / (int)blockDim.x;
    for (int rd = 0; rd < rounds; ++rd) {   // uniform trip count: every thread meets the barrier
      const int unit = rd * (int)blockDim.x + (int)threadIdx.x;
      const bool act = unit < units;
      const int wq = act ? unit % W4 : 0, ir = act ? unit / W4 : 0;
      const int w0 = wq * CB, i0 = ir * RB;
      const bool mid = odd && ir == IR - 1;
      C klo[RB][CB], khi[RB][CB], kmid[CB];
      C cT = 0;
      if (act) {
        // the plane terms of this thread's rows, and the F / Acc rows of its stage
        // update, are requested before the contraction
        T k1[RB][CB], k2[RB][CB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const long long g1 = base + (i0 + r) * Si + w0, g2 = base + (N - i0 - r) * Si + w0;
          ld4<T>(Kp + g1, k1[r]);
          ld4<T>(Kp + g2, k2[r]);
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
          ld4<C>(su + (size_t)ii * S + w0, ev);
          ld4<C>(su + (size_t)(N - ii) * S + w0, ov);
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
        cT = t.cosT[w0 / NP];   // 4 | w0, 8 | NP: the 4 columns share one Theta row
        const C ckf = sgn * cT;
        if (odd) {
          C um[CB];
          ld4<C>(su + (size_t)(N / 2) * S + w0, um);
#pragma unroll
          for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int cc = 0; cc < CB; ++cc)
              ae[r][cc] = fmac((C)2 * sMc[i0 + r], um[cc], ae[r][cc]);
        }
        if (mid) {
          C am[CB] = {0, 0, 0, 0};
#pragma unroll 8
          for (int ii = 0; ii < hh; ++ii) {
            C ov[CB];
            ld4<C>(su + (size_t)(N - ii) * S + w0, ov);
            const C mr = sMr[ii];
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) am[cc] = fmac(mr, ov[cc], am[cc]);
          }
          T km[CB];
          C ka[CB];
          ld4<T>(Kp + base + (N / 2) * Si + w0, km);
          ld4<C>(sK + (size_t)(N / 2) * S + w0, ka);
#pragma unroll
          for (int cc = 0; cc < CB; ++cc) kmid[cc] = (C)km[cc] + ka[cc] + ckf * am[cc];
        }
        const C ck = ckf * (C)0.5;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const int i = i0 + r;
          C a1[CB], a2[CB];
          ld4<C>(sK + (size_t)i * S + w0, a1);
          ld4<C>(sK + (size_t)(N - i) * S + w0, a2);
          if (i < n64) {
            C d1[CB], d2[CB];
            ld4<C>(sR + (size_t)i * S + w0, d1);
            ld4<C>(sR + (size_t)(n64 + i) * S + w0, d2);
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) {
              klo[r][cc] = (C)k1[r][cc] + a1[cc] + ckf * d1[cc];
              khi[r][cc] = (C)k2[r][cc] + a2[cc] + ckf * d2[cc];
            }
          } else {
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) {
              klo[r][cc] = (C)k1[r][cc] + a1[cc] + ck * (ao[r][cc] + ae[r][cc]);
              khi[r][cc] = (C)k2[r][cc] + a2[cc] + ck * (ao[r][cc] - ae[r][cc]);
            }
          }
        }
        if (i0 == 0) {   // rows 0 and N of these columns: the Tau rows read them
          st4<C>(sBnd + w0, klo[0]);
          st4<C>(sBnd + S + w0, khi[0]);
        }
      }
      __syncthreads();
      if (act) {
        C kb[CB];
        const int b = cT > (C)0 ? 0 : N;   // inflow node: cos(Theta) > 0 at R1
        if (tau) ld4<C>(sBnd + (b ? S : 0) + w0, kb);
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
    if (nbuf == 1) {
      __syncthreads();   // the staging buffer is free again
      if (next < ntiles) stage(next, sm + fs.su);
      cp_async_commit();
    } else {
      cur ^= 1;
    }
  }
  cp_async_wait0();
}

}  // namespace ts
