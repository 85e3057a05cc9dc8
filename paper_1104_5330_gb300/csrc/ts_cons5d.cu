// The conservative form of App. A (Eq. Cohercons) and the number balance of the
// grid's operator (Eqs. Cons, Npho, Flux).
//
// State Fhat = r^2 sin(theta) sin(Theta) F. Its r, theta and phi fluxes are a
// velocity that is constant along the axis times Fhat, so the plane and radial
// passes of the advective form serve unchanged -- with the theta tables of the
// odd double-Fourier-sphere continuation (Fhat carries sin theta: the reflected
// node holds minus Fhat at the partner), which the grid builds in place of the
// even ones. This file holds the angular pass of the conservative form:
//   K = sgn [ -(1/r) (sin Th D_Th Fhat + cos Th P Fhat)              (Theta flux)
//             - (sin Th cot th / r) D_Ph (sin Ph Fhat) ]              (Phi flux)
//       + r^2 sin th sin Th eta - (kappa + kappa_s) Fhat
//       + kappa_s sin Th (J + b omega.H + c omega.M~.omega)[Fhat / sin Th]
// D_Th on the odd continuation (partner at Phi + pi, minus sign), P the removal
// of the Nyquist bin of the doubled Theta circle, the moments J, H, M~ of
// G = Fhat / sin Th (those of F times r^2 sin th, which the volume element's
// factor cancels). The DFS pair (k, m), (k, m + NP/2) is formed once:
//   s = Fhat(m) + Fhat(m+h), d = Fhat(m) - Fhat(m+h):
//   D_Th Fhat (k, m) = P s + Q d,  (k, m+h) = P s - Q d
// (P = (A + B)/2, Q = (A - B)/2 of the odd continuation's halves A, B), and the
// circulant Phi derivative on the pair halves of v = sin Ph Fhat:
//   sig = v(q) + v(q+h), del = v(q) - v(q+h):
//   D v (p) = (Ms sig + Md del)/2,  D v (p+h) = (Ms sig - Md del)/2,
// half the multiply-adds of the dense products. P and Q are centro-antisymmetric
// (the Theta nodes are symmetric about pi/2), so rows k and NT-1-k come from the
// Theta-even and -odd parts of s and d through half-size tables: a quarter of the
// dense Theta multiply-adds in all. Since sin(Ph_{q+h}) = -sin(Ph_q), sig and del
// are sin(Ph_q) d(q) and sin(Ph_q) s(q): the kernel folds sin(Ph_q)/2 into Ms, Md
// and needs no array of v. The Nyquist bin of the doubled circle (2 NT nodes, the
// reflected node 2NT-1-j carrying -Fhat(j, m+h)) is
//   c(m) = (1/2NT) sum_j (-1)^j (Fhat(j, m) + Fhat(j, m+h)),
//   P Fhat (k, m) = Fhat(k, m) - (-1)^k c(m),   c(m + h) = c(m).
// The pass runs in the grid's element type: double for TS_FP64, float (tables and
// arithmetic) for the float precisions.
//
// Number balance: one warp per angular block sums the block's Theta-Phi
// quadrature of F, K, cos Th F and the source; a second kernel reduces each
// group's blocks in a fixed order.
#include <algorithm>

#include "ts_internal.h"

namespace ts {

namespace {

constexpr int kConsThreads = 256;

struct ConsTile {
  int nb;        // angular blocks per CTA
  size_t bytes;  // dynamic shared memory
};

// Shared layout (elements of T): the Theta halves folded over k -> NT-1-k, Pe,
// Po, Qe, Qo [h][h] (h = NT/2, each with its 1/2) | the Phi pair-half tables
// times sin(Phi_q)/2, Ms, Md [hP][hP] | q_k / sin Th_k [NT], padded to 16 bytes |
// per block: the field [S], the pair sums and differences s, d [NT][hP] each,
// their Theta-even and -odd parts es, os, ed, od [h][hP] each, the Nyquist bins
// [hP], the ten moments and eight scalars.
constexpr int kConsScalars = 8;
size_t cons_table_elems(const Dims& d, size_t es) {
  const size_t hP = d.NP / 2, v = 16 / es;
  return ((size_t)d.NT * d.NT + 2 * hP * hP + d.NT + v - 1) / v * v;
}
size_t cons_block_elems(const Dims& d) {
  const size_t S = (size_t)d.NT * d.NP;
  return 3 * S + d.NP / 2 + 10 + kConsScalars;
}

ConsTile cons_tile(const Dims& d, size_t es) {
  const size_t tab = cons_table_elems(d, es) * es, blk = cons_block_elems(d) * es;
  // two CTAs per SM when a few blocks fit in half the shared memory, else one
  const size_t half = 110 * 1024, full = 220 * 1024;
  const size_t budget = tab + 2 * blk <= half ? half : full;
  long long nb = budget > tab ? (long long)((budget - tab) / blk) : 0;
  nb = std::min<long long>(nb, 16);
  // enough CTAs for every SM
  while (nb > 1 && (d.nblk + nb - 1) / nb < 2 * 152) --nb;
  ConsTile t;
  t.nb = (int)std::max<long long>(nb, 1);
  t.bytes = tab + (size_t)t.nb * blk;
  return t;
}

// One thread per output quadruple (k, NT-1-k) x (c, c + hP), k < NT/2, c < hP:
//   Theta: P s at rows k, NT-1-k from the Theta-even/odd parts of s (P is
//   centro-antisymmetric): A1 = sum Pe e, A2 = sum Po o give P s (k) = A1 + A2,
//   P s (NT-1-k) = A2 - A1; Q d alike; D_Th Fhat (k, c) = P s + Q d,
//   (k, c + hP) = P s - Q d.
//   Phi: v = sin Ph Fhat has pair sums sin(Ph_q) d_q and differences sin(Ph_q) s_q
//   (sin(Ph_{q+hP}) = -sin(Ph_q)), so the tables carry sin(Ph_q)/2 and act on d, s.
// T: the element type of the field, of the tables and of the arithmetic (double
// for TS_FP64, float for the float precisions).
template <typename T>
__global__ void __launch_bounds__(kConsThreads)
k_angular_cons(Problem p, Tables<T> t, const T* __restrict__ U, T* __restrict__ K, T sgn,
               int collision, int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP, hP = NP / 2, H = NT * hP, h = NT / 2,
            Hh = h * hP;
  constexpr int kVec = 16 / sizeof(T);
  const int tabn = (NT * NT + 2 * hP * hP + NT + kVec - 1) / kVec * kVec;
  T* sPe = reinterpret_cast<T*>(smem_raw);   // [kk][k], k, kk < h
  T* sPo = sPe + h * h;
  T* sQe = sPo + h * h;
  T* sQo = sQe + h * h;
  T* sMs = sQo + h * h;                      // [q][c] x sin(Ph_q)/2
  T* sMd = sMs + hP * hP;
  T* sq = sMd + hP * hP;                     // q_k / sin Th_k
  T* su = reinterpret_cast<T*>(smem_raw) + tabn;   // [nb][S], 16-byte aligned
  T* ss = su + (size_t)nb * S;               // [nb][NT][hP]
  T* sd = ss + (size_t)nb * H;
  T* ses = sd + (size_t)nb * H;              // [nb][h][hP]
  T* sos = ses + (size_t)nb * Hh;
  T* sed = sos + (size_t)nb * Hh;
  T* sod = sed + (size_t)nb * Hh;
  T* sc = sod + (size_t)nb * Hh;             // Nyquist bins [nb][hP]
  T* sJ = sc + (size_t)nb * hP;              // moments [10][nb]
  T* sB = sJ + (size_t)10 * nb;              // scalars [nb][kConsScalars]
  const long long b0 = (long long)blockIdx.x * nb;
  const int nbb = (int)min((long long)nb, d.nblk - b0);
  const int kf = kernel_form(p, collision);
  const bool aniso = kf >= KF_LINEAR, quad = kf >= KF_QUADRATIC;

  for (int x = threadIdx.x; x < h * h; x += blockDim.x) {
    sPe[x] = t.PeThT[x];
    sPo[x] = t.PoThT[x];
    sQe[x] = t.QeThT[x];
    sQo[x] = t.QoThT[x];
  }
  for (int x = threadIdx.x; x < hP * hP; x += blockDim.x) {
    const T w = (T)0.5 * t.sinP[x / hP];
    sMs[x] = w * t.MsPhT[x];
    sMd[x] = w * t.MdPhT[x];
  }
  for (int x = threadIdx.x; x < NT; x += blockDim.x) sq[x] = t.qdir[x] / t.sinT[x];
  {
    // S is a multiple of 4 (even NT, NP): the blocks are whole 16-byte vectors
    const uint4* src = reinterpret_cast<const uint4*>(U + b0 * S);
    uint4* dst = reinterpret_cast<uint4*>(su);
    const int nv = (int)((size_t)nbb * S * sizeof(T) / 16);
    for (int x = threadIdx.x; x < nv; x += blockDim.x) dst[x] = src[x];
  }
  __syncthreads();
  // DFS pair sums and differences
  for (int x = threadIdx.x; x < nbb * H; x += blockDim.x) {
    const int bb = x / H, r = x - bb * H, k = r / hP, q = r - k * hP;
    const T a = su[bb * S + k * NP + q], b = su[bb * S + k * NP + q + hP];
    ss[x] = a + b;
    sd[x] = a - b;
  }
  if (collision) {
    // moments of G = Fhat / sin Th, one warp per block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bb = warp; bb < nbb; bb += blockDim.x >> 5) {
      T mo[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // J, H (3), M (6)
      for (int x = lane; x < S; x += 32) {
        const int k = x / NP, m = x - k * NP;
        const T u = su[bb * S + x];
        mo[0] = fma(sq[k], u, mo[0]);
        if (aniso) {
          const T qu = sq[k] * u, qs = t.qdir[k] * u, ct = t.cosT[k];
          const T cp = t.cosP[m], sp = t.sinP[m];
          mo[1] = fma(ct, qu, mo[1]);
          mo[2] = fma(cp, qs, mo[2]);
          mo[3] = fma(sp, qs, mo[3]);
          if (quad) {
            const T qss = t.sinT[k] * qs;
            mo[4] = fma(ct * ct, qu, mo[4]);
            mo[5] = fma(cp * cp, qss, mo[5]);
            mo[6] = fma(sp * sp, qss, mo[6]);
            mo[7] = fma(cp * sp, qss, mo[7]);
            mo[8] = fma(ct * cp, qs, mo[8]);
            mo[9] = fma(ct * sp, qs, mo[9]);
          }
        }
      }
      const int na = quad ? 10 : aniso ? 4 : 1;
#pragma unroll
      for (int a = 0; a < 10; ++a)
        if (a < na)
          for (int o = 16; o; o >>= 1) mo[a] += __shfl_xor_sync(0xffffffffu, mo[a], o);
      if (lane == 0) {
#pragma unroll
        for (int a = 0; a < 10; ++a)
          if (a < na) sJ[a * nb + bb] = mo[a];
      }
    }
  }
  __syncthreads();
  // Theta-even/odd parts of s and d; Nyquist bins; per-block scalars
  for (int x = threadIdx.x; x < nbb * Hh; x += blockDim.x) {
    const int bb = x / Hh, r = x - bb * Hh, kk = r / hP, q = r - kk * hP;
    const T* bs = ss + (size_t)bb * H;
    const T* bd = sd + (size_t)bb * H;
    const T s1 = bs[kk * hP + q], s2 = bs[(NT - 1 - kk) * hP + q];
    const T d1 = bd[kk * hP + q], d2 = bd[(NT - 1 - kk) * hP + q];
    ses[x] = s1 + s2;
    sos[x] = s1 - s2;
    sed[x] = d1 + d2;
    sod[x] = d1 - d2;
  }
  for (int x = threadIdx.x; x < nbb * hP; x += blockDim.x) {
    const int bb = x / hP, q = x - bb * hP;
    T c = 0;
    for (int j = 0; j < NT; ++j) {
      const T v = ss[(size_t)bb * H + j * hP + q];
      c += (j & 1) ? -v : v;
    }
    sc[x] = c / (T)(2 * NT);
  }
  for (int bb = threadIdx.x; bb < nbb; bb += blockDim.x) {
    const long long blk = b0 + bb;
    const int j = (int)((blk / d.Np) % d.Nt);
    const int i = (int)((blk / ((long long)d.Np * d.Nt)) % d.Nr);
    const T ir = t.inv_r[i];
    T* B = sB + bb * kConsScalars;
    B[0] = -sgn * ir;                 // factor of the streaming terms
    B[1] = t.cot_th[j];
    if (collision) {
      const T ks = (T)p.kaps[blk];
      B[2] = (T)p.kap[blk] + ks;                                    // loss rate
      B[3] = (T)p.eta[blk] * t.sin_th[j] / (ir * ir) + ks * sJ[bb];  // eta r^2 sin th + ks J
      B[4] = (aniso && p.scb) ? ks * (T)p.scb[blk] : (T)0;
      B[5] = quad ? ks * (T)p.scc[blk] : (T)0;
    } else {
      B[2] = B[3] = B[4] = B[5] = 0;
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nbb * Hh; x += blockDim.x) {
    const int bb = x / Hh, r = x - bb * Hh, k = r / hP, c = r - k * hP;
    const int k2 = NT - 1 - k;
    const T* es = ses + (size_t)bb * Hh;
    const T* os = sos + (size_t)bb * Hh;
    const T* ed = sed + (size_t)bb * Hh;
    const T* od = sod + (size_t)bb * Hh;
    T A1 = 0, A2 = 0, B1 = 0, B2 = 0;
    for (int kk = 0; kk < h; ++kk) {
      const int w = kk * hP + c, e = kk * h + k;
      A1 = fma(sPe[e], es[w], A1);
      A2 = fma(sPo[e], os[w], A2);
      B1 = fma(sQe[e], ed[w], B1);
      B2 = fma(sQo[e], od[w], B2);
    }
    const T* s1 = ss + (size_t)bb * H + k * hP;
    const T* d1 = sd + (size_t)bb * H + k * hP;
    const T* s2 = ss + (size_t)bb * H + k2 * hP;
    const T* d2 = sd + (size_t)bb * H + k2 * hP;
    T M1 = 0, N1 = 0, M2 = 0, N2 = 0;
    for (int q = 0; q < hP; ++q) {
      const T ms = sMs[q * hP + c], md = sMd[q * hP + c];
      M1 = fma(ms, d1[q], M1);
      N1 = fma(md, s1[q], N1);
      M2 = fma(ms, d2[q], M2);
      N2 = fma(md, s2[q], N2);
    }
    const T* B = sB + bb * kConsScalars;
    const T A = B[0], cot = B[1], kl = B[2], eg0 = B[3], kb = B[4], kc = B[5];
    const T ny = sc[bb * hP + c];
    const long long blk = b0 + bb;
    T* Kb = K + blk * S;
    const T* ub = su + (size_t)bb * S;
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const int kr = row ? k2 : k;
      const T Ps = row ? A2 - A1 : A1 + A2, Qd = row ? B2 - B1 : B1 + B2;
      const T Ms = row ? M2 : M1, Md = row ? N2 : N1;
      const T sT = t.sinT[kr], cT = t.cosT[kr];
      const T nyk = (kr & 1) ? -ny : ny;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int m = c + half * hP;
        const T dT = half ? Ps - Qd : Ps + Qd;
        const T dP = half ? Ms - Md : Ms + Md;
        const T u = ub[kr * NP + m];
        T tt = fma(cot, dP, dT);
        tt = fma(cT, u - nyk, sT * tt);
        T v = A * tt;
        if (collision) {
          T eg = eg0;
          if (aniso) {
            const T* M = sJ + bb;
            const T cp = t.cosP[m], sp = t.sinP[m];
            eg += kb * (cT * M[nb] + sT * (cp * M[2 * nb] + sp * M[3 * nb]));
            if (quad) {
              const T j3 = M[0] * (T)(1.0 / 3.0);
              eg += kc * (cT * cT * (M[4 * nb] - j3) +
                          sT * sT * (cp * cp * (M[5 * nb] - j3) + sp * sp * (M[6 * nb] - j3) +
                                     (T)2 * cp * sp * M[7 * nb]) +
                          (T)2 * cT * sT * (cp * M[8 * nb] + sp * M[9 * nb]));
            }
          }
          v = fma(sT, eg, fma(-kl, u, v));
        }
        Kb[kr * NP + m] = v;
      }
    }
  }
}

// Per angular block (one warp each): the block's shares of N, dN/dt, J_R1, J_R2
// and S. w = [wr (Nr) | wt (Nt) | wT (NT)]: the radial, theta and Theta weights
// of the state's number integral; cons: the source carries r^2 sin th sin Th.
template <typename T>
__global__ void __launch_bounds__(256)
k_balance_blocks(Dims d, Tables<double> t, const double* __restrict__ kap,
                 const double* __restrict__ eta, const double* __restrict__ w, int cons,
                 double rho1, double rho2, const T* __restrict__ F, const T* __restrict__ K,
                 double* __restrict__ part) {
  const int NT = d.NT, NP = d.NP, S = NT * NP;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const double* wr = w;
  const double* wt = w + d.Nr;
  const double* wT = wt + d.Nt;
  const double dA = (2.0 * M_PI / d.Np) * (2.0 * M_PI / NP);
  for (long long blk = warp; blk < d.nblk; blk += nw) {
    const int j = (int)((blk / d.Np) % d.Nt);
    const int i = (int)((blk / ((long long)d.Np * d.Nt)) % d.Nr);
    const double ka = kap[blk], et = eta[blk];
    const double r2s = t.sin_th[j] / (t.inv_r[i] * t.inv_r[i]);
    double aN = 0.0, aK = 0.0, aJ = 0.0, aS = 0.0;
    for (int x = lane; x < S; x += 32) {
      const int k = x / NP;
      const double f = (double)F[blk * S + x], q = wT[k];
      aN = fma(q, f, aN);
      aK = fma(q, (double)K[blk * S + x], aK);
      aJ = fma(q * t.cosT[k], f, aJ);
      aS = fma(q, (cons ? et * r2s * t.sinT[k] : et) - ka * f, aS);
    }
    for (int o = 16; o; o >>= 1) {
      aN += __shfl_xor_sync(0xffffffffu, aN, o);
      aK += __shfl_xor_sync(0xffffffffu, aK, o);
      aJ += __shfl_xor_sync(0xffffffffu, aJ, o);
      aS += __shfl_xor_sync(0xffffffffu, aS, o);
    }
    if (lane == 0) {
      const double ws = wt[j] * dA;
      double* o = part + blk * 5;
      o[0] = wr[i] * ws * aN;
      o[1] = i == 0 ? rho1 * ws * aJ : 0.0;
      o[2] = i == d.Nr - 1 ? rho2 * ws * aJ : 0.0;
      o[3] = wr[i] * ws * aK;
      o[4] = wr[i] * ws * aS;
    }
  }
}

// One CTA per group: the group's block shares summed in a fixed order.
__global__ void __launch_bounds__(256)
k_balance_groups(const double* __restrict__ part, long long per, double* __restrict__ out) {
  __shared__ double red[5][256];
  const int g = blockIdx.x;
  double a[5] = {0, 0, 0, 0, 0};
  for (long long b = threadIdx.x; b < per; b += blockDim.x)
    for (int c = 0; c < 5; ++c) a[c] += part[((long long)g * per + b) * 5 + c];
  for (int c = 0; c < 5; ++c) red[c][threadIdx.x] = a[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int c = 0; c < 5; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[g * 5 + threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

template <typename T>
cudaError_t launch_angular_cons(const Problem& p, const Tables<T>& t, const T* U, T* K, T sgn,
                                bool collision, cudaStream_t s) {
  const ConsTile c = cons_tile(p.d, sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(k_angular_cons<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.bytes);
  if (e != cudaSuccess) return e;
  const long long nct = (p.d.nblk + c.nb - 1) / c.nb;
  k_angular_cons<T><<<(unsigned)nct, kConsThreads, c.bytes, s>>>(p, t, U, K, sgn,
                                                                 collision ? 1 : 0, c.nb);
  return cudaGetLastError();
}

template cudaError_t launch_angular_cons<double>(const Problem&, const Tables<double>&,
                                                 const double*, double*, double, bool,
                                                 cudaStream_t);
template cudaError_t launch_angular_cons<float>(const Problem&, const Tables<float>&,
                                                const float*, float*, float, bool, cudaStream_t);

template <typename T>
cudaError_t launch_number_balance(const Problem& p, const Tables<double>& t, const double* w,
                                  int cons, double rho1, double rho2, const T* F, const T* K,
                                  double* part, double* out, cudaStream_t s) {
  const long long warps = std::min<long long>(p.d.nblk, 152LL * 64);
  k_balance_blocks<T><<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(p.d, t, p.kap, p.eta, w, cons,
                                                                   rho1, rho2, F, K, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_balance_groups<<<p.d.G, 256, 0, s>>>(part, p.d.nblk / p.d.G, out);
  return cudaGetLastError();
}

template cudaError_t launch_number_balance<double>(const Problem&, const Tables<double>&,
                                                   const double*, int, double, double,
                                                   const double*, const double*, double*,
                                                   double*, cudaStream_t);
template cudaError_t launch_number_balance<float>(const Problem&, const Tables<double>&,
                                                  const double*, int, double, double,
                                                  const float*, const float*, double*, double*,
                                                  cudaStream_t);

}  // namespace ts
