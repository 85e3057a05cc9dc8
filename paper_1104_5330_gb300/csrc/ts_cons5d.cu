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
// half the multiply-adds of the dense products. The Nyquist bin of the doubled
// circle (2 NT nodes, the reflected node 2NT-1-j carrying -Fhat(j, m+h)) is
//   c(m) = (1/2NT) sum_j (-1)^j (Fhat(j, m) + Fhat(j, m+h)),
//   P Fhat (k, m) = Fhat(k, m) - (-1)^k c(m),   c(m + h) = c(m).
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

// Shared layout (doubles): P, Q [NT][NT] | Ms, Md [hP][hP] | per block: the
// field [S], the pair sums and differences s, d [NT][hP] each, sig, del
// [NT][hP] each, the Nyquist bins [hP] and the ten moments.
size_t cons_table_doubles(const Dims& d) {
  const size_t hP = d.NP / 2;
  return 2 * (size_t)d.NT * d.NT + 2 * hP * hP;
}
size_t cons_block_doubles(const Dims& d) {
  const size_t S = (size_t)d.NT * d.NP;
  return 3 * S + d.NP / 2 + 10;
}

ConsTile cons_tile(const Dims& d) {
  const size_t tab = cons_table_doubles(d) * 8, blk = cons_block_doubles(d) * 8;
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

__global__ void __launch_bounds__(kConsThreads)
k_angular_cons(Problem p, Tables<double> t, const double* __restrict__ U,
               double* __restrict__ K, double sgn, int collision, int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims d = p.d;
  const int NT = d.NT, NP = d.NP, S = NT * NP, hP = NP / 2, H = NT * hP;
  double* sP = reinterpret_cast<double*>(smem_raw);   // [k'][k]
  double* sQ = sP + NT * NT;
  double* sMs = sQ + NT * NT;                         // [q][p]
  double* sMd = sMs + hP * hP;
  double* su = sMd + hP * hP;                         // [nb][S]
  double* ss = su + (size_t)nb * S;                   // [nb][NT][hP]
  double* sd = ss + (size_t)nb * H;
  double* sg = sd + (size_t)nb * H;                   // sig [nb][NT][hP]
  double* sl = sg + (size_t)nb * H;                   // del
  double* sc = sl + (size_t)nb * H;                   // Nyquist bins [nb][hP]
  double* sJ = sc + (size_t)nb * hP;                  // moments [10][nb]
  const long long b0 = (long long)blockIdx.x * nb;
  const int nbb = (int)min((long long)nb, d.nblk - b0);
  const int kf = kernel_form(p, collision);
  const bool aniso = kf >= KF_LINEAR, quad = kf >= KF_QUADRATIC;

  for (int x = threadIdx.x; x < NT * NT; x += blockDim.x) {
    sP[x] = t.PThT[x];
    sQ[x] = t.QThT[x];
  }
  for (int x = threadIdx.x; x < hP * hP; x += blockDim.x) {
    sMs[x] = t.MsPhT[x];
    sMd[x] = t.MdPhT[x];
  }
  {
    const double2* src = reinterpret_cast<const double2*>(U + b0 * S);
    double2* dst = reinterpret_cast<double2*>(su);
    for (int x = threadIdx.x; x < nbb * S / 2; x += blockDim.x) dst[x] = src[x];
  }
  __syncthreads();
  // pair sums and differences of Fhat and of sin Ph Fhat
  for (int x = threadIdx.x; x < nbb * H; x += blockDim.x) {
    const int bb = x / H, r = x - bb * H, k = r / hP, q = r - k * hP;
    const double a = su[bb * S + k * NP + q], b = su[bb * S + k * NP + q + hP];
    ss[x] = a + b;
    sd[x] = a - b;
    const double va = t.sinP[q] * a, vb = t.sinP[q + hP] * b;
    sg[x] = va + vb;
    sl[x] = va - vb;
  }
  __syncthreads();
  // Nyquist bins of the doubled Theta circle
  for (int x = threadIdx.x; x < nbb * hP; x += blockDim.x) {
    const int bb = x / hP, q = x - bb * hP;
    double c = 0.0;
    for (int j = 0; j < NT; ++j) {
      const double v = ss[(size_t)bb * H + j * hP + q];
      c += (j & 1) ? -v : v;
    }
    sc[x] = c / (2.0 * NT);
  }
  if (collision) {
    // moments of G = Fhat / sin Th, one warp per block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bb = warp; bb < nbb; bb += blockDim.x >> 5) {
      double mo[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // J, H (3), M (6)
      for (int x = lane; x < S; x += 32) {
        const int k = x / NP, m = x - k * NP;
        const double qu = t.qdir[k] * su[bb * S + x] / t.sinT[k];
        mo[0] += qu;
        if (aniso) {
          const double qs = t.sinT[k] * qu, ct = t.cosT[k];
          const double cp = t.cosP[m], sp = t.sinP[m];
          mo[1] = fma(ct, qu, mo[1]);
          mo[2] = fma(cp, qs, mo[2]);
          mo[3] = fma(sp, qs, mo[3]);
          if (quad) {
            const double qss = t.sinT[k] * qs;
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
  // one thread per output pair (k, c), (k, c + hP)
  for (int x = threadIdx.x; x < nbb * H; x += blockDim.x) {
    const int bb = x / H, r = x - bb * H, k = r / hP, c = r - k * hP;
    const double* bs = ss + (size_t)bb * H;
    const double* bd = sd + (size_t)bb * H;
    double Ps = 0.0, Qd = 0.0;
    for (int kk = 0; kk < NT; ++kk) {
      Ps = fma(sP[kk * NT + k], bs[kk * hP + c], Ps);
      Qd = fma(sQ[kk * NT + k], bd[kk * hP + c], Qd);
    }
    const double* bg = sg + (size_t)bb * H + k * hP;
    const double* bl = sl + (size_t)bb * H + k * hP;
    double Ms = 0.0, Md = 0.0;
    for (int q = 0; q < hP; ++q) {
      Ms = fma(sMs[q * hP + c], bg[q], Ms);
      Md = fma(sMd[q * hP + c], bl[q], Md);
    }
    const long long blk = b0 + bb;
    int g, i, j, l;
    {
      l = (int)(blk % d.Np);
      long long qq = blk / d.Np;
      j = (int)(qq % d.Nt);
      qq /= d.Nt;
      i = (int)(qq % d.Nr);
      g = (int)(qq / d.Nr);
      (void)g;
      (void)l;
    }
    const double ir = t.inv_r[i], sT = t.sinT[k], cT = t.cosT[k];
    const double ny = (k & 1) ? -sc[bb * hP + c] : sc[bb * hP + c];
    const double aP = -sT * t.cot_th[j] * ir;
    double kap = 0.0, eta = 0.0, ks = 0.0, kb = 0.0, kc = 0.0, jac = 0.0;
    if (collision) {
      kap = p.kap[blk];
      eta = p.eta[blk];
      ks = p.kaps[blk];
      if (aniso && p.scb) kb = ks * p.scb[blk];
      if (quad) kc = ks * p.scc[blk];
      jac = sT * t.sin_th[j] / (ir * ir);
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int m = c + half * hP;
      const double dT = half ? Ps - Qd : Ps + Qd;
      const double dP = 0.5 * (half ? Ms - Md : Ms + Md);
      const double u = su[bb * S + k * NP + m];
      double v = sgn * (-ir * (sT * dT + cT * (u - ny)) + aP * dP);
      if (collision) {
        const double* M = sJ + bb;
        double gain = ks * M[0];
        const double cp = t.cosP[m], sp = t.sinP[m];
        if (aniso && p.scb) gain += kb * (cT * M[nb] + sT * (cp * M[2 * nb] + sp * M[3 * nb]));
        if (quad) {
          const double j3 = M[0] / 3.0;
          gain += kc * (cT * cT * (M[4 * nb] - j3) +
                        sT * sT * (cp * cp * (M[5 * nb] - j3) + sp * sp * (M[6 * nb] - j3) +
                                   2.0 * cp * sp * M[7 * nb]) +
                        2.0 * cT * sT * (cp * M[8 * nb] + sp * M[9 * nb]));
        }
        v += jac * eta - (kap + ks) * u + sT * gain;
      }
      K[blk * S + k * NP + m] = v;
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

size_t angular_cons_smem(const Dims& d) { return cons_tile(d).bytes; }

cudaError_t launch_angular_cons(const Problem& p, const Tables<double>& t, const double* U,
                                double* K, double sgn, bool collision, cudaStream_t s) {
  const ConsTile c = cons_tile(p.d);
  cudaError_t e = cudaFuncSetAttribute(k_angular_cons, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)c.bytes);
  if (e != cudaSuccess) return e;
  const long long nct = (p.d.nblk + c.nb - 1) / c.nb;
  k_angular_cons<<<(unsigned)nct, kConsThreads, c.bytes, s>>>(p, t, U, K, sgn, collision ? 1 : 0,
                                                              c.nb);
  return cudaGetLastError();
}

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
