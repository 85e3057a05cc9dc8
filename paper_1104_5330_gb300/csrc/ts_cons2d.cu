// The conservative 2-D (r, Theta) formulation of App. B on the GPU.
//
// Spherically symmetric radiation F(r, Theta) written for the conservative
// variable Fhat = r^2 sin(Theta) F (App. B, Eq. flux):
//   dFhat/dt = - cos Th dFhat/dr + (1/r) (sin Th dFhat/dTh + cos Th P Fhat)
//              + kappa_s [ - Fhat + sin Th int_0^pi k_c(Th, Th') Fhat(Th') dTh' ]   (Eq. speccons)
//   k_c(Th, Th') = (1/2) (1 + c (cos^2 Th cos^2 Th' + (1/2) sin^2 Th sin^2 Th' - 1/3)),
// the Phi'-average of the kernel (1/4pi)(1 + c (mu^2 - 1/3)) (c = 3/4: the
// Thomson form printed in Eq. speccons). r: Chebyshev-Gauss-Lobatto
// differentiation; Theta: pole-free nodes, Fhat odd on the doubled circle
// (its reflected node carries -Fhat), Fourier derivative with the Nyquist mode
// zeroed; P removes the Nyquist sine mode of Fhat, the alternating pattern
// (-1)^k on the nodes, so that the Theta term integrates to zero exactly; the
// Theta' integral by Fejer's first rule on Fhat / sin Th'. Tau inflow rows (the
// rate at each direction's inflow node is zero) and classical RK4.
//
// One CTA per problem keeps its whole (r, Theta) tile, the stage input, the
// stage derivative and the RK4 accumulator in shared memory and runs every
// step of the call there: no global traffic between stages or steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ts_internal.h"

namespace {

constexpr int kC2Threads = 256;

struct C2Tables {
  const double* Dr;    // [Nr][Nr] d/dr, [out][in] (three-zone grid: directions with cos Th > 0)
  const double* Dr2;   // three-zone grid: d/dr of the directions with cos Th < 0
  const double* Dt;    // [NT][NT] d/dTh of odd functions on the doubled circle, [out][in]
  const double* cT;    // cos Th_k
  const double* sT;    // sin Th_k
  const double* q;     // Fejer_k / sin Th_k: int_0^pi h dTh for odd h
  const double* ir;    // 1 / r_i
  const double* ts;    // T_N(x_i) = +-1
  const double* wr;    // int dr weights (Clenshaw-Curtis)
};

struct C2Problem {
  int Nr, NT, P;
  double c;            // kernel parameter
  int tau;             // Tau inflow rows (three-zone grid: held outer inflow nodes)
  int zoned;           // three-zone radial grid: Dr / Dr2 by direction
  const double* ks;    // [P][Nr] kappa_s
  const double* g1;    // [P][NT/2] inflow Fhat at R1 (cos Th > 0)
  const double* g2;    // [P][NT/2] inflow Fhat at R2 (cos Th < 0)
};

// Shared layout (doubles): Dr | Dt | cT sT q ir ts wr | ks | F U K Acc | row sums 4 Nr | kb NT
// | Dr2 (three-zone grid)
__host__ __device__ inline size_t c2_smem(int Nr, int NT, bool zoned = false) {
  const size_t n = (size_t)Nr * NT;
  return ((size_t)Nr * Nr + (size_t)NT * NT + 3 * (size_t)NT + 4 * (size_t)Nr + 4 * n +
          4 * (size_t)Nr + 2 * (size_t)NT + 4 + (zoned ? (size_t)Nr * Nr : 0)) *
         sizeof(double);
}

// K = rhs(U) for one problem, all in shared memory; tau: Tau rows.
__device__ void c2_rhs(const C2Problem& z, const double* Dr, const double* Dr2, const double* Dt,
                       const double* cT, const double* sT, const double* q, const double* ir,
                       const double* ts, const double* ks, const double* U, double* K,
                       double* rows, double* kb, bool tau) {
  const int Nr = z.Nr, NT = z.NT, n = Nr * NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* nyq = rows;            // Nyquist coefficient of each row
  double* S0 = rows + Nr;        // int Fhat' dTh'
  double* Scc = rows + 2 * Nr;   // int cos^2 Th' Fhat' dTh'
  double* Sss = rows + 3 * Nr;   // int sin^2 Th' Fhat' dTh'
  for (int i = warp; i < Nr; i += nw) {
    double a = 0, s0 = 0, sc = 0, ss = 0;
    for (int k = lane; k < NT; k += 32) {
      const double u = U[i * NT + k], qu = q[k] * u;
      a += (k & 1) ? -u : u;
      s0 += qu;
      sc = fma(cT[k] * cT[k], qu, sc);
      ss = fma(sT[k] * sT[k], qu, ss);
    }
    for (int o = 16; o; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      sc += __shfl_xor_sync(0xffffffffu, sc, o);
      ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    if (lane == 0) {
      nyq[i] = a / NT;
      S0[i] = s0;
      Scc[i] = sc;
      Sss[i] = ss;
    }
  }
  __syncthreads();
  const double c = z.c;
  for (int x = threadIdx.x; x < n; x += blockDim.x) {
    const int i = x / NT, k = x - i * NT;
    double dr = 0, dt = 0;
    const double* D = (z.zoned && !(cT[k] > 0)) ? Dr2 : Dr;   // three-zone grid: by direction
    for (int ii = 0; ii < Nr; ++ii) dr = fma(D[i * Nr + ii], U[ii * NT + k], dr);
    for (int kk = 0; kk < NT; ++kk) dt = fma(Dt[k * NT + kk], U[i * NT + kk], dt);
    const double u = U[x];
    const double pu = u - ((k & 1) ? -nyq[i] : nyq[i]);
    const double ct = cT[k], st = sT[k];
    const double stream = -ct * dr + (st * dt + ct * pu) * ir[i];
    const double gain =
        st * 0.5 * (S0[i] + c * (ct * ct * Scc[i] + 0.5 * st * st * Sss[i] - S0[i] / 3.0));
    K[x] = stream + ks[i] * (gain - u);
  }
  __syncthreads();
  if (tau && z.zoned) {   // three-zone grid: each direction's outer inflow node holds its data
    for (int k = threadIdx.x; k < NT; k += blockDim.x) K[(cT[k] > 0 ? 0 : Nr - 1) * NT + k] = 0.0;
    __syncthreads();
  } else if (tau) {
    for (int k = threadIdx.x; k < NT; k += blockDim.x) {
      const int b = cT[k] > 0 ? 0 : Nr - 1;
      kb[k] = -K[b * NT + k] * ts[b];   // alpha = (0 - K(r_b)) / T_N(x_b), T_N(x_b) = +-1
    }
    __syncthreads();
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
      const int i = x / NT, k = x - i * NT;
      K[x] += kb[k] * ts[i];
    }
    __syncthreads();
  }
}

// mode 0: nsteps RK4 steps of Fhat in place; 1: K = rhs(Fhat); 2: balance
// (out[3 p .. 3 p + 3] = N, J_R1, J_R2 and out2[p] = dN/dt + J_R2 - J_R1 of the
// operator without boundary rows).
__global__ void __launch_bounds__(kC2Threads)
k_cons2d(C2Problem z, C2Tables t, double* Fh, double* Kout, double* out, double* out2,
         double dt, int nsteps, int mode) {
  extern __shared__ __align__(16) double sm[];
  const int Nr = z.Nr, NT = z.NT, n = Nr * NT;
  const int p = blockIdx.x;
  double* Dr = sm;
  double* Dt = Dr + Nr * Nr;
  double* cT = Dt + NT * NT;
  double* sT = cT + NT;
  double* q = sT + NT;
  double* ir = q + NT;
  double* ts = ir + Nr;
  double* wr = ts + Nr;
  double* ks = wr + Nr;
  double* F = ks + Nr;
  double* U = F + n;
  double* K = U + n;
  double* Acc = K + n;
  double* rows = Acc + n;
  double* kb = rows + 4 * Nr;
  double* Dr2 = kb + NT + 4;
  for (int x = threadIdx.x; x < Nr * Nr; x += blockDim.x) Dr[x] = t.Dr[x];
  if (z.zoned)
    for (int x = threadIdx.x; x < Nr * Nr; x += blockDim.x) Dr2[x] = t.Dr2[x];
  for (int x = threadIdx.x; x < NT * NT; x += blockDim.x) Dt[x] = t.Dt[x];
  for (int x = threadIdx.x; x < NT; x += blockDim.x) {
    cT[x] = t.cT[x];
    sT[x] = t.sT[x];
    q[x] = t.q[x];
  }
  for (int x = threadIdx.x; x < Nr; x += blockDim.x) {
    ir[x] = t.ir[x];
    ts[x] = t.ts[x];
    wr[x] = t.wr[x];
    ks[x] = z.ks[(long long)p * Nr + x];
  }
  double* Fg = Fh + (long long)p * n;
  for (int x = threadIdx.x; x < n; x += blockDim.x) F[x] = Fg[x];
  __syncthreads();
  const bool tau = z.tau != 0;
  if (mode == 1) {
    c2_rhs(z, Dr, Dr2, Dt, cT, sT, q, ir, ts, ks, F, K, rows, kb, tau);
    for (int x = threadIdx.x; x < n; x += blockDim.x) Kout[(long long)p * n + x] = K[x];
    return;
  }
  if (mode == 2) {
    c2_rhs(z, Dr, Dr2, Dt, cT, sT, q, ir, ts, ks, F, K, rows, kb, false);
    // per row: int dTh of K and of Fhat (warp sums), then fixed-order sums over r
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < Nr; i += nw) {
      double a = 0, b = 0;
      for (int k = lane; k < NT; k += 32) {
        a = fma(q[k], K[i * NT + k], a);
        b = fma(q[k], F[i * NT + k], b);
      }
      for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        rows[i] = a;
        rows[Nr + i] = b;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double w = 8.0 * M_PI * M_PI;
      double dN = 0, N = 0, J1 = 0, J2 = 0;
      for (int i = 0; i < Nr; ++i) {
        dN = fma(wr[i], rows[i], dN);
        N = fma(wr[i], rows[Nr + i], N);
      }
      for (int k = 0; k < NT; ++k) {
        J1 = fma(q[k] * cT[k], F[k], J1);
        J2 = fma(q[k] * cT[k], F[(Nr - 1) * NT + k], J2);
      }
      out[3 * p] = w * N;
      out[3 * p + 1] = w * J1;
      out[3 * p + 2] = w * J2;
      out2[p] = w * dN + w * J2 - w * J1;
    }
    return;
  }
  for (int step = 0; step < nsteps; ++step) {
    for (int s = 0; s < 4; ++s) {
      c2_rhs(z, Dr, Dr2, Dt, cT, sT, q, ir, ts, ks, s == 0 ? F : U, K, rows, kb, tau);
      for (int x = threadIdx.x; x < n; x += blockDim.x) {
        const double k = K[x];
        if (s == 0) {
          Acc[x] = k;
          U[x] = F[x] + 0.5 * dt * k;
        } else if (s < 3) {
          Acc[x] += 2.0 * k;
          U[x] = F[x] + (s == 1 ? 0.5 * dt : dt) * k;
        } else {
          F[x] += dt / 6.0 * (Acc[x] + k);
        }
      }
      __syncthreads();
    }
  }
  for (int x = threadIdx.x; x < n; x += blockDim.x) Fg[x] = F[x];
}

// F = inflow data at the inflow nodes (r = R1 with cos Th > 0, r = R2 otherwise).
__global__ void k_cons2d_inflow(C2Problem z, double* Fh) {
  const int NT = z.NT, h = NT / 2;
  const long long n = (long long)z.P * NT;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n;
       x += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(x / NT), k = (int)(x - (long long)p * NT);
    double* F = Fh + (long long)p * z.Nr * NT;
    if (k < h) F[k] = z.g1 ? z.g1[(long long)p * h + k] : 0.0;
    else F[(z.Nr - 1) * NT + k] = z.g2 ? z.g2[(long long)p * h + (k - h)] : 0.0;
  }
}

}  // namespace

struct ts_cons2d {
  ts_cons2d_desc desc;
  std::vector<double> r, Theta;
  double* tab = nullptr;        // device tables
  C2Tables t{};
  double *ks = nullptr, *g1 = nullptr, *g2 = nullptr;
  bool coeffs = false;
};

extern "C" {

ts_status ts_cons2d_create(const ts_cons2d_desc* desc, ts_cons2d** out) {
  if (!out) return ts::fail_status(TS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!desc) return ts::fail_status(TS_ERR_ARG, "desc is NULL");
  const ts_cons2d_desc& d = *desc;
  if (!(d.R1 > 0.0) || !(d.R2 > d.R1) || !std::isfinite(d.R2) || d.problems < 1 ||
      !std::isfinite(d.scatter_c))
    return ts::fail_status(TS_ERR_ARG, "need 0 < R1 < R2, problems >= 1, finite c");
  if (d.Nr < 3 || d.Nr > 129 || d.NTheta < 2 || d.NTheta > 64 || (d.NTheta % 2))
    return ts::fail_status(TS_ERR_UNSUPPORTED, "sizes: need 3 <= Nr <= 129, even 2 <= NTheta <= 64");
  if (d.bc != TS_BC_TAU_INFLOW && d.bc != TS_BC_NONE)
    return ts::fail_status(TS_ERR_UNSUPPORTED, "unknown bc");
  if (d.radial != TS_RADIAL_CHEBYSHEV && d.radial != TS_RADIAL_ZONED)
    return ts::fail_status(TS_ERR_UNSUPPORTED, "radial: TS_RADIAL_CHEBYSHEV or TS_RADIAL_ZONED");
  const bool zoned = d.radial == TS_RADIAL_ZONED;
  if (zoned && (d.zone_nodes < 2 || d.Nr - 2 * (d.zone_nodes - 1) < 3 || !(d.zone_width > 0.0) ||
                !(d.zone_width < 0.5)))
    return ts::fail_status(TS_ERR_UNSUPPORTED,
                           "zoned radial grid: need zone_nodes >= 2, Nr - 2 (zone_nodes - 1) >= 3, "
                           "0 < zone_width < 1/2");
  if (c2_smem(d.Nr, d.NTheta, zoned) > 227 * 1024)
    return ts::fail_status(TS_ERR_UNSUPPORTED, "tile too large for one CTA's shared memory");
  const int Nr = d.Nr, NT = d.NTheta, N = Nr - 1;
  ts_cons2d* G = new ts_cons2d();
  G->desc = d;
  // three-zone grid (App. B): nA uniform nodes per edge zone of width w, the nB
  // Gauss-Lobatto nodes of [R1 + w, R2 - w] between them (shared interfaces)
  const int nA = zoned ? d.zone_nodes : 0, nB = zoned ? Nr - 2 * (nA - 1) : 0;
  const double zw = zoned ? d.zone_width * (d.R2 - d.R1) : 0.0, zh = zoned ? zw / (nA - 1) : 0.0;
  const int iB0 = nA - 1, iB1 = nA - 1 + nB - 1;
  for (int i = 0; i < Nr; ++i) {
    if (!zoned) {
      G->r.push_back(0.5 * (d.R1 + d.R2) - 0.5 * (d.R2 - d.R1) * std::cos(M_PI * i / N));
    } else {
      const double a = d.R1 + zw, b = d.R2 - zw;
      if (i < nA) G->r.push_back(d.R1 + zh * i);
      else if (i < iB1) G->r.push_back(0.5 * (a + b) - 0.5 * (b - a) * std::cos(M_PI * (i - iB0) / (nB - 1)));
      else G->r.push_back(b + zh * (i - iB1));
    }
  }
  for (int k = 0; k < NT; ++k) G->Theta.push_back(M_PI * (k + 0.5) / NT);
  // tables: d/dr; d/dTh of odd functions on the doubled circle (A - B of its
  // Fourier derivative, node 2NT-1-k' carrying -Fhat(k')); Fejer / sin Th;
  // 1/r; T_N(x_i); Clenshaw-Curtis x (R2-R1)/2
  std::vector<double> Dr = zoned ? std::vector<double>((size_t)Nr * Nr, 0.0)
                                 : ts::cheb_diff_matrix(Nr, d.R1, d.R2);
  std::vector<double> Dr2 = Dr;
  if (zoned) {
    // the zoned derivative of each direction class as a matrix ([out][in]):
    // upwind differences in the edge zones (none at the outer inflow node), the
    // central Chebyshev rows plus the interface Tau correction
    //   d(i) += T_N(x_i)/T_N(x_b) (dFD(b) - dB(b)),  b the inflow interface,
    // every row linear in the line's values
    const std::vector<double> DB = ts::cheb_diff_matrix(nB, d.R1 + zw, d.R2 - zw);
    auto tN = [&](int j) { return ((nB - 1 - j) % 2) ? -1.0 : 1.0; };
    for (int dir = 0; dir < 2; ++dir) {   // 0: cos Th > 0 (inflow at R1), 1: cos Th < 0
      std::vector<double>& Z = dir == 0 ? Dr : Dr2;
      const int b = dir == 0 ? 0 : nB - 1;          // central inflow interface
      // dFD(b) - dB(b) as a row over the line
      std::vector<double> c((size_t)Nr, 0.0);
      if (dir == 0) {
        c[iB0] += 1.0 / zh;
        c[iB0 - 1] -= 1.0 / zh;
      } else {
        c[iB1 + 1] += 1.0 / zh;
        c[iB1] -= 1.0 / zh;
      }
      for (int j = 0; j < nB; ++j) c[iB0 + j] -= DB[(size_t)b * nB + j];
      for (int i = 0; i < Nr; ++i) {
        double* row = &Z[(size_t)i * Nr];
        const bool central = dir == 0 ? (i > iB0 && i <= iB1) : (i >= iB0 && i < iB1);
        if (central) {
          const int ib = i - iB0;
          for (int j = 0; j < nB; ++j) row[iB0 + j] += DB[(size_t)ib * nB + j];
          const double s = tN(ib) / tN(b);
          for (int j = 0; j < Nr; ++j) row[j] += s * c[j];
        } else if (dir == 0 && i > 0) {
          row[i] += 1.0 / zh;
          row[i - 1] -= 1.0 / zh;
        } else if (dir == 1 && i < N) {
          row[i + 1] += 1.0 / zh;
          row[i] -= 1.0 / zh;
        }
      }
    }
  }
  const std::vector<double> Dc = ts::fourier_diff_matrix(2 * NT);
  std::vector<double> Dt((size_t)NT * NT);
  for (int k = 0; k < NT; ++k)
    for (int kk = 0; kk < NT; ++kk)
      Dt[(size_t)k * NT + kk] = Dc[(size_t)k * 2 * NT + kk] - Dc[(size_t)k * 2 * NT + (2 * NT - 1 - kk)];
  const std::vector<double> wF = ts::fejer_weights(NT);
  const std::vector<double> cc = ts::clenshaw_curtis_weights(Nr);
  std::vector<double> cT(NT), sT(NT), q(NT), ir(Nr), tsg(Nr), wr(Nr);
  for (int k = 0; k < NT; ++k) {
    cT[k] = std::cos(G->Theta[k]);
    sT[k] = std::sin(G->Theta[k]);
    q[k] = wF[k] / sT[k];
  }
  for (int i = 0; i < Nr; ++i) {
    ir[i] = 1.0 / G->r[i];
    tsg[i] = ((N - i) % 2) ? -1.0 : 1.0;
    wr[i] = cc[i] * 0.5 * (d.R2 - d.R1);
  }
  if (zoned) {   // trapezoid in the edge zones, Clenshaw-Curtis in the central one
    const std::vector<double> ccB = ts::clenshaw_curtis_weights(nB);
    std::fill(wr.begin(), wr.end(), 0.0);
    for (int i = 0; i < nA; ++i) {
      const double t = zh * ((i == 0 || i == nA - 1) ? 0.5 : 1.0);
      wr[i] += t;
      wr[iB1 + i] += t;
    }
    for (int j = 0; j < nB; ++j) wr[iB0 + j] += ccB[j] * 0.5 * (d.R2 - d.R1 - 2 * zw);
  }
  std::vector<const std::vector<double>*> parts = {&Dr, &Dr2, &Dt, &cT, &sT, &q, &ir, &tsg, &wr};
  size_t tot = 0;
  for (auto* v : parts) tot += v->size();
  std::vector<double> host;
  host.reserve(tot);
  for (auto* v : parts) host.insert(host.end(), v->begin(), v->end());
  cudaError_t e = cudaMalloc(&G->tab, tot * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(G->tab, host.data(), tot * sizeof(double), cudaMemcpyHostToDevice);
  const double* ptr = G->tab;
  const double** slots[] = {&G->t.Dr, &G->t.Dr2, &G->t.Dt, &G->t.cT, &G->t.sT,
                            &G->t.q,  &G->t.ir,  &G->t.ts, &G->t.wr};
  for (size_t a = 0; a < parts.size(); ++a) {
    *slots[a] = ptr;
    ptr += parts[a]->size();
  }
  const size_t nks = (size_t)d.problems * Nr * sizeof(double);
  const size_t ng = (size_t)d.problems * (NT / 2) * sizeof(double);
  if (e == cudaSuccess) e = cudaMalloc(&G->ks, nks);
  if (e == cudaSuccess) e = cudaMalloc(&G->g1, ng);
  if (e == cudaSuccess) e = cudaMalloc(&G->g2, ng);
  if (e == cudaSuccess) e = cudaMemset(G->ks, 0, nks);
  if (e == cudaSuccess) e = cudaMemset(G->g1, 0, ng);
  if (e == cudaSuccess) e = cudaMemset(G->g2, 0, ng);
  if (e != cudaSuccess) {
    ts_cons2d_destroy(G);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? ts::fail_status(TS_ERR_OOM, "device allocation failed")
                                          : ts::cuda_status(e, "ts_cons2d_create");
  }
  *out = G;
  return TS_OK;
}

ts_status ts_cons2d_destroy(ts_cons2d* g) {
  if (!g) return TS_OK;
  cudaDeviceSynchronize();
  for (void* p : {(void*)g->tab, (void*)g->ks, (void*)g->g1, (void*)g->g2})
    if (p) cudaFree(p);
  delete g;
  return TS_OK;
}

ts_status ts_cons2d_nodes(const ts_cons2d* g, double* r_host, double* Theta_host) {
  if (!g) return ts::fail_status(TS_ERR_ARG, "grid is NULL");
  if (r_host) std::memcpy(r_host, g->r.data(), g->r.size() * sizeof(double));
  if (Theta_host) std::memcpy(Theta_host, g->Theta.data(), g->Theta.size() * sizeof(double));
  return TS_OK;
}

ts_status ts_cons2d_set_coeffs(ts_cons2d* g, const double* kappa_s, const double* inflow_R1,
                               const double* inflow_R2, void* stream) {
  if (!g) return ts::fail_status(TS_ERR_ARG, "grid is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ts_cons2d_desc& d = g->desc;
  const size_t nks = (size_t)d.problems * d.Nr * sizeof(double);
  const size_t ng = (size_t)d.problems * (d.NTheta / 2) * sizeof(double);
  const void* src[] = {kappa_s, inflow_R1, inflow_R2};
  void* dst[] = {g->ks, g->g1, g->g2};
  const size_t nb[] = {nks, ng, ng};
  for (int a = 0; a < 3; ++a) {
    cudaError_t e = src[a] ? cudaMemcpyAsync(dst[a], src[a], nb[a], cudaMemcpyDeviceToDevice, st)
                           : cudaMemsetAsync(dst[a], 0, nb[a], st);
    if (e != cudaSuccess) return ts::cuda_status(e, "ts_cons2d_set_coeffs");
  }
  g->coeffs = true;
  return TS_OK;
}

static C2Problem c2_problem(const ts_cons2d* g) {
  C2Problem z;
  z.Nr = g->desc.Nr;
  z.NT = g->desc.NTheta;
  z.P = g->desc.problems;
  z.c = g->desc.scatter_c;
  z.tau = g->desc.bc == TS_BC_TAU_INFLOW ? 1 : 0;
  z.zoned = g->desc.radial == TS_RADIAL_ZONED ? 1 : 0;
  z.ks = g->ks;
  z.g1 = g->g1;
  z.g2 = g->g2;
  return z;
}

static ts_status c2_launch(ts_cons2d* g, double* Fh, double* K, double* out, double* out2,
                           double dt, int nsteps, int mode, void* stream, const char* where) {
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(k_cons2d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return ts::cuda_status(e, where);
    init = true;
  }
  const size_t smem = c2_smem(g->desc.Nr, g->desc.NTheta, g->desc.radial == TS_RADIAL_ZONED);
  k_cons2d<<<g->desc.problems, kC2Threads, smem, static_cast<cudaStream_t>(stream)>>>(
      c2_problem(g), g->t, Fh, K, out, out2, dt, nsteps, mode);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TS_OK : ts::cuda_status(e, where);
}

ts_status ts_cons2d_apply_inflow(ts_cons2d* g, double* Fhat, void* stream) {
  if (!g || !Fhat) return ts::fail_status(TS_ERR_ARG, "NULL argument");
  const long long n = (long long)g->desc.problems * g->desc.NTheta;
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 4096);
  k_cons2d_inflow<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(c2_problem(g), Fhat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TS_OK : ts::cuda_status(e, "ts_cons2d_apply_inflow");
}

ts_status ts_cons2d_rhs(ts_cons2d* g, const double* Fhat, double* K, void* stream) {
  if (!g || !Fhat || !K) return ts::fail_status(TS_ERR_ARG, "NULL argument");
  if (!g->coeffs) return ts::fail_status(TS_ERR_STATE, "ts_cons2d_set_coeffs has not been called");
  return c2_launch(g, const_cast<double*>(Fhat), K, nullptr, nullptr, 0.0, 0, 1, stream,
                   "ts_cons2d_rhs");
}

ts_status ts_cons2d_step(ts_cons2d* g, double* Fhat, double dt, int nsteps, void* stream) {
  if (!g || !Fhat) return ts::fail_status(TS_ERR_ARG, "NULL argument");
  if (!std::isfinite(dt) || nsteps < 0) return ts::fail_status(TS_ERR_ARG, "need finite dt, nsteps >= 0");
  if (!g->coeffs) return ts::fail_status(TS_ERR_STATE, "ts_cons2d_set_coeffs has not been called");
  if (nsteps == 0) return TS_OK;
  return c2_launch(g, Fhat, nullptr, nullptr, nullptr, dt, nsteps, 0, stream, "ts_cons2d_step");
}

ts_status ts_cons2d_balance(ts_cons2d* g, const double* Fhat, double* NJ, double* residual,
                            void* stream) {
  if (!g || !Fhat || !NJ || !residual) return ts::fail_status(TS_ERR_ARG, "NULL argument");
  if (!g->coeffs) return ts::fail_status(TS_ERR_STATE, "ts_cons2d_set_coeffs has not been called");
  return c2_launch(g, const_cast<double*>(Fhat), nullptr, NJ, residual, 0.0, 0, 2, stream,
                   "ts_cons2d_balance");
}

}  // extern "C"
