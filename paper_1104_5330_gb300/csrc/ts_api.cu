// Host side of the transport-step library: tables, grid lifecycle and the C ABI
// declared in include/ts.h.
//
// Tables are built here from closed forms, not from transforms:
//  * d/dr: the Chebyshev-Gauss-Lobatto differentiation matrix in barycentric
//    form, D_ij = (w_j/w_i)/(x_i - x_j), w_j = (-1)^j delta_j (delta = 1/2 at the
//    ends), diagonal = minus the row sum; scaled by 2/(R2-R1).
//  * Fourier derivative on M equispaced nodes of a 2 pi circle, Nyquist mode
//    zeroed: D_jk = (1/2)(-1)^(j-k) cot((j-k) pi/M), D_jj = 0. For theta and
//    Theta the circle is the doubled (double-Fourier-sphere) circle of 2N
//    nodes; node 2N-1-j carries F at the partner point, which splits the
//    matrix into A[j][j'] = D[j][j'] and B[j][j'] = D[j][2N-1-j'].
//  * Fejer's first rule on pi (k+1/2)/N and Clenshaw-Curtis weights on the
//    Gauss-Lobatto nodes from their cosine-sum closed forms.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ts_internal.h"

using ts::Dims;
using ts::Launch;
using ts::Tables;

namespace {

thread_local std::string g_err;

ts_status fail(ts_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

ts_status cuda_fail(cudaError_t e, const char* where) {
  return fail(TS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

using ts::Vec;
using ts::HostTables;

// ------------------------------------------------------------------ tables
Vec cheb_diff(int Nr, double R1, double R2) {
  const int N = Nr - 1;
  Vec x(Nr), w(Nr), D((size_t)Nr * Nr, 0.0);
  for (int i = 0; i < Nr; ++i) {
    x[i] = -std::cos(M_PI * i / N);
    w[i] = ((i % 2) ? -1.0 : 1.0) * ((i == 0 || i == N) ? 0.5 : 1.0);
  }
  for (int i = 0; i < Nr; ++i) {
    double diag = 0.0;
    for (int j = 0; j < Nr; ++j) {
      if (i == j) continue;
      // x_i - x_j = 2 sin(pi (i+j)/(2N)) sin(pi (i-j)/(2N)), accurate near the ends
      const double dx = 2.0 * std::sin(M_PI * (i + j) / (2.0 * N)) * std::sin(M_PI * (i - j) / (2.0 * N));
      const double v = (w[j] / w[i]) / dx;
      D[(size_t)i * Nr + j] = v;
      diag -= v;
    }
    D[(size_t)i * Nr + i] = diag;
  }
  const double s = 2.0 / (R2 - R1);
  for (double& v : D) v *= s;
  return D;
}

Vec fourier_diff(int M) {
  Vec D((size_t)M * M, 0.0);
  for (int j = 0; j < M; ++j)
    for (int k = 0; k < M; ++k) {
      if (j == k) continue;
      const int q = j - k;
      D[(size_t)j * M + k] = 0.5 * (((q % 2) + 2) % 2 ? -1.0 : 1.0) / std::tan(q * M_PI / M);
    }
  return D;
}

// Filter on M equispaced circle nodes: F_jk = (1/M) sum_q sigma(|q|) e^{i q (j-k) h}.
Vec fourier_filter(int M, double kmax, double alpha, int order) {
  Vec Fm((size_t)M * M);
  auto sig = [&](double q) { return std::exp(-alpha * std::pow(q / kmax, order)); };
  for (int j = 0; j < M; ++j)
    for (int k = 0; k < M; ++k) {
      const double a = 2.0 * M_PI * (j - k) / M;
      double s = sig(0.0);
      for (int q = 1; q < M / 2; ++q) s += 2.0 * sig(q) * std::cos(q * a);
      if (M % 2 == 0) s += sig(M / 2) * std::cos((M / 2) * a);
      else s += 2.0 * sig(M / 2) * std::cos((M / 2) * a);
      Fm[(size_t)j * M + k] = s / M;
    }
  return Fm;
}

// Filter in r: sum_k T_k(x_i) sigma(k/N) c_k with c_k the Chebyshev coefficients
// of the nodal values (discrete orthogonality on the Gauss-Lobatto nodes).
Vec cheb_filter(int Nr, double alpha, int order) {
  const int N = Nr - 1;
  Vec Fm((size_t)Nr * Nr, 0.0);
  for (int i = 0; i < Nr; ++i)
    for (int ip = 0; ip < Nr; ++ip) {
      double s = 0.0;
      const double cip = (ip == 0 || ip == N) ? 2.0 : 1.0;
      for (int k = 0; k <= N; ++k) {
        const double ck = (k == 0 || k == N) ? 2.0 : 1.0;
        const double Ti = std::cos(M_PI * k * (N - i) / N);
        const double Tip = std::cos(M_PI * k * (N - ip) / N);
        s += Ti * std::exp(-alpha * std::pow((double)k / N, order)) * 2.0 / (N * ck * cip) * Tip;
      }
      Fm[(size_t)i * Nr + ip] = s;
    }
  return Fm;
}

void dfs_split(const Vec& Dc, int N, Vec& A, Vec& B) {
  const int M = 2 * N;
  A.assign((size_t)N * N, 0.0);
  B.assign((size_t)N * N, 0.0);
  for (int j = 0; j < N; ++j)
    for (int jp = 0; jp < N; ++jp) {
      A[(size_t)j * N + jp] = Dc[(size_t)j * M + jp];
      B[(size_t)j * N + jp] = Dc[(size_t)j * M + (M - 1 - jp)];
    }
}

// Fejer's first rule for int_0^pi g(t) sin t dt on t_k = pi (k+1/2)/N.
Vec fejer(int N) {
  Vec w(N);
  for (int k = 0; k < N; ++k) {
    const double t = M_PI * (k + 0.5) / N;
    double s = 0.0;
    for (int m = 1; m <= N / 2; ++m) s += std::cos(2.0 * m * t) / (4.0 * m * m - 1.0);
    w[k] = 2.0 / N * (1.0 - 2.0 * s);
  }
  return w;
}

// Clenshaw-Curtis weights for int_{-1}^{1} on the Nr Gauss-Lobatto nodes.
Vec clenshaw_curtis(int Nr) {
  const int N = Nr - 1;
  Vec w(Nr);
  for (int i = 0; i <= N; ++i) {
    double s = 1.0;
    for (int k = 1; k <= N / 2; ++k) {
      const double b = (2 * k == N) ? 1.0 : 2.0;
      s -= b / (4.0 * k * k - 1.0) * std::cos(2.0 * k * i * M_PI / N);
    }
    w[i] = ((i == 0 || i == N) ? 1.0 : 2.0) / N * s;
  }
  return w;
}

Vec transpose(const Vec& M, int rows, int cols) {
  Vec T((size_t)rows * cols);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) T[(size_t)j * rows + i] = M[(size_t)i * cols + j];
  return T;
}


// Ordered list of the tables that go to the device (the order of Tables<C>).
std::vector<const Vec*> device_list(const HostTables& h, std::vector<Vec>& tmp) {
  const int Nr = (int)h.r.size(), Nt = (int)h.theta.size(), Np = (int)h.phi.size();
  const int NT = (int)h.Theta.size(), NP = (int)h.Phi.size();
  tmp.clear();
  tmp.reserve(14);
  tmp.push_back(transpose(h.Dr, Nr, Nr));
  tmp.push_back(transpose(h.Ath, Nt, Nt));
  tmp.push_back(transpose(h.Bth, Nt, Nt));
  tmp.push_back(transpose(h.Dph, Np, Np));
  tmp.push_back(transpose(h.ATh, NT, NT));
  tmp.push_back(transpose(h.BTh, NT, NT));
  tmp.push_back(transpose(h.DPh, NP, NP));
  tmp.push_back(transpose(h.Fr, Nr, Nr));
  tmp.push_back(transpose(h.FthA, Nt, Nt));
  tmp.push_back(transpose(h.FthB, Nt, Nt));
  tmp.push_back(transpose(h.Fph, Np, Np));
  tmp.push_back(transpose(h.FThA, NT, NT));
  tmp.push_back(transpose(h.FThB, NT, NT));
  tmp.push_back(transpose(h.FPh, NP, NP));
  return {&tmp[0], &tmp[1], &tmp[2], &tmp[3], &tmp[4], &tmp[5], &tmp[6],
          &h.Dr, &h.Ath, &h.Bth, &h.Dph, &h.ATh, &h.BTh, &h.DPh,
          &h.inv_r, &h.inv_sinth, &h.cot_th, &h.sin_th, &h.cos_th, &h.sin_ph, &h.cos_ph,
          &h.cosT, &h.sinT, &h.cosP, &h.sinP, &h.tsign, &h.qdir,
          &tmp[7], &tmp[8], &tmp[9], &tmp[10], &tmp[11], &tmp[12], &tmp[13],
          &h.PthT, &h.QthT, &h.PThT, &h.QThT, &h.EpT, &h.OpT, &h.DrMc, &h.DrMr,
          &h.TcBhi, &h.TcBlo,
          &h.PthA, &h.QthA, &h.PThA, &h.QThA, &h.EpTa, &h.OpTa, &h.DrMca, &h.DrMra,
          &h.MsPhT, &h.MdPhT, &h.MsphT, &h.MdphT,
          &h.PeThT, &h.PoThT, &h.QeThT, &h.QoThT, &h.PethT, &h.PothT, &h.QethT, &h.QothT,
          &h.PeThA, &h.PoThA, &h.QeThA, &h.QoThA, &h.PethA, &h.PothA, &h.QethA, &h.QothA,
          &h.MsPhA, &h.MdPhA, &h.MsphA, &h.MdphA};
}

// Even/odd forms of the derivative matrices (see Tables in ts_internal.h).
// DFS pair: for F at a node and G at its partner, A F + B G = P (F+G) + Q (F-G)
// and at the partner A G + B F = P (F+G) - Q (F-G), P = (A+B)/2, Q = (A-B)/2.
// TF32 rounding, to nearest with ties away from zero on the 13 dropped bits.
float tf32_round(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  float y;
  std::memcpy(&y, &b, 4);
  return y;
}

// D_r as the tensor cores' B operand: B[n = i][k = i'] = D_r[i][i'] split into
// TF32 hi + lo, zero-padded to (N_r up to 16) x (N_r up to 8), stored as 8-row
// x 4-column core matrices, core (n/8, k/4) at float offset ((n/8) KC + k/4) 32.
void tc_tables(HostTables& h) {
  const int Nr = (int)h.r.size(), Kpad = (Nr + 7) / 8 * 8, Npad = (Nr + 15) / 16 * 16;
  const int KC = Kpad / 4;
  h.TcBhi.assign((size_t)Npad * Kpad, 0.0);
  h.TcBlo.assign((size_t)Npad * Kpad, 0.0);
  for (int n = 0; n < Nr; ++n)
    for (int k = 0; k < Nr; ++k) {
      const double v = h.Dr[(size_t)n * Nr + k];
      const float hi = tf32_round((float)v);
      const float lo = tf32_round((float)(v - (double)hi));
      const size_t o = (size_t)((n / 8) * KC + k / 4) * 32 + (n % 8) * 4 + (k % 4);
      h.TcBhi[o] = hi;
      h.TcBlo[o] = lo;
    }
}

// bf16 rounding to nearest, ties to even (finite inputs).
uint16_t bf16_rne(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
float bf16_value(uint16_t h) {
  const uint32_t b = (uint32_t)h << 16;
  float y;
  std::memcpy(&y, &b, 4);
  return y;
}

// D_r as three bf16 terms (each the rounding of what the previous ones leave),
// the tensor cores' B operand of the BF16x3 radial pass: zero-padded to (N_r up
// to 16) x (N_r up to 16), 8-row x 8-element core matrices, core (n/8, k/8) at
// element offset ((n/8) KC + k/8) 64, KC = Kpad/8; the terms one after another.
std::vector<uint16_t> tc_tables_bf16(const HostTables& h) {
  const int Nr = (int)h.r.size(), Kpad = (Nr + 15) / 16 * 16, Npad = (Nr + 15) / 16 * 16;
  const int KC = Kpad / 8;
  const size_t T = (size_t)Npad * Kpad;
  std::vector<uint16_t> out(3 * T, 0);
  for (int n = 0; n < Nr; ++n)
    for (int k = 0; k < Nr; ++k) {
      double v = h.Dr[(size_t)n * Nr + k];
      const size_t o = (size_t)((n / 8) * KC + k / 8) * 64 + (n % 8) * 8 + (k % 8);
      for (int term = 0; term < 3; ++term) {
        const uint16_t b = bf16_rne((float)v);
        out[term * T + o] = b;
        v -= (double)bf16_value(b);
      }
    }
  return out;
}

// The angular pass's tensor-core B operands (16 x 16 direction blocks), each split
// into TF32 hi + lo in the K-major core layout (8-row x 4-column core matrices,
// core (n/8, k/4) at float offset ((n/8) KC + k/4) 32):
//   W1[n = k][kk] = A[k][kk] (kk < 16), B[k][kk - 16] (kk >= 16): the DFS pair of the
//   doubled Theta circle, K = 32;  W2[n = m][kk = m'] = D_Phi[m][m'], K = 16.
// Order: W1 hi, W1 lo, W2 hi, W2 lo.
std::vector<float> tc_angular_tables(const HostTables& h) {
  const int N = 16;
  std::vector<float> out((size_t)2 * N * 32 + 2 * N * 16, 0.f);
  auto put = [&](size_t base, int KC, int n, int k, double v, size_t term) {
    const float hi = tf32_round((float)v);
    const float lo = tf32_round((float)(v - (double)hi));
    const size_t o = (size_t)((n / 8) * KC + k / 4) * 32 + (n % 8) * 4 + (k % 4);
    out[base + o] = hi;
    out[base + term + o] = lo;
  };
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < 2 * N; ++k)
      put(0, 8, n, k, k < N ? h.ATh[(size_t)n * N + k] : h.BTh[(size_t)n * N + (k - N)],
          (size_t)N * 32);
  const size_t b2 = (size_t)2 * N * 32;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) put(b2, 4, n, k, h.DPh[(size_t)n * N + k], (size_t)N * 16);
  return out;
}

void even_odd_tables(HostTables& h) {
  auto pq = [](const Vec& A, const Vec& B, int N, Vec& PT, Vec& QT) {
    PT.assign((size_t)N * N, 0.0);
    QT.assign((size_t)N * N, 0.0);
    for (int o = 0; o < N; ++o)
      for (int i = 0; i < N; ++i) {
        PT[(size_t)i * N + o] = 0.5 * (A[(size_t)o * N + i] + B[(size_t)o * N + i]);
        QT[(size_t)i * N + o] = 0.5 * (A[(size_t)o * N + i] - B[(size_t)o * N + i]);
      }
  };
  pq(h.Ath, h.Bth, (int)h.theta.size(), h.PthT, h.QthT);
  pq(h.ATh, h.BTh, (int)h.Theta.size(), h.PThT, h.QThT);
  // radial: D[N-i][N-i'] = -D[i][i'] on the symmetric Gauss-Lobatto nodes, so the
  // pair (i, N-i) needs only E = u_i' + u_{N-i'} and O = u_i' - u_{N-i'}:
  //   D u (i)   = 1/2 (sum_i' Op[i][i'] O_i' + sum_i' Ep[i][i'] E_i' + 2 D[i][M] u_M)
  //   D u (N-i) = 1/2 (sum_i' Op[i][i'] O_i' - sum_i' Ep[i][i'] E_i' - 2 D[i][M] u_M)
  //   D u (M)   = sum_i' D[M][i'] O_i'                    (middle node M = N/2, odd Nr)
  const int Nr = (int)h.r.size(), N = Nr - 1, hh = Nr / 2;
  h.EpT.assign((size_t)hh * hh, 0.0);
  h.OpT.assign((size_t)hh * hh, 0.0);
  h.DrMc.assign(hh, 0.0);
  h.DrMr.assign(hh, 0.0);
  for (int i = 0; i < hh; ++i)
    for (int ip = 0; ip < hh; ++ip) {
      const double a = h.Dr[(size_t)i * Nr + ip], b = h.Dr[(size_t)i * Nr + (N - ip)];
      h.EpT[(size_t)ip * hh + i] = a + b;
      h.OpT[(size_t)ip * hh + i] = a - b;
    }
  if (Nr % 2) {
    const int M = N / 2;
    for (int i = 0; i < hh; ++i) {
      h.DrMc[i] = h.Dr[(size_t)i * Nr + M];
      h.DrMr[i] = h.Dr[(size_t)M * Nr + i];
    }
  }
  // the transposes: DFS halves read [in][out] = [j][j'] of A^T, i.e. A itself
  auto pqa = [](const Vec& A, const Vec& B, int N, Vec& PA, Vec& QA) {
    PA.assign((size_t)N * N, 0.0);
    QA.assign((size_t)N * N, 0.0);
    for (size_t x = 0; x < (size_t)N * N; ++x) {
      PA[x] = 0.5 * (A[x] + B[x]);
      QA[x] = 0.5 * (A[x] - B[x]);
    }
  };
  pqa(h.Ath, h.Bth, (int)h.theta.size(), h.PthA, h.QthA);
  pqa(h.ATh, h.BTh, (int)h.Theta.size(), h.PThA, h.QThA);
  // M = D_r^T, M[i][i'] = D[i'][i]: the same folding as above
  h.EpTa.assign((size_t)hh * hh, 0.0);
  h.OpTa.assign((size_t)hh * hh, 0.0);
  h.DrMca.assign(hh, 0.0);
  h.DrMra.assign(hh, 0.0);
  for (int i = 0; i < hh; ++i)
    for (int ip = 0; ip < hh; ++ip) {
      const double a = h.Dr[(size_t)ip * Nr + i], b = h.Dr[(size_t)(N - ip) * Nr + i];
      h.EpTa[(size_t)ip * hh + i] = a + b;
      h.OpTa[(size_t)ip * hh + i] = a - b;
    }
  if (Nr % 2) {
    const int M = N / 2;
    for (int i = 0; i < hh; ++i) {
      h.DrMca[i] = h.Dr[(size_t)M * Nr + i];
      h.DrMra[i] = h.Dr[(size_t)i * Nr + M];
    }
  }
  // Fourier derivative on DFS pair halves (D circulant, so D[p+N/2][q+N/2] = D[p][q]):
  // MsT[p'][p] = D[p][p'] + D[p][p'+N/2], MdT[p'][p] = D[p][p'] - D[p][p'+N/2]
  auto halves = [](const Vec& D, int N, Vec& MsT, Vec& MdT) {
    const int h = N / 2;
    MsT.assign((size_t)h * h, 0.0);
    MdT.assign((size_t)h * h, 0.0);
    for (int p = 0; p < h; ++p)
      for (int q = 0; q < h; ++q) {
        const double a = D[(size_t)p * N + q], b = D[(size_t)p * N + q + h];
        MsT[(size_t)q * h + p] = a + b;
        MdT[(size_t)q * h + p] = a - b;
      }
  };
  halves(h.DPh, (int)h.Phi.size(), h.MsPhT, h.MdPhT);
  halves(h.Dph, (int)h.phi.size(), h.MsphT, h.MdphT);
  // P and Q (from their transposed [in][out] forms) folded over k -> n-1-k:
  // FeT[k'][k] = P[k][k'] + P[k][n-1-k'], FoT[k'][k] = P[k][k'] - P[k][n-1-k']
  auto fold = [](const Vec& PT, int n, Vec& FeT, Vec& FoT) {
    const int h = n / 2;
    FeT.assign((size_t)h * h, 0.0);
    FoT.assign((size_t)h * h, 0.0);
    for (int k = 0; k < h; ++k)
      for (int kp = 0; kp < h; ++kp) {
        const double a = PT[(size_t)kp * n + k], b = PT[(size_t)(n - 1 - kp) * n + k];
        FeT[(size_t)kp * h + k] = a + b;
        FoT[(size_t)kp * h + k] = a - b;
      }
  };
  const int nT = (int)h.Theta.size(), nt = (int)h.theta.size();
  fold(h.PThT, nT, h.PeThT, h.PoThT);
  fold(h.QThT, nT, h.QeThT, h.QoThT);
  // the angular pass takes the 1/2 of the Theta folding from its tables
  for (Vec* v : {&h.PeThT, &h.PoThT, &h.QeThT, &h.QoThT})
    for (double& x : *v) x *= 0.5;
  fold(h.PthT, nt, h.PethT, h.PothT);
  fold(h.QthT, nt, h.QethT, h.QothT);
  // the adjoint's operators: P^T, Q^T are read [in][out] as PthA, PThA (= P, Q)
  fold(h.PThA, nT, h.PeThA, h.PoThA);
  fold(h.QThA, nT, h.QeThA, h.QoThA);
  fold(h.PthA, nt, h.PethA, h.PothA);
  fold(h.QthA, nt, h.QethA, h.QothA);
  const int nP = (int)h.Phi.size(), np = (int)h.phi.size();
  halves(transpose(h.DPh, nP, nP), nP, h.MsPhA, h.MdPhA);
  halves(transpose(h.Dph, np, np), np, h.MsphA, h.MdphA);
}

template <typename C>
cudaError_t upload_tables(const HostTables& h, void** mem, Tables<C>* t) {
  std::vector<Vec> tmp;
  std::vector<const Vec*> list = device_list(h, tmp);
  size_t n = 0;
  for (const Vec* v : list) n += (v->size() + 31) / 32 * 32;
  std::vector<C> host(n, (C)0);
  C* dev = nullptr;
  cudaError_t e = cudaMalloc((void**)&dev, n * sizeof(C));
  if (e != cudaSuccess) return e;
  C** slots[] = {&t->DrT, &t->AthT, &t->BthT, &t->DphT, &t->AThT, &t->BThT, &t->DPhT,
                 &t->Dr, &t->Ath, &t->Bth, &t->Dph, &t->ATh, &t->BTh, &t->DPh,
                 &t->inv_r, &t->inv_sinth, &t->cot_th, &t->sin_th, &t->cos_th, &t->sin_ph,
                 &t->cos_ph, &t->cosT, &t->sinT, &t->cosP, &t->sinP, &t->tsign, &t->qdir,
                 &t->FrT, &t->FthAT, &t->FthBT, &t->FphT, &t->FThAT, &t->FThBT, &t->FPhT,
                 &t->PthT, &t->QthT, &t->PThT, &t->QThT, &t->EpT, &t->OpT, &t->DrMc, &t->DrMr,
                 &t->TcBhi, &t->TcBlo,
                 &t->PthA, &t->QthA, &t->PThA, &t->QThA, &t->EpTa, &t->OpTa, &t->DrMca,
                 &t->DrMra, &t->MsPhT, &t->MdPhT, &t->MsphT, &t->MdphT,
                 &t->PeThT, &t->PoThT, &t->QeThT, &t->QoThT, &t->PethT, &t->PothT,
                 &t->QethT, &t->QothT,
                 &t->PeThA, &t->PoThA, &t->QeThA, &t->QoThA, &t->PethA, &t->PothA,
                 &t->QethA, &t->QothA, &t->MsPhA, &t->MdPhA, &t->MsphA, &t->MdphA};
  size_t off = 0;
  for (size_t a = 0; a < list.size(); ++a) {
    for (size_t b = 0; b < list[a]->size(); ++b) host[off + b] = (C)(*list[a])[b];
    *slots[a] = dev + off;
    off += (list[a]->size() + 31) / 32 * 32;
  }
  e = cudaMemcpy(dev, host.data(), n * sizeof(C), cudaMemcpyHostToDevice);
  *mem = dev;
  return e;
}

HostTables build_tables(const ts_grid_desc& g) {
  HostTables h;
  const int Nr = g.Nr, Nt = g.Ntheta, Np = g.Nphi, NT = g.NTheta, NP = g.NPhi;
  const int N = Nr - 1;
  const bool fd = g.radial == TS_RADIAL_UPWIND_FD;
  const bool zoned = g.radial == TS_RADIAL_ZONED;
  // zoned: edge zones of zone_nodes uniform nodes, width w; central Chebyshev zone
  const int zA = g.zone_nodes, zB = Nr - 2 * (g.zone_nodes - 1);
  const double zw = g.zone_width * (g.R2 - g.R1), zh = zoned ? zw / (zA - 1) : 0.0;
  for (int i = 0; i < Nr; ++i) {
    if (zoned) {
      const double a = g.R1 + zw, b = g.R2 - zw;
      if (i < zA) h.r.push_back(g.R1 + zh * i);
      else if (i < zA - 1 + zB - 1) h.r.push_back(0.5 * (a + b) - 0.5 * (b - a) *
                                                  std::cos(M_PI * (i - (zA - 1)) / (zB - 1)));
      else h.r.push_back(b + zh * (i - (zA - 1 + zB - 1)));
    } else {
      h.r.push_back(fd ? g.R1 + (g.R2 - g.R1) * i / N
                       : 0.5 * (g.R1 + g.R2) - 0.5 * (g.R2 - g.R1) * std::cos(M_PI * i / N));
    }
  }
  for (int j = 0; j < Nt; ++j) h.theta.push_back(M_PI * (j + 0.5) / Nt);
  for (int l = 0; l < Np; ++l) h.phi.push_back(2.0 * M_PI * l / Np);
  for (int k = 0; k < NT; ++k) h.Theta.push_back(M_PI * (k + 0.5) / NT);
  for (int m = 0; m < NP; ++m) h.Phi.push_back(2.0 * M_PI * m / NP);

  h.Dr = cheb_diff(Nr, g.R1, g.R2);
  dfs_split(fourier_diff(2 * Nt), Nt, h.Ath, h.Bth);
  h.Dph = fourier_diff(Np);
  dfs_split(fourier_diff(2 * NT), NT, h.ATh, h.BTh);
  h.DPh = fourier_diff(NP);
  if (g.form == TS_FORM_CONSERVATIVE) {
    // Fhat carries sin(theta) sin(Theta): its continuation to a reflected node of
    // either doubled circle is minus its value at the partner
    for (double& x : h.Bth) x = -x;
    for (double& x : h.BTh) x = -x;
  }

  const double fa = g.filter_alpha > 0 ? g.filter_alpha : 36.0;
  const int fo = g.filter_order > 0 ? g.filter_order : 16;
  h.Fr = cheb_filter(Nr, fa, fo);
  if (fd || zoned) {   // no radial filter on the finite-difference and zoned grids
    h.Fr.assign((size_t)Nr * Nr, 0.0);
    for (int i = 0; i < Nr; ++i) h.Fr[(size_t)i * Nr + i] = 1.0;
  }
  dfs_split(fourier_filter(2 * Nt, Nt, fa, fo), Nt, h.FthA, h.FthB);
  h.Fph = fourier_filter(Np, Np / 2, fa, fo);
  dfs_split(fourier_filter(2 * NT, NT, fa, fo), NT, h.FThA, h.FThB);
  h.FPh = fourier_filter(NP, NP / 2, fa, fo);

  for (int i = 0; i < Nr; ++i) {
    h.inv_r.push_back(1.0 / h.r[i]);
    h.tsign.push_back(((N - i) % 2) ? -1.0 : 1.0);  // T_N(x_i) = cos(pi (N - i)) on these nodes
  }
  for (int j = 0; j < Nt; ++j) {
    const double s = std::sin(h.theta[j]), c = std::cos(h.theta[j]);
    h.inv_sinth.push_back(1.0 / s);
    h.cot_th.push_back(c / s);
    h.sin_th.push_back(s);
    h.cos_th.push_back(c);
  }
  for (int l = 0; l < Np; ++l) {
    h.sin_ph.push_back(std::sin(h.phi[l]));
    h.cos_ph.push_back(std::cos(h.phi[l]));
  }
  const Vec fT = fejer(NT);
  for (int k = 0; k < NT; ++k) {
    h.cosT.push_back(std::cos(h.Theta[k]));
    h.sinT.push_back(std::sin(h.Theta[k]));
    // J = (1/4pi) int F dOmega = sum_k fejer_k (2pi/NP)/(4pi) sum_m F_km
    h.qdir.push_back(fT[k] / (2.0 * NP));
  }
  for (int m = 0; m < NP; ++m) {
    h.cosP.push_back(std::cos(h.Phi[m]));
    h.sinP.push_back(std::sin(h.Phi[m]));
  }
  const Vec cc = clenshaw_curtis(Nr);
  for (int i = 0; i < Nr; ++i) {
    // int r^2 dr: Clenshaw-Curtis on the Chebyshev nodes, trapezoid on the uniform ones
    const double w = fd ? (g.R2 - g.R1) / N * ((i == 0 || i == N) ? 0.5 : 1.0)
                        : cc[i] * 0.5 * (g.R2 - g.R1);
    h.wr.push_back(w * h.r[i] * h.r[i]);
  }
  if (zoned) {   // trapezoid in the edge zones, Clenshaw-Curtis in the central one
    const Vec ccB = clenshaw_curtis(zB);
    Vec w(Nr, 0.0);
    const int iB0 = zA - 1, iB1 = zA - 1 + zB - 1;
    for (int i = 0; i < zA; ++i) {
      const double t = zh * ((i == 0 || i == zA - 1) ? 0.5 : 1.0);
      w[i] += t;
      w[iB1 + i] += t;
    }
    for (int j = 0; j < zB; ++j) w[iB0 + j] += ccB[j] * 0.5 * (g.R2 - g.R1 - 2 * zw);
    for (int i = 0; i < Nr; ++i) h.wr[i] = w[i] * h.r[i] * h.r[i];
  }
  h.wth = fejer(Nt);
  even_odd_tables(h);
  tc_tables(h);
  h.fluxw.resize((size_t)Nt * Np * NT * NP);
  for (int j = 0; j < Nt; ++j)
    for (int l = 0; l < Np; ++l)
      for (int k = 0; k < NT; ++k)
        for (int m = 0; m < NP; ++m)
          h.fluxw[(((size_t)j * Np + l) * NT + k) * NP + m] =
              g.R2 * g.R2 * h.wth[j] * (2.0 * M_PI / Np) * fT[k] * h.cosT[k] * (2.0 * M_PI / NP);
  return h;
}

}  // namespace

void ts::set_last_error(const std::string& msg) { g_err = msg; }
ts::Vec ts::cheb_diff_matrix(int Nr, double R1, double R2) { return cheb_diff(Nr, R1, R2); }
ts::Vec ts::fourier_diff_matrix(int M) { return fourier_diff(M); }
ts::Vec ts::fejer_weights(int N) { return fejer(N); }
ts::Vec ts::clenshaw_curtis_weights(int Nr) { return clenshaw_curtis(Nr); }
ts_status ts::fail_status(ts_status s, const std::string& msg) { return fail(s, msg); }
ts_status ts::cuda_status(cudaError_t e, const char* where) { return cuda_fail(e, where); }

namespace {

ts::Problem make_problem(const ts_grid* g) {
  ts::Problem p;
  p.d = g->d;
  p.tp = g->tp;
  p.bc = g->desc.bc;
  p.n_fp64_rows = g->desc.precision == TS_FP32_R64 ? 2 : 0;
  p.kap = g->kap;
  p.eta = g->eta;
  p.kaps = g->kaps;
  p.scb = g->aniso ? g->scb : nullptr;
  p.scc = g->quad ? g->scc : nullptr;
  p.gR1 = g->gR1;
  p.gR2 = g->gR2;
  p.tc = !ts::tc_supported(g->d.Nr)             ? ts::TC_NONE
         : g->desc.precision == TS_TF32X3 ? ts::TC_TF32X3
         : g->desc.precision == TS_BF16X3 ? ts::TC_BF16X3
                                          : ts::TC_NONE;
  p.tcb16 = g->tcb16;
  p.err = g->err;
  p.wait_operand = g->wait_operand > 0 ? g->wait_operand : ts::kDefaultWaitIters;
  if (g->wait_operand < 0) p.wait_operand = 0;
  p.plane_store = 0;
  p.ep64 = g->t64.EpT;
  p.op64 = g->t64.OpT;
  p.mc64 = g->t64.DrMc;
  p.tcang = g->tcang;
  if (g->sn > 0) {   // one slice of groups: every per-group pointer offset to group s0
    const long long per = g->d.nblk / g->d.G;
    const long long infl = (long long)g->d.Nt * g->d.Np * (g->d.NT / 2) * g->d.NP;
    p.d.G = g->sn;
    p.d.total = (long long)g->sn * g->d.S_g;
    p.d.nblk = per * g->sn;
    p.kap += g->s0 * per;
    p.eta += g->s0 * per;
    p.kaps += g->s0 * per;
    if (p.scb) p.scb += g->s0 * per;
    if (p.scc) p.scc += g->s0 * per;
    p.gR1 = static_cast<const char*>(p.gR1) + g->s0 * infl * (long long)g->es;
    p.gR2 = static_cast<const char*>(p.gR2) + g->s0 * infl * (long long)g->es;
  }
  return p;
}

// A workspace field of the grid at the current group slice.
template <typename T>
T* work(const ts_grid* g, void* base) {
  return static_cast<T*>(base) + (g->sn > 0 ? g->s0 * g->d.S_g : 0);
}

size_t field_bytes(const ts_grid* g) { return (size_t)g->d.total * g->es; }

}  // namespace

ts::Problem ts::problem_of(const ts_grid* g) { return make_problem(g); }

namespace {

// Optional per-launch event timing (ts_step_profile). Each launch is
// bracketed by two events on the launching stream; `kind` selects the bucket.
struct Profiler {
  cudaStream_t st;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  cudaError_t mark() {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    return cudaEventRecord(e, st);
  }
  cudaError_t begin() { return mark(); }
  cudaError_t end(int k) {
    kind.push_back(k);
    return mark();
  }
  void collect(double* ms, int* n) {
    for (size_t a = 0; a < kind.size(); ++a) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[2 * a], ev[2 * a + 1]);
      if (ms) ms[kind[a]] += t;
      if (n) n[kind[a]] += 1;
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    kind.clear();
  }
};

#define TS_TIMED(prof, k, call)                              \
  do {                                                       \
    if (e == cudaSuccess && (prof)) e = (prof)->begin();     \
    if (e == cudaSuccess) e = (call);                        \
    if (e == cudaSuccess && (prof)) e = (prof)->end(k);      \
  } while (0)

// The radial pass of the grid's radial discretisation: the spectral pass
// (Chebyshev nodes) or the one-sided differences of the hybrid grid.
template <typename T, typename C>
cudaError_t radial_pass(const ts_grid* g, const ts::Problem& p, const Tables<C>& t, const T* U,
                        const T* K, C sgn, bool tau, int mode, T* F, T* Acc, T* Uout, T* out,
                        double dt, cudaStream_t st) {
  if (g->desc.radial == TS_RADIAL_UPWIND_FD)
    return ts::launch_radial_fd<T, C>(p, t, U, K, sgn, tau, mode, F, Acc, Uout, out, dt,
                                      (g->desc.R2 - g->desc.R1) / (g->desc.Nr - 1), st);
  if (g->desc.radial == TS_RADIAL_ZONED) {
    const C* zt = static_cast<const C*>(sizeof(C) == 8 ? g->zt64 : g->zt32);
    return ts::launch_radial_zoned<T, C>(p, t, zt, g->zA, g->zB, g->zh, U, K, sgn, tau, mode,
                                         F, Acc, Uout, out, dt, st);
  }
  return Launch<T, C>::radial(p, t, g->t64.Dr, U, K, sgn, tau, mode, F, Acc, Uout, out, dt, st);
}

// One stage derivative of `in` and the radial pass's output `mode`: the angular,
// plane and radial passes, or -- float grids with a fused plan -- the plane
// pass writing its terms into the grid's K and the fused angular + radial pass.
template <typename T, typename C>
cudaError_t stage_passes(ts_grid* g, const ts::Problem& p, const Tables<C>& t, const T* in, T* K,
                         C sgn, bool collision, bool tau, int mode, T* F, T* Acc, T* Uout,
                         T* out, double dt, cudaStream_t st, Profiler* prof) {
  cudaError_t e = cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    if (p.tp.fnb > 0) {
      ts::Problem pp = p;
      pp.plane_store = 1;
      TS_TIMED(prof, 1, (Launch<T, C>::plane(pp, t, in, K, sgn, st)));
      TS_TIMED(prof, 2, (ts::launch_fused(p, t, g->t64.Dr, in, K, sgn, collision, tau, mode, F,
                                          Acc, Uout, out, dt, st)));
      return e;
    }
  }
  if constexpr (std::is_same<T, C>::value) {
    if (g->desc.form == TS_FORM_CONSERVATIVE) {
      TS_TIMED(prof, 0, (ts::launch_angular_cons<T>(p, t, in, K, sgn, collision, st)));
    } else {
      TS_TIMED(prof, 0, (Launch<T, C>::angular(p, t, in, K, sgn, collision, st)));
    }
  } else {
    TS_TIMED(prof, 0, (Launch<T, C>::angular(p, t, in, K, sgn, collision, st)));
  }
  TS_TIMED(prof, 1, (Launch<T, C>::plane(p, t, in, K, sgn, st)));
  TS_TIMED(prof, 2, (radial_pass<T, C>(g, p, t, in, K, sgn, tau, mode, F, Acc, Uout, out, dt,
                                       st)));
  return e;
}

template <typename T, typename C>
cudaError_t run_stage(ts_grid* g, const Tables<C>& t, const T* in, T* F, int s, bool collision,
                      double dt, cudaStream_t st, Profiler* prof) {
  const ts::Problem p = make_problem(g);
  T* K = work<T>(g, g->K);
  T* U = work<T>(g, g->U);
  T* Acc = work<T>(g, g->Acc);
  return stage_passes<T, C>(g, p, t, in, K, (C)-1, collision, g->desc.bc == TS_BC_TAU_INFLOW,
                            ts::RAD_STAGE0 + s, F, Acc, U, nullptr, dt, st, prof);
}

template <typename T, typename C>
cudaError_t run_steps(ts_grid* g, const Tables<C>& t, T* F, double dt, int nsteps,
                      cudaStream_t st, Profiler* prof = nullptr, const void* key = nullptr) {
  const bool split = g->desc.scheme == TS_RK4_SPLIT_IMPLICIT;
  const ts::Problem p = make_problem(g);
  cudaError_t e = cudaSuccess;
  if (g->desc.scheme == TS_AB2) {
    // one stage derivative per step; the radial pass finishes K and applies the
    // Adams-Bashforth update in place, keeping K in Acc for the next step
    if (g->hist_F != (key ? key : F)) g->hist = false;
    g->hist_F = key ? key : F;
    T* K = work<T>(g, g->K);
    T* Acc = work<T>(g, g->Acc);
    const bool tau = g->desc.bc == TS_BC_TAU_INFLOW;
    for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
      e = stage_passes<T, C>(g, p, t, F, K, (C)-1, true, tau,
                             g->hist ? ts::RAD_AB2 : ts::RAD_AB2_START, F, Acc, nullptr, nullptr,
                             dt, st, prof);
      if (e == cudaSuccess) g->hist = true;
      if (g->desc.filter_on) TS_TIMED(prof, 3, (Launch<T, C>::filter(p, t, F, K, st)));
    }
    if (e != cudaSuccess) g->hist = false;
    return e;
  }
  for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
    for (int s = 0; s < 4 && e == cudaSuccess; ++s)
      e = run_stage<T, C>(g, t, s == 0 ? F : work<T>(g, g->U), F, s, !split, dt, st, prof);
    if (split) TS_TIMED(prof, 3, (Launch<T, C>::implicit_collision(p, t, F, dt, st)));
    if (g->desc.filter_on) TS_TIMED(prof, 3, (Launch<T, C>::filter(p, t, F, work<T>(g, g->K), st)));
  }
  return e;
}

template <typename T, typename C>
cudaError_t run_rhs(ts_grid* g, const Tables<C>& t, const T* F, T* K, bool liouville_only,
                    cudaStream_t st) {
  const ts::Problem p = make_problem(g);
  const C sgn = liouville_only ? (C)1 : (C)-1;
  return stage_passes<T, C>(g, p, t, F, K, sgn, !liouville_only,
                            !liouville_only && g->desc.bc == TS_BC_TAU_INFLOW, ts::RAD_RHS,
                            nullptr, nullptr, nullptr, K, 0.0, st, nullptr);
}

template <typename T, typename C>
cudaError_t run_adjoint(ts_grid* g, const Tables<C>& t, const T* Fn, T* lam, double* gk,
                        double* ge, double dt, cudaStream_t st) {
  const ts::Problem p = make_problem(g);
  const bool tau = g->desc.bc == TS_BC_TAU_INFLOW;
  T* K = static_cast<T*>(g->K);
  T* junk = static_cast<T*>(g->Acc);
  T* U2 = static_cast<T*>(g->adj[0]);
  T* U3 = static_cast<T*>(g->adj[1]);
  T* U4 = static_cast<T*>(g->adj[2]);
  T* Kb = static_cast<T*>(g->adj[3]);
  T* lt = static_cast<T*>(g->adj[4]);
  T* Ub = static_cast<T*>(g->adj[5]);
  T* lacc = static_cast<T*>(g->adj[6]);
  T* Fmut = const_cast<T*>(Fn);  // stage modes 0..2 only read F
  // forward recomputation of the stage inputs U2, U3, U4
  const T* ins[3] = {Fn, U2, U3};
  T* outs[3] = {U2, U3, U4};
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
    e = Launch<T, C>::angular(p, t, ins[s], K, (C)-1, true, st);
    if (e == cudaSuccess) e = Launch<T, C>::plane(p, t, ins[s], K, (C)-1, st);
    if (e == cudaSuccess)
      e = Launch<T, C>::radial(p, t, g->t64.Dr, ins[s], K, (C)-1, tau, ts::RAD_STAGE0 + s,
                               Fmut, junk, outs[s], nullptr, dt, st);
  }
  // reverse sweep: stage 4, 3, 2, 1
  const T* Us[4] = {Fn, U2, U3, U4};
  const double wl[4] = {0.0, dt / 6.0, dt / 3.0, dt / 3.0};   // weight of lam in Kbar_{s-1}
  const double wu[4] = {0.0, 0.5 * dt, 0.5 * dt, dt};         // weight of Ubar_s in Kbar_{s-1}
  for (int s = 3; s >= 0 && e == cudaSuccess; --s) {
    if (s == 3) e = Launch<T, C>::radial_T(p, t, lam, dt / 6.0, tau, lt, Ub, st);
    else e = Launch<T, C>::radial_T(p, t, Kb, 1.0, tau, lt, Ub, st);
    if (e == cudaSuccess) e = Launch<T, C>::plane_T(p, t, lt, Ub, st);
    if (e == cudaSuccess)
      e = Launch<T, C>::angular_T(p, t, lt, Ub, Us[s], gk, ge, lam, s == 3 ? lam : lacc,
                                  s == 0 ? lam : lacc, s == 0 ? nullptr : Kb, wl[s], wu[s], st);
  }
  return e;
}

// mu = a lam + b lam_prev, then lam_prev = lam (the AB2 adjoint's stage weights and
// the shift of its two time levels)
template <typename T>
__global__ void k_ab2_mu(const T* lam, T* lam_prev, T* mu, double a, double b, long long n) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n;
       x += (long long)gridDim.x * blockDim.x) {
    const double l = (double)lam[x];
    mu[x] = (T)(a * l + b * (double)lam_prev[x]);
    lam_prev[x] = (T)l;
  }
}

template <typename T, typename C>
cudaError_t run_adjoint_ab2(ts_grid* g, const Tables<C>& t, const T* Fn, T* lam, T* lam_prev,
                            double* gk, double* ge, double dt, bool first, cudaStream_t st) {
  const ts::Problem p = make_problem(g);
  const bool tau = g->desc.bc == TS_BC_TAU_INFLOW;
  T* mu = static_cast<T*>(g->adj[3]);
  T* lt = static_cast<T*>(g->adj[4]);
  T* Ub = static_cast<T*>(g->adj[5]);
  const long long n = g->d.total;
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
  k_ab2_mu<T><<<blocks, 256, 0, st>>>(lam, lam_prev, mu, dt * (first ? 1.0 : 1.5), -0.5 * dt, n);
  cudaError_t e = cudaGetLastError();
  // lam <- lam + A^T Tau^T mu; the gradients from Tau^T mu and F_n
  if (e == cudaSuccess) e = Launch<T, C>::radial_T(p, t, mu, 1.0, tau, lt, Ub, st);
  if (e == cudaSuccess) e = Launch<T, C>::plane_T(p, t, lt, Ub, st);
  if (e == cudaSuccess)
    e = Launch<T, C>::angular_T(p, t, lt, Ub, Fn, gk, ge, lam, lam, lam, nullptr, 0.0, 0.0, st);
  return e;
}

ts_status adjoint_workspace(ts_grid* g) {
  if (g->adj[0]) return TS_OK;
  const char* poison = std::getenv("TS_POISON_WORKSPACE");   // see ts_create_grid
  for (int a = 0; a < 7; ++a) {
    cudaError_t e = cudaMalloc(&g->adj[a], field_bytes(g));
    if (e == cudaSuccess && poison && poison[0] == '1')
      e = cudaMemset(g->adj[a], 0xFF, field_bytes(g));
    if (e != cudaSuccess) {
      for (int b = 0; b <= a; ++b) {
        if (g->adj[b]) cudaFree(g->adj[b]);
        g->adj[b] = nullptr;
      }
      cudaGetLastError();
      return fail(TS_ERR_OOM, "adjoint workspace allocation failed");
    }
  }
  return TS_OK;
}

bool fits(const ts_grid_desc& g, size_t es) {
  const size_t mx = 227 * 1024;
  const size_t a = (size_t)(2 * g.NTheta * g.NTheta + g.NPhi * g.NPhi + 2 * g.NTheta * g.NPhi + 1) * es;
  const size_t p = (size_t)(2 * g.Ntheta * g.Ntheta + g.Nphi * g.Nphi + 2 * g.Ntheta * g.Nphi * 2) * es;
  const size_t r = (size_t)(g.Nr * g.Nr + 2 * g.Nr * 8) * es;
  return a <= mx && p <= mx && r <= mx;
}

ts_status check_F(const ts_grid* g, const void* F) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  if (!F) return fail(TS_ERR_ARG, "field pointer is NULL");
  if (!ts::aligned16(F)) return fail(TS_ERR_ARG, "field pointer is not 16-byte aligned");
  return TS_OK;
}

// A device output or adjoint field: non-NULL and 16-byte aligned.
ts_status check_out(const void* p, const char* what) {
  if (!p) return fail(TS_ERR_ARG, std::string(what) + " is NULL");
  if (!ts::aligned16(p)) return fail(TS_ERR_ARG, std::string(what) + " is not 16-byte aligned");
  return TS_OK;
}

}  // namespace

namespace {

// Power iteration of ts_stable_dt. Partial sums of squares of (y - y0) per
// block (fixed grid, deterministic order), written back into y.
constexpr int kPiBlocks = 304, kPiThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPiThreads)
k_pi_sub_norm(T* y, const T* y0, long long n, double* part) {
  __shared__ double red[kPiThreads];
  double a = 0.0;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n;
       x += (long long)gridDim.x * blockDim.x) {
    const double v = y0 ? (double)y[x] - (double)y0[x] : (double)y[x];
    if (y0) y[x] = (T)v;
    a = fma(v, v, a);
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// norm = sqrt(sum of the partials); logs[it] = log(norm) (it >= 0)
__global__ void k_pi_finish(const double* part, int np, double* norm, double* logs, int it) {
  __shared__ double red[kPiThreads];
  double a = 0.0;
  for (int x = threadIdx.x; x < np; x += blockDim.x) a += part[x];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *norm = sqrt(red[0]);
    if (it >= 0) logs[it] = log(*norm);
  }
}

template <typename T>
__global__ void k_pi_scale(const T* y, T* x, long long n, const double* norm) {
  const double s = 1.0 / *norm;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = (T)((double)y[i] * s);
}

template <typename T, typename C>
cudaError_t power_iteration(ts_grid* g, const Tables<C>& t, const T* x0, int iters,
                            std::vector<double>& logs, cudaStream_t st) {
  const long long n = g->d.total;
  T* x = static_cast<T*>(g->U);
  T* y = static_cast<T*>(g->K);
  T* y0 = static_cast<T*>(g->Acc);
  double* part = g->piw;
  double* norm = g->piw + kPiBlocks;
  double* lg = g->piw + kPiBlocks + 1;
  // y0 = K(0): the affine part (emissivity, inflow rows)
  cudaError_t e = cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), st);
  if (e == cudaSuccess) e = run_rhs<T, C>(g, t, x, y0, false, st);
  // x = x0 / |x0|
  if (e == cudaSuccess) {
    k_pi_sub_norm<T><<<kPiBlocks, kPiThreads, 0, st>>>(const_cast<T*>(x0), nullptr, n, part);
    k_pi_finish<<<1, kPiThreads, 0, st>>>(part, kPiBlocks, norm, lg, -1);
    k_pi_scale<T><<<kPiBlocks, kPiThreads, 0, st>>>(x0, x, n, norm);
    e = cudaGetLastError();
  }
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    e = run_rhs<T, C>(g, t, x, y, false, st);                // y = K(x)
    if (e != cudaSuccess) break;
    k_pi_sub_norm<T><<<kPiBlocks, kPiThreads, 0, st>>>(y, y0, n, part);   // y = K(x) - K(0)
    k_pi_finish<<<1, kPiThreads, 0, st>>>(part, kPiBlocks, norm, lg, it);
    k_pi_scale<T><<<kPiBlocks, kPiThreads, 0, st>>>(y, x, n, norm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    logs.assign(iters, 0.0);
    e = cudaMemcpyAsync(logs.data(), lg, iters * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace

cudaError_t ts::step_grid(ts_grid* g, void* F, double dt, int nsteps, cudaStream_t st) {
  return g->es == 8 ? run_steps<double, double>(g, g->t64, (double*)F, dt, nsteps, st)
                    : run_steps<float, float>(g, g->t32, (float*)F, dt, nsteps, st);
}

namespace {
template <typename T, typename C>
cudaError_t ab2_step(ts_grid* g, const Tables<C>& t, T* F, double dt, bool first,
                     cudaStream_t st) {
  const ts::Problem p = make_problem(g);
  T* K = work<T>(g, g->K);
  T* Acc = work<T>(g, g->Acc);
  cudaError_t e = stage_passes<T, C>(g, p, t, F, K, (C)-1, true, g->desc.bc == TS_BC_TAU_INFLOW,
                                     first ? ts::RAD_AB2_START : ts::RAD_AB2, F, Acc, nullptr,
                                     nullptr, dt, st, nullptr);
  if (e == cudaSuccess && g->desc.filter_on) e = Launch<T, C>::filter(p, t, F, K, st);
  return e;
}
}  // namespace

cudaError_t ts::step_grid_ab2(ts_grid* g, void* F, double dt, bool first, cudaStream_t st) {
  return g->es == 8 ? ab2_step<double, double>(g, g->t64, (double*)F, dt, first, st)
                    : ab2_step<float, float>(g, g->t32, (float*)F, dt, first, st);
}

void ts::set_ab2_history(ts_grid* g, const void* F) {
  g->hist = true;
  g->hist_F = F;
}

extern "C" {

const char* ts_last_error(void) { return g_err.c_str(); }

const char* ts_version(void) { return "ts 0.1 (sm_103a, 6-D spectral transport step)"; }

size_t ts_field_elems(const ts_grid* g) { return g ? (size_t)g->d.total : 0; }

ts_status ts_create_grid(const ts_grid_desc* desc, ts_grid** out) {
  if (!out) return fail(TS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(TS_ERR_ARG, "desc is NULL");
  const ts_grid_desc& g = *desc;
  if (!(g.R1 > 0.0) || !(g.R2 > g.R1) || !std::isfinite(g.R2))
    return fail(TS_ERR_ARG, "need 0 < R1 < R2");
  if (g.groups < 1) return fail(TS_ERR_ARG, "groups must be >= 1");
  if (g.Nr < 3 || g.Nr > 129 || g.Ntheta < 2 || g.Ntheta > 64 || g.Nphi < 2 || g.Nphi > 64 ||
      g.NTheta < 2 || g.NTheta > 64 || g.NPhi < 2 || g.NPhi > 64 || (g.Nphi % 2) ||
      (g.NTheta % 2) || (g.NPhi % 2))
    return fail(TS_ERR_UNSUPPORTED,
                "sizes: need 3<=Nr<=129, 2<=Ntheta<=64, even 2..64 for Nphi, NTheta, NPhi");
  if (g.precision != TS_FP64 && g.precision != TS_FP32 && g.precision != TS_FP32_R64 &&
      g.precision != TS_TF32X3 && g.precision != TS_BF16X3)
    return fail(TS_ERR_UNSUPPORTED, "unknown precision");
  if (g.scheme != TS_RK4 && g.scheme != TS_RK4_SPLIT_IMPLICIT && g.scheme != TS_AB2)
    return fail(TS_ERR_UNSUPPORTED, "unknown scheme");
  if (g.bc != TS_BC_TAU_INFLOW && g.bc != TS_BC_NONE) return fail(TS_ERR_UNSUPPORTED, "unknown bc");
  if (g.radial != TS_RADIAL_CHEBYSHEV && g.radial != TS_RADIAL_UPWIND_FD &&
      g.radial != TS_RADIAL_ZONED)
    return fail(TS_ERR_UNSUPPORTED, "unknown radial discretisation");
  if (g.radial != TS_RADIAL_CHEBYSHEV && g.precision != TS_FP64 && g.precision != TS_FP32)
    return fail(TS_ERR_UNSUPPORTED,
                "the finite-difference and zoned radial grids run in TS_FP64 or TS_FP32");
  if (g.radial == TS_RADIAL_ZONED &&
      (g.zone_nodes < 2 || g.Nr - 2 * (g.zone_nodes - 1) < 3 || !(g.zone_width > 0.0) ||
       !(g.zone_width < 0.5)))
    return fail(TS_ERR_UNSUPPORTED,
                "zoned radial grid: need zone_nodes >= 2, Nr - 2 (zone_nodes - 1) >= 3, "
                "0 < zone_width < 1/2");
  if (g.form != TS_FORM_ADVECTIVE && g.form != TS_FORM_CONSERVATIVE)
    return fail(TS_ERR_UNSUPPORTED, "unknown form");
  if (g.form == TS_FORM_CONSERVATIVE &&
      (g.radial != TS_RADIAL_CHEBYSHEV || g.scheme == TS_RK4_SPLIT_IMPLICIT || g.filter_on))
    return fail(TS_ERR_UNSUPPORTED,
                "the conservative form runs on the Chebyshev radial grid with TS_RK4 or "
                "TS_AB2, unfiltered");
  const size_t es = g.precision == TS_FP64 ? 8 : 4;
  if (!fits(g, es)) return fail(TS_ERR_UNSUPPORTED, "grid too large for one shared-memory tile");

  ts_grid* G = new ts_grid();
  G->desc = g;
  G->es = es;
  Dims& d = G->d;
  d.G = g.groups; d.Nr = g.Nr; d.Nt = g.Ntheta; d.Np = g.Nphi; d.NT = g.NTheta; d.NP = g.NPhi;
  d.S_l = (long long)g.NTheta * g.NPhi;
  d.S_j = d.S_l * g.Nphi;
  d.S_i = d.S_j * g.Ntheta;
  d.S_g = d.S_i * g.Nr;
  d.total = d.S_g * g.groups;
  d.nblk = (long long)g.groups * g.Nr * g.Ntheta * g.Nphi;
  G->h = build_tables(g);
  {
    const char* gen = std::getenv("TS_GENERIC_PASSES");  // 1: plain passes only (testing)
    G->tp.rb = (gen && gen[0] == '1') ? 0 : ts::rb_mask(d, (int)es, g.precision == TS_FP32_R64 ? 2 : 0);
    if (g.radial != TS_RADIAL_CHEBYSHEV) G->tp.rb &= ~4;   // no even/odd radial form
    // fused angular + radial pass: float grids with the even/odd angular and radial
    // forms (not the tensor-core radial precisions) whose tile fits shared memory
    // (TS_FUSED=1 selects it; its contractions are not yet faster than the three
    // passes', so the three-pass form stays the default)
    const char* fz = std::getenv("TS_FUSED");
    const bool tc = g.precision == TS_TF32X3 || g.precision == TS_BF16X3;
    const bool want = es == 4 && !tc && (G->tp.rb & 5) == 5 && fz && fz[0] == '1' &&
                      g.form == TS_FORM_ADVECTIVE;   // the fused pass is the advective one
    if (!want || !ts::fused_plan(d, g.precision == TS_FP32_R64 ? 2 : 0, &G->tp.fnb, &G->tp.fnbuf))
      G->tp.fnb = G->tp.fnbuf = 0;
  }

  cudaError_t e = upload_tables<double>(G->h, &G->tab64, &G->t64);
  if (e == cudaSuccess && g.precision != TS_FP64) e = upload_tables<float>(G->h, &G->tab32, &G->t32);
  if (e == cudaSuccess && g.precision == TS_TF32X3 && g.NTheta == 16 && g.NPhi == 16 &&
      g.radial == TS_RADIAL_CHEBYSHEV) {
    // TS_TC_ANGULAR=1 puts the angular pass on the tensor cores too; it is correct
    // but slower than the SIMT pass (each CTA's split -> MMA -> epilogue runs in
    // series on K = 16..32 contractions), so the SIMT pass stays the default
    const char* on = std::getenv("TS_TC_ANGULAR");
    if (on && on[0] == '1') {
      const std::vector<float> w = tc_angular_tables(G->h);
      e = cudaMalloc((void**)&G->tcang, w.size() * sizeof(float));
      if (e == cudaSuccess)
        e = cudaMemcpy(G->tcang, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess && g.radial == TS_RADIAL_ZONED) {
    G->zA = g.zone_nodes;
    G->zB = g.Nr - 2 * (g.zone_nodes - 1);
    const double w = g.zone_width * (g.R2 - g.R1);
    G->zh = w / (G->zA - 1);
    // the central zone's Gauss-Lobatto matrix D ([out][in]) folded over its
    // centro-antisymmetry: Ep, Op = (D[i][j] +- D[i][M-j]) / 2 (i, j < H),
    // Dm[i] = D[i][M/2], Mr[j] = D[M/2][j] (odd nB), then T_N on its nodes
    const int nB = G->zB, M = nB - 1, Hh = nB / 2;
    const Vec D = cheb_diff(nB, g.R1 + w, g.R2 - w);
    Vec zt;
    for (int i = 0; i < Hh; ++i)
      for (int j = 0; j < Hh; ++j) zt.push_back(0.5 * (D[i * nB + j] + D[i * nB + M - j]));
    for (int i = 0; i < Hh; ++i)
      for (int j = 0; j < Hh; ++j) zt.push_back(0.5 * (D[i * nB + j] - D[i * nB + M - j]));
    for (int i = 0; i < Hh; ++i) zt.push_back((nB & 1) ? D[i * nB + Hh] : 0.0);
    for (int j = 0; j < Hh; ++j) zt.push_back((nB & 1) ? D[Hh * nB + j] : 0.0);
    for (int j = 0; j < nB; ++j) zt.push_back(((nB - 1 - j) % 2) ? -1.0 : 1.0);
    e = cudaMalloc(&G->zt64, zt.size() * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpy(G->zt64, zt.data(), zt.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && g.precision != TS_FP64) {
      std::vector<float> zf(zt.begin(), zt.end());
      e = cudaMalloc(&G->zt32, zf.size() * sizeof(float));
      if (e == cudaSuccess)
        e = cudaMemcpy(G->zt32, zf.data(), zf.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess && g.precision == TS_BF16X3) {
    const std::vector<uint16_t> b16 = tc_tables_bf16(G->h);
    e = cudaMalloc(&G->tcb16, b16.size() * sizeof(uint16_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(G->tcb16, b16.data(), b16.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  }
  const size_t ncoef = (size_t)d.nblk * sizeof(double);
  const size_t ninfl = (size_t)g.groups * g.Ntheta * g.Nphi * (g.NTheta / 2) * g.NPhi * es;
  const size_t nf = (size_t)d.total * es;
  void** bufs[] = {(void**)&G->kap, (void**)&G->eta, (void**)&G->kaps, &G->gR1, &G->gR2,
                   &G->U, &G->K, &G->Acc, (void**)&G->wr, (void**)&G->wth,
                   (void**)&G->partN, (void**)&G->partJ, (void**)&G->err};
  const size_t sizes[] = {ncoef, ncoef, ncoef, ninfl, ninfl, nf, nf, nf,
                          (size_t)g.Nr * 8, (size_t)g.Ntheta * 8, ncoef,
                          (size_t)g.groups * 2 * g.Ntheta * g.Nphi * 8, sizeof(int)};
  // TS_POISON_WORKSPACE=1 (testing): the workspace fields U, K, Acc start as
  // NaN (all bits set) instead of zero, so that a read of a workspace element
  // no pass has written shows up as NaN in the result
  const char* poison = std::getenv("TS_POISON_WORKSPACE");
  const bool nan_ws = poison && poison[0] == '1';
  for (int b = 0; b < 13 && e == cudaSuccess; ++b) {
    e = cudaMalloc(bufs[b], sizes[b]);
    const bool ws = b >= 5 && b <= 7;
    if (e == cudaSuccess) e = cudaMemset(*bufs[b], ws && nan_ws ? 0xFF : 0, sizes[b]);
  }
  if (e == cudaSuccess) {
    // the number integral's weights: int r^2 dr, Fejer in cos theta and cos Theta
    // (F); int dr and Fejer on Fhat / sin in theta and Theta (Fhat)
    const bool cons = g.form == TS_FORM_CONSERVATIVE;
    const Vec fT = fejer(g.NTheta);
    Vec w;
    for (int i = 0; i < g.Nr; ++i) w.push_back(cons ? G->h.wr[i] / (G->h.r[i] * G->h.r[i]) : G->h.wr[i]);
    for (int j = 0; j < g.Ntheta; ++j) w.push_back(cons ? G->h.wth[j] / G->h.sin_th[j] : G->h.wth[j]);
    for (int k = 0; k < g.NTheta; ++k) w.push_back(cons ? fT[k] / G->h.sinT[k] : fT[k]);
    e = cudaMalloc((void**)&G->balw, w.size() * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpy(G->balw, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(G->wr, G->h.wr.data(), g.Nr * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(G->wth, G->h.wth.data(), g.Ntheta * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    ts_destroy_grid(G);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? fail(TS_ERR_OOM, "device allocation failed")
                                          : cuda_fail(e, "ts_create_grid");
  }
  *out = G;
  return TS_OK;
}

ts_status ts_destroy_grid(ts_grid* g) {
  if (!g) return TS_OK;
  cudaDeviceSynchronize();
  void* ptrs[] = {g->tab64, g->tab32, g->kap, g->eta, g->kaps, g->gR1, g->gR2, g->U, g->K,
                  g->Acc, g->wr, g->wth, g->partN, g->partJ, g->io, g->err, g->tcb16,
                  g->scb, g->scc, g->tcang, g->zt64, g->zt32, g->balw};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : g->adj)
    if (p) cudaFree(p);
  if (g->piw) cudaFree(g->piw);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  if (g->cs_in) cudaStreamDestroy(g->cs_in);
  if (g->cs_out) cudaStreamDestroy(g->cs_out);
  delete g;
  return TS_OK;
}

ts_status ts_grid_nodes(const ts_grid* g, double* r, double* th, double* ph, double* Th,
                        double* Ph) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  if (r) std::memcpy(r, g->h.r.data(), g->h.r.size() * 8);
  if (th) std::memcpy(th, g->h.theta.data(), g->h.theta.size() * 8);
  if (ph) std::memcpy(ph, g->h.phi.data(), g->h.phi.size() * 8);
  if (Th) std::memcpy(Th, g->h.Theta.data(), g->h.Theta.size() * 8);
  if (Ph) std::memcpy(Ph, g->h.Phi.data(), g->h.Phi.size() * 8);
  return TS_OK;
}

ts_status ts_set_coeffs(ts_grid* g, const double* kappa, const double* eta,
                        const double* kappa_s, const void* inflow_R1, const void* inflow_R2,
                        void* stream) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nc = (size_t)g->d.nblk * sizeof(double);
  const size_t ni = (size_t)g->d.G * g->d.Nt * g->d.Np * (g->d.NT / 2) * g->d.NP * g->es;
  const void* src[] = {kappa, eta, kappa_s, inflow_R1, inflow_R2};
  void* dst[] = {g->kap, g->eta, g->kaps, g->gR1, g->gR2};
  const size_t n[] = {nc, nc, nc, ni, ni};
  for (int a = 0; a < 5; ++a) {
    cudaError_t e = src[a] ? cudaMemcpyAsync(dst[a], src[a], n[a], cudaMemcpyDeviceToDevice, st)
                           : cudaMemsetAsync(dst[a], 0, n[a], st);
    if (e != cudaSuccess) return cuda_fail(e, "ts_set_coeffs");
  }
  g->coeffs = true;
  g->hist = false;
  return TS_OK;
}

ts_status ts_reset_history(ts_grid* g) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  g->hist = false;
  return TS_OK;
}

ts_status ts_set_scattering_anisotropy(ts_grid* g, const double* b, void* stream) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  g->hist = false;
  if (!b) {
    g->aniso = false;
    ++g->gen;
    return TS_OK;
  }
  if (g->d.NT < 3 || g->d.NP < 3)
    return fail(TS_ERR_UNSUPPORTED, "anisotropic scattering needs NTheta >= 3 and NPhi >= 3");
  const size_t nc = (size_t)g->d.nblk * sizeof(double);
  if (!g->scb) {
    cudaError_t e = cudaMalloc((void**)&g->scb, nc);
    if (e != cudaSuccess) {
      g->scb = nullptr;
      return cuda_fail(e, "ts_set_scattering_anisotropy");
    }
  }
  cudaError_t e = cudaMemcpyAsync(g->scb, b, nc, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ts_set_scattering_anisotropy");
  g->aniso = true;
  ++g->gen;
  return TS_OK;
}

ts_status ts_set_scattering_quadrupole(ts_grid* g, const double* c, void* stream) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  g->hist = false;
  if (!c) {
    g->quad = false;
    ++g->gen;
    return TS_OK;
  }
  if (g->desc.scheme == TS_RK4_SPLIT_IMPLICIT && (g->d.NT < 6 || g->d.NP < 6))
    return fail(TS_ERR_UNSUPPORTED,
                "the split scheme with a mu^2 term needs NTheta >= 6 and NPhi >= 6");
  const size_t nc = (size_t)g->d.nblk * sizeof(double);
  if (!g->scc) {
    cudaError_t e = cudaMalloc((void**)&g->scc, nc);
    if (e != cudaSuccess) {
      g->scc = nullptr;
      return cuda_fail(e, "ts_set_scattering_quadrupole");
    }
  }
  cudaError_t e = cudaMemcpyAsync(g->scc, c, nc, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ts_set_scattering_quadrupole");
  g->quad = true;
  ++g->gen;
  return TS_OK;
}

ts_status ts_apply_inflow(ts_grid* g, void* F, void* stream) {
  ts_status s = check_F(g, F);
  if (s != TS_OK) return s;
  g->hist = false;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ts::Problem p = make_problem(g);
  cudaError_t e = g->es == 8 ? Launch<double, double>::apply_inflow(p, (double*)F, st)
                             : Launch<float, float>::apply_inflow(p, (float*)F, st);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_apply_inflow");
}

namespace {
// Steps of the device field F; `key` identifies the caller's field for the
// TS_AB2 history (the device pointer, or the host pointer of ts_step_host).
ts_status step_device(ts_grid* g, void* F, double dt, int nsteps, cudaStream_t st,
                      const void* key) {
  if (!std::isfinite(dt) || nsteps < 0) return fail(TS_ERR_ARG, "need finite dt, nsteps >= 0");
  if (!g->coeffs) return fail(TS_ERR_STATE, "ts_set_coeffs has not been called");
  cudaError_t e = g->es == 8 ? run_steps<double, double>(g, g->t64, (double*)F, dt, nsteps, st,
                                                         nullptr, key)
                             : run_steps<float, float>(g, g->t32, (float*)F, dt, nsteps, st,
                                                       nullptr, key);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_step");
}
}  // namespace

ts_status ts_step(ts_grid* g, void* F, double dt, int nsteps, void* stream) {
  ts_status s = check_F(g, F);
  if (s != TS_OK) return s;
  return step_device(g, F, dt, nsteps, static_cast<cudaStream_t>(stream), F);
}

ts_status ts_step_profile(ts_grid* g, void* F, double dt, int nsteps, double* pass_ms,
                          int* launches, void* stream) {
  ts_status s = check_F(g, F);
  if (s != TS_OK) return s;
  if (!std::isfinite(dt) || nsteps < 0) return fail(TS_ERR_ARG, "need finite dt, nsteps >= 0");
  if (!g->coeffs) return fail(TS_ERR_STATE, "ts_set_coeffs has not been called");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Profiler prof{st, {}, {}};
  cudaError_t e = g->es == 8 ? run_steps<double, double>(g, g->t64, (double*)F, dt, nsteps, st, &prof)
                             : run_steps<float, float>(g, g->t32, (float*)F, dt, nsteps, st, &prof);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (pass_ms) for (int a = 0; a < 4; ++a) pass_ms[a] = 0.0;
  if (launches) for (int a = 0; a < 4; ++a) launches[a] = 0;
  if (e == cudaSuccess) prof.collect(pass_ms, launches);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_step_profile");
}

ts_status ts_step_host(ts_grid* g, void* F_host, double dt, int nsteps, void* stream) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  if (!F_host) return fail(TS_ERR_ARG, "field pointer is NULL");
  ts_status s = TS_OK;
  if (!std::isfinite(dt) || nsteps < 0) return fail(TS_ERR_ARG, "need finite dt, nsteps >= 0");
  if (!g->coeffs) return fail(TS_ERR_STATE, "ts_set_coeffs has not been called");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nb = field_bytes(g);
  if (!g->io) {
    cudaError_t e = cudaMalloc(&g->io, nb);
    if (e != cudaSuccess) {
      g->io = nullptr;
      cudaGetLastError();
      return fail(TS_ERR_OOM, "ts_step_host: device buffer allocation failed");
    }
  }
  const int G = g->d.G;
  // Groups per pipelined chunk. Each chunk's step is a separate set of launches,
  // so a chunk costs launch gaps and partial waves; on a GB300 (pinned copies at
  // about 200 GB/s each way) two chunks paid off for the short float steps and
  // none for the double ones, whose step time dwarfs the copies.
  const int cg = g->es == 8 ? G : (G + 1) / 2;
  const int nch = (G + cg - 1) / cg;
  if (g->desc.scheme == TS_AB2 || nch == 1) {
    // one copy each way around the whole step (the AB2 history covers all groups)
    cudaError_t e = cudaMemcpyAsync(g->io, F_host, nb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "ts_step_host (to device)");
    s = step_device(g, g->io, dt, nsteps, st, F_host);
    if (s != TS_OK) return s;
    e = cudaMemcpyAsync(F_host, g->io, nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_step_host (to host)");
  }
  // Groups are independent: group k's steps run on `stream` while group k+1 is
  // copied in on one copy stream and group k-1 copied out on another, so only
  // the first group's copy in and the last group's copy out are exposed.
  cudaError_t e = cudaSuccess;
  if (!g->cs_in) e = cudaStreamCreateWithFlags(&g->cs_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !g->cs_out) e = cudaStreamCreateWithFlags(&g->cs_out, cudaStreamNonBlocking);
  while (e == cudaSuccess && (int)g->ev.size() < 2 * nch + 2) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) g->ev.push_back(ev);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ts_step_host (streams)");
  cudaEvent_t* in_done = g->ev.data();            // [nch]: chunk k is on the device
  cudaEvent_t* step_done = g->ev.data() + nch;    // [nch]: chunk k's steps are done
  cudaEvent_t start = g->ev[2 * nch], out_done = g->ev[2 * nch + 1];
  const size_t gb = (size_t)g->d.S_g * g->es;     // bytes of one group
  char* dev = static_cast<char*>(g->io);
  char* host = static_cast<char*>(F_host);
  // the copies follow the caller's earlier work on `stream`
  e = cudaEventRecord(start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->cs_in, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->cs_out, start, 0);
  for (int k = 0; k < nch && e == cudaSuccess; ++k) {
    const int n = std::min(cg, G - k * cg);
    const size_t off = (size_t)k * cg * gb;
    e = cudaMemcpyAsync(dev + off, host + off, n * gb, cudaMemcpyHostToDevice, g->cs_in);
    if (e == cudaSuccess) e = cudaEventRecord(in_done[k], g->cs_in);
  }
  g->hist = false;
  for (int k = 0; k < nch && e == cudaSuccess; ++k) {
    const int n = std::min(cg, G - k * cg);
    const size_t off = (size_t)k * cg * gb;
    e = cudaStreamWaitEvent(st, in_done[k], 0);
    if (e != cudaSuccess) break;
    g->s0 = k * cg;
    g->sn = n;
    e = g->es == 8 ? run_steps<double, double>(g, g->t64, reinterpret_cast<double*>(dev + off),
                                               dt, nsteps, st)
                   : run_steps<float, float>(g, g->t32, reinterpret_cast<float*>(dev + off), dt,
                                             nsteps, st);
    g->s0 = g->sn = 0;
    if (e == cudaSuccess) e = cudaEventRecord(step_done[k], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->cs_out, step_done[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(host + off, dev + off, n * gb, cudaMemcpyDeviceToHost, g->cs_out);
  }
  g->s0 = g->sn = 0;
  if (e == cudaSuccess) e = cudaEventRecord(out_done, g->cs_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, out_done, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_step_host");
}

ts_status ts_rhs(ts_grid* g, const void* F, void* K, void* stream) {
  ts_status s = check_F(g, F);
  if (s != TS_OK) return s;
  s = check_out(K, "K");
  if (s != TS_OK) return s;
  if (!g->coeffs) return fail(TS_ERR_STATE, "ts_set_coeffs has not been called");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = g->es == 8 ? run_rhs<double, double>(g, g->t64, (const double*)F, (double*)K, false, st)
                             : run_rhs<float, float>(g, g->t32, (const float*)F, (float*)K, false, st);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_rhs");
}

ts_status ts_liouville(ts_grid* g, const void* F, void* LF, void* stream) {
  ts_status s = check_F(g, F);
  if (s != TS_OK) return s;
  s = check_out(LF, "LF");
  if (s != TS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = g->es == 8 ? run_rhs<double, double>(g, g->t64, (const double*)F, (double*)LF, true, st)
                             : run_rhs<float, float>(g, g->t32, (const float*)F, (float*)LF, true, st);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_liouville");
}

ts_status ts_adjoint_step_ab2(ts_grid* g, const void* F_n, void* lambda, void* lambda_prev,
                              double* grad_kappa, double* grad_eta, double dt, int first,
                              void* stream) {
  ts_status s = check_F(g, F_n);
  if (s != TS_OK) return s;
  if (!lambda || !lambda_prev || !grad_kappa || !grad_eta)
    return fail(TS_ERR_ARG, "NULL adjoint argument");
  if (!ts::aligned16(lambda) || !ts::aligned16(lambda_prev))
    return fail(TS_ERR_ARG, "lambda and lambda_prev must be 16-byte aligned");
  if (!std::isfinite(dt)) return fail(TS_ERR_ARG, "dt must be finite");
  if (!g->coeffs) return fail(TS_ERR_STATE, "ts_set_coeffs has not been called");
  if (g->desc.scheme != TS_AB2 || g->desc.filter_on)
    return fail(TS_ERR_UNSUPPORTED, "ts_adjoint_step_ab2 covers the TS_AB2 scheme without filter");
  if (g->desc.radial != TS_RADIAL_CHEBYSHEV || g->desc.form != TS_FORM_ADVECTIVE)
    return fail(TS_ERR_UNSUPPORTED, "adjoint covers the advective form on the Chebyshev radial grid");
  s = adjoint_workspace(g);
  if (s != TS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = g->es == 8
      ? run_adjoint_ab2<double, double>(g, g->t64, (const double*)F_n, (double*)lambda,
                                        (double*)lambda_prev, grad_kappa, grad_eta, dt, first != 0, st)
      : run_adjoint_ab2<float, float>(g, g->t32, (const float*)F_n, (float*)lambda,
                                      (float*)lambda_prev, grad_kappa, grad_eta, dt, first != 0, st);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_adjoint_step_ab2");
}

ts_status ts_set_history(ts_grid* g, const void* F, const void* K_prev, void* stream) {
  ts_status s = check_F(g, F);
  if (s != TS_OK) return s;
  if (!K_prev) return fail(TS_ERR_ARG, "K_prev is NULL");
  if (g->desc.scheme != TS_AB2) return fail(TS_ERR_UNSUPPORTED, "the history belongs to TS_AB2");
  cudaError_t e = cudaMemcpyAsync(g->Acc, K_prev, field_bytes(g), cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ts_set_history");
  g->hist = true;
  g->hist_F = F;
  return TS_OK;
}

ts_status ts_adjoint_step(ts_grid* g, const void* F_n, void* lambda, double* grad_kappa,
                          double* grad_eta, double dt, void* stream) {
  ts_status s = check_F(g, F_n);
  if (s != TS_OK) return s;
  if (!lambda || !grad_kappa || !grad_eta) return fail(TS_ERR_ARG, "NULL adjoint argument");
  if (!ts::aligned16(lambda)) return fail(TS_ERR_ARG, "lambda must be 16-byte aligned");
  if (!std::isfinite(dt)) return fail(TS_ERR_ARG, "dt must be finite");
  if (!g->coeffs) return fail(TS_ERR_STATE, "ts_set_coeffs has not been called");
  if (g->desc.scheme != TS_RK4 || g->desc.filter_on)
    return fail(TS_ERR_UNSUPPORTED, "adjoint covers the TS_RK4 scheme without filter");
  if (g->desc.radial != TS_RADIAL_CHEBYSHEV || g->desc.form != TS_FORM_ADVECTIVE)
    return fail(TS_ERR_UNSUPPORTED, "adjoint covers the advective form on the Chebyshev radial grid");
  s = adjoint_workspace(g);
  if (s != TS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = g->es == 8
      ? run_adjoint<double, double>(g, g->t64, (const double*)F_n, (double*)lambda, grad_kappa, grad_eta, dt, st)
      : run_adjoint<float, float>(g, g->t32, (const float*)F_n, (float*)lambda, grad_kappa, grad_eta, dt, st);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_adjoint_step");
}

ts_status ts_flux_weights(ts_grid* g, double* w, void* stream) {
  if (!g || !w) return fail(TS_ERR_ARG, "NULL argument");
  if (g->desc.form != TS_FORM_ADVECTIVE)
    return fail(TS_ERR_UNSUPPORTED, "ts_flux_weights: advective form only (ts_number_balance)");
  cudaError_t e = cudaMemcpyAsync(w, g->h.fluxw.data(), g->h.fluxw.size() * 8,
                                  cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_flux_weights");
}

ts_status ts_moments(ts_grid* g, const void* F, double* F0, double* F1, double* N, double* JR1,
                     double* JR2, void* stream) {
  ts_status s = check_F(g, F);
  if (s != TS_OK) return s;
  if (g->desc.form != TS_FORM_ADVECTIVE)
    return fail(TS_ERR_UNSUPPORTED, "ts_moments: advective form only (ts_number_balance)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ts::Problem p = make_problem(g);
  cudaError_t e = g->es == 8
      ? Launch<double, double>::moments(p, g->t64, g->wr, g->wth, (const double*)F, F0, F1,
                                        g->partN, g->partJ, N, JR1, JR2, g->desc.R1, g->desc.R2, st)
      : Launch<float, float>::moments(p, g->t64, g->wr, g->wth, (const float*)F, F0, F1,
                                      g->partN, g->partJ, N, JR1, JR2, g->desc.R1, g->desc.R2, st);
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_moments");
}

ts_status ts_number_balance(ts_grid* g, const void* F, double* out, void* stream) {
  ts_status s = check_F(g, F);
  if (s != TS_OK) return s;
  if (!out) return fail(TS_ERR_ARG, "ts_number_balance: out is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ts::Problem p = make_problem(g);
  const bool cons = g->desc.form == TS_FORM_CONSERVATIVE;
  const double rho1 = cons ? 1.0 : g->desc.R1 * g->desc.R1;
  const double rho2 = cons ? 1.0 : g->desc.R2 * g->desc.R2;
  void* K = nullptr;
  double* part = nullptr;   // [nblk][5] block shares, then [G][5] results
  cudaError_t e = cudaMalloc(&K, field_bytes(g));
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&part, ((size_t)g->d.nblk + (size_t)g->d.G) * 5 * sizeof(double));
  if (e == cudaSuccess) {
    double* res = part + (size_t)g->d.nblk * 5;
    if (g->es == 8) {
      double* Kd = static_cast<double*>(K);
      e = stage_passes<double, double>(g, p, g->t64, static_cast<const double*>(F), Kd, -1.0,
                                       true, false, ts::RAD_RHS, nullptr, nullptr, nullptr, Kd,
                                       0.0, st, nullptr);
      if (e == cudaSuccess)
        e = ts::launch_number_balance<double>(p, g->t64, g->balw, cons ? 1 : 0, rho1, rho2,
                                              static_cast<const double*>(F), Kd, part, res, st);
    } else {
      float* Kf = static_cast<float*>(K);
      e = stage_passes<float, float>(g, p, g->t32, static_cast<const float*>(F), Kf, -1.0f, true,
                                     false, ts::RAD_RHS, nullptr, nullptr, nullptr, Kf, 0.0, st,
                                     nullptr);
      if (e == cudaSuccess)
        e = ts::launch_number_balance<float>(p, g->t64, g->balw, cons ? 1 : 0, rho1, rho2,
                                             static_cast<const float*>(F), Kf, part, res, st);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, res, (size_t)g->d.G * 5 * sizeof(double), cudaMemcpyDeviceToHost,
                          st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (K) cudaFree(K);
  if (part) cudaFree(part);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(TS_ERR_OOM, "ts_number_balance: device allocation failed");
  }
  return e == cudaSuccess ? TS_OK : cuda_fail(e, "ts_number_balance");
}

ts_status ts_set_wait_limit(ts_grid* g, long long operand_wait_iterations) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  // 0 restores the default; a negative value makes the wait give up at once
  g->wait_operand = operand_wait_iterations == 0 ? 0
                    : operand_wait_iterations < 0 ? -1 : operand_wait_iterations;
  ++g->gen;
  return TS_OK;
}

ts_status ts_stable_dt(ts_grid* g, const void* x0, int iters, double* rho_host,
                       double* dt_max_host, void* stream) {
  ts_status s = check_F(g, x0);
  if (s != TS_OK) return s;
  if (iters < 2 || iters > 100000) return fail(TS_ERR_ARG, "ts_stable_dt: need 2 <= iters <= 100000");
  if (!g->coeffs) return fail(TS_ERR_STATE, "ts_set_coeffs has not been called");
  if (!g->piw || g->piw_n < iters) {
    if (g->piw) cudaFree(g->piw);
    g->piw = nullptr;
    g->piw_n = 0;
    cudaError_t e = cudaMalloc(&g->piw, (kPiBlocks + 1 + (size_t)iters) * sizeof(double));
    if (e != cudaSuccess) {
      g->piw = nullptr;
      cudaGetLastError();
      return fail(TS_ERR_OOM, "ts_stable_dt: scratch allocation failed");
    }
    g->piw_n = iters;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<double> logs;
  cudaError_t e = g->es == 8
      ? power_iteration<double, double>(g, g->t64, (const double*)x0, iters, logs, st)
      : power_iteration<float, float>(g, g->t32, (const float*)x0, iters, logs, st);
  if (e != cudaSuccess) return cuda_fail(e, "ts_stable_dt");
  double m = 0.0;
  const int h = iters / 2;
  for (int it = h; it < iters; ++it) m += logs[it];
  const double rho = std::exp(m / (iters - h));
  if (!std::isfinite(rho)) return fail(TS_ERR_ARG, "ts_stable_dt: start field gave no finite estimate");
  if (rho_host) *rho_host = rho;
  if (dt_max_host) *dt_max_host = rho > 0.0 ? 2.6 / rho : INFINITY;
  g->hist = false;
  return TS_OK;
}

ts_status ts_sync_status(ts_grid* g, void* stream) {
  if (!g) return fail(TS_ERR_ARG, "grid is NULL");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ts_sync_status");
  int flag = 0;
  e = cudaMemcpy(&flag, g->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "ts_sync_status");
  if (flag) {
    const int zero = 0;
    cudaMemcpy(g->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
    return fail(TS_ERR_TIMEOUT, "a bounded device-side wait ran out; results of that call are invalid");
  }
  return TS_OK;
}

}  // extern "C"
