// Internal declarations of the transport-step library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ts.h"

namespace ts {

// Sets the text that ts_last_error() returns on the calling thread.
void set_last_error(const std::string& msg);

// Sizes and strides of F[g][i][j][l][k][m] (m = Phi fastest).
struct Dims {
  int G, Nr, Nt, Np, NT, NP;
  long long S_l;      // stride of l (phi)      = NT*NP  (one angular block)
  long long S_j;      // stride of j (theta)    = Np*NT*NP
  long long S_i;      // stride of i (r)        = Nt*Np*NT*NP
  long long S_g;      // stride of g (group)    = Nr*S_i
  long long total;    // G*S_g
  long long nblk;     // G*Nr*Nt*Np angular blocks
};

// Device copies of the per-axis tables in the compute type C. Derivative
// matrices are stored TRANSPOSED ([input][output]) so that threads which
// differ in their output index read consecutive addresses.
template <typename C>
struct Tables {
  C *DrT, *AthT, *BthT, *DphT, *AThT, *BThT, *DPhT;   // forward derivative matrices, transposed
  C *Dr, *Ath, *Bth, *Dph, *ATh, *BTh, *DPh;          // the same, untransposed (adjoint = transpose)
  C *inv_r, *inv_sinth, *cot_th, *sin_th, *cos_th, *sin_ph, *cos_ph;
  C *cosT, *sinT, *cosP, *sinP, *tsign, *qdir;
  C *FrT, *FthAT, *FthBT, *FphT, *FThAT, *FThBT, *FPhT;  // filter matrices, transposed
};

// Everything a kernel launch needs about the problem.
struct Problem {
  Dims d;
  int bc;            // ts_bc
  int n_fp64_rows;   // radial rows at each end accumulated in double (float grids)
  const double* kap; // [G][Nr][Nt][Np]
  const double* eta;
  const double* kaps;
  const void* gR1;   // inflow data, element type of the grid
  const void* gR2;
};

// Output mode of the radial pass (the last pass of a stage).
enum RadialMode {
  RAD_RHS = 0,     // write the finished stage derivative K to `out`
  RAD_STAGE0 = 1,  // Acc = K;        U = F + dt/2 K
  RAD_STAGE1 = 2,  // Acc += 2K;      U = F + dt/2 K
  RAD_STAGE2 = 3,  // Acc += 2K;      U = F + dt K
  RAD_STAGE3 = 4   // F = F + dt/6 (Acc + K)
};

template <typename T, typename C>
struct Launch {
  // K = sgn*(a_Th dTh U + a_Ph dPh U) [+ eta - (kappa+kappa_s) U + kappa_s J(U)]
  static cudaError_t angular(const Problem& p, const Tables<C>& t, const T* U, T* K, C sgn,
                             bool collision, cudaStream_t s);
  // K += sgn*(a_th dth U + a_ph dph U)
  static cudaError_t plane(const Problem& p, const Tables<C>& t, const T* U, T* K, C sgn,
                           cudaStream_t s);
  // K += sgn*a_r dr U; Tau rows (if tau); then the output selected by mode
  static cudaError_t radial(const Problem& p, const Tables<C>& t, const double* Dr64,
                            const T* U, const T* K, C sgn, bool tau, int mode, T* F, T* Acc,
                            T* Uout, T* out, double dt, cudaStream_t s);
  // adjoint passes (transposes of the three forward passes)
  static cudaError_t radial_T(const Problem& p, const Tables<C>& t, const T* X, double scale,
                              bool tau, T* lt, T* Ubar, cudaStream_t s);
  static cudaError_t plane_T(const Problem& p, const Tables<C>& t, const T* lt, T* Ubar,
                             cudaStream_t s);
  static cudaError_t angular_T(const Problem& p, const Tables<C>& t, const T* lt,
                               const T* Ubar, const T* Us, double* gk, double* ge,
                               const T* lam, const T* lam_in, T* lam_out, T* Kbar_out,
                               double wl, double wu, cudaStream_t s);
  // split scheme, inflow data, filter, moments
  static cudaError_t implicit_collision(const Problem& p, const Tables<C>& t, T* F, double dt,
                                        cudaStream_t s);
  static cudaError_t apply_inflow(const Problem& p, T* F, cudaStream_t s);
  static cudaError_t filter(const Problem& p, const Tables<C>& t, T* F, T* tmp,
                            cudaStream_t s);
  static cudaError_t moments(const Problem& p, const Tables<double>& t64, const double* wr,
                             const double* wth, const T* F, double* F0, double* F1,
                             double* partN, double* partJ, double* N, double* JR1,
                             double* JR2, double R1, double R2, cudaStream_t s);
};

}  // namespace ts
