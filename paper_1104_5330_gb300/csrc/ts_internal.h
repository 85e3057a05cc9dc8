// Internal declarations of the transport-step library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ts.h"

namespace ts {

// Exact widening of a float to a double by the IEEE-754 binary32 and binary64
// layouts (sign kept, exponent rebiased by 1023 - 127 = 896, significand shifted
// up by 52 - 23 = 29 bits), on the integer units; zero maps to zero, and the rare
// subnormal, infinite or NaN inputs take the conversion instruction. Used where
// the FP64 pipe, not the integer units, bounds a pass.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (e == 0xFFu || (e == 0u && m != 0u)) return (double)f;
  const uint64_t mag = e ? ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29) : 0ull;
  return __longlong_as_double((long long)(((uint64_t)(u >> 31) << 63) | mag));
}

// Device fields are read and written with 16-byte vector accesses and
// 16-byte asynchronous copies: the entry points require 16-byte alignment.
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }


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
  // Even/odd forms used by the register-blocked passes:
  //  DFS axes: P = (A + B)/2 acts on F + F(partner), Q = (A - B)/2 on F - F(partner),
  //  stored [in][out]; radial: the centro-antisymmetric D_r folded onto h = Nr/2
  //  output pairs (i, N-i): EpT[i'][i] = D[i][i'] + D[i][N-i'], OpT[i'][i] =
  //  D[i][i'] - D[i][N-i'], DrMc[i] = D[i][N/2], DrMr[i'] = D[N/2][i'] (odd Nr).
  C *PthT, *QthT, *PThT, *QThT, *EpT, *OpT, *DrMc, *DrMr;
  // The same for the transposed matrices (adjoint passes): PthA[j][j'] =
  // (A+B)[j][j']/2, QthA = (A-B)/2 ([in][out] of the transpose), Theta alike;
  // EpTa, OpTa, DrMca, DrMra from D_r^T (also centro-antisymmetric).
  C *PthA, *QthA, *PThA, *QThA, *EpTa, *OpTa, *DrMca, *DrMra;
  // Fourier derivative on the halves of a DFS pair: for s(p) = u(p) + u(p+N/2),
  // d(p) = u(p) - u(p+N/2), p < N/2, the circulant D gives
  //   (D u)(p) = (Ms s + Md d)(p) / 2,  (D u)(p + N/2) = (Ms s - Md d)(p) / 2,
  // Ms[p][p'] = D[p][p'] + D[p][p'+N/2], Md[p][p'] = D[p][p'] - D[p][p'+N/2]:
  // half the multiply-adds of D. Stored [p'][p] (MsPhT, MdPhT for Phi; MsphT,
  // MdphT for phi).
  C *MsPhT, *MdPhT, *MsphT, *MdphT;
  // P and Q of the DFS Theta (and theta) circles are centro-antisymmetric (the
  // nodes are symmetric about pi/2 and the derivative is odd): folded onto
  // n/2 output pairs (k, n-1-k) like D_r, PeT[k'][k] = P[k][k'] + P[k][n-1-k'],
  // PoT[k'][k] = P[k][k'] - P[k][n-1-k'] (k, k' < n/2), Q alike.
  C *PeThT, *PoThT, *QeThT, *QoThT, *PethT, *PothT, *QethT, *QothT;
  // The same foldings of the transposed operators (adjoint passes): P^T, Q^T
  // folded over k -> n-1-k, and D^T (circulant too) on the pair halves.
  C *PeThA, *PoThA, *QeThA, *QoThA, *PethA, *PothA, *QethA, *QothA;
  C *MsPhA, *MdPhA, *MsphA, *MdphA;
  // D_r split into TF32 high and low halves in the tensor-core operand layout
  // (N_r padded to 16 rows x N_r padded to 8 columns, 8 x 4 core matrices).
  C *TcBhi, *TcBlo;
};

// Tile shapes of the passes; 0 selects the built-in heuristic.
//   nb: angular blocks per CTA; c: Phi column pairs per plane tile; W: columns
//   per radial tile. The *T fields are the same for the adjoint passes.
struct TileParams {
  int nb = 0, c = 0, W = 0, nbT = 0, cT = 0, WT = 0;
  // Bit mask of forward passes that use the register-blocked even/odd form
  // (1 angular, 2 plane, 4 radial); set from the grid's sizes.
  int rb = 0;
  // Fused angular + radial pass (float grids whose tile fits shared memory):
  // angular blocks per chunk and U staging buffers; fnb = 0: three passes.
  int fnb = 0, fnbuf = 0;
};

// Output rows per thread of the register-blocked passes: angular 2 in float and
// 1 in double (each with its Theta mirror rows), radial 2 (row pairs), plane 2.
constexpr int kRBPlane = 2;
__host__ __device__ constexpr int rb_ang(int elem_bytes) { return elem_bytes == 4 ? 2 : 1; }
__host__ __device__ constexpr int rb_rad(int elem_bytes) { return elem_bytes == 4 ? 2 : 2; }

// Per-block scalars of the angular passes. Register-blocked form: J, kappa,
// eta, kappa_s, 1/r, cot(theta), kappa_s b, H_r, H_theta, H_phi, kappa_s c,
// M_rr, M_thth, M_phph, M_thph, M_rth, M_rph (H, M: the first and second
// angular moments in the local frame e_r, e_theta, e_phi); run-time form: J, H
// and M; adjoint form: the same sums of lt plus kappa_s c sum lt.
constexpr int kAngScalars = 17;
constexpr int kAngMoments = 11;

// Forms of the angular pass by scattering kernel: isotropic, with the mu term,
// with the mu and mu^2 terms.
enum KernelForm { KF_ISO = 0, KF_LINEAR = 1, KF_QUADRATIC = 2 };

// Which forward passes of a grid can use the register-blocked even/odd form.
inline int rb_mask(const Dims& d, int elem_bytes, int n64) {
  int m = 0;
  if (d.NT % (2 * rb_ang(elem_bytes)) == 0 && d.NP % 8 == 0) m |= 1;
  if (d.Nt % kRBPlane == 0 && d.Np % 2 == 0 && d.NP % 8 == 0) m |= 2;
  if (d.Nr >= 9 && (d.Nr / 2) % rb_rad(elem_bytes) == 0 && (d.NT * d.NP) % 4 == 0 && n64 <= 2)
    m |= 4;
  return m;
}

// Everything a kernel launch needs about the problem.
struct Problem {
  Dims d;
  TileParams tp;
  int bc;            // ts_bc
  int n_fp64_rows;   // radial rows at each end accumulated in double (float grids)
  const double* kap; // [G][Nr][Nt][Np]
  const double* eta;
  const double* kaps;
  const double* scb; // b and c of the scattering kernel (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3)),
  const double* scc; // mu = omega.omega', [G][Nr][Nt][Np] each; NULL: that term is zero
  const void* gR1;   // inflow data, element type of the grid
  const void* gR2;
  int tc;            // TcKind: radial pass on the tensor cores (float grids)
  const void* tcb16; // BF16x3: the three bf16 terms of D_r in the MMA's B layout
  int* err;          // device flag set by a bounded wait that ran out
  long long wait_operand;  // bound (iterations) of the tensor-core pass's operand wait
  int plane_store;         // 1: the plane pass writes K = its terms (fused stages), 0: adds
  // D_r folded onto the row pairs (i, N-i) in double ([ii][i], see Tables::EpT) and
  // its middle column: the double-precision end rows of float grids
  const double *ep64, *op64, *mc64;
  // TS_TF32X3 with 16 x 16 direction blocks: the Theta (DFS pair, K = 32) and Phi
  // (K = 16) derivative matrices split into TF32 hi + lo in the tensor-core B
  // layout (W1 hi, W1 lo, W2 hi, W2 lo); NULL: the angular pass runs on the SIMT units
  const float* tcang;
};

__host__ __device__ inline int kernel_form(const Problem& p, int collision) {
  if (!collision) return KF_ISO;
  return p.scc ? KF_QUADRATIC : p.scb ? KF_LINEAR : KF_ISO;
}

// Default bound (spin iterations) of the device-side waits of the tensor-core
// radial pass.
constexpr long long kDefaultWaitIters = 1LL << 24;

// Operand forms of the tensor-core radial pass.
enum TcKind { TC_NONE = 0, TC_TF32X3 = 1, TC_BF16X3 = 2 };

// Radial pass on the tensor cores (float grids; defined with the float kernels).
cudaError_t launch_radial_tc(const Problem& p, const Tables<float>& t, const float* U,
                             const float* K, float sgn, bool tau, int mode, float* F, float* Acc,
                             float* Uout, float* out, double dt, cudaStream_t s);
// Fused angular + radial pass of a stage (float grids; defined with the float
// kernels in ts_f32.cu). fused_plan picks the chunk and staging-buffer counts
// that fit shared memory (returns false if none does); launch_fused runs the
// pass on the plane terms the plane pass wrote into Kp.
bool fused_plan(const Dims& d, int n64, int* nb, int* nbuf);
cudaError_t launch_fused(const Problem& p, const Tables<float>& t, const double* Dr64,
                         const float* U, const float* Kp, float sgn, bool collision, bool tau,
                         int mode, float* F, float* Acc, float* Uout, float* out, double dt,
                         cudaStream_t s);
// Angular pass on the tensor cores (TS_TF32X3, 16 x 16 direction blocks, isotropic
// kernel; defined with the float kernels).
cudaError_t launch_angular_tc(const Problem& p, const Tables<float>& t, const float* U, float* K,
                              float sgn, bool collision, cudaStream_t s);
// Radial pass of the hybrid grid (uniform r nodes, one-sided upwind differences;
// `hold`: zero rate at the inflow nodes). Defined in ts_fd.cu.
template <typename T, typename C>
cudaError_t launch_radial_fd(const Problem& p, const Tables<C>& t, const T* U, const T* K, C sgn,
                             bool hold, int mode, T* F, T* Acc, T* Uout, T* out, double dt,
                             double dr, cudaStream_t s);

// Radial pass of the three-zone grid (App. B; defined in ts_zoned.cu): ZT the
// central zone's folded differentiation tables [Ep H*H | Op H*H | Dm H | Mr H |
// T_N on its nB nodes] (H = nB/2), nA nodes per edge zone, h the edge-zone
// spacing.
template <typename T, typename C>
cudaError_t launch_radial_zoned(const Problem& p, const Tables<C>& t, const C* ZT, int nA, int nB,
                                double h, const T* U, const T* K, C sgn, bool hold, int mode,
                                T* F, T* Acc, T* Uout, T* out, double dt, cudaStream_t s);

// The conservative form of App. A (defined in ts_cons5d.cu): the angular pass on
// Fhat = r^2 sin th sin Th F (the grid's Theta tables are those of the odd
// continuation), in the grid's element type; the number balance of a grid's
// operator, w = [radial | theta | Theta] weights of the state's number integral,
// cons: the source term carries the volume element, part: nblk x 5 doubles, out:
// G x 5 doubles (N, J_R1, J_R2, dN/dt, S).
template <typename T>
cudaError_t launch_angular_cons(const Problem& p, const Tables<T>& t, const T* U, T* K, T sgn,
                                bool collision, cudaStream_t s);
template <typename T>
cudaError_t launch_number_balance(const Problem& p, const Tables<double>& t, const double* w,
                                  int cons, double rho1, double rho2, const T* F, const T* K,
                                  double* part, double* out, cudaStream_t s);

// Whether the tensor-core radial pass handles N_r (its tile must fit shared memory).
inline bool tc_supported(int Nr) { return Nr >= 3 && Nr <= 81; }

// Output mode of the radial pass (the last pass of a stage).
enum RadialMode {
  RAD_RHS = 0,     // write the finished stage derivative K to `out`
  RAD_STAGE0 = 1,  // Acc = K;        U = F + dt/2 K
  RAD_STAGE1 = 2,  // Acc += 2K;      U = F + dt/2 K
  RAD_STAGE2 = 3,  // Acc += 2K;      U = F + dt K
  RAD_STAGE3 = 4,  // F = F + dt/6 (Acc + K)
  RAD_AB2 = 5,     // F = F + dt (3/2 K - 1/2 Acc);  Acc = K   (Acc: K of the previous step)
  RAD_AB2_START = 6  // F = F + dt K;  Acc = K
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

typedef std::vector<double> Vec;

// Host copies of the per-axis tables (derivative matrices [out][in]).
struct HostTables {
  Vec r, theta, phi, Theta, Phi;
  Vec Dr, Ath, Bth, Dph, ATh, BTh, DPh;          // [out][in]
  Vec Fr, FthA, FthB, Fph, FThA, FThB, FPh;      // filter [out][in]
  Vec inv_r, inv_sinth, cot_th, sin_th, cos_th, sin_ph, cos_ph;
  Vec cosT, sinT, cosP, sinP, tsign, qdir;
  Vec wr, wth, fluxw;
  Vec PthT, QthT, PThT, QThT, EpT, OpT, DrMc, DrMr;   // even/odd forms (see Tables)
  Vec PthA, QthA, PThA, QThA, EpTa, OpTa, DrMca, DrMra;  // even/odd forms of the transposes
  Vec MsPhT, MdPhT, MsphT, MdphT;                     // pair-half Fourier derivatives
  Vec PeThT, PoThT, QeThT, QoThT, PethT, PothT, QethT, QothT;   // folded P, Q
  Vec PeThA, PoThA, QeThA, QoThA, PethA, PothA, QethA, QothA;   // folded P^T, Q^T
  Vec MsPhA, MdPhA, MsphA, MdphA;                                // D^T on pair halves
  Vec TcBhi, TcBlo;                                   // tensor-core operand of D_r
};

ts_status fail_status(ts_status s, const std::string& msg);

// Host tables shared by the grid types (closed forms, see ts_api.cu):
// Chebyshev-Gauss-Lobatto differentiation matrix on [R1, R2] ([out][in]); the
// periodic Fourier derivative on M equispaced nodes of a 2 pi circle (Nyquist
// zeroed); Fejer's first rule for int_0^pi g(t) sin t dt on pi (k+1/2)/N;
// Clenshaw-Curtis weights for int_{-1}^{1} on the Nr Gauss-Lobatto nodes.
Vec cheb_diff_matrix(int Nr, double R1, double R2);
Vec fourier_diff_matrix(int M);
Vec fejer_weights(int N);
Vec clenshaw_curtis_weights(int Nr);
ts_status cuda_status(cudaError_t e, const char* where);

}  // namespace ts

// The grid behind the opaque ts_grid handle of include/ts.h.
struct ts_grid {
  ts_grid_desc desc;
  ts::Dims d;
  size_t es = 8;
  ts::HostTables h;
  void* tab64 = nullptr;
  void* tab32 = nullptr;
  ts::Tables<double> t64{};
  ts::Tables<float> t32{};
  double *kap = nullptr, *eta = nullptr, *kaps = nullptr;
  void *gR1 = nullptr, *gR2 = nullptr;
  bool coeffs = false;
  void *U = nullptr, *K = nullptr, *Acc = nullptr;
  void* adj[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double *wr = nullptr, *wth = nullptr, *partN = nullptr, *partJ = nullptr;
  double* piw = nullptr;  // power iteration: partial sums, norms and their logs (ts_stable_dt)
  int piw_n = 0;
  int* err = nullptr;    // device flag: a bounded device-side wait ran out
  void* io = nullptr;
  ts::TileParams tp{};   // tile shapes (0 = built-in heuristic); set by ts_autotune
  void* tcb16 = nullptr; // TS_BF16X3: bf16 terms of D_r (tensor-core B operand)
  double* scb = nullptr; // b of the scattering kernel (ts_set_scattering_anisotropy)
  bool aniso = false;    // scb holds values in use
  double* scc = nullptr; // c of the scattering kernel (ts_set_scattering_quadrupole)
  bool quad = false;     // scc holds values in use
  unsigned gen = 0;      // bumped when the launch parameters change (batched steps re-upload)
  bool hist = false;     // TS_AB2: Acc holds K of the previous step of hist_F
  const void* hist_F = nullptr;
  long long wait_operand = 0;  // 0: the default bound (ts_set_wait_limit)
  float* tcang = nullptr;      // angular tensor-core operand terms (Problem::tcang)
  // TS_RADIAL_ZONED: the central zone's folded differentiation tables and T_N on
  // its nodes, in double (zt64) and, for float grids, in float (zt32)
  void *zt64 = nullptr, *zt32 = nullptr;
  int zA = 0, zB = 0;          // nodes per edge zone, nodes of the central zone
  // weights of the state's number integral (ts_number_balance): radial [Nr] |
  // theta [Ntheta] | Theta [NTheta], device doubles
  double* balw = nullptr;
  double zh = 0.0;             // edge-zone node spacing
  // Group slice the launches cover (ts_step_host's per-group pipeline): groups
  // s0 .. s0+sn-1, every pointer of the problem and the workspace offset to
  // group s0; sn = 0: all groups.
  int s0 = 0, sn = 0;
  // Copy streams and per-group events of the pipelined ts_step_host.
  cudaStream_t cs_in = nullptr, cs_out = nullptr;
  std::vector<cudaEvent_t> ev;
};

namespace ts {
Problem problem_of(const ts_grid* g);
// nsteps steps of the device field F on `st` by the grid's own single-problem
// passes (the compiled line-length forms where the sizes have them); kernel
// launches only, so a stream capture can record them.
cudaError_t step_grid(ts_grid* g, void* F, double dt, int nsteps, cudaStream_t st);
// One TS_AB2 step of F by the grid's own passes with the history taken as given:
// forward Euler when `first`, else F + dt (3/2 K_n - 1/2 K_{n-1}) with K_{n-1} in
// the grid's Acc (kernel launches only, for a stream capture); and the record
// that the grid's Acc now holds the history of F.
cudaError_t step_grid_ab2(ts_grid* g, void* F, double dt, bool first, cudaStream_t st);
void set_ab2_history(ts_grid* g, const void* F);
}  // namespace ts
