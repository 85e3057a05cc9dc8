// Launch configuration of the transport-step kernels (tile sizes per pass).
#pragma once

#include <algorithm>

#include "ts_kernels_rb.cuh"

namespace ts {

// Shared-memory budget per CTA used when choosing tile sizes; kernels opt in
// to the full 227 KB once so that large grids still fit one tile.
constexpr size_t kSmemBudget = 96 * 1024;
constexpr size_t kSmemMax = 227 * 1024;

// Opt a kernel in to the largest dynamic shared memory the SM allows next to
// the kernel's own static shared memory.
template <typename K>
static cudaError_t allow_smem(K kernel) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(kSmemMax - a.sharedSizeBytes));
}

static inline unsigned grid1(long long n) { return (unsigned)n; }

// Shared memory of one tile of each forward pass (rb: register-blocked form).
// The register-blocked forms also hold the even/odd sums and differences, and
// the angular one a transposed copy of its blocks.
template <typename C>
size_t smem_angular(const Dims& d, int nb, bool rb) {
  const size_t S = (size_t)d.NT * d.NP, mats = 2 * d.NT * d.NT + d.NP * d.NP;
  if (!rb) return (mats + nb * S + (size_t)kAngMoments * nb) * sizeof(C);
  return (mats + nb * (S + (size_t)ang_ss(d.NT, d.NP) + ang_us<C>(d.NT, d.NP)) +
          (size_t)kAngScalars * nb) *
         sizeof(C);
}
template <typename C>
size_t smem_plane(const Dims& d, int c, bool rb) {
  return (size_t)(2 * d.Nt * d.Nt + d.Np * d.Np + (rb ? 2 : 1) * d.Nt * d.Np * 2 * c) * sizeof(C);
}
template <typename C>
size_t smem_radial(const Dims& d, int W, bool rb) {
  if (!rb) return (size_t)(d.Nr * d.Nr + 2 * d.Nr * W) * sizeof(C);
  const int hh = d.Nr / 2;   // E, O, middle row, K rows 0 and N, up to 4 double-precision rows
  return (size_t)(2 * ((hh * hh + 3) & ~3) + 2 * ((hh + 3) & ~3) + (2 * hh + 7) * W) * sizeof(C);
}

// Persistent forms. The angular one stages the next tile into its single
// staging buffer once the current tile is prepared; the plane one keeps two
// staging buffers.
template <typename C>
size_t smem_angular_pp(const Dims& d, int nb) {
  return smem_angular<C>(d, nb, true);
}
template <typename C>
size_t smem_plane_pp(const Dims& d, int c) {
  return smem_plane<C>(d, c, true) + (size_t)d.Nt * d.Np * 2 * c * sizeof(C);
}

// CTAs of a persistent kernel: as many as fit on the GPU at this shared-memory size.
template <typename K>
static int persistent_ctas(K kernel, size_t smem, long long ntiles) {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  return (int)std::max<long long>(1, std::min<long long>(ntiles, (long long)occ * nsm));
}

// Two CTAs of the persistent kernels share an SM when each stays below this.
constexpr size_t kSmemHalf = 113 * 1024;   // 228 KB per SM, 1 KB reserved per CTA

// Built-in tile shapes: fill 256 threads with work while staying in the budget
// (two CTAs per SM for the persistent register-blocked forms).
template <typename T, typename C>
static int angular_nb(const Dims& d, int ntiles, bool rb = false) {
  const int S = d.NT * d.NP;
  if (rb && ntiles == 1) {
    // threads' units per block: RB rows with their mirrors, 4 column pairs
    const int per = (d.NT / 2 / rb_ang((int)sizeof(C))) * (d.NP / 8);
    int nb = std::max(1, (kThreads + per - 1) / per);
    while (nb > 1 && smem_angular<C>(d, nb, true) > kSmemHalf) --nb;
    // The persistent CTAs (two per SM) take tiles in turn: the busiest one runs
    // ceil(tiles / CTAs) rounds. Down to 3/4 of the largest tile, take the
    // smallest block count that needs no more rounds (the same number of rounds
    // with less staging and preparation each, the last round fuller).
    static int nsm = 0;
    if (!nsm) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (nsm < 1) nsm = 1;
    }
    const long long ctas = 2LL * nsm;
    auto rounds = [&](int b) { return ((d.nblk + b - 1) / b + ctas - 1) / ctas; };
    const long long r0 = rounds(nb);
    int best = nb;
    for (int b = nb - 1; b >= std::max(1, 3 * nb / 4); --b)
      if (rounds(b) == r0) best = b;
    return best;
  }
  int nb = std::max(1, 2048 / S);
  const size_t mats = (size_t)(2 * d.NT * d.NT + d.NP * d.NP) * sizeof(C);
  while (nb > 1 && mats + (size_t)nb * (ntiles * S + 4) * sizeof(C) > kSmemBudget) nb /= 2;
  return nb;
}

template <typename T, typename C>
static int plane_c(const Dims& d, int ntiles, bool rb = false) {
  const int hP = d.NP / 2;
  const size_t mats = (size_t)(2 * d.Nt * d.Nt + d.Np * d.Np) * sizeof(C);
  int best = rb ? 4 : 1;
  const int tiles = rb ? 3 * ntiles : ntiles;   // rb: two staging buffers + sums/diffs
  const size_t budget = rb ? kSmemHalf : kSmemBudget;
  for (int c = 1; c <= hP; ++c) {
    if (hP % c || (rb && c % 4)) continue;
    if (mats + (size_t)tiles * d.Nt * d.Np * 2 * c * sizeof(C) <= budget) best = c;
  }
  return best;
}

template <typename T, typename C>
static int radial_W(const Dims& d, int ntiles, bool rb = false) {
  const int S = d.NT * d.NP;
  int W;
  if (rb) {   // about one unit (RB row pairs x 4 columns) per thread
    const int hh = d.Nr / 2;
    W = std::max(4, std::min(S, (4 * kThreads * rb_rad((int)sizeof(C)) / std::max(1, hh)) & ~3));
    while (W > 4 && smem_radial<C>(d, W, true) > kSmemHalf) W = (W / 2) & ~3;
    return std::max(4, W);
  }
  W = std::min(S, sizeof(C) == 8 ? 64 : 128);
  while (W > 8 && (size_t)(d.Nr * d.Nr + ntiles * d.Nr * W) * sizeof(C) > kSmemBudget) W /= 2;
  return W;
}

// Launches with the line lengths fixed at compile time for the common grids
// (16, 24, 32 angular nodes -- also 8, and whole Phi rows per tile, in the
// plane pass; 17, 33, 65 radial nodes), and the run-time form (template
// argument 0) for every other size.

template <typename T, typename C, int A, int B, int KF>
static cudaError_t angular_pp_form(const Problem& p, const Tables<C>& t, const T* U, T* K, C sgn,
                                   int collision, int nb, long long ntiles, cudaStream_t s) {
  static const cudaError_t e = allow_smem(k_angular_pp<T, C, A, B, KF>);  // once per kernel
  if (e != cudaSuccess) return e;
  const size_t smem = smem_angular_pp<C>(p.d, nb);
  const int ctas = persistent_ctas(k_angular_pp<T, C, A, B, KF>, smem, ntiles);
  k_angular_pp<T, C, A, B, KF><<<ctas, kThreads, smem, s>>>(p, t, U, K, sgn, collision, nb,
                                                            ntiles);
  return cudaGetLastError();
}
template <typename T, typename C, int A, int B>
static cudaError_t angular_pp(const Problem& p, const Tables<C>& t, const T* U, T* K, C sgn,
                              int collision, int nb, long long ntiles, cudaStream_t s) {
  switch (kernel_form(p, collision)) {
    case KF_QUADRATIC:
      return angular_pp_form<T, C, A, B, KF_QUADRATIC>(p, t, U, K, sgn, collision, nb, ntiles, s);
    case KF_LINEAR:
      return angular_pp_form<T, C, A, B, KF_LINEAR>(p, t, U, K, sgn, collision, nb, ntiles, s);
    default:
      return angular_pp_form<T, C, A, B, KF_ISO>(p, t, U, K, sgn, collision, nb, ntiles, s);
  }
}

template <typename T, typename C, int N>
static cudaError_t plane_pp(const Problem& p, const Tables<C>& t, const T* U, T* K, C sgn, int c,
                            long long ntiles, cudaStream_t s) {
  static const cudaError_t e = allow_smem(k_plane_pp<T, C, N>);  // once per kernel
  if (e != cudaSuccess) return e;
  const size_t smem = smem_plane_pp<C>(p.d, c);
  const int ctas = persistent_ctas(k_plane_pp<T, C, N>, smem, ntiles);
  k_plane_pp<T, C, N><<<ctas, kThreads, smem, s>>>(p, t, U, K, sgn, c, ntiles);
  return cudaGetLastError();
}

template <typename T, typename C, int R>
static cudaError_t radial_eo(const Problem& p, const Tables<C>& t, const double* Dr64,
                             const T* U, const T* K, C sgn, int tau, int mode, T* F, T* Acc,
                             T* Uout, T* out, C dt, int W, long long ntiles, cudaStream_t s) {
  static const cudaError_t e = allow_smem(k_radial_eo<T, C, R>);  // once per kernel
  if (e != cudaSuccess) return e;
  const size_t smem = smem_radial<C>(p.d, W, true);
  k_radial_eo<T, C, R><<<grid1(ntiles), kThreads, smem, s>>>(p, t, Dr64, U, K, sgn, tau, mode, F,
                                                             Acc, Uout, out, dt, W);
  return cudaGetLastError();
}

template <typename T, typename C, int N, int KT>
static cudaError_t plane_sq(const Problem& p, const Tables<C>& t, const T* U, T* K, C sgn,
                            cudaStream_t s) {
  static const cudaError_t e = allow_smem(k_plane_sq<T, C, N, KT>);  // once per kernel
  if (e != cudaSuccess) return e;
  const size_t smem = smem_plane_sq<N, KT, C>();
  const long long ntiles = (long long)p.d.G * p.d.Nr * (N / KT);
  const int ctas = persistent_ctas(k_plane_sq<T, C, N, KT>, smem, ntiles);
  k_plane_sq<T, C, N, KT><<<ctas, kThreads, smem, s>>>(p, t, U, K, sgn, ntiles);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::angular(const Problem& p, const Tables<C>& t, const T* U, T* K, C sgn,
                                  bool collision, cudaStream_t s) {
  const Dims& d = p.d;
  if constexpr (sizeof(T) == 4) {
    if (p.tcang && d.NT == 16 && d.NP == 16 && kernel_form(p, collision ? 1 : 0) == KF_ISO)
      return launch_angular_tc(p, t, U, K, sgn, collision, s);
  }
  const bool rb = p.tp.rb & 1;
  const int nb = p.tp.nb > 0 ? p.tp.nb : angular_nb<T, C>(d, 1, rb);
  const long long ntiles = (d.nblk + nb - 1) / nb;
  const int col = collision ? 1 : 0;
  if (rb) {
    switch (ang_spec(d)) {
      case 16: return angular_pp<T, C, 16, 16>(p, t, U, K, sgn, col, nb, ntiles, s);
      case 24: return angular_pp<T, C, 24, 24>(p, t, U, K, sgn, col, nb, ntiles, s);
      case 32: return angular_pp<T, C, 32, 32>(p, t, U, K, sgn, col, nb, ntiles, s);
      case 2416: return angular_pp<T, C, 24, 16>(p, t, U, K, sgn, col, nb, ntiles, s);
      default: return angular_pp<T, C, 0, 0>(p, t, U, K, sgn, col, nb, ntiles, s);
    }
  }
  static const cudaError_t e = allow_smem(k_angular<T, C>);  // once per kernel
  if (e != cudaSuccess) return e;
  const size_t smem = smem_angular<C>(d, nb, rb);
  k_angular<T, C><<<grid1(ntiles), kThreads, smem, s>>>(p, t, U, K, sgn, col, nb);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::plane(const Problem& p, const Tables<C>& t, const T* U, T* K, C sgn,
                                cudaStream_t s) {
  const Dims& d = p.d;
  const bool rb = p.tp.rb & 2;
  const int c = p.tp.c > 0 ? p.tp.c : plane_c<T, C>(d, 1, rb);
  const long long nct = (long long)d.G * d.Nr * d.NT * (d.NP / 2 / c);
  if (rb) {
    switch (plane_spec(d, c)) {
      case 8: return plane_pp<T, C, 8>(p, t, U, K, sgn, c, nct, s);
      case 16:
        // two Theta values per tile in float (RB 2), one in double (RB 1): 256 units
        if constexpr (sizeof(C) == 4) return plane_sq<T, C, 16, 2>(p, t, U, K, sgn, s);
        else return plane_sq<T, C, 16, 1>(p, t, U, K, sgn, s);
      case 24: return plane_pp<T, C, 24>(p, t, U, K, sgn, c, nct, s);
      case 32: return plane_pp<T, C, 32>(p, t, U, K, sgn, c, nct, s);
      default: return plane_pp<T, C, 0>(p, t, U, K, sgn, c, nct, s);
    }
  }
  static const cudaError_t e = allow_smem(k_plane<T, C>);  // once per kernel
  if (e != cudaSuccess) return e;
  const size_t smem = smem_plane<C>(d, c, rb);
  k_plane<T, C><<<grid1(nct), kThreads, smem, s>>>(p, t, U, K, sgn, c);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::radial(const Problem& p, const Tables<C>& t, const double* Dr64,
                                 const T* U, const T* K, C sgn, bool tau, int mode, T* F, T* Acc,
                                 T* Uout, T* out, double dt, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (p.tc)
      return launch_radial_tc(p, t, U, K, sgn, tau, mode, F, Acc, Uout, out, dt, s);
  }
  const Dims& d = p.d;
  const bool rb = p.tp.rb & 4;
  int W = p.tp.W > 0 ? p.tp.W : radial_W<T, C>(d, 2, rb);
  // the double-precision end rows are computed by 4 threads per 4 columns before
  // the tile's barrier: twice the columns keep every thread of the CTA busy there
  if (rb && p.n_fp64_rows > 0 && p.tp.W <= 0 && 2 * W <= d.NT * d.NP &&
      smem_radial<C>(d, 2 * W, true) <= kSmemHalf)
    W *= 2;
  const int S = d.NT * d.NP;
  const long long nct = (long long)d.G * d.Nt * d.Np * ((S + W - 1) / W);
  const int ta = tau ? 1 : 0;
  if (rb) {
    switch (rad_spec(d)) {
      case 17: return radial_eo<T, C, 17>(p, t, Dr64, U, K, sgn, ta, mode, F, Acc, Uout, out, (C)dt, W, nct, s);
      case 33: return radial_eo<T, C, 33>(p, t, Dr64, U, K, sgn, ta, mode, F, Acc, Uout, out, (C)dt, W, nct, s);
      case 65: return radial_eo<T, C, 65>(p, t, Dr64, U, K, sgn, ta, mode, F, Acc, Uout, out, (C)dt, W, nct, s);
      default: return radial_eo<T, C, 0>(p, t, Dr64, U, K, sgn, ta, mode, F, Acc, Uout, out, (C)dt, W, nct, s);
    }
  }
  static const cudaError_t e = allow_smem(k_radial<T, C>);  // once per kernel
  if (e != cudaSuccess) return e;
  const size_t smem = smem_radial<C>(d, W, rb);
  k_radial<T, C><<<grid1(nct), kThreads, smem, s>>>(p, t, Dr64, U, K, sgn, ta, mode, F, Acc, Uout,
                                                    out, (C)dt, W);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::radial_T(const Problem& p, const Tables<C>& t, const T* X,
                                   double scale, bool tau, T* lt, T* Ubar, cudaStream_t s) {
  static bool init = false;
  if (!init) {
    const cudaError_t ea = allow_smem(k_radial_T<T, C>);
    if (ea != cudaSuccess) return ea;
    init = true;
  }
  const Dims& d = p.d;
  const int W = p.tp.WT > 0 ? p.tp.WT : radial_W<T, C>(d, 2);
  const int S = d.NT * d.NP;
  const size_t smem = (size_t)(d.Nr * d.Nr + 2 * d.Nr * W) * sizeof(C);
  const long long nct = (long long)d.G * d.Nt * d.Np * ((S + W - 1) / W);
  k_radial_T<T, C><<<grid1(nct), kThreads, smem, s>>>(p, t, X, (C)scale, tau ? 1 : 0, lt, Ubar,
                                                      W);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::plane_T(const Problem& p, const Tables<C>& t, const T* lt, T* Ubar,
                                  cudaStream_t s) {
  static bool init = false;
  if (!init) {
    cudaError_t ea = allow_smem(k_plane_T<T, C>);
    if (ea == cudaSuccess) ea = allow_smem(k_plane_T_fold<T, C>);
    if (ea != cudaSuccess) return ea;
    init = true;
  }
  const Dims& d = p.d;
  const int c = p.tp.cT > 0 ? p.tp.cT : plane_c<T, C>(d, 2);
  const size_t smem =
      (size_t)(2 * d.Nt * d.Nt + d.Np * d.Np + 2 * d.Nt * d.Np * 2 * c) * sizeof(C);
  const long long nct = (long long)d.G * d.Nr * d.NT * (d.NP / 2 / c);
  if (d.Nt % 2 == 0)   // theta folding needs the mirror of every row
    k_plane_T_fold<T, C><<<grid1(nct), kThreads, smem, s>>>(p, t, lt, Ubar, c);
  else
    k_plane_T<T, C><<<grid1(nct), kThreads, smem, s>>>(p, t, lt, Ubar, c);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::angular_T(const Problem& p, const Tables<C>& t, const T* lt,
                                    const T* Ubar, const T* Us, double* gk, double* ge,
                                    const T* lam, const T* lam_in, T* lam_out, T* Kbar_out,
                                    double wl, double wu, cudaStream_t s) {
  static bool init = false;
  if (!init) {
    const cudaError_t ea = allow_smem(k_angular_T<T, C>);
    if (ea != cudaSuccess) return ea;
    init = true;
  }
  const Dims& d = p.d;
  const int nb = p.tp.nbT > 0 ? p.tp.nbT : angular_nb<T, C>(d, 2);
  const size_t smem =
      (size_t)(2 * d.NT * d.NT + d.NP * d.NP + nb * (2 * d.NT * d.NP + kAngMoments)) * sizeof(C);
  k_angular_T<T, C><<<grid1((d.nblk + nb - 1) / nb), kThreads, smem, s>>>(
      p, t, lt, Ubar, Us, gk, ge, lam, lam_in, lam_out, Kbar_out, (C)wl, (C)wu, nb);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::implicit_collision(const Problem& p, const Tables<C>& t, T* F,
                                             double dt, cudaStream_t s) {
  const int nb = kThreads / 32;
  k_implicit_collision<T, C><<<grid1((p.d.nblk + nb - 1) / nb), kThreads, 0, s>>>(p, t, F, dt,
                                                                                 nb);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::apply_inflow(const Problem& p, T* F, cudaStream_t s) {
  const Dims& d = p.d;
  const long long n = (long long)d.G * d.Nt * d.Np * d.NT * d.NP;
  const long long blocks = std::min<long long>((n + 255) / 256, 152 * 32);
  k_apply_inflow<T><<<grid1(std::max<long long>(blocks, 1)), 256, 0, s>>>(p, F);
  return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t Launch<T, C>::filter(const Problem& p, const Tables<C>& t, T* F, T* tmp,
                                 cudaStream_t s) {
  const long long blocks = std::min<long long>((p.d.total + 255) / 256, 152 * 64);
  const unsigned b = grid1(std::max<long long>(blocks, 1));
  k_filter_axis<T, C><<<b, 256, 0, s>>>(p, t.FrT, nullptr, 0, F, tmp);
  k_filter_axis<T, C><<<b, 256, 0, s>>>(p, t.FthAT, t.FthBT, 1, tmp, F);
  k_filter_axis<T, C><<<b, 256, 0, s>>>(p, t.FphT, nullptr, 2, F, tmp);
  k_filter_axis<T, C><<<b, 256, 0, s>>>(p, t.FThAT, t.FThBT, 3, tmp, F);
  k_filter_axis<T, C><<<b, 256, 0, s>>>(p, t.FPhT, nullptr, 4, F, tmp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(F, tmp, (size_t)p.d.total * sizeof(T), cudaMemcpyDeviceToDevice, s);
}

template <typename T, typename C>
cudaError_t Launch<T, C>::moments(const Problem& p, const Tables<double>& t64, const double* wr,
                                  const double* wth, const T* F, double* F0, double* F1,
                                  double* partN, double* partJ, double* N, double* JR1,
                                  double* JR2, double R1, double R2, cudaStream_t s) {
  const Dims& d = p.d;
  const int wpb = kThreads / 32;
  k_moments<T><<<grid1((d.nblk + wpb - 1) / wpb), kThreads, 0, s>>>(p, t64, wr, wth, F, F0, F1,
                                                                     partN, partJ, R1, R2);
  k_moments_reduce<<<d.G, kThreads, 0, s>>>(d, partN, partJ, N, JR1, JR2);
  return cudaGetLastError();
}

}  // namespace ts
