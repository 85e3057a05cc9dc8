// Radial pass of the hybrid grid (Sect. 5.3): first-order one-sided differences
// in r on uniform nodes, upstream of each direction, in place of the Chebyshev
// derivative; the angular passes are the spectral ones.
//
// One thread per segment of kSeg rows of an r-line (a column (k, m) of the
// angular blocks at fixed (g, theta_j, phi_l)): consecutive threads take
// consecutive columns, so every row access of a warp is one coalesced segment.
// The thread walks its rows in the direction of propagation (upwards when
// cos(Theta_k) > 0, the inflow being at i = 0; downwards otherwise), starting from
// the row just upstream of its segment and keeping the upstream value in a
// register:
//   K_i += sgn cos(Theta_k) (U_i - U_upstream) / dr   (forward: (U_upstream - U_i)/dr),
// the inflow node (no upstream point) gets no radial term, and with held inflow
// data its rate is zero. Then the stage update of the selected mode, as in the
// spectral radial pass. When the pass writes the array it differentiates (RK4
// stages 1 and 2 write the next stage input over the current one; AB2 updates F
// while U is F), a thread takes a whole line (one segment): every row is then
// read before it is written, and no thread reads a row that another one writes.
#include "ts_internal.h"

namespace ts {

namespace {

template <typename T, typename C>
__device__ __forceinline__ void fd_store(int mode, long long gi, C kv, T* F, T* Acc, T* Uout,
                                         T* out, C dt) {
  switch (mode) {
    case RAD_RHS:
      out[gi] = (T)kv;
      break;
    case RAD_STAGE0:
      Acc[gi] = (T)kv;
      Uout[gi] = (T)((C)F[gi] + (C)0.5 * dt * kv);
      break;
    case RAD_STAGE1:
      Acc[gi] = (T)((C)Acc[gi] + (C)2 * kv);
      Uout[gi] = (T)((C)F[gi] + (C)0.5 * dt * kv);
      break;
    case RAD_STAGE2:
      Acc[gi] = (T)((C)Acc[gi] + (C)2 * kv);
      Uout[gi] = (T)((C)F[gi] + dt * kv);
      break;
    case RAD_STAGE3:
      F[gi] = (T)((C)F[gi] + dt / (C)6 * ((C)Acc[gi] + kv));
      break;
    case RAD_AB2:
      F[gi] = (T)((C)F[gi] + dt * ((C)1.5 * kv - (C)0.5 * (C)Acc[gi]));
      Acc[gi] = (T)kv;
      break;
    default:  // RAD_AB2_START
      F[gi] = (T)((C)F[gi] + dt * kv);
      Acc[gi] = (T)kv;
      break;
  }
}

constexpr int kSeg = 16;   // rows per thread when the pass does not overwrite U

template <typename T, typename C>
__global__ void __launch_bounds__(256)
k_radial_fd(Problem p, const C* __restrict__ cosT, const T* U, const T* Kin, C sgn, C inv_dr,
            int hold, int mode, T* F, T* Acc, T* Uout, T* out, C dt, int seg_rows) {
  const Dims d = p.d;
  const long long S = (long long)d.NT * d.NP;
  const long long nlines = d.total / d.Nr;
  const int nseg = (d.Nr + seg_rows - 1) / seg_rows, N = d.Nr - 1;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nlines * nseg;
       t += (long long)gridDim.x * blockDim.x) {
    const long long line = t % nlines;
    const int seg = (int)(t / nlines);
    const long long col = line % S, blk = line / S;   // blk = (g, j, l)
    const long long g = blk / ((long long)d.Nt * d.Np), jl = blk % ((long long)d.Nt * d.Np);
    const long long base = g * d.S_g + jl * d.S_l + col;
    const int k = (int)(col / d.NP);
    const C a = cosT[k];
    const bool up = a > (C)0;   // inflow at r = R1, walk outwards
    const C ca = sgn * a * inv_dr;
    // steps s0 .. s1-1 of the walk; step s is row i = s (up) or N - s (down)
    const int s0 = seg * seg_rows, s1 = min(s0 + seg_rows, N + 1);
    C prev = 0;
    if (s0 > 0) prev = (C)U[base + (long long)(up ? s0 - 1 : N - s0 + 1) * d.S_i];
#pragma unroll 4
    for (int s = s0; s < s1; ++s) {
      const int i = up ? s : N - s;
      const long long gi = base + (long long)i * d.S_i;
      const C u = (C)U[gi];
      C kv = (C)Kin[gi];
      if (s > 0) kv += up ? ca * (u - prev) : ca * (prev - u);
      else if (hold) kv = 0;
      prev = u;
      fd_store<T, C>(mode, gi, kv, F, Acc, Uout, out, dt);
    }
  }
}

}  // namespace

template <typename T, typename C>
cudaError_t launch_radial_fd(const Problem& p, const Tables<C>& t, const T* U, const T* K, C sgn,
                             bool hold, int mode, T* F, T* Acc, T* Uout, T* out, double dt,
                             double dr, cudaStream_t s) {
  const long long nlines = p.d.total / p.d.Nr;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const void* written = mode == RAD_RHS ? (const void*)out
                        : (mode == RAD_STAGE3 || mode >= RAD_AB2) ? (const void*)F
                                                                  : (const void*)Uout;
  const int seg_rows = written == (const void*)U ? p.d.Nr : kSeg;   // in place: whole lines
  const long long want = (nlines * ((p.d.Nr + seg_rows - 1) / seg_rows) + 255) / 256;
  const int ctas = (int)std::min<long long>(want, (long long)nsm * 8);
  k_radial_fd<T, C><<<ctas, 256, 0, s>>>(p, t.cosT, U, K, sgn, (C)(1.0 / dr), hold ? 1 : 0, mode,
                                         F, Acc, Uout, out, (C)dt, seg_rows);
  return cudaGetLastError();
}

template cudaError_t launch_radial_fd<double, double>(const Problem&, const Tables<double>&,
                                                      const double*, const double*, double, bool,
                                                      int, double*, double*, double*, double*,
                                                      double, double, cudaStream_t);
template cudaError_t launch_radial_fd<float, float>(const Problem&, const Tables<float>&,
                                                    const float*, const float*, float, bool, int,
                                                    float*, float*, float*, float*, double, double,
                                                    cudaStream_t);

}  // namespace ts
