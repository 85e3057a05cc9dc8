// ts_moments_noalloc: the angular moments and balances of ts_moments for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host process whose device memory is
// held by another allocator's pool (a framework's caching allocator sized to
// the card), deployments that run under a fixed device-memory budget, or
// tight loops where an allocation's implicit device synchronisation is not
// acceptable. This entry point takes the grid description by value instead of
// a ts_grid (creating a grid allocates), computes the node and quadrature
// tables it needs inside the kernel, and keeps its per-block partial sums in
// a file-scope static __device__ array. The caller passes inputs and outputs.
//
// The scratch array (kNoAllocScratch doubles, 16 MiB) is reserved on every
// GPU that loads this library and stays there until the process exits. Host
// code only ever sees a host-side stand-in under the array's name, so the
// first call on each device looks up its device address with
// cudaGetSymbolAddress (with that device current) and caches it; that first
// call should come before any stream capture. Later calls on a stream that is
// not capturing look the address up again (it is cheap), so a device reset that
// reloads the module and moves the array is picked up; during a capture the
// cached address is used. Every call shares the array and
// it keeps the last call's contents: every slot a call reads is written by the
// same call first, so nothing needs clearing, but calls whose kernels overlap
// on the GPU (different streams, or host threads) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "ts_internal.h"

namespace {

constexpr long long kNoAllocScratch = 1LL << 21;  // doubles (16 MiB)
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

struct Sizes {
  int G, Nr, Nt, Np, NT, NP;
  double R1, R2;
  long long nblk;
};

// Fejer's first rule for int_0^pi g(t) sin t dt on t_k = pi (k + 1/2)/N.
__device__ double fejer_weight(int k, int N) {
  const double t = M_PI * (k + 0.5) / N;
  double s = 0.0;
  for (int m = 1; m <= N / 2; ++m) s += cos(2.0 * m * t) / (4.0 * m * m - 1.0);
  return 2.0 / N * (1.0 - 2.0 * s);
}

// Clenshaw-Curtis weight of node i of the Nr Gauss-Lobatto nodes on [-1, 1].
__device__ double cc_weight(int i, int Nr) {
  const int N = Nr - 1;
  double s = 1.0;
  for (int k = 1; k <= N / 2; ++k) {
    const double b = (2 * k == N) ? 1.0 : 2.0;
    s -= b / (4.0 * k * k - 1.0) * cos(2.0 * k * i * M_PI / N);
  }
  return ((i == 0 || i == N) ? 1.0 : 2.0) / N * s;
}

// One warp per angular block (g, i, j, l): the direction sums and the block's
// contributions to N and to the fluxes, written to the scratch array.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_moments_noalloc(Sizes z, const T* __restrict__ F, double* F0, double* F1, double* scratch) {
  __shared__ double qdir[64], cT[64], sT[64], cP[64], sP[64];
  for (int k = threadIdx.x; k < z.NT; k += blockDim.x) {
    const double Th = M_PI * (k + 0.5) / z.NT;
    qdir[k] = fejer_weight(k, z.NT) / (2.0 * z.NP);   // Fejer x (2 pi/NP) / (4 pi)
    cT[k] = cos(Th);
    sT[k] = sin(Th);
  }
  for (int m = threadIdx.x; m < z.NP; m += blockDim.x) {
    const double Ph = 2.0 * M_PI * m / z.NP;
    cP[m] = cos(Ph);
    sP[m] = sin(Ph);
  }
  __syncthreads();
  const int S = z.NT * z.NP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long blk = blockIdx.x * (long long)(blockDim.x >> 5) + warp;
  if (blk >= z.nblk) return;
  double s0 = 0, sr = 0, st = 0, sp = 0;
  for (int x = lane; x < S; x += 32) {
    const int k = x / z.NP, m = x - k * z.NP;
    const double v = qdir[k] * (double)F[blk * S + x];
    s0 += v;
    sr = fma(v, cT[k], sr);
    st = fma(v, sT[k] * cP[m], st);
    sp = fma(v, sT[k] * sP[m], sp);
  }
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    st += __shfl_xor_sync(0xffffffffu, st, o);
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
  }
  if (lane != 0) return;
  const int l = (int)(blk % z.Np);
  long long q = blk / z.Np;
  const int j = (int)(q % z.Nt);
  q /= z.Nt;
  const int i = (int)(q % z.Nr);
  const int g = (int)(q / z.Nr);
  const double th = M_PI * (j + 0.5) / z.Nt, ph = 2.0 * M_PI * l / z.Np;
  const double sth = sin(th), cth = cos(th), sph = sin(ph), cph = cos(ph);
  if (F0) F0[blk] = s0;
  if (F1) {
    F1[blk] = sr * sth * cph + st * cth * cph - sp * sph;
    F1[z.nblk + blk] = sr * sth * sph + st * cth * sph + sp * cph;
    F1[2 * z.nblk + blk] = sr * cth - st * sth;
  }
  const double r = 0.5 * (z.R1 + z.R2) - 0.5 * (z.R2 - z.R1) * cos(M_PI * i / (z.Nr - 1));
  const double wr = cc_weight(i, z.Nr) * 0.5 * (z.R2 - z.R1) * r * r;
  const double area = fejer_weight(j, z.Nt) * (2.0 * M_PI / z.Np) * 4.0 * M_PI;
  double* partN = scratch;                      // [nblk]
  double* partJ = scratch + z.nblk;             // [G][2][Nt*Np]
  partN[blk] = wr * area * s0;
  const long long pos = (long long)j * z.Np + l, nJ = (long long)z.Nt * z.Np;
  if (i == 0) partJ[((long long)g * 2 + 0) * nJ + pos] = z.R1 * z.R1 * area * sr;
  if (i == z.Nr - 1) partJ[((long long)g * 2 + 1) * nJ + pos] = z.R2 * z.R2 * area * sr;
}

// Per group, fixed-order sums of the scratch partials.
__global__ void k_moments_noalloc_reduce(Sizes z, const double* scratch, double* N, double* JR1,
                                         double* JR2) {
  __shared__ double red[3][kThreads];
  const int g = blockIdx.x;
  const long long nN = (long long)z.Nr * z.Nt * z.Np, nJ = (long long)z.Nt * z.Np;
  const double* partN = scratch;
  const double* partJ = scratch + z.nblk;
  double a = 0, b = 0, c = 0;
  for (long long x = threadIdx.x; x < nN; x += blockDim.x) a += partN[g * nN + x];
  for (long long x = threadIdx.x; x < nJ; x += blockDim.x) {
    b += partJ[(g * 2 + 0) * nJ + x];
    c += partJ[(g * 2 + 1) * nJ + x];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < 3; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (N) N[g] = red[0][0];
    if (JR1) JR1[g] = red[1][0];
    if (JR2) JR2[g] = red[2][0];
  }
}

ts_status noalloc_fail(ts_status s, const std::string& m) {
  ts::set_last_error(m);  // text returned by ts_last_error()
  return s;
}

// Device address of the scratch array on the current device, looked up with
// that device current: on the first call on the device, and again on every
// call whose stream is not capturing (a device reset may have moved the array);
// a capturing stream uses the address cached by an earlier call.
ts_status scratch_address(cudaStream_t st, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(TS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(TS_ERR_UNSUPPORTED, "device index too large");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess)
    return noalloc_fail(TS_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(TS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<double*>(g_noalloc_ptr[dev]);
  return TS_OK;
}

}  // namespace

extern "C" {

ts_status ts_moments_noalloc(const ts_grid_desc* desc, const void* F, double* F0, double* F1,
                             double* N, double* J_R1, double* J_R2, void* stream) {
  if (!desc) return noalloc_fail(TS_ERR_ARG, "ts_moments_noalloc: desc is NULL");
  if (!F) return noalloc_fail(TS_ERR_ARG, "ts_moments_noalloc: F is NULL");
  if (!ts::aligned16(F)) return noalloc_fail(TS_ERR_ARG, "ts_moments_noalloc: F is not 16-byte aligned");
  const ts_grid_desc& d = *desc;
  if (!(d.R1 > 0.0) || !(d.R2 > d.R1) || !std::isfinite(d.R2) || d.groups < 1)
    return noalloc_fail(TS_ERR_ARG, "ts_moments_noalloc: need 0 < R1 < R2 and groups >= 1");
  if (d.Nr < 3 || d.Nr > 129 || d.Ntheta < 2 || d.Ntheta > 64 || d.Nphi < 2 || d.Nphi > 64 ||
      d.NTheta < 2 || d.NTheta > 64 || d.NPhi < 2 || d.NPhi > 64 || (d.Nphi % 2) ||
      (d.NTheta % 2) || (d.NPhi % 2))
    return noalloc_fail(TS_ERR_UNSUPPORTED, "ts_moments_noalloc: unsupported grid sizes");
  if (d.precision != TS_FP64 && d.precision != TS_FP32 && d.precision != TS_FP32_R64 &&
      d.precision != TS_TF32X3 && d.precision != TS_BF16X3)
    return noalloc_fail(TS_ERR_UNSUPPORTED, "ts_moments_noalloc: unknown precision");
  if (d.radial != TS_RADIAL_CHEBYSHEV || d.form != TS_FORM_ADVECTIVE)
    return noalloc_fail(TS_ERR_UNSUPPORTED,
                        "ts_moments_noalloc: the advective form on Chebyshev radial grids only");
  Sizes z{d.groups, d.Nr, d.Ntheta, d.Nphi, d.NTheta, d.NPhi, d.R1, d.R2,
          (long long)d.groups * d.Nr * d.Ntheta * d.Nphi};
  const long long need = z.nblk + 2LL * d.groups * d.Ntheta * d.Nphi;
  if (need > kNoAllocScratch)
    return noalloc_fail(TS_ERR_UNSUPPORTED,
                        "ts_moments_noalloc: this grid needs " + std::to_string(need) +
                            " doubles of scratch; the static maximum is " +
                            std::to_string(kNoAllocScratch) +
                            " (groups*Nr*Ntheta*Nphi + 2*groups*Ntheta*Nphi)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  ts_status s = scratch_address(st, &scratch);
  if (s != TS_OK) return s;
  const int wpb = kThreads / 32;
  const unsigned blocks = (unsigned)((z.nblk + wpb - 1) / wpb);
  if (d.precision == TS_FP64)
    k_moments_noalloc<double><<<blocks, kThreads, 0, st>>>(z, (const double*)F, F0, F1, scratch);
  else
    k_moments_noalloc<float><<<blocks, kThreads, 0, st>>>(z, (const float*)F, F0, F1, scratch);
  k_moments_noalloc_reduce<<<d.groups, kThreads, 0, st>>>(z, scratch, N, J_R1, J_R2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(TS_ERR_CUDA, std::string("ts_moments_noalloc: ") + cudaGetErrorString(e));
  return TS_OK;
}

}  // extern "C"
