// Radial pass on the 5th-generation tensor cores (tcgen05), split-TF32.
//
// One CTA (4 warps) owns 128 consecutive (Theta, Phi) columns of one (g,
// theta, phi) position and all N_r radial nodes. The radial derivative of
// those 128 r-lines is one matrix product
//     D[w][i] = sum_i' u[i'][w] Dr[i][i']        (M = 128 columns, N = N_r padded
//                                                 to 16, K = N_r padded to 8)
// issued by one thread as tcgen05.mma kind::tf32 with the accumulator in
// tensor memory (TMEM lane = column w). Operands are split into TF32 high and
// low parts, x = hi + lo, and D = A_hi B_hi + A_hi B_lo + A_lo B_hi is
// accumulated in FP32 (the lo*lo term, 2^-22 relative, is dropped). The
// matrix halves are prepared on the host in the canonical no-swizzle K-major
// layout (8-row x 16-byte core matrices) and copied into shared memory by the
// bulk-copy (TMA) engine; the data tile is split and laid out by the threads.
// After the MMAs complete, every thread reads its column's N_r results from
// TMEM (tcgen05.ld) and applies the r term, the Tau rows and the RK4 stage
// update for its own r-line. Every wait is bounded: if it runs out, the kernel
// sets the grid's error flag (ts_sync_status reports TS_ERR_TIMEOUT), waits a
// bounded time for its own operations in flight, frees its TMEM and returns.
#pragma once

#include <stdint.h>

#include "ts_kernels_rb.cuh"

namespace ts {

constexpr long long kWaitIters = 1LL << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(addr), "r"(parity) : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (long long it = 0; it < kWaitIters; ++it)
    if (mbar_try(addr, parity)) return true;
  return false;
}

// Shared-memory matrix descriptor: no swizzle, K-major core matrices.
//   lbo: byte distance between core matrices adjacent along K,
//   sbo: byte distance between 8-row groups along M or N.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;                // base offset 0, swizzle none
}

// Instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      :: "r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

struct TcShape {
  int Kpad, Npad, KC, tmem_cols;
  size_t offA, offAlo, offB, offBlo, offOut, offBar, bytes;
};

__host__ __device__ inline TcShape tc_shape(int Nr) {
  TcShape s;
  s.Kpad = (Nr + 7) / 8 * 8;
  s.Npad = (Nr + 15) / 16 * 16;
  s.KC = s.Kpad / 4;
  int c = 32;
  while (c < s.Npad) c *= 2;
  s.tmem_cols = c;
  const size_t a = (size_t)128 * s.Kpad * 4, b = (size_t)s.Npad * s.Kpad * 4;
  s.offA = 0;
  s.offAlo = a;
  s.offB = 2 * a;
  s.offBlo = 2 * a + b;
  s.offOut = 2 * a + 2 * b;                                  // [Nr][128] results
  s.offBar = s.offOut + (size_t)Nr * 128 * 4;
  s.offBar = (s.offBar + 15) / 16 * 16;
  s.bytes = s.offBar + 32;                                   // 2 mbarriers + TMEM slot
  return s;
}

// Byte offset of element (row, k) in a K-major no-swizzle operand with KC
// 16-byte core columns: core (row/8, k/4) at ((row/8) KC + k/4) 128.
__device__ __forceinline__ uint32_t core_off(int row, int k, int KC) {
  return (uint32_t)((((row >> 3) * KC + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

__global__ void __launch_bounds__(128, 1)
k_radial_tc(Problem p, Tables<float> t, const float* __restrict__ BhiG,
            const float* __restrict__ BloG, const float* U, const float* Kin, float sgn,
            int tau, int mode, float* F, float* Acc, float* Uout, float* out, float dt) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nr = d.Nr, NP = d.NP, S = d.NT * d.NP;
  const TcShape sh = tc_shape(Nr);
  unsigned char* sA = smem_raw + sh.offA;
  unsigned char* sAl = smem_raw + sh.offAlo;
  unsigned char* sB = smem_raw + sh.offB;
  unsigned char* sBl = smem_raw + sh.offBlo;
  float* sOut = reinterpret_cast<float*>(smem_raw + sh.offOut);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + sh.offBar);   // [0] copy, [1] mma
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + sh.offBar + 16);
  const int tid = threadIdx.x, warp = tid >> 5;

  const int nchunk = (S + 127) / 128;
  long long q = blockIdx.x;
  const int chunk = (int)(q % nchunk);
  q /= nchunk;
  const int l = (int)(q % d.Np);
  q /= d.Np;
  const int j = (int)(q % d.Nt);
  const int g = (int)(q / d.Nt);
  const int c0 = chunk * 128;
  const int Wc = min(128, S - c0);
  const long long base = (long long)g * d.S_g + (long long)j * d.S_j + (long long)l * d.S_l + c0;

  const uint32_t bar0 = smem_u32(&bar[0]), bar1 = smem_u32(&bar[1]);
  const uint32_t bbytes = (uint32_t)(sh.Npad * sh.Kpad * 4);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {  // matrix halves: bulk copies, completion counted in bytes on bar0
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar0), "r"(2 * bbytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(sB)), "l"(BhiG), "r"(bbytes), "r"(bar0) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(sBl)), "l"(BloG), "r"(bbytes), "r"(bar0) : "memory");
  }
  if (warp == 0) {  // TMEM accumulator: tmem_cols fp32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tslot)), "r"(sh.tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // data tile -> A operand (rows = columns w, K = radial node), split hi/lo;
  // columns beyond the tile and nodes beyond N_r are zero
  for (int x = tid; x < sh.Kpad * 128; x += 128) {
    const int k = x >> 7, w = x & 127;
    float v = 0.f;
    if (k < Nr && w < Wc) v = U[base + (long long)k * d.S_i + w];
    const uint32_t hi = tf32_rna(v);
    const uint32_t lo = tf32_rna(v - __uint_as_float(hi));
    const uint32_t o = core_off(w, k, sh.KC);
    *reinterpret_cast<uint32_t*>(sA + o) = hi;
    *reinterpret_cast<uint32_t*>(sAl + o) = lo;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  bool ok = true;
  if (tid == 0) {
    ok = mbar_wait(bar0, 0);
    if (ok) {
      const uint32_t idesc = umma_idesc_tf32(128, sh.Npad);
      const uint32_t lbo = 128, sboA = (uint32_t)sh.KC * 128, sboB = sboA;
      const uint32_t aH = smem_u32(sA), aL = smem_u32(sAl), bH = smem_u32(sB), bL = smem_u32(sBl);
      for (int ks = 0; ks < sh.Kpad / 8; ++ks) {
        const uint32_t off = (uint32_t)ks * 256;  // two 16-byte core columns of K
        umma_tf32(tmem, umma_desc(aH + off, lbo, sboA), umma_desc(bH + off, lbo, sboB), idesc,
                  ks > 0);
        umma_tf32(tmem, umma_desc(aH + off, lbo, sboA), umma_desc(bL + off, lbo, sboB), idesc, 1);
        umma_tf32(tmem, umma_desc(aL + off, lbo, sboA), umma_desc(bH + off, lbo, sboB), idesc, 1);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
          :: "r"(bar1) : "memory");
    }
  }
  // every thread waits for the products (bounded)
  const bool done = __syncthreads_and(ok ? 1 : 0) && mbar_wait(bar1, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool all_done = __syncthreads_and(done ? 1 : 0);
  if (!all_done) {
    if (tid == 0 && p.err) atomicExch(p.err, 1);
    mbar_wait(bar0, 0);  // let our own copies land before the CTA exits
    if (ok) mbar_wait(bar1, 0);
  } else {
    // TMEM -> registers -> shared: this thread's column w = tid (TMEM lane)
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c = 0; c < sh.Npad; c += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(lane_base + (uint32_t)c));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (c + e < Nr) sOut[(c + e) * 128 + tid] = __uint_as_float(r[e]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(sh.tmem_cols) : "memory");
  }
  if (!all_done) return;
  // epilogue on this thread's r-line: r term, Tau rows, stage update
  const int w = tid;
  if (w >= Wc) return;
  const int k = (c0 + w) / NP;
  const float ck = sgn * t.cosT[k];
  const int b = t.cosT[k] > 0.f ? 0 : Nr - 1;
  const float kb = Kin[base + (long long)b * d.S_i + w] + ck * sOut[b * 128 + w];
  const float tb = t.tsign[b];
  for (int i = 0; i < Nr; ++i) {
    const long long gi = base + (long long)i * d.S_i + w;
    float kv = Kin[gi] + ck * sOut[i * 128 + w];
    if (tau) kv -= kb * tb * t.tsign[i];
    switch (mode) {
      case RAD_RHS:
        out[gi] = kv;
        break;
      case RAD_STAGE0:
        Acc[gi] = kv;
        Uout[gi] = F[gi] + 0.5f * dt * kv;
        break;
      case RAD_STAGE1:
        Acc[gi] = Acc[gi] + 2.f * kv;
        Uout[gi] = F[gi] + 0.5f * dt * kv;
        break;
      case RAD_STAGE2:
        Acc[gi] = Acc[gi] + 2.f * kv;
        Uout[gi] = F[gi] + dt * kv;
        break;
      default:
        F[gi] = F[gi] + dt / 6.f * (Acc[gi] + kv);
        break;
    }
  }
}

}  // namespace ts
