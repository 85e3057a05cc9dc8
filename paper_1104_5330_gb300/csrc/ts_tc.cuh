// Radial pass on the 5th-generation tensor cores (tcgen05), split operands.
//
// One CTA (8 warps, two threads per column) owns 128 consecutive (Theta, Phi)
// columns of one (g, theta, phi) position and all N_r radial nodes. The radial
// derivative of
// those 128 r-lines is one matrix product
//     D[w][i] = sum_i' u[i'][w] Dr[i][i']        (M = 128 columns, N = N_r padded
//                                                 to 16, K = N_r padded to the
//                                                 MMA's K step)
// issued by one thread as tcgen05.mma with the accumulator in tensor memory
// (TMEM lane = column w). Two operand forms, both accumulated in FP32:
//  * TF32x3 (kind::tf32): x = hi + lo, hi = TF32(x), lo = TF32(x - hi);
//    D = A_hi B_hi + A_hi B_lo + A_lo B_hi (lo*lo, 2^-22 relative, dropped);
//  * BF16x3 (kind::f16 with bf16 operands): x = b0 + b1 + b2, each bf16 the
//    rounding of what the previous terms leave; the six products of total
//    order <= 2 (b0c0, b0c1, b1c0, b0c2, b1c1, b2c0), smallest first.
// The matrix terms are prepared on the host in the canonical no-swizzle
// K-major layout (8-row x 16-byte core matrices) and copied into shared
// memory by the bulk-copy (TMA) engine; the data tile's lines are staged
// raw by cp.async (with the epilogue's lines requested into L2 meanwhile), then
// split and laid out by the threads. After the MMAs complete, the two threads
// of each column read its N_r results from TMEM (tcgen05.ld, alternate 8-row
// groups) and apply the r term, the Tau rows and the RK4 stage update to their
// rows of the r-line, loading each group of rows before storing any of them. Every wait is bounded: if it runs out, the kernel
// sets the grid's error flag (ts_sync_status reports TS_ERR_TIMEOUT), waits a
// bounded time for its own operations in flight, frees its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "ts_kernels_rb.cuh"

namespace ts {

constexpr long long kWaitIters = kDefaultWaitIters;

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

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity,
                                          long long iters = kWaitIters) {
  for (long long it = 0; it < iters; ++it)
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

// Instruction descriptors: D f32, A and B K-major; kind::tf32 with tf32
// operands (format 2), kind::f16 with bf16 operands (format 1).
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
  if constexpr (KIND == TC_TF32X3)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

// Operand form: element bytes, operand terms, elements per 16-byte core
// column, K of one MMA.
template <int KIND>
struct TcForm {
  static constexpr int EB = KIND == TC_TF32X3 ? 4 : 2;
  static constexpr int NTERM = KIND == TC_TF32X3 ? 2 : 3;
  static constexpr int KE = 16 / EB;
  static constexpr int KSTEP = 32 / EB;
};

struct TcShape {
  int Kpad, Npad, KC, tmem_cols;
  size_t offA, offB, offBar, offU, bytes, a_bytes, b_bytes;
};

template <int KIND>
__host__ __device__ inline TcShape tc_shape(int Nr) {
  using Fm = TcForm<KIND>;
  TcShape s;
  s.Kpad = (Nr + Fm::KSTEP - 1) / Fm::KSTEP * Fm::KSTEP;
  s.Npad = (Nr + 15) / 16 * 16;
  s.KC = s.Kpad / Fm::KE;
  int c = 32;
  while (c < s.Npad) c *= 2;
  s.tmem_cols = c;
  s.a_bytes = (size_t)128 * s.Kpad * Fm::EB;
  s.b_bytes = (size_t)s.Npad * s.Kpad * Fm::EB;
  s.offA = 0;                                                 // NTERM data terms
  s.offB = Fm::NTERM * s.a_bytes;                             // NTERM matrix terms
  s.offBar = s.offB + Fm::NTERM * s.b_bytes;
  s.offBar = (s.offBar + 15) / 16 * 16;
  s.offU = s.offBar + 32;                                     // 2 mbarriers + TMEM slot
  s.bytes = s.offU + (size_t)Nr * 128 * sizeof(float);        // the tile's lines, raw
  return s;
}

// Byte offset of element (row, k) in a K-major no-swizzle operand with KC
// 16-byte core columns of KE elements: core (row/8, k/KE) at ((row/8) KC + k/KE) 128.
template <int KE, int EB>
__device__ __forceinline__ uint32_t core_off(int row, int k, int KC) {
  return (uint32_t)((((row >> 3) * KC + k / KE) << 7) + ((row & 7) << 4) + (k % KE) * EB);
}

// Split one core row (KE consecutive K elements of one operand row, 16 bytes
// per term) into the operand terms and store each term with one 16-byte store
// at byte offset o of its tile (term stride a_bytes): a load phase of 8 lanes
// writes one whole 128-byte core matrix.
template <int KIND>
__device__ __forceinline__ void split_store_row(const float (&v)[TcForm<KIND>::KE],
                                                unsigned char* sA, uint32_t o, size_t stride) {
  if constexpr (KIND == TC_TF32X3) {
    uint4 hi, lo;
    uint32_t* h = reinterpret_cast<uint32_t*>(&hi);
    uint32_t* w = reinterpret_cast<uint32_t*>(&lo);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = tf32_rna(v[e]);
      w[e] = tf32_rna(v[e] - __uint_as_float(h[e]));
    }
    *reinterpret_cast<uint4*>(sA + o) = hi;
    *reinterpret_cast<uint4*>(sA + stride + o) = lo;
  } else {
    uint4 t0, t1, t2;
    __nv_bfloat16* b0 = reinterpret_cast<__nv_bfloat16*>(&t0);
    __nv_bfloat16* b1 = reinterpret_cast<__nv_bfloat16*>(&t1);
    __nv_bfloat16* b2 = reinterpret_cast<__nv_bfloat16*>(&t2);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      b0[e] = __float2bfloat16_rn(v[e]);
      const float r1 = v[e] - __bfloat162float(b0[e]);
      b1[e] = __float2bfloat16_rn(r1);
      b2[e] = __float2bfloat16_rn(r1 - __bfloat162float(b1[e]));
    }
    *reinterpret_cast<uint4*>(sA + o) = t0;
    *reinterpret_cast<uint4*>(sA + stride + o) = t1;
    *reinterpret_cast<uint4*>(sA + 2 * stride + o) = t2;
  }
}

// 16 consecutive TMEM columns of this warp's 32 lanes (one per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

// 8 consecutive TMEM columns of this warp's 32 lanes (one per thread).
__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
}

// Threads per CTA: two per column of the 128-column tile (warps w and w + 4
// read the same TMEM lanes, each finishing alternate 8-row groups).
constexpr int kTcThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kTcThreads, 3)
k_radial_tc(Problem p, Tables<float> t, const void* __restrict__ Bterms, const float* U,
            const float* Kin, float sgn, int tau, int mode, float* F, float* Acc, float* Uout,
            float* out, float dt) {
  using Fm = TcForm<KIND>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Dims d = p.d;
  const int Nr = d.Nr, NP = d.NP, S = d.NT * d.NP;
  const TcShape sh = tc_shape<KIND>(Nr);
  unsigned char* sA = smem_raw + sh.offA;
  unsigned char* sB = smem_raw + sh.offB;
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
  const uint32_t bbytes = (uint32_t)(Fm::NTERM * sh.b_bytes);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {  // matrix terms (contiguous in global memory): one bulk copy on bar0
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar0), "r"(bbytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(sB)), "l"(Bterms), "r"(bbytes), "r"(bar0) : "memory");
  }
  if (warp == 0) {  // TMEM accumulator: tmem_cols fp32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tslot)), "r"(sh.tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the tile's N_r lines into shared memory as raw floats, every 16-byte copy in
  // flight at once (cp.async; columns beyond the tile are zero), and the lines
  // of K, F and Acc that the epilogue reads requested into L2 meanwhile
  float* sU = reinterpret_cast<float*>(smem_raw + sh.offU);
  for (int x = tid; x < Nr * 32; x += kTcThreads) {
    const int i = x >> 5, c4 = (x & 31) * 4;
    if (c4 < Wc) {
      copy4<true, float, float>(sU + i * 128 + c4, U + base + (long long)i * d.S_i + c4);
    } else {
      const float z[4] = {0.f, 0.f, 0.f, 0.f};
      st4<float>(sU + i * 128 + c4, z);
    }
  }
  cp_async_commit();
  {
    const int lane = tid & 31;
    const int cw = (warp & 3) * 32;   // this warp's 32 columns: one 128-byte line per row
    if (cw < Wc) {
      for (int i = lane + 32 * (warp >> 2); i < Nr; i += 64) {
        const long long gi = base + (long long)i * d.S_i + cw;
        prefetch_l2(Kin + gi);
        if (mode != RAD_RHS) prefetch_l2(F + gi);
        if (mode == RAD_STAGE1 || mode == RAD_STAGE2 || mode == RAD_STAGE3 || mode == RAD_AB2)
          prefetch_l2(Acc + gi);
      }
    }
  }
  cp_async_wait0();
  __syncthreads();
  // data tile -> A operand terms (rows = columns w, K = radial node), one core
  // row (KE nodes of one column) per thread and step; nodes beyond N_r are zero
  for (int x = tid; x < sh.KC * 128; x += kTcThreads) {
    const int kq = x >> 7, w = x & 127;
    float v[Fm::KE];
#pragma unroll
    for (int e = 0; e < Fm::KE; ++e) {
      const int kk = kq * Fm::KE + e;
      v[e] = kk < Nr ? sU[kk * 128 + w] : 0.f;
    }
    split_store_row<KIND>(v, sA, core_off<Fm::KE, Fm::EB>(w, kq * Fm::KE, sh.KC), sh.a_bytes);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  bool ok = true;
  if (tid == 0) {
    // the operand wait's bound is p.wait_operand (the default, or a shorter one
    // set with ts_set_wait_limit to exercise the timeout path)
    ok = mbar_wait(bar0, 0, p.wait_operand);
    if (ok) {
      const uint32_t idesc = KIND == TC_TF32X3 ? umma_idesc_tf32(128, sh.Npad)
                                               : umma_idesc_bf16(128, sh.Npad);
      const uint32_t lbo = 128, sbo = (uint32_t)sh.KC * 128;
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      const uint32_t as = (uint32_t)sh.a_bytes, bs = (uint32_t)sh.b_bytes;
      for (int ks = 0; ks < sh.Kpad / Fm::KSTEP; ++ks) {
        const uint32_t off = (uint32_t)ks * 256;  // two 16-byte core columns of K
        auto mma = [&](int ta, int tb, uint32_t acc) {
          umma<KIND>(tmem, umma_desc(a0 + ta * as + off, lbo, sbo),
                     umma_desc(b0 + tb * bs + off, lbo, sbo), idesc, acc);
        };
        if constexpr (KIND == TC_TF32X3) {
          mma(1, 0, ks > 0);
          mma(0, 1, 1);
          mma(0, 0, 1);
        } else {
          mma(2, 0, ks > 0);
          mma(1, 1, 1);
          mma(0, 2, 1);
          mma(1, 0, 1);
          mma(0, 1, 1);
          mma(0, 0, 1);
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
          :: "r"(bar1) : "memory");
    }
  }
  // every thread waits for the products (bounded); `issued` is CTA-wide: the
  // MMAs and their commit were issued only if thread 0's operand wait succeeded
  const bool issued = __syncthreads_and(ok ? 1 : 0);
  const bool done = issued && mbar_wait(bar1, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool all_done = __syncthreads_and(done ? 1 : 0);
  if (!all_done) {
    if (tid == 0 && p.err) atomicExch(p.err, 1);
    // let our own bulk copy and MMAs finish before the CTA exits (full bound)
    mbar_wait(bar0, 0);
    if (issued) mbar_wait(bar1, 0);
  } else {
    // epilogue on this thread's r-line (column w = TMEM lane; the two threads of
    // a column take alternate 8-row groups): r term, Tau rows, stage update,
    // reading the products from TMEM 8 rows at a time (the loads of a warp are
    // issued by all its lanes); the loads of each group are all issued before
    // any of its stores
    const int w = tid & 127, half = tid >> 7;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const bool act = w < Wc;
    const int k = act ? (c0 + w) / NP : 0;
    const float ck = sgn * t.cosT[k];
    const int b = t.cosT[k] > 0.f ? 0 : Nr - 1;
    float dv[8];
    tmem_ld8(lane_base + (uint32_t)((Nr - 1) / 8 * 8), dv);   // group holding row N
    const float dN = dv[(Nr - 1) % 8];
    tmem_ld8(lane_base, dv);                                  // group holding row 0
    const float db = b == 0 ? dv[0] : dN;
    const long long Si = d.S_i;
    const float* Kc = Kin + base + w;   // this column's lines
    const float* Fc = F + base + w;
    const float* Ac = Acc + base + w;
    const float kb = act ? Kc[(long long)b * Si] + ck * db : 0.f;
    const float tb = t.tsign[b];
    // every update mode as dst = f + cv (cw v + ca ac), Acc = aa ac + ab v
    const bool rhs = mode == RAD_RHS;
    const bool rA = mode == RAD_STAGE1 || mode == RAD_STAGE2 || mode == RAD_STAGE3 ||
                    mode == RAD_AB2;
    const bool wA = !rhs && mode != RAD_STAGE3;
    float cv = dt, cw = 1.f, ca = 0.f, aa = 0.f, ab = 1.f;
    if (mode == RAD_STAGE0 || mode == RAD_STAGE1) cv = 0.5f * dt;
    if (mode == RAD_STAGE1 || mode == RAD_STAGE2) { aa = 1.f; ab = 2.f; }
    if (mode == RAD_STAGE3) { cv = dt / 6.f; ca = 1.f; }
    if (mode == RAD_AB2) { cw = 1.5f; ca = -0.5f; }
    // RK4 stages 0-2 write the next stage input; stage 3 and AB2 update F in
    // place (the A tile was staged before the MMAs)
    float* dst = (rhs ? out : (mode >= RAD_STAGE3 ? F : Uout)) + base + w;
    float* Aw = Acc + base + w;
    for (int c = 8 * half; c < Nr; c += 16) {
      tmem_ld8(lane_base + (uint32_t)c, dv);
      if (!act) continue;
      const long long r0 = (long long)c * Si;
      float kv[8], f[8], ac[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        f[e] = ac[e] = kv[e] = 0.f;
        if (c + e < Nr) {
          const long long o = r0 + e * Si;
          kv[e] = Kc[o];
          if (!rhs) f[e] = Fc[o];
          if (rA) ac[e] = Ac[o];
        }
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = c + e;
        if (i >= Nr) break;
        const long long o = r0 + e * Si;
        float v = kv[e] + ck * dv[e];
        if (tau) v -= kb * tb * t.tsign[i];
        if (rhs) {
          dst[o] = v;
          continue;
        }
        dst[o] = f[e] + cv * (cw * v + ca * ac[e]);
        if (wA) Aw[o] = aa * ac[e] + ab * v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(sh.tmem_cols) : "memory");
  }
}

}  // namespace ts
