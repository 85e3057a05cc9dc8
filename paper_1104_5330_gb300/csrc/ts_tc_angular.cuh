// Angular pass on the 5th-generation tensor cores (tcgen05), split-TF32
// operands, for 16 x 16 direction blocks (N_Theta = N_Phi = 16).
//
// One CTA (4 warps, persistent) takes 8 consecutive angular blocks per tile:
// 128 lines of each of the two contractions of the pass,
//   Theta (on the double-Fourier-sphere circle, partner column m + 8):
//     D1[(b, m)][k] = sum_{k' < 16} A[k][k'] F(b, k', m) + B[k][k'] F(b, k', m + 8 mod 16)
//     (M = 128 lines (block, column), N = 16, K = 32),
//   Phi (periodic Fourier derivative):
//     D2[(b, k)][m] = sum_{m'} D[m][m'] F(b, k, m')   (M = 128 lines (block, row), N = 16, K = 16),
// issued by one thread as tcgen05.mma kind::tf32 with the accumulators in
// tensor memory: every operand split x = hi + lo (hi = TF32(x), lo = TF32(x - hi)),
// three products hi*hi + hi*lo + lo*hi per K step (lo*lo, 2^-22 relative,
// dropped), accumulated in FP32. The blocks are staged by 16-byte cp.async into
// a padded layout (the next tile's copy runs while the current one is
// computed); each thread splits one line of each operand into the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices). The derivative
// matrices' terms are prepared on the host in the same layout and copied once
// per CTA by the bulk-copy engine. Epilogue: the Phi results go through shared
// memory to the threads holding the Theta results of the same column, which add
// a_Theta dF/dTh + a_Phi dF/dPh, the emission, absorption and isotropic
// scattering (J by a segmented warp reduction) and store K column by column.
// Every wait is bounded; on a timeout the kernel sets the grid's error flag,
// drains its own copies and products with the full bound, frees its tensor
// memory and returns.
#pragma once

#include "ts_tc.cuh"

namespace ts {

struct TcAng {
  static constexpr int N = 16, BPT = 8, LINES = 128, K1 = 32, K2 = 16;
  static constexpr int RS = 20;                 // staging row stride (floats): conflict-free rows
  static constexpr int BS = N * RS + 16;        // staging block stride: two blocks per warp apart
  static constexpr int PS = N * N + 16;         // exchange block stride
  static constexpr int KC1 = K1 / 4, KC2 = K2 / 4;
  // byte offsets in shared memory
  static constexpr int st_bytes = BPT * BS * 4;              // one staging buffer
  static constexpr int x_bytes = LINES * K1 * 4;             // one term of the Theta operand
  static constexpr int y_bytes = LINES * K2 * 4;             // one term of the Phi operand
  static constexpr int w1_bytes = N * K1 * 4, w2_bytes = N * K2 * 4;
  static constexpr int off_st = 0;
  static constexpr int off_x = off_st + 2 * st_bytes;
  static constexpr int off_y = off_x + 2 * x_bytes;          // also the exchange tile
  static constexpr int off_w = off_y + 2 * y_bytes;          // W1 hi, W1 lo, W2 hi, W2 lo
  static constexpr int w_bytes = 2 * w1_bytes + 2 * w2_bytes;
  static constexpr int off_bar = off_w + w_bytes;
  static constexpr int bytes = off_bar + 32;
  static constexpr int tmem_cols = 32;                       // D1: columns 0..15, D2: 16..31
  static_assert(2 * y_bytes >= BPT * PS * 4, "exchange tile must fit the Phi operand");
};

__global__ void __launch_bounds__(128, 2)
k_angular_tc(Problem p, Tables<float> t, const float* __restrict__ Wterms,
             const float* __restrict__ U, float* __restrict__ K, float sgn, int collision,
             long long ntiles) {
  using S = TcAng;
  constexpr int N = S::N, BPT = S::BPT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* st = reinterpret_cast<float*>(smem_raw + S::off_st);
  unsigned char* sX = smem_raw + S::off_x;
  unsigned char* sY = smem_raw + S::off_y;
  float* sP = reinterpret_cast<float*>(smem_raw + S::off_y);   // exchange, after the products
  unsigned char* sW = smem_raw + S::off_w;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + S::off_bar);   // [0] W copy, [1] MMA
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + S::off_bar + 16);
  const Dims& d = p.d;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t bar0 = smem_u32(&bar[0]), bar1 = smem_u32(&bar[1]);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {   // the derivative matrices' terms (contiguous): one bulk copy
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar0), "r"((uint32_t)S::w_bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(sW)), "l"(Wterms), "r"((uint32_t)S::w_bytes), "r"(bar0) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tslot)), "r"(S::tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // stage the BPT blocks of a tile (each 256 contiguous floats) into the padded layout
  auto stage = [&](long long tile, float* dst) {
    const long long b0 = tile * BPT;
    const int nbb = (int)min((long long)BPT, d.nblk - b0);
    for (int x = tid; x < nbb * N * (N / 4); x += 128) {
      const int c4 = x & 3, k = (x >> 2) & (N - 1), b = x >> 6;
      copy4<true, float, float>(dst + b * S::BS + k * S::RS + 4 * c4,
                                U + (b0 + b) * (N * N) + k * N + 4 * c4);
    }
  };

  long long tile = blockIdx.x;
  int cur = 0;
  if (tile < ntiles) stage(tile, st);
  cp_async_commit();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  const int b = tid >> 4, c = tid & 15;   // line (block b, column or row c) of this thread
  bool wok = true;                        // the matrix terms have landed (thread 0)
  bool failed = false;
  uint32_t phase = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    float* sb = st + cur * (BPT * S::BS);
    cp_async_wait0();
    __syncthreads();   // this tile staged; the previous tile's epilogue is done
    const long long next = tile + gridDim.x;
    if (next < ntiles) stage(next, st + (cur ^ 1) * (BPT * S::BS));
    cp_async_commit();
    const long long b0 = tile * BPT;
    const int nbb = (int)min((long long)BPT, d.nblk - b0);
    const bool act = b < nbb;
    // split: Theta operand line (b, m = c) over K = (k', partner half); Phi operand
    // line (b, k = c) over K = m'; lines of missing blocks are zero
    const float* fb = sb + b * S::BS;
    float jpart = 0.f;
#pragma unroll
    for (int kq = 0; kq < S::KC1; ++kq) {
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int kk = kq * 4 + e;
        const int col = kk < N ? c : (c + N / 2) & (N - 1);
        v[e] = act ? fb[(kk & (N - 1)) * S::RS + col] : 0.f;
        if (kk < N) jpart = fmaf(t.qdir[kk], v[e], jpart);
      }
      split_store_row<TC_TF32X3>(v, sX, core_off<4, 4>(tid, kq * 4, S::KC1), S::x_bytes);
    }
#pragma unroll
    for (int kq = 0; kq < S::KC2; ++kq) {
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (act) ld4<float>(fb + c * S::RS + 4 * kq, v);
      split_store_row<TC_TF32X3>(v, sY, core_off<4, 4>(tid, kq * 4, S::KC2), S::y_bytes);
    }
    // J of block b: the 16 threads of the block hold its column sums
#pragma unroll
    for (int o = 8; o; o >>= 1) jpart += __shfl_xor_sync(0xffffffffu, jpart, o);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    bool ok = true;
    if (tid == 0) {
      if (wok && phase == 0) wok = mbar_wait(bar0, 0, p.wait_operand);
      ok = wok;
      if (ok) {
        const uint32_t idesc = umma_idesc_tf32(128, N);
        const uint32_t x0 = smem_u32(sX), y0 = smem_u32(sY), w0 = smem_u32(sW);
        const uint32_t w1lo = w0 + S::w1_bytes, w2 = w0 + 2 * S::w1_bytes;
        const uint32_t w2lo = w2 + S::w2_bytes;
#pragma unroll
        for (int ks = 0; ks < S::K1 / 8; ++ks) {
          const uint32_t off = (uint32_t)ks * 256;   // two 16-byte core columns of K
          umma<TC_TF32X3>(tmem, umma_desc(x0 + S::x_bytes + off, 128, S::KC1 * 128),
                          umma_desc(w0 + off, 128, S::KC1 * 128), idesc, ks > 0);
          umma<TC_TF32X3>(tmem, umma_desc(x0 + off, 128, S::KC1 * 128),
                          umma_desc(w1lo + off, 128, S::KC1 * 128), idesc, 1);
          umma<TC_TF32X3>(tmem, umma_desc(x0 + off, 128, S::KC1 * 128),
                          umma_desc(w0 + off, 128, S::KC1 * 128), idesc, 1);
        }
#pragma unroll
        for (int ks = 0; ks < S::K2 / 8; ++ks) {
          const uint32_t off = (uint32_t)ks * 256;
          umma<TC_TF32X3>(tmem + 16, umma_desc(y0 + S::y_bytes + off, 128, S::KC2 * 128),
                          umma_desc(w2 + off, 128, S::KC2 * 128), idesc, ks > 0);
          umma<TC_TF32X3>(tmem + 16, umma_desc(y0 + off, 128, S::KC2 * 128),
                          umma_desc(w2lo + off, 128, S::KC2 * 128), idesc, 1);
          umma<TC_TF32X3>(tmem + 16, umma_desc(y0 + off, 128, S::KC2 * 128),
                          umma_desc(w2 + off, 128, S::KC2 * 128), idesc, 1);
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
            :: "r"(bar1) : "memory");
      }
    }
    const bool issued = __syncthreads_and(ok ? 1 : 0);
    const bool done = issued && mbar_wait(bar1, phase & 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!__syncthreads_and(done ? 1 : 0)) {
      if (tid == 0 && p.err) atomicExch(p.err, 1);
      if (issued) mbar_wait(bar1, phase & 1);   // our own products, full bound
      failed = true;
      break;
    }
    ++phase;
    // epilogue: Phi results -> exchange tile [b][k][m]; Theta results stay here
    float dph[16], dth[16];
    tmem_ld16(lane_base + 16, dph);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float w4[4] = {dph[4 * q], dph[4 * q + 1], dph[4 * q + 2], dph[4 * q + 3]};
      st4<float>(sP + b * S::PS + c * N + 4 * q, w4);
    }
    tmem_ld16(lane_base, dth);
    __syncthreads();
    if (act) {
      const long long blk = b0 + b;
      int g, i, j, l;
      decode_block(d, blk, g, i, j, l);
      const float ir = t.inv_r[i], ct = t.cot_th[j];
      const int m = c;
      const float ap = t.sinP[m] * ct;
      float src = 0.f, kks = 0.f;
      if (collision) {
        const float ks = (float)p.kaps[blk];
        src = (float)p.eta[blk] + ks * jpart;
        kks = (float)p.kap[blk] + ks;
      }
      float* out = K + blk * (N * N) + m;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float aT = sgn * -t.sinT[k] * ir;
        float v = aT * (dth[k] + ap * sP[b * S::PS + k * N + m]);
        if (collision) v += src - kks * fb[k * S::RS + m];
        out[k * N] = v;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    cur ^= 1;
  }
  cp_async_wait0();
  if (tid == 0 && phase == 0 && !failed) mbar_wait(bar0, 0);   // no tile ran: let the copy land
  if (tid == 0 && failed && !wok) mbar_wait(bar0, 0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(S::tmem_cols) : "memory");
  }
}

}  // namespace ts
