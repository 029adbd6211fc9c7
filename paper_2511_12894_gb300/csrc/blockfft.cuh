// Block FFT of B complex64 points held by one thread block: B/16 threads, 16
// points per thread, Stockham radix-16 stages through shared memory plus one
// final radix-2/4/8 stage when log2(B) is not a multiple of 4.
//
// Stage with radix R and Ns = product of the earlier radices maps butterfly b
// (k = b mod Ns) as  a[t] = in[b + t B/R] * w^(t k),  w = exp(sign 2 pi i / (Ns R)),
// a = DFT_R(a),  out[(b - k) R + k + t Ns] = a[t]  (natural order after the last stage).
//
// Input: before run(), thread `tid` holds v[t] = x[tid + t B/16] for t < 16.
// Output: after run(), thread `tid` holds, for q < 16/RL and t < RL,
//   v[q RL + t] = X[b + t B/RL],  b = tid + q NT   (RL = radix of the last stage).
// Shared memory: B + B/16 float2 (index p is stored at p + p/16, which makes the
// stride-16 writes of the first stage bank-conflict free).
//
// Twiddles come from per-stage tables laid out in thread order: the stage with
// radix R and Ns has a table of R*Ns entries, entry t*Ns + k = exp(-2 pi i t k / (R Ns)),
// so the loads of a warp are contiguous.  A stage reads the rows t = 1, 2, 4 and 8 and forms
// the other powers by complex products (a last stage of radix 2 or 4 reads only row 1).  The tables of the middle stages and of the
// last stage follow each other; a block size B needs block_table_size<B>() entries
// (built on the host by block_fft_tables).
#pragma once

#include "cplx.cuh"

namespace rf {

__device__ __forceinline__ int bf_pad(int p) { return p + (p >> 4); }

// Multiplies a[t], 0 < t < R (R = 8 or 16), by w^t (conjugated for SIGN = +1) where w^t is
// table entry t * stride: the entries t = 1 and 4 are loaded and the others formed by complex
// products (w^2 = w w, w^8 = w^4 w^4, at most three products deep: a few ulp), which keeps 13 of
// the 15 table loads of a radix-16 stage off the load/store pipe, the scarcer one in the block
// transforms (loading all 15 made the 2^23-sample step 12% slower, loading 4 was 2% slower).
template <int R, int SIGN>
__device__ __forceinline__ void apply_stage_twiddles(float2* a, const float2* __restrict__ tw, int stride) {
  static_assert(R == 8 || R == 16, "radix");
  float2 w[R];
  w[1] = __ldg(tw + stride);
  w[4] = __ldg(tw + 4 * stride);
  w[2] = cmul(w[1], w[1]);
  w[3] = cmul(w[2], w[1]);
  w[5] = cmul(w[4], w[1]);
  w[6] = cmul(w[4], w[2]);
  w[7] = cmul(w[4], w[3]);
  if constexpr (R == 16) {
    w[8] = cmul(w[4], w[4]);
#pragma unroll
    for (int t = 9; t < 16; ++t) w[t] = cmul(w[8], w[t - 8]);
  }
#pragma unroll
  for (int t = 1; t < R; ++t) a[t] = tw_apply<SIGN>(a[t], w[t]);
}

template <int B>
struct BlockFFTShape {
  static constexpr int LOGB = (B == 256) ? 8 : (B == 512) ? 9 : (B == 1024) ? 10 : (B == 2048) ? 11
                            : (B == 4096) ? 12 : (B == 8192) ? 13 : (B == 16384) ? 14 : -1;
  static_assert(LOGB > 0, "block size");
  static constexpr int NT = B / 16;
  static constexpr int N16 = LOGB / 4;                 // radix-16 stages
  static constexpr int REM = LOGB % 4;
  static constexpr int RL = REM ? (1 << REM) : 16;     // radix of the last stage
  static constexpr int SMEM = B + B / 16;              // float2 entries
};

// Radix-16 stages between the first and the last stage.
template <int B>
__host__ __device__ constexpr int block_mid_stages() {
  return (BlockFFTShape<B>::REM ? BlockFFTShape<B>::N16 : BlockFFTShape<B>::N16 - 1) - 1;
}

// Entries of the stage twiddle tables of block size B: 16 Ns per middle stage, then B for
// the last stage.
template <int B>
__host__ __device__ constexpr int block_table_size() {
  int s = 0, ns = 16;
  for (int st = 0; st < block_mid_stages<B>(); ++st) {
    s += 16 * ns;
    ns *= 16;
  }
  return s + B;
}

// tw: the stage tables of B.  SIGN: -1 forward, +1 inverse (unnormalised).  tid: the
// thread's index within the transform (0 .. B/16 - 1); several transforms can share a thread
// block, each with its own shared-memory region, as long as every thread of the block calls
// block_fft (it synchronises the whole block).
// Every access of a stage is base + t * stride in the padded index (the strides are
// multiples of 16, so pad(base + t stride) = pad(base) + t (stride + stride / 16)), which
// lets the compiler use one base register and immediate offsets.
template <int B, int SIGN>
__device__ __forceinline__ void block_fft(float2 (&v)[16], float2* sm, const float2* __restrict__ tw, int tid) {
  using S = BlockFFTShape<B>;
  constexpr int NT = S::NT;
  // first stage: Ns = 1, no twiddles, out[b*16 + t] at padded index 17 b + t
  dft<16, SIGN>(v);
  {
    float2* o = sm + 17 * tid;
#pragma unroll
    for (int t = 0; t < 16; ++t) o[t] = v[t];
  }
  __syncthreads();
  int Ns = 16;
  // middle radix-16 stages (all but the last stage)
  constexpr int MID = block_mid_stages<B>();
  constexpr int RSTR = B / 16 + B / 256;  // padded stride of the stage reads
#pragma unroll
  for (int st = 0; st < MID; ++st) {
    {
      const float2* in = sm + bf_pad(tid);
#pragma unroll
      for (int t = 0; t < 16; ++t) v[t] = in[t * RSTR];
    }
    __syncthreads();
    const int k = tid & (Ns - 1);
    apply_stage_twiddles<16, SIGN>(v, tw + k, Ns);
    dft<16, SIGN>(v);
    {
      float2* o = sm + bf_pad((tid - k) * 16 + k);
      const int wstr = Ns + Ns / 16;
#pragma unroll
      for (int t = 0; t < 16; ++t) o[t * wstr] = v[t];
    }
    __syncthreads();
    tw += 16 * Ns;
    Ns *= 16;
  }
  // last stage: radix RL, Ns = B / RL, every butterfly index b < Ns so k = b
  constexpr int RL = S::RL;
  constexpr int LSTR = B / RL + B / (16 * RL);
  // for RL <= 4, w^1 of butterfly b = tid + q NT is that of tid times exp(-2 pi i q / 16)
  // (NT / B = 1/16): one table load for the thread, exact-constant rotations for the others
  [[maybe_unused]] const float2 w1t = RL <= 4 ? __ldg(tw + (B / RL) + tid) : make_float2(1.f, 0.f);
  static_for<0, 16 / RL>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int b = tid + q * NT;
    float2 a[RL];
    const float2* in = sm + bf_pad(b);
#pragma unroll
    for (int t = 0; t < RL; ++t) a[t] = in[t * LSTR];
    if constexpr (RL <= 4) {
      // w^t for t < RL from w^1 (the table's t = 1 row): the square (and cube) cost a complex
      // product each (about 1 ulp more error)
      const float2 w1 = rot16<q, -1>(w1t);
      a[1] = tw_apply<SIGN>(a[1], w1);
      if constexpr (RL == 4) {
        const float2 w2 = cmul(w1, w1);
        a[2] = tw_apply<SIGN>(a[2], w2);
        a[3] = tw_apply<SIGN>(a[3], cmul(w2, w1));
      }
    } else {
      apply_stage_twiddles<RL, SIGN>(a, tw + b, B / RL);
    }
    dft<RL, SIGN>(a);
#pragma unroll
    for (int t = 0; t < RL; ++t) v[q * RL + t] = a[t];
  });
}

// One transform per thread block (tid = threadIdx.x).
template <int B, int SIGN>
__device__ __forceinline__ void block_fft(float2 (&v)[16], float2* sm, const float2* __restrict__ tw) {
  block_fft<B, SIGN>(v, sm, tw, (int)threadIdx.x);
}

}  // namespace rf
