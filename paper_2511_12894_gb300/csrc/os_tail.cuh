// Overlap-save block epilogue shared by the single-pass and two-phase forms: the window-peak
// key packing and warp reduction, the per-thread window scan, and the tail of an output block
// (inverse block transform, then the series or the fused window peaks).
//
// A window peak is kept as a 64-bit key (float bits of |z|^2) << 32 | (2^32 - 1 - i), so that
// atomicMax orders by value and then by the smallest index.
#pragma once

#include "blockfft.cuh"

namespace rf {

// Row stride of a partition spectrum: B bins, or the Hermitian half (bins 0..B/2, padded).
__host__ __device__ constexpr int os_row(int B, bool herm) { return herm ? B / 2 + 8 : B; }

__device__ __forceinline__ unsigned long long pack_key(float v, unsigned int i) {
  return ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xffffffffu - i);
}

// Largest packed key of the warp: the largest high word (value bits), then the largest low
// word among the lanes holding it (the smallest index), two 32-bit warp reductions in place of
// a 64-bit shuffle tree.  Key 0 (no output) never wins against a real key, whose low word is
// at least 2^31.
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k) {
  const unsigned hi = (unsigned)(k >> 32);
  const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? (unsigned)k : 0u);
  return ((unsigned long long)mh << 32) | ml;
}


// Window peaks of this thread's CH consecutive outputs mv[0..cnt) whose first sample index is
// i0 (later ones step by one and wrap to 0 at n), merged into the packed keys kj[window].
// Warp-wide: every lane of the warp calls it (lanes without outputs pass cnt = 0).
template <int CH>
__device__ __forceinline__ void window_keys(const float (&mv)[CH], int cnt, int i0, int64_t n, int64_t W,
                                            int64_t nw, int fastwin, unsigned long long* __restrict__ kj) {
  const int lane = threadIdx.x & 31;
  // sample index and window of this thread's first output; its outputs i0 + e (wrapping to
  // 0 at n) lie in window w0 below e_b = min(W - r0, n - i0) and in the next window w1 (w0 + 1,
  // or 0 after the wrap) from e_b on: at most two windows when W >= CH, which fastwin implies
  const int w0 = i0 / (int)W;
  const int r0 = i0 - w0 * (int)W;
  const int to_wrap = (int)n - i0;
  const int e_b = min((int)W - r0, to_wrap);
  const int w1 = to_wrap <= (int)W - r0 ? 0 : w0 + 1;
  const int wA = __shfl_sync(0xffffffffu, w0, 0);
  const int wB = (wA + 1 == (int)nw) ? 0 : wA + 1;
  // per window the largest |z|^2 and its first position (strict > keeps the first of equals)
  float b0 = -1.f, b1 = -1.f;
  int e0 = 0, e1 = 0;
#pragma unroll
  for (int e = 0; e < CH; ++e) {
    const float m = mv[e];
    if (e < cnt) {
      if (e < e_b) {
        if (m > b0) {
          b0 = m;
          e0 = e;
        }
      } else if (m > b1) {
        b1 = m;
        e1 = e;
      }
    }
  }
  unsigned long long kA = 0, kB = 0;
  bool slow = !fastwin;
  auto put = [&](int w, unsigned long long k) {
    if (w == wA) kA = max(kA, k);
    else if (w == wB) kB = max(kB, k);
    else slow = true;
  };
  if (b0 >= 0.f) put(w0, pack_key(b0, (unsigned int)(i0 + e0)));
  if (b1 >= 0.f) put(w1, pack_key(b1, (unsigned int)(i0 + e1 >= (int)n ? i0 + e1 - (int)n : i0 + e1)));
  const bool any_slow = __any_sync(0xffffffffu, slow);
  if (any_slow) {
    // per output, stepping the index and window by one (wrapping at n)
    int i = i0, w = w0, r = r0;
#pragma unroll
    for (int e = 0; e < CH; ++e) {
      if (e < cnt) atomicMax(kj + w, pack_key(mv[e], (unsigned int)i));
      ++i;
      ++r;
      if (i == (int)n) {
        i = 0;
        w = 0;
        r = 0;
      } else if (r == (int)W) {
        ++w;
        r = 0;
      }
    }
  } else {
    kA = warp_max_key(kA);
    kB = warp_max_key(kB);
    if (lane == 0) {
      if (kA) atomicMax(kj + wA, kA);
      if (kB) atomicMax(kj + wB, kB);
    }
  }
}

// Tail of output block s of one neighbour: v holds the partition sums of this thread's 16 bins
// (bins tid + t B/16); inverse B-point transform, then the outputs at block positions LP .. B - 1
// (pre-relabel indices s H + t - LP, relabelled by the first lag m0) go to the series row zrow
// or, as window peaks, into the keys row kj.  Every thread of the block calls it.
template <int B, int Q, bool WINMAX>
__device__ __forceinline__ void os_block_tail(float2 (&v)[16], int s, int64_t m0, int64_t n,
                                              float2* __restrict__ zrow, unsigned long long* __restrict__ kj,
                                              int64_t W, int64_t nw, int fastwin, const float2* __restrict__ tw,
                                              float2* sm) {
  using S = BlockFFTShape<B>;
  constexpr int NT = S::NT;
  constexpr int LP = B / Q;
  constexpr int H = B - LP;
  constexpr int RL = S::RL;
  constexpr int CH = H / NT;
  const int tid = threadIdx.x;
  const int64_t mask = n - 1;
  block_fft<B, +1>(v, sm, tw);
  const int64_t o0 = (int64_t)s * H;                // pre-relabel index of block position LP
  const int64_t base = (o0 + m0) & mask;            // its output index
  const int64_t lim = n - o0;                       // block positions LP + t with t < lim exist
  if (!WINMAX) {
#pragma unroll
    for (int q = 0; q < 16 / RL; ++q)
#pragma unroll
      for (int t = 0; t < RL; ++t) {
        const int idx = tid + q * NT + t * (B / RL);
        if (idx >= LP && idx - LP < lim) zrow[(base + idx - LP) & mask] = v[q * RL + t];
      }
    __syncthreads();  // the next block's FFT overwrites the shared memory read above
  } else {
    __syncthreads();  // the last FFT stage has finished reading shared memory
    float* mag = reinterpret_cast<float*>(sm);
#pragma unroll
    for (int q = 0; q < 16 / RL; ++q)
#pragma unroll
      for (int t = 0; t < RL; ++t) {
        const int idx = tid + q * NT + t * (B / RL);
        if (idx >= LP) {
          const float2 y = v[q * RL + t];
          mag[idx - LP] = y.x * y.x + y.y * y.y;
        }
      }
    __syncthreads();
    const int qbase = tid * CH;
    float mv[CH];
    if constexpr (CH % 4 == 0) {
#pragma unroll
      for (int e = 0; e < CH; e += 4)
        *reinterpret_cast<float4*>(mv + e) = *reinterpret_cast<const float4*>(mag + qbase + e);
    } else {
#pragma unroll
      for (int e = 0; e < CH; e += 2)
        *reinterpret_cast<float2*>(mv + e) = *reinterpret_cast<const float2*>(mag + qbase + e);
    }
    // outputs of this thread that exist (all but possibly in the last block)
    const int64_t avail = lim - qbase;
    const int cnt = avail <= 0 ? 0 : (avail >= CH ? CH : (int)avail);
    window_keys<CH>(mv, cnt, (int)((base + qbase) & mask), n, W, nw, fastwin, kj);
    __syncthreads();  // mag (shared memory) is reused by the next block's FFT
  }
}

}  // namespace rf
