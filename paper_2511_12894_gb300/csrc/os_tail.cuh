// Overlap-save block epilogue shared by the single-pass and two-phase forms: the window-peak
// key packing and warp reduction, the per-thread window scan, and the tail of an output block
// (inverse block transform, then the series or the fused window peaks), on one CTA or, for
// 32768-point blocks, on a CTA pair.
//
// A window peak is kept as a 64-bit key (float bits of |z|^2) << 32 | (2^32 - 1 - i), so that
// atomicMax orders by value and then by the smallest index.
#pragma once

#include <cstdint>

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

// ------------------------------------------------------- 32768-point blocks on CTA pairs
// A block of B2 = 32768 points is split by the parity of its bins between the two CTAs of a
// cluster: CTA r holds Y[2k' + r], k' < BH = 16384, and transforms it with the 16384-point
// block FFT; the halves combine as
//   y[t] = E0[t] + w^t E1[t],  y[t + BH] = E0[t] - w^t E1[t],  t < BH,  w = exp(+2 pi i / B2),
// each CTA computing half of the t and reading the other CTA's half from distributed shared
// memory.  Spectra of this layout are stored parity-split: bin 2k' + r at r BH + k'.
constexpr int kBH = 16384;
constexpr int kB2 = 2 * kBH;

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of both CTAs arrives; memory written before is visible after (release/acquire).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_peer_addr(const void* p, unsigned rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ float2 ld_peer_f2(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

// Tail of output block s of one neighbour on a CTA pair: v holds this CTA's parity half of the
// block's partition sums (bins r BH + tid + t BH/16 of the parity-split row).  Both CTAs call
// it for the same blocks and so pass the same cluster barriers: transform, store the half in
// shared memory, barrier, combine (reading the peer's half), barrier (the peer is done with
// this CTA's half, so the next transform may rewrite it), then the outputs at block positions
// LP .. B2 - 1 go to the series row zrow or, as window peaks, into the keys row kj.
// Shared memory: the block FFT's, then BH floats of magnitudes.  r: this CTA's rank in the
// pair; peer: the peer CTA's sm (cluster_peer_addr(sm, r ^ 1)).
template <int Q, bool WINMAX>
__device__ __forceinline__ void os2_block_tail(float2 (&v)[16], int s, int64_t m0, int64_t n,
                                               float2* __restrict__ zrow, unsigned long long* __restrict__ kj,
                                               int64_t W, int64_t nw, int fastwin, const float2* __restrict__ tw,
                                               const float2* __restrict__ twc, float2* sm, unsigned r, uint32_t peer) {
  using S = BlockFFTShape<kBH>;
  constexpr int NT = S::NT;
  constexpr int RL = S::RL;
  constexpr int LP = kB2 / Q;  // outputs start at block position LP (<= BH)
  constexpr int H = kB2 - LP;
  static_assert(Q == 2 || Q == 4, "partition ratio");
  const int tid = threadIdx.x;
  const int64_t mask = n - 1;
  const int tb = (int)r * (kBH / 2) + tid * 8;  // this thread's first position in the scan
  float* mag_lo = reinterpret_cast<float*>(sm + S::SMEM);  // |y|^2 of t, per CTA range
  float* mag_hi = mag_lo + kBH / 2;                         // |y|^2 of t + BH
  block_fft<kBH, +1>(v, sm, tw);
  __syncthreads();  // the last stage has read shared memory
#pragma unroll
  for (int qq = 0; qq < 16 / RL; ++qq)
#pragma unroll
    for (int t = 0; t < RL; ++t) sm[tid + qq * NT + t * (kBH / RL)] = v[qq * RL + t];
  cluster_sync_all();  // both halves in shared memory
  // combine: this CTA takes t = r BH/2 + e NT + tid, e < 8 (consecutive lanes, consecutive t)
  const int64_t o0 = (int64_t)s * H;  // pre-relabel index of block position LP
  const int64_t lim = n - o0;         // positions LP + u with u < lim exist
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int t = (int)r * (kBH / 2) + e * NT + tid;
    const float2 eo = sm[t];
    const float2 ep = ld_peer_f2(peer + (uint32_t)t * 8u);
    const float2 e0 = r ? ep : eo;
    const float2 e1 = r ? eo : ep;
    const float2 x = cmulc(e1, __ldg(twc + t));  // w^t E1, twc = exp(-2 pi i t / B2)
    const float2 ylo = cadd(e0, x), yhi = csub(e0, x);
    if (!WINMAX) {
      if (t >= LP && t - LP < lim) zrow[(o0 + m0 + t - LP) & mask] = ylo;
      if (t + kBH - LP < lim) zrow[(o0 + m0 + t + kBH - LP) & mask] = yhi;
    } else {
      mag_lo[e * NT + tid] = ylo.x * ylo.x + ylo.y * ylo.y;
      mag_hi[e * NT + tid] = yhi.x * yhi.x + yhi.y * yhi.y;
    }
  }
  cluster_sync_all();  // the peer has read this CTA's half; the magnitudes are in place
  if (WINMAX) {
    // runs of 8 consecutive positions per thread: t = tb + e (kept when tb >= LP; LP and tb
    // are multiples of 8) and t = tb + BH + e (always kept since LP <= BH)
    float ml[8], mh[8];
    *reinterpret_cast<float4*>(ml) = *reinterpret_cast<const float4*>(mag_lo + tid * 8);
    *reinterpret_cast<float4*>(ml + 4) = *reinterpret_cast<const float4*>(mag_lo + tid * 8 + 4);
    *reinterpret_cast<float4*>(mh) = *reinterpret_cast<const float4*>(mag_hi + tid * 8);
    *reinterpret_cast<float4*>(mh + 4) = *reinterpret_cast<const float4*>(mag_hi + tid * 8 + 4);
    auto count = [&](int64_t u0) { return u0 >= lim ? 0 : (lim - u0 >= 8 ? 8 : (int)(lim - u0)); };
    const int cl = tb >= LP ? count(tb - LP) : 0;
    const int ch = count(tb + kBH - LP);
    window_keys<8>(ml, cl, (int)((o0 + m0 + tb - LP) & mask), n, W, nw, fastwin, kj);
    window_keys<8>(mh, ch, (int)((o0 + m0 + tb + kBH - LP) & mask), n, W, nw, fastwin, kj);
  }
}

// Shared memory of a CTA of the pair layout: the block FFT's and the magnitudes.
constexpr size_t os2_tail_smem() { return sizeof(float2) * BlockFFTShape<kBH>::SMEM + sizeof(float) * kBH; }

// ------------------------------------------------------- 32768-point blocks on one CTA (Q = 2)
// With the block's spectrum split by bin parity (Y[2k' + r] at r BH + k'), the inverse
// transforms E_r of the halves give y[t + BH] = E_0[t] - w^t E_1[t], w = exp(+2 pi i / B2),
// t < BH: at Q = 2 exactly the kept outputs (block positions LP = BH .. B2 - 1).  One CTA runs the
// two 16384-point transforms in turn: E_0 is parked in natural order in a scratch row of its own
// (global memory that stays in L2: one row per resident CTA), E_1 is staged in shared memory,
// and no cluster exchange is needed.  Shared memory: os2_tail_smem().

// The two half transforms: load(h, v) fills v with half h (bins tid + t BH/16 of the half).
template <typename Load>
__device__ __forceinline__ void pair1_halves(Load&& load, float2* __restrict__ e0, const float2* __restrict__ tw,
                                             float2* sm) {
  using S = BlockFFTShape<kBH>;
  constexpr int NT = S::NT;
  constexpr int RL = S::RL;
  const int tid = threadIdx.x;
  // one loop body, so that the code holds one transform
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    float2 v[16];
    load(h, v);
    block_fft<kBH, +1>(v, sm, tw);
    __syncthreads();  // the last stage has read shared memory
#pragma unroll
    for (int q = 0; q < 16 / RL; ++q)
#pragma unroll
      for (int t = 0; t < RL; ++t) {
        const int idx = tid + q * NT + t * (kBH / RL);
        if (h == 0)
          __stcg(e0 + idx, v[q * RL + t]);
        else
          sm[idx] = v[q * RL + t];
      }
  }
  __syncthreads();  // E_1 staged; E_0 of every thread written to the scratch row
}

// The kept outputs of block s (pre-relabel index s BH of block position BH), relabelled by the
// first lag m0, to the series row zrow or, as window peaks, into the keys row kj.  Every thread of
// the CTA calls it; it ends with a barrier (shared memory and the scratch row are free again).
template <bool WINMAX>
__device__ __forceinline__ void pair1_tail(const float2* __restrict__ e0, const float2* __restrict__ twc, int s,
                                           int64_t m0, int64_t n, float2* __restrict__ zrow,
                                           unsigned long long* __restrict__ kj, int64_t W, int64_t nw, int fastwin,
                                           float2* sm) {
  using S = BlockFFTShape<kBH>;
  constexpr int NT = S::NT;
  constexpr int CH = kBH / NT;  // kept outputs per thread in the window scan
  const int tid = threadIdx.x;
  const int64_t mask = n - 1;
  float* mag = reinterpret_cast<float*>(sm + S::SMEM);
  const int64_t o0 = (int64_t)s * kBH;
  const int64_t base = (o0 + m0) & mask;
  const int64_t lim = n - o0;  // kept positions BH + t with t < lim exist
  // y[t + BH] at t = tid + j NT (consecutive lanes, consecutive t).  The table entry of t is
  // formed as twc[tid] twc[NT j] (about 1 ulp more): one entry per thread and one per j that the
  // whole block shares, instead of 128 KB of table per block.
  const float2 wt = __ldg(twc + tid);
#pragma unroll 4
  for (int j = 0; j < 16; ++j) {
    const int idx = tid + j * NT;
    const float2 w = j == 0 ? wt : cmul(wt, __ldg(twc + j * NT));
    const float2 yh = csub(__ldcg(e0 + idx), cmulc(sm[idx], w));
    if (!WINMAX) {
      if (idx < lim) zrow[(base + idx) & mask] = yh;
    } else {
      mag[idx] = yh.x * yh.x + yh.y * yh.y;
    }
  }
  if (WINMAX) {
    __syncthreads();
    float mv[CH];
#pragma unroll
    for (int e = 0; e < CH; e += 4)
      *reinterpret_cast<float4*>(mv + e) = *reinterpret_cast<const float4*>(mag + tid * CH + e);
    const int64_t avail = lim - (int64_t)tid * CH;
    const int cnt = avail <= 0 ? 0 : (avail >= CH ? CH : (int)avail);
    window_keys<CH>(mv, cnt, (int)((base + (int64_t)tid * CH) & mask), n, W, nw, fastwin, kj);
  }
  __syncthreads();
}

// a warp's scan in pair1_tail covers 32 x 16 consecutive positions: at most two windows when W >= 512
constexpr int pair1_warp_span() { return 32 * 16; }

}  // namespace rf
